"""ZNSSD forward and adjoint on the GPU against the FP64 oracle and against
central finite differences.

Workload: the 8-pair differentiation set (1024x1024, affine deformation and
noise of the affine workload, subset 31, step 8, search +-20); pairs 0 and 1
are used.  Shapes are the imposed affine field at every POI centre (close to
the optimum, where the gradient with respect to p is small) and a seeded
perturbation of it (du = dv = 0.3 px, gradient terms 3e-3) where it is O(1).
Neither comes from the CUDA path.
"""
import numpy as np
import pytest

import oracle
from workloads import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def setup():
    import torch
    out = []
    for pair in (0, 1):
        p = configs.affine1024x8(pair)
        nx, ny = oracle.grid(1024, 1024, p.subset, p.step, p.radius)
        b = p.subset // 2 + p.radius + 2
        k = np.arange(nx * ny)
        x0 = (b + (k % nx) * p.step).astype(np.float64)
        y0 = (b + (k // nx) * p.step).astype(np.float64)
        gt = np.stack(p.deformation.displacement(x0, y0), 1).astype(np.float32)
        out.append((p, torch.from_numpy(gt).to("cuda:0").contiguous()))
    return out


def _gpu_adjoint(p, shapes, f32=True):
    import torch

    import paper_1905_06228_gb300 as dic
    dev = shapes.device
    h = dic.dic_create(p.subset, p.step, p.radius)
    try:
        if f32:
            tf = torch.from_numpy(p.ref.astype(np.float32)).to(dev)
            tg = torch.from_numpy(p.defm.astype(np.float32)).to(dev)
            dic.dic_set_pair_f32(h, tf, tg)
        else:
            tf = torch.from_numpy(p.ref).to(dev)
            tg = torch.from_numpy(p.defm).to(dev)
            dic.dic_set_pair(h, tf, tg)
        n = shapes.shape[0]
        lp = torch.empty(n, dtype=torch.float32, device=dev)
        tot = torch.empty((), dtype=torch.float32, device=dev)
        dic.dic_znssd(h, shapes, lp, tot)
        dg = torch.empty((p.ref.shape[0], p.ref.shape[1]), dtype=torch.float32, device=dev)
        dp = torch.empty_like(shapes)
        dic.dic_backward(h, shapes, None, 1.0, dg, dp)
        torch.cuda.synchronize()
        return lp.cpu().numpy(), float(tot), dg.cpu().numpy(), dp.cpu().numpy()
    finally:
        dic.dic_destroy(h)


def _perturbed(shapes):
    import torch
    g = torch.Generator(device="cpu").manual_seed(5)
    d = torch.zeros_like(shapes.cpu())
    d[:, 0] = 0.3 * (2 * torch.rand(shapes.shape[0], generator=g) - 1)
    d[:, 3] = 0.3 * (2 * torch.rand(shapes.shape[0], generator=g) - 1)
    d[:, [1, 2, 4, 5]] = 3e-3 * (2 * torch.rand(shapes.shape[0], 4, generator=g) - 1)
    return (shapes + d.to(shapes.device)).contiguous()


@pytest.mark.parametrize("perturb", [False, True])
@pytest.mark.parametrize("f32", [True, False])
def test_adjoint_matches_oracle(setup, perturb, f32):
    for p, shapes in setup:
        s = _perturbed(shapes) if perturb else shapes
        lp, tot, dg, dp = _gpu_adjoint(p, s, f32=f32)
        pk = s.cpu().numpy().astype(np.float64)
        rl, rdg, rdp, rlp = oracle.znssd(p.ref, p.defm, p.subset, p.step, p.radius, pk,
                                         per_poi=True)
        # per-POI losses and their sum
        assert np.abs(lp - rlp).max() < 1e-5 + 1e-4 * np.abs(rlp).max()
        assert tot == pytest.approx(rl, rel=1e-4)
        # shape gradients, POI by POI, relative to each POI's largest component
        scale = np.maximum(np.abs(rdp).max(1, keepdims=True), 1e-6 * np.abs(rdp).max())
        assert (np.abs(dp - rdp) / scale).max() < 1e-3
        # image gradient: relative L2 and max error
        err = dg - rdg
        assert np.linalg.norm(err) / np.linalg.norm(rdg) < 1e-3
        assert np.abs(err).max() < 1e-3 * np.abs(rdg).max()


def test_adjoint_matches_central_differences_on_oracle_forward(setup):
    """Central differences (h = 1e-3) of the FP64 oracle's forward against the
    GPU adjoint, for sampled POIs / parameters and sampled pixels."""
    p, shapes = setup[0]
    s = _perturbed(shapes)
    _, _, dg, dp = _gpu_adjoint(p, s)
    pk = s.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(2)
    f64 = p.ref.astype(np.float64)
    g64 = p.defm.astype(np.float64)
    h = 1e-3
    # parameter units: px for u, v and px / M for the gradient terms (so a
    # step moves the subset corners by ~h px, as in the convergence norm)
    unit = np.array([1.0, 1.0 / (p.subset // 2), 1.0 / (p.subset // 2), 1.0,
                     1.0 / (p.subset // 2), 1.0 / (p.subset // 2)])
    for k in rng.choice(len(pk), 6, replace=False):
        fd = np.zeros(6)
        for a in range(6):
            pp, pm = pk[k].copy(), pk[k].copy()
            pp[a] += h * unit[a]
            pm[a] -= h * unit[a]
            lpp = oracle.znssd(f64, g64, p.subset, p.step, p.radius, pp[None], poi_idx=[k],
                               grad=False)
            lpm = oracle.znssd(f64, g64, p.subset, p.step, p.radius, pm[None], poi_idx=[k],
                               grad=False)
            fd[a] = (lpp - lpm) / (2 * h * unit[a])
        # relative error of the POI's gradient vector, in parameter units
        assert np.abs((dp[k] - fd) * unit).max() <= 1e-3 * np.abs(fd * unit).max()
    # pixels under one POI's subset
    nx = oracle.grid(1024, 1024, p.subset, p.step, p.radius)[0]
    k = 700
    b = p.subset // 2 + p.radius + 2
    x0, y0 = b + (k % nx) * p.step, b + (k // nx) * p.step
    for _ in range(8):
        yy = y0 + int(pk[k, 3]) + rng.integers(-10, 11)
        xx = x0 + int(pk[k, 0]) + rng.integers(-10, 11)
        gp_, gm_ = g64.copy(), g64.copy()
        gp_[yy, xx] += h
        gm_[yy, xx] -= h
        lpp = oracle.znssd(f64, gp_, p.subset, p.step, p.radius, pk, grad=False)
        lpm = oracle.znssd(f64, gm_, p.subset, p.step, p.radius, pk, grad=False)
        fd = (lpp - lpm) / (2 * h)
        assert abs(dg[yy, xx] - fd) <= 1e-3 * max(abs(fd), 1e-3 * np.abs(dg).max())


def test_adjoint_matches_central_differences_on_gpu_forward(setup):
    """The same check on the GPU's own FP32 forward (per-POI losses), with
    steps large enough for FP32: 1e-3 for p, 0.25 grey levels for pixels."""
    import torch

    import paper_1905_06228_gb300 as dic
    p, shapes = setup[0]
    s = _perturbed(shapes)
    _, _, dg, dp = _gpu_adjoint(p, s)
    dev = s.device
    h = dic.dic_create(p.subset, p.step, p.radius)
    try:
        tf = torch.from_numpy(p.ref.astype(np.float32)).to(dev)
        tg = torch.from_numpy(p.defm.astype(np.float32)).to(dev)
        dic.dic_set_pair_f32(h, tf, tg)
        n = s.shape[0]
        lp = torch.empty(n, dtype=torch.float32, device=dev)

        def losses(shp):
            dic.dic_znssd(h, shp.contiguous(), lp, None)
            torch.cuda.synchronize()
            return lp.cpu().numpy().astype(np.float64)

        rng = np.random.default_rng(4)
        ks = rng.choice(n, 8, replace=False)
        unit = np.array([1.0, 1.0 / (p.subset // 2), 1.0 / (p.subset // 2), 1.0,
                         1.0 / (p.subset // 2), 1.0 / (p.subset // 2)])
        fd = np.zeros((n, 6))
        for a in range(6):
            hh = 1e-3 * unit[a]
            sp, sm = s.clone(), s.clone()
            sp[:, a] += hh
            sm[:, a] -= hh
            fd[:, a] = (losses(sp) - losses(sm)) / (2 * hh)
        for k in ks:
            assert np.abs((dp[k] - fd[k]) * unit).max() <= 2e-3 * np.abs(fd[k] * unit).max()
        # pixel derivative of the summed loss
        base = s.contiguous()
        nx = oracle.grid(1024, 1024, p.subset, p.step, p.radius)[0]
        k = 900
        b = p.subset // 2 + p.radius + 2
        x0, y0 = b + (k % nx) * p.step, b + (k // nx) * p.step
        # pixels under this POI's subset whose gradient is significant: an
        # FP32 loss difference cannot resolve a gradient far below the maximum
        ys = slice(y0 + int(s[k, 3]) - 12, y0 + int(s[k, 3]) + 13)
        xs = slice(x0 + int(s[k, 0]) - 12, x0 + int(s[k, 0]) + 13)
        win = np.abs(dg[ys, xs])
        cand = np.argwhere(win > 0.1 * np.abs(dg).max())
        assert len(cand) >= 6
        for j in rng.choice(len(cand), 6, replace=False):
            yy, xx = ys.start + int(cand[j][0]), xs.start + int(cand[j][1])
            hp = 1.0
            tg[yy, xx] += hp
            dic.dic_set_pair_f32(h, tf, tg)
            lpp = losses(base).sum()
            tg[yy, xx] -= 2 * hp
            dic.dic_set_pair_f32(h, tf, tg)
            lpm = losses(base).sum()
            tg[yy, xx] += hp
            fd = (lpp - lpm) / (2 * hp)
            assert abs(dg[yy, xx] - fd) <= 2e-3 * abs(fd)
    finally:
        dic.dic_destroy(h)


def test_autograd_function(setup):
    """torch.autograd.Function over the C ABI: loss.backward() gives the
    adjoint's gradients."""
    import torch

    import paper_1905_06228_gb300 as dic
    p, shapes = setup[1]
    s = _perturbed(shapes)
    dev = s.device
    f = torch.from_numpy(p.ref.astype(np.float32)).to(dev)
    g = torch.from_numpy(p.defm.astype(np.float32)).to(dev).requires_grad_(True)
    sp = s.clone().requires_grad_(True)
    h = dic.dic_create(p.subset, p.step, p.radius)
    try:
        loss = 3.0 * dic.znssd_loss(g, sp, f, h)
        loss.backward()
        torch.cuda.synchronize()
    finally:
        dic.dic_destroy(h)
    lp, tot, dg, dp = _gpu_adjoint(p, s)
    assert float(loss) == pytest.approx(3.0 * tot, rel=1e-5)
    gg = g.grad.cpu().numpy()
    assert np.linalg.norm(gg - 3.0 * dg) / np.linalg.norm(3.0 * dg) < 1e-4
    assert np.abs(sp.grad.cpu().numpy() - 3.0 * dp).max() <= 1e-4 * np.abs(3.0 * dp).max()
