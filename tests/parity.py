"""Helpers shared by the GPU parity tests: run the CUDA path through the C
ABI and compare it with the FP64 oracle on the same inputs."""
from __future__ import annotations

import numpy as np

import oracle

# Tolerances of the comparison (FP32 GPU path against the FP64 oracle).
TOL_UV = 1e-3      # px, u and v
TOL_GRAD = 1e-5    # displacement gradients ux, uy, vx, vy
TOL_ZNCC = 1e-5    # Eq. 1 values
NAMES = ("u", "ux", "uy", "v", "vx", "vy")


def run_gpu(f: np.ndarray, g: np.ndarray, subset: int, step: int, radius: int,
            method: int = 0, solve_bits: int = 32, tol: float = 1e-3, max_iter: int = 50,
            device: str = "cuda:0", pitch_pad: int = 0, subpixel: bool = True,
            form: int = 0, interp: int = 0) -> dict:
    import torch

    import paper_1905_06228_gb300 as dic
    H, W = f.shape
    if pitch_pad:
        # images inside a wider, unaligned buffer: exercises the plain-load path
        buf_f = torch.zeros((H, W + pitch_pad), dtype=torch.uint8, device=device)
        buf_g = torch.zeros((H, W + pitch_pad), dtype=torch.uint8, device=device)
        buf_f[:, :W] = torch.from_numpy(f)
        buf_g[:, :W] = torch.from_numpy(g)
        tf, tg, pitch = buf_f, buf_g, W + pitch_pad
    else:
        tf = torch.from_numpy(np.ascontiguousarray(f)).to(device)
        tg = torch.from_numpy(np.ascontiguousarray(g)).to(device)
        pitch = W
    h = dic.dic_create(subset, step, radius, 1, tol, max_iter)
    try:
        if solve_bits != 32:
            dic.dic_set_solve_precision(h, solve_bits)
        if form:
            dic.dic_set_form(h, form)
        if interp:
            dic.dic_set_interpolation(h, interp)
        dic.dic_set_pair(h, tf, tg, W, H, pitch)
        n, nx, ny = dic.dic_num_pois(h)
        out = {"n": n, "nx": nx, "ny": ny}
        if n == 0:
            return out
        t = lambda dt: torch.empty(n, dtype=dt, device=device)
        u0, v0, z0, s0 = t(torch.int32), t(torch.int32), t(torch.float32), t(torch.uint8)
        dic.dic_integer_search(h, u0, v0, z0, s0)
        res = dict(u0=u0, v0=v0, zncc0=z0, status0=s0)
        if subpixel:
            o = {k: t(torch.float32) for k in ("u", "v", "ux", "uy", "vx", "vy", "zncc")}
            o["iters"] = t(torch.int32)
            o["status"] = t(torch.uint8)
            dic.dic_subpixel(h, method, u0, v0, s0, o["u"], o["v"], o["ux"], o["uy"], o["vx"],
                             o["vy"], o["zncc"], o["iters"], o["status"])
            res.update(o)
        torch.cuda.synchronize()
        out.update({k: v.cpu().numpy() for k, v in res.items()})
        if subpixel:
            out["p"] = np.stack([out[k] for k in NAMES], 1).astype(np.float64)
        return out
    finally:
        dic.dic_destroy(h)


def compare_search(gpu: dict, ref: dict, idx=None) -> None:
    sel = slice(None) if idx is None else idx
    np.testing.assert_array_equal(gpu["status0"][sel], ref["status"])
    np.testing.assert_array_equal(gpu["u0"][sel], ref["u0"])
    np.testing.assert_array_equal(gpu["v0"][sel], ref["v0"])
    assert np.abs(gpu["zncc0"][sel] - ref["zncc"]).max() < TOL_ZNCC


def oracle_iterates(f, g, subset, step, radius, start: dict, method: int, ref: dict, k,
                    idx=None, interp: int = 0) -> np.ndarray:
    """The oracle's shape after k[j] solves for POI j: its recorded trajectory
    where it ran that far, else a rerun capped at k[j] solves with a
    tolerance that never stops it.  A solve whose update was rejected (the
    subset would leave the image, or the step is not finite) counts in the
    iteration count but leaves the shape unchanged, so the trajectory has no
    entry for it: the shape is then the one before it."""
    k = np.asarray(k)
    out = np.full((len(k), 6), np.nan)
    have = k <= ref["iters"]
    rows = np.nonzero(have)[0]
    out[rows] = ref["traj"][rows, k[rows]]
    rej = rows[np.isnan(out[rows]).any(1) & (k[rows] >= 1)]
    out[rej] = ref["traj"][rej, k[rej] - 1]
    sel = None if idx is None else np.asarray(idx)
    for kk in np.unique(k[~have]):
        rows = np.nonzero(~have & (k == kk))[0]
        sub = oracle.subpixel(f, g, subset, step, radius, start["u0"][rows], start["v0"][rows],
                              start["status"][rows], method=method, tol=1e-300,
                              max_iter=int(kk), poi_idx=(sel[rows] if sel is not None else rows),
                              interp=interp)
        out[rows] = sub["p"]
    return out


def compare_subpixel(gpu: dict, f, g, subset, step, radius, start: dict, method: int,
                     tol: float = 1e-3, max_iter: int = 50, idx=None,
                     min_iter_agreement: float = 0.99, min_compared: float = 0.99,
                     interp: int = 0, label: str = "", grad_outliers: float = 0.0) -> dict:
    """Every POI's sub-pixel result against the FP64 oracle (reading P1).

    * Statuses agree exactly, POI by POI (a swap between OK and MAX_ITER, the
      FP32 stop test falling on the other side of the tolerance at the cap,
      is counted and allowed for at most 0.1 % of the POIs).
    * Iteration counts agree on at least ``min_iter_agreement`` of the POIs.
    * Shapes: the GPU's shape after its k solves against the oracle's
      iterate after k solves (the stop test can end the two runs one solve
      apart), u and v within 1e-3 px, gradients within 1e-5.  Every POI that
      converged (OK) must be inside the tolerance.  A POI that did not
      converge (MAX_ITER, or OUT_OF_BOUNDS: the last in-bounds iterate of an
      iteration that left the image) followed a non-contracting iteration
      whose FP32 and FP64 rounding differences grow with every solve, so its
      shape is not a parity quantity: it is counted ("wandering") when it
      falls outside the tolerance, and checked for validity instead -- its
      reported ZNCC must equal the oracle's Eq. 1 at the GPU's own returned
      shape.  The share of POIs compared inside the tolerance must reach
      ``min_compared``.
    * ``grad_outliers`` (reading R18b, FA-NR over the bilinear interpolation
      of Eq. 5 only): that share of the converged POIs may have gradients
      outside 1e-5 but inside 1e-4, u and v still inside 1e-3 px.  Eq. 5's
      gradient jumps at cell edges, so a sample that FP32 places on the
      other side of an edge than FP64 changes the Jacobian and moves the
      fixed point by a fraction of one sample's jump.
    * ZNCC: a converged POI reports Eq. 1 at the shape its last solve
      sampled (reading R11), compared with the oracle's Eq. 1 at its iterate
      after k - 1 solves; every other POI that ran reports Eq. 1 at its
      returned shape, compared with the oracle's Eq. 1 at that same shape.
      Both within 1e-5.
    """
    sel = np.arange(len(gpu["u"])) if idx is None else np.asarray(idx)
    ref = oracle.subpixel(f, g, subset, step, radius, start["u0"], start["v0"], start["status"],
                          method=method, tol=tol, max_iter=max_iter, poi_idx=idx,
                          trajectory=True, interp=interp)
    gp = gpu["p"][sel]
    git = gpu["iters"][sel]
    gst = gpu["status"][sel]
    rit, rst = ref["iters"], ref["status"]
    n = len(gst)
    swap = (gst != rst) & np.isin(gst, (0, 3)) & np.isin(rst, (0, 3))
    assert swap.sum() <= 0.001 * n, ("OK/MAX_ITER swaps", int(swap.sum()))
    np.testing.assert_array_equal(gst[~swap], rst[~swap], err_msg=label + " statuses")
    agree = float((git == rit).mean())
    # small samples: one differing count is always allowed
    assert (git != rit).sum() <= max(1, int((1 - min_iter_agreement) * n)), (
        label, "iteration agreement", agree)

    want = oracle_iterates(f, g, subset, step, radius, start, method, ref, git, idx, interp)
    err = np.abs(gp - want)
    # NaN (no comparable iterate) counts as outside the tolerance
    over = ~(err[:, [0, 3]].max(1) < TOL_UV) | ~(err[:, [1, 2, 4, 5]].max(1) < TOL_GRAD)
    ran = git >= 1
    conv = ran & (gst == 0)
    wander = ran & (gst != 0)
    n_grad_outliers = 0
    if grad_outliers > 0:
        soft = (conv & over & (err[:, [0, 3]].max(1) < TOL_UV) &
                (err[:, [1, 2, 4, 5]].max(1) < 10 * TOL_GRAD))
        n_grad_outliers = int(soft.sum())
        assert n_grad_outliers <= grad_outliers * conv.sum(), (label, "gradient outliers",
                                                               n_grad_outliers)
        over = over & ~soft
    bad = np.nonzero(conv & over)[0]
    assert len(bad) == 0, dict(label=label, poi=bad[:5], gpu=gp[bad[:5]], want=want[bad[:5]],
                               git=git[bad[:5]], rit=rit[bad[:5]])
    n_wander_over = int((wander & over).sum())
    compared = int(ran.sum()) - n_wander_over
    assert compared >= min_compared * ran.sum(), (label, "compared", compared, int(ran.sum()))

    # ZNCC: converged POIs at the oracle's iterate after k - 1 solves,
    # every other POI that ran at the GPU's returned shape
    zg = gpu["zncc"][sel]
    zs_conv = np.nonzero(conv)[0]
    zerr_conv = 0.0
    if len(zs_conv):
        before = oracle_iterates(f, g, subset, step, radius,
                                 {k: v[zs_conv] for k, v in start.items()
                                  if k in ("u0", "v0", "status")},
                                 method, {k: (v[zs_conv] if hasattr(v, "__len__") else v)
                                          for k, v in ref.items()},
                                 git[zs_conv] - 1, sel[zs_conv], interp)
        c = oracle.zncc_at(f, g, subset, step, radius, before,
                           poi_idx=sel[zs_conv], interp=interp)
        zerr_conv = float(np.abs(zg[zs_conv] - c).max())
        assert zerr_conv < TOL_ZNCC, (label, "zncc converged", zerr_conv)
    zs_other = np.nonzero(ran & np.isin(gst, (2, 3)))[0]
    zerr_other = 0.0
    if len(zs_other):
        c = oracle.zncc_at(f, g, subset, step, radius, gp[zs_other].astype(np.float64),
                           poi_idx=sel[zs_other], interp=interp)
        zerr_other = float(np.abs(zg[zs_other] - c).max())
        assert zerr_other < TOL_ZNCC, (label, "zncc at returned shape", zerr_other)
    st = dict(label=label, n=n, ran=int(ran.sum()), converged=int(conv.sum()),
              not_converged=int(wander.sum()), wandering_outside_tol=n_wander_over,
              compared_within_tol=compared, iter_agreement=agree, ok_maxiter_swaps=int(swap.sum()),
              gradient_outliers=n_grad_outliers,
              max_err_uv=float(err[ran][:, [0, 3]].max(initial=0)),
              max_err_grad=float(err[ran][:, [1, 2, 4, 5]].max(initial=0)),
              max_err_zncc_converged=zerr_conv, max_err_zncc_other=zerr_other)
    print("parity", st)
    return st


# ------------------------------------------------ second-order shape function
NAMES2 = ("u", "ux", "uy", "uxx", "uxy", "uyy", "v", "vx", "vy", "vxx", "vxy", "vyy")


def run_gpu2(f, g, subset, step, radius, solve_bits=64, form=1, device="cuda:0"):
    """Integer search and second-order IC-GN through the C ABI."""
    import torch

    import paper_1905_06228_gb300 as dic
    tf = torch.from_numpy(np.ascontiguousarray(f)).to(device)
    tg = torch.from_numpy(np.ascontiguousarray(g)).to(device)
    h = dic.dic_create(subset, step, radius, 2)
    try:
        dic.dic_set_solve_precision(h, solve_bits)
        dic.dic_set_form(h, form)
        dic.dic_set_pair(h, tf, tg)
        n, nx, ny = dic.dic_num_pois(h)
        t = lambda dt: torch.empty(n, dtype=dt, device=device)
        u0, v0, z0, s0 = t(torch.int32), t(torch.int32), t(torch.float32), t(torch.uint8)
        dic.dic_integer_search(h, u0, v0, z0, s0)
        p12 = torch.empty((n, 12), dtype=torch.float32, device=device)
        zn, it, st = t(torch.float32), t(torch.int32), t(torch.uint8)
        dic.dic_subpixel2(h, 0, u0, v0, s0, p12, zn, it, st)
        torch.cuda.synchronize()
        out = dict(n=n, nx=nx, ny=ny, u0=u0, v0=v0, zncc0=z0, status0=s0, p=p12, zncc=zn,
                   iters=it, status=st)
        return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}
    finally:
        dic.dic_destroy(h)


def compare_subpixel2(gpu, f, g, subset, step, radius, start, tol=1e-3, max_iter=50,
                      idx=None, min_compared=0.99, label="") -> dict:
    """Second-order IC-GN against the oracle under the rules of
    compare_subpixel (statuses exact, shapes at the GPU's iteration count,
    converged POIs all inside the tolerance, ZNCC at the sampled iterate);
    idx selects grid POIs (start holds the oracle's search at those POIs).
    Tolerances: u, v 1e-3 px; first derivatives 1e-5; second derivatives
    2e-5 / M -- the same displacement at the subset edge (M px from the
    centre, where a second-derivative term moves a point by up to M^2 times
    it) as the first-derivative tolerance."""
    sel = np.arange(len(gpu["iters"])) if idx is None else np.asarray(idx)
    ref = oracle.subpixel2(f, g, subset, step, radius, start["u0"], start["v0"],
                           start["status"], tol=tol, max_iter=max_iter, poi_idx=idx,
                           trajectory=True)
    M = subset // 2
    tol2 = 2 * TOL_GRAD / M
    gp, git, gst = gpu["p"][sel].astype(np.float64), gpu["iters"][sel], gpu["status"][sel]
    rit, rst = ref["iters"], ref["status"]
    n = len(gst)
    swap = (gst != rst) & np.isin(gst, (0, 3)) & np.isin(rst, (0, 3))
    assert swap.sum() <= 0.001 * n, (label, "OK/MAX_ITER swaps", int(swap.sum()))
    np.testing.assert_array_equal(gst[~swap], rst[~swap], err_msg=label + " statuses")
    assert (git != rit).sum() <= max(1, int(0.01 * n)), (label, "iteration agreement")

    def iterate(k):
        out = np.full((n, 12), np.nan)
        have = k <= rit
        rows = np.nonzero(have)[0]
        out[rows] = ref["traj"][rows, k[rows]]
        rej = rows[np.isnan(out[rows]).any(1) & (k[rows] >= 1)]
        out[rej] = ref["traj"][rej, k[rej] - 1]
        for kk in np.unique(k[~have]):
            rows = np.nonzero(~have & (k == kk))[0]
            sub = oracle.subpixel2(f, g, subset, step, radius, start["u0"][rows],
                                   start["v0"][rows], start["status"][rows], tol=1e-300,
                                   max_iter=int(kk), poi_idx=sel[rows])
            out[rows] = sub["p"]
        return out

    want = iterate(git)
    err = np.abs(gp - want)
    e_uv = err[:, [0, 6]].max(1)
    e_g1 = err[:, [1, 2, 7, 8]].max(1)
    e_g2 = err[:, [3, 4, 5, 9, 10, 11]].max(1)
    over = ~(e_uv < TOL_UV) | ~(e_g1 < TOL_GRAD) | ~(e_g2 < tol2)
    ran = git >= 1
    conv = ran & (gst == 0)
    bad = np.nonzero(conv & over)[0]
    assert len(bad) == 0, dict(label=label, poi=bad[:5], gpu=gp[bad[:3]], want=want[bad[:3]],
                               e=(e_uv[bad[:5]], e_g1[bad[:5]], e_g2[bad[:5]]))
    wander = ran & (gst != 0)
    n_w = int((wander & over).sum())
    assert int(ran.sum()) - n_w >= min_compared * ran.sum(), (label, "compared")
    zc = np.nonzero(conv)[0]
    zerr = 0.0
    if len(zc):
        before = iterate(np.where(conv, git - 1, 0))[zc]
        c = oracle.zncc_at2(f, g, subset, step, radius, before, poi_idx=sel[zc])
        zerr = float(np.abs(gpu["zncc"][sel][zc] - c).max())
        assert zerr < TOL_ZNCC, (label, "zncc", zerr)
    st = dict(label=label, n=n, converged=int(conv.sum()), wandering_outside_tol=n_w,
              max_err_uv=float(e_uv[ran].max(initial=0)),
              max_err_grad=float(e_g1[ran].max(initial=0)),
              max_err_grad2=float(e_g2[ran].max(initial=0)), tol_grad2=tol2,
              max_err_zncc=zerr)
    print("parity2", st)
    return st
