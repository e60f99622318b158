"""Second-order (12-parameter) IC-GN on the GPU against the FP64 oracle:
an imposed quadratic field on re-rendered speckles, the bench workload's
affine field, and several subset widths."""
import numpy as np
import pytest

import oracle
from workloads import configs
from workloads.speckle import Quadratic, Rigid, render_pair

from parity import compare_search, compare_subpixel2, run_gpu2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _quadratic(noise):
    d = Quadratic(cu=(1.6, 0.004, -0.003, 8e-4, -5e-4, 6e-4),
                  cv=(-0.9, 0.002, 0.005, -6e-4, 7e-4, 5e-4), cx=127.5, cy=127.5)
    f, g = render_pair(411, 256, 256, 3200, d, noise, pad=30.0)
    return f, g, d


@pytest.mark.parametrize("noise,solve_bits", [(0.0, 64), (1.0, 64), (1.0, 32)])
def test_quadratic_field(noise, solve_bits):
    f, g, d = _quadratic(noise)
    subset, step, r = 31, 8, 12
    gpu = run_gpu2(f, g, subset, step, r, solve_bits=solve_bits)
    ref = oracle.integer_search(f, g, subset, step, r)
    compare_search(gpu, ref)
    compare_subpixel2(gpu, f, g, subset, step, r, ref, label=f"quadratic noise {noise}")
    # the imposed field at the POIs: the paper's usual 0.05 px
    nx = gpu["nx"]
    b = subset // 2 + r + 2
    k = np.arange(gpu["n"])
    x0 = (b + (k % nx) * step).astype(float)
    y0 = (b + (k // nx) * step).astype(float)
    truth = np.stack(d.displacement2(x0, y0), 1)
    ok = gpu["status"] == 0
    assert ok.mean() > 0.95
    assert np.abs(gpu["p"][ok][:, [0, 6]] - truth[ok][:, [0, 6]]).max() < 0.05


def test_affine1024_sampled(affine1024):
    """The bench workload (subset 31, step 5, +-20) with the second-order
    shape: the integer search at every POI, the refinement on an evenly
    spaced tenth of them against the oracle."""
    p = affine1024
    gpu = run_gpu2(p.ref, p.defm, p.subset, p.step, p.radius)
    ref = oracle.integer_search(p.ref, p.defm, p.subset, p.step, p.radius)
    compare_search(gpu, ref)
    idx = np.arange(0, gpu["n"], 10)
    start = {k: ref[k][idx] for k in ("u0", "v0", "status")}
    st = compare_subpixel2(gpu, p.ref, p.defm, p.subset, p.step, p.radius, start, idx=idx,
                           label="affine1024")
    assert st["converged"] > 0.98 * len(idx)


@pytest.mark.parametrize("subset,step,radius,size", [(15, 7, 4, 96), (21, 9, 4, 110),
                                                     (41, 16, 5, 150)])
def test_subset_widths(subset, step, radius, size):
    d = Quadratic(cu=(0.8, 0.003, -0.002, 4e-4, -3e-4, 3e-4),
                  cv=(-0.6, 0.002, 0.004, -3e-4, 4e-4, 2e-4), cx=size / 2, cy=size / 2)
    f, g = render_pair(500 + subset, size, size, int(0.05 * size * size), d, 1.0, pad=20.0)
    gpu = run_gpu2(f, g, subset, step, radius)
    ref = oracle.integer_search(f, g, subset, step, radius)
    compare_search(gpu, ref)
    compare_subpixel2(gpu, f, g, subset, step, radius, ref, label=f"subset {subset}")


def test_second_order_arguments():
    import torch

    import paper_1905_06228_gb300 as dic
    f, g = configs.tiny(3, 64, 64, 160, Rigid(1.0, 0.5))
    tf, tg = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    h = dic.dic_create(15, 8, 3, 2)
    try:
        dic.dic_set_pair(h, tf, tg)
        n, _, _ = dic.dic_num_pois(h)
        t = lambda dt: torch.zeros(n, dtype=dt, device="cuda:0")
        p12 = torch.empty((n, 12), dtype=torch.float32, device="cuda:0")
        with pytest.raises(dic.DICError) as e:
            dic.dic_subpixel2(h, dic.DIC_FANR, t(torch.int32), t(torch.int32), t(torch.uint8),
                              p12, t(torch.float32), t(torch.int32), t(torch.uint8))
        assert e.value.code == dic.DIC_ERR_UNSUPPORTED
        with pytest.raises(dic.DICError) as e:
            dic.dic_subpixel(h, 0, *[t(torch.int32)] * 2, t(torch.uint8),
                             *[t(torch.float32)] * 7, t(torch.int32), t(torch.uint8))
        assert e.value.code == dic.DIC_ERR_STATE
    finally:
        dic.dic_destroy(h)
