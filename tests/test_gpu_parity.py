"""GPU path against the FP64 oracle, element by element, through the C ABI.

Integer displacements must be bit-exact; u, v within 1e-3 px, displacement
gradients within 1e-5 and ZNCC within 1e-5 (FP32 kernels against FP64).
"""
import numpy as np
import pytest

import oracle
from workloads import configs
from workloads.speckle import Affine, Rigid

from parity import compare_search, compare_subpixel, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


# ------------------------------------------------------------ small workload
@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("solve_bits", [32, 64])
def test_rigid256_full(rigid256, method, solve_bits):
    p = rigid256
    gpu = run_gpu(p.ref, p.defm, p.subset, p.step, p.radius, method=method, solve_bits=solve_bits)
    ref = oracle.integer_search(p.ref, p.defm, p.subset, p.step, p.radius)
    assert gpu["n"] == 484
    compare_search(gpu, ref)
    compare_subpixel(gpu, p.ref, p.defm, p.subset, p.step, p.radius, ref, method,
                     label=f"rigid256 m{method} fp{solve_bits}")


# ------------------------------------------------- bench workload, all POIs
@pytest.fixture(scope="module")
def affine_search(affine1024):
    p = affine1024
    return oracle.integer_search(p.ref, p.defm, p.subset, p.step, p.radius)


@pytest.mark.parametrize("method,solve_bits,form", [(0, 32, 1), (0, 64, 1), (1, 32, 1),
                                                    (1, 64, 1), (0, 64, 0)])
def test_affine1024_full(affine1024, affine_search, method, solve_bits, form):
    """The bench workload (1024x1024, subset 31, step 5, search +-20) at all
    36100 POIs: integer search bit-exact in both search forms, every POI's
    sub-pixel result against the oracle."""
    p = affine1024
    gpu = run_gpu(p.ref, p.defm, p.subset, p.step, p.radius, method=method,
                  solve_bits=solve_bits, form=form)
    assert gpu["n"] == 36100
    compare_search(gpu, affine_search)
    st = compare_subpixel(gpu, p.ref, p.defm, p.subset, p.step, p.radius, affine_search, method,
                          label=f"affine1024 m{method} fp{solve_bits} form{form}")
    assert st["compared_within_tol"] == st["n"] == 36100
    assert (np.abs(gpu["u0"]) <= p.radius).all() and (np.abs(gpu["v0"]) <= p.radius).all()
    assert np.isfinite(gpu["p"]).all()
    assert (gpu["status"] == 0).mean() > 0.99


# ------------------------------------------ bilinear interpolation (Eq. 5)
@pytest.mark.parametrize("method", [0, 1])
def test_bilinear_rigid256_full(rigid256, method):
    """Sub-pixel refinement over the bilinear interpolation of Eq. 5
    against the oracle with the same interpolation, every POI."""
    p = rigid256
    gpu = run_gpu(p.ref, p.defm, p.subset, p.step, p.radius, method=method, solve_bits=64,
                  interp=1)
    ref = oracle.integer_search(p.ref, p.defm, p.subset, p.step, p.radius)
    compare_search(gpu, ref)
    compare_subpixel(gpu, p.ref, p.defm, p.subset, p.step, p.radius, ref, method,
                     interp=oracle.BILINEAR, label=f"rigid256 bilinear m{method}")
    assert np.abs(gpu["u"] - 3.4).max() < 0.1 and np.abs(gpu["v"] + 2.7).max() < 0.1


@pytest.mark.parametrize("method", [0, 1])
def test_bilinear_affine1024_full(affine1024, affine_search, method):
    """Eq. 5 interpolation on the bench workload, all 36100 POIs."""
    p = affine1024
    gpu = run_gpu(p.ref, p.defm, p.subset, p.step, p.radius, method=method, solve_bits=64,
                  form=1, interp=1)
    compare_search(gpu, affine_search)
    compare_subpixel(gpu, p.ref, p.defm, p.subset, p.step, p.radius, affine_search, method,
                     interp=oracle.BILINEAR, label=f"affine1024 bilinear m{method}",
                     grad_outliers=0.001 if method == 1 else 0.0)
    # FA-NR over Eq. 5 follows a gradient that jumps at cell edges, so a few
    # POIs oscillate to the iteration cap (the oracle's do too: the statuses
    # agree POI by POI); IC-GN's gradient is f's and smooth
    assert (gpu["status"] == 0).mean() > (0.99 if method == 0 else 0.97)


def test_bilinear_argument_checks():
    import torch

    import paper_1905_06228_gb300 as dic
    h = dic.dic_create(21, 5, 10)
    try:
        with pytest.raises(dic.DICError) as e:
            dic.dic_set_interpolation(h, 5)
        assert e.value.code == dic.DIC_ERR_ARG
        f, g = configs.tiny(90, 96, 96, 400)
        tf, tg = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
        dic.dic_set_interpolation(h, dic.DIC_INTERP_BILINEAR)
        dic.dic_set_pairs(h, [(tf, tg, 15, 8, 4)])
        total, _ = dic.dic_batch_pois(h, 1)
        out = dic.batch_outputs(total, torch.device("cuda:0"))
        with pytest.raises(dic.DICError) as e:
            dic.dic_run_batch(h, 0, out)
        assert e.value.code == dic.DIC_ERR_UNSUPPORTED
    finally:
        dic.dic_destroy(h)


# --------------------------------------------------------------- edge cases
def test_smallest_subset_search():
    """Subset 3 (N = 9 < 32 lanes): integer search bit-exact.  The
    6-parameter fit over 9 points is degenerate (on this input only 2 of 36
    POIs converge, after ~20 iterations, at |grad u| ~ 0.8), so its sub-pixel
    result is not a parity case."""
    f, g = configs.tiny(1003, 24, 24, 17, Rigid(1.4, -0.7), noise=1.5)
    gpu = run_gpu(f, g, 3, 3, 1, subpixel=False)
    ref = oracle.integer_search(f, g, 3, 3, 1)
    assert gpu["n"] == len(ref["u0"]) == 36
    compare_search(gpu, ref)


@pytest.mark.parametrize("subset,step,radius,size", [
    (5, 2, 3, 28),      # ragged: N = 25 < 32 lanes
    (9, 4, 0, 40),      # R = 0: a single candidate
    (15, 6, 4, 80),     # column layout, two subset rows per warp
    (31, 9, 5, 110),    # column layout, one subset row per warp
    (33, 9, 4, 96),     # N = 1089 > 1024: FP32 blocks flushed to int32
    (41, 12, 6, 120),
    (51, 20, 5, 140),
    (63, 30, 3, 150),   # largest subset
])
@pytest.mark.parametrize("method", [0, 1])
def test_sizes(subset, step, radius, size, method):
    """Every POI against the oracle.  Subsets 5 and 9 are smaller than the
    speckles (radius 2.5-4 px), so most of their six-parameter fits are
    ill-posed and do not converge; their non-converged shapes are not a
    parity quantity (checked for validity instead, see compare_subpixel),
    and the bar on POIs inside the tolerance is 0.9 there, 0.99 elsewhere."""
    f, g = configs.tiny(1000 + subset, size, size, int(0.03 * size * size),
                        Rigid(1.4, -0.7), noise=1.5)
    gpu = run_gpu(f, g, subset, step, radius, method=method, solve_bits=64)
    ref = oracle.integer_search(f, g, subset, step, radius)
    assert gpu["n"] == len(ref["u0"]) > 0
    compare_search(gpu, ref)
    compare_subpixel(gpu, f, g, subset, step, radius, ref, method,
                     min_compared=0.9 if subset <= 9 else 0.99,
                     label=f"subset {subset} m{method}")


def test_unaligned_pitch_uses_plain_loads():
    f, g = configs.tiny(77, 90, 70, 190, Rigid(-2.2, 1.3), noise=1.0)
    a = run_gpu(f, g, 11, 5, 4, method=0)
    b = run_gpu(f, g, 11, 5, 4, method=0, pitch_pad=3)
    ref = oracle.integer_search(f, g, 11, 5, 4)
    compare_search(a, ref)
    compare_search(b, ref)
    np.testing.assert_array_equal(a["p"], b["p"])


def test_too_small_image_has_no_pois():
    f, g = configs.tiny(5, 30, 30, 20)
    gpu = run_gpu(f, g, 21, 5, 10)
    assert gpu["n"] == 0


def test_zero_variance_and_ties():
    # flat reference -> ZERO_VAR_REF; flat target -> ZERO_VAR_DEF
    flat = np.full((40, 40), 90, np.uint8)
    g, _ = configs.tiny(4, 40, 40, 60)
    a = run_gpu(flat, g, 5, 5, 2)
    compare_search(a, oracle.integer_search(flat, g, 5, 5, 2))
    assert (a["status"] == 1).all() and (a["iters"] == 0).all()
    b = run_gpu(g, flat, 5, 5, 2)
    compare_search(b, oracle.integer_search(g, flat, 5, 5, 2))
    assert (b["status"] == 6).all()
    # exact ties: period-3 texture, lowest linear index wins
    rng = np.random.default_rng(3)
    period = rng.integers(0, 256, (40, 3)).astype(np.uint8)
    gg = np.ascontiguousarray(np.tile(period, (1, 14)))
    ff = np.ascontiguousarray(np.roll(gg, -1, axis=1))
    c = run_gpu(ff, gg, 5, 5, 3, subpixel=False)
    compare_search(c, oracle.integer_search(ff, gg, 5, 5, 3))
    assert (c["u0"] == -2).all()


def test_planted_shift_exact():
    big, _ = configs.tiny(11, 140, 140, 700)
    for du, dv in ((7, -5), (-9, 3)):
        f = np.ascontiguousarray(big[20:120, 20:120])
        g = np.ascontiguousarray(big[20 - dv:120 - dv, 20 - du:120 - du])
        gpu = run_gpu(f, g, 15, 6, 10, method=0)
        assert (gpu["u0"] == du).all() and (gpu["v0"] == dv).all()
        assert np.abs(gpu["zncc0"] - 1).max() < 1e-6
        ok = gpu["status"] == 0
        assert np.abs(gpu["p"][ok] - [du, 0, 0, dv, 0, 0]).max() < 1e-4


def test_affine_recovery_accuracy(affine1024):
    """Imposed affine field: the GPU result is within the paper's usual
    accuracy (0.05 px) at every converged POI."""
    p = affine1024
    gpu = run_gpu(p.ref, p.defm, p.subset, p.step, p.radius, method=0, solve_bits=64)
    b = p.subset // 2 + p.radius + 2
    n = gpu["n"]
    x0 = (b + (np.arange(n) % gpu["nx"]) * p.step).astype(float)
    y0 = (b + (np.arange(n) // gpu["nx"]) * p.step).astype(float)
    gt = np.stack(p.deformation.displacement(x0, y0), 1)
    ok = gpu["status"] == 0
    e = np.abs(gpu["p"] - gt)[ok]
    assert e[:, [0, 3]].max() < 0.05 and e[:, [0, 3]].mean() < 0.01
    assert e[:, [1, 2, 4, 5]].mean() < 1e-3


def test_repeatable_bitwise(rigid256):
    p = rigid256
    a = run_gpu(p.ref, p.defm, p.subset, p.step, p.radius, method=1)
    b = run_gpu(p.ref, p.defm, p.subset, p.step, p.radius, method=1)
    for k in ("u0", "v0", "zncc0", "p", "zncc", "iters", "status"):
        np.testing.assert_array_equal(a[k], b[k])
