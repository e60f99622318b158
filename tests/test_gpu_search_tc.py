"""Tensor-core form of the integer search (tcgen05, BF16 x BF16 -> FP32)
against the FP32 form (bitwise: same exact integers) and the FP64 oracle."""
import numpy as np
import pytest

import oracle
from workloads import configs
from workloads.speckle import Affine, Rigid

from parity import compare_search, run_gpu

pytestmark = pytest.mark.gpu
TC = 1
INT_KEYS = ("u0", "v0", "zncc0", "status0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _both(f, g, s, st, r):
    a = run_gpu(f, g, s, st, r, subpixel=False, form=0)
    b = run_gpu(f, g, s, st, r, subpixel=False, form=TC)
    assert a["n"] == b["n"]
    for k in INT_KEYS:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    return b


def test_rigid256(rigid256):
    p = rigid256
    b = _both(p.ref, p.defm, p.subset, p.step, p.radius)
    compare_search(b, oracle.integer_search(p.ref, p.defm, p.subset, p.step, p.radius))


def test_no_wait_gave_up_on_a_normal_run(affine1024):
    """After a full tensor-core search, FP32 search and sub-pixel pass on the
    affine workload, the device error flag of the bounded waits is clear."""
    import torch

    import paper_1905_06228_gb300 as dic
    p = affine1024
    h = dic.dic_create(p.subset, p.step, p.radius)
    try:
        tf = torch.from_numpy(p.ref).cuda()
        tg = torch.from_numpy(p.defm).cuda()
        dic.dic_set_pair(h, tf, tg)
        n, _, _ = dic.dic_num_pois(h)
        t = lambda dt: torch.empty(n, dtype=dt, device="cuda")
        o = [t(torch.int32), t(torch.int32), t(torch.float32), t(torch.uint8)]
        for form in (TC, 0):
            dic.dic_set_form(h, form)
            dic.dic_integer_search(h, *o)
        dic.dic_check(h)
    finally:
        dic.dic_destroy(h)


def test_affine1024(affine1024):
    p = affine1024
    b = _both(p.ref, p.defm, p.subset, p.step, p.radius)
    idx = np.sort(np.random.default_rng(3).choice(b["n"], 800, replace=False))
    compare_search(b, oracle.integer_search(p.ref, p.defm, p.subset, p.step, p.radius,
                                            poi_idx=idx), idx)


@pytest.mark.parametrize("subset,step,radius,size", [
    (5, 2, 3, 28), (9, 4, 0, 40), (11, 4, 3, 96), (15, 5, 5, 128), (21, 7, 8, 200),
    (33, 9, 4, 96), (41, 12, 6, 120), (51, 20, 5, 140), (63, 30, 3, 150),
])
def test_sizes(subset, step, radius, size):
    f, g = configs.tiny(2000 + subset, size, size - 4, int(0.03 * size * size),
                        Affine(0.003, -0.002, 0.4, 1.2, -0.8, size / 2, size / 2), noise=1.5)
    b = _both(f, g, subset, step, radius)
    compare_search(b, oracle.integer_search(f, g, subset, step, radius))


def test_mixed_and_sine_pairs():
    for p in (configs.mixed(2), configs.mixed(0), configs.sine2048(0)):
        b = _both(p.ref, p.defm, p.subset, p.step, p.radius)
        idx = np.sort(np.random.default_rng(4).choice(b["n"], min(b["n"], 300), replace=False))
        compare_search(b, oracle.integer_search(p.ref, p.defm, p.subset, p.step, p.radius,
                                                poi_idx=idx), idx)


def test_ties_flat_and_planted():
    rng = np.random.default_rng(3)
    period = rng.integers(0, 256, (40, 3)).astype(np.uint8)
    gg = np.ascontiguousarray(np.tile(period, (1, 14)))
    ff = np.ascontiguousarray(np.roll(gg, -1, axis=1))
    b = _both(ff, gg, 5, 5, 3)
    assert (b["u0"] == -2).all()
    flat = np.full((40, 40), 90, np.uint8)
    g, _ = configs.tiny(4, 40, 40, 60)
    _both(flat, g, 5, 5, 2)
    _both(g, flat, 5, 5, 2)
    big, _ = configs.tiny(11, 140, 140, 700)
    f = np.ascontiguousarray(big[20:120, 20:120])
    g = np.ascontiguousarray(big[20 + 5:120 + 5, 20 - 7:120 - 7])
    b = _both(f, g, 15, 6, 10)
    assert (b["u0"] == 7).all() and (b["v0"] == -5).all()


@pytest.mark.parametrize("subset,step,radius,size", [
    (9, 2, 20, 120),     # 24 x 28 POIs meet a tile: 3 chunks of 10 rows (N = 240 -> 256)
    (15, 3, 30, 200),    # 23 x 26 POIs: 3 chunks
])
def test_chunked_poi_blocks(subset, step, radius, size):
    """A tile's POI block larger than one MMA's N = 256 is split into row
    chunks, one CTA each; every chunk's POIs get their slots."""
    f, g = configs.tiny(3000 + subset, size, size, int(0.03 * size * size),
                        Affine(0.004, -0.003, 0.6, 2.2, -1.4, size / 2, size / 2), noise=1.5)
    b = _both(f, g, subset, step, radius)
    compare_search(b, oracle.integer_search(f, g, subset, step, radius))


def test_large_radius_many_slots():
    """Subset 41, step 13, radius 85 (the largest window of the mixed-size
    batch): 276 tiles per POI window (slot index beyond 8 bits), three
    accumulators x 112 POIs = 512 TMEM columns, two chunks.  The FP32 form's
    window does not fit shared memory, so the oracle is the only reference."""
    size = 256
    f, g = configs.tiny(3100, size, size, int(0.035 * size * size),
                        Affine(0.01, -0.008, 1.5, 31.0, -57.0, size / 2, size / 2), noise=1.0)
    b = run_gpu(f, g, 41, 13, 85, subpixel=False, form=TC)
    assert b["n"] == 16
    compare_search(b, oracle.integer_search(f, g, 41, 13, 85))


def test_odd_pitch_images():
    """Images inside wider buffers with an odd row pitch (not 16-byte aligned):
    the tensor-core form reads them with plain loads into its own phase
    images and template bank, so the results equal the unpadded case."""
    f, g = configs.tiny(79, 150, 110, 520, Affine(0.004, 0.002, -0.5, -3.2, 2.1, 75, 55),
                        noise=1.0)
    a = run_gpu(f, g, 15, 5, 6, subpixel=False, form=TC)
    b = run_gpu(f, g, 15, 5, 6, subpixel=False, form=TC, pitch_pad=3)
    for k in INT_KEYS:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    compare_search(b, oracle.integer_search(f, g, 15, 5, 6))


def test_unsupported_geometry_is_reported():
    import torch

    import paper_1905_06228_gb300 as dic
    f, g = configs.tiny(8, 300, 300, 2000)
    h = dic.dic_create(9, 1, 125)   # step 1: 257 POI columns meet one tile (N > 256)
    try:
        dic.dic_set_form(h, TC)
        tf = torch.from_numpy(f).cuda()
        tg = torch.from_numpy(g).cuda()
        dic.dic_set_pair(h, tf, tg)
        n, _, _ = dic.dic_num_pois(h)
        z = torch.empty(n, dtype=torch.int32, device="cuda")
        with pytest.raises(dic.DICError) as e:
            dic.dic_integer_search(h, z, z, z.float(), z.to(torch.uint8))
        assert e.value.code == dic.DIC_ERR_UNSUPPORTED
    finally:
        dic.dic_destroy(h)
