"""Batched form: many pairs of uneven size, subset and search radius in one
CUDA graph of persistent kernels, against the single-pair path (bitwise:
same arithmetic) and against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from workloads import configs
from workloads.speckle import Affine, Rigid

from parity import compare_search, compare_subpixel, run_gpu

pytestmark = pytest.mark.gpu
KEYS = ("u0", "v0", "zncc0", "status0", "u", "v", "ux", "uy", "vx", "vy", "zncc", "iters",
        "status")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _run_batch(pairs, method=0, solve_bits=32, autotune=False, repeat=1, form=0, shape=None):
    """pairs: list of (f, g, subset, step, radius) numpy uint8 pairs; form 1
    runs the tensor-core integer search; shape = (warps_per_cta, grid_mult)
    of the sub-pixel launches."""
    import torch

    import paper_1905_06228_gb300 as dic
    dev = torch.device("cuda:0")
    tens = [(torch.from_numpy(np.ascontiguousarray(f)).to(dev),
             torch.from_numpy(np.ascontiguousarray(g)).to(dev), s, st, r)
            for f, g, s, st, r in pairs]
    h = dic.dic_create(21, 5, 10)
    try:
        if solve_bits != 32:
            dic.dic_set_solve_precision(h, solve_bits)
        if form:
            dic.dic_set_form(h, form)
        dic.dic_set_pairs(h, tens)
        if shape is not None:
            dic.dic_set_batch_shape(h, *shape)
        total, offs = dic.dic_batch_pois(h, len(pairs))
        out = dic.batch_outputs(total, dev)
        chosen = None
        if autotune:
            chosen = dic.dic_autotune(h, method, out)
        for _ in range(repeat):
            dic.dic_run_batch(h, method, out)
        torch.cuda.synchronize()
        res = {k: v.cpu().numpy() for k, v in out.items()}
        return res, offs, chosen
    finally:
        dic.dic_destroy(h)


def _slice(res, offs, k):
    return {key: res[key][offs[k]:offs[k + 1]] for key in KEYS}


def _mixed_small_pairs():
    out = []
    specs = [(128, 15, 5, 5), (200, 21, 7, 8), (256, 31, 10, 6), (160, 41, 13, 4),
             (320, 51, 17, 9), (96, 11, 4, 3)]
    for i, (size, subset, step, radius) in enumerate(specs):
        f, g = configs.tiny(500 + i, size, size - 8 * (i % 3), int(0.035 * size * size),
                            Affine(0.004, -0.003, 0.5, 1.3 - i, 0.7 * i - 1.1,
                                   size / 2, size / 2), noise=1.5)
        out.append((f, g, subset, step, radius))
    return out


def test_batch_equals_single_pair_path_bitwise():
    pairs = _mixed_small_pairs()
    res, offs, _ = _run_batch(pairs, method=0)
    for k, (f, g, s, st, r) in enumerate(pairs):
        single = run_gpu(f, g, s, st, r, method=0)
        b = _slice(res, offs, k)
        assert offs[k + 1] - offs[k] == single["n"]
        for key in KEYS:
            np.testing.assert_array_equal(b[key], single[key], err_msg=f"pair {k} {key}")


@pytest.mark.parametrize("method", [0, 1])
def test_batch_against_oracle(method):
    pairs = _mixed_small_pairs()
    res, offs, _ = _run_batch(pairs, method=method, solve_bits=64)
    for k, (f, g, s, st, r) in enumerate(pairs):
        b = _slice(res, offs, k)
        ref = oracle.integer_search(f, g, s, st, r)
        compare_search(b, ref)
        b["p"] = np.stack([b[n] for n in ("u", "ux", "uy", "v", "vx", "vy")], 1).astype(np.float64)
        compare_subpixel(b, f, g, s, st, r, ref, method, label=f"batch pair {k} m{method}")


def test_graph_replay_and_autotune_keep_results():
    pairs = _mixed_small_pairs()[:3]
    a, _, _ = _run_batch(pairs, repeat=1)
    b, _, chosen = _run_batch(pairs, autotune=True, repeat=2)
    assert chosen[0] in (2, 4, 8) and chosen[1] in (1, 2)
    for key in KEYS:
        np.testing.assert_array_equal(a[key], b[key])


def test_mixed32_512px_pairs():
    """The eight 512x512 pairs of the mixed-size batch (random affine,
    noise 1-3, subset from {15..51}), full size, sampled against the oracle."""
    pairs = []
    for k in range(8):
        p = configs.mixed(k)
        pairs.append((p.ref, p.defm, p.subset, p.step, p.radius))
    res, offs, _ = _run_batch(pairs, method=0, solve_bits=64)
    rng = np.random.default_rng(1)
    for k, (f, g, s, st, r) in enumerate(pairs):
        b = _slice(res, offs, k)
        n = offs[k + 1] - offs[k]
        idx = np.sort(rng.choice(n, min(n, 120), replace=False))
        ref = oracle.integer_search(f, g, s, st, r, poi_idx=idx)
        compare_search(b, ref, idx)
        b["p"] = np.stack([b[n_] for n_ in ("u", "ux", "uy", "v", "vx", "vy")], 1).astype(
            np.float64)
        compare_subpixel(b, f, g, s, st, r, ref, 0, idx=idx, label=f"pair {k}")


def test_sine2048_pairs():
    """Two full-size pairs of the uniform 2048x2048 sinusoidal batch (subset
    41 -- the exact FP32 correlation flushes to int32 -- step 8, search +-24)."""
    pairs = []
    for k in range(2):
        p = configs.sine2048(k)
        pairs.append((p.ref, p.defm, p.subset, p.step, p.radius))
    res, offs, _ = _run_batch(pairs, method=0, solve_bits=64)
    assert offs[1] == 60025 and offs[2] == 120050
    rng = np.random.default_rng(2)
    for k, (f, g, s, st, r) in enumerate(pairs):
        b = _slice(res, offs, k)
        idx = np.sort(rng.choice(60025, 200, replace=False))
        ref = oracle.integer_search(f, g, s, st, r, poi_idx=idx)
        compare_search(b, ref, idx)
        b["p"] = np.stack([b[n_] for n_ in ("u", "ux", "uy", "v", "vx", "vy")], 1).astype(
            np.float64)
        compare_subpixel(b, f, g, s, st, r, ref, 0, idx=idx, label=f"pair {k}")
        assert (b["status"] == 0).mean() > 0.95


def test_batch_tensor_core_search_equals_fp32_batch():
    """The batch graph with the tensor-core search (one search per pair, shared
    scratch) gives bitwise the results of the FP32 batch form: same exact
    integer winners, hence the same sub-pixel starts and iterates."""
    pairs = _mixed_small_pairs()
    a, offs_a, _ = _run_batch(pairs, method=0)
    b, offs_b, _ = _run_batch(pairs, method=0, form=1, repeat=2)
    np.testing.assert_array_equal(offs_a, offs_b)
    for key in KEYS:
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)


@pytest.mark.parametrize("method", [0, 1])
def test_overlapped_subpixel_launches_equal_persistent(method):
    """Per-pair sub-pixel launches on a second stream, overlapping the next
    pairs' tensor-core searches ({0, 0}), give bitwise the persistent
    kernel's results (same per-POI arithmetic), on replay too; the
    autotuner may choose either shape."""
    pairs = _mixed_small_pairs()
    a, _, _ = _run_batch(pairs, method=method, form=1, shape=(8, 2))
    b, _, _ = _run_batch(pairs, method=method, form=1, shape=(0, 0), repeat=3)
    for key in KEYS:
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)
    c, _, chosen = _run_batch(pairs[:3], method=method, form=1, autotune=True, repeat=2)
    assert tuple(chosen) in {(2, 1), (2, 2), (4, 1), (4, 2), (8, 1), (8, 2), (0, 0)}
    for key in KEYS:
        np.testing.assert_array_equal(c[key], a[key][:len(c[key])], err_msg=key)


def test_batch_shape_arguments():
    import torch

    import paper_1905_06228_gb300 as dic
    f, g = configs.tiny(78, 128, 128, 600)
    tf, tg = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    h = dic.dic_create(15, 5, 5)
    try:
        with pytest.raises(dic.DICError) as e:
            dic.dic_set_batch_shape(h, 4, 1)
        assert e.value.code == dic.DIC_ERR_STATE
        dic.dic_set_pairs(h, [(tf, tg)])
        for bad in ((3, 1), (4, 3), (0, 1), (-1, 0)):
            with pytest.raises(dic.DICError) as e:
                dic.dic_set_batch_shape(h, *bad)
            assert e.value.code == dic.DIC_ERR_ARG
        dic.dic_set_batch_shape(h, 0, 0)     # needs the tensor-core form
        total, _ = dic.dic_batch_pois(h, 1)
        out = dic.batch_outputs(total, torch.device("cuda:0"))
        with pytest.raises(dic.DICError) as e:
            dic.dic_run_batch(h, 0, out)
        assert e.value.code == dic.DIC_ERR_ARG
    finally:
        dic.dic_destroy(h)


def test_mixed32_large_window_pairs_tensor_core():
    """The 4096x4096 pairs of the mixed-size batch with the largest search
    windows (radius 85 with subset 41; radius 63 with subset 31; radius 43
    with subset 15 and 638401 POIs), which the FP32 form's shared-memory
    window cannot hold or holds only in part, in one tensor-core batch,
    sampled against the oracle."""
    pairs = []
    for k in (25, 28, 29):
        p = configs.mixed(k)
        pairs.append((p.ref, p.defm, p.subset, p.step, p.radius))
    res, offs, _ = _run_batch(pairs, method=0, solve_bits=32, form=1)
    rng = np.random.default_rng(5)
    for k, (f, g, s, st, r) in enumerate(pairs):
        b = _slice(res, offs, k)
        n = offs[k + 1] - offs[k]
        idx = np.sort(rng.choice(n, 24, replace=False))
        ref = oracle.integer_search(f, g, s, st, r, poi_idx=idx)
        compare_search(b, ref, idx)
        b["p"] = np.stack([b[n_] for n_ in ("u", "ux", "uy", "v", "vx", "vy")], 1).astype(
            np.float64)
        compare_subpixel(b, f, g, s, st, r, ref, 0, idx=idx, label=f"pair {k}")


def test_set_pairs_rejects_oversized_window():
    import torch

    import paper_1905_06228_gb300 as dic
    img = torch.zeros((600, 600), dtype=torch.uint8, device="cuda:0")
    h = dic.dic_create(21, 5, 10)
    try:
        # step 1, radius 120: neither the FP32 window nor one row of the
        # tensor-core POI block (4 accumulators x 256 POIs) fits
        with pytest.raises(dic.DICError) as e:
            dic.dic_set_pairs(h, [(img, img, 51, 1, 120)])
        assert e.value.code == dic.DIC_ERR_UNSUPPORTED
        assert "pair 0" in dic.dic_last_error(h)
    finally:
        dic.dic_destroy(h)


def test_fp32_batch_rejects_tensor_core_only_pair():
    import torch

    import paper_1905_06228_gb300 as dic
    f, g = configs.tiny(77, 600, 600, 12000)
    tf, tg = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    h = dic.dic_create(21, 5, 10)
    try:
        dic.dic_set_pairs(h, [(tf, tg, 21, 7, 10), (tf, tg, 51, 10, 120)])
        total, _ = dic.dic_batch_pois(h, 2)
        out = dic.batch_outputs(total, torch.device("cuda:0"))
        with pytest.raises(dic.DICError) as e:
            dic.dic_run_batch(h, 0, out)
        assert e.value.code == dic.DIC_ERR_UNSUPPORTED
        assert "pair 1" in dic.dic_last_error(h)
        dic.dic_set_form(h, 1)
        dic.dic_run_batch(h, 0, out)
        torch.cuda.synchronize()
        assert (out["status0"][:total].cpu().numpy() <= 6).all()
    finally:
        dic.dic_destroy(h)
