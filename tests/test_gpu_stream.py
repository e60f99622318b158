"""Consecutive-frame streams (the paper's evaluation with the reference
updated after every pair, Sections 3 and 5.1): each pushed frame is the
target of a pair whose reference is the previous frame.  Every pair's
outputs equal the single-pair calls on (previous frame, frame) bitwise
(same kernels, same arithmetic), over more frames than the ring holds, and
match the FP64 oracle."""
import numpy as np
import pytest

import oracle
from workloads import configs

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


@pytest.fixture(scope="module")
def small_sequence():
    return configs.tensile_sequence(frames=7, size=256, n_speckles=2500, noise=1.0)


def run_stream(frames, subset, step, radius, method=0, form=1, solve_bits=64, interp=0,
               reuse_input=False):
    """Push every frame; return the outputs of pairs 1 .. len(frames)-1."""
    import torch

    import paper_1905_06228_gb300 as dic
    dev = torch.device("cuda:0")
    h = dic.dic_create(subset, step, radius)
    try:
        dic.dic_set_form(h, form)
        dic.dic_set_solve_precision(h, solve_bits)
        if interp:
            dic.dic_set_interpolation(h, interp)
        outs = []
        buf = torch.empty(frames[0].shape, dtype=torch.uint8, device=dev)
        for k, f in enumerate(frames):
            t = torch.from_numpy(np.ascontiguousarray(f)).to(dev)
            if reuse_input:  # one caller buffer for every frame: the push copies it
                buf.copy_(t)
                t = buf
            if k == 0:
                dic.dic_stream_push(h, t, method)
                n, _, _ = dic.dic_num_pois(h)
                continue
            o = dic.batch_outputs(n, dev)
            dic.dic_stream_push(h, t, method, o)
            outs.append(o)
        dic.dic_stream_flush(h)
        torch.cuda.synchronize()
        return [{k: v.cpu().numpy() for k, v in o.items()} for o in outs]
    finally:
        dic.dic_destroy(h)


@pytest.mark.parametrize("form,method", [(1, 0), (0, 0), (1, 1)])
def test_pairs_equal_single_pair_calls(small_sequence, form, method):
    seq = small_sequence
    fr, s, st, r = seq["frames"], seq["subset"], seq["step"], seq["radius"]
    got = run_stream(fr, s, st, r, method=method, form=form)
    assert len(got) == len(fr) - 1
    for k in range(1, len(fr)):
        want = run_gpu(fr[k - 1], fr[k], s, st, r, method=method, solve_bits=64, form=form)
        for key in KEYS:
            np.testing.assert_array_equal(got[k - 1][key], want[key], err_msg=f"pair {k} {key}")


def test_caller_buffer_reused_between_pushes(small_sequence):
    """The push copies the frame into the library's ring, so one caller
    buffer can carry every frame."""
    seq = small_sequence
    fr, s, st, r = seq["frames"], seq["subset"], seq["step"], seq["radius"]
    a = run_stream(fr, s, st, r)
    b = run_stream(fr, s, st, r, reuse_input=True)
    for x, y in zip(a, b):
        for key in KEYS:
            np.testing.assert_array_equal(x[key], y[key])


def test_pairs_against_oracle(small_sequence):
    seq = small_sequence
    fr, s, st, r = seq["frames"], seq["subset"], seq["step"], seq["radius"]
    got = run_stream(fr, s, st, r, method=0)
    for k in (1, 4, 6):
        g = got[k - 1]
        ref = oracle.integer_search(fr[k - 1], fr[k], s, st, r)
        compare_search(g, ref)
        g["p"] = np.stack([g[n] for n in ("u", "ux", "uy", "v", "vx", "vy")], 1).astype(
            np.float64)
        compare_subpixel(g, fr[k - 1], fr[k], s, st, r, ref, 0, label=f"stream pair {k}")


def test_tensile1024_pairs_against_oracle():
    """The tensile workload (1024x1024, subset 31, step 5, search +-12):
    every POI of two consecutive pairs against the oracle, and the imposed
    per-frame increment recovered within the paper's usual 0.05 px."""
    seq = configs.tensile_sequence(frames=3)
    fr, s, st, r = seq["frames"], seq["subset"], seq["step"], seq["radius"]
    got = run_stream(fr, s, st, r, method=0)
    for k in (1, 2):
        g = got[k - 1]
        ref = oracle.integer_search(fr[k - 1], fr[k], s, st, r)
        compare_search(g, ref)
        g["p"] = np.stack([g[n] for n in ("u", "ux", "uy", "v", "vx", "vy")], 1).astype(
            np.float64)
        compare_subpixel(g, fr[k - 1], fr[k], s, st, r, ref, 0, label=f"tensile pair {k}")
        assert (g["status"] == 0).mean() > 0.99
    # frame k-1 -> k: the increment of the map in frame k-1's coordinates
    m1, m2 = seq["maps"][1], seq["maps"][2]
    b = s // 2 + r + 2
    nx = (1024 - 1 - 2 * b) // st + 1
    kk = np.arange(nx * nx)
    x0 = (b + (kk % nx) * st).astype(float)
    y0 = (b + (kk // nx) * st).astype(float)
    xr, yr = m1.inverse(x0, y0)            # reference points of frame 1's pixels
    x2, y2 = m2.forward(xr, yr)            # where frame 2 shows them
    ok = got[1]["status"] == 0
    assert np.abs(got[1]["u"][ok] - (x2 - x0)[ok]).max() < 0.05
    assert np.abs(got[1]["v"][ok] - (y2 - y0)[ok]).max() < 0.05


def test_stream_arguments_and_reset(small_sequence):
    import torch

    import paper_1905_06228_gb300 as dic
    fr = small_sequence["frames"]
    dev = torch.device("cuda:0")
    lib = dic.lib()
    h = dic.dic_create(21, 8, 6)
    try:
        dic.dic_stream_flush(h)  # nothing pending: no-op
        with pytest.raises(dic.DICError) as e:
            dic.dic_num_pois(h)
        assert e.value.code == dic.DIC_ERR_STATE
        t0 = torch.from_numpy(fr[0]).to(dev)
        t1 = torch.from_numpy(fr[1]).to(dev)
        dic.dic_stream_push(h, t0, 0)
        n, _, _ = dic.dic_num_pois(h)
        assert n > 0
        # the second push needs its outputs; a frame of another size is refused
        assert lib.dic_stream_push(h, t1.data_ptr(), 256, 256, 256, 0, None) == dic.DIC_ERR_ARG
        small = torch.zeros((128, 128), dtype=torch.uint8, device=dev)
        o = dic.batch_outputs(n, dev)
        with pytest.raises(dic.DICError) as e:
            dic.dic_stream_push(h, small, 0, o)
        assert e.value.code == dic.DIC_ERR_ARG
        assert lib.dic_stream_push(h, t1.data_ptr(), 256, 256, 256, 7, None) == dic.DIC_ERR_ARG
        dic.dic_stream_push(h, t1, 0, o)
        # after a reset the next push starts a new sequence (of another size)
        dic.dic_stream_reset(h)
        dic.dic_stream_push(h, small, 0)
        n2, _, _ = dic.dic_num_pois(h)
        assert n2 < n
        torch.cuda.synchronize()
        want = run_gpu(fr[0], fr[1], 21, 8, 6, method=0, solve_bits=32, form=0)
        np.testing.assert_array_equal(o["u0"].cpu().numpy(), want["u0"])
        np.testing.assert_array_equal(o["u"].cpu().numpy(), want["u"])
    finally:
        dic.dic_destroy(h)
