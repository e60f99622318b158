"""The allocation-free sub-pixel call against the regular call.

dic_subpixel_noalloc serves callers that must not call cudaMalloc/cudaFree
(real-time loops that cannot take the device synchronisation, plug-ins whose
host application owns the device-memory budget).  Its scratch is one fixed
array inside the library shared by every call, so this test makes two calls
in a row on different image pairs and checks each against dic_set_pair +
dic_subpixel on the same inputs, within the parity tolerances of the suite.
This file is collected last so that a failure here comes after every other
test has run.
"""
import numpy as np
import pytest

from workloads import configs
from workloads.speckle import Rigid

pytestmark = pytest.mark.gpu

TOL_UV, TOL_GRAD, TOL_ZNCC = 1e-3, 1e-5, 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _regular(dic, tf, tg, subset, step, radius, method, solve_bits=32):
    import torch
    h = dic.dic_create(subset, step, radius, 1, 1e-3, 50)
    try:
        if solve_bits != 32:
            dic.dic_set_solve_precision(h, solve_bits)
        dic.dic_set_pair(h, tf, tg)
        n, _, _ = dic.dic_num_pois(h)
        t = lambda dt: torch.empty(n, dtype=dt, device=tf.device)
        s = dict(u0=t(torch.int32), v0=t(torch.int32), z0=t(torch.float32), st=t(torch.uint8))
        dic.dic_integer_search(h, s["u0"], s["v0"], s["z0"], s["st"])
        o = {k: t(torch.float32) for k in ("u", "v", "ux", "uy", "vx", "vy", "zncc")}
        o["iters"] = t(torch.int32)
        o["status"] = t(torch.uint8)
        dic.dic_subpixel(h, method, s["u0"], s["v0"], s["st"], o["u"], o["v"], o["ux"], o["uy"],
                         o["vx"], o["vy"], o["zncc"], o["iters"], o["status"])
        torch.cuda.synchronize()
        return s, o
    finally:
        dic.dic_destroy(h)


def _noalloc(dic, tf, tg, subset, step, radius, method, s, got, solve_bits=32, stream=None):
    dic.dic_subpixel_noalloc(tf, tg, subset, step, radius, method, s["u0"], s["v0"], s["st"],
                             got["u"], got["v"], got["ux"], got["uy"], got["vx"], got["vy"],
                             got["zncc"], got["iters"], got["status"], solve_bits=solve_bits,
                             stream=stream)


def test_noalloc_matches_regular_path_two_calls():
    import torch

    import paper_1905_06228_gb300 as dic
    dev = torch.device("cuda:0")
    p = configs.rigid256()
    f2, g2 = configs.tiny(4242, 200, 180, 1300, Rigid(-1.7, 2.2), noise=1.0)
    side = torch.cuda.Stream(dev)
    # (images, subset, step, radius, method, solve precision, stream): the
    # second call runs the FP64 solve on a stream other than the default one
    cases = [(p.ref, p.defm, 21, 10, 10, dic.DIC_ICGN, 32, None),
             (f2, g2, 17, 9, 6, dic.DIC_FANR, 64, side)]
    for ref, defm, subset, step, radius, method, bits, stream in cases:
        tf = torch.from_numpy(np.ascontiguousarray(ref)).to(dev)
        tg = torch.from_numpy(np.ascontiguousarray(defm)).to(dev)
        s, want = _regular(dic, tf, tg, subset, step, radius, method, bits)
        n = len(s["u0"])
        assert n > 0
        got = {k: torch.full_like(v, -7) for k, v in want.items()}
        if stream is not None:
            stream.wait_stream(torch.cuda.current_stream(dev))
        _noalloc(dic, tf, tg, subset, step, radius, method, s, got, bits, stream)
        torch.cuda.synchronize()
        w = {k: v.cpu().numpy() for k, v in want.items()}
        g = {k: v.cpu().numpy() for k, v in got.items()}
        np.testing.assert_array_equal(g["status"], w["status"])
        np.testing.assert_array_equal(g["iters"], w["iters"])
        for k in ("u", "v"):
            assert np.abs(g[k] - w[k]).max() < TOL_UV
        for k in ("ux", "uy", "vx", "vy"):
            assert np.abs(g[k] - w[k]).max() < TOL_GRAD
        assert np.abs(g["zncc"] - w["zncc"]).max() < TOL_ZNCC


def test_noalloc_allocates_no_device_memory():
    """After a first call (which may load the library's module on the
    device), further calls leave the device's free memory unchanged: no
    cudaMalloc, no cudaFree, no allocation by the caching allocator."""
    import torch

    import paper_1905_06228_gb300 as dic
    dev = torch.device("cuda:0")
    p = configs.rigid256()
    tf = torch.from_numpy(np.ascontiguousarray(p.ref)).to(dev)
    tg = torch.from_numpy(np.ascontiguousarray(p.defm)).to(dev)
    s, want = _regular(dic, tf, tg, 21, 10, 10, dic.DIC_ICGN)
    got = {k: torch.empty_like(v) for k, v in want.items()}
    _noalloc(dic, tf, tg, 21, 10, 10, dic.DIC_ICGN, s, got)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    reserved0 = torch.cuda.memory_reserved(dev)
    for bits in (32, 64, 32):
        _noalloc(dic, tf, tg, 21, 10, 10, dic.DIC_ICGN, s, got, bits)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
    assert torch.cuda.memory_reserved(dev) == reserved0


def test_noalloc_rejects_images_over_the_limit():
    import torch

    import paper_1905_06228_gb300 as dic
    big = torch.zeros((257, 256), dtype=torch.uint8, device="cuda:0")
    z = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    with pytest.raises(dic.DICError) as e:
        dic.dic_subpixel_noalloc(big, big, 21, 10, 10, dic.DIC_ICGN, z, z, z, z, z, z, z, z, z,
                                 z, z, z)
    assert e.value.code == dic.DIC_ERR_ARG
