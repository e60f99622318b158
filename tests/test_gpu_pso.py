"""Particle swarm integer search on the GPU (Section 2.1, Eqs. 2-4; the
modified swarm with the star search, Sections 3 and 5) against the FP64
oracle on the same uniforms: integer displacement, status, generations run
and distinct pixels evaluated bit-exact, ZNCC within 1e-5."""
import numpy as np
import pytest

import oracle
from workloads import configs, swarm
from workloads.speckle import Rigid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def run_pso(f, g, subset, step, radius, rand, modified, c1=2.0, c2=2.0, vinit=None,
            stop=(995, 1000)):
    import torch

    import paper_1905_06228_gb300 as dic
    dev = torch.device("cuda:0")
    h = dic.dic_create(subset, step, radius)
    # the library borrows the image pointers: keep both tensors alive
    tf = torch.from_numpy(np.ascontiguousarray(f)).to(dev)
    tg = torch.from_numpy(np.ascontiguousarray(g)).to(dev)
    try:
        dic.dic_set_pair(h, tf, tg)
        n, _, _ = dic.dic_num_pois(h)
        t = lambda dt: torch.empty(n, dtype=dt, device=dev)
        o = dict(u0=t(torch.int32), v0=t(torch.int32), zncc=t(torch.float32),
                 status=t(torch.uint8), generations=t(torch.int32), evaluations=t(torch.int32))
        ur = torch.from_numpy(np.ascontiguousarray(rand)).to(dev)
        dic.dic_pso_search(h, ur, o["u0"], o["v0"], o["zncc"], o["status"], o["generations"],
                           o["evaluations"], modified=modified, c1=c1, c2=c2, vinit=vinit,
                           stop=stop)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in o.items()}
    finally:
        dic.dic_destroy(h)


def compare(gpu, ref):
    for k in ("u0", "v0", "status", "generations", "evaluations"):
        np.testing.assert_array_equal(gpu[k], ref[k], err_msg=k)
    assert np.abs(gpu["zncc"] - ref["zncc"]).max() < 1e-5


@pytest.mark.parametrize("modified", [False, True])
def test_rigid256_every_poi(rigid256, modified):
    p = rigid256
    nx, ny = oracle.grid(256, 256, p.subset, p.step, p.radius)
    rand = swarm.uniforms(1, nx * ny)
    gpu = run_pso(p.ref, p.defm, p.subset, p.step, p.radius, rand, modified)
    ref = oracle.pso_search(p.ref, p.defm, p.subset, p.step, p.radius, rand, modified=modified)
    compare(gpu, ref)


@pytest.mark.parametrize("modified", [False, True])
def test_affine1024_every_poi(affine1024, modified):
    """The bench workload (36100 POIs, subset 31, search +-20), both swarms,
    every POI; the modified swarm agrees with the brute-force argmax far more
    often than the standard one (Section 5)."""
    p = affine1024
    rand = swarm.uniforms(1, 36100)
    gpu = run_pso(p.ref, p.defm, p.subset, p.step, p.radius, rand, modified)
    ref = oracle.pso_search(p.ref, p.defm, p.subset, p.step, p.radius, rand, modified=modified)
    compare(gpu, ref)
    assert gpu["evaluations"].max() <= (1250 if modified else 250)


@pytest.mark.parametrize("particles,gens,stop,c", [
    (33, 8, (3, 4), (1.49445, 1.49445)),   # partial second slot, 0.75 stop, other c
    (64, 3, (995, 1000), (2.0, 2.0)),      # two full slots
    (1, 5, (0, 1), (2.0, 2.0)),            # one particle; stop after the first generation
])
@pytest.mark.parametrize("modified", [False, True])
def test_swarm_shapes_and_stop_rules(particles, gens, stop, c, modified):
    f, g = configs.tiny(71, 96, 90, 300, Rigid(2.6, -1.3), noise=1.0)
    subset, step, radius = 15, 7, 6
    nx, ny = oracle.grid(96, 90, subset, step, radius)
    rand = swarm.uniforms(3, nx * ny, generations=gens, particles=particles)
    gpu = run_pso(f, g, subset, step, radius, rand, modified, c1=c[0], c2=c[1], vinit=1.7,
                  stop=stop)
    ref = oracle.pso_search(f, g, subset, step, radius, rand, modified=modified, c1=c[0],
                            c2=c[1], vinit=1.7, stop=stop)
    compare(gpu, ref)
    if stop == (0, 1):  # C >= 0 ends the swarm at the generation that reaches it
        assert (gpu["zncc"][gpu["generations"] < gens] >= 0).all()
        assert (gpu["generations"][gpu["zncc"] < 0] == gens).all()


@pytest.mark.parametrize("subset,step,radius,size", [(5, 3, 2, 30), (41, 12, 6, 120),
                                                     (63, 30, 3, 150)])
def test_subset_sizes(subset, step, radius, size):
    """Template words per lane at each register-slot size (8, 16, 32)."""
    f, g = configs.tiny(1000 + subset, size, size, int(0.03 * size * size), Rigid(1.4, -0.7),
                        noise=1.5)
    nx, ny = oracle.grid(size, size, subset, step, radius)
    rand = swarm.uniforms(5, nx * ny)
    for modified in (False, True):
        gpu = run_pso(f, g, subset, step, radius, rand, modified)
        ref = oracle.pso_search(f, g, subset, step, radius, rand, modified=modified)
        compare(gpu, ref)


def test_flat_subsets_and_planted_shift():
    flat = np.full((60, 60), 90, np.uint8)
    g, _ = configs.tiny(4, 60, 60, 120)
    nx, ny = oracle.grid(60, 60, 7, 6, 3)
    rand = swarm.uniforms(9, nx * ny)
    a = run_pso(flat, g, 7, 6, 3, rand, True)
    compare(a, oracle.pso_search(flat, g, 7, 6, 3, rand, modified=True))
    assert (a["status"] == 1).all() and (a["generations"] == 0).all()
    b = run_pso(g, flat, 7, 6, 3, rand, False)
    compare(b, oracle.pso_search(g, flat, 7, 6, 3, rand, modified=False))
    assert (b["status"] == 6).all()
    big, _ = configs.tiny(11, 140, 140, 700)
    f = np.ascontiguousarray(big[20:120, 20:120])
    gg = np.ascontiguousarray(big[20 + 3:120 + 3, 20 - 4:120 - 4])
    nx, ny = oracle.grid(100, 100, 15, 6, 8)
    rand = swarm.uniforms(2, nx * ny)
    c = run_pso(f, gg, 15, 6, 8, rand, True)
    compare(c, oracle.pso_search(f, gg, 15, 6, 8, rand, modified=True))
    assert ((c["u0"] == 4) & (c["v0"] == -3)).mean() > 0.9


def test_argument_checks():
    import torch

    import paper_1905_06228_gb300 as dic
    lib = dic.lib()
    f, g = configs.tiny(5, 64, 64, 150)
    dev = torch.device("cuda:0")
    h = dic.dic_create(9, 8, 3)
    try:
        z = torch.zeros(8, dtype=torch.int32, device=dev)
        assert lib.dic_pso_search(h, 0, 50, 5, 2.0, 2.0, 1.0, 995, 1000, z.data_ptr(),
                                  *[z.data_ptr()] * 6) == dic.DIC_ERR_STATE
        tf, tg = torch.from_numpy(f).to(dev), torch.from_numpy(g).to(dev)
        dic.dic_set_pair(h, tf, tg)
        for bad in ((0, 65, 5, 995, 1000), (2, 50, 5, 995, 1000), (0, 50, 0, 995, 1000),
                    (0, 50, 5, -1, 1000), (0, 50, 5, 995, 0), (0, 50, 5, 995, (1 << 20) + 1)):
            m, pp, gg, sn, sd = bad
            assert lib.dic_pso_search(h, m, pp, gg, 2.0, 2.0, 1.0, sn, sd, z.data_ptr(),
                                      *[z.data_ptr()] * 6) == dic.DIC_ERR_ARG, bad
        assert lib.dic_pso_search(h, 0, 50, 5, float("nan"), 2.0, 1.0, 995, 1000, z.data_ptr(),
                                  *[z.data_ptr()] * 6) == dic.DIC_ERR_ARG
    finally:
        dic.dic_destroy(h)
