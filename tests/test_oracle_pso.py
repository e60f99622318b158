"""Pins of the oracle's particle swarm integer search (Section 2.1, Eqs. 2-4)
and of the modified swarm with the star search folded in (Sections 3, 5).

The swarm's random numbers are inputs, so a test can choose them: with
r1 = r2 = 0 the swarm flies ballistically under the inertia weight of Eq. 4
alone; with a single term switched on and r = 1 a particle lands exactly on
the point that term pulls it to.  Those special cases have closed forms.
The search results are pinned to Eq. 1 written out here and to the
brute-force search (itself pinned in ``test_oracle_pins.py``).
"""
import math

import numpy as np
import pytest

import oracle
from workloads import configs, swarm
from workloads.speckle import Rigid

NEVER = (2, 1)   # stop threshold C >= 2: never reached, every generation runs


def _eq1_at(f, g, x0, y0, m, du, dv):
    """Eq. 1 written out (means subtracted, float64) at one offset; -inf if flat."""
    a = f[y0 - m:y0 + m + 1, x0 - m:x0 + m + 1].astype(np.float64)
    b = g[y0 + dv - m:y0 + dv + m + 1, x0 + du - m:x0 + du + m + 1].astype(np.float64)
    a = a - a.mean()
    b = b - b.mean()
    den = math.sqrt((a * a).sum()) * math.sqrt((b * b).sum())
    return (a * b).sum() / den if den > 0 else -math.inf


def _centre(k, nx, subset, step, r):
    b = subset // 2 + r + 2
    return b + (k % nx) * step, b + (k // nx) * step


def _pair(seed=3, size=64, noise=2.0, shift=(2.4, -1.6)):
    return configs.tiny(seed, size, size, size * size // 12, Rigid(*shift), noise=noise)


def _rand(n, gens, parts, seed=5):
    return swarm.uniforms(seed, n, gens, parts)


# ------------------------------------------------ Eqs. 3 and 4 (r1 = r2 = 0)
@pytest.mark.parametrize("gmax", [5, 8])
def test_ballistic_flight_follows_inertia_weight(gmax):
    """r1 = r2 = 0: v(t+1) = w(t) v(t) and p(t+1) = p(t) + v(t+1), clamped to
    the window; w falls linearly from 0.9 by 1/(2 Gmax) per generation
    (0.4 at Gmax).  Start: p uniform over [-R, R), v over [-vinit, vinit)."""
    f, g = _pair()
    subset, step, r, parts, vinit = 9, 40, 6, 7, 2.5
    u = _rand(1, gmax, parts)
    u[:, 1:] = 0.0
    res = oracle.pso_search(f, g, subset, step, r, u, vinit=vinit, stop=NEVER,
                            poi_idx=[0], trace=True)
    tr = res["trace"][0]
    assert res["generations"][0] == gmax
    p = r * (2 * u[0, 0, :, 0:2] - 1)
    v = vinit * (2 * u[0, 0, :, 2:4] - 1)
    np.testing.assert_array_equal(tr[0, :, 0:2], p)
    np.testing.assert_array_equal(tr[0, :, 2:4], v)
    w = 0.9
    for t in range(1, gmax):
        v = w * v
        p = np.clip(p + v, -r, r)
        np.testing.assert_allclose(tr[t, :, 2:4], v, rtol=0, atol=1e-13)
        np.testing.assert_allclose(tr[t, :, 0:2], p, rtol=0, atol=1e-12)
        w -= 1.0 / (2 * gmax)
    assert w == pytest.approx(0.4 + 1.0 / (2 * gmax))   # last update used w(Gmax-1)


def test_window_clamp_engages():
    """Positions stay inside [-R, R] and sit on the wall when they overshoot."""
    f, g = _pair()
    u = _rand(4, 5, 20)
    res = oracle.pso_search(f, g, 9, 12, 5, u, vinit=40.0, stop=NEVER, poi_idx=[0, 1, 2, 3],
                            trace=True)
    pos = res["trace"][..., 0:2]
    assert np.nanmax(np.abs(pos)) <= 5
    assert (np.abs(pos[:, 1:]) == 5).mean() > 0.3


# ------------------------------------------------------------- Eq. 2 terms
def test_cognitive_term_pulls_onto_own_best_pixel():
    """One particle, v(0) = 0, c2 = 0, c1 = 1: p(1) = p(0) + r1 (q(0) - p(0))
    with q(0) its nearest pixel (its pbest after generation 0).  r1 = (1, 1/4)
    moves x onto the pixel and y a quarter of the way."""
    f, g = _pair()
    u = _rand(1, 2, 1)
    u[0, 1, 0] = (1.0, 0.25, 0.7, 0.3)
    res = oracle.pso_search(f, g, 9, 12, 6, u, c1=1.0, c2=0.0, vinit=0.0, stop=NEVER,
                            poi_idx=[1], trace=True)
    tr = res["trace"][0]
    p0, q0 = tr[0, 0, 0:2], tr[0, 0, 4:6]
    np.testing.assert_array_equal(q0, np.floor(p0 + 0.5))
    np.testing.assert_array_equal(tr[0, 0, 6:8], q0)          # pbest = evaluated pixel
    np.testing.assert_allclose(tr[1, 0, 0], q0[0], atol=1e-14)
    np.testing.assert_allclose(tr[1, 0, 1], p0[1] + 0.25 * (q0[1] - p0[1]), atol=1e-14)
    np.testing.assert_allclose(tr[1, 0, 2:4], tr[1, 0, 0:2] - p0, atol=1e-14)


def test_social_term_reads_r2_not_r1():
    """The same pull through the c2 term: r2 = (1, 1/4), r1 set to other values
    that would move the particle elsewhere if the c2 term read them."""
    f, g = _pair()
    u = _rand(1, 2, 1)
    u[0, 1, 0] = (0.7, 0.3, 1.0, 0.25)
    res = oracle.pso_search(f, g, 9, 12, 6, u, c1=0.0, c2=1.0, vinit=0.0, stop=NEVER,
                            poi_idx=[1], trace=True)
    tr = res["trace"][0]
    p0, q0 = tr[0, 0, 0:2], tr[0, 0, 4:6]
    np.testing.assert_allclose(tr[1, 0, 0], q0[0], atol=1e-14)
    np.testing.assert_allclose(tr[1, 0, 1], p0[1] + 0.25 * (q0[1] - p0[1]), atol=1e-14)


def test_coefficient_times_random_number():
    """c2 = 2, r2 = 1/2 is the same pull as c2 = 1, r2 = 1."""
    f, g = _pair()
    u = _rand(1, 3, 9)
    a, b = u.copy(), u.copy()
    a[0, 1:, :, 2:4] = 0.5
    b[0, 1:, :, 2:4] = 1.0
    ra = oracle.pso_search(f, g, 9, 12, 6, a, c1=0.0, c2=2.0, vinit=0.0, stop=NEVER,
                           poi_idx=[2], trace=True)
    rb = oracle.pso_search(f, g, 9, 12, 6, b, c1=0.0, c2=1.0, vinit=0.0, stop=NEVER,
                           poi_idx=[2], trace=True)
    np.testing.assert_array_equal(ra["trace"], rb["trace"])


def test_social_term_collapses_swarm_onto_gbest():
    """v(0) = 0, c1 = 0, c2 = 1, r2 = 1: after one update every particle sits on
    gbest, the pixel of generation 0 with the largest Eq. 1 value (first
    particle on ties)."""
    f, g = _pair(seed=8)
    subset, step, r, parts = 9, 12, 6, 10
    nx, ny = oracle.grid(f.shape[1], f.shape[0], subset, step, r)
    k = nx * ny // 2
    x0, y0 = _centre(k, nx, subset, step, r)
    u = _rand(1, 2, parts, seed=11)
    u[0, 1, :, 2:4] = 1.0
    res = oracle.pso_search(f, g, subset, step, r, u, c1=0.0, c2=1.0, vinit=0.0, stop=NEVER,
                            poi_idx=[k], trace=True)
    tr = res["trace"][0]
    c = [_eq1_at(f, g, x0, y0, subset // 2, int(q[0]), int(q[1])) for q in tr[0, :, 4:6]]
    gb = tr[0, int(np.argmax(c)), 4:6]
    np.testing.assert_allclose(tr[1, :, 0:2], np.broadcast_to(gb, (parts, 2)), atol=1e-14)
    # after generation 1 (all particles on gbest) the result is gbest
    assert (res["u0"][0], res["v0"][0]) == (int(gb[0]), int(gb[1]))
    assert res["zncc"][0] == pytest.approx(max(c), abs=1e-12)


def test_pbest_is_best_pixel_seen_so_far():
    """Each particle's pbest after generation t is the first pixel, among those
    it evaluated in generations 0..t, with the largest Eq. 1 value."""
    f, g = _pair(seed=6, noise=3.0)
    subset, step, r, parts, gens = 9, 12, 6, 12, 5
    nx, _ = oracle.grid(f.shape[1], f.shape[0], subset, step, r)
    u = _rand(4, gens, parts, seed=9)
    res = oracle.pso_search(f, g, subset, step, r, u, stop=NEVER, poi_idx=[4, 5, 6, 7],
                            trace=True)
    moved = 0
    for j, k in enumerate([4, 5, 6, 7]):
        if res["status"][j] != oracle.ST_OK:
            continue
        x0, y0 = _centre(k, nx, subset, step, r)
        tr = res["trace"][j]
        for i in range(parts):
            best, bc = None, -math.inf
            for t in range(gens):
                q = tuple(tr[t, i, 4:6].astype(int))
                c = _eq1_at(f, g, x0, y0, subset // 2, *q)
                if best is None or c > bc:
                    best, bc = q, c
                assert tuple(tr[t, i, 6:8].astype(int)) == best
                moved += q != best
    assert moved > 20      # particles often stand on worse pixels than their best


def test_gbest_keeps_first_particle_on_exact_ties():
    """A texture of period 3 in x matches the reference exactly at every third
    horizontal offset (C = 1 at several pixels).  With c1 = 0, c2 = 1, r2 = 1
    and v(0) = 0 the whole swarm lands on gbest after one update: the pixel
    of the lowest-numbered particle that found an exact match."""
    rng = np.random.default_rng(3)
    period = rng.integers(0, 256, (60, 3)).astype(np.uint8)
    g = np.ascontiguousarray(np.tile(period, (1, 20)))        # 60 x 60, period 3 in x
    f = np.ascontiguousarray(np.roll(g, -1, axis=1))           # exact at du = 1 + 3k, dv = 0
    subset, step, r, parts = 7, 30, 4, 60
    nx, ny = oracle.grid(60, 60, subset, step, r)
    m = subset // 2
    u = swarm.uniforms(8, nx * ny, 2, parts)
    u[:, 1, :, 2:4] = 1.0
    res = oracle.pso_search(f, g, subset, step, r, u, c1=0.0, c2=1.0, vinit=0.0, stop=NEVER,
                            trace=True)
    ties = 0
    for k in range(nx * ny):
        x0, y0 = _centre(k, nx, subset, step, r)
        tr = res["trace"][k]
        ref = f[y0 - m:y0 + m + 1, x0 - m:x0 + m + 1]
        exact = [i for i in range(parts)
                 if np.array_equal(ref, g[y0 + int(tr[0, i, 5]) - m:y0 + int(tr[0, i, 5]) + m + 1,
                                          x0 + int(tr[0, i, 4]) - m:x0 + int(tr[0, i, 4]) + m + 1])]
        assert exact
        ties += len({tuple(tr[0, i, 4:6]) for i in exact}) > 1
        gb = tr[0, exact[0], 4:6]
        np.testing.assert_allclose(tr[1, :, 0:2], np.broadcast_to(gb, (parts, 2)), atol=1e-13)
    assert ties >= 1


# ------------------------------------------------------------ star search
def test_modified_swarm_takes_best_of_five():
    """Generation 0 of the modified swarm: each particle's best is the best of
    its nearest pixel and the four around it that lie in the window (Eq. 1
    written out; ties keep the centre, then +x, -x, +y, -y), and it moves
    there."""
    f, g = _pair(seed=9, noise=3.0)
    subset, step, r, parts = 9, 12, 5, 40
    nx, _ = oracle.grid(f.shape[1], f.shape[0], subset, step, r)
    u = _rand(3, 2, parts, seed=2)
    u[:, 1:] = 0.0                                  # generation 1: no pull, v(0) = 0
    res = oracle.pso_search(f, g, subset, step, r, u, modified=True, vinit=0.0, stop=NEVER,
                            poi_idx=[0, 1, 2], trace=True)
    star = [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)]
    checked = 0
    for k in range(3):
        if res["status"][k] == oracle.ST_ZERO_VAR_REF:   # flat corner: no swarm
            continue
        checked += 1
        x0, y0 = _centre(k, nx, subset, step, r)
        tr = res["trace"][k]
        for i in range(parts):
            q = tr[0, i, 4:6].astype(int)
            best, bc = None, -math.inf
            for sx, sy in star:
                du, dv = q[0] + sx, q[1] + sy
                if abs(du) > r or abs(dv) > r:
                    continue
                c = _eq1_at(f, g, x0, y0, subset // 2, du, dv)
                if best is None or c > bc:
                    best, bc = (du, dv), c
            assert tuple(tr[0, i, 6:8].astype(int)) == best
            np.testing.assert_array_equal(tr[1, i, 0:2], best)  # moved there, v = 0
    assert checked >= 2


# ----------------------------------------------------- search results
@pytest.mark.parametrize("modified", [False, True])
def test_result_is_best_evaluated_pixel_and_brute_force_where_high(modified, affine1024):
    """The reported offset carries the largest Eq. 1 value of every pixel the
    swarm evaluated; where that value reaches 0.995 it is the brute-force
    argmax; a swarm that stopped early had reached 0.995."""
    pr = affine1024
    nx, ny = oracle.grid(1024, 1024, pr.subset, pr.step, pr.radius)
    idx = np.random.default_rng(4).choice(nx * ny, 60, replace=False)
    u = swarm.uniforms(3, len(idx))
    res = oracle.pso_search(pr.ref, pr.defm, pr.subset, pr.step, pr.radius, u,
                            modified=modified, poi_idx=idx, trace=True)
    bfs = oracle.integer_search(pr.ref, pr.defm, pr.subset, pr.step, pr.radius, poi_idx=idx)
    m, r = pr.subset // 2, pr.radius
    star = [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)] if modified else [(0, 0)]
    for j, k in enumerate(idx):
        x0, y0 = _centre(k, nx, pr.subset, pr.step, r)
        c = _eq1_at(pr.ref, pr.defm, x0, y0, m, res["u0"][j], res["v0"][j])
        assert res["zncc"][j] == pytest.approx(c, abs=1e-12)
        gens = res["generations"][j]
        tr = res["trace"][j]
        assert np.isnan(tr[gens:]).all() and not np.isnan(tr[:gens]).any()
        seen = set()
        for q in tr[:gens, :, 4:6].reshape(-1, 2).astype(int):
            for sx, sy in star:
                du, dv = q[0] + sx, q[1] + sy
                if abs(du) <= r and abs(dv) <= r and (du, dv) not in seen:
                    seen.add((du, dv))
                    assert _eq1_at(pr.ref, pr.defm, x0, y0, m, du, dv) <= c + 1e-12
        if not modified:
            assert res["evaluations"][j] == len(seen)
        else:
            assert len({tuple(q) for q in tr[:gens, :, 4:6].reshape(-1, 2)}) \
                <= res["evaluations"][j] <= len(seen)
        if res["zncc"][j] >= 0.995:
            assert (res["u0"][j], res["v0"][j]) == (bfs["u0"][j], bfs["v0"][j])
        if gens < u.shape[1]:
            assert res["zncc"][j] >= 0.995


@pytest.mark.parametrize("du,dv", [(3, -2), (-4, 5)])
def test_planted_shift_found_and_modified_converges_faster(du, dv):
    """g(x + du, y + dv) = f(x, y) exactly: where the swarm finds the shift its
    C is 1 and it stops at once.  The modified swarm finds it on more POIs in
    fewer generations (Section 5)."""
    big, _ = configs.tiny(12, 140, 140, 1400)
    f = np.ascontiguousarray(big[10:130, 10:130])
    g = np.ascontiguousarray(big[10 - dv:130 - dv, 10 - du:130 - du])
    subset, step, r = 15, 6, 8
    nx, ny = oracle.grid(120, 120, subset, step, r)
    u = swarm.uniforms(21, nx * ny)
    out = {}
    for mod in (False, True):
        res = oracle.pso_search(f, g, subset, step, r, u, modified=mod)
        hit = (res["u0"] == du) & (res["v0"] == dv)
        assert np.abs(res["zncc"][hit] - 1.0).max() < 1e-14
        assert (res["zncc"][~hit] < 1.0 - 1e-9).all()
        assert (res["generations"][hit] <= 5).all()
        out[mod] = (hit.mean(), res["generations"].mean())
    assert out[True][0] >= 0.95
    assert out[True][0] > out[False][0] and out[True][1] < out[False][1]


def test_exact_stop_threshold():
    """stop = 1/1 (C >= 1, tested exactly) ends the swarm in the generation
    that first reaches the planted shift; none after it runs."""
    big, _ = configs.tiny(13, 90, 90, 600)
    f = np.ascontiguousarray(big[6:84, 6:84])
    g = np.ascontiguousarray(big[5:83, 4:82])    # g(x + 2, y + 1) = f(x, y)
    u = swarm.uniforms(4, 9)
    res = oracle.pso_search(f, g, 11, 8, 4, u, modified=True, stop=(1, 1),
                            poi_idx=np.arange(9), trace=True)
    for j in range(9):
        gens = res["generations"][j]
        found = (res["u0"][j], res["v0"][j]) == (2, 1)
        assert found == (res["zncc"][j] >= 1.0 - 1e-14)
        if found:
            # the shift is among generation gens-1's bests and not before
            bests = res["trace"][j, :, :, 6:8]
            assert ((bests[gens - 1] == (2, 1)).all(axis=1)).any()
            assert not ((bests[:gens - 1] == (2, 1)).all(axis=2)).any()
        else:
            assert gens == 5


def test_zero_variance_statuses():
    """Flat reference subset: no correlation, no swarm.  Flat target: every
    pixel is undefined, the swarm runs all generations and reports none."""
    flat = np.full((40, 40), 90, np.uint8)
    g, _ = configs.tiny(4, 40, 40, 60)
    nx, ny = oracle.grid(40, 40, 5, 4, 3)
    u = swarm.uniforms(1, nx * ny, 3, 6)
    res = oracle.pso_search(flat, g, 5, 4, 3, u)
    assert (res["status"] == oracle.ST_ZERO_VAR_REF).all() and (res["generations"] == 0).all()
    res2 = oracle.pso_search(g, flat, 5, 4, 3, u)
    assert (res2["status"] == oracle.ST_ZERO_VAR_DEF).all()
    assert (res2["zncc"] == 0).all() and (res2["generations"] == 3).all()


def test_argument_errors():
    f, g = _pair()
    u = _rand(1, 2, 3)
    with pytest.raises(ValueError):
        oracle.pso_search(f, g, 9, 12, 6, u, stop=(1, 0), poi_idx=[0])
    with pytest.raises(ValueError):
        oracle.pso_search(f, g, 9, 12, 6, u, stop=(-1, 2), poi_idx=[0])
    with pytest.raises(ValueError):
        oracle.pso_search(f, g, 9, 12, 6, u, poi_idx=[10 ** 6])   # no such POI


def _golden_counts():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "swarm_evaluation_counts.txt")
    out = {}
    for line in open(path):
        line = line.split("#", 1)[0].split()
        if line:
            out[line[0]] = int(line[1])
    return out


def test_evaluation_counts_printed_in_section5():
    """Section 5's counts: at most 250 (standard) and 1250 (modified) Eq. 1
    evaluations per POI for 50 particles and 5 generations, reached when no
    pixel repeats (a wide window, particles in ballistic flight)."""
    gold = _golden_counts()
    parts, gens = gold["particles"], gold["generations"]
    r, subset = 1000, 9
    size = 2 * (subset // 2 + r + 2) + 9
    img = np.random.default_rng(5).integers(0, 256, (size, size), dtype=np.uint8)
    nx, ny = oracle.grid(size, size, subset, 3, r)
    assert nx * ny == 9
    u = swarm.uniforms(6, nx * ny, gens, parts)
    u[:, 0, :, 0:2] = 0.1 + 0.8 * u[:, 0, :, 0:2]    # start at most 0.8 R out: no wall
    u[:, 0, :, 2:4] = 0.8 + 0.2 * u[:, 0, :, 2:4]    # v(0) in [0.6, 1] vinit per direction
    u[:, 1:] = 0.0
    for mod, key in ((False, "max_evaluations_standard"), (True, "max_evaluations_modified")):
        res = oracle.pso_search(img, img, subset, 3, r, u, modified=mod, vinit=60.0,
                                stop=NEVER)
        assert (res["generations"] == gens).all()
        assert res["evaluations"].max() == gold[key]
        assert (res["evaluations"] <= gold[key]).all()
