"""Pins of the FP64 oracle to facts the paper and the mathematics fix.

None of these compares the oracle with itself: each checks it against a
closed form, an invariance of Eq. 1, brute force written independently here,
a special case with a known exact answer, or the accuracy the paper states
(0.1 px guaranteed, usually below 0.05 px; Section 3).
"""
import math

import numpy as np
import pytest

import oracle
from workloads import configs
from workloads.speckle import Rigid


# ----------------------------------------------------------------- POI grid
@pytest.mark.parametrize("w,h,subset,step,r,count", [
    (256, 256, 21, 10, 10, 484),       # rigid256: 22 x 22
    (1024, 1024, 31, 5, 20, 36100),    # affine1024: 190 x 190
    (2048, 2048, 41, 8, 24, 60025),    # sine2048x64: 245 x 245 per pair
    (1024, 1024, 31, 8, 20, 14161),    # affine1024x8: 119 x 119 per pair
])
def test_grid_counts(w, h, subset, step, r, count):
    nx, ny = oracle.grid(w, h, subset, step, r)
    assert nx * ny == count
    m = subset // 2
    b = m + r + 2
    # last centre keeps the search window plus the 4x4 stencil inside
    assert b + (nx - 1) * step + m + r + 2 <= w - 1


def test_grid_empty_when_image_too_small():
    assert oracle.grid(20, 20, 21, 5, 10) == (0, 0)


# ----------------------------------------------------- ZNCC / integer search
def _eq1_map(f, g, x0, y0, m, r):
    """Eq. 1 written out literally (means subtracted, float64), all offsets."""
    a = f[y0 - m:y0 + m + 1, x0 - m:x0 + m + 1].astype(np.float64)
    a = a - a.mean()
    out = np.full((2 * r + 1, 2 * r + 1), -np.inf)
    for dv in range(-r, r + 1):
        for du in range(-r, r + 1):
            b = g[y0 + dv - m:y0 + dv + m + 1, x0 + du - m:x0 + du + m + 1].astype(np.float64)
            b = b - b.mean()
            den = math.sqrt((a * a).sum()) * math.sqrt((b * b).sum())
            if den > 0:
                out[dv + r, du + r] = (a * b).sum() / den
    return out


@pytest.mark.parametrize("seed,anti", [(1, False), (2, False), (3, True)])
def test_search_matches_brute_force_eq1(seed, anti):
    """Brute force (Section 2.1) over Eq. 1 on tiny inputs, including an
    anti-correlated pair where most candidates have C < 0."""
    f, g = configs.tiny(seed, 28, 26, 35, Rigid(1.3, -0.6), noise=3.0)
    if anti:
        g = (255 - g).astype(np.uint8)
    subset, step, r = 5, 2, 3
    res = oracle.integer_search(f, g, subset, step, r)
    m = subset // 2
    b = m + r + 2
    n_checked = 0
    for k in range(res["nx"] * res["ny"]):
        x0 = b + (k % res["nx"]) * step
        y0 = b + (k // res["nx"]) * step
        cmap = _eq1_map(f, g, x0, y0, m, r)
        if not np.isfinite(cmap).any():     # flat reference or flat targets
            assert res["status"][k] in (oracle.ST_ZERO_VAR_REF, oracle.ST_ZERO_VAR_DEF)
            continue
        assert res["status"][k] == oracle.ST_OK
        best = np.argmax(cmap)          # first maximum in (dv, du) row-major order
        flat = np.sort(cmap.ravel())[::-1]
        assert res["zncc"][k] == pytest.approx(flat[0], abs=1e-12)
        # the chosen offset attains the maximum of the literal Eq. 1 map
        assert cmap[res["v0"][k] + r, res["u0"][k] + r] == pytest.approx(flat[0], abs=1e-12)
        if flat[0] - flat[1] > 1e-9:     # no near-tie: offset is unique
            assert (res["v0"][k], res["u0"][k]) == (best // (2 * r + 1) - r, best % (2 * r + 1) - r)
            n_checked += 1
    assert n_checked > 0.6 * res["nx"] * res["ny"]


def test_identical_subsets_give_one():
    """C = 1 exactly for g = f (Section 2.1: maximum when grey levels equal)."""
    f, _ = configs.tiny(7, 40, 40, 80)
    res = oracle.integer_search(f, f, 7, 3, 4)
    assert (res["u0"] == 0).all() and (res["v0"] == 0).all()
    assert np.abs(res["zncc"] - 1.0).max() < 1e-14


@pytest.mark.parametrize("du,dv", [(3, -2), (-4, 1), (0, 4)])
def test_planted_integer_shift(du, dv):
    """g(x + du, y + dv) = f(x, y) is found exactly, with C = 1."""
    big, _ = configs.tiny(11, 64, 64, 250)
    f = big[8:56, 8:56]
    g = big[8 - dv:56 - dv, 8 - du:56 - du]
    res = oracle.integer_search(np.ascontiguousarray(f), np.ascontiguousarray(g), 9, 4, 5)
    assert (res["u0"] == du).all() and (res["v0"] == dv).all()
    assert np.abs(res["zncc"] - 1.0).max() < 1e-14


def test_affine_intensity_invariance_exact():
    """C is invariant under g -> a g + b, a > 0 (Eq. 1); sign flips for a < 0."""
    f, g = configs.tiny(5, 32, 32, 60, Rigid(0.4, 1.7), noise=2.0)
    f = (f // 3).astype(np.uint8)
    g = (g // 3).astype(np.uint8)            # range 0..85
    g2 = (2 * g.astype(np.int32) + 30).astype(np.uint8)   # a=2, b=30, still 8-bit
    r1 = oracle.integer_search(f, g, 7, 2, 3)
    r2 = oracle.integer_search(f, g2, 7, 2, 3)
    assert (r1["u0"] == r2["u0"]).all() and (r1["v0"] == r2["v0"]).all()
    assert np.abs(r1["zncc"] - r2["zncc"]).max() < 1e-13
    # a = -1: each C becomes -C; the single-candidate search (R = 0) shows it
    g3 = (255 - g.astype(np.int32)).astype(np.uint8)
    s1 = oracle.integer_search(f, g, 7, 2, 0)
    s3 = oracle.integer_search(f, g3, 7, 2, 0)
    assert np.abs(s1["zncc"] + s3["zncc"]).max() < 1e-13


def test_tie_keeps_lowest_linear_index():
    """Equal C at several offsets: the lowest (dv+R)(2R+1)+(du+R) wins."""
    rng = np.random.default_rng(3)
    period = rng.integers(0, 256, (40, 3)).astype(np.uint8)
    g = np.tile(period, (1, 14))             # 40 x 42, period 3 in x
    f = np.roll(g, -1, axis=1)               # f(x) = g(x+1): C = 1 at du = 1 + 3k
    res = oracle.integer_search(f, g, 5, 5, 3)
    assert res["nx"] * res["ny"] > 0
    # candidates with C = 1 at dv = 0: du in {-2, 1}; the lowest index is du = -2
    assert (res["u0"] == -2).all() and (res["v0"] == 0).all()
    assert np.abs(res["zncc"] - 1.0).max() < 1e-14


def test_zero_variance_statuses():
    f = np.full((30, 30), 77, np.uint8)
    g, _ = configs.tiny(4, 30, 30, 40)
    res = oracle.integer_search(f, g, 5, 3, 2)
    assert (res["status"] == oracle.ST_ZERO_VAR_REF).all()
    assert (res["zncc"] == 0).all()
    res2 = oracle.integer_search(g, f, 5, 3, 2)
    assert (res2["status"] == oracle.ST_ZERO_VAR_DEF).all()
    assert (res2["u0"] == -2).all() and (res2["v0"] == -2).all()


# ------------------------------------------------------------------ bicubic
def test_bicubic_nodes_and_central_difference():
    rng = np.random.default_rng(0)
    img = rng.uniform(0, 255, (12, 14))
    for y in range(1, 10):
        for x in range(1, 12):
            v, gx, gy = oracle.bicubic(img, x, y)
            assert v == pytest.approx(img[y, x], abs=1e-12)
            assert gx == pytest.approx(0.5 * (img[y, x + 1] - img[y, x - 1]), abs=1e-12)
            assert gy == pytest.approx(0.5 * (img[y + 1, x] - img[y - 1, x]), abs=1e-12)


def test_bicubic_reproduces_quadratics():
    """The Keys kernel with a = -1/2 reproduces every quadratic exactly (its
    third-order accuracy); any other a, or a wrong basis row, fails here."""
    yy, xx = np.mgrid[0:16, 0:16].astype(np.float64)
    c = [3.0, 0.7, -1.1, 0.05, -0.03, 0.08]
    q = lambda x, y: c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y
    img = q(xx, yy)
    rng = np.random.default_rng(1)
    for _ in range(200):
        x, y = rng.uniform(1, 12.999, 2)
        v, gx, gy = oracle.bicubic(img, x, y)
        assert v == pytest.approx(q(x, y), abs=1e-10)
        assert gx == pytest.approx(c[1] + 2 * c[3] * x + c[4] * y, abs=1e-10)
        assert gy == pytest.approx(c[2] + c[4] * x + 2 * c[5] * y, abs=1e-10)


def test_bicubic_does_not_reproduce_cubics():
    """Guard on the previous pin: the kernel is cubic convolution, not a
    cubic spline through cubics, so a cubic image is not exact."""
    yy, xx = np.mgrid[0:16, 0:16].astype(np.float64)
    img = 0.01 * xx ** 3
    v, _, _ = oracle.bicubic(img, 5.25, 5.0)
    assert abs(v - 0.01 * 5.25 ** 3) > 1e-4


# ------------------------------------------------------ bilinear (Eq. 5)
def test_bilinear_nodes_and_bilinear_functions():
    """Eq. 5 interpolates the four surrounding pixels, so it equals the
    pixel at every node and reproduces any function a + b x + c y + d x y
    exactly, value and gradient (b + d y, c + d x), on every cell."""
    rng = np.random.default_rng(2)
    img = rng.uniform(0, 255, (10, 11))
    for y in range(0, 9):
        for x in range(0, 10):
            assert oracle.bilinear(img, x, y)[0] == img[y, x]
    yy, xx = np.mgrid[0:12, 0:12].astype(np.float64)
    c = [3.0, 0.7, -1.1, 0.09]
    b = lambda x, y: c[0] + c[1] * x + c[2] * y + c[3] * x * y
    img = b(xx, yy)
    for _ in range(200):
        x, y = rng.uniform(0, 10.999, 2)
        v, gx, gy = oracle.bilinear(img, x, y)
        assert v == pytest.approx(b(x, y), abs=1e-11)
        assert gx == pytest.approx(c[1] + c[3] * y, abs=1e-11)
        assert gy == pytest.approx(c[2] + c[3] * x, abs=1e-11)


def test_bilinear_is_continuous_and_not_quadratic():
    """Across a cell boundary the value is continuous (the two patches
    agree on their common edge); a quadratic is not reproduced, which tells
    Eq. 5 apart from the bicubic kernel: x^2 between the nodes 2 and 3 is the
    chord, 6.5 at x = 2.5, not 6.25."""
    rng = np.random.default_rng(3)
    img = rng.uniform(0, 255, (8, 8))
    for y in (1.3, 2.7, 4.0):
        left = oracle.bilinear(img, 3.0 - 1e-9, y)[0]
        right = oracle.bilinear(img, 3.0, y)[0]
        assert left == pytest.approx(right, abs=1e-6)
    yy, xx = np.mgrid[0:8, 0:8].astype(np.float64)
    assert oracle.bilinear(xx ** 2, 2.5, 4.0)[0] == pytest.approx(6.5, abs=1e-12)
    assert oracle.bicubic(xx ** 2, 2.5, 4.0)[0] == pytest.approx(6.25, abs=1e-12)


# --------------------------------------------------------------- sub-pixel
@pytest.mark.parametrize("interp", [oracle.BICUBIC, oracle.BILINEAR])
@pytest.mark.parametrize("method", [oracle.ICGN, oracle.FANR])
@pytest.mark.parametrize("du,dv", [(2, -1), (-3, 2)])
def test_subpixel_exact_integer_shift_fixed_point(method, du, dv, interp):
    """g(x + du, y + dv) = f(x, y) exactly.  Both interpolants equal the
    pixels at integer nodes, so p = (du, 0, 0, dv, 0, 0) makes every
    residual zero: it is an exact fixed point.  Started one pixel away in
    each direction, the iteration must come back to it (through sub-pixel
    positions) to round-off, with C = 1."""
    big, _ = configs.tiny(17, 96, 96, 420)
    f = np.ascontiguousarray(big[10:86, 10:86]).astype(np.float64)
    g = np.ascontiguousarray(big[10 - dv:86 - dv, 10 - du:86 - du]).astype(np.float64)
    subset, step, r = 15, 6, 4
    n = int(np.prod(oracle.grid(76, 76, subset, step, r)))
    z = np.zeros(n, np.int32)
    s = oracle.subpixel(f, g, subset, step, r, z + du + 1, z + dv - 1, np.zeros(n, np.uint8),
                        method=method, tol=1e-11, max_iter=100, interp=interp)
    ok = s["status"] == oracle.ST_OK
    assert ok.mean() > 0.9
    want = np.array([du, 0, 0, dv, 0, 0], np.float64)
    assert np.abs(s["p"][ok] - want).max() < 1e-9
    assert np.abs(s["zncc"][ok] - 1.0).max() < 1e-12
    assert (s["iters"][ok] >= 3).all()


def test_icgn_and_fanr_contract_at_the_same_rate():
    """Near the exact fixed point of an integer shift the two methods are the
    same linear iteration: IC-GN's gradients of f (central differences)
    equal FA-NR's gradients of the interpolated g there (the Keys derivative
    at a node is the central difference), so their Hessians, residuals and
    steps agree to first order.  Each POI's asymptotic contraction rate
    (geometric mean of e(k+1)/e(k) over 1e-9 < e < 1e-4) must agree."""
    big, _ = configs.tiny(17, 96, 96, 420)
    du, dv = 2, -1
    f = np.ascontiguousarray(big[10:86, 10:86]).astype(np.float64)
    g = np.ascontiguousarray(big[10 - dv:86 - dv, 10 - du:86 - du]).astype(np.float64)
    subset, step, r = 15, 6, 4
    n = int(np.prod(oracle.grid(76, 76, subset, step, r)))
    z = np.zeros(n, np.int32)
    want = np.array([du, 0, 0, dv, 0, 0], np.float64)
    rates = []
    for method in (oracle.ICGN, oracle.FANR):
        s = oracle.subpixel(f, g, subset, step, r, z + du + 1, z + dv - 1, np.zeros(n, np.uint8),
                            method=method, tol=0.0, max_iter=80, trajectory=True)
        e = np.linalg.norm(s["traj"] - want, axis=-1)
        rk = np.full(n, np.nan)
        for k in range(n):
            sel = [i for i in range(1, 80) if 1e-9 < e[k, i] < 1e-4 and np.isfinite(e[k, i + 1])]
            if len(sel) >= 3:
                rk[k] = np.exp(np.mean(np.log(e[k, [i + 1 for i in sel]] / e[k, sel])))
        rates.append(rk)
    ok = np.isfinite(rates[0]) & np.isfinite(rates[1])
    assert ok.mean() > 0.9
    assert (rates[0][ok] < 0.9).all()                       # they do contract
    assert (np.abs(rates[0][ok] - rates[1][ok]) < 0.01).mean() >= 0.95


def _warp_matrix(p):
    return np.array([[1 + p[1], p[2], p[0]], [p[4], 1 + p[5], p[3]], [0, 0, 1]], np.float64)


@pytest.mark.parametrize("method", [oracle.ICGN, oracle.FANR])
def test_stop_rule_from_trajectory(method):
    """Reading R9: a POI stops at the first solve whose step has
    sqrt(du^2 + dv^2 + M^2 (dux^2 + duy^2 + dvx^2 + dvy^2)) < tol.  The steps
    are recovered from the returned trajectory without the oracle's update
    code: FA-NR adds the step (p_k - p_(k-1)); IC-GN composes with its
    inverse, so W(dp) = W(p_k)^-1 W(p_(k-1)) as 3x3 matrices."""
    f, g = configs.tiny(21, 64, 64, 260, Rigid(0.6, -0.35), noise=1.0)
    f = f.astype(np.float64)
    g = g.astype(np.float64)
    subset, step, r, tol = 15, 4, 3, 1e-3
    m = subset // 2
    res0 = oracle.integer_search(f.astype(np.uint8), g.astype(np.uint8), subset, step, r)
    s = oracle.subpixel(f, g, subset, step, r, res0["u0"], res0["v0"], res0["status"],
                        method=method, tol=tol, max_iter=50, trajectory=True)
    checked = 0
    for k in np.flatnonzero(s["status"] == oracle.ST_OK):
        n = s["iters"][k]
        norms = []
        for i in range(1, n + 1):
            a, b = s["traj"][k, i - 1], s["traj"][k, i]
            if method == oracle.FANR:
                d = b - a
            else:
                wd = np.linalg.solve(_warp_matrix(b), _warp_matrix(a))
                d = np.array([wd[0, 2], wd[0, 0] - 1, wd[0, 1], wd[1, 2], wd[1, 0], wd[1, 1] - 1])
            norms.append(math.sqrt(d[0] ** 2 + d[3] ** 2 + m * m * (d[1] ** 2 + d[2] ** 2 +
                                                                  d[4] ** 2 + d[5] ** 2)))
        assert norms[-1] < tol * (1 + 1e-9)
        assert all(x >= tol * (1 - 1e-9) for x in norms[:-1])
        checked += 1
    assert checked > 50


def test_fanr_lands_on_the_dense_grid_minimum_of_znssd(rigid256):
    """Brute force over the objective: on noise-free speckles (rigid256),
    ZNSSD = 2 - 2C (Eq. 1) evaluated on a dense (u, v) grid of 5e-4 px
    around FA-NR's result (gradient parameters held at FA-NR's values) is
    smallest at FA-NR's (u, v), within one grid step.  IC-GN's fixed point
    (stationary for its reference-gradient Jacobian rather than the target
    gradient) lies within 3e-3 px of it; the two methods agree within
    5e-3 px."""
    pr = rigid256
    f8, g8 = pr.ref, pr.defm
    f, g = f8.astype(np.float64), g8.astype(np.float64)
    subset, step, r = pr.subset, pr.step, pr.radius
    idx = np.arange(0, 484, 61)
    s0 = oracle.integer_search(f8, g8, subset, step, r, poi_idx=idx)
    res = [oracle.subpixel(f, g, subset, step, r, s0["u0"], s0["v0"], s0["status"], method=m,
                           tol=1e-8, max_iter=200, poi_idx=idx)
           for m in (oracle.ICGN, oracle.FANR)]
    assert (res[0]["status"] == oracle.ST_OK).all() and (res[1]["status"] == oracle.ST_OK).all()
    assert np.abs(res[0]["p"][:, [0, 3]] - res[1]["p"][:, [0, 3]]).max() < 5e-3
    h, kk = 5e-4, 6
    steps = h * np.arange(-kk, kk + 1)
    for j, k in enumerate(idx):
        grid_p = np.repeat(res[1]["p"][j][None], len(steps) ** 2, 0)
        grid_p[:, 0] += np.repeat(steps, len(steps))
        grid_p[:, 3] += np.tile(steps, len(steps))
        _, per = oracle.znssd(f, g, subset, step, r, grid_p, poi_idx=np.full(len(grid_p), k),
                              grad=False, per_poi=True)
        i = int(np.argmin(per))
        assert i // len(steps) not in (0, 2 * kk) and i % len(steps) not in (0, 2 * kk)
        best = grid_p[i, [0, 3]]
        assert np.abs(best - res[1]["p"][j, [0, 3]]).max() <= h + 1e-12      # FA-NR
        assert np.abs(best - res[0]["p"][j, [0, 3]]).max() <= 3e-3           # IC-GN


@pytest.mark.parametrize("method", [oracle.ICGN, oracle.FANR])
def test_subpixel_rigid_speckle_accuracy(rigid256, method):
    """Imposed rigid field (3.4, -2.7) px on analytically re-rendered
    speckles: within the paper's usual accuracy (0.05 px), small bias."""
    p = rigid256
    r = oracle.integer_search(p.ref, p.defm, p.subset, p.step, p.radius)
    assert (r["u0"] >= 3).all() and (r["u0"] <= 4).all() and (r["v0"] == -3).all()
    s = oracle.subpixel(p.ref, p.defm, p.subset, p.step, p.radius, r["u0"], r["v0"], r["status"],
                        method=method)
    assert (s["status"] == oracle.ST_OK).all()
    eu, ev = s["u"] - 3.4, s["v"] + 2.7
    assert abs(eu.mean()) < 0.02 and abs(ev.mean()) < 0.02
    assert np.abs(eu).max() < 0.05 and np.abs(ev).max() < 0.05
    grads = s["p"][:, [1, 2, 4, 5]]
    assert np.abs(grads).mean() < 2e-3 and np.abs(grads).max() < 1e-2
    assert s["zncc"].min() > 0.99


@pytest.mark.parametrize("method", [oracle.ICGN, oracle.FANR])
def test_subpixel_rigid_speckle_accuracy_bilinear(rigid256, method):
    """The same field with the bilinear interpolation of Eq. 5: within the
    paper's guaranteed 0.1 px (Section 3), and measurably less accurate than
    bicubic on the same POIs (the interpolation error the paper trades for
    computation, Section 2.2)."""
    p = rigid256
    r = oracle.integer_search(p.ref, p.defm, p.subset, p.step, p.radius)
    kw = dict(method=method)
    s1 = oracle.subpixel(p.ref, p.defm, p.subset, p.step, p.radius, r["u0"], r["v0"],
                         r["status"], interp=oracle.BILINEAR, **kw)
    s3 = oracle.subpixel(p.ref, p.defm, p.subset, p.step, p.radius, r["u0"], r["v0"],
                         r["status"], **kw)
    assert (s1["status"] == oracle.ST_OK).all()
    e1 = np.hypot(s1["u"] - 3.4, s1["v"] + 2.7)
    e3 = np.hypot(s3["u"] - 3.4, s3["v"] + 2.7)
    assert e1.max() < 0.1 and e1.mean() < 0.02
    assert e1.mean() > e3.mean()
    assert s1["zncc"].min() > 0.99


def test_subpixel_affine_speckle_accuracy(affine1024):
    p = affine1024
    nx, ny = oracle.grid(1024, 1024, p.subset, p.step, p.radius)
    idx = np.sort(np.random.default_rng(0).choice(nx * ny, 200, replace=False))
    r = oracle.integer_search(p.ref, p.defm, p.subset, p.step, p.radius, poi_idx=idx)
    s = oracle.subpixel(p.ref, p.defm, p.subset, p.step, p.radius, r["u0"], r["v0"],
                        r["status"], poi_idx=idx)
    b = p.subset // 2 + p.radius + 2
    x0 = (b + (idx % nx) * p.step).astype(float)
    y0 = (b + (idx // nx) * p.step).astype(float)
    gt = np.stack(p.deformation.displacement(x0, y0), 1)
    e = np.abs(s["p"] - gt)
    assert (s["status"] == oracle.ST_OK).all()
    assert e[:, [0, 3]].max() < 0.05 and e[:, [0, 3]].mean() < 0.01
    assert e[:, [1, 2, 4, 5]].mean() < 1e-3 and e[:, [1, 2, 4, 5]].max() < 5e-3


@pytest.mark.parametrize("method", [oracle.ICGN, oracle.FANR])
def test_subpixel_affine_intensity_invariance(method):
    """ZNSSD normalisation: g -> a g + b leaves p and C unchanged."""
    f, g = configs.tiny(21, 48, 48, 120, Rigid(0.6, -0.35), noise=1.0)
    f = f.astype(np.float64)
    g = g.astype(np.float64)
    kw = dict(subset=11, step=6, radius=2)
    n = np.prod(oracle.grid(48, 48, 11, 6, 2))
    z = np.zeros(n, np.int32)
    s1 = oracle.subpixel(f, g, u0=z + 1, v0=z, status0=np.zeros(n, np.uint8), method=method, **kw)
    s2 = oracle.subpixel(f, 1.7 * g + 13.0, u0=z + 1, v0=z, status0=np.zeros(n, np.uint8),
                         method=method, **kw)
    assert np.abs(s1["p"] - s2["p"]).max() < 1e-9
    assert np.abs(s1["zncc"] - s2["zncc"]).max() < 1e-12
    assert (s1["iters"] == s2["iters"]).all()


def test_subpixel_status_paths():
    f, g = configs.tiny(9, 48, 48, 120, Rigid(0.6, -0.35), noise=1.0)
    kw = dict(subset=11, step=6, radius=2)
    n = np.prod(oracle.grid(48, 48, 11, 6, 2))
    z = np.zeros(n, np.int32)
    ok = np.zeros(n, np.uint8)
    # iteration cap: one solve cannot meet a 1e-12 tolerance
    s = oracle.subpixel(f, g, u0=z + 1, v0=z, status0=ok, tol=1e-12, max_iter=1, **kw)
    assert (s["status"] == oracle.ST_MAX_ITER).all() and (s["iters"] == 1).all()
    # statuses from the integer search pass straight through
    bad = np.full(n, oracle.ST_ZERO_VAR_REF, np.uint8)
    s = oracle.subpixel(f, g, u0=z, v0=z, status0=bad, **kw)
    assert (s["status"] == oracle.ST_ZERO_VAR_REF).all() and (s["iters"] == 0).all()
    # a start that pushes the subset against the image edge stops in bounds
    s = oracle.subpixel(f, g, u0=z - 9, v0=z, status0=ok, **kw)
    assert (s["status"] != oracle.ST_OK).any()
    # flat reference subset -> zero variance even if the search was skipped
    flat = np.full((48, 48), 50.0)
    s = oracle.subpixel(flat, g, u0=z, v0=z, status0=ok, **kw)
    assert (s["status"] == oracle.ST_ZERO_VAR_REF).all()


def test_nonfinite_and_singular_statuses():
    """A NaN grey level inside the warped subset makes the sums non-finite
    (status NONFINITE, no step taken); a reference that varies along x only
    has fy = 0 everywhere, so IC-GN's Hessian (rows of fy terms all zero) is
    singular (status SINGULAR) while the shape stays at its start."""
    f, g = configs.tiny(9, 48, 48, 120, Rigid(0.6, -0.35), noise=1.0)
    f = f.astype(np.float64)
    g = g.astype(np.float64)
    subset, step, r = 11, 6, 2
    nx, ny = oracle.grid(48, 48, subset, step, r)
    n = nx * ny
    z = np.zeros(n, np.int32)
    ok = np.zeros(n, np.uint8)
    gn = g.copy()
    gn[:, :] = np.nan                                  # every subset sees NaN
    for method in (oracle.ICGN, oracle.FANR):
        s = oracle.subpixel(f, gn, subset, step, r, z, z, ok, method=method)
        assert (s["status"] == oracle.ST_NONFINITE).all()
        assert (s["p"] == 0).all() and (s["iters"] == 0).all()
    ramp = np.tile(np.sin(np.arange(48) * 0.7) * 60 + 100, (48, 1))   # varies along x only
    s = oracle.subpixel(ramp, g, subset, step, r, z, z, ok, method=oracle.ICGN)
    assert (s["status"] == oracle.ST_SINGULAR).all()
    assert (s["p"] == 0).all() and (s["iters"] == 0).all()
    # FA-NR builds its Hessian from the target each iteration: singular at the
    # first solve when g varies along x only
    s = oracle.subpixel(f, ramp, subset, step, r, z, z, ok, method=oracle.FANR)
    assert (s["status"] == oracle.ST_SINGULAR).all()
    assert (s["p"] == 0).all() and (s["iters"] == 1).all()
    # one NaN pixel stops only the POIs whose subsets contain it
    k = n // 2
    b = subset // 2 + r + 2
    x0, y0 = b + (k % nx) * step, b + (k // nx) * step
    g1 = g.copy()
    g1[y0, x0] = np.nan
    s = oracle.subpixel(f, g1, subset, step, r, z, z, ok, method=oracle.ICGN)
    xs, ys = b + (np.arange(n) % nx) * step, b + (np.arange(n) // nx) * step
    near = (np.abs(xs - x0) <= subset // 2 + 2) & (np.abs(ys - y0) <= subset // 2 + 2)
    assert s["status"][k] == oracle.ST_NONFINITE
    assert (s["status"][~near] != oracle.ST_NONFINITE).all()


def test_bounds_rule_at_its_edges():
    """Reading R12: a shape is usable while every corner of the warped subset
    lies in [1, W-2) x [1, H-2) (the 4x4 stencil stays inside).  The ZNSSD
    skips (loss 0) exactly the shapes that break it; probe each edge with
    translations that put the extreme corner just inside and on it."""
    f, g = configs.tiny(9, 48, 48, 120, Rigid(0.6, -0.35), noise=1.0)
    f = f.astype(np.float64)
    g = g.astype(np.float64)
    subset, step, r = 11, 6, 2
    m = subset // 2
    nx, ny = oracle.grid(48, 48, subset, step, r)
    b = m + r + 2
    x0 = y0 = b                                    # POI 0, top-left corner at (x0-m, y0-m)
    eps = 1e-9
    lo = 1.0 - (x0 - m)                            # u that puts the left edge at x = 1
    hi = (48 - 2.0) - (x0 + m)                     # u that puts the right edge at x = W - 2
    cases = [((lo, 0.0), True), ((lo - eps, 0.0), False),
             ((hi - eps, 0.0), True), ((hi, 0.0), False),
             ((0.0, lo), True), ((0.0, lo - eps), False),
             ((0.0, hi - eps), True), ((0.0, hi), False)]
    p = np.zeros((len(cases), 6))
    for i, ((u, v), _) in enumerate(cases):
        p[i, 0], p[i, 3] = u, v
    _, per = oracle.znssd(f, g, subset, step, r, p, poi_idx=np.zeros(len(cases), np.int64),
                          grad=False, per_poi=True)
    for (uv, inside), loss in zip(cases, per):
        assert (loss > 0) == inside, (uv, inside, loss)
    # a gradient term moves the edges apart: with u = lo + 0.1 m the left
    # edge sits at x = 1 - (ux - 0.1) m, inside for ux just below 0.1
    q = np.zeros((2, 6))
    q[:, 0] = lo + 0.1 * m
    q[0, 1] = 0.1 - 1e-6
    q[1, 1] = 0.1 + 1e-6
    _, per2 = oracle.znssd(f, g, subset, step, r, q, poi_idx=np.zeros(2, np.int64), grad=False,
                           per_poi=True)
    assert per2[0] > 0 and per2[1] == 0


# -------------------------------------------------------- ZNSSD and adjoint
def _adjoint_case():
    f, g = configs.tiny(31, 40, 40, 100, Rigid(0.8, 0.3), noise=1.0)
    f = f.astype(np.float64)
    g = g.astype(np.float64)
    n = int(np.prod(oracle.grid(40, 40, 9, 7, 2)))
    rng = np.random.default_rng(5)
    p = np.zeros((n, 6))
    p[:, 0] = 0.8 + rng.uniform(-0.3, 0.3, n)
    p[:, 3] = 0.3 + rng.uniform(-0.3, 0.3, n)
    p[:, [1, 2, 4, 5]] = rng.uniform(-3e-3, 3e-3, (n, 4))
    return f, g, p, dict(subset=9, step=7, radius=2)


def test_znssd_zero_at_exact_match_and_equals_2_minus_2c():
    f, g = configs.tiny(2, 40, 40, 100)
    n = int(np.prod(oracle.grid(40, 40, 9, 7, 2)))
    loss = oracle.znssd(f, f, 9, 7, 2, np.zeros((n, 6)), grad=False)
    assert abs(loss) < 1e-20
    # ZNSSD = 2 - 2 C per subset (both normalised vectors have unit norm)
    f2, g2 = configs.tiny(3, 40, 40, 100, Rigid(0.4, 0.2), noise=2.0)
    z = np.zeros(n, np.int32)
    s = oracle.subpixel(f2, g2, 9, 7, 2, z, z, np.zeros(n, np.uint8))
    loss = oracle.znssd(f2, g2, 9, 7, 2, s["p"], grad=False)
    assert loss == pytest.approx(np.sum(2 - 2 * s["zncc"]), rel=1e-10)


def test_adjoint_matches_central_differences():
    f, g, p, kw = _adjoint_case()
    loss, dg, dp = oracle.znssd(f, g, p=p, **kw)
    h = 1e-5
    for k in range(p.shape[0]):
        for a in range(6):
            pp, pm = p.copy(), p.copy()
            pp[k, a] += h
            pm[k, a] -= h
            fd = (oracle.znssd(f, g, p=pp, grad=False, **kw)
                  - oracle.znssd(f, g, p=pm, grad=False, **kw)) / (2 * h)
            assert dp[k, a] == pytest.approx(fd, rel=1e-5, abs=1e-7 * max(1.0, abs(fd)))
    rng = np.random.default_rng(8)
    touched = np.argwhere(dg != 0)
    for (y, x) in touched[rng.choice(len(touched), 40, replace=False)]:
        gp, gm = g.copy(), g.copy()
        gp[y, x] += 1e-3
        gm[y, x] -= 1e-3
        fd = (oracle.znssd(f, gp, p=p, grad=False, **kw)
              - oracle.znssd(f, gm, p=p, grad=False, **kw)) / 2e-3
        assert dg[y, x] == pytest.approx(fd, rel=1e-5, abs=1e-9)


# ------------------------------------------------- Eq. 1 at a given shape
@pytest.mark.parametrize("interp", [oracle.BICUBIC, oracle.BILINEAR])
def test_zncc_at_integer_shapes_is_the_exact_search_value(interp):
    """At integer shapes every warped point is a pixel, where both
    interpolants give the pixel itself, so Eq. 1 at (u0, 0, 0, v0, 0, 0)
    must be the brute-force search's value, which comes from exact integer
    sums (independent code); and Eq. 1 written out literally here at a few
    POIs."""
    f, g = configs.tiny(31, 64, 60, 160, Rigid(1.6, -2.3), noise=2.0)
    s = oracle.integer_search(f, g, 9, 6, 4)
    n = len(s["u0"])
    p = np.zeros((n, 6))
    p[:, 0], p[:, 3] = s["u0"], s["v0"]
    c = oracle.zncc_at(f, g, 9, 6, 4, p, interp=interp)
    assert np.abs(c - s["zncc"]).max() < 1e-12
    nx = s["nx"]
    b = 4 + 4 + 2
    for k in (0, n // 2, n - 1):
        x0, y0 = b + (k % nx) * 6, b + (k // nx) * 6
        lit = _eq1_map(f, g, x0, y0, 4, 4)[s["v0"][k] + 4, s["u0"][k] + 4]
        assert abs(c[k] - lit) < 1e-12


def test_zncc_at_invariance_bounds_and_flat_subsets():
    """Eq. 1 at a non-integer shape is invariant under g -> a g + b (a > 0)
    and flips sign for a < 0; it equals 1 - L/2 with L the summed ZNSSD of
    the same subset; shapes that push a corner off [1, W-2) and flat
    reference subsets give NaN."""
    f, g = configs.tiny(32, 70, 70, 200, Rigid(0.4, 0.7), noise=1.0)
    nx, ny = oracle.grid(70, 70, 11, 7, 3)
    n = nx * ny
    rng = np.random.default_rng(5)
    p = np.column_stack([rng.uniform(-1, 1, n), rng.uniform(-0.02, 0.02, n),
                         rng.uniform(-0.02, 0.02, n), rng.uniform(-1, 1, n),
                         rng.uniform(-0.02, 0.02, n), rng.uniform(-0.02, 0.02, n)])
    c = oracle.zncc_at(f, g, 11, 7, 3, p)
    assert np.isfinite(c).all() and (np.abs(c) <= 1 + 1e-12).all()
    c2 = oracle.zncc_at(f, 1.7 * g.astype(np.float64) + 13.0, 11, 7, 3, p)
    assert np.abs(c2 - c).max() < 1e-12
    c3 = oracle.zncc_at(f, 255.0 - g.astype(np.float64), 11, 7, 3, p)
    assert np.abs(c3 + c).max() < 1e-12
    _, _, _, lp = oracle.znssd(f, g, 11, 7, 3, p, per_poi=True)
    assert np.abs((1 - lp / 2) - c).max() < 1e-12
    q = p.copy()
    q[0, 0] = -40.0
    assert np.isnan(oracle.zncc_at(f, g, 11, 7, 3, q)[0])
    flat = np.full_like(f, 77)
    assert np.isnan(oracle.zncc_at(flat, g, 11, 7, 3, p)).all()


@pytest.mark.parametrize("interp", [oracle.BICUBIC, oracle.BILINEAR])
def test_zncc_at_non_integer_shape_written_out(interp):
    """Eq. 1 written out here at a non-integer first-order shape: the warp of
    every subset point, the (separately pinned) interpolant sampled point by
    point, means subtracted, normalised."""
    f, g = configs.tiny(33, 48, 48, 110, Rigid(0.3, -0.2), noise=1.0)
    subset, step, r = 7, 9, 2
    nx, ny = oracle.grid(48, 48, subset, step, r)
    k = nx + 1
    x0, y0 = 3 + 2 + 2 + (k % nx) * step, 3 + 2 + 2 + (k // nx) * step
    pk = np.array([0.37, 0.021, -0.013, -0.61, 0.008, 0.017])
    p = np.zeros((nx * ny, 6))
    p[k] = pk
    c = oracle.zncc_at(f, g, subset, step, r, p, interp=interp)[k]
    sample = oracle.bicubic if interp == oracle.BICUBIC else oracle.bilinear
    a, b = [], []
    for dy in range(-3, 4):
        for dx in range(-3, 4):
            a.append(float(f[y0 + dy, x0 + dx]))
            x = x0 + dx + pk[0] + pk[1] * dx + pk[2] * dy
            y = y0 + dy + pk[3] + pk[4] * dx + pk[5] * dy
            b.append(sample(g, x, y)[0])
    a, b = np.array(a) - np.mean(a), np.array(b) - np.mean(b)
    lit = (a * b).sum() / math.sqrt((a * a).sum() * (b * b).sum())
    assert abs(c - lit) < 1e-12


# --------------------------------------------- second-order shape function
def test_warp2_matrix_rows_are_the_warped_monomials_to_second_order():
    """Rows 4-6 of the 6x6 representation give xi', eta', 1 exactly; rows
    1-3 give xi'^2, xi' eta', eta'^2 up to terms of third and higher order
    (the difference shrinks eightfold when (xi, eta) halves)."""
    # every coefficient well away from zero, so each product term of the
    # matrix matters
    p = np.array([1.3, 0.04, -0.03, 0.02, -0.015, 0.01, -0.9, 0.025, 0.035, -0.012, 0.018,
                  0.02])
    Mx = oracle.warp2_matrix(p)

    def exact(xi, eta):
        e = np.array([1, xi, eta, 0.5 * xi * xi, xi * eta, 0.5 * eta * eta])
        xs = xi + p[:6] @ e
        ys = eta + p[6:] @ e
        return np.array([xs * xs, xs * ys, ys * ys, xs, ys, 1.0])

    def lifted(xi, eta):
        return Mx @ np.array([xi * xi, xi * eta, eta * eta, xi, eta, 1.0])

    for a, b in ((0.07, -0.04), (-0.03, 0.09)):
        d1 = exact(a, b) - lifted(a, b)
        d2 = exact(a / 2, b / 2) - lifted(a / 2, b / 2)
        assert np.abs(d1[3:]).max() < 1e-13 and np.abs(d2[3:]).max() < 1e-13
        # rows 1-3: the dropped terms are cubic (and quartic) in (xi, eta),
        # so near the origin the remainder shrinks eightfold when (xi, eta)
        # halves; a missing or wrong second-order term would shrink it
        # only fourfold
        ratio = np.abs(d2[:3]) / np.abs(d1[:3])
        assert ((ratio > 0.11) & (ratio < 0.14)).all(), ratio


def test_compose2_identity_and_first_order_case():
    """W(p) W(0)^-1 = W(p); for first-order p and dp the update is the 3x3
    affine composition P D^-1 (written out here)."""
    rng = np.random.default_rng(8)
    p = rng.normal(0, [1, 0.02, 0.02, 0.001, 0.001, 0.001, 1, 0.02, 0.02, 0.001, 0.001, 0.001])
    assert np.abs(oracle.compose2(p, np.zeros(12)) - p).max() < 1e-14
    p1 = np.zeros(12)
    d1 = np.zeros(12)
    p1[[0, 1, 2, 6, 7, 8]] = [2.3, 0.01, -0.02, -1.1, 0.015, 0.004]
    d1[[0, 1, 2, 6, 7, 8]] = [0.05, 0.001, 0.002, -0.03, -0.0015, 0.001]

    def aff(q):
        return np.array([[1 + q[1], q[2], q[0]], [q[7], 1 + q[8], q[6]], [0, 0, 1]])
    want = aff(p1) @ np.linalg.inv(aff(d1))
    got = oracle.compose2(p1, d1)
    assert np.abs(got[[3, 4, 5, 9, 10, 11]]).max() < 1e-15
    np.testing.assert_allclose([got[1] + 1, got[2], got[0], got[7], got[8] + 1, got[6]],
                               [want[0, 0], want[0, 1], want[0, 2], want[1, 0], want[1, 1],
                                want[1, 2]], rtol=0, atol=1e-13)


@pytest.mark.parametrize("method", [oracle.ICGN, oracle.FANR])
def test_subpixel2_integer_shift_fixed_point(method):
    big, _ = configs.tiny(21, 120, 120, 500)
    f = np.ascontiguousarray(big[10:110, 10:110])
    g = np.ascontiguousarray(big[10 - 2:110 - 2, 10 - 3:110 - 3])  # shift (3, 2)
    s = oracle.integer_search(f, g, 21, 10, 6)
    u0 = s["u0"] - 1
    v0 = s["v0"] + 1
    r = oracle.subpixel2(f, g, 21, 10, 6, u0, v0, s["status"], method=method, tol=1e-10)
    ok = r["status"] == 0
    assert ok.mean() > 0.9
    want = np.zeros(12)
    want[0], want[6] = 3, 2
    assert np.abs(r["p"][ok] - want).max() < 1e-8
    assert np.abs(r["zncc"][ok] - 1).max() < 1e-12


def _quadratic_pair(noise=0.0):
    from workloads.speckle import Quadratic, render_pair
    d = Quadratic(cu=(1.6, 0.004, -0.003, 8e-4, -5e-4, 6e-4),
                  cv=(-0.9, 0.002, 0.005, -6e-4, 7e-4, 5e-4), cx=127.5, cy=127.5)
    f, g = render_pair(411, 256, 256, 3200, d, noise, pad=30.0)
    return f, g, d


@pytest.mark.parametrize("method", [oracle.ICGN, oracle.FANR])
def test_subpixel2_recovers_an_imposed_quadratic_field(method):
    """Noise-free speckles under a quadratic field: the second-order shape
    recovers u, v and all ten derivatives at every POI (the first-order
    shape cannot follow the curvature and misses it)."""
    f, g, d = _quadratic_pair()
    subset, step, r = 31, 16, 12
    s = oracle.integer_search(f, g, subset, step, r)
    res = oracle.subpixel2(f, g, subset, step, r, s["u0"], s["v0"], s["status"], method=method)
    nx = s["nx"]
    b = subset // 2 + r + 2
    k = np.arange(len(s["u0"]))
    x0 = (b + (k % nx) * step).astype(float)
    y0 = (b + (k // nx) * step).astype(float)
    truth = np.stack(d.displacement2(x0, y0), 1)
    ok = res["status"] == 0
    assert ok.mean() > 0.95
    e = np.abs(res["p"] - truth)[ok]
    assert e[:, [0, 6]].max() < 0.02 and e[:, [0, 6]].mean() < 0.005
    assert e[:, [1, 2, 7, 8]].mean() < 5e-4
    assert e[:, [3, 4, 5, 9, 10, 11]].mean() < 1e-4
    first = oracle.subpixel(f, g, subset, step, r, s["u0"], s["v0"], s["status"], method=method)
    e1 = np.abs(first["p"] - truth[:, [0, 1, 2, 6, 7, 8]])[first["status"] == 0]
    assert e[:, [1, 2, 7, 8]].mean() < 0.5 * e1[:, [1, 2, 4, 5]].mean()


@pytest.mark.parametrize("method", [oracle.ICGN, oracle.FANR])
def test_subpixel2_on_an_affine_field(affine1024, method):
    """Where the field is affine (noise sigma 2) the second-order terms come
    out near zero and u, v stay within the paper's usual 0.05 px of the
    imposed field, as the first-order refinement's do."""
    p = affine1024
    idx = np.arange(0, 36100, 97)
    s = oracle.integer_search(p.ref, p.defm, p.subset, p.step, p.radius, poi_idx=idx)
    r2 = oracle.subpixel2(p.ref, p.defm, p.subset, p.step, p.radius, s["u0"], s["v0"],
                          s["status"], method=method, poi_idx=idx)
    ok = r2["status"] == 0
    assert ok.mean() > 0.98
    b = p.subset // 2 + p.radius + 2
    x0 = (b + (idx % 190) * p.step).astype(float)
    y0 = (b + (idx // 190) * p.step).astype(float)
    gt = np.stack(p.deformation.displacement(x0, y0), 1)
    assert np.abs(r2["p"][ok][:, [0, 6]] - gt[ok][:, [0, 3]]).max() < 0.05
    assert np.abs(r2["p"][ok][:, [1, 2, 7, 8]] - gt[ok][:, [1, 2, 4, 5]]).mean() < 2e-3
    assert np.abs(r2["p"][ok][:, [3, 4, 5, 9, 10, 11]]).mean() < 5e-4


def test_zncc_at2_reduces_to_first_order_and_is_invariant():
    """Eq. 1 at a second-order shape with zero second derivatives is Eq. 1 at
    the first-order shape (independent sampling code), and it is invariant
    under g -> a g + b."""
    f, g = configs.tiny(34, 70, 70, 200, Rigid(0.4, 0.7), noise=1.0)
    nx, ny = oracle.grid(70, 70, 11, 7, 3)
    n = nx * ny
    rng = np.random.default_rng(6)
    p1 = np.column_stack([rng.uniform(-1, 1, n), rng.uniform(-0.02, 0.02, n),
                          rng.uniform(-0.02, 0.02, n), rng.uniform(-1, 1, n),
                          rng.uniform(-0.02, 0.02, n), rng.uniform(-0.02, 0.02, n)])
    p2 = np.zeros((n, 12))
    p2[:, [0, 1, 2, 6, 7, 8]] = p1
    c1 = oracle.zncc_at(f, g, 11, 7, 3, p1)
    c2 = oracle.zncc_at2(f, g, 11, 7, 3, p2)
    assert np.abs(c1 - c2).max() < 1e-12
    p2[:, [3, 4, 5, 9, 10, 11]] = rng.uniform(-3e-3, 3e-3, (n, 6))
    c3 = oracle.zncc_at2(f, g, 11, 7, 3, p2)
    c4 = oracle.zncc_at2(f, 1.7 * g.astype(np.float64) + 13.0, 11, 7, 3, p2)
    assert np.isfinite(c3).all() and np.abs(c3 - c4).max() < 1e-12
    assert np.abs(c3 - c2).max() > 1e-6  # the second-order terms move the samples
