"""FP64 CPU oracle of the DIC hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it.

The arithmetic lives in ``dic_oracle.c`` (plain C, FP64 / exact int64 sums);
this module compiles it with gcc and wraps it with ctypes.  Every function
follows the paper's method as stated in the C file's header:

* ``integer_search``  -- Eq. 1 (Section 2/2.1) with brute-force search.
* ``subpixel``        -- IC-GN / Newton-Raphson (Section 2.2, Table 2) with
                         a first-order warp and Keys bicubic interpolation.
* ``znssd``           -- summed ZNSSD and its hand-derived FP64 gradient.
* ``zncc_at``         -- Eq. 1 at given shapes (interpolated target subset).
* ``subpixel2``       -- both methods with a second-order (12-parameter) shape.
* ``bicubic``         -- the bicubic interpolant itself (Section 2.2).
* ``pso_search``      -- particle swarm integer search (Section 2.1, Eqs. 2-4)
                         and the modified swarm with the star search folded in.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dic_oracle.c")
_LIB = os.path.join(_HERE, "libdicoracle.so")
_lock = threading.Lock()
_lib = None

ST_OK, ST_ZERO_VAR_REF, ST_OUT_OF_BOUNDS, ST_MAX_ITER, ST_NONFINITE, ST_SINGULAR, \
    ST_ZERO_VAR_DEF = range(7)
ICGN, FANR = 0, 1
BICUBIC, BILINEAR = 0, 1  # interpolation of g: Keys cubic convolution, or Eq. 5


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2 -fopenmp, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-std=c11",
                               "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            i32, i64, dbl = C.c_int, C.c_int64, C.c_double
            lib.dico_grid.argtypes = [i32, i32, i32, i32, i32, P, P]
            lib.dico_grid.restype = i32
            lib.dico_integer_search.argtypes = [P, P, i32, i32, i32, i32, i32, i32, P, i64,
                                                i32, P, P, P, P]
            lib.dico_integer_search.restype = i32
            lib.dico_subpixel.argtypes = [P, P, i32, i32, i32, i32, i32, i32, i32, dbl, i32,
                                          P, i64, P, P, P, i32, P, P, P, P, P]
            lib.dico_subpixel.restype = i32
            lib.dico_subpixel_interp.argtypes = [P, P, i32, i32, i32, i32, i32, i32, i32, i32,
                                                 dbl, i32, P, i64, P, P, P, i32, P, P, P, P,
                                                 P]
            lib.dico_subpixel_interp.restype = i32
            lib.dico_bilinear.argtypes = [P, i32, i32, i32, dbl, dbl, P, P]
            lib.dico_bilinear.restype = dbl
            lib.dico_bicubic.argtypes = [P, i32, i32, i32, dbl, dbl, P, P]
            lib.dico_bicubic.restype = dbl
            lib.dico_znssd.argtypes = [P, P, i32, i32, i32, i32, i32, i32, P, i64, P, P, P, P, P]
            lib.dico_znssd.restype = i32
            lib.dico_subpixel2.argtypes = [P, P, i32, i32, i32, i32, i32, i32, i32, dbl, i32,
                                           P, i64, P, P, P, i32, P, P, P, P, P]
            lib.dico_subpixel2.restype = i32
            lib.dico_zncc_at2.argtypes = [P, P, i32, i32, i32, i32, i32, i32, P, i64, P, i32, P]
            lib.dico_zncc_at2.restype = i32
            lib.dico_compose2.argtypes = [P, P, P]
            lib.dico_compose2.restype = i32
            lib.dico_warp2_matrix.argtypes = [P, P]
            lib.dico_warp2_matrix.restype = None
            lib.dico_zncc_at.argtypes = [P, P, i32, i32, i32, i32, i32, i32, i32, P, i64, P,
                                         i32, P]
            lib.dico_zncc_at.restype = i32
            lib.dico_pso_search.argtypes = [P, P, i32, i32, i32, i32, i32, i32, P, i64, i32,
                                            i32, i32, dbl, dbl, dbl, i64, i64, P, i32, P, P,
                                            P, P, P, P, P]
            lib.dico_pso_search.restype = i32
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def default_threads() -> int:
    return os.cpu_count() or 1


def grid(width: int, height: int, subset: int, step: int, radius: int) -> tuple[int, int]:
    nx, ny = C.c_int(), C.c_int()
    if _load().dico_grid(width, height, subset, step, radius, C.byref(nx), C.byref(ny)):
        raise ValueError("bad grid arguments")
    return nx.value, ny.value


def _idx(poi_idx):
    if poi_idx is None:
        return None, -1
    a = np.ascontiguousarray(poi_idx, dtype=np.int64)
    return a, len(a)


def integer_search(f: np.ndarray, g: np.ndarray, subset: int, step: int, radius: int,
                   poi_idx=None, threads: int | None = None) -> dict:
    f = np.ascontiguousarray(f, np.uint8)
    g = np.ascontiguousarray(g, np.uint8)
    assert f.shape == g.shape and f.ndim == 2
    H, W = f.shape
    nx, ny = grid(W, H, subset, step, radius)
    idx, n = _idx(poi_idx)
    if idx is None:
        n = nx * ny
    u0 = np.zeros(n, np.int32)
    v0 = np.zeros(n, np.int32)
    zn = np.zeros(n, np.float64)
    st = np.zeros(n, np.uint8)
    rc = _load().dico_integer_search(_ptr(f), _ptr(g), W, H, W, subset, step, radius,
                                     _ptr(idx), n if idx is not None else -1,
                                     threads or default_threads(),
                                     _ptr(u0), _ptr(v0), _ptr(zn), _ptr(st))
    if rc:
        raise ValueError("oracle integer_search failed")
    return dict(u0=u0, v0=v0, zncc=zn, status=st, nx=nx, ny=ny)


def subpixel(f: np.ndarray, g: np.ndarray, subset: int, step: int, radius: int,
             u0, v0, status0, method: int = ICGN, tol: float = 1e-3, max_iter: int = 50,
             poi_idx=None, threads: int | None = None, trajectory: bool = False,
             interp: int = BICUBIC) -> dict:
    f = np.ascontiguousarray(f, np.float64)
    g = np.ascontiguousarray(g, np.float64)
    H, W = f.shape
    nx, ny = grid(W, H, subset, step, radius)
    idx, n = _idx(poi_idx)
    if idx is None:
        n = nx * ny
    u0 = np.ascontiguousarray(u0, np.int32)
    v0 = np.ascontiguousarray(v0, np.int32)
    status0 = np.ascontiguousarray(status0, np.uint8)
    assert len(u0) == n and len(v0) == n and len(status0) == n
    p = np.zeros((n, 6), np.float64)
    zn = np.zeros(n, np.float64)
    it = np.zeros(n, np.int32)
    st = np.zeros(n, np.uint8)
    traj = np.zeros((n, max_iter + 1, 6), np.float64) if trajectory else None
    rc = _load().dico_subpixel_interp(_ptr(f), _ptr(g), W, H, W, subset, step, radius,
                                      method, interp, tol, max_iter, _ptr(idx),
                                      n if idx is not None else -1, _ptr(u0), _ptr(v0),
                                      _ptr(status0), threads or default_threads(), _ptr(p),
                                      _ptr(zn), _ptr(it), _ptr(st), _ptr(traj))
    if rc:
        raise ValueError("oracle subpixel failed")
    out = dict(p=p, u=p[:, 0], ux=p[:, 1], uy=p[:, 2], v=p[:, 3], vx=p[:, 4], vy=p[:, 5],
               zncc=zn, iters=it, status=st, nx=nx, ny=ny)
    if trajectory:
        out["traj"] = traj
    return out


NAMES2 = ("u", "ux", "uy", "uxx", "uxy", "uyy", "v", "vx", "vy", "vxx", "vxy", "vyy")


def subpixel2(f: np.ndarray, g: np.ndarray, subset: int, step: int, radius: int, u0, v0,
              status0, method: int = ICGN, tol: float = 1e-3, max_iter: int = 50,
              poi_idx=None, threads: int | None = None, trajectory: bool = False) -> dict:
    """Sub-pixel refinement with the second-order (12-parameter) shape
    function, p = (u, ux, uy, uxx, uxy, uyy, v, vx, vy, vxx, vxy, vyy)."""
    f = np.ascontiguousarray(f, np.float64)
    g = np.ascontiguousarray(g, np.float64)
    H, W = f.shape
    nx, ny = grid(W, H, subset, step, radius)
    idx, n = _idx(poi_idx)
    if idx is None:
        n = nx * ny
    u0 = np.ascontiguousarray(u0, np.int32)
    v0 = np.ascontiguousarray(v0, np.int32)
    status0 = np.ascontiguousarray(status0, np.uint8)
    p = np.zeros((n, 12), np.float64)
    zn = np.zeros(n, np.float64)
    it = np.zeros(n, np.int32)
    st = np.zeros(n, np.uint8)
    traj = np.zeros((n, max_iter + 1, 12), np.float64) if trajectory else None
    rc = _load().dico_subpixel2(_ptr(f), _ptr(g), W, H, W, subset, step, radius, method, tol,
                                max_iter, _ptr(idx), n if idx is not None else -1, _ptr(u0),
                                _ptr(v0), _ptr(status0), threads or default_threads(), _ptr(p),
                                _ptr(zn), _ptr(it), _ptr(st), _ptr(traj))
    if rc:
        raise ValueError("oracle subpixel2 failed")
    out = dict(p=p, zncc=zn, iters=it, status=st, nx=nx, ny=ny)
    out.update({k: p[:, j] for j, k in enumerate(NAMES2)})
    if trajectory:
        out["traj"] = traj
    return out


def zncc_at2(f: np.ndarray, g: np.ndarray, subset: int, step: int, radius: int, p: np.ndarray,
             poi_idx=None, threads: int | None = None) -> np.ndarray:
    """Eq. 1 at second-order shapes p (n x 12), bicubic; NaN where the warped
    subset leaves the image or a subset is flat."""
    f = np.ascontiguousarray(f, np.float64)
    g = np.ascontiguousarray(g, np.float64)
    H, W = f.shape
    idx, n = _idx(poi_idx)
    if idx is None:
        nx, ny = grid(W, H, subset, step, radius)
        n = nx * ny
    p = np.ascontiguousarray(p, np.float64).reshape(n, 12)
    out = np.zeros(n, np.float64)
    if _load().dico_zncc_at2(_ptr(f), _ptr(g), W, H, W, subset, step, radius, _ptr(idx),
                             n if idx is not None else -1, _ptr(p), threads or default_threads(),
                             _ptr(out)):
        raise ValueError("oracle zncc_at2 failed")
    return out


def warp2_matrix(p) -> np.ndarray:
    p = np.ascontiguousarray(p, np.float64)
    out = np.zeros(36, np.float64)
    _load().dico_warp2_matrix(_ptr(p), _ptr(out))
    return out.reshape(6, 6)


def compose2(p, dp) -> np.ndarray:
    """W(p) W(dp)^-1 of two second-order shapes (the IC-GN update)."""
    p = np.ascontiguousarray(p, np.float64)
    dp = np.ascontiguousarray(dp, np.float64)
    out = np.zeros(12, np.float64)
    if _load().dico_compose2(_ptr(p), _ptr(dp), _ptr(out)):
        raise ValueError("singular update")
    return out


def zncc_at(f: np.ndarray, g: np.ndarray, subset: int, step: int, radius: int, p: np.ndarray,
            poi_idx=None, interp: int = BICUBIC, threads: int | None = None) -> np.ndarray:
    """Eq. 1 at the given shapes ``p`` (n x 6): reference subset against the
    interpolated target grey levels at the warped subset points.  NaN where
    the warped subset leaves the image or either subset is flat."""
    f = np.ascontiguousarray(f, np.float64)
    g = np.ascontiguousarray(g, np.float64)
    H, W = f.shape
    idx, n = _idx(poi_idx)
    if idx is None:
        nx, ny = grid(W, H, subset, step, radius)
        n = nx * ny
    p = np.ascontiguousarray(p, np.float64).reshape(n, 6)
    out = np.zeros(n, np.float64)
    rc = _load().dico_zncc_at(_ptr(f), _ptr(g), W, H, W, subset, step, radius, interp,
                              _ptr(idx), n if idx is not None else -1, _ptr(p),
                              threads or default_threads(), _ptr(out))
    if rc:
        raise ValueError("oracle zncc_at failed")
    return out


def bicubic(img: np.ndarray, x: float, y: float) -> tuple[float, float, float]:
    img = np.ascontiguousarray(img, np.float64)
    H, W = img.shape
    gx, gy = C.c_double(), C.c_double()
    v = _load().dico_bicubic(_ptr(img), W, H, W, float(x), float(y), C.byref(gx), C.byref(gy))
    return v, gx.value, gy.value


def bilinear(img: np.ndarray, x: float, y: float) -> tuple[float, float, float]:
    """Eq. 5 at (x, y): value and the gradient of the patch (NaN outside)."""
    img = np.ascontiguousarray(img, np.float64)
    H, W = img.shape
    gx, gy = C.c_double(), C.c_double()
    v = _load().dico_bilinear(_ptr(img), W, H, W, float(x), float(y), C.byref(gx), C.byref(gy))
    return v, gx.value, gy.value


def znssd(f: np.ndarray, g: np.ndarray, subset: int, step: int, radius: int, p: np.ndarray,
          poi_idx=None, grad: bool = True, per_poi: bool = False):
    """Summed ZNSSD at shape parameters ``p`` (n x 6) and, optionally, its
    gradient with respect to every pixel of ``g`` and every row of ``p``
    (and the per-POI losses)."""
    f = np.ascontiguousarray(f, np.float64)
    g = np.ascontiguousarray(g, np.float64)
    H, W = f.shape
    idx, n = _idx(poi_idx)
    if idx is None:
        nx, ny = grid(W, H, subset, step, radius)
        n = nx * ny
    p = np.ascontiguousarray(p, np.float64).reshape(n, 6)
    loss = C.c_double()
    dg = np.zeros((H, W), np.float64) if grad else None
    dp = np.zeros((n, 6), np.float64) if grad else None
    lp = np.zeros(n, np.float64) if per_poi else None
    rc = _load().dico_znssd(_ptr(f), _ptr(g), W, H, W, subset, step, radius, _ptr(idx),
                            n if idx is not None else -1, _ptr(p), C.byref(loss), _ptr(lp),
                            _ptr(dg), _ptr(dp))
    if rc:
        raise ValueError("oracle znssd failed")
    out = (loss.value, dg, dp) if grad else (loss.value,)
    if per_poi:
        out = out + (lp,)
    return out if len(out) > 1 else out[0]


def pso_search(f: np.ndarray, g: np.ndarray, subset: int, step: int, radius: int,
               rand: np.ndarray, modified: bool = False, c1: float = 2.0, c2: float = 2.0,
               vinit: float | None = None, stop: tuple[int, int] = (995, 1000),
               poi_idx=None, threads: int | None = None, trace: bool = False) -> dict:
    """Particle swarm integer search (Eqs. 2-4) over the same window as the
    brute-force search.  ``rand`` holds the swarm's uniforms, shape
    (POIs, generations, particles, 4): generation 0 draws the start position
    and velocity, generation t >= 1 the r1 (x, y) and r2 (x, y) of Eq. 2.
    ``stop`` = (n, d) ends a POI's swarm once its best C >= n / d.
    ``vinit`` (pixels, default radius / 4) scales the start velocity.
    With ``trace`` the result holds ``trace[k, t, i] = (px, py, vx, vy, qx, qy,
    bx, by)``: particle i's position and velocity when generation t is
    evaluated, its nearest pixel and its best pixel afterwards (NaN for
    generations not run)."""
    f = np.ascontiguousarray(f, np.uint8)
    g = np.ascontiguousarray(g, np.uint8)
    assert f.shape == g.shape and f.ndim == 2
    H, W = f.shape
    nx, ny = grid(W, H, subset, step, radius)
    idx, n = _idx(poi_idx)
    if idx is None:
        n = nx * ny
    rand = np.ascontiguousarray(rand, np.float64)
    assert rand.ndim == 4 and rand.shape[0] == n and rand.shape[3] == 4
    gmax, particles = rand.shape[1], rand.shape[2]
    if vinit is None:
        vinit = radius / 4.0
    u0 = np.zeros(n, np.int32)
    v0 = np.zeros(n, np.int32)
    zn = np.zeros(n, np.float64)
    st = np.zeros(n, np.uint8)
    gens = np.zeros(n, np.int32)
    evals = np.zeros(n, np.int32)
    tr = np.full((n, gmax, particles, 8), np.nan) if trace else None
    rc = _load().dico_pso_search(_ptr(f), _ptr(g), W, H, W, subset, step, radius, _ptr(idx),
                                 n if idx is not None else -1, int(bool(modified)), particles,
                                 gmax, float(c1), float(c2), float(vinit), int(stop[0]),
                                 int(stop[1]), _ptr(rand), threads or default_threads(),
                                 _ptr(u0), _ptr(v0), _ptr(zn), _ptr(st), _ptr(gens),
                                 _ptr(evals), _ptr(tr))
    if rc:
        raise ValueError("oracle pso_search failed (%d)" % rc)
    out = dict(u0=u0, v0=v0, zncc=zn, status=st, generations=gens, evaluations=evals,
               nx=nx, ny=ny)
    if trace:
        out["trace"] = tr
    return out
