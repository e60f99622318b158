"""GB300 digital-image-correlation hot path: thin Python binding of the C ABI.

The functions below carry the names of ``include/dic.h`` and only marshal
arguments (device pointers of torch tensors, sizes) into the CUDA library
``libdicgb.so``; every step of the computation runs in its kernels.  There is
no CPU fallback: if the library cannot be loaded, or no CUDA device is
present when work is requested, a ``RuntimeError`` is raised.

Method (Thoma & Ravi): brute-force ZNCC integer search (Eq. 1, Section 2.1)
then first-order IC-GN or Newton-Raphson sub-pixel refinement over bicubic
(or bilinear, Eq. 5) interpolation (Section 2.2, Table 2), for every POI of a
regular grid.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdicgb.so")

DIC_OK, DIC_ERR_ARG, DIC_ERR_CUDA, DIC_ERR_OOM, DIC_ERR_STATE, DIC_ERR_TIMEOUT, \
    DIC_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
DIC_ICGN, DIC_FANR = 0, 1
DIC_FORM_PLAIN_FP32, DIC_FORM_BF16TC = 0, 1
DIC_INTERP_BICUBIC, DIC_INTERP_BILINEAR = 0, 1
DIC_PEAK_FP32_FMA, DIC_PEAK_SMEM_ATOMIC_F32 = 0, 1
POI_OK, POI_ZERO_VAR_REF, POI_OUT_OF_BOUNDS, POI_MAX_ITER, POI_NONFINITE, POI_SINGULAR, \
    POI_ZERO_VAR_DEF = range(7)

_STATUS_NAMES = {0: "DIC_OK", -1: "DIC_ERR_ARG", -2: "DIC_ERR_CUDA", -3: "DIC_ERR_OOM",
                 -4: "DIC_ERR_STATE", -5: "DIC_ERR_TIMEOUT", -6: "DIC_ERR_UNSUPPORTED"}

_lock = threading.Lock()
_lib = None

P = C.c_void_p
i32 = C.c_int
f32 = C.c_float

class dic_pair_desc(C.Structure):
    _fields_ = [("ref_dev", P), ("def_dev", P), ("width", i32), ("height", i32),
                ("pitch_bytes", i32), ("subset_size", i32), ("grid_step", i32),
                ("search_radius", i32)]


class dic_batch_out(C.Structure):
    _fields_ = [(n, P) for n in ("u0", "v0", "zncc0", "status0", "u", "v", "ux", "uy", "vx", "vy",
                                 "zncc", "iters", "status")]


# name -> (restype, argtypes); mirrors include/dic.h
SIGNATURES = {
    "dic_version": (i32, []),
    "dic_create": (i32, [C.POINTER(P), i32, i32, i32, i32, f32, i32]),
    "dic_destroy": (None, [P]),
    "dic_last_error": (C.c_char_p, [P]),
    "dic_check": (i32, [P]),
    "dic_set_stream": (i32, [P, P]),
    "dic_set_form": (i32, [P, i32]),
    "dic_set_solve_precision": (i32, [P, i32]),
    "dic_set_interpolation": (i32, [P, i32]),
    "dic_set_pair": (i32, [P, P, P, i32, i32, i32]),
    "dic_set_pair_f32": (i32, [P, P, P, i32, i32, i32]),
    "dic_num_pois": (i32, [P, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]),
    "dic_znssd": (i32, [P, P, P, P]),
    "dic_set_pairs": (i32, [P, i32, C.POINTER(dic_pair_desc)]),
    "dic_batch_pois": (i32, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "dic_run_batch": (i32, [P, i32, C.POINTER(dic_batch_out)]),
    "dic_autotune": (i32, [P, i32, C.POINTER(dic_batch_out), C.POINTER(i32)]),
    "dic_set_batch_shape": (i32, [P, i32, i32]),
    "dic_stream_push": (i32, [P, P, i32, i32, i32, i32, C.POINTER(dic_batch_out)]),
    "dic_stream_flush": (i32, [P]),
    "dic_stream_reset": (i32, [P]),
    "dic_backward": (i32, [P, P, P, f32, P, P]),
    "dic_integer_search": (i32, [P, P, P, P, P]),
    "dic_pso_search": (i32, [P, i32, i32, i32, C.c_double, C.c_double, C.c_double, i32, i32,
                             P, P, P, P, P, P, P]),
    "dic_subpixel": (i32, [P, i32, P, P, P, P, P, P, P, P, P, P, P, P]),
    "dic_subpixel2": (i32, [P, i32, P, P, P, P, P, P, P]),
    "dic_measure_peak": (i32, [i32, P, C.POINTER(C.c_double)]),
    "dic_subpixel_noalloc": (i32, [P, P, i32, i32, i32, i32, i32, i32, i32, f32, i32, i32,
                                   P, P, P, P, P, P, P, P, P, P, P, P, P]),
}


class DICError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        super().__init__(f"{_STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def build() -> str:
    from . import _build
    return _build.build()


def lib():
    """Load libdicgb.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run build())")
            l = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(l, name)
                fn.restype = res
                fn.argtypes = args
            _lib = l
    return _lib


def _check(code: int, h=None):
    if code != DIC_OK:
        msg = lib().dic_last_error(h).decode() if h else ""
        raise DICError(code, msg)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return C.c_void_p(t)
    if not t.is_cuda:
        raise RuntimeError("expected a CUDA tensor (the library takes device pointers)")
    if not t.is_contiguous():
        raise RuntimeError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- C names
def dic_version() -> int:
    return lib().dic_version()


def dic_create(subset_size: int, grid_step: int, search_radius: int, shape_order: int = 1,
               conv_tol: float = 1e-3, max_iter: int = 50):
    h = P()
    _check(lib().dic_create(C.byref(h), subset_size, grid_step, search_radius, shape_order,
                            conv_tol, max_iter))
    _RADIUS[h.value] = search_radius
    return h


def dic_destroy(h) -> None:
    lib().dic_destroy(h)


def dic_last_error(h) -> str:
    return lib().dic_last_error(h).decode()


def dic_check(h) -> None:
    """Raise DICError(DIC_ERR_TIMEOUT) if a bounded device wait gave up."""
    _check(lib().dic_check(h), h)


def dic_set_stream(h, stream) -> None:
    ptr = stream if isinstance(stream, int) else (stream.cuda_stream if stream is not None else 0)
    _check(lib().dic_set_stream(h, C.c_void_p(ptr)), h)


def dic_set_form(h, form: int) -> None:
    _check(lib().dic_set_form(h, form), h)


def dic_set_solve_precision(h, bits: int) -> None:
    _check(lib().dic_set_solve_precision(h, bits), h)


def dic_set_interpolation(h, interp: int) -> None:
    _check(lib().dic_set_interpolation(h, interp), h)


def dic_set_pair(h, ref, defm, width: int | None = None, height: int | None = None,
                 pitch: int | None = None) -> None:
    if ref.dtype.itemsize != 1 or defm.dtype.itemsize != 1:
        raise RuntimeError("images must be 8-bit")
    hgt, wid = ref.shape[-2:]
    _check(lib().dic_set_pair(h, _ptr(ref), _ptr(defm), width or wid, height or hgt,
                              pitch or ref.stride(-2)), h)


def dic_set_pair_f32(h, ref, defm, width: int | None = None, height: int | None = None,
                     pitch: int | None = None) -> None:
    import torch
    if ref.dtype != torch.float32 or defm.dtype != torch.float32:
        raise RuntimeError("images must be float32")
    hgt, wid = ref.shape[-2:]
    _check(lib().dic_set_pair_f32(h, _ptr(ref), _ptr(defm), width or wid, height or hgt,
                                  pitch or ref.stride(-2)), h)


def dic_znssd(h, p6, loss_per_poi=None, loss_total=None) -> None:
    _check(lib().dic_znssd(h, _ptr(p6), _ptr(loss_per_poi), _ptr(loss_total)), h)


def dic_backward(h, p6, grad_loss, scale: float, dL_ddef, dL_dp=None) -> None:
    _check(lib().dic_backward(h, _ptr(p6), _ptr(grad_loss), scale, _ptr(dL_ddef), _ptr(dL_dp)),
           h)


def dic_set_pairs(h, pairs) -> None:
    """pairs: sequence of (ref, def) 8-bit device tensors or
    (ref, def, subset, step, radius) tuples."""
    arr = (dic_pair_desc * len(pairs))()
    for k, pr in enumerate(pairs):
        ref, defm = pr[0], pr[1]
        subset, step, radius = (pr[2], pr[3], pr[4]) if len(pr) > 2 else (0, 0, -1)
        hgt, wid = ref.shape[-2:]
        arr[k] = dic_pair_desc(_ptr(ref), _ptr(defm), wid, hgt, ref.stride(-2), subset, step,
                               radius)
    _check(lib().dic_set_pairs(h, len(pairs), arr), h)


def dic_batch_pois(h, n_pairs: int):
    total = C.c_int64()
    offs = (C.c_int64 * (n_pairs + 1))()
    _check(lib().dic_batch_pois(h, C.byref(total), offs), h)
    return total.value, list(offs)


def _batch_out(out: dict) -> dic_batch_out:
    return dic_batch_out(*[_ptr(out[k]) for k in ("u0", "v0", "zncc0", "status0", "u", "v",
                                                  "ux", "uy", "vx", "vy", "zncc", "iters",
                                                  "status")])


def dic_run_batch(h, method: int, out: dict) -> None:
    o = _batch_out(out)
    _check(lib().dic_run_batch(h, method, C.byref(o)), h)


def dic_autotune(h, method: int, out: dict) -> tuple[int, int]:
    o = _batch_out(out)
    chosen = (i32 * 2)()
    _check(lib().dic_autotune(h, method, C.byref(o), chosen), h)
    return chosen[0], chosen[1]


def dic_set_batch_shape(h, warps_per_cta: int, grid_mult: int) -> None:
    _check(lib().dic_set_batch_shape(h, warps_per_cta, grid_mult), h)


def dic_stream_push(h, frame, method: int = DIC_ICGN, out: dict | None = None) -> None:
    """Push the next 8-bit frame of a sequence; from the second frame on,
    ``out`` (see batch_outputs) receives the pair (previous frame, frame)."""
    if frame.dtype.itemsize != 1 or frame.is_floating_point():
        raise RuntimeError("frames must be 8-bit")
    hgt, wid = frame.shape[-2:]
    o = C.byref(_batch_out(out)) if out is not None else None
    _check(lib().dic_stream_push(h, _ptr(frame), wid, hgt, frame.stride(-2), method, o), h)


def dic_stream_flush(h) -> None:
    _check(lib().dic_stream_flush(h), h)


def dic_stream_reset(h) -> None:
    _check(lib().dic_stream_reset(h), h)


def batch_outputs(total: int, device):
    import torch
    out = {k: torch.empty(total, dtype=torch.int32, device=device) for k in ("u0", "v0", "iters")}
    for k in ("zncc0", "u", "v", "ux", "uy", "vx", "vy", "zncc"):
        out[k] = torch.empty(total, dtype=torch.float32, device=device)
    for k in ("status0", "status"):
        out[k] = torch.empty(total, dtype=torch.uint8, device=device)
    return out


def dic_num_pois(h) -> tuple[int, int, int]:
    n, nx, ny = i32(), i32(), i32()
    _check(lib().dic_num_pois(h, C.byref(n), C.byref(nx), C.byref(ny)), h)
    return n.value, nx.value, ny.value


def dic_integer_search(h, u0, v0, zncc0, status) -> None:
    _check(lib().dic_integer_search(h, _ptr(u0), _ptr(v0), _ptr(zncc0), _ptr(status)), h)


def dic_subpixel2(h, method, u0, v0, status0, p12, zncc, iters, status) -> None:
    """Second-order refinement (handle of shape order 2); p12 is a float32
    device tensor (n_pois, 12)."""
    _check(lib().dic_subpixel2(h, method, _ptr(u0), _ptr(v0), _ptr(status0), _ptr(p12),
                               _ptr(zncc), _ptr(iters), _ptr(status)), h)


def dic_pso_search(h, uniforms, u0, v0, zncc0, status, gens, evals, modified: bool = False,
                   c1: float = 2.0, c2: float = 2.0, vinit: float | None = None,
                   stop: tuple[int, int] = (995, 1000)) -> None:
    """Particle swarm integer search (Eqs. 2-4), or the modified swarm with
    the star search; ``uniforms`` is a float64 device tensor
    (n_pois, generations, particles, 4).  vinit defaults to radius / 4."""
    import torch
    if uniforms.dtype != torch.float64 or uniforms.dim() != 4 or uniforms.shape[3] != 4:
        raise RuntimeError("uniforms: float64 tensor (n_pois, generations, particles, 4)")
    n, _, _ = dic_num_pois(h)
    if uniforms.shape[0] != n:
        raise RuntimeError("uniforms: one row per POI")
    if vinit is None:
        vinit = _handle_radius(h) / 4.0
    _check(lib().dic_pso_search(h, int(bool(modified)), uniforms.shape[2], uniforms.shape[1],
                                float(c1), float(c2), float(vinit), int(stop[0]), int(stop[1]),
                                _ptr(uniforms), _ptr(u0), _ptr(v0), _ptr(zncc0), _ptr(status),
                                _ptr(gens), _ptr(evals)), h)


_RADIUS = {}


def _handle_radius(h) -> int:
    v = _RADIUS.get(h.value if hasattr(h, "value") else int(h))
    if v is None:
        raise RuntimeError("vinit needed: handle not created by dic_create of this binding")
    return v


def dic_subpixel(h, method, u0, v0, status0, u, v, ux, uy, vx, vy, zncc, iters, status) -> None:
    _check(lib().dic_subpixel(h, method, _ptr(u0), _ptr(v0), _ptr(status0), _ptr(u), _ptr(v),
                              _ptr(ux), _ptr(uy), _ptr(vx), _ptr(vy), _ptr(zncc), _ptr(iters),
                              _ptr(status)), h)


def dic_subpixel_noalloc(ref, defm, subset_size, grid_step, search_radius, method, u0, v0,
                         status0, u, v, ux, uy, vx, vy, zncc, iters, status, conv_tol=1e-3,
                         max_iter=50, solve_bits=32, stream=None, width=None, height=None,
                         pitch=None) -> None:
    """Sub-pixel refinement with no device allocation (images up to 65536
    pixels); see include/dic.h.  Both images are 8-bit with the same shape
    and row stride (the library reads both with ref's geometry)."""
    if ref.dtype.itemsize != 1 or defm.dtype.itemsize != 1 or ref.is_floating_point() \
            or defm.is_floating_point():
        raise RuntimeError("images must be 8-bit")
    if tuple(ref.shape) != tuple(defm.shape) or ref.stride(-2) != defm.stride(-2):
        raise RuntimeError("reference and deformed images need the same shape and row stride")
    hgt, wid = ref.shape[-2:]
    sp = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(lib().dic_subpixel_noalloc(_ptr(ref), _ptr(defm), width or wid, height or hgt,
                                      pitch or ref.stride(-2), subset_size, grid_step,
                                      search_radius, method, conv_tol, max_iter, solve_bits,
                                      _ptr(u0), _ptr(v0), _ptr(status0), _ptr(u), _ptr(v),
                                      _ptr(ux), _ptr(uy), _ptr(vx), _ptr(vy), _ptr(zncc),
                                      _ptr(iters), _ptr(status), C.c_void_p(sp)))


def dic_measure_peak(kind: int, stream=None) -> float:
    """Measured FP32 FMA flop/s (DIC_PEAK_FP32_FMA) or shared-memory float
    atomic adds/s (DIC_PEAK_SMEM_ATOMIC_F32) of the current device."""
    sp = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    r = C.c_double()
    _check(lib().dic_measure_peak(kind, C.c_void_p(sp), C.byref(r)))
    return r.value


# ------------------------------------------------------------ convenience
class DIC:
    """Handle owner with torch-allocated outputs (device memory and streams
    come from PyTorch; the computation is the library's)."""

    def __init__(self, subset: int, step: int, radius: int, tol: float = 1e-3,
                 max_iter: int = 50, solve_bits: int = 32, stream=None):
        self.h = dic_create(subset, step, radius, 1, tol, max_iter)
        self.subset, self.step, self.radius = subset, step, radius
        if solve_bits != 32:
            dic_set_solve_precision(self.h, solve_bits)
        if stream is not None:
            dic_set_stream(self.h, stream)
        self._pair = None

    def close(self):
        if self.h is not None:
            dic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_pair(self, ref, defm):
        dic_set_pair(self.h, ref, defm)
        self._pair = (ref, defm)  # keep the borrowed images alive
        return dic_num_pois(self.h)

    def integer_search(self, out=None):
        import torch
        n, _, _ = dic_num_pois(self.h)
        dev = self._pair[0].device
        if out is None:
            out = dict(u0=torch.empty(n, dtype=torch.int32, device=dev),
                       v0=torch.empty(n, dtype=torch.int32, device=dev),
                       zncc0=torch.empty(n, dtype=torch.float32, device=dev),
                       status0=torch.empty(n, dtype=torch.uint8, device=dev))
        if n:
            dic_integer_search(self.h, out["u0"], out["v0"], out["zncc0"], out["status0"])
        return out

    def subpixel(self, start, method=DIC_ICGN, out=None):
        import torch
        n, _, _ = dic_num_pois(self.h)
        dev = self._pair[0].device
        if out is None:
            out = {k: torch.empty(n, dtype=torch.float32, device=dev)
                   for k in ("u", "v", "ux", "uy", "vx", "vy", "zncc")}
            out["iters"] = torch.empty(n, dtype=torch.int32, device=dev)
            out["status"] = torch.empty(n, dtype=torch.uint8, device=dev)
        if n:
            dic_subpixel(self.h, method, start["u0"], start["v0"], start["status0"], out["u"],
                         out["v"], out["ux"], out["uy"], out["vx"], out["vy"], out["zncc"],
                         out["iters"], out["status"])
        return out

    def run(self, ref, defm, method=DIC_ICGN):
        self.set_pair(ref, defm)
        s = self.integer_search()
        r = self.subpixel(s, method)
        r.update(s)
        return r


# ------------------------------------------------------ differentiation
def _autograd():
    import torch

    class ZNSSD(torch.autograd.Function):
        """Summed ZNSSD of every subset at shapes ``p`` (n_pois x 6) over the
        float deformed image ``g``; gradients with respect to ``g`` (through
        the bicubic interpolation) and ``p`` come from the library's adjoint
        kernel.  ``f`` is the fixed reference image."""

        @staticmethod
        def forward(ctx, g, p, f, h):
            g = g.contiguous()
            p = p.contiguous()
            dic_set_pair_f32(h, f, g)
            total = torch.empty((), dtype=torch.float32, device=g.device)
            dic_znssd(h, p, None, total)
            ctx.save_for_backward(g, p, f)
            ctx.h = h
            return total

        @staticmethod
        def backward(ctx, grad_out):
            g, p, f = ctx.saved_tensors
            h = ctx.h
            dic_set_pair_f32(h, f, g)
            n = p.shape[0]
            w = grad_out.reshape(1).expand(n).contiguous()
            dg = torch.empty_like(g)
            dp = torch.empty_like(p)
            dic_backward(h, p, w, 1.0, dg, dp)
            return dg, dp, None, None

    return ZNSSD


_ZNSSD = None


def znssd_loss(g, p, f, h):
    """Differentiable summed ZNSSD (torch.autograd.Function over the C ABI)."""
    global _ZNSSD
    if _ZNSSD is None:
        _ZNSSD = _autograd()
    return _ZNSSD.apply(g, p, f, h)
