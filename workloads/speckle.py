"""Seeded synthetic speckle image pairs (input generation only).

This module produces the inputs that both the CUDA path and the CPU oracle
consume.  It holds none of the correlation method's arithmetic: no ZNCC, no
interpolation kernel, no warp update.  It renders an analytic intensity field
(a sum of Gaussian speckles on a constant background) at pixel centres, once
in the reference frame and once in the deformed frame through the inverse of
a known deformation map, then adds Gaussian noise, clips to [0, 255] and
rounds half-to-even to 8-bit grey levels.

The paper's two test sets (a tensile specimen series and a public DIC image
series, Section 3) are not available; these renders stand in for them with
the image sizes, speckle densities and deformations of the benchmark
workloads listed in ``workloads.configs``.

Intensity model (one speckle k with centre c_k, radius r_k, peak A_k)::

    I(x) = 20 + sum_k A_k * exp(-|x - c_k|^2 / r_k^2) * [|x - c_k| < 4 r_k]

The deformed image is g(x') = I(phi^-1(x')) for a deformation phi mapping
reference coordinates to deformed coordinates (x' = x + u(x)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BACKGROUND = 20.0
CUTOFF = 4.0  # speckle support radius in units of r_k


def _sin(x):
    return x.sin() if hasattr(x, "sin") and not isinstance(x, np.ndarray) else np.sin(x)


def _cos(x):
    return x.cos() if hasattr(x, "cos") and not isinstance(x, np.ndarray) else np.cos(x)


# ---------------------------------------------------------------------------
# Deformation maps.  Each provides forward(x, y) -> (x', y') and
# inverse(x', y') -> (x, y) on float64 arrays, plus the exact displacement
# and displacement gradient at reference points (ground truth for tests).
# ---------------------------------------------------------------------------
@dataclass
class Rigid:
    tx: float
    ty: float

    def forward(self, x, y):
        return x + self.tx, y + self.ty

    def inverse(self, xp, yp):
        return xp - self.tx, yp - self.ty

    def displacement(self, x, y):
        x = np.asarray(x, np.float64)
        y = np.asarray(y, np.float64)
        z = np.zeros(np.broadcast(x, y).shape)
        return (z + self.tx, z + self.ty, z, z, z, z)


@dataclass
class Affine:
    """x' = c + Rot(theta) diag(1+exx, 1+eyy) (x - c) + t, c = image centre."""
    exx: float
    eyy: float
    theta_deg: float
    tx: float
    ty: float
    cx: float
    cy: float

    def _mat(self):
        th = math.radians(self.theta_deg)
        c, s = math.cos(th), math.sin(th)
        a = np.array([[c * (1 + self.exx), -s * (1 + self.eyy)],
                      [s * (1 + self.exx), c * (1 + self.eyy)]], np.float64)
        return a

    def forward(self, x, y):
        a = self._mat()
        dx, dy = x - self.cx, y - self.cy
        return (self.cx + a[0, 0] * dx + a[0, 1] * dy + self.tx,
                self.cy + a[1, 0] * dx + a[1, 1] * dy + self.ty)

    def inverse(self, xp, yp):
        ai = np.linalg.inv(self._mat())
        dx, dy = xp - self.cx - self.tx, yp - self.cy - self.ty
        return (self.cx + ai[0, 0] * dx + ai[0, 1] * dy,
                self.cy + ai[1, 0] * dx + ai[1, 1] * dy)

    def displacement(self, x, y):
        x = np.asarray(x, np.float64)
        y = np.asarray(y, np.float64)
        xp, yp = self.forward(x, y)
        a = self._mat()
        z = np.zeros(np.broadcast(x, y).shape)
        return (xp - x, z + a[0, 0] - 1, z + a[0, 1],
                yp - y, z + a[1, 0], z + a[1, 1] - 1)


@dataclass
class Sinusoidal:
    """u = au sin(2 pi y / ly) + tx,  v = av cos(2 pi x / lx) + ty (reference frame)."""
    au: float = 2.0
    ly: float = 128.0
    av: float = 1.5
    lx: float = 96.0
    tx: float = 0.0
    ty: float = 0.0

    def forward(self, x, y):
        return (x + self.au * np.sin(2 * np.pi * y / self.ly) + self.tx,
                y + self.av * np.cos(2 * np.pi * x / self.lx) + self.ty)

    def inverse(self, xp, yp, iters: int = 16):
        # Fixed point x = x' - u(x); the map u has Lipschitz constant
        # max(2 pi au / ly, 2 pi av / lx) ~ 0.098, so 16 sweeps reach 1e-16 px.
        x = xp - self.tx
        y = yp - self.ty
        for _ in range(iters):
            x = xp - self.tx - self.au * _sin(2 * np.pi * y / self.ly)
            y = yp - self.ty - self.av * _cos(2 * np.pi * x / self.lx)
        return x, y

    def displacement(self, x, y):
        x = np.asarray(x, np.float64)
        y = np.asarray(y, np.float64)
        z = np.zeros(np.broadcast(x, y).shape)
        u = self.au * np.sin(2 * np.pi * y / self.ly) + self.tx + z
        v = self.av * np.cos(2 * np.pi * x / self.lx) + self.ty + z
        uy = self.au * 2 * np.pi / self.ly * np.cos(2 * np.pi * y / self.ly) + z
        vx = -self.av * 2 * np.pi / self.lx * np.sin(2 * np.pi * x / self.lx) + z
        return (u, z, uy, v, vx, z)


@dataclass
class Quadratic:
    """x' = x + u, y' = y + v with u, v quadratic in (X, Y) = (x - cx, y - cy):
    u = cu[0] + cu[1] X + cu[2] Y + cu[3] X^2/2 + cu[4] X Y + cu[5] Y^2/2
    (v likewise with cv), the field a second-order subset shape reproduces."""
    cu: tuple
    cv: tuple
    cx: float
    cy: float

    @staticmethod
    def _q(c, X, Y):
        return c[0] + c[1] * X + c[2] * Y + 0.5 * c[3] * X * X + c[4] * X * Y + 0.5 * c[5] * Y * Y

    def forward(self, x, y):
        X, Y = x - self.cx, y - self.cy
        return x + self._q(self.cu, X, Y), y + self._q(self.cv, X, Y)

    def inverse(self, xp, yp, iters: int = 60):
        # fixed point x = x' - u(x); the map's Jacobian stays well below 1 on
        # the images it is used for
        x, y = xp, yp
        for _ in range(iters):
            X, Y = x - self.cx, y - self.cy
            x = xp - self._q(self.cu, X, Y)
            y = yp - self._q(self.cv, X, Y)
        return x, y

    def displacement2(self, x, y):
        """The 12 second-order shape parameters at reference points (x, y):
        (u, ux, uy, uxx, uxy, uyy, v, vx, vy, vxx, vxy, vyy)."""
        x = np.asarray(x, np.float64)
        y = np.asarray(y, np.float64)
        X, Y = x - self.cx, y - self.cy
        out = []
        for c in (self.cu, self.cv):
            out += [self._q(c, X, Y), c[1] + c[3] * X + c[4] * Y, c[2] + c[4] * X + c[5] * Y,
                    c[3] + 0 * X, c[4] + 0 * X, c[5] + 0 * X]
        return tuple(out)


@dataclass
class SpeckleSet:
    cx: np.ndarray
    cy: np.ndarray
    r: np.ndarray
    amp: np.ndarray


def draw_speckles(rng: np.random.Generator, n: int, width: int, height: int,
                  pad: float, r_range=(2.5, 4.0), amp_range=(60.0, 200.0)) -> SpeckleSet:
    """Uniform centres over the image padded by ``pad`` px on every side."""
    cx = rng.uniform(-pad, width - 1 + pad, n)
    cy = rng.uniform(-pad, height - 1 + pad, n)
    r = rng.uniform(*r_range, n)
    amp = rng.uniform(*amp_range, n)
    return SpeckleSet(cx, cy, r, amp)


def _render(sp: SpeckleSet, width: int, height: int, inverse, forward,
            chunk: int = 4096) -> np.ndarray:
    """Evaluate the analytic field at every pixel centre of the target frame.

    ``inverse`` maps target-frame pixel coordinates to reference coordinates;
    ``forward`` maps speckle centres into the target frame to find their
    footprints.  Returns float64 (height, width).  The sums run in torch
    (float64; on the GPU when one is present), only to make large renders
    fast: the field is the same at any summation order up to rounding.
    """
    import torch
    dev = torch.device("cuda" if torch.cuda.is_available() else "cpu")
    img = torch.full((height * width,), BACKGROUND, dtype=torch.float64, device=dev)
    if len(sp.cx) == 0:
        return img.reshape(height, width).cpu().numpy()
    # footprint half size: support radius 4 r_max plus a margin for the local
    # stretch of the map (strains and rotations here are below 5 %)
    h = int(math.ceil(CUTOFF * float(sp.r.max()) * 1.1)) + 2
    off = torch.arange(-h, h + 1, device=dev)
    oy, ox = torch.meshgrid(off, off, indexing="ij")
    oy = oy.reshape(-1)
    ox = ox.reshape(-1)
    pcx, pcy = forward(sp.cx, sp.cy)
    # reference coordinates of every target pixel, evaluated once
    gy, gx = torch.meshgrid(torch.arange(height, dtype=torch.float64, device=dev),
                            torch.arange(width, dtype=torch.float64, device=dev), indexing="ij")
    inv_x, inv_y = inverse(gx, gy)
    inv_x = inv_x.reshape(-1).contiguous()
    inv_y = inv_y.reshape(-1).contiguous()
    del gx, gy
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64)).to(dev)
    cx, cy, r, amp = t(sp.cx), t(sp.cy), t(sp.r), t(sp.amp)
    qx = torch.from_numpy(np.rint(pcx).astype(np.int64)).to(dev)
    qy = torch.from_numpy(np.rint(pcy).astype(np.int64)).to(dev)
    for s in range(0, len(sp.cx), chunk):
        e = min(s + chunk, len(sp.cx))
        px = qx[s:e, None] + ox[None, :]
        py = qy[s:e, None] + oy[None, :]
        ok = (px >= 0) & (px < width) & (py >= 0) & (py < height)
        k0, k1 = torch.nonzero(ok, as_tuple=True)
        idx = py[k0, k1] * width + px[k0, k1]
        ks = k0 + s
        dx = inv_x[idx] - cx[ks]
        dy = inv_y[idx] - cy[ks]
        d2 = dx * dx + dy * dy
        rr = r[ks]
        val = amp[ks] * torch.exp(-d2 / (rr * rr))
        val = torch.where(d2 < (CUTOFF * rr) ** 2, val, torch.zeros_like(val))
        img.index_add_(0, idx, val)
    return img.reshape(height, width).cpu().numpy()


def quantise(img: np.ndarray) -> np.ndarray:
    """Clip to [0, 255] and round half-to-even to uint8."""
    return np.rint(np.clip(img, 0.0, 255.0)).astype(np.uint8)


@dataclass
class Pair:
    ref: np.ndarray          # uint8 (H, W)
    defm: np.ndarray         # uint8 (H, W)
    deformation: object      # map with forward/inverse/displacement
    subset: int
    step: int
    radius: int
    meta: dict = field(default_factory=dict)


def render_pair(seed: int, width: int, height: int, n_speckles: int, deformation,
                noise_sigma: float = 0.0, pad: float | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Render (reference, deformed) uint8 images with a PCG64 stream of ``seed``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if pad is None:
        pad = 4 * 4.0 + 8.0
    sp = draw_speckles(rng, n_speckles, width, height, pad)
    ident = (lambda x, y: (x, y))
    f = _render(sp, width, height, ident, ident)
    g = _render(sp, width, height, deformation.inverse, deformation.forward)
    if noise_sigma > 0:
        f = f + rng.normal(0.0, noise_sigma, f.shape)
        g = g + rng.normal(0.0, noise_sigma, g.shape)
    return quantise(f), quantise(g)


def render_sequence(seed: int, width: int, height: int, n_speckles: int, deformations,
                    noise_sigma: float = 0.0, pad: float | None = None) -> list[np.ndarray]:
    """Render a frame sequence of one speckle pattern: frame k is the field
    seen through ``deformations[k]`` (None = undeformed), with its own
    noise draw; one PCG64 stream of ``seed`` for speckles and noise."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if pad is None:
        pad = 4 * 4.0 + 8.0
    sp = draw_speckles(rng, n_speckles, width, height, pad)
    ident = (lambda x, y: (x, y))
    frames = []
    for d in deformations:
        img = _render(sp, width, height, d.inverse if d else ident, d.forward if d else ident)
        if noise_sigma > 0:
            img = img + rng.normal(0.0, noise_sigma, img.shape)
        frames.append(quantise(img))
    return frames
