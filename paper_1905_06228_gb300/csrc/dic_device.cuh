// dic_device.cuh -- device helpers shared by the sub-pixel and adjoint
// kernels: warp reductions, the walk over a lane's subset points, bicubic
// evaluation from the float image, and the subset-in-image test.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dic {

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums over the warp of 8 values per lane, returned to every lane in v.
// Halving exchanges (xor 16, 8, 4) leave each lane one value's partial sum,
// two more exchanges complete it, and eight shuffles gather the eight sums:
// 17 shuffles instead of 40 for eight warp_sum calls.  The additions pair
// the lanes exactly as warp_sum does (xor 16, 8, 4, 2, 1), so every result
// equals warp_sum's bit for bit.
__device__ __forceinline__ void warp_sum8(float (&v)[8], int lane) {
  float w[4], x[2];
  {
    const bool up = lane & 16;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float send = up ? v[k] : v[k + 4];
      const float keep = up ? v[k + 4] : v[k];
      w[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
  }
  {
    const bool up = lane & 8;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float send = up ? w[k] : w[k + 2];
      const float keep = up ? w[k + 2] : w[k];
      x[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
  }
  const bool up = lane & 4;
  float y = (up ? x[1] : x[0]) + __shfl_xor_sync(0xffffffffu, up ? x[0] : x[1], 4);
  y += __shfl_xor_sync(0xffffffffu, y, 2);
  y += __shfl_xor_sync(0xffffffffu, y, 1);
  // lane l holds the sum of value 4 b16 + 2 b8 + b4 (its bits 16, 8, 4)
#pragma unroll
  for (int j = 0; j < 8; ++j)
    v[j] = __shfl_sync(0xffffffffu, y, ((j >> 2) & 1) * 16 + ((j >> 1) & 1) * 8 + (j & 1) * 4);
}

// Sum over the warp of 32 values per lane, scattered: lane l returns the
// sum of every lane's v[l] (five halving exchanges, 31 shuffles in all).
__device__ __forceinline__ float reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool up = lane & h;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const float send = up ? v[k] : v[k + h];
      const float keep = up ? v[k + h] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  return v[0];
}

// Keys (a = -1/2) weights of the taps -1, 0, 1, 2 at fractional offset t.
__device__ __forceinline__ void keys_weights(float t, float w[4]) {
  const float t2 = t * t, t3 = t2 * t;
  w[0] = fmaf(-0.5f, t3, fmaf(-0.5f, t, t2));
  w[1] = fmaf(1.5f, t3, fmaf(-2.5f, t2, 1.f));
  w[2] = fmaf(-1.5f, t3, fmaf(2.f, t2, 0.5f * t));
  w[3] = 0.5f * (t3 - t2);
}

// Derivatives dw/dt of the Keys weights.
__device__ __forceinline__ void keys_dweights(float t, float w[4]) {
  const float t2 = t * t;
  w[0] = fmaf(-1.5f, t2, fmaf(2.f, t, -0.5f));
  w[1] = fmaf(4.5f, t2, -5.f * t);
  w[2] = fmaf(-4.5f, t2, fmaf(4.f, t, 0.5f));
  w[3] = fmaf(1.5f, t2, -t);
}

// Bicubic (Keys a = -1/2) value of the image at (x + tx, y + ty), cell =
// y*W + x, from the 4x4 pixels y-1..y+2, x-1..x+2 (and, with DERIV, the
// derivatives along x and y).  Lanes of a warp interpolate consecutive
// pixels of a subset row, so each of the 16 loads of a warp covers one or
// two cache lines of a small, L1-resident footprint.
template <bool DERIV>
__device__ __forceinline__ float bicubic(const float* __restrict__ img, int W, size_t cell,
                                         float tx, float ty, float& gx, float& gy) {
  float wx[4], wy[4];
  keys_weights(tx, wx);
  keys_weights(ty, wy);
  const float* r = img + cell - W - 1;
  float row[4], drow[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const float p0 = __ldg(r), p1 = __ldg(r + 1), p2 = __ldg(r + 2), p3 = __ldg(r + 3);
    row[l] = fmaf(wx[3], p3, fmaf(wx[2], p2, fmaf(wx[1], p1, wx[0] * p0)));
    if (DERIV) {
      float dx[4];
      keys_dweights(tx, dx);
      drow[l] = fmaf(dx[3], p3, fmaf(dx[2], p2, fmaf(dx[1], p1, dx[0] * p0)));
    }
    r += W;
  }
  if (DERIV) {
    float dy[4];
    keys_dweights(ty, dy);
    gx = fmaf(wy[3], drow[3], fmaf(wy[2], drow[2], fmaf(wy[1], drow[1], wy[0] * drow[0])));
    gy = fmaf(dy[3], row[3], fmaf(dy[2], row[2], fmaf(dy[1], row[1], dy[0] * row[0])));
  }
  return fmaf(wy[3], row[3], fmaf(wy[2], row[2], fmaf(wy[1], row[1], wy[0] * row[0])));
}

// ---- packed FP32 (Blackwell f32x2: two FP32 operations per instruction).
// Each packed operation rounds every half exactly like its scalar form, so
// the helpers below give bitwise the results of keys_weights / bicubic /
// locate.
// Reciprocal of an FP64 pivot 2^-100 <= d < 2^100 with no FP64-pipe
// conversion (each FP64 instruction is costly on this GPU): an FP32 view of
// d made from its high word by integer moves (the exponent rebiased, the
// top 20 mantissa bits), its FP32 reciprocal, widened back to a double
// exactly by integer moves, then two Newton steps in FP64 (at least 20 ->
// 40 -> 80 correct bits).
__device__ __forceinline__ double rcp_pivot(double d) {
  const unsigned hi = (unsigned)__double2hiint(d);
  const float df = __uint_as_float((hi << 3) + 0x40000000u);  // exponent - 896
  const unsigned yb = __float_as_uint(__frcp_rn(df));
  double y = __hiloint2double((int)((yb >> 3) + (896u << 20)), (int)(yb << 29));
  y = fma(y, fma(-d, y, 1.0), y);
  return fma(y, fma(-d, y, 1.0), y);
}

// Pivot test of the FP64 sweeps: 2^-100 <= d < 2^100 (positive, finite and
// within rcp_pivot's range), from the high word with integer compares.
__device__ __forceinline__ bool pivot_ok(double d) {
  const int hk = __double2hiint(d);
  return hk >= 0x39B00000 && hk < 0x46300000;
}

__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// Keys weights of both axes at once: w[k] = (weight of tap k-1 along x at
// t.x, the same along y at t.y); same operation order as keys_weights.
__device__ __forceinline__ void keys_weights2(float2 t, float2 w[4]) {
  const float2 t2 = __fmul2_rn(t, t), t3 = __fmul2_rn(t2, t);
  w[0] = __ffma2_rn(dup2(-0.5f), t3, __ffma2_rn(dup2(-0.5f), t, t2));
  w[1] = __ffma2_rn(dup2(1.5f), t3, __ffma2_rn(dup2(-2.5f), t2, dup2(1.f)));
  w[2] = __ffma2_rn(dup2(-1.5f), t3, __ffma2_rn(dup2(2.f), t2, __fmul2_rn(dup2(0.5f), t)));
  w[3] = __fmul2_rn(dup2(0.5f), __ffma2_rn(t2, dup2(-1.f), t3));  // 0.5 (t3 - t2)
}

// Bicubic value at fractional offsets t of cell (as bicubic<false>): the
// four horizontal 4-tap sums run as two packed pairs of rows.
__device__ __forceinline__ float bicubic2(const float* __restrict__ img, int W, size_t cell,
                                          float2 t) {
  float2 w[4];
  keys_weights2(t, w);
  const float* r = img + cell - W - 1;
  float2 rr[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float* a = r + (size_t)(2 * h) * W;
    const float* b = a + W;
    float2 acc = __fmul2_rn(dup2(w[0].x), make_float2(__ldg(a), __ldg(b)));
    acc = __ffma2_rn(dup2(w[1].x), make_float2(__ldg(a + 1), __ldg(b + 1)), acc);
    acc = __ffma2_rn(dup2(w[2].x), make_float2(__ldg(a + 2), __ldg(b + 2)), acc);
    rr[h] = __ffma2_rn(dup2(w[3].x), make_float2(__ldg(a + 3), __ldg(b + 3)), acc);
  }
  return fmaf(w[3].y, rr[1].y, fmaf(w[2].y, rr[1].x, fmaf(w[1].y, rr[0].y, w[0].y * rr[0].x)));
}

// The same value from the tap quads of an 8-bit image: gq[y*W + x] holds
// the BF16 of g[y][x-1 .. x+2] (exact), so each stencil row is one 8-byte
// load; a BF16 becomes its float by a shift or a mask (integer ALU, no
// conversion).  Bitwise equal to bicubic2 on the float copy.
__device__ __forceinline__ float bicubic_q(const uint2* __restrict__ gq, int W, size_t cell,
                                           float2 t) {
  float2 w[4];
  keys_weights2(t, w);
  const uint2* r = gq + cell - W;
  float2 rr[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const uint2 qa = __ldg(r + (size_t)(2 * h) * W), qb = __ldg(r + (size_t)(2 * h + 1) * W);
    const float2 p0 = make_float2(__uint_as_float(qa.x << 16), __uint_as_float(qb.x << 16));
    const float2 p1 =
        make_float2(__uint_as_float(qa.x & 0xFFFF0000u), __uint_as_float(qb.x & 0xFFFF0000u));
    const float2 p2 = make_float2(__uint_as_float(qa.y << 16), __uint_as_float(qb.y << 16));
    const float2 p3 =
        make_float2(__uint_as_float(qa.y & 0xFFFF0000u), __uint_as_float(qb.y & 0xFFFF0000u));
    float2 acc = __fmul2_rn(dup2(w[0].x), p0);
    acc = __ffma2_rn(dup2(w[1].x), p1, acc);
    acc = __ffma2_rn(dup2(w[2].x), p2, acc);
    rr[h] = __ffma2_rn(dup2(w[3].x), p3, acc);
  }
  return fmaf(w[3].y, rr[1].y, fmaf(w[2].y, rr[1].x, fmaf(w[1].y, rr[0].y, w[0].y * rr[0].x)));
}

// Value and gradient of the bicubic patch from the tap quads (as
// bicubic<true> on the float copy, same operations and order: bitwise
// equal), for FA-NR's Jacobian.
__device__ __forceinline__ float bicubic_q_grad(const uint2* __restrict__ gq, int W, size_t cell,
                                                float tx, float ty, float& gx, float& gy) {
  float wx[4], wy[4], dx[4], dy[4];
  keys_weights(tx, wx);
  keys_weights(ty, wy);
  keys_dweights(tx, dx);
  keys_dweights(ty, dy);
  const uint2* r = gq + cell - W;
  float row[4], drow[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const uint2 q = __ldg(r + (size_t)l * W);
    const float p0 = __uint_as_float(q.x << 16), p1 = __uint_as_float(q.x & 0xFFFF0000u);
    const float p2 = __uint_as_float(q.y << 16), p3 = __uint_as_float(q.y & 0xFFFF0000u);
    row[l] = fmaf(wx[3], p3, fmaf(wx[2], p2, fmaf(wx[1], p1, wx[0] * p0)));
    drow[l] = fmaf(dx[3], p3, fmaf(dx[2], p2, fmaf(dx[1], p1, dx[0] * p0)));
  }
  gx = fmaf(wy[3], drow[3], fmaf(wy[2], drow[2], fmaf(wy[1], drow[1], wy[0] * drow[0])));
  gy = fmaf(dy[3], row[3], fmaf(dy[2], row[2], fmaf(dy[1], row[1], dy[0] * row[0])));
  return fmaf(wy[3], row[3], fmaf(wy[2], row[2], fmaf(wy[1], row[1], wy[0] * row[0])));
}

// The warp W(xi; p) of one shape, for packed point offsets (dx, dx), (dy, dy):
// local position l = (u + (1+ux) dx + uy dy, v + vx dx + (1+vy) dy), with
// the operation order of locate.  floor(l) comes from one round-down add of
// 1.5 * 2^23 (exact for |l| < 2^22: the sum's unit is 1), whose bits minus
// those of 1.5 * 2^23 are the integer floor, so no conversion instruction
// is issued.
struct WarpAffine {
  static constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
  static constexpr int kMagicBits = 0x4B400000;
  float2 a, b, o;
  int xm, ym;
  __device__ __forceinline__ WarpAffine(const float p[6], int x0, int y0)
      : a(make_float2(1.f + p[1], p[4])),
        b(make_float2(p[2], 1.f + p[5])),
        o(make_float2(p[0], p[3])),
        xm(x0 - kMagicBits),
        ym(y0 - kMagicBits) {}
  __device__ __forceinline__ size_t locate(float2 DX, float2 DY, int W, int H, float2& t) const {
    return locate_l(__ffma2_rn(b, DY, __ffma2_rn(a, DX, o)), W, H, t);
  }
  // the same from the local displacement l itself
  __device__ __forceinline__ size_t locate_l(float2 l, int W, int H, float2& t) const {
    const float2 r = __fadd2_rd(l, dup2(kMagic));
    const float2 fl = __fadd2_rn(r, dup2(-kMagic));
    t = __ffma2_rn(fl, dup2(-1.f), l);  // l - floor(l), one rounding as in locate
    int ix = __float_as_int(r.x) + xm, iy = __float_as_int(r.y) + ym;
    ix = min(max(ix, 1), W - 3);  // memory safety only; bounds are checked on p
    iy = min(max(iy, 1), H - 3);
    return (size_t)iy * W + ix;
  }
};

// Subset point walk with float offsets held as packed duplicates (dx, dx),
// (dy, dy) (small integers, exact), for the packed warp and sums.
struct PtWalk2 {
  float2 DX, DY;
  float ddx, ddy, fM, fS;
  __device__ __forceinline__ PtWalk2(int lane, int S, int M)
      : DX(dup2((float)(lane % S - M))),
        DY(dup2((float)(lane / S - M))),
        ddx((float)(32 % S)),
        ddy((float)(32 / S)),
        fM((float)M),
        fS((float)S) {}
  __device__ __forceinline__ void next() {
    DX = __fadd2_rn(DX, dup2(ddx));
    DY = __fadd2_rn(DY, dup2(ddy));
    if (DX.x > fM) {
      DX = __fadd2_rn(DX, dup2(-fS));
      DY = __fadd2_rn(DY, dup2(1.f));
    }
  }
};

// Bilinear grey level (Eq. 5, Section 2.2) at fractional offsets (x', y') =
// (tx, ty) of the cell whose top-left pixel is `cell`:
//   G = a00 + a10 x' + a01 y' + a11 x' y',
// the coefficients solving the linear system of the four surrounding pixels
// (a00 = p00, a10 = p10 - p00, a01 = p01 - p00, a11 = p11 - p10 - p01 + p00);
// with DERIV also the gradient of that patch (a10 + a11 y', a01 + a11 x').
template <bool DERIV>
__device__ __forceinline__ float bilinear(const float* __restrict__ img, int W, size_t cell,
                                          float tx, float ty, float& gx, float& gy) {
  const float p00 = __ldg(img + cell), p10 = __ldg(img + cell + 1);
  const float p01 = __ldg(img + cell + W), p11 = __ldg(img + cell + W + 1);
  const float a10 = p10 - p00, a01 = p01 - p00, a11 = (p11 - p10) - a01;
  if (DERIV) {
    gx = fmaf(a11, ty, a10);
    gy = fmaf(a11, tx, a01);
  }
  return fmaf(fmaf(a11, tx, a01), ty, fmaf(a10, tx, p00));
}

// Subset point walk of one lane: points i = lane, lane+32, ... in row-major
// (dy outer) order, with (dx, dy) advanced incrementally.
struct PtWalk {
  int dx, dy, ddx, ddy, S, M;
  __device__ __forceinline__ PtWalk(int lane, int S_, int M_) : S(S_), M(M_) {
    dy = lane / S - M;
    dx = lane % S - M;
    ddy = 32 / S;
    ddx = 32 % S;
  }
  __device__ __forceinline__ void next() {
    dx += ddx;
    dy += ddy;
    if (dx > M) {
      dx -= S;
      dy += 1;
    }
  }
};

// Location of a warped point: its cell (top-left pixel) and fractional offsets.
__device__ __forceinline__ size_t locate(const float p[6], int dx, int dy, int x0, int y0, int W,
                                         int H, float& tx, float& ty) {
  const float lx = fmaf(p[2], (float)dy, fmaf(1.f + p[1], (float)dx, p[0]));
  const float ly = fmaf(1.f + p[5], (float)dy, fmaf(p[4], (float)dx, p[3]));
  const float fx = floorf(lx), fy = floorf(ly);
  tx = lx - fx;
  ty = ly - fy;
  int ix = x0 + (int)fx, iy = y0 + (int)fy;
  ix = min(max(ix, 1), W - 3);  // memory safety only; bounds are checked on p
  iy = min(max(iy, 1), H - 3);
  return (size_t)iy * W + ix;
}

__device__ __forceinline__ bool corners_in(const float p[6], int x0, int y0, int M, int W, int H) {
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float cx = (c & 1) ? (float)M : -(float)M, cy = (c & 2) ? (float)M : -(float)M;
    const float lx = fmaf(p[2], cy, fmaf(1.f + p[1], cx, p[0]));
    const float ly = fmaf(1.f + p[5], cy, fmaf(p[4], cx, p[3]));
    const float x = (float)x0 + lx, y = (float)y0 + ly;
    ok = ok && (x >= 1.f) && (x < (float)(W - 2)) && (y >= 1.f) && (y < (float)(H - 2));
  }
  return ok;
}

// corners_in for a converged warp: lane l tests corner l & 3 with the same
// arithmetic, and the warp votes (one corner's instructions per lane
// instead of four).
__device__ __forceinline__ bool corners_in_warp(const float p[6], int x0, int y0, int M, int W,
                                                int H, int lane) {
  const int c = lane & 3;
  const float cx = (c & 1) ? (float)M : -(float)M, cy = (c & 2) ? (float)M : -(float)M;
  const float lx = fmaf(p[2], cy, fmaf(1.f + p[1], cx, p[0]));
  const float ly = fmaf(1.f + p[5], cy, fmaf(p[4], cx, p[3]));
  const float x = (float)x0 + lx, y = (float)y0 + ly;
  const bool ok = (x >= 1.f) && (x < (float)(W - 2)) && (y >= 1.f) && (y < (float)(H - 2));
  return __all_sync(0xffffffffu, ok);
}

// float of an exact 64-bit integer without the 64-bit conversion (which runs
// on the FP64 pipe): sign * (hi * 2^32 + lo) of the magnitude, relative
// error below 2^-23 for |v| < 2^56.
__device__ __forceinline__ float ll_to_float(long long v) {
  const unsigned long long a = (unsigned long long)(v < 0 ? -v : v);
  const float f = fmaf((float)(unsigned)(a >> 32), 4294967296.0f, (float)(unsigned)a);
  return v < 0 ? -f : f;
}

// ZNCC C = num / sqrt(Df Dg) of Eq. 1 from the exact integer sums
// (num = N Sab - Sa Sb, Df = N Saa - Sa^2, Dg = N Sbb - Sb^2), in FP32:
// three conversions, a product, a square root and a quotient, so the
// relative error stays below 1e-6.  Both integer-search forms report this.
__device__ __forceinline__ float zncc_of(long long num, long long df, long long dg) {
  return ll_to_float(num) / sqrtf(ll_to_float(df) * ll_to_float(dg));
}

}  // namespace dic
