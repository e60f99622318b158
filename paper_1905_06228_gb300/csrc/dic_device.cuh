// dic_device.cuh -- device helpers shared by the sub-pixel and adjoint
// kernels: warp reductions, the walk over a lane's subset points, bicubic
// evaluation from the coefficient table, and the subset-in-image test.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dic {

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Bicubic value (and optionally derivatives) from one table cell.
// The table is four planes of float4: plane n holds, per cell, the
// coefficients of ty^n (1, tx, tx^2, tx^3).  Lanes of a warp interpolate
// consecutive pixels of a subset row, so each plane load of a warp covers
// contiguous cache lines.
template <bool DERIV>
__device__ __forceinline__ float bicubic(const float4* __restrict__ lut, size_t plane,
                                         size_t cell, float tx, float ty, float& gx, float& gy) {
  const float4 a0 = __ldg(lut + cell), a1 = __ldg(lut + plane + cell),
               a2 = __ldg(lut + 2 * plane + cell), a3 = __ldg(lut + 3 * plane + cell);
  const float r0 = fmaf(fmaf(fmaf(a0.w, tx, a0.z), tx, a0.y), tx, a0.x);
  const float r1 = fmaf(fmaf(fmaf(a1.w, tx, a1.z), tx, a1.y), tx, a1.x);
  const float r2 = fmaf(fmaf(fmaf(a2.w, tx, a2.z), tx, a2.y), tx, a2.x);
  const float r3 = fmaf(fmaf(fmaf(a3.w, tx, a3.z), tx, a3.y), tx, a3.x);
  if (DERIV) {
    const float d0 = fmaf(fmaf(3.f * a0.w, tx, 2.f * a0.z), tx, a0.y);
    const float d1 = fmaf(fmaf(3.f * a1.w, tx, 2.f * a1.z), tx, a1.y);
    const float d2 = fmaf(fmaf(3.f * a2.w, tx, 2.f * a2.z), tx, a2.y);
    const float d3 = fmaf(fmaf(3.f * a3.w, tx, 2.f * a3.z), tx, a3.y);
    gx = fmaf(fmaf(fmaf(d3, ty, d2), ty, d1), ty, d0);
    gy = fmaf(fmaf(3.f * r3, ty, 2.f * r2), ty, r1);
  }
  return fmaf(fmaf(fmaf(r3, ty, r2), ty, r1), ty, r0);
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

// Location of a warped point: table cell and fractional offsets.
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

// Keys (a = -1/2) weights of the taps -1, 0, 1, 2 at fractional offset t.
__device__ __forceinline__ void keys_weights(float t, float w[4]) {
  const float t2 = t * t, t3 = t2 * t;
  w[0] = -0.5f * t3 + t2 - 0.5f * t;
  w[1] = 1.5f * t3 - 2.5f * t2 + 1.f;
  w[2] = -1.5f * t3 + 2.f * t2 + 0.5f * t;
  w[3] = 0.5f * t3 - 0.5f * t2;
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
