// k_adjoint.cu -- summed ZNSSD of the subsets and its hand-written adjoint.
//
// For POI k with shape p_k (held fixed: the gradient does not go through the
// iterative solver) and subset points i:
//
//   ft_i = (f_i - fbar)/df,  gt_i = (g(W(xi_i; p_k)) - gbar)/dg,
//   L_k  = sum_i (ft_i - gt_i)^2                       (ZNSSD = 2 - 2 C, Eq. 1)
//
// with g read through the bicubic interpolant (Section 2.2).  With
// C = sum ft gt, the derivative with respect to the interpolated samples is
//
//   dL_k/dg_i = (2/dg) (C gt_i - ft_i),
//
// which reaches every pixel of the deformed image through the transposed
// bicubic stencil (16 Keys weights per sample) and every shape parameter
// through dg_i/dp = grad g(W) dW/dp = [gx, gx dx, gx dy, gy, gy dx, gy dy].
//
// One warp per POI.  Pass 1 samples g for gbar, dg and C; pass 2 re-samples
// value and derivatives, accumulates L_k and dL/dp, and scatters dL/dg_i.
// Scatter goes to a per-warp shared-memory tile covering the warped subset
// (one shared atomic per stencil tap), then the tile is added to global
// memory once; if the footprint does not fit the tile the taps go to global
// memory directly.  A POI whose subset is out of bounds or flat contributes
// nothing.
#include "dic_device.cuh"
#include "dic_internal.cuh"

namespace dic {
namespace {

constexpr int kWarps = 4;
constexpr int kTile = 48;  // side of the per-warp scatter tile (pixels)

template <typename TP>
__device__ __forceinline__ float ref_px(const AdjointParams& p, size_t i);
template <>
__device__ __forceinline__ float ref_px<uint8_t>(const AdjointParams& p, size_t i) {
  return (float)p.ref[i];
}
template <>
__device__ __forceinline__ float ref_px<float>(const AdjointParams& p, size_t i) {
  return p.ref_f32[i];
}

template <typename TP>
__global__ void __launch_bounds__(32 * kWarps) adjoint_kernel(const AdjointParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t poi = (int64_t)blockIdx.x * kWarps + wid;
  if (poi >= p.n_pois) return;
  const int S = p.S, M = p.M, N = S * S, W = p.W, H = p.H;
  float* sfc = reinterpret_cast<float*>(smem) + (size_t)wid * N;
  float* tile = reinterpret_cast<float*>(smem + (size_t)kWarps * N * sizeof(float)) +
                (size_t)wid * kTile * kTile;
  const int x0 = M + p.R + 2 + (int)(poi % p.nx) * p.step;
  const int y0 = M + p.R + 2 + (int)(poi / p.nx) * p.step;
  float prm[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) prm[k] = p.p6[poi * 6 + k];

  auto finish_empty = [&]() {
    if (lane == 0) {
      if (p.loss_poi) p.loss_poi[poi] = 0.f;
      if (p.backward && p.dL_dp)
        for (int k = 0; k < 6; ++k) p.dL_dp[poi * 6 + k] = 0.f;
    }
  };
  if (!corners_in(prm, x0, y0, M, W, H)) {
    finish_empty();
    return;
  }
  // reference subset
  float fsum = 0.f;
  {
    PtWalk w(lane, S, M);
    for (int i = lane; i < N; i += 32, w.next()) {
      const float f = ref_px<TP>(p, (size_t)(y0 + w.dy) * p.pitch + (x0 + w.dx));
      sfc[i] = f;
      fsum += f;
    }
  }
  fsum = warp_sum(fsum);
  const float fbar = fsum / (float)N;
  float q = 0.f;
  for (int i = lane; i < N; i += 32) {
    const float fc = sfc[i] - fbar;
    sfc[i] = fc;
    q = fmaf(fc, fc, q);
  }
  q = warp_sum(q);
  const float df = sqrtf(q);
  // pass 1: gbar, dg, C (shift c = fbar keeps the sums well conditioned)
  const float c = fbar;
  float s0 = 0.f, s1 = 0.f, sfg = 0.f;
  {
    PtWalk w(lane, S, M);
    for (int i = lane; i < N; i += 32, w.next()) {
      float tx, ty, gx, gy;
      const size_t cell = locate(prm, w.dx, w.dy, x0, y0, W, H, tx, ty);
      const float d = bicubic<false>(p.gimg, W, cell, tx, ty, gx, gy) - c;
      s0 += d;
      s1 = fmaf(d, d, s1);
      sfg = fmaf(sfc[i], d, sfg);
    }
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  sfg = warp_sum(sfg);
  const float gm = s0 / (float)N;  // gbar - c
  const float dg = sqrtf(fmaxf(s1 - s0 * gm, 0.f));
  if (!(df > 0.f) || !(dg > 0.f)) {
    finish_empty();
    return;
  }
  const float C = sfg / (df * dg);
  const float idf = 1.f / df, idg = 1.f / dg;
  float wgt = 0.f;
  if (p.backward) wgt = p.scale * (p.grad_loss ? p.grad_loss[poi] : 1.f);

  // footprint of the warped subset for the scatter tile
  int tx0 = 0, ty0 = 0;
  bool use_tile = false;
  if (p.backward) {
    float xmin = 1e30f, xmax = -1e30f, ymin = 1e30f, ymax = -1e30f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float cx = (k & 1) ? (float)M : -(float)M, cy = (k & 2) ? (float)M : -(float)M;
      const float lx = fmaf(prm[2], cy, fmaf(1.f + prm[1], cx, prm[0]));
      const float ly = fmaf(1.f + prm[5], cy, fmaf(prm[4], cx, prm[3]));
      xmin = fminf(xmin, lx);
      xmax = fmaxf(xmax, lx);
      ymin = fminf(ymin, ly);
      ymax = fmaxf(ymax, ly);
    }
    tx0 = x0 + (int)floorf(xmin) - 2;
    ty0 = y0 + (int)floorf(ymin) - 2;
    const int tw = x0 + (int)floorf(xmax) + 3 - tx0, th = y0 + (int)floorf(ymax) + 3 - ty0;
    use_tile = tw < kTile && th < kTile;
    if (use_tile)
      for (int i = lane; i < kTile * kTile; i += 32) tile[i] = 0.f;
    __syncwarp();
  }

  // pass 2: loss, dL/dp, scatter of dL/dg
  float loss = 0.f, gp[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  {
    PtWalk w(lane, S, M);
    for (int i = lane; i < N; i += 32, w.next()) {
      float tx, ty, gx = 0.f, gy = 0.f;
      const size_t cell = locate(prm, w.dx, w.dy, x0, y0, W, H, tx, ty);
      const float d = bicubic<true>(p.gimg, W, cell, tx, ty, gx, gy) - c;
      const float ft = sfc[i] * idf, gt = (d - gm) * idg;
      const float e = ft - gt;
      loss = fmaf(e, e, loss);
      if (!p.backward) continue;
      const float dgi = wgt * 2.f * idg * (C * gt - ft);
      const float a = dgi * gx, b = dgi * gy;
      const float fdx = (float)w.dx, fdy = (float)w.dy;
      gp[0] += a;
      gp[1] = fmaf(a, fdx, gp[1]);
      gp[2] = fmaf(a, fdy, gp[2]);
      gp[3] += b;
      gp[4] = fmaf(b, fdx, gp[4]);
      gp[5] = fmaf(b, fdy, gp[5]);
      float wx[4], wy[4];
      keys_weights(tx, wx);
      keys_weights(ty, wy);
      const int ix = (int)(cell % (size_t)W), iy = (int)(cell / (size_t)W);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const float rl = dgi * wy[l];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int yy = iy - 1 + l, xx = ix - 1 + k;
          if (use_tile)
            atomicAdd(&tile[(yy - ty0) * kTile + (xx - tx0)], rl * wx[k]);
          else
            atomicAdd(&p.dL_ddef[(size_t)yy * W + xx], rl * wx[k]);
        }
      }
    }
  }
  loss = warp_sum(loss);
  if (lane == 0) {
    if (p.loss_poi) p.loss_poi[poi] = loss;
    if (p.loss_total) atomicAdd(p.loss_total, loss);
  }
  if (!p.backward) return;
#pragma unroll
  for (int k = 0; k < 6; ++k) gp[k] = warp_sum(gp[k]);
  if (lane == 0 && p.dL_dp)
    for (int k = 0; k < 6; ++k) p.dL_dp[poi * 6 + k] = gp[k];
  if (use_tile) {
    __syncwarp();
    for (int i = lane; i < kTile * kTile; i += 32) {
      const float v = tile[i];
      if (v != 0.f) {
        const int yy = ty0 + i / kTile, xx = tx0 + i % kTile;
        atomicAdd(&p.dL_ddef[(size_t)yy * W + xx], v);
      }
    }
  }
}

template <typename TP>
cudaError_t launch_tp(const AdjointParams& p, cudaStream_t st) {
  const size_t smem = (size_t)kWarps * (p.S * p.S + kTile * kTile) * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(adjoint_kernel<TP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const unsigned grid = (unsigned)((p.n_pois + kWarps - 1) / kWarps);
  adjoint_kernel<TP><<<grid, 32 * kWarps, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adjoint(const AdjointParams& p, cudaStream_t st) {
  if (p.n_pois == 0) return cudaSuccess;
  return p.ref_f32 ? launch_tp<float>(p, st) : launch_tp<uint8_t>(p, st);
}

}  // namespace dic
