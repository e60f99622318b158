// k_subpixel2.cu -- IC-GN sub-pixel refinement with a second-order subset
// shape function (an extension of Section 2.2's first-order warp).
//
// p = (u, ux, uy, uxx, uxy, uyy, v, vx, vy, vxx, vxy, vyy); a subset point
// (dx, dy) maps to x0 + dx + p[0..5] . e, y0 + dy + p[6..11] . e with the
// basis e = (1, dx, dy, dx^2/2, dx dy, dy^2/2).
//   SD_i = [fx e_i, fy e_i] (12), H = sum SD^T SD (12 x 12, once per POI),
//   r_i  = (f_i - fbar) - (df/dg)(g_i - gbar),  dp = -H^-1 sum SD_i r_i,
//   W(p) <- W(p) W(dp)^-1 in the 6 x 6 representation of a quadratic warp
//   acting on (xi^2, xi eta, eta^2, xi, eta, 1), terms above second order
//   dropped; the new p comes from rows 4 and 5 of the product.
//   Stop when |dp| < tol, |dp|^2 = du^2 + dv^2 + M^2 (first derivatives^2)
//   + (M^2/2)^2 (dxx^2, dyy^2 terms) + M^4 (dxy^2 terms); an update that
//   moves any warped subset point outside [1, W-2) x [1, H-2) is rejected
//   (status OUT_OF_BOUNDS).
//
// One warp per POI, lanes over the subset points as in the first-order
// kernel.  H is summed in three passes (the xx block with sum SD_x and
// sum SD_x (f - fbar), the yy block likewise, the xy block) so that no pass
// holds more than 36 running sums per lane; the passes meet by the warp
// reduce-scatter.  H is inverted once, scaled to a unit diagonal, by the
// symmetric sweep (solve precision) on its 78-entry lower triangle in shared
// memory, three entries per lane.  The warp composition runs in FP32 on
// every lane (a 6 x 6 elimination with two right-hand sides).
#include "dic_device.cuh"
#include "dic_internal.cuh"

namespace dic {
namespace {

constexpr int kWarps2 = 4;

template <typename T>
__device__ __forceinline__ T rcp2(T d);
template <>
__device__ __forceinline__ float rcp2<float>(float d) {
  return __frcp_rn(d);
}

// (i, j) of packed lower-triangle entry e of a 12 x 12 matrix.
__device__ __forceinline__ void tri_ij(int e, int& i, int& j) {
  i = 0;
#pragma unroll
  for (int r = 1; r < 12; ++r) i += e >= r * (r + 1) / 2 ? 1 : 0;
  j = e - i * (i + 1) / 2;
}
__device__ __forceinline__ int tri(int i, int j) {
  return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i;
}

template <typename TP>
__device__ __forceinline__ const TP* ref2(const SubpixelParams& p);
template <>
__device__ __forceinline__ const uint8_t* ref2<uint8_t>(const SubpixelParams& p) {
  return p.ref;
}
template <>
__device__ __forceinline__ const float* ref2<float>(const SubpixelParams& p) {
  return p.ref_f32;
}
__device__ __forceinline__ float px2(uint8_t b) { return (float)b; }
__device__ __forceinline__ float px2(float f) { return f; }

// Per-point record: (gx, gy) and f (later f - fbar), 16 bytes.
struct Pt2 {
  float gx, gy, f, pad;
};

// Shared memory of one warp.
struct Smem2 {
  size_t pts, hs, swp, hinv, ssd, sbf, total;
};
__host__ __device__ inline Smem2 smem2_layout(int N) {
  Smem2 L;
  size_t o = 0;
  L.pts = o;  o += (size_t)N * sizeof(Pt2);
  L.hs = o;   o += 80 * sizeof(float);    // H, packed lower triangle (FP32 sums)
  L.swp = o;  o += 80 * sizeof(double);   // sweep work (solve precision)
  L.hinv = o; o += 144 * sizeof(double);  // H^-1, full, row-major
  L.ssd = o;  o += 12 * sizeof(float);
  L.sbf = o;  o += 12 * sizeof(float);
  L.total = (o + 15) / 16 * 16;
  return L;
}

// Basis values of point (dx, dy): e = (1, dx, dy, dx^2/2, dx dy, dy^2/2).
__device__ __forceinline__ void basis(float dx, float dy, float e[6]) {
  e[0] = 1.f;
  e[1] = dx;
  e[2] = dy;
  e[3] = 0.5f * dx * dx;
  e[4] = dx * dy;
  e[5] = 0.5f * dy * dy;
}

// Warped local displacement of point e under p (x and y).
__device__ __forceinline__ float2 warp2(const float p[12], const float e[6]) {
  float lx = p[0], ly = p[6];
#pragma unroll
  for (int k = 1; k < 6; ++k) {
    lx = fmaf(p[k], e[k], lx);
    ly = fmaf(p[6 + k], e[k], ly);
  }
  return make_float2(lx + e[1], ly + e[2]);
}

// Rows 4 and 5 of M(p) M(dp)^-1 (the IC-GN update), FP32: solve
// x M(dp) = a and y M(dp) = b for a, b the coefficient rows of p, by
// Gaussian elimination with partial pivoting on M(dp)^T.  Returns false if
// the matrix is singular.
__device__ __forceinline__ bool compose2(const float p[12], const float dp[12], float out[12]) {
  const float A1 = 0.5f * dp[3], A2 = dp[4], A3 = 0.5f * dp[5], A4 = 1.f + dp[1], A5 = dp[2],
              A6 = dp[0];
  const float B1 = 0.5f * dp[9], B2 = dp[10], B3 = 0.5f * dp[11], B4 = dp[7], B5 = 1.f + dp[8],
              B6 = dp[6];
  // M(dp), row-major
  float Mx[6][6] = {
      {A4 * A4 + 2 * A1 * A6, 2 * A4 * A5 + 2 * A2 * A6, A5 * A5 + 2 * A3 * A6, 2 * A4 * A6,
       2 * A5 * A6, A6 * A6},
      {A4 * B4 + A1 * B6 + A6 * B1, A4 * B5 + A5 * B4 + A2 * B6 + A6 * B2,
       A5 * B5 + A3 * B6 + A6 * B3, A4 * B6 + A6 * B4, A5 * B6 + A6 * B5, A6 * B6},
      {B4 * B4 + 2 * B1 * B6, 2 * B4 * B5 + 2 * B2 * B6, B5 * B5 + 2 * B3 * B6, 2 * B4 * B6,
       2 * B5 * B6, B6 * B6},
      {A1, A2, A3, A4, A5, A6},
      {B1, B2, B3, B4, B5, B6},
      {0.f, 0.f, 0.f, 0.f, 0.f, 1.f}};
  // system M^T z = r for r = a^T, b^T: augmented rows of M^T
  float T[6][8];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
#pragma unroll
    for (int j = 0; j < 6; ++j) T[i][j] = Mx[j][i];
  }
  // right-hand sides: the rows of p's matrix (coefficients on w)
  const float a[6] = {0.5f * p[3], p[4], 0.5f * p[5], 1.f + p[1], p[2], p[0]};
  const float b[6] = {0.5f * p[9], p[10], 0.5f * p[11], p[7], 1.f + p[8], p[6]};
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    T[i][6] = a[i];
    T[i][7] = b[i];
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    int piv = c;
    float best = fabsf(T[c][c]);
#pragma unroll
    for (int i = c + 1; i < 6; ++i)
      if (fabsf(T[i][c]) > best) {
        best = fabsf(T[i][c]);
        piv = i;
      }
    if (!(best > 0.f)) return false;
#pragma unroll
    for (int i = c + 1; i < 6; ++i)
      if (i == piv) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float t = T[c][j];
          T[c][j] = T[i][j];
          T[i][j] = t;
        }
      }
    const float inv = 1.f / T[c][c];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      if (i == c) continue;
      const float m = T[i][c] * inv;
#pragma unroll
      for (int j = c; j < 8; ++j) T[i][j] = fmaf(-m, T[c][j], T[i][j]);
    }
  }
  float z[2][6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    z[0][i] = T[i][6] / T[i][i];
    z[1][i] = T[i][7] / T[i][i];
  }
  out[3] = 2.f * z[0][0];
  out[4] = z[0][1];
  out[5] = 2.f * z[0][2];
  out[1] = z[0][3] - 1.f;
  out[2] = z[0][4];
  out[0] = z[0][5];
  out[9] = 2.f * z[1][0];
  out[10] = z[1][1];
  out[11] = 2.f * z[1][2];
  out[7] = z[1][3];
  out[8] = z[1][4] - 1.f;
  out[6] = z[1][5];
  return true;
}

// Every point of the warped subset inside [1, W-2) x [1, H-2) (warp-wide).
__device__ __forceinline__ bool all_in(const float p[12], int x0, int y0, int S, int M, int W,
                                       int H, int lane) {
  bool ok = true;
  PtWalk w(lane, S, M);
  for (int i = lane; i < S * S; i += 32, w.next()) {
    float e[6];
    basis((float)w.dx, (float)w.dy, e);
    const float2 l = warp2(p, e);
    const float x = (float)x0 + l.x, y = (float)y0 + l.y;
    ok = ok && x >= 1.f && x < (float)(W - 2) && y >= 1.f && y < (float)(H - 2);
  }
  return __all_sync(0xffffffffu, ok);
}

template <typename TS, typename TP>
__global__ void __launch_bounds__(32 * kWarps2) subpixel2_kernel(const SubpixelParams p,
                                                                 float* __restrict__ p12) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t poi = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
  if (poi >= p.n_pois) return;
  const int S = p.S, M = p.M, N = S * S, W = p.W, H = p.H;
  const Smem2 L = smem2_layout(N);
  unsigned char* base = smem + (size_t)wid * L.total;
  Pt2* pts = reinterpret_cast<Pt2*>(base + L.pts);
  float* hs = reinterpret_cast<float*>(base + L.hs);
  TS* swp = reinterpret_cast<TS*>(base + L.swp);
  TS* hinv = reinterpret_cast<TS*>(base + L.hinv);
  float* ssd = reinterpret_cast<float*>(base + L.ssd);
  float* sbf = reinterpret_cast<float*>(base + L.sbf);
  const int x0 = M + p.R + 2 + (int)(poi % p.nx) * p.step;
  const int y0 = M + p.R + 2 + (int)(poi / p.nx) * p.step;
  const TP* fimg = ref2<TP>(p);

  float prm[12] = {(float)p.u0[poi], 0.f, 0.f, 0.f, 0.f, 0.f,
                   (float)p.v0[poi], 0.f, 0.f, 0.f, 0.f, 0.f};
  auto write_out = [&](float zn, int it, uint8_t st) {
    if (lane == 0) {
      p.zncc[poi] = zn;
      p.iters[poi] = it;
      p.status[poi] = st;
    }
#pragma unroll
    for (int k = 0; k < 12; ++k)
      if (lane == k) p12[poi * 12 + k] = prm[k];
  };
  const uint8_t st0 = p.st0[poi];
  if (st0 != kOk) {
    write_out(0.f, 0, st0);
    return;
  }

  // ---- reference subset: f and its gradient per point, sum of f
  float fsum = 0.f;
  {
    PtWalk w(lane, S, M);
    for (int i = lane; i < N; i += 32, w.next()) {
      const float f = px2(fimg[(size_t)(y0 + w.dy) * p.pitch + (x0 + w.dx)]);
      const float2 gr = p.grad[(size_t)(y0 + w.dy) * W + (x0 + w.dx)];
      pts[i] = Pt2{gr.x, gr.y, f, 0.f};
      fsum += f;
    }
  }
  fsum = warp_sum(fsum);
  const float fbar = fsum / (float)N;
  // ---- H in three passes: xx block (+ sum SD_x, sum SD_x fc), yy block
  // (likewise), xy block; each lane's sums meet by reduce-scatter
  float q = 0.f;
#pragma unroll 1
  for (int blk = 0; blk < 2; ++blk) {
    float h[21], s[6], sf[6];
#pragma unroll
    for (int k = 0; k < 21; ++k) h[k] = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) s[k] = sf[k] = 0.f;
    PtWalk w(lane, S, M);
    for (int i = lane; i < N; i += 32, w.next()) {
      Pt2 r = pts[i];
      const float fc = r.f - fbar;
      if (blk == 0) q = fmaf(fc, fc, q);
      const float g = blk == 0 ? r.gx : r.gy;
      float e[6], sd[6];
      basis((float)w.dx, (float)w.dy, e);
#pragma unroll
      for (int k = 0; k < 6; ++k) sd[k] = g * e[k];
      int t = 0;
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        s[a] += sd[a];
        sf[a] = fmaf(sd[a], fc, sf[a]);
#pragma unroll
        for (int b = 0; b <= a; ++b, ++t) h[t] = fmaf(sd[a], sd[b], h[t]);
      }
    }
    float v[32];
#pragma unroll
    for (int k = 0; k < 21; ++k) v[k] = h[k];
#pragma unroll
    for (int k = 0; k < 6; ++k) v[21 + k] = s[k];
#pragma unroll
    for (int k = 0; k < 5; ++k) v[27 + k] = sf[k];
    const float last = warp_sum(sf[5]);
    const float mine = reduce_scatter32(v, lane);
    if (lane < 21) {
      int a, b;
      tri_ij(lane, a, b);  // (a, b) of the 6 x 6 block, a >= b
      hs[tri(6 * blk + a, 6 * blk + b)] = mine;
    } else if (lane < 27) {
      ssd[6 * blk + lane - 21] = mine;
    } else {
      sbf[6 * blk + lane - 27] = mine;
    }
    if (lane == 0) sbf[6 * blk + 5] = last;
  }
  {
    // xy block: entries (6 + a, b), a, b in 0..5: sum (fy e_a)(fx e_b)
    float h[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) h[k] = 0.f;
    PtWalk w(lane, S, M);
    for (int i = lane; i < N; i += 32, w.next()) {
      const Pt2 r = pts[i];
      float e[6];
      basis((float)w.dx, (float)w.dy, e);
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        const float ya = r.gy * e[a];
#pragma unroll
        for (int b = 0; b < 6; ++b) h[6 * a + b] = fmaf(ya, r.gx * e[b], h[6 * a + b]);
      }
    }
    float v[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = h[k];
    float rest[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) rest[k] = warp_sum(h[32 + k]);
    const float mine = reduce_scatter32(v, lane);
    hs[tri(6 + lane / 6, lane % 6)] = mine;
    if (lane < 4) {
      const int k = 32 + lane;
      float r = rest[0];
#pragma unroll
      for (int j = 1; j < 4; ++j) r = lane == j ? rest[j] : r;
      hs[tri(6 + k / 6, k % 6)] = r;
    }
  }
  q = warp_sum(q);
  const float df = sqrtf(q);
  // f - fbar into the records for the iterations
  for (int i = lane; i < N; i += 32) pts[i].f -= fbar;
  __syncwarp();
  if (!(df > 0.f)) {
    write_out(0.f, 0, kZeroVarRef);
    return;
  }

  // ---- H^-1: unit-diagonal scaling, symmetric sweep (solve precision),
  // three lower-triangle entries per lane (lanes 0..25), shared memory
  float dsc[12];
  bool okd = true;
#pragma unroll
  for (int a = 0; a < 12; ++a) {
    const float hd = hs[tri(a, a)];
    okd = okd && hd > 0.f && isfinite(hd);
    dsc[a] = hd > 0.f ? rsqrtf(hd) : 1.f;
  }
  int ei[3], ej[3];
  TS av[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int e = lane + 32 * c;
    if (e < 78) {
      tri_ij(e, ei[c], ej[c]);
      float di = dsc[0], dj = dsc[0];
#pragma unroll
      for (int a = 1; a < 12; ++a) {
        di = ei[c] == a ? dsc[a] : di;
        dj = ej[c] == a ? dsc[a] : dj;
      }
      av[c] = (TS)(hs[e] * (di * dj));
      swp[e] = av[c];
    } else {
      ei[c] = ej[c] = 0;
      av[c] = TS(0);
    }
  }
  __syncwarp();
  bool ok = okd;
#pragma unroll 1
  for (int k = 0; k < 12; ++k) {
    const TS akk = swp[tri(k, k)];
    TS d;
    if constexpr (sizeof(TS) == 8) {  // no FP64 compares or conversions (see rcp_pivot)
      ok = ok && pivot_ok(akk);
      d = rcp_pivot(ok ? akk : 1.0);
    } else {
      ok = ok && akk > TS(0) && akk < TS(3e38);
      d = rcp2<TS>(ok ? akk : TS(1));
    }
    TS nv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // an entry of row or column k is a_ik (a_kj) itself: its new value
      // a / a_kk is the other operand times 1/a_kk, one multiply
      const int i = ei[c], j = ej[c];
      const bool ik = i == k, jk = j == k;
      const TS aik = swp[tri(i, k)], ajk = swp[tri(j, k)];
      const TS t = (ik ? ajk : aik) * d;
      TS r = fma(-t, ik ? aik : ajk, av[c]);
      if (ik || jk) r = t;
      if (ik && jk) r = -d;
      nv[c] = r;
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      av[c] = nv[c];
      if (lane + 32 * c < 78) swp[lane + 32 * c] = nv[c];
    }
    __syncwarp();
  }
  if (!ok) {
    write_out(0.f, 0, kSingular);
    return;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int e = lane + 32 * c;
    if (e < 78) {
      const int i = ei[c], j = ej[c];
      float di = dsc[0], dj = dsc[0];
#pragma unroll
      for (int a = 1; a < 12; ++a) {
        di = i == a ? dsc[a] : di;
        dj = j == a ? dsc[a] : dj;
      }
      const TS hv = -av[c] * (TS)(di * dj);
      hinv[i * 12 + j] = hv;
      hinv[j * 12 + i] = hv;
    }
  }
  __syncwarp();
  if (!all_in(prm, x0, y0, S, M, W, H, lane)) {
    write_out(0.f, 0, kOutOfBounds);
    return;
  }

  const float c = fbar;
  const float invN = 1.f / (float)N;
  const float m2 = (float)M * (float)M, q2 = 0.25f * m2 * m2, m4 = m2 * m2;
  uint8_t st = kMaxIter;
  int it_done = 0;
  float zn = 0.f;
  bool have_zn = false;
  // The bounds test of an accepted update is taken in the next pass, from
  // the positions that pass computes anyway (the same arithmetic as
  // all_in); a shape that fails it is undone as if it had been refused, so
  // statuses, shapes and iteration counts are those of testing it at once.
  // Only the shape a POI returns is tested by all_in.
  // the shape before the last accepted update, entry a on lane a
  float pprev = 0.f;
  auto undo = [&]() {
#pragma unroll
    for (int a = 0; a < 12; ++a) prm[a] = __shfl_sync(0xffffffffu, pprev, a);
  };
  bool pending = false;  // prm is an update not yet tested against the bounds
  for (int it = 1; it <= p.max_iter; ++it) {
    float s0 = 0.f, s1 = 0.f, sfd = 0.f;
    float2 acc[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] = dup2(0.f);
    bool inb = true;
    PtWalk w(lane, S, M);
    for (int i = lane; i < N; i += 32, w.next()) {
      float e[6];
      basis((float)w.dx, (float)w.dy, e);
      float g;
      if (it == 1) {
        // the start shape is an integer shift: every sample is a pixel
        g = p.gimg[(size_t)(y0 + w.dy + (int)prm[6]) * W + (x0 + w.dx + (int)prm[0])];
      } else {
        const float2 l = warp2(prm, e);
        if (pending) {
          const float x = (float)x0 + l.x, y = (float)y0 + l.y;
          inb = inb && x >= 1.f && x < (float)(W - 2) && y >= 1.f && y < (float)(H - 2);
        }
        const float fx = floorf(l.x), fy = floorf(l.y);
        float2 t = make_float2(l.x - fx, l.y - fy);
        int ix = x0 + (int)fx, iy = y0 + (int)fy;
        ix = min(max(ix, 1), W - 3);  // memory safety only; bounds are checked on p
        iy = min(max(iy, 1), H - 3);
        const size_t cell = (size_t)iy * W + ix;
        if (sizeof(TP) == 1)
          g = bicubic_q(p.gq, W, cell, t);
        else
          g = bicubic2(p.gimg, W, cell, t);
      }
      const Pt2 r = pts[i];
      const float d = g - c;
      s0 += d;
      s1 = fmaf(d, d, s1);
      sfd = fmaf(r.f, d, sfd);
      const float2 ab = make_float2(r.gx * d, r.gy * d);
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[k] = __ffma2_rn(ab, dup2(e[k]), acc[k]);
    }
    if (pending) {
      if (!__all_sync(0xffffffffu, inb)) {
        undo();
        st = kOutOfBounds;
        break;
      }
      pending = false;
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    float bsum[12];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      bsum[k] = warp_sum(acc[k].x);
      bsum[6 + k] = warp_sum(acc[k].y);
    }
    const float gm = s0 * invN;
    const float var = s1 - s0 * gm;
    const float dg = sqrtf(fmaxf(var, 0.f));
    if (!(dg > 0.f) || !isfinite(dg)) {
      st = kNonFinite;
      break;
    }
    const float ratio = df / dg;
    float rhs[12];
#pragma unroll
    for (int a = 0; a < 12; ++a) rhs[a] = sbf[a] - ratio * (bsum[a] - gm * ssd[a]);
    // dp = -H^-1 rhs: lanes 0..23, two lanes per row, six products each
    float dp[12];
    {
      const int r = min(lane >> 1, 11), half = lane & 1;
      const TS* hr = hinv + r * 12 + 6 * half;
      TS sacc = TS(0);
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        float rk = rhs[0];
#pragma unroll
        for (int j = 1; j < 12; ++j) rk = (6 * half + k) == j ? rhs[j] : rk;
        sacc = fma(hr[k], (TS)rk, sacc);
      }
      sacc += __shfl_xor_sync(0xffffffffu, sacc, 1);
      const float mine = (float)(-sacc);
#pragma unroll
      for (int a = 0; a < 12; ++a) dp[a] = __shfl_sync(0xffffffffu, mine, 2 * a);
    }
    it_done = it;
    bool fin = true;
#pragma unroll
    for (int a = 0; a < 12; ++a) fin = fin && isfinite(dp[a]);
    if (!fin) {
      st = kNonFinite;
      break;
    }
    float pn[12];
    if (!compose2(prm, dp, pn)) {
      st = kNonFinite;
      break;
    }
#pragma unroll
    for (int a = 0; a < 12; ++a) {
      pprev = lane == a ? prm[a] : pprev;
      prm[a] = pn[a];
    }
    pending = true;
    const float nrm = sqrtf(dp[0] * dp[0] + dp[6] * dp[6] +
                            m2 * (dp[1] * dp[1] + dp[2] * dp[2] + dp[7] * dp[7] + dp[8] * dp[8]) +
                            q2 * (dp[3] * dp[3] + dp[5] * dp[5] + dp[9] * dp[9] + dp[11] * dp[11]) +
                            m4 * (dp[4] * dp[4] + dp[10] * dp[10]));
    if (nrm < p.tol) {
      if (!all_in(prm, x0, y0, S, M, W, H, lane)) {
        undo();
        st = kOutOfBounds;
        break;
      }
      zn = warp_sum(sfd) / (df * dg);  // at the last sampled shape, as the first-order path
      have_zn = true;
      st = kOk;
      break;
    }
  }
  // iteration cap: the last update was accepted but never sampled
  if (pending && st == kMaxIter && !all_in(prm, x0, y0, S, M, W, H, lane)) {
    undo();
    st = kOutOfBounds;
  }
  if (!have_zn) {
    float s0 = 0.f, s1 = 0.f, sfg = 0.f;
    PtWalk w(lane, S, M);
    for (int i = lane; i < N; i += 32, w.next()) {
      float e[6];
      basis((float)w.dx, (float)w.dy, e);
      const float2 l = warp2(prm, e);
      const float fx = floorf(l.x), fy = floorf(l.y);
      int ix = min(max(x0 + (int)fx, 1), W - 3), iy = min(max(y0 + (int)fy, 1), H - 3);
      float gx, gy;
      const float d = bicubic<false>(p.gimg, W, (size_t)iy * W + ix, l.x - fx, l.y - fy, gx, gy) - c;
      s0 += d;
      s1 = fmaf(d, d, s1);
      sfg = fmaf(pts[i].f, d, sfg);
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    sfg = warp_sum(sfg);
    const float dgf = sqrtf(fmaxf(s1 - s0 * s0 * invN, 0.f));
    zn = dgf > 0.f ? sfg / (df * dgf) : 0.f;
  }
  write_out(zn, it_done, st);
}

template <typename TS, typename TP>
cudaError_t launch2(const SubpixelParams& p, float* p12, cudaStream_t st) {
  // kWarps2 warps per CTA, fewer where the subset's records would not fit
  const size_t wb = smem2_layout(p.S * p.S).total;
  int wpc = kWarps2;
  while (wpc > 1 && (size_t)wpc * wb > 227 * 1024) --wpc;
  const size_t smem = (size_t)wpc * wb;
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(subpixel2_kernel<TS, TP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((p.n_pois + wpc - 1) / wpc);
  subpixel2_kernel<TS, TP><<<grid, 32 * wpc, smem, st>>>(p, p12);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_subpixel2(const SubpixelParams& p, int solve_fp64, float* p12,
                             cudaStream_t st) {
  if (p.n_pois == 0) return cudaSuccess;
  if (p.ref_f32)
    return solve_fp64 ? launch2<double, float>(p, p12, st) : launch2<float, float>(p, p12, st);
  if (!p.gq) return cudaErrorInvalidValue;
  return solve_fp64 ? launch2<double, uint8_t>(p, p12, st) : launch2<float, uint8_t>(p, p12, st);
}

}  // namespace dic
