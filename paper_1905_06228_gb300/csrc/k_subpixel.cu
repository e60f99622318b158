// k_subpixel.cu -- sub-pixel refinement: IC-GN and FA-NR (Section 2.2, Table 2).
//
// One warp per POI; lane l owns subset points i = l, l+32, ...  Per-point
// reference data (the gradient of f and f) lives in shared memory for the
// whole solve; the deformed image is interpolated with Keys weights
// evaluated per sample, from its BF16 tap quads (IC-GN, 8-bit pairs) or its
// float copy.
//
// Warp:   W(xi; p) = (x0 + dx + u + ux dx + uy dy, y0 + dy + v + vx dx + vy dy).
// IC-GN:  SD_i = grad f_i dW/dp, H = sum SD^T SD (once per POI),
//         r_i = (f_i - fbar) - (df/dg)(g_i - gbar),
//         dp = -H^-1 sum SD_i r_i,   W(p) <- W(p) W(dp)^-1.
// FA-NR:  J_i = grad g(W(xi_i; p)) dW/dp (derivative of the bicubic patch),
//         dp = (sum J^T J)^-1 sum J_i [(dg/df)(f_i - fbar) - (g_i - gbar)],
//         p <- p + dp  (Gauss-Newton form of Newton-Raphson).
// Stop:   |dp|_c = sqrt(du^2 + dv^2 + M^2 (dux^2+duy^2+dvx^2+dvy^2)) < tol,
//         else after max_iter solves; an update that moves a subset corner
//         outside [1, W-2) x [1, H-2) is rejected (status OUT_OF_BOUNDS).
//
// Each iteration is ONE pass over the points: with the shift c = fbar the
// lane accumulates S0 = sum (g-c), S1 = sum (g-c)^2 and sum SD_k (g-c) (or
// the FA-NR sums); then gbar = c + S0/N, dg^2 = S1 - S0^2/N and the
// right-hand side follow exactly as in the formulas above.  The 6x6 solve is
// FP32 or FP64, chosen per launch: the matrix, scaled to a unit diagonal,
// is inverted by the symmetric sweep operator with one lane per entry of
// its lower triangle (pivot reciprocals refined by Newton's iteration, no
// divisions) into shared memory, and lane k < 6 forms row k of H^-1 times
// the right-hand side; IC-GN inverts H once per POI, FA-NR its Gauss-Newton
// matrix every iteration.  Each pass also accumulates
// sum (f-fbar)(g-c), so a POI that converges reports Eq. 1 at the shape its
// last pass sampled (the returned shape differs by the final update, below
// tol, at a stationary point of C: the two values differ by O(|dp|^2));
// other POIs get one extra pass at the returned shape.

// Build options: resident CTAs per SM requested from the register allocator
// (IC-GN, FA-NR), warps per CTA, and the unroll of the per-point loop.
#ifndef DIC_SUB_MINB
#define DIC_SUB_MINB 4
#endif
// FA-NR (39 sums per sample): 4 CTAs/SM, 96 registers without spills
// (1.05 ms on affine1024 against 1.13 ms at 3 CTAs/SM and 1.39 ms at 146
// registers and 2 CTAs/SM)
#ifndef DIC_SUB_MINB_NR
#define DIC_SUB_MINB_NR 4
#endif
#ifndef DIC_SUB_UNROLL
#define DIC_SUB_UNROLL 1
#endif

#include "dic_device.cuh"
#include "dic_internal.cuh"

namespace dic {
namespace {

// warps per CTA: 5 x 4 CTAs = 20 warps per SM at 96 registers per thread
// (no spills; 8 x 3 at 80 registers spilled and ran 5 % slower)
#ifndef DIC_SUB_WPC
#define DIC_SUB_WPC 5
#endif
constexpr int kWarpsPerCta = DIC_SUB_WPC;
constexpr int kPointUnroll = DIC_SUB_UNROLL;

// 1/sqrt(d): FP32 estimate refined by Newton's iteration for 1/y^2 = d,
// y <- y (3/2 - d y^2 / 2), which doubles the correct bits per step.
template <typename T>
__device__ __forceinline__ T rsqrt_refined(T d);
template <>
__device__ __forceinline__ float rsqrt_refined<float>(float d) {
  float y = rsqrtf(d);
  return y * (1.5f - 0.5f * d * y * y);
}

// 1/d: FP32 reciprocal refined by Newton's iteration y <- y + y (1 - d y)
// in the solve precision (each step doubles the correct bits).
template <typename T>
__device__ __forceinline__ T rcp_refined(T d);
template <>
__device__ __forceinline__ float rcp_refined<float>(float d) {
  return __frcp_rn(d);
}

__device__ __forceinline__ int packed_index(int r, int c) {  // entry (r, c) of a packed lower triangle
  return r >= c ? r * (r + 1) / 2 + c : c * (c + 1) / 2 + r;
}

// Entry (i, j), i >= j, of a packed lower-triangular 6x6 held by lane
// l = i (i+1)/2 + j (lanes >= 21 get (5, 5) and hold no entry).
__device__ __forceinline__ void packed_entry(int lane, int& i, int& j) {
  i = 0;
#pragma unroll
  for (int r = 1; r < 6; ++r) i += lane >= r * (r + 1) / 2 ? 1 : 0;
  j = min(lane - i * (i + 1) / 2, i);
}

// Inverse of a symmetric positive definite 6x6 by the symmetric sweep
// operator, one lane per entry of the lower triangle (lane l < 21 passes
// its entry h = A_ij, (i, j) from packed_entry).  Pivot k (k = 0..5)
// replaces a_kk by -1/a_kk, every other entry of row / column k by
// a_ik / a_kk, and the remaining entries by a_ij - a_ik a_jk / a_kk; after
// the six pivots the entries hold -A^-1 (Gauss-Jordan elimination in
// symmetric form; the pivots are the successive Schur complements, positive
// for a positive definite A, so no pivoting is needed).  Each step costs a
// few instructions for the whole warp, instead of a full factorisation
// repeated on every lane.  A lane of row or column k holds a_ik (or a_kj)
// itself, so its new value a / a_kk is the product of the other operand's
// selection with 1/a_kk: one multiply per step for every lane.  Returns
// false on every lane if a pivot is not positive and finite (FP64: not in
// [2^-100, 2^100), tested on the high word with integer compares);
// out = (A^-1)_ij on lanes < 21.
template <typename T>
__device__ __forceinline__ bool sweep_inverse6(float h, int i, int j, T& out) {
  T a = (T)h;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const T akk = __shfl_sync(0xffffffffu, a, k * (k + 1) / 2 + k);
    const T aik = __shfl_sync(0xffffffffu, a, packed_index(i, k));
    const T ajk = __shfl_sync(0xffffffffu, a, packed_index(j, k));
    T d;
    if constexpr (sizeof(T) == 8) {
      ok = ok && pivot_ok(akk);
      d = rcp_pivot(ok ? akk : 1.0);
    } else {
      ok = ok && akk > T(0) && akk < T(3e38);
      d = rcp_refined<T>(ok ? akk : T(1));
    }
    const bool ik = i == k, jk = j == k;
    const T t = (ik ? ajk : aik) * d;  // a * d on the lanes of row / column k
    T r = fma(-t, ik ? aik : ajk, a);
    if (ik || jk) r = t;
    if (ik && jk) r = -d;
    a = r;
  }
  out = -a;
  return ok;
}

// H^-1 into shared memory (36 solve-precision values, row-major) from the 21
// entries of a symmetric positive definite H held one per lane (lane l < 21:
// packed entry l, see packed_entry): H is first scaled symmetrically to a
// unit diagonal (Hs = D H D, D_ii = H_ii^-1/2; H^-1 = D Hs^-1 D) -- the
// translation and gradient columns differ in scale by ~M^2, which the
// elimination then does not see -- then inverted by the sweep.  D_ii D_jj is
// rounded to FP32 before the solve-precision product (relative 6e-8, below
// the FP32 sums that form H).  Returns false (every lane) if H is not
// positive definite.
template <typename TS>
__device__ __forceinline__ bool invert_to_smem(float mine, int lane, TS* hinv) {
  float dsc[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    const float hd = __shfl_sync(0xffffffffu, mine, a * (a + 1) / 2 + a);
    dsc[a] = hd > 0.f ? rsqrt_refined<float>(hd) : 1.f;
  }
  int ei, ej;
  packed_entry(lane, ei, ej);
  float di = dsc[0], dj = dsc[0];
#pragma unroll
  for (int a = 1; a < 6; ++a) {
    di = ei == a ? dsc[a] : di;
    dj = ej == a ? dsc[a] : dj;
  }
  TS hij;
  if (!sweep_inverse6<TS>(mine * (di * dj), ei, ej, hij)) return false;
  if (lane < 21) {
    const TS hv = hij * (TS)(di * dj);
    hinv[ei * 6 + ej] = hv;
    hinv[ej * 6 + ei] = hv;
  }
  __syncwarp();
  return true;
}

// Row a of H^-1 (shared memory, solve precision) times rhs, for a = 0..5,
// on every lane.  Lanes 0..17 each form two products of row lane/3
// (columns 2 (lane % 3) and + 1); the three partial sums of a row meet on
// lane 3a by two shuffles, so the solve precision's work is two conversions,
// a multiply, a multiply-add and two adds per warp instead of six
// conversions and six multiply-adds.
template <typename TS>
__device__ __forceinline__ void apply_hinv(const TS* hinv, const float (&rhs)[6], int lane,
                                           float (&out)[6]) {
  const int r = min(lane / 3, 5), j = 2 * (lane % 3);
  float b0 = rhs[0], b1 = rhs[1];
  if (j == 2) b0 = rhs[2], b1 = rhs[3];
  if (j == 4) b0 = rhs[4], b1 = rhs[5];
  const TS* hr = hinv + r * 6 + j;
  TS acc = hr[0] * (TS)b0;
  acc = fma(hr[1], (TS)b1, acc);
  const TS a1 = __shfl_down_sync(0xffffffffu, acc, 1);
  const TS a2 = __shfl_down_sync(0xffffffffu, acc, 2);
  const float mine = (float)((acc + a1) + a2);
#pragma unroll
  for (int a = 0; a < 6; ++a) out[a] = __shfl_sync(0xffffffffu, mine, 3 * a);
}

// 8-bit pixel as float without a conversion instruction: its bits OR'd into
// the mantissa of 2^23, minus 2^23 (exact).
__device__ __forceinline__ float pixel_value(uint8_t b) {
  return __uint_as_float(0x4B000000u | (uint32_t)b) - 8388608.0f;
}
__device__ __forceinline__ float pixel_value(float f) { return f; }

// W(p) <- W(p) W(dp)^-1 for the first-order warp.
__device__ __forceinline__ void compose_inverse(float p[6], const float dp[6]) {
  const float a = 1.f + dp[1], b = dp[2], c = dp[4], d = 1.f + dp[5];
  const float det = a * d - b * c;
  const float rdet = __frcp_rn(det);
  const float ia = d * rdet, ib = -b * rdet, ic = -c * rdet, id = a * rdet;
  const float itx = -(ia * dp[0] + ib * dp[3]);
  const float ity = -(ic * dp[0] + id * dp[3]);
  const float P00 = 1.f + p[1], P01 = p[2], P02 = p[0];
  const float P10 = p[4], P11 = 1.f + p[5], P12 = p[3];
  const float n00 = P00 * ia + P01 * ic, n01 = P00 * ib + P01 * id;
  const float n02 = P00 * itx + P01 * ity + P02;
  const float n10 = P10 * ia + P11 * ic, n11 = P10 * ib + P11 * id;
  const float n12 = P10 * itx + P11 * ity + P12;
  p[0] = n02;
  p[1] = n00 - 1.f;
  p[2] = n01;
  p[3] = n12;
  p[4] = n10;
  p[5] = n11 - 1.f;
}

template <typename T>
__device__ __forceinline__ const T* ref_ptr(const SubpixelParams& p);
template <>
__device__ __forceinline__ const uint8_t* ref_ptr<uint8_t>(const SubpixelParams& p) {
  return p.ref;
}
template <>
__device__ __forceinline__ const float* ref_ptr<float>(const SubpixelParams& p) {
  return p.ref_f32;
}

// Per-point reference data kept in shared memory: the gradient of f and f.
// 8-bit images: BF16, 8 bytes per point.  Central differences of 8-bit
// pixels are k/2 with |k| <= 255 and the pixels integers below 256: at most
// 8 significant bits, so their FP32 encodings end in 16 zero bits and the
// upper halves (BF16) are exact; unpacking is a shift and a mask (integer
// ALU), f is stored as its full FP32 bits.  Float images: FP32, 16 bytes.
template <typename TP>
struct PointStore;
template <>
struct PointStore<uint8_t> {
  struct alignas(8) T {
    uint32_t g;  // BF16 of df/dx (low half), df/dy (high half)
    uint32_t f;  // FP32 bits of f (low half zero)
  };
  static __device__ __forceinline__ T pack(float2 g, float f) {
    return T{(__float_as_uint(g.x) >> 16) | (__float_as_uint(g.y) & 0xFFFF0000u),
             __float_as_uint(f)};
  }
  static __device__ __forceinline__ void unpack(const T& t, float2& g, float& f) {
    g = make_float2(__uint_as_float(t.g << 16), __uint_as_float(t.g & 0xFFFF0000u));
    f = __uint_as_float(t.f);
  }
};
template <>
struct PointStore<float> {
  struct alignas(16) T {
    float2 g;
    float f, pad;
  };
  static __device__ __forceinline__ T pack(float2 g, float f) { return T{g, f, 0.f}; }
  static __device__ __forceinline__ void unpack(const T& t, float2& g, float& f) {
    g = t.g;
    f = t.f;
  }
};

// Shared memory of one warp: N point records, then (16-byte aligned) H^-1
// as 36 solve-precision values, then the IC-GN constants sum SD and
// sum SD (f - fbar) (6 floats each).
__host__ __device__ inline size_t warp_smem_bytes(int N, size_t point_bytes) {
  return ((size_t)N * point_bytes + 15) / 16 * 16 + 36 * sizeof(double) + 12 * sizeof(float);
}

// IC-GN of one POI of an 8-bit pair (bicubic interpolation, or bilinear with
// BIL) when the subset width is 31 or 15 (LPR = 32 or 16 lanes per subset row): lane c of
// each group of LPR lanes owns column dx = c - M of every (32 / LPR)-th row
// (the last lane of a group idles), so dx is constant per lane.  The
// arithmetic is the generic path's; what changes is where the work lands:
//  - the set-up keeps per-lane sums of g_a g_b, g_a g_b dy, g_a g_b dy^2,
//    g_a, g_a dy, g_a (f - fbar) and g_a (f - fbar) dy (a, b in {x, y}) and
//    multiplies by the lane's dx (and dx^2) once, instead of every product
//    of the SD vector per point;
//  - a sample's local displacement is one multiply-add from the lane's
//    column term (u + (1+ux) dx, v + vx dx) and dy -- the same two
//    roundings as the generic walk, so the same sample positions -- and the
//    walk is a row step;
//  - sum SD_1 (g - c) and sum SD_4 (g - c) are dx times the lane's
//    sum SD_0 (g - c) and sum SD_3 (g - c), formed once per pass;
//  - the point records hold f - fbar instead of f.
template <typename TS, int LPR, bool BIL>
__device__ __forceinline__ void icgn_col_poi(const SubpixelParams& p, int64_t poi, int lane,
                                             unsigned char* wsm) {
  using PS = PointStore<uint8_t>;
  using G = PS::T;
  constexpr int S = LPR - 1, M = S / 2, N = S * S, RPP = 32 / LPR;
  const int x0 = M + p.R + 2 + (int)(poi % p.nx) * p.step;
  const int y0 = M + p.R + 2 + (int)(poi / p.nx) * p.step;
  const int W = p.W, H = p.H;
  G* spt = reinterpret_cast<G*>(wsm);
  TS* hinv = reinterpret_cast<TS*>(wsm + ((size_t)N * sizeof(G) + 15) / 16 * 16);
  float* ssd = reinterpret_cast<float*>(hinv + 36);  // sum SD
  float* sbf = ssd + 6;                              // sum SD (f - fbar)
  const int col = lane % LPR, row0 = lane / LPR;
  const bool act = col < S;
  const float fdx = (float)(col - M);

  const uint8_t st0 = p.st0[poi];
  float prm[6] = {(float)p.u0[poi], 0.f, 0.f, (float)p.v0[poi], 0.f, 0.f};
  auto write_out = [&](float zn, int it, uint8_t st) {
    if (lane == 0) {
      p.u[poi] = prm[0];
      p.ux[poi] = prm[1];
      p.uy[poi] = prm[2];
      p.v[poi] = prm[3];
      p.vx[poi] = prm[4];
      p.vy[poi] = prm[5];
      p.zncc[poi] = zn;
      p.iters[poi] = it;
      p.status[poi] = st;
    }
  };
  if (st0 != kOk) {
    write_out(0.f, 0, st0);
    return;
  }

  // ---- reference subset into shared memory, sum of f (exact)
  float fsum = 0.f;
  if (act) {
#pragma unroll 4
    for (int r = row0; r < S; r += RPP) {
      const float f = pixel_value(p.ref[(size_t)(y0 + r - M) * p.pitch + (x0 + col - M)]);
      fsum += f;
      spt[r * S + col] = PS::pack(p.grad[(size_t)(y0 + r - M) * W + (x0 + col - M)], f);
    }
  }
  fsum = warp_sum(fsum);
  const float fbar = fsum / (float)N;
  // ---- per-lane sums (each lane reads back only the records it wrote)
  float2 g0 = dup2(0.f), g1 = dup2(0.f), g2 = dup2(0.f);   // sum g_a^2 (dy^0,1,2)
  float2 s0 = dup2(0.f), s1 = dup2(0.f);                    // sum g_a (dy^0,1)
  float2 fs0 = dup2(0.f), fs1 = dup2(0.f);                  // sum g_a fc (dy^0,1)
  float c0 = 0.f, c1 = 0.f, c2 = 0.f, q = 0.f;              // sum gx gy (dy^0,1,2)
  if (act) {
#pragma unroll 2
    for (int r = row0; r < S; r += RPP) {
      const int i = r * S + col;
      float2 gr;
      float f;
      PS::unpack(spt[i], gr, f);
      const float fc = f - fbar;
      spt[i].f = __float_as_uint(fc);
      q = fmaf(fc, fc, q);
      const float dy = (float)(r - M);
      const float2 dy2 = dup2(dy);
      const float2 t = __fmul2_rn(gr, gr), tdy = __fmul2_rn(t, dy2);
      g0 = __fadd2_rn(g0, t);
      g1 = __fadd2_rn(g1, tdy);
      g2 = __ffma2_rn(tdy, dy2, g2);
      const float c = gr.x * gr.y, cdy = c * dy;
      c0 += c;
      c1 += cdy;
      c2 = fmaf(cdy, dy, c2);
      s0 = __fadd2_rn(s0, gr);
      s1 = __ffma2_rn(gr, dy2, s1);
      const float2 gfc = __fmul2_rn(gr, dup2(fc));
      fs0 = __fadd2_rn(fs0, gfc);
      fs1 = __ffma2_rn(gfc, dy2, fs1);
    }
  }
  // the lane's share of the 33 sums, in the order of the generic path: H
  // (packed lower triangle of SD = (gx e, gy e), e = (1, dx, dy)), sum SD,
  // sum SD (f - fbar)
  float v[32];
  {
    const float dx = act ? fdx : 0.f, dxx = dx * dx;
    // xx block: (0,0) (1,0) (1,1) (2,0) (2,1) (2,2)
    v[0] = g0.x; v[1] = dx * g0.x; v[2] = dxx * g0.x;
    v[3] = g1.x; v[4] = dx * g1.x; v[5] = g2.x;
    // row 3 (gy e0): xy block then yy (3,3)
    v[6] = c0; v[7] = dx * c0; v[8] = c1; v[9] = g0.y;
    // row 4 (gy e1): xy, then yy (4,3) (4,4)
    v[10] = dx * c0; v[11] = dxx * c0; v[12] = dx * c1; v[13] = dx * g0.y; v[14] = dxx * g0.y;
    // row 5 (gy e2): xy, then yy (5,3) (5,4) (5,5)
    v[15] = c1; v[16] = dx * c1; v[17] = c2; v[18] = g1.y; v[19] = dx * g1.y; v[20] = g2.y;
    v[21] = s0.x; v[22] = dx * s0.x; v[23] = s1.x;
    v[24] = s0.y; v[25] = dx * s0.y; v[26] = s1.y;
    v[27] = fs0.x; v[28] = dx * fs0.x; v[29] = fs1.x;
    v[30] = fs0.y; v[31] = dx * fs0.y;
  }
  const float last = warp_sum(fs1.y);  // sum SD_5 (f - fbar)
  const float mine = reduce_scatter32(v, lane);
  q = warp_sum(q);
  const float df = sqrtf(q);
  if (!(df > 0.f)) {
    write_out(0.f, 0, kZeroVarRef);
    return;
  }
  if (lane >= 21 && lane < 27) ssd[lane - 21] = mine;
  if (lane >= 27) sbf[lane - 27] = mine;
  if (lane == 0) sbf[5] = last;
  if (!invert_to_smem<TS>(mine, lane, hinv)) {
    write_out(0.f, 0, kSingular);
    return;
  }
  if (!corners_in_warp(prm, x0, y0, M, W, H, lane)) {
    write_out(0.f, 0, kOutOfBounds);
    return;
  }

  const float c = fbar;
  const float invN = 1.f / (float)N;
  const float m2 = (float)M * (float)M;
  uint8_t st = kMaxIter;
  int it_done = 0;
  float zn = 0.f;
  bool have_zn = false;
  for (int it = 1; it <= p.max_iter; ++it) {
    float s0s = 0.f, s1s = 0.f, sfd = 0.f;
    float2 a03 = dup2(0.f), a25 = dup2(0.f);
    auto absorb = [&](int i, float g, float dy) {
      const float d = g - c;
      s0s += d;
      s1s = fmaf(d, d, s1s);
      float2 gr;
      float fc;
      PS::unpack(spt[i], gr, fc);
      sfd = fmaf(fc, d, sfd);
      const float2 ab = __fmul2_rn(gr, dup2(d));
      a03 = __fadd2_rn(a03, ab);
      a25 = __ffma2_rn(ab, dup2(dy), a25);
    };
    if (act) {
      if (it == 1) {
        // integer start: every sample is a pixel (see the generic path)
        const float* gb =
            p.gimg + (size_t)(y0 + (int)prm[3] - M) * W + (x0 + (int)prm[0] + col - M);
#pragma unroll 4
        for (int r = row0; r < S; r += RPP)
          absorb(r * S + col, __ldg(gb + (size_t)r * W), (float)(r - M));
      } else {
        const WarpAffine wa(prm, x0, y0);
        const float2 la = __ffma2_rn(wa.a, dup2(fdx), wa.o);
#pragma unroll 2
        for (int r = row0; r < S; r += RPP) {
          const float dy = (float)(r - M);
          float2 t;
          const size_t cell = wa.locate_l(__ffma2_rn(wa.b, dup2(dy), la), W, H, t);
          float g;
          if (BIL) {
            float gx, gy;
            g = bilinear<false>(p.gimg, W, cell, t.x, t.y, gx, gy);
          } else {
            g = bicubic_q(p.gq, W, cell, t);
          }
          absorb(r * S + col, g, dy);
        }
      }
    }
    const float2 a14 = __fmul2_rn(a03, dup2(act ? fdx : 0.f));
    float acc[6];
    {
      float sums[8] = {s0s, s1s, a03.x, a14.x, a25.x, a03.y, a14.y, a25.y};
      warp_sum8(sums, lane);
      s0s = sums[0];
      s1s = sums[1];
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[k] = sums[k + 2];
    }
    const float gm = s0s * invN;  // gbar - c
    const float var = s1s - s0s * gm;
    const float dg = sqrtf(fmaxf(var, 0.f));
    if (!(dg > 0.f) || !isfinite(dg)) {
      st = kNonFinite;
      break;
    }
    float dp[6], rhs[6];
    const float ratio = df / dg;
#pragma unroll
    for (int a = 0; a < 6; ++a) rhs[a] = sbf[a] - ratio * (acc[a] - gm * ssd[a]);
    apply_hinv<TS>(hinv, rhs, lane, dp);
#pragma unroll
    for (int a = 0; a < 6; ++a) dp[a] = -dp[a];
    it_done = it;
    bool fin = true;
#pragma unroll
    for (int a = 0; a < 6; ++a) fin = fin && isfinite(dp[a]);
    if (!fin) {
      st = kNonFinite;
      break;
    }
    float pn[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) pn[a] = prm[a];
    compose_inverse(pn, dp);
    if (!corners_in_warp(pn, x0, y0, M, W, H, lane)) {
      st = kOutOfBounds;
      break;
    }
#pragma unroll
    for (int a = 0; a < 6; ++a) prm[a] = pn[a];
    const float nrm = sqrtf(dp[0] * dp[0] + dp[3] * dp[3] +
                            m2 * (dp[1] * dp[1] + dp[2] * dp[2] + dp[4] * dp[4] + dp[5] * dp[5]));
    if (nrm < p.tol) {
      zn = warp_sum(sfd) / (df * dg);
      have_zn = true;
      st = kOk;
      break;
    }
  }
  // ---- Eq. 1 at the returned shape (POIs that did not converge)
  if (!have_zn) {
    float s0s = 0.f, s1s = 0.f, sfg = 0.f;
    if (act) {
      for (int r = row0; r < S; r += RPP) {
        float tx, ty, gx, gy;
        const size_t cell = locate(prm, col - M, r - M, x0, y0, W, H, tx, ty);
        const float d = (BIL ? bilinear<false>(p.gimg, W, cell, tx, ty, gx, gy)
                             : bicubic<false>(p.gimg, W, cell, tx, ty, gx, gy)) - c;
        float2 gr;
        float fc;
        PS::unpack(spt[r * S + col], gr, fc);
        s0s += d;
        s1s = fmaf(d, d, s1s);
        sfg = fmaf(fc, d, sfg);
      }
    }
    s0s = warp_sum(s0s);
    s1s = warp_sum(s1s);
    sfg = warp_sum(sfg);
    const float var = s1s - s0s * s0s * invN;
    const float dgf = sqrtf(fmaxf(var, 0.f));
    zn = dgf > 0.f ? sfg / (df * dgf) : 0.f;
  }
  write_out(zn, it_done, st);
}

// Refinement of one POI by one warp; wsm is the warp's shared block.  BIL:
// bilinear interpolation of g (Eq. 5) instead of bicubic.
template <bool FANR, typename TS, typename TP, bool BIL = false>
__device__ __forceinline__ void subpixel_poi(const SubpixelParams& p, int64_t poi, int lane,
                                             unsigned char* wsm) {
  if constexpr (!FANR && sizeof(TP) == 1) {
    // subset widths whose rows fill a warp (or half of one): column layout
    if (p.S == 31) return icgn_col_poi<TS, 32, BIL>(p, poi, lane, wsm);
    if (p.S == 15) return icgn_col_poi<TS, 16, BIL>(p, poi, lane, wsm);
  }
  using PS = PointStore<TP>;
  using G = typename PS::T;
  const int S = p.S, M = p.M, N = S * S;
  const int x0 = M + p.R + 2 + (int)(poi % p.nx) * p.step;
  const int y0 = M + p.R + 2 + (int)(poi / p.nx) * p.step;
  const int W = p.W, H = p.H;
  G* spt = reinterpret_cast<G*>(wsm);
  TS* hinv = reinterpret_cast<TS*>(wsm + ((size_t)N * sizeof(G) + 15) / 16 * 16);
  float* ssd = reinterpret_cast<float*>(hinv + 36);  // sum SD
  float* sbf = ssd + 6;                              // sum SD (f - fbar)
  const TP* fimg = ref_ptr<TP>(p);
  // 8-bit pairs sample g from the BF16 tap quads (exact)
  constexpr bool kQuads = sizeof(TP) == 1;

  const uint8_t st0 = p.st0[poi];
  float prm[6] = {(float)p.u0[poi], 0.f, 0.f, (float)p.v0[poi], 0.f, 0.f};
  auto write_out = [&](float zn, int it, uint8_t st) {
    if (lane == 0) {
      p.u[poi] = prm[0];
      p.ux[poi] = prm[1];
      p.uy[poi] = prm[2];
      p.v[poi] = prm[3];
      p.vx[poi] = prm[4];
      p.vy[poi] = prm[5];
      p.zncc[poi] = zn;
      p.iters[poi] = it;
      p.status[poi] = st;
    }
  };
  if (st0 != kOk) {
    write_out(0.f, 0, st0);
    return;
  }

  // ---- reference subset: fbar, df, gradients (and for IC-GN the Hessian
  // and the constant sums of the right-hand side)
  float fsum = 0.f;
  {
    PtWalk w(lane, S, M);
    for (int i = lane; i < N; i += 32, w.next()) {
      const float f = pixel_value(fimg[(size_t)(y0 + w.dy) * p.pitch + (x0 + w.dx)]);
      fsum += f;
      spt[i] = PS::pack(p.grad[(size_t)(y0 + w.dy) * W + (x0 + w.dx)], f);
    }
  }
  fsum = warp_sum(fsum);  // exact for 8-bit images: integer sum below 2^24
  const float fbar = fsum / (float)N;
  float q = 0.f;
  // IC-GN: SD = (gx, gx dx, gx dy, gy, gy dx, gy dy) = (gx e, gy e) with
  // e = (1, dx, dy).  Packed pairs: sp[a] = (gx e_a, gy e_a); the xx and yy
  // blocks of H as pairs hp[ab] = (sum gx e_a gx e_b, sum gy e_a gy e_b),
  // a >= b; the xy block as scalars hxy[3a+b] = sum gy e_a gx e_b; the sums
  // of SD and of SD (f - fbar) as pairs.  Every entry is accumulated with
  // the same products and order as sd_a sd_b point by point.
  float2 hp[6], ssum[3], sfc[3];
  float hxy[9];
#pragma unroll
  for (int k = 0; k < 6; ++k) hp[k] = dup2(0.f);
#pragma unroll
  for (int k = 0; k < 3; ++k) ssum[k] = sfc[k] = dup2(0.f);
#pragma unroll
  for (int k = 0; k < 9; ++k) hxy[k] = 0.f;
  {
    PtWalk2 w(lane, S, M);
    for (int i = lane; i < N; i += 32, w.next()) {
      float2 gr;
      float f;
      PS::unpack(spt[i], gr, f);
      const float fc = f - fbar;
      q = fmaf(fc, fc, q);
      if (!FANR) {
        const float2 sp[3] = {gr, __fmul2_rn(gr, w.DX), __fmul2_rn(gr, w.DY)};
        const float2 fcc = dup2(fc);
        int k = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          ssum[a] = __fadd2_rn(ssum[a], sp[a]);
          sfc[a] = __ffma2_rn(sp[a], fcc, sfc[a]);
#pragma unroll
          for (int b = 0; b <= a; ++b, ++k) hp[k] = __ffma2_rn(sp[a], sp[b], hp[k]);
#pragma unroll
          for (int b = 0; b < 3; ++b) hxy[3 * a + b] = fmaf(sp[a].y, sp[b].x, hxy[3 * a + b]);
        }
      }
    }
  }
  if (!FANR) {
    // the 33 sums: H (21, packed lower, SD order), sum SD (6), sum SD (f -
    // fbar) (6).  A reduce-scatter over the warp leaves sum k on lane k for
    // the first 32; the last one and q are reduced whole.
    float v[32];
    {
      int k = 0;
      // rows 0..2 (xx block)
#pragma unroll
      for (int a = 0, t = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b, ++t) v[k++] = hp[t].x;
      // rows 3..5: xy block, then yy block
#pragma unroll
      for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b) v[k++] = hxy[3 * a + b];
#pragma unroll
        for (int b = 0; b <= a; ++b) v[k++] = hp[a * (a + 1) / 2 + b].y;
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) v[21 + a] = ssum[a].x, v[24 + a] = ssum[a].y;
#pragma unroll
      for (int a = 0; a < 3; ++a) v[27 + a] = sfc[a].x;
      v[30] = sfc[0].y;
      v[31] = sfc[1].y;
    }
    const float last = warp_sum(sfc[2].y);  // sum SD_5 (f - fbar)
    const float mine = reduce_scatter32(v, lane);
    q = warp_sum(q);
    const float df = sqrtf(q);
    if (!(df > 0.f)) {
      write_out(0.f, 0, kZeroVarRef);
      return;
    }
    if (lane >= 21 && lane < 27) ssd[lane - 21] = mine;
    if (lane >= 27) sbf[lane - 27] = mine;
    if (lane == 0) sbf[5] = last;
    // invert H once (in the solve precision), one lane per entry of its
    // lower triangle; H^-1 goes to shared memory and lane k < 6 reads row k
    // in every iteration, so an iteration's solve is six multiply-adds per
    // lane.
    if (!invert_to_smem<TS>(mine, lane, hinv)) {
      write_out(0.f, 0, kSingular);
      return;
    }
  } else {
    q = warp_sum(q);
  }
  const float df = sqrtf(q);
  if (!(df > 0.f)) {
    write_out(0.f, 0, kZeroVarRef);
    return;
  }
  if (!corners_in_warp(prm, x0, y0, M, W, H, lane)) {
    write_out(0.f, 0, kOutOfBounds);
    return;
  }

  const float c = fbar;
  const float invN = 1.f / (float)N;
  const float m2 = (float)M * (float)M;
  uint8_t st = kMaxIter;
  int it_done = 0;
  float zn = 0.f;
  bool have_zn = false;  // Eq. 1 already known (converged: at the last sampled shape)
  for (int it = 1; it <= p.max_iter; ++it) {
    float s0 = 0.f, s1 = 0.f, sfd = 0.f;
    float acc[FANR ? 39 : 6];
#pragma unroll
    for (int k = 0; k < (FANR ? 39 : 6); ++k) acc[k] = 0.f;
    // IC-GN sums in packed pairs: (SD0, SD3), (SD1, SD4), (SD2, SD5) . (g - c)
    float2 a03 = dup2(0.f), a14 = dup2(0.f), a25 = dup2(0.f);
    // one sample: g (and, for FA-NR, its gradient) at point i with packed
    // offsets (dx, dx), (dy, dy)
    auto absorb = [&](int i, float g, float gx, float gy, float2 DX, float2 DY) {
      const float d = g - c;
      s0 += d;
      s1 = fmaf(d, d, s1);
      float2 gr;
      float f;
      PS::unpack(spt[i], gr, f);
      const float fc = f - fbar;
      sfd = fmaf(fc, d, sfd);
      if (!FANR) {
        const float2 ab = __fmul2_rn(gr, dup2(d));  // (SD0, SD3) (g - c)
        a03 = __fadd2_rn(a03, ab);
        a14 = __ffma2_rn(ab, DX, a14);
        a25 = __ffma2_rn(ab, DY, a25);
      } else {
        const float fdx = DX.x, fdy = DY.x;
        const float J[6] = {gx, gx * fdx, gx * fdy, gy, gy * fdx, gy * fdy};
        int k = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int b = 0; b <= a; ++b, ++k) acc[k] = fmaf(J[a], J[b], acc[k]);  // 21 sums
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          acc[21 + a] = fmaf(J[a], d, acc[21 + a]);   // sum J (g - c)
          acc[27 + a] = fmaf(J[a], fc, acc[27 + a]);  // sum J (f - fbar)
          acc[33 + a] += J[a];                        // sum J
        }
      }
    };
    if (it == 1) {
      // The first iteration samples at the integer start (u0, v0) with zero
      // gradients: every sample lies on a pixel, where the Keys weights are
      // exactly (0, 1, 0, 0) and their derivatives (-1/2, 0, 1/2, 0), so the
      // interpolant is the pixel and its gradient the central differences --
      // bitwise what the interpolating path below computes, from one load
      // per sample (five for FA-NR).  With bilinear interpolation the patch
      // at a pixel gives the pixel and the forward differences (a10, a01).
      // The walk matches PtWalk2's.
      const float* gb = p.gimg + (size_t)(y0 + (int)prm[3]) * W + (x0 + (int)prm[0]);
      float2 DX = dup2((float)(lane % S - M)), DY = dup2((float)(lane / S - M));
      const float ddx = (float)(32 % S), ddy = (float)(32 / S), fM = (float)M, fS = (float)S;
      int off = (lane / S - M) * W + (lane % S - M);
      const int doff = (32 / S) * W + 32 % S, dwrap = W - S;
      // unrolled so that several samples' loads are in flight (measured:
      // IC-GN 4 -> 0.627 ms against 0.660 ms not unrolled, FA-NR 2)
      constexpr int kPixUnroll = FANR ? 2 : 4;
#pragma unroll kPixUnroll
      for (int i = lane; i < N; i += 32) {
        const float* gp = gb + off;
        float gx = 0.f, gy = 0.f;
        if (FANR && BIL) {
          gx = __ldg(gp + 1) - __ldg(gp);
          gy = __ldg(gp + W) - __ldg(gp);
        } else if (FANR) {
          gx = fmaf(0.5f, __ldg(gp + 1), -0.5f * __ldg(gp - 1));
          gy = fmaf(0.5f, __ldg(gp + W), -0.5f * __ldg(gp - W));
        }
        absorb(i, __ldg(gp), gx, gy, DX, DY);
        DX = __fadd2_rn(DX, dup2(ddx));
        DY = __fadd2_rn(DY, dup2(ddy));
        off += doff;
        if (DX.x > fM) {
          DX = __fadd2_rn(DX, dup2(-fS));
          DY = __fadd2_rn(DY, dup2(1.f));
          off += dwrap;
        }
      }
    } else if (FANR && (S == 31 || S == 15)) {
      // FA-NR in the column walk of the IC-GN column layout: lane c of each
      // group of LPR = S + 1 lanes owns column dx = c - M of every
      // (32 / LPR)-th row (the last lane of a group idles).  With dx
      // constant per lane, the 39 sums come from 21 per-lane moments in dy,
      // multiplied by the lane's dx once after the pass; the samples and
      // their positions are the generic walk's.
      const int LPR = S + 1, col = lane % LPR, RPP = 32 / LPR;
      if (col < S) {
        const float fdx = (float)(col - M), dxx = fdx * fdx;
        const WarpAffine wa(prm, x0, y0);
        const float2 la = __ffma2_rn(wa.a, dup2(fdx), wa.o);
        float2 q0 = dup2(0.f), q1 = dup2(0.f), q2 = dup2(0.f);  // (gx^2, gy^2) dy^0,1,2
        float c0 = 0.f, c1 = 0.f, c2 = 0.f;                      // gx gy dy^0,1,2
        float2 e0 = dup2(0.f), e1 = dup2(0.f);                   // (gx, gy) (g - c) dy^0,1
        float2 h0 = dup2(0.f), h1 = dup2(0.f);                   // (gx, gy) (f - fbar) dy^0,1
        float2 j0 = dup2(0.f), j1 = dup2(0.f);                   // (gx, gy) dy^0,1
#pragma unroll 2
        for (int r = lane / LPR; r < S; r += RPP) {
          const float dy = (float)(r - M);
          const float2 dy2 = dup2(dy);
          float2 t;
          const size_t cell = wa.locate_l(__ffma2_rn(wa.b, dy2, la), W, H, t);
          float gx, gy, g;
          if (BIL)
            g = bilinear<true>(p.gimg, W, cell, t.x, t.y, gx, gy);
          else if (kQuads)
            g = bicubic_q_grad(p.gq, W, cell, t.x, t.y, gx, gy);
          else
            g = bicubic<true>(p.gimg, W, cell, t.x, t.y, gx, gy);
          const float d = g - c;
          s0 += d;
          s1 = fmaf(d, d, s1);
          float2 gr;
          float f;
          PS::unpack(spt[r * S + col], gr, f);
          const float fc = f - fbar;
          sfd = fmaf(fc, d, sfd);
          const float2 gg = make_float2(gx, gy);
          const float2 sq = __fmul2_rn(gg, gg), sqdy = __fmul2_rn(sq, dy2);
          q0 = __fadd2_rn(q0, sq);
          q1 = __fadd2_rn(q1, sqdy);
          q2 = __ffma2_rn(sqdy, dy2, q2);
          const float cx = gx * gy, cxdy = cx * dy;
          c0 += cx;
          c1 += cxdy;
          c2 = fmaf(cxdy, dy, c2);
          const float2 gd = __fmul2_rn(gg, dup2(d));
          e0 = __fadd2_rn(e0, gd);
          e1 = __ffma2_rn(gd, dy2, e1);
          const float2 gf = __fmul2_rn(gg, dup2(fc));
          h0 = __fadd2_rn(h0, gf);
          h1 = __ffma2_rn(gf, dy2, h1);
          j0 = __fadd2_rn(j0, gg);
          j1 = __ffma2_rn(gg, dy2, j1);
        }
        // J = (gx, gx dx, gx dy, gy, gy dx, gy dy): J^T J (lower triangle,
        // row by row), then sum J (g - c), sum J (f - fbar), sum J
        acc[0] = q0.x; acc[1] = fdx * q0.x; acc[2] = dxx * q0.x;
        acc[3] = q1.x; acc[4] = fdx * q1.x; acc[5] = q2.x;
        acc[6] = c0; acc[7] = fdx * c0; acc[8] = c1; acc[9] = q0.y;
        acc[10] = fdx * c0; acc[11] = dxx * c0; acc[12] = fdx * c1; acc[13] = fdx * q0.y;
        acc[14] = dxx * q0.y;
        acc[15] = c1; acc[16] = fdx * c1; acc[17] = c2; acc[18] = q1.y; acc[19] = fdx * q1.y;
        acc[20] = q2.y;
        acc[21] = e0.x; acc[22] = fdx * e0.x; acc[23] = e1.x;
        acc[24] = e0.y; acc[25] = fdx * e0.y; acc[26] = e1.y;
        acc[27] = h0.x; acc[28] = fdx * h0.x; acc[29] = h1.x;
        acc[30] = h0.y; acc[31] = fdx * h0.y; acc[32] = h1.y;
        acc[33] = j0.x; acc[34] = fdx * j0.x; acc[35] = j1.x;
        acc[36] = j0.y; acc[37] = fdx * j0.y; acc[38] = j1.y;
      }
    } else {
      const WarpAffine wa(prm, x0, y0);
      PtWalk2 w(lane, S, M);
#pragma unroll kPointUnroll
      for (int i = lane; i < N; i += 32, w.next()) {
        float2 t;
        float gx = 0.f, gy = 0.f;
        const size_t cell = wa.locate(w.DX, w.DY, W, H, t);
        float g;
        if (BIL)
          g = bilinear<FANR>(p.gimg, W, cell, t.x, t.y, gx, gy);
        else if (FANR && kQuads)
          g = bicubic_q_grad(p.gq, W, cell, t.x, t.y, gx, gy);
        else if (FANR)
          g = bicubic<true>(p.gimg, W, cell, t.x, t.y, gx, gy);
        else if (kQuads)
          g = bicubic_q(p.gq, W, cell, t);
        else
          g = bicubic2(p.gimg, W, cell, t);
        absorb(i, g, gx, gy, w.DX, w.DY);
      }
    }
    if (!FANR) {
      acc[0] = a03.x;
      acc[1] = a14.x;
      acc[2] = a25.x;
      acc[3] = a03.y;
      acc[4] = a14.y;
      acc[5] = a25.y;
    }
    // IC-GN: s0, s1 and the six sums together (warp_sum8).  FA-NR: the
    // first 32 of its 39 sums by a reduce-scatter (sum k on lane k: J^T J
    // on lanes 0..20, sum J (g - c) on 21..26, sum J (f - fbar) of J_0..J_4
    // on 27..31), s0, s1 and six of the other 7 together, the last whole
    float fa_mine = 0.f;
    {
      const int k0 = FANR ? 32 : 0;
      float sums[8] = {s0, s1, acc[k0], acc[k0 + 1], acc[k0 + 2], acc[k0 + 3], acc[k0 + 4],
                       acc[k0 + 5]};
      if constexpr (FANR) {
        float v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = acc[k];
        fa_mine = reduce_scatter32(v, lane);
        acc[38] = warp_sum(acc[38]);
      }
      warp_sum8(sums, lane);
      s0 = sums[0];
      s1 = sums[1];
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[k0 + k] = sums[k + 2];
    }
    const float gm = s0 * invN;  // gbar - c
    const float var = s1 - s0 * gm;
    const float dg = sqrtf(fmaxf(var, 0.f));
    if (!(dg > 0.f) || !isfinite(dg)) {
      st = kNonFinite;
      break;
    }
    float dp[6], rhs[6];
    bool ok;
    if (!FANR) {
      const float ratio = df / dg;
#pragma unroll
      for (int a = 0; a < 6; ++a) rhs[a] = sbf[a] - ratio * (acc[a] - gm * ssd[a]);
      apply_hinv<TS>(hinv, rhs, lane, dp);
#pragma unroll
      for (int a = 0; a < 6; ++a) dp[a] = -dp[a];
      ok = true;
    } else {
      // rhs_a = ratio sum J_a (f - fbar) - (sum J_a (g - c) - gm sum J_a),
      // formed on lane 21 + a, then broadcast
      const float ratio = dg / df;
      const float jf = __shfl_sync(0xffffffffu, fa_mine, min(lane + 6, 31));
      float r = 0.f;
      if (lane >= 21 && lane < 27) {
        const int a = lane - 21;
        float sj = acc[33];
#pragma unroll
        for (int b = 1; b < 6; ++b) sj = a == b ? acc[33 + b] : sj;
        r = ratio * (a < 5 ? jf : acc[32]) - (fa_mine - gm * sj);
      }
#pragma unroll
      for (int a = 0; a < 6; ++a) rhs[a] = __shfl_sync(0xffffffffu, r, 21 + a);
      // dp = (J^T J)^-1 rhs: the sweep inverse (solve precision) into shared
      // memory, lane k < 6 forms row k . rhs
      ok = invert_to_smem<TS>(fa_mine, lane, hinv);
      if (!ok) {
        it_done = it;
        st = kSingular;
        break;
      }
      apply_hinv<TS>(hinv, rhs, lane, dp);
    }
    it_done = it;
    bool fin = true;
#pragma unroll
    for (int a = 0; a < 6; ++a) fin = fin && isfinite(dp[a]);
    if (!fin) {
      st = kNonFinite;
      break;
    }
    float pn[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) pn[a] = prm[a];
    if (!FANR) {
      compose_inverse(pn, dp);
    } else {
#pragma unroll
      for (int a = 0; a < 6; ++a) pn[a] += dp[a];
    }
    if (!corners_in_warp(pn, x0, y0, M, W, H, lane)) {
      st = kOutOfBounds;
      break;
    }
#pragma unroll
    for (int a = 0; a < 6; ++a) prm[a] = pn[a];
    const float nrm = sqrtf(dp[0] * dp[0] + dp[3] * dp[3] +
                            m2 * (dp[1] * dp[1] + dp[2] * dp[2] + dp[4] * dp[4] + dp[5] * dp[5]));
    if (nrm < p.tol) {
      // Eq. 1 at this iteration's sampled shape: sum fc (g - gbar) =
      // sum fc (g - c) because sum fc = 0.  The returned shape differs from it
      // by the last update (|dp| < tol), where C is stationary, so the two
      // values differ by O(|dp|^2): below 1e-7 for tol = 1e-3.
      zn = warp_sum(sfd) / (df * dg);
      have_zn = true;
      st = kOk;
      break;
    }
  }

  // ---- Eq. 1 at the returned shape (POIs that did not converge)
  if (!have_zn) {
    float s0 = 0.f, s1 = 0.f, sfg = 0.f;
    PtWalk w(lane, S, M);
    for (int i = lane; i < N; i += 32, w.next()) {
      float tx, ty, gx, gy;
      const size_t cell = locate(prm, w.dx, w.dy, x0, y0, W, H, tx, ty);
      const float d = (BIL ? bilinear<false>(p.gimg, W, cell, tx, ty, gx, gy)
                           : bicubic<false>(p.gimg, W, cell, tx, ty, gx, gy)) - c;
      float2 gr;
      float f;
      PS::unpack(spt[i], gr, f);
      s0 += d;
      s1 = fmaf(d, d, s1);
      sfg = fmaf(f - fbar, d, sfg);
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    sfg = warp_sum(sfg);
    const float var = s1 - s0 * s0 * invN;
    const float dgf = sqrtf(fmaxf(var, 0.f));
    // sum fc (g - gbar) = sum fc (g - c) because sum fc = 0
    zn = dgf > 0.f ? sfg / (df * dgf) : 0.f;
  }
  write_out(zn, it_done, st);
}

// One warp per POI of one pair.
template <bool FANR, typename TS, typename TP, bool BIL>
__global__ void __launch_bounds__(32 * kWarpsPerCta, FANR ? DIC_SUB_MINB_NR : DIC_SUB_MINB)
subpixel_kernel(const SubpixelParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t poi = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
  if (poi >= p.n_pois) return;
  const size_t wb = warp_smem_bytes(p.S * p.S, sizeof(typename PointStore<TP>::T));
  subpixel_poi<FANR, TS, TP, BIL>(p, poi, lane, smem + (size_t)wid * wb);
}

// Persistent form over many pairs: every warp repeatedly takes the next POI
// of the batch from a global counter, so POIs with many iterations do not
// hold back a whole CTA.  nmax = largest subset size N of the batch.
// resident warps per SM the persistent kernel asks the register allocator
// for (as the single-pair kernel: 20 for IC-GN, 15 for FA-NR)
template <bool FANR, int WPC>
constexpr int batch_min_blocks() {
  return (FANR ? 15 : 20) / WPC > 1 ? (FANR ? 15 : 20) / WPC : 1;
}

template <bool FANR, typename TS, int WPC>
__global__ void __launch_bounds__(32 * WPC, batch_min_blocks<FANR, WPC>())
subpixel_batch_kernel(const SubpixelParams* __restrict__ jobs,
                      const int64_t* __restrict__ offsets, int njobs, int nmax,
                      unsigned long long* counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // batches hold 8-bit pairs only
  unsigned char* wsm =
      smem + (size_t)wid * warp_smem_bytes(nmax, sizeof(PointStore<uint8_t>::T));
  const int64_t total = offsets[njobs];
  for (;;) {
    long long item = 0;
    if (lane == 0) item = (long long)atomicAdd(counter, 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= total) break;
    int lo = 0, hi = njobs;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (offsets[mid] <= item) lo = mid; else hi = mid;
    }
    subpixel_poi<FANR, TS, uint8_t>(jobs[lo], item - offsets[lo], lane, wsm);
    __syncwarp();
  }
}

template <bool FANR, typename TS, typename TP, bool BIL>
cudaError_t launch_one(const SubpixelParams& p, cudaStream_t st) {
  // kWarpsPerCta warps per CTA, fewer where the subset's shared memory
  // would not fit (large subsets)
  const size_t wb = warp_smem_bytes(p.S * p.S, sizeof(typename PointStore<TP>::T));
  int wpc = kWarpsPerCta;
  while (wpc > 1 && (size_t)wpc * wb > 227 * 1024) wpc >>= 1;
  const size_t smem = (size_t)wpc * wb;
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  if (smem > 48 * 1024) {
    // the limit, not this launch's size: a graph may hold launches of
    // several subset sizes, each checked against the attribute when it runs
    cudaError_t e = cudaFuncSetAttribute(subpixel_kernel<FANR, TS, TP, BIL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
  }
  const unsigned grid = (unsigned)((p.n_pois + wpc - 1) / wpc);
  subpixel_kernel<FANR, TS, TP, BIL><<<grid, 32 * wpc, smem, st>>>(p);
  return cudaGetLastError();
}

template <bool FANR, typename TS, int WPC>
cudaError_t launch_batch_one(const SubpixelParams* jobs, const int64_t* offsets, int njobs,
                             int nmax, unsigned long long* counter, int grid, cudaStream_t st) {
  const size_t smem = (size_t)WPC * warp_smem_bytes(nmax, sizeof(PointStore<uint8_t>::T));
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(subpixel_batch_kernel<FANR, TS, WPC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (grid <= 0) {  // (resident CTAs x SMs) x max(1, -grid)
    int occ = 0, dev = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, subpixel_batch_kernel<FANR, TS, WPC>,
                                                  32 * WPC, smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = (occ > 0 ? occ : 1) * sms * (grid < 0 ? -grid : 1);
  }
  subpixel_batch_kernel<FANR, TS, WPC><<<grid, 32 * WPC, smem, st>>>(jobs, offsets, njobs, nmax,
                                                                    counter);
  return cudaGetLastError();
}

template <bool FANR, typename TS>
cudaError_t launch_batch_wpc(int wpc, const SubpixelParams* jobs, const int64_t* offsets,
                             int njobs, int nmax, unsigned long long* counter, int grid,
                             cudaStream_t st) {
  switch (wpc) {
    case 2: return launch_batch_one<FANR, TS, 2>(jobs, offsets, njobs, nmax, counter, grid, st);
    case 4: return launch_batch_one<FANR, TS, 4>(jobs, offsets, njobs, nmax, counter, grid, st);
    case 8: return launch_batch_one<FANR, TS, 8>(jobs, offsets, njobs, nmax, counter, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_subpixel_batch(const SubpixelParams* jobs, const int64_t* offsets, int njobs,
                                  int nmax, int method, int solve_fp64, int wpc,
                                  unsigned long long* counter, int grid, cudaStream_t st) {
  if (method == DIC_ICGN)
    return solve_fp64 ? launch_batch_wpc<false, double>(wpc, jobs, offsets, njobs, nmax, counter,
                                                        grid, st)
                      : launch_batch_wpc<false, float>(wpc, jobs, offsets, njobs, nmax, counter,
                                                       grid, st);
  return solve_fp64 ? launch_batch_wpc<true, double>(wpc, jobs, offsets, njobs, nmax, counter,
                                                     grid, st)
                    : launch_batch_wpc<true, float>(wpc, jobs, offsets, njobs, nmax, counter,
                                                    grid, st);
}

template <bool BIL>
cudaError_t launch_interp(const SubpixelParams& p, int method, int solve_fp64, cudaStream_t st) {
  if (p.ref_f32) {
    if (method == DIC_ICGN)
      return solve_fp64 ? launch_one<false, double, float, BIL>(p, st)
                        : launch_one<false, float, float, BIL>(p, st);
    return solve_fp64 ? launch_one<true, double, float, BIL>(p, st)
                      : launch_one<true, float, float, BIL>(p, st);
  }
  if (method == DIC_ICGN)
    return solve_fp64 ? launch_one<false, double, uint8_t, BIL>(p, st)
                      : launch_one<false, float, uint8_t, BIL>(p, st);
  return solve_fp64 ? launch_one<true, double, uint8_t, BIL>(p, st)
                    : launch_one<true, float, uint8_t, BIL>(p, st);
}

cudaError_t launch_subpixel(const SubpixelParams& p, int method, int solve_fp64,
                            cudaStream_t st, int bilinear) {
  if (p.n_pois == 0) return cudaSuccess;
  if (!p.ref_f32 && !p.gq) return cudaErrorInvalidValue;  // 8-bit pairs need the tap quads
  return bilinear ? launch_interp<true>(p, method, solve_fp64, st)
                  : launch_interp<false>(p, method, solve_fp64, st);
}

}  // namespace dic
