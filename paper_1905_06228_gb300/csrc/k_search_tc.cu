// k_search_tc.cu -- brute-force ZNCC integer search (Eq. 1, Section 2.1) as
// a BF16 tensor-core contraction (tcgen05, TMEM accumulators).
//
// Correlation sums as one implicit GEMM across POIs.  Let a "position" be an
// absolute top-left corner (Y, X) of a subset in the deformed image; POI p
// (top-left (yp-M, xp-M)) needs every position with |Y-(yp-M)|, |X-(xp-M)|
// <= R.  For a tile of 128 positions (16 rows x 8 columns) and the N POIs
// whose windows meet the tile:
//
//   D[m][n] = sum_ty sum_tx  G[Y0+q+ty][X0+r+tx] * T_n[ty][tx],   m = 8q + r
//
// A (M = 128 positions x K = taps) is read through a K-major no-swizzle
// shared-memory descriptor from eight shifted copies of each image row
// (core matrix = 8 positions x 8 taps), so the step ty -> ty+1 is only a
// descriptor offset of one image row; B (N POIs x K) is the ty-th template
// row of every POI, streamed per ty from a template bank with cp.async.
// Both operands use 128-byte 8-tap blocks (LBO = 128 B) and 8-row groups of
// one row's blocks (SBO = TWK/8 * 128 B).
// One tcgen05.mma.kind::f16 (BF16 x BF16 -> FP32, M=128, N<=256, K=16) per
// 16 taps; the accumulator lives in TMEM.
//
// Exactness: a = f-128 and b = g-128 are integers in [-128, 127], exact in
// BF16; |ab| <= 2^14, so any sum of at most 1024 products is an integer
// below 2^24 and the FP32 accumulation is exact.  Subsets wider than 32 use
// several accumulators (blocks of floor(1024/TWK) template rows), added in
// int32 by the epilogue.  The candidate scores then use the same exact
// integers as the FP32 form: num = N Sab - Sa Sb, Dg = N Sbb - Sb^2, with
// Sa, Saa per POI and Sb, Sbb per position (box sums of the tile).
//
// Epilogue: TMEM -> registers -> shared memory (transposed), then thread n
// scans the 128 positions for POI n and keeps the exact best (float
// pre-filter, exact 128-bit comparison, lowest linear index on ties).  Each
// (tile, POI) best goes to a slot; a final kernel reduces a POI's slots
// exactly and re-ranks its top four candidates by recomputing their sums on
// the CUDA cores from the images, so the integer result is bit-identical to
// the FP32 form and to the oracle.
#include <algorithm>

#include "dic_internal.cuh"

namespace dic {
namespace {

constexpr int kThreads = 256;
constexpr int kTileQ = 16;  // position rows per tile
constexpr int kTileR = 8;   // position columns per tile
constexpr int kStages = 3;  // template-row stages in flight

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// 64-bit shared-memory matrix descriptor: K-major, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;               // base offset 0, relative LBO, layout "no swizzle" (0)
}

// Instruction descriptor: kind::f16, BF16 A and B, FP32 D, both K-major.
__host__ __device__ __forceinline__ uint32_t make_idesc(int M, int N) {
  return (1u << 4)                     // D format: F32
         | (1u << 7)                   // A format: BF16
         | (1u << 10)                  // B format: BF16
         | ((uint32_t)(N >> 3) << 17)  // N / 8
         | ((uint32_t)(M >> 4) << 24); // M / 16
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
  for (long long i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

struct Cand {
  long long num, dg;
  int l;
};

// float of an exact 64-bit integer without the 64-bit conversion (which runs
// on the FP64 pipe): hi * 2^32 + lo, relative error ~1e-7
__device__ __forceinline__ float ll_to_float(long long v) {
  const int hi = (int)(v >> 32);
  const unsigned lo = (unsigned)(v & 0xffffffffll);
  return fmaf((float)hi, 4294967296.0f, (float)lo);
}

__device__ __forceinline__ bool zncc_greater(long long na, long long da, long long nb,
                                             long long db) {
  if (na >= 0 && nb < 0) return true;
  if (na < 0 && nb >= 0) return false;
  unsigned long long aa = (unsigned long long)(na < 0 ? -na : na);
  unsigned long long ab = (unsigned long long)(nb < 0 ? -nb : nb);
  unsigned __int128 lhs = (unsigned __int128)aa * aa * (unsigned __int128)(unsigned long long)db;
  unsigned __int128 rhs = (unsigned __int128)ab * ab * (unsigned __int128)(unsigned long long)da;
  return na >= 0 ? (lhs > rhs) : (lhs < rhs);
}

__device__ __forceinline__ bool cand_better(const Cand& a, const Cand& b) {
  if (a.l == INT_MAX) return false;
  if (b.l == INT_MAX) return true;
  if (zncc_greater(a.num, a.dg, b.num, b.dg)) return true;
  if (zncc_greater(b.num, b.dg, a.num, a.dg)) return false;
  return a.l < b.l;
}

// ------------------------------------------------------------ phase images
// Eight copies of each image shifted by s = 0..7 pixels, as centred BF16:
//   ph[img][s][y][c] = I[y][c + s] - 128  (0 outside the image)
// so that any run of 8 consecutive pixels starting at column x is one
// aligned 16-byte chunk: copy s = x mod 8 at column x - s.  One thread per
// 16-byte chunk.
__global__ void phase_kernel(const SearchTcParams p) {
  const int64_t chunk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int cpr = p.phw / 8;  // chunks per row
  const int64_t per_img = (int64_t)8 * p.phh * cpr;
  if (chunk >= 2 * per_img) return;
  const int im = (int)(chunk / per_img);
  int64_t rem = chunk % per_img;
  const int sft = (int)(rem / ((int64_t)p.phh * cpr));
  rem %= (int64_t)p.phh * cpr;
  const int y = (int)(rem / cpr), c = (int)(rem % cpr) * 8;
  const uint8_t* src = im ? p.def : p.ref;
  uint32_t w[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    uint32_t h2[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int x = c + sft + 2 * e + k;
      const int v = (x < p.W && y < p.H) ? (int)src[(size_t)y * p.pitch + x] - 128 : 0;
      h2[k] = __float_as_uint((float)v) >> 16;  // small integers are exact in BF16
    }
    w[e] = h2[0] | (h2[1] << 16);
  }
  uint16_t* dst = (im ? p.gph : p.fph) + ((size_t)sft * p.phh + y) * p.phw + c;
  *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
}

// ------------------------------------------------------------ box-sum map
// posbox[py*pw + px] = (sum b, sum b^2) over the S x S subset whose top-left
// is the position (ymin+py, xmin+px); b = g - 128, 0 outside the image.
// 32 x 32 positions per CTA, separable sums through shared memory.
constexpr int kBoxT = 32;
__global__ void __launch_bounds__(256) boxmap_kernel(const SearchTcParams p, int which) {
  const uint8_t* img = which ? p.def : p.ref;
  int2* out = which ? p.posbox : p.fbox;
  extern __shared__ __align__(16) unsigned char smem[];
  const int S = p.S, span = kBoxT + S - 1;
  int* rowb = reinterpret_cast<int*>(smem);          // [span][span] bytes - 128
  int2* hs = reinterpret_cast<int2*>(rowb + span * span);  // [span][kBoxT]
  const int px0 = blockIdx.x * kBoxT, py0 = blockIdx.y * kBoxT;
  const int X0 = p.xmin + px0, Y0 = p.ymin + py0;
  for (int i = threadIdx.x; i < span * span; i += blockDim.x) {
    const int r = i / span, c = i % span, y = Y0 + r, x = X0 + c;
    rowb[i] = (x >= 0 && x < p.W && y >= 0 && y < p.H)
                  ? (int)img[(size_t)y * p.pitch + x] - 128 : 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < span * kBoxT; i += blockDim.x) {
    const int r = i / kBoxT, c = i % kBoxT;
    int a = 0, b = 0;
    for (int t = 0; t < S; ++t) {
      const int v = rowb[r * span + c + t];
      a += v;
      b += v * v;
    }
    hs[i] = make_int2(a, b);
  }
  __syncthreads();
  const int pw = p.ntx * 8;
  for (int i = threadIdx.x; i < kBoxT * kBoxT; i += blockDim.x) {
    const int r = i / kBoxT, c = i % kBoxT;
    if (py0 + r >= p.nty * 16 || px0 + c >= pw) continue;
    int a = 0, b = 0;
    for (int t = 0; t < S; ++t) {
      const int2 v = hs[(r + t) * kBoxT + c];
      a += v.x;
      b += v.y;
    }
    out[(size_t)(py0 + r) * pw + (px0 + c)] = make_int2(a, b);
  }
}

// ------------------------------------------------------------ tile kernel
struct TileLayout {
  int rows;    // image rows of the tile: kTileQ + S - 1
  int KB;      // 8-tap blocks per template row: TWK / 8
  int sboA;    // bytes per image row in the A buffer: KB * 128
  int stageB;  // bytes per template-row stage: KB * Npad * 16 (8-row groups of KB*128)
  size_t off_bar, off_tmem, off_pos, off_a, off_b, off_d, total;
};

__host__ __device__ inline size_t al(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline TileLayout tile_layout(int S, int TWK, int npad) {
  TileLayout L;
  L.rows = kTileQ + S - 1;
  L.KB = TWK / 8;
  L.sboA = L.KB * 128;
  L.stageB = L.KB * npad * 16;
  size_t o = 0;
  L.off_bar = o;  o += 8 * (kStages + 1);
  L.off_tmem = o; o += 8;
  o = al(o, 16);  L.off_pos = o;  o += (size_t)kTileQ * kTileR * 16;  // dg, sb, 1/dg
  o = al(o, 128);
  // A buffer and B stages; the transposed accumulator reuses this region
  // once the last MMA has completed
  const size_t ab = (size_t)L.rows * L.sboA + (size_t)kStages * L.stageB;
  const size_t dd = (size_t)npad * (kTileQ * kTileR + 1) * 4;
  L.off_a = o;
  L.off_b = o + (size_t)L.rows * L.sboA;
  L.off_d = o;
  o += ab > dd ? ab : dd;
  L.total = o;
  return L;
}

__global__ void __launch_bounds__(kThreads, 3) tile_kernel(const SearchTcParams p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = p.S, M = p.M, R = p.R, TWK = p.twk, NP = p.npad;
  const TileLayout L = tile_layout(S, TWK, NP);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.off_bar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.off_tmem);
  long long* pdg = reinterpret_cast<long long*>(smem + L.off_pos);  // Dg per position
  int* psb = reinterpret_cast<int*>(pdg + kTileQ * kTileR);            // Sb per position
  float* pinv = reinterpret_cast<float*>(psb + kTileQ * kTileR);       // 1 / Dg
  unsigned char* abuf = smem + L.off_a;
  unsigned char* bbuf = smem + L.off_b;
  int* dsm = reinterpret_cast<int*>(smem + L.off_d);

  // tile origin (absolute positions) and its POI block
  const int tile = blockIdx.x;
  const int X0 = p.xmin + (tile % p.ntx) * kTileR;
  const int Y0 = p.ymin + (tile / p.ntx) * kTileQ;
  const int B = M + R + 2;
  // POI column k is met iff x_k - M - R <= X0 + 7 and x_k - M + R >= X0
  auto ceil_div = [](int a, int b) { return a >= 0 ? (a + b - 1) / b : -((-a) / b); };
  auto floor_div = [](int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
  const int kc0 = max(0, ceil_div(X0 + M - R - B, p.step));
  const int kr0 = max(0, ceil_div(Y0 + M - R - B, p.step));
  const int kc1 = min(p.nx - 1, floor_div(X0 + kTileR - 1 + M + R - B, p.step));
  const int kr1 = min(p.ny - 1, floor_div(Y0 + kTileQ - 1 + M + R - B, p.step));

  // ---- setup: barriers, TMEM allocation (warp 0)
  const uint32_t ncols = p.tmem_cols;
  if (tid == 0) {
    for (int i = 0; i <= kStages; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[i])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // ---- per-position box statistics (from the map)
  const long long N = (long long)S * S;
  if (tid < kTileQ * kTileR) {
    const int q = tid / kTileR, r = tid % kTileR;
    const int2 bx = p.posbox[(size_t)(Y0 - p.ymin + q) * (p.ntx * 8) + (X0 - p.xmin + r)];
    const long long dg = N * (long long)bx.y - (long long)bx.x * bx.x;
    pdg[tid] = dg;
    psb[tid] = bx.x;
    pinv[tid] = dg ? 1.0f / ll_to_float(dg) : 0.f;
  }
  // ---- A buffer: eight shifted copies per image row and 8-tap block,
  //   abuf[row*sboA + kb*128 + r*16 + e*2] = g[Y0+row][X0 + r + 8kb + e] - 128,
  // one aligned 16-byte chunk of phase image (X0 + r) mod 8 each; taps at or
  // beyond S are zero-filled (the template's padding)
  for (int i = tid; i < L.rows * L.KB * 8; i += kThreads) {
    const int row = i / (L.KB * 8), rem = i % (L.KB * 8), kb = rem >> 3, r = rem & 7;
    const int x = X0 + r + 8 * kb, sft = x & 7;
    const uint16_t* src = p.gph + ((size_t)sft * p.phh + (Y0 + row)) * p.phw + (x - sft);
    const int valid = min(max(S - 8 * kb, 0), 8);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(
                     smem_u32(abuf + row * L.sboA + kb * 128 + r * 16)),
                 "l"(src), "r"(2 * valid)
                 : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // ---- main loop over template rows: B(ty) streams two rows ahead of the
  // MMAs; a stage is refilled once the MMAs that read it have committed
  const int nbr = kr1 - kr0 + 1, nbc = kc1 - kc0 + 1;
  const uint32_t idesc = make_idesc(128, NP);
  const int rows_per_acc = p.rows_per_acc;
  // this thread's 16-byte copies (same for every ty): POI n of the block,
  // 8-tap block kb; at most NP*KB/256 <= 8 per thread
  constexpr int kMaxCopies = 8;
  const uint16_t* csrc[kMaxCopies];
  uint32_t cdst[kMaxCopies], cbytes[kMaxCopies];
  int ncopy = 0;
  for (int i = tid; i < NP * L.KB && ncopy < kMaxCopies; i += kThreads, ++ncopy) {
    const int n = i % NP, kb = i / NP;
    const int bi = n / p.ncols_max, bj = n % p.ncols_max;
    const bool have = n < p.nrows_max * p.ncols_max && bi < nbr && bj < nbc;
    // template row ty of POI (kr, kc): f[yl + ty][xl + 8kb .. +7]
    const int xl = have ? B + (kc0 + bj) * p.step - M : 0;
    const int yl = have ? B + (kr0 + bi) * p.step - M : 0;
    const int x = xl + 8 * kb, sft = x & 7;
    csrc[ncopy] = p.fph + ((size_t)sft * p.phh + yl) * p.phw + (x - sft);
    cdst[ncopy] = (uint32_t)((n >> 3) * L.KB * 128 + kb * 128 + (n & 7) * 16);
    cbytes[ncopy] = have ? 16u : 0u;
  }
  const uint32_t bbase = smem_u32(bbuf);
  auto issue_b = [&](int row) {
    const uint32_t stage = bbase + (uint32_t)((row % kStages) * L.stageB);
    for (int k = 0; k < ncopy; ++k)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(stage + cdst[k]),
                   "l"(csrc[k] + (size_t)row * p.phw), "r"(cbytes[k])
                   : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  int failed = 0;
  issue_b(0);
  if (S > 1) issue_b(1);
  for (int ty = 0; ty < S; ++ty) {
    if (ty + 1 < S)
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    else
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int acc = ty / rows_per_acc;
      const uint32_t dcol = tmem + (uint32_t)(acc * NP);
      const uint32_t a_base = smem_u32(abuf) + (uint32_t)(ty * L.sboA);
      const uint32_t b_base = bbase + (uint32_t)((ty % kStages) * L.stageB);
      for (int j = 0; j < TWK / 16; ++j) {
        const uint64_t ad = make_desc(a_base + j * 256, 128, (uint32_t)L.sboA);
        const uint64_t bd = make_desc(b_base + j * 256, 128, (uint32_t)L.sboA);
        const uint32_t accum = (ty % rows_per_acc == 0 && j == 0) ? 0u : 1u;
        asm volatile(
            "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(dcol),
            "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&bars[ty % kStages]))
          : "memory");
    }
    if (ty + 2 < S) {
      // stage (ty+2) % 3 was read by the MMAs of row ty-1: one thread polls
      // their commit, the others sleep at the barrier
      if (ty >= 1) {
        if (tid == 0) {
          const int prev = ty - 1;
          const uint32_t par = (uint32_t)((prev / kStages) & 1);
          if (!mbar_wait(smem_u32(&bars[prev % kStages]), par, 1ll << 26)) failed = 1;
        }
        __syncthreads();
      }
      issue_b(ty + 2);
    }
  }
  bool ok = !__syncthreads_or(failed);
  // all MMAs done: commit once more on the last barrier and wait
  if (ok && tid == 0) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&bars[kStages]))
        : "memory");
  }
  {
    const int failed = (ok && tid == 0) ? !mbar_wait(smem_u32(&bars[kStages]), 0, 1ll << 26) : 0;
    if (__syncthreads_or(failed)) ok = false;
  }
  if (!ok) {
    if (tid == 0) {
      atomicOr(p.err_flag, 2u);
      // give in-flight tensor-core work a bounded chance to finish
      mbar_wait(smem_u32(&bars[kStages]), 0, 1ll << 24);
    }
    __syncthreads();
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // ---- accumulators -> shared memory, transposed: dsm[n][m] (int32 sums)
  const int nacc = (S + rows_per_acc - 1) / rows_per_acc;
  if (ok) {
    const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
    const int m = quarter * 32 + lane;
    for (int c0 = (warp >> 2) * 16; c0 < NP; c0 += (kThreads / 128) * 16) {
      int sum[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) sum[k] = 0;
      for (int a = 0; a < nacc; ++a) {
        uint32_t v[16];
        const uint32_t addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(a * NP + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
              "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
              "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(addr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int k = 0; k < 16; ++k) sum[k] += __float2int_rn(__uint_as_float(v[k]));
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) dsm[(c0 + k) * (kTileQ * kTileR + 1) + m] = sum[k];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
  }
  if (!ok) return;

  // ---- per-POI scan of the tile's positions (two threads per POI when the
  // block has at most 128 POIs: even and odd position rows)
  const int split = NP <= kThreads / 2 ? 2 : 1;
  const int n = tid / split, half = tid % split;
  const bool active = n < NP;
  const int bi = active ? n / p.ncols_max : 0, bj = active ? n % p.ncols_max : 0;
  const bool valid_poi =
      active && n < p.nrows_max * p.ncols_max && bi < nbr && bj < nbc;
  const int kr = kr0 + bi, kc = kc0 + bj;
  const int64_t poi = (int64_t)kr * p.nx + kc;
  const int xl = B + kc * p.step - M, yl = B + kr * p.step - M;  // POI's subset top-left
  const int ow = 2 * R + 1;
  Cand best{0, 1, INT_MAX};
  if (valid_poi) {
    const int2 fb = p.fbox[(size_t)(yl - p.ymin) * (p.ntx * 8) + (xl - p.xmin)];
    const long long sa = fb.x;
    float best_f = -3.0e38f;
    const int* drow = dsm + n * (kTileQ * kTileR + 1);
    const int r_lo = max(0, xl - R - X0), r_hi = min(kTileR - 1, xl + R - X0);
    const int q_lo = max(0, yl - R - Y0), q_hi = min(kTileQ - 1, yl + R - Y0);
    for (int q = q_lo + half; q <= q_hi; q += split)
      for (int r = r_lo; r <= r_hi; ++r) {
        const int m = q * kTileR + r;
        const int du = X0 + r - xl, dv = Y0 + q - yl;
        const long long dg = pdg[m];
        if (dg == 0) continue;
        const long long num = N * (long long)drow[m] - sa * (long long)psb[m];
        const float fn = ll_to_float(num);
        const float score = fn * fabsf(fn) * pinv[m];  // sign(C) C^2 Df
        if (score < best_f - 1e-5f * fabsf(best_f) - 1e-30f) continue;
        Cand c{num, dg, (dv + R) * ow + (du + R)};
        if (cand_better(c, best)) {
          best = c;
          best_f = fmaxf(best_f, score);
        }
      }
  }
  if (split == 2) {  // partner threads are adjacent lanes
    Cand o;
    o.num = __shfl_xor_sync(0xffffffffu, best.num, 1);
    o.dg = __shfl_xor_sync(0xffffffffu, best.dg, 1);
    o.l = __shfl_xor_sync(0xffffffffu, best.l, 1);
    if (cand_better(o, best)) best = o;
  }
  if (!valid_poi || half) return;
  // slot of this tile among the POI's tiles
  const int tx_first = (xl - R - p.xmin) / kTileR, ty_first = (yl - R - p.ymin) / kTileQ;
  const int slot = ((Y0 - p.ymin) / kTileQ - ty_first) * p.slots_x + ((X0 - p.xmin) / kTileR -
                                                                     tx_first);
  SlotCand* sc = p.slots + (size_t)poi * p.nslots + slot;
  sc->num = best.num;
  sc->dg = best.dg;
  sc->l = best.l;
}

// ------------------------------------------------------------ final reduce
// One warp per POI: exact top four over the POI's slots (each lane keeps a
// sorted top four of its slots, then four warp-wide exact argmax rounds),
// then the re-rank: the winner, and every other of the four whose score is
// within 1e-3 of it, get their sums recomputed from the images on the CUDA
// cores and are compared exactly again.
__device__ __forceinline__ void insert4(Cand t[4], Cand c) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (cand_better(c, t[k])) {
      const Cand x = t[k];
      t[k] = c;
      c = x;
    }
}

__device__ __forceinline__ float cand_score(const Cand& c) {
  const float n = ll_to_float(c.num);
  return n * fabsf(n) / ll_to_float(c.dg);  // sign(C) C^2 Df
}

__global__ void reduce_kernel(const SearchTcParams p) {
  const int lane = threadIdx.x & 31;
  const int64_t poi = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (poi >= p.n_pois) return;
  const int S = p.S, M = p.M, R = p.R, ow = 2 * R + 1;
  const int x0 = M + R + 2 + (int)(poi % p.nx) * p.step;
  const int y0 = M + R + 2 + (int)(poi / p.nx) * p.step;
  const int2 fb = p.fbox[(size_t)(y0 - M - p.ymin) * (p.ntx * 8) + (x0 - M - p.xmin)];
  const longlong2 fs = make_longlong2(fb.x, fb.y);
  const long long N = (long long)S * S;
  const long long Df = N * fs.y - fs.x * fs.x;
  if (Df == 0) {
    if (lane == 0) {
      p.u0[poi] = 0;
      p.v0[poi] = 0;
      p.zncc0[poi] = 0.f;
      p.status[poi] = kZeroVarRef;
    }
    return;
  }
  Cand loc[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) loc[k] = Cand{0, 1, INT_MAX};
  for (int s0 = lane; s0 < p.nslots; s0 += 32) {
    const SlotCand sc = p.slots[(size_t)poi * p.nslots + s0];
    // an unwritten slot (all bits set) or a tile without a candidate
    if (sc.l >= 0 && sc.l < ow * ow) insert4(loc, Cand{sc.num, sc.dg, sc.l});
  }
  Cand top[4];
  int ntop = 0;
  float w0 = 0.f;
  for (int k = 0; k < 4; ++k) {
    if (k == 1) {
      // later rounds only if some remaining candidate scores within 1e-3 of
      // the winner (only those can be reordered by the re-rank)
      const float sc = loc[0].l == INT_MAX ? -3.0e38f : cand_score(loc[0]);
      if (!__any_sync(0xffffffffu, sc >= w0 - 1e-3f * fabsf(w0))) break;
    }
    Cand c = loc[0];
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      Cand d;
      d.num = __shfl_xor_sync(0xffffffffu, c.num, o);
      d.dg = __shfl_xor_sync(0xffffffffu, c.dg, o);
      d.l = __shfl_xor_sync(0xffffffffu, c.l, o);
      if (cand_better(d, c)) c = d;
    }
    if (c.l == INT_MAX) break;
    if (k == 0) w0 = cand_score(c);
    top[ntop++] = c;
    if (loc[0].l == c.l) {  // positions are unique across slots
      loc[0] = loc[1];
      loc[1] = loc[2];
      loc[2] = loc[3];
      loc[3] = Cand{0, 1, INT_MAX};
    }
  }
  Cand best{0, 1, INT_MAX};
  const float w = ntop ? cand_score(top[0]) : 0.f;
  for (int k = 0; k < ntop; ++k) {
    if (k > 0 && cand_score(top[k]) < w - 1e-3f * fabsf(w)) continue;
    const int du = top[k].l % ow - R, dv = top[k].l / ow - R;
    long long sab = 0, sb = 0, sbb = 0;
    for (int ty = 0; ty < S; ++ty) {
      const uint8_t* fr = p.ref + (size_t)(y0 - M + ty) * p.pitch + (x0 - M);
      const uint8_t* gr = p.def + (size_t)(y0 - M + ty + dv) * p.pitch + (x0 - M + du);
      for (int tx = lane; tx < S; tx += 32) {
        const int a = (int)fr[tx] - 128, b = (int)gr[tx] - 128;
        sab += a * b;
        sb += b;
        sbb += b * b;
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      sab += __shfl_xor_sync(0xffffffffu, sab, o);
      sb += __shfl_xor_sync(0xffffffffu, sb, o);
      sbb += __shfl_xor_sync(0xffffffffu, sbb, o);
    }
    const Cand c{N * sab - fs.x * sb, N * sbb - sb * sb, top[k].l};
    if (c.dg != 0 && cand_better(c, best)) best = c;
  }
  if (lane == 0) {
    if (best.l == INT_MAX) {
      p.u0[poi] = -R;
      p.v0[poi] = -R;
      p.zncc0[poi] = 0.f;
      p.status[poi] = kZeroVarDef;
    } else {
      p.u0[poi] = best.l % ow - R;
      p.v0[poi] = best.l / ow - R;
      p.zncc0[poi] = (float)((double)best.num / sqrt((double)Df * (double)best.dg));
      p.status[poi] = kOk;
    }
  }
}

}  // namespace

// Geometry of the tensor-core form for one pair; returns false if the POI
// block of a tile would exceed N = 256.
bool search_tc_geometry(int W, int H, int S, int step, int R, int nx, int ny, SearchTcParams* g) {
  const int M = S / 2, B = M + R + 2;
  g->S = S;
  g->M = M;
  g->R = R;
  g->step = step;
  g->nx = nx;
  g->ny = ny;
  g->twk = (S + 15) / 16 * 16;
  g->ncols_max = (2 * R + kTileR - 1) / step + 1;
  g->nrows_max = (2 * R + kTileQ - 1) / step + 1;
  const int nused = g->ncols_max * g->nrows_max;
  g->npad = (nused + 15) / 16 * 16;
  if (g->npad > 256 || nx == 0 || ny == 0) return false;
  g->rows_per_acc = 1024 / g->twk;
  if (g->rows_per_acc > S) g->rows_per_acc = S;
  const int nacc = (S + g->rows_per_acc - 1) / g->rows_per_acc;
  int cols = 32;
  while (cols < nacc * g->npad) cols *= 2;
  if (cols > 512) return false;
  g->tmem_cols = cols;
  g->xmin = B - M - R;
  g->ymin = B - M - R;
  const int xmax = B + (nx - 1) * step - M + R, ymax = B + (ny - 1) * step - M + R;
  g->ntx = (xmax - g->xmin) / kTileR + 1;
  g->nty = (ymax - g->ymin) / kTileQ + 1;
  // tiles met by one POI window (2R+1 positions) in x and y
  g->slots_x = (2 * R + kTileR - 1) / kTileR + 1;
  g->slots_y = (2 * R + kTileQ - 1) / kTileQ + 1;
  g->nslots = g->slots_x * g->slots_y;
  // phase images cover every A row / column a tile touches and every
  // template row, with room for an 8-column chunk past the last tap
  const int wneed = std::max(W, g->xmin + g->ntx * kTileR + g->twk + 16);
  const int hneed = std::max(H, g->ymin + g->nty * kTileQ + S + 1);
  g->phw = (wneed + 7) / 8 * 8;
  g->phh = hneed;
  return true;
}

size_t search_tc_smem(const SearchTcParams& g) {
  return tile_layout(g.S, g.twk, g.npad).total;
}

size_t search_tc_phase_elems(const SearchTcParams& g) {
  return (size_t)2 * 8 * g.phh * g.phw;
}

size_t search_tc_posbox_elems(const SearchTcParams& g) {
  return (size_t)g.ntx * 8 * (size_t)g.nty * 16;
}

cudaError_t launch_search_tc(const SearchTcParams& p, cudaStream_t st) {
  if (p.n_pois == 0) return cudaSuccess;
  const unsigned wblocks = (unsigned)((p.n_pois + 7) / 8);
  cudaError_t e;
  {
    const int64_t chunks = (int64_t)2 * 8 * p.phh * (p.phw / 8);
    phase_kernel<<<(unsigned)((chunks + 255) / 256), 256, 0, st>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // slots of tiles that meet no position of a POI stay "empty"
  e = cudaMemsetAsync(p.slots, 0xff, sizeof(SlotCand) * (size_t)p.n_pois * p.nslots, st);
  if (e != cudaSuccess) return e;
  {
    const int span = kBoxT + p.S - 1;
    const size_t bsm = (size_t)span * span * 4 + (size_t)span * kBoxT * 8;
    if (bsm > 48 * 1024) {
      e = cudaFuncSetAttribute(boxmap_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)bsm);
      if (e != cudaSuccess) return e;
    }
    dim3 grid((p.ntx * 8 + kBoxT - 1) / kBoxT, (p.nty * 16 + kBoxT - 1) / kBoxT);
    boxmap_kernel<<<grid, 256, bsm, st>>>(p, 1);
    boxmap_kernel<<<grid, 256, bsm, st>>>(p, 0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t smem = search_tc_smem(p);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  e = cudaFuncSetAttribute(tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  tile_kernel<<<(unsigned)(p.ntx * p.nty), kThreads, smem, st>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce_kernel<<<wblocks, 256, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace dic
