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

__device__ __forceinline__ uint16_t to_bf16_bits(int v) {
  // small integers are exact in bf16: take the top half of the float
  return (uint16_t)(__float_as_uint((float)v) >> 16);
}

struct Cand {
  long long num, dg;
  int l;
};

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

// ------------------------------------------------------------ template bank
// bank[(poi*S + ty)*TWK + tx] = f[y0-M+ty][x0-M+tx] - 128 (bf16), 0 for
// tx >= S; sums[poi] = (sum a, sum a^2).  One warp per POI.
__global__ void bank_kernel(const SearchTcParams p) {
  const int lane = threadIdx.x & 31;
  const int64_t poi = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (poi >= p.n_pois) return;
  const int S = p.S, M = p.M, TWK = p.twk;
  const int x0 = M + p.R + 2 + (int)(poi % p.nx) * p.step;
  const int y0 = M + p.R + 2 + (int)(poi / p.nx) * p.step;
  uint16_t* row = p.bank + (size_t)poi * S * TWK;
  long long s = 0, q = 0;
  for (int i = lane; i < S * TWK; i += 32) {
    const int ty = i / TWK, tx = i % TWK;
    int a = 0;
    if (tx < S) {
      a = (int)p.ref[(size_t)(y0 - M + ty) * p.pitch + (x0 - M + tx)] - 128;
      s += a;
      q += a * a;
    }
    row[i] = to_bf16_bits(a);
  }
  for (int o = 16; o; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    q += __shfl_xor_sync(0xffffffffu, q, o);
  }
  if (lane == 0) p.sums[poi] = make_longlong2(s, q);
}

// ------------------------------------------------------------ tile kernel
struct TileLayout {
  int rows;    // image rows of the tile: kTileQ + S - 1
  int cols;    // image columns: kTileR + TWK - 1 (staged bytes)
  int KB;      // 8-tap blocks per template row: TWK / 8
  int sboA;    // bytes per image row in the A buffer: KB * 128
  int stageB;  // bytes per template-row stage: KB * Npad * 16 (8-row groups of KB*128)
  size_t off_bar, off_tmem, off_img, off_box, off_a, off_b, off_d, total;
};

__host__ __device__ inline size_t al(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline TileLayout tile_layout(int S, int TWK, int npad) {
  TileLayout L;
  L.rows = kTileQ + S - 1;
  L.cols = kTileR + TWK - 1;
  L.KB = TWK / 8;
  L.sboA = L.KB * 128;
  L.stageB = L.KB * npad * 16;
  size_t o = 0;
  L.off_bar = o;  o += 8 * (kStages + 1);
  L.off_tmem = o; o += 8;
  o = al(o, 16);  L.off_img = o;  o += (size_t)L.rows * al(L.cols, 4);
  o = al(o, 16);  L.off_box = o;  o += (size_t)kTileQ * kTileR * 8;
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

__global__ void __launch_bounds__(kThreads, 1) tile_kernel(const SearchTcParams p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = p.S, M = p.M, R = p.R, TWK = p.twk, NP = p.npad;
  const TileLayout L = tile_layout(S, TWK, NP);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.off_bar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.off_tmem);
  uint8_t* img = smem + L.off_img;
  int2* box = reinterpret_cast<int2*>(smem + L.off_box);
  unsigned char* abuf = smem + L.off_a;
  unsigned char* bbuf = smem + L.off_b;
  int* dsm = reinterpret_cast<int*>(smem + L.off_d);
  const int imgw = (int)al(L.cols, 4);

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
  // ---- stage the image rectangle (bytes), zero outside the image
  for (int i = tid; i < L.rows * L.cols; i += kThreads) {
    const int r = i / L.cols, c = i % L.cols;
    const int y = Y0 + r, x = X0 + c;
    img[r * imgw + c] = (x >= 0 && x < p.W && y >= 0 && y < p.H)
                            ? p.def[(size_t)y * p.pitch + x] : (uint8_t)128;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // ---- A buffer: eight shifted copies per image row and 8-tap block
  //   abuf[row*sboA + kb*128 + r*16 + e*2] = g[Y0+row][X0 + r + 8kb + e] - 128
  for (int i = tid; i < L.rows * L.KB * 8; i += kThreads) {
    const int row = i / (L.KB * 8), rem = i % (L.KB * 8), kb = rem >> 3, r = rem & 7;
    const uint8_t* src = img + row * imgw + r + 8 * kb;
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e)
      w[e] = (uint32_t)to_bf16_bits((int)src[2 * e] - 128) |
             ((uint32_t)to_bf16_bits((int)src[2 * e + 1] - 128) << 16);
    *reinterpret_cast<uint4*>(abuf + row * L.sboA + kb * 128 + r * 16) =
        make_uint4(w[0], w[1], w[2], w[3]);
  }
  // ---- box sums of b and b^2 for the 128 positions (exact integers)
  if (tid < kTileQ * kTileR) {
    const int q = tid / kTileR, r = tid % kTileR;
    int s = 0, s2 = 0;
    for (int ty = 0; ty < S; ++ty) {
      const uint8_t* src = img + (q + ty) * imgw + r;
      for (int tx = 0; tx < S; ++tx) {
        const int b = (int)src[tx] - 128;
        s += b;
        s2 += b * b;
      }
    }
    box[tid] = make_int2(s, s2);
  }
  // make generic-proxy shared-memory writes visible to the tensor core
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();

  // ---- main loop over template rows
  const int nbr = kr1 - kr0 + 1, nbc = kc1 - kc0 + 1;
  const uint32_t idesc = make_idesc(128, NP);
  const int rows_per_acc = p.rows_per_acc;
  bool ok = true;
  for (int ty = 0; ty < S; ++ty) {
    const int st = ty % kStages;
    unsigned char* bst = bbuf + (size_t)st * L.stageB;
    if (ty >= kStages) {
      // the MMAs of row ty - kStages read this stage: wait for their commit
      const uint32_t par = (uint32_t)(((ty - kStages) / kStages) & 1);
      const int failed = (tid == 0) ? !mbar_wait(smem_u32(&bars[st]), par, 1ll << 26) : 0;
      if (__syncthreads_or(failed)) {
        ok = false;
        break;
      }
    }
    // B stage: POI n of the block (n = i*ncols_max + j) in 8-row groups,
    //   bst[(n/8)*KB*128 + kb*128 + (n%8)*16] = T_n[ty][8kb .. 8kb+7]
    for (int i = tid; i < NP * L.KB; i += kThreads) {
      const int n = i % NP, kb = i / NP;
      const int bi = n / p.ncols_max, bj = n % p.ncols_max;
      const uint32_t dst = smem_u32(bst + (size_t)(n >> 3) * L.KB * 128 + kb * 128 + (n & 7) * 16);
      const bool have = n < p.nrows_max * p.ncols_max && bi < nbr && bj < nbc;
      const int64_t poi = have ? (int64_t)(kr0 + bi) * p.nx + (kc0 + bj) : 0;
      const uint16_t* src = p.bank + ((size_t)poi * S + ty) * TWK + kb * 8;
      const uint32_t bytes = have ? 16u : 0u;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                   "r"(bytes)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int acc = ty / rows_per_acc;
      const uint32_t dcol = tmem + (uint32_t)(acc * NP);
      const uint32_t a_base = smem_u32(abuf) + (uint32_t)(ty * L.sboA);
      const uint32_t b_base = smem_u32(bst);
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
              smem_u32(&bars[st]))
          : "memory");
    }
  }
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
    if (tid == 0) atomicOr(p.err_flag, 2u);
    // give in-flight tensor-core work a bounded chance to finish
    mbar_wait(smem_u32(&bars[kStages]), 0, 1ll << 24);
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

  // ---- per-POI scan of the tile's positions
  const int n = tid;
  if (n >= NP) return;
  const int bi = n / p.ncols_max, bj = n % p.ncols_max;
  if (n >= p.nrows_max * p.ncols_max || bi >= nbr || bj >= nbc) return;
  const int kr = kr0 + bi, kc = kc0 + bj;
  const int64_t poi = (int64_t)kr * p.nx + kc;
  const int xl = B + kc * p.step - M, yl = B + kr * p.step - M;  // POI's subset top-left
  const longlong2 fs = p.sums[poi];
  const long long N = (long long)S * S;
  const int ow = 2 * R + 1;
  Cand best{0, 1, INT_MAX};
  float best_f = -3.0e38f;
  const int* drow = dsm + n * (kTileQ * kTileR + 1);
  for (int m = 0; m < kTileQ * kTileR; ++m) {
    const int q = m >> 3, r = m & 7;
    const int du = X0 + r - xl, dv = Y0 + q - yl;
    if (du < -R || du > R || dv < -R || dv > R) continue;
    const int2 bx = box[m];
    const long long sb = bx.x, sbb = bx.y;
    const long long dg = N * sbb - sb * sb;
    if (dg == 0) continue;
    const long long num = N * (long long)drow[m] - fs.x * sb;
    const float fn = (float)num;
    const float score = fn * fabsf(fn) / (float)dg;  // sign(C) C^2 Df
    if (score < best_f - 1e-5f * fabsf(best_f) - 1e-30f) continue;
    Cand c{num, dg, (dv + R) * ow + (du + R)};
    if (cand_better(c, best)) {
      best = c;
      best_f = fmaxf(best_f, score);
    }
  }
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
// One warp per POI: exact argmax over the POI's slots, then an exact re-rank
// of its four best candidates with sums recomputed from the images.
__global__ void reduce_kernel(const SearchTcParams p) {
  const int lane = threadIdx.x & 31;
  const int64_t poi = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (poi >= p.n_pois) return;
  const int S = p.S, M = p.M, R = p.R, ow = 2 * R + 1;
  const int x0 = M + R + 2 + (int)(poi % p.nx) * p.step;
  const int y0 = M + R + 2 + (int)(poi / p.nx) * p.step;
  const longlong2 fs = p.sums[poi];
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
  // four best slot candidates, kept by every lane (exact comparisons)
  Cand top[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) top[k] = Cand{0, 1, INT_MAX};
  for (int s0 = 0; s0 < p.nslots; s0 += 32) {
    Cand c{0, 1, INT_MAX};
    if (s0 + lane < p.nslots) {
      const SlotCand sc = p.slots[(size_t)poi * p.nslots + s0 + lane];
      // an unwritten slot (all bits set) or a tile without a candidate
      if (sc.l >= 0 && sc.l < ow * ow) c = Cand{sc.num, sc.dg, sc.l};
    }
    for (int src = 0; src < 32; ++src) {
      Cand d;
      d.num = __shfl_sync(0xffffffffu, c.num, src);
      d.dg = __shfl_sync(0xffffffffu, c.dg, src);
      d.l = __shfl_sync(0xffffffffu, c.l, src);
      if (d.l == INT_MAX) continue;
      // insert into top[] (sorted best first)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (cand_better(d, top[k])) {
          Cand t = top[k];
          top[k] = d;
          d = t;
        }
      }
    }
  }
  // exact re-rank: recompute sum a*b for each of the four on the CUDA cores
  Cand best{0, 1, INT_MAX};
  for (int k = 0; k < 4; ++k) {
    if (top[k].l == INT_MAX) continue;
    const int du = top[k].l % ow - R, dv = top[k].l / ow - R;
    long long sab = 0, sb = 0, sbb = 0;
    for (int i = lane; i < S * S; i += 32) {
      const int ty = i / S, tx = i % S;
      const int a = (int)p.ref[(size_t)(y0 - M + ty) * p.pitch + (x0 - M + tx)] - 128;
      const int b = (int)p.def[(size_t)(y0 - M + ty + dv) * p.pitch + (x0 - M + tx + du)] - 128;
      sab += a * b;
      sb += b;
      sbb += b * b;
    }
    for (int o = 16; o; o >>= 1) {
      sab += __shfl_xor_sync(0xffffffffu, sab, o);
      sb += __shfl_xor_sync(0xffffffffu, sb, o);
      sbb += __shfl_xor_sync(0xffffffffu, sbb, o);
    }
    Cand c{N * sab - fs.x * sb, N * sbb - sb * sb, top[k].l};
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
  (void)W;
  (void)H;
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
  return true;
}

size_t search_tc_smem(const SearchTcParams& g) {
  return tile_layout(g.S, g.twk, g.npad).total;
}

cudaError_t launch_search_tc(const SearchTcParams& p, cudaStream_t st) {
  if (p.n_pois == 0) return cudaSuccess;
  const unsigned wblocks = (unsigned)((p.n_pois + 7) / 8);
  bank_kernel<<<wblocks, 256, 0, st>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // slots of tiles that meet no position of a POI stay "empty"
  e = cudaMemsetAsync(p.slots, 0xff, sizeof(SlotCand) * (size_t)p.n_pois * p.nslots, st);
  if (e != cudaSuccess) return e;
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
