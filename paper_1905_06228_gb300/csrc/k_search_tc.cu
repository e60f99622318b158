// k_search_tc.cu -- brute-force ZNCC integer search (Eq. 1, Section 2.1) as
// a BF16 tensor-core contraction (tcgen05, TMEM accumulators, TMA).
//
// Correlation sums as one implicit GEMM across POIs.  Let a "position" be an
// absolute top-left corner (Y, X) of a subset in the deformed image; POI p
// (top-left (yp-M, xp-M)) needs every position with |Y-(yp-M)|, |X-(xp-M)|
// <= R.  For a tile of 128 positions (16 rows x 8 columns, X0 a multiple of
// 8) and the block of POIs whose windows meet the tile:
//
//   D[m][n] = sum_ty sum_tx  G[Y0+q+ty][X0+r+tx] * T_n[ty][tx],   m = 8q + r
//
// Operands are K-major.  A template row is padded to TWK taps (16, 32 or 64).
//  A (M = 128 positions): rows of TWK taps (2*TWK bytes, the swizzle width
//    of its TMA box and descriptor); row (q, r) at image row Y0+q+ty holds
//    g[Y0+q+ty][X0+r ..] - 128, i.e. row Y0+q+ty of the phase image r (the
//    copy of g shifted by r columns).  One 3-D TMA box loads all tile rows
//    once; an 8-row group is one image row, so the step ty -> ty+1 is a
//    descriptor offset of one group.
//  B (N = POI block): rows of 64 taps (128 bytes, 128-byte swizzle), each
//    holding SUB = 64 / TWK consecutive template rows of one POI from the
//    template bank; one 4-D TMA box per operand row j loads the template
//    rows SUB*j .. SUB*j + SUB-1 of the whole block, streamed through a
//    ring of stages.  The four K = 16 MMAs of a stage each take their A
//    descriptor at the image row of their template row; MMAs of template
//    rows at or beyond S are not issued.
//
// The tile kernel is persistent and warp-specialised: one lane streams A
// and B by TMA, one lane issues the MMAs (tcgen05.mma kind::f16, BF16 x BF16
// -> FP32, M=128, K=16 per instruction) into one of two TMEM accumulator
// buffers, and eight epilogue warps score the other buffer, all paired by
// mbarriers.
//
// Exactness: a = f-128 and b = g-128 are integers in [-128, 127], exact in
// BF16; |ab| <= 2^14, so any sum of at most 1024 products is an integer of
// magnitude at most 2^24 and the FP32 accumulation is exact.  Subsets wider
// than 32 use several accumulators (blocks of floor(1024/S) template rows:
// the taps at or beyond S are zero, so a block holds at most 1024 nonzero
// products), added in int32 by the epilogue.  Candidate scores use the exact integers
// num = N Sab - Sa Sb, Dg = N Sbb - Sb^2, with Sa, Saa per POI and Sb, Sbb
// per position (box sums of f and g).
//
// Epilogue: each warp reads one lane quarter of TMEM (32 positions) x 16
// POIs, scores sign(num) num^2 / Dg in FP32 (errors bounded, see
// score_block) and keeps each POI's best two, and the exact sum at the best,
// by warp max reductions; a POI's float winner is its exact tile
// winner when it clears the second by 5e-4, otherwise the warps of the four
// lane quarters compare the near-tied positions exactly from the sums in
// TMEM.  Each (tile, POI) winner goes to a slot; a final kernel reduces a
// POI's slots exactly (lowest linear index on ties), so the integer result
// is bit-identical to the FP32 form and to the oracle.
#include <algorithm>

#include "dic_device.cuh"
#include "dic_internal.cuh"

namespace dic {
namespace {

constexpr int kMaxSlots = 1024;  // tiles met by one POI window (10-bit index)
constexpr int kTileQ = 16;  // position rows per tile
constexpr int kTileR = 8;   // position columns per tile

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// 64-bit shared-memory matrix descriptor, K-major with a row swizzle of
// `rb` bytes (32, 64 or 128: each operand row holds rb bytes of K, 8-row
// groups are 8*rb bytes apart, 16-byte chunks XOR-permuted within a group
// exactly as the TMA's swizzle of the same width writes them).  Steps of K
// inside a row advance the start address; the leading offset is unused.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, int rb) {
  const uint64_t layout = rb == 128 ? 2 : rb == 64 ? 4 : 6;  // SWIZZLE_128B / 64B / 32B
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                               // leading byte offset (unused)
  d |= (uint64_t)(((8 * rb) >> 4) & 0x3FFF) << 32;      // stride byte offset: 8-row group
  d |= (uint64_t)1 << 46;                               // descriptor version for tcgen05
  d |= layout << 61;
  return d;
}

// Instruction descriptor: kind::f16, BF16 A and B, FP32 D, both K-major.
__host__ __device__ __forceinline__ uint32_t make_idesc(int M, int N) {
  return (1u << 4)                     // D format: F32
         | (1u << 7)                   // A format: BF16
         | (1u << 10)                  // B format: BF16
         | ((uint32_t)(N >> 3) << 17)  // N / 8
         | ((uint32_t)(M >> 4) << 24); // M / 16
}

// Wait for the phase of the given parity to complete.  Each try_wait may
// park the thread for up to kSuspendNs (it wakes when the phase completes),
// so waiting threads take no issue slots; after `limit` tries (about
// limit * 10 us) the wait gives up and returns false.
constexpr uint32_t kSuspendNs = 10000;
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit) {
  for (int i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(kSuspendNs)
        : "memory");
    if (done) return true;
  }
  return false;
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

// BF16 bits of (byte - 128), exactly: the float 2^23 + byte minus 2^23 + 128
// (one integer OR and one FP32 add instead of an int-to-float conversion).
__device__ __forceinline__ uint32_t centred_bf16(uint32_t byte) {
  return __float_as_uint(__uint_as_float(0x4B000000u | byte) - 8388736.0f) >> 16;
}

// ------------------------------------------------------------ phase images
// Eight copies of the deformed image shifted by s = 0..7 pixels, as centred
// BF16:  ph[s][y][c] = g[y][c + s] - 128  (0 outside the image),
// so that any run of 8 consecutive pixels starting at column x is one
// aligned 16-byte chunk: copy s = x mod 8 at column x - s.  One thread per
// 8-column chunk (y, c): it reads g[y][c .. c+14] once and writes that
// chunk of all eight copies.
__global__ void phase_kernel(const SearchTcParams p) {
  const int cpr = p.phw / 8;  // chunks per row
  const int chunk = blockIdx.x * blockDim.x + threadIdx.x;
  if (chunk >= p.phh * cpr) return;
  const int y = chunk / cpr;
  const int c = (chunk - y * cpr) * 8;
  const bool yin = y < p.H;
  const uint8_t* row = p.def + (size_t)(yin ? y : 0) * p.pitch;
  uint32_t h[16];
#pragma unroll
  for (int k = 0; k < 15; ++k) {
    const int x = c + k;
    // small integers are exact in BF16; 0 outside the image
    h[k] = (yin && x < p.W) ? centred_bf16(row[x]) : 0u;
  }
  h[15] = 0u;
#pragma unroll
  for (int sft = 0; sft < 8; ++sft) {
    uint16_t* dst = p.gph + ((size_t)sft * p.phh + y) * p.phw + c;
    *reinterpret_cast<uint4*>(dst) =
        make_uint4(h[sft] | (h[sft + 1] << 16), h[sft + 2] | (h[sft + 3] << 16),
                   h[sft + 4] | (h[sft + 5] << 16), h[sft + 6] | (h[sft + 7] << 16));
  }
}

// ------------------------------------------------------------ template bank
// B operand rows of every POI's subset of f, centred BF16: a bank row holds,
// for each POI column kc, 64 taps = SUB template rows of TWK taps,
//   bank[(b*nx + kc)*64 + s*TWK + tx] = f[y(b) + s][xl(kc) + tx] - 128
// (tx < S, else 0), xl(kc) the subsets' left edge.  Two row orders:
//  - by image row (bank_overlap = 1): y(b) = top row of the first POI row +
//    b, so operand row j of POI row kr is bank row kr*step + SUB*j, and the
//    tensor map's POI-row and operand-row strides overlap (step and SUB
//    bank rows); an image row is stored SUB times instead of S/step times;
//  - stacked (bank_overlap = 0): b = kr*sj + j, y(b) = top row of POI row kr
//    + SUB*j, template rows at or beyond S stored as zeros.
// One thread per 16-byte chunk (8 taps, never across two template rows) of
// kBankRows consecutive bank rows, their loads in flight together.
constexpr int kBankRows = 4;

__global__ void bank_kernel(const SearchTcParams p) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.nx * 8) return;
  const int kc = t >> 3, kb = t & 7;
  const int B = p.M + p.R + 2;
  const int s = (8 * kb) / p.twk, tx0 = 8 * kb - s * p.twk;
  const uint8_t* col = p.ref + (B + kc * p.step - p.M);
  uint32_t w[kBankRows][4];
#pragma unroll
  for (int i = 0; i < kBankRows; ++i) {
    const int b = blockIdx.y * kBankRows + i;
    int ytop = B - p.M + b, ty_lim = INT_MAX;  // image row of sub-row 0, template rows left
    if (!p.bank_overlap) {
      const int kr = b / p.sj, j = b - kr * p.sj;
      ytop = B - p.M + kr * p.step + p.sub * j;
      ty_lim = p.S - p.sub * j;
    }
    const int y = ytop + s;
    const bool row_ok = b < p.bank_rows && s < ty_lim && y < p.H;
    const uint8_t* src = col + (size_t)(row_ok ? y : 0) * p.pitch;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      uint32_t h2[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int tx = tx0 + 2 * e + k;
        h2[k] = (row_ok && tx < p.S) ? centred_bf16(src[tx]) : 0u;
      }
      w[i][e] = h2[0] | (h2[1] << 16);
    }
  }
#pragma unroll
  for (int i = 0; i < kBankRows; ++i) {
    const int b = blockIdx.y * kBankRows + i;
    if (b < p.bank_rows)
      *reinterpret_cast<uint4*>(p.bank + ((size_t)b * p.nx + kc) * 64 + 8 * kb) =
          make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
  }
}

// ------------------------------------------------------------ box-sum maps
// map[py*pw + px] = (sum v, sum v^2) over the S x S subset whose top-left is
// the position (ymin+py, xmin+px), v = image - 128 (0 outside the image):
// blockIdx.z = 0 for f (POI sums, fbox), 1 for g (position sums, posbox).
// A CTA covers kBoxX x kBoxY outputs: the centred pixels go to shared
// memory, then separable sums, each thread sliding an S-wide window over
// kBoxSegR consecutive outputs of a row, then kBoxSegC of a column (one add
// and one subtract per output after the first).  All sums are exact
// integers.
constexpr int kBoxX = 64, kBoxY = 32, kBoxSegR = 16, kBoxSegC = 8;

// Row strides in shared memory: pixels padded to an odd number of words and
// row sums to kBoxX + 1 int2, so that lanes walking consecutive rows hit
// distinct banks.
__host__ __device__ inline int boxmap_vstride(int S) { return (kBoxX + S - 1) | 1; }
constexpr int kBoxHs = kBoxX + 1;

__host__ __device__ inline size_t boxmap_smem(int S) {
  return (size_t)(kBoxY + S - 1) * boxmap_vstride(S) * 4 + (size_t)(kBoxY + S - 1) * kBoxHs * 8;
}

__global__ void __launch_bounds__(256) boxmap_kernel(const SearchTcParams p) {
  const int which = blockIdx.z;
  const uint8_t* img = which ? p.def : p.ref;
  int2* out = which ? p.posbox : p.fbox;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int S = p.S, sw = kBoxX + S - 1, sh = kBoxY + S - 1, vs = boxmap_vstride(S);
  int* v = reinterpret_cast<int*>(smem);                    // [sh][vs]
  int2* hs = reinterpret_cast<int2*>(v + (size_t)sh * vs);  // [sh][kBoxHs]
  const int px0 = blockIdx.x * kBoxX, py0 = blockIdx.y * kBoxY;
  const int X0 = p.xmin + px0, Y0 = p.ymin + py0;
  // pixels: warp w takes rows w, w + 8, ...; each lane up to four columns
  // (sw <= kBoxX + 63 for S <= 64), the loads of up to eight rows in flight
  {
    const int lane = threadIdx.x & 31;
#pragma unroll 8
    for (int r = threadIdx.x >> 5; r < sh; r += blockDim.x >> 5) {
      const int y = Y0 + r;
      const bool yin = y >= 0 && y < p.H;
      const uint8_t* row = img + (size_t)(yin ? y : 0) * p.pitch;
      int px[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int c = lane + 32 * k, x = X0 + c;
        px[k] = (c < sw && yin && x >= 0 && x < p.W) ? (int)row[x] - 128 : 0;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (lane + 32 * k < sw) v[r * vs + lane + 32 * k] = px[k];
    }
  }
  __syncthreads();
  // rows: thread t -> row t % sh, segment t / sh
  for (int t = threadIdx.x; t < sh * (kBoxX / kBoxSegR); t += blockDim.x) {
    const int r = t % sh, c0 = (t / sh) * kBoxSegR;
    const int* row = v + (size_t)r * vs + c0;
    int a = 0, b = 0;
#pragma unroll 8
    for (int k = 0; k < S; ++k) {
      const int x = row[k];
      a += x;
      b += x * x;
    }
    int2* o = hs + (size_t)r * kBoxHs + c0;
    o[0] = make_int2(a, b);
#pragma unroll
    for (int j = 1; j < kBoxSegR; ++j) {
      const int xo = row[j - 1], xi = row[j + S - 1];
      a += xi - xo;
      b += xi * xi - xo * xo;
      o[j] = make_int2(a, b);
    }
  }
  __syncthreads();
  // columns: thread t -> column t % kBoxX, segment t / kBoxX
  const int pw = p.ntx * 8, ph = p.nty * 16;
  for (int t = threadIdx.x; t < kBoxX * (kBoxY / kBoxSegC); t += blockDim.x) {
    const int c = t % kBoxX, r0 = (t / kBoxX) * kBoxSegC;
    const int2* col = hs + (size_t)r0 * kBoxHs + c;
    int a = 0, b = 0;
#pragma unroll 8
    for (int k = 0; k < S; ++k) {
      const int2 x = col[(size_t)k * kBoxHs];
      a += x.x;
      b += x.y;
    }
    const int px = px0 + c;
#pragma unroll
    for (int j = 0; j < kBoxSegC; ++j) {
      if (j > 0) {
        const int2 xo = col[(size_t)(j - 1) * kBoxHs], xi = col[(size_t)(j + S - 1) * kBoxHs];
        a += xi.x - xo.x;
        b += xi.y - xo.y;
      }
      const int py = py0 + r0 + j;
      if (px < pw && py < ph) out[(size_t)py * pw + px] = make_int2(a, b);
    }
  }
}

// ------------------------------------------------------------ tile kernel
// A work item is one tile of positions with one chunk of its POI block.  The
// kernel is persistent (one CTA per SM, CTA c takes the items c, c + grid,
// ...) and warp-specialised:
//  - warp 0 (one lane) streams, per item, the A rows into one of p.abufs A
//    buffers and the B stages into a ring of p.stages that runs on across
//    items, with TMA;
//  - warp 1 (one lane) issues the item's MMAs into one of p.accbufs TMEM
//    accumulator buffers and commits them to the item's barriers;
//  - kEpiWarps epilogue warps score a finished buffer while the MMAs of the
//    next item run in the other.
// Barriers: a_full/a_empty per A buffer, b_full/b_empty per stage,
// acc_full/acc_empty per accumulator buffer.  Every wait is bounded: a wait
// that gives up sets the abort word and err_flag, and each role then leaves
// its loop (the epilogue warps decide together, at a barrier).
constexpr int kMaxStages = 16;
constexpr int kEpiWarps = 8;                      // two per TMEM lane quarter
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kThreads = 64 + kEpiThreads;
constexpr int kEpiGroups = kEpiWarps / 4;         // warps per lane quarter
constexpr int kWaitLimit = 1 << 17;  // try_wait calls before giving up (~1.3 s)
// err_flag bits of the tile kernel: 2 | the wait that gave up
constexpr unsigned kGaveUpAEmpty = 1u << 4;    // producer: A buffer free
constexpr unsigned kGaveUpBEmpty = 1u << 5;    // producer: B stage free
constexpr unsigned kGaveUpAccEmpty = 1u << 6;  // MMA: accumulator buffer read
constexpr unsigned kGaveUpAFull = 1u << 7;     // MMA: A rows landed
constexpr unsigned kGaveUpBFull = 1u << 8;     // MMA: B stage landed
constexpr unsigned kGaveUpAccFull = 1u << 9;   // epilogue: accumulator complete
constexpr unsigned kGaveUpDone = 1u << 10;     // MMA: last MMAs complete

constexpr int kRowB = 128;  // bytes of a B operand row (64 taps): its swizzle width
constexpr int kTieRound = 32;  // near ties resolved per round (rare: well under 1 %)
constexpr int kPos = kTileQ * kTileR;  // positions per tile (the MMA's M)

struct TileLayout {
  int rows;    // image rows of the tile: kTileQ + S - 1
  int RB;      // bytes of one A operand row (TWK taps): its swizzle width
  int grp;     // bytes of an 8-row group of A: 8 * RB (one image row)
  int abytes;  // bytes of one A buffer, rounded to 1024
  int stageB;  // bytes per B stage: Npad * kRowB
  size_t off_bar, off_misc, off_pos, off_poi, off_red, off_tie, off_tc, off_a, off_b, total;
};

__host__ __device__ inline size_t al(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Best candidate of one quarter of a tie's positions (exact sums).
struct TieCand {
  long long num, dg;
  int l, pad;
};

__host__ __device__ inline TileLayout tile_layout(int S, int TWK, int npad, int stages,
                                                  int abufs) {
  TileLayout L;
  L.rows = kTileQ + S - 1;
  L.RB = 2 * TWK;
  L.grp = 8 * L.RB;
  L.abytes = (int)al((size_t)L.rows * L.grp, 1024);
  L.stageB = npad * kRowB;
  size_t o = 0;
  L.off_bar = o;  o += 8 * (2 * kMaxStages + 9);
  L.off_misc = o; o += 16;                                   // TMEM base, abort, tie count
  o = al(o, 16);  L.off_pos = o;  o += (size_t)kPos * 16;    // dg, sb, 1/dg
  L.off_poi = o;  o += (size_t)npad * 16;                    // per-POI window and sums
  L.off_red = o;  o += (size_t)4 * npad * 16;                // per-quarter best two + sum
  L.off_tie = o;  o += (size_t)npad * 8;                     // near-tie list
  L.off_tc = o;   o += (size_t)4 * kTieRound * sizeof(TieCand);  // per-quarter tie winners
  o = al(o, 1024);  // swizzle atoms of the operands start on 1024-byte boundaries
  L.off_a = o;    o += (size_t)abufs * L.abytes;
  L.off_b = o;    o += (size_t)stages * L.stageB;
  L.total = o;
  return L;
}

// Per-POI data of a tile's block.  cx, cy: left / top end of the POI's
// window in tile coordinates (a position (q, r) of the tile is in the window
// iff 0 <= r - cx <= 2R and 0 <= q - cy <= 2R); kNoPoi for a padding column
// or a POI without reference variance.
struct PoiInfo {
  int cx, cy;
  float saf;  // Sa as float (exact: |Sa| < 2^24)
  int sa;
};
constexpr int kNoPoi = -(1 << 20);

// Order-preserving map of a float onto int (larger float -> larger int).
__device__ __forceinline__ int f2key(float s) {
  const int i = __float_as_int(s);
  return i ^ ((i >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float key2f(int k) {
  return __int_as_float(k ^ ((k >> 31) & 0x7fffffff));
}

// Best-two merge of (largest, second largest) key pairs.
__device__ __forceinline__ void merge2(int& mx, int& sc, int omx, int osc) {
  sc = max(max(sc, osc), min(mx, omx));
  mx = max(mx, omx);
}

// Sums of the accumulator for lane quarter `quarter`, columns c .. c+15 of
// every accumulator of a buffer (one accumulator: the exact FP32 sums as
// bits; several: their int32 total).
template <bool kWide>
__device__ __forceinline__ void load_sums(uint32_t tmem, int nacc, int np, int quarter, int c,
                                          uint32_t (&val)[16]) {
#pragma unroll
  for (int k = 0; k < 16; ++k) val[k] = 0;
  for (int a = 0; a < nacc; ++a) {
    uint32_t v[16];
    const uint32_t addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(a * np + c);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k)
      val[k] = kWide ? (uint32_t)((int)val[k] + __float2int_rn(__uint_as_float(v[k]))) : v[k];
  }
}

// Columns c .. c+15 of lane quarter `quarter` of a one-accumulator buffer:
// the load only (tcgen05.wait::ld makes them valid).
__device__ __forceinline__ void tmem_ld16(uint32_t tmem, int quarter, int c,
                                          uint32_t (&v)[16]) {
  const uint32_t addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(addr));
}

// Scores of one (quarter, 16-column) block of an accumulator buffer and
// their per-POI best two over the quarter's 32 positions, with the sum at
// the best.
//
// Position m = 32*quarter + lane (row q = m/8, column r = m%8 of the tile)
// holds the sums of POIs c0..c0+15.  The score sign(num) num^2 / Dg orders a
// POI's candidates like its ZNCC.  Without wide sums (one accumulator,
// |Sab| < 2^24 exact in FP32) num is formed in FP32 from exact operands:
// Sa*Sb as an exact two-float product, N*Sab - hi in one FMA, then - lo;
// its error is at most 2^-23 |num| + 2^-14.  With wide sums num is exact in
// 64-bit integers and only the final conversion rounds.  Either way a
// score's relative error, including the position index packed into the
// low 7 bits of its key, stays below 1.5e-4 for num != 0, and |score| <
// 4e-9 when num = 0; the winner test relies on this.
template <bool kWide>
__device__ __forceinline__ void score_block(const SearchTcParams& p, const uint32_t (&val)[16],
                                            int quarter, int lane, int c0, int rr, int q,
                                            float sbf, int sb, float pinv_m, const PoiInfo* poi,
                                            int4* red) {
  const int NP = p.npad, R2 = 2 * p.R, m = quarter * 32 + lane;
  const long long N = (long long)p.S * p.S;
  const float Nf = (float)N;
  int key[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const PoiInfo pi = poi[c0 + k];
    const bool in = (unsigned)(rr - pi.cx) <= (unsigned)R2 && (unsigned)(q - pi.cy) <= (unsigned)R2;
    float nf;
    if (kWide) {
      nf = ll_to_float(N * (long long)(int)val[k] - (long long)pi.sa * sb);
    } else {
      const float hi = pi.saf * sbf;
      const float lo = fmaf(pi.saf, sbf, -hi);
      nf = fmaf(Nf, __uint_as_float(val[k]), -hi) - lo;
    }
    const float s = nf * fabsf(nf) * pinv_m;
    key[k] = in ? ((f2key(s) & ~127) | m) : INT_MIN;
  }
  // per POI, the best and second-best keys over the warp's 32 positions by
  // warp max reductions (a valid key is unique: its low 7 bits hold the
  // position); the lane holding the best stores the POI's entry with the
  // sum at the best, lane 0 stores it where the POI has no candidate here
  int4* out = red + quarter * NP + c0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int mx = __reduce_max_sync(0xffffffffu, key[k]);
    const int sc = __reduce_max_sync(0xffffffffu, key[k] == mx ? INT_MIN : key[k]);
    if (mx != INT_MIN ? (mx & 31) == lane : lane == 0)
      out[k] = make_int4(mx, sc, (int)val[k], 0);
  }
}

// POI n of a tile's block (row-major over ncols_max x nrows_max): operand
// row n of B.
__device__ __forceinline__ void block_poi(const SearchTcParams& p, int n, int& bi, int& bj) {
  bi = n / p.ncols_max;
  bj = n % p.ncols_max;
}

// Tile origin (absolute positions; X0 a multiple of 8) and POI block of a
// work item; false if the item meets no POI (a chunk past the block's last
// row, or a tile in a gap between windows when the grid step exceeds
// 2R + 8): every role skips such items alike.
struct TileItem {
  int X0, Y0, kc0, kr0, nbr, nbc;
};

__device__ __forceinline__ bool tile_item(const SearchTcParams& p, int item, TileItem& t) {
  const int tile = item / p.nchunk, chunk = item - tile * p.nchunk;
  const int M = p.M, R = p.R, B = M + R + 2;
  t.X0 = p.xmin + (tile % p.ntx) * kTileR;
  t.Y0 = p.ymin + (tile / p.ntx) * kTileQ;
  // POI column k is met iff x_k - M - R <= X0 + 7 and x_k - M + R >= X0
  auto ceil_div = [](int a, int b) { return a >= 0 ? (a + b - 1) / b : -((-a) / b); };
  auto floor_div = [](int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
  t.kc0 = max(0, ceil_div(t.X0 + M - R - B, p.step));
  t.kr0 = max(0, ceil_div(t.Y0 + M - R - B, p.step)) + chunk * p.nrows_max;
  const int kc1 = min(p.nx - 1, floor_div(t.X0 + kTileR - 1 + M + R - B, p.step));
  const int kr1 = min(p.ny - 1, floor_div(t.Y0 + kTileQ - 1 + M + R - B, p.step));
  t.nbr = min(kr1 - t.kr0 + 1, p.nrows_max);
  t.nbc = kc1 - t.kc0 + 1;
  return t.nbr > 0 && t.nbc > 0;
}

__device__ __forceinline__ void epi_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory");
}
// true on every epilogue thread if v is true on any
__device__ __forceinline__ bool epi_any(bool v) {
  uint32_t r;
  asm volatile(
      "{ .reg .pred p, q; setp.ne.u32 p, %1, 0; bar.red.or.pred q, 1, %2, p; "
      "selp.u32 %0, 1, 0, q; }"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kEpiThreads)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Issue helpers for a converged warp: elect.sync picks one lane (the same
// lowest active lane every time), which issues the operation.
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "{ .reg .b32 r; .reg .pred e; elect.sync r|e, 0xffffffff; "
      "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0]; }" ::"r"(
          bar)
      : "memory");
}
__device__ __forceinline__ void umma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{ .reg .b32 r; .reg .pred e, p; elect.sync r|e, 0xffffffff; setp.ne.b32 p, %4, 0; "
      "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void tma_expect(uint32_t bar, uint32_t bytes) {
  asm volatile(
      "{ .reg .b32 r; .reg .pred e; elect.sync r|e, 0xffffffff; "
      "@e mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1; }" ::"r"(bar),
      "r"(bytes)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, int c0, int c1,
                                            int c2, uint32_t bar) {
  asm volatile(
      "{ .reg .b32 r; .reg .pred e; elect.sync r|e, 0xffffffff; "
      "@e cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5]; }" ::"r"(dst),
      "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* tm, int c0, int c1,
                                            int c2, int c3, uint32_t bar) {
  asm volatile(
      "{ .reg .b32 r; .reg .pred e; elect.sync r|e, 0xffffffff; "
      "@e cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5}], [%6]; }" ::"r"(dst),
      "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}
// The MMAs of one B stage: SUB template rows of 64 / SUB taps, KPR = 4 / SUB
// MMAs of 16 taps each, straight-line with constant descriptor offsets.
// (ty, rin, dcol, ad_row): the next template row, its row within the
// current accumulator, that accumulator's TMEM column, its A descriptor.
template <int SUB>
__device__ __forceinline__ void issue_stage(uint32_t& dcol, uint64_t& ad_row, uint64_t bd, int& ty,
                                            int& rin, int S, int rows_per_acc, uint32_t a_step,
                                            uint32_t np, uint32_t idesc) {
  constexpr int KPR = 4 / SUB;
#pragma unroll
  for (int sr = 0; sr < SUB; ++sr) {
    if (ty < S) {
#pragma unroll
      for (int kk = 0; kk < KPR; ++kk)
        umma_f16(dcol, ad_row + (uint64_t)(2 * kk), bd + (uint64_t)(2 * (sr * KPR + kk)), idesc,
                 (rin == 0 && kk == 0) ? 0u : 1u);
      ++ty;
      ad_row += a_step;
      if (++rin == rows_per_acc) {
        rin = 0;
        dcol += np;
      }
    }
  }
}

// A wait of the whole warp, decided by lane 0's observation (uniform).
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity, int limit) {
  const int ok = mbar_wait(bar, parity, limit) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__global__ void __launch_bounds__(kThreads, 1)
    tile_kernel(const SearchTcParams p, const __grid_constant__ CUtensorMap tmA,
                const __grid_constant__ CUtensorMap tmB) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = p.S, R = p.R, TWK = p.twk, NP = p.npad, NST = p.stages;
  const int NAB = p.abufs, NACB = p.accbufs;
  const TileLayout L = tile_layout(S, TWK, NP, NST, NAB);
  uint64_t* b_full = reinterpret_cast<uint64_t*>(smem + L.off_bar);
  uint64_t* b_empty = b_full + kMaxStages;
  uint64_t* a_full = b_empty + kMaxStages;  // [2]
  uint64_t* a_empty = a_full + 2;           // [2]
  uint64_t* acc_full = a_empty + 2;         // [2]
  uint64_t* acc_empty = acc_full + 2;       // [2]
  uint64_t* done = acc_empty + 2;           // every MMA of the CTA completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.off_misc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* nties = reinterpret_cast<int*>(tmem_slot + 2);
  long long* pdg = reinterpret_cast<long long*>(smem + L.off_pos);  // Dg per position
  int* psb = reinterpret_cast<int*>(pdg + kPos);                     // Sb per position
  float* pinv = reinterpret_cast<float*>(psb + kPos);                // 1 / Dg
  PoiInfo* poi = reinterpret_cast<PoiInfo*>(smem + L.off_poi);
  int4* red = reinterpret_cast<int4*>(smem + L.off_red);
  int2* ties = reinterpret_cast<int2*>(smem + L.off_tie);  // (POI n, threshold bits)
  TieCand* tcand = reinterpret_cast<TieCand*>(smem + L.off_tc);
  unsigned char* abuf = smem + L.off_a;
  unsigned char* bbuf = smem + L.off_b;

  const int nitems = p.ntx * p.nty * p.nchunk;
  const long long N = (long long)S * S;
  const int nblock = p.ncols_max * p.nrows_max;  // POIs (operand rows) loaded per stage
  const int rows_per_acc = p.rows_per_acc;
  const int nacc = (S + rows_per_acc - 1) / rows_per_acc;
  const uint32_t bufcols = (uint32_t)(nacc * NP);  // TMEM columns of one accumulator buffer

  if (tid == 0) {
    *abort_flag = 0;
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
    for (int i = 0; i < NST; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&b_full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&b_empty[i])));
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&a_full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&a_empty[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&acc_full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&acc_empty[i])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(done)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"((uint32_t)p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  auto give_up = [&](unsigned site) {
    *abort_flag = 1;
    atomicOr(p.err_flag, 2u | site);
  };

  if (warp == 0) {
    // ---- producer: the whole warp runs the loop (uniform control flow and
    // operands), one elected lane issues each copy
    int i = 0, gs = 0;  // items and B stages issued
    int st = 0;
    uint32_t ephase = 0;  // parity of the b_empty phase awaited on this lap of the ring
    unsigned failed = 0;
    for (int item = blockIdx.x; item < nitems && !failed; item += gridDim.x) {
      TileItem t;
      if (!tile_item(p, item, t)) continue;
      if (*abort_flag) break;
      // A buffer ab is free once the MMAs of its previous item completed
      const int ab = NAB == 2 ? (i & 1) : 0, ua = NAB == 2 ? (i >> 1) : i;
      if (ua > 0 && !mbar_wait_warp(smem_u32(&a_empty[ab]), (uint32_t)((ua - 1) & 1), kWaitLimit)) {
        failed = kGaveUpAEmpty;
        break;
      }
      // A rows Y0 .. Y0+rows-1, positions r = 0..7 of the tile's row: the
      // TWK taps from column X0 + r, i.e. row r of phase image r (an 8-row
      // group is one image row)
      tma_expect(smem_u32(&a_full[ab]), (uint32_t)(L.rows * L.grp));
      tma_load_3d(smem_u32(abuf + (size_t)ab * L.abytes), &tmA, t.X0, 0, t.Y0,
                  smem_u32(&a_full[ab]));
      ++i;
      // B stages: operand row j (template rows SUB*j ..) of every POI of
      // the block, the ncols_max x nrows_max patch of the bank landing as
      // operand rows n = bi * ncols_max + bj of 64 taps
      for (int j = 0; j < p.sj; ++j) {
        if (gs >= NST && !mbar_wait_warp(smem_u32(&b_empty[st]), ephase, kWaitLimit)) {
          failed = kGaveUpBEmpty;
          break;
        }
        const uint32_t fb = smem_u32(&b_full[st]);
        tma_expect(fb, (uint32_t)(nblock * kRowB));
        tma_load_4d(smem_u32(bbuf + (size_t)st * L.stageB), &tmB, 0, t.kc0, t.kr0, j, fb);
        ++gs;
        if (++st == NST) {
          st = 0;
          if (gs > NST) ephase ^= 1u;  // the first lap waits on nothing
        }
      }
    }
    if (failed && lane == 0) give_up(failed);
    __syncwarp();
    if (*abort_flag) {
      // let the copies still in flight land (bounded) before the CTA leaves
      for (int g = max(0, gs - NST); g < gs; ++g)
        mbar_wait_warp(smem_u32(&b_full[g % NST]), (uint32_t)((g / NST) & 1), kWaitLimit / 16);
      for (int k = max(0, i - NAB); k < i; ++k) {
        const int ab = NAB == 2 ? (k & 1) : 0, ua = NAB == 2 ? (k >> 1) : k;
        mbar_wait_warp(smem_u32(&a_full[ab]), (uint32_t)(ua & 1), kWaitLimit / 16);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer: the whole warp runs the loop, one elected lane issues
    // each MMA and commit.  Descriptors are advanced by adding (byte offset
    // >> 4) to their start-address field.  MMA k of a stage covers taps
    // 16k .. 16k+15 of the B row: template row ty = SUB*j + k / KPR, taps
    // 16 (k % KPR) .. of A's image row Y0 + q + ty; the MMAs of template rows
    // at or beyond S are not issued.
    const uint32_t idesc = make_idesc(128, NP);
    const uint64_t bd0 = make_desc(smem_u32(bbuf), kRowB);
    const uint32_t a_step = (uint32_t)L.grp >> 4, b_step = (uint32_t)L.stageB >> 4;
    const int SUB = p.sub;
    int i = 0, st = 0;
    uint32_t fphase = 0;
    uint64_t bd_st = bd0;
    unsigned failed = 0;
    for (int item = blockIdx.x; item < nitems && !failed; item += gridDim.x) {
      TileItem t;
      if (!tile_item(p, item, t)) continue;
      if (*abort_flag) break;
      const int b = NACB == 2 ? (i & 1) : 0, ub = NACB == 2 ? (i >> 1) : i;
      const int ab = NAB == 2 ? (i & 1) : 0, ua = NAB == 2 ? (i >> 1) : i;
      // the epilogue has read this accumulator buffer's previous item
      if (ub > 0 &&
          !mbar_wait_warp(smem_u32(&acc_empty[b]), (uint32_t)((ub - 1) & 1), kWaitLimit)) {
        failed = kGaveUpAccEmpty;
        break;
      }
      if (!mbar_wait_warp(smem_u32(&a_full[ab]), (uint32_t)(ua & 1), kWaitLimit)) {
        failed = kGaveUpAFull;
        break;
      }
      const uint64_t ad0 = make_desc(smem_u32(abuf + (size_t)ab * L.abytes), L.RB);
      const uint32_t dbase = tmem + (uint32_t)b * bufcols;
      // template row ty, its accumulator (dcol) and row within it (rin),
      // advanced by counters (no divisions on the issue path)
      int ty = 0, rin = 0;
      uint32_t dcol = dbase;
      uint64_t ad_row = ad0;
      for (int j = 0; j < p.sj; ++j) {
        if (!mbar_wait_warp(smem_u32(&b_full[st]), fphase, kWaitLimit)) {
          failed = kGaveUpBFull;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (SUB == 4)
          issue_stage<4>(dcol, ad_row, bd_st, ty, rin, S, rows_per_acc, a_step, (uint32_t)NP, idesc);
        else if (SUB == 2)
          issue_stage<2>(dcol, ad_row, bd_st, ty, rin, S, rows_per_acc, a_step, (uint32_t)NP, idesc);
        else
          issue_stage<1>(dcol, ad_row, bd_st, ty, rin, S, rows_per_acc, a_step, (uint32_t)NP, idesc);
        umma_commit(smem_u32(&b_empty[st]));  // the stage is free once these complete
        if (++st == NST) {
          st = 0;
          fphase ^= 1u;
          bd_st = bd0;
        } else {
          bd_st += b_step;
        }
      }
      if (failed) break;
      umma_commit(smem_u32(&a_empty[ab]));
      umma_commit(smem_u32(&acc_full[b]));
      ++i;
    }
    if (failed && lane == 0) give_up(failed);
    // every MMA issued so far has completed before the CTA leaves
    umma_commit(smem_u32(done));
    if (!mbar_wait_warp(smem_u32(done), 0, kWaitLimit) && lane == 0) give_up(kGaveUpDone);
  } else {
    // ---- epilogue warps
    const int et = tid - 64;                       // 0 .. kEpiThreads-1
    const int quarter = warp & 3;                  // TMEM lane quarter of this warp
    const int grp = (warp - 2) >> 2;               // 0 .. kEpiGroups-1
    const int wide = nacc > 1;
    const int ow = 2 * R + 1;
    const float Nf = (float)N;
    const int B = p.M + R + 2;
    // box sums of an item's positions (thread et < kPos) and of its POI et
    // (et < NP; kEpiThreads >= 256 >= NP), loaded one item ahead
    static_assert(kEpiThreads >= 256, "one POI of a block per epilogue thread");
    auto next_item = [&](int item, TileItem& t) {
      while (item < nitems && !tile_item(p, item, t)) item += gridDim.x;
      return item;
    };
    auto load_sums_of = [&](const TileItem& t, int2& pb, int2& fb) {
      pb = make_int2(0, 0);
      fb = make_int2(0, 0);
      if (et < kPos)
        pb = p.posbox[(size_t)(t.Y0 - p.ymin + et / kTileR) * (p.ntx * 8) +
                      (t.X0 - p.xmin + et % kTileR)];
      int bi, bj;
      block_poi(p, et, bi, bj);
      if (et < nblock && bi < t.nbr && bj < t.nbc) {
        const int xl = B + (t.kc0 + bj) * p.step - p.M, yl = B + (t.kr0 + bi) * p.step - p.M;
        fb = p.fbox[(size_t)(yl - p.ymin) * (p.ntx * 8) + (xl - p.xmin)];
      }
    };
    int i = 0;
    TileItem t;
    int item = next_item(blockIdx.x, t);
    int2 pb_next, fb_next;
    if (item < nitems) load_sums_of(t, pb_next, fb_next);
    while (item < nitems) {
      const int X0 = t.X0, Y0 = t.Y0, kc0 = t.kc0, kr0 = t.kr0;
      const int b = NACB == 2 ? (i & 1) : 0, ub = NACB == 2 ? (i >> 1) : i;
      // ---- per-position box statistics and per-POI window / sums
      if (et < kPos) {
        const int2 bx = pb_next;
        const long long dg = N * (long long)bx.y - (long long)bx.x * bx.x;
        pdg[et] = dg;
        psb[et] = bx.x;
        pinv[et] = dg ? 1.0f / ll_to_float(dg) : 0.f;
      }
      if (et < NP) {
        int bi, bj;
        block_poi(p, et, bi, bj);
        PoiInfo pi{kNoPoi, kNoPoi, 0.f, 0};
        const int2 fb = fb_next;
        // a POI without reference variance is decided by the reduce kernel
        if (et < nblock && bi < t.nbr && bj < t.nbc &&
            N * (long long)fb.y - (long long)fb.x * fb.x != 0) {
          const int xl = B + (kc0 + bj) * p.step - p.M, yl = B + (kr0 + bi) * p.step - p.M;
          pi = PoiInfo{xl - X0 - R, yl - Y0 - R, (float)fb.x, fb.x};
        }
        poi[et] = pi;
      }
      const int item_next = next_item(item + gridDim.x, t);
      if (item_next < nitems) load_sums_of(t, pb_next, fb_next);
      if (et == 0) *nties = 0;
      // ---- the accumulator of this item
      const bool got = mbar_wait(smem_u32(&acc_full[b]), (uint32_t)(ub & 1), kWaitLimit);
      if (epi_any(!got || *abort_flag)) {  // also the barrier before the scores
        if (!got) give_up(kGaveUpAccFull);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t tbuf = tmem + (uint32_t)b * bufcols;
      // ---- scores: each warp takes its lane quarter (32 positions) and
      // every kEpiGroups-th 16-column block of POIs
      __syncwarp();
      {
        const int m = quarter * 32 + lane, q = m / kTileR, r = m % kTileR;
        const int rr = pdg[m] != 0 ? r : r + (1 << 21);  // Dg = 0: in no window
        const float pinv_m = pinv[m];
        const int sb = psb[m];
        const float sbf = (float)sb;
        constexpr int kStep = kEpiGroups * 16;
        if (wide) {
          for (int c0 = grp * 16; c0 < NP; c0 += kStep) {
            uint32_t val[16];
            load_sums<true>(tbuf, nacc, NP, quarter, c0, val);
            score_block<true>(p, val, quarter, lane, c0, rr, q, sbf, sb, pinv_m, poi, red);
          }
        } else {
          // two blocks' sums loaded under one wait
          for (int c0 = grp * 16; c0 < NP; c0 += 2 * kStep) {
            const bool two = c0 + kStep < NP;
            uint32_t va[16], vb[16];
            tmem_ld16(tbuf, quarter, c0, va);
            if (two) tmem_ld16(tbuf, quarter, c0 + kStep, vb);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            score_block<false>(p, va, quarter, lane, c0, rr, q, sbf, sb, pinv_m, poi, red);
            if (two)
              score_block<false>(p, vb, quarter, lane, c0 + kStep, rr, q, sbf, sb, pinv_m, poi,
                                 red);
          }
        }
      }
      epi_sync();
      // ---- per-POI winner of the tile: merge the four quarters' best two.
      // The float winner is the exact winner if its magnitude exceeds 1e-8
      // and it clears the second by 5e-4 of that magnitude: float scores err
      // by less than 1.5e-4 (relative) where num != 0, and by less than 4e-9
      // where num = 0, so the exact order of the two cannot differ.
      // Otherwise (a near tie) the POI's positions whose float score is
      // within 5e-4 (+1e-8) of the best are compared exactly, lowest linear
      // index on ties; no position outside that band can be the tile's
      // maximum.
      auto cand_at = [&](const PoiInfo& pi, int raw, int m) {
        const int sab = wide ? raw : __float2int_rn(__int_as_float(raw));
        return Cand{N * (long long)sab - (long long)pi.sa * psb[m], pdg[m],
                    (m / kTileR - pi.cy) * ow + (m % kTileR - pi.cx)};
      };
      auto write_slot = [&](const PoiInfo& pi, int n, const Cand& best) {
        int bi, bj;
        block_poi(p, n, bi, bj);
        const int64_t poi_k = (int64_t)(kr0 + bi) * p.nx + (kc0 + bj);
        const int xl = pi.cx + X0 + R, yl = pi.cy + Y0 + R;
        // slot of this tile among the POI's tiles
        const int tx_first = (xl - R - p.xmin) / kTileR, ty_first = (yl - R - p.ymin) / kTileQ;
        const int slot = ((Y0 - p.ymin) / kTileQ - ty_first) * p.slots_x +
                         ((X0 - p.xmin) / kTileR - tx_first);
        SlotCand* s = p.slots + (size_t)poi_k * p.nslots + slot;
        s->num = best.num;
        s->dg = best.dg;
        s->l = best.l;
      };
      for (int n = et; n < NP; n += kEpiThreads) {
        const PoiInfo pi = poi[n];
        if (pi.cx == kNoPoi) continue;
        int4 r0 = red[n];
        int mx = r0.x, sc = r0.y, v = r0.z;
#pragma unroll
        for (int qq = 1; qq < 4; ++qq) {
          const int4 rq = red[qq * NP + n];
          sc = max(max(sc, rq.y), min(mx, rq.x));
          if (rq.x > mx) {
            mx = rq.x;
            v = rq.z;
          }
        }
        if (mx == INT_MIN) {
          write_slot(pi, n, Cand{0, 1, INT_MAX});
          continue;
        }
        const float fm = key2f(mx);
        if (fabsf(fm) > 1e-8f && (sc == INT_MIN || key2f(sc) < fm - 5e-4f * fabsf(fm))) {
          write_slot(pi, n, cand_at(pi, v, mx & 127));
        } else {
          const int k = atomicAdd(nties, 1);
          ties[k] = make_int2(n, __float_as_int(fm - 5e-4f * fabsf(fm) - 1e-8f));
        }
      }
      epi_sync();
      // ---- near ties, kTieRound at a time: the warps of lane group grp
      // take every kEpiGroups-th tie, each warp its quarter's positions,
      // reading the sums of the tie's column back from TMEM; then one
      // thread per tie merges the four quarters' candidates
      const int ntie = *nties;
      for (int base = 0; base < ntie; base += kTieRound) {
        const int nround = min(kTieRound, ntie - base);
        __syncwarp();
        for (int k = grp; k < nround; k += kEpiGroups) {
          const int n = ties[base + k].x;
          const float thr = __int_as_float(ties[base + k].y);
          const PoiInfo pi = poi[n];
          int raw = 0;
          for (int a = 0; a < nacc; ++a) {
            uint32_t v;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
                         : "=r"(v)
                         : "r"(tbuf + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(a * NP + n)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            raw = wide ? raw + __float2int_rn(__uint_as_float(v)) : (int)v;
          }
          const int m = quarter * 32 + lane, q = m / kTileR, r = m % kTileR;
          Cand best{0, 1, INT_MAX};
          if ((unsigned)(r - pi.cx) <= (unsigned)(2 * R) &&
              (unsigned)(q - pi.cy) <= (unsigned)(2 * R) && pdg[m] != 0) {
            float nf;
            if (wide) {
              nf = ll_to_float(N * (long long)raw - (long long)pi.sa * psb[m]);
            } else {
              const float sbf = (float)psb[m], hi = pi.saf * sbf, lo = fmaf(pi.saf, sbf, -hi);
              nf = fmaf(Nf, __int_as_float(raw), -hi) - lo;
            }
            if (nf * fabsf(nf) * pinv[m] >= thr) best = cand_at(pi, raw, m);
          }
#pragma unroll
          for (int o = 16; o; o >>= 1) {
            Cand d;
            d.num = __shfl_xor_sync(0xffffffffu, best.num, o);
            d.dg = __shfl_xor_sync(0xffffffffu, best.dg, o);
            d.l = __shfl_xor_sync(0xffffffffu, best.l, o);
            if (cand_better(d, best)) best = d;
          }
          if (lane == 0) tcand[k * 4 + quarter] = TieCand{best.num, best.dg, best.l, 0};
        }
        epi_sync();
        for (int k = et; k < nround; k += kEpiThreads) {
          const int n = ties[base + k].x;
          Cand best{0, 1, INT_MAX};
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const TieCand c = tcand[k * 4 + qq];
            const Cand d{c.num, c.dg, c.l};
            if (cand_better(d, best)) best = d;
          }
          write_slot(poi[n], n, best);
        }
        epi_sync();  // tcand is free for the next round
      }
      // the buffer's last TMEM read is done: release it to the MMA issuer
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      epi_sync();
      if (et == 0) mbar_arrive(smem_u32(&acc_empty[b]));
      epi_sync();  // smem of this item is free for the next
      ++i;
      item = item_next;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)p.tmem_cols)
                 : "memory");
  }
}

// ------------------------------------------------------------ final reduce
// kRedLanes lanes per POI.  Each slot holds the exact winner of one tile (or no
// candidate).  Lanes score their slots in float from the exact sums (error
// below 1e-6 plus 2^-13 from the slot index packed into the key, relative;
// exactly 0 where num = 0) and the warp keeps the best two; if the best's
// magnitude exceeds 1e-8 and it clears the second by 1e-3 of that magnitude
// it is the POI's winner, otherwise the slots within 2e-3 (+1e-8) of the
// best are compared exactly, lowest linear index on ties.
__device__ __forceinline__ float cand_score(long long num, long long dg) {
  const float n = ll_to_float(num);
  return n * fabsf(n) * __frcp_rn(ll_to_float(dg));  // sign(C) C^2 Df
}

constexpr int kRedLanes = 8;  // lanes per POI of the reduce kernel (4 POIs per warp)

__global__ void reduce_kernel(const SearchTcParams p) {
  const int lane = threadIdx.x & 31, sub = lane & (kRedLanes - 1);
  const int64_t poi =
      ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (32 / kRedLanes) +
      lane / kRedLanes;
  // no early exit: every lane takes part in the warp's shuffles
  const bool live = poi < p.n_pois;
  const int64_t pq = live ? poi : 0;
  const int S = p.S, M = p.M, R = p.R, ow = 2 * R + 1;
  const int x0 = M + R + 2 + (int)(pq % p.nx) * p.step;
  const int y0 = M + R + 2 + (int)(pq / p.nx) * p.step;
  const SlotCand* sl = p.slots + (size_t)pq * p.nslots;
  // The slots of the tiles that meet the POI's window, (tx, ty) from
  // (xl - R, yl - R) to (xl + R, yl + R) in tile units: the tile kernel has
  // written each of them (a winner, or no candidate); the other slots of
  // the POI's slots_x x slots_y block are never written and never read.
  const int xl = x0 - M, yl = y0 - M;
  const int nsx = (xl + R - p.xmin) / kTileR - (xl - R - p.xmin) / kTileR + 1;
  const int nsy = (yl + R - p.ymin) / kTileQ - (yl - R - p.ymin) / kTileQ + 1;
  auto used = [&](int s) { return s % p.slots_x < nsx && s / p.slots_x < nsy; };
  auto valid = [&](int l) { return l >= 0 && l < ow * ow; };  // not "no candidate"
  // the first slot of each lane is loaded together with the POI's own sums
  SlotCand c0{0, 1, -1, 0};
  if (live && sub < p.nslots && used(sub)) c0 = sl[sub];
  const int2 fb = p.fbox[(size_t)(y0 - M - p.ymin) * (p.ntx * 8) + (x0 - M - p.xmin)];
  const long long N = (long long)S * S;
  const long long Df = N * (long long)fb.y - (long long)fb.x * fb.x;
  const bool act = live && Df != 0;
  int mx = INT_MIN, sc = INT_MIN;
  if (act) {
    if (valid(c0.l))
      merge2(mx, sc, (f2key(cand_score(c0.num, c0.dg)) & ~(kMaxSlots - 1)) | sub, INT_MIN);
    for (int s = sub + kRedLanes; s < p.nslots; s += kRedLanes) {
      if (!used(s)) continue;
      const SlotCand c = sl[s];
      if (valid(c.l))
        merge2(mx, sc, (f2key(cand_score(c.num, c.dg)) & ~(kMaxSlots - 1)) | s, INT_MIN);
    }
  }
#pragma unroll
  for (int o = kRedLanes / 2; o; o >>= 1) {  // within the POI's lanes
    const int omx = __shfl_xor_sync(0xffffffffu, mx, o);
    const int osc = __shfl_xor_sync(0xffffffffu, sc, o);
    merge2(mx, sc, omx, osc);
  }
  Cand best{0, 1, INT_MAX};
  bool tie = false;
  float thr = 0.f;
  if (act && mx != INT_MIN) {
    const float fm = key2f(mx);
    if (fabsf(fm) > 1e-8f && (sc == INT_MIN || key2f(sc) < fm - 1e-3f * fabsf(fm))) {
      const SlotCand w = sl[mx & (kMaxSlots - 1)];
      best = Cand{w.num, w.dg, w.l};
    } else {
      tie = true;
      thr = fm - 2e-3f * fabsf(fm) - 1e-8f;
    }
  }
  if (__any_sync(0xffffffffu, tie)) {
    Cand tb{0, 1, INT_MAX};
    if (tie) {
      for (int s = sub; s < p.nslots; s += kRedLanes) {
        if (!used(s)) continue;
        const SlotCand c = sl[s];
        if (valid(c.l) && cand_score(c.num, c.dg) >= thr) {
          const Cand d{c.num, c.dg, c.l};
          if (cand_better(d, tb)) tb = d;
        }
      }
    }
#pragma unroll
    for (int o = kRedLanes / 2; o; o >>= 1) {
      Cand d;
      d.num = __shfl_xor_sync(0xffffffffu, tb.num, o);
      d.dg = __shfl_xor_sync(0xffffffffu, tb.dg, o);
      d.l = __shfl_xor_sync(0xffffffffu, tb.l, o);
      if (cand_better(d, tb)) tb = d;
    }
    if (tie) best = tb;
  }
  if (live && sub == 0) {
    if (Df == 0) {
      p.u0[poi] = 0;
      p.v0[poi] = 0;
      p.zncc0[poi] = 0.f;
      p.status[poi] = kZeroVarRef;
    } else if (best.l == INT_MAX) {
      p.u0[poi] = -R;
      p.v0[poi] = -R;
      p.zncc0[poi] = 0.f;
      p.status[poi] = kZeroVarDef;
    } else {
      p.u0[poi] = best.l % ow - R;
      p.v0[poi] = best.l / ow - R;
      p.zncc0[poi] = zncc_of(best.num, Df, best.dg);
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
  if (S > 64) return false;
  g->twk = S <= 16 ? 16 : S <= 32 ? 32 : 64;  // one swizzle width per A operand row
  g->sub = 64 / g->twk;
  g->sj = (S + g->sub - 1) / g->sub;
  if (nx == 0 || ny == 0) return false;
  // exact FP32 sums: at most 1024 nonzero products of |ab| <= 2^14 per
  // accumulator (taps at or beyond S are zero in the bank)
  g->rows_per_acc = 1024 / S;
  if (g->rows_per_acc > S) g->rows_per_acc = S;
  const int nacc = (S + g->rows_per_acc - 1) / g->rows_per_acc;
  // POI block of a tile: ncols x nrows_all POIs.  One CTA takes nrows_max
  // rows of it (a chunk), as many as keep the MMA's N <= 256 and the nacc
  // accumulators within 512 TMEM columns; chunks are balanced.
  g->ncols_max = (2 * R + kTileR - 1) / step + 1;
  const int nrows_all = (2 * R + kTileQ - 1) / step + 1;
  auto npad_of = [&](int r) { return (g->ncols_max * r + 15) / 16 * 16; };
  int rmax = 0;
  for (int r = 1; r <= nrows_all; ++r)
    if (npad_of(r) <= 256 && nacc * npad_of(r) <= 512) rmax = r;
  if (rmax == 0) return false;  // one row of POIs already exceeds N = 256
  g->nchunk = (nrows_all + rmax - 1) / rmax;
  g->nrows_max = (nrows_all + g->nchunk - 1) / g->nchunk;
  g->npad = npad_of(g->nrows_max);
  // two TMEM accumulator buffers where they fit in 512 columns, else one
  g->accbufs = 2 * nacc * g->npad <= 512 ? 2 : 1;
  int cols = 32;
  while (cols < g->accbufs * nacc * g->npad) cols *= 2;
  if (cols > 512) return false;
  g->tmem_cols = cols;
  // two A buffers where they fit beside at least two B stages, then as many
  // B stages as fit (one CTA per SM)
  {
    auto fits = [&](int st, int ab) {
      return tile_layout(S, g->twk, g->npad, st, ab).total <= 227 * 1024;
    };
    if (fits(2, 2)) g->abufs = 2;
    else if (fits(2, 1)) g->abufs = 1;
    else return false;
    int st = 2;
    while (st < kMaxStages && fits(st + 1, g->abufs)) ++st;
    g->stages = st;
  }
  g->arows = kTileQ + S - 1;
  g->xmin = (B - M - R) & ~7;  // tile columns start at multiples of 8 (TMA of A)
  g->ymin = B - M - R;
  const int xmax = B + (nx - 1) * step - M + R, ymax = B + (ny - 1) * step - M + R;
  g->ntx = (xmax - g->xmin) / kTileR + 1;
  g->nty = (ymax - g->ymin) / kTileQ + 1;
  // tiles met by one POI window (2R+1 positions) in x and y
  g->slots_x = (2 * R + kTileR - 1) / kTileR + 1;
  g->slots_y = (2 * R + kTileQ - 1) / kTileQ + 1;
  g->nslots = g->slots_x * g->slots_y;
  if (g->nslots > kMaxSlots) return false;  // slot index packed in 10 bits by the reduce
  // template bank: by image row where that is the smaller order (the
  // caller switches to the stacked order if the tensor map encoder refuses
  // the overlapping strides)
  {
    const long long over = (long long)(ny - 1) * step + (long long)g->sub * g->sj;
    const long long stacked = (long long)ny * g->sj;
    if (!search_tc_bank_order(g, over < stacked ? 1 : 0)) return false;
  }
  // phase images cover every A row / column a tile touches and every
  // template row, with room for an 8-column chunk past the last tap
  const int wneed = std::max(W, g->xmin + g->ntx * kTileR + g->twk + 16);
  const int hneed = std::max(H, g->ymin + g->nty * kTileQ + S + 1);
  g->phw = (wneed + 7) / 8 * 8;
  g->phh = hneed;
  // grid rows of the bank launch, 32-bit chunk indices of the phase images
  if (g->phh > 65535 || (long long)g->phh * g->phw >= (1ll << 31))
    return false;
  return true;
}

size_t search_tc_smem(const SearchTcParams& g) {
  return tile_layout(g.S, g.twk, g.npad, g.stages, g.abufs).total;
}

size_t search_tc_gph_elems(const SearchTcParams& g) { return (size_t)8 * g.phh * g.phw; }

size_t search_tc_phase_elems(const SearchTcParams& g) {
  return search_tc_gph_elems(g) + (size_t)g.bank_rows * g.nx * 64;
}

bool search_tc_bank_order(SearchTcParams* g, int overlap) {
  const long long rows = overlap ? (long long)(g->ny - 1) * g->step + (long long)g->sub * g->sj
                                 : (long long)g->ny * g->sj;
  // grid rows of the bank launch; bank of at most 2^32 elements
  if (rows > 65535 || (double)rows * g->nx * 64 >= 4294967296.0) return false;
  g->bank_overlap = overlap;
  g->bank_rows = (int)rows;
  return true;
}

size_t search_tc_posbox_elems(const SearchTcParams& g) {
  return (size_t)g.ntx * 8 * (size_t)g.nty * 16;
}

cudaError_t launch_boxmaps(const SearchTcParams& p, cudaStream_t st) {
  const size_t bsm = boxmap_smem(p.S);
  if (bsm > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(boxmap_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       227 * 1024);
  if (e != cudaSuccess) return e;
  dim3 grid((p.ntx * 8 + kBoxX - 1) / kBoxX, (p.nty * 16 + kBoxY - 1) / kBoxY, 2);
  boxmap_kernel<<<grid, 256, bsm, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_search_tc(const SearchTcParams& p, const CUtensorMap* tmA,
                             const CUtensorMap* tmB, cudaStream_t st, cudaStream_t side,
                             cudaEvent_t fork, cudaEvent_t join) {
  if (p.n_pois == 0) return cudaSuccess;
  const int pois_per_block = (256 / 32) * (32 / kRedLanes);
  const unsigned rblocks = (unsigned)((p.n_pois + pois_per_block - 1) / pois_per_block);
  cudaError_t e;
  // phase images and template bank (on side, beside the box-sum maps, when
  // given), then the box-sum maps
  const cudaStream_t pst = side ? side : st;
  if (side) {
    e = cudaEventRecord(fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, fork, 0);
    if (e != cudaSuccess) return e;
  }
  {
    const int chunks = p.phh * (p.phw / 8);  // 8-column chunks of a phase image
    phase_kernel<<<(chunks + 255) / 256, 256, 0, pst>>>(p);
    const int per_row = p.nx * 8;  // 16-byte chunks of a bank row
    bank_kernel<<<dim3((per_row + 127) / 128, (p.bank_rows + kBankRows - 1) / kBankRows), 128,
                  0, pst>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  {
    const size_t bsm = boxmap_smem(p.S);
    if (bsm > 227 * 1024) return cudaErrorInvalidConfiguration;
    e = cudaFuncSetAttribute(boxmap_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024);
    if (e != cudaSuccess) return e;
    dim3 grid((p.ntx * 8 + kBoxX - 1) / kBoxX, (p.nty * 16 + kBoxY - 1) / kBoxY, 2);
    boxmap_kernel<<<grid, 256, bsm, st>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (side) {
    e = cudaEventRecord(join, side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, join, 0);
    if (e != cudaSuccess) return e;
  }
  const size_t smem = search_tc_smem(p);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  // the limit, not this launch's size: a graph may hold launches of several
  // geometries, each checked against the attribute when the graph runs
  e = cudaFuncSetAttribute(tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int nitems = p.ntx * p.nty * p.nchunk;
  tile_kernel<<<(unsigned)std::max(1, std::min(nitems, nsm)), kThreads, smem, st>>>(p, *tmA, *tmB);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce_kernel<<<rblocks, 256, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace dic
