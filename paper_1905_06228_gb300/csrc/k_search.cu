// k_search.cu -- brute-force ZNCC integer search (Eq. 1, Section 2.1).
//
// One CTA per POI.  The reference subset (S x S, S = 2M+1) and the search
// window ((S+2R) x (S+2R)) are staged in shared memory by two TMA tile loads
// (8-bit boxes whose x origin is rounded down to 16 bytes; plain loads when
// the images are not 16-byte aligned).  Every candidate offset (du, dv) in
// [-R, R]^2 is then scored exactly:
//
//   with a = f - 128, b = g - 128 (exact in FP32, |a|,|b| <= 128):
//     Sa, Saa        integer sums of the subset (block reduction)
//     Sb, Sbb        integer box sums of the displaced subset (separable
//                    sliding sums over the byte window, in-place)
//     Sab            FP32 FMA correlation, register-blocked: a thread owns 12
//                    consecutive du of one dv; every partial sum is an
//                    integer below 2^24 (at most 1024 products of |ab| <=
//                    2^14 per float accumulator; flushed to int32 beyond),
//                    so the FP32 result is exact
//     num = N Sab - Sa Sb,  Df = N Saa - Sa^2,  Dg = N Sbb - Sb^2
//   C = num / sqrt(Df Dg) is Eq. 1 (covariance and variances are invariant
//   under the -128 shift).
//
// Candidates are compared exactly -- sign of num first, then num_a^2 Dg_b
// against num_b^2 Dg_a in 128-bit integers -- first within a thread, then by
// warp shuffles, then across warps; ties keep the lowest linear index
// (dv+R)(2R+1)+(du+R).  Dg = 0 (flat target) is never preferred.
#include "dic_device.cuh"
#include "dic_internal.cuh"

namespace dic {
namespace {

constexpr int TN = 12;         // outputs (consecutive du) per thread task
constexpr int kMaxThreads = 256;

struct Cand {
  long long num;
  long long dg;
  int l;  // linear index; INT_MAX = none
};

// 1 if C_a > C_b strictly (same Df > 0 on both sides).
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

// a preferred over b: valid and larger, or equal and lower index.
__device__ __forceinline__ bool cand_better(const Cand& a, const Cand& b) {
  if (a.l == INT_MAX) return false;
  if (b.l == INT_MAX) return true;
  if (zncc_greater(a.num, a.dg, b.num, b.dg)) return true;
  if (zncc_greater(b.num, b.dg, a.num, a.dg)) return false;
  return a.l < b.l;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Bounded wait on an mbarrier phase.  Returns false if the limit was hit.
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

struct Layout {
  int span;       // S + 2R
  int ow;         // outputs per row = 2R+1
  int strips;     // ceil(ow / TN)
  int WS;         // float window row stride
  int BWg, BWf;   // byte box widths (window, template)
  size_t off_bar, off_wb, off_tb, off_wf, off_tf, off_hs, off_red, total;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <int TW>
__host__ __device__ inline Layout make_layout(int S, int R) {
  Layout L;
  L.span = S + 2 * R;
  L.ow = 2 * R + 1;
  L.strips = (L.ow + TN - 1) / TN;
  int need = L.strips * TN + TW - 1;
  int ws = (need + 3) / 4 * 4;
  while (ws % 32 != 16) ws += 4;  // rows of a warp phase land on distinct banks
  L.WS = ws;
  L.BWg = tma_box_width(L.span);
  L.BWf = tma_box_width(S);
  size_t o = 0;
  L.off_bar = o;  o += 16;
  o = align_up(o, 128); L.off_wb = o; o += (size_t)L.span * L.BWg;
  o = align_up(o, 128); L.off_tb = o; o += (size_t)S * L.BWf;
  o = align_up(o, 16);  L.off_wf = o; o += (size_t)L.span * L.WS * 4;
  o = align_up(o, 16);  L.off_tf = o; o += (size_t)S * TW * 4;
  o = align_up(o, 16);  L.off_hs = o; o += (size_t)L.span * L.ow * 8;
  o = align_up(o, 16);  L.off_red = o; o += (kMaxThreads / 32) * 32 + 64;
  L.total = o;
  return L;
}

// The search of one POI by the whole CTA (any block size that is a multiple
// of 32, up to kMaxThreads).  TMA staging is used when p.use_tma is set and
// the tensor maps are given (one TMA transaction per call: parity 0).
template <int TW>
__device__ __forceinline__ void search_poi(const SearchParams& p, int64_t poi,
                                           const CUtensorMap* tm_ref, const CUtensorMap* tm_def,
                                           unsigned char* smem) {
  const int S = p.S, M = p.M, R = p.R;
  const Layout L = make_layout<TW>(S, R);
  const int x0 = M + R + 2 + (int)(poi % p.nx) * p.step;
  const int y0 = M + R + 2 + (int)(poi / p.nx) * p.step;
  const int tid = threadIdx.x, nthr = blockDim.x;

  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.off_bar);
  uint8_t* wb = smem + L.off_wb;
  uint8_t* tb = smem + L.off_tb;
  float* wf = reinterpret_cast<float*>(smem + L.off_wf);
  float* tf = reinterpret_cast<float*>(smem + L.off_tf);
  int2* hs = reinterpret_cast<int2*>(smem + L.off_hs);
  long long* red = reinterpret_cast<long long*>(smem + L.off_red);

  // ---- stage bytes: template box at (x0-M, y0-M), window at (x0-M-R, y0-M-R)
  const int wx = x0 - M - R, wy = y0 - M - R, tx0 = x0 - M, ty0 = y0 - M;
  int ox_g, ox_f;
  if (p.use_tma && tm_ref && tm_def) {
    ox_g = wx & 15;
    ox_f = tx0 & 15;
    if (tid == 0) {
      const uint32_t b = smem_u32(bar);
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      const uint32_t bytes = (uint32_t)(L.span * L.BWg + S * L.BWf);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes)
                   : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
          "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(wb)),
          "l"(tm_def), "r"(wx - ox_g), "r"(wy), "r"(b)
          : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
          "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(tb)),
          "l"(tm_ref), "r"(tx0 - ox_f), "r"(ty0), "r"(b)
          : "memory");
    }
    __syncthreads();  // barrier initialised before anyone polls it
    if (!mbar_wait(smem_u32(bar), 0, 1ll << 24)) {
      if (tid == 0) atomicOr(p.err_flag, 1u);
      // the copies may still land: keep waiting (bounded) before leaving
      mbar_wait(smem_u32(bar), 0, 1ll << 24);
      return;
    }
  } else {
    ox_g = 0;
    ox_f = 0;
    for (int i = tid; i < L.span * L.span; i += nthr) {
      int r = i / L.span, c = i % L.span;
      wb[r * L.BWg + c] = p.def[(size_t)(wy + r) * p.pitch + wx + c];
    }
    for (int i = tid; i < S * S; i += nthr) {
      int r = i / S, c = i % S;
      tb[r * L.BWf + c] = p.ref[(size_t)(ty0 + r) * p.pitch + tx0 + c];
    }
    __syncthreads();
  }

  // ---- centred floats, template sums
  long long sa = 0, saa = 0;
  for (int i = tid; i < S * TW; i += nthr) {
    int r = i / TW, c = i % TW;
    float v = 0.f;
    if (c < S) {
      int a = (int)tb[r * L.BWf + ox_f + c] - 128;
      sa += a;
      saa += a * a;
      v = (float)a;
    }
    tf[i] = v;
  }
  for (int i = tid; i < L.span * L.WS; i += nthr) {
    int r = i / L.WS, c = i % L.WS;
    wf[i] = c < L.span ? (float)((int)wb[r * L.BWg + ox_g + c] - 128) : 0.f;
  }
  // ---- horizontal sliding sums of b and b^2 over S columns, per (row, du)
  for (int t = tid; t < L.span * L.strips; t += nthr) {
    const int r = t / L.strips, du0 = (t % L.strips) * TN;
    const uint8_t* row = wb + r * L.BWg + ox_g;
    int s = 0, q = 0;
    for (int c = 0; c < S; ++c) {
      int b = (int)row[du0 + c] - 128;
      s += b;
      q += b * b;
    }
    for (int j = 0; j < TN && du0 + j < L.ow; ++j) {
      if (j) {
        int bi = (int)row[du0 + j + S - 1] - 128, bo = (int)row[du0 + j - 1] - 128;
        s += bi - bo;
        q += bi * bi - bo * bo;
      }
      hs[r * L.ow + du0 + j] = make_int2(s, q);
    }
  }
  // block reduction of the template sums
  for (int o = 16; o; o >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    saa += __shfl_xor_sync(0xffffffffu, saa, o);
  }
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
  if (lane == 0) {
    red[2 * warp] = sa;
    red[2 * warp + 1] = saa;
  }
  __syncthreads();
  // ---- vertical sliding sums in place: hs[dv][du] <- box sums at (dv, du)
  for (int du = tid; du < L.ow; du += nthr) {
    int s = 0, q = 0;
    for (int r = 0; r < S; ++r) {
      int2 h = hs[r * L.ow + du];
      s += h.x;
      q += h.y;
    }
    for (int dv = 0; dv < L.ow; ++dv) {
      int2 old = hs[dv * L.ow + du];
      hs[dv * L.ow + du] = make_int2(s, q);
      if (dv + S < L.span) {
        int2 in = hs[(dv + S) * L.ow + du];
        s += in.x - old.x;
        q += in.y - old.y;
      }
    }
  }
  long long Sa = 0, Saa = 0;
  for (int w = 0; w < nwarps; ++w) {
    Sa += red[2 * w];
    Saa += red[2 * w + 1];
  }
  const long long N = (long long)S * S;
  const long long Df = N * Saa - Sa * Sa;
  __syncthreads();  // box sums, floats ready; red[] free again

  if (Df == 0) {
    if (tid == 0) {
      p.u0[poi] = 0;
      p.v0[poi] = 0;
      p.zncc0[poi] = 0.f;
      p.status[poi] = kZeroVarRef;
    }
    return;
  }

  // ---- correlation: thread task = (dv, strip of TN du)
  constexpr bool kFlush = TW > 32;
  constexpr int RF = 1024 / TW;  // rows per exact FP32 accumulation block
  Cand best{0, 1, INT_MAX};
  const int ntask = L.ow * L.strips;
  for (int t = tid; t < ntask; t += nthr) {
    const int dv = t / L.strips, du0 = (t % L.strips) * TN;
    float acc[TN];
    int iacc[TN];
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      acc[j] = 0.f;
      iacc[j] = 0;
    }
    int since = 0;
    for (int ty = 0; ty < S; ++ty) {
      const float4* wrow = reinterpret_cast<const float4*>(wf + (ty + dv) * L.WS + du0);
      const float4* trow = reinterpret_cast<const float4*>(tf + ty * TW);
      constexpr int NW = (TN + TW - 1 + 3) / 4;
      float w[NW * 4];
#pragma unroll
      for (int k = 0; k < NW; ++k) {
        float4 v = wrow[k];
        w[4 * k] = v.x;
        w[4 * k + 1] = v.y;
        w[4 * k + 2] = v.z;
        w[4 * k + 3] = v.w;
      }
#pragma unroll
      for (int k = 0; k < TW / 4; ++k) {
        const float4 tv = trow[k];
        const float tt[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[j] = fmaf(tt[e], w[4 * k + e + j], acc[j]);
      }
      if (kFlush && ++since == RF) {
        since = 0;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          iacc[j] += __float2int_rn(acc[j]);
          acc[j] = 0.f;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int du = du0 + j;
      if (du >= L.ow) break;
      const int2 bx = hs[dv * L.ow + du];
      const long long sb = bx.x, sbb = bx.y;
      const long long sab = (long long)iacc[j] + (long long)__float2int_rn(acc[j]);
      const long long dg = N * sbb - sb * sb;
      if (dg == 0) continue;
      Cand c{N * sab - Sa * sb, dg, dv * L.ow + du};
      if (cand_better(c, best)) best = c;
    }
  }
  // ---- argmax: warp shuffles, then across warps
  for (int o = 16; o; o >>= 1) {
    Cand c;
    c.num = __shfl_xor_sync(0xffffffffu, best.num, o);
    c.dg = __shfl_xor_sync(0xffffffffu, best.dg, o);
    c.l = __shfl_xor_sync(0xffffffffu, best.l, o);
    if (cand_better(c, best)) best = c;
  }
  if (lane == 0) {
    red[3 * warp] = best.num;
    red[3 * warp + 1] = best.dg;
    red[3 * warp + 2] = best.l;
  }
  __syncthreads();
  if (tid == 0) {
    Cand b{red[0], red[1], (int)red[2]};
    for (int w = 1; w < nwarps; ++w) {
      Cand c{red[3 * w], red[3 * w + 1], (int)red[3 * w + 2]};
      if (cand_better(c, b)) b = c;
    }
    if (b.l == INT_MAX) {
      p.u0[poi] = -R;
      p.v0[poi] = -R;
      p.zncc0[poi] = 0.f;
      p.status[poi] = kZeroVarDef;
    } else {
      p.u0[poi] = b.l % L.ow - R;
      p.v0[poi] = b.l / L.ow - R;
      p.zncc0[poi] = zncc_of(b.num, Df, b.dg);
      p.status[poi] = kOk;
    }
  }
}

// One CTA per POI of one pair.
template <int TW>
__global__ void __launch_bounds__(kMaxThreads)
search_kernel(const SearchParams p, const __grid_constant__ CUtensorMap tm_ref,
              const __grid_constant__ CUtensorMap tm_def) {
  extern __shared__ __align__(128) unsigned char smem[];
  if ((int64_t)blockIdx.x >= p.n_pois) return;
  search_poi<TW>(p, blockIdx.x, &tm_ref, &tm_def, smem);
}

// Persistent form over many pairs: each CTA takes the next POI of the whole
// batch from a global counter (items ordered pair by pair, so one pair's
// window data stays hot in L2), finds its pair by bisection of the prefix
// offsets, and searches it with plain staging loads.
template <int TW>
__global__ void __launch_bounds__(kMaxThreads)
search_batch_kernel(const SearchParams* __restrict__ jobs, const int64_t* __restrict__ offsets,
                    int njobs, unsigned long long* counter) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ long long item_s;
  const int64_t total = offsets[njobs];
  for (;;) {
    if (threadIdx.x == 0) item_s = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t item = item_s;
    __syncthreads();
    if (item >= total) break;
    int lo = 0, hi = njobs;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (offsets[mid] <= item) lo = mid; else hi = mid;
    }
    const SearchParams p = jobs[lo];
    search_poi<TW>(p, item - offsets[lo], nullptr, nullptr, smem);
    __syncthreads();
  }
}

template <int TW>
cudaError_t launch_tw(const SearchParams& p, const CUtensorMap* tr, const CUtensorMap* td,
                      cudaStream_t st) {
  const Layout L = make_layout<TW>(p.S, p.R);
  if (L.total > 227 * 1024) return cudaErrorInvalidConfiguration;
  if (L.total > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(search_kernel<TW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L.total);
    if (e != cudaSuccess) return e;
  }
  int tasks = L.ow * L.strips;
  int thr = ((tasks + 31) / 32) * 32;
  if (thr > kMaxThreads) thr = kMaxThreads;
  search_kernel<TW><<<(unsigned)p.n_pois, thr, L.total, st>>>(p, *tr, *td);
  return cudaGetLastError();
}

template <int TW>
cudaError_t launch_batch_tw(const SearchParams* jobs, const int64_t* offsets, int njobs,
                            unsigned long long* counter, size_t smem, int grid, cudaStream_t st) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(search_batch_kernel<TW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  search_batch_kernel<TW><<<grid, kMaxThreads, smem, st>>>(jobs, offsets, njobs, counter);
  return cudaGetLastError();
}

template <int TW>
int batch_ctas_per_sm(size_t smem) {
  int n = 0;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(search_batch_kernel<TW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, search_batch_kernel<TW>, kMaxThreads, smem);
  return n;
}

}  // namespace

size_t search_smem_bytes(int S, int R);

#define DIC_TW_SWITCH(tw, CALL)                                                          \
  switch (tw) {                                                                          \
    case 4: CALL(4); case 8: CALL(8); case 12: CALL(12); case 16: CALL(16);            \
    case 20: CALL(20); case 24: CALL(24); case 28: CALL(28); case 32: CALL(32);        \
    case 36: CALL(36); case 40: CALL(40); case 44: CALL(44); case 48: CALL(48);        \
    case 52: CALL(52); case 56: CALL(56); case 60: CALL(60); case 64: CALL(64);        \
    default: break;                                                                      \
  }

cudaError_t launch_search_batch(int tw, const SearchParams* jobs, const int64_t* offsets,
                                int njobs, unsigned long long* counter, size_t smem, int grid,
                                cudaStream_t st) {
#define DIC_CALL(T) return launch_batch_tw<T>(jobs, offsets, njobs, counter, smem, grid, st)
  DIC_TW_SWITCH(tw, DIC_CALL)
#undef DIC_CALL
  return cudaErrorInvalidValue;
}

int search_batch_occupancy(int tw, size_t smem) {
#define DIC_CALL(T) return batch_ctas_per_sm<T>(smem)
  DIC_TW_SWITCH(tw, DIC_CALL)
#undef DIC_CALL
  return 0;
}

cudaError_t launch_search(const SearchParams& p, const CUtensorMap* tm_ref,
                          const CUtensorMap* tm_def, cudaStream_t st) {
  if (p.n_pois == 0) return cudaSuccess;
  const int tw = (p.S + 3) / 4 * 4;
  switch (tw) {
    case 4: return launch_tw<4>(p, tm_ref, tm_def, st);
    case 8: return launch_tw<8>(p, tm_ref, tm_def, st);
    case 12: return launch_tw<12>(p, tm_ref, tm_def, st);
    case 16: return launch_tw<16>(p, tm_ref, tm_def, st);
    case 20: return launch_tw<20>(p, tm_ref, tm_def, st);
    case 24: return launch_tw<24>(p, tm_ref, tm_def, st);
    case 28: return launch_tw<28>(p, tm_ref, tm_def, st);
    case 32: return launch_tw<32>(p, tm_ref, tm_def, st);
    case 36: return launch_tw<36>(p, tm_ref, tm_def, st);
    case 40: return launch_tw<40>(p, tm_ref, tm_def, st);
    case 44: return launch_tw<44>(p, tm_ref, tm_def, st);
    case 48: return launch_tw<48>(p, tm_ref, tm_def, st);
    case 52: return launch_tw<52>(p, tm_ref, tm_def, st);
    case 56: return launch_tw<56>(p, tm_ref, tm_def, st);
    case 60: return launch_tw<60>(p, tm_ref, tm_def, st);
    case 64: return launch_tw<64>(p, tm_ref, tm_def, st);
    default: return cudaErrorInvalidValue;
  }
}

size_t search_smem_bytes(int S, int R) {
  const int tw = (S + 3) / 4 * 4;
  // the layout depends on TW only through the template row width
  Layout L;
  switch (tw) {
#define DIC_CASE(T) case T: L = make_layout<T>(S, R); break;
    DIC_CASE(4) DIC_CASE(8) DIC_CASE(12) DIC_CASE(16) DIC_CASE(20) DIC_CASE(24) DIC_CASE(28)
    DIC_CASE(32) DIC_CASE(36) DIC_CASE(40) DIC_CASE(44) DIC_CASE(48) DIC_CASE(52)
    DIC_CASE(56) DIC_CASE(60) DIC_CASE(64)
#undef DIC_CASE
    default: return (size_t)-1;
  }
  return L.total;
}

}  // namespace dic
