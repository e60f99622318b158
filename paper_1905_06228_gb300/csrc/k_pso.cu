// k_pso.cu -- integer search by particle swarm optimisation (Section 2.1,
// Eqs. 2-4) and by the modified swarm whose particles also evaluate the four
// pixels around their own, the star search folded into the swarm (Sections
// 3 and 5).
//
// Per POI, with the swarm's random numbers as inputs rand[k][t][i][0..3]
// (uniforms in [0,1); t the generation, i the particle):
//   t = 0   p_i = R (2 u_0 - 1, 2 u_1 - 1),  v_i = vinit (2 u_2 - 1, 2 u_3 - 1)
//   t >= 1  v <- ((w v) + (c1 r1)(pbest - p)) + (c2 r2)(gbest - p)   (Eq. 2)
//           with w = 0.9 - (t - 1) / (2 gmax)                          (Eq. 4)
//           and r1 = (u_0, u_1), r2 = (u_2, u_3) per direction; then
//           p <- p + v (Eq. 3), clamped to [-R, R] per direction.
//   Every generation each particle evaluates Eq. 1 at its nearest pixel
//   q = floor(p + 1/2); the modified swarm also evaluates q +- (1, 0) and
//   q +- (0, 1) inside the window, keeps the best of the five (ties: centre,
//   +x, -x, +y, -y) and moves onto it.  pbest takes the evaluated pixel if
//   it is strictly better (at t = 0 unconditionally); gbest then takes the
//   first strictly better pbest in particle order.  The swarm stops after
//   gmax generations or after the first generation whose gbest reaches
//   C >= stop_num / stop_den, tested exactly.
// The particle arithmetic is FP64 with every product and sum rounded on its
// own (no fused multiply-add), in the order written above, so every integer
// decision -- the nearest pixel, the clamp, the comparisons -- is the one an
// FP64 evaluation of the same formulas in that order takes.
//
// Layout: one warp per POI.  The search window of g ((S + 2R)^2 bytes) is
// staged in shared memory; each lane holds a fixed share of the reference
// subset as packed 4-byte words in registers.  Eq. 1 at a pixel (du, dv) is
// computed from exact integer sums: Sfg = sum f g by byte dot products
// (dp4a) over the lanes' words and a warp reduction; Sg, Sgg from the box-sum
// map of g, Sf, Sff from the map of f.  A pixel is evaluated at most once per
// POI (a table of Sfg in shared memory), so the evaluation count is the
// number of distinct pixels the swarm visited.  Candidates compare exactly
// (sign of num, then num_a^2 den_b against num_b^2 den_a in 128-bit
// integers); a pixel whose target subset is flat ranks below all others.
#include "dic_device.cuh"
#include "dic_internal.cuh"

namespace dic {
namespace {

constexpr int kMaxParticles = 64;  // two particles per lane

struct Zc {
  long long num, den;  // C = num / sqrt(Df den)
  bool def;            // den != 0
};

// a strictly better than b (same Df > 0).
__device__ __forceinline__ bool zc_greater(const Zc& a, const Zc& b) {
  if (!a.def) return false;
  if (!b.def) return true;
  if (a.num >= 0 && b.num < 0) return true;
  if (a.num < 0 && b.num >= 0) return false;
  const unsigned long long na = (unsigned long long)(a.num < 0 ? -a.num : a.num);
  const unsigned long long nb = (unsigned long long)(b.num < 0 ? -b.num : b.num);
  const unsigned __int128 lhs = (unsigned __int128)na * na * (unsigned long long)b.den;
  const unsigned __int128 rhs = (unsigned __int128)nb * nb * (unsigned long long)a.den;
  return a.num >= 0 ? lhs > rhs : lhs < rhs;
}

// C >= sn / sd exactly (num >= 0; sn, sd <= 2^20).
__device__ __forceinline__ bool zc_at_least(const Zc& a, long long df, long long sn,
                                            long long sd) {
  if (!a.def || a.num < 0) return false;
  const unsigned __int128 n2 = (unsigned __int128)(unsigned long long)a.num * (unsigned long long)a.num;
  const unsigned __int128 lhs = n2 * (unsigned long long)(sd * sd);
  const unsigned __int128 rhs = (unsigned __int128)(unsigned long long)(sn * sn) *
                                (unsigned long long)df * (unsigned long long)a.den;
  return lhs >= rhs;
}

__device__ __forceinline__ Zc shfl_zc(const Zc& z, int src) {
  Zc o;
  o.num = __shfl_sync(0xffffffffu, z.num, src);
  o.den = __shfl_sync(0xffffffffu, z.den, src);
  o.def = __shfl_sync(0xffffffffu, (int)z.def, src) != 0;
  return o;
}

__device__ __forceinline__ int iabs(int x) { return x < 0 ? -x : x; }

template <int SLOTS>
__global__ void __launch_bounds__(128) pso_kernel(const PsoParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t poi = (int64_t)blockIdx.x * p.warps + wid;
  if (poi >= p.n_pois) return;
  const int S = p.S, M = p.M, R = p.R, span = S + 2 * R, ow = 2 * R + 1, WP = p.wp;
  const int P = p.particles;
  const long long N = (long long)S * S;
  unsigned char* win = smem + (size_t)wid * p.warp_smem;         // [span][WP] bytes of g
  int* memo = reinterpret_cast<int*>(win + (size_t)span * WP);   // [ow][ow] Sfg, -1 = not yet
  int2* gbox = reinterpret_cast<int2*>(memo + (size_t)ow * ow);  // [P][5] box sums of g
  const int x0 = M + R + 2 + (int)(poi % p.nx) * p.step;
  const int y0 = M + R + 2 + (int)(poi / p.nx) * p.step;

  // ---- window of g, evaluation table, the lanes' words of the reference subset
  {
    const uint8_t* src = p.def + (size_t)(y0 - M - R) * p.pitch + (x0 - M - R);
    for (int i = lane; i < span * span; i += 32) {
      const int r = i / span, c = i - r * span;
      win[r * WP + c] = __ldg(src + (size_t)r * p.pitch + c);
    }
    for (int i = lane; i < ow * ow; i += 32) memo[i] = -1;
  }
  const int wpr = (S + 3) / 4;  // words per subset row
  unsigned fw[SLOTS];
  int off[SLOTS];
#pragma unroll
  for (int j = 0; j < SLOTS; ++j) {
    const int q = lane + 32 * j;
    fw[j] = 0u;
    off[j] = 0;
    if (q < S * wpr) {
      const int r = q / wpr, k = q - r * wpr;
      const uint8_t* fr = p.ref + (size_t)(y0 - M + r) * p.pitch + (x0 - M + 4 * k);
      unsigned w = 0u;
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (4 * k + b < S) w |= (unsigned)__ldg(fr + b) << (8 * b);
      fw[j] = w;
      off[j] = r * WP + 4 * k;
    }
  }
  const int2 fb = __ldg(p.fbox + (size_t)(y0 - M - p.ymin) * p.pw + (x0 - M - p.xmin));
  const long long Sf = (long long)fb.x + 128 * N;  // sums of f itself (the map is centred)
  const long long Df = N * (long long)fb.y - (long long)fb.x * fb.x;
  __syncwarp();
  auto write_out = [&](int u, int v, float zn, uint8_t st, int gens, int evals) {
    if (lane == 0) {
      p.u0[poi] = u;
      p.v0[poi] = v;
      p.zncc0[poi] = zn;
      p.status[poi] = st;
      p.gens[poi] = gens;
      p.evals[poi] = evals;
    }
  };
  if (Df == 0) {
    write_out(0, 0, 0.f, kZeroVarRef, 0, 0);
    return;
  }

  // Eq. 1 at pixel (du, dv) of the window, its box sums given; every lane
  // returns the same value.
  int evals = 0;
  auto evaluate = [&](int du, int dv, int2 box) -> Zc {
    const int slot = (dv + R) * ow + (du + R);
    int sfg = memo[slot];
    if (sfg < 0) {
      const int base = (R + dv) * WP + (R + du);
      const int sh = (base & 3) * 8, ab = base & ~3;
      unsigned acc = 0u;
#pragma unroll
      for (int j = 0; j < SLOTS; ++j) {
        const unsigned* w = reinterpret_cast<const unsigned*>(win + ab + off[j]);
        acc = __dp4a(fw[j], __funnelshift_r(w[0], w[1], sh), acc);
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      sfg = (int)acc;
      __syncwarp();
      if (lane == 0) memo[slot] = sfg;
      __syncwarp();
      ++evals;
    }
    const long long sg = (long long)box.x + 128 * N;
    Zc z;
    z.den = N * (long long)box.y - (long long)box.x * box.x;
    z.num = N * (long long)sfg - Sf * sg;
    z.def = z.den != 0;
    return z;
  };
  auto box_of = [&](int du, int dv) -> int2 {
    return __ldg(p.posbox + (size_t)(y0 - M + dv - p.ymin) * p.pw + (x0 - M + du - p.xmin));
  };

  // ---- particles: particle i lives on lane i % 32, slot i / 32
  double px[2], py[2], vx[2], vy[2];
  int qx[2], qy[2], bx[2], by[2];
  Zc pbc[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    px[s] = py[s] = vx[s] = vy[s] = 0.0;
    qx[s] = qy[s] = bx[s] = by[s] = 0;
    pbc[s] = Zc{0, 0, false};
  }
  int gbx = 0, gby = 0;
  Zc gc{0, 0, false};
  int gens = 0;
  const double dR = (double)R;
  const double* rbase = p.rand + (size_t)poi * p.gmax * P * 4;
  for (int t = 0; t < p.gmax; ++t) {
    const double* rt = rbase + (size_t)t * P * 4;
    const double w = __dsub_rn(0.9, __ddiv_rn((double)(t - 1), __dmul_rn(2.0, (double)p.gmax)));
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int i = lane + 32 * s;
      if (i >= P) continue;
      const double u0 = __ldg(rt + i * 4), u1 = __ldg(rt + i * 4 + 1);
      const double u2 = __ldg(rt + i * 4 + 2), u3 = __ldg(rt + i * 4 + 3);
      if (t == 0) {
        px[s] = __dmul_rn(dR, __dsub_rn(__dmul_rn(2.0, u0), 1.0));
        py[s] = __dmul_rn(dR, __dsub_rn(__dmul_rn(2.0, u1), 1.0));
        vx[s] = __dmul_rn(p.vinit, __dsub_rn(__dmul_rn(2.0, u2), 1.0));
        vy[s] = __dmul_rn(p.vinit, __dsub_rn(__dmul_rn(2.0, u3), 1.0));
      } else {
        // Eq. 2, then Eq. 3 and the window clamp, per direction
        const double ix = __dmul_rn(w, vx[s]);
        const double cx = __dmul_rn(__dmul_rn(p.c1, u0), __dsub_rn((double)bx[s], px[s]));
        const double sx = __dmul_rn(__dmul_rn(p.c2, u2), __dsub_rn((double)gbx, px[s]));
        vx[s] = __dadd_rn(__dadd_rn(ix, cx), sx);
        const double nx = __dadd_rn(px[s], vx[s]);
        px[s] = nx < -dR ? -dR : (nx > dR ? dR : nx);
        const double iy = __dmul_rn(w, vy[s]);
        const double cy = __dmul_rn(__dmul_rn(p.c1, u1), __dsub_rn((double)by[s], py[s]));
        const double sy = __dmul_rn(__dmul_rn(p.c2, u3), __dsub_rn((double)gby, py[s]));
        vy[s] = __dadd_rn(__dadd_rn(iy, cy), sy);
        const double ny = __dadd_rn(py[s], vy[s]);
        py[s] = ny < -dR ? -dR : (ny > dR ? dR : ny);
      }
      qx[s] = (int)floor(__dadd_rn(px[s], 0.5));
      qy[s] = (int)floor(__dadd_rn(py[s], 0.5));
    }
    // box sums of every pixel this generation evaluates, fetched together
    // (one round of memory latency per generation)
    const int npts = p.modified ? 5 : 1;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int i = lane + 32 * s;
      if (i >= P) continue;
      for (int j = 0; j < npts; ++j) {
        const int du = qx[s] + (j == 1 ? 1 : j == 2 ? -1 : 0);
        const int dv = qy[s] + (j == 3 ? 1 : j == 4 ? -1 : 0);
        if (iabs(du) <= R && iabs(dv) <= R) gbox[i * 5 + j] = box_of(du, dv);
      }
    }
    __syncwarp();
    // evaluations, particle by particle (the table makes the order matter
    // only for which evaluation computes a pixel first)
    for (int i = 0; i < P; ++i) {
      const int src = i & 31, s = i >> 5;
      const int cqx = __shfl_sync(0xffffffffu, s ? qx[1] : qx[0], src);
      const int cqy = __shfl_sync(0xffffffffu, s ? qy[1] : qy[0], src);
      int best_x = cqx, best_y = cqy;
      Zc bc = evaluate(cqx, cqy, gbox[i * 5]);
      if (p.modified) {
#pragma unroll
        for (int j = 1; j < 5; ++j) {
          const int du = cqx + (j == 1 ? 1 : j == 2 ? -1 : 0);
          const int dv = cqy + (j == 3 ? 1 : j == 4 ? -1 : 0);
          if (iabs(du) > R || iabs(dv) > R) continue;
          const Zc z = evaluate(du, dv, gbox[i * 5 + j]);
          if (zc_greater(z, bc)) {
            best_x = du;
            best_y = dv;
            bc = z;
          }
        }
      }
      if (lane == src) {
#pragma unroll
        for (int ss = 0; ss < 2; ++ss) {
          if (ss != s) continue;
          if (p.modified) {
            px[ss] = (double)best_x;
            py[ss] = (double)best_y;
          }
          if (t == 0 || zc_greater(bc, pbc[ss])) {
            bx[ss] = best_x;
            by[ss] = best_y;
            pbc[ss] = bc;
          }
        }
      }
    }
    __syncwarp();
    // gbest: the first particle (in particle order) holding the largest
    // pbest, taken if it beats the current gbest strictly (at t = 0 it is
    // taken unconditionally) -- what a scan in particle order with a strict
    // comparison yields
    Zc mz = pbc[0];
    int mi = lane, mx = bx[0], my = by[0];
    if (lane + 32 < P && zc_greater(pbc[1], mz)) {
      mz = pbc[1];
      mi = lane + 32;
      mx = bx[1];
      my = by[1];
    }
    if (lane >= P) mi = 1 << 30;  // no particle on this lane
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const Zc oz = shfl_zc(mz, lane ^ o);
      const int oi = __shfl_xor_sync(0xffffffffu, mi, o);
      const int ox = __shfl_xor_sync(0xffffffffu, mx, o);
      const int oy = __shfl_xor_sync(0xffffffffu, my, o);
      bool take;
      if (oi >= (1 << 30)) take = false;
      else if (mi >= (1 << 30)) take = true;
      else if (zc_greater(oz, mz)) take = true;
      else if (zc_greater(mz, oz)) take = false;
      else take = oi < mi;
      if (take) {
        mz = oz;
        mi = oi;
        mx = ox;
        my = oy;
      }
    }
    if (t == 0 || zc_greater(mz, gc)) {
      gc = mz;
      gbx = mx;
      gby = my;
    }
    gens = t + 1;
    if (zc_at_least(gc, Df, p.stop_num, p.stop_den)) break;
  }
  if (!gc.def) {
    write_out(gbx, gby, 0.f, kZeroVarDef, gens, evals);
    return;
  }
  write_out(gbx, gby, zncc_of(gc.num, Df, gc.den), kOk, gens, evals);
}

template <int SLOTS>
cudaError_t launch_slots(const PsoParams& p, cudaStream_t st) {
  const size_t smem = (size_t)p.warps * p.warp_smem;
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(pso_kernel<SLOTS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((p.n_pois + p.warps - 1) / p.warps);
  pso_kernel<SLOTS><<<grid, 32 * p.warps, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

size_t pso_warp_smem(int S, int R, int particles, int* wp) {
  if (particles < 1 || particles > kMaxParticles) return 0;
  const int span = S + 2 * R, ow = 2 * R + 1;
  // row pitch: room for the word after the last one a lane reads, a
  // multiple of 4 bytes and an odd number of words (rows spread over banks)
  int w = (span + 8 + 3) / 4;
  if ((w & 1) == 0) ++w;
  if (wp) *wp = 4 * w;
  const size_t bytes = (size_t)span * 4 * w + (size_t)ow * ow * sizeof(int) +
                       (size_t)particles * 5 * sizeof(int2);
  const size_t aligned = (bytes + 15) / 16 * 16;
  return aligned <= 227 * 1024 ? aligned : 0;
}

cudaError_t launch_pso(const PsoParams& p, cudaStream_t st) {
  if (p.n_pois == 0) return cudaSuccess;
  const int slots = (p.S * ((p.S + 3) / 4) + 31) / 32;
  if (slots <= 8) return launch_slots<8>(p, st);
  if (slots <= 16) return launch_slots<16>(p, st);
  if (slots <= 32) return launch_slots<32>(p, st);
  return cudaErrorInvalidValue;
}

}  // namespace dic
