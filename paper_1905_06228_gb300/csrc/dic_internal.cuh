// dic_internal.cuh -- handle layout and kernel launch interfaces shared by the
// translation units of the CUDA library (not part of the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dic.h"

namespace dic {

// POI status codes (mirrors DIC_POI_* of dic.h).
enum : uint8_t {
  kOk = 0,
  kZeroVarRef = 1,
  kOutOfBounds = 2,
  kMaxIter = 3,
  kNonFinite = 4,
  kSingular = 5,
  kZeroVarDef = 6
};

constexpr int kMaxSubset = 63;

// Geometry of one bound image pair.
struct PairGeom {
  int W = 0, H = 0, pitch = 0;
  int nx = 0, ny = 0;
  int64_t n_pois = 0;
};

// Parameters of the integer search kernel.
struct SearchParams {
  const uint8_t* ref;
  const uint8_t* def;
  int W, H, pitch;
  int S, M, R, step, nx;
  int64_t n_pois;
  int use_tma;
  int32_t* u0;
  int32_t* v0;
  float* zncc0;
  uint8_t* status;
  unsigned int* err_flag;  // set when a bounded wait gives up
};

// Best candidate of one (position tile, POI) pair in the tensor-core search.
struct SlotCand {
  long long num, dg;
  int l, pad;
};

// Parameters of the tensor-core integer search (k_search_tc.cu).
struct SearchTcParams {
  const uint8_t* ref;
  const uint8_t* def;
  int W, H, pitch;
  int S, M, R, step, nx, ny;
  int64_t n_pois;
  int twk;           // template row width padded to 16 taps (taps per A operand row)
  int sub;           // template rows per B operand row of 64 taps: 64 / twk
  int sj;            // B operand rows per template: ceil(S / sub)
  int bank_overlap;  // 1: bank rows by image row, 0: [ny][sj] (see bank_kernel)
  int bank_rows;
  int npad;          // N of the MMA (POIs per tile block, padded to 16)
  int ncols_max, nrows_max;  // POI block of a tile's CTA (columns, rows of one chunk)
  int nchunk;                // CTAs per tile, each taking nrows_max rows of POIs
  int arows;                 // image rows of a tile's A buffer
  int rows_per_acc;  // template rows per exact FP32 accumulator
  int tmem_cols;
  int accbufs;       // TMEM accumulator buffers of the tile kernel (1 or 2)
  int abufs;         // A buffers of the tile kernel (1 or 2)
  int stages;        // B stages of the tile kernel's ring
  int xmin, ymin, ntx, nty;
  int slots_x, slots_y, nslots;
  uint16_t* bank;    // [bank_rows][nx][64] centred BF16 subsets of f (see bank_kernel)
  uint16_t* gph;     // [8][phh][phw] centred BF16 copies of g shifted by 0..7
  int phh, phw;
  int2* fbox;        // like posbox, for the reference image (POI sums)
  SlotCand* slots;   // [n_pois][nslots]
  int2* posbox;      // [nty*16][ntx*8] box sums of the position domain
  int32_t* u0;
  int32_t* v0;
  float* zncc0;
  uint8_t* status;
  unsigned int* err_flag;
};

// Parameters of the particle swarm integer search (k_pso.cu).
struct PsoParams {
  const uint8_t* ref;
  const uint8_t* def;
  int W, H, pitch;
  int S, M, R, step, nx;
  int64_t n_pois;
  int modified, particles, gmax;
  double c1, c2, vinit;
  long long stop_num, stop_den;
  const double* rand;  // [n_pois][gmax][particles][4]
  const int2* posbox;  // box sums (sum b - 128, sum (b - 128)^2) of g per subset top-left
  const int2* fbox;    // the same for f
  int xmin, ymin, pw;  // top-left (x, y) of map entry 0, map row length
  int wp;              // byte pitch of a warp's window rows in shared memory
  int warps;           // warps (POIs) per CTA
  size_t warp_smem;    // shared bytes per warp
  int32_t* u0;
  int32_t* v0;
  float* zncc0;
  uint8_t* status;
  int32_t* gens;
  int32_t* evals;
};

// Parameters of the sub-pixel kernels.  The reference image is 8-bit
// (ref) or float (ref_f32 != nullptr); pitch is in elements.
struct SubpixelParams {
  const uint8_t* ref = nullptr;
  const float* ref_f32 = nullptr;
  const float2* grad;  // central-difference gradients of f, W*H
  const float* gimg;   // deformed image as float, W*H
  const uint2* gq = nullptr;  // 8-bit pairs: BF16 tap quads of g, W*H (required)
  int W, H, pitch;
  int S, M, R, step, nx;
  int64_t n_pois;
  int max_iter;
  float tol;
  const int32_t* u0;
  const int32_t* v0;
  const uint8_t* st0;
  float* u;
  float* v;
  float* ux;
  float* uy;
  float* vx;
  float* vy;
  float* zncc;
  int32_t* iters;
  uint8_t* status;
};

// Parameters of the ZNSSD forward / adjoint kernel.
struct AdjointParams {
  const uint8_t* ref = nullptr;
  const float* ref_f32 = nullptr;
  const float* gimg;   // deformed image as float, W*H
  int W, H, pitch;
  int S, M, R, step, nx;
  int64_t n_pois;
  const float* p6;          // [n_pois][6]
  float* loss_poi;          // may be null
  float* loss_total;        // may be null (zeroed by the caller)
  int backward;             // 0: forward only
  const float* grad_loss;   // [n_pois] upstream weights or null (= 1)
  float scale;
  float* dL_ddef;           // [H][W], zeroed by the caller
  float* dL_dp;             // [n_pois][6] or null
};

// Launchers (each returns the cudaError_t of its launch).
cudaError_t launch_precompute(const uint8_t* ref, const uint8_t* def, int W, int H,
                              int pitch, float2* grad, float* gimg, uint2* gq, cudaStream_t st);
cudaError_t launch_precompute_f32(const float* ref, const float* def, int W, int H,
                                  int pitch, float2* grad, float* gimg, cudaStream_t st);
cudaError_t launch_adjoint(const AdjointParams& p, cudaStream_t st);

bool search_tc_geometry(int W, int H, int S, int step, int R, int nx, int ny, SearchTcParams* g);
size_t search_tc_smem(const SearchTcParams& g);
size_t search_tc_posbox_elems(const SearchTcParams& g);
size_t search_tc_phase_elems(const SearchTcParams& g);  // phase images + template bank
size_t search_tc_gph_elems(const SearchTcParams& g);
// Sets the bank's row order (1: by image row, 0: stacked) and its row
// count; false if that order exceeds the bank's limits.
bool search_tc_bank_order(SearchTcParams* g, int overlap);
// With side (and its two events) the phase images and template bank run on
// side, forked from st, beside the box-sum maps, and st joins it before the
// tile kernel.
cudaError_t launch_search_tc(const SearchTcParams& p, const CUtensorMap* tmA,
                             const CUtensorMap* tmB, cudaStream_t st, cudaStream_t side = nullptr,
                             cudaEvent_t fork = nullptr, cudaEvent_t join = nullptr);
// Box-sum maps of f (fbox) and g (posbox) over p.xmin, p.ymin, p.ntx * 8 by
// p.nty * 16 subset top-left positions (reads p.ref, p.def, W, H, pitch, S).
cudaError_t launch_boxmaps(const SearchTcParams& p, cudaStream_t st);
// Shared bytes per warp of the swarm search (window, evaluation table, the
// generation's box sums); 0 if the geometry is not supported.
size_t pso_warp_smem(int S, int R, int particles, int* wp);
cudaError_t launch_pso(const PsoParams& p, cudaStream_t st);

// Persistent multi-pair launchers.  jobs / offsets are device arrays; the
// POIs of job k are items [offsets[k], offsets[k+1]); counter starts at 0.
cudaError_t launch_search_batch(int tw, const SearchParams* jobs, const int64_t* offsets,
                                int njobs, unsigned long long* counter, size_t smem, int grid,
                                cudaStream_t st);
int search_batch_occupancy(int tw, size_t smem);
size_t search_smem_bytes(int S, int R);
cudaError_t launch_subpixel_batch(const SubpixelParams* jobs, const int64_t* offsets, int njobs,
                                  int nmax, int method, int solve_fp64, int wpc,
                                  unsigned long long* counter, int grid, cudaStream_t st);
cudaError_t launch_search(const SearchParams& p, const CUtensorMap* tm_ref,
                          const CUtensorMap* tm_def, cudaStream_t st);
// IC-GN with the second-order shape function; p12 receives [n_pois][12]
cudaError_t launch_subpixel2(const SubpixelParams& p, int solve_fp64, float* p12,
                             cudaStream_t st);
// bilinear: 1 for the bilinear interpolation of Eq. 5, 0 for bicubic (Keys)
cudaError_t launch_subpixel(const SubpixelParams& p, int method, int solve_fp64,
                            cudaStream_t st, int bilinear = 0);

// Size of the byte box that TMA stages for a subset / search window.
__host__ __device__ inline int tma_box_width(int span) { return ((span + 15 + 15) / 16) * 16; }

}  // namespace dic

namespace dic {
// State of a bound batch (dic_set_pairs).
struct BatchPair {
  dic_pair_desc d;
  int S, M, R, step, nx, ny, tw;
  int64_t n, off;
  size_t px_off;
  bool fp32_ok = false;     // the FP32 search window fits shared memory
  bool tc_ok = false;       // the tensor-core search geometry exists
  SearchTcParams tc{};      // its geometry (scratch pointers filled per graph)
};
struct BatchClass {  // pairs sharing the search template width
  int tw;
  std::vector<int> pairs;
  size_t smem;
  SearchParams* d_jobs = nullptr;
  int64_t* d_offsets = nullptr;
};
struct BatchState {
  std::vector<BatchPair> pairs;
  std::vector<BatchClass> classes;
  int64_t total = 0;
  int nmax = 0;
  size_t px_total = 0;
  float* gimg = nullptr;
  float2* grad = nullptr;
  uint2* gq = nullptr;
  SubpixelParams* d_pjobs = nullptr;
  int64_t* d_offsets = nullptr;
  unsigned long long* d_counters = nullptr;
  cudaStream_t cap = nullptr;
  cudaStream_t side = nullptr;     // sub-pixel launches overlapped with searches
  std::vector<cudaEvent_t> evs;    // fork / per-pair / join events of the capture
  std::vector<SubpixelParams> pj;  // host copy of the per-pair sub-pixel jobs
  cudaGraphExec_t exec = nullptr;
  dic_batch_out last_out{};
  int last_method = -1, last_wpc = 0, last_mult = 0, last_bits = 0, last_form = -1;
  // tensor-core search scratch, shared by the pairs' searches (they run one
  // after another on the graph's stream), sized for the largest pair
  uint16_t* tc_phase = nullptr;
  int2* tc_fbox = nullptr;
  int2* tc_posbox = nullptr;
  SlotCand* tc_slots = nullptr;
  // sub-pixel launch shape: warps per CTA x persistent grid multiple, or
  // wpc = grid_mult = 0 for per-pair launches on the side stream, each
  // overlapping the next pair's tensor-core search
  int wpc = 4, grid_mult = 1;
};
}  // namespace dic

namespace dic {
// State of a consecutive-frame stream (dic_stream_push): a ring of three
// frame slots, each holding the frame (copied, 16-byte pitch) and its
// precompute (gradient field for its turn as reference; float copy and tap
// quads for its turn as target); the sub-pixel launches run on a second
// stream, ordered by events.
struct StreamState {
  int W = 0, H = 0, pitch = 0;  // pitch of the ring's frames (bytes)
  long long frames = 0;         // frames pushed since the last reset
  uint8_t* frame[3] = {};
  float2* grad[3] = {};
  float* gimg[3] = {};
  uint2* gq[3] = {};
  size_t px = 0;                // pixels per slot allocated
  cudaStream_t side = nullptr;
  cudaEvent_t searched = nullptr;    // a pair's integer search is done
  cudaEvent_t refined[3] = {};       // pair k's sub-pixel work is done (k % 3)
  bool pending = false;              // a pair's sub-pixel work not yet joined
};
}  // namespace dic

struct dic_s {
  int subset = 0, M = 0, step = 0, R = 0, shape_order = 1, max_iter = 0;
  float tol = 0.f;
  int form = DIC_FORM_PLAIN_FP32;
  int solve_bits = 32;
  int interp = DIC_INTERP_BICUBIC;
  cudaStream_t stream = nullptr;
  // The pair's precompute runs on pre_side, forked from stream, so that it
  // overlaps the integer search; the kernels that read its output wait on
  // pre_done (pre_pending: recorded for the current pair)
  cudaStream_t pre_side = nullptr;
  cudaEvent_t pre_fork = nullptr, pre_done = nullptr;
  bool pre_pending = false;
  // the tensor-core search's phase images and bank run on search_side
  // beside its box-sum maps
  cudaStream_t search_side = nullptr;
  cudaEvent_t search_fork = nullptr, search_join = nullptr;

  bool have_pair = false;
  const uint8_t* ref = nullptr;
  const uint8_t* def = nullptr;
  const float* ref_f32 = nullptr;  // set instead of ref/def for float pairs
  const float* def_f32 = nullptr;
  dic::PairGeom g;

  float* gimg = nullptr;
  float2* grad = nullptr;
  uint2* gq = nullptr;    // tap quads of an 8-bit deformed image
  size_t scratch_px = 0;  // capacity in pixels
  unsigned int* err_flag = nullptr;

  bool tma_ok = false;
  CUtensorMap tm_ref{}, tm_def{};

  dic::BatchState* batch = nullptr;
  dic::StreamState* seq = nullptr;

  // scratch of the tensor-core search form
  uint16_t* tc_phase = nullptr;
  int2* tc_fbox = nullptr;
  dic::SlotCand* tc_slots = nullptr;
  int2* tc_posbox = nullptr;
  size_t tc_phase_elems = 0, tc_pois = 0, tc_slot_elems = 0, tc_posbox_elems = 0;

  std::string last_error;
};
