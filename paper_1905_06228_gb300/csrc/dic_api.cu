// dic_api.cu -- the C ABI declared in include/dic.h: argument checking, the
// handle's device scratch, TMA descriptors and kernel launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>

#include "dic_internal.cuh"

namespace dic {
size_t search_smem_bytes(int S, int R);
}

namespace {

constexpr int kVersion = 10000;  // 1.0.0

dic_status fail(dic_t h, dic_status st, const char* fmt, ...) {
  if (h) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    h->last_error = buf;
  }
  return st;
}

dic_status cuda_fail(dic_t h, cudaError_t e, const char* what) {
  return fail(h, DIC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D uint8 tensor map over an image with a box of (box_w bytes, box_h rows).
bool encode_u8(CUtensorMap* tm, const uint8_t* base, int W, int H, int pitch, int box_w,
               int box_h) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
  cuuint64_t strides[1] = {(cuuint64_t)pitch};
  cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Tensor maps of the tensor-core search (BF16).
//  A: 3-D over the eight phase images [8][phh][phw]: (column, phase r,
//     image row), box (TWK, 8, tile rows): image row = 8-row group, r = row,
//     swizzle of the row width (2*TWK bytes);
//  B: 4-D over the template bank [bank_rows][nx][64]: (tap, POI column, POI
//     row, operand row j), box (64, ncols, nrows, 1): one stage of a tile's
//     POI block, 128-byte swizzle.  Bank row of (kr, j): kr*step + SUB*j by
//     image row (overlapping strides), kr*sj + j stacked.
bool encode_bank_map(CUtensorMap* tmb, void* bank, int nx, int ny, int sj, cuuint64_t kr_rows,
                     cuuint64_t j_rows, int ncols, int nrows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t row = (cuuint64_t)nx * 128;  // bytes per bank row
  cuuint64_t dims[4] = {64, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)sj};
  cuuint64_t str[3] = {128, row * kr_rows, row * j_rows};
  cuuint32_t box[4] = {64, (cuuint32_t)ncols, (cuuint32_t)nrows, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(tmb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, bank, dims, str, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_tc(CUtensorMap* tma, CUtensorMap* tmb, const dic::SearchTcParams& t) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const CUtensorMapSwizzle sw = t.twk == 64   ? CU_TENSOR_MAP_SWIZZLE_128B
                                : t.twk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                              : CU_TENSOR_MAP_SWIZZLE_32B;
  {
    cuuint64_t dims[3] = {(cuuint64_t)t.phw, 8, (cuuint64_t)t.phh};
    cuuint64_t str[2] = {(cuuint64_t)t.phh * t.phw * 2, (cuuint64_t)t.phw * 2};
    cuuint32_t box[3] = {(cuuint32_t)t.twk, 8, (cuuint32_t)t.arows};
    cuuint32_t es[3] = {1, 1, 1};
    if (fn(tma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, t.gph, dims, str, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  const cuuint64_t kr_rows = t.bank_overlap ? (cuuint64_t)t.step : (cuuint64_t)t.sj;
  const cuuint64_t j_rows = t.bank_overlap ? (cuuint64_t)t.sub : 1;
  return encode_bank_map(tmb, t.bank, t.nx, t.ny, t.sj, kr_rows, j_rows, t.ncols_max,
                         t.nrows_max);
}

// Whether the tensor map encoder takes the bank by image row (strides of
// the POI-row and operand-row dimensions that overlap).  Asked once, with a
// map that is never used; no memory is accessed.
bool bank_overlap_ok() {
  static int ok = -1;
  if (ok < 0) {
    alignas(128) static unsigned char probe[128];
    CUtensorMap tm;
    ok = encode_bank_map(&tm, probe, 20, 20, 16, 5, 2, 10, 12) ? 1 : 0;
  }
  return ok == 1;
}

// Geometry of the tensor-core search, with the bank's row order the
// encoder accepts.
bool tc_geometry(int W, int H, int S, int step, int R, int nx, int ny, dic::SearchTcParams* t) {
  if (!dic::search_tc_geometry(W, H, S, step, R, nx, ny, t)) return false;
  if (t->bank_overlap && !bank_overlap_ok()) return dic::search_tc_bank_order(t, 0);
  return true;
}

void grid_of(int W, int H, int S, int step, int R, int* nx, int* ny) {
  const int B = S / 2 + R + 2;
  const int ax = W - 1 - 2 * B, ay = H - 1 - 2 * B;
  *nx = ax >= 0 ? ax / step + 1 : 0;
  *ny = ay >= 0 ? ay / step + 1 : 0;
}

}  // namespace

extern "C" {

int dic_version(void) { return kVersion; }

dic_status dic_create(dic_t* out, int subset_size, int grid_step, int search_radius,
                      int shape_order, float conv_tol, int max_iter) {
  if (!out) return DIC_ERR_ARG;
  *out = nullptr;
  if (subset_size < 3 || subset_size > dic::kMaxSubset || (subset_size & 1) == 0 ||
      grid_step < 1 || search_radius < 0 || search_radius > 1000 || !(conv_tol > 0.f) ||
      max_iter < 1)
    return DIC_ERR_ARG;
  if (shape_order != 1 && shape_order != 2) return DIC_ERR_UNSUPPORTED;
  dic_t h = new (std::nothrow) dic_s;
  if (!h) return DIC_ERR_OOM;
  h->subset = subset_size;
  h->M = subset_size / 2;
  h->step = grid_step;
  h->R = search_radius;
  h->shape_order = shape_order;
  h->tol = conv_tol;
  h->max_iter = max_iter;
  *out = h;
  return DIC_OK;
}

}  // extern "C"

namespace {

void free_batch(dic::BatchState* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->gimg) cudaFree(b->gimg);
  if (b->grad) cudaFree(b->grad);
  if (b->gq) cudaFree(b->gq);
  if (b->d_pjobs) cudaFree(b->d_pjobs);
  if (b->d_offsets) cudaFree(b->d_offsets);
  if (b->d_counters) cudaFree(b->d_counters);
  if (b->tc_phase) cudaFree(b->tc_phase);
  if (b->tc_fbox) cudaFree(b->tc_fbox);
  if (b->tc_posbox) cudaFree(b->tc_posbox);
  if (b->tc_slots) cudaFree(b->tc_slots);
  for (auto& c : b->classes) {
    if (c.d_jobs) cudaFree(c.d_jobs);
    if (c.d_offsets) cudaFree(c.d_offsets);
  }
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->side) cudaStreamDestroy(b->side);
  for (cudaEvent_t ev : b->evs) cudaEventDestroy(ev);
  delete b;
}

void free_stream(dic::StreamState* q) {
  if (!q) return;
  if (q->side) cudaStreamSynchronize(q->side);
  for (int k = 0; k < 3; ++k) {
    if (q->frame[k]) cudaFree(q->frame[k]);
    if (q->grad[k]) cudaFree(q->grad[k]);
    if (q->gimg[k]) cudaFree(q->gimg[k]);
    if (q->gq[k]) cudaFree(q->gq[k]);
    if (q->refined[k]) cudaEventDestroy(q->refined[k]);
  }
  if (q->searched) cudaEventDestroy(q->searched);
  if (q->side) cudaStreamDestroy(q->side);
  delete q;
}

}  // namespace

extern "C" {

void dic_destroy(dic_t h) {
  if (!h) return;
  free_batch(h->batch);
  free_stream(h->seq);
  if (h->gimg) cudaFree(h->gimg);
  if (h->grad) cudaFree(h->grad);
  if (h->gq) cudaFree(h->gq);
  if (h->err_flag) cudaFree(h->err_flag);
  if (h->tc_phase) cudaFree(h->tc_phase);
  if (h->tc_fbox) cudaFree(h->tc_fbox);
  if (h->tc_slots) cudaFree(h->tc_slots);
  if (h->tc_posbox) cudaFree(h->tc_posbox);
  if (h->pre_side) cudaStreamDestroy(h->pre_side);
  if (h->pre_fork) cudaEventDestroy(h->pre_fork);
  if (h->pre_done) cudaEventDestroy(h->pre_done);
  if (h->search_side) cudaStreamDestroy(h->search_side);
  if (h->search_fork) cudaEventDestroy(h->search_fork);
  if (h->search_join) cudaEventDestroy(h->search_join);
  delete h;
}

const char* dic_last_error(dic_t h) { return h ? h->last_error.c_str() : "null handle"; }

dic_status dic_check(dic_t h) {
  if (!h) return DIC_ERR_ARG;
  if (!h->err_flag) return DIC_OK;  // nothing launched yet
  unsigned int flag = 0;
  cudaError_t e = h->pre_pending ? cudaStreamWaitEvent(h->stream, h->pre_done, 0) : cudaSuccess;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&flag, h->err_flag, sizeof flag, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "error-flag read");
  if (flag == 0) return DIC_OK;
  e = cudaMemsetAsync(h->err_flag, 0, sizeof(unsigned int), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "error-flag reset");
  return fail(h, DIC_ERR_TIMEOUT,
              "a bounded device wait gave up (flag 0x%x: 1 FP32 search staging, 2 tensor-core "
              "tile pipeline, with 0x10 A free, 0x20 B stage free, 0x40 accumulator read, "
              "0x80 A landed, 0x100 B landed, 0x200 accumulator complete, 0x400 last MMAs); "
              "the affected integer-search results are incomplete",
              flag);
}

dic_status dic_set_stream(dic_t h, void* s) {
  if (!h) return DIC_ERR_ARG;
  h->stream = static_cast<cudaStream_t>(s);
  return DIC_OK;
}

dic_status dic_set_form(dic_t h, dic_form form) {
  if (!h) return DIC_ERR_ARG;
  if (form == DIC_FORM_PLAIN_FP32) {
    h->form = form;
    return DIC_OK;
  }
  if (form == DIC_FORM_BF16TC) {
    h->form = form;
    return DIC_OK;
  }
  return fail(h, DIC_ERR_ARG, "unknown form %d", (int)form);
}

dic_status dic_set_solve_precision(dic_t h, int bits) {
  if (!h) return DIC_ERR_ARG;
  if (bits != 32 && bits != 64) return fail(h, DIC_ERR_ARG, "solve precision must be 32 or 64");
  h->solve_bits = bits;
  return DIC_OK;
}

dic_status dic_set_interpolation(dic_t h, dic_interp interp) {
  if (!h) return DIC_ERR_ARG;
  if (interp != DIC_INTERP_BICUBIC && interp != DIC_INTERP_BILINEAR)
    return fail(h, DIC_ERR_ARG, "unknown interpolation %d", (int)interp);
  h->interp = interp;
  return DIC_OK;
}

}  // extern "C"

namespace {

// Common part of dic_set_pair / dic_set_pair_f32: geometry, scratch, and the
// precompute launch.
// Stream for the pair's precompute: a side stream that first waits for all
// earlier work on the handle's stream (which may still read the previous
// pair's gradient and float image), so that the precompute overlaps the
// integer search.  While the handle's stream is being captured into a graph
// (or if the side stream cannot be made) it is the handle's stream itself.
cudaStream_t pre_stream(dic_t h) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return h->stream;
  }
  if (!h->pre_side) {
    if (cudaStreamCreateWithFlags(&h->pre_side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->pre_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->pre_done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (h->pre_side) cudaStreamDestroy(h->pre_side);
      if (h->pre_fork) cudaEventDestroy(h->pre_fork);
      if (h->pre_done) cudaEventDestroy(h->pre_done);
      h->pre_side = nullptr;
      h->pre_fork = h->pre_done = nullptr;
      return h->stream;
    }
  }
  if (cudaEventRecord(h->pre_fork, h->stream) != cudaSuccess ||
      cudaStreamWaitEvent(h->pre_side, h->pre_fork, 0) != cudaSuccess) {
    cudaGetLastError();
    return h->stream;
  }
  return h->pre_side;
}

// Side stream of the tensor-core search's set-up kernels (nullptr while st
// is being captured into a graph, or if it cannot be made).
cudaStream_t search_side(dic_t h, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return nullptr;
  }
  if (!h->search_side) {
    if (cudaStreamCreateWithFlags(&h->search_side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->search_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->search_join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (h->search_side) cudaStreamDestroy(h->search_side);
      if (h->search_fork) cudaEventDestroy(h->search_fork);
      if (h->search_join) cudaEventDestroy(h->search_join);
      h->search_side = nullptr;
      h->search_fork = h->search_join = nullptr;
    }
  }
  return h->search_side;
}

// The handle's stream waits for the current pair's precompute.
cudaError_t pre_join(dic_t h) {
  return h->pre_pending ? cudaStreamWaitEvent(h->stream, h->pre_done, 0) : cudaSuccess;
}

dic_status bind_pair(dic_t h, const void* ref, const void* def, bool f32, int width, int height,
                     int pitch) {
  if (!h) return DIC_ERR_ARG;
  h->have_pair = false;
  if (!ref || !def) return fail(h, DIC_ERR_ARG, "null image pointer");
  if (width < 4 || height < 4 || pitch < width)
    return fail(h, DIC_ERR_ARG, "bad image size %dx%d pitch %d", width, height, pitch);
  int nx, ny;
  grid_of(width, height, h->subset, h->step, h->R, &nx, &ny);
  const size_t px = (size_t)width * height;
  if (px > h->scratch_px) {
    if (h->gimg) cudaFree(h->gimg);
    if (h->grad) cudaFree(h->grad);
    if (h->gq) cudaFree(h->gq);
    h->gimg = nullptr;
    h->grad = nullptr;
    h->gq = nullptr;
    h->scratch_px = 0;
    if (cudaMalloc(&h->gimg, px * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&h->grad, px * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&h->gq, px * sizeof(uint2)) != cudaSuccess) {
      cudaGetLastError();
      if (h->gimg) cudaFree(h->gimg);
      if (h->grad) cudaFree(h->grad);
      h->gimg = nullptr;
      h->grad = nullptr;
      return fail(h, DIC_ERR_OOM, "cannot allocate %zu bytes of scratch", px * 20);
    }
    h->scratch_px = px;
  }
  if (!h->err_flag) {
    if (cudaMalloc(&h->err_flag, sizeof(unsigned int)) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, DIC_ERR_OOM, "cannot allocate error flag");
    }
    cudaMemsetAsync(h->err_flag, 0, sizeof(unsigned int), h->stream);
  }
  h->g.W = width;
  h->g.H = height;
  h->g.pitch = pitch;
  h->g.nx = nx;
  h->g.ny = ny;
  h->g.n_pois = (int64_t)nx * ny;
  cudaError_t e;
  h->pre_pending = false;
  const cudaStream_t pst = pre_stream(h);
  if (f32) {
    h->ref = h->def = nullptr;
    h->ref_f32 = static_cast<const float*>(ref);
    h->def_f32 = static_cast<const float*>(def);
    h->tma_ok = false;
    e = dic::launch_precompute_f32(h->ref_f32, h->def_f32, width, height, pitch, h->grad, h->gimg,
                                   pst);
  } else {
    h->ref_f32 = h->def_f32 = nullptr;
    h->ref = static_cast<const uint8_t*>(ref);
    h->def = static_cast<const uint8_t*>(def);
    // TMA staging needs 16-byte aligned bases and pitch, and boxes <= 256.
    const int span = h->subset + 2 * h->R;
    const int bwg = dic::tma_box_width(span), bwf = dic::tma_box_width(h->subset);
    h->tma_ok = ((uintptr_t)ref % 16 == 0) && ((uintptr_t)def % 16 == 0) && (pitch % 16 == 0) &&
                bwg <= 256 && span <= 256 &&
                encode_u8(&h->tm_def, h->def, width, height, pitch, bwg, span) &&
                encode_u8(&h->tm_ref, h->ref, width, height, pitch, bwf, h->subset);
    e = dic::launch_precompute(h->ref, h->def, width, height, pitch, h->grad, h->gimg, h->gq,
                               pst);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "precompute launch");
  if (pst != h->stream) {
    e = cudaEventRecord(h->pre_done, pst);
    if (e != cudaSuccess) return cuda_fail(h, e, "precompute event");
    h->pre_pending = true;
  }
  h->have_pair = true;
  return DIC_OK;
}

dic_status run_adjoint(dic_t h, const float* p6, float* loss_poi, float* loss_total, int backward,
                       const float* grad_loss, float scale, float* dL_ddef, float* dL_dp) {
  if (!h) return DIC_ERR_ARG;
  if (!h->have_pair) return fail(h, DIC_ERR_STATE, "no image pair set");
  if (h->g.n_pois > 0 && !p6) return fail(h, DIC_ERR_ARG, "null shape array");
  if (backward && !dL_ddef) return fail(h, DIC_ERR_ARG, "null image gradient");
  if (loss_total) cudaMemsetAsync(loss_total, 0, sizeof(float), h->stream);
  if (backward)
    cudaMemsetAsync(dL_ddef, 0, sizeof(float) * (size_t)h->g.W * h->g.H, h->stream);
  if (h->g.n_pois == 0) return DIC_OK;
  if (cudaError_t je = pre_join(h); je != cudaSuccess) return cuda_fail(h, je, "precompute join");
  dic::AdjointParams p;
  p.ref = h->ref;
  p.ref_f32 = h->ref_f32;
  p.gimg = h->gimg;
  p.W = h->g.W;
  p.H = h->g.H;
  p.pitch = h->g.pitch;
  p.S = h->subset;
  p.M = h->M;
  p.R = h->R;
  p.step = h->step;
  p.nx = h->g.nx;
  p.n_pois = h->g.n_pois;
  p.p6 = p6;
  p.loss_poi = loss_poi;
  p.loss_total = loss_total;
  p.backward = backward;
  p.grad_loss = grad_loss;
  p.scale = scale;
  p.dL_ddef = dL_ddef;
  p.dL_dp = dL_dp;
  cudaError_t e = dic::launch_adjoint(p, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint launch");
  return DIC_OK;
}

}  // namespace

extern "C" {

dic_status dic_set_pair(dic_t h, const uint8_t* ref, const uint8_t* def, int width, int height,
                        int pitch) {
  return bind_pair(h, ref, def, false, width, height, pitch);
}

dic_status dic_set_pair_f32(dic_t h, const float* ref, const float* def, int width, int height,
                            int pitch_elems) {
  if (h && (((uintptr_t)ref | (uintptr_t)def) % 4 != 0))
    return fail(h, DIC_ERR_ARG, "float images must be 4-byte aligned");
  return bind_pair(h, ref, def, true, width, height, pitch_elems);
}

dic_status dic_znssd(dic_t h, const float* p6, float* loss_per_poi, float* loss_total) {
  return run_adjoint(h, p6, loss_per_poi, loss_total, 0, nullptr, 0.f, nullptr, nullptr);
}

dic_status dic_backward(dic_t h, const float* p6, const float* grad_loss, float scale,
                        float* dL_ddef, float* dL_dp) {
  return run_adjoint(h, p6, nullptr, nullptr, 1, grad_loss, scale, dL_ddef, dL_dp);
}

dic_status dic_num_pois(dic_t h, int* n_pois, int* nx, int* ny) {
  if (!h) return DIC_ERR_ARG;
  if (!h->have_pair && !(h->seq && h->seq->frames > 0))
    return fail(h, DIC_ERR_STATE, "no image pair set");
  if (n_pois) *n_pois = (int)h->g.n_pois;
  if (nx) *nx = h->g.nx;
  if (ny) *ny = h->g.ny;
  return DIC_OK;
}

dic_status dic_pso_search(dic_t h, int modified, int particles, int generations, double c1,
                          double c2, double vinit, int stop_num, int stop_den,
                          const double* uniforms, int32_t* u0, int32_t* v0, float* zncc0,
                          uint8_t* status, int32_t* gens, int32_t* evals) {
  if (!h) return DIC_ERR_ARG;
  if (!h->have_pair) return fail(h, DIC_ERR_STATE, "no image pair set");
  if (h->ref_f32)
    return fail(h, DIC_ERR_UNSUPPORTED, "swarm search needs an 8-bit pair (exact sums)");
  if ((modified != 0 && modified != 1) || particles < 1 || particles > 64 || generations < 1 ||
      generations > 1000 || stop_num < 0 || stop_num > (1 << 20) || stop_den < 1 ||
      stop_den > (1 << 20) || !std::isfinite(c1) || !std::isfinite(c2) ||
      !std::isfinite(vinit))
    return fail(h, DIC_ERR_ARG,
                "swarm arguments: modified 0/1, particles 1..64, generations 1..1000, "
                "0 <= stop_num <= 2^20, 1 <= stop_den <= 2^20, finite coefficients");
  if (h->g.n_pois == 0) return DIC_OK;
  if (!uniforms || !u0 || !v0 || !zncc0 || !status || !gens || !evals)
    return fail(h, DIC_ERR_ARG, "null pointer");
  int wp = 0;
  const size_t wsm = dic::pso_warp_smem(h->subset, h->R, particles, &wp);
  if (wsm == 0)
    return fail(h, DIC_ERR_UNSUPPORTED, "swarm search: window and table exceed shared memory");
  // box-sum maps of f and g over every subset top-left a window reaches
  const int B = h->M + h->R + 2;
  dic::SearchTcParams t{};
  t.ref = h->ref;
  t.def = h->def;
  t.W = h->g.W;
  t.H = h->g.H;
  t.pitch = h->g.pitch;
  t.S = h->subset;
  t.xmin = B - h->M - h->R;
  t.ymin = B - h->M - h->R;
  const int spanx = (h->g.nx - 1) * h->step + 2 * h->R + 1;
  const int spany = (h->g.ny - 1) * h->step + 2 * h->R + 1;
  t.ntx = (spanx + 7) / 8;
  t.nty = (spany + 15) / 16;
  const size_t pbe = dic::search_tc_posbox_elems(t);
  if (pbe > h->tc_posbox_elems) {
    if (h->tc_posbox) cudaFree(h->tc_posbox);
    if (h->tc_fbox) cudaFree(h->tc_fbox);
    h->tc_posbox = nullptr;
    h->tc_fbox = nullptr;
    h->tc_posbox_elems = 0;
    if (cudaMalloc(&h->tc_posbox, pbe * sizeof(int2)) != cudaSuccess ||
        cudaMalloc(&h->tc_fbox, pbe * sizeof(int2)) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, DIC_ERR_OOM, "cannot allocate swarm search scratch");
    }
    h->tc_posbox_elems = pbe;
  }
  t.posbox = h->tc_posbox;
  t.fbox = h->tc_fbox;
  cudaError_t e = dic::launch_boxmaps(t, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "box-sum map launch");
  dic::PsoParams p{};
  p.ref = h->ref;
  p.def = h->def;
  p.W = h->g.W;
  p.H = h->g.H;
  p.pitch = h->g.pitch;
  p.S = h->subset;
  p.M = h->M;
  p.R = h->R;
  p.step = h->step;
  p.nx = h->g.nx;
  p.n_pois = h->g.n_pois;
  p.modified = modified;
  p.particles = particles;
  p.gmax = generations;
  p.c1 = c1;
  p.c2 = c2;
  p.vinit = vinit;
  p.stop_num = stop_num;
  p.stop_den = stop_den;
  p.rand = uniforms;
  p.posbox = t.posbox;
  p.fbox = t.fbox;
  p.xmin = t.xmin;
  p.ymin = t.ymin;
  p.pw = t.ntx * 8;
  p.wp = wp;
  p.warp_smem = wsm;
  p.warps = (int)std::min<size_t>(4, (227 * 1024) / wsm);
  p.u0 = u0;
  p.v0 = v0;
  p.zncc0 = zncc0;
  p.status = status;
  p.gens = gens;
  p.evals = evals;
  e = dic::launch_pso(p, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "swarm search launch");
  e = pre_join(h);  // the pair's precompute ran beside the search
  return e == cudaSuccess ? DIC_OK : cuda_fail(h, e, "precompute join");
}

}  // extern "C"

namespace {

// Integer search of the 8-bit images (ref, def) with the handle's geometry
// (h->g), form and search scratch, on stream st; tma_ok / tm_ref / tm_def
// describe TMA staging of those images for the FP32 form.
dic_status search_images(dic_t h, const uint8_t* ref, const uint8_t* def, bool tma_ok,
                         const CUtensorMap* tm_ref, const CUtensorMap* tm_def, int32_t* u0,
                         int32_t* v0, float* zncc0, uint8_t* status, cudaStream_t st) {
  if (h->form == DIC_FORM_BF16TC) {
    dic::SearchTcParams t{};
    if (!tc_geometry(h->g.W, h->g.H, h->subset, h->step, h->R, h->g.nx, h->g.ny,
                                 &t) ||
        dic::search_tc_smem(t) > 227 * 1024)
      return fail(h, DIC_ERR_UNSUPPORTED,
                  "tensor-core search: one row of a tile's POI block exceeds N = 256 (grid "
                  "step too small for this radius), or the geometry exceeds shared memory");
    const size_t phase = dic::search_tc_phase_elems(t);
    const size_t slots = (size_t)h->g.n_pois * t.nslots;
    if (phase > h->tc_phase_elems || (size_t)h->g.n_pois > h->tc_pois ||
        slots > h->tc_slot_elems) {
      if (h->tc_phase) cudaFree(h->tc_phase);
      if (h->tc_slots) cudaFree(h->tc_slots);
      h->tc_phase = nullptr;
      h->tc_slots = nullptr;
      h->tc_phase_elems = h->tc_pois = h->tc_slot_elems = 0;
      if (cudaMalloc(&h->tc_phase, phase * sizeof(uint16_t)) != cudaSuccess ||
          cudaMalloc(&h->tc_slots, slots * sizeof(dic::SlotCand)) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, DIC_ERR_OOM, "cannot allocate tensor-core search scratch");
      }
      h->tc_phase_elems = phase;
      h->tc_pois = (size_t)h->g.n_pois;
      h->tc_slot_elems = slots;
    }
    t.ref = ref;
    t.def = def;
    t.W = h->g.W;
    t.H = h->g.H;
    t.pitch = h->g.pitch;
    t.n_pois = h->g.n_pois;
    const size_t pbe = dic::search_tc_posbox_elems(t);
    if (pbe > h->tc_posbox_elems) {
      if (h->tc_posbox) cudaFree(h->tc_posbox);
      if (h->tc_fbox) cudaFree(h->tc_fbox);
      h->tc_posbox = nullptr;
      h->tc_fbox = nullptr;
      h->tc_posbox_elems = 0;
      if (cudaMalloc(&h->tc_posbox, pbe * sizeof(int2)) != cudaSuccess ||
          cudaMalloc(&h->tc_fbox, pbe * sizeof(int2)) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, DIC_ERR_OOM, "cannot allocate tensor-core search scratch");
      }
      h->tc_posbox_elems = pbe;
    }
    t.gph = h->tc_phase;
    t.bank = h->tc_phase + dic::search_tc_gph_elems(t);
    t.fbox = h->tc_fbox;
    t.slots = h->tc_slots;
    t.posbox = h->tc_posbox;
    t.u0 = u0;
    t.v0 = v0;
    t.zncc0 = zncc0;
    t.status = status;
    t.err_flag = h->err_flag;
    CUtensorMap tma, tmb;
    if (!encode_tc(&tma, &tmb, t))
      return fail(h, DIC_ERR_UNSUPPORTED, "tensor-core search: tensor map encoding failed");
    const cudaStream_t side = search_side(h, st);
    cudaError_t e = dic::launch_search_tc(t, &tma, &tmb, st, side, h->search_fork, h->search_join);
    if (e != cudaSuccess) return cuda_fail(h, e, "tensor-core search launch");
    return DIC_OK;
  }
  if (dic::search_smem_bytes(h->subset, h->R) > 227 * 1024)
    return fail(h, DIC_ERR_UNSUPPORTED, "search window too large for shared memory");
  dic::SearchParams p;
  p.ref = ref;
  p.def = def;
  p.W = h->g.W;
  p.H = h->g.H;
  p.pitch = h->g.pitch;
  p.S = h->subset;
  p.M = h->M;
  p.R = h->R;
  p.step = h->step;
  p.nx = h->g.nx;
  p.n_pois = h->g.n_pois;
  p.use_tma = tma_ok ? 1 : 0;
  p.u0 = u0;
  p.v0 = v0;
  p.zncc0 = zncc0;
  p.status = status;
  p.err_flag = h->err_flag;
  cudaError_t e = dic::launch_search(p, tm_ref, tm_def, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "integer search launch");
  return DIC_OK;
}

// Sub-pixel refinement with the handle's geometry and options: reference
// image ref (8-bit) with its gradient field grad, deformed image as float
// gimg and tap quads gq, on stream st.
dic_status subpixel_images(dic_t h, dic_method method, const uint8_t* ref, const float2* grad,
                           const float* gimg, const uint2* gq, const int32_t* u0,
                           const int32_t* v0, const uint8_t* status0, float* u, float* v,
                           float* ux, float* uy, float* vx, float* vy, float* zncc,
                           int32_t* iters, uint8_t* status, cudaStream_t st) {
  dic::SubpixelParams p;
  p.ref = ref;
  p.grad = grad;
  p.gimg = gimg;
  p.gq = gq;
  p.W = h->g.W;
  p.H = h->g.H;
  p.pitch = h->g.pitch;
  p.S = h->subset;
  p.M = h->M;
  p.R = h->R;
  p.step = h->step;
  p.nx = h->g.nx;
  p.n_pois = h->g.n_pois;
  p.max_iter = h->max_iter;
  p.tol = h->tol;
  p.u0 = u0;
  p.v0 = v0;
  p.st0 = status0;
  p.u = u;
  p.v = v;
  p.ux = ux;
  p.uy = uy;
  p.vx = vx;
  p.vy = vy;
  p.zncc = zncc;
  p.iters = iters;
  p.status = status;
  cudaError_t e = dic::launch_subpixel(p, (int)method, h->solve_bits == 64, st,
                                       h->interp == DIC_INTERP_BILINEAR);
  if (e != cudaSuccess) return cuda_fail(h, e, "subpixel launch");
  return DIC_OK;
}

}  // namespace

extern "C" {

dic_status dic_integer_search(dic_t h, int32_t* u0, int32_t* v0, float* zncc0,
                              uint8_t* status) {
  if (!h) return DIC_ERR_ARG;
  if (!h->have_pair) return fail(h, DIC_ERR_STATE, "no image pair set");
  if (h->ref_f32)
    return fail(h, DIC_ERR_UNSUPPORTED, "integer search needs an 8-bit pair (exact sums)");
  if (h->g.n_pois == 0) return DIC_OK;
  if (!u0 || !v0 || !zncc0 || !status) return fail(h, DIC_ERR_ARG, "null output pointer");
  const dic_status st = search_images(h, h->ref, h->def, h->tma_ok, &h->tm_ref, &h->tm_def, u0,
                                      v0, zncc0, status, h->stream);
  if (st != DIC_OK) return st;
  // the pair's precompute ran beside the search; later work on the stream
  // comes after both
  const cudaError_t e = pre_join(h);
  return e == cudaSuccess ? DIC_OK : cuda_fail(h, e, "precompute join");
}



dic_status dic_subpixel2(dic_t h, dic_method method, const int32_t* u0, const int32_t* v0,
                         const uint8_t* status0, float* p12, float* zncc, int32_t* iters,
                         uint8_t* status) {
  if (!h) return DIC_ERR_ARG;
  if (method != DIC_ICGN && method != DIC_FANR) return fail(h, DIC_ERR_ARG, "unknown method");
  if (h->shape_order != 2)
    return fail(h, DIC_ERR_STATE, "second-order refinement needs a handle of shape order 2");
  if (method != DIC_ICGN)
    return fail(h, DIC_ERR_UNSUPPORTED, "second-order shape: IC-GN only on the device");
  if (h->interp != DIC_INTERP_BICUBIC)
    return fail(h, DIC_ERR_UNSUPPORTED, "second-order shape: bicubic interpolation only");
  if (!h->have_pair) return fail(h, DIC_ERR_STATE, "no image pair set");
  if (h->g.n_pois == 0) return DIC_OK;
  if (!u0 || !v0 || !status0 || !p12 || !zncc || !iters || !status)
    return fail(h, DIC_ERR_ARG, "null pointer");
  dic::SubpixelParams p;
  p.ref = h->ref;
  p.ref_f32 = h->ref_f32;
  p.grad = h->grad;
  p.gimg = h->gimg;
  p.gq = h->ref ? h->gq : nullptr;
  p.W = h->g.W;
  p.H = h->g.H;
  p.pitch = h->g.pitch;
  p.S = h->subset;
  p.M = h->M;
  p.R = h->R;
  p.step = h->step;
  p.nx = h->g.nx;
  p.n_pois = h->g.n_pois;
  p.max_iter = h->max_iter;
  p.tol = h->tol;
  p.u0 = u0;
  p.v0 = v0;
  p.st0 = status0;
  p.zncc = zncc;
  p.iters = iters;
  p.status = status;
  cudaError_t e = pre_join(h);
  if (e != cudaSuccess) return cuda_fail(h, e, "precompute join");
  e = dic::launch_subpixel2(p, h->solve_bits == 64, p12, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "second-order subpixel launch");
  return DIC_OK;
}

dic_status dic_subpixel(dic_t h, dic_method method, const int32_t* u0, const int32_t* v0,
                        const uint8_t* status0, float* u, float* v, float* ux, float* uy,
                        float* vx, float* vy, float* zncc, int32_t* iters, uint8_t* status) {
  if (!h) return DIC_ERR_ARG;
  if (method != DIC_ICGN && method != DIC_FANR) return fail(h, DIC_ERR_ARG, "unknown method");
  if (h->shape_order != 1)
    return fail(h, DIC_ERR_STATE, "a handle of shape order 2 refines with dic_subpixel2");
  if (!h->have_pair) return fail(h, DIC_ERR_STATE, "no image pair set");
  if (h->g.n_pois == 0) return DIC_OK;
  if (!u0 || !v0 || !status0 || !u || !v || !ux || !uy || !vx || !vy || !zncc || !iters ||
      !status)
    return fail(h, DIC_ERR_ARG, "null pointer");
  dic::SubpixelParams p;
  p.ref = h->ref;
  p.ref_f32 = h->ref_f32;
  p.grad = h->grad;
  p.gimg = h->gimg;
  p.gq = h->ref ? h->gq : nullptr;
  p.W = h->g.W;
  p.H = h->g.H;
  p.pitch = h->g.pitch;
  p.S = h->subset;
  p.M = h->M;
  p.R = h->R;
  p.step = h->step;
  p.nx = h->g.nx;
  p.n_pois = h->g.n_pois;
  p.max_iter = h->max_iter;
  p.tol = h->tol;
  p.u0 = u0;
  p.v0 = v0;
  p.st0 = status0;
  p.u = u;
  p.v = v;
  p.ux = ux;
  p.uy = uy;
  p.vx = vx;
  p.vy = vy;
  p.zncc = zncc;
  p.iters = iters;
  p.status = status;
  cudaError_t e = pre_join(h);
  if (e != cudaSuccess) return cuda_fail(h, e, "precompute join");
  e = dic::launch_subpixel(p, (int)method, h->solve_bits == 64, h->stream,
                           h->interp == DIC_INTERP_BILINEAR);
  if (e != cudaSuccess) return cuda_fail(h, e, "subpixel launch");
  return DIC_OK;
}

// ------------------------------------------------------------------ batches
}  // extern "C"

namespace {

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& v) {
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(dst, sizeof(T) * v.size());
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
}

// Fill the per-pair job arrays for the given outputs and copy them to the
// device (synchronous; done only when the graph is rebuilt).
dic_status write_jobs(dic_t h, const dic_batch_out& o, int solve_bits) {
  dic::BatchState* b = h->batch;
  std::vector<dic::SubpixelParams> pj(b->pairs.size());
  for (size_t k = 0; k < b->pairs.size(); ++k) {
    const dic::BatchPair& bp = b->pairs[k];
    dic::SubpixelParams& p = pj[k];
    p.ref = bp.d.ref_dev;
    p.grad = b->grad + bp.px_off;
    p.gimg = b->gimg + bp.px_off;
    p.gq = b->gq + bp.px_off;
    p.W = bp.d.width;
    p.H = bp.d.height;
    p.pitch = bp.d.pitch_bytes;
    p.S = bp.S;
    p.M = bp.M;
    p.R = bp.R;
    p.step = bp.step;
    p.nx = bp.nx;
    p.n_pois = bp.n;
    p.max_iter = h->max_iter;
    p.tol = h->tol;
    p.u0 = o.u0 + bp.off;
    p.v0 = o.v0 + bp.off;
    p.st0 = o.status0 + bp.off;
    p.u = o.u + bp.off;
    p.v = o.v + bp.off;
    p.ux = o.ux + bp.off;
    p.uy = o.uy + bp.off;
    p.vx = o.vx + bp.off;
    p.vy = o.vy + bp.off;
    p.zncc = o.zncc + bp.off;
    p.iters = o.iters + bp.off;
    p.status = o.status + bp.off;
  }
  if (cudaMemcpy(b->d_pjobs, pj.data(), sizeof(dic::SubpixelParams) * pj.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(h, DIC_ERR_CUDA, "job upload failed");
  b->pj = pj;
  for (auto& c : b->classes) {
    std::vector<dic::SearchParams> sj;
    for (int k : c.pairs) {
      const dic::BatchPair& bp = b->pairs[k];
      dic::SearchParams q{};
      q.ref = bp.d.ref_dev;
      q.def = bp.d.def_dev;
      q.W = bp.d.width;
      q.H = bp.d.height;
      q.pitch = bp.d.pitch_bytes;
      q.S = bp.S;
      q.M = bp.M;
      q.R = bp.R;
      q.step = bp.step;
      q.nx = bp.nx;
      q.n_pois = bp.n;
      q.use_tma = 0;
      q.u0 = o.u0 + bp.off;
      q.v0 = o.v0 + bp.off;
      q.zncc0 = o.zncc0 + bp.off;
      q.status = o.status0 + bp.off;
      q.err_flag = h->err_flag;
      sj.push_back(q);
    }
    if (cudaMemcpy(c.d_jobs, sj.data(), sizeof(dic::SearchParams) * sj.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(h, DIC_ERR_CUDA, "job upload failed");
  }
  (void)solve_bits;
  return DIC_OK;
}

// Scratch of the tensor-core search for the largest pair of the batch
// (allocated once; the pairs' searches run one after another and share it).
dic_status batch_tc_scratch(dic_t h) {
  dic::BatchState* b = h->batch;
  if (b->tc_phase) return DIC_OK;
  size_t phase = 0, pbe = 0, slots = 0;
  for (const dic::BatchPair& bp : b->pairs) {
    if (!bp.tc_ok) continue;  // no POI (checked by build_graph)
    phase = std::max(phase, dic::search_tc_phase_elems(bp.tc));
    pbe = std::max(pbe, dic::search_tc_posbox_elems(bp.tc));
    slots = std::max(slots, (size_t)bp.n * bp.tc.nslots);
  }
  if (cudaMalloc(&b->tc_phase, phase * sizeof(uint16_t)) != cudaSuccess ||
      cudaMalloc(&b->tc_fbox, pbe * sizeof(int2)) != cudaSuccess ||
      cudaMalloc(&b->tc_posbox, pbe * sizeof(int2)) != cudaSuccess ||
      cudaMalloc(&b->tc_slots, std::max<size_t>(slots, 1) * sizeof(dic::SlotCand)) !=
          cudaSuccess) {
    cudaGetLastError();
    // all or nothing: a later call must not find part of the scratch
    if (b->tc_phase) cudaFree(b->tc_phase);
    if (b->tc_fbox) cudaFree(b->tc_fbox);
    if (b->tc_posbox) cudaFree(b->tc_posbox);
    if (b->tc_slots) cudaFree(b->tc_slots);
    b->tc_phase = nullptr;
    b->tc_fbox = b->tc_posbox = nullptr;
    b->tc_slots = nullptr;
    return fail(h, DIC_ERR_OOM, "cannot allocate tensor-core search scratch for the batch");
  }
  return DIC_OK;
}

dic_status build_graph(dic_t h, dic_method method, const dic_batch_out& o) {
  dic::BatchState* b = h->batch;
  const bool tc = h->form == DIC_FORM_BF16TC;
  const bool overlap = b->grid_mult == 0;
  if (overlap && !tc)
    return fail(h, DIC_ERR_ARG, "overlapped per-pair sub-pixel launches need the tensor-core form");
  for (size_t k = 0; k < b->pairs.size(); ++k) {
    const dic::BatchPair& bp = b->pairs[k];
    if (bp.n > 0 && !(tc ? bp.tc_ok : bp.fp32_ok))
      return fail(h, DIC_ERR_UNSUPPORTED,
                  "pair %zu: subset %d, step %d, radius %d not supported by the %s search", k,
                  bp.S, bp.step, bp.R, tc ? "tensor-core" : "FP32");
  }
  dic_status st = write_jobs(h, o, h->solve_bits);
  if (st != DIC_OK) return st;
  if (tc && (st = batch_tc_scratch(h)) != DIC_OK) return st;
  // per-pair tensor-core search parameters and tensor maps (by value in the
  // graph's kernel nodes)
  std::vector<dic::SearchTcParams> tcp;
  std::vector<CUtensorMap> tma, tmb;
  if (tc) {
    tcp.resize(b->pairs.size());
    tma.resize(b->pairs.size());
    tmb.resize(b->pairs.size());
    for (size_t k = 0; k < b->pairs.size(); ++k) {
      const dic::BatchPair& bp = b->pairs[k];
      dic::SearchTcParams& t = tcp[k];
      t = bp.tc;
      t.ref = bp.d.ref_dev;
      t.def = bp.d.def_dev;
      t.W = bp.d.width;
      t.H = bp.d.height;
      t.pitch = bp.d.pitch_bytes;
      t.n_pois = bp.n;
      t.gph = b->tc_phase;
      t.bank = b->tc_phase + dic::search_tc_gph_elems(t);
      t.fbox = b->tc_fbox;
      t.posbox = b->tc_posbox;
      t.slots = b->tc_slots;
      t.u0 = o.u0 + bp.off;
      t.v0 = o.v0 + bp.off;
      t.zncc0 = o.zncc0 + bp.off;
      t.status = o.status0 + bp.off;
      t.err_flag = h->err_flag;
      if (bp.n > 0 && !encode_tc(&tma[k], &tmb[k], t))
        return fail(h, DIC_ERR_UNSUPPORTED, "pair %zu: tensor map encoding failed", k);
    }
  }
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t cs = b->cap;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return cuda_fail(h, e, "graph capture");
  cudaError_t le = cudaMemsetAsync(b->d_counters, 0,
                                   sizeof(unsigned long long) * (b->classes.size() + 1), cs);
  for (const dic::BatchPair& bp : b->pairs) {
    if (le != cudaSuccess) break;
    le = dic::launch_precompute(bp.d.ref_dev, bp.d.def_dev, bp.d.width, bp.d.height,
                                bp.d.pitch_bytes, b->grad + bp.px_off, b->gimg + bp.px_off,
                                b->gq + bp.px_off, cs);
  }
  // integer search: the tensor-core form pair by pair (each launch fills
  // the GPU: tens of thousands of tile CTAs per 2048^2 pair), or one
  // persistent FP32 kernel per template-width class over a work counter.
  // Overlapped mode: pair k's sub-pixel kernel runs on the side stream as
  // soon as its search is done, beside the searches of the pairs after it
  // (tensor pipe and FP32 pipes in use at once); the side stream forks from
  // and joins back into the capture stream.
  if (overlap && le == cudaSuccess) {
    le = cudaEventRecord(b->evs[0], cs);
    if (le == cudaSuccess) le = cudaStreamWaitEvent(b->side, b->evs[0], 0);
  }
  for (size_t k = 0; tc && k < b->pairs.size() && le == cudaSuccess; ++k) {
    if (b->pairs[k].n == 0) continue;
    le = dic::launch_search_tc(tcp[k], &tma[k], &tmb[k], cs);
    if (overlap && le == cudaSuccess) {
      le = cudaEventRecord(b->evs[1 + k], cs);
      if (le == cudaSuccess) le = cudaStreamWaitEvent(b->side, b->evs[1 + k], 0);
      if (le == cudaSuccess)
        le = dic::launch_subpixel(b->pj[k], (int)method, h->solve_bits == 64, b->side);
    }
  }
  if (overlap && le == cudaSuccess) {
    le = cudaEventRecord(b->evs[b->pairs.size() + 1], b->side);
    if (le == cudaSuccess) le = cudaStreamWaitEvent(cs, b->evs[b->pairs.size() + 1], 0);
  }
  for (size_t c = 0; !tc && c < b->classes.size() && le == cudaSuccess; ++c) {
    dic::BatchClass& cl = b->classes[c];
    int occ = dic::search_batch_occupancy(cl.tw, cl.smem);
    int64_t items = 0;
    for (int k : cl.pairs) items += b->pairs[k].n;
    int64_t grid = (int64_t)(occ > 0 ? occ : 1) * sms * b->grid_mult;
    if (grid > items) grid = items;
    if (grid < 1) grid = 1;
    le = dic::launch_search_batch(cl.tw, cl.d_jobs, cl.d_offsets, (int)cl.pairs.size(),
                                  b->d_counters + c, cl.smem, (int)grid, cs);
  }
  if (le == cudaSuccess && !overlap) {
    // grid <= 0 asks the launcher for (resident CTAs x SMs) x -grid
    le = dic::launch_subpixel_batch(b->d_pjobs, b->d_offsets, (int)b->pairs.size(), b->nmax,
                                    (int)method, h->solve_bits == 64, b->wpc,
                                    b->d_counters + b->classes.size(), -b->grid_mult, cs);
  }
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cs, &graph);
  if (le != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(h, le, "batch launch during capture");
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "graph capture end");
  e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiate");
  b->last_out = o;
  b->last_method = (int)method;
  b->last_wpc = b->wpc;
  b->last_mult = b->grid_mult;
  b->last_bits = h->solve_bits;
  b->last_form = h->form;
  return DIC_OK;
}

bool same_out(const dic_batch_out& a, const dic_batch_out& b) {
  return memcmp(&a, &b, sizeof a) == 0;
}

}  // namespace

extern "C" {

dic_status dic_set_pairs(dic_t h, int n_pairs, const dic_pair_desc* descs) {
  if (!h) return DIC_ERR_ARG;
  free_batch(h->batch);
  h->batch = nullptr;
  if (n_pairs < 1 || !descs) return fail(h, DIC_ERR_ARG, "need at least one pair descriptor");
  dic::BatchState* b = new (std::nothrow) dic::BatchState;
  if (!b) return DIC_ERR_OOM;
  int64_t off = 0;
  size_t px = 0;
  for (int k = 0; k < n_pairs; ++k) {
    dic::BatchPair bp;
    bp.d = descs[k];
    bp.S = bp.d.subset_size > 0 ? bp.d.subset_size : h->subset;
    bp.step = bp.d.grid_step > 0 ? bp.d.grid_step : h->step;
    bp.R = bp.d.search_radius >= 0 ? bp.d.search_radius : h->R;
    bp.M = bp.S / 2;
    if (!bp.d.ref_dev || !bp.d.def_dev || bp.d.width < 4 || bp.d.height < 4 ||
        bp.d.pitch_bytes < bp.d.width || bp.S < 3 || bp.S > dic::kMaxSubset || (bp.S & 1) == 0 ||
        bp.R > 1000) {
      delete b;
      return fail(h, DIC_ERR_ARG, "bad descriptor for pair %d", k);
    }
    grid_of(bp.d.width, bp.d.height, bp.S, bp.step, bp.R, &bp.nx, &bp.ny);
    bp.fp32_ok = dic::search_smem_bytes(bp.S, bp.R) <= 227 * 1024;
    bp.tc_ok = tc_geometry(bp.d.width, bp.d.height, bp.S, bp.step, bp.R, bp.nx,
                                       bp.ny, &bp.tc) &&
               dic::search_tc_smem(bp.tc) <= 227 * 1024;
    if (!bp.fp32_ok && !bp.tc_ok && bp.nx > 0 && bp.ny > 0) {
      delete b;
      return fail(h, DIC_ERR_UNSUPPORTED,
                  "pair %d: search window (subset %d, step %d, radius %d) fits neither search "
                  "form",
                  k, bp.S, bp.step, bp.R);
    }
    bp.n = (int64_t)bp.nx * bp.ny;
    bp.off = off;
    bp.px_off = px;
    bp.tw = (bp.S + 3) / 4 * 4;
    off += bp.n;
    px += (size_t)bp.d.width * bp.d.height;
    if (bp.S * bp.S > b->nmax) b->nmax = bp.S * bp.S;
    b->pairs.push_back(bp);
    if (!bp.fp32_ok) continue;  // tensor-core search only
    bool placed = false;
    for (auto& c : b->classes)
      if (c.tw == bp.tw) {
        c.pairs.push_back(k);
        c.smem = std::max(c.smem, dic::search_smem_bytes(bp.S, bp.R));
        placed = true;
      }
    if (!placed) {
      dic::BatchClass c;
      c.tw = bp.tw;
      c.pairs.push_back(k);
      c.smem = dic::search_smem_bytes(bp.S, bp.R);
      b->classes.push_back(c);
    }
  }
  b->total = off;
  b->px_total = px;
  h->batch = b;
  if (!h->err_flag) {
    if (cudaMalloc(&h->err_flag, sizeof(unsigned int)) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, DIC_ERR_OOM, "cannot allocate error flag");
    }
    cudaMemset(h->err_flag, 0, sizeof(unsigned int));
  }
  std::vector<int64_t> offs;
  for (auto& bp : b->pairs) offs.push_back(bp.off);
  offs.push_back(off);
  cudaError_t e = cudaMalloc(&b->gimg, px * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&b->grad, px * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&b->gq, px * sizeof(uint2));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_pjobs, sizeof(dic::SubpixelParams) * n_pairs);
  if (e == cudaSuccess) e = upload(&b->d_offsets, offs);
  if (e == cudaSuccess)
    e = cudaMalloc(&b->d_counters, sizeof(unsigned long long) * (b->classes.size() + 1));
  for (auto& c : b->classes) {
    if (e != cudaSuccess) break;
    std::vector<int64_t> co{0};
    for (int k : c.pairs) co.push_back(co.back() + b->pairs[k].n);
    e = cudaMalloc(&c.d_jobs, sizeof(dic::SearchParams) * c.pairs.size());
    if (e == cudaSuccess) e = upload(&c.d_offsets, co);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    int lo = 0, hi = 0;  // the side stream at the highest priority
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    e = cudaStreamCreateWithPriority(&b->side, cudaStreamNonBlocking, hi);
  }
  for (int k = 0; e == cudaSuccess && k < n_pairs + 2; ++k) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->evs.push_back(ev);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    h->batch = nullptr;
    return fail(h, DIC_ERR_OOM, "cannot allocate batch scratch (%zu pixels)", px);
  }
  return DIC_OK;
}

dic_status dic_batch_pois(dic_t h, int64_t* total, int64_t* offsets) {
  if (!h) return DIC_ERR_ARG;
  if (!h->batch) return fail(h, DIC_ERR_STATE, "no batch set");
  if (total) *total = h->batch->total;
  if (offsets) {
    for (size_t k = 0; k < h->batch->pairs.size(); ++k) offsets[k] = h->batch->pairs[k].off;
    offsets[h->batch->pairs.size()] = h->batch->total;
  }
  return DIC_OK;
}

dic_status dic_run_batch(dic_t h, dic_method method, const dic_batch_out* out) {
  if (!h) return DIC_ERR_ARG;
  if (!h->batch) return fail(h, DIC_ERR_STATE, "no batch set");
  if (method != DIC_ICGN && method != DIC_FANR) return fail(h, DIC_ERR_ARG, "unknown method");
  if (!out) return fail(h, DIC_ERR_ARG, "null output descriptor");
  dic::BatchState* b = h->batch;
  if (h->interp != DIC_INTERP_BICUBIC)
    return fail(h, DIC_ERR_UNSUPPORTED, "the batch form interpolates bicubically only");
  if (b->total == 0) return DIC_OK;
  const dic_batch_out& o = *out;
  if (!o.u0 || !o.v0 || !o.zncc0 || !o.status0 || !o.u || !o.v || !o.ux || !o.uy || !o.vx ||
      !o.vy || !o.zncc || !o.iters || !o.status)
    return fail(h, DIC_ERR_ARG, "null output array");
  if (!b->exec || !same_out(b->last_out, o) || b->last_method != (int)method ||
      b->last_wpc != b->wpc || b->last_mult != b->grid_mult || b->last_bits != h->solve_bits ||
      b->last_form != h->form) {
    dic_status st = build_graph(h, method, o);
    if (st != DIC_OK) return st;
  }
  cudaError_t e = cudaGraphLaunch(b->exec, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
  return DIC_OK;
}

dic_status dic_set_batch_shape(dic_t h, int warps_per_cta, int grid_mult) {
  if (!h) return DIC_ERR_ARG;
  if (!h->batch) return fail(h, DIC_ERR_STATE, "no batch set");
  const bool persistent = (warps_per_cta == 2 || warps_per_cta == 4 || warps_per_cta == 8) &&
                          (grid_mult == 1 || grid_mult == 2);
  if (!persistent && !(warps_per_cta == 0 && grid_mult == 0))
    return fail(h, DIC_ERR_ARG, "batch shape {%d, %d}: want {2|4|8, 1|2} or {0, 0}",
                warps_per_cta, grid_mult);
  h->batch->wpc = warps_per_cta;
  h->batch->grid_mult = grid_mult;
  return DIC_OK;
}

dic_status dic_autotune(dic_t h, dic_method method, const dic_batch_out* out, int* chosen) {
  if (!h) return DIC_ERR_ARG;
  if (!h->batch) return fail(h, DIC_ERR_STATE, "no batch set");
  dic::BatchState* b = h->batch;
  // persistent sub-pixel kernel: warps per CTA x grid multiple; with the
  // tensor-core search also per-pair launches overlapped with the searches
  // (encoded {0, 0})
  std::vector<std::pair<int, int>> cands;
  for (int w : {2, 4, 8})
    for (int m : {1, 2}) cands.push_back({w, m});
  if (h->form == DIC_FORM_BF16TC) cands.push_back({0, 0});
  float best = 1e30f;
  int bw = b->wpc, bm = b->grid_mult;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (const auto& c : cands) {
    b->wpc = c.first;
    b->grid_mult = c.second;
    dic_status st = dic_run_batch(h, method, out);  // builds and warms up
    if (st != DIC_OK) continue;
    cudaEventRecord(e0, h->stream);
    for (int r = 0; r < 3; ++r) dic_run_batch(h, method, out);
    cudaEventRecord(e1, h->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      bw = c.first;
      bm = c.second;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->wpc = bw;
  b->grid_mult = bm;
  if (chosen) {
    chosen[0] = bw;
    chosen[1] = bm;
  }
  return best < 1e30f ? DIC_OK : fail(h, DIC_ERR_CUDA, "no candidate ran");
}


// ------------------------------------------------------- frame streams
dic_status dic_stream_push(dic_t h, const uint8_t* frame, int width, int height, int pitch_bytes,
                           dic_method method, const dic_batch_out* out) {
  if (!h) return DIC_ERR_ARG;
  if (!frame) return fail(h, DIC_ERR_ARG, "null frame pointer");
  if (width < 4 || height < 4 || pitch_bytes < width)
    return fail(h, DIC_ERR_ARG, "bad frame size %dx%d pitch %d", width, height, pitch_bytes);
  if (method != DIC_ICGN && method != DIC_FANR) return fail(h, DIC_ERR_ARG, "unknown method");
  if (!h->seq) {
    h->seq = new (std::nothrow) dic::StreamState();
    if (!h->seq) return fail(h, DIC_ERR_OOM, "cannot allocate the stream state");
  }
  dic::StreamState* q = h->seq;
  const long long k = q->frames;
  if (k > 0 && (width != q->W || height != q->H))
    return fail(h, DIC_ERR_ARG, "frame %dx%d differs from the sequence's %dx%d", width, height,
                q->W, q->H);
  int nx = 0, ny = 0;
  grid_of(width, height, h->subset, h->step, h->R, &nx, &ny);
  const int64_t n = (int64_t)nx * ny;
  if (k > 0 && n > 0 &&
      (!out || !out->u0 || !out->v0 || !out->zncc0 || !out->status0 || !out->u || !out->v ||
       !out->ux || !out->uy || !out->vx || !out->vy || !out->zncc || !out->iters ||
       !out->status))
    return fail(h, DIC_ERR_ARG, "null output array");
  if (k == 0) {
    // a new sequence: (re)allocate the ring for this frame size
    const int rp = (width + 15) / 16 * 16;
    const size_t px = (size_t)width * height;
    if (q->pending && q->side) cudaStreamSynchronize(q->side);
    q->pending = false;
    if (rp != q->pitch || height != q->H || px > q->px) {
      for (int j = 0; j < 3; ++j) {
        if (q->frame[j]) cudaFree(q->frame[j]);
        if (q->grad[j]) cudaFree(q->grad[j]);
        if (q->gimg[j]) cudaFree(q->gimg[j]);
        if (q->gq[j]) cudaFree(q->gq[j]);
        q->frame[j] = nullptr;
        q->grad[j] = nullptr;
        q->gimg[j] = nullptr;
        q->gq[j] = nullptr;
      }
      q->px = 0;
      for (int j = 0; j < 3; ++j)
        if (cudaMalloc(&q->frame[j], (size_t)rp * height) != cudaSuccess ||
            cudaMalloc(&q->grad[j], px * sizeof(float2)) != cudaSuccess ||
            cudaMalloc(&q->gimg[j], px * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&q->gq[j], px * sizeof(uint2)) != cudaSuccess) {
          cudaGetLastError();
          return fail(h, DIC_ERR_OOM, "cannot allocate the frame ring (%zu bytes)",
                      3 * ((size_t)rp * height + 20 * px));
        }
      q->px = px;
    }
    if (!q->side) {
      if (cudaStreamCreateWithFlags(&q->side, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&q->searched, cudaEventDisableTiming) != cudaSuccess)
        return cuda_fail(h, cudaGetLastError(), "stream set-up");
      for (int j = 0; j < 3; ++j)
        if (cudaEventCreateWithFlags(&q->refined[j], cudaEventDisableTiming) != cudaSuccess)
          return cuda_fail(h, cudaGetLastError(), "stream set-up");
    }
    if (!h->err_flag) {
      if (cudaMalloc(&h->err_flag, sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, DIC_ERR_OOM, "cannot allocate error flag");
      }
      cudaMemsetAsync(h->err_flag, 0, sizeof(unsigned int), h->stream);
    }
    q->W = width;
    q->H = height;
    q->pitch = rp;
    // the stream's geometry replaces a bound pair
    h->have_pair = false;
    h->g.W = width;
    h->g.H = height;
    h->g.pitch = rp;
    h->g.nx = nx;
    h->g.ny = ny;
    h->g.n_pois = n;
  }
  const int s = (int)(k % 3);
  cudaStream_t st = h->stream;
  cudaError_t e = cudaSuccess;
  // slot s last served as the reference of pair k-2 (its sub-pixel work on
  // the second stream) before this frame overwrites it
  if (k >= 3) e = cudaStreamWaitEvent(st, q->refined[(k - 2) % 3], 0);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(q->frame[s], q->pitch, frame, pitch_bytes, width, height,
                          cudaMemcpyDeviceToDevice, st);
  // the frame's precompute, once: gradients (its turn as reference), float
  // copy and tap quads (its turn as target)
  if (e == cudaSuccess)
    e = dic::launch_precompute(q->frame[s], q->frame[s], width, height, q->pitch, q->grad[s],
                               q->gimg[s], q->gq[s], st);
  if (e != cudaSuccess) return cuda_fail(h, e, "frame copy / precompute");
  if (k >= 1 && n > 0) {
    const int r = (int)((k - 1) % 3);
    // integer search of pair (k-1, k) on the handle's stream
    CUtensorMap tmr{}, tmd{};
    const int span = h->subset + 2 * h->R;
    const int bwg = dic::tma_box_width(span), bwf = dic::tma_box_width(h->subset);
    const bool tma = bwg <= 256 && span <= 256 &&
                     encode_u8(&tmd, q->frame[s], width, height, q->pitch, bwg, span) &&
                     encode_u8(&tmr, q->frame[r], width, height, q->pitch, bwf, h->subset);
    dic_status ds = search_images(h, q->frame[r], q->frame[s], tma, &tmr, &tmd, out->u0, out->v0,
                                  out->zncc0, out->status0, st);
    if (ds != DIC_OK) return ds;
    // its sub-pixel refinement on the second stream, overlapping the next
    // pair's search
    e = cudaEventRecord(q->searched, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(q->side, q->searched, 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "stream ordering");
    ds = subpixel_images(h, method, q->frame[r], q->grad[r], q->gimg[s], q->gq[s], out->u0,
                         out->v0, out->status0, out->u, out->v, out->ux, out->uy, out->vx,
                         out->vy, out->zncc, out->iters, out->status, q->side);
    if (ds != DIC_OK) return ds;
    e = cudaEventRecord(q->refined[k % 3], q->side);
    // the previous pair's outputs join the handle's stream (after this
    // pair's search has been enqueued)
    if (e == cudaSuccess && q->pending) e = cudaStreamWaitEvent(st, q->refined[(k - 1) % 3], 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "stream ordering");
    q->pending = true;
  }
  q->frames = k + 1;
  return DIC_OK;
}

dic_status dic_stream_flush(dic_t h) {
  if (!h) return DIC_ERR_ARG;
  dic::StreamState* q = h->seq;
  if (!q || !q->pending) return DIC_OK;
  cudaError_t e = cudaStreamWaitEvent(h->stream, q->refined[(q->frames - 1) % 3], 0);
  if (e != cudaSuccess) return cuda_fail(h, e, "stream flush");
  q->pending = false;
  return DIC_OK;
}

dic_status dic_stream_reset(dic_t h) {
  if (!h) return DIC_ERR_ARG;
  dic_status st = dic_stream_flush(h);
  if (st != DIC_OK) return st;
  if (h->seq) h->seq->frames = 0;
  return DIC_OK;
}

}  // extern "C"
