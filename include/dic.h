/*
 * dic.h -- C ABI of the GB300 digital-image-correlation hot path.
 *
 * Method: Thoma & Ravi, "Significance of parallel computing on the
 * performance of Digital Image Correlation algorithms in MATLAB".  For every
 * point of interest (POI) on a regular grid of the reference image f, the
 * library finds the integer displacement that maximises the zero-normalised
 * cross-correlation (ZNCC, Eq. 1) of a (2M+1)x(2M+1) subset by brute-force
 * search (Section 2.1), then refines it to sub-pixel accuracy with a
 * first-order (6-parameter, affine) subset shape function over bicubically
 * (or, on request, bilinearly: Eq. 5) interpolated deformed-image grey
 * levels, by the inverse-compositional Gauss-Newton algorithm or by
 * forward-additive Newton-Raphson (Section 2.2, Table 2).
 *
 * Conventions shared by every call:
 *  - Images are 8-bit grey, row-major, pixel (x, y) at byte y*pitch + x;
 *    x is the column, y the row.
 *  - All image and array pointers are DEVICE pointers.  The caller allocates
 *    and owns them; the library never frees caller memory and keeps image
 *    pointers only as borrowed references between dic_set_pair and the next
 *    dic_set_pair / dic_destroy (the images must stay alive and unchanged).
 *  - The library owns its scratch (float copy and tap quads of the deformed
 *    image, gradient field; the search forms' and batches' own scratch),
 *    allocates it on first use (dic_set_pair, dic_integer_search,
 *    dic_set_pairs, dic_run_batch) and frees it in dic_destroy.
 *  - Work is enqueued asynchronously on the stream given to dic_set_stream
 *    (default: the legacy default stream).  Argument errors are returned
 *    synchronously; a CUDA launch error is returned as DIC_ERR_CUDA with the
 *    message in dic_last_error.  Per-POI numerical outcomes are reported in
 *    the per-POI status arrays, never as a call failure.
 *  - POI k lies at x0 = B + (k % nx)*step, y0 = B + (k / nx)*step with
 *    B = M + R + 2, so the whole search window and the 4x4 interpolation
 *    stencil of every integer start stay inside the image.  The paper does
 *    not state a grid; this margin is the reading used here.
 *  - Shape vector order p = (u, ux, uy, v, vx, vy); the warp of subset point
 *    (dx, dy) is (x0 + dx + u + ux*dx + uy*dy, y0 + dy + v + vx*dx + vy*dy).
 *  - Calls on one handle are not thread-safe; distinct handles are.
 */
#ifndef DIC_GB300_H
#define DIC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dic_s *dic_t;

typedef enum {
  DIC_OK = 0,
  DIC_ERR_ARG = -1,         /* invalid argument (null, size, alignment)        */
  DIC_ERR_CUDA = -2,        /* CUDA runtime error; see dic_last_error           */
  DIC_ERR_OOM = -3,         /* device allocation of library scratch failed      */
  DIC_ERR_STATE = -4,       /* call out of order (e.g. no pair set)             */
  DIC_ERR_TIMEOUT = -5,     /* a bounded device wait gave up                    */
  DIC_ERR_UNSUPPORTED = -6  /* valid request this build does not implement      */
} dic_status;

typedef enum { DIC_ICGN = 0, DIC_FANR = 1 } dic_method;

/* Integer-search arithmetic.  Both forms return the same argmax. */
typedef enum {
  DIC_FORM_PLAIN_FP32 = 0, /* FP32 FMA correlation per POI, exact integer sums  */
  DIC_FORM_BF16TC = 1      /* BF16 tensor-core correlation (tcgen05) across POIs,
                              exact FP32 accumulation, exact comparison of the
                              near-tied candidates of every tile and POI       */
} dic_form;

/* Interpolation of the deformed image between pixels (Section 2.2). */
typedef enum {
  DIC_INTERP_BICUBIC = 0,  /* Keys cubic convolution, a = -1/2, 4x4 pixels      */
  DIC_INTERP_BILINEAR = 1  /* Eq. 5: a00 + a10 x' + a01 y' + a11 x'y' on 2x2    */
} dic_interp;

/* Per-POI status codes written by dic_integer_search / dic_subpixel. */
enum {
  DIC_POI_OK = 0,
  DIC_POI_ZERO_VAR_REF = 1,  /* flat reference subset: Eq. 1 undefined           */
  DIC_POI_OUT_OF_BOUNDS = 2, /* an update would move the subset off the image     */
  DIC_POI_MAX_ITER = 3,      /* iteration cap reached; last shape still returned  */
  DIC_POI_NONFINITE = 4,     /* flat target subset or non-finite update           */
  DIC_POI_SINGULAR = 5,      /* 6x6 Gauss-Newton matrix not positive definite     */
  DIC_POI_ZERO_VAR_DEF = 6   /* every candidate target subset is flat             */
};

/* Library version as an integer major*10000 + minor*100 + patch. */
int dic_version(void);

/* Create a handle.
 *   subset_size    odd, >= 3 and <= 63 (the paper's (2M+1), Section 2.1)
 *   grid_step      POI spacing in pixels, >= 1
 *   search_radius  R >= 0: offsets [-R, R]^2 are searched (Section 2.1 uses a
 *                  fixed window around the reference position)
 *   shape_order    1 = first-order 6-parameter warp (dic_subpixel), or
 *                  2 = second-order 12-parameter warp (dic_subpixel2, an
 *                  extension: the paper's refinement is first-order);
 *                  anything else returns DIC_ERR_UNSUPPORTED
 *   conv_tol       stop when |dp| < conv_tol, with
 *                  |dp| = sqrt(du^2 + dv^2 + M^2 (dux^2+duy^2+dvx^2+dvy^2))
 *   max_iter       maximum Gauss-Newton solves per POI, >= 1
 * Host-only: touches no GPU.  *out is NULL on failure. */
dic_status dic_create(dic_t *out, int subset_size, int grid_step, int search_radius,
                      int shape_order, float conv_tol, int max_iter);

/* Release the handle and its device scratch.  NULL is accepted. */
void dic_destroy(dic_t h);

/* Message of the last failed call on this handle ("" if none). */
const char *dic_last_error(dic_t h);

/* Failure report of the device side.  Every wait inside the search kernels
 * (on a TMA copy or an MMA, through an mbarrier) is bounded; a kernel whose
 * wait gives up records it in the handle's error flag, waits (bounded) for
 * its own copies in flight and returns, leaving its results incomplete.
 * dic_check synchronises the handle's stream, reads the flag and returns
 * DIC_ERR_TIMEOUT (clearing the flag; dic_last_error names the kernel and,
 * for the tensor-core tile kernel, which wait gave up: A buffer free, B
 * stage free, accumulator read, A landed, B landed, accumulator complete,
 * last MMAs) if it is set, DIC_OK otherwise (also before any launch);
 * DIC_ERR_CUDA if the stream itself failed.  No counterpart in the paper. */
dic_status dic_check(dic_t h);

/* Stream for all later work (a cudaStream_t passed as void*; NULL = default). */
dic_status dic_set_stream(dic_t h, void *cuda_stream);

/* Integer-search arithmetic form (see dic_form).  The tensor-core form splits
 * the POIs whose search windows meet a 16x8 block of positions into row
 * chunks of at most 256 (and 512 TMEM columns of accumulators); it needs one
 * row of that block, (2R+8)/step + 1 POIs, to fit, and returns
 * DIC_ERR_UNSUPPORTED from dic_integer_search otherwise.  It allocates
 * scratch on first use: a BF16 copy of every subset (2*S*TWK bytes per POI,
 * TWK = 16, 32 or 64 >= S), eight shifted BF16 copies of g (16 bytes per
 * pixel), box-sum maps and one 24-byte winner slot per (position tile,
 * POI). */
dic_status dic_set_form(dic_t h, dic_form form);

/* Precision of the per-POI 6x6 Gauss-Newton solve: 32 (FP32) or 64 (FP64):
 * the matrix is inverted in that precision (symmetric Gauss-Jordan sweep
 * on its unit-diagonal scaling) and multiplied by the right-hand side.  The
 * per-point work is FP32 either way.  Default 32. */
dic_status dic_set_solve_precision(dic_t h, int bits);

/* Interpolation of g in dic_subpixel (Section 2.2): DIC_INTERP_BICUBIC
 * (default) or DIC_INTERP_BILINEAR (Eq. 5; FA-NR then takes the gradient of
 * the bilinear patch the sample falls in, IC-GN keeps the central-difference
 * gradients of f).  dic_run_batch, dic_znssd / dic_backward and
 * dic_subpixel_noalloc interpolate bicubically; dic_run_batch returns
 * DIC_ERR_UNSUPPORTED with bilinear set.  DIC_ERR_ARG for other values. */
dic_status dic_set_interpolation(dic_t h, dic_interp interp);

/* Bind a reference/deformed image pair (device pointers, borrowed) and
 * enqueue the precompute kernel: central-difference gradients of f, g as
 * float, and g's BF16 tap quads (the four taps of a bicubic stencil row per
 * pixel; Section 2.2's interpolation evaluates its weights per sample
 * instead of the look-up table of its ref. [18]).
 *   width, height  >= 4 pixels each
 *   pitch_bytes    >= width; both pointers 16-byte aligned and pitch a
 *                  multiple of 16 enable TMA staging, otherwise plain loads
 * Allocates scratch of 20 bytes per pixel on first use or growth
 * (DIC_ERR_OOM on failure).  The precompute runs on a stream of the
 * handle's own that first waits for everything already queued on the
 * handle's stream, so that it overlaps the next integer search; it is joined
 * back into the handle's stream by the first of dic_integer_search,
 * dic_pso_search, dic_subpixel, dic_subpixel2, dic_znssd, dic_backward and
 * dic_check, so work queued on the handle's stream after any of them comes
 * after it.  The images must not be rewritten before such a call.  While
 * the handle's stream is being captured into a graph the precompute stays on
 * that stream. */
dic_status dic_set_pair(dic_t h, const uint8_t *ref_dev, const uint8_t *def_dev,
                        int width, int height, int pitch_bytes);

/* Float variant of dic_set_pair for real-valued images (pitch in elements,
 * 4-byte aligned).  It serves differentiation with respect to the deformed
 * image (dic_backward) and sub-pixel refinement of float data;
 * dic_integer_search needs 8-bit images (exact sums) and returns
 * DIC_ERR_UNSUPPORTED on a float pair. */
dic_status dic_set_pair_f32(dic_t h, const float *ref_dev, const float *def_dev, int width,
                            int height, int pitch_elems);

/* Grid size of the bound pair: n_pois = nx * ny (0 if the image is too
 * small for one POI).  Any output pointer may be NULL. */
dic_status dic_num_pois(dic_t h, int *n_pois, int *nx, int *ny);

/* Brute-force integer search (Eq. 1, Section 2.1) for every POI.
 * Outputs (device, n_pois each): u0, v0 = best integer offset in [-R, R];
 * zncc0 = its ZNCC; status = DIC_POI_OK / ZERO_VAR_REF / ZERO_VAR_DEF.
 * Every candidate's sums are exact integers; ties keep the lowest linear
 * index (v0+R)(2R+1)+(u0+R).  Requires dic_set_pair (else DIC_ERR_STATE). */
dic_status dic_integer_search(dic_t h, int32_t *u0, int32_t *v0, float *zncc0,
                              uint8_t *status);

/* Integer search by particle swarm optimisation (Section 2.1, Eqs. 2-4), or
 * by the modified swarm whose particles also evaluate the four pixels
 * around their own every generation and move to the best of the five (the
 * star search the paper folds into the swarm, Sections 3 and 5), over the
 * same window [-R, R]^2 as dic_integer_search.  Per POI and generation t:
 *   t = 0   position R (2u0 - 1, 2u1 - 1), velocity vinit (2u2 - 1, 2u3 - 1)
 *   t >= 1  v <- ((w v) + (c1 r1)(pbest - p)) + (c2 r2)(gbest - p)  (Eq. 2),
 *           w = 0.9 - (t - 1) / (2 generations)                     (Eq. 4),
 *           r1 = (u0, u1), r2 = (u2, u3) per direction; p <- p + v  (Eq. 3),
 *           clamped to [-R, R] per direction
 *   Eq. 1 at the nearest pixel floor(p + 1/2) (and the modified swarm's star
 *   pixels inside the window; ties: centre, +x, -x, +y, -y); pbest takes a
 *   strictly better pixel; gbest the first strictly better pbest in particle
 *   order.  Stop after the first generation whose gbest has
 *   C >= stop_num / stop_den (tested exactly), else after `generations`.
 * The particle arithmetic is FP64, each product and sum rounded on its own in
 * that order; Eq. 1 comes from exact integer sums and candidates compare
 * exactly as in dic_integer_search.  The swarm's random numbers are inputs:
 *   uniforms      device, [n_pois][generations][particles][4] doubles in
 *                 [0, 1): generation 0 holds the start draws, generation
 *                 t >= 1 the r1 (x, y) and r2 (x, y) of the update into t
 *   particles     1..64 (Section 5 uses 50); generations 1..1000 (5)
 *   c1, c2, vinit finite (the paper fixes none of them; 2, 2 and R/4 are
 *                 the values used elsewhere in this library's documentation)
 *   stop_num/den  0..2^20 / 1..2^20 (995/1000 stops at C >= 0.995)
 * Outputs (device, n_pois each): u0, v0 = gbest; zncc0 = its Eq. 1 (FP32 from
 * the exact sums); status OK / ZERO_VAR_REF / ZERO_VAR_DEF (every pixel the
 * swarm saw has a flat target subset); gens = generations run (0 for a flat
 * reference); evals = distinct pixels evaluated (each pixel once per POI).
 * Requires dic_set_pair with an 8-bit pair (else DIC_ERR_STATE /
 * DIC_ERR_UNSUPPORTED); DIC_ERR_ARG for the ranges above or a null pointer;
 * DIC_ERR_UNSUPPORTED if the window and the pixel table of one POI exceed
 * shared memory.  Reuses the handle's box-sum scratch (8 bytes per subset
 * position of f and of g, allocated on first use). */
dic_status dic_pso_search(dic_t h, int modified, int particles, int generations, double c1,
                          double c2, double vinit, int stop_num, int stop_den,
                          const double *uniforms, int32_t *u0, int32_t *v0, float *zncc0,
                          uint8_t *status, int32_t *gens, int32_t *evals);

/* Sub-pixel refinement (Section 2.2) of every POI from the integer start
 * (u0, v0, status0), e.g. the outputs of dic_integer_search.  POIs whose
 * status0 is not DIC_POI_OK are passed through with zero gradients.
 * Outputs (device, n_pois each): the six shape parameters, zncc (Eq. 1 at the
 * returned shape; for a converged POI, at the shape its last iteration
 * sampled, which differs from the returned one by the final update, below
 * the tolerance, at a stationary point of Eq. 1), iters (solves performed)
 * and status. */
dic_status dic_subpixel(dic_t h, dic_method method, const int32_t *u0, const int32_t *v0,
                        const uint8_t *status0, float *u, float *v, float *ux, float *uy,
                        float *vx, float *vy, float *zncc, int32_t *iters,
                        uint8_t *status);

/* Sub-pixel refinement with the second-order subset shape function
 * (handles created with shape_order 2; an extension of Section 2.2's
 * first-order warp):
 *   p = (u, ux, uy, uxx, uxy, uyy, v, vx, vy, vxx, vxy, vyy), point (dx, dy)
 *   -> (x0 + dx + p[0..5] . e, y0 + dy + p[6..11] . e),
 *   e = (1, dx, dy, dx^2/2, dx dy, dy^2/2).
 * IC-GN: SD = [fx e, fy e], H = sum SD^T SD (12 x 12, inverted once per POI
 * in the handle's solve precision), dp = -H^-1 sum SD r, and
 * W(p) <- W(p) W(dp)^-1 composed in the 6 x 6 representation of a
 * quadratic warp acting on (dx^2, dx dy, dy^2, dx, dy, 1), terms above
 * second order dropped.  Stop when |dp| < conv_tol with
 * |dp|^2 = du^2 + dv^2 + M^2 (first derivatives)^2 + (M^2/2)^2 (uxx, uyy,
 * vxx, vyy)^2 + M^4 (uxy, vxy)^2; an update that moves any warped subset
 * point outside [1, W-2) x [1, H-2) is rejected (DIC_POI_OUT_OF_BOUNDS).
 *   p12  device [n_pois][12], row-major, in the order above
 * Other arguments and outputs as dic_subpixel.  DIC_ERR_STATE for a handle of
 * shape order 1 or without a pair; DIC_ERR_UNSUPPORTED for DIC_FANR or
 * bilinear interpolation (the device path is IC-GN over bicubic
 * interpolation); DIC_ERR_ARG for a null pointer. */
dic_status dic_subpixel2(dic_t h, dic_method method, const int32_t *u0, const int32_t *v0,
                         const uint8_t *status0, float *p12, float *zncc, int32_t *iters,
                         uint8_t *status);

/* ---------------------------------------------------------------- batches
 * Many image pairs of uneven size in one go -- the GPU form of the paper's
 * parallelism over whole image pairs (Section 2.3, Table 6). */
typedef struct {
  const uint8_t *ref_dev;  /* device, borrowed (as dic_set_pair)             */
  const uint8_t *def_dev;
  int width, height, pitch_bytes;
  int subset_size;         /* odd 3..63, or <= 0 for the handle's value      */
  int grid_step;           /* >= 1, or <= 0 for the handle's value           */
  int search_radius;       /* >= 0, or < 0 for the handle's value            */
} dic_pair_desc;

/* Outputs of a batch: device arrays of total_pois elements; the POIs of pair
 * k occupy [offsets[k], offsets[k+1]) (see dic_batch_pois), each pair's in
 * its own grid order.  Integer-search outputs and sub-pixel outputs as in
 * dic_integer_search / dic_subpixel. */
typedef struct {
  int32_t *u0, *v0;
  float *zncc0;
  uint8_t *status0;
  float *u, *v, *ux, *uy, *vx, *vy, *zncc;
  int32_t *iters;
  uint8_t *status;
} dic_batch_out;

/* Bind n_pairs pairs (host array of descriptors, copied).  Allocates the
 * precompute scratch of every pair (20 bytes per pixel; DIC_ERR_OOM on
 * failure) and validates every descriptor (DIC_ERR_ARG); a pair that neither
 * search form can run (FP32: the search window must fit shared memory;
 * tensor-core: see dic_set_form) returns DIC_ERR_UNSUPPORTED naming it in
 * dic_last_error.  Replaces any earlier batch. */
dic_status dic_set_pairs(dic_t h, int n_pairs, const dic_pair_desc *descs);

/* Total POIs of the bound batch and, if offsets is not NULL, the host array
 * of n_pairs + 1 prefix offsets. */
dic_status dic_batch_pois(dic_t h, int64_t *total, int64_t *offsets);

/* Run precompute, integer search and sub-pixel refinement of the whole batch
 * as one CUDA graph on the handle's stream: per-pair precompute launches;
 * the integer search in the handle's form (tensor-core: one search per pair
 * on shared scratch, allocated on first use for the largest pair; FP32: one
 * persistent kernel per subset-width class over a work counter); then one
 * persistent sub-pixel kernel whose warps take POIs from a global counter,
 * or per-pair sub-pixel launches overlapping the next searches (see
 * dic_set_batch_shape).  The graph is built on the first call and rebuilt
 * when method, outputs, form or tuning change; later calls only launch it.
 * Requires dic_set_pairs.  DIC_ERR_UNSUPPORTED names a pair the form cannot
 * run, or when bilinear interpolation is set. */
dic_status dic_run_batch(dic_t h, dic_method method, const dic_batch_out *out);

/* Sub-pixel launch shape of later dic_run_batch calls: warps_per_cta 2, 4
 * or 8 with grid_mult 1 or 2 (one persistent kernel over all pairs, grid =
 * grid_mult x resident CTAs), or {0, 0}: per-pair launches on a second
 * stream, each overlapping the searches of the pairs after it (tensor-core
 * form only; dic_run_batch returns DIC_ERR_ARG otherwise).  Use it to
 * re-apply a shape dic_autotune chose earlier.  DIC_ERR_STATE without a
 * batch, DIC_ERR_ARG for any other shape. */
dic_status dic_set_batch_shape(dic_t h, int warps_per_cta, int grid_mult);

/* Time the batch under each candidate launch shape (sub-pixel warps per CTA
 * 2/4/8 x persistent grid 1x/2x the resident CTAs; with the tensor-core
 * search form also per-pair sub-pixel launches, each overlapping the next
 * pairs' searches on a second stream) and keep the fastest for later
 * dic_run_batch calls.  Runs the batch several times (outputs are
 * overwritten).  chosen (may be NULL) receives {warps_per_cta, grid_mult},
 * {0, 0} for the overlapped per-pair launches. */
dic_status dic_autotune(dic_t h, dic_method method, const dic_batch_out *out, int *chosen);

/* ---------------------------------------------------------- frame streams
 * Consecutive-frame processing as the paper evaluates its image series
 * (Sections 3 and 5.1): every new frame is the target of one pair whose
 * reference is the previous frame, so the reference is updated after every
 * evaluation and consecutive frames differ by small displacements.
 *
 * dic_stream_push copies the frame (device pointer; width, height, pitch as
 * in dic_set_pair) into a ring of three slots inside the library and runs
 * its precompute once: the gradient field serves the frame's later turn as
 * reference, the float copy and tap quads its turn as target.  The first
 * push of a sequence (after dic_create or dic_stream_reset) only stores the
 * frame; out may be NULL.  Every later push runs the pair (previous frame,
 * this frame): the integer search in the handle's form on the handle's
 * stream, then the sub-pixel refinement (method; the handle's solve
 * precision, interpolation and tolerances) on a second stream of the
 * library, so that a pair's refinement overlaps the next pair's search.
 *   out       device arrays of n_pois elements each (dic_num_pois after the
 *             first push), as in dic_integer_search / dic_subpixel
 * Ordering: the copy of the frame runs on the handle's stream, so the
 * caller may reuse its frame buffer once that stream has passed this push.
 * A pair's outputs are complete for any work enqueued on the handle's stream
 * after the next push, or after dic_stream_flush; keep each push's out
 * arrays alive and untouched until then.
 * The first push fixes the sequence's frame size (later frames of another
 * size: DIC_ERR_ARG) and the handle's POI grid; it replaces a pair bound by
 * dic_set_pair (bind one again before dic_integer_search / dic_subpixel).
 * Allocates the ring on the first push of a size (3 x (pitch x height + 20
 * bytes per pixel); DIC_ERR_OOM on failure), a stream and four events.
 * DIC_ERR_ARG for a null frame, bad sizes, an unknown method or a null
 * output array of a pair; DIC_ERR_CUDA / DIC_ERR_UNSUPPORTED as the
 * single-pair calls. */
dic_status dic_stream_push(dic_t h, const uint8_t *frame_dev, int width, int height,
                           int pitch_bytes, dic_method method, const dic_batch_out *out);

/* Make the last pushed pair's outputs complete for later work on the
 * handle's stream (an event wait on that stream; no host synchronisation). */
dic_status dic_stream_flush(dic_t h);

/* End the sequence (after a flush): the next push starts a new one. */
dic_status dic_stream_reset(dic_t h);

/* Summed ZNSSD of the subsets at given shapes: for POI k,
 *   L_k = sum_i [ (f_i - fbar)/df - (g(W(xi_i; p_k)) - gbar)/dg ]^2 = 2 - 2 C_k,
 * C_k being Eq. 1 at shape p_k with bicubically interpolated g.
 *   p6            device [n_pois][6] shapes (u, ux, uy, v, vx, vy)
 *   loss_per_poi  device [n_pois] or NULL
 *   loss_total    device scalar (zeroed, then summed into) or NULL
 * A POI whose warped subset leaves [1, W-2) x [1, H-2), or whose reference
 * or target subset is flat, contributes 0. */
dic_status dic_znssd(dic_t h, const float *p6, float *loss_per_poi, float *loss_total);

/* Adjoint of dic_znssd with the shapes held fixed (the gradient does not go
 * through the iterative solver): with upstream weight
 * w_k = scale * (grad_loss ? grad_loss[k] : 1),
 *   dL_ddef  device [height][width] dense, zeroed by the callee, receives
 *            sum_k w_k dL_k/dg through the transposed bicubic stencil
 *   dL_dp    device [n_pois][6] or NULL, receives w_k dL_k/dp_k.
 * Float atomics accumulate dL_ddef, so its summation order is not fixed. */
dic_status dic_backward(dic_t h, const float *p6, const float *grad_loss, float scale,
                        float *dL_ddef, float *dL_dp);

/* ------------------------------------------------------------ measurement
 * Throughput peaks of the units that bound the kernels which have neither a
 * tensor-core nor an HBM roofline, measured on the current device by a
 * microbenchmark (no counterpart in the paper; the benchmark divides the
 * kernels' algorithmic rates by them):
 *   DIC_PEAK_FP32_FMA         FP32 multiply-add throughput, flop/s (2 per FMA),
 *                             the unit of the sub-pixel refinement
 *   DIC_PEAK_SMEM_ATOMIC_F32  shared-memory float atomic adds per second, the
 *                             unit of dic_backward's scatter into its tiles
 * Runs four launches of a few milliseconds on cuda_stream (NULL = default),
 * synchronises, and writes the best of the last three to *rate.  Allocates
 * and frees a small device buffer.  DIC_ERR_ARG for an unknown kind or a
 * null rate; DIC_ERR_CUDA if a launch fails. */
enum { DIC_PEAK_FP32_FMA = 0, DIC_PEAK_SMEM_ATOMIC_F32 = 1 };
dic_status dic_measure_peak(int kind, void *cuda_stream, double *rate);

/* Sub-pixel refinement that allocates no device memory.  The paper has no
 * counterpart; this call exists for callers that must not call cudaMalloc /
 * cudaFree -- e.g. real-time acquisition loops that cannot absorb the device
 * synchronisation those calls imply, or plug-ins whose host application owns
 * the whole device-memory budget through its own allocator.
 *
 * Same arithmetic as dic_set_pair (precompute) followed by dic_subpixel, but
 * without a handle: the precompute output goes to one fixed array inside the
 * library (a static device symbol of 1.25 MiB, held by every GPU that loads
 * the library until the process exits), in three regions of 65536 pixels
 * each: the float deformed image (4 bytes per pixel), the gradient field of
 * the reference (8 bytes per pixel) and the BF16 tap quads of the deformed
 * image (8 bytes per pixel).
 *   - width * height must be <= 65536 pixels (e.g. 256 x 256); larger
 *     images, search_radius > 1000 (as dic_create), and every other invalid
 *     argument return DIC_ERR_ARG before any GPU work is enqueued.  Other
 *     arguments as in dic_create / dic_set_pair / dic_subpixel; ref_dev and
 *     def_dev share width, height and pitch_bytes; solve_bits is 32 or 64;
 *     cuda_stream may be NULL.
 *   - Allocates nothing: no cudaMalloc, no cudaFree, no library allocator.
 *   - Every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress, which allocates nothing); the first call on a
 *     device may load the library's module there, so make it before any
 *     stream capture.  Then the call enqueues two kernels.
 *   - All calls share the one array.  Each call overwrites every entry it
 *     reads, so no clearing is needed, but calls whose work overlaps on the
 *     GPU (different streams, or host threads) race on the array: serialise
 *     them, e.g. on one stream.
 *   - Returns DIC_ERR_CUDA if a launch fails. */
dic_status dic_subpixel_noalloc(const uint8_t *ref_dev, const uint8_t *def_dev, int width,
                                int height, int pitch_bytes, int subset_size, int grid_step,
                                int search_radius, dic_method method, float conv_tol,
                                int max_iter, int solve_bits, const int32_t *u0,
                                const int32_t *v0, const uint8_t *status0, float *u, float *v,
                                float *ux, float *uy, float *vx, float *vy, float *zncc,
                                int32_t *iters, uint8_t *status, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* DIC_GB300_H */
