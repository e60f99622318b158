// dic_noalloc.cu -- sub-pixel refinement that allocates no device memory.
//
// Who needs it: callers that must not call cudaMalloc / cudaFree.  Examples
// are real-time acquisition loops, where cudaFree (and often cudaMalloc)
// synchronises the whole device and stalls other streams, and plug-ins
// inside a host application whose own allocator owns the device memory
// budget, where a stray allocation breaks its accounting.
//
// The regular path keeps the float deformed image, its BF16 tap quads and
// the reference gradient field in scratch that dic_set_pair allocates.  Here
// the same two
// kernels (precompute, then sub-pixel refinement) run on a fixed scratch
// array that lives in this file as a static __device__ symbol.  Every GPU
// that loads the library holds kNoAllocScratchBytes of it until the process
// exits.
#include "dic_internal.cuh"

namespace {

// Largest image (width * height, pixels) this entry point accepts.
constexpr size_t kNoAllocMaxPixels = 256 * 256;
// Float deformed image (one float per pixel), the gradient field (one
// float2 per pixel), then the tap quads of the deformed image (one uint2 per
// pixel): 1.25 MiB.
constexpr size_t kGimgBytes = kNoAllocMaxPixels * sizeof(float);
constexpr size_t kGradBytes = kNoAllocMaxPixels * sizeof(float2);
constexpr size_t kNoAllocScratchBytes = kGimgBytes + kGradBytes + kNoAllocMaxPixels * sizeof(uint2);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the array on the current device.  In host code the
// symbol's name is only a host-side stand-in, so the address has to come
// from the runtime.  It is looked up on every call (the lookup allocates
// nothing), so a module reloaded after a device reset is found again.
cudaError_t scratch_on_current_device(unsigned char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<unsigned char*>(p);
  return cudaSuccess;
}

}  // namespace

extern "C" dic_status dic_subpixel_noalloc(
    const uint8_t* ref_dev, const uint8_t* def_dev, int width, int height, int pitch_bytes,
    int subset_size, int grid_step, int search_radius, dic_method method, float conv_tol,
    int max_iter, int solve_bits, const int32_t* u0, const int32_t* v0, const uint8_t* status0,
    float* u, float* v, float* ux, float* uy, float* vx, float* vy, float* zncc,
    int32_t* iters, uint8_t* status, void* cuda_stream) {
  if (!ref_dev || !def_dev || width < 4 || height < 4 || pitch_bytes < width)
    return DIC_ERR_ARG;
  if ((size_t)width * (size_t)height > kNoAllocMaxPixels) return DIC_ERR_ARG;
  if (subset_size < 3 || subset_size > dic::kMaxSubset || (subset_size & 1) == 0 ||
      grid_step < 1 || search_radius < 0 || search_radius > 1000 || !(conv_tol > 0.f) ||
      max_iter < 1)
    return DIC_ERR_ARG;
  if (method != DIC_ICGN && method != DIC_FANR) return DIC_ERR_ARG;
  if (solve_bits != 32 && solve_bits != 64) return DIC_ERR_ARG;
  // the margin B = M + R + 2 in 64 bits (R <= 1000 keeps it small; the
  // grid is empty unless 2B < width and 2B < height)
  const int M = subset_size / 2;
  const int64_t B = (int64_t)M + search_radius + 2;
  const int64_t ax = (int64_t)width - 1 - 2 * B, ay = (int64_t)height - 1 - 2 * B;
  const int nx = ax >= 0 ? (int)(ax / grid_step + 1) : 0;
  const int ny = ay >= 0 ? (int)(ay / grid_step + 1) : 0;
  if ((int64_t)nx * ny == 0) return DIC_OK;
  if (!u0 || !v0 || !status0 || !u || !v || !ux || !uy || !vx || !vy || !zncc || !iters ||
      !status)
    return DIC_ERR_ARG;

  unsigned char* scratch = nullptr;
  if (scratch_on_current_device(&scratch) != cudaSuccess) return DIC_ERR_CUDA;
  float* gimg = reinterpret_cast<float*>(scratch);
  float2* grad = reinterpret_cast<float2*>(scratch + kGimgBytes);
  uint2* gq = reinterpret_cast<uint2*>(scratch + kGimgBytes + kGradBytes);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

  // The precompute kernel writes every float pixel, gradient and tap quad of
  // the width x height image (zeros on the border), so nothing left over
  // from an earlier call is ever read and no clearing is needed.
  if (dic::launch_precompute(ref_dev, def_dev, width, height, pitch_bytes, grad, gimg, gq,
                             st) != cudaSuccess)
    return DIC_ERR_CUDA;

  dic::SubpixelParams p;
  p.ref = ref_dev;
  p.grad = grad;
  p.gimg = gimg;
  p.gq = gq;
  p.W = width;
  p.H = height;
  p.pitch = pitch_bytes;
  p.S = subset_size;
  p.M = M;
  p.R = search_radius;
  p.step = grid_step;
  p.nx = nx;
  p.n_pois = (int64_t)nx * ny;
  p.max_iter = max_iter;
  p.tol = conv_tol;
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
  if (dic::launch_subpixel(p, (int)method, solve_bits == 64, st) != cudaSuccess)
    return DIC_ERR_CUDA;
  return DIC_OK;
}
