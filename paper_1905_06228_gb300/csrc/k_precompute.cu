// k_precompute.cu -- reference gradients and the float deformed image.
//
// IC-GN (Section 2.2) needs the reference-image gradients at integer pixels;
// both sub-pixel methods interpolate the deformed image bicubically.  This
// kernel produces, in one pass over HBM:
//
//  grad[y*W + x] = ( (f[x+1]-f[x-1])/2 , (f[y+1]-f[y-1])/2 )  for interior
//                  pixels, 0 on the one-pixel border.  Central differences
//                  equal the derivative of the Keys (a = -1/2) interpolant at
//                  the nodes, so IC-GN's steepest-descent images are
//                  consistent with the interpolation used for g.
//  gimg[y*W + x] = g[y][x] as float (dense, unpadded), the samples the
//                  bicubic evaluation reads.
//  gq[y*W + x]   = (8-bit pairs, if gq is given) the four horizontal taps
//                  g[y][x-1 .. x+2] of a bicubic stencil whose cell starts
//                  at column x, as BF16 (exact for 8-bit values; 0 outside
//                  the image), 8 bytes: one load per stencil row instead of
//                  four.
//
// The paper keeps interpolation results in look-up tables; here the bicubic
// weights are evaluated per sample instead (a table of 16 coefficients per
// pixel is 64 B/px, too large to stay in L1 for the subsets resident on an
// SM, while 4 B/px does).
//
// Pixels are 8-bit or float (the float form serves differentiation with
// respect to real-valued deformed-image pixels); pitch is in elements.
// Bytes per pixel: 1 (f) + 1 (g) read, 8 (grad) + 4 (gimg) (+ 8 (gq))
// written.
#include "dic_internal.cuh"

namespace dic {
namespace {

constexpr int TX = 32;  // tile width (pixels) = threads in x
constexpr int TY = 16;  // tile height (pixels)
constexpr int BY = 8;   // threads in y; each thread does TY/BY rows

// BF16 bits of an 8-bit value (its FP32 encoding has 16 trailing zero bits).
__device__ __forceinline__ uint32_t bf16_of_byte(uint32_t b) {
  return __float_as_uint((float)b) >> 16;
}

template <typename T>
__global__ void __launch_bounds__(TX* BY)
precompute_kernel(const T* __restrict__ ref, const T* __restrict__ def, int W,
                  int H, int pitch, float2* __restrict__ grad, float* __restrict__ gimg,
                  uint2* __restrict__ gq) {
  __shared__ float sf[TY + 2][TX + 3];  // f rows y0-1 .. y0+TY,   cols x0-1 .. x0+TX
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int tid = threadIdx.y * TX + threadIdx.x;
  for (int i = tid; i < (TY + 2) * (TX + 2); i += TX * BY) {
    int r = i / (TX + 2), c = i % (TX + 2);
    int y = y0 - 1 + r, x = x0 - 1 + c;
    sf[r][c] = (x >= 0 && x < W && y >= 0 && y < H) ? (float)ref[(size_t)y * pitch + x] : 0.f;
  }
  __syncthreads();
  const int x = x0 + threadIdx.x;
  if (x >= W) return;
#pragma unroll
  for (int j = 0; j < TY / BY; ++j) {
    const int ly = threadIdx.y + j * BY;
    const int y = y0 + ly;
    if (y >= H) break;
    const int lx = threadIdx.x;
    float2 gr = make_float2(0.f, 0.f);
    if (x >= 1 && x <= W - 2 && y >= 1 && y <= H - 2) {
      gr.x = 0.5f * (sf[ly + 1][lx + 2] - sf[ly + 1][lx]);
      gr.y = 0.5f * (sf[ly + 2][lx + 1] - sf[ly][lx + 1]);
    }
    grad[(size_t)y * W + x] = gr;
    gimg[(size_t)y * W + x] = (float)def[(size_t)y * pitch + x];
    if (gq) {
      const T* row = def + (size_t)y * pitch;
      uint32_t h[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int xx = x - 1 + k;
        h[k] = (xx >= 0 && xx < W) ? bf16_of_byte((uint32_t)row[xx]) : 0u;
      }
      gq[(size_t)y * W + x] = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
    }
  }
}

}  // namespace

cudaError_t launch_precompute(const uint8_t* ref, const uint8_t* def, int W, int H, int pitch,
                              float2* grad, float* gimg, uint2* gq, cudaStream_t st) {
  dim3 block(TX, BY);
  dim3 grid((W + TX - 1) / TX, (H + TY - 1) / TY);
  precompute_kernel<uint8_t><<<grid, block, 0, st>>>(ref, def, W, H, pitch, grad, gimg, gq);
  return cudaGetLastError();
}

cudaError_t launch_precompute_f32(const float* ref, const float* def, int W, int H, int pitch,
                                  float2* grad, float* gimg, cudaStream_t st) {
  dim3 block(TX, BY);
  dim3 grid((W + TX - 1) / TX, (H + TY - 1) / TY);
  precompute_kernel<float><<<grid, block, 0, st>>>(ref, def, W, H, pitch, grad, gimg, nullptr);
  return cudaGetLastError();
}

}  // namespace dic
