// k_precompute.cu -- reference gradients and bicubic coefficient table.
//
// Section 2.2 of the paper interpolates the deformed image bicubically and
// (through its ref. [18]) stores results needed many times in look-up
// tables; IC-GN needs the reference-image gradients at integer pixels.  This
// kernel produces both in one pass over HBM:
//
//  grad[y*W + x] = ( (f[x+1]-f[x-1])/2 , (f[y+1]-f[y-1])/2 )  for interior
//                  pixels, 0 on the one-pixel border.  Central differences
//                  equal the derivative of the Keys (a = -1/2) interpolant at
//                  the nodes, so IC-GN's steepest-descent images are
//                  consistent with the interpolation used for g.
//  lut[(n*H + y)*W + x] = (A[n][0], A[n][1], A[n][2], A[n][3]), the
//                  coefficients of g(x+tx, y+ty) = sum_{n,m} A[n][m] ty^n tx^m
//                  on the cell [x, x+1) x [y, y+1), with A = K P K^T, P the
//                  4x4 pixels g[y-1..y+2][x-1..x+2] and K the power basis of
//                  the Keys a = -1/2 weights; valid cells 1 <= x <= W-3,
//                  1 <= y <= H-3, zero elsewhere.
//
// Pixels are 8-bit or float (the float form serves differentiation with
// respect to real-valued deformed-image pixels); pitch is in elements.
//
// Bytes per pixel: 1 (f) + 1 (g) read, 8 (grad) + 64 (lut) written.  Each
// warp writes 32 consecutive float4 of one plane per store (512 B), so every
// store is a full-line coalesced write; the sub-pixel kernels read the
// planes the same way (lanes interpolate consecutive pixels).
#include "dic_internal.cuh"

namespace dic {
namespace {

constexpr int TX = 32;  // tile width (pixels) = threads in x
constexpr int TY = 16;  // tile height (pixels)
constexpr int BY = 8;   // threads in y; each thread does TY/BY rows

// Power-basis matrix of the Keys a = -1/2 weights: w_k(t) = sum_m K[m][k] t^m
// for the taps k = -1, 0, 1, 2 (columns).
__device__ __forceinline__ void keys_basis(float K[4][4]) {
  K[0][0] = 0.f;   K[0][1] = 1.f;   K[0][2] = 0.f;   K[0][3] = 0.f;
  K[1][0] = -0.5f; K[1][1] = 0.f;   K[1][2] = 0.5f;  K[1][3] = 0.f;
  K[2][0] = 1.f;   K[2][1] = -2.5f; K[2][2] = 2.f;   K[2][3] = -0.5f;
  K[3][0] = -0.5f; K[3][1] = 1.5f;  K[3][2] = -1.5f; K[3][3] = 0.5f;
}

template <typename T>
__global__ void __launch_bounds__(TX* BY)
precompute_kernel(const T* __restrict__ ref, const T* __restrict__ def, int W,
                  int H, int pitch, float2* __restrict__ grad, float4* __restrict__ lut) {
  __shared__ float sg[TY + 3][TX + 4];  // g rows y0-1 .. y0+TY+1, cols x0-1 .. x0+TX+2
  __shared__ float sf[TY + 2][TX + 3];  // f rows y0-1 .. y0+TY,   cols x0-1 .. x0+TX
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int tid = threadIdx.y * TX + threadIdx.x;
  for (int i = tid; i < (TY + 3) * (TX + 3); i += TX * BY) {
    int r = i / (TX + 3), c = i % (TX + 3);
    int y = y0 - 1 + r, x = x0 - 1 + c;
    sg[r][c] = (x >= 0 && x < W && y >= 0 && y < H) ? (float)def[(size_t)y * pitch + x] : 0.f;
  }
  for (int i = tid; i < (TY + 2) * (TX + 2); i += TX * BY) {
    int r = i / (TX + 2), c = i % (TX + 2);
    int y = y0 - 1 + r, x = x0 - 1 + c;
    sf[r][c] = (x >= 0 && x < W && y >= 0 && y < H) ? (float)ref[(size_t)y * pitch + x] : 0.f;
  }
  __syncthreads();
  float K[4][4];
  keys_basis(K);
  const int x = x0 + threadIdx.x;
  if (x >= W) return;
  const size_t plane = (size_t)W * H;
#pragma unroll
  for (int j = 0; j < TY / BY; ++j) {
    const int ly = threadIdx.y + j * BY;
    const int y = y0 + ly;
    if (y >= H) break;
    const int lx = threadIdx.x;
    // gradients of f
    float2 gr = make_float2(0.f, 0.f);
    if (x >= 1 && x <= W - 2 && y >= 1 && y <= H - 2) {
      gr.x = 0.5f * (sf[ly + 1][lx + 2] - sf[ly + 1][lx]);
      gr.y = 0.5f * (sf[ly + 2][lx + 1] - sf[ly][lx + 1]);
    }
    grad[(size_t)y * W + x] = gr;
    // bicubic coefficients of g on cell (x, y)
    float A[4][4];
    if (x >= 1 && x <= W - 3 && y >= 1 && y <= H - 3) {
      // T[l][m] = sum_k P[l][k] K[m][k]   (P rows l = y-1..y+2)
      float T[4][4];
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const float p0 = sg[ly + l][lx], p1 = sg[ly + l][lx + 1], p2 = sg[ly + l][lx + 2],
                    p3 = sg[ly + l][lx + 3];
#pragma unroll
        for (int m = 0; m < 4; ++m) T[l][m] = p0 * K[m][0] + p1 * K[m][1] + p2 * K[m][2] + p3 * K[m][3];
      }
#pragma unroll
      for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int m = 0; m < 4; ++m)
          A[n][m] = K[n][0] * T[0][m] + K[n][1] * T[1][m] + K[n][2] * T[2][m] + K[n][3] * T[3][m];
    } else {
#pragma unroll
      for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int m = 0; m < 4; ++m) A[n][m] = 0.f;
    }
#pragma unroll
    for (int n = 0; n < 4; ++n)
      lut[n * plane + (size_t)y * W + x] = make_float4(A[n][0], A[n][1], A[n][2], A[n][3]);
  }
}

}  // namespace

cudaError_t launch_precompute(const uint8_t* ref, const uint8_t* def, int W, int H, int pitch,
                              float2* grad, float4* lut, cudaStream_t st) {
  dim3 block(TX, BY);
  dim3 grid((W + TX - 1) / TX, (H + TY - 1) / TY);
  precompute_kernel<uint8_t><<<grid, block, 0, st>>>(ref, def, W, H, pitch, grad, lut);
  return cudaGetLastError();
}

cudaError_t launch_precompute_f32(const float* ref, const float* def, int W, int H, int pitch,
                                  float2* grad, float4* lut, cudaStream_t st) {
  dim3 block(TX, BY);
  dim3 grid((W + TX - 1) / TX, (H + TY - 1) / TY);
  precompute_kernel<float><<<grid, block, 0, st>>>(ref, def, W, H, pitch, grad, lut);
  return cudaGetLastError();
}

}  // namespace dic
