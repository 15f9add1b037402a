// Support kernels: padded-grid copy-in, the plain FP32 CUDA-core direct stencil (the
// comparator of the tensor-core path), FP64 error norms, and the device status word.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace spst {

namespace {

__device__ int g_status_word;
__device__ double g_norm_acc[4];

// ---------------------------------------------------------------------------------------
// Copy-in: unpadded H x W -> padded (H + 2G) x Wp.  Ghost cells hold the periodic images
// (periodic) or zeros (Dirichlet); columns beyond W + 2G are zero.
// ---------------------------------------------------------------------------------------
__global__ void pad_copy2d_kernel(const float* __restrict__ in, float* __restrict__ out, int H, int W, int G,
                                  int64_t Wp, int periodic) {
  const int64_t Hp = (int64_t)H + 2 * G;
  const int64_t total = Hp * Wp;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t yp = i / Wp, xp = i % Wp;
    int64_t y = yp - G, x = xp - G;
    float v = 0.f;
    if (xp < (int64_t)W + 2 * G) {
      if (periodic) {
        y = y < 0 ? y + H : (y >= H ? y - H : y);
        x = x < 0 ? x + W : (x >= W ? x - W : x);
        v = in[y * W + x];
      } else if (y >= 0 && y < H && x >= 0 && x < W) {
        v = in[y * W + x];
      }
    }
    out[i] = v;
  }
}

// ---------------------------------------------------------------------------------------
// Plain FP32 direct stencil: each CTA stages a (TY + 2r) x (TX + 2r) [x (TZ + 2r)] input
// tile in shared memory (coalesced loads, boundary rule applied on load) and each thread
// computes outputs with FP32 FMAs in fixed offset order.  One time step per launch.
// ---------------------------------------------------------------------------------------
constexpr int DTX = 64, DTY = 16;

__global__ void direct2d_kernel(const __grid_constant__ DirectParams p, const float* __restrict__ in,
                                float* __restrict__ out) {
  extern __shared__ float tile[];
  const int r = p.radius;
  const int tw = DTX + 2 * r, th = DTY + 2 * r;
  const int64_t H = p.H, W = p.W;
  const int64_t x0 = (int64_t)blockIdx.x * DTX, y0 = (int64_t)blockIdx.y * DTY;
  for (int i = threadIdx.x; i < tw * th; i += blockDim.x) {
    const int ty = i / tw, tx = i % tw;
    int64_t y = y0 + ty - r, x = x0 + tx - r;
    float v = 0.f;
    if (p.periodic) {
      y = y < 0 ? y + H : (y >= H ? y - H : y);
      x = x < 0 ? x + W : (x >= W ? x - W : x);
      v = in[y * W + x];
    } else if (y >= 0 && y < H && x >= 0 && x < W) {
      v = in[y * W + x];
    }
    tile[i] = v;
  }
  __syncthreads();
  const int npts = p.npts;
  for (int i = threadIdx.x; i < DTX * DTY; i += blockDim.x) {
    const int ly = i / DTX, lx = i % DTX;
    const int64_t y = y0 + ly, x = x0 + lx;
    if (y >= H || x >= W) continue;
    float acc = 0.f;
    for (int q = 0; q < npts; q++) acc = fmaf(p.w[q], tile[(ly + r + p.off[q][1]) * tw + (lx + r + p.off[q][2])], acc);
    out[y * W + x] = acc;
  }
}

constexpr int D3X = 32, D3Y = 8, D3Z = 4;

__global__ void direct3d_kernel(const __grid_constant__ DirectParams p, const float* __restrict__ in,
                                float* __restrict__ out) {
  extern __shared__ float tile[];
  const int r = p.radius;
  const int tw = D3X + 2 * r, th = D3Y + 2 * r, td = D3Z + 2 * r;
  const int64_t D = p.D, H = p.H, W = p.W;
  const int64_t x0 = (int64_t)blockIdx.x * D3X, y0 = (int64_t)blockIdx.y * D3Y, z0 = (int64_t)blockIdx.z * D3Z;
  for (int i = threadIdx.x; i < tw * th * td; i += blockDim.x) {
    const int tz = i / (tw * th), ty = (i / tw) % th, tx = i % tw;
    int64_t z = z0 + tz - r, y = y0 + ty - r, x = x0 + tx - r;
    float v = 0.f;
    if (p.periodic) {
      z = z < 0 ? z + D : (z >= D ? z - D : z);
      y = y < 0 ? y + H : (y >= H ? y - H : y);
      x = x < 0 ? x + W : (x >= W ? x - W : x);
      v = in[(z * H + y) * W + x];
    } else if (z >= 0 && z < D && y >= 0 && y < H && x >= 0 && x < W) {
      v = in[(z * H + y) * W + x];
    }
    tile[i] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < D3X * D3Y * D3Z; i += blockDim.x) {
    const int lz = i / (D3X * D3Y), ly = (i / D3X) % D3Y, lx = i % D3X;
    const int64_t z = z0 + lz, y = y0 + ly, x = x0 + lx;
    if (z >= D || y >= H || x >= W) continue;
    float acc = 0.f;
    for (int q = 0; q < p.npts; q++)
      acc = fmaf(p.w[q], tile[((lz + r + p.off[q][0]) * th + (ly + r + p.off[q][1])) * tw + (lx + r + p.off[q][2])],
                 acc);
    out[(z * H + y) * W + x] = acc;
  }
}

// ---------------------------------------------------------------------------------------
// FP64 norms: sum (x-ref)^2, sum ref^2, max |x-ref|, max |ref| (non-negative doubles compare
// like their bit patterns, so the maxima use 64-bit integer atomicMax).
// ---------------------------------------------------------------------------------------
__global__ void norms_kernel(const float* __restrict__ x, const float* __restrict__ ref, int64_t n,
                             double* __restrict__ acc) {
  double s0 = 0.0, s1 = 0.0, m0 = 0.0, m1 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = (double)x[i], b = (double)ref[i];
    const double d = a - b;
    s0 += d * d;
    s1 += b * b;
    m0 = fmax(m0, fabs(d));
    m1 = fmax(m1, fabs(b));
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
    m0 = fmax(m0, __shfl_down_sync(0xffffffffu, m0, o));
    m1 = fmax(m1, __shfl_down_sync(0xffffffffu, m1, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[0], s0);
    atomicAdd(&acc[1], s1);
    atomicMax((unsigned long long*)&acc[2], (unsigned long long)__double_as_longlong(m0));
    atomicMax((unsigned long long*)&acc[3], (unsigned long long)__double_as_longlong(m1));
  }
}

}  // namespace

cudaError_t launch_pad_copy2d(const float* in, float* padded, int H, int W, int G, int64_t Wp, int periodic,
                              cudaStream_t stream) {
  const int64_t total = ((int64_t)H + 2 * G) * Wp;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  pad_copy2d_kernel<<<(unsigned)blocks, 256, 0, stream>>>(in, padded, H, W, G, Wp, periodic);
  return cudaGetLastError();
}

cudaError_t launch_direct_step(const DirectParams& p, const float* in, float* out, cudaStream_t stream) {
  const int r = p.radius;
  if (p.ndim == 2) {
    dim3 grid((unsigned)((p.W + DTX - 1) / DTX), (unsigned)((p.H + DTY - 1) / DTY));
    size_t smem = (size_t)(DTX + 2 * r) * (DTY + 2 * r) * sizeof(float);
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(direct2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    direct2d_kernel<<<grid, 256, smem, stream>>>(p, in, out);
  } else {
    dim3 grid((unsigned)((p.W + D3X - 1) / D3X), (unsigned)((p.H + D3Y - 1) / D3Y), (unsigned)((p.D + D3Z - 1) / D3Z));
    size_t smem = (size_t)(D3X + 2 * r) * (D3Y + 2 * r) * (D3Z + 2 * r) * sizeof(float);
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(direct3d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    direct3d_kernel<<<grid, 256, smem, stream>>>(p, in, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_error_norms(const float* x, const float* ref, int64_t n, double* acc, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(acc, 0, 4 * sizeof(double), stream);
  if (e != cudaSuccess) return e;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  norms_kernel<<<(unsigned)blocks, 256, 0, stream>>>(x, ref, n, acc);
  return cudaGetLastError();
}

double* device_norm_accumulator() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_norm_acc) != cudaSuccess) return nullptr;
  return (double*)p;
}

int* device_status_word() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) return nullptr;
  return (int*)p;
}

}  // namespace spst
