// The optional FP64 correction step: one time step of the stencil (Sec. 2.2) computed on the
// CUDA cores with FP64 sums, between the tensor-core sweeps of a run (every k-th step when a
// plan enables it).  Each output is the FP64 sum over the nonzero weights, in (dz, dy, dx)
// order, of weight x input, rounded once to FP32.
#include <cuda_runtime.h>

#include "correction.h"

namespace spst {

namespace {

__device__ __forceinline__ int64_t wrap(int64_t v, int64_t n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// A thread per destination cell (x fastest), grid-stride.
__global__ void __launch_bounds__(256) fp64_step_kernel(const __grid_constant__ Fp64StepParams p,
                                                      const float* __restrict__ src, float* __restrict__ dst_padded,
                                                      float* __restrict__ dst_unpadded) {
  asm volatile("griddepcontrol.launch_dependents;");
  const int64_t G = p.G;
  const bool out_padded = dst_unpadded == nullptr;
  // the destination box: padded extents, or the true ones for an unpadded result
  const int64_t ex = out_padded ? p.W + 2 * G : p.W;
  const int64_t ey = p.ndim >= 2 ? (out_padded ? p.H + 2 * G : p.H) : 1;
  const int64_t ez = p.ndim == 3 ? (out_padded ? p.D + 2 * G : p.D) : 1;
  const int64_t shift = out_padded ? G : 0;  // destination index minus true coordinate
  const int64_t n = ex * ey * ez;
  const int64_t plane = p.Hp * p.Wp;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t xd = i % ex, yd = (i / ex) % ey, zd = i / (ex * ey);
    // the interior position this cell takes its value from
    int64_t x = xd - shift, y = p.ndim >= 2 ? yd - shift : 0, z = p.ndim == 3 ? zd - shift : 0;
    bool inside = x >= 0 && x < p.W && y >= 0 && y < p.H && z >= 0 && z < p.D;
    if (!inside && p.periodic) {
      x = wrap(x, p.W);
      y = wrap(y, p.H);
      z = wrap(z, p.D);
      inside = true;
    }
    double s = 0.0;
    if (inside) {
      // the source's ghost cells hold the images (or zeros) of every neighbour within G
      const float* c = src + (p.ndim == 3 ? (z + G) * plane : 0) + (p.ndim >= 2 ? (y + G) * p.Wp : 0) + (x + G);
      for (int k = 0; k < p.npts; k++)
        s = fma(p.w[k], (double)c[p.off[k][0] * plane + p.off[k][1] * p.Wp + p.off[k][2]], s);
    }
    if (out_padded) {
      dst_padded[(p.ndim == 3 ? zd * plane : 0) + (p.ndim >= 2 ? yd * p.Wp : 0) + xd] = (float)s;
    } else {
      dst_unpadded[i] = (float)s;
    }
  }
}

}  // namespace

cudaError_t launch_fp64_step(const Fp64StepParams& p, const float* src, float* dst_padded, float* dst_unpadded,
                             cudaStream_t stream) {
  if (p.G < 1 || p.npts < 1 || p.npts > 343 || (!dst_padded && !dst_unpadded)) return cudaErrorInvalidValue;
  const int64_t ex = p.W + 2 * p.G, ey = p.ndim >= 2 ? p.H + 2 * p.G : 1, ez = p.ndim == 3 ? p.D + 2 * p.G : 1;
  const int64_t n = ex * ey * ez;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  fp64_step_kernel<<<(unsigned)blocks, 256, 0, stream>>>(p, src, dst_padded, dst_unpadded);
  return cudaGetLastError();
}

}  // namespace spst
