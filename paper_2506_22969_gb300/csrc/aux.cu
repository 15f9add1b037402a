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
// Largest |v| seen by the calling warp's threads, folded into *maxabs (non-negative floats
// order like their bit patterns).
__device__ __forceinline__ void fold_maxabs(unsigned* maxabs, float m) {
  if (!maxabs) return;
  const unsigned b = __reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(m)));
  if ((threadIdx.x & 31) == 0) atomicMax(maxabs, b);
}

// One padded row dst[0, Wp) from source row src[0, W) with G ghost cells each side (wrapped
// images, or zeros when not periodic or when the row itself lies outside: inside = false),
// zeros past W + 2G; the block's threads take four elements each per step (independent
// loads in flight), and *m collects max |value|.
__device__ __forceinline__ void copy_padded_row(const float* __restrict__ src, float* __restrict__ dst, int64_t W,
                                                int G, int64_t Wp, int periodic, bool inside, float* m) {
  const int64_t step = 4 * (int64_t)blockDim.x;
  for (int64_t x0 = threadIdx.x; x0 < Wp; x0 += step) {
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int64_t xp = x0 + k * (int64_t)blockDim.x;
      int64_t x = xp - G;
      v[k] = 0.f;
      if (xp < W + 2 * G) {
        if (periodic) {
          x = x < 0 ? x + W : (x >= W ? x - W : x);
          v[k] = src[x];
        } else if (inside && x >= 0 && x < W) {
          v[k] = src[x];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int64_t xp = x0 + k * (int64_t)blockDim.x;
      if (xp < Wp) {
        dst[xp] = v[k];
        *m = fmaxf(*m, fabsf(v[k]));
      }
    }
  }
}

// Lets the next sweep (launched with programmatic stream serialization) start its set-up
// while this kernel runs; the sweep reads the grids only after its griddepcontrol.wait,
// which waits for this kernel to complete and its writes to be visible.
__device__ __forceinline__ void allow_next_sweep() { asm volatile("griddepcontrol.launch_dependents;"); }

__global__ void pad_copy2d_kernel(const float* __restrict__ in, float* __restrict__ out, int H, int W, int G,
                                  int64_t Wp, int periodic, unsigned* maxabs) {
  allow_next_sweep();
  // a CTA per padded row (grid-stride over rows), its threads along x
  const int64_t Hp = (int64_t)H + 2 * G;
  float m = 0.f;
  for (int64_t yp = blockIdx.x; yp < Hp; yp += gridDim.x) {
    int64_t y = yp - G;
    bool inside = true;
    if (periodic)
      y = y < 0 ? y + H : (y >= H ? y - H : y);
    else
      inside = y >= 0 && y < H;
    const float* src = in + (inside ? y * W : 0);
    float* dst = out + yp * Wp;
    copy_padded_row(src, dst, W, G, Wp, periodic, inside, &m);
  }
  fold_maxabs(maxabs, m);
}

__global__ void pad_copy1d_kernel(const float* __restrict__ in, float* __restrict__ out, int64_t W, int G,
                                  int64_t Wp, int periodic, unsigned* maxabs) {
  allow_next_sweep();
  // block b copies segment [b * 1024, (b + 1) * 1024) of the padded line (grid-stride)
  float m = 0.f;
  constexpr int64_t kSeg = 1024;
  for (int64_t s0 = (int64_t)blockIdx.x * kSeg; s0 < Wp; s0 += (int64_t)gridDim.x * kSeg) {
    const int64_t n = Wp - s0 < kSeg ? Wp - s0 : kSeg;
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int64_t xp = s0 + threadIdx.x + k * (int64_t)blockDim.x;
      int64_t x = xp - G;
      v[k] = 0.f;
      if (xp < s0 + n && xp < W + 2 * G) {
        if (periodic) {
          x = x < 0 ? x + W : (x >= W ? x - W : x);
          v[k] = in[x];
        } else if (x >= 0 && x < W) {
          v[k] = in[x];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int64_t xp = s0 + threadIdx.x + k * (int64_t)blockDim.x;
      if (xp < s0 + n) {
        out[xp] = v[k];
        m = fmaxf(m, fabsf(v[k]));
      }
    }
  }
  fold_maxabs(maxabs, m);
}

// Periodic 1D ghosts: cell i < G holds x = i - G, the image of x + W; cell W + G + i holds
// x = W + i, the image of i.
__global__ void ghost_refresh1d_kernel(float* line, int64_t W, int G) {
  allow_next_sweep();
  for (int i = threadIdx.x; i < G; i += blockDim.x) {
    line[i] = line[i + W];
    line[W + G + i] = line[G + i];
  }
}

// ---------------------------------------------------------------------------------------
// Plain FP32 direct stencil: each CTA stages a (TY + 2r) x (TX + 2r) [x (TZ + 2r)] input
// tile in shared memory (coalesced loads, boundary rule applied on load) and each thread
// computes outputs with FP32 FMAs in fixed offset order.  One time step per launch.
// ---------------------------------------------------------------------------------------
// 2D: a CTA covers 128 x 32 outputs with 256 threads; thread (column cx, half ch) computes
// the 16 outputs of column cx in rows 16ch .. 16ch+15.  It walks the 16 + 2R input rows of
// its strip once, loading each row's 2R+1 horizontal neighbours from shared memory, and adds
// each loaded value into every output row that uses it, in the fixed offset order (dy, dx)
// lexicographic per output (weights live in registers).
constexpr int DTX = 128, DTY = 32, DSTRIP = 16;

template <int R>
__global__ void __launch_bounds__(256) direct2d_kernel(const __grid_constant__ DirectParams p,
                                                       const float* __restrict__ in, float* __restrict__ out) {
  extern __shared__ float tile[];
  constexpr int K = 2 * R + 1;
  constexpr int TW = DTX + 2 * R, TH = DTY + 2 * R;
  const int64_t H = p.H, W = p.W;
  const int64_t x0 = (int64_t)blockIdx.x * DTX, y0 = (int64_t)blockIdx.y * DTY;
  for (int i = threadIdx.x; i < TW * TH; i += blockDim.x) {
    const int ty = i / TW, tx = i % TW;
    int64_t y = y0 + ty - R, x = x0 + tx - R;
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
  float w[K][K];
#pragma unroll
  for (int a = 0; a < K; a++)
#pragma unroll
    for (int b = 0; b < K; b++) w[a][b] = p.wdense[a * K + b];
  __syncthreads();
  const int cx = threadIdx.x % DTX, ch = threadIdx.x / DTX;
  float acc[DSTRIP];
#pragma unroll
  for (int k = 0; k < DSTRIP; k++) acc[k] = 0.f;
  // input row r (strip-relative, 0 .. DSTRIP+2R-1) feeds output k through weight row dy = r - k
#pragma unroll
  for (int dy = 0; dy < K; dy++) {
#pragma unroll
    for (int k = 0; k < DSTRIP; k++) {
      const float* row = tile + (ch * DSTRIP + k + dy) * TW + cx;
#pragma unroll
      for (int dx = 0; dx < K; dx++) acc[k] = fmaf(w[dy][dx], row[dx], acc[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < DSTRIP; k++) {
    const int64_t y = y0 + ch * DSTRIP + k, x = x0 + cx;
    if (y < H && x < W) out[y * W + x] = acc[k];
  }
}

// ---------------------------------------------------------------------------------------
// Register-marching comparators for grids whose width is a multiple of 4 (every float4 row
// access aligned).  A warp owns 128 consecutive columns (a float4 per lane) and walks the
// input rows (2D) or planes (3D, radius 1) of its segment once, in order.  Each input row's
// 4 + 2R values per lane (its float4; R halo values from each neighbouring lane by shuffle,
// or from global memory at the warp's edges) are added into the 2R+1 outputs that use them,
// which wait in registers; an output is stored (float4) once its last input has been added.
// Per output the FMAs run in lexicographic offset order ((dy, dx) in 2D, (dz, dy, dx) in
// 3D), zero weights of the dense cube included (an FMA with weight 0 leaves a finite sum
// unchanged); the weights are operands from the kernel's constant parameters.
// ---------------------------------------------------------------------------------------
constexpr int DSEG = 64;   // 2D: most output rows per warp (fewer when the grid has few columns)
constexpr int D3SEG = 32;  // 3D: output planes per warp
constexpr int DWARPS = 4;  // warps per CTA

__device__ __forceinline__ float f4c(const float4& v, int j) { return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w; }

// One input row's loads for a lane: its float4 at columns x .. x+3 and, at the warp's edges,
// the R halo columns on each side that no neighbouring lane holds (zeros for a row of zeros:
// row null).
template <int R>
struct RowLoad {
  float4 v;
  float hl[R], hr[R];  // columns x-R .. x-1 and x+4 .. x+3+R
};
template <int R>
__device__ __forceinline__ RowLoad<R> load_row(const float* __restrict__ row, int64_t x, bool active, bool left_shfl,
                                               bool right_shfl, int64_t xl, int64_t xr) {
  RowLoad<R> r;
  r.v = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 hl = r.v, hr = r.v;
  if (row && active) {
    r.v = *reinterpret_cast<const float4*>(row + x);
    if (!left_shfl && xl >= 0) hl = *reinterpret_cast<const float4*>(row + xl);
    if (!right_shfl && xr >= 0) hr = *reinterpret_cast<const float4*>(row + xr);
  }
#pragma unroll
  for (int m = 0; m < R; m++) {
    r.hl[m] = f4c(hl, 4 - R + m);
    r.hr[m] = f4c(hr, m);
  }
  return r;
}

// The 4 + 2R values of one input row around the lane's four columns x .. x+3 (s[R + j] is
// column x + j, j = -R .. 3 + R): the lane's own float4, R halo values from each neighbouring
// lane by shuffle, or the edge values loaded by load_row.
template <int R>
__device__ __forceinline__ void row_values(const RowLoad<R>& r, bool left_shfl, bool right_shfl,
                                           float (&s)[4 + 2 * R]) {
#pragma unroll
  for (int j = 0; j < 4; j++) s[R + j] = f4c(r.v, j);
#pragma unroll
  for (int m = 0; m < R; m++) {
    const float up = __shfl_up_sync(0xffffffffu, f4c(r.v, 4 - R + m), 1);
    const float dn = __shfl_down_sync(0xffffffffu, f4c(r.v, m), 1);
    s[m] = left_shfl ? up : r.hl[m];
    s[R + 4 + m] = right_shfl ? dn : r.hr[m];
  }
}

template <int R>
__global__ void __launch_bounds__(DWARPS * 32) direct2d_reg_kernel(const __grid_constant__ DirectParams p,
                                                                    const float* __restrict__ in,
                                                                    float* __restrict__ out, int seg) {
  constexpr int K = 2 * R + 1;
  const int lane = threadIdx.x & 31;
  const int64_t H = p.H, W = p.W;
  const int64_t xw = ((int64_t)blockIdx.x * DWARPS + (threadIdx.x >> 5)) * 128;
  if (xw >= W) return;  // the whole warp
  const int64_t x = xw + 4 * lane;
  const bool active = x < W;
  const int64_t y0 = (int64_t)blockIdx.y * seg;
  // halo columns: from lane l-1 / l+1 inside the warp and the grid, else one float4 column
  // (wrapped when periodic; -1: outside a Dirichlet grid, zeros)
  const bool left_shfl = lane > 0, right_shfl = lane < 31 && x + 4 < W;
  const int64_t xl = x - 4 >= 0 ? x - 4 : (p.periodic ? W - 4 : -1);
  const int64_t xr = x + 4 < W ? x + 4 : (p.periodic ? 0 : -1);
  float acc[K][4];
#pragma unroll
  for (int k = 0; k < K; k++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[k][j] = 0.f;
  // input rows y0 - R .. y0 + nout + R - 1: each wraps at most once (H >= R)
  const int nout = (int)(H - y0 < seg ? H - y0 : seg);
  const int nrows = nout + 2 * R;
  auto row_ptr = [&](int i) -> const float* {  // input row y0 - R + i, null for a row of zeros
    int64_t r = y0 - R + i;
    if (p.periodic) return in + (r < 0 ? r + H : (r >= H ? r - H : r)) * W;
    return (r >= 0 && r < H) ? in + r * W : nullptr;
  };
  // (the rows of a K-row block are independent: their loads need no explicit prefetch, and
  // one measured slower here, 626 -> 511 GStencil/s for the 9-point box at 4096^2)
  for (int ib = 0; ib < nrows; ib += K) {
#pragma unroll
    for (int ii = 0; ii < K; ii++) {
      const int i = ib + ii;  // input row y0 - R + i
      if (i >= nrows) break;
      const RowLoad<R> cur = load_row<R>(row_ptr(i), x, active, left_shfl, right_shfl, xl, xr);
      float s[4 + 2 * R];
      row_values<R>(cur, left_shfl, right_shfl, s);
      // output row y0 + i - R - a takes this row through weight row a (a = -R .. R); its
      // accumulator slot is (i - R - a) mod K (compile-time: ib is a multiple of K)
#pragma unroll
      for (int a = -R; a <= R; a++) {
        const int slot = ((ii - R - a) % K + 2 * K) % K;
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
          for (int b = -R; b <= R; b++)
            acc[slot][j] = fmaf(p.wdense[(a + R) * K + (b + R)], s[R + j + b], acc[slot][j]);
      }
      // output row y0 + i - 2R has now taken its last input row
      const int done = ((ii - 2 * R) % K + 2 * K) % K;
      const int oy = i - 2 * R;
      if (oy >= 0 && active)
        *reinterpret_cast<float4*>(out + (y0 + oy) * W + x) =
            make_float4(acc[done][0], acc[done][1], acc[done][2], acc[done][3]);
#pragma unroll
      for (int j = 0; j < 4; j++) acc[done][j] = 0.f;
    }
  }
}

// 3D, radius 1: warp w of the CTA owns rows y .. y + D3ROWS - 1 (y = (blockIdx.y * DWARPS +
// w) * D3ROWS) and 128 columns; it walks the D3SEG + 2 input planes of its z segment, taking
// rows y-1 .. y+D3ROWS of each.  STAR: only the 7 points of the star (the other weights are
// zero), in the same order; two rows per warp (the dense cube keeps one, for registers).
template <bool STAR, int D3ROWS = STAR ? 2 : 1>
__global__ void __launch_bounds__(DWARPS * 32, 4) direct3d_reg_kernel(const __grid_constant__ DirectParams p,
                                                                    const float* __restrict__ in,
                                                                    float* __restrict__ out) {
  constexpr int NR = D3ROWS + 2;  // input rows per plane
  const int lane = threadIdx.x & 31;
  const int64_t D = p.D, H = p.H, W = p.W;
  const int64_t xw = (int64_t)blockIdx.x * 128;
  const int64_t y = ((int64_t)blockIdx.y * DWARPS + (threadIdx.x >> 5)) * D3ROWS;
  if (y >= H) return;  // the whole warp
  const int64_t x = xw + 4 * lane;
  const bool active = x < W;
  const int64_t z0 = (int64_t)blockIdx.z * D3SEG;
  const bool left_shfl = lane > 0, right_shfl = lane < 31 && x + 4 < W;
  const int64_t xl = x - 4 >= 0 ? x - 4 : (p.periodic ? W - 4 : -1);
  const int64_t xr = x + 4 < W ? x + 4 : (p.periodic ? 0 : -1);
  // input row d of a plane is y - 1 + d (wrapped once when periodic: H >= 1 and
  // y + D3ROWS <= H + D3ROWS - 1); rows past the grid's end, or outside a Dirichlet grid, read zeros
  int64_t ys[NR];
  bool yin[NR];
#pragma unroll
  for (int d = 0; d < NR; d++) {
    int64_t yy = y + d - 1;
    yin[d] = p.periodic || (yy >= 0 && yy < H);
    while (yy < 0) yy += H;
    while (yy >= H) yy -= H;
    ys[d] = yy;
  }
  float acc[3][D3ROWS][4];
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int r = 0; r < D3ROWS; r++)
#pragma unroll
      for (int j = 0; j < 4; j++) acc[k][r][j] = 0.f;
  // input planes z0 - 1 .. z0 + nout: each wraps at most once
  const int nout = (int)(D - z0 < D3SEG ? D - z0 : D3SEG);
  const int npl = nout + 2;
  auto load_plane = [&](int i, RowLoad<1> (&rl)[NR]) {  // input plane z0 - 1 + i
    int64_t z = z0 - 1 + i;
    bool zin = true;
    if (p.periodic)
      z = z < 0 ? z + D : (z >= D ? z - D : z);
    else
      zin = z >= 0 && z < D;
#pragma unroll
    for (int d = 0; d < NR; d++)
      rl[d] = load_row<1>((zin && yin[d]) ? in + (z * H + ys[d]) * W : nullptr, x, active, left_shfl, right_shfl, xl,
                          xr);
  };
  // the loads of the next input plane are issued before this plane's FMAs
  RowLoad<1> next[NR];
  load_plane(0, next);
  for (int ib = 0; ib < npl; ib += 3) {
#pragma unroll
    for (int ii = 0; ii < 3; ii++) {
      const int i = ib + ii;  // input plane z0 - 1 + i
      if (i >= npl) break;
      RowLoad<1> cur[NR];
#pragma unroll
      for (int d = 0; d < NR; d++) cur[d] = next[d];
      if (i + 1 < npl) load_plane(i + 1, next);
      float s[NR][6];
#pragma unroll
      for (int d = 0; d < NR; d++) row_values<1>(cur[d], left_shfl, right_shfl, s[d]);
#pragma unroll
      for (int a = -1; a <= 1; a++) {
        const int slot = ((ii - 1 - a) % 3 + 6) % 3;
#pragma unroll
        for (int r = 0; r < D3ROWS; r++)
#pragma unroll
          for (int j = 0; j < 4; j++)
#pragma unroll
            for (int dy = 0; dy < 3; dy++)
#pragma unroll
              for (int dx = 0; dx < 3; dx++) {
                const int nz = (a != 0 ? 1 : 0) + (dy != 1 ? 1 : 0) + (dx != 1 ? 1 : 0);
                if (STAR && nz > 1) continue;
                acc[slot][r][j] = fmaf(p.wdense[((a + 1) * 3 + dy) * 3 + dx], s[r + dy][j + dx], acc[slot][r][j]);
              }
      }
      const int done = ((ii - 2) % 3 + 3) % 3;
      const int oz = i - 2;
#pragma unroll
      for (int r = 0; r < D3ROWS; r++) {
        if (oz >= 0 && active && y + r < H)
          *reinterpret_cast<float4*>(out + ((z0 + oz) * H + y + r) * W + x) =
              make_float4(acc[done][r][0], acc[done][r][1], acc[done][r][2], acc[done][r][3]);
#pragma unroll
        for (int j = 0; j < 4; j++) acc[done][r][j] = 0.f;
      }
    }
  }
}

// 1D: a CTA covers 2048 outputs; each thread computes 8 of them, 256 apart (coalesced), in
// the fixed offset order.
constexpr int E1X = 2048;

template <int R>
__global__ void __launch_bounds__(256) direct1d_kernel(const __grid_constant__ DirectParams p,
                                                       const float* __restrict__ in, float* __restrict__ out) {
  __shared__ float tile[E1X + 2 * R];
  const int64_t W = p.W, x0 = (int64_t)blockIdx.x * E1X;
  for (int i = threadIdx.x; i < E1X + 2 * R; i += blockDim.x) {
    int64_t x = x0 + i - R;
    float v = 0.f;
    if (p.periodic) {
      x = x < 0 ? x + W : (x >= W ? x - W : x);
      v = in[x];
    } else if (x >= 0 && x < W) {
      v = in[x];
    }
    tile[i] = v;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < E1X / 256; k++) {
    const int lx = (int)threadIdx.x + 256 * k;
    float acc = 0.f;
#pragma unroll
    for (int d = 0; d < 2 * R + 1; d++) acc = fmaf(p.wdense[d], tile[lx + d], acc);
    if (x0 + lx < W) out[x0 + lx] = acc;
  }
}

// 3D, radius 1: a CTA covers 32 x 8 x 16 outputs (x, y, z); thread (x, y) keeps the 16
// outputs of its z column in registers and adds each staged input into every output that
// uses it.  Per output the FMAs run over the dense 3 x 3 x 3 cube in (dz, dy, dx) order,
// zero weights included (an FMA with weight 0 leaves a finite sum unchanged, so the result
// equals the sparse loop's over the nonzero points in the same order).
constexpr int E3X = 32, E3Y = 8, E3Z = 16;

__global__ void __launch_bounds__(256) direct3d_r1_kernel(const __grid_constant__ DirectParams p,
                                                          const float* __restrict__ in, float* __restrict__ out) {
  constexpr int TW = E3X + 2, TH = E3Y + 2, TD = E3Z + 2;
  __shared__ float tile[TD * TH * TW];
  __shared__ int64_t row_off[TD * TH];  // source offset of tile row (z, y), -1: outside (zeros)
  const int64_t D = p.D, H = p.H, W = p.W;
  const int64_t x0 = (int64_t)blockIdx.x * E3X, y0 = (int64_t)blockIdx.y * E3Y, z0 = (int64_t)blockIdx.z * E3Z;
  // the boundary rule along z and y is applied once per tile row, along x per element
  for (int r = threadIdx.x; r < TD * TH; r += blockDim.x) {
    int64_t z = z0 + r / TH - 1, y = y0 + r % TH - 1;
    if (p.periodic) {
      z = z < 0 ? z + D : (z >= D ? z - D : z);
      y = y < 0 ? y + H : (y >= H ? y - H : y);
      row_off[r] = (z * H + y) * W;
    } else {
      row_off[r] = (z >= 0 && z < D && y >= 0 && y < H) ? (z * H + y) * W : -1;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < TW * TH * TD; i += blockDim.x) {
    const int r = i / TW, tx = i - r * TW;
    int64_t x = x0 + tx - 1;
    const int64_t off = row_off[r];
    float v = 0.f;
    if (p.periodic) {
      x = x < 0 ? x + W : (x >= W ? x - W : x);
      v = in[off + x];
    } else if (off >= 0 && x >= 0 && x < W) {
      v = in[off + x];
    }
    tile[i] = v;
  }
  __syncthreads();
  const int cx = threadIdx.x % E3X, cy = threadIdx.x / E3X;
  float acc[E3Z];
#pragma unroll
  for (int k = 0; k < E3Z; k++) acc[k] = 0.f;
  // input plane zz (tile-relative) feeds output k through weight plane dz = zz - k
#pragma unroll
  for (int zz = 0; zz < TD; zz++) {
#pragma unroll
    for (int dy = 0; dy < 3; dy++) {
#pragma unroll
      for (int dx = 0; dx < 3; dx++) {
        const float v = tile[(zz * TH + cy + dy) * TW + cx + dx];
#pragma unroll
        for (int dz = 0; dz < 3; dz++) {
          const int k = zz - dz;
          if (k >= 0 && k < E3Z) acc[k] = fmaf(p.wdense[(dz * 3 + dy) * 3 + dx], v, acc[k]);
        }
      }
    }
  }
  const int64_t y = y0 + cy, x = x0 + cx;
  if (y < H && x < W) {
#pragma unroll
    for (int k = 0; k < E3Z; k++)
      if (z0 + k < D) out[((z0 + k) * H + y) * W + x] = acc[k];
  }
}

// 3D, radius 2-3: a CTA covers 32 x 8 x 4 outputs, FMAs over the nonzero points in order.
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
  // the difference and the maxima in FP32 (x - ref rounds once, 2^-24 relative), the sums of
  // squares in FP64; FP64 throughput, not memory, bounds a kernel that does more in FP64
  double s0 = 0.0, s1 = 0.0;
  float m0f = 0.f, m1f = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float a = x[i], b = ref[i];
    const float d = a - b;
    s0 = fma((double)d, (double)d, s0);
    s1 = fma((double)b, (double)b, s1);
    m0f = fmaxf(m0f, fabsf(d));
    m1f = fmaxf(m1f, fabsf(b));
  }
  double m0 = m0f, m1 = m1f;
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


// ---------------------------------------------------------------------------------------
// Dirichlet band of a fused sweep.  The composed t-step kernel is exact only at points at
// least (t-1)r from every edge, because the zero boundary is imposed once per sweep instead
// of after every step.  Each CTA recomputes a rectangle of the band (the top and bottom
// rows [0, bw) and [H-bw, H), then the left and right columns of the rows in between) from
// the sweep's input: it stages the rectangle widened by t*r on each side (zeros outside the
// grid), takes t single steps in shared memory with the zero boundary re-imposed after each
// one, and writes the rectangle.  Window cells whose stencil leaves the window become
// invalid; that error moves r cells inward per step, so after t steps it has not reached
// the rectangle.
// ---------------------------------------------------------------------------------------
__global__ void band2d_kernel(const BandParams p) {
  allow_next_sweep();
  extern __shared__ float bsm[];
  const int H = p.H, W = p.W, bw = p.bw, seg = p.seg, r = p.radius;
  const int top_h = bw < H ? bw : H;
  const int bot_y0 = (H - bw > top_h) ? H - bw : top_h;
  const int mid_h = H - 2 * bw;
  const int left_w = bw < W ? bw : W;
  const int right_x0 = (W - bw > left_w) ? W - bw : left_w;
  int b = (int)blockIdx.x, ty0, ty1, tx0, tx1;
  if (b < p.nx) {
    ty0 = 0, ty1 = top_h, tx0 = b * seg, tx1 = min(W, tx0 + seg);
  } else if ((b -= p.nx) < p.nx) {
    ty0 = bot_y0, ty1 = H, tx0 = b * seg, tx1 = min(W, tx0 + seg);
  } else if ((b -= p.nx) < p.ny) {
    ty0 = bw + b * seg, ty1 = min(bw + mid_h, ty0 + seg), tx0 = 0, tx1 = left_w;
  } else {
    b -= p.ny;
    ty0 = bw + b * seg, ty1 = min(bw + mid_h, ty0 + seg), tx0 = right_x0, tx1 = W;
  }
  if (ty0 >= ty1 || tx0 >= tx1) return;
  const int M = p.t * r;
  const int wy0 = ty0 - M, wx0 = tx0 - M;
  const int WH = ty1 - ty0 + 2 * M, WW = tx1 - tx0 + 2 * M;
  const int n = WH * WW;
  float* a = bsm;
  float* c = bsm + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int y = wy0 + i / WW, x = wx0 + i % WW;
    a[i] = (y >= 0 && y < H && x >= 0 && x < W) ? p.src[(int64_t)(y + p.src_off) * p.src_pitch + x + p.src_off] : 0.f;
  }
  __syncthreads();
  const int side = 2 * r + 1;
  for (int s = 0; s < p.t; s++) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int yy = i / WW, xx = i % WW;
      const int y = wy0 + yy, x = wx0 + xx;
      float v = 0.f;
      if (y >= 0 && y < H && x >= 0 && x < W && yy >= r && yy < WH - r && xx >= r && xx < WW - r) {
        const float* q = a + (yy - r) * WW + (xx - r);
        for (int dy = 0; dy < side; dy++)
          for (int dx = 0; dx < side; dx++) v = fmaf(p.w[dy * side + dx], q[dy * WW + dx], v);
      }
      c[i] = v;
    }
    __syncthreads();
    float* tmp = a;
    a = c;
    c = tmp;
  }
  const int th = ty1 - ty0, tw = tx1 - tx0;
  for (int i = threadIdx.x; i < th * tw; i += blockDim.x) {
    const int y = ty0 + i / tw, x = tx0 + i % tw;
    p.dst[(int64_t)(y + p.dst_off) * p.dst_pitch + x + p.dst_off] = a[(y - wy0) * WW + (x - wx0)];
  }
}


// ---------------------------------------------------------------------------------------
// 3D Dirichlet frame of a fused radius-1 sweep of depth t: the cells within bw = t - 1 of a
// face need step-by-step values (the fused kernel sees the zero boundary only once).  The
// frame is cut into boxes: z slabs (z < bw or z >= D - bw, all y and x), y slabs (the other
// z, y < bw or y >= H - bw), x slabs (the other z and y, x < bw or x >= W - bw), each cut into
// chunks of up to kB3 x kB3 cells across.  A CTA stages its box widened by t cells (zeros
// outside the grid), takes t FP32 steps in shared memory with the zero boundary re-imposed,
// FMAs in (dz, dy, dx) order, and writes the box.
// ---------------------------------------------------------------------------------------
constexpr int kB3 = 32;

__global__ void band3d_kernel(const Band3DParams p) {
  allow_next_sweep();
  extern __shared__ float b3[];
  const int D = p.D, H = p.H, W = p.W, bw = p.bw, t = p.t;
  const int zlo = bw < D ? bw : D, zhi0 = (D - bw > zlo) ? D - bw : zlo;  // z slabs [0, zlo), [zhi0, D)
  const int ylo = bw < H ? bw : H, yhi0 = (H - bw > ylo) ? H - bw : ylo;
  const int xlo = bw < W ? bw : W, xhi0 = (W - bw > xlo) ? W - bw : xlo;
  int b = (int)blockIdx.x;
  int z0, z1, y0, y1, x0, x1;
  const int nz_slab = p.nzy * p.nzx, ny_slab = p.nyz * p.nyx, nx_slab = p.nxz * p.nxy;
  if (b < 2 * nz_slab) {
    const int s = b / nz_slab, c = b % nz_slab;
    z0 = s ? zhi0 : 0, z1 = s ? D : zlo;
    y0 = (c / p.nzx) * kB3, y1 = min(H, y0 + kB3), x0 = (c % p.nzx) * kB3, x1 = min(W, x0 + kB3);
  } else if ((b -= 2 * nz_slab) < 2 * ny_slab) {
    const int s = b / ny_slab, c = b % ny_slab;
    z0 = zlo + (c / p.nyx) * kB3, z1 = min(zhi0, z0 + kB3);
    y0 = s ? yhi0 : 0, y1 = s ? H : ylo;
    x0 = (c % p.nyx) * kB3, x1 = min(W, x0 + kB3);
  } else {
    b -= 2 * ny_slab;
    if (b >= 2 * nx_slab) return;
    const int s = b / nx_slab, c = b % nx_slab;
    z0 = zlo + (c / p.nxy) * kB3, z1 = min(zhi0, z0 + kB3);
    y0 = ylo + (c % p.nxy) * kB3, y1 = min(yhi0, y0 + kB3);
    x0 = s ? xhi0 : 0, x1 = s ? W : xlo;
  }
  if (z0 >= z1 || y0 >= y1 || x0 >= x1) return;
  const int wz0 = z0 - t, wy0 = y0 - t, wx0 = x0 - t;
  const int WD = z1 - z0 + 2 * t, WH = y1 - y0 + 2 * t, WW = x1 - x0 + 2 * t;
  const int n = WD * WH * WW;
  float* a = b3;
  float* c = b3 + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int zz = i / (WH * WW), yy = (i / WW) % WH, xx = i % WW;
    const int z = wz0 + zz, y = wy0 + yy, x = wx0 + xx;
    a[i] = (z >= 0 && z < D && y >= 0 && y < H && x >= 0 && x < W)
               ? p.src[(int64_t)(z + p.src_off) * p.src_plane + (int64_t)(y + p.src_off) * p.src_pitch + x + p.src_off]
               : 0.f;
  }
  __syncthreads();
  for (int s = 0; s < t; s++) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int zz = i / (WH * WW), yy = (i / WW) % WH, xx = i % WW;
      const int z = wz0 + zz, y = wy0 + yy, x = wx0 + xx;
      float v = 0.f;
      if (z >= 0 && z < D && y >= 0 && y < H && x >= 0 && x < W && zz >= 1 && zz < WD - 1 && yy >= 1 &&
          yy < WH - 1 && xx >= 1 && xx < WW - 1) {
        const float* q = a + ((zz - 1) * WH + (yy - 1)) * WW + (xx - 1);
        for (int dz = 0; dz < 3; dz++)
          for (int dy = 0; dy < 3; dy++)
            for (int dx = 0; dx < 3; dx++) v = fmaf(p.w[(dz * 3 + dy) * 3 + dx], q[(dz * WH + dy) * WW + dx], v);
      }
      c[i] = v;
    }
    __syncthreads();
    float* tmp = a;
    a = c;
    c = tmp;
  }
  const int bd = z1 - z0, bh = y1 - y0, bwid = x1 - x0;
  for (int i = threadIdx.x; i < bd * bh * bwid; i += blockDim.x) {
    const int z = z0 + i / (bh * bwid), y = y0 + (i / bwid) % bh, x = x0 + i % bwid;
    p.dst[(int64_t)(z + p.dst_off) * p.dst_plane + (int64_t)(y + p.dst_off) * p.dst_pitch + x + p.dst_off] =
        a[((z - wz0) * WH + (y - wy0)) * WW + (x - wx0)];
  }
}

// ---------------------------------------------------------------------------------------
// 3D copy-in: unpadded D x H x W -> padded (D + 2G) x (H + 2G) x Wp; ghost cells hold the
// periodic images or zeros; columns beyond W + 2G are zero.  One thread per padded cell.
// ---------------------------------------------------------------------------------------
__global__ void pad_copy3d_kernel(const float* __restrict__ in, float* __restrict__ out, int D, int H, int W, int G,
                                  int64_t Wp, int periodic, unsigned* maxabs) {
  allow_next_sweep();
  // a CTA per padded row (grid-stride over rows), its threads along x: the row's source row
  // is found once, and loads and stores are contiguous
  const int64_t Hp = (int64_t)H + 2 * G, Dp = (int64_t)D + 2 * G;
  const int64_t rows = Dp * Hp;
  float m = 0.f;
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    int64_t z = row / Hp - G, y = row % Hp - G;
    bool inside = true;
    if (periodic) {
      z = z < 0 ? z + D : (z >= D ? z - D : z);
      y = y < 0 ? y + H : (y >= H ? y - H : y);
    } else {
      inside = z >= 0 && z < D && y >= 0 && y < H;
    }
    const float* src = in + (inside ? (z * H + y) * W : 0);
    float* dst = out + row * Wp;
    copy_padded_row(src, dst, W, G, Wp, periodic, inside, &m);
  }
  fold_maxabs(maxabs, m);
}

// Periodic ghost shell of a padded 3D grid rewritten from the interior it wraps to (after a
// sweep that wrote the interior only).  One thread per padded cell of each padded row; rows
// wholly in the interior only touch their 2G ghost columns.
__global__ void ghost_refresh3d_kernel(float* __restrict__ g3, int D, int H, int W, int G, int64_t Wp) {
  allow_next_sweep();
  const int64_t Hp = (int64_t)H + 2 * G, Dp = (int64_t)D + 2 * G;
  const int64_t rows = Dp * Hp;
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const int64_t yp = r % Hp, zp = r / Hp;
    const bool ghost_row = yp < G || yp >= H + G || zp < G || zp >= D + G;
    int64_t z = zp - G, y = yp - G;
    z = z < 0 ? z + D : (z >= D ? z - D : z);
    y = y < 0 ? y + H : (y >= H ? y - H : y);
    const float* src = g3 + ((z + G) * Hp + (y + G)) * Wp + G;
    float* dst = g3 + r * Wp;
    for (int64_t xp = threadIdx.x; xp < (int64_t)W + 2 * G; xp += blockDim.x) {
      const bool ghost_col = xp < G || xp >= W + G;
      if (!ghost_row && !ghost_col) continue;
      int64_t x = xp - G;
      x = x < 0 ? x + W : (x >= W ? x - W : x);
      dst[xp] = src[x];
    }
  }
}

}  // namespace

cudaError_t launch_pad_copy3d(const float* in, float* padded, int D, int H, int W, int G, int64_t Wp, int periodic,
                              unsigned* maxabs, cudaStream_t stream) {
  const int64_t rows = ((int64_t)D + 2 * G) * ((int64_t)H + 2 * G);
  const int64_t blocks = rows < 152 * 32 ? rows : 152 * 32;
  pad_copy3d_kernel<<<(unsigned)blocks, 128, 0, stream>>>(in, padded, D, H, W, G, Wp, periodic, maxabs);
  return cudaGetLastError();
}

cudaError_t launch_ghost_refresh3d(float* padded, int D, int H, int W, int G, int64_t Wp, cudaStream_t stream) {
  const int64_t rows = ((int64_t)D + 2 * G) * ((int64_t)H + 2 * G);
  const int64_t blocks = rows < 152 * 32 ? rows : 152 * 32;
  ghost_refresh3d_kernel<<<(unsigned)blocks, 128, 0, stream>>>(padded, D, H, W, G, Wp);
  return cudaGetLastError();
}

cudaError_t launch_pad_copy1d(const float* in, float* out, int64_t W, int G, int64_t Wp, int periodic,
                              unsigned* maxabs, cudaStream_t stream) {
  int64_t blocks = (Wp + 1023) / 1024;
  if (blocks > 152 * 16) blocks = 152 * 16;
  pad_copy1d_kernel<<<(unsigned)blocks, 256, 0, stream>>>(in, out, W, G, Wp, periodic, maxabs);
  return cudaGetLastError();
}

cudaError_t launch_ghost_refresh1d(float* line, int64_t W, int G, cudaStream_t stream) {
  ghost_refresh1d_kernel<<<1, 64, 0, stream>>>(line, W, G);
  return cudaGetLastError();
}

cudaError_t launch_pad_copy2d(const float* in, float* padded, int H, int W, int G, int64_t Wp, int periodic,
                              unsigned* maxabs, cudaStream_t stream) {
  const int64_t rows = (int64_t)H + 2 * G;
  const int64_t blocks = rows < 152 * 32 ? rows : 152 * 32;
  pad_copy2d_kernel<<<(unsigned)blocks, 256, 0, stream>>>(in, padded, H, W, G, Wp, periodic, maxabs);
  return cudaGetLastError();
}

template <int R>
static cudaError_t launch_direct2d(const DirectParams& p, const float* in, float* out, cudaStream_t stream) {
  if (p.W % 4 == 0) {
    // rows per warp: DSEG, fewer when the grid has too few warps for the SMs (about 48 warps
    // per SM); a shorter segment re-reads 2R more rows per segment, mostly from L2
    const int64_t col_warps = (p.W + 127) / 128;
    int64_t seg = DSEG;
    while (seg > 8 && col_warps * ((p.H + seg - 1) / seg) < 152 * 48) seg /= 2;
    dim3 g((unsigned)((p.W + 128 * DWARPS - 1) / (128 * DWARPS)), (unsigned)((p.H + seg - 1) / seg));
    direct2d_reg_kernel<R><<<g, DWARPS * 32, 0, stream>>>(p, in, out, (int)seg);
    return cudaGetLastError();
  }
  dim3 grid((unsigned)((p.W + DTX - 1) / DTX), (unsigned)((p.H + DTY - 1) / DTY));
  const size_t smem = (size_t)(DTX + 2 * R) * (DTY + 2 * R) * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(direct2d_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  direct2d_kernel<R><<<grid, 256, smem, stream>>>(p, in, out);
  return cudaGetLastError();
}

size_t band2d_smem_bytes(int bw, int t, int radius, int seg) {
  const size_t M = (size_t)t * radius;
  const size_t a = ((size_t)bw + 2 * M) * ((size_t)seg + 2 * M);
  return 2 * a * sizeof(float);
}

cudaError_t launch_band2d(BandParams p, cudaStream_t stream) {
  if (p.t < 2 || p.bw <= 0) return cudaSuccess;
  // largest segment (128 down to 8) whose two window buffers fit in shared memory
  int seg = 128;
  while (seg > 8 && band2d_smem_bytes(p.bw, p.t, p.radius, seg) > 200 * 1024) seg /= 2;
  const size_t smem = band2d_smem_bytes(p.bw, p.t, p.radius, seg);
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  p.seg = seg;
  p.nx = (p.W + seg - 1) / seg;
  const int mid = p.H - 2 * p.bw;
  p.ny = mid > 0 ? (mid + seg - 1) / seg : 0;
  const int blocks = 2 * p.nx + 2 * p.ny;
  cudaError_t e = cudaFuncSetAttribute(band2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  band2d_kernel<<<blocks, 256, smem, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_band3d(Band3DParams p, cudaStream_t stream) {
  if (p.t < 2 || p.bw <= 0) return cudaSuccess;
  auto cdiv = [](int a, int b) { return a > 0 ? (a + b - 1) / b : 0; };
  const int zmid = p.D - 2 * p.bw > 0 ? p.D - 2 * p.bw : 0, ymid = p.H - 2 * p.bw > 0 ? p.H - 2 * p.bw : 0;
  p.nzy = cdiv(p.H, kB3);
  p.nzx = cdiv(p.W, kB3);
  p.nyz = cdiv(zmid, kB3);
  p.nyx = cdiv(p.W, kB3);
  p.nxz = cdiv(zmid, kB3);
  p.nxy = cdiv(ymid, kB3);
  const int blocks = 2 * (p.nzy * p.nzx + p.nyz * p.nyx + p.nxz * p.nxy);
  // the largest box: bw x kB3 x kB3 (or kB3 x kB3 x kB3 when bw > kB3), widened by t per side
  const int e = kB3 + 2 * p.t, thin = (p.bw < kB3 ? p.bw : kB3) + 2 * p.t;
  const size_t smem = 2 * (size_t)e * e * thin * sizeof(float);
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t err = cudaFuncSetAttribute(band3d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  if (blocks > 0) band3d_kernel<<<blocks, 256, smem, stream>>>(p);
  return cudaGetLastError();
}

template <int R>
static cudaError_t launch_direct1d(const DirectParams& p, const float* in, float* out, cudaStream_t stream) {
  direct1d_kernel<R><<<(unsigned)((p.W + E1X - 1) / E1X), 256, 0, stream>>>(p, in, out);
  return cudaGetLastError();
}

cudaError_t launch_direct_step(const DirectParams& p, const float* in, float* out, cudaStream_t stream) {
  const int r = p.radius;
  if (p.ndim == 1) {
    switch (r) {
      case 1: return launch_direct1d<1>(p, in, out, stream);
      case 2: return launch_direct1d<2>(p, in, out, stream);
      case 3: return launch_direct1d<3>(p, in, out, stream);
      case 4: return launch_direct1d<4>(p, in, out, stream);
      default: return cudaErrorInvalidValue;
    }
  }
  if (p.ndim == 2) {
    switch (r) {
      case 1: return launch_direct2d<1>(p, in, out, stream);
      case 2: return launch_direct2d<2>(p, in, out, stream);
      case 3: return launch_direct2d<3>(p, in, out, stream);
      case 4: return launch_direct2d<4>(p, in, out, stream);
      default: return cudaErrorInvalidValue;
    }
  }
  if (r == 1 && p.W % 4 == 0) {
    bool star = true;  // only the centre and the six axis neighbours are nonzero
    for (int idx = 0; idx < 27; idx++) {
      const int a = idx / 9, b = (idx / 3) % 3, c = idx % 3;
      if ((a != 1) + (b != 1) + (c != 1) > 1 && p.wdense[idx] != 0.f) star = false;
    }
    const int rows = star ? 2 : 1;  // output rows per warp (the kernels' D3ROWS)
    dim3 g((unsigned)((p.W + 127) / 128), (unsigned)((p.H + DWARPS * rows - 1) / (DWARPS * rows)),
           (unsigned)((p.D + D3SEG - 1) / D3SEG));
    if (star)
      direct3d_reg_kernel<true><<<g, DWARPS * 32, 0, stream>>>(p, in, out);
    else
      direct3d_reg_kernel<false><<<g, DWARPS * 32, 0, stream>>>(p, in, out);
    return cudaGetLastError();
  }
  if (r == 1) {
    dim3 grid((unsigned)((p.W + E3X - 1) / E3X), (unsigned)((p.H + E3Y - 1) / E3Y), (unsigned)((p.D + E3Z - 1) / E3Z));
    direct3d_r1_kernel<<<grid, 256, 0, stream>>>(p, in, out);
    return cudaGetLastError();
  }
  dim3 grid((unsigned)((p.W + D3X - 1) / D3X), (unsigned)((p.H + D3Y - 1) / D3Y), (unsigned)((p.D + D3Z - 1) / D3Z));
  size_t smem = (size_t)(D3X + 2 * r) * (D3Y + 2 * r) * (D3Z + 2 * r) * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(direct3d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  direct3d_kernel<<<grid, 256, smem, stream>>>(p, in, out);
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
