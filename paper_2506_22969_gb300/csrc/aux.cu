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
#ifndef SPST_D2_PREFETCH
#define SPST_D2_PREFETCH 0  // 2D, radius >= 2: load input row i + 1 before row i's FMAs
#endif
#ifndef SPST_D2_MINB
#define SPST_D2_MINB 0  // 2D: resident CTAs per SM the register budget must allow (0: no bound)
#endif
#if SPST_D2_MINB > 0
#define SPST_D2_BOUNDS __launch_bounds__(128, SPST_D2_MINB)
#else
#define SPST_D2_BOUNDS __launch_bounds__(128)
#endif
#ifndef SPST_D3_ROWS_STAR
#define SPST_D3_ROWS_STAR 3  // 3D radius-1 star: output rows per warp
#endif
#ifndef SPST_D3_ROWS_BOX
#define SPST_D3_ROWS_BOX 3  // 3D radius-1 box: output rows per warp
#endif
#ifndef SPST_D3_MINB
#define SPST_D3_MINB 4  // 3D: resident CTAs per SM the register budget must allow
#endif
#ifndef SPST_D3_SEG
#define SPST_D3_SEG 32  // 3D: most output planes per warp
#endif
#ifndef SPST_D3_FILL
#define SPST_D3_FILL 1  // 3D: waves of resident CTAs the z segments are shortened to fill
#endif
constexpr int DSEG = 64;   // 2D, radius 1: most output rows per warp (fewer when the grid has few columns)
constexpr int D3SEG = SPST_D3_SEG;
constexpr int DWARPS = 4;  // warps per CTA (128 threads)

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
__global__ void SPST_D2_BOUNDS direct2d_reg_kernel(const __grid_constant__ DirectParams p,
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
  // radius 1: the rows of a K-row block are independent and their loads need no explicit
  // prefetch (one measured slower, 626 -> 511 GStencil/s for the 9-point box at 4096^2);
  // larger radii may load row i + 1 before row i's FMAs (SPST_D2_PREFETCH)
  constexpr bool PF = SPST_D2_PREFETCH && R >= 2;
  RowLoad<R> nxt;
  if constexpr (PF) nxt = load_row<R>(row_ptr(0), x, active, left_shfl, right_shfl, xl, xr);
  for (int ib = 0; ib < nrows; ib += K) {
#pragma unroll
    for (int ii = 0; ii < K; ii++) {
      const int i = ib + ii;  // input row y0 - R + i
      if (i >= nrows) break;
      RowLoad<R> cur;
      if constexpr (PF) {
        cur = nxt;
        if (i + 1 < nrows) nxt = load_row<R>(row_ptr(i + 1), x, active, left_shfl, right_shfl, xl, xr);
      } else {
        cur = load_row<R>(row_ptr(i), x, active, left_shfl, right_shfl, xl, xr);
      }
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

// 3D, radius 1: warp w of the CTA owns rows y .. y + ROWS - 1 (y = (blockIdx.y * DWARPS + w) *
// ROWS) and 128 columns; it walks the zseg + 2 input planes of its z segment, taking rows
// y - 1 .. y + ROWS of each.  Each input row is consumed (its 6 values per lane) and then
// refilled with the same row of the next plane, so a row's loads are in flight for a whole
// plane of FMAs.  STAR: only the 7 points of the star (the other weights are zero), in the
// same order.
template <bool STAR, int ROWS>
__global__ void __launch_bounds__(DWARPS * 32, SPST_D3_MINB) direct3d_reg_kernel(const __grid_constant__ DirectParams p,
                                                                    const float* __restrict__ in,
                                                                    float* __restrict__ out, int zseg) {
  constexpr int NR = ROWS + 2;  // input rows per plane
  const int lane = threadIdx.x & 31;
  const int64_t D = p.D, H = p.H, W = p.W;
  const int64_t xw = (int64_t)blockIdx.x * 128;
  const int64_t y = ((int64_t)blockIdx.y * DWARPS + (threadIdx.x >> 5)) * ROWS;
  if (y >= H) return;  // the whole warp
  const int64_t x = xw + 4 * lane;
  const bool active = x < W;
  const int64_t z0 = (int64_t)blockIdx.z * zseg;
  const bool left_shfl = lane > 0, right_shfl = lane < 31 && x + 4 < W;
  const int64_t xl = x - 4 >= 0 ? x - 4 : (p.periodic ? W - 4 : -1);
  const int64_t xr = x + 4 < W ? x + 4 : (p.periodic ? 0 : -1);
  // input row d of a plane is y - 1 + d, wrapped when periodic (H >= 1: a row index below
  // H + ROWS wraps a bounded number of times); rows outside a Dirichlet grid, and the rows
  // past the grid's end of the last warp, read zeros
  int yrow[NR];
  bool yin[NR];
#pragma unroll
  for (int d = 0; d < NR; d++) {
    int64_t yy = y + d - 1;
    yin[d] = p.periodic || (yy >= 0 && yy < H);
    while (yy < 0) yy += H;
    while (yy >= H) yy -= H;
    yrow[d] = (int)yy;
  }
  float acc[3][ROWS][4];
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int r = 0; r < ROWS; r++)
#pragma unroll
      for (int j = 0; j < 4; j++) acc[k][r][j] = 0.f;
  // input planes z0 - 1 .. z0 + nout: each wraps at most once
  const int nout = (int)(D - z0 < zseg ? D - z0 : zseg);
  const int npl = nout + 2;
  auto plane_base = [&](int i) -> const float* {  // input plane z0 - 1 + i, null for zeros
    int64_t z = z0 - 1 + i;
    if (p.periodic) return in + (z < 0 ? z + D : (z >= D ? z - D : z)) * H * W;
    return (z >= 0 && z < D) ? in + z * H * W : nullptr;
  };
  RowLoad<1> cur[NR];
  {
    const float* base = plane_base(0);
#pragma unroll
    for (int d = 0; d < NR; d++)
      cur[d] = load_row<1>((base && yin[d]) ? base + (int64_t)yrow[d] * W : nullptr, x, active, left_shfl, right_shfl, xl, xr);
  }
  for (int ib = 0; ib < npl; ib += 3) {
#pragma unroll
    for (int ii = 0; ii < 3; ii++) {
      const int i = ib + ii;  // input plane z0 - 1 + i
      if (i >= npl) break;
      const bool more = i + 1 < npl;
      const float* nbase = more ? plane_base(i + 1) : nullptr;
#pragma unroll
      for (int d = 0; d < NR; d++) {
        float s[6];
        row_values<1>(cur[d], left_shfl, right_shfl, s);
        if (more)
          cur[d] = load_row<1>((nbase && yin[d]) ? nbase + (int64_t)yrow[d] * W : nullptr, x, active, left_shfl, right_shfl, xl, xr);
        // input row d reaches output row r through dy = d - r; output plane z0 + i - 1 - a
        // through dz = a (accumulator slot (i - 1 - a) mod 3)
#pragma unroll
        for (int a = -1; a <= 1; a++) {
          const int slot = ((ii - 1 - a) % 3 + 6) % 3;
#pragma unroll
          for (int r = 0; r < ROWS; r++) {
            const int dy = d - r;
            if (dy < 0 || dy > 2) continue;
#pragma unroll
            for (int j = 0; j < 4; j++)
#pragma unroll
              for (int dx = 0; dx < 3; dx++) {
                if (STAR && (a != 0) + (dy != 1) + (dx != 1) > 1) continue;
                acc[slot][r][j] = fmaf(p.wdense[((a + 1) * 3 + dy) * 3 + dx], s[j + dx], acc[slot][r][j]);
              }
          }
        }
      }
      // output plane z0 + i - 2 has now taken its last input plane
      const int done = ((ii - 2) % 3 + 3) % 3;
      const int oz = i - 2;
#pragma unroll
      for (int r = 0; r < ROWS; r++) {
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
// z, y < bw or y >= H - bw), x slabs (the other z and y, x < bw or x >= W - bw).  A box spans
// the slab's thickness, band3d_lane(t) cells along its lane axis (x for z and y slabs, y for
// x slabs) and kB3 cells along its other long axis.  A CTA stages its box widened by t cells
// (zeros outside the grid) and takes t FP32 steps in shared memory; step s computes only the
// cells within t - 1 - s of the box that lie inside the grid (the cells outside stay zero:
// the boundary rule), a warp per row along the lane axis, FMAs in (dz, dy, dx) order (STAR:
// the 7 points of the star only, the other weights being zero).
// ---------------------------------------------------------------------------------------
constexpr int kB3 = 32;
// box extent along the lane axis: the widest step region (the box widened by t - 1 per side)
// then spans at most 32 lanes
__host__ __device__ constexpr int band3d_lane(int t) { return 34 - 2 * t > 8 ? 34 - 2 * t : 8; }

template <bool STAR>
__global__ void __launch_bounds__(256) band3d_kernel(const Band3DParams p) {
  allow_next_sweep();
  extern __shared__ float b3[];
  const int D = p.D, H = p.H, W = p.W, bw = p.bw, t = p.t, L = band3d_lane(p.t);
  const int dim[3] = {D, H, W};
  const int zlo = bw < D ? bw : D, zhi0 = (D - bw > zlo) ? D - bw : zlo;  // z slabs [0, zlo), [zhi0, D)
  const int ylo = bw < H ? bw : H, yhi0 = (H - bw > ylo) ? H - bw : ylo;
  const int xlo = bw < W ? bw : W, xhi0 = (W - bw > xlo) ? W - bw : xlo;
  int b = (int)blockIdx.x;
  int lo[3], hi[3];  // the box, (z, y, x)
  int la;            // lane axis: 2 (x) or 1 (y)
  const int nz_slab = p.nzy * p.nzx, ny_slab = p.nyz * p.nyx, nx_slab = p.nxz * p.nxy;
  if (b < 2 * nz_slab) {
    const int s = b / nz_slab, c = b % nz_slab;
    lo[0] = s ? zhi0 : 0, hi[0] = s ? D : zlo;
    lo[1] = (c / p.nzx) * kB3, hi[1] = min(H, lo[1] + kB3);
    lo[2] = (c % p.nzx) * L, hi[2] = min(W, lo[2] + L);
    la = 2;
  } else if ((b -= 2 * nz_slab) < 2 * ny_slab) {
    const int s = b / ny_slab, c = b % ny_slab;
    lo[0] = zlo + (c / p.nyx) * kB3, hi[0] = min(zhi0, lo[0] + kB3);
    lo[1] = s ? yhi0 : 0, hi[1] = s ? H : ylo;
    lo[2] = (c % p.nyx) * L, hi[2] = min(W, lo[2] + L);
    la = 2;
  } else {
    b -= 2 * ny_slab;
    if (b >= 2 * nx_slab) return;
    const int s = b / nx_slab, c = b % nx_slab;
    lo[0] = zlo + (c / p.nxy) * kB3, hi[0] = min(zhi0, lo[0] + kB3);
    lo[1] = ylo + (c % p.nxy) * L, hi[1] = min(yhi0, lo[1] + L);
    lo[2] = s ? xhi0 : 0, hi[2] = s ? W : xlo;
    la = 1;
  }
  if (lo[0] >= hi[0] || lo[1] >= hi[1] || lo[2] >= hi[2]) return;
  // staged box: cells lo - t .. hi + t - 1 per axis; row pitch odd (conflict-free lanes along y)
  int w0[3], S[3];
#pragma unroll
  for (int a = 0; a < 3; a++) w0[a] = lo[a] - t, S[a] = hi[a] - lo[a] + 2 * t;
  const int sy = S[2] | 1, sz = sy * S[1];
  float* a = b3;
  float* c = b3 + sz * S[0];
  // staging, kBatch loads in flight per thread.  The source is padded with zeros at least t
  // cells deep on every side (the launcher checks src_off >= t), so the staged box is read
  // without bounds checks.  A thread's cell advances by blockDim.x cells per iteration through
  // mixed-radix carries, its source and shared-memory offsets with it (no division per cell).
  const int ns = S[0] * S[1] * S[2], S12 = S[1] * S[2];
  const int nt = (int)blockDim.x;
  const int adz = nt / S12, adr = nt - adz * S12, ady = adr / S[2], adx = adr - ady * S[2];
  const int64_t pl = p.src_plane, pi = p.src_pitch;
  const float* sb = p.src + (int64_t)(w0[0] + p.src_off) * pl + (int64_t)(w0[1] + p.src_off) * pi + w0[2] + p.src_off;
  int cy, cx;
  int64_t go;  // source offset of the thread's cell from sb
  int ko;      // its shared-memory offset
  {
    const int cz = (int)threadIdx.x / S12, cr = (int)threadIdx.x - cz * S12;
    cy = cr / S[2], cx = cr - cy * S[2];
    go = cz * pl + cy * pi + cx;
    ko = cz * sz + cy * sy + cx;
  }
  const int64_t gstep = adz * pl + ady * pi + adx, gcx = pi - S[2], gcy = pl - S[1] * pi;
  const int kstep = adz * sz + ady * sy + adx, kcx = sy - S[2], kcy = sz - S[1] * sy;
  constexpr int kBatch = 8;
  for (int i0 = threadIdx.x; i0 < ns; i0 += kBatch * nt) {
    float v[kBatch];
    int kk[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; u++) {
      const bool in_box = i0 + u * nt < ns;
      v[u] = in_box ? sb[go] : 0.f;
      kk[u] = in_box ? ko : -1;
      cx += adx, go += gstep, ko += kstep;
      if (cx >= S[2]) cx -= S[2], cy++, go += gcx, ko += kcx;
      cy += ady;
      if (cy >= S[1]) cy -= S[1], go += gcy, ko += kcy;
    }
#pragma unroll
    for (int u = 0; u < kBatch; u++)
      if (kk[u] >= 0) {
        a[kk[u]] = v[u];
        c[kk[u]] = 0.f;
      }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int ra = la == 2 ? 1 : 2;  // the row axis besides z
  const int lst = la == 2 ? 1 : sy, rst = ra == 2 ? 1 : sy;
  for (int s = 0; s < t; s++) {
    // step s: the box widened by e = t - 1 - s, clipped to the grid, in staged coordinates
    const int e = t - 1 - s;
    int rl[3], nr[3];
#pragma unroll
    for (int q = 0; q < 3; q++) {
      const int l = max(lo[q] - e, 0), h = min(hi[q] + e, dim[q]);
      rl[q] = l - w0[q], nr[q] = h - l;
    }
    const int nra = ra == 2 ? nr[2] : nr[1], rla = ra == 2 ? rl[2] : rl[1];  // the row axis
    const int nla = la == 2 ? nr[2] : nr[1], lla = la == 2 ? rl[2] : rl[1];  // the lane axis
    // warp w takes rows w, w + nwarps, ... of the nr[0] x nra rows (z, then the row axis),
    // advanced by carries
    const int rows = nr[0] * nra, rz = nwarps / nra, rr = nwarps - rz * nra;
    int iz = rl[0] + warp / nra, ir = rla + warp % nra;
    for (int row = warp; row < rows; row += nwarps, iz += rz, ir += rr) {
      if (ir >= rla + nra) ir -= nra, iz++;
      for (int kl = lane; kl < nla; kl += 32) {
        const int k = iz * sz + ir * rst + (lla + kl) * lst;
        const float* q = a + k - sz - sy - 1;
        float v = 0.f;
#pragma unroll
        for (int dz = 0; dz < 3; dz++)
#pragma unroll
          for (int dy = 0; dy < 3; dy++)
#pragma unroll
            for (int dx = 0; dx < 3; dx++) {
              if (STAR && (dz != 1) + (dy != 1) + (dx != 1) > 1) continue;  // a zero weight
              v = fmaf(p.w[(dz * 3 + dy) * 3 + dx], q[dz * sz + dy * sy + dx], v);
            }
        c[k] = v;
      }
    }
    __syncthreads();
    float* tmp = a;
    a = c;
    c = tmp;
  }
  const int bd = hi[0] - lo[0], bh = hi[1] - lo[1], bx = hi[2] - lo[2], bhx = bh * bx;
  const int odz = nt / bhx, odr = nt - odz * bhx, ody = odr / bx, odx = odr - ody * bx;
  int oz = (int)threadIdx.x / bhx, orr = (int)threadIdx.x - oz * bhx, oy = orr / bx, ox = orr - oy * bx;
  for (int i = threadIdx.x; i < bd * bhx; i += nt) {
    p.dst[(int64_t)(lo[0] + oz + p.dst_off) * p.dst_plane + (int64_t)(lo[1] + oy + p.dst_off) * p.dst_pitch + lo[2] + ox +
          p.dst_off] = a[(oz + t) * sz + (oy + t) * sy + ox + t];
    ox += odx;
    if (ox >= bx) ox -= bx, oy++;
    oy += ody;
    if (oy >= bh) oy -= bh, oz++;
    oz += odz;
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
// sweep that wrote the interior only; needs G <= D, H, W).  Three disjoint sets of ghost cells,
// each read from interior cells only: whole padded rows of the z ghost planes and the y ghost
// rows of the interior planes, a warp per row along x; then the 2G x ghost cells of every
// interior row, a thread per cell.
__global__ void __launch_bounds__(256) ghost_refresh3d_kernel(float* __restrict__ g3, int D, int H, int W, int G,
                                                              int64_t Wp) {
  allow_next_sweep();
  const int Hp = H + 2 * G, Wr = W + 2 * G;
  const int64_t plane = (int64_t)Hp * Wp;
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int rows_z = 2 * G * Hp, rows = rows_z + D * 2 * G;
  for (int r = gw; r < rows; r += nw) {
    int zp, yp;
    if (r < rows_z) {
      const int k = r / Hp;  // ghost plane k: padded plane k (k < G) or D + k
      yp = r - k * Hp;
      zp = k < G ? k : D + k;
    } else {
      const int q = r - rows_z, zi = q / (2 * G), k = q - zi * 2 * G;
      zp = G + zi;
      yp = k < G ? k : H + k;
    }
    int z = zp - G, y = yp - G;
    z = z < 0 ? z + D : (z >= D ? z - D : z);
    y = y < 0 ? y + H : (y >= H ? y - H : y);
    const float* src = g3 + (z + G) * plane + (int64_t)(y + G) * Wp + G;
    float* dst = g3 + zp * plane + (int64_t)yp * Wp;
    for (int xp = lane; xp < Wr; xp += 32) {
      int x = xp - G;
      x = x < 0 ? x + W : (x >= W ? x - W : x);
      dst[xp] = src[x];
    }
  }
  const int64_t ncells = (int64_t)D * H * 2 * G;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ncells; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / (2 * G);
    const int k = (int)(i - row * 2 * G);
    const int64_t zi = row / H, yi = row - zi * H;
    const int xp = k < G ? k : W + k;
    int x = xp - G;
    x = x < 0 ? x + W : x - W;
    float* rp = g3 + (zi + G) * plane + (yi + G) * Wp;
    rp[xp] = rp[G + x];
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
  if (G <= 0) return cudaSuccess;
  ghost_refresh3d_kernel<<<152 * 4, 256, 0, stream>>>(padded, D, H, W, G, Wp);
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
    const int64_t col_warps = (p.W + 127) / 128, col_blocks = (p.W + 128 * DWARPS - 1) / (128 * DWARPS);
    int64_t seg = DSEG;
    if (R == 1) {
      while (seg > 8 && col_warps * ((p.H + seg - 1) / seg) < 152 * 48) seg /= 2;
    } else {
      // FMA-bound radii: whole waves of resident CTAs (a partial last wave leaves SMs with
      // half the warps), segments of 8-128 rows (a segment re-reads 2R rows; small grids take
      // short segments to give every SM work)
      static int slots = 0;  // resident CTAs on the device
      if (slots == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, direct2d_reg_kernel<R>, DWARPS * 32, 0);
        slots = sms * (per_sm > 0 ? per_sm : 1);
      }
      const int64_t waves = (col_blocks * ((p.H + 127) / 128) + slots - 1) / slots;
      const int64_t nseg = (int64_t)slots * waves / col_blocks;
      seg = (p.H + (nseg > 0 ? nseg : 1) - 1) / (nseg > 0 ? nseg : 1);
      seg = seg < 8 ? 8 : (seg > 128 ? 128 : seg);
    }
    dim3 g((unsigned)col_blocks, (unsigned)((p.H + seg - 1) / seg));
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
  const int L = band3d_lane(p.t);
  const int zmid = p.D - 2 * p.bw > 0 ? p.D - 2 * p.bw : 0, ymid = p.H - 2 * p.bw > 0 ? p.H - 2 * p.bw : 0;
  p.nzy = cdiv(p.H, kB3);
  p.nzx = cdiv(p.W, L);
  p.nyz = cdiv(zmid, kB3);
  p.nyx = cdiv(p.W, L);
  p.nxz = cdiv(zmid, kB3);
  p.nxy = cdiv(ymid, L);
  const int blocks = 2 * (p.nzy * p.nzx + p.nyz * p.nyx + p.nxz * p.nxy);
  // the largest staged box, two buffers: a slab of thickness bw (at most) by kB3 by L, widened
  // by t per side, with the row pitch rounded up to odd
  const size_t e = kB3 + 2 * p.t, l = L + 2 * p.t, th = p.bw + 2 * p.t;
  const size_t zy = th * e * (l | 1), xs = e * l * (th | 1);
  const size_t smem = 2 * (zy > xs ? zy : xs) * sizeof(float);
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  if (p.src_off < p.t) return cudaErrorInvalidValue;  // the staged boxes reach t cells outside
  bool star = true;  // only the centre and the six axis neighbours are nonzero
  for (int idx = 0; idx < 27; idx++)
    if ((idx / 9 != 1) + ((idx / 3) % 3 != 1) + (idx % 3 != 1) > 1 && p.w[idx] != 0.f) star = false;
  const auto kern = star ? band3d_kernel<true> : band3d_kernel<false>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  if (blocks > 0) kern<<<blocks, 256, smem, stream>>>(p);
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
    const int rows = star ? SPST_D3_ROWS_STAR : SPST_D3_ROWS_BOX;  // output rows per warp
    // planes per warp: D3SEG, halved (down to 8) while the grid has fewer CTAs than
    // SPST_D3_FILL waves of resident CTAs (SPST_D3_MINB per SM)
    const int64_t cols = (p.W + 127) / 128, rowb = (p.H + DWARPS * rows - 1) / (DWARPS * rows);
    int zseg = D3SEG;
    while (zseg > 8 && cols * rowb * ((p.D + zseg - 1) / zseg) < 152 * SPST_D3_MINB * SPST_D3_FILL) zseg /= 2;
    dim3 g((unsigned)cols, (unsigned)rowb, (unsigned)((p.D + zseg - 1) / zseg));
    if (star)
      direct3d_reg_kernel<true, SPST_D3_ROWS_STAR><<<g, DWARPS * 32, 0, stream>>>(p, in, out, zseg);
    else
      direct3d_reg_kernel<false, SPST_D3_ROWS_BOX><<<g, DWARPS * 32, 0, stream>>>(p, in, out, zseg);
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
