// Internal launch interface between the host runtime (capi.cpp) and the CUDA kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace spst {

#ifndef SPST_EPI_WARPS
#define SPST_EPI_WARPS 8
#endif
constexpr int kEpiWarps = SPST_EPI_WARPS;  // epilogue warps (4 or 8)
// warps: TMA, MMA, 2 spare, kEpiWarps epilogue, 16 gather
constexpr int kSweepThreads = (4 + kEpiWarps + 16) * 32;
constexpr int kHaloStages = 2;
constexpr int kMaxBSlots = 8;        // ring of B'' K chunks (the launcher fills the shared memory left)
constexpr int kPieceBytes = 16 * 576;  // one K-chunk (32 x 128, 16-bit) of B' in the padded K-major layout
constexpr int kLBO = 144;              // bytes between K-adjacent core matrices
constexpr int kSBO = 576;              // bytes between 8-patch groups

struct Sweep2DParams {
  int H, W;             // true grid extents (rows, columns)
  int D;                // planes (3D; 1 for 2D)
  int dim3;             // 1: 3D sweep (Tile3D patches and tiles, 3D TMA box)
  int dim1;             // 1: 1D sweep (Tile1D patches and tiles, rows of the 2D view of the line)
  int tall;             // 2D: 1 = 8 x 16 patches (16 across, 8 down a tile), 0 = 16 x 8 (8 across, 16 down)
  int G;                // ghost width of the input padded grid
  int tiles_x, tiles_y, tiles_z, num_tiles;
  int P, box_h, box_d;  // shared-memory tile pitch (floats), height (rows), depth (planes) = TMA box
  int kpad, kchunks;    // K after padding, number of 32-wide chunks
  int a_pieces;         // 16-bit pieces of the weights resident in TMEM (1..3)
  int b_pieces;         // 16-bit pieces of the grid data per B'' element (1: single word, 2: hi + lo)
  int nterms;           // MMAs per K chunk; term i multiplies A piece term_a[i] by B piece term_b[i]
  int term_a[4], term_b[4];
  int nacc;             // TMEM accumulators (2: the epilogue of one tile overlaps the next tile's MMAs)
  int dense;            // 1: the dense-MMA ablation (uncompressed A' in TMEM, dense kind::f16, K = 16)
  int lo_acc;           // split operands: 1 = the terms after the first go to a low-order accumulator
                        // (128 columns after the main one) that the epilogue adds in FP32; nacc = 1
  int nslots;           // B'' chunk slots in shared memory (1..kMaxBSlots; set by launch_sweep2d)
  int early_tma;        // 1: tile 0's halo load is issued before the set-up (set by launch_sweep2d)
  int hstages;          // halo tile stages in shared memory: 2 (the next tile loads during the gather) or 1
  int fp16;             // operand type: 1 = FP16, 0 = BF16
  float wscale;         // 2^-s: the weight pieces hold w * 2^s
  const int32_t* lut;         // [kpad] tile-word offsets (device)
  const uint32_t* a_words;    // [pieces][128][kpad/4] TMEM image of A'' (device)
  const uint32_t* meta_words; // [128][kchunks] TMEM image of the metadata (device)
  float S_hi, S_lo;     // sum of the sweep's weights as an FP32 pair
  float* out;           // output grid base
  int64_t out_pitch;    // floats per output row
  int64_t out_plane;    // floats per output plane (3D)
  int out_off;          // ghost width of the output grid (0 for an unpadded grid)
  int out_ghost;        // 1: periodic padded output, also write the ghost images
  // FP16 operands: the grid data enter B'' scaled by 2^k, k = floor(log2(2^13 / (2 max|u0|
  // growth))), so that hi and lo pieces stay normal; max|u0| is read from *maxabs (written by
  // the copy-in), growth bounds max|u| / max|u0| over the run (sum of |w| to the power of
  // the steps).  maxabs null: k = 0.
  const unsigned* maxabs;
  float growth;
  int* status;          // device status word
  unsigned long long wait_ns;  // bound of every device-side wait
};

// A batch launch: up to kMultiMaxJobs grids swept by one launch of at most kMultiMaxCtas CTAs
// (job j gets CTAs cta_first[j] .. cta_first[j] + cta_count[j] - 1).  Passed by value as the
// kernel's parameter block (about 23 KB).
constexpr int kMultiMaxJobs = 64, kMultiMaxCtas = 256;
struct MultiSweepParams {
  CUtensorMap tmap[kMultiMaxJobs];  // 64-byte aligned: first member
  Sweep2DParams job[kMultiMaxJobs];
  int cta_first[kMultiMaxJobs], cta_count[kMultiMaxJobs];
  int16_t cta_job[kMultiMaxCtas];
  int njobs, nctas;
};
// Launches one batch sweep: job j's sweep with tensor map maps[j] and parameters prm[j] (the
// jobs share the kernel template: FP16 or BF16, single or split words, dimensionality).  The
// SMs are shared out by tile count (each job gets at least one CTA).  Returns the launch error.
cudaError_t launch_sweep2d_multi(const CUtensorMap* maps, const Sweep2DParams* prm, int njobs, int num_sms,
                                 cudaStream_t stream);

// Shared-memory bytes the sweep kernel needs for this geometry (with p.nslots chunk slots).
size_t sweep2d_smem_bytes(const Sweep2DParams& p);
// Largest chunk-slot count (<= kMaxBSlots) that fits the per-CTA shared memory, or 0.
int sweep2d_max_slots(const Sweep2DParams& p);
// Whether the sweep kernel fits shared memory for this geometry (p.hstages halo stages,
// >= 2 chunk slots, and the set-up staging of A'' and the metadata).
bool sweep2d_fits(const Sweep2DParams& p);
// Halo stages for this geometry: 2 where they fit beside the chunk slots, else 1, else 0.
int sweep2d_halo_stages(const Sweep2DParams& p);
// Whether launch_sweep2d lets a sweep overlap its set-up with the previous kernel
// (programmatic dependent launch; on by default, per host thread).
void sweep2d_set_programmatic_launch(bool on);
// Launches one sparse sweep (grid = min(num_tiles, SMs)); returns the launch error.
cudaError_t launch_sweep2d(const CUtensorMap& tmap_in, const Sweep2DParams& p, int num_sms, cudaStream_t stream);

// Timeline trace of CTA 0 of the sweep kernel (debugging aid): enable/disable (clears the
// buffer) and read up to n entries ([role][tile][start, end], roles TMA, MMA, gather, epilogue).
cudaError_t sweep_trace_enable(int on);
cudaError_t sweep_trace_read(unsigned long long* out, int n);

// Copies an unpadded H x W grid into a padded (H+2G) x Wp grid: interior, ghosts (periodic
// images or zeros) and the slack columns (zeros).
// maxabs (may be null): receives max |in| (atomicMax on the float bits; the caller zeroes it).
cudaError_t launch_pad_copy2d(const float* in, float* padded, int H, int W, int G, int64_t Wp, int periodic,
                              unsigned* maxabs, cudaStream_t stream);
// 3D copy-in: unpadded D x H x W -> padded (D + 2G) x (H + 2G) x Wp.
cudaError_t launch_pad_copy3d(const float* in, float* padded, int D, int H, int W, int G, int64_t Wp, int periodic,
                              unsigned* maxabs, cudaStream_t stream);
// Rewrites the periodic ghost shell of a padded 3D grid from its interior.
cudaError_t launch_ghost_refresh3d(float* padded, int D, int H, int W, int G, int64_t Wp, cudaStream_t stream);

struct DirectParams {
  int ndim;
  int64_t D, H, W;      // extents (D = 1 for 2D)
  int radius;
  int periodic;
  int npts;
  int off[343][3];      // offsets (z, y, x) of the nonzero weights
  float w[343];         // their weights (FP32 FMAs in this order)
  float wdense[81];     // the dense cube (zeros included): 1D 2r+1 and 2D (2r+1)^2 for r <= 4, 3D 27 for r = 1
};
// 1D copy-in of a line of W cells into its padded copy (G ghost cells each side, length Wp),
// periodic images or zeros in the ghosts, and max |in| into *maxabs when it is not null.
cudaError_t launch_pad_copy1d(const float* in, float* out, int64_t W, int G, int64_t Wp, int periodic,
                              unsigned* maxabs, cudaStream_t stream);
// Periodic 1D: copies the wrapped images into the G ghost cells at each end of a padded line.
cudaError_t launch_ghost_refresh1d(float* line, int64_t W, int G, cudaStream_t stream);
// One FP32 CUDA-core step in -> out.
cudaError_t launch_direct_step(const DirectParams& p, const float* in, float* out, cudaStream_t stream);

// Dirichlet band of a fused sweep of depth t >= 2: exact step-by-step FP32 values in the
// frame of width bw = (t-1)*radius inside the grid edges, from the sweep's input.
struct BandParams {
  const float* src;       // the sweep's input grid
  int64_t src_pitch;      // floats per row of src
  int src_off;            // ghost width of src (cell (0,0) at src[src_off * src_pitch + src_off])
  float* dst;             // the sweep's output grid (band cells overwritten)
  int64_t dst_pitch;
  int dst_off;
  int H, W;
  int radius, t, bw;
  int seg, nx, ny;        // set by launch_band2d
  float w[81];            // single-step weights, dense (2r+1)^2 [dy][dx], r <= 4
};
cudaError_t launch_band2d(BandParams p, cudaStream_t stream);

// 3D, radius 1: the Dirichlet frame of width bw = t - 1 on the six faces of a fused sweep of
// depth t >= 2, recomputed step by step in FP32 from the sweep's input.
struct Band3DParams {
  const float* src;       // the sweep's input grid (padded: ghost width src_off, zeros outside)
  int64_t src_pitch, src_plane;
  int src_off;
  float* dst;             // the sweep's output grid (frame cells overwritten)
  int64_t dst_pitch, dst_plane;
  int dst_off;
  int D, H, W;
  int t, bw;
  int nzx, nzy, nyz, nyx, nxz, nxy;  // chunk counts of the z, y and x slabs (set by launch_band3d)
  float w[27];            // single-step weights, dense 3 x 3 x 3 [dz][dy][dx]
};
cudaError_t launch_band3d(Band3DParams p, cudaStream_t stream);

// FP64 norms of x against ref (see sparstencil_error_norms); acc: 4 doubles of device memory.
cudaError_t launch_error_norms(const float* x, const float* ref, int64_t n, double* acc, cudaStream_t stream);

// Address of the library's device status word on the current device.
int* device_status_word();
// Address of the 4-double norm accumulator on the current device.
double* device_norm_accumulator();

}  // namespace spst
