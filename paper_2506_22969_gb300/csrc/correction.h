// Launch interface of the optional FP64 CUDA-core correction step (correction.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace spst {

// One time step in FP64 arithmetic on the plan's padded ping-pong grids.
struct Fp64StepParams {
  int ndim;                 // 1, 2 or 3
  int64_t D, H, W;          // true extents (D = H = 1 below the dimensionality)
  int G;                    // ghost width of both padded grids
  int64_t Wp, Hp;           // padded row length (floats) and padded rows per plane
  int periodic;             // 1: wrapped images in the ghost cells, 0: zero (Dirichlet) ghosts
  int npts;                 // nonzero weights of the single-step stencil
  int off[343][3];          // their offsets (z, y, x), in (dz, dy, dx) lexicographic order
  double w[343];            // their weights (FP64, as given to the planner)
};

// src: a padded grid whose ghost cells hold the boundary images (periodic) or zeros.
// dst_padded (when dst_unpadded is null): every cell of the padded box [0, D+2G) x [0, H+2G)
// x [0, W+2G) receives the step's value at its interior position (wrapped when periodic,
// zero outside a Dirichlet grid), so the next sweep finds its ghosts filled; columns past
// W + 2G are left alone.  dst_unpadded: the D x H x W result only (the run's last step).
cudaError_t launch_fp64_step(const Fp64StepParams& p, const float* src, float* dst_padded, float* dst_unpadded,
                             cudaStream_t stream);

}  // namespace spst
