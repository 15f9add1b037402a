// Host planner: Adaptive Layout Morphing (Sec. 3.1), Structured Sparsity Conversion
// (Sec. 3.2) and the kernel-generation tables (Sec. 3.3) for one sweep of a stencil.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace spst {

// Operand encodings of the tensor-core path.
enum class Word { FP16 = 0, BF16 = 1 };

// Geometry of the 2D sweep kernel: one CTA tile is NX x NY patches of R1 x R2 outputs
// (128 x 128 outputs); the MMA is M = R1*R2 = 128 rows (outputs of a patch) by
// N = NX*NY = 128 columns (patches), K = 32 logical (16 stored) per instruction.
struct Tile2D {
  static constexpr int R1 = 16;   // outputs per patch along x
  static constexpr int R2 = 8;    // outputs per patch along y
  static constexpr int NX = 8;    // patches per tile along x
  static constexpr int NY = 16;   // patches per tile along y
  static constexpr int M = R1 * R2;
  static constexpr int N = NX * NY;
  static constexpr int TX = NX * R1;  // 128
  static constexpr int TY = NY * R2;  // 128
  static constexpr int KCHUNK = 32;   // logical K per tcgen05.mma.sp (kind::f16)
};

// Geometry of the 1D sweep kernel: a patch is R1 = 128 consecutive outputs (M = 128 rows); a
// CTA tile is N = 128 patches = 16384 outputs.  The padded line is read through a 2D view of
// rows of ROW floats, so a tile's halo is one TMA box of whole rows.
struct Tile1D {
  static constexpr int R1 = 128;
  static constexpr int N = 128;
  static constexpr int M = R1;
  static constexpr int TX = N * R1;  // 16384
  static constexpr int ROW = 256;    // floats per row of the 2D view
};

// Geometry of the 3D sweep kernel: a patch is R1 x R2 x R3 = 8 x 4 x 4 outputs (x, y, z),
// M = 128 rows; a CTA tile is NX x NY x NZ = 8 x 4 x 4 patches = 64 x 16 x 16 outputs,
// N = 128 columns.
struct Tile3D {
  static constexpr int R1 = 8, R2 = 4, R3 = 4;
  static constexpr int NX = 8, NY = 4, NZ = 4;
  static constexpr int M = R1 * R2 * R3;
  static constexpr int N = NX * NY * NZ;
  static constexpr int TX = NX * R1;  // 64
  static constexpr int TY = NY * R2;  // 16
  static constexpr int TZ = NZ * R3;  // 16
};

// Tables for one sweep kind (t fused steps).
struct SweepTables {
  int ndim = 2;
  int t = 1;        // time steps fused in this sweep
  int R = 1;        // fused radius t*r
  int kt = 3;       // fused stencil width 2R+1
  int r1 = Tile2D::R1, r2 = Tile2D::R2, r3 = 1;
  int g = 0, mb = 0, mz = 1;  // local block size (kt+r1-1), block count (kt+r2-1), z blocks
  int kprime = 0;   // columns of A'
  int kpad = 0;     // K after matching, pair dropping and padding to a multiple of 32
  int zero_cols = 0;       // zero nodes inserted by Algorithm 1
  int dropped_pairs = 0;   // matched pairs whose two columns are both all-zero (removed)
  int bank_conflicts = 0;  // repeated residues left by the chunk packing (0: conflict-free gather)
  int pairing = 0;         // 0: Algorithm 1's pairs; 1: maximum matching on the actual support
  std::vector<double> wfused;     // (2R+1)^ndim composed weights (FP64)
  std::vector<float> wfused32;    // the same rounded to FP32 (the values the pieces split)
  std::vector<int> order;         // kpad: original A' column per permuted position, -1 = zero column
  // Weights as an exact (or as exact as the word allows) sum of up to three 16-bit pieces,
  // w * 2^wscale_log2 = piece0 + piece1 + piece2; pieces that are all zero are dropped.
  int a_pieces = 1;
  int wscale_log2 = 0;
  std::vector<float> a_val[3];    // [M][kpad/2] compressed values per piece (exact 16-bit values as float)
  std::vector<uint8_t> a_idx;     // [M][kpad/2] in-group positions 0..3
  std::vector<uint32_t> a_words;  // [a_pieces][M][kpad/4] packed 16-bit pairs (TMEM image of A'')
  std::vector<uint32_t> meta_words;  // [M lanes][kpad/32] TMEM image of the 2:4 metadata
  std::vector<int32_t> lut;       // [kpad] tile-word offset relative to the patch base
  double S = 0.0;                 // sum of the fused weights (FP64)
  float S_hi = 0.f, S_lo = 0.f;   // S = S_hi + S_lo (FP32 pair), used by the epilogue
};

struct PlanGeometry {
  int ndim = 2;
  int64_t H = 0, W = 0, D = 1;    // grid extents (D = 1 for 2D): z, y, x = D, H, W
  int G = 1;                      // ghost width of the padded ping-pong grids (= max fused radius)
  int64_t Hp = 0, Wp = 0, Dp = 1; // padded extents
  int P = 0;                      // shared-memory tile pitch (floats) = TMA box width
  int box_h = 0;                  // TMA box height
  int64_t tiles_x = 0, tiles_y = 0, tiles_z = 1, num_tiles = 0;
  int box_d = 1;                  // TMA box depth (3D)
  // 2D crush factors (r1 outputs along x by r2 along y per patch, r1 * r2 = 128): (16, 8), the
  // default, or (8, 16); the tile stays 128 x 128 outputs either way
  int r1 = Tile2D::R1, r2 = Tile2D::R2;
};

// Column pairing of the 2:4 conversion: Algorithm 1's pairs, a maximum matching on the
// stencil's actual support, or whichever of the two needs fewer K chunks.
enum class Pairing { Auto = -1, Algorithm1 = 0, Matching = 1 };

// Composes t steps of the offset-indexed cube w (radius r, ndim axes) into one cube of
// radius t*r (FP64): W_{j+1}[o] = sum_{a+b=o} W_j[a] w[b].
std::vector<double> compose_weights(const std::vector<double>& w, int ndim, int r, int t);

// Algorithm 1 (hierarchical two-level matching) on n = m*g nodes; returns the pairs in the
// order M1 (block p ascending, t ascending) then M2 (block ascending, u ascending);
// -1 marks an inserted zero node.
std::vector<std::pair<int, int>> hierarchical_matching(int n, int g, int k);

// Packs matched pairs (with their tile offsets) into the minimum number of K chunks of
// `slots` pairs such that the gather's loads are free of bank conflicts; fills order/lut
// (padding pairs are zero columns) and returns 0, or returns -1 when that is impossible.
int arrange_pairs(const std::vector<std::pair<int, int>>& pairs, const std::vector<std::pair<int, int>>& offs,
                  int slots, std::vector<int>* order_out, std::vector<int32_t>* lut_out);

// Packs pairs into chunks of `slots` pairs with as few bank repeats as a fixed-seed local
// search finds (offsets of -1 mark zero columns, free to read any word); fills order/lut and
// returns the number of repeats.
int pack_pairs_min_repeats(const std::vector<std::pair<int, int>>& pairs, const std::vector<std::pair<int, int>>& offs,
                           int slots, std::vector<int>* order_out, std::vector<int32_t>* lut_out);

// Algorithm 1 applied level by level for a nested staircase (the 3D reading): block pairing
// at the outermost level (sizes[0] blocks of prod(sizes[1..]) columns, stride
// max(floor(m/2), k)), matched blocks paired elementwise, recursion into each unmatched
// block.  For two levels it is hierarchical_matching.
std::vector<std::pair<int, int>> hierarchical_matching_nd(const std::vector<int>& sizes, int k);

// Builds the sweep tables of a 2D (geo.ndim = 2, patches of geo.r1 x geo.r2) or 3D (geo.ndim = 3, Tile3D) stencil
// (fused cube `wfused` of radius R) for the ghost width G, tile pitch P (and box height of a
// 3D tile plane) of `geo`, and operand encoding `word`.  max_pieces: number of 16-bit pieces
// the weights may use (1..3).  Returns an empty string or an error message.
std::string build_sweep_tables_2d(const std::vector<double>& wfused, int R, const PlanGeometry& geo, Word word,
                                  int max_pieces, bool drop_zero_pairs, SweepTables* out,
                                  Pairing pairing = Pairing::Auto);

// Analytical cost model of Sec. 3.3 (T = max(T_compute, T_memory)) for a candidate (r1, r2):
// returns seconds per sweep for an H x W grid.  Used to rank layouts.
double layout_cost_seconds(int kt, int r1, int r2, int64_t H, int64_t W, int kpad, double tensor_flops,
                           double hbm_bytes_per_s, double smem_bytes_per_s);

// Round-to-nearest-even conversions (host side) of an FP32 value to FP16 / BF16, returned
// as the 16-bit pattern and as the exact value in FP32.
uint16_t to_half_bits(float x, Word word);
// TMEM image of the uncompressed permuted A' (the dense-MMA ablation): [a_pieces][M][kpad/2]
// words, column j of lane rho holding K elements 2j (low half) and 2j+1; the 2:4 zeros are
// stored explicitly.
std::vector<uint32_t> dense_a_words(const SweepTables& T, Word word);
// Maximum-cardinality matching of a general graph given by adjacency lists (Edmonds' blossom
// algorithm); returns each vertex's mate, -1 for unmatched vertices.
std::vector<int> max_cardinality_matching(const std::vector<std::vector<int>>& adj);
float half_bits_to_float(uint16_t h, Word word);

}  // namespace spst
