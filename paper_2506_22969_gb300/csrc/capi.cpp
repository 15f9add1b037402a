// C ABI of the SparStencil GB300 library: plans, workspaces and sweep scheduling.
#include "sparstencil.h"

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <list>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "correction.h"
#include "kernels.h"
#include "planner.h"

using spst::PlanGeometry;
using spst::SweepTables;
using spst::Tile2D;
using spst::Tile1D;
using spst::Tile3D;

namespace {

thread_local std::string g_last_error;
uint64_t g_wait_ns = 2000000000ull;

sparstencil_status fail(sparstencil_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

sparstencil_status cuda_fail(cudaError_t e, const char* what) {
  return fail(SPST_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SPST_CUDA(call, what)                      \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_tiled() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

struct DeviceTables {
  int32_t* lut = nullptr;
  uint32_t* a_words = nullptr;
  uint32_t* meta = nullptr;
  void release() {
    cudaFree(lut);
    cudaFree(a_words);
    cudaFree(meta);
    lut = nullptr;
    a_words = nullptr;
    meta = nullptr;
  }
};

bool is_split(sparstencil_dtype d) { return d == SPST_FP16_SPLIT || d == SPST_BF16_SPLIT; }

// Programmatic dependent launch between sweeps: on, except while a CUDA graph is captured
// (this thread's setting, mirrored here so that a run can restore it)
thread_local bool t_pdl_on = true;
void set_programmatic_launch(bool on) {
  t_pdl_on = on;
  spst::sweep2d_set_programmatic_launch(on);
}

// TMEM columns: accumulators (128 each) + A'' pieces + metadata (8-column pairs of chunks),
// or for the dense ablation the uncompressed A' pieces (K/2 columns each) and no metadata.
// Returns the tile buffers that fit in the 512 columns: two accumulators when they fit, else
// one, else 0 (does not fit); with the low-order accumulator (lo) a tile takes 256 columns
// and there is at most one buffer.
int tmem_accumulators(const SweepTables& T, bool lo = false, bool dense = false) {
  const int rest = dense ? T.a_pieces * (T.kpad / 2) : T.a_pieces * (T.kpad / 4) + 8 * ((T.kpad / 32 + 1) / 2);
  if (lo) return 256 + rest <= 512 ? 1 : 0;
  if (256 + rest <= 512) return 2;
  if (128 + rest <= 512) return 1;
  return 0;
}
spst::Word word_of(sparstencil_dtype d) {
  return (d == SPST_FP16 || d == SPST_FP16_SPLIT) ? spst::Word::FP16 : spst::Word::BF16;
}

}  // namespace

namespace {
std::atomic<uint64_t> g_plan_uid{1};
}

struct sparstencil_plan_s {
  uint64_t uid = g_plan_uid.fetch_add(1);  // never reused (keys the batch graph cache)
  sparstencil_shape shape;
  int ndim = 2, radius = 1;
  sparstencil_dtype dtype;
  sparstencil_boundary bc;
  int requested_t = 1, t = 1, t_max = 1;
  bool lo_acc = false;  // split operands: low-order MMA terms in an accumulator of their own
  int fp64_every = 0;   // k > 0: every k-th time step of a run is an FP64 CUDA-core step
  bool dense = false;   // the dense-MMA ablation (uncompressed A', dense tcgen05 MMAs)
  bool autotune_pending = false;  // fusion_depth 0: t (and the layout) chosen by timing at the first run
  spst::Pairing pairing_pref = spst::Pairing::Auto;  // column pairing of the 2:4 conversion
  bool layout_fixed = false;  // set by sparstencil_plan_set_layout: the search keeps this layout
  std::vector<double> w64;  // input weights (FP32 values promoted exactly)
  PlanGeometry geo;
  SweepTables full;
  std::map<int, SweepTables> rem;  // remainder sweeps keyed by depth
  double planner_ms = 0.0;
  // device state
  int device = -1, num_sms = 0;
  std::map<int, DeviceTables> dev_tables;  // keyed by sweep depth
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_owned = false;
  bool ws_ready = false;
  CUtensorMap tmap[2];
  float* stage_in = nullptr;
  float* stage_out = nullptr;
  unsigned* maxabs = nullptr;  // FP16 operands: max |input| of the current run (device word)
  float growth = 1.f;          // bound on max|u| / max|u0| over the current run

  ~sparstencil_plan_s() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (device >= 0) cudaSetDevice(device);
    for (auto& kv : dev_tables) kv.second.release();
    if (ws_owned) cudaFree(ws);
    cudaFree(stage_in);
    cudaFree(stage_out);
    cudaFree(maxabs);
    if (cur >= 0) cudaSetDevice(cur);
  }

  size_t grid_floats() const { return (size_t)geo.Dp * (size_t)geo.Hp * (size_t)geo.Wp; }
  size_t cells() const { return (size_t)geo.D * (size_t)geo.H * (size_t)geo.W; }
  float* pad(int i) const { return (float*)((char*)ws + (size_t)i * ((grid_floats() * 4 + 255) & ~(size_t)255)); }
};

namespace {

// Process-wide cache of planner tables.  The tables depend on the composed weights, the
// fused radius, the word, the piece count and the tile geometry (pitch, box height, ghost
// width), not on the grid's extents, so plans of one stencil on grids of different sizes
// (a job server's usual load) share them.  Bounded: cleared when it holds kTableCacheMax sets.
constexpr size_t kTableCacheMax = 64;
std::mutex g_table_cache_mu;
std::map<std::string, SweepTables> g_table_cache;

std::string tables_cached(const std::vector<double>& wf, int R, const PlanGeometry& geo, spst::Word word, int pieces,
                          SweepTables* out, spst::Pairing pairing) {
  std::string key;
  auto put = [&](const void* q, size_t n) { key.append((const char*)q, n); };
  const int ints[8] = {R, geo.ndim, geo.P, geo.box_h, geo.G, pieces, geo.r1, (int)pairing};
  put(ints, sizeof(ints));
  put(&word, sizeof(word));
  put(wf.data(), wf.size() * sizeof(double));
  {
    std::lock_guard<std::mutex> lock(g_table_cache_mu);
    auto it = g_table_cache.find(key);
    if (it != g_table_cache.end()) {
      *out = it->second;
      return "";
    }
  }
  std::string err = spst::build_sweep_tables_2d(wf, R, geo, word, pieces, true, out, pairing);
  if (!err.empty()) return err;
  std::lock_guard<std::mutex> lock(g_table_cache_mu);
  if (g_table_cache.size() >= kTableCacheMax) g_table_cache.clear();
  g_table_cache.emplace(std::move(key), *out);
  return "";
}

// Inputs one patch's outputs read through the composed stencil wf of radius R (the nonzero
// columns of A', a lower bound on K_pad): |patch + support(wf)|, counted on a bitmap.
int64_t patch_inputs(const std::vector<double>& wf, int ndim, int R, const PlanGeometry& geo) {
  const int kt = 2 * R + 1;
  const int r1 = ndim == 1 ? Tile1D::R1 : ndim == 2 ? geo.r1 : Tile3D::R1;
  const int r2 = ndim == 1 ? 1 : ndim == 2 ? geo.r2 : Tile3D::R2;
  const int r3 = ndim == 3 ? Tile3D::R3 : 1;
  const int kz = ndim == 3 ? kt : 1, ky = ndim >= 2 ? kt : 1;
  const int bx = r1 + kt - 1, by = r2 + ky - 1, bz = r3 + kz - 1;
  std::vector<char> hit((size_t)bx * by * bz, 0);
  for (int z = 0; z < kz; z++)
    for (int y = 0; y < ky; y++)
      for (int x = 0; x < kt; x++) {
        if (wf[((size_t)z * ky + y) * kt + x] == 0.0) continue;
        for (int oz = 0; oz < r3; oz++)
          for (int oy = 0; oy < r2; oy++)
            for (int ox = 0; ox < r1; ox++) hit[((size_t)(z + oz) * by + (y + oy)) * bx + (x + ox)] = 1;
      }
  int64_t n = 0;
  for (char h : hit) n += h;
  return n;
}

std::string build_tables(sparstencil_plan_t p, int depth, SweepTables* out) {
  std::vector<double> wf = spst::compose_weights(p->w64, p->ndim, p->radius, depth);
  {
    // cheap rejection before the matching: even with the fewest pieces (two) and no zero
    // columns, K_pad >= the patch's input count, and the A'' pieces, metadata and one
    // accumulator must fit the 512 TMEM columns
    const int64_t kmin = (patch_inputs(wf, p->ndim, depth * p->radius, p->geo) + 31) / 32 * 32;
    const int64_t need = (p->dense ? 2 * (kmin / 2) : 2 * (kmin / 4) + 8 * ((kmin / 32 + 1) / 2)) +
                         (p->lo_acc ? 256 : 128);
    if (need > 512) return std::string("stencil too wide for TMEM (kpad >= ") + std::to_string(kmin) + ")";
  }
  // Weight pieces: single-word operands use two 16-bit pieces.  BF16 split operands use three
  // (exact for FP32 weights); FP16 split operands two, which hold 22 significant bits of each
  // scaled weight: a third FP16 piece sits below the rounding of the FP32 accumulator it is
  // added to and would only cost an MMA term.  A fused BF16 split sweep (t >= 2) whose three
  // pieces would leave TMEM room for only one accumulator uses two: the second accumulator lets
  // the next tile's MMAs overlap this tile's write-back and the fourth MMA term goes away,
  // while the weight rounding (<= 2^-17 relative per fused weight) is shared by t steps;
  // measured on the periodic Fourier closed form over 100 steps at t = 3 the rel-L2 error stays
  // below 1e-6.
  // With the low-order accumulator a tile's two accumulators take 256 columns, and the dense
  // ablation's uncompressed A' takes twice the columns; in every case two pieces replace three
  // when they leave room for more tile buffers.
  const int pieces = (is_split(p->dtype) && word_of(p->dtype) == spst::Word::BF16) ? 3 : 2;
  std::string err = tables_cached(wf, depth * p->radius, p->geo, word_of(p->dtype), pieces, out, p->pairing_pref);
  if (!err.empty()) return err;
  const int buffers3 = tmem_accumulators(*out, p->lo_acc, p->dense);
  const bool retry = buffers3 == 0 || (!p->lo_acc && depth >= 2 && buffers3 < 2);
  if (pieces == 3 && retry) {
    SweepTables two;
    err = tables_cached(wf, depth * p->radius, p->geo, word_of(p->dtype), 2, &two, p->pairing_pref);
    if (!err.empty()) return err;
    if (tmem_accumulators(two, p->lo_acc, p->dense) > tmem_accumulators(*out, p->lo_acc, p->dense))
      *out = std::move(two);
  }
  out->t = depth;
  if (tmem_accumulators(*out, p->lo_acc, p->dense) == 0)
    return std::string("stencil too wide for TMEM (kpad ") + std::to_string(out->kpad) +
           (p->lo_acc ? ", with the low-order accumulator)" : ")");
  return "";
}

// Geometry of the padded ping-pong grids and halo tiles for ghost width t_max * radius;
// returns an empty string or the reason the grid cannot be planned.
std::string plan_geometry(sparstencil_plan_t p) {
  PlanGeometry& g = p->geo;
  const bool d3 = g.ndim == 3;
  g.G = p->t_max * p->radius;
  if (g.G > 60) return "fused radius too large";
  if (g.ndim == 1) {
    // the padded line (G ghost cells each side) is read as rows of Tile1D::ROW floats; a
    // tile's halo is the whole rows covering its 16384 outputs and 2G ghosts
    if (g.W < 2 * g.G || g.W < 4) return "grid smaller than twice the fused radius";
    if (g.W > (1ll << 30)) return "grid extent too large";
    g.Dp = g.Hp = 1;
    g.Wp = (g.W + 2 * g.G + Tile1D::ROW - 1) / Tile1D::ROW * Tile1D::ROW;
    g.P = Tile1D::ROW;
    g.box_h = (Tile1D::TX + 2 * g.G + Tile1D::ROW - 1) / Tile1D::ROW;
    g.box_d = 1;
    g.tiles_x = (g.W + Tile1D::TX - 1) / Tile1D::TX;
    g.tiles_y = g.tiles_z = 1;
    g.num_tiles = g.tiles_x;
    if (g.num_tiles > (1ll << 30)) return "too many tiles";
    return "";
  }
  if (g.H < 2 * g.G || g.W < 2 * g.G || g.W < 4 || (d3 && g.D < 2 * g.G))
    return "grid smaller than twice the fused radius";
  if (g.H > (1 << 30) || g.W > (1 << 30) || g.D > (1 << 30)) return "grid extent too large";
  g.Hp = g.H + 2 * g.G;
  g.Dp = d3 ? g.D + 2 * g.G : 1;
  g.Wp = ((g.W + 2 * g.G) + 3) / 4 * 4;
  const int tx = d3 ? Tile3D::TX : Tile2D::TX, ty = d3 ? Tile3D::TY : Tile2D::TY;
  g.P = (tx + 2 * g.G + 3) / 4 * 4;
  g.box_h = ty + 2 * g.G;
  g.box_d = d3 ? Tile3D::TZ + 2 * g.G : 1;
  g.tiles_x = (g.W + tx - 1) / tx;
  g.tiles_y = (g.H + ty - 1) / ty;
  g.tiles_z = d3 ? (g.D + Tile3D::TZ - 1) / Tile3D::TZ : 1;
  g.num_tiles = g.tiles_x * g.tiles_y * g.tiles_z;
  if (g.num_tiles > (1ll << 30)) return "too many tiles";
  return "";
}

const SweepTables* tables_for(sparstencil_plan_t p, int depth, std::string* err) {
  if (depth == p->t) return &p->full;
  auto it = p->rem.find(depth);
  if (it != p->rem.end()) return &it->second;
  SweepTables T;
  *err = build_tables(p, depth, &T);
  if (!err->empty()) return nullptr;
  return &(p->rem[depth] = std::move(T));
}

// Uploads a depth's tables on first use.  The copies are ordered on `stream`, ahead of the
// kernels that read them (the host vectors are pageable: each copy is staged before the
// call returns).
sparstencil_status ensure_device_tables(sparstencil_plan_t p, int depth, const SweepTables& T, DeviceTables** out,
                                        cudaStream_t stream) {
  // keyed by depth and layout (patch shape, pairing): the fusion-depth search times several
  auto& dt = p->dev_tables[depth * 8 + (p->geo.r1 == 8 ? 4 : 0) + ((int)p->pairing_pref + 1)];
  if (!dt.lut) {
    const std::vector<uint32_t> dense_words = p->dense ? spst::dense_a_words(T, word_of(p->dtype)) : std::vector<uint32_t>();
    const std::vector<uint32_t>& aw = p->dense ? dense_words : T.a_words;
    SPST_CUDA(cudaMalloc(&dt.lut, T.lut.size() * 4), "cudaMalloc(lut)");
    SPST_CUDA(cudaMalloc(&dt.a_words, aw.size() * 4), "cudaMalloc(a_words)");
    SPST_CUDA(cudaMalloc(&dt.meta, T.meta_words.size() * 4), "cudaMalloc(meta)");
    SPST_CUDA(cudaMemcpyAsync(dt.lut, T.lut.data(), T.lut.size() * 4, cudaMemcpyHostToDevice, stream), "upload lut");
    SPST_CUDA(cudaMemcpyAsync(dt.a_words, aw.data(), aw.size() * 4, cudaMemcpyHostToDevice, stream), "upload A''");
    SPST_CUDA(cudaMemcpyAsync(dt.meta, T.meta_words.data(), T.meta_words.size() * 4, cudaMemcpyHostToDevice, stream),
              "upload metadata");
  }
  *out = &dt;
  return SPST_OK;
}

// Dirichlet band of a sweep of depth `depth` (nothing to do for periodic grids or depth 1):
// src is the sweep's input (padded), dst its output.
cudaError_t launch_band(sparstencil_plan_t p, int depth, const float* src, float* dst, int64_t dst_pitch, int dst_off,
                        cudaStream_t stream) {
  if (p->bc != SPST_DIRICHLET_ZERO || depth < 2) return cudaSuccess;
  spst::BandParams b;
  std::memset(&b, 0, sizeof(b));
  b.src = src;
  b.src_pitch = p->geo.Wp;
  b.src_off = p->geo.G;
  b.dst = dst;
  b.dst_pitch = dst_pitch;
  b.dst_off = dst_off;
  b.H = (int)p->geo.H;
  b.W = (int)p->geo.W;
  b.radius = p->radius;
  b.t = depth;
  b.bw = (depth - 1) * p->radius;
  for (size_t i = 0; i < p->w64.size() && i < 81; i++) b.w[i] = (float)p->w64[i];
  return spst::launch_band2d(b, stream);
}

sparstencil_status make_tmaps(sparstencil_plan_t p) {
  EncodeTiledFn enc = get_encode_tiled();
  if (!enc) return fail(SPST_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  const PlanGeometry& g = p->geo;
  for (int i = 0; i < 2; i++) {
    CUresult r;
    if (g.ndim == 1) {
      cuuint64_t gdim[2] = {(cuuint64_t)Tile1D::ROW, (cuuint64_t)(g.Wp / Tile1D::ROW)};
      cuuint64_t gstr[1] = {(cuuint64_t)Tile1D::ROW * 4};
      cuuint32_t box[2] = {(cuuint32_t)g.P, (cuuint32_t)g.box_h};
      cuuint32_t es[2] = {1, 1};
      r = enc(&p->tmap[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p->pad(i), gdim, gstr, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else if (g.ndim == 3) {
      cuuint64_t gdim[3] = {(cuuint64_t)g.Wp, (cuuint64_t)g.Hp, (cuuint64_t)g.Dp};
      cuuint64_t gstr[2] = {(cuuint64_t)g.Wp * 4, (cuuint64_t)g.Wp * (cuuint64_t)g.Hp * 4};
      cuuint32_t box[3] = {(cuuint32_t)g.P, (cuuint32_t)g.box_h, (cuuint32_t)g.box_d};
      cuuint32_t es[3] = {1, 1, 1};
      r = enc(&p->tmap[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, p->pad(i), gdim, gstr, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
      cuuint64_t gdim[2] = {(cuuint64_t)g.Wp, (cuuint64_t)g.Hp};
      cuuint64_t gstr[1] = {(cuuint64_t)g.Wp * 4};
      cuuint32_t box[2] = {(cuuint32_t)g.P, (cuuint32_t)g.box_h};
      cuuint32_t es[2] = {1, 1};
      r = enc(&p->tmap[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p->pad(i), gdim, gstr, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) return fail(SPST_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  }
  return SPST_OK;
}

sparstencil_status ensure_device(sparstencil_plan_t p, cudaStream_t stream) {
  int dev = 0;
  SPST_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (p->device >= 0 && p->device != dev) return fail(SPST_ERR_INVALID, "plan is bound to another device");
  if (p->device < 0) {
    cudaDeviceProp prop;
    SPST_CUDA(cudaGetDeviceProperties(&prop, dev), "cudaGetDeviceProperties");
    if (prop.major != 10 || prop.minor != 3)
      return fail(SPST_ERR_UNSUPPORTED, "this library is built for sm_103a (GB300)");
    p->device = dev;
    p->num_sms = prop.multiProcessorCount;
  }
  if (!p->ws) {
    size_t need = sparstencil_workspace_bytes(p);
    void* w = nullptr;
    if (cudaMalloc(&w, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(SPST_ERR_NOMEM, "workspace allocation failed");
    }
    p->ws = w;
    p->ws_bytes = need;
    p->ws_owned = true;
    SPST_CUDA(cudaMemsetAsync(w, 0, need, stream), "zero workspace");
    p->ws_ready = false;
  }
  if (!p->maxabs && word_of(p->dtype) == spst::Word::FP16) {
    void* m = nullptr;
    if (cudaMalloc(&m, sizeof(unsigned)) != cudaSuccess) {
      cudaGetLastError();
      return fail(SPST_ERR_NOMEM, "allocation of the data-scale word failed");
    }
    p->maxabs = (unsigned*)m;
  }
  if (!p->ws_ready) {
    sparstencil_status s = make_tmaps(p);
    if (s != SPST_OK) return s;
    p->ws_ready = true;
  }
  return SPST_OK;
}

// Optional per-launch timing: events[0] before the copy-in, events[i+1] after launch i.
struct LaunchTimer {
  std::vector<cudaEvent_t> ev;
  int sweeps = 0;  // sweep launches between the second and the last event
  sparstencil_status record(cudaStream_t s) {
    cudaEvent_t e;
    SPST_CUDA(cudaEventCreate(&e), "cudaEventCreate");
    ev.push_back(e);
    SPST_CUDA(cudaEventRecord(e, s), "cudaEventRecord");
    return SPST_OK;
  }
  ~LaunchTimer() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};

// Launch parameters of a sweep of depth T.depth that depend only on the plan and the tables.
spst::Sweep2DParams sweep_params(sparstencil_plan_t p, const SweepTables& T, const DeviceTables& dt, int* status) {
  const PlanGeometry& g = p->geo;
  spst::Sweep2DParams prm;
  std::memset(&prm, 0, sizeof(prm));
  prm.H = (int)g.H;
  prm.W = (int)g.W;
  prm.D = (int)g.D;
  prm.dim3 = g.ndim == 3 ? 1 : 0;
  prm.dim1 = g.ndim == 1 ? 1 : 0;
  prm.tall = (g.ndim == 2 && g.r1 == 8) ? 1 : 0;
  prm.G = g.G;
  prm.tiles_x = (int)g.tiles_x;
  prm.tiles_y = (int)g.tiles_y;
  prm.tiles_z = (int)g.tiles_z;
  prm.num_tiles = (int)g.num_tiles;
  prm.P = g.P;
  prm.box_h = g.box_h;
  prm.box_d = g.box_d;
  prm.kpad = T.kpad;
  prm.kchunks = T.kpad / 32;
  prm.a_pieces = T.a_pieces;
  prm.b_pieces = is_split(p->dtype) ? 2 : 1;
  prm.nterms = 0;
  prm.term_a[prm.nterms] = 0;
  prm.term_b[prm.nterms++] = 0;
  if (prm.b_pieces == 2) {
    prm.term_a[prm.nterms] = 0;
    prm.term_b[prm.nterms++] = 1;
  }
  for (int pc = 1; pc < T.a_pieces; pc++) {
    prm.term_a[prm.nterms] = pc;
    prm.term_b[prm.nterms++] = 0;
  }
  prm.nacc = tmem_accumulators(T, p->lo_acc, p->dense);
  prm.lo_acc = p->lo_acc ? 1 : 0;
  prm.dense = p->dense ? 1 : 0;
  prm.fp16 = word_of(p->dtype) == spst::Word::FP16 ? 1 : 0;
  prm.wscale = std::ldexp(1.0f, -T.wscale_log2);
  prm.lut = dt.lut;
  prm.a_words = dt.a_words;
  prm.meta_words = dt.meta;
  prm.S_hi = T.S_hi;
  prm.S_lo = T.S_lo;
  prm.maxabs = p->maxabs;
  prm.growth = p->growth;
  prm.status = status;
  prm.wait_ns = g_wait_ns;
  prm.hstages = spst::sweep2d_halo_stages(prm);
  return prm;
}

// Fusion-depth search of a plan made with fusion_depth 0 (the layout search of Sec. 3.3,
// done by measurement): copies `in` into the padded grid, times two sweeps of every
// candidate depth after one warm-up sweep, and keeps the depth with the least time per time
// step.  Synchronises the stream; the caller's run then starts from a fresh copy-in.
// Copy-in of a caller grid into the plan's padded grid `pad` (2D or 3D).
// FP16 plans also record max |in| for the data scale (see Sweep2DParams::maxabs), and
// `steps` (the run's time steps) bounds its growth: max|u| <= max|u0| * (sum |w|)^steps.
cudaError_t copy_in(sparstencil_plan_t p, const float* in, float* pad, int64_t steps, cudaStream_t stream,
                    unsigned* maxabs) {
  const PlanGeometry& g = p->geo;
  const int periodic = p->bc == SPST_PERIODIC ? 1 : 0;
  if (maxabs) {
    cudaError_t e = cudaMemsetAsync(maxabs, 0, sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    double sabs = 0.0;
    for (double w : p->w64) sabs += std::fabs(w);
    const double growth = std::pow(std::max(sabs, 1.0), (double)steps);
    p->growth = (float)std::min(growth, 1e30);
  }
  if (g.ndim == 1) return spst::launch_pad_copy1d(in, pad, g.W, g.G, g.Wp, periodic, maxabs, stream);
  if (g.ndim == 3)
    return spst::launch_pad_copy3d(in, pad, (int)g.D, (int)g.H, (int)g.W, g.G, g.Wp, periodic, maxabs, stream);
  return spst::launch_pad_copy2d(in, pad, (int)g.H, (int)g.W, g.G, g.Wp, periodic, maxabs, stream);
}

// Output parameters of a sweep that writes the padded grid `pad` (or, last, the caller's
// unpadded `out`).  A 3D sweep writes the interior only; its periodic ghost shell is then
// refreshed by after_sweep.
void set_output(sparstencil_plan_t p, spst::Sweep2DParams* prm, float* pad, float* out, bool last) {
  const PlanGeometry& g = p->geo;
  prm->out = last ? out : pad;
  prm->out_pitch = last ? g.W : g.Wp;
  prm->out_plane = last ? g.W * g.H : g.Wp * g.Hp;
  prm->out_off = last ? 0 : g.G;
  prm->out_ghost = (!last && p->bc == SPST_PERIODIC && g.ndim == 2) ? 1 : 0;
}

// Work after a sweep of depth `depth` from padded grid `src` into prm.out: the Dirichlet band
// of a fused 2D sweep, or the periodic ghost shell of a 3D padded output.
cudaError_t after_sweep(sparstencil_plan_t p, int depth, const float* src, const spst::Sweep2DParams& prm, bool last,
                        cudaStream_t stream) {
  const PlanGeometry& g = p->geo;
  if (g.ndim == 1) {
    if (last || p->bc != SPST_PERIODIC) return cudaSuccess;
    return spst::launch_ghost_refresh1d(prm.out, g.W, g.G, stream);
  }
  if (g.ndim == 3) {
    if (p->bc == SPST_DIRICHLET_ZERO) {
      if (depth < 2) return cudaSuccess;
      spst::Band3DParams b;
      std::memset(&b, 0, sizeof(b));
      b.src = src;
      b.src_pitch = g.Wp;
      b.src_plane = g.Wp * g.Hp;
      b.src_off = g.G;
      b.dst = prm.out;
      b.dst_pitch = prm.out_pitch;
      b.dst_plane = prm.out_plane;
      b.dst_off = prm.out_off;
      b.D = (int)g.D;
      b.H = (int)g.H;
      b.W = (int)g.W;
      b.t = depth;
      b.bw = depth - 1;
      for (size_t i = 0; i < p->w64.size() && i < 27; i++) b.w[i] = (float)p->w64[i];
      return spst::launch_band3d(b, stream);
    }
    if (last) return cudaSuccess;
    return spst::launch_ghost_refresh3d(prm.out, (int)g.D, (int)g.H, (int)g.W, g.G, g.Wp, stream);
  }
  return launch_band(p, depth, src, prm.out, prm.out_pitch, prm.out_off, stream);
}

// Depths the first run of an autotuned plan times: every depth up to the plan's maximum, or
// in 1D (where the maximum reaches 60 / radius) the powers of two below it and the maximum.
std::vector<int> autotune_depths(const sparstencil_plan_s* p) {
  std::vector<int> d;
  for (int t = 1; t <= p->t_max; t = p->geo.ndim == 1 ? 2 * t : t + 1) d.push_back(t);
  if (d.back() != p->t_max) d.push_back(p->t_max);
  return d;
}

// A layout of the sweep tables: the 2D patch shape (r1 = 16: 16 x 8, r1 = 8: 8 x 16) and the
// column pairing of the 2:4 conversion.
struct Layout {
  int r1;
  spst::Pairing pairing;
};

// Switches the plan's tables to layout L: the full sweep's tables are rebuilt (from the
// process-wide cache when another plan built them), remainder tables are dropped (rebuilt on
// demand); device tables are keyed by layout and stay.  Returns "" or the planner's reason.
std::string apply_layout(sparstencil_plan_t p, const Layout& L) {
  const PlanGeometry old_geo = p->geo;
  const spst::Pairing old_pairing = p->pairing_pref;
  if (p->geo.ndim == 2) {
    p->geo.r1 = L.r1;
    p->geo.r2 = 128 / L.r1;
  }
  p->pairing_pref = L.pairing;
  SweepTables T;
  const std::string err = build_tables(p, p->t, &T);
  if (!err.empty()) {
    p->geo = old_geo;
    p->pairing_pref = old_pairing;
    return err;
  }
  p->full = std::move(T);
  p->rem.clear();
  return "";
}

// The layouts the first run of an autotuned plan times: both 2D patch shapes, and for a
// support smaller than its box (stars, custom masks) both pairings where they differ.
std::vector<Layout> autotune_layouts(sparstencil_plan_t p) {
  std::vector<Layout> out;
  if (p->layout_fixed) return {Layout{p->geo.r1, p->pairing_pref}};
  const std::vector<int> shapes = p->geo.ndim == 2 ? std::vector<int>{16, 8} : std::vector<int>{p->geo.r1};
  for (int r1 : shapes) {
    Layout a{r1, spst::Pairing::Algorithm1}, m{r1, spst::Pairing::Matching};
    if (!apply_layout(p, a).empty()) continue;
    const int a_pairing = p->full.pairing;
    out.push_back(a);
    if (apply_layout(p, m).empty() && p->full.pairing != a_pairing) out.push_back(m);
  }
  return out;
}

// The layout search of Sec. 3.3 (Eq. 11, the argmin over the candidate layouts), done by
// measurement for a plan made with fusion_depth 0: copies `in` into the padded grid and, for
// every candidate layout (patch shape, pairing) and fusion depth, times two sweeps after one
// warm-up sweep; keeps the candidate with the least time per time step.  Synchronises the
// stream; the caller's run then starts from a fresh copy-in.
sparstencil_status autotune_depth(sparstencil_plan_t p, const float* in, cudaStream_t stream) {
  int* status = spst::device_status_word();
  if (!status) return fail(SPST_ERR_CUDA, "device status word unavailable");
  const Layout start{p->geo.r1, p->pairing_pref};
  const std::vector<Layout> layouts = autotune_layouts(p);
  if (layouts.empty()) {
    apply_layout(p, start);
    p->autotune_pending = false;
    return SPST_OK;
  }
  const std::vector<int> depths = autotune_depths(p);
  // every candidate's tables are uploaded ahead of the copy-in kernel, so that no copy sits
  // between two sweeps (a sweep's set-up may overlap the kernel before it)
  for (const Layout& L : layouts) {
    if (!apply_layout(p, L).empty()) continue;
    for (int depth : depths) {
      std::string err;
      const SweepTables* T = tables_for(p, depth, &err);
      DeviceTables* dt = nullptr;
      sparstencil_status su = T ? ensure_device_tables(p, depth, *T, &dt, stream) : SPST_OK;
      if (su != SPST_OK) return su;
    }
  }
  SPST_CUDA(copy_in(p, in, p->pad(0), 3 * p->t_max, stream, p->maxabs), "pad copy");
  cudaEvent_t e0, e1;
  SPST_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(SPST_ERR_CUDA, "cudaEventCreate");
  }
  int best_t = p->t;
  Layout best_l = layouts[0];
  double best_ms = 1e300;
  sparstencil_status s = SPST_OK;
  for (size_t li = 0; li < layouts.size() && s == SPST_OK; li++) {
    if (!apply_layout(p, layouts[li]).empty()) continue;
    for (size_t di = 0; di < depths.size() && s == SPST_OK; di++) {
      const int depth = depths[di];
      std::string err;
      const SweepTables* T = tables_for(p, depth, &err);
      if (!T) continue;
      DeviceTables* dt = nullptr;
      if ((s = ensure_device_tables(p, depth, *T, &dt, stream)) != SPST_OK) break;
      int cur = 0;
      float ms = 0.f;
      for (int k = 0; k < 3 && s == SPST_OK; k++) {
        if (k == 1 && cudaEventRecord(e0, stream) != cudaSuccess) s = fail(SPST_ERR_CUDA, "cudaEventRecord");
        spst::Sweep2DParams prm = sweep_params(p, *T, *dt, status);
        set_output(p, &prm, p->pad(1 - cur), nullptr, false);
        if (spst::launch_sweep2d(p->tmap[cur], prm, p->num_sms, stream) != cudaSuccess ||
            after_sweep(p, depth, p->pad(cur), prm, false, stream) != cudaSuccess)
          s = fail(SPST_ERR_CUDA, "autotune sweep launch");
        cur = 1 - cur;
      }
      if (s != SPST_OK) break;
      if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        s = fail(SPST_ERR_CUDA, "autotune timing");
        break;
      }
      const double per_step = (double)ms / (2.0 * depth);
      if (per_step < best_ms) {
        best_ms = per_step;
        best_t = depth;
        best_l = layouts[li];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != SPST_OK) return s;
  std::string err = apply_layout(p, best_l);
  if (!err.empty()) return fail(SPST_ERR_UNSUPPORTED, err);
  if (best_t != p->t) {
    const SweepTables* T = tables_for(p, best_t, &err);
    if (!T) return fail(SPST_ERR_UNSUPPORTED, err);
    SweepTables chosen = *T;
    p->rem[p->t] = std::move(p->full);
    p->full = std::move(chosen);
    p->rem.erase(best_t);
    // device tables are keyed by depth and layout and stay valid
    p->t = best_t;
  }
  p->autotune_pending = false;
  return SPST_OK;
}

// Parameters of the FP64 correction step on the plan's padded grids.
spst::Fp64StepParams fp64_params(sparstencil_plan_t p) {
  const PlanGeometry& g = p->geo;
  spst::Fp64StepParams f;
  std::memset(&f, 0, sizeof(f));
  f.ndim = g.ndim;
  f.D = g.ndim == 3 ? g.D : 1;
  f.H = g.ndim >= 2 ? g.H : 1;
  f.W = g.W;
  f.G = g.G;
  f.Wp = g.Wp;
  f.Hp = g.ndim == 3 ? g.Hp : 1;
  f.periodic = p->bc == SPST_PERIODIC ? 1 : 0;
  const int r = p->radius, side = 2 * r + 1;
  const int nz = g.ndim == 3 ? side : 1, ny = g.ndim >= 2 ? side : 1;
  for (int a = 0; a < nz; a++)
    for (int b = 0; b < ny; b++)
      for (int c = 0; c < side; c++) {
        const double w = p->w64[((size_t)a * ny + b) * side + c];
        if (w == 0.0) continue;
        f.off[f.npts][0] = g.ndim == 3 ? a - r : 0;
        f.off[f.npts][1] = g.ndim >= 2 ? b - r : 0;
        f.off[f.npts][2] = c - r;
        f.w[f.npts] = w;
        f.npts++;
      }
  if (f.npts == 0) {  // all weights zero: one zero term keeps the kernel's sum defined
    f.npts = 1;
    f.w[0] = 0.0;
  }
  return f;
}

sparstencil_status run_sweeps(sparstencil_plan_t p, const float* in, float* out, int64_t T, cudaStream_t stream,
                              LaunchTimer* timer = nullptr) {
  sparstencil_status s = ensure_device(p, stream);
  if (s != SPST_OK) return s;
  if (T == 0) {
    SPST_CUDA(cudaMemcpyAsync(out, in, p->cells() * 4, cudaMemcpyDeviceToDevice, stream), "copy in->out");
    return SPST_OK;
  }
  if (p->autotune_pending && (s = autotune_depth(p, in, stream)) != SPST_OK) return s;
  // the run's operations: tensor-core sweeps of p->t steps (and remainder sweeps), and with
  // the FP64 correction on, an FP64 step (depth 0 here) in place of every k-th time step
  std::vector<int> sweeps;
  auto add_sweeps = [&](int64_t n) {
    for (int64_t i = 0; i < n / p->t; i++) sweeps.push_back(p->t);
    if (n % p->t) sweeps.push_back((int)(n % p->t));
  };
  if (p->fp64_every > 0) {
    const int64_t k = p->fp64_every;
    for (int64_t done = 0; done < T;) {
      const int64_t tc = std::min<int64_t>(k - 1, T - done);
      add_sweeps(tc);
      done += tc;
      if (done < T) {
        sweeps.push_back(0);
        done++;
      }
    }
  } else {
    add_sweeps(T);
  }
  int* status = spst::device_status_word();
  if (!status) return fail(SPST_ERR_CUDA, "device status word unavailable");
  // Every table upload is enqueued before the copy-in kernel: a sweep reads its tables
  // during its set-up, which may overlap the previous kernel (programmatic dependent launch),
  // so no upload may sit between two sweeps.
  std::vector<const SweepTables*> tabs(sweeps.size(), nullptr);
  std::vector<DeviceTables*> dtabs(sweeps.size(), nullptr);
  for (size_t i = 0; i < sweeps.size(); i++) {
    if (sweeps[i] == 0) continue;  // an FP64 step
    std::string err;
    tabs[i] = tables_for(p, sweeps[i], &err);
    if (!tabs[i]) return fail(SPST_ERR_UNSUPPORTED, err);
    s = ensure_device_tables(p, sweeps[i], *tabs[i], &dtabs[i], stream);
    if (s != SPST_OK) return s;
  }
  // a run that the caller captures into a CUDA graph keeps its programmatic launches: stream
  // capture records them as programmatic edges between the sweeps
  const bool pdl_before = t_pdl_on;
  struct RestorePdl {
    bool on;
    ~RestorePdl() { set_programmatic_launch(on); }
  } restore_pdl{pdl_before};
  if (timer && (s = timer->record(stream)) != SPST_OK) return s;
  SPST_CUDA(copy_in(p, in, p->pad(0), T, stream, p->maxabs), "pad copy");
  if (timer && (s = timer->record(stream)) != SPST_OK) return s;
  int cur = 0;
  int tc_sweeps = 0;
  for (size_t i = 0; i < sweeps.size(); i++) {
    const bool last = (i + 1 == sweeps.size());
    if (sweeps[i] == 0) {
      SPST_CUDA(spst::launch_fp64_step(fp64_params(p), p->pad(cur), last ? nullptr : p->pad(1 - cur),
                                       last ? out : nullptr, stream),
                "FP64 step launch");
      cur = 1 - cur;
      continue;
    }
    tc_sweeps++;
    spst::Sweep2DParams prm = sweep_params(p, *tabs[i], *dtabs[i], status);
    set_output(p, &prm, p->pad(1 - cur), out, last);
    SPST_CUDA(spst::launch_sweep2d(p->tmap[cur], prm, p->num_sms, stream), "sweep launch");
    SPST_CUDA(after_sweep(p, sweeps[i], p->pad(cur), prm, last, stream), "band or ghost launch");
    cur = 1 - cur;
  }
  // one event after all sweeps: an event between two sweeps would stop the next one from
  // overlapping its set-up with the previous one (programmatic dependent launch)
  if (timer) {
    timer->sweeps = tc_sweeps;
    if ((s = timer->record(stream)) != SPST_OK) return s;
  }
  return SPST_OK;
}

bool shape_mask_ok(sparstencil_shape shape, int ndim, int r, const float* w) {
  const int side = 2 * r + 1;
  int total = 1;
  for (int i = 0; i < ndim; i++) total *= side;
  for (int idx = 0; idx < total; idx++) {
    int rem = idx, nonc = 0;
    for (int d = 0; d < ndim; d++) {
      if (rem % side != r) nonc++;
      rem /= side;
    }
    if (shape == SPST_STAR && nonc > 1 && w[idx] != 0.f) return false;
    if (!std::isfinite(w[idx])) return false;
  }
  return true;
}

}  // namespace


// ---------------------------------------------------------------------------------------
// Runs with caller-provided device buffers and no allocation (used by the allocation-free
// entry point in noalloc.cu): scratch holds the two padded grids, tables the device copies
// of the planner tables (half for the full sweep, half for the remainder sweep).
// ---------------------------------------------------------------------------------------
namespace spst {

sparstencil_status report_error(sparstencil_status s, const char* msg) { return fail(s, msg); }

sparstencil_status run_plan_with_buffers(sparstencil_plan_t p, const float* in, float* out, int64_t T,
                                         cudaStream_t stream, float* scratch, size_t scratch_floats,
                                         uint32_t* tables, size_t table_words, unsigned* maxabs_word) {
  if (!p || !in || !out) return fail(SPST_ERR_INVALID, "null plan or grid");
  if (T < 0) return fail(SPST_ERR_INVALID, "timesteps must be >= 0");
  if (in == out) return fail(SPST_ERR_INVALID, "in and out must not alias");
  if (p->fp64_every > 0) return fail(SPST_ERR_UNSUPPORTED, "the allocation-free run does not take the FP64 correction step");
  int dev = 0, major = 0, minor = 0, sms = 0;
  SPST_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  SPST_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev), "device attribute");
  SPST_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev), "device attribute");
  SPST_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
  if (major != 10 || minor != 3) return fail(SPST_ERR_UNSUPPORTED, "this library is built for sm_103a (GB300)");
  const PlanGeometry& g = p->geo;
  if (g.ndim != 2) return fail(SPST_ERR_UNSUPPORTED, "the allocation-free path runs 2D plans only");
  if (p->dense) return fail(SPST_ERR_UNSUPPORTED, "the allocation-free path runs sparse MMAs only");
  const size_t grid = ((size_t)g.Hp * (size_t)g.Wp + 63) & ~(size_t)63;  // 256-byte aligned grids
  if (2 * grid > scratch_floats)
    return fail(SPST_ERR_UNSUPPORTED, "grid too large for the allocation-free path: needs " + std::to_string(grid) +
                                          " padded cells per ping-pong grid, the static scratch holds " +
                                          std::to_string(scratch_floats / 2));
  if (T == 0) {
    SPST_CUDA(cudaMemcpyAsync(out, in, p->cells() * 4, cudaMemcpyDeviceToDevice, stream), "copy in->out");
    return SPST_OK;
  }
  std::vector<int> sweeps((size_t)(T / p->t), p->t);
  if (T % p->t) sweeps.push_back((int)(T % p->t));
  // device copies of the tables of each sweep depth used (at most two)
  struct Region {
    int depth;
    const SweepTables* T;
    int32_t* lut;
    uint32_t* a_words;
    uint32_t* meta;
  } regions[2];
  int nreg = 0;
  const size_t half_words = table_words / 2;
  for (int depth : sweeps) {
    bool seen = false;
    for (int r = 0; r < nreg; r++) seen |= regions[r].depth == depth;
    if (seen) continue;
    std::string err;
    const SweepTables* Tt = tables_for(p, depth, &err);
    if (!Tt) return fail(SPST_ERR_UNSUPPORTED, err);
    const size_t need = Tt->lut.size() + Tt->a_words.size() + Tt->meta_words.size();
    if (need > half_words) return fail(SPST_ERR_UNSUPPORTED, "planner tables too large for the static table area");
    uint32_t* base = tables + (size_t)nreg * half_words;
    Region& rg = regions[nreg++];
    rg.depth = depth;
    rg.T = Tt;
    rg.lut = (int32_t*)base;
    rg.a_words = base + Tt->lut.size();
    rg.meta = rg.a_words + Tt->a_words.size();
    SPST_CUDA(cudaMemcpyAsync(rg.lut, Tt->lut.data(), Tt->lut.size() * 4, cudaMemcpyHostToDevice, stream), "lut");
    SPST_CUDA(cudaMemcpyAsync(rg.a_words, Tt->a_words.data(), Tt->a_words.size() * 4, cudaMemcpyHostToDevice, stream),
              "A''");
    SPST_CUDA(cudaMemcpyAsync(rg.meta, Tt->meta_words.data(), Tt->meta_words.size() * 4, cudaMemcpyHostToDevice,
                              stream),
              "metadata");
  }
  float* pad[2] = {scratch, scratch + grid};
  CUtensorMap tm[2];
  EncodeTiledFn enc = get_encode_tiled();
  if (!enc) return fail(SPST_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  for (int i = 0; i < 2; i++) {
    cuuint64_t gdim[2] = {(cuuint64_t)g.Wp, (cuuint64_t)g.Hp};
    cuuint64_t gstr[1] = {(cuuint64_t)g.Wp * 4};
    cuuint32_t box[2] = {(cuuint32_t)g.P, (cuuint32_t)g.box_h};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(&tm[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, pad[i], gdim, gstr, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SPST_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  }
  int* status = device_status_word();
  if (!status) return fail(SPST_ERR_CUDA, "device status word unavailable");
  // the static arrays keep the previous call's contents: the second grid's ghost cells and
  // slack columns must start at zero (the copy-in writes every cell of the first grid)
  SPST_CUDA(cudaMemsetAsync(pad[1], 0, grid * 4, stream), "clear scratch");
  unsigned* maxabs = word_of(p->dtype) == Word::FP16 ? maxabs_word : nullptr;
  SPST_CUDA(copy_in(p, in, pad[0], T, stream, maxabs), "pad copy");
  int cur = 0;
  for (size_t i = 0; i < sweeps.size(); i++) {
    const Region* rg = nullptr;
    for (int r = 0; r < nreg; r++)
      if (regions[r].depth == sweeps[i]) rg = &regions[r];
    const bool last = (i + 1 == sweeps.size());
    DeviceTables dtv;
    dtv.lut = rg->lut;
    dtv.a_words = rg->a_words;
    dtv.meta = rg->meta;
    Sweep2DParams prm = sweep_params(p, *rg->T, dtv, status);  // dtv borrows the static tables
    prm.maxabs = maxabs;
    set_output(p, &prm, pad[1 - cur], out, last);
    prm.status = status;
    prm.wait_ns = g_wait_ns;
    SPST_CUDA(launch_sweep2d(tm[cur], prm, sms, stream), "sweep launch");
    SPST_CUDA(launch_band(p, sweeps[i], pad[cur], prm.out, prm.out_pitch, prm.out_off, stream), "band launch");
    cur = 1 - cur;
  }
  return SPST_OK;
}

}  // namespace spst

namespace {

// Instantiated batch graphs, keyed by everything a captured batch depends on: per job the
// plan's uid, its workspace, fusion depth and MMA options, the grids and the step count.  A
// repeated sparstencil_run_batch with the same key replays the graph without preparing,
// capturing or instantiating again.  Entries holding a plan are dropped when the plan is
// destroyed; at most kBatchCacheMax are kept (least recently used first out).
constexpr size_t kBatchCacheMax = 16;
struct BatchGraph {
  std::vector<uint64_t> key;
  int device;
  cudaGraphExec_t exec;
};
std::mutex g_batch_mu;
std::list<BatchGraph> g_batch_cache;  // most recently used first

std::vector<uint64_t> batch_key(const sparstencil_plan_t* plans, const float* const* in, float* const* out,
                                const int64_t* steps, int n) {
  std::vector<uint64_t> k;
  k.reserve((size_t)n * 7);
  for (int i = 0; i < n; i++) {
    const sparstencil_plan_s* p = plans[i];
    k.push_back(p->uid);
    k.push_back((uint64_t)(uintptr_t)p->ws);
    k.push_back(((uint64_t)p->t << 2) | (p->lo_acc ? 1u : 0u) | (p->dense ? 2u : 0u));
    k.push_back((uint64_t)(uintptr_t)in[i]);
    k.push_back((uint64_t)(uintptr_t)out[i]);
    k.push_back((uint64_t)steps[i]);
    k.push_back(p->autotune_pending || !p->ws_ready ? 1u : 0u);
  }
  return k;
}

// Enqueues a prepared batch on `stream` (captured by the caller): every job's copy-in, then
// for each sweep index s one launch of the multi-grid sweep kernel per kernel template
// (FP16 or BF16, single or split words, dimensionality) and per kMultiMaxJobs jobs, over the
// jobs that have a sweep s, each followed by those jobs' Dirichlet bands or periodic ghost
// refreshes.  Job j's sweeps alternate between its own two padded grids and its last sweep
// writes out[j], as in sparstencil_run.
sparstencil_status enqueue_batch(const sparstencil_plan_t* plans, const float* const* in, float* const* out,
                                 const int64_t* steps, int n, cudaStream_t stream) {
  int* status = spst::device_status_word();
  if (!status) return fail(SPST_ERR_CUDA, "device status word unavailable");
  std::vector<std::vector<int>> sweeps(n);
  size_t max_sweeps = 0;
  for (int i = 0; i < n; i++) {
    sparstencil_plan_t p = plans[i];
    if (steps[i] == 0) {
      SPST_CUDA(cudaMemcpyAsync(out[i], in[i], p->cells() * 4, cudaMemcpyDeviceToDevice, stream), "copy in->out");
      continue;
    }
    sweeps[i].assign((size_t)(steps[i] / p->t), p->t);
    if (steps[i] % p->t) sweeps[i].push_back((int)(steps[i] % p->t));
    max_sweeps = std::max(max_sweeps, sweeps[i].size());
    SPST_CUDA(copy_in(p, in[i], p->pad(0), steps[i], stream, p->maxabs), "pad copy");
  }
  // kernel template of a job: FP16 or BF16, single or split words, dimensionality
  auto group = [&](int i) {
    return (word_of(plans[i]->dtype) == spst::Word::FP16 ? 1 : 0) + (is_split(plans[i]->dtype) ? 2 : 0) +
           4 * plans[i]->geo.ndim + (plans[i]->geo.ndim == 2 && plans[i]->geo.r1 == 8 ? 16 : 0);
  };
  std::vector<CUtensorMap> maps;
  std::vector<spst::Sweep2DParams> prms;
  std::vector<int> members;
  for (size_t s = 0; s < max_sweeps; s++) {
    std::vector<char> done(n, 0);
    for (int i0 = 0; i0 < n; i0++) {
      if (done[i0] || s >= sweeps[i0].size()) continue;
      const int g = group(i0);
      members.clear();
      for (int i = i0; i < n && (int)members.size() < spst::kMultiMaxJobs; i++)
        if (!done[i] && s < sweeps[i].size() && group(i) == g) {
          members.push_back(i);
          done[i] = 1;
        }
      maps.clear();
      prms.clear();
      for (int i : members) {
        sparstencil_plan_t p = plans[i];
        const int depth = sweeps[i][s];
        std::string err;
        const SweepTables* T = tables_for(p, depth, &err);
        if (!T) return fail(SPST_ERR_UNSUPPORTED, err);
        DeviceTables* dt = nullptr;
        sparstencil_status st = ensure_device_tables(p, depth, *T, &dt, stream);
        if (st != SPST_OK) return st;
        const int cur = (int)(s & 1);
        spst::Sweep2DParams prm = sweep_params(p, *T, *dt, status);
        set_output(p, &prm, p->pad(1 - cur), out[i], s + 1 == sweeps[i].size());
        maps.push_back(p->tmap[cur]);
        prms.push_back(prm);
      }
      SPST_CUDA(spst::launch_sweep2d_multi(maps.data(), prms.data(), (int)members.size(), plans[i0]->num_sms, stream),
                "batch sweep launch");
      for (size_t k = 0; k < members.size(); k++) {
        const int i = members[k];
        const int cur = (int)(s & 1);
        SPST_CUDA(after_sweep(plans[i], sweeps[i][s], plans[i]->pad(cur), prms[k], s + 1 == sweeps[i].size(), stream),
                  "band or ghost launch");
      }
    }
  }
  return SPST_OK;
}

void drop_batch_graphs_of(uint64_t uid) {
  std::lock_guard<std::mutex> lock(g_batch_mu);
  for (auto it = g_batch_cache.begin(); it != g_batch_cache.end();) {
    bool uses = false;
    for (size_t j = 0; j < it->key.size(); j += 7) uses |= it->key[j] == uid;
    if (uses) {
      cudaGraphExecDestroy(it->exec);
      it = g_batch_cache.erase(it);
    } else {
      ++it;
    }
  }
}

}  // namespace

extern "C" {

const char* sparstencil_last_error(void) { return g_last_error.c_str(); }

const char* sparstencil_version(void) { return "sparstencil-gb300 0.1 (sm_103a)"; }

sparstencil_status sparstencil_set_wait_limit_ns(uint64_t ns) {
  g_wait_ns = ns ? ns : 2000000000ull;
  return SPST_OK;
}

sparstencil_status sparstencil_plan(sparstencil_shape shape, int radius, const float* weights, int ndim,
                                    const int64_t* dims, sparstencil_dtype dtype, sparstencil_boundary bc,
                                    int fusion_depth, sparstencil_plan_t* out_plan) {
  auto t0 = std::chrono::steady_clock::now();
  if (!out_plan) return fail(SPST_ERR_INVALID, "out_plan is null");
  *out_plan = nullptr;
  if (!weights || !dims) return fail(SPST_ERR_INVALID, "weights or dims is null");
  if (shape < SPST_STAR || shape > SPST_CUSTOM) return fail(SPST_ERR_INVALID, "bad shape");
  if (dtype < SPST_FP16 || dtype > SPST_BF16_SPLIT) return fail(SPST_ERR_INVALID, "bad dtype");
  if (bc != SPST_DIRICHLET_ZERO && bc != SPST_PERIODIC) return fail(SPST_ERR_INVALID, "bad boundary");
  if (radius < 1) return fail(SPST_ERR_INVALID, "radius must be >= 1");
  if (fusion_depth < 0) return fail(SPST_ERR_INVALID, "fusion_depth must be >= 0");
  if (ndim < 1 || ndim > 3) return fail(SPST_ERR_UNSUPPORTED, "ndim must be 1, 2 or 3");
  for (int i = 0; i < ndim; i++)
    if (dims[i] <= 0) return fail(SPST_ERR_INVALID, "grid extents must be positive");
  if (!shape_mask_ok(shape, ndim, radius, weights))
    return fail(SPST_ERR_INVALID, "weights are not finite or lie outside the stencil shape");
  std::unique_ptr<sparstencil_plan_s> p(new (std::nothrow) sparstencil_plan_s());
  if (!p) return fail(SPST_ERR_NOMEM, "host allocation failed");
  p->shape = shape;
  p->ndim = ndim;
  p->radius = radius;
  p->dtype = dtype;
  p->bc = bc;
  p->requested_t = fusion_depth;
  p->t = fusion_depth == 0 ? 1 : fusion_depth;
  // Dirichlet fusion needs the exact frame of each sweep: the 2D band kernel (radius <= 4) or
  // the 3D one (radius 1); 1D Dirichlet plans run one step per sweep
  auto dirichlet_fusion_ok = [&]() { return (ndim == 2 && radius <= 4) || (ndim == 3 && radius == 1); };
  if (bc == SPST_DIRICHLET_ZERO && p->t > 1 && !dirichlet_fusion_ok())
    return fail(SPST_ERR_UNSUPPORTED,
                "temporal fusion with a Dirichlet boundary needs a 2D grid with radius <= 4 or a 3D grid with radius 1");
  p->t_max = p->t;
  // fusion_depth 0: the deepest depth whose tables fit is planned (searched down from 6 in 2D,
  // 3 in 3D); the first run times the depths up to it and keeps the fastest per time step.
  // 1D: K grows by only 2r columns per fused step (k' = kt + 127), so the search starts at the
  // largest fused radius the tiles allow (60)
  const int t_deep = ndim == 1 ? std::max(1, 60 / radius) : ndim == 2 ? 6 : 3;
  const int t_try = fusion_depth == 0 ? ((bc == SPST_DIRICHLET_ZERO && !dirichlet_fusion_ok()) ? 1 : t_deep) : p->t;
  const int side = 2 * radius + 1;
  p->w64.resize((size_t)side * (ndim >= 2 ? side : 1) * (ndim == 3 ? side : 1));
  for (size_t i = 0; i < p->w64.size(); i++) p->w64[i] = (double)weights[i];
  PlanGeometry& g = p->geo;
  g.ndim = ndim;
  g.D = ndim == 3 ? dims[0] : 1;
  g.H = ndim >= 2 ? dims[ndim - 2] : 1;
  g.W = dims[ndim - 1];
  std::string err;
  for (int tm = t_try; tm >= 1; tm--) {
    p->t = p->t_max = tm;
    err = plan_geometry(p.get());
    if (err.empty()) err = build_tables(p.get(), p->t, &p->full);
    if (err.empty()) {
      spst::Sweep2DParams probe;
      std::memset(&probe, 0, sizeof(probe));
      probe.P = g.P;
      probe.box_h = g.box_h;
      probe.box_d = g.box_d;
      probe.kpad = p->full.kpad;
      probe.kchunks = p->full.kpad / 32;
      probe.a_pieces = p->full.a_pieces;
      probe.b_pieces = is_split(dtype) ? 2 : 1;
      if (spst::sweep2d_halo_stages(probe) == 0) err = "halo tile of the fused radius does not fit in shared memory";
    }
    if (err.empty() && fusion_depth == 0 && ndim == 3 && is_split(dtype) && tm > 1) {
      // 3D split operands meet their tolerance over long runs only with the low-order
      // accumulator (one accumulator: 1.0e-5 on 512^3 over 50 steps at t = 1, 2.1e-5 fused
      // t = 2), so the search keeps the depths where it fits (for BF16, beside three pieces)
      p->lo_acc = true;
      SweepTables lo;
      const bool lo_fits = build_tables(p.get(), tm, &lo).empty() && (dtype == SPST_FP16_SPLIT || lo.a_pieces == 3);
      p->lo_acc = false;
      if (!lo_fits) err = "the low-order accumulator does not fit at this depth";
    }
    if (err.empty() || fusion_depth != 0) break;
  }
  if (!err.empty()) return fail(SPST_ERR_UNSUPPORTED, err);
  // FP16 split operands carry 22 significant bits of data and weights, so the roundings of
  // the MMA chain dominate their error: they take the low-order accumulator where it fits.
  // BF16 split operands take it for 3D plans where all three weight pieces still fit beside
  // it: a 3D step runs 9-12 K chunks of 3-4 MMAs per output (2D and 1D fused sweeps spread
  // far fewer MMAs over each step), and measured on Heat-3D 512^3 over 50 steps it brings the
  // error from 1.16e-5 to 3.5e-6.
  if (dtype == SPST_FP16_SPLIT || (dtype == SPST_BF16_SPLIT && ndim == 3)) {
    p->lo_acc = true;
    SweepTables T;
    const bool ok = build_tables(p.get(), p->t, &T).empty() && (dtype == SPST_FP16_SPLIT || T.a_pieces == 3);
    if (ok)
      p->full = std::move(T);
    else
      p->lo_acc = false;
  }
  p->autotune_pending = fusion_depth == 0;
  p->planner_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out_plan = p.release();
  return SPST_OK;
}

sparstencil_status sparstencil_plan_set_fp64_correction(sparstencil_plan_t plan, int every_k) {
  if (!plan) return fail(SPST_ERR_INVALID, "plan is null");
  if (every_k < 0) return fail(SPST_ERR_INVALID, "every_k must be >= 0");
  plan->fp64_every = every_k;
  return SPST_OK;
}

sparstencil_status sparstencil_plan_set_low_accumulator(sparstencil_plan_t plan, int enable) {
  if (!plan) return fail(SPST_ERR_INVALID, "plan is null");
  if (enable && !is_split(plan->dtype)) return fail(SPST_ERR_INVALID, "the low-order accumulator needs a split dtype");
  if (!plan->dev_tables.empty()) return fail(SPST_ERR_INVALID, "set the accumulator mode before the plan's first run");
  if ((enable != 0) == plan->lo_acc) return SPST_OK;
  const bool old = plan->lo_acc;
  plan->lo_acc = enable != 0;
  SweepTables T;
  const std::string err = build_tables(plan, plan->t, &T);
  if (!err.empty()) {
    plan->lo_acc = old;
    return fail(SPST_ERR_UNSUPPORTED, err);
  }
  plan->full = std::move(T);
  plan->rem.clear();
  return SPST_OK;
}

sparstencil_status sparstencil_plan_set_layout(sparstencil_plan_t plan, int r1, int pairing) {
  if (!plan) return fail(SPST_ERR_INVALID, "plan is null");
  if (!plan->dev_tables.empty()) return fail(SPST_ERR_INVALID, "set the layout before the plan's first run");
  if (pairing < -1 || pairing > 1) return fail(SPST_ERR_INVALID, "pairing must be -1, 0 or 1");
  if (plan->geo.ndim == 2 ? (r1 != 16 && r1 != 8) : r1 != plan->full.r1)
    return fail(SPST_ERR_UNSUPPORTED, plan->geo.ndim == 2 ? "2D patches are 16 x 8 (r1 = 16) or 8 x 16 (r1 = 8)"
                                                          : "1D and 3D plans have one patch shape");
  const std::string err = apply_layout(plan, Layout{r1, (spst::Pairing)pairing});
  if (!err.empty()) return fail(SPST_ERR_UNSUPPORTED, err);
  plan->layout_fixed = true;  // a fusion-depth search keeps this layout
  return SPST_OK;
}

sparstencil_status sparstencil_plan_set_dense_ablation(sparstencil_plan_t plan, int enable) {
  if (!plan) return fail(SPST_ERR_INVALID, "plan is null");
  if (!plan->dev_tables.empty()) return fail(SPST_ERR_INVALID, "set the MMA form before the plan's first run");
  if ((enable != 0) == plan->dense) return SPST_OK;
  const bool old = plan->dense, old_lo = plan->lo_acc;
  plan->dense = enable != 0;
  SweepTables T;
  std::string err = build_tables(plan, plan->t, &T);
  if (!err.empty() && plan->lo_acc) {  // the uncompressed A' leaves no room for both
    plan->lo_acc = false;
    err = build_tables(plan, plan->t, &T);
  }
  if (err.empty() && plan->dense) {
    spst::Sweep2DParams probe;
    std::memset(&probe, 0, sizeof(probe));
    probe.P = plan->geo.P;
    probe.box_h = plan->geo.box_h;
    probe.box_d = plan->geo.box_d;
    probe.kpad = T.kpad;
    probe.kchunks = T.kpad / 32;
    probe.a_pieces = T.a_pieces;
    probe.b_pieces = is_split(plan->dtype) ? 2 : 1;
    probe.dense = 1;
    if (!spst::sweep2d_fits(probe)) err = "the dense A' staging does not fit in shared memory";
  }
  if (!err.empty()) {
    plan->dense = old;
    plan->lo_acc = old_lo;
    return fail(SPST_ERR_UNSUPPORTED, err);
  }
  plan->full = std::move(T);
  plan->rem.clear();
  return SPST_OK;
}

sparstencil_status sparstencil_plan_destroy(sparstencil_plan_t plan) {
  if (!plan) return fail(SPST_ERR_INVALID, "plan is null");
  drop_batch_graphs_of(plan->uid);
  delete plan;
  return SPST_OK;
}

size_t sparstencil_workspace_bytes(sparstencil_plan_t plan) {
  if (!plan) return 0;
  return 2 * ((plan->grid_floats() * 4 + 255) & ~(size_t)255);
}

sparstencil_status sparstencil_bind_workspace(sparstencil_plan_t plan, void* dev, size_t bytes, cudaStream_t stream) {
  if (!plan || !dev) return fail(SPST_ERR_INVALID, "plan or workspace is null");
  if (((uintptr_t)dev) & 255) return fail(SPST_ERR_INVALID, "workspace must be 256-byte aligned");
  if (bytes < sparstencil_workspace_bytes(plan)) return fail(SPST_ERR_NOMEM, "workspace too small");
  drop_batch_graphs_of(plan->uid);
  if (plan->ws_owned) cudaFree(plan->ws);
  plan->ws = dev;
  plan->ws_bytes = bytes;
  plan->ws_owned = false;
  plan->ws_ready = false;
  SPST_CUDA(cudaMemsetAsync(dev, 0, sparstencil_workspace_bytes(plan), stream), "zero workspace");
  return SPST_OK;
}

sparstencil_status sparstencil_run(sparstencil_plan_t plan, const float* in, float* out, int64_t timesteps,
                                   cudaStream_t stream) {
  if (!plan || !in || !out) return fail(SPST_ERR_INVALID, "null plan or grid");
  if (timesteps < 0) return fail(SPST_ERR_INVALID, "timesteps must be >= 0");
  if (in == out) return fail(SPST_ERR_INVALID, "in and out must not alias");
  return run_sweeps(plan, in, out, timesteps, stream);
}

sparstencil_status sparstencil_run_profiled(sparstencil_plan_t plan, const float* in, float* out, int64_t timesteps,
                                            cudaStream_t stream, double* copy_in_ms, double* sweeps_ms,
                                            int* num_sweeps) {
  if (!plan || !in || !out) return fail(SPST_ERR_INVALID, "null plan or grid");
  if (timesteps < 0) return fail(SPST_ERR_INVALID, "timesteps must be >= 0");
  if (in == out) return fail(SPST_ERR_INVALID, "in and out must not alias");
  LaunchTimer timer;
  sparstencil_status s = run_sweeps(plan, in, out, timesteps, stream, &timer);
  if (s != SPST_OK) return s;
  SPST_CUDA(cudaStreamSynchronize(stream), "stream sync");
  double cin = 0.0, sw = 0.0;
  for (size_t i = 1; i < timer.ev.size(); i++) {
    float ms = 0.f;
    SPST_CUDA(cudaEventElapsedTime(&ms, timer.ev[i - 1], timer.ev[i]), "cudaEventElapsedTime");
    if (i == 1) {
      cin = ms;
    } else {
      sw += ms;
    }
  }
  if (copy_in_ms) *copy_in_ms = cin;
  if (sweeps_ms) *sweeps_ms = sw;
  if (num_sweeps) *num_sweeps = timer.sweeps;
  return SPST_OK;
}

namespace {
// Host-buffer run: H2D into the plan's staging grid (or, when `zero_copy` and the input is
// page-locked memory the device can address, the copy-in kernel reads it directly), the
// sweeps, D2H from the staging output; synchronises the stream when `sync`.
sparstencil_status run_host_impl(sparstencil_plan_t plan, const float* in_host, float* out_host, int64_t timesteps,
                                 cudaStream_t stream, bool zero_copy, bool sync) {
  if (!plan || !in_host || !out_host) return fail(SPST_ERR_INVALID, "null plan or grid");
  if (timesteps < 0) return fail(SPST_ERR_INVALID, "timesteps must be >= 0");
  sparstencil_status s = ensure_device(plan, stream);
  if (s != SPST_OK) return s;
  const size_t bytes = plan->cells() * 4;
  if (!plan->stage_in) {
    if (cudaMalloc(&plan->stage_in, bytes) != cudaSuccess || cudaMalloc(&plan->stage_out, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(SPST_ERR_NOMEM, "staging allocation failed");
    }
  }
  const float* src = plan->stage_in;
  cudaPointerAttributes at;
  if (zero_copy && timesteps > 0 && cudaPointerGetAttributes(&at, in_host) == cudaSuccess &&
      at.type == cudaMemoryTypeHost && at.devicePointer)
    src = (const float*)at.devicePointer;
  else
    cudaGetLastError();
  if (src == plan->stage_in)
    SPST_CUDA(cudaMemcpyAsync(plan->stage_in, in_host, bytes, cudaMemcpyHostToDevice, stream), "H2D");
  s = run_sweeps(plan, src, plan->stage_out, timesteps, stream);
  if (s != SPST_OK) return s;
  SPST_CUDA(cudaMemcpyAsync(out_host, plan->stage_out, bytes, cudaMemcpyDeviceToHost, stream), "D2H");
  if (sync) SPST_CUDA(cudaStreamSynchronize(stream), "stream sync");
  return SPST_OK;
}
}  // namespace

sparstencil_status sparstencil_run_host(sparstencil_plan_t plan, const float* in_host, float* out_host,
                                        int64_t timesteps, cudaStream_t stream) {
  // page-locked input that the device can address is read by the copy-in kernel itself,
  // which saves the staging copy of a lone run
  return run_host_impl(plan, in_host, out_host, timesteps, stream, true, true);
}

sparstencil_status sparstencil_run_host_async(sparstencil_plan_t plan, const float* in_host, float* out_host,
                                              int64_t timesteps, cudaStream_t stream) {
  // the copies go through the copy engines, so that they overlap other streams' sweeps
  return run_host_impl(plan, in_host, out_host, timesteps, stream, false, false);
}

sparstencil_status sparstencil_run_batch(const sparstencil_plan_t* plans, const float* const* in, float* const* out,
                                         const int64_t* steps, int n, cudaStream_t stream) {
  if (n < 0 || (n > 0 && (!plans || !in || !out || !steps))) return fail(SPST_ERR_INVALID, "bad batch arguments");
  if (n == 0) return SPST_OK;
  for (int i = 0; i < n; i++) {
    if (!plans[i] || !in[i] || !out[i]) return fail(SPST_ERR_INVALID, "null plan or grid in the batch");
    if (plans[i]->fp64_every > 0) return fail(SPST_ERR_UNSUPPORTED, "batched plans cannot take the FP64 correction step");
    if (steps[i] < 0) return fail(SPST_ERR_INVALID, "timesteps must be >= 0");
    if (in[i] == out[i]) return fail(SPST_ERR_INVALID, "in and out must not alias");
    for (int j = 0; j < i; j++)
      if (plans[j] == plans[i]) return fail(SPST_ERR_INVALID, "plans in a batch must be distinct");
  }
  int dev = 0;
  SPST_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  {
    // a batch already captured with the same plans, plan state, grids and steps: replay it
    const std::vector<uint64_t> key = batch_key(plans, in, out, steps, n);
    std::lock_guard<std::mutex> lock(g_batch_mu);
    for (auto it = g_batch_cache.begin(); it != g_batch_cache.end(); ++it) {
      if (it->device != dev || it->key != key) continue;
      g_batch_cache.splice(g_batch_cache.begin(), g_batch_cache, it);
      SPST_CUDA(cudaGraphLaunch(g_batch_cache.front().exec, stream), "launch batch graph");
      return SPST_OK;
    }
  }
  // Everything that allocates, uploads or synchronises happens before the capture: device
  // state, the fusion-depth search of autotuned plans, and the tables of every sweep depth.
  for (int i = 0; i < n; i++) {
    sparstencil_plan_t p = plans[i];
    sparstencil_status s = ensure_device(p, stream);
    if (s != SPST_OK) return s;
    if (steps[i] > 0 && p->autotune_pending && (s = autotune_depth(p, in[i], stream)) != SPST_OK) return s;
    const int depths[2] = {p->t, (int)(steps[i] % p->t)};
    for (int d : depths) {
      if (d <= 0 || steps[i] == 0) continue;
      std::string err;
      const SweepTables* T = tables_for(p, d, &err);
      if (!T) return fail(SPST_ERR_UNSUPPORTED, err);
      DeviceTables* dt = nullptr;
      if ((s = ensure_device_tables(p, d, *T, &dt, stream)) != SPST_OK) return s;
    }
  }
  SPST_CUDA(cudaStreamSynchronize(stream), "stream sync");
  // One CUDA graph, captured on a stream of its own: the copy-ins, then one multi-grid sweep
  // launch per sweep index (consecutive sweeps keep their programmatic dependent launches,
  // recorded as programmatic edges).
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  sparstencil_status s = SPST_OK;
  const bool pdl_before = t_pdl_on;
  auto cleanup = [&]() {
    set_programmatic_launch(pdl_before);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
  };
  auto cuda_ok = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && s == SPST_OK) s = cuda_fail(e, what);
    return s == SPST_OK;
  };
  if (!cuda_ok(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "create capture stream")) {
    cleanup();
    return s;
  }
  set_programmatic_launch(true);
  if (cuda_ok(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "begin capture")) {
    s = enqueue_batch(plans, in, out, steps, n, cap);
    const cudaError_t ee = cudaStreamEndCapture(cap, &graph);  // always ends the capture
    cuda_ok(ee, "end capture");
  }
  if (s == SPST_OK && cuda_ok(cudaGraphInstantiate(&exec, graph, 0), "instantiate batch graph"))
    cuda_ok(cudaGraphLaunch(exec, stream), "launch batch graph");
  if (s == SPST_OK) {
    // keep the executable graph for repeated batches (keyed after the preparation above,
    // which fixed every plan's workspace and fusion depth)
    std::lock_guard<std::mutex> lock(g_batch_mu);
    g_batch_cache.push_front(BatchGraph{batch_key(plans, in, out, steps, n), dev, exec});
    exec = nullptr;
    while (g_batch_cache.size() > kBatchCacheMax) {
      cudaGraphExecDestroy(g_batch_cache.back().exec);
      g_batch_cache.pop_back();
    }
  }
  cleanup();  // the launched graph keeps its own copy of the work
  return s;
}

sparstencil_status sparstencil_query(sparstencil_plan_t plan, sparstencil_plan_info* info) {
  if (!plan || !info) return fail(SPST_ERR_INVALID, "null plan or info");
  std::memset(info, 0, sizeof(*info));
  info->ndim = plan->ndim;
  info->radius = plan->radius;
  info->fusion_depth = plan->t;
  info->r1 = plan->full.r1;
  info->r2 = plan->full.r2;
  info->r3 = plan->full.r3;
  info->kprime = plan->full.kprime;
  info->kpad = plan->full.kpad;
  info->zero_columns = plan->full.zero_cols;
  info->mma_terms = (is_split(plan->dtype) ? 2 : 1) + plan->full.a_pieces - 1;
  info->tile_outputs = Tile2D::TX * Tile2D::TY;
  info->num_tiles = plan->geo.num_tiles;
  info->planner_ms = plan->planner_ms;
  info->ghost = plan->geo.G;
  info->tile_pitch = plan->geo.P;
  info->tile_rows = plan->geo.box_h;
  info->bank_conflicts = plan->full.bank_conflicts;
  info->low_accumulator = plan->lo_acc ? 1 : 0;
  info->dense_ablation = plan->dense ? 1 : 0;
  info->pairing = plan->full.pairing;
  info->fp64_every = plan->fp64_every;
  return SPST_OK;
}

sparstencil_status sparstencil_cost_model(sparstencil_plan_t plan, int depth, double tensor_flops, double hbm_bytes_per_s,
                                          double smem_bytes_per_s, double* seconds_per_step) {
  if (!plan || !seconds_per_step) return fail(SPST_ERR_INVALID, "null argument");
  if (depth < 1 || depth > plan->t_max) return fail(SPST_ERR_INVALID, "depth must be in 1..the plan's fusion depth");
  if (!(tensor_flops > 0) || !(hbm_bytes_per_s > 0) || !(smem_bytes_per_s > 0))
    return fail(SPST_ERR_INVALID, "rates must be positive");
  std::string err;
  const SweepTables* T = depth == plan->t ? &plan->full : tables_for(plan, depth, &err);
  if (!T) return fail(SPST_ERR_UNSUPPORTED, err);
  // Eq. 6-11 with the plan's layout: m' = 128 rows, k' = A' columns, n' = outputs / m'
  // patches; one MMA per 32-row K chunk, 128-patch tile and MMA term; data_R + data_W = 8 B
  // per output; data_transR = data_transW = k' (m'/2 + n') 16-bit elements per operand piece.
  const double cells = (double)plan->cells();
  const double mprime = 128.0, kprime = (double)T->kprime, nprime = cells / mprime;
  const int terms = (is_split(plan->dtype) ? 2 : 1) + T->a_pieces - 1;
  const double n_mma = (double)(T->kpad / 32) * std::ceil(nprime / 128.0) * terms;
  const double t_compute = n_mma * 2.0 * 128.0 * 128.0 * 32.0 / tensor_flops;
  const double data_rw = 8.0 * cells;
  const double trans = kprime * (mprime / 2.0 + nprime) * 2.0 * (is_split(plan->dtype) ? 2 : 1);
  const double t_memory = std::max(data_rw / hbm_bytes_per_s, 2.0 * trans / smem_bytes_per_s);
  *seconds_per_step = std::max(t_compute, t_memory) / depth;
  return SPST_OK;
}

sparstencil_status sparstencil_table_kpad(sparstencil_plan_t plan, int which, int remainder_depth, int* kpad) {
  if (!plan || !kpad) return fail(SPST_ERR_INVALID, "null argument");
  std::string err;
  const SweepTables* T = which == 0 ? &plan->full : tables_for(plan, remainder_depth, &err);
  if (!T) return fail(SPST_ERR_UNSUPPORTED, err);
  *kpad = T->kpad;
  return SPST_OK;
}

sparstencil_status sparstencil_plan_tables(sparstencil_plan_t plan, int which, int remainder_depth, int* order,
                                           float* a_hi, float* a_lo, uint8_t* a_idx, int* lut, double* fused_w) {
  if (!plan) return fail(SPST_ERR_INVALID, "plan is null");
  if (which == 1 && remainder_depth < 1) return fail(SPST_ERR_INVALID, "remainder depth must be >= 1");
  std::string err;
  const SweepTables* T = which == 0 ? &plan->full : tables_for(plan, remainder_depth, &err);
  if (!T) return fail(SPST_ERR_UNSUPPORTED, err);
  if (order) std::memcpy(order, T->order.data(), T->order.size() * sizeof(int));
  const size_t nvals = T->a_val[0].size();
  const double unscale = std::ldexp(1.0, -T->wscale_log2);
  if (a_hi)
    for (size_t i = 0; i < nvals; i++) a_hi[i] = (float)((double)T->a_val[0][i] * unscale);
  if (a_lo)  // the remaining pieces, summed in FP64 and rounded once to FP32
    for (size_t i = 0; i < nvals; i++)
      a_lo[i] = (float)(((double)T->a_val[1][i] + (double)T->a_val[2][i]) * unscale);
  if (a_idx) std::memcpy(a_idx, T->a_idx.data(), T->a_idx.size());
  if (lut) std::memcpy(lut, T->lut.data(), T->lut.size() * sizeof(int));
  if (fused_w) std::memcpy(fused_w, T->wfused.data(), T->wfused.size() * sizeof(double));
  return SPST_OK;
}

sparstencil_status sparstencil_direct_run(int radius, const float* weights, int ndim, const int64_t* dims,
                                          sparstencil_boundary bc, const float* in, float* out, float* work,
                                          int64_t timesteps, cudaStream_t stream) {
  if (!weights || !dims || !in || !out || !work) return fail(SPST_ERR_INVALID, "null argument");
  if (ndim < 1 || ndim > 3) return fail(SPST_ERR_UNSUPPORTED, "ndim must be 1, 2 or 3");
  if (radius < 1 || (ndim <= 2 && radius > 4) || (ndim == 3 && radius > 3))
    return fail(SPST_ERR_UNSUPPORTED, "radius out of range");
  if (timesteps < 0) return fail(SPST_ERR_INVALID, "timesteps must be >= 0");
  spst::DirectParams prm;
  std::memset(&prm, 0, sizeof(prm));
  prm.ndim = ndim;
  prm.D = ndim == 3 ? dims[0] : 1;
  prm.H = ndim >= 2 ? dims[ndim - 2] : 1;
  prm.W = dims[ndim - 1];
  prm.radius = radius;
  prm.periodic = bc == SPST_PERIODIC ? 1 : 0;
  const int side = 2 * radius + 1;
  int total = ndim == 3 ? side * side * side : (ndim == 2 ? side * side : side);
  for (int idx = 0; idx < total; idx++) {
    if (weights[idx] == 0.f) continue;
    if (prm.npts >= 343) return fail(SPST_ERR_UNSUPPORTED, "too many stencil points");
    int rem = idx, o[3] = {0, 0, 0};
    for (int d = ndim - 1; d >= 0; d--) {
      o[3 - ndim + d] = rem % side - radius;
      rem /= side;
    }
    prm.off[prm.npts][0] = o[0];
    prm.off[prm.npts][1] = o[1];
    prm.off[prm.npts][2] = o[2];
    prm.w[prm.npts] = weights[idx];
    prm.npts++;
  }
  if (ndim <= 2 || radius == 1)
    for (int idx = 0; idx < total; idx++) prm.wdense[idx] = weights[idx];
  if (prm.H < (ndim >= 2 ? radius : 1) || prm.W < radius || prm.D < (ndim == 3 ? radius : 1))
    return fail(SPST_ERR_UNSUPPORTED, "grid smaller than the radius");
  const size_t bytes = (size_t)prm.D * prm.H * prm.W * 4;
  if (timesteps == 0) {
    SPST_CUDA(cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, stream), "copy in->out");
    return SPST_OK;
  }
  const float* src = in;
  for (int64_t s = 0; s < timesteps; s++) {
    float* dst = ((timesteps - 1 - s) % 2 == 0) ? out : work;
    SPST_CUDA(spst::launch_direct_step(prm, src, dst, stream), "direct step");
    src = dst;
  }
  return SPST_OK;
}

sparstencil_status sparstencil_error_norms(const float* x, const float* ref, int64_t n, double* out_host,
                                           cudaStream_t stream) {
  if (!x || !ref || !out_host || n < 0) return fail(SPST_ERR_INVALID, "bad norm arguments");
  double* acc = spst::device_norm_accumulator();
  if (!acc) return fail(SPST_ERR_CUDA, "norm accumulator unavailable");
  SPST_CUDA(spst::launch_error_norms(x, ref, n, acc, stream), "norm kernel");
  SPST_CUDA(cudaMemcpyAsync(out_host, acc, 4 * sizeof(double), cudaMemcpyDeviceToHost, stream), "norm D2H");
  SPST_CUDA(cudaStreamSynchronize(stream), "stream sync");
  return SPST_OK;
}

sparstencil_status sparstencil_trace(int enable) {
  const cudaError_t e = spst::sweep_trace_enable(enable ? 1 : 0);
  if (e == cudaErrorNotSupported)
    return fail(SPST_ERR_UNSUPPORTED, "library built without tracing (set SPARSTENCIL_DEBUG_TRACE=1 when building)");
  SPST_CUDA(e, "trace enable");
  return SPST_OK;
}

sparstencil_status sparstencil_trace_read(uint64_t* out, int n) {
  if (!out || n < 0) return fail(SPST_ERR_INVALID, "bad trace buffer");
  SPST_CUDA(spst::sweep_trace_read((unsigned long long*)out, n), "trace read");
  return SPST_OK;
}

sparstencil_status sparstencil_device_status(cudaStream_t stream) {
  int* w = spst::device_status_word();
  if (!w) return fail(SPST_ERR_CUDA, "device status word unavailable");
  SPST_CUDA(cudaStreamSynchronize(stream), "stream sync");
  int v = 0;
  SPST_CUDA(cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost), "read status");
  int zero = 0;
  SPST_CUDA(cudaMemcpy(w, &zero, sizeof(int), cudaMemcpyHostToDevice), "clear status");
  if (v != 0) return fail((sparstencil_status)v, "device-side error recorded");
  return SPST_OK;
}

sparstencil_status sparstencil_stream_status(cudaStream_t stream) { return sparstencil_device_status(stream); }

}  // extern "C"
