// Sparse tensor-core stencil sweep for 2D grids on sm_103a (GB300).
//
// One launch = one sweep of t fused time steps over the whole grid.  The method is the
// matrix form of Sec. 3: every r2 x r1 output patch is one column of D = A'' B'', where A''
// is the crushed staircase (Sec. 3.1) after the 2:4 permutation (Sec. 3.2) and B'' holds
// the patch's deduplicated input window in the permuted K order.  The kernel follows the
// three-stage template of Sec. 3.3 (load -> sparse MMA -> write back, double-buffered),
// re-planned for Blackwell:
//   * warp 0 streams 128 x 128-output halo tiles from the padded input grid with TMA
//     (cp.async.bulk.tensor.2d) into a 2-stage ring;
//   * warps 8-23 build B'' one 32-row K chunk at a time from the tile through the lookup
//     table (Sec. 3.3), subtract a per-patch reference value (so the tensor cores see
//     deviations, see below), convert to FP16/BF16 (split: hi and lo words) and store
//     into a 3-slot ring in the UMMA K-major layout;
//   * warp 1 issues tcgen05.mma.sp (kind::f16, M = 128, N = 128, K = 32) with A'' and its
//     2:4 metadata resident in TMEM, accumulating in FP32 in one of one or two TMEM
//     accumulators.  The weights are held as an exact sum of up to three 16-bit pieces and
//     the data as one word (single) or hi + lo (split); each K chunk issues the term table
//     A_i B_j given by the host (single: A_0 B_0 + A_1 B_0; split: A_0 B_0 + A_0 B_1 + A_1 B_0
//     + A_2 B_0), so weight rounding never enters the result as a systematic error;
//   * warps 4-7 drain the accumulator with tcgen05.ld, add back reference * sum(weights)
//     and store coalesced rows (plus periodic ghost images when writing a padded grid).
// Per-patch reference: out = c * S + sum_kappa A''[rho,kappa] (B''[kappa,n] - c) equals the
// stencil exactly for any c; with c = the patch's own input value the operands are small
// deviations, so operand rounding and accumulation errors do not bias the mean field.
// Every mbarrier wait is bounded by %globaltimer; a timeout records SPST_ERR_TIMEOUT.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <type_traits>

#include "kernels.h"

namespace spst {

namespace {

constexpr int kStatusTimeout = 5;
// Bound of the waits that drain a CTA's own copies and MMAs before it exits (independent of
// the caller's wait limit, so that a short limit never lets a CTA leave with work in flight).
constexpr uint64_t kDrainNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Non-suspending probe of the phase (mbarrier.test_wait).
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// try_wait may suspend the thread for several microseconds before it reports an incomplete
// phase, so a wait limit below this is enforced with test_wait polls instead (the limit then
// holds to within a poll, at the cost of spinning).
constexpr uint64_t kSuspendingPollMinNs = 100000;
__device__ __forceinline__ bool mbar_poll(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  return limit_ns < kSuspendingPollMinNs ? mbar_test(bar, parity) : mbar_try(bar, parity);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns, volatile int* abort_flag,
                                          int* status) {
  if (mbar_poll(bar, parity, limit_ns)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    if (mbar_poll(bar, parity, limit_ns)) return true;
    if (abort_flag && *abort_flag) return false;
    if (gtimer() - t0 > limit_ns) {
      if (abort_flag) *abort_flag = 1;
      atomicCAS(status, 0, kStatusTimeout);
      return false;
    }
  }
}

// Warp-uniform bounded wait.  SPST_POLL_ALL_LANES = 1: every lane polls the barrier (each
// lane acquires the phase itself) and the give-up decision is lane 0's; = 0: lane 0 alone
// waits and the warp synchronises behind it.
#ifndef SPST_POLL_ALL_LANES
#define SPST_POLL_ALL_LANES 1
#endif
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns, volatile int* abort_flag,
                                          int* status) {
#if SPST_POLL_ALL_LANES
  // the clock is read only once the first poll has failed: a wait that is already satisfied
  // costs one poll and one vote
  if (__all_sync(0xffffffffu, mbar_test(bar, parity))) return true;
  const uint64_t t0 = gtimer();
  const int lane = threadIdx.x & 31;
  while (true) {
    const bool d = mbar_poll(bar, parity, limit_ns);
    if (__all_sync(0xffffffffu, d)) return true;
    int give_up = 0;
    if (lane == 0) give_up = (*abort_flag) ? 1 : ((gtimer() - t0 > limit_ns) ? 2 : 0);
    give_up = __shfl_sync(0xffffffffu, give_up, 0);
    if (give_up) {
      if (lane == 0 && give_up == 2) {
        *abort_flag = 1;
        atomicCAS(status, 0, kStatusTimeout);
      }
      return false;
    }
  }
#else
  int ok = 1;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, limit_ns, abort_flag, status) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
#endif
}

__device__ __forceinline__ uint64_t make_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; no swizzle, base offset 0
  return d;
}

// tcgen05.commit by one elected lane of a converged warp: the barrier gets one arrival when
// every tcgen05 operation the issuing thread started before it has completed.
__device__ __forceinline__ void commit_elected(uint32_t bar) {
  asm volatile(
      "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}" ::"r"(bar)
      : "memory");
}

// One K chunk's MMAs (1 to 4 terms: A piece x B piece) and the commit that frees the chunk's
// B'' slot, issued by one elected lane of a converged warp in a single block.  The first term
// goes to the accumulator at d, the others to the one at d1 (d1 = d, or the low-order
// accumulator); en / en1: accumulate onto d / d1 for the first term that writes each (0 for
// the tile's first chunk).
#define SPST_MMA_SP(D, A, B, P) " @e tcgen05.mma.sp.cta_group::1.kind::f16 [" D "], [" A "], " B ", [%9], %10, " P ";\n"
#define SPST_COMMIT " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%12];\n"
#define SPST_PREDS \
  "{\n .reg .pred e, q, q1, t;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 q, %11, 0;\n setp.ne.b32 q1, %14, 0;\n" \
  " setp.eq.b32 t, %11, %11;\n"
__device__ __forceinline__ void issue_chunk(int nterms, uint32_t d, uint32_t d1, uint32_t a0, uint32_t a1, uint32_t a2,
                                            uint32_t a3, uint64_t b0, uint64_t b1, uint64_t b2, uint64_t b3, uint32_t meta,
                                            uint32_t idesc, uint32_t en, uint32_t en1, uint32_t bar) {
#define SPST_CHUNK_OPERANDS                                                                                   \
  "r"(d), "r"(a0), "r"(a1), "r"(a2), "r"(a3), "l"(b0), "l"(b1), "l"(b2), "l"(b3), "r"(meta), "r"(idesc), "r"(en), \
      "r"(bar), "r"(d1), "r"(en1)
  switch (nterms) {
    case 1:
      asm volatile(SPST_PREDS SPST_MMA_SP("%0", "%1", "%5", "q") SPST_COMMIT "}" ::SPST_CHUNK_OPERANDS : "memory");
      break;
    case 2:
      asm volatile(SPST_PREDS SPST_MMA_SP("%0", "%1", "%5", "q") SPST_MMA_SP("%13", "%2", "%6", "q1")
                       SPST_COMMIT "}" ::SPST_CHUNK_OPERANDS
                   : "memory");
      break;
    case 3:
      asm volatile(SPST_PREDS SPST_MMA_SP("%0", "%1", "%5", "q") SPST_MMA_SP("%13", "%2", "%6", "q1")
                       SPST_MMA_SP("%13", "%3", "%7", "t") SPST_COMMIT "}" ::SPST_CHUNK_OPERANDS
                   : "memory");
      break;
    default:
      asm volatile(SPST_PREDS SPST_MMA_SP("%0", "%1", "%5", "q") SPST_MMA_SP("%13", "%2", "%6", "q1")
                       SPST_MMA_SP("%13", "%3", "%7", "t") SPST_MMA_SP("%13", "%4", "%8", "t") SPST_COMMIT
                   "}" ::SPST_CHUNK_OPERANDS
                   : "memory");
      break;
  }
#undef SPST_CHUNK_OPERANDS
#undef SPST_PREDS
}

// One dense MMA (kind::f16, M = 128, N = 128, K = 16; A in TMEM, B from a shared-memory
// descriptor) by one elected lane of a converged warp; acc = 0 overwrites the accumulator.
__device__ __forceinline__ void mma_dense_elected(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred e, q;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 q, %4, 0;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, q;\n}" ::"r"(d),
      "r"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi, int fp16) {
  uint32_t r;
  if (fp16)
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  else
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ void unpack2(uint32_t v, int fp16, float& lo, float& hi) {
  if (fp16) {
    unsigned short a = (unsigned short)(v & 0xffffu), b = (unsigned short)(v >> 16);
    asm("cvt.f32.f16 %0, %1;" : "=f"(lo) : "h"(a));
    asm("cvt.f32.f16 %0, %1;" : "=f"(hi) : "h"(b));
  } else {
    lo = __uint_as_float(v << 16);
    hi = __uint_as_float(v & 0xffff0000u);
  }
}

__device__ __forceinline__ float lds_f32(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ int2 lds_v2_s32(uint32_t a) {
  int2 v;
  asm volatile("ld.shared.v2.s32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ float4 lds_v4_f32(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts_u32(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void sts_f32(uint32_t a, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

// Optional timeline trace of CTA 0 (off unless enabled from the host): per role and tile,
// the %globaltimer when the role's first wait for the tile completed and when it finished
// the tile.  Layout: [role 0 TMA, 1 MMA, 2 gather warp, 3 epilogue warp][tile < 64][2].
constexpr int kTraceTiles = 64;
__device__ int g_trace_on;
__device__ unsigned long long g_trace[4 * kTraceTiles * 2];

// Built in only with -DSPST_TRACE=1 (the stamps cost ~15% of the sweep's time).
#ifndef SPST_TRACE
#define SPST_TRACE 0
#endif
__device__ __forceinline__ void trace(bool on, int role, int li, int ev) {
#if SPST_TRACE
  if (on && li < kTraceTiles) g_trace[(role * kTraceTiles + li) * 2 + ev] = gtimer();
#endif
}
// Chunk-level clock64 stamps in CTA 0 for tile 1: [source][chunk < 16][4], sources 0 and 1
// the first and the last gather warp (chunk start, slot free, stores issued, chunk
// published), source 2 the MMA issuer (chunk's B'' complete, MMAs issued, -, -).
constexpr int kTraceChunkWords = 3 * 16 * 4 + 2 * 16 * 16;  // + [gather warp][chunk] publish / stored stamps
__device__ unsigned long long g_trace_chunks[kTraceChunkWords];
__device__ __forceinline__ void trace_chunk(bool on, int src, int kc, int ev) {
  if (SPST_TRACE && on && kc < 16) {
    unsigned long long c;
    asm volatile("mov.u64 %0, %%clock64;" : "=l"(c));
    g_trace_chunks[(src * 16 + kc) * 4 + ev] = c;
  }
}

struct SmemLayout {
  uint32_t halo_stride, off_b, slot_bytes, off_lut, off_cv, off_bar, total;
  __host__ __device__ explicit SmemLayout(const Sweep2DParams& p) {
    uint32_t halo = (uint32_t)p.box_d * (uint32_t)p.box_h * (uint32_t)p.P * 4u;
    halo_stride = (halo + 1023u) & ~1023u;
    off_b = halo_stride * (uint32_t)(p.hstages == 1 ? 1 : kHaloStages);
    slot_bytes = (uint32_t)p.b_pieces * (uint32_t)kPieceBytes;
    off_lut = off_b + slot_bytes * (uint32_t)p.nslots;
    off_cv = off_lut + (((uint32_t)p.kpad * 4u + 15u) & ~15u);
    off_bar = off_cv + 2u * 128u * 4u;
    total = off_bar + 512u;
  }
};

// barrier indices (8 bytes each, from off_bar)
constexpr int BAR_HFULL = 0, BAR_HEMPTY = 2, BAR_BFULL = 4, BAR_BEMPTY = 4 + kMaxBSlots,
              BAR_AFULL = 4 + 2 * kMaxBSlots, BAR_AEMPTY = BAR_AFULL + 2, BAR_CVFULL = BAR_AEMPTY + 2,
              BAR_CVEMPTY = BAR_CVFULL + 2, BAR_FINAL = BAR_CVEMPTY + 2;
constexpr int BAR_COUNT = BAR_FINAL + 1;  // 29 barriers = 232 bytes, below the TMEM slot at +256
static_assert(BAR_COUNT * 8 <= 256, "barrier area overlaps the TMEM slot");
constexpr uint32_t TMEM_COLS = 512;

constexpr int k1dTile = 16384, k1dRow = 256;  // 1D: outputs per tile, floats per row of the 2D view
constexpr int kGatherWarp0 = 4 + kEpiWarps;                     // the last 16 warps build B''
constexpr int kGatherWarps = kSweepThreads / 32 - kGatherWarp0;  // 16
constexpr int kItems = 64 / kGatherWarps;                        // patch pairs per gather warp per chunk

// DIM = 1: 1D sweep (patches of 128 consecutive outputs, tiles of 128 patches read as whole
// rows of a 2D view of the padded line); DIM = 2: 2D sweep (Tile2D: 16 x 8 patches, 128 x 128
// tiles); DIM = 3: 3D sweep (Tile3D:
// 8 x 4 x 4 patches, 64 x 16 x 16 tiles).  Patch n of a 3D tile, with n = a*16 + h*8 + b, is
// (px, py, pz) = (4(a&1) + 2h + (b&1), b>>1, a>>1): the two half-warps of a gather warp take
// patches n and n+8, 16 words apart in x, as in 2D.
// The sweep of one grid by CTA `cta` of the `ncta` CTAs given to it: tiles cta, cta + ncta, ...
// tmap_in: the TMA map of the input padded grid (kernel parameter space).
template <int FP16, int SPLIT, int DIM, int TALL>
__device__ __forceinline__ void sweep_body(const CUtensorMap* tmap_in, const Sweep2DParams& p, const int cta,
                                           const int ncta) {
  constexpr bool DIM3 = DIM == 3, DIM1 = DIM == 1;
  constexpr bool kTall = DIM == 2 && TALL != 0;  // 2D 8 x 16 patches (compiled apart: the 16 x 8 path is unchanged)
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  uint8_t* smem = smem_raw + (sbase - raw);
  const SmemLayout L(p);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar0 = sbase + L.off_bar;
  auto bar = [&](int i) -> uint32_t { return bar0 + 8u * (uint32_t)i; };
  uint32_t* tmem_slot = (uint32_t*)(smem + L.off_bar + 256);               // 16-byte aligned
  volatile int* abort_flag = (volatile int*)(smem + L.off_bar + 272);
  int32_t* lut_s = (int32_t*)(smem + L.off_lut);
  const int pieces = p.a_pieces;
  const int acols = p.dense ? p.kpad / 2 : p.kpad / 4;  // TMEM columns per A piece
  const int nacc = p.nacc;
  const uint64_t wait_ns = p.wait_ns;

  // ---------------- set-up ----------------
  if (threadIdx.x == 0) {
    mbar_init(bar(BAR_HFULL + 0), 1);
    mbar_init(bar(BAR_HFULL + 1), 1);
    mbar_init(bar(BAR_HEMPTY + 0), kGatherWarps);
    mbar_init(bar(BAR_HEMPTY + 1), kGatherWarps);
    for (int s = 0; s < p.nslots; s++) {
      mbar_init(bar(BAR_BFULL + s), kGatherWarps);
      mbar_init(bar(BAR_BEMPTY + s), 1);
    }
    for (int a = 0; a < 2; a++) {
      mbar_init(bar(BAR_AFULL + a), 1);
      mbar_init(bar(BAR_AEMPTY + a), kEpiWarps);
      mbar_init(bar(BAR_CVFULL + a), kGatherWarps);
      mbar_init(bar(BAR_CVEMPTY + a), kEpiWarps);
    }
    mbar_init(bar(BAR_FINAL), 1);
    abort_flag[0] = 0;
    abort_flag[1] = 0;
    abort_flag[2] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  for (int i = threadIdx.x; i < p.kpad; i += blockDim.x) lut_s[i] = p.lut[i];
  // A'' pieces and metadata: all threads copy them (16-byte loads) into a staging area that
  // overlays halo stage 1 and the chunk slots (free until the main loop), rows padded so that
  // the epilogue warps read them back without bank conflicts; then those warps store them to
  // TMEM (lane = output row of the patch).
  const int apitch = acols + 4;                       // words per staged A'' row
  const int mpitch = p.kchunks | 1;                   // words per staged metadata row (odd)
  const uint32_t stage_a = sbase;  // staging area (shared address)
  const uint32_t stage_m = stage_a + 4u * (uint32_t)(pieces * 128 * apitch);
  {
    const int q4 = acols / 4;  // uint4 per A'' row
    const uint4* src = reinterpret_cast<const uint4*>(p.a_words);
    for (int i = threadIdx.x; i < pieces * 128 * q4; i += blockDim.x) {
      const uint4 v = src[i];
      const int row = i / q4, c4 = i % q4;  // row = piece * 128 + lane
      const uint32_t a = stage_a + 4u * (uint32_t)(row * apitch + 4 * c4);
      asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                   : "memory");
    }
    if (!p.dense)
      for (int i = threadIdx.x; i < 128 * p.kchunks; i += blockDim.x)
        sts_u32(stage_m + 4u * (uint32_t)((i / p.kchunks) * mpitch + i % p.kchunks), p.meta_words[i]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;
  // accumulators first (nacc of them, each 128 columns, or 256 with the low-order accumulator
  // right after the main one), then the A'' pieces, then the metadata
  const uint32_t acc_stride = p.lo_acc ? 256u : 128u;
  const uint32_t a_col = acc_stride * (uint32_t)nacc;
  const uint32_t meta_col = a_col + (uint32_t)(pieces * acols);

  if (warp >= 4 && warp < 8) {
    const int q = warp - 4;
    const int row = 32 * q + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
    for (int pc = 0; pc < pieces; pc++) {
      const uint32_t ra = stage_a + 4u * (uint32_t)((pc * 128 + row) * apitch);
      for (int c = 0; c < acols; c += 8) {
        uint32_t v[8];
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                     : "r"(ra + 4u * (uint32_t)c));
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                     : "r"(ra + 4u * (uint32_t)(c + 4)));
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(
                         lane_addr + a_col + (uint32_t)(pc * acols + c)),
                     "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]));
      }
    }
    // chunk c's metadata column: an 8-column-aligned pair per two chunks, the instruction's
    // sparsity selector (0/1) picks the column inside the pair (none for the dense ablation)
    for (int c = 0; c < (p.dense ? 0 : p.kchunks); c++) {
      uint32_t v;
      asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(stage_m + 4u * (uint32_t)(row * mpitch + c)));
      asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(
                       lane_addr + meta_col + 8u * (uint32_t)(c >> 1) + (uint32_t)(c & 1)),
                   "r"(v));
    }
    asm volatile("tcgen05.wait::st.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  // Programmatic dependent launch: the set-up above reads only this launch's tables (written
  // before the previous kernel started) and may overlap the previous sweep; the grids are
  // read and written only after that sweep has completed and its writes are visible.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // the next sweep may be scheduled now; its own griddepcontrol.wait orders its grid
  // accesses after this grid's completion
  asm volatile("griddepcontrol.launch_dependents;");
  // FP16 data scale 2^k (read after the wait: the copy-in wrote max|u0|)
  float dscale = 1.f, dscale_inv = 1.f;
  if (FP16 && p.maxabs) {
    const float bound = 2.f * __uint_as_float(*(const volatile unsigned*)p.maxabs) * p.growth;
    if (bound > 1e-30f && bound < 3.0e38f) {
      int e;
      frexpf(8192.f / bound, &e);  // 8192 / bound = f * 2^e, f in [0.5, 1)
      const int kk = min(max(e - 1, -60), 60);
      dscale = ldexpf(1.f, kk);
      dscale_inv = ldexpf(1.f, -kk);
    }
  }

  const int ntiles_cta = (p.num_tiles > cta) ? (p.num_tiles - 1 - cta) / ncta + 1 : 0;
  const bool tr = (blockIdx.x == 0) && g_trace_on;
  const bool hs2 = p.hstages != 1;  // two halo stages (one: the next tile loads after this one's gather)

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      const uint32_t bytes = (uint32_t)p.box_d * (uint32_t)p.box_h * (uint32_t)p.P * 4u;
      int issued = 0;
      for (int li = 0; li < ntiles_cta; li++) {
        // halo stage and the number of its earlier uses (two stages, or one when the fused
        // radius leaves room for a single halo tile only)
        const int stage = hs2 ? li & 1 : 0, use = hs2 ? li >> 1 : li;
        if (use >= 1 && !mbar_wait(bar(BAR_HEMPTY + stage), (use - 1) & 1, wait_ns, abort_flag, p.status)) break;
        const int tt = cta + li * ncta;
        const uint32_t dst = sbase + (uint32_t)stage * L.halo_stride;
        trace(tr, 0, li, 0);
        mbar_expect_tx(bar(BAR_HFULL + stage), bytes);
        if (DIM1) {
          // whole rows of the 2D view of the padded line: tile tt starts at row tt * 64
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                  dst),
              "l"(tmap_in), "r"(0), "r"(tt * (k1dTile / k1dRow)), "r"(bar(BAR_HFULL + stage))
              : "memory");
        } else if (DIM3) {
          const int tx = tt % p.tiles_x, ty = (tt / p.tiles_x) % p.tiles_y, tz = tt / (p.tiles_x * p.tiles_y);
          asm volatile(
              "cp.async.bulk.tensor.3d.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
                  dst),
              "l"(tmap_in), "r"(tx * 64), "r"(ty * 16), "r"(tz * 16), "r"(bar(BAR_HFULL + stage))
              : "memory");
        } else {
          const int x0 = (tt % p.tiles_x) * 128, y0 = (tt / p.tiles_x) * 128;
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                  dst),
              "l"(tmap_in), "r"(x0), "r"(y0), "r"(bar(BAR_HFULL + stage))
              : "memory");
        }
        issued++;
      }
      // the CTA never exits with one of its copies in flight (at most the last one per stage can be)
      const int nst = hs2 ? 2 : 1;
      for (int li = (issued > nst ? issued - nst : 0); li < issued; li++)
        mbar_wait(bar(BAR_HFULL + (hs2 ? li & 1 : 0)), (hs2 ? li >> 1 : li) & 1, kDrainNs, nullptr, p.status);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    // The whole warp runs the loop (warp-uniform waits and addresses) and one elected lane
    // issues each tcgen05 instruction.  The per-term operand addresses are fixed before the
    // tile loop, so an MMA costs an add or two: the issue loop is a single latency chain, and
    // at about 70 cycles per sparse 128x128x32 MMA any dependent work in it is exposed.
    uint32_t idesc = 0;
    idesc |= 1u << 2;                      // sparse
    idesc |= 1u << 4;                      // D = FP32
    idesc |= (p.fp16 ? 0u : 1u) << 7;      // A: FP16 (0) / BF16 (1)
    idesc |= (p.fp16 ? 0u : 1u) << 10;     // B: FP16 (0) / BF16 (1)
    idesc |= (uint32_t)(128 >> 3) << 17;   // N = 128
    idesc |= (uint32_t)(128 >> 4) << 24;   // M = 128
    const uint32_t idesc_dense = idesc & ~(1u << 2);  // the same shape and types, dense
    const int nterms = p.nterms;
    uint32_t a_term[4], b_term[4];  // TMEM address of the term's A'' piece; B piece offset (16-byte units)
#pragma unroll
    for (int t = 0; t < 4; t++) {
      a_term[t] = tmem + a_col + (uint32_t)((t < nterms ? p.term_a[t] : 0) * acols);
      b_term[t] = (uint32_t)((t < nterms ? p.term_b[t] : 0) * (kPieceBytes >> 4));
    }
    // descriptor of slot 0, piece 0; the start-address field (bits 0-13, 16-byte units) of
    // any slot and piece stays below 2^14 (shared memory < 256 KB), so offsets add to the low word
    const uint64_t desc0 = make_sdesc(sbase + L.off_b, kLBO, kSBO);
    const uint32_t dlo0 = (uint32_t)desc0, dhi = (uint32_t)(desc0 >> 32);
    const uint32_t slot_step = L.slot_bytes >> 4;
    // the tile loop, compiled once for sparse and once for dense MMAs (the issue loop is a
    // latency chain: the MMA form is fixed outside it)
    auto issue_tiles = [&](auto dense_tag) {
      constexpr bool kDense = decltype(dense_tag)::value;
      uint32_t mslot = 0, mphase = 0;  // chunk ring position and wrap parity
      bool ok = true;
      for (int li = 0; li < ntiles_cta && ok; li++) {
        const int acc = li % nacc, use = li / nacc;
        if (use > 0 && !warp_wait(bar(BAR_AEMPTY + acc), (use - 1) & 1, wait_ns, abort_flag, p.status)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        trace(tr && lane == 0, 1, li, 0);
        const uint32_t dcol = tmem + (uint32_t)acc * acc_stride;
        const uint32_t dcol1 = p.lo_acc ? dcol + 128u : dcol;
        for (int kc = 0; kc < p.kchunks; kc++) {
          const uint32_t slot = mslot, su = mphase;
          if (++mslot == (uint32_t)p.nslots) {
            mslot = 0;
            mphase ^= 1u;
          }
          if (!warp_wait(bar(BAR_BFULL + slot), su & 1, wait_ns, abort_flag, p.status)) {
            ok = false;
            break;
          }
          trace_chunk(tr && li == 1 && lane == 0, 2, kc, 0);
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t blo = dlo0 + slot * slot_step;
          const uint32_t meta = tmem + meta_col + 8u * (uint32_t)(kc >> 1);
          const uint32_t idesc_kc = idesc | (uint32_t)(kc & 1);  // sparsity selector
          const uint32_t a8 = 8u * (uint32_t)kc;
          const uint64_t b0 = ((uint64_t)dhi << 32) | (uint64_t)(blo + b_term[0]);
          const uint64_t b1 = ((uint64_t)dhi << 32) | (uint64_t)(blo + b_term[1]);
          const uint64_t b2 = ((uint64_t)dhi << 32) | (uint64_t)(blo + b_term[2]);
          const uint64_t b3 = ((uint64_t)dhi << 32) | (uint64_t)(blo + b_term[3]);
          if constexpr (kDense) {
            // dense ablation: two K = 16 MMAs per term and chunk (A columns 16kc and 16kc + 8,
            // B rows 0-15 and 16-31 of the chunk: two core matrices of 16 bytes along K = 2 LBO)
            const uint64_t bt[4] = {b0, b1, b2, b3};
  #pragma unroll
            for (int t = 0; t < 4; t++) {
              if (t < nterms) {
  #pragma unroll
                for (int h = 0; h < 2; h++) {
                  const uint32_t acc = (h > 0 || kc > 0) ? 1u : (t == 0 ? 0u : (t == 1 && p.lo_acc ? 0u : 1u));
                  mma_dense_elected(t == 0 ? dcol : dcol1, a_term[t] + 16u * (uint32_t)kc + 8u * (uint32_t)h,
                                    bt[t] + (uint64_t)(h * (2 * kLBO >> 4)), idesc_dense, acc);
                }
              }
            }
            commit_elected(bar(BAR_BEMPTY + slot));
          } else {
            issue_chunk(nterms, dcol, dcol1, a_term[0] + a8, a_term[1] + a8, a_term[2] + a8, a_term[3] + a8, b0, b1, b2,
                        b3, meta, idesc_kc, kc > 0 ? 1u : 0u, (kc > 0 || !p.lo_acc) ? 1u : 0u, bar(BAR_BEMPTY + slot));
          }
          trace_chunk(tr && li == 1 && lane == 0, 2, kc, 1);
        }
        if (!ok) break;
        commit_elected(bar(BAR_AFULL + acc));
        trace(tr && lane == 0, 1, li, 1);
      }
    };
    if (p.dense)
      issue_tiles(std::integral_constant<bool, true>());
    else
      issue_tiles(std::integral_constant<bool, false>());
    // every MMA issued above completes before TMEM is released
    commit_elected(bar(BAR_FINAL));
    if (lane == 0) mbar_wait(bar(BAR_FINAL), 0, kDrainNs, nullptr, p.status);
    __syncwarp();
  } else if (warp >= 4 && warp < 4 + kEpiWarps) {
    // ---------------- epilogue ----------------
    // warp 4 + q + 4h reads TMEM lanes 32q .. 32q+31 (its lane quarter) and, with 8 epilogue
    // warps, accumulator columns 64h .. 64h+63
    const int q = (warp - 4) & 3;
    constexpr int kGroups = 8 / (kEpiWarps / 4);  // 16-column groups per warp
    const int cg0 = ((warp - 4) >> 2) * kGroups;
    const int rho = 32 * q + lane;
    // row rho of a patch: 2D (ry, rx) = (rho / 16, rho % 16); 3D (rz, ry, rx) = (rho / 32,
    // rho / 8 % 4, rho % 8)
    const int rz = DIM3 ? rho >> 5 : 0;
    const int ry = DIM3 ? (rho >> 3) & 3 : (kTall ? rho >> 3 : rho >> 4);
    const int rx = DIM3 ? rho & 7 : (kTall ? rho & 7 : rho & 15);
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
    const uint32_t cv_s = sbase + L.off_cv;
    const float out_scale = p.wscale * dscale_inv;  // undoes the weight and data scales (powers of two)
    const int G = p.out_off;
    const int64_t pitch8 = 8 * p.out_pitch;
    for (int li = 0; li < ntiles_cta; li++) {
      const int acc = li % nacc, use = li / nacc;
      if (!warp_wait(bar(BAR_AFULL + acc), use & 1, wait_ns, abort_flag, p.status)) break;
      if (!warp_wait(bar(BAR_CVFULL + (li & 1)), (li >> 1) & 1, wait_ns, abort_flag, p.status)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      trace(tr && warp == 4 && lane == 0, 3, li, 0);
      const int tt = cta + li * ncta;
      if (DIM1) {
        // column n of the accumulator is patch n: outputs x0 + 128n + rho, a lane per output
        const int64_t x0 = (int64_t)tt * k1dTile;
        const bool full1 = x0 + k1dTile <= p.W;
        float* ob = p.out + G + x0 + rho;
#pragma unroll 1
        for (int cg = cg0; cg < cg0 + kGroups; cg++) {
          uint32_t v[16];
          const uint32_t acc_addr = lane_addr + (uint32_t)acc * acc_stride + (uint32_t)(cg * 16);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(acc_addr));
          if (SPLIT && p.lo_acc) {
            uint32_t l[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(l[0]), "=r"(l[1]), "=r"(l[2]), "=r"(l[3]), "=r"(l[4]), "=r"(l[5]), "=r"(l[6]), "=r"(l[7]),
                  "=r"(l[8]), "=r"(l[9]), "=r"(l[10]), "=r"(l[11]), "=r"(l[12]), "=r"(l[13]), "=r"(l[14]), "=r"(l[15])
                : "r"(acc_addr + 128u));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int j = 0; j < 16; j++) v[j] = __float_as_uint(__uint_as_float(v[j]) + __uint_as_float(l[j]));
          }
          float c[16];
          const uint32_t ca = cv_s + (uint32_t)((li & 1) * 128 + cg * 16) * 4u;
#pragma unroll
          for (int k4 = 0; k4 < 4; k4++) {
            const float4 c4 = lds_v4_f32(ca + 16u * k4);
            c[4 * k4] = c4.x;
            c[4 * k4 + 1] = c4.y;
            c[4 * k4 + 2] = c4.z;
            c[4 * k4 + 3] = c4.w;
          }
          asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
          for (int j = 0; j < 16; j++) {
            const int n = cg * 16 + j;
            const float val = fmaf(c[j], p.S_lo, fmaf(c[j], p.S_hi, __uint_as_float(v[j]) * out_scale));
            if (full1 || x0 + n * 128 + rho < p.W) ob[n * 128] = val;
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(bar(BAR_AEMPTY + acc));
          mbar_arrive(bar(BAR_CVEMPTY + (li & 1)));
        }
        continue;
      }
      const int tx = tt % p.tiles_x, ty = DIM3 ? (tt / p.tiles_x) % p.tiles_y : tt / p.tiles_x;
      const int x0 = tx * (DIM3 ? 64 : 128), y0 = ty * (DIM3 ? 16 : 128);
      const int z0 = DIM3 ? (tt / (p.tiles_x * p.tiles_y)) * 16 : 0;
      // full tiles store without bounds checks; 2D tiles that touch the ghost band of a periodic
      // padded output also write the images of their band outputs (a 3D sweep's ghost shell
      // is refreshed by a separate kernel)
      const bool full = DIM3 ? (z0 + 16 <= p.D && y0 + 16 <= p.H && x0 + 64 <= p.W)
                             : ((y0 + 128 <= p.H) && (x0 + 128 <= p.W));
      const bool ghost = !DIM3 && p.out_ghost && (y0 < G || y0 + 128 > p.H - G || x0 < G || x0 + 128 > p.W - G);
      float* obase = p.out + (int64_t)(z0 + G + rz) * (DIM3 ? p.out_plane : 0) + (int64_t)(y0 + G + ry) * p.out_pitch +
                     (x0 + G + rx);
#pragma unroll 1
      for (int cg = cg0; cg < cg0 + kGroups; cg++) {
        uint32_t v[16];
        const uint32_t acc_addr = lane_addr + (uint32_t)acc * acc_stride + (uint32_t)(cg * 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(acc_addr));
        if (SPLIT && p.lo_acc) {
          // the low-order accumulator, added in FP32 (RN) to the main one
          uint32_t l[16];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(l[0]), "=r"(l[1]), "=r"(l[2]), "=r"(l[3]), "=r"(l[4]), "=r"(l[5]), "=r"(l[6]), "=r"(l[7]),
                "=r"(l[8]), "=r"(l[9]), "=r"(l[10]), "=r"(l[11]), "=r"(l[12]), "=r"(l[13]), "=r"(l[14]), "=r"(l[15])
              : "r"(acc_addr + 128u));
          asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
          for (int j = 0; j < 16; j++) v[j] = __float_as_uint(__uint_as_float(v[j]) + __uint_as_float(l[j]));
        }
        float c[16];
        const uint32_t ca = cv_s + (uint32_t)((li & 1) * 128 + cg * 16) * 4u;
#pragma unroll
        for (int k4 = 0; k4 < 4; k4++) {
          const float4 c4 = lds_v4_f32(ca + 16u * k4);
          c[4 * k4] = c4.x;
          c[4 * k4 + 1] = c4.y;
          c[4 * k4 + 2] = c4.z;
          c[4 * k4 + 3] = c4.w;
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        float val[16];
#pragma unroll
        for (int j = 0; j < 16; j++) val[j] = fmaf(c[j], p.S_lo, fmaf(c[j], p.S_hi, __uint_as_float(v[j]) * out_scale));
        if (DIM3) {
          // columns cg*16 + j are patches (px, py, pz) = (4(cg&1) + 2(j/8) + (j&1), (j&7)/2, cg/2)
          const int pz = cg >> 1, pxh = (cg & 1) << 2;
          const int64_t zoff = (int64_t)pz * 4 * p.out_plane;
#pragma unroll
          for (int j = 0; j < 16; j++) {
            const int px = pxh | ((j >> 3) << 1) | (j & 1), py = (j & 7) >> 1;
            const int64_t o = zoff + (int64_t)py * 4 * p.out_pitch + px * 8;
            if (full || (z0 + pz * 4 + rz < p.D && y0 + py * 4 + ry < p.H && x0 + px * 8 + rx < p.W)) obase[o] = val[j];
          }
          continue;
        }
        // column cg*16 + j is the patch whose outputs start yoff rows and xoff columns into
        // the tile: 16 x 8 patches (py, px) = (cg/4*8 + j%8, (2cg + j/8) % 8); tall 8 x 16
        // patches (py, px) = (cg, 4((j%8)/2) + 2(j/8) + j%2)
        auto yoff = [&](int j) { return kTall ? cg * 16 : (((cg >> 2) << 3) + (j & 7)) * 8; };
        auto xoff = [&](int j) {
          return kTall ? (4 * ((j & 7) >> 1) + 2 * (j >> 3) + (j & 1)) * 8 : (((2 * cg) & 7) + (j >> 3)) * 16;
        };
        if (full && !kTall) {
          const int py0 = (cg >> 2) << 3, px0 = (2 * cg) & 7;
#pragma unroll
          for (int j = 0; j < 16; j++) obase[(int64_t)(py0 + (j & 7)) * pitch8 + (px0 + (j >> 3)) * 16] = val[j];
        } else if (full) {
          const int64_t row = (int64_t)cg * 2 * pitch8;  // 16 rows per patch
#pragma unroll
          for (int j = 0; j < 16; j++) obase[row + (4 * ((j & 7) >> 1) + 2 * (j >> 3) + (j & 1)) * 8] = val[j];
        } else {
#pragma unroll
          for (int j = 0; j < 16; j++) {
            const int y = y0 + yoff(j) + ry, x = x0 + xoff(j) + rx;
            if (y < p.H && x < p.W) obase[(int64_t)yoff(j) * p.out_pitch + xoff(j)] = val[j];
          }
        }
        if (ghost) {
          for (int j = 0; j < 16; j++) {
            const int y = y0 + yoff(j) + ry, x = x0 + xoff(j) + rx;
            if (y >= p.H || x >= p.W) continue;
            const bool by = (y < G) || (y >= p.H - G), bx = (x < G) || (x >= p.W - G);
            if (!by && !bx) continue;
            const int yi = y < G ? y + p.H + G : (y >= p.H - G ? y - p.H + G : -1);
            const int xi = x < G ? x + p.W + G : (x >= p.W - G ? x - p.W + G : -1);
            if (yi >= 0) p.out[(int64_t)yi * p.out_pitch + (x + G)] = val[j];
            if (xi >= 0) p.out[(int64_t)(y + G) * p.out_pitch + xi] = val[j];
            if (yi >= 0 && xi >= 0) p.out[(int64_t)yi * p.out_pitch + xi] = val[j];
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(bar(BAR_AEMPTY + acc));
        mbar_arrive(bar(BAR_CVEMPTY + (li & 1)));
      }
      trace(tr && warp == 4 && lane == 0, 3, li, 1);
    }
  } else if (warp >= kGatherWarp0) {
    // ---------------- B'' gather ----------------
    // Lane (h, pl) handles pair pl (K rows 2pl, 2pl+1) of each chunk for patch n0 + 8h of each
    // of its patch pairs: the two patches are one x-step apart (their tile offsets differ by 16
    // words, so the half-warps use disjoint banks) and land in different 8-patch groups (their
    // B'' offsets differ by SBO = 16 words mod 32).  All loads of a chunk are issued before
    // any of them is used, and before the wait for the chunk's slot.
    const int gw = warp - kGatherWarp0;
    const int h = lane >> 4, pl = lane & 15;
    const uint32_t pairoff = (uint32_t)((pl >> 2) * kLBO + (pl & 3) * 4);
    const int P = p.P, G = p.G;
    uint32_t slot = 0, sphase = 0, used = 0;  // chunk ring position, wrap parity, chunks written
    int base_i[kItems], n_i[kItems];
    uint32_t soff_i[kItems];
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      const int pp = gw + kGatherWarps * i;
      const int n = (pp >> 3) * 16 + (pp & 7) + 8 * h;
      n_i[i] = n;
      if (DIM1) {
        base_i[i] = 4 * (n * 128);  // patch n: outputs 128n .. 128n+127 of the tile
      } else if (DIM3) {
        const int a = n >> 4, b = n & 7;
        const int px = ((a & 1) << 2) | (h << 1) | (b & 1), py = b >> 1, pz = a >> 1;
        base_i[i] = 4 * (pz * 4 * p.box_h * P + py * 4 * P + px * 8);
      } else if (kTall) {
        // 8 x 16 patches: column n = 16 py + 8 hb + e is patch (px, py) = (4(e>>1) + 2hb + (e&1),
        // n >> 4), so the half-warps' patches (hb = h) are two patches, 16 words, apart in x
        const int e = n & 7, hb = (n >> 3) & 1;
        const int px = 4 * (e >> 1) + 2 * hb + (e & 1), py = n >> 4;
        base_i[i] = 4 * (py * 16 * P + px * 8);
      } else {
        const int px = (n >> 3) & 7, py = ((n >> 6) << 3) + (n & 7);
        base_i[i] = 4 * (py * 8 * P + px * 16);
      }
      soff_i[i] = (uint32_t)((n >> 3) * kSBO + (n & 7) * 16) + pairoff;
    }
    const uint32_t lut_sa = sbase + L.off_lut + 8u * (uint32_t)pl;
    // this lane's sample of the patch constant's 8 inputs (bits of pl mod 8: 3D z, y, x;
    // 2D row, then two bits of column)
    const int sm = pl & 7;
    const uint32_t c_off =
        4u * (uint32_t)(DIM1 ? sm
                             : DIM3 ? (sm >> 2) * p.box_h * P + ((sm >> 1) & 1) * P + (sm & 1) : (sm >> 2) * P + (sm & 3));
    for (int li = 0; li < ntiles_cta; li++) {
      const int stage = hs2 ? li & 1 : 0;
      if (!warp_wait(bar(BAR_HFULL + stage), (hs2 ? li >> 1 : li) & 1, wait_ns, abort_flag, p.status)) break;
      trace(tr && gw == 0 && lane == 0, 2, li, 0);
      const uint32_t tile_s = sbase + (uint32_t)stage * L.halo_stride;
      uint32_t ba[kItems];
      float c_i[kItems];
#pragma unroll
      for (int i = 0; i < kItems; i++) {
        ba[i] = tile_s + (uint32_t)base_i[i];
        // the patch constant: the mean of the 8 inputs in the middle of the patch's outputs
        // (2D rows 3-4 x columns 6-9 of its 8 rows x 16 columns, rows 7-8 x columns 2-5 of a
        // tall 16 x 8 patch; 3D the central 2 x 2 x 2 of its 4 x 4 x 8).
        // Any c gives the same sum (sum w (u - c) + c sum w); the MMAs round their FP32
        // partial sums, so c should keep |u - c| small: near the local value for smooth data
        // with an offset, near the local mean (not one sample of it) for rough zero-mean data
        // The 16 lanes of a half-warp share the patch: lane pl loads sample pl mod 8 and an
        // xor butterfly over 8 lanes sums them (the same sum in every lane: each level adds
        // the same two partial sums, and FP32 addition is commutative).
        const uint32_t m0 = ba[i] + 4u * (uint32_t)(DIM1 ? G + 60
                                                         : DIM3 ? (G + 1) * p.box_h * P + (G + 1) * P + G + 3
                                                                : kTall ? (G + 7) * P + G + 2 : (G + 3) * P + G + 6);
        float cs = lds_f32(m0 + c_off);
        cs += __shfl_xor_sync(0xffffffffu, cs, 1);
        cs += __shfl_xor_sync(0xffffffffu, cs, 2);
        cs += __shfl_xor_sync(0xffffffffu, cs, 4);
        c_i[i] = 0.125f * cs;
      }
      // the patch constants go to a two-slot area of their own, so that building B'' for this
      // tile never waits for the epilogue that is draining the accumulator
      const int cvs = li & 1;
      if (li >= 2 && !warp_wait(bar(BAR_CVEMPTY + cvs), ((li >> 1) - 1) & 1, wait_ns, abort_flag, p.status)) break;
      if (pl == 0) {
#pragma unroll
        for (int i = 0; i < kItems; i++) sts_f32(sbase + L.off_cv + 4u * (uint32_t)(cvs * 128 + n_i[i]), c_i[i]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(BAR_CVFULL + cvs));
      bool ok = true;
      // Software pipeline: chunk kc's values are loaded one chunk ahead, and the lookup-table
      // entries of chunk kc+2 two chunks ahead, so no shared-memory load of this warp waits
      // on another one; the next chunk's loads are issued after this chunk's proxy fence,
      // which then waits for this chunk's stores only.
      const bool trc = tr && (gw == 0 || gw == kGatherWarps - 1) && lane == 0 && li == 1;
      const int tsrc = gw == 0 ? 0 : 1;
      float va[kItems], vb[kItems];
      int2 lab_next;  // LUT entries of the next chunk to load
      {
        const int2 lab0 = lds_v2_s32(lut_sa);
        lab_next = p.kchunks > 1 ? lds_v2_s32(lut_sa + 128u) : lab0;
        const uint32_t la = 4u * (uint32_t)lab0.x, lb = 4u * (uint32_t)lab0.y;
#pragma unroll
        for (int i = 0; i < kItems; i++) {
          va[i] = lds_f32(ba[i] + la);
          vb[i] = lds_f32(ba[i] + lb);
        }
      }
      for (int kc = 0; kc < p.kchunks; kc++) {
        trace_chunk(trc, tsrc, kc, 0);
        if (used >= (uint32_t)p.nslots &&
            !warp_wait(bar(BAR_BEMPTY + slot), sphase ^ 1u, wait_ns, abort_flag, p.status)) {
          ok = false;
          break;
        }
        trace_chunk(trc, tsrc, kc, 1);
        const uint32_t bs = sbase + L.off_b + slot * L.slot_bytes;
#pragma unroll
        for (int i = 0; i < kItems; i++) {
          const float da = (va[i] - c_i[i]) * dscale;
          const float db = (vb[i] - c_i[i]) * dscale;
          const uint32_t hi = pack2(da, db, FP16);
          sts_u32(bs + soff_i[i], hi);
          if (SPLIT) {
            float ha, hb;
            unpack2(hi, FP16, ha, hb);
            sts_u32(bs + kPieceBytes + soff_i[i], pack2(da - ha, db - hb, FP16));
          }
        }
        trace_chunk(trc, tsrc, kc, 2);
#if SPST_TRACE
        if (tr && li == 1 && lane == 0 && kc < 16) {
          unsigned long long c;
          asm volatile("mov.u64 %0, %%clock64;" : "=l"(c)::"memory");
          g_trace_chunks[3 * 16 * 4 + 16 * 16 + gw * 16 + kc] = c;
        }
#endif
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor core
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(BAR_BFULL + slot));
        used++;
        if (++slot == (uint32_t)p.nslots) {
          slot = 0;
          sphase ^= 1u;
        }
        trace_chunk(trc, tsrc, kc, 3);
#if SPST_TRACE
        if (tr && li == 1 && lane == 0 && kc < 16) {
          unsigned long long c;
          asm volatile("mov.u64 %0, %%clock64;" : "=l"(c));
          g_trace_chunks[3 * 16 * 4 + gw * 16 + kc] = c;
        }
#endif
        if (kc + 1 < p.kchunks) {
          const uint32_t la = 4u * (uint32_t)lab_next.x, lb = 4u * (uint32_t)lab_next.y;
#pragma unroll
          for (int i = 0; i < kItems; i++) {
            va[i] = lds_f32(ba[i] + la);
            vb[i] = lds_f32(ba[i] + lb);
          }
          if (kc + 2 < p.kchunks) lab_next = lds_v2_s32(lut_sa + 128u * (uint32_t)(kc + 2));
        }
      }
      if (!ok) break;
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(BAR_HEMPTY + stage));
      trace(tr && gw == 0 && lane == 0, 2, li, 1);
    }
  }

  // ---------------- teardown ----------------
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// One grid per launch: every CTA takes its share of the grid's tiles.
template <int FP16, int SPLIT, int DIM, int TALL = 0>
__global__ void __launch_bounds__(kSweepThreads, 1)
    sweep2d_kernel(const __grid_constant__ CUtensorMap tmap_in, const __grid_constant__ Sweep2DParams p) {
  sweep_body<FP16, SPLIT, DIM, TALL>(&tmap_in, p, (int)blockIdx.x, (int)gridDim.x);
}

// Many grids per launch (a batch's sweeps of one index): CTA b works on job cta_job[b], as CTA
// b - cta_first[job] of the cta_count[job] CTAs given to that job, with the job's own tables,
// tensor map and output; a CTA never changes job, so its set-up (TMEM tables, lookup table)
// is the single-grid one.
template <int FP16, int SPLIT, int DIM, int TALL = 0>
__global__ void __launch_bounds__(kSweepThreads, 1) sweep2d_multi_kernel(const __grid_constant__ MultiSweepParams m) {
  const int j = m.cta_job[blockIdx.x];
  sweep_body<FP16, SPLIT, DIM, TALL>(&m.tmap[j], m.job[j], (int)blockIdx.x - m.cta_first[j], m.cta_count[j]);
}

}  // namespace

size_t sweep2d_smem_bytes(const Sweep2DParams& p) { return (size_t)SmemLayout(p).total + 1024; }

cudaError_t sweep_trace_enable(int on) {
  if (!SPST_TRACE) return cudaErrorNotSupported;
  cudaError_t e = cudaMemcpyToSymbol(g_trace_on, &on, sizeof(int));
  if (e != cudaSuccess) return e;
  static const unsigned long long zeros[4 * kTraceTiles * 2] = {0};
  static const unsigned long long zc[kTraceChunkWords] = {0};
  e = cudaMemcpyToSymbol(g_trace_chunks, zc, sizeof(zc));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(g_trace, zeros, sizeof(zeros));
}

cudaError_t sweep_trace_read(unsigned long long* out, int n) {
  const int n1 = 4 * kTraceTiles * 2;
  cudaError_t e = cudaMemcpyFromSymbol(out, g_trace, (size_t)(n < n1 ? n : n1) * sizeof(unsigned long long));
  if (e != cudaSuccess || n <= n1) return e;
  const int n2 = (n - n1 < kTraceChunkWords) ? n - n1 : kTraceChunkWords;
  return cudaMemcpyFromSymbol(out + n1, g_trace_chunks, (size_t)n2 * sizeof(unsigned long long));
}

#ifndef SPST_SLOT_CAP
#define SPST_SLOT_CAP kMaxBSlots
#endif
// Bytes of the A'' / metadata staging area used during set-up.
static size_t staging_bytes(const Sweep2DParams& p) {
  const int acols = p.dense ? p.kpad / 2 : p.kpad / 4;
  return 4u * ((size_t)p.a_pieces * 128 * (acols + 4) + (p.dense ? 0 : (size_t)128 * (p.kchunks | 1)));
}

int sweep2d_max_slots(const Sweep2DParams& p) {
  Sweep2DParams q = p;
  for (int n = SPST_SLOT_CAP; n >= 1; n--) {
    q.nslots = n;
    if (sweep2d_smem_bytes(q) <= 232448) return n;
  }
  return 0;
}

int sweep2d_halo_stages(const Sweep2DParams& p_in) {
  Sweep2DParams p = p_in;
  for (int s = kHaloStages; s >= 1; s--) {
    p.hstages = s;
    if (sweep2d_fits(p)) return s;
  }
  return 0;
}

bool sweep2d_fits(const Sweep2DParams& p_in) {
  Sweep2DParams p = p_in;
  p.nslots = sweep2d_max_slots(p);
  if (p.nslots < 2) return false;
  return staging_bytes(p) <= (size_t)SmemLayout(p).off_lut;
}

namespace {
thread_local bool t_pdl = true;
}
void sweep2d_set_programmatic_launch(bool on) { t_pdl = on; }

namespace {
// The chunk-slot count and early-TMA flag of a sweep (as launch_sweep2d sets them); false if
// the geometry does not fit.
bool finish_params(Sweep2DParams* p) {
  p->nslots = sweep2d_max_slots(*p);
  if (p->nslots < 2) return false;
  const SmemLayout L(*p);
  const size_t need = staging_bytes(*p);
  p->early_tma = (need <= (size_t)(L.off_lut - L.halo_stride)) ? 1 : 0;
  return need <= (size_t)L.off_lut;
}

// The kernel instance of a sweep's template parameters (operand word, split, dimensionality,
// 2D patch shape).
using SingleKernel = void (*)(const CUtensorMap, const Sweep2DParams);
using MultiKernel = void (*)(const MultiSweepParams);
template <template <int, int, int, int> class Sel>
typename Sel<0, 0, 2, 0>::type pick_kernel(const Sweep2DParams& p) {
  const bool s = p.b_pieces > 1;
  if (p.dim3) return p.fp16 ? (s ? Sel<1, 1, 3, 0>::get() : Sel<1, 0, 3, 0>::get()) : (s ? Sel<0, 1, 3, 0>::get() : Sel<0, 0, 3, 0>::get());
  if (p.dim1) return p.fp16 ? (s ? Sel<1, 1, 1, 0>::get() : Sel<1, 0, 1, 0>::get()) : (s ? Sel<0, 1, 1, 0>::get() : Sel<0, 0, 1, 0>::get());
  if (p.tall) return p.fp16 ? (s ? Sel<1, 1, 2, 1>::get() : Sel<1, 0, 2, 1>::get()) : (s ? Sel<0, 1, 2, 1>::get() : Sel<0, 0, 2, 1>::get());
  return p.fp16 ? (s ? Sel<1, 1, 2, 0>::get() : Sel<1, 0, 2, 0>::get()) : (s ? Sel<0, 1, 2, 0>::get() : Sel<0, 0, 2, 0>::get());
}
template <int A, int B, int C, int D>
struct SelSingle {
  using type = SingleKernel;
  static type get() { return sweep2d_kernel<A, B, C, D>; }
};
template <int A, int B, int C, int D>
struct SelMulti {
  using type = MultiKernel;
  static type get() { return sweep2d_multi_kernel<A, B, C, D>; }
};
}  // namespace

cudaError_t launch_sweep2d_multi(const CUtensorMap* maps, const Sweep2DParams* prm, int njobs, int num_sms,
                                 cudaStream_t stream) {
  if (njobs < 1 || njobs > kMultiMaxJobs) return cudaErrorInvalidValue;
  thread_local MultiSweepParams m;  // about 23 KB: kept off the stack
  std::memset(&m, 0, sizeof(m));
  m.njobs = njobs;
  size_t smem = 0;
  int64_t total_tiles = 0;
  for (int j = 0; j < njobs; j++) {
    m.tmap[j] = maps[j];
    m.job[j] = prm[j];
    if (!finish_params(&m.job[j])) return cudaErrorInvalidConfiguration;
    if (m.job[j].fp16 != prm[0].fp16 || m.job[j].b_pieces != prm[0].b_pieces || m.job[j].dim3 != prm[0].dim3 ||
        m.job[j].dim1 != prm[0].dim1)
      return cudaErrorInvalidValue;
    if (m.job[j].tall != prm[0].tall) return cudaErrorInvalidValue;
    const size_t s = sweep2d_smem_bytes(m.job[j]);
    smem = s > smem ? s : smem;
    total_tiles += m.job[j].num_tiles;
  }
  // CTAs: one per job, then the rest one at a time to the job with the most tiles per CTA
  int ctas = num_sms < kMultiMaxCtas ? num_sms : kMultiMaxCtas;
  if (total_tiles < ctas) ctas = (int)total_tiles;
  if (ctas < njobs) return cudaErrorInvalidConfiguration;
  for (int j = 0; j < njobs; j++) m.cta_count[j] = 1;
  for (int c = njobs; c < ctas; c++) {
    int best = -1;
    double best_load = 0.0;
    for (int j = 0; j < njobs; j++) {
      if (m.cta_count[j] >= m.job[j].num_tiles) continue;
      const double load = (double)m.job[j].num_tiles / m.cta_count[j];
      if (load > best_load) {
        best_load = load;
        best = j;
      }
    }
    if (best < 0) break;
    m.cta_count[best]++;
  }
  int next = 0;
  for (int j = 0; j < njobs; j++) {
    m.cta_first[j] = next;
    for (int c = 0; c < m.cta_count[j]; c++) m.cta_job[next + c] = (int16_t)j;
    next += m.cta_count[j];
  }
  m.nctas = next;
  const MultiKernel kern = pick_kernel<SelMulti>(m.job[0]);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)m.nctas);
  cfg.blockDim = dim3(kSweepThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = t_pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, m);
}

cudaError_t launch_sweep2d(const CUtensorMap& tmap_in, const Sweep2DParams& p_in, int num_sms, cudaStream_t stream) {
  Sweep2DParams p = p_in;
  p.nslots = sweep2d_max_slots(p);
  if (p.nslots < 2) return cudaErrorInvalidConfiguration;
  {
    const SmemLayout L(p);
    const size_t need = staging_bytes(p);
    p.early_tma = (need <= (size_t)(L.off_lut - L.halo_stride)) ? 1 : 0;
    if (need > (size_t)L.off_lut) return cudaErrorInvalidConfiguration;
  }
  const size_t smem = sweep2d_smem_bytes(p);
  const SingleKernel kern = pick_kernel<SelSingle>(p);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = p.num_tiles < num_sms ? p.num_tiles : num_sms;
  if (grid < 1) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kSweepThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = t_pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, tmap_in, p);
}

}  // namespace spst
