/*
 * sparstencil.h — C ABI of the GB300 (sm_103a) SparStencil library.
 *
 * The library runs iterated constant-coefficient stencils (Sec. 2.2: every grid point
 * becomes the weighted sum of its neighbours, repeated for T time steps; weights are
 * indexed by offset and not flipped, as in the Box-2D9P pseudo-code) as 2:4
 * structured-sparse matrix multiplies D = (A o M) B + C on tcgen05 sparse tensor cores
 * (Eq. 1-2).  A host planner applies Adaptive Layout Morphing (Sec. 3.1: flatten, then
 * horizontal and vertical duplicate crush into a staircase matrix A'), Structured
 * Sparsity Conversion (Sec. 3.2: conflict graph + Algorithm 1, then the permutation
 * invariant transformation) and the kernel-generation tables (Sec. 3.3: 2:4 metadata and
 * the gather lookup table).  Each sweep then runs as one persistent kernel: TMA halo tile
 * -> shared-memory gather of B' -> tcgen05.mma.sp with FP32 accumulation in TMEM ->
 * coalesced write-back.
 *
 * Conventions shared by every entry point
 *   - Every call returns a sparstencil_status and never aborts or throws.  On failure
 *     sparstencil_last_error() returns a thread-local message.
 *   - Grids are FP32, contiguous, row-major; dims[0] is the slowest axis.  Device grids
 *     are caller-owned and must not alias.  Weights are host FP32, a dense cube of side
 *     2r+1 (same axis order, entry for offset o at index sum_i (o_i + r)(2r+1)^(d-1-i)).
 *   - Calls that take a cudaStream_t only enqueue work on it (asynchronous) unless stated.
 *   - Device-side waits are bounded; a kernel that gives up records SPST_ERR_TIMEOUT in the
 *     library's device status word, read with sparstencil_device_status().
 */
#ifndef SPARSTENCIL_H_
#define SPARSTENCIL_H_

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sparstencil_plan_s* sparstencil_plan_t; /* opaque, library-owned */

typedef enum {
  SPST_OK = 0,
  SPST_ERR_INVALID = 1,      /* bad argument (null pointer, bad size, bad enum, ...) */
  SPST_ERR_UNSUPPORTED = 2,  /* valid request outside what this library implements */
  SPST_ERR_NOMEM = 3,        /* device or host allocation failed, or workspace too small */
  SPST_ERR_CUDA = 4,         /* a CUDA runtime/driver call failed */
  SPST_ERR_TIMEOUT = 5,      /* a bounded device wait gave up */
  SPST_ERR_DEVICE_CHECK = 6  /* a device-side consistency check failed */
} sparstencil_status;

typedef enum { SPST_STAR = 0, SPST_BOX = 1, SPST_CUSTOM = 2 } sparstencil_shape;

/* Operand precision on the tensor cores (accumulation is always FP32 in TMEM).
 * Single-word modes round each operand once (RN-even); split modes carry every operand
 * as hi + lo and issue A_hi B_hi + A_hi B_lo + A_lo B_hi into one accumulator. */
typedef enum { SPST_FP16 = 0, SPST_BF16 = 1, SPST_FP16_SPLIT = 2, SPST_BF16_SPLIT = 3 } sparstencil_dtype;

typedef enum { SPST_DIRICHLET_ZERO = 0, SPST_PERIODIC = 1 } sparstencil_boundary;

/* Description of a plan (sparstencil_query). */
typedef struct {
  int ndim;            /* 1, 2 or 3 */
  int radius;          /* stencil radius r */
  int fusion_depth;    /* t: time steps fused per sweep (composed kernel of radius t*r) */
  int r1, r2, r3;      /* crush factors (outputs per patch along x, y, z); r1*r2*r3 = 128 */
  int kprime;          /* k' = columns of the staircase matrix A' (Sec. 3.3, m'/k'/n') */
  int kpad;            /* K after matching and padding to the MMA's K (multiple of 32) */
  int zero_columns;    /* zero columns inserted by Algorithm 1 (before padding) */
  int mma_terms;       /* tensor-core MMAs per K chunk (1 single, 3 split) */
  int tile_outputs;    /* outputs per CTA tile */
  int64_t num_tiles;   /* tiles per sweep */
  double planner_ms;   /* host time spent in sparstencil_plan */
  int ghost;           /* ghost width G of the padded ping-pong grids (= largest fused radius) */
  int tile_pitch;      /* floats per row of the shared-memory halo tile (TMA box width) */
  int tile_rows;       /* rows of the halo tile (TMA box height) */
  int bank_conflicts;  /* residue repeats left by the planner's chunk packing (0: the B'' gather
                          reads shared memory without bank conflicts) */
  int low_accumulator; /* 1: split terms after A_hi B_hi accumulate separately (see below) */
  int dense_ablation;  /* 1: dense tcgen05 MMAs on the uncompressed A' (see below) */
  int pairing;         /* column pairs of the 2:4 conversion: 0 = Algorithm 1 (Sec. 3.2), 1 = a
                          maximum matching on the stencil's actual support, taken when the
                          support is smaller than the box and that needs fewer K chunks */
  int fp64_every;      /* k of the FP64 correction step (0: off; see
                          sparstencil_plan_set_fp64_correction) */
} sparstencil_plan_info;

/* Builds a plan for `shape` stencils of radius `radius` on an ndim grid (1, 2 or 3) of extents dims.
 *   weights: host FP32 cube (see conventions), copied; for SPST_STAR/SPST_BOX only the
 *            shape's points may be nonzero (checked), SPST_CUSTOM accepts any support.
 *   fusion_depth: t >= 1 fuses t steps per sweep; 0 lets the library choose: the plan
 *            takes the deepest depth whose tables fit TMEM and shared memory, searched
 *            from 6 down to 1 in 2D, from 60 / radius in 1D and from 3 in 3D
 *            (Dirichlet fusion: 2D, radius <= 4), and the first sparstencil_run
 *            times two sweeps of every depth up to it (1D: of the powers of two below it and
 *            of the maximum), for every candidate layout (see sparstencil_plan_set_layout), on
 *            its own input (after one warm-up sweep each; that call synchronises its stream
 *            once) and keeps the combination with the least time per step.
 *            sparstencil_query reports the planned maximum depth until then.
 *   out_plan: receives the plan (owned by the library until sparstencil_plan_destroy).
 * Host only (no device work).  Errors: SPST_ERR_INVALID, SPST_ERR_UNSUPPORTED
 * (ndim not 1, 2 or 3, radius too large for TMEM, ...), SPST_ERR_NOMEM.
 * Follows the problem statement of Sec. 2.2 and the planning steps of Sec. 3.1-3.3. */
sparstencil_status sparstencil_plan(sparstencil_shape shape, int radius, const float* weights, int ndim,
                                    const int64_t* dims, sparstencil_dtype dtype, sparstencil_boundary bc,
                                    int fusion_depth, sparstencil_plan_t* out_plan);

/* Split dtypes only: enable != 0 sends the low-order MMA terms (A_hi B_lo, A_lo B_hi, ...) to
 * a TMEM accumulator of their own, which the epilogue adds in FP32 to the A_hi B_hi one.
 * Every tensor-core MMA rounds its FP32 result once; with one accumulator each low-order term
 * costs a rounding at the magnitude of the whole partial sum, with two only the A_hi B_hi
 * chain does (about 3x less error on rough data, e.g. zero-mean 3D grids over 50 steps).
 * A tile then takes 256 TMEM columns, so the next tile's MMAs no longer overlap this tile's
 * write-back; BF16 split keeps three weight pieces only where they fit beside them (with two
 * pieces its weight rounding, 2^-17, outweighs what the second accumulator saves).
 * Default: on for SPST_FP16_SPLIT plans where it fits (their operands hold 22 bits, so the
 * MMA roundings dominate) and for 3D SPST_BF16_SPLIT plans where it fits beside three weight
 * pieces (a 3D step runs many more MMAs per output than a fused 2D or 1D step), off
 * otherwise.
 * Must be called before the plan's first run (it rebuilds the host tables).
 * Errors: SPST_ERR_INVALID (null plan, single-word dtype, plan already ran),
 * SPST_ERR_UNSUPPORTED (the plan's fusion depth does not fit in TMEM this way; the plan is
 * left unchanged).  Host only. */
sparstencil_status sparstencil_plan_set_low_accumulator(sparstencil_plan_t plan, int enable);

/* Fixes the plan's layout instead of leaving it to the search of a fusion_depth-0 plan:
 *   r1:      2D patch shape, 16 (16 x 8 outputs per patch, 8 patches across a 128 x 128 tile,
 *            the default) or 8 (8 x 16, 16 across); 1D and 3D plans accept only their own r1
 *            (128 and 8)
 *   pairing: column pairing of the 2:4 conversion (Sec. 3.2): 0 = Algorithm 1, 1 = a maximum
 *            matching on the stencil's actual support (stars, custom masks), -1 = whichever
 *            needs fewer K chunks (the default)
 * A plan made with fusion_depth 0 otherwise times, at its first run, every depth of its search
 * with both 2D patch shapes and, for supports smaller than their box, both pairings, and keeps
 * the fastest combination (the layout search of Sec. 3.3, Eq. 11, done by measurement);
 * sparstencil_query reports the choice (r1, r2, pairing).  Must be called before the plan's
 * first run.  Errors: SPST_ERR_INVALID (null plan, bad pairing, plan already ran),
 * SPST_ERR_UNSUPPORTED (other r1, or the layout does not fit; the plan is left unchanged).
 * Host only. */
sparstencil_status sparstencil_plan_set_layout(sparstencil_plan_t plan, int r1, int pairing);

/* The dense-versus-sparse ablation: enable != 0 runs the same morphed, permuted A' (Sec. 3.1-3.2)
 * as dense tcgen05 MMAs (kind::f16, K = 16 per instruction, the 2:4 zeros stored explicitly in
 * TMEM, no metadata) instead of sparse ones (Eq. 1, K = 32 per instruction).  Same tables, same
 * gather and epilogue, same results up to the MMA summation order; it shows what the 2:4
 * structure buys.  The uncompressed A' takes twice the TMEM columns, so a plan may fall back to
 * one accumulator, to two BF16 split weight pieces, or (FP16 split) leave the low-order
 * accumulator off.  The allocation-free run does not take such plans.  Must be called before the plan's first
 * run.  Errors: SPST_ERR_INVALID (null plan, plan already ran), SPST_ERR_UNSUPPORTED (the
 * uncompressed A' does not fit in TMEM or its staging in shared memory; the plan is left
 * unchanged).  Host only. */
sparstencil_status sparstencil_plan_set_dense_ablation(sparstencil_plan_t plan, int enable);

/* Runs `timesteps` stencil steps: out = S^timesteps in (Sec. 2.2), on `stream`.
 *   in, out: device FP32 grids of prod(dims) elements, caller-owned, must not alias;
 *            in is only read.
 *   timesteps = 0 copies in to out.
 * Uses the plan's workspace (bound, or allocated on first use: SPST_ERR_NOMEM on failure).
 * Asynchronous: enqueues the sweeps (ceil(timesteps / t) kernels plus one copy-in) and
 * returns.  Calls on one plan must not overlap on the GPU (they share the workspace).
 * A run may be captured into a CUDA graph (stream capture on `stream`) once the plan has run
 * once with the same timesteps (workspace and tables on the device, fusion depth chosen);
 * the capture records the sweeps' programmatic dependent launches as programmatic edges. */
sparstencil_status sparstencil_run(sparstencil_plan_t plan, const float* in, float* out, int64_t timesteps,
                                   cudaStream_t stream);

/* Same as sparstencil_run with HOST grids: brings in (host) to the device, runs, and copies
 * the result back to out (host), all on `stream`.  Page-locked input that the device can
 * address (cudaHostAlloc / cudaHostRegister) is read directly by the copy-in kernel; other
 * input is first copied to a device staging grid.  Synchronises the stream before
 * returning. */
sparstencil_status sparstencil_run_host(sparstencil_plan_t plan, const float* in_host, float* out_host,
                                        int64_t timesteps, cudaStream_t stream);

/* Same as sparstencil_run_host, but asynchronous: the host-to-device copy into the plan's
 * staging grid, the sweeps and the device-to-host copy are queued on `stream` (copies on the
 * copy engines) and the call returns without synchronising, so that runs of several plans
 * on several streams overlap one run's copies with another's sweeps.  in_host and out_host
 * must stay valid (and out_host unread) until `stream` has passed the run; page-locked
 * memory makes the copies asynchronous.  A plan holds one staging pair: at most one run of
 * a plan may be in flight (runs of one plan on one stream are ordered by the stream). */
sparstencil_status sparstencil_run_host_async(sparstencil_plan_t plan, const float* in_host, float* out_host,
                                              int64_t timesteps, cudaStream_t stream);

/* Same as sparstencil_run, but records CUDA events before and after the copy into the
 * padded grid and after the last sweep, and synchronises `stream` before returning:
 *   copy_in_ms:  device time of the copy into the padded grid (may be NULL)
 *   sweeps_ms:   device time from the end of that copy to the end of the last sweep, gaps
 *                between consecutive sweeps included (may be NULL)
 *   num_sweeps:  number of sweep kernels launched (may be NULL)
 * Used by the benchmark to report the sweep kernel's own bandwidth. */
sparstencil_status sparstencil_run_profiled(sparstencil_plan_t plan, const float* in, float* out, int64_t timesteps,
                                            cudaStream_t stream, double* copy_in_ms, double* sweeps_ms,
                                            int* num_sweeps);

/* Allocation-free variant of sparstencil_run, for callers that cannot call cudaMalloc:
 * services that forbid device allocation once running (cudaMalloc can synchronise the
 * device) and processes whose device memory belongs to a framework allocator with a fixed
 * budget.  The paper has no counterpart; this is a deployment convenience.
 *   plan, in, out, timesteps, stream: as for sparstencil_run (in and out stay caller-owned).
 * Instead of the plan's workspace it uses two file-scope static device arrays that every
 * GPU loading the library holds until exit: 32 MiB of ping-pong grids (at most 4,194,304
 * padded cells per grid, e.g. a 2040 x 2040 grid with ghost width 4) and 512 KiB of
 * planner tables.  Larger grids are rejected with SPST_ERR_UNSUPPORTED and a message.
 * It calls no cudaMalloc, cudaFree or allocating library routine; the first call on a
 * device resolves the arrays' device addresses (cudaGetSymbolAddress).  All calls share the
 * arrays: each call clears what must
 * start at zero and uploads the plan's tables from host memory (cudaMemcpyAsync on
 * `stream`), and calls that overlap on the GPU race.  2D sparse plans only.  The plan
 * runs at the depth sparstencil_query reports: a plan made with fusion_depth 0 that no
 * sparstencil_run has tuned yet runs at its deepest planned depth (this entry point times
 * no depths). */
sparstencil_status sparstencil_run_noalloc(sparstencil_plan_t plan, const float* in, float* out, int64_t timesteps,
                                           cudaStream_t stream);

/* Optional FP64 correction step (not in the paper's method): with every_k = k >= 1, time
 * steps k, 2k, 3k, ... of each run are each computed by one CUDA-core step in FP64
 * arithmetic from the FP32 state (every nonzero weight times its input summed in FP64 in
 * (dz, dy, dx) order, rounded once to FP32), and the k - 1 steps between them by the plan's
 * tensor-core sweeps (fused as usual, with a remainder sweep where k - 1 is not a multiple
 * of the depth).  every_k = 1 runs every step in FP64; 0 (the default) turns it off.
 * sparstencil_run, _run_host, _run_host_async and _run_profiled honour it;
 * sparstencil_run_batch and sparstencil_run_noalloc reject such plans with
 * SPST_ERR_UNSUPPORTED.  Errors: SPST_ERR_INVALID (null plan, every_k < 0). */
sparstencil_status sparstencil_plan_set_fp64_correction(sparstencil_plan_t plan, int every_k);

/* Releases the plan and every device buffer the library allocated for it. */
sparstencil_status sparstencil_plan_destroy(sparstencil_plan_t plan);

/* Bytes of device workspace the plan needs (two padded ping-pong grids). */
size_t sparstencil_workspace_bytes(sparstencil_plan_t plan);

/* Binds caller-owned device memory as the plan's workspace (>= sparstencil_workspace_bytes,
 * 256-byte aligned).  The library never frees it.  Zero-fills it on `stream`. */
sparstencil_status sparstencil_bind_workspace(sparstencil_plan_t plan, void* dev, size_t bytes,
                                              cudaStream_t stream);

/* Runs n independent jobs (plans[i] on in[i] -> out[i] for steps[i] steps) as one CUDA
 * graph launched on `stream`: the jobs' copy-ins, then for each sweep index s one persistent
 * launch of the multi-grid sweep kernel over every job that has a sweep s (per kernel
 * template: FP16 or BF16, single or split words, dimensionality; at most 64 jobs per
 * launch).  The launch shares the SMs out by tile count, at least one CTA per job; a CTA
 * works on one job's tiles with that job's tables and tensor map, so many small grids share
 * the GPU in each launch.  Dirichlet bands and periodic ghost refreshes of the jobs that
 * need them follow each launch.  Plans must be distinct.  The first call for a set of jobs prepares every plan (workspace, the
 * fusion-depth search of fusion_depth-0 plans, device tables), synchronises `stream`,
 * captures and instantiates the graph and launches it.  The library keeps the instantiated
 * graph (up to 16 of them, least recently used dropped first): a later call with the same
 * plans in the same state (workspace, fusion depth), the same grids and the same step counts
 * only launches it, asynchronously and without synchronising.  Destroying a plan or binding
 * it a new workspace drops the graphs that use it.  Results equal those of sparstencil_run
 * on each job (same plans, same kernels).  Errors as sparstencil_run, plus
 * SPST_ERR_INVALID for repeated plans. */
sparstencil_status sparstencil_run_batch(const sparstencil_plan_t* plans, const float* const* in,
                                         float* const* out, const int64_t* steps, int n, cudaStream_t stream);

/* The cost model of Sec. 3.3 (Eq. 6-11), T = max(T_compute, T_memory), for a sweep of depth
 * `depth` (1 .. the plan's fusion depth) of this plan, written to *seconds_per_step as the
 * sweep's time divided by depth.  T_compute = executed sparse MMA flops / tensor_flops (one
 * 128x128x32 MMA per K chunk, 128-patch tile and MMA term); T_memory = max(8 B per output /
 * hbm_bytes_per_s, (data_transR + data_transW) / smem_bytes_per_s) with data_trans =
 * k'(m'/2 + n') 16-bit elements per operand piece (reading: m means m').  The rates are the
 * caller's (measured or nominal).  Host only; builds the depth's tables if needed.
 * Errors: SPST_ERR_INVALID (null pointers, depth out of range, rates not positive). */
sparstencil_status sparstencil_cost_model(sparstencil_plan_t plan, int depth, double tensor_flops,
                                          double hbm_bytes_per_s, double smem_bytes_per_s,
                                          double* seconds_per_step);

/* Fills *info (host only). */
sparstencil_status sparstencil_query(sparstencil_plan_t plan, sparstencil_plan_info* info);

/* Copies the planner's tables for one sweep kind (which = 0: full sweeps of depth t,
 * which = 1: the remainder sweep of depth timesteps mod t, built on demand for
 * `remainder_depth` >= 1) into caller host arrays; any pointer may be NULL.
 *   order:      kpad ints, original column of A' per permuted K position, -1 = zero column
 *   a_hi, a_lo: 128 * kpad/2 floats, compressed A'' values: a_hi is the first 16-bit piece
 *               of each weight, a_lo the sum of its remaining pieces (single-word modes keep
 *               two pieces, split modes three, or two for a fused sweep whose three pieces
 *               would leave TMEM room for only one accumulator; with three BF16 pieces
 *               a_hi + a_lo is the FP32 weight)
 *   a_idx:      128 * kpad/2 bytes, in-group position (0..3) of each compressed value
 *   lut:        kpad ints, tile-word offset gathered for each permuted K position
 *   fused_w:    (2tr+1)^ndim doubles, the composed weights of the sweep
 * Host only.  Sizes come from sparstencil_query (kpad) for which = 0; for which = 1 call
 * sparstencil_table_kpad first. */
sparstencil_status sparstencil_plan_tables(sparstencil_plan_t plan, int which, int remainder_depth, int* order,
                                           float* a_hi, float* a_lo, uint8_t* a_idx, int* lut, double* fused_w);

/* kpad of the sweep kind selected as in sparstencil_plan_tables (host only). */
sparstencil_status sparstencil_table_kpad(sparstencil_plan_t plan, int which, int remainder_depth, int* kpad);

/* Plain FP32 CUDA-core direct stencil (the comparator): one launch per time step, FP32
 * FMAs in fixed offset order, no tensor cores and no temporal blocking.
 *   in, out: device FP32 grids; work: device scratch of prod(dims) floats (ping-pong);
 *   all caller-owned.  Asynchronous on `stream`. */
sparstencil_status sparstencil_direct_run(int radius, const float* weights, int ndim, const int64_t* dims,
                                          sparstencil_boundary bc, const float* in, float* out, float* work,
                                          int64_t timesteps, cudaStream_t stream);

/* FP64 error norms of x against ref (device FP32 arrays of n elements):
 * out_host[0] = sum (x-ref)^2, [1] = sum ref^2, [2] = max|x-ref|, [3] = max|ref|.
 * Synchronises `stream`.  Used for verification only (not on the timed path). */
sparstencil_status sparstencil_error_norms(const float* x, const float* ref, int64_t n, double* out_host,
                                           cudaStream_t stream);

/* Reads and clears the library's device status word on the current device after
 * synchronising `stream`: SPST_OK, or the first device-side error recorded
 * (SPST_ERR_TIMEOUT, SPST_ERR_DEVICE_CHECK). */
sparstencil_status sparstencil_device_status(cudaStream_t stream);

/* The same as sparstencil_device_status (the name the problem statement's interface uses). */
sparstencil_status sparstencil_stream_status(cudaStream_t stream);

/* Sets the bound (nanoseconds) of every device-side wait; 0 restores the default (2 s).
 * Host only; applies to launches made after the call. */
sparstencil_status sparstencil_set_wait_limit_ns(uint64_t ns);

/* Debugging aid, present only in libraries built with tracing (build.py with the
 * environment variable SPARSTENCIL_DEBUG_TRACE=1; otherwise SPST_ERR_UNSUPPORTED, because the
 * stamps slow the sweep by ~15%): enable (1) or disable (0) the sweep kernel's timeline
 * trace on the current device.  When enabled, CTA 0 of each sweep records %globaltimer stamps (nanoseconds) for
 * its first 64 tiles: per role (0 TMA producer, 1 MMA issuer, 2 first B'' gather warp,
 * 3 first epilogue warp) the time its first wait for the tile completed and the time it
 * finished the tile.  Enabling clears the buffer.  Synchronous; not for timed runs. */
sparstencil_status sparstencil_trace(int enable);

/* Copies up to n trace entries to host memory; synchronous.  Entries 0..511: layout
 * [role][tile][start, end] (4 x 64 x 2, nanoseconds); entries 512..703: clock64 stamps of
 * the K chunks of CTA 0's second tile, [source][chunk < 16][4]: sources 0 and 1 the first and
 * the last B'' gather warp (chunk start, chunk slot free, stores issued, chunk
 * published), source 2 the MMA issuer (chunk complete in shared memory, MMAs issued);
 * entries 704..959: [gather warp < 16][chunk < 16] publish stamps of the same tile;
 * entries 960..1215: the same warps' stamps just before the chunk's proxy fence. */
sparstencil_status sparstencil_trace_read(uint64_t* out, int n);

/* ---------------------------------------------------------------------------------------
 * Serving: a request loop over the library (not in the paper; the runtime that takes
 * stencil jobs as they arrive).  A dispatcher thread admits jobs in arrival order when one
 * of `slots` execution slots (CUDA streams) is free and the job's device bytes fit under
 * `hbm_budget_bytes` next to the jobs running; each admitted job copies its grid in (unless
 * it is already on the device), runs and copies its result out (unless it stays on the
 * device) on its own stream, side by side with the others, and releases its slot and bytes
 * when its work completes.  A job that can never fit the budget fails with SPST_ERR_NOMEM.
 * Plans are pooled by stencil and grid and reused by later jobs; the server's device
 * allocations come from a memory pool of its own that keeps up to the budget resident
 * between jobs (no allocation reaches the driver once the pool has grown).  2D and 3D jobs
 * run the sparse tensor-core path (sparstencil_run).  Results equal those of the same job
 * run alone.
 * --------------------------------------------------------------------------------------- */
typedef struct sparstencil_server_s* sparstencil_server_t;

typedef struct {
  sparstencil_shape shape;
  int radius;
  const float* weights;      /* host cube as for sparstencil_plan, copied at submission */
  int ndim;                  /* 2 or 3 (the server takes 2D and 3D jobs; 1D plans run through
                                sparstencil_run) */
  const int64_t* dims;       /* copied at submission */
  sparstencil_dtype dtype;
  sparstencil_boundary bc;
  int fusion_depth;          /* as for sparstencil_plan */
  int64_t timesteps;
  const float* in_host;      /* host grid, read when the job is admitted (keep it valid until
                                the job completes); page-locked memory lets the copies of
                                different jobs overlap; NULL when in_device is given */
  float* out_host;           /* host result, written before the job is reported complete;
                                NULL when out_device is given */
  double arrival_s;          /* arrival time on the server clock (sparstencil_server_clock);
                                negative: the time of submission */
  const float* in_device;    /* device grid resident across jobs (caller-owned, ready when the
                                job is submitted, unchanged until it completes): read in place,
                                no host copy; NULL when in_host is given */
  float* out_device;         /* device grid that receives the result in place (caller-owned,
                                not aliasing in_device); NULL when out_host is given */
} sparstencil_job;

typedef struct {
  int64_t job_id;
  int status;                /* sparstencil_status of the job */
  double arrival_s, admit_s, done_s;  /* server clock, seconds */
  size_t device_bytes;       /* bytes counted against the budget while it ran */
} sparstencil_job_result;

typedef struct {
  int64_t submitted, completed, failed;
  double p50_s, p99_s, mean_s, max_s;  /* latency (completion - arrival) of completed jobs */
  size_t peak_bytes;                   /* largest sum of admitted jobs' bytes */
  double gstencil_per_s;               /* completed point-steps / (last completion - first arrival) */
  size_t pool_reserved_bytes;          /* device memory the server's pool holds resident now */
  size_t pool_high_bytes;              /* the most it has held */
} sparstencil_server_summary;

/* Starts a server on the current device.  slots in 1..64. */
sparstencil_status sparstencil_server_create(size_t hbm_budget_bytes, int slots, sparstencil_server_t* out);
/* Seconds since the server started (the clock of arrival_s and the results). */
double sparstencil_server_clock(sparstencil_server_t server);
/* Queues a job (plans it on the host now); *job_id receives its id.  Exactly one of in_host
 * and in_device, and one of out_host and out_device, must be given (SPST_ERR_INVALID
 * otherwise).  A job's device bytes (counted against the budget) are the grids the server
 * allocates for it (one per host-side grid) plus the plan's workspace.  Thread-safe. */
sparstencil_status sparstencil_server_submit(sparstencil_server_t server, const sparstencil_job* job,
                                             int64_t* job_id);
/* Waits up to timeout_s for a job to finish; SPST_ERR_TIMEOUT if it has not. */
sparstencil_status sparstencil_server_wait(sparstencil_server_t server, int64_t job_id, double timeout_s,
                                           sparstencil_job_result* res);
/* Waits up to timeout_s until no job is queued or running. */
sparstencil_status sparstencil_server_drain(sparstencil_server_t server, double timeout_s);
sparstencil_status sparstencil_server_stats(sparstencil_server_t server, sparstencil_server_summary* out);
/* Finishes the queued and running jobs, then stops the server and frees its plans. */
sparstencil_status sparstencil_server_destroy(sparstencil_server_t server);
/* The admission policy replayed on the host (no device work): for n jobs with arrival
 * times, run durations and device bytes, admit_s[i] / done_s[i] receive when job i would be
 * admitted and finish (done = admit + duration), -1 for a job larger than the budget. */
sparstencil_status sparstencil_server_simulate(size_t hbm_budget_bytes, int slots, int n, const double* arrival_s,
                                               const double* duration_s, const size_t* bytes, double* admit_s,
                                               double* done_s);

/* Thread-local description of the last failure in this thread ("" if none). */
const char* sparstencil_last_error(void);

/* Library version string. */
const char* sparstencil_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPARSTENCIL_H_ */
