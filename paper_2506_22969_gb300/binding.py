"""Thin ctypes binding of the C ABI in include/sparstencil.h (argument marshalling only).

Every computation runs inside libsparstencil.so; this module converts tensors and arrays
to raw pointers and status codes to exceptions.  Device grids are torch CUDA tensors
(FP32, contiguous); streams are torch streams (default: the current stream).  Loading
fails loudly when the in-tree library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsparstencil.so")

STAR, BOX, CUSTOM = 0, 1, 2
FP16, BF16, FP16_SPLIT, BF16_SPLIT = 0, 1, 2, 3
DIRICHLET, PERIODIC = 0, 1

_DTYPES = {"fp16": FP16, "bf16": BF16, "fp16_split": FP16_SPLIT, "bf16_split": BF16_SPLIT}
_BCS = {"dirichlet": DIRICHLET, "periodic": PERIODIC}
_SHAPES = {"star": STAR, "box": BOX, "custom": CUSTOM}
_STATUS = {0: "OK", 1: "INVALID", 2: "UNSUPPORTED", 3: "NOMEM", 4: "CUDA", 5: "TIMEOUT", 6: "DEVICE_CHECK"}


class SparStencilError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sparstencil error {_STATUS.get(code, code)}: {msg}")
        self.code = code


class PlanInfo(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("radius", ctypes.c_int), ("fusion_depth", ctypes.c_int),
                ("r1", ctypes.c_int), ("r2", ctypes.c_int), ("r3", ctypes.c_int), ("kprime", ctypes.c_int),
                ("kpad", ctypes.c_int), ("zero_columns", ctypes.c_int), ("mma_terms", ctypes.c_int),
                ("tile_outputs", ctypes.c_int), ("num_tiles", ctypes.c_int64), ("planner_ms", ctypes.c_double),
                ("ghost", ctypes.c_int), ("tile_pitch", ctypes.c_int), ("tile_rows", ctypes.c_int),
                ("bank_conflicts", ctypes.c_int), ("low_accumulator", ctypes.c_int),
                ("dense_ablation", ctypes.c_int), ("pairing", ctypes.c_int), ("fp64_every", ctypes.c_int)]


class Job(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int), ("radius", ctypes.c_int), ("weights", ctypes.c_void_p),
                ("ndim", ctypes.c_int), ("dims", ctypes.c_void_p), ("dtype", ctypes.c_int), ("bc", ctypes.c_int),
                ("fusion_depth", ctypes.c_int), ("timesteps", ctypes.c_int64), ("in_host", ctypes.c_void_p),
                ("out_host", ctypes.c_void_p), ("arrival_s", ctypes.c_double), ("in_device", ctypes.c_void_p),
                ("out_device", ctypes.c_void_p)]


class JobResult(ctypes.Structure):
    _fields_ = [("job_id", ctypes.c_int64), ("status", ctypes.c_int), ("arrival_s", ctypes.c_double),
                ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double), ("device_bytes", ctypes.c_size_t)]


class ServerSummary(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("p50_s", ctypes.c_double), ("p99_s", ctypes.c_double), ("mean_s", ctypes.c_double),
                ("max_s", ctypes.c_double), ("peak_bytes", ctypes.c_size_t), ("gstencil_per_s", ctypes.c_double),
                ("pool_reserved_bytes", ctypes.c_size_t), ("pool_high_bytes", ctypes.c_size_t)]


EXPORTS = ["sparstencil_plan", "sparstencil_plan_set_layout", "sparstencil_run", "sparstencil_run_profiled", "sparstencil_run_host",
           "sparstencil_run_host_async", "sparstencil_plan_set_fp64_correction",
           "sparstencil_run_noalloc", "sparstencil_plan_destroy",
           "sparstencil_workspace_bytes", "sparstencil_bind_workspace", "sparstencil_run_batch", "sparstencil_query",
           "sparstencil_plan_tables", "sparstencil_table_kpad", "sparstencil_direct_run", "sparstencil_error_norms",
           "sparstencil_device_status", "sparstencil_set_wait_limit_ns", "sparstencil_trace",
           "sparstencil_trace_read", "sparstencil_last_error",
           "sparstencil_version", "sparstencil_server_create", "sparstencil_server_clock",
           "sparstencil_server_submit", "sparstencil_server_wait", "sparstencil_server_drain",
           "sparstencil_server_stats", "sparstencil_server_destroy", "sparstencil_server_simulate"]

_lib = None


def load():
    """Loads libsparstencil.so (raises FileNotFoundError if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FileNotFoundError(f"{LIB_PATH} is missing: run __graft_entry__.build() (or python -m "
                                "paper_2506_22969_gb300.build) first")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.sparstencil_plan.argtypes = [i32, i32, vp, i32, vp, i32, i32, i32, ctypes.POINTER(vp)]
    lib.sparstencil_run.argtypes = [vp, vp, vp, i64, vp]
    lib.sparstencil_run_host.argtypes = [vp, vp, vp, i64, vp]
    lib.sparstencil_run_host_async.argtypes = [vp, vp, vp, i64, vp]
    lib.sparstencil_run_profiled.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp]
    lib.sparstencil_run_noalloc.argtypes = [vp, vp, vp, i64, vp]
    lib.sparstencil_plan_destroy.argtypes = [vp]
    lib.sparstencil_plan_set_low_accumulator.argtypes = [vp, i32]
    lib.sparstencil_plan_set_fp64_correction.argtypes = [vp, i32]
    lib.sparstencil_plan_set_dense_ablation.argtypes = [vp, i32]
    lib.sparstencil_plan_set_layout.argtypes = [vp, i32, i32]
    lib.sparstencil_cost_model.argtypes = [vp, i32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.POINTER(ctypes.c_double)]
    lib.sparstencil_workspace_bytes.argtypes = [vp]
    lib.sparstencil_workspace_bytes.restype = ctypes.c_size_t
    lib.sparstencil_bind_workspace.argtypes = [vp, vp, ctypes.c_size_t, vp]
    lib.sparstencil_run_batch.argtypes = [vp, vp, vp, vp, i32, vp]
    lib.sparstencil_query.argtypes = [vp, ctypes.POINTER(PlanInfo)]
    lib.sparstencil_plan_tables.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp]
    lib.sparstencil_table_kpad.argtypes = [vp, i32, i32, ctypes.POINTER(i32)]
    lib.sparstencil_direct_run.argtypes = [i32, vp, i32, vp, i32, vp, vp, vp, i64, vp]
    lib.sparstencil_error_norms.argtypes = [vp, vp, i64, vp, vp]
    lib.sparstencil_device_status.argtypes = [vp]
    lib.sparstencil_set_wait_limit_ns.argtypes = [ctypes.c_uint64]
    lib.sparstencil_trace.argtypes = [i32]
    lib.sparstencil_trace_read.argtypes = [vp, i32]
    lib.sparstencil_last_error.restype = ctypes.c_char_p
    lib.sparstencil_version.restype = ctypes.c_char_p
    lib.sparstencil_server_create.argtypes = [ctypes.c_size_t, i32, ctypes.POINTER(vp)]
    lib.sparstencil_server_clock.argtypes = [vp]
    lib.sparstencil_server_clock.restype = ctypes.c_double
    lib.sparstencil_server_submit.argtypes = [vp, ctypes.POINTER(Job), ctypes.POINTER(i64)]
    lib.sparstencil_server_wait.argtypes = [vp, i64, ctypes.c_double, ctypes.POINTER(JobResult)]
    lib.sparstencil_server_drain.argtypes = [vp, ctypes.c_double]
    lib.sparstencil_server_stats.argtypes = [vp, ctypes.POINTER(ServerSummary)]
    lib.sparstencil_server_destroy.argtypes = [vp]
    lib.sparstencil_server_simulate.argtypes = [ctypes.c_size_t, i32, i32, vp, vp, vp, vp, vp]
    for name in EXPORTS:
        if name.startswith("sparstencil_") and name not in ("sparstencil_workspace_bytes", "sparstencil_last_error",
                                                            "sparstencil_version", "sparstencil_server_clock"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(code: int):
    if code != 0:
        raise SparStencilError(code, load().sparstencil_last_error().decode())


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("device grids must be contiguous float32 CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def _code(table, v):
    return table[v] if isinstance(v, str) else int(v)


class Plan:
    """A planned stencil (sparstencil_plan); destroys itself when garbage-collected."""

    def __init__(self, weights, dims, dtype="bf16", bc="periodic", fusion_depth=1, shape="box",
                 low_accumulator=None, dense=False, layout=None):
        lib = load()
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32))
        self.ndim = w.ndim
        self.radius = (w.shape[0] - 1) // 2
        self.dims = tuple(int(d) for d in dims)
        if len(self.dims) != w.ndim or any(s != w.shape[0] for s in w.shape):
            raise ValueError("weights must be a (2r+1)^ndim cube with ndim = len(dims)")
        d = np.ascontiguousarray(np.asarray(self.dims, dtype=np.int64))
        h = ctypes.c_void_p()
        _check(lib.sparstencil_plan(_code(_SHAPES, shape), self.radius, w.ctypes.data, w.ndim, d.ctypes.data,
                                    _code(_DTYPES, dtype), _code(_BCS, bc), int(fusion_depth), ctypes.byref(h)))
        self._h = h
        self._ws = None
        if low_accumulator is not None:  # None: the library's default for the dtype
            self.set_low_accumulator(bool(low_accumulator))
        if dense:
            self.set_dense_ablation(True)
        if layout is not None:  # (r1, pairing); None: the library's default or search
            self.set_layout(*layout)

    def cost_model(self, depth, tensor_flops, hbm_bytes_per_s, smem_bytes_per_s) -> float:
        """sparstencil_cost_model: the Sec. 3.3 model's seconds per time step at this depth."""
        out = ctypes.c_double()
        _check(load().sparstencil_cost_model(self._h, int(depth), float(tensor_flops), float(hbm_bytes_per_s),
                                             float(smem_bytes_per_s), ctypes.byref(out)))
        return out.value

    def set_dense_ablation(self, enable=True):
        """sparstencil_plan_set_dense_ablation: dense tcgen05 MMAs on the uncompressed A'
        (before the first run)."""
        _check(load().sparstencil_plan_set_dense_ablation(self._h, 1 if enable else 0))

    def set_layout(self, r1, pairing=-1):
        """sparstencil_plan_set_layout: 2D patch shape (r1 = 16: 16 x 8, r1 = 8: 8 x 16) and
        column pairing (0 Algorithm 1, 1 maximum matching, -1 fewer chunks), before the first run."""
        _check(load().sparstencil_plan_set_layout(self._h, int(r1), int(pairing)))

    def set_low_accumulator(self, enable=True):
        """sparstencil_plan_set_low_accumulator: split terms after A_hi B_hi go to a TMEM
        accumulator of their own (before the first run)."""
        _check(load().sparstencil_plan_set_low_accumulator(self._h, 1 if enable else 0))

    def set_fp64_correction(self, every_k: int):
        """sparstencil_plan_set_fp64_correction: every k-th time step of a run in FP64 on the
        CUDA cores (0: off)."""
        _check(load().sparstencil_plan_set_fp64_correction(self._h, int(every_k)))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.sparstencil_plan_destroy(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def info(self) -> PlanInfo:
        info = PlanInfo()
        _check(load().sparstencil_query(self._h, ctypes.byref(info)))
        return info

    def workspace_bytes(self) -> int:
        return int(load().sparstencil_workspace_bytes(self._h))

    def bind_workspace(self, tensor, stream=None):
        _check(load().sparstencil_bind_workspace(self._h, ctypes.c_void_p(tensor.data_ptr()),
                                                 tensor.numel() * tensor.element_size(), _stream_ptr(stream)))
        self._ws = tensor

    def run(self, x, out, steps: int, stream=None):
        _check(load().sparstencil_run(self._h, _dev_ptr(x), _dev_ptr(out), int(steps), _stream_ptr(stream)))
        return out

    def run_noalloc(self, x, out, steps: int, stream=None):
        """sparstencil_run_noalloc: same result as run(), no device allocation (static scratch)."""
        _check(load().sparstencil_run_noalloc(self._h, _dev_ptr(x), _dev_ptr(out), int(steps), _stream_ptr(stream)))
        return out

    def run_profiled(self, x, out, steps: int, stream=None):
        """Runs and returns (copy_in_ms, sweeps_ms, num_sweeps) from CUDA events (synchronises)."""
        cin, sw, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        _check(load().sparstencil_run_profiled(self._h, _dev_ptr(x), _dev_ptr(out), int(steps), _stream_ptr(stream),
                                               ctypes.byref(cin), ctypes.byref(sw), ctypes.byref(n)))
        return cin.value, sw.value, n.value

    def run_host(self, x_host, out_host, steps: int, stream=None):
        """Host FP32 grids (numpy arrays or CPU tensors, ideally pinned)."""
        _check(load().sparstencil_run_host(self._h, ctypes.c_void_p(_host_ptr(x_host)),
                                           ctypes.c_void_p(_host_ptr(out_host)), int(steps), _stream_ptr(stream)))
        return out_host

    def run_host_async(self, x_host, out_host, steps: int, stream=None):
        """Queues a host-buffer run on `stream` without waiting (sparstencil_run_host_async):
        keep both buffers alive and out_host unread until the stream has passed it."""
        _check(load().sparstencil_run_host_async(self._h, ctypes.c_void_p(_host_ptr(x_host)),
                                                 ctypes.c_void_p(_host_ptr(out_host)), int(steps),
                                                 _stream_ptr(stream)))
        return out_host

    def tables(self, which: int = 0, remainder_depth: int = 0):
        """Planner tables (host only): order, a_hi, a_lo, a_idx, lut, fused weights."""
        lib = load()
        kp = ctypes.c_int()
        _check(lib.sparstencil_table_kpad(self._h, which, remainder_depth, ctypes.byref(kp)))
        kpad = kp.value
        info = self.info()
        t = info.fusion_depth if which == 0 else remainder_depth
        side = 2 * t * self.radius + 1
        order = np.zeros(kpad, np.int32)
        a_hi = np.zeros((128, kpad // 2), np.float32)
        a_lo = np.zeros((128, kpad // 2), np.float32)
        a_idx = np.zeros((128, kpad // 2), np.uint8)
        lut = np.zeros(kpad, np.int32)
        fw = np.zeros((side,) * self.ndim, np.float64)
        _check(lib.sparstencil_plan_tables(self._h, which, remainder_depth, order.ctypes.data, a_hi.ctypes.data,
                                           a_lo.ctypes.data, a_idx.ctypes.data, lut.ctypes.data, fw.ctypes.data))
        return dict(order=order, a_hi=a_hi, a_lo=a_lo, a_idx=a_idx, lut=lut, fused_w=fw, kpad=kpad)


def _host_ptr(a):
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != torch.float32 or not a.is_contiguous():
                raise TypeError("host grids must be contiguous float32 CPU tensors")
            return a.data_ptr()
    except ImportError:  # pragma: no cover
        pass
    if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]):
        raise TypeError("host grids must be contiguous float32 arrays")
    return a.ctypes.data


def direct_run(weights, x, out, work, steps: int, bc="periodic", stream=None):
    """Plain FP32 CUDA-core stencil (sparstencil_direct_run)."""
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32))
    d = np.ascontiguousarray(np.asarray(tuple(x.shape), dtype=np.int64))
    _check(load().sparstencil_direct_run((w.shape[0] - 1) // 2, w.ctypes.data, w.ndim, d.ctypes.data, _code(_BCS, bc),
                                         _dev_ptr(x), _dev_ptr(out), _dev_ptr(work), int(steps), _stream_ptr(stream)))
    return out


def error_norms(x, ref, stream=None):
    """(rel_l2, rel_linf, raw[4]) of device grid x against device grid ref, in FP64 on the GPU."""
    raw = np.zeros(4, np.float64)
    _check(load().sparstencil_error_norms(_dev_ptr(x), _dev_ptr(ref), x.numel(), raw.ctypes.data,
                                          _stream_ptr(stream)))
    l2 = float(np.sqrt(raw[0]) / max(np.sqrt(raw[1]), 1e-300))
    linf = float(raw[2] / max(raw[3], 1e-300))
    return l2, linf, raw


def device_status(stream=None) -> int:
    """Reads and clears the device status word (0 = OK, 5 = a bounded wait timed out)."""
    return int(load().sparstencil_device_status(_stream_ptr(stream)))


def set_wait_limit_ns(ns: int):
    _check(load().sparstencil_set_wait_limit_ns(int(ns)))


def trace(enable: bool):
    """Enables/disables the sweep kernel's CTA-0 timeline trace (clears it)."""
    _check(load().sparstencil_trace(1 if enable else 0))


def trace_read():
    """(tiles, chunks, publish): tiles = int64 [role(TMA, MMA, gather, epilogue)][tile<64][start,
    end] in ns; chunks = int64 [source(first gather warp, last gather warp, MMA issuer)][chunk<16][4]
    and publish = int64 [publish, stores done][gather warp][chunk<16] in clock cycles."""
    out = np.zeros(4 * 64 * 2 + 3 * 16 * 4 + 2 * 16 * 16, np.uint64)
    _check(load().sparstencil_trace_read(out.ctypes.data, out.size))
    tiles = out[:512].reshape(4, 64, 2).astype(np.int64)
    chunks = out[512:512 + 192].reshape(3, 16, 4).astype(np.int64)
    return tiles, chunks, out[512 + 192:].reshape(2, 16, 16).astype(np.int64)


def run_batch(plans, xs, outs, steps, stream=None):
    n = len(plans)
    hp = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    ip = (ctypes.c_void_p * n)(*[_dev_ptr(x).value for x in xs])
    op = (ctypes.c_void_p * n)(*[_dev_ptr(o).value for o in outs])
    st = (ctypes.c_int64 * n)(*[int(s) for s in steps])
    _check(load().sparstencil_run_batch(hp, ip, op, st, n, _stream_ptr(stream)))


class Server:
    """Stencil-job server (sparstencil_server_*): jobs are admitted in arrival order under an
    HBM budget onto `slots` CUDA streams and run side by side."""

    def __init__(self, hbm_budget_bytes: int, slots: int = 8):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.sparstencil_server_create(int(hbm_budget_bytes), int(slots), ctypes.byref(h)))
        self.handle = h
        self._keep = {}  # job id -> host arrays the server reads or writes

    def clock(self) -> float:
        return load().sparstencil_server_clock(self.handle)

    def submit(self, weights, grid_in, grid_out, steps, dtype="bf16", bc="periodic", fusion_depth=1,
               shape="box", arrival_s=-1.0) -> int:
        """grid_in / grid_out: contiguous float32 numpy arrays or CPU torch tensors (host grids,
        copied by the server; page-locked memory lets jobs' copies overlap), or CUDA float32
        tensors (device grids resident across jobs, read and written in place: the input must
        be ready when the job is submitted).  The server keeps references until the job is
        waited."""
        w = np.ascontiguousarray(weights, dtype=np.float32)
        ndim = w.ndim
        shp = tuple(grid_in.shape)
        if len(shp) != ndim or tuple(grid_out.shape) != shp:
            raise ValueError("grid rank or shape mismatch")
        d = np.asarray(shp, dtype=np.int64)
        in_h, in_d = _grid_ptrs(grid_in)
        out_h, out_d = _grid_ptrs(grid_out)
        job = Job(_code(_SHAPES, shape), (w.shape[0] - 1) // 2, w.ctypes.data, ndim, d.ctypes.data,
                  _code(_DTYPES, dtype), _code(_BCS, bc), int(fusion_depth), int(steps),
                  in_h, out_h, float(arrival_s), in_d, out_d)
        jid = ctypes.c_int64()
        _check(load().sparstencil_server_submit(self.handle, ctypes.byref(job), ctypes.byref(jid)))
        self._keep[jid.value] = (grid_in, grid_out)
        return jid.value

    def wait(self, job_id: int, timeout_s: float = 600.0) -> JobResult:
        r = JobResult()
        _check(load().sparstencil_server_wait(self.handle, int(job_id), float(timeout_s), ctypes.byref(r)))
        self._keep.pop(job_id, None)
        return r

    def drain(self, timeout_s: float = 600.0):
        _check(load().sparstencil_server_drain(self.handle, float(timeout_s)))

    def stats(self) -> ServerSummary:
        s = ServerSummary()
        _check(load().sparstencil_server_stats(self.handle, ctypes.byref(s)))
        return s

    def close(self):
        if self.handle:
            _check(load().sparstencil_server_destroy(self.handle))
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _grid_ptrs(a):
    """(host pointer, device pointer) of a serving job's grid, one of them None."""
    try:
        import torch
        if isinstance(a, torch.Tensor) and a.is_cuda:
            if a.dtype != torch.float32 or not a.is_contiguous():
                raise TypeError("device grids must be contiguous float32 CUDA tensors")
            return None, a.data_ptr()
    except ImportError:  # pragma: no cover
        pass
    return _host_ptr(a), None


def server_simulate(budget: int, slots: int, arrival_s, duration_s, nbytes):
    """The server's admission policy replayed on the host: (admit_s, done_s) per job."""
    a = np.ascontiguousarray(arrival_s, dtype=np.float64)
    d = np.ascontiguousarray(duration_s, dtype=np.float64)
    b = np.ascontiguousarray(nbytes, dtype=np.uint64)
    n = a.size
    adm = np.zeros(n)
    done = np.zeros(n)
    _check(load().sparstencil_server_simulate(int(budget), int(slots), n, a.ctypes.data, d.ctypes.data, b.ctypes.data,
                                              adm.ctypes.data, done.ctypes.data))
    return adm, done
