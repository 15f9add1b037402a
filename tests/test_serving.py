"""The serving runtime on the GPU: jobs of different stencils, sizes, precisions, step
counts and ranks submitted while others run give exactly the results they give alone, and
the HBM budget bounds the bytes of the jobs running at any time."""
import numpy as np
import pytest

from paper_2506_22969_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_22969_gb300 import build
    build.build()
    binding.load()
    return torch


JOBS = [  # (shape, r, recipe, dims, steps, bc, dtype, t)
    ("box", 1, "random", (384, 256), 30, "periodic", "bf16_split", 3),
    ("star", 3, "gaussian", (256, 512), 12, "periodic", "bf16", 1),
    ("box", 3, "gaussian", (300, 260), 9, "periodic", "bf16_split", 1),
    ("star", 1, "heat", (512, 512), 8, "dirichlet", "fp16", 1),
    ("box", 1, "random", (200, 328), 17, "dirichlet", "bf16_split", 2),
    ("star", 1, "heat", (40, 48, 56), 6, "dirichlet", "fp16_split", 1),
    ("box", 1, "random", (32, 40, 24), 5, "periodic", "fp16", 1),
    ("box", 2, "random", (256, 256), 21, "periodic", "bf16", 3),
]


def _alone(torch, w, u, shape, dims, T, bc, dtype, t):
    x = torch.from_numpy(u).cuda()
    y = torch.empty_like(x)
    plan = binding.Plan(w, dims, dtype=dtype, bc=bc, fusion_depth=t, shape=shape)
    plan.run(x, y, T)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def _make(k, job):
    shape, r, recipe, dims, T, bc, dtype, t = job
    w = inputs.stencil_weights(shape, len(dims), r, recipe, seed=40 + k)
    u = inputs.uniform01(50 + k, dims)
    return w, u


def test_results_in_the_mix_equal_alone(torch_cuda):
    torch = torch_cuda
    srv = binding.Server(hbm_budget_bytes=8 << 30, slots=4)
    outs, ids = [], []
    for rep in range(2):  # every job twice, so plans are reused by later jobs
        for k, job in enumerate(JOBS):
            shape, r, recipe, dims, T, bc, dtype, t = job
            w, u = _make(k, job)
            hin = torch.from_numpy(u).pin_memory()
            hout = torch.full(dims, float("nan")).pin_memory()
            ids.append(srv.submit(w, hin, hout, T, dtype=dtype, bc=bc, fusion_depth=t, shape=shape))
            outs.append((k, hout))
    srv.drain()
    for jid in ids:
        assert srv.wait(jid).status == 0
    st = srv.stats()
    assert st.completed == len(ids) and st.failed == 0 and st.p99_s >= st.p50_s > 0
    alone = {}
    for k, hout in outs:
        if k not in alone:
            shape, r, recipe, dims, T, bc, dtype, t = JOBS[k]
            w, u = _make(k, JOBS[k])
            alone[k] = _alone(torch, w, u, shape, dims, T, bc, dtype, t)
        np.testing.assert_array_equal(hout.numpy(), alone[k])
    srv.close()
    assert binding.device_status() == 0


def test_budget_bounds_running_bytes(torch_cuda):
    torch = torch_cuda
    w = inputs.stencil_weights("box", 2, 1, "random", seed=3)
    dims = (1024, 1024)
    u = inputs.uniform01(7, dims)
    probe = binding.Plan(w, dims, dtype="bf16", bc="periodic", fusion_depth=3)
    job_bytes = 2 * 1024 * 1024 * 4 + probe.workspace_bytes()
    budget = int(2.5 * job_bytes)  # room for two jobs at a time
    srv = binding.Server(hbm_budget_bytes=budget, slots=8)
    hin = torch.from_numpy(u).pin_memory()
    outs = [torch.empty(dims).pin_memory() for _ in range(6)]
    ids = [srv.submit(w, hin, o, 60, dtype="bf16", bc="periodic", fusion_depth=3) for o in outs]
    # a job that can never fit fails without blocking the others
    big = np.zeros((4096, 4096), np.float32)
    big_out = np.zeros_like(big)
    bad = srv.submit(w, big, big_out, 1, dtype="bf16", bc="periodic", fusion_depth=3)
    srv.drain()
    res = [srv.wait(j) for j in ids]
    assert srv.wait(bad).status == 3
    assert all(r.status == 0 and r.device_bytes == job_bytes for r in res)
    for r in res:  # at most two jobs overlap
        overlap = sum(1 for q in res if q.admit_s <= r.admit_s < q.done_s)
        assert overlap <= 2
    assert srv.stats().peak_bytes <= budget
    for o in outs[1:]:
        assert np.array_equal(o.numpy(), outs[0].numpy())
    srv.close()


def test_device_resident_grids(torch_cuda):
    """Jobs whose grids stay on the device (CUDA tensors, read and written in place) mixed
    with host-grid jobs: each result equals the job run alone; a run continued from a
    resident output by a second job equals one run of the summed steps (BF16 operands,
    fused depth dividing both step counts, so the two sequences of sweeps are the same); the
    server counts only the grids it allocates against the budget, and its memory pool keeps
    the freed memory resident."""
    torch = torch_cuda
    srv = binding.Server(hbm_budget_bytes=8 << 30, slots=4)
    resident, host_jobs = [], []
    for k, job in enumerate(JOBS):
        shape, r, recipe, dims, T, bc, dtype, t = job
        w, u = _make(k, job)
        x = torch.from_numpy(u).cuda()
        y = torch.full_like(x, float("nan"))
        torch.cuda.synchronize()  # the input is ready before the job is submitted
        resident.append((k, srv.submit(w, x, y, T, dtype=dtype, bc=bc, fusion_depth=t, shape=shape), x, y))
        hin = torch.from_numpy(u).pin_memory()
        hout = torch.full(dims, float("nan")).pin_memory()
        host_jobs.append((k, srv.submit(w, hin, hout, T, dtype=dtype, bc=bc, fusion_depth=t, shape=shape), hout))
    srv.drain()
    for k, jid, x, y in resident:
        res = srv.wait(jid)
        assert res.status == 0
        shape, r, recipe, dims, T, bc, dtype, t = JOBS[k]
        plan = binding.Plan(inputs.stencil_weights(shape, len(dims), r, recipe, seed=40 + k), dims, dtype=dtype,
                            bc=bc, fusion_depth=t, shape=shape)
        assert res.device_bytes == plan.workspace_bytes()  # the caller's grids are not counted
        w, u = _make(k, JOBS[k])
        np.testing.assert_array_equal(y.cpu().numpy(), _alone(torch, w, u, shape, dims, T, bc, dtype, t))
    for k, jid, hout in host_jobs:
        assert srv.wait(jid).status == 0
        np.testing.assert_array_equal(hout.numpy(), resident[k][3].cpu().numpy())
    # a grid advanced by two jobs in place on the device
    w = inputs.stencil_weights("box", 2, 1, "random", seed=9)
    u = inputs.uniform01(11, (384, 256))
    a = torch.from_numpy(u).cuda()
    b, c = torch.empty_like(a), torch.empty_like(a)
    torch.cuda.synchronize()
    assert srv.wait(srv.submit(w, a, b, 6, dtype="bf16", fusion_depth=3)).status == 0
    assert srv.wait(srv.submit(w, b, c, 9, dtype="bf16", fusion_depth=3)).status == 0
    np.testing.assert_array_equal(c.cpu().numpy(), _alone(torch, w, u, "box", (384, 256), 15, "periodic", "bf16", 3))
    st = srv.stats()
    assert st.failed == 0 and st.pool_high_bytes > 0 and st.pool_reserved_bytes > 0
    srv.close()
    assert binding.device_status() == 0


def test_job_grid_arguments_are_checked(torch_cuda):
    """A job must give exactly one of the host and device input (and output) grids, and its
    device grids must not alias."""
    import ctypes
    torch = torch_cuda
    srv = binding.Server(hbm_budget_bytes=1 << 30, slots=2)
    lib = binding.load()
    w = inputs.stencil_weights("box", 2, 1, "random", seed=1)
    d = np.asarray((64, 64), np.int64)
    x = torch.zeros(64, 64, device="cuda")
    h = np.zeros((64, 64), np.float32)
    base = dict(shape=binding.BOX, radius=1, weights=w.ctypes.data, ndim=2, dims=d.ctypes.data, dtype=binding.BF16,
                bc=binding.PERIODIC, fusion_depth=1, timesteps=1, arrival_s=-1.0)
    for ins, outs in [((h.ctypes.data, x.data_ptr()), (h.ctypes.data, None)),  # both inputs
                      ((None, None), (h.ctypes.data, None)),                   # no input
                      ((None, x.data_ptr()), (None, x.data_ptr()))]:            # aliasing device grids
        job = binding.Job(**base, in_host=ins[0], in_device=ins[1], out_host=outs[0], out_device=outs[1])
        jid = ctypes.c_int64()
        assert lib.sparstencil_server_submit(srv.handle, ctypes.byref(job), ctypes.byref(jid)) == 1  # SPST_ERR_INVALID
    srv.close()
