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
