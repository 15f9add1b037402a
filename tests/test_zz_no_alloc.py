"""The allocation-free entry point, sparstencil_run_noalloc, through the C ABI.

It serves callers that cannot call cudaMalloc (services that forbid device allocation
once running, processes whose device memory belongs to a framework allocator with a fixed
budget): the ping-pong grids and tables live in static device arrays of the library.  It
runs the same kernels on the same planner tables as sparstencil_run, so its output must
equal sparstencil_run's bit for bit, on consecutive calls that share those arrays (the
second with another input of smaller magnitude, so that a stale data-scale word or stale
scratch from the first call would change the result).  A call on a fresh plan must not
change the device's free memory.  This file is collected last so a stop-at-first-failure
run has already run every other test.
"""
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


CASES = [
    # (shape, r, recipe, dims, steps, bc, dtype, t): a periodic fused run with a remainder
    # sweep; a Dirichlet run on another geometry (stale ghost cells must not leak); a fused
    # Dirichlet run with a remainder sweep (the band kernel writes the frame of each sweep)
    ("box", 1, "random", (300, 260), 10, "periodic", "bf16_split", 3),
    ("star", 1, "heat", (512, 512), 8, "dirichlet", "fp16", 1),
    ("box", 1, "random", (300, 260), 10, "dirichlet", "bf16_split", 3),
    ("star", 1, "heat", (200, 296), 9, "dirichlet", "fp16", 4),
]


@pytest.mark.parametrize("shape,r,recipe,dims,steps,bc,dtype,t", CASES)
def test_noalloc_equals_run_on_consecutive_calls(torch_cuda, shape, r, recipe, dims, steps, bc, dtype, t):
    torch = torch_cuda
    w = inputs.stencil_weights(shape, 2, r, recipe, seed=11)
    plan = binding.Plan(w, dims, dtype=dtype, bc=bc, fusion_depth=t, shape=shape)
    grids = [inputs.uniform01(5, dims), (0.25 * inputs.uniform_pm1(6, dims)).astype(np.float32)]
    for u in grids:  # two calls in a row on the shared static arrays
        x = torch.from_numpy(u).cuda()
        ref = torch.empty_like(x)
        plan.run(x, ref, steps)
        got = torch.full_like(x, float("nan"))
        plan.run_noalloc(x, got, steps)
        torch.cuda.synchronize()
        assert binding.device_status() == 0
        assert torch.equal(got, ref)


def test_noalloc_allocates_no_device_memory(torch_cuda):
    """A run through the allocation-free entry point on a plan that has never run (no
    workspace, no device tables) leaves the device's free memory unchanged.  A first call
    on another plan of the same kind runs beforehand, so that loading the library's kernels
    and static arrays onto the device is not counted."""
    torch = torch_cuda
    dims, steps = (300, 260), 10
    w = inputs.stencil_weights("box", 2, 1, "random", seed=3)
    x = torch.from_numpy(inputs.uniform01(7, dims)).cuda()
    y = torch.empty_like(x)
    warm = binding.Plan(w, dims, dtype="bf16_split", bc="dirichlet", fusion_depth=3)
    warm.run_noalloc(x, y, steps)
    torch.cuda.synchronize()
    fresh = binding.Plan(w, dims, dtype="bf16_split", bc="dirichlet", fusion_depth=3)
    free0, _ = torch.cuda.mem_get_info()
    fresh.run_noalloc(x, y, steps)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert binding.device_status() == 0
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_grids_beyond_the_static_limit(torch_cuda):
    torch = torch_cuda
    w = inputs.stencil_weights("box", 2, 1, "random", seed=2)
    plan = binding.Plan(w, (4096, 4096), dtype="bf16", bc="periodic")
    x = torch.zeros((4096, 4096), dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(binding.SparStencilError) as e:
        plan.run_noalloc(x, y, 1)
    assert e.value.code == 2 and "allocation-free" in str(e.value)
