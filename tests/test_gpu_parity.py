"""GPU parity: the sparse tensor-core path (through the C ABI) against the FP64 oracle.

Tolerances (FP64, after the full run): rel-L2 over the whole grid <= 2e-3 for single-word
operands (FP16/BF16) and 1e-5 for split hi+lo operands; rel-Linf = max|x - ref| / max|ref|
<= ten times that (2e-2 / 1e-4), so that a handful of wrong outputs fails even where it
barely moves rel-L2; the plain FP32 CUDA-core comparator 1e-6 (rel-L2) and 1e-5 (rel-Linf).
Sampled full-size cases apply the same bounds to the sampled points.
"""
import numpy as np
import pytest

from paper_2506_22969_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp16": 2e-3, "bf16": 2e-3, "fp16_split": 1e-5, "bf16_split": 1e-5}
LINF = {k: 10 * v for k, v in TOL.items()}


def _rel(vals, ref):
    """(rel-L2, rel-Linf) of sampled or whole-grid values against the oracle's."""
    vals = np.asarray(vals, np.float64)
    ref = np.asarray(ref, np.float64)
    d = vals - ref
    return (float(np.sqrt(np.sum(d * d) / np.sum(ref * ref))), float(np.max(np.abs(d)) / np.max(np.abs(ref))))


def _assert_tol(l2, linf, dtype, *ctx):
    assert l2 <= TOL[dtype], (dtype, l2, linf) + ctx
    assert linf <= LINF[dtype], (dtype, l2, linf) + ctx


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_22969_gb300 import build
    build.build()
    binding.load()
    return torch


def _run_sparse(torch, u, w, steps, dtype, bc, t, shape, low_accumulator=None, dense=False):
    plan = binding.Plan(w, u.shape, dtype=dtype, bc=bc, fusion_depth=t, shape=shape,
                        low_accumulator=low_accumulator, dense=dense)
    x = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32)).cuda()
    y = torch.empty_like(x)
    plan.run(x, y, steps)
    assert binding.device_status() == 0
    return y.cpu().numpy().astype(np.float64), plan


CASES = [
    # (shape, r, recipe, dims, steps, bc, dtype, t)
    ("star", 1, "heat", (512, 512), 8, "dirichlet", "fp16", 1),
    ("star", 1, "heat", (512, 512), 8, "dirichlet", "bf16_split", 1),
    ("box", 1, "random", (300, 260), 20, "periodic", "bf16", 1),
    ("box", 1, "random", (300, 260), 20, "periodic", "bf16_split", 1),
    ("box", 1, "random", (256, 384), 10, "periodic", "fp16_split", 1),
    ("box", 1, "random", (130, 200), 7, "dirichlet", "bf16", 1),
    ("box", 1, "random", (384, 320), 10, "periodic", "bf16_split", 3),
    ("box", 1, "random", (256, 256), 11, "periodic", "bf16", 2),
    ("star", 3, "gaussian", (260, 300), 6, "periodic", "bf16_split", 1),
    ("box", 3, "gaussian", (260, 300), 6, "periodic", "bf16", 1),
    ("box", 3, "gaussian", (200, 256), 5, "dirichlet", "fp16_split", 1),
    ("box", 2, "random", (128, 128), 4, "periodic", "bf16_split", 1),
    # Dirichlet with temporal fusion: the fused kernel plus the exact band of width (t-1)r
    ("star", 1, "heat", (512, 512), 8, "dirichlet", "fp16", 3),
    ("star", 1, "heat", (512, 512), 8, "dirichlet", "bf16_split", 3),
    ("box", 1, "random", (130, 200), 10, "dirichlet", "bf16_split", 4),
    ("box", 2, "gaussian", (300, 260), 7, "dirichlet", "bf16_split", 2),
    ("star", 3, "gaussian", (260, 300), 9, "dirichlet", "bf16", 2),
    ("box", 3, "gaussian", (260, 300), 8, "periodic", "bf16_split", 2),
    # deep fusion (the 2D search goes to t = 6 where the tables fit TMEM)
    ("box", 1, "random", (300, 260), 13, "periodic", "bf16_split", 6),
    ("box", 1, "random", (300, 260), 13, "periodic", "bf16", 6),
    ("box", 1, "random", (256, 384), 10, "periodic", "fp16_split", 5),
    ("box", 1, "random", (256, 384), 9, "periodic", "fp16", 4),
    ("star", 1, "heat", (512, 512), 8, "dirichlet", "fp16", 6),
    ("star", 1, "heat", (200, 296), 9, "dirichlet", "bf16_split", 4),
    ("box", 2, "random", (260, 300), 7, "periodic", "bf16_split", 3),
]


@pytest.mark.parametrize("shape,r,recipe,dims,steps,bc,dtype,t", CASES)
def test_sparse_matches_oracle(torch_cuda, oracle_mod, shape, r, recipe, dims, steps, bc, dtype, t):
    w = inputs.stencil_weights(shape, 2, r, recipe, seed=11)
    u = inputs.uniform01(5, dims)
    ref = oracle_mod.run(u, w, bc, steps)
    got, _ = _run_sparse(torch_cuda, u, w, steps, dtype, bc, t, shape)
    l2, linf = oracle_mod.rel_errors(got, ref)
    assert np.all(np.isfinite(got))
    _assert_tol(l2, linf, dtype)
    if bc == "dirichlet" and t > 1:
        # the frame the fused kernel cannot produce must meet the tolerance on its own
        bw = (t - 1) * r
        band = np.ones(dims, dtype=bool)
        band[bw:-bw, bw:-bw] = False
        _assert_tol(*_rel(got[band], ref[band]), dtype, "band")


@pytest.mark.parametrize("shape,r,recipe,dims,steps,bc,dtype,t", [
    ("box", 1, "random", (300, 260), 20, "periodic", "bf16_split", 1),
    ("box", 1, "random", (300, 260), 13, "periodic", "bf16_split", 6),
    ("star", 1, "heat", (512, 512), 8, "dirichlet", "fp16", 3),
    ("box", 3, "gaussian", (260, 300), 8, "periodic", "bf16", 2),
    ("star", 3, "gaussian", (200, 256), 5, "dirichlet", "fp16_split", 1),
    ("box", 2, "random", (130, 200), 7, "dirichlet", "bf16_split", 2),
])
def test_tall_patch_layout_matches_oracle(torch_cuda, oracle_mod, shape, r, recipe, dims, steps, bc, dtype, t):
    """8 x 16 patches (sparstencil_plan_set_layout r1 = 8): the gather's patch map, the
    epilogue's output map, the periodic ghost images and the Dirichlet band all follow it."""
    torch = torch_cuda
    w = inputs.stencil_weights(shape, 2, r, recipe, seed=11)
    u = inputs.uniform01(5, dims)
    ref = oracle_mod.run(u, w, bc, steps)
    plan = binding.Plan(w, dims, dtype=dtype, bc=bc, fusion_depth=t, shape=shape, layout=(8, -1))
    assert plan.info().r1 == 8 and plan.info().r2 == 16
    x = torch.from_numpy(u).cuda()
    y = torch.full_like(x, float("nan"))
    plan.run(x, y, steps)
    assert binding.device_status() == 0
    got = y.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got))
    _assert_tol(*oracle_mod.rel_errors(got, ref), dtype)


def test_layout_search_matches_oracle(torch_cuda, oracle_mod):
    """fusion_depth 0 searches depth x patch shape (x pairing for a star): the chosen layout is
    reported and the run meets the tolerance; a second run repeats it bit for bit."""
    torch = torch_cuda
    for shape, r, recipe in (("box", 1, "random"), ("star", 3, "gaussian")):
        w = inputs.stencil_weights(shape, 2, r, recipe, seed=4)
        u = inputs.uniform01(9, (520, 390))
        plan = binding.Plan(w, u.shape, dtype="bf16_split", bc="periodic", fusion_depth=0, shape=shape)
        x = torch.from_numpy(u).cuda()
        y1, y2 = torch.empty_like(x), torch.empty_like(x)
        plan.run(x, y1, 12)
        info = plan.info()
        assert info.r1 in (16, 8) and info.r1 * info.r2 == 128 and info.pairing in (0, 1)
        plan.run(x, y2, 12)
        assert binding.device_status() == 0
        assert torch.equal(y1, y2)
        ref = oracle_mod.run(u, w, "periodic", 12)
        _assert_tol(*oracle_mod.rel_errors(y1.cpu().numpy().astype(np.float64), ref), "bf16_split", shape)


def test_zero_and_one_step(torch_cuda, oracle_mod):
    w = inputs.stencil_weights("box", 2, 1, "random", seed=3)
    u = inputs.uniform01(6, (200, 136))
    got0, _ = _run_sparse(torch_cuda, u, w, 0, "bf16", "periodic", 1, "box")
    np.testing.assert_array_equal(got0, u.astype(np.float64))
    got1, _ = _run_sparse(torch_cuda, u, w, 1, "bf16_split", "periodic", 1, "box")
    _assert_tol(*oracle_mod.rel_errors(got1, oracle_mod.run(u, w, "periodic", 1)), "bf16_split")


def test_autotuned_depth_matches_oracle(torch_cuda, oracle_mod):
    """fusion_depth 0: the first run picks a depth by timing; results meet the split
    tolerance and a second run with the chosen depth repeats the first bit for bit."""
    torch = torch_cuda
    w = inputs.stencil_weights("box", 2, 1, "random", seed=4)
    u = inputs.uniform01(9, (300, 260))
    plan = binding.Plan(w, u.shape, dtype="bf16_split", bc="periodic", fusion_depth=0)
    x = torch.from_numpy(u).cuda()
    y1 = torch.empty_like(x)
    y2 = torch.empty_like(x)
    plan.run(x, y1, 20)
    t = plan.info().fusion_depth
    assert 1 <= t <= 6
    plan.run(x, y2, 20)
    assert binding.device_status() == 0
    assert torch.equal(y1, y2)
    ref = oracle_mod.run(u, w, "periodic", 20)
    _assert_tol(*oracle_mod.rel_errors(y1.cpu().numpy().astype(np.float64), ref), "bf16_split")


def test_closed_form_fourier_mode(torch_cuda):
    """Periodic closed form, no oracle: u0 = 1/2 + 1/2 cos(theta.x) evolves to
    1/2 S^T + 1/2 Re(lambda^T e^{i theta.x}), S = sum w, lambda = sum_o w[o] e^{i theta.o};
    100 steps on the split path."""
    H, W = 256, 384
    w = inputs.stencil_weights("box", 2, 1, "random", seed=8)
    w64 = w.astype(np.float64)
    th = np.array([2 * np.pi * 3 / H, 2 * np.pi * 5 / W])
    y, x = np.mgrid[0:H, 0:W]
    phase = th[0] * y + th[1] * x
    lam = sum(w64[a + 1, b + 1] * np.exp(1j * (th[0] * a + th[1] * b)) for a in (-1, 0, 1) for b in (-1, 0, 1))
    S = float(np.sum(w64))
    T = 100
    u0 = 0.5 + 0.5 * np.cos(phase)
    ref = 0.5 * S ** T + 0.5 * np.real(lam ** T * np.exp(1j * phase))
    got, _ = _run_sparse(torch_cuda, u0, w, T, "bf16_split", "periodic", 1, "box")
    _assert_tol(*_rel(got, ref), "bf16_split")


def test_closed_form_sine_mode_dirichlet_fused(torch_cuda):
    """Dirichlet closed form, no oracle: for the Heat-2D star the zero-boundary sine mode
    u0 = sin(pi p (y+1)/(H+1)) sin(pi q (x+1)/(W+1)) is an eigenvector with eigenvalue
    lambda = 1/2 + 1/4 cos(pi p/(H+1)) + 1/4 cos(pi q/(W+1)); 100 steps fused 3 at a time
    (the band path supplies the frame the fused kernel cannot)."""
    H, W, pm, qm, T = 250, 300, 2, 3, 100
    w = inputs.stencil_weights("star", 2, 1, "heat", seed=0)
    y, x = np.mgrid[0:H, 0:W]
    u0 = np.sin(np.pi * pm * (y + 1) / (H + 1)) * np.sin(np.pi * qm * (x + 1) / (W + 1))
    lam = 0.5 + 0.25 * np.cos(np.pi * pm / (H + 1)) + 0.25 * np.cos(np.pi * qm / (W + 1))
    u32 = u0.astype(np.float32)
    ref = lam ** T * u32.astype(np.float64)
    got, _ = _run_sparse(torch_cuda, u32, w, T, "bf16_split", "dirichlet", 3, "star")
    _assert_tol(*_rel(got, ref), "bf16_split")


def test_direct_fp32_matches_oracle(torch_cuda, oracle_mod):
    torch = torch_cuda
    for shape, r, recipe, bc in [("box", 1, "random", "periodic"), ("star", 3, "gaussian", "dirichlet"),
                                 ("box", 3, "gaussian", "periodic")]:
        w = inputs.stencil_weights(shape, 2, r, recipe, seed=4)
        u = inputs.uniform01(7, (130, 200))
        x = torch.from_numpy(u).cuda()
        out = torch.empty_like(x)
        work = torch.empty_like(x)
        binding.direct_run(w, x, out, work, 9, bc=bc)
        ref = oracle_mod.run(u, w, bc, 9)
        l2, linf = oracle_mod.rel_errors(out.cpu().numpy(), ref)
        assert l2 <= 1e-6 and linf <= 1e-5, (shape, r, bc, l2, linf)


@pytest.mark.parametrize("dims,r,bc", [
    ((20, 64), 4, "periodic"),     # fewer rows than a warp's segment: every row wraps once at most
    ((70, 132), 3, "dirichlet"),   # width not a multiple of 128: a partly idle warp
    ((130, 516), 1, "periodic"),   # several warps across, ragged last segment
    ((96, 260), 2, "dirichlet"),
])
def test_direct_fp32_ragged(torch_cuda, oracle_mod, dims, r, bc):
    """The register-marching FP32 comparator on ragged 2D grids (widths a multiple of 4)."""
    torch = torch_cuda
    w = inputs.stencil_weights("box", 2, r, "random", seed=9)
    u = inputs.uniform01(3, dims)
    x = torch.from_numpy(u).cuda()
    out, work = torch.empty_like(x), torch.empty_like(x)
    binding.direct_run(w, x, out, work, 5, bc=bc)
    l2, linf = oracle_mod.rel_errors(out.cpu().numpy(), oracle_mod.run(u, w, bc, 5))
    assert l2 <= 1e-6 and linf <= 1e-5, (l2, linf)


@pytest.mark.parametrize("shape,dims,bc", [("box", (5, 12, 132), "periodic"), ("box", (37, 9, 260), "dirichlet"),
                                           ("box", (33, 20, 36), "periodic"), ("star", (37, 10, 260), "periodic"),
                                           ("star", (9, 13, 36), "dirichlet")])
def test_direct_fp32_3d_ragged(torch_cuda, oracle_mod, shape, dims, bc):
    """The 3D radius-1 comparator (box and star kernels, three rows per warp) with fewer planes
    than a warp's segment, row counts not a multiple of a warp's rows, and ragged widths."""
    torch = torch_cuda
    w = inputs.stencil_weights(shape, 3, 1, "random", seed=10)
    u = inputs.uniform_pm1(4, dims)
    x = torch.from_numpy(u).cuda()
    out, work = torch.empty_like(x), torch.empty_like(x)
    binding.direct_run(w, x, out, work, 4, bc=bc)
    l2, linf = oracle_mod.rel_errors(out.cpu().numpy(), oracle_mod.run(u, w, bc, 4))
    assert l2 <= 1e-6 and linf <= 1e-5, (l2, linf)


def test_direct_fp32_3d(torch_cuda, oracle_mod):
    torch = torch_cuda
    w = inputs.stencil_weights("box", 3, 1, "random", seed=5)
    u = inputs.uniform_pm1(3, (20, 24, 40))
    x = torch.from_numpy(u).cuda()
    out, work = torch.empty_like(x), torch.empty_like(x)
    binding.direct_run(w, x, out, work, 5, bc="dirichlet")
    ref = oracle_mod.run(u, w, "dirichlet", 5)
    l2, linf = oracle_mod.rel_errors(out.cpu().numpy(), ref)
    assert l2 <= 1e-6 and linf <= 1e-5, (l2, linf)


def test_error_norms_kernel(torch_cuda):
    torch = torch_cuda
    a = inputs.uniform01(1, (1000, 37))
    b = inputs.uniform01(2, (1000, 37))
    l2, linf, raw = binding.error_norms(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
    d = a.astype(np.float64) - b.astype(np.float64)
    assert abs(raw[0] - np.sum(d * d)) <= 1e-9 * np.sum(d * d)
    assert raw[2] == np.max(np.abs(d)) and raw[3] == np.max(np.abs(b.astype(np.float64)))


def test_run_host_equals_run(torch_cuda):
    torch = torch_cuda
    w = inputs.stencil_weights("box", 2, 1, "random", seed=3)
    u = inputs.uniform01(6, (256, 256))
    plan = binding.Plan(w, u.shape, dtype="bf16_split", bc="periodic")
    x = torch.from_numpy(u).cuda()
    y = torch.empty_like(x)
    plan.run(x, y, 12)
    host_out = torch.empty((256, 256), dtype=torch.float32).pin_memory()
    plan.run_host(torch.from_numpy(u).pin_memory(), host_out, 12)
    np.testing.assert_array_equal(host_out.numpy(), y.cpu().numpy())


def test_run_host_async_pipelined_equals_run(torch_cuda):
    """Asynchronous host-buffer runs of two plans alternating on two streams (the pipelined
    end-to-end mode): every run's result equals the device-buffer run of its input."""
    torch = torch_cuda
    w = inputs.stencil_weights("box", 2, 3, "gaussian", seed=3)
    dims = (520, 390)
    plans = [binding.Plan(w, dims, dtype="bf16_split", bc="periodic", fusion_depth=2) for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    us = [inputs.uniform01(20 + i, dims) for i in range(6)]
    hin = [torch.from_numpy(u).pin_memory() for u in us]
    hout = [torch.full(dims, float("nan")).pin_memory() for _ in us]
    for i in range(len(us)):
        plans[i % 2].run_host_async(hin[i], hout[i], 7, stream=streams[i % 2])
    torch.cuda.synchronize()
    for i, u in enumerate(us):
        x = torch.from_numpy(u).cuda()
        y = torch.empty_like(x)
        plans[0].run(x, y, 7)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(hout[i].numpy(), y.cpu().numpy())
    assert binding.device_status() == 0


def test_full_size_box9_sampled(torch_cuda, oracle_mod):
    """Box-2D9P 4096^2, periodic, 100 steps (the benchmark workload): sampled points against
    the dependence-cone oracle, both precisions, in the launch configuration the bench times."""
    cfg = inputs.CONFIGS["box2d9p_4096"]
    w = inputs.stencil_weights(cfg["shape"], 2, cfg["radius"], cfg["recipe"], seed=cfg["seed"])
    u = inputs.make_grid(cfg["grid"], cfg["seed"], cfg["dims"])
    rng = np.random.default_rng(0)
    pts = [tuple(int(v) for v in rng.integers(0, 4096, 2)) for _ in range(24)] + [(0, 0), (4095, 4095), (0, 4095)]
    ref = oracle_mod.points(u, w, "periodic", cfg["steps"], pts)
    for dtype in ("bf16", "bf16_split"):
        got, _ = _run_sparse(torch_cuda, u, w, cfg["steps"], dtype, "periodic", 1, "box")
        vals = np.array([got[p] for p in pts])
        _assert_tol(*_rel(vals, ref), dtype)


def test_bounded_wait_reports_timeout(torch_cuda):
    """A wait limit far below a tile's load time makes every CTA's first wait run out: the
    kernel drains its own copies, frees TMEM, returns, and the host reads SPST_ERR_TIMEOUT;
    the context stays usable."""
    torch = torch_cuda
    w = inputs.stencil_weights("box", 2, 1, "random", seed=3)
    u = inputs.uniform01(6, (512, 512))
    plan = binding.Plan(w, u.shape, dtype="bf16", bc="periodic")
    x = torch.from_numpy(u).cuda()
    y = torch.empty_like(x)
    binding.set_wait_limit_ns(1)
    try:
        plan.run(x, y, 2)
        assert binding.device_status() == 5
    finally:
        binding.set_wait_limit_ns(0)
    plan.run(x, y, 2)
    assert binding.device_status() == 0


def test_run_captured_in_a_cuda_graph(torch_cuda):
    """A run captured into a CUDA graph (after one plain run) replays to the same result,
    bit for bit, and leaves later plain runs unchanged."""
    torch = torch_cuda
    w = inputs.stencil_weights("star", 2, 1, "heat", seed=1)
    u = inputs.uniform01(3, (512, 512))
    plan = binding.Plan(w, u.shape, dtype="fp16", bc="dirichlet", fusion_depth=0, shape="star")
    x = torch.from_numpy(u).cuda()
    y0, y1, y2 = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
    plan.run(x, y0, 8)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.run(x, y1, 8)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    plan.run(x, y2, 8)
    torch.cuda.synchronize()
    assert binding.device_status() == 0
    assert torch.equal(y1, y0) and torch.equal(y2, y0)


def test_batch_graph_equals_individual_runs(torch_cuda):
    """sparstencil_run_batch (one CUDA graph, jobs side by side) gives each job exactly the
    result of sparstencil_run on its own: mixed sizes, stencils, precisions, boundaries and
    step counts, including a zero-step job and an autotuned plan."""
    torch = torch_cuda
    jobs = [("star", 3, "gaussian", (256, 384), 7, "periodic", "bf16", 1),
            ("box", 3, "gaussian", (384, 256), 5, "periodic", "bf16_split", 1),
            ("box", 1, "random", (200, 136), 10, "dirichlet", "bf16_split", 3),
            ("star", 1, "heat", (512, 512), 8, "dirichlet", "fp16", 1),
            ("box", 2, "random", (300, 260), 0, "periodic", "bf16", 1),
            ("box", 1, "random", (260, 300), 9, "periodic", "bf16_split", 0)]
    plans, xs, alone, outs, steps = [], [], [], [], []
    for k, (shape, r, recipe, dims, T, bc, dtype, t) in enumerate(jobs):
        w = inputs.stencil_weights(shape, 2, r, recipe, seed=20 + k)
        u = inputs.uniform01(30 + k, dims)
        x = torch.from_numpy(u).cuda()
        plan = binding.Plan(w, dims, dtype=dtype, bc=bc, fusion_depth=t, shape=shape)
        y = torch.empty_like(x)
        plan.run(x, y, T)  # alone (an autotuned plan fixes its depth here)
        plans.append(plan)
        xs.append(x)
        alone.append(y)
        outs.append(torch.full_like(x, float("nan")))
        steps.append(T)
    binding.run_batch(plans, xs, outs, steps)
    torch.cuda.synchronize()
    assert binding.device_status() == 0
    for a, b in zip(alone, outs):
        assert torch.equal(a, b)
    # the same batch again replays the kept graph; new inputs in the same buffers flow through it
    for o in outs:
        o.fill_(float("nan"))
    for k, x in enumerate(xs):
        x.copy_(torch.from_numpy(inputs.uniform01(60 + k, tuple(x.shape))).cuda())
    binding.run_batch(plans, xs, outs, steps)
    torch.cuda.synchronize()
    assert binding.device_status() == 0
    for plan, x, o, T in zip(plans, xs, outs, steps):
        y = torch.empty_like(x)
        plan.run(x, y, T)
        assert torch.equal(y, o)


CASES_3D = [
    # (shape, recipe, dims, steps, bc, dtype): 3D sparse sweep (Tile3D), ragged and full tiles
    ("box", "random", (40, 36, 72), 5, "periodic", "bf16_split"),
    ("star", "random", (34, 50, 130), 6, "dirichlet", "fp16"),
    ("box", "random", (32, 32, 128), 10, "periodic", "bf16"),
    ("star", "heat", (17, 20, 66), 7, "periodic", "bf16_split"),
]


@pytest.mark.parametrize("shape,recipe,dims,steps,bc,dtype", CASES_3D)
def test_sparse_3d_matches_oracle(torch_cuda, oracle_mod, shape, recipe, dims, steps, bc, dtype):
    w = inputs.stencil_weights(shape, 3, 1, recipe, seed=12)
    u = inputs.uniform_pm1(6, dims)
    ref = oracle_mod.run(u, w, bc, steps)
    got, _ = _run_sparse(torch_cuda, u, w, steps, dtype, bc, 1, shape)
    l2, linf = oracle_mod.rel_errors(got, ref)
    assert np.all(np.isfinite(got))
    _assert_tol(l2, linf, dtype)


@pytest.mark.parametrize("dims,steps,bc,dtype", [
    ((34, 50, 130), 7, "dirichlet", "fp16"),         # fused sweeps, a remainder sweep, the 3D band
    ((34, 50, 130), 7, "dirichlet", "bf16_split"),
    ((40, 36, 72), 6, "periodic", "bf16"),           # ghost shell of width 2
    ((17, 20, 66), 5, "periodic", "fp16_split"),
    ((18, 21, 70), 5, "dirichlet", "bf16"),          # band boxes ragged along every axis
])
def test_sparse_3d_fused_matches_oracle(torch_cuda, oracle_mod, dims, steps, bc, dtype):
    """3D radius-1 star fused two steps per sweep (one halo stage in shared memory); zero
    Dirichlet boundaries take the frame of width 1 from the 3D band kernel."""
    w = inputs.stencil_weights("star", 3, 1, "random", seed=12)
    u = inputs.uniform_pm1(6, dims)
    ref = oracle_mod.run(u, w, bc, steps)
    got, plan = _run_sparse(torch_cuda, u, w, steps, dtype, bc, 2, "star")
    assert plan.info().fusion_depth == 2
    l2, linf = oracle_mod.rel_errors(got, ref)
    assert np.all(np.isfinite(got))
    _assert_tol(l2, linf, dtype)


def test_full_size_box3d27p_sampled(torch_cuda, oracle_mod):
    """Box-3D27P 256^3, zero Dirichlet boundary, 50 steps, split operands: sampled points
    against the dependence-cone oracle."""
    cfg = inputs.CONFIGS["box3d27p_256"]
    w = inputs.stencil_weights(cfg["shape"], 3, 1, cfg["recipe"], seed=cfg["seed"])
    u = inputs.make_grid(cfg["grid"], cfg["seed"], cfg["dims"])
    got, _ = _run_sparse(torch_cuda, u, w, cfg["steps"], "bf16_split", cfg["bc"], 1, cfg["shape"])
    rng = np.random.default_rng(2)
    pts = [tuple(int(rng.integers(0, d)) for d in cfg["dims"]) for _ in range(5)] + [(0, 0, 0), (255, 255, 255)]
    ref = oracle_mod.points(u, w, cfg["bc"], cfg["steps"], pts)
    vals = np.array([got[p] for p in pts])
    _assert_tol(*_rel(vals, ref), "bf16_split")


@pytest.mark.parametrize("name,npts", [("star2d13p_8192", 6), ("box2d49p_8192", 6)])
def test_full_size_c4_sampled(torch_cuda, oracle_mod, name, npts):
    """Star-2D13P / Box-2D49P 8192^2, 200 steps, Gaussian weights, periodic, in the suite's
    launch configuration (autotuned fusion depth), single-word and split BF16: sampled points
    against the dependence-cone oracle (several seconds of FP64 work per point, on host threads)."""
    cfg = inputs.CONFIGS[name]
    w = inputs.stencil_weights(cfg["shape"], 2, cfg["radius"], cfg["recipe"], seed=cfg["seed"])
    u = inputs.make_grid(cfg["grid"], cfg["seed"], cfg["dims"])
    rng = np.random.default_rng(5)
    pts = [tuple(int(rng.integers(0, d)) for d in cfg["dims"]) for _ in range(npts - 3)]
    pts += [(0, 8191), (127, 128), (8191, 0)]  # grid corners and a tile corner
    ref = oracle_mod.points(u, w, cfg["bc"], cfg["steps"], pts)
    for dtype in ("bf16", "bf16_split"):
        got, plan = _run_sparse(torch_cuda, u, w, cfg["steps"], dtype, cfg["bc"], 0, cfg["shape"])
        vals = np.array([got[p] for p in pts])
        _assert_tol(*_rel(vals, ref), dtype, plan.info().fusion_depth)


def test_full_size_heat3d_sampled(torch_cuda, oracle_mod):
    """Heat-3D 7-point star 512^3 with random weights, zero Dirichlet boundary, 50 steps on
    zero-mean data, FP16 split operands (low-order accumulator by default): sampled points,
    corners included, against the dependence-cone oracle."""
    cfg = inputs.CONFIGS["heat3d_512"]
    w = inputs.stencil_weights(cfg["shape"], 3, 1, cfg["recipe"], seed=cfg["seed"])
    u = inputs.make_grid(cfg["grid"], cfg["seed"], cfg["dims"])
    got, plan = _run_sparse(torch_cuda, u, w, cfg["steps"], "fp16_split", cfg["bc"], 1, cfg["shape"])
    assert plan.info().low_accumulator == 1
    rng = np.random.default_rng(4)
    pts = [tuple(int(rng.integers(0, d)) for d in cfg["dims"]) for _ in range(6)] + [(0, 0, 0), (511, 0, 511)]
    ref = oracle_mod.points(u, w, cfg["bc"], cfg["steps"], pts)
    vals = np.array([got[p] for p in pts])
    _assert_tol(*_rel(vals, ref), "fp16_split")


@pytest.mark.parametrize("ndim,shape,dims,steps,bc,dtype,t", [
    (3, "star", (48, 40, 136), 20, "dirichlet", "fp16_split", 1),
    (3, "box", (32, 36, 128), 12, "periodic", "bf16_split", 1),
    (2, "box", (300, 260), 20, "periodic", "bf16_split", 3),
    (2, "star", (260, 300), 9, "dirichlet", "fp16_split", 2),
])
def test_low_accumulator_matches_oracle(torch_cuda, oracle_mod, ndim, shape, dims, steps, bc, dtype, t):
    """Split operands with the low-order terms in an accumulator of their own: the result
    meets the split tolerance on zero-mean data, and its error is no larger than with one
    accumulator (every MMA rounds its FP32 sum once, so fewer roundings land on the large
    partial sums)."""
    w = inputs.stencil_weights(shape, ndim, 1, "random", seed=13)
    u = inputs.uniform_pm1(7, dims)
    ref = oracle_mod.run(u, w, bc, steps)
    one, _ = _run_sparse(torch_cuda, u, w, steps, dtype, bc, t, shape, low_accumulator=False)
    two, plan = _run_sparse(torch_cuda, u, w, steps, dtype, bc, t, shape, low_accumulator=True)
    assert plan.info().low_accumulator == 1
    l2_one = oracle_mod.rel_errors(one, ref)[0]
    l2_two, linf_two = oracle_mod.rel_errors(two, ref)
    assert np.all(np.isfinite(two))
    _assert_tol(l2_two, linf_two, dtype)
    assert l2_two <= 1.05 * l2_one, (l2_two, l2_one)


@pytest.mark.parametrize("ndim,shape,r,recipe,dims,steps,bc,dtype,t", [
    (2, "box", 1, "random", (300, 260), 12, "periodic", "bf16", 1),
    (2, "box", 1, "random", (260, 300), 9, "periodic", "bf16_split", 3),
    (2, "star", 3, "gaussian", (256, 384), 6, "dirichlet", "bf16", 1),
    (2, "box", 3, "gaussian", (256, 256), 4, "periodic", "bf16", 1),
    (3, "box", 1, "random", (32, 36, 128), 8, "periodic", "fp16_split", 1),
    (3, "star", 1, "random", (20, 40, 70), 5, "dirichlet", "fp16", 1),
])
def test_dense_ablation_matches_oracle(torch_cuda, oracle_mod, ndim, shape, r, recipe, dims, steps, bc, dtype, t):
    """The dense-MMA ablation (uncompressed A', dense kind::f16 MMAs) computes the same
    stencil: within the dtype's tolerance of the oracle, like the sparse path."""
    w = inputs.stencil_weights(shape, ndim, r, recipe, seed=14)
    u = inputs.uniform01(8, dims)
    ref = oracle_mod.run(u, w, bc, steps)
    got, plan = _run_sparse(torch_cuda, u, w, steps, dtype, bc, t, shape, dense=True)
    assert plan.info().dense_ablation == 1
    l2, linf = oracle_mod.rel_errors(got, ref)
    assert np.all(np.isfinite(got))
    _assert_tol(l2, linf, dtype)


CASES_1D = [
    # (shape, r, recipe, length, steps, bc, dtype, t): 1D sweep (patches of 128 outputs, tiles
    # of 16384), ragged, sub-tile and multi-tile lengths
    ("star", 1, "heat", 100000, 20, "dirichlet", "fp16", 1),
    ("star", 1, "heat", 3 * 16384 + 100, 30, "periodic", "bf16_split", 4),
    ("box", 2, "random", 50000, 12, "periodic", "bf16", 3),
    ("box", 2, "random", 70000, 9, "dirichlet", "fp16_split", 1),
    ("star", 1, "random", 300, 5, "periodic", "bf16", 1),
    ("box", 3, "gaussian", 40000, 16, "periodic", "bf16_split", 0),
    # deep 1D fusion (fused radius 60) with a remainder sweep
    ("star", 1, "heat", 3 * 16384 + 100, 130, "periodic", "fp16", 60),
    ("box", 2, "random", 50000, 70, "periodic", "bf16_split", 30),
]


@pytest.mark.parametrize("shape,r,recipe,length,steps,bc,dtype,t", CASES_1D)
def test_sparse_1d_matches_oracle(torch_cuda, oracle_mod, shape, r, recipe, length, steps, bc, dtype, t):
    w = inputs.stencil_weights(shape, 1, r, recipe, seed=15)
    u = inputs.uniform01(9, (length,))
    ref = oracle_mod.run(u, w, bc, steps)
    got, plan = _run_sparse(torch_cuda, u, w, steps, dtype, bc, t, shape)
    assert plan.info().ndim == 1
    l2, linf = oracle_mod.rel_errors(got, ref)
    assert np.all(np.isfinite(got))
    _assert_tol(l2, linf, dtype, plan.info().fusion_depth)


def test_closed_form_fourier_mode_1d(torch_cuda):
    """Periodic 1D with random weights, fused 8 steps per sweep: u = 1/2 + cos(theta x) / 2
    gives u_T = S^T / 2 + Re(lambda^T e^{i theta x}) / 2 with lambda = sum_o w[o] e^{i theta o}."""
    L, T = 5 * 16384 + 4096, 200
    w = inputs.stencil_weights("box", 1, 2, "random", seed=16).astype(np.float64)
    th = 2 * np.pi * 7 / L
    x = np.arange(L)
    lam = sum(w[o + 2] * np.exp(1j * th * o) for o in range(-2, 3))
    u0 = (0.5 + 0.5 * np.cos(th * x)).astype(np.float32)
    ref = 0.5 * float(np.sum(w)) ** T + 0.5 * np.real(lam ** T * np.exp(1j * th * x))
    got, plan = _run_sparse(torch_cuda, u0, w.astype(np.float32), T, "bf16_split", "periodic", 8, "box")
    assert plan.info().fusion_depth == 8
    _assert_tol(*_rel(got, ref), "bf16_split")


@pytest.mark.parametrize("name", ["heat1d", "1d5p"])
def test_full_size_1d_sampled(torch_cuda, oracle_mod, name):
    """Heat-1D / 1D5P at the paper's size (10,240,000 points, 10,000 steps, periodic), in the
    suite's launch configuration (autotuned depth), split BF16: sampled points against the
    dependence-cone oracle."""
    cfg = inputs.CONFIGS[name]
    w = inputs.stencil_weights(cfg["shape"], 1, cfg["radius"], cfg["recipe"], seed=cfg["seed"])
    u = inputs.make_grid(cfg["grid"], cfg["seed"], cfg["dims"])
    got, plan = _run_sparse(torch_cuda, u, w, cfg["steps"], "bf16_split", cfg["bc"], 0, cfg["shape"])
    pts = [(0,), (5120000,), (10239999,)]
    ref = oracle_mod.points(u, w, cfg["bc"], cfg["steps"], pts)
    vals = np.array([got[p] for p in pts])
    _assert_tol(*_rel(vals, ref), "bf16_split", plan.info().fusion_depth)


def _custom(mask, seed):
    rng = np.random.default_rng(seed)
    w = np.where(mask, 0.05 + 0.95 * rng.random(mask.shape), 0.0)
    return (w / w.sum()).astype(np.float32)


@pytest.mark.parametrize("name,dims,steps,bc,dtype,t", [
    ("upwind2d", (300, 260), 12, "periodic", "bf16_split", 2),
    ("upwind2d", (256, 200), 7, "dirichlet", "fp16", 1),
    ("knight2d", (260, 300), 9, "periodic", "bf16", 1),
    ("forward3d", (40, 36, 72), 6, "periodic", "fp16_split", 1),
])
def test_custom_mask_matches_oracle(torch_cuda, oracle_mod, name, dims, steps, bc, dtype, t):
    """Arbitrary (asymmetric, non-staircase) masks through the CUSTOM shape: the sparse path
    matches the oracle at the dtype's tolerance."""
    mask = {"upwind2d": np.array([[1, 1, 0], [1, 1, 0], [0, 0, 0]], bool),
            "knight2d": np.array([[0, 1, 0, 1, 0], [1, 0, 0, 0, 1], [0, 0, 1, 0, 0], [1, 0, 0, 0, 1],
                                  [0, 1, 0, 1, 0]], bool)}.get(name)
    if mask is None:
        mask = np.zeros((3, 3, 3), bool)
        mask[1, 1, 1] = mask[2, 1, 1] = mask[1, 2, 1] = mask[1, 1, 2] = True
    w = _custom(mask, 32)
    u = inputs.uniform01(10, dims)
    ref = oracle_mod.run(u, w, bc, steps)
    got, plan = _run_sparse(torch_cuda, u, w, steps, dtype, bc, t, "custom")
    l2, linf = oracle_mod.rel_errors(got, ref)
    assert np.all(np.isfinite(got))
    _assert_tol(l2, linf, dtype, plan.info().pairing)


@pytest.mark.parametrize("ndim,dims,bc,t,steps", [
    (1, (40000,), "periodic", 3, 6),
    (1, (40000,), "dirichlet", 1, 3),
    (2, (200, 296), "periodic", 3, 6),
    (2, (200, 296), "dirichlet", 3, 6),
    (3, (40, 36, 72), "periodic", 1, 2),
    (3, (40, 36, 72), "dirichlet", 1, 2),
])
@pytest.mark.parametrize("dtype", ["bf16", "bf16_split", "fp16", "fp16_split"])
def test_degenerate_stencils(torch_cuda, oracle_mod, ndim, dims, bc, t, steps, dtype):
    """Degenerate stencils (ragged grids, fused sweeps where the plan allows them): all
    weights zero gives exact zeros; the centre weight alone returns the input; a unit weight
    at offset +1 along the last axis or -1 along the first translates the grid (the oracle's
    exact shift), each within the dtype's tolerance."""
    u = inputs.uniform01(7, dims)
    zero = np.zeros((3,) * ndim, np.float32)
    got, _ = _run_sparse(torch_cuda, u, zero, steps, dtype, bc, t, "box")
    assert np.all(got == 0.0)
    cases = []
    ident = zero.copy()
    ident[(1,) * ndim] = 1.0
    cases.append(ident)
    for axis, sign in ((ndim - 1, 1), (0, -1)):
        w = zero.copy()
        idx = [1] * ndim
        idx[axis] = 1 + sign
        w[tuple(idx)] = 1.0
        cases.append(w)
    for w in cases:
        ref = oracle_mod.run(u, w, bc, steps)
        got, plan = _run_sparse(torch_cuda, u, w, steps, dtype, bc, t, "box")
        assert plan.info().fusion_depth == t
        l2, linf = oracle_mod.rel_errors(got, ref)
        assert np.all(np.isfinite(got))
        _assert_tol(l2, linf, dtype, np.argwhere(w).tolist())


@pytest.mark.parametrize("ndim,shape,r,dims,steps,bc,dtype,t", [
    (2, "box", 6, (300, 260), 3, "periodic", "bf16_split", 1),
    (2, "box", 6, (260, 300), 3, "dirichlet", "fp16", 1),
    (2, "star", 9, (300, 260), 3, "periodic", "bf16_split", 1),
    (2, "star", 4, (300, 260), 4, "periodic", "bf16", 2),
    (1, "box", 60, (40000,), 4, "periodic", "bf16_split", 1),
    (1, "star", 30, (40000,), 4, "periodic", "fp16_split", 2),
])
def test_widest_stencils_match_oracle(torch_cuda, oracle_mod, ndim, shape, r, dims, steps, bc, dtype, t):
    """The widest stencils whose tables fit TMEM (2D: a 13 x 13 box or a radius-9 star,
    K_pad = 576; a radius-4 star fused to radius 8; 1D: fused radius 60) match the oracle
    at the dtype's tolerance."""
    w = inputs.stencil_weights(shape, ndim, r, "gaussian", seed=17)
    u = inputs.uniform01(12, dims)
    ref = oracle_mod.run(u, w, bc, steps)
    got, plan = _run_sparse(torch_cuda, u, w, steps, dtype, bc, t, shape)
    assert plan.info().fusion_depth == t
    l2, linf = oracle_mod.rel_errors(got, ref)
    assert np.all(np.isfinite(got))
    _assert_tol(l2, linf, dtype, plan.info().kpad)


@pytest.mark.parametrize("ndim,shape,r,dims,bc,dtype,t,k,steps", [
    (2, "box", 1, (300, 260), "periodic", "bf16_split", 3, 1, 7),     # every step in FP64
    (2, "box", 1, (300, 260), "dirichlet", "bf16_split", 3, 4, 17),   # sweeps of 3, bands, FP64 every 4th step
    (2, "star", 3, (260, 300), "periodic", "fp16_split", 2, 5, 13),
    (3, "star", 1, (20, 40, 70), "dirichlet", "fp16_split", 2, 3, 8),
    (3, "box", 1, (20, 24, 72), "periodic", "bf16_split", 1, 2, 6),   # ghost shell written by both kinds of step
    (1, "box", 2, (40000,), "periodic", "bf16_split", 8, 5, 23),
])
def test_fp64_correction_matches_oracle(torch_cuda, oracle_mod, ndim, shape, r, dims, bc, dtype, t, k, steps):
    """The optional FP64 correction step: every k-th time step on the CUDA cores in FP64, the
    others in tensor-core sweeps (remainder sweeps between the FP64 steps).  With k = 1 every
    step is FP64 and the result is within the FP32 rounding of the stored state of the oracle;
    otherwise within the split tolerance."""
    torch = torch_cuda
    recipe = "gaussian" if r == 3 else "random"
    w = inputs.stencil_weights(shape, ndim, r, recipe, seed=13)
    u = inputs.uniform_pm1(9, dims) if ndim == 3 else inputs.uniform01(9, dims)
    plan = binding.Plan(w, dims, dtype=dtype, bc=bc, fusion_depth=t, shape=shape)
    plan.set_fp64_correction(k)
    assert plan.info().fp64_every == k
    x = torch.from_numpy(u).cuda()
    y = torch.full_like(x, float("nan"))
    plan.run(x, y, steps)
    torch.cuda.synchronize()
    assert binding.device_status() == 0
    got = y.cpu().numpy()
    assert np.all(np.isfinite(got))
    l2, linf = oracle_mod.rel_errors(got, oracle_mod.run(u, w, bc, steps))
    if k == 1:
        assert l2 <= 1e-6 and linf <= 1e-5, (l2, linf)
    else:
        _assert_tol(l2, linf, dtype)


def test_fp64_correction_rejected_by_batch_and_noalloc(torch_cuda):
    torch = torch_cuda
    w = inputs.stencil_weights("box", 2, 1, "random", seed=1)
    plan = binding.Plan(w, (128, 128), dtype="bf16", bc="periodic", fusion_depth=1)
    plan.set_fp64_correction(3)
    x = torch.zeros(128, 128, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(binding.SparStencilError):
        binding.run_batch([plan], [x], [y], [4])
    with pytest.raises(binding.SparStencilError):
        plan.run_noalloc(x, y, 4)
