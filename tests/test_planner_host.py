"""Host-only checks of the C-ABI library: it loads, exports every declared symbol, and its
planner tables are bit-exact against the oracle's literal restatement of Sec. 3.1-3.3.

No GPU is needed: sparstencil_plan and sparstencil_plan_tables are host-only calls.
"""
import os
import re

import numpy as np
import pytest

from oracle import morph
from oracle.morph import ZERO
from paper_2506_22969_gb300 import binding, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_22969_gb300 import build
    build.build()
    return binding.load()


def test_library_exports_every_declared_symbol(lib):
    with open(os.path.join(ROOT, "include", "sparstencil.h")) as f:
        text = f.read()
    declared = set(re.findall(r"\b(sparstencil_[a-z0-9_]+)\s*\(", text))
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert set(binding.EXPORTS) <= declared


def _bf16(x):
    import torch
    return torch.tensor(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def _fp16(x):
    return np.asarray(x, np.float32).astype(np.float16).astype(np.float32)


def _oracle_order(wf, k, r1, r2, drop=True):
    """Algorithm 1 order, dropping pairs whose two A' columns are all zero, padded to 32."""
    A = morph.crushed_weights(wf, r1, r2)
    g, mb = k + r1 - 1, k + r2 - 1
    nz = np.any(A != 0, axis=0)
    _, _, M = morph.hierarchical_matching(g * mb, g, k)
    order = []
    for a, b in M:
        if drop and not nz[a] and (b == ZERO or not nz[b]):
            continue
        order.extend([a, b])
    while len(order) % 32:
        order.append(ZERO)
    return A, np.array(order)


def _composed(w, t):
    """t-step kernel read off the oracle: one impulse, t steps, correlation orientation."""
    import oracle
    r = (w.shape[0] - 1) // 2
    R = t * r
    n = 4 * R + 3
    u = np.zeros((n, n))
    c = n // 2
    u[c, c] = 1.0
    out = oracle.run(u, w.astype(np.float64), "periodic", t)
    return out[c - R:c + R + 1, c - R:c + R + 1][::-1, ::-1]


CASES = [("star", 1, "heat", 1, "bf16"), ("box", 1, "random", 1, "bf16_split"), ("box", 1, "random", 2, "bf16"),
         ("box", 1, "random", 3, "fp16_split"), ("star", 3, "gaussian", 1, "bf16_split"),
         ("box", 3, "gaussian", 1, "fp16"), ("box", 2, "random", 1, "bf16"),
         # the widest 2D stencils whose tables fit TMEM (K_pad = 576)
         ("box", 6, "gaussian", 1, "bf16_split"), ("star", 9, "gaussian", 1, "fp16")]


# the tall 8 x 16 patch layout (sparstencil_plan_set_layout r1 = 8)
CASES_TALL = [("star", 1, "heat", 1, "bf16"), ("box", 1, "random", 3, "bf16_split"),
              ("star", 3, "gaussian", 1, "bf16_split"), ("box", 3, "gaussian", 2, "fp16")]


@pytest.mark.parametrize("r1", [16, 8])
@pytest.mark.parametrize("shape,r,recipe,t,dtype", CASES + CASES_TALL)
def test_planner_tables_against_oracle(lib, oracle_mod, shape, r, recipe, t, dtype, r1):
    if r1 == 8 and (shape, r, recipe, t, dtype) not in CASES_TALL:
        pytest.skip("tall layout checked on its own cases")
    w = inputs.stencil_weights(shape, 2, r, recipe, seed=7)
    plan = binding.Plan(w, (300, 260), dtype=dtype, bc="periodic", fusion_depth=t, shape=shape, layout=(r1, -1))
    info = plan.info()
    tb = plan.tables()
    k = 2 * t * r + 1
    # composed weights equal the oracle's t-step impulse response
    np.testing.assert_allclose(tb["fused_w"], _composed(w, t), rtol=1e-13, atol=1e-16)
    wf32 = tb["fused_w"].astype(np.float32).astype(np.float64)
    A, alg1 = _oracle_order(wf32, k, r1, 128 // r1)
    assert info.r1 == r1 and info.r2 == 128 // r1 and info.kprime == A.shape[1]
    order = tb["order"]
    assert info.kpad == len(order) and info.kpad % 32 == 0

    def pairset(o):
        return sorted(tuple(sorted((int(o[2 * i]), int(o[2 * i + 1])))) for i in range(len(o) // 2)
                      if not (o[2 * i] == ZERO and o[2 * i + 1] == ZERO))
    if info.pairing == 0:
        # the planner keeps Algorithm 1's pairs (as unordered pairs) and may reorder and orient them
        assert shape == "box" or len(order) <= len(alg1)
        assert len(order) == len(alg1) and pairset(order) == pairset(alg1)
    else:
        # a support smaller than the box: a maximum matching on it, with fewer K chunks than
        # Algorithm 1 and the oracle's zero-column count (maximum matchings all have one size)
        pytest.importorskip("networkx")
        assert shape != "box" and len(order) < len(alg1)
        _, zeros = morph.max_matching_pairs(A)
        assert info.zero_columns == zeros
        E = morph.conflict_graph(A)
        nzc = np.where(np.any(A != 0, axis=0))[0]
        ps = pairset(order)
        assert sorted(v for pr in ps for v in pr if v != ZERO) == sorted(nzc.tolist())
        assert all(a == ZERO or b == ZERO or not E[a, b] for a, b in ps)
        assert len(ps) == (len(nzc) + zeros) // 2
    # gather bank rule: in every 32-row chunk the 16 first-column offsets, and the 16
    # second-column offsets, are distinct mod 16 (up to the repeats the plan reports)
    lut = tb["lut"]
    repeats = 0
    for kc in range(len(order) // 32):
        for side in (0, 1):
            r = lut[kc * 32 + side:(kc + 1) * 32:2] % 16
            repeats += 16 - len(set(r.tolist()))
    assert repeats <= info.bank_conflicts
    # decompress and check 2:4, values and un-permutation to A'
    split = dtype.endswith("split")
    fp16 = dtype.startswith("fp16")
    rnd = _fp16 if fp16 else _bf16
    s = 11 - int(np.frexp(np.max(np.abs(wf32)))[1]) if fp16 else 0  # FP16 pieces hold w * 2^s
    sc = 2.0 ** s
    dense_hi = morph.decompress_2_4(tb["a_hi"].astype(np.float64), tb["a_idx"])
    dense_lo = morph.decompress_2_4(tb["a_lo"].astype(np.float64), tb["a_idx"])
    assert morph.satisfies_2_4(dense_hi) and morph.satisfies_2_4(dense_hi + dense_lo)
    Ap = morph.apply_permutation(A, list(order))
    np.testing.assert_array_equal(dense_hi, rnd(Ap * sc) / sc)
    # weight pieces: BF16 split operands use three (two for a fused sweep that needs the TMEM
    # for a second accumulator), FP16 split and single-word operands two; one MMA term per
    # piece, plus one for the data's low part with split operands
    pieces = info.mma_terms - (1 if split else 0)
    # three pieces leave no TMEM for an accumulator (128 columns) when the A'' pieces
    # (K_pad/4 columns each) and the metadata (8 columns per two chunks) take more than 384
    three_fit = 3 * (info.kpad // 4) + 8 * ((info.kpad // 32 + 1) // 2) <= 512 - 128
    assert pieces in (1, 2, 3) and (pieces == 3 or not split or t >= 2 or fp16 or not three_fit)
    if pieces == 3 and not fp16:
        # three BF16 pieces hold every FP32 weight exactly
        np.testing.assert_array_equal(dense_hi + dense_lo, Ap)
    elif pieces == 3:
        # FP16's third piece is limited by the subnormal step 2^-24 of the scaled weights
        assert np.max(np.abs(dense_hi + dense_lo - Ap)) <= 2.0 ** -24 * np.max(np.abs(wf32))
    else:
        np.testing.assert_array_equal(dense_lo, rnd((Ap * sc).astype(np.float32) - (dense_hi * sc).astype(np.float32)) / sc)
    # metadata positions: distinct and ascending inside each group
    idx = tb["a_idx"].reshape(128, -1, 2)
    assert np.all(idx[:, :, 0] < idx[:, :, 1])


def _emulate_sweep(plan, tb, u, bc, dense):
    """Host emulation of one sweep through the planner's LUT: padded grid -> halo tiles ->
    B'' gathered by LUT -> dense A'' @ B'' -> outputs by the patch map."""
    info = plan.info()
    H, W = u.shape
    G, P, bh = info.ghost, info.tile_pitch, info.tile_rows
    Wp = (W + 2 * G + 3) // 4 * 4
    up = np.zeros((H + 2 * G, Wp))
    yy, xx = np.mgrid[-G:H + G, -G:W + G]
    if bc == "periodic":
        up[:, :W + 2 * G] = u[yy % H, xx % W]
    else:
        inside = (yy >= 0) & (yy < H) & (xx >= 0) & (xx < W)
        up[:, :W + 2 * G] = np.where(inside, u[np.clip(yy, 0, H - 1), np.clip(xx, 0, W - 1)], 0.0)
    out = np.full((H, W), np.nan)
    lut = tb["lut"]
    for ty in range((H + 127) // 128):
        for tx in range((W + 127) // 128):
            tile = np.zeros((bh, P))
            blk = up[ty * 128:ty * 128 + bh, tx * 128:tx * 128 + P]
            tile[:blk.shape[0], :blk.shape[1]] = blk
            flat = tile.ravel()
            r1 = info.r1
            r2 = 128 // r1
            for n in range(128):
                if r1 == 16:
                    px, py = (n >> 3) & 7, ((n >> 6) << 3) + (n & 7)
                else:  # tall 8 x 16 patches: n = 16 py + 8 hb + e
                    e, hb = n & 7, (n >> 3) & 1
                    px, py = 4 * (e >> 1) + 2 * hb + (e & 1), n >> 4
                base = py * r2 * P + px * r1
                col = dense @ flat[base + lut]
                for rho in range(128):
                    y, x = ty * 128 + py * r2 + rho // r1, tx * 128 + px * r1 + rho % r1
                    if y < H and x < W:
                        out[y, x] = col[rho]
    return out


@pytest.mark.parametrize("bc,shape,r,t,r1", [("periodic", "box", 1, 1, 16), ("dirichlet", "star", 1, 1, 16),
                                             ("periodic", "box", 1, 2, 16), ("periodic", "star", 3, 1, 16),
                                             ("periodic", "box", 1, 1, 8), ("dirichlet", "star", 3, 1, 8),
                                             ("periodic", "box", 1, 2, 8)])
def test_lut_emulation_reproduces_oracle_step(lib, oracle_mod, bc, shape, r, t, r1):
    """Bit-level check of every table the kernel consumes: with exact dyadic weights the
    emulated sweep (LUT gather, permuted A'', patch map) equals t oracle steps exactly."""
    side = 2 * r + 1
    mask = inputs.stencil_mask(shape, 2, r)
    w = np.where(mask, np.arange(1, side * side + 1).reshape(side, side) / 256.0, 0.0).astype(np.float32)
    u = np.random.default_rng(3).integers(-8, 9, size=(140, 200)).astype(np.float64) / 8.0
    plan = binding.Plan(w, u.shape, dtype="bf16", bc=bc, fusion_depth=t, shape=shape, layout=(r1, -1))
    tb = plan.tables()
    dense = morph.decompress_2_4(tb["a_hi"].astype(np.float64) + tb["a_lo"], tb["a_idx"])
    ref = oracle_mod.run(u, w.astype(np.float64), bc, t)
    if t == 1:
        got = _emulate_sweep(plan, tb, u, bc, dense)
        np.testing.assert_array_equal(got, ref)
    else:
        # fused weights are not exact in BF16: compare with the oracle at the weight rounding level
        dense64 = morph.apply_permutation(morph.crushed_weights(tb["fused_w"], r1, 128 // r1), list(tb["order"]))
        got = _emulate_sweep(plan, tb, u, bc, dense64)
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def test_remainder_tables(lib):
    w = inputs.stencil_weights("box", 2, 1, "random", seed=2)
    plan = binding.Plan(w, (512, 512), dtype="bf16", bc="periodic", fusion_depth=3)
    t3 = plan.tables(0)
    t1 = plan.tables(1, remainder_depth=1)
    t2 = plan.tables(1, remainder_depth=2)
    assert t3["fused_w"].shape == (7, 7) and t2["fused_w"].shape == (5, 5) and t1["fused_w"].shape == (3, 3)
    np.testing.assert_array_equal(t1["fused_w"], w.astype(np.float64))


@pytest.mark.parametrize("kwargs,code", [
    (dict(dims=(0, 64)), 1), (dict(dtype=9), 1), (dict(bc=5), 1),
    (dict(dims=(1, 64)), 2), (dict(fusion_depth=-1), 1)])
def test_plan_rejects_bad_arguments(lib, kwargs, code):
    w = inputs.stencil_weights("box", 2, 1, "random", seed=2)
    args = dict(dims=(64, 64), dtype="bf16", bc="periodic", fusion_depth=1)
    args.update(kwargs)
    with pytest.raises(binding.SparStencilError) as e:
        binding.Plan(w, **args)
    assert e.value.code == code


def test_binding_checks_rank(lib):
    w = inputs.stencil_weights("box", 2, 1, "random", seed=2)
    with pytest.raises(ValueError):
        binding.Plan(w, (64, 64, 64))


def test_star_plan_rejects_off_axis_weight(lib):
    w = inputs.stencil_weights("box", 2, 1, "random", seed=2)
    with pytest.raises(binding.SparStencilError) as e:
        binding.Plan(w, (64, 64), shape="star")
    assert e.value.code == 1


def test_cost_model_orders_layouts():
    """Sec. 3.3 cost model sanity: the crushed layout moves fewer shared-memory bytes than
    plain flattening (r1 = r2 = 1), in the oracle's own morph dimensions."""
    mp1, kp1, np1 = morph.morph_dims(3, 1, 1, 4098, 4098)
    mp2, kp2, np2 = morph.morph_dims(3, 16, 8, 4098, 4098)
    trans1 = kp1 * (mp1 / 2 + np1)
    trans2 = kp2 * (mp2 / 2 + np2)
    assert trans2 < trans1 / 5


def test_autotune_plan_takes_the_deepest_depth_that_fits(lib):
    """fusion_depth 0 plans the deepest depth whose tables fit (2D: of 6 down to 1; the first
    run then times each depth up to it)."""
    w = inputs.stencil_weights("box", 2, 1, "random", seed=2)
    p = binding.Plan(w, (512, 512), dtype="bf16_split", bc="periodic", fusion_depth=0)
    # 3x3 box: t = 6 (K_pad 576) fits; t = 7 (K_pad 672) would not, and is not searched
    assert p.info().fusion_depth == 6 and p.info().ghost == 6 and p.info().kpad == 576
    with pytest.raises(binding.SparStencilError) as e:
        binding.Plan(w, (512, 512), dtype="bf16_split", bc="periodic", fusion_depth=7)
    assert e.value.code == 2
    # 1D: K grows by 2r columns per step, so the search starts at a fused radius of 60
    w1 = inputs.stencil_weights("star", 1, 1, "heat", seed=2)
    p1 = binding.Plan(w1, (100000,), dtype="bf16_split", bc="periodic", fusion_depth=0)
    assert p1.info().fusion_depth == 60 and p1.info().ghost == 60 and p1.info().kpad == 256
    w12 = inputs.stencil_weights("box", 1, 2, "random", seed=2)
    assert binding.Plan(w12, (100000,), dtype="fp16", bc="periodic", fusion_depth=0).info().fusion_depth == 30
    # a depth whose patch input count alone cannot fit TMEM is rejected before any matching
    with pytest.raises(binding.SparStencilError) as e:
        binding.Plan(w, (512, 512), dtype="bf16_split", bc="periodic", fusion_depth=20)
    assert e.value.code == 2 and "kpad >= 2688" in str(e.value)
    # 5x5 box: t = 3 (fused radius 6, K_pad 576) is the deepest that fits
    w2 = inputs.stencil_weights("box", 2, 2, "random", seed=2)
    p2 = binding.Plan(w2, (512, 512), dtype="bf16_split", bc="periodic", fusion_depth=0)
    assert p2.info().fusion_depth == 3 and p2.info().kpad == 576
    # 7x7 box, split: t = 3 (K_pad 960) does not fit TMEM; t = 2 (K_pad 576) fits with two
    # BF16 weight pieces beside one accumulator
    w3 = inputs.stencil_weights("box", 2, 3, "gaussian", seed=2)
    p3 = binding.Plan(w3, (512, 512), dtype="bf16_split", bc="periodic", fusion_depth=0)
    assert p3.info().fusion_depth == 2 and p3.info().mma_terms == 3
    # 3D radius 1: the 7-point star fuses two steps (K_pad 512, one halo stage of 68 x 20 x 20
    # floats), also with a zero Dirichlet boundary (the 3D band kernel); the 27-point box needs
    # K_pad >= 768 at t = 2 and stays at t = 1
    w7 = inputs.stencil_weights("star", 3, 1, "random", seed=2)
    for bc in ("dirichlet", "periodic"):
        p7 = binding.Plan(w7, (64, 64, 64), dtype="fp16", bc=bc, fusion_depth=0, shape="star")
        assert p7.info().fusion_depth == 2 and p7.info().kpad == 512 and p7.info().ghost == 2
    w27 = inputs.stencil_weights("box", 3, 1, "random", seed=2)
    assert binding.Plan(w27, (64, 64, 64), dtype="fp16", bc="dirichlet", fusion_depth=0).info().fusion_depth == 1
    # 3D split operands keep the depths where the low-order accumulator fits (t = 1 here)
    for dt in ("fp16_split", "bf16_split"):
        ps = binding.Plan(w7, (64, 64, 64), dtype=dt, bc="dirichlet", fusion_depth=0, shape="star")
        assert ps.info().fusion_depth == 1 and ps.info().low_accumulator == 1


def test_layout_setting(lib):
    """sparstencil_plan_set_layout: 2D patches 16 x 8 or 8 x 16, pairings -1 / 0 / 1; other
    shapes and 1D/3D shapes are refused and leave the plan unchanged."""
    w = inputs.stencil_weights("star", 2, 3, "gaussian", seed=2)
    p = binding.Plan(w, (300, 260), dtype="bf16", bc="periodic", fusion_depth=1, shape="star")
    assert (p.info().r1, p.info().r2) == (16, 8)
    p.set_layout(8, 0)
    assert (p.info().r1, p.info().r2, p.info().pairing) == (8, 16, 0)
    p.set_layout(8, 1)
    assert p.info().pairing == 1
    for r1, pairing, code in ((12, -1, 2), (16, 3, 1)):
        with pytest.raises(binding.SparStencilError) as e:
            p.set_layout(r1, pairing)
        assert e.value.code == code
    assert (p.info().r1, p.info().pairing) == (8, 1)
    w3 = inputs.stencil_weights("box", 3, 1, "random", seed=2)
    p3 = binding.Plan(w3, (32, 32, 64), dtype="bf16", bc="periodic", fusion_depth=1)
    with pytest.raises(binding.SparStencilError) as e:
        p3.set_layout(16, -1)
    assert e.value.code == 2
    p3.set_layout(8, -1)


def test_low_accumulator_setting(lib):
    """The low-order accumulator: split dtypes only, before the first run; a tile then takes
    256 TMEM columns, so BF16 split keeps three weight pieces only where they fit beside it,
    and a plan whose tables do not fit is refused and left as it was."""
    w = inputs.stencil_weights("box", 2, 1, "random", seed=2)
    single = binding.Plan(w, (256, 256), dtype="bf16", fusion_depth=1)
    with pytest.raises(binding.SparStencilError) as e:
        single.set_low_accumulator(True)
    assert e.value.code == 1 and single.info().low_accumulator == 0
    # box 3x3 at t = 1: three BF16 pieces (3 * 48 + 8 * 2 columns) fit beside two accumulators
    p1 = binding.Plan(w, (256, 256), dtype="bf16_split", fusion_depth=1, low_accumulator=True)
    assert p1.info().low_accumulator == 1 and p1.info().mma_terms == 4
    # box 3x3 at t = 3 (kpad 320): three pieces would need 3 * 80 + 40 + 256 > 512 columns
    p3 = binding.Plan(w, (512, 512), dtype="bf16_split", fusion_depth=3)
    assert p3.info().mma_terms == 3
    p3.set_low_accumulator(True)
    assert p3.info().low_accumulator == 1 and p3.info().mma_terms == 3
    p3.set_low_accumulator(False)
    assert p3.info().low_accumulator == 0
    # a 7x7 box at t = 1 (K_pad 320): checked against the TMEM budget of the second accumulator
    w7 = inputs.stencil_weights("box", 2, 3, "gaussian", seed=2)
    p7 = binding.Plan(w7, (512, 512), dtype="fp16_split", fusion_depth=1)
    kpad = p7.info().kpad
    if 256 + 2 * (kpad // 4) + 8 * ((kpad // 32 + 1) // 2) > 512:
        with pytest.raises(binding.SparStencilError) as e:
            p7.set_low_accumulator(True)
        assert e.value.code == 2 and p7.info().low_accumulator == 0
    # FP16 split plans take it by default where it fits (3D radius 1, two pieces); it can be
    # switched off before the first run
    for shape in ("star", "box"):
        w3 = inputs.stencil_weights(shape, 3, 1, "random", seed=3)
        p = binding.Plan(w3, (64, 64, 128), dtype="fp16_split", fusion_depth=1, shape=shape)
        assert p.info().low_accumulator == 1 and p.info().mma_terms == 3
        p.set_low_accumulator(False)
        assert p.info().low_accumulator == 0 and p.info().mma_terms == 3
    assert binding.Plan(w, (256, 256), dtype="bf16_split", fusion_depth=1).info().low_accumulator == 0


def test_dense_ablation_setting(lib):
    """The dense-MMA ablation: set before the first run; the uncompressed A' takes K/2 TMEM
    columns per piece, and a plan whose A' does not fit is refused and left as it was."""
    w = inputs.stencil_weights("box", 2, 1, "random", seed=2)
    p = binding.Plan(w, (256, 256), dtype="bf16_split", fusion_depth=1)
    info = p.info()
    p.set_dense_ablation(True)
    assert p.info().dense_ablation == 1 and p.info().kpad == info.kpad
    p.set_dense_ablation(False)
    assert p.info().dense_ablation == 0
    # FP16 split 3D: the low-order accumulator gives way to the uncompressed A'
    w3 = inputs.stencil_weights("box", 3, 1, "random", seed=3)
    p3 = binding.Plan(w3, (32, 32, 128), dtype="fp16_split", fusion_depth=1, shape="box")
    assert p3.info().low_accumulator == 1
    p3.set_dense_ablation(True)
    assert p3.info().dense_ablation == 1 and p3.info().low_accumulator == 0
    # a 7x7 box at t = 2 (K_pad 576): two uncompressed pieces of 288 columns do not fit
    w7 = inputs.stencil_weights("box", 2, 3, "gaussian", seed=2)
    p7 = binding.Plan(w7, (512, 512), dtype="bf16", fusion_depth=2)
    with pytest.raises(binding.SparStencilError) as e:
        p7.set_dense_ablation(True)
    assert e.value.code == 2 and p7.info().dense_ablation == 0
    # at t = 1 (K_pad 320) split operands fit with two pieces (three would not)
    p71 = binding.Plan(w7, (512, 512), dtype="bf16_split", fusion_depth=1, dense=True)
    assert p71.info().dense_ablation == 1 and p71.info().mma_terms == 3


def _custom_weights(mask, seed):
    """Positive weights on an arbitrary mask (offset-indexed cube), normalised to sum 1."""
    rng = np.random.default_rng(seed)
    w = np.where(mask, 0.05 + 0.95 * rng.random(mask.shape), 0.0)
    return (w / w.sum()).astype(np.float32)


CUSTOM_MASKS = {
    # 2D upwind corner: centre, west, north, north-west (asymmetric)
    "upwind2d": np.array([[1, 1, 0], [1, 1, 0], [0, 0, 0]], bool),
    # 2D knight moves plus centre, radius 2
    "knight2d": np.array([[0, 1, 0, 1, 0], [1, 0, 0, 0, 1], [0, 0, 1, 0, 0], [1, 0, 0, 0, 1], [0, 1, 0, 1, 0]], bool),
    # 3D: centre and the three "forward" neighbours
    "forward3d": np.zeros((3, 3, 3), bool),
}
CUSTOM_MASKS["forward3d"][1, 1, 1] = CUSTOM_MASKS["forward3d"][2, 1, 1] = True
CUSTOM_MASKS["forward3d"][1, 2, 1] = CUSTOM_MASKS["forward3d"][1, 1, 2] = True


@pytest.mark.parametrize("name,t", [("upwind2d", 1), ("upwind2d", 2), ("knight2d", 1), ("forward3d", 1)])
def test_custom_mask_tables(lib, name, t):
    """CUSTOM shapes: any support inside the cube.  The tables hold the oracle's A' after
    un-permutation, every pair holds at most one nonzero per row, and with the maximum-matching
    pairing the zero columns equal the optimum of Problem 1 on the support."""
    mask = CUSTOM_MASKS[name]
    w = _custom_weights(mask, 31)
    nd = mask.ndim
    dims = (300, 260) if nd == 2 else (40, 36, 72)
    plan = binding.Plan(w, dims, dtype="bf16_split", bc="periodic", fusion_depth=t, shape="custom")
    info = plan.info()
    tb = plan.tables()
    wf32 = tb["fused_w"].astype(np.float32).astype(np.float64)
    A = morph.crushed_weights(wf32, 16, 8) if nd == 2 else morph.crushed_weights_3d(wf32, 8, 4, 4)
    dense = morph.decompress_2_4(tb["a_hi"].astype(np.float64) + tb["a_lo"], tb["a_idx"])
    assert morph.satisfies_2_4(dense)
    order = tb["order"]
    Ap = morph.apply_permutation(A, list(order))
    if info.mma_terms == 4:
        np.testing.assert_array_equal(dense, Ap)
    else:
        assert np.max(np.abs(dense - Ap)) <= 2.0 ** -15 * np.max(np.abs(A))
    E = morph.conflict_graph(A)
    for i in range(len(order) // 2):
        a, b = int(order[2 * i]), int(order[2 * i + 1])
        assert a == ZERO or b == ZERO or not E[a, b]
    if info.pairing == 1:
        pytest.importorskip("networkx")
        _, zeros = morph.max_matching_pairs(A)
        assert info.zero_columns == zeros


def test_plans_of_one_stencil_share_tables(lib):
    """Planner tables depend on the stencil and the tile geometry, not on the grid's extents:
    plans of one stencil on grids of different sizes get the same tables (from the
    process-wide cache), and a stencil with other weights gets its own."""
    w = inputs.stencil_weights("star", 3, 1, "random", seed=21)
    a = binding.Plan(w, (40, 36, 72), dtype="bf16_split", fusion_depth=1, shape="star").tables()
    b = binding.Plan(w, (64, 48, 200), dtype="bf16_split", fusion_depth=1, shape="star").tables()
    for k in ("order", "lut", "a_hi", "a_lo", "a_idx"):
        np.testing.assert_array_equal(a[k], b[k])
    w2 = w.copy()
    w2[1, 1, 1] *= 0.5
    c = binding.Plan(w2, (40, 36, 72), dtype="bf16_split", fusion_depth=1, shape="star").tables()
    assert not np.array_equal(a["a_hi"] + a["a_lo"], c["a_hi"] + c["a_lo"])


def test_cost_model_entry_point(lib):
    """sparstencil_cost_model (Eq. 6-11): with a fast tensor pipe the HBM term binds and the
    time per step falls as 1/t; with a slow one the compute term binds and grows with the
    executed MMAs (K chunks x terms); bad arguments are refused."""
    w = inputs.stencil_weights("box", 2, 1, "random", seed=2)
    p = binding.Plan(w, (4096, 4096), dtype="bf16_split", fusion_depth=3)
    fast = (1e18, 6790e9, 1e18)
    per_step = [p.cost_model(t, *fast) for t in (1, 2, 3)]
    hbm = 8.0 * 4096 * 4096 / 6790e9
    np.testing.assert_allclose(per_step, [hbm, hbm / 2, hbm / 3], rtol=1e-12)
    slow = (1e12, 1e18, 1e18)
    t3 = p.cost_model(3, *slow)
    info = p.info()
    n_mma = (info.kpad // 32) * (4096 * 4096 // 128 // 128) * info.mma_terms
    assert t3 == pytest.approx(n_mma * 2 * 128 * 128 * 32 / 1e12 / 3, rel=1e-12)
    for bad in ((0, *fast), (4, *fast), (1, 0.0, 1e9, 1e9)):
        with pytest.raises(binding.SparStencilError) as e:
            p.cost_model(*bad)
        assert e.value.code == 1


@pytest.mark.parametrize("shape,r,t,dtype", [("star", 1, 1, "bf16_split"), ("box", 2, 1, "bf16"),
                                           ("star", 1, 4, "fp16_split"), ("box", 2, 3, "bf16_split"),
                                           ("box", 60, 1, "bf16_split"), ("star", 30, 2, "fp16")])
def test_planner_tables_1d_against_oracle(lib, shape, r, t, dtype):
    """1D plans (patches of 128 consecutive outputs): A' is the single local staircase of
    Sec. 3.1 (r1 = 128), the pairs are Algorithm 1's on one block, the LUT reads column c of
    the patch window at tile word c + G - R, and the decompressed A'' un-permutes to A'."""
    w = inputs.stencil_weights(shape, 1, r, "random", seed=7)
    plan = binding.Plan(w, (100000,), dtype=dtype, bc="periodic", fusion_depth=t, shape=shape)
    info = plan.info()
    tb = plan.tables()
    k = 2 * t * r + 1
    np.testing.assert_allclose(tb["fused_w"], _composed_1d(w, t), rtol=1e-13, atol=1e-16)
    wf32 = tb["fused_w"].astype(np.float32).astype(np.float64)
    A = morph.local_staircase(wf32, 128)
    assert info.r1 == 128 and info.kprime == A.shape[1] == k + 127
    _, _, M = morph.hierarchical_matching(A.shape[1], A.shape[1], k)
    alg = [v for pr in M for v in pr]
    order = tb["order"]

    def pairset(o):
        return sorted(tuple(sorted((int(o[2 * i]), int(o[2 * i + 1])))) for i in range(len(o) // 2)
                      if not (o[2 * i] == ZERO and o[2 * i + 1] == ZERO))
    assert info.pairing == 0 and pairset(order) == pairset(alg)
    assert info.kpad == len(order) == (len(alg) + 31) // 32 * 32
    G, R = info.ghost, t * r
    real = order != ZERO
    np.testing.assert_array_equal(tb["lut"][real], order[real] + G - R)
    dense = morph.decompress_2_4(tb["a_hi"].astype(np.float64) + tb["a_lo"], tb["a_idx"])
    assert morph.satisfies_2_4(dense)
    Ap = morph.apply_permutation(A, list(order))
    if dtype == "bf16_split" and info.mma_terms == 4:
        np.testing.assert_array_equal(dense, Ap)  # three BF16 pieces: exact
    else:
        assert np.max(np.abs(dense - Ap)) <= 2.0 ** -15 * np.max(np.abs(A))


def _composed_1d(w, t):
    """t-step 1D kernel read off the oracle: one impulse, t steps."""
    import oracle
    r = (w.shape[0] - 1) // 2
    R = t * r
    n = 4 * R + 3
    u = np.zeros(n)
    u[n // 2] = 1.0
    out = oracle.run(u, w.astype(np.float64), "periodic", t)
    return out[n // 2 - R:n // 2 + R + 1][::-1]


def _oracle_order_3d(wf, k, r1, r2, r3):
    """The 3D reading: nested staircase A' and Algorithm 1 applied level by level."""
    A = morph.crushed_weights_3d(wf, r1, r2, r3)
    g, mb, mz = k + r1 - 1, k + r2 - 1, k + r3 - 1
    nz = np.any(A != 0, axis=0)
    order = []
    for a, b in morph.hierarchical_matching_nd([mz, mb, g], k):
        if not nz[a] and (b == ZERO or not nz[b]):
            continue
        order.extend([a, b])
    while len(order) % 32:
        order.append(ZERO)
    return A, np.array(order)


@pytest.mark.parametrize("shape,recipe,dtype", [("box", "random", "bf16"), ("star", "random", "bf16_split"),
                                                ("box", "random", "fp16")])
def test_planner_tables_3d_against_oracle(lib, shape, recipe, dtype):
    """3D plans (Tile3D: 8 x 4 x 4 patches): same pair set as the oracle's level-by-level
    Algorithm 1 (box) or a maximum matching on the actual support (star, fewer K chunks),
    2:4 holds, and the decompressed A'' un-permutes to the oracle's A'."""
    w = inputs.stencil_weights(shape, 3, 1, recipe, seed=7)
    plan = binding.Plan(w, (40, 36, 72), dtype=dtype, bc="periodic", fusion_depth=1, shape=shape)
    info = plan.info()
    tb = plan.tables()
    wf32 = tb["fused_w"].astype(np.float32).astype(np.float64)
    np.testing.assert_array_equal(wf32, w.astype(np.float64))
    A, alg = _oracle_order_3d(wf32, 3, 8, 4, 4)
    assert info.r1 == 8 and info.r2 == 4 and info.r3 == 4 and info.kprime == A.shape[1]
    order = tb["order"]

    def pairset(o):
        return sorted(tuple(sorted((int(o[2 * i]), int(o[2 * i + 1])))) for i in range(len(o) // 2)
                      if not (o[2 * i] == ZERO and o[2 * i + 1] == ZERO))
    if info.pairing == 0:
        assert pairset(order) == pairset(alg) and info.kpad == len(alg)
    else:
        pytest.importorskip("networkx")
        assert shape == "star" and info.kpad < len(alg)
        _, zeros = morph.max_matching_pairs(A)
        assert info.zero_columns == zeros
        nzc = np.where(np.any(A != 0, axis=0))[0]
        ps = pairset(order)
        assert sorted(v for pr in ps for v in pr if v != ZERO) == sorted(nzc.tolist())
        assert len(ps) == (len(nzc) + zeros) // 2
    dense = morph.decompress_2_4(tb["a_hi"].astype(np.float64) + tb["a_lo"], tb["a_idx"])
    assert morph.satisfies_2_4(dense)
    Ap = morph.apply_permutation(A, list(order))
    if dtype == "bf16_split":
        np.testing.assert_array_equal(dense, Ap)  # three BF16 pieces: exact
    else:
        assert np.max(np.abs(dense - Ap)) <= 2.0 ** -16 * np.max(np.abs(A))


def _emulate_sweep_3d(plan, tb, u, bc, dense):
    """Host emulation of one 3D sweep through the planner's LUT: padded grid -> halo boxes
    (64+2G) x (16+2G) x (16+2G) -> B'' gathered by LUT -> dense A'' @ B'' -> outputs by the
    patch map of the 3D kernel."""
    info = plan.info()
    D, H, W = u.shape
    G, P, bh = info.ghost, info.tile_pitch, info.tile_rows
    bd = 16 + 2 * G
    Wp = (W + 2 * G + 3) // 4 * 4
    up = np.zeros((D + 2 * G, H + 2 * G, Wp))
    zz, yy, xx = np.mgrid[-G:D + G, -G:H + G, -G:W + G]
    if bc == "periodic":
        up[:, :, :W + 2 * G] = u[zz % D, yy % H, xx % W]
    else:
        inside = (zz >= 0) & (zz < D) & (yy >= 0) & (yy < H) & (xx >= 0) & (xx < W)
        up[:, :, :W + 2 * G] = np.where(inside, u[np.clip(zz, 0, D - 1), np.clip(yy, 0, H - 1),
                                                  np.clip(xx, 0, W - 1)], 0.0)
    out = np.full((D, H, W), np.nan)
    lut = tb["lut"]
    for tz in range((D + 15) // 16):
        for ty in range((H + 15) // 16):
            for tx in range((W + 63) // 64):
                tile = np.zeros((bd, bh, P))
                blk = up[tz * 16:tz * 16 + bd, ty * 16:ty * 16 + bh, tx * 64:tx * 64 + P]
                tile[:blk.shape[0], :blk.shape[1], :blk.shape[2]] = blk
                flat = tile.ravel()
                for n in range(128):
                    a, h, b = n >> 4, (n >> 3) & 1, n & 7
                    px, py, pz = ((a & 1) << 2) | (h << 1) | (b & 1), b >> 1, a >> 1
                    base = pz * 4 * bh * P + py * 4 * P + px * 8
                    col = dense @ flat[base + lut]
                    for rho in range(128):
                        z = tz * 16 + pz * 4 + (rho >> 5)
                        y = ty * 16 + py * 4 + ((rho >> 3) & 3)
                        x = tx * 64 + px * 8 + (rho & 7)
                        if z < D and y < H and x < W:
                            out[z, y, x] = col[rho]
    return out


@pytest.mark.parametrize("bc,shape", [("periodic", "box"), ("dirichlet", "star")])
def test_lut_emulation_3d_reproduces_oracle_step(lib, oracle_mod, bc, shape):
    """Bit-level check of the 3D tables the kernel consumes: with dyadic weights and data
    the emulated sweep equals one oracle step exactly."""
    mask = inputs.stencil_mask(shape, 3, 1)
    w = np.where(mask, np.arange(1, 28).reshape(3, 3, 3) / 256.0, 0.0).astype(np.float32)
    u = np.random.default_rng(5).integers(-8, 9, size=(20, 18, 70)).astype(np.float64) / 8.0
    plan = binding.Plan(w, u.shape, dtype="bf16", bc=bc, fusion_depth=1, shape=shape)
    tb = plan.tables()
    dense = morph.decompress_2_4(tb["a_hi"].astype(np.float64) + tb["a_lo"], tb["a_idx"])
    got = _emulate_sweep_3d(plan, tb, u, bc, dense)
    ref = oracle_mod.run(u, w.astype(np.float64), bc, 1)
    np.testing.assert_array_equal(got, ref)


def test_fp64_correction_setting(lib):
    """The FP64 correction step's period is recorded in the plan (0 turns it off) and a
    negative period is rejected."""
    w = inputs.stencil_weights("box", 2, 1, "random", seed=1)
    plan = binding.Plan(w, (256, 256), dtype="bf16_split", bc="periodic", fusion_depth=3)
    assert plan.info().fp64_every == 0
    plan.set_fp64_correction(5)
    assert plan.info().fp64_every == 5
    plan.set_fp64_correction(0)
    assert plan.info().fp64_every == 0
    with pytest.raises(binding.SparStencilError):
        plan.set_fp64_correction(-1)
