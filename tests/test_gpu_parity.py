"""GPU parity: the CUDA path against the FP64 oracle, element by element.

Bars (Eq. 5 read per array; see oracle/check.py): relative L2 <= 1e-6 and
max-abs <= 4e-6 * max(max|X|, max|Y_ref|) for the accepted paths.  Every case
runs through the C ABI on seeded synthetic inputs; batch sizes span several
CTAs and end in a ragged tail.
"""
import numpy as np
import pytest

from paper_2609_28519_gb300 import inputs

pytestmark = pytest.mark.gpu

FUSED_SHAPES = [(h, w) for h in (8, 16, 32) for w in (8, 16, 32)] + [(64, 64)]
RING_SHAPES = [(64, 64), (64, 128), (128, 64), (128, 128)]
SEPARABLE_SHAPES = [(256, 256), (64, 256), (256, 128), (128, 512), (1024, 1024), (2048, 64),
                    (512, 2048), (24, 40), (12, 8), (768, 64)]
KINDS = ["forward", "inverse", "roundtrip"]


def _ref(o, kind, x, norm):
    if kind == "forward":
        return o.forward(x, norm)
    if kind == "inverse":
        return o.inverse(x, norm)
    return x.astype(np.float64)


def _run(plan, kind, x_np, dev):
    import torch
    x = torch.from_numpy(x_np).to(dev)
    y = plan.execute(kind, x)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def _assert_parity(o, y, ref, x, norm, kind, tag):
    m = o.metrics(y, ref, x, output_relative=(norm == 1 and kind != "roundtrip"))
    assert m["nonfinite"] == 0, tag
    assert m["zero_input_violations"] == 0, tag
    assert m["e_rel_max"] <= o.ERR_REL_TOL, (tag, m["e_rel_max"])
    assert m["max_abs_ratio_max"] <= o.MAX_ABS_TOL, (tag, m["max_abs_ratio_max"])
    return m


@pytest.mark.parametrize("h,w", FUSED_SHAPES)
@pytest.mark.parametrize("norm", [0, 1])
def test_fused_shapes_all_kinds(oracle_mod, cuda_dev, h, w, norm):
    from paper_2609_28519_gb300 import Plan
    plan = Plan(h, w, norm=norm, path="fp32")
    assert plan.info().variant == 1
    per_chunk = 16 if (h * w <= 64 or h * w == 256) else (8 if max(h, w) <= 32 else 2)
    batch = 5 * per_chunk + 3  # several chunks and a ragged tail
    x = inputs.uniform(1000 + h * 7 + w, batch, h, w)
    for kind in KINDS:
        y = _run(plan, kind, x, cuda_dev)
        _assert_parity(oracle_mod, y, _ref(oracle_mod, kind, x, norm), x, norm, kind, (h, w, norm, kind))


@pytest.mark.parametrize("h,w", FUSED_SHAPES[:9])
def test_fused_tiled_all_shapes(oracle_mod, cuda_dev, h, w):
    """Image strips for every fused shape: the column pass runs packed column
    pairs for w >= 16 and the row pass packed row pairs where a thread has two
    rows; every block row ends in a partial chunk of tiles, and input and
    output sit in wider buffers (leading dimension > width) whose padding
    must stay untouched."""
    import torch
    from paper_2609_28519_gb300 import Plan
    g = 16 if (h * w <= 64 or (w <= 16 and h * w <= 256)) else 8  # tiles per chunk of a strip
    tpr = 2 * g + 3
    rows, cols = 3 * h, tpr * w
    img = inputs.gaussian(2500 + h + 5 * w, 1, rows, cols)[0]
    blocks = inputs.image_to_blocks(img, h, w)
    src = torch.zeros(rows, cols + 12, device=cuda_dev)
    src[:, :cols] = torch.from_numpy(img).to(cuda_dev)
    plan = Plan(h, w, path="fp32")
    assert plan.info().variant == 1
    for kind in KINDS:
        dst = torch.full((rows, cols + 8), float("nan"), device=cuda_dev)
        plan.execute_tiled(kind, src[:, :cols], dst[:, :cols])
        torch.cuda.synchronize()
        got = inputs.image_to_blocks(dst[:, :cols].cpu().numpy(), h, w)
        _assert_parity(oracle_mod, got, _ref(oracle_mod, kind, blocks, 0), blocks, 0, kind, ("strip", h, w, kind))
        assert torch.isnan(dst[:, cols:]).all(), (h, w, kind)


@pytest.mark.parametrize("h,w,extra", [(8, 8, 3), (8, 16, 6), (16, 8, 3), (16, 16, 6), (32, 8, 6), (32, 16, 3)])
def test_tiled_persistent_many_chunks(oracle_mod, cuda_dev, h, w, extra):
    """Image strips on images of more than 8000 chunks, so that every CTA of
    the persistent ring takes several chunks and every stage's barrier turns
    over more than once; each block row ends in a partial chunk of 3 or 6
    tiles.  Every direction, and the spectral step, against the oracle on
    every block."""
    import torch
    from paper_2609_28519_gb300 import Plan
    g = 16 if (h * w <= 64 or (w <= 16 and h * w <= 256)) else 8  # tiles per chunk of a strip
    tpr = 2 * g + extra
    rows, cols = 2752 * h, tpr * w
    img = inputs.gaussian(2700 + h + 5 * w, 1, rows, cols)[0]
    blocks = inputs.image_to_blocks(img, h, w)
    src = torch.from_numpy(img).to(cuda_dev)
    plan = Plan(h, w, path="fp32")
    assert plan.info().variant == 1
    for kind in KINDS:
        dst = torch.full_like(src, float("nan"))
        plan.execute_tiled(kind, src, dst)
        torch.cuda.synchronize()
        got = inputs.image_to_blocks(dst.cpu().numpy(), h, w)
        _assert_parity(oracle_mod, got, _ref(oracle_mod, kind, blocks, 0), blocks, 0, kind, ("persistent", h, w, kind))
    lam = inputs.poisson_diagonal(h, w)
    plan.set_spectral(lam)
    dst = torch.full_like(src, float("nan"))
    plan.execute_tiled("spectral", src, dst)
    torch.cuda.synchronize()
    got = inputs.image_to_blocks(dst.cpu().numpy(), h, w)
    _assert_spectral(oracle_mod, got, blocks, lam, ("persistent-spectral", h, w))


@pytest.mark.parametrize("h,w,rows,cols", [(16, 16, 2048, 2048), (16, 16, 2048, 1920), (16, 16, 2048, 1840),
                                           (8, 16, 1024, 2048)])
def test_tiled_one_wave_images(oracle_mod, cuda_dev, h, w, rows, cols):
    """Images of 16 x 16 blocks whose strip chunks all fit in one wave of
    one-chunk CTAs but not of the persistent two-stage ones (the 2048^2 image
    is 1024 chunks of 16 tiles; each warp owns four tiles of a chunk): full
    last chunks, 8 tiles (two warps idle) and 3 tiles (one warp with a
    partial quarter), next to a neighbouring shape; every direction, and for
    16 x 16 the spectral step, against the oracle on every block."""
    import torch
    from paper_2609_28519_gb300 import Plan
    img = inputs.ramp_image(2600 + rows + cols + h, rows, cols)
    blocks = inputs.image_to_blocks(img, h, w)
    src = torch.from_numpy(img).to(cuda_dev)
    plan = Plan(h, w, path="fp32")
    for kind in KINDS:
        dst = torch.full_like(src, float("nan"))
        plan.execute_tiled(kind, src, dst)
        torch.cuda.synchronize()
        got = inputs.image_to_blocks(dst.cpu().numpy(), h, w)
        _assert_parity(oracle_mod, got, _ref(oracle_mod, kind, blocks, 0), blocks, 0, kind, ("wave", h, w, rows, cols, kind))
        # in place: each warp reads its whole quarter before it writes it back
        same = src.clone()
        plan.execute_tiled(kind, same, same)
        torch.cuda.synchronize()
        assert torch.equal(same, dst), ("wave in place", h, w, rows, cols, kind)
    if h == w == 16:
        lam = inputs.poisson_diagonal(h, w)
        plan.set_spectral(lam)
        dst = torch.full_like(src, float("nan"))
        plan.execute_tiled("spectral", src, dst)
        torch.cuda.synchronize()
        got = inputs.image_to_blocks(dst.cpu().numpy(), h, w)
        _assert_spectral(oracle_mod, got, blocks, lam, ("wave-spectral", rows, cols))


@pytest.mark.parametrize("h,w", RING_SHAPES)
@pytest.mark.parametrize("norm", [0, 1])
def test_ring_shapes_all_kinds(oracle_mod, cuda_dev, h, w, norm):
    """Sides 64 and 128 (the warp-specialized ring kernels, 128-point lines
    split over two threads): a few arrays, fewer than the CTAs."""
    from paper_2609_28519_gb300 import Plan
    plan = Plan(h, w, norm=norm, path="fp32")
    assert plan.info().variant == 1
    x = inputs.gaussian(1500 + h + 3 * w, 7, h, w)
    for kind in KINDS:
        y = _run(plan, kind, x, cuda_dev)
        _assert_parity(oracle_mod, y, _ref(oracle_mod, kind, x, norm), x, norm, kind, (h, w, norm, kind))


@pytest.mark.parametrize("h,w", RING_SHAPES)
def test_ring_wraparound_replicated(oracle_mod, cuda_dev, h, w):
    """Enough arrays that every CTA goes around its slot ring several times
    (every slot and barrier phase in use), plus a ragged tail: the batch
    repeats 5 distinct arrays, so every copy must give the same bits, and the
    distinct ones must match the oracle."""
    import torch
    from paper_2609_28519_gb300 import Plan
    sms = torch.cuda.get_device_properties(cuda_dev).multi_processor_count
    ring = 12 if (h, w) == (64, 64) else (3 if (h, w) == (128, 128) else 6)
    batch = sms * (3 * ring + 1) + 11
    base = inputs.uniform(1700 + h + w, 5, h, w)
    plan = Plan(h, w, path="fp32")
    x = torch.from_numpy(base).to(cuda_dev).repeat(batch // 5 + 1, 1, 1)[:batch].contiguous()
    for kind in KINDS:
        y = plan.execute(kind, x)
        torch.cuda.synchronize()
        first = y[:5].cpu().numpy()
        _assert_parity(oracle_mod, first, _ref(oracle_mod, kind, base, 0), base, 0, kind, (h, w, kind))
        ref_bits = torch.from_numpy(first).to(cuda_dev)
        idx = torch.arange(batch, device=cuda_dev) % 5
        assert torch.equal(y, ref_bits[idx]), (h, w, kind)
        del y
    del x
    torch.cuda.empty_cache()


@pytest.mark.parametrize("h,w", SEPARABLE_SHAPES)
@pytest.mark.parametrize("norm", [0, 1])
def test_separable_shapes(oracle_mod, cuda_dev, h, w, norm):
    """Shapes beyond the fused kernels: FFT line passes for power-of-two sides
    64..2048, dense passes otherwise."""
    from paper_2609_28519_gb300 import Plan
    plan = Plan(h, w, norm=norm, path="fp32")
    assert plan.info().variant == 2
    batch = 3 if h * w <= 65536 else 2
    x = inputs.gaussian(2000 + h + w, batch, h, w)
    for kind in KINDS:
        y = _run(plan, kind, x, cuda_dev)
        _assert_parity(oracle_mod, y, _ref(oracle_mod, kind, x, norm), x, norm, kind, (h, w, norm, kind))


SMALL_DENSE_SHAPES = [(26, 32), (24, 40), (40, 24), (1, 4), (5, 8), (3, 12), (12, 12), (20, 20), (36, 60),
                      (48, 48), (60, 60), (64, 24), (24, 64), (63, 64)]


@pytest.mark.parametrize("h,w", SMALL_DENSE_SHAPES)
@pytest.mark.parametrize("norm", [0, 1])
def test_small_dense_shapes(oracle_mod, cuda_dev, h, w, norm):
    """Sides up to 64 without a fused kernel (non-power-of-two sides, the
    paper's 26 among them): the dense operators applied in shared memory, one
    read and one write, no workspace; batches large enough for several
    iterations per CTA (26 x 32, 60 x 60) and a ragged last group."""
    from paper_2609_28519_gb300 import Plan
    plan = Plan(h, w, norm=norm, path="fp32")
    info = plan.info()
    assert info.variant == 2 and info.workspace_bytes == 0
    batch = min(5000, max(7, 2_000_000 // (h * w))) + 3
    x = inputs.gaussian(8100 + 7 * h + w + norm, batch, h, w)
    for kind in KINDS:
        y = _run(plan, kind, x, cuda_dev)
        _assert_parity(oracle_mod, y, _ref(oracle_mod, kind, x, norm), x, norm, kind, ("small", h, w, norm, kind))


@pytest.mark.parametrize("h,w,path,batch", [(8, 8, "fp32", 3001), (16, 16, "fp32", 3001), (32, 16, "fp32", 1201),
                                            (64, 64, "fp32", 701), (128, 128, "fp32", 331), (256, 256, "fp32", 41),
                                            (100, 100, "fp32", 61), (16, 16, "split_tc", 2001),
                                            (32, 32, "split_tc", 1201), (8, 8, "split_tc", 3001),
                                            (256, 128, "split_tc", 41)])
def test_nonfinite_arrays_stay_apart_all_routes(oracle_mod, cuda_dev, h, w, path, batch):
    """Every route: arrays holding inf or NaN give non-finite results of
    their own, and every other array of the batch stays exact (forward and
    round trip), over batches that take several chunks, tiles or slots per
    CTA."""
    from paper_2609_28519_gb300 import Plan
    x = inputs.gaussian(8400 + h + w + len(path), batch, h, w)
    bad = np.arange(0, batch, 13)
    x[bad, h // 2, w // 3] = np.inf
    x[bad[1::2], h - 1, 0] = np.nan
    good = np.setdiff1d(np.arange(batch), bad)
    plan = Plan(h, w, path=path)
    for kind in ("forward", "roundtrip"):
        y = _run(plan, kind, x, cuda_dev)
        _assert_parity(oracle_mod, y[good], _ref(oracle_mod, kind, x[good], 0), x[good], 0, kind,
                       ("nonfinite-apart", h, w, path, kind))


def test_small_dense_nonfinite_arrays_stay_apart(oracle_mod, cuda_dev):
    """A non-finite value in some arrays of a batch (26 rows: two zero
    padding rows in shared memory) leaves every other array exact, through
    the several groups each CTA transforms in turn with the same buffers."""
    import torch
    from paper_2609_28519_gb300 import Plan
    h, w = 26, 32
    x = inputs.gaussian(8300, 6001, h, w)
    bad = np.arange(0, 6001, 97)
    x[bad, 3, 5] = np.inf
    x[bad[1::2], 7, 9] = np.nan
    plan = Plan(h, w)
    good = np.setdiff1d(np.arange(6001), bad)
    for kind in KINDS:
        y = _run(plan, kind, x, cuda_dev)
        _assert_parity(oracle_mod, y[good], _ref(oracle_mod, kind, x[good], 0), x[good], 0, kind,
                       ("small-nonfinite", kind))


def test_small_dense_inplace_and_tiles(oracle_mod, cuda_dev):
    """The on-chip dense route in place, on image tiles (leading dimensions
    wider than the image, the margin untouched) and with range protection on
    tiles."""
    import ctypes
    import torch
    from paper_2609_28519_gb300 import Plan, native
    h, w = 24, 40
    plan = Plan(h, w)
    x = inputs.uniform(8200, 333, h, w)
    d = torch.from_numpy(x).to(cuda_dev)
    plan.execute("forward", d, d)
    torch.cuda.synchronize()
    _assert_parity(oracle_mod, d.cpu().numpy(), oracle_mod.forward(x, 0), x, 0, "forward", "small-inplace")
    rows, cols = h * 20, w * 12
    img = inputs.ramp_image(8201, rows, cols)
    ld = cols + 36
    src = torch.zeros(rows, ld, device=cuda_dev)
    src[:, :cols] = torch.from_numpy(img).to(cuda_dev)
    dst = torch.full_like(src, float("nan"))
    L = native.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    blocks = inputs.image_to_blocks(img, h, w)
    for kind, code, ref in (("forward", 1, oracle_mod.forward(blocks, 0)), ("inverse", 2, oracle_mod.inverse(blocks, 0))):
        st = L.bdct_execute_tiled(plan.handle, code, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                                  rows, cols, ld, ld, stream)
        assert st == 0
        torch.cuda.synchronize()
        assert torch.isnan(dst[:, cols:]).all()  # the margin beyond the image is untouched
        got = inputs.image_to_blocks(dst[:, :cols].cpu().numpy(), h, w)
        _assert_parity(oracle_mod, got, ref, blocks, 0, kind, ("small-tiled", kind))
    plan.set_range_protection(True)
    big = (img * np.float32(1e35)).astype(np.float32)
    src[:, :cols] = torch.from_numpy(big).to(cuda_dev)
    st = L.bdct_execute_tiled(plan.handle, 1, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                              rows, cols, ld, ld, stream)
    assert st == 0
    torch.cuda.synchronize()
    bb = inputs.image_to_blocks(big, h, w)
    got = inputs.image_to_blocks(dst[:, :cols].cpu().numpy(), h, w)
    _assert_parity(oracle_mod, got, oracle_mod.forward(bb, 0), bb, 0, "forward", "small-tiled-protected")


def test_paper_input_categories(oracle_mod, cuda_dev):
    """Section 6 categories: impulses, cosine modes, cancellation, neighbouring
    floats, weak perturbations, amplitudes 2^-100..2^90, constant, zero."""
    from paper_2609_28519_gb300 import Plan
    for n in (8, 16, 32):
        x = inputs.paper_categories(31, n)
        plan = Plan(n, n, path="fp32")
        for kind in KINDS:
            y = _run(plan, kind, x, cuda_dev)
            _assert_parity(oracle_mod, y, _ref(oracle_mod, kind, x, 0), x, 0, kind, (n, kind))


def test_config_8x8_batch_1024(oracle_mod, cuda_dev):
    """1024 row-major 8x8 blocks, uniform[-1,1], seed 1: F, I and RT."""
    from paper_2609_28519_gb300 import Plan
    x = inputs.uniform(1, 1024, 8, 8)
    plan = Plan(8, 8)
    for kind in KINDS:
        y = _run(plan, kind, x, cuda_dev)
        m = _assert_parity(oracle_mod, y, _ref(oracle_mod, kind, x, 0), x, 0, kind, kind)
        # FP32 error magnitude in line with the paper's Table 3 (1.37e-7 at 8x8)
        assert m["e_rel_max"] < 10 * 1.37e-7


def test_config_image_16x16_tiles(oracle_mod, cuda_dev):
    """2048x2048 image (N(0,1) + 0.01(i+j), seed 2) cut into 16384 16x16
    blocks: forward then inverse per block, through the tiled view and as a
    contiguous batch; fused round trip as well."""
    import torch
    from paper_2609_28519_gb300 import Plan
    img = inputs.ramp_image(2)
    blocks = inputs.image_to_blocks(img, 16, 16)
    plan = Plan(16, 16)
    dimg = torch.from_numpy(img).to(cuda_dev)
    spec = plan.execute_tiled("forward", dimg)
    back = plan.execute_tiled("inverse", spec)
    rt = plan.execute_tiled("roundtrip", dimg)
    torch.cuda.synchronize()
    spec_b = inputs.image_to_blocks(spec.cpu().numpy(), 16, 16)
    ref = oracle_mod.forward(blocks, 0)
    _assert_parity(oracle_mod, spec_b, ref, blocks, 0, "forward", "tiled-forward")
    back_b = inputs.image_to_blocks(back.cpu().numpy(), 16, 16)
    # inverse compared with the oracle inverse of the GPU spectrum
    ref_i = oracle_mod.inverse(spec_b, 0)
    _assert_parity(oracle_mod, back_b, ref_i, spec_b, 0, "inverse", "tiled-inverse")
    # forward then inverse returns the image within two FP32 transforms
    _assert_parity(oracle_mod, back_b, blocks.astype(np.float64), blocks, 0, "roundtrip", "f-then-i")
    rt_b = inputs.image_to_blocks(rt.cpu().numpy(), 16, 16)
    _assert_parity(oracle_mod, rt_b, blocks.astype(np.float64), blocks, 0, "roundtrip", "tiled-rt")
    # the contiguous batch (scalar cores) and the tiled view (packed cores for
    # the column pass) agree up to rounding order (Section 2.1)
    db = torch.from_numpy(blocks).to(cuda_dev)
    spec2 = plan.forward(db).cpu().numpy()
    _assert_parity(oracle_mod, spec2, ref, blocks, 0, "forward", "contiguous-forward")
    scale = np.maximum(np.abs(blocks).max(axis=(1, 2), keepdims=True),
                       np.abs(spec_b).max(axis=(1, 2), keepdims=True))
    assert np.all(np.abs(spec2.astype(np.float64) - spec_b) <= 4e-6 * scale)


@pytest.mark.parametrize("n", [8, 16, 32, 64, 128, 256])
def test_sweep_full_size_sampled(oracle_mod, cuda_dev, n):
    """Square sweep at full size (>= 512 MiB of input per run), three
    distributions, outputs checked on sampled arrays."""
    import torch
    from paper_2609_28519_gb300 import Plan
    batch = (512 << 20) // (4 * n * n)
    plan = Plan(n, n)
    rng = np.random.default_rng(n)
    x = torch.empty((batch, n, n), dtype=torch.float32, device=cuda_dev)
    x.uniform_(-1.0, 1.0, generator=torch.Generator(device=cuda_dev).manual_seed(3000 + n))
    y = torch.empty_like(x)
    for kind in KINDS:
        plan.execute(kind, x, y)
        torch.cuda.synchronize()
        idx = np.sort(rng.choice(batch, size=min(batch, 48 if n <= 64 else 12), replace=False))
        idx[-1] = batch - 1  # always include the last array (tail of the grid)
        xs = x[idx].cpu().numpy()
        ys = y[idx].cpu().numpy()
        _assert_parity(oracle_mod, ys, _ref(oracle_mod, kind, xs, 0), xs, 0, kind, (n, kind))
    del x, y
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n", [8, 16, 32, 64, 128, 256])
def test_sweep_distributions(oracle_mod, cuda_dev, n):
    """Extreme amplitudes (+-1e30 mixed with +-1e-30) and a weak 1e-6 cosine on
    a unit cosine: accepted by the global bars; the weak coefficient's own
    relative error is reported (Section 6: weak components can hide)."""
    from paper_2609_28519_gb300 import Plan
    plan = Plan(n, n)
    b = 16 if n <= 64 else 4
    xe = inputs.extreme(40 + n, b, n, n)
    for kind in KINDS:
        y = _run(plan, kind, xe, cuda_dev)
        _assert_parity(oracle_mod, y, _ref(oracle_mod, kind, xe, 0), xe, 0, kind, ("extreme", n, kind))
    xw, modes = inputs.weak_cosine(50 + n, b, n)
    y = _run(plan, "forward", xw, cuda_dev)
    ref = oracle_mod.forward(xw, 0)
    _assert_parity(oracle_mod, y, ref, xw, 0, "forward", ("weak", n))
    k2, l2 = modes[:, 2], modes[:, 3]
    weak_ref = ref[np.arange(b), k2, l2]
    weak_got = y[np.arange(b), k2, l2]
    weak_rel = np.abs(weak_got - weak_ref) / np.abs(weak_ref)
    assert np.all(np.isfinite(weak_rel))  # reported, not accepted


@pytest.mark.parametrize("h,w", RING_SHAPES)
def test_ring_tiled_image(oracle_mod, cuda_dev, h, w):
    """Blocks of a 1024x512 image read and written in place in the image
    (one bulk copy per block row), all three directions."""
    import torch
    from paper_2609_28519_gb300 import Plan
    img = inputs.ramp_image(9, 1024, 512)
    blocks = inputs.image_to_blocks(img, h, w)
    plan = Plan(h, w)
    d = torch.from_numpy(img).to(cuda_dev)
    for kind in KINDS:
        out = plan.execute_tiled(kind, d)
        torch.cuda.synchronize()
        got = inputs.image_to_blocks(out.cpu().numpy(), h, w)
        _assert_parity(oracle_mod, got, _ref(oracle_mod, kind, blocks, 0), blocks, 0, kind, ("tiled", h, w, kind))


def test_graph_capture_equals_direct_calls(cuda_dev):
    """Calls captured by the user into a CUDA graph and replayed give the same
    bits as the same calls made directly: the one-wave image route, a
    persistent fused batch, the ring kernel and the two-pass line engine
    (workspace reused inside the graph)."""
    import torch
    from paper_2609_28519_gb300 import Plan
    img = torch.from_numpy(inputs.ramp_image(31, 2048, 2048)).to(cuda_dev)
    cases = [(Plan(16, 16, path="fp32"), "tiled", img)]
    for (h, w, b) in [(16, 16, 4096), (64, 64, 300), (256, 256, 40)]:
        cases.append((Plan(h, w, path="fp32"), "batch", torch.from_numpy(inputs.uniform(32 + h, b, h, w)).to(cuda_dev)))
    for plan, mode, x in cases:
        for kind in KINDS:
            direct = torch.empty_like(x)
            replayed = torch.full_like(x, float("nan"))
            call = (lambda o, st=None: plan.execute_tiled(kind, x, o, st)) if mode == "tiled" else \
                   (lambda o, st=None: plan.execute(kind, x, o, st))
            call(direct)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            cs = torch.cuda.Stream(cuda_dev)
            cs.wait_stream(torch.cuda.current_stream(cuda_dev))
            with torch.cuda.graph(g, stream=cs):
                call(replayed, cs)
            g.replay()
            torch.cuda.synchronize()
            assert torch.equal(direct, replayed), (mode, tuple(x.shape), kind)


def test_inplace_and_tail_and_guards(oracle_mod, cuda_dev):
    import torch
    from paper_2609_28519_gb300 import Plan
    plan = Plan(16, 16)
    x_np = inputs.uniform(77, 37, 16, 16)
    ref = oracle_mod.forward(x_np, 0)
    # guard bands around the output and an unchanged input (Section 6)
    guard = 1024
    buf = torch.full((guard + 37 * 256 + guard,), 12345.0, device=cuda_dev)
    out = buf[guard:guard + 37 * 256].view(37, 16, 16)
    x = torch.from_numpy(x_np).to(cuda_dev)
    x_before = x.clone()
    plan.forward(x, out)
    torch.cuda.synchronize()
    assert torch.equal(x, x_before)
    assert torch.all(buf[:guard] == 12345.0) and torch.all(buf[-guard:] == 12345.0)
    _assert_parity(oracle_mod, out.cpu().numpy(), ref, x_np, 0, "forward", "guarded")
    # exact in-place
    plan.forward(x, x)
    torch.cuda.synchronize()
    assert np.array_equal(x.cpu().numpy(), out.cpu().numpy())


@pytest.mark.parametrize("h,w,path", [(64, 64, "auto"), (128, 128, "auto"), (64, 128, "auto"), (256, 256, "auto"),
                                      (768, 64, "auto"), (16, 16, "split_tc"), (32, 32, "split_tc"),
                                      (64, 64, "split_tc")])
def test_exact_inplace_large_sides(oracle_mod, cuda_dev, h, w, path):
    """in == out on the ring kernels (TMA copies read and write the same
    arrays), on the line and dense routes (through the plan workspace) and on
    the tensor-core route (each tile written only after its rows were read):
    the result equals the out-of-place one bit for bit and matches the
    oracle."""
    import torch
    from paper_2609_28519_gb300 import Plan
    plan = Plan(h, w, path=path)
    x_np = inputs.uniform(88 + h + w, 9, h, w)
    x = torch.from_numpy(x_np).to(cuda_dev)
    for kind in KINDS:
        ref_gpu = plan.execute(kind, x)
        y = x.clone()
        plan.execute(kind, y, y)
        torch.cuda.synchronize()
        assert torch.equal(y, ref_gpu), (h, w, kind)
        _assert_parity(oracle_mod, y.cpu().numpy(), _ref(oracle_mod, kind, x_np, 0), x_np, 0, kind, ("inplace", h, w, kind))


def test_argument_errors_on_device(cuda_dev):
    import torch
    from paper_2609_28519_gb300 import Plan, BdctError, native
    plan = Plan(16, 16, kind=native.FORWARD)
    x = torch.zeros(4, 16, 16, device=cuda_dev)
    with pytest.raises(BdctError) as e:
        plan.inverse(x)
    assert e.value.code == "ERR_KIND"
    buf = torch.zeros(8 * 256 + 4, device=cuda_dev)
    with pytest.raises(BdctError) as e:
        plan.forward(buf[1:1 + 4 * 256].view(4, 16, 16), buf[:4 * 256].view(4, 16, 16))
    assert e.value.code in ("ERR_ALIGN", "ERR_ALIAS")
    with pytest.raises(BdctError) as e:
        plan.forward(buf[4:4 + 4 * 256].view(4, 16, 16), buf[:4 * 256].view(4, 16, 16))
    assert e.value.code == "ERR_ALIAS"
    # batch 0 is a no-op
    L = native.lib()
    assert L.bdct_execute(plan.handle, 1, None, None, 0, None) == 0
    with pytest.raises(BdctError):
        Plan(16, 12, path="bf16")


def test_bounded_wait_gives_up_with_status(cuda_dev):
    """A wait on a barrier nothing completes gives up after its limit, records
    BDCT_ERR_DEVICE_TIMEOUT and leaves the context usable."""
    import torch
    from paper_2609_28519_gb300 import Plan, native
    L = native.lib()
    assert L.bdct_selftest_wait_timeout(20000) == 8
    # the context still works afterwards
    plan = Plan(8, 8)
    x = torch.ones(4, 8, 8, device=cuda_dev)
    y = plan.forward(x)
    torch.cuda.synchronize()
    assert abs(float(y[0, 0, 0]) - 8.0) < 1e-5
    assert plan.device_status() == 0


# ------------------------------------------------------------ tensor-core route
@pytest.mark.parametrize("n", [16, 32, 64])
@pytest.mark.parametrize("norm", [0, 1])
def test_split_tc_accepted(oracle_mod, cuda_dev, n, norm):
    """Split-BF16 tcgen05 route, three terms / six products: accepted bars."""
    from paper_2609_28519_gb300 import Plan
    plan = Plan(n, n, norm=norm, path="split_tc")
    assert plan.info().variant == 3
    per_tile = 128 // n
    batch = 7 * per_tile + 1  # several tiles and a ragged tail
    x = inputs.uniform(4000 + n + norm, batch, n, n)
    for kind in KINDS:
        y = _run(plan, kind, x, cuda_dev)
        _assert_parity(oracle_mod, y, _ref(oracle_mod, kind, x, norm), x, norm, kind, ("tc", n, norm, kind))
    assert plan.device_status() == 0


@pytest.mark.parametrize("n", [16, 64])
def test_split_tc_report_only_variants(oracle_mod, cuda_dev, n):
    """hi/lo (2 terms, 3 products) and single BF16: reported, not accepted.
    Their errors must sit where the term count puts them."""
    from paper_2609_28519_gb300 import Plan
    x = inputs.uniform(4100 + n, 16, n, n)
    ref = oracle_mod.forward(x, 0)
    errs = {}
    for path in ("split_hilo", "bf16"):
        y = _run(Plan(n, n, path=path), "forward", x, cuda_dev)
        errs[path] = oracle_mod.metrics(y, ref, x)["e_rel_max"]
    assert 1e-7 < errs["split_hilo"] < 1e-4
    assert 1e-4 < errs["bf16"] < 3e-2


def test_split_tc_image_tiles(oracle_mod, cuda_dev):
    """The 2048x2048 image as 16x16 blocks through the tensor-core route."""
    import torch
    from paper_2609_28519_gb300 import Plan
    img = inputs.ramp_image(2)
    blocks = inputs.image_to_blocks(img, 16, 16)
    plan = Plan(16, 16, path="split_tc")
    dimg = torch.from_numpy(img).to(cuda_dev)
    spec = plan.execute_tiled("forward", dimg)
    back = plan.execute_tiled("inverse", spec)
    torch.cuda.synchronize()
    spec_b = inputs.image_to_blocks(spec.cpu().numpy(), 16, 16)
    _assert_parity(oracle_mod, spec_b, oracle_mod.forward(blocks, 0), blocks, 0, "forward", "tc-tiled")
    back_b = inputs.image_to_blocks(back.cpu().numpy(), 16, 16)
    _assert_parity(oracle_mod, back_b, blocks.astype(np.float64), blocks, 0, "roundtrip", "tc-f-then-i")


def test_auto_path_choice(cuda_dev):
    from paper_2609_28519_gb300 import Plan
    assert Plan(64, 64).info().variant == 1
    assert Plan(16, 16).info().variant == 1
    assert Plan(128, 128).info().variant == 1
    assert Plan(64, 128).info().variant == 1
    assert Plan(256, 256).info().variant == 2
    assert Plan(64, 64, path="split_tc").info().variant == 3


# ------------------------------------------------------------ ragged batches
def _ragged_inputs(shapes, seed):
    import numpy as np
    arrs = [inputs.uniform(seed + i, 1, r, c)[0] for i, (r, c) in enumerate(shapes)]
    return arrs


def _pack(rg, arrs, dev):
    import torch
    flat = torch.zeros(rg.total, dtype=torch.float32)
    for a, off in zip(arrs, rg.in_off):
        flat[int(off):int(off) + a.size] = torch.from_numpy(a.ravel())
    return flat.to(dev)


def _unpack(rg, flat, shapes):
    f = flat.cpu().numpy()
    return [f[int(o):int(o) + r * c].reshape(r, c) for o, (r, c) in zip(rg.out_off, shapes)]


def test_ragged_mixed_shapes_against_oracle(oracle_mod, cuda_dev):
    """Mixed squares and rectangles in one ragged execution: every array
    against the oracle; ragged output bit-equal to per-array plan calls on the
    same path; graph replay equal to the captured first call."""
    import torch
    from paper_2609_28519_gb300 import Plan, Ragged
    rng = np.random.default_rng(44)
    base = [(8, 8), (16, 16), (32, 32), (64, 64), (128, 128), (256, 256), (64, 256), (128, 512), (16, 8),
            (32, 16), (24, 40)]
    shapes = [base[int(i)] for i in rng.integers(0, len(base), size=40)] + [(768, 1024)]
    arrs = _ragged_inputs(shapes, 500)
    rg = Ragged(shapes)
    classes = rg.classes()
    assert sum(c["count"] for c in classes) == len(shapes)
    x = _pack(rg, arrs, cuda_dev)
    for kind in ("forward", "inverse", "roundtrip"):
        y = torch.full_like(x, float("nan"))
        rg.execute(kind, x, y)
        torch.cuda.synchronize()
        first = y.clone()
        rg.execute(kind, x, y)  # graph replay
        torch.cuda.synchronize()
        assert torch.equal(first, y)
        outs = _unpack(rg, y, shapes)
        for a, o, (r, c) in zip(arrs, outs, shapes):
            ref = _ref(oracle_mod, kind, a[None], 0)[0]
            _assert_parity(oracle_mod, o[None], ref[None], a[None], 0, kind, ("ragged", r, c, kind))
        # the same path through a per-array plan gives the same bits
        by_shape = {(c["rows"], c["cols"]): c["path"] for c in classes}
        for i in (0, len(shapes) - 1):
            r, c = shapes[i]
            pl = Plan(r, c, path={1: "fp32", 2: "split_tc"}[by_shape[(r, c)]])
            single = pl.execute(kind, torch.from_numpy(arrs[i][None]).to(cuda_dev))
            torch.cuda.synchronize()
            assert np.array_equal(single.cpu().numpy()[0], outs[i])


def test_ragged_full_workload_sampled(oracle_mod, cuda_dev):
    """4096 arrays drawn by seed from the nine shapes (~1.6 GiB), forward and
    inverse in one graph launch each; sampled arrays against the oracle."""
    import torch
    from paper_2609_28519_gb300 import Ragged
    shapes = inputs.ragged_shapes(4, 4096)
    rg = Ragged(shapes, kind=1 | 2)
    x = torch.empty(rg.total, dtype=torch.float32, device=cuda_dev)
    x.uniform_(-1.0, 1.0, generator=torch.Generator(device=cuda_dev).manual_seed(4))
    y = torch.empty_like(x)
    rng = np.random.default_rng(4)
    pick = rng.choice(len(shapes), 10, replace=False)
    for kind in ("forward", "inverse"):
        rg.execute(kind, x, y)
        torch.cuda.synchronize()
        for i in pick:
            r, c = shapes[i]
            o = int(rg.in_off[i])
            a = x[o:o + r * c].view(1, r, c).cpu().numpy()
            got = y[o:o + r * c].view(1, r, c).cpu().numpy()
            _assert_parity(oracle_mod, got, _ref(oracle_mod, kind, a, 0), a, 0, kind, ("ragged-full", r, c, kind))


# ------------------------------------------------------------ host-buffer execution
def test_host_buffers_tiled_and_batch(oracle_mod, cuda_dev):
    """bdct_execute_tiled_host / bdct_execute_host: host in, directions applied
    on the device in order, host out; equal to the device-buffer calls."""
    import torch
    from paper_2609_28519_gb300 import Plan
    img = inputs.ramp_image(2, 1024, 2048)
    plan = Plan(16, 16)
    plan.set_host_staging(1 << 20)  # several chunks, so the pipeline overlaps and wraps
    h_in = torch.from_numpy(img).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    plan.execute_tiled_host(["forward"], h_in, h_out)
    torch.cuda.synchronize()
    d = torch.from_numpy(img).to(cuda_dev)
    ref = plan.execute_tiled("forward", d)
    torch.cuda.synchronize()
    assert np.array_equal(h_out.numpy(), ref.cpu().numpy())
    plan.execute_tiled_host(["forward", "inverse"], h_in, h_out)
    torch.cuda.synchronize()
    blocks = inputs.image_to_blocks(img, 16, 16)
    back = inputs.image_to_blocks(h_out.numpy(), 16, 16)
    _assert_parity(oracle_mod, back, blocks.astype(np.float64), blocks, 0, "roundtrip", "host-f-then-i")
    # contiguous batch, several chunks and a ragged tail
    x = inputs.uniform(77, 1000, 32, 32)
    p32 = Plan(32, 32)
    p32.set_host_staging(64 * 32 * 32 * 4)
    hx = torch.from_numpy(x).pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    p32.execute_host(["forward"], hx, hy)
    torch.cuda.synchronize()
    _assert_parity(oracle_mod, hy.numpy(), oracle_mod.forward(x, 0), x, 0, "forward", "host-batch")


# ------------------------------------------------------------ large whole arrays
@pytest.mark.parametrize("h,w", [(1024, 768), (768, 1024), (768, 768)])
def test_large_non_power_of_two_against_oracle(oracle_mod, cuda_dev, h, w):
    """768-point lines (radix-3 FFT stage) against the full oracle."""
    from paper_2609_28519_gb300 import Plan
    plan = Plan(h, w)
    assert plan.info().variant == 2
    x = inputs.gaussian(6000 + h + w, 1, h, w)
    for kind in KINDS:
        y = _run(plan, kind, x, cuda_dev)
        _assert_parity(oracle_mod, y, _ref(oracle_mod, kind, x, 0), x, 0, kind, (h, w, kind))


@pytest.mark.parametrize("n", [2048, 4096])
def test_large_full_rank_against_oracle(oracle_mod, cuda_dev, n):
    """Whole n x n Gaussian arrays (the 4096^2 arrays of the large-array
    workload, and 2048^2): forward against the oracle's forward of X, inverse
    against the oracle's inverse of the same X read as a spectrum, round trip
    against X itself -- every element, at the accepted bars.  The oracle
    shares each array between the host threads (a few seconds per
    direction)."""
    from paper_2609_28519_gb300 import Plan
    plan = Plan(n, n)
    assert plan.info().variant == 2
    x = inputs.gaussian(5000 + n, 1, n, n)
    for kind in KINDS:
        y = _run(plan, kind, x, cuda_dev)
        _assert_parity(oracle_mod, y, _ref(oracle_mod, kind, x, 0), x, 0, kind, ("large", n, kind))


# ------------------------------------------------------------ spectral operator (Prop. 1, Eq. 4)
def _assert_spectral(o, y, x, lam, tag):
    """Eq. 5 read for the composition U^T Lambda U: the error relative to
    max|Lambda| times the input, i.e. the transform bars applied to
    U^T (Lambda / max|Lambda|) U (Lambda = 1 gives the round-trip check)."""
    s = float(np.max(np.abs(lam)))
    return _assert_parity(o, np.asarray(y, np.float64) / s, o.spectral(x, lam) / s, x, 0, "roundtrip", tag)


SPECTRAL_CASES = [(h, w, "fp32") for (h, w) in FUSED_SHAPES[:9]] + [
    (64, 64, "fp32"), (128, 128, "fp32"), (64, 128, "fp32"), (16, 16, "split_tc"), (32, 32, "split_tc"),
    (64, 64, "split_tc"), (256, 256, "fp32"), (64, 256, "fp32"), (24, 40, "fp32"), (40, 100, "fp32")]


@pytest.mark.parametrize("h,w,path", SPECTRAL_CASES)
@pytest.mark.parametrize("norm", [0, 1])
def test_spectral_against_oracle(oracle_mod, cuda_dev, h, w, path, norm):
    """Transform -- diagonal -- inverse: fused in one pass (sides 8..32, tensor
    cores), composed from forward, diagonal and inverse elsewhere; a seeded
    diagonal and the Poisson diagonal, several chunks and a ragged tail.  The
    composition is the normalized one under both plan normalizations."""
    from paper_2609_28519_gb300 import Plan
    plan = Plan(h, w, norm=norm, path=path)
    batch = 37 if h * w <= 4096 else 5
    x = inputs.uniform(7000 + h + 3 * w + norm, batch, h, w)
    for lam in (inputs.random_diagonal(7100 + h + w, h, w, -2.0, 3.0), inputs.poisson_diagonal(h, w)):
        plan.set_spectral(lam)
        y = _run(plan, "spectral", x, cuda_dev)
        _assert_spectral(oracle_mod, y, x, lam, ("spectral", h, w, path, norm))
    # Lambda = 1 is the round trip
    plan.set_spectral(np.ones((h, w)))
    y = _run(plan, "spectral", x, cuda_dev)
    _assert_parity(oracle_mod, y, x.astype(np.float64), x, 0, "roundtrip", ("spectral-identity", h, w, path))


@pytest.mark.parametrize("path", ["fp32", "split_tc"])
def test_spectral_image_16x16_poisson(oracle_mod, cuda_dev, path):
    """The 2048x2048 image as 16384 16x16 blocks, each solved with the
    Poisson diagonal (the phase-unwrapping block step, Section 1.1) through
    the tiled view in one call; in place as well; every block against the
    oracle."""
    import torch
    from paper_2609_28519_gb300 import Plan
    img = inputs.ramp_image(2)
    blocks = inputs.image_to_blocks(img, 16, 16)
    lam = inputs.poisson_diagonal(16, 16)
    plan = Plan(16, 16, path=path)
    plan.set_spectral(lam)
    d = torch.from_numpy(img).to(cuda_dev)
    out = plan.execute_tiled("spectral", d)
    torch.cuda.synchronize()
    got = inputs.image_to_blocks(out.cpu().numpy(), 16, 16)
    _assert_spectral(oracle_mod, got, blocks, lam, ("spectral-image", path))
    d2 = d.clone()
    plan.execute_tiled("spectral", d2, d2)
    torch.cuda.synchronize()
    assert torch.equal(d2, out)


def test_spectral_host_buffers_and_errors(oracle_mod, cuda_dev):
    import torch
    from paper_2609_28519_gb300 import BdctError, Plan, native
    # host image through the tiled host pipeline: spectral step on the device
    img = inputs.ramp_image(3, 512, 1024)
    plan = Plan(16, 16)
    lam = inputs.poisson_diagonal(16, 16)
    plan.set_spectral(lam)
    plan.set_host_staging(1 << 19)
    h_in = torch.from_numpy(img).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    plan.execute_tiled_host(["spectral"], h_in, h_out)
    torch.cuda.synchronize()
    blocks = inputs.image_to_blocks(img, 16, 16)
    _assert_spectral(oracle_mod, inputs.image_to_blocks(h_out.numpy(), 16, 16), blocks, lam, "spectral-host")
    # a plan without the spectral direction, and a diagonal never set
    x = torch.zeros(2, 16, 16, device=cuda_dev)
    p_f = Plan(16, 16, kind=native.FORWARD)
    with pytest.raises(BdctError) as e:
        p_f.set_spectral(lam)
    assert e.value.code == "ERR_KIND"
    with pytest.raises(BdctError) as e:
        p_f.spectral(x)
    assert e.value.code == "ERR_KIND"
    with pytest.raises(BdctError) as e:
        Plan(16, 16).spectral(x)
    assert e.value.code == "ERR_INVALID_ARG"


# ------------------------------------------------------------ tensor-core separable passes
TG_SHAPES = [(8, 8), (128, 128), (256, 256), (16, 64), (64, 16), (32, 128), (128, 32), (64, 256), (192, 320),
             (128, 512)]


@pytest.mark.parametrize("h,w", TG_SHAPES)
@pytest.mark.parametrize("norm", [0, 1])
def test_split_tc_passes_against_oracle(oracle_mod, cuda_dev, h, w, norm):
    """Split-BF16 tcgen05 passes (three terms, six products, two TMEM
    accumulators): squares beyond 64, rectangles, multiples of 64 that are
    not powers of two, and 8 x 8 as one Kronecker product.  Forward, inverse,
    round trip and the spectral direction against the oracle; several row
    tiles and a ragged tail."""
    from paper_2609_28519_gb300 import Plan
    plan = Plan(h, w, norm=norm, path="split_tc")
    assert plan.info().variant == 4
    batch = 300 if h * w <= 64 else (5 if h * w <= 65536 else 2)
    x = inputs.uniform(8000 + h + 7 * w + norm, batch, h, w)
    for kind in KINDS:
        y = _run(plan, kind, x, cuda_dev)
        _assert_parity(oracle_mod, y, _ref(oracle_mod, kind, x, norm), x, norm, kind, ("tg", h, w, norm, kind))
    lam = inputs.poisson_diagonal(h, w)
    plan.set_spectral(lam)
    _assert_spectral(oracle_mod, _run(plan, "spectral", x, cuda_dev), x, lam, ("tg-spectral", h, w))
    assert plan.device_status() == 0


@pytest.mark.parametrize("h,w,b", [(1024, 1024, 2), (4096, 4096, 1), (1024, 768, 1), (768, 1024, 1)])
def test_split_tc_large_arrays_against_oracle(oracle_mod, cuda_dev, h, w, b):
    """The large-array shapes (1024^2, 4096^2, 1024 x 768) on the split-BF16
    tensor-core passes, full-rank Gaussian inputs: forward, inverse and
    round trip against the oracle at the accepted bars."""
    from paper_2609_28519_gb300 import Plan
    plan = Plan(h, w, kind=1 | 2 | 4, path="split_tc")
    assert plan.info().variant == 4
    x = inputs.gaussian(8500 + h + w, b, h, w)
    for kind in KINDS:
        y = _run(plan, kind, x, cuda_dev)
        _assert_parity(oracle_mod, y, _ref(oracle_mod, kind, x, 0), x, 0, kind, ("tg-large", h, w, kind))


def test_split_tc_passes_inplace_report_only_and_ragged(oracle_mod, cuda_dev):
    import torch
    from paper_2609_28519_gb300 import Plan, Ragged
    # exact in place, Kronecker and two-pass routes
    for (h, w) in [(8, 8), (128, 64)]:
        plan = Plan(h, w, path="split_tc")
        x_np = inputs.uniform(8600 + h + w, 40, h, w)
        x = torch.from_numpy(x_np).to(cuda_dev)
        for kind in KINDS:
            ref_gpu = plan.execute(kind, x)
            y = x.clone()
            plan.execute(kind, y, y)
            torch.cuda.synchronize()
            assert torch.equal(y, ref_gpu), (h, w, kind)
    # report-only term counts sit where they should
    x = inputs.uniform(8700, 8, 128, 128)
    ref = oracle_mod.forward(x, 0)
    e_hilo = oracle_mod.metrics(_run(Plan(128, 128, path="split_hilo"), "forward", x, cuda_dev), ref, x)["e_rel_max"]
    e_bf16 = oracle_mod.metrics(_run(Plan(128, 128, path="bf16"), "forward", x, cuda_dev), ref, x)["e_rel_max"]
    assert 1e-7 < e_hilo < 1e-4 and 1e-4 < e_bf16 < 3e-2, (e_hilo, e_bf16)
    # a ragged batch on the tensor-core path: indexed arrays through both routes
    shapes = [(8, 8), (16, 16), (128, 128), (64, 256), (8, 8), (128, 128), (32, 32)] * 3
    arrs = _ragged_inputs(shapes, 8800)
    rg = Ragged(shapes, path="split_tc")
    xr = _pack(rg, arrs, cuda_dev)
    for kind in ("forward", "inverse", "roundtrip"):
        y = torch.full_like(xr, float("nan"))
        rg.execute(kind, xr, y)
        torch.cuda.synchronize()
        for a, o, (r, c) in zip(arrs, _unpack(rg, y, shapes), shapes):
            _assert_parity(oracle_mod, o[None], _ref(oracle_mod, kind, a[None], 0), a[None], 0, kind,
                           ("tg-ragged", r, c, kind))


# ------------------------------------------------------------ range protection (Section 6 boundary cases)
def boundary_diagnostics(o, dev, sizes=(8, 16, 32, 64), kinds=KINDS, paths=("fp32",)):
    """Run the boundary suite with range protection off and on; returns the
    per-setting counts (checks, representable, failed) and the failures."""
    from paper_2609_28519_gb300 import Plan
    res = {}
    for protect in (False, True):
        tot = {"checks": 0, "representable": 0, "failed": 0, "failures": []}
        for path in paths:
            for n in sizes:
                plan = Plan(n, n, path=path)
                if protect:
                    plan.set_range_protection(True)
                x, labels = inputs.boundary_suite(9000 + n, n)
                for kind in kinds:
                    y = _run(plan, kind, x, dev)
                    m = o.boundary_metrics(y, _ref(o, kind, x, 0), x)
                    tot["checks"] += m["checks"]
                    tot["representable"] += m["n_representable"]
                    tot["failed"] += m["n_failed"]
                    tot["failures"] += [(path, n, kind, labels[i]) for i in range(len(labels))
                                        if m["representable"][i] and not m["passed"][i]]
        res["protected" if protect else "unprotected"] = tot
    return res


def test_range_protection_boundary_suite(oracle_mod, cuda_dev, record_property):
    """Section 6 boundary diagnostics regenerated synthetically (subnormal,
    mixed, near-FLT_MAX amplitudes; 14 cases x 3 directions x 4 sizes):
    without protection the overflowing intermediates and subnormal arithmetic
    fail some checks (reported, not accepted); with per-array power-of-two
    scaling every case whose exact result is representable passes, and
    ordinary inputs give the same bits with protection on as off."""
    import torch
    from paper_2609_28519_gb300 import Plan
    res = boundary_diagnostics(oracle_mod, cuda_dev)
    for k in ("unprotected", "protected"):
        record_property(f"boundary_{k}", {kk: res[k][kk] for kk in ("checks", "representable", "failed")})
    print("boundary diagnostics:", {k: {kk: v[kk] for kk in ("checks", "representable", "failed")}
                                    for k, v in res.items()})
    assert res["protected"]["failed"] == 0, res["protected"]["failures"]
    assert res["unprotected"]["failed"] > 0  # the suite does reach the boundary
    # ordinary inputs: protection changes nothing (power-of-two scaling is exact)
    for (h, w, path) in [(16, 16, "fp32"), (64, 128, "fp32"), (256, 256, "fp32"), (32, 32, "split_tc"),
                         (128, 128, "split_tc")]:
        x = torch.from_numpy(inputs.uniform(9100 + h + w, 9, h, w)).to(cuda_dev)
        a, b = Plan(h, w, path=path), Plan(h, w, path=path)
        b.set_range_protection(True)
        for kind in KINDS:
            ya, yb = a.execute(kind, x), b.execute(kind, x)
            torch.cuda.synchronize()
            # every core is linear, and scaling all inputs by a power of two
            # scales every rounding with them: the same bits
            assert torch.equal(ya, yb), (h, w, path, kind)
    # the tiled view with protection, in place
    img = torch.from_numpy(inputs.ramp_image(5, 256, 512) * np.float32(2.0 ** 120)).to(cuda_dev)
    p = Plan(16, 16)
    p.set_range_protection(True)
    out = p.execute_tiled("forward", img.clone())
    blocks = inputs.image_to_blocks(img.cpu().numpy(), 16, 16)
    torch.cuda.synchronize()
    m = oracle_mod.boundary_metrics(inputs.image_to_blocks(out.cpu().numpy(), 16, 16), oracle_mod.forward(blocks, 0),
                                    blocks)
    assert m["n_failed"] == 0


@pytest.mark.parametrize("h,w", [(192, 192), (384, 384), (1536, 1536), (384, 1536), (1536, 192), (192, 1024),
                                 (768, 384)])
@pytest.mark.parametrize("norm", [0, 1])
def test_radix3_lines_against_oracle(oracle_mod, cuda_dev, h, w, norm):
    """Sides 3 * 2^k (192, 384, 768, 1536) on the FFT line engine (one radix-3
    stage in the half-length FFT), alone and mixed with powers of two."""
    from paper_2609_28519_gb300 import Plan
    plan = Plan(h, w, norm=norm, path="fp32")
    assert plan.info().variant == 2
    x = inputs.gaussian(9500 + h + 3 * w + norm, 2 if h * w <= 1 << 20 else 1, h, w)
    for kind in KINDS:
        y = _run(plan, kind, x, cuda_dev)
        _assert_parity(oracle_mod, y, _ref(oracle_mod, kind, x, norm), x, norm, kind, ("radix3", h, w, norm, kind))


def test_spectral_ring_tiled_and_chunk_sizes(oracle_mod, cuda_dev):
    """The spectral direction on image blocks of the ring shapes, in place;
    and the workspace chunk of the separable routes changes nothing but the
    launch count (bit-equal results for 1-array and default chunks, the
    spectral direction included)."""
    import torch
    from paper_2609_28519_gb300 import Plan
    img = inputs.ramp_image(11, 256, 384)
    for (h, w) in [(64, 64), (128, 64)]:
        lam = inputs.random_diagonal(11 + h + w, h, w, -1.0, 2.0)
        plan = Plan(h, w)
        plan.set_spectral(lam)
        d = torch.from_numpy(img).to(cuda_dev)
        out = plan.execute_tiled("spectral", d)
        d2 = d.clone()
        plan.execute_tiled("spectral", d2, d2)
        torch.cuda.synchronize()
        assert torch.equal(out, d2)
        blocks = inputs.image_to_blocks(img, h, w)
        _assert_spectral(oracle_mod, inputs.image_to_blocks(out.cpu().numpy(), h, w), blocks, lam,
                         ("spectral-ring-tiled", h, w))
    for (h, w, path) in [(256, 256, "fp32"), (384, 192, "fp32"), (24, 40, "fp32"), (256, 128, "split_tc")]:
        x = torch.from_numpy(inputs.uniform(9700 + h + w, 7, h, w)).to(cuda_dev)
        plan = Plan(h, w, path=path)
        plan.set_spectral(inputs.random_diagonal(9800 + h + w, h, w, -1.0, 2.0))
        kinds = KINDS + ["spectral"]
        ref = {k: plan.execute(k, x) for k in kinds}
        plan.set_chunk_bytes(1)  # one array per chunk: seven rounds of passes
        for k in kinds:
            y = plan.execute(k, x)
            torch.cuda.synchronize()
            assert torch.equal(y, ref[k]), (h, w, path, k)
