"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each check ties the oracle to the paper's definitions (Eq. 1, Eq. 2,
Section 7.1 rectangles, Section 2.1 round trip and REDFT normalization) via
something independent of its own code: brute-force double sums with libm
cosines, SciPy's DCT, hand-derived closed forms, and algebraic invariants.
The planted-fault tests at the end show that a dropped term, a wrong scale,
a wrong index, a transposed operand or swapped axes each break a pin.
"""
import math

import numpy as np
import pytest

from paper_2609_28519_gb300 import inputs

SHAPES_SMALL = [(1, 1), (2, 2), (3, 3), (4, 4), (8, 8), (16, 16), (1, 4), (4, 1),
                (3, 5), (8, 16), (16, 8), (24, 8)]


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


# ---------------------------------------------------------------- cosine table
def test_cospi_frac_exact_points(oracle_mod):
    o = oracle_mod
    assert o.cospi_frac(0, 7) == 1.0
    assert o.cospi_frac(7, 7) == -1.0
    assert o.cospi_frac(14, 7) == 1.0
    assert o.cospi_frac(8, 16) == 0.0          # cos(pi/2)
    assert o.cospi_frac(24, 16) == 0.0         # cos(3pi/2)
    assert o.cospi_frac(3 * 64, 64) == -1.0
    assert abs(o.cospi_frac(1, 4) - math.sqrt(0.5)) < 1e-16
    assert abs(o.cospi_frac(1, 3) - 0.5) < 1e-16
    assert abs(o.cospi_frac(2, 3) + 0.5) < 1e-16
    for m in range(0, 200):
        assert abs(o.cospi_frac(m, 37) - math.cos(math.pi * m / 37)) < 1e-14


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("h,w", SHAPES_SMALL)
@pytest.mark.parametrize("norm", [0, 1])
def test_bruteforce_matches_separable(oracle_mod, h, w, norm):
    o = oracle_mod
    x = inputs.uniform(11 + h * 31 + w, 3, h, w)
    for d, fn in (("forward", o.forward), ("inverse", o.inverse)):
        ref = o.bruteforce(x, d, norm)
        got = fn(x, norm)
        assert _rel(got, ref) < 1e-13, (d, h, w, norm)


# ---------------------------------------------------------------- SciPy
@pytest.mark.parametrize("h,w", [(8, 8), (16, 16), (32, 32), (64, 64), (128, 128), (256, 256),
                                 (8, 64), (64, 8), (64, 256), (24, 40), (3, 7)])
def test_scipy_special_case(oracle_mod, h, w):
    fft = pytest.importorskip("scipy.fft")
    o = oracle_mod
    x = inputs.gaussian(5 + h + w, 2, h, w)
    xd = x.astype(np.float64)
    # orthonormal DCT-II / DCT-III pair (Eq. 2)
    assert _rel(o.forward(x, 0), fft.dctn(xd, type=2, norm="ortho", axes=(1, 2))) < 1e-13
    assert _rel(o.inverse(x, 0), fft.idctn(xd, type=2, norm="ortho", axes=(1, 2))) < 1e-13
    # REDFT10 = SciPy's unnormalized type-2 DCT; REDFT01 = 2n x SciPy's idct per axis
    assert _rel(o.forward(x, 1), fft.dctn(xd, type=2, axes=(1, 2))) < 1e-13
    assert _rel(o.inverse(x, 1), fft.idctn(xd, type=2, axes=(1, 2)) * (4.0 * h * w)) < 1e-13


# ---------------------------------------------------------------- closed forms
def test_hand_derived_four_point(oracle_mod):
    """DCT-II (orthonormal) of [1, 2, 3, 4], derived by hand from Eq. 1."""
    o = oracle_mod
    c1, c3 = math.cos(math.pi / 8), math.cos(3 * math.pi / 8)
    expect = np.array([5.0, -(3 * c1 + c3) / math.sqrt(2), 0.0, (c1 - 3 * c3) / math.sqrt(2)])
    got = o.forward(np.array([[[1, 2, 3, 4]]], np.float32), 0).ravel()
    assert np.max(np.abs(got - expect)) < 1e-14
    # 2 x 2: Q_2 = [[1, 1], [1, -1]] / sqrt(2); impulse at (0, 0) -> all 1/2
    y = o.forward(np.array([[[1, 0], [0, 0]]], np.float32), 0)[0]
    assert np.max(np.abs(y - 0.5)) < 1e-15
    y = o.forward(np.array([[[1, 2], [3, 4]]], np.float32), 0)[0]
    assert np.max(np.abs(y - np.array([[5.0, -1.0], [-2.0, 0.0]]))) < 1e-14


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16, 64, 256])
def test_orthonormal_matrix(oracle_mod, n):
    q = oracle_mod.matrix(n, "forward", 0)
    assert np.max(np.abs(q @ q.T - np.eye(n))) < 1e-13
    qi = oracle_mod.matrix(n, "inverse", 0)
    assert np.max(np.abs(qi - q.T)) == 0.0


@pytest.mark.parametrize("h,w", [(8, 8), (16, 16), (32, 64), (256, 256), (24, 8)])
def test_constant_gives_dc_only(oracle_mod, h, w):
    c = 0.625
    y = oracle_mod.forward(np.full((1, h, w), c, np.float32), 0)[0]
    assert abs(y[0, 0] - c * math.sqrt(h * w)) < 1e-12 * math.sqrt(h * w)
    y[0, 0] = 0.0
    assert np.max(np.abs(y)) < 1e-12


@pytest.mark.parametrize("h,w", [(8, 8), (16, 16), (64, 64), (16, 32)])
def test_pure_cosine_single_coefficient(oracle_mod, h, w):
    rng = np.random.default_rng(h * w)
    for _ in range(4):
        k0, l0 = int(rng.integers(h)), int(rng.integers(w))
        ci = np.cos(np.pi * (2 * np.arange(h) + 1) * k0 / (2 * h))
        cj = np.cos(np.pi * (2 * np.arange(w) + 1) * l0 / (2 * w))
        x = np.outer(ci, cj)[None].astype(np.float32)
        y = oracle_mod.forward(x, 0)[0]
        beta_h = math.sqrt(h) if k0 == 0 else math.sqrt(h / 2)
        beta_w = math.sqrt(w) if l0 == 0 else math.sqrt(w / 2)
        # input is float32-rounded: allow for that rounding only
        assert abs(y[k0, l0] - beta_h * beta_w) < 1e-6 * beta_h * beta_w
        y[k0, l0] = 0.0
        assert np.max(np.abs(y)) < 1e-6


def test_impulse_response_scale(oracle_mod):
    """Impulse at (i0, j0) gives the outer product of two Q columns (Section 2.1)."""
    o = oracle_mod
    h, w = 16, 8
    qh, qw = o.matrix(h, "forward", 0), o.matrix(w, "forward", 0)
    for (i0, j0) in [(0, 0), (5, 3), (15, 7)]:
        x = np.zeros((1, h, w), np.float32)
        x[0, i0, j0] = 1.0
        y = o.forward(x, 0)[0]
        assert np.max(np.abs(y - np.outer(qh[:, i0], qw[:, j0]))) < 1e-15
    # DC of an impulse is 1/sqrt(hw) under ORTHO and 4 under REDFT10
    x = np.zeros((1, h, w), np.float32)
    x[0, 3, 2] = 1.0
    assert abs(o.forward(x, 0)[0, 0, 0] - 1 / math.sqrt(h * w)) < 1e-15
    assert abs(o.forward(x, 1)[0, 0, 0] - 4.0) < 1e-14


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("h,w", [(8, 8), (16, 16), (32, 32), (8, 64), (128, 32), (24, 16)])
def test_invariants(oracle_mod, h, w):
    o = oracle_mod
    x = inputs.uniform(100 + h + w, 4, h, w)
    z = inputs.gaussian(200 + h + w, 4, h, w)
    y = o.forward(x, 0)
    # Parseval under orthonormal scaling
    assert np.allclose(np.linalg.norm(y.reshape(4, -1), axis=1),
                       np.linalg.norm(x.astype(np.float64).reshape(4, -1), axis=1), rtol=1e-13)
    # round trip returns X (both normalizations)
    for norm in (0, 1):
        assert _rel(o.roundtrip(x, norm), x.astype(np.float64)) < 1e-13
    # REDFT01 o REDFT10 = 2n I per axis (the pair factor of Section 2.1)
    for n in (h, w):
        pair = o.matrix(n, "inverse", 1) @ o.matrix(n, "forward", 1)
        assert np.max(np.abs(pair - 2.0 * n * np.eye(n))) < 1e-12 * n
    # adjointness <C(X), Z> = <X, C^{-1}(Z)>
    lhs = np.sum(y * z.astype(np.float64), axis=(1, 2))
    rhs = np.sum(x.astype(np.float64) * o.inverse(z, 0), axis=(1, 2))
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)
    # linearity
    a, b = np.float32(0.5), np.float32(-2.0)
    comb = (a * x + b * z).astype(np.float32)
    assert _rel(o.forward(comb, 0), a * y + b * o.forward(z, 0)) < 1e-6  # comb is float32-rounded
    # rectangle orientation: C_{h x w}(X)^T = C_{w x h}(X^T)
    xt = np.ascontiguousarray(np.transpose(x, (0, 2, 1)))
    assert _rel(np.transpose(y, (0, 2, 1)), o.forward(xt, 0)) < 1e-14


def test_paper_categories_parseval(oracle_mod):
    o = oracle_mod
    for n in (8, 16, 32):
        x = inputs.paper_categories(7, n)
        y = o.forward(x, 0)
        nx = np.linalg.norm(x.astype(np.float64).reshape(len(x), -1), axis=1)
        ny = np.linalg.norm(y.reshape(len(x), -1), axis=1)
        assert np.allclose(ny, nx, rtol=1e-12, atol=0)
        # the all-zero input gives an exactly zero output
        assert np.all(y[-1] == 0.0)


def test_threads_do_not_change_results(oracle_mod):
    o = oracle_mod
    x = inputs.uniform(3, 37, 16, 8)
    a = o.forward(x, 0, threads=1)
    b = o.forward(x, 0, threads=5)
    assert np.array_equal(a, b)
    assert o.default_threads() >= 1


# ---------------------------------------------------------------- spectral operator (Prop. 1, Eq. 4)
def _neumann_laplacian(phi: np.ndarray) -> np.ndarray:
    """5-point Laplacian with reflecting borders (ghost cells equal to the
    border cells), plain stencil arithmetic on each trailing h x w array."""
    p = np.asarray(phi, dtype=np.float64)
    up = np.concatenate([p[..., :1, :], p[..., :-1, :]], axis=-2)
    down = np.concatenate([p[..., 1:, :], p[..., -1:, :]], axis=-2)
    left = np.concatenate([p[..., :, :1], p[..., :, :-1]], axis=-1)
    right = np.concatenate([p[..., :, 1:], p[..., :, -1:]], axis=-1)
    return up + down + left + right - 4.0 * p


@pytest.mark.parametrize("h,w,b", [(8, 8, 3), (16, 16, 2), (8, 32, 2), (5, 7, 2), (256, 256, 1)])
def test_spectral_identity_is_round_trip(oracle_mod, h, w, b):
    o = oracle_mod
    x = inputs.uniform(400 + h + w, b, h, w)
    assert _rel(o.spectral(x, np.ones((h, w))), x.astype(np.float64)) < 1e-13


@pytest.mark.parametrize("h,w", [(8, 8), (16, 16), (8, 16), (5, 7), (32, 24)])
def test_spectral_cosine_modes_are_eigenvectors(oracle_mod, h, w):
    """A separable cosine mode c_k0(i) c_l0(j) is an eigenvector of
    U^T Lambda U with eigenvalue Lambda[k0, l0] (an asymmetric Lambda, so a
    transposed table is caught)."""
    o = oracle_mod
    lam = inputs.random_diagonal(7 + h * w, h, w)
    rng = np.random.default_rng(h + 3 * w)
    modes = [(0, 0), (0, w - 1), (h - 1, 0), (1, 2 % w)] + [
        (int(rng.integers(h)), int(rng.integers(w))) for _ in range(4)]
    i = np.arange(h)[:, None]
    j = np.arange(w)[None, :]
    for (k0, l0) in modes:
        x = (np.cos(np.pi * (2 * i + 1) * k0 / (2 * h)) * np.cos(np.pi * (2 * j + 1) * l0 / (2 * w)))
        x = x.astype(np.float32)[None]
        got = o.spectral(x, lam)
        # x is the float32 rounding of the mode (relative error <= 2^-24 per
        # element), whose residual is scaled by at most max|Lambda| + Lambda[k0, l0]
        assert _rel(got, lam[k0, l0] * x.astype(np.float64)) < 4 * 2.0 ** -24 * 2.0 / lam[k0, l0], (k0, l0)


@pytest.mark.parametrize("h,w", [(16, 16), (32, 24), (8, 64), (256, 256)])
def test_spectral_poisson_inverts_neumann_laplacian(oracle_mod, h, w):
    """Textbook special case: the DCT-II diagonalizes the 5-point Laplacian
    with reflecting borders, so U^T Lambda_P U applied to L(phi) returns phi
    minus its mean (the (0, 0) mode is the Laplacian's null space)."""
    o = oracle_mod
    phi = inputs.gaussian(600 + h + w, 2, h, w).astype(np.float64)
    f = _neumann_laplacian(phi)
    got = o.spectral(f.astype(np.float32), inputs.poisson_diagonal(h, w))
    # f is rounded to float32 for the call, so compare against the exact
    # solve of the rounded right-hand side's error budget: Lambda_P is at most
    # ~ (h^2 + w^2) / (2 pi^2) in size
    want = phi - phi.mean(axis=(1, 2), keepdims=True)
    amp = (h * h + w * w) / (2 * np.pi ** 2)
    assert _rel(got, want) < 1e-7 * amp, _rel(got, want)


@pytest.mark.parametrize("h,w", [(1, 1), (2, 3), (3, 2), (4, 4), (3, 5)])
def test_spectral_bruteforce_tiny(oracle_mod, h, w):
    """Direct quadruple sum with libm cosines (numpy), no separable form."""
    o = oracle_mod
    x = inputs.uniform(33 + h * w, 2, h, w)
    lam = inputs.random_diagonal(34 + h * w, h, w, -1.0, 1.0)
    a = lambda k, n: math.sqrt((1.0 if k == 0 else 2.0) / n)
    out = np.zeros((2, h, w))
    for b in range(2):
        for i in range(h):
            for j in range(w):
                acc = 0.0
                for k in range(h):
                    for l in range(w):
                        coef = 0.0
                        for i2 in range(h):
                            for j2 in range(w):
                                coef += (float(x[b, i2, j2]) * math.cos(math.pi * (2 * i2 + 1) * k / (2 * h))
                                         * math.cos(math.pi * (2 * j2 + 1) * l / (2 * w)))
                        coef *= a(k, h) * a(l, w)
                        acc += (lam[k, l] * coef * a(k, h) * a(l, w) * math.cos(math.pi * (2 * i + 1) * k / (2 * h))
                                * math.cos(math.pi * (2 * j + 1) * l / (2 * w)))
                out[b, i, j] = acc
    assert _rel(o.spectral(x, lam), out) < 1e-13


def test_spectral_symmetric_and_linear_in_lambda(oracle_mod):
    o = oracle_mod
    h, w = 16, 24
    x = inputs.uniform(71, 2, h, w)
    z = inputs.uniform(72, 2, h, w)
    l1 = inputs.random_diagonal(73, h, w)
    l2 = inputs.random_diagonal(74, h, w, -3.0, 1.0)
    sx = o.spectral(x, l1)
    # a real diagonal gives a symmetric operator: <S X, Z> = <X, S Z>
    assert np.allclose(np.sum(sx * z, axis=(1, 2)), np.sum(x.astype(np.float64) * o.spectral(z, l1), axis=(1, 2)),
                       rtol=1e-12, atol=1e-12)
    # linear in Lambda
    assert _rel(o.spectral(x, 2.0 * l1 - l2), 2.0 * sx - o.spectral(x, l2)) < 1e-13


# ---------------------------------------------------------------- checker sensitivity
def _checker_cases(o, h, w):
    x = inputs.uniform(17, 3, h, w)
    y = o.forward(x, 0)
    return x, y


@pytest.mark.parametrize("h,w", [(8, 8), (16, 16), (64, 32)])
def test_checker_accepts_fp32_rounding_and_rejects_faults(oracle_mod, h, w):
    """Section 6 fault injection: scale, sign, orientation, component loss."""
    o = oracle_mod
    x, y = _checker_cases(o, h, w)
    ok = o.metrics(y.astype(np.float32), y, x)
    assert o.accept(ok)
    faults = {
        "scale": y * (1 + 1e-4),
        "sign": y.copy(),
        "orientation": np.transpose(y, (0, 2, 1)).copy() if h == w else y[:, ::-1, :].copy(),
        "component_loss": y.copy(),
    }
    faults["sign"][:, 1, 2] *= -1
    faults["component_loss"][:, 2, 1] = 0.0
    for name, bad in faults.items():
        m = o.metrics(bad.astype(np.float32), y, x)
        assert not o.accept(m), name
    # zero input: any non-zero output is a violation
    z = np.zeros((1, h, w), np.float32)
    bad = np.zeros((1, h, w), np.float32)
    bad[0, 0, 0] = 1e-30
    assert not o.accept(o.metrics(bad, o.forward(z, 0), z))
    assert o.accept(o.metrics(np.zeros_like(z), o.forward(z, 0), z))


# ---------------------------------------------------------------- planted faults
def _pins_fail(o) -> list:
    """A fast subset of the pins; returns the names of those that fail."""
    failed = []
    for (h, w) in [(8, 8), (8, 16)]:
        x = inputs.uniform(5, 2, h, w)
        for norm in (0, 1):
            for d, fn in (("forward", o.forward), ("inverse", o.inverse)):
                if _rel(fn(x, norm), o.bruteforce(x, d, norm)) > 1e-12:
                    failed.append(f"bruteforce-{d}-{norm}-{h}x{w}")
    x = inputs.uniform(6, 2, 8, 8)
    if _rel(o.roundtrip(x, 0), x.astype(np.float64)) > 1e-12:
        failed.append("roundtrip")
    # spectral operator: a cosine mode is an eigenvector with eigenvalue Lambda[k0, l0]
    lam = inputs.random_diagonal(9, 8, 8)
    i = np.arange(8)[:, None]
    xm = (np.cos(np.pi * (2 * i + 1) * 1 / 16) * np.cos(np.pi * (2 * i.T + 1) * 3 / 16)).astype(np.float32)[None]
    if _rel(o.spectral(xm, lam), lam[1, 3] * xm.astype(np.float64)) > 1e-6:
        failed.append("spectral-mode")
    return failed


@pytest.mark.parametrize("fault", [1, 2, 3, 4, 5, 6])
def test_planted_fault_breaks_a_pin(oracle_mod, fault):
    o = oracle_mod
    assert _pins_fail(o) == []
    o.set_fault(fault)
    try:
        assert _pins_fail(o) != [], f"fault {fault} slipped through"
    finally:
        o.set_fault(0)
    assert _pins_fail(o) == []


def test_boundary_metrics_flags_overflow_and_accepts_rounding(oracle_mod):
    """The boundary checker: the exact result rounded to float32 passes, an
    infinity where the result is representable fails, a non-representable
    case is not counted, and an error far above the rounding floor fails."""
    o = oracle_mod
    x, labels = inputs.boundary_suite(3, 8)
    ref = o.forward(x, 0)
    with np.errstate(over="ignore"):
        y32 = ref.astype(np.float32)
    m = o.boundary_metrics(y32, ref, x)
    assert m["n_failed"] == 0 and m["n_representable"] == m["checks"] - int(np.sum(~m["representable"]))
    bad = y32.astype(np.float64).copy()
    k = labels.index("constant FLT_MAX/2n")
    bad[k, 0, 0] = np.inf
    assert not o.boundary_metrics(bad, ref, x)["passed"][k]
    sub = labels.index("uniform*2^-130")
    bad2 = ref.copy()
    bad2[sub] *= 1.001
    assert not o.boundary_metrics(bad2, ref, x)["passed"][sub]
    assert not m["representable"][labels.index("constant 2^127")]
