"""Seeded synthetic inputs for the 2D DCT workloads (numpy only).

This module is shared by the tests, the benchmark and smoke(): it draws the
arrays that both the CUDA path and the FP64 oracle are fed.  It holds no part
of the transform itself.  Every generator takes an explicit seed and returns
contiguous float32 arrays of shape (batch, h, w) unless stated otherwise.

Workload recipes (the paper's timing pools and its 474-array verification
dataset are not available, so these synthetic distributions stand in for
them; see Section 6 of the paper for the input categories):

* ``uniform``         i.i.d. uniform[-1, 1]
* ``gaussian``        i.i.d. N(0, 1)
* ``ramp_image``      N(0, 1) + 0.01 (i + j) on a whole image, global coords
* ``extreme``         sign +-1 (p = 1/2) times 1e30 (p = 1/2) else 1e-30
* ``weak_cosine``     unit cosine mode plus a 1e-6 cosine mode, modes >= 1
* ``paper_categories`` impulses, cosine modes, cancelling neighbours,
  neighbouring floats, weak perturbations of a strong constant, amplitudes
  2^-100 .. 2^90 (Section 6 input categories, regenerated synthetically)
* ``ragged_shapes``   shapes drawn uniformly from the nine mixed shapes
* ``boundary_suite``  extreme-amplitude cases (Section 6 boundary diagnostics,
  regenerated synthetically): deep and shallow subnormals, mixed subnormal /
  normal, amplitudes near FLT_MAX, constants near FLT_MAX / n
* ``random_diagonal`` a seeded h x w spectral diagonal, uniform in [lo, hi]
* ``poisson_diagonal`` the inverse eigenvalues of the 5-point Laplacian with
  reflecting (Neumann) borders, the diagonal of a least-squares phase-
  unwrapping solve (Section 1.1); 0 at (0, 0)
"""
from __future__ import annotations

import numpy as np

RAGGED_SHAPES = [(8, 8), (16, 16), (32, 32), (64, 64), (128, 128), (256, 256),
                 (64, 256), (128, 512), (768, 1024)]


def uniform(seed: int, batch: int, h: int, w: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(batch, h, w)).astype(np.float32)


def gaussian(seed: int, batch: int, h: int, w: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=(batch, h, w), dtype=np.float32)


def ramp_image(seed: int, rows: int = 2048, cols: int = 2048) -> np.ndarray:
    """Whole image N(0,1) + 0.01 (i + j), i and j global pixel coordinates."""
    rng = np.random.default_rng(seed)
    img = rng.standard_normal(size=(rows, cols), dtype=np.float32)
    ramp = (np.arange(rows, dtype=np.float32)[:, None] + np.arange(cols, dtype=np.float32)[None, :])
    return (img + np.float32(0.01) * ramp).astype(np.float32)


def image_to_blocks(img: np.ndarray, bh: int, bw: int) -> np.ndarray:
    """(R, C) image -> (R/bh * C/bw, bh, bw) blocks in row-major block order."""
    r, c = img.shape
    return np.ascontiguousarray(
        img.reshape(r // bh, bh, c // bw, bw).transpose(0, 2, 1, 3).reshape(-1, bh, bw))


def blocks_to_image(blocks: np.ndarray, rows: int, cols: int) -> np.ndarray:
    bh, bw = blocks.shape[-2:]
    return np.ascontiguousarray(
        blocks.reshape(rows // bh, cols // bw, bh, bw).transpose(0, 2, 1, 3).reshape(rows, cols))


def extreme(seed: int, batch: int, h: int, w: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    sign = np.where(rng.random(size=(batch, h, w)) < 0.5, -1.0, 1.0)
    mag = np.where(rng.random(size=(batch, h, w)) < 0.5, 1e30, 1e-30)
    return (sign * mag).astype(np.float32)


def _mode(n: int, k: int) -> np.ndarray:
    i = np.arange(n, dtype=np.float64)
    return np.cos(np.pi * (2.0 * i + 1.0) * k / (2.0 * n))


def weak_cosine(seed: int, batch: int, n: int, weak: float = 1e-6):
    """X = c_k1(i) c_l1(j) + weak * c_k2(i) c_l2(j), modes drawn per array.

    Returns (x, modes) with modes an int array (batch, 4) = (k1, l1, k2, l2),
    all in [1, n-1] and (k1, l1) != (k2, l2).
    """
    rng = np.random.default_rng(seed)
    x = np.empty((batch, n, n), dtype=np.float32)
    modes = np.empty((batch, 4), dtype=np.int64)
    for b in range(batch):
        while True:
            k1, l1, k2, l2 = (int(v) for v in rng.integers(1, n, size=4))
            if (k1, l1) != (k2, l2):
                break
        modes[b] = (k1, l1, k2, l2)
        x[b] = (np.outer(_mode(n, k1), _mode(n, l1))
                + weak * np.outer(_mode(n, k2), _mode(n, l2))).astype(np.float32)
    return x, modes


def paper_categories(seed: int, n: int, h: int | None = None) -> np.ndarray:
    """A small batch covering the Section 6 input categories for one shape."""
    h = n if h is None else h
    w = n
    rng = np.random.default_rng(seed)
    out = []
    # impulses at a corner, the centre and a random spot
    for (i0, j0) in [(0, 0), (h // 2, w // 2), (int(rng.integers(h)), int(rng.integers(w)))]:
        a = np.zeros((h, w), np.float32)
        a[i0, j0] = 1.0
        out.append(a)
    # separable cosine modes
    for _ in range(2):
        k, l = int(rng.integers(h)), int(rng.integers(w))
        out.append(np.outer(_mode(h, k), _mode(w, l)).astype(np.float32))
    # nearly cancelling neighbours
    a = rng.uniform(-1, 1, size=(h, w)).astype(np.float32)
    a[:, 1::2] = -a[:, 0::2] * np.float32(1.0 + 2.0 ** -20)
    out.append(a)
    # neighbouring floats: 1.0 and its successors
    base = np.float32(1.0)
    steps = rng.integers(0, 4, size=(h, w)).astype(np.int32)
    out.append((np.full((h, w), base, np.float32).view(np.int32) + steps).view(np.float32))
    # weak perturbation of a strong constant
    out.append((np.float32(1000.0) + np.float32(1e-3) * rng.uniform(-1, 1, size=(h, w))).astype(np.float32))
    # random arrays scaled to amplitudes 2^-100 .. 2^90
    for e in (-100, -40, 0, 40, 90):
        out.append((rng.uniform(-1, 1, size=(h, w)) * 2.0 ** e).astype(np.float32))
    # constant and all-zero inputs
    out.append(np.full((h, w), 0.75, np.float32))
    out.append(np.zeros((h, w), np.float32))
    return np.stack(out).astype(np.float32)


def ragged_shapes(seed: int, count: int = 4096, shapes=None):
    """Shapes for a ragged batch, each drawn uniformly from ``shapes``."""
    shapes = RAGGED_SHAPES if shapes is None else shapes
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, len(shapes), size=count)
    return [shapes[int(i)] for i in idx]


def random_diagonal(seed: int, h: int, w: int, lo: float = 0.5, hi: float = 2.0) -> np.ndarray:
    """A seeded spectral diagonal Lambda (float64, h x w), i.i.d. uniform[lo, hi]."""
    return np.random.default_rng(seed).uniform(lo, hi, size=(h, w))


def poisson_diagonal(h: int, w: int) -> np.ndarray:
    """1 / (2 cos(pi k / h) + 2 cos(pi l / w) - 4) for (k, l) != (0, 0), and 0 at
    (0, 0): the inverse eigenvalues of the 5-point Laplacian with reflecting
    borders on an h x w grid (float64).  An application-side operator (the
    diagonal of a Poisson solve), not part of the transform."""
    k = np.arange(h, dtype=np.float64)[:, None]
    l = np.arange(w, dtype=np.float64)[None, :]
    ev = 2.0 * np.cos(np.pi * k / h) + 2.0 * np.cos(np.pi * l / w) - 4.0
    ev[0, 0] = 1.0
    lam = 1.0 / ev
    lam[0, 0] = 0.0
    return lam


def boundary_suite(seed: int, n: int):
    """Boundary-diagnostic inputs for n x n arrays (float32), one array per
    case; returns (x, labels)."""
    rng = np.random.default_rng(seed)
    u = lambda: rng.uniform(-1.0, 1.0, size=(n, n))
    cases = []
    for e in (-149, -140, -130, -127):          # subnormal and edge-of-normal amplitudes
        cases.append((f"uniform*2^{e}", u() * 2.0 ** e))
    mix = u() * 2.0 ** -120
    mix[rng.random(size=(n, n)) < 0.5] *= 2.0 ** -20
    cases.append(("mixed 2^-120 / 2^-140", mix))
    for e in (120, 125, 126, 127):              # near the top of the range
        cases.append((f"uniform*2^{e}", u() * 2.0 ** e))
    big = float(np.finfo(np.float32).max) / (2 * n)  # orthonormal results stay below FLT_MAX / 2
    checker = np.where((np.add.outer(np.arange(n), np.arange(n)) % 2) == 0, 1.0, -1.0)
    cases.append(("constant FLT_MAX/2n", np.full((n, n), big)))
    cases.append(("uniform*FLT_MAX/2n", u() * big))
    cases.append(("checkerboard*FLT_MAX/2n", checker * big))
    cases.append(("constant 2^127", np.full((n, n), 2.0 ** 127)))
    cases.append(("checkerboard*2^127", checker * 2.0 ** 127))
    x = np.stack([c[1] for c in cases]).astype(np.float32)
    return x, [c[0] for c in cases]
