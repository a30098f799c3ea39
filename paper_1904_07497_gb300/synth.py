"""Seeded synthetic inputs for RES-PCA workloads.

This module only draws inputs; it holds none of the method's arithmetic, so
that the CUDA path and the CPU oracle can share it.  Every generator uses
numpy's PCG64 with a fixed drawing order, returns the data matrix X as float32
in column-major (Fortran) order, d x n (a column is one sample / frame), and
the ground-truth parts in float64 for reporting.

Workload shapes follow the paper's experiments (Sec. 5): video frames of
240 x 320 pixels as columns (Table 1: Highway, Camera Parameter), 1-3 static
backgrounds plus a sparse moving foreground; and random low-rank plus sparse
+-1 corruption matrices of the kind used to study RPCA recovery.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Problem:
    X: np.ndarray          # float32, (d, n), Fortran order
    L0: np.ndarray | None  # float64 ground-truth low-rank part (None if not kept)
    S0: np.ndarray | None  # float64 ground-truth sparse part (None if not kept)
    rank: int              # number of clusters / backgrounds to ask for (c)
    truth_labels: np.ndarray | None = None


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def lowrank_sparse(d: int, n: int, r: int, sparsity: float, seed: int,
                   var: float | None = None, keep_parts: bool = True) -> Problem:
    """X = U V^T + S0: U (d x r), V (n x r) with i.i.d. N(0, var) entries
    (var defaults to 1/max(d, n)); S0 has Bernoulli(sparsity) support with
    values +1 / -1 drawn with equal probability.

    Drawing order: U, V, support mask, signs."""
    if var is None:
        var = 1.0 / max(d, n)
    g = _rng(seed)
    sd = np.sqrt(var)
    U = g.standard_normal((d, r)) * sd
    V = g.standard_normal((n, r)) * sd
    # (n, d) C-order is the same memory as (d, n) Fortran order.
    mask = g.random((n, d), dtype=np.float32) < np.float32(sparsity)
    signs = g.integers(0, 2, size=(n, d), dtype=np.int8)
    S0t = np.where(mask, (2 * signs - 1).astype(np.float32), np.float32(0.0))
    L0t = V @ U.T                                      # (n, d) float64
    Xt = (L0t + S0t).astype(np.float32)
    X = Xt.T                                           # (d, n) Fortran view
    if not keep_parts:
        return Problem(X=X, L0=None, S0=None, rank=r)
    return Problem(X=X, L0=L0t.T, S0=S0t.T.astype(np.float64), rank=r)


def clustered_columns(d: int, n: int, c: int, seed: int, sparsity: float = 0.0) -> Problem:
    """Columns are exact copies of c distinct random base columns (a
    union of c rank-one groups), optionally with +-1 sparse corruption.
    truth_labels gives the group of every column (each group non-empty)."""
    g = _rng(seed)
    base = g.standard_normal((d, c))
    labels = np.concatenate([np.arange(c), g.integers(0, c, size=n - c)]).astype(np.int32)
    g.shuffle(labels)
    L0 = base[:, labels]
    S0 = np.zeros((d, n))
    if sparsity > 0:
        mask = g.random((d, n)) < sparsity
        S0 = np.where(mask, 2.0 * g.integers(0, 2, size=(d, n)) - 1.0, 0.0)
    X = np.asfortranarray((L0 + S0).astype(np.float32))
    return Problem(X=X, L0=L0, S0=S0, rank=c, truth_labels=labels)


def rings(d: int, n: int, c: int, seed: int, noise: float = 0.05) -> Problem:
    """Nonlinear groups: c concentric circles (radii 1..c) in a random 2-D
    plane of R^d, n points spread over them as evenly as possible at uniform
    angles, plus isotropic N(0, noise^2) noise.  No hyperplane or centroid
    rule separates the groups; a neighbourhood graph does.  truth_labels is
    the circle of every point.

    Drawing order: plane basis, angles, noise."""
    g = _rng(seed)
    Q, _ = np.linalg.qr(g.standard_normal((d, 2)))
    labels = (np.arange(n) % c).astype(np.int32)
    ang = g.uniform(0.0, 2.0 * np.pi, size=n)
    r = labels.astype(np.float64) + 1.0
    P2 = np.stack([r * np.cos(ang), r * np.sin(ang)])          # 2 x n
    X = Q @ P2 + noise * g.standard_normal((d, n))
    X = np.asfortranarray(X.astype(np.float32))
    return Problem(X=X, L0=None, S0=None, rank=c, truth_labels=labels)


def _smooth_image(g: np.random.Generator, h: int, w: int, sigma: float) -> np.ndarray:
    """Gaussian-blurred white noise, min-max scaled to [0, 1]."""
    noise = g.random((h, w))
    # Separable Gaussian blur with reflect padding (plain numpy convolution).
    rad = int(3 * sigma)
    t = np.arange(-rad, rad + 1)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    k /= k.sum()
    p = np.pad(noise, ((rad, rad), (0, 0)), mode="reflect")
    img = np.apply_along_axis(lambda col: np.convolve(col, k, mode="valid"), 0, p)
    p = np.pad(img, ((0, 0), (rad, rad)), mode="reflect")
    img = np.apply_along_axis(lambda row: np.convolve(row, k, mode="valid"), 1, p)
    lo, hi = img.min(), img.max()
    return (img - lo) / (hi - lo)


def video(n: int = 2000, height: int = 240, width: int = 320, n_backgrounds: int = 3,
          seed: int = 0, n_rects: int = 4, keep_parts: bool = False) -> Problem:
    """Surveillance-video stand-in: d = height*width pixels per column, n frames.

    Low-rank part: n_backgrounds smooth random images in [0, 1]; frames use
    them in contiguous segments (frame k uses background floor(k*B/n)).
    Foreground: n_rects axis-aligned rectangles with a fixed random texture
    (values U[0,1]) moving with constant velocity and bouncing off the
    borders; they occlude the background.  The rectangle sizes are drawn so
    that their total area is 2-10 % of the frame."""
    g = _rng(seed)
    d = height * width
    bgs = [_smooth_image(g, height, width, sigma=8.0) for _ in range(n_backgrounds)]
    frac = g.uniform(0.02, 0.10)
    shares = g.dirichlet(np.ones(n_rects)) * frac * d
    rects = []
    for a in shares:
        aspect = g.uniform(0.5, 2.0)
        rh = int(np.clip(np.sqrt(a * aspect), 2, height - 1))
        rw = int(np.clip(a / rh, 2, width - 1))
        y = g.uniform(0, height - rh)
        x = g.uniform(0, width - rw)
        vy = g.uniform(-3, 3)
        vx = g.uniform(-3, 3)
        tex = g.random((rh, rw)).astype(np.float32)
        rects.append([y, x, vy, vx, rh, rw, tex])
    Xt = np.empty((n, d), dtype=np.float32)            # (n, d) C == (d, n) F
    labels = np.empty(n, dtype=np.int32)
    for k in range(n):
        b = (k * n_backgrounds) // n
        labels[k] = b
        frame = bgs[b].astype(np.float32).copy()
        for rc in rects:
            y, x, vy, vx, rh, rw, tex = rc
            iy, ix = int(y), int(x)
            frame[iy:iy + rh, ix:ix + rw] = tex
            y, x = y + vy, x + vx
            if y < 0 or y > height - rh:
                vy = -vy
                y = min(max(y, 0.0), float(height - rh))
            if x < 0 or x > width - rw:
                vx = -vx
                x = min(max(x, 0.0), float(width - rw))
            rc[0], rc[1], rc[2], rc[3] = y, x, vy, vx
        Xt[k] = frame.reshape(-1)
    X = Xt.T
    if not keep_parts:
        return Problem(X=X, L0=None, S0=None, rank=n_backgrounds, truth_labels=labels)
    L0 = np.stack([bgs[b].reshape(-1) for b in labels], axis=1)
    return Problem(X=X, L0=L0, S0=X.astype(np.float64) - L0, rank=n_backgrounds,
                   truth_labels=labels)


@dataclass
class BatchEntry:
    d: int
    n: int
    r: int
    sparsity: float
    seed: int


def batch_table(count: int = 256, seed: int = 0, d_range=(200, 4000), n_range=(100, 2000),
                r_range=(2, 20), s_range=(0.01, 0.2)) -> list[BatchEntry]:
    """Shapes of a batch of uneven problems: d and n log-uniform, rank
    uniform on the integers, sparsity uniform."""
    g = _rng(seed)
    out = []
    for k in range(count):
        d = int(round(np.exp(g.uniform(np.log(d_range[0]), np.log(d_range[1])))))
        n = int(round(np.exp(g.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        r = int(g.integers(r_range[0], r_range[1] + 1))
        s = float(g.uniform(*s_range))
        out.append(BatchEntry(d=d, n=n, r=min(r, n), sparsity=s, seed=int(seed) * 100003 + k))
    return out


def batch_problem(e: BatchEntry, keep_parts: bool = False) -> Problem:
    return lowrank_sparse(e.d, e.n, e.r, e.sparsity, e.seed, keep_parts=keep_parts)


def warmstart_problem(seed: int, d: int = 2000, n: int = 2000, r_range=(10, 50),
                      s_range=(0.05, 0.2)) -> Problem:
    """Training / held-out problems for a learned warm start: d = n = 2000,
    rank uniform on 10..50, sparsity uniform on [0.05, 0.2]."""
    g = _rng(seed ^ 0x5EED)
    r = int(g.integers(r_range[0], r_range[1] + 1))
    s = float(g.uniform(*s_range))
    return lowrank_sparse(d, n, r, s, seed, keep_parts=False)
