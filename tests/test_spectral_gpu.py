"""GPU parity of the spectral p step (Sec. 4.2's nonlinear alternative to
K-means) through the C ABI, against the FP64 oracle in oracle/spectral.py.

Labels are compared exactly (both sides run the same seeded k-means++ and
Lloyd on embeddings that differ only by a rotation within the eigenspace and
by rounding); sigma^2 and the c-th eigenvalue within 1e-5 relative; the
solver's iterates within the 1e-5 bound of the other parity tests.
"""
import time

import numpy as np
import pytest

import oracle
from oracle import spectral as osp
from paper_1904_07497_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCALE = 0.004   # sigma^2 / mean squared distance for circles of radii 1..c with 0.05 noise


def _dev(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float32).T)).cuda().T


def _host(t):
    return t.T.contiguous().cpu().numpy().T.astype(np.float64)


def _same_partition(a, b):
    m = {}
    for x, y in zip(np.asarray(a).tolist(), np.asarray(b).tolist()):
        if m.setdefault(x, y) != y:
            return False
    return len(set(m.values())) == len(m)


@pytest.fixture(scope="module")
def lib():
    from paper_1904_07497_gb300 import respca
    respca.load()
    return respca


@pytest.mark.parametrize("n,c,scale", [(600, 3, SCALE), (1200, 4, 0.002)])
def test_spectral_labels_match_oracle(lib, n, c, scale):
    pr = synth.rings(10, n, c, seed=3, noise=0.05)
    X64 = pr.X.astype(np.float64)
    s = lib.Solver(p_step=1, spectral_scale=scale)
    try:
        p, info = lib.respca_spectral_labels(s.h, _dev(pr.X), c)
    finally:
        s.close()
    p = p.cpu().numpy()
    _, w, _ = osp.embedding(X64, c, scale)
    _, _, s2 = osp.affinity(X64, scale)
    ref = osp.labels(X64, c, scale, seed=0)
    print(info)
    assert info["converged"]
    assert info["sigma2"] == pytest.approx(s2, rel=1e-5)
    assert info["theta_c"] == pytest.approx(w[0], abs=1e-5)
    assert np.array_equal(p, ref)
    assert _same_partition(p, pr.truth_labels)


def test_spectral_labels_block_case_and_timing(lib):
    """Four far-apart Gaussian blobs, n = 4096 in d = 64: the indicator
    subspace is found (labels = the blobs, same as the oracle); prints the
    time of one spectral p step."""
    g = np.random.default_rng(12)
    c, n, d = 4, 4096, 64
    truth = g.integers(0, c, size=n)
    centers = 10.0 * g.standard_normal((d, c))
    X = (centers[:, truth] + g.standard_normal((d, n))).astype(np.float32)
    s = lib.Solver(p_step=1, spectral_scale=0.05)
    try:
        Xd = _dev(X)
        p, info = lib.respca_spectral_labels(s.h, Xd, c)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p, info = lib.respca_spectral_labels(s.h, Xd, c)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    finally:
        s.close()
    print(f"spectral p step n={n} d={d} c={c}: {dt * 1e3:.2f} ms, {info}")
    p = p.cpu().numpy()
    assert info["converged"]
    assert _same_partition(p, truth)
    assert np.array_equal(p, osp.labels(X.astype(np.float64), c, 0.05, seed=0))


def test_spectral_solve_matches_oracle_iterations(lib):
    """Five iterations of the solver with the spectral p step from the
    spectral labels of X, against the oracle's iteration with the same p step."""
    pr = synth.rings(10, 600, 3, seed=5, noise=0.05)
    X64 = pr.X.astype(np.float64)
    d, n = X64.shape
    c, T, rho0 = 3, 5, 0.5
    lam = float(np.sqrt(max(d, n)))
    s = lib.Solver(p_step=1, spectral_scale=SCALE, rho0=rho0)
    try:
        L = torch.zeros((n, d), device="cuda").T
        S = torch.zeros((n, d), device="cuda").T
        p = torch.empty(n, device="cuda", dtype=torch.int32)
        st = lib.respca_solve(s.h, _dev(pr.X), c, L, S, p, tol=0.0, max_iter=T)
    finally:
        s.close()
    assert st["iters"] == T
    p0 = osp.labels(X64, c, SCALE, seed=0)
    ref = oracle.State(np.zeros((d, n), order="F"), np.zeros((d, n), order="F"), np.zeros((d, n), order="F"),
                       p0.astype(np.int32), rho0)
    for _ in range(T):
        ref, _ = osp.iteration(X64, ref, c, lam, SCALE, seed=0)
    Lg, Sg = _host(L), _host(S)
    eL = np.linalg.norm(Lg - ref.L) / np.linalg.norm(ref.L)
    eS = np.linalg.norm(Sg - ref.S) / max(np.linalg.norm(ref.S), 1e-2 * np.linalg.norm(X64))
    print(f"L rel {eL:.2e} S rel {eS:.2e}, S active {np.mean(ref.S != 0):.3f}")
    assert np.array_equal(p.cpu().numpy(), ref.labels)
    assert eL <= 1e-5 and eS <= 1e-5


def test_spectral_solve_keeps_the_circles(lib):
    """A whole solve to 1e-6 on concentric circles: with the spectral p step
    the groups are the circles; with K-means they are not."""
    pr = synth.rings(10, 600, 3, seed=7, noise=0.05)
    d, n = pr.X.shape
    out = {}
    for ps in (0, 1):
        s = lib.Solver(p_step=ps, spectral_scale=SCALE)
        try:
            r = s.solve(_dev(pr.X), 3, tol=1e-6)
        finally:
            s.close()
        out[ps] = r
        print(ps, r.stats["iters"], r.stats["converged"], r.stats["ms_total"])
    assert out[1].stats["converged"]
    assert _same_partition(out[1].p.cpu().numpy(), pr.truth_labels)
    assert not _same_partition(out[0].p.cpu().numpy(), pr.truth_labels)
