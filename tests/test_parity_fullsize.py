"""Parity at the benchmark's full size: d = n = 10^4, rank 50, 10 % +-1
corruption, c = 50 and the rank bound c = 100 (400 MB per FP32 array), in the
launch configuration bench.py times (tensor-core search over every column,
152 CTAs; c = 100 takes the two-slab centroid layout).

Two iterations from the zero state with seeded labels and rho0 = 1 (so the
S step is active from the first iteration), at most 3 Lloyd passes per p
step (so the oracle's passes over 10^8 elements stay few; it also exercises
the device-run Lloyd loop stopping at its cap), run on the GPU and in the
FP64 oracle; labels must agree exactly and L, S element by element within the
FP32 tolerance of the other parity tests.  The oracle's inputs come from the
seeded generator only.  The oracle needs one to two minutes of one host core
per case.
"""
import numpy as np
import pytest

import oracle
from paper_1904_07497_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.mark.parametrize("c", [50, 100])
def test_two_iterations_at_full_size(c):
    from paper_1904_07497_gb300 import respca
    oracle.build()
    d = n = 10000
    T, rho0 = 2, 1.0
    pr = synth.lowrank_sparse(d, n, 50, 0.10, seed=0, keep_parts=False)
    p0 = (np.random.default_rng(123).integers(0, c, n)).astype(np.int32)
    p0[:c] = np.arange(c)
    X = torch.from_numpy(np.ascontiguousarray(pr.X.T)).cuda().T
    s = respca.Solver(seed=0, rho0=rho0, ramp_skip=False, kmeans_max_iter=3)
    r = s.solve(X, c, tol=0.0, max_iter=T, p0=torch.from_numpy(p0).cuda())
    torch.cuda.synchronize()
    pg = r.p.cpu().numpy()
    Lg = r.L.T.contiguous().cpu().numpy().T
    Sg = r.S.T.contiguous().cpu().numpy().T
    s.close()
    del X
    X64 = pr.X.astype(np.float64)
    del pr
    ref, _ = oracle.solve(X64, c, rho0=rho0, tol=0.0, max_iter=T, p0=p0, km_max=3)
    np.testing.assert_array_equal(pg, ref.labels)
    assert np.count_nonzero(ref.S) > 0.01 * ref.S.size          # S active
    for G, E, floor in ((Lg, ref.L, 0.0), (Sg, ref.S, 1.0)):
        scale = max(np.abs(E).max(), floor)
        err = 0.0
        for j0 in range(0, n, 1000):                              # bounded host memory
            diff = np.abs(G[:, j0:j0 + 1000].astype(np.float64) - E[:, j0:j0 + 1000])
            err = max(err, diff.max())
        assert err <= 1e-5 * scale + 1e-7, err
    eL = np.linalg.norm(Lg.astype(np.float64) - ref.L) / np.linalg.norm(ref.L)
    assert eL <= 1e-5
