"""The bf16 phase of the precision = 1 schedule (BF16 storage of L, S, Theta
and X, FP32 arithmetic, then FP32 continuation).

The bf16 phase is pinned element by element against the oracle's own step
functions (FP64) with the same BF16 rounding applied where the GPU stores:
X once, L after the L step (the p and S steps read the stored L), S and
Theta after their steps.  The two differ only where an FP32 and an FP64
value fall on different sides of a BF16 rounding boundary, so elements agree
to one BF16 ulp and almost all agree exactly.
"""
import numpy as np
import pytest

import oracle
from paper_1904_07497_gb300 import synth

torch = pytest.importorskip("torch")


def bf16(a):
    """Round to BF16 (nearest, ties to even) through FP32, as the GPU stores."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    return np.asfortranarray(out.reshape(f.shape))


def bf16_ulp(a):
    """Spacing of BF16 numbers at |a| (8 significant bits)."""
    m = np.abs(np.asarray(a, dtype=np.float64))
    e = np.floor(np.log2(np.where(m > 0, m, 1.0)))
    return np.where(m > 0, 2.0 ** (e - 7), 0.0)


def test_bf16_rounding_matches_torch():
    g = np.random.default_rng(0)
    x = np.concatenate([g.standard_normal(5000) * 10.0 ** g.integers(-6, 6, 5000),
                        [0.0, -0.0, 1.0, -1.0, 1.00390625, 1.01171875]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(bf16(x).ravel(), ref)


def _emulate(X32, p0, c, lam, rho, T, kappa=1.5):
    Xb = bf16(X32)
    d, n = Xb.shape
    L = np.zeros((d, n), order="F")
    S = np.zeros((d, n), order="F")
    Th = np.zeros((d, n), order="F")
    for _ in range(T):
        Lf, _, _ = oracle.l_step(Xb, S, Th, rho, lam, p0, c)    # Eq. (18)
        Lr = bf16(Lf)
        Sf = oracle.s_step(Xb, Lr, Th, rho)                    # Eq. (24) on the stored L
        Thf = oracle.theta_step(Xb, Lr, Sf, Th, rho)            # Eq. (25)
        L, S, Th = Lr, bf16(Sf), bf16(Thf)
        rho *= kappa
    return L, S


@pytest.mark.gpu
@pytest.mark.parametrize("T", [1, 2, 3])
def test_bf16_phase_matches_rounded_oracle_steps(T):
    from paper_1904_07497_gb300 import respca
    oracle.build()
    pr = synth.clustered_columns(256, 200, 4, seed=11, sparsity=0.05)
    X32 = pr.X.astype(np.float32)
    d, n = X32.shape
    c = 4
    lam = float(np.sqrt(max(d, n)))
    s = respca.Solver(seed=1, rho0=3.0, ramp_skip=False, precision=1, switch_tol=0.0)
    X = torch.from_numpy(np.ascontiguousarray(X32.T)).cuda().T
    p0 = torch.from_numpy(pr.truth_labels.astype(np.int32)).cuda()
    res = s.solve(X, c, tol=0.0, max_iter=T, p0=p0)
    torch.cuda.synchronize()
    assert res.stats["bf16_iters"] == T
    np.testing.assert_array_equal(res.p.cpu().numpy(), pr.truth_labels)
    Lg = res.L.T.contiguous().cpu().numpy().T.astype(np.float64)
    Sg = res.S.T.contiguous().cpu().numpy().T.astype(np.float64)
    s.close()
    Le, Se = _emulate(X32, pr.truth_labels, c, lam, 3.0, T)
    assert np.count_nonzero(Se) > 0.01 * Se.size          # the S step is active
    for G, E in ((Lg, Le), (Sg, Se)):
        diff = np.abs(G - E)
        assert np.all(diff <= bf16_ulp(E) * (1 + 1e-9) + 1e-30), diff.max()
        assert np.count_nonzero(diff) <= 0.02 * diff.size


@pytest.mark.gpu
def test_bf16_then_fp32_reaches_tolerance():
    """precision = 1 runs a bf16 phase, widens the state and reaches tol in
    FP32; its answer is reported against the FP64 oracle's beside the FP32
    path's (the iteration is path dependent, so both are compared at their
    own convergence)."""
    from paper_1904_07497_gb300 import respca
    oracle.build()
    pr = synth.lowrank_sparse(600, 400, 10, 0.1, seed=5)
    X32 = pr.X.astype(np.float32)
    c = 10
    X = torch.from_numpy(np.ascontiguousarray(X32.T)).cuda().T
    out = {}
    for prec in (0, 1):
        s = respca.Solver(seed=2, precision=prec)
        r = s.solve(X, c, tol=1e-6, max_iter=500)
        torch.cuda.synchronize()
        out[prec] = (r.L.T.contiguous().cpu().numpy().T.astype(np.float64),
                     r.S.T.contiguous().cpu().numpy().T.astype(np.float64), r.stats)
        s.close()
    st0, st1 = out[0][2], out[1][2]
    assert st0["converged"] == 1 and st1["converged"] == 1
    assert st0["bf16_iters"] == 0 and st1["bf16_iters"] >= 1
    assert st1["err"] <= 1e-6
    ost, _ = oracle.solve(X32.astype(np.float64), c, tol=1e-6, max_iter=500, seed=2)
    Lo, So = ost.L, ost.S
    nX = np.linalg.norm(X32)
    e = {k: (np.linalg.norm(out[k][0] - Lo) / nX, np.linalg.norm(out[k][1] - So) / nX) for k in (0, 1)}
    print("rel. to ||X||: FP32 path L %.2e S %.2e | bf16 + FP32 path L %.2e S %.2e"
          % (e[0][0], e[0][1], e[1][0], e[1][1]))
    assert e[0][0] <= 1e-4 and e[0][1] <= 1e-4
    assert e[1][0] <= 1e-2 and e[1][1] <= 1e-2
