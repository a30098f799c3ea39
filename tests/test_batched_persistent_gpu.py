"""The batched solve in one persistent launch (respca_solve_batched_persistent)
against the FP64 oracle, problem by problem, and against single solves.

Tolerance as the other parity tests: labels identical, L and S within 1e-5
relative Frobenius error and element by element within 1e-5 of the largest
entry, after a fixed iteration count from the same k-means++ seed.
"""
import numpy as np
import pytest

import oracle
from paper_1904_07497_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED = 7


def _dev(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float32).T)).cuda().T


def _host(t):
    return t.T.contiguous().cpu().numpy().T.astype(np.float64)


def _check_state(L, S, ref, X64, tol=1e-5):
    eL = np.linalg.norm(L - ref.L) / max(np.linalg.norm(ref.L), 1e-300)
    sS = max(np.linalg.norm(ref.S), 1e-2 * np.linalg.norm(X64))
    eS = np.linalg.norm(S - ref.S) / sS
    assert eL <= tol and eS <= tol, (eL, eS)
    assert np.abs(L - ref.L).max() <= tol * np.abs(ref.L).max() + 1e-7
    assert np.abs(S - ref.S).max() <= tol * max(np.abs(ref.S).max(), 1.0) + 1e-7


def _problems(shapes, max_iter, tol, p0s=None):
    out, host = [], []
    for k, (d, n, c, sp) in enumerate(shapes):
        pr = synth.lowrank_sparse(d, n, max(2, min(c, 20)), sp, seed=100 + k)
        X = _dev(pr.X)
        q = dict(X=X, c=c, L=torch.zeros((n, d), device="cuda").T, S=torch.zeros((n, d), device="cuda").T,
                 p=torch.full((n,), -5, device="cuda", dtype=torch.int32), tol=tol, max_iter=max_iter)
        if p0s is not None and p0s[k] is not None:
            q["p0"] = torch.from_numpy(p0s[k]).cuda()
        out.append(q)
        host.append(pr.X.astype(np.float64))
    return out, host


# ragged d and n; c covering the three column-item widths (c <= 16, <= 32, <= 64)
SHAPES = [(333, 257, 5, 0.05), (130, 90, 3, 0.10), (700, 300, 24, 0.05), (96, 200, 40, 0.10),
          (1030, 140, 12, 0.05), (64, 64, 1, 0.10)]


@pytest.fixture(scope="module")
def solver():
    from paper_1904_07497_gb300 import respca
    respca.load()
    s = respca.Solver(seed=SEED)
    yield s
    s.close()


def test_persistent_batch_matches_oracle_fixed_iterations(solver):
    from paper_1904_07497_gb300 import respca
    probs, X64s = _problems(SHAPES, 30, 0.0)
    stats, opt = respca.respca_solve_batched_persistent(solver.h, probs)
    torch.cuda.synchronize()
    assert opt.tuned_rows in (64, 128) and opt.tuned_ctas_per_sm in (1, 2)
    for q, X64, st in zip(probs, X64s, stats):
        ref, rs = oracle.solve(X64, q["c"], tol=0.0, max_iter=30, seed=SEED)
        assert st["iters"] == 30
        assert st["init_lloyd_passes"] == rs["init_lloyd_steps"]
        np.testing.assert_array_equal(q["p"].cpu().numpy(), ref.labels)
        _check_state(_host(q["L"]), _host(q["S"]), ref, X64)
        # FP32 squares in per-lane partial sums of at most 32 terms, then FP64:
        # relative error below 33 * 2^-24
        assert st["x_norm"] == pytest.approx(np.linalg.norm(X64), rel=2e-6)


def test_persistent_batch_to_tolerance(solver):
    """Solved to 1e-6: each problem stops within one iteration of the oracle,
    and matches the oracle at its own iteration count."""
    from paper_1904_07497_gb300 import respca
    probs, X64s = _problems(SHAPES[:4], 500, 1e-6)
    stats, _ = respca.respca_solve_batched_persistent(solver.h, probs)
    for q, X64, st in zip(probs, X64s, stats):
        assert st["converged"] == 1 and st["err"] <= 1e-6
        _, rs = oracle.solve(X64, q["c"], tol=1e-6, max_iter=500, seed=SEED)
        assert abs(st["iters"] - rs["iters"]) <= 1
        ref, _ = oracle.solve(X64, q["c"], tol=0.0, max_iter=st["iters"], seed=SEED)
        np.testing.assert_array_equal(q["p"].cpu().numpy(), ref.labels)
        _check_state(_host(q["L"]), _host(q["S"]), ref, X64)


def test_persistent_batch_agrees_with_single_solves(solver):
    """The C4-like family (d log-uniform, n log-uniform, rank = c): the same
    labels and iteration counts as respca_solve, L and S to FP32 rounding."""
    from paper_1904_07497_gb300 import respca
    entries = synth.batch_table(10, seed=5, d_range=(100, 900), n_range=(60, 500))
    probs, singles = [], []
    for e in entries:
        pr = synth.batch_problem(e)
        d, n = pr.X.shape
        X = _dev(pr.X)
        probs.append(dict(X=X, c=e.r, L=torch.zeros((n, d), device="cuda").T,
                          S=torch.zeros((n, d), device="cuda").T,
                          p=torch.zeros(n, device="cuda", dtype=torch.int32), tol=1e-6, max_iter=300))
        r = solver.solve(X, e.r, tol=1e-6, max_iter=300)
        singles.append((r.p.cpu().numpy(), _host(r.L), _host(r.S), r.stats))
    stats, _ = respca.respca_solve_batched_persistent(solver.h, probs)
    for q, st, (p1, L1, S1, s1) in zip(probs, stats, singles):
        np.testing.assert_array_equal(q["p"].cpu().numpy(), p1)
        assert st["iters"] == s1["iters"] and st["converged"] == 1
        L, S = _host(q["L"]), _host(q["S"])
        assert np.linalg.norm(L - L1) <= 1e-5 * np.linalg.norm(L1)
        assert np.linalg.norm(S - S1) <= 1e-5 * max(np.linalg.norm(S1), 1e-2 * np.linalg.norm(L1))


def test_persistent_batch_p0_and_per_problem_errors(solver):
    """p0 given for one problem; a NaN in another (that problem alone
    fails, with NONFINITE); the rest are still solved."""
    from paper_1904_07497_gb300 import respca
    shapes = SHAPES[:3]
    X64a = synth.lowrank_sparse(*shapes[0][:2], 5, 0.05, seed=100).X.astype(np.float64)
    p0a, _ = oracle.init_labels(X64a, shapes[0][2], seed=11)
    probs, X64s = _problems(shapes, 20, 0.0, p0s=[p0a, None, None])
    probs[1]["X"][3, 4] = float("nan")
    with pytest.raises(respca.RespcaError) as e:
        respca.respca_solve_batched_persistent(solver.h, probs)
    assert e.value.status == respca.RESPCA_ERR_NONFINITE_INPUT
    for k in (0, 2):
        ref, _ = oracle.solve(X64s[k], probs[k]["c"], tol=0.0, max_iter=20, seed=SEED,
                              p0=p0a if k == 0 else None)
        np.testing.assert_array_equal(probs[k]["p"].cpu().numpy(), ref.labels)
        _check_state(_host(probs[k]["L"]), _host(probs[k]["S"]), ref, X64s[k])


def test_persistent_batch_bounded_wait_times_out():
    """With a limit of one empty poll, a CTA that finds no work gives up: the
    launch ends (every CTA leaves at its next item boundary) and the call
    returns RESPCA_ERR_TIMEOUT; the handle and the GPU stay usable."""
    from paper_1904_07497_gb300 import respca
    s = respca.Solver(seed=SEED)
    probs, X64s = _problems([(100, 80, 3, 0.05), (90, 70, 2, 0.05)], 20, 0.0)
    opt = respca.respca_batch_options()
    opt.spin_limit = 1
    opt.tile_rows, opt.ctas_per_sm = 64, 1
    with pytest.raises(respca.RespcaError) as e:
        respca.respca_solve_batched_persistent(s.h, probs, opt)
    assert e.value.status == respca.RESPCA_ERR_TIMEOUT
    stats, _ = respca.respca_solve_batched_persistent(s.h, probs)
    for q, X64, st in zip(probs, X64s, stats):
        ref, _ = oracle.solve(X64, q["c"], tol=0.0, max_iter=20, seed=SEED)
        np.testing.assert_array_equal(q["p"].cpu().numpy(), ref.labels)
        _check_state(_host(q["L"]), _host(q["S"]), ref, X64)
    s.close()
