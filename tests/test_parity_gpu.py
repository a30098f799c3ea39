"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle.

Tolerance: the FP32 path must match the FP64 oracle within 1e-5 relative
Frobenius error after a fixed iteration count, labels identical.  Element by
element, |L_gpu - L_oracle| <= 1e-5 * max|L_oracle| (and likewise for S);
Theta is compared through Theta/rho, the quantity the iteration uses.
"""
import numpy as np
import pytest

import oracle
from paper_1904_07497_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(A, dtype=None):
    """numpy (d, n) -> column-major CUDA tensor (d, n)."""
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(A).T))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda().T


def _host(t):
    return t.T.contiguous().cpu().numpy().T.astype(np.float64)


@pytest.fixture(scope="module")
def solver():
    from paper_1904_07497_gb300 import respca
    respca.load()
    s = respca.Solver(seed=3)
    yield s
    s.close()


def _rel(a, b, scale=None):
    den = np.linalg.norm(b) if scale is None else scale
    return np.linalg.norm(a - b) / max(den, 1e-300)


def _check_state(L, S, ref, X64, tol=1e-5):
    eL = _rel(L, ref.L)
    sS = max(np.linalg.norm(ref.S), 1e-2 * np.linalg.norm(X64))
    eS = _rel(S, ref.S, sS)
    assert eL <= tol, f"L rel err {eL:.3e}"
    assert eS <= tol, f"S rel err {eS:.3e}"
    assert np.abs(L - ref.L).max() <= tol * np.abs(ref.L).max() + 1e-7
    assert np.abs(S - ref.S).max() <= tol * max(np.abs(ref.S).max(), 1.0) + 1e-7
    return eL, eS


def _run(solver, X32, c, T, p0, warm=None, tol=0.0):
    from paper_1904_07497_gb300 import respca
    d, n = X32.shape
    X = _dev(X32)
    L = torch.zeros((n, d), device="cuda").T
    S = torch.zeros((n, d), device="cuda").T
    p = torch.zeros(n, device="cuda", dtype=torch.int32)
    wst = None
    Th = None
    if warm is not None:
        L.copy_(_dev(warm.L.astype(np.float32)))
        S.copy_(_dev(warm.S.astype(np.float32)))
        p.copy_(torch.from_numpy(warm.labels).cuda())
        Th = torch.zeros((n, d), device="cuda").T
        Th.copy_(_dev(warm.Theta.astype(np.float32)))
        wst = respca.respca_warm(Theta=Th.data_ptr(), rho=warm.rho, warm=1)
    st = respca.respca_solve(solver.h, X, c, L, S, p, tol=tol, max_iter=T,
                             p0=None if p0 is None else torch.from_numpy(p0).cuda(), warm=wst)
    torch.cuda.synchronize()
    out = dict(L=_host(L), S=_host(S), p=p.cpu().numpy(), stats=st)
    if Th is not None:
        out["Theta"] = _host(Th)
        out["rho"] = wst.rho
    return out


def _rounded(state):
    s = state.copy()
    s.L = s.L.astype(np.float32).astype(np.float64)
    s.S = s.S.astype(np.float32).astype(np.float64)
    s.Theta = s.Theta.astype(np.float32).astype(np.float64)
    return s


# ------------------------------------------------------------------ one iteration
@pytest.mark.parametrize("T", [0, 12, 22, 26, 31, 40])
def test_single_iteration_from_oracle_state(solver, T):
    """From the same (FP32-representable) state, one GPU iteration equals one
    oracle iteration: ramp (T <= 20), S activation (22), label churn (26-31),
    convergence (40)."""
    pr = synth.lowrank_sparse(500, 500, 25, 0.05, seed=0)
    X64 = pr.X.astype(np.float64)
    c, lam = 25, np.sqrt(500)
    p0, _ = oracle.init_labels(X64, c, seed=0)
    st = oracle.State(np.zeros((500, 500), order="F"), np.zeros((500, 500), order="F"),
                      np.zeros((500, 500), order="F"), p0, 1e-4)
    for _ in range(T):
        st, *_ = oracle.iteration(X64, st, c, lam)
    st = _rounded(st)
    ref, norms, _, _ = oracle.iteration(X64, st, c, lam)
    got = _run(solver, pr.X, c, 1, None, warm=st)
    np.testing.assert_array_equal(got["p"], ref.labels)
    _check_state(got["L"], got["S"], ref, X64)
    tr_ref = ref.Theta / st.rho
    tr_got = got["Theta"] / st.rho
    assert np.abs(tr_got - tr_ref).max() <= 1e-5 * max(np.abs(X64).max(), 1.0)
    assert got["rho"] == pytest.approx(st.rho * 1.5, rel=1e-15)
    e_ref = max(norms) / np.linalg.norm(X64)
    assert got["stats"]["err"] == pytest.approx(e_ref, rel=1e-4, abs=1e-7)


# ------------------------------------------------------------------ fixed count
@pytest.mark.parametrize("T", [30, 60])
def test_c1_fixed_iterations(solver, T):
    """d = n = 500, rank 25, 5 % +-1 corruption, c = 25: 30 iterations (S
    active, labels moving) and 60 (past convergence to 1e-6)."""
    pr = synth.lowrank_sparse(500, 500, 25, 0.05, seed=0)
    X64 = pr.X.astype(np.float64)
    p0, _ = oracle.init_labels(X64, 25, seed=0)
    ref, rs = oracle.solve(X64, 25, tol=0.0, max_iter=T, p0=p0)
    got = _run(solver, pr.X, 25, T, p0)
    assert got["stats"]["iters"] == T
    np.testing.assert_array_equal(got["p"], ref.labels)
    _check_state(got["L"], got["S"], ref, X64)


def test_c1_to_tolerance(solver):
    """Solve to the Sec. 5 criterion at 1e-6: the GPU stops within one
    iteration of the oracle and its result matches the oracle's at the same
    iteration count."""
    pr = synth.lowrank_sparse(500, 500, 25, 0.05, seed=1)
    X64 = pr.X.astype(np.float64)
    p0, _ = oracle.init_labels(X64, 25, seed=1)
    ref, rs = oracle.solve(X64, 25, tol=1e-6, max_iter=500, p0=p0)
    got = _run(solver, pr.X, 25, 500, p0, tol=1e-6)
    assert got["stats"]["converged"] == 1
    assert abs(got["stats"]["iters"] - rs["iters"]) <= 1
    ref2, _ = oracle.solve(X64, 25, tol=0.0, max_iter=got["stats"]["iters"], p0=p0)
    np.testing.assert_array_equal(got["p"], ref2.labels)
    _check_state(got["L"], got["S"], ref2, X64)
    assert np.linalg.norm(X64 - got["L"] - got["S"]) / np.linalg.norm(X64) <= 2e-6


# ------------------------------------------------------------------ shapes
@pytest.mark.parametrize("d,n,c,rank,sp", [
    (37, 41, 3, 3, 0.1),        # scalar path (d % 4 != 0), single partial tile per cluster
    (1203, 70, 4, 4, 0.05),     # three row chunks with a ragged tail, scalar path
    (1028, 97, 5, 5, 0.1),      # vector path, ragged chunk tail, partial tiles
    (64, 300, 1, 4, 0.05),      # one cluster
    (48, 40, 40, 3, 0.05),      # c = n: every column its own cluster
    (256, 200, 130, 8, 0.05),   # more clusters than one 64-wide register block
])
def test_shapes_and_edges(solver, d, n, c, rank, sp):
    pr = synth.lowrank_sparse(d, n, rank, sp, seed=d + n + c)
    X64 = pr.X.astype(np.float64)
    p0 = np.arange(n, dtype=np.int32) if c == n else oracle.init_labels(X64, c, seed=2)[0]
    ref, _ = oracle.solve(X64, c, tol=0.0, max_iter=35, p0=p0)
    got = _run(solver, pr.X, c, 35, p0)
    np.testing.assert_array_equal(got["p"], ref.labels)
    _check_state(got["L"], got["S"], ref, X64)


def test_video_shaped(solver):
    """Tall-skinny frames-as-columns with 3 backgrounds (reduced size)."""
    pr = synth.video(n=240, height=48, width=64, n_backgrounds=3, seed=4)
    X64 = pr.X.astype(np.float64)
    p0, _ = oracle.init_labels(X64, 3, seed=1)
    ref, rs = oracle.solve(X64, 3, tol=0.0, max_iter=40, p0=p0)
    got = _run(solver, pr.X, 3, 40, p0)
    np.testing.assert_array_equal(got["p"], ref.labels)
    _check_state(got["L"], got["S"], ref, X64)


@pytest.mark.parametrize("dt", ["bf16", "f32"])
def test_tall_video_frames(solver, dt):
    """Full-size video frames (d = 76800 = 240 x 320 pixels) as columns: each
    column spans many row chunks of the fused pass, whose partial sums are
    combined across CTAs.  64 frames, 3 backgrounds, X in BF16 (the video
    workload's storage) or FP32; the oracle runs on the same stored values."""
    from paper_1904_07497_gb300 import respca
    pr = synth.video(n=64, height=240, width=320, n_backgrounds=3, seed=6)
    tdt = torch.bfloat16 if dt == "bf16" else torch.float32
    Xh = torch.from_numpy(np.ascontiguousarray(pr.X.T)).to(tdt)
    X64 = Xh.float().numpy().T.astype(np.float64)
    p0, _ = oracle.init_labels(X64, 3, seed=1)
    ref, _ = oracle.solve(X64, 3, tol=0.0, max_iter=30, p0=p0)
    X = Xh.cuda().T
    d, n = X.shape
    L = torch.zeros((n, d), device="cuda").T
    S = torch.zeros((n, d), device="cuda").T
    p = torch.zeros(n, device="cuda", dtype=torch.int32)
    st = respca.respca_solve(solver.h, X, 3, L, S, p, tol=0.0, max_iter=30,
                             p0=torch.from_numpy(p0).cuda())
    assert st["iters"] == 30
    assert np.count_nonzero(ref.S) > 0
    np.testing.assert_array_equal(p.cpu().numpy(), ref.labels)
    _check_state(_host(L), _host(S), ref, X64)


@pytest.mark.parametrize("dt", ["bf16", "f16"])
def test_half_precision_x(solver, dt):
    """X stored in BF16 / FP16: the oracle runs on the same rounded values."""
    from paper_1904_07497_gb300 import respca
    tdt = torch.bfloat16 if dt == "bf16" else torch.float16
    pr = synth.lowrank_sparse(256, 180, 6, 0.05, seed=9)
    Xh = torch.from_numpy(np.ascontiguousarray(pr.X.T)).to(tdt)
    X64 = Xh.float().numpy().T.astype(np.float64)
    p0, _ = oracle.init_labels(X64, 6, seed=1)
    ref, _ = oracle.solve(X64, 6, tol=0.0, max_iter=30, p0=p0)
    X = Xh.cuda().T
    d, n = X.shape
    L = torch.zeros((n, d), device="cuda").T
    S = torch.zeros((n, d), device="cuda").T
    p = torch.zeros(n, device="cuda", dtype=torch.int32)
    respca.respca_solve(solver.h, X, 6, L, S, p, tol=0.0, max_iter=30, p0=torch.from_numpy(p0).cuda())
    np.testing.assert_array_equal(p.cpu().numpy(), ref.labels)
    _check_state(_host(L), _host(S), ref, X64)


# ------------------------------------------------------------------ initial labels
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_init_labels_match_oracle(seed):
    from paper_1904_07497_gb300 import respca
    s = respca.Solver(seed=seed)
    pr = synth.lowrank_sparse(300, 260, 12, 0.05, seed=30 + seed)
    X64 = pr.X.astype(np.float64)
    want, steps = oracle.init_labels(X64, 12, seed=seed)
    p, passes = s.init_labels(_dev(pr.X), 12)
    s.close()
    np.testing.assert_array_equal(p.cpu().numpy(), want)
    assert passes == steps


def test_full_solve_without_p0(solver):
    """Cold start with the library's own k-means++ + Lloyd initial labels."""
    from paper_1904_07497_gb300 import respca
    s = respca.Solver(seed=5)
    pr = synth.lowrank_sparse(200, 150, 5, 0.05, seed=44)
    X64 = pr.X.astype(np.float64)
    ref, _ = oracle.solve(X64, 5, tol=0.0, max_iter=40, seed=5)
    res = s.solve(_dev(pr.X), 5, tol=0.0, max_iter=40)
    s.close()
    np.testing.assert_array_equal(res.p.cpu().numpy(), ref.labels)
    _check_state(_host(res.L), _host(res.S), ref, X64)


# ------------------------------------------------------------------ host API, errors
def test_solve_host_matches_device(solver):
    from paper_1904_07497_gb300 import respca
    pr = synth.lowrank_sparse(130, 90, 4, 0.1, seed=50)
    p0, _ = oracle.init_labels(pr.X.astype(np.float64), 4, seed=0)
    dev = _run(solver, pr.X, 4, 25, p0)
    Xh = torch.from_numpy(np.ascontiguousarray(pr.X.T)).T
    L = torch.zeros((90, 130)).T
    S = torch.zeros((90, 130)).T
    p = torch.zeros(90, dtype=torch.int32)
    respca.respca_solve_host(solver.h, Xh, 4, L, S, p, tol=0.0, max_iter=25, p0=torch.from_numpy(p0))
    np.testing.assert_array_equal(p.numpy(), dev["p"])
    np.testing.assert_array_equal(L.numpy().astype(np.float64), dev["L"])
    np.testing.assert_array_equal(S.numpy().astype(np.float64), dev["S"])


def test_zero_input(solver):
    got = _run(solver, np.zeros((40, 30), dtype=np.float32), 3, 10, None)
    assert np.all(got["L"] == 0) and np.all(got["S"] == 0)
    assert got["stats"]["iters"] == 0 and got["stats"]["converged"] == 1


def test_errors(solver):
    from paper_1904_07497_gb300 import respca
    X = np.ones((20, 10), dtype=np.float32)
    X[3, 4] = np.nan
    with pytest.raises(respca.RespcaError) as e:
        _run(solver, X, 2, 5, None)
    assert e.value.status == respca.RESPCA_ERR_NONFINITE_INPUT
    X[3, 4] = 1.0
    with pytest.raises(respca.RespcaError) as e:
        _run(solver, X, 11, 5, None)
    assert e.value.status == respca.RESPCA_ERR_INVALID_ARG
    with pytest.raises(respca.RespcaError) as e:
        _run(solver, X, 2, 5, np.array([0, 1, 2] + [0] * 7, dtype=np.int32))
    assert e.value.status == respca.RESPCA_ERR_INVALID_ARG
    # the handle still works after errors
    got = _run(solver, X, 2, 3, None)
    assert got["stats"]["iters"] >= 1


def test_batched_matches_single(solver):
    from paper_1904_07497_gb300 import respca
    probs, singles = [], []
    for k, e in enumerate(synth.batch_table(4, seed=3, d_range=(60, 300), n_range=(40, 200))):
        pr = synth.batch_problem(e)
        d, n = pr.X.shape
        X = _dev(pr.X)
        q = dict(X=X, c=e.r, L=torch.zeros((n, d), device="cuda").T,
                 S=torch.zeros((n, d), device="cuda").T,
                 p=torch.zeros(n, device="cuda", dtype=torch.int32), tol=0.0, max_iter=20)
        probs.append(q)
        singles.append(_run(solver, pr.X, e.r, 20, None))
    respca.respca_solve_batched(solver.h, probs)
    for q, s in zip(probs, singles):
        np.testing.assert_array_equal(q["p"].cpu().numpy(), s["p"])
        np.testing.assert_array_equal(_host(q["L"]), s["L"])


def _batch(entries, lanes, tol, max_iter):
    from paper_1904_07497_gb300 import respca
    s = respca.Solver(seed=7, batch_lanes=lanes)
    probs = []
    for e in entries:
        pr = synth.batch_problem(e)
        d, n = pr.X.shape
        probs.append(dict(X=_dev(pr.X), c=e.r, L=torch.zeros((n, d), device="cuda").T,
                          S=torch.zeros((n, d), device="cuda").T,
                          p=torch.zeros(n, device="cuda", dtype=torch.int32), tol=tol,
                          max_iter=max_iter))
    stats = respca.respca_solve_batched(s.h, probs)
    torch.cuda.synchronize()
    out = [(q["p"].cpu().numpy(), _host(q["L"]), _host(q["S"]), st) for q, st in zip(probs, stats)]
    s.close()
    return out


def test_batched_lanes_match_one_at_a_time():
    """Concurrent lanes (each with its own stream and workspace, problems taken
    largest first) give every problem exactly its one-at-a-time result."""
    entries = synth.batch_table(12, seed=5, d_range=(100, 900), n_range=(60, 500))
    seq = _batch(entries, 1, 1e-6, 300)
    par = _batch(entries, 5, 1e-6, 300)
    for a, b in zip(seq, par):
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])
        np.testing.assert_array_equal(a[2], b[2])
        assert a[3]["iters"] == b[3]["iters"] and a[3]["converged"] == b[3]["converged"] == 1
        assert a[3]["err"] == b[3]["err"]


# ------------------------------------------------------------------ search paths
def _solve_impl(impl, X32, c, T, p0=None, seed=4, dtype=None):
    from paper_1904_07497_gb300 import respca
    s = respca.Solver(seed=seed, search_impl=impl)
    X = _dev(X32, dtype)
    res = s.solve(X, c, tol=0.0, max_iter=T, p0=None if p0 is None else torch.from_numpy(p0).cuda())
    torch.cuda.synchronize()
    out = (res.p.cpu().numpy(), _host(res.L), _host(res.S), res.stats)
    s.close()
    return out


@pytest.mark.parametrize("d,n,c,T", [
    (2048, 700, 50, 40),     # tensor-core search, several d splits
    (333, 300, 20, 35),      # ragged d (scalar loads), partial 128-column tile
    (512, 600, 256, 30),     # largest tensor-core centroid count
    (256, 400, 257, 25),     # one above: the CUDA-core kernel
])
def test_search_paths_agree(d, n, c, T):
    """The tensor-core search and the CUDA-core search both return the exact
    argmin of the stored values, so whole solves agree bit for bit."""
    pr = synth.lowrank_sparse(d, n, min(c, 40), 0.1, seed=d + c)
    a = _solve_impl(0, pr.X, c, T)
    b = _solve_impl(1, pr.X, c, T)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2], b[2])
    assert a[3]["lloyd_passes"] == b[3]["lloyd_passes"]


def test_search_paths_agree_bf16_x():
    pr = synth.lowrank_sparse(640, 500, 16, 0.1, seed=91)
    a = _solve_impl(0, pr.X, 16, 30, dtype=torch.bfloat16)
    b = _solve_impl(1, pr.X, 16, 30, dtype=torch.bfloat16)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


# ------------------------------------------------------------------ 16-bit search operand
def _solve_cfg(X32, c, T, dtype=None, tol=0.0, timing=True, **cfg):
    from paper_1904_07497_gb300 import respca
    s = respca.Solver(seed=4, timing=timing, **cfg)
    res = s.solve(_dev(X32, dtype), c, tol=tol, max_iter=T)
    torch.cuda.synchronize()
    out = (res.p.cpu().numpy(), _host(res.L), _host(res.S), res.stats)
    s.close()
    return out


@pytest.mark.parametrize("d,n,c,T", [
    (2048, 1300, 50, 40),    # stacked centroids (c <= 64), several 256-column tiles, ragged last tile
    (780, 777, 33, 35),      # d not a multiple of 64 (the last slab reads zeros past d), ragged n
    (1000, 900, 100, 30),    # two A slabs (64 < c <= 128)
])
def test_fp16_copy_search_matches_fp32_search(d, n, c, T):
    """With FP32 state the p step's all-column search reads an FP16 copy
    fp16(s L) of L, widens each decision by ||L_j - fp16(s L_j) / s|| and the
    centroids' split error, and re-decides near ties from the FP32 L: labels
    and state equal the FP32-operand tensor-core search and
    the CUDA-core search bit for bit.  The timing mode counts the all-column
    passes that read the copy."""
    pr = synth.lowrank_sparse(d, n, min(c, 40), 0.1, seed=d + n)
    a = _solve_cfg(pr.X, c, T, search_impl=0)
    b = _solve_cfg(pr.X, c, T, search_impl=2)
    r = _solve_cfg(pr.X, c, T, search_impl=1)
    assert a[3]["dense16_passes"] > 0, "the all-column search never read the copy"
    assert b[3]["dense_passes"] > 0 and b[3]["dense16_passes"] == 0
    assert a[3]["rechecked_columns"] > 0, "no near tie was re-decided"
    for x in (b, r):
        np.testing.assert_array_equal(a[0], x[0])
        np.testing.assert_array_equal(a[1], x[1])
        np.testing.assert_array_equal(a[2], x[2])
    assert a[3]["lloyd_passes"] == b[3]["lloyd_passes"] == r[3]["lloyd_passes"]


def test_16bit_data_search_matches_cuda_core():
    """16-bit data searched directly (no widening term): BF16 X for the initial
    labels' all-column passes, and BF16 state in the bf16 phase (precision =
    1).  Labels and state equal the CUDA-core search's."""
    pr = synth.lowrank_sparse(1024, 900, 30, 0.1, seed=17)
    kw = dict(precision=1, switch_tol=0.0, ramp_skip=False)
    a = _solve_cfg(pr.X, 30, 20, dtype=torch.bfloat16, search_impl=0, **kw)
    r = _solve_cfg(pr.X, 30, 20, dtype=torch.bfloat16, search_impl=1, **kw)
    assert a[3]["bf16_iters"] > 0
    assert a[3]["dense16_passes"] > 0, "the all-column search never read BF16 data"
    np.testing.assert_array_equal(a[0], r[0])
    np.testing.assert_array_equal(a[1], r[1])
    np.testing.assert_array_equal(a[2], r[2])


def test_fp16_copy_search_device_loop():
    """Large enough for the device-run Lloyd loop (a captured graph, timing
    off): the copy-operand solve equals the CUDA-core solve bit for bit."""
    pr = synth.lowrank_sparse(2048, 2200, 40, 0.1, seed=23)
    a = _solve_cfg(pr.X, 48, 30, timing=False, search_impl=0)
    r = _solve_cfg(pr.X, 48, 30, timing=False, search_impl=1)
    for k in range(3):
        np.testing.assert_array_equal(a[k], r[k])
    assert a[3]["lloyd_passes"] == r[3]["lloyd_passes"]


def test_fp16_copy_search_full_size():
    """At the d = n = 10^4, rank 50, c = 50 workload, in the launch
    configuration bench.py times (device-run Lloyd loop, timing off), the solve
    with the FP16 copy equals the FP32-operand solve bit for bit: labels, L, S
    and the iteration count to 1e-6."""
    pr = synth.lowrank_sparse(10000, 10000, 50, 0.10, 0, keep_parts=False)
    a = _solve_cfg(pr.X, 50, 500, tol=1e-6, timing=False, search_impl=0)
    b = _solve_cfg(pr.X, 50, 500, tol=1e-6, timing=False, search_impl=2)
    assert a[3]["converged"] == b[3]["converged"] == 1
    assert a[3]["iters"] == b[3]["iters"]
    assert a[3]["lloyd_passes"] == b[3]["lloyd_passes"]
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2], b[2])


# ------------------------------------------------------------------ two-slab dense search
@pytest.mark.parametrize("d,n,c,T", [
    (780, 700, 65, 30),       # smallest count past the stacked layout (Npad = 80); d, n ragged to the tiles
    (1000, 900, 100, 30),     # the rank bound 2r = 100 of the large single-matrix workload
    (1024, 1100, 128, 26),    # largest count of the swapped-operand search
])
def test_two_slab_dense_search_matches_oracle(d, n, c, T):
    """For 64 < c <= 128 the all-column tensor-core search holds the raw
    centroids and their TF32 lo parts in two 128-row A slabs (rows i and
    128 + i) and sums three products per 8 rows.  Labels must equal the
    oracle's and L, S match it element by element; the timing mode proves the
    all-column kernel ran (it needs 16-byte columns, so d is a multiple of 4)."""
    from paper_1904_07497_gb300 import respca
    pr = synth.lowrank_sparse(d, n, 40, 0.1, seed=d + c)
    X64 = pr.X.astype(np.float64)
    p0, _ = oracle.init_labels(X64, c, seed=2)
    ref, _ = oracle.solve(X64, c, tol=0.0, max_iter=T, p0=p0)
    s = respca.Solver(seed=3, timing=True)
    r = s.solve(_dev(pr.X), c, tol=0.0, max_iter=T, p0=torch.from_numpy(p0).cuda())
    torch.cuda.synchronize()
    st = r.stats
    got = (r.p.cpu().numpy(), _host(r.L), _host(r.S))
    s.close()
    assert st["iters"] == T
    assert st["dense_passes"] > 0, "the all-column search did not run"
    np.testing.assert_array_equal(got[0], ref.labels)
    _check_state(got[1], got[2], ref, X64)


# ------------------------------------------------------------------ ramp skip
@pytest.mark.parametrize("kind", ["lowrank", "video"])
def test_ramp_skip_matches_step_by_step(kind):
    """The closed-form ramp (S = 0, no label move) gives the same labels and
    iteration count as running every iteration, and L, S equal to FP32 rounding."""
    from paper_1904_07497_gb300 import respca
    if kind == "lowrank":
        pr = synth.lowrank_sparse(500, 500, 25, 0.05, seed=0)
        c = 25
    else:
        pr = synth.video(n=240, height=48, width=64, n_backgrounds=3, seed=4)
        c = 3
    X64 = pr.X.astype(np.float64)
    p0, _ = oracle.init_labels(X64, c, seed=0)
    outs = []
    for skip in (True, False):
        s = respca.Solver(seed=0, ramp_skip=skip)
        res = s.solve(_dev(pr.X), c, tol=1e-6, max_iter=500, p0=torch.from_numpy(p0).cuda())
        torch.cuda.synchronize()
        outs.append((res.p.cpu().numpy(), _host(res.L), _host(res.S), res.stats))
        s.close()
    (pa, La, Sa, sa), (pb, Lb, Sb, sb) = outs
    assert sa["iters"] == sb["iters"]
    assert sa["lloyd_passes"] < sb["lloyd_passes"]          # the ramp really was skipped
    np.testing.assert_array_equal(pa, pb)
    assert np.linalg.norm(La - Lb) <= 1e-6 * np.linalg.norm(Lb)
    assert np.linalg.norm(Sa - Sb) <= 1e-6 * max(np.linalg.norm(Sb), 1e-3 * np.linalg.norm(X64))


def test_column_norms_match_oracle():
    """Sec. 6 anomaly score ||S_j||_2 of a solve's S, against the oracle's on
    the same FP32 values (ragged d, a column of zeros, strided leading dim)."""
    from paper_1904_07497_gb300 import respca
    g = np.random.default_rng(4)
    d, n = 333, 257
    S32 = (g.standard_normal((d, n)) * (g.random((d, n)) < 0.1)).astype(np.float32)
    S32[:, 9] = 0.0
    big = torch.zeros((n, d + 3), device="cuda")
    big[:, :d].copy_(torch.from_numpy(np.ascontiguousarray(S32.T)))
    S = big[:, :d].T                                        # lds = d + 3
    got = respca.respca_column_norms(S).cpu().numpy().astype(np.float64)
    ref = oracle.column_norms(S32.astype(np.float64))
    np.testing.assert_allclose(got, ref, rtol=2e-6, atol=0)
    assert got[9] == 0.0


# ------------------------------------------------------------------ l2,1 S norm
def _outlier_columns(d, n, r, n_out, seed):
    """Rank-r columns plus n_out whole columns replaced by unrelated values
    (sample-specific corruption, the case the l2,1 norm models)."""
    g = np.random.default_rng(seed)
    L0 = g.standard_normal((d, r)) @ g.standard_normal((r, n)) / np.sqrt(r)
    X = L0.copy()
    out = g.choice(n, n_out, replace=False)
    X[:, out] = 3.0 * g.standard_normal((d, n_out))
    return np.asfortranarray(X.astype(np.float32)), out


@pytest.fixture(scope="module")
def solver_l21():
    from paper_1904_07497_gb300 import respca
    s = respca.Solver(seed=3, s_norm=1)
    yield s
    s.close()


@pytest.mark.parametrize("T", [0, 14, 30])
def test_l21_single_iteration_from_oracle_state(solver_l21, T):
    """One GPU l2,1 iteration from an oracle state equals the oracle's."""
    X32, _ = _outlier_columns(300, 260, 6, 12, seed=2)
    X64 = X32.astype(np.float64)
    c, lam = 6, np.sqrt(300)
    p0, _ = oracle.init_labels(X64, c, seed=0)
    st = oracle.State(np.zeros((300, 260), order="F"), np.zeros((300, 260), order="F"),
                      np.zeros((300, 260), order="F"), p0, 1e-2)
    for _ in range(T):
        st, *_ = oracle.iteration(X64, st, c, lam, snorm=1)
    st = _rounded(st)
    ref, norms, _, _ = oracle.iteration(X64, st, c, lam, snorm=1)
    got = _run(solver_l21, X32, c, 1, None, warm=st)
    np.testing.assert_array_equal(got["p"], ref.labels)
    _check_state(got["L"], got["S"], ref, X64)
    tr_ref = ref.Theta / st.rho
    tr_got = got["Theta"] / st.rho
    assert np.abs(tr_got - tr_ref).max() <= 1e-5 * max(np.abs(X64).max(), 1.0)
    e_ref = max(norms) / np.linalg.norm(X64)
    assert got["stats"]["err"] == pytest.approx(e_ref, rel=1e-4, abs=1e-7)


def test_l21_fixed_iterations_and_convergence():
    """40 l2,1 iterations from the same labels match the oracle; a solve to
    1e-6 converges, with the outlying columns carrying the largest
    ||S_j||_2 (the Sec. 6 score)."""
    from paper_1904_07497_gb300 import respca
    X32, out = _outlier_columns(300, 260, 6, 12, seed=2)
    X64 = X32.astype(np.float64)
    c = 6
    p0, _ = oracle.init_labels(X64, c, seed=0)
    ref, _ = oracle.solve(X64, c, tol=0.0, max_iter=40, p0=p0, snorm=1)
    s = respca.Solver(seed=3, s_norm=1)
    X = _dev(X32)
    r = s.solve(X, c, tol=0.0, max_iter=40, p0=torch.from_numpy(p0).cuda())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(r.p.cpu().numpy(), ref.labels)
    _check_state(_host(r.L), _host(r.S), ref, X64)
    r2 = s.solve(X, c, tol=1e-6, max_iter=500)
    torch.cuda.synchronize()
    assert r2.stats["converged"] == 1 and r2.stats["err"] <= 1e-6
    score = respca.respca_column_norms(r2.S).cpu().numpy()
    top = set(np.argsort(-score)[:len(out)].tolist())
    assert top == set(out.tolist())
    s.close()


def test_device_lloyd_loop_matches_host_loop():
    """The Lloyd passes run as a device loop (CUDA graph, problems of >= 4M
    elements) or, with the library's event timing on, driven by the host; the
    two run the same kernels in the same order, so whole solves agree bit for
    bit, pass counts included."""
    from paper_1904_07497_gb300 import respca
    pr = synth.lowrank_sparse(2048, 2048, 20, 0.1, seed=17)
    X = _dev(pr.X)
    out = []
    for timing in (False, True):
        s = respca.Solver(seed=5, timing=timing)
        r = s.solve(X, 20, tol=1e-6, max_iter=300)
        torch.cuda.synchronize()
        out.append((r.p.cpu().numpy(), _host(r.L), _host(r.S), r.stats))
        s.close()
    (pa, La, Sa, sa), (pb, Lb, Sb, sb) = out
    np.testing.assert_array_equal(pa, pb)
    np.testing.assert_array_equal(La, Lb)
    np.testing.assert_array_equal(Sa, Sb)
    assert sa["iters"] == sb["iters"] and sa["converged"] == 1
    assert sa["lloyd_passes"] == sb["lloyd_passes"] and sa["lloyd_passes"] > sa["iters"]
