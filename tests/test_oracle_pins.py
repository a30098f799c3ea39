"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check here reaches the oracle's result by a route other than the
oracle's own code: a dense linear solve instead of the closed form, literal
matrix definitions instead of the sum-of-squares shortcut, brute force over
all partitions, scalar minimisation, exact probabilities, closed-form special
cases, and identities that follow from the update equations.  A dropped term,
a wrong sign or index, or a transposed operand in the oracle fails one of
them.  Paper: Peng et al., RES-PCA (arXiv 1904.07497).
"""
import itertools
import os

import numpy as np
import pytest

from paper_1904_07497_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_state(d, n, c, seed, rho=0.7):
    g = np.random.default_rng(seed)
    X = np.asfortranarray(g.standard_normal((d, n)))
    S = np.asfortranarray(g.standard_normal((d, n)) * (g.random((d, n)) < 0.2))
    T = np.asfortranarray(np.clip(g.standard_normal((d, n)), -1, 1))
    labels = np.concatenate([np.arange(c), g.integers(0, c, n - c)]).astype(np.int32)
    g.shuffle(labels)
    return X, S, T, labels, rho


# ------------------------------------------------------------------ generator
def test_splitmix64_published_vector(oracle_mod):
    want = [int(x) for x in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if x.strip() and not x.startswith("#")]
    assert oracle_mod.splitmix64_stream(1234567, len(want)) == want


def test_uniform_is_top53_bits(oracle_mod):
    raw = oracle_mod.splitmix64_stream(99, 50)
    u = oracle_mod.uniform_stream(99, 50)
    assert u == [(r >> 11) / 2.0 ** 53 for r in raw]
    assert all(0.0 <= x < 1.0 for x in u)


# ------------------------------------------------------------------ L step
@pytest.mark.parametrize("lam,rho", [(3.0, 0.5), (22.36, 1e-4), (0.1, 40.0)])
def test_l_step_equals_dense_inverse(oracle_mod, lam, rho):
    """Eq. (15): P_i(L) = rho P_i(D) (2 lam M_i + rho I)^-1 by a dense solve,
    against the Sherman-Morrison-Woodbury closed form of Eq. (18)."""
    d, n, c = 7, 23, 4
    X, S, T, labels, _ = _rand_state(d, n, c, 1)
    L, _, cnt = oracle_mod.l_step(X, S, T, rho, lam, labels, c)
    D = X - S + T / rho
    for i in range(c):
        cols = np.where(labels == i)[0]
        ni = len(cols)
        M = np.eye(ni) - np.ones((ni, ni)) / ni
        A = 2 * lam * M + rho * np.eye(ni)
        Pi = np.linalg.solve(A, rho * D[:, cols].T).T   # A symmetric
        # the dense route loses cond(A) = (2 lam + rho) / rho digits
        tol = 1e-14 * np.linalg.cond(A)
        np.testing.assert_allclose(L[:, cols], Pi, rtol=tol, atol=tol * np.abs(Pi).max())
        assert cnt[i] == ni


def test_l_step_first_order_condition(oracle_mod):
    """Eq. (14): 2 lam P_i(L) M_i + rho P_i(L) - rho P_i(D) = 0."""
    d, n, c, lam, rho = 5, 17, 3, 2.5, 0.3
    X, S, T, labels, _ = _rand_state(d, n, c, 2)
    L, _, _ = oracle_mod.l_step(X, S, T, rho, lam, labels, c)
    D = X - S + T / rho
    for i in range(c):
        cols = np.where(labels == i)[0]
        ni = len(cols)
        M = np.eye(ni) - np.ones((ni, ni)) / ni
        R = 2 * lam * L[:, cols] @ M + rho * L[:, cols] - rho * D[:, cols]
        assert np.abs(R).max() < 1e-12


def test_l_step_minimises_subproblem(oracle_mod):
    """Eq. (10): the L step's output has a lower subproblem value than any
    perturbation of it (the subproblem is strictly convex)."""
    d, n, c, lam, rho = 4, 12, 3, 1.7, 0.9
    X, S, T, labels, _ = _rand_state(d, n, c, 3)
    L, _, _ = oracle_mod.l_step(X, S, T, rho, lam, labels, c)
    D = X - S + T / rho

    def f(Lm):
        tr = 0.0
        for i in range(c):
            p = (labels == i).astype(float)
            P = np.diag(p)
            M = np.eye(n) - np.ones((n, n)) / p.sum()
            tr += np.trace(Lm @ P @ M @ P @ Lm.T)
        return lam * tr + rho / 2 * np.sum((X - Lm - S + T / rho) ** 2)

    f0 = f(L)
    g = np.random.default_rng(0)
    for _ in range(20):
        assert f(L + 1e-3 * g.standard_normal(L.shape)) > f0
    # and D itself (lambda-term ignored) is worse unless clusters are exact
    assert f(D) >= f0


def test_l_step_special_cases(oracle_mod):
    d, n, c, rho = 6, 9, 9, 0.4
    X, S, T, _, _ = _rand_state(d, n, 3, 4)
    D = X - S + T / rho
    # every column its own cluster: M_i = 0, so L = D
    L, _, _ = oracle_mod.l_step(X, S, T, rho, 5.0, np.arange(n, dtype=np.int32), n)
    np.testing.assert_allclose(L, D, rtol=1e-13, atol=1e-13)
    # lambda = 0: no variance term, L = D
    lab = np.array([0, 1, 2, 0, 1, 2, 0, 1, 2], dtype=np.int32)
    L, _, _ = oracle_mod.l_step(X, S, T, rho, 0.0, lab, 3)
    np.testing.assert_allclose(L, D, rtol=1e-13, atol=1e-13)
    # one cluster: a D + (1 - a) (row mean) 1^T with a = rho / (2 lam + rho)
    lam = 1.3
    a = rho / (2 * lam + rho)
    L, _, _ = oracle_mod.l_step(X, S, T, rho, lam, np.zeros(n, dtype=np.int32), 1)
    want = a * D + (1 - a) * D.mean(axis=1, keepdims=True)
    np.testing.assert_allclose(L, want, rtol=1e-12, atol=1e-12)


def test_cluster_means_of_l_equal_those_of_d(oracle_mod):
    """M_i 1 = 0 in Eq. (14): the L step keeps each cluster's mean."""
    d, n, c, lam, rho = 8, 30, 4, 10.0, 0.05
    X, S, T, labels, _ = _rand_state(d, n, c, 5)
    L, muD, _ = oracle_mod.l_step(X, S, T, rho, lam, labels, c)
    muL, _ = oracle_mod.cluster_means(L, labels, c)
    np.testing.assert_allclose(muL, muD, rtol=1e-12, atol=1e-12)
    D = X - S + T / rho
    for i in range(c):
        np.testing.assert_allclose(muD[:, i], D[:, labels == i].mean(axis=1), rtol=1e-12)


# ------------------------------------------------------------------ objective
def test_trace_form_equals_within_cluster_ss(oracle_mod):
    """Eq. (8) trace terms, built literally from d(p_i) and I - 11^T/n_i,
    equal the K-means sum of squares of Eq. (20) the oracle evaluates; the
    size in the denominator must be the count n_i (reading of ||p_i||)."""
    d, n, c, lam = 5, 14, 3, 0.8
    g = np.random.default_rng(6)
    L = g.standard_normal((d, n))
    labels = np.array([0, 1, 2] * 4 + [0, 1], dtype=np.int32)
    tr = 0.0
    tr_literal_2norm = 0.0
    for i in range(c):
        p = (labels == i).astype(float)
        P = np.diag(p)
        one = np.ones((n, 1))
        tr += np.trace(L @ P @ (np.eye(n) - one @ one.T / p.sum()) @ P @ L.T)
        tr_literal_2norm += np.trace(L @ P @ (np.eye(n) - one @ one.T / np.linalg.norm(p)) @ P @ L.T)
    got = oracle_mod.objective(L, np.zeros((d, n)), labels, c, lam)
    assert got == pytest.approx(lam * tr, rel=1e-12)
    assert abs(lam * tr_literal_2norm - got) > 1e-3 * abs(got)


def test_variance_model_pairwise_identity(oracle_mod):
    """Sec. 3: sum_i sum_j ||L_i - L_j||^2 = 2 n sum_i ||L_i - mean||^2
    (Eq. (5) rewritten), i.e. the c = 1 case of the model objective."""
    d, n, lam = 4, 11, 1.0
    g = np.random.default_rng(7)
    L = g.standard_normal((d, n))
    pair = sum(np.sum((L[:, i] - L[:, j]) ** 2) for i in range(n) for j in range(n))
    ss = oracle_mod.objective(L, np.zeros((d, n)), np.zeros(n, dtype=np.int32), 1, lam)
    assert pair == pytest.approx(2 * n * ss, rel=1e-12)


def test_objective_l1_term(oracle_mod):
    d, n = 3, 4
    S = np.arange(12, dtype=float).reshape(d, n) - 5.5
    assert oracle_mod.objective(np.zeros((d, n)), S, np.zeros(n, dtype=np.int32), 1, 2.0) == \
        pytest.approx(np.abs(S).sum())


# ------------------------------------------------------------------ K-means
def test_assign_matches_library_argmin(oracle_mod):
    from scipy.spatial.distance import cdist
    g = np.random.default_rng(8)
    Y = g.standard_normal((6, 40))
    mu = g.standard_normal((6, 5))
    p, _ = oracle_mod.assign(Y, mu, np.zeros(40, dtype=np.int32))
    want = np.argmin(cdist(Y.T, mu.T, "sqeuclidean"), axis=1)
    np.testing.assert_array_equal(p, want)
    # inactive clusters never win
    act = np.array([1, 0, 1, 1, 0], dtype=np.uint8)
    p, _ = oracle_mod.assign(Y, mu, np.zeros(40, dtype=np.int32), act)
    dist = cdist(Y.T, mu.T, "sqeuclidean")
    dist[:, act == 0] = np.inf
    np.testing.assert_array_equal(p, np.argmin(dist, axis=1))


def test_assign_ties_go_to_lowest_index(oracle_mod):
    mu = np.array([[1.0, -1.0, 1.0], [0.0, 0.0, 0.0]])
    Y = np.array([[0.0], [0.0]])                   # equidistant from all three
    p, ch = oracle_mod.assign(Y, mu, np.array([2], dtype=np.int32))
    assert p[0] == 0 and ch == 1
    Y2 = np.array([[1.0], [0.0]])                  # tie between clusters 0 and 2
    p, _ = oracle_mod.assign(Y2, mu, np.array([2], dtype=np.int32))
    assert p[0] == 0


def _ss(Y, labels):
    s = 0.0
    for i in np.unique(labels):
        cols = Y[:, labels == i]
        s += np.sum((cols - cols.mean(axis=1, keepdims=True)) ** 2)
    return s


def test_lloyd_monotone_and_fixed_point(oracle_mod):
    g = np.random.default_rng(9)
    Y = np.concatenate([g.standard_normal((4, 30)) + 3 * k for k in range(3)], axis=1)
    Y = Y[:, g.permutation(90)]
    c = 3
    mu0 = Y[:, :c].copy()
    prev = np.inf
    for km in range(1, 12):
        p, _, _, steps, _ = oracle_mod.lloyd(Y, -np.ones(90, dtype=np.int32), mu0, km_max=km)
        cur = _ss(Y, p)
        assert cur <= prev + 1e-9
        prev = cur
    # the converged labels: every column is nearest to its own cluster mean
    p, _, _, steps, _ = oracle_mod.lloyd(Y, -np.ones(90, dtype=np.int32), mu0, km_max=100)
    assert steps < 100
    mu = np.stack([Y[:, p == i].mean(axis=1) for i in range(c)], axis=1)
    dist = ((Y[:, :, None] - mu[:, None, :]) ** 2).sum(axis=0)
    np.testing.assert_array_equal(np.argmin(dist, axis=1), p)


def _partitions(n, c):
    for lab in itertools.product(range(c), repeat=n):
        if len(set(lab)) == c and lab[0] == 0:
            yield np.array(lab, dtype=np.int32)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lloyd_against_brute_force(oracle_mod, seed):
    """n = 7, c = 3: the global optimum over all partitions is a Lloyd fixed
    point, and Lloyd from any start never beats it."""
    g = np.random.default_rng(100 + seed)
    Y = g.standard_normal((2, 7))
    c = 3
    best = min(_partitions(7, c), key=lambda p: _ss(Y, p))
    gmin = _ss(Y, best)
    mu = np.stack([Y[:, best == i].mean(axis=1) for i in range(c)], axis=1)
    p, _, _, steps, ch = oracle_mod.lloyd(Y, best, mu, km_max=100)
    assert ch == 0 and steps == 1
    for start in range(5):
        mu0 = Y[:, g.choice(7, c, replace=False)]
        p, *_ = oracle_mod.lloyd(Y, -np.ones(7, dtype=np.int32), mu0, km_max=100)
        assert _ss(Y, p) >= gmin - 1e-12


def test_kmeanspp_first_centre_and_distinctness(oracle_mod):
    g = np.random.default_rng(10)
    X = g.standard_normal((3, 12))
    for seed in range(10):
        centers = oracle_mod.kmeanspp(X, 12, seed)
        u0 = oracle_mod.uniform_stream(seed, 1)[0]
        assert centers[0] == int(u0 * 12)
        assert sorted(centers.tolist()) == list(range(12))   # c = n: each column once


def test_kmeanspp_d2_sampling_probabilities(oracle_mod):
    """The second centre is column j with probability D(j)^2 / sum D^2: an
    exact distribution, checked by a chi-square test over many seeds."""
    X = np.array([[0.0, 1.0, 3.0, 7.0]])
    counts = np.zeros((4, 4))
    for seed in range(6000):
        c0, c1 = oracle_mod.kmeanspp(X, 2, seed)
        counts[c0, c1] += 1
    from scipy.stats import chisquare
    for f in range(4):
        d2 = (X[0] - X[0, f]) ** 2
        prob = d2 / d2.sum()
        obs = counts[f]
        keep = prob > 0
        assert obs[~keep].sum() == 0
        res = chisquare(obs[keep], prob[keep] * obs.sum())
        assert res.pvalue > 1e-4


def test_init_labels_finds_separated_groups(oracle_mod):
    pr = synth.clustered_columns(20, 60, 4, seed=11)
    p, steps = oracle_mod.init_labels(pr.X, 4, seed=3)
    # co-membership equals the truth
    same_truth = pr.truth_labels[:, None] == pr.truth_labels[None, :]
    same = p[:, None] == p[None, :]
    assert np.array_equal(same, same_truth)


# ------------------------------------------------------------------ S and Theta
def test_soft_threshold_solves_scalar_problem(oracle_mod):
    """Eq. (23)-(24) elementwise: S_ij minimises (1/rho)|s| + 1/2 (B_ij - s)^2."""
    from scipy.optimize import minimize_scalar
    g = np.random.default_rng(12)
    rho = 0.8
    X = g.standard_normal((3, 5)) * 3
    L = g.standard_normal((3, 5))
    T = np.clip(g.standard_normal((3, 5)), -1, 1)
    S = oracle_mod.s_step(X, L, T, rho)
    B = X - L + T / rho
    for b, s in zip(B.ravel(), S.ravel()):
        r = minimize_scalar(lambda v: abs(v) / rho + 0.5 * (b - v) ** 2,
                            bounds=(-20, 20), method="bounded", options={"xatol": 1e-10})
        assert s == pytest.approx(r.x, abs=1e-6)
    # sign(0) = 0 and |B| <= 1/rho gives exactly 0
    Z = oracle_mod.s_step(np.zeros((1, 3)), np.zeros((1, 3)), np.array([[0.0, 0.5, -0.8]]), rho)
    assert np.all(Z == 0.0)


def test_theta_step_identity(oracle_mod):
    """After the S step, Eq. (25) gives Theta + rho (X - L - S) = rho (B - S)
    = clip(rho B, -1, 1): the multiplier lies in the subdifferential of the
    l1 norm at S."""
    g = np.random.default_rng(13)
    rho = 2.3
    X = g.standard_normal((4, 6)) * 2
    L = g.standard_normal((4, 6))
    T = np.clip(g.standard_normal((4, 6)), -1, 1)
    S = oracle_mod.s_step(X, L, T, rho)
    Tn = oracle_mod.theta_step(X, L, S, T, rho)
    B = X - L + T / rho
    np.testing.assert_allclose(Tn, np.clip(rho * B, -1, 1), rtol=1e-12, atol=1e-12)
    assert np.all(np.abs(Tn) <= 1 + 1e-15)
    nz = S != 0
    np.testing.assert_allclose(Tn[nz], np.sign(S[nz]), atol=1e-12)


# ------------------------------------------------------------------ iteration
def test_block_descent_of_the_lagrangian(oracle_mod):
    """Eq. (9) at fixed (Theta, rho): the L, p and S updates each minimise
    over their block, so the augmented Lagrangian never increases."""
    d, n, c, lam, rho = 6, 40, 4, 2.0, 0.6
    X, S, T, labels, _ = _rand_state(d, n, c, 14, rho)
    L0 = np.zeros((d, n))
    f0 = oracle_mod.lagrangian(X, L0, S, T, labels, c, lam, rho)
    L, mu, cnt = oracle_mod.l_step(X, S, T, rho, lam, labels, c)
    f1 = oracle_mod.lagrangian(X, L, S, T, labels, c, lam, rho)
    p, *_ = oracle_mod.lloyd(L, labels, mu, (cnt > 0).astype(np.uint8), km_max=100)
    f2 = oracle_mod.lagrangian(X, L, S, T, p, c, lam, rho)
    Sn = oracle_mod.s_step(X, L, T, rho)
    f3 = oracle_mod.lagrangian(X, L, Sn, T, p, c, lam, rho)
    assert f1 <= f0 + 1e-12 and f2 <= f1 + 1e-12 and f3 <= f2 + 1e-12


def test_iteration_cluster_sum_identity(oracle_mod):
    """From Eq. (14) (M_i 1 = 0) and Eq. (25): for each cluster i of the
    labels used by the L step, sum_j Theta_{t+1} = rho_t sum_j (S_t - S_{t+1})."""
    pr = synth.lowrank_sparse(30, 50, 3, 0.1, seed=15)
    X = pr.X.astype(np.float64)
    c, lam = 3, np.sqrt(50)
    p0, _ = oracle_mod.init_labels(X, c, seed=1)
    st = oracle_mod.State(np.zeros((30, 50), order="F"), np.zeros((30, 50), order="F"),
                          np.zeros((30, 50), order="F"), p0, 1e-4)
    checked = 0
    for t in range(45):
        nxt, norms, ch, _ = oracle_mod.iteration(X, st, c, lam)
        for i in range(c):
            cols = st.labels == i
            lhs = nxt.Theta[:, cols].sum(axis=1)
            rhs = st.rho * (st.S[:, cols] - nxt.S[:, cols]).sum(axis=1)
            np.testing.assert_allclose(lhs, rhs, atol=1e-9 * max(1.0, np.abs(rhs).max()))
        assert np.all(np.abs(nxt.Theta) <= 1 + 1e-12)
        checked += 1
        st = nxt
    assert checked == 45


def test_first_iteration_closed_form(oracle_mod):
    """From the zero state, iteration 1 gives L = a X + (1-a) mu(X) with
    a = rho0/(2 lam + rho0), then S = soft(X - L, 1/rho0)."""
    pr = synth.lowrank_sparse(12, 20, 2, 0.1, seed=16)
    X = pr.X.astype(np.float64)
    c, lam, rho0 = 2, 4.0, 1e-4
    p0 = np.array([0, 1] * 10, dtype=np.int32)
    st, _ = oracle_mod.solve(X, c, lam=lam, rho0=rho0, tol=0.0, max_iter=1, p0=p0, km_max=1)
    a = rho0 / (2 * lam + rho0)
    mu = np.stack([X[:, p0 == i].mean(axis=1) for i in range(c)], axis=1)
    Lw = a * X + (1 - a) * mu[:, p0]
    np.testing.assert_allclose(st.L, Lw, rtol=1e-12, atol=1e-12)
    B = X - Lw
    Sw = np.sign(B) * np.maximum(np.abs(B) - 1 / rho0, 0)
    np.testing.assert_allclose(st.S, Sw, atol=1e-12)
    assert st.rho == pytest.approx(1.5e-4)


# ------------------------------------------------------------------ whole solve
def test_exact_recovery_on_repeated_columns(oracle_mod):
    """No corruption and columns that repeat c base columns: with the true
    labels every column equals its cluster mean, so L = X, S = 0 and the
    criterion is met at the second iteration (the first moves L off 0)."""
    pr = synth.clustered_columns(15, 40, 4, seed=17)
    X = pr.X.astype(np.float64)
    st, stats = oracle_mod.solve(X, 4, tol=1e-12, max_iter=10, p0=pr.truth_labels)
    assert stats["iters"] == 2 and stats["converged"] == 1
    np.testing.assert_allclose(st.L, X, rtol=1e-14, atol=1e-14)
    assert np.all(st.S == 0)


@pytest.mark.parametrize("mode", ["c_eq_n", "lambda0"])
def test_degenerate_models_return_x(oracle_mod, mode):
    g = np.random.default_rng(18)
    X = g.standard_normal((5, 8))
    if mode == "c_eq_n":
        st, stats = oracle_mod.solve(X, 8, tol=1e-12, max_iter=10, p0=np.arange(8, dtype=np.int32))
    else:
        st, stats = oracle_mod.solve(X, 2, lam=1e-300, tol=1e-12, max_iter=10,
                                     p0=np.array([0, 1] * 4, dtype=np.int32))
    np.testing.assert_allclose(st.L, X, rtol=1e-12, atol=1e-12)
    assert np.abs(st.S).max() < 1e-12 and stats["converged"] == 1


def test_converges_on_lowrank_sparse(oracle_mod):
    """Stopping rule of Sec. 5 met at exit; the KKT conditions of Eq. (8)
    hold approximately: |Theta| <= 1, Theta = sign(S) on the support."""
    pr = synth.lowrank_sparse(80, 60, 4, 0.05, seed=19)
    X = pr.X.astype(np.float64)
    st, stats = oracle_mod.solve(X, 4, tol=1e-6, max_iter=500, seed=2)
    assert stats["converged"] == 1
    assert stats["err"] <= 1e-6
    assert np.linalg.norm(X - st.L - st.S) / np.linalg.norm(X) <= 1e-6
    assert stats["iters"] < 120
    assert np.all(np.abs(st.Theta) <= 1 + 1e-12)
    nz = st.S != 0
    np.testing.assert_allclose(st.Theta[nz], np.sign(st.S[nz]), atol=1e-9)


def test_warm_start_continues_the_same_path(oracle_mod):
    pr = synth.lowrank_sparse(40, 30, 3, 0.1, seed=20)
    X = pr.X.astype(np.float64)
    full, s_full = oracle_mod.solve(X, 3, tol=0.0, max_iter=30, seed=5)
    half, _ = oracle_mod.solve(X, 3, tol=0.0, max_iter=18, seed=5)
    rest, _ = oracle_mod.solve(X, 3, tol=0.0, max_iter=12, warm=half)
    np.testing.assert_array_equal(rest.L, full.L)
    np.testing.assert_array_equal(rest.S, full.S)
    np.testing.assert_array_equal(rest.labels, full.labels)
    assert rest.rho == full.rho


def test_zero_input_and_invalid_args(oracle_mod):
    st, stats = oracle_mod.solve(np.zeros((4, 5)), 2)
    assert stats["iters"] == 0 and np.all(st.L == 0) and np.all(st.S == 0)
    with pytest.raises(ValueError):
        oracle_mod.solve(np.ones((4, 5)), 6)        # c > n
    with pytest.raises(ValueError):
        oracle_mod.solve(np.ones((4, 5)), 0)
    with pytest.raises(ValueError):
        oracle_mod.solve(np.ones((4, 5)), 2, p0=np.array([0, 1, 2, 0, 1], dtype=np.int32))


def test_fro_matches_library_norm(oracle_mod):
    g = np.random.default_rng(21)
    A = g.standard_normal((13, 7)) * 3.0
    assert oracle_mod.fro(A) == pytest.approx(np.linalg.norm(A), rel=1e-14)
    assert oracle_mod.fro(np.zeros((3, 2))) == 0.0


# ------------------------------------------------------------------ Sec. 6 anomaly score
def test_column_norms_match_library_and_special_cases(oracle_mod):
    """||S_j||_2 per column: against numpy's norm, a one-hot column gives |v|,
    a zero column 0, and scaling S scales every score."""
    g = np.random.default_rng(21)
    S = np.asfortranarray(g.standard_normal((53, 17)))
    S[:, 3] = 0.0
    S[:, 5] = 0.0
    S[7, 5] = -2.5
    got = oracle_mod.column_norms(S)
    np.testing.assert_allclose(got, np.linalg.norm(S, axis=0), rtol=1e-14, atol=0)
    assert got[3] == 0.0 and got[5] == 2.5
    np.testing.assert_allclose(oracle_mod.column_norms(3.0 * S), 3.0 * got, rtol=1e-14)


# ------------------------------------------------------------------ l2,1 S norm (Sec. 3 alternative)
def test_l21_s_step_is_the_prox(oracle_mod):
    """Block soft-thresholding minimises (1/rho)||S||_{2,1} + 1/2||S - B||^2
    column by column: no random perturbation lowers the objective, a column
    with rho ||B_j|| <= 1 is zeroed, and with d = 1 it reduces to the l1 step."""
    g = np.random.default_rng(5)
    d, n, rho = 6, 9, 1.7
    X = np.asfortranarray(g.standard_normal((d, n)))
    L = np.asfortranarray(g.standard_normal((d, n)) * 0.3)
    T = np.asfortranarray(np.clip(g.standard_normal((d, n)), -1, 1))
    B = X - L + T / rho
    B[:, 2] *= 0.2 / (rho * np.linalg.norm(B[:, 2]))   # a column below the threshold
    X2 = np.asfortranarray(B + L - T / rho)
    S = oracle_mod.s_step_l21(X2, L, T, rho)
    obj = lambda s, b: np.linalg.norm(s) / rho + 0.5 * np.sum((s - b) ** 2)
    for j in range(n):
        b = X2[:, j] - L[:, j] + T[:, j] / rho
        f0 = obj(S[:, j], b)
        for _ in range(200):
            pert = S[:, j] + g.standard_normal(d) * 10.0 ** g.uniform(-6, -1)
            assert obj(pert, b) >= f0 - 1e-12
    assert np.all(S[:, 2] == 0.0)
    X1 = np.asfortranarray(g.standard_normal((1, 40)))
    L1 = np.asfortranarray(g.standard_normal((1, 40)) * 0.1)
    T1 = np.asfortranarray(np.zeros((1, 40)))
    np.testing.assert_allclose(oracle_mod.s_step_l21(X1, L1, T1, 2.0), oracle_mod.s_step(X1, L1, T1, 2.0),
                               rtol=1e-14, atol=1e-15)


def test_l21_theta_is_a_subgradient(oracle_mod):
    """After an l2,1 iteration, every column of Theta lies in the subdifferential
    of ||.||_2 at S_j: S_j / ||S_j|| where S_j != 0, otherwise inside the unit ball."""
    g = np.random.default_rng(8)
    d, n, c = 12, 30, 3
    X = np.asfortranarray(g.standard_normal((d, n)))
    X[:, 5] += 6.0   # a strongly outlying column
    st = oracle_mod.State(np.zeros((d, n), order="F"), np.zeros((d, n), order="F"),
                          np.zeros((d, n), order="F"), (np.arange(n) % c).astype(np.int32), 0.8)
    for _ in range(4):
        st, _, _, _ = oracle_mod.iteration(X, st, c, 2.0, snorm=1)
    nz = 0
    for j in range(n):
        s = st.S[:, j]
        t = st.Theta[:, j]
        ns = np.linalg.norm(s)
        if ns > 0:
            nz += 1
            np.testing.assert_allclose(t, s / ns, rtol=1e-10, atol=1e-12)
        else:
            assert np.linalg.norm(t) <= 1.0 + 1e-12
    assert nz >= 1


# ------------------------------------------------------------------ warm-start network (oracle)
def test_warmnet_plain_schedule_equals_oracle_iterations(oracle_mod):
    """With zero log multipliers the network's layers are the plain iterations
    with the labels fixed: on well-separated groups (where the p step keeps
    every label) K layers equal K oracle iterations."""
    from oracle import warmnet
    pr = synth.clustered_columns(40, 36, 3, seed=4, sparsity=0.1)
    X = pr.X.astype(np.float64)
    c, lam, kappa = 3, 3.0, 1.5
    st = oracle_mod.State(np.zeros(X.shape, order="F"), np.zeros(X.shape, order="F"),
                          np.zeros(X.shape, order="F"), pr.truth_labels.astype(np.int32), 0.9)
    for _ in range(3):
        st, *_ = oracle_mod.iteration(X, st, c, lam)
    assert np.array_equal(st.labels, pr.truth_labels)
    K = 4
    rho_k, tau_k = warmnet.schedule(st.rho, kappa, np.zeros(K), np.zeros(K))
    L, S, T = warmnet.forward(X, st.labels, c, lam, st.S, st.Theta, rho_k, tau_k)
    ref = st
    for _ in range(K):
        ref, *_ = oracle_mod.iteration(X, ref, c, lam)
    assert np.array_equal(ref.labels, pr.truth_labels)
    np.testing.assert_allclose(L, ref.L, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(S, ref.S, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(T, ref.Theta, rtol=1e-10, atol=1e-12)


def test_warmnet_schedule_multipliers():
    from oracle import warmnet
    r, t = warmnet.schedule(2.0, 1.5, [0.0, np.log(3.0)], [0.0, np.log(0.5)])
    np.testing.assert_allclose(r, [2.0, 2.0 * 1.5 * 3.0])
    np.testing.assert_allclose(t, [0.5, 0.5 / (2.0 * 1.5 * 3.0)])


def test_warmnet_mlp_grad_matches_finite_differences():
    """The MLP's analytic gradient against central differences of its forward."""
    from oracle import warmnet
    nz, H, nout = 3, 5, 4
    g = np.random.default_rng(7)
    P = g.standard_normal(H * nz + H + nout * H + nout)
    z = g.standard_normal(nz)
    gout = g.standard_normal(nout)
    G = warmnet.mlp_grad(P, z, gout, nz, H, nout)
    h = 1e-6
    fd = np.empty_like(P)
    for i in range(P.size):
        e = np.zeros_like(P)
        e[i] = h
        fp = gout @ warmnet.mlp_forward(P + e, z, nz, H, nout)[0]
        fm = gout @ warmnet.mlp_forward(P - e, z, nz, H, nout)[0]
        fd[i] = (fp - fm) / (2 * h)
    np.testing.assert_allclose(G, fd, rtol=1e-7, atol=1e-8)


def test_warmnet_adam_first_step_is_signed_lr():
    """With bias correction, Adam's first step moves every parameter by
    lr * g / (|g| + eps): lr times the sign of its gradient."""
    from oracle import warmnet
    g = np.array([3.0, -0.5, 1e-3, -20.0])
    P, _, _ = warmnet.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01, eps=1e-12)
    np.testing.assert_allclose(P, -0.01 * np.sign(g), rtol=1e-8)


def _same_partition(a, b):
    m = {}
    for x, y in zip(np.asarray(a).tolist(), np.asarray(b).tolist()):
        if m.setdefault(x, y) != y:
            return False
    return len(set(m.values())) == len(m)


def test_spectral_mean_sq_distance_closed_form():
    """Mean squared distance over pairs i != j equals
    2n/(n-1) (mean ||y||^2 - ||mean y||^2)."""
    from oracle import spectral
    Y = np.random.default_rng(3).standard_normal((4, 37)) + 2.0
    n = Y.shape[1]
    closed = 2 * n / (n - 1) * (np.mean(np.sum(Y * Y, axis=0)) - np.sum(Y.mean(axis=1) ** 2))
    assert spectral.mean_sq_distance(Y) == pytest.approx(closed, rel=1e-12)


def test_spectral_block_diagonal_affinity_gives_indicator_subspace():
    """Groups so far apart that every cross affinity underflows to 0: M is
    block diagonal, its top c eigenvalues are exactly 1, and their
    eigenspace is spanned by D^{1/2} 1_g of each group g (M D^{1/2} 1_g =
    D^{-1/2} A 1_g = D^{1/2} 1_g)."""
    from oracle import spectral
    g = np.random.default_rng(8)
    c, per, d = 3, 15, 5
    Y = np.concatenate([100.0 * k + 0.1 * g.standard_normal((d, per)) for k in range(c)], axis=1)
    truth = np.repeat(np.arange(c), per)
    scale = 0.05 / spectral.mean_sq_distance(Y)
    A, deg, _ = spectral.affinity(Y, scale)
    assert np.all(A[truth[:, None] != truth[None, :]] == 0.0)
    U, w, E = spectral.embedding(Y, c, scale)
    np.testing.assert_allclose(w, 1.0, atol=1e-12)
    P = np.zeros((c * per, c * per))
    for k in range(c):
        v = np.where(truth == k, np.sqrt(deg), 0.0)
        v /= np.linalg.norm(v)
        P += np.outer(v, v)
    np.testing.assert_allclose(U @ U.T, P, atol=1e-10)
    # the row-normalised embedding collapses every group to one point
    for k in range(c):
        Ek = E[:, truth == k]
        assert np.abs(Ek - Ek[:, :1]).max() < 1e-10
    assert _same_partition(spectral.labels(Y, c, scale, seed=0), truth)


def test_spectral_labels_recover_rings_where_kmeans_fails(oracle_mod):
    """Concentric circles: the spectral p step finds the circles, K-means on
    the columns does not (Sec. 4.2's reason for a nonlinear p step)."""
    from oracle import spectral
    pr = synth.rings(10, 600, 3, seed=3, noise=0.05)
    X = pr.X.astype(np.float64)
    assert _same_partition(spectral.labels(X, 3, 0.004, seed=0), pr.truth_labels)
    pk, _ = oracle_mod.init_labels(X, 3, 0)
    assert not _same_partition(pk, pr.truth_labels)
