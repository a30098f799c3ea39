"""GPU parity of the learned warm start (an addition to the paper's method):
the unrolled layers, their reverse pass, the MLP and the Adam step, each
through the C ABI, against the FP64 oracle in oracle/warmnet.py; then the
gain of a trained network on held-out problems of the d = n = 2000 family.

Tolerances: forward values within 2e-5 of the FP64 oracle relative to the
largest entry of X (L, S) or of Theta; gradients within 1e-3 of the largest
component of the finite-difference gradient of the oracle's FP64 loss.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import warmnet as onet
from paper_1904_07497_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K = 8


def _dev(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float32).T)).cuda().T


def _host(t):
    return t.T.contiguous().cpu().numpy().T.astype(np.float64)


@pytest.fixture(scope="module")
def lib():
    from paper_1904_07497_gb300 import respca
    respca.load()
    return respca


@pytest.fixture(scope="module")
def case():
    """700 x 300 (two row chunks, ragged tail; ten tiles), four groups with
    10% sparse +-1 outliers; the state after three oracle iterations."""
    pr = synth.clustered_columns(700, 300, 4, seed=11, sparsity=0.1)
    X = pr.X.astype(np.float32).astype(np.float64)
    c, lam = 4, 3.0
    st = oracle.State(np.zeros(X.shape, order="F"), np.zeros(X.shape, order="F"),
                      np.zeros(X.shape, order="F"), pr.truth_labels.astype(np.int32), 0.9)
    for _ in range(3):
        st, *_ = oracle.iteration(X, st, c, lam)
    # the GPU sees the state rounded to FP32; the oracle starts from the same values
    S0 = st.S.astype(np.float32).astype(np.float64)
    T0 = st.Theta.astype(np.float32).astype(np.float64)
    g = np.random.default_rng(5)
    m = g.uniform(-0.5, 0.5, 2 * K)
    mt = g.uniform(-0.5, 0.5, 2 * K)
    rho_t, tau_t = onet.schedule(st.rho, 1.5, mt[:K], mt[K:])
    Lt, St, _ = onet.forward(X, st.labels, c, lam, S0, T0, rho_t, tau_t)
    Lt = Lt.astype(np.float32).astype(np.float64)
    St = St.astype(np.float32).astype(np.float64)
    return dict(X=X, p=st.labels, c=c, lam=lam, S0=S0, T0=T0, rho=st.rho, m=m, Lt=Lt, St=St,
                scale=1.0 / np.sum(X * X))


def _gpu_forward(lib, net, cs, rho_k, tau_k):
    d, n = cs["X"].shape
    X = _dev(cs["X"])
    p = torch.from_numpy(cs["p"].astype(np.int32)).cuda()
    L, S, T = (torch.empty((n, d), device="cuda").T for _ in range(3))
    lib.respca_net_forward(net, X, p, cs["c"], cs["lam"], _dev(cs["S0"]), _dev(cs["T0"]), rho_k, tau_k,
                           L, S, T)
    torch.cuda.synchronize()
    return X, p, L, S, T


def test_net_forward_matches_oracle(lib, case):
    rho_k, tau_k = lib.respca_net_schedule(case["rho"], 1.5, case["m"])
    r_ref, t_ref = onet.schedule(case["rho"], 1.5, case["m"][:K], case["m"][K:])
    np.testing.assert_allclose(rho_k, r_ref, rtol=1e-6)
    np.testing.assert_allclose(tau_k, t_ref, rtol=1e-6)
    net = lib.respca_net_create()
    try:
        _, _, L, S, T = _gpu_forward(lib, net, case, rho_k, tau_k)
        Lr, Sr, Tr = onet.forward(case["X"], case["p"], case["c"], case["lam"], case["S0"], case["T0"],
                                  r_ref, t_ref)
        xs = np.abs(case["X"]).max()
        eL = np.abs(_host(L) - Lr).max() / xs
        eS = np.abs(_host(S) - Sr).max() / xs
        eT = np.abs(_host(T) - Tr).max() / max(np.abs(Tr).max(), 1e-30)
        print(f"forward max err: L {eL:.2e} S {eS:.2e} Theta {eT:.2e}; active S {np.mean(Sr != 0):.3f}")
        assert np.mean(Sr != 0) > 0.01          # the thresholds matter in this case
        assert eL <= 2e-5 and eS <= 2e-5 and eT <= 2e-5
    finally:
        lib.respca_net_destroy(net)


def test_net_forward_scalar_rows_match_oracle(lib):
    """d = 514 (not a multiple of 4): the kernels take one row per slot
    instead of 16-byte accesses; same check as above on two row chunks."""
    pr = synth.clustered_columns(514, 90, 3, seed=2, sparsity=0.1)
    X = pr.X.astype(np.float32).astype(np.float64)
    st = oracle.State(np.zeros(X.shape, order="F"), np.zeros(X.shape, order="F"),
                      np.zeros(X.shape, order="F"), pr.truth_labels.astype(np.int32), 0.9)
    for _ in range(3):
        st, *_ = oracle.iteration(X, st, 3, 3.0)
    cs = dict(X=X, p=st.labels, c=3, lam=3.0, S0=st.S.astype(np.float32).astype(np.float64),
              T0=st.Theta.astype(np.float32).astype(np.float64))
    m = np.random.default_rng(6).uniform(-0.5, 0.5, 2 * K)
    rho_k, tau_k = lib.respca_net_schedule(st.rho, 1.5, m)
    net = lib.respca_net_create()
    try:
        _, _, L, S, T = _gpu_forward(lib, net, cs, rho_k, tau_k)
    finally:
        lib.respca_net_destroy(net)
    Lr, Sr, Tr = onet.forward(X, st.labels, 3, 3.0, cs["S0"], cs["T0"], rho_k, tau_k)
    xs = np.abs(X).max()
    assert np.abs(_host(L) - Lr).max() <= 2e-5 * xs
    assert np.abs(_host(S) - Sr).max() <= 2e-5 * xs
    assert np.abs(_host(T) - Tr).max() <= 2e-5 * max(np.abs(Tr).max(), 1e-30)


def _oracle_loss(cs, rho_k, tau_k):
    L, S, _ = onet.forward(cs["X"], cs["p"], cs["c"], cs["lam"], cs["S0"], cs["T0"], rho_k, tau_k)
    return onet.loss(L, S, cs["Lt"], cs["St"], cs["scale"])


def test_net_gradients_match_oracle_finite_differences(lib, case):
    rho_k, tau_k = lib.respca_net_schedule(case["rho"], 1.5, case["m"])
    net = lib.respca_net_create()
    try:
        keep = _gpu_forward(lib, net, case, rho_k, tau_k)   # X must outlive the backward pass
        loss, g_rho, g_tau, g_m = lib.respca_net_backward(net, _dev(case["Lt"]), _dev(case["St"]),
                                                          case["scale"], K)
        del keep
    finally:
        lib.respca_net_destroy(net)
    r0, t0 = onet.schedule(case["rho"], 1.5, case["m"][:K], case["m"][K:])
    ref_loss = _oracle_loss(case, r0, t0)
    assert abs(loss - ref_loss) <= 1e-4 * ref_loss
    fd_rho, fd_tau, fd_m = np.zeros(K), np.zeros(K), np.zeros(2 * K)
    for k in range(K):
        for vec, out in ((r0, fd_rho), (t0, fd_tau)):
            h = 1e-6 * vec[k]
            up, dn = vec.copy(), vec.copy()
            up[k] += h
            dn[k] -= h
            args_up = (up, t0) if vec is r0 else (r0, up)
            args_dn = (dn, t0) if vec is r0 else (r0, dn)
            out[k] = (_oracle_loss(case, *args_up) - _oracle_loss(case, *args_dn)) / (2 * h)
    for i in range(2 * K):
        h = 1e-6
        up, dn = case["m"].copy(), case["m"].copy()
        up[i] += h
        dn[i] -= h
        fu = _oracle_loss(case, *onet.schedule(case["rho"], 1.5, up[:K], up[K:]))
        fdn = _oracle_loss(case, *onet.schedule(case["rho"], 1.5, dn[:K], dn[K:]))
        fd_m[i] = (fu - fdn) / (2 * h)
    for name, g, fd in (("rho", g_rho, fd_rho), ("tau", g_tau, fd_tau), ("m", g_m, fd_m)):
        err = np.abs(np.asarray(g) - fd).max() / np.abs(fd).max()
        print(f"grad {name}: max rel err {err:.2e}  |fd|max {np.abs(fd).max():.3e}")
        assert err <= 1e-3, (name, g, fd)


def test_mlp_and_adam_match_oracle(lib):
    nz, H, nout = 6, 64, 16
    g = np.random.default_rng(9)
    P = g.standard_normal(H * nz + H + nout * H + nout) * 0.3
    z = g.standard_normal(nz)
    gout = g.standard_normal(nout)
    Pd = torch.tensor(P, dtype=torch.float32, device="cuda")
    zd = torch.tensor(z, dtype=torch.float32, device="cuda")
    gd = torch.tensor(gout, dtype=torch.float32, device="cuda")
    out = torch.empty(nout, device="cuda")
    hid = torch.empty(H, device="cuda")
    lib.respca_mlp_forward(Pd, nz, H, nout, zd, out, hid)
    o_ref, h_ref = onet.mlp_forward(P.astype(np.float32), z.astype(np.float32), nz, H, nout)
    np.testing.assert_allclose(out.cpu().numpy(), o_ref, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(hid.cpu().numpy(), h_ref, rtol=1e-5, atol=1e-6)
    G = torch.empty_like(Pd)
    lib.respca_mlp_backward(Pd, nz, H, nout, zd, hid, gd, G)
    G_ref = onet.mlp_grad(P.astype(np.float32), z.astype(np.float32), gout.astype(np.float32), nz, H, nout)
    np.testing.assert_allclose(G.cpu().numpy(), G_ref, rtol=1e-4, atol=1e-5)
    lib.respca_mlp_backward(Pd, nz, H, nout, zd, hid, gd, G, accumulate=True)
    np.testing.assert_allclose(G.cpu().numpy(), 2 * G_ref, rtol=1e-4, atol=2e-5)
    M = torch.zeros_like(Pd)
    V = torch.zeros_like(Pd)
    Gh = G.cpu().numpy().astype(np.float64)
    P1, M1, V1 = onet.adam_step(P.astype(np.float32).astype(np.float64), Gh, 0 * Gh, 0 * Gh, 1, 1e-2)
    P2, _, _ = onet.adam_step(P1, Gh, M1, V1, 2, 1e-2)
    lib.respca_adam_step(Pd, G, M, V, lr=1e-2, t=1)
    lib.respca_adam_step(Pd, G, M, V, lr=1e-2, t=2)
    np.testing.assert_allclose(Pd.cpu().numpy(), P2, rtol=1e-5, atol=1e-6)


def test_stop_after_ramp_is_the_closed_form_prefix(lib):
    """stop_after_ramp returns the state after the closed-form leading
    iterations: S = 0, and the same L as a full solve capped at that count."""
    pr = synth.lowrank_sparse(600, 500, 10, 0.1, seed=21, keep_parts=False)
    X = _dev(pr.X)
    d, n = pr.X.shape
    ramp = lib.Solver(stop_after_ramp=True)
    full = lib.Solver()
    try:
        L1, S1, T1 = (torch.empty((n, d), device="cuda").T for _ in range(3))
        p1 = torch.empty(n, device="cuda", dtype=torch.int32)
        w = lib.respca_warm()
        w.Theta = T1.data_ptr()
        st = lib.respca_solve(ramp.h, X, 10, L1, S1, p1, warm=w)
        T = st["iters"]
        assert T > 0 and st["fused_launches"] == 0
        assert float(S1.abs().max()) == 0.0
        ref = full.solve(X, 10, max_iter=T)
        assert ref.stats["fused_launches"] == 0
        assert torch.equal(L1, ref.L) and torch.equal(p1, ref.p)
        assert w.rho == pytest.approx(1e-4 * 1.5 ** T, rel=1e-12)
    finally:
        ramp.close()
        full.close()


def test_warm_start_gain_on_held_out_problems(lib):
    """Train on 8 problems of the d = n = 2000 family (rank 10..50, sparsity
    0.05..0.2, c = rank) and evaluate on 3 held-out seeds.  Every run reaches
    1e-6; the learned network needs fewer iterations in total (closed-form
    ramp + layers + plain continuation) and less wall time than the plain
    solver; its answer is another stationary point of Eq. (8) whose objective
    stays within 1e-3 of the plain answer's (the labels may differ: the
    p step's local optimum depends on the path)."""
    from paper_1904_07497_gb300.warmnet import WarmStart
    ws = WarmStart(layers=K, seed=0)
    try:
        def prob(seed):
            pr = synth.warmstart_problem(seed)
            return _dev(pr.X), pr.rank
        train = [ws.sample(*prob(s)) for s in range(8)]
        hist = ws.fit(train, steps=600, lr=3e-2)
        print(f"loss {hist[0]:.3e} -> {hist[-1]:.3e}")
        assert hist[-1] < 0.2 * hist[0]
        rows = []
        for s in range(10**6, 10**6 + 3):
            X, c = prob(s)
            ws.plain.solve(X, c)                      # warm-up of both paths before timing
            ws.solve(X, c)
            ref = ws.plain.solve(X, c)
            L, S, p, info = ws.solve(X, c)
            lam = ref.stats["lambda"]
            o_ref = oracle.objective(_host(ref.L), _host(ref.S), ref.p.cpu().numpy(), c, lam)
            o_net = oracle.objective(_host(L), _host(S), p.cpu().numpy(), c, lam)
            print(f"seed {s}: plain {ref.stats['iters']} it {ref.stats['ms_total']:.2f} ms | net {info}"
                  f" objective rel {o_net / o_ref - 1:.2e}")
            assert ref.stats["converged"] and info["converged"]
            assert abs(o_net / o_ref - 1) <= 1e-3
            rows.append((ref.stats["iters"], info["total_iters"], ref.stats["ms_total"], info["ms"]))
        r = np.array(rows, dtype=np.float64).mean(axis=0)
        print(f"mean: plain {r[0]:.2f} it {r[2]:.2f} ms | learned {r[1]:.2f} it {r[3]:.2f} ms")
        assert r[1] < r[0] and r[3] < r[2]
    finally:
        ws.close()


# ------------------------------------------------------------------ inference forward
def _bf16(A):
    """FP64 values rounded to BF16 (torch's round-to-nearest-even) and back."""
    t = torch.from_numpy(np.ascontiguousarray(A)).to(torch.bfloat16).to(torch.float64)
    return t.numpy()


def _infer(lib, cs, X, rho_k, tau_k, storage):
    d, n = cs["X"].shape
    p = torch.from_numpy(cs["p"].astype(np.int32)).cuda()
    L, S, T = (torch.empty((n, d), device="cuda").T for _ in range(3))
    net = lib.respca_net_create()
    try:
        lib.respca_net_infer(net, X, p, cs["c"], cs["lam"], _dev(cs["S0"]), _dev(cs["T0"]), rho_k, tau_k,
                             L, S, T, storage=storage)
        torch.cuda.synchronize()
    finally:
        lib.respca_net_destroy(net)
    return _host(L), _host(S), _host(T)


def test_net_infer_fp32_matches_oracle_and_forward(lib, case):
    """Inference with FP32 intermediate states: the same layers as the
    training forward pass (same per-element arithmetic), so it matches the
    FP64 oracle within the forward tolerance and the training forward to
    FP32 rounding of the D sums."""
    rho_k, tau_k = lib.respca_net_schedule(case["rho"], 1.5, case["m"])
    L, S, T = _infer(lib, case, _dev(case["X"]), rho_k, tau_k, 0)
    Lr, Sr, Tr = onet.forward(case["X"], case["p"], case["c"], case["lam"], case["S0"], case["T0"],
                              rho_k, tau_k)
    xs = np.abs(case["X"]).max()
    assert np.abs(L - Lr).max() <= 2e-5 * xs
    assert np.abs(S - Sr).max() <= 2e-5 * xs
    assert np.abs(T - Tr).max() <= 2e-5 * max(np.abs(Tr).max(), 1e-30)
    net = lib.respca_net_create()
    try:
        _, _, Lf, Sf, Tf = _gpu_forward(lib, net, case, rho_k, tau_k)
    finally:
        lib.respca_net_destroy(net)
    assert np.abs(L - _host(Lf)).max() <= 1e-6 * xs
    assert np.abs(S - _host(Sf)).max() <= 1e-6 * xs


def test_net_infer_bf16_storage_matches_rounded_oracle(lib, case):
    """X in BF16 and the intermediate layers' S, Theta stored in BF16: the
    oracle runs the same layers in FP64 on the same BF16 X and rounds S and
    Theta to BF16 where the GPU stores them.  An FP32 and an FP64 result may
    round to neighbouring BF16 values, so stored values differ by at most one
    BF16 ulp (2^-8 relative) in a few elements; the last layer's FP32 outputs
    must then lie within 2^-9 relative Frobenius error (the per-store rounding
    bound) and 4 BF16 ulps of the largest entry element-wise."""
    rho_k, tau_k = lib.respca_net_schedule(case["rho"], 1.5, case["m"])
    Xb64 = _bf16(case["X"])
    Xb = torch.from_numpy(np.ascontiguousarray(case["X"].T)).to(torch.bfloat16).cuda().T
    L, S, T = _infer(lib, case, Xb, rho_k, tau_k, 1)
    Sr, Tr = case["S0"], case["T0"]
    for k in range(K):
        Lr, Sr, Tr = onet.forward(Xb64, case["p"], case["c"], case["lam"], Sr, Tr, [rho_k[k]], [tau_k[k]])
        if k + 1 < K:
            Sr, Tr = _bf16(Sr), _bf16(Tr)
    for got, want in ((L, Lr), (S, Sr), (T, Tr)):
        scale = max(np.abs(want).max(), np.abs(Xb64).max())
        assert np.linalg.norm(got - want) <= 2.0 ** -9 * max(np.linalg.norm(want), 1e-30)
        assert np.abs(got - want).max() <= 2.0 ** -6 * scale
