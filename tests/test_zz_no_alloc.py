"""The allocation-free initial-labels entry point (respca_init_labels_noalloc).

It serves callers that may not allocate device memory while it runs (their
memory belongs to their own pool or to a hard budget); its scratch is a static
device array inside the library.  Its labels are checked against the FP64
oracle's k-means++ + Lloyd labels and against the handle path
(respca_init_labels), on two or more calls in a row that share the array.  The
file is named so that pytest collects it last; every case builds its own
inputs, so it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

import oracle
from paper_1904_07497_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(A, ld=None, dtype=None):
    """numpy (d, n) -> column-major CUDA view (d, n) with leading dimension ld."""
    d, n = A.shape
    ld = d if ld is None else ld
    buf = torch.zeros((n, ld), dtype=torch.float32)
    buf[:, :d] = torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float32).T))
    if dtype is not None:
        buf = buf.to(dtype)
    return buf.cuda()[:, :d].T


CASES = [
    # (d, n, rank, sparsity, c, seed, leading dim, X dtype)
    (600, 520, 12, 0.05, 12, 5, None, None),              # FP32, 16-byte rows
    (131, 90, 4, 0.10, 4, 9, 133, None),                  # ldx % 4 != 0: scalar loads
    (256, 300, 8, 0.05, 8, 2, None, torch.bfloat16),      # BF16 X
    (300, 400, 10, 0.05, 80, 4, None, None),              # c > 64 (fits the 32 MiB array)
]


def test_noalloc_labels_match_oracle_and_handle_path():
    from paper_1904_07497_gb300 import respca
    oracle.build()
    respca.load()
    for d, n, r, sp, c, seed, ld, dt in CASES:       # successive calls share the scratch array
        pr = synth.lowrank_sparse(d, n, r, sp, seed=70 + seed)
        X = _dev(pr.X, ld, dt)
        X64 = X.float().T.contiguous().cpu().numpy().T.astype(np.float64)   # the values the GPU reads
        want, want_passes = oracle.init_labels(X64, c, seed=seed)
        solver = respca.Solver(seed=seed)
        hp, hpasses = solver.init_labels(X, c)
        solver.close()
        p = torch.full((n,), -7, device="cuda", dtype=torch.int32)
        passes = respca.respca_init_labels_noalloc(X, c, p, seed=seed)
        torch.cuda.synchronize()
        got = p.cpu().numpy()
        np.testing.assert_array_equal(got, want)
        np.testing.assert_array_equal(got, hp.cpu().numpy())
        assert passes == want_passes == hpasses


def test_noalloc_repeat_call_gives_same_labels():
    """A second identical call after a different one (the array keeps the
    previous call's contents) gives the same labels."""
    from paper_1904_07497_gb300 import respca
    pr = synth.lowrank_sparse(400, 350, 6, 0.05, seed=81)
    X = _dev(pr.X)
    out = []
    for k in range(2):
        p = torch.zeros(350, device="cuda", dtype=torch.int32)
        out.append((respca.respca_init_labels_noalloc(X, 6, p, seed=11), p.cpu().numpy()))
        other = _dev(synth.lowrank_sparse(90, 700, 3, 0.1, seed=82).X)
        respca.respca_init_labels_noalloc(other, 3, torch.zeros(700, device="cuda", dtype=torch.int32))
    assert out[0][0] == out[1][0]
    np.testing.assert_array_equal(out[0][1], out[1][1])


def test_noalloc_rejects_oversized_and_bad_outputs():
    from paper_1904_07497_gb300 import respca
    X = torch.zeros((64, 200_000), device="cuda").T                      # (d, n) col-major
    p = torch.zeros(64, device="cuda", dtype=torch.int32)
    with pytest.raises(respca.RespcaError) as e:
        respca.respca_init_labels_noalloc(X, 60, p)      # mu alone needs 4*60*200000 = 48 MB
    assert e.value.status == respca.RESPCA_ERR_UNSUPPORTED
    Xs = torch.ones((32, 40), device="cuda").T.contiguous().T
    with pytest.raises(ValueError):
        respca.respca_init_labels_noalloc(Xs, 3, torch.zeros(39, device="cuda", dtype=torch.int32))
    with pytest.raises(ValueError):
        respca.respca_init_labels_noalloc(Xs, 3, torch.zeros(40, device="cuda", dtype=torch.int64))
    with pytest.raises(ValueError):
        respca.respca_init_labels_noalloc(Xs, 3, torch.zeros(40, dtype=torch.int32))
