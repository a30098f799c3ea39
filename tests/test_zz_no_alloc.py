"""The allocation-free initial-labels entry point (respca_init_labels_noalloc)
gives the same labels as respca_init_labels, on two calls in a row.

It exists for callers that may not allocate device memory while it runs
(CUDA-graph capture, caller-owned memory pools, hard budgets); its scratch is
a static device array inside the library.  The file is named so that pytest
collects it last."""
import numpy as np
import pytest

from paper_1904_07497_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A).T)).cuda().T


def test_noalloc_labels_match_handle_path_twice():
    from paper_1904_07497_gb300 import respca
    respca.load()
    cases = [(synth.lowrank_sparse(600, 520, 12, 0.05, seed=71), 12, 5),
             (synth.lowrank_sparse(130, 90, 4, 0.1, seed=72), 4, 9)]
    for pr, c, seed in cases:          # a larger call, then a smaller one
        X = _dev(pr.X)
        n = X.shape[1]
        solver = respca.Solver(seed=seed)
        want, want_passes = solver.init_labels(X, c)
        solver.close()
        p = torch.full((n,), -7, device="cuda", dtype=torch.int32)
        passes = respca.respca_init_labels_noalloc(X, c, p, seed=seed)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(p.cpu().numpy(), want.cpu().numpy())
        assert passes == want_passes


def test_noalloc_rejects_oversized_requests():
    from paper_1904_07497_gb300 import respca
    X = torch.zeros((200_000, 64), device="cuda").T.contiguous().T   # (d, n) col-major
    p = torch.zeros(64, device="cuda", dtype=torch.int32)
    with pytest.raises(respca.RespcaError) as e:
        respca.respca_init_labels_noalloc(X, 60, p)      # mu alone needs 4*60*200000 = 48 MB
    assert e.value.status == respca.RESPCA_ERR_UNSUPPORTED
