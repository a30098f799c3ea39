"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/respca.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?\s*\**\s*(respca_[a-z_]+)\s*\(",
                            src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1904_07497_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for want in ["respca_create", "respca_solve", "respca_solve_batched", "respca_destroy",
                 "respca_solve_host", "respca_init_labels", "respca_config_default",
                 "respca_status_string", "respca_last_error"]:
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), f"{name} not exported"


def test_status_strings_and_defaults(lib):
    from paper_1904_07497_gb300 import respca
    respca._lib = None
    cfg = respca.respca_config_default()
    assert cfg.rho0 == 1e-4 and cfg.kappa == 1.5 and cfg.kmeans_max_iter == 100
    l = respca.load()
    assert l.respca_status_string(0) == b"ok"
    assert l.respca_status_string(2) == b"non-finite input"
    assert l.respca_destroy(None) == 0


def test_binding_struct_sizes_match_header(lib):
    """The ctypes mirrors must have the C layout (compiled probe with gcc)."""
    import subprocess
    import tempfile
    from paper_1904_07497_gb300 import respca
    src = ('#include "respca.h"\n#include <stdio.h>\n#include <stddef.h>\n'
           'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n",'
           ' sizeof(respca_config),'
           ' sizeof(respca_stats), sizeof(respca_warm), sizeof(respca_problem),'
           ' offsetof(respca_stats, ms_total), offsetof(respca_problem, p),'
           ' sizeof(respca_spectral_info), offsetof(respca_config, spectral_scale),'
           ' offsetof(respca_stats, x_norm), sizeof(respca_batch_options),'
           ' offsetof(respca_batch_options, ms_kernel), offsetof(respca_stats, ms_dense16),'
           ' offsetof(respca_stats, dense16_passes), offsetof(respca_stats, copy16_iters));return 0;}\n')
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "probe.c")
        exe = os.path.join(td, "probe")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        got = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(respca.respca_config), ctypes.sizeof(respca.respca_stats),
            ctypes.sizeof(respca.respca_warm), ctypes.sizeof(respca.respca_problem),
            respca.respca_stats.ms_total.offset, respca.respca_problem.p.offset,
            ctypes.sizeof(respca.respca_spectral_info), respca.respca_config.spectral_scale.offset,
            respca.respca_stats.x_norm.offset, ctypes.sizeof(respca.respca_batch_options),
            respca.respca_batch_options.ms_kernel.offset, respca.respca_stats.ms_dense16.offset,
            respca.respca_stats.dense16_passes.offset, respca.respca_stats.copy16_iters.offset]
    assert got == want


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1904_07497_gb300 import respca
    monkeypatch.setattr(respca, "_lib", None)
    monkeypatch.setattr(respca, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="not built"):
        respca.load()


def test_config_validation_needs_no_gpu(lib):
    """respca_create rejects inconsistent settings before touching a device."""
    from paper_1904_07497_gb300 import respca
    l = respca.load()
    h = ctypes.c_void_p()
    for field, value in (("p_step", 2), ("precision", 3), ("s_norm", 5), ("stop_after_ramp", 7)):
        cfg = respca.respca_config_default()
        setattr(cfg, field, value)
        assert l.respca_create(ctypes.byref(h), ctypes.byref(cfg)) == respca.RESPCA_ERR_INVALID_ARG, field
    cfg = respca.respca_config_default()
    cfg.p_step, cfg.precision = 1, 1          # the spectral p step runs in FP32 only
    assert l.respca_create(ctypes.byref(h), ctypes.byref(cfg)) == respca.RESPCA_ERR_INVALID_ARG
    cfg = respca.respca_config_default()
    cfg.p_step, cfg.spectral_scale = 1, 0.0
    assert l.respca_create(ctypes.byref(h), ctypes.byref(cfg)) == respca.RESPCA_ERR_INVALID_ARG


def test_net_schedule_matches_oracle(lib):
    """respca_net_schedule is host arithmetic: rho_k = rho kappa^k e^theta_k,
    tau_k = e^phi_k / rho_k, checked against the FP64 network oracle."""
    import numpy as np
    from oracle import warmnet
    from paper_1904_07497_gb300 import respca
    g = np.random.default_rng(4)
    m = g.uniform(-1.0, 1.0, 16).astype(np.float32)
    r, t = respca.respca_net_schedule(0.37, 1.5, m.tolist())
    r_ref, t_ref = warmnet.schedule(0.37, 1.5, m[:8].astype(np.float64), m[8:].astype(np.float64))
    np.testing.assert_allclose(r, r_ref, rtol=1e-14)
    np.testing.assert_allclose(t, t_ref, rtol=1e-14)
    with pytest.raises(respca.RespcaError):
        respca.respca_net_schedule(-1.0, 1.5, m.tolist())
