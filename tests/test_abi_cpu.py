"""C ABI checks that need no GPU: the library loads, exports every symbol the header
declares, and rejects invalid arguments before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ulisse.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1501_05427_gb300 import build, ulisse
    build.build()
    return ulisse.load()


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(ulisse_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_api():
    names = _declared()
    for required in ("ulisse_create", "ulisse_kmv", "ulisse_solve", "ulisse_grad",
                     "ulisse_sgld_step", "ulisse_destroy", "ulisse_last_error"):
        assert required in names


def test_every_declared_symbol_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_1501_05427_gb300 import ulisse
    assert sorted(ulisse.EXPORTED) == _declared()


def test_config_default(lib):
    from paper_1501_05427_gb300 import ulisse
    cfg = ulisse.ulisse_config_default()
    assert cfg.q == 1.0 and cfg.beta == 1.0 and cfg.eps == 1e-8
    assert cfg.n_probes == 4 and cfg.probe_refresh == 1 and cfg.precision == 0
    # the fields after the original ones sit where the C struct has them
    assert cfg.pcg_delta == 0.0 and cfg.pcg_inner_tol == 1e-2 and cfg.pcg_inner_max == 100


@pytest.mark.parametrize("n,d,bad_cfg", [(0, 2, None), (10, 0, None), (10, 17, None),
                                         (10, 2, "n_probes"), (10, 2, "beta"),
                                         (10, 2, "q"), (10, 2, "refresh"), (10, 2, "cross"),
                                         (10, 2, "pcg_delta"), (10, 2, "pcg_tol"),
                                         (10, 2, "pcg_max"), (10, 2, "pcg_warm")])
def test_create_rejects_bad_arguments(lib, n, d, bad_cfg):
    from paper_1501_05427_gb300 import ulisse
    cfg = ulisse.ulisse_config_default()
    if bad_cfg == "n_probes":
        cfg.n_probes = 0
    elif bad_cfg == "beta":
        cfg.beta = -1.0
    elif bad_cfg == "q":
        cfg.q = float("nan")
    elif bad_cfg == "refresh":
        cfg.probe_refresh = 0
    elif bad_cfg == "cross":
        cfg.tc_cross_term = 3
    elif bad_cfg == "pcg_delta":
        cfg.pcg_delta = -0.5
    elif bad_cfg == "pcg_tol":
        cfg.pcg_delta, cfg.pcg_inner_tol = 0.1, 1.0
    elif bad_cfg == "pcg_max":
        cfg.pcg_delta, cfg.pcg_inner_max = 0.1, 0
    elif bad_cfg == "pcg_warm":
        cfg.pcg_delta, cfg.warm_start_probes = 0.1, 1
    X = np.zeros((max(n, 1), max(d, 1)), np.float32)
    y = np.zeros(max(n, 1), np.float32)
    h = ctypes.c_void_p()
    st = lib.ulisse_create_host(ctypes.byref(h), X.ctypes.data_as(ctypes.c_void_p),
                                y.ctypes.data_as(ctypes.c_void_p), n, d, ctypes.byref(cfg), None)
    assert st == ulisse.ULISSE_ERR_ARG
    assert not h.value
    assert len(lib.ulisse_last_error(None)) > 0


def test_null_pointers_rejected(lib):
    from paper_1501_05427_gb300 import ulisse
    cfg = ulisse.ulisse_config_default()
    h = ctypes.c_void_p()
    assert lib.ulisse_create(ctypes.byref(h), None, None, 10, 2, ctypes.byref(cfg), None) == 1
    assert lib.ulisse_kmv(None, None, -1, None, 1, None) == ulisse.ULISSE_ERR_ARG
    assert lib.ulisse_grad(None, None, 0, None, None) == ulisse.ULISSE_ERR_ARG
    assert lib.ulisse_dk_bilinear(None, None, None, None, 1, None, None) == ulisse.ULISSE_ERR_ARG
    assert lib.ulisse_kmv_noalloc_status(None, None) == ulisse.ULISSE_ERR_ARG
    assert lib.ulisse_set_tune(None, None, 0) == ulisse.ULISSE_ERR_ARG
    lib.ulisse_destroy(None)


def test_package_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1501_05427_gb300 import ulisse
    monkeypatch.setattr(ulisse, "_lib", None)
    monkeypatch.setattr(ulisse, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        ulisse.load()


def test_measure_ex2_rate_rejects_bad_arguments(lib):
    from paper_1501_05427_gb300 import ulisse
    r = ctypes.c_double()
    assert lib.ulisse_measure_ex2_rate(None, 0, ctypes.byref(r), None) == ulisse.ULISSE_ERR_ARG
    assert lib.ulisse_measure_ex2_rate(None, 5, None, None) == ulisse.ULISSE_ERR_ARG


def test_predict_rejects_bad_arguments(lib):
    from paper_1501_05427_gb300 import ulisse
    assert lib.ulisse_predict(None, None, None, 1, 0, None, None) == ulisse.ULISSE_ERR_ARG
