"""Host-side checks of the C ABI (no GPU): the library builds and loads, it
exports every entry point include/fr.h declares, and its host arithmetic
(Sec. 5.4 amortisation formulas, configuration space, cost-model features)
behaves as specified.  No kernel is launched here."""
import math
import os

import pytest

from paper_1910_08498_gb300 import _lib as L

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "amortization_examples.txt")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(L.LIB_PATH):
        from paper_1910_08498_gb300.build import build
        build()
    return L.lib()


def test_every_declared_symbol_is_exported(lib):
    names = L.declared_symbols()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_abi_version_and_param_count(lib):
    hdr = open(L.HEADER).read()
    assert "#define FR_ABI_VERSION 1" in hdr
    assert L.fr_mlp_num_params() == 16 * 64 + 64 + 64 * 64 + 64 + 64 + 1


def _golden():
    rows = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        kind, *kv = line.split()
        rows[kind] = {k: float(v) for k, v in (x.split("=") for x in kv)}
    return rows


def test_paper_worked_examples(lib):
    g = _golden()
    inv = g["invocations"]
    n = L.fr_invocations_to_amortize(inv["rp"], inv["s"], inv["t_avg"], inv["t_well"])
    assert n == pytest.approx(inv["n"], rel=1e-12)
    sm = g["samples"]
    s = L.fr_random_search_steps(sm["r"], sm["p"])
    assert math.ceil(s) == sm["s"]
    assert s == pytest.approx(229.105, abs=1e-3)


def test_relative_performance_consistent_with_invocations(lib):
    # Eq. (performance) at the n of Eq. (invocations) gives back 1/rp... i.e.
    # the ratio of runtimes T_dyn / T_orac equals 1 / rp_required
    for rp, s, ta, tw in [(0.9, 100, 10, 5), (0.95, 50, 3, 2), (0.8, 230, 7, 1)]:
        n = L.fr_invocations_to_amortize(rp, s, ta, tw)
        ratio = L.fr_relative_performance(s, ta, tw, n)
        assert 1.0 / ratio == pytest.approx(rp, rel=1e-12)
    assert L.fr_relative_performance(0, 10, 5, 100) == 1.0
    assert L.fr_relative_performance(100, 5, 5, 100) == 1.0


def test_configuration_space(lib):
    n = L.fr_num_configs()
    assert n == 55
    descs = [L.fr_describe_config(i) for i in range(n)]
    assert len(set(descs)) == n
    assert sum(d.startswith("gather ") for d in descs) == 36
    assert sum(d.startswith("gather2 ") for d in descs) == 11
    assert sum("w=otf" in d for d in descs) == 12
    assert sum("w=poly" in d for d in descs) == 27
    with pytest.raises(L.FrError):
        L.fr_describe_config(n)


def test_features_normalised_and_distinct(lib):
    feats = [tuple(L.fr_config_features(i, 256, 5000, 1.9)) for i in range(L.fr_num_configs())]
    assert len(set(feats)) == len(feats)
    for f in feats:
        assert len(f) == 16 and all(-1e-6 <= x <= 1.5 for x in f)
    a = L.fr_config_features(0, 128, 1000, 1.9)
    b = L.fr_config_features(0, 256, 1000, 1.9)
    assert a[9] != b[9]


def test_error_strings(lib):
    for s in range(10):
        assert L.fr_error_string(s)
    assert L.fr_error_string(123) == "unknown status"


def test_create_rejects_bad_arguments_without_touching_a_device(lib):
    import ctypes
    h = ctypes.c_void_p(1)
    bad = [(31, L.fr_blob(1.9, 15.0, 0, 10000), L.FR_ERR_UNSUPPORTED),
           (4, L.fr_blob(1.9, 15.0, 0, 10000), L.FR_ERR_INVALID_ARG),
           (1024, L.fr_blob(1.9, 15.0, 0, 10000), L.FR_ERR_INVALID_ARG),
           (32, L.fr_blob(1.9, 15.0, 1, 10000), L.FR_ERR_UNSUPPORTED),
           (32, L.fr_blob(3.5, 15.0, 0, 10000), L.FR_ERR_UNSUPPORTED),
           (32, L.fr_blob(-1.0, 15.0, 0, 10000), L.FR_ERR_INVALID_ARG),
           (32, L.fr_blob(1.9, 15.0, 0, 1), L.FR_ERR_INVALID_ARG)]
    for S, b, want in bad:
        assert lib.fr_create(S, ctypes.byref(b), ctypes.byref(h)) == want
        assert h.value is None
    assert lib.fr_insert(None, None, 0, None, 1, None) == L.FR_ERR_INVALID_ARG
    assert lib.fr_destroy(None) == L.FR_OK
