"""The C-ABI library builds, loads and exports every entry point of include/tpcf.h.

Also checks the library's host-side planning (exact integer thresholds) against
the oracle; no CUDA work is launched, so these run without a GPU.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import __graft_entry__
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tp():
    __graft_entry__.build()
    import paper_2205_11852_gb300 as tp
    return tp


def header_functions():
    src = open(os.path.join(ROOT, "include", "tpcf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\s*\*)\s*(tpcf_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(tp):
    names = header_functions()
    assert len(names) >= 10
    lib = ctypes.CDLL(str(tp._binding._LIBPATH))
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(tp.EXPORTED)


def test_library_is_sm103a_build(tp):
    # the build script compiles for exactly one target: sm_103a
    import importlib.util
    spec = importlib.util.spec_from_file_location("b", os.path.join(ROOT, "paper_2205_11852_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


@pytest.mark.parametrize("geom,L", [(0, 1000.0), (1, 2400.0), (0, 333.3), (1, 77.7)])
def test_thresholds_match_oracle(tp, geom, L):
    rng = np.random.default_rng(11)
    edges = np.concatenate([[0.0], np.sort(rng.uniform(0.0, L / 3.2, 60))])
    edges = np.unique(edges)
    b = tp.make_binning(edges, 1, geom, L)
    assert tp.tpcf_thresholds(b) == oracle.thresholds(edges, geom, L)
    # exactly representable squares are not rounded up
    b2 = tp.make_binning([0.0, 1.0, 2.0, 3.0], 1, tp.TPCF_PERIODIC, 1024.0)
    assert tp.tpcf_thresholds(b2) == [0, 2 ** 44, 2 ** 46, 9 * 2 ** 44]


def test_thresholds_tiny_and_linear_edges(tp):
    for edges, L, geom in (([0.0, 1e-9, 1e-6, 0.5], 10.0, 0), (list(np.linspace(0, 200, 41)), 1000.0, 0),
                           (list(np.linspace(0, 200, 41)), 2400.0, 1)):
        b = tp.make_binning(edges, 1, geom, L)
        assert tp.tpcf_thresholds(b) == oracle.thresholds(edges, geom, L)


def test_bad_binning_rejected_on_host(tp):
    with pytest.raises(tp.TpcfError):
        tp.tpcf_thresholds(tp.make_binning([0.0, 2.0, 1.0], 1, tp.TPCF_PERIODIC, 100.0))
    with pytest.raises(tp.TpcfError):
        tp.tpcf_thresholds(tp.make_binning([0.0, 40.0], 1, tp.TPCF_PERIODIC, 100.0))  # s_max > L/3


def test_multipole_matrix_matches_oracle(tp):
    """The host-side Legendre multipole matrix of the C ABI against the oracle's (no GPU needed)."""
    for n_s, n_mu, ells in ((1, 1, (0,)), (2, 4, (0, 2, 4)), (40, 10, (0, 2, 4)), (3, 100, (4, 0, 8))):
        P = tp.tpcf_multipole_matrix(n_s, n_mu, ells)
        ref = oracle.multipole_matrix(n_s, n_mu, ells)
        assert np.max(np.abs(P - ref)) <= 1e-13
    for bad in ((1,), (0, 3), (-2,), (66,)):
        with pytest.raises(tp.TpcfError):
            tp.tpcf_multipole_matrix(2, 4, bad)


def test_binding_constants_match_header(tp):
    """Every TPCF_ constant the binding exports has the value include/tpcf.h defines."""
    src = open(os.path.join(ROOT, "include", "tpcf.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"^#define\s+(TPCF_\w+)\s+(-?\d+)", src, flags=re.M)}
    names = [n for n in dir(tp) if n.startswith("TPCF_")]
    assert {"TPCF_HOST_INPUT", "TPCF_BATCHED", "TPCF_PER_LAUNCH", "TPCF_ERR_RANGE"} <= set(names)
    for n in names:
        assert n in defs, n
        assert getattr(tp, n) == defs[n], n
