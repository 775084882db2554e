"""tpcf_lc_cov_noalloc: the float64 LC covariance for callers that cannot allocate.

Some callers cannot call cudaMalloc while they run (services that reserve all
GPU memory at start-up, code that must not trigger cudaMalloc's implicit device
synchronisation).  The allocation-free entry point keeps its scratch in a fixed
array inside the library; here it is called through the C ABI and checked
against tpcf_lc_cov on two calls in a row, within the covariance tolerance of
the other tests (1e-12, normalised by sqrt(C^a_ii C^a_jj)).  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2205_11852_gb300 as tp
    return tp


def _noalloc(tp, xa1, xa2, xb, M_a, M):
    n_mock, nbin = xa1.shape
    outs = [torch.full((nbin, nbin), float("nan"), dtype=torch.float64, device="cuda:0") for _ in range(5)]
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = tp.lib().tpcf_lc_cov_noalloc(p(xa1), p(xa2), p(xb), n_mock, nbin, M_a, float(M), *[p(o) for o in outs],
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, dict(zip(("C_lc", "Ca", "Cb", "A", "B"), outs))


def test_noalloc_matches_lc_cov_twice(tp):
    ctx = tp.Context(0)
    for call, (seed, n_mock, nbin, M) in enumerate(((51, 150, 37, 50.0), (52, 301, 200, float("inf")))):
        xs = [torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")
              for a in synth.synthetic_xi_variants(seed, n_mock, nbin)]
        rc, got = _noalloc(tp, *xs, 1, M)
        assert rc == tp.TPCF_OK, call
        ref = ctx.tpcf_lc_cov(*xs, 1, M, tp.TPCF_FP64)
        torch.cuda.synchronize()
        d = torch.sqrt(torch.diag(ref["Ca"]))
        scale = torch.outer(d, d)
        for k in ("C_lc", "Ca", "Cb", "A", "B"):
            err = (torch.abs(got[k] - ref[k]) / scale).max().item()
            assert err <= 1e-12, (call, k, err)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(tp):
    x = torch.zeros((2, 1), dtype=torch.float64, device="cuda:0")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    # 3 * 2 * 900 + 3 * 900 + 3 * 900^2 > 2^21: refused before any GPU work
    rc = tp.lib().tpcf_lc_cov_noalloc(p(x), p(x), p(x), 2, 900, 1, 50.0, p(x), None, None, None, None, None)
    assert rc == tp.TPCF_ERR_RANGE
