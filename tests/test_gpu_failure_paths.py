"""Failure paths of the library, each made without faulting the GPU.

* Bounded device wait: the split-precision Gram kernel's wait for its
  tensor-core products has a limit (a context option).  With the test-only
  switch one CTA waits for its operand copies and then issues no product and
  no commit, so with a short limit its wait runs out while nothing of it is in
  flight: the kernel reports the timeout, frees its tensor memory and
  returns.  tpcf_sync must return TPCF_ERR_TIMEOUT, and the same context must
  then give the correct covariance (against the float64 oracle).
* Allocation failure: TPCF_TEST_FAIL_ALLOC=n fails the context's n-th device
  allocation on the host.  The call returns TPCF_ERR_NOMEM with nothing
  enqueued, and the next call on the context counts correctly (against the
  oracle).
* Launch failure: TPCF_TEST_FAIL_COUNT=n makes the n-th tpcf_count return
  TPCF_ERR_CUDA as a failed launch would; the context then refuses work with
  TPCF_ERR_STATE, and a new context works.
"""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def tp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2205_11852_gb300 as tp
    return tp


def _cov_err(got, ref):
    d = np.sqrt(np.abs(np.diag(ref["Ca"])))
    return float(np.max(np.abs(got - ref["C_lc"]) / np.outer(d, d)))


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_gram_wait_runs_out_then_context_recovers(tp, prec):
    pr = {"tf32x3": tp.TPCF_TF32X3, "bf16x3": tp.TPCF_BF16X3}[prec]
    xs = synth.synthetic_xi_variants(61, 300, 200)
    gx = [torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in xs]
    ref = oracle.lc_cov(*xs, 1, 50.0)
    ctx = tp.Context(0)
    try:
        ctx.tpcf_set_option(tp.TPCF_OPT_WAIT_LIMIT, 2000)
        ctx.tpcf_set_option(tp.TPCF_OPT_TEST_SKIP_MMA, 1)
        ctx.tpcf_lc_cov(*gx, 1, 50.0, pr, want_parts=False)
        with pytest.raises(tp.TpcfError) as ei:
            ctx.tpcf_sync()
        assert ei.value.code == tp.TPCF_ERR_TIMEOUT
        # the same context, default limit, no skip: a correct covariance
        ctx.tpcf_set_option(tp.TPCF_OPT_TEST_SKIP_MMA, 0)
        ctx.tpcf_set_option(tp.TPCF_OPT_WAIT_LIMIT, 0)
        out = ctx.tpcf_lc_cov(*gx, 1, 50.0, pr, want_parts=False)
        assert ctx.tpcf_sync() == tp.TPCF_OK
        assert _cov_err(out["C_lc"].cpu().numpy(), ref) <= 1e-6
    finally:
        ctx.close()


def test_wait_limit_option_validated(tp):
    ctx = tp.Context(0)
    try:
        with pytest.raises(tp.TpcfError) as ei:
            ctx.tpcf_set_option(tp.TPCF_OPT_WAIT_LIMIT, -1)
        assert ei.value.code == tp.TPCF_ERR_ARG
    finally:
        ctx.close()


def _small_case(tp):
    w = synth.SMALL
    mk = w.make_mock(3, n_d=1500)
    ob = oracle.Binning(w.s_edges, w.n_mu, oracle.PERIODIC, w.L)
    ref = oracle.count_mock(mk.data, mk.randoms, ob)
    n_r = [len(r) for r in mk.randoms]
    dm = [{"data": torch.from_numpy(np.ascontiguousarray(mk.data)).to(DEV),
           "randoms": torch.from_numpy(np.ascontiguousarray(np.concatenate(mk.randoms))).to(DEV),
           "offsets": [0, n_r[0], n_r[0] + n_r[1]]}]
    return dm, tp.make_binning(w.s_edges, w.n_mu, tp.TPCF_PERIODIC, w.L), ref


def _assert_counts(out, ref):
    assert np.array_equal(out["dd"][0].cpu().numpy(), ref["DD"])
    assert np.array_equal(out["dr"][0].cpu().numpy(), ref["DR"])
    assert np.array_equal(out["rr"][0].cpu().numpy(), ref["RR"])


@pytest.mark.parametrize("nth", [1, 3])
def test_injected_allocation_failure_then_recovery(tp, nth, monkeypatch):
    dm, b, ref = _small_case(tp)
    monkeypatch.setenv("TPCF_TEST_FAIL_ALLOC", str(nth))
    ctx = tp.Context(0)
    monkeypatch.delenv("TPCF_TEST_FAIL_ALLOC")
    try:
        with pytest.raises(tp.TpcfError) as ei:
            ctx.tpcf_count(dm, b)
        assert ei.value.code == tp.TPCF_ERR_NOMEM
        assert ctx.tpcf_sync() == tp.TPCF_OK
        out = ctx.tpcf_count(dm, b)
        assert ctx.tpcf_sync() == tp.TPCF_OK
        _assert_counts(out, ref)
    finally:
        ctx.close()


def test_injected_launch_failure_marks_context_unusable(tp, monkeypatch):
    dm, b, ref = _small_case(tp)
    monkeypatch.setenv("TPCF_TEST_FAIL_COUNT", "2")
    ctx = tp.Context(0)
    monkeypatch.delenv("TPCF_TEST_FAIL_COUNT")
    try:
        out = ctx.tpcf_count(dm, b)
        assert ctx.tpcf_sync() == tp.TPCF_OK
        _assert_counts(out, ref)
        with pytest.raises(tp.TpcfError) as ei:
            ctx.tpcf_count(dm, b)
        assert ei.value.code == tp.TPCF_ERR_CUDA
        for call in (lambda: ctx.tpcf_sync(), lambda: ctx.tpcf_count(dm, b)):
            with pytest.raises(tp.TpcfError) as ei:
                call()
            assert ei.value.code == tp.TPCF_ERR_STATE
    finally:
        ctx.close()
    ctx2 = tp.Context(0)
    try:
        out = ctx2.tpcf_count(dm, b)
        assert ctx2.tpcf_sync() == tp.TPCF_OK
        _assert_counts(out, ref)
    finally:
        ctx2.close()
