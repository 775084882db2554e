"""Accuracy of the covariance estimates on the GPU (Sect. 3, Sect. 5.3):
element variances of the LC and sample covariances, the predicted and the
measured chi^2, and the eigenvalue check, against the oracle."""
import math

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


@pytest.fixture(scope="module")
def ctx(tp):
    c = tp.Context(0)
    yield c
    c.close()


def _lc_parts(nbin, n_mock, seed):
    xa1, xa2, xb = synth.synthetic_xi_variants(seed, n_mock, nbin)
    return oracle.lc_cov(xa1, xa2, xb, 1, 50.0)


def _d(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("nbin", [1, 37, 200, 600])
@pytest.mark.parametrize("M_a,M", [(1, 50.0), (1, math.inf), (2, 4.0)])
def test_covcov_var_parity(tp, ctx, nbin, M_a, M):
    ref = _lc_parts(nbin, 300, 80 + nbin)
    A, B = ref["A"], ref["B"]
    var = ctx.tpcf_covcov_var(_d(A), _d(B), 300, M_a, M)
    vs = ctx.tpcf_covcov_var(_d(ref["C_lc"]), None, 300)
    assert ctx.tpcf_sync() == tp.TPCF_OK
    want = oracle.covcov_var(A, B, 300, M_a, M)
    want_s = oracle.covcov_var(ref["C_lc"], None, 300)
    assert np.max(np.abs(var.cpu().numpy() - want) / np.abs(want).max()) <= 1e-13
    assert np.max(np.abs(vs.cpu().numpy() - want_s) / np.abs(want_s).max()) <= 1e-13


@pytest.mark.parametrize("nbin", [1, 40, 200, 600])
def test_chi2_parity(tp, ctx, nbin):
    ref = _lc_parts(nbin, 300, 90 + nbin)
    other = _lc_parts(nbin, 300, 190 + nbin)
    A, B, C = (_d(ref[k]) for k in ("A", "B", "C_lc"))
    p_lc = ctx.tpcf_chi2_predict(A, B, C, 1, 50.0)
    p_smp = ctx.tpcf_chi2_predict(C, None, C)
    meas = ctx.tpcf_chi2(_d(other["C_lc"]), C, C)
    assert ctx.tpcf_sync() == tp.TPCF_OK
    assert float(p_lc) == pytest.approx(oracle.chi2_predict(ref["A"], ref["B"], ref["C_lc"], 1, 50.0), rel=1e-12)
    assert float(p_smp) == pytest.approx(oracle.chi2_predict(ref["C_lc"], None, ref["C_lc"]), rel=1e-12)
    assert float(meas) == pytest.approx(oracle.chi2(other["C_lc"], ref["C_lc"], ref["C_lc"]), rel=1e-12)


@pytest.mark.parametrize("n", [1, 2, 3, 37, 200, 472, 473, 600, 1024])
def test_eigvalsh_parity(tp, ctx, n):
    """Eigenvalues of an LC covariance built from few mocks (indefinite once nbin > n_mock: A is a
    difference of covariances) against LAPACK; 472 is the largest order whose matrix the reduction keeps in
    the cluster's shared memory, 473 the smallest it reduces in device memory."""
    ref = _lc_parts(n, max(2, min(n // 2, 400)), 100 + n)
    C = 0.5 * (ref["C_lc"] + ref["C_lc"].T)
    w = ctx.tpcf_eigvalsh(_d(C))
    assert ctx.tpcf_sync() == tp.TPCF_OK
    want = oracle.eigvalsh(C)
    scale = max(np.abs(want).max(), 1e-300)
    assert np.max(np.abs(w.cpu().numpy() - want)) <= 1e-11 * scale
    if n >= 37:
        assert want[0] < 0.0 and w.cpu().numpy()[0] < 0.0     # the check the paper recommends


def test_eigvalsh_structured(tp, ctx):
    """Already-diagonal input (no reflection needed), repeated eigenvalues, a known spectrum."""
    rng = np.random.default_rng(9)
    D = np.diag(rng.uniform(-1.0, 3.0, 50))
    Q, _ = np.linalg.qr(rng.standard_normal((64, 64)))
    lam = np.sort(np.concatenate([np.full(10, 2.0), rng.uniform(-5.0, 5.0, 54)]))
    K = (Q * lam) @ Q.T
    K = 0.5 * (K + K.T)
    for M, want in ((D, np.sort(np.diag(D))), (K, lam), (np.zeros((5, 5)), np.zeros(5))):
        w = ctx.tpcf_eigvalsh(_d(M))
        assert ctx.tpcf_sync() == tp.TPCF_OK
        assert np.max(np.abs(w.cpu().numpy() - want)) <= 1e-12 * max(1.0, np.abs(want).max())


def test_accuracy_calls_reject_bad_arguments(tp, ctx):
    Z = torch.zeros((4, 4), dtype=torch.float64, device=DEV)
    with pytest.raises(tp.TpcfError):
        ctx.tpcf_covcov_var(Z, Z, 1)                 # n_mock < 2
    with pytest.raises(tp.TpcfError):
        ctx.tpcf_covcov_var(Z, Z, 10, 2, 1.0)        # M < M_a
    with pytest.raises(tp.TpcfError):
        ctx.tpcf_eigvalsh(torch.zeros((1025, 1025), dtype=torch.float64, device=DEV))
