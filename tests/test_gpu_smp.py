"""The brute-force (Smp) covariance path on the GPU, against the oracle.

Smp is the estimate the LC covariance replaces (Sect. 2.1, Sect. 2.2): every
mock is counted against all M = 50 random subsets in one batched launch,
the split Landy-Szalay estimator runs over all of them, and the covariance is
the plain sample covariance of Eq. (bruteforce) over the mocks.
"""
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


def _cov_err(C, ref):
    d = np.sqrt(np.diag(ref))
    return float(np.max(np.abs(C - ref) / np.outer(d, d)))


@pytest.mark.parametrize("n_mock,nbin", [(2, 3), (57, 40), (301, 200), (3500, 200), (130, 400)])
@pytest.mark.parametrize("prec,tol", [("TPCF_FP64", 1e-12), ("TPCF_TF32X3", 1e-6), ("TPCF_BF16X3", 1e-6)])
def test_sample_cov_parity(tp, ctx, n_mock, nbin, prec, tol):
    """Eq. (bruteforce) for one variant: float64 within 1e-12, the split-precision tensor-core Gram
    within 1e-6 (normalised by the oracle's diagonal)."""
    xi = synth.synthetic_xi_variants(61, n_mock, nbin)[2]
    C = ctx.tpcf_sample_cov(torch.from_numpy(np.ascontiguousarray(xi)).to(DEV), getattr(tp, prec))
    assert ctx.tpcf_sync() == tp.TPCF_OK
    err = _cov_err(C.cpu().numpy(), oracle.sample_cov(xi))
    assert err <= tol, err


def test_sample_cov_rejects_bad_arguments(tp, ctx):
    xi = torch.zeros((1, 5), dtype=torch.float64, device=DEV)
    with pytest.raises(tp.TpcfError):
        ctx.tpcf_sample_cov(xi)
    with pytest.raises(tp.TpcfError):
        ctx.tpcf_sample_cov(torch.zeros((4, 5), dtype=torch.float64, device=DEV), precision=99)


def test_smp_m50_counts_ls_cov(tp, ctx):
    """Five Neyman-Scott mocks, each with M = 50 random subsets of N_d points, 10 s bins on [10, 60) x 3 mu bins:
    counts bit-exact, xi over all 50 subsets within 1e-12, Smp covariance within 1e-12."""
    n, n_mock, M = 1200, 5, 50
    w = synth.SMALL
    mocks = [w.make_mock(200 + m, n_d=n, M=M) for m in range(n_mock)]
    edges = np.linspace(10.0, 60.0, 11)
    tb = tp.make_binning(edges, 3, tp.TPCF_PERIODIC, w.L)
    ob = oracle.Binning(edges, 3, oracle.PERIODIC, w.L)
    dm = [{"data": torch.from_numpy(mk.data).to(DEV),
           "randoms": torch.from_numpy(np.concatenate(mk.randoms)).to(DEV),
           "offsets": [i * n for i in range(M + 1)]} for mk in mocks]
    out = ctx.tpcf_count(dm, tb, mode=tp.TPCF_BATCHED)
    assert ctx.tpcf_sync() == tp.TPCF_OK
    assert out["dr"].shape == (n_mock, M, ob.nbin) and out["rr"].shape == (n_mock, M, ob.nbin)
    refs = [oracle.count_mock(mk.data, mk.randoms, ob) for mk in mocks]
    for m, ref in enumerate(refs):
        assert np.array_equal(out["dd"][m].cpu().numpy(), ref["DD"]), m
        assert np.array_equal(out["dr"][m].cpu().numpy(), ref["DR"]), m
        assert np.array_equal(out["rr"][m].cpu().numpy(), ref["RR"]), m
    sel = list(range(M))
    n_d, n_r = [n] * n_mock, [[n] * M for _ in range(n_mock)]
    xi = ctx.tpcf_ls(out["dd"], out["dr"], out["rr"], n_d, n_r, sel)
    assert ctx.tpcf_sync() == tp.TPCF_OK
    xi_ref = np.array([oracle.ls(r["DD"], r["DR"], r["RR"], n, [n] * M, sel) for r in refs])
    assert np.max(np.abs(xi.cpu().numpy() - xi_ref) / (1.0 + np.abs(xi_ref))) <= 1e-12
    C = ctx.tpcf_sample_cov(xi, tp.TPCF_FP64)
    assert ctx.tpcf_sync() == tp.TPCF_OK
    assert _cov_err(C.cpu().numpy(), oracle.sample_cov(xi_ref)) <= 1e-12

