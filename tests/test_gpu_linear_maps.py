"""Linear maps before the covariance on the GPU (Sect. 2.3, Sect. 4.3): wider
bins from the pair counts, xi rows mapped by a matrix (the Legendre
multipoles), and the LC covariance of the mapped xi."""
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


def _dev(mk):
    offs = [0] + list(np.cumsum([len(r) for r in mk.randoms]))
    return {"data": torch.from_numpy(mk.data).to(DEV),
            "randoms": torch.from_numpy(np.concatenate(mk.randoms)).to(DEV), "offsets": offs}


@pytest.mark.parametrize("f_s,f_mu", [(1, 1), (2, 5), (4, 10), (5, 1), (20, 2), (40, 10)])
def test_rebin_counts_equal_direct_coarse_counts(tp, ctx, f_s, f_mu):
    """Counts in 40 s x 10 mu bins re-binned on the GPU equal the GPU's and the oracle's direct counts
    with the merged edges, bit for bit (incl. the 1-D function from counts co-added over mu)."""
    L, n = 600.0, 3000
    mocks = [synth.Workload("t", 71, 2, "periodic", L, (0, 0, 0), n, 2, 120.0, 40, 10, "x",
                            n_parent=5e-5, sigma=3.0).make_mock(m) for m in range(2)]
    fine = np.linspace(0.0, 120.0, 41)
    tf = tp.make_binning(fine, 10, tp.TPCF_PERIODIC, L)
    tc = tp.make_binning(fine[::f_s], 10 // f_mu, tp.TPCF_PERIODIC, L)
    oc = oracle.Binning(fine[::f_s], 10 // f_mu, oracle.PERIODIC, L)
    dm = [_dev(mk) for mk in mocks]
    of = ctx.tpcf_count(dm, tf)
    oc_gpu = ctx.tpcf_count(dm, tc)
    assert ctx.tpcf_sync() == tp.TPCF_OK
    for k in ("dd", "dr", "rr"):
        rb = ctx.tpcf_rebin_counts(of[k], 40, 10, f_s, f_mu)
        assert ctx.tpcf_sync() == tp.TPCF_OK
        assert torch.equal(rb, oc_gpu[k]), k
    for m, mk in enumerate(mocks):
        ref = oracle.count_mock(mk.data, mk.randoms, oc)
        assert np.array_equal(ctx.tpcf_rebin_counts(of["dd"], 40, 10, f_s, f_mu)[m].cpu().numpy(), ref["DD"])
        assert np.array_equal(ctx.tpcf_rebin_counts(of["rr"], 40, 10, f_s, f_mu)[m].cpu().numpy(), ref["RR"])


def test_rebin_rejects_bad_factors(tp, ctx):
    c = torch.zeros((3, 40 * 10), dtype=torch.int64, device=DEV)
    for f_s, f_mu in ((3, 1), (1, 3), (0, 1), (1, 0)):
        with pytest.raises(tp.TpcfError):
            ctx.tpcf_rebin_counts(c, 40, 10, f_s, f_mu)


@pytest.mark.parametrize("n_mock,n_s,n_mu,ells", [(1, 1, 1, (0,)), (57, 40, 10, (0, 2, 4)),
                                                  (301, 40, 5, (0, 2, 4)), (3500, 40, 5, (0, 2))])
def test_project_multipoles_parity(tp, ctx, n_mock, n_s, n_mu, ells):
    """xi rows mapped onto multipoles on the GPU against the oracle's matrix product (float64, 1e-12)."""
    nbin = n_s * n_mu
    xi = synth.synthetic_xi_variants(72, max(2, n_mock), nbin)[0][:n_mock]
    P = tp.tpcf_multipole_matrix(n_s, n_mu, ells)
    y = ctx.tpcf_project(torch.from_numpy(P).to(DEV), torch.from_numpy(np.ascontiguousarray(xi)).to(DEV))
    assert ctx.tpcf_sync() == tp.TPCF_OK
    ref = oracle.project(oracle.multipole_matrix(n_s, n_mu, ells), xi)
    scale = np.abs(xi).max(axis=1, keepdims=True) * n_mu + 1.0
    assert np.max(np.abs(y.cpu().numpy() - ref) / scale) <= 1e-12


def test_project_general_matrix_ragged(tp, ctx):
    """A dense random map with ragged sizes (tile tails in every dimension)."""
    rng = np.random.default_rng(73)
    P = rng.standard_normal((37, 203))
    x = rng.standard_normal((65, 203))
    y = ctx.tpcf_project(torch.from_numpy(P).to(DEV), torch.from_numpy(x).to(DEV))
    assert ctx.tpcf_sync() == tp.TPCF_OK
    ref = oracle.project(P, x)
    assert np.max(np.abs(y.cpu().numpy() - ref)) <= 1e-12 * np.abs(P).sum(axis=1).max() * np.abs(x).max()


@pytest.mark.parametrize("prec,tol", [("TPCF_FP64", 1e-12), ("TPCF_TF32X3", 1e-6)])
def test_lc_covariance_of_multipoles(tp, ctx, prec, tol):
    """The LC covariance of the multipoles (xi_a1, xi_a2, xi_b each mapped by the multipole matrix) against
    the oracle's; in float64 it also equals P C^LC P^T of the (s, mu) covariance (linearity)."""
    n_s, n_mu, n_mock = 40, 5, 400
    xa1, xa2, xb = synth.synthetic_xi_variants(74, n_mock, n_s * n_mu)
    P = tp.tpcf_multipole_matrix(n_s, n_mu, (0, 2, 4))
    Pd = torch.from_numpy(P).to(DEV)
    g = [torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in (xa1, xa2, xb)]
    y = [ctx.tpcf_project(Pd, a) for a in g]
    out = ctx.tpcf_lc_cov(*y, 1, 50.0, getattr(tp, prec))
    assert ctx.tpcf_sync() == tp.TPCF_OK
    Po = oracle.multipole_matrix(n_s, n_mu, (0, 2, 4))
    ref = oracle.lc_cov(*(oracle.project(Po, a) for a in (xa1, xa2, xb)), 1, 50.0)
    d = np.sqrt(np.diag(ref["Ca"]))
    sc = np.outer(d, d)
    assert np.max(np.abs(out["C_lc"].cpu().numpy() - ref["C_lc"]) / sc) <= tol
    if prec == "TPCF_FP64":
        full = oracle.lc_cov(xa1, xa2, xb, 1, 50.0)["C_lc"]
        assert np.max(np.abs(out["C_lc"].cpu().numpy() - Po @ full @ Po.T) / sc) <= 1e-10
    assert math.isfinite(float(out["C_lc"].abs().max()))
