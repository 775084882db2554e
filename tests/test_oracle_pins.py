"""Pins of the CPU oracle against facts it does not compute itself.

Each test checks the oracle against something independent: hand-worked
edge cases (tests/golden), a library pair counter (scipy's k-d tree),
exact arbitrary-precision arithmetic (mpmath), float64 re-derivations of
distances and angles, pair-total and split-sum invariants, analytic shell
volumes, the closed-form correlation function of the Neyman-Scott process,
numpy's covariance routine, the algebraic identities of the linear
construction (Eqs. CovAB and LCdef) and the analytic Poisson covariance of
Eq. (randomtheory).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _snap(u, geometry, L, origin=(0.0, 0.0, 0.0)):
    """Grid coordinates -> float64 positions exactly on the grid (x = u / q)."""
    bits = 32 if geometry == oracle.PERIODIC else 30
    return (np.asarray(u, dtype=np.float64).T * (L / 2.0 ** bits)) + np.asarray(origin)


# ---------------------------------------------------------------------------
# quantisation and thresholds
# ---------------------------------------------------------------------------

def test_quantize_special_values():
    L = 1000.0
    x = np.array([[0.0, L / 2, L / 4], [L, -1e-300, 3 * L / 4], [2 * L + L / 8, -L / 8, 0.0]])
    u = oracle.quantize(x, oracle.PERIODIC, L)
    assert u[:, 0].tolist() == [0, 2 ** 31, 2 ** 30]
    # x = L wraps to 0; a tiny negative value wraps to the top of the box (t - floor(t) rounds to 1)
    assert u[0, 1] == 0 and u[1, 1] == 0 and u[2, 1] == 3 * 2 ** 30
    assert u[:, 2].tolist() == [2 ** 29, 7 * 2 ** 29, 0]
    uo = oracle.quantize(np.array([[10.0, 10.0, 10.0], [10.0 + 600.0, 10.0, 10.0 + 1200 - 1e-9]]),
                         oracle.OPEN, 1200.0, origin=(10.0, 10.0, 10.0))
    assert uo[:, 0].tolist() == [0, 0, 0]
    assert uo[0, 1] == 2 ** 29 and uo[2, 1] == 2 ** 30 - 1
    with pytest.raises(ValueError):
        oracle.quantize(np.array([[9.0, 10.0, 10.0]]), oracle.OPEN, 1200.0, origin=(10.0, 10.0, 10.0))


def test_quantize_grid_points_roundtrip():
    rng = np.random.default_rng(3)
    for geom, L, bits in ((oracle.PERIODIC, 512.0, 32), (oracle.OPEN, 2048.0, 30)):
        u = rng.integers(0, 2 ** bits, size=(3, 1000), dtype=np.uint64).astype(np.uint32)
        x = _snap(u, geom, L)
        assert np.array_equal(oracle.quantize(x, geom, L), u)


def test_thresholds_exact_vs_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 400
    rng = np.random.default_rng(5)
    for geom, L in ((oracle.PERIODIC, 1000.0), (oracle.OPEN, 2400.0), (oracle.PERIODIC, 333.3)):
        edges = np.sort(rng.uniform(0, L / 2.5, 50))
        T = oracle.thresholds(edges, geom, L)
        bits = 32 if geom == oracle.PERIODIC else 30
        for e, t in zip(edges, T):
            v = mpmath.mpf(float(e)) ** 2 * (mpmath.mpf(2) ** bits / mpmath.mpf(float(L))) ** 2
            assert mpmath.mpf(t - 1) < v <= mpmath.mpf(t)
    # a value that is exactly an integer must not be rounded up
    assert oracle.thresholds([1.0, 2.0], oracle.PERIODIC, 1024.0) == [2 ** 44, 2 ** 46]


# ---------------------------------------------------------------------------
# pair counts: hand-worked edges
# ---------------------------------------------------------------------------

def _hist_of_pair(a, b, binning):
    ua = np.array(a, dtype=np.uint32).reshape(3, 1)
    ub = np.array(b, dtype=np.uint32).reshape(3, 1)
    return oracle.count_pairs(ua, ub, binning)


@pytest.mark.parametrize("section", ["periodic", "open_midpoint"])
def test_golden_edge_pairs(section):
    g = json.load(open(os.path.join(GOLDEN, "edge_pairs.json")))[section]
    if section == "periodic":
        b = oracle.Binning(g["s_edges"], g["n_mu"], oracle.PERIODIC, g["L"])
    else:
        b = oracle.Binning(g["s_edges"], g["n_mu"], oracle.OPEN, g["L"], los=oracle.LOS_MIDPOINT,
                           observer=g["observer"])
        assert b.obs_u == [0, 50 * 2 ** 20, 50 * 2 ** 20]
    for p in g["pairs"]:
        for x, y in ((p["a"], p["b"]), (p["b"], p["a"])):  # symmetric in the pair order
            h, unb = _hist_of_pair(x, y, b)
            if p["bin"] < 0:
                assert unb == 1 and h.sum() == 0, p["why"]
            else:
                assert unb == 0 and h[p["bin"]] == 1 and h.sum() == 1, p["why"]
        # the same pair as a two-point auto count
        ua = np.array([p["a"], p["b"]], dtype=np.uint32).T.copy()
        h, unb = oracle.count_pairs(ua, None, b)
        assert h.sum() + unb == 1
        if p["bin"] >= 0:
            assert h[p["bin"]] == 1


# ---------------------------------------------------------------------------
# pair counts vs a library pair counter and float64 re-derivations
# ---------------------------------------------------------------------------

def _far_from_edges(d, edges, rel=1e-9):
    e = np.asarray(edges)[None, :]
    return not np.any(np.abs(d[:, None] - e) <= rel * np.maximum(e, 1e-300))


@pytest.mark.parametrize("clustered", [False, True])
def test_counts_vs_kdtree_periodic(clustered):
    L = 500.0
    rng = synth.rng_for(900, int(clustered), 0)
    n = 700
    if clustered:
        x = synth.neyman_scott(rng, n, L, 2e-6, 6.0)
        y = synth.neyman_scott(rng, n + 13, L, 2e-6, 6.0)
    else:
        x = synth.uniform_box(rng, n, L)
        y = synth.uniform_box(rng, n + 13, L)
    edges = np.linspace(0.0, 120.0, 13)
    b = oracle.Binning(edges, 1, oracle.PERIODIC, L)
    ux, uy = oracle.quantize(x, b.geometry, L), oracle.quantize(y, b.geometry, L)
    xs, ys = _snap(ux, b.geometry, L), _snap(uy, b.geometry, L)
    tx, ty = cKDTree(xs, boxsize=L), cKDTree(ys, boxsize=L)
    # guard: no pair sits within 1e-9 of an edge, so closed/half-open conventions agree
    dxy = tx.sparse_distance_matrix(ty, edges[-1] * 1.01, output_type="ndarray")["v"]
    assert _far_from_edges(dxy, edges[1:])
    # cross count
    cum = tx.count_neighbors(ty, edges[1:] * (1 - 1e-12))  # pairs with d < e (strict)
    expect = np.diff(np.concatenate([[0], cum]))
    h, unb = oracle.count_pairs(ux, uy, b)
    assert np.array_equal(h, expect)
    assert h.sum() + unb == n * (n + 13)
    # auto count: ordered pairs incl. self pairs -> unordered distinct pairs
    cum_auto = tx.count_neighbors(tx, edges[1:] * (1 - 1e-12))
    cum_auto = (cum_auto - n) // 2
    expect_auto = np.diff(np.concatenate([[0], cum_auto]))
    ha, unba = oracle.count_pairs(ux, None, b)
    assert np.array_equal(ha, expect_auto)
    assert ha.sum() + unba == n * (n - 1) // 2


def test_counts_vs_kdtree_open():
    rng = synth.rng_for(901, 0, 0)
    x = synth.shell_octant_uniform(rng, 900, 600.0, 1200.0)
    b = oracle.Binning(np.linspace(0, 150.0, 7), 1, oracle.OPEN, 1200.0)
    ux = oracle.quantize(x, oracle.OPEN, 1200.0)
    xs = _snap(ux, oracle.OPEN, 1200.0)
    t = cKDTree(xs)
    cum = (t.count_neighbors(t, np.asarray(b.s_edges[1:]) * (1 - 1e-12)) - len(xs)) // 2
    h, unb = oracle.count_pairs(ux, None, b)
    assert np.array_equal(h, np.diff(np.concatenate([[0], cum])))


def _float_bins(xa, xb, edges, n_mu, L=None, obs=None):
    """(s, mu) bin of every pair from float64 positions: s by searchsorted, mu = |cos|."""
    d = xa[:, None, :] - xb[None, :, :]
    if L is not None:
        d -= L * np.round(d / L)
    s = np.sqrt((d * d).sum(-1))
    if obs is None:
        mu = np.abs(d[..., 0]) / np.where(s > 0, s, 1)
    else:
        los = 0.5 * (xa[:, None, :] + xb[None, :, :]) - obs
        mu = np.abs((d * los).sum(-1)) / np.where(s > 0, s, 1) / np.linalg.norm(los, axis=-1)
    mu = np.where(s > 0, mu, 0.0)
    k = np.searchsorted(edges, s, side="right") - 1
    j = np.minimum(np.floor(mu * n_mu).astype(int), n_mu - 1)
    return s, mu, k, j


@pytest.mark.parametrize("geom", ["periodic_x", "open_midpoint", "open_x"])
def test_mu_bins_vs_float64(geom):
    n_mu = 7
    edges = np.array([0.0, 10.0, 25.0, 40.0, 60.0])
    if geom == "periodic_x":
        L = 300.0
        rng = synth.rng_for(902, 0, 0)
        xa, xb = synth.neyman_scott(rng, 300, L, 1e-5, 8.0), synth.uniform_box(rng, 280, L)
        b = oracle.Binning(edges, n_mu, oracle.PERIODIC, L)
        obs = None
        Lw = L
    else:
        L = 1000.0
        rng = synth.rng_for(902, 1, 0)
        xa = synth.shell_octant_uniform(rng, 300, 500.0, 560.0)
        xb = synth.shell_octant_uniform(rng, 280, 500.0, 560.0)
        if geom == "open_midpoint":
            b = oracle.Binning(edges, n_mu, oracle.OPEN, L, los=oracle.LOS_MIDPOINT, observer=(0, 0, 0))
            obs = np.zeros(3)
        else:
            b = oracle.Binning(edges, n_mu, oracle.OPEN, L, los=oracle.LOS_X)
            obs = None
        Lw = None
    ua, ub = oracle.quantize(xa, b.geometry, L), oracle.quantize(xb, b.geometry, L)
    xa, xb = _snap(ua, b.geometry, L), _snap(ub, b.geometry, L)
    if geom == "open_x":
        s, mu, k, j = _float_bins(xa, xb, edges, n_mu)
    else:
        s, mu, k, j = _float_bins(xa, xb, edges, n_mu, L=Lw, obs=obs)
    inr = (k >= 0) & (k < len(edges) - 1)
    # guard: nothing within 1e-9 of an s or mu edge
    assert _far_from_edges(s.ravel(), edges[1:])
    mu_in = mu[inr]
    assert not np.any(np.abs(mu_in[:, None] - np.arange(1, n_mu)[None, :] / n_mu) < 1e-9)
    expect = np.bincount((k * n_mu + j)[inr], minlength=b.nbin)
    h, unb = oracle.count_pairs(ua, ub, b)
    assert np.array_equal(h, expect)
    assert unb == (~inr).sum()


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------

def test_symmetry_and_split_sum():
    L = 400.0
    m = synth.SMALL.make_mock(0, n_d=500, M=2)
    b = oracle.Binning(np.linspace(0, 90.0, 10), 4, oracle.PERIODIC, L)
    qd = oracle.quantize(m.data, b.geometry, L)
    q1, q2 = (oracle.quantize(r, b.geometry, L) for r in m.randoms)
    dr, _ = oracle.count_pairs(qd, q1, b)
    rd, _ = oracle.count_pairs(q1, qd, b)
    assert np.array_equal(dr, rd)
    rr1, u1 = oracle.count_pairs(q1, None, b)
    rr2, u2 = oracle.count_pairs(q2, None, b)
    r12, u12 = oracle.count_pairs(q1, q2, b)
    rr_all, u_all = oracle.count_pairs(np.concatenate([q1, q2], axis=1), None, b)
    assert np.array_equal(rr_all, rr1 + rr2 + r12)  # unsplit RR = split RR + cross-subset pairs
    n = q1.shape[1]
    assert rr_all.sum() + u_all == (2 * n) * (2 * n - 1) // 2
    # DR against the union of subsets is additive
    dr2, _ = oracle.count_pairs(qd, q2, b)
    dr_all, _ = oracle.count_pairs(qd, np.concatenate([q1, q2], axis=1), b)
    assert np.array_equal(dr_all, dr + dr2)


def test_empty_catalogues():
    b = oracle.Binning([0.0, 1.0], 1, oracle.PERIODIC, 10.0)
    e = np.zeros((3, 0), np.uint32)
    one = np.zeros((3, 1), np.uint32)
    assert oracle.count_pairs(e, None, b)[0].sum() == 0
    assert oracle.count_pairs(one, None, b)[0].sum() == 0
    assert oracle.count_pairs(one, e, b)[0].sum() == 0
    assert oracle.count_pairs(e, one, b)[0].sum() == 0


def test_binning_rejects_bad_geometry():
    with pytest.raises(ValueError):
        oracle.Binning([0.0, 50.0], 1, oracle.PERIODIC, 100.0)  # s_max = L/2
    with pytest.raises(ValueError):
        oracle.Binning([0.0, 2.0, 1.0], 1, oracle.PERIODIC, 100.0)
    with pytest.raises(ValueError):
        oracle.Binning([0.0, 10.0], 2, oracle.PERIODIC, 100.0, los=oracle.LOS_MIDPOINT)


def test_uniform_counts_match_shell_volumes():
    """E[RR_k] = N(N-1)/2 * V_k / L^3 for uniform points in a periodic box; mu uniform on [0,1]."""
    L, n = 200.0, 3000
    edges = np.linspace(0.0, 40.0, 9)
    n_mu = 4
    b = oracle.Binning(edges, n_mu, oracle.PERIODIC, L)
    u = oracle.quantize(synth.uniform_box(synth.rng_for(903, 0, 0), n, L), b.geometry, L)
    h, _ = oracle.count_pairs(u, None, b)
    vk = 4.0 / 3.0 * math.pi * (edges[1:] ** 3 - edges[:-1] ** 3) / L ** 3
    expect = np.repeat(n * (n - 1) / 2 * vk / n_mu, n_mu)
    z = (h - expect) / np.sqrt(expect)
    assert np.all(np.abs(z) < 5.0)
    chi2 = float((z ** 2).sum())
    assert chi2 < b.nbin + 6 * math.sqrt(2 * b.nbin)


# ---------------------------------------------------------------------------
# Landy-Szalay estimator
# ---------------------------------------------------------------------------

def test_ls_hand_values():
    g = json.load(open(os.path.join(GOLDEN, "ls_hand.json")))
    for c in g["cases"]:
        xi = oracle.ls(c["DD"], c["DR"], c["RR"], c["n_d"], c["n_r"], c["sel"])
        exp = np.array([np.nan if v is None else v for v in c["xi"]])
        assert np.allclose(xi, exp, rtol=1e-15, atol=1e-15, equal_nan=True), c["why"]


def test_ls_uniform_data_mean_zero():
    """Uniform 'data' has xi = 0 (Sect. 4.2): the mean estimate over mocks is consistent with zero."""
    L, n = 300.0, 600
    edges = np.array([0.0, 20.0, 40.0, 60.0])
    b = oracle.Binning(edges, 1, oracle.PERIODIC, L)
    xis = []
    for m in range(40):
        d = oracle.quantize(synth.uniform_box(synth.rng_for(904, m, 0), n, L), b.geometry, L)
        r = oracle.quantize(synth.uniform_box(synth.rng_for(904, m, 1), n, L), b.geometry, L)
        c = oracle.count_mock_u32(d, [r], b)
        xis.append(oracle.ls(c["DD"], c["DR"], c["RR"], n, [n], [0]))
    xis = np.array(xis)
    z = xis.mean(0) / (xis.std(0, ddof=1) / math.sqrt(len(xis)))
    assert np.all(np.abs(z) < 4.5)


def test_ls_neyman_scott_closed_form():
    """Pair counts + LS recover the closed-form xi of the Neyman-Scott generator."""
    L, n, n_p, sigma = 400.0, 3000, 4e-6, 4.0
    edges = np.array([0.0, 3.0, 6.0, 9.0, 12.0, 16.0])
    b = oracle.Binning(edges, 1, oracle.PERIODIC, L)
    est = []
    for m in range(4):
        rng = synth.rng_for(905, m, 0)
        n_par = max(1, int(rng.poisson(n_p * L ** 3)))  # what neyman_scott draws first
        d = synth.neyman_scott(synth.rng_for(905, m, 0), n, L, n_p, sigma)
        r1 = synth.uniform_box(synth.rng_for(905, m, 1), n, L)
        r2 = synth.uniform_box(synth.rng_for(905, m, 2), n, L)
        c = oracle.count_mock(d, [r1, r2], b)
        xi = oracle.ls(c["DD"], c["DR"], c["RR"], n, [n, n], [0, 1])
        # exact pair-separation density for a fixed parent count: xi = (V/N_p) g(r) - 1/N_p
        rs = np.linspace(edges[0], edges[-1], 20001)
        g = np.exp(-rs ** 2 / (4 * sigma ** 2)) / (4 * math.pi * sigma ** 2) ** 1.5
        V = L ** 3
        xi_r = V / n_par * g - 1.0 / n_par
        w = rs ** 2
        theory = []
        for k in range(len(edges) - 1):
            sel = (rs >= edges[k]) & (rs < edges[k + 1])
            theory.append(np.trapezoid(xi_r[sel] * w[sel], rs[sel]) / np.trapezoid(w[sel], rs[sel]))
        est.append(xi / np.array(theory))
    ratio = np.mean(est, axis=0)
    assert np.all(np.abs(ratio[:3] - 1.0) < 0.15), ratio


# ---------------------------------------------------------------------------
# covariances
# ---------------------------------------------------------------------------

def test_sample_cov_matches_numpy():
    rng = np.random.default_rng(7)
    x = rng.normal(size=(57, 23)) @ rng.normal(size=(23, 23))
    assert np.allclose(oracle.sample_cov(x), np.cov(x, rowvar=False, ddof=1), rtol=1e-13, atol=1e-14)
    # ill-conditioned: large common offset, small spread (two-pass centring)
    y = 1e6 + 1e-3 * rng.normal(size=(200, 9))
    c = oracle.sample_cov(y)
    ref = np.cov(y - y.mean(0), rowvar=False, ddof=1)
    assert np.allclose(c, ref, rtol=1e-9, atol=1e-18)
    with pytest.raises(ValueError):
        oracle.sample_cov(y[:1])


def test_lc_identities():
    rng = np.random.default_rng(8)
    xa1, xa2, xb = synth.synthetic_xi_variants(77, 300, 12)
    for M_a in (1, 3):
        r = oracle.lc_cov(xa1, xa2, xb, M_a, 2 * M_a)
        assert np.allclose(r["C_lc"], r["Cb"], rtol=1e-12, atol=1e-18)        # M = 2 M_a -> C^b
        r1 = oracle.lc_cov(xa1, xa2, xb, M_a, M_a)
        assert np.allclose(r1["C_lc"], r1["Ca"], rtol=1e-12, atol=1e-18)      # M = M_a -> C^a
        rinf = oracle.lc_cov(xa1, xa2, xb, M_a, math.inf)
        assert np.array_equal(rinf["C_lc"], rinf["A"])                         # M -> inf -> A
        # linear in 1/M
        c10, c20, c40 = (oracle.lc_cov(xa1, xa2, xb, M_a, M)["C_lc"] for M in (10, 20, 40))
        assert np.allclose(c20 - c40, (c10 - c20) / 2, rtol=1e-9, atol=1e-16)
        # Eq. (CovAB) with (M_a, M_b = 2 M_a) gives the same A and B
        A, B = oracle.cov_ab(r["Ca"], r["Cb"], M_a, 2 * M_a)
        assert np.allclose(A, r["A"], rtol=1e-12, atol=1e-18)
        assert np.allclose(B, r["B"], rtol=1e-12, atol=1e-18)
    # C^a is the mean of the two single-catalogue sample covariances
    r = oracle.lc_cov(xa1, xa2, xb, 1, 50)
    assert np.allclose(r["Ca"], 0.5 * (np.cov(xa1, rowvar=False) + np.cov(xa2, rowvar=False)), rtol=1e-12)
    assert np.allclose(r["Cb"], np.cov(xb, rowvar=False), rtol=1e-12)
    del rng


@pytest.mark.slow
def test_lc_matches_poisson_theory():
    """Uniform data: diagonal covariance of Eq. (randomtheory), 2/(N_d(N_d-1)) (1 + 3/M) / G_p at large N.

    C^a (M=1), C^b (M=2) and the LC extrapolation to M = inf are compared with
    the analytic values, averaged over bins, at 4.5 sigma of the sampling error.
    """
    # bins hold ~1e3 pairs, so the linearisation behind the formula (large RR counts) holds
    L, n, n_mock = 300.0, 1500, 400
    edges = np.array([10.0, 20.0, 30.0, 40.0, 50.0])
    b = oracle.Binning(edges, 1, oracle.PERIODIC, L)
    xa1, xa2, xb = [], [], []
    for m in range(n_mock):
        d = oracle.quantize(synth.uniform_box(synth.rng_for(906, m, 0), n, L), b.geometry, L)
        r1 = oracle.quantize(synth.uniform_box(synth.rng_for(906, m, 1), n, L), b.geometry, L)
        r2 = oracle.quantize(synth.uniform_box(synth.rng_for(906, m, 2), n, L), b.geometry, L)
        c = oracle.count_mock_u32(d, [r1, r2], b)
        xa1.append(oracle.ls(c["DD"], c["DR"], c["RR"], n, [n, n], [0]))
        xa2.append(oracle.ls(c["DD"], c["DR"], c["RR"], n, [n, n], [1]))
        xb.append(oracle.ls(c["DD"], c["DR"], c["RR"], n, [n, n], [0, 1]))
    Gp = 4.0 / 3.0 * math.pi * (edges[1:] ** 3 - edges[:-1] ** 3) / L ** 3

    def theory(M):
        nr = M * n
        return (2.0 / (n * (n - 1)) + 4.0 / (n * nr) + 2.0 / (nr * (n - 1))) / Gp

    lc = oracle.lc_cov(np.array(xa1), np.array(xa2), np.array(xb), 1, math.inf)
    for mat, M, tol in ((lc["Ca"], 1, 0.16), (lc["Cb"], 2, 0.16), (lc["A"], math.inf, 0.35)):
        ratio = np.diag(mat) / (theory(M) if M != math.inf else 2.0 / (n * (n - 1)) / Gp)
        assert abs(ratio.mean() - 1.0) < tol, (M, ratio)


# ---------------------------------------------------------------------------
# linear maps: wider bins and Legendre multipoles (Sect. 2.3, Sect. 4.3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("f_s,f_mu", [(1, 1), (2, 3), (3, 6), (4, 1), (1, 2), (12, 6)])
def test_rebin_counts_equals_counting_with_merged_edges(f_s, f_mu):
    """Combining f_s consecutive half-open s bins and f_mu uniform |mu| bins must give exactly the counts
    of a direct brute-force count with the merged edges (the bins partition the same integer ranges)."""
    rng = np.random.default_rng(12)
    L = 200.0
    x = rng.random((700, 3)) * L
    y = rng.random((500, 3)) * L
    n_s, n_mu = 12, 6
    fine = np.linspace(0.0, 48.0, n_s + 1)
    bf = oracle.Binning(fine, n_mu, oracle.PERIODIC, L)
    bc = oracle.Binning(fine[::f_s], n_mu // f_mu, oracle.PERIODIC, L)
    qx, qy = oracle.quantize(x, oracle.PERIODIC, L), oracle.quantize(y, oracle.PERIODIC, L)
    for ub in (None, qy):
        h_f = oracle.count_pairs(qx, ub, bf)[0]
        h_c = oracle.count_pairs(qx, ub, bc)[0]
        assert h_c.sum() > 0
        assert np.array_equal(oracle.rebin_counts(h_f, n_s, n_mu, f_s, f_mu), h_c)
    stacked = np.stack([h_f, 2 * h_f])
    assert np.array_equal(oracle.rebin_counts(stacked, n_s, n_mu, f_s, f_mu)[1], 2 * h_c)


def test_multipole_matrix_closed_forms():
    """Entries against the explicit polynomials P_2 = (3mu^2 - 1)/2, P_4 = (35mu^4 - 30mu^2 + 3)/8:
    for |mu| bins, (2l+1)/2 int_{-1}^{1} doubles the [0, 1] integral."""
    n_mu = 4
    P = oracle.multipole_matrix(1, n_mu, (0, 2, 4))
    a2 = lambda m: (m ** 3 - m) / 2.0                         # int_0^m P_2
    a4 = lambda m: (7 * m ** 5 - 10 * m ** 3 + 3 * m) / 8.0    # int_0^m P_4
    e = np.arange(n_mu + 1) / n_mu
    for j in range(n_mu):
        assert P[0, j] == pytest.approx(e[j + 1] - e[j], abs=1e-15)
        assert P[1, j] == pytest.approx(5.0 * (a2(e[j + 1]) - a2(e[j])), abs=1e-14)
        assert P[2, j] == pytest.approx(9.0 * (a4(e[j + 1]) - a4(e[j])), abs=1e-14)
    assert P[1, 0] == pytest.approx(-0.5859375, abs=1e-15)    # 5 (1/64 - 1/4) / 2


def test_multipole_matrix_invariants():
    """A constant xi has only a monopole; odd multipoles of an |mu|-binned xi vanish; a xi made of the
    bin averages of A_0 + A_2 P_2 + A_4 P_4 gives back (A_0, A_2, A_4) as the bins shrink."""
    n_s, n_mu = 3, 200
    P = oracle.multipole_matrix(n_s, n_mu, (0, 1, 2, 3, 4))
    const = np.full(n_s * n_mu, 2.5)
    m = P @ const
    assert np.allclose(m[:n_s], 2.5, atol=1e-14) and np.allclose(m[n_s:], 0.0, atol=1e-13)
    from numpy.polynomial import legendre as npl
    A = {0: [1.0, -0.3, 4.0], 2: [0.5, 2.0, -1.0], 4: [-0.25, 0.1, 3.0]}
    e = np.arange(n_mu + 1) / n_mu
    xi = np.zeros(n_s * n_mu)
    for ell, amps in A.items():
        anti = npl.Legendre.basis(ell).integ()
        avg = (anti(e[1:]) - anti(e[:-1])) * n_mu               # bin average of P_l on [mu_j, mu_j+1]
        for k in range(n_s):
            xi[k * n_mu:(k + 1) * n_mu] += amps[k] * avg
    m = P @ xi
    for i, ell in enumerate((0, 1, 2, 3, 4)):
        want = np.array(A.get(ell, [0.0] * n_s))
        assert np.allclose(m[i * n_s:(i + 1) * n_s], want, rtol=5e-4, atol=1e-4), ell   # O(dmu^2) error


def test_project_hand_worked():
    """A non-square map worked by hand: y[m] = P xi[m] for P of 2 x 3 and two mocks (a transposed
    or row-swapped product gives other numbers or the wrong shape)."""
    P = np.array([[1.0, 2.0, 0.0],
                  [0.0, -1.0, 3.0]])
    xi = np.array([[1.0, 10.0, 100.0],
                   [-2.0, 0.5, 4.0]])
    y = oracle.project(P, xi)
    assert y.shape == (2, 2)
    # mock 0: (1 + 20 + 0, 0 - 10 + 300); mock 1: (-2 + 1 + 0, 0 - 0.5 + 12)
    assert np.array_equal(y, np.array([[21.0, 290.0], [-1.0, 11.5]]))


def test_project_recovers_multipole_amplitudes_per_mock():
    """Mocks whose xi rows are bin averages of sum_l A_l^(m)(s) P_l(|mu|) with their own amplitudes:
    project(multipole_matrix, xi) returns every mock's (A_0, A_2, A_4) in the (ell, s) row order."""
    from numpy.polynomial import legendre as npl
    n_s, n_mu, ells = 2, 400, (0, 2, 4)
    P = oracle.multipole_matrix(n_s, n_mu, ells)
    e = np.arange(n_mu + 1) / n_mu
    rng = np.random.default_rng(7)
    amps = rng.normal(size=(3, len(ells), n_s))               # [mock][ell][s]
    xi = np.zeros((3, n_s * n_mu))
    for m in range(3):
        for i, ell in enumerate(ells):
            anti = npl.Legendre.basis(ell).integ()
            avg = (anti(e[1:]) - anti(e[:-1])) * n_mu
            for k in range(n_s):
                xi[m, k * n_mu:(k + 1) * n_mu] += amps[m, i, k] * avg
    y = oracle.project(P, xi)
    assert y.shape == (3, len(ells) * n_s)
    assert np.allclose(y, amps.reshape(3, -1), rtol=1e-4, atol=1e-4)   # O(dmu^2) bin-average error


# ---------------------------------------------------------------------------
# covariance of covariance and chi^2 (Sect. 3, Sect. 5.3), pinned by Monte Carlo
# ---------------------------------------------------------------------------

def _mc_lc(M_a, M, N, T, seed):
    """Simulate the LC construction for Gaussian xi: x and x' (the estimates with the two M_a random
    catalogues) share the data part s (covariance S) and carry independent random-catalogue parts
    (covariance R); xi of the joint catalogue is (x + x') / 2, as in the derivation of Eq. (Cfastx)."""
    rng = np.random.default_rng(seed)
    S = np.array([[2.0, 0.5, 0.2], [0.5, 1.5, 0.3], [0.2, 0.3, 1.0]])
    R = np.array([[1.0, 0.4, 0.0], [0.4, 2.0, 0.5], [0.0, 0.5, 0.8]])
    Ls, Lr = np.linalg.cholesky(S), np.linalg.cholesky(R)
    est_lc, est_smp = [], []
    for _ in range(T):
        s = rng.standard_normal((N, 3)) @ Ls.T
        x = s + rng.standard_normal((N, 3)) @ Lr.T
        xp = s + rng.standard_normal((N, 3)) @ Lr.T
        Ca = 0.5 * oracle.sample_cov(x) + 0.5 * oracle.sample_cov(xp)
        Cb = oracle.sample_cov(0.5 * (x + xp))
        A = 2 * Cb - Ca
        B = 2 * M_a * (Ca - Cb)
        est_lc.append(A + B / M)
        est_smp.append(oracle.sample_cov(x))
    # ensemble values: cov(x) = S + R = A + B / M_a, cov(x, x') = S = A
    return np.array(est_lc), np.array(est_smp), S, M_a * R


@pytest.mark.parametrize("M_a,M", [(1, 5.0), (1, 50.0), (2, 3.0), (1, 2.0)])
def test_covcov_lc_and_smp_against_monte_carlo(M_a, M):
    """Var(C_ij) of Eqs. (covcov_brute) and (covcov_fast) against the scatter of simulated estimates:
    the reading D = A + B / (2 M_a) matches, the printed A + B / M_a would be off by up to 2x."""
    N, T = 8, 12000
    lc, smp, A, B = _mc_lc(M_a, M, N, T, seed=int(10 * M) + M_a)
    v_lc = oracle.covcov_var(A, B, N, M_a, M)
    v_smp = oracle.covcov_var(A + B / M_a, None, N)
    # relative standard error of a variance from T samples ~ sqrt(2 / T) (1.3 %), plus heavier tails
    assert np.allclose(lc.var(axis=0, ddof=1), v_lc, rtol=0.07), (lc.var(axis=0, ddof=1), v_lc)
    assert np.allclose(smp.var(axis=0, ddof=1), v_smp, rtol=0.07)
    if M != 2.0 * M_a:
        wrong = oracle.covcov_var(A - B / (2.0 * M_a) + B / M_a, B, N, M_a, M)   # D = A + B / M_a
        assert np.max(np.abs(lc.var(axis=0, ddof=1) / wrong - 1.0)) > 0.2
    # chi^2: the mean measured chi^2_N times (N - 1) is the predicted chi^2_2
    C_true = A + B / M
    m = np.mean([oracle.chi2(c, C_true, C_true) for c in lc]) * (N - 1)
    assert m == pytest.approx(oracle.chi2_predict(A, B, C_true, M_a, M), rel=0.05)


def test_covcov_special_cases():
    """LC at M = 2 M_a equals the sample-covariance form of C(2 M_a); identity covariance gives
    <chi^2_2> = 1 + 1/n for the sample covariance."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((6, 6))
    A = X @ X.T
    Y = rng.standard_normal((6, 6))
    B = Y @ Y.T
    for M_a in (1, 3):
        lc = oracle.covcov_var(A, B, 11, M_a, 2.0 * M_a)
        smp = oracle.covcov_var(A + B / (2.0 * M_a), None, 11)
        assert np.allclose(lc, smp, rtol=1e-13)
    for n in (1, 4, 40):
        eye = np.eye(n)
        assert oracle.chi2_predict(eye, None, eye) == pytest.approx(1.0 + 1.0 / n, rel=1e-14)
    assert oracle.chi2(A, A, A) == 0.0


def test_eigvalsh_known_spectrum():
    rng = np.random.default_rng(6)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    lam = np.sort(np.concatenate([rng.uniform(-2, 5, 27), [1.5, 1.5, 1.5]]))
    C = (Q * lam) @ Q.T
    assert np.allclose(oracle.eigvalsh(0.5 * (C + C.T)), lam, atol=1e-12)
