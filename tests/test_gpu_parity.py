"""GPU parity: the CUDA library against the CPU oracle, through the C ABI.

Counts must match bit for bit; float64 estimator steps within 1e-12
(|x - x_oracle| / (1 + |x_oracle|) for xi; |C - C_oracle| / sqrt(C^a_ii C^a_jj)
for covariance elements).  Inputs are seeded synthetic catalogues shaped like
the measurement workloads: Neyman-Scott data with uniform randoms in periodic
boxes, and a cut-sky octant shell with a midpoint line of sight.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


DEV = "cuda:0"


def _mocks_to_device(mocks):
    out = []
    for mk in mocks:
        n_r = [len(r) for r in mk.randoms]
        offs = [0] + list(np.cumsum(n_r))
        out.append({"data": torch.from_numpy(np.ascontiguousarray(mk.data)).to(DEV),
                    "randoms": torch.from_numpy(np.ascontiguousarray(np.concatenate(mk.randoms)
                                                                     if mk.randoms else np.zeros((0, 3)))).to(DEV),
                    "offsets": offs})
    return out


def _check_counts(ctx, tp, mocks, tb, ob, modes=(0, 1), terms=7, kernels=(1, 2), want_direct=None):
    """Counts of both pair counters (TPCF_KERNEL_DIRECT, which takes the direct counter where the
    binning suits it, and TPCF_KERNEL_GENERAL) in every mode, bit for bit against the oracle."""
    dm = _mocks_to_device(mocks)
    refs = [oracle.count_mock(mk.data, mk.randoms, ob) for mk in mocks]
    out = None
    for kern in kernels:
        ctx.tpcf_set_option(tp.TPCF_OPT_KERNEL, kern)
        try:
            out = _check_counts_once(ctx, tp, refs, dm, modes, terms, tb)
            info = ctx.tpcf_last_count_info()
            if kern == tp.TPCF_KERNEL_GENERAL:
                assert info["pair_kernel"] == tp.TPCF_KERNEL_GENERAL
            elif want_direct is not None:
                assert info["pair_kernel"] == (tp.TPCF_KERNEL_DIRECT if want_direct else tp.TPCF_KERNEL_GENERAL)
        finally:
            ctx.tpcf_set_option(tp.TPCF_OPT_KERNEL, tp.TPCF_KERNEL_AUTO)
    return out


def _check_counts_once(ctx, tp, refs, dm, modes, terms, tb):
    for mode in modes:
        out = ctx.tpcf_count(dm, tb, terms=terms, mode=mode)
        assert ctx.tpcf_sync() == tp.TPCF_OK
        info = ctx.tpcf_last_count_info()
        tot = 0
        for m, ref in enumerate(refs):
            if terms & 1:
                assert np.array_equal(out["dd"][m].cpu().numpy(), ref["DD"]), (mode, m, "DD")
                tot += ref["DD"].sum()
            if terms & 2:
                assert np.array_equal(out["dr"][m].cpu().numpy(), ref["DR"]), (mode, m, "DR")
                tot += ref["DR"].sum()
            if terms & 4:
                assert np.array_equal(out["rr"][m].cpu().numpy(), ref["RR"]), (mode, m, "RR")
                tot += ref["RR"].sum()
        assert info["n_binned"] == tot
        assert info["n_candidates"] >= tot
    return out


def _periodic(L, edges, n_mu):
    import paper_2205_11852_gb300 as tp
    return tp.make_binning(edges, n_mu, tp.TPCF_PERIODIC, L), oracle.Binning(edges, n_mu, oracle.PERIODIC, L)


# ---------------------------------------------------------------------------
# counts
# ---------------------------------------------------------------------------

def test_counts_periodic_s_only(tp, ctx):
    """Small-workload shape: Neyman-Scott data, 2 random subsets, 20 linear s bins to s_max = L/5."""
    L = 500.0
    mocks = [synth.SMALL.make_mock(m, n_d=2500, M=2) for m in range(3)]
    tb, ob = _periodic(L, np.linspace(0, 100.0, 21), 1)
    _check_counts(ctx, tp, mocks, tb, ob, want_direct=True)


def test_counts_periodic_s_mu(tp, ctx):
    """Mid-workload shape scaled down: 40 s x 10 mu bins, plane-parallel line of sight."""
    L = 400.0
    w = synth.Workload("t", 31, 2, "periodic", L, (0, 0, 0), 3000, 2, 80.0, 40, 10, "x", n_parent=4e-5, sigma=3.0)
    mocks = [w.make_mock(m) for m in range(2)]
    tb, ob = _periodic(L, w.s_edges, 10)
    _check_counts(ctx, tp, mocks, tb, ob, want_direct=True)


@pytest.mark.parametrize("subdiv", [1, 2, 3, 4])
def test_counts_any_mesh_subdivision(tp, ctx, subdiv):
    L = 300.0
    w = synth.Workload("t", 32, 1, "periodic", L, (0, 0, 0), 1800, 2, 60.0, 12, 5, "x", n_parent=5e-5, sigma=2.0)
    mocks = [w.make_mock(0)]
    tb, ob = _periodic(L, w.s_edges, 5)
    ctx.tpcf_set_cell_subdiv(subdiv)
    try:
        _check_counts(ctx, tp, mocks, tb, ob, modes=(0,))
    finally:
        ctx.tpcf_set_cell_subdiv(0)


def test_counts_neighbourhood_beyond_one_filter_window(tp, ctx):
    """Dense periodic box: about 44 points per mesh cell at subdivision 3, so the neighbour runs of a cell hold
    ~13 700 raw points, more than one filter window (12 288), and every unit's b side is filtered and tiled in two
    windows.  D x R counts must still equal the brute-force oracle bit for bit."""
    L = 150.0
    rng = np.random.default_rng(20261203)
    n = 150_000
    d = synth.neyman_scott(rng, n, L, 2e-3, 1.0)
    r = synth.uniform_box(np.random.default_rng(7), n, L)
    mocks = [synth.Mock(d, [r])]
    tb, ob = _periodic(L, np.linspace(0, 30.0, 16), 4)
    ctx.tpcf_set_cell_subdiv(3)
    try:
        _check_counts(ctx, tp, mocks, tb, ob, modes=(0,), terms=2)
    finally:
        ctx.tpcf_set_cell_subdiv(0)


@pytest.mark.parametrize("los", ["s", "x", "midpoint"])
def test_counts_dense_self_cells(tp, ctx, los):
    """Clumps of 300, 129, 65 and 63 points in cubes of 1 Mpc/h over a sparse background: self cells with more
    points than a b-tile (128) and than an a-chunk (64), odd chunk lengths, and tiles that mix a cell's own
    points with its neighbours'.  Auto and cross counts, both counters, two mesh subdivisions, bit for bit."""
    L = 200.0
    rng = synth.rng_for(38, 0, 0)
    centres = rng.random((4, 3)) * (L - 20.0) + 10.0
    clumps = [c + rng.random((n, 3)) for c, n in zip(centres, (300, 129, 65, 63))]
    d = np.concatenate(clumps + [rng.random((700, 3)) * L])
    r = [np.concatenate([clumps[1] + 0.25, rng.random((600, 3)) * L]), rng.random((555, 3)) * L]
    mocks = [synth.Mock(d, r)]
    edges = np.linspace(0, 30.0, 13)
    n_mu = 1 if los == "s" else 4
    if los == "midpoint":
        obs = (-50.0, 20.0, 300.0)
        tb = tp.make_binning(edges, n_mu, tp.TPCF_OPEN, L + 1.0, los=tp.TPCF_LOS_MIDPOINT, observer=obs)
        ob = oracle.Binning(edges, n_mu, oracle.OPEN, L + 1.0, los=oracle.LOS_MIDPOINT, observer=obs)
    else:
        tb, ob = _periodic(L, edges, n_mu)
    for sd in (2, 3):
        ctx.tpcf_set_cell_subdiv(sd)
        try:
            _check_counts(ctx, tp, mocks, tb, ob, want_direct=True)
        finally:
            ctx.tpcf_set_cell_subdiv(0)


def test_counts_open_midpoint(tp, ctx):
    """Cut-sky octant shell, observer at the origin, midpoint line of sight (batching shape, scaled)."""
    L = 600.0
    w = synth.Workload("t", 33, 2, "open", L, (0, 0, 0), 2500, 2, 50.0, 20, 5, "midpoint",
                       n_parent=2e-5, sigma=3.0, shell=(300.0, 600.0))
    mocks = [w.make_mock(m) for m in range(2)]
    edges = np.linspace(0, 50.0, 21)
    tb = tp.make_binning(edges, 5, tp.TPCF_OPEN, L, los=tp.TPCF_LOS_MIDPOINT, observer=(0, 0, 0))
    ob = oracle.Binning(edges, 5, oracle.OPEN, L, los=oracle.LOS_MIDPOINT, observer=(0, 0, 0))
    _check_counts(ctx, tp, mocks, tb, ob, want_direct=True)


def test_counts_open_midpoint_observer_inside(tp, ctx):
    """Midpoint line of sight with the observer inside the catalogues: pairs whose midpoint lies at (or next
    to) the observer, where the line of sight vanishes (mu = 0 by definition) or is set by a few grid units,
    plus duplicated points (d = 0) and a pair placed symmetrically about the observer."""
    L = 200.0
    rng = synth.rng_for(37, 0, 0)
    obs = np.array([100.0, 100.0, 100.0])
    d = rng.random((1500, 3)) * L
    # pairs placed symmetrically about the observer (l vanishes up to the grid rounding), and a duplicate
    d[:4] = [obs + [3.0, 1.0, -2.0], obs - [3.0, 1.0, -2.0], obs + [0.5, 0.0, 0.0], obs - [0.5, 0.0, 0.0]]
    d[4] = d[5]
    r = [rng.random((1500, 3)) * L for _ in range(2)]
    mocks = [synth.Mock(d, r)]
    edges = np.linspace(0, 30.0, 13)
    tb = tp.make_binning(edges, 4, tp.TPCF_OPEN, L, los=tp.TPCF_LOS_MIDPOINT, observer=tuple(obs))
    ob = oracle.Binning(edges, 4, oracle.OPEN, L, los=oracle.LOS_MIDPOINT, observer=tuple(obs))
    _check_counts(ctx, tp, mocks, tb, ob, want_direct=True)


def test_counts_open_plane_parallel_slab(tp, ctx):
    """Open slab geometry with the x line of sight (the paper's slab setup, Sect. 4.1, scaled)."""
    L = 300.0
    rng = synth.rng_for(34, 0, 0)
    d = rng.random((2000, 3)) * np.array([L, L, L / 5])
    r = [rng.random((2000, 3)) * np.array([L, L, L / 5]) for _ in range(2)]
    mocks = [synth.Mock(d, r)]
    edges = np.linspace(0, 40.0, 17)
    tb = tp.make_binning(edges, 8, tp.TPCF_OPEN, L, los=tp.TPCF_LOS_X)
    ob = oracle.Binning(edges, 8, oracle.OPEN, L, los=oracle.LOS_X)
    _check_counts(ctx, tp, mocks, tb, ob)


@pytest.mark.parametrize("los", ["x", "midpoint"])
def test_counts_paper_binning_200x100(tp, ctx, los):
    """The paper's own binning (Sect. 4.3: bins of 1 Mpc/h on [0, 200], 100 mu bins, 20 000 bins, a block
    histogram of 80 KB) in the paper's slab (1500 x 1500 x 300, Sect. 4.1) with 5000 points per catalogue, x
    line of sight as in the paper; with the midpoint line of sight the binning is beyond the exact mu test's
    128-bit range and must be refused."""
    dims = np.array([1500.0, 1500.0, 300.0])
    d = synth.uniform_slab(synth.rng_for(35, 0, 0), 5000, dims)
    r = [synth.uniform_slab(synth.rng_for(35, 0, 1 + i), 5000, dims) for i in range(2)]
    edges = np.linspace(0.0, 200.0, 201)
    if los == "midpoint":
        # n_mu^2 D2 |l|^2 passes 2^128 in a 1500 Mpc/h cube at 2^30 grid units: the exact mu test cannot be
        # formed, and the library refuses the binning as the oracle does
        with pytest.raises(ValueError):
            oracle.Binning(edges, 100, oracle.OPEN, 1500.0, los=oracle.LOS_MIDPOINT, observer=(0, 0, 0))
        tb = tp.make_binning(edges, 100, tp.TPCF_OPEN, 1500.0, los=tp.TPCF_LOS_MIDPOINT, observer=(0, 0, 0))
        with pytest.raises(tp.TpcfError) as e:
            ctx.tpcf_count(_mocks_to_device([synth.Mock(d, r)]), tb)
        assert e.value.code == tp.TPCF_ERR_RANGE
        return
    tb = tp.make_binning(edges, 100, tp.TPCF_OPEN, 1500.0, los=tp.TPCF_LOS_X)
    ob = oracle.Binning(edges, 100, oracle.OPEN, 1500.0, los=oracle.LOS_X)
    out = _check_counts(ctx, tp, [synth.Mock(d, r)], tb, ob)
    assert out["dd"].shape[-1] == 20000 and int(out["dd"].sum()) > 100000


def test_binning_beyond_shared_memory_refused(tp, ctx):
    """256 s x 256 mu bins: a 256 KB block histogram cannot sit in shared memory, so the count is refused
    with TPCF_ERR_RANGE (nothing is enqueued) and the context stays usable."""
    d = synth.uniform_slab(synth.rng_for(36, 0, 0), 500, (1500.0, 1500.0, 300.0))
    mk = _mocks_to_device([synth.Mock(d, [d[:250], d[250:]])])
    tb = tp.make_binning(np.linspace(0.0, 200.0, 257), 256, tp.TPCF_OPEN, 1500.0, los=tp.TPCF_LOS_X)
    with pytest.raises(tp.TpcfError) as e:
        ctx.tpcf_count(mk, tb)
    assert e.value.code == tp.TPCF_ERR_RANGE
    ok = tp.make_binning(np.linspace(0.0, 200.0, 21), 4, tp.TPCF_OPEN, 1500.0, los=tp.TPCF_LOS_X)
    ctx.tpcf_count(mk, ok)
    assert ctx.tpcf_sync() == tp.TPCF_OK


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_counts_golden_edge_pairs(tp, ctx, kernel):
    """Hand-worked pairs at exact bin edges, through the default (autotuned) choice, the direct counter
    (for the periodic section's linear bins) and the general one."""
    ctx.tpcf_set_option(tp.TPCF_OPT_KERNEL, kernel)
    try:
        _golden_edge_pairs(tp, ctx)
    finally:
        ctx.tpcf_set_option(tp.TPCF_OPT_KERNEL, tp.TPCF_KERNEL_AUTO)


def _golden_edge_pairs(tp, ctx):
    g = json.load(open(os.path.join(GOLDEN, "edge_pairs.json")))
    for section in ("periodic", "open_midpoint"):
        s = g[section]
        if section == "periodic":
            tb = tp.make_binning(s["s_edges"], s["n_mu"], tp.TPCF_PERIODIC, s["L"])
        else:
            tb = tp.make_binning(s["s_edges"], s["n_mu"], tp.TPCF_OPEN, s["L"], los=tp.TPCF_LOS_MIDPOINT,
                                 observer=s["observer"])
        nbin = len(s["s_edges"]) - 1
        nbin *= s["n_mu"]
        for p in s["pairs"]:
            a = torch.tensor(np.array(p["a"], dtype=np.uint32).reshape(3, 1).view(np.int32), device=DEV)
            b = torch.tensor(np.array(p["b"], dtype=np.uint32).reshape(3, 1).view(np.int32), device=DEV)
            ab = torch.tensor(np.array([p["a"], p["b"]], dtype=np.uint32).T.copy().view(np.int32), device=DEV)
            # cross: D = {a}, R_1 = {b};  auto: RR of R_2 = {a, b}
            rr = torch.cat([b, ab], dim=1).contiguous()
            mk = {"data_u32": a.contiguous(), "randoms_u32": rr, "offsets": [0, 1, 3]}
            out = ctx.tpcf_count([mk], tb)
            assert ctx.tpcf_sync() == tp.TPCF_OK
            exp = np.zeros(nbin, np.int64)
            if p["bin"] >= 0:
                exp[p["bin"]] = 1
            assert np.array_equal(out["dr"][0, 0].cpu().numpy(), exp), p["why"]
            assert np.array_equal(out["rr"][0, 1].cpu().numpy(), exp), p["why"]
            assert out["dd"][0].sum().item() == 0 and out["rr"][0, 0].sum().item() == 0


def test_counts_duplicates_tiny_and_empty(tp, ctx):
    L = 200.0
    rng = np.random.default_rng(1)
    base = rng.random((40, 3)) * L
    dup = np.repeat(base, 7, axis=0)                       # 7 coincident copies of each point
    tiny = base[:1]
    empty = np.zeros((0, 3))
    tb, ob = _periodic(L, np.array([0.0, 0.5, 10.0, 30.0, 60.0]), 3)
    cases = [synth.Mock(dup, [dup[:100], base]), synth.Mock(tiny, [tiny, empty]), synth.Mock(empty, [base, tiny]),
             synth.Mock(base, [empty, empty])]
    _check_counts(ctx, tp, cases, tb, ob)


def test_counts_duplicates_linear_bins(tp, ctx):
    """Coincident and near-coincident points (s = 0 and s of a few grid units, where the direct counter's
    mu interval is widened past one bin) with linear bins and mu bins: both counters against the oracle."""
    L = 200.0
    rng = np.random.default_rng(11)
    base = rng.random((60, 3)) * L
    near = base + rng.normal(size=base.shape) * 1e-7 * L    # a few hundred grid units apart
    dup = np.concatenate([np.repeat(base, 5, axis=0), np.mod(near, L)])
    tb, ob = _periodic(L, np.linspace(0.0, 40.0, 9), 6)
    cases = [synth.Mock(dup, [dup[:150], np.mod(near, L)]), synth.Mock(base, [np.repeat(base[:10], 3, axis=0), base])]
    _check_counts(ctx, tp, cases, tb, ob, want_direct=True)


def test_u32_input_matches_float_input(tp, ctx):
    L = 400.0
    mk = synth.SMALL.make_mock(5, n_d=1500, M=2)
    tb, ob = _periodic(L, np.linspace(0, 100.0, 11), 4)
    f = ctx.tpcf_count(_mocks_to_device([mk]), tb)
    ctx.tpcf_sync()
    qd = oracle.quantize(mk.data, oracle.PERIODIC, L)
    qr = np.concatenate([oracle.quantize(r, oracle.PERIODIC, L) for r in mk.randoms], axis=1)
    m = {"data_u32": torch.from_numpy(qd.view(np.int32).copy()).to(DEV),
         "randoms_u32": torch.from_numpy(qr.view(np.int32).copy()).to(DEV), "offsets": [0, 1500, 3000]}
    u = ctx.tpcf_count([m], tb)
    ctx.tpcf_sync()
    for k in ("dd", "dr", "rr"):
        assert torch.equal(f[k], u[k])


@pytest.mark.parametrize("mode", [0, 1])
def test_counts_from_host_arrays(tp, ctx, mode):
    """Host catalogues (TPCF_HOST_INPUT: pinned and pageable, float64 and pre-quantised) give the counts of
    the same catalogues on the device, bit for bit; mixing host and device catalogues is refused."""
    L = 400.0
    mks = [synth.SMALL.make_mock(7 + m, n_d=1200 + 300 * m, M=2) for m in range(2)]
    tb, _ = _periodic(L, np.linspace(0, 100.0, 11), 4)
    ref = ctx.tpcf_count(_mocks_to_device(mks), tb, mode=mode)
    host = []
    for m, mk in enumerate(mks):
        h = {"data": torch.from_numpy(np.ascontiguousarray(mk.data)),
             "randoms": torch.from_numpy(np.ascontiguousarray(np.concatenate(mk.randoms))),
             "offsets": [0] + list(np.cumsum([len(r) for r in mk.randoms]))}
        if m == 0:
            h = {k: (v.pin_memory() if torch.is_tensor(v) else v) for k, v in h.items()}
        host.append(h)
    got = ctx.tpcf_count(host, tb, mode=mode)
    qd = oracle.quantize(mks[1].data, oracle.PERIODIC, L)
    qr = np.concatenate([oracle.quantize(r, oracle.PERIODIC, L) for r in mks[1].randoms], axis=1)
    hu = [host[0], {"data_u32": torch.from_numpy(qd.view(np.int32).copy()).pin_memory(),
                    "randoms_u32": torch.from_numpy(qr.view(np.int32).copy()), "offsets": host[1]["offsets"]}]
    got_u = ctx.tpcf_count(hu, tb, mode=mode)
    assert ctx.tpcf_sync() == tp.TPCF_OK
    for k in ("dd", "dr", "rr"):
        assert torch.equal(got[k], ref[k]), k
        assert torch.equal(got_u[k], ref[k]), k
    with pytest.raises(ValueError):
        ctx.tpcf_count([_mocks_to_device(mks)[0], host[1]], tb, mode=mode)


@pytest.mark.parametrize("kern", [1, 2])
def test_counts_host_input_in_groups(tp, ctx, kern):
    """A batched host-input call of a tuned shape runs in groups of consecutive mocks whose copies overlap
    the previous group's count (here with 1 KiB groups, so every mock is a group up to the limit of 8):
    counts equal the oracle's and the device-input call's bit for bit, on two calls in a row (the staging
    buffers reused; pinned and pageable host memory) and with uneven mocks; the launch counters are the
    groups' sums."""
    L = 400.0
    mks = [synth.SMALL.make_mock(40 + m, n_d=700 + 290 * m, M=2) for m in range(10)]
    tb, ob = _periodic(L, np.linspace(0, 60.0, 13), 4)
    refs = [oracle.count_mock(mk.data, mk.randoms, ob) for mk in mks]
    ctx.tpcf_set_option(tp.TPCF_OPT_KERNEL, kern)
    try:
        dev = ctx.tpcf_count(_mocks_to_device(mks), tb)          # tunes the shape
        host = [{"data": torch.from_numpy(np.ascontiguousarray(mk.data)).pin_memory(),
                 "randoms": torch.from_numpy(np.ascontiguousarray(np.concatenate(mk.randoms))).pin_memory(),
                 "offsets": [0] + list(np.cumsum([len(r) for r in mk.randoms]))} for mk in mks]
        ctx.tpcf_set_option(tp.TPCF_OPT_HOST_GROUP_KB, 1)
        # the second call: the mocks reversed, half of them from pageable memory
        pageable = [dict(h, data=torch.from_numpy(np.ascontiguousarray(mks[m].data)),
                         randoms=torch.from_numpy(np.ascontiguousarray(np.concatenate(mks[m].randoms))))
                    if m % 2 else h for m, h in enumerate(host)]
        for rep in range(2):
            got = ctx.tpcf_count(host if rep == 0 else pageable[::-1], tb)
            assert ctx.tpcf_sync() == tp.TPCF_OK
            info = ctx.tpcf_last_count_info()
            assert 2 <= info["n_paircount_launches"] <= 8
            order = list(range(10)) if rep == 0 else list(range(9, -1, -1))
            tot = 0
            for i, m in enumerate(order):
                assert np.array_equal(got["dd"][i].cpu().numpy(), refs[m]["DD"]), (rep, m)
                assert np.array_equal(got["dr"][i].cpu().numpy(), refs[m]["DR"]), (rep, m)
                assert np.array_equal(got["rr"][i].cpu().numpy(), refs[m]["RR"]), (rep, m)
                for k in ("dd", "dr", "rr"):
                    assert torch.equal(got[k][i], dev[k][m]), (rep, m, k)
                tot += refs[m]["DD"].sum() + refs[m]["DR"].sum() + refs[m]["RR"].sum()
            assert info["n_binned"] == tot
            assert info["n_candidates"] >= tot
        ctx.tpcf_set_option(tp.TPCF_OPT_HOST_GROUP_KB, 0)        # never grouped: one launch
        got = ctx.tpcf_count(host, tb)
        assert ctx.tpcf_sync() == tp.TPCF_OK
        assert ctx.tpcf_last_count_info()["n_paircount_launches"] == 1
        for k in ("dd", "dr", "rr"):
            assert torch.equal(got[k], dev[k]), k
    finally:
        ctx.tpcf_set_option(tp.TPCF_OPT_HOST_GROUP_KB, 262144)
        ctx.tpcf_set_option(tp.TPCF_OPT_KERNEL, tp.TPCF_KERNEL_AUTO)
    with pytest.raises(tp.TpcfError):
        ctx.tpcf_set_option(tp.TPCF_OPT_HOST_GROUP_KB, -1)


def test_terms_subset_and_output_untouched(tp, ctx):
    L = 300.0
    mk = synth.SMALL.make_mock(6, n_d=800, M=2)
    tb, ob = _periodic(L, np.linspace(0, 50.0, 6), 1)
    ref = oracle.count_mock(mk.data, mk.randoms, ob)
    out = ctx.tpcf_count(_mocks_to_device([mk]), tb, terms=tp.TPCF_DR)
    ctx.tpcf_sync()
    assert np.array_equal(out["dr"][0].cpu().numpy(), ref["DR"])


def test_open_geometry_position_outside_cube_reports_range(tp, ctx):
    edges = np.linspace(0, 10.0, 3)
    tb = tp.make_binning(edges, 1, tp.TPCF_OPEN, 100.0)
    d = torch.tensor([[1.0, 1.0, 1.0], [150.0, 1.0, 1.0]], dtype=torch.float64, device=DEV)
    ctx.tpcf_count([{"data": d, "randoms": d.clone(), "offsets": [0, 2]}], tb)
    with pytest.raises(tp.TpcfError) as e:
        ctx.tpcf_sync()
    assert e.value.code == tp.TPCF_ERR_RANGE
    # the context stays usable
    d2 = torch.tensor([[1.0, 1.0, 1.0], [5.0, 1.0, 1.0]], dtype=torch.float64, device=DEV)
    out = ctx.tpcf_count([{"data": d2, "randoms": d2.clone(), "offsets": [0, 2]}], tb)
    assert ctx.tpcf_sync() == tp.TPCF_OK
    assert out["dd"][0].tolist() == [1, 0]


def test_bad_arguments_rejected(tp, ctx):
    tb = tp.make_binning([0.0, 10.0], 1, tp.TPCF_PERIODIC, 100.0)
    d = torch.zeros((3, 3), dtype=torch.float64, device=DEV)
    with pytest.raises(tp.TpcfError):
        ctx.tpcf_count([{"data": d, "randoms": d, "offsets": [0, 3]}], tb, terms=0)
    with pytest.raises(tp.TpcfError):
        ctx.tpcf_count([{"data": d, "randoms": d, "offsets": [0, 2, 1]}], tb)
    tbad = tp.make_binning([0.0, 40.0], 1, tp.TPCF_PERIODIC, 100.0)
    with pytest.raises(tp.TpcfError) as e:
        ctx.tpcf_count([{"data": d, "randoms": d, "offsets": [0, 3]}], tbad)
    assert e.value.code == tp.TPCF_ERR_RANGE


# ---------------------------------------------------------------------------
# estimator and covariance
# ---------------------------------------------------------------------------

def _xi_err(x, r):
    both_nan = np.isnan(x) & np.isnan(r)
    e = np.abs(x - r) / (1.0 + np.abs(r))
    e[both_nan] = 0.0
    return float(np.nanmax(e)) if e.size else 0.0, bool(np.all(np.isnan(x) == np.isnan(r)))


def test_ls_parity(tp, ctx):
    rng = np.random.default_rng(4)
    n_mock, M, nbin = 7, 3, 33
    n_d = rng.integers(50, 5000, n_mock)
    n_r = rng.integers(50, 9000, (n_mock, M))
    DD = rng.integers(0, 10 ** 9, (n_mock, nbin))
    DR = rng.integers(0, 10 ** 9, (n_mock, M, nbin))
    RR = rng.integers(0, 10 ** 9, (n_mock, M, nbin))
    RR[2, :, 5] = 0                            # an empty bin -> NaN + warning
    g = [torch.from_numpy(a).to(DEV) for a in (DD, DR, RR)]
    for sel in ([0], [1], [0, 1], [0, 1, 2], [2, 0]):
        xi = ctx.tpcf_ls(*g, n_d, n_r, sel)
        rc = ctx.tpcf_sync()
        ref = np.array([oracle.ls(DD[m], DR[m], RR[m], n_d[m], n_r[m], sel) for m in range(n_mock)])
        err, nan_ok = _xi_err(xi.cpu().numpy(), ref)
        assert nan_ok and err <= 1e-12, (sel, err)
        assert rc == tp.TPCF_WARN_EMPTY_BIN


@pytest.mark.parametrize("M", [1.0, 2.0, 50.0, math.inf])
def test_lc_fp64_parity(tp, ctx, M):
    xa1, xa2, xb = synth.synthetic_xi_variants(41, 120, 37)
    g = [torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in (xa1, xa2, xb)]
    out = ctx.tpcf_lc_cov(*g, 1, M, tp.TPCF_FP64)
    ctx.tpcf_sync()
    ref = oracle.lc_cov(xa1, xa2, xb, 1, M)
    d = np.sqrt(np.diag(ref["Ca"]))
    scale = np.outer(d, d)
    for k in ("C_lc", "Ca", "Cb", "A", "B"):
        err = np.max(np.abs(out[k].cpu().numpy() - ref[k]) / scale)
        assert err <= 1e-12, (k, err)


def test_lc_fp64_ragged_large_nbin(tp, ctx):
    xa1, xa2, xb = synth.synthetic_xi_variants(42, 301, 200)
    g = [torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in (xa1, xa2, xb)]
    out = ctx.tpcf_lc_cov(*g, 1, 50.0, tp.TPCF_FP64)
    ctx.tpcf_sync()
    ref = oracle.lc_cov(xa1, xa2, xb, 1, 50.0)
    d = np.sqrt(np.diag(ref["Ca"]))
    err = np.max(np.abs(out["C_lc"].cpu().numpy() - ref["C_lc"]) / np.outer(d, d))
    assert err <= 1e-12


def test_end_to_end_counts_ls_lc(tp, ctx):
    """Counts -> split LS (R1, R2, R1 u R2) -> LC covariance, all on the GPU, against the oracle chain."""
    L = 300.0
    n, n_mock = 900, 6
    mocks = [synth.SMALL.make_mock(100 + m, n_d=n, M=2) for m in range(n_mock)]
    tb, ob = _periodic(L, np.linspace(0, 60.0, 7), 2)
    out = ctx.tpcf_count(_mocks_to_device(mocks), tb)
    xs = {}
    for key, sel in (("a1", [0]), ("a2", [1]), ("b", [0, 1])):
        xs[key] = ctx.tpcf_ls(out["dd"], out["dr"], out["rr"], [n] * n_mock, [[n, n]] * n_mock, sel)
    cov = ctx.tpcf_lc_cov(xs["a1"], xs["a2"], xs["b"], 1, 50.0, tp.TPCF_FP64)
    ctx.tpcf_sync()
    ref_x = {k: [] for k in xs}
    for mk in mocks:
        c = oracle.count_mock(mk.data, mk.randoms, ob)
        for key, sel in (("a1", [0]), ("a2", [1]), ("b", [0, 1])):
            ref_x[key].append(oracle.ls(c["DD"], c["DR"], c["RR"], n, [n, n], sel))
    for key in xs:
        err, _ = _xi_err(xs[key].cpu().numpy(), np.array(ref_x[key]))
        assert err <= 1e-12
    ref = oracle.lc_cov(*(np.array(ref_x[k]) for k in ("a1", "a2", "b")), 1, 50.0)
    d = np.sqrt(np.abs(np.diag(ref["Ca"])))
    assert np.max(np.abs(cov["C_lc"].cpu().numpy() - ref["C_lc"]) / np.outer(d, d)) <= 1e-12


# ---------------------------------------------------------------------------
# full-size mock of the mid workload (1e5 data points, 2 x 1e5 randoms, 40 x 10 bins)
# ---------------------------------------------------------------------------

@pytest.mark.slow
def test_full_size_mid_mock_bit_exact(tp, ctx):
    w = synth.MID
    mk = w.make_mock(0)
    tb = tp.make_binning(w.s_edges, w.n_mu, tp.TPCF_PERIODIC, w.L)
    ob = oracle.Binning(w.s_edges, w.n_mu, oracle.PERIODIC, w.L)
    dm = _mocks_to_device([mk])
    out = ctx.tpcf_count(dm, tb, mode=tp.TPCF_BATCHED)
    ctx.tpcf_sync()
    ref = oracle.count_mock(mk.data, mk.randoms, ob)
    assert np.array_equal(out["dd"][0].cpu().numpy(), ref["DD"])
    assert np.array_equal(out["dr"][0].cpu().numpy(), ref["DR"])
    assert np.array_equal(out["rr"][0].cpu().numpy(), ref["RR"])
    out2 = ctx.tpcf_count(dm, tb, mode=tp.TPCF_PER_LAUNCH)
    ctx.tpcf_sync()
    for k in ("dd", "dr", "rr"):
        assert torch.equal(out[k], out2[k])


# ---------------------------------------------------------------------------
# split-precision covariance on the tensor cores
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec_name", ["TPCF_TF32X3", "TPCF_BF16X3"])
@pytest.mark.parametrize("n_mock,nbin", [(2, 5), (64, 37), (301, 200), (3500, 200), (130, 400), (400, 1000)])
def test_lc_split_precision_within_1e6(tp, ctx, prec_name, n_mock, nbin):
    """Gram products in TF32x3 / BF16x3 with FP32 accumulation: every covariance element
    within 1e-6 of the float64 oracle, normalised by sqrt(C^a_ii C^a_jj); 400 x 1000 has 36 tile
    pairs per variant (more CTAs than SMs, one chunk of slices each)."""
    xa1, xa2, xb = synth.synthetic_xi_variants(43, n_mock, nbin)
    g = [torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in (xa1, xa2, xb)]
    out = ctx.tpcf_lc_cov(*g, 1, 50.0, getattr(tp, prec_name))
    assert ctx.tpcf_sync() == tp.TPCF_OK
    ref = oracle.lc_cov(xa1, xa2, xb, 1, 50.0)
    d = np.sqrt(np.diag(ref["Ca"]))
    scale = np.outer(d, d)
    for k in ("C_lc", "Ca", "Cb", "A", "B"):
        err = np.max(np.abs(out[k].cpu().numpy() - ref[k]) / scale)
        assert err <= 1e-6, (k, err)


# ---------------------------------------------------------------------------
# batched path: CUDA-graph replay and autotuner
# ---------------------------------------------------------------------------

def test_graph_replay_bit_identical_and_timed(tp):
    L = 300.0
    w = synth.Workload("t", 35, 3, "periodic", L, (0, 0, 0), 1200, 2, 60.0, 12, 4, "x", n_parent=5e-5, sigma=2.0)
    mocks = [w.make_mock(m) for m in range(3)]
    tb, ob = _periodic(L, w.s_edges, 4)
    dm = _mocks_to_device(mocks)
    c = tp.Context(0)
    c.tpcf_set_option(tp.TPCF_OPT_GRAPHS, 0)
    ref = c.tpcf_count(dm, tb)
    c.tpcf_sync()
    assert c.tpcf_last_count_info()["graph_replay"] == 0
    c.tpcf_set_option(tp.TPCF_OPT_GRAPHS, 1)
    out = {k: torch.empty_like(v) for k, v in ref.items()}
    c.tpcf_count(dm, tb, out=out)            # captures
    c.tpcf_set_timing(True)
    for _ in range(3):
        for v in out.values():
            v.fill_(-7)                      # replays must rewrite every output
        c.tpcf_count(dm, tb, out=out)
    assert c.tpcf_sync() == tp.TPCF_OK
    info = c.tpcf_last_count_info()
    assert info["graph_replay"] == 1 and info["timed_calls"] == 3 and info["paircount_ms"] > 0
    for k in ("dd", "dr", "rr"):
        assert torch.equal(out[k], ref[k])
    o = oracle.count_mock(mocks[1].data, mocks[1].randoms, ob)
    assert np.array_equal(out["rr"][1].cpu().numpy(), o["RR"])
    c.close()


def test_autotuner_choice_is_exact(tp):
    L = 400.0
    w = synth.Workload("t", 36, 8, "periodic", L, (0, 0, 0), 1500, 2, 80.0, 20, 5, "x", n_parent=3e-5, sigma=3.0)
    mocks = [w.make_mock(m) for m in range(8)]
    tb, ob = _periodic(L, w.s_edges, 5)
    c = tp.Context(0)
    dm = _mocks_to_device(mocks)
    out = c.tpcf_count(dm, tb)
    c.tpcf_sync()
    info = c.tpcf_last_count_info()
    # the tuner chose a counter (linear bins, x line of sight: both apply), a subdivision, a unit size
    # (the direct counter's is 64) and a grid of whole blocks per SM
    assert info["pair_kernel"] in (tp.TPCF_KERNEL_DIRECT, tp.TPCF_KERNEL_GENERAL)
    assert info["cell_subdiv"] in (2, 3, 4) and info["unit_chunk"] in (64, 128)
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    assert info["pair_blocks"] > 0 and info["pair_blocks"] % n_sm == 0
    for m in (0, 7):
        o = oracle.count_mock(mocks[m].data, mocks[m].randoms, ob)
        assert np.array_equal(out["dd"][m].cpu().numpy(), o["DD"])
        assert np.array_equal(out["dr"][m].cpu().numpy(), o["DR"])
    # the per-launch path runs the tuned configuration and gives the same counts
    pl = c.tpcf_count(dm, tb, mode=tp.TPCF_PER_LAUNCH)
    c.tpcf_sync()
    info2 = c.tpcf_last_count_info()
    assert (info2["pair_kernel"], info2["cell_subdiv"]) == (info["pair_kernel"], info["cell_subdiv"])
    for k in ("dd", "dr", "rr"):
        assert torch.equal(out[k], pl[k])
    c.close()
