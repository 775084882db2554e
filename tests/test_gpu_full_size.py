"""Full-size parity for the cut-sky batching and the large periodic workloads.

A whole full-size mock is beyond the brute-force oracle (5e11 pair tests for
a 1e6-point catalogue), so each catalogue X is split into a sample S (its
first S_N points) and the rest X'.  Every count then decomposes exactly:

    auto(X)    = auto(X') + auto(S) + cross(S, X')
    cross(X,Y) = cross(X', Y') + cross(S_X, Y) + cross(X', S_Y)

The library counts the full mock and the reduced mock (X' for every
catalogue) in the batched launch the benchmark uses; the oracle counts every
term that involves a sample point, by brute force over the full-size partner
catalogues.  The identities must hold bit for bit.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

DEV = "cuda:0"
S_N = 1000


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


def _dev(data, randoms):
    offs = [0] + list(np.cumsum([len(r) for r in randoms]))
    return {"data": torch.from_numpy(np.ascontiguousarray(data)).to(DEV),
            "randoms": torch.from_numpy(np.ascontiguousarray(np.concatenate(randoms))).to(DEV),
            "offsets": offs}


def _oracle_sample_terms(mk, ob, origin):
    """Brute-force counts of every pair that involves a sample point."""
    q = lambda x: oracle.quantize(x, ob.geometry, ob.L, origin)
    d, rs = q(mk.data), [q(r) for r in mk.randoms]
    sd, dp = d[:, :S_N], d[:, S_N:]
    out = {"DD": oracle.count_pairs(sd, None, ob)[0] + oracle.count_pairs(sd, dp, ob)[0], "DR": [], "RR": []}
    for r in rs:
        sr, rp = r[:, :S_N], r[:, S_N:]
        out["DR"].append(oracle.count_pairs(sd, r, ob)[0] + oracle.count_pairs(sr, dp, ob)[0])
        out["RR"].append(oracle.count_pairs(sr, None, ob)[0] + oracle.count_pairs(sr, rp, ob)[0])
    return out


def _check_decomposition(ctx, tp, mocks, tb, ob, origin=(0.0, 0.0, 0.0), want_direct=True):
    """Both pair counters (TPCF_KERNEL_DIRECT, which must take the direct counter here, and
    TPCF_KERNEL_GENERAL) against the same oracle sample counts."""
    refs = [_oracle_sample_terms(mk, ob, origin) for mk in mocks]
    full = None
    for kern in (tp.TPCF_KERNEL_DIRECT, tp.TPCF_KERNEL_GENERAL):
        ctx.tpcf_set_option(tp.TPCF_OPT_KERNEL, kern)
        try:
            full = ctx.tpcf_count([_dev(mk.data, mk.randoms) for mk in mocks], tb, mode=tp.TPCF_BATCHED)
            assert ctx.tpcf_sync() == tp.TPCF_OK
            ran = ctx.tpcf_last_count_info()["pair_kernel"]
            assert ran == (kern if want_direct else tp.TPCF_KERNEL_GENERAL), (kern, ran)
            red = ctx.tpcf_count([_dev(mk.data[S_N:], [r[S_N:] for r in mk.randoms]) for mk in mocks], tb,
                                 mode=tp.TPCF_BATCHED)
            assert ctx.tpcf_sync() == tp.TPCF_OK
        finally:
            ctx.tpcf_set_option(tp.TPCF_OPT_KERNEL, tp.TPCF_KERNEL_AUTO)
        for m, mk in enumerate(mocks):
            ref = refs[m]
            dd = full["dd"][m].cpu().numpy()
            assert dd.sum() > 0
            assert np.array_equal(dd, red["dd"][m].cpu().numpy() + ref["DD"]), (kern, m, "DD")
            for i in range(len(mk.randoms)):
                assert np.array_equal(full["dr"][m, i].cpu().numpy(),
                                      red["dr"][m, i].cpu().numpy() + ref["DR"][i]), (kern, m, i, "DR")
                assert np.array_equal(full["rr"][m, i].cpu().numpy(),
                                      red["rr"][m, i].cpu().numpy() + ref["RR"][i]), (kern, m, i, "RR")
    return full


def test_large_periodic_mock_full_size(tp, ctx):
    """One mock of the large periodic workload: 1e6 Neyman-Scott points, 2 x 1e6 randoms, L = 2000,
    40 s x 10 mu bins to 200, x line of sight."""
    w = synth.SCALE
    mk = w.make_mock(0)
    assert len(mk.data) == 1_000_000 and all(len(r) == 1_000_000 for r in mk.randoms)
    tb = tp.make_binning(w.s_edges, w.n_mu, tp.TPCF_PERIODIC, w.L)
    ob = oracle.Binning(w.s_edges, w.n_mu, oracle.PERIODIC, w.L)
    full = _check_decomposition(ctx, tp, [mk], tb, ob)
    # DR is symmetric in its catalogues: count R_1 x D with the roles swapped
    sw = ctx.tpcf_count([_dev(mk.randoms[0], [mk.data])], tb, terms=tp.TPCF_DR, mode=tp.TPCF_BATCHED)
    assert ctx.tpcf_sync() == tp.TPCF_OK
    assert torch.equal(sw["dr"][0, 0], full["dr"][0, 0])


def test_cut_sky_uneven_mocks_full_size(tp, ctx):
    """Cut-sky octant shell 1200-2400, observer at the origin, midpoint line of sight, 40 s x 5 mu bins:
    three mocks of uneven size, including both ends of the 50k-400k range, in one batched launch."""
    w = synth.BATCHING
    mocks = [w.make_mock(0, n_d=400_000), w.make_mock(1), w.make_mock(2, n_d=50_000)]
    tb = tp.make_binning(w.s_edges, w.n_mu, tp.TPCF_OPEN, w.L, los=tp.TPCF_LOS_MIDPOINT, observer=w.observer)
    ob = oracle.Binning(w.s_edges, w.n_mu, oracle.OPEN, w.L, los=oracle.LOS_MIDPOINT, observer=w.observer)
    _check_decomposition(ctx, tp, mocks, tb, ob)
