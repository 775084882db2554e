// tpcf_count: binned pair counts of many mocks (Sect. 2.1 DD, DR_i, RR_i;
// Sect. 4.3 (s, mu) bins) -- host orchestration.
//
//   prepare()  validates the call and builds, on the host, the plan (exact
//              thresholds, FP32 bands, mesh), the catalogue and term tables
//              and the workspace layout;
//   enqueue()  puts the whole GPU sequence on a stream: quantisation and
//              cell keys, counting sort by cell, work-unit list, and the pair
//              count (one persistent launch, or one launch per term);
//   the batched path captures enqueue() once as a CUDA graph per call shape
//              and replays it; an autotuner picks the pair counter (direct
//              or general), the mesh subdivision, the work-unit size and the
//              blocks per SM of a new shape by timing candidates on a few of
//              its mocks;
//   host input (TPCF_HOST_INPUT) is staged into the context's workspace,
//              in groups of mocks whose copies overlap the previous group's
//              count when the shape is already tuned (count_host_grouped).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

using namespace tpcf;
using namespace tpcf::detail;

namespace {

struct RqCopy {
    uint32_t *dst;
    const uint32_t *src;
    size_t n, pitch;
};

struct Setup {
    Plan pl;
    std::vector<Cat> cats;
    std::vector<Term> terms;
    std::vector<RqCopy> rq;
    int M = 0;
    unsigned mask = 0;
    size_t NT = 0, ncc = 0, ntc = 0, tmp_n = 0;
    uint32_t max_n = 0;
    unsigned long long units_bound = 0;
    int chunk = UNIT_CHUNK;
    int smem = 0, blocks = 0;
    bool direct = false;            // the direct pair counter (pairdirect.cu) runs
    DirectParams dp;
    int claim_units = 1;            // direct counter: units per block claim
    double L = 0, origin[3] = {0, 0, 0};
    // outputs to clear
    int64_t *dd = nullptr, *dr = nullptr, *rr = nullptr;
    size_t n_dd = 0, n_drr = 0;
    // workspace
    void *uq = nullptr, *keys = nullptr, *us = nullptr, *pf = nullptr, *pcx = nullptr, *cc = nullptr,
         *cs = nullptr, *tmp = nullptr, *uc = nullptr, *ust = nullptr, *units = nullptr, *claim = nullptr,
         *rqbuf = nullptr, *bscr = nullptr;
    // small tables (host bytes and layout)
    std::vector<unsigned char> small;
    size_t o_cats = 0, o_terms = 0, o_orig = 0, o_tab = 0;
};

// Validate and build everything host-side for one call; allocates workspace.
int prepare(tpcf_ctx *ctx, const tpcf_mock *mocks, int n_mock, const tpcf_binning *binning, unsigned terms,
            int64_t *dd, int64_t *dr, int64_t *rr, int mode, const Tuned &cfg, Setup &S)
{
    const int subdiv = cfg.subdiv, chunk = cfg.chunk;
    // the tuned counter, else the context's preference (untuned AUTO: the general counter)
    const int kern = cfg.kernel >= 0 ? cfg.kernel
                                     : (ctx->kernel_pref == TPCF_KERNEL_AUTO ? TPCF_KERNEL_GENERAL : ctx->kernel_pref);
    int rc;
    if ((rc = validate_binning(ctx, binning))) return rc;
    if (n_mock < 0 || (n_mock > 0 && !mocks)) return fail(ctx, TPCF_ERR_ARG, "mocks is NULL");
    if (terms == 0 || (terms & ~7u)) return fail(ctx, TPCF_ERR_ARG, "terms must be a non-empty mask of DD|DR|RR");
    if (mode != TPCF_BATCHED && mode != TPCF_PER_LAUNCH) return fail(ctx, TPCF_ERR_ARG, "bad mode");
    if ((terms & TPCF_DD) && !dd) return fail(ctx, TPCF_ERR_ARG, "dd output is NULL");
    if ((terms & TPCF_DR) && !dr) return fail(ctx, TPCF_ERR_ARG, "dr output is NULL");
    if ((terms & TPCF_RR) && !rr) return fail(ctx, TPCF_ERR_ARG, "rr output is NULL");
    const bool need_d = terms & (TPCF_DD | TPCF_DR);
    const bool need_r = terms & (TPCF_DR | TPCF_RR);
    int M = -1;
    unsigned long long n_total = 0, max_cat = 0, n_cat_est = 0, n_terms_est = 0;
    for (int m = 0; m < n_mock; m++) {
        const tpcf_mock &mk = mocks[m];
        if (need_d) {
            if (mk.n_d < 0) return fail(ctx, TPCF_ERR_ARG, "n_d < 0");
            if (mk.n_d > 0 && !mk.data_xyz == !mk.data_u32)
                return fail(ctx, TPCF_ERR_ARG, "give exactly one of data_xyz / data_u32");
            n_total += (unsigned long long)mk.n_d;
            max_cat = std::max<unsigned long long>(max_cat, mk.n_d);
            n_cat_est++;
        }
        if (need_r) {
            if (mk.M < 1) return fail(ctx, TPCF_ERR_ARG, "M must be >= 1");
            if (M >= 0 && mk.M != M) return fail(ctx, TPCF_ERR_ARG, "all mocks need the same M");
            M = mk.M;
            if (!mk.rand_offsets) return fail(ctx, TPCF_ERR_ARG, "rand_offsets is NULL");
            if (mk.rand_offsets[0] != 0) return fail(ctx, TPCF_ERR_ARG, "rand_offsets[0] must be 0");
            for (int i = 0; i < mk.M; i++) {
                if (mk.rand_offsets[i + 1] < mk.rand_offsets[i])
                    return fail(ctx, TPCF_ERR_ARG, "rand_offsets must be non-decreasing");
                max_cat = std::max<unsigned long long>(max_cat, mk.rand_offsets[i + 1] - mk.rand_offsets[i]);
                n_cat_est++;
            }
            const int64_t nr = mk.rand_offsets[mk.M];
            if (nr > 0 && !mk.rand_xyz == !mk.rand_u32)
                return fail(ctx, TPCF_ERR_ARG, "give exactly one of rand_xyz / rand_u32");
            n_total += (unsigned long long)nr;
        }
    }
    if (n_total >= (1ull << 31)) return fail(ctx, TPCF_ERR_RANGE, "more than 2^31 points in one call");
    if (M < 0) M = 0;
    S.M = M;
    S.mask = terms;
    for (int m = 0; m < n_mock; m++)
        n_terms_est += ((terms & TPCF_DD) ? 1 : 0) +
                       (unsigned long long)M * (((terms & TPCF_DR) ? 1 : 0) + ((terms & TPCF_RR) ? 1 : 0));

    // mesh cap: a few cells per point of the largest catalogue, and the
    // (catalogue x cell) and (term x cell) tables indexable in 32 bits
    unsigned long long max_cells = std::max<unsigned long long>(64, 4 * max_cat);
    max_cells = std::min<unsigned long long>(max_cells, 1ull << 24);
    const unsigned long long tabs = std::max<unsigned long long>(1, std::max(n_cat_est, n_terms_est));
    max_cells = std::min<unsigned long long>(max_cells, ((1ull << 32) - 2) / tabs);

    std::string perr;
    if ((rc = build_plan(*binning, subdiv, max_cells, S.pl, perr))) return fail(ctx, rc, perr);
    if ((rc = check_mu_width(ctx, binning, S.pl.prm))) return rc;
    const CountParams &prm = S.pl.prm;
    S.chunk = std::max(32, std::min(chunk, UNIT_CHUNK));
    if (kern != TPCF_KERNEL_GENERAL) {
        int sm_sm = 0, sm_blk = 0, resv = 0;
        if (cudaDeviceGetAttribute(&sm_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&sm_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, ctx->device) != cudaSuccess) {
            cudaGetLastError();
            sm_sm = 0;
        }
        if (sm_sm > 0 && build_direct(*binning, S.pl, sm_sm, sm_blk, resv, max_cat, S.dp)) {
            S.direct = true;
            S.chunk = std::min(S.chunk, DIRECT_ACHUNK);
        }
    }
    // The pair counters add into 32-bit shared-memory counters: one unit adds
    // at most chunk x (points of one catalogue) pairs to any counter, which
    // must stay below 2^32 (the direct counter drains before the sum over
    // units could reach 2^31).
    if (max_cat > 0) {
        const unsigned long long cap = ((1ull << 32) - 1) / max_cat;
        if (cap < 16) return fail(ctx, TPCF_ERR_RANGE, "a catalogue above 2^28 points would overflow the 32-bit pair counters");
        if ((unsigned long long)S.chunk > cap) S.chunk = (int)(cap & ~15ull);
    }
    S.L = binning->box_L;
    for (int c = 0; c < 3; c++) S.origin[c] = binning->origin[c];

    // catalogues and terms
    uint32_t p0 = 0;
    std::vector<int> rand_cat0(n_mock, -1);
    for (int m = 0; m < n_mock; m++) {
        const tpcf_mock &mk = mocks[m];
        const int cd = (int)S.cats.size();
        if (need_d) {
            Cat c;
            c.xyz = mk.data_xyz;
            c.u32 = mk.data_xyz ? nullptr : mk.data_u32;
            c.p0 = p0;
            c.n = (uint32_t)mk.n_d;
            p0 += c.n;
            S.max_n = std::max(S.max_n, c.n);
            S.cats.push_back(c);
        }
        const int cr = (int)S.cats.size();
        rand_cat0[m] = cr;
        if (need_r) {
            for (int i = 0; i < M; i++) {
                Cat c;
                const int64_t o0 = mk.rand_offsets[i], o1 = mk.rand_offsets[i + 1];
                c.xyz = mk.rand_xyz ? mk.rand_xyz + 3 * o0 : nullptr;
                c.u32 = nullptr;   // pre-quantised subsets are gathered below
                c.p0 = p0;
                c.n = (uint32_t)(o1 - o0);
                p0 += c.n;
                S.max_n = std::max(S.max_n, c.n);
                S.cats.push_back(c);
            }
        }
        const int nbin = prm.nbin;
        if (terms & TPCF_DD) S.terms.push_back(Term{cd, cd, 1, 0, (long long *)dd + (size_t)m * nbin});
        for (int i = 0; i < M; i++) {
            if (terms & TPCF_DR)
                S.terms.push_back(Term{cd, cr + i, 0, 0, (long long *)dr + ((size_t)m * M + i) * nbin});
            if (terms & TPCF_RR)
                S.terms.push_back(Term{cr + i, cr + i, 1, 0, (long long *)rr + ((size_t)m * M + i) * nbin});
        }
    }
    // longest first: mocks in decreasing order of their pair count (the sum over their terms of n_a n_b,
    // or n (n - 1) / 2 for an auto count), each mock's terms kept together (its catalogues stay in L2), so
    // that the units claimed last, at the end of a launch, belong to the cheapest mocks
    {
        auto cost = [&](const Term &t) {
            const double na = (double)S.cats[t.cat_a].n, nb = (double)S.cats[t.cat_b].n;
            return t.auto_pairs ? 0.5 * na * (na - 1.0) : na * nb;
        };
        const size_t per = S.terms.size() / std::max(1, n_mock);   // every mock adds the same number of terms
        std::vector<double> mc(n_mock, 0.0);
        for (size_t k = 0; k < S.terms.size(); k++) mc[k / std::max<size_t>(1, per)] += cost(S.terms[k]);
        std::vector<int> order(n_mock);
        for (int m = 0; m < n_mock; m++) order[m] = m;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return mc[x] > mc[y]; });
        std::vector<Term> sorted;
        sorted.reserve(S.terms.size());
        for (int m : order)
            for (size_t k = 0; k < per; k++) sorted.push_back(S.terms[(size_t)m * per + k]);
        S.terms.swap(sorted);
    }
    S.dd = (terms & TPCF_DD) ? dd : nullptr;
    S.dr = (terms & TPCF_DR) ? dr : nullptr;
    S.rr = (terms & TPCF_RR) ? rr : nullptr;
    S.n_dd = (size_t)n_mock * prm.nbin;
    S.n_drr = (size_t)n_mock * M * prm.nbin;
    S.NT = (size_t)n_total;
    if (S.NT == 0 || S.terms.empty()) return TPCF_OK;

    S.ncc = S.cats.size() * (size_t)prm.n_cells + 1;
    if (S.ncc >= (1ull << 32)) return fail(ctx, TPCF_ERR_RANGE, "too many catalogues x cells");
    S.ntc = S.terms.size() * (size_t)prm.n_cells + 1;
    if (S.ntc >= (1ull << 32)) return fail(ctx, TPCF_ERR_RANGE, "too many terms x cells");
    for (const Term &t : S.terms) {
        const unsigned long long n = S.cats[t.cat_a].n;
        S.units_bound += n / S.chunk + std::min<unsigned long long>(n, prm.n_cells) + 1;
    }
    S.tmp_n = std::max(scan_tmp_elems(S.ncc), scan_tmp_elems(S.ntc));

    // workspace
    const size_t NT = S.NT;
    if ((rc = ensure(ctx, "uq", 3 * NT * 4, &S.uq))) return rc;
    if ((rc = ensure(ctx, "keys", NT * 4, &S.keys))) return rc;
    if ((rc = ensure(ctx, "us", 3 * NT * 4, &S.us))) return rc;
    if ((rc = ensure(ctx, "pf", NT * 16, &S.pf))) return rc;
    if ((rc = ensure(ctx, "pcx", NT * 2, &S.pcx))) return rc;
    if ((rc = ensure(ctx, "cellcount", S.ncc * 4, &S.cc))) return rc;
    if ((rc = ensure(ctx, "cellstart", S.ncc * 4, &S.cs))) return rc;
    if ((rc = ensure(ctx, "scantmp", S.tmp_n * 4, &S.tmp))) return rc;
    if ((rc = ensure(ctx, "ucount", S.ntc * 4, &S.uc))) return rc;
    if ((rc = ensure(ctx, "ustart", S.ntc * 4, &S.ust))) return rc;
    if ((rc = ensure(ctx, "units", S.units_bound * sizeof(Unit), &S.units))) return rc;
    if ((rc = ensure(ctx, "claim", std::max<size_t>(256, 4 * (S.terms.size() + 1)), &S.claim))) return rc;

    // pre-quantised randoms: one [3][n_r] array per mock, gathered into a
    // compact [3][n] block per subset
    size_t rq_elems = 0;
    if (need_r)
        for (int m = 0; m < n_mock; m++)
            if (!mocks[m].rand_xyz && mocks[m].rand_offsets[M] > 0) rq_elems += 3 * (size_t)mocks[m].rand_offsets[M];
    if (rq_elems) {
        if ((rc = ensure(ctx, "rq", rq_elems * 4, &S.rqbuf))) return rc;
        size_t off = 0;
        for (int m = 0; m < n_mock; m++) {
            const tpcf_mock &mk = mocks[m];
            if (mk.rand_xyz || mk.rand_offsets[M] == 0) continue;
            const size_t nr = (size_t)mk.rand_offsets[M];
            for (int i = 0; i < M; i++) {
                const size_t o0 = (size_t)mk.rand_offsets[i], n = (size_t)(mk.rand_offsets[i + 1] - o0);
                uint32_t *dst = (uint32_t *)S.rqbuf + off;
                if (n > 0) S.rq.push_back(RqCopy{dst, mk.rand_u32 + o0, n, nr});
                S.cats[rand_cat0[m] + i].u32 = dst;
                off += 3 * n;
            }
        }
    }

    // small tables: cats | terms | orig | table
    S.o_cats = 0;
    S.o_terms = al(S.o_cats + S.cats.size() * sizeof(Cat));
    S.o_orig = al(S.o_terms + S.terms.size() * sizeof(Term));
    S.o_tab = al(S.o_orig + S.pl.orig.size() * 4);
    S.small.assign(al(S.o_tab + S.pl.table.size() * 2), 0);
    std::memcpy(S.small.data() + S.o_cats, S.cats.data(), S.cats.size() * sizeof(Cat));
    std::memcpy(S.small.data() + S.o_terms, S.terms.data(), S.terms.size() * sizeof(Term));
    std::memcpy(S.small.data() + S.o_orig, S.pl.orig.data(), S.pl.orig.size() * 4);
    std::memcpy(S.small.data() + S.o_tab, S.pl.table.data(), S.pl.table.size() * 2);

    // launch shape (host queries, outside any capture)
    if (S.direct) {
        cudaError_t e = pairdirect_set_attrs(S.dp, prm.n_mu > 1);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "pairdirect_set_attrs");
        const int occ = pairdirect_max_blocks_per_sm(S.dp, prm.n_mu > 1);
        if (occ < 1) return fail(ctx, TPCF_ERR_CUDA, "the direct pair counter does not fit on an SM");
        S.smem = S.dp.smem;
        S.blocks = ctx->n_sm * (cfg.bps > 0 ? std::min(cfg.bps, occ) : occ);
        // units per block claim, at most 2^30 pairs per counter: about eight claims per block in the
        // batched launch; in the one-launch-per-term mode one claim per block of the term's share (every
        // claim ends in a block barrier, which a launch of one term cannot amortise)
        const unsigned long long by_work =
            mode == TPCF_PER_LAUNCH
                ? std::max<unsigned long long>(1, (S.units_bound / std::max<size_t>(1, S.terms.size()) + S.blocks - 1) /
                                                      (unsigned long long)S.blocks)
                : std::max<unsigned long long>(1, S.units_bound / (8ull * S.blocks));
        const unsigned long long by_wrap = std::max<unsigned long long>(1, (1ull << 30) / S.dp.unit_pair_bound);
        S.claim_units = (int)std::min<unsigned long long>({by_work, by_wrap, 4096ull});
        return TPCF_OK;
    }
    S.smem = paircount_smem_bytes(prm, 8);
    {
        // the block histogram (4 nbin bytes) sits in shared memory beside the queues
        int optin = 0;
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device) != cudaSuccess) {
            cudaGetLastError();
            optin = 0;
        }
        if (optin > 0 && S.smem > optin)
            return fail(ctx, TPCF_ERR_RANGE, "the binning needs " + std::to_string(S.smem) +
                                                 " bytes of shared memory per block; the device allows " +
                                                 std::to_string(optin));
    }
    cudaError_t e = paircount_set_attrs(prm, S.smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "paircount_set_attrs");
    const int occ = paircount_max_blocks_per_sm(prm, 8, S.smem);
    S.blocks = ctx->n_sm * (cfg.bps > 0 ? std::min(cfg.bps, occ) : occ);
    if ((rc = ensure(ctx, "pairscratch", paircount_scratch_bytes(S.blocks), &S.bscr))) return rc;
    return TPCF_OK;
}

// Every GPU step of one call, on stream s.  `small` holds S.small on the
// device.  ev0/ev1 (may be null) are recorded around the pair-count kernels;
// `external` makes them event-record nodes when the stream is being captured.
int enqueue(tpcf_ctx *ctx, const Setup &S, int mode, cudaStream_t s, void *small, cudaEvent_t ev0, cudaEvent_t ev1,
            bool external, int &kernels)
{
    const CountParams &prm = S.pl.prm;
    kernels = 0;
    if (S.dd) CK(cudaMemsetAsync(S.dd, 0, S.n_dd * 8, s));
    if (S.dr && S.n_drr) CK(cudaMemsetAsync(S.dr, 0, S.n_drr * 8, s));
    if (S.rr && S.n_drr) CK(cudaMemsetAsync(S.rr, 0, S.n_drr * 8, s));
    CK(cudaMemsetAsync(ctx->stats, 0, 8 * sizeof(unsigned long long), s));
    if (S.NT == 0 || S.terms.empty()) {
        CK(cudaMemcpyAsync(ctx->stats_host, ctx->stats, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        return TPCF_OK;
    }
    for (const RqCopy &c : S.rq)
        CK(cudaMemcpy2DAsync(c.dst, c.n * 4, c.src, c.pitch * 4, c.n * 4, 3, cudaMemcpyDeviceToDevice, s));
    const Cat *d_cats = (const Cat *)((const char *)small + S.o_cats);
    const Term *d_terms = (const Term *)((const char *)small + S.o_terms);
    const uint32_t *d_orig = (const uint32_t *)((const char *)small + S.o_orig);
    const int16_t *d_tab = (const int16_t *)((const char *)small + S.o_tab);
    const int n_cat = (int)S.cats.size(), n_terms = (int)S.terms.size();
    uint32_t *cc = (uint32_t *)S.cc, *cs = (uint32_t *)S.cs, *tmp = (uint32_t *)S.tmp;
    uint32_t *uc = (uint32_t *)S.uc, *ust = (uint32_t *)S.ust;

    // mesh build: quantise + keys + cell histogram, scan, scatter
    CK(cudaMemsetAsync(cc, 0, S.ncc * 4, s));
    CK(launch_quantize_keys(d_cats, n_cat, S.max_n, prm, S.L, S.origin, (uint32_t)S.NT, (uint32_t *)S.uq,
                            (uint32_t *)S.keys, cc, ctx->status, s));
    CK(launch_scan_u32(cc, cs, S.ncc, tmp, S.tmp_n, s));
    CK(cudaMemsetAsync(cc, 0, S.ncc * 4, s));
    CK(launch_scatter(d_cats, n_cat, S.max_n, prm, (uint32_t *)S.uq, (uint32_t *)S.keys, cs, cc, d_orig,
                      (uint32_t)S.NT, (uint32_t *)S.us, (float4 *)S.pf, (uint16_t *)S.pcx, s));
    kernels += 5;

    Mesh mesh;
    mesh.pf = (const float4 *)S.pf;
    mesh.pcx = (const uint16_t *)S.pcx;
    mesh.us = (const uint32_t *)S.us;
    mesh.n_total = (uint32_t)S.NT;
    mesh.cellstart = cs;
    mesh.orig = d_orig;
    PairLaunch L;
    L.warps_per_block = 8;
    L.smem_bytes = S.smem;
    L.chunk = S.chunk;
    L.scratch = S.bscr;
    if (mode == TPCF_BATCHED || S.direct) {
        // the work-unit list (the direct counter uses it in both modes)
        CK(cudaMemsetAsync(uc + (S.ntc - 1), 0, 4, s));
        CK(launch_unit_count(d_terms, n_terms, d_cats, prm.n_cells, cs, S.chunk, uc, s));
        CK(launch_scan_u32(uc, ust, S.ntc, tmp, S.tmp_n, s));
        CK(launch_unit_fill(d_terms, n_terms, d_cats, prm.n_cells, cs, S.chunk, ust, (Unit *)S.units, s));
        CK(cudaMemsetAsync(S.claim, 0, 4 * (S.terms.size() + 1), s));
        kernels += 5;
    }
    if (mode == TPCF_BATCHED) {
        L.persistent = 1;
        L.term = 0;
        L.blocks = S.blocks;
        if (ev0) CK(cudaEventRecordWithFlags(ev0, s, external ? cudaEventRecordExternal : cudaEventRecordDefault));
        if (S.direct) {
            L.chunk = S.claim_units;
            CK(launch_pairdirect(prm, S.dp, mesh, d_terms, (const Unit *)S.units, ust + (S.ntc - 1),
                                 (unsigned *)S.claim, ctx->stats, L, s));
        } else {
            CK(launch_paircount(prm, mesh, d_terms, d_cats, (const Unit *)S.units, ust + (S.ntc - 1),
                                (unsigned *)S.claim, d_tab, ctx->stats, ctx->status, L, s));
        }
        if (ev1) CK(cudaEventRecordWithFlags(ev1, s, external ? cudaEventRecordExternal : cudaEventRecordDefault));
        kernels += 1;
        CK(cudaMemcpyAsync(ctx->stats + 3, ust + (S.ntc - 1), 4, cudaMemcpyDeviceToDevice, s));
    } else {
        if (ev0) CK(cudaEventRecordWithFlags(ev0, s, external ? cudaEventRecordExternal : cudaEventRecordDefault));
        for (int t = 0; t < n_terms; t++) {
            L.persistent = 0;
            L.term = t;
            if (S.direct) {
                // one launch per term over that term's units, each with its own claim counter;
                // claims start at the term's share per block and shrink (guided), so that few
                // block barriers (each waits for the block's slowest warp) fall in one launch
                L.blocks = S.blocks;
                L.chunk = std::max(1, S.claim_units);
                CK(launch_pairdirect(prm, S.dp, mesh, d_terms, (const Unit *)S.units, ust + (S.ntc - 1),
                                     (unsigned *)S.claim + 1 + t, ctx->stats, L, s));
            } else {
                L.blocks = std::min(S.blocks, prm.n_cells);   // blocks stride over the cells
                CK(launch_paircount(prm, mesh, d_terms, d_cats, nullptr, nullptr, nullptr, d_tab, ctx->stats,
                                    ctx->status, L, s));
            }
        }
        if (ev1) CK(cudaEventRecordWithFlags(ev1, s, external ? cudaEventRecordExternal : cudaEventRecordDefault));
        kernels += n_terms;
    }
    CK(cudaMemcpyAsync(ctx->stats_host, ctx->stats, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    return TPCF_OK;
}

// small tables through the context's pinned staging area (direct path)
int upload_small(tpcf_ctx *ctx, const Setup &S, cudaStream_t s, void **dev)
{
    int rc;
    if ((rc = ensure(ctx, "small", S.small.size(), dev))) return rc;
    void *host;
    if ((rc = staging(ctx, S.small.size(), &host))) return rc;
    std::memcpy(host, S.small.data(), S.small.size());
    CK(cudaMemcpyAsync(*dev, host, S.small.size(), cudaMemcpyHostToDevice, s));
    return staging_done(ctx, s);
}

// an event pair [2 k, 2 k + 1] of v for the k-th timed span, or -1
int event_pair(std::vector<cudaEvent_t> &v, int k)
{
    if (k >= 4096) return -1;
    while ((int)v.size() < 2 * (k + 1)) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        v.push_back(e);
    }
    return k;
}

// timing slot for this call, or -1
int timing_slot(tpcf_ctx *ctx)
{
    if (!ctx->timing || ctx->n_timed >= 4096) return -1;
    const int slot = ctx->n_timed;
    while ((int)ctx->ev.size() < 2 * (slot + 1)) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        ctx->ev.push_back(e);
    }
    return slot;
}

std::string graph_key(const Setup &S, int mode, tpcf_ctx *ctx)
{
    std::string k;
    auto put = [&](const void *p, size_t n) { k.append((const char *)p, n); };
    put(&S.pl.prm, sizeof(CountParams));
    put(&S.direct, sizeof(S.direct));
    put(&S.dp, sizeof(S.dp));
    put(&mode, sizeof(mode));
    put(&S.chunk, sizeof(S.chunk));
    put(&S.blocks, sizeof(S.blocks));
    put(&S.NT, sizeof(S.NT));
    put(&S.L, sizeof(S.L));
    put(S.origin, sizeof(S.origin));
    put(S.small.data(), S.small.size());   // catalogue pointers, sizes, outputs, cell corners, table
    for (const RqCopy &c : S.rq) put(&c, sizeof(c));
    const void *ws[] = {S.uq, S.keys, S.us, S.pf, S.pcx, S.cc, S.cs, S.tmp, S.uc, S.ust, S.units, S.claim,
                        S.rqbuf, S.bscr, S.dd, S.dr, S.rr, ctx->stats, ctx->stats_host, ctx->status};
    put(ws, sizeof(ws));
    return k;
}

int run_graph(tpcf_ctx *ctx, const Setup &S, int mode, cudaStream_t s, int slot)
{
    const std::string key = graph_key(S, mode, ctx);
    GraphEntry *g = nullptr;
    for (GraphEntry &e : ctx->graphs)
        if (e.key == key) g = &e;
    if (!g) {
        // room for every group of a grouped host-input call beside a few other call shapes
        if (ctx->graphs.size() >= (size_t)(2 * PIPE_GROUPS_MAX + 8)) {
            auto oldest = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                                           [](const GraphEntry &a, const GraphEntry &b) { return a.last_use < b.last_use; });
            CK(cudaDeviceSynchronize());
            if (oldest->exec) cudaGraphExecDestroy(oldest->exec);
            if (oldest->graph) cudaGraphDestroy(oldest->graph);
            if (oldest->small) cudaFree(oldest->small);
            ctx->graphs.erase(oldest);
        }
        GraphEntry ne;
        ne.key = key;
        CK(cudaMalloc(&ne.small, S.small.size()));
        CK(cudaMemcpy(ne.small, S.small.data(), S.small.size(), cudaMemcpyHostToDevice));
        // capture on the context's own stream, then replay on the caller's
        CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        int kernels = 0;
        const int rc = enqueue(ctx, S, mode, ctx->cap_stream, ne.small, ctx->scratch_ev[0], ctx->scratch_ev[1], true,
                               kernels);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(ctx->cap_stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            cudaFree(ne.small);
            return rc;
        }
        if (ec != cudaSuccess) {
            cudaFree(ne.small);
            return cuda_fail(ctx, ec, "cudaStreamEndCapture");
        }
        ne.kernels = kernels;
        // the two event-record nodes, in capture order
        size_t n_nodes = 0;
        CK(cudaGraphGetNodes(graph, nullptr, &n_nodes));
        std::vector<cudaGraphNode_t> nodes(n_nodes);
        CK(cudaGraphGetNodes(graph, nodes.data(), &n_nodes));
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType t;
            CK(cudaGraphNodeGetType(nd, &t));
            if (t == cudaGraphNodeTypeEventRecord) {
                cudaEvent_t ev;
                CK(cudaGraphEventRecordNodeGetEvent(nd, &ev));
                if (ev == ctx->scratch_ev[0]) ne.ev_node[0] = nd;
                if (ev == ctx->scratch_ev[1]) ne.ev_node[1] = nd;
            }
        }
        const cudaError_t ei = cudaGraphInstantiate(&ne.exec, graph, 0);
        if (ei != cudaSuccess) {
            cudaGraphDestroy(graph);
            cudaFree(ne.small);
            return cuda_fail(ctx, ei, "cudaGraphInstantiate");
        }
        ne.graph = graph;
        ctx->graphs.push_back(std::move(ne));
        g = &ctx->graphs.back();
    }
    g->last_use = ++ctx->use_clock;
    cudaEvent_t e0 = slot >= 0 ? ctx->ev[2 * slot] : ctx->scratch_ev[0];
    cudaEvent_t e1 = slot >= 0 ? ctx->ev[2 * slot + 1] : ctx->scratch_ev[1];
    if (g->ev_node[0]) CK(cudaGraphExecEventRecordNodeSetEvent(g->exec, g->ev_node[0], e0));
    if (g->ev_node[1]) CK(cudaGraphExecEventRecordNodeSetEvent(g->exec, g->ev_node[1], e1));
    CK(cudaGraphLaunch(g->exec, s));
    ctx->last_kernels = g->kernels;
    ctx->last_graph = true;
    return TPCF_OK;
}

int run_direct(tpcf_ctx *ctx, const Setup &S, int mode, cudaStream_t s, int slot)
{
    void *small = nullptr;
    int rc;
    if (!S.small.empty() && (rc = upload_small(ctx, S, s, &small))) return rc;
    int kernels = 0;
    rc = enqueue(ctx, S, mode, s, small, slot >= 0 ? ctx->ev[2 * slot] : nullptr,
                 slot >= 0 ? ctx->ev[2 * slot + 1] : nullptr, false, kernels);
    if (rc) return rc;
    ctx->last_kernels = kernels;
    ctx->last_graph = false;
    return TPCF_OK;
}

// Autotuner: time candidate (subdivision, unit size) pairs on a few mocks.
// Autotuner: times one batched count of the first few mocks per candidate
// (at least 6, and all the mocks of a workload under 2e6 points).
// Stage 1: pair counter (both, when the context leaves the choice to the
// library) x mesh subdivision {2, 3, 4} x unit size {64, 128} (the direct
// counter's unit is fixed at 64 a-points).  Stage 2, for the winner: fewer
// blocks per SM than fit (the persistent grid's occupancy).  Each candidate
// is timed twice (six times when a run takes under 2 ms) and its fastest run
// kept.
int autotune(tpcf_ctx *ctx, const tpcf_mock *mocks, int n_mock, const tpcf_binning *binning, unsigned terms,
             int64_t *dd, int64_t *dr, int64_t *rr, cudaStream_t s, Tuned &best)
{
    // at least 6 mocks, more while they hold under 2e6 points in all (a tiny
    // workload is timed whole: its launch latency and tail depend on its size)
    int n_try = std::min(n_mock, 6);
    {
        double pts = 0;
        for (int m = 0; m < n_mock; m++) {
            const tpcf_mock &mk = mocks[m];
            if (terms & (TPCF_DD | TPCF_DR)) pts += (double)std::max<int64_t>(0, mk.n_d);
            if ((terms & (TPCF_DR | TPCF_RR)) && mk.rand_offsets && mk.M >= 1) pts += (double)mk.rand_offsets[mk.M];
            if (pts > 2e6) break;
            n_try = std::max(n_try, m + 1);
        }
    }
    static const int subdivs[] = {2, 3, 4};
    static const int chunks[] = {64, 128};
    std::vector<int> kernels;
    if (ctx->kernel_pref == TPCF_KERNEL_AUTO) kernels = {TPCF_KERNEL_GENERAL, TPCF_KERNEL_DIRECT};
    else kernels = {ctx->kernel_pref};
    cudaEvent_t t0, t1;
    CK(cudaEventCreate(&t0));
    CK(cudaEventCreate(&t1));
    float best_ms = 1e30f;
    int rc = TPCF_OK;
    int best_occ = 0;
    // time candidate c; rc != 0 stops the search, a mesh or counter that does not fit is skipped
    auto trial = [&](const Tuned &c, int &occ_out) -> float {
        Setup S;
        if ((rc = prepare(ctx, mocks, n_try, binning, terms, dd, dr, rr, TPCF_BATCHED, c, S))) {
            if (rc == TPCF_ERR_RANGE) rc = TPCF_OK;   // mesh not possible at this subdivision
            return 1e30f;
        }
        if (c.kernel == TPCF_KERNEL_DIRECT && !S.direct) return 1e30f;   // the general counter's timing is its own
        occ_out = S.blocks / std::max(1, ctx->n_sm);
        float ms = 1e30f;
        // two runs, six when they are short (launch latency makes those noisy)
        for (int rep = 0; rep < (rep >= 2 && ms < 2.0f ? 6 : 2) && rc == TPCF_OK; rep++) {
            cudaError_t e = cudaEventRecord(t0, s);
            if (e == cudaSuccess) rc = run_direct(ctx, S, TPCF_BATCHED, s, -1);
            if (e == cudaSuccess && rc == TPCF_OK) e = cudaEventRecord(t1, s);
            if (e == cudaSuccess && rc == TPCF_OK) e = cudaEventSynchronize(t1);
            float x = 0;
            if (e == cudaSuccess && rc == TPCF_OK) e = cudaEventElapsedTime(&x, t0, t1);
            if (e != cudaSuccess) rc = cuda_fail(ctx, e, "autotune timing");
            ms = std::min(ms, x);
        }
        return ms;
    };
    for (int kern : kernels)
        for (int sd : subdivs)
            for (int ch : chunks) {
                if (kern == TPCF_KERNEL_DIRECT && ch != chunks[0]) continue;
                Tuned c;
                c.subdiv = sd;
                c.chunk = ch;
                c.kernel = kern;
                int occ = 0;
                const float ms = trial(c, occ);
                if (rc) goto done;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = c;
                    best_occ = occ;
                }
            }
    for (int bps = best_occ - 1; bps >= 1 && bps >= best_occ - 2; bps--) {
        Tuned c = best;
        c.bps = bps;
        int occ = 0;
        const float ms = trial(c, occ);
        if (rc) goto done;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
done:
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    return rc;
}

std::string tune_key(tpcf_ctx *ctx, const tpcf_mock *mocks, int n_mock, const tpcf_binning *b, unsigned terms)
{
    std::string k;
    auto put = [&](const void *p, size_t n) { k.append((const char *)p, n); };
    put(&b->geometry, sizeof(int));
    put(&b->box_L, sizeof(double));
    put(&b->los, sizeof(int));
    put(&b->n_s, sizeof(int));
    put(&b->n_mu, sizeof(int));
    put(b->s_edges, sizeof(double) * (b->n_s + 1));
    put(&terms, sizeof(terms));
    put(&ctx->device, sizeof(ctx->device));
    k.append(ctx->device_id);
    put(&ctx->kernel_pref, sizeof(ctx->kernel_pref));
    // size class: log2 of the mean catalogue size, and of the number of mocks
    // (a call of a few mocks fills the GPU differently from one of many)
    double pts = 0;
    for (int m = 0; m < n_mock; m++) pts += (double)mocks[m].n_d;
    const int cls = n_mock > 0 ? (int)std::log2(1.0 + pts / n_mock) : 0;
    const int mcls = (int)std::log2(1.0 + (double)std::max(0, n_mock));
    put(&cls, sizeof(cls));
    put(&mcls, sizeof(mcls));
    return k;
}

}  // namespace

namespace tpcf {
namespace detail {

void release_graphs(tpcf_ctx *ctx)
{
    for (GraphEntry &e : ctx->graphs) {
        if (e.exec) cudaGraphExecDestroy(e.exec);
        if (e.graph) cudaGraphDestroy(e.graph);
        if (e.small) cudaFree(e.small);
    }
    ctx->graphs.clear();
}

}  // namespace detail
}  // namespace tpcf

namespace {

// TPCF_HOST_INPUT: the mocks' position arrays are host memory.
// check_host_mocks checks their fields and returns the bytes each mock
// stages; stage_host_mocks copies mocks [0, n_mock) into the workspace
// buffer `name` on stream s (one copy per run of arrays that follow one
// another in host memory) and dm receives them with the staged device
// pointers.
int check_host_mocks(tpcf_ctx *ctx, const tpcf_mock *mocks, int n_mock, unsigned terms, std::vector<size_t> &bytes)
{
    if (n_mock < 0 || (n_mock > 0 && !mocks)) return fail(ctx, TPCF_ERR_ARG, "mocks is NULL");
    const bool need_d = terms & (TPCF_DD | TPCF_DR);
    const bool need_r = terms & (TPCF_DR | TPCF_RR);
    bytes.assign(n_mock, 0);
    for (int m = 0; m < n_mock; m++) {
        const tpcf_mock &mk = mocks[m];
        if (need_d) {
            if (mk.n_d < 0) return fail(ctx, TPCF_ERR_ARG, "n_d < 0");
            if (mk.n_d > 0 && !mk.data_xyz == !mk.data_u32)
                return fail(ctx, TPCF_ERR_ARG, "give exactly one of data_xyz / data_u32");
            if (mk.n_d > 0) bytes[m] += (size_t)mk.n_d * (mk.data_xyz ? 24 : 12);
        }
        if (need_r) {
            if (mk.M < 1 || !mk.rand_offsets || mk.rand_offsets[0] != 0)
                return fail(ctx, TPCF_ERR_ARG, "M >= 1 and rand_offsets starting at 0 are required");
            if (mk.M != mocks[0].M) return fail(ctx, TPCF_ERR_ARG, "all mocks need the same M");
            for (int i = 0; i < mk.M; i++)
                if (mk.rand_offsets[i + 1] < mk.rand_offsets[i])
                    return fail(ctx, TPCF_ERR_ARG, "rand_offsets must be non-decreasing");
            const int64_t nr = mk.rand_offsets[mk.M];
            if (nr > 0 && !mk.rand_xyz == !mk.rand_u32)
                return fail(ctx, TPCF_ERR_ARG, "give exactly one of rand_xyz / rand_u32");
            if (nr > 0) bytes[m] += (size_t)nr * (mk.rand_xyz ? 24 : 12);
        }
    }
    return TPCF_OK;
}

int stage_host_mocks(tpcf_ctx *ctx, const tpcf_mock *mocks, int n_mock, unsigned terms, const char *name,
                     cudaStream_t s, std::vector<tpcf_mock> &dm)
{
    const bool need_d = terms & (TPCF_DD | TPCF_DR);
    const bool need_r = terms & (TPCF_DR | TPCF_RR);
    auto al256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    dm.assign(mocks, mocks + n_mock);
    // every array to stage, in order; arrays that follow one another in host
    // memory are copied as one run (one copy for a caller's single buffer)
    struct Item {
        const char *src;
        size_t bytes, align;
        const void **field;   // the staged mock's pointer to redirect
    };
    std::vector<Item> items;
    for (int m = 0; m < n_mock; m++) {
        tpcf_mock &mk = dm[m];
        if (need_d && mk.n_d > 0) {
            if (mk.data_xyz) items.push_back({(const char *)mk.data_xyz, (size_t)mk.n_d * 24, 8, (const void **)&mk.data_xyz});
            else items.push_back({(const char *)mk.data_u32, (size_t)mk.n_d * 12, 4, (const void **)&mk.data_u32});
        }
        if (need_r && mk.rand_offsets[mk.M] > 0) {
            const size_t nr = (size_t)mk.rand_offsets[mk.M];
            if (mk.rand_xyz) items.push_back({(const char *)mk.rand_xyz, nr * 24, 8, (const void **)&mk.rand_xyz});
            else items.push_back({(const char *)mk.rand_u32, nr * 12, 4, (const void **)&mk.rand_u32});
        }
    }
    if (items.empty()) return TPCF_OK;
    // device layout: run r starts on a 256-byte boundary; an array inside a
    // run keeps its host offset from the run's start
    std::vector<size_t> dev_off(items.size());
    std::vector<size_t> run_first;   // index of each run's first item
    size_t cursor = 0, run_dev = 0;
    const char *run_src = nullptr, *run_end = nullptr;
    for (size_t k = 0; k < items.size(); k++) {
        const Item &it = items[k];
        const bool joins = run_src && it.src == run_end && (run_dev + (size_t)(it.src - run_src)) % it.align == 0;
        if (!joins) {
            run_dev = al256(cursor);
            run_src = it.src;
            run_first.push_back(k);
        }
        dev_off[k] = run_dev + (size_t)(it.src - run_src);
        run_end = it.src + it.bytes;
        cursor = dev_off[k] + it.bytes;
    }
    void *buf = nullptr;
    int rc;
    if ((rc = ensure(ctx, name, cursor, &buf))) return rc;
    char *dev = (char *)buf;
    for (size_t r = 0; r < run_first.size(); r++) {
        const size_t k0 = run_first[r], k1 = (r + 1 < run_first.size()) ? run_first[r + 1] : items.size();
        const Item &a = items[k0], &b = items[k1 - 1];
        CK(cudaMemcpyAsync(dev + dev_off[k0], a.src, (size_t)(b.src + b.bytes - a.src), cudaMemcpyHostToDevice, s));
    }
    for (size_t k = 0; k < items.size(); k++) *items[k].field = dev + dev_off[k];
    return TPCF_OK;
}

// A batched host-input count in G groups of consecutive mocks (G >= 2):
// group g is staged into workspace buffer g mod 2 on the context's copy
// stream while group g - 1 is counted on the call's stream, so only the first
// group's copy adds to the call's time.  Each group is a whole batched count
// (plan, mesh, one pair-count launch) of its mocks with the configuration
// cfg, writing its rows of dd, dr, rr; every count is exact, so the result
// equals that of one batched call.  The launch counters of the groups are
// summed for tpcf_last_count_info.
int count_host_grouped(tpcf_ctx *ctx, const tpcf_mock *mocks, int n_mock, const tpcf_binning *binning,
                       unsigned terms, int64_t *dd, int64_t *dr, int64_t *rr, const Tuned &cfg,
                       const std::vector<size_t> &bytes, int G, cudaStream_t s)
{
    cudaStream_t cs = ctx->copy_stream;
    cudaEvent_t *ev = ctx->pipe_ev.data();
    // group boundaries by staged bytes, every group non-empty: the first group
    // takes half a share and the others one each, since only the first copy is
    // not hidden behind a count
    size_t total = 0;
    for (size_t b : bytes) total += b;
    std::vector<int> first(G + 1, n_mock);
    first[0] = 0;
    {
        size_t acc = 0;
        int g = 1;
        for (int m = 0; m < n_mock && g < G; m++) {
            acc += bytes[m];
            // boundary g at (g - 1/2) / (G - 1/2) of the bytes
            if ((double)acc * (2.0 * G - 1.0) >= (double)total * (2.0 * g - 1.0) && m + 1 < n_mock)
                first[g++] = m + 1;
        }
        G = g;
        first[G] = n_mock;
    }
    const bool need_r = terms & (TPCF_DR | TPCF_RR);
    const size_t nbin = (size_t)binning->n_s * (size_t)binning->n_mu;
    const size_t M = need_r ? (size_t)mocks[0].M : 0;
    void *accp = nullptr;
    int rc;
    if ((rc = ensure(ctx, "stats_acc", 8 * sizeof(unsigned long long), &accp))) return rc;
    unsigned long long *acc = (unsigned long long *)accp;
    // the copies start after the call's earlier work on s and after the
    // previous grouped call (which may still read the staging buffers)
    CK(cudaEventRecord(ev[0], s));
    CK(cudaStreamWaitEvent(cs, ev[0], 0));
    CK(cudaStreamWaitEvent(cs, ev[1], 0));
    std::vector<tpcf_mock> staged;
    Setup S;
    for (int g = 0; g < G; g++) {
        const int m0 = first[g], n = first[g + 1] - first[g];
        if (g >= 2) CK(cudaStreamWaitEvent(cs, ev[3 + 2 * (g - 2)], 0));   // buffer g mod 2 read by group g - 2
        const int st = ctx->timing ? event_pair(ctx->stage_ev, ctx->n_stage_timed) : -1;
        if (st >= 0) CK(cudaEventRecord(ctx->stage_ev[2 * st], cs));
        if ((rc = stage_host_mocks(ctx, mocks + m0, n, terms, (g & 1) ? "hostin1" : "hostin0", cs, staged)))
            return rc;
        if (st >= 0) {
            CK(cudaEventRecord(ctx->stage_ev[2 * st + 1], cs));
            ctx->n_stage_timed++;
        }
        CK(cudaEventRecord(ev[2 + 2 * g], cs));
        CK(cudaStreamWaitEvent(s, ev[2 + 2 * g], 0));
        S = Setup();
        if ((rc = prepare(ctx, staged.data(), n, binning, terms, dd ? dd + (size_t)m0 * nbin : nullptr,
                          dr ? dr + (size_t)m0 * M * nbin : nullptr, rr ? rr + (size_t)m0 * M * nbin : nullptr,
                          TPCF_BATCHED, cfg, S)))
            return rc;
        const int slot = timing_slot(ctx);
        if (ctx->use_graphs && S.NT > 0 && !S.terms.empty())
            rc = run_graph(ctx, S, TPCF_BATCHED, s, slot);
        else
            rc = run_direct(ctx, S, TPCF_BATCHED, s, slot);
        if (rc) return rc;
        if (slot >= 0) ctx->n_timed++;
        CK(launch_stats_accum(ctx->stats, acc, g == 0, s));
        CK(cudaEventRecord(ev[3 + 2 * g], s));
    }
    CK(cudaMemcpyAsync(ctx->stats_host, acc, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(ev[1], s));
    ctx->last_subdiv = cfg.subdiv;
    ctx->last_nc = S.pl.prm.n_c;
    ctx->last_chunk = S.chunk;
    ctx->last_blocks = S.blocks;
    ctx->last_direct = S.direct;
    ctx->last_launches = G;
    return TPCF_OK;
}

}  // namespace

extern "C" int tpcf_count(tpcf_ctx *ctx, const tpcf_mock *mocks, int n_mock, const tpcf_binning *binning,
                          unsigned terms, int64_t *dd, int64_t *dr, int64_t *rr, int mode, void *stream)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (ctx->fail_count_at > 0 && ++ctx->n_count == ctx->fail_count_at)
        return cuda_fail(ctx, cudaErrorLaunchFailure, "tpcf_count (TPCF_TEST_FAIL_COUNT)");
    cudaStream_t s = (cudaStream_t)stream;
    // timing: the call's whole span on its stream, and the host-input copy
    const int call_slot = ctx->timing ? event_pair(ctx->call_ev, ctx->n_call_timed) : -1;
    if (call_slot >= 0) CK(cudaEventRecord(ctx->call_ev[2 * call_slot], s));
    std::vector<tpcf_mock> staged;
    if (mode & TPCF_HOST_INPUT) {
        mode &= ~TPCF_HOST_INPUT;
        if (mode != TPCF_BATCHED && mode != TPCF_PER_LAUNCH) return fail(ctx, TPCF_ERR_ARG, "bad mode");
        if ((rc = validate_binning(ctx, binning))) return rc;
        if (terms == 0 || (terms & ~7u)) return fail(ctx, TPCF_ERR_ARG, "terms must be a non-empty mask of DD|DR|RR");
        std::vector<size_t> bytes;
        if ((rc = check_host_mocks(ctx, mocks, n_mock, terms, bytes))) return rc;
        // a batched call whose configuration is already known (pinned, untuned
        // or in the tune cache) and that stages at least two groups' worth of
        // positions runs in groups, each copy overlapping the previous group's
        // count; otherwise everything is staged, then counted (and tuned)
        size_t total = 0;
        for (size_t b : bytes) total += b;
        const size_t gb = (size_t)ctx->group_kb << 10;
        const int G = gb ? (int)std::min<size_t>({(size_t)PIPE_GROUPS_MAX, total / gb, (size_t)n_mock}) : 1;
        if (mode == TPCF_BATCHED && G >= 2) {
            Tuned cfg;
            bool known = true;
            if (ctx->subdiv_pin) {
                cfg.subdiv = ctx->subdiv_pin;
            } else if (ctx->autotune) {
                auto it = ctx->tune_cache.find(tune_key(ctx, mocks, n_mock, binning, terms));
                if (it == ctx->tune_cache.end()) known = false;
                else cfg = it->second;
            }
            if (known) {
                if ((rc = count_host_grouped(ctx, mocks, n_mock, binning, terms, dd, dr, rr, cfg, bytes, G, s)))
                    return rc;
                CK(cudaEventRecord(ctx->done, s));
                if (call_slot >= 0) {
                    CK(cudaEventRecord(ctx->call_ev[2 * call_slot + 1], s));
                    ctx->n_call_timed++;
                }
                return TPCF_OK;
            }
        }
        const int st = ctx->timing ? event_pair(ctx->stage_ev, ctx->n_stage_timed) : -1;
        if (st >= 0) CK(cudaEventRecord(ctx->stage_ev[2 * st], s));
        if ((rc = stage_host_mocks(ctx, mocks, n_mock, terms, "hostin", s, staged))) return rc;
        if (st >= 0) {
            CK(cudaEventRecord(ctx->stage_ev[2 * st + 1], s));
            ctx->n_stage_timed++;
        }
        mocks = staged.data();
    }
    // shape-level validation first, so that tuning never sees a bad call
    if ((rc = validate_binning(ctx, binning))) return rc;
    Tuned cfg;
    if (ctx->subdiv_pin) {
        cfg.subdiv = ctx->subdiv_pin;
    } else if (ctx->autotune && mode == TPCF_PER_LAUNCH && n_mock > 0) {
        // the per-launch path runs the configuration tuned for the batched one, if any
        auto it = ctx->tune_cache.find(tune_key(ctx, mocks, n_mock, binning, terms));
        if (it != ctx->tune_cache.end()) cfg = it->second;
    } else if (ctx->autotune && mode == TPCF_BATCHED && n_mock > 0) {
        const std::string tk = tune_key(ctx, mocks, n_mock, binning, terms);
        auto it = ctx->tune_cache.find(tk);
        if (it == ctx->tune_cache.end()) {
            Setup probe;
            if ((rc = prepare(ctx, mocks, n_mock, binning, terms, dd, dr, rr, mode, cfg, probe)))
                return rc;
            Tuned t;
            if ((rc = autotune(ctx, mocks, n_mock, binning, terms, dd, dr, rr, s, t))) return rc;
            it = ctx->tune_cache.emplace(tk, t).first;
        }
        cfg = it->second;
    }
    Setup S;
    if ((rc = prepare(ctx, mocks, n_mock, binning, terms, dd, dr, rr, mode, cfg, S))) return rc;
    ctx->last_subdiv = cfg.subdiv;
    ctx->last_nc = S.pl.prm.n_c;
    ctx->last_chunk = S.chunk;
    ctx->last_blocks = S.blocks;
    ctx->last_direct = S.direct;
    ctx->last_launches = S.terms.empty() || S.NT == 0 ? 0 : (mode == TPCF_BATCHED ? 1 : (int)S.terms.size());
    const int slot = timing_slot(ctx);
    if (mode == TPCF_BATCHED && ctx->use_graphs && S.NT > 0 && !S.terms.empty())
        rc = run_graph(ctx, S, mode, s, slot);
    else
        rc = run_direct(ctx, S, mode, s, slot);
    if (rc) return rc;
    if (slot >= 0) ctx->n_timed++;
    CK(cudaEventRecord(ctx->done, s));
    if (call_slot >= 0) {
        CK(cudaEventRecord(ctx->call_ev[2 * call_slot + 1], s));
        ctx->n_call_timed++;
    }
    return TPCF_OK;
}
