// C ABI of libtpcf: context, argument validation, workspace, and the three
// stages tpcf_count (Sect. 2.1 pair counts), tpcf_ls (split Landy-Szalay,
// Sect. 2.1) and tpcf_lc_cov (Eqs. bruteforce, R1R2, LCdef).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "plan.h"

using namespace tpcf;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct PinBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct tpcf_ctx {
    int device = 0;
    int n_sm = 0;
    std::string err;
    bool broken = false;
    // workspace
    std::map<std::string, DevBuf> bufs;
    PinBuf staging;
    cudaEvent_t staging_free = nullptr;   // recorded after the last copy out of `staging`
    bool staging_pending = false;
    int *status = nullptr;                // device status word
    unsigned long long *stats = nullptr;  // device [4]
    unsigned long long *stats_host = nullptr;  // pinned [4]
    // timing: one event pair per timed tpcf_count
    bool timing = false;
    std::vector<cudaEvent_t> ev;          // [2 * k]
    int n_timed = 0;
    cudaEvent_t done = nullptr;           // recorded after the stats copy of the last tpcf_count
    int last_launches = 0;
    int last_kernels = 0;
    // planner
    int subdiv_pin = 0;
    std::map<std::string, int> tune_cache;
    int last_subdiv = 0, last_nc = 0;
    unsigned long long last_units_bound = 0;
};

namespace {

int fail(tpcf_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}

int cuda_fail(tpcf_ctx *c, cudaError_t e, const char *where)
{
    if (c) {
        c->err = std::string(where) + ": " + cudaGetErrorString(e);
        if (e != cudaErrorInvalidValue && e != cudaErrorMemoryAllocation) c->broken = true;
    }
    return e == cudaErrorMemoryAllocation ? TPCF_ERR_NOMEM : TPCF_ERR_CUDA;
}

#define CK(expr)                                          \
    do {                                                  \
        cudaError_t _e = (expr);                          \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, #expr); \
    } while (0)

// device buffer `name` with at least `bytes` bytes (contents not preserved on growth)
int ensure(tpcf_ctx *ctx, const char *name, size_t bytes, void **out)
{
    DevBuf &b = ctx->bufs[name];
    if (b.bytes < bytes) {
        if (b.p) {
            cudaError_t e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaDeviceSynchronize");
            cudaFree(b.p);
            b.p = nullptr;
            b.bytes = 0;
        }
        size_t want = std::max(bytes + bytes / 8, (size_t)256);
        cudaError_t e = cudaMalloc(&b.p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            e = cudaMalloc(&b.p, bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                b.p = nullptr;
                return fail(ctx, TPCF_ERR_NOMEM, std::string("device allocation of ") + name + " failed");
            }
            want = bytes;
        }
        b.bytes = want;
    }
    *out = b.p;
    return TPCF_OK;
}

// pinned staging area for small host->device tables; waits for its previous use
int staging(tpcf_ctx *ctx, size_t bytes, void **out)
{
    if (ctx->staging_pending) {
        cudaError_t e = cudaEventSynchronize(ctx->staging_free);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventSynchronize");
        ctx->staging_pending = false;
    }
    if (ctx->staging.bytes < bytes) {
        if (ctx->staging.p) cudaFreeHost(ctx->staging.p);
        ctx->staging.p = nullptr;
        ctx->staging.bytes = 0;
        size_t want = std::max(bytes * 2, (size_t)(1 << 20));
        cudaError_t e = cudaMallocHost(&ctx->staging.p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, TPCF_ERR_NOMEM, "pinned staging allocation failed");
        }
        ctx->staging.bytes = want;
    }
    *out = ctx->staging.p;
    return TPCF_OK;
}

int staging_done(tpcf_ctx *ctx, cudaStream_t s)
{
    CK(cudaEventRecord(ctx->staging_free, s));
    ctx->staging_pending = true;
    return TPCF_OK;
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

int check_ctx(tpcf_ctx *ctx)
{
    if (!ctx) return TPCF_ERR_ARG;
    if (ctx->broken) return fail(ctx, TPCF_ERR_STATE, "context unusable after an earlier CUDA error: " + ctx->err);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return TPCF_OK;
}

int validate_binning(tpcf_ctx *ctx, const tpcf_binning *b)
{
    if (!b) return fail(ctx, TPCF_ERR_ARG, "binning is NULL");
    if (b->geometry != TPCF_PERIODIC && b->geometry != TPCF_OPEN) return fail(ctx, TPCF_ERR_ARG, "bad geometry");
    if (!(b->box_L > 0) || !std::isfinite(b->box_L)) return fail(ctx, TPCF_ERR_ARG, "box_L must be positive");
    if (b->n_s < 1 || b->n_s > MAX_NS) return fail(ctx, TPCF_ERR_ARG, "n_s must be in [1, 256]");
    if (b->n_mu < 1 || (long long)b->n_s * b->n_mu > MAX_NBIN)
        return fail(ctx, TPCF_ERR_ARG, "n_mu must be >= 1 with n_s * n_mu <= 4096");
    if (!b->s_edges) return fail(ctx, TPCF_ERR_ARG, "s_edges is NULL");
    if (!(b->s_edges[0] >= 0)) return fail(ctx, TPCF_ERR_ARG, "s edges must be >= 0");
    for (int k = 0; k < b->n_s; k++)
        if (!(b->s_edges[k + 1] > b->s_edges[k]) || !std::isfinite(b->s_edges[k + 1]))
            return fail(ctx, TPCF_ERR_ARG, "s edges must be strictly increasing and finite");
    if (b->los != TPCF_LOS_X && b->los != TPCF_LOS_MIDPOINT) return fail(ctx, TPCF_ERR_ARG, "bad line of sight");
    const double smax = b->s_edges[b->n_s];
    if (b->geometry == TPCF_PERIODIC) {
        if (b->n_mu > 1 && b->los != TPCF_LOS_X)
            return fail(ctx, TPCF_ERR_ARG, "periodic geometry supports the x line of sight only");
        if (!(smax * 3.0 <= b->box_L))
            return fail(ctx, TPCF_ERR_RANGE, "periodic geometry needs s_max <= box_L / 3");
    } else {
        for (int c = 0; c < 3; c++)
            if (!std::isfinite(b->origin[c])) return fail(ctx, TPCF_ERR_ARG, "origin must be finite");
        if (b->n_mu > 1 && b->los == TPCF_LOS_MIDPOINT) {
            for (int c = 0; c < 3; c++) {
                if (!std::isfinite(b->observer[c])) return fail(ctx, TPCF_ERR_ARG, "observer must be finite");
                const double t = (b->observer[c] - b->origin[c]) / b->box_L;
                if (!(std::fabs(t) < 4.0)) return fail(ctx, TPCF_ERR_RANGE, "observer too far from the cube");
            }
        }
    }
    return TPCF_OK;
}

// 128-bit width check of the exact mu test (n_mu^2 * D2max * |l|max^2 < 2^127)
int check_mu_width(tpcf_ctx *ctx, const tpcf_binning *b, const CountParams &p)
{
    if (b->n_mu <= 1) return TPCF_OK;
    const long double d2max = (long double)(p.T[b->n_s] - 1);
    long double l2 = 1.0L;
    if (b->los == TPCF_LOS_MIDPOINT) {
        l2 = 0;
        const long double top = (long double)((1ull << 31) - 2);
        for (int c = 0; c < 3; c++) {
            const long double o = (long double)p.obs[c];
            const long double m = std::max(std::fabs(2 * o), std::fabs(top - 2 * o));
            l2 += m * m;
        }
    }
    const long double v = (long double)(b->n_mu * b->n_mu) * d2max * l2;
    if (!(v < std::ldexp(1.0L, 126)))
        return fail(ctx, TPCF_ERR_RANGE, "mu test exceeds the 128-bit range for this geometry");
    return TPCF_OK;
}

}  // namespace

extern "C" {

int tpcf_create(tpcf_ctx **out, int cuda_device)
{
    if (!out) return TPCF_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || cuda_device < 0 || cuda_device >= n) {
        cudaGetLastError();
        return TPCF_ERR_ARG;
    }
    tpcf_ctx *ctx = new tpcf_ctx();
    ctx->device = cuda_device;
    cudaError_t e = cudaSetDevice(cuda_device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, cuda_device);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->staging_free, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->stats, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->stats_host, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(ctx->status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->stats, 0, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaGetLastError();
        tpcf_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? TPCF_ERR_NOMEM : TPCF_ERR_CUDA;
    }
    std::memset(ctx->stats_host, 0, 4 * sizeof(unsigned long long));
    *out = ctx;
    return TPCF_OK;
}

void tpcf_destroy(tpcf_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto &kv : ctx->bufs)
        if (kv.second.p) cudaFree(kv.second.p);
    if (ctx->staging.p) cudaFreeHost(ctx->staging.p);
    if (ctx->staging_free) cudaEventDestroy(ctx->staging_free);
    if (ctx->done) cudaEventDestroy(ctx->done);
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    if (ctx->status) cudaFree(ctx->status);
    if (ctx->stats) cudaFree(ctx->stats);
    if (ctx->stats_host) cudaFreeHost(ctx->stats_host);
    cudaGetLastError();
    delete ctx;
}

const char *tpcf_last_error(const tpcf_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int tpcf_sync(tpcf_ctx *ctx, void *stream)
{
    if (!ctx) return TPCF_ERR_ARG;
    if (ctx->broken) return fail(ctx, TPCF_ERR_STATE, "context unusable after an earlier CUDA error: " + ctx->err);
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    int st = 0;
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(&st, ctx->status, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemset(ctx->status, 0, sizeof(int)));
    if (st & STATUS_RANGE) return fail(ctx, TPCF_ERR_RANGE, "a position lies outside the bounding cube");
    if (st & STATUS_TIMEOUT) return fail(ctx, TPCF_ERR_TIMEOUT, "a bounded device wait gave up");
    if (st & STATUS_EMPTY_BIN) return fail(ctx, TPCF_WARN_EMPTY_BIN, "rr = 0 in some bin: xi is NaN there");
    return TPCF_OK;
}

int tpcf_thresholds(tpcf_ctx *ctx, const tpcf_binning *binning, uint64_t *T_out)
{
    if (!T_out) return fail(ctx, TPCF_ERR_ARG, "T_out is NULL");
    int rc = validate_binning(ctx, binning);
    if (rc) return rc;
    const int bits = binning->geometry == TPCF_PERIODIC ? 32 : 30;
    for (int k = 0; k <= binning->n_s; k++) {
        unsigned long long T;
        if (!exact_threshold(binning->s_edges[k], binning->box_L, bits, T))
            return fail(ctx, TPCF_ERR_RANGE, "separation range exceeds the 64-bit squared-distance range");
        T_out[k] = T;
    }
    return TPCF_OK;
}

int tpcf_set_timing(tpcf_ctx *ctx, int enable)
{
    if (!ctx) return TPCF_ERR_ARG;
    ctx->timing = enable != 0;
    ctx->n_timed = 0;
    return TPCF_OK;
}

int tpcf_set_cell_subdiv(tpcf_ctx *ctx, int subdiv)
{
    if (!ctx) return TPCF_ERR_ARG;
    if (subdiv < 0 || subdiv > 4) return fail(ctx, TPCF_ERR_ARG, "subdiv must be in 0..4");
    ctx->subdiv_pin = subdiv;
    return TPCF_OK;
}

int tpcf_last_count_info(tpcf_ctx *ctx, tpcf_count_info *info)
{
    if (!ctx) return TPCF_ERR_ARG;
    if (!info) return TPCF_OK;
    std::memset(info, 0, sizeof(*info));
    CK(cudaSetDevice(ctx->device));
    CK(cudaEventSynchronize(ctx->done));
    info->n_candidates = (int64_t)ctx->stats_host[0];
    info->n_binned = (int64_t)ctx->stats_host[1];
    info->n_exact = (int64_t)ctx->stats_host[2];
    info->n_units = (int64_t)ctx->stats_host[3];
    info->n_paircount_launches = ctx->last_launches;
    info->cell_subdiv = ctx->last_subdiv;
    info->cells_per_axis = ctx->last_nc;
    info->n_kernels = ctx->last_kernels;
    double total = 0.0;
    for (int i = 0; i < ctx->n_timed; i++) {
        float ms = 0;
        CK(cudaEventSynchronize(ctx->ev[2 * i + 1]));
        CK(cudaEventElapsedTime(&ms, ctx->ev[2 * i], ctx->ev[2 * i + 1]));
        total += ms;
    }
    info->paircount_ms = total;
    info->timed_calls = ctx->n_timed;
    return TPCF_OK;
}

int tpcf_count(tpcf_ctx *ctx, const tpcf_mock *mocks, int n_mock, const tpcf_binning *binning, unsigned terms,
               int64_t *dd, int64_t *dr, int64_t *rr, int mode, void *stream)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
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
    unsigned long long n_total = 0;
    for (int m = 0; m < n_mock; m++) {
        const tpcf_mock &mk = mocks[m];
        if (need_d) {
            if (mk.n_d < 0) return fail(ctx, TPCF_ERR_ARG, "n_d < 0");
            if (mk.n_d > 0 && !mk.data_xyz == !mk.data_u32)
                return fail(ctx, TPCF_ERR_ARG, "give exactly one of data_xyz / data_u32");
            n_total += (unsigned long long)mk.n_d;
        }
        if (need_r) {
            if (mk.M < 1) return fail(ctx, TPCF_ERR_ARG, "M must be >= 1");
            if (M >= 0 && mk.M != M) return fail(ctx, TPCF_ERR_ARG, "all mocks need the same M");
            M = mk.M;
            if (!mk.rand_offsets) return fail(ctx, TPCF_ERR_ARG, "rand_offsets is NULL");
            if (mk.rand_offsets[0] != 0) return fail(ctx, TPCF_ERR_ARG, "rand_offsets[0] must be 0");
            for (int i = 0; i < mk.M; i++)
                if (mk.rand_offsets[i + 1] < mk.rand_offsets[i])
                    return fail(ctx, TPCF_ERR_ARG, "rand_offsets must be non-decreasing");
            const int64_t nr = mk.rand_offsets[mk.M];
            if (nr > 0 && !mk.rand_xyz == !mk.rand_u32)
                return fail(ctx, TPCF_ERR_ARG, "give exactly one of rand_xyz / rand_u32");
            n_total += (unsigned long long)nr;
        }
    }
    if (n_total >= (1ull << 31)) return fail(ctx, TPCF_ERR_RANGE, "more than 2^31 points in one call");
    if (M < 0) M = 0;

    // mesh cap: a few cells per point of the largest catalogue, and the
    // (catalogue x cell) and (term x cell) tables indexable in 32 bits
    unsigned long long max_cat = 0, n_cat_est = 0, n_terms_est = 0;
    for (int m = 0; m < n_mock; m++) {
        if (need_d) { max_cat = std::max<unsigned long long>(max_cat, mocks[m].n_d); n_cat_est++; }
        if (need_r)
            for (int i = 0; i < M; i++) {
                max_cat = std::max<unsigned long long>(max_cat, mocks[m].rand_offsets[i + 1] - mocks[m].rand_offsets[i]);
                n_cat_est++;
            }
        n_terms_est += ((terms & TPCF_DD) ? 1 : 0) + (unsigned long long)M * (((terms & TPCF_DR) ? 1 : 0) + ((terms & TPCF_RR) ? 1 : 0));
    }
    unsigned long long max_cells = std::max<unsigned long long>(64, 4 * max_cat);
    max_cells = std::min<unsigned long long>(max_cells, 1ull << 24);
    const unsigned long long tabs = std::max<unsigned long long>(1, std::max(n_cat_est, n_terms_est));
    max_cells = std::min<unsigned long long>(max_cells, ((1ull << 32) - 2) / tabs);

    // plan (subdivision pinned, or the default)
    int subdiv = ctx->subdiv_pin ? ctx->subdiv_pin : 3;
    Plan pl;
    std::string perr;
    if ((rc = build_plan(*binning, subdiv, max_cells, pl, perr))) return fail(ctx, rc, perr);
    if ((rc = check_mu_width(ctx, binning, pl.prm))) return rc;
    const CountParams &prm = pl.prm;
    ctx->last_subdiv = subdiv;
    ctx->last_nc = prm.n_c;

    // catalogues and terms
    std::vector<Cat> cats;
    std::vector<Term> tlist;
    const int per_mock = (need_d ? 1 : 0) + (need_r ? M : 0);
    uint32_t p0 = 0, max_n = 0;
    for (int m = 0; m < n_mock; m++) {
        const tpcf_mock &mk = mocks[m];
        const int cd = (int)cats.size();
        if (need_d) {
            Cat c;
            c.xyz = mk.data_xyz;
            c.u32 = mk.data_xyz ? nullptr : mk.data_u32;
            c.p0 = p0;
            c.n = (uint32_t)mk.n_d;
            p0 += c.n;
            max_n = std::max(max_n, c.n);
            cats.push_back(c);
        }
        const int cr = (int)cats.size();
        if (need_r) {
            for (int i = 0; i < M; i++) {
                Cat c;
                const int64_t o0 = mk.rand_offsets[i], o1 = mk.rand_offsets[i + 1];
                c.xyz = mk.rand_xyz ? mk.rand_xyz + 3 * o0 : nullptr;
                // pre-quantised randoms: the [3][n_r] array of all subsets; the
                // mesh build reads rows with stride n_r, handled by a copy below
                c.u32 = nullptr;
                c.p0 = p0;
                c.n = (uint32_t)(o1 - o0);
                p0 += c.n;
                max_n = std::max(max_n, c.n);
                cats.push_back(c);
            }
        }
        const int nbin = prm.nbin;
        if (terms & TPCF_DD) tlist.push_back(Term{cd, cd, 1, 0, (long long *)dd + (size_t)m * nbin});
        for (int i = 0; i < M; i++) {
            if (terms & TPCF_DR)
                tlist.push_back(Term{cd, cr + i, 0, 0, (long long *)dr + ((size_t)m * M + i) * nbin});
            if (terms & TPCF_RR)
                tlist.push_back(Term{cr + i, cr + i, 1, 0, (long long *)rr + ((size_t)m * M + i) * nbin});
        }
        (void)per_mock;
    }
    const int n_cat = (int)cats.size();
    const int n_terms = (int)tlist.size();

    // zero the requested outputs
    const size_t nb = (size_t)prm.nbin * sizeof(int64_t);
    if (n_mock > 0) {
        if (terms & TPCF_DD) CK(cudaMemsetAsync(dd, 0, nb * n_mock, s));
        if ((terms & TPCF_DR) && M > 0) CK(cudaMemsetAsync(dr, 0, nb * n_mock * M, s));
        if ((terms & TPCF_RR) && M > 0) CK(cudaMemsetAsync(rr, 0, nb * n_mock * M, s));
    }
    ctx->last_launches = 0;
    ctx->last_kernels = 0;
    if (n_total == 0 || n_terms == 0) {
        CK(cudaMemsetAsync(ctx->stats, 0, 4 * sizeof(unsigned long long), s));
        CK(cudaMemcpyAsync(ctx->stats_host, ctx->stats, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CK(cudaEventRecord(ctx->done, s));
        return TPCF_OK;
    }

    // pre-quantised randoms are given as one [3][n_r] array per mock; gather
    // each subset into a contiguous [3][n] staging region on the device
    const size_t NT = (size_t)n_total;
    const size_t ncc = (size_t)n_cat * prm.n_cells + 1;
    if (ncc >= (1ull << 32)) return fail(ctx, TPCF_ERR_RANGE, "too many catalogues x cells");
    const size_t ntc = (size_t)n_terms * prm.n_cells + 1;
    if (ntc >= (1ull << 32)) return fail(ctx, TPCF_ERR_RANGE, "too many terms x cells");
    // bound on the number of units
    unsigned long long units_bound = 0;
    for (const Term &t : tlist) {
        const unsigned long long n = cats[t.cat_a].n;
        units_bound += n / UNIT_CHUNK + std::min<unsigned long long>(n, prm.n_cells) + 1;
    }

    void *w_uq, *w_keys, *w_us, *w_pf, *w_pcx, *w_cc, *w_cs, *w_tmp, *w_uc, *w_ust, *w_units, *w_small, *w_claim;
    const size_t tmp_n = std::max(scan_tmp_elems(ncc), scan_tmp_elems(ntc));
    if ((rc = ensure(ctx, "uq", 3 * NT * 4, &w_uq))) return rc;
    if ((rc = ensure(ctx, "keys", NT * 4, &w_keys))) return rc;
    if ((rc = ensure(ctx, "us", 3 * NT * 4, &w_us))) return rc;
    if ((rc = ensure(ctx, "pf", NT * 16, &w_pf))) return rc;
    if ((rc = ensure(ctx, "pcx", NT * 2, &w_pcx))) return rc;
    if ((rc = ensure(ctx, "cellcount", ncc * 4, &w_cc))) return rc;
    if ((rc = ensure(ctx, "cellstart", ncc * 4, &w_cs))) return rc;
    if ((rc = ensure(ctx, "scantmp", tmp_n * 4, &w_tmp))) return rc;
    if ((rc = ensure(ctx, "ucount", ntc * 4, &w_uc))) return rc;
    if ((rc = ensure(ctx, "ustart", ntc * 4, &w_ust))) return rc;
    if ((rc = ensure(ctx, "units", units_bound * sizeof(Unit), &w_units))) return rc;
    if ((rc = ensure(ctx, "claim", 256, &w_claim))) return rc;

    // pre-quantised random subsets need a compact [3][n] copy each
    std::vector<std::pair<size_t, size_t>> rq_copies;  // (cat index, mock)
    size_t rq_elems = 0;
    if (need_r) {
        for (int m = 0; m < n_mock; m++)
            if (!mocks[m].rand_xyz && mocks[m].rand_offsets[M] > 0) rq_elems += 3 * (size_t)mocks[m].rand_offsets[M];
    }
    void *w_rq = nullptr;
    if (rq_elems) {
        if ((rc = ensure(ctx, "rq", rq_elems * 4, &w_rq))) return rc;
        size_t off = 0;
        for (int m = 0, ci = 0; m < n_mock; m++) {
            const int cr = ci + (need_d ? 1 : 0);
            ci += per_mock;
            const tpcf_mock &mk = mocks[m];
            if (mk.rand_xyz || mk.rand_offsets[M] == 0) continue;
            const size_t nr = (size_t)mk.rand_offsets[M];
            for (int i = 0; i < M; i++) {
                const size_t o0 = (size_t)mk.rand_offsets[i], n = (size_t)(mk.rand_offsets[i + 1] - mk.rand_offsets[i]);
                uint32_t *dst = (uint32_t *)w_rq + off;
                if (n > 0) {
                    CK(cudaMemcpy2DAsync(dst, n * 4, mk.rand_u32 + o0, nr * 4, n * 4, 3, cudaMemcpyDeviceToDevice, s));
                }
                cats[cr + i].u32 = dst;
                off += 3 * n;
            }
        }
    }

    // small tables through pinned staging: cats | terms | orig | table
    const size_t o_cats = 0;
    const size_t o_terms = al(o_cats + cats.size() * sizeof(Cat));
    const size_t o_orig = al(o_terms + tlist.size() * sizeof(Term));
    const size_t o_tab = al(o_orig + pl.orig.size() * 4);
    const size_t small_bytes = al(o_tab + pl.table.size() * 2);
    if ((rc = ensure(ctx, "small", small_bytes, &w_small))) return rc;
    void *host;
    if ((rc = staging(ctx, small_bytes, &host))) return rc;
    std::memcpy((char *)host + o_cats, cats.data(), cats.size() * sizeof(Cat));
    std::memcpy((char *)host + o_terms, tlist.data(), tlist.size() * sizeof(Term));
    std::memcpy((char *)host + o_orig, pl.orig.data(), pl.orig.size() * 4);
    std::memcpy((char *)host + o_tab, pl.table.data(), pl.table.size() * 2);
    CK(cudaMemcpyAsync(w_small, host, small_bytes, cudaMemcpyHostToDevice, s));
    if ((rc = staging_done(ctx, s))) return rc;
    const Cat *d_cats = (const Cat *)((char *)w_small + o_cats);
    const Term *d_terms = (const Term *)((char *)w_small + o_terms);
    const uint32_t *d_orig = (const uint32_t *)((char *)w_small + o_orig);
    const int16_t *d_tab = (const int16_t *)((char *)w_small + o_tab);

    uint32_t *uq = (uint32_t *)w_uq, *keys = (uint32_t *)w_keys, *us = (uint32_t *)w_us;
    float4 *pf = (float4 *)w_pf;
    uint32_t *cc = (uint32_t *)w_cc, *cs = (uint32_t *)w_cs, *tmp = (uint32_t *)w_tmp;
    uint32_t *uc = (uint32_t *)w_uc, *ust = (uint32_t *)w_ust;
    Unit *units = (Unit *)w_units;

    // mesh build
    CK(cudaMemsetAsync(cc, 0, ncc * 4, s));
    CK(launch_quantize_keys(d_cats, n_cat, max_n, prm, binning->box_L, binning->origin, (uint32_t)NT, uq, keys,
                            cc, ctx->status, s));
    CK(launch_scan_u32(cc, cs, ncc, tmp, tmp_n, s));
    CK(cudaMemsetAsync(cc, 0, ncc * 4, s));
    CK(launch_scatter(d_cats, n_cat, max_n, prm, uq, keys, cs, cc, d_orig, (uint32_t)NT, us, pf, (uint16_t *)w_pcx,
                      s));

    Mesh mesh;
    mesh.pf = pf;
    mesh.pcx = (const uint16_t *)w_pcx;
    mesh.us = us;
    mesh.n_total = (uint32_t)NT;
    mesh.cellstart = cs;
    mesh.orig = d_orig;

    const int warps = 8;
    const int smem = paircount_smem_bytes(prm, warps);
    CK(paircount_set_attrs(prm, smem));
    CK(cudaMemsetAsync(ctx->stats, 0, 4 * sizeof(unsigned long long), s));
    int slot = -1;
    if (ctx->timing && ctx->n_timed < 4096) {
        slot = ctx->n_timed;
        while ((int)ctx->ev.size() < 2 * (slot + 1)) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            ctx->ev.push_back(e);
        }
    }
    // kernels of the mesh build: quantize, 3-kernel scan, scatter
    ctx->last_kernels = 5;
    if (mode == TPCF_BATCHED) {
        // unit list: count, 3-kernel scan, fill
        ctx->last_kernels += 5;
        CK(cudaMemsetAsync(uc + (ntc - 1), 0, 4, s));
        CK(launch_unit_count(d_terms, n_terms, d_cats, prm.n_cells, cs, UNIT_CHUNK, uc, s));
        CK(launch_scan_u32(uc, ust, ntc, tmp, tmp_n, s));
        CK(launch_unit_fill(d_terms, n_terms, d_cats, prm.n_cells, cs, UNIT_CHUNK, ust, units, s));
        CK(cudaMemsetAsync(w_claim, 0, 4, s));
        PairLaunch L;
        L.warps_per_block = warps;
        L.persistent = 1;
        L.term = 0;
        L.smem_bytes = smem;
        L.blocks = ctx->n_sm * paircount_max_blocks_per_sm(prm, warps, smem);
        if (slot >= 0) CK(cudaEventRecord(ctx->ev[2 * slot], s));
        CK(launch_paircount(prm, mesh, d_terms, d_cats, units, ust + (ntc - 1), (unsigned *)w_claim, d_tab,
                            ctx->stats, ctx->status, L, s));
        if (slot >= 0) CK(cudaEventRecord(ctx->ev[2 * slot + 1], s));
        ctx->last_launches = 1;
        ctx->last_kernels += 1;
        CK(cudaMemsetAsync(ctx->stats + 3, 0, 8, s));
        CK(cudaMemcpyAsync(ctx->stats + 3, ust + (ntc - 1), 4, cudaMemcpyDeviceToDevice, s));
    } else {
        if (slot >= 0) CK(cudaEventRecord(ctx->ev[2 * slot], s));
        for (int t = 0; t < n_terms; t++) {
            PairLaunch L;
            L.warps_per_block = warps;
            L.persistent = 0;
            L.term = t;
            L.smem_bytes = smem;
            L.blocks = prm.n_cells;
            CK(launch_paircount(prm, mesh, d_terms, d_cats, units, nullptr, nullptr, d_tab, ctx->stats,
                                ctx->status, L, s));
        }
        if (slot >= 0) CK(cudaEventRecord(ctx->ev[2 * slot + 1], s));
        ctx->last_launches = n_terms;
        ctx->last_kernels += n_terms;
    }
    if (slot >= 0) ctx->n_timed++;
    CK(cudaMemcpyAsync(ctx->stats_host, ctx->stats, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(ctx->done, s));
    return TPCF_OK;
}

int tpcf_ls(tpcf_ctx *ctx, const int64_t *dd, const int64_t *dr, const int64_t *rr, const int64_t *n_d,
            const int64_t *n_r, int n_mock, int M, int nbin, const int *sel, int n_sel, double *xi, void *stream)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_mock < 0 || M < 1 || nbin < 1 || n_sel < 1 || n_sel > M) return fail(ctx, TPCF_ERR_ARG, "bad sizes");
    if (!dd || !dr || !rr || !n_d || !n_r || !sel || !xi) return fail(ctx, TPCF_ERR_ARG, "NULL argument");
    for (int i = 0; i < n_sel; i++)
        if (sel[i] < 0 || sel[i] >= M) return fail(ctx, TPCF_ERR_ARG, "sel index out of range");
    for (int m = 0; m < n_mock; m++) {
        if (n_d[m] < 2) return fail(ctx, TPCF_ERR_ARG, "N_d must be >= 2");
        for (int i = 0; i < n_sel; i++)
            if (n_r[(size_t)m * M + sel[i]] < 2) return fail(ctx, TPCF_ERR_ARG, "N_r,i must be >= 2");
    }
    if (n_mock == 0) return TPCF_OK;
    const size_t o_n = 0;
    const size_t o_sel = al((size_t)n_mock * (1 + M) * 8);
    const size_t bytes = al(o_sel + (size_t)n_sel * 4);
    void *w, *host;
    if ((rc = ensure(ctx, "ls_small", bytes, &w))) return rc;
    if ((rc = staging(ctx, bytes, &host))) return rc;
    long long *hn = (long long *)((char *)host + o_n);
    for (int m = 0; m < n_mock; m++) {
        hn[(size_t)m * (1 + M)] = n_d[m];
        for (int i = 0; i < M; i++) hn[(size_t)m * (1 + M) + 1 + i] = n_r[(size_t)m * M + i];
    }
    std::memcpy((char *)host + o_sel, sel, (size_t)n_sel * 4);
    CK(cudaMemcpyAsync(w, host, bytes, cudaMemcpyHostToDevice, s));
    if ((rc = staging_done(ctx, s))) return rc;
    CK(launch_ls((const long long *)dd, (const long long *)dr, (const long long *)rr,
                 (const long long *)((char *)w + o_n), (const int *)((char *)w + o_sel), n_sel, n_mock, M, nbin,
                 xi, ctx->status, s));
    return TPCF_OK;
}

int tpcf_lc_cov(tpcf_ctx *ctx, const double *xi_a1, const double *xi_a2, const double *xi_b, int n_mock, int nbin,
                int M_a, double M, int precision, double *C_lc, double *Ca, double *Cb, double *A, double *B,
                void *stream)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (!xi_a1 || !xi_a2 || !xi_b || !C_lc) return fail(ctx, TPCF_ERR_ARG, "NULL argument");
    if (n_mock < 2) return fail(ctx, TPCF_ERR_ARG, "n_mock must be >= 2");
    if (nbin < 1 || nbin > 65536) return fail(ctx, TPCF_ERR_ARG, "bad nbin");
    if (M_a < 1) return fail(ctx, TPCF_ERR_ARG, "M_a must be >= 1");
    if (!(M >= (double)M_a)) return fail(ctx, TPCF_ERR_ARG, "M must be >= M_a (or +inf)");
    if (precision == TPCF_FP64) {
        const size_t elems = 3 * (size_t)n_mock * nbin + 3 * (size_t)nbin + 3 * (size_t)nbin * nbin;
        void *w;
        if ((rc = ensure(ctx, "lc_work", elems * 8, &w))) return rc;
        CK(launch_lc_fp64(xi_a1, xi_a2, xi_b, n_mock, nbin, (double *)w, M_a, M, C_lc, Ca, Cb, A, B, s));
        return TPCF_OK;
    }
    if (precision == TPCF_TF32X3 || precision == TPCF_BF16X3) {
        const size_t bytes = lc_split_work_bytes(n_mock, nbin, precision);
        void *w;
        if ((rc = ensure(ctx, "lc_split_work", bytes, &w))) return rc;
        cudaError_t e = launch_lc_split(xi_a1, xi_a2, xi_b, n_mock, nbin, precision, w, bytes, M_a, M, C_lc, Ca,
                                        Cb, A, B, ctx->status, s);
        if (e == cudaErrorNotSupported) return fail(ctx, TPCF_ERR_ARG, "split-precision covariance unavailable");
        CK(e);
        return TPCF_OK;
    }
    return fail(ctx, TPCF_ERR_ARG, "bad precision");
}

}  // extern "C"
