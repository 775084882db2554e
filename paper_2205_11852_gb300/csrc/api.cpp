// C ABI of libtpcf: context, argument validation, workspace, and the three
// stages tpcf_count (Sect. 2.1 pair counts), tpcf_ls (split Landy-Szalay,
// Sect. 2.1) and tpcf_lc_cov (Eqs. bruteforce, R1R2, LCdef).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "ctx.h"

using namespace tpcf;

namespace tpcf {
namespace detail {

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
        if (ctx->fail_alloc_at > 0 && ++ctx->n_alloc == ctx->fail_alloc_at)
            return fail(ctx, TPCF_ERR_NOMEM, std::string("device allocation of ") + name +
                                                 " failed (TPCF_TEST_FAIL_ALLOC)");
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

GramOpts gram_opts(const tpcf_ctx *ctx)
{
    GramOpts o;
    o.n_sm = ctx->n_sm;
    o.wait_limit = ctx->gram_wait_limit;
    o.test_skip_mma = ctx->test_skip_mma;
    return o;
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
        return fail(ctx, TPCF_ERR_ARG, "n_mu must be >= 1 with n_s * n_mu <= 65536");
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

}  // namespace detail
}  // namespace tpcf

using namespace tpcf::detail;

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
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->scratch_ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->scratch_ev[1]);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
    for (int k = 0; k < 2 + 2 * tpcf::PIPE_GROUPS_MAX && e == cudaSuccess; k++) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) ctx->pipe_ev.push_back(ev);
    }
    if (e == cudaSuccess) e = cudaMalloc(&ctx->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->stats, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->stats_host, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(ctx->status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->stats, 0, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaGetLastError();
        tpcf_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? TPCF_ERR_NOMEM : TPCF_ERR_CUDA;
    }
    std::memset(ctx->stats_host, 0, 8 * sizeof(unsigned long long));
    {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, cuda_device) == cudaSuccess)
            ctx->device_id = std::string(prop.name) + "/" + std::to_string(prop.multiProcessorCount) + "/" +
                             std::to_string(prop.major) + "." + std::to_string(prop.minor);
        cudaGetLastError();
    }
    if (const char *v = std::getenv("TPCF_TEST_FAIL_ALLOC")) ctx->fail_alloc_at = std::atoll(v);
    if (const char *v = std::getenv("TPCF_TEST_FAIL_COUNT")) ctx->fail_count_at = std::atoll(v);
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
    release_graphs(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    for (cudaEvent_t e : ctx->pipe_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->scratch_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->done) cudaEventDestroy(ctx->done);
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->call_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->stage_ev) cudaEventDestroy(e);
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
    ctx->n_call_timed = 0;
    ctx->n_stage_timed = 0;
    return TPCF_OK;
}

int tpcf_set_cell_subdiv(tpcf_ctx *ctx, int subdiv)
{
    if (!ctx) return TPCF_ERR_ARG;
    if (subdiv < 0 || subdiv > 4) return fail(ctx, TPCF_ERR_ARG, "subdiv must be in 0..4");
    ctx->subdiv_pin = subdiv;
    return TPCF_OK;
}

int tpcf_set_option(tpcf_ctx *ctx, int option, int value)
{
    if (!ctx) return TPCF_ERR_ARG;
    switch (option) {
    case TPCF_OPT_GRAPHS: ctx->use_graphs = value != 0; break;
    case TPCF_OPT_AUTOTUNE: ctx->autotune = value != 0; break;
    case TPCF_OPT_KERNEL:
        if (value != TPCF_KERNEL_AUTO && value != TPCF_KERNEL_DIRECT && value != TPCF_KERNEL_GENERAL)
            return fail(ctx, TPCF_ERR_ARG, "TPCF_OPT_KERNEL takes TPCF_KERNEL_AUTO, _DIRECT or _GENERAL");
        ctx->kernel_pref = value;
        break;
    case TPCF_OPT_WAIT_LIMIT:
        if (value < 0) return fail(ctx, TPCF_ERR_ARG, "TPCF_OPT_WAIT_LIMIT must be >= 0");
        ctx->gram_wait_limit = value;
        break;
    case TPCF_OPT_TEST_SKIP_MMA: ctx->test_skip_mma = value != 0; break;
    case TPCF_OPT_HOST_GROUP_KB:
        if (value < 0) return fail(ctx, TPCF_ERR_ARG, "TPCF_OPT_HOST_GROUP_KB must be >= 0");
        ctx->group_kb = value;
        break;
    default: return fail(ctx, TPCF_ERR_ARG, "unknown option");
    }
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
    {
        const unsigned long long *st = ctx->stats_host;
        const unsigned long long t0 = ~st[4], span = st[5] > t0 ? st[5] - t0 : 0ull;
        info->idle_frac = (ctx->last_launches == 1 && st[7] > 0 && span > 0 && st[4] != 0)
                              ? 1.0 - (double)st[6] / ((double)st[7] * (double)span)
                              : -1.0;
    }
    info->n_paircount_launches = ctx->last_launches;
    info->cell_subdiv = ctx->last_subdiv;
    info->cells_per_axis = ctx->last_nc;
    info->n_kernels = ctx->last_kernels;
    info->unit_chunk = ctx->last_chunk;
    info->graph_replay = ctx->last_graph ? 1 : 0;
    info->pair_kernel = ctx->last_direct ? TPCF_KERNEL_DIRECT : TPCF_KERNEL_GENERAL;
    info->pair_blocks = ctx->last_blocks;
    double total = 0.0;
    for (int i = 0; i < ctx->n_timed; i++) {
        float ms = 0;
        CK(cudaEventSynchronize(ctx->ev[2 * i + 1]));
        CK(cudaEventElapsedTime(&ms, ctx->ev[2 * i], ctx->ev[2 * i + 1]));
        total += ms;
    }
    info->paircount_ms = total;
    info->timed_calls = ctx->n_timed;
    auto span_sum = [&](const std::vector<cudaEvent_t> &ev, int n, double &out) -> cudaError_t {
        out = 0.0;
        for (int i = 0; i < n; i++) {
            float ms = 0;
            cudaError_t e = cudaEventSynchronize(ev[2 * i + 1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
            if (e != cudaSuccess) return e;
            out += ms;
        }
        return cudaSuccess;
    };
    CK(span_sum(ctx->call_ev, ctx->n_call_timed, info->call_ms));
    CK(span_sum(ctx->stage_ev, ctx->n_stage_timed, info->stage_ms));
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
        const int ns = fp64_splits(n_mock, nbin, 3);
        void *w;
        if ((rc = ensure(ctx, "lc_work", fp64_work_elems(n_mock, nbin, 3, ns) * 8, &w))) return rc;
        CK(launch_lc_fp64_split(xi_a1, xi_a2, xi_b, n_mock, nbin, (double *)w, ns, M_a, M, C_lc, Ca, Cb, A, B, s));
        return TPCF_OK;
    }
    if (precision == TPCF_TF32X3 || precision == TPCF_BF16X3) {
        const size_t bytes = lc_split_work_bytes(n_mock, nbin, precision, ctx->n_sm);
        void *w;
        if ((rc = ensure(ctx, "lc_split_work", bytes, &w))) return rc;
        cudaError_t e = launch_lc_split(xi_a1, xi_a2, xi_b, n_mock, nbin, precision, w, bytes, M_a, M, C_lc, Ca,
                                        Cb, A, B, ctx->status, gram_opts(ctx), s);
        if (e == cudaErrorNotSupported) return fail(ctx, TPCF_ERR_ARG, "split-precision covariance unavailable");
        CK(e);
        return TPCF_OK;
    }
    return fail(ctx, TPCF_ERR_ARG, "bad precision");
}

int tpcf_sample_cov(tpcf_ctx *ctx, const double *xi, int n_mock, int nbin, int precision, double *C, void *stream)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (!xi || !C) return fail(ctx, TPCF_ERR_ARG, "NULL argument");
    if (n_mock < 2) return fail(ctx, TPCF_ERR_ARG, "n_mock must be >= 2");
    if (nbin < 1 || nbin > 65536) return fail(ctx, TPCF_ERR_ARG, "bad nbin");
    if (precision == TPCF_FP64) {
        const int ns = fp64_splits(n_mock, nbin, 1);
        void *w;
        if ((rc = ensure(ctx, "lc_work", fp64_work_elems(n_mock, nbin, 1, ns) * 8, &w))) return rc;
        CK(launch_cov_fp64(xi, n_mock, nbin, (double *)w, C, s, ns));
        return TPCF_OK;
    }
    if (precision == TPCF_TF32X3 || precision == TPCF_BF16X3) {
        const size_t bytes = lc_split_work_bytes(n_mock, nbin, precision, ctx->n_sm, 1);
        void *w;
        if ((rc = ensure(ctx, "lc_split_work", bytes, &w))) return rc;
        cudaError_t e = launch_cov_split(xi, n_mock, nbin, precision, w, bytes, C, ctx->status, gram_opts(ctx), s);
        if (e == cudaErrorNotSupported) return fail(ctx, TPCF_ERR_ARG, "split-precision covariance unavailable");
        CK(e);
        return TPCF_OK;
    }
    return fail(ctx, TPCF_ERR_ARG, "bad precision");
}

int tpcf_rebin_counts(tpcf_ctx *ctx, const int64_t *in, int64_t rows, int n_s, int n_mu, int f_s, int f_mu,
                      int64_t *out, void *stream)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (rows < 0 || n_s < 1 || n_mu < 1 || f_s < 1 || f_mu < 1 || n_s % f_s || n_mu % f_mu)
        return fail(ctx, TPCF_ERR_ARG, "bad re-binning shape (factors must divide n_s and n_mu)");
    if (rows > 0 && (!in || !out)) return fail(ctx, TPCF_ERR_ARG, "NULL argument");
    CK(launch_rebin((const long long *)in, rows, n_s, n_mu, f_s, f_mu, (long long *)out, (cudaStream_t)stream));
    return TPCF_OK;
}

int tpcf_project(tpcf_ctx *ctx, const double *P, int n_out, int nbin, const double *xi, int n_mock, double *y,
                 void *stream)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (n_out < 1 || nbin < 1 || n_mock < 0 || n_mock > 65535 * 32) return fail(ctx, TPCF_ERR_ARG, "bad shape");
    if (n_mock > 0 && (!P || !xi || !y)) return fail(ctx, TPCF_ERR_ARG, "NULL argument");
    CK(launch_project(P, n_out, nbin, xi, n_mock, y, (cudaStream_t)stream));
    return TPCF_OK;
}

int tpcf_covcov_var(tpcf_ctx *ctx, const double *A, const double *B, int nbin, int M_a, double M, int n_mock,
                    double *var, void *stream)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!A || !var) return fail(ctx, TPCF_ERR_ARG, "NULL argument");
    if (nbin < 1 || nbin > 65536 || n_mock < 2) return fail(ctx, TPCF_ERR_ARG, "bad shape");
    if (B && (M_a < 1 || !(M >= (double)M_a))) return fail(ctx, TPCF_ERR_ARG, "need M_a >= 1 and M >= M_a");
    CK(launch_covcov(A, B, nbin, M_a, M, n_mock, var, (cudaStream_t)stream));
    return TPCF_OK;
}

int tpcf_chi2_predict(tpcf_ctx *ctx, const double *A, const double *B, const double *C_ref, int nbin, int M_a,
                      double M, double *chi2_2, void *stream)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!A || !C_ref || !chi2_2) return fail(ctx, TPCF_ERR_ARG, "NULL argument");
    if (nbin < 1 || nbin > 65536) return fail(ctx, TPCF_ERR_ARG, "bad nbin");
    if (B && (M_a < 1 || !(M >= (double)M_a))) return fail(ctx, TPCF_ERR_ARG, "need M_a >= 1 and M >= M_a");
    void *w;
    if ((rc = ensure(ctx, "chi2_work", chi2_work_bytes(), &w))) return rc;
    CK(launch_chi2(0, A, B, C_ref, nbin, M_a, M, (double *)w, chi2_2, (cudaStream_t)stream));
    return TPCF_OK;
}

int tpcf_chi2(tpcf_ctx *ctx, const double *C_est, const double *C_true, const double *C_ref, int nbin, double *chi2,
              void *stream)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!C_est || !C_true || !C_ref || !chi2) return fail(ctx, TPCF_ERR_ARG, "NULL argument");
    if (nbin < 1 || nbin > 65536) return fail(ctx, TPCF_ERR_ARG, "bad nbin");
    void *w;
    if ((rc = ensure(ctx, "chi2_work", chi2_work_bytes(), &w))) return rc;
    CK(launch_chi2(1, C_est, C_true, C_ref, nbin, 1, 2.0, (double *)w, chi2, (cudaStream_t)stream));
    return TPCF_OK;
}

int tpcf_eigvalsh(tpcf_ctx *ctx, const double *C, int n, double *w, void *stream)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!C || !w) return fail(ctx, TPCF_ERR_ARG, "NULL argument");
    if (n < 1 || n > 1024) return fail(ctx, TPCF_ERR_ARG, "eigenvalues need 1 <= n <= 1024");
    void *wk;
    if ((rc = ensure(ctx, "eig_work", eig_work_bytes(n), &wk))) return rc;
    CK(launch_eigvalsh(C, n, (double *)wk, w, (cudaStream_t)stream));
    return TPCF_OK;
}

int tpcf_multipole_matrix(int n_s, int n_mu, const int *ells, int n_ell, double *P)
{
    if (n_s < 1 || n_mu < 1 || n_ell < 1 || !ells || !P) return TPCF_ERR_ARG;
    int lmax = 0;
    for (int i = 0; i < n_ell; i++) {
        if (ells[i] < 0 || ells[i] > 64 || (ells[i] & 1)) return TPCF_ERR_ARG;
        lmax = std::max(lmax, ells[i]);
    }
    // Legendre values P_0 .. P_{lmax+1} at the n_mu + 1 uniform |mu| edges (Bonnet recurrence)
    std::vector<double> leg((size_t)(n_mu + 1) * (lmax + 2));
    for (int j = 0; j <= n_mu; j++) {
        const double x = (double)j / n_mu;
        double *L = &leg[(size_t)j * (lmax + 2)];
        L[0] = 1.0;
        if (lmax + 1 >= 1) L[1] = x;
        for (int n = 1; n + 1 <= lmax + 1; n++) L[n + 1] = ((2.0 * n + 1.0) * x * L[n] - n * L[n - 1]) / (n + 1.0);
    }
    // xi_l(s_k) = (2l+1)/2 int_{-1}^{1} xi P_l dmu = (2l+1) sum_j xi_kj int_{mu_j}^{mu_j+1} P_l dmu (even l),
    // with (2l+1) int P_l = [P_{l+1} - P_{l-1}] for l >= 1 and [mu] for l = 0
    const size_t nbin = (size_t)n_s * n_mu;
    std::fill(P, P + (size_t)n_ell * n_s * nbin, 0.0);
    for (int i = 0; i < n_ell; i++) {
        const int l = ells[i];
        for (int j = 0; j < n_mu; j++) {
            const double *L0 = &leg[(size_t)j * (lmax + 2)], *L1 = &leg[(size_t)(j + 1) * (lmax + 2)];
            const double w = l == 0 ? (double)(j + 1) / n_mu - (double)j / n_mu
                                    : (L1[l + 1] - L0[l + 1]) - (L1[l - 1] - L0[l - 1]);
            for (int k = 0; k < n_s; k++) P[((size_t)i * n_s + k) * nbin + (size_t)k * n_mu + j] = w;
        }
    }
    return TPCF_OK;
}

}  // extern "C"
