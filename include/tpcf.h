/*
 * tpcf.h -- C ABI of the GB300 pair-count / Landy-Szalay / linear-construction
 * covariance library.
 *
 * The library computes, for many mock catalogues at once, the three stages of
 * the linear-construction (LC) covariance of the two-point correlation
 * function:
 *   1. tpcf_count  -- binned pair counts DD, DR_i, RR_i in (s, mu)   (Sect. 2.1, Sect. 4.3)
 *   2. tpcf_ls     -- the split Landy-Szalay estimator                (Sect. 2.1)
 *   3. tpcf_lc_cov -- sample covariances and their linear combination
 *                     (Eqs. bruteforce, R1R2, LCdef)                   (Sect. 2.2-2.3)
 *
 * Conventions shared by every entry point
 *   - All array arguments named as device arrays are CUDA device pointers
 *     owned by the caller; the library never frees or retains them past the
 *     call's stream work.  Host arrays are read during the call only.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Calls validate their arguments synchronously, then enqueue the
 *     GPU work on `stream` and return without waiting.  Errors found on the
 *     device (e.g. a position outside the bounding cube) are reported by
 *     tpcf_sync().
 *   - Return codes: TPCF_OK (0), a positive warning, or a negative error.
 *     After an error, tpcf_last_error() gives a one-line description.
 *   - A context is bound to one CUDA device and is not thread-safe: use one
 *     context per host thread.
 */
#ifndef TPCF_H
#define TPCF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define TPCF_OK               0
#define TPCF_WARN_EMPTY_BIN   1   /* some rr = 0: those xi entries are NaN */
#define TPCF_ERR_ARG         -1   /* invalid argument (NULL pointer, bad size, bad enum) */
#define TPCF_ERR_RANGE       -2   /* geometry/binning outside the exact-integer range, or a
                                     position outside the bounding cube (open geometry) */
#define TPCF_ERR_CUDA        -3   /* a CUDA runtime call failed */
#define TPCF_ERR_NOMEM       -4   /* device or pinned-host allocation failed */
#define TPCF_ERR_TIMEOUT     -5   /* a bounded device wait gave up */
#define TPCF_ERR_STATE       -6   /* context unusable after an earlier CUDA error */

/* ---- enums ------------------------------------------------------------- */
#define TPCF_PERIODIC   0         /* periodic cube of side box_L, minimum-image separations */
#define TPCF_OPEN       1         /* non-periodic; all points inside the cube [origin, origin+box_L)^3 */

#define TPCF_LOS_X        0       /* plane-parallel line of sight along x (Sect. 4.1) */
#define TPCF_LOS_MIDPOINT 1       /* line of sight from the observer to the pair midpoint (open only) */

#define TPCF_DD  1u               /* term mask bits for tpcf_count */
#define TPCF_DR  2u
#define TPCF_RR  4u

#define TPCF_BATCHED     0        /* all mocks and terms in one persistent launch (default) */
#define TPCF_PER_LAUNCH  1        /* one kernel launch per (mock, term, subset): baseline */
#define TPCF_HOST_INPUT  2        /* OR into mode: the mocks' position arrays are host memory */

#define TPCF_FP64    0            /* covariance arithmetic entirely in float64 */
#define TPCF_TF32X3  1            /* Gram products on tensor cores, 3-term TF32 split, FP32 accumulate */
#define TPCF_BF16X3  2            /* Gram products on tensor cores, 3-piece BF16 split, FP32 accumulate */

typedef struct tpcf_ctx tpcf_ctx;

/*
 * Create a context on CUDA device `cuda_device`.  The context owns the
 * workspace (grown on demand, reused across calls), the autotuner cache and
 * a device status word.  *out is set to NULL on failure.
 * Returns TPCF_OK, TPCF_ERR_ARG, TPCF_ERR_CUDA or TPCF_ERR_NOMEM.
 */
int tpcf_create(tpcf_ctx **out, int cuda_device);

/* Release every resource of the context (waits for its outstanding work). NULL is a no-op. */
void tpcf_destroy(tpcf_ctx *ctx);

/*
 * Wait for all work the context enqueued on `stream`, then read and clear
 * the device status word.  Returns TPCF_OK, TPCF_WARN_EMPTY_BIN (from
 * tpcf_ls), TPCF_ERR_RANGE (a position outside the bounding cube),
 * TPCF_ERR_TIMEOUT, or TPCF_ERR_CUDA.
 */
int tpcf_sync(tpcf_ctx *ctx, void *stream);

/* One-line description of the last error or warning on this context ("" if none). */
const char *tpcf_last_error(const tpcf_ctx *ctx);

/*
 * Geometry and binning (Sect. 4.3: bins in separation s and in mu, the
 * cosine of the angle between the line of sight and the pair separation).
 *   s bins   : half-open [s_edges[k], s_edges[k+1]), k = 0..n_s-1, edges strictly
 *              increasing and >= 0 (host array of n_s+1 doubles).
 *   mu bins  : n_mu uniform bins of |mu| on [0, 1], the top bin closed; n_mu = 1 gives
 *              s-only counts.  mu = 0 for coincident points.
 *   histogram index of (k, j) is k * n_mu + j (s-major); nbin = n_s * n_mu.
 * Positions are quantised to integer grid coordinates (2^32 per box side for
 * TPCF_PERIODIC, 2^30 per bounding-cube side for TPCF_OPEN) and every bin
 * decision is exact on those integers.  Limits: n_s <= 256, nbin <= 65536
 * and the block histogram within shared memory (about 44 000 bins on a
 * 227 KB device; above about 400 bins fewer blocks share an SM);
 * periodic boxes need s_max <= box_L / 3 and the x line of sight.
 */
typedef struct {
    int     geometry;        /* TPCF_PERIODIC or TPCF_OPEN */
    double  box_L;           /* periodic box side, or bounding-cube side */
    double  origin[3];       /* lower corner of the bounding cube (open); ignored for periodic */
    int     los;             /* TPCF_LOS_X or TPCF_LOS_MIDPOINT */
    double  observer[3];     /* observer position for TPCF_LOS_MIDPOINT */
    int     n_s;             /* number of s bins */
    const double *s_edges;   /* host, n_s + 1 values */
    int     n_mu;            /* number of |mu| bins, >= 1 */
} tpcf_binning;

/*
 * One mock: a data catalogue D and M random sub-catalogues R_1..R_M (the
 * split random catalogue of Sect. 2.1).  Give each catalogue either as
 * float64 positions (`*_xyz`, device, row-major [n][3]) or as pre-quantised
 * grid coordinates (`*_u32`, device, structure-of-arrays [3][n]); the other
 * pointer is NULL.  The random points are one array; subset i is the index
 * range [rand_offsets[i], rand_offsets[i+1]) with rand_offsets a HOST array
 * of M+1 non-decreasing values starting at 0.
 */
typedef struct {
    const double   *data_xyz;
    const uint32_t *data_u32;
    int64_t         n_d;
    const double   *rand_xyz;
    const uint32_t *rand_u32;
    const int64_t  *rand_offsets;   /* host, M + 1 */
    int             M;
} tpcf_mock;

/*
 * Binned pair counts of every mock (Sect. 2.1 DD, DR_i, RR_i; Sect. 4.3 bins).
 *   DD   : unordered pairs of distinct points of D
 *   DR_i : all pairs (a in D, b in R_i)
 *   RR_i : unordered pairs of distinct points of R_i (pairs across
 *          sub-catalogues are not counted: the split estimator)
 * Outputs (device, int64, overwritten for the requested terms):
 *   dd[n_mock][nbin], dr[n_mock][M][nbin], rr[n_mock][M][nbin]
 * Every mock must have the same M when TPCF_DR or TPCF_RR is requested.
 * `terms` is a mask of TPCF_DD | TPCF_DR | TPCF_RR; unrequested outputs may
 * be NULL.  `mode` selects TPCF_BATCHED or TPCF_PER_LAUNCH; both give
 * identical counts.  With TPCF_HOST_INPUT or-ed into `mode`, data_xyz,
 * data_u32, rand_xyz and rand_u32 are HOST arrays (same layouts): the call
 * copies them into the context's device workspace on `stream` before
 * counting (asynchronously from pinned memory, so they must stay unchanged
 * until the stream has passed the call; pageable memory is copied before the
 * call returns).  A batched host-input call whose configuration is already
 * known (subdivision pinned, autotuning off, or the shape tuned by an earlier
 * batched call) and whose positions fill at least two groups of
 * TPCF_OPT_HOST_GROUP_KB runs in up to 8 groups of consecutive mocks: each
 * group's copy (on a stream of the context's own) overlaps the count of the
 * previous group, so only the first copy adds to the call's time; the counts
 * are those of one batched call.  The outputs stay device memory.  Returns TPCF_OK or a negative error (nothing enqueued);
 * TPCF_ERR_RANGE when the binning cannot be counted exactly on the integer
 * grid: a squared separation beyond 64 bits, a periodic s_max above L/3, or
 * (n_mu > 1) n_mu^2 D2_max |l|^2_max >= 2^126 for the exact mu test, where
 * |l|^2_max = 1 on the x line of sight and, on the midpoint line of sight,
 * the largest |u_a + u_b - 2 u_obs|^2 over the cube (open grid units), or a
 * block histogram (4 nbin bytes) that does not fit in the device's shared
 * memory beside the queues.
 */
int tpcf_count(tpcf_ctx *ctx, const tpcf_mock *mocks, int n_mock, const tpcf_binning *binning,
               unsigned terms, int64_t *dd, int64_t *dr, int64_t *rr, int mode, void *stream);

/*
 * Split Landy-Szalay estimator of Sect. 2.1 for each mock, over the random
 * sub-catalogues listed in sel[0..n_sel) (host, indices into 0..M-1):
 *   dd = DD / (N_d (N_d - 1) / 2)
 *   dr = (1/n_sel) sum_{i in sel} DR_i / (N_d N_r,i)
 *   rr = (1/n_sel) sum_{i in sel} RR_i / (N_r,i (N_r,i - 1) / 2)
 *   xi = (dd - 2 dr) / rr + 1                     (float64; NaN where rr = 0)
 * With N_r,i = N_d these are the paper's normalisations.  sel = {0} gives
 * xi(D, R_1); sel = {0, 1} gives xi(D, R_1 u R_2) with the split RR.
 * Inputs: dd[n_mock][nbin], dr/rr[n_mock][M][nbin] (device int64);
 * n_d[n_mock], n_r[n_mock][M] (host).  Output xi[n_mock][nbin] (device float64).
 * Needs N_d >= 2 and N_r,i >= 2.  A bin with rr = 0 makes tpcf_sync return
 * TPCF_WARN_EMPTY_BIN.
 */
int tpcf_ls(tpcf_ctx *ctx, const int64_t *dd, const int64_t *dr, const int64_t *rr,
            const int64_t *n_d, const int64_t *n_r, int n_mock, int M, int nbin,
            const int *sel, int n_sel, double *xi, void *stream);

/*
 * Linear-construction covariance, Eqs. (R1R2) and (LCdef):
 *   C^a  = (Cov[xi(D,R1)] + Cov[xi(D,R2)]) / 2,  C^b = Cov[xi(D, R1 u R2)]
 *   A    = 2 C^b - C^a,   B = 2 M_a (C^a - C^b),   C^LC = A + B / M
 * with Cov the sample covariance over the n_mock mocks, Eq. (bruteforce):
 * 1/(N-1) sum (xi - mean)(xi - mean)^T.  M = +INFINITY gives C^LC = A.
 * Inputs xi_a1, xi_a2, xi_b: device float64 [n_mock][nbin].
 * Outputs: C_lc required; Ca, Cb, A, B may be NULL; all device float64 [nbin][nbin].
 * `precision`: TPCF_FP64 (all float64), TPCF_TF32X3 or TPCF_BF16X3 (the
 * centred Gram products on tensor cores in split precision with FP32
 * accumulation over K-chunks and a float64 sum; means and the final
 * combination stay float64).  Needs n_mock >= 2, M_a >= 1, M >= M_a.
 */
int tpcf_lc_cov(tpcf_ctx *ctx, const double *xi_a1, const double *xi_a2, const double *xi_b,
                int n_mock, int nbin, int M_a, double M, int precision,
                double *C_lc, double *Ca, double *Cb, double *A, double *B, void *stream);

/*
 * Sample covariance of one correlation-function variant over the mocks,
 * Eq. (bruteforce): C = 1/(N-1) sum_m (xi_m - mean)(xi_m - mean)^T.  This is
 * the brute-force (Smp) estimate the LC covariance is compared with: xi from
 * tpcf_ls over all M random subsets (Sect. 2.1, Sect. 2.2).
 * Input xi: device float64 [n_mock][nbin]; output C: device float64
 * [nbin][nbin] (caller-owned, fully overwritten).  `precision` as in
 * tpcf_lc_cov.  Needs n_mock >= 2 and 1 <= nbin <= 65536 (TPCF_ERR_ARG
 * otherwise); TPCF_ERR_NOMEM if the workspace cannot grow.  Enqueued on
 * `stream`; returns without waiting.
 */
int tpcf_sample_cov(tpcf_ctx *ctx, const double *xi, int n_mock, int nbin, int precision, double *C,
                    void *stream);

/*
 * Linear maps applied before the covariance.  The LC construction holds for
 * any linear function of the correlation function (Sect. 2.3): multipoles,
 * the projected function, wider bins.  Apply the same map to xi_a1, xi_a2
 * and xi_b, then call tpcf_lc_cov; the result is P C^LC P^T.
 */

/*
 * Re-binning of pair counts into wider bins (Sect. 4.3: bins combined into
 * wider ones, and the 1-D function from counts co-added over mu):
 *   out[r][k'][j'] = sum_{k = f_s k'}^{f_s k' + f_s - 1} sum_{j = f_mu j'}^{f_mu j' + f_mu - 1} in[r][k][j]
 * `in`: device int64 [rows][n_s][n_mu] (any stack of DD, DR_i, RR_i
 * histograms, s-major); `out`: device int64 [rows][n_s/f_s][n_mu/f_mu].
 * With half-open s bins and uniform |mu| bins the result equals counting
 * with the merged edges directly.  f_s must divide n_s and f_mu divide n_mu
 * (TPCF_ERR_ARG otherwise).  Enqueued on `stream`.
 */
int tpcf_rebin_counts(tpcf_ctx *ctx, const int64_t *in, int64_t rows, int n_s, int n_mu, int f_s, int f_mu,
                      int64_t *out, void *stream);

/*
 * y[m][o] = sum_b P[o][b] xi[m][b] in float64: a linear map of every mock's
 * xi row.  P: device float64 [n_out][nbin]; xi: device float64
 * [n_mock][nbin]; y: device float64 [n_mock][n_out] (caller-owned, not
 * aliasing xi).  Needs n_out, nbin >= 1 and 0 <= n_mock <= 2097120
 * (TPCF_ERR_ARG otherwise).  Enqueued on `stream`.
 */
int tpcf_project(tpcf_ctx *ctx, const double *P, int n_out, int nbin, const double *xi, int n_mock, double *y,
                 void *stream);

/*
 * Host-side: the matrix of the Legendre multipoles of Sect. 4.3,
 *   xi_l(s) = (2l+1)/2 int_{-1}^{1} xi(s, mu) P_l(mu) dmu,
 * for xi binned in n_s s bins x n_mu uniform |mu| bins on [0, 1] (s-major).
 * Because xi depends on |mu| and l is even, the integral is twice the one
 * on [0, 1], and over a bin (2l+1) int P_l = [P_{l+1} - P_{l-1}] (l >= 1),
 * [mu] (l = 0).  Output P: HOST float64 [n_ell * n_s][n_s * n_mu], row
 * (i, k) = multipole ells[i] at s bin k.  Each ells[i] must be even and in
 * [0, 64] (odd multipoles vanish for |mu| bins); TPCF_ERR_ARG otherwise.
 */
int tpcf_multipole_matrix(int n_s, int n_mu, const int *ells, int n_ell, double *P);

/*
 * Accuracy of a covariance estimate (Sect. 3), for Gaussian xi.
 *
 * tpcf_covcov_var: var[i][j] = Var(C_ij), the diagonal k = i, l = j of the
 * covariance of covariance.
 *   B != NULL -- LC covariance, Eq. (covcov_fast):
 *     (N-1) Var = D_ii D_jj + D_ij^2 + (1/(2 M_a) - 1/M)^2 (B_ii B_jj + B_ij^2)
 *     with A, B the LC components (Eq. CABdef; their estimates stand in for
 *     the ensemble values, Sect. 3.3) and D = A + B / (2 M_a).  The paper
 *     prints D = A + B / M_a; the form here follows from Eq. (covcov)
 *     applied to Eq. (Cfastx) term by term, and is the one for which the two
 *     forms (covcov_fast) and (covcov_fast2) agree and LC equals the sample
 *     covariance at M = 2 M_a.
 *   B == NULL -- sample covariance, Eq. (covcov_brute): A is the covariance C,
 *     (N-1) Var = C_ii C_jj + C_ij^2.
 * A, B: device float64 [nbin][nbin]; var: device float64 [nbin][nbin];
 * n_mock = N >= 2.  With B: M_a >= 1 and M >= M_a (M = +INFINITY allowed).
 *
 * tpcf_chi2_predict: *chi2_2 (device float64 scalar) = the predicted
 * <chi^2_2> of Sect. 5.3, (1/N_bin^2) sum_ij (N-1) Var(C_ij) / (R_ii R_jj),
 * with (A, B) as in tpcf_covcov_var (B = NULL: sample covariance) and R =
 * C_ref the normalising covariance.  <chi^2_N> = <chi^2_2> / (N - 1).
 *
 * tpcf_chi2: *chi2 (device scalar) = Eq. (chi2),
 *   (1/N_bin^2) sum_ij (C_est,ij - C_true,ij)^2 / (C_ref,ii C_ref,jj).
 *
 * tpcf_eigvalsh: the eigenvalues w[n] (device float64, ascending) of the
 * symmetric matrix C[n][n] (device float64; only symmetric input is
 * meaningful), for checking that an LC covariance is positive definite
 * before it is inverted (Sect. 3.4).  Householder reduction to tridiagonal
 * form (one cluster of 8 blocks, the matrix in their shared memory up to
 * n = 472, in device memory above), then 32-way multisection on Sturm counts
 * taken on the continuants of T - x I (one warp per eigenvalue); absolute
 * accuracy about n * 1e-16 * max|w|.
 * Needs 1 <= n <= 1024 (TPCF_ERR_ARG otherwise).
 *
 * All four enqueue on `stream` and return without waiting; they share the
 * context's workspace, so calls on different streams must not overlap.
 */
int tpcf_covcov_var(tpcf_ctx *ctx, const double *A, const double *B, int nbin, int M_a, double M, int n_mock,
                    double *var, void *stream);
int tpcf_chi2_predict(tpcf_ctx *ctx, const double *A, const double *B, const double *C_ref, int nbin, int M_a,
                      double M, double *chi2_2, void *stream);
int tpcf_chi2(tpcf_ctx *ctx, const double *C_est, const double *C_true, const double *C_ref, int nbin, double *chi2,
              void *stream);
int tpcf_eigvalsh(tpcf_ctx *ctx, const double *C, int n, double *w, void *stream);

/*
 * tpcf_lc_cov_noalloc -- tpcf_lc_cov in TPCF_FP64 that allocates nothing.
 * (A library addition; the paper has no counterpart.)
 *
 * For callers that cannot allocate device memory while they run: services
 * that reserve all of their GPU memory at start-up and treat any later
 * cudaMalloc as a failure, and code that must not trigger the implicit device
 * synchronisation that cudaMalloc / cudaFree can cause.  It needs no context
 * (creating one allocates).  Inputs, outputs and their meaning are those of
 * tpcf_lc_cov; the result equals tpcf_lc_cov(..., TPCF_FP64, ...) up to
 * float64 rounding.
 *
 * Its scratch is one fixed array of 2^21 doubles (16 MiB) compiled into the
 * library; every GPU that loads the library holds it until the process exits.
 * Limit: 3*n_mock*nbin + 3*nbin + 3*nbin*nbin <= 2^21, else TPCF_ERR_RANGE
 * (e.g. nbin = 400 with n_mock <= 1347).
 * Every call looks up the array's device address in the current device's
 * context (so it stays valid after cudaDeviceReset); the first call on a
 * device may load the library's device code, so make it before any stream
 * capture.  All calls share the one array: calls whose GPU work overlaps (on
 * different streams, or from different threads) race and give wrong results,
 * so serialise them.  The array keeps the last call's contents; nothing in it
 * needs to start at zero.  Work is enqueued on `stream` (cudaStream_t, NULL =
 * legacy default stream) on the current CUDA device; the call returns without
 * waiting.  Returns TPCF_OK, TPCF_ERR_ARG, TPCF_ERR_RANGE or TPCF_ERR_CUDA.
 */
int tpcf_lc_cov_noalloc(const double *xi_a1, const double *xi_a2, const double *xi_b, int n_mock, int nbin,
                        int M_a, double M, double *C_lc, double *Ca, double *Cb, double *A, double *B,
                        void *stream);

/*
 * The exact integer s-bin thresholds tpcf_count uses (host only, no GPU work):
 * T[k] = ceil(s_edges[k]^2 q^2) with q = 2^32 / box_L (periodic) or
 * 2^30 / box_L (open), so that a pair with squared grid separation D2 lies
 * in s-bin k iff T[k] <= D2 < T[k+1] (Sect. 4.3 bins, half-open).
 * T_out: host array of n_s + 1 values.  Returns TPCF_OK, TPCF_ERR_ARG or
 * TPCF_ERR_RANGE (edges beyond the 63-bit range or the geometry's limits).
 * `ctx` may be NULL.
 */
int tpcf_thresholds(tpcf_ctx *ctx, const tpcf_binning *binning, uint64_t *T_out);

/*
 * Work statistics of the last tpcf_count on this context, valid after
 * tpcf_sync: candidate pairs tested by the pair-count kernel(s), pairs
 * that fell in a bin, pairs that needed the exact integer recheck, the
 * number of work units, the number of kernels the call launched, and the
 * mesh it used.  When timing is enabled, paircount_ms is the total device
 * time of the pair-count kernels of every tpcf_count since timing was
 * (re-)enabled, over timed_calls calls, measured with CUDA events recorded
 * on the launch stream around those kernels.
 */
typedef struct {
    int64_t n_candidates;
    int64_t n_binned;
    int64_t n_exact;
    int64_t n_units;
    double  paircount_ms;
    int     n_paircount_launches;   /* 1 for a batched call, one per term per launch mode, one per group of a
                                       grouped host-input call (whose counters are the groups' sums) */
    int     cell_subdiv;      /* cells per s_max along an axis */
    int     cells_per_axis;
    int     n_kernels;        /* kernels launched by the last tpcf_count */
    int     timed_calls;      /* pair-count spans accumulated in paircount_ms (a grouped call adds one per group) */
    int     unit_chunk;       /* a-points per work unit, chosen by the autotuner */
    int     graph_replay;     /* 1: the batched launch was a replay of a captured CUDA graph */
    int     pair_kernel;      /* TPCF_KERNEL_DIRECT or TPCF_KERNEL_GENERAL: the pair counter that ran */
    int     pair_blocks;      /* blocks of the persistent pair-count grid (SMs x blocks per SM) */
    double  idle_frac;        /* one batched launch: share of warp time between the first warp's start and
                                 the last warp's end that warps spent finished (the last-wave tail);
                                 -1 when the call made several launches or none */
    double  call_ms;          /* with timing: the timed calls' whole spans on their streams (events at the
                                 call's first and last enqueued operation), summed */
    double  stage_ms;         /* with timing: the host-input copies of the timed TPCF_HOST_INPUT calls, summed */
} tpcf_count_info;

int tpcf_last_count_info(tpcf_ctx *ctx, tpcf_count_info *info);

/*
 * Enable (1) or disable (0) CUDA-event timing of the pair-count kernels.
 * Enabling resets the accumulated time; at most 4096 calls are accumulated.
 */
int tpcf_set_timing(tpcf_ctx *ctx, int enable);

/*
 * Pin the chaining-mesh subdivision (cells per s_max along an axis, 1..4),
 * or 0 to let the autotuner choose.  For tests and benchmarks.
 */
int tpcf_set_cell_subdiv(tpcf_ctx *ctx, int subdiv);

/*
 * Options of the batched pair count (both on by default):
 *   TPCF_OPT_GRAPHS   -- capture the batched tpcf_count (mesh build, work list
 *                        and the persistent pair-count launch) as a CUDA graph
 *                        on first use and replay it while the plan, buffers and
 *                        outputs of the call stay the same.  The first call of
 *                        a new shape must not itself be under stream capture.
 *   TPCF_OPT_AUTOTUNE -- on the first batched call of a new workload shape,
 *                        time candidates on a few of the mocks (all of them
 *                        below 2e6 points) and keep the fastest: the pair
 *                        counter (both, under TPCF_KERNEL_AUTO), the mesh
 *                        subdivision {2, 3, 4} and the work-unit size
 *                        {64, 128}, then fewer blocks per SM for the winner
 *                        (cached per context, keyed by the binning, the
 *                        classes log2 of the mean catalogue size and of the
 *                        number of mocks, and the device's name, SM count and
 *                        compute capability).  A pinned subdivision disables
 *                        it.
 *   TPCF_OPT_KERNEL   -- which pair counter runs: TPCF_KERNEL_DIRECT (the
 *                        direct counter wherever the binning suits it -- s bins
 *                        linear from 0 with the x line of sight or s only, and
 *                        a histogram that fits shared memory with its copies --
 *                        else the general one), TPCF_KERNEL_GENERAL (always the
 *                        general counter) or TPCF_KERNEL_AUTO (the default: the
 *                        autotuner times both and keeps the faster; without a
 *                        tuned entry, the general counter).  The per-launch
 *                        mode runs the configuration tuned for the batched
 *                        call of the same shape.  Both counters give identical
 *                        counts.
 * and of the split-precision covariances (tpcf_lc_cov, tpcf_sample_cov with
 * TPCF_TF32X3 / TPCF_BF16X3):
 *   TPCF_OPT_WAIT_LIMIT    -- bound, in polls of about 64 ns, of the Gram
 *                        kernel's wait for its tensor-core products before it
 *                        reads them (0, the default: 2^26).  A wait that runs
 *                        out makes the next tpcf_sync return TPCF_ERR_TIMEOUT;
 *                        the kernel frees its tensor memory and returns.  The
 *                        waits for bulk copies keep the built-in bound.
 *   TPCF_OPT_HOST_GROUP_KB -- smallest group, in KiB of staged positions, of
 *                        a grouped host-input count (see tpcf_count; default
 *                        262144, i.e. 256 MiB; 0 never groups).
 *   TPCF_OPT_TEST_SKIP_MMA -- tests only: when non-zero, one CTA of the Gram
 *                        kernel waits for its operand copies and then issues
 *                        no tensor-core product, so that the wait above runs
 *                        out with nothing in flight (the result is garbage and
 *                        the status TPCF_ERR_TIMEOUT).  0 by default.
 * Returns TPCF_OK or TPCF_ERR_ARG.
 *
 * Test hooks read from the environment when a context is created:
 * TPCF_TEST_FAIL_ALLOC=n makes the context's n-th device allocation fail
 * (the call returns TPCF_ERR_NOMEM with nothing enqueued; the context stays
 * usable), and TPCF_TEST_FAIL_COUNT=n makes the n-th tpcf_count return
 * TPCF_ERR_CUDA as if a launch had failed, before it enqueues anything (the
 * context is then unusable, as after a real CUDA error).
 */
#define TPCF_OPT_GRAPHS    1
#define TPCF_OPT_AUTOTUNE  2
#define TPCF_OPT_KERNEL    3
#define TPCF_OPT_WAIT_LIMIT    4
#define TPCF_OPT_TEST_SKIP_MMA 5
#define TPCF_OPT_HOST_GROUP_KB 6
#define TPCF_KERNEL_AUTO     0
#define TPCF_KERNEL_DIRECT   1
#define TPCF_KERNEL_GENERAL  2
int tpcf_set_option(tpcf_ctx *ctx, int option, int value);

#ifdef __cplusplus
}
#endif
#endif /* TPCF_H */
