// Internal declarations shared by the CUDA translation units of libtpcf.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "tpcf.h"

namespace tpcf {

constexpr int MAX_NS = 256;          // s bins
constexpr int MAX_NBIN = 65536;      // s bins x mu bins (the block histogram must also fit in shared memory)
constexpr int MAX_NC = 1024;         // mesh cells per axis
constexpr int MAX_ROWS = 81;         // (2K+1)^2 neighbour rows, K <= 4
constexpr int MAX_TABLE = 16384;     // s-bin lookup slots

// s-bin lookup: each slot of the table holds k, the bin of the slot's d2
// values below edge k+1 (-1: below the first edge, n_s: beyond the last),
// after which d2 is compared with the band of edge k+1 only.  CODE_AMBIG
// marks a slot that spans several edge bands: always recheck exactly.
constexpr int16_t CODE_AMBIG = 0x7FFF;

// One pair-count term: histogram of pairs between catalogue A and catalogue B.
struct Term {
    int cat_a;
    int cat_b;
    int auto_pairs;        // 1: A == B, unordered pairs of distinct points
    int pad;
    long long *hist;       // caller's int64 output row [nbin]
};

// One catalogue in the packed point arrays.
struct Cat {
    const double *xyz;     // caller's float64 [n][3], or nullptr
    const uint32_t *u32;   // caller's pre-quantised [3][n] (row stride n), or nullptr
    uint32_t p0;           // first index in the packed arrays
    uint32_t n;            // number of points
};

// A work unit: a chunk of the points of one mesh cell of catalogue A, paired
// against the neighbourhood of that cell in catalogue B for term t.
struct Unit {
    int term;
    int cell;              // linear cell index in catalogue A
    uint32_t a0, a1;       // packed sorted index range of the a-points
};

// Everything the pair-count kernels need, passed by value.
struct CountParams {
    int geometry;          // TPCF_PERIODIC | TPCF_OPEN
    int los;               // TPCF_LOS_X | TPCF_LOS_MIDPOINT
    int n_s, n_mu, nbin;
    int n_c;               // cells per axis
    int n_cells;           // n_c^3
    int bits;              // 32 (periodic) or 30 (open)
    int n_rows;            // neighbour rows (dz, dy) with a non-empty x range
    int8_t row_dz[MAX_ROWS], row_dy[MAX_ROWS], row_kx[MAX_ROWS];
    // s-bin lookup over float bit patterns of d2 + tab_bias
    int tab_shift;         // key = bits(d2 + tab_bias) >> tab_shift
    uint32_t tab_key0;     // first key in the table
    int tab_n;             // table slots
    float tab_bias;
    float hit_max;         // upper band of T_ns: d2 >= hit_max is never binned
    float dot_margin;      // slack of the dot-product candidate test
    float mu_c1, mu_c2;    // mu ambiguity band (see the kernel)
    float mu_c3;
    float mu_c1r;          // midpoint line of sight: mu_c1 / n_mu (rounded up)
    float inv_nmu2;        // 1 / n_mu^2
    int linear;            // edges e_k = k * ds exactly: s bin = floor(sqrt(D2) / (q ds))
    float s_scale;         // 1 / (n_mu q ds): u = d2 * (n_mu / sqrt(d2)) * s_scale = sqrt(d2) / (q ds)
    float s_c0, s_c1;      // s band for the linear path: beta_s = s_c0 + s_c1 * u
    float s_lo_mul, s_hi_mul;  // linear path, v = d2 * (n_mu / sqrt(d2)): u* lies in
                               // [v s_lo_mul - s_c0, v s_hi_mul + s_c0] (directed roundings)
    float s_top;           // 1.5 * 2^23 + n_s: floor(u_lo) + 1.5 * 2^23 < s_top <=> s bin < n_s
    float f_nmu;           // n_mu as a float
    float sent_d2, sent_dx;    // x-path queue sentinel: s half a bin past the last edge, mu mid-bin
    long long obs[3];      // observer in grid units (midpoint line of sight)
    unsigned long long T[MAX_NS + 1];        // exact squared edges in grid units
    float lo[MAX_NS + 2], hi[MAX_NS + 2];    // float bands: d2 < lo => D2 < T; d2 >= hi => D2 >= T;
                                             // entry n_s+1 is +inf
};

// Constants of the direct pair counter (pairdirect.cu): linear s bins from 0
// with the x line of sight or s only.  Every coordinate it handles is in
// units of one s bin, relative to the integer lower corner of the unit's
// cell; the error bounds behind m, cs and d2min are derived in plan.cpp.
struct DirectParams {
    int R;             // histogram copies (lane l adds to copy l mod R)
    int W;             // warps per block (one block per SM)
    int C;             // histogram columns, 1 << logC: signed mu columns from -CO, or 1 (s only)
    int logC;
    int CO;            // column of mu bin 0 (the signed mu bin j sits in column j + CO)
    int rows;          // n_s + 1: the last row takes every pair at or beyond the last edge
    int smem;          // dynamic shared memory bytes
    int mid;           // 1: mu from the midpoint line of sight
    unsigned long long unit_pair_bound;   // pairs one unit can add to one histogram counter
    float inv_qds;     // grid units -> bin units
    float nmu;         // n_mu
    float m;           // mu margin in units of n_mu bins: t in [dx'- r, dx'+ r] brackets n_mu mu
    float cs;          // s residual bound: floor(u) is the bin when |u - floor(u) - 1/2| <= cs
    float tiny;        // d2 addend (keeps rsqrt finite; with mu bins it also bounds r)
    float hit;         // filter: squared box distance (bin^2) below which a b-point is kept
    float s_top;       // 2^23 + n_s: the clamped row of pairs beyond the last edge
    float pad2;
    // midpoint line of sight: t = n_mu mu is certain when |t - floor(t) - 1/2| <= c05 - c1 r - c3 rl
    // (r = 1 / |d|, rl = 1 / |l| as computed); tinyl keeps rl finite
    float c1, c3, c05, tinyl;
};

// Workspace layout produced by the mesh build and consumed by the counters.
struct Mesh {
    const float4 *pf;          // sorted: cell-relative float coords, .w = -|f|^2 / 2
    const uint16_t *pcx;       // sorted: cell x index of each point
    const uint32_t *us;        // sorted exact grid coords [3][n_total]
    uint32_t n_total;
    const uint32_t *cellstart; // [n_cat * n_cells + 1] global sorted start of each (cat, cell)
    const uint32_t *orig;      // [n_c + 1] integer lower corner of each cell column
};

// device status bits (written with atomicOr, read by tpcf_sync)
constexpr int STATUS_RANGE = 1;        // position outside the bounding cube
constexpr int STATUS_EMPTY_BIN = 2;    // rr == 0 in the LS estimator
constexpr int STATUS_TIMEOUT = 4;      // bounded wait gave up

// ---- launchers (each returns cudaError_t of the launch) ----
cudaError_t launch_quantize_keys(const Cat *cats, int n_cat, uint32_t max_n, const CountParams &p,
                                 double L, const double *origin, uint32_t n_total, uint32_t *uq,
                                 uint32_t *keys, uint32_t *cellcount, int *status, cudaStream_t s);
cudaError_t launch_scan_u32(const uint32_t *in, uint32_t *out, size_t n, uint32_t *tmp, size_t tmp_n,
                            cudaStream_t s);
size_t scan_tmp_elems(size_t n);
cudaError_t launch_scatter(const Cat *cats, int n_cat, uint32_t max_n, const CountParams &p,
                           const uint32_t *uq, const uint32_t *keys, const uint32_t *cellstart,
                           uint32_t *cursor, const uint32_t *orig, uint32_t n_total, uint32_t *us,
                           float4 *pf, uint16_t *pcx, cudaStream_t s);
cudaError_t launch_unit_count(const Term *terms, int n_terms, const Cat *cats, int n_cells,
                              const uint32_t *cellstart, int chunk, uint32_t *ucount, cudaStream_t s);
cudaError_t launch_stats_accum(const unsigned long long *stats, unsigned long long *acc, int first, cudaStream_t s);
cudaError_t launch_unit_fill(const Term *terms, int n_terms, const Cat *cats, int n_cells,
                             const uint32_t *cellstart, int chunk, const uint32_t *ustart, Unit *units,
                             cudaStream_t s);

struct PairLaunch {
    int blocks;            // grid size
    int warps_per_block;
    int persistent;        // 1: claim units from a global counter; 0: one block per cell of one term
    int term;              // per-launch mode: the term
    int smem_bytes;
    int chunk;             // a-points per work unit (per-launch mode)
    void *scratch;         // paircount_scratch_bytes(blocks) of device memory: filtered neighbour windows
};
cudaError_t launch_paircount(const CountParams &p, const Mesh &m, const Term *terms, const Cat *cats,
                             const Unit *units, const uint32_t *n_units, unsigned *claim,
                             const int16_t *table, unsigned long long *stats, int *status,
                             const PairLaunch &pl, cudaStream_t s);
int paircount_smem_bytes(const CountParams &p, int warps_per_block);
size_t paircount_scratch_bytes(int blocks);
cudaError_t paircount_set_attrs(const CountParams &p, int smem_bytes);
int paircount_max_blocks_per_sm(const CountParams &p, int warps_per_block, int smem_bytes);

// direct pair counter (pairdirect.cu): one block of DIRECT_WARPS warps per SM, no global scratch
constexpr int DIRECT_ACHUNK = 64;    // a-points per work unit
constexpr int DIRECT_WARPS = 16;
cudaError_t launch_pairdirect(const CountParams &p, const DirectParams &d, const Mesh &m, const Term *terms,
                              const Unit *units, const uint32_t *n_units, unsigned *claim, unsigned long long *stats,
                              const PairLaunch &pl, cudaStream_t s);
size_t pairdirect_smem_bytes(const CountParams &p, int R, int C, int W);
cudaError_t pairdirect_set_attrs(const DirectParams &d, int mu);
int pairdirect_max_blocks_per_sm(const DirectParams &d, int mu);

// ---- estimator launchers ----
cudaError_t launch_ls(const long long *dd, const long long *dr, const long long *rr,
                      const long long *nd_nr /* [n_mock][1+M] */, const int *sel, int n_sel,
                      int n_mock, int M, int nbin, double *xi, int *status, cudaStream_t s);
cudaError_t launch_lc_fp64(const double *xi_a1, const double *xi_a2, const double *xi_b, int n_mock,
                           int nbin, double *work /* 3*n_mock*nbin + 3*nbin + 3*nbin*nbin */,
                           int M_a, double M, double *C_lc, double *Ca, double *Cb, double *A, double *B,
                           cudaStream_t s);
// Launch options of the split-precision Gram kernel: the SM count its grid is
// sized for, the bound (polls) of the epilogue's wait for the MMA chain, and a
// test-only switch under which one CTA issues no MMA so that this wait runs out.
struct GramOpts {
    int n_sm = 1;
    long long wait_limit = 0;   // 0: the built-in bound
    int test_skip_mma = 0;
};
cudaError_t launch_lc_split(const double *xi_a1, const double *xi_a2, const double *xi_b, int n_mock,
                            int nbin, int precision, void *work, size_t work_bytes, int M_a, double M,
                            double *C_lc, double *Ca, double *Cb, double *A, double *B, int *status,
                            const GramOpts &opt, cudaStream_t s);
// work bytes of the split-precision path for n_var variants (3: LC, 1: one sample covariance) on n_sm SMs
size_t lc_split_work_bytes(int n_mock, int nbin, int precision, int n_sm, int n_var = 3);
// float64 covariance paths with the mocks split into n_split ranges (fp64_splits picks a count that fills
// the GPU); work holds fp64_work_elems(n_mock, nbin, n_var, n_split) doubles
int fp64_splits(int n_mock, int nbin, int n_var);
size_t fp64_work_elems(int n_mock, int nbin, int n_var, int n_split);
cudaError_t launch_lc_fp64_split(const double *xi_a1, const double *xi_a2, const double *xi_b, int n_mock, int nbin,
                                 double *work, int n_split, int M_a, double M, double *C_lc, double *Ca, double *Cb,
                                 double *A, double *B, cudaStream_t s);
// sample covariance C[nbin][nbin] of one variant xi[n_mock][nbin], Eq. (bruteforce)
cudaError_t launch_cov_fp64(const double *xi, int n_mock, int nbin, double *work, double *C, cudaStream_t s,
                            int n_split);
cudaError_t launch_cov_split(const double *xi, int n_mock, int nbin, int precision, void *work, size_t work_bytes,
                             double *C, int *status, const GramOpts &opt, cudaStream_t s);
// column means mean[n_var][nbin] of the first n_var xi variants
cudaError_t launch_means(const double *xi_a1, const double *xi_a2, const double *xi_b, int n_var, int n_mock,
                         int nbin, double *mean, cudaStream_t s);
// LC combination from the three Gram blocks G[3][nbin][nbin] (float64)
cudaError_t launch_combine(const double *G, int nbin, int n_mock, int M_a, double M, double *C_lc, double *Ca,
                           double *Cb, double *A, double *B, cudaStream_t s);
// C = G / (n_mock - 1) for one Gram block
cudaError_t launch_scale(const double *G, int nbin, int n_mock, double *C, cudaStream_t s);

// ---- linear maps before the covariance (project.cu) ----
// out[rows][n_s/f_s][n_mu/f_mu] = group sums of in[rows][n_s][n_mu] (int64)
cudaError_t launch_rebin(const long long *in, long long rows, int n_s, int n_mu, int f_s, int f_mu, long long *out,
                         cudaStream_t s);
// y[n_mock][n_out] = x[n_mock][nbin] P^T, P [n_out][nbin] (float64)
cudaError_t launch_project(const double *P, int n_out, int nbin, const double *x, int n_mock, double *y,
                           cudaStream_t s);

// ---- accuracy of the covariance estimates (covcov.cu) ----
// var[i][j] = Var(C_ij): LC form with B (D = A + B / (2 M_a)), sample-covariance form with B = NULL (A = C)
cudaError_t launch_covcov(const double *A, const double *B, int nbin, int M_a, double M, int n_mock, double *var,
                          cudaStream_t s);
size_t chi2_work_bytes();
// mode 0: predicted chi^2_2 from (X = A, Y = B or NULL); mode 1: measured chi^2 of X against Y; R normalises
cudaError_t launch_chi2(int mode, const double *X, const double *Y, const double *R, int nbin, int M_a, double M,
                        double *work, double *out, cudaStream_t s);
size_t eig_work_bytes(int n);
// ascending eigenvalues w[n] of the symmetric C[n][n] (n <= 1024)
cudaError_t launch_eigvalsh(const double *C, int n, double *work, double *w, cudaStream_t s);

}  // namespace tpcf
