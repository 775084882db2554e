// Split Landy-Szalay estimator (Sect. 2.1), the sample covariance
// (Eq. bruteforce) and the linear-construction covariance (Eqs. R1R2, LCdef)
// in float64.
#include <cmath>

#include "tpcf_internal.h"

namespace tpcf {

namespace {

// xi[m][b] over the selected random subsets (Sect. 2.1):
//   dd = DD / (N_d (N_d-1)/2), dr = mean_i DR_i / (N_d N_r,i),
//   rr = mean_i RR_i / (N_r,i (N_r,i-1)/2), xi = (dd - 2 dr) / rr + 1
__global__ void ls_kernel(const long long *__restrict__ dd, const long long *__restrict__ dr,
                          const long long *__restrict__ rr, const long long *__restrict__ nd_nr,
                          const int *__restrict__ sel, int n_sel, int n_mock, int M, int nbin,
                          double *__restrict__ xi, int *__restrict__ status)
{
    const size_t total = (size_t)n_mock * nbin;
    bool empty = false;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(t / nbin), b = (int)(t % nbin);
        const long long *nn = nd_nr + (size_t)m * (1 + M);
        const double nd = (double)nn[0];
        const double ddn = (double)dd[(size_t)m * nbin + b] / (nd * (nd - 1.0) / 2.0);
        double drn = 0.0, rrn = 0.0;
        for (int k = 0; k < n_sel; k++) {
            const int i = sel[k];
            const double nr = (double)nn[1 + i];
            const size_t o = ((size_t)m * M + i) * nbin + b;
            drn += (double)dr[o] / (nd * nr);
            rrn += (double)rr[o] / (nr * (nr - 1.0) / 2.0);
        }
        drn /= (double)n_sel;
        rrn /= (double)n_sel;
        double v;
        if (rrn == 0.0) {
            v = __longlong_as_double(0x7ff8000000000000ll);
            empty = true;
        } else {
            v = (ddn - 2.0 * drn) / rrn + 1.0;
        }
        xi[t] = v;
    }
    if (empty) atomicOr(status, STATUS_EMPTY_BIN);
}

// column means of the three variants: mean[v][b].  A block of 32 x 32
// threads takes 32 columns of one variant: thread (tx, ty) sums rows ty,
// ty + 32, ... of column tx in four interleaved partial sums (so that loads
// of consecutive rows are in flight together, and a warp reads 32 consecutive
// columns of a row), then the 32 row groups are added in shared memory in a
// fixed order.
constexpr int MEAN_COLS = 32, MEAN_ROWS = 32;
__global__ void __launch_bounds__(MEAN_COLS * MEAN_ROWS) mean_kernel(const double *__restrict__ x0,
                                                                     const double *__restrict__ x1,
                                                                     const double *__restrict__ x2, int n_mock,
                                                                     int nbin, double *__restrict__ mean)
{
    __shared__ double part[MEAN_ROWS][MEAN_COLS + 1];
    const int v = blockIdx.y;
    const double *x = v == 0 ? x0 : (v == 1 ? x1 : x2);
    const int tx = threadIdx.x % MEAN_COLS, ty = threadIdx.x / MEAN_COLS;
    const int b = blockIdx.x * MEAN_COLS + tx;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    if (b < nbin) {
        int m = ty;
        for (; m + 3 * MEAN_ROWS < n_mock; m += 4 * MEAN_ROWS) {
#pragma unroll
            for (int k = 0; k < 4; k++) s[k] += x[(size_t)(m + k * MEAN_ROWS) * nbin + b];
        }
        // at most three rows remain
        if (m < n_mock) s[0] += x[(size_t)m * nbin + b];
        if (m + MEAN_ROWS < n_mock) s[1] += x[(size_t)(m + MEAN_ROWS) * nbin + b];
        if (m + 2 * MEAN_ROWS < n_mock) s[2] += x[(size_t)(m + 2 * MEAN_ROWS) * nbin + b];
    }
    part[ty][tx] = (s[0] + s[1]) + (s[2] + s[3]);
    __syncthreads();
    if (ty == 0 && b < nbin) {
        double t = 0.0;
        for (int r = 0; r < MEAN_ROWS; r++) t += part[r][tx];
        mean[(size_t)v * nbin + b] = t / (double)n_mock;
    }
}

// centred residuals Y[v][m][b] = x_v[m][b] - mean[v][b]
__global__ void centre_kernel(const double *__restrict__ x0, const double *__restrict__ x1,
                              const double *__restrict__ x2, int n_mock, int nbin,
                              const double *__restrict__ mean, double *__restrict__ Y)
{
    const int v = blockIdx.y;
    const double *x = v == 0 ? x0 : (v == 1 ? x1 : x2);
    const size_t total = (size_t)n_mock * nbin;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x)
        Y[(size_t)v * total + t] = x[t] - mean[(size_t)v * nbin + (t % nbin)];
}

// G[v] = Y[v]^T Y[v] (nbin x nbin), float64, 64x64 tiles, 4x4 per thread.
// With n_split > 1, blockIdx.z = v * n_split + split and the block sums the
// mocks [split * k_len, (split + 1) * k_len) into its own partial Gram
// G + (v * n_split + split) * nbin^2 (summed afterwards in a fixed order).
constexpr int GT = 64, GK = 16;
__global__ void __launch_bounds__(256) gram_fp64_kernel(const double *__restrict__ Y, int n_mock, int nbin,
                                                         double *__restrict__ G, int n_split = 1, int k_len = 0)
{
    __shared__ double As[GK][GT + 1];
    __shared__ double Bs[GK][GT + 1];
    const int v = blockIdx.z / n_split, split = blockIdx.z % n_split;
    const double *y = Y + (size_t)v * n_mock * nbin;
    double *g = G + (size_t)blockIdx.z * nbin * nbin;
    const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
    if (j0 + GT <= i0) return;  // below the diagonal block row: filled by symmetry
    const int k_begin = n_split > 1 ? split * k_len : 0;
    const int k_end = n_split > 1 ? min(n_mock, k_begin + k_len) : n_mock;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int k0 = k_begin; k0 < k_end; k0 += GK) {
        for (int e = threadIdx.x; e < GK * GT; e += 256) {
            const int kk = e / GT, c = e % GT;
            const int k = k0 + kk;
            As[kk][c] = (k < k_end && i0 + c < nbin) ? y[(size_t)k * nbin + i0 + c] : 0.0;
            Bs[kk][c] = (k < k_end && j0 + c < nbin) ? y[(size_t)k * nbin + j0 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; kk++) {
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; r++) a[r] = As[kk][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; c++) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
            if (i < nbin && j < nbin && j >= i) {
                g[(size_t)i * nbin + j] = acc[r][c];
                g[(size_t)j * nbin + i] = acc[r][c];
            }
        }
}

// G[v] = sum over the splits of the partial Grams, in split order
__global__ void split_sum_kernel(const double *__restrict__ part, int n_var, int n_split, size_t nn,
                                 double *__restrict__ G)
{
    const size_t total = (size_t)n_var * nn;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t v = t / nn, e = t % nn;
        const double *p = part + v * n_split * nn + e;
        double s = 0.0;
        for (int k = 0; k < n_split; k++) s += p[(size_t)k * nn];
        G[t] = s;
    }
}

// LC combination in float64 (Eqs. R1R2, LCdef):
//   Ca = (G1 + G2) / (2 (N-1)), Cb = Gb / (N-1), A = 2 Cb - Ca,
//   B = 2 M_a (Ca - Cb), C = A + B / M
__global__ void combine_kernel(const double *__restrict__ G, int nbin, int n_mock, int M_a, double M,
                               double *__restrict__ C_lc, double *__restrict__ Ca_o, double *__restrict__ Cb_o,
                               double *__restrict__ A_o, double *__restrict__ B_o)
{
    const size_t nn = (size_t)nbin * nbin;
    const double inv = 1.0 / (double)(n_mock - 1);
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (size_t)gridDim.x * blockDim.x) {
        const double c1 = G[t] * inv, c2 = G[nn + t] * inv, cb = G[2 * nn + t] * inv;
        const double ca = 0.5 * c1 + 0.5 * c2;
        const double a = 2.0 * cb - ca;
        const double bb = 2.0 * (double)M_a * (ca - cb);
        C_lc[t] = a + bb / M;
        if (Ca_o) Ca_o[t] = ca;
        if (Cb_o) Cb_o[t] = cb;
        if (A_o) A_o[t] = a;
        if (B_o) B_o[t] = bb;
    }
}

// sample covariance of one variant, Eq. (bruteforce): C = G / (N - 1)
__global__ void scale_kernel(const double *__restrict__ G, size_t nn, int n_mock, double *__restrict__ C)
{
    const double inv = 1.0 / (double)(n_mock - 1);
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (size_t)gridDim.x * blockDim.x)
        C[t] = G[t] * inv;
}

int blocks_for(size_t n, int threads) { return (int)std::min<size_t>((n + threads - 1) / threads, 152 * 16); }

// float64 Gram products of n_var centred variants; returns G [n_var][nbin][nbin] inside work.
// n_split > 1 splits the mocks into n_split ranges (partials after G in work, summed in split order).
double *gram_fp64(const double *x0, const double *x1, const double *x2, int n_var, int n_mock, int nbin,
                  double *work, cudaStream_t s, int n_split = 1)
{
    double *Y = work;
    double *mean = Y + (size_t)n_var * n_mock * nbin;
    double *G = mean + (size_t)n_var * nbin;
    mean_kernel<<<dim3((nbin + MEAN_COLS - 1) / MEAN_COLS, n_var), MEAN_COLS * MEAN_ROWS, 0, s>>>(x0, x1, x2, n_mock,
                                                                                              nbin, mean);
    centre_kernel<<<dim3(std::max(1, blocks_for((size_t)n_mock * nbin, 256)), n_var), 256, 0, s>>>(
        x0, x1, x2, n_mock, nbin, mean, Y);
    const int nt = (nbin + GT - 1) / GT;
    if (n_split <= 1) {
        gram_fp64_kernel<<<dim3(nt, nt, n_var), 256, 0, s>>>(Y, n_mock, nbin, G);
        return G;
    }
    const int k_len = ((n_mock + n_split - 1) / n_split + GK - 1) / GK * GK;
    double *part = G + (size_t)n_var * nbin * nbin;
    gram_fp64_kernel<<<dim3(nt, nt, n_var * n_split), 256, 0, s>>>(Y, n_mock, nbin, part, n_split, k_len);
    const size_t nn = (size_t)nbin * nbin;
    split_sum_kernel<<<blocks_for((size_t)n_var * nn, 256), 256, 0, s>>>(part, n_var, n_split, nn, G);
    return G;
}

}  // namespace

cudaError_t launch_ls(const long long *dd, const long long *dr, const long long *rr, const long long *nd_nr,
                      const int *sel, int n_sel, int n_mock, int M, int nbin, double *xi, int *status,
                      cudaStream_t s)
{
    const size_t total = (size_t)n_mock * nbin;
    ls_kernel<<<std::max(1, blocks_for(total, 256)), 256, 0, s>>>(dd, dr, rr, nd_nr, sel, n_sel, n_mock, M, nbin,
                                                                  xi, status);
    return cudaGetLastError();
}

cudaError_t launch_lc_fp64(const double *xi_a1, const double *xi_a2, const double *xi_b, int n_mock, int nbin,
                           double *work, int M_a, double M, double *C_lc, double *Ca, double *Cb, double *A,
                           double *B, cudaStream_t s)
{
    const double *G = gram_fp64(xi_a1, xi_a2, xi_b, 3, n_mock, nbin, work, s);
    combine_kernel<<<std::max(1, blocks_for((size_t)nbin * nbin, 256)), 256, 0, s>>>(G, nbin, n_mock, M_a, M, C_lc,
                                                                                     Ca, Cb, A, B);
    return cudaGetLastError();
}

int fp64_splits(int n_mock, int nbin, int n_var)
{
    // enough blocks to fill the GPU: (upper-triangle tiles x variants x splits) ~ 2 per SM, splits of >= 64 mocks
    const int nt = (nbin + GT - 1) / GT;
    const int tiles = n_var * nt * (nt + 1) / 2;
    const int want = std::max(1, (2 * 152 + tiles - 1) / tiles);
    return std::max(1, std::min(want, n_mock / 64));
}

size_t fp64_work_elems(int n_mock, int nbin, int n_var, int n_split)
{
    const size_t nn = (size_t)nbin * nbin;
    return (size_t)n_var * n_mock * nbin + (size_t)n_var * nbin + (size_t)n_var * nn +
           (n_split > 1 ? (size_t)n_var * n_split * nn : 0);
}

cudaError_t launch_lc_fp64_split(const double *xi_a1, const double *xi_a2, const double *xi_b, int n_mock, int nbin,
                                 double *work, int n_split, int M_a, double M, double *C_lc, double *Ca, double *Cb,
                                 double *A, double *B, cudaStream_t s)
{
    const double *G = gram_fp64(xi_a1, xi_a2, xi_b, 3, n_mock, nbin, work, s, n_split);
    combine_kernel<<<std::max(1, blocks_for((size_t)nbin * nbin, 256)), 256, 0, s>>>(G, nbin, n_mock, M_a, M, C_lc,
                                                                                     Ca, Cb, A, B);
    return cudaGetLastError();
}

cudaError_t launch_cov_fp64(const double *xi, int n_mock, int nbin, double *work, double *C, cudaStream_t s,
                            int n_split)
{
    const double *G = gram_fp64(xi, xi, xi, 1, n_mock, nbin, work, s, n_split);
    scale_kernel<<<std::max(1, blocks_for((size_t)nbin * nbin, 256)), 256, 0, s>>>(G, (size_t)nbin * nbin, n_mock,
                                                                                  C);
    return cudaGetLastError();
}

cudaError_t launch_means(const double *xi_a1, const double *xi_a2, const double *xi_b, int n_var, int n_mock,
                         int nbin, double *mean, cudaStream_t s)
{
    mean_kernel<<<dim3((nbin + MEAN_COLS - 1) / MEAN_COLS, n_var), MEAN_COLS * MEAN_ROWS, 0, s>>>(
        xi_a1, xi_a2, xi_b, n_mock, nbin, mean);
    return cudaGetLastError();
}

cudaError_t launch_scale(const double *G, int nbin, int n_mock, double *C, cudaStream_t s)
{
    scale_kernel<<<std::max(1, blocks_for((size_t)nbin * nbin, 256)), 256, 0, s>>>(G, (size_t)nbin * nbin, n_mock,
                                                                                  C);
    return cudaGetLastError();
}

cudaError_t launch_combine(const double *G, int nbin, int n_mock, int M_a, double M, double *C_lc, double *Ca,
                           double *Cb, double *A, double *B, cudaStream_t s)
{
    combine_kernel<<<std::max(1, blocks_for((size_t)nbin * nbin, 256)), 256, 0, s>>>(G, nbin, n_mock, M_a, M, C_lc,
                                                                                     Ca, Cb, A, B);
    return cudaGetLastError();
}

}  // namespace tpcf
