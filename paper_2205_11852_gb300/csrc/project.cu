// Linear maps applied before the covariance (Sect. 2.3: the LC construction
// holds for any linear function of the correlation function): re-binning of
// the pair counts into wider (s, mu) bins, and projection of xi rows with a
// matrix, e.g. onto the Legendre multipoles of Sect. 4.3.
#include <algorithm>

#include "tpcf_internal.h"

namespace tpcf {
namespace {

// out[r][k'][j'] = sum_{k in group k', j in group j'} in[r][k][j]   (int64, exact)
__global__ void rebin_kernel(const long long *__restrict__ in, long long rows, int n_s, int n_mu, int f_s, int f_mu,
                             long long *__restrict__ out)
{
    const int ns2 = n_s / f_s, nm2 = n_mu / f_mu, nb2 = ns2 * nm2;
    const long long total = rows * nb2;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / nb2;
        const int b2 = (int)(t - r * nb2);
        const int k2 = b2 / nm2, j2 = b2 - k2 * nm2;
        const long long *src = in + r * (long long)n_s * n_mu;
        long long s = 0;
        for (int k = k2 * f_s; k < (k2 + 1) * f_s; k++)
            for (int j = j2 * f_mu; j < (j2 + 1) * f_mu; j++) s += src[(long long)k * n_mu + j];
        out[t] = s;
    }
}

// y[m][o] = sum_b P[o][b] x[m][b]  (float64; 32 x 32 output tiles, 2 x 2 per thread)
constexpr int PT = 32, PK = 32;
__global__ void __launch_bounds__(256) project_kernel(const double *__restrict__ P, int n_out, int nbin,
                                                       const double *__restrict__ x, int n_mock,
                                                       double *__restrict__ y)
{
    __shared__ double Xs[PT][PK + 1];
    __shared__ double Ps[PT][PK + 1];
    const int m0 = blockIdx.y * PT, o0 = blockIdx.x * PT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[2][2] = {};
    for (int k0 = 0; k0 < nbin; k0 += PK) {
        for (int e = threadIdx.x; e < PT * PK; e += 256) {
            const int r = e / PK, c = e % PK, k = k0 + c;
            Xs[r][c] = (m0 + r < n_mock && k < nbin) ? x[(size_t)(m0 + r) * nbin + k] : 0.0;
            Ps[r][c] = (o0 + r < n_out && k < nbin) ? P[(size_t)(o0 + r) * nbin + k] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int c = 0; c < PK; c++) {
            const double a0 = Xs[ty][c], a1 = Xs[ty + 16][c];
            const double b0 = Ps[tx][c], b1 = Ps[tx + 16][c];
            acc[0][0] = fma(a0, b0, acc[0][0]);
            acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][0] = fma(a1, b0, acc[1][0]);
            acc[1][1] = fma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) {
            const int m = m0 + ty + 16 * i, o = o0 + tx + 16 * j;
            if (m < n_mock && o < n_out) y[(size_t)m * n_out + o] = acc[i][j];
        }
}

}  // namespace

cudaError_t launch_rebin(const long long *in, long long rows, int n_s, int n_mu, int f_s, int f_mu, long long *out,
                         cudaStream_t s)
{
    const long long total = rows * (long long)(n_s / f_s) * (n_mu / f_mu);
    if (total <= 0) return cudaSuccess;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 16);
    rebin_kernel<<<blocks, 256, 0, s>>>(in, rows, n_s, n_mu, f_s, f_mu, out);
    return cudaGetLastError();
}

cudaError_t launch_project(const double *P, int n_out, int nbin, const double *x, int n_mock, double *y,
                           cudaStream_t s)
{
    if (n_mock <= 0 || n_out <= 0) return cudaSuccess;
    const dim3 grid((n_out + PT - 1) / PT, (n_mock + PT - 1) / PT);
    project_kernel<<<grid, 256, 0, s>>>(P, n_out, nbin, x, n_mock, y);
    return cudaGetLastError();
}

}  // namespace tpcf
