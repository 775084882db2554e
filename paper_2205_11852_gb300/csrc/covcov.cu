// Accuracy of the covariance estimates (Sect. 3): the covariance of the
// sample and LC covariances for Gaussian xi (Eqs. covcov, covcov_brute,
// covcov_fast), the chi^2 accuracy measure of Eq. (chi2) and its predicted
// value, and the eigenvalues of a symmetric matrix, used to check whether an
// LC covariance is positive definite before it is inverted (Sect. 3.4).
#include <algorithm>
#include <cmath>

#include "tpcf_internal.h"

namespace tpcf {
namespace {

// Variance of each covariance element, Eq. (covcov_fast) at k = i, l = j:
//   (N-1) Var(C_ij) = D_ii D_jj + D_ij^2 + c^2 (B_ii B_jj + B_ij^2)
// D = A + w B.  LC: w = 1/(2 M_a), c = 1/(2 M_a) - 1/M.  Sample covariance,
// Eq. (covcov_brute): B absent (c = 0) and A = C.
__device__ __forceinline__ double covcov_term(const double *A, const double *B, int n, int i, int j, double w,
                                              double c2)
{
    const size_t ii = (size_t)i * n + i, jj = (size_t)j * n + j, ij = (size_t)i * n + j;
    double dii = A[ii], djj = A[jj], dij = A[ij];
    double t = 0.0;
    if (B) {
        const double bii = B[ii], bjj = B[jj], bij = B[ij];
        dii = fma(w, bii, dii);
        djj = fma(w, bjj, djj);
        dij = fma(w, bij, dij);
        t = c2 * fma(bii, bjj, bij * bij);
    }
    return fma(dii, djj, dij * dij) + t;
}

__global__ void covcov_kernel(const double *__restrict__ A, const double *__restrict__ B, int n, double w, double c2,
                              double inv_nm1, double *__restrict__ var)
{
    const size_t nn = (size_t)n * n;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (size_t)gridDim.x * blockDim.x)
        var[t] = covcov_term(A, B, n, (int)(t / n), (int)(t % n), w, c2) * inv_nm1;
}

constexpr int RED_BLOCKS = 152 * 2, RED_THREADS = 256;

// sum over the block (blockDim.x a multiple of 32, at most 1024), in a fixed
// order; the result is valid in thread 0
__device__ double block_sum(double v)
{
    __shared__ double part[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) s += part[k];
    __syncthreads();
    return s;
}

// per-block partial sums over (i, j) of a normalised term:
//   mode 0: covcov_term / (R_ii R_jj)                 (predicted chi^2_2)
//   mode 1: (X_ij - Y_ij)^2 / (R_ii R_jj)             (measured chi^2, Eq. chi2)
__global__ void __launch_bounds__(RED_THREADS) chi2_partial(int mode, const double *__restrict__ X,
                                                            const double *__restrict__ Y, const double *__restrict__ R,
                                                            int n, double w, double c2, double *__restrict__ part)
{
    const size_t nn = (size_t)n * n;
    double s = 0.0;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / n), j = (int)(t % n);
        const double norm = R[(size_t)i * n + i] * R[(size_t)j * n + j];
        double v;
        if (mode == 0) {
            v = covcov_term(X, Y, n, i, j, w, c2);
        } else {
            const double d = X[t] - Y[t];
            v = d * d;
        }
        s += v / norm;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(RED_THREADS) chi2_final(const double *__restrict__ part, int n_part, double scale,
                                                          double *__restrict__ out)
{
    double s = 0.0;
    for (int k = threadIdx.x; k < n_part; k += blockDim.x) s += part[k];
    s = block_sum(s);
    if (threadIdx.x == 0) *out = s * scale;
}

// ---- eigenvalues of a symmetric matrix ----
constexpr int TRI_CTAS = 8, TRI_THREADS = 512;

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// all threads of the cluster; orders this cluster's global-memory writes
// before the barrier ahead of its reads after it
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Householder reduction of the symmetric matrix a[n][n] (overwritten) to
// tridiagonal form d[n], e[n-1] by one cluster of TRI_CTAS blocks: for each
// column k the reflector H = I - beta v v^T zeroes a[k+2.., k] and the
// trailing block B becomes H B H = B - v w^T - w v^T with p = beta B v,
// w = p - (beta p.v / 2) v.  Block r owns the rows i = r mod TRI_CTAS: it
// forms p_i for them (to pg in global memory), and after a cluster barrier
// every block forms w from all of p and updates its own rows; a second
// barrier ends the column.  v, beta and w are computed by every block alike
// (the same data and operation order), so every block takes the same branch
// at each barrier.
__global__ void __cluster_dims__(TRI_CTAS, 1, 1) __launch_bounds__(TRI_THREADS)
    tridiag_kernel(double *__restrict__ a, int n, double *__restrict__ d, double *__restrict__ e,
                   double *__restrict__ pg)
{
    extern __shared__ double sh[];
    double *v = sh;            // [n]
    double *w = sh + n;        // [n]
    __shared__ double s_alpha, s_beta, s_k;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int rank = (int)cluster_rank();
    for (int k = 0; k + 2 < n; k++) {
        const int m0 = k + 1;   // the reflector acts on rows/cols m0..n-1
        // x = a[m0.., k] = a[k, m0..] (symmetric); alpha = -sign(x0) |x|
        const double *rk = a + (size_t)k * n;
        double ss = 0.0;
        for (int i = m0 + 1 + tid; i < n; i += blockDim.x) ss = fma(rk[i], rk[i], ss);
        const double tail = block_sum(ss);
        if (tid == 0) {
            const double x0 = rk[m0];
            if (tail == 0.0) {
                s_alpha = x0;      // column already reduced: H = I
                s_beta = 0.0;
            } else {
                const double nx = sqrt(fma(x0, x0, tail));
                const double alpha = x0 > 0.0 ? -nx : nx;
                const double v0 = x0 - alpha;
                s_alpha = alpha;
                s_beta = 2.0 / fma(v0, v0, tail);   // 2 / (v.v)
                v[m0] = v0;
            }
            if (rank == 0) {
                d[k] = rk[k];
                e[k] = s_alpha;
            }
        }
        __syncthreads();
        const double beta = s_beta;
        if (beta == 0.0) continue;   // nothing written in this column: no barrier needed
        for (int i = m0 + 1 + tid; i < n; i += blockDim.x) v[i] = rk[i];
        __syncthreads();
        // p_i = beta (B v)_i for this block's rows, one warp per row
        const int r0 = m0 + ((rank - m0) % TRI_CTAS + TRI_CTAS) % TRI_CTAS;   // first own row >= m0
        for (int i = r0 + TRI_CTAS * warp; i < n; i += TRI_CTAS * nw) {
            const double *row = a + (size_t)i * n;
            double t = 0.0;
            for (int j = m0 + lane; j < n; j += 32) t = fma(row[j], v[j], t);
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) pg[i] = beta * t;
        }
        cluster_sync_all();
        double pv = 0.0;
        for (int i = m0 + tid; i < n; i += blockDim.x) pv = fma(pg[i], v[i], pv);
        pv = block_sum(pv);
        if (tid == 0) s_k = 0.5 * beta * pv;
        __syncthreads();
        const double K = s_k;
        for (int i = m0 + tid; i < n; i += blockDim.x) w[i] = fma(-K, v[i], pg[i]);
        __syncthreads();
        // this block's rows of B - v w^T - w v^T
        const int m = n - m0, nr = (n - r0 + TRI_CTAS - 1) / TRI_CTAS;
        for (int t = tid; t < nr * m; t += blockDim.x) {
            const int i = r0 + TRI_CTAS * (t / m), j = m0 + t % m;
            double *x = a + (size_t)i * n + j;
            *x = fma(-v[i], w[j], fma(-w[i], v[j], *x));
        }
        cluster_sync_all();
    }
    if (rank == 0 && tid == 0) {
        if (n >= 2) {
            d[n - 2] = a[(size_t)(n - 2) * n + (n - 2)];
            e[n - 2] = a[(size_t)(n - 1) * n + (n - 2)];
        }
        d[n - 1] = a[(size_t)(n - 1) * n + (n - 1)];
    }
}

// a double in block `rank`'s shared memory at the offset of `p` in this block's
__device__ __forceinline__ double ld_cluster(const double *p, uint32_t rank)
{
    const uint32_t la = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t ra;
    double v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(rank));
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(ra) : "memory");
    return v;
}

// Shared-memory bytes of tridiag_smem_kernel for order n: block r's rows
// (ceil(n / TRI_CTAS) of n doubles), v, w and the p of its rows.
size_t tri_smem_bytes(int n)
{
    const size_t R = ((size_t)n + TRI_CTAS - 1) / TRI_CTAS;
    return (R * (size_t)n + 2 * (size_t)n + R) * sizeof(double);
}

// The same reduction with the matrix held in the cluster's shared memory
// (orders whose rows fit: n <= 472): block r keeps the rows
// i = r mod TRI_CTAS (local row t = global row r + TRI_CTAS t), reads row k
// and the other blocks' p_i from their shared memory through the cluster's
// address space, and updates its own rows in place; the input C is only read.
__global__ void __cluster_dims__(TRI_CTAS, 1, 1) __launch_bounds__(TRI_THREADS)
    tridiag_smem_kernel(const double *__restrict__ C, int n, double *__restrict__ d, double *__restrict__ e)
{
    extern __shared__ double sh[];
    const int R = (n + TRI_CTAS - 1) / TRI_CTAS;
    double *rows = sh;                    // [R][n]
    double *v = rows + (size_t)R * n;     // [n]
    double *w = v + n;                    // [n]
    double *p = w + n;                    // [R], by local row
    __shared__ double s_alpha, s_beta, s_k;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int rank = (int)cluster_rank();
    const int nown = (n - rank + TRI_CTAS - 1) / TRI_CTAS;   // rows of this block (n > rank: n >= 3 here)
    for (int idx = tid; idx < nown * n; idx += blockDim.x) {
        const int t = idx / n, j = idx % n;
        rows[(size_t)t * n + j] = C[(size_t)(rank + TRI_CTAS * t) * n + j];
    }
    cluster_sync_all();
    for (int k = 0; k + 2 < n; k++) {
        const int m0 = k + 1;
        const uint32_t ok = (uint32_t)(k % TRI_CTAS);      // the block that holds row k
        const double *rk = rows + (size_t)(k / TRI_CTAS) * n;   // row k, at its offset in block ok
        double ss = 0.0;
        for (int i = m0 + 1 + tid; i < n; i += blockDim.x) {
            const double x = ld_cluster(rk + i, ok);
            v[i] = x;
            ss = fma(x, x, ss);
        }
        const double tail = block_sum(ss);
        if (tid == 0) {
            const double x0 = ld_cluster(rk + m0, ok);
            if (tail == 0.0) {
                s_alpha = x0;      // column already reduced: H = I
                s_beta = 0.0;
            } else {
                const double nx = sqrt(fma(x0, x0, tail));
                const double alpha = x0 > 0.0 ? -nx : nx;
                const double v0 = x0 - alpha;
                s_alpha = alpha;
                s_beta = 2.0 / fma(v0, v0, tail);   // 2 / (v.v)
                v[m0] = v0;
            }
            if ((uint32_t)rank == ok) d[k] = rk[k];
            if (rank == 0) e[k] = s_alpha;
        }
        __syncthreads();
        const double beta = s_beta;
        if (beta == 0.0) continue;   // nothing written in this column: no barrier needed
        // p_i = beta (B v)_i for this block's rows i >= m0, one warp per row
        const int t0 = (m0 - rank + TRI_CTAS - 1) / TRI_CTAS > 0 ? (m0 - rank + TRI_CTAS - 1) / TRI_CTAS : 0;
        for (int t = t0 + warp; t < nown; t += nw) {
            const double *row = rows + (size_t)t * n;
            double x = 0.0;
            for (int j = m0 + lane; j < n; j += 32) x = fma(row[j], v[j], x);
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) p[t] = beta * x;
        }
        cluster_sync_all();
        double pv = 0.0;
        for (int i = m0 + tid; i < n; i += blockDim.x) {
            const double pi = ld_cluster(p + i / TRI_CTAS, (uint32_t)(i % TRI_CTAS));
            w[i] = pi;
            pv = fma(pi, v[i], pv);
        }
        pv = block_sum(pv);
        if (tid == 0) s_k = 0.5 * beta * pv;
        __syncthreads();
        const double K = s_k;
        for (int i = m0 + tid; i < n; i += blockDim.x) w[i] = fma(-K, v[i], w[i]);   // p becomes w
        __syncthreads();
        const int m = n - m0, nr = nown - t0;
        for (int idx = tid; idx < nr * m; idx += blockDim.x) {
            const int t = t0 + idx / m, j = m0 + idx % m, i = rank + TRI_CTAS * t;
            double *x = rows + (size_t)t * n + j;
            *x = fma(-v[i], w[j], fma(-w[i], v[j], *x));
        }
        cluster_sync_all();
    }
    cluster_sync_all();   // no block leaves while another may still read its shared memory
    if (tid == 0) {
        const int i2 = n - 2, i1 = n - 1;
        if (i2 % TRI_CTAS == rank) d[i2] = rows[(size_t)(i2 / TRI_CTAS) * n + i2];
        if (i1 % TRI_CTAS == rank) {
            e[i2] = rows[(size_t)(i1 / TRI_CTAS) * n + i2];
            d[i1] = rows[(size_t)(i1 / TRI_CTAS) * n + i1];
        }
    }
}

// Number of eigenvalues below x of the tridiagonal T = (d, e) scaled so that
// its Gershgorin norm lies in [1, 2) (e2[i] = e[i]^2), without division: the
// continuants p_i of T - x I (its leading principal minors, p_{-1} = 1,
// p_i = (d_i - x) p_{i-1} - e2_{i-1} p_{i-2}) change sign exactly where the
// ratios q_i = p_i / p_{i-1} of the Sturm sequence are negative, and each step
// rounds like the ratio form's (one relative error on e2 p_{i-2}, one on the
// result), so the count is that of a matrix within a few ulps of T.  A zero
// p_i stands for the ratio -pivmin.  p_i and p_{i-1} are rescaled together by
// a power of two (exactly) whenever p_i leaves [2^-300, 2^300]; with
// |q_i| in [pivmin, 3 + 1 / pivmin] and pivmin = 2^-400 no step leaves the
// range of normal doubles.  Three FP64 operations per step where the ratio
// form needs a division (GB300's FP64 pipe is the bound).
__device__ int sturm_count(const double *d, const double *e2, int n, double x)
{
    constexpr double pivmin = 0x1p-400;
    double pm = 1.0, p = d[0] - x;
    if (p == 0.0) p = -pivmin;
    int c = p < 0.0;
    for (int i = 1; i < n; i++) {
        double pn = fma(d[i] - x, p, -(e2[i - 1] * pm));
        if (((__double2hiint(pn) & 0x7fffffff) | __double2loint(pn)) == 0) pn = -pivmin * p;
        c += (__double2hiint(pn) ^ __double2hiint(p)) < 0;   // the signs differ
        pm = p;
        p = pn;
        const int eb = (__double2hiint(p) >> 20) & 0x7ff;
        if (eb > 1023 + 300 || eb < 1023 - 300) {
            p = scalbn(p, 1023 - eb);
            pm = scalbn(pm, 1023 - eb);
        }
    }
    return c;
}

// eigenvalue i (ascending) by multisection on the Sturm count, one warp per
// eigenvalue: from the Gershgorin interval, each step the lanes j < 31 count
// the eigenvalues below lo + (j + 1)(hi - lo) / 32 and the bracket becomes
// the first of the 32 sub-intervals whose upper end counts more than i, so a
// step gains 5 bits where bisection gains 1 (the FP64 Sturm counts are
// spread over all SMs instead of one thread each); it stops when a step no
// longer shrinks the bracket (a few ulps), at most 64 steps.  The block stages
// T scaled by a power of two (exactly) to a norm in [1, 2) in shared memory.
constexpr int EIG_WARPS = 2;   // eigenvalues per block

__global__ void __launch_bounds__(32 * EIG_WARPS) multisect_kernel(const double *__restrict__ d,
                                                                   const double *__restrict__ e, int n,
                                                                   double *__restrict__ w)
{
    extern __shared__ double sde[];
    double *ds = sde, *e2s = sde + n;   // [n] each
    const int lane = threadIdx.x & 31, i = blockIdx.x * EIG_WARPS + (threadIdx.x >> 5);
    double lo = INFINITY, hi = -INFINITY, nrm = 0.0;
    for (int k = lane; k < n; k += 32) {
        const double r = (k > 0 ? fabs(e[k - 1]) : 0.0) + (k + 1 < n ? fabs(e[k]) : 0.0);
        lo = fmin(lo, d[k] - r);
        hi = fmax(hi, d[k] + r);
        nrm = fmax(nrm, fabs(d[k]) + r);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        nrm = fmax(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
    }
    const int ks = nrm > 0.0 ? ilogb(nrm) : 0;   // T / 2^ks has its norm in [1, 2)
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        ds[k] = scalbn(d[k], -ks);
        const double ek = k + 1 < n ? scalbn(e[k], -ks) : 0.0;
        e2s[k] = ek * ek;
    }
    __syncthreads();
    if (i >= n) return;   // whole warps, after the block's last barrier
    const double pad = 4e-16 * n;
    lo = scalbn(lo, -ks) - pad;
    hi = scalbn(hi, -ks) + pad;
    for (int it = 0; it < 64; it++) {
        const double step = (hi - lo) * (1.0 / 32.0);
        const double x = fmin(fma((double)(lane + 1), step, lo), hi);
        const bool above = lane < 31 && sturm_count(ds, e2s, n, x) > i;
        const unsigned mk = __ballot_sync(0xffffffffu, above);
        const int f = mk ? __ffs(mk) - 1 : 31;   // sub-interval f: (x_{f-1}, x_f]
        const double xf = __shfl_sync(0xffffffffu, x, f), xp = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
        const double nlo = f > 0 ? xp : lo, nhi = f < 31 ? xf : hi;
        if (!(nlo > lo || nhi < hi)) break;
        lo = nlo;
        hi = nhi;
    }
    if (lane == 0) w[i] = scalbn(0.5 * (lo + hi), ks);
}

int blocks_for(size_t n, int threads) { return (int)std::max<size_t>(1, std::min<size_t>((n + threads - 1) / threads, 152 * 16)); }

}  // namespace

cudaError_t launch_covcov(const double *A, const double *B, int nbin, int M_a, double M, int n_mock, double *var,
                          cudaStream_t s)
{
    const double w = B ? 0.5 / M_a : 0.0;
    const double c = B ? 0.5 / M_a - 1.0 / M : 0.0;
    covcov_kernel<<<blocks_for((size_t)nbin * nbin, 256), 256, 0, s>>>(A, B, nbin, w, c * c,
                                                                        1.0 / (double)(n_mock - 1), var);
    return cudaGetLastError();
}

size_t chi2_work_bytes() { return RED_BLOCKS * sizeof(double); }

cudaError_t launch_chi2(int mode, const double *X, const double *Y, const double *R, int nbin, int M_a, double M,
                        double *work, double *out, cudaStream_t s)
{
    double w = 0.0, c = 0.0;
    if (mode == 0 && Y) {
        w = 0.5 / M_a;
        c = 0.5 / M_a - 1.0 / M;
    }
    const int nb = std::min(RED_BLOCKS, blocks_for((size_t)nbin * nbin, RED_THREADS));
    chi2_partial<<<nb, RED_THREADS, 0, s>>>(mode, X, Y, R, nbin, w, c * c, work);
    chi2_final<<<1, RED_THREADS, 0, s>>>(work, nb, 1.0 / ((double)nbin * nbin), out);
    return cudaGetLastError();
}

size_t eig_work_bytes(int n) { return ((size_t)n * n + 3 * (size_t)n) * sizeof(double); }

cudaError_t launch_eigvalsh(const double *C, int n, double *work, double *w, cudaStream_t s)
{
    double *a = work, *d = work + (size_t)n * n, *e = d + n, *pg = e + n;
    cudaError_t err;
    const size_t sb = tri_smem_bytes(n);
    if (n >= 3 && sb <= (size_t)(226 << 10)) {
        // the matrix fits in the cluster's shared memory
        err = cudaFuncSetAttribute(tridiag_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
        if (err != cudaSuccess) return err;
        tridiag_smem_kernel<<<TRI_CTAS, TRI_THREADS, sb, s>>>(C, n, d, e);
    } else {
        err = cudaMemcpyAsync(a, C, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, s);
        if (err != cudaSuccess) return err;
        tridiag_kernel<<<TRI_CTAS, TRI_THREADS, 2 * (size_t)n * sizeof(double), s>>>(a, n, d, e, pg);
    }
    multisect_kernel<<<(n + EIG_WARPS - 1) / EIG_WARPS, 32 * EIG_WARPS, 2 * (size_t)n * sizeof(double), s>>>(d, e,
                                                                                                          n, w);
    return cudaGetLastError();
}

}  // namespace tpcf
