/*
 * CPU oracle: exact brute-force pair counts.  TEST INFRASTRUCTURE ONLY --
 * only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this; the product path never does.
 *
 * Pair counting of Sect. 2.1 (DD, DR_i and RR_i counts of the split
 * Landy-Szalay estimator) and Sect. 4.3 (binning in separation r and in mu,
 * the cosine of the angle between the line of sight and the pair
 * separation).  Every pair is visited (O(N^2)); no spatial structure.
 *
 * Positions arrive already quantised to unsigned integer grid coordinates
 * (structure-of-arrays [3][n]).  Distances are exact integers:
 *   periodic:  Delta_c = (int32)(u_a,c - u_b,c)   (two's complement minimum image)
 *   open:      Delta_c = (int64)u_a,c - (int64)u_b,c
 *   D2 = sum_c Delta_c^2                          (uint64, never overflows)
 * s-bin k holds T[k] <= D2 < T[k+1] (half-open), with T[] the squared bin
 * edges in grid units rounded up to integers (built by the Python side in
 * exact rational arithmetic).
 * mu-bin j (of n_mu uniform bins of |mu| on [0,1], the top edge closed) is the
 * largest j <= n_mu-1 with  n_mu^2 (Delta . l)^2 >= j^2 D2 |l|^2,  where l is
 * the line of sight: the x axis (plane-parallel, Sect. 4.1) or the pair
 * midpoint direction u_a + u_b - 2 u_obs.  D2 = 0 or l = 0 give mu = 0.
 * Products are evaluated in unsigned 128-bit integers; the caller has checked
 * that they fit.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

typedef unsigned __int128 u128;
typedef __int128 i128;

enum { GEOM_PERIODIC = 0, GEOM_OPEN = 1 };
enum { LOS_X = 0, LOS_MIDPOINT = 1 };

/* largest k with T[k] <= D2, or -1 when D2 is below T[0] or at/above T[n_s] */
static int s_bin_of(uint64_t D2, const uint64_t *T, int n_s)
{
    if (D2 < T[0] || D2 >= T[n_s]) return -1;
    int k = 0;
    while (k + 1 < n_s && T[k + 1] <= D2) k++;
    return k;
}

/* largest j in [0, n_mu-1] with n_mu^2 * num >= j^2 * den; den == 0 -> 0 */
static int mu_bin_of(u128 num, u128 den, int n_mu)
{
    if (n_mu <= 1 || den == 0) return 0;
    u128 lhs = (u128)(n_mu * n_mu) * num;
    int j = n_mu - 1;
    while (j > 0 && lhs < (u128)(j * j) * den) j--;
    return j;
}

static void pair_bin(const uint32_t *a, int64_t na, int64_t i,
                     const uint32_t *b, int64_t nb, int64_t j,
                     int geom, int los, const int64_t *obs,
                     int n_s, const uint64_t *T, int n_mu,
                     int64_t *hist, int64_t *unbinned)
{
    int64_t d[3];
    for (int c = 0; c < 3; c++) {
        uint32_t ua = a[(int64_t)c * na + i], ub = b[(int64_t)c * nb + j];
        if (geom == GEOM_PERIODIC) d[c] = (int32_t)(uint32_t)(ua - ub);
        else d[c] = (int64_t)ua - (int64_t)ub;
    }
    uint64_t D2 = 0;
    for (int c = 0; c < 3; c++) D2 += (uint64_t)(d[c] * d[c]);
    int k = s_bin_of(D2, T, n_s);
    if (k < 0) { (*unbinned)++; return; }
    int m = 0;
    if (n_mu > 1) {
        u128 num, den;
        if (los == LOS_X) {
            num = (u128)(uint64_t)(d[0] * d[0]);
            den = (u128)D2;
        } else {
            i128 l[3], dot = 0;
            u128 l2 = 0;
            for (int c = 0; c < 3; c++) {
                l[c] = (i128)a[(int64_t)c * na + i] + (i128)b[(int64_t)c * nb + j] - 2 * (i128)obs[c];
                dot += (i128)d[c] * l[c];
                l2 += (u128)(l[c] * l[c]);
            }
            u128 adot = (u128)(dot < 0 ? -dot : dot);
            num = adot * adot;
            den = (u128)D2 * l2;
        }
        m = mu_bin_of(num, den, n_mu);
    }
    hist[(int64_t)k * n_mu + m]++;
}

/*
 * Count pairs between catalogue a (na points) and catalogue b (nb points).
 * b == NULL: auto-count of a with itself over unordered pairs i < j.
 * hist[n_s * n_mu] (s-major) and *unbinned are overwritten.
 * obs: observer in grid units (used only for LOS_MIDPOINT).
 * Returns 0, or -1 when the per-thread scratch cannot be allocated.
 */
int oracle_count_pairs(const uint32_t *a, int64_t na, const uint32_t *b, int64_t nb,
                       int geom, int los, const int64_t *obs,
                       int n_s, const uint64_t *T, int n_mu,
                       int64_t *hist, int64_t *unbinned)
{
    const int auto_count = (b == NULL);
    if (auto_count) { b = a; nb = na; }
    const int64_t nbin = (int64_t)n_s * n_mu;
    memset(hist, 0, sizeof(int64_t) * (size_t)nbin);
    *unbinned = 0;
    /* one private histogram per thread, summed after the loop */
    const int nth = omp_get_max_threads();
    int64_t *priv = (int64_t *)calloc((size_t)nth * (size_t)(nbin + 1), sizeof(int64_t));
    if (!priv) return -1;

#pragma omp parallel num_threads(nth)
    {
        int64_t *h = priv + (size_t)omp_get_thread_num() * (size_t)(nbin + 1);
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < na; i++) {
            for (int64_t j = auto_count ? i + 1 : 0; j < nb; j++)
                pair_bin(a, na, i, b, nb, j, geom, los, obs, n_s, T, n_mu, h, &h[nbin]);
        }
    }
    for (int t = 0; t < nth; t++) {
        const int64_t *h = priv + (size_t)t * (size_t)(nbin + 1);
        for (int64_t x = 0; x < nbin; x++) hist[x] += h[x];
        *unbinned += h[nbin];
    }
    free(priv);
    return 0;
}
