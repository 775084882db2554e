// Chaining-mesh build: quantisation to integer grid coordinates, cell keys,
// a one-digit counting (radix) sort of every catalogue by cell, and the
// work-unit list of the pair counter.  All catalogues of all mocks are
// processed by the same launches.
//
// The grid-coordinate convention is the exact-count convention of the
// library (Sect. 2.1 pair counts are decided on these integers):
//   periodic: t = x / L; t -= floor(t); u = floor(t * 2^32), 2^32 -> 0
//   open:     t = (x - x0) / L, required in [0, 1); u = floor(t * 2^30)
// Each step is a single IEEE float64 operation with round-to-nearest, so the
// host and the device produce identical integers.
#include <algorithm>

#include "tpcf_internal.h"

namespace tpcf {

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ uint32_t quantize_periodic(double x, double L)
{
    double t = __ddiv_rn(x, L);
    t = __dsub_rn(t, floor(t));
    double v = floor(__dmul_rn(t, 4294967296.0));
    if (v >= 4294967296.0) v -= 4294967296.0;
    return (uint32_t)(unsigned long long)v;
}

// returns false when the position lies outside [0, 1) of the bounding cube
__device__ __forceinline__ bool quantize_open(double x, double x0, double L, uint32_t &u)
{
    double t = __ddiv_rn(__dsub_rn(x, x0), L);
    if (!(t >= 0.0) || !(t < 1.0)) { u = 0; return false; }
    u = (uint32_t)(unsigned long long)floor(__dmul_rn(t, 1073741824.0));
    return true;
}

__device__ __forceinline__ uint32_t cell_of(uint32_t u, int n_c, int bits)
{
    return (uint32_t)(((unsigned long long)u * (unsigned long long)n_c) >> bits);
}

__global__ void quantize_keys_kernel(const Cat *__restrict__ cats, int n_cat, int n_cells, int n_c, int bits,
                                     int geometry, double L, double ox, double oy, double oz,
                                     uint32_t n_total, uint32_t *__restrict__ uq,
                                     uint32_t *__restrict__ keys, uint32_t *__restrict__ cellcount,
                                     int *__restrict__ status)
{
    bool bad = false;
    for (int c = blockIdx.y; c < n_cat; c += gridDim.y) {
    const Cat cat = cats[c];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cat.n; i += gridDim.x * blockDim.x) {
        uint32_t u[3];
        if (cat.xyz) {
            const double *x = cat.xyz + 3ull * i;
            if (geometry == TPCF_PERIODIC) {
                u[0] = quantize_periodic(x[0], L);
                u[1] = quantize_periodic(x[1], L);
                u[2] = quantize_periodic(x[2], L);
            } else {
                bool ok = quantize_open(x[0], ox, L, u[0]);
                ok &= quantize_open(x[1], oy, L, u[1]);
                ok &= quantize_open(x[2], oz, L, u[2]);
                bad |= !ok;
            }
        } else {
            u[0] = cat.u32[i];
            u[1] = cat.u32[(size_t)cat.n + i];
            u[2] = cat.u32[2 * (size_t)cat.n + i];
            if (geometry == TPCF_OPEN && ((u[0] | u[1] | u[2]) >> 30)) {
                bad = true;
                u[0] = u[1] = u[2] = 0;
            }
        }
        const uint32_t cx = cell_of(u[0], n_c, bits), cy = cell_of(u[1], n_c, bits),
                       cz = cell_of(u[2], n_c, bits);
        const uint32_t key = (uint32_t)c * (uint32_t)n_cells + (cz * n_c + cy) * n_c + cx;
        const uint32_t p = cat.p0 + i;
        uq[p] = u[0];
        uq[(size_t)n_total + p] = u[1];
        uq[2 * (size_t)n_total + p] = u[2];
        keys[p] = key;
        atomicAdd(&cellcount[key], 1u);
    }
    }
    if (bad) atomicOr(status, STATUS_RANGE);
}

__global__ void scatter_kernel(const Cat *__restrict__ cats, int n_cat, int n_c, int bits,
                               const uint32_t *__restrict__ uq, const uint32_t *__restrict__ keys,
                               const uint32_t *__restrict__ cellstart, uint32_t *__restrict__ cursor,
                               const uint32_t *__restrict__ orig, uint32_t n_total,
                               uint32_t *__restrict__ us, float4 *__restrict__ pf, uint16_t *__restrict__ pcx)
{
    for (int c = blockIdx.y; c < n_cat; c += gridDim.y) {
    const Cat cat = cats[c];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cat.n; i += gridDim.x * blockDim.x) {
        const uint32_t p = cat.p0 + i;
        const uint32_t key = keys[p];
        const uint32_t pos = cellstart[key] + atomicAdd(&cursor[key], 1u);
        const uint32_t ux = uq[p], uy = uq[(size_t)n_total + p], uz = uq[2 * (size_t)n_total + p];
        us[pos] = ux;
        us[(size_t)n_total + pos] = uy;
        us[2 * (size_t)n_total + pos] = uz;
        const uint32_t cx = cell_of(ux, n_c, bits), cy = cell_of(uy, n_c, bits),
                       cz = cell_of(uz, n_c, bits);
        // offsets from the cell's integer lower corner are below one cell width
        const float fx = (float)(ux - orig[cx]), fy = (float)(uy - orig[cy]), fz = (float)(uz - orig[cz]);
        const float nh = -0.5f * __fmaf_rn(fz, fz, __fmaf_rn(fy, fy, __fmul_rn(fx, fx)));
        pf[pos] = make_float4(fx, fy, fz, nh);
        pcx[pos] = (uint16_t)cx;
    }
    }
}

// ---- exclusive scan of uint32 (reduce tiles, scan tile sums, scan tiles) ----

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_sums, uint32_t &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;  // inclusive warp prefix
    }
    __syncthreads();
    total = warp_sums[(blockDim.x >> 5) - 1];
    const uint32_t before = (warp > 0) ? warp_sums[warp - 1] : 0u;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(SCAN_THREADS) tile_reduce_kernel(const uint32_t *__restrict__ in, size_t n,
                                                                   uint32_t *__restrict__ sums)
{
    __shared__ uint32_t ws[32];
    const size_t base = (size_t)blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_ITEMS;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++)
        if (base + k < n) s += in[base + k];
    uint32_t total;
    block_exclusive_scan(s, ws, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_sums_kernel(uint32_t *sums, size_t n)
{
    __shared__ uint32_t ws[32];
    uint32_t carry = 0;
    for (size_t b = 0; b < n; b += SCAN_THREADS) {
        const size_t i = b + threadIdx.x;
        const uint32_t v = (i < n) ? sums[i] : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(v, ws, total);
        if (i < n) sums[i] = carry + ex;
        carry += total;
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) tile_scan_kernel(const uint32_t *__restrict__ in,
                                                                 uint32_t *__restrict__ out, size_t n,
                                                                 const uint32_t *__restrict__ sums)
{
    __shared__ uint32_t ws[32];
    const size_t base = (size_t)blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        v[k] = (base + k < n) ? in[base + k] : 0u;
        s += v[k];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(s, ws, total) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

// ---- work units ----

__global__ void unit_count_kernel(const Term *__restrict__ terms, int n_terms, const Cat *__restrict__ cats,
                                  int n_cells, const uint32_t *__restrict__ cellstart, int chunk,
                                  uint32_t *__restrict__ ucount)
{
    const size_t total = (size_t)n_terms * n_cells;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int t = (int)(i / n_cells), cell = (int)(i % n_cells);
        const size_t gk = (size_t)terms[t].cat_a * n_cells + cell;
        const uint32_t n = cellstart[gk + 1] - cellstart[gk];
        ucount[i] = (n + chunk - 1) / chunk;
    }
}

__global__ void unit_fill_kernel(const Term *__restrict__ terms, int n_terms, const Cat *__restrict__ cats,
                                 int n_cells, const uint32_t *__restrict__ cellstart, int chunk,
                                 const uint32_t *__restrict__ ustart, Unit *__restrict__ units)
{
    const size_t total = (size_t)n_terms * n_cells;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t u0 = ustart[i], u1 = ustart[i + 1];
        if (u0 == u1) continue;
        const int t = (int)(i / n_cells), cell = (int)(i % n_cells);
        const size_t gk = (size_t)terms[t].cat_a * n_cells + cell;
        const uint32_t s0 = cellstart[gk], s1 = cellstart[gk + 1];
        for (uint32_t j = 0; j < u1 - u0; j++) {
            Unit u;
            u.term = t;
            u.cell = cell;
            u.a0 = s0 + j * (uint32_t)chunk;
            u.a1 = min(s1, u.a0 + (uint32_t)chunk);
            units[u0 + j] = u;
        }
    }
}

int grid_for(size_t n, int threads, int cap)
{
    size_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (size_t)cap) b = cap;
    return (int)b;
}

// Counters of one pair-count launch (stats[8], see record_warp_span) added
// into a call's running total: sums, except the earliest start and latest end.
__global__ void stats_accum_kernel(const unsigned long long *__restrict__ st, unsigned long long *__restrict__ acc,
                                   int first)
{
    const int i = threadIdx.x;
    if (i >= 8) return;
    const unsigned long long v = st[i];
    acc[i] = first ? v : ((i == 4 || i == 5) ? (acc[i] > v ? acc[i] : v) : acc[i] + v);
}

}  // namespace

size_t scan_tmp_elems(size_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

cudaError_t launch_scan_u32(const uint32_t *in, uint32_t *out, size_t n, uint32_t *tmp, size_t tmp_n,
                            cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const size_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles > tmp_n) return cudaErrorInvalidValue;
    tile_reduce_kernel<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, tmp);
    scan_sums_kernel<<<1, SCAN_THREADS, 0, s>>>(tmp, tiles);
    tile_scan_kernel<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, tmp);
    return cudaGetLastError();
}

cudaError_t launch_quantize_keys(const Cat *cats, int n_cat, uint32_t max_n, const CountParams &p,
                                 double L, const double *origin, uint32_t n_total, uint32_t *uq,
                                 uint32_t *keys, uint32_t *cellcount, int *status, cudaStream_t s)
{
    if (n_cat == 0 || max_n == 0) return cudaSuccess;
    dim3 grid(grid_for(max_n, 256, 4096), std::min(n_cat, 65535));
    quantize_keys_kernel<<<grid, 256, 0, s>>>(cats, n_cat, p.n_cells, p.n_c, p.bits, p.geometry, L, origin[0],
                                              origin[1], origin[2], n_total, uq, keys, cellcount, status);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const Cat *cats, int n_cat, uint32_t max_n, const CountParams &p,
                           const uint32_t *uq, const uint32_t *keys, const uint32_t *cellstart,
                           uint32_t *cursor, const uint32_t *orig, uint32_t n_total, uint32_t *us,
                           float4 *pf, uint16_t *pcx, cudaStream_t s)
{
    if (n_cat == 0 || max_n == 0) return cudaSuccess;
    dim3 grid(grid_for(max_n, 256, 4096), std::min(n_cat, 65535));
    scatter_kernel<<<grid, 256, 0, s>>>(cats, n_cat, p.n_c, p.bits, uq, keys, cellstart, cursor, orig, n_total, us,
                                        pf, pcx);
    return cudaGetLastError();
}

cudaError_t launch_unit_count(const Term *terms, int n_terms, const Cat *cats, int n_cells,
                              const uint32_t *cellstart, int chunk, uint32_t *ucount, cudaStream_t s)
{
    const size_t total = (size_t)n_terms * n_cells;
    unit_count_kernel<<<grid_for(total, 256, 152 * 32), 256, 0, s>>>(terms, n_terms, cats, n_cells, cellstart,
                                                                      chunk, ucount);
    return cudaGetLastError();
}

cudaError_t launch_unit_fill(const Term *terms, int n_terms, const Cat *cats, int n_cells,
                             const uint32_t *cellstart, int chunk, const uint32_t *ustart, Unit *units,
                             cudaStream_t s)
{
    const size_t total = (size_t)n_terms * n_cells;
    unit_fill_kernel<<<grid_for(total, 256, 152 * 32), 256, 0, s>>>(terms, n_terms, cats, n_cells, cellstart,
                                                                     chunk, ustart, units);
    return cudaGetLastError();
}

cudaError_t launch_stats_accum(const unsigned long long *stats, unsigned long long *acc, int first, cudaStream_t s)
{
    stats_accum_kernel<<<1, 32, 0, s>>>(stats, acc, first);
    return cudaGetLastError();
}

}  // namespace tpcf
