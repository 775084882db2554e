// Binned pair counting on the chaining mesh (Sect. 2.1: DD, DR_i, RR_i
// counts; Sect. 4.3: bins in separation s and in mu).
//
// Work decomposition.  A unit is a chunk of the sorted points of one mesh
// cell A of catalogue a, to be paired with every point of catalogue b in the
// neighbourhood of A.  A warp owns a unit.  The neighbourhood is walked as
// rows of cells (dz, dy) whose x-runs are contiguous in the cell-sorted
// point order; each run is cut into tiles of 32*P b-points, one P-vector per
// lane, shifted into A's frame once per tile.  The a-points are then
// broadcast to the warp one at a time (uniform loads served by L1), so one
// load feeds 32*P pair tests.
//
// Per pair: FP32 d^2 from cell-relative coordinates and a compare with the
// top edge.  Pairs that may be in range are appended to a lane-private queue
// in shared memory; the queue is binned in bulk so that the binning code
// runs with every lane busy.  Binning looks up the s bin from the bit
// pattern of d^2 (each table slot spans at most one bin edge) and the mu bin
// from n_mu |mu| = n_mu |dx| / sqrt(d^2).  A pair whose d^2 or mu lies within
// the rigorous FP32 error band of a bin edge is rebinned exactly from the
// integer grid coordinates (64-bit squared distances, 128-bit mu test), so
// every count equals the integer definition bit for bit.
//
// Histograms are privatised per warp in shared memory (int32) and added to
// the caller's int64 histogram when the warp finishes a unit.
#include "plan.h"

namespace tpcf {

namespace {

constexpr int P = 4;          // b-points per lane
constexpr int QN = 16;        // queue slots per lane
constexpr float FAR = 3.0e18f;

typedef unsigned __int128 u128;
typedef __int128 i128;

struct Smem {
    int *hist;                 // [warps][nbin]
    float4 *queue;             // [warps][QN][32]
    uint16_t *table;           // [tab_n]
    uint32_t *orig;            // [n_c + 1]
    float *lo, *hi;            // [n_s + 1]
    unsigned long long *T;     // [n_s + 1]
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline size_t smem_layout(const CountParams &p, int warps, size_t *off)
{
    size_t o = 0;
    off[0] = o; o = align16(o + sizeof(unsigned long long) * (p.n_s + 1));   // T
    off[1] = o; o = align16(o + sizeof(float4) * (size_t)warps * QN * 32);    // queue
    off[2] = o; o = align16(o + sizeof(int) * (size_t)warps * p.nbin);       // hist
    off[3] = o; o = align16(o + sizeof(float) * (p.n_s + 1));                // lo
    off[4] = o; o = align16(o + sizeof(float) * (p.n_s + 1));                // hi
    off[5] = o; o = align16(o + sizeof(uint32_t) * (p.n_c + 1));             // orig
    off[6] = o; o = align16(o + sizeof(uint16_t) * p.tab_n);                 // table
    return o;
}

// Exact bin of the pair (ia, ib) from integer grid coordinates; -1 if unbinned.
__device__ __noinline__ int exact_bin(const CountParams &prm, const unsigned long long *T,
                                      const uint32_t *__restrict__ us, uint32_t N, uint32_t ia, uint32_t ib)
{
    long long d[3];
    uint32_t ua[3], ub[3];
    unsigned long long D2 = 0;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        ua[c] = us[(size_t)c * N + ia];
        ub[c] = us[(size_t)c * N + ib];
        d[c] = (prm.geometry == TPCF_PERIODIC) ? (long long)(int)(ua[c] - ub[c])
                                               : (long long)ua[c] - (long long)ub[c];
        D2 += (unsigned long long)(d[c] * d[c]);
    }
    const int n_s = prm.n_s;
    if (D2 < T[0] || D2 >= T[n_s]) return -1;
    int lo = 0, hi = n_s - 1;        // largest k with T[k] <= D2
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T[mid] <= D2) lo = mid; else hi = mid - 1;
    }
    const int k = lo;
    const int n_mu = prm.n_mu;
    int j = 0;
    if (n_mu > 1) {
        u128 num, den;
        if (prm.los == TPCF_LOS_X) {
            num = (u128)(unsigned long long)(d[0] * d[0]);
            den = (u128)D2;
        } else {
            i128 dot = 0;
            u128 l2 = 0;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const i128 l = (i128)ua[c] + (i128)ub[c] - 2 * (i128)prm.obs[c];
                dot += (i128)d[c] * l;
                l2 += (u128)(l * l);
            }
            const u128 ad = (u128)(dot < 0 ? -dot : dot);
            num = ad * ad;
            den = (u128)D2 * l2;
        }
        if (den != 0) {
            const u128 lhs = (u128)(unsigned)(n_mu * n_mu) * num;
            j = n_mu - 1;
            while (j > 0 && lhs < (u128)(unsigned)(j * j) * den) j--;
        }
    }
    return k * n_mu + j;
}

template <bool MU, bool MID>
struct Warp {
    const CountParams &prm;
    const Smem &sm;
    const Mesh &m;
    int *hist;         // this warp's histogram
    float4 *q;         // this warp's queue
    int lane;
    // unit state
    uint32_t a0, a1;
    float gx, gy, gz;  // 2 (corner(A) - observer), midpoint line of sight
    unsigned long long n_cand;
    unsigned n_exact, n_binned;

    __device__ Warp(const CountParams &p, const Smem &s, const Mesh &mm, int w, int l)
        : prm(p), sm(s), m(mm), lane(l), n_cand(0), n_exact(0), n_binned(0)
    {
        hist = s.hist + (size_t)w * p.nbin;
        q = s.queue + (size_t)w * QN * 32;
    }

    // Classify a queued pair; returns the bin, -1 (unbinned) or -2 (recheck exactly).
    __device__ __forceinline__ int classify(float d2, float dx, uint32_t ia, const float (&bx)[P],
                                            const float (&by)[P], const float (&bz)[P], int p) const
    {
        uint32_t key = __float_as_uint(d2) >> prm.tab_shift;
        key = max(key, prm.tab_key0) - prm.tab_key0;
        key = min(key, (uint32_t)(prm.tab_n - 1));
        const uint16_t c = sm.table[key];
        int k;
        bool amb = false;
        if (c & CODE_EDGE) {
            const int e = c & 0x7FFF;
            const float hi = sm.hi[e];
            k = (d2 >= hi) ? e : e - 1;
            amb = (d2 >= sm.lo[e]) && (d2 < hi);
        } else if (c == CODE_AMBIG) {
            return -2;
        } else {
            k = c;   // a bin, or CODE_DISCARD (>= n_s)
        }
        if (amb) return -2;
        if (k < 0 || k >= prm.n_s) return -1;
        if (!MU) return k;
        float t, beta;
        if (!MID) {
            const float r = rsqrtf(d2);
            t = fabsf(dx) * r * (float)prm.n_mu;
            beta = fmaf(prm.mu_c1, r, prm.mu_c2);
        } else {
            const float4 a = __ldg(m.pf + ia);
            float px = 0.f, py = 0.f, pz = 0.f;
#pragma unroll
            for (int i = 0; i < P; i++)
                if (i == p) { px = bx[i]; py = by[i]; pz = bz[i]; }
            const float ex = a.x - px, ey = a.y - py, ez = a.z - pz;
            const float lx = gx + a.x + px, ly = gy + a.y + py, lz = gz + a.z + pz;
            const float dot = fmaf(ez, lz, fmaf(ey, ly, ex * lx));
            const float l2 = fmaf(lz, lz, fmaf(ly, ly, lx * lx));
            const float rs = rsqrtf(d2), rl = rsqrtf(l2);
            t = fabsf(dot) * rs * rl * (float)prm.n_mu;
            beta = fmaf(prm.mu_c1, rs, fmaf(prm.mu_c3, rl, prm.mu_c2));
        }
        if (!(beta < 0.05f)) return -2;
        const float fl = floorf(t);
        const float f = t - fl;
        int j = (int)fl;
        const bool near_lo = !(f >= beta);
        const bool near_hi = !(f <= 1.0f - beta);
        if ((near_lo && j >= 1 && j <= prm.n_mu - 1) || (near_hi && j + 1 >= 1 && j + 1 <= prm.n_mu - 1))
            return -2;
        j = min(max(j, 0), prm.n_mu - 1);
        return k * prm.n_mu + j;
    }

    __device__ __forceinline__ void flush(int &qn, uint32_t base, const float (&bx)[P], const float (&by)[P],
                                          const float (&bz)[P])
    {
        const int qmax = __reduce_max_sync(0xffffffffu, (unsigned)qn);
        for (int k = 0; k < qmax; k++) {
            if (k < qn) {
                const float4 e = q[k * 32 + lane];
                const uint32_t ia = __float_as_uint(e.z);
                const int p = __float_as_int(e.w);
                int bin = classify(e.x, e.y, ia, bx, by, bz, p);
                if (bin == -2) {
                    bin = exact_bin(prm, sm.T, m.us, m.n_total, ia, base + lane + 32u * p);
                    n_exact++;
                }
                if (bin >= 0) {
                    atomicAdd(&hist[bin], 1);
                    n_binned++;
                }
            }
        }
        qn = 0;
        __syncwarp();
    }

    // All pairs (a in [a0, a1), b in [s0, s1)); b shifted into A's frame.
    // self: the b run is cell A itself in an auto count, keep ia < ib only.
    __device__ void run(uint32_t s0, uint32_t s1, uint32_t orig_ax, float sy, float sz, bool self)
    {
        for (uint32_t base = s0; base < s1; base += 32u * P) {
            float bx[P], by[P], bz[P];
#pragma unroll
            for (int p = 0; p < P; p++) {
                const uint32_t i = base + lane + 32u * p;
                if (i < s1) {
                    const float4 v = __ldg(m.pf + i);
                    const int cx = __float_as_int(v.w);
                    const float sx = (float)(int)(sm.orig[cx] - orig_ax);
                    bx[p] = __fadd_rn(v.x, sx);
                    by[p] = __fadd_rn(v.y, sy);
                    bz[p] = __fadd_rn(v.z, sz);
                } else {
                    bx[p] = by[p] = bz[p] = FAR;
                }
            }
            const uint32_t nb = min(s1 - base, 32u * P);
            n_cand += (unsigned long long)nb * (a1 - a0);
            int qn = 0;
            const float hit_max = prm.hit_max;
            for (uint32_t ia = a0; ia < a1; ia++) {
                const float4 a = __ldg(m.pf + ia);
#pragma unroll
                for (int p = 0; p < P; p++) {
                    const float dx = __fsub_rn(a.x, bx[p]);
                    const float dy = __fsub_rn(a.y, by[p]);
                    const float dz = __fsub_rn(a.z, bz[p]);
                    const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
                    bool hit = d2 < hit_max;
                    if (self) hit = hit && (ia < base + lane + 32u * p);
                    if (hit) {
                        q[qn * 32 + lane] = make_float4(d2, dx, __uint_as_float(ia), __int_as_float(p));
                        qn++;
                    }
                }
                if (__any_sync(0xffffffffu, qn > QN - P)) flush(qn, base, bx, by, bz);
            }
            if (__any_sync(0xffffffffu, qn > 0)) flush(qn, base, bx, by, bz);
        }
    }

    __device__ void flush_hist(long long *out)
    {
        __syncwarp();
        for (int b = lane; b < prm.nbin; b += 32) {
            const int v = hist[b];
            if (v) {
                atomicAdd((unsigned long long *)&out[b], (unsigned long long)(long long)v);
                hist[b] = 0;
            }
        }
        __syncwarp();
    }

    __device__ void unit(const Unit &un, const Term &tm)
    {
        const int n_c = prm.n_c;
        const int ax = un.cell % n_c, ay = (un.cell / n_c) % n_c, az = un.cell / (n_c * n_c);
        const bool periodic = prm.geometry == TPCF_PERIODIC;
        const uint32_t *cs = m.cellstart + (size_t)tm.cat_b * prm.n_cells;
        a0 = un.a0;
        a1 = un.a1;
        const uint32_t oax = sm.orig[ax], oay = sm.orig[ay], oaz = sm.orig[az];
        if (MID) {
            gx = 2.0f * (float)((long long)oax - prm.obs[0]);
            gy = 2.0f * (float)((long long)oay - prm.obs[1]);
            gz = 2.0f * (float)((long long)oaz - prm.obs[2]);
        }
        unsigned long long since_flush = 0;
        for (int r = 0; r < prm.n_rows; r++) {
            const int dz = prm.row_dz[r], dy = prm.row_dy[r], kx = prm.row_kx[r];
            if (tm.auto_pairs && (dz < 0 || (dz == 0 && dy < 0))) continue;
            int z = az + dz, y = ay + dy;
            if (periodic) {
                z = z < 0 ? z + n_c : (z >= n_c ? z - n_c : z);
                y = y < 0 ? y + n_c : (y >= n_c ? y - n_c : y);
            } else if (z < 0 || z >= n_c || y < 0 || y >= n_c) {
                continue;
            }
            const float sy = (float)(int)(sm.orig[y] - oay);
            const float sz = (float)(int)(sm.orig[z] - oaz);
            const uint32_t rowkey = ((uint32_t)z * n_c + (uint32_t)y) * n_c;
            int xlo = ax - kx, xhi = ax + kx;
            const unsigned long long before = n_cand;
            if (tm.auto_pairs && dz == 0 && dy == 0) {
                run(cs[rowkey + ax], cs[rowkey + ax + 1], oax, sy, sz, true);
                xlo = ax + 1;
            }
            if (xlo <= xhi) {
                if (periodic) {
                    if (xlo < 0) {
                        run(cs[rowkey + xlo + n_c], cs[rowkey + n_c], oax, sy, sz, false);
                        run(cs[rowkey], cs[rowkey + xhi + 1], oax, sy, sz, false);
                    } else if (xhi >= n_c) {
                        run(cs[rowkey + xlo], cs[rowkey + n_c], oax, sy, sz, false);
                        run(cs[rowkey], cs[rowkey + xhi - n_c + 1], oax, sy, sz, false);
                    } else {
                        run(cs[rowkey + xlo], cs[rowkey + xhi + 1], oax, sy, sz, false);
                    }
                } else {
                    xlo = max(xlo, 0);
                    xhi = min(xhi, n_c - 1);
                    if (xlo <= xhi) run(cs[rowkey + xlo], cs[rowkey + xhi + 1], oax, sy, sz, false);
                }
            }
            // int32 per-warp bins: drain well before 2^31 pairs can accumulate
            since_flush += n_cand - before;
            if (since_flush > (1ull << 30)) {
                flush_hist(tm.hist);
                since_flush = 0;
            }
        }
        flush_hist(tm.hist);
    }
};

template <bool MU, bool MID>
__global__ void __launch_bounds__(128) paircount_kernel(const __grid_constant__ CountParams prm, const Mesh m,
                                                        const Term *__restrict__ terms,
                                                        const Unit *__restrict__ units,
                                                        const uint32_t *__restrict__ n_units_p,
                                                        unsigned *__restrict__ claim,
                                                        const uint16_t *__restrict__ table_g,
                                                        unsigned long long *__restrict__ stats,
                                                        int persistent, int term_pl, int chunk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warps = blockDim.x >> 5;
    size_t off[7];
    smem_layout(prm, warps, off);
    Smem sm;
    sm.T = (unsigned long long *)(smem_raw + off[0]);
    sm.queue = (float4 *)(smem_raw + off[1]);
    sm.hist = (int *)(smem_raw + off[2]);
    sm.lo = (float *)(smem_raw + off[3]);
    sm.hi = (float *)(smem_raw + off[4]);
    sm.orig = (uint32_t *)(smem_raw + off[5]);
    sm.table = (uint16_t *)(smem_raw + off[6]);
    for (int i = threadIdx.x; i <= prm.n_s; i += blockDim.x) {
        sm.T[i] = prm.T[i];
        sm.lo[i] = prm.lo[i];
        sm.hi[i] = prm.hi[i];
    }
    for (int i = threadIdx.x; i <= prm.n_c; i += blockDim.x) sm.orig[i] = m.orig[i];
    for (int i = threadIdx.x; i < prm.tab_n; i += blockDim.x) sm.table[i] = table_g[i];
    for (int i = threadIdx.x; i < warps * prm.nbin; i += blockDim.x) sm.hist[i] = 0;
    __syncthreads();

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Warp<MU, MID> wp(prm, sm, m, w, lane);
    if (persistent) {
        const uint32_t n_units = *n_units_p;
        for (;;) {
            uint32_t u = 0;
            if (lane == 0) u = atomicAdd(claim, 1u);
            u = __shfl_sync(0xffffffffu, u, 0);
            if (u >= n_units) break;
            const Unit un = units[u];
            wp.unit(un, terms[un.term]);
        }
    } else {
        // one block per cell of catalogue a of one term; warps split the cell's chunks
        const Term tm = terms[term_pl];
        const int cell = blockIdx.x;
        const size_t gk = (size_t)tm.cat_a * prm.n_cells + cell;
        const uint32_t s0 = m.cellstart[gk], s1 = m.cellstart[gk + 1];
        for (uint32_t a = s0 + (uint32_t)w * chunk; a < s1; a += (uint32_t)warps * chunk) {
            Unit un;
            un.term = term_pl;
            un.cell = cell;
            un.a0 = a;
            un.a1 = min(s1, a + (uint32_t)chunk);
            wp.unit(un, tm);
        }
    }
    // work statistics
    unsigned long long ex = wp.n_exact, bn = wp.n_binned;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ex += __shfl_down_sync(0xffffffffu, ex, o);
        bn += __shfl_down_sync(0xffffffffu, bn, o);
    }
    if (lane == 0) {
        atomicAdd(&stats[0], wp.n_cand);
        atomicAdd(&stats[1], bn);
        atomicAdd(&stats[2], ex);
    }
}

template <bool MU, bool MID>
void *kernel_ptr()
{
    return (void *)paircount_kernel<MU, MID>;
}

void *select_kernel(const CountParams &p)
{
    const bool mu = p.n_mu > 1;
    const bool mid = mu && p.los == TPCF_LOS_MIDPOINT;
    if (!mu) return kernel_ptr<false, false>();
    if (!mid) return kernel_ptr<true, false>();
    return kernel_ptr<true, true>();
}

}  // namespace

int paircount_smem_bytes(const CountParams &p, int warps_per_block)
{
    size_t off[7];
    return (int)smem_layout(p, warps_per_block, off);
}

cudaError_t paircount_set_attrs(const CountParams &p, int smem_bytes)
{
    return cudaFuncSetAttribute(select_kernel(p), cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
}

int paircount_max_blocks_per_sm(const CountParams &p, int warps_per_block, int smem_bytes)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, select_kernel(p), warps_per_block * 32, smem_bytes) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_paircount(const CountParams &p, const Mesh &m, const Term *terms, const Cat *cats,
                             const Unit *units, const uint32_t *n_units, unsigned *claim,
                             const uint16_t *table, unsigned long long *stats, int *status,
                             const PairLaunch &pl, cudaStream_t s)
{
    (void)cats;
    (void)status;
    const int chunk = UNIT_CHUNK;
    void *args[] = {(void *)&p,      (void *)&m,     (void *)&terms,      (void *)&units,
                    (void *)&n_units, (void *)&claim, (void *)&table,     (void *)&stats,
                    (void *)&pl.persistent, (void *)&pl.term, (void *)&chunk};
    return cudaLaunchKernel(select_kernel(p), dim3(pl.blocks), dim3(pl.warps_per_block * 32), args,
                            (size_t)pl.smem_bytes, s);
}

}  // namespace tpcf
