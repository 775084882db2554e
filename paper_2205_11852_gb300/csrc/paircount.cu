// Binned pair counting on the chaining mesh (Sect. 2.1: DD, DR_i, RR_i
// counts; Sect. 4.3: bins in separation s and in mu).
//
// Work decomposition.  A unit is a chunk of at most 256 sorted points of one
// mesh cell A of catalogue a, to be paired with every point of catalogue b in
// the neighbourhood of A.  A thread block owns a unit: the a-chunk and the
// histogram live in shared memory, and the warps share the b side.  The
// neighbourhood is walked as rows of cells (dz, dy) whose x-runs are
// contiguous in the cell-sorted point order; every run is cut into tiles of
// 32*P b-points, and the tiles are dealt to the warps.  A warp loads its tile
// once, one P-vector per lane, shifted into A's frame, then streams the
// a-chunk past it by broadcast shared-memory loads.
//
// Per pair, a dot-product form of the range test,
//     a.b' - |a|^2/2  >=  (|b'|^2 - H)/2 - margin,
// costs three FMAs and one compare (|a|^2/2 is stored with the point,
// (|b'|^2 - H)/2 is per lane), with a margin that makes it a superset of the
// direct FP32 test d2 < H.  A passing pair appends a 16-bit entry (a index,
// b slot) to a lane-private queue in shared memory, branch-free.  Queues are
// binned in bulk: the direct FP32 d2 and dx are recomputed, the s bin comes
// from a table indexed by the bit pattern of d2 (one compare against the
// band of the next edge), the mu bin from n_mu |dx| / sqrt(d2).  A pair whose
// d2 or mu lies within the rigorous FP32 error band of a bin edge is rebinned
// exactly from the integer grid coordinates (64-bit squared distances,
// 128-bit mu test), so every count equals the integer definition bit for bit.
#include "plan.h"

namespace tpcf {

namespace {

constexpr int P = 4;            // b-points per lane
constexpr int TILE = 32 * P;    // b-points per warp tile
constexpr int QN = 24;          // queue slots per lane (16-bit entries)
constexpr int WARPS = 8;        // warps per block
constexpr int MAX_SEGS = 2 * MAX_ROWS + 2;

typedef unsigned __int128 u128;
typedef __int128 i128;

// A run of b-points: cells x0..x1 of one neighbour row, contiguous in the
// cell-sorted order.  Runs are concatenated, and the concatenation is cut
// into full tiles, so a tile may span several rows.
struct Seg {
    uint32_t s0;           // first b index
    uint32_t off0;         // offset of s0 in the concatenation of the unit's runs
    float sy, sz;          // row shift into A's frame
};

struct Smem {
    float4 *a;                 // [UNIT_CHUNK]
    int *hist;                 // [nbin]
    uint16_t *queue;           // [WARPS][QN][32]
    uint16_t *compact;         // [WARPS][QN * 32]
    float4 *bcopy;             // [WARPS][P][32]: b' in A's frame, .w = b index (bits)
    int16_t *table;            // [tab_n]
    float2 *lohi;              // [n_s + 2]
    uint32_t *orig;            // [n_c + 1]
    unsigned long long *T;     // [n_s + 1]
    Seg *segs;                 // [MAX_SEGS + 1], the last one a sentinel
    int *misc;                 // [8]: unit, n_segs, packed points, next tile, self s0, self s1
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline size_t smem_layout(const CountParams &p, size_t *off)
{
    size_t o = 0;
    off[0] = o; o = align16(o + sizeof(unsigned long long) * (p.n_s + 1));  // T
    off[1] = o; o = align16(o + sizeof(float4) * UNIT_CHUNK);              // a chunk
    off[2] = o; o = align16(o + sizeof(float4) * WARPS * P * 32);           // b copies
    off[3] = o; o = align16(o + sizeof(uint16_t) * WARPS * QN * 32 * 2);    // queues + compacted copies
    off[4] = o; o = align16(o + sizeof(int) * p.nbin);                      // histogram
    off[5] = o; o = align16(o + sizeof(float2) * (p.n_s + 2));              // edge bands
    off[6] = o; o = align16(o + sizeof(uint32_t) * (p.n_c + 1));            // cell corners
    off[7] = o; o = align16(o + sizeof(int16_t) * (p.linear ? 0 : p.tab_n)); // s table
    off[8] = o; o = align16(o + sizeof(Seg) * (MAX_SEGS + 1));              // segments
    off[9] = o; o = align16(o + sizeof(int) * 8);
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

__device__ __forceinline__ uint32_t warp_exclusive_sum(uint32_t v, int lane, uint32_t &total)
{
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// MUFU reciprocal square root without denormal handling (relative error
// within 2 ulp); every use carries that error in its ambiguity band
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 32-bit shared-memory accesses (addresses from __cvta_generic_to_shared)
__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
// 16-bit shared accesses through 32-bit registers (the load zero-extends,
// the store keeps the low half)
__device__ __forceinline__ void sts16(uint32_t a, uint32_t v)
{
    asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t lds16(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
// queue push: store v at the head slot; advance the head (one 64-byte slot
// row) only when t >= h
__device__ __forceinline__ void push_if_ge(uint32_t &head, uint32_t v, float t, float h)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ge.f32 p, %1, %2;\n\t"
        "st.shared.u16 [%0], %3;\n\t"
        "@p add.u32 %0, %0, 64;\n\t}"
        : "+r"(head)
        : "f"(t), "f"(h), "r"(v)
        : "memory");
}
__device__ __forceinline__ float4 lds128(uint32_t a)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a)
                 : "memory");
    return v;
}
__device__ __forceinline__ void red_inc(uint32_t a)
{
    asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(a) : "memory");
}
// histogram increment when bin >= 0, without a branch
__device__ __forceinline__ void red_inc_if(uint32_t base, int bin)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .u32 a;\n\t"
        "setp.ge.s32 p, %1, 0;\n\t"
        "mad.lo.u32 a, %1, 4, %0;\n\t"
        "@p red.shared.add.u32 [a], 1;\n\t}" ::"r"(base),
        "r"(bin)
        : "memory");
}
// 16-bit shared load when live (else 0), without a branch
__device__ __forceinline__ uint32_t lds16_if(uint32_t a, bool live)
{
    uint32_t v;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %2, 0;\n\t"
        "mov.u32 %0, 0;\n\t"
        "@p ld.shared.u16 %0, [%1];\n\t}"
        : "=r"(v)
        : "r"(a), "r"((int)live)
        : "memory");
    return v;
}
// 16-bit shared store when pred, without a branch
__device__ __forceinline__ void sts16_if(uint32_t a, uint32_t v, bool pred)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %2, 0;\n\t"
        "@p st.shared.u16 [%0], %1;\n\t}" ::"r"(a),
        "r"(v), "r"((int)pred)
        : "memory");
}

// Binning constants, copied from the launch parameters into registers once.
struct BinConst {
    float tab_bias, inv_nmu2, s_scale, s_c0, s_c1, mu_c1, mu_c2, mu_c3, hit_max, dot_margin;
    uint32_t tab_key0, tab_last;
    int tab_shift, n_s, n_mu;
};

template <bool MU, bool MID, bool LIN>
struct Ctx {
    const CountParams &prm;
    const Smem &sm;
    const Mesh &m;
    BinConst c;
    int lane, warp;
    uint32_t q;                // this lane's queue column (shared address of slot 0)
    uint32_t cq;               // this warp's compacted queue (shared address)
    uint32_t bc;               // this warp's b copies (shared address; .w: b index)
    uint32_t abase;            // the a-chunk (shared address)
    uint32_t hbase;            // the block histogram (shared address)
    uint32_t a0, na;           // current unit's a-chunk
    float gx, gy, gz;          // 2 (corner(A) - observer), midpoint line of sight
    unsigned n_exact, n_binned;

    // Bin of a queued pair: >= 0, -1 (not binned) or -2 (recheck exactly).
    // Straight-line code: every lane runs the same instructions.
    __device__ __forceinline__ int classify(float d2, float dx, const float4 &a, const float4 &b) const
    {
        const float big = 12582912.0f;   // 1.5 * 2^23: x + big rounds x to an integer
        bool amb = false, valid;
        int k;
        float r = 0.0f;
        if (LIN) {
            // s bin = floor(u), u = sqrt(d2) / (q ds); ambiguous near an interior
            // edge or near s_max
            r = rsqrt_approx(__fmul_rn(d2, c.inv_nmu2));      // n_mu / sqrt(d2)
            const float u = __fmul_rn(__fmul_rn(d2, r), c.s_scale);
            const float mf = __fadd_rn(u, big);
            const int ki = __float_as_int(mf) - 0x4B400000;
            const float ds = __fsub_rn(u, __fsub_rn(mf, big));
            // near an edge (or NaN: d2 = 0).  The s = 0 edge needs no recheck
            // but costs nothing to include; s_max is an edge like the others.
            amb = !(fabsf(ds) >= __fmaf_rn(c.s_c1, u, c.s_c0));
            k = ki - (ds < 0.0f ? 1 : 0);
            valid = (unsigned)k < (unsigned)c.n_s;
        } else {
            const uint32_t key = min((__float_as_uint(__fadd_rn(d2, c.tab_bias)) >> c.tab_shift) - c.tab_key0,
                                     c.tab_last);
            k = sm.table[key];
            amb = (k == CODE_AMBIG);
            k = amb ? -1 : k;
            const float2 lh = sm.lohi[k + 1];
            const bool ge_hi = d2 >= lh.y;
            amb |= (d2 >= lh.x) && !ge_hi;
            k += ge_hi ? 1 : 0;
            valid = (unsigned)k < (unsigned)c.n_s;
        }
        int bin = k;
        if (MU) {
            float t, beta;
            if (!MID) {
                if (!LIN) r = rsqrt_approx(__fmul_rn(d2, c.inv_nmu2));   // n_mu / sqrt(d2)
                t = __fmul_rn(fabsf(dx), r);
                beta = __fmaf_rn(c.mu_c1, r, c.mu_c2);
            } else {
                const float ex = __fsub_rn(a.x, b.x), ey = __fsub_rn(a.y, b.y), ez = __fsub_rn(a.z, b.z);
                const float lx = __fadd_rn(__fadd_rn(gx, a.x), b.x);
                const float ly = __fadd_rn(__fadd_rn(gy, a.y), b.y);
                const float lz = __fadd_rn(__fadd_rn(gz, a.z), b.z);
                const float dot = __fmaf_rn(ez, lz, __fmaf_rn(ey, ly, __fmul_rn(ex, lx)));
                const float l2 = __fmaf_rn(lz, lz, __fmaf_rn(ly, ly, __fmul_rn(lx, lx)));
                const float rs = rsqrt_approx(d2), rl = rsqrt_approx(l2);
                t = __fmul_rn(__fmul_rn(__fmul_rn(fabsf(dot), rs), rl), (float)c.n_mu);
                beta = __fmaf_rn(c.mu_c1, rs, __fmaf_rn(c.mu_c3, rl, c.mu_c2));
            }
            // the pair is ambiguous when t = n_mu |mu| (>= 0) lies within beta
            // of an integer (a mu edge; 0 and n_mu need no recheck but cost
            // nothing to include), or is NaN (d2 = 0)
            const float mf = __fadd_rn(t, big);
            const int mi = __float_as_int(mf) - 0x4B400000;
            const float d = __fsub_rn(t, __fsub_rn(mf, big));
            amb |= !(fabsf(d) >= beta);
            const int j = min(mi - (d < 0.0f ? 1 : 0), c.n_mu - 1);   // mu = 1 in the top bin
            bin = k * c.n_mu + j;
        }
        return amb ? -2 : (valid ? bin : -1);
    }

    // Bin of queue entry v (a index | b copy index << 8).
    __device__ __forceinline__ int bin_of(uint32_t v) const
    {
        const float4 a = lds128(abase + 16u * (v & 255u));
        const float4 b = lds128(bc + 16u * (v >> 8));
        const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y), dz = __fsub_rn(a.z, b.z);
        const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
        return classify(d2, dx, a, b);
    }

    // Bin every queued pair.  The lanes' queues are first packed into one
    // warp-contiguous list (a index | b copy index << 8), so that the binning
    // loop runs with all lanes busy whatever the spread of per-lane counts.
    // Pairs that need the exact recheck are rechecked at the end.  n = this
    // lane's count.
    __device__ __forceinline__ void flush(uint32_t n)
    {
        uint32_t total;
        const uint32_t pos = warp_exclusive_sum(n, lane, total);
        const uint32_t nmax = __reduce_max_sync(0xffffffffu, n);
        for (uint32_t k = 0; k < nmax; k++) {
            const bool mine = k < n;
            const uint32_t v = lds16_if(q + k * 64u, mine);   // a index | (p * 32 + lane) << 8
            sts16_if(cq + 2u * (pos + k), v, mine);
        }
        __syncwarp();
        uint32_t n_amb = 0;
        const uint32_t lt = (1u << lane) - 1u;
        // two entries per lane per pass (independent work for the scheduler)
        for (uint32_t w0 = 0; w0 < total; w0 += 64) {
            const uint32_t e0 = w0 + lane, e1 = e0 + 32u;
            const bool live0 = e0 < total, live1 = e1 < total;
            const uint32_t v0 = lds16_if(cq + 2u * e0, live0);
            const uint32_t v1 = lds16_if(cq + 2u * e1, live1);
            int bin0 = bin_of(v0), bin1 = bin_of(v1);   // dead slots read entry 0: in bounds, discarded
            bin0 = live0 ? bin0 : -1;
            bin1 = live1 ? bin1 : -1;
            red_inc_if(hbase, bin0);
            red_inc_if(hbase, bin1);
            const unsigned am0 = __ballot_sync(0xffffffffu, bin0 == -2);
            const unsigned am1 = __ballot_sync(0xffffffffu, bin1 == -2);
            if (am0 | am1) {
                // rare: keep the entries for the exact recheck, written over
                // entries this loop has already consumed
                __syncwarp();
                sts16_if(cq + 2u * (n_amb + __popc(am0 & lt)), v0, bin0 == -2);
                n_amb += __popc(am0);
                sts16_if(cq + 2u * (n_amb + __popc(am1 & lt)), v1, bin1 == -2);
                n_amb += __popc(am1);
            }
        }
        __syncwarp();
        for (uint32_t e = lane; e < n_amb; e += 32) {
            const uint32_t v = lds16(cq + 2u * e);
            const float4 b = lds128(bc + 16u * (v >> 8));
            const int bin = exact_bin(prm, sm.T, m.us, m.n_total, a0 + (v & 255u), __float_as_uint(b.w));
            n_exact++;
            if (bin >= 0) red_inc(hbase + 4u * (uint32_t)bin);
        }
        __syncwarp();
    }

    // Load one b-point into lane registers (shifted into A's frame) and into
    // the warp's b copies used by the flush.
    __device__ __forceinline__ void load_b(int p, bool ok, uint32_t i, float sy, float sz, uint32_t orig_ax,
                                           float (&bx)[P], float (&by)[P], float (&bz)[P], float (&hb)[P]) const
    {
        if (ok) {
            const float4 v = __ldg(m.pf + i);
            const int cx = m.pcx[i];
            const float sx = (float)(int)(sm.orig[cx] - orig_ax);
            bx[p] = __fadd_rn(v.x, sx);
            by[p] = __fadd_rn(v.y, sy);
            bz[p] = __fadd_rn(v.z, sz);
            const float b2 = __fmaf_rn(bz[p], bz[p], __fmaf_rn(by[p], by[p], __fmul_rn(bx[p], bx[p])));
            hb[p] = __fsub_rn(__fmul_rn(0.5f, __fsub_rn(b2, c.hit_max)), c.dot_margin);
        } else {
            bx[p] = by[p] = bz[p] = 0.0f;
            hb[p] = __int_as_float(0x7f800000);   // +inf: never passes
            i = 0;
        }
        asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(bc + 16u * (uint32_t)(p * 32 + lane)),
                     "f"(bx[p]), "f"(by[p]), "f"(bz[p]), "f"(__uint_as_float(i))
                     : "memory");
    }

    // all pairs of the a-chunk with one tile of b-points: the self cell of an
    // auto count (SELF, indices base..s1) or a packed tile at offset o_base of
    // the concatenated runs (n_seg runs, total points).
    template <bool SELF>
    __device__ __forceinline__ void tile(uint32_t base, uint32_t s1, uint32_t o_base, int n_seg, uint32_t total,
                                         uint32_t orig_ax)
    {
        float bx[P], by[P], bz[P], hb[P];
        if (SELF) {
#pragma unroll
            for (int p = 0; p < P; p++) {
                const uint32_t i = base + lane + 32u * p;
                load_b(p, i < s1, i, 0.0f, 0.0f, orig_ax, bx, by, bz, hb);
            }
        } else {
            // locate the run of this lane's first point, then walk forward
            const uint32_t o0 = o_base + lane;
            int lo = 0, hi = n_seg - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (sm.segs[mid].off0 <= o0) lo = mid; else hi = mid - 1;
            }
            int g = lo;
#pragma unroll
            for (int p = 0; p < P; p++) {
                const uint32_t o = o0 + 32u * p;
                while (g + 1 < n_seg && sm.segs[g + 1].off0 <= o) g++;
                const Seg sg = sm.segs[g];
                load_b(p, o < total, sg.s0 + (o - sg.off0), sg.sy, sg.sz, orig_ax, bx, by, bz, hb);
            }
        }
        __syncwarp();
        // Every candidate writes the head slot of the lane's queue column; only
        // a hit advances the head (64 bytes: one slot of 32 lanes), so the
        // stores stay branch-free.  A flush comes before 2P more pushes could
        // run past QN slots.
        uint32_t head = q;
        const uint32_t lim = q + (uint32_t)(QN - 2 * P) * 64u;
        const uint32_t ib0 = base + lane;   // used by SELF tiles only
        const uint32_t lane8 = (uint32_t)lane << 8;
        uint32_t ai = 0;
        for (; ai + 1 < na; ai += 2) {
            const float4 a = lds128(abase + 16u * ai), cc = lds128(abase + 16u * (ai + 1));
#pragma unroll
            for (int p = 0; p < P; p++) {
                const float t = __fmaf_rn(a.x, bx[p], __fmaf_rn(a.y, by[p], __fmaf_rn(a.z, bz[p], a.w)));
                const float h = (!SELF || a0 + ai < ib0 + 32u * p) ? hb[p] : INFINITY;
                push_if_ge(head, (ai | lane8) | (uint32_t)(p << 13), t, h);   // kept only on a hit
            }
#pragma unroll
            for (int p = 0; p < P; p++) {
                const float t = __fmaf_rn(cc.x, bx[p], __fmaf_rn(cc.y, by[p], __fmaf_rn(cc.z, bz[p], cc.w)));
                const float h = (!SELF || a0 + ai + 1 < ib0 + 32u * p) ? hb[p] : INFINITY;
                push_if_ge(head, ((ai + 1) | lane8) | (uint32_t)(p << 13), t, h);
            }
            if (__any_sync(0xffffffffu, head > lim)) {
                flush((head - q) >> 6);
                head = q;
            }
        }
        if (ai < na) {
            const float4 a = lds128(abase + 16u * ai);
#pragma unroll
            for (int p = 0; p < P; p++) {
                const float t = __fmaf_rn(a.x, bx[p], __fmaf_rn(a.y, by[p], __fmaf_rn(a.z, bz[p], a.w)));
                const float h = (!SELF || a0 + ai < ib0 + 32u * p) ? hb[p] : INFINITY;
                push_if_ge(head, (ai | lane8) | (uint32_t)(p << 13), t, h);
            }
        }
        if (__any_sync(0xffffffffu, head != q)) flush((head - q) >> 6);
    }
};

// The unit's b runs, built by one warp (one lane per neighbour row): the
// self cell of an auto count apart, every other run concatenated in row order
// with its offset in the concatenation.
__device__ void build_segments(const CountParams &prm, const Smem &sm, const Mesh &m, const Term &tm, int cell,
                               int lane)
{
    const int n_c = prm.n_c;
    const int ax = cell % n_c, ay = (cell / n_c) % n_c, az = cell / (n_c * n_c);
    const bool periodic = prm.geometry == TPCF_PERIODIC;
    const uint32_t *cs = m.cellstart + (size_t)tm.cat_b * prm.n_cells;
    const uint32_t oay = sm.orig[ay], oaz = sm.orig[az];
    uint32_t ns_total = 0, pts_total = 0;
    if (lane == 0) {
        sm.misc[4] = 0;
        sm.misc[5] = 0;
    }
    __syncwarp();
    for (int r0 = 0; r0 < prm.n_rows; r0 += 32) {
        const int r = r0 + lane;
        uint32_t s0[2], s1[2];
        int nl = 0;
        float sy = 0.f, sz = 0.f;
        if (r < prm.n_rows) {
            const int dz = prm.row_dz[r], dy = prm.row_dy[r], kx = prm.row_kx[r];
            bool use = !(tm.auto_pairs && (dz < 0 || (dz == 0 && dy < 0)));
            int z = az + dz, y = ay + dy;
            if (periodic) {
                z = z < 0 ? z + n_c : (z >= n_c ? z - n_c : z);
                y = y < 0 ? y + n_c : (y >= n_c ? y - n_c : y);
            } else if (z < 0 || z >= n_c || y < 0 || y >= n_c) {
                use = false;
            }
            if (use) {
                sy = (float)(int)(sm.orig[y] - oay);
                sz = (float)(int)(sm.orig[z] - oaz);
                const uint32_t rowkey = ((uint32_t)z * n_c + (uint32_t)y) * n_c;
                int xlo = ax - kx, xhi = ax + kx;
                auto add = [&](uint32_t a, uint32_t b) {
                    if (b > a) {
                        s0[nl] = a;
                        s1[nl] = b;
                        nl++;
                    }
                };
                if (tm.auto_pairs && dz == 0 && dy == 0) {
                    sm.misc[4] = (int)cs[rowkey + ax];
                    sm.misc[5] = (int)cs[rowkey + ax + 1];
                    xlo = ax + 1;
                }
                if (xlo <= xhi) {
                    if (periodic) {
                        if (xlo < 0) {
                            add(cs[rowkey + xlo + n_c], cs[rowkey + n_c]);
                            add(cs[rowkey], cs[rowkey + xhi + 1]);
                        } else if (xhi >= n_c) {
                            add(cs[rowkey + xlo], cs[rowkey + n_c]);
                            add(cs[rowkey], cs[rowkey + xhi - n_c + 1]);
                        } else {
                            add(cs[rowkey + xlo], cs[rowkey + xhi + 1]);
                        }
                    } else {
                        xlo = max(xlo, 0);
                        xhi = min(xhi, n_c - 1);
                        if (xlo <= xhi) add(cs[rowkey + xlo], cs[rowkey + xhi + 1]);
                    }
                }
            }
        }
        uint32_t pl = 0;
        for (int i = 0; i < nl; i++) pl += s1[i] - s0[i];
        uint32_t n_all, p_all;
        const uint32_t n_ex = warp_exclusive_sum((uint32_t)nl, lane, n_all);
        uint32_t p_ex = warp_exclusive_sum(pl, lane, p_all);
        for (int i = 0; i < nl; i++) {
            Seg g;
            g.s0 = s0[i];
            g.off0 = pts_total + p_ex;
            g.sy = sy;
            g.sz = sz;
            sm.segs[ns_total + n_ex + i] = g;
            p_ex += s1[i] - s0[i];
        }
        ns_total += n_all;
        pts_total += p_all;
    }
    if (lane == 0) {
        sm.misc[1] = (int)ns_total;
        sm.misc[2] = (int)pts_total;
    }
}

template <bool MU, bool MID, bool LIN>
__global__ void __launch_bounds__(WARPS * 32, 4) paircount_kernel(const __grid_constant__ CountParams prm, const Mesh m,
                                                                const Term *__restrict__ terms,
                                                                const Unit *__restrict__ units,
                                                                const uint32_t *__restrict__ n_units_p,
                                                                unsigned *__restrict__ claim,
                                                                const int16_t *__restrict__ table_g,
                                                                unsigned long long *__restrict__ stats,
                                                                int persistent, int term_pl, int chunk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    size_t off[10];
    smem_layout(prm, off);
    Smem sm;
    sm.T = (unsigned long long *)(smem_raw + off[0]);
    sm.a = (float4 *)(smem_raw + off[1]);
    sm.bcopy = (float4 *)(smem_raw + off[2]);
    sm.queue = (uint16_t *)(smem_raw + off[3]);
    sm.hist = (int *)(smem_raw + off[4]);
    sm.lohi = (float2 *)(smem_raw + off[5]);
    sm.orig = (uint32_t *)(smem_raw + off[6]);
    sm.table = (int16_t *)(smem_raw + off[7]);
    sm.segs = (Seg *)(smem_raw + off[8]);
    sm.misc = (int *)(smem_raw + off[9]);
    const int tid = threadIdx.x;
    for (int i = tid; i <= prm.n_s; i += blockDim.x) sm.T[i] = prm.T[i];
    for (int i = tid; i <= prm.n_s + 1; i += blockDim.x) sm.lohi[i] = make_float2(prm.lo[i], prm.hi[i]);
    for (int i = tid; i <= prm.n_c; i += blockDim.x) sm.orig[i] = m.orig[i];
    if (!LIN)
        for (int i = tid; i < prm.tab_n; i += blockDim.x) sm.table[i] = table_g[i];
    for (int i = tid; i < prm.nbin; i += blockDim.x) sm.hist[i] = 0;

    BinConst bcst;
    bcst.tab_bias = prm.tab_bias;
    bcst.inv_nmu2 = prm.inv_nmu2;
    bcst.s_scale = prm.s_scale;
    bcst.s_c0 = prm.s_c0;
    bcst.s_c1 = prm.s_c1;
    bcst.mu_c1 = prm.mu_c1;
    bcst.mu_c2 = prm.mu_c2;
    bcst.mu_c3 = prm.mu_c3;
    bcst.hit_max = prm.hit_max;
    bcst.dot_margin = prm.dot_margin;
    bcst.tab_key0 = prm.tab_key0;
    bcst.tab_last = (uint32_t)(prm.tab_n - 1);
    bcst.tab_shift = prm.tab_shift;
    bcst.n_s = prm.n_s;
    bcst.n_mu = prm.n_mu;
    Ctx<MU, MID, LIN> cx{prm, sm, m, bcst, tid & 31, tid >> 5, 0u, 0u, 0u, 0u, 0u, 0, 0, 0.f, 0.f, 0.f, 0u, 0u};
    const uint32_t qw = saddr(sm.queue) + (uint32_t)cx.warp * (QN * 32 * 2 * 2);
    cx.q = qw + 2u * (uint32_t)cx.lane;
    cx.cq = qw + QN * 32 * 2;
    cx.bc = saddr(sm.bcopy) + (uint32_t)cx.warp * (P * 32 * 16);
    cx.abase = saddr(sm.a);
    cx.hbase = saddr(sm.hist);
    unsigned long long n_cand = 0;

    // per-launch mode: this block walks the chunks of one cell of one term
    const uint32_t n_units = persistent ? *n_units_p : 0u;
    uint32_t pl_a = 0, pl_end = 0;
    if (!persistent) {
        const size_t gk = (size_t)terms[term_pl].cat_a * prm.n_cells + blockIdx.x;
        pl_a = m.cellstart[gk];
        pl_end = m.cellstart[gk + 1];
    }
    __syncthreads();

    for (;;) {
        Unit un;
        if (persistent) {
            if (tid == 0) sm.misc[0] = (int)atomicAdd(claim, 1u);
            __syncthreads();
            const uint32_t u = (uint32_t)sm.misc[0];
            if (u >= n_units) break;
            un = units[u];
        } else {
            if (pl_a >= pl_end) break;
            un.term = term_pl;
            un.cell = blockIdx.x;
            un.a0 = pl_a;
            un.a1 = min(pl_end, pl_a + (uint32_t)chunk);
            pl_a = un.a1;
        }
        const Term tm = terms[un.term];
        cx.a0 = un.a0;
        cx.na = un.a1 - un.a0;
        for (uint32_t i = tid; i < cx.na; i += blockDim.x) sm.a[i] = __ldg(m.pf + un.a0 + i);
        if (cx.warp == 0) build_segments(prm, sm, m, tm, un.cell, cx.lane);
        if (tid == 0) sm.misc[3] = 0;
        const int n_c = prm.n_c;
        const int ax = un.cell % n_c, ay = (un.cell / n_c) % n_c, az = un.cell / (n_c * n_c);
        const uint32_t oax = sm.orig[ax];
        if (MID) {
            cx.gx = 2.0f * (float)((long long)oax - prm.obs[0]);
            cx.gy = 2.0f * (float)((long long)sm.orig[ay] - prm.obs[1]);
            cx.gz = 2.0f * (float)((long long)sm.orig[az] - prm.obs[2]);
        }
        __syncthreads();
        const int ns = sm.misc[1];
        const uint32_t total = (uint32_t)sm.misc[2];
        const uint32_t self0 = (uint32_t)sm.misc[4], self1 = (uint32_t)sm.misc[5];
        const uint32_t n_self = (self1 - self0 + TILE - 1) / TILE;
        const uint32_t nt = n_self + (total + TILE - 1) / TILE;
        // tiles are claimed one at a time from a shared counter (its first
        // WARPS values are implicit), so warps finish a unit together
        for (uint32_t ti = cx.warp; ti < nt;) {
            if (ti < n_self) {
                const uint32_t base = self0 + ti * TILE;
                n_cand += (unsigned long long)min(self1 - base, (uint32_t)TILE) * cx.na;
                cx.template tile<true>(base, self1, 0u, ns, total, oax);
            } else {
                const uint32_t ob = (ti - n_self) * TILE;
                n_cand += (unsigned long long)min(total - ob, (uint32_t)TILE) * cx.na;
                cx.template tile<false>(0u, 0u, ob, ns, total, oax);
            }
            uint32_t nx = 0;
            if (cx.lane == 0) nx = (uint32_t)atomicAdd(&sm.misc[3], 1) + WARPS;
            ti = __shfl_sync(0xffffffffu, nx, 0);
        }
        __syncthreads();
        // drain the block histogram into the term's int64 histogram
        for (int b = tid; b < prm.nbin; b += blockDim.x) {
            const int v = sm.hist[b];
            cx.n_binned += (unsigned)v;   // every binned pair passes through the block histogram
            if (v) {
                atomicAdd((unsigned long long *)&tm.hist[b], (unsigned long long)(long long)v);
                sm.hist[b] = 0;
            }
        }
        __syncthreads();
    }
    // work statistics (per-lane candidate counts are warp-uniform: count lane 0 only)
    unsigned long long ex = cx.n_exact, bn = cx.n_binned, cd = (cx.lane == 0) ? n_cand : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ex += __shfl_down_sync(0xffffffffu, ex, o);
        bn += __shfl_down_sync(0xffffffffu, bn, o);
        cd += __shfl_down_sync(0xffffffffu, cd, o);
    }
    if (cx.lane == 0) {
        atomicAdd(&stats[0], cd);
        atomicAdd(&stats[1], bn);
        atomicAdd(&stats[2], ex);
    }
}

template <bool MU, bool MID, bool LIN>
void *kernel_ptr()
{
    return (void *)paircount_kernel<MU, MID, LIN>;
}

void *select_kernel(const CountParams &p)
{
    const bool mu = p.n_mu > 1;
    const bool mid = mu && p.los == TPCF_LOS_MIDPOINT;
    const bool lin = p.linear != 0;
    if (!mu) return lin ? kernel_ptr<false, false, true>() : kernel_ptr<false, false, false>();
    if (!mid) return lin ? kernel_ptr<true, false, true>() : kernel_ptr<true, false, false>();
    return lin ? kernel_ptr<true, true, true>() : kernel_ptr<true, true, false>();
}

}  // namespace

int paircount_smem_bytes(const CountParams &p, int warps_per_block)
{
    (void)warps_per_block;
    size_t off[10];
    return (int)smem_layout(p, off);
}

cudaError_t paircount_set_attrs(const CountParams &p, int smem_bytes)
{
    return cudaFuncSetAttribute(select_kernel(p), cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
}

int paircount_max_blocks_per_sm(const CountParams &p, int warps_per_block, int smem_bytes)
{
    (void)warps_per_block;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, select_kernel(p), WARPS * 32, smem_bytes) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_paircount(const CountParams &p, const Mesh &m, const Term *terms, const Cat *cats,
                             const Unit *units, const uint32_t *n_units, unsigned *claim, const int16_t *table,
                             unsigned long long *stats, int *status, const PairLaunch &pl, cudaStream_t s)
{
    (void)cats;
    (void)status;
    void *args[] = {(void *)&p,     (void *)&m,     (void *)&terms,         (void *)&units,   (void *)&n_units,
                    (void *)&claim, (void *)&table, (void *)&stats,         (void *)&pl.persistent,
                    (void *)&pl.term, (void *)&pl.chunk};
    return cudaLaunchKernel(select_kernel(p), dim3(pl.blocks), dim3(WARPS * 32), args, (size_t)pl.smem_bytes, s);
}

}  // namespace tpcf
