// Binned pair counting on the chaining mesh (Sect. 2.1: DD, DR_i, RR_i
// counts; Sect. 4.3: bins in separation s and in mu).
//
// Work decomposition.  A unit is a chunk of at most 128 sorted points of one
// mesh cell A of catalogue a, to be paired with every point of catalogue b in
// the neighbourhood of A.  A thread block owns a unit: the a-chunk and the
// histogram live in shared memory, and the warps share the b side.  The
// neighbourhood is walked as rows of cells (dz, dy) whose x-runs are
// contiguous in the cell-sorted point order.  The warps first filter the
// runs: a b-point is kept only if its distance to the a-chunk's bounding box
// is below the last edge's band, and the survivors (shifted into A's frame)
// go to the block's scratch window in global memory.  The window is cut into
// tiles of 32*P points dealt to the warps; a warp loads its tile once, one
// P-vector per lane, then streams the a-chunk past it by broadcast
// shared-memory loads.
//
// Line of sight along x (every periodic box).  Per pair the lane forms the
// FP32 differences and d2 = dx^2 + dy^2 + dz^2 and appends (d2, dx) to its
// own queue column in shared memory, branch-free: the store always happens
// and only a pair with d2 below the last edge's band advances the column
// head.  A flush bins the columns in place, four entries per lane per pass:
// the s and mu bins are floors of FP32 estimates, each bracketed by a
// rigorous error interval, so no point is read back from shared memory.
// Slots without a pending entry hold a sentinel pair that classifies as
// certain and lands in a spare word, so the passes need no count tests.  A
// pair whose interval contains a bin edge (about 3 in 10^4) is identified by
// replaying its lane's pushes since the flush window began, set aside, and
// rechecked exactly from the integer grid coordinates (64-bit squared
// distances, 128-bit mu test), 32 at a time, so every count equals the
// integer definition bit for bit.
//
// Midpoint line of sight (cut-sky).  The mu of a pair needs both points, so
// the queue holds 16-bit (a index, b slot) entries, pushed after a
// dot-product range test (a.b' - |a|^2/2 >= (|b'|^2 - H)/2 - margin: three
// FMAs and a compare), compacted per warp and binned from the a-chunk and
// the tile's b copies; its rechecks go through the same 32-at-a-time list.
#include "pair_device.cuh"

namespace tpcf {

namespace {

constexpr int P = 4;            // b-points per lane
constexpr int TILE = 32 * P;    // b-points per warp tile
constexpr int QN = 24;          // queue slots per lane, midpoint path (16-bit entries)
constexpr int QX = 23;          // queue slots per lane, x line of sight (8-byte entries)
constexpr int XCAP = 96;        // per-warp list of pairs awaiting the exact recheck (global scratch)
constexpr int WARPS = 8;        // warps per block
constexpr int CAP = 12288;      // raw neighbour points filtered per window
constexpr int NB = 16;          // distance buckets of the window order
constexpr int SCR_W = CAP + 8 * 32;                 // float4 scratch per block: survivors per warp (+ rounding)
constexpr int SCR = SCR_W + CAP + WARPS * XCAP * 8 / 16;   // + the bucket-ordered window + the recheck lists
// misc[]: [0] unit, [1] runs, [2] run points, [3] tile counter, [4..5] self range, [M_CNT..] window counts,
// [M_BKT..] survivors per distance bucket, [M_POS..] next free position of each bucket
constexpr int M_CNT = 8;        // [WARPS] survivors per warp in the current window
constexpr int M_BKT = 16;       // [NB]
constexpr int M_POS = M_BKT + NB;   // [NB]
constexpr int M_N = M_POS + NB;
constexpr int MAX_SEGS = 2 * MAX_ROWS + 2;
static_assert(P == 4, "tile_x unrolls four b-points per lane");
static_assert((QX + 1) % 4 == 0, "x-path flush passes read four rows and stay in the lane's column");
static_assert((SCR * 16) % 128 == 0 && (SCR_W * 16) % 128 == 0 && (CAP * 16) % 128 == 0,
              "per-block scratch regions start on 128-byte lines (discard_l2)");
static_assert(UNIT_CHUNK % 32 == 0 && UNIT_CHUNK <= 128 && UNIT_CHUNK <= WARPS * 32, "a-chunk load and box");

// A run of b-points: cells x0..x1 of one neighbour row, contiguous in the
// cell-sorted order.  Runs are concatenated, and the concatenation is cut
// into full tiles, so a tile may span several rows.
struct Seg {
    uint32_t s0;           // first b index
    uint32_t off0;         // offset of s0 in the concatenation of the unit's runs
    float sy, sz;          // row shift into A's frame
};

// Shared memory.  Fixed-size arrays sit at compile-time offsets (first the
// ones both paths use, then the path's own), so their addresses fold into
// the instructions; the arrays sized by the binning follow.
__host__ __device__ constexpr uint32_t al16(uint32_t x) { return (x + 15u) & ~15u; }
constexpr uint32_t O_MISC = 0;                                          // int [M_N]
constexpr uint32_t O_STAT = al16(O_MISC + 4 * M_N);                     // u64 [3][WARPS]: candidates, binned, exact
constexpr uint32_t O_A = al16(O_STAT + 8 * 3 * WARPS);                  // float4 [UNIT_CHUNK + 8]: a-chunk
                                                                        // (.w = -|a|^2/2), per-warp box partials
constexpr uint32_t O_SEG = al16(O_A + 16 * (UNIT_CHUNK + 8));           // Seg [MAX_SEGS + 1]
constexpr uint32_t O_B = al16(O_SEG + 16 * (MAX_SEGS + 1));             // midpoint: float4 [WARPS][P][32] b copies
                                                                        // (.w = b index)
// (midpoint: slot s = p * 32 + lane is stored at s + s / 32, so that one
// lane's P slots fall in different bank groups)
__host__ __device__ constexpr uint32_t o_q(bool mid) { return al16(O_B + (mid ? 16u * WARPS * P * 33 : 0u)); }
// queues: x: (d2, dx) [WARPS][QX + 1][32]; midpoint: u16 [WARPS][QN][32] + compacted [WARPS][QN * 32]
__host__ __device__ constexpr uint32_t o_x(bool mid)
{
    return al16(o_q(mid) + (mid ? 2u * WARPS * QN * 32 * 2 : 8u * WARPS * (QX + 1) * 32));
}
__host__ __device__ constexpr uint32_t o_var(bool mid) { return o_x(mid); }

// offsets of the arrays sized by the binning: T u64 [n_s + 1], hist int
// [nbin + max(32, n_mu)] (spare words: per-lane dummies of the x path's adds,
// and the bins past the last edge of the linear path), lohi float2 [n_s + 2], orig u32
// [n_c + 1], table i16 [tab_n], sxf float [n_c] (x shift of each cell column into
// the current unit's frame)
struct VarOff {
    uint32_t T, hist, lohi, orig, table, sxf, end;
};
__host__ __device__ inline VarOff var_offsets(const CountParams &p, bool mid)
{
    VarOff v;
    v.T = o_var(mid);
    v.hist = al16(v.T + 8u * (uint32_t)(p.n_s + 1));
    v.lohi = al16(v.hist + 4u * (uint32_t)(p.nbin + (p.n_mu > 32 ? p.n_mu : 32)));
    v.orig = al16(v.lohi + 8u * (uint32_t)(p.n_s + 2));
    v.table = al16(v.orig + 4u * (uint32_t)(p.n_c + 1));
    v.sxf = al16(v.table + (p.linear ? 0u : 2u * (uint32_t)p.tab_n));
    v.end = al16(v.sxf + 4u * (uint32_t)p.n_c);
    return v;
}

__host__ __device__ inline bool uses_midpoint(const CountParams &p) { return p.n_mu > 1 && p.los == TPCF_LOS_MIDPOINT; }

extern __shared__ __align__(16) unsigned char smem_raw[];

__device__ __forceinline__ int *sh_misc() { return (int *)(smem_raw + O_MISC); }
__device__ __forceinline__ unsigned long long *sh_stat() { return (unsigned long long *)(smem_raw + O_STAT); }
__device__ __forceinline__ float4 *sh_a() { return (float4 *)(smem_raw + O_A); }
__device__ __forceinline__ Seg *sh_segs() { return (Seg *)(smem_raw + O_SEG); }
template <bool MID>
__device__ __forceinline__ uint32_t *sh_orig(const CountParams &p)
{
    return (uint32_t *)(smem_raw + var_offsets(p, MID).orig);
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

// x path push: store (d2, e) at the column head; advance the head (one slot
// row of 32 lanes x 8 bytes) only when d2 < h.  NaN never passes.
__device__ __forceinline__ void push_if_lt(uint32_t &head, float d2, uint32_t e, float h)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.lt.f32 p, %1, %2;\n\t"
        "st.shared.v2.b32 [%0], {%3, %4};\n\t"
        "@p add.u32 %0, %0, 256;\n\t}"
        : "+r"(head)
        : "f"(d2), "f"(h), "r"(__float_as_uint(d2)), "r"(e)
        : "memory");
}
__device__ __forceinline__ void sts64(uint32_t a, float x, float y)
{
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(x), "f"(y) : "memory");
}
__device__ __forceinline__ float2 lds64(uint32_t a)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
// Drop the 128-byte lines [p, p + bytes) from L2 without writing them back
// (their data is dead; a later store writes the line afresh).  Thread t of
// nt takes every nt-th line.  p is 128-byte aligned and the lines belong to
// the calling block alone.
__device__ __forceinline__ void discard_l2(const void *p, uint32_t bytes, uint32_t t, uint32_t nt)
{
    for (uint32_t o = t * 128u; o < bytes; o += nt * 128u)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"((const char *)p + o) : "memory");
}

// Bounding box of an a-chunk (cell-relative coordinates).
struct Box {
    float lx, ly, lz, hx, hy, hz;
};

// Classification of a queued pair: its histogram slot as a shared address
// (meaningful when good), good = binned and outside every error band, amb =
// inside an error band (recheck exactly).  Neither: beyond the last edge.
struct Cls {
    uint32_t addr;
    bool good, amb;
};

template <bool MU, bool MID, bool LIN>
struct Ctx {
    const CountParams &prm;
    const Mesh &m;
    int lane, warp;
    uint32_t q;                // this lane's queue column (shared address of slot 0)
    uint32_t cq;               // this warp's compacted queue (shared address)
    uint32_t bc;               // this warp's b copies (midpoint path; .w: b index)
    uint32_t n_list;           // entries in it (warp-uniform)
    uint32_t hdum;             // this lane's spare word after the histogram
    float4 *scr;               // this block's scratch: the current window's surviving b-points
    uint32_t R;                // per-warp region length of the current window (entries)
    uint32_t abase;            // the a-chunk (shared address)
    uint32_t hbase;            // the block histogram (shared address)
    uint32_t hadj;             // hbase minus the bias of the encoded bin keys (see classify)
    uint32_t a0, na;           // current unit's a-chunk
    float gx, gy, gz;          // 2 (corner(A) - observer), midpoint line of sight
    unsigned n_exact, n_binned;

    // Every bin decision is a floor of an FP32 estimate x of an exact value
    // x* whose error bound gives an interval [x_lo, x_hi] around it, computed
    // with directed roundings so that it certainly holds x*.  With
    // B = 1.5 * 2^23, fadd_rd(x, B) = floor(x) + B exactly for |x| < 2^22, so
    // the floors of both ends are compared as floats: equal means the bin is
    // certain, different means an edge (or NaN, from d2 = 0) lies inside the
    // interval and the pair is rechecked exactly.  The bit pattern of
    // floor(x_lo) + B is the bin plus the pattern of B; the histogram address
    // absorbs that bias (hadj).  Straight-line code: every lane runs the same
    // instructions.
    __device__ __forceinline__ Cls classify(float d2, float dx, float dy, float dz, const float4 &a, const float4 &b) const
    {
        const float big = 12582912.0f;   // 1.5 * 2^23
        Cls o;
        bool amb, valid;
        uint32_t ks;                      // s bin, biased (LIN: + bits of B)
        float r = 0.0f;
        if (LIN) {
            // u* = sqrt(D2) / (q ds); v = n_mu sqrt(d2) and u = v * s_scale
            r = rsqrt_approx(__fmul_rn(d2, prm.inv_nmu2));   // n_mu / sqrt(d2)
            const float v = __fmul_rn(d2, r);
            const float flo = __fadd_rd(__fmaf_rd(v, prm.s_lo_mul, -prm.s_c0), big);
            const float fhi = __fadd_rd(__fmaf_ru(v, prm.s_hi_mul, prm.s_c0), big);
            amb = !(flo == fhi);
            valid = flo < prm.s_top;
            ks = __float_as_uint(flo);
        } else {
            const uint32_t key = min((__float_as_uint(__fadd_rn(d2, prm.tab_bias)) >> prm.tab_shift) - prm.tab_key0,
                                     (uint32_t)(prm.tab_n - 1));
            int k = ((const int16_t *)(smem_raw + var_offsets(prm, MID).table))[key];
            amb = (k == CODE_AMBIG);
            k = amb ? -1 : k;
            const float2 lh = ((const float2 *)(smem_raw + var_offsets(prm, MID).lohi))[k + 1];
            const bool ge_hi = d2 >= lh.y;
            amb |= (d2 >= lh.x) && !ge_hi;
            k += ge_hi ? 1 : 0;
            // at or beyond the last edge's band a pair is certainly not binned
            // (the x-path queue sentinel lies there)
            const bool beyond = d2 >= prm.hit_max;
            amb = amb && !beyond;
            valid = !beyond && (unsigned)k < (unsigned)prm.n_s;
            ks = (uint32_t)k;
        }
        if (MU) {
            // t* = n_mu |mu|; the top edge t* = n_mu (mu = 1) is an edge like the
            // others, so a pair there is rechecked and never needs a clamp
            float tlo, thi;
            if (!MID) {
                if (!LIN) r = rsqrt_approx(__fmul_rn(d2, prm.inv_nmu2));   // n_mu / sqrt(d2)
                const float bt = __fmaf_ru(prm.mu_c1, r, prm.mu_c2);
                tlo = __fmaf_rd(fabsf(dx), r, -bt);
                thi = __fmaf_ru(fabsf(dx), r, bt);
            } else {
                // t = n_mu |dot| / (|d| |l|) = |dot| r rl with r = n_mu / |d| (the
                // s path's rsqrt); the band's 1/|d| term is mu_c1 rs = mu_c1r r
                if (!LIN) r = rsqrt_approx(__fmul_rn(d2, prm.inv_nmu2));
                const float lx = __fadd_rn(__fadd_rn(gx, a.x), b.x);
                const float ly = __fadd_rn(__fadd_rn(gy, a.y), b.y);
                const float lz = __fadd_rn(__fadd_rn(gz, a.z), b.z);
                const float dot = __fmaf_rn(dz, lz, __fmaf_rn(dy, ly, __fmul_rn(dx, lx)));
                const float l2 = __fmaf_rn(lz, lz, __fmaf_rn(ly, ly, __fmul_rn(lx, lx)));
                const float rl = rsqrt_approx(l2);
                const float t = __fmul_rn(__fmul_rn(fabsf(dot), r), rl);
                const float bt = __fmaf_ru(prm.mu_c1r, r, __fmaf_ru(prm.mu_c3, rl, prm.mu_c2));
                tlo = __fsub_rd(t, bt);
                thi = __fadd_ru(t, bt);
            }
            const float jlo = __fadd_rd(tlo, big), jhi = __fadd_rd(thi, big);
            amb |= !(jlo == jhi);
            o.addr = hadj + 4u * (ks * (uint32_t)prm.n_mu + __float_as_uint(jlo));
        } else {
            o.addr = hadj + 4u * ks;
        }
        o.amb = amb;
        // linear bins: an unambiguous pair past the last edge has s bin n_s
        // exactly (d2 is below the last edge's band), so its address falls
        // in the spare words after the histogram and needs no test
        o.good = LIN ? !amb : (valid && !amb);
        return o;
    }

    // Padded position of b copy slot s (see o_q).
    __device__ __forceinline__ uint32_t bslot(uint32_t s) const { return s + (s >> 5); }

    // Classification of queue entry v (a index | b copy index << 8).
    __device__ __forceinline__ Cls bin_of(uint32_t v) const
    {
        const float4 a = lds128(abase + 16u * (v & 255u));
        const float4 b = lds128(bc + 16u * bslot(v >> 8));
        const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y), dz = __fsub_rn(a.z, b.z);
        const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
        return classify(d2, dx, dy, dz, a, b);
    }

    // Midpoint path: bin every queued pair.  The lanes' queues are first packed into one
    // warp-contiguous list (a index | b copy index << 8), so that the binning
    // loop runs with all lanes busy whatever the spread of per-lane counts.
    // Pairs that need the exact recheck go to the warp's recheck list, which
    // is rechecked 32 at a time.  n = this lane's count.
    __device__ __forceinline__ void flush_mid(uint32_t n)
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
        const uint32_t lt = (1u << lane) - 1u;
        // two entries per lane per pass (independent work for the scheduler)
        for (uint32_t w0 = 0; w0 < total; w0 += 64) {
            const uint32_t e0 = w0 + lane, e1 = e0 + 32u;
            const bool live0 = e0 < total, live1 = e1 < total;
            const uint32_t v0 = lds16_if(cq + 2u * e0, live0);
            const uint32_t v1 = lds16_if(cq + 2u * e1, live1);
            const Cls c0 = bin_of(v0), c1 = bin_of(v1);   // dead slots read entry 0: in bounds, discarded
            red_x(c0.addr, live0 && c0.good);
            red_x(c1.addr, live1 && c1.good);
            const bool x0 = live0 && c0.amb, x1 = live1 && c1.amb;
            const unsigned am0 = __ballot_sync(0xffffffffu, x0);
            const unsigned am1 = __ballot_sync(0xffffffffu, x1);
            if (am0 | am1) {
                // rare: the pair (a index, b index) goes to the recheck list
                // (at most 31 + 64 entries after this, within XCAP)
                if (x0) xlist()[n_list + __popc(am0 & lt)] = make_uint2(a0 + (v0 & 255u), b_index(v0 >> 8));
                n_list += __popc(am0);
                if (x1) xlist()[n_list + __popc(am1 & lt)] = make_uint2(a0 + (v1 & 255u), b_index(v1 >> 8));
                n_list += __popc(am1);
                if (n_list >= 32) recheck_list();
            }
        }
    }

    // b index of b copy slot s (its .w).
    __device__ __forceinline__ uint32_t b_index(uint32_t s) const
    {
        uint32_t i;
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(i) : "r"(bc + 16u * bslot(s) + 12u) : "memory");
        return i;
    }

    // ---- neighbour filtering ----

    // The a-chunk's bounding box from the per-warp partials stored after it
    // (cell-relative coordinates are >= 0, so float bit patterns order as
    // unsigned integers).
    __device__ __forceinline__ Box chunk_box() const
    {
        unsigned b[6] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u, 0u};
#pragma unroll
        for (int w = 0; w < UNIT_CHUNK / 32; w++) {
            const float4 p0 = sh_a()[UNIT_CHUNK + w], p1 = sh_a()[UNIT_CHUNK + 4 + w];
            b[0] = min(b[0], __float_as_uint(p0.x));
            b[1] = min(b[1], __float_as_uint(p0.y));
            b[2] = min(b[2], __float_as_uint(p0.z));
            b[3] = max(b[3], __float_as_uint(p0.w));
            b[4] = max(b[4], __float_as_uint(p1.x));
            b[5] = max(b[5], __float_as_uint(p1.y));
        }
        return {__uint_as_float(b[0]), __uint_as_float(b[1]), __uint_as_float(b[2]),
                __uint_as_float(b[3]), __uint_as_float(b[4]), __uint_as_float(b[5])};
    }

    // The window's box in the form the filter and the bucket order use:
    // centre, half-widths (rounded outward, so [c - h, c + h] holds every
    // a-point) and the bucket scale NB / dmax^2, dmax bounding the distance
    // of any survivor from the centre.
    struct WinBox {
        float cx, cy, cz, hx, hy, hz, kscale;
    };
    __device__ __forceinline__ WinBox win_box() const
    {
        const Box bb = chunk_box();
        WinBox w;
        w.cx = 0.5f * (bb.lx + bb.hx);
        w.cy = 0.5f * (bb.ly + bb.hy);
        w.cz = 0.5f * (bb.lz + bb.hz);
        w.hx = __fadd_ru(__fmul_ru(0.5f, __fsub_ru(bb.hx, bb.lx)), __fmul_ru(1.0f / 8388608.0f, w.cx));
        w.hy = __fadd_ru(__fmul_ru(0.5f, __fsub_ru(bb.hy, bb.ly)), __fmul_ru(1.0f / 8388608.0f, w.cy));
        w.hz = __fadd_ru(__fmul_ru(0.5f, __fsub_ru(bb.hz, bb.lz)), __fmul_ru(1.0f / 8388608.0f, w.cz));
        const float dm = sqrtf(prm.hit_max) + sqrtf(w.hx * w.hx + w.hy * w.hy + w.hz * w.hz);
        w.kscale = (float)NB / (dm * dm);
        return w;
    }
    // Distance bucket of a survivor (squared distance from the box centre in
    // NB equal steps): points of one bucket have similar hit rates, so tiles
    // cut from the bucket order load the lanes evenly.  Only the order
    // depends on it, never a count.
    __device__ __forceinline__ uint32_t bucket_of(float ex, float ey, float ez, const WinBox &w) const
    {
        const float ux = __fsub_rn(ex, w.cx), uy = __fsub_rn(ey, w.cy), uz = __fsub_rn(ez, w.cz);
        const float d2c = __fmaf_rn(uz, uz, __fmaf_rn(uy, uy, __fmul_rn(ux, ux)));
        return min(__float2uint_rz(__fmul_rn(d2c, w.kscale)), (uint32_t)(NB - 1));
    }

    // Filter raw neighbour points [w0, w0 + win) of the unit's concatenated
    // runs: a point enters the window's list only if its distance to the
    // a-chunk's bounding box is below the last edge's band (with a relative
    // margin of 2^-16 over the FP32 box distance), so no pair the push test
    // could pass is lost.  Warp w filters the w-th slice of the window and
    // appends survivors (b' in A's frame, .w = b index) to its own region of
    // the block's scratch, in order, counting them per warp and per distance
    // bucket in misc.
    __device__ __forceinline__ void filter_window(uint32_t w0, uint32_t win, int n_seg)
    {
        const WinBox wb = win_box();
        R = (((win + WARPS - 1) / WARPS) + 31u) & ~31u;
        const uint32_t r0 = w0 + (uint32_t)warp * R, r1 = min(r0 + R, w0 + win);
        const float hf = prm.hit_max * (1.0f + 1.0f / 65536.0f);
        const float *sxf = (const float *)(smem_raw + var_offsets(prm, MID).sxf);
        float4 *dst = scr + (size_t)warp * R;
        uint32_t cnt = 0;
        if (r0 < r1) {
            const uint32_t o_first = r0 + lane;
            int lo = 0, hi = n_seg - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (sh_segs()[mid].off0 <= o_first) lo = mid; else hi = mid - 1;
            }
            int g = lo;
            const uint32_t lt = (1u << lane) - 1u;
            for (uint32_t c = r0; c < r1; c += 32) {
                const uint32_t o = c + (uint32_t)lane;
                while (g + 1 < n_seg && sh_segs()[g + 1].off0 <= o) g++;
                bool keep = false;
                float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
                if (o < r1) {
                    const Seg sg = sh_segs()[g];
                    const uint32_t i = sg.s0 + (o - sg.off0);
                    const float4 v = __ldg(m.pf + i);
                    e.x = __fadd_rn(v.x, sxf[m.pcx[i]]);
                    e.y = __fadd_rn(v.y, sg.sy);
                    e.z = __fadd_rn(v.z, sg.sz);
                    e.w = __uint_as_float(i);
                    // box as centre and half-widths: per axis q = max(|x - c| - h, 0)
                    const float qx = fmaxf(__fsub_rn(fabsf(__fsub_rn(e.x, wb.cx)), wb.hx), 0.0f);
                    const float qy = fmaxf(__fsub_rn(fabsf(__fsub_rn(e.y, wb.cy)), wb.hy), 0.0f);
                    const float qz = fmaxf(__fsub_rn(fabsf(__fsub_rn(e.z, wb.cz)), wb.hz), 0.0f);
                    keep = __fmaf_rn(qz, qz, __fmaf_rn(qy, qy, __fmul_rn(qx, qx))) < hf;
                }
                const unsigned mk = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    dst[cnt + __popc(mk & lt)] = e;
                    atomicAdd(&sh_misc()[M_BKT + bucket_of(e.x, e.y, e.z, wb)], 1);
                }
                cnt += __popc(mk);
            }
        }
        if (lane == 0) sh_misc()[M_CNT + warp] = (int)cnt;
    }

    // After the filter's barrier: the start of every bucket in the window's
    // order (warp 0), and the bucket counters cleared for the next window.
    __device__ __forceinline__ void bucket_starts() const
    {
        const int c = lane < NB ? sh_misc()[M_BKT + lane] : 0;
        int x = c;
#pragma unroll
        for (int o = 1; o < NB; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane < NB) {
            sh_misc()[M_POS + lane] = x - c;
            sh_misc()[M_BKT + lane] = 0;
        }
    }

    // The bucket-ordered window list (written by scatter_window).
    __device__ __forceinline__ float4 *lst() const { return scr + SCR_W; }

    // After bucket_starts' barrier: this warp's survivors move to their
    // buckets' places in the window list (the order within a bucket is
    // arbitrary).
    __device__ __forceinline__ void scatter_window() const
    {
        const WinBox wb = win_box();
        const uint32_t cnt = (uint32_t)sh_misc()[M_CNT + warp];
        const float4 *src = scr + (size_t)warp * R;
        for (uint32_t e = lane; e < cnt; e += 32) {
            const float4 v = src[e];   // written by this warp: plain (coherent) load
            const uint32_t pos = (uint32_t)atomicAdd(&sh_misc()[M_POS + bucket_of(v.x, v.y, v.z, wb)], 1);
            lst()[pos] = v;
        }
        // this warp's region is spent (each lane has used what it read)
        __syncwarp();
        discard_l2(src, (cnt * 16u + 127u) & ~127u, (uint32_t)lane, 32u);
    }

    // ---- x line of sight ----

    // This warp's list of pairs set aside for the exact recheck (global
    // scratch after the block's window; written and read by this warp only).
    __device__ __forceinline__ uint2 *xlist() const { return (uint2 *)(scr + SCR_W + CAP) + (size_t)warp * XCAP; }

    // Exact recheck of the set-aside pairs, one per lane.
    __device__ __forceinline__ void recheck_list()
    {
        __syncwarp();
        for (uint32_t e = lane; e < n_list; e += 32) {
            uint2 pr;
            pr = xlist()[e];
            const int bin = exact_bin(prm, (const unsigned long long *)(smem_raw + var_offsets(prm, MID).T), m.us, m.n_total, pr.x, pr.y);
            n_exact++;
            if (bin >= 0) red_inc(hbase + 4u * (uint32_t)bin);
        }
        __syncwarp();
        n_list = 0;
    }

    // d2 and dx of (a-chunk point a, this lane's b-point p), FP32 in A's frame.
    template <int p>
    __device__ __forceinline__ float d2_x(const float4 &a, const float (&bx)[P], const float (&by)[P],
                                          const float (&bz)[P], float &dx) const
    {
        dx = __fsub_rn(a.x, bx[p]);
        const float dy = __fsub_rn(a.y, by[p]), dz = __fsub_rn(a.z, bz[p]);
        return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    }

    // Push threshold of (a-chunk point ai, b slot p): the last edge's band,
    // or 0 (never passes) for a self-cell pair that is not a < b.
    template <bool SELF>
    __device__ __forceinline__ float thr_x(uint32_t ai, uint32_t ib) const
    {
        return (!SELF || a0 + ai < ib) ? prm.hit_max : 0.0f;
    }

    // The pair behind this lane's queue entry k (the k-th push that advanced
    // its head since the flush window began at a-chunk index a_lo): the
    // window's pushes are replayed in push order (a ascending, then p) with
    // the same FP32 arithmetic.  Rare (ambiguous pairs only) and divergent.
    template <bool SELF>
    __device__ __forceinline__ void find_pair(uint32_t k, uint32_t a_lo, uint32_t ib0, const float (&bx)[P],
                                              const float (&by)[P], const float (&bz)[P], uint32_t &ai_out,
                                              uint32_t &p_out) const
    {
        uint32_t j = 0;
        ai_out = a_lo;
        p_out = 0;
        for (uint32_t ai = a_lo; ai < na; ai++) {
            const float4 a = lds128(abase + 16u * ai);
            float dx;
            const float d0 = d2_x<0>(a, bx, by, bz, dx), d1 = d2_x<1>(a, bx, by, bz, dx);
            const float d2v = d2_x<2>(a, bx, by, bz, dx), d3 = d2_x<3>(a, bx, by, bz, dx);
            const bool h0 = d0 < thr_x<SELF>(ai, ib0), h1 = d1 < thr_x<SELF>(ai, ib0 + 32u);
            const bool h2 = d2v < thr_x<SELF>(ai, ib0 + 64u), h3 = d3 < thr_x<SELF>(ai, ib0 + 96u);
            const uint32_t c = (uint32_t)h0 + (uint32_t)h1 + (uint32_t)h2 + (uint32_t)h3;
            if (j + c > k) {
                uint32_t r = k - j, p = 0;
                if (h0) { if (r == 0) { p = 0; goto done; } r--; }
                if (h1) { if (r == 0) { p = 1; goto done; } r--; }
                if (h2) { if (r == 0) { p = 2; goto done; } r--; }
                p = 3;
            done:
                ai_out = ai;
                p_out = p;
                return;
            }
            j += c;
        }
    }

    // Append this lane's entry k (when x) to the recheck list at its ballot
    // rank.  The b index of slot p: the self cell's sorted index ib0 + 32 p,
    // or the point at filtered position ib0 + 32 p of the window.
    template <bool SELF>
    __device__ __forceinline__ void set_aside(bool x, uint32_t k, unsigned am, uint32_t lt, uint32_t a_lo, uint32_t ib0,
                                              const float (&bx)[P], const float (&by)[P], const float (&bz)[P])
    {
        if (x) {
            uint32_t ai, p, ib;
            find_pair<SELF>(k, a_lo, ib0, bx, by, bz, ai, p);
            if (SELF) {
                ib = ib0 + 32u * p;
            } else {
                ib = __float_as_uint(lst()[ib0 + 32u * p].w);   // written by this block: plain load
            }
            xlist()[n_list + __popc(am & lt)] = make_uint2(a0 + ai, ib);
        }
        n_list += __popc(am);
    }

    // Histogram increment when ok, as an unpredicated add: a lane with
    // nothing to count adds to its own spare word after the histogram.
    __device__ __forceinline__ void red_x(uint32_t addr, bool ok) const
    {
        const uint32_t at = ok ? addr : hdum;
        asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(at) : "memory");
    }

    // Bin this lane's column (n entries; the window's pushes began at a-chunk
    // index a_lo), four entries per lane per pass.  Every slot that holds no
    // pending entry holds the sentinel (prm.sent_d2, prm.sent_dx), which
    // classifies as a certain pair half a bin past the last edge (its add
    // lands in a spare word), so no pass needs a per-lane count test: the
    // head slot, which the last miss overwrote, is reset here, and every
    // slot is reset after it is read.  QX + 1 is a multiple of 4, so the
    // passes never leave the lane's own column.
    template <bool SELF>
    __device__ __forceinline__ void flush_x(uint32_t n, uint32_t a_lo, uint32_t ib0, const float (&bx)[P],
                                            const float (&by)[P], const float (&bz)[P])
    {
        const uint32_t nmax = __reduce_max_sync(0xffffffffu, n);
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        const float sd2 = prm.sent_d2, sdx = prm.sent_dx;
        sts64(q + n * 256u, sd2, sdx);
        uint32_t amask = 0;   // bit k: entry k lies in an error band (QX < 32 slots)
        for (uint32_t k = 0; k < nmax; k += 4) {
            const uint32_t bit = 1u << k;
#pragma unroll
            for (uint32_t h = 0; h < 4; h += 2) {
                const uint32_t a0s = q + (k + h) * 256u, a1s = a0s + 256u;
                const float2 e0 = lds64(a0s), e1 = lds64(a1s);
                sts64(a0s, sd2, sdx);
                sts64(a1s, sd2, sdx);
                const Cls c0 = classify(e0.x, e0.y, 0.f, 0.f, z, z), c1 = classify(e1.x, e1.y, 0.f, 0.f, z, z);
                red_x(c0.addr, c0.good);
                red_x(c1.addr, c1.good);
                if (c0.amb) amask |= bit << h;
                if (c1.amb) amask |= bit << (h + 1);
            }
        }
        if (__any_sync(0xffffffffu, amask != 0)) {
            // rare: set the ambiguous entries aside, one per lane per round
            // (at most 31 + 32 in the list after a round, within XCAP)
            const uint32_t lt = (1u << lane) - 1u;
            for (;;) {
                const bool x = amask != 0;
                const unsigned am = __ballot_sync(0xffffffffu, x);
                if (!am) break;
                const uint32_t k = x ? (uint32_t)(__ffs(amask) - 1) : 0u;
                set_aside<SELF>(x, k, am, lt, a_lo, ib0, bx, by, bz);
                amask &= amask - 1u;
                if (n_list >= 32) recheck_list();
            }
        }
    }

    // One pair: push (d2, dx) when d2 < h.
    template <int p>
    __device__ __forceinline__ void push_x(uint32_t &head, const float4 &a, const float (&bx)[P], const float (&by)[P],
                                           const float (&bz)[P], float h) const
    {
        float dx;
        const float d2 = d2_x<p>(a, bx, by, bz, dx);
        push_if_lt(head, d2, __float_as_uint(dx), h);
    }

    // Load one b-point (shifted into A's frame) into lane registers; a
    // missing point sits at 1e30, where d2 overflows to +inf and never passes.
    __device__ __forceinline__ void load_bx(int p, bool ok, uint32_t i, float sy, float sz, uint32_t orig_ax,
                                            float (&bx)[P], float (&by)[P], float (&bz)[P]) const
    {
        if (ok) {
            const float4 v = __ldg(m.pf + i);
            const int cx = m.pcx[i];
            const float sx = (float)(int)(sh_orig<MID>(prm)[cx] - orig_ax);
            bx[p] = __fadd_rn(v.x, sx);
            by[p] = __fadd_rn(v.y, sy);
            bz[p] = __fadd_rn(v.z, sz);
        } else {
            bx[p] = by[p] = bz[p] = 1e30f;
        }
    }

    // all pairs of the a-chunk with one tile of b-points: the self cell of an
    // auto count (SELF, indices base..s1) or a packed tile at offset o_base of
    // the concatenated runs (n_seg runs, total points).
    template <bool SELF>
    __device__ __forceinline__ void tile_x(uint32_t base, uint32_t s1, uint32_t o_base, int n_seg, uint32_t total,
                                           uint32_t orig_ax)
    {
        float bx[P], by[P], bz[P];
        if (SELF) {
#pragma unroll
            for (int p = 0; p < P; p++) {
                const uint32_t i = base + lane + 32u * p;
                load_bx(p, i < s1, i, 0.0f, 0.0f, orig_ax, bx, by, bz);
            }
        } else {
#pragma unroll
            for (int p = 0; p < P; p++) {
                const uint32_t f = o_base + (uint32_t)lane + 32u * p;
                if (f < total) {
                    const float4 e = lst()[f];   // written by this block: plain (coherent) load
                    bx[p] = e.x;
                    by[p] = e.y;
                    bz[p] = e.z;
                } else {
                    bx[p] = by[p] = bz[p] = 1e30f;
                }
            }
        }
        // A flush comes before 2P more pushes could run past QX slots.
        uint32_t head = q, a_lo = 0;
        const uint32_t lim = q + (uint32_t)(QX - 2 * P) * 256u;
        // SELF: the sorted index of slot 0 (the a < b test and the rechecks);
        // else the filtered position of slot 0 (the rechecks)
        const uint32_t ib0 = (SELF ? base : o_base) + lane;
        uint32_t ai = 0;
        for (; ai + 1 < na; ai += 2) {
            const float4 a = lds128(abase + 16u * ai), c = lds128(abase + 16u * (ai + 1));
            push_x<0>(head, a, bx, by, bz, thr_x<SELF>(ai, ib0));
            push_x<1>(head, a, bx, by, bz, thr_x<SELF>(ai, ib0 + 32u));
            push_x<2>(head, a, bx, by, bz, thr_x<SELF>(ai, ib0 + 64u));
            push_x<3>(head, a, bx, by, bz, thr_x<SELF>(ai, ib0 + 96u));
            push_x<0>(head, c, bx, by, bz, thr_x<SELF>(ai + 1, ib0));
            push_x<1>(head, c, bx, by, bz, thr_x<SELF>(ai + 1, ib0 + 32u));
            push_x<2>(head, c, bx, by, bz, thr_x<SELF>(ai + 1, ib0 + 64u));
            push_x<3>(head, c, bx, by, bz, thr_x<SELF>(ai + 1, ib0 + 96u));
            if (__any_sync(0xffffffffu, head > lim)) {
                flush_x<SELF>((head - q) >> 8, a_lo, ib0, bx, by, bz);
                head = q;
                a_lo = ai + 2;
            }
        }
        if (ai < na) {
            const float4 a = lds128(abase + 16u * ai);
            push_x<0>(head, a, bx, by, bz, thr_x<SELF>(ai, ib0));
            push_x<1>(head, a, bx, by, bz, thr_x<SELF>(ai, ib0 + 32u));
            push_x<2>(head, a, bx, by, bz, thr_x<SELF>(ai, ib0 + 64u));
            push_x<3>(head, a, bx, by, bz, thr_x<SELF>(ai, ib0 + 96u));
        }
        if (__any_sync(0xffffffffu, head != q)) flush_x<SELF>((head - q) >> 8, a_lo, ib0, bx, by, bz);
    }

    // ---- midpoint line of sight ----

    // Load one b-point into lane registers (shifted into A's frame) and into
    // the warp's b copies used by the flush.
    __device__ __forceinline__ void put_b(int p, bool ok, float x, float y, float z, uint32_t i, float (&bx)[P],
                                          float (&by)[P], float (&bz)[P], float (&hb)[P]) const
    {
        if (!ok) {
            // a missing point sits at 1e18 per axis: its threshold (~1.5e36)
            // exceeds every a.b' (|a| < 2^31, so below 1e28) and never passes
            x = y = z = 1e18f;
            i = 0;
        }
        bx[p] = x;
        by[p] = y;
        bz[p] = z;
        const float b2 = __fmaf_rn(z, z, __fmaf_rn(y, y, __fmul_rn(x, x)));
        hb[p] = __fsub_rn(__fmul_rn(0.5f, __fsub_rn(b2, prm.hit_max)), prm.dot_margin);
        asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(bc + 16u * bslot((uint32_t)(p * 32 + lane))),
                     "f"(bx[p]), "f"(by[p]), "f"(bz[p]), "f"(__uint_as_float(i))
                     : "memory");
    }

    // This lane's b-points and push thresholds from the warp's b copies (a
    // missing point was stored at 1e18 per axis, so its threshold never passes).
    __device__ __forceinline__ void reload_b(float (&bx)[P], float (&by)[P], float (&bz)[P], float (&hb)[P]) const
    {
#pragma unroll
        for (int p = 0; p < P; p++) {
            const float4 v = lds128(bc + 16u * bslot((uint32_t)(p * 32 + lane)));
            bx[p] = v.x;
            by[p] = v.y;
            bz[p] = v.z;
            const float b2 = __fmaf_rn(v.z, v.z, __fmaf_rn(v.y, v.y, __fmul_rn(v.x, v.x)));
            hb[p] = __fsub_rn(__fmul_rn(0.5f, __fsub_rn(b2, prm.hit_max)), prm.dot_margin);
        }
    }

    // all pairs of the a-chunk with one tile of b-points: the self cell of an
    // auto count (SELF, indices base..s1) or a packed tile at offset o_base of
    // the concatenated runs (n_seg runs, total points).
    template <bool SELF>
    __device__ __forceinline__ void tile_mid(uint32_t base, uint32_t s1, uint32_t o_base, int n_seg, uint32_t total,
                                         uint32_t orig_ax)
    {
        float bx[P], by[P], bz[P], hb[P];
        if (SELF) {
            // the self cell: A's own frame, no shift
#pragma unroll
            for (int p = 0; p < P; p++) {
                const uint32_t i = base + lane + 32u * p;
                const bool ok = i < s1;
                const float4 v = ok ? __ldg(m.pf + i) : make_float4(0.f, 0.f, 0.f, 0.f);
                put_b(p, ok, v.x, v.y, v.z, i, bx, by, bz, hb);
            }
        } else {
#pragma unroll
            for (int p = 0; p < P; p++) {
                const uint32_t f = o_base + (uint32_t)lane + 32u * p;
                const bool ok = f < total;
                const float4 e = ok ? lst()[f] : make_float4(0.f, 0.f, 0.f, 0.f);
                put_b(p, ok, e.x, e.y, e.z, __float_as_uint(e.w), bx, by, bz, hb);
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
                flush_mid((head - q) >> 6);
                head = q;
                // the b-points come back from the warp's copies: not held in
                // registers across the flush, whose binning needs them
                reload_b(bx, by, bz, hb);
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
        if (__any_sync(0xffffffffu, head != q)) flush_mid((head - q) >> 6);
    }
};

// The unit's b runs, built by one warp (one lane per neighbour row): the
// self cell of an auto count apart, every other run concatenated in row order
// with its offset in the concatenation.
template <bool MID>
__device__ void build_segments(const CountParams &prm, const Mesh &m, const Term &tm, int cell,
                               int lane)
{
    const int n_c = prm.n_c;
    const int ax = cell % n_c, ay = (cell / n_c) % n_c, az = cell / (n_c * n_c);
    const bool periodic = prm.geometry == TPCF_PERIODIC;
    const uint32_t *cs = m.cellstart + (size_t)tm.cat_b * prm.n_cells;
    const uint32_t oay = sh_orig<MID>(prm)[ay], oaz = sh_orig<MID>(prm)[az];
    uint32_t ns_total = 0, pts_total = 0;
    if (lane == 0) {
        sh_misc()[4] = 0;
        sh_misc()[5] = 0;
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
                sy = (float)(int)(sh_orig<MID>(prm)[y] - oay);
                sz = (float)(int)(sh_orig<MID>(prm)[z] - oaz);
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
                    sh_misc()[4] = (int)cs[rowkey + ax];
                    sh_misc()[5] = (int)cs[rowkey + ax + 1];
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
            sh_segs()[ns_total + n_ex + i] = g;
            p_ex += s1[i] - s0[i];
        }
        ns_total += n_all;
        pts_total += p_all;
    }
    if (lane == 0) {
        sh_misc()[1] = (int)ns_total;
        sh_misc()[2] = (int)pts_total;
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
                                                                float4 *__restrict__ scratch,
                                                                int persistent, int term_pl, int chunk)
{
    const VarOff vo = var_offsets(prm, MID);
    const int tid = threadIdx.x;
    const unsigned long long t_start = gtimer();
    {
        unsigned long long *T = (unsigned long long *)(smem_raw + vo.T);
        float2 *lohi = (float2 *)(smem_raw + vo.lohi);
        uint32_t *orig = (uint32_t *)(smem_raw + vo.orig);
        int *hist = (int *)(smem_raw + vo.hist);
        for (int i = tid; i <= prm.n_s; i += blockDim.x) T[i] = prm.T[i];
        for (int i = tid; i <= prm.n_s + 1; i += blockDim.x) lohi[i] = make_float2(prm.lo[i], prm.hi[i]);
        for (int i = tid; i <= prm.n_c; i += blockDim.x) orig[i] = m.orig[i];
        if (!LIN) {
            int16_t *table = (int16_t *)(smem_raw + vo.table);
            for (int i = tid; i < prm.tab_n; i += blockDim.x) table[i] = table_g[i];
        }
        for (int i = tid; i < prm.nbin; i += blockDim.x) hist[i] = 0;
        if (tid < 3 * WARPS) sh_stat()[tid] = 0ull;
    }

    Ctx<MU, MID, LIN> cx{prm, m, tid & 31, tid >> 5, 0u, 0u, 0u, 0u, 0u, nullptr, 0u, 0u, 0u, 0u, 0u, 0u,
                         0.f, 0.f, 0.f, 0u, 0u};
    cx.scr = scratch + (size_t)blockIdx.x * SCR;
    const uint32_t sbase = saddr(smem_raw);
    cx.hdum = sbase + vo.hist + 4u * ((uint32_t)prm.nbin + (uint32_t)cx.lane);
    if (MID) {
        const uint32_t qw = sbase + o_q(true) + (uint32_t)cx.warp * (QN * 32 * 2 * 2);
        cx.q = qw + 2u * (uint32_t)cx.lane;
        cx.cq = qw + QN * 32 * 2;
        cx.bc = sbase + O_B + (uint32_t)cx.warp * (P * 33 * 16);
    } else {
        cx.q = sbase + o_q(false) + (uint32_t)cx.warp * ((QX + 1) * 32 * 8) + 8u * (uint32_t)cx.lane;
    }
    cx.abase = sbase + O_A;
    cx.hbase = sbase + vo.hist;
    if (!MID)
        for (uint32_t k = 0; k <= (uint32_t)QX; k++) sts64(cx.q + k * 256u, prm.sent_d2, prm.sent_dx);
    {
        // classify encodes the s bin with the bias of B's bit pattern on the
        // linear path, the mu bin always (see classify)
        const uint32_t kB = 0x4B400000u;
        const uint32_t sb = LIN ? kB : 0u;
        cx.hadj = cx.hbase - 4u * (MU ? sb * (uint32_t)prm.n_mu + kB : sb);
    }

    // per-launch mode: this block walks the chunks of cells blockIdx.x,
    // blockIdx.x + gridDim.x, ... of one term
    const uint32_t n_units = persistent ? *n_units_p : 0u;
    uint32_t pl_a = 0, pl_end = 0, pl_next = blockIdx.x, pl_cell = 0;
    // the first unit is claimed here, every later one during the previous
    // unit's drain (the barrier that ends a unit publishes it)
    if (tid == 0) {
        sh_misc()[0] = persistent ? (int)atomicAdd(claim, 1u) : 0;
        sh_misc()[3] = 0;
    }
    if (tid < NB) sh_misc()[M_BKT + tid] = 0;
    __syncthreads();

    for (;;) {
        Unit un;
        if (persistent) {
            const uint32_t u = (uint32_t)sh_misc()[0];
            if (u >= n_units) break;
            un = units[u];
        } else {
            while (pl_a >= pl_end && pl_next < (uint32_t)prm.n_cells) {
                const size_t gk = (size_t)terms[term_pl].cat_a * prm.n_cells + pl_next;
                pl_a = m.cellstart[gk];
                pl_end = m.cellstart[gk + 1];
                pl_cell = pl_next;
                pl_next += gridDim.x;
            }
            if (pl_a >= pl_end) break;
            un.term = term_pl;
            un.cell = (int)pl_cell;
            un.a0 = pl_a;
            un.a1 = min(pl_end, pl_a + (uint32_t)chunk);
            pl_a = un.a1;
        }
        cx.a0 = un.a0;
        cx.na = un.a1 - un.a0;
        {
            // the a-chunk and its bounding box (cell-relative coordinates are
            // >= 0, so float bit patterns order as unsigned integers)
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            const bool ok = (uint32_t)tid < cx.na;   // na <= UNIT_CHUNK <= blockDim.x
            if (ok) {
                v = __ldg(m.pf + un.a0 + tid);
                sh_a()[tid] = v;
            }
            if (tid < UNIT_CHUNK) {
                const unsigned bx = __float_as_uint(v.x), by = __float_as_uint(v.y), bz = __float_as_uint(v.z);
                const unsigned lx = __reduce_min_sync(0xffffffffu, ok ? bx : 0xFFFFFFFFu);
                const unsigned ly = __reduce_min_sync(0xffffffffu, ok ? by : 0xFFFFFFFFu);
                const unsigned lz = __reduce_min_sync(0xffffffffu, ok ? bz : 0xFFFFFFFFu);
                const unsigned hx = __reduce_max_sync(0xffffffffu, ok ? bx : 0u);
                const unsigned hy = __reduce_max_sync(0xffffffffu, ok ? by : 0u);
                const unsigned hz = __reduce_max_sync(0xffffffffu, ok ? bz : 0u);
                // per-warp partial boxes after the a-chunk (chunk_box)
                if (cx.lane == 0) {
                    sh_a()[UNIT_CHUNK + cx.warp] = make_float4(__uint_as_float(lx), __uint_as_float(ly),
                                                             __uint_as_float(lz), __uint_as_float(hx));
                    sh_a()[UNIT_CHUNK + 4 + cx.warp] = make_float4(__uint_as_float(hy), __uint_as_float(hz), 0.f, 0.f);
                }
            }
        }
        if (cx.warp == 0) build_segments<MID>(prm, m, terms[un.term], un.cell, cx.lane);
        const int n_c = prm.n_c;
        const int ax = un.cell % n_c, ay = (un.cell / n_c) % n_c, az = un.cell / (n_c * n_c);
        const uint32_t oax = sh_orig<MID>(prm)[ax];
        {
            // x shift of every cell column into A's frame, for the filter
            float *sxf = (float *)(smem_raw + vo.sxf);
            for (int c = tid; c < n_c; c += blockDim.x) sxf[c] = (float)(int)(sh_orig<MID>(prm)[c] - oax);
        }
        if (MID) {
            cx.gx = 2.0f * (float)((long long)oax - prm.obs[0]);
            cx.gy = 2.0f * (float)((long long)sh_orig<MID>(prm)[ay] - prm.obs[1]);
            cx.gz = 2.0f * (float)((long long)sh_orig<MID>(prm)[az] - prm.obs[2]);
        }
        __syncthreads();
        const int ns = sh_misc()[1];
        const uint32_t total = (uint32_t)sh_misc()[2];
        const uint32_t self0 = (uint32_t)sh_misc()[4], self1 = (uint32_t)sh_misc()[5];
        const uint32_t n_self = (self1 - self0 + TILE - 1) / TILE;
        // The neighbour runs are filtered window by window into the block's
        // scratch and tiled densely; the self cell (auto counts) is tiled
        // directly in the first window.
        for (uint32_t w0 = 0;; w0 += CAP) {
            const uint32_t win = min((uint32_t)CAP, total - min(total, w0));
            cx.filter_window(w0, win, ns);
            __syncthreads();
            if (cx.warp == 0) cx.bucket_starts();
            uint32_t F = 0;
#pragma unroll
            for (int k = 0; k < WARPS; k++) F += (uint32_t)sh_misc()[M_CNT + k];
            __syncthreads();
            cx.scatter_window();
            __syncthreads();
            const uint32_t ns_w = (w0 == 0) ? n_self : 0u;
            const uint32_t nt = ns_w + (F + TILE - 1) / TILE;
            // tiles are claimed one at a time from a shared counter (its first
            // WARPS values are implicit), so warps finish a window together
            for (uint32_t ti = cx.warp; ti < nt;) {
                if (ti < ns_w) {
                    const uint32_t base = self0 + ti * TILE;
                    if (cx.lane == 0) sh_stat()[cx.warp] += (unsigned long long)min(self1 - base, (uint32_t)TILE) * cx.na;
                    if (MID) cx.template tile_mid<true>(base, self1, 0u, ns, F, oax);
                    else cx.template tile_x<true>(base, self1, 0u, ns, F, oax);
                } else {
                    const uint32_t ob = (ti - ns_w) * TILE;
                    if (cx.lane == 0) sh_stat()[cx.warp] += (unsigned long long)min(F - ob, (uint32_t)TILE) * cx.na;
                    if (MID) cx.template tile_mid<false>(0u, 0u, ob, ns, F, oax);
                    else cx.template tile_x<false>(0u, 0u, ob, ns, F, oax);
                }
                uint32_t nx = 0;
                if (cx.lane == 0) nx = (uint32_t)atomicAdd(&sh_misc()[3], 1) + WARPS;
                ti = __shfl_sync(0xffffffffu, nx, 0);
            }
            const bool last = w0 + CAP >= total;
            if (last && cx.n_list) cx.recheck_list();   // the list refers to this unit's histogram
            __syncthreads();   // every warp is done with this window's scratch, counter and histogram adds
            if (tid == 0) sh_misc()[3] = 0;
            discard_l2(cx.lst(), (F * 16u + 127u) & ~127u, (uint32_t)tid, blockDim.x);   // the window list is spent
            if (last) break;
        }
        // drain the block histogram into the term's int64 histogram
        if (persistent && tid == 0) sh_misc()[0] = (int)atomicAdd(claim, 1u);   // the next unit
        long long *const th = terms[un.term].hist;
        for (int b = tid; b < prm.nbin; b += blockDim.x) {
            // 32-bit counters read as unsigned: a unit adds fewer than 2^32 pairs
            // to any bin (the host caps the unit size by the largest catalogue)
            const unsigned v = ((unsigned *)(smem_raw + vo.hist))[b];
            cx.n_binned += v;   // every binned pair passes through the block histogram
            if (v) {
                atomicAdd((unsigned long long *)&th[b], (unsigned long long)v);
                ((unsigned *)(smem_raw + vo.hist))[b] = 0u;
            }
        }
        __syncthreads();
    }
    // work statistics (candidate counts are kept per warp in shared memory)
    unsigned long long ex = cx.n_exact, bn = cx.n_binned, cd = (cx.lane == 0) ? sh_stat()[cx.warp] : 0ull;
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
        record_warp_span(stats, t_start);
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
    return (int)var_offsets(p, uses_midpoint(p)).end;
}

size_t paircount_scratch_bytes(int blocks) { return (size_t)blocks * SCR * sizeof(float4); }

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
    float4 *scratch = (float4 *)pl.scratch;
    void *args[] = {(void *)&p,     (void *)&m,     (void *)&terms, (void *)&units,        (void *)&n_units,
                    (void *)&claim, (void *)&table, (void *)&stats, (void *)&scratch,      (void *)&pl.persistent,
                    (void *)&pl.term, (void *)&pl.chunk};
    return cudaLaunchKernel(select_kernel(p), dim3(pl.blocks), dim3(WARPS * 32), args, (size_t)pl.smem_bytes, s);
}

}  // namespace tpcf
