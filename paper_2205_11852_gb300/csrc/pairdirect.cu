// Direct binned pair counting on the chaining mesh (Sect. 2.1: DD, DR_i and
// RR_i counts; Sect. 4.3: bins in separation s and in mu) for linear s bins
// starting at 0: s only, mu with the line of sight along x, or mu with the
// line of sight from the observer to the pair's midpoint (cut-sky mocks).
//
// Work decomposition.  A unit is a chunk of at most 64 sorted points of one
// mesh cell A, paired with the neighbourhood of A in catalogue b.  Each warp
// owns a unit on its own: it stages the a-chunk in its region of shared
// memory, streams the b-points of the neighbourhood (the self cell of an
// auto count as it is, every other neighbour cell through a filter that
// keeps a point only if its distance to the a-chunk's bounding box is below
// the last edge) into its own buffer, and counts every full tile of 128
// b-points (4 per lane) against the a-chunk as soon as it is there.  The
// warps of a block share one histogram, so a block works through a chunk of
// consecutive units of one term at a time (units are ordered by term); block
// barriers come only between such chunks.
//
// Arithmetic.  Coordinates are exact integer offsets from A's lower corner,
// converted once to FP32 in units of one s bin, so the s bin of a pair is
// floor(u) with u its FP32 separation.  Two pairs run side by side in packed
// FP32 (f32x2) arithmetic.  Per pair: d2 from the differences, r = rsqrt(d2)
// (MUFU), S = floor(d2 r) by one round-toward-zero FMA onto a power-of-two
// offset, the residual d2 r - floor(d2 r) - 1/2 by one more FMA, and the
// signed mu bin T = floor(n_mu dx r) at both ends of the error interval
// [n_mu dx - m, n_mu dx + m] r.  A pair is certain when its s residual lies
// within cs of 1/2 and both mu floors agree; cs and m come from a rigorous
// bound on the FP32 errors (plan.cpp).  Every pair, certain or not, is added
// to the histogram at (S, T-) with one shared-memory atomic; a pair at or
// beyond the last edge lands in the histogram's spare last row.  The check
// costs two compares per pair, or-ed into one predicate per a-point; an
// a-point with an uncertain pair in any lane takes the rare path, which
// recomputes its pairs with a flag each, takes back the uncertain ones' adds
// and rechecks them exactly from the integer coordinates (64-bit squared
// distances, a 128-bit mu test), 32 at a time, so every count equals the
// integer definition bit for bit.  With the midpoint line of sight the mu
// bin comes from l = a + b - 2 o (o the observer), mu = (l.d) r rl with
// rl = rsqrt(|l|^2), its floor and residual against a per-pair bound
// c2 + c1 r + c3 rl (plan.cpp), the rest as above.
//
// Histogram.  R copies of a (n_s + 1) x C table of 32-bit counters, lane l
// adding to copy l mod R, so the 32 adds of a warp fall in distinct banks
// (R = 32) or at most two per bank (R = 16).  mu is binned by sign, C =
// 2 n_mu + 2 columns from -n_mu - 1 to n_mu, and folded to |mu| when the
// table is drained into the term's int64 histogram: when the block moves to
// another term, or before its 32-bit counters could wrap.
#include "pair_device.cuh"

namespace tpcf {

namespace {

constexpr int NP = 4;               // b-points per lane
constexpr int NQ = NP / 2;          // packed pairs per lane
constexpr int TB = 32 * NP;         // b-points per tile
constexpr int BUF = TB + 128;       // per-warp b buffer: a tile plus one filter pass
constexpr int XCAP = 96;            // per-warp list of pairs awaiting the exact recheck
constexpr float MAG_S = 8388608.0f;       // 2^23: fma.rz(d2, r, MAG_S) = 2^23 + floor(d2 r) for 0 <= d2 r < 2^23
constexpr uint32_t MAG_S_BITS = 0x4B000000u;
constexpr float MAG_T = 12582912.0f;      // 1.5 * 2^23: = 1.5 * 2^23 + floor(t) for |t| < 2^22
constexpr uint32_t MAG_T_BITS = 0x4B400000u;
constexpr float FAR = 1.0e5f;             // a padding b-point: far beyond every edge, still finite
static_assert(DIRECT_ACHUNK % 32 == 0 && DIRECT_ACHUNK <= 64, "a-chunk load: two points per lane");

__host__ __device__ constexpr uint32_t al16(uint32_t x) { return (x + 15u) & ~15u; }

// Shared memory: the block's histogram, T, misc words, then one region per
// warp: a-records (3 float4 per a-point), the b buffer (float4: x, y, z in
// bins and the b index), the unit's runs (first index, offset in the
// concatenation) and the recheck list.
struct DOff {
    uint32_t hist, T, misc, warp0, wstride;
    uint32_t arec, buf, runs, xl;   // offsets inside a warp's region
    uint32_t end;
};
__host__ __device__ inline DOff d_off(int n_s, int n_rows, int R, int C, int W)
{
    DOff o;
    o.hist = 0;
    o.T = al16(4u * (uint32_t)((n_s + 1) * C * R));
    o.misc = al16(o.T + 8u * (uint32_t)(n_s + 1));
    o.warp0 = o.misc + 64u;
    o.arec = 0;
    o.buf = o.arec + 48u * DIRECT_ACHUNK;
    o.runs = o.buf + 16u * BUF;
    o.xl = al16(o.runs + 8u * (uint32_t)(2 * n_rows + 1));
    o.wstride = al16(o.xl + 8u * XCAP);
    o.end = o.warp0 + o.wstride * (uint32_t)W;
    return o;
}

extern __shared__ __align__(16) unsigned char dsm[];

__device__ __forceinline__ void red_add(uint32_t a, uint32_t v)
{
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// An a-point's record, each value duplicated for the packed operands: -a_x,
// -a_y, -a_z, then with the x line of sight p = m - n_mu a_x, q = -m - n_mu a_x,
// with the midpoint line of sight (p, q, w) = a - 2 o (o: the observer).
struct ARec {
    float2 nax, nay, naz, p, q, w;
};

// Histogram address of a pair with s-row word bits(S) and signed-mu-column
// word bits(T-): (bits(S) << LS) + (bits(T-) << LT) + Kl, with LT = log2(4 R)
// and LS = LT + log2(C), so that the row and column strides are shifts.
template <int R, int LOGC>
struct Sh {
    static constexpr int LT = R == 32 ? 7 : (R == 16 ? 6 : -1);
    static constexpr int LS = LT + LOGC;
    static_assert(LT > 0, "R is 16 or 32");
};

__device__ __forceinline__ uint64_t u64of(float2 v) { return *reinterpret_cast<uint64_t *>(&v); }

// Constant operand pairs of the packed arithmetic (the last five: midpoint
// line of sight only).
struct K2 {
    uint64_t tiny, ms, m1, mh, mt, nm, tinyl, mhalf, c1n, c3n, c05;
};

// One packed pair of pairs (b_p, a), (b_p', a) in hand-written PTX: the
// packed s floor word S and s residual FS (the tiny addend, r = rsqrt(d2) by
// MUFU) and, with mu bins, the signed mu floor words.  V = 1 (x line of
// sight): TP, TM = the floors at both ends of the error interval.  V = 2
// (midpoint line of sight): l = b + (a - 2 o), mu = (l.d) r rl with
// rl = rsqrt(|l|^2 + tinyl), TM = floor(n_mu mu), TP = its residual
// n_mu mu - TM - 1/2, CB = 1/2 - c2 - c1 r - c3 rl (certain when |TP| <= CB).
template <int V>
__device__ __forceinline__ void pair2_core(uint64_t bx, uint64_t by, uint64_t bz, const ARec &a, const K2 &k,
                                           uint64_t &S, uint64_t &FS, uint64_t &TP, uint64_t &TM, uint64_t &CB)
{
    if (V == 2) {
        asm("{\n\t"
            ".reg .b64 dx, dy, dz, d2, r, h, lx, ly, lz, q, l2, rl, w, mu, ht, cb;\n\t"
            ".reg .f32 d2x, d2y, rx, ry, l2x, l2y, rlx, rly;\n\t"
            "add.rn.f32x2 dx, %5, %8;\n\t"
            "add.rn.f32x2 dy, %6, %9;\n\t"
            "add.rn.f32x2 dz, %7, %10;\n\t"
            "fma.rn.f32x2 d2, dx, dx, %14;\n\t"
            "fma.rn.f32x2 d2, dy, dy, d2;\n\t"
            "fma.rn.f32x2 d2, dz, dz, d2;\n\t"
            "mov.b64 {d2x, d2y}, d2;\n\t"
            "rsqrt.approx.ftz.f32 rx, d2x;\n\t"
            "rsqrt.approx.ftz.f32 ry, d2y;\n\t"
            "mov.b64 r, {rx, ry};\n\t"
            "fma.rz.f32x2 %0, d2, r, %15;\n\t"
            "fma.rn.f32x2 h, %0, %16, %17;\n\t"
            "fma.rn.f32x2 %1, d2, r, h;\n\t"
            "add.rn.f32x2 lx, %5, %11;\n\t"
            "add.rn.f32x2 ly, %6, %12;\n\t"
            "add.rn.f32x2 lz, %7, %13;\n\t"
            "mul.rn.f32x2 q, lx, dx;\n\t"
            "fma.rn.f32x2 q, ly, dy, q;\n\t"
            "fma.rn.f32x2 q, lz, dz, q;\n\t"
            "fma.rn.f32x2 l2, lx, lx, %20;\n\t"
            "fma.rn.f32x2 l2, ly, ly, l2;\n\t"
            "fma.rn.f32x2 l2, lz, lz, l2;\n\t"
            "mov.b64 {l2x, l2y}, l2;\n\t"
            "rsqrt.approx.ftz.f32 rlx, l2x;\n\t"
            "rsqrt.approx.ftz.f32 rly, l2y;\n\t"
            "mov.b64 rl, {rlx, rly};\n\t"
            "mul.rn.f32x2 w, r, rl;\n\t"
            "mul.rn.f32x2 mu, q, w;\n\t"
            "fma.rz.f32x2 %3, mu, %19, %18;\n\t"
            "fma.rn.f32x2 ht, %3, %16, %18;\n\t"
            "fma.rn.f32x2 %2, mu, %19, ht;\n\t"
            "add.rn.f32x2 %2, %2, %21;\n\t"
            "fma.rn.f32x2 cb, %23, rl, %24;\n\t"
            "fma.rn.f32x2 %4, %22, r, cb;\n\t"
            "}"
            : "=&l"(S), "=&l"(FS), "=&l"(TP), "=&l"(TM), "=&l"(CB)
            : "l"(bx), "l"(by), "l"(bz), "l"(u64of(a.nax)), "l"(u64of(a.nay)), "l"(u64of(a.naz)), "l"(u64of(a.p)),
              "l"(u64of(a.q)), "l"(u64of(a.w)), "l"(k.tiny), "l"(k.ms), "l"(k.m1), "l"(k.mh), "l"(k.mt), "l"(k.nm),
              "l"(k.tinyl), "l"(k.mhalf), "l"(k.c1n), "l"(k.c3n), "l"(k.c05));
    } else if (V == 1) {
        asm("{\n\t"
            ".reg .b64 dx, dy, dz, d2, r, h, xp, xm;\n\t"
            ".reg .f32 d2x, d2y, rx, ry;\n\t"
            "add.rn.f32x2 dx, %4, %7;\n\t"
            "add.rn.f32x2 dy, %5, %8;\n\t"
            "add.rn.f32x2 dz, %6, %9;\n\t"
            "fma.rn.f32x2 d2, dx, dx, %12;\n\t"
            "fma.rn.f32x2 d2, dy, dy, d2;\n\t"
            "fma.rn.f32x2 d2, dz, dz, d2;\n\t"
            "mov.b64 {d2x, d2y}, d2;\n\t"
            "rsqrt.approx.ftz.f32 rx, d2x;\n\t"
            "rsqrt.approx.ftz.f32 ry, d2y;\n\t"
            "mov.b64 r, {rx, ry};\n\t"
            "fma.rz.f32x2 %0, d2, r, %13;\n\t"
            "fma.rn.f32x2 h, %0, %14, %15;\n\t"
            "fma.rn.f32x2 %1, d2, r, h;\n\t"
            "fma.rn.f32x2 xp, %4, %17, %10;\n\t"
            "fma.rn.f32x2 xm, %4, %17, %11;\n\t"
            "fma.rz.f32x2 %2, xp, r, %16;\n\t"
            "fma.rz.f32x2 %3, xm, r, %16;\n\t"
            "}"
            : "=&l"(S), "=&l"(FS), "=&l"(TP), "=&l"(TM)
            : "l"(bx), "l"(by), "l"(bz), "l"(u64of(a.nax)), "l"(u64of(a.nay)), "l"(u64of(a.naz)), "l"(u64of(a.p)),
              "l"(u64of(a.q)), "l"(k.tiny), "l"(k.ms), "l"(k.m1), "l"(k.mh), "l"(k.mt), "l"(k.nm));
        CB = 0;
    } else {
        asm("{\n\t"
            ".reg .b64 dx, dy, dz, d2, r, h;\n\t"
            ".reg .f32 d2x, d2y, rx, ry;\n\t"
            "add.rn.f32x2 dx, %2, %5;\n\t"
            "add.rn.f32x2 dy, %3, %6;\n\t"
            "add.rn.f32x2 dz, %4, %7;\n\t"
            "fma.rn.f32x2 d2, dx, dx, %8;\n\t"
            "fma.rn.f32x2 d2, dy, dy, d2;\n\t"
            "fma.rn.f32x2 d2, dz, dz, d2;\n\t"
            "mov.b64 {d2x, d2y}, d2;\n\t"
            "rsqrt.approx.ftz.f32 rx, d2x;\n\t"
            "rsqrt.approx.ftz.f32 ry, d2y;\n\t"
            "mov.b64 r, {rx, ry};\n\t"
            "fma.rz.f32x2 %0, d2, r, %9;\n\t"
            "fma.rn.f32x2 h, %0, %10, %11;\n\t"
            "fma.rn.f32x2 %1, d2, r, h;\n\t"
            "}"
            : "=&l"(S), "=&l"(FS)
            : "l"(bx), "l"(by), "l"(bz), "l"(u64of(a.nax)), "l"(u64of(a.nay)), "l"(u64of(a.naz)), "l"(k.tiny),
              "l"(k.ms), "l"(k.m1), "l"(k.mh));
        TP = TM = CB = 0;
    }
}

__device__ __forceinline__ float lo_f(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi_f(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }

// Histogram addresses of the two pairs: the s row (S clamped to the spare
// last row) and, with mu bins, the signed mu column of T-.
template <bool MU, int LS, int LT>
__device__ __forceinline__ void pair_addr(uint64_t S, uint64_t TM, float stop, uint32_t Kl, uint32_t &a0,
                                          uint32_t &a1)
{
    a0 = Kl + (__float_as_uint(fminf(lo_f(S), stop)) << LS);
    a1 = Kl + (__float_as_uint(fminf(hi_f(S), stop)) << LS);
    if (MU) {
        a0 += (uint32_t)TM << LT;
        a1 += (uint32_t)(TM >> 32) << LT;
    }
}

// Rare path: two pairs recomputed with one uncertainty flag each, by the
// same instructions as the hot path's PTX block (so bit for bit the same
// addresses and decisions).
template <int V, int LS, int LT>
__device__ __forceinline__ void pair2_flags(uint64_t bx, uint64_t by, uint64_t bz, const ARec &a, const K2 &k,
                                            float cs, float stop, uint32_t Kl, uint32_t &a0, uint32_t &a1, bool &f0,
                                            bool &f1)
{
    uint64_t S, FS, TP, TM, CB;
    pair2_core<V>(bx, by, bz, a, k, S, FS, TP, TM, CB);
    pair_addr<(V > 0), LS, LT>(S, TM, stop, Kl, a0, a1);
    f0 = fabsf(lo_f(FS)) > cs;
    f1 = fabsf(hi_f(FS)) > cs;
    if (V == 1) {
        f0 = f0 || lo_f(TP) != lo_f(TM);
        f1 = f1 || hi_f(TP) != hi_f(TM);
    } else if (V == 2) {
        f0 = f0 || fabsf(lo_f(TP)) > lo_f(CB);
        f1 = f1 || fabsf(hi_f(TP)) > hi_f(CB);
    }
}

// One a-point against this lane's four b-points (two packed pairs q = 0, 1),
// in one block of hand-written PTX so that the uncertainty of all four pairs
// accumulates in one predicate (setp with .or): the four histogram adds, and
// whether some pair of this lane is uncertain.  The loop runs two a-points per
// iteration (two independent blocks the scheduler interleaves) under one vote.  CHK (self
// cell): a pair with a >= b goes to the lane's spare word instead.
// Operands: %0 the lane's uncertainty; %1-%6 b (x, y, z) of q = 0, 1; %7-%11 the a-record;
// %12-%17 constants; %18 cs; %19 the s clamp; %20 Kl; %21, %22 LS, LT;
// CHK: %23 a index, %24-%27 b indices of slots 0-3, %28 spare word.
#define PD_DIFF(BX, BY, BZ)                          \
    "add.rn.f32x2 dx, " BX ", %7;\n\t"                 \
    "add.rn.f32x2 dy, " BY ", %8;\n\t"                 \
    "add.rn.f32x2 dz, " BZ ", %9;\n\t"                 \
    "fma.rn.f32x2 d2, dx, dx, %12;\n\t"                \
    "fma.rn.f32x2 d2, dy, dy, d2;\n\t"                 \
    "fma.rn.f32x2 d2, dz, dz, d2;\n\t"                 \
    "mov.b64 {d2x, d2y}, d2;\n\t"                      \
    "rsqrt.approx.ftz.f32 rx, d2x;\n\t"                \
    "rsqrt.approx.ftz.f32 ry, d2y;\n\t"                \
    "mov.b64 r, {rx, ry};\n\t"                         \
    "fma.rz.f32x2 s, d2, r, %13;\n\t"                  \
    "fma.rn.f32x2 h, s, %14, %15;\n\t"                 \
    "fma.rn.f32x2 fs, d2, r, h;\n\t"                   \
    "mov.b64 {sx, sy}, s;\n\t"                         \
    "mov.b64 {fx, fy}, fs;\n\t"                        \
    "abs.f32 fx, fx;\n\t"                              \
    "abs.f32 fy, fy;\n\t"                              \
    "setp.gtu.or.f32 p, fx, %18, p;\n\t"               \
    "setp.gtu.or.f32 p, fy, %18, p;\n\t"               \
    "min.f32 sx, sx, %19;\n\t"                         \
    "min.f32 sy, sy, %19;\n\t"                         \
    "mov.b32 ux, sx;\n\t"                              \
    "mov.b32 uy, sy;\n\t"                              \
    "shl.b32 ux, ux, %21;\n\t"                         \
    "shl.b32 uy, uy, %21;\n\t"                         \
    "add.u32 ux, ux, %20;\n\t"                         \
    "add.u32 uy, uy, %20;\n\t"
#define PD_MU(BX)                                    \
    "fma.rn.f32x2 xp, " BX ", %17, %10;\n\t"           \
    "fma.rn.f32x2 xm, " BX ", %17, %11;\n\t"           \
    "fma.rz.f32x2 tp, xp, r, %16;\n\t"                 \
    "fma.rz.f32x2 tm, xm, r, %16;\n\t"                 \
    "mov.b64 {px, py}, tp;\n\t"                        \
    "mov.b64 {mx, my}, tm;\n\t"                        \
    "setp.neu.or.f32 p, px, mx, p;\n\t"                \
    "setp.neu.or.f32 p, py, my, p;\n\t"                \
    "mov.b32 vx, mx;\n\t"                              \
    "mov.b32 vy, my;\n\t"                              \
    "shl.b32 vx, vx, %22;\n\t"                         \
    "shl.b32 vy, vy, %22;\n\t"                         \
    "add.u32 ux, ux, vx;\n\t"                          \
    "add.u32 uy, uy, vy;\n\t"
#define PD_CHK(IB0, IB1)                             \
    "setp.lt.u32 c, %23, " IB0 ";\n\t"                 \
    "selp.b32 ux, ux, %28, c;\n\t"                     \
    "setp.lt.u32 c, %23, " IB1 ";\n\t"                 \
    "selp.b32 uy, uy, %28, c;\n\t"
#define PD_RED                                       \
    "red.shared.add.u32 [ux], 1;\n\t"                  \
    "red.shared.add.u32 [uy], 1;\n\t"
#define PD_HEAD                                                                     \
    "{\n\t"                                                                           \
    ".reg .b64 dx, dy, dz, d2, r, s, h, fs, xp, xm, tp, tm;\n\t"                      \
    ".reg .f32 d2x, d2y, rx, ry, sx, sy, fx, fy, px, py, mx, my;\n\t"                 \
    ".reg .b32 ux, uy, vx, vy;\n\t"                                                   \
    ".reg .pred p, c;\n\t"                                                            \
    "setp.ne.u32 p, %20, %20;\n\t"
#define PD_TAIL                                      \
    "selp.u32 %0, 1, 0, p;\n\t"                        \
    "}"

// Midpoint line of sight.  Operands: %0 the lane's uncertainty; %1-%6 b;
// %7-%9 -a; %10-%12 a - 2 o; %13-%23 constants (tiny, ms, m1, mh, mt, nm,
// tinyl, -1/2, c1n, c3n, c05); %24 cs; %25 the s clamp; %26 Kl; %27, %28 LS,
// LT; self-cell tiles: %29 the a index, %30-%33 b limits, %34 the spare word.
// The mu residual is (n_mu mu - floor(n_mu mu)) - 1/2: 1.5 * 2^23 - 1/2 has no
// FP32 form, so the half is subtracted after the fraction.
#define PM_PAIR(BX, BY, BZ)                          \
    "add.rn.f32x2 dx, " BX ", %7;\n\t"                 \
    "add.rn.f32x2 dy, " BY ", %8;\n\t"                 \
    "add.rn.f32x2 dz, " BZ ", %9;\n\t"                 \
    "fma.rn.f32x2 d2, dx, dx, %13;\n\t"                \
    "fma.rn.f32x2 d2, dy, dy, d2;\n\t"                 \
    "fma.rn.f32x2 d2, dz, dz, d2;\n\t"                 \
    "mov.b64 {d2x, d2y}, d2;\n\t"                      \
    "rsqrt.approx.ftz.f32 rx, d2x;\n\t"                \
    "rsqrt.approx.ftz.f32 ry, d2y;\n\t"                \
    "mov.b64 r, {rx, ry};\n\t"                         \
    "fma.rz.f32x2 s, d2, r, %14;\n\t"                  \
    "fma.rn.f32x2 h, s, %15, %16;\n\t"                 \
    "fma.rn.f32x2 fs, d2, r, h;\n\t"                   \
    "add.rn.f32x2 lx, " BX ", %10;\n\t"                \
    "add.rn.f32x2 ly, " BY ", %11;\n\t"                \
    "add.rn.f32x2 lz, " BZ ", %12;\n\t"                \
    "mul.rn.f32x2 q, lx, dx;\n\t"                      \
    "fma.rn.f32x2 q, ly, dy, q;\n\t"                   \
    "fma.rn.f32x2 q, lz, dz, q;\n\t"                   \
    "fma.rn.f32x2 l2, lx, lx, %19;\n\t"                \
    "fma.rn.f32x2 l2, ly, ly, l2;\n\t"                 \
    "fma.rn.f32x2 l2, lz, lz, l2;\n\t"                 \
    "mov.b64 {l2x, l2y}, l2;\n\t"                      \
    "rsqrt.approx.ftz.f32 rlx, l2x;\n\t"               \
    "rsqrt.approx.ftz.f32 rly, l2y;\n\t"               \
    "mov.b64 rl, {rlx, rly};\n\t"                      \
    "mul.rn.f32x2 w, r, rl;\n\t"                       \
    "mul.rn.f32x2 mu, q, w;\n\t"                       \
    "fma.rz.f32x2 tm, mu, %18, %17;\n\t"               \
    "fma.rn.f32x2 ht, tm, %15, %17;\n\t"               \
    "fma.rn.f32x2 fm, mu, %18, ht;\n\t"                \
    "add.rn.f32x2 fm, fm, %20;\n\t"                    \
    "fma.rn.f32x2 cb, %22, rl, %23;\n\t"               \
    "fma.rn.f32x2 cb, %21, r, cb;\n\t"                 \
    "mov.b64 {sx, sy}, s;\n\t"                         \
    "mov.b64 {fx, fy}, fs;\n\t"                        \
    "mov.b64 {gx, gy}, fm;\n\t"                        \
    "mov.b64 {kx, ky}, cb;\n\t"                        \
    "mov.b64 {mx, my}, tm;\n\t"                        \
    "abs.f32 fx, fx;\n\t"                              \
    "abs.f32 fy, fy;\n\t"                              \
    "abs.f32 gx, gx;\n\t"                              \
    "abs.f32 gy, gy;\n\t"                              \
    "setp.gtu.or.f32 p, fx, %24, p;\n\t"               \
    "setp.gtu.or.f32 p, fy, %24, p;\n\t"               \
    "setp.gtu.or.f32 p, gx, kx, p;\n\t"                \
    "setp.gtu.or.f32 p, gy, ky, p;\n\t"                \
    "min.f32 sx, sx, %25;\n\t"                         \
    "min.f32 sy, sy, %25;\n\t"                         \
    "mov.b32 ux, sx;\n\t"                              \
    "mov.b32 uy, sy;\n\t"                              \
    "shl.b32 ux, ux, %27;\n\t"                         \
    "shl.b32 uy, uy, %27;\n\t"                         \
    "add.u32 ux, ux, %26;\n\t"                         \
    "add.u32 uy, uy, %26;\n\t"                         \
    "mov.b32 vx, mx;\n\t"                              \
    "mov.b32 vy, my;\n\t"                              \
    "shl.b32 vx, vx, %28;\n\t"                         \
    "shl.b32 vy, vy, %28;\n\t"                         \
    "add.u32 ux, ux, vx;\n\t"                          \
    "add.u32 uy, uy, vy;\n\t"
#define PM_CHK(IB0, IB1)                             \
    "setp.lt.u32 c, %29, " IB0 ";\n\t"                 \
    "selp.b32 ux, ux, %34, c;\n\t"                     \
    "setp.lt.u32 c, %29, " IB1 ";\n\t"                 \
    "selp.b32 uy, uy, %34, c;\n\t"
#define PM_RED                                       \
    "red.shared.add.u32 [ux], 1;\n\t"                  \
    "red.shared.add.u32 [uy], 1;\n\t"
#define PM_HEAD                                                                                \
    "{\n\t"                                                                                      \
    ".reg .b64 dx, dy, dz, d2, r, s, h, fs, lx, ly, lz, q, l2, rl, w, mu, tm, ht, fm, cb;\n\t"   \
    ".reg .f32 d2x, d2y, rx, ry, l2x, l2y, rlx, rly, sx, sy, fx, fy, gx, gy, kx, ky, mx, my;\n\t" \
    ".reg .b32 ux, uy, vx, vy;\n\t"                                                              \
    ".reg .pred p, c;\n\t"                                                                       \
    "setp.ne.u32 p, %26, %26;\n\t"

template <int V, bool CHK, int LS, int LT>
__device__ __forceinline__ bool apoint(const float2 (&BX)[NQ], const float2 (&BY)[NQ], const float2 (&BZ)[NQ],
                                       const ARec &a, const K2 &k, float cs, float stop, uint32_t Kl, uint32_t ia,
                                       const uint32_t (&IB)[NP], uint32_t dump)
{
    static_assert(NQ == 2, "the PTX block covers two packed pairs");
    constexpr bool MU = V > 0;
    uint32_t any;
    if (V == 2) {
#define PM_IN                                                                                                    \
    "l"(u64of(BX[0])), "l"(u64of(BY[0])), "l"(u64of(BZ[0])), "l"(u64of(BX[1])), "l"(u64of(BY[1])),             \
        "l"(u64of(BZ[1])), "l"(u64of(a.nax)), "l"(u64of(a.nay)), "l"(u64of(a.naz)), "l"(u64of(a.p)),            \
        "l"(u64of(a.q)), "l"(u64of(a.w)), "l"(k.tiny), "l"(k.ms), "l"(k.m1), "l"(k.mh), "l"(k.mt), "l"(k.nm),   \
        "l"(k.tinyl), "l"(k.mhalf), "l"(k.c1n), "l"(k.c3n), "l"(k.c05), "f"(cs), "f"(stop), "r"(Kl), "n"(LS), \
        "n"(LT)
        if (CHK)
            asm volatile(PM_HEAD PM_PAIR("%1", "%2", "%3") PM_CHK("%30", "%31") PM_RED PM_PAIR("%4", "%5", "%6")
                             PM_CHK("%32", "%33") PM_RED "selp.u32 %0, 1, 0, p;\n\t}"
                         : "=r"(any)
                         : PM_IN, "r"(ia), "r"(IB[0]), "r"(IB[1]), "r"(IB[2]), "r"(IB[3]), "r"(dump)
                         : "memory");
        else
            asm volatile(PM_HEAD PM_PAIR("%1", "%2", "%3") PM_RED PM_PAIR("%4", "%5", "%6") PM_RED
                         "selp.u32 %0, 1, 0, p;\n\t}"
                         : "=r"(any)
                         : PM_IN
                         : "memory");
#undef PM_IN
        return any != 0;
    }
#define PD_IN                                                                                                     \
    "l"(u64of(BX[0])), "l"(u64of(BY[0])), "l"(u64of(BZ[0])), "l"(u64of(BX[1])), "l"(u64of(BY[1])),              \
        "l"(u64of(BZ[1])), "l"(u64of(a.nax)), "l"(u64of(a.nay)), "l"(u64of(a.naz)), "l"(u64of(a.p)),             \
        "l"(u64of(a.q)), "l"(k.tiny), "l"(k.ms), "l"(k.m1), "l"(k.mh), "l"(k.mt), "l"(k.nm), "f"(cs), "f"(stop), \
        "r"(Kl), "n"(LS), "n"(LT)
    if (MU && CHK) {
        asm volatile(PD_HEAD PD_DIFF("%1", "%2", "%3") PD_MU("%1") PD_CHK("%24", "%25") PD_RED
                         PD_DIFF("%4", "%5", "%6") PD_MU("%4") PD_CHK("%26", "%27") PD_RED PD_TAIL
                     : "=r"(any)
                     : PD_IN, "r"(ia), "r"(IB[0]), "r"(IB[1]), "r"(IB[2]), "r"(IB[3]), "r"(dump)
                     : "memory");
    } else if (MU) {
        asm volatile(PD_HEAD PD_DIFF("%1", "%2", "%3") PD_MU("%1") PD_RED PD_DIFF("%4", "%5", "%6") PD_MU("%4")
                         PD_RED PD_TAIL
                     : "=r"(any)
                     : PD_IN
                     : "memory");
    } else if (CHK) {
        asm volatile(PD_HEAD PD_DIFF("%1", "%2", "%3") PD_CHK("%24", "%25") PD_RED PD_DIFF("%4", "%5", "%6")
                         PD_CHK("%26", "%27") PD_RED PD_TAIL
                     : "=r"(any)
                     : PD_IN, "r"(ia), "r"(IB[0]), "r"(IB[1]), "r"(IB[2]), "r"(IB[3]), "r"(dump)
                     : "memory");
    } else {
        asm volatile(PD_HEAD PD_DIFF("%1", "%2", "%3") PD_RED PD_DIFF("%4", "%5", "%6") PD_RED PD_TAIL
                     : "=r"(any)
                     : PD_IN
                     : "memory");
    }
#undef PD_IN
    return any != 0;
}
#undef PD_DIFF
#undef PD_MU
#undef PD_CHK
#undef PD_RED
#undef PD_HEAD
#undef PD_TAIL
#undef PM_PAIR
#undef PM_CHK
#undef PM_RED
#undef PM_HEAD

// Per-lane histogram address constants (see Sh).
struct Addr {
    uint32_t Kl;
    uint32_t hb;      // histogram base (shared address) + 4 (lane mod R)
    uint32_t dump;    // this lane's word in the spare last row
};

// A warp's shared-memory region and its pending exact rechecks.
struct WarpMem {
    float4 *arec;     // a-records of the unit's a-chunk
    float4 *buf;      // b buffer: x, y, z in bins and the b index
    uint2 *runs;      // the unit's runs: (first b index, offset in their concatenation)
    uint2 *xl;        // pairs (a index, b index) awaiting the exact recheck
};

template <bool MID>
__device__ __forceinline__ ARec load_a(const float4 *arec, uint32_t ai)
{
    const float4 r0 = arec[3 * ai], r1 = arec[3 * ai + 1];
    if (MID) {
        const float4 r2 = arec[3 * ai + 2];
        return ARec{make_float2(r0.x, r0.y), make_float2(r0.z, r0.w), make_float2(r1.x, r1.y),
                    make_float2(r1.z, r1.w), make_float2(r2.x, r2.y), make_float2(r2.z, r2.w)};
    }
    const float2 r2 = *(const float2 *)&arec[3 * ai + 2];
    return ARec{make_float2(r0.x, r0.y), make_float2(r0.z, r0.w), make_float2(r1.x, r1.y), make_float2(r1.z, r1.w),
                r2, make_float2(0.f, 0.f)};
}

__device__ __forceinline__ void xl_put(uint2 *xl, uint32_t i, uint32_t ia, uint32_t ib) { xl[i] = make_uint2(ia, ib); }

// exact recheck of the n listed pairs, one per lane; returns the number rechecked by this lane
template <bool MU, int R, int LOGC>
__device__ __forceinline__ uint32_t recheck(const CountParams &prm, const DirectParams &dp, const Mesh &m,
                                            const unsigned long long *T, const uint2 *xl, uint32_t n, uint32_t hb,
                                            int lane)
{
    __syncwarp();
    uint32_t cnt = 0;
    for (uint32_t e = (uint32_t)lane; e < n; e += 32) {
        const uint2 pr = xl[e];
        const int bin = exact_bin(prm, T, m.us, m.n_total, pr.x, pr.y);
        cnt++;
        if (bin >= 0) {
            const uint32_t k = (uint32_t)bin / (uint32_t)prm.n_mu, j = (uint32_t)bin % (uint32_t)prm.n_mu;
            const uint32_t col = MU ? j + (uint32_t)dp.CO : 0u;
            red_add(hb + (k << Sh<R, LOGC>::LS) + (col << Sh<R, LOGC>::LT), 1u);
        }
    }
    __syncwarp();
    return cnt;
}

// this lane's b-points of the tile (buffer slots 32 p + lane, packed in
// pairs p = 2q, 2q + 1); slots at or past nb are padding
__device__ __forceinline__ void load_tile(const float4 *buf, uint32_t nb, int lane, float2 (&BX)[NQ], float2 (&BY)[NQ],
                                          float2 (&BZ)[NQ])
{
#pragma unroll
    for (int q = 0; q < NQ; q++) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const uint32_t s = 32u * (uint32_t)(2 * q + h) + (uint32_t)lane;
            const float4 v = s < nb ? buf[s] : make_float4(FAR, FAR, FAR, 0.0f);
            if (h) {
                BX[q].y = v.x;
                BY[q].y = v.y;
                BZ[q].y = v.z;
            } else {
                BX[q].x = v.x;
                BY[q].x = v.y;
                BZ[q].x = v.z;
            }
        }
    }
}

// Every pair of the a-chunk (na points from sorted index a0) with the first nb
// entries of the warp's buffer; CHK: the first nself entries are points of
// the a-chunk's own cell (an auto count), of whose pairs only a < b count.
// Padding slots hold far-away points whose adds land in the spare last row.
// The a-points run two at a time, the last of an odd chunk alone.  The
// pairs of one a-point or their
// uncertainty into one predicate per lane; when any lane's is set, the
// a-points' pairs are recomputed with a flag each, and each uncertain pair's
// add is taken back and the pair joins the recheck list.
template <int V, int R, int LOGC, bool CHK>
__device__ __forceinline__ void tile(const CountParams &prm, const DirectParams &dp, const Mesh &m,
                                     const unsigned long long *T, const WarpMem &wm, const Addr &ad, uint32_t nb,
                                     uint32_t nself, uint32_t na, uint32_t a0, int lane, uint32_t &n_list,
                                     unsigned long long &n_exact, unsigned long long &n_cand)
{
    constexpr bool MU = V > 0, MID = V == 2;
    float2 BX[NQ], BY[NQ], BZ[NQ];
    load_tile(wm.buf, nb, lane, BX, BY, BZ);
    // CHK: a self-cell slot counts a pair when a < b, any other real slot
    // always, a padding slot never
    uint32_t IB[NP] = {0u, 0u, 0u, 0u};
    if (CHK) {
#pragma unroll
        for (int p = 0; p < NP; p++) {
            const uint32_t s = 32u * (uint32_t)p + (uint32_t)lane;
            IB[p] = s < nself ? __float_as_uint(wm.buf[s].w) : (s < nb ? 0xFFFFFFFFu : 0u);
        }
    }
    // slot p of this lane holds a b-point (not padding): bit p
    uint32_t live = 0;
#pragma unroll
    for (int p = 0; p < NP; p++) live |= (32u * (uint32_t)p + (uint32_t)lane < nb ? 1u : 0u) << p;
    n_cand += (unsigned long long)nb * na;
    constexpr int LS = Sh<R, LOGC>::LS, LT = Sh<R, LOGC>::LT;
    const K2 k2{u64of(make_float2(dp.tiny, dp.tiny)), u64of(make_float2(MAG_S, MAG_S)), u64of(make_float2(-1.0f, -1.0f)),
                u64of(make_float2(MAG_S - 0.5f, MAG_S - 0.5f)), u64of(make_float2(MAG_T, MAG_T)),
                u64of(make_float2(dp.nmu, dp.nmu)),
                MID ? u64of(make_float2(dp.tinyl, dp.tinyl)) : 0ull,
                MID ? u64of(make_float2(-0.5f, -0.5f)) : 0ull,
                MID ? u64of(make_float2(-dp.c1, -dp.c1)) : 0ull,
                MID ? u64of(make_float2(-dp.c3, -dp.c3)) : 0ull,
                MID ? u64of(make_float2(dp.c05, dp.c05)) : 0ull};
    const uint32_t lt = (1u << lane) - 1u;
    // a-point ai had an uncertain pair in some lane: recompute its pairs with
    // one flag each (padding slots and, in the self cell, pairs a >= b never
    // count), take back each uncertain pair's add and put it on the recheck list
    auto settle = [&](uint32_t ai) {
        const ARec a = load_a<MID>(wm.arec, ai);
        const uint32_t ia = a0 + ai;
        uint32_t xs[NP];
        bool fl[NP];
#pragma unroll
        for (int q = 0; q < NQ; q++)
            pair2_flags<V, LS, LT>(u64of(BX[q]), u64of(BY[q]), u64of(BZ[q]), a, k2, dp.cs, dp.s_top, ad.Kl,
                                    xs[2 * q], xs[2 * q + 1], fl[2 * q], fl[2 * q + 1]);
        uint32_t xm = 0;
#pragma unroll
        for (int p = 0; p < NP; p++) xm |= (fl[p] && (!CHK || ia < IB[p]) ? 1u : 0u) << p;
        xm &= live;
#pragma unroll 1
        for (int p = 0; p < NP; p++) {
            const bool x = (xm >> p) & 1u;
            const unsigned mk = __ballot_sync(0xffffffffu, x);
            if (mk) {
                if (x) {
                    red_add(p == 0 ? xs[0] : (p == 1 ? xs[1] : (p == 2 ? xs[2] : xs[3])), 0xFFFFFFFFu);
                    xl_put(wm.xl, n_list + __popc(mk & lt), ia,
                           __float_as_uint(wm.buf[32u * (uint32_t)p + (uint32_t)lane].w));
                }
                n_list += __popc(mk);
                if (n_list >= XCAP - 32) {
                    n_exact += recheck<MU, R, LOGC>(prm, dp, m, T, wm.xl, n_list, ad.hb, lane);
                    n_list = 0;
                }
            }
        }
    };
    uint32_t ai = 0;
#pragma unroll 1
    for (; ai + 1 < na; ai += 2) {
        const ARec a = load_a<MID>(wm.arec, ai), a2 = load_a<MID>(wm.arec, ai + 1);
        const bool u0 = apoint<V, CHK, LS, LT>(BX, BY, BZ, a, k2, dp.cs, dp.s_top, ad.Kl, a0 + ai, IB, ad.dump);
        const bool u1 = apoint<V, CHK, LS, LT>(BX, BY, BZ, a2, k2, dp.cs, dp.s_top, ad.Kl, a0 + ai + 1, IB, ad.dump);
        if (__any_sync(0xffffffffu, u0 || u1)) {
#pragma unroll 1
            for (uint32_t j = ai; j < ai + 2; j++) settle(j);
        }
    }
    if (ai < na) {   // the last a-point of an odd chunk
        const ARec a = load_a<MID>(wm.arec, ai);
        if (__any_sync(0xffffffffu,
                       apoint<V, CHK, LS, LT>(BX, BY, BZ, a, k2, dp.cs, dp.s_top, ad.Kl, a0 + ai, IB, ad.dump)))
            settle(ai);
    }
    __syncwarp();
}

// x, y, z of sorted point i in bins relative to the corner (ox, oy, oz)
__device__ __forceinline__ float4 bpoint(const DirectParams &dp, uint32_t i, uint32_t ux, uint32_t uy, uint32_t uz,
                                         uint32_t ox, uint32_t oy, uint32_t oz)
{
    return make_float4(__fmul_rn(__int2float_rn((int)(ux - ox)), dp.inv_qds),
                       __fmul_rn(__int2float_rn((int)(uy - oy)), dp.inv_qds),
                       __fmul_rn(__int2float_rn((int)(uz - oz)), dp.inv_qds), __uint_as_float(i));
}

// The unit: a-chunk [un.a0, un.a1) of cell un.cell against the term's neighbourhood.
template <int V, int R, int LOGC>
__device__ __forceinline__ void unit(const CountParams &prm, const DirectParams &dp, const Mesh &m,
                                     const unsigned long long *T, const WarpMem &wm, const Addr &ad, const Unit &un,
                                     const Term &tm, int lane, uint32_t &n_list, unsigned long long &n_exact,
                                     unsigned long long &n_cand)
{
    const int n_c = prm.n_c;
    const int ax = un.cell % n_c, ay = (un.cell / n_c) % n_c, az = un.cell / (n_c * n_c);
    const uint32_t ox = m.orig[ax], oy = m.orig[ay], oz = m.orig[az];
    const size_t N = m.n_total;
    const uint32_t a0 = un.a0, na = un.a1 - un.a0;
    // the a-chunk in bin units relative to A's corner, as packed records
    // (-x, -x, -y, -y), then (-z, -z, m - n_mu x, ...), (-m - n_mu x, ..., 0, 0)
    // (x line of sight) or (-z, -z, x - 2 o_x, ...), (y - 2 o_y, ..., z - 2 o_z, ...)
    // (midpoint line of sight, o the observer in the same frame), and its box
    float o2x = 0.f, o2y = 0.f, o2z = 0.f;
    if (V == 2) {
        o2x = 2.0f * __fmul_rn(__ll2float_rn(prm.obs[0] - (long long)ox), dp.inv_qds);
        o2y = 2.0f * __fmul_rn(__ll2float_rn(prm.obs[1] - (long long)oy), dp.inv_qds);
        o2z = 2.0f * __fmul_rn(__ll2float_rn(prm.obs[2] - (long long)oz), dp.inv_qds);
    }
    float lx = INFINITY, ly = INFINITY, lz = INFINITY, hx = -INFINITY, hy = -INFINITY, hz = -INFINITY;
    for (uint32_t i = (uint32_t)lane; i < na; i += 32) {
        const size_t g = a0 + i;
        const float4 p = bpoint(dp, (uint32_t)g, m.us[g], m.us[N + g], m.us[2 * N + g], ox, oy, oz);
        wm.arec[3 * i] = make_float4(-p.x, -p.x, -p.y, -p.y);
        if (V == 2) {
            const float lax = __fsub_rn(p.x, o2x), lay = __fsub_rn(p.y, o2y), laz = __fsub_rn(p.z, o2z);
            wm.arec[3 * i + 1] = make_float4(-p.z, -p.z, lax, lax);
            wm.arec[3 * i + 2] = make_float4(lay, lay, laz, laz);
        } else {
            const float fxp = __fmul_rn(p.x, dp.nmu);
            const float cp = __fsub_rn(dp.m, fxp), cm = __fsub_rn(-dp.m, fxp);
            wm.arec[3 * i + 1] = make_float4(-p.z, -p.z, cp, cp);
            wm.arec[3 * i + 2] = make_float4(cm, cm, 0.f, 0.f);
        }
        lx = fminf(lx, p.x);
        ly = fminf(ly, p.y);
        lz = fminf(lz, p.z);
        hx = fmaxf(hx, p.x);
        hy = fmaxf(hy, p.y);
        hz = fmaxf(hz, p.z);
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, s));
        ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, s));
        lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, s));
        hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, s));
        hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, s));
        hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, s));
    }
    // centre and half-widths, rounded outward
    const float cxb = 0.5f * (lx + hx), cyb = 0.5f * (ly + hy), czb = 0.5f * (lz + hz);
    const float e = 1.0f / 1048576.0f;
    const float hxb = __fadd_ru(__fmul_ru(0.5f, __fsub_ru(hx, lx)), __fmul_ru(e, fabsf(cxb) + 1.0f));
    const float hyb = __fadd_ru(__fmul_ru(0.5f, __fsub_ru(hy, ly)), __fmul_ru(e, fabsf(cyb) + 1.0f));
    const float hzb = __fadd_ru(__fmul_ru(0.5f, __fsub_ru(hz, lz)), __fmul_ru(e, fabsf(czb) + 1.0f));

    // the unit's b runs, one lane per neighbour row (dz, dy), each a contiguous
    // x-run of cells; an auto count takes half of the neighbourhood and the
    // self cell separately
    const bool periodic = prm.geometry == TPCF_PERIODIC;
    const uint32_t *cs = m.cellstart + (size_t)tm.cat_b * prm.n_cells;
    uint32_t n_run = 0, total = 0, self0 = 0, self1 = 0;
    for (int r0 = 0; r0 < prm.n_rows; r0 += 32) {
        const int r = r0 + lane;
        uint32_t s0[2], s1[2];
        int nl = 0;
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
                    self0 = cs[rowkey + ax];
                    self1 = cs[rowkey + ax + 1];
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
            wm.runs[n_run + n_ex + i] = make_uint2(s0[i], total + p_ex);
            p_ex += s1[i] - s0[i];
        }
        n_run += n_all;
        total += p_all;
    }
    self0 = __reduce_max_sync(0xffffffffu, self0);
    self1 = __reduce_max_sync(0xffffffffu, self1);
    if (lane == 0) wm.runs[n_run] = make_uint2(0u, total);   // sentinel: the concatenation's end
    __syncwarp();

    const uint32_t lt = (1u << lane) - 1u;
    // The buffer fills with the self cell's points first (auto counts: pairs
    // a < b, no filter), at most a tile at a time, then with the neighbour
    // runs' points that pass the filter: four raw points per lane per pass
    // (their twelve loads in flight together), survivors appended.  A tile is
    // counted whenever TB points are there, and once more for the rest.  One
    // call site per kind of tile keeps the kernel's hot code small.
    uint32_t nbuf = 0, cself = self0, c = 0;
    int g = 0;
    for (;;) {
        uint32_t nself = 0;
        if (cself < self1) {   // the buffer is empty here: self points come first
            nself = min((uint32_t)TB, self1 - cself);
            for (uint32_t e2 = (uint32_t)lane; e2 < nself; e2 += 32) {
                const size_t gi = cself + e2;
                wm.buf[e2] = bpoint(dp, (uint32_t)gi, m.us[gi], m.us[N + gi], m.us[2 * N + gi], ox, oy, oz);
            }
            cself += nself;
            nbuf = nself;
        }
        while (nbuf < TB && c < total) {
            uint32_t idx[4];
            bool ok[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t o2 = c + 32u * (uint32_t)k + (uint32_t)lane;
                ok[k] = o2 < total;
                while (g + 1 < (int)n_run && wm.runs[g + 1].y <= o2) g++;
                idx[k] = ok[k] ? wm.runs[g].x + (o2 - wm.runs[g].y) : 0u;
            }
            uint32_t ux[4], uy[4], uz[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                ux[k] = ok[k] ? __ldg(m.us + idx[k]) : 0u;
                uy[k] = ok[k] ? __ldg(m.us + N + idx[k]) : 0u;
                uz[k] = ok[k] ? __ldg(m.us + 2 * N + idx[k]) : 0u;
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const float4 p = bpoint(dp, idx[k], ux[k], uy[k], uz[k], ox, oy, oz);
                const float qx = fmaxf(__fsub_rn(fabsf(__fsub_rn(p.x, cxb)), hxb), 0.0f);
                const float qy = fmaxf(__fsub_rn(fabsf(__fsub_rn(p.y, cyb)), hyb), 0.0f);
                const float qz = fmaxf(__fsub_rn(fabsf(__fsub_rn(p.z, czb)), hzb), 0.0f);
                const bool keep = ok[k] && __fmaf_rn(qz, qz, __fmaf_rn(qy, qy, __fmul_rn(qx, qx))) < dp.hit;
                const unsigned mk = __ballot_sync(0xffffffffu, keep);
                if (keep) wm.buf[nbuf + __popc(mk & lt)] = p;
                nbuf += __popc(mk);
            }
            c += 128;
        }
        if (nbuf == 0) break;
        const uint32_t nt = min(nbuf, (uint32_t)TB);
        __syncwarp();
        if (nself)
            tile<V, R, LOGC, true>(prm, dp, m, T, wm, ad, nt, nself, na, a0, lane, n_list, n_exact, n_cand);
        else
            tile<V, R, LOGC, false>(prm, dp, m, T, wm, ad, nt, 0u, na, a0, lane, n_list, n_exact, n_cand);
        // the leftovers (fewer than 128) move to the front
        const uint32_t left = nbuf - nt;
        if (left) {
            float4 v[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t s = 32u * (uint32_t)k + (uint32_t)lane;
                v[k] = s < left ? wm.buf[TB + s] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t s = 32u * (uint32_t)k + (uint32_t)lane;
                if (s < left) wm.buf[s] = v[k];
            }
            __syncwarp();
        }
        nbuf = left;
    }
}

// drain the table into term t's int64 histogram and clear it (whole block)
template <bool MU, int R, int LOGC>
__device__ __forceinline__ unsigned long long drain(const CountParams &prm, const DirectParams &dp,
                                                    const Term *terms, uint32_t *hist, uint32_t hwords, int t)
{
    __syncthreads();
    long long *const th = terms[t].hist;
    const int n_mu = prm.n_mu;
    unsigned long long binned = 0;
    for (int b = threadIdx.x; b < prm.nbin; b += blockDim.x) {
        const int k = b / n_mu, j = b % n_mu;
        unsigned long long sum = 0;
        // mu bin j: signed columns j and -1 - j
        const uint32_t c1 = MU ? (uint32_t)(j + dp.CO) : 0u, c2 = MU ? (uint32_t)(dp.CO - 1 - j) : 0u;
        const uint4 *w1 = (const uint4 *)(hist + (((uint32_t)k << LOGC) + c1) * (uint32_t)R);
#pragma unroll
        for (int c = 0; c < R / 4; c++) {
            const uint4 v = w1[c];
            sum += (unsigned long long)v.x + v.y + v.z + v.w;
        }
        if (MU) {
            const uint4 *w2 = (const uint4 *)(hist + (((uint32_t)k << LOGC) + c2) * (uint32_t)R);
#pragma unroll
            for (int c = 0; c < R / 4; c++) {
                const uint4 v = w2[c];
                sum += (unsigned long long)v.x + v.y + v.z + v.w;
            }
        }
        if (sum) atomicAdd((unsigned long long *)&th[b], sum);
        binned += sum;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < hwords; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    return binned;
}

template <int V, int R, int W, int LOGC>
__global__ void __launch_bounds__(W * 32, 1)
    pairdirect_kernel(const __grid_constant__ CountParams prm, const __grid_constant__ DirectParams dp, const Mesh m,
                      const Term *__restrict__ terms, const Unit *__restrict__ units,
                      const uint32_t *__restrict__ n_units_p, unsigned *__restrict__ claim,
                      unsigned long long *__restrict__ stats, int term_only, int chunk)
{
    constexpr bool MU = V > 0;
    const DOff o = d_off(prm.n_s, prm.n_rows, R, dp.C, W);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long t_start = gtimer();
    uint32_t *hist = (uint32_t *)(dsm + o.hist);
    unsigned long long *Tsh = (unsigned long long *)(dsm + o.T);
    unsigned *misc = (unsigned *)(dsm + o.misc);
    const uint32_t hwords = (uint32_t)(dp.rows * dp.C * R);
    for (uint32_t i = tid; i < hwords; i += blockDim.x) hist[i] = 0u;
    for (int i = tid; i <= prm.n_s; i += blockDim.x) Tsh[i] = prm.T[i];

    unsigned char *wr = dsm + o.warp0 + (size_t)warp * o.wstride;
    const WarpMem wm{(float4 *)(wr + o.arec), (float4 *)(wr + o.buf), (uint2 *)(wr + o.runs), (uint2 *)(wr + o.xl)};
    Addr ad;
    ad.hb = saddr(dsm) + o.hist + 4u * ((uint32_t)lane & (uint32_t)(R - 1));
    constexpr int LS = Sh<R, LOGC>::LS, LT = Sh<R, LOGC>::LT;
    if (MU)
        ad.Kl = ad.hb + ((uint32_t)dp.CO << LT) - (MAG_S_BITS << LS) - (MAG_T_BITS << LT);
    else
        ad.Kl = ad.hb - (MAG_S_BITS << LS);
    ad.dump = ad.hb + ((uint32_t)prm.n_s << LS);
    uint32_t n_list = 0;
    unsigned long long n_exact = 0, n_cand = 0, binned = 0;

    // Chunks of consecutive units are claimed by the block and worked through
    // term by term, their units claimed one at a time by the warps.  The table
    // is drained when the term changes, or before the pairs added since the
    // last drain could reach 2^31 in one counter (a unit adds at most
    // unit_pair_bound to any counter, and a chunk at most 2^30).  With
    // term_only >= 0 (one launch per term) only that term's units are claimed.
    const uint32_t n_all = *n_units_p;
    uint32_t u_lo = 0, u_hi = n_all;
    if (term_only >= 0) {
        uint32_t lo = 0, hi = n_all;   // first unit of a term >= term_only
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (units[mid].term < term_only) lo = mid + 1; else hi = mid;
        }
        u_lo = lo;
        hi = n_all;                    // first unit of a term > term_only
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (units[mid].term <= term_only) lo = mid + 1; else hi = mid;
        }
        u_hi = lo;
    }
    // Claims shrink toward the end (guided self-scheduling): a block takes
    // half of the remaining units' fair share, at most chunk units and at
    // least chunk / 32 or two per warp (fewer would leave warps idle), so the
    // last claims, which set the launch's tail, are short.  A stale read of
    // the counter only changes a claim's length; the atomic add keeps the
    // claims disjoint and covering.
    const uint32_t csize = (uint32_t)chunk, span = u_hi - u_lo;
    const uint32_t cmin = min(csize, max(csize / 32u, 2u * (uint32_t)W));
    int cur_term = -1;
    unsigned long long since = 0;
    __syncthreads();
    for (;;) {
        if (tid == 0) {
            const uint32_t cur = *(volatile unsigned *)claim;
            const uint32_t rem = cur < span ? span - cur : 0u;
            const uint32_t sz = max(cmin, min(csize, rem / (2u * gridDim.x)));
            misc[0] = u_lo + atomicAdd(claim, sz);
            misc[2] = sz;
        }
        __syncthreads();
        const uint32_t c0 = misc[0];
        if (c0 >= u_hi) break;
        const uint32_t c1 = min(u_hi, c0 + misc[2]);
        uint32_t s = c0;
        while (s < c1) {
            const int t = units[s].term;
            // the end of term t inside [s, c1)
            uint32_t lo = s, hi = c1;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (units[mid].term == t) lo = mid; else hi = mid;
            }
            const uint32_t e = hi;
            const unsigned long long seg = (unsigned long long)(e - s) * dp.unit_pair_bound;
            if (cur_term >= 0 && (t != cur_term || since + seg >= (1ull << 31))) {
                if (n_list) {   // pending rechecks belong to the table being drained
                    n_exact += recheck<MU, R, LOGC>(prm, dp, m, Tsh, wm.xl, n_list, ad.hb, lane);
                    n_list = 0;
                }
                binned += drain<MU, R, LOGC>(prm, dp, terms, hist, hwords, cur_term);
                since = 0;
            }
            cur_term = t;
            since += seg;
            if (tid == 0) misc[1] = s;
            __syncthreads();
            const Term tm = terms[t];
            for (;;) {
                uint32_t u = 0;
                if (lane == 0) u = atomicAdd(&misc[1], 1u);
                u = __shfl_sync(0xffffffffu, u, 0);
                if (u >= e) break;
                unit<V, R, LOGC>(prm, dp, m, Tsh, wm, ad, units[u], tm, lane, n_list, n_exact, n_cand);
            }
            __syncthreads();
            s = e;
        }
    }
    if (cur_term >= 0) {
        if (n_list) {
            n_exact += recheck<MU, R, LOGC>(prm, dp, m, Tsh, wm.xl, n_list, ad.hb, lane);
            n_list = 0;
        }
        binned += drain<MU, R, LOGC>(prm, dp, terms, hist, hwords, cur_term);
    }
    unsigned long long ex = n_exact, bn = binned, cd = lane == 0 ? n_cand : 0ull;
#pragma unroll
    for (int s2 = 16; s2 > 0; s2 >>= 1) {
        ex += __shfl_down_sync(0xffffffffu, ex, s2);
        bn += __shfl_down_sync(0xffffffffu, bn, s2);
        cd += __shfl_down_sync(0xffffffffu, cd, s2);
    }
    if (lane == 0) {
        atomicAdd(&stats[0], cd);
        atomicAdd(&stats[1], bn);
        atomicAdd(&stats[2], ex);
        record_warp_span(stats, t_start);
    }
}

template <int V, int R, int W, int LOGC>
void *dkernel()
{
    return (void *)pairdirect_kernel<V, R, W, LOGC>;
}

// kernel for (mode: 0 s only, 1 mu along x, 2 mu from the midpoint; copies, warps,
// column bits); nullptr when not built
void *select_direct(int V, int R, int W, int logC)
{
    if (W != DIRECT_WARPS) return nullptr;
    constexpr int DW = DIRECT_WARPS;
    if (V == 0) return R == 32 ? dkernel<0, 32, DW, 0>() : dkernel<0, 16, DW, 0>();
    if (V == 1 && logC == 5) return R == 32 ? dkernel<1, 32, DW, 5>() : dkernel<1, 16, DW, 5>();
    if (V == 1 && logC == 6) return R == 32 ? dkernel<1, 32, DW, 6>() : dkernel<1, 16, DW, 6>();
    if (V == 2 && logC == 5) return R == 32 ? dkernel<2, 32, DW, 5>() : dkernel<2, 16, DW, 5>();
    if (V == 2 && logC == 6) return R == 32 ? dkernel<2, 32, DW, 6>() : dkernel<2, 16, DW, 6>();
    return nullptr;
}

int mode_of(const DirectParams &d, bool mu) { return !mu ? 0 : (d.mid ? 2 : 1); }

}  // namespace

size_t pairdirect_smem_bytes(const CountParams &p, int R, int C, int W)
{
    return d_off(p.n_s, p.n_rows, R, C, W).end;
}

cudaError_t pairdirect_set_attrs(const DirectParams &d, int mu)
{
    void *k = select_direct(mode_of(d, mu != 0), d.R, d.W, d.logC);
    if (!k) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, d.smem);
}

int pairdirect_max_blocks_per_sm(const DirectParams &d, int mu)
{
    void *k = select_direct(mode_of(d, mu != 0), d.R, d.W, d.logC);
    int nb = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, d.W * 32, d.smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

cudaError_t launch_pairdirect(const CountParams &p, const DirectParams &d, const Mesh &m, const Term *terms,
                              const Unit *units, const uint32_t *n_units, unsigned *claim, unsigned long long *stats,
                              const PairLaunch &pl, cudaStream_t s)
{
    void *k = select_direct(mode_of(d, p.n_mu > 1), d.R, d.W, d.logC);
    if (!k) return cudaErrorInvalidValue;
    const int term_only = pl.persistent ? -1 : pl.term;
    void *args[] = {(void *)&p,      (void *)&d,     (void *)&m,     (void *)&terms,     (void *)&units,
                    (void *)&n_units, (void *)&claim, (void *)&stats, (void *)&term_only, (void *)&pl.chunk};
    return cudaLaunchKernel(k, dim3(pl.blocks), dim3(d.W * 32), args, (size_t)d.smem, s);
}

}  // namespace tpcf
