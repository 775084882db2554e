// Split-precision Gram products of the LC covariance on the 5th-generation
// tensor cores (tcgen05), Eqs. (bruteforce), (R1R2), (LCdef).
//
// The sample covariances need G_v = Y_v^T Y_v for the three centred
// correlation-function variants v (R1, R2, R1 u R2), Y_v = xi_v - mean_v of
// shape [n_mock][nbin].  Y is split into pieces that the tensor cores take
// exactly:
//   TF32X3: y = hi + lo (tf32 each), G ~ hi.hi + hi.lo + lo.hi         (3 products)
//   BF16X3: y = h + m + l (bf16 each), G ~ hh + hm + mh + hl + lh + mm  (6 products)
// A CTA (one per SM) owns one 128 x 128 output tile of one variant and a
// chunk of K-slices of 16 mocks: its operand tiles arrive by bulk copies
// (cp.async.bulk, the TMA engine, completing on mbarriers) into two stages,
// one thread issues each slice's tcgen05.mma chains into one of two FP32
// accumulator sets in tensor memory, and eight warps read each finished set
// back with tcgen05.ld and add it into a shared FP32 tile by compensated
// (Kahan) summation while the next slice multiplies; the tile becomes the
// chunk's partial Gram, which a reduction kernel sums over the chunks in
// float64, in chunk order.  The leading product (hi.hi) and the much smaller
// correction products go to two separate accumulators, so the FP32 rounding of
// an accumulator spans one slice's exact products and the corrections do not
// round against the leading sum.
//
// Operand tiles are written by the split kernel directly in the canonical
// K-major, non-swizzled layout of the tensor-core descriptors: 8-row x
// 16-byte core matrices, LBO = 128 bytes between core matrices along K and
// SBO = (32 * elem / 16) * 128 bytes between 8-row groups.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "tpcf_internal.h"

namespace tpcf {
namespace {

constexpr int TM = 128;          // rows (bins) per tile, M = N of the MMA
constexpr int KS = 16;           // mocks per K-slice
constexpr int TMEM_COLS = 4 * TM; // two accumulator sets of (leading product, corrections)
constexpr int GRAM_EPI_WARPS = 8;  // the epilogue: warp w reads TMEM lanes 32 (w mod 4).. and columns half w / 4
constexpr int GRAM_THREADS = 32 * (GRAM_EPI_WARPS + 1);   // + one warp for the loads and MMAs
static_assert(GRAM_EPI_WARPS == 8 && TM == 128, "two warpgroups split a 128-column tile (drain and store)");
constexpr long long SPIN_LIMIT = 1ll << 26;
constexpr int NSTAGE = 2;                    // K-slices in flight per CTA
constexpr int TPAD = TM + 1;                 // row stride (floats) of the shared tile

template <int PREC>
struct Split;

template <>
struct Split<TPCF_TF32X3> {
    static constexpr int ELEM = 4;                           // bytes
    static constexpr int PIECES = 2;
    static constexpr int K_MMA = 8;                          // K per tcgen05.mma (kind::tf32)
    static constexpr int N_PROD = 3;
    // products hi.hi, hi.lo, lo.hi: piece of A and of B for product q
    __host__ __device__ static constexpr int pa(int q) { return q == 2 ? 1 : 0; }
    __host__ __device__ static constexpr int pb(int q) { return q == 1 ? 1 : 0; }
    static constexpr uint32_t FMT = 2;                       // TF32 operand format
};
template <>
struct Split<TPCF_BF16X3> {
    static constexpr int ELEM = 2;
    static constexpr int PIECES = 3;
    static constexpr int K_MMA = 16;                         // kind::f16
    static constexpr int N_PROD = 6;
    // products hh, hm, mh, hl, lh, mm
    __host__ __device__ static constexpr int pa(int q) { return q == 2 ? 1 : (q == 4 ? 2 : (q == 5 ? 1 : 0)); }
    __host__ __device__ static constexpr int pb(int q) { return q == 1 ? 1 : (q == 3 ? 2 : (q == 5 ? 1 : 0)); }
    static constexpr uint32_t FMT = 1;                       // BF16 operand format
};

template <int PREC>
__host__ __device__ constexpr int tile_bytes() { return TM * KS * Split<PREC>::ELEM; }

template <int PREC>
__host__ __device__ constexpr int sbo_bytes() { return (KS * Split<PREC>::ELEM / 16) * 128; }

// byte offset of element (row r, k) inside a K-major non-swizzled tile
template <int PREC>
__device__ __forceinline__ uint32_t tile_offset(int r, int k)
{
    constexpr int per = 16 / Split<PREC>::ELEM;              // elements per core-matrix row
    return (uint32_t)((r >> 3) * sbo_bytes<PREC>() + (k / per) * 128 + (r & 7) * 16 + (k % per) * Split<PREC>::ELEM);
}

__device__ __forceinline__ uint32_t tf32_rna(float x)
{
    uint32_t y;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
    return y;
}

// centred residuals, split into pieces, written as operand tiles
// tiles[v][piece][rb][ks]
template <int PREC>
__global__ void split_kernel(const double *__restrict__ x0, const double *__restrict__ x1,
                             const double *__restrict__ x2, const double *__restrict__ mean, int n_mock, int nbin,
                             int n_rb, int n_ks, unsigned char *__restrict__ tiles)
{
    const int v = blockIdx.z;
    const double *x = v == 0 ? x0 : (v == 1 ? x1 : x2);
    const int rb = blockIdx.y, ks = blockIdx.x;
    constexpr int TB = tile_bytes<PREC>();
    constexpr int NP = Split<PREC>::PIECES;
    for (int e = threadIdx.x; e < TM * KS; e += blockDim.x) {
        const int r = e % TM, k = e / TM;
        const int i = rb * TM + r, m = ks * KS + k;
        const double y = (i < nbin && m < n_mock) ? x[(size_t)m * nbin + i] - mean[(size_t)v * nbin + i] : 0.0;
        const uint32_t off = tile_offset<PREC>(r, k);
        if (PREC == TPCF_TF32X3) {
            const uint32_t hi = tf32_rna((float)y);
            const uint32_t lo = tf32_rna((float)(y - (double)__uint_as_float(hi)));
            unsigned char *t0 = tiles + ((((size_t)v * NP + 0) * n_rb + rb) * n_ks + ks) * TB;
            unsigned char *t1 = tiles + ((((size_t)v * NP + 1) * n_rb + rb) * n_ks + ks) * TB;
            *(uint32_t *)(t0 + off) = hi;
            *(uint32_t *)(t1 + off) = lo;
        } else {
            const __nv_bfloat16 h = __double2bfloat16(y);
            const double r1 = y - (double)__bfloat162float(h);
            const __nv_bfloat16 mm = __double2bfloat16(r1);
            const double r2 = r1 - (double)__bfloat162float(mm);
            const __nv_bfloat16 l = __double2bfloat16(r2);
            unsigned char *t0 = tiles + ((((size_t)v * NP + 0) * n_rb + rb) * n_ks + ks) * TB;
            unsigned char *t1 = tiles + ((((size_t)v * NP + 1) * n_rb + rb) * n_ks + ks) * TB;
            unsigned char *t2 = tiles + ((((size_t)v * NP + 2) * n_rb + rb) * n_ks + ks) * TB;
            *(__nv_bfloat16 *)(t0 + off) = h;
            *(__nv_bfloat16 *)(t1 + off) = mm;
            *(__nv_bfloat16 *)(t2 + off) = l;
        }
    }
}

// ---- inline PTX: mbarrier, bulk copy, tcgen05 ----

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: false if the barrier did not complete within the limit
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit)
{
    for (long long i = 0; i < limit; i++) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 64) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// non-swizzled K-major shared-memory matrix descriptor
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version for tcgen05
    return d;                 // base offset 0, no swizzle
}

template <int PREC>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    if (PREC == TPCF_TF32X3) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// instruction descriptor: FP32 accumulate, K-major A and B, M = N = 128
template <int PREC>
__host__ __device__ constexpr uint32_t instr_desc()
{
    return (1u << 4)                          // D format: F32
           | (Split<PREC>::FMT << 7)          // A format
           | (Split<PREC>::FMT << 10)         // B format
           | ((uint32_t)(TM >> 3) << 17)      // N / 8
           | ((uint32_t)(TM >> 4) << 24);     // M / 16
}

template <int PREC>
__host__ __device__ constexpr int stage_bytes() { return 2 * Split<PREC>::PIECES * tile_bytes<PREC>(); }

// shared memory: NSTAGE stages | FP32 tile sums and compensations [2][TM][TPAD] | full[NSTAGE], empty[NSTAGE],
// accf[2], accfree[2], done barriers | TMEM slot | flags
template <int PREC>
constexpr int gram_smem_bytes() { return NSTAGE * stage_bytes<PREC>() + 8 * TM * TPAD + 8 * (2 * NSTAGE + 5) + 16; }

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// One CTA (one per SM): output tile (bi, bj) of variant v over the K-slices
// [k0, k0 + n) of chunk kc.  Warp 4 keeps NSTAGE slices of operand tiles in
// flight (bulk copies completing on full[stage]) and issues each slice's MMA
// chain into accumulator set i % 2 of tensor memory (columns 256 (i % 2) +
// [0, 128): leading product, + [128, 256): corrections), once the epilogue has
// drained that set's previous slice (accfree).  Warps 0-3 (TMEM lanes = tile
// rows) read each finished set (accf) and add its two accumulators into a
// shared [column][row] tile by compensated (Kahan) FP32 summation (the FP64
// pipe is too slow for this on the SMs), so the tile holds the chunk's sum to
// about one FP32 rounding while the tensor cores work on slice i + 1.  At the end the
// tile is written to P[kc][v] (both triangles) with stores of 32 consecutive
// doubles per warp.
//
// Every wait is bounded.  The epilogue's waits for the products give up after
// done_limit polls (a context option); skip_mma (tests only) makes CTA
// (0, 0, 0) wait for its first loads and then issue no MMA and no commit, so
// that this wait runs out with no copy or MMA in flight.
template <int PREC>
__global__ void __launch_bounds__(GRAM_THREADS, 1) gram_tc_kernel(const unsigned char *__restrict__ tiles, int nbin,
                                                                 int n_rb, int n_ks, int spc, double *__restrict__ P,
                                                                 int *__restrict__ status, long long done_limit,
                                                                 int skip_mma)
{
    constexpr int TB = tile_bytes<PREC>();
    constexpr int NP = Split<PREC>::PIECES;
    constexpr int SB = stage_bytes<PREC>();
    extern __shared__ __align__(128) unsigned char smem[];
    float *tsum = (float *)(smem + NSTAGE * SB);              // [TM columns][TPAD]
    float *tcmp = tsum + TM * TPAD;                           // Kahan compensations, same layout
    uint64_t *full = (uint64_t *)(tcmp + TM * TPAD);
    uint64_t *empty = full + NSTAGE;
    uint64_t *accf = empty + NSTAGE;
    uint64_t *accfree = accf + 2;
    uint64_t *done = accfree + 2;
    uint32_t *slot = (uint32_t *)(done + 1);
    int *flag = (int *)(slot + 1);   // [0]: a done commit was issued or skipped on purpose, [1]: all slices multiplied

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // blockIdx.x enumerates the upper-triangle tile pairs (bi <= bj) row by row
    int bi = 0, rest = (int)blockIdx.x;
    while (rest >= n_rb - bi) {
        rest -= n_rb - bi;
        bi++;
    }
    const int bj = bi + rest;
    const int v = blockIdx.y, kc = blockIdx.z;
    const int k0 = kc * spc, n = min(n_ks, k0 + spc) - k0;   // n >= 1 by the host's chunking
    const bool skip = skip_mma && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;

    if (warp == 0) tmem_alloc(slot, TMEM_COLS);
    if (tid == 0) {
        for (int i = 0; i < NSTAGE; i++) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int k = 0; k < 2; k++) {
            mbar_init(&accf[k], 1);
            mbar_init(&accfree[k], GRAM_EPI_WARPS);
        }
        mbar_init(done, 1);
        mbar_fence_init();
        flag[0] = 0;
        flag[1] = 0;
    }
    for (int e = tid; e < 2 * TM * TPAD; e += blockDim.x) tsum[e] = 0.0f;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;

    if (warp == GRAM_EPI_WARPS) {
        if (lane == 0) {
            auto issue = [&](int i) {   // the operand tiles of slice k0 + i into stage i % NSTAGE
                unsigned char *sa = smem + (i % NSTAGE) * SB, *sb = sa + NP * TB;
                mbar_expect_tx(&full[i % NSTAGE], (uint32_t)SB);
                for (int p = 0; p < NP; p++) {
                    const size_t base = ((size_t)v * NP + p) * n_rb;
                    bulk_g2s(sa + p * TB, tiles + ((base + bi) * n_ks + k0 + i) * TB, TB, &full[i % NSTAGE]);
                    bulk_g2s(sb + p * TB, tiles + ((base + bj) * n_ks + k0 + i) * TB, TB, &full[i % NSTAGE]);
                }
            };
            int issued = 0, waited = 0, mma_slices = 0;
            bool ok = true;
            for (; issued < min(NSTAGE, n); issued++) issue(issued);
            for (int i = 0; i < n; i++) {
                ok = mbar_wait(&full[i % NSTAGE], (uint32_t)(i / NSTAGE) & 1u, SPIN_LIMIT);
                if (!ok) break;
                waited = i + 1;
                if (skip) {
                    if (waited == issued) break;   // every copy in flight has landed
                    continue;
                }
                // accumulator set i % 2 is free once the epilogue has drained slice i - 2
                if (i >= 2) {
                    ok = mbar_wait(&accfree[i % 2], (uint32_t)((i - 2) / 2) & 1u, SPIN_LIMIT);
                    if (!ok) break;
                }
                tc_fence_after();
                constexpr uint32_t idesc = instr_desc<PREC>();
                constexpr int steps = KS / Split<PREC>::K_MMA;
                const uint32_t sa = smem_addr(smem + (i % NSTAGE) * SB), sb = sa + NP * TB;
                const uint32_t set = tmem + (uint32_t)((i % 2) * 2 * TM);
#pragma unroll
                for (int q = 0; q < Split<PREC>::N_PROD; q++) {
                    const uint32_t a0 = sa + Split<PREC>::pa(q) * TB;
                    const uint32_t b0 = sb + Split<PREC>::pb(q) * TB;
#pragma unroll
                    for (int st = 0; st < steps; st++) {
                        // each MMA step covers two core matrices along K (2 x 128 bytes); product 0
                        // accumulates in the set's columns [0, 128), the others in [128, 256); the first
                        // step of each accumulator overwrites it
                        const uint64_t da = smem_desc(a0 + st * 256, 128, sbo_bytes<PREC>());
                        const uint64_t db = smem_desc(b0 + st * 256, 128, sbo_bytes<PREC>());
                        const uint32_t d = set + (q == 0 ? 0u : (uint32_t)TM);
                        const bool init = st == 0 && (q == 0 || q == 1);
                        mma<PREC>(d, da, db, idesc, init ? 0u : 1u);
                    }
                }
                mma_commit(&empty[i % NSTAGE]);
                mma_commit(&accf[i % 2]);
                mma_slices = i + 1;
                if (issued < n) {   // refill this stage once its products have read it
                    ok = mbar_wait(&empty[i % NSTAGE], (uint32_t)(i / NSTAGE) & 1u, SPIN_LIMIT);
                    if (!ok) break;
                    issue(issued++);
                }
            }
            if (mma_slices > 0) mma_commit(done);
            // copies still in flight after a wait gave up get one more bounded wait each
            for (int i = waited; i < issued; i++)
                if (!mbar_wait(&full[i % NSTAGE], (uint32_t)(i / NSTAGE) & 1u, SPIN_LIMIT)) break;
            flag[0] = (mma_slices > 0 || skip) ? 1 : 0;
            flag[1] = (ok && mma_slices == n) ? 1 : 0;
            if (!ok) atomicOr(status, STATUS_TIMEOUT);
        }
    } else {
        // epilogue: row = this thread's TMEM lane; the two warpgroups take the
        // columns [0, TM / 2) and [TM / 2, TM) of both accumulators
        const int wr = warp & 3, c_lo = (warp >> 2) * (TM / 2);
        const int r = wr * 32 + lane;
        bool fine = true;
        for (int i = 0; i < n && fine; i++) {
            fine = mbar_wait(&accf[i % 2], (uint32_t)(i / 2) & 1u, done_limit);
            if (!fine) {
                fine = mbar_wait(&accf[i % 2], (uint32_t)(i / 2) & 1u, done_limit);
                if (!fine) break;
            }
            tc_fence_after();
            const uint32_t set = tmem + ((uint32_t)(wr * 32) << 16) + (uint32_t)((i % 2) * 2 * TM);
#pragma unroll 1
            for (int c0 = c_lo; c0 < c_lo + TM / 2; c0 += 32) {
                uint32_t lo[32], hi[32];
                tmem_ld32(set + (uint32_t)c0, lo);
                tmem_ld32(set + (uint32_t)(TM + c0), hi);
#pragma unroll
                for (int j = 0; j < 32; j++) {
                    const int e = (c0 + j) * TPAD + r;
                    float sum = tsum[e], cmp = tcmp[e];
                    // two compensated additions (the leading product, then the corrections)
                    float y = __fsub_rn(__uint_as_float(lo[j]), cmp);
                    float t = __fadd_rn(sum, y);
                    cmp = __fsub_rn(__fsub_rn(t, sum), y);
                    sum = t;
                    y = __fsub_rn(__uint_as_float(hi[j]), cmp);
                    t = __fadd_rn(sum, y);
                    cmp = __fsub_rn(__fsub_rn(t, sum), y);
                    tsum[e] = t;
                    tcmp[e] = cmp;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accfree[i % 2]);
        }
        if (!fine && lane == 0) atomicOr(status, STATUS_TIMEOUT);
    }
    __syncthreads();
    // every product has completed before tensor memory is released (bounded)
    bool good = flag[1] != 0;
    if (flag[0]) {
        bool fin = mbar_wait(done, 0, done_limit);
        if (!fin) fin = mbar_wait(done, 0, done_limit);
        good = good && fin;
    }
    if (!good && tid == 0) atomicOr(status, STATUS_TIMEOUT);
    if (good && warp < GRAM_EPI_WARPS) {
        double *g = P + ((size_t)kc * gridDim.y + v) * nbin * nbin;
        // the epilogue warps' 256 threads: t in [0, TM) and a half h of the other index
        const int t = (warp * 32 + lane) & (TM - 1), h0 = ((warp * 32 + lane) / TM) * (TM / 2);
        // the block itself: thread t takes column t (consecutive threads, consecutive doubles)
        const int col = bj * TM + t;
        if (col < nbin) {
            for (int rr = h0; rr < h0 + TM / 2; rr++) {
                const int row = bi * TM + rr;
                if (row >= nbin) break;
                g[(size_t)row * nbin + col] = (double)tsum[t * TPAD + rr] - (double)tcmp[t * TPAD + rr];
            }
        }
        // the transposed block of an off-diagonal pair: thread t takes row t
        const int row = bi * TM + t;
        if (bi != bj && row < nbin) {
            for (int c = h0; c < h0 + TM / 2; c++) {
                const int cc = bj * TM + c;
                if (cc >= nbin) break;
                g[(size_t)cc * nbin + row] = (double)tsum[c * TPAD + t] - (double)tcmp[c * TPAD + t];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// G[v][i][j] = sum over the chunks kc of P[kc][v][i][j], in chunk order (deterministic)
__global__ void reduce_partials_kernel(const double *__restrict__ P, int n_kc, size_t per, double *__restrict__ G)
{
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < per; e += (size_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < n_kc; k++) acc += P[(size_t)k * per + e];
        G[e] = acc;
    }
}

// K-chunking of the Gram grid: n_kc chunks of spc slices each, as many as fit
// in one wave (one CTA per SM: 512 TMEM columns and ~200 KB of shared memory
// each; one CTA more than the SMs would run a second wave of one CTA and
// double the kernel's time); the FP32 rounding spans one 16-mock slice
// whatever the chunk length.  The partials then take at most about n_sm x 2 TM^2 x 8 bytes
// (n_kc x n_var x nbin^2 doubles with n_kc ~ n_sm / (n_var x tile pairs)).
struct Chunking {
    int spc, n_kc;
};

Chunking chunking(int n_mock, int nbin, int n_var, int n_sm)
{
    const int n_rb = (nbin + TM - 1) / TM, n_ks = (n_mock + KS - 1) / KS;
    const long long np = (long long)n_rb * (n_rb + 1) / 2;
    long long want = std::max<long long>(1, (long long)std::max(1, n_sm) / (np * n_var));
    want = std::min<long long>(want, n_ks);
    const int spc = (int)((n_ks + want - 1) / want);
    return Chunking{spc, (n_ks + spc - 1) / spc};
}

template <int PREC>
size_t tiles_bytes(int n_mock, int nbin, int n_var)
{
    const size_t n_rb = (nbin + TM - 1) / TM, n_ks = (n_mock + KS - 1) / KS;
    return (size_t)n_var * Split<PREC>::PIECES * n_rb * n_ks * tile_bytes<PREC>();
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

template <int PREC>
size_t work_bytes_of(int n_mock, int nbin, int n_var, int n_sm)
{
    const Chunking c = chunking(n_mock, nbin, n_var, n_sm);
    const size_t g = (size_t)n_var * nbin * nbin * 8;
    return al256(tiles_bytes<PREC>(n_mock, nbin, n_var)) + al256(g) + al256((size_t)c.n_kc * g) +
           al256((size_t)n_var * nbin * 8);
}

// n_var = 3: the LC covariance of (x0, x1, x2); n_var = 1: the sample covariance of x0 into C_lc
template <int PREC>
cudaError_t run(const double *x0, const double *x1, const double *x2, int n_var, int n_mock, int nbin, void *work,
                size_t work_bytes, int M_a, double M, double *C_lc, double *Ca, double *Cb, double *A, double *B,
                int *status, const GramOpts &opt, cudaStream_t s)
{
    const int n_rb = (nbin + TM - 1) / TM, n_ks = (n_mock + KS - 1) / KS;
    if (n_rb > 90) return cudaErrorInvalidValue;
    const Chunking ch = chunking(n_mock, nbin, n_var, opt.n_sm);
    if (ch.n_kc > 65535) return cudaErrorInvalidValue;
    unsigned char *w = (unsigned char *)work;
    unsigned char *tiles = w;
    const size_t g = (size_t)n_var * nbin * nbin;
    size_t o = al256(tiles_bytes<PREC>(n_mock, nbin, n_var));
    double *G = (double *)(w + o);
    o += al256(g * 8);
    double *P = (double *)(w + o);
    o += al256((size_t)ch.n_kc * g * 8);
    double *mean = (double *)(w + o);
    o += al256((size_t)n_var * nbin * 8);
    if (o > work_bytes) return cudaErrorInvalidValue;
    cudaError_t e = launch_means(x0, x1, x2, n_var, n_mock, nbin, mean, s);
    if (e != cudaSuccess) return e;
    split_kernel<PREC><<<dim3(n_ks, n_rb, n_var), 256, 0, s>>>(x0, x1, x2, mean, n_mock, nbin, n_rb, n_ks, tiles);
    const int np = n_rb * (n_rb + 1) / 2;   // upper-triangle tile pairs
    const int smem = gram_smem_bytes<PREC>();
    e = cudaFuncSetAttribute(gram_tc_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    gram_tc_kernel<PREC><<<dim3(np, n_var, ch.n_kc), GRAM_THREADS, smem, s>>>(
        tiles, nbin, n_rb, n_ks, ch.spc, P, status, opt.wait_limit > 0 ? opt.wait_limit : SPIN_LIMIT,
        opt.test_skip_mma);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int rb = (int)std::min<size_t>((g + 255) / 256, 4096);
    reduce_partials_kernel<<<rb, 256, 0, s>>>(P, ch.n_kc, g, G);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (n_var == 1) return launch_scale(G, nbin, n_mock, C_lc, s);
    return launch_combine(G, nbin, n_mock, M_a, M, C_lc, Ca, Cb, A, B, s);
}

}  // namespace

size_t lc_split_work_bytes(int n_mock, int nbin, int precision, int n_sm, int n_var)
{
    return precision == TPCF_BF16X3 ? work_bytes_of<TPCF_BF16X3>(n_mock, nbin, n_var, n_sm)
                                    : work_bytes_of<TPCF_TF32X3>(n_mock, nbin, n_var, n_sm);
}

cudaError_t launch_lc_split(const double *xi_a1, const double *xi_a2, const double *xi_b, int n_mock, int nbin,
                            int precision, void *work, size_t work_bytes, int M_a, double M, double *C_lc,
                            double *Ca, double *Cb, double *A, double *B, int *status, const GramOpts &opt,
                            cudaStream_t s)
{
    if (precision == TPCF_TF32X3)
        return run<TPCF_TF32X3>(xi_a1, xi_a2, xi_b, 3, n_mock, nbin, work, work_bytes, M_a, M, C_lc, Ca, Cb, A, B,
                                status, opt, s);
    if (precision == TPCF_BF16X3)
        return run<TPCF_BF16X3>(xi_a1, xi_a2, xi_b, 3, n_mock, nbin, work, work_bytes, M_a, M, C_lc, Ca, Cb, A, B,
                                status, opt, s);
    return cudaErrorNotSupported;
}

cudaError_t launch_cov_split(const double *xi, int n_mock, int nbin, int precision, void *work, size_t work_bytes,
                             double *C, int *status, const GramOpts &opt, cudaStream_t s)
{
    if (precision == TPCF_TF32X3)
        return run<TPCF_TF32X3>(xi, xi, xi, 1, n_mock, nbin, work, work_bytes, 1, 2.0, C, nullptr, nullptr,
                                nullptr, nullptr, status, opt, s);
    if (precision == TPCF_BF16X3)
        return run<TPCF_BF16X3>(xi, xi, xi, 1, n_mock, nbin, work, work_bytes, 1, 2.0, C, nullptr, nullptr,
                                nullptr, nullptr, status, opt, s);
    return cudaErrorNotSupported;
}

}  // namespace tpcf
