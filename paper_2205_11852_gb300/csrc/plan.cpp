// Host-side planning of a pair count: exact integer bin thresholds, the FP32
// error bands around them, the s-bin lookup table over FP32 bit patterns,
// and the chaining-mesh neighbourhood.
//
// Binning definition (Sect. 4.3 bins; exact on integer grid coordinates):
// a pair with squared grid separation D2 lies in s-bin k iff
// T_k <= D2 < T_{k+1}, T_k = ceil(e_k^2 q^2), q = 2^32/L (periodic) or
// 2^30/L (open).  T_k is computed here in exact integer arithmetic.
#include "plan.h"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <vector>

namespace tpcf {

namespace {

// Minimal unsigned big integer (little-endian 32-bit limbs), enough for
// ceil(a * 2^s / b) with a, b < 2^106 and a quotient below 2^64.
struct Big {
    static constexpr int N = 14;
    uint32_t d[N];
    Big() { std::memset(d, 0, sizeof(d)); }
    explicit Big(unsigned long long v) : Big() { d[0] = (uint32_t)v; d[1] = (uint32_t)(v >> 32); }
    static Big mul(unsigned long long a, unsigned long long b)
    {
        Big r;
        const uint32_t x[2] = {(uint32_t)a, (uint32_t)(a >> 32)}, y[2] = {(uint32_t)b, (uint32_t)(b >> 32)};
        for (int i = 0; i < 2; i++) {
            unsigned long long carry = 0;
            for (int j = 0; j < 2; j++) {
                unsigned long long t = (unsigned long long)x[i] * y[j] + r.d[i + j] + carry;
                r.d[i + j] = (uint32_t)t;
                carry = t >> 32;
            }
            int k = i + 2;
            while (carry) {
                unsigned long long t = (unsigned long long)r.d[k] + carry;
                r.d[k++] = (uint32_t)t;
                carry = t >> 32;
            }
        }
        return r;
    }
    Big shl(int s) const
    {
        Big r;
        const int w = s / 32, b = s % 32;
        for (int i = N - 1; i >= 0; i--) {
            unsigned long long v = 0;
            if (i - w >= 0) v = (unsigned long long)d[i - w] << b;
            if (b && i - w - 1 >= 0) v |= (unsigned long long)d[i - w - 1] >> (32 - b);
            r.d[i] = (uint32_t)v;
        }
        return r;
    }
    int cmp(const Big &o) const
    {
        for (int i = N - 1; i >= 0; i--)
            if (d[i] != o.d[i]) return d[i] < o.d[i] ? -1 : 1;
        return 0;
    }
    void sub(const Big &o)
    {
        long long borrow = 0;
        for (int i = 0; i < N; i++) {
            long long t = (long long)d[i] - o.d[i] - borrow;
            borrow = t < 0;
            d[i] = (uint32_t)(t + (borrow << 32));
        }
    }
    bool zero() const
    {
        for (int i = 0; i < N; i++)
            if (d[i]) return false;
        return true;
    }
};

// v = m * 2^e with m a 53-bit integer (v > 0, finite)
void decompose(double v, unsigned long long &m, int &e)
{
    int ex;
    double fr = std::frexp(v, &ex);           // v = fr * 2^ex, fr in [0.5, 1)
    m = (unsigned long long)std::ldexp(fr, 53);
    e = ex - 53;
}

double ulp_f32(double x)
{
    if (x <= 0) return std::ldexp(1.0, -149);
    int ex;
    std::frexp(x, &ex);                        // x in [2^(ex-1), 2^ex)
    return std::ldexp(1.0, ex - 1 - 23);
}

float down_f(double x)
{
    float f = (float)x;
    if ((double)f > x) f = std::nextafter(f, -INFINITY);
    return f;
}

float up_f(double x)
{
    float f = (float)x;
    if ((double)f < x) f = std::nextafter(f, INFINITY);
    return f;
}

}  // namespace

// T = ceil(e^2 * 2^(2 bits) / L^2); returns false if T >= 2^63.
bool exact_threshold(double e, double L, int bits, unsigned long long &T)
{
    if (e == 0.0) { T = 0; return true; }
    const double est = (e / L) * (e / L) * std::ldexp(1.0, 2 * bits);
    if (!(est < 4.0e18)) return false;
    if (est < 0.25) { T = 1; return true; }
    unsigned long long me, mL;
    int ee, eL;
    decompose(e, me, ee);
    decompose(L, mL, eL);
    const int s = 2 * ee + 2 * bits - 2 * eL;  // value = me^2 2^s / mL^2
    Big num = Big::mul(me, me), den = Big::mul(mL, mL);
    if (s >= 0) num = num.shl(s); else den = den.shl(-s);
    // long division; the quotient is below 2^64
    unsigned long long q = 0;
    for (int i = 63; i >= 0; i--) {
        Big t = den.shl(i);
        if (t.cmp(num) <= 0) {
            num.sub(t);
            q |= 1ull << i;
        }
    }
    T = q + (num.zero() ? 0 : 1);
    return T < (1ull << 63);
}

int build_plan(const tpcf_binning &b, int subdiv, unsigned long long max_cells, Plan &pl, std::string &err)
{
    CountParams &p = pl.prm;
    std::memset(&p, 0, sizeof(p));
    p.geometry = b.geometry;
    p.los = b.los;
    p.n_s = b.n_s;
    p.n_mu = b.n_mu;
    p.nbin = b.n_s * b.n_mu;
    p.bits = (b.geometry == TPCF_PERIODIC) ? 32 : 30;
    const double L = b.box_L;
    const double s_max = b.s_edges[b.n_s];

    // exact thresholds
    for (int k = 0; k <= b.n_s; k++) {
        if (!exact_threshold(b.s_edges[k], L, p.bits, p.T[k])) {
            err = "separation range exceeds the 64-bit squared-distance range";
            return TPCF_ERR_RANGE;
        }
    }
    const unsigned long long Tmax = p.T[b.n_s];
    if (Tmax == 0) { err = "s_max must be positive"; return TPCF_ERR_ARG; }

    // mesh: the largest n_c (cells per axis) whose cells still reach no
    // further than `subdiv` neighbours, capped by max_cells
    const unsigned long long full = 1ull << p.bits;
    const double Tn = (double)Tmax * (1.0 + 1e-12) + 1.0;
    // reach: largest offset o whose cells can hold a pair closer than s_max,
    // i.e. ((o - 1) Wmin + 1)^2 < T_ns
    auto reach = [&](unsigned long long Wmin) {
        int K = 0;
        while (K <= 8) {
            const double m = (double)K * (double)Wmin + 1.0;
            if (m * m >= Tn) break;
            K++;
        }
        return K;
    };
    int n_c = (int)std::floor(subdiv * L / s_max);
    n_c = std::max(1, std::min(n_c, MAX_NC));
    while (n_c > 1 && (unsigned long long)n_c * n_c * n_c > max_cells) n_c--;
    while (n_c > 1 && reach(full / (unsigned long long)n_c) > subdiv) n_c--;
    int K = reach(full / (unsigned long long)n_c);
    if (b.geometry == TPCF_PERIODIC) {
        // distinct offsets in [-K, K] must map to distinct cells
        while (n_c < 2 * K + 1 && n_c < MAX_NC) {
            n_c++;
            K = reach(full / (unsigned long long)n_c);
        }
        if (n_c < 2 * K + 1) {
            err = "periodic box too small for the separation range (need s_max <= L/3)";
            return TPCF_ERR_RANGE;
        }
    }
    if (K > 4) {
        err = "mesh reach above 4 cells";
        return TPCF_ERR_RANGE;
    }
    const unsigned long long Wmin = full / (unsigned long long)n_c;
    const unsigned long long Wmax = (full + n_c - 1) / (unsigned long long)n_c;
    p.n_c = n_c;
    p.n_cells = n_c * n_c * n_c;
    pl.K = K;
    pl.subdiv = subdiv;
    pl.orig.resize(n_c + 1);
    for (int c = 0; c <= n_c; c++) {
        const unsigned long long o = ((unsigned long long)c * full + n_c - 1) / n_c;
        pl.orig[c] = (uint32_t)o;  // 2^32 wraps to 0; only differences are used
    }

    // neighbour rows (dz, dy) with the x reach of each
    auto m1 = [&](int o) -> double {
        if (o == 0) return 0.0;
        const double m = (double)(std::abs(o) - 1) * (double)Wmin + 1.0;
        return m * m;
    };
    p.n_rows = 0;
    for (int dz = -K; dz <= K; dz++)
        for (int dy = -K; dy <= K; dy++) {
            const double base = m1(dz) + m1(dy);
            if (base >= Tn) continue;
            int kx = 0;
            while (kx + 1 <= K && base + m1(kx + 1) < Tn) kx++;
            p.row_dz[p.n_rows] = (int8_t)dz;
            p.row_dy[p.n_rows] = (int8_t)dy;
            p.row_kx[p.n_rows] = (int8_t)kx;
            p.n_rows++;
        }

    // FP32 error model.  Coordinates are cell-relative floats; a b-point is
    // shifted into A's frame by the integer corner difference.  Every value in
    // the chain stays below (K+2) * Wmax in magnitude, and each of the five
    // roundings costs at most half an ulp there.
    const double E = 3.0 * ulp_f32((double)(K + 2) * (double)Wmax);
    const double u = std::ldexp(1.0, -24);
    const double g3 = 3.0 * u / (1.0 - 3.0 * u);
    auto err_at = [&](double T) -> double {
        const double r = std::sqrt(T);
        const double a = 2.0 * std::sqrt(3.0) * E * r + 3.0 * E * E;
        return 2.0 * (a + g3 * (T + a)) + 4.0;   // x2 safety, +4 grid units^2
    };
    for (int k = 0; k <= b.n_s; k++) {
        const double T = (double)p.T[k];
        if (p.T[k] == 0) {
            p.lo[k] = 0.0f;
            p.hi[k] = 0.0f;
        } else {
            const double e = err_at(T);
            p.lo[k] = down_f(T - e);
            p.hi[k] = up_f(T + e);
        }
    }
    p.lo[b.n_s + 1] = INFINITY;
    p.hi[b.n_s + 1] = INFINITY;
    p.hit_max = p.hi[b.n_s];
    pl.E_delta = E;

    // Dot-product candidate test  a.b' - |a|^2/2 >= (|b'|^2 - H)/2 - margin:
    // the margin covers the roundings of both sides (|a| <= sqrt3 W,
    // |b'| <= sqrt3 (K+1) W) and the 3u relative error of the direct d2.
    {
        const double W2 = (double)Wmax * (double)Wmax;
        const double H = (double)p.hit_max;
        const double k1 = (double)(K + 1);
        p.dot_margin = up_f(2.0 * u * ((6.0 + 9.0 * k1 + 12.0 * k1 * k1) * W2 + 2.6 * H));
    }

    // mu band: |t - t*| <= beta with t = n_mu |mu| computed in FP32
    p.inv_nmu2 = 1.0f / (float)(b.n_mu * b.n_mu);
    if (b.los == TPCF_LOS_X) {
        // beta = mu_c1 * r + mu_c2, r = n_mu / sqrt(d2)
        p.mu_c1 = (float)(1.1 * (1.0 + std::sqrt(3.0)) * E);
        // the kernel bounds t* by fma(|dx|, r, -/+beta), i.e. around the exact
        // product |dx| r rather than its rounding: one more ulp of n_mu
        p.mu_c2 = (float)(b.n_mu * (std::ldexp(1.0, -19) + std::ldexp(1.0, -23)));
    } else {
        // observer in open grid units; l = u_a + u_b - 2 u_obs
        for (int c = 0; c < 3; c++)
            p.obs[c] = (long long)std::floor(((b.observer[c] - b.origin[c]) / L) * std::ldexp(1.0, 30));
        double gmax = 0.0;
        for (int c = 0; c < 3; c++)
            gmax = std::max(gmax, 2.0 * std::max(std::fabs((double)p.obs[c]),
                                                 std::fabs(std::ldexp(1.0, 30) - (double)p.obs[c])));
        const double lmax = gmax + 2.0 * (K + 2) * (double)Wmax;
        const double El = 0.5 * ulp_f32(gmax) + 2.0 * E + 2.0 * ulp_f32(lmax);
        // beta = mu_c1 / sqrt(d2) + mu_c3 / |l| + mu_c2
        p.mu_c1 = (float)(b.n_mu * 2.2 * std::sqrt(3.0) * E);
        p.mu_c2 = (float)(b.n_mu * std::ldexp(1.0, -18));
        p.mu_c3 = (float)(b.n_mu * 2.2 * std::sqrt(3.0) * El);
        p.mu_c1r = up_f((double)p.mu_c1 / b.n_mu);
    }

    // Linear bins starting at 0 (e_k = k e_1 exactly): the s bin is
    // floor(u*), u* = sqrt(D2) / (q e_1), and |u - u*| <= s_c0 + s_c1 u for the
    // FP32 estimate u (d2 error, 2-ulp rsqrt, three roundings).
    {
        bool lin = b.s_edges[0] == 0.0 && b.n_s >= 1;
        const double e1 = b.s_edges[1];
        for (int k = 1; lin && k <= b.n_s; k++) lin = std::fma((double)k, e1, -b.s_edges[k]) == 0.0;
        const double q = std::ldexp(1.0, p.bits) / L;
        const double qds = q * e1;
        p.linear = lin ? 1 : 0;
        p.s_scale = (float)(1.0 / ((double)b.n_mu * qds));
        p.s_c0 = (float)(1.5 * (std::sqrt(3.0) * E / qds + 1.5 * E * E / (qds * qds)) + 1e-6);
        p.s_c1 = (float)std::ldexp(1.0, -19);
        // u = fl(v s_scale) with v = fl(d2 r); |u - u*| <= s_c0 + s_c1 u gives
        // v s_scale (1 - 2^-24)(1 - s_c1) - s_c0 <= u* <= v s_scale (1 + 2^-24)(1 + s_c1) + s_c0
        const double sc = (double)p.s_scale, r24 = std::ldexp(1.0, -24);
        p.s_lo_mul = down_f(sc * (1.0 - (double)p.s_c1) * (1.0 - r24) * (1.0 - r24));
        p.s_hi_mul = up_f(sc * (1.0 + (double)p.s_c1) * (1.0 + r24) * (1.0 + r24));
    }
    p.s_top = 12582912.0f + (float)b.n_s;
    p.f_nmu = (float)b.n_mu;
    // queue sentinel: separation (n_s + 1/2) / n_s times the last edge (past
    // its band, half a bin past it for linear bins), |mu| = 1 / (2 n_mu)
    {
        const double smax_q = b.s_edges[b.n_s] * std::ldexp(1.0, p.bits) / L;
        const double s_sent = smax_q * (b.n_s + 0.5) / b.n_s;
        p.sent_d2 = (float)(s_sent * s_sent);
        p.sent_dx = (float)(0.5 * s_sent / b.n_mu);
    }

    // s-bin table over FP32 bit patterns of d2 + bias.  The bias (a power of
    // two well below the first positive edge band) keeps every key at or
    // above the table's first key.
    double vmin = INFINITY;
    for (int k = 0; k <= b.n_s; k++)
        if (p.T[k] > 0) vmin = std::min(vmin, (double)p.lo[k]);
    double bias = std::isfinite(vmin) && vmin > 0 ? std::ldexp(1.0, (int)std::floor(std::log2(vmin)) - 2)
                                                  : 1.0;
    bias = std::max(bias, std::ldexp(1.0, -100));
    p.tab_bias = (float)bias;
    int mb = 8;
    for (;; mb--) {
        const int sh = 23 - mb;
        uint32_t k0, ke;
        float fb = (float)bias, fhm = up_f((double)p.hit_max + bias);
        std::memcpy(&k0, &fb, 4);
        std::memcpy(&ke, &fhm, 4);
        k0 >>= sh;
        ke >>= sh;
        const long long n = (long long)ke - (long long)k0 + 1;
        if (n <= MAX_TABLE || mb <= 4) {
            p.tab_shift = sh;
            p.tab_key0 = k0;
            p.tab_n = (int)std::min<long long>(n, MAX_TABLE);
            break;
        }
    }
    pl.table.assign(p.tab_n, CODE_AMBIG);
    for (int i = 0; i < p.tab_n; i++) {
        const uint32_t key = p.tab_key0 + (uint32_t)i;
        uint32_t blo = key << p.tab_shift, bhi = (key + 1) << p.tab_shift;
        float flo, fhi;
        std::memcpy(&flo, &blo, 4);
        std::memcpy(&fhi, &bhi, 4);
        // d2 values whose rounded d2 + bias lands in this slot
        const double slack = ulp_f32((double)fhi);
        const double vlo = (i == 0) ? -INFINITY : (double)flo - bias - slack;
        const double vhi = (i == p.tab_n - 1) ? INFINITY : (double)fhi - bias + slack;
        int passed = 0, slot = 0;
        for (int k = 0; k <= b.n_s; k++) {
            if (p.T[k] == 0 || (double)p.hi[k] <= vlo) passed++;
            else if ((double)p.lo[k] >= vhi) {}
            else slot++;
        }
        pl.table[i] = (slot <= 1) ? (int16_t)(passed - 1) : CODE_AMBIG;
    }
    return TPCF_OK;
}

// Direct pair counter (pairdirect.cu).  Coordinates are x = RN(RN(float(dx_grid)) inv)
// with inv = RN(1 / (q ds)), dx_grid the exact integer offset from the unit's
// cell corner, so |x| <= Xb bins.  The bounds follow every rounding of the
// kernel's arithmetic:
//   E    : one coordinate's error (conversion and scaling; the common
//          relative error kappa of inv is carried separately),
//   e_d  : a coordinate difference's error for pairs below n_s + 2 bins
//          (2 E plus the subtraction's rounding),
//   d2   : |d2 - s*^2| <= 2 sqrt3 e_d s* + 3 e_d^2 + gamma_3 d2 (three fused
//          roundings, the tiny addend included), and for the s* >= 1/2 near
//          any edge sqrt(d2) + s* >= 1.99 s*, so
//          |sqrt(d2) - s*| <= dsq = 1.01 (sqrt3 e_d + 1.5 e_d^2 / 0.5 + gamma_3 (n_s + 2) / 1.99),
//   u    = d2 r exactly inside the FMA, r = rsqrt(d2) within rho = 2^-22.5 (the
//          hardware's measured worst case over all inputs is 2^-22.94).
// The s residual band is eps_s = 1.1 (dsq + rho (n_s + 1.5) + kappa (n_s + 1) +
// tiny) + 2^-24: a pair with |u - floor(u) - 1/2| <= 1/2 - eps_s has s* in the
// same bin.  The mu interval: n_mu dx -+ m, one rounding each way from the
// exact product n_mu b_x, times r, brackets n_mu dx* / s* when m >= m0 =
// 1.1 (n_mu 2E + 1.5 ulp(n_mu Xb + 1) + n_mu rho (n_s + 1) + n_mu dsq) (the
// common scale cancels in mu) plus the bias of the d2 addend (see below).
bool build_direct(const tpcf_binning &b, const Plan &pl, int smem_sm, int smem_block, int reserved,
                  unsigned long long max_cat, DirectParams &d)
{
    const CountParams &p = pl.prm;
    std::memset(&d, 0, sizeof(d));
    if (!p.linear) return false;
    const bool mu = p.n_mu > 1;
    const bool mid = mu && p.los == TPCF_LOS_MIDPOINT;
    if (mu && p.los != TPCF_LOS_X && !mid) return false;
    const double L = b.box_L;
    const double q = std::ldexp(1.0, p.bits) / L;
    const double qds = q * b.s_edges[1];
    const float inv = (float)(1.0 / qds);
    const double u24 = std::ldexp(1.0, -24);
    const double kappa = std::fabs((double)inv * qds - 1.0);
    const double Wmax = std::ldexp(1.0, p.bits) / (double)p.n_c + 1.0;
    const double Xg = (double)(pl.K + 1) * Wmax;
    const double Xb = Xg / qds * (1.0 + std::ldexp(1.0, -20));
    const double E = 0.5 * ulp_f32(Xg) / qds * (1.0 + std::ldexp(1.0, -20)) + 0.5 * ulp_f32(Xb);
    const double n_s = p.n_s, n_mu = p.n_mu;
    const double e_d = 2.0 * E + 0.5 * ulp_f32(n_s + 2.0);
    const double g3 = 3.0 * u24 / (1.0 - 3.0 * u24);
    const double rho = std::pow(2.0, -22.5);
    const double dsq = 1.01 * (std::sqrt(3.0) * e_d + 3.0 * e_d * e_d + g3 * (n_s + 2.0) / 1.99);
    // mu margin (below) and the d2 addend: s only, a negligible 2^-60; with mu
    // bins, tiny = m0^2 / n_mu, which biases r = rsqrt(d2 + tiny) low by at
    // most n_mu tiny / (2 s) <= m0 / 4 in the mu interval for s >= 2 m0, and
    // leaves the interval wider than one bin (always rechecked) below 2 m0
    double m0 = 0.0;
    if (mid) {
        // Midpoint line of sight, l = a + b - 2 o in bin units (o: the observer
        // relative to the cell's corner).  mu = (l.d) r rl from the computed
        // vectors differs from the exact one by at most the angle each vector's
        // rounding turns it, sqrt3 E_l / |l| + sqrt3 e_d / |d|, plus the
        // arithmetic (the dot product gamma3, d2 and |l|^2 gamma3 and rsqrt rho
        // each, two products): c1 r + c3 rl + c2 in units of n_mu mu.  The
        // addends tiny, tinyl bias r, rl low by at most sqrt(tiny) r / 2 (resp.
        // rl), folded into c1, c3 (x 1.5); below d2 = tiny, c1 r > 1/2 so the
        // pair is always rechecked.  |mu| <= 1 + 2^-20 by Cauchy-Schwarz on the
        // computed vectors, so the signed column stays within n_mu + 1.
        const double Og0 = std::max({std::fabs((double)p.obs[0]), std::fabs((double)p.obs[1]),
                                     std::fabs((double)p.obs[2])});
        const double Og = Og0 + std::ldexp(1.0, p.bits) + Wmax;      // |observer - any cell corner|, grid units
        const double Ob = Og / qds * (1.0 + std::ldexp(1.0, -20));
        const double E_o = 0.5 * ulp_f32(Og) / qds * (1.0 + std::ldexp(1.0, -20)) + 0.5 * ulp_f32(Ob);
        const double LAb = Xb + 2.0 * Ob * (1.0 + u24);
        const double Lb = Xb + LAb;
        const double E_l = 2.0 * E + 2.0 * E_o + 0.5 * ulp_f32(LAb) + 0.5 * ulp_f32(Lb);
        const double c1_0 = n_mu * 1.1 * std::sqrt(3.0) * e_d, c3_0 = n_mu * 1.1 * std::sqrt(3.0) * E_l;
        const double c2 = 1.1 * n_mu * (2.0 * g3 + 2.0 * rho + 2.0 * u24) + std::ldexp(1.0, -22);
        d.c1 = up_f(1.5 * 1.01 * c1_0);
        d.c3 = up_f(1.5 * 1.01 * c3_0);
        d.c05 = down_f(0.5 - c2);
        d.tinyl = down_f((c3_0 / n_mu) * (c3_0 / n_mu));
        if (!(d.c1 < 0.05f) || !(d.c3 < 0.05f) || !(d.c05 > 0.45f) || !(d.tinyl >= 1.0e-30f)) return false;
        m0 = c1_0 / n_mu;   // tiny = (c1_0 / n_mu)^2 below
    } else if (mu) {
        m0 = 1.1 * (n_mu * 2.0 * E + 1.5 * ulp_f32(n_mu * Xb + 1.0) + n_mu * rho * (n_s + 1.0) + n_mu * dsq);
        if (!(m0 < 0.04)) return false;
    }
    const float tiny = mid ? down_f(m0 * m0) : (mu ? down_f(m0 * m0 / n_mu) : (float)std::ldexp(1.0, -60));
    if (!(tiny > 0.0f)) return false;
    const double eps_s = 1.1 * (dsq + rho * (n_s + 1.5) + kappa * (n_s + 1.0) + (double)tiny) + u24;
    if (!(eps_s < 0.05)) return false;
    d.cs = down_f(0.5 - eps_s);
    d.logC = 0;
    d.CO = 0;
    if (mu) {
        d.m = mid ? 0.0f : up_f(1.25 * m0 * (1.0 + 1e-6));
        // |t+-| <= n_mu + m / sqrt(tiny) (x line of sight), |t| <= n_mu (1 + 2^-20)
        // (midpoint): signed columns j in [-CO, CO - 1]
        const double ext = mid ? 1.0 : (double)d.m / std::sqrt((double)tiny);
        d.CO = p.n_mu + 1 + (int)std::ceil(ext);
        d.mid = mid ? 1 : 0;
        int lc = 0;
        while ((1 << lc) < 2 * d.CO) lc++;
        if (lc < 5) lc = 5;
        if (lc > 6) return false;
        d.logC = lc;
    }
    d.tiny = tiny;
    d.inv_qds = inv;
    d.nmu = (float)p.n_mu;
    d.hit = up_f((n_s + 0.01) * (n_s + 0.01));
    // every pair's d2 is at least tiny, a normal float, so r = rsqrt(d2) is
    // finite and every histogram address stays inside the table
    if (!(d.tiny >= 1.0e-30f) || !std::isfinite(d.m) || !(d.cs > 0.4f) || !(inv > 0.0f)) return false;
    d.s_top = (float)(8388608.0 + n_s);
    d.C = 1 << d.logC;
    d.rows = p.n_s + 1;
    // one block of DIRECT_WARPS warps per SM (their registers fill the
    // register file), with 32 histogram copies when they fit beside the
    // warps' regions, else 16
    const long long budget = (long long)std::min(smem_block, smem_sm - reserved);
    for (int W : {DIRECT_WARPS}) {
        for (int R : {32, 16}) {
            const long long need = (long long)pairdirect_smem_bytes(p, R, d.C, W);
            if (need <= budget) {
                d.R = R;
                d.W = W;
                d.smem = (int)need;
                // in one unit a lane pairs at most 64 a-points with at most
                // max_cat / 32 + 16 b-points (its tile slots), and 32 / R
                // lanes share a counter copy
                d.unit_pair_bound = (unsigned long long)DIRECT_ACHUNK *
                                    (max_cat / (unsigned long long)R + 512ull / (unsigned long long)R + 16ull);
                return true;
            }
        }
    }
    return false;
}

}  // namespace tpcf
