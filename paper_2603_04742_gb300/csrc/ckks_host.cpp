// CKKS encoding and decoding on the host (client side): the inverse canonical
// embedding restricted to real slot values, in double-double arithmetic so
// that every rounding to an integer coefficient is the exact one.
//
// Slot j < N/2 is the evaluation at zeta^(5^j), zeta = exp(i pi / N).  A real
// slot vector z at scale 2^b is the polynomial with coefficients
//   m_k = round(2^b * (2/N) * sum_j z_j cos(pi k 5^j / N)),   k < N,
// rounded half away from zero.  With Z of length M = 2N holding z_j at index
// 5^j mod 2N, the sum is the real part of the length-M DFT of Z at k.
// Decoding evaluates the coefficients at zeta^(5^j): the length-M DFT with
// the opposite sign, read at 5^j mod 2N.
//
// Double-double: a value is hi + lo with |lo| <= ulp(hi)/2 (Dekker 1971,
// Knuth's two-sum); products use fma, exact on every IEEE machine.
#include <cmath>
#include <cstring>

#include "internal.h"

namespace hespmv {
namespace {

struct dd {
    double hi, lo;
};

inline dd two_sum(double a, double b) {
    const double s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
inline dd quick_two_sum(double a, double b) {
    const double s = a + b;
    return {s, b - (s - a)};
}
inline dd two_prod(double a, double b) {
    const double p = a * b;
    return {p, std::fma(a, b, -p)};
}
inline dd add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
inline dd neg(dd a) { return {-a.hi, -a.lo}; }
inline dd sub(dd a, dd b) { return add(a, neg(b)); }
inline dd mul(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}
inline dd mul_d(dd a, double b) {
    dd p = two_prod(a.hi, b);
    p.lo += a.lo * b;
    return quick_two_sum(p.hi, p.lo);
}
inline dd div_d(dd a, double b) {
    const double q1 = a.hi / b;
    dd r = sub(a, two_prod(q1, b));
    const double q2 = r.hi / b;
    r = sub(r, two_prod(q2, b));
    const double q3 = r.hi / b;
    dd q = quick_two_sum(q1, q2);
    return add(q, {q3, 0.0});
}

// pi to double-double precision
const dd kPi = {3.141592653589793116e+00, 1.224646799147353207e-16};

// cos and sin of x in [0, pi/4] by their Taylor series (terms below 1e-40)
void cos_sin(dd x, dd &c, dd &s) {
    const dd x2 = mul(x, x);
    dd tc = {1.0, 0.0}, ts = x;
    c = tc;
    s = ts;
    for (int k = 1; k <= 24; ++k) {
        tc = div_d(mul(neg(tc), x2), (double)((2 * k - 1) * (2 * k)));
        ts = div_d(mul(neg(ts), x2), (double)((2 * k) * (2 * k + 1)));
        c = add(c, tc);
        s = add(s, ts);
    }
}

struct Trig {
    std::vector<dd> c, s;  // cos, sin of pi k / N for k < N
};

void make_trig(int log2n, Trig &T) {
    const int N = 1 << log2n, Q = N / 4;
    std::vector<dd> c0(Q + 1), s0(Q + 1);
    for (int k = 0; k <= Q; ++k) cos_sin(mul_d(kPi, (double)k / N), c0[k], s0[k]);
    T.c.assign(N, {0, 0});
    T.s.assign(N, {0, 0});
    for (int k = 0; k < N; ++k) {
        const int r = k <= N / 2 ? k : N - k;   // angle pi r / N in [0, pi/2]
        dd cr, sr;
        if (r <= Q) {
            cr = c0[r];
            sr = s0[r];
        } else {                                 // pi/2 - pi r / N = pi (N/2 - r) / N
            cr = s0[N / 2 - r];
            sr = c0[N / 2 - r];
        }
        T.c[k] = k <= N / 2 ? cr : neg(cr);      // cos(pi - a) = -cos(a)
        T.s[k] = sr;                             // sin(pi - a) = sin(a)
    }
}

// In-place radix-2 DFT of length M = 2N: X[k] = sum_n x[n] exp(sign i pi n k / N)
void dft(std::vector<dd> &re, std::vector<dd> &im, const Trig &T, int sign) {
    const int M = (int)re.size(), N = M / 2;
    int bits = 0;
    while ((1 << bits) < M) ++bits;
    for (int i = 0; i < M; ++i) {
        int j = 0;
        for (int b = 0; b < bits; ++b) j |= ((i >> b) & 1) << (bits - 1 - b);
        if (j > i) {
            std::swap(re[i], re[j]);
            std::swap(im[i], im[j]);
        }
    }
    for (int len = 2; len <= M; len <<= 1) {
        const int half = len / 2, step = M / len;  // twiddle angle pi (j * step) / N
        for (int base = 0; base < M; base += len)
            for (int j = 0; j < half; ++j) {
                const int k = j * step;               // < N
                const dd wr = T.c[k], wi = sign > 0 ? T.s[k] : neg(T.s[k]);
                const int a = base + j, b = a + half;
                const dd vr = sub(mul(re[b], wr), mul(im[b], wi));
                const dd vi = add(mul(re[b], wi), mul(im[b], wr));
                re[b] = sub(re[a], vr);
                im[b] = sub(im[a], vi);
                re[a] = add(re[a], vr);
                im[a] = add(im[a], vi);
            }
    }
    (void)N;
}

// round half away from zero of hi + lo (|value| < 2^62), decided exactly
int64_t round_dd(dd v) {
    const bool negv = v.hi < 0 || (v.hi == 0 && v.lo < 0);
    const dd a = negv ? neg(v) : v;
    const double fl = std::floor(a.hi);
    int64_t r;
    if (fl == a.hi) {
        // integral hi: the value is hi + lo, and rounding up at a half is
        // away from zero because the value is non-negative
        r = (int64_t)fl + (int64_t)std::floor(a.lo + 0.5);
    } else {
        // hi < 2^52 is not integral, so 0 < (hi - fl) + lo < 1; t is exact and
        // the comparison t >= -lo decides (hi - fl) + lo >= 1/2 without rounding
        const double t = (a.hi - fl) - 0.5;
        r = (int64_t)fl + (t >= -a.lo ? 1 : 0);
    }
    return negv ? -r : r;
}

}  // namespace

struct CkksCodec {
    int log2n = 0;
    Trig T;
};

CkksCodec *ckks_codec(int log2n) {
    CkksCodec *c = new CkksCodec();
    c->log2n = log2n;
    make_trig(log2n, c->T);
    return c;
}

void ckks_codec_free(CkksCodec *c) { delete c; }

std::string ckks_encode(const CkksCodec &C, const double *z, size_t n, int scale_bits, int64_t *coef) {
    const int N = 1 << C.log2n, M = 2 * N;
    if (n > (size_t)N / 2) return "more values than N/2 slots";
    std::vector<dd> re(M, {0, 0}), im(M, {0, 0});
    uint64_t e = 1;
    for (size_t j = 0; j < n; ++j) {
        if (!std::isfinite(z[j])) return "value is not finite";
        re[e] = {z[j], 0.0};
        e = e * 5 % (uint64_t)M;
    }
    dft(re, im, C.T, -1);
    const double f = std::ldexp(1.0, scale_bits + 1 - C.log2n);  // 2^b * 2 / N, exact
    for (int k = 0; k < N; ++k) {
        const dd v = mul_d(re[k], f);
        if (!(std::fabs(v.hi) < 4.0e18)) return "coefficient beyond 2^62: scale too large";
        coef[k] = round_dd(v);
    }
    return "";
}

void ckks_decode(const CkksCodec &C, const double *coef, size_t n, double inv_scale, double *z) {
    const int N = 1 << C.log2n, M = 2 * N;
    std::vector<dd> re(M, {0, 0}), im(M, {0, 0});
    for (int k = 0; k < N; ++k) re[k] = {coef[k], 0.0};
    dft(re, im, C.T, +1);
    uint64_t e = 1;
    for (size_t j = 0; j < n; ++j) {
        z[j] = (re[e].hi + re[e].lo) * inv_scale;
        e = e * 5 % (uint64_t)M;
    }
}

// ------------------------------------------------------------ CRT to real
// Centred [x]_Q from its residues, exactly (multi-word integers), then to a
// double: x = sum_i [x_i * (Q/q_i)^-1]_{q_i} * (Q/q_i) - u Q, 0 <= u < L.
struct CrtReal {
    int L = 0, W = 0;
    std::vector<uint64_t> q, qhat_inv, Q, Qhalf, Qhat;  // Qhat: [L][W]
};

namespace {
typedef unsigned __int128 u128;

void mul_small(std::vector<uint64_t> &a, uint64_t m) {
    uint64_t carry = 0;
    for (uint64_t &w : a) {
        const u128 p = (u128)w * m + carry;
        w = (uint64_t)p;
        carry = (uint64_t)(p >> 64);
    }
}
// a += b * m
void add_mul(uint64_t *a, const uint64_t *b, uint64_t m, int W) {
    uint64_t carry = 0;
    for (int k = 0; k < W; ++k) {
        const u128 p = (u128)b[k] * m + a[k] + carry;
        a[k] = (uint64_t)p;
        carry = (uint64_t)(p >> 64);
    }
}
bool geq(const uint64_t *a, const uint64_t *b, int W) {
    for (int k = W - 1; k >= 0; --k)
        if (a[k] != b[k]) return a[k] > b[k];
    return true;
}
void sub_in(uint64_t *a, const uint64_t *b, int W) {  // a -= b (a >= b)
    uint64_t borrow = 0;
    for (int k = 0; k < W; ++k) {
        const u128 d = (u128)a[k] - b[k] - borrow;
        a[k] = (uint64_t)d;
        borrow = (uint64_t)(d >> 64) & 1;
    }
}
double to_double(const uint64_t *a, int W) {
    double d = 0;
    for (int k = W - 1; k >= 0; --k) d = d * 18446744073709551616.0 + (double)a[k];
    return d;
}
uint64_t powmod(uint64_t a, uint64_t e, uint64_t m) {
    uint64_t r = 1;
    a %= m;
    for (; e; e >>= 1) {
        if (e & 1) r = (uint64_t)((u128)r * a % m);
        a = (uint64_t)((u128)a * a % m);
    }
    return r;
}
}  // namespace

CrtReal *crt_real(const uint64_t *q, int L) {
    CrtReal *c = new CrtReal();
    c->L = L;
    c->W = (64 * L) / 64 + 2;   // Q < 2^(64 L)
    c->q.assign(q, q + L);
    c->Q.assign(c->W, 0);
    c->Q[0] = 1;
    for (int i = 0; i < L; ++i) mul_small(c->Q, q[i]);
    c->Qhalf = c->Q;  // floor(Q / 2)
    for (int k = 0; k < c->W; ++k)
        c->Qhalf[k] = (c->Q[k] >> 1) | (k + 1 < c->W ? (c->Q[k + 1] << 63) : 0);
    c->Qhat.assign((size_t)L * c->W, 0);
    c->qhat_inv.resize(L);
    for (int i = 0; i < L; ++i) {
        std::vector<uint64_t> h(c->W, 0);
        h[0] = 1;
        uint64_t hm = 1;
        for (int o = 0; o < L; ++o)
            if (o != i) {
                mul_small(h, q[o]);
                hm = (uint64_t)((u128)hm * (q[o] % q[i]) % q[i]);
            }
        std::copy(h.begin(), h.end(), c->Qhat.begin() + (size_t)i * c->W);
        c->qhat_inv[i] = powmod(hm, q[i] - 2, q[i]);
    }
    return c;
}

void crt_real_free(CrtReal *c) { delete c; }

void crt_to_double(const CrtReal &c, const uint64_t *x, int N, double *out) {
    const int L = c.L, W = c.W;
    std::vector<uint64_t> acc(W);
    for (int k = 0; k < N; ++k) {
        std::fill(acc.begin(), acc.end(), 0);
        for (int i = 0; i < L; ++i) {
            const uint64_t y = (uint64_t)((u128)x[(size_t)i * N + k] * c.qhat_inv[i] % c.q[i]);
            add_mul(acc.data(), &c.Qhat[(size_t)i * W], y, W);
        }
        while (geq(acc.data(), c.Q.data(), W)) sub_in(acc.data(), c.Q.data(), W);
        if (geq(acc.data(), c.Qhalf.data(), W) && !std::equal(acc.begin(), acc.end(), c.Qhalf.begin())) {
            std::vector<uint64_t> neg(c.Q);
            sub_in(neg.data(), acc.data(), W);      // Q - x
            out[k] = -to_double(neg.data(), W);
        } else {
            out[k] = to_double(acc.data(), W);
        }
    }
}

}  // namespace hespmv
