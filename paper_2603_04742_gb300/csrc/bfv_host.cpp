// BFV constants for exact Chinese remaindering (host), and BFV decryption of
// coefficient residues: m = round(t x / Q) mod t for the centred x = [x]_Q.
//
// Multi-word integers are little-endian arrays of 64-bit words; negative
// values are two's complement over the array's width.
#include <cmath>

#include "internal.h"

namespace hespmv {
namespace {

typedef unsigned __int128 u128;

uint64_t mulm(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((u128)a * b % m); }
uint64_t powm(uint64_t a, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m;
    a %= m;
    for (; e; e >>= 1) {
        if (e & 1) r = mulm(r, a, m);
        a = mulm(a, a, m);
    }
    return r;
}
uint64_t invm(uint64_t a, uint64_t p) { return powm(a % p, p - 2, p); }
uint64_t shoup(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }

void mul_small(std::vector<uint64_t> &a, uint64_t m) {
    uint64_t carry = 0;
    for (uint64_t &w : a) {
        const u128 p = (u128)w * m + carry;
        w = (uint64_t)p;
        carry = (uint64_t)(p >> 64);
    }
}
uint64_t mod_small(const std::vector<uint64_t> &a, uint64_t m) {
    u128 r = 0;
    for (size_t k = a.size(); k-- > 0;) r = ((r << 64) | a[k]) % m;
    return (uint64_t)r;
}
std::vector<uint64_t> half(const std::vector<uint64_t> &a) {
    std::vector<uint64_t> h(a.size());
    for (size_t k = 0; k < a.size(); ++k) h[k] = (a[k] >> 1) | (k + 1 < a.size() ? a[k + 1] << 63 : 0);
    return h;
}
int words_for(const std::vector<uint64_t> &primes) {
    double bits = 0;
    for (uint64_t q : primes) bits += std::log2((double)q);
    return (int)std::ceil((bits + 2) / 64.0) + 1;   // room for a sign and sums of terms
}
// product of all primes but `skip` (or all, skip < 0), W words
std::vector<uint64_t> product(const std::vector<uint64_t> &primes, int skip, int W) {
    std::vector<uint64_t> r(W, 0);
    r[0] = 1;
    for (int i = 0; i < (int)primes.size(); ++i)
        if (i != skip) mul_small(r, primes[i]);
    return r;
}

}  // namespace

BfvLayout bfv_layout(const HostTables &h) {
    BfvLayout o;
    const int64_t L = h.L, nB = h.nB, wq = h.wq, wb = h.wb;
    int64_t at = 0;
    o.qhat = at;     at += L * wq;
    o.Q = at;        at += wq;
    o.Qhalf = at;    at += wq;
    o.qhat_inv = at; at += 2 * L;       // Shoup pairs
    o.bhat = at;     at += nB * wb;
    o.B = at;        at += wb;
    o.Bhalf = at;    at += wb;
    o.bhat_inv = at; at += 2 * nB;
    o.pow_b = at;    at += 2 * nB * (wq + 1);  // 2^(64 k) mod b_j, k <= wq (Shoup pairs)
    o.pow_q = at;    at += 2 * L * (wb + 1);   // 2^(64 k) mod q_i, k <= wb (Shoup pairs)
    o.qinv_b = at;   at += 2 * nB;
    o.t_b = at;      at += 2 * nB;
    o.t_q = at;      at += 2 * L;
    o.size = at;
    return o;
}

bool bfv_tables(const hespmv_params &p, HostTables &h, std::string &err) {
    const int L = h.L, nB = h.nB;
    const std::vector<uint64_t> qs(h.q.begin(), h.q.begin() + L);
    const std::vector<uint64_t> bs(h.q.begin() + h.iB, h.q.begin() + h.iB + nB);
    h.wq = words_for(qs);
    h.wb = words_for(bs);
    if (h.wq > 16 || h.wb > 16 || nB > 16) {
        err = "BFV: Q and the auxiliary basis must stay below 1000 bits (16 primes)";
        return false;
    }
    const uint64_t t = p.t;
    const BfvLayout o = bfv_layout(h);
    std::vector<uint64_t> &c = h.bfv_const;
    c.assign(o.size, 0);
    const std::vector<uint64_t> Q = product(qs, -1, h.wq), B = product(bs, -1, h.wb);
    for (int i = 0; i < L; ++i) {
        const std::vector<uint64_t> qh = product(qs, i, h.wq);
        std::copy(qh.begin(), qh.end(), c.begin() + o.qhat + (int64_t)i * h.wq);
        const uint64_t inv = invm(mod_small(qh, qs[i]), qs[i]);
        c[o.qhat_inv + 2 * i] = inv;
        c[o.qhat_inv + 2 * i + 1] = shoup(inv, qs[i]);
        uint64_t pw = 1;
        const uint64_t r64 = (uint64_t)(((u128)1 << 64) % qs[i]);
        for (int k = 0; k <= h.wb; ++k) {
            c[o.pow_q + (int64_t)i * 2 * (h.wb + 1) + 2 * k] = pw;
            c[o.pow_q + (int64_t)i * 2 * (h.wb + 1) + 2 * k + 1] = shoup(pw, qs[i]);
            pw = mulm(pw, r64, qs[i]);
        }
        c[o.t_q + 2 * i] = t % qs[i];
        c[o.t_q + 2 * i + 1] = shoup(t % qs[i], qs[i]);
    }
    std::copy(Q.begin(), Q.end(), c.begin() + o.Q);
    const std::vector<uint64_t> Qh = half(Q), Bh = half(B);
    std::copy(Qh.begin(), Qh.end(), c.begin() + o.Qhalf);
    std::copy(B.begin(), B.end(), c.begin() + o.B);
    std::copy(Bh.begin(), Bh.end(), c.begin() + o.Bhalf);
    for (int j = 0; j < nB; ++j) {
        const uint64_t b = bs[j];
        const std::vector<uint64_t> bh = product(bs, j, h.wb);
        std::copy(bh.begin(), bh.end(), c.begin() + o.bhat + (int64_t)j * h.wb);
        const uint64_t inv = invm(mod_small(bh, b), b);
        c[o.bhat_inv + 2 * j] = inv;
        c[o.bhat_inv + 2 * j + 1] = shoup(inv, b);
        uint64_t pw = 1;
        const uint64_t r64 = (uint64_t)(((u128)1 << 64) % b);
        for (int k = 0; k <= h.wq; ++k) {
            c[o.pow_b + (int64_t)j * 2 * (h.wq + 1) + 2 * k] = pw;
            c[o.pow_b + (int64_t)j * 2 * (h.wq + 1) + 2 * k + 1] = shoup(pw, b);
            pw = mulm(pw, r64, b);
        }
        const uint64_t qinv = invm(mod_small(Q, b), b);
        c[o.qinv_b + 2 * j] = qinv;
        c[o.qinv_b + 2 * j + 1] = shoup(qinv, b);
        c[o.t_b + 2 * j] = t % b;
        c[o.t_b + 2 * j + 1] = shoup(t % b, b);
    }
    // Delta = floor(Q/t) = (Q - (Q mod t)) / t: mod q_i that is -(Q mod t) * t^-1
    const uint64_t qmodt = mod_small(Q, t);
    h.bfv_delta.assign((size_t)L * 2, 0);
    for (int i = 0; i < L; ++i) {
        const uint64_t d = mulm((qs[i] - qmodt % qs[i]) % qs[i], invm(t % qs[i], qs[i]), qs[i]);
        h.bfv_delta[2 * i] = d;
        h.bfv_delta[2 * i + 1] = shoup(d, qs[i]);
    }
    h.bfv_qinv_t = invm(qmodt, t);
    return true;
}

void bfv_decrypt_coef(const HostTables &h, const uint64_t *x, uint64_t *m) {
    // t x = Q m' + r with r = [t x]_Q centred, so round(t x / Q) = m' (|r| < Q/2)
    // and m' = -r Q^-1 mod t
    const int L = h.L, N = h.N, W = h.wq;
    const BfvLayout o = bfv_layout(h);
    const uint64_t *c = h.bfv_const.data(), t = h.t;
    std::vector<uint64_t> acc(W);
    for (int k = 0; k < N; ++k) {
        std::fill(acc.begin(), acc.end(), 0);
        for (int i = 0; i < L; ++i) {
            const uint64_t q = h.q[i];
            const uint64_t r = mulm(x[(size_t)i * N + k], t % q, q);
            const uint64_t y = mulm(r, c[o.qhat_inv + 2 * i], q);
            uint64_t carry = 0;
            for (int w = 0; w < W; ++w) {
                const u128 s = (u128)c[o.qhat + (int64_t)i * W + w] * y + acc[w] + carry;
                acc[w] = (uint64_t)s;
                carry = (uint64_t)(s >> 64);
            }
        }
        auto geq = [&](const uint64_t *b) {
            for (int w = W - 1; w >= 0; --w)
                if (acc[w] != b[w]) return acc[w] > b[w];
            return true;
        };
        auto sub = [&](const uint64_t *b, std::vector<uint64_t> &a) {
            uint64_t br = 0;
            for (int w = 0; w < W; ++w) {
                const u128 d = (u128)a[w] - b[w] - br;
                a[w] = (uint64_t)d;
                br = (uint64_t)(d >> 64) & 1;
            }
        };
        while (geq(c + o.Q)) sub(c + o.Q, acc);
        uint64_t rt;  // [t x]_Q mod t, centred representative
        if (geq(c + o.Qhalf) && !std::equal(acc.begin(), acc.end(), c + o.Qhalf)) {
            std::vector<uint64_t> neg(c + o.Q, c + o.Q + W);
            sub(acc.data(), neg);                   // Q - acc = |r|
            rt = (t - mod_small(neg, t)) % t;
        } else {
            rt = mod_small(acc, t);
        }
        m[k] = mulm((t - rt) % t, h.bfv_qinv_t, t);
    }
}

}  // namespace hespmv
