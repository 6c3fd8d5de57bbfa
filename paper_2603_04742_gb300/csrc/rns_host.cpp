// Host construction of the RNS parameter tables: prime search, roots of
// unity, twiddle tables (with Shoup companions) and the base-conversion
// constants of hybrid key switching.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace hespmv {

typedef unsigned __int128 u128;

static uint64_t mulm(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((u128)a * b % m); }

static uint64_t powm(uint64_t a, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m;
    a %= m;
    for (; e; e >>= 1) {
        if (e & 1) r = mulm(r, a, m);
        a = mulm(a, a, m);
    }
    return r;
}

static uint64_t invm(uint64_t a, uint64_t p) { return powm(a % p, p - 2, p); }

static uint64_t shoup(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }

// Deterministic Miller-Rabin for 64-bit n (bases 2..37 suffice below 3.3e24).
static bool prime64(uint64_t n) {
    static const uint64_t bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (uint64_t b : bases)
        if (n % b == 0) return n == b;
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        ++s;
    }
    for (uint64_t a : bases) {
        uint64_t x = powm(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; ++r) {
            x = mulm(x, x, n);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}

// Smallest primitive 2N-th root of unity mod prime q (q = 1 mod 2N).  Every
// primitive 2N-th root is an odd power of one of them; scan those powers.
static uint64_t smallest_2n_root(uint64_t q, uint64_t N) {
    uint64_t g = 2;
    while (powm(g, (q - 1) / 2, q) != q - 1) ++g;  // a quadratic non-residue
    uint64_t r = powm(g, (q - 1) / (2 * N), q);   // order exactly 2N
    uint64_t r2 = mulm(r, r, q), cur = r, best = r;
    for (uint64_t k = 1; k < N; ++k) {
        cur = mulm(cur, r2, q);
        if (cur < best) best = cur;
    }
    return best;
}

uint32_t host_bitrev(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int b = 0; b < bits; ++b) r |= ((x >> b) & 1u) << (bits - 1 - b);
    return r;
}

uint32_t ntt_index_of_exponent(uint64_t e, int log2n) {
    return host_bitrev((uint32_t)((e - 1) / 2), log2n);
}

static int bitlen(uint64_t x) { return 64 - __builtin_clzll(x); }

bool build_tables(const hespmv_params &p, HostTables &h, std::string &err) {
    if (p.log2n < 4 || p.log2n > 15) { err = "log2n must be in [4, 15]"; return false; }
    if (p.L < 1 || p.L > 16 || p.K < 1 || p.K > 4) { err = "need 1<=L<=16, 1<=K<=4"; return false; }
    if (p.dnum < 1 || p.dnum > p.L) { err = "need 1 <= dnum <= L"; return false; }
    const int bits = p.prime_bits ? p.prime_bits : 50;
    if (bits < 20 || bits > 50) { err = "prime_bits must be in [20, 50]"; return false; }
    h.log2n = p.log2n;
    h.N = 1 << p.log2n;
    h.L = p.L;
    h.K = p.K;
    h.dnum = p.dnum;
    h.alpha = (p.L + p.dnum - 1) / p.dnum;
    if ((p.L + h.alpha - 1) / h.alpha != p.dnum) { err = "dnum leaves an empty digit"; return false; }
    h.slots = p.slots ? p.slots : h.N / 2;
    if (h.slots < 1 || h.slots > h.N / 2) { err = "slots must be in [1, N/2]"; return false; }
    const uint64_t N = (uint64_t)h.N, twoN = 2 * N;
    const bool ckks = p.scheme == HESPMV_SCHEME_CKKS, bfv = p.scheme == HESPMV_SCHEME_BFV;
    if (p.scheme != HESPMV_SCHEME_BGV && !ckks && !bfv) { err = "unknown scheme"; return false; }
    if (bfv && p.K < h.alpha) { err = "BFV needs K >= alpha (P must cover a key-switching digit)"; return false; }
    h.scheme = p.scheme;
    if (ckks) {
        if (p.t != 0) { err = "CKKS takes no plaintext modulus (t = 0)"; return false; }
        if (p.scale_bits < 10 || p.scale_bits > 60 || p.mask_scale_bits < 1 || p.mask_scale_bits > 60) {
            err = "CKKS scales: scale_bits in [10, 60], mask_scale_bits in [1, 60]";
            return false;
        }
        if (p.K < h.alpha) { err = "CKKS needs K >= alpha (P must cover a key-switching digit)"; return false; }
        h.scale_bits = p.scale_bits;
        h.mask_scale_bits = p.mask_scale_bits;
    } else if (p.t < 3 || p.t >= (1ull << 50) || p.t % twoN != 1 || !prime64(p.t)) {
        err = "t must be a prime below 2^50 with t = 1 mod 2N";
        return false;
    }
    // the t of every key, encryption and key-switching formula (BGV only: t e)
    const uint64_t tk = (ckks || bfv) ? 1 : p.t;
    h.t = ckks ? 1 : p.t;  // plaintext modulus (none for CKKS)
    // ciphertext primes: descending from the largest q < 2^bits, q = 1 mod 2N
    h.q.clear();
    uint64_t cand = (((1ull << bits) - 2) / twoN) * twoN + 1;
    while ((int)h.q.size() < p.L + p.K + (ckks ? 1 : 0)) {
        if (cand < twoN) { err = "not enough NTT primes"; return false; }
        if (prime64(cand) && cand != p.t) h.q.push_back(cand);
        cand -= twoN;
    }
    // last table entry: t (BGV plaintext NTT); CKKS has no plaintext modulus
    // and keeps the next NTT prime there, unused
    if (!ckks) h.q.push_back(p.t);
    if (bfv) {
        // auxiliary basis B for the exact HE-Mult: B > 2 t N Q bounds both the
        // integer tensor (|d| <= N Q^2 / 2 needs Q B > N Q^2) and its scaled
        // and rounded value (|z| <= t N Q / 2 + 1)
        double need = std::log2((double)p.t) + p.log2n + 2.0;
        for (int i = 0; i < p.L; ++i) need += std::log2((double)h.q[i]);
        h.iB = (int)h.q.size();
        double have = 0;
        while (have < need) {
            if (cand < twoN) { err = "not enough NTT primes for the BFV auxiliary basis"; return false; }
            if (prime64(cand) && cand != p.t) {
                h.q.push_back(cand);
                have += std::log2((double)cand);
            }
            cand -= twoN;
        }
        h.nB = (int)h.q.size() - h.iB;
    }
    h.pack_bits = 0;
    for (int i = 0; i < p.L; ++i) h.pack_bits = std::max(h.pack_bits, 64 - __builtin_clzll(h.q[i]));
    const int M = (int)h.q.size();
    h.psi.resize(M);
    h.mc.resize(M);
    h.tw.assign((size_t)M * 4 * N, 0);
    std::vector<uint64_t> pw(N), ipw(N);
    for (int m = 0; m < M; ++m) {
        const uint64_t q = h.q[m];
        const uint64_t psi = smallest_2n_root(q, N);
        h.psi[m] = psi;
        const uint64_t ipsi = invm(psi, q);
        pw[0] = ipw[0] = 1;
        for (uint64_t e = 1; e < N; ++e) {
            pw[e] = mulm(pw[e - 1], psi, q);
            ipw[e] = mulm(ipw[e - 1], ipsi, q);
        }
        uint64_t *T = &h.tw[(size_t)m * 4 * N];
        for (uint64_t k = 0; k < N; ++k) {
            uint32_t b = host_bitrev((uint32_t)k, p.log2n);
            T[2 * k] = pw[b];  // forward pairs (w, Shoup), then inverse pairs
            T[2 * k + 1] = shoup(pw[b], q);
            T[2 * N + 2 * k] = ipw[b];
            T[2 * N + 2 * k + 1] = shoup(ipw[b], q);
        }
        ModConst &c = h.mc[m];
        memset(&c, 0, sizeof(c));
        c.q = q;
        c.k = bitlen(q);
        c.mu = (uint64_t)(((u128)1 << (2 * c.k)) / q);
        c.bs = std::max(0, 2 * c.k - 64);
        c.bmu = (uint64_t)(((u128)1 << (64 + c.bs)) / q);
        c.ninv = invm(N % q, q);
        c.ninv_s = shoup(c.ninv, q);
        c.w1ninv = mulm(T[2 * N + 2], c.ninv, q);
        c.w1ninv_s = shoup(c.w1ninv, q);
        uint64_t inv = q;  // Newton iteration for q^-1 mod 2^64 (q odd)
        for (int it = 0; it < 6; ++it) inv *= 2 - q * inv;
        c.qneg = 0 - inv;
        c.rmod = (0 - q) % q;
        c.one_s = shoup(1, q);
    }
    const int L = p.L, K = p.K, LK = L + K, A = h.alpha;
    // ModUp constants
    h.modup_inv.assign((size_t)p.dnum * A * 2, 0);
    h.modup_mod.assign((size_t)p.dnum * A * LK * 2, 0);
    for (int j = 0; j < p.dnum; ++j) {
        const int i0 = j * A, i1 = std::min(L, (j + 1) * A);
        for (int i = i0; i < i1; ++i) {
            const uint64_t qi = h.q[i];
            uint64_t prod = 1;
            for (int o = i0; o < i1; ++o)
                if (o != i) prod = mulm(prod, h.q[o] % qi, qi);
            const uint64_t inv = invm(prod, qi);
            h.modup_inv[((size_t)j * A + (i - i0)) * 2 + 0] = inv;
            h.modup_inv[((size_t)j * A + (i - i0)) * 2 + 1] = shoup(inv, qi);
            for (int l = 0; l < LK; ++l) {
                const uint64_t ql = h.q[l];
                uint64_t v = 1;
                for (int o = i0; o < i1; ++o)
                    if (o != i) v = mulm(v, h.q[o] % ql, ql);
                size_t at = (((size_t)j * A + (i - i0)) * LK + l) * 2;
                h.modup_mod[at] = v;
                h.modup_mod[at + 1] = shoup(v, ql);
            }
        }
    }
    // ModDown constants
    h.md_pk.assign((size_t)K * 2, 0);
    h.md_phat.assign((size_t)K * L * 2, 0);
    h.md_t.assign((size_t)L * 2, 0);
    h.md_pinv.assign((size_t)L * 2, 0);
    h.p_mod_q.assign((size_t)L * 2, 0);
    h.p_mont.assign((size_t)L, 0);
    h.p_mont2.assign((size_t)L, 0);
    for (int k = 0; k < K; ++k) {
        const uint64_t pk = h.q[L + k];
        uint64_t phat = 1;
        for (int o = 0; o < K; ++o)
            if (o != k) phat = mulm(phat, h.q[L + o] % pk, pk);
        const uint64_t v = mulm(invm(tk % pk, pk), invm(phat, pk), pk);
        h.md_pk[k * 2] = v;
        h.md_pk[k * 2 + 1] = shoup(v, pk);
        for (int i = 0; i < L; ++i) {
            const uint64_t qi = h.q[i];
            uint64_t ph = 1;
            for (int o = 0; o < K; ++o)
                if (o != k) ph = mulm(ph, h.q[L + o] % qi, qi);
            h.md_phat[((size_t)k * L + i) * 2] = ph;
            h.md_phat[((size_t)k * L + i) * 2 + 1] = shoup(ph, qi);
        }
    }
    for (int i = 0; i < L; ++i) {
        const uint64_t qi = h.q[i];
        uint64_t P = 1;
        for (int k = 0; k < K; ++k) P = mulm(P, h.q[L + k] % qi, qi);
        h.p_mod_q[i * 2] = P;
        h.p_mod_q[i * 2 + 1] = shoup(P, qi);
        h.p_mont[i] = mulm(P, (0 - qi) % qi, qi);
        h.p_mont2[i] = mulm(h.p_mont[i], (0 - qi) % qi, qi);
        const uint64_t pinv = invm(P, qi);
        h.md_pinv[i * 2] = pinv;
        h.md_pinv[i * 2 + 1] = shoup(pinv, qi);
        h.md_t[i * 2] = tk % qi;
        h.md_t[i * 2 + 1] = shoup(tk % qi, qi);
    }
    // decryption CRT constants
    h.dec.assign((size_t)L * 4 + 2, 0);
    h.dec_inv_q.assign(L, 0.0);
    // (Qhat_i^-1 mod q_i; BGV also Qhat_i mod t and Q mod t)
    const uint64_t tt = ckks ? h.q[LK] : p.t;  // CKKS: harmless stand-in, unused
    uint64_t Qt = 1;
    for (int i = 0; i < L; ++i) {
        const uint64_t qi = h.q[i];
        uint64_t prod = 1, prod_t = 1;
        for (int o = 0; o < L; ++o)
            if (o != i) {
                prod = mulm(prod, h.q[o] % qi, qi);
                prod_t = mulm(prod_t, h.q[o] % tt, tt);
            }
        const uint64_t inv = invm(prod, qi);
        h.dec[i * 4 + 0] = inv;
        h.dec[i * 4 + 1] = shoup(inv, qi);
        h.dec[i * 4 + 2] = prod_t;
        h.dec[i * 4 + 3] = shoup(prod_t, tt);
        h.dec_inv_q[i] = 1.0 / (double)qi;
        Qt = mulm(Qt, qi % tt, tt);
    }
    h.dec[(size_t)L * 4] = Qt;
    h.dec[(size_t)L * 4 + 1] = shoup(Qt, tt);
    h.t_mod.resize(LK);
    for (int l = 0; l < LK; ++l) h.t_mod[l] = tk % h.q[l];
    // fused key-switching constants
    h.ks_zc.assign((size_t)L * 4, 0);
    for (int i = 0; i < L; ++i) {
        const int j = i / A;
        const uint64_t qi = h.q[i], qinv = h.modup_inv[((size_t)j * A + (i - j * A)) * 2];
        const uint64_t c0 = mulm(h.mc[i].ninv, qinv, qi), c1 = mulm(h.mc[i].w1ninv, qinv, qi);
        h.ks_zc[i * 4 + 0] = c0;
        h.ks_zc[i * 4 + 1] = shoup(c0, qi);
        h.ks_zc[i * 4 + 2] = c1;
        h.ks_zc[i * 4 + 3] = shoup(c1, qi);
    }
    h.ks_yc.assign((size_t)K * 4, 0);
    h.md_phat_t.assign((size_t)K * L * 2, 0);
    for (int k = 0; k < K; ++k) {
        const uint64_t pk = h.q[L + k], v = h.md_pk[k * 2];
        const uint64_t c0 = mulm(h.mc[L + k].ninv, v, pk), c1 = mulm(h.mc[L + k].w1ninv, v, pk);
        h.ks_yc[k * 4 + 0] = c0;
        h.ks_yc[k * 4 + 1] = shoup(c0, pk);
        h.ks_yc[k * 4 + 2] = c1;
        h.ks_yc[k * 4 + 3] = shoup(c1, pk);
        for (int i = 0; i < L; ++i) {
            const uint64_t qi = h.q[i];
            const uint64_t w = mulm(h.md_phat[((size_t)k * L + i) * 2], tk % qi, qi);
            h.md_phat_t[((size_t)k * L + i) * 2] = w;
            h.md_phat_t[((size_t)k * L + i) * 2 + 1] = shoup(w, qi);
        }
    }
    // conversion factors times the first forward stage's twiddle (pair 1 of
    // the target prime's forward table)
    auto w0 = [&](int l) { return h.tw[(size_t)l * 4 * N + 2]; };
    h.modup_modw.assign(h.modup_mod.size(), 0);
    for (size_t at = 0; at < h.modup_mod.size(); at += 2) {
        const int l = (int)((at / 2) % LK);
        const uint64_t ql = h.q[l], v = mulm(h.modup_mod[at], w0(l), ql);
        h.modup_modw[at] = v;
        h.modup_modw[at + 1] = shoup(v, ql);
    }
    h.md_phat_tw.assign(h.md_phat_t.size(), 0);
    for (size_t at = 0; at < h.md_phat_t.size(); at += 2) {
        const int i = (int)((at / 2) % L);
        const uint64_t qi = h.q[i], v = mulm(h.md_phat_t[at], w0(i), qi);
        h.md_phat_tw[at] = v;
        h.md_phat_tw[at + 1] = shoup(v, qi);
    }
    if (bfv && !bfv_tables(p, h, err)) return false;
    // batching slot positions
    h.slot_idx.resize(N);
    uint64_t e = 1;
    for (uint64_t j = 0; j < N / 2; ++j) {
        h.slot_idx[j] = (int32_t)ntt_index_of_exponent(e, p.log2n);
        h.slot_idx[N / 2 + j] = (int32_t)ntt_index_of_exponent(twoN - e, p.log2n);
        e = e * 5 % twoN;
    }
    return true;
}

}  // namespace hespmv
