// Device modular arithmetic for word-size primes (q < 2^62; the contexts use
// primes below 2^50 and a plaintext modulus t below 2^50).
#pragma once
#include <cstdint>

namespace hespmv {

// Per-modulus constants, resident in device memory.
struct ModConst {
    uint64_t q;
    uint64_t mu;      // Barrett: floor(2^(2k) / q)
    uint64_t ninv;    // N^-1 mod q
    uint64_t ninv_s;  // Shoup companion of ninv
    uint64_t w1ninv;  // psi^-1 * N^-1 mod q (last inverse butterfly)
    uint64_t w1ninv_s;
    int32_t k;        // bit length of q
    int32_t bs;       // max(0, 2k - 64): shift of the quotient estimate of mul_mod
    uint64_t qneg;    // -q^-1 mod 2^64 (Montgomery reduction)
    uint64_t rmod;    // 2^64 mod q (to Montgomery form)
    uint64_t one_s;   // floor(2^64 / q): Shoup companion of 1 (full reduction)
    uint64_t bmu;     // floor(2^(64 + bs) / q): quotient factor of mul_mod
};

#ifdef __CUDACC__
__device__ __forceinline__ uint64_t add_mod(uint64_t a, uint64_t b, uint64_t q) {
    uint64_t s = a + b;
    return s >= q ? s - q : s;
}

__device__ __forceinline__ uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t q) {
    return a >= b ? a - b : a + q - b;
}

// a * w mod q for a constant w < q with ws = floor(w * 2^64 / q); any a < 2^64.
// The quotient estimate is low by at most one, so one subtraction suffices.
__device__ __forceinline__ uint64_t mul_shoup(uint64_t a, uint64_t w, uint64_t ws, uint64_t q) {
    uint64_t qh = __umul64hi(a, ws);
    uint64_t r = a * w - qh * q;
    return r >= q ? r - q : r;
}

// Same, result left in [0, 2q).
__device__ __forceinline__ uint64_t mul_shoup_lazy(uint64_t a, uint64_t w, uint64_t ws,
                                                   uint64_t q) {
    uint64_t qh = __umul64hi(a, ws);
    return a * w - qh * q;
}

// Same, with the quotient estimated from three of the four 32 x 32-bit partial
// products of a * ws (the low-by-low product and the low halves of the cross
// products are dropped): the estimate is low by at most three, so the result
// is in [0, 4q).  For q < 2^50 and any a < 2^64.
__device__ __forceinline__ uint64_t mul_shoup_lazy4(uint64_t a, uint64_t w, uint64_t ws,
                                                    uint64_t q) {
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
    const uint32_t s0 = (uint32_t)ws, s1 = (uint32_t)(ws >> 32);
    const uint64_t qh = (uint64_t)a1 * s1 + __umulhi(a1, s0) + __umulhi(a0, s1);
    return a * w - qh * q;
}

// Barrett reduction of a 128-bit value x = hi:lo < 2^(2k), q of k bits:
// q1 = x >> (k-1), q3 = (q1 * mu) >> (k+1), r = x - q3 q in [0, 3q).
__device__ __forceinline__ uint64_t barrett_reduce(uint64_t hi, uint64_t lo, uint64_t q,
                                                   uint64_t mu, int k) {
    uint64_t q1 = (hi << (65 - k)) | (lo >> (k - 1));
    uint64_t plo = q1 * mu;
    uint64_t phi = __umul64hi(q1, mu);
    uint64_t q3 = (phi << (63 - k)) | (plo >> (k + 1));
    uint64_t r = lo - q3 * q;
    if (r >= q) r -= q;
    if (r >= q) r -= q;
    return r;
}

// a * b = hi:lo from its four 32 x 32 -> 64-bit partial products (any a, b):
// the middle sums cannot overflow (each is below 2^64 - 2^32).
__device__ __forceinline__ void mul_wide(uint64_t a, uint64_t b, uint64_t &hi, uint64_t &lo) {
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32), b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
    const uint64_t p00 = (uint64_t)a0 * b0;
    const uint64_t mid = (uint64_t)a0 * b1 + (p00 >> 32);
    const uint64_t mid2 = (uint64_t)a1 * b0 + (uint32_t)mid;
    lo = (mid2 << 32) | (uint32_t)p00;
    hi = (uint64_t)a1 * b1 + (mid >> 32) + (mid2 >> 32);
}

// a * b mod q for a, b < q (any x = a b < 2^(2k), k the bit length of q <= 62).
// Barrett-style: x1 = x >> s (s = max(0, 2k - 64), so x1 < 2^64) times
// bmu = floor(2^(64+s) / q), high word, estimates floor(x / q) low by at most
// two (each floor costs less than one); dropping the low-by-low partial
// product of that high word costs at most one more, so x - estimate * q,
// taken mod 2^64, is in [0, 4q).
__device__ __forceinline__ uint64_t mul_mod(uint64_t a, uint64_t b, const ModConst &m) {
    uint64_t hi, lo;
    mul_wide(a, b, hi, lo);
    const uint64_t x1 = m.bs ? (hi << (64 - m.bs)) | (lo >> m.bs) : lo;
    const uint32_t x0 = (uint32_t)x1, x1h = (uint32_t)(x1 >> 32);
    const uint32_t u0 = (uint32_t)m.bmu, u1 = (uint32_t)(m.bmu >> 32);
    const uint64_t mid = (uint64_t)x0 * u1;
    const uint64_t mid2 = (uint64_t)x1h * u0 + (uint32_t)mid;
    const uint64_t qe = (uint64_t)x1h * u1 + (mid >> 32) + (mid2 >> 32);
    uint64_t r = lo - qe * m.q;
    r = r >= 2 * m.q ? r - 2 * m.q : r;
    return r >= m.q ? r - m.q : r;
}

// SplitMix64 (Steele, Lea, Flood 2014): output i of the generator with
// state s is mix(s + (i + 1) * gamma).
__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t splitmix_at(uint64_t state, uint64_t i) {
    return splitmix_mix(state + (i + 1) * 0x9E3779B97F4A7C15ull);
}

// A sum of products a * b kept as its three 32-bit partial-product columns:
// value = s0 + 2^32 sm + 2^64 sh.  Each product costs four 32 x 32 -> 64-bit
// multiplies.  The column sums cannot overflow while the middle terms
// a0 b1 + a1 b0 of all products (plus 2^32 per carry out of s0) stay below
// 2^64: e.g. at most 64 products with a < 2^57, b < 2^51 (< 2^58 each), or
// 4096 products with a, b < 2^50 (< 2^51 each).
struct Acc3 {
    uint64_t s0 = 0, sm = 0, sh = 0;
};
__device__ __forceinline__ void mac3(Acc3 &c, uint64_t a, uint64_t b) {
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32), b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
    const uint64_t p0 = (uint64_t)a0 * b0;
    c.s0 += p0;
    c.sm += (uint64_t)a0 * b1 + (uint64_t)a1 * b0 + ((uint64_t)(c.s0 < p0) << 32);
    c.sh += (uint64_t)a1 * b1;
}
// the 128-bit value hi:lo of an Acc3
__device__ __forceinline__ void fold3(const Acc3 &c, uint64_t &hi, uint64_t &lo) {
    lo = c.s0 + (c.sm << 32);
    hi = c.sh + (c.sm >> 32) + (lo < c.s0);
}

__device__ __forceinline__ uint64_t redc(uint64_t hi, uint64_t lo, uint64_t q, uint64_t qneg) {
    const uint64_t m = lo * qneg;
    uint64_t r = hi + __umul64hi(m, q) + (lo != 0);
    return r >= q ? r - q : r;
}

#endif  // __CUDACC__

}  // namespace hespmv
