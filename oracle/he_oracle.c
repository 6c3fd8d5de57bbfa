/*
 * Oracle arithmetic kernels (TEST INFRASTRUCTURE ONLY).
 *
 * This file is part of the CPU oracle that the GPU library is checked
 * against.  Only the test suite, the package smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code with the GPU
 * library.  Every routine is written for clarity, not speed: each modular
 * product is an exact 128-bit product followed by the C `%` operator.
 *
 * Ring: R_q = Z_q[X]/(X^N + 1), N a power of two, q prime, q = 1 mod 2N.
 * The NTT convention follows the RLWE setting of the paper's HE layer
 * (Section 2.1): index i of the evaluation vector holds
 *     a(psi^(2*brv(i) + 1)) mod q,
 * brv = bit reversal on log2(N) bits, psi a primitive 2N-th root of unity.
 * It is computed here in the textbook way: twist by psi^j, a cyclic
 * length-N transform with omega = psi^2 (iterative radix-2 decimation in
 * time, bit-reversed input), then the outputs are placed in bit-reversed
 * order.  Parity of this routine is pinned in the tests against the O(N^2)
 * definition and against schoolbook negacyclic convolution.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a * (u128)b) % q);
}

static uint64_t powmod(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

static uint64_t bitrev(uint64_t x, int bits) {
    uint64_t r = 0;
    for (int b = 0; b < bits; b++) {
        r = (r << 1) | (x & 1);
        x >>= 1;
    }
    return r;
}

/* out[k] = a[k] * b[k] mod q, for any 64-bit inputs. */
void or_mulmod_vec(const uint64_t *a, const uint64_t *b, uint64_t *out,
                   int64_t n, uint64_t q) {
    for (int64_t k = 0; k < n; k++) out[k] = mulmod(a[k], b[k], q);
}

/* out[k] = a[k] * s mod q, for any 64-bit inputs. */
void or_mulmod_scalar(const uint64_t *a, uint64_t s, uint64_t *out,
                      int64_t n, uint64_t q) {
    for (int64_t k = 0; k < n; k++) out[k] = mulmod(a[k], s, q);
}

/* Cyclic transform in place: A[k] = sum_j A_in[j] * w^(j*k) mod q.
 * Textbook iterative radix-2 DIT: bit-reverse permutation, then butterflies
 * over blocks of length 2, 4, ..., n. */
static void cyclic_ntt(uint64_t *A, int logn, uint64_t w, uint64_t q) {
    int64_t n = (int64_t)1 << logn;
    for (int64_t i = 0; i < n; i++) {
        int64_t j = (int64_t)bitrev((uint64_t)i, logn);
        if (j > i) {
            uint64_t tmp = A[i];
            A[i] = A[j];
            A[j] = tmp;
        }
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
        uint64_t wlen = powmod(w, (uint64_t)(n / len), q);
        for (int64_t start = 0; start < n; start += len) {
            uint64_t wj = 1;
            for (int64_t j = 0; j < len / 2; j++) {
                uint64_t u = A[start + j];
                uint64_t v = mulmod(A[start + j + len / 2], wj, q);
                A[start + j] = (u + v) % q;
                A[start + j + len / 2] = (u + q - v) % q;
                wj = mulmod(wj, wlen, q);
            }
        }
    }
}

/* Forward negacyclic NTT in place: a -> [a(psi^(2 brv(i) + 1))]_i. */
void or_ntt_forward(uint64_t *a, int logn, uint64_t q, uint64_t psi) {
    int64_t n = (int64_t)1 << logn;
    uint64_t *b = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    uint64_t pj = 1;
    for (int64_t j = 0; j < n; j++) { /* twist: b_j = a_j psi^j */
        b[j] = mulmod(a[j] % q, pj, q);
        pj = mulmod(pj, psi, q);
    }
    /* b -> B[k] = sum_j b_j psi^(2jk) = a(psi^(2k+1)) */
    cyclic_ntt(b, logn, mulmod(psi, psi, q), q);
    for (int64_t i = 0; i < n; i++) a[i] = b[bitrev((uint64_t)i, logn)];
    free(b);
}

/* Inverse of or_ntt_forward, in place. */
void or_ntt_inverse(uint64_t *a, int logn, uint64_t q, uint64_t psi) {
    int64_t n = (int64_t)1 << logn;
    uint64_t *b = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    /* undo the output order: B[k] = a[brv(k)] */
    for (int64_t k = 0; k < n; k++) b[k] = a[bitrev((uint64_t)k, logn)] % q;
    /* inverse cyclic transform: b_j = n^-1 sum_k B[k] omega^(-jk) */
    uint64_t psi_inv = powmod(psi, q - 2, q);
    cyclic_ntt(b, logn, mulmod(psi_inv, psi_inv, q), q);
    uint64_t n_inv = powmod((uint64_t)n % q, q - 2, q);
    /* untwist: a_j = b_j psi^(-j) */
    uint64_t pj = 1;
    for (int64_t j = 0; j < n; j++) {
        a[j] = mulmod(mulmod(b[j], n_inv, q), pj, q);
        pj = mulmod(pj, psi_inv, q);
    }
    free(b);
}
