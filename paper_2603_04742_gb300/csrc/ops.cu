// Elementwise ciphertext kernels, the key-switching stages, samplers and the
// encode / decrypt helpers.  Grid-stride loops over flat word indices; every
// access is coalesced along the coefficient index.
#include "async_copy.cuh"
#include "kernels.h"

namespace hespmv {

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t n) {
    int64_t g = (n + kThreads - 1) / kThreads;
    if (g > 152 * 16) g = 152 * 16;  // grid-stride beyond 16 CTAs per SM
    return (int)(g < 1 ? 1 : g);
}

#define GRID_STRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__global__ void k_add(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t total, int log2n,
                      int L, const ModConst *mc) {
    GRID_STRIDE(i, total) {
        const int l = (int)((i >> log2n) % L);
        out[i] = add_mod(a[i], b[i], mc[l].q);
    }
}

__global__ void k_tensor(const uint64_t *a, const uint64_t *b, uint64_t *d, int64_t total,
                         int log2n, int L, const ModConst *mc) {
    // total = n * L * N (one thread per coefficient of each ciphertext limb)
    const int64_t LN = (int64_t)L << log2n;
    GRID_STRIDE(i, total) {
        const int64_t item = i / LN, r = i - item * LN;
        const int l = (int)(r >> log2n);
        const ModConst m = mc[l];
        const uint64_t *A = a + item * 2 * LN, *B = b + item * 2 * LN;
        const uint64_t a0 = A[r], a1 = A[LN + r], b0 = B[r], b1 = B[LN + r];
        uint64_t *D = d + item * 3 * LN;
        D[r] = mul_mod(a0, b0, m);
        D[LN + r] = add_mod(mul_mod(a0, b1, m), mul_mod(a1, b0, m), m.q);
        D[2 * LN + r] = mul_mod(a1, b1, m);
    }
}

__device__ __forceinline__ uint64_t mont_reduce(uint64_t hi, uint64_t lo, uint64_t q,
                                                uint64_t qneg) {
    const uint64_t m = lo * qneg;
    uint64_t r = hi + __umul64hi(m, q) + (lo != 0);
    return r >= q ? r - q : r;
}

// ct * pt with the plaintext in Montgomery form (mask plaintexts)
__global__ void k_cmult(const uint64_t *ct, const uint64_t *pt, uint64_t *out, int64_t total,
                        int log2n, int L, const ModConst *mc) {
    const int64_t LN = (int64_t)L << log2n;
    GRID_STRIDE(i, total) {
        const int64_t r = i % LN;
        const ModConst m = mc[(int)(r >> log2n)];
        const uint64_t a = ct[i], b = pt[r];
        out[i] = mont_reduce(__umul64hi(a, b), a * b, m.q, m.qneg);
    }
}

// the Montgomery reduction (times 2^-64 mod q) of an Acc3 below q 2^64
__device__ __forceinline__ uint64_t acc3_reduce(const Acc3 &c, const ModConst &m) {
    uint64_t hi, lo;
    fold3(c, hi, lo);
    return mont_reduce(hi, lo, m.q, m.qneg);
}

// out = sum_k w_k * mask_k over the nterms ciphertexts w_k = w0 + k * 2LN
// (Algorithm 4, inter-chunk aggregation); masks in Montgomery form, 128-bit
// sums reduced once per block of 4096 terms.  Each thread takes two
// consecutive words (16-byte loads); the block stages the mask addresses in
// shared memory, 256 at a time.  A streaming pass: every term word is read
// once (evict-first loads), the masks (few distinct, shared by all threads
// of a word) through the read-only path; four terms' loads are issued before
// their products so each thread keeps eight 16-byte loads in flight.
__global__ __launch_bounds__(256, 3) void k_mask_acc(const uint64_t *w0, const uint64_t *const *masks, int nterms,
                                                     uint64_t *out, int64_t total, int log2n, int L,
                                                     const ModConst *mc) {
    constexpr int U = 4;
    __shared__ const uint64_t *sm_masks[256];
    const int64_t LN = (int64_t)L << log2n, CT = 2 * LN;
    const int64_t i = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);  // total = 2LN, even
    const bool active = i < total;
    const int64_t r = active ? i % LN : 0;
    const ModConst m = mc[(int)(r >> log2n)];
    // terms and masks are residues below q < 2^50: three-column sums of up to
    // 4096 products, below 2^112 < q 2^64 for the Montgomery reduction
    uint64_t s0 = 0, s1 = 0;
    Acc3 c0, c1;
    for (int kb = 0; kb < nterms; kb += 256) {  // 256 divides the 4096-term reduction interval
        const int kn = min(256, nterms - kb);
        __syncthreads();
        if ((int)threadIdx.x < kn) sm_masks[threadIdx.x] = masks[kb + threadIdx.x];
        __syncthreads();
        if (!active) continue;
        const uint64_t *w = w0 + (int64_t)kb * CT + i;
        int k = 0;
        for (; k + U <= kn; k += U) {
            ulonglong2 a[U], b[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                a[u] = __ldcs((const ulonglong2 *)(w + (int64_t)(k + u) * CT));
                b[u] = __ldg((const ulonglong2 *)(sm_masks[k + u] + r));
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                mac3(c0, a[u].x, b[u].x);
                mac3(c1, a[u].y, b[u].y);
            }
        }
        for (; k < kn; ++k) {
            const ulonglong2 a = __ldcs((const ulonglong2 *)(w + (int64_t)k * CT));
            const ulonglong2 b = __ldg((const ulonglong2 *)(sm_masks[k] + r));
            mac3(c0, a.x, b.x);
            mac3(c1, a.y, b.y);
        }
        if (((kb + kn) & 4095) == 0) {  // 4096 terms: reduce
            s0 = add_mod(s0, acc3_reduce(c0, m), m.q);
            s1 = add_mod(s1, acc3_reduce(c1, m), m.q);
            c0 = Acc3{};
            c1 = Acc3{};
        }
    }
    if (!active) return;
    s0 = add_mod(s0, acc3_reduce(c0, m), m.q);
    s1 = add_mod(s1, acc3_reduce(c1, m), m.q);
    *(ulonglong2 *)(out + i) = make_ulonglong2(s0, s1);
}

// dst[di[s]] (=, +=) src[si[s]] (through the Galois permutation if perm),
// s < m whole ciphertexts; a null index list is the identity
__global__ void k_ct_move(uint64_t *dst, const int32_t *di, const uint64_t *src, const int32_t *si,
                          const int32_t *perm, int add, int64_t total, int log2n, int L,
                          const ModConst *mc) {
    const int64_t CT = (int64_t)2 * L << log2n;
    GRID_STRIDE(i, total) {
        const int64_t s = i / CT, w = i - s * CT;
        const int64_t ds = di ? di[s] : s, ss = si ? si[s] : s;
        const int64_t sw = perm ? ((w >> log2n) << log2n) + perm[w & ((1 << log2n) - 1)] : w;
        const uint64_t v = src[ss * CT + sw];
        uint64_t *o = dst + ds * CT + w;
        if (add) {
            const uint64_t q = mc[(w >> log2n) % L].q;
            *o = add_mod(*o, v, q);
        } else {
            *o = v;
        }
    }
}

__global__ void k_to_mont_limbs(uint64_t *x, int64_t total, int log2n, int prime0, int nl,
                                const ModConst *mc) {
    GRID_STRIDE(i, total) {
        const ModConst m = mc[prime0 + (int)((i >> log2n) % nl)];
        x[i] = mul_mod(x[i], m.rmod, m);
    }
}

__global__ void k_cmult_acc(uint64_t *acc, const uint64_t *w, const uint64_t *pt, int64_t total,
                            int log2n, int L, const ModConst *mc, int first) {
    const int64_t LN = (int64_t)L << log2n;
    GRID_STRIDE(i, total) {
        const int64_t r = i % LN;
        const int l = (int)(r >> log2n);
        const uint64_t v = mul_mod(w[i], pt[r], mc[l]);
        acc[i] = first ? v : add_mod(acc[i], v, mc[l].q);
    }
}

// prod = (a0 * x0, a0 * x1): ciphertext x times the plaintext a0 (HE-CMult)
__global__ void k_pt_ct_mul(const uint64_t *a, const uint64_t *x, uint64_t *prod, int64_t total,
                            int log2n, int L, const ModConst *mc) {
    const int64_t LN = (int64_t)L << log2n;
    GRID_STRIDE(i, total) {  // total = n * L * N
        const int64_t item = i / LN, r = i - item * LN;
        const ModConst m = mc[(int)(r >> log2n)];
        const uint64_t p = a[item * 2 * LN + r];
        prod[item * 2 * LN + r] = mul_mod(p, x[item * 2 * LN + r], m);
        prod[item * 2 * LN + LN + r] = mul_mod(p, x[item * 2 * LN + LN + r], m);
    }
}

__global__ void k_permute(const uint64_t *in, uint64_t *out, const int32_t *perm, int64_t total,
                          int log2n) {
    GRID_STRIDE(i, total) {
        const int64_t p = i >> log2n;
        const int64_t k = i & ((1 << log2n) - 1);
        out[i] = in[(p << log2n) + perm[k]];
    }
}

__global__ void k_mul_limbs(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t total,
                            int log2n, int prime0, int n_limbs, const ModConst *mc) {
    GRID_STRIDE(i, total) {
        const int l = prime0 + (int)((i >> log2n) % n_limbs);
        out[i] = mul_mod(a[i], b[i], mc[l]);
    }
}

__global__ void k_copy_strided(const uint64_t *src, int64_t ss, uint64_t *dst, int64_t ds,
                               int64_t words, int64_t total) {
    GRID_STRIDE(i, total) {
        const int64_t item = i / words, w = i - item * words;
        dst[item * ds + w] = src[item * ss + w];
    }
}

// ModUp: for item, digit j and coefficient k, raise the digit's residues to
// every prime of Q u P (fast base conversion, unsigned representatives).
// ext [n][dnum][L+K][N] (coefficient domain).
__global__ void k_modup(const uint64_t *dcoef, uint64_t *ext, int64_t total, int log2n, int L,
                        int K, int dnum, int alpha, const ModConst *mc, const uint64_t *inv,
                        const uint64_t *qmod) {
    const int N = 1 << log2n, LK = L + K;
    GRID_STRIDE(i, total) {  // total = n * dnum * N
        const int k = (int)(i & (N - 1));
        const int64_t r = i >> log2n;
        const int j = (int)(r % dnum);
        const int64_t item = r / dnum;
        const int i0 = j * alpha, i1 = min(L, (j + 1) * alpha);
        const uint64_t *X = dcoef + item * ((int64_t)L << log2n);
        uint64_t z[16];
        for (int s = i0; s < i1; ++s) {
            const uint64_t *c = inv + ((int64_t)j * alpha + (s - i0)) * 2;
            z[s - i0] = mul_shoup(X[((int64_t)s << log2n) + k], c[0], c[1], mc[s].q);
        }
        uint64_t *E = ext + (item * dnum + j) * ((int64_t)LK << log2n);
        for (int l = 0; l < LK; ++l) {
            uint64_t v;
            if (l >= i0 && l < i1) {
                v = X[((int64_t)l << log2n) + k];
            } else {
                const uint64_t ql = mc[l].q;
                v = 0;
                for (int s = i0; s < i1; ++s) {
                    const uint64_t *c = qmod + (((int64_t)j * alpha + (s - i0)) * LK + l) * 2;
                    v = add_mod(v, mul_shoup(z[s - i0], c[0], c[1], ql), ql);
                }
            }
            E[((int64_t)l << log2n) + k] = v;
        }
    }
}

// acc[c][l] = sum_j ext[j][l] * key[j][c][l]; the key is in Montgomery form,
// so one reduction of the 128-bit sum gives the plain residue
__global__ void k_inner(const uint64_t *ext, const uint64_t *key, uint64_t *acc, int64_t total,
                        int log2n, int L, int K, int dnum, const ModConst *mc) {
    const int LK = L + K;
    const int64_t LKN = (int64_t)LK << log2n;
    GRID_STRIDE(i, total) {  // total = n * LK * N
        const int64_t item = i / LKN, r = i - item * LKN;
        const int l = (int)(r >> log2n);
        const ModConst m = mc[l];
        uint64_t h0 = 0, l0 = 0, h1 = 0, l1 = 0;
        for (int j = 0; j < dnum; ++j) {
            const uint64_t e = ext[(item * dnum + j) * LKN + r];
            const uint64_t w0 = key[(int64_t)(2 * j) * LKN + r], w1 = key[(int64_t)(2 * j + 1) * LKN + r];
            uint64_t lo = e * w0;
            l0 += lo;
            h0 += __umul64hi(e, w0) + (l0 < lo);
            lo = e * w1;
            l1 += lo;
            h1 += __umul64hi(e, w1) + (l1 < lo);
        }
        acc[(item * 2) * LKN + r] = mont_reduce(h0, l0, m.q, m.qneg);
        acc[(item * 2 + 1) * LKN + r] = mont_reduce(h1, l1, m.q, m.qneg);
    }
}

__global__ void k_to_mont(uint64_t *x, int64_t total, int log2n, int LK, const ModConst *mc) {
    GRID_STRIDE(i, total) {
        const ModConst m = mc[(i >> log2n) % LK];
        x[i] = mul_mod(x[i], m.rmod, m);
    }
}

// ModDown, first half: from the special-prime residues (coefficient domain)
// y_k = x_k * t^-1 * Phat_k^-1 mod p_k, delta_i = t * sum_k y_k * Phat_k mod q_i.
__global__ void k_moddown_delta(const uint64_t *acc, uint64_t *delta, int64_t total, int log2n,
                                int L, int K, const ModConst *mc, const uint64_t *md_pk,
                                const uint64_t *md_phat, const uint64_t *md_t) {
    const int LK = L + K;
    const int N = 1 << log2n;
    GRID_STRIDE(i, total) {  // total = n * 2 * N
        const int k = (int)(i & (N - 1));
        const int64_t ic = i >> log2n;  // item*2 + c
        const uint64_t *A = acc + ic * ((int64_t)LK << log2n);
        uint64_t y[4];
        for (int s = 0; s < K; ++s)
            y[s] = mul_shoup(A[((int64_t)(L + s) << log2n) + k], md_pk[2 * s], md_pk[2 * s + 1],
                             mc[L + s].q);
        uint64_t *D = delta + ic * ((int64_t)L << log2n);
        for (int l = 0; l < L; ++l) {
            const uint64_t ql = mc[l].q;
            uint64_t v = 0;
            for (int s = 0; s < K; ++s) {
                const uint64_t *c = md_phat + ((int64_t)s * L + l) * 2;
                v = add_mod(v, mul_shoup(y[s], c[0], c[1], ql), ql);
            }
            D[((int64_t)l << log2n) + k] = mul_shoup(v, md_t[2 * l], md_t[2 * l + 1], ql);
        }
    }
}

__global__ void k_moddown_final(const uint64_t *acc, const uint64_t *delta, const uint64_t *add,
                                int64_t add_is, int64_t add_cs, int add_mask, uint64_t *out,
                                int64_t total, int log2n, int L, int K, const ModConst *mc,
                                const uint64_t *md_pinv) {
    const int LK = L + K;
    const int64_t LN = (int64_t)L << log2n;
    GRID_STRIDE(i, total) {  // total = n * 2 * L * N
        const int64_t ic = i / LN, r = i - ic * LN;
        const int64_t item = ic >> 1;
        const int c = (int)(ic & 1);
        const int l = (int)(r >> log2n);
        const uint64_t q = mc[l].q;
        const uint64_t x = acc[ic * ((int64_t)LK << log2n) + r];
        uint64_t v = mul_shoup(sub_mod(x, delta[i], q), md_pinv[2 * l], md_pinv[2 * l + 1], q);
        if (add && ((add_mask >> c) & 1)) v = add_mod(v, add[item * add_is + c * add_cs + r], q);
        out[i] = v;
    }
}

__global__ void k_sample_signed(uint64_t seed, uint64_t stream0, uint64_t step, int kind,
                                int64_t *out, int64_t total, int log2n) {
    GRID_STRIDE(i, total) {
        const int64_t item = i >> log2n;
        const int64_t k = i & ((1 << log2n) - 1);
        const uint64_t key = splitmix_at(seed, stream0 + (uint64_t)item * step);
        const uint64_t r = splitmix_at(key, (uint64_t)k);
        int64_t v;
        if (kind == kTernary) {
            v = (int64_t)(r % 3ull) - 1;
        } else {
            v = (int64_t)__popcll(r & 0x1FFFFFull) - (int64_t)__popcll((r >> 21) & 0x1FFFFFull);
        }
        out[i] = v;
    }
}

__global__ void k_signed_to_limbs(const int64_t *coef, uint64_t *out, int64_t total, int log2n,
                                  int prime0, int n_limbs, const ModConst *mc) {
    GRID_STRIDE(i, total) {  // total = n_items * n_limbs * N
        const int64_t k = i & ((1 << log2n) - 1);
        const int64_t r = i >> log2n;
        const int64_t item = r / n_limbs;
        const int l = prime0 + (int)(r - item * n_limbs);
        const uint64_t q = mc[l].q;
        const int64_t v = coef[(item << log2n) + k];
        out[i] = v >= 0 ? (uint64_t)v % q : q - ((uint64_t)(-v) % q == 0 ? q : (uint64_t)(-v) % q);
    }
}

__global__ void k_sample_uniform(uint64_t key, uint64_t *out, int64_t total, int log2n, int prime0,
                                 const ModConst *mc) {
    GRID_STRIDE(i, total) {  // total = n_limbs * N; limb-local counter i
        const int l = prime0 + (int)(i >> log2n);
        const ModConst m = mc[l];
        const uint64_t hi = splitmix_at(key, 2 * (uint64_t)i) % m.q;
        const uint64_t lo = splitmix_at(key, 2 * (uint64_t)i + 1) % m.q;
        // (hi * 2^64 + lo) mod q with 2^64 mod q = (2^64 - q) mod q
        const uint64_t two64 = (0ull - m.q) % m.q;
        out[i] = add_mod(mul_mod(hi, two64, m), lo, m.q);
    }
}

__global__ void k_ksk_combine(const uint64_t *a, const uint64_t *e, const uint64_t *s,
                              const uint64_t *sp, uint64_t *b, int64_t total, int log2n, int L,
                              int i0, int i1, const ModConst *mc, const uint64_t *t_mod,
                              const uint64_t *p_mod_q) {
    GRID_STRIDE(i, total) {  // total = (L+K) * N
        const int l = (int)(i >> log2n);
        const ModConst m = mc[l];
        uint64_t v = sub_mod(mul_mod(e[i], t_mod[l], m), mul_mod(a[i], s[i], m), m.q);
        if (l >= i0 && l < i1) v = add_mod(v, mul_mod(sp[i], p_mod_q[2 * l], m), m.q);
        b[i] = v;
    }
}

__global__ void k_pk_combine(const uint64_t *a, const uint64_t *e, const uint64_t *s, uint64_t *pk0,
                             int64_t total, int log2n, const ModConst *mc, const uint64_t *t_mod) {
    GRID_STRIDE(i, total) {  // total = L * N
        const int l = (int)(i >> log2n);
        const ModConst m = mc[l];
        pk0[i] = sub_mod(mul_mod(e[i], t_mod[l], m), mul_mod(a[i], s[i], m), m.q);
    }
}

__global__ void k_enc_combine(const uint64_t *u, const uint64_t *e0, const uint64_t *e1,
                              const uint64_t *msg, const uint64_t *pk, uint64_t *ct, int64_t total,
                              int log2n, int L, const ModConst *mc, const uint64_t *t_mod) {
    const int64_t LN = (int64_t)L << log2n;
    GRID_STRIDE(i, total) {  // total = n * L * N
        const int64_t item = i / LN, r = i - item * LN;
        const int l = (int)(r >> log2n);
        const ModConst m = mc[l];
        const uint64_t uu = u[i];
        uint64_t c0 = add_mod(mul_mod(uu, pk[r], m), mul_mod(e0[i], t_mod[l], m), m.q);
        c0 = add_mod(c0, msg[i], m.q);
        const uint64_t c1 = add_mod(mul_mod(uu, pk[LN + r], m), mul_mod(e1[i], t_mod[l], m), m.q);
        ct[item * 2 * LN + r] = c0;
        ct[item * 2 * LN + LN + r] = c1;
    }
}

__global__ void k_scatter_slots(const int64_t *vals, int64_t nvals, uint64_t *E, int64_t total,
                                int log2n, const int32_t *slot_idx, uint64_t t) {
    const int N = 1 << log2n;
    GRID_STRIDE(i, total) {  // total = n * N, j = slot number (row 0: j < N/2)
        const int64_t item = i >> log2n;
        const int j = (int)(i & (N - 1));
        uint64_t v = 0;
        if (j < N / 2 && j < nvals) {
            const int64_t x = vals[item * nvals + j];
            const uint64_t r = (uint64_t)(x >= 0 ? x : -x) % t;
            v = (x >= 0 || r == 0) ? r : t - r;
        }
        E[(item << log2n) + slot_idx[j]] = v;
    }
}

__global__ void k_lift(const uint64_t *msg, uint64_t *out, int64_t total, int log2n, int L,
                       const ModConst *mc, uint64_t t) {
    const int64_t LN = (int64_t)L << log2n;
    GRID_STRIDE(i, total) {  // total = n * L * N
        const int64_t item = i / LN, r = i - item * LN;
        const int l = (int)(r >> log2n);
        const int64_t k = r & ((1 << log2n) - 1);
        const uint64_t q = mc[l].q;
        const uint64_t v = msg[(item << log2n) + k];
        // centred representative of v mod t, reduced mod q_l (t < q_l)
        out[i] = (2 * v <= t) ? v : q - (t - v);
    }
}

__global__ void k_dec_phase(const uint64_t *ct, const uint64_t *s, uint64_t *x, int64_t total,
                            int log2n, int L, const ModConst *mc) {
    const int64_t LN = (int64_t)L << log2n;
    GRID_STRIDE(i, total) {  // total = L * N
        const int l = (int)(i >> log2n);
        x[i] = add_mod(ct[i], mul_mod(ct[LN + i], s[i], mc[l]), mc[l].q);
    }
}

__global__ void k_crt_to_t(const uint64_t *x, uint64_t *msg, int N, int log2n, int L,
                           const ModConst *mc, const uint64_t *dec, const double *inv_q,
                           uint64_t t) {
    GRID_STRIDE(k, (int64_t)N) {
        double frac = 0.0;
        uint64_t acc = 0;
        for (int l = 0; l < L; ++l) {
            const uint64_t y = mul_shoup(x[((int64_t)l << log2n) + k], dec[4 * l], dec[4 * l + 1],
                                         mc[l].q);
            frac += (double)y * inv_q[l];
            acc = add_mod(acc, mul_shoup(y, dec[4 * l + 2], dec[4 * l + 3], t), t);
        }
        // sum_l y_l Qhat_l = x + v Q with v = round(frac) for the centred x
        const uint64_t v = (uint64_t)llrint(frac);
        const uint64_t vq = mul_shoup(v, dec[4 * L], dec[4 * L + 1], t);
        msg[k] = sub_mod(acc, vq, t);
    }
}

__global__ void k_gather_slots(const uint64_t *E, uint64_t *slots, int N, const int32_t *slot_idx) {
    GRID_STRIDE(j, (int64_t)N) { slots[j] = E[slot_idx[j]]; }
}

// CKKS rescale, step 2: x [2n][N] holds the last limb of every component in
// coefficient form ([0, ql)); y [2n][nl1][N] receives its centred value
// (x - ql when x > ql / 2) reduced mod q_i for i < nl1
__global__ void k_rescale_lift(const uint64_t *x, uint64_t *y, int64_t total, int log2n, int nl1, uint64_t ql,
                               const ModConst *mc) {
    const int64_t N = (int64_t)1 << log2n;
    GRID_STRIDE(j, total) {  // total = 2n * nl1 * N
        const int64_t ic = j / (nl1 * N), rem = j - ic * nl1 * N;
        const int i = (int)(rem >> log2n);
        const uint64_t v = x[ic * N + (rem & (N - 1))], qi = mc[i].q;
        uint64_t r;
        if (v > ql / 2) {  // negative representative v - ql
            const uint64_t m = (ql - v) % qi;
            r = m ? qi - m : 0;
        } else {
            r = v % qi;
        }
        y[j] = r;
    }
}

// CKKS rescale, step 4: out[ic][i] = (ct[ic][i] - y[ic][i]) * ql^-1 mod q_i,
// out [2n][nl1][N]; ct has nl1 + 1 limbs per component; qinv [nl1][2] holds
// ql^-1 mod q_i with its Shoup companion
__global__ void k_rescale_final(const uint64_t *ct, const uint64_t *y, uint64_t *out, int64_t total, int log2n,
                                int nl1, const uint64_t *qinv, const ModConst *mc) {
    const int64_t N = (int64_t)1 << log2n;
    GRID_STRIDE(j, total) {
        const int64_t ic = j / (nl1 * N), rem = j - ic * nl1 * N;
        const int i = (int)(rem >> log2n);
        const uint64_t q = mc[i].q, c = ct[ic * (nl1 + 1) * N + rem], v = y[j];
        out[j] = mul_shoup(c >= v ? c - v : c + q - v, qinv[2 * i], qinv[2 * i + 1], q);
    }
}

}  // namespace

#define LAUNCH(kern, total, st, ...)                                  \
    do {                                                              \
        const int64_t _t = (total);                                   \
        if (_t > 0) {                                                 \
            const int _r = prof_begin(c, #kern, st);                  \
            kern<<<grid_for(_t), kThreads, 0, st>>>(__VA_ARGS__);     \
            prof_end(c, _r, st);                                      \
        }                                                             \
        return cudaGetLastError();                                    \
    } while (0)

cudaError_t op_add(const Ctx &c, const uint64_t *a, const uint64_t *b, uint64_t *out,
                   size_t n_polys, cudaStream_t st) {
    const int64_t total = (int64_t)n_polys * c.L * c.N;
    LAUNCH(k_add, total, st, a, b, out, total, c.log2n, c.L, c.c->d.mc);
}

cudaError_t op_tensor(const Ctx &c, const uint64_t *a, const uint64_t *b, uint64_t *d, size_t n,
                      cudaStream_t st) {
    const int64_t total = (int64_t)n * c.L * c.N;
    LAUNCH(k_tensor, total, st, a, b, d, total, c.log2n, c.L, c.c->d.mc);
}

cudaError_t op_pt_ct_mul(const Ctx &c, const uint64_t *a, const uint64_t *x, uint64_t *prod,
                         size_t n, cudaStream_t st) {
    const int64_t total = (int64_t)n * c.L * c.N;
    LAUNCH(k_pt_ct_mul, total, st, a, x, prod, total, c.log2n, c.L, c.c->d.mc);
}

cudaError_t op_cmult(const Ctx &c, const uint64_t *ct, const uint64_t *pt, uint64_t *out, size_t n,
                     cudaStream_t st) {
    const int64_t total = (int64_t)n * 2 * c.L * c.N;
    LAUNCH(k_cmult, total, st, ct, pt, out, total, c.log2n, c.L, c.c->d.mc);
}

cudaError_t op_mask_acc(const Ctx &c, const uint64_t *w0, const uint64_t *const *masks,
                        int nterms, uint64_t *out, cudaStream_t st) {
    const int64_t total = (int64_t)2 * c.L * c.N;  // words; one thread per two
    const int r = prof_begin(c, "k_mask_acc", st);
    k_mask_acc<<<(unsigned)((total / 2 + 255) / 256), 256, 0, st>>>(w0, masks, nterms, out, total, c.log2n, c.L,
                                                                    c.c->d.mc);
    prof_end(c, r, st);
    return cudaGetLastError();
}

cudaError_t op_ct_move(const Ctx &c, uint64_t *dst, const int32_t *di, const uint64_t *src,
                       const int32_t *si, const int32_t *perm, bool add, int m, cudaStream_t st) {
    const int64_t total = (int64_t)m * 2 * c.L * c.N;
    LAUNCH(k_ct_move, total, st, dst, di, src, si, perm, add ? 1 : 0, total, c.log2n, c.L,
           c.c->d.mc);
}

cudaError_t op_to_mont_limbs(const Ctx &c, uint64_t *x, int prime0, int n_limbs, size_t n_items,
                             cudaStream_t st) {
    const int64_t total = (int64_t)n_items * n_limbs * c.N;
    LAUNCH(k_to_mont_limbs, total, st, x, total, c.log2n, prime0, n_limbs, c.c->d.mc);
}

cudaError_t op_cmult_acc(const Ctx &c, uint64_t *acc, const uint64_t *w, const uint64_t *pt,
                         bool first, cudaStream_t st) {
    const int64_t total = (int64_t)2 * c.L * c.N;
    LAUNCH(k_cmult_acc, total, st, acc, w, pt, total, c.log2n, c.L, c.c->d.mc, first ? 1 : 0);
}

cudaError_t op_permute(const Ctx &c, const uint64_t *in, uint64_t *out, const int32_t *perm,
                       size_t n_limbs_total, cudaStream_t st) {
    const int64_t total = (int64_t)n_limbs_total * c.N;
    LAUNCH(k_permute, total, st, in, out, perm, total, c.log2n);
}

cudaError_t op_mul_limbs(const Ctx &c, const uint64_t *a, const uint64_t *b, uint64_t *out,
                         int prime0, int n_limbs, size_t n_items, cudaStream_t st) {
    const int64_t total = (int64_t)n_items * n_limbs * c.N;
    LAUNCH(k_mul_limbs, total, st, a, b, out, total, c.log2n, prime0, n_limbs, c.c->d.mc);
}

cudaError_t op_copy_strided(const Ctx &c, const uint64_t *src, int64_t src_stride, uint64_t *dst,
                            int64_t dst_stride, int64_t words, size_t n_items, cudaStream_t st) {
    const int64_t total = words * (int64_t)n_items;
    LAUNCH(k_copy_strided, total, st, src, src_stride, dst, dst_stride, words, total);
}

cudaError_t op_to_mont(const Ctx &c, uint64_t *x, size_t n_items, cudaStream_t st) {
    const int64_t total = (int64_t)n_items * (c.L + c.K) * c.N;
    LAUNCH(k_to_mont, total, st, x, total, c.log2n, c.L + c.K, c.c->d.mc);
}

cudaError_t op_modup(const Ctx &c, const uint64_t *dcoef, uint64_t *ext, size_t n, cudaStream_t st) {
    const int64_t total = (int64_t)n * c.dnum * c.N;
    LAUNCH(k_modup, total, st, dcoef, ext, total, c.log2n, c.L, c.K, c.dnum, c.alpha, c.c->d.mc,
           c.c->d.modup_inv, c.c->d.modup_mod);
}

cudaError_t op_inner(const Ctx &c, const uint64_t *ext, const uint64_t *key, uint64_t *acc, size_t n,
                     cudaStream_t st) {
    const int64_t total = (int64_t)n * (c.L + c.K) * c.N;
    LAUNCH(k_inner, total, st, ext, key, acc, total, c.log2n, c.L, c.K, c.dnum, c.c->d.mc);
}

cudaError_t op_moddown_delta(const Ctx &c, const uint64_t *acc, uint64_t *delta, size_t n,
                             cudaStream_t st) {
    const int64_t total = (int64_t)n * 2 * c.N;
    LAUNCH(k_moddown_delta, total, st, acc, delta, total, c.log2n, c.L, c.K, c.c->d.mc,
           c.c->d.md_pk, c.c->d.md_phat, c.c->d.md_t);
}

cudaError_t op_moddown_final(const Ctx &c, const uint64_t *acc, const uint64_t *delta,
                             const uint64_t *add, int64_t add_item_stride, int64_t add_comp_stride,
                             int add_mask, uint64_t *out, size_t n, cudaStream_t st) {
    const int64_t total = (int64_t)n * 2 * c.L * c.N;
    LAUNCH(k_moddown_final, total, st, acc, delta, add, add_item_stride, add_comp_stride, add_mask,
           out, total, c.log2n, c.L, c.K, c.c->d.mc, c.c->d.md_pinv);
}

cudaError_t op_sample_signed(const Ctx &c, uint64_t seed, uint64_t stream0, uint64_t step, int kind,
                             int64_t *out, size_t n_items, cudaStream_t st) {
    const int64_t total = (int64_t)n_items * c.N;
    LAUNCH(k_sample_signed, total, st, seed, stream0, step, kind, out, total, c.log2n);
}

cudaError_t op_signed_to_limbs(const Ctx &c, const int64_t *coef, uint64_t *out, int prime0,
                               int n_limbs, size_t n_items, cudaStream_t st) {
    const int64_t total = (int64_t)n_items * n_limbs * c.N;
    LAUNCH(k_signed_to_limbs, total, st, coef, out, total, c.log2n, prime0, n_limbs, c.c->d.mc);
}

cudaError_t op_sample_uniform(const Ctx &c, uint64_t seed, uint64_t stream, uint64_t *out,
                              int prime0, int n_limbs, cudaStream_t st) {
    const int64_t total = (int64_t)n_limbs * c.N;
    // stream key = SplitMix64(seed).output[stream], computed like the device helper
    uint64_t z = seed + (stream + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    const uint64_t key = z ^ (z >> 31);
    LAUNCH(k_sample_uniform, total, st, key, out, total, c.log2n, prime0, c.c->d.mc);
}

cudaError_t op_ksk_combine(const Ctx &c, const uint64_t *a, const uint64_t *e, const uint64_t *s,
                           const uint64_t *sp, int digit, uint64_t *b, cudaStream_t st) {
    const int64_t total = (int64_t)(c.L + c.K) * c.N;
    const int i0 = digit * c.alpha, i1 = std::min(c.L, (digit + 1) * c.alpha);
    LAUNCH(k_ksk_combine, total, st, a, e, s, sp, b, total, c.log2n, c.L, i0, i1, c.c->d.mc,
           c.c->d.t_mod, c.c->d.p_mod_q);
}

cudaError_t op_pk_combine(const Ctx &c, const uint64_t *a, const uint64_t *e, const uint64_t *s,
                          uint64_t *pk0, cudaStream_t st) {
    const int64_t total = (int64_t)c.L * c.N;
    LAUNCH(k_pk_combine, total, st, a, e, s, pk0, total, c.log2n, c.c->d.mc, c.c->d.t_mod);
}

cudaError_t op_enc_combine(const Ctx &c, const uint64_t *u, const uint64_t *e0, const uint64_t *e1,
                           const uint64_t *m, const uint64_t *pk, uint64_t *ct, size_t n,
                           cudaStream_t st) {
    const int64_t total = (int64_t)n * c.L * c.N;
    LAUNCH(k_enc_combine, total, st, u, e0, e1, m, pk, ct, total, c.log2n, c.L, c.c->d.mc,
           c.c->d.t_mod);
}

cudaError_t op_scatter_slots(const Ctx &c, const int64_t *vals, int64_t nvals, uint64_t *E,
                             size_t n, cudaStream_t st) {
    const int64_t total = (int64_t)n * c.N;
    LAUNCH(k_scatter_slots, total, st, vals, nvals, E, total, c.log2n, c.c->d.slot_idx, c.c->h.t);
}

cudaError_t op_lift(const Ctx &c, const uint64_t *m, uint64_t *out, size_t n, cudaStream_t st) {
    const int64_t total = (int64_t)n * c.L * c.N;
    LAUNCH(k_lift, total, st, m, out, total, c.log2n, c.L, c.c->d.mc, c.c->h.t);
}

cudaError_t op_dec_phase(const Ctx &c, const uint64_t *ct, const uint64_t *s, uint64_t *x,
                         cudaStream_t st) {
    const int64_t total = (int64_t)c.L * c.N;
    LAUNCH(k_dec_phase, total, st, ct, s, x, total, c.log2n, c.L, c.c->d.mc);
}

cudaError_t op_rescale_lift(const Ctx &c, const uint64_t *x, uint64_t *y, size_t n_comp, int nl1, uint64_t ql,
                            cudaStream_t st) {
    const int64_t total = (int64_t)n_comp * nl1 * c.N;
    LAUNCH(k_rescale_lift, total, st, x, y, total, c.log2n, nl1, ql, c.c->d.mc);
}

cudaError_t op_rescale_final(const Ctx &c, const uint64_t *ct, const uint64_t *y, uint64_t *out, size_t n_comp,
                             int nl1, const uint64_t *qinv, cudaStream_t st) {
    const int64_t total = (int64_t)n_comp * nl1 * c.N;
    LAUNCH(k_rescale_final, total, st, ct, y, out, total, c.log2n, nl1, qinv, c.c->d.mc);
}

cudaError_t op_crt_to_t(const Ctx &c, const uint64_t *x, uint64_t *m, cudaStream_t st) {
    LAUNCH(k_crt_to_t, (int64_t)c.N, st, x, m, c.N, c.log2n, c.L, c.c->d.mc, c.c->d.dec,
           c.c->d.dec_inv_q, c.c->h.t);
}

cudaError_t op_gather_slots(const Ctx &c, const uint64_t *E, uint64_t *slots, cudaStream_t st) {
    LAUNCH(k_gather_slots, (int64_t)c.N, st, E, slots, c.N, c.c->d.slot_idx);
}

// Self-test of the bounded waits: a barrier that expects 16 bytes no copy
// ever delivers; every thread's wait runs out after a few polls and the
// device error word is set.  Nothing faults and nothing is left in flight.
__global__ void k_wait_probe(int *err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], 16;" ::"r"(smem_u32(&bar)) : "memory");
    }
    __syncthreads();
    mbar_wait(&bar, 0, 1024, err);
}

// a table of device addresses from launch parameters
constexpr int kPtrBatch = 256;
struct PtrBatch {
    const uint64_t *p[kPtrBatch];
};
__global__ void k_write_ptrs(const uint64_t **dst, PtrBatch b, int n) {
    if ((int)threadIdx.x < n) dst[threadIdx.x] = b.p[threadIdx.x];
}

cudaError_t op_write_ptrs(const Ctx &c, const uint64_t **dst, const std::vector<const uint64_t *> &ptrs,
                          cudaStream_t st) {
    for (size_t i0 = 0; i0 < ptrs.size(); i0 += kPtrBatch) {
        const int n = (int)std::min<size_t>(kPtrBatch, ptrs.size() - i0);
        PtrBatch b{};
        for (int i = 0; i < n; ++i) b.p[i] = ptrs[i0 + i];
        const int r = prof_begin(c, "k_write_ptrs", st);
        k_write_ptrs<<<1, kPtrBatch, 0, st>>>(dst + i0, b, n);
        prof_end(c, r, st);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t op_wait_probe(const Ctx &c, cudaStream_t st) {
    k_wait_probe<<<1, 32, 0, st>>>(c.c->d.err);
    return cudaGetLastError();
}

// Packed ciphertext limbs (W bits per residue, little-endian bit string per
// limb of limb_words words) -> u64 residues, one thread per residue; two
// arrays per launch (blockIdx.y).  The second word is read only when the
// residue crosses into it, which stays inside the limb.  A residue not below
// its prime is stored reduced and flagged in the device error word.
__global__ void k_ct_unpack(const uint64_t *pa, uint64_t *oa, const uint64_t *pb, uint64_t *ob,
                            int64_t total, int log2n, int L, int W, int64_t limb_words,
                            const ModConst *mc, int *err) {
    const uint64_t *in = blockIdx.y ? pb : pa;
    uint64_t *out = blockIdx.y ? ob : oa;
    const uint64_t mask = W == 64 ? ~0ull : (1ull << W) - 1;
    const int64_t nmask = (1LL << log2n) - 1;
    GRID_STRIDE(i, total) {
        const int64_t limb = i >> log2n, bit = (i & nmask) * W;
        const uint64_t *src = in + limb * limb_words + (bit >> 6);
        const int sh = (int)(bit & 63);
        uint64_t v = src[0] >> sh;
        if (sh + W > 64) v |= src[1] << (64 - sh);
        v &= mask;
        const uint64_t q = mc[limb % L].q;
        if (v >= q) {
            v %= q;
            atomicExch(err, kErrBadResidue);
        }
        out[i] = v;
    }
}

// u64 residues (each below 2^W) -> packed limbs, one thread per output word:
// the residues whose bits meet word w of a limb are those with
// k W < 64 w + 64 and k W + W > 64 w.
__global__ void k_ct_pack(const uint64_t *in, uint64_t *out, int64_t total_words, int log2n, int W,
                          int64_t limb_words) {
    const int64_t N = 1LL << log2n;
    GRID_STRIDE(i, total_words) {
        const int64_t limb = i / limb_words, b0 = (i - limb * limb_words) * 64;
        const uint64_t *src = in + (limb << log2n);
        int64_t k1 = (b0 + 64 + W - 1) / W;
        if (k1 > N) k1 = N;
        uint64_t word = 0;
        for (int64_t k = b0 / W; k < k1; ++k) {
            const int64_t sh = k * W - b0;  // in (-W, 64)
            word |= sh >= 0 ? src[k] << sh : src[k] >> -sh;
        }
        out[i] = word;
    }
}

cudaError_t op_ct_unpack(const Ctx &c, const uint64_t *pa, uint64_t *oa, const uint64_t *pb, uint64_t *ob,
                         size_t n, cudaStream_t st) {
    const int64_t total = (int64_t)n * 2 * c.L * c.N;
    if (total == 0) return cudaSuccess;
    const int W = c.c->h.pack_bits;
    const int64_t lw = ((int64_t)c.N * W + 63) / 64;
    const int r = prof_begin(c, "k_ct_unpack", st);
    k_ct_unpack<<<dim3(grid_for(total), pb ? 2 : 1), kThreads, 0, st>>>(pa, oa, pb, ob, total, c.log2n, c.L,
                                                                         W, lw, c.c->d.mc, c.c->d.err);
    prof_end(c, r, st);
    return cudaGetLastError();
}

cudaError_t op_ct_pack(const Ctx &c, const uint64_t *in, uint64_t *out, size_t n, cudaStream_t st) {
    const int W = c.c->h.pack_bits;
    const int64_t lw = ((int64_t)c.N * W + 63) / 64, total = (int64_t)n * 2 * c.L * lw;
    if (total == 0) return cudaSuccess;
    const int r = prof_begin(c, "k_ct_pack", st);
    k_ct_pack<<<grid_for(total), kThreads, 0, st>>>(in, out, total, c.log2n, W, lw);
    prof_end(c, r, st);
    return cudaGetLastError();
}

}  // namespace hespmv
