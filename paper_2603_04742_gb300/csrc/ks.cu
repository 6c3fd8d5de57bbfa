// Fused hybrid key switching (N >= 2^11).
//
// For n polynomials d (NTT domain over Q) and a key [dnum][2][L+K][N] held in
// Montgomery form, seven launches compute
//   out_c = (sum_j ModUp_j(d) * key_j,c  -  delta_c) * P^-1  (+ addend),
//   delta_c = t * Conv_{P->Q}([x_c * t^-1]_P),  x_c the P-limbs of the sum:
//  1. inverse NTT of d, row pass                         (d -> dc)
//     (with HE-Mult fused in, d = a1 * b1 is formed here, in step 4 and the
//     addend (a0 b0, a0 b1 + a1 b0) in step 7: no tensor in memory)
//  2. inverse NTT column pass, N^-1 * Qhat^-1 folded in  (dc -> z)
//  3. ModUp + forward column pass: one CTA raises a digit's z columns to
//     every other prime and transforms them                 (z -> ext)
//  4. forward row pass of the raised limbs, in place             (ext)
//     and the inner product with the key: the digit's own primes use d
//     directly; 128-bit sums, one Montgomery reduction           (-> acc)
//  5. inverse NTT of acc's P limbs, t^-1 * Phat^-1 * N^-1 folded in (-> y)
//  6. ModDown conversion (t folded in) + forward column pass   (y -> dh)
//  7. forward row pass of delta + (acc - delta) * P^-1 + addend  (-> out)
// Scratch per item (words): L*N (dc, z) + dnum*(L+K)*N (ext) + 2*(L+K)*N
// (acc) + 2*L*N (dh).
#include "kernels.h"
#include "ntt_core.cuh"

namespace hespmv {

struct KsArgs {
    const ModConst *mc;
    const uint64_t *tw;        // [modulus][4][N]
    const uint64_t *zc;        // [L][4]  fold constants of step 2
    const uint64_t *yc;        // [K][4]  fold constants of step 5
    const uint64_t *modup_mod; // [dnum][alpha][L+K][2]
    const uint64_t *phat_t;    // [K][L][2]  Phat_k * t mod q_i
    const uint64_t *pinv;      // [L][2]
    int log2n, L, K, dnum, alpha;
};

// Input of a key switch: d (NTT domain, item stride ds), or, fused with the
// tensor product of HE-Mult, d = a1 * b1 for ciphertexts a = ta + i*ts,
// b = tb + i*ts, whose (a0 b0, a0 b1 + a1 b0) is then the addend.
struct KsSrc {
    const uint64_t *d;
    int64_t ds;
    const uint64_t *ta, *tb;
    int64_t ts;
};

__device__ __forceinline__ uint64_t src_d2(const KsSrc &s, const ModConst &mc, int64_t item,
                                           int64_t off, int64_t LN) {
    if (s.d) return s.d[item * s.ds + off];
    return mul_mod(s.ta[item * s.ts + LN + off], s.tb[item * s.ts + LN + off], mc);
}

__device__ __forceinline__ uint64_t redc(uint64_t hi, uint64_t lo, uint64_t q, uint64_t qneg) {
    const uint64_t m = lo * qneg;
    uint64_t r = hi + __umul64hi(m, q) + (lo != 0);
    return r >= q ? r - q : r;
}

// inverse row pass: src (item stride ss, limb k at +k*N) -> dst (stride ds)
template <int LR>
__global__ __launch_bounds__(kNttThreads) void k_ks_intt_rows(KsArgs a, const uint64_t *src,
                                                              int64_t ss, uint64_t *dst,
                                                              int64_t ds, int nl, int prime0) {
    constexpr int M = 1 << LR, TR = kNttTile / M, P = M / 8;
    __shared__ uint64_t sm[kRowTileWords];
    const int N = 1 << a.log2n, n1 = a.log2n - LR;
    const int item = blockIdx.y / nl, k = blockIdx.y - item * nl, prime = prime0 + k;
    const uint64_t q = a.mc[prime].q;
    const TwPair *itw = (const TwPair *)(a.tw + (int64_t)prime * 4 * N + 2 * N);
    const int t = threadIdx.x, rr = t / P, j = t % P, row = blockIdx.x * TR + rr;
    const uint64_t *in = src + item * ss + (int64_t)k * N + (int64_t)row * M;
    uint64_t *out = dst + item * ds + (int64_t)k * N + (int64_t)row * M;
    uint64_t v[8];
    load8(v, in + 8 * j);  // = Pass<LR>::last(j, e)
    inv_body<LR, false>(v, j, (1u << n1) + row, sm, RowIdx<M>{rr}, itw, q);
#pragma unroll
    for (int e = 0; e < 8; ++e) out[Pass<LR>::first(j, e)] = v[e];
}

// first inverse row pass of the key switch: from the input (or a1 * b1)
template <int LR>
__global__ __launch_bounds__(kNttThreads) void k_ks_intt_rows_src(KsArgs a, KsSrc s, uint64_t *dst) {
    constexpr int M = 1 << LR, TR = kNttTile / M, P = M / 8;
    __shared__ uint64_t sm[kRowTileWords];
    const int N = 1 << a.log2n, n1 = a.log2n - LR, L = a.L;
    const int item = blockIdx.y / L, k = blockIdx.y - item * L;
    const ModConst mc = a.mc[k];
    const TwPair *itw = (const TwPair *)(a.tw + (int64_t)k * 4 * N + 2 * N);
    const int t = threadIdx.x, rr = t / P, j = t % P, row = blockIdx.x * TR + rr;
    const int64_t off = (int64_t)k * N + (int64_t)row * M, LN = (int64_t)L * N;
    uint64_t v[8];
    if (s.d) {
        load8(v, s.d + item * s.ds + off + 8 * j);
    } else {  // d2 = a1 * b1
        uint64_t x[8], y[8];
        load8(x, s.ta + item * s.ts + LN + off + 8 * j);
        load8(y, s.tb + item * s.ts + LN + off + 8 * j);
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = mul_mod(x[e], y[e], mc);
    }
    inv_body<LR, false>(v, j, (1u << n1) + row, sm, RowIdx<M>{rr}, itw, mc.q);
    uint64_t *out = dst + (int64_t)item * LN + off;
#pragma unroll
    for (int e = 0; e < 8; ++e) out[Pass<LR>::first(j, e)] = v[e];
}

// inverse column pass in place with per-limb fold constants fc[k][4]
template <int LC>
__global__ __launch_bounds__(kNttThreads) void k_ks_intt_cols(KsArgs a, uint64_t *x, int64_t is,
                                                              int nl, int prime0,
                                                              const uint64_t *fc) {
    constexpr int M = 1 << LC, TC = kNttTile / M;
    __shared__ uint64_t sm[kNttTile];
    const int N = 1 << a.log2n, C = N >> LC;
    const int item = blockIdx.y / nl, k = blockIdx.y - item * nl, prime = prime0 + k;
    const uint64_t q = a.mc[prime].q;
    const TwPair *itw = (const TwPair *)(a.tw + (int64_t)prime * 4 * N + 2 * N);
    const int t = threadIdx.x, cc = t % TC, j = t / TC;
    uint64_t *col = x + item * is + (int64_t)k * N + blockIdx.x * TC + cc;
    const uint64_t *f = fc + 4 * k;
    uint64_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = col[(int64_t)Pass<LC>::last(j, e) * C];
    inv_body<LC, true>(v, j, 1, sm, ColIdx<TC>{cc}, itw, q, f[0], f[1], f[2], f[3]);
#pragma unroll
    for (int e = 0; e < 8; ++e) col[(int64_t)Pass<LC>::first(j, e) * C] = v[e];
}

// ModUp of digit jd to every prime outside it, fused with the forward column
// pass: z [n][L][N] -> ext [n][dnum][L+K][N] (column-pass output, [0, 4q))
template <int LC>
__global__ __launch_bounds__(kNttThreads) void k_ks_modup_cols(KsArgs a, const uint64_t *z,
                                                               uint64_t *ext) {
    constexpr int M = 1 << LC, TC = kNttTile / M;
    __shared__ uint64_t sm[kNttTile];
    const int N = 1 << a.log2n, C = N >> LC, L = a.L, LK = a.L + a.K;
    const int item = blockIdx.y / a.dnum, jd = blockIdx.y - item * a.dnum;
    const int i0 = jd * a.alpha, i1 = min(L, i0 + a.alpha), na = i1 - i0;
    const int t = threadIdx.x, cc = t % TC, j = t / TC;
    const int64_t cofs = blockIdx.x * TC + cc;
    uint64_t zs[4][8];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        if (s < na) {
            const uint64_t *src = z + ((int64_t)item * L + i0 + s) * N + cofs;
#pragma unroll
            for (int e = 0; e < 8; ++e) zs[s][e] = src[(int64_t)Pass<LC>::first(j, e) * C];
        }
    }
    uint64_t *dst0 = ext + ((int64_t)item * a.dnum + jd) * LK * N + cofs;
    for (int l = 0; l < LK; ++l) {
        if (l >= i0 && l < i1) continue;
        const uint64_t q = a.mc[l].q, q2 = 2 * q;
        const TwPair *tw = (const TwPair *)(a.tw + (int64_t)l * 4 * N);
        uint64_t v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = 0;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (s < na) {
                const uint64_t *cst = a.modup_mod + (((int64_t)jd * a.alpha + s) * LK + l) * 2;
                const uint64_t w = cst[0], ws = cst[1];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    uint64_t x = v[e] + mul_shoup_lazy(zs[s][e], w, ws, q);
                    v[e] = x >= q2 ? x - q2 : x;
                }
            }
        }
        fwd_body<LC>(v, j, 1, sm, ColIdx<TC>{cc}, tw, q);
        uint64_t *dst = dst0 + (int64_t)l * N;
#pragma unroll
        for (int e = 0; e < 8; ++e) dst[(int64_t)Pass<LC>::last(j, e) * C] = v[e];
    }
}

// Forward row pass, in place, of every raised limb: ext[item][jd][l] for the
// primes l outside digit jd (output unreduced, < 32q).
template <int LR>
__global__ __launch_bounds__(kNttThreads) void k_ks_rows_fwd(KsArgs a, uint64_t *ext) {
    constexpr int M = 1 << LR, TR = kNttTile / M, P = M / 8;
    __shared__ uint64_t sm[kRowTileWords];
    const int N = 1 << a.log2n, n1 = a.log2n - LR, LK = a.L + a.K;
    const int l = blockIdx.y % LK, jd = (blockIdx.y / LK) % a.dnum;
    const int64_t item = blockIdx.y / (LK * a.dnum);
    const int i0 = jd * a.alpha, i1 = min(a.L, i0 + a.alpha);
    if (l >= i0 && l < i1) return;  // the digit's own primes keep d itself
    const uint64_t q = a.mc[l].q;
    const TwPair *tw = (const TwPair *)(a.tw + (int64_t)l * 4 * N);
    const int t = threadIdx.x, rr = t / P, j = t % P, row = blockIdx.x * TR + rr;
    uint64_t *x = ext + ((item * a.dnum + jd) * LK + l) * N + (int64_t)row * M;
    uint64_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = x[Pass<LR>::first(j, e)];
    fwd_body<LR>(v, j, (1u << n1) + row, sm, RowIdx<M>{rr}, tw, q);
    store8(x + 8 * j, v);
}

// Inner product with the key: acc[item][c][l] = sum_j e_j * key[j][c][l]
// with e_j = ext[item][j][l] (< 32q) or, on digit j's own primes, d itself.
// Keys are in Montgomery form, so the 128-bit sum needs one reduction.
// Items vary fastest so a key limb stays in L2 while every item uses it.
__global__ __launch_bounds__(256) void k_ks_mac(KsArgs a, KsSrc s, const uint64_t *ext,
                                                const uint64_t *key, uint64_t *acc, int n) {
    // grid: x = coefficient pairs, y = l * n + item
    const int N = 1 << a.log2n, LK = a.L + a.K;
    const int l = blockIdx.y / n;
    const int64_t item = blockIdx.y - (int64_t)l * n;
    const int64_t k = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (k >= N) return;
    const ModConst mc = a.mc[l];
    uint64_t h0a = 0, l0a = 0, h0b = 0, l0b = 0, h1a = 0, l1a = 0, h1b = 0, l1b = 0;
    for (int jd = 0; jd < a.dnum; ++jd) {
        const int i0 = jd * a.alpha, i1 = min(a.L, i0 + a.alpha);
        ulonglong2 e;
        if (l >= i0 && l < i1) {
            if (s.d) {
                e = *(const ulonglong2 *)(s.d + item * s.ds + (int64_t)l * N + k);
            } else {
                const int64_t o = item * s.ts + ((int64_t)a.L + l) * N + k;
                const ulonglong2 x = *(const ulonglong2 *)(s.ta + o), y = *(const ulonglong2 *)(s.tb + o);
                e = make_ulonglong2(mul_mod(x.x, y.x, mc), mul_mod(x.y, y.y, mc));
            }
        } else {
            e = *(const ulonglong2 *)(ext + ((item * a.dnum + jd) * LK + l) * N + k);
        }
        const ulonglong2 w0 = __ldg((const ulonglong2 *)(key + ((int64_t)(2 * jd) * LK + l) * N + k));
        const ulonglong2 w1 = __ldg((const ulonglong2 *)(key + ((int64_t)(2 * jd + 1) * LK + l) * N + k));
        uint64_t p;
        p = e.x * w0.x; l0a += p; h0a += __umul64hi(e.x, w0.x) + (l0a < p);
        p = e.y * w0.y; l0b += p; h0b += __umul64hi(e.y, w0.y) + (l0b < p);
        p = e.x * w1.x; l1a += p; h1a += __umul64hi(e.x, w1.x) + (l1a < p);
        p = e.y * w1.y; l1b += p; h1b += __umul64hi(e.y, w1.y) + (l1b < p);
    }
    uint64_t *o0 = acc + (item * 2 * LK + l) * N + k;
    uint64_t *o1 = o0 + (int64_t)LK * N;
    *(ulonglong2 *)o0 = make_ulonglong2(redc(h0a, l0a, mc.q, mc.qneg), redc(h0b, l0b, mc.q, mc.qneg));
    *(ulonglong2 *)o1 = make_ulonglong2(redc(h1a, l1a, mc.q, mc.qneg), redc(h1b, l1b, mc.q, mc.qneg));
}

// ModDown conversion of y (P limbs of acc, coefficient domain) to each Q prime
// with t folded in, fused with the forward column pass: -> dh [n][2][L][N]
template <int LC>
__global__ __launch_bounds__(kNttThreads) void k_ks_moddown_cols(KsArgs a, const uint64_t *acc,
                                                                 uint64_t *dh) {
    constexpr int M = 1 << LC, TC = kNttTile / M;
    __shared__ uint64_t sm[kNttTile];
    const int N = 1 << a.log2n, C = N >> LC, L = a.L, K = a.K, LK = L + K;
    const int ic = blockIdx.y;  // item * 2 + component
    const int t = threadIdx.x, cc = t % TC, j = t / TC;
    const int64_t cofs = blockIdx.x * TC + cc;
    uint64_t ys[4][8];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        if (s < K) {
            const uint64_t *src = acc + ((int64_t)ic * LK + L + s) * N + cofs;
#pragma unroll
            for (int e = 0; e < 8; ++e) ys[s][e] = src[(int64_t)Pass<LC>::first(j, e) * C];
        }
    }
    for (int i = 0; i < L; ++i) {
        const uint64_t q = a.mc[i].q, q2 = 2 * q;
        const TwPair *tw = (const TwPair *)(a.tw + (int64_t)i * 4 * N);
        uint64_t v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = 0;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (s < K) {
                const uint64_t w = a.phat_t[((int64_t)s * L + i) * 2];
                const uint64_t ws = a.phat_t[((int64_t)s * L + i) * 2 + 1];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    uint64_t x = v[e] + mul_shoup_lazy(ys[s][e], w, ws, q);
                    v[e] = x >= q2 ? x - q2 : x;
                }
            }
        }
        fwd_body<LC>(v, j, 1, sm, ColIdx<TC>{cc}, tw, q);
        uint64_t *dst = dh + ((int64_t)ic * L + i) * N + cofs;
#pragma unroll
        for (int e = 0; e < 8; ++e) dst[(int64_t)Pass<LC>::last(j, e) * C] = v[e];
    }
}

// Forward row pass of delta, then out = (acc - delta) * P^-1 (+ addend).
template <int LR>
__global__ __launch_bounds__(kNttThreads) void k_ks_rows_final(KsArgs a, const uint64_t *acc,
                                                               const uint64_t *dh,
                                                               const uint64_t *add, int64_t add_is,
                                                               int64_t add_cs, int add_mask,
                                                               KsSrc s, uint64_t *out) {
    constexpr int M = 1 << LR, TR = kNttTile / M, P = M / 8;
    __shared__ uint64_t sm[kRowTileWords];
    const int N = 1 << a.log2n, n1 = a.log2n - LR, L = a.L, LK = L + a.K;
    const int ic = blockIdx.y / L, i = blockIdx.y - ic * L;
    const int item = ic >> 1, c = ic & 1;
    const ModConst mc = a.mc[i];
    const uint64_t q = mc.q;
    const TwPair *tw = (const TwPair *)(a.tw + (int64_t)i * 4 * N);
    const int t = threadIdx.x, rr = t / P, j = t % P, row = blockIdx.x * TR + rr;
    const int64_t rofs = (int64_t)row * M;
    const uint64_t *src = dh + ((int64_t)ic * L + i) * N + rofs;
    const uint64_t *x = acc + ((int64_t)ic * LK + i) * N + rofs;
    const bool has_add = add && ((add_mask >> c) & 1);
    const uint64_t *ad = has_add ? add + item * add_is + c * add_cs + (int64_t)i * N + rofs : nullptr;
    // operands of the epilogue, fetched before the transform
    uint64_t xa[8], xd[8];
    const bool tensor = s.ta != nullptr;
    const int64_t LN = (int64_t)L * N, toff = item * s.ts + (int64_t)i * N + rofs;
    load8(xa, x + 8 * j);
    if (tensor) {  // d0 = a0 b0, d1 = a0 b1 + a1 b0
        uint64_t a0[8], b0[8];
        load8(a0, s.ta + toff + 8 * j);
        load8(b0, s.tb + toff + 8 * j);
        if (c == 0) {
#pragma unroll
            for (int e = 0; e < 8; ++e) xd[e] = mul_mod(a0[e], b0[e], mc);
        } else {
            uint64_t a1[8], b1[8];
            load8(a1, s.ta + toff + LN + 8 * j);
            load8(b1, s.tb + toff + LN + 8 * j);
#pragma unroll
            for (int e = 0; e < 8; ++e)
                xd[e] = add_mod(mul_mod(a0[e], b1[e], mc), mul_mod(a1[e], b0[e], mc), q);
        }
    } else if (has_add) {
        load8(xd, ad + 8 * j);
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) xd[e] = 0;
    }
    uint64_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = src[Pass<LR>::first(j, e)];
    fwd_body<LR>(v, j, (1u << n1) + row, sm, RowIdx<M>{rr}, tw, q);
    const uint64_t w = a.pinv[2 * i], ws = a.pinv[2 * i + 1];
    uint64_t *o = out + ((int64_t)ic * L + i) * N + rofs;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        // delta < 32q unreduced: (acc + 32q - delta) * P^-1, fully reduced
        const uint64_t r = mul_shoup(xa[e] + 32 * q - v[e], w, ws, q);
        v[e] = add_mod(r, xd[e], q);
    }
    store8(o + 8 * j, v);
}

template <int LC, int LR>
static cudaError_t ks_fused(const Ctx &c, const KsArgs &a, const KsSrc &s, const uint64_t *key,
                            uint64_t *out, const uint64_t *add, int64_t add_is, int64_t add_cs,
                            int add_mask, int n, uint64_t *scratch, cudaStream_t st) {
    const int64_t N = c.N, L = c.L, K = c.K, LK = L + K;
    uint64_t *z = scratch;
    uint64_t *ext = z + n * L * N;
    uint64_t *acc = ext + n * c.dnum * LK * N;
    uint64_t *dh = acc + n * 2 * LK * N;
    const int gc = (int)((N >> LC) / (kNttTile >> LC)), gr = (int)((N >> LR) / (kNttTile >> LR));
    int r;
    r = prof_begin(c, "k_ks_intt_rows", st);
    k_ks_intt_rows_src<LR><<<dim3(gr, n * L), kNttThreads, 0, st>>>(a, s, z);
    prof_end(c, r, st);
    r = prof_begin(c, "k_ks_intt_cols", st);
    k_ks_intt_cols<LC><<<dim3(gc, n * L), kNttThreads, 0, st>>>(a, z, L * N, (int)L, 0, a.zc);
    prof_end(c, r, st);
    r = prof_begin(c, "k_ks_modup_cols", st);
    k_ks_modup_cols<LC><<<dim3(gc, n * c.dnum), kNttThreads, 0, st>>>(a, z, ext);
    prof_end(c, r, st);
    r = prof_begin(c, "k_ks_rows_fwd", st);
    k_ks_rows_fwd<LR><<<dim3(gr, n * c.dnum * LK), kNttThreads, 0, st>>>(a, ext);
    prof_end(c, r, st);
    r = prof_begin(c, "k_ks_mac", st);
    k_ks_mac<<<dim3((unsigned)((N / 2 + 255) / 256), (unsigned)(n * LK)), 256, 0, st>>>(a, s, ext, key, acc, n);
    prof_end(c, r, st);
    r = prof_begin(c, "k_ks_intt_rows", st);
    k_ks_intt_rows<LR><<<dim3(gr, n * 2 * K), kNttThreads, 0, st>>>(a, acc + L * N, LK * N,
                                                                    acc + L * N, LK * N, (int)K,
                                                                    (int)L);
    prof_end(c, r, st);
    r = prof_begin(c, "k_ks_intt_cols", st);
    k_ks_intt_cols<LC><<<dim3(gc, n * 2 * K), kNttThreads, 0, st>>>(a, acc + L * N, LK * N,
                                                                     (int)K, (int)L, a.yc);
    prof_end(c, r, st);
    r = prof_begin(c, "k_ks_moddown_cols", st);
    k_ks_moddown_cols<LC><<<dim3(gc, n * 2), kNttThreads, 0, st>>>(a, acc, dh);
    prof_end(c, r, st);
    r = prof_begin(c, "k_ks_rows_final", st);
    k_ks_rows_final<LR><<<dim3(gr, n * 2 * L), kNttThreads, 0, st>>>(a, acc, dh, add, add_is,
                                                                      add_cs, add_mask, s, out);
    prof_end(c, r, st);
    return cudaGetLastError();
}

bool ks_fused_supported(const Ctx &c) {
    return c.log2n >= 11 && c.log2n <= 15 && c.alpha <= 4 && c.K <= 4;
}

static cudaError_t ks_dispatch(const Ctx &c, const KsArgs &a, const KsSrc &s, const uint64_t *key,
                               uint64_t *out, const uint64_t *add, int64_t add_is, int64_t add_cs,
                               int add_mask, int m, uint64_t *scratch, cudaStream_t st) {
    switch (c.log2n) {
        case 15: return ks_fused<7, 8>(c, a, s, key, out, add, add_is, add_cs, add_mask, m, scratch, st);
        case 14: return ks_fused<7, 7>(c, a, s, key, out, add, add_is, add_cs, add_mask, m, scratch, st);
        case 13: return ks_fused<6, 7>(c, a, s, key, out, add, add_is, add_cs, add_mask, m, scratch, st);
        case 12: return ks_fused<6, 6>(c, a, s, key, out, add, add_is, add_cs, add_mask, m, scratch, st);
        case 11: return ks_fused<5, 6>(c, a, s, key, out, add, add_is, add_cs, add_mask, m, scratch, st);
        default: return cudaErrorInvalidValue;
    }
}

static KsArgs ks_args(const Ctx &c) {
    const hespmv_ctx *h = c.c;
    KsArgs a;
    a.mc = h->d.mc;
    a.tw = h->d.tw;
    a.zc = h->d.ks_zc;
    a.yc = h->d.ks_yc;
    a.modup_mod = h->d.modup_mod;
    a.phat_t = h->d.md_phat_t;
    a.pinv = h->d.md_pinv;
    a.log2n = c.log2n;
    a.L = c.L;
    a.K = c.K;
    a.dnum = c.dnum;
    a.alpha = c.alpha;
    return a;
}

// grid.y of the widest launch is n * dnum * (L+K): items per launch
static size_t ks_max_items(const Ctx &c) {
    return 65535 / ((size_t)std::max(2, c.dnum) * (c.L + c.K));
}

cudaError_t keyswitch_fused(const Ctx &c, const uint64_t *d, int64_t d_stride, const uint64_t *key,
                            uint64_t *out, const uint64_t *add, int64_t add_is, int64_t add_cs,
                            int add_mask, size_t n, uint64_t *scratch, cudaStream_t st) {
    const KsArgs a = ks_args(c);
    const size_t maxn = ks_max_items(c);
    for (size_t i0 = 0; i0 < n; i0 += maxn) {
        const int m = (int)std::min(maxn, n - i0);
        KsSrc s{d + i0 * d_stride, d_stride, nullptr, nullptr, 0};
        cudaError_t e = ks_dispatch(c, a, s, key, out + i0 * 2 * c.L * c.N,
                                    add ? add + i0 * add_is : nullptr, add_is, add_cs, add_mask, m,
                                    scratch, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t relin_tensor_fused(const Ctx &c, const uint64_t *A, const uint64_t *B,
                               const uint64_t *rlk, uint64_t *out, size_t n, uint64_t *scratch,
                               cudaStream_t st) {
    const KsArgs a = ks_args(c);
    const int64_t CT = 2 * (int64_t)c.L * c.N;
    const size_t maxn = ks_max_items(c);
    for (size_t i0 = 0; i0 < n; i0 += maxn) {
        const int m = (int)std::min(maxn, n - i0);
        KsSrc s{nullptr, 0, A + i0 * CT, B + i0 * CT, CT};
        cudaError_t e = ks_dispatch(c, a, s, rlk, out + i0 * CT, nullptr, 0, 0, 0, m, scratch, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace hespmv
