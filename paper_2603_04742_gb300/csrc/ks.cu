// Fused hybrid key switching (N >= 2^11).
//
// For n polynomials d (NTT domain over Q) and a key [dnum][2][L+K][N] held in
// Montgomery form, seven launches compute
//   out_c = (sum_j ModUp_j(d) * key_j,c  -  delta_c) * P^-1  (+ addend),
//   delta_c = t * Conv_{P->Q}([x_c * t^-1]_P),  x_c the P-limbs of the sum:
//  1. inverse NTT of d, row pass                         (d -> dc)
//     (with HE-Mult fused in, d = a1 * b1 is formed here and in step 4, and
//     the addend (a0 b0, a0 b1 + a1 b0) in step 4: no tensor in memory)
//  2. ModUp: one CTA takes a digit's column tiles through the inverse
//     column pass (N^-1 * Qhat^-1 folded in), raises them to every other
//     prime and runs those primes' forward column pass     (dc -> ext)
//  4. forward row pass of the raised limbs, in place             (ext)
//     and the inner product with the key: the digit's own primes use d
//     directly; the addend enters on the Q primes times P; 128-bit sums,
//     one Montgomery reduction                                     (-> acc)
//  5. inverse NTT row pass of acc's P limbs                         (-> y)
//  6. inverse column pass of y (t^-1 * Phat^-1 * N^-1 folded in), ModDown
//     conversion (t folded in) and forward column pass        (y -> dh)
//  7. forward row pass of delta, (acc - delta) * P^-1            (-> out)
// Scratch per item (words): L*N (dc, z) + dnum*(L+K)*N (ext) + 2*(L+K)*N
// (acc) + 2*L*N (dh).
#include <algorithm>

#include "async_copy.cuh"
#include "kernels.h"
#include "ntt_core.cuh"
#include "persist.h"

namespace hespmv {


// the HE-Mult operands of item i
__device__ __forceinline__ const uint64_t *src_a(const KsSrc &s, int64_t i) {
    return s.tap ? s.tap[i] : s.ta + i * s.ts;
}
__device__ __forceinline__ const uint64_t *src_b(const KsSrc &s, int64_t i) {
    return s.tbp ? s.tbp[i] : s.tb + i * s.ts;
}

// residue k of a packed limb; one not below q is reduced and flagged
__device__ __forceinline__ uint64_t packed_residue(const uint64_t *limb, int64_t k, int W, uint64_t q,
                                                   int *err) {
    const int64_t bit = k * W;
    const uint64_t *p = limb + (bit >> 6);
    const int sh = (int)(bit & 63);
    uint64_t v = p[0] >> sh;
    if (sh + W > 64) v |= p[1] << (64 - sh);
    v &= (1ull << W) - 1;  // W < 64
    if (v >= q) {
        v %= q;
        atomicExch(err, kErrBadResidue);
    }
    return v;
}

// (a b + c d) * 2^-64 mod q, left in [0, 2q) (a, b, c, d < q < 2^50, so
// the 128-bit sum stays below q * 2^64)
__device__ __forceinline__ uint64_t mont_lazy(uint64_t a, uint64_t b, uint64_t c, uint64_t d,
                                              const ModConst &m) {
    uint64_t lo = a * b, hi = __umul64hi(a, b);
    const uint64_t l2 = c * d;
    hi += __umul64hi(c, d);
    lo += l2;
    hi += lo < l2;
    const uint64_t t = lo * m.qneg;
    return hi + __umul64hi(t, m.q) + (lo != 0);
}

// Launch bounds: the row passes fit 48 registers (5 CTAs, 40 warps per SM)
// and the final row pass of 2^8 points 64 (4 CTAs) without spilling, which took 8 us off
// each of the forward and final row passes on the stencil ring; the
// conversion kernels and the key product stay at 3 CTAs per SM (at 64
// registers they spill and gain nothing).

// inverse row pass: src (item stride ss, limb k at +k*N) -> dst (stride ds);
// tile (bx, by): row block bx of limb by % nl of item by / nl
template <int LR>
__device__ __forceinline__ void ks_intt_rows_tile(const KsArgs &a, const uint64_t *src, int64_t ss,
                                                  uint64_t *dst, int64_t ds, int nl, int prime0, int bx,
                                                  int by, uint64_t *sm) {
    constexpr int M = 1 << LR, TR = kNttTile / M, P = M / 8;
    const int N = 1 << a.log2n, n1 = a.log2n - LR;
    const int item = by / nl, k = by - item * nl, prime = prime0 + k;
    const uint64_t q = a.mc[prime].q;
    const TwPair *itw = (const TwPair *)(a.tw + (int64_t)prime * 4 * N + 2 * N);
    const int t = threadIdx.x, rr = t / P, j = t % P, row = bx * TR + rr;
    const uint64_t *in = src + item * ss + (int64_t)k * N + (int64_t)row * M;
    uint64_t *out = dst + item * ds + (int64_t)k * N + (int64_t)row * M;
    uint64_t v[8];
    load8(v, in + 8 * j);  // = Pass<LR>::last(j, e)
    inv_body<LR, false>(v, j, (1u << n1) + row, sm, RowIdxW<M>(rr), itw, q);
#pragma unroll
    for (int e = 0; e < 8; ++e) out[Pass<LR>::first(j, e)] = v[e];
}

template <int LR>
__global__ __launch_bounds__(kNttThreads, 5) void k_ks_intt_rows(KsArgs a, const uint64_t *src,
                                                              int64_t ss, uint64_t *dst,
                                                              int64_t ds, int nl, int prime0) {
    __shared__ uint64_t sm[kRowTileWords];
    ks_intt_rows_tile<LR>(a, src, ss, dst, ds, nl, prime0, blockIdx.x, blockIdx.y, sm);
}

// first inverse row pass of the key switch: from the input (or a1 * b1)
template <int LR>
__device__ __forceinline__ void ks_intt_rows_src_tile(const KsArgs &a, const KsSrc &s, uint64_t *dst, int bx,
                                                      int by, uint64_t *sm) {
    constexpr int M = 1 << LR, TR = kNttTile / M, P = M / 8;
    const int N = 1 << a.log2n, n1 = a.log2n - LR, L = a.L;
    const int item = by / L, k = by - item * L;
    const ModConst mc = a.mc[k];
    const TwPair *itw = (const TwPair *)(a.tw + (int64_t)k * 4 * N + 2 * N);
    const int t = threadIdx.x, rr = t / P, j = t % P, row = bx * TR + rr;
    const int64_t off = (int64_t)k * N + (int64_t)row * M, LN = (int64_t)L * N;
    uint64_t v[8];
    if (s.d && s.perm) {  // rotation: d through the Galois permutation
        const uint64_t *base = s.d + (int64_t)(s.idx ? s.idx[item] : item) * s.ds + (int64_t)k * N;
        const int32_t *pm = s.perm + (int64_t)row * M + 8 * j;
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = base[pm[e]];
    } else if (s.d) {
        load8(v, s.d + (int64_t)(s.idx ? s.idx[item] : item) * s.ds + off + 8 * j);
    } else if (s.pk_bits) {  // d2 = a1 * b1 from packed operands
        const int64_t limb = (int64_t)(L + k) * s.pk_lw, c0 = (int64_t)row * M + 8 * j;
        const uint64_t *pa = src_a(s, item) + limb, *pb = src_b(s, item) + limb;
#pragma unroll
        for (int e = 0; e < 8; ++e)
            v[e] = mul_mod(packed_residue(pa, c0 + e, s.pk_bits, mc.q, a.err),
                           packed_residue(pb, c0 + e, s.pk_bits, mc.q, a.err), mc);
    } else {  // d2 = a1 * b1
        uint64_t x[8], y[8];
        load8(x, src_a(s, item) + LN + off + 8 * j);
        load8(y, src_b(s, item) + LN + off + 8 * j);
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = mul_mod(x[e], y[e], mc);
    }
    inv_body<LR, false>(v, j, (1u << n1) + row, sm, RowIdxW<M>(rr), itw, mc.q);
    uint64_t *out = dst + (int64_t)item * LN + off;
#pragma unroll
    for (int e = 0; e < 8; ++e) out[Pass<LR>::first(j, e)] = v[e];
}

template <int LR>
__global__ __launch_bounds__(kNttThreads) void k_ks_intt_rows_src(KsArgs a, KsSrc s, uint64_t *dst) {
    __shared__ uint64_t sm[kRowTileWords];
    ks_intt_rows_src_tile<LR>(a, s, dst, blockIdx.x, blockIdx.y, sm);
}

// ModUp of digit jd to every prime outside it, fused with the forward column
// pass: z [n][L][N] -> ext [n][dnum][L+K][N] (column-pass output, unreduced:
// conversion sums below 4 alpha q <= 16q, then 4q per stage)
// With nparts > 1 the digit's raised limbs are split into nparts ranges and
// this tile makes range `part` (each part redoes the digit's inverse pass):
// more CTAs for key switches of few ciphertexts.
template <int LC, int AMAX>
__device__ __forceinline__ void ks_modup_cols_tile(const KsArgs &a, const uint64_t *z, uint64_t *ext, int bx,
                                                   int by, uint64_t *sm, int part = 0, int nparts = 1) {
    constexpr int M = 1 << LC, TC = kNttTile / M;
    const int N = 1 << a.log2n, C = N >> LC, L = a.L, LK = a.L + a.K;
    const int item = by / a.dnum, jd = by - item * a.dnum;
    const int i0 = jd * a.alpha, i1 = min(L, i0 + a.alpha), na = i1 - i0;
    const int t = threadIdx.x, cc = t % TC, j = t / TC;
    const int64_t cofs = (int64_t)bx * TC + cc;
    // the digit's own limbs: inverse column pass of the row-pass output, with
    // N^-1 * Qhat^-1 folded in (coefficients of d times the ModUp factor)
    uint64_t zs[AMAX][8];
#pragma unroll
    for (int s = 0; s < AMAX; ++s) {
        if (s < na) {
            const int pi = i0 + s;
            const uint64_t *src = z + ((int64_t)item * L + pi) * N + cofs;
#pragma unroll
            for (int e = 0; e < 8; ++e) zs[s][e] = src[(int64_t)Pass<LC>::last(j, e) * C];
            const TwPair *itw = (const TwPair *)(a.tw + (int64_t)pi * 4 * N + 2 * N);
            const uint64_t *f = a.zc + 4 * pi;
            inv_body<LC, true>(zs[s], j, 1, sm, ColIdx<TC>{cc}, itw, a.mc[pi].q, f[0], f[1], f[2], f[3]);
        }
    }
    uint64_t *dst0 = ext + ((int64_t)item * a.dnum + jd) * LK * N + cofs;
    const int cnt = LK - na, e0 = part * cnt / nparts, e1 = (part + 1) * cnt / nparts;
    for (int e = e0; e < e1; ++e) {
        const int l = e < i0 ? e : e + na;  // the primes outside the digit, in order
        const uint64_t q = a.mc[l].q;
        const TwPair *tw = (const TwPair *)(a.tw + (int64_t)l * 4 * N);
        uint64_t v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = 0;
#pragma unroll
        for (int s = 0; s < AMAX; ++s) {
            if (s < na) {
                const int64_t at = (((int64_t)jd * a.alpha + s) * LK + l) * 2;
                const uint64_t w = a.modup_mod[at], ws = a.modup_mod[at + 1];
                const uint64_t ww = a.modup_modw[at], wws = a.modup_modw[at + 1];
#pragma unroll
                for (int e = 0; e < 4; ++e) v[e] += mul_shoup_lazy4(zs[s][e], w, ws, q);  // < 4q each
#pragma unroll
                for (int e = 4; e < 8; ++e) v[e] += mul_shoup_lazy4(zs[s][e], ww, wws, q);  // stage 0's w y
            }
        }
        fwd_body<LC, 4 * AMAX>(v, j, 1, sm, ColIdx<TC>{cc}, tw, q);
        uint64_t *dst = dst0 + (int64_t)l * N;
#pragma unroll
        for (int e = 0; e < 8; ++e) dst[(int64_t)Pass<LC>::last(j, e) * C] = v[e];
    }
}

template <int LC, int AMAX>
__global__ __launch_bounds__(kNttThreads, AMAX <= 2 ? 3 : 2) void k_ks_modup_cols(KsArgs a, const uint64_t *z,
                                                                                 uint64_t *ext, int nparts) {
    __shared__ uint64_t sm[kNttTile];
    ks_modup_cols_tile<LC, AMAX>(a, z, ext, blockIdx.x, blockIdx.y / nparts, sm, blockIdx.y % nparts, nparts);
}

// Forward row pass, in place, of every raised limb: ext[item][jd][l] for the
// primes l outside digit jd (output unreduced, < 80q).
// tile: row block bx of raised limb l of digit jd of `item` (l outside the digit)
template <int LR>
__device__ __forceinline__ void ks_rows_fwd_tile(const KsArgs &a, uint64_t *ext, int bx, int64_t item, int jd,
                                                 int l, uint64_t *sm) {
    constexpr int M = 1 << LR, TR = kNttTile / M, P = M / 8;
    const int N = 1 << a.log2n, n1 = a.log2n - LR, LK = a.L + a.K;
    const uint64_t q = a.mc[l].q;
    const TwPair *tw = (const TwPair *)(a.tw + (int64_t)l * 4 * N);
    const int t = threadIdx.x, rr = t / P, j = t % P, row = bx * TR + rr;
    uint64_t *x = ext + ((item * a.dnum + jd) * LK + l) * N + (int64_t)row * M;
    uint64_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = x[Pass<LR>::first(j, e)];
    fwd_body<LR>(v, j, (1u << n1) + row, sm, RowIdxW<M>(rr), tw, q);
    store8(x + 8 * j, v);
}

template <int LR>
__global__ __launch_bounds__(kNttThreads, 5) void k_ks_rows_fwd(KsArgs a, uint64_t *ext) {
    __shared__ uint64_t sm[kRowTileWords];
    const int LK = a.L + a.K;
    const int l = blockIdx.y % LK, jd = (blockIdx.y / LK) % a.dnum;
    const int64_t item = blockIdx.y / (LK * a.dnum);
    const int i0 = jd * a.alpha, i1 = min(a.L, i0 + a.alpha);
    if (l >= i0 && l < i1) return;  // the digit's own primes keep d itself
    ks_rows_fwd_tile<LR>(a, ext, blockIdx.x, item, jd, l, sm);
}

// The same row pass with persistent CTAs walking the 2048-word row tiles:
// the TMA engine (cp.async.bulk) brings the next tile into the second
// shared buffer while the current one is transformed.  A schedule option
// (the autotuner times both; on the stencil ring the direct kernel wins).
template <int LR>
__global__ __launch_bounds__(kNttThreads) void k_ks_rows_fwd_tma(KsArgs a, uint64_t *ext, int n_tiles,
                                                                 int log_gr) {
    constexpr int M = 1 << LR, TR = kNttTile / M, P = M / 8;
    extern __shared__ __align__(128) uint64_t dyn[];
    uint64_t *const buf0 = dyn, *const buf1 = dyn + kNttTile;
    uint64_t *sm = dyn + 2 * kNttTile, *bars = sm + kRowTileWords;
    const int N = 1 << a.log2n, n1 = a.log2n - LR, LK = a.L + a.K;
    const int t = threadIdx.x, rr = t / P, j = t % P;
    // tile id = (limb block) * 2^log_gr + x (32-bit: fewer than 2^31 tiles);
    // the digit's own primes keep d itself
    auto skip = [&](int id) {
        const int y = id >> log_gr, l = y % LK, jd = (y / LK) % a.dnum;
        const int i0 = jd * a.alpha;
        return l >= i0 && l < min(a.L, i0 + a.alpha);
    };
    auto next = [&](int id) {
        while (id < n_tiles && skip(id)) id += gridDim.x;
        return id;
    };
    auto tile = [&](int id) { return ext + (int64_t)id * kNttTile; };  // N = 2^log_gr * kNttTile
    if (t == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    int id = next(blockIdx.x);
    if (t == 0 && id < n_tiles) bulk_load(buf0, tile(id), kNttTile * 8, &bars[0]);
    uint32_t ph0 = 0, ph1 = 0;  // parity each buffer's barrier completes next
    int cur = 0;
    bool pending = false;  // a prefetch into the other buffer is in flight
    while (id < n_tiles) {
        uint64_t *const b = cur ? buf1 : buf0, *const other = cur ? buf0 : buf1;
        const int nid = next(id + gridDim.x);
        if (t == 0 && nid < n_tiles) {  // `other` was released by the barrier ending the last tile
            fence_proxy_async_smem();
            bulk_load(other, tile(nid), kNttTile * 8, &bars[cur ^ 1]);
        }
        pending = nid < n_tiles;
        if (!__syncthreads_and(mbar_wait(&bars[cur], cur ? ph1 : ph0, kWaitPolls, a.err))) break;
        if (cur) ph1 ^= 1; else ph0 ^= 1;
        const int y = id >> log_gr;
        const int l = y % LK, row = (id & ((1 << log_gr) - 1)) * TR + rr;
        const uint64_t q = a.mc[l].q;
        const TwPair *tw = (const TwPair *)(a.tw + (int64_t)l * 4 * N);
        uint64_t v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = b[rr * M + Pass<LR>::first(j, e)];
        fwd_body<LR>(v, j, (1u << n1) + row, sm, RowIdx<M>{rr}, tw, q);
        store8(tile(id) + rr * M + 8 * j, v);
        __syncthreads();  // b fully read before it is refilled
        id = nid;
        cur ^= 1;
        pending = false;
    }
    // after a timed-out wait: let an issued prefetch land before the CTA exits
    if (t == 0 && pending) mbar_wait(&bars[cur ^ 1], cur ? ph0 : ph1, kWaitPolls, a.err);
}

constexpr size_t kRowsTmaSmem = (2 * kNttTile + kRowTileWords + 2) * sizeof(uint64_t);

// persistent grid of the TMA row pass: its resident CTAs on the whole GPU
// (set by ks_prepare, outside any stream capture)
template <int LR>
int &rows_fwd_blocks() {
    static int blocks = 152 * 4;
    return blocks;
}

template <int LR>
cudaError_t rows_fwd_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_ks_rows_fwd_tma<LR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kRowsTmaSmem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0, dev = 0;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ks_rows_fwd_tma<LR>, kNttThreads,
                                                           kRowsTmaSmem)))
        return e;
    rows_fwd_blocks<LR>() = std::max(1, per_sm) * std::max(1, sms);
    return cudaSuccess;
}

// Inner product with the key: acc[item][c][l] = sum_j e_j * key[j][c][l]
// with e_j = ext[item][j][l] (< 80q) or, on digit j's own primes, d itself.
// Keys are in Montgomery form, so the 128-bit sum needs one reduction.
// On the Q primes the addend y_c of the output, times P, joins the sum
// (P * 2^64 mod q as its factor): (acc + P y - delta) * P^-1 = (acc - delta)
// * P^-1 + y exactly, and P y vanishes on the P primes that ModDown reads.
// With HE-Mult fused (s.ta), y = (a0 b0, a0 b1 + a1 b0) and d = a1 b1.
// Items vary fastest so a key limb stays in L2 while every item uses it.
// DN > 0: dnum known at compile time, every digit's loads issued before the
// first product; DN = 0: any dnum, one digit at a time.
template <int DN>
__device__ __forceinline__ void ks_mac_tile(const KsArgs &a, const KsSrc &s, const KsAdd &ad, const uint64_t *ext,
                                            const uint64_t *key, uint64_t *acc, int n, int IT, int bx, int by) {
    // tiles: x = blocks of 256 coefficient pairs, y = l * ceil(n / IT) + item
    // group; IT items per thread share the key loads
    const int N = 1 << a.log2n, LK = a.L + a.K;
    const int ng = (n + IT - 1) / IT;
    const int l = by / ng;
    const int64_t item0 = (int64_t)(by - l * ng) * IT;
    const int64_t k = 2 * ((int64_t)bx * 256 + threadIdx.x);
    if (k >= N) return;
    const ModConst mc = a.mc[l];
#pragma unroll 1
    for (int it = 0; it < IT; ++it) {
    const int64_t item = item0 + it;
    if (item >= n) break;
    constexpr int B = DN > 0 ? DN : 1;
    const int dnum = DN > 0 ? DN : a.dnum;
    Acc3 c0a, c0b, c1a, c1b;  // (component, coefficient) sums
    // addend terms (Q primes only) and, fused, d = a1 b1
    ulonglong2 own = make_ulonglong2(0, 0);
    if (l < a.L) {
        ulonglong2 y0 = make_ulonglong2(0, 0), y1 = make_ulonglong2(0, 0);
        uint64_t pm = a.pmont[l];
        if (s.ta || s.tap) {
            ulonglong2 a0, b0, a1, b1;
            if (s.pk_bits) {
                const uint64_t q = mc.q;
                const int W = s.pk_bits;
                const uint64_t *pa0 = src_a(s, item) + (int64_t)l * s.pk_lw;
                const uint64_t *pb0 = src_b(s, item) + (int64_t)l * s.pk_lw;
                const uint64_t *pa1 = pa0 + (int64_t)a.L * s.pk_lw, *pb1 = pb0 + (int64_t)a.L * s.pk_lw;
                a0 = make_ulonglong2(packed_residue(pa0, k, W, q, a.err), packed_residue(pa0, k + 1, W, q, a.err));
                b0 = make_ulonglong2(packed_residue(pb0, k, W, q, a.err), packed_residue(pb0, k + 1, W, q, a.err));
                a1 = make_ulonglong2(packed_residue(pa1, k, W, q, a.err), packed_residue(pa1, k + 1, W, q, a.err));
                b1 = make_ulonglong2(packed_residue(pb1, k, W, q, a.err), packed_residue(pb1, k + 1, W, q, a.err));
            } else {
                const int64_t o = (int64_t)l * N + k, LN = (int64_t)a.L * N;
                const uint64_t *ia = src_a(s, item), *ib = src_b(s, item);
                a0 = *(const ulonglong2 *)(ia + o);
                b0 = *(const ulonglong2 *)(ib + o);
                a1 = *(const ulonglong2 *)(ia + o + LN);
                b1 = *(const ulonglong2 *)(ib + o + LN);
            }
            own = make_ulonglong2(mul_mod(a1.x, b1.x, mc), mul_mod(a1.y, b1.y, mc));
            // y0, y1 as Montgomery residues (times 2^-64, in [0, 2q)); their
            // factor P * 2^128 mod q restores the scale in the final reduction
            y0 = make_ulonglong2(mont_lazy(a0.x, b0.x, 0, 0, mc), mont_lazy(a0.y, b0.y, 0, 0, mc));
            y1 = make_ulonglong2(mont_lazy(a0.x, b1.x, a1.x, b0.x, mc), mont_lazy(a0.y, b1.y, a1.y, b0.y, mc));
            pm = a.pmont2[l];
        } else if (s.perm) {  // rotation: d and the addend through the Galois permutation
            const int32_t p0 = s.perm[k], p1 = s.perm[k + 1];
            const uint64_t *dl = s.d + (int64_t)(s.idx ? s.idx[item] : item) * s.ds + (int64_t)l * N;
            own = make_ulonglong2(dl[p0], dl[p1]);
            if (ad.p) {
                const int32_t q0 = ad.perm ? ad.perm[k] : (int32_t)k, q1 = ad.perm ? ad.perm[k + 1] : (int32_t)k + 1;
                const uint64_t *base = ad.p + (int64_t)(ad.idx ? ad.idx[item] : item) * ad.is + (int64_t)l * N;
                if (ad.mask & 1) y0 = make_ulonglong2(base[q0], base[q1]);
                if (ad.mask & 2) y1 = make_ulonglong2(base[ad.cs + q0], base[ad.cs + q1]);
            }
        } else {
            own = *(const ulonglong2 *)(s.d + (int64_t)(s.idx ? s.idx[item] : item) * s.ds + (int64_t)l * N + k);
            if (ad.p) {
                const uint64_t *base = ad.p + (int64_t)(ad.idx ? ad.idx[item] : item) * ad.is + (int64_t)l * N + k;
                if (ad.mask & 1) y0 = *(const ulonglong2 *)base;
                if (ad.mask & 2) y1 = *(const ulonglong2 *)(base + ad.cs);
            }
        }
        mac3(c0a, y0.x, pm);
        mac3(c0b, y0.y, pm);
        mac3(c1a, y1.x, pm);
        mac3(c1b, y1.y, pm);
    }
    for (int j0 = 0; j0 < dnum; j0 += B) {
        ulonglong2 e[B], w0[B], w1[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const int jd = j0 + u;
            const int i0 = jd * a.alpha, i1 = min(a.L, i0 + a.alpha);
            w0[u] = __ldg((const ulonglong2 *)(key + ((int64_t)(2 * jd) * LK + l) * N + k));
            w1[u] = __ldg((const ulonglong2 *)(key + ((int64_t)(2 * jd + 1) * LK + l) * N + k));
            if (l >= i0 && l < i1)
                e[u] = own;
            else
                e[u] = *(const ulonglong2 *)(ext + ((item * dnum + jd) * LK + l) * N + k);
        }
#pragma unroll
        for (int u = 0; u < B; ++u) {
            mac3(c0a, e[u].x, w0[u].x);
            mac3(c0b, e[u].y, w0[u].y);
            mac3(c1a, e[u].x, w1[u].x);
            mac3(c1b, e[u].y, w1[u].y);
        }
    }
    uint64_t *o0 = acc + (item * 2 * LK + l) * N + k;
    uint64_t *o1 = o0 + (int64_t)LK * N;
    uint64_t h0a, l0a, h0b, l0b, h1a, l1a, h1b, l1b;
    fold3(c0a, h0a, l0a);
    fold3(c0b, h0b, l0b);
    fold3(c1a, h1a, l1a);
    fold3(c1b, h1b, l1b);
    *(ulonglong2 *)o0 = make_ulonglong2(redc(h0a, l0a, mc.q, mc.qneg), redc(h0b, l0b, mc.q, mc.qneg));
    *(ulonglong2 *)o1 = make_ulonglong2(redc(h1a, l1a, mc.q, mc.qneg), redc(h1b, l1b, mc.q, mc.qneg));
    }
}

template <int DN>
__global__ __launch_bounds__(256, DN >= 5 ? 2 : 3) void k_ks_mac(KsArgs a, KsSrc s, KsAdd ad, const uint64_t *ext,
                                                                 const uint64_t *key, uint64_t *acc, int n, int IT) {
    ks_mac_tile<DN>(a, s, ad, ext, key, acc, n, IT, blockIdx.x, blockIdx.y);
}

// ModDown conversion of y (P limbs of acc, coefficient domain) to each Q prime
// with t folded in, fused with the forward column pass: -> dh [n][2][L][N]
// nparts > 1: this tile makes the Q limbs of range `part` of nparts (each
// part redoes the inverse pass of the P limbs).
template <int LC, int KMAX>
__device__ __forceinline__ void ks_moddown_cols_tile(const KsArgs &a, const uint64_t *acc, uint64_t *dh, int bx,
                                                     int by, uint64_t *sm, int part = 0, int nparts = 1) {
    constexpr int M = 1 << LC, TC = kNttTile / M;
    const int N = 1 << a.log2n, C = N >> LC, L = a.L, K = a.K, LK = L + K;
    const int ic = by;  // item * 2 + component
    const int t = threadIdx.x, cc = t % TC, j = t / TC;
    const int64_t cofs = (int64_t)bx * TC + cc;
    // the P limbs: inverse column pass of the row-pass output, with
    // t^-1 * Phat^-1 * N^-1 folded in
    uint64_t ys[KMAX][8];
#pragma unroll
    for (int s = 0; s < KMAX; ++s) {
        if (s < K) {
            const uint64_t *src = acc + ((int64_t)ic * LK + L + s) * N + cofs;
#pragma unroll
            for (int e = 0; e < 8; ++e) ys[s][e] = src[(int64_t)Pass<LC>::last(j, e) * C];
            const TwPair *itw = (const TwPair *)(a.tw + (int64_t)(L + s) * 4 * N + 2 * N);
            const uint64_t *f = a.yc + 4 * s;
            inv_body<LC, true>(ys[s], j, 1, sm, ColIdx<TC>{cc}, itw, a.mc[L + s].q, f[0], f[1], f[2], f[3]);
        }
    }
    for (int i = part * L / nparts, i1 = (part + 1) * L / nparts; i < i1; ++i) {
        const uint64_t q = a.mc[i].q;
        const TwPair *tw = (const TwPair *)(a.tw + (int64_t)i * 4 * N);
        uint64_t v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = 0;
#pragma unroll
        for (int s = 0; s < KMAX; ++s) {
            if (s < K) {
                const int64_t at = ((int64_t)s * L + i) * 2;
                const uint64_t w = a.phat_t[at], ws = a.phat_t[at + 1];
                const uint64_t ww = a.phat_tw[at], wws = a.phat_tw[at + 1];
#pragma unroll
                for (int e = 0; e < 4; ++e) v[e] += mul_shoup_lazy4(ys[s][e], w, ws, q);  // < 4q each
#pragma unroll
                for (int e = 4; e < 8; ++e) v[e] += mul_shoup_lazy4(ys[s][e], ww, wws, q);  // stage 0's w y
            }
        }
        fwd_body<LC, 4 * KMAX>(v, j, 1, sm, ColIdx<TC>{cc}, tw, q);
        uint64_t *dst = dh + ((int64_t)ic * L + i) * N + cofs;
#pragma unroll
        for (int e = 0; e < 8; ++e) dst[(int64_t)Pass<LC>::last(j, e) * C] = v[e];
    }
}

template <int LC, int KMAX>
__global__ __launch_bounds__(kNttThreads, KMAX <= 2 ? 3 : 2) void k_ks_moddown_cols(KsArgs a, const uint64_t *acc,
                                                                                   uint64_t *dh, int nparts) {
    __shared__ uint64_t sm[kNttTile];
    ks_moddown_cols_tile<LC, KMAX>(a, acc, dh, blockIdx.x, blockIdx.y / nparts, sm, blockIdx.y % nparts, nparts);
}

// Forward row pass of delta, then out = (acc - delta) * P^-1 (the addend is
// already in acc, times P).
// With `post` (a ciphertext batch like out, read at the same words), its
// residues are added to the result: w + Rot(x) in one pass.
template <int LR>
__device__ __forceinline__ void ks_rows_final_tile(const KsArgs &a, const uint64_t *acc, const uint64_t *dh,
                                                   uint64_t *out, const int32_t *oidx, const uint64_t *post,
                                                   int bx, int by, uint64_t *sm) {
    constexpr int M = 1 << LR, TR = kNttTile / M, P = M / 8;
    const int N = 1 << a.log2n, n1 = a.log2n - LR, L = a.L, LK = L + a.K;
    const int ic = by / L, i = by - ic * L;  // ic = item * 2 + component
    const uint64_t q = a.mc[i].q;
    const TwPair *tw = (const TwPair *)(a.tw + (int64_t)i * 4 * N);
    const int t = threadIdx.x, rr = t / P, j = t % P, row = bx * TR + rr;
    const int64_t rofs = (int64_t)row * M;
    const uint64_t *src = dh + ((int64_t)ic * L + i) * N + rofs;
    // item ic / 2 writes ciphertext slot oidx[ic / 2] when given (uniform per CTA)
    const int64_t oc = oidx ? (int64_t)oidx[ic >> 1] * 2 + (ic & 1) : ic;
    uint64_t xa[8], v[8];
    load8(xa, acc + ((int64_t)ic * LK + i) * N + rofs + 8 * j);  // fetched before the transform
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = src[Pass<LR>::first(j, e)];
    fwd_body<LR>(v, j, (1u << n1) + row, sm, RowIdxW<M>(rr), tw, q);
    const uint64_t w = a.pinv[2 * i], ws = a.pinv[2 * i + 1];
#pragma unroll
    for (int e = 0; e < 8; ++e)  // delta < 80q unreduced: (acc + 128q - delta) * P^-1, fully reduced
        v[e] = mul_shoup(xa[e] + 128 * q - v[e], w, ws, q);
    const int64_t o = (oc * L + i) * N + rofs + 8 * j;
    if (post) {
        uint64_t pv[8];
        load8(pv, post + o);
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = add_mod(v[e], pv[e], q);
    }
    store8(out + o, v);
}

template <int LR>
__global__ __launch_bounds__(kNttThreads, LR >= 8 ? 4 : 1) void k_ks_rows_final(KsArgs a, const uint64_t *acc,
                                                                               const uint64_t *dh, uint64_t *out,
                                                                               const int32_t *oidx) {
    __shared__ uint64_t sm[kRowTileWords];
    ks_rows_final_tile<LR>(a, acc, dh, out, oidx, nullptr, blockIdx.x, blockIdx.y, sm);
}

// Parts of a column-pass launch of `ctas` CTAs that each make `outputs`
// limbs: split (doubling) while the launch stays within one wave of 3 CTAs
// per SM, so key switches of few ciphertexts are not left on a few SMs.
// one wave of 3 CTAs of 256 threads per SM on the current device
static int wave3() {
    static int wave = 0;
    if (!wave) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        wave = 3 * std::max(1, sms);
    }
    return wave;
}

static int col_parts(int ctas, int outputs) {
    const int wave = wave3();
    int parts = 1;
    while (2 * parts <= outputs && 2 * parts * ctas <= wave) parts *= 2;
    return parts;
}

// Items per thread of the key product (1, 2, 4 or 8): the most that keeps
// two waves of 3 CTAs per SM, `per_item` CTAs per item group.  A thread's
// items reuse its key words from L1; fewer, longer CTAs also leave room for
// the kernels of a second compute stream.
static int mac_items_per_thread(int n, int per_item) {
    const int wave = wave3();
    int it = 8;
    while (it > 1 && (int64_t)((n + it - 1) / it) * per_item < 2 * wave) it /= 2;
    return it;
}

template <int LC, int LR>
static cudaError_t ks_fused(const Ctx &c, const KsArgs &a, const KsSrc &s, const uint64_t *key,
                            uint64_t *out, const KsAdd &ad, const int32_t *oidx, int n, uint64_t *scratch,
                            cudaStream_t st) {
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
    r = prof_begin(c, "k_ks_modup_cols", st);
    {
        const int parts = col_parts(gc * n * c.dnum, (int)LK - c.alpha);
        const dim3 g(gc, n * c.dnum * parts);
        if (c.alpha <= 2)
            k_ks_modup_cols<LC, 2><<<g, kNttThreads, 0, st>>>(a, z, ext, parts);
        else
            k_ks_modup_cols<LC, 4><<<g, kNttThreads, 0, st>>>(a, z, ext, parts);
    }
    prof_end(c, r, st);
    if (c.rows_tma) {
        r = prof_begin(c, "k_ks_rows_fwd_tma", st);
        const int tiles = (int)(n * c.dnum * LK * gr);  // n is capped so this stays below 2^31
        int log_gr = 0;
        while ((1 << log_gr) < gr) ++log_gr;
        const int grid = std::min(tiles, rows_fwd_blocks<LR>());
        k_ks_rows_fwd_tma<LR><<<grid, kNttThreads, kRowsTmaSmem, st>>>(a, ext, tiles, log_gr);
    } else {
        r = prof_begin(c, "k_ks_rows_fwd", st);
        k_ks_rows_fwd<LR><<<dim3(gr, n * c.dnum * LK), kNttThreads, 0, st>>>(a, ext);
    }
    prof_end(c, r, st);
    r = prof_begin(c, "k_ks_mac", st);
    {
        const int IT = mac_items_per_thread(n, (int)(LK * ((N / 2 + 255) / 256)));
        const dim3 g((unsigned)((N / 2 + 255) / 256), (unsigned)(((n + IT - 1) / IT) * LK));
        switch (c.dnum) {
            case 2: k_ks_mac<2><<<g, 256, 0, st>>>(a, s, ad, ext, key, acc, n, IT); break;
            case 3: k_ks_mac<3><<<g, 256, 0, st>>>(a, s, ad, ext, key, acc, n, IT); break;
            case 4: k_ks_mac<4><<<g, 256, 0, st>>>(a, s, ad, ext, key, acc, n, IT); break;
            case 5: k_ks_mac<5><<<g, 256, 0, st>>>(a, s, ad, ext, key, acc, n, IT); break;
            default: k_ks_mac<0><<<g, 256, 0, st>>>(a, s, ad, ext, key, acc, n, IT); break;
        }
    }
    prof_end(c, r, st);
    r = prof_begin(c, "k_ks_intt_rows", st);
    k_ks_intt_rows<LR><<<dim3(gr, n * 2 * K), kNttThreads, 0, st>>>(a, acc + L * N, LK * N,
                                                                    acc + L * N, LK * N, (int)K,
                                                                    (int)L);
    prof_end(c, r, st);
    r = prof_begin(c, "k_ks_moddown_cols", st);
    {
        const int parts = col_parts(gc * n * 2, (int)L);
        const dim3 g(gc, n * 2 * parts);
        if (c.K <= 2)
            k_ks_moddown_cols<LC, 2><<<g, kNttThreads, 0, st>>>(a, acc, dh, parts);
        else
            k_ks_moddown_cols<LC, 4><<<g, kNttThreads, 0, st>>>(a, acc, dh, parts);
    }
    prof_end(c, r, st);
    r = prof_begin(c, "k_ks_rows_final", st);
    k_ks_rows_final<LR><<<dim3(gr, n * 2 * L), kNttThreads, 0, st>>>(a, acc, dh, out, oidx);
    prof_end(c, r, st);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Persistent evaluation (the program structures are described in persist.h).

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// count a finished tile: a release add, ordered after the CTA's writes of the
// tile (they precede it by the CTA barrier)
__device__ __forceinline__ void red_release_add_u32(uint32_t *p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

static_assert(kMaskTileWords == 2 * 4 * kNttThreads, "a mask tile is 2 x 4 words per thread");

// masked accumulation, one 2048-word tile of the output ciphertext [2][L][N]:
// out = sum_k terms[k] * masks[k], the 128-bit sums reduced (Montgomery) once
// per 4096 terms; each thread takes 2 x 4 consecutive words
__device__ __forceinline__ void mask_tile(const KsArgs &a, const PMask &J, int bx) {
    const int64_t LN = (int64_t)a.L << a.log2n;
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        const int64_t i0 = (int64_t)bx * kMaskTileWords + half * (kMaskTileWords / 2) + 4 * threadIdx.x;
        const int64_t r0 = i0 % LN;
        const ModConst &mc = a.mc[(int)(r0 >> a.log2n)];
        const uint64_t q = mc.q, qneg = mc.qneg;
        uint64_t s[4] = {0, 0, 0, 0};
        for (int k0 = 0; k0 < J.nterms; k0 += 4096) {
            const int k1 = min(J.nterms, k0 + 4096);
            Acc3 c[4];  // residues below q < 2^50: 4096 products fit (modarith.cuh)
            for (int k = k0; k < k1; ++k) {
                const ulonglong2 *w = (const ulonglong2 *)(J.terms[k] + i0);
                const ulonglong2 *m = (const ulonglong2 *)(J.masks[k] + r0);
                const ulonglong2 w0 = __ldcs(w), w1 = __ldcs(w + 1), m0 = m[0], m1 = m[1];
                const uint64_t wv[4] = {w0.x, w0.y, w1.x, w1.y}, mv[4] = {m0.x, m0.y, m1.x, m1.y};
#pragma unroll
                for (int e = 0; e < 4; ++e) mac3(c[e], wv[e], mv[e]);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                uint64_t hi, lo;
                fold3(c[e], hi, lo);
                s[e] = add_mod(s[e], redc(hi, lo, q, qneg), q);
            }
        }
        ulonglong2 *o = (ulonglong2 *)(J.out + i0);
        o[0] = make_ulonglong2(s[0], s[1]);
        o[1] = make_ulonglong2(s[2], s[3]);
    }
}

// raised limb e (0 <= e < dnum (L+K) - L, own primes skipped) -> (digit, prime)
__device__ __forceinline__ void raised_limb(const KsArgs &a, int e, int &jd, int &l) {
    const int LK = a.L + a.K;
    for (jd = 0; jd < a.dnum; ++jd) {
        const int i0 = jd * a.alpha, own = max(0, min(a.L, i0 + a.alpha) - i0);
        if (e < LK - own) {
            l = e < i0 ? e : e + own;
            return;
        }
        e -= LK - own;
    }
    jd = a.dnum - 1;
    l = LK - 1;  // not reached for e in range
}

// The tile kinds of the persistent kernel (inlined: the key-switch constants
// stay kernel parameters, read from the constant bank).
struct PScratch {
    uint64_t *z, *ext, *acc, *dh;
};
__device__ __forceinline__ PScratch persist_scratch(const KsArgs &a, const PInst &I) {
    const int64_t N = 1 << a.log2n, L = a.L, LK = a.L + a.K, n = I.n;
    PScratch r;
    r.z = I.scratch;
    r.ext = r.z + n * L * N;
    r.acc = r.ext + n * a.dnum * LK * N;
    r.dh = r.acc + n * 2 * LK * N;
    return r;
}

template <int LR>
__device__ __forceinline__ void pt_intt(const KsArgs &a, const PInst &I, int bx, int by, uint64_t *sm) {
    ks_intt_rows_src_tile<LR>(a, I.s, persist_scratch(a, I).z, bx, by, sm);
}
template <int LC>
__device__ __forceinline__ void pt_modup(const KsArgs &a, const PInst &I, int bx, int by, uint64_t *sm) {
    const PScratch w = persist_scratch(a, I);
    ks_modup_cols_tile<LC, 2>(a, w.z, w.ext, bx, by, sm);
}
template <int LR>
__device__ __forceinline__ void pt_rows_fwd(const KsArgs &a, const PInst &I, int bx, int by, uint64_t *sm) {
    const int ext_limbs = a.dnum * (a.L + a.K) - a.L;
    const int item = by / ext_limbs;
    int jd, l;
    raised_limb(a, by - item * ext_limbs, jd, l);
    ks_rows_fwd_tile<LR>(a, persist_scratch(a, I).ext, bx, item, jd, l, sm);
}
__device__ __forceinline__ void pt_mac(const KsArgs &a, const PInst &I, int bx, int by) {
    const PScratch w = persist_scratch(a, I);
    ks_mac_tile<0>(a, I.s, I.ad, w.ext, I.key, w.acc, I.n, 2, bx, by);
}
template <int LR>
__device__ __forceinline__ void pt_intt_p(const KsArgs &a, const PInst &I, int bx, int by, uint64_t *sm) {
    const int64_t LN = (int64_t)a.L << a.log2n, LKN = (int64_t)(a.L + a.K) << a.log2n;
    uint64_t *acc = persist_scratch(a, I).acc;
    ks_intt_rows_tile<LR>(a, acc + LN, LKN, acc + LN, LKN, a.K, a.L, bx, by, sm);
}
template <int LC>
__device__ __forceinline__ void pt_moddown(const KsArgs &a, const PInst &I, int bx, int by, uint64_t *sm) {
    const PScratch w = persist_scratch(a, I);
    ks_moddown_cols_tile<LC, 2>(a, w.acc, w.dh, bx, by, sm);
}
template <int LR>
__device__ __forceinline__ void pt_final(const KsArgs &a, const PInst &I, int bx, int by, uint64_t *sm) {
    const PScratch w = persist_scratch(a, I);
    ks_rows_final_tile<LR>(a, w.acc, w.dh, I.out, I.oidx, I.post, bx, by, sm);
}
__device__ __forceinline__ void pt_mask(const KsArgs &a, const PMask &J, int bx) { mask_tile(a, J, bx); }

template <int LC, int LR>
__device__ __forceinline__ void persist_tile(const KsArgs &a, const PProg &P, int kind, int inst, int bx, int by,
                                             uint64_t *sm) {
    switch (kind) {
        case kPhIntt: pt_intt<LR>(a, P.inst[inst], bx, by, sm); break;
        case kPhModUp: pt_modup<LC>(a, P.inst[inst], bx, by, sm); break;
        case kPhRowsFwd: pt_rows_fwd<LR>(a, P.inst[inst], bx, by, sm); break;
        case kPhMac: pt_mac(a, P.inst[inst], bx, by); break;
        case kPhInttP: pt_intt_p<LR>(a, P.inst[inst], bx, by, sm); break;
        case kPhModDown: pt_moddown<LC>(a, P.inst[inst], bx, by, sm); break;
        case kPhFinal: pt_final<LR>(a, P.inst[inst], bx, by, sm); break;
        case kPhMask: pt_mask(a, P.mask[inst], bx); break;
        default: break;  // kPhNone
    }
}

// 4 CTAs of 256 threads per SM (64 registers; the conversion kernels and the
// key product spill a little, which measured faster than 3 or 2 CTAs).
template <int LC, int LR>
__global__ __launch_bounds__(kNttThreads, 4) void k_ks_persist(const KsArgs a, PProg P) {
    __shared__ __align__(16) uint64_t sm[kRowTileWords];
    __shared__ int s_kind, s_inst, s_gx, s_local, s_p;
    uint32_t *const next = P.ctr + P.nph, *const stop = P.ctr + P.nph + 1;
    // thread 0 holds the CTA's next two tiles: t0 with its table entry, and
    // t1, claimed while the current tile runs (tiles are still taken in
    // increasing order, so the lowest unfinished tile never waits on
    // anything unfinished)
    int t0 = 0, t1 = 0, cur = -1;
    uint64_t i0 = 0;
    if (threadIdx.x == 0) {
        t0 = (int)atomicAdd(next, 1u);
        t1 = (int)atomicAdd(next, 1u);
        if (t0 < P.total) i0 = P.info[t0];
    }
    for (;;) {
        if (threadIdx.x == 0) {
            int p = -1;
            if (t0 < P.total && *(volatile uint32_t *)stop == 0) {
                p = (int)(i0 >> 32);
                if (p != cur) {  // a new phase: its descriptor, then its dependencies
                    const PPhase &ph = P.ph[p];
                    s_kind = ph.kind;
                    s_inst = ph.inst;
                    s_gx = ph.gx;
                    const uint64_t ns0 = global_ns();
                    for (int d = 0; d < ph.ndep && p >= 0; ++d) {
                        const int q = P.deps[ph.dep0 + d];
                        const uint32_t need = (uint32_t)(P.off[q + 1] - P.off[q]);
                        for (uint32_t spin = 0; ld_relaxed_u32(P.ctr + q) < need; ++spin) {
                            if (*(volatile uint32_t *)stop) {
                                p = -1;
                                break;
                            }
                            if (global_ns() - ns0 > (uint64_t)P.wait_ns) {
                                atomicExch(a.err, kErrSchedTimeout);
                                atomicExch(stop, 1u);
                                p = -1;
                                break;
                            }
                            __nanosleep(spin < 32 ? 32 : 256);
                        }
                    }
                    fence_acq_rel_gpu();  // acquire: the dependencies' writes are visible after this
                    cur = p;
                }
            }
            s_p = p;
            s_local = (int)(uint32_t)i0;
        }
        __syncthreads();
        const int p = s_p;
        if (p < 0) break;
        const int kind = s_kind, inst = s_inst, gx = s_gx, local = s_local;
        uint64_t i1 = 0;
        int t2 = 0;
        if (threadIdx.x == 0) {  // both complete while the tile runs
            if (t1 < P.total) i1 = P.info[t1];
            t2 = (int)atomicAdd(next, 1u);
        }
        persist_tile<LC, LR>(a, P, kind, inst, local % gx, local / gx, sm);
        __syncthreads();  // every thread's writes of the tile precede the count
        if (threadIdx.x == 0) {
            red_release_add_u32(P.ctr + p, 1u);
            t0 = t1;
            i0 = i1;
            t1 = t2;
        }
    }
}

// resident CTAs of the persistent kernel on the whole GPU, per NTT split
// (set by ks_prepare, outside any stream capture)
template <int LC, int LR>
int &persist_blocks() {
    static int blocks = 152 * 3;
    return blocks;
}

template <int LC, int LR>
cudaError_t persist_prepare() {
    int per_sm = 0, sms = 0, dev = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ks_persist<LC, LR>, kNttThreads, 0)))
        return e;
    persist_blocks<LC, LR>() = std::max(1, per_sm) * std::max(1, sms);
    return cudaSuccess;
}

template <int LC, int LR>
static cudaError_t persist_run(const KsArgs &a, const PProg &P, int max_blocks, cudaStream_t st) {
    int grid = std::min(P.total, persist_blocks<LC, LR>());
    if (max_blocks > 0) grid = std::min(grid, max_blocks);
    k_ks_persist<LC, LR><<<std::max(1, grid), kNttThreads, 0, st>>>(a, P);
    return cudaGetLastError();
}

bool ks_fused_supported(const Ctx &c) {
    return c.log2n >= 11 && c.log2n <= 15 && c.alpha <= 4 && c.K <= 4;
}

// NTT split of the two passes, N = 2^LC (column pass) x 2^LR (row pass):
// variant 0 is the default, variant 1 the alternative the autotuner tries.
static cudaError_t ks_dispatch(const Ctx &c, const KsArgs &a, const KsSrc &s, const uint64_t *key,
                               uint64_t *out, const KsAdd &ad, int m, uint64_t *scratch, cudaStream_t st,
                               const int32_t *oidx = nullptr) {
#define KS_CALL(LC, LR) ks_fused<LC, LR>(c, a, s, key, out, ad, oidx, m, scratch, st)
    const bool alt = c.ks_split == 1;
    switch (c.log2n) {
        case 15: return alt ? KS_CALL(8, 7) : KS_CALL(7, 8);
        case 14: return alt ? KS_CALL(6, 8) : KS_CALL(7, 7);
        case 13: return alt ? KS_CALL(7, 6) : KS_CALL(6, 7);
        case 12: return alt ? KS_CALL(5, 7) : KS_CALL(6, 6);
        case 11: return alt ? KS_CALL(6, 5) : KS_CALL(5, 6);
        default: return cudaErrorInvalidValue;
    }
#undef KS_CALL
}

int ks_split_variants(const Ctx &c) { return ks_fused_supported(c) ? 2 : 1; }

cudaError_t ks_prepare(const Ctx &c) {
    if (!ks_fused_supported(c)) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    switch (c.log2n) {  // the row-pass sizes of both NTT splits, and the persistent kernel's
        case 15: (e = rows_fwd_prepare<8>()) || (e = rows_fwd_prepare<7>()) ||
                 (e = persist_prepare<7, 8>()) || (e = persist_prepare<8, 7>()); break;
        case 14: (e = rows_fwd_prepare<7>()) || (e = rows_fwd_prepare<8>()) ||
                 (e = persist_prepare<7, 7>()) || (e = persist_prepare<6, 8>()); break;
        case 13: (e = rows_fwd_prepare<7>()) || (e = rows_fwd_prepare<6>()) ||
                 (e = persist_prepare<6, 7>()) || (e = persist_prepare<7, 6>()); break;
        case 12: (e = rows_fwd_prepare<6>()) || (e = rows_fwd_prepare<7>()) ||
                 (e = persist_prepare<6, 6>()) || (e = persist_prepare<5, 7>()); break;
        case 11: (e = rows_fwd_prepare<6>()) || (e = rows_fwd_prepare<5>()) ||
                 (e = persist_prepare<5, 6>()) || (e = persist_prepare<6, 5>()); break;
        default: break;
    }
    return e;
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
    a.modup_modw = h->d.modup_modw;
    a.phat_tw = h->d.md_phat_tw;
    a.pinv = h->d.md_pinv;
    a.pmont = h->d.p_mont;
    a.pmont2 = h->d.p_mont2;
    a.err = h->d.err;
    a.log2n = c.log2n;
    a.L = c.L;
    a.K = c.K;
    a.dnum = c.dnum;
    a.alpha = c.alpha;
    return a;
}

static KsArgs ks_args(const Ctx &c);

bool persist_supported(const Ctx &c) { return ks_fused_supported(c) && c.alpha <= 2 && c.K <= 2; }

cudaError_t persist_launch(const Ctx &c, const PProg &P, int max_blocks, cudaStream_t st) {
    if (!persist_supported(c)) return cudaErrorInvalidValue;
    const KsArgs a = ks_args(c);
    const bool alt = c.ks_split == 1;
    switch (c.log2n) {
        case 15: return alt ? persist_run<8, 7>(a, P, max_blocks, st) : persist_run<7, 8>(a, P, max_blocks, st);
        case 14: return alt ? persist_run<6, 8>(a, P, max_blocks, st) : persist_run<7, 7>(a, P, max_blocks, st);
        case 13: return alt ? persist_run<7, 6>(a, P, max_blocks, st) : persist_run<6, 7>(a, P, max_blocks, st);
        case 12: return alt ? persist_run<5, 7>(a, P, max_blocks, st) : persist_run<6, 6>(a, P, max_blocks, st);
        case 11: return alt ? persist_run<6, 5>(a, P, max_blocks, st) : persist_run<5, 6>(a, P, max_blocks, st);
        default: return cudaErrorInvalidValue;
    }
}

// tiles of each stage of a persistent key switch of n items, in stage order
void persist_stage_tiles(const Ctx &c, int n, int32_t gx[7], int32_t gy[7]) {
    const bool alt = c.ks_split == 1;
    int LC = 0;
    switch (c.log2n) {
        case 15: LC = alt ? 8 : 7; break;
        case 14: LC = alt ? 6 : 7; break;
        case 13: LC = alt ? 7 : 6; break;
        case 12: LC = alt ? 5 : 6; break;
        default: LC = alt ? 6 : 5; break;
    }
    const int LR = c.log2n - LC, N = c.N, LK = c.L + c.K;
    const int gc = (N >> LC) / (kNttTile >> LC), gr = (N >> LR) / (kNttTile >> LR);
    const int ext = c.dnum * LK - c.L;
    const int32_t x[7] = {gr, gc, gr, (N / 2 + 255) / 256, gr, gc, gr};
    const int32_t y[7] = {n * c.L, n * c.dnum, n * ext, ((n + 1) / 2) * LK, n * 2 * c.K, 2 * n, 2 * n * c.L};
    for (int i = 0; i < 7; ++i) {
        gx[i] = x[i];
        gy[i] = y[i];
    }
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
        const KsAdd ad{add ? add + i0 * add_is : nullptr, add_is, add_cs, add_mask};
        cudaError_t e = ks_dispatch(c, a, s, key, out + i0 * 2 * c.L * c.N, ad, m, scratch, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t relin_tensor_fused(const Ctx &c, const uint64_t *A, const uint64_t *B,
                               const uint64_t *rlk, uint64_t *out, size_t n, uint64_t *scratch,
                               cudaStream_t st, int pk_bits) {
    const KsArgs a = ks_args(c);
    const int64_t CT = 2 * (int64_t)c.L * c.N;
    const int64_t lw = pk_bits ? ((int64_t)c.N * pk_bits + 63) / 64 : 0;
    const int64_t TS = pk_bits ? 2 * c.L * lw : CT;  // words per input ciphertext
    const size_t maxn = ks_max_items(c);
    for (size_t i0 = 0; i0 < n; i0 += maxn) {
        const int m = (int)std::min(maxn, n - i0);
        KsSrc s{nullptr, 0, A + i0 * TS, B + i0 * TS, TS, pk_bits, lw};
        cudaError_t e = ks_dispatch(c, a, s, rlk, out + i0 * CT, KsAdd{nullptr, 0, 0, 0}, m, scratch, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t relin_tensor_fused_ptrs(const Ctx &c, const uint64_t *const *ta, const uint64_t *const *tb,
                                    const uint64_t *rlk, uint64_t *out, size_t n, uint64_t *scratch,
                                    cudaStream_t st) {
    const KsArgs a = ks_args(c);
    const int64_t CT = 2 * (int64_t)c.L * c.N;
    const size_t maxn = ks_max_items(c);
    for (size_t i0 = 0; i0 < n; i0 += maxn) {
        const int m = (int)std::min(maxn, n - i0);
        KsSrc s{nullptr, 0, nullptr, nullptr, CT};
        s.tap = ta + i0;
        s.tbp = tb + i0;
        cudaError_t e = ks_dispatch(c, a, s, rlk, out + i0 * CT, KsAdd{nullptr, 0, 0, 0}, m, scratch, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t rotate_fused_inplace(const Ctx &c, uint64_t *cts, const int32_t *idx, const int32_t *perm,
                                 const uint64_t *gk, size_t n, uint64_t *scratch, cudaStream_t st) {
    const KsArgs a = ks_args(c);
    const int64_t LN = (int64_t)c.L * c.N, CT = 2 * LN;
    const size_t maxn = ks_max_items(c);
    for (size_t i0 = 0; i0 < n; i0 += maxn) {
        const int m = (int)std::min(maxn, n - i0);
        KsSrc s{cts + LN, CT, nullptr, nullptr, 0};
        s.idx = idx + i0;
        s.perm = perm;
        const KsAdd ad{cts, CT, LN, 1, idx + i0, perm};
        cudaError_t e = ks_dispatch(c, a, s, gk, cts, ad, m, scratch, st, idx + i0);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace hespmv
