// Negacyclic NTT / inverse NTT over word-size primes, batched over limbs.
//
// Forward: Cooley-Tukey with the 2N-th root folded into the twiddles, so
// index i of the output holds a(psi^(2*bitrev(i)+1)).  Stage s (s = 0..logN-1)
// has m = 2^s groups; the pair (j, j+t), t = N/2^(s+1), in group i uses
// W = psi^bitrev(m+i).  Inverse: Gentleman-Sande with psi^-bitrev(m+i) in the
// reverse stage order, N^-1 folded into the last stage.
//
// A limb of N = 2^n words is viewed as R x C (R = 2^n1 rows, C = 2^n2
// contiguous columns).  The first n1 stages only pair words of the same
// column, the last n2 stages only words of the same row, so the transform is
// two tile passes over shared memory ("columns" then "rows"; the inverse in
// the opposite order).  Small rings (N <= 4096) run one "rows" pass with
// n1 = 0.
#include "internal.h"
#include "ntt_core.cuh"

namespace hespmv {

struct NttArgs {
    uint64_t *data;
    int64_t item_stride;  // words between items
    int n_limbs;          // limbs per item (contiguous, N words apart)
    int prime0;           // modulus index of limb 0
    const ModConst *mc;
    const uint64_t *tw;   // [modulus][4][N]
    int log2n;
};

__device__ __forceinline__ void limb_of(const NttArgs &a, uint64_t *&x, int &prime) {
    const int N = 1 << a.log2n;
    const int limb = blockIdx.y;
    const int item = limb / a.n_limbs;
    const int k = limb - item * a.n_limbs;
    x = a.data + (int64_t)item * a.item_stride + (int64_t)k * N;
    prime = a.prime0 + k;
}

// First n1 forward stages on columns [c0, c0+TC) of the R x C view.
__global__ void k_ntt_fwd_cols(NttArgs a, int n1, int TC) {
    extern __shared__ uint64_t sm[];
    uint64_t *x;
    int prime;
    limb_of(a, x, prime);
    const int N = 1 << a.log2n;
    const int R = 1 << n1, C = N >> n1;
    const uint64_t q = a.mc[prime].q;
    const uint64_t *tw = a.tw + (int64_t)prime * 4 * N;  // (w, Shoup) pairs
    const int c0 = blockIdx.x * TC;
    for (int e = threadIdx.x; e < R * TC; e += blockDim.x) {
        const int r = e / TC, cc = e - r * TC;
        sm[e] = x[(int64_t)r * C + c0 + cc];
    }
    __syncthreads();
    for (int s = 0; s < n1; ++s) {
        const int half = R >> (s + 1), m = 1 << s;
        for (int b = threadIdx.x; b < (R / 2) * TC; b += blockDim.x) {
            const int cc = b % TC, bb = b / TC;
            const int grp = bb / half, pos = bb - grp * half;
            const int r = grp * 2 * half + pos;
            const uint64_t W = tw[2 * (m + grp)], Ws = tw[2 * (m + grp) + 1];
            const uint64_t u = sm[r * TC + cc];
            const uint64_t v = mul_shoup(sm[(r + half) * TC + cc], W, Ws, q);
            sm[r * TC + cc] = add_mod(u, v, q);
            sm[(r + half) * TC + cc] = sub_mod(u, v, q);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < R * TC; e += blockDim.x) {
        const int r = e / TC, cc = e - r * TC;
        x[(int64_t)r * C + c0 + cc] = sm[e];
    }
}

// Last n2 forward stages on rows [r0, r0+TR).
__global__ void k_ntt_fwd_rows(NttArgs a, int n1, int TR) {
    extern __shared__ uint64_t sm[];
    uint64_t *x;
    int prime;
    limb_of(a, x, prime);
    const int N = 1 << a.log2n;
    const int C = N >> n1;
    const uint64_t q = a.mc[prime].q;
    const uint64_t *tw = a.tw + (int64_t)prime * 4 * N;  // (w, Shoup) pairs
    const int r0 = blockIdx.x * TR;
    uint64_t *base = x + (int64_t)r0 * C;
    for (int e = threadIdx.x; e < TR * C; e += blockDim.x) sm[e] = base[e];
    __syncthreads();
    for (int s = n1; s < a.log2n; ++s) {
        const int m = 1 << s, t = N >> (s + 1);
        const int per_row = C / (2 * t);
        for (int b = threadIdx.x; b < TR * (C / 2); b += blockDim.x) {
            const int rr = b / (C / 2), bb = b - rr * (C / 2);
            const int grp = bb / t, pos = bb - grp * t;
            const int idx = rr * C + grp * 2 * t + pos;
            const int i = (r0 + rr) * per_row + grp;
            const uint64_t u = sm[idx];
            const uint64_t v = mul_shoup(sm[idx + t], tw[2 * (m + i)], tw[2 * (m + i) + 1], q);
            sm[idx] = add_mod(u, v, q);
            sm[idx + t] = sub_mod(u, v, q);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < TR * C; e += blockDim.x) base[e] = sm[e];
}

// Inverse stages logN-1 .. n1 on rows (N^-1 folded in when n1 == 0).
__global__ void k_ntt_inv_rows(NttArgs a, int n1, int TR) {
    extern __shared__ uint64_t sm[];
    uint64_t *x;
    int prime;
    limb_of(a, x, prime);
    const int N = 1 << a.log2n;
    const int C = N >> n1;
    const ModConst mc = a.mc[prime];
    const uint64_t q = mc.q;
    const uint64_t *itw = a.tw + (int64_t)prime * 4 * N + 2 * N;  // (w, Shoup) pairs
    const int r0 = blockIdx.x * TR;
    uint64_t *base = x + (int64_t)r0 * C;
    for (int e = threadIdx.x; e < TR * C; e += blockDim.x) sm[e] = base[e];
    __syncthreads();
    for (int s = a.log2n - 1; s >= n1; --s) {
        const int m = 1 << s, t = N >> (s + 1);
        const int per_row = C / (2 * t);
        for (int b = threadIdx.x; b < TR * (C / 2); b += blockDim.x) {
            const int rr = b / (C / 2), bb = b - rr * (C / 2);
            const int grp = bb / t, pos = bb - grp * t;
            const int idx = rr * C + grp * 2 * t + pos;
            const int i = (r0 + rr) * per_row + grp;
            const uint64_t u = sm[idx], v = sm[idx + t];
            if (s == 0) {
                sm[idx] = mul_shoup(u + v, mc.ninv, mc.ninv_s, q);
                sm[idx + t] = mul_shoup(u + q - v, mc.w1ninv, mc.w1ninv_s, q);
            } else {
                sm[idx] = add_mod(u, v, q);
                sm[idx + t] = mul_shoup(u + q - v, itw[2 * (m + i)], itw[2 * (m + i) + 1], q);
            }
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < TR * C; e += blockDim.x) base[e] = sm[e];
}

// Inverse stages n1-1 .. 0 on columns, N^-1 folded into stage 0.
__global__ void k_ntt_inv_cols(NttArgs a, int n1, int TC) {
    extern __shared__ uint64_t sm[];
    uint64_t *x;
    int prime;
    limb_of(a, x, prime);
    const int N = 1 << a.log2n;
    const int R = 1 << n1, C = N >> n1;
    const ModConst mc = a.mc[prime];
    const uint64_t q = mc.q;
    const uint64_t *itw = a.tw + (int64_t)prime * 4 * N + 2 * N;  // (w, Shoup) pairs
    const int c0 = blockIdx.x * TC;
    for (int e = threadIdx.x; e < R * TC; e += blockDim.x) {
        const int r = e / TC, cc = e - r * TC;
        sm[e] = x[(int64_t)r * C + c0 + cc];
    }
    __syncthreads();
    for (int s = n1 - 1; s >= 0; --s) {
        const int half = R >> (s + 1), m = 1 << s;
        for (int b = threadIdx.x; b < (R / 2) * TC; b += blockDim.x) {
            const int cc = b % TC, bb = b / TC;
            const int grp = bb / half, pos = bb - grp * half;
            const int r = grp * 2 * half + pos;
            const uint64_t u = sm[r * TC + cc], v = sm[(r + half) * TC + cc];
            if (s == 0) {
                sm[r * TC + cc] = mul_shoup(u + v, mc.ninv, mc.ninv_s, q);
                sm[(r + half) * TC + cc] = mul_shoup(u + q - v, mc.w1ninv, mc.w1ninv_s, q);
            } else {
                sm[r * TC + cc] = add_mod(u, v, q);
                sm[(r + half) * TC + cc] = mul_shoup(u + q - v, itw[2 * (m + grp)], itw[2 * (m + grp) + 1], q);
            }
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < R * TC; e += blockDim.x) {
        const int r = e / TC, cc = e - r * TC;
        x[(int64_t)r * C + c0 + cc] = sm[e];
    }
}


// ---------------------------------------------------------------------------
// Register-blocked passes (N >= 2^11: a limb holds at least one 2048-word
// tile), see ntt_core.cuh.  Bounded to 48 registers (5 CTAs per SM) where
// that does not spill: 1-3 % faster per pass at N = 2^15.

// Column pass, forward: local stages 0 .. LOGM-1 of the R = 2^LOGM rows.
template <int LOGM>
__global__ __launch_bounds__(kNttThreads, 5) void k_fntt_cols(NttArgs a) {
    constexpr int M = 1 << LOGM, TC = kNttTile / M;
    constexpr int R1 = Sched<LOGM>::R1, R2 = Sched<LOGM>::R2;
    __shared__ uint64_t sm[kNttTile];
    uint64_t *x;
    int prime;
    limb_of(a, x, prime);
    const int N = 1 << a.log2n, C = N >> LOGM;
    const uint64_t q = a.mc[prime].q;
    const TwPair *tw = (const TwPair *)(a.tw + (int64_t)prime * 4 * N);
    const int t = threadIdx.x, cc = t % TC, j = t / TC;
    uint64_t *col = x + blockIdx.x * TC + cc;
    uint64_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = col[(int64_t)elem_pos<LOGM, 0, 3>(j, e) * C];
    fwd_round<LOGM, 0, 3>(v, j, 1, tw, q);
#pragma unroll
    for (int e = 0; e < 8; ++e) sm[elem_pos<LOGM, 0, 3>(j, e) * TC + cc] = v[e];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = sm[elem_pos<LOGM, 3, R1>(j, e) * TC + cc];
    fwd_round<LOGM, 3, R1>(v, j, 1, tw, q);
    if constexpr (R2 > 0) {
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 8; ++e) sm[elem_pos<LOGM, 3, R1>(j, e) * TC + cc] = v[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = sm[elem_pos<LOGM, 3 + R1, R2>(j, e) * TC + cc];
        fwd_round<LOGM, 3 + R1, R2>(v, j, 1, tw, q);
#pragma unroll
        for (int e = 0; e < 8; ++e) col[(int64_t)elem_pos<LOGM, 3 + R1, R2>(j, e) * C] = v[e];
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) col[(int64_t)elem_pos<LOGM, 3, R1>(j, e) * C] = v[e];
    }
}

// Row pass, forward: local stages of each C = 2^LOGM row; output reduced.
template <int LOGM>
__global__ __launch_bounds__(kNttThreads, 5) void k_fntt_rows(NttArgs a) {
    constexpr int M = 1 << LOGM, TR = kNttTile / M, P = M / 8;
    constexpr int R1 = Sched<LOGM>::R1, R2 = Sched<LOGM>::R2;
    __shared__ uint64_t sm[kRowTileWords];
    uint64_t *x;
    int prime;
    limb_of(a, x, prime);
    const int N = 1 << a.log2n, n1 = a.log2n - LOGM;
    const uint64_t q = a.mc[prime].q, one_s = a.mc[prime].one_s;
    const TwPair *tw = (const TwPair *)(a.tw + (int64_t)prime * 4 * N);
    const int t = threadIdx.x, rr = t / P, j = t % P;
    const int row = blockIdx.x * TR + rr;
    const uint32_t twb = (1u << n1) + row;
    uint64_t *base = x + (int64_t)row * M;
    const RowIdx<M> si{rr};
    uint64_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = base[elem_pos<LOGM, 0, 3>(j, e)];
    fwd_round<LOGM, 0, 3>(v, j, twb, tw, q);
#pragma unroll
    for (int e = 0; e < 8; ++e) sm[si(elem_pos<LOGM, 0, 3>(j, e))] = v[e];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = sm[si(elem_pos<LOGM, 3, R1>(j, e))];
    fwd_round<LOGM, 3, R1>(v, j, twb, tw, q);
    if constexpr (R2 > 0) {
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 8; ++e) sm[si(elem_pos<LOGM, 3, R1>(j, e))] = v[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = sm[si(elem_pos<LOGM, 3 + R1, R2>(j, e))];
        fwd_round<LOGM, 3 + R1, R2>(v, j, twb, tw, q);
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = reduce_full(v[e], q, one_s);
        store8(base + 8 * j, v);  // = elem_pos<LOGM, 3 + R1, R2>(j, e)
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = reduce_full(v[e], q, one_s);
        store8(base + 8 * j, v);  // = elem_pos<LOGM, 3, R1>(j, e)
    }
}

// Row pass, inverse: local stages LOGM-1 .. 0 of each row (first inverse pass).
template <int LOGM>
__global__ __launch_bounds__(kNttThreads, 5) void k_intt_rows(NttArgs a) {
    constexpr int M = 1 << LOGM, TR = kNttTile / M, P = M / 8;
    constexpr int R1 = Sched<LOGM>::R1, R2 = Sched<LOGM>::R2;
    __shared__ uint64_t sm[kRowTileWords];
    uint64_t *x;
    int prime;
    limb_of(a, x, prime);
    const int N = 1 << a.log2n, n1 = a.log2n - LOGM;
    const uint64_t q = a.mc[prime].q;
    const TwPair *itw = (const TwPair *)(a.tw + (int64_t)prime * 4 * N + 2 * N);
    const int t = threadIdx.x, rr = t / P, j = t % P;
    const int row = blockIdx.x * TR + rr;
    const uint32_t twb = (1u << n1) + row;
    uint64_t *base = x + (int64_t)row * M;
    const RowIdx<M> si{rr};
    uint64_t v[8];
    if constexpr (R2 > 0) {
        load8(v, base + 8 * j);  // = elem_pos<LOGM, 3 + R1, R2>(j, e)
        inv_round<LOGM, 3 + R1, R2>(v, j, twb, itw, q);
#pragma unroll
        for (int e = 0; e < 8; ++e) sm[si(elem_pos<LOGM, 3 + R1, R2>(j, e))] = v[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = sm[si(elem_pos<LOGM, 3, R1>(j, e))];
    } else {
        load8(v, base + 8 * j);  // = elem_pos<LOGM, 3, R1>(j, e)
    }
    inv_round<LOGM, 3, R1>(v, j, twb, itw, q);
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 8; ++e) sm[si(elem_pos<LOGM, 3, R1>(j, e))] = v[e];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = sm[si(elem_pos<LOGM, 0, 3>(j, e))];
    inv_round<LOGM, 0, 3>(v, j, twb, itw, q);
#pragma unroll
    for (int e = 0; e < 8; ++e) base[elem_pos<LOGM, 0, 3>(j, e)] = v[e];
}

// Column pass, inverse: local stages LOGM-1 .. 0 of the columns, with N^-1
// folded into stage 0; output reduced to [0, q).
template <int LOGM>
__global__ __launch_bounds__(kNttThreads, LOGM >= 7 ? 5 : 1) void k_intt_cols(NttArgs a) {
    constexpr int M = 1 << LOGM, TC = kNttTile / M;
    constexpr int R1 = Sched<LOGM>::R1, R2 = Sched<LOGM>::R2;
    __shared__ uint64_t sm[kNttTile];
    uint64_t *x;
    int prime;
    limb_of(a, x, prime);
    const int N = 1 << a.log2n, C = N >> LOGM;
    const ModConst mc = a.mc[prime];
    const uint64_t q = mc.q;
    const TwPair *itw = (const TwPair *)(a.tw + (int64_t)prime * 4 * N + 2 * N);
    const int t = threadIdx.x, cc = t % TC, j = t / TC;
    uint64_t *col = x + blockIdx.x * TC + cc;
    uint64_t v[8];
    if constexpr (R2 > 0) {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = col[(int64_t)elem_pos<LOGM, 3 + R1, R2>(j, e) * C];
        inv_round<LOGM, 3 + R1, R2>(v, j, 1, itw, q);
#pragma unroll
        for (int e = 0; e < 8; ++e) sm[elem_pos<LOGM, 3 + R1, R2>(j, e) * TC + cc] = v[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = sm[elem_pos<LOGM, 3, R1>(j, e) * TC + cc];
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = col[(int64_t)elem_pos<LOGM, 3, R1>(j, e) * C];
    }
    inv_round<LOGM, 3, R1>(v, j, 1, itw, q);
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 8; ++e) sm[elem_pos<LOGM, 3, R1>(j, e) * TC + cc] = v[e];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = sm[elem_pos<LOGM, 0, 3>(j, e) * TC + cc];
    inv_round_last<LOGM, 3>(v, j, 1, itw, q, mc.ninv, mc.ninv_s, mc.w1ninv, mc.w1ninv_s);
#pragma unroll
    for (int e = 0; e < 8; ++e) col[(int64_t)elem_pos<LOGM, 0, 3>(j, e) * C] = v[e];
}

template <int LC, int LR>
static void launch_fast(const NttArgs &a, const Ctx &c, int total, bool inverse, cudaStream_t st) {
    const int N = c.N;
    dim3 gc((N >> LC) / (kNttTile >> LC), total), gr((N >> LR) / (kNttTile >> LR), total);
    int r;
    if (!inverse) {
        r = prof_begin(c, "k_fntt_cols", st);
        k_fntt_cols<LC><<<gc, kNttThreads, 0, st>>>(a);
        prof_end(c, r, st);
        r = prof_begin(c, "k_fntt_rows", st);
        k_fntt_rows<LR><<<gr, kNttThreads, 0, st>>>(a);
        prof_end(c, r, st);
    } else {
        r = prof_begin(c, "k_intt_rows", st);
        k_intt_rows<LR><<<gr, kNttThreads, 0, st>>>(a);
        prof_end(c, r, st);
        r = prof_begin(c, "k_intt_cols", st);
        k_intt_cols<LC><<<gc, kNttThreads, 0, st>>>(a);
        prof_end(c, r, st);
    }
}

cudaError_t launch_ntt(const Ctx &c, uint64_t *data, int prime0, int n_limbs, int n_items,
                       int64_t item_stride, bool inverse, cudaStream_t st) {
    if (n_items <= 0 || n_limbs <= 0) return cudaSuccess;
    NttArgs a;
    a.data = data;
    a.item_stride = item_stride;
    a.n_limbs = n_limbs;
    a.prime0 = prime0;
    a.mc = c.c->d.mc;
    a.tw = c.c->d.tw;
    a.log2n = c.log2n;
    const int N = c.N;
    const int total = n_limbs * n_items;
    if (total > 65535) {
        // grid.y limit: split into slices of whole items
        const int per = 65535 / n_limbs;
        for (int i0 = 0; i0 < n_items; i0 += per) {
            cudaError_t e = launch_ntt(c, data + (int64_t)i0 * item_stride, prime0, n_limbs,
                                       std::min(per, n_items - i0), item_stride, inverse, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    switch (c.log2n) {  // register-blocked two-pass transform, R = 2^(n/2) rows
        case 15: launch_fast<7, 8>(a, c, total, inverse, st); return cudaGetLastError();
        case 14: launch_fast<7, 7>(a, c, total, inverse, st); return cudaGetLastError();
        case 13: launch_fast<6, 7>(a, c, total, inverse, st); return cudaGetLastError();
        case 12: launch_fast<6, 6>(a, c, total, inverse, st); return cudaGetLastError();
        case 11: launch_fast<5, 6>(a, c, total, inverse, st); return cudaGetLastError();
        default: break;
    }
    if (c.log2n <= 12) {
        dim3 grid(1, total);
        const int thr = std::min(256, N / 2);
        const size_t smem = (size_t)N * 8;
        const int r = prof_begin(c, inverse ? "k_ntt_inv_rows" : "k_ntt_fwd_rows", st);
        if (inverse)
            k_ntt_inv_rows<<<grid, thr, smem, st>>>(a, 0, 1);
        else
            k_ntt_fwd_rows<<<grid, thr, smem, st>>>(a, 0, 1);
        prof_end(c, r, st);
        return cudaGetLastError();
    }
    const int n1 = c.log2n / 2;
    const int R = 1 << n1, C = N >> n1;
    const int TC = std::max(1, 2048 / R), TR = std::max(1, 2048 / C);
    const size_t smc = (size_t)R * TC * 8, smr = (size_t)TR * C * 8;
    dim3 gc(C / TC, total), gr(R / TR, total);
    int r;
    if (!inverse) {
        r = prof_begin(c, "k_ntt_fwd_cols", st);
        k_ntt_fwd_cols<<<gc, 256, smc, st>>>(a, n1, TC);
        prof_end(c, r, st);
        r = prof_begin(c, "k_ntt_fwd_rows", st);
        k_ntt_fwd_rows<<<gr, 256, smr, st>>>(a, n1, TR);
        prof_end(c, r, st);
    } else {
        r = prof_begin(c, "k_ntt_inv_rows", st);
        k_ntt_inv_rows<<<gr, 256, smr, st>>>(a, n1, TR);
        prof_end(c, r, st);
        r = prof_begin(c, "k_ntt_inv_cols", st);
        k_ntt_inv_cols<<<gc, 256, smc, st>>>(a, n1, TC);
        prof_end(c, r, st);
    }
    return cudaGetLastError();
}

}  // namespace hespmv
