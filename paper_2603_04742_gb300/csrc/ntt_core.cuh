// Register-blocked negacyclic NTT building blocks.
//
// A limb of N = 2^n words is transformed as two passes over an R x C view
// (R = 2^n1 rows, C = 2^n2 contiguous columns): the first n1 Cooley-Tukey
// stages pair words of one column, the last n2 words of one row.  Each pass is
// a length-M sub-transform (M = R or C) done by 256 threads on a 2048-word
// tile in rounds of up to three stages: a thread holds 8 words in registers,
// runs the round's butterflies, and words are re-dealt through shared memory
// between rounds.
//
// Round (S0, NS) covers local stages S0 .. S0+NS-1.  Value e of thread j is
// element k = e mod 2^NS of group G = j*(8 >> NS) + (e >> NS), at position
//     rho = hi * (M >> S0) + k * LO + lo,  LO = M >> (S0+NS),  G = hi*LO + lo,
// so the round's butterflies pair values inside one thread.  At local stage s
// the pair's twiddle is psi^bitrev(twb * 2^s + grp) with grp = rho / (M >> s);
// twb = 1 for the column pass and 2^n1 + row for the row pass (stage offset
// n1), which reproduces the index m + i of the textbook loop.
//
// Lazy ranges: forward butterflies let values grow by 4q per stage (no
// reduction until the consumer's Shoup or Montgomery product); inverse
// (Gentleman-Sande) butterflies keep [0, 4q).  Both take their products with
// a three-partial-product Shoup quotient estimate, result in [0, 4q).  Twiddles are (w, Shoup) pairs,
// one 16-byte load per butterfly.
#pragma once
#include "modarith.cuh"

namespace hespmv {

constexpr int kNttThreads = 256;
constexpr int kNttTile = 2048;  // words per CTA

// (x, y) -> (x + w y, x - w y + 4q) without reducing x: w y is taken in
// [0, 4q), so each stage raises the bound by at most 4q.  Inputs below 16q
// (base-conversion sums of up to four lazy products) stay below
// (16 + 4 log2 N) q <= 76q < 2^57 after a whole transform; when the
// conversion also forms stage 0's products (below 4 alpha q <= 16q, see
// fwd_round), that stage adds up to 16q: below 88q < 2^57.
__device__ __forceinline__ void ct_bfly(uint64_t &x, uint64_t &y, uint64_t w, uint64_t ws,
                                        uint64_t q, uint64_t q2) {
    const uint64_t t = mul_shoup_lazy4(y, w, ws, q);
    y = x + 2 * q2 - t;
    x = x + t;
}

// any 64-bit value -> [0, q) (Shoup product by 1)
__device__ __forceinline__ uint64_t reduce_full(uint64_t x, uint64_t q, uint64_t one_s) {
    return mul_shoup(x, 1, one_s, q);
}

// x, y in [0, 4q) -> (x + y, (x - y) w) in [0, 4q)  (q2 = 2q)
__device__ __forceinline__ void gs_bfly(uint64_t &x, uint64_t &y, uint64_t w, uint64_t ws,
                                        uint64_t q, uint64_t q2) {
    const uint64_t q4 = 2 * q2;
    uint64_t u = x + y;
    u = u >= q4 ? u - q4 : u;
    const uint64_t v = mul_shoup_lazy4(x + q4 - y, w, ws, q);
    x = u;
    y = v;
}

__device__ __forceinline__ uint64_t reduce4(uint64_t x, uint64_t q, uint64_t q2) {
    x = x >= q2 ? x - q2 : x;
    return x >= q ? x - q : x;
}

template <int LOGM, int S0, int NS>
__device__ __forceinline__ int elem_pos(int j, int e) {
    constexpr int LO = (1 << LOGM) >> (S0 + NS);
    const int G = j * (8 >> NS) + (e >> NS);
    const int k = e & ((1 << NS) - 1);
    const int lo = G % LO, hi = G / LO;
    return hi * ((1 << LOGM) >> S0) + k * LO + lo;
}

// local group of value e at local stage S0 + u
template <int LOGM, int S0, int NS>
__device__ __forceinline__ int elem_group(int j, int e, int u) {
    constexpr int LO = (1 << LOGM) >> (S0 + NS);
    const int G = j * (8 >> NS) + (e >> NS);
    const int k = e & ((1 << NS) - 1);
    return (G / LO) * (1 << u) + (k >> (NS - u));
}

typedef ulonglong2 TwPair;  // (w, floor(w 2^64 / q))

// PRE > 0 (first round of a column pass only: S0 = 0, twb = 1, where stage
// 0 has the single twiddle psi^bitrev(1)): the caller has already formed
// that stage's products, v[e + 4] = w * y below PRE * q, so stage 0 is
// (x, t) -> (x + t, x + PRE q - t) without multiplies.
template <int LOGM, int S0, int NS, int PRE = 0>
__device__ __forceinline__ void fwd_round(uint64_t (&v)[8], int j, uint32_t twb,
                                          const TwPair *__restrict__ tw, uint64_t q) {
    static_assert(PRE == 0 || (S0 == 0 && NS == 3), "stage 0 products only in a first round");
    const uint64_t q2 = 2 * q;
#pragma unroll
    for (int u = 0; u < NS; ++u) {
        const int dist = 1 << (NS - 1 - u);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            if ((e & ((1 << NS) - 1)) & dist) continue;
            if (PRE > 0 && u == 0) {
                const uint64_t t = v[e + dist];
                v[e + dist] = v[e] + PRE * q - t;
                v[e] += t;
                continue;
            }
            const uint32_t ti = (twb << (S0 + u)) + elem_group<LOGM, S0, NS>(j, e, u);
            const TwPair p = __ldg(tw + ti);
            ct_bfly(v[e], v[e + dist], p.x, p.y, q, q2);
        }
    }
}

// inverse round: stages S0+NS-1 down to S0; `last` folds the final
// constants (c_lo for the upper output, c_hi for the lower) into stage 0
template <int LOGM, int S0, int NS>
__device__ __forceinline__ void inv_round(uint64_t (&v)[8], int j, uint32_t twb,
                                          const TwPair *__restrict__ itw, uint64_t q) {
    const uint64_t q2 = 2 * q;
#pragma unroll
    for (int u = NS - 1; u >= 0; --u) {
        const int dist = 1 << (NS - 1 - u);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            if ((e & ((1 << NS) - 1)) & dist) continue;
            const uint32_t ti = (twb << (S0 + u)) + elem_group<LOGM, S0, NS>(j, e, u);
            const TwPair p = __ldg(itw + ti);
            gs_bfly(v[e], v[e + dist], p.x, p.y, q, q2);
        }
    }
}

// Final inverse stage 0 of a full transform (twb == 1, S0 == 0): outputs are
// scaled by the given constants and fully reduced:
//   upper = (x + y) * c0,   lower = (x - y) * c1   (c1 includes psi^-bitrev(1))
template <int LOGM, int NS>
__device__ __forceinline__ void inv_round_last(uint64_t (&v)[8], int j, uint32_t twb,
                                               const TwPair *__restrict__ itw, uint64_t q,
                                               uint64_t c0, uint64_t c0s, uint64_t c1,
                                               uint64_t c1s) {
    const uint64_t q2 = 2 * q;
#pragma unroll
    for (int u = NS - 1; u >= 1; --u) {
        const int dist = 1 << (NS - 1 - u);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            if ((e & ((1 << NS) - 1)) & dist) continue;
            const uint32_t ti = (twb << u) + elem_group<LOGM, 0, NS>(j, e, u);
            const TwPair p = __ldg(itw + ti);
            gs_bfly(v[e], v[e + dist], p.x, p.y, q, q2);
        }
    }
    const int dist = 1 << (NS - 1);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        if ((e & ((1 << NS) - 1)) & dist) continue;
        const uint64_t x = v[e], y = v[e + dist];
        v[e] = mul_shoup(x + y, c0, c0s, q);
        v[e + dist] = mul_shoup(x + 2 * q2 - y, c1, c1s, q);
    }
}

// Round schedules: forward rounds of 3 stages, the remainder last.
template <int LOGM>
struct Sched {
    static constexpr int R0 = 3;
    static constexpr int R1 = LOGM - 3 >= 3 ? 3 : LOGM - 3;
    static constexpr int R2 = LOGM - 3 - R1;  // 0, 1 or 2
};

}  // namespace hespmv

namespace hespmv {

// In the last round of every pass, thread j holds the 8 consecutive
// positions 8j .. 8j+7: row passes move them with four 16-byte accesses.
__device__ __forceinline__ void load8(uint64_t (&v)[8], const uint64_t *p) {
    const ulonglong2 *s = (const ulonglong2 *)p;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const ulonglong2 t = s[k];
        v[2 * k] = t.x;
        v[2 * k + 1] = t.y;
    }
}
__device__ __forceinline__ void store8(uint64_t *p, const uint64_t (&v)[8]) {
    ulonglong2 *d = (ulonglong2 *)p;
#pragma unroll
    for (int k = 0; k < 4; ++k) d[k] = make_ulonglong2(v[2 * k], v[2 * k + 1]);
}

// Positions of a thread's 8 values in the first and last forward rounds.
template <int LOGM>
struct Pass {
    static constexpr int R1 = Sched<LOGM>::R1, R2 = Sched<LOGM>::R2;
    static constexpr int LS0 = R2 > 0 ? 3 + R1 : 3;
    static constexpr int LNS = R2 > 0 ? R2 : R1;
    __device__ static __forceinline__ int first(int j, int e) { return elem_pos<LOGM, 0, 3>(j, e); }
    __device__ static __forceinline__ int last(int j, int e) { return elem_pos<LOGM, LS0, LNS>(j, e); }
};

// The barrier between the rounds of a pass: the whole CTA, or only the warp
// when the index map keeps every warp's values in a region of its own (a row
// tile whose rows are each held by one warp's threads).
template <class SIdx>
__device__ __forceinline__ void tile_sync() {
    if constexpr (SIdx::kWarpLocal)
        __syncwarp();
    else
        __syncthreads();
}

// Forward sub-transform of one tile.  On entry v[e] holds the element at
// Pass::first(j, e); on return the result at Pass::last(j, e), raised by at
// most 2q per stage (unreduced).
// `si` maps a position to its shared-memory word.  Starts with a barrier, so
// a CTA can run it repeatedly on the same shared buffer.
// PRE > 0: column pass (twb = 1) whose stage-0 products the caller formed
// (see fwd_round).
template <int LOGM, int PRE = 0, class SIdx>
__device__ __forceinline__ void fwd_body(uint64_t (&v)[8], int j, uint32_t twb, uint64_t *sm,
                                         SIdx si, const TwPair *__restrict__ tw, uint64_t q) {
    constexpr int R1 = Sched<LOGM>::R1, R2 = Sched<LOGM>::R2;
    fwd_round<LOGM, 0, 3, PRE>(v, j, twb, tw, q);
    tile_sync<SIdx>();
#pragma unroll
    for (int e = 0; e < 8; ++e) sm[si(elem_pos<LOGM, 0, 3>(j, e))] = v[e];
    tile_sync<SIdx>();
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = sm[si(elem_pos<LOGM, 3, R1>(j, e))];
    fwd_round<LOGM, 3, R1>(v, j, twb, tw, q);
    if constexpr (R2 > 0) {
        tile_sync<SIdx>();
#pragma unroll
        for (int e = 0; e < 8; ++e) sm[si(elem_pos<LOGM, 3, R1>(j, e))] = v[e];
        tile_sync<SIdx>();
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = sm[si(elem_pos<LOGM, 3 + R1, R2>(j, e))];
        fwd_round<LOGM, 3 + R1, R2>(v, j, twb, tw, q);
    }
}

// Inverse sub-transform of one tile.  On entry v[e] holds the element at
// Pass::last(j, e) (in [0, 4q)); on return Pass::first(j, e).  With FOLD the
// final stage scales by (c0, c1) and reduces fully (only for the last pass of
// a transform, twb == 1); otherwise outputs are in [0, 4q).
template <int LOGM, bool FOLD, class SIdx>
__device__ __forceinline__ void inv_body(uint64_t (&v)[8], int j, uint32_t twb, uint64_t *sm,
                                         SIdx si, const TwPair *__restrict__ itw, uint64_t q,
                                         uint64_t c0 = 0, uint64_t c0s = 0, uint64_t c1 = 0,
                                         uint64_t c1s = 0) {
    constexpr int R1 = Sched<LOGM>::R1, R2 = Sched<LOGM>::R2;
    if constexpr (R2 > 0) {
        inv_round<LOGM, 3 + R1, R2>(v, j, twb, itw, q);
        tile_sync<SIdx>();
#pragma unroll
        for (int e = 0; e < 8; ++e) sm[si(elem_pos<LOGM, 3 + R1, R2>(j, e))] = v[e];
        tile_sync<SIdx>();
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = sm[si(elem_pos<LOGM, 3, R1>(j, e))];
    }
    inv_round<LOGM, 3, R1>(v, j, twb, itw, q);
    tile_sync<SIdx>();
#pragma unroll
    for (int e = 0; e < 8; ++e) sm[si(elem_pos<LOGM, 3, R1>(j, e))] = v[e];
    tile_sync<SIdx>();
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = sm[si(elem_pos<LOGM, 0, 3>(j, e))];
    if constexpr (FOLD)
        inv_round_last<LOGM, 3>(v, j, twb, itw, q, c0, c0s, c1, c1s);
    else
        inv_round<LOGM, 0, 3>(v, j, twb, itw, q);
}

// Shared-memory index maps: column tiles (row-major, TC columns) and row
// tiles (TR rows of M words).
template <int TC>
struct ColIdx {
    static constexpr bool kWarpLocal = false;
    int cc;
    __device__ __forceinline__ int operator()(int pos) const { return pos * TC + cc; }
};
// Row tiles get one padding word per 8 so that the strided positions of
// the later rounds fall into distinct banks.
template <int M>
struct RowIdx {
    static constexpr bool kWarpLocal = false;
    int rr;
    __device__ __forceinline__ int operator()(int pos) const {
        return rr * (M + M / 8) + pos + (pos >> 3);
    }
};
// The same map for a row tile whose row rr is held by threads rr * M / 8 ..
// rr * M / 8 + M / 8 - 1 (M <= 256: one warp holds whole rows), so the
// exchanges between rounds need only warp barriers.  A caller that reuses
// the shared buffer for anything else separates the uses with a CTA barrier.
template <int M>
struct RowIdxW : RowIdx<M> {
    static_assert(M / 8 <= 32 && 32 % (M / 8) == 0, "a row within one warp");
    static constexpr bool kWarpLocal = true;
    __device__ __forceinline__ explicit RowIdxW(int r) : RowIdx<M>{r} {}
};
constexpr int kRowTileWords = kNttTile + kNttTile / 8;

}  // namespace hespmv
