// BFV HE-Mult: the integer tensor of the centred inputs, scaled by t/Q and
// rounded, exactly (Fan-Vercauteren's definition; the paper's Pyfhel/BFV).
//
// For n ciphertext pairs (a, b), NTT domain over Q:
//  1. a, b to coefficients over Q (INTT);
//  2. each coefficient's centred value x in (-Q/2, Q/2] by exact Chinese
//     remaindering (multi-word), reduced to every prime of the auxiliary
//     basis B;
//  3. NTT over B; tensor d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1 over Q u B
//     (Q B > N Q^2 holds the integer products exactly); INTT over Q u B;
//  4. z = round(t d / Q) = (t d - r) / Q with r = [t d]_Q centred (|r| < Q/2,
//     no ties since Q is odd and prime to t): r exactly from the Q residues,
//     z mod b_j = (t d_j - r mod b_j) Q^-1, then z exactly from its B residues
//     (B > 2|z|) and reduced to every q_i;
//  5. NTT over Q.  Relinearisation follows as for BGV (with t = 1 keys).
// Multi-word values: little-endian 64-bit words, two's complement, at most
// 16 words (Q and B below 1000 bits).
#include <algorithm>

#include "kernels.h"

namespace hespmv {
namespace {

constexpr int kMaxW = 16;

struct BfvArgs {
    const ModConst *mc;
    const uint64_t *k;  // packed constants (BfvLayout offsets below)
    BfvLayout o;
    int L, nB, iB, wq, wb, log2n;
    uint64_t t;
};

// Word counts: WT > 0 fixes the width at compile time (loops unroll, values
// stay in registers); WT = 0 takes the runtime width w <= kMaxW.
template <int WT>
struct Wd {
    static constexpr int cap = WT > 0 ? WT : kMaxW;
    __device__ static __forceinline__ int of(int w) { return WT > 0 ? WT : w; }
};

// acc[0..W) += h[0..W) * y
template <int WT>
__device__ __forceinline__ void mw_addmul(uint64_t *acc, const uint64_t *h, uint64_t y, int w) {
    const int W = Wd<WT>::of(w);
    uint64_t carry = 0;
#pragma unroll
    for (int k = 0; k < Wd<WT>::cap; ++k) {
        if (k >= W) break;
        const uint64_t lo = h[k] * y, hi = __umul64hi(h[k], y);
        uint64_t s = acc[k] + lo;
        uint64_t c1 = s < lo;
        s += carry;
        c1 += s < carry;
        acc[k] = s;
        carry = hi + c1;
    }
}

// acc (below n M) -> its centred residue mod M, two's complement
template <int WT>
__device__ __forceinline__ void reduce_centre(uint64_t *acc, int n, int w, const uint64_t *M,
                                              const uint64_t *Mhalf) {
    const int W = Wd<WT>::of(w);
    for (int it = 0; it < n; ++it) {
        bool ge = true;
#pragma unroll
        for (int k = Wd<WT>::cap - 1; k >= 0; --k) {
            if (k >= W) continue;
            if (acc[k] != M[k]) {
                ge = acc[k] > M[k];
                break;
            }
        }
        if (!ge) break;
        uint64_t br = 0;
#pragma unroll
        for (int k = 0; k < Wd<WT>::cap; ++k) {
            if (k >= W) break;
            const uint64_t d = acc[k] - M[k] - br;
            br = (acc[k] < M[k] || (acc[k] == M[k] && br)) ? 1 : 0;
            acc[k] = d;
        }
    }
    bool gt = false;  // acc > Mhalf
#pragma unroll
    for (int k = Wd<WT>::cap - 1; k >= 0; --k) {
        if (k >= W) continue;
        if (acc[k] != Mhalf[k]) {
            gt = acc[k] > Mhalf[k];
            break;
        }
    }
    if (gt) {
        uint64_t br = 0;
#pragma unroll
        for (int k = 0; k < Wd<WT>::cap; ++k) {
            if (k >= W) break;
            const uint64_t d = acc[k] - M[k] - br;
            br = (acc[k] < M[k] || (acc[k] == M[k] && br)) ? 1 : 0;
            acc[k] = d;
        }
    }
}

// acc[0..W) = centred sum_i [x_i hat_i^-1] hat_i mod M for residues
// x_i = res[i * stride] (times t first when tq is given)
template <int WT>
__device__ __forceinline__ void crt_centred(uint64_t *acc, const uint64_t *res, int64_t stride, int n,
                                            int w, const ModConst *mc, const uint64_t *hat,
                                            const uint64_t *hat_inv, const uint64_t *M,
                                            const uint64_t *Mhalf, const uint64_t *tq) {
    const int W = Wd<WT>::of(w);
#pragma unroll
    for (int k = 0; k < Wd<WT>::cap; ++k)
        if (k < W) acc[k] = 0;
    for (int i = 0; i < n; ++i) {
        const uint64_t q = mc[i].q;
        uint64_t x = res[(int64_t)i * stride];
        if (tq) x = mul_shoup(x, tq[2 * i], tq[2 * i + 1], q);     // t * x mod q
        const uint64_t y = mul_shoup(x, hat_inv[2 * i], hat_inv[2 * i + 1], q);
        mw_addmul<WT>(acc, hat + (int64_t)i * W, y, w);
    }
    reduce_centre<WT>(acc, n, w, M, Mhalf);
}

// two's complement W-word value mod q; pw[2k], pw[2k+1] = 2^(64 k) mod q and
// its Shoup companion, k <= W: one lazy Shoup product per word (< 2q each,
// the sum stays below 2^64), one full reduction at the end
template <int WT>
__device__ __forceinline__ uint64_t mod_word(const uint64_t *a, int w, const ModConst &m,
                                             const uint64_t *pw) {
    const int W = Wd<WT>::of(w);
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < Wd<WT>::cap; ++k) {
        if (k >= W) break;
        s += mul_shoup_lazy(a[k], pw[2 * k], pw[2 * k + 1], m.q);
    }
    uint64_t r = mul_shoup(s, 1, m.one_s, m.q);
    if ((int64_t)a[W - 1] < 0) r = sub_mod(r, pw[2 * W], m.q);  // minus 2^(64 W)
    return r;
}

// 2: centred extension of the four input polynomials to B
template <int WQ>
__global__ void k_bfv_extend(BfvArgs a, const uint64_t *coef, uint64_t *ext, int64_t total) {
    const int64_t N = 1LL << a.log2n, LN = (int64_t)a.L * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t poly = i >> a.log2n, k = i & (N - 1);  // poly = item * 4 + p
        uint64_t x[Wd<WQ>::cap];
        crt_centred<WQ>(x, coef + poly * LN + k, N, a.L, a.wq, a.mc, a.k + a.o.qhat, a.k + a.o.qhat_inv,
                        a.k + a.o.Q, a.k + a.o.Qhalf, nullptr);
        uint64_t *out = ext + poly * (int64_t)a.nB * N + k;
        for (int j = 0; j < a.nB; ++j)
            out[(int64_t)j * N] = mod_word<WQ>(x, a.wq, a.mc[a.iB + j],
                                               a.k + a.o.pow_b + (int64_t)j * 2 * (a.wq + 1));
    }
}

// 3: tensor over Q u B (NTT domain): a, b [n][2][L][N]; ext [n][4][nB][N]
// (a0, a1, b0, b1); d [n][3][L + nB][N]
__global__ void k_bfv_tensor(BfvArgs a, const uint64_t *A, const uint64_t *Bc, const uint64_t *ext,
                             uint64_t *d, int64_t total) {
    const int64_t N = 1LL << a.log2n, LB = a.L + a.nB, LN = (int64_t)a.L * N, BN = (int64_t)a.nB * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t item = i / (LB * N), r = i - item * LB * N;
        const int l = (int)(r >> a.log2n);
        const int64_t k = r & (N - 1);
        uint64_t a0, a1, b0, b1;
        ModConst m;
        if (l < a.L) {
            m = a.mc[l];
            const int64_t o = item * 2 * LN + (int64_t)l * N + k;
            a0 = A[o], a1 = A[o + LN], b0 = Bc[o], b1 = Bc[o + LN];
        } else {
            const int j = l - a.L;
            m = a.mc[a.iB + j];
            const int64_t o = item * 4 * BN + (int64_t)j * N + k;
            a0 = ext[o], a1 = ext[o + BN], b0 = ext[o + 2 * BN], b1 = ext[o + 3 * BN];
        }
        uint64_t *o = d + item * 3 * LB * N + (int64_t)l * N + k;
        o[0] = mul_mod(a0, b0, m);
        o[LB * N] = add_mod(mul_mod(a0, b1, m), mul_mod(a1, b0, m), m.q);
        o[2 * LB * N] = mul_mod(a1, b1, m);
    }
}

// 4: scale and round, coefficient domain: d [n][3][L + nB][N] -> z [n][3][L][N]
template <int WQ, int WB>
__global__ void k_bfv_scale(BfvArgs a, const uint64_t *d, uint64_t *z, int64_t total) {
    const int64_t N = 1LL << a.log2n, LB = a.L + a.nB;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t comp = i >> a.log2n, k = i & (N - 1);  // comp = item * 3 + c
        const uint64_t *dq = d + comp * LB * N + k, *db = dq + (int64_t)a.L * N;
        uint64_t r[Wd<WQ>::cap];
        // r = [t d]_Q, centred
        crt_centred<WQ>(r, dq, N, a.L, a.wq, a.mc, a.k + a.o.qhat, a.k + a.o.qhat_inv, a.k + a.o.Q,
                        a.k + a.o.Qhalf, a.k + a.o.t_q);
        // z mod b_j = (t d_j - r) Q^-1, accumulated straight into z's exact
        // reconstruction from its B residues
        uint64_t zz[Wd<WB>::cap];
        const int W = Wd<WB>::of(a.wb);
#pragma unroll
        for (int u = 0; u < Wd<WB>::cap; ++u)
            if (u < W) zz[u] = 0;
        for (int j = 0; j < a.nB; ++j) {
            const ModConst m = a.mc[a.iB + j];
            const uint64_t *tb = a.k + a.o.t_b + 2 * j, *qi = a.k + a.o.qinv_b + 2 * j;
            const uint64_t *bi = a.k + a.o.bhat_inv + 2 * j;
            const uint64_t td = mul_shoup(db[(int64_t)j * N], tb[0], tb[1], m.q);
            const uint64_t rj = mod_word<WQ>(r, a.wq, m, a.k + a.o.pow_b + (int64_t)j * 2 * (a.wq + 1));
            const uint64_t zj = mul_shoup(sub_mod(td, rj, m.q), qi[0], qi[1], m.q);
            mw_addmul<WB>(zz, a.k + a.o.bhat + (int64_t)j * W, mul_shoup(zj, bi[0], bi[1], m.q), a.wb);
        }
        reduce_centre<WB>(zz, a.nB, a.wb, a.k + a.o.B, a.k + a.o.Bhalf);
        uint64_t *out = z + comp * (int64_t)a.L * N + k;
        for (int l = 0; l < a.L; ++l)
            out[(int64_t)l * N] = mod_word<WB>(zz, a.wb, a.mc[l],
                                               a.k + a.o.pow_q + (int64_t)l * 2 * (a.wb + 1));
    }
}

// plaintext m in [0, t) (coefficients) -> Delta * m over Q
__global__ void k_bfv_delta(const uint64_t *m, uint64_t *out, int64_t total, int log2n, int L,
                            const ModConst *mc, const uint64_t *delta) {
    const int64_t N = 1LL << log2n, LN = (int64_t)L << log2n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t item = i / LN, r = i - item * LN;
        const int l = (int)(r >> log2n);
        const ModConst q = mc[l];
        const uint64_t v = barrett_reduce(0, m[(item << log2n) + (r & (N - 1))], q.q, q.mu, q.k);
        out[i] = mul_mod(v, delta[2 * l], q);
    }
}

BfvArgs bfv_args(const Ctx &c) {
    const HostTables &h = c.c->h;
    BfvArgs a;
    a.mc = c.c->d.mc;
    a.k = c.c->d.bfv_const;
    a.o = bfv_layout(h);
    a.L = h.L;
    a.nB = h.nB;
    a.iB = h.iB;
    a.wq = h.wq;
    a.wb = h.wb;
    a.log2n = h.log2n;
    a.t = h.t;
    return a;
}

unsigned grid_for(int64_t total, int threads) {
    const int64_t b = (total + threads - 1) / threads;
    return (unsigned)std::min<int64_t>(b, 152 * 64);
}

}  // namespace

size_t bfv_tensor_words(const Ctx &c, size_t n) {
    const HostTables &h = c.c->h;
    return n * (size_t)(7 * h.L + 7 * h.nB) * c.N;
}

cudaError_t bfv_tensor(const Ctx &c, const uint64_t *A, const uint64_t *B, uint64_t *out, size_t n,
                       uint64_t *scratch, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const BfvArgs a = bfv_args(c);
    const int64_t N = c.N, L = c.L, nB = a.nB, LN = L * N, LB = L + nB;
    uint64_t *coef = scratch;                    // [n][4][L][N]
    uint64_t *ext = coef + n * 4 * LN;           // [n][4][nB][N]
    uint64_t *d = ext + n * 4 * nB * N;          // [n][3][L + nB][N]
    cudaError_t e;
    // 1. a, b -> coefficients over Q
    if ((e = cudaMemcpy2DAsync(coef, 4 * LN * 8, A, 2 * LN * 8, 2 * LN * 8, n, cudaMemcpyDeviceToDevice, st)))
        return e;
    if ((e = cudaMemcpy2DAsync(coef + 2 * LN, 4 * LN * 8, B, 2 * LN * 8, 2 * LN * 8, n,
                               cudaMemcpyDeviceToDevice, st)))
        return e;
    if ((e = launch_ntt(c, coef, 0, (int)L, (int)(4 * n), LN, true, st))) return e;
    // 2. centred extension to B
    int r = prof_begin(c, "k_bfv_extend", st);
    int64_t total = (int64_t)n * 4 * N;
    switch (a.wq) {
        case 4: k_bfv_extend<4><<<grid_for(total, 128), 128, 0, st>>>(a, coef, ext, total); break;
        case 5: k_bfv_extend<5><<<grid_for(total, 128), 128, 0, st>>>(a, coef, ext, total); break;
        case 8: k_bfv_extend<8><<<grid_for(total, 128), 128, 0, st>>>(a, coef, ext, total); break;
        default: k_bfv_extend<0><<<grid_for(total, 128), 128, 0, st>>>(a, coef, ext, total); break;
    }
    prof_end(c, r, st);
    if ((e = launch_ntt(c, ext, a.iB, (int)nB, (int)(4 * n), nB * N, false, st))) return e;
    // 3. tensor over Q u B, back to coefficients
    r = prof_begin(c, "k_bfv_tensor", st);
    total = (int64_t)n * LB * N;
    k_bfv_tensor<<<grid_for(total, 256), 256, 0, st>>>(a, A, B, ext, d, total);
    prof_end(c, r, st);
    if ((e = launch_ntt(c, d, 0, (int)L, (int)(3 * n), LB * N, true, st))) return e;
    if ((e = launch_ntt(c, d + LN, a.iB, (int)nB, (int)(3 * n), LB * N, true, st))) return e;
    // 4. scale and round, 5. NTT over Q
    r = prof_begin(c, "k_bfv_scale", st);
    total = (int64_t)n * 3 * N;
    if (a.wq == 4 && a.wb == 5)
        k_bfv_scale<4, 5><<<grid_for(total, 128), 128, 0, st>>>(a, d, out, total);
    else if (a.wq == 5 && a.wb == 6)
        k_bfv_scale<5, 6><<<grid_for(total, 128), 128, 0, st>>>(a, d, out, total);
    else if (a.wq == 8 && a.wb == 9)
        k_bfv_scale<8, 9><<<grid_for(total, 128), 128, 0, st>>>(a, d, out, total);
    else
        k_bfv_scale<0, 0><<<grid_for(total, 128), 128, 0, st>>>(a, d, out, total);
    prof_end(c, r, st);
    if ((e = launch_ntt(c, out, 0, (int)L, (int)(3 * n), LN, false, st))) return e;
    return cudaGetLastError();
}

cudaError_t op_bfv_delta(const Ctx &c, const uint64_t *m, uint64_t *out, size_t n, cudaStream_t st) {
    const int64_t total = (int64_t)n * c.L * c.N;
    if (total == 0) return cudaSuccess;
    int r = prof_begin(c, "k_bfv_delta", st);
    k_bfv_delta<<<grid_for(total, 256), 256, 0, st>>>(m, out, total, c.log2n, c.L, c.c->d.mc,
                                                      c.c->d.bfv_delta);
    prof_end(c, r, st);
    return cudaGetLastError();
}

}  // namespace hespmv
