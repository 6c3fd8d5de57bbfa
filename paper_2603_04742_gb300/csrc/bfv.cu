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

// acc[0..W) = centred sum_i y_i * hat_i mod M (residues res[i * stride])
__device__ void crt_centred(uint64_t *acc, const uint64_t *res, int64_t stride, int n, int W,
                            const ModConst *mc, const uint64_t *hat, const uint64_t *hat_inv,
                            const uint64_t *M, const uint64_t *Mhalf, const uint64_t *tq) {
    for (int w = 0; w < W; ++w) acc[w] = 0;
    for (int i = 0; i < n; ++i) {
        const uint64_t q = mc[i].q;
        uint64_t x = res[(int64_t)i * stride];
        if (tq) x = mul_shoup(x, tq[2 * i], tq[2 * i + 1], q);     // t * x mod q
        const uint64_t y = mul_shoup(x, hat_inv[2 * i], hat_inv[2 * i + 1], q);
        const uint64_t *h = hat + (int64_t)i * W;
        uint64_t carry = 0;
        for (int w = 0; w < W; ++w) {
            const uint64_t lo = h[w] * y, hi = __umul64hi(h[w], y);
            uint64_t s = acc[w] + lo;
            uint64_t c1 = s < lo;
            s += carry;
            c1 += s < carry;
            acc[w] = s;
            carry = hi + c1;
        }
    }
    // reduce below M (the sum is below n M), then centre
    for (int it = 0; it < n; ++it) {
        bool ge = true;
        for (int w = W - 1; w >= 0; --w)
            if (acc[w] != M[w]) {
                ge = acc[w] > M[w];
                break;
            }
        if (!ge) break;
        uint64_t br = 0;
        for (int w = 0; w < W; ++w) {
            const uint64_t d = acc[w] - M[w] - br;
            br = (acc[w] < M[w] || (acc[w] == M[w] && br)) ? 1 : 0;
            acc[w] = d;
        }
    }
    bool gt = false;  // acc > Mhalf
    for (int w = W - 1; w >= 0; --w)
        if (acc[w] != Mhalf[w]) {
            gt = acc[w] > Mhalf[w];
            break;
        }
    if (gt) {
        uint64_t br = 0;
        for (int w = 0; w < W; ++w) {
            const uint64_t d = acc[w] - M[w] - br;
            br = (acc[w] < M[w] || (acc[w] == M[w] && br)) ? 1 : 0;
            acc[w] = d;
        }
    }
}

// two's complement W-word value mod p; pw[k] = 2^(64 k) mod p for k <= W
__device__ uint64_t mod_word(const uint64_t *a, int W, const ModConst &m, const uint64_t *pw) {
    uint64_t r = 0;
    for (int w = 0; w < W; ++w) {
        const uint64_t aw = barrett_reduce(0, a[w], m.q, m.mu, m.k);
        r = add_mod(r, mul_mod(aw, pw[w], m), m.q);
    }
    if ((int64_t)a[W - 1] < 0) r = sub_mod(r, pw[W], m.q);  // minus 2^(64 W)
    return r;
}

// 2: centred extension of the four input polynomials to B
__global__ void k_bfv_extend(BfvArgs a, const uint64_t *coef, uint64_t *ext, int64_t total) {
    const int64_t N = 1LL << a.log2n, LN = (int64_t)a.L * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t poly = i >> a.log2n, k = i & (N - 1);  // poly = item * 4 + p
        uint64_t x[kMaxW];
        crt_centred(x, coef + poly * LN + k, N, a.L, a.wq, a.mc, a.k + a.o.qhat, a.k + a.o.qhat_inv,
                    a.k + a.o.Q, a.k + a.o.Qhalf, nullptr);
        uint64_t *out = ext + poly * (int64_t)a.nB * N + k;
        for (int j = 0; j < a.nB; ++j)
            out[(int64_t)j * N] = mod_word(x, a.wq, a.mc[a.iB + j], a.k + a.o.pow_b + (int64_t)j * (a.wq + 1));
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
__global__ void k_bfv_scale(BfvArgs a, const uint64_t *d, uint64_t *z, int64_t total) {
    const int64_t N = 1LL << a.log2n, LB = a.L + a.nB;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t comp = i >> a.log2n, k = i & (N - 1);  // comp = item * 3 + c
        const uint64_t *dq = d + comp * LB * N + k, *db = dq + (int64_t)a.L * N;
        uint64_t r[kMaxW];
        // r = [t d]_Q, centred
        crt_centred(r, dq, N, a.L, a.wq, a.mc, a.k + a.o.qhat, a.k + a.o.qhat_inv, a.k + a.o.Q,
                    a.k + a.o.Qhalf, a.k + a.o.t_q);
        // z mod b_j = (t d_j - r) Q^-1, kept in place of d's B residues (registers)
        uint64_t zb[kMaxW];
        for (int j = 0; j < a.nB; ++j) {
            const ModConst m = a.mc[a.iB + j];
            const uint64_t *tb = a.k + a.o.t_b + 2 * j, *qi = a.k + a.o.qinv_b + 2 * j;
            const uint64_t td = mul_shoup(db[(int64_t)j * N], tb[0], tb[1], m.q);
            const uint64_t rj = mod_word(r, a.wq, m, a.k + a.o.pow_b + (int64_t)j * (a.wq + 1));
            zb[j] = mul_shoup(sub_mod(td, rj, m.q), qi[0], qi[1], m.q);
        }
        // z exactly from its B residues, then to every q_i
        uint64_t zz[kMaxW];
        crt_centred(zz, zb, 1, a.nB, a.wb, a.mc + a.iB, a.k + a.o.bhat, a.k + a.o.bhat_inv, a.k + a.o.B,
                    a.k + a.o.Bhalf, nullptr);
        uint64_t *out = z + comp * (int64_t)a.L * N + k;
        for (int l = 0; l < a.L; ++l)
            out[(int64_t)l * N] = mod_word(zz, a.wb, a.mc[l], a.k + a.o.pow_q + (int64_t)l * (a.wb + 1));
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
    k_bfv_extend<<<grid_for(total, 128), 128, 0, st>>>(a, coef, ext, total);
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
    k_bfv_scale<<<grid_for(total, 128), 128, 0, st>>>(a, d, out, total);
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
