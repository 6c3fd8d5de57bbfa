// Internal structures of the hespmv library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/hespmv.h"
#include "modarith.cuh"

namespace hespmv {

constexpr int kMaxPrimes = 21;  // L + K + 1 (t) <= 16 + 4 + 1

// Host-side parameter tables (built once per context, then uploaded).
struct HostTables {
    int log2n = 0, N = 0, L = 0, K = 0, dnum = 0, alpha = 0, slots = 0;
    int scheme = 0, scale_bits = 0, mask_scale_bits = 0;  // CKKS: scales 2^bits
    // BFV: auxiliary basis B = table entries [iB, iB + nB); multi-word
    // constants of exact Chinese remaindering over Q (wq words) and B (wb)
    int nB = 0, iB = 0, wq = 0, wb = 0;
    int pack_bits = 0;  // bits per residue of packed ciphertexts: max bit length of q_0..q_{L-1}
    std::vector<uint64_t> bfv_delta;   // [L][2] floor(Q/t) mod q_i, Shoup pair
    std::vector<uint64_t> bfv_const;   // packed, see BfvLayout
    uint64_t bfv_qinv_t = 0;           // Q^-1 mod t (decryption)
    uint64_t t = 0;  // plaintext modulus (BGV); 1 for CKKS (its formulas' t)
    std::vector<uint64_t> q;     // L + K + 1 moduli: Q, then P, then t
    std::vector<uint64_t> psi;   // primitive 2N-th roots (index L+K: zeta for t)
    std::vector<ModConst> mc;    // per modulus
    // twiddles per modulus: [N][2] (psi^bitrev(k), Shoup) then [N][2] (psi^-bitrev(k), Shoup)
    std::vector<uint64_t> tw;
    // ModUp constants, per digit j, source prime i (local index), target l:
    //   qhat_inv[j][i] (Shoup pair) and qhat_mod[j][i][l] (Shoup pair)
    std::vector<uint64_t> modup_inv;   // [dnum][alpha][2]
    std::vector<uint64_t> modup_mod;   // [dnum][alpha][L+K][2]
    // ModDown constants: per special prime k: (t^-1 * Phat_k^-1 mod p_k) Shoup pair,
    // per (k, i): Phat_k mod q_i Shoup pair; per i: t mod q_i, P^-1 mod q_i Shoup pairs
    std::vector<uint64_t> md_pk;       // [K][2]
    std::vector<uint64_t> md_phat;     // [K][L][2]
    std::vector<uint64_t> md_t;        // [L][2]
    std::vector<uint64_t> md_pinv;     // [L][2]
    // gadget: P mod q_i (Shoup pair) for the Q primes
    std::vector<uint64_t> p_mod_q;     // [L][2]
    // P * 2^64 mod q_i: P in Montgomery form, for sums reduced by REDC
    std::vector<uint64_t> p_mont;      // [L]
    std::vector<uint64_t> p_mont2;     // [L] P * 2^128 mod q_i
    // slot positions in the NTT domain: [N/2] for row 0, then [N/2] for row 1
    std::vector<int32_t> slot_idx;
    // decryption CRT: per Q prime (Qhat_i^-1 mod q_i, Shoup) and (Qhat_i mod t, Shoup),
    // then (Q mod t, Shoup) and 1/q_i as doubles
    std::vector<uint64_t> dec;         // [L][4] + [2]
    std::vector<double> dec_inv_q;     // [L]
    std::vector<uint64_t> t_mod;       // t mod q_l, [L+K]
    // fused key switching: inverse-NTT fold constants (c0, c0 Shoup, c1, c1
    // Shoup) producing [x * Qhat^-1]_{q_i} (ks_zc, per Q prime) and
    // [x * t^-1 * Phat_k^-1]_{p_k} (ks_yc, per P prime); Phat_k * t mod q_i
    std::vector<uint64_t> ks_zc;       // [L][4]
    std::vector<uint64_t> ks_yc;       // [K][4]
    std::vector<uint64_t> md_phat_t;   // [K][L][2]
    // the same conversion factors times the first forward butterfly stage's
    // twiddle of the target prime (psi_l^bitrev(1), one per column pass):
    // the fused conversions form the products of that stage directly
    std::vector<uint64_t> modup_modw;  // [dnum][alpha][L+K][2]
    std::vector<uint64_t> md_phat_tw;  // [K][L][2]
};

// Device copies of the tables.
struct DevTables {
    ModConst *mc = nullptr;
    uint64_t *tw = nullptr;
    uint64_t *modup_inv = nullptr;
    uint64_t *modup_mod = nullptr;
    uint64_t *md_pk = nullptr;
    uint64_t *md_phat = nullptr;
    uint64_t *md_t = nullptr;
    uint64_t *md_pinv = nullptr;
    uint64_t *p_mod_q = nullptr;
    uint64_t *p_mont = nullptr;
    uint64_t *p_mont2 = nullptr;
    int32_t *slot_idx = nullptr;
    uint64_t *dec = nullptr;
    double *dec_inv_q = nullptr;
    uint64_t *t_mod = nullptr;
    uint64_t *ks_zc = nullptr;
    uint64_t *ks_yc = nullptr;
    uint64_t *md_phat_t = nullptr;
    uint64_t *modup_modw = nullptr;
    uint64_t *md_phat_tw = nullptr;
    uint64_t *bfv_delta = nullptr;
    uint64_t *bfv_const = nullptr;
    int *err = nullptr;  // device error word written by bounded waits
};

bool build_tables(const hespmv_params &p, HostTables &h, std::string &err);

// Offsets (words) of the BFV constants in HostTables::bfv_const
struct BfvLayout {
    int64_t qhat, Q, Qhalf, qhat_inv, bhat, B, Bhalf, bhat_inv, pow_b, pow_q, qinv_b, t_b, t_q, size;
};
BfvLayout bfv_layout(const HostTables &h);
bool bfv_tables(const hespmv_params &p, HostTables &h, std::string &err);
// BFV decryption of phase residues x [L][N] (coefficient domain):
// m = round(t [x]_Q / Q) mod t, exactly
void bfv_decrypt_coef(const HostTables &h, const uint64_t *x, uint64_t *m);

// Host-side bit reversal, primality and roots (used by the table builder).
uint32_t host_bitrev(uint32_t x, int bits);
uint32_t ntt_index_of_exponent(uint64_t e, int log2n);  // e odd, mod 2N

// ------------------------------------------------------------------ format
struct Chunk {
    int32_t h = 0, c = 0, part = 0;
    int64_t slot0 = 0;    // offset of this chunk's h*c slots in the concatenated arrays
};

struct Partition {
    int32_t row0 = 0, rows = 0;
    std::vector<int64_t> va;   // CSSC value array
    std::vector<int64_t> src;  // CSR position of each CSSC entry (real values)
    std::vector<int32_t> ci;   // CSSC column indices
    std::vector<int64_t> cp;   // Lmax + 1
    std::vector<int32_t> rm;   // local row of sorted row p
    int32_t chunk0 = 0, n_chunks = 0;
};

struct Plan {
    int32_t rows = 0, cols = 0, s = 0;
    int64_t nnz = 0;
    std::vector<Partition> parts;
    std::vector<Chunk> chunks;
    std::vector<int64_t> slot_vals;   // concatenated chunk slot values
    std::vector<int32_t> slot_ci;     // concatenated chunk slot column indices
    std::vector<int64_t> slot_src;    // CSR position of each slot value, -1 = padding
    bool has_values = true;           // integer values given (else positions only)
    bool has_src = false;             // slot_src filled (plans built from a CSR)
};

// Returns empty string on success.
std::string build_plan(int32_t rows, int32_t cols, int64_t nnz, const int64_t *rowptr,
                       const int32_t *colidx, const int64_t *vals, int32_t s, Plan &plan);
// Chunks (Algorithm 2) of every partition whose CP, VA and CI are set.
void chunk_plan(Plan &plan);

// CKKS encoding of real slot values (host, double-double; ckks_host.cpp)
struct CkksCodec;
CkksCodec *ckks_codec(int log2n);
void ckks_codec_free(CkksCodec *c);
// n <= N/2 values -> N integer coefficients at scale 2^scale_bits; "" or an error
std::string ckks_encode(const CkksCodec &C, const double *z, size_t n, int scale_bits,
                        int64_t *coef);
// N real coefficients -> the first n slot values times inv_scale
void ckks_decode(const CkksCodec &C, const double *coef, size_t n, double inv_scale, double *z);
// centred [x]_Q of residues x [L][N] as doubles (exact CRT, then rounding)
struct CrtReal;
CrtReal *crt_real(const uint64_t *q, int L);
void crt_real_free(CrtReal *c);
void crt_to_double(const CrtReal &c, const uint64_t *x, int N, double *out);
// totalSum rotation amounts of a chunk (r rows, c columns) in order; flags
// tell whether the step rotates the running sum (doubling) or the original.
void total_sum_steps(int32_t r, int32_t c, std::vector<int32_t> &steps,
                     std::vector<uint8_t> &from_original);

// ------------------------------------------------------------ profiling
// While enabled, each kernel launch is bracketed by two CUDA events recorded
// on the launch stream; collect() sums the elapsed times per kernel name.
struct Profiler {
    bool on = false;
    struct Rec {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<Rec> recs;
    std::vector<std::string> names;
    std::map<std::string, int> ids;
    std::vector<int64_t> launches;
    std::vector<double> ms;
    cudaError_t collect();
    void reset();
    ~Profiler();
};

// ------------------------------------------------------------ kernels (host launchers)
struct Ctx;
int prof_begin(const Ctx &c, const char *name, cudaStream_t st);
cudaError_t mulmod_rate(const HostTables &h, int kind, double *rate);
void prof_end(const Ctx &c, int rec, cudaStream_t st);
// NTT of n_items x n_limbs polynomials, item stride in words; limb k uses prime0 + k.
cudaError_t launch_ntt(const Ctx &c, uint64_t *data, int prime0, int n_limbs, int n_items,
                       int64_t item_stride, bool inverse, cudaStream_t st);

}  // namespace hespmv

namespace hespmv {
// Batched totalSum schedule of a set of matrices (Algorithm 4, rotations):
// chunks that rotate are processed in groups; per round, every rotating
// chunk's rotation runs as one batched key switch per Galois element, bits
// in increasing order (each chunk's own chain stays least significant first).
struct RotOp {
    enum Kind { kVInit, kCurFromProd, kCurFromV, kElem, kAdd } kind;
    uint32_t g = 0;         // Galois element (kElem)
    int m = 0;              // items
    int64_t a = -1, b = -1; // offsets of the index lists in d_idx (-1: identity)
};
// A persistent evaluation program resident on the device (api.cu builds it).
struct PersistPlan;
struct RotPlan {
    int GR = 0;             // group capacity
    std::vector<RotOp> ops;
    int32_t *d_idx = nullptr;
    size_t idx_bytes = 0;
};
}  // namespace hespmv

// The opaque handles of the C ABI.
struct hespmv_ctx {
    hespmv_params p{};
    hespmv::HostTables h;
    hespmv::DevTables d;
    std::string err;
    int device = 0;
    std::vector<std::pair<void *, size_t>> allocs;  // table/key blocks owned by the context
    size_t owned_bytes = 0;
    // keys (device)
    bool have_keys = false;
    bool has_sk = false;       // the secret key is present (keygen, or loaded with it)
    uint64_t *sk = nullptr;    // [L+K][N]
    uint64_t *pk = nullptr;    // [2][L][N]
    uint64_t *rlk = nullptr;   // [dnum][2][L+K][N]
    std::map<uint32_t, uint64_t *> gk;          // Galois element -> key
    std::map<uint32_t, int32_t *> perms;        // Galois element -> device permutation [N]
    std::map<int32_t, uint64_t *> masks;        // r -> mask plaintext [L][N]
    // workspace
    void *ws = nullptr;
    size_t ws_bytes = 0;
    hespmv::Profiler *prof = nullptr;
    // rotation schedules, keyed by the matrices' ids
    std::map<std::vector<uint64_t>, hespmv::RotPlan *> rot_plans;
    uint64_t next_uid = 1;
    // CUDA graphs of evaluations, keyed by workspace, matrices and buffers
    bool use_graphs = true;
    std::map<std::vector<uint64_t>, cudaGraphExec_t> graphs;
    cudaStream_t cap_stream = nullptr;
    // schedule choices (0: default); results do not depend on them
    size_t tune_G = 0;   // HE-Mult batch: ciphertexts per fused key switch
    size_t tune_GR = 0;  // totalSum round width: ciphertexts per rotation round
    int ks_split = 0;    // fused key switch: NTT split variant (column/row pass sizes)
    int rows_tma = 0;    // fused key switch: persistent TMA-fed forward row pass
    int persistent = 0;  // 1: one persistent launch per evaluation (tune_G = its HE-Mult group)
    int persist_blocks = 0;  // CTAs of the persistent launch (0: every resident CTA)
    int streams = 1;     // device evaluations: HE-Mult groups alternate over 1 or 2 streams
    // persistent evaluation programs, keyed by matrices, buffers, workspace and group
    std::map<std::vector<uint64_t>, hespmv::PersistPlan *> persist_plans;
    // staging for evaluations from host buffers, and the side stream and
    // events that overlap their uploads with the HE-Mult groups
    void *io = nullptr;
    size_t io_bytes = 0;
    int *err_host = nullptr;  // page-locked copy of the device error word (packed host path)
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> copy_events;
    // HE-Mult groups of host evaluations alternate between the evaluation
    // stream and this one (each with its own scratch), so that a group's
    // kernels fill the tails of the previous group's; joined by join_event
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t join_event = nullptr;
    int upload_groups = 0;  // upload groups of host evaluations (0: default)
    // pipelined packed host evaluations: kSlots staging slots used in turn; a
    // slot's uploads wait for slot_free[s], recorded when the evaluation that
    // used it last has copied its result out
    static constexpr int kSlots = 3;
    void *aio[kSlots] = {};
    size_t aio_bytes[kSlots] = {};
    cudaEvent_t slot_free[kSlots] = {};
    bool slot_used[kSlots] = {};
    int aslot = 0;
    // CKKS rescale: q_{L-1}^-1 mod q_i with Shoup companions, [L-1][2] (device, first use)
    uint64_t *rescale_inv = nullptr;
    // CKKS encoder tables and CRT constants (host, made on first use)
    hespmv::CkksCodec *codec = nullptr;
    hespmv::CrtReal *crt = nullptr;
};

struct hespmv_cssc {
    hespmv_ctx *ctx = nullptr;
    hespmv::Plan plan;
    std::vector<int32_t> steps;   // distinct rotation steps
    int64_t n_rot = 0, n_ks = 0;
    const uint64_t **d_masks = nullptr;  // device: mask plaintext of each chunk
    uint64_t uid = 0;                    // unique per context (schedule cache key)
    bool prepared = false;               // masks, mask table, permutations resident
    bool shape_only = false;             // chunk shapes without values, indices, RM
};

struct hespmv_ctbatch {
    hespmv_ctx *ctx = nullptr;
    uint64_t *data = nullptr;
    size_t n = 0;
    size_t bytes = 0;
};

namespace hespmv {
struct Ctx {
    const hespmv_ctx *c;
    int N, L, K, dnum, alpha, log2n;
    int ks_split, rows_tma;
};
inline Ctx view(const hespmv_ctx *c) {
    return Ctx{c, c->h.N, c->h.L, c->h.K, c->h.dnum, c->h.alpha, c->h.log2n, c->ks_split, c->rows_tma};
}
}  // namespace hespmv
