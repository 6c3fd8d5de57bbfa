// C-ABI entry points of hespmv: context and tables, key generation,
// client-side format and encryption, the cloud evaluation of Algorithms 1
// and 4, decryption, and the HE primitives.
#include <algorithm>
#include <cstring>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <initializer_list>
#include <mutex>
#include <set>
#include <thread>
#include <unordered_map>

#include <nvtx3/nvToolsExt.h>

#include "kernels.h"

using namespace hespmv;

namespace hespmv {
// A persistent evaluation program in one device block: the context's
// key-switch constants, phases, tile offsets, dependencies, key-switch
// instances, mask jobs, pointer tables and counters (PProg points into it).
struct PersistPlan {
    void *blob = nullptr;
    size_t bytes = 0;
    PProg prog{};
    int64_t n_ks = 0, n_phases = 0;  // key switches and phases of the program
};
}  // namespace hespmv

namespace {

const uint64_t kSecretStream = 1, kPkAStream = 2, kPkEStream = 3;
const uint64_t kEncBase = 1ull << 62;
// a dependency wait of the persistent kernel gives up after this long
const int64_t kPersistWaitNs = 4000000000ll;
uint64_t ksk_a_stream(uint64_t kid, uint64_t j) { return 16 + 2 * (kid * 64 + j); }

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// NVTX range for profilers (a no-op when none is attached)
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

#define FAIL(code, msg)        \
    do {                       \
        ctx->err = (msg);      \
        return (code);         \
    } while (0)

#define NEED_DEVICE(ctx)                                                      \
    do {                                                                      \
        if ((ctx)->device < 0) FAIL(HESPMV_E_INVALID, "host-only context");  \
    } while (0)

#define CK(x)                                                                          \
    do {                                                                               \
        cudaError_t _e = (x);                                                          \
        if (_e != cudaSuccess) FAIL(HESPMV_E_CUDA, std::string(#x) + ": " + cudaGetErrorString(_e)); \
    } while (0)

void *dev_alloc(hespmv_ctx *ctx, size_t bytes) {
    bytes = std::max<size_t>(bytes, 256);
    void *p = nullptr;
    if (ctx->p.alloc) {
        p = ctx->p.alloc(bytes, ctx->p.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void dev_free(hespmv_ctx *ctx, void *p) {
    if (!p) return;
    if (ctx->p.free)
        ctx->p.free(p, ctx->p.alloc_user);
    else
        cudaFree(p);
}

// allocation owned by the context until destroy
template <class T>
T *owned(hespmv_ctx *ctx, size_t count) {
    const size_t bytes = count * sizeof(T);
    void *p = dev_alloc(ctx, bytes);
    if (p) {
        ctx->allocs.push_back({p, bytes});
        ctx->owned_bytes += bytes;
    }
    return (T *)p;
}

template <class T>
bool upload(hespmv_ctx *ctx, T *&dst, const std::vector<T> &src) {
    dst = owned<T>(ctx, std::max<size_t>(src.size(), 1));
    if (!dst) return false;
    return cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
}

// workspace of at least `bytes`; reallocation waits for the device first
uint64_t *workspace(hespmv_ctx *ctx, size_t bytes) {
    if (ctx->ws_bytes >= bytes) return (uint64_t *)ctx->ws;
    cudaDeviceSynchronize();
    const size_t old = ctx->ws_bytes;  // grow by at least half, so creeping sizes reallocate rarely
    dev_free(ctx, ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    size_t want = std::max(bytes, old * 3 / 2);
    ctx->ws = dev_alloc(ctx, want);
    if (!ctx->ws) {
        ctx->ws = dev_alloc(ctx, bytes);
        want = bytes;
    }
    if (!ctx->ws) return nullptr;
    ctx->ws_bytes = want;
    return (uint64_t *)ctx->ws;
}

// words of key-switching scratch for n items
size_t ks_words(const Ctx &c, size_t n) {
    const size_t LK = c.L + c.K;
    return n * (size_t)c.N * (c.L + c.dnum * LK + 2 * LK + 2 * c.L);
}

// Hybrid key switch of n polynomials d (item stride d_stride words) with `key`;
// out [n][2][L][N] = ModDown(sum_j ModUp_j(d) * key_j) (+ add per add_mask).
cudaError_t keyswitch_n(const Ctx &c, const uint64_t *d, int64_t d_stride, const uint64_t *key,
                        uint64_t *out, const uint64_t *add, int64_t add_is, int64_t add_cs,
                        int add_mask, size_t n, uint64_t *scratch, cudaStream_t st) {
    if (ks_fused_supported(c))
        return keyswitch_fused(c, d, d_stride, key, out, add, add_is, add_cs, add_mask, n, scratch,
                               st);
    const int64_t N = c.N, L = c.L, LK = c.L + c.K;
    uint64_t *dcoef = scratch;
    uint64_t *ext = dcoef + n * L * N;
    uint64_t *acc = ext + n * c.dnum * LK * N;
    uint64_t *delta = acc + n * 2 * LK * N;
    cudaError_t e;
    if ((e = op_copy_strided(c, d, d_stride, dcoef, L * N, L * N, n, st))) return e;
    if ((e = launch_ntt(c, dcoef, 0, (int)L, (int)n, L * N, true, st))) return e;
    if ((e = op_modup(c, dcoef, ext, n, st))) return e;
    if ((e = launch_ntt(c, ext, 0, (int)LK, (int)(n * c.dnum), LK * N, false, st))) return e;
    if ((e = op_inner(c, ext, key, acc, n, st))) return e;
    if ((e = launch_ntt(c, acc + L * N, (int)L, c.K, (int)(n * 2), LK * N, true, st))) return e;
    if ((e = op_moddown_delta(c, acc, delta, n, st))) return e;
    if ((e = launch_ntt(c, delta, 0, (int)L, (int)(n * 2), L * N, false, st))) return e;
    return op_moddown_final(c, acc, delta, add, add_is, add_cs, add_mask, out, n, st);
}

uint32_t pow5(uint64_t e, uint64_t twoN) {
    uint64_t r = 1, b = 5 % twoN;
    for (; e; e >>= 1) {
        if (e & 1) r = r * b % twoN;
        b = b * b % twoN;
    }
    return (uint32_t)r;
}

// Galois elements applied, in order, for a left rotation by k.
std::vector<uint32_t> rotation_chain(const hespmv_ctx *ctx, int64_t k) {
    const uint64_t N = ctx->h.N, half = N / 2, twoN = 2 * N;
    k %= (int64_t)half;
    if (k < 0) k += half;
    std::vector<uint32_t> out;
    if (k == 0) return out;
    if (ctx->p.rot_policy == HESPMV_ROT_EXACT) {
        out.push_back(pow5((uint64_t)k, twoN));
        return out;
    }
    for (int b = 0; (k >> b) != 0; ++b)
        if ((k >> b) & 1) out.push_back(pow5(1ull << b, twoN));
    return out;
}

const int32_t *galois_perm(hespmv_ctx *ctx, uint32_t g) {
    auto it = ctx->perms.find(g);
    if (it != ctx->perms.end()) return it->second;
    const int N = ctx->h.N, logn = ctx->h.log2n;
    const uint64_t twoN = 2 * (uint64_t)N;
    std::vector<int32_t> perm(N);
    for (int i = 0; i < N; ++i) {
        const uint64_t e = (2 * (uint64_t)host_bitrev((uint32_t)i, logn) + 1) * g % twoN;
        perm[i] = (int32_t)ntt_index_of_exponent(e, logn);
    }
    int32_t *d = nullptr;
    if (!upload(ctx, d, perm)) return nullptr;
    ctx->perms[g] = d;
    return d;
}

int make_ksk(hespmv_ctx *ctx, uint64_t seed, uint64_t kid, const uint64_t *sp, uint64_t *out,
             uint64_t *tmp_e, int64_t *coef) {
    const Ctx c = view(ctx);
    const int64_t LK = c.L + c.K, N = c.N, LKN = LK * N;
    for (int j = 0; j < c.dnum; ++j) {
        uint64_t *b = out + (2 * j) * LKN, *a = out + (2 * j + 1) * LKN;
        CK(op_sample_uniform(c, seed, ksk_a_stream(kid, j), a, 0, (int)LK, 0));
        CK(op_sample_signed(c, seed, ksk_a_stream(kid, j) + 1, 0, kCbd21, coef, 1, 0));
        CK(op_signed_to_limbs(c, coef, tmp_e, 0, (int)LK, 1, 0));
        CK(launch_ntt(c, tmp_e, 0, (int)LK, 1, LKN, false, 0));
        CK(op_ksk_combine(c, a, tmp_e, ctx->sk, sp, j, b, 0));
    }
    // keys are kept in Montgomery form (key * 2^64 mod q): the inner product
    // then needs one reduction per sum of products
    CK(op_to_mont(c, out, 2 * c.dnum, 0));
    return HESPMV_OK;
}

int check_ctx(hespmv_ctx *ctx) { return ctx ? HESPMV_OK : HESPMV_E_INVALID; }

// device buffers handed to the key switch are read with 16-byte vector loads
bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }
// every device buffer of a call: the kernels move 16-byte words through all of them
bool aligned16(std::initializer_list<const void *> ps) {
    for (const void *p : ps)
        if (!aligned16(p)) return false;
    return true;
}

// CKKS encoder tables of the context, made on first use
CkksCodec *get_codec(hespmv_ctx *ctx) {
    if (!ctx->codec) ctx->codec = ckks_codec(ctx->h.log2n);
    return ctx->codec;
}

// HE-Mult tensor of n ciphertext pairs -> d [n][3][L][N]: BGV's limb-wise
// products, or BFV's exact scale and round (scratch: tensor_scratch_words)
size_t tensor_scratch_words(const Ctx &c, size_t n) {
    return c.c->h.scheme == HESPMV_SCHEME_BFV ? bfv_tensor_words(c, n) : 0;
}
cudaError_t tensor_n(const Ctx &c, const uint64_t *a, const uint64_t *b, uint64_t *d, size_t n,
                     uint64_t *scratch, cudaStream_t st) {
    if (c.c->h.scheme == HESPMV_SCHEME_BFV) return bfv_tensor(c, a, b, d, n, scratch, st);
    return op_tensor(c, a, b, d, n, st);
}

const uint64_t *mask_plaintext(hespmv_ctx *ctx, int32_t r, cudaStream_t st) {
    auto it = ctx->masks.find(r);
    if (it != ctx->masks.end()) return it->second;
    const Ctx c = view(ctx);
    const int N = c.N;
    uint64_t *m = owned<uint64_t>(ctx, (size_t)c.L * N);
    void *tmp = dev_alloc(ctx, (size_t)N * 8 * 2);
    if (!m || !tmp) {
        dev_free(ctx, tmp);
        return nullptr;
    }
    bool ok;
    if (ctx->h.scheme == HESPMV_SCHEME_CKKS) {
        // r ones at the mask scale, encoded on the host, lifted over Q
        std::vector<double> ones(N / 2, 0.0);
        for (int j = 0; j < r && j < N / 2; ++j) ones[j] = 1.0;
        std::vector<int64_t> coef(N);
        CkksCodec *codec = get_codec(ctx);
        ok = codec && ckks_encode(*codec, ones.data(), N / 2, ctx->h.mask_scale_bits, coef.data()).empty();
        int64_t *dcoef = (int64_t *)tmp;
        ok = ok && cudaMemcpyAsync(dcoef, coef.data(), N * 8, cudaMemcpyHostToDevice, st) == cudaSuccess;
        ok = ok && op_signed_to_limbs(c, dcoef, m, 0, c.L, 1, st) == cudaSuccess;
        ok = ok && cudaStreamSynchronize(st) == cudaSuccess;  // coef is host memory
    } else {
        std::vector<int64_t> ones(N / 2, 0);
        for (int j = 0; j < r && j < N / 2; ++j) ones[j] = 1;
        int64_t *dvals = (int64_t *)tmp;
        uint64_t *E = (uint64_t *)tmp + N;  // words [N, 2N) of tmp
        ok = cudaMemcpyAsync(dvals, ones.data(), (N / 2) * 8, cudaMemcpyHostToDevice, st) == cudaSuccess;
        ok = ok && op_scatter_slots(c, dvals, N / 2, E, 1, st) == cudaSuccess;
        ok = ok && launch_ntt(c, E, c.L + c.K, 1, 1, N, true, st) == cudaSuccess;
        ok = ok && op_lift(c, E, m, 1, st) == cudaSuccess;
        ok = ok && cudaStreamSynchronize(st) == cudaSuccess;  // `ones` is host memory
    }
    ok = ok && launch_ntt(c, m, 0, c.L, 1, (int64_t)c.L * N, false, st) == cudaSuccess;
    // Montgomery form: mask products then need one reduction per sum
    ok = ok && op_to_mont_limbs(c, m, 0, c.L, 1, st) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
    dev_free(ctx, tmp);
    if (!ok) return nullptr;
    ctx->masks[r] = m;
    return m;
}

int batch_new(hespmv_ctx *ctx, size_t n, hespmv_ctbatch **out) {
    const size_t words = n * 2 * (size_t)ctx->h.L * ctx->h.N;
    hespmv_ctbatch *b = new hespmv_ctbatch();
    b->ctx = ctx;
    b->n = n;
    b->bytes = words * 8;
    b->data = (uint64_t *)dev_alloc(ctx, b->bytes);
    if (!b->data) {
        delete b;
        FAIL(HESPMV_E_NOMEM, "ciphertext batch allocation failed");
    }
    *out = b;
    return HESPMV_OK;
}

// Rotate n ciphertexts by k (chain of Galois elements); out must not alias src.
// scratch: 3 ciphertext batches of n + ks_words(n).
int rotate_n(hespmv_ctx *ctx, const uint64_t *src, int32_t k, uint64_t *out, size_t n,
             uint64_t *scratch, cudaStream_t st) {
    const Ctx c = view(ctx);
    const int64_t LN = (int64_t)c.L * c.N, CT = 2 * LN;
    std::vector<uint32_t> chain = rotation_chain(ctx, k);
    if (chain.empty()) {
        CK(cudaMemcpyAsync(out, src, n * CT * 8, cudaMemcpyDeviceToDevice, st));
        return HESPMV_OK;
    }
    uint64_t *perm_buf = scratch;
    uint64_t *bufs[2] = {perm_buf + n * CT, perm_buf + 2 * n * CT};
    uint64_t *ks = perm_buf + 3 * n * CT;
    const uint64_t *cur = src;
    for (size_t s = 0; s < chain.size(); ++s) {
        const uint32_t g = chain[s];
        auto it = ctx->gk.find(g);
        if (it == ctx->gk.end()) FAIL(HESPMV_E_INVALID, "missing Galois key for element " + std::to_string(g));
        const int32_t *perm = galois_perm(ctx, g);
        if (!perm) FAIL(HESPMV_E_NOMEM, "permutation upload failed");
        // the last step writes `out`; earlier ones alternate between two buffers
        uint64_t *dst = (s + 1 == chain.size()) ? out : bufs[s & 1];
        CK(op_permute(c, cur, perm_buf, perm, n * 2 * c.L, st));
        CK(keyswitch_n(c, perm_buf + LN, CT, it->second, dst, perm_buf, CT, LN, 1, n, ks, st));
        cur = dst;
    }
    if (cur != out) CK(cudaMemcpyAsync(out, cur, n * CT * 8, cudaMemcpyDeviceToDevice, st));
    return HESPMV_OK;
}

// Batched totalSum schedule for the given matrices (host part): ops and the
// index lists they refer to.
void build_rotation_ops(hespmv_ctx *ctx, size_t n_inst, const hespmv_cssc *const *ms, int GR,
                        RotPlan *P, std::vector<int32_t> &idx) {
    struct RC {
        int32_t k;
        std::vector<int32_t> steps;
        std::vector<uint8_t> orig;
    };
    std::vector<RC> rcs;
    int32_t k0 = 0;
    for (size_t i = 0; i < n_inst; ++i) {
        for (const Chunk &ch : ms[i]->plan.chunks) {
            RC r;
            r.k = k0++;
            total_sum_steps(ch.h, ch.c, r.steps, r.orig);
            if (!r.steps.empty()) rcs.push_back(std::move(r));
        }
    }
    P->GR = GR;
    P->ops.clear();
    idx.clear();
    auto push = [&](const std::vector<int32_t> &v) {
        const int64_t off = (int64_t)idx.size();
        idx.insert(idx.end(), v.begin(), v.end());
        return off;
    };
    const bool exact = ctx->p.rot_policy == HESPMV_ROT_EXACT;
    const uint64_t twoN = 2 * (uint64_t)ctx->h.N;
    for (size_t g0 = 0; g0 < rcs.size(); g0 += GR) {
        const size_t gn = std::min<size_t>(GR, rcs.size() - g0);
        std::vector<int32_t> gk(gn);
        size_t maxr = 0;
        for (size_t g = 0; g < gn; ++g) {
            gk[g] = rcs[g0 + g].k;
            maxr = std::max(maxr, rcs[g0 + g].steps.size());
        }
        RotOp v;
        v.kind = RotOp::kVInit;
        v.m = (int)gn;
        v.b = push(gk);
        P->ops.push_back(v);
        for (size_t r = 0; r < maxr; ++r) {
            std::vector<int32_t> pg, pk, vg;  // from prod (group id, chunk id), from V
            std::vector<int32_t> act, actk;
            for (size_t g = 0; g < gn; ++g) {
                const RC &c = rcs[g0 + g];
                if (r >= c.steps.size()) continue;
                act.push_back((int32_t)g);
                actk.push_back(c.k);
                if (c.orig[r])
                    vg.push_back((int32_t)g);
                else {
                    pg.push_back((int32_t)g);
                    pk.push_back(c.k);
                }
            }
            if (!pg.empty()) {
                RotOp o;
                o.kind = RotOp::kCurFromProd;
                o.m = (int)pg.size();
                o.a = push(pg);
                o.b = push(pk);
                P->ops.push_back(o);
            }
            if (!vg.empty()) {
                RotOp o;
                o.kind = RotOp::kCurFromV;
                o.m = (int)vg.size();
                o.a = push(vg);
                o.b = o.a;
                P->ops.push_back(o);
            }
            if (exact) {
                std::map<int32_t, std::vector<int32_t>> by_amount;
                for (size_t s = 0; s < act.size(); ++s)
                    by_amount[rcs[g0 + act[s]].steps[r]].push_back(act[s]);
                for (auto &kv : by_amount) {
                    RotOp o;
                    o.kind = RotOp::kElem;
                    o.g = rotation_chain(ctx, kv.first).at(0);
                    o.m = (int)kv.second.size();
                    o.a = push(kv.second);
                    P->ops.push_back(o);
                }
            } else {
                for (int b = 0; b < 31; ++b) {
                    std::vector<int32_t> S;
                    for (int32_t g : act)
                        if ((rcs[g0 + g].steps[r] >> b) & 1) S.push_back(g);
                    if (S.empty()) continue;
                    RotOp o;
                    o.kind = RotOp::kElem;
                    o.g = pow5(1ull << b, twoN);
                    o.m = (int)S.size();
                    o.a = push(S);
                    P->ops.push_back(o);
                }
            }
            RotOp o;
            o.kind = RotOp::kAdd;
            o.m = (int)act.size();
            o.a = push(actk);
            o.b = push(act);
            P->ops.push_back(o);
        }
    }
    P->idx_bytes = idx.size() * sizeof(int32_t);
}

// The schedule with its index lists on the device, cached per matrix set.
RotPlan *rotation_plan(hespmv_ctx *ctx, size_t n_inst, const hespmv_cssc *const *ms, int GR) {
    std::vector<uint64_t> key;
    key.push_back((uint64_t)GR);
    for (size_t i = 0; i < n_inst; ++i) key.push_back(ms[i]->uid);
    auto it = ctx->rot_plans.find(key);
    if (it != ctx->rot_plans.end()) return it->second;
    RotPlan *P = new RotPlan();
    std::vector<int32_t> idx;
    build_rotation_ops(ctx, n_inst, ms, GR, P, idx);
    if (!idx.empty()) {
        P->d_idx = (int32_t *)dev_alloc(ctx, P->idx_bytes);
        if (!P->d_idx || cudaMemcpy(P->d_idx, idx.data(), P->idx_bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
            dev_free(ctx, P->d_idx);
            delete P;
            return nullptr;
        }
    }
    ctx->rot_plans[key] = P;
    return P;
}

// packed ciphertexts: words of one limb and of one ciphertext
size_t packed_limb_words(const HostTables &h) { return ((size_t)h.N * h.pack_bits + 63) / 64; }
size_t packed_ct_words(const HostTables &h) { return 2 * (size_t)h.L * packed_limb_words(h); }

// Default upload groups of a host evaluation.  On the stencil workload
// (27 chunks, 177 MB packed) 4 to 7 groups are within 2 % of each other, 7
// the fastest; fewer groups delay the first HE-Mult, more make each fused key
// switch too small.
constexpr size_t kUploadGroups = 7;
// Pipelined evaluations overlap a call's uploads with the previous call's
// compute, so the groups only need to let the HE-Mult start before the whole
// upload has landed: 2 groups (1048 SpMV/s on the stencil) beat 1 (975), 4
// (1012) and 7 (884).
constexpr size_t kPipelinedUploadGroups = 2;

// upload (and HE-Mult) group sizes of a host evaluation of nc chunks
std::vector<size_t> upload_group_sizes(const hespmv_ctx *ctx, size_t nc, bool pipelined = false) {
    const size_t dflt = pipelined ? kPipelinedUploadGroups : kUploadGroups;
    const size_t groups = std::min(std::max<size_t>(nc, 1),
                                   ctx->upload_groups > 0 ? (size_t)ctx->upload_groups : dflt);
    std::vector<size_t> g;
    for (size_t k = 0; k < groups; ++k) g.push_back((nc * (k + 1)) / groups - (nc * k) / groups);
    if (g.empty() || g[0] == 0) g.assign(1, std::max<size_t>(nc, 1));
    return g;
}

// status of a device error word value
int status_of_code(hespmv_ctx *ctx, int v) {
    if (v == 0) return HESPMV_OK;
    if (v == kErrBadResidue) FAIL(HESPMV_E_INVALID, "a packed input residue was not below its prime");
    if (v == kErrSchedTimeout)
        FAIL(HESPMV_E_TIMEOUT, "a dependency wait of the persistent evaluation ran out; its results are incomplete");
    FAIL(HESPMV_E_TIMEOUT, "a device-side wait ran out (code " + std::to_string(v) + ")");
}

struct SpmvPrep {
    size_t total_chunks = 0, rot_chunks = 0, G = 1, GR = 1;
    RotPlan *rp = nullptr;
    size_t need_bytes = 0;
    bool pt_matrix = false;  // matrix operand in the clear: HE-CMult, no key switch
    // host operands of a single instance: each HE-Mult group's chunks are
    // uploaded on the context's copy stream and waited for by that group only
    const uint64_t *hA = nullptr, *hX = nullptr;
    // packed host operands: staged in pkA / pkX (pk_words per ciphertext),
    // unpacked on the copy stream group by group
    uint64_t *pkA = nullptr, *pkX = nullptr;
    int64_t pk_words = 0;
    // HE-Mult groups alternate between two streams, each with its own
    // tensor / key-switch scratch of mult_w words
    bool dual = false;
    size_t mult_w = 0;
    // totalSum rotation groups (GR chunks each, independent of one another)
    // alternate between the two streams, each with its own rot_w words
    bool dual_rot = false;
    size_t rot_w = 0;
    // HE-Mult group sizes of a host evaluation (empty: groups of G)
    std::vector<size_t> gsz;
    // pipelined host evaluation: the uploads wait for this event (or nothing)
    // instead of the evaluation stream's earlier work
    bool pipelined = false;
    cudaEvent_t copy_after = nullptr;
};

// HE-Mult groups of an evaluation over `total` chunks: (first chunk, count)
std::vector<std::pair<size_t, size_t>> mult_groups(const SpmvPrep &pp, size_t total) {
    std::vector<std::pair<size_t, size_t>> g;
    size_t g0 = 0;
    for (size_t k = 0; g0 < total; ++k) {
        // never above G: the scratch holds G ciphertexts
        const size_t n = std::min(total - g0, k < pp.gsz.size() ? std::min(pp.gsz[k], pp.G) : pp.G);
        g.push_back({g0, n});
        g0 += n;
    }
    return g;
}

// Per-matrix device state an evaluation reads: mask plaintexts (cached per
// chunk height), the matrix's mask table, the Galois permutations of its
// rotations.  May synchronise and allocate (first use of a matrix only).
int prepare_matrix(hespmv_ctx *ctx, const hespmv_cssc *cm, cudaStream_t st) {
    hespmv_cssc *m = const_cast<hespmv_cssc *>(cm);
    if (m->prepared) return HESPMV_OK;
    for (const Chunk &ch : m->plan.chunks)
        if (!mask_plaintext(ctx, ch.h, st)) FAIL(HESPMV_E_NOMEM, "mask plaintext creation failed");
    if (!m->plan.chunks.empty()) {
        std::vector<const uint64_t *> tab;
        for (const Chunk &ch : m->plan.chunks) tab.push_back(ctx->masks[ch.h]);
        m->d_masks = (const uint64_t **)dev_alloc(ctx, tab.size() * sizeof(void *));
        if (!m->d_masks) FAIL(HESPMV_E_NOMEM, "mask table allocation failed");
        CK(cudaMemcpy(m->d_masks, tab.data(), tab.size() * sizeof(void *), cudaMemcpyHostToDevice));
    }
    for (int32_t k : m->steps)
        for (uint32_t g : rotation_chain(ctx, k))
            if (!galois_perm(ctx, g)) FAIL(HESPMV_E_NOMEM, "permutation upload failed");
    m->prepared = true;
    return HESPMV_OK;
}

// batch sizes and workspace bytes of an evaluation over the given chunk counts
void spmv_sizes(const Ctx &c, size_t total_chunks, size_t rot_chunks, SpmvPrep &pp,
                size_t max_G = 0) {
    size_t tune_G = c.c->tune_G;
    const size_t tune_GR = c.c->tune_GR;
    if (max_G) tune_G = std::min(tune_G ? tune_G : 32, max_G);
    const int64_t LN = (int64_t)c.L * c.N, CT = 2 * LN;
    pp.total_chunks = total_chunks;
    pp.rot_chunks = rot_chunks;
    pp.G = std::max<size_t>(1, std::min<size_t>(total_chunks, tune_G ? tune_G : 32));
    pp.GR = std::max<size_t>(1, std::min<size_t>(rot_chunks, tune_GR ? tune_GR : c.N >= (1 << 15) ? 32 : 64));
    const size_t prod_w = total_chunks * CT;
    const size_t mult_w = pp.G * 3 * LN + std::max(ks_words(c, pp.G), tensor_scratch_words(c, pp.G));
    const size_t rot_w = rot_chunks ? 4 * pp.GR * CT + ks_words(c, pp.GR) : 0;
    pp.mult_w = mult_w;
    pp.rot_w = rot_w;
    pp.need_bytes = (prod_w + std::max(mult_w, rot_w)) * 8;
}

// Everything an evaluation needs besides kernel launches: per-matrix state,
// the (cached) rotation schedule, the workspace size.
int spmv_prepare(hespmv_ctx *ctx, size_t n_inst, const hespmv_cssc *const *ms, SpmvPrep &pp,
                 cudaStream_t st, size_t max_G = 0) {
    const Ctx c = view(ctx);
    size_t total = 0, rot = 0;
    for (size_t i = 0; i < n_inst; ++i) {
        int rc = prepare_matrix(ctx, ms[i], st);
        if (rc) return rc;
        total += ms[i]->plan.chunks.size();
        for (const Chunk &ch : ms[i]->plan.chunks) rot += ch.c > 1;
    }
    spmv_sizes(c, total, rot, pp, max_G);
    pp.rp = nullptr;
    if (rot) {
        pp.rp = rotation_plan(ctx, n_inst, ms, (int)pp.GR);
        if (!pp.rp) FAIL(HESPMV_E_NOMEM, "rotation schedule upload failed");
    }
    return HESPMV_OK;
}

// ------------------------------------------------------------ persistent evaluation

// levels by which consecutive HE-Mult groups of a persistent program are
// staggered in its work queue (tune_GR overrides it)
constexpr int kPersistStagger = 0;

// HE-Mult group of a persistent evaluation: ciphertexts per key switch
size_t persist_group(const hespmv_ctx *ctx, size_t total) {
    const size_t G = ctx->tune_G ? ctx->tune_G : 16;
    return std::max<size_t>(1, std::min(G, std::max<size_t>(total, 1)));
}

// Workspace words of a persistent evaluation: the HE-Mult products, the
// key-switch scratch of every HE-Mult group, and per rotating chunk its
// running sum, its rotation buffer and its own key-switch scratch (the
// chunks' totalSum chains run concurrently).
size_t persist_ws_words(const Ctx &c, size_t total, size_t rot, size_t G) {
    const size_t CT = 2 * (size_t)c.L * c.N;
    size_t w = total * CT;
    for (size_t g0 = 0; g0 < total; g0 += G) w += ks_words(c, std::min(G, total - g0));
    return w + rot * (2 * CT + ks_words(c, 1));
}

bool persist_usable(const hespmv_ctx *ctx, bool pt_matrix, const uint64_t *hA) {
    return ctx->persistent && !pt_matrix && !hA && ctx->h.scheme != HESPMV_SCHEME_BFV &&
           persist_supported(view(ctx));
}

void persist_free(hespmv_ctx *ctx, PersistPlan *P) {
    if (!P) return;
    dev_free(ctx, P->blob);
    delete P;
}

void drop_persist_plans(hespmv_ctx *ctx) {
    if (ctx->persist_plans.empty()) return;
    cudaDeviceSynchronize();  // no launch may still read a program
    for (auto &kv : ctx->persist_plans) persist_free(ctx, kv.second);
    ctx->persist_plans.clear();
}

// host form of a phase while the program is built
struct HostPhase {
    PPhase p{};
    std::vector<int32_t> deps;
    int32_t grp = 0;  // HE-Mult group it belongs to (the latest one, for masked sums)
};

// Program of one evaluation (Algorithm 1 cloud lines and Algorithm 4 for
// every chunk of every matrix given):
//  * HE-Mult with relinearisation: one fused key switch per group of G
//    consecutive chunks (operands through tables of addresses), results in
//    the product buffers;
//  * totalSum of each chunk with c > 1: its chain of rotations, one key
//    switch per Galois element (power-of-two policy: one per set bit, least
//    significant first), each step's last key switch adding the running sum
//    (or, for the first step, the product) as it writes the new running sum;
//  * one masked accumulation per partition into the result.
// Every phase depends on the phases that write what it reads (a key
// switch's first stage on the one before it in its chunk's chain, each
// further stage on the previous stage; a masked sum on the last key switch
// of each of its chunks).  Phases are ordered by depth, deeper remaining
// chains first at equal depth, so every dependency precedes its user.
int persist_build(hespmv_ctx *ctx, size_t n_inst, const hespmv_cssc *const *ms, const uint64_t *const *A,
                  const uint64_t *const *X, uint64_t *const *Y, uint64_t *ws, size_t G, int stagger,
                  PersistPlan *P) {
    const Ctx c = view(ctx);
    const int64_t LN = (int64_t)c.L * c.N, CT = 2 * LN;
    std::vector<HostPhase> ph;
    std::vector<PInst> inst;
    std::vector<PMask> mask;
    std::vector<std::vector<const uint64_t *>> tabs;  // address tables, placed in the blob
    std::vector<size_t> inst_tab, mask_tab;           // first of each one's two tables
    int32_t gx[7], gy[7];
    auto add_ks = [&](const PInst &I, std::vector<int32_t> deps0, size_t tab, int32_t grp) -> int32_t {
        persist_stage_tiles(c, I.n, gx, gy);
        const int32_t ii = (int32_t)inst.size();
        inst.push_back(I);
        inst_tab.push_back(tab);
        int32_t prev = -1;
        for (int s = 0; s < 7; ++s) {
            HostPhase h;
            h.grp = grp;
            h.p.kind = kPhIntt + s;
            h.p.inst = ii;
            h.p.gx = gx[s];
            h.p.tiles = gx[s] * gy[s];
            if (s == 0)
                h.deps = deps0;
            else
                h.deps.assign(1, prev);
            prev = (int32_t)ph.size();
            ph.push_back(std::move(h));
        }
        return prev;
    };
    std::vector<std::pair<size_t, size_t>> all;  // (matrix, chunk)
    for (size_t i = 0; i < n_inst; ++i)
        for (size_t k = 0; k < ms[i]->plan.chunks.size(); ++k) all.push_back({i, k});
    const size_t total = all.size();
    uint64_t *prod = ws, *cur = ws + total * CT;
    // HE-Mult groups
    std::vector<int32_t> last_ph(total, -1);
    for (size_t g0 = 0; g0 < total; g0 += G) {
        const size_t gn = std::min(G, total - g0);
        const size_t ta = tabs.size();
        tabs.emplace_back();
        tabs.emplace_back();
        for (size_t u = 0; u < gn; ++u) {
            const size_t i = all[g0 + u].first, k = all[g0 + u].second;
            tabs[ta].push_back(A[i] + k * CT);
            tabs[ta + 1].push_back(X[i] + k * CT);
        }
        PInst I{};
        I.s = KsSrc{nullptr, 0, nullptr, nullptr, CT};
        I.ad = KsAdd{nullptr, 0, 0, 0};
        I.key = ctx->rlk;
        I.out = prod + g0 * CT;
        I.scratch = cur;
        I.n = (int32_t)gn;
        cur += ks_words(c, gn);
        const int32_t f = add_ks(I, {}, ta, (int32_t)(g0 / G));
        for (size_t u = 0; u < gn; ++u) last_ph[g0 + u] = f;
    }
    // totalSum chains
    std::vector<const uint64_t *> term(total);
    for (size_t g = 0; g < total; ++g) {
        const Chunk &ch = ms[all[g].first]->plan.chunks[all[g].second];
        uint64_t *Pg = prod + g * CT;
        const uint64_t *w = Pg;  // running sum (Algorithm 4: w = ctV first)
        std::vector<int32_t> steps;
        std::vector<uint8_t> orig;
        total_sum_steps(ch.h, ch.c, steps, orig);
        if (!steps.empty()) {
            uint64_t *Wg = cur, *Cg = cur + CT, *scr = cur + 2 * CT;
            cur += 2 * CT + ks_words(c, 1);
            int32_t prev = last_ph[g];
            for (size_t r = 0; r < steps.size(); ++r) {
                const std::vector<uint32_t> chain = rotation_chain(ctx, steps[r]);
                const uint64_t *src = orig[r] ? Pg : w;
                for (size_t j = 0; j < chain.size(); ++j) {
                    auto kit = ctx->gk.find(chain[j]);
                    if (kit == ctx->gk.end())
                        FAIL(HESPMV_E_INVALID, "missing Galois key for element " + std::to_string(chain[j]));
                    auto pit = ctx->perms.find(chain[j]);
                    if (pit == ctx->perms.end()) FAIL(HESPMV_E_INVALID, "missing Galois permutation");
                    const bool last = j + 1 == chain.size();
                    const uint64_t *in = j == 0 ? src : Cg;
                    PInst I{};
                    I.s = KsSrc{in + LN, CT, nullptr, nullptr, 0};
                    I.s.perm = pit->second;
                    I.ad = KsAdd{in, CT, LN, 1, nullptr, pit->second};
                    I.key = kit->second;
                    I.out = last ? Wg : Cg;
                    I.post = last ? w : nullptr;
                    I.scratch = scr;
                    I.n = 1;
                    prev = add_ks(I, {prev}, SIZE_MAX, (int32_t)(g / G));
                }
                w = Wg;
            }
            last_ph[g] = prev;
        }
        term[g] = w;
    }
    // masked accumulation per partition
    const int32_t mask_tiles = (int32_t)(CT / kMaskTileWords);
    for (size_t i = 0, g0 = 0; i < n_inst; g0 += ms[i]->plan.chunks.size(), ++i) {
        const Plan &pl = ms[i]->plan;
        for (size_t p = 0; p < pl.parts.size(); ++p) {
            const Partition &Pt = pl.parts[p];
            const size_t tt = tabs.size();
            tabs.emplace_back();
            tabs.emplace_back();
            HostPhase h;
            for (int32_t q = 0; q < Pt.n_chunks; ++q) {
                const size_t g = g0 + Pt.chunk0 + q;
                auto mit = ctx->masks.find(pl.chunks[Pt.chunk0 + q].h);
                if (mit == ctx->masks.end()) FAIL(HESPMV_E_INVALID, "mask plaintext missing");
                tabs[tt].push_back(term[g]);
                tabs[tt + 1].push_back(mit->second);
                h.deps.push_back(last_ph[g]);
                h.grp = std::max(h.grp, (int32_t)(g / G));
            }
            std::sort(h.deps.begin(), h.deps.end());
            h.deps.erase(std::unique(h.deps.begin(), h.deps.end()), h.deps.end());
            PMask J{};
            J.out = Y[i] + p * CT;
            J.nterms = Pt.n_chunks;
            h.p.kind = kPhMask;
            h.p.inst = (int32_t)mask.size();
            h.p.gx = mask_tiles;
            h.p.tiles = mask_tiles;
            mask.push_back(J);
            mask_tab.push_back(tt);
            ph.push_back(std::move(h));
        }
    }
    // order: by depth, group g's phases `stagger` levels behind group g-1's
    // (so a phase's inputs were usually finished well before a CTA takes
    // it), then the longer remaining chain, then creation.  Depth grows and
    // the group never shrinks along a dependency, so every dependency keeps
    // a smaller key than its user.
    const size_t nph = ph.size();
    std::vector<int32_t> level(nph, 0), tail(nph, 1), order(nph), pos(nph);
    for (size_t p = 0; p < nph; ++p)
        for (int32_t d : ph[p].deps) level[p] = std::max(level[p], level[d] + 1);
    for (size_t p = nph; p-- > 0;)
        for (int32_t d : ph[p].deps) tail[d] = std::max(tail[d], tail[p] + 1);
    for (size_t p = 0; p < nph; ++p) order[p] = (int32_t)p;
    auto key = [&](int32_t p) { return (int64_t)level[p] + (int64_t)stagger * ph[p].grp; };
    std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        if (key(a) != key(b)) return key(a) < key(b);
        if (tail[a] != tail[b]) return tail[a] > tail[b];
        return a < b;
    });
    for (size_t k = 0; k < nph; ++k) pos[order[k]] = (int32_t)k;
    std::vector<PPhase> fph(nph);
    std::vector<int32_t> off(nph + 1, 0), deps;
    int64_t tiles = 0;
    for (size_t k = 0; k < nph; ++k) {
        const HostPhase &h = ph[order[k]];
        fph[k] = h.p;
        fph[k].dep0 = (int32_t)deps.size();
        fph[k].ndep = (int32_t)h.deps.size();
        for (int32_t d : h.deps) {
            if (pos[d] >= (int32_t)k) FAIL(HESPMV_E_INVALID, "persistent program: a dependency follows its user");
            deps.push_back(pos[d]);
        }
        off[k] = (int32_t)tiles;
        tiles += h.p.tiles;
        if (tiles >= (int64_t)INT32_MAX) FAIL(HESPMV_E_UNSUPPORTED, "persistent program: too many tiles");
    }
    off[nph] = (int32_t)tiles;
    // one device block: phases | offsets | deps | instances | masks | tables | tile table | counters
    auto al = [](size_t b) { return (b + 15) & ~(size_t)15; };
    size_t ntab = 0;
    for (const auto &t : tabs) ntab += t.size();
    const size_t o_ph = 0, o_off = al(o_ph + nph * sizeof(PPhase)),
                 o_dep = al(o_off + (nph + 1) * sizeof(int32_t)), o_inst = al(o_dep + deps.size() * sizeof(int32_t)),
                 o_mask = al(o_inst + inst.size() * sizeof(PInst)), o_tab = al(o_mask + mask.size() * sizeof(PMask)),
                 o_info = al(o_tab + ntab * sizeof(void *)), o_ctr = al(o_info + (size_t)tiles * sizeof(uint64_t)),
                 bytes = al(o_ctr + (nph + 2) * sizeof(uint32_t));
    P->blob = dev_alloc(ctx, bytes);
    if (!P->blob) FAIL(HESPMV_E_NOMEM, "persistent program allocation failed");
    P->bytes = bytes;
    char *base = (char *)P->blob;
    std::vector<size_t> tab_off(tabs.size());
    std::vector<const uint64_t *> flat;
    for (size_t t = 0; t < tabs.size(); ++t) {
        tab_off[t] = o_tab + flat.size() * sizeof(void *);
        flat.insert(flat.end(), tabs[t].begin(), tabs[t].end());
    }
    for (size_t i = 0; i < inst.size(); ++i)
        if (inst_tab[i] != SIZE_MAX) {
            inst[i].s.tap = (const uint64_t *const *)(base + tab_off[inst_tab[i]]);
            inst[i].s.tbp = (const uint64_t *const *)(base + tab_off[inst_tab[i] + 1]);
        }
    for (size_t j = 0; j < mask.size(); ++j) {
        mask[j].terms = (const uint64_t *const *)(base + tab_off[mask_tab[j]]);
        mask[j].masks = (const uint64_t *const *)(base + tab_off[mask_tab[j] + 1]);
    }
    std::vector<char> img(bytes, 0);
    if (nph) memcpy(img.data() + o_ph, fph.data(), nph * sizeof(PPhase));
    memcpy(img.data() + o_off, off.data(), (nph + 1) * sizeof(int32_t));
    if (!deps.empty()) memcpy(img.data() + o_dep, deps.data(), deps.size() * sizeof(int32_t));
    if (!inst.empty()) memcpy(img.data() + o_inst, inst.data(), inst.size() * sizeof(PInst));
    if (!mask.empty()) memcpy(img.data() + o_mask, mask.data(), mask.size() * sizeof(PMask));
    if (!flat.empty()) memcpy(img.data() + o_tab, flat.data(), flat.size() * sizeof(void *));
    {
        uint64_t *info = (uint64_t *)(img.data() + o_info);
        for (size_t k = 0; k < nph; ++k)
            for (int32_t l = 0; l < fph[k].tiles; ++l) *info++ = ((uint64_t)k << 32) | (uint32_t)l;
    }
    CK(cudaMemcpy(P->blob, img.data(), bytes, cudaMemcpyHostToDevice));
    PProg &g = P->prog;
    g.ph = (const PPhase *)(base + o_ph);
    g.off = (const int32_t *)(base + o_off);
    g.info = (const uint64_t *)(base + o_info);
    g.deps = (const int32_t *)(base + o_dep);
    g.inst = (const PInst *)(base + o_inst);
    g.mask = (const PMask *)(base + o_mask);
    g.ctr = (uint32_t *)(base + o_ctr);
    g.nph = (int32_t)nph;
    g.total = (int32_t)tiles;
    g.wait_ns = kPersistWaitNs;
    P->n_ks = (int64_t)inst.size();
    P->n_phases = (int64_t)nph;
    return HESPMV_OK;
}

// The program of this evaluation (built on first use; cached per matrices,
// buffers, workspace, HE-Mult group and NTT split).
int persist_plan(hespmv_ctx *ctx, size_t n_inst, const hespmv_cssc *const *ms, const uint64_t *const *A,
                 const uint64_t *const *X, uint64_t *const *Y, uint64_t *ws, size_t G, PersistPlan **out) {
    const int stagger = ctx->tune_GR ? (int)ctx->tune_GR : kPersistStagger;
    std::vector<uint64_t> key{(uint64_t)(uintptr_t)ws, (uint64_t)G, (uint64_t)ctx->ks_split, (uint64_t)stagger};
    for (size_t i = 0; i < n_inst; ++i) {
        key.push_back(ms[i]->uid);
        key.push_back((uint64_t)(uintptr_t)A[i]);
        key.push_back((uint64_t)(uintptr_t)X[i]);
        key.push_back((uint64_t)(uintptr_t)Y[i]);
    }
    auto it = ctx->persist_plans.find(key);
    if (it != ctx->persist_plans.end()) {
        *out = it->second;
        return HESPMV_OK;
    }
    if (ctx->persist_plans.size() >= 64) {  // cached graphs may use the plans
        cudaDeviceSynchronize();
        for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
        ctx->graphs.clear();
        drop_persist_plans(ctx);
    }
    PersistPlan *P = new PersistPlan();
    const int rc = persist_build(ctx, n_inst, ms, A, X, Y, ws, G, stagger, P);
    if (rc) {
        persist_free(ctx, P);
        return rc;
    }
    ctx->persist_plans[key] = P;
    *out = P;
    return HESPMV_OK;
}

// Launch the program on st: counters cleared, then one persistent launch.
int persist_enqueue(hespmv_ctx *ctx, const PersistPlan *P, cudaStream_t st) {
    const Ctx c = view(ctx);
    Range r("hespmv: persistent evaluation");
    CK(cudaMemsetAsync(P->prog.ctr, 0, (P->prog.nph + 2) * sizeof(uint32_t), st));
    const int pr = prof_begin(c, "k_ks_persist", st);
    CK(persist_launch(c, P->prog, ctx->persist_blocks, st));
    prof_end(c, pr, st);
    return HESPMV_OK;
}

// Cloud evaluation of one or more SpMVs (Algorithm 1 cloud lines + Algorithm 4):
// kernel launches and memsets only, on stream st, in workspace ws.
int spmv_enqueue(hespmv_ctx *ctx, size_t n_inst, const hespmv_cssc *const *ms,
                 const uint64_t *const *A, const uint64_t *const *X, uint64_t *const *Y,
                 const SpmvPrep &pp, uint64_t *ws, cudaStream_t st) {
    const Ctx c = view(ctx);
    const int64_t N = c.N, LN = (int64_t)c.L * N, CT = 2 * LN;
    const size_t G = pp.G, GR = pp.GR;
    const size_t prod_w = pp.total_chunks * CT;
    uint64_t *prod = ws, *dbuf = prod + prod_w, *scr = dbuf + G * 3 * LN;
    Range r_eval("hespmv: evaluation");
    // 1) HE-Mult of every chunk pair, G at a time across instances (HE-CMult
    //    when the matrix is in the clear)
    if (pp.pt_matrix) {
        Range r("hespmv: HE-CMult");
        size_t k0 = 0;
        for (size_t i = 0; i < n_inst; ++i) {
            const size_t nk = ms[i]->plan.chunks.size();
            CK(op_pt_ct_mul(c, A[i], X[i], prod + k0 * CT, nk, st));
            k0 += nk;
        }
    } else {
        Range r("hespmv: HE-Mult + relinearisation");
        std::vector<std::pair<size_t, size_t>> all;  // (instance, chunk)
        all.reserve(pp.total_chunks);
        for (size_t i = 0; i < n_inst; ++i)
            for (size_t k = 0; k < ms[i]->plan.chunks.size(); ++k) all.push_back({i, k});
        const std::vector<std::pair<size_t, size_t>> groups = mult_groups(pp, all.size());
        if (!pp.hA && pp.dual) {  // fork the second compute stream
            CK(cudaEventRecord(ctx->copy_events[0], st));
            CK(cudaStreamWaitEvent(ctx->aux_stream, ctx->copy_events[0], 0));
        }
        if (pp.hA) {  // uploads on the side stream, one event per group
            cudaStream_t cs = ctx->copy_stream;
            CK(cudaEventRecord(ctx->copy_events[0], st));  // fork
            if (!pp.pipelined)
                CK(cudaStreamWaitEvent(cs, ctx->copy_events[0], 0));
            else if (pp.copy_after)  // the staging slot's previous evaluation is done with it
                CK(cudaStreamWaitEvent(cs, pp.copy_after, 0));
            if (pp.dual) CK(cudaStreamWaitEvent(ctx->aux_stream, ctx->copy_events[0], 0));
            for (size_t gi = 1; gi <= groups.size(); ++gi) {
                const size_t g0 = groups[gi - 1].first, gn = groups[gi - 1].second;
                if (pp.pkA) {  // packed: the group's compute stream unpacks
                    const int64_t PW = pp.pk_words;
                    CK(cudaMemcpyAsync(pp.pkA + g0 * PW, pp.hA + g0 * PW, gn * PW * 8, cudaMemcpyHostToDevice,
                                       cs));
                    CK(cudaMemcpyAsync(pp.pkX + g0 * PW, pp.hX + g0 * PW, gn * PW * 8, cudaMemcpyHostToDevice,
                                       cs));
                } else {
                    CK(cudaMemcpyAsync((uint64_t *)A[0] + g0 * CT, pp.hA + g0 * CT, gn * CT * 8,
                                       cudaMemcpyHostToDevice, cs));
                    CK(cudaMemcpyAsync((uint64_t *)X[0] + g0 * CT, pp.hX + g0 * CT, gn * CT * 8,
                                       cudaMemcpyHostToDevice, cs));
                }
                CK(cudaEventRecord(ctx->copy_events[gi], cs));
            }
        }
        for (size_t gi = 1; gi <= groups.size(); ++gi) {
            const size_t g0 = groups[gi - 1].first, gn = groups[gi - 1].second;
            const size_t i = all[g0].first, k = all[g0].second;
            // odd groups of a dual schedule: second stream, second scratch
            const bool alt = pp.dual && (gi & 1) == 0;
            cudaStream_t gs = alt ? ctx->aux_stream : st;
            uint64_t *gd = dbuf + (alt ? pp.mult_w : 0), *gscr = scr + (alt ? pp.mult_w : 0);
            if (pp.hA) CK(cudaStreamWaitEvent(gs, ctx->copy_events[gi], 0));  // this group's chunks
            const bool bgv = ctx->h.scheme != HESPMV_SCHEME_BFV;  // BGV and CKKS tensors are limb-wise
            if (bgv && ks_fused_supported(c) && all[g0 + gn - 1].first == i) {
                // one matrix's consecutive chunks: tensor product fused into the key switch,
                // reading packed host operands directly where given
                if (pp.pkA)
                    CK(relin_tensor_fused(c, pp.pkA + g0 * pp.pk_words, pp.pkX + g0 * pp.pk_words, ctx->rlk,
                                          prod + g0 * CT, gn, gscr, gs, ctx->h.pack_bits));
                else
                    CK(relin_tensor_fused(c, A[i] + k * CT, X[i] + k * CT, ctx->rlk, prod + g0 * CT, gn,
                                          gscr, gs));
                continue;
            }
            if (bgv && ks_fused_supported(c) && !pp.pkA) {
                // chunks of several SpMVs: the fused tensor reads each item's
                // operands through a table of addresses (in the unused tensor buffer)
                std::vector<const uint64_t *> ptrs(2 * gn);
                for (size_t u = 0; u < gn; ++u) {
                    const size_t ii = all[g0 + u].first, kk = all[g0 + u].second;
                    ptrs[u] = A[ii] + kk * CT;
                    ptrs[gn + u] = X[ii] + kk * CT;
                }
                const uint64_t **tab = (const uint64_t **)gd;
                CK(op_write_ptrs(c, tab, ptrs, gs));
                CK(relin_tensor_fused_ptrs(c, tab, tab + gn, ctx->rlk, prod + g0 * CT, gn, gscr, gs));
                continue;
            }
            if (pp.pkA)
                CK(op_ct_unpack(c, pp.pkA + g0 * pp.pk_words, (uint64_t *)A[0] + g0 * CT,
                                pp.pkX + g0 * pp.pk_words, (uint64_t *)X[0] + g0 * CT, gn, gs));
            size_t s = 0;
            while (s < gn) {  // tensor over runs of one instance's consecutive chunks
                const size_t ii = all[g0 + s].first, kk = all[g0 + s].second;
                size_t run = 1;
                while (s + run < gn && all[g0 + s + run].first == ii) ++run;
                CK(tensor_n(c, A[ii] + kk * CT, X[ii] + kk * CT, gd + s * 3 * LN, run, gscr, gs));
                s += run;
            }
            CK(keyswitch_n(c, gd + 2 * LN, 3 * LN, ctx->rlk, prod + g0 * CT, gd, 3 * LN, LN, 3, gn, gscr,
                           gs));
        }
        if (pp.dual) {  // join the second stream
            CK(cudaEventRecord(ctx->join_event, ctx->aux_stream));
            CK(cudaStreamWaitEvent(st, ctx->join_event, 0));
        }
    }
    // 2) totalSum: batched rotation rounds; groups of GR chunks are
    //    independent, and alternate between two streams when dual_rot
    if (pp.rp) {
        Range r("hespmv: totalSum rotations");
        uint64_t *V = dbuf, *CUR = V + GR * CT, *PB = CUR + GR * CT, *OB = PB + GR * CT;
        uint64_t *ks = OB + GR * CT;
        const int32_t *I = pp.rp->d_idx;
        const cudaStream_t st0 = st;
        if (pp.dual_rot) {  // fork: every HE-Mult product is ready on st
            CK(cudaEventRecord(ctx->copy_events[0], st0));
            CK(cudaStreamWaitEvent(ctx->aux_stream, ctx->copy_events[0], 0));
        }
        int64_t gi = -1;
        for (const RotOp &o : pp.rp->ops) {
            if (o.kind == RotOp::kVInit && pp.dual_rot) {  // a new group: its stream and scratch
                ++gi;
                st = (gi & 1) ? ctx->aux_stream : st0;
                V = dbuf + ((gi & 1) ? pp.rot_w : 0);
                CUR = V + GR * CT;
                PB = CUR + GR * CT;
                OB = PB + GR * CT;
                ks = OB + GR * CT;
            }
            switch (o.kind) {
                case RotOp::kVInit:
                    CK(op_ct_move(c, V, nullptr, prod, I + o.b, nullptr, false, o.m, st));
                    break;
                case RotOp::kCurFromProd:
                    CK(op_ct_move(c, CUR, I + o.a, prod, I + o.b, nullptr, false, o.m, st));
                    break;
                case RotOp::kCurFromV:
                    CK(op_ct_move(c, CUR, I + o.a, V, I + o.b, nullptr, false, o.m, st));
                    break;
                case RotOp::kElem: {
                    auto it = ctx->gk.find(o.g);
                    if (it == ctx->gk.end())
                        FAIL(HESPMV_E_INVALID, "missing Galois key for element " + std::to_string(o.g));
                    auto pit = ctx->perms.find(o.g);
                    if (pit == ctx->perms.end()) FAIL(HESPMV_E_INVALID, "missing Galois permutation");
                    if (ks_fused_supported(c)) {  // permutation and slot scatter inside the key switch
                        CK(rotate_fused_inplace(c, CUR, I + o.a, pit->second, it->second, o.m, ks, st));
                        break;
                    }
                    CK(op_ct_move(c, PB, nullptr, CUR, I + o.a, pit->second, false, o.m, st));
                    CK(keyswitch_n(c, PB + LN, CT, it->second, OB, PB, CT, LN, 1, o.m, ks, st));
                    CK(op_ct_move(c, CUR, I + o.a, OB, nullptr, nullptr, false, o.m, st));
                    break;
                }
                case RotOp::kAdd:
                    CK(op_ct_move(c, prod, I + o.a, CUR, I + o.b, nullptr, true, o.m, st));
                    break;
            }
        }
        st = st0;
        if (pp.dual_rot) {  // join
            CK(cudaEventRecord(ctx->join_event, ctx->aux_stream));
            CK(cudaStreamWaitEvent(st, ctx->join_event, 0));
        }
    }
    // 3) masked accumulation per partition
    Range r_mask("hespmv: masked accumulation");
    size_t k0 = 0;
    for (size_t i = 0; i < n_inst; ++i) {
        const Plan &pl = ms[i]->plan;
        for (size_t p = 0; p < pl.parts.size(); ++p) {
            uint64_t *res = Y[i] + p * CT;
            const Partition &P = pl.parts[p];
            if (P.n_chunks == 0) {
                CK(cudaMemsetAsync(res, 0, CT * 8, st));
                continue;
            }
            CK(op_mask_acc(c, prod + (k0 + P.chunk0) * CT, ms[i]->d_masks + P.chunk0, P.n_chunks, res,
                           st));
        }
        k0 += pl.chunks.size();
    }
    return HESPMV_OK;
}

// Persistent evaluation on `st` (one launch; see persist_build), replayed
// from a CUDA graph of the memset and the launch when graphs are enabled.
int spmv_persistent(hespmv_ctx *ctx, size_t n_inst, const hespmv_cssc *const *ms, const uint64_t *const *A,
                    const uint64_t *const *X, uint64_t *const *Y, cudaStream_t st) {
    const Ctx c = view(ctx);
    size_t total = 0, rot = 0;
    for (size_t i = 0; i < n_inst; ++i) {
        const int rc = prepare_matrix(ctx, ms[i], st);
        if (rc) return rc;
        total += ms[i]->plan.chunks.size();
        for (const Chunk &ch : ms[i]->plan.chunks) rot += ch.c > 1;
    }
    const size_t G = persist_group(ctx, total);
    uint64_t *ws = workspace(ctx, std::max<size_t>(256, persist_ws_words(c, total, rot, G) * 8));
    if (!ws) FAIL(HESPMV_E_NOMEM, "workspace allocation failed");
    PersistPlan *P = nullptr;
    int rc = persist_plan(ctx, n_inst, ms, A, X, Y, ws, G, &P);
    if (rc) return rc;
    const bool profiling = ctx->prof && ctx->prof->on;
    if (!ctx->use_graphs || profiling) return persist_enqueue(ctx, P, st);
    const std::vector<uint64_t> key{~0ull, (uint64_t)(uintptr_t)P, (uint64_t)ctx->persist_blocks};
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
        if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        rc = persist_enqueue(ctx, P, ctx->cap_stream);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) FAIL(HESPMV_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) FAIL(HESPMV_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        it = ctx->graphs.emplace(key, exec).first;
    }
    CK(cudaGraphLaunch(it->second, st));
    return HESPMV_OK;
}

// Evaluate on `st`: replays a CUDA graph of the same evaluation (same
// matrices, buffers and workspace) when one is cached, else captures one on
// the context's capture stream; runs eagerly while profiling is on or when
// graphs are disabled.
int spmv_core(hespmv_ctx *ctx, size_t n_inst, const hespmv_cssc *const *ms,
              const uint64_t *const *A, const uint64_t *const *X, uint64_t *const *Y,
              cudaStream_t st, bool pt_matrix = false, const uint64_t *hA = nullptr,
              const uint64_t *hX = nullptr, const std::vector<size_t> *gsz = nullptr,
              uint64_t *pkA = nullptr, uint64_t *pkX = nullptr, bool pipelined = false,
              cudaEvent_t copy_after = nullptr) {
    if (persist_usable(ctx, pt_matrix, hA)) return spmv_persistent(ctx, n_inst, ms, A, X, Y, st);
    SpmvPrep pp;
    size_t max_G = 0;
    if (gsz)
        for (size_t v : *gsz) max_G = std::max(max_G, v);
    int rc = spmv_prepare(ctx, n_inst, ms, pp, st, max_G);
    if (rc) return rc;
    if (gsz) pp.gsz = *gsz;
    pp.pipelined = pipelined;
    pp.copy_after = copy_after;
    pp.pt_matrix = pt_matrix;
    pp.hA = hA;
    pp.hX = hX;
    pp.pkA = pkA;
    pp.pkX = pkX;
    pp.pk_words = (int64_t)packed_ct_words(ctx->h);
    const size_t n_groups = mult_groups(pp, pp.total_chunks).size();
    // two or more HE-Mult groups of a host evaluation (always) or of a device
    // evaluation (schedule choice): two compute streams, groups alternating,
    // each stream with its own scratch, so one group's kernels fill the
    // other's tail waves
    if (!pt_matrix && n_groups > 1 && (hA || ctx->streams == 2)) {
        if (!ctx->aux_stream) CK(cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking));
        if (!ctx->join_event) CK(cudaEventCreateWithFlags(&ctx->join_event, cudaEventDisableTiming));
        pp.dual = true;
        pp.need_bytes += pp.mult_w * 8;
    }
    // two or more rotation groups: alternate them over two streams too
    if (ctx->streams == 2 && pp.rp && pp.rot_chunks > pp.GR) {
        if (!ctx->aux_stream) CK(cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking));
        if (!ctx->join_event) CK(cudaEventCreateWithFlags(&ctx->join_event, cudaEventDisableTiming));
        pp.dual_rot = true;
        pp.need_bytes = std::max(pp.need_bytes, (pp.total_chunks * 2 * (size_t)ctx->h.L * ctx->h.N + 2 * pp.rot_w) * 8);
    }
    // one event per upload group plus the fork
    const size_t n_events = std::max<size_t>(hA ? n_groups + 1 : (pp.dual ? 1 : 0), pp.dual_rot ? 1 : 0);
    if (hA && !ctx->copy_stream) CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    while (ctx->copy_events.size() < n_events) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->copy_events.push_back(e);
    }
    uint64_t *ws = workspace(ctx, pp.need_bytes);
    if (!ws) FAIL(HESPMV_E_NOMEM, "workspace allocation failed");
    const bool profiling = ctx->prof && ctx->prof->on;
    // pipelined host evaluations launch eagerly: a graph launch would order
    // its uploads after the stream's earlier evaluations
    if (!ctx->use_graphs || profiling || pipelined) return spmv_enqueue(ctx, n_inst, ms, A, X, Y, pp, ws, st);
    std::vector<uint64_t> key;
    key.push_back((uint64_t)(uintptr_t)ws);
    key.push_back(pt_matrix ? 1 : 0);
    key.push_back((uint64_t)(uintptr_t)hA);
    key.push_back((uint64_t)(uintptr_t)hX);
    key.push_back((uint64_t)(uintptr_t)pkA);
    key.push_back((uint64_t)(uintptr_t)pkX);
    key.push_back(pp.dual ? 1 : 0);
    key.push_back(pp.G);
    for (size_t v : pp.gsz) key.push_back(v);
    for (size_t i = 0; i < n_inst; ++i) {
        key.push_back(ms[i]->uid);
        key.push_back((uint64_t)(uintptr_t)A[i]);
        key.push_back((uint64_t)(uintptr_t)X[i]);
        key.push_back((uint64_t)(uintptr_t)Y[i]);
    }
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
        if (ctx->graphs.size() >= 64) {
            for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
            ctx->graphs.clear();
        }
        if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        rc = spmv_enqueue(ctx, n_inst, ms, A, X, Y, pp, ws, ctx->cap_stream);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) FAIL(HESPMV_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) FAIL(HESPMV_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        it = ctx->graphs.emplace(key, exec).first;
    }
    CK(cudaGraphLaunch(it->second, st));
    return HESPMV_OK;
}

}  // namespace

extern "C" {

const char *hespmv_version(void) { return "hespmv 0.1 (sm_103a)"; }

const char *hespmv_last_error(const hespmv_ctx *ctx) {
    return ctx ? ctx->err.c_str() : "null context";
}

int hespmv_create(const hespmv_params *p, hespmv_ctx **out) {
    if (!p || !out) return HESPMV_E_INVALID;
    *out = nullptr;
    if ((p->alloc == nullptr) != (p->free == nullptr)) return HESPMV_E_INVALID;
    if (p->rot_policy != HESPMV_ROT_POW2 && p->rot_policy != HESPMV_ROT_EXACT) return HESPMV_E_INVALID;
    hespmv_ctx *ctx = new hespmv_ctx();
    ctx->p = *p;
    ctx->device = p->device;
    if (!build_tables(*p, ctx->h, ctx->err)) {
        const int code = HESPMV_E_UNSUPPORTED;
        *out = ctx;  // keep the message readable
        return code;
    }
    if (p->device == -1) {  // host-only: format layer and parameter tables
        *out = ctx;
        return HESPMV_OK;
    }
    DeviceGuard g(ctx->device);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || p->device < 0 || p->device >= ndev) {
        cudaGetLastError();
        ctx->err = "no CUDA device " + std::to_string(p->device);
        *out = ctx;
        return HESPMV_E_CUDA;
    }
    HostTables &h = ctx->h;
    DevTables &d = ctx->d;
    bool ok = upload(ctx, d.mc, h.mc) && upload(ctx, d.tw, h.tw) && upload(ctx, d.modup_inv, h.modup_inv) &&
              upload(ctx, d.modup_mod, h.modup_mod) && upload(ctx, d.md_pk, h.md_pk) &&
              upload(ctx, d.md_phat, h.md_phat) && upload(ctx, d.md_t, h.md_t) &&
              upload(ctx, d.md_pinv, h.md_pinv) && upload(ctx, d.p_mod_q, h.p_mod_q) &&
              upload(ctx, d.p_mont, h.p_mont) && upload(ctx, d.p_mont2, h.p_mont2) &&
              upload(ctx, d.slot_idx, h.slot_idx) && upload(ctx, d.dec, h.dec) &&
              upload(ctx, d.dec_inv_q, h.dec_inv_q) && upload(ctx, d.t_mod, h.t_mod) &&
              upload(ctx, d.ks_zc, h.ks_zc) && upload(ctx, d.ks_yc, h.ks_yc) &&
              upload(ctx, d.md_phat_t, h.md_phat_t) && upload(ctx, d.modup_modw, h.modup_modw) &&
              upload(ctx, d.md_phat_tw, h.md_phat_tw);
    if (ok && h.scheme == HESPMV_SCHEME_BFV)
        ok = upload(ctx, d.bfv_delta, h.bfv_delta) && upload(ctx, d.bfv_const, h.bfv_const);
    if (ok) {
        d.err = owned<int>(ctx, 1);
        ok = d.err && cudaMemset(d.err, 0, sizeof(int)) == cudaSuccess;
    }
    if (ok && ks_prepare(view(ctx)) != cudaSuccess) {
        cudaGetLastError();
        ctx->err = "key-switch launch setup failed";
        *out = ctx;
        return HESPMV_E_CUDA;
    }
    if (!ok) {
        ctx->err = "table upload failed";
        *out = ctx;
        return HESPMV_E_NOMEM;
    }
    *out = ctx;
    return HESPMV_OK;
}

void hespmv_destroy(hespmv_ctx *ctx) {
    if (!ctx) return;
    if (ctx->codec) ckks_codec_free(ctx->codec);
    if (ctx->crt) crt_real_free(ctx->crt);
    if (ctx->device < 0) {
        delete ctx;
        return;
    }
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    for (auto &a : ctx->allocs) dev_free(ctx, a.first);
    dev_free(ctx, ctx->ws);
    dev_free(ctx, ctx->io);
    for (auto &kv : ctx->rot_plans) {
        dev_free(ctx, kv.second->d_idx);
        delete kv.second;
    }
    for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
    drop_persist_plans(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
    for (int s = 0; s < hespmv_ctx::kSlots; ++s) {
        if (ctx->slot_free[s]) cudaEventDestroy(ctx->slot_free[s]);
        dev_free(ctx, ctx->aio[s]);
    }
    if (ctx->join_event) cudaEventDestroy(ctx->join_event);
    if (ctx->err_host) cudaFreeHost(ctx->err_host);
    for (cudaEvent_t e : ctx->copy_events) cudaEventDestroy(e);
    delete ctx->prof;
    delete ctx;
}

int hespmv_ctx_moduli(const hespmv_ctx *ctx, uint64_t *moduli, uint64_t *psi, uint64_t *zeta) {
    if (!ctx || ctx->h.q.empty()) return HESPMV_E_INVALID;
    const int LK = ctx->h.L + ctx->h.K;
    if (moduli) memcpy(moduli, ctx->h.q.data(), LK * 8);
    if (psi) memcpy(psi, ctx->h.psi.data(), LK * 8);
    if (zeta) *zeta = ctx->h.psi[LK];
    return HESPMV_OK;
}

int hespmv_ctx_device_bytes(const hespmv_ctx *ctx, size_t *bytes) {
    if (!ctx || !bytes) return HESPMV_E_INVALID;
    *bytes = ctx->owned_bytes + ctx->ws_bytes + ctx->io_bytes;
    for (size_t b : ctx->aio_bytes) *bytes += b;
    return HESPMV_OK;
}

int hespmv_keygen(hespmv_ctx *ctx, uint64_t seed, const int32_t *rot_steps, size_t n_steps) {
    if (!ctx || ctx->h.q.empty()) return HESPMV_E_INVALID;
    if (n_steps && !rot_steps) FAIL(HESPMV_E_INVALID, "rot_steps is NULL");
    NEED_DEVICE(ctx);
    DeviceGuard g(ctx->device);
    const Ctx c = view(ctx);
    const int64_t N = c.N, L = c.L, LK = c.L + c.K, LKN = LK * N;
    if (!ctx->sk) {
        ctx->sk = owned<uint64_t>(ctx, LKN);
        ctx->pk = owned<uint64_t>(ctx, 2 * L * N);
        ctx->rlk = owned<uint64_t>(ctx, (size_t)c.dnum * 2 * LKN);
        if (!ctx->sk || !ctx->pk || !ctx->rlk) FAIL(HESPMV_E_NOMEM, "key allocation failed");
    }
    void *tmp = dev_alloc(ctx, (size_t)(2 * LKN + N) * 8);
    if (!tmp) FAIL(HESPMV_E_NOMEM, "keygen scratch allocation failed");
    uint64_t *tmp_e = (uint64_t *)tmp, *sp = tmp_e + LKN;
    int64_t *coef = (int64_t *)(sp + LKN);
    int rc = HESPMV_OK;
    do {
        // secret key s: ternary, NTT over Q u P
        if (op_sample_signed(c, seed, kSecretStream, 0, kTernary, coef, 1, 0) ||
            op_signed_to_limbs(c, coef, ctx->sk, 0, (int)LK, 1, 0) ||
            launch_ntt(c, ctx->sk, 0, (int)LK, 1, LKN, false, 0)) {
            rc = HESPMV_E_CUDA;
            break;
        }
        // public key (-a s + t e, a)
        uint64_t *pk1 = ctx->pk + L * N;
        if (op_sample_uniform(c, seed, kPkAStream, pk1, 0, (int)L, 0) ||
            op_sample_signed(c, seed, kPkEStream, 0, kCbd21, coef, 1, 0) ||
            op_signed_to_limbs(c, coef, tmp_e, 0, (int)L, 1, 0) ||
            launch_ntt(c, tmp_e, 0, (int)L, 1, L * N, false, 0) ||
            op_pk_combine(c, pk1, tmp_e, ctx->sk, ctx->pk, 0)) {
            rc = HESPMV_E_CUDA;
            break;
        }
        // relinearisation key: s' = s^2
        if (op_mul_limbs(c, ctx->sk, ctx->sk, sp, 0, (int)LK, 1, 0)) {
            rc = HESPMV_E_CUDA;
            break;
        }
        if ((rc = make_ksk(ctx, seed, 0, sp, ctx->rlk, tmp_e, coef))) break;
        // Galois keys
        std::set<uint32_t> elts;
        const int64_t half = N / 2;
        if (rot_steps == nullptr) {
            if (ctx->p.rot_policy == HESPMV_ROT_POW2)
                for (int64_t b = 1; b < half; b <<= 1) elts.insert(pow5((uint64_t)b, 2 * N));
        } else {
            for (size_t i = 0; i < n_steps; ++i)
                for (uint32_t e : rotation_chain(ctx, rot_steps[i])) elts.insert(e);
        }
        for (uint32_t e : elts) {
            uint64_t *key = ctx->gk.count(e) ? ctx->gk[e] : owned<uint64_t>(ctx, (size_t)c.dnum * 2 * LKN);
            const int32_t *perm = galois_perm(ctx, e);
            if (!key || !perm) {
                rc = HESPMV_E_NOMEM;
                ctx->err = "Galois key allocation failed";
                break;
            }
            ctx->gk[e] = key;
            if (op_permute(c, ctx->sk, sp, perm, LK, 0)) {
                rc = HESPMV_E_CUDA;
                break;
            }
            if ((rc = make_ksk(ctx, seed, e, sp, key, tmp_e, coef))) break;
        }
    } while (0);
    cudaError_t e = cudaDeviceSynchronize();
    dev_free(ctx, tmp);
    if (rc == HESPMV_E_CUDA && ctx->err.empty()) ctx->err = "keygen kernel launch failed";
    if (rc) return rc;
    if (e != cudaSuccess) FAIL(HESPMV_E_CUDA, std::string("keygen: ") + cudaGetErrorString(e));
    ctx->have_keys = true;
    ctx->has_sk = true;
    return HESPMV_OK;
}

int hespmv_key_export(hespmv_ctx *ctx, int32_t which, uint32_t galois_elt, uint64_t *host_out,
                      size_t n_words) {
    if (!ctx || !host_out) return HESPMV_E_INVALID;
    if (!ctx->have_keys) FAIL(HESPMV_E_INVALID, "no keys");
    NEED_DEVICE(ctx);
    DeviceGuard g(ctx->device);
    const size_t N = ctx->h.N, L = ctx->h.L, LK = L + ctx->h.K;
    const uint64_t *src = nullptr;
    size_t words = 0;
    switch (which) {
        case HESPMV_KEY_SECRET: src = ctx->sk; words = LK * N; break;
        case HESPMV_KEY_PUBLIC: src = ctx->pk; words = 2 * L * N; break;
        case HESPMV_KEY_RELIN: src = ctx->rlk; words = ctx->h.dnum * 2 * LK * N; break;
        case HESPMV_KEY_GALOIS: {
            auto it = ctx->gk.find(galois_elt);
            if (it == ctx->gk.end()) FAIL(HESPMV_E_INVALID, "no Galois key for that element");
            src = it->second;
            words = ctx->h.dnum * 2 * LK * N;
            break;
        }
        default: FAIL(HESPMV_E_INVALID, "unknown key kind");
    }
    if (n_words != words) FAIL(HESPMV_E_INVALID, "n_words does not match the key size");
    CK(cudaMemcpy(host_out, src, words * 8, cudaMemcpyDeviceToHost));
    if (which == HESPMV_KEY_RELIN || which == HESPMV_KEY_GALOIS) {
        // out of Montgomery form: x * 2^-64 mod q_l
        typedef unsigned __int128 u128;
        for (size_t l = 0; l < LK; ++l) {
            const uint64_t q = ctx->h.q[l];
            const uint64_t r = (uint64_t)(((u128)1 << 64) % q);
            uint64_t rinv = 1, b = r, e = q - 2;  // r^(q-2) = r^-1
            for (; e; e >>= 1) {
                if (e & 1) rinv = (uint64_t)((u128)rinv * b % q);
                b = (uint64_t)((u128)b * b % q);
            }
            for (size_t blk = 0; blk < words / (LK * N); ++blk) {
                uint64_t *w = host_out + (blk * LK + l) * N;
                for (size_t k = 0; k < N; ++k) w[k] = (uint64_t)((u128)w[k] * rinv % q);
            }
        }
    }
    return HESPMV_OK;
}

// rotation counts, distinct steps and the schedule-cache id of a new plan
static void finish_cssc(hespmv_ctx *ctx, hespmv_cssc *m) {
    std::set<int32_t> st;
    std::vector<int32_t> steps;
    std::vector<uint8_t> orig;
    m->n_rot = m->n_ks = 0;
    for (const Chunk &ch : m->plan.chunks) {
        total_sum_steps(ch.h, ch.c, steps, orig);
        m->n_rot += (int64_t)steps.size();
        for (int32_t k : steps) {
            st.insert(k);
            m->n_ks += (int64_t)rotation_chain(ctx, k).size();
        }
    }
    m->steps.assign(st.begin(), st.end());
    m->uid = ctx->next_uid++;
}

int hespmv_encode_cssc(hespmv_ctx *ctx, int32_t rows, int32_t cols, int64_t nnz,
                       const int64_t *rowptr, const int32_t *colidx, const int64_t *vals,
                       int64_t max_abs_x, hespmv_cssc **out) {
    if (!ctx || !out || ctx->h.q.empty()) return HESPMV_E_INVALID;
    *out = nullptr;
    hespmv_cssc *m = new hespmv_cssc();
    m->ctx = ctx;
    std::string err = build_plan(rows, cols, nnz, rowptr, colidx, vals, ctx->h.slots, m->plan);
    if (!err.empty()) {
        delete m;
        FAIL(HESPMV_E_INVALID, "malformed CSR: " + err);
    }
    if (max_abs_x > 0 && vals && ctx->h.scheme != HESPMV_SCHEME_CKKS) {
        typedef unsigned __int128 u128;
        const u128 half_t = (u128)ctx->h.t;
        for (int32_t i = 0; i < rows; ++i) {
            u128 s = 0;
            bool big = false;
            for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
                const int64_t v = vals[k];
                s += (u128)(v < 0 ? -(u128)v : (u128)v);
                if (s > ((u128)1 << 64)) big = true;
            }
            if (big || 2 * s * (u128)max_abs_x >= half_t) {
                delete m;
                FAIL(HESPMV_E_RANGE, "row " + std::to_string(i) +
                                         ": sum |a_ij| * max|x| could reach t/2");
            }
        }
    }
    finish_cssc(ctx, m);
    *out = m;
    return HESPMV_OK;
}

void hespmv_cssc_free(hespmv_cssc *m) {
    if (!m) return;
    if (m->d_masks) {
        DeviceGuard g(m->ctx->device);
        cudaDeviceSynchronize();
        dev_free(m->ctx, (void *)m->d_masks);
    }
    delete m;
}

int hespmv_cssc_info(const hespmv_cssc *m, int32_t *n_parts, int32_t *n_chunks, int64_t *n_rot,
                     int64_t *n_keyswitch, int32_t *rows, int32_t *cols, int64_t *nnz) {
    if (!m) return HESPMV_E_INVALID;
    if (n_parts) *n_parts = (int32_t)m->plan.parts.size();
    if (n_chunks) *n_chunks = (int32_t)m->plan.chunks.size();
    if (n_rot) *n_rot = m->n_rot;
    if (n_keyswitch) *n_keyswitch = m->n_ks;
    if (rows) *rows = m->plan.rows;
    if (cols) *cols = m->plan.cols;
    if (nnz) *nnz = m->plan.nnz;
    return HESPMV_OK;
}

int hespmv_cssc_chunks(const hespmv_cssc *m, int32_t *h, int32_t *c, int32_t *part) {
    if (!m) return HESPMV_E_INVALID;
    for (size_t k = 0; k < m->plan.chunks.size(); ++k) {
        if (h) h[k] = m->plan.chunks[k].h;
        if (c) c[k] = m->plan.chunks[k].c;
        if (part) part[k] = m->plan.chunks[k].part;
    }
    return HESPMV_OK;
}

int hespmv_cssc_colindex(const hespmv_cssc *m, const int32_t **ci, size_t *len) {
    if (!m || !ci || !len || m->shape_only) return HESPMV_E_INVALID;
    *ci = m->plan.slot_ci.data();
    *len = m->plan.slot_ci.size();
    return HESPMV_OK;
}

int hespmv_cssc_arrays(const hespmv_cssc *m, int32_t part, const int64_t **va, const int32_t **ci,
                       size_t *nnz_part, const int64_t **cp, size_t *cp_len, const int32_t **rm,
                       size_t *rm_len, int32_t *row0) {
    if (!m || m->shape_only || part < 0 || part >= (int32_t)m->plan.parts.size())
        return HESPMV_E_INVALID;
    const Partition &P = m->plan.parts[part];
    if (va) *va = P.va.data();
    if (ci) *ci = P.ci.data();
    if (nnz_part) *nnz_part = P.va.size();
    if (cp) *cp = P.cp.data();
    if (cp_len) *cp_len = P.cp.size();
    if (rm) *rm = P.rm.data();
    if (rm_len) *rm_len = P.rm.size();
    if (row0) *row0 = P.row0;
    return HESPMV_OK;
}

int hespmv_cssc_rotation_steps(const hespmv_cssc *m, int32_t *steps, size_t cap, size_t *n) {
    if (!m || !n) return HESPMV_E_INVALID;
    *n = m->steps.size();
    for (size_t i = 0; i < m->steps.size() && i < cap && steps; ++i) steps[i] = m->steps[i];
    return HESPMV_OK;
}

int hespmv_ctbatch_create(hespmv_ctx *ctx, size_t n_ct, hespmv_ctbatch **out) {
    if (!ctx || !out) return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    DeviceGuard g(ctx->device);
    return batch_new(ctx, n_ct, out);
}

void hespmv_ctbatch_free(hespmv_ctbatch *b) {
    if (!b) return;
    DeviceGuard g(b->ctx->device);
    dev_free(b->ctx, b->data);
    delete b;
}

int hespmv_ctbatch_data(const hespmv_ctbatch *b, uint64_t **dev, size_t *n_ct) {
    if (!b) return HESPMV_E_INVALID;
    if (dev) *dev = b->data;
    if (n_ct) *n_ct = b->n;
    return HESPMV_OK;
}

int hespmv_ctbatch_upload(hespmv_ctbatch *b, const uint64_t *host, size_t n_ct, void *stream) {
    if (!b || !host || n_ct > b->n) return HESPMV_E_INVALID;
    hespmv_ctx *ctx = b->ctx;
    DeviceGuard g(ctx->device);
    CK(cudaMemcpyAsync(b->data, host, n_ct * 2 * ctx->h.L * ctx->h.N * 8, cudaMemcpyHostToDevice,
                       (cudaStream_t)stream));
    return HESPMV_OK;
}

int hespmv_ctbatch_download(const hespmv_ctbatch *b, uint64_t *host, size_t n_ct, void *stream) {
    if (!b || !host || n_ct > b->n) return HESPMV_E_INVALID;
    hespmv_ctx *ctx = b->ctx;
    DeviceGuard g(ctx->device);
    CK(cudaMemcpyAsync(host, b->data, n_ct * 2 * ctx->h.L * ctx->h.N * 8, cudaMemcpyDeviceToHost,
                       (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return HESPMV_OK;
}

// ------------------------------------------------------------ serialization
// Little-endian byte streams; every field is 8-byte aligned.  Readers check
// each length against the bytes left before touching or allocating anything.
}  // extern "C"

namespace {

const uint32_t kCsscMagic = 0x53435348u;  // "HSCS"
const uint32_t kCtMagic = 0x54435348u;    // "HSCT"
const uint32_t kKeyMagic = 0x594B5348u;   // "HSKY"
const uint32_t kSerVersion = 1;

struct Writer {
    uint8_t *p;
    size_t cap, n = 0;
    void put(const void *src, size_t bytes) {
        if (p && n + bytes <= cap) std::memcpy(p + n, src, bytes);
        n += bytes;
    }
    template <class T>
    void val(T v) { put(&v, sizeof(T)); }
    template <class T>
    void arr(const std::vector<T> &v) {
        put(v.data(), v.size() * sizeof(T));
        const size_t pad = (8 - (v.size() * sizeof(T)) % 8) % 8;
        const uint64_t zero = 0;
        put(&zero, pad);
    }
};

struct Reader {
    const uint8_t *p;
    size_t len, n = 0;
    bool ok = true;
    bool take(void *dst, size_t bytes) {
        if (!ok || bytes > len - n) return ok = false;
        std::memcpy(dst, p + n, bytes);
        n += bytes;
        return true;
    }
    template <class T>
    bool val(T &v) { return take(&v, sizeof(T)); }
    template <class T>
    bool arr(std::vector<T> &v, uint64_t count) {
        if (!ok || count > (len - n) / sizeof(T)) return ok = false;
        v.resize(count);
        if (!take(v.data(), count * sizeof(T))) return false;
        const size_t pad = (8 - (count * sizeof(T)) % 8) % 8;
        if (pad > len - n) return ok = false;
        n += pad;
        return true;
    }
};

// FNV-1a over the ciphertext moduli and t: ciphertexts load only into a
// context with the same ring
uint64_t ring_fingerprint(const hespmv_ctx *ctx) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) {
        for (int b = 0; b < 8; ++b) {
            h ^= (v >> (8 * b)) & 0xff;
            h *= 1099511628211ull;
        }
    };
    mix((uint64_t)ctx->h.log2n);
    for (int l = 0; l < ctx->h.L; ++l) mix(ctx->h.q[l]);
    mix(ctx->h.t);
    mix((uint64_t)ctx->h.scheme);
    mix((uint64_t)ctx->h.scale_bits);
    mix((uint64_t)ctx->h.mask_scale_bits);
    return h;
}

}  // namespace

extern "C" {

int hespmv_cssc_serialize(const hespmv_cssc *m, int32_t kind, void *buf, size_t cap, size_t *len) {
    if (!m || !len || (kind != HESPMV_SER_FULL && kind != HESPMV_SER_SHAPE)) return HESPMV_E_INVALID;
    if (kind == HESPMV_SER_FULL && m->shape_only) return HESPMV_E_INVALID;
    const Plan &pl = m->plan;
    Writer w{(uint8_t *)buf, cap};
    w.val(kCsscMagic);
    w.val(kSerVersion);
    w.val((uint32_t)kind);
    w.val((uint32_t)pl.s);
    w.val((int32_t)pl.rows);
    w.val((int32_t)pl.cols);
    w.val((int64_t)pl.nnz);
    w.val((uint64_t)pl.parts.size());
    for (const Partition &P : pl.parts) {
        w.val((int32_t)P.row0);
        w.val((int32_t)P.rows);
        w.val((int64_t)P.va.size());
        w.val((int64_t)P.cp.size());
        w.arr(P.cp);
        if (kind == HESPMV_SER_FULL) {
            w.arr(P.va);
            w.arr(P.ci);
            w.arr(P.rm);
        }
    }
    *len = w.n;
    if (buf && cap < w.n) return HESPMV_E_INVALID;
    return HESPMV_OK;
}

int hespmv_cssc_deserialize(hespmv_ctx *ctx, const void *buf, size_t len, hespmv_cssc **out) {
    if (!ctx || !buf || !out || ctx->h.q.empty()) return HESPMV_E_INVALID;
    *out = nullptr;
    Reader r{(const uint8_t *)buf, len};
    uint32_t magic = 0, ver = 0, kind = 0, s = 0;
    int32_t rows = 0, cols = 0;
    int64_t nnz = 0;
    uint64_t n_parts = 0;
    r.val(magic), r.val(ver), r.val(kind), r.val(s), r.val(rows), r.val(cols), r.val(nnz), r.val(n_parts);
    if (!r.ok || magic != kCsscMagic || ver != kSerVersion) FAIL(HESPMV_E_INVALID, "not a CSSC stream");
    if (kind != HESPMV_SER_FULL && kind != HESPMV_SER_SHAPE) FAIL(HESPMV_E_INVALID, "unknown CSSC kind");
    if ((int32_t)s != ctx->h.slots) FAIL(HESPMV_E_INVALID, "CSSC chunk capacity differs from the context's");
    if (rows < 0 || cols < 0 || nnz < 0) FAIL(HESPMV_E_INVALID, "negative CSSC size");
    const uint64_t want_parts = rows ? ((uint64_t)rows + s - 1) / s : 0;
    if (n_parts != want_parts) FAIL(HESPMV_E_INVALID, "partition count does not match rows");
    const bool full = kind == HESPMV_SER_FULL;
    hespmv_cssc *m = new hespmv_cssc();
    m->ctx = ctx;
    m->shape_only = !full;
    Plan &pl = m->plan;
    pl.rows = rows, pl.cols = cols, pl.nnz = nnz, pl.s = (int32_t)s;
    std::string err;
    int64_t total = 0;
    for (uint64_t k = 0; k < n_parts && err.empty(); ++k) {
        Partition P;
        int64_t nnz_part = 0, cp_len = 0;
        r.val(P.row0), r.val(P.rows), r.val(nnz_part), r.val(cp_len);
        if (!r.ok) { err = "truncated"; break; }
        if ((int64_t)P.row0 != (int64_t)k * s || P.rows != std::min<int64_t>(s, rows - (int64_t)k * s)) {
            err = "partition bounds";
            break;
        }
        if (nnz_part < 0 || cp_len < 1 || !r.arr(P.cp, (uint64_t)cp_len)) { err = "bad CP"; break; }
        if (P.cp[0] != 0 || P.cp.back() != nnz_part) { err = "CP ends"; break; }
        for (int64_t j = 0; j + 1 < cp_len && err.empty(); ++j) {
            const int64_t h = P.cp[j + 1] - P.cp[j];
            if (h < 1 || h > P.rows) err = "column height out of range";
            else if (j > 0 && h > P.cp[j] - P.cp[j - 1]) err = "column heights increase";
        }
        if (!err.empty()) break;
        total += nnz_part;
        if (full) {
            if (!r.arr(P.va, (uint64_t)nnz_part) || !r.arr(P.ci, (uint64_t)nnz_part) ||
                !r.arr(P.rm, (uint64_t)P.rows)) {
                err = "truncated";
                break;
            }
            std::vector<uint8_t> seen(P.rows, 0);
            for (int32_t v : P.rm) {
                if (v < 0 || v >= P.rows || seen[v]) { err = "RM is not a permutation"; break; }
                seen[v] = 1;
            }
            // sorted row p holds CI[CP[j] + p] for the columns j taller than p;
            // a CSR row's columns ascend strictly
            for (int64_t j = 0; j + 1 < cp_len && err.empty(); ++j)
                for (int64_t p = 0; p < P.cp[j + 1] - P.cp[j]; ++p) {
                    const int32_t c = P.ci[P.cp[j] + p];
                    if (c < 0 || c >= cols) { err = "column index out of range"; break; }
                    if (j > 0 && c <= P.ci[P.cp[j - 1] + p]) { err = "row columns not ascending"; break; }
                }
        } else {
            P.va.assign((size_t)nnz_part, 0);
            P.ci.assign((size_t)nnz_part, -1);
        }
        pl.parts.push_back(std::move(P));
    }
    if (err.empty() && (total != nnz || r.n != len)) err = "length mismatch";
    if (!err.empty()) {
        delete m;
        FAIL(HESPMV_E_INVALID, "CSSC stream: " + err);
    }
    chunk_plan(pl);
    finish_cssc(ctx, m);
    *out = m;
    return HESPMV_OK;
}

int hespmv_ctbatch_serialize(const hespmv_ctbatch *b, void *buf, size_t cap, size_t *len) {
    if (!b || !len) return HESPMV_E_INVALID;
    hespmv_ctx *ctx = b->ctx;
    const size_t words = b->n * 2 * (size_t)ctx->h.L * ctx->h.N;
    const size_t head = 4 * 4 + 2 * 8;
    *len = head + words * 8;
    if (!buf) return HESPMV_OK;
    if (cap < *len) FAIL(HESPMV_E_INVALID, "buffer too small");
    Writer w{(uint8_t *)buf, cap};
    w.val(kCtMagic);
    w.val(kSerVersion);
    w.val((uint32_t)ctx->h.log2n);
    w.val((uint32_t)ctx->h.L);
    w.val((uint64_t)b->n);
    w.val(ring_fingerprint(ctx));
    DeviceGuard g(ctx->device);
    CK(cudaMemcpy((uint8_t *)buf + head, b->data, words * 8, cudaMemcpyDeviceToHost));
    return HESPMV_OK;
}

int hespmv_ctbatch_deserialize(hespmv_ctx *ctx, const void *buf, size_t len, hespmv_ctbatch **out) {
    if (!ctx || !buf || !out) return HESPMV_E_INVALID;
    *out = nullptr;
    NEED_DEVICE(ctx);
    Reader r{(const uint8_t *)buf, len};
    uint32_t magic = 0, ver = 0, log2n = 0, L = 0;
    uint64_t n = 0, fp = 0;
    r.val(magic), r.val(ver), r.val(log2n), r.val(L), r.val(n), r.val(fp);
    if (!r.ok || magic != kCtMagic || ver != kSerVersion) FAIL(HESPMV_E_INVALID, "not a ciphertext stream");
    if ((int)log2n != ctx->h.log2n || (int)L != ctx->h.L || fp != ring_fingerprint(ctx))
        FAIL(HESPMV_E_INVALID, "ciphertexts belong to another ring");
    const size_t N = ctx->h.N, per_ct = 2 * (size_t)L * N;
    if (n > (len - r.n) / 8 / per_ct || r.n + n * per_ct * 8 != len)
        FAIL(HESPMV_E_INVALID, "ciphertext stream length mismatch");
    const uint8_t *src = (const uint8_t *)buf + r.n;
    for (size_t i = 0; i < n * 2 * L; ++i) {  // every residue reduced mod its prime
        const uint64_t q = ctx->h.q[i % L];
        for (size_t k = 0; k < N; ++k) {
            uint64_t v;
            std::memcpy(&v, src + (i * N + k) * 8, 8);
            if (v >= q) FAIL(HESPMV_E_INVALID, "residue not reduced mod q");
        }
    }
    DeviceGuard g(ctx->device);
    hespmv_ctbatch *b = nullptr;
    int rc = batch_new(ctx, n, &b);
    if (rc) return rc;
    if (n && cudaMemcpy(b->data, src, n * per_ct * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
        hespmv_ctbatch_free(b);
        FAIL(HESPMV_E_CUDA, "ciphertext upload failed");
    }
    *out = b;
    return HESPMV_OK;
}

// Encode and encrypt (or, plain, only encode) the chunks of one operand.
// BGV: integer values (matrix values from the plan, or x); CKKS: real values
// `real` (the matrix's CSR values, or x) encoded at 2^scale_bits.
// ------------------------------------------------------------ key transfer
// "HSKY", version, what, Galois key count, ring fingerprint, then [sk], pk,
// rlk and each Galois key (u64 element, key), all as the device holds them.
int hespmv_keys_serialize(hespmv_ctx *ctx, int32_t what, void *buf, size_t cap, size_t *len) {
    if (!ctx || !len || (what != HESPMV_KEYS_EVAL && what != HESPMV_KEYS_ALL)) return HESPMV_E_INVALID;
    if (!ctx->have_keys) FAIL(HESPMV_E_INVALID, "no keys");
    if (what == HESPMV_KEYS_ALL && !ctx->has_sk) FAIL(HESPMV_E_INVALID, "no secret key in this context");
    NEED_DEVICE(ctx);
    const size_t N = ctx->h.N, L = ctx->h.L, LK = L + ctx->h.K, KW = (size_t)ctx->h.dnum * 2 * LK * N;
    const size_t words = (what == HESPMV_KEYS_ALL ? LK * N : 0) + 2 * L * N + KW + ctx->gk.size() * (1 + KW);
    *len = 24 + words * 8;
    if (!buf) return HESPMV_OK;
    if (cap < *len) FAIL(HESPMV_E_INVALID, "buffer too small");
    Writer w{(uint8_t *)buf, cap};
    w.val(kKeyMagic);
    w.val(kSerVersion);
    w.val((uint32_t)what);
    w.val((uint32_t)ctx->gk.size());
    w.val(ring_fingerprint(ctx));
    DeviceGuard g(ctx->device);
    uint8_t *p = (uint8_t *)buf + w.n;
    auto take = [&](const uint64_t *dev, size_t n) {
        const cudaError_t e = cudaMemcpy(p, dev, n * 8, cudaMemcpyDeviceToHost);
        p += n * 8;
        return e == cudaSuccess;
    };
    bool ok = true;
    if (what == HESPMV_KEYS_ALL) ok = take(ctx->sk, LK * N);
    ok = ok && take(ctx->pk, 2 * L * N) && take(ctx->rlk, KW);
    for (auto &kv : ctx->gk) {
        const uint64_t e = kv.first;
        std::memcpy(p, &e, 8);
        p += 8;
        ok = ok && take(kv.second, KW);
    }
    if (!ok) FAIL(HESPMV_E_CUDA, "key download failed");
    return HESPMV_OK;
}

int hespmv_keys_deserialize(hespmv_ctx *ctx, const void *buf, size_t len) {
    if (!ctx || !buf) return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    Reader r{(const uint8_t *)buf, len};
    uint32_t magic = 0, ver = 0, what = 0, ng = 0;
    uint64_t fp = 0;
    r.val(magic), r.val(ver), r.val(what), r.val(ng), r.val(fp);
    if (!r.ok || magic != kKeyMagic || ver != kSerVersion) FAIL(HESPMV_E_INVALID, "not a key stream");
    if (what != HESPMV_KEYS_EVAL && what != HESPMV_KEYS_ALL) FAIL(HESPMV_E_INVALID, "unknown key kind");
    if (fp != ring_fingerprint(ctx)) FAIL(HESPMV_E_INVALID, "keys belong to another ring");
    const size_t N = ctx->h.N, L = ctx->h.L, LK = L + ctx->h.K, KW = (size_t)ctx->h.dnum * 2 * LK * N;
    const size_t words = (what == HESPMV_KEYS_ALL ? LK * N : 0) + 2 * L * N + KW;
    if (ng > (len - r.n) / 8 / (1 + KW) || r.n + (words + (size_t)ng * (1 + KW)) * 8 != len)
        FAIL(HESPMV_E_INVALID, "key stream length mismatch");
    const uint8_t *p = (const uint8_t *)buf + r.n;
    // every residue below its prime: limb l of an [.][LK][N] or [.][L][N] block
    auto check = [&](const uint8_t *src, size_t n, size_t limbs) {
        for (size_t i = 0; i < n; ++i) {
            uint64_t v;
            std::memcpy(&v, src + i * 8, 8);
            if (v >= ctx->h.q[(i / N) % limbs]) return false;
        }
        return true;
    };
    {
        const uint8_t *q = p;
        bool ok = true;
        if (what == HESPMV_KEYS_ALL) ok = check(q, LK * N, LK), q += LK * N * 8;
        ok = ok && check(q, 2 * L * N, L);
        q += 2 * L * N * 8;
        ok = ok && check(q, KW, LK);
        q += KW * 8;
        std::set<uint64_t> seen;
        for (uint32_t k = 0; ok && k < ng; ++k) {
            uint64_t e;
            std::memcpy(&e, q, 8);
            ok = e % 2 == 1 && e < 2 * N && seen.insert(e).second && check(q + 8, KW, LK);
            q += (1 + KW) * 8;
        }
        if (!ok) FAIL(HESPMV_E_INVALID, "key stream holds an invalid residue or Galois element");
    }
    DeviceGuard g(ctx->device);
    if (!ctx->sk) {
        ctx->sk = owned<uint64_t>(ctx, LK * N);
        ctx->pk = owned<uint64_t>(ctx, 2 * L * N);
        ctx->rlk = owned<uint64_t>(ctx, KW);
        if (!ctx->sk || !ctx->pk || !ctx->rlk) FAIL(HESPMV_E_NOMEM, "key allocation failed");
    }
    auto put = [&](uint64_t *dev, size_t n) {
        const bool ok = cudaMemcpy(dev, p, n * 8, cudaMemcpyHostToDevice) == cudaSuccess;
        p += n * 8;
        return ok;
    };
    bool ok = true;
    if (what == HESPMV_KEYS_ALL)
        ok = put(ctx->sk, LK * N);
    else
        ok = cudaMemset(ctx->sk, 0, LK * N * 8) == cudaSuccess;
    ok = ok && put(ctx->pk, 2 * L * N) && put(ctx->rlk, KW);
    for (uint32_t k = 0; ok && k < ng; ++k) {
        uint64_t e;
        std::memcpy(&e, p, 8);
        p += 8;
        uint64_t *key = ctx->gk.count((uint32_t)e) ? ctx->gk[(uint32_t)e] : owned<uint64_t>(ctx, KW);
        if (!key) FAIL(HESPMV_E_NOMEM, "key allocation failed");
        ctx->gk[(uint32_t)e] = key;
        ok = put(key, KW);
    }
    if (!ok) FAIL(HESPMV_E_CUDA, "key upload failed");
    ctx->have_keys = true;
    ctx->has_sk = what == HESPMV_KEYS_ALL;
    return HESPMV_OK;
}

static int encrypt_impl(hespmv_ctx *ctx, const hespmv_cssc *m, int32_t which, const int64_t *x,
                        const double *real, uint64_t seed, bool plain, hespmv_ctbatch **out) {
    if (!ctx || !m || !out) return HESPMV_E_INVALID;
    const bool ckks = ctx->h.scheme == HESPMV_SCHEME_CKKS;
    if (!ctx->have_keys && !plain) FAIL(HESPMV_E_INVALID, "keygen first");
    if (which != HESPMV_MATRIX && which != HESPMV_VECTOR) FAIL(HESPMV_E_INVALID, "bad operand kind");
    if (m->shape_only) FAIL(HESPMV_E_INVALID, "a shape-only CSSC has no values or column indices");
    if (ckks != (real != nullptr))
        FAIL(HESPMV_E_INVALID, ckks ? "a CKKS context encrypts real values (hespmv_encrypt_real)"
                                    : "a BGV context encrypts integers (hespmv_encrypt)");
    if (!ckks && which == HESPMV_VECTOR && !x && m->plan.cols > 0) FAIL(HESPMV_E_INVALID, "x is NULL");
    if (!ckks && which == HESPMV_MATRIX && !m->plan.has_values)
        FAIL(HESPMV_E_INVALID, "the CSSC was built without values");
    if (ckks && which == HESPMV_MATRIX && m->plan.nnz > 0 && !m->plan.has_src)
        FAIL(HESPMV_E_INVALID, "the CSSC does not map slots to CSR positions (deserialized plan)");
    NEED_DEVICE(ctx);
    DeviceGuard g(ctx->device);
    const Ctx c = view(ctx);
    const Plan &pl = m->plan;
    const size_t n = pl.chunks.size();
    const int64_t N = c.N, half = N / 2, L = c.L, LN = L * N;
    hespmv_ctbatch *b = nullptr;
    int rc = batch_new(ctx, n, &b);
    if (rc) return rc;
    const size_t G = std::max<size_t>(1, std::min<size_t>(n, 64));
    // per group: vals (half int64), E (N), mq, u, e0, e1 ([L][N] each), coef (N int64)
    const size_t words = G * (half + N + 4 * LN + N);
    uint64_t *ws = workspace(ctx, words * 8);
    if (!ws) {
        hespmv_ctbatch_free(b);
        FAIL(HESPMV_E_NOMEM, "workspace allocation failed");
    }
    int64_t *dvals = (int64_t *)ws;
    uint64_t *E = ws + G * half, *mq = E + G * N, *u = mq + G * LN;
    int64_t *coef = (int64_t *)(u + 3 * G * LN);
    std::vector<int64_t> host(G * (ckks ? N : half));
    std::vector<double> zs(ckks ? half : 0);
    CkksCodec *codec = ckks ? get_codec(ctx) : nullptr;
    for (size_t k0 = 0; k0 < n; k0 += G) {
        const size_t gn = std::min(G, n - k0);
        // u, e0, e1 back to back at this group's size: one transform of 3*gn items
        uint64_t *e0 = u + gn * LN, *e1 = e0 + gn * LN;
        std::fill(host.begin(), host.end(), 0);
        for (size_t k = 0; k < gn; ++k) {
            const Chunk &ch = pl.chunks[k0 + k];
            const int64_t cnt = (int64_t)ch.h * ch.c;
            if (ckks) {  // slot values, then the chunk's N coefficients
                for (int64_t s = 0; s < cnt; ++s) {
                    const int64_t at = which == HESPMV_MATRIX ? pl.slot_src[ch.slot0 + s]
                                                              : pl.slot_ci[ch.slot0 + s];
                    zs[s] = at >= 0 ? real[at] : 0.0;
                }
                const std::string e = ckks_encode(*codec, zs.data(), cnt, ctx->h.scale_bits, &host[k * N]);
                if (!e.empty()) {
                    hespmv_ctbatch_free(b);
                    FAIL(HESPMV_E_RANGE, "CKKS encoding: " + e);
                }
                continue;
            }
            for (int64_t s = 0; s < cnt; ++s) {
                if (which == HESPMV_MATRIX) {
                    host[k * half + s] = pl.slot_vals[ch.slot0 + s];
                } else {
                    const int32_t ci = pl.slot_ci[ch.slot0 + s];
                    host[k * half + s] = ci >= 0 ? x[ci] : 0;
                }
            }
        }
        const uint64_t sbase = kEncBase + 4 * (uint64_t)k0;
        bool ok;
        if (ckks) {  // coefficients (in E's words) -> residues over Q
            ok = cudaMemcpy(E, host.data(), gn * N * 8, cudaMemcpyHostToDevice) == cudaSuccess;
            ok = ok && !op_signed_to_limbs(c, (const int64_t *)E, mq, 0, (int)L, gn, 0);
        } else {
            ok = cudaMemcpy(dvals, host.data(), gn * half * 8, cudaMemcpyHostToDevice) == cudaSuccess;
            ok = ok && !op_scatter_slots(c, dvals, half, E, gn, 0);
            ok = ok && !launch_ntt(c, E, c.L + c.K, 1, (int)gn, N, true, 0);
            // BFV puts the message at Delta = floor(Q/t); plaintexts that only
            // multiply (the plain matrix) keep the centred lift
            if (ctx->h.scheme == HESPMV_SCHEME_BFV && !plain)
                ok = ok && !op_bfv_delta(c, E, mq, gn, 0);
            else
                ok = ok && !op_lift(c, E, mq, gn, 0);
        }
        ok = ok && !launch_ntt(c, mq, 0, (int)L, (int)gn, LN, false, 0);
        if (plain) {  // trivial ciphertexts (m, 0): the plaintext itself
            uint64_t *dst = b->data + k0 * 2 * LN;
            for (size_t k = 0; ok && k < gn; ++k) {
                ok = cudaMemcpyAsync(dst + k * 2 * LN, mq + k * LN, LN * 8, cudaMemcpyDeviceToDevice, 0) == cudaSuccess &&
                     cudaMemsetAsync(dst + k * 2 * LN + LN, 0, LN * 8, 0) == cudaSuccess;
            }
            ok = ok && cudaDeviceSynchronize() == cudaSuccess;
            if (!ok) {
                hespmv_ctbatch_free(b);
                FAIL(HESPMV_E_CUDA, "plain encoding failed");
            }
            continue;
        }
        ok = ok && !op_sample_signed(c, seed, sbase + 1, 4, kTernary, coef, gn, 0);
        ok = ok && !op_signed_to_limbs(c, coef, u, 0, (int)L, gn, 0);
        ok = ok && !op_sample_signed(c, seed, sbase + 2, 4, kCbd21, coef, gn, 0);
        ok = ok && !op_signed_to_limbs(c, coef, e0, 0, (int)L, gn, 0);
        ok = ok && !op_sample_signed(c, seed, sbase + 3, 4, kCbd21, coef, gn, 0);
        ok = ok && !op_signed_to_limbs(c, coef, e1, 0, (int)L, gn, 0);
        ok = ok && !launch_ntt(c, u, 0, (int)L, (int)(3 * gn), LN, false, 0);
        ok = ok && !op_enc_combine(c, u, e0, e1, mq, ctx->pk, b->data + k0 * 2 * LN, gn, 0);
        ok = ok && cudaDeviceSynchronize() == cudaSuccess;
        if (!ok) {
            hespmv_ctbatch_free(b);
            FAIL(HESPMV_E_CUDA, std::string("encrypt: ") + cudaGetErrorString(cudaGetLastError()));
        }
    }
    *out = b;
    return HESPMV_OK;
}

int hespmv_encrypt(hespmv_ctx *ctx, const hespmv_cssc *m, int32_t which, const int64_t *x,
                   uint64_t seed, hespmv_ctbatch **out) {
    return encrypt_impl(ctx, m, which, x, nullptr, seed, false, out);
}

int hespmv_encode_matrix_plain(hespmv_ctx *ctx, const hespmv_cssc *m, hespmv_ctbatch **out) {
    return encrypt_impl(ctx, m, HESPMV_MATRIX, nullptr, nullptr, 0, true, out);
}

int hespmv_encrypt_real(hespmv_ctx *ctx, const hespmv_cssc *m, int32_t which, const double *values,
                        uint64_t seed, hespmv_ctbatch **out) {
    if (ctx && m && !values && (which == HESPMV_VECTOR ? m->plan.cols : m->plan.nnz) > 0)
        FAIL(HESPMV_E_INVALID, "values is NULL");
    static const double none = 0.0;
    return encrypt_impl(ctx, m, which, nullptr, values ? values : &none, seed, false, out);
}

int hespmv_encode_matrix_plain_real(hespmv_ctx *ctx, const hespmv_cssc *m, const double *vals,
                                    hespmv_ctbatch **out) {
    if (ctx && m && !vals && m->plan.nnz > 0) FAIL(HESPMV_E_INVALID, "vals is NULL");
    static const double none = 0.0;
    return encrypt_impl(ctx, m, HESPMV_MATRIX, nullptr, vals ? vals : &none, 0, true, out);
}

int hespmv_spmv(hespmv_ctx *ctx, const hespmv_cssc *m, const hespmv_ctbatch *A,
                const hespmv_ctbatch *X, hespmv_ctbatch **y, void *stream) {
    return hespmv_spmv_batched(ctx, 1, &m, &A, &X, y, stream);
}

int hespmv_spmv_batched(hespmv_ctx *ctx, size_t n, const hespmv_cssc *const *m,
                        const hespmv_ctbatch *const *A, const hespmv_ctbatch *const *X,
                        hespmv_ctbatch **y, void *stream) {
    if (!ctx || (n && (!m || !A || !X || !y))) return HESPMV_E_INVALID;
    if (!ctx->have_keys) FAIL(HESPMV_E_INVALID, "keygen first");
    NEED_DEVICE(ctx);
    DeviceGuard g(ctx->device);
    std::vector<const uint64_t *> a(n), x(n);
    std::vector<uint64_t *> out(n);
    for (size_t i = 0; i < n; ++i) {
        if (!m[i] || !A[i] || !X[i]) FAIL(HESPMV_E_INVALID, "null handle");
        const size_t nc = m[i]->plan.chunks.size(), np = m[i]->plan.parts.size();
        if (A[i]->n < nc || X[i]->n < nc) FAIL(HESPMV_E_INVALID, "operand batches are smaller than the chunk count");
        if (y[i] == nullptr) {
            int rc = batch_new(ctx, np, &y[i]);
            if (rc) return rc;
        } else if (y[i]->n < np) {
            FAIL(HESPMV_E_INVALID, "result batch is smaller than the partition count");
        }
        a[i] = A[i]->data;
        x[i] = X[i]->data;
        out[i] = y[i]->data;
    }
    return spmv_core(ctx, n, m, a.data(), x.data(), out.data(), (cudaStream_t)stream);
}

int hespmv_spmv_ptmatrix(hespmv_ctx *ctx, const hespmv_cssc *m, const hespmv_ctbatch *A,
                         const hespmv_ctbatch *X, hespmv_ctbatch **y, void *stream) {
    if (!ctx || !m || !A || !X || !y) return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    if (!ctx->have_keys) FAIL(HESPMV_E_INVALID, "keygen first");
    DeviceGuard g(ctx->device);
    const size_t nc = m->plan.chunks.size(), np = m->plan.parts.size();
    if (A->n < nc || X->n < nc) FAIL(HESPMV_E_INVALID, "operand batches are smaller than the chunk count");
    if (*y == nullptr) {
        int rc = batch_new(ctx, np, y);
        if (rc) return rc;
    } else if ((*y)->n < np) {
        FAIL(HESPMV_E_INVALID, "result batch is smaller than the partition count");
    }
    const uint64_t *a = A->data, *x = X->data;
    uint64_t *out = (*y)->data;
    return spmv_core(ctx, 1, &m, &a, &x, &out, (cudaStream_t)stream, true);
}

int hespmv_spmv_host(hespmv_ctx *ctx, const hespmv_cssc *m, const uint64_t *A_host,
                     const uint64_t *X_host, uint64_t *y_host, void *stream) {
    if (!ctx || !m || !A_host || !X_host || !y_host) return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    DeviceGuard g(ctx->device);
    const size_t nc = m->plan.chunks.size(), np = m->plan.parts.size();
    const size_t ct_bytes = 2 * (size_t)ctx->h.L * ctx->h.N * 8;
    cudaStream_t st = (cudaStream_t)stream;
    // device staging owned by the context, grown on demand
    const size_t need = (2 * nc + np) * ct_bytes;
    if (ctx->io_bytes < need) {
        cudaDeviceSynchronize();
        dev_free(ctx, ctx->io);
        ctx->io = dev_alloc(ctx, need);
        ctx->io_bytes = ctx->io ? need : 0;
    }
    uint64_t *io = (uint64_t *)ctx->io;
    if (!io) FAIL(HESPMV_E_NOMEM, "staging allocation failed");
    uint64_t *dA = io, *dX = io + nc * ct_bytes / 8, *dY = dX + nc * ct_bytes / 8;
    // uploads overlap the HE-Mult: groups of chunks (hespmv_set_upload_groups),
    // each key switch waiting only for its own chunks, consecutive groups on
    // two streams
    const uint64_t *pa = dA, *px = dX;
    uint64_t *py = dY;
    const std::vector<size_t> gsz = upload_group_sizes(ctx, nc);
    int rc = spmv_core(ctx, 1, &m, &pa, &px, &py, st, false, A_host, X_host, &gsz);
    if (!rc && (cudaMemcpyAsync(y_host, dY, np * ct_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)) {
        rc = HESPMV_E_CUDA;
        ctx->err = "download failed";
    }
    cudaStreamSynchronize(st);
    return rc;
}

int hespmv_ct_packed_words(const hespmv_ctx *ctx, size_t *words, int32_t *bits) {
    if (!ctx) return HESPMV_E_INVALID;
    if (words) *words = packed_ct_words(ctx->h);
    if (bits) *bits = ctx->h.pack_bits;
    return HESPMV_OK;
}

int hespmv_ct_pack(const hespmv_ctx *ctx, const uint64_t *cts, size_t n_ct, uint64_t *packed) {
    if (!ctx || (n_ct && (!cts || !packed))) return HESPMV_E_INVALID;
    const HostTables &h = ctx->h;
    const int W = h.pack_bits, L = h.L, N = h.N;
    const size_t LW = packed_limb_words(h);
    for (size_t limb = 0; limb < n_ct * 2 * L; ++limb) {
        const uint64_t q = h.q[limb % L], *src = cts + limb * N;
        uint64_t *dst = packed + limb * LW;
        std::fill(dst, dst + LW, 0);
        for (int k = 0; k < N; ++k) {
            const uint64_t v = src[k];
            if (v >= q) return HESPMV_E_INVALID;
            const uint64_t bit = (uint64_t)k * W;
            const int sh = (int)(bit & 63);
            dst[bit >> 6] |= v << sh;
            if (sh + W > 64) dst[(bit >> 6) + 1] |= v >> (64 - sh);
        }
    }
    return HESPMV_OK;
}

int hespmv_ct_unpack(const hespmv_ctx *ctx, const uint64_t *packed, size_t n_ct, uint64_t *cts) {
    if (!ctx || (n_ct && (!cts || !packed))) return HESPMV_E_INVALID;
    const HostTables &h = ctx->h;
    const int W = h.pack_bits, L = h.L, N = h.N;
    const size_t LW = packed_limb_words(h);
    const uint64_t mask = W == 64 ? ~0ull : (1ull << W) - 1;
    const uint64_t used = (uint64_t)N * W - 64 * (LW - 1);  // bits of the last word in use
    for (size_t limb = 0; limb < n_ct * 2 * L; ++limb) {
        const uint64_t q = h.q[limb % L], *src = packed + limb * LW;
        uint64_t *dst = cts + limb * N;
        if (used < 64 && (src[LW - 1] >> used)) return HESPMV_E_INVALID;
        for (int k = 0; k < N; ++k) {
            const uint64_t bit = (uint64_t)k * W;
            const int sh = (int)(bit & 63);
            uint64_t v = src[bit >> 6] >> sh;
            if (sh + W > 64) v |= src[(bit >> 6) + 1] << (64 - sh);
            v &= mask;
            if (v >= q) return HESPMV_E_INVALID;
            dst[k] = v;
        }
    }
    return HESPMV_OK;
}

int hespmv_spmv_host_packed(hespmv_ctx *ctx, const hespmv_cssc *m, const uint64_t *A_packed,
                            const uint64_t *X_packed, uint64_t *y_packed, void *stream) {
    if (!ctx || !m || !A_packed || !X_packed || !y_packed) return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    DeviceGuard g(ctx->device);
    const size_t nc = m->plan.chunks.size(), np = m->plan.parts.size();
    const size_t CT = 2 * (size_t)ctx->h.L * ctx->h.N, PW = packed_ct_words(ctx->h);
    cudaStream_t st = (cudaStream_t)stream;
    // device staging owned by the context, grown on demand: unpacked A, X, y,
    // then packed A, X, y
    const size_t need = (2 * nc + np) * (CT + PW) * 8;
    if (ctx->io_bytes < need) {
        cudaDeviceSynchronize();
        dev_free(ctx, ctx->io);
        ctx->io = dev_alloc(ctx, need);
        ctx->io_bytes = ctx->io ? need : 0;
    }
    uint64_t *io = (uint64_t *)ctx->io;
    if (!io) FAIL(HESPMV_E_NOMEM, "staging allocation failed");
    if (!ctx->err_host && cudaHostAlloc((void **)&ctx->err_host, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
        ctx->err_host = nullptr;
        FAIL(HESPMV_E_NOMEM, "page-locked status word allocation failed");
    }
    uint64_t *dA = io, *dX = dA + nc * CT, *dY = dX + nc * CT;
    uint64_t *pA = dY + np * CT, *pX = pA + nc * PW, *pY = pX + nc * PW;
    const uint64_t *a = dA, *x = dX;
    uint64_t *y = dY;
    const Ctx c = view(ctx);
    *ctx->err_host = 0;
    const std::vector<size_t> gsz = upload_group_sizes(ctx, nc);
    int rc = spmv_core(ctx, 1, &m, &a, &x, &y, st, false, A_packed, X_packed, &gsz, pA, pX);
    if (!rc && (op_ct_pack(c, dY, pY, np, st) != cudaSuccess ||
                cudaMemcpyAsync(y_packed, pY, np * PW * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaMemcpyAsync(ctx->err_host, ctx->d.err, sizeof(int), cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)) {
        rc = HESPMV_E_CUDA;
        ctx->err = "packed evaluation failed";
    }
    cudaStreamSynchronize(st);
    if (!rc && *ctx->err_host) {
        const int v = *ctx->err_host;
        if (cudaMemset(ctx->d.err, 0, sizeof(int)) != cudaSuccess) FAIL(HESPMV_E_CUDA, "status reset failed");
        return status_of_code(ctx, v);
    }
    return rc;
}

int hespmv_spmv_host_packed_async(hespmv_ctx *ctx, const hespmv_cssc *m, const uint64_t *A_packed,
                                  const uint64_t *X_packed, uint64_t *y_packed, void *stream) {
    if (!ctx || !m || !A_packed || !X_packed || !y_packed) return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    DeviceGuard g(ctx->device);
    const size_t nc = m->plan.chunks.size(), np = m->plan.parts.size();
    const size_t CT = 2 * (size_t)ctx->h.L * ctx->h.N, PW = packed_ct_words(ctx->h);
    cudaStream_t st = (cudaStream_t)stream;
    const int s = ctx->aslot;
    // staging of this slot: unpacked A, X, y, then packed A, X, y
    const size_t need = (2 * nc + np) * (CT + PW) * 8;
    if (ctx->aio_bytes[s] < need) {
        cudaDeviceSynchronize();
        dev_free(ctx, ctx->aio[s]);
        ctx->aio[s] = dev_alloc(ctx, need);
        ctx->aio_bytes[s] = ctx->aio[s] ? need : 0;
        ctx->slot_used[s] = false;
    }
    uint64_t *io = (uint64_t *)ctx->aio[s];
    if (!io) FAIL(HESPMV_E_NOMEM, "staging allocation failed");
    if (!ctx->slot_free[s]) CK(cudaEventCreateWithFlags(&ctx->slot_free[s], cudaEventDisableTiming));
    uint64_t *dA = io, *dX = dA + nc * CT, *dY = dX + nc * CT;
    uint64_t *pA = dY + np * CT, *pX = pA + nc * PW, *pY = pX + nc * PW;
    const uint64_t *a = dA, *x = dX;
    uint64_t *y = dY;
    const Ctx c = view(ctx);
    const std::vector<size_t> gsz = upload_group_sizes(ctx, nc, true);
    int rc = spmv_core(ctx, 1, &m, &a, &x, &y, st, false, A_packed, X_packed, &gsz, pA, pX, true,
                       ctx->slot_used[s] ? ctx->slot_free[s] : nullptr);
    if (rc) return rc;
    CK(op_ct_pack(c, dY, pY, np, st));
    CK(cudaMemcpyAsync(y_packed, pY, np * PW * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(ctx->slot_free[s], st));
    ctx->slot_used[s] = true;
    ctx->aslot = (s + 1) % hespmv_ctx::kSlots;
    return HESPMV_OK;
}

int hespmv_decrypt_slots(hespmv_ctx *ctx, const hespmv_ctbatch *b, size_t index,
                         uint64_t *slots_out) {
    if (!ctx || !b || !slots_out || index >= b->n) return HESPMV_E_INVALID;
    if (ctx->h.scheme == HESPMV_SCHEME_CKKS) FAIL(HESPMV_E_INVALID, "CKKS: hespmv_decrypt_real_slots");
    if (!ctx->have_keys) FAIL(HESPMV_E_INVALID, "keygen first");
    if (!ctx->has_sk) FAIL(HESPMV_E_INVALID, "this context holds evaluation keys only (no secret key)");
    NEED_DEVICE(ctx);
    DeviceGuard g(ctx->device);
    {  // results that a timed-out device wait left incomplete are not decrypted
        const int rc = hespmv_device_status(ctx, nullptr);
        if (rc) return rc;
    }
    const Ctx c = view(ctx);
    const int64_t N = c.N, LN = (int64_t)c.L * N;
    uint64_t *ws = workspace(ctx, (LN + 2 * N) * 8);
    if (!ws) FAIL(HESPMV_E_NOMEM, "workspace allocation failed");
    uint64_t *x = ws, *msg = x + LN, *slots = msg + N;
    CK(op_dec_phase(c, b->data + index * 2 * LN, ctx->sk, x, 0));
    CK(launch_ntt(c, x, 0, c.L, 1, LN, true, 0));
    if (ctx->h.scheme == HESPMV_SCHEME_BFV) {
        // m = round(t [x]_Q / Q) mod t, exactly, on the host (client side)
        std::vector<uint64_t> res(LN), m(N);
        CK(cudaMemcpy(res.data(), x, LN * 8, cudaMemcpyDeviceToHost));
        bfv_decrypt_coef(ctx->h, res.data(), m.data());
        CK(cudaMemcpy(msg, m.data(), N * 8, cudaMemcpyHostToDevice));
    } else {
        CK(op_crt_to_t(c, x, msg, 0));
    }
    CK(launch_ntt(c, msg, c.L + c.K, 1, 1, N, false, 0));
    CK(op_gather_slots(c, msg, slots, 0));
    CK(cudaMemcpy(slots_out, slots, N * 8, cudaMemcpyDeviceToHost));
    return HESPMV_OK;
}

int hespmv_decrypt_real_slots(hespmv_ctx *ctx, const hespmv_ctbatch *b, size_t index,
                              int32_t scale_bits, double *slots_out) {
    if (!ctx || !b || !slots_out || index >= b->n || scale_bits < 0 || scale_bits > 1000)
        return HESPMV_E_INVALID;
    if (ctx->h.scheme != HESPMV_SCHEME_CKKS) FAIL(HESPMV_E_INVALID, "not a CKKS context");
    if (!ctx->have_keys) FAIL(HESPMV_E_INVALID, "keygen first");
    if (!ctx->has_sk) FAIL(HESPMV_E_INVALID, "this context holds evaluation keys only (no secret key)");
    NEED_DEVICE(ctx);
    DeviceGuard g(ctx->device);
    {  // results that a timed-out device wait left incomplete are not decrypted
        const int rc = hespmv_device_status(ctx, nullptr);
        if (rc) return rc;
    }
    const Ctx c = view(ctx);
    const int64_t N = c.N, LN = (int64_t)c.L * N;
    uint64_t *x = workspace(ctx, LN * 8);
    if (!x) FAIL(HESPMV_E_NOMEM, "workspace allocation failed");
    CK(op_dec_phase(c, b->data + index * 2 * LN, ctx->sk, x, 0));
    CK(launch_ntt(c, x, 0, c.L, 1, LN, true, 0));
    std::vector<uint64_t> res(LN);
    CK(cudaMemcpy(res.data(), x, LN * 8, cudaMemcpyDeviceToHost));
    if (!ctx->crt) ctx->crt = crt_real(ctx->h.q.data(), c.L);
    std::vector<double> coef(N);
    crt_to_double(*ctx->crt, res.data(), (int)N, coef.data());
    ckks_decode(*get_codec(ctx), coef.data(), N / 2, std::ldexp(1.0, -scale_bits), slots_out);
    return HESPMV_OK;
}

int hespmv_decrypt_real(hespmv_ctx *ctx, const hespmv_cssc *m, const hespmv_ctbatch *y,
                        double *out_rows) {
    if (!ctx || !m || !y || (!out_rows && m->plan.rows)) return HESPMV_E_INVALID;
    if (y->n < m->plan.parts.size()) FAIL(HESPMV_E_INVALID, "result batch too small");
    if (m->shape_only) FAIL(HESPMV_E_INVALID, "a shape-only CSSC has no row map");
    const int total = 2 * ctx->h.scale_bits + ctx->h.mask_scale_bits;
    std::vector<double> slots(ctx->h.N / 2);
    for (size_t p = 0; p < m->plan.parts.size(); ++p) {
        int rc = hespmv_decrypt_real_slots(ctx, y, p, total, slots.data());
        if (rc) return rc;
        const Partition &P = m->plan.parts[p];
        for (int32_t idx = 0; idx < P.rows; ++idx) out_rows[P.row0 + P.rm[idx]] = slots[idx];
    }
    return HESPMV_OK;
}

int hespmv_rescale(hespmv_ctx *ctx, const uint64_t *ct, uint64_t *out, size_t n, void *stream) {
    if (!ctx || !ct || !out) return HESPMV_E_INVALID;
    if (ctx->h.scheme != HESPMV_SCHEME_CKKS) FAIL(HESPMV_E_INVALID, "rescaling is defined here for CKKS contexts");
    if (ctx->h.L < 2) FAIL(HESPMV_E_INVALID, "a rescaled ciphertext needs at least one prime left");
    NEED_DEVICE(ctx);
    if (!aligned16({ct, out})) FAIL(HESPMV_E_INVALID, "device buffers must be 16-byte aligned");
    if (n == 0) return HESPMV_OK;
    DeviceGuard g(ctx->device);
    const Ctx c = view(ctx);
    const int L = c.L, nl1 = L - 1;
    const int64_t N = c.N;
    const uint64_t ql = ctx->h.q[L - 1];
    if (!ctx->rescale_inv) {  // q_{L-1}^-1 mod q_i, Shoup pairs
        std::vector<uint64_t> t(2 * nl1);
        for (int i = 0; i < nl1; ++i) {
            const uint64_t qi = ctx->h.q[i];
            uint64_t r = 1, b = ql % qi;
            for (uint64_t e = qi - 2; e; e >>= 1) {
                if (e & 1) r = (uint64_t)((unsigned __int128)r * b % qi);
                b = (uint64_t)((unsigned __int128)b * b % qi);
            }
            t[2 * i] = r;
            t[2 * i + 1] = (uint64_t)(((unsigned __int128)r << 64) / qi);
        }
        if (!upload(ctx, ctx->rescale_inv, t)) FAIL(HESPMV_E_NOMEM, "rescale constants upload failed");
    }
    const size_t nc = 2 * n;  // components
    uint64_t *x = workspace(ctx, (nc * N + nc * nl1 * N) * 8);
    if (!x) FAIL(HESPMV_E_NOMEM, "workspace allocation failed");
    uint64_t *y = x + nc * N;
    cudaStream_t st = (cudaStream_t)stream;
    // the last limb of every component, to coefficient form mod q_{L-1}
    CK(op_copy_strided(c, ct + (int64_t)nl1 * N, (int64_t)L * N, x, N, N, nc, st));
    CK(launch_ntt(c, x, L - 1, 1, (int)nc, N, true, st));
    // centred, lifted to q_0 .. q_{L-2} and back to the NTT domain
    CK(op_rescale_lift(c, x, y, nc, nl1, ql, st));
    CK(launch_ntt(c, y, 0, nl1, (int)nc, (int64_t)nl1 * N, false, st));
    CK(op_rescale_final(c, ct, y, out, nc, nl1, ctx->rescale_inv, st));
    return HESPMV_OK;
}

int hespmv_decrypt_real_level(hespmv_ctx *ctx, const uint64_t *ct, int32_t limbs, double scale,
                              double *slots_out) {
    if (!ctx || !ct || !slots_out || !(scale > 0)) return HESPMV_E_INVALID;
    if (ctx->h.scheme != HESPMV_SCHEME_CKKS) FAIL(HESPMV_E_INVALID, "not a CKKS context");
    if (limbs < 1 || limbs > ctx->h.L) FAIL(HESPMV_E_INVALID, "limbs must be in [1, L]");
    if (!ctx->have_keys || !ctx->has_sk) FAIL(HESPMV_E_INVALID, "the secret key is needed");
    NEED_DEVICE(ctx);
    if (!aligned16(ct)) FAIL(HESPMV_E_INVALID, "device buffers must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    Ctx c = view(ctx);
    c.L = limbs;  // the first `limbs` primes (and secret-key limbs)
    const int64_t N = c.N, LN = (int64_t)limbs * N;
    uint64_t *x = workspace(ctx, LN * 8);
    if (!x) FAIL(HESPMV_E_NOMEM, "workspace allocation failed");
    CK(op_dec_phase(c, ct, ctx->sk, x, 0));
    CK(launch_ntt(c, x, 0, limbs, 1, LN, true, 0));
    std::vector<uint64_t> res(LN);
    CK(cudaMemcpy(res.data(), x, LN * 8, cudaMemcpyDeviceToHost));
    CrtReal *crt = crt_real(ctx->h.q.data(), limbs);
    std::vector<double> coef(N);
    crt_to_double(*crt, res.data(), (int)N, coef.data());
    crt_real_free(crt);
    ckks_decode(*get_codec(ctx), coef.data(), N / 2, 1.0 / scale, slots_out);
    return HESPMV_OK;
}

int hespmv_ckks_encode(hespmv_ctx *ctx, const double *z, size_t n, int32_t scale_bits, int64_t *coef) {
    if (!ctx || (!z && n) || !coef || ctx->h.q.empty()) return HESPMV_E_INVALID;
    if (n > (size_t)ctx->h.N / 2) FAIL(HESPMV_E_INVALID, "more values than N/2 slots");
    if (scale_bits < 0 || scale_bits > 62) FAIL(HESPMV_E_INVALID, "scale_bits must be in [0, 62]");
    const std::string e = ckks_encode(*get_codec(ctx), z, n, scale_bits, coef);
    if (!e.empty()) FAIL(HESPMV_E_RANGE, e);
    return HESPMV_OK;
}

int hespmv_decrypt(hespmv_ctx *ctx, const hespmv_cssc *m, const hespmv_ctbatch *y,
                   int64_t *out_rows) {
    if (!ctx || !m || !y || (!out_rows && m->plan.rows)) return HESPMV_E_INVALID;
    if (ctx->h.scheme == HESPMV_SCHEME_CKKS) FAIL(HESPMV_E_INVALID, "CKKS results: hespmv_decrypt_real");
    if (y->n < m->plan.parts.size()) FAIL(HESPMV_E_INVALID, "result batch too small");
    if (m->shape_only) FAIL(HESPMV_E_INVALID, "a shape-only CSSC has no row map");
    const uint64_t t = ctx->h.t;
    std::vector<uint64_t> slots(ctx->h.N);
    for (size_t p = 0; p < m->plan.parts.size(); ++p) {
        int rc = hespmv_decrypt_slots(ctx, y, p, slots.data());
        if (rc) return rc;
        const Partition &P = m->plan.parts[p];
        for (int32_t idx = 0; idx < P.rows; ++idx) {
            const uint64_t v = slots[idx];
            out_rows[P.row0 + P.rm[idx]] = (2 * v > t) ? (int64_t)v - (int64_t)t : (int64_t)v;
        }
    }
    return HESPMV_OK;
}

int hespmv_ntt_forward(hespmv_ctx *ctx, uint64_t *data, int32_t prime0, int32_t n_limbs,
                       int32_t n_items, void *stream) {
    if (!ctx || !data || prime0 < 0 || n_limbs < 1 || prime0 + n_limbs > ctx->h.L + ctx->h.K + 1)
        return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    if (!aligned16(data)) FAIL(HESPMV_E_INVALID, "device buffers must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    CK(launch_ntt(view(ctx), data, prime0, n_limbs, n_items, (int64_t)n_limbs * ctx->h.N, false,
                  (cudaStream_t)stream));
    return HESPMV_OK;
}

int hespmv_ntt_inverse(hespmv_ctx *ctx, uint64_t *data, int32_t prime0, int32_t n_limbs,
                       int32_t n_items, void *stream) {
    if (!ctx || !data || prime0 < 0 || n_limbs < 1 || prime0 + n_limbs > ctx->h.L + ctx->h.K + 1)
        return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    if (!aligned16(data)) FAIL(HESPMV_E_INVALID, "device buffers must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    CK(launch_ntt(view(ctx), data, prime0, n_limbs, n_items, (int64_t)n_limbs * ctx->h.N, true,
                  (cudaStream_t)stream));
    return HESPMV_OK;
}

int hespmv_he_add(hespmv_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t *out, size_t n,
                  void *stream) {
    if (!ctx || !a || !b || !out) return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    if (!aligned16({a, b, out})) FAIL(HESPMV_E_INVALID, "device buffers must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    CK(op_add(view(ctx), a, b, out, 2 * n, (cudaStream_t)stream));
    return HESPMV_OK;
}

int hespmv_he_tensor(hespmv_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t *d, size_t n,
                     void *stream) {
    if (!ctx || !a || !b || !d) return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    if (!aligned16({a, b, d})) FAIL(HESPMV_E_INVALID, "device buffers must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    const Ctx c = view(ctx);
    uint64_t *scr = nullptr;
    if (const size_t w = tensor_scratch_words(c, n)) {
        scr = workspace(ctx, w * 8);
        if (!scr) FAIL(HESPMV_E_NOMEM, "workspace allocation failed");
    }
    CK(tensor_n(c, a, b, d, n, scr, (cudaStream_t)stream));
    return HESPMV_OK;
}

int hespmv_he_relin(hespmv_ctx *ctx, const uint64_t *d, uint64_t *out, size_t n, void *stream) {
    if (!ctx || !d || !out) return HESPMV_E_INVALID;
    if (!ctx->have_keys) FAIL(HESPMV_E_INVALID, "keygen first");
    NEED_DEVICE(ctx);
    if (!aligned16({d, out})) FAIL(HESPMV_E_INVALID, "device buffers must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    const Ctx c = view(ctx);
    const int64_t LN = (int64_t)c.L * c.N;
    uint64_t *ws = workspace(ctx, ks_words(c, n) * 8);
    if (!ws) FAIL(HESPMV_E_NOMEM, "workspace allocation failed");
    CK(keyswitch_n(c, d + 2 * LN, 3 * LN, ctx->rlk, out, d, 3 * LN, LN, 3, n, ws,
                   (cudaStream_t)stream));
    return HESPMV_OK;
}

int hespmv_he_mult(hespmv_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t *out, size_t n,
                   void *stream) {
    if (!ctx || !a || !b || !out) return HESPMV_E_INVALID;
    if (!ctx->have_keys) FAIL(HESPMV_E_INVALID, "keygen first");
    NEED_DEVICE(ctx);
    if (!aligned16({a, b, out})) FAIL(HESPMV_E_INVALID, "device buffers must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    const Ctx c = view(ctx);
    const int64_t LN = (int64_t)c.L * c.N;
    uint64_t *ws = workspace(ctx, (n * 3 * LN + std::max(ks_words(c, n), tensor_scratch_words(c, n))) * 8);
    if (!ws) FAIL(HESPMV_E_NOMEM, "workspace allocation failed");
    cudaStream_t st = (cudaStream_t)stream;
    CK(tensor_n(c, a, b, ws, n, ws + n * 3 * LN, st));
    CK(keyswitch_n(c, ws + 2 * LN, 3 * LN, ctx->rlk, out, ws, 3 * LN, LN, 3, n, ws + n * 3 * LN, st));
    return HESPMV_OK;
}

int hespmv_he_rotate(hespmv_ctx *ctx, const uint64_t *ct, int32_t k, uint64_t *out, size_t n,
                     void *stream) {
    if (!ctx || !ct || !out || ct == out) return HESPMV_E_INVALID;
    if (!ctx->have_keys) FAIL(HESPMV_E_INVALID, "keygen first");
    NEED_DEVICE(ctx);
    if (!aligned16({ct, out})) FAIL(HESPMV_E_INVALID, "device buffers must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    const Ctx c = view(ctx);
    const int64_t CT = 2 * (int64_t)c.L * c.N;
    uint64_t *ws = workspace(ctx, (3 * n * CT + ks_words(c, n)) * 8);
    if (!ws) FAIL(HESPMV_E_NOMEM, "workspace allocation failed");
    return rotate_n(ctx, ct, k, out, n, ws, (cudaStream_t)stream);
}

int hespmv_he_cmult_mask(hespmv_ctx *ctx, const uint64_t *ct, int32_t r, uint64_t *out, size_t n,
                         void *stream) {
    if (!ctx || !ct || !out || r < 0) return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    if (!aligned16({ct, out})) FAIL(HESPMV_E_INVALID, "device buffers must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    const uint64_t *m = mask_plaintext(ctx, r, (cudaStream_t)stream);
    if (!m) FAIL(HESPMV_E_NOMEM, "mask creation failed");
    CK(op_cmult(view(ctx), ct, m, out, n, (cudaStream_t)stream));
    return HESPMV_OK;
}

int hespmv_keyswitch(hespmv_ctx *ctx, const uint64_t *d, uint32_t galois_elt, uint64_t *out,
                     size_t n, void *stream) {
    if (!ctx || !d || !out) return HESPMV_E_INVALID;
    if (!ctx->have_keys) FAIL(HESPMV_E_INVALID, "keygen first");
    NEED_DEVICE(ctx);
    if (!aligned16({d, out})) FAIL(HESPMV_E_INVALID, "device buffers must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    const uint64_t *key = ctx->rlk;
    if (galois_elt) {
        auto it = ctx->gk.find(galois_elt);
        if (it == ctx->gk.end()) FAIL(HESPMV_E_INVALID, "no Galois key for that element");
        key = it->second;
    }
    const Ctx c = view(ctx);
    const int64_t LN = (int64_t)c.L * c.N;
    uint64_t *ws = workspace(ctx, ks_words(c, n) * 8);
    if (!ws) FAIL(HESPMV_E_NOMEM, "workspace allocation failed");
    CK(keyswitch_n(c, d, LN, key, out, nullptr, 0, 0, 0, n, ws, (cudaStream_t)stream));
    return HESPMV_OK;
}

// ------------------------------------------------------------ autotuning
}  // extern "C"

namespace {

void drop_graphs(hespmv_ctx *ctx) {
    for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
    ctx->graphs.clear();
    drop_persist_plans(ctx);  // the device is idle (callers synchronise first)
}

struct TuneState {
    size_t G, GR;
    int split, rows_tma;
    int persistent = 0, blocks = 0;
    int streams = 1;
};

void apply_tuning(hespmv_ctx *ctx, const TuneState &s) {
    if (ctx->tune_G != s.G || ctx->tune_GR != s.GR || ctx->ks_split != s.split ||
        ctx->rows_tma != s.rows_tma || ctx->persistent != s.persistent || ctx->persist_blocks != s.blocks ||
        ctx->streams != s.streams)
        drop_graphs(ctx);
    ctx->tune_G = s.G;
    ctx->tune_GR = s.GR;
    ctx->ks_split = s.split;
    ctx->rows_tma = s.rows_tma;
    ctx->persistent = s.persistent;
    ctx->persist_blocks = s.blocks;
    ctx->streams = s.streams;
}

}  // namespace

extern "C" {

int hespmv_set_tuning(hespmv_ctx *ctx, const hespmv_tuning *t) {
    if (!ctx || !t) return HESPMV_E_INVALID;
    if (t->mult_batch < 0 || t->rot_batch < 0 || t->mult_batch > 4096 || t->rot_batch > 4096)
        FAIL(HESPMV_E_INVALID, "batch sizes must be in [0, 4096]");
    if (t->ntt_split < 0 || t->ntt_split >= ks_split_variants(view(ctx)))
        FAIL(HESPMV_E_INVALID, "no such NTT split for this ring");
    if (t->rows_tma < 0 || t->rows_tma > (ks_fused_supported(view(ctx)) ? 1 : 0))
        FAIL(HESPMV_E_INVALID, "no such row-pass form for this ring");
    if (t->persistent < 0 || t->persistent > 1 || (t->persistent && !persist_supported(view(ctx))))
        FAIL(HESPMV_E_INVALID, "no persistent evaluation for this ring");
    if (t->persist_blocks < 0) FAIL(HESPMV_E_INVALID, "persist_blocks must be >= 0");
    if (t->streams < 0 || t->streams > 2) FAIL(HESPMV_E_INVALID, "streams must be 0, 1 or 2");
    const TuneState ts{(size_t)t->mult_batch, (size_t)t->rot_batch, t->ntt_split, t->rows_tma, t->persistent,
                       t->persist_blocks, t->streams == 2 ? 2 : 1};
    if (ctx->device >= 0) {
        DeviceGuard g(ctx->device);
        cudaDeviceSynchronize();
        apply_tuning(ctx, ts);
    } else {
        apply_tuning(ctx, ts);
    }
    return HESPMV_OK;
}

int hespmv_set_upload_groups(hespmv_ctx *ctx, int32_t groups) {
    if (!ctx || groups < 0 || groups > 64) return HESPMV_E_INVALID;
    ctx->upload_groups = groups;
    return HESPMV_OK;
}

int hespmv_get_upload_groups(const hespmv_ctx *ctx, int32_t *groups) {
    if (!ctx || !groups) return HESPMV_E_INVALID;
    *groups = ctx->upload_groups > 0 ? ctx->upload_groups : 0;
    return HESPMV_OK;
}

int hespmv_get_tuning(const hespmv_ctx *ctx, hespmv_tuning *t) {
    if (!ctx || !t) return HESPMV_E_INVALID;
    *t = hespmv_tuning{};
    t->mult_batch = (int32_t)ctx->tune_G;
    t->rot_batch = (int32_t)ctx->tune_GR;
    t->ntt_split = ctx->ks_split;
    t->rows_tma = ctx->rows_tma;
    t->persistent = ctx->persistent;
    t->persist_blocks = ctx->persist_blocks;
    t->streams = ctx->streams;
    t->ms = 0;
    return HESPMV_OK;
}

int hespmv_autotune(hespmv_ctx *ctx, size_t n, const hespmv_cssc *const *m,
                    const hespmv_ctbatch *const *A, const hespmv_ctbatch *const *X, int32_t reps,
                    hespmv_tuning *best, hespmv_tuning *tried, size_t cap, size_t *n_tried) {
    if (!ctx || !n || !m || !A || !X || !best || reps < 1) return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    if (!ctx->have_keys) FAIL(HESPMV_E_INVALID, "keygen first");
    DeviceGuard g(ctx->device);
    const Ctx c = view(ctx);
    std::vector<const uint64_t *> a(n), x(n);
    std::vector<uint64_t *> out(n);
    std::vector<hespmv_ctbatch *> ys(n, nullptr);
    size_t total = 0, rot = 0;
    auto release = [&]() {
        for (hespmv_ctbatch *y : ys) hespmv_ctbatch_free(y);
    };
    for (size_t i = 0; i < n; ++i) {
        if (!m[i] || !A[i] || !X[i]) {
            release();
            FAIL(HESPMV_E_INVALID, "null handle");
        }
        const size_t nc = m[i]->plan.chunks.size();
        if (A[i]->n < nc || X[i]->n < nc) {
            release();
            FAIL(HESPMV_E_INVALID, "operand batches are smaller than the chunk count");
        }
        int rc = batch_new(ctx, m[i]->plan.parts.size(), &ys[i]);
        if (rc) {
            release();
            return rc;
        }
        a[i] = A[i]->data;
        x[i] = X[i]->data;
        out[i] = ys[i]->data;
        total += nc;
        for (const Chunk &ch : m[i]->plan.chunks) rot += ch.c > 1;
    }
    const TuneState orig{ctx->tune_G, ctx->tune_GR, ctx->ks_split, ctx->rows_tma};
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    bool ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    std::vector<hespmv_tuning> log;
    std::string err;
    int err_rc = HESPMV_OK;
    // time one setting; returns ms, or -1 when its workspace would not fit
    auto measure = [&](const TuneState &s) -> double {
        apply_tuning(ctx, s);
        SpmvPrep pp;
        spmv_sizes(c, total, rot, pp);
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        hespmv_tuning rec{};
        rec.mult_batch = (int32_t)pp.G;
        rec.rot_batch = (int32_t)pp.GR;
        rec.ntt_split = s.split;
        rec.rows_tma = s.rows_tma;
        rec.persistent = s.persistent;
        rec.persist_blocks = s.blocks;
        rec.streams = s.streams;
        if (s.streams == 2 && total > pp.G) pp.need_bytes += pp.mult_w * 8;  // the second stream's scratch
        if (s.streams == 2 && rot > pp.GR)
            pp.need_bytes = std::max(pp.need_bytes, (total * 2 * (size_t)c.L * c.N + 2 * pp.rot_w) * 8);
        if (s.persistent) {  // one launch: HE-Mult group G, concurrent totalSum chains
            const size_t Gp = persist_group(ctx, total);
            pp.need_bytes = persist_ws_words(c, total, rot, Gp) * 8;
            rec.mult_batch = (int32_t)Gp;
            rec.rot_batch = s.GR ? (int32_t)s.GR : kPersistStagger;
        }
        if (pp.need_bytes > ctx->ws_bytes && pp.need_bytes - ctx->ws_bytes > free_b / 10 * 9) {
            rec.ms = -1;
            log.push_back(rec);
            return -1;
        }
        int rc = spmv_core(ctx, n, m, a.data(), x.data(), out.data(), st);  // warm-up / capture
        if (rc == HESPMV_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = HESPMV_E_CUDA;
        if (rc == HESPMV_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = HESPMV_E_CUDA;
        for (int32_t r = 0; rc == HESPMV_OK && r < reps; ++r)
            rc = spmv_core(ctx, n, m, a.data(), x.data(), out.data(), st);
        float ms = 0;
        if (rc == HESPMV_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = HESPMV_E_CUDA;
        if (rc != HESPMV_OK) {
            err_rc = rc;
            err = ctx->err.empty() ? "evaluation failed while tuning" : ctx->err;
            return -2;
        }
        rec.ms = ms / reps;
        log.push_back(rec);
        return rec.ms;
    };
    TuneState cur{0, 0, 0, 0}, bestS = cur;
    double best_ms = ok ? measure(cur) : -2;
    if (best_ms < 0 && err_rc == HESPMV_OK && ok) {
        err_rc = HESPMV_E_NOMEM;
        err = "the default schedule does not fit in device memory";
    }
    if (!ok && err_rc == HESPMV_OK) {
        err_rc = HESPMV_E_CUDA;
        err = "stream/event creation failed";
    }
    auto consider = [&](const TuneState &s) {
        if (err_rc != HESPMV_OK) return;
        const double t = measure(s);
        if (t >= 0 && t < best_ms) {
            best_ms = t;
            bestS = s;
        }
    };
    // coordinate descent: NTT split, then the HE-Mult batch, then the rotation round width
    for (int v = 1; v < ks_split_variants(c); ++v) consider({bestS.G, bestS.GR, v, bestS.rows_tma});
    if (ks_fused_supported(c)) consider({bestS.G, bestS.GR, bestS.split, 1});
    {
        std::vector<size_t> gs;
        for (size_t v = 1; v < 128 && v < total; v *= 2) gs.push_back(v);
        gs.push_back(std::min<size_t>(total, 128));
        const TuneState base = bestS;
        for (size_t v : gs) consider({v, base.GR, base.split, base.rows_tma});
    }
    if (rot > 0) {
        std::vector<size_t> grs;
        for (size_t v = 4; v < 512 && v < rot; v *= 2) grs.push_back(v);
        grs.push_back(std::min<size_t>(rot, 512));
        const TuneState base = bestS;
        for (size_t v : grs) consider({base.G, v, base.split, base.rows_tma});
    }
    // two compute streams: the HE-Mult groups alternate between them (groups of
    // about a half and a quarter of the chunks, and the best group so far)
    if (total > 1) {
        const TuneState base = bestS;
        std::set<size_t> gd;
        for (size_t v : {(total + 1) / 2, (total + 3) / 4, base.G ? base.G : (size_t)32})
            if (v >= 1 && v < total) gd.insert(v);
        for (size_t v : gd) consider({v, base.GR, base.split, base.rows_tma, 0, 0, 2});
    }
    if (rot > 1) {  // rotation groups over two streams: about a half and a quarter of the rotating chunks
        const TuneState base = bestS;
        std::set<size_t> gr;
        for (size_t v : {(rot + 1) / 2, (rot + 3) / 4})
            if (v >= 1 && v < rot) gr.insert(v);
        for (size_t v : gr) consider({base.G, v, base.split, base.rows_tma, 0, 0, 2});
    }
    // the NTT split and the row-pass form again, under the best staged schedule
    if (ks_fused_supported(c)) {
        const TuneState base = bestS;
        for (int v = 0; v < ks_split_variants(c); ++v)
            for (int tma = 0; tma <= 1; ++tma)
                if (v != base.split || tma != base.rows_tma)
                    consider({base.G, base.GR, v, tma, 0, 0, base.streams});
    }
    // the persistent form: HE-Mult groups of 4, 16, 64 (capped), then the other NTT split
    if (persist_supported(c) && ctx->h.scheme != HESPMV_SCHEME_BFV) {
        const TuneState staged = bestS;
        std::set<size_t> pg;
        for (size_t v : {4, 16, 64}) pg.insert(std::max<size_t>(1, std::min(v, total)));
        for (size_t v : pg) consider({v, 0, staged.split, 0, 1, 0});
        if (bestS.persistent)
            for (int v = 0; v < ks_split_variants(c); ++v)
                if (v != bestS.split) consider({bestS.G, 0, v, 0, 1, 0});
    }
    if (st) cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    release();
    if (err_rc != HESPMV_OK) {
        apply_tuning(ctx, orig);
        FAIL(err_rc, err);
    }
    apply_tuning(ctx, bestS);
    best->mult_batch = (int32_t)bestS.G;
    best->rot_batch = (int32_t)bestS.GR;
    best->ntt_split = bestS.split;
    best->rows_tma = bestS.rows_tma;
    best->persistent = bestS.persistent;
    best->persist_blocks = bestS.blocks;
    best->streams = bestS.streams;
    if (bestS.persistent) {
        best->mult_batch = (int32_t)persist_group(ctx, total);
        best->rot_batch = bestS.GR ? (int32_t)bestS.GR : kPersistStagger;
    }
    best->ms = best_ms;
    if (n_tried) *n_tried = log.size();
    for (size_t i = 0; tried && i < log.size() && i < cap; ++i) tried[i] = log[i];
    return HESPMV_OK;
}

int hespmv_device_status(hespmv_ctx *ctx, int32_t *code) {
    if (!ctx) return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    DeviceGuard g(ctx->device);
    int v = 0;
    CK(cudaMemcpy(&v, ctx->d.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (code) *code = v;
    if (v) CK(cudaMemset(ctx->d.err, 0, sizeof(int)));
    return status_of_code(ctx, v);
}

int hespmv_selftest_wait_timeout(hespmv_ctx *ctx, int32_t *code) {
    if (!ctx) return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    DeviceGuard g(ctx->device);
    CK(op_wait_probe(view(ctx), 0));
    CK(cudaDeviceSynchronize());
    return hespmv_device_status(ctx, code);
}

int hespmv_selftest_persist_timeout(hespmv_ctx *ctx, int32_t *code) {
    if (!ctx) return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    DeviceGuard g(ctx->device);
    const Ctx c = view(ctx);
    if (!persist_supported(c)) FAIL(HESPMV_E_UNSUPPORTED, "no persistent evaluation for this ring");
    // three one-tile phases without work; the second waits for the third,
    // which the launch's only CTA can never reach: the wait must give up
    const PPhase ph[3] = {{kPhNone, 0, 1, 1, 0, 0}, {kPhNone, 0, 1, 1, 0, 1}, {kPhNone, 0, 1, 1, 1, 0}};
    const int32_t off[4] = {0, 1, 2, 3}, deps[1] = {2};
    const uint64_t info[3] = {0, 1ull << 32, 2ull << 32};
    const size_t o_ph = 0, o_off = o_ph + sizeof(ph), o_dep = o_off + sizeof(off), o_info = o_dep + 16,
                 o_ctr = o_info + sizeof(info), bytes = o_ctr + 5 * sizeof(uint32_t);
    std::vector<char> img(bytes, 0);
    memcpy(img.data() + o_ph, ph, sizeof(ph));
    memcpy(img.data() + o_off, off, sizeof(off));
    memcpy(img.data() + o_dep, deps, sizeof(deps));
    memcpy(img.data() + o_info, info, sizeof(info));
    char *blob = (char *)dev_alloc(ctx, bytes);
    if (!blob) FAIL(HESPMV_E_NOMEM, "self-test allocation failed");
    PProg P{};
    P.ph = (const PPhase *)(blob + o_ph);
    P.off = (const int32_t *)(blob + o_off);
    P.deps = (const int32_t *)(blob + o_dep);
    P.info = (const uint64_t *)(blob + o_info);
    P.ctr = (uint32_t *)(blob + o_ctr);
    P.nph = 3;
    P.total = 3;
    P.wait_ns = 2000000;  // 2 ms
    cudaError_t e = cudaMemcpy(blob, img.data(), bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = persist_launch(c, P, 1, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    dev_free(ctx, blob);
    if (e != cudaSuccess) FAIL(HESPMV_E_CUDA, std::string("persistent self-test: ") + cudaGetErrorString(e));
    return hespmv_device_status(ctx, code);
}

int hespmv_set_graphs(hespmv_ctx *ctx, int32_t enable) {
    if (!ctx) return HESPMV_E_INVALID;
    ctx->use_graphs = enable != 0;
    return HESPMV_OK;
}

int hespmv_profile_enable(hespmv_ctx *ctx, int32_t enable) {
    if (!ctx) return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    DeviceGuard g(ctx->device);
    if (!ctx->prof) ctx->prof = new Profiler();
    if (enable) {
        cudaDeviceSynchronize();
        ctx->prof->reset();
    }
    ctx->prof->on = enable != 0;
    return HESPMV_OK;
}

int hespmv_profile_count(hespmv_ctx *ctx, int32_t *n) {
    if (!ctx || !n) return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    DeviceGuard g(ctx->device);
    if (!ctx->prof) {
        *n = 0;
        return HESPMV_OK;
    }
    CK(ctx->prof->collect());
    *n = (int32_t)ctx->prof->names.size();
    return HESPMV_OK;
}

int hespmv_profile_entry(hespmv_ctx *ctx, int32_t i, const char **name, int64_t *launches,
                         double *ms) {
    if (!ctx || !ctx->prof || i < 0 || i >= (int32_t)ctx->prof->launches.size()) return HESPMV_E_INVALID;
    if (name) *name = ctx->prof->names[i].c_str();
    if (launches) *launches = ctx->prof->launches[i];
    if (ms) *ms = ctx->prof->ms[i];
    return HESPMV_OK;
}

int hespmv_mulmod_rate(hespmv_ctx *ctx, int32_t kind, double *per_second) {
    if (!ctx || !per_second || (kind != 0 && kind != 1)) return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    DeviceGuard g(ctx->device);
    CK(mulmod_rate(ctx->h, kind, per_second));
    return HESPMV_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Key switching without device allocation.
//
// Some callers cannot allocate device memory at the moment they need a key
// switch: code that runs while another allocator owns the device's free
// memory (a framework pool that has reserved it), or a latency-sensitive loop
// that cannot pay for cudaMalloc/cudaFree, which may synchronise the device.
// hespmv_keyswitch_noalloc runs the same pipeline as hespmv_keyswitch but
// takes its scratch from the fixed array below, which the library reserves on
// every GPU where it is loaded and holds until the process exits.
namespace {

constexpr size_t kNoAllocScratchBytes = 32ull << 20;  // 32 MiB
constexpr size_t kNoAllocScratchWords = kNoAllocScratchBytes / 8;
static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocScratchWords];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
uint64_t *g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};

// Device address of the array on `dev` (which must be current); looked up
// once per device.  Host code cannot use the symbol itself: on the host it
// names a stand-in, not the device memory.
uint64_t *noalloc_scratch(int dev, std::string &err) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        err = "device ordinal out of range for the reserved scratch table";
        return nullptr;
    }
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return nullptr;
        }
        g_noalloc_addr[dev] = (uint64_t *)p;
    }
    return g_noalloc_addr[dev];
}

}  // namespace

extern "C" int hespmv_keyswitch_noalloc(hespmv_ctx *ctx, const uint64_t *d, uint32_t galois_elt,
                                        uint64_t *out, size_t n, void *stream) {
    if (!ctx || !d || !out) return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    if (!aligned16({d, out})) FAIL(HESPMV_E_INVALID, "device buffers must be 16-byte aligned");
    if (!ctx->have_keys) FAIL(HESPMV_E_INVALID, "keygen first");
    DeviceGuard g(ctx->device);
    const uint64_t *key = ctx->rlk;
    if (galois_elt) {
        auto it = ctx->gk.find(galois_elt);
        if (it == ctx->gk.end()) FAIL(HESPMV_E_INVALID, "no Galois key for that element");
        key = it->second;
    }
    const Ctx c = view(ctx);
    const size_t per = ks_words(c, 1);
    if (n == 0) return HESPMV_OK;
    if (n > kNoAllocScratchWords / per)  // divided, not multiplied: a huge n cannot wrap past the check
        FAIL(HESPMV_E_INVALID, "hespmv_keyswitch_noalloc: " + std::to_string(n) +
                                   " ciphertexts need more scratch than the reserved " +
                                   std::to_string(kNoAllocScratchBytes) + "; at most " +
                                   std::to_string(kNoAllocScratchWords / per) +
                                   " per call with these parameters");
    std::string err;
    uint64_t *scratch = noalloc_scratch(ctx->device, err);
    if (!scratch) FAIL(HESPMV_E_CUDA, err);
    // every stage writes the scratch words it later reads, so nothing in the
    // shared array has to start at zero
    const int64_t LN = (int64_t)c.L * c.N;
    CK(keyswitch_n(c, d, LN, key, out, nullptr, 0, 0, 0, n, scratch, (cudaStream_t)stream));
    return HESPMV_OK;
}

// ---------------------------------------------------------------------------
// Serving: continuous batching of SpMV requests (resident keys and operands).
namespace {

typedef std::chrono::steady_clock Clock;

struct ServeReq {
    uint64_t ticket = 0;
    const hespmv_cssc *m = nullptr;
    const uint64_t *A = nullptr, *X = nullptr;
    uint64_t *y = nullptr;  // null: result kept in slot scratch and dropped
    Clock::time_point t_sub;
};

struct ServeSlot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    uint64_t *ws = nullptr;     // workspace (evaluation + dropped results)
    size_t cap = 0;             // bytes
    int32_t *d_idx = nullptr;   // rotation schedule arena (device)
    int32_t *h_idx = nullptr;   // its pinned host staging
    size_t idx_cap = 0;         // int32 entries
    bool busy = false;
    std::vector<ServeReq> reqs;
    RotPlan plan;
};

}  // namespace

struct hespmv_server {
    hespmv_ctx *ctx = nullptr;
    std::vector<ServeSlot> slots;
    int32_t max_batch = 1;
    std::mutex mu;       // queue, tickets, counters
    std::mutex ctx_mu;   // context state (caches) shared by submit and the loop
    std::condition_variable cv;
    std::deque<ServeReq> queue;
    std::unordered_map<uint64_t, int64_t> done;  // ticket -> latency ns (-1: failed)
    uint64_t next_ticket = 1;
    bool stopping = false;
    std::thread th;
    int64_t submitted = 0, completed = 0, batches = 0, rejected = 0, max_inflight = 0;
    int err = HESPMV_OK;
    std::string errmsg;
};

namespace {

const size_t kServeIdxCap = 1 << 20;  // schedule entries per slot (4 MiB)

size_t slot_need(const Ctx &c, const std::vector<ServeReq> &reqs) {
    size_t total = 0, rot = 0, drop = 0;
    for (const ServeReq &r : reqs) {
        total += r.m->plan.chunks.size();
        for (const Chunk &ch : r.m->plan.chunks) rot += ch.c > 1;
        if (!r.y) drop += r.m->plan.parts.size();
    }
    SpmvPrep pp;
    spmv_sizes(c, total, rot, pp);
    return pp.need_bytes + drop * 2 * (size_t)c.L * c.N * 8;
}

// Launch one batch on a free slot (server thread).
int serve_launch(hespmv_server *s, ServeSlot &sl, std::vector<ServeReq> &batch) {
    hespmv_ctx *ctx = s->ctx;
    const Ctx c = view(ctx);
    const size_t n = batch.size();
    const int64_t CT = 2 * (int64_t)c.L * c.N;
    std::vector<const hespmv_cssc *> ms(n);
    std::vector<const uint64_t *> A(n), X(n);
    std::vector<uint64_t *> Y(n);
    size_t total = 0, rot = 0, drop = 0;
    for (size_t i = 0; i < n; ++i) {
        ms[i] = batch[i].m;
        A[i] = batch[i].A;
        X[i] = batch[i].X;
        total += ms[i]->plan.chunks.size();
        for (const Chunk &ch : ms[i]->plan.chunks) rot += ch.c > 1;
    }
    SpmvPrep pp;
    spmv_sizes(c, total, rot, pp);
    uint64_t *dropbuf = sl.ws + pp.need_bytes / 8;
    for (size_t i = 0; i < n; ++i) {
        if (batch[i].y) {
            Y[i] = batch[i].y;
        } else {
            Y[i] = dropbuf + drop * CT;
            drop += ms[i]->plan.parts.size();
        }
    }
    if (rot) {
        std::vector<int32_t> idx;
        build_rotation_ops(ctx, n, ms.data(), (int)pp.GR, &sl.plan, idx);
        if (idx.size() > sl.idx_cap) FAIL(HESPMV_E_REJECTED, "batch schedule exceeds the slot arena");
        memcpy(sl.h_idx, idx.data(), idx.size() * sizeof(int32_t));
        CK(cudaMemcpyAsync(sl.d_idx, sl.h_idx, idx.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                           sl.st));
        sl.plan.d_idx = sl.d_idx;
        pp.rp = &sl.plan;
    }
    int rc = spmv_enqueue(ctx, n, ms.data(), A.data(), X.data(), Y.data(), pp, sl.ws, sl.st);
    if (rc) return rc;
    CK(cudaEventRecord(sl.ev, sl.st));
    sl.reqs = std::move(batch);
    sl.busy = true;
    return HESPMV_OK;
}

void serve_loop(hespmv_server *s) {
    hespmv_ctx *ctx = s->ctx;
    cudaSetDevice(ctx->device);
    const Ctx c = view(ctx);
    for (;;) {
        // harvest finished slots
        int inflight = 0;
        for (ServeSlot &sl : s->slots) {
            if (!sl.busy) continue;
            cudaError_t e = cudaEventQuery(sl.ev);
            if (e == cudaErrorNotReady) {
                ++inflight;
                continue;
            }
            const Clock::time_point now = Clock::now();
            std::lock_guard<std::mutex> lock(s->mu);
            for (const ServeReq &r : sl.reqs) {
                s->done[r.ticket] =
                    e == cudaSuccess
                        ? std::chrono::duration_cast<std::chrono::nanoseconds>(now - r.t_sub).count()
                        : -1;
                ++s->completed;
            }
            if (e != cudaSuccess && !s->err) {
                s->err = HESPMV_E_CUDA;
                s->errmsg = std::string("serving batch: ") + cudaGetErrorString(e);
            }
            sl.reqs.clear();
            sl.busy = false;
        }
        // admit: fill every free slot from the queue (first come, first served)
        for (ServeSlot &sl : s->slots) {
            if (sl.busy) continue;
            std::vector<ServeReq> batch;
            {
                std::lock_guard<std::mutex> lock(s->mu);
                while (!s->queue.empty() && (int32_t)batch.size() < s->max_batch) {
                    batch.push_back(s->queue.front());
                    if (slot_need(c, batch) > sl.cap) {
                        batch.pop_back();
                        break;
                    }
                    s->queue.pop_front();
                }
            }
            if (batch.empty()) continue;
            std::vector<ServeReq> keep = batch;
            int rc;
            {
                std::lock_guard<std::mutex> clock(s->ctx_mu);
                rc = serve_launch(s, sl, batch);
            }
            std::lock_guard<std::mutex> lock(s->mu);
            if (rc) {
                for (const ServeReq &r : keep) {
                    s->done[r.ticket] = -1;
                    ++s->completed;
                }
                if (!s->err) {
                    s->err = rc;
                    s->errmsg = ctx->err;
                }
            } else {
                ++s->batches;
                ++inflight;
            }
        }
        {
            std::unique_lock<std::mutex> lock(s->mu);
            s->max_inflight = std::max<int64_t>(s->max_inflight, inflight);
            if (s->stopping && s->queue.empty() && inflight == 0) break;
            if (s->queue.empty() || inflight == (int)s->slots.size())
                s->cv.wait_for(lock, std::chrono::microseconds(inflight ? 20 : 200));
        }
    }
}

void server_release(hespmv_server *s) {
    for (ServeSlot &sl : s->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.st) cudaStreamDestroy(sl.st);
        dev_free(s->ctx, sl.ws);
        dev_free(s->ctx, sl.d_idx);
        if (sl.h_idx) cudaFreeHost(sl.h_idx);
    }
    s->slots.clear();
}

}  // namespace

extern "C" {

int hespmv_server_start(hespmv_ctx *ctx, int32_t slots, size_t mem_budget_bytes, int32_t max_batch,
                        hespmv_server **out) {
    if (!ctx || !out || slots < 1 || slots > 16 || max_batch < 1 || mem_budget_bytes == 0)
        return HESPMV_E_INVALID;
    NEED_DEVICE(ctx);
    if (!ctx->have_keys) FAIL(HESPMV_E_INVALID, "keygen first");
    DeviceGuard g(ctx->device);
    hespmv_server *s = new hespmv_server();
    s->ctx = ctx;
    s->max_batch = max_batch;
    s->slots.resize(slots);
    const size_t cap = mem_budget_bytes / slots;
    for (ServeSlot &sl : s->slots) {
        sl.cap = cap;
        sl.idx_cap = kServeIdxCap;
        bool ok = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) == cudaSuccess &&
                  cudaMallocHost((void **)&sl.h_idx, sl.idx_cap * sizeof(int32_t)) == cudaSuccess;
        sl.ws = ok ? (uint64_t *)dev_alloc(ctx, cap) : nullptr;
        sl.d_idx = sl.ws ? (int32_t *)dev_alloc(ctx, sl.idx_cap * sizeof(int32_t)) : nullptr;
        if (!sl.d_idx) {
            server_release(s);
            delete s;
            FAIL(HESPMV_E_NOMEM, "serving slot allocation failed");
        }
    }
    s->th = std::thread(serve_loop, s);
    *out = s;
    return HESPMV_OK;
}

int hespmv_server_submit(hespmv_server *s, const hespmv_cssc *m, const hespmv_ctbatch *A,
                         const hespmv_ctbatch *X, hespmv_ctbatch *y, uint64_t *ticket) {
    if (!s || !m || !A || !X || !ticket) return HESPMV_E_INVALID;
    hespmv_ctx *ctx = s->ctx;
    const size_t nc = m->plan.chunks.size();
    if (A->n < nc || X->n < nc || (y && y->n < m->plan.parts.size())) return HESPMV_E_INVALID;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stopping) return HESPMV_E_INVALID;
        if (s->err) return s->err;
    }
    if (!m->prepared) {
        // first request of a matrix: make its masks and tables resident (the
        // caller's thread; the serving thread never allocates)
        std::lock_guard<std::mutex> lock(s->ctx_mu);
        DeviceGuard g(ctx->device);
        int rc = prepare_matrix(ctx, m, nullptr);
        if (rc) return rc;
    }
    ServeReq r;
    r.m = m;
    r.A = A->data;
    r.X = X->data;
    r.y = y ? y->data : nullptr;
    const Ctx c = view(ctx);
    std::vector<ServeReq> one{r};
    if (slot_need(c, one) > s->slots[0].cap) {
        std::lock_guard<std::mutex> lock(s->mu);
        ++s->rejected;
        ctx->err = "request needs more device memory than a serving slot holds";
        return HESPMV_E_REJECTED;
    }
    {
        std::lock_guard<std::mutex> lock(s->mu);
        r.ticket = s->next_ticket++;
        r.t_sub = Clock::now();
        s->queue.push_back(r);
        ++s->submitted;
        *ticket = r.ticket;
    }
    s->cv.notify_one();
    return HESPMV_OK;
}

int hespmv_server_poll(hespmv_server *s, uint64_t ticket, int32_t *done, int64_t *latency_ns) {
    if (!s || !done) return HESPMV_E_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->done.find(ticket);
    if (it == s->done.end()) {
        *done = 0;
        if (latency_ns) *latency_ns = 0;
        return HESPMV_OK;
    }
    *done = it->second >= 0 ? 1 : -1;
    if (latency_ns) *latency_ns = it->second;
    return it->second >= 0 ? HESPMV_OK : (s->err ? s->err : HESPMV_E_CUDA);
}

int hespmv_server_stats(hespmv_server *s, int64_t *submitted, int64_t *completed, int64_t *batches,
                        int64_t *rejected, int64_t *max_inflight) {
    if (!s) return HESPMV_E_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    if (submitted) *submitted = s->submitted;
    if (completed) *completed = s->completed;
    if (batches) *batches = s->batches;
    if (rejected) *rejected = s->rejected;
    if (max_inflight) *max_inflight = s->max_inflight;
    return HESPMV_OK;
}

int hespmv_server_stop(hespmv_server *s, int64_t timeout_ms) {
    if (!s) return HESPMV_E_INVALID;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stopping = true;
    }
    s->cv.notify_one();
    // wait for the queue to drain and the last batches to finish, bounded
    const Clock::time_point t0 = Clock::now();
    bool timed_out = false;
    for (;;) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            if (s->completed >= s->submitted) break;
        }
        if (timeout_ms >= 0 &&
            std::chrono::duration_cast<std::chrono::milliseconds>(Clock::now() - t0).count() > timeout_ms) {
            timed_out = true;
            break;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    int rc = HESPMV_OK;
    if (timed_out) {
        // the loop still owns in-flight work: keep it running until it drains
        s->th.join();
        rc = HESPMV_E_TIMEOUT;
    } else {
        s->th.join();
    }
    DeviceGuard g(s->ctx->device);
    const int err = s->err;
    server_release(s);
    delete s;
    return rc ? rc : err;
}

}  // extern "C"
