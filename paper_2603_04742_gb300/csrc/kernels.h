// Host launchers of the elementwise, key-switching, sampling and
// encode/decrypt kernels.  All run on the given stream; sizes in words.
#pragma once
#include "internal.h"
#include "persist.h"

namespace hespmv {

// ct batches [n][2][L][N]
cudaError_t op_add(const Ctx &c, const uint64_t *a, const uint64_t *b, uint64_t *out, size_t n_polys,
                   cudaStream_t st);   // n_polys polynomials of L limbs
cudaError_t op_tensor(const Ctx &c, const uint64_t *a, const uint64_t *b, uint64_t *d, size_t n,
                      cudaStream_t st);
// prod[i] = (a[i].c0 * x[i].c0, a[i].c0 * x[i].c1) for n pairs (plaintext a in normal form)
cudaError_t op_pt_ct_mul(const Ctx &c, const uint64_t *a, const uint64_t *x, uint64_t *prod,
                         size_t n, cudaStream_t st);
// out = ct * pt (pt [L][N] in Montgomery form, shared by all n ciphertexts)
cudaError_t op_cmult(const Ctx &c, const uint64_t *ct, const uint64_t *pt, uint64_t *out, size_t n,
                     cudaStream_t st);
// acc (one ct) += w (one ct) * pt
cudaError_t op_cmult_acc(const Ctx &c, uint64_t *acc, const uint64_t *w, const uint64_t *pt,
                         bool first, cudaStream_t st);
// out = sum_k w_k * masks[k] for w_k = w0 + k ciphertexts (masks: Montgomery form)
cudaError_t op_mask_acc(const Ctx &c, const uint64_t *w0, const uint64_t *const *masks,
                        int nterms, uint64_t *out, cudaStream_t st);
// dst[di[s]] (= or +=) src[si[s]], optionally through a Galois permutation,
// for m whole ciphertexts; null index lists mean s
cudaError_t op_ct_move(const Ctx &c, uint64_t *dst, const int32_t *di, const uint64_t *src,
                       const int32_t *si, const int32_t *perm, bool add, int m, cudaStream_t st);
// x <- x * 2^64 mod q over n_items x n_limbs limbs with moduli prime0..
cudaError_t op_to_mont_limbs(const Ctx &c, uint64_t *x, int prime0, int n_limbs, size_t n_items,
                             cudaStream_t st);
// out[p][i] = in[p][perm[i]] for n_polys polynomials (limbs are polynomials here)
cudaError_t op_permute(const Ctx &c, const uint64_t *in, uint64_t *out, const int32_t *perm,
                       size_t n_limbs_total, cudaStream_t st);
// pointwise product of two arrays of polynomials over limbs [prime0, prime0+n_limbs)
cudaError_t op_mul_limbs(const Ctx &c, const uint64_t *a, const uint64_t *b, uint64_t *out,
                         int prime0, int n_limbs, size_t n_items, cudaStream_t st);
// copy n_items strided blocks of `words` words
cudaError_t op_copy_strided(const Ctx &c, const uint64_t *src, int64_t src_stride, uint64_t *dst,
                            int64_t dst_stride, int64_t words, size_t n_items, cudaStream_t st);

// key switching pieces, n items
cudaError_t op_modup(const Ctx &c, const uint64_t *dcoef, uint64_t *ext, size_t n, cudaStream_t st);
cudaError_t op_inner(const Ctx &c, const uint64_t *ext, const uint64_t *key, uint64_t *acc, size_t n,
                     cudaStream_t st);
cudaError_t op_moddown_delta(const Ctx &c, const uint64_t *acc, uint64_t *delta, size_t n,
                             cudaStream_t st);
// out[c] = (acc[c] - delta[c]) * P^-1 (+ add_c), add given as base + item/component strides;
// add_mask bit c selects which components get the addend
cudaError_t op_moddown_final(const Ctx &c, const uint64_t *acc, const uint64_t *delta,
                             const uint64_t *add, int64_t add_item_stride, int64_t add_comp_stride,
                             int add_mask, uint64_t *out, size_t n, cudaStream_t st);

// fused hybrid key switch (ks.cu), keys in Montgomery form
bool ks_fused_supported(const Ctx &c);
// BFV HE-Mult tensor (exact scale and round), n ciphertext pairs in the
// NTT domain -> out [n][3][L][N] (NTT domain); scratch of bfv_tensor_words(n)
size_t bfv_tensor_words(const Ctx &c, size_t n);
cudaError_t bfv_tensor(const Ctx &c, const uint64_t *A, const uint64_t *B, uint64_t *out, size_t n,
                       uint64_t *scratch, cudaStream_t st);
// BFV message lift: coefficients m in [0, t) -> Delta * m over Q, [n][L][N]
cudaError_t op_bfv_delta(const Ctx &c, const uint64_t *m, uint64_t *out, size_t n, cudaStream_t st);
// number of NTT split variants the fused key switch offers for this ring
int ks_split_variants(const Ctx &c);
// one-time launch setup of the fused key switch (shared-memory limits and
// persistent grid sizes); call outside any stream capture
cudaError_t ks_prepare(const Ctx &c);
// self-test: a bounded wait that runs out and sets the device error word
cudaError_t op_wait_probe(const Ctx &c, cudaStream_t st);
// device error word code of the unpack kernel (kErrWaitTimeout = 1 is the
// bounded waits')
constexpr int kErrBadResidue = 2;
// packed ciphertexts (h.pack_bits bits per residue, whole-word limbs) <-> u64
// residues, n ciphertexts; unpack converts pa -> oa and, when pb is given,
// pb -> ob in the same launch; a residue not below its prime sets
// kErrBadResidue in the device error word
cudaError_t op_ct_unpack(const Ctx &c, const uint64_t *pa, uint64_t *oa, const uint64_t *pb, uint64_t *ob,
                         size_t n, cudaStream_t st);
cudaError_t op_ct_pack(const Ctx &c, const uint64_t *in, uint64_t *out, size_t n, cudaStream_t st);
cudaError_t keyswitch_fused(const Ctx &c, const uint64_t *d, int64_t d_stride, const uint64_t *key,
                            uint64_t *out, const uint64_t *add, int64_t add_is, int64_t add_cs,
                            int add_mask, size_t n, uint64_t *scratch, cudaStream_t st);
// relin_tensor_fused with item i's operands at ta[i] and tb[i] (device
// tables of ciphertext addresses): HE-Mult groups across several SpMVs
cudaError_t relin_tensor_fused_ptrs(const Ctx &c, const uint64_t *const *ta, const uint64_t *const *tb,
                                    const uint64_t *rlk, uint64_t *out, size_t n, uint64_t *scratch,
                                    cudaStream_t st);
// dst[0..n) = ptrs[0..n) (device table of addresses, written on the stream
// from launch parameters, so a captured graph replays it)
cudaError_t op_write_ptrs(const Ctx &c, const uint64_t **dst, const std::vector<const uint64_t *> &ptrs,
                          cudaStream_t st);
// HE-Rot of n ciphertexts in place, fused (requires ks_fused_supported):
// slot idx[i] of cts [..][2][L][N] becomes its image under the Galois
// automorphism of permutation perm (NTT domain), key-switched with gk; the
// slots must be distinct
cudaError_t rotate_fused_inplace(const Ctx &c, uint64_t *cts, const int32_t *idx, const int32_t *perm,
                                 const uint64_t *gk, size_t n, uint64_t *scratch, cudaStream_t st);
// relinearised HE-Mult of n ciphertext pairs (A + i*2LN, B + i*2LN) with the
// tensor product fused into the key switch (requires ks_fused_supported);
// pk_bits > 0: A and B are packed ciphertexts of that many bits per residue
// (a residue not below its prime sets kErrBadResidue)
cudaError_t relin_tensor_fused(const Ctx &c, const uint64_t *A, const uint64_t *B,
                               const uint64_t *rlk, uint64_t *out, size_t n, uint64_t *scratch,
                               cudaStream_t st, int pk_bits = 0);
// persistent evaluation (ks.cu): rings with N = 2^11 .. 2^15, alpha <= 2, K <= 2
bool persist_supported(const Ctx &c);
// one launch of the program P (counters zeroed beforehand), at most
// max_blocks CTAs (0: every resident CTA of the GPU)
cudaError_t persist_launch(const Ctx &c, const PProg &P, int max_blocks, cudaStream_t st);
// virtual grid (x, y) of each of the 7 stages of a persistent key switch of n items
void persist_stage_tiles(const Ctx &c, int n, int32_t gx[7], int32_t gy[7]);
// x <- x * 2^64 mod q over n_items x (L+K) limbs (keys to Montgomery form)
cudaError_t op_to_mont(const Ctx &c, uint64_t *x, size_t n_items, cudaStream_t st);

// sampling: signed coefficients [n_items][N]; stream of item k = stream0 + k * step
enum SampleKind { kTernary = 0, kCbd21 = 1 };
cudaError_t op_sample_signed(const Ctx &c, uint64_t seed, uint64_t stream0, uint64_t step, int kind,
                             int64_t *out, size_t n_items, cudaStream_t st);
// signed coefficients -> residues over limbs [prime0, prime0+n_limbs): out [n_items][n_limbs][N]
cudaError_t op_signed_to_limbs(const Ctx &c, const int64_t *coef, uint64_t *out, int prime0,
                               int n_limbs, size_t n_items, cudaStream_t st);
// uniform residues (NTT domain by definition) over limbs [prime0, prime0+n_limbs)
cudaError_t op_sample_uniform(const Ctx &c, uint64_t seed, uint64_t stream, uint64_t *out,
                              int prime0, int n_limbs, cudaStream_t st);
// key digit: b = -a*s + t*e + g*sp over all L+K limbs; g = P mod q_l on digit limbs
cudaError_t op_ksk_combine(const Ctx &c, const uint64_t *a, const uint64_t *e, const uint64_t *s,
                           const uint64_t *sp, int digit, uint64_t *b, cudaStream_t st);
// pk0 = -a*s + t*e over Q
cudaError_t op_pk_combine(const Ctx &c, const uint64_t *a, const uint64_t *e, const uint64_t *s,
                          uint64_t *pk0, cudaStream_t st);
// ct = (u pk0 + t e0 + m, u pk1 + t e1) for n items; u,e0,e1,m [n][L][N]
cudaError_t op_enc_combine(const Ctx &c, const uint64_t *u, const uint64_t *e0, const uint64_t *e1,
                           const uint64_t *m, const uint64_t *pk, uint64_t *ct, size_t n,
                           cudaStream_t st);

// encoding: values [n][nvals] (int64) -> E [n][N] mod t at the slot positions of row 0
cudaError_t op_scatter_slots(const Ctx &c, const int64_t *vals, int64_t nvals, uint64_t *E,
                             size_t n, cudaStream_t st);
// m [n][N] in [0,t) -> centred residues over Q: out [n][L][N]
cudaError_t op_lift(const Ctx &c, const uint64_t *m, uint64_t *out, size_t n, cudaStream_t st);
// x [L][N] = c0 + c1*s
cudaError_t op_dec_phase(const Ctx &c, const uint64_t *ct, const uint64_t *s, uint64_t *x,
                         cudaStream_t st);
// CKKS rescale: x [n_comp][N] last limbs in coefficient form -> y
// [n_comp][nl1][N] their centred values mod q_0..q_{nl1-1}; then out =
// (ct - y) * ql^-1 (ct: nl1 + 1 limbs per component, y already in the NTT
// domain), qinv [nl1][2] Shoup pairs
cudaError_t op_rescale_lift(const Ctx &c, const uint64_t *x, uint64_t *y, size_t n_comp, int nl1, uint64_t ql,
                            cudaStream_t st);
cudaError_t op_rescale_final(const Ctx &c, const uint64_t *ct, const uint64_t *y, uint64_t *out, size_t n_comp,
                             int nl1, const uint64_t *qinv, cudaStream_t st);
// x coef [L][N] -> m [N] = ([x]_Q centred) mod t
cudaError_t op_crt_to_t(const Ctx &c, const uint64_t *x, uint64_t *m, cudaStream_t st);
// slots[j] = E[slot_idx[j]] for j < N
cudaError_t op_gather_slots(const Ctx &c, const uint64_t *E, uint64_t *slots, cudaStream_t st);

}  // namespace hespmv
