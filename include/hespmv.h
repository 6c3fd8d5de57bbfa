/*
 * hespmv: encrypted sparse matrix-vector multiplication over the CSSC format
 * on one NVIDIA GB300 GPU (sm_103a).
 *
 * Method: "Efficient Privacy-Preserving Sparse Matrix-Vector Multiplication
 * Using Homomorphic Encryption" (CSSC format, Section 4.3; Algorithms 1-5).
 * The matrix owner encodes its CSR matrix as CSSC, splits it into
 * ciphertext-sized chunks and encrypts the chunk values; the vector owner
 * reorganises its vector by the chunk column indices and encrypts it; the
 * evaluator multiplies chunk pairs, aggregates rows by rotate-and-add and
 * masks, and returns one ciphertext per row partition; the key holder
 * decrypts and undoes the row permutation.
 *
 * Scheme: BGV over an RNS basis Q = q_0..q_{L-1} (NTT-friendly primes below
 * 2^50) with K special primes for hybrid key switching in dnum digits, and
 * plaintext modulus t (prime, t = 1 mod 2N).  Plaintext slots: row 0 of the
 * batching encoding (N/2 slots), rotated left by HE-Rot (Section 2.1).
 *
 * Conventions common to every call
 *  - Every function returns HESPMV_OK (0) or an error code below; nothing
 *    throws across this interface.  hespmv_last_error() gives a message.
 *  - Ciphertext layout on the device: uint64 words [2][L][N] per ciphertext,
 *    component-major, limb-major, residues in [0, q_l), NTT domain with index
 *    i holding the evaluation at psi_l^(2*bitrev(i)+1).  A batch of n
 *    ciphertexts is n such blocks back to back.
 *  - "device" pointers are CUDA device addresses on the context's device;
 *    "host" pointers are ordinary host memory owned by the caller, read or
 *    written only during the call (or, for *_async, until the stream reaches
 *    the copy).
 *  - Device memory the library needs comes from params.alloc/params.free
 *    when given (the Python binding passes PyTorch's caching allocator),
 *    else from cudaMalloc/cudaFree.
 *  - Work is enqueued on the caller's stream (cudaStream_t passed as void*;
 *    NULL = legacy default stream).  Calls without a stream argument
 *    (keygen, encrypt, decrypt, uploads of keys) synchronise the device
 *    before returning.
 *  - A context's evaluations share its workspace: evaluations enqueued on
 *    different streams must not overlap (order them, or use one stream, or
 *    the server of hespmv_server_*, whose slots have their own workspaces).
 */
#ifndef HESPMV_H
#define HESPMV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define HESPMV_OK 0
#define HESPMV_E_INVALID 1     /* bad argument, malformed CSR, wrong sizes   */
#define HESPMV_E_NOMEM 2       /* an allocation failed                        */
#define HESPMV_E_CUDA 3        /* a CUDA runtime call or kernel failed        */
#define HESPMV_E_RANGE 4       /* declared value bounds could reach t/2       */
#define HESPMV_E_UNSUPPORTED 5 /* parameters outside what the kernels handle  */
#define HESPMV_E_TIMEOUT 6     /* a bounded device-side wait expired          */
#define HESPMV_E_REJECTED 7    /* admission control refused a request         */

/* rotation key policy */
#define HESPMV_ROT_POW2 0  /* keys for 2^i; rotation by k chains its set bits, LSB first */
#define HESPMV_ROT_EXACT 1 /* one key per requested step                                */

/* which operand hespmv_encrypt encodes */
#define HESPMV_MATRIX 0
#define HESPMV_VECTOR 1

/* which key hespmv_key_export copies out */
/* CSSC serialization kinds */
#define HESPMV_SER_FULL 0  /* every array: VA, CI, CP, RM (Client A's own copy)              */
#define HESPMV_SER_SHAPE 1 /* CP only: the chunk shapes the cloud needs (rList, cList)         */

#define HESPMV_KEY_SECRET 0 /* s in the NTT domain over the L+K primes: [L+K][N]   */
#define HESPMV_KEY_PUBLIC 1 /* (pk0, pk1): [2][L][N]                               */
#define HESPMV_KEY_RELIN 2  /* relinearisation key: [dnum][2][L+K][N]              */
#define HESPMV_KEY_GALOIS 3 /* Galois key of element g: [dnum][2][L+K][N]          */

typedef void *(*hespmv_alloc_fn)(size_t bytes, void *user);
typedef void (*hespmv_free_fn)(void *ptr, void *user);

typedef struct hespmv_params {
    int32_t log2n;      /* ring degree N = 2^log2n, 4 <= log2n <= 15          */
    int32_t L;          /* ciphertext primes, 1..16                             */
    int32_t K;          /* special primes, 1..4                                 */
    int32_t dnum;       /* key-switching digits; alpha = ceil(L/dnum)           */
    uint64_t t;         /* plaintext modulus: prime, t = 1 mod 2N, t < 2^50     */
    int32_t prime_bits; /* ciphertext prime size; 0 means 50 (the only size run) */
    int32_t rot_policy; /* HESPMV_ROT_POW2 or HESPMV_ROT_EXACT                  */
    int32_t slots;      /* chunk capacity s; 0 means N/2 (row 0 of the slots)   */
    int32_t device;     /* CUDA device ordinal; -1 = host-only context (format
                           layer and parameter tables, no device calls)       */
    hespmv_alloc_fn alloc; /* optional device allocator (NULL: cudaMalloc)     */
    hespmv_free_fn free;   /* its matching free                                 */
    void *alloc_user;      /* passed back to alloc/free                         */
    int32_t scheme;        /* HESPMV_SCHEME_BGV (0, integers mod t),
                              HESPMV_SCHEME_CKKS (real values; t must be 0) or
                              HESPMV_SCHEME_BFV (integers mod t)                */
    int32_t scale_bits;    /* CKKS: matrix and vector scale 2^scale_bits, 10..60 */
    int32_t mask_scale_bits; /* CKKS: scale of the 0/1 masks, 1..60            */
    int32_t reserved;
} hespmv_params;

/* Schemes.  CKKS (the approximate scheme the paper names as the alternative
 * for real values, Section 6) runs the same circuit: every key, encryption
 * and key switch is the BGV one with t = 1 (errors e instead of t*e, plain
 * ModDown), no rescaling (all L primes throughout), and a SpMV result
 * carries scale 2^(2 scale_bits + mask_scale_bits).  It needs K >= alpha so
 * that P covers a key-switching digit. */
#define HESPMV_SCHEME_BGV 0
#define HESPMV_SCHEME_CKKS 1
/* BFV (the paper's scheme, Section 5): the BGV slots and keys with t = 1 in
 * their formulas, the message at Delta = floor(Q/t), and HE-Mult as defined:
 * d' = [round(t d / Q)]_Q for the integer tensor d of the centred inputs,
 * computed exactly in an auxiliary basis B > 2 t N Q.  Needs K >= alpha. */
#define HESPMV_SCHEME_BFV 2

typedef struct hespmv_ctx hespmv_ctx;         /* scheme, tables, keys, workspace */
typedef struct hespmv_cssc hespmv_cssc;       /* CSSC + partitions + chunk plan */
typedef struct hespmv_ctbatch hespmv_ctbatch; /* device ciphertexts [n][2][L][N] */

/* Message of the last failing call on this context (never NULL). */
const char *hespmv_last_error(const hespmv_ctx *ctx);

/* Library version string (never NULL). */
const char *hespmv_version(void);

/* ------------------------------------------------------------------ context */

/* Create a context: chooses the primes (largest q < 2^prime_bits with
 * q = 1 mod 2N, descending; first L form Q, next K form P), the smallest
 * primitive 2N-th roots, twiddle and RNS tables, all resident on the device.
 * The paper fixes one BFV parameter set (Section 5); the parameters here
 * are the caller's.  *ctx receives a handle released by hespmv_destroy. */
int hespmv_create(const hespmv_params *p, hespmv_ctx **ctx);
void hespmv_destroy(hespmv_ctx *ctx);

/* Copy out the moduli (L+K words: Q then P) and roots psi (L+K words); the
 * plaintext root zeta goes to *zeta.  Any pointer may be NULL. */
int hespmv_ctx_moduli(const hespmv_ctx *ctx, uint64_t *moduli, uint64_t *psi, uint64_t *zeta);

/* Bytes of device memory the context holds now (tables, keys, workspace,
 * cached masks). */
int hespmv_ctx_device_bytes(const hespmv_ctx *ctx, size_t *bytes);

/* -------------------------------------------------------------------- keys */

/* Generate the secret key, public key, relinearisation key and the Galois
 * keys from `seed` (Section 5: one relinearisation key set plus rotation
 * keys).  rot_steps lists the left-rotation amounts to support (n_steps
 * entries; n_steps = 0 generates no Galois key); rot_steps = NULL with the
 * POW2 policy generates every power of two below N/2.  Randomness:
 * SplitMix64 streams derived from seed.  Synchronous. */
int hespmv_keygen(hespmv_ctx *ctx, uint64_t seed, const int32_t *rot_steps, size_t n_steps);

/* Copy a key to host memory (layouts at HESPMV_KEY_*); n_words must be the
 * exact size.  galois_elt selects the Galois key (ignored otherwise). */
int hespmv_key_export(hespmv_ctx *ctx, int32_t which, uint32_t galois_elt, uint64_t *host_out,
                      size_t n_words);

/* ------------------------------------------------------- format (client A) */

/* Build the CSSC form of a CSR matrix (Algorithm 5: rows by descending
 * non-zero count, stable; left alignment; column-major VA/CI; CP of length
 * Lmax+1), partition it into blocks of at most s rows (Section 4.7) and cut
 * each block into chunks (Algorithm 2, padded-area capacity h*c <= s).
 * rowptr[rows+1], colidx[nnz] strictly ascending within each row, values
 * vals[nnz] (integers; fixed-point values are quantised by the caller; NULL
 * records the pattern only, for CKKS contexts, whose values are given to
 * hespmv_encrypt_real).
 * max_abs_x > 0 declares |x_j| <= max_abs_x; if any row could then reach
 * t/2 the call fails with HESPMV_E_RANGE.  max_abs_x <= 0 skips the check.
 * Host only (no device work).  Release with hespmv_cssc_free. */
int hespmv_encode_cssc(hespmv_ctx *ctx, int32_t rows, int32_t cols, int64_t nnz,
                       const int64_t *rowptr, const int32_t *colidx, const int64_t *vals,
                       int64_t max_abs_x, hespmv_cssc **out);
void hespmv_cssc_free(hespmv_cssc *m);

/* Counts: partitions, chunks (= ciphertexts per operand), rotations that
 * Algorithm 4 performs (HE-Rot calls), elementary key switches they take
 * under the context's policy, rows, cols, nnz. Any pointer may be NULL. */
int hespmv_cssc_info(const hespmv_cssc *m, int32_t *n_parts, int32_t *n_chunks, int64_t *n_rot,
                     int64_t *n_keyswitch, int32_t *rows, int32_t *cols, int64_t *nnz);

/* Per chunk: rows h (rList), columns c (cList), partition index.  Arrays of
 * n_chunks entries; any may be NULL. */
int hespmv_cssc_chunks(const hespmv_cssc *m, int32_t *h, int32_t *c, int32_t *part);

/* The chunk column indices Client A sends to Client B (Algorithm 1): chunk
 * k's h*c slot indices, concatenated in chunk order; -1 marks padding.
 * *ci points into the handle (valid until hespmv_cssc_free). */
int hespmv_cssc_colindex(const hespmv_cssc *m, const int32_t **ci, size_t *len);

/* The CSSC arrays of partition `part` (Algorithm 5): pointers into the
 * handle.  VA/CI have nnz_part entries, CP has Lmax+1, RM has the
 * partition's rows (local row indices). */
int hespmv_cssc_arrays(const hespmv_cssc *m, int32_t part, const int64_t **va, const int32_t **ci,
                       size_t *nnz_part, const int64_t **cp, size_t *cp_len, const int32_t **rm,
                       size_t *rm_len, int32_t *row0);

/* Distinct left-rotation amounts Algorithm 4 needs for this matrix
 * (ascending).  Writes at most cap entries; *n receives the total. */
int hespmv_cssc_rotation_steps(const hespmv_cssc *m, int32_t *steps, size_t cap, size_t *n);

/* Key transfer: the key holder hands the evaluator its evaluation keys
 * (public key, relinearisation key, Galois keys) without the secret key.
 * Format: "HSKY", version, kind, Galois key count, ring fingerprint, then
 * [sk [L+K][N]] (HESPMV_KEYS_ALL only), pk [2][L][N], rlk
 * [dnum][2][L+K][N], and per Galois key its element (u64) and key, as the
 * device holds them (key-switching keys in Montgomery form x 2^64 mod q).
 * buf NULL: *len receives the size only.  Deserialize validates the ring,
 * the length, every residue and every Galois element (HESPMV_E_INVALID) and
 * replaces the context's keys; a context loaded with HESPMV_KEYS_EVAL
 * evaluates and encrypts but refuses to decrypt.  Synchronous. */
#define HESPMV_KEYS_EVAL 0
#define HESPMV_KEYS_ALL 1
int hespmv_keys_serialize(hespmv_ctx *ctx, int32_t what, void *buf, size_t cap, size_t *len);
int hespmv_keys_deserialize(hespmv_ctx *ctx, const void *buf, size_t len);

/* Serialize a CSSC plan (Algorithm 1: what Client A keeps, or the chunk
 * shapes it hands to the cloud).  Format, little-endian, fields 8-byte
 * aligned: magic "HSCS", version, kind, s, rows, cols, nnz, n_parts, then
 * per partition row0, rows, nnz_part, |CP|, CP[], and for HESPMV_SER_FULL
 * VA[], CI[], RM[].  buf NULL: *len receives the size only; cap < size:
 * HESPMV_E_INVALID with *len set.  A shape-only plan serializes only as
 * HESPMV_SER_SHAPE.  Host only. */
int hespmv_cssc_serialize(const hespmv_cssc *m, int32_t kind, void *buf, size_t cap, size_t *len);
/* Rebuild a plan from hespmv_cssc_serialize output (chunks recomputed by
 * Algorithm 2).  Every length, bound, permutation and ordering is checked
 * before use: HESPMV_E_INVALID with a message on any inconsistency,
 * including a chunk capacity s other than the context's.  A shape-only plan
 * evaluates (spmv) but refuses encrypt, decrypt, colindex and arrays.  Host
 * only.  Release with hespmv_cssc_free. */
int hespmv_cssc_deserialize(hespmv_ctx *ctx, const void *buf, size_t len, hespmv_cssc **out);

/* --------------------------------------------------------- ciphertext batch */

int hespmv_ctbatch_create(hespmv_ctx *ctx, size_t n_ct, hespmv_ctbatch **out);
void hespmv_ctbatch_free(hespmv_ctbatch *b);
/* Device address and count of a batch. */
int hespmv_ctbatch_data(const hespmv_ctbatch *b, uint64_t **dev, size_t *n_ct);
/* Host <-> device copies of n_ct whole ciphertexts, on `stream`. */
int hespmv_ctbatch_upload(hespmv_ctbatch *b, const uint64_t *host, size_t n_ct, void *stream);
int hespmv_ctbatch_download(const hespmv_ctbatch *b, uint64_t *host, size_t n_ct, void *stream);
/* Serialize a batch for transfer between parties: magic "HSCT", version,
 * log2 N, L, n_ct, a fingerprint of (N, q_0..q_{L-1}, t), then the n_ct
 * ciphertexts [2][L][N] as little-endian u64.  buf NULL: *len receives the
 * size only.  Synchronous (waits for the device copy). */
int hespmv_ctbatch_serialize(const hespmv_ctbatch *b, void *buf, size_t cap, size_t *len);
/* Load a serialized batch into a new device batch of this context.  Fails
 * with HESPMV_E_INVALID if the stream is truncated or longer than its
 * header says, comes from another ring, or holds a residue >= its prime.
 * Synchronous. */
int hespmv_ctbatch_deserialize(hespmv_ctx *ctx, const void *buf, size_t len, hespmv_ctbatch **out);

/* Encode and encrypt one operand (Algorithm 1, Client A / Client B).
 * which = HESPMV_MATRIX: the chunk values; HESPMV_VECTOR: x (cols entries)
 * reorganised by the chunk column indices (Algorithm 3).  Ciphertext k uses
 * encryption randomness stream k of `seed`.  *out gets n_chunks
 * ciphertexts.  Synchronous. */
int hespmv_encrypt(hespmv_ctx *ctx, const hespmv_cssc *m, int32_t which, const int64_t *x,
                   uint64_t seed, hespmv_ctbatch **out);

/* CKKS contexts: encode and encrypt real values (Client A: the matrix values
 * in the CSR order given to hespmv_encode_cssc, nnz entries; Client B: x,
 * cols entries), each chunk's slots encoded at 2^scale_bits (the inverse
 * canonical embedding, rounded half away from zero; see hespmv_ckks_encode)
 * and encrypted as hespmv_encrypt does.  HESPMV_E_RANGE if a coefficient
 * would reach 2^62.  Plans read back by hespmv_cssc_deserialize lack the
 * CSR positions and refuse the matrix.  Synchronous. */
int hespmv_encrypt_real(hespmv_ctx *ctx, const hespmv_cssc *m, int32_t which, const double *values,
                        uint64_t seed, hespmv_ctbatch **out);
/* CKKS plaintext-matrix mode: the matrix chunks encoded, not encrypted. */
int hespmv_encode_matrix_plain_real(hespmv_ctx *ctx, const hespmv_cssc *m, const double *vals,
                                    hespmv_ctbatch **out);
/* CKKS encoding of n <= N/2 real slot values at 2^scale_bits: slot j is the
 * evaluation at zeta^(5^j), zeta = exp(i pi / N), and
 *   coef[k] = round(2^scale_bits * (2/N) * sum_j z_j cos(pi k 5^j / N)),
 * k < N, rounded half away from zero (double-double arithmetic: the exact
 * rounding).  Host only; HESPMV_E_RANGE beyond 2^62. */
int hespmv_ckks_encode(hespmv_ctx *ctx, const double *z, size_t n, int32_t scale_bits,
                       int64_t *coef);

/* ------------------------------------------------------------ evaluation */

/* The cloud lines of Algorithm 1 with Aggregation (Algorithm 4): for every
 * chunk k, HE-Mult(A_k, X_k) with relinearisation; per chunk the totalSum
 * rotate-and-add over its c column blocks of stride h; then per partition
 * res = sum_k intraRes_k * mask_{h_k}.  A and X hold n_chunks ciphertexts.
 * If *y is NULL a batch of n_parts ciphertexts is created; otherwise *y
 * must hold n_parts ciphertexts and is overwritten.  Enqueued on stream. */
int hespmv_spmv(hespmv_ctx *ctx, const hespmv_cssc *m, const hespmv_ctbatch *A,
                const hespmv_ctbatch *X, hespmv_ctbatch **y, void *stream);

/* Plaintext-matrix mode (the trust model of the Rhombus comparison in
 * Section 5: the evaluator holds the matrix in the clear, only the vector is
 * encrypted).  hespmv_encode_matrix_plain encodes the chunk values as trivial
 * ciphertexts (m, 0) in the NTT domain (no randomness; keys not needed);
 * hespmv_spmv_ptmatrix evaluates Algorithm 1 with HE-CMult in place of HE-Mult
 * (no relinearisation), then Algorithm 4 as hespmv_spmv. */
int hespmv_encode_matrix_plain(hespmv_ctx *ctx, const hespmv_cssc *m, hespmv_ctbatch **out);
int hespmv_spmv_ptmatrix(hespmv_ctx *ctx, const hespmv_cssc *m, const hespmv_ctbatch *A,
                         const hespmv_ctbatch *X, hespmv_ctbatch **y, void *stream);

/* hespmv_spmv from host buffers: copies A_host and X_host (n_chunks
 * ciphertexts each) to the device, evaluates, copies the n_parts result
 * ciphertexts to y_host, and synchronises `stream`. */
int hespmv_spmv_host(hespmv_ctx *ctx, const hespmv_cssc *m, const uint64_t *A_host,
                     const uint64_t *X_host, uint64_t *y_host, void *stream);

/* Packed ciphertexts (the wire form of hespmv_spmv_host_packed).  RNS
 * residues are uniform below primes of at most W = max_i bitlen(q_i) bits
 * (i < L), so a residue takes W bits instead of 64: each limb of a
 * ciphertext [2][L][N] becomes ceil(N W / 64) little-endian u64 words, with
 * residue k in bits [k W, k W + W) of the limb's bit string (bit b of the
 * string is bit b mod 64 of word b / 64; the unused high bits of a limb's
 * last word are zero).  *words receives the words of one packed ciphertext
 * and *bits receives W (either may be NULL).  Host only. */
int hespmv_ct_packed_words(const hespmv_ctx *ctx, size_t *words, int32_t *bits);
/* n_ct ciphertexts [n_ct][2][L][N] -> packed (n_ct * words u64, caller-owned).
 * HESPMV_E_INVALID if a residue is not below its prime.  Host only. */
int hespmv_ct_pack(const hespmv_ctx *ctx, const uint64_t *cts, size_t n_ct, uint64_t *packed);
/* The inverse; HESPMV_E_INVALID if a residue is not below its prime or a
 * padding bit is set.  Host only. */
int hespmv_ct_unpack(const hespmv_ctx *ctx, const uint64_t *packed, size_t n_ct, uint64_t *cts);
/* hespmv_spmv_host on packed buffers: A_packed and X_packed hold n_chunks
 * packed ciphertexts each and are copied to the device in groups (the
 * copies of later groups overlapping the HE-Mult of earlier ones; the fused
 * HE-Mult reads the packed residues directly, other paths unpack each group
 * first); y_packed receives the n_parts results, packed on the
 * device.  A residue that is not below its prime is evaluated reduced modulo
 * the prime and the call returns HESPMV_E_INVALID.  Synchronises `stream`.
 * Page-locked host buffers (cudaHostAlloc) make the copies asynchronous. */
int hespmv_spmv_host_packed(hespmv_ctx *ctx, const hespmv_cssc *m, const uint64_t *A_packed,
                            const uint64_t *X_packed, uint64_t *y_packed, void *stream);
/* Pipelined form of hespmv_spmv_host_packed for a stream of independent
 * evaluations: enqueues the uploads, the evaluation and the result download
 * and returns without waiting.  Consecutive calls use three staging slots in
 * turn, so a call's uploads run while earlier calls compute; a slot is
 * refilled only once the call that used it before has copied its result out
 * (ordered on the device, the host never blocks).  A_packed, X_packed and
 * y_packed must stay valid and unmodified until `stream` has passed the call
 * (e.g. cudaStreamSynchronize); the uploads run on the context's own copy
 * stream, ordered after the slot's previous evaluation only.  Consecutive
 * calls must use the same stream (the evaluations share the workspace).  Kernels are
 * launched one by one (no graph).  A residue not below its prime is reported
 * by hespmv_device_status, not by this call. */
int hespmv_spmv_host_packed_async(hespmv_ctx *ctx, const hespmv_cssc *m, const uint64_t *A_packed,
                                  const uint64_t *X_packed, uint64_t *y_packed, void *stream);
/* Upload groups of the host-buffer evaluations (1..64; 0 restores the
 * defaults: 7 for the synchronous calls, 2 for the pipelined one;
 * hespmv_get_upload_groups gives 0 while the defaults apply).  The chunks are uploaded in that many groups; the HE-Mult of a
 * group starts when its own upload has landed, and consecutive groups run on
 * two streams so that one group's kernels fill the tails of the other's.
 * More groups start the work earlier but give each fused key switch fewer
 * ciphertexts.  Results do not depend on it.  Host only. */
int hespmv_set_upload_groups(hespmv_ctx *ctx, int32_t groups);
int hespmv_get_upload_groups(const hespmv_ctx *ctx, int32_t *groups);

/* Many independent SpMVs in one batched evaluation (same context and keys):
 * every stage runs once over the chunks of all n instances.  y[i] as in
 * hespmv_spmv. */
int hespmv_spmv_batched(hespmv_ctx *ctx, size_t n, const hespmv_cssc *const *m,
                        const hespmv_ctbatch *const *A, const hespmv_ctbatch *const *X,
                        hespmv_ctbatch **y, void *stream);

/* ---------------------------------------------------------- key holder */

/* Decrypt the n_parts result ciphertexts and undo the row permutation
 * (Algorithm 1, last lines): out_rows[rows] receives the centred values.
 * Synchronous. */
int hespmv_decrypt(hespmv_ctx *ctx, const hespmv_cssc *m, const hespmv_ctbatch *y,
                   int64_t *out_rows);

/* Decrypt ciphertext `index` of a batch to its N slot values in [0, t):
 * row 0 slots 0..N/2-1 then row 1. Synchronous. */
/* CKKS: decrypt (exact CRT of [c0 + c1 s]_Q, centred), decode the N/2 slots
 * and divide by 2^scale_bits.  hespmv_decrypt_real un-permutes the rows of
 * a SpMV result, whose scale is 2^(2 scale_bits + mask_scale_bits).
 * Synchronous. */
int hespmv_decrypt_real_slots(hespmv_ctx *ctx, const hespmv_ctbatch *b, size_t index,
                              int32_t scale_bits, double *slots_out);
int hespmv_decrypt_real(hespmv_ctx *ctx, const hespmv_cssc *m, const hespmv_ctbatch *y,
                        double *out_rows);

/* CKKS rescaling (the paper evaluates one HE-Mult per chunk and keeps every
 * ciphertext at the top level, so its SpMV needs none; Section 6 names CKKS,
 * whose deeper circuits rescale after products -- the RNS form of Cheon,
 * Han, Kim, Kim and Song 2018).  ct: n ciphertexts [n][2][L][N] on the
 * device (NTT domain, all L primes); out: [n][2][L-1][N], each component c
 * replaced by (c - r) / q_{L-1}, r the centred remainder of c mod q_{L-1}
 * (the quotient rounded to nearest), so the plaintext and its scale are
 * divided by q_{L-1}.  16-byte aligned, out must not alias ct.  CKKS
 * contexts with L >= 2 only (E_INVALID otherwise).  Enqueued on stream; uses
 * the context's workspace (3 n N words). */
int hespmv_rescale(hespmv_ctx *ctx, const uint64_t *ct, uint64_t *out, size_t n, void *stream);
/* Decrypt one CKKS ciphertext [2][limbs][N] on the device over the first
 * `limbs` primes (a rescaled ciphertext has L - 1), exact CRT of
 * [c0 + c1 s] centred, decode the N/2 slots and divide by `scale` (any
 * positive value: a rescaled scale is 2^k / q_{L-1}).  Synchronous. */
int hespmv_decrypt_real_level(hespmv_ctx *ctx, const uint64_t *ct, int32_t limbs, double scale,
                              double *slots_out);

int hespmv_decrypt_slots(hespmv_ctx *ctx, const hespmv_ctbatch *b, size_t index,
                         uint64_t *slots_out);

/* ------------------------------------------------------------ serving */

/* A serving loop with continuous batching (keys and operands resident in
 * HBM).  A host thread takes queued requests first come first served into
 * batched evaluations; each of `slots` concurrent evaluations runs on its own
 * stream with its own workspace of mem_budget_bytes / slots bytes, so batches
 * overlap on the device and new requests are admitted as soon as a slot and
 * its memory free up (at most max_batch requests per evaluation).  A request
 * whose own footprint exceeds a slot is rejected (HESPMV_E_REJECTED).  While
 * a server runs, its context must only be used through the hespmv_server_*
 * calls (plus reads of ciphertext batches that are not in flight). */
typedef struct hespmv_server hespmv_server;
int hespmv_server_start(hespmv_ctx *ctx, int32_t slots, size_t mem_budget_bytes, int32_t max_batch,
                        hespmv_server **out);
/* Queue an SpMV of matrix m on device operands A, X (as for hespmv_spmv).
 * The result goes to y (n_parts ciphertexts), or is computed and dropped when
 * y is NULL.  *ticket identifies the request.  Thread-safe.  The first request
 * of a matrix makes its mask plaintexts resident (synchronous). */
int hespmv_server_submit(hespmv_server *s, const hespmv_cssc *m, const hespmv_ctbatch *A,
                         const hespmv_ctbatch *X, hespmv_ctbatch *y, uint64_t *ticket);
/* *done = 1 once the request's device work has finished (its y is final),
 * 0 while queued or running, -1 if its batch failed.  *latency_ns = time from
 * submission to the loop's observation of completion (host steady clock). */
int hespmv_server_poll(hespmv_server *s, uint64_t ticket, int32_t *done, int64_t *latency_ns);
int hespmv_server_stats(hespmv_server *s, int64_t *submitted, int64_t *completed, int64_t *batches,
                        int64_t *rejected, int64_t *max_inflight);
/* Drain and stop: waits at most timeout_ms (< 0: no limit) for every
 * submitted request; returns HESPMV_E_TIMEOUT if the wait expired (the loop is
 * then still joined after its in-flight batches finish), then releases the
 * slots and the handle. */
int hespmv_server_stop(hespmv_server *s, int64_t timeout_ms);

/* -------------------------------------------------- HE primitives (device) */
/* All pointers below are device addresses of n whole ciphertexts (or
 * polynomials where stated), 16-byte aligned (E_INVALID otherwise); in-place
 * use (out == in) is allowed except where noted.  Enqueued on stream. */

/* Forward / inverse negacyclic NTT of n_items x n_limbs polynomials stored
 * back to back (16-byte aligned, residues in [0, q)); limb k of each item uses
 * modulus index prime0 + k (0..L-1 = Q, L..L+K-1 = P, L+K = t). */
int hespmv_ntt_forward(hespmv_ctx *ctx, uint64_t *data, int32_t prime0, int32_t n_limbs,
                       int32_t n_items, void *stream);
int hespmv_ntt_inverse(hespmv_ctx *ctx, uint64_t *data, int32_t prime0, int32_t n_limbs,
                       int32_t n_items, void *stream);

/* HE-Add (Section 2.1). */
int hespmv_he_add(hespmv_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t *out, size_t n,
                  void *stream);
/* Tensor product: d = (a0 b0, a0 b1 + a1 b0, a1 b1), out [n][3][L][N]. */
int hespmv_he_tensor(hespmv_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t *d, size_t n,
                     void *stream);
/* Relinearise d [n][3][L][N] -> out [n][2][L][N] (out must not alias d). */
int hespmv_he_relin(hespmv_ctx *ctx, const uint64_t *d, uint64_t *out, size_t n, void *stream);
/* HE-Mult (Section 2.1): tensor + relinearisation. */
int hespmv_he_mult(hespmv_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t *out, size_t n,
                   void *stream);
/* HE-Rot (Section 2.1): slot j of the result holds slot j+k (each row);
 * under POW2 a chain of key switches. out must not alias ct. */
int hespmv_he_rotate(hespmv_ctx *ctx, const uint64_t *ct, int32_t k, uint64_t *out, size_t n,
                     void *stream);
/* HE-CMult by the mask [1]^r [0]^(N/2-r) of Algorithm 4. */
int hespmv_he_cmult_mask(hespmv_ctx *ctx, const uint64_t *ct, int32_t r, uint64_t *out, size_t n,
                         void *stream);
/* Hybrid key switch of polynomials d [n][L][N] with the relinearisation key
 * (galois_elt = 0) or the Galois key of galois_elt: out [n][2][L][N]. */
int hespmv_keyswitch(hespmv_ctx *ctx, const uint64_t *d, uint32_t galois_elt, uint64_t *out,
                     size_t n, void *stream);

/* Key switch that allocates no device memory.  The paper has no counterpart:
 * this is a deployment aid.  Same arguments and result as hespmv_keyswitch,
 * but the scratch comes from one fixed 32 MiB array in device memory that the
 * library reserves on every GPU where it is loaded (held until the process
 * exits), instead of from the context's workspace.  It is for callers that
 * must not allocate device memory where they call it: code that runs while
 * another allocator owns the device's free memory (a framework pool that has
 * reserved it), and latency-sensitive loops that cannot pay for
 * cudaMalloc/cudaFree, which may synchronise the device.
 *  - Limit: n ciphertexts need n * 8*N*(L + dnum*(L+K) + 2*(L+K) + 2*L) bytes
 *    of scratch (about 21 MiB each at N = 2^15, L = 8, K = 2, dnum = 4);
 *    beyond 32 MiB the call fails with HESPMV_E_INVALID and says how many fit.
 *  - The first call on a device sets it up: it looks up the array's device
 *    address (cudaGetSymbolAddress) with that device current.  Make that first
 *    call before any stream capture.
 *  - All calls share the one array, which keeps the last call's contents;
 *    nothing in it has to start at zero (each stage writes the scratch it
 *    reads).  Calls that overlap on the GPU (several streams or threads) race
 *    on the array: serialise them. */
int hespmv_keyswitch_noalloc(hespmv_ctx *ctx, const uint64_t *d, uint32_t galois_elt,
                             uint64_t *out, size_t n, void *stream);

/* ------------------------------------------------------------ autotuning */

/* Schedule of an evaluation.  None of these changes a result bit: they set
 * how many ciphertexts share one launch of each stage and how the NTTs of
 * the fused key switch are split into their column and row passes. */
typedef struct hespmv_tuning {
    int32_t mult_batch; /* HE-Mult stage: ciphertexts per fused key switch (0: 32)        */
    int32_t rot_batch;  /* totalSum: ciphertexts per batched rotation round
                           (0: 32 at N = 2^15, else 64); in the persistent form: the
                           levels by which consecutive HE-Mult groups are staggered
                           in the work queue (0: none)                                */
    int32_t ntt_split;  /* fused key switch NTT split: 0 = default, 1 = alternative
                           (N = 2^LC x 2^LR with LC and LR exchanged or shifted by one)  */
    int32_t rows_tma;   /* fused key switch forward row pass: 0 = one CTA per tile,
                           1 = persistent CTAs fed by bulk asynchronous copies      */
    int32_t persistent; /* 1: each evaluation of device-resident operands is ONE
                           persistent launch (Algorithm 1's HE-Mults in groups of
                           mult_batch (0: 16) chunks, every chunk's Algorithm 4
                           totalSum chain and masked sum as a program of
                           dependent tiles taken from a device work queue);
                           0: staged launches.  Rings with alpha <= 2, K <= 2,
                           N = 2^11 .. 2^15; not BFV.                              */
    int32_t persist_blocks; /* CTAs of the persistent launch (0: all resident)     */
    int32_t streams;    /* staged device evaluations: 2 = consecutive HE-Mult groups
                           alternate between two streams (each with its own scratch),
                           so one group's kernels fill the other's tail waves;
                           0 or 1 = one stream.  Host-buffer evaluations always use
                           two when they have two or more groups.                  */
    double ms;          /* hespmv_autotune: device time of one evaluation             */
} hespmv_tuning;

/* Apply a schedule (e.g. one cached from an earlier hespmv_autotune).  Waits
 * for the device and drops captured graphs.  HESPMV_E_INVALID for negative
 * or huge batch sizes or a split the ring does not offer. */
int hespmv_set_tuning(hespmv_ctx *ctx, const hespmv_tuning *t);
int hespmv_get_tuning(const hespmv_ctx *ctx, hespmv_tuning *t);

/* Autotuner: times the evaluation of the given SpMVs (as hespmv_spmv_batched
 * would run them, into its own result buffers, on its own stream) under
 * candidate schedules -- each NTT split, each row-pass form, then HE-Mult
 * batches 1, 2, 4, ... up to 128, then rotation round widths 4, 8, ... up to
 * 512 (capped by the chunk counts), then two compute streams with HE-Mult
 * batches of about a half and a quarter of the chunks and rotation rounds of
 * about a half and a quarter of the rotating chunks, then every NTT split and
 * row-pass form again under the best so far, then the persistent form with
 * HE-Mult groups of 4, 16 and 64 -- by coordinate descent from the default,
 * `reps` timed evaluations after one warm-up each, skipping any whose
 * workspace would not fit in free device memory.  Applies the fastest and
 * returns it in *best; tried[0 .. min(cap, *n_tried)) lists every setting
 * timed (effective batch sizes; ms = -1: skipped).  Synchronous. */
int hespmv_autotune(hespmv_ctx *ctx, size_t n, const hespmv_cssc *const *m,
                    const hespmv_ctbatch *const *A, const hespmv_ctbatch *const *X, int32_t reps,
                    hespmv_tuning *best, hespmv_tuning *tried, size_t cap, size_t *n_tried);

/* Evaluations (hespmv_spmv, hespmv_spmv_batched, hespmv_spmv_host) are
 * recorded once into a CUDA graph per set of matrices, buffers and workspace
 * and replayed afterwards (one launch per evaluation).  enable = 0 makes
 * every evaluation launch its kernels one by one.  Graphs are not used while
 * profiling is enabled.  Default: enabled. */
/* Device-side waits (the bulk-copy barriers of the key-switch row pass, and
 * the dependency waits of the persistent evaluation, which give up after 4 s)
 * are bounded; one that runs out records an error code in the context (1:
 * copy barrier, 3: persistent dependency) and its kernel stops early.  This call reads and clears it:
 * HESPMV_E_TIMEOUT if set (results since the last check are invalid), else
 * HESPMV_OK.  Decryption calls it first.  Synchronous. */
int hespmv_device_status(hespmv_ctx *ctx, int32_t *code);
/* Self-test of that path: launches a kernel whose wait cannot complete (a
 * barrier expecting bytes no copy delivers), which gives up after a few
 * polls; returns HESPMV_E_TIMEOUT and leaves the context usable. */
int hespmv_selftest_wait_timeout(hespmv_ctx *ctx, int32_t *code);
/* The same for the persistent evaluation's dependency waits: a launch of one
 * CTA whose second work tile depends on a third that it can never reach; the
 * wait gives up after 2 ms, records code 3 and every CTA stops.  Returns
 * HESPMV_E_TIMEOUT with *code = 3 (read and cleared as above); the context
 * stays usable.  HESPMV_E_UNSUPPORTED on rings without the persistent form. */
int hespmv_selftest_persist_timeout(hespmv_ctx *ctx, int32_t *code);

int hespmv_set_graphs(hespmv_ctx *ctx, int32_t enable);

/* ------------------------------------------------------------ measurement */

/* Per-kernel device time.  While enabled, each kernel launch of the library
 * is bracketed by two CUDA events recorded on its stream (enabling clears
 * earlier records; the events add host work per launch, not device work). */
int hespmv_profile_enable(hespmv_ctx *ctx, int32_t enable);
/* Synchronise the device, fold the recorded events into per-kernel totals
 * and return in *n the number of distinct kernels seen since enabling. */
int hespmv_profile_count(hespmv_ctx *ctx, int32_t *n);
/* Kernel i < *n of hespmv_profile_count: its name (valid until the next
 * enable), launches and summed device milliseconds. */
int hespmv_profile_entry(hespmv_ctx *ctx, int32_t i, const char **name, int64_t *launches,
                         double *ms);
/* Issue rate of 64-bit modular multiplications on the context's device
 * (per second), measured by a microbenchmark of independent dependency
 * chains: kind 0 multiplies by a constant with a precomputed quotient
 * (Shoup), kind 1 multiplies two variable operands (Barrett).  Synchronous;
 * allocates its own small buffer with cudaMalloc. */
int hespmv_mulmod_rate(hespmv_ctx *ctx, int32_t kind, double *per_second);

#ifdef __cplusplus
}
#endif
#endif /* HESPMV_H */
