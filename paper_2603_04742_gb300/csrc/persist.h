// Key-switch operand descriptors and the persistent evaluation program
// (shared by the device code in ks.cu and the program builder in api.cu).
#pragma once
#include <cstdint>

#include "modarith.cuh"

namespace hespmv {

// Constants of the fused key switch (device tables of the context).
struct KsArgs {
    const ModConst *mc;
    const uint64_t *tw;        // [modulus][4][N]
    const uint64_t *zc;        // [L][4]  fold constants of step 2
    const uint64_t *yc;        // [K][4]  fold constants of step 5
    const uint64_t *modup_mod; // [dnum][alpha][L+K][2]
    const uint64_t *phat_t;    // [K][L][2]  Phat_k * t mod q_i
    const uint64_t *modup_modw;  // modup_mod times the target prime's first forward twiddle
    const uint64_t *phat_tw;     // phat_t times the target prime's first forward twiddle
    const uint64_t *pinv;      // [L][2]
    const uint64_t *pmont;     // [L]     P * 2^64 mod q_i
    const uint64_t *pmont2;    // [L]     P * 2^128 mod q_i
    int *err;                  // device error word (bounded waits)
    int log2n, L, K, dnum, alpha;
};

// Input of a key switch: d (NTT domain, item stride ds), or, fused with the
// tensor product of HE-Mult, d = a1 * b1 for ciphertexts a = ta + i*ts,
// b = tb + i*ts, whose (a0 b0, a0 b1 + a1 b0) is then the addend.
// With pk_bits > 0, ta and tb hold packed ciphertexts (pk_bits bits per
// residue, limbs of pk_lw words, ts words per ciphertext), read and checked
// here instead of in a separate unpack pass.
// With idx, item i reads slot idx[i] of d (stride ds); with perm, coefficient
// c of each limb reads coefficient perm[c] (a Galois automorphism in the NTT
// domain), so a rotation's permutation needs no separate pass.
struct KsSrc {
    const uint64_t *d;
    int64_t ds;
    const uint64_t *ta, *tb;
    int64_t ts;
    int pk_bits = 0;
    int64_t pk_lw = 0;
    const int32_t *idx = nullptr;
    const int32_t *perm = nullptr;
    // per-item ciphertext addresses (device tables) instead of ta/tb + i*ts:
    // HE-Mult groups that span several SpMVs of a batched evaluation
    const uint64_t *const *tap = nullptr;
    const uint64_t *const *tbp = nullptr;
};

// Addend of the key switch's output: component c (add_mask bit c) of
// add + item * is + c * cs, [L][N] each (item -> idx[item], coefficient
// c -> perm[c] when given, as for KsSrc).
struct KsAdd {
    const uint64_t *p;
    int64_t is, cs;
    int mask;
    const int32_t *idx = nullptr;
    const int32_t *perm = nullptr;
};

// ---------------------------------------------------------------------------
// Persistent evaluation.  One launch of k_ks_persist runs a whole evaluation
// (Algorithm 1's HE-Mults, Algorithm 4's totalSum rotations and masked sums
// of every chunk of every SpMV in it) as a program of phases: a phase is one
// stage of one key switch (over n ciphertexts) or the masked accumulation of
// one partition, cut into tiles of one CTA's work.  Tiles are numbered phase
// by phase; CTAs take the next tile from one global counter, wait until the
// phases it depends on have finished all their tiles, run it, and count it
// done.  Dependencies point to earlier phases only, so the lowest unfinished
// tile is always held by a running CTA whose inputs are complete: the
// program cannot deadlock, whatever the number of resident CTAs.  Every wait
// is bounded in time (PProg::wait_ns); one that runs out records
// kErrSchedTimeout in the device error word and makes every CTA stop.
enum PhaseKind : int32_t {
    kPhIntt = 1,     // inverse row pass of the input (HE-Mult: a1 * b1)
    kPhModUp = 2,    // inverse column pass, base conversion, forward column pass
    kPhRowsFwd = 3,  // forward row pass of the raised limbs (own primes skipped)
    kPhMac = 4,      // inner product with the key (plus the output addend)
    kPhInttP = 5,    // inverse row pass of the special-prime limbs
    kPhModDown = 6,  // ModDown conversion with its column passes
    kPhFinal = 7,    // forward row pass of delta, (acc - delta) * P^-1 (+ post)
    kPhMask = 8,     // masked accumulation of one partition (Algorithm 4)
    kPhNone = 9,     // no work (self-test programs)
};

struct PPhase {
    int32_t kind, inst;  // inst: index into PProg::inst (key switches) or ::mask
    int32_t gx, tiles;   // tile (bx, by) = (i % gx, i / gx)
    int32_t dep0, ndep;  // PProg::deps[dep0 .. dep0 + ndep)
};

// One key switch of n items: the arguments of the staged launches, and its
// scratch [z | ext | acc | dh] as in the staged form.
struct PInst {
    KsSrc s;
    KsAdd ad;
    const uint64_t *key;
    uint64_t *out;
    const int32_t *oidx;
    const uint64_t *post;  // added to the result when given
    uint64_t *scratch;
    int32_t n, pad;
};

// out = sum_k terms[k] * masks[k] (Montgomery-form masks), one ciphertext
struct PMask {
    const uint64_t *const *terms;
    const uint64_t *const *masks;
    uint64_t *out;
    int32_t nterms, pad;
};

struct PProg {
    const PPhase *ph;
    const int32_t *off;   // [nph + 1]: first tile of each phase
    const uint64_t *info; // [total]: tile -> phase << 32 | tile within the phase
    const int32_t *deps;
    const PInst *inst;
    const PMask *mask;
    uint32_t *ctr;        // [nph] finished tiles per phase, then the next tile, then the stop flag
    int32_t nph, total;
    int64_t wait_ns;
};

constexpr int kMaskTileWords = 2048;  // output words per masked-accumulation tile
constexpr int kErrSchedTimeout = 3;  // device error word: a dependency wait of the persistent kernel ran out

}  // namespace hespmv
