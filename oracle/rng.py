"""Counter-based randomness of the oracle (TEST INFRASTRUCTURE ONLY).

The scheme draws its secret, errors and uniform masks from SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): state s, i-th output (0-based) = mix(s + (i+1)*gamma) with
gamma = 0x9E3779B97F4A7C15 and the published 64-bit finaliser.  The GPU
library implements the same published generator in its own code.

Derivation used by the scheme (a stream is a 64-bit label):
    key(seed, stream) = SplitMix64(seed).output[stream]
    draw(seed, stream, ctr) = SplitMix64(key(seed, stream)).output[ctr]
Samplers (from one draw r each, or two for a uniform residue):
    ternary     (r mod 3) - 1
    CBD(21)     popcount(r & (2^21-1)) - popcount((r >> 21) & (2^21-1))
    uniform q   (r_hi * 2^64 + r_lo) mod q, r_hi = draw(2c), r_lo = draw(2c+1)
"""
import numpy as np

from . import native

GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK = (1 << 64) - 1

# stream labels
S_SECRET = 1
S_PK_A = 2
S_PK_E = 3
ENC_BASE = 1 << 62


def ksk_a_stream(kid: int, j: int) -> int:
    """Stream of the uniform part of digit j of key-switching key `kid`
    (kid 0 = relinearisation key, kid = g for the Galois element g)."""
    return 16 + 2 * (kid * 64 + j)


def ksk_e_stream(kid: int, j: int) -> int:
    return 16 + 2 * (kid * 64 + j) + 1


def enc_stream(ct_index: int, what: int) -> int:
    """Streams of ciphertext number ct_index: what = 1 (u), 2 (e0), 3 (e1)."""
    return ENC_BASE + 4 * ct_index + what


def _mix_int(z: int) -> int:
    z = ((z ^ (z >> 30)) * M1) & MASK
    z = ((z ^ (z >> 27)) * M2) & MASK
    return z ^ (z >> 31)


def splitmix_output(state: int, i: int) -> int:
    return _mix_int((state + (i + 1) * GAMMA) & MASK)


def stream_key(seed: int, stream: int) -> int:
    return splitmix_output(seed & MASK, stream)


def draws(seed: int, stream: int, ctr0: int, count: int) -> np.ndarray:
    """draw(seed, stream, ctr) for ctr in [ctr0, ctr0+count), as uint64."""
    key = stream_key(seed, stream)
    # exact 64-bit wrap-around arithmetic done with Python ints, vectorised
    # through an object array to keep it obviously exact
    ctr = np.arange(ctr0, ctr0 + count, dtype=object)
    z = (key + (ctr + 1) * GAMMA) % (1 << 64)
    z = ((z ^ (z >> 30)) * M1) % (1 << 64)
    z = ((z ^ (z >> 27)) * M2) % (1 << 64)
    z = z ^ (z >> 31)
    return z.astype(np.uint64)


def ternary(seed: int, stream: int, n: int) -> np.ndarray:
    r = draws(seed, stream, 0, n)
    return (r % np.uint64(3)).astype(np.int64) - 1


def cbd21(seed: int, stream: int, n: int) -> np.ndarray:
    r = draws(seed, stream, 0, n)
    lo = r & np.uint64((1 << 21) - 1)
    hi = (r >> np.uint64(21)) & np.uint64((1 << 21) - 1)
    return np.bitwise_count(lo).astype(np.int64) - np.bitwise_count(hi).astype(np.int64)


def uniform_limbs(seed: int, stream: int, moduli, N: int) -> np.ndarray:
    """Uniform residues, limb i over moduli[i]; coefficient c of limb i uses
    draws 2(i*N+c) (high word) and 2(i*N+c)+1 (low word)."""
    out = np.empty((len(moduli), N), dtype=np.uint64)
    for i, q in enumerate(moduli):
        r = draws(seed, stream, 2 * i * N, 2 * N)
        hi = r[0::2] % np.uint64(q)
        lo = r[1::2] % np.uint64(q)
        two64 = (1 << 64) % q
        v = native.mulmod_scalar(hi, two64, q)
        out[i] = (v + lo) % np.uint64(q)
    return out
