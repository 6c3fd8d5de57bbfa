"""BFV variant of the oracle (TEST INFRASTRUCTURE ONLY).

The paper's scheme (Section 5: Pyfhel/BFV, Fan and Vercauteren 2012).  Same
plaintext space and batching slots as the BGV oracle; the message sits in the
high part of the ciphertext instead of the low part:

* keys and key switching as in the BGV oracle with t = 1 in their formulas
  (errors e, plain ModDown out = (x - Conv_{P->Q}([x]_P)) * P^-1);
* encryption ct = (u pk0 + e0 + Delta [m]_t, u pk1 + e1), Delta = floor(Q/t),
  m with coefficients in [0, t);
* decryption m = [round(t [c0 + c1 s]_Q / Q)]_t;
* HE-Mult: with a, b the centred representatives in (-Q/2, Q/2] of the
  input coefficients, the products over the integers
      d0 = a0 b0,  d1 = a0 b1 + a1 b0,  d2 = a1 b1   (in Z[X]/(X^N + 1))
  are scaled and rounded, d_i' = [round(t d_i / Q)]_Q (no ties: Q is odd and
  prime to t), then relinearised;
* HE-CMult multiplies by the centred plaintext polynomial (no Delta), HE-Add
  and HE-Rot are those of the BGV oracle.

The integer products are taken exactly: residues modulo auxiliary NTT primes
(below 2^45, so none is a ciphertext prime) whose product exceeds twice the
largest possible |d_i|, multiplied in the NTT domain by the oracle's own NTT,
and recombined by Chinese remaindering with Python integers.
"""
import numpy as np

from . import native
from .bgv import Oracle
from .params import Params, min_primitive_root_2n, ntt_primes


def _crt_basis(N: int, bound_bits: int):
    """NTT primes below 2^45 (q = 1 mod 2N) whose product exceeds 2^bound_bits."""
    primes, prod = [], 1
    for q in ntt_primes(N, 45, 64):
        primes.append(q)
        prod *= q
        if prod.bit_length() > bound_bits:
            return primes, prod
    raise ValueError("auxiliary primes exhausted")


def negacyclic_z(a, b, bound_bits):
    """Exact a * b in Z[X]/(X^N + 1) for integer lists a, b whose product
    coefficients are below 2^(bound_bits - 1) in magnitude."""
    N = len(a)
    primes, P = _crt_basis(N, bound_bits)
    res = []
    for q in primes:
        psi = min_primitive_root_2n(q, N)
        aq = np.array([x % q for x in a], dtype=np.uint64)
        bq = np.array([x % q for x in b], dtype=np.uint64)
        prod = native.mulmod(native.ntt(aq, q, psi), native.ntt(bq, q, psi), q)
        res.append(native.intt(prod, q, psi).tolist())
    terms = [(P // q) * pow(P // q, -1, q) for q in primes]
    out = []
    for k in range(N):
        v = sum(r[k] * c for r, c in zip(res, terms)) % P
        out.append(v - P if 2 * v > P else v)
    return out


class BfvOracle(Oracle):
    def __init__(self, params: Params):
        assert params.scheme == "bfv"
        super().__init__(params)
        self.delta = params.Q // params.t

    def _centred_coef(self, x_ntt):
        """NTT-domain residues over Q -> centred integer coefficients."""
        p = self.p
        Q = p.Q
        cols = [self.intt(x_ntt[l], l).tolist() for l in range(p.L)]
        terms = []
        for l in range(p.L):
            Qh = Q // p.q[l]
            terms.append(Qh * pow(Qh, -1, p.q[l]) % Q)
        out = []
        for k in range(p.N):
            v = sum(cols[l][k] * terms[l] for l in range(p.L)) % Q
            out.append(v - Q if 2 * v > Q else v)
        return out

    def encrypt(self, m_coef, seed, ct_index):
        """m_coef in [0, t): Delta * m is added where BGV adds m (the noise
        terms already carry t = 1 through Params.t_ks)."""
        scaled = [int(v) * self.delta for v in np.asarray(m_coef, dtype=object)]
        zero = np.zeros(self.p.N, dtype=np.uint64)
        ct = super().encrypt(zero, seed, ct_index)       # BGV lift of 0 is 0
        dm = self.ntt_signed(scaled, range(self.p.L))
        for l in range(self.p.L):
            q = self.p.q[l]
            ct[0, l] = (ct[0, l] + dm[l]) % np.uint64(q)
        return ct

    def decrypt(self, ct):
        """-> plaintext coefficients in [0, t)."""
        p = self.p
        Q, t = p.Q, p.t
        out = []
        for v in self.decrypt_centered(ct):
            num = t * v
            r = (2 * num + Q) // (2 * Q)      # round(t v / Q), no ties (Q odd)
            out.append(r % t)
        return np.array(out, dtype=np.uint64)

    def noise_bits(self, ct):
        """log2 of the largest |v - Delta * round(t v / Q)|, v = [c0 + c1 s]_Q
        (decryption is correct while it stays below Delta / 2)."""
        Q, t = self.p.Q, self.p.t
        m = 0
        for v in self.decrypt_centered(ct):
            r = (2 * t * v + Q) // (2 * Q)
            m = max(m, abs(v - self.delta * r))
        return m.bit_length()

    def tensor(self, a, b):
        """Scaled and rounded integer tensor product, NTT domain over Q."""
        p = self.p
        Q, t, N = p.Q, p.t, p.N
        a0, a1 = self._centred_coef(a[0]), self._centred_coef(a[1])
        b0, b1 = self._centred_coef(b[0]), self._centred_coef(b[1])
        bound = 2 * (Q.bit_length() + 1) + N.bit_length() + 2
        d0 = negacyclic_z(a0, b0, bound)
        d2 = negacyclic_z(a1, b1, bound)
        d1 = [x + y for x, y in zip(negacyclic_z(a0, b1, bound), negacyclic_z(a1, b0, bound))]
        out = np.empty((3, p.L, N), dtype=np.uint64)
        for c, d in enumerate((d0, d1, d2)):
            z = [(2 * t * v + Q) // (2 * Q) for v in d]  # round(t d / Q)
            out[c] = self.ntt_signed(z, range(p.L))
        return out
