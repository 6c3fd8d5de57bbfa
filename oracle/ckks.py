"""CKKS variant of the oracle (TEST INFRASTRUCTURE ONLY).

The paper evaluates with BFV and names CKKS (approximate arithmetic over real
numbers; Cheon, Kim, Kim and Song 2017, cited in Section 2) as an alternative
scheme in its conclusions (Section 6).  The SpMV is the same circuit; only the
plaintext encoding changes.  Ciphertext arithmetic here is the oracle's RNS
scheme with t = 1 (Params(scheme="ckks")): keys b = -a s + e + g s',
encryption (u pk0 + e0 + m, u pk1 + e1), and key switching ends with the plain
ModDown out = (x - Conv_{P->Q}([x]_P)) * P^-1.

Encoding (the inverse canonical embedding, restricted to real slot values):
slot j < N/2 is the evaluation at zeta^(5^j), zeta = exp(i pi / N); a real
slot vector z at scale Delta is the integer polynomial

    m_k = round(Delta * (2/N) * sum_j z_j * cos(pi * k * 5^j / N)),

rounded half away from zero.  The sum is taken with numpy's FFT (fp64) and
every coefficient whose fp64 value lies within 2^-6 of a rounding boundary
is recomputed from the sum itself: exact products z_j * cos (cosines to 40
digits) summed by math.fsum, so the result is the exact rounding.  Decoding evaluates the centred coefficients at
zeta^(5^j) (fp64 FFT) and divides by the scale.  The SpMV does not rescale:
every ciphertext keeps all L primes and the scales multiply (matrix x vector
x mask), so a SpMV result carries scale 2^(2 scale_bits + mask_scale_bits).
`rescale` (division by the last prime, rounded) is the primitive a deeper
circuit, or a smaller result to send back, would use.
"""
import math
from fractions import Fraction

import mpmath
import numpy as np

from . import native
from .bgv import Oracle, _addm
from .params import Params

# fp64 FFT error on a coefficient stays far below this at the sizes used
# (N <= 2^15, scale <= 2^40, |z| <= 2^7); coefficients whose fp64 value is
# closer than this to a rounding boundary are recomputed exactly
_TIE_WINDOW = 2.0 ** -6
_COS = {}


def slot_exponents(N: int, n: int):
    """5^j mod 2N for j < n."""
    out, e = [], 1
    for _ in range(n):
        out.append(e)
        e = e * 5 % (2 * N)
    return out


def _cos_table(N: int):
    """cos(pi i / N), i < 2N, as (hi, lo) float64 pairs (40-digit mpmath)."""
    if N not in _COS:
        mpmath.mp.dps = 40
        hi = np.empty(2 * N)
        lo = np.empty(2 * N)
        for i in range(2 * N):
            c = mpmath.cos(mpmath.pi * i / N)
            hi[i] = float(c)
            lo[i] = float(c - mpmath.mpf(hi[i]))
        _COS[N] = (hi, lo)
    return _COS[N]


def _split(x):
    t = 134217729.0 * x          # 2^27 + 1 (Dekker)
    h = t - (t - x)
    return h, x - h


def _two_prod(a, b):
    """a * b = p + e exactly, elementwise (Dekker's product)."""
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def _round_half_away(v: Fraction) -> int:
    a = abs(v)
    r = math.floor(a + Fraction(1, 2))
    return r if v >= 0 else -r


def exact_coefficient(z, ex, k: int, N: int, scale_bits: int, guess: int) -> int:
    """m_k from the defining sum: products z_j * cos as exact float pairs,
    summed with math.fsum relative to the integer `guess` (so the fractional
    part keeps its full precision), then rounded half away from zero."""
    hi, lo = _cos_table(N)
    idx = (k * ex) % (2 * N)
    p, e = _two_prod(z, hi[idx])
    t = z * lo[idx]
    f = 2.0 ** (scale_bits + 1) / N     # a power of two: exact scaling
    d = math.fsum(np.concatenate([p * f, e * f, t * f, [-float(guess)]]))
    return _round_half_away(Fraction(guess) + Fraction(d))


def encode(z, N: int, scale_bits: int, exact_all: bool = False):
    """Real slot values z (len <= N/2) -> N integer coefficients (Python ints)."""
    z = np.asarray(z, dtype=np.float64)
    n = len(z)
    assert n <= N // 2
    ex = np.array(slot_exponents(N, n), dtype=np.int64)
    Z = np.zeros(2 * N, dtype=np.complex128)
    Z[ex] = z
    F = np.fft.fft(Z)                      # F[k] = sum_j z_j exp(-i pi k e_j / N)
    approx = F.real[:N] * (2.0 / N) * float(2 ** scale_bits)
    assert np.max(np.abs(approx), initial=0.0) < 2.0 ** 50, "coefficients beyond 2^50"
    out = []
    for k in range(N):
        v = float(approx[k])
        frac = abs(v) - math.floor(abs(v))
        if exact_all or abs(frac - 0.5) < _TIE_WINDOW:
            out.append(exact_coefficient(z, ex, k, N, scale_bits, int(round(v))))
        else:
            out.append(int(math.copysign(math.floor(abs(v) + 0.5), v)))
    return out


def decode(coef, N: int, n: int, scale: float):
    """Centred integer coefficients -> the first n real slot values / scale."""
    A = np.zeros(2 * N, dtype=np.float64)
    A[:N] = [float(c) for c in coef]
    G = np.fft.ifft(A) * (2 * N)           # G[e] = sum_k m_k exp(+i pi k e / N)
    ex = slot_exponents(N, n)
    return np.array([G[e].real for e in ex]) / scale


class CkksOracle(Oracle):
    """The oracle's scheme with t = 1 and CKKS encoding."""

    def __init__(self, params: Params):
        assert params.scheme == "ckks"
        super().__init__(params)

    @property
    def delta_bits(self):
        return self.p.scale_bits

    def encode(self, row0, row1=None, scale_bits=None):
        assert row1 is None
        return encode(row0, self.p.N, self.p.scale_bits if scale_bits is None else scale_bits)

    def lift(self, m_coef):
        """Signed integer coefficients -> NTT over Q."""
        return self.ntt_signed(m_coef, range(self.p.L))

    def plaintext_ntt(self, row0, row1=None):
        """Masks: 0/1 slots at the mask scale."""
        return self.lift(self.encode(row0, row1, self.p.mask_scale_bits))

    def decrypt(self, ct):
        return self.decrypt_centered(ct)

    def decode_ct(self, ct, n, scale_bits_total):
        return decode(self.decrypt_centered(ct), self.p.N, n, float(2 ** scale_bits_total))

    def rescale(self, ct):
        """Rescaling (the RNS form of dividing by the last prime; Cheon, Han,
        Kim, Kim and Song 2018): a ciphertext over q_0..q_{l-1} (NTT domain,
        l limbs) -> one over q_0..q_{l-2}, each component c replaced by
        (c - r) / q_{l-1} with r the centred remainder of c mod q_{l-1}
        (so the quotient is c / q_{l-1} rounded to nearest).  Limb-wise:
        r is the last limb in coefficient form, centred, lifted to q_i and
        transformed; c'_i = (c_i - r_i) * q_{l-1}^-1 mod q_i.  The plaintext
        and the scale are divided by q_{l-1}.  (The SpMV circuit needs no
        rescaling; this is the primitive a deeper circuit would use.)"""
        p = self.p
        nl = ct.shape[1]
        assert nl >= 2
        ql = p.q[nl - 1]
        out = np.zeros((ct.shape[0], nl - 1, p.N), dtype=np.uint64)
        for c in range(ct.shape[0]):
            x = self.intt(ct[c, nl - 1], nl - 1)
            r = [int(v) - ql if int(v) > ql // 2 else int(v) for v in x]
            for i in range(nl - 1):
                qi = p.q[i]
                ri = self.ntt(np.array([v % qi for v in r], dtype=np.uint64), i)
                inv = pow(ql, qi - 2, qi)
                diff = [(int(a) - int(b)) % qi for a, b in zip(ct[c, i], ri)]
                out[c, i] = np.array([d * inv % qi for d in diff], dtype=np.uint64)
        return out

    def decrypt_level(self, ct):
        """[c0 + c1 s] over the first l = ct.shape[1] primes, centred, as
        Python integers (the decryption of a rescaled ciphertext)."""
        p = self.p
        nl = ct.shape[1]
        x = [self.intt(_addm(ct[0, l], native.mulmod(ct[1, l], self.s[l], p.q[l]), p.q[l]), l)
             for l in range(nl)]
        Q = 1
        for l in range(nl):
            Q *= p.q[l]
        out = []
        for k in range(p.N):
            v = 0
            for l in range(nl):
                Qh = Q // p.q[l]
                v += int(x[l][k]) * (Qh * pow(Qh, -1, p.q[l]) % Q)
            v %= Q
            out.append(v - Q if v > Q // 2 else v)
        return out
