"""Scheme parameters of the oracle (TEST INFRASTRUCTURE ONLY).

The paper fixes a BFV parameter set for its CPU experiments (Section 5:
N = 8192, t = 65537, log2 Q = 200, relinearisation keys and power-of-two
rotation keys) and otherwise leaves the RNS layout to the HE library.  The
readings used here:

* ciphertext primes: q = k*2N + 1, taken in descending order from the largest
  such value below 2^bits, keeping those that are prime; the first L primes
  form Q, the next K form the special modulus P;
* psi_i: the smallest primitive 2N-th root of unity modulo q_i;
* hybrid key switching with dnum digits of alpha = ceil(L / dnum) primes,
  digit j holding the Q primes [j*alpha, min(L, (j+1)*alpha)).

Everything here is plain Python integer arithmetic.
"""
from dataclasses import dataclass, field
from typing import List

_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin (exact for n < 3.3e24 with these bases)."""
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def ntt_primes(N: int, bits: int, count: int) -> List[int]:
    """The `count` largest primes q < 2^bits with q = 1 mod 2N, descending."""
    m = 2 * N
    q = ((2 ** bits - 2) // m) * m + 1
    out = []
    while len(out) < count:
        if q < m:
            raise ValueError("ran out of candidates")
        if is_prime(q):
            out.append(q)
        q -= m
    return out


def plain_modulus(N: int, lower: int) -> int:
    """Smallest prime t >= lower with t = 1 mod 2N (batching-friendly)."""
    m = 2 * N
    t = ((lower - 1 + m - 1) // m) * m + 1
    while not is_prime(t):
        t += m
    return t


def min_primitive_root_2n(q: int, N: int) -> int:
    """Smallest primitive 2N-th root of unity modulo prime q (q = 1 mod 2N).

    A quadratic non-residue g gives one primitive root g^((q-1)/2N); every
    primitive 2N-th root is an odd power of it, and the minimum is taken.
    """
    assert (q - 1) % (2 * N) == 0
    g = 2
    while pow(g, (q - 1) // 2, q) != q - 1:
        g += 1
    r = pow(g, (q - 1) // (2 * N), q)
    r2 = r * r % q
    best, cur = r, r
    for _ in range(N - 1):
        cur = cur * r2 % q
        if cur < best:
            best = cur
    return best


def bitrev(x: int, bits: int) -> int:
    r = 0
    for _ in range(bits):
        r = (r << 1) | (x & 1)
        x >>= 1
    return r


@dataclass
class Params:
    """An RNS parameter set (Q primes, P primes, digits, plaintext t).

    scheme "bgv": integer slots mod t.  scheme "ckks": real slots at scale
    2^scale_bits; t is then 1 in every formula (keys, encryption, ModDown),
    which turns the BGV error terms t*e into e and the key-switching
    correction into the plain ModDown of CKKS."""
    log2n: int
    L: int
    K: int
    dnum: int
    t: int
    bits: int = 50
    slots: int = 0          # chunk capacity s; 0 means N/2
    q: List[int] = field(default_factory=list)   # L + K moduli, Q first
    psi: List[int] = field(default_factory=list)
    zeta: int = 0           # primitive 2N-th root mod t
    scheme: str = "bgv"
    scale_bits: int = 40    # CKKS: matrix and vector scale
    mask_scale_bits: int = 30  # CKKS: scale of the 0/1 masks

    def __post_init__(self):
        N = self.N
        if self.slots == 0:
            self.slots = N // 2
        assert 1 <= self.slots <= N // 2
        if self.scheme == "ckks":
            self.t = 1
            self.zeta = 1
        else:
            assert self.scheme in ("bgv", "bfv")
            assert (self.t - 1) % (2 * N) == 0 and is_prime(self.t)
        self.alpha = -(-self.L // self.dnum)
        assert -(-self.L // self.alpha) == self.dnum, "every digit must be non-empty"
        # CKKS adds the key-switching noise (about N * Q_j / P) to the message
        # itself, so P must cover a digit: K >= alpha primes of equal size
        assert self.scheme != "ckks" or self.K >= self.alpha, "CKKS needs K >= alpha"
        # BFV holds the message at Q/t: the same holds for its key switches
        assert self.scheme != "bfv" or self.K >= self.alpha, "BFV needs K >= alpha"
        if not self.q:
            self.q = ntt_primes(N, self.bits, self.L + self.K)
        if not self.psi:
            self.psi = [min_primitive_root_2n(q, N) for q in self.q]
        if not self.zeta:
            self.zeta = min_primitive_root_2n(self.t, N)

    @property
    def N(self) -> int:
        return 1 << self.log2n

    @property
    def t_ks(self) -> int:
        """The t of the key, encryption and key-switching formulas: t for
        BGV (errors t*e, ModDown with the t-correction), 1 for BFV and CKKS."""
        return self.t if self.scheme == "bgv" else 1

    @property
    def Q(self) -> int:
        r = 1
        for q in self.q[:self.L]:
            r *= q
        return r

    @property
    def P(self) -> int:
        r = 1
        for p in self.q[self.L:]:
            r *= p
        return r

    def digit(self, j: int) -> List[int]:
        """Indices of the Q primes in key-switching digit j."""
        return list(range(j * self.alpha, min(self.L, (j + 1) * self.alpha)))

    def ntt_index(self, e: int) -> int:
        """NTT position i holding the evaluation at psi^e (e odd, mod 2N)."""
        e %= 2 * self.N
        assert e % 2 == 1
        return bitrev((e - 1) // 2, self.log2n)

    def slot_index(self, row: int, j: int) -> int:
        """NTT position of batching slot j of row 0 or 1.

        Slot j of row 0 is the evaluation at zeta^(5^j), of row 1 at
        zeta^(-5^j) (rotation by k maps slot j+k to slot j in each row).
        """
        e = pow(5, j, 2 * self.N)
        if row == 1:
            e = 2 * self.N - e
        return self.ntt_index(e)
