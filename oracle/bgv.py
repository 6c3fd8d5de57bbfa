"""BGV-RNS scheme of the oracle (TEST INFRASTRUCTURE ONLY).

The paper evaluates its SpMV with Pyfhel/BFV (Section 5) and uses four HE
operations (Section 2.1): HE-Add, HE-Mult (ciphertext x ciphertext, followed
by relinearisation), HE-CMult (ciphertext x plaintext) and HE-Rot (left
rotation of the slot vector).  This oracle realises them in BGV over an RNS
basis with the same plaintext space Z_t[X]/(X^N+1) and the same batching
slots, so every decryption equals BFV's.  Readings (the paper is silent):

* secret key uniform ternary, errors centred binomial with eta = 21;
* public-key encryption ct = (u*pk0 + t*e0 + m, u*pk1 + t*e1);
* hybrid key switching: digit j of ciphertext polynomial d is raised from its
  alpha primes to all L+K primes by fast base conversion with unsigned
  representatives, multiplied with key digit j, summed over digits, and
  brought back to Q by dividing by P with the BGV correction
  delta = t * Conv_{P->Q}([x * t^-1]_P), out = (x - delta) * P^-1;
* key digit j: b_j = -a_j s + t e_j + g_j s',  a_j uniform over Q u P, with
  g_j = P * (Q/Q_j) * [(Q/Q_j)^-1 mod Q_j] (so g_j = P mod q_i on the
  primes of digit j and 0 elsewhere);
* rotation by k uses the Galois element 5^k mod 2N; with power-of-two keys a
  rotation by k is a chain over the set bits of k, least significant first.

Polynomials are numpy uint64 arrays of shape (limbs, N) in the NTT domain
unless the name says `coef`.  Ciphertexts are arrays of shape (2, L, N).
"""
import numpy as np

from . import native, rng
from .params import Params, bitrev


def _inv(a: int, q: int) -> int:
    return pow(a % q, -1, q)


def _addm(a, b, q):
    return (a + b) % np.uint64(q)


def _subm(a, b, q):
    return (a + np.uint64(q) - b) % np.uint64(q)


class Oracle:
    def __init__(self, params: Params):
        self.p = params
        N = params.N
        # NTT positions of the N/2 slots of each row
        e = 1
        idx0, idx1 = [], []
        for _ in range(N // 2):
            idx0.append(params.ntt_index(e))
            idx1.append(params.ntt_index(2 * N - e))
            e = e * 5 % (2 * N)
        self.slot_idx0 = np.array(idx0, dtype=np.int64)
        self.slot_idx1 = np.array(idx1, dtype=np.int64)
        self.counts = {}

    # ------------------------------------------------------------- helpers
    def _count(self, name, k=1):
        self.counts[name] = self.counts.get(name, 0) + k

    def ntt(self, coef, l):
        return native.ntt(coef, self.p.q[l], self.p.psi[l])

    def intt(self, a, l):
        return native.intt(a, self.p.q[l], self.p.psi[l])

    def limbs_from_signed(self, c, limbs):
        """Signed integer coefficients -> residues on the given limbs (coef)."""
        c = np.asarray(c, dtype=object)
        return np.array([(c % self.p.q[l]).astype(np.uint64) for l in limbs],
                        dtype=np.uint64).reshape(len(limbs), -1)

    def ntt_signed(self, c, limbs):
        coef = self.limbs_from_signed(c, limbs)
        return np.array([self.ntt(coef[k], l) for k, l in enumerate(limbs)])

    def automorphism_perm(self, g):
        """perm[i] with (sigma_g a)_ntt[i] = a_ntt[perm[i]], sigma_g: X -> X^g."""
        p = self.p
        N = p.N
        perm = np.empty(N, dtype=np.int64)
        for i in range(N):
            e = (2 * bitrev(i, p.log2n) + 1) * g % (2 * N)
            perm[i] = p.ntt_index(e)
        return perm

    # ------------------------------------------------------------ encoding
    def encode(self, row0, row1=None):
        """Batch encoding: slot values (integers, any sign) -> m coef mod t."""
        p = self.p
        t = p.t
        E = np.zeros(p.N, dtype=np.uint64)
        r0 = np.asarray(row0, dtype=object) % t
        E[self.slot_idx0[:len(r0)]] = r0.astype(np.uint64)
        if row1 is not None:
            r1 = np.asarray(row1, dtype=object) % t
            E[self.slot_idx1[:len(r1)]] = r1.astype(np.uint64)
        return native.intt(E, t, p.zeta)

    def decode(self, m_coef):
        """m coef mod t -> (row0 slots, row1 slots) in [0, t)."""
        p = self.p
        E = native.ntt(m_coef, p.t, p.zeta)
        return E[self.slot_idx0], E[self.slot_idx1]

    def lift(self, m_coef):
        """Plaintext coef in [0,t) -> centred integers -> NTT over Q."""
        t = self.p.t
        c = np.asarray(m_coef, dtype=object)
        c = np.where(2 * c <= t, c, c - t)
        return self.ntt_signed(c, range(self.p.L))

    def plaintext_ntt(self, row0, row1=None):
        return self.lift(self.encode(row0, row1))

    # -------------------------------------------------------------- keygen
    def keygen(self, seed, galois_elements=()):
        p = self.p
        N, L, K, t = p.N, p.L, p.K, p.t_ks
        all_limbs = range(L + K)
        s = rng.ternary(seed, rng.S_SECRET, N)
        self.s_coef = s
        self.s = self.ntt_signed(s, all_limbs)           # over Q u P
        a = rng.uniform_limbs(seed, rng.S_PK_A, p.q[:L], N)
        e = self.ntt_signed(rng.cbd21(seed, rng.S_PK_E, N), range(L))
        pk0 = np.empty_like(a)
        for l in range(L):
            q = p.q[l]
            pk0[l] = _addm(_subm(np.zeros(N, np.uint64), native.mulmod(a[l], self.s[l], q), q),
                           native.mulmod_scalar(e[l], t, q), q)
        self.pk = (pk0, a)
        s2 = np.array([native.mulmod(self.s[l], self.s[l], p.q[l]) for l in all_limbs])
        self.rlk = self.make_ksk(seed, 0, s2)
        self.gk = {}
        for g in galois_elements:
            perm = self.automorphism_perm(g)
            self.gk[g] = self.make_ksk(seed, g, self.s[:, perm])

    def gadget_residue(self, j, l):
        """g_j mod q_l for g_j = P * (Q/Q_j) * [(Q/Q_j)^-1]_{Q_j}."""
        p = self.p
        Qj = 1
        for i in p.digit(j):
            Qj *= p.q[i]
        Qt = p.Q // Qj
        g = p.P * Qt * _inv(Qt, Qj)
        return g % p.q[l]

    def make_ksk(self, seed, kid, sp):
        """Key switching key from s' (NTT over Q u P) to s: [dnum][2][L+K][N]."""
        p = self.p
        N, L, K, t = p.N, p.L, p.K, p.t_ks
        key = np.empty((p.dnum, 2, L + K, N), dtype=np.uint64)
        for j in range(p.dnum):
            a = rng.uniform_limbs(seed, rng.ksk_a_stream(kid, j), p.q, N)
            e = self.ntt_signed(rng.cbd21(seed, rng.ksk_e_stream(kid, j), N), range(L + K))
            for l in range(L + K):
                q = p.q[l]
                b = _subm(native.mulmod_scalar(e[l], t, q), native.mulmod(a[l], self.s[l], q), q)
                b = _addm(b, native.mulmod_scalar(sp[l], self.gadget_residue(j, l), q), q)
                key[j, 0, l] = b
                key[j, 1, l] = a[l]
        return key

    # ------------------------------------------------- encryption/decryption
    def encrypt(self, m_coef, seed, ct_index):
        p = self.p
        N, L, t = p.N, p.L, p.t_ks
        u = self.ntt_signed(rng.ternary(seed, rng.enc_stream(ct_index, 1), N), range(L))
        e0 = self.ntt_signed(rng.cbd21(seed, rng.enc_stream(ct_index, 2), N), range(L))
        e1 = self.ntt_signed(rng.cbd21(seed, rng.enc_stream(ct_index, 3), N), range(L))
        m = self.lift(m_coef)
        ct = np.empty((2, L, N), dtype=np.uint64)
        for l in range(L):
            q = p.q[l]
            ct[0, l] = _addm(_addm(native.mulmod(u[l], self.pk[0][l], q),
                                   native.mulmod_scalar(e0[l], t, q), q), m[l], q)
            ct[1, l] = _addm(native.mulmod(u[l], self.pk[1][l], q),
                             native.mulmod_scalar(e1[l], t, q), q)
        return ct

    def decrypt_centered(self, ct):
        """[c0 + c1 s]_Q as centred Python integers (one per coefficient)."""
        p = self.p
        L = p.L
        x = [self.intt(_addm(ct[0, l], native.mulmod(ct[1, l], self.s[l], p.q[l]), p.q[l]), l)
             for l in range(L)]
        Q = p.Q
        terms = []
        for l in range(L):
            Qh = Q // p.q[l]
            terms.append((Qh * _inv(Qh, p.q[l])) % Q)
        out = []
        cols = [xl.tolist() for xl in x]
        for c in range(p.N):
            v = 0
            for l in range(L):
                v += cols[l][c] * terms[l]
            v %= Q
            if 2 * v >= Q:
                v -= Q
            out.append(v)
        return out

    def decrypt(self, ct):
        """-> plaintext coef in [0, t)."""
        t = self.p.t
        return np.array([v % t for v in self.decrypt_centered(ct)], dtype=np.uint64)

    def noise_bits(self, ct):
        """log2 of the largest |[c0 + c1 s]_Q| (must stay below log2(Q/2))."""
        m = max(abs(v) for v in self.decrypt_centered(ct))
        return m.bit_length()

    # ------------------------------------------------------------ HE ops
    def add(self, a, b):
        self._count("add")
        out = np.empty_like(a)
        for c in range(a.shape[0]):
            for l in range(self.p.L):
                out[c, l] = _addm(a[c, l], b[c, l], self.p.q[l])
        return out

    def tensor(self, a, b):
        """(d0, d1, d2) = (a0 b0, a0 b1 + a1 b0, a1 b1), limb by limb."""
        p = self.p
        d = np.empty((3, p.L, p.N), dtype=np.uint64)
        for l in range(p.L):
            q = p.q[l]
            d[0, l] = native.mulmod(a[0, l], b[0, l], q)
            d[1, l] = _addm(native.mulmod(a[0, l], b[1, l], q), native.mulmod(a[1, l], b[0, l], q), q)
            d[2, l] = native.mulmod(a[1, l], b[1, l], q)
        return d

    def base_convert(self, x_coef, src, dst):
        """Fast base conversion of coefficient-domain residues x_coef (one row
        per prime index in `src`) to the primes in `dst`:
            y_l = sum_i [x_i * (S/s_i)^-1]_{s_i} * (S/s_i) mod q_l,
        S the product of the source primes, with the unsigned representative
        of each bracket.  The integer sum equals x + u*S for some 0 <= u < |src|.
        """
        q = self.p.q
        S = 1
        for i in src:
            S *= q[i]
        z = [native.mulmod_scalar(x_coef[k], _inv(S // q[i], q[i]), q[i])
             for k, i in enumerate(src)]
        out = np.zeros((len(dst), x_coef.shape[1]), dtype=np.uint64)
        for m, l in enumerate(dst):
            for k, i in enumerate(src):
                out[m] = _addm(out[m], native.mulmod_scalar(z[k], (S // q[i]) % q[l], q[l]), q[l])
        return out

    def keyswitch(self, d, key):
        """Hybrid key switch of d (NTT over Q) with `key` -> (ks0, ks1) over Q."""
        self._count("keyswitch")
        p = self.p
        N, L, K, t = p.N, p.L, p.K, p.t_ks
        q = p.q
        d_coef = np.array([self.intt(d[i], i) for i in range(L)])
        acc = np.zeros((2, L + K, N), dtype=np.uint64)
        for j in range(p.dnum):
            # ModUp: digit j raised from its primes to every prime of Q u P
            Dj = p.digit(j)
            others = [l for l in range(L + K) if l not in Dj]
            conv = self.base_convert(d_coef[Dj], Dj, others)
            ext = np.empty((L + K, N), dtype=np.uint64)
            for l in Dj:
                ext[l] = d[l]
            for m, l in enumerate(others):
                ext[l] = self.ntt(conv[m], l)
            # inner product with key digit j
            for c in range(2):
                for l in range(L + K):
                    acc[c, l] = _addm(acc[c, l], native.mulmod(ext[l], key[j, c, l], q[l]), q[l])
        # ModDown: divide by P with the t-correction
        Pidx = list(range(L, L + K))
        out = np.empty((2, L, N), dtype=np.uint64)
        for c in range(2):
            y = np.array([native.mulmod_scalar(self.intt(acc[c, l], l), _inv(t, q[l]), q[l])
                          for l in Pidx])
            conv = self.base_convert(y, Pidx, list(range(L)))
            for i in range(L):
                delta = self.ntt(native.mulmod_scalar(conv[i], t % q[i], q[i]), i)
                out[c, i] = native.mulmod_scalar(_subm(acc[c, i], delta, q[i]),
                                                 _inv(p.P, q[i]), q[i])
        return out

    def relinearize(self, d):
        self._count("relin")
        ks = self.keyswitch(d[2], self.rlk)
        out = np.empty((2, self.p.L, self.p.N), dtype=np.uint64)
        for l in range(self.p.L):
            q = self.p.q[l]
            out[0, l] = _addm(d[0, l], ks[0, l], q)
            out[1, l] = _addm(d[1, l], ks[1, l], q)
        return out

    def mult(self, a, b):
        """HE-Mult: tensor product followed by relinearisation."""
        self._count("mult")
        return self.relinearize(self.tensor(a, b))

    def apply_galois(self, ct, g):
        """sigma_g on both components, then key switch c1 back to s."""
        perm = self.automorphism_perm(g)
        c0 = ct[0][:, perm]
        c1 = ct[1][:, perm]
        ks = self.keyswitch(c1, self.gk[g])
        out = np.empty_like(ct)
        for l in range(self.p.L):
            q = self.p.q[l]
            out[0, l] = _addm(c0[l], ks[0, l], q)
            out[1, l] = ks[1, l]
        return out

    def rotation_elements(self, k, policy="pow2"):
        """Galois elements applied, in order, for a left rotation by k."""
        N = self.p.N
        k %= N // 2
        if k == 0:
            return []
        if policy == "exact":
            return [pow(5, k, 2 * N)]
        out = []
        b = 0
        while k >> b:
            if (k >> b) & 1:
                out.append(pow(5, 1 << b, 2 * N))
            b += 1
        return out

    def rotate(self, ct, k, policy="pow2"):
        """HE-Rot: slot j of the result holds slot j+k of the input."""
        self._count("rot")
        for g in self.rotation_elements(k, policy):
            ct = self.apply_galois(ct, g)
        return ct

    def cmult(self, ct, pt_ntt):
        """HE-CMult with a plaintext already lifted to Q in the NTT domain."""
        self._count("cmult")
        out = np.empty_like(ct)
        for c in range(2):
            for l in range(self.p.L):
                out[c, l] = native.mulmod(ct[c, l], pt_ntt[l], self.p.q[l])
        return out
