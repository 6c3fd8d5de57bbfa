"""Pins of the oracle's arithmetic against definitions it does not use itself:
O(N^2) transform definition, schoolbook negacyclic convolution, a library
primality test, brute-force root search, direct evaluation at the batching
roots, big-integer CRT, and published generator outputs."""
import json
import os
import random

import numpy as np
import pytest
import sympy

from oracle import native, rng
from oracle.bgv import Oracle
from oracle.params import (Params, bitrev, is_prime, min_primitive_root_2n, ntt_primes,
                           plain_modulus)
from paper_2603_04742_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def ntt_definition(a, q, psi, logn):
    N = 1 << logn
    return [sum(a[j] * pow(psi, (2 * bitrev(i, logn) + 1) * j, q) for j in range(N)) % q
            for i in range(N)]


def negacyclic_schoolbook(a, b, q):
    N = len(a)
    out = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            if k < N:
                out[k] += a[i] * b[j]
            else:
                out[k - N] -= a[i] * b[j]
    return [x % q for x in out]


@pytest.mark.parametrize("logn,bits", [(3, 20), (4, 50), (6, 50), (7, 40)])
def test_ntt_matches_definition(logn, bits):
    N = 1 << logn
    q = ntt_primes(N, bits, 1)[0]
    psi = min_primitive_root_2n(q, N)
    r = random.Random(logn)
    a = [r.randrange(q) for _ in range(N)]
    assert [int(v) for v in native.ntt(np.array(a, dtype=np.uint64), q, psi)] == \
        ntt_definition(a, q, psi, logn)


@pytest.mark.parametrize("logn", [4, 5, 8])
def test_ntt_convolution_and_roundtrip(logn):
    N = 1 << logn
    q = ntt_primes(N, 50, 2)[1]
    psi = min_primitive_root_2n(q, N)
    r = random.Random(100 + logn)
    a = [r.randrange(q) for _ in range(N)]
    b = [r.randrange(q) for _ in range(N)]
    A = native.ntt(np.array(a, dtype=np.uint64), q, psi)
    B = native.ntt(np.array(b, dtype=np.uint64), q, psi)
    c = native.intt(native.mulmod(A, B, q), q, psi)
    assert [int(v) for v in c] == negacyclic_schoolbook(a, b, q)
    assert [int(v) for v in native.intt(A, q, psi)] == a


def test_mulmod_exact():
    r = random.Random(3)
    q = ntt_primes(1 << 12, 50, 1)[0]
    a = [r.randrange(1 << 64) for _ in range(200)]
    b = [r.randrange(1 << 64) for _ in range(200)]
    got = native.mulmod(np.array(a, dtype=np.uint64), np.array(b, dtype=np.uint64), q)
    assert [int(v) for v in got] == [x * y % q for x, y in zip(a, b)]
    s = r.randrange(1 << 64)
    got = native.mulmod_scalar(np.array(a, dtype=np.uint64), s, q)
    assert [int(v) for v in got] == [x * s % q for x in a]


def test_is_prime_matches_library():
    r = random.Random(5)
    cands = [r.randrange(1 << 50) | 1 for _ in range(300)] + list(range(2, 500))
    cands += [1125899906826241, 1125899906826241 + 2 * 4096]
    for n in cands:
        assert is_prime(n) == sympy.isprime(n), n


@pytest.mark.parametrize("logn,count", [(12, 4), (14, 6), (15, 10), (5, 3)])
def test_ntt_primes_are_the_largest(logn, count):
    N = 1 << logn
    got = ntt_primes(N, 50, count)
    # independent scan with the library primality test
    want, q = [], (1 << 50) - 1
    while q % (2 * N) != 1:
        q -= 1
    while len(want) < count:
        if sympy.isprime(q):
            want.append(q)
        q -= 2 * N
    assert got == want
    assert all(x < (1 << 50) and x % (2 * N) == 1 for x in got)


def test_plain_moduli_of_the_configs():
    for name, (logn, L, K, dnum, t) in synth.RING.items():
        N = 1 << logn
        assert sympy.isprime(t) and t % (2 * N) == 1
    # smallest such primes above the stated bounds (c1 is the paper's 65537)
    lows = {"c2": 2 ** 24, "c3": 2 ** 40, "c4": 2 ** 20, "c5": 2 ** 20}
    for name, lo in lows.items():
        logn, t = synth.RING[name][0], synth.RING[name][4]
        N = 1 << logn
        assert plain_modulus(N, lo) == t
        assert sympy.nextprime(lo - 1) <= t
        assert all(not sympy.isprime(x) for x in range(lo + (1 - lo) % (2 * N), t, 2 * N)
                   if x >= lo)
    assert synth.RING["c1"][4] == 65537 and 65536 % (2 << 12) == 0


@pytest.mark.parametrize("q,N", [(17, 4), (97, 16), (257, 64), (7681, 256), (12289, 512)])
def test_min_primitive_root_bruteforce(q, N):
    want = min(x for x in range(2, q) if pow(x, N, q) == q - 1)
    assert min_primitive_root_2n(q, N) == want


def test_primitive_root_property_large():
    N = 1 << 15
    for q in ntt_primes(N, 50, 3):
        psi = min_primitive_root_2n(q, N)
        assert pow(psi, N, q) == q - 1


def test_splitmix64_reference_outputs():
    g = json.load(open(os.path.join(GOLD, "splitmix64_seed1234567.json")))
    outs = [rng.splitmix_output(g["seed"], i) for i in range(len(g["outputs"]))]
    assert outs == [int(x) for x in g["outputs"]]
    # the vectorised draw path agrees with the scalar definition
    key = rng.stream_key(99, 7)
    d = rng.draws(99, 7, 5, 4)
    assert [int(x) for x in d] == [rng.splitmix_output(key, 5 + i) for i in range(4)]


def test_samplers_statistics():
    n = 1 << 16
    s = rng.ternary(1, 2, n)
    assert set(np.unique(s)) == {-1, 0, 1}
    for v in (-1, 0, 1):
        assert abs(np.mean(s == v) - 1 / 3) < 0.01
    e = rng.cbd21(1, 3, n)
    assert e.min() >= -21 and e.max() <= 21
    assert abs(e.mean()) < 0.05 and abs(e.var() - 10.5) < 0.3
    q = ntt_primes(1 << 12, 50, 1)[0]
    u = rng.uniform_limbs(1, 4, [q], 1 << 14)[0]
    assert int(u.max()) < q
    assert abs(float(u.astype(np.float64).mean()) / q - 0.5) < 0.01
    # the residue is the 128-bit value (hi, lo) reduced mod q
    d = rng.draws(1, 4, 0, 2)
    assert int(u[0]) == ((int(d[0]) << 64) + int(d[1])) % q


def test_encoding_matches_root_evaluation():
    p = Params(log2n=5, L=1, K=1, dnum=1, t=193)   # 193 = 6*32 + 1
    orc = Oracle(p)
    r = random.Random(9)
    row0 = [r.randrange(p.t) for _ in range(p.N // 2)]
    row1 = [r.randrange(p.t) for _ in range(p.N // 2)]
    m = [int(v) for v in orc.encode(row0, row1)]
    z = p.zeta
    for j in range(p.N // 2):
        e = pow(5, j, 2 * p.N)
        ev0 = sum(m[k] * pow(z, e * k, p.t) for k in range(p.N)) % p.t
        ev1 = sum(m[k] * pow(z, (2 * p.N - e) * k, p.t) for k in range(p.N)) % p.t
        assert ev0 == row0[j] and ev1 == row1[j]
    d0, d1 = orc.decode(np.array(m, dtype=np.uint64))
    assert [int(v) for v in d0] == row0 and [int(v) for v in d1] == row1


def test_automorphism_permutation_matches_coefficient_map():
    p = Params(log2n=6, L=1, K=1, dnum=1, t=257)
    orc = Oracle(p)
    q, psi, N = p.q[0], p.psi[0], p.N
    r = random.Random(4)
    a = [r.randrange(q) for _ in range(N)]
    for g in (5, 25, 2 * N - 1, 3):
        # sigma_g(a)(X) = a(X^g): coefficient j goes to j*g mod 2N, sign flips past N
        b = [0] * N
        for j in range(N):
            k = j * g % (2 * N)
            if k < N:
                b[k] = (b[k] + a[j]) % q
            else:
                b[k - N] = (b[k - N] - a[j]) % q
        A = native.ntt(np.array(a, dtype=np.uint64), q, psi)
        B = native.ntt(np.array(b, dtype=np.uint64), q, psi)
        perm = orc.automorphism_perm(g)
        assert np.array_equal(A[perm], B)


@pytest.mark.parametrize("L,K,dnum", [(3, 1, 3), (8, 2, 4), (5, 2, 2)])
def test_base_conversion_crt(L, K, dnum):
    p = Params(log2n=4, L=L, K=K, dnum=dnum, t=97)
    orc = Oracle(p)
    r = random.Random(L * 10 + K)
    for j in range(p.dnum):
        Dj = p.digit(j)
        S = 1
        for i in Dj:
            S *= p.q[i]
        x = [r.randrange(S) for _ in range(p.N)]
        x_coef = np.array([[v % p.q[i] for v in x] for i in Dj], dtype=np.uint64)
        dst = [l for l in range(L + K) if l not in Dj]
        y = orc.base_convert(x_coef, Dj, dst)
        for c in range(p.N):
            # some u in [0, |Dj|) makes x + u*S agree on every target prime
            ok = [u for u in range(len(Dj))
                  if all(int(y[m, c]) == (x[c] + u * S) % p.q[l] for m, l in enumerate(dst))]
            assert ok, (j, c)


def test_gadget_residues():
    p = Params(log2n=4, L=8, K=2, dnum=4, t=97)
    orc = Oracle(p)
    for j in range(p.dnum):
        for l in range(p.L + p.K):
            want = (p.P % p.q[l]) if (l < p.L and l in p.digit(j)) else 0
            assert orc.gadget_residue(j, l) == want
