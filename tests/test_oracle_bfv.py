"""Pins of the oracle's BFV variant (CPU): the exact integer product against
schoolbook multiplication, the scale-and-round against its definition
computed directly, encryption/decryption, HE-Mult, rotation and masking on
slots, and the SpMV equal to A x."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import bfv as OB
from oracle import spmv as S
from oracle.params import Params, plain_modulus
from paper_2603_04742_gb300 import synth


def schoolbook(a, b):
    N = len(a)
    out = [0] * N
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            if i + j < N:
                out[i + j] += x * y
            else:
                out[i + j - N] -= x * y
    return out


def test_negacyclic_z_exact():
    g = np.random.default_rng(1)
    N = 16
    a = [int(v) for v in g.integers(-2 ** 60, 2 ** 60, N)]
    a = [x * 2 ** 40 + 12345 for x in a]                 # ~100-bit coefficients
    b = [int(v) * 2 ** 37 - 7 for v in g.integers(-2 ** 60, 2 ** 60, N)]
    assert OB.negacyclic_z(a, b, 2 * 101 + 6) == schoolbook(a, b)


def bfv_oracle(logn=6, L=3, K=1, dnum=3, tbits=16, slots=0):
    N = 1 << logn
    return OB.BfvOracle(Params(log2n=logn, L=L, K=K, dnum=dnum, t=plain_modulus(N, 1 << tbits),
                               scheme="bfv", slots=slots))


def test_tensor_is_the_defining_scale_and_round():
    orc = bfv_oracle(logn=4)
    orc.keygen(2)
    p = orc.p
    g = np.random.default_rng(3)
    a = orc.encrypt(orc.encode(g.integers(0, p.t, p.N // 2)), 5, 0)
    b = orc.encrypt(orc.encode(g.integers(0, p.t, p.N // 2)), 5, 1)
    d = orc.tensor(a, b)
    A = [orc._centred_coef(a[0]), orc._centred_coef(a[1])]
    Bc = [orc._centred_coef(b[0]), orc._centred_coef(b[1])]
    raw = [schoolbook(A[0], Bc[0]),
           [x + y for x, y in zip(schoolbook(A[0], Bc[1]), schoolbook(A[1], Bc[0]))],
           schoolbook(A[1], Bc[1])]
    Q, t = p.Q, p.t
    for c in range(3):
        # round(t x / Q) with exact rational arithmetic, then centred mod Q
        want = [math.floor(Fraction(t * x, Q) + Fraction(1, 2)) % Q for x in raw[c]]
        want = [w - Q if 2 * w > Q else w for w in want]
        assert orc._centred_coef(d[c]) == want


def test_encrypt_mult_rotate_mask_on_slots():
    orc = bfv_oracle(logn=6, L=3, K=1, dnum=3, tbits=17)
    p = orc.p
    N, t = p.N, p.t
    orc.keygen(4, [pow(5, 1, 2 * N), pow(5, 2, 2 * N)])
    g = np.random.default_rng(5)
    x, y = g.integers(0, t, N // 2), g.integers(0, t, N // 2)
    cx = orc.encrypt(orc.encode(x), 7, 0)
    cy = orc.encrypt(orc.encode(y), 7, 1)
    assert np.array_equal(orc.decode(orc.decrypt(cx))[0], x)
    prod = orc.mult(cx, cy)
    assert np.array_equal(orc.decode(orc.decrypt(prod))[0], (x.astype(object) * y) % t)
    rot = orc.rotate(prod, 3)
    assert np.array_equal(orc.decode(orc.decrypt(rot))[0], np.roll((x.astype(object) * y) % t, -3))
    masked = orc.cmult(cx, S.mask_ntt(orc, 9))
    assert np.array_equal(orc.decode(orc.decrypt(masked))[0], np.where(np.arange(N // 2) < 9, x, 0))
    assert orc.noise_bits(cx) < orc.noise_bits(prod) < orc.delta.bit_length() - 1


def test_spmv_bfv_equals_Ax():
    orc = bfv_oracle(logn=7, L=3, K=1, dnum=3, tbits=20, slots=30)
    A, x = synth.small_matrix(4, 70, 50, 400, -9, 9)
    plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, orc.p.slots)
    steps = sorted({k for ch in plan.chunks for k in S.rotation_steps(ch.c, ch.h)})
    orc.keygen(6, sorted({e for k in steps for e in orc.rotation_elements(k)}))
    res = S.spmv(orc, plan, S.encrypt_matrix(orc, plan, 2), S.encrypt_vector(orc, plan, x, 3))
    assert list(S.decrypt_result(orc, plan, res)) == list(A.matvec(x))
