"""Pins of the oracle's CKKS encoding and scheme (CPU): the FFT path equals
the defining sum evaluated exactly; closed forms (a constant slot vector is
a constant polynomial); the slot-wise product of the negacyclic product and
the slot rotation of the automorphism X -> X^(5^k); encryption, HE-Mult,
rotation, masking and the whole SpMV decode to the real results within the
rounding and noise bounds."""
import math

import numpy as np
import pytest

from oracle import ckks
from oracle import spmv as S
from oracle.params import Params
from paper_2603_04742_gb300 import synth


def negacyclic(a, b):
    N = len(a)
    out = [0] * N
    for i, x in enumerate(a):
        if x == 0:
            continue
        for j, y in enumerate(b):
            k = i + j
            if k < N:
                out[k] += x * y
            else:
                out[k - N] -= x * y
    return out


@pytest.mark.parametrize("logn,seed", [(4, 1), (6, 2), (8, 3), (8, 4)])
def test_fft_path_equals_exact_sum(logn, seed):
    N = 1 << logn
    g = np.random.default_rng(seed)
    for n in (N // 2, N // 2 - 3, 1):
        z = g.uniform(-2, 2, n)
        assert ckks.encode(z, N, 30) == ckks.encode(z, N, 30, exact_all=True)


def test_constant_slots_give_a_constant_polynomial():
    N = 1 << 6
    for c in (1.0, -0.375, 3.25):
        m = ckks.encode([c] * (N // 2), N, 20)
        assert m[0] == round(c * 2 ** 20) and all(v == 0 for v in m[1:])


def test_single_slot_closed_form():
    # z = e_j: m_k = round(Delta * 2/N * cos(pi k 5^j / N))
    N = 1 << 5
    for j in (0, 1, 7):
        z = [0.0] * (N // 2)
        z[j] = 1.0
        m = ckks.encode(z, N, 24)
        e = pow(5, j, 2 * N)
        want = [int(math.copysign(math.floor(abs(v) + 0.5), v))
                for v in (2 ** 24 * 2 / N * math.cos(math.pi * k * e / N) for k in range(N))]
        assert m == want


def test_decode_inverts_encode_within_rounding():
    N = 1 << 8
    g = np.random.default_rng(5)
    z = g.uniform(-1, 1, N // 2)
    d = ckks.decode(ckks.encode(z, N, 30), N, N // 2, 2.0 ** 30)
    # each of N coefficients is off by at most 1/2
    assert np.max(np.abs(d - z)) <= (N / 2) / 2 ** 30 * 1.01


def test_product_and_rotation_act_on_slots():
    N = 1 << 6
    g = np.random.default_rng(6)
    z1, z2 = g.uniform(-1, 1, N // 2), g.uniform(-1, 1, N // 2)
    m1, m2 = ckks.encode(z1, N, 20), ckks.encode(z2, N, 20)
    prod = ckks.decode(negacyclic(m1, m2), N, N // 2, 2.0 ** 40)
    assert np.max(np.abs(prod - z1 * z2)) < 1e-4
    for k in (1, 5, 17):
        gk = pow(5, k, 2 * N)
        rot = [0] * N
        for i, c in enumerate(m1):        # X^i -> X^(i g), X^N = -1
            e = i * gk % (2 * N)
            if e < N:
                rot[e] += c
            else:
                rot[e - N] -= c
        r = ckks.decode(rot, N, N // 2, 2.0 ** 20)
        assert np.max(np.abs(r - np.roll(z1, -k))) < 1e-4


def ckks_oracle(logn=8, L=4, K=2, dnum=2, scale=30, mscale=20, slots=0):
    p = Params(log2n=logn, L=L, K=K, dnum=dnum, t=0, scheme="ckks", scale_bits=scale,
               mask_scale_bits=mscale, slots=slots)
    return ckks.CkksOracle(p)


def test_scheme_ops_decode_to_real_results():
    orc = ckks_oracle()
    N = orc.p.N
    orc.keygen(3, [pow(5, 1, 2 * N), pow(5, 4, 2 * N)])
    g = np.random.default_rng(7)
    a, b = g.uniform(-1, 1, N // 2), g.uniform(-1, 1, N // 2)
    ca = orc.encrypt(orc.encode(a), 9, 0)
    cb = orc.encrypt(orc.encode(b), 9, 1)
    # fresh noise: a few hundred per coefficient at most, N of them per slot
    tol = 256.0 * N / 2 ** 30
    assert np.max(np.abs(orc.decode_ct(ca, N // 2, 30) - a)) < tol
    prod = orc.mult(ca, cb)
    assert np.max(np.abs(orc.decode_ct(prod, N // 2, 60) - a * b)) < 3 * tol
    rot = orc.rotate(ca, 5)                   # chain 1 + 4
    assert np.max(np.abs(orc.decode_ct(rot, N // 2, 30) - np.roll(a, -5))) < 2 * tol
    masked = orc.cmult(ca, S.mask_ntt(orc, 10))
    want = np.where(np.arange(N // 2) < 10, a, 0.0)
    # plus the mask's own rounding: N/2 coefficients off by 1/2 at scale 2^20
    assert np.max(np.abs(orc.decode_ct(masked, N // 2, 50) - want)) < 2 * tol + N / 2 ** 21


def test_ckks_needs_p_to_cover_a_digit():
    with pytest.raises(AssertionError):
        Params(log2n=6, L=4, K=1, dnum=2, t=0, scheme="ckks")


def test_spmv_real_values_within_tolerance():
    orc = ckks_oracle(logn=7, L=4, K=1, dnum=4, scale=30, mscale=20, slots=24)
    A, _ = synth.small_matrix(11, 60, 40, 300)
    g = np.random.default_rng(12)
    A.vals = g.uniform(-1, 1, A.nnz)
    x = g.uniform(-1, 1, A.cols)
    plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, orc.p.slots)
    steps = sorted({k for ch in plan.chunks for k in S.rotation_steps(ch.c, ch.h)})
    orc.keygen(4, sorted({e for k in steps for e in orc.rotation_elements(k)}))
    ca = S.encrypt_matrix(orc, plan, 2)
    cx = S.encrypt_vector(orc, plan, x, 3)
    y = S.decrypt_result_real(orc, plan, S.spmv(orc, plan, ca, cx))
    ref = A.dense() @ x
    assert len(plan.parts) == 3
    assert np.max(np.abs(y - ref)) <= 1e-3 * max(1.0, np.max(np.abs(ref)))


def _crt_centred(res, q):
    """The integer in (-Q/2, Q/2] with the given residues (Python big ints)."""
    Q = 1
    for v in q:
        Q *= v
    x = 0
    for r, v in zip(res, q):
        Qh = Q // v
        x += int(r) * Qh * pow(Qh, -1, v)
    x %= Q
    return x - Q if x > Q // 2 else x


@pytest.mark.parametrize("logn,L", [(5, 3), (6, 4)])
def test_rescale_is_exact_division_by_the_last_prime(logn, L):
    """Each coefficient c of each component, as an integer over q_0..q_{L-1},
    becomes (c - r) / q_{L-1} with r = c mod q_{L-1} centred: checked with
    big-integer Chinese remaindering against the oracle's limb-wise form."""
    orc = ckks_oracle(logn=logn, L=L, K=1, dnum=L, scale=20, mscale=10)
    p = orc.p
    g = np.random.default_rng(logn)
    ct = np.stack([np.stack([g.integers(0, p.q[l], size=p.N, dtype=np.uint64) for l in range(L)])
                   for _ in range(2)])
    out = orc.rescale(ct)
    assert out.shape == (2, L - 1, p.N)
    ql = p.q[L - 1]
    for c in range(2):
        coef = [orc.intt(ct[c, l], l) for l in range(L)]
        got = [orc.intt(out[c, l], l) for l in range(L - 1)]
        for k in range(p.N):
            x = _crt_centred([coef[l][k] for l in range(L)], p.q[:L])
            r = x % ql
            r = r - ql if r > ql // 2 else r
            assert (x - r) % ql == 0
            want = (x - r) // ql
            for l in range(L - 1):
                assert int(got[l][k]) == want % p.q[l], (c, k, l)


def test_rescale_divides_the_plaintext():
    """decrypt(rescale(c)) = decrypt(c) / q_{L-1} within (1 + ||s||_1) / 2
    (the rounding of both components, the second times the ternary secret),
    and slot values encoded at scale 2^20 q_{L-1} decode at scale 2^20."""
    orc = ckks_oracle(logn=6, L=3, K=1, dnum=3, scale=20, mscale=10)
    p = orc.p
    N = p.N
    orc.keygen(5, [])
    ql = p.q[p.L - 1]
    g = np.random.default_rng(3)
    z = g.uniform(-1, 1, N // 2)
    # slots at scale 2^20 * q_{L-1}: the encoding at 2^20 times q_{L-1}
    # (coefficients of about 2^70, within Q of 3 x 50 bits)
    m = [v * ql for v in ckks.encode(z, N, 20)]
    ct = orc.encrypt(m, 4, 0)
    d0 = orc.decrypt_level(ct)
    out = orc.rescale(ct)
    d1 = orc.decrypt_level(out)
    s1 = int(sum(1 for v in orc.intt(orc.s[0], 0) if v != 0))   # ||s||_1 for a ternary secret
    bound = (1 + s1) / 2
    assert max(abs(b * ql - a) for a, b in zip(d0, d1)) <= bound * ql
    zz = ckks.decode(np.array(d1, dtype=np.float64), N, N // 2, float(2 ** 20))
    assert np.max(np.abs(zz - z)) < 1e-3
