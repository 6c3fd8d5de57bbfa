"""Pins of the oracle's scheme: every HE operation of Section 2.1 checked
through decryption (slotwise semantics), noise below Q/2, and the end-to-end
statement that decrypting the encrypted SpMV gives A.x exactly."""
import random

import numpy as np
import pytest

from oracle.bgv import Oracle
from oracle.params import Params
from oracle import spmv as S
from paper_2603_04742_gb300 import synth


def make(logn=6, L=3, K=1, dnum=3, t=257, gels=(), seed=7):
    p = Params(log2n=logn, L=L, K=K, dnum=dnum, t=t)
    orc = Oracle(p)
    orc.keygen(seed, gels)
    return orc


def rand_slots(orc, seed):
    r = random.Random(seed)
    n = orc.p.N // 2
    return [r.randrange(orc.p.t) for _ in range(n)], [r.randrange(orc.p.t) for _ in range(n)]


def enc(orc, rows, seed, idx=0):
    return orc.encrypt(orc.encode(*rows), seed, idx)


def dec(orc, ct):
    a, b = orc.decode(orc.decrypt(ct))
    return [int(v) for v in a], [int(v) for v in b]


@pytest.mark.parametrize("cfg", [(6, 3, 1, 3, 257), (5, 4, 2, 2, 193), (6, 8, 2, 4, 257)])
def test_encrypt_decrypt_add(cfg):
    orc = make(*cfg)
    x, y = rand_slots(orc, 1), rand_slots(orc, 2)
    cx, cy = enc(orc, x, 11, 0), enc(orc, y, 11, 1)
    assert dec(orc, cx) == (x[0], x[1])
    t = orc.p.t
    s = dec(orc, orc.add(cx, cy))
    assert s == ([(a + b) % t for a, b in zip(x[0], y[0])], [(a + b) % t for a, b in zip(x[1], y[1])])


@pytest.mark.parametrize("cfg", [(6, 3, 1, 3, 257), (5, 4, 2, 2, 193), (6, 8, 2, 4, 257)])
def test_mult_relinearise(cfg):
    orc = make(*cfg)
    t = orc.p.t
    x, y = rand_slots(orc, 3), rand_slots(orc, 4)
    cx, cy = enc(orc, x, 5, 0), enc(orc, y, 5, 1)
    d = orc.tensor(cx, cy)
    # the 3-component tensor decrypts with (1, s, s^2) before relinearisation
    prod = orc.mult(cx, cy)
    assert dec(orc, prod) == ([a * b % t for a, b in zip(x[0], y[0])],
                              [a * b % t for a, b in zip(x[1], y[1])])
    assert orc.noise_bits(prod) < orc.p.Q.bit_length() - 2
    assert d.shape[0] == 3


@pytest.mark.parametrize("policy", ["pow2", "exact"])
def test_rotation_is_left_shift_per_row(policy):
    p = Params(log2n=6, L=3, K=1, dnum=3, t=257)
    orc = Oracle(p)
    steps = [1, 3, 6, 13, 31]
    gels = set()
    for k in steps:
        gels.update(orc.rotation_elements(k, policy))
    orc.keygen(9, sorted(gels))
    x = rand_slots(orc, 6)
    cx = enc(orc, x, 8)
    for k in steps:
        got = dec(orc, orc.rotate(cx, k, policy))
        assert got == (list(np.roll(x[0], -k)), list(np.roll(x[1], -k))), k


def test_keyswitch_identity_from_known_key():
    """Switching s'*d from a key for s' = s^2 equals the relinearised form:
    decrypt(d0 + ks0, d1 + ks1) = d0 + d1 s + d2 s^2."""
    orc = make(5, 4, 2, 2, 193)
    x, y = rand_slots(orc, 1), rand_slots(orc, 2)
    d = orc.tensor(enc(orc, x, 3, 0), enc(orc, y, 3, 1))
    ks = orc.keyswitch(d[2], orc.rlk)
    # phase of (0 + ks0, ks1) must equal d2 * s^2 up to t*noise: decrypt both
    # sides' contributions through the full relinearised ciphertext instead
    full = orc.relinearize(d)
    t = orc.p.t
    assert dec(orc, full)[0] == [a * b % t for a, b in zip(x[0], y[0])]
    assert ks.shape == (2, orc.p.L, orc.p.N)


def test_mask_cmult():
    orc = make()
    t = orc.p.t
    x = rand_slots(orc, 4)
    r = 11
    w = orc.cmult(enc(orc, x, 2), S.mask_ntt(orc, r))
    got = dec(orc, w)
    assert got[0] == [v if j < r else 0 for j, v in enumerate(x[0])]
    assert got[1] == [0] * (orc.p.N // 2)


def _run_spmv(A, x, p, policy="pow2", kseed=1, mseed=2, vseed=3):
    orc = Oracle(p)
    plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, p.slots)
    gels = set()
    for ch in plan.chunks:
        for k in S.rotation_steps(ch.c, ch.h):
            gels.update(orc.rotation_elements(k, policy))
    orc.keygen(kseed, sorted(gels))
    ca = S.encrypt_matrix(orc, plan, mseed)
    cx = S.encrypt_vector(orc, plan, x, vseed)
    orc.counts.clear()
    res = S.spmv(orc, plan, ca, cx, policy)
    return orc, plan, res, S.decrypt_result(orc, plan, res)


@pytest.mark.parametrize("policy", ["pow2", "exact"])
def test_spmv_small_with_partitions(policy):
    A, x = synth.small_matrix(21, 45, 30, 150, -7, 7)
    p = Params(log2n=5, L=3, K=1, dnum=3, t=7681)   # 16 slots: 3 partitions
    orc, plan, res, y = _run_spmv(A, x, p, policy)
    assert len(plan.parts) == 3
    assert list(y) == list(A.matvec(x))
    # Table 3: one HE-Mult and one HE-CMult per chunk; rotations from totalSum
    n_ct = len(plan.chunks)
    assert orc.counts["mult"] == n_ct and orc.counts["cmult"] == n_ct
    rots = sum(len(S.rotation_steps(ch.c, ch.h)) for ch in plan.chunks)
    assert orc.counts.get("rot", 0) == rots
    cmax = max(ch.c for ch in plan.chunks)
    assert rots <= 2 * n_ct * max(1, np.log2(cmax))
    for r in res:
        assert orc.noise_bits(r) < p.Q.bit_length() - 2


def test_spmv_c1_end_to_end():
    A, x = synth.workload("c1")
    logn, L, K, dnum, t = synth.RING["c1"]
    p = Params(log2n=logn, L=L, K=K, dnum=dnum, t=t)
    orc, plan, res, y = _run_spmv(A, x, p)
    assert list(y) == list(A.matvec(x))
    # remaining noise budget (bits) stays well above zero
    assert p.Q.bit_length() - 1 - orc.noise_bits(res[0]) > 20


def test_spmv_plain_matrix_mode():
    """Plaintext matrix times encrypted vector (HE-CMult per chunk) decrypts
    to A.x, with one multiplicative level fewer than the ciphertext mode."""
    A, x = synth.small_matrix(31, 60, 50, 300, -9, 9)
    p = Params(log2n=6, L=3, K=1, dnum=3, t=12289)
    orc = Oracle(p)
    plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, p.slots)
    gels = set()
    for ch in plan.chunks:
        for k in S.rotation_steps(ch.c, ch.h):
            gels.update(orc.rotation_elements(k))
    orc.keygen(5, sorted(gels))
    pts = S.encode_matrix_plain(orc, plan)
    cx = S.encrypt_vector(orc, plan, x, 6)
    orc.counts.clear()
    res = S.spmv_plain_matrix(orc, plan, pts, cx)
    assert list(S.decrypt_result(orc, plan, res)) == list(A.matvec(x))
    assert orc.counts.get("mult", 0) == 0 and orc.counts["cmult"] == 2 * len(plan.chunks)
