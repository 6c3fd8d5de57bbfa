"""Packed ciphertext wire format (host side): W = max bit length of the
ciphertext primes per residue, one little-endian bit string per limb, padded
to whole 64-bit words.  The layout is restated here with Python integers and
compared word for word with the library's packing."""
import numpy as np
import pytest

from paper_2603_04742_gb300 import synth
from paper_2603_04742_gb300.api import Context
from paper_2603_04742_gb300.binding import HespmvError


def host_ctx(name="c1"):
    logn, L, K, dnum, t = synth.RING[name]
    return Context(logn, L, K, dnum, t, device=-1, torch_alloc=False)


def reference_pack(cts, q, W):
    """[n][2][L][N] residues -> [n][2 L ceil(N W / 64)] words via one Python
    integer per limb: residue k occupies bits [k W, k W + W)."""
    n, _, L, N = cts.shape
    lw = (N * W + 63) // 64
    out = np.zeros((n, 2 * L * lw), dtype=np.uint64)
    for i in range(n):
        for c in range(2):
            for l in range(L):
                acc = 0
                for k in range(N):
                    acc |= int(cts[i, c, l, k]) << (k * W)
                limb = (c * L + l) * lw
                for w in range(lw):
                    out[i, limb + w] = (acc >> (64 * w)) & ((1 << 64) - 1)
    return out


def random_cts(ctx, n, seed):
    rng = np.random.default_rng(seed)
    q = np.array(ctx.moduli()[0][:ctx.L], dtype=np.uint64)
    cts = rng.integers(0, 1 << 62, size=(n, 2, ctx.L, ctx.N), dtype=np.uint64)
    cts %= q[None, None, :, None]
    cts[0, 0, 0, :4] = q[0] - 1          # the largest residue
    cts[0, 1, ctx.L - 1, -3:] = 0
    return cts, q


def test_packed_size_and_width():
    ctx = host_ctx()
    words, bits = ctx.ct_packed_words()
    q = ctx.moduli()[0][:ctx.L]
    assert bits == max(int(x).bit_length() for x in q) == 50
    assert words == 2 * ctx.L * ((ctx.N * bits + 63) // 64)
    # 50 of 64 bits: the packed ciphertext is 25/32 of the plain one
    assert words * 64 == 2 * ctx.L * ctx.N * 50


def test_pack_matches_reference_layout_and_round_trips():
    ctx = host_ctx()
    cts, q = random_cts(ctx, 2, 7)
    packed = ctx.ct_pack(cts)
    _, W = ctx.ct_packed_words()
    assert np.array_equal(packed, reference_pack(cts, q, W))
    assert np.array_equal(ctx.ct_unpack(packed), cts)


def test_pack_rejects_unreduced_residue():
    ctx = host_ctx()
    cts, q = random_cts(ctx, 1, 8)
    cts[0, 1, 2, 17] = q[2]
    with pytest.raises(HespmvError):
        ctx.ct_pack(cts)


def test_unpack_rejects_unreduced_residue():
    ctx = host_ctx()
    cts, q = random_cts(ctx, 1, 9)
    packed = ctx.ct_pack(cts)
    _, W = ctx.ct_packed_words()
    # residue 5 of limb 0 set to q_0 (its bits lie in word 5 W / 64)
    bad = packed.copy()
    k, v = 5, int(q[0])
    lo = k * W
    for w in range(lo // 64, (lo + W - 1) // 64 + 1):
        m = 0
        for b in range(64 * w, 64 * w + 64):
            if lo <= b < lo + W:
                m |= 1 << (b - 64 * w)
        keep = int(bad[0, w]) & ~m
        sh = lo - 64 * w
        part = (v << sh) if sh >= 0 else (v >> -sh)
        bad[0, w] = (keep | (part & m)) & ((1 << 64) - 1)
    with pytest.raises(HespmvError):
        ctx.ct_unpack(bad)
    # round trip on a second ring (N = 2^10); N W is a multiple of 64 for
    # every supported N, so no limb has padding bits
    ctx2 = Context(10, 3, 1, 3, 40961, device=-1, torch_alloc=False)
    words, W2 = ctx2.ct_packed_words()
    assert ctx2.N * W2 % 64 == 0 and words == 2 * ctx2.L * ctx2.N * W2 // 64
    cts2, _ = random_cts(ctx2, 3, 10)
    assert np.array_equal(ctx2.ct_unpack(ctx2.ct_pack(cts2)), cts2)


def test_upload_groups_setting():
    ctx = host_ctx()
    assert ctx.get_upload_groups() == 0          # the defaults
    ctx.set_upload_groups(3)
    assert ctx.get_upload_groups() == 3
    ctx.set_upload_groups(0)
    assert ctx.get_upload_groups() == 0
    for bad in (-1, 65):
        with pytest.raises(HespmvError):
            ctx.set_upload_groups(bad)
