"""The library's CKKS encoder (host, double-double) against the oracle's
exact encoding, bit for bit, and CKKS context parameter checks.  No GPU."""
import numpy as np
import pytest

from oracle import ckks as OC
from paper_2603_04742_gb300 import binding as B
from paper_2603_04742_gb300.api import Context


def ckks_ctx(logn, L=3, K=1, dnum=3, **kw):
    return Context(logn, L, K, dnum, 0, device=-1, torch_alloc=False, scheme="ckks", **kw)


@pytest.mark.parametrize("logn,seed,scale", [(4, 1, 20), (6, 2, 30), (10, 3, 40), (12, 4, 40)])
def test_encoder_matches_oracle(logn, seed, scale):
    ctx = ckks_ctx(logn)
    N = 1 << logn
    g = np.random.default_rng(seed)
    for n, lo, hi in ((N // 2, -1, 1), (N // 2 - 5, -100, 100), (3, -1e-3, 1e-3)):
        z = g.uniform(lo, hi, n)
        assert list(ctx.ckks_encode(z, scale)) == OC.encode(z, N, scale)


def test_encoder_matches_oracle_n32768():
    ctx = ckks_ctx(15, L=8, K=2, dnum=4)
    N = 1 << 15
    z = np.random.default_rng(9).uniform(-1, 1, N // 2)
    assert list(ctx.ckks_encode(z, 40)) == OC.encode(z, N, 40)


def test_encoder_closed_forms_and_ties():
    ctx = ckks_ctx(6)
    N = 64
    # constant slots: a constant polynomial, including exact halves
    for c in (1.0, -0.375, 2.5 / 2 ** 10, -2.5 / 2 ** 10):
        m = ctx.ckks_encode([c] * (N // 2), 10)
        want = int(np.sign(c) * np.floor(abs(c) * 2 ** 10 + 0.5))
        assert m[0] == want and not m[1:].any()


def test_encoder_range_and_parameter_errors():
    ctx = ckks_ctx(6)
    with pytest.raises(B.HespmvError) as e:
        ctx.ckks_encode([1e6] * 32, 60)
    assert e.value.code == B.HESPMV_E_RANGE
    with pytest.raises(B.HespmvError):
        ctx.ckks_encode(np.zeros(33), 20)       # more than N/2 values
    with pytest.raises(B.HespmvError):          # CKKS takes t = 0
        Context(6, 3, 1, 3, 12289, device=-1, torch_alloc=False, scheme="ckks")
    with pytest.raises(B.HespmvError):          # K < alpha: P does not cover a digit
        Context(6, 4, 1, 2, 0, device=-1, torch_alloc=False, scheme="ckks")
    with pytest.raises(B.HespmvError):
        ckks_ctx(6, scale_bits=70)


def test_ckks_plan_keeps_positions_only():
    ctx = ckks_ctx(8, slots=20)
    from paper_2603_04742_gb300 import synth
    A, _ = synth.small_matrix(2, 50, 30, 200)
    vals = np.random.default_rng(3).uniform(-1, 1, A.nnz)
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, vals)
    assert m.n_parts == 3 and m.n_chunks > 3
