"""CKKS on the GPU: keys, ciphertexts and SpMV results bit-exact with the
oracle's CKKS variant from the same seeds, and decryptions within the
stated tolerance of the float64 SpMV (1e-3 relative in the max norm; the
noise and rounding bounds give far less)."""
import numpy as np
import pytest

from oracle import ckks as OC
from oracle import spmv as S
from oracle.params import Params
from paper_2603_04742_gb300 import binding as B
from paper_2603_04742_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-3


def pair(logn, L, K, dnum, scale=40, mscale=30, slots=0):
    from paper_2603_04742_gb300.api import Context
    ctx = Context(logn, L, K, dnum, 0, scheme="ckks", scale_bits=scale, mask_scale_bits=mscale,
                  slots=slots)
    orc = OC.CkksOracle(Params(log2n=logn, L=L, K=K, dnum=dnum, t=0, scheme="ckks",
                               scale_bits=scale, mask_scale_bits=mscale, slots=slots))
    return ctx, orc


def keys(ctx, orc, m, seed):
    steps = m.rotation_steps()
    ctx.keygen(seed, steps)
    orc.keygen(seed, sorted({e for k in steps for e in orc.rotation_elements(k)}))


def real_workload(A, seed):
    g = np.random.default_rng(seed)
    A.vals = g.uniform(-1, 1, A.nnz)
    return A, g.uniform(-1, 1, A.cols)


def check_result(ctx, m, y, A, x):
    out = ctx.decrypt_real(m, y)
    ref = A.matvec(x)
    err = np.max(np.abs(out - ref)) / max(1.0, np.max(np.abs(ref)))
    assert err <= TOL, err
    return err


def test_ckks_keys_ciphertexts_and_spmv_bit_exact():
    logn, L, K, dnum, _ = synth.RING["c1"]
    ctx, orc = pair(logn, L, K, dnum)
    A, _ = synth.workload("c1")
    A, x = real_workload(A, 31)
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    keys(ctx, orc, m, 5)
    assert np.array_equal(ctx.key_export(B.HESPMV_KEY_RELIN).reshape(orc.rlk.shape), orc.rlk)
    plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, orc.p.slots)
    ca = ctx.encrypt_real(m, B.HESPMV_MATRIX, A.vals, seed=2)
    cx = ctx.encrypt_real(m, B.HESPMV_VECTOR, x, seed=3)
    oa = S.encrypt_matrix(orc, plan, 2)
    ox = S.encrypt_vector(orc, plan, x, 3)
    ga, gx = ca.download(), cx.download()
    for k in range(len(oa)):
        assert np.array_equal(ga[k], oa[k]) and np.array_equal(gx[k], ox[k]), k
    y = ctx.spmv(m, ca, cx)
    torch.cuda.synchronize()
    ores = S.spmv(orc, plan, oa, ox)
    gy = y.download()
    for p in range(len(ores)):
        assert np.array_equal(gy[p], ores[p]), p
    check_result(ctx, m, y, A, x)
    oy = S.decrypt_result_real(orc, plan, ores)
    assert np.max(np.abs(ctx.decrypt_real(m, y) - oy)) < 1e-9


def test_ckks_partitions_and_plain_matrix():
    ctx, orc = pair(10, 3, 1, 3, scale=36, mscale=24, slots=40)
    A, _ = synth.small_matrix(7, 150, 90, 1400)
    A, x = real_workload(A, 8)
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    keys(ctx, orc, m, 6)
    assert m.n_parts == 4
    ca = ctx.encrypt_real(m, B.HESPMV_MATRIX, A.vals, seed=4)
    cx = ctx.encrypt_real(m, B.HESPMV_VECTOR, x, seed=5)
    y = ctx.spmv(m, ca, cx)
    torch.cuda.synchronize()
    check_result(ctx, m, y, A, x)
    plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, orc.p.slots)
    ores = S.spmv(orc, plan, S.encrypt_matrix(orc, plan, 4), S.encrypt_vector(orc, plan, x, 5))
    gy = y.download()
    for p in range(len(ores)):
        assert np.array_equal(gy[p], ores[p]), p
    # the evaluator holding the matrix in the clear
    pa = ctx.encode_matrix_plain_real(m, A.vals)
    yp = ctx.spmv_ptmatrix(m, pa, cx)
    torch.cuda.synchronize()
    check_result(ctx, m, yp, A, x)


def test_ckks_c2_float_variant():
    """The mid configuration's float variant: N(0,1) entries at scale 2^40."""
    logn, L, K, dnum, _ = synth.RING["c2"]
    ctx, orc = pair(logn, L, K, dnum, scale=40, mscale=30)
    A, _ = synth.workload("c2")
    g = np.random.default_rng(77)
    A.vals = g.standard_normal(A.nnz)
    x = g.standard_normal(A.cols)
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    keys(ctx, orc, m, 9)
    ca = ctx.encrypt_real(m, B.HESPMV_MATRIX, A.vals, seed=10)
    cx = ctx.encrypt_real(m, B.HESPMV_VECTOR, x, seed=11)
    y = ctx.spmv(m, ca, cx)
    torch.cuda.synchronize()
    assert check_result(ctx, m, y, A, x) < 1e-6
    plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, orc.p.slots)
    ores = S.spmv(orc, plan, S.encrypt_matrix(orc, plan, 10), S.encrypt_vector(orc, plan, x, 11))
    gy = y.download()
    for p in range(len(ores)):
        assert np.array_equal(gy[p], ores[p]), p


def test_ckks_c3_stencil_float_full_size():
    """The large configuration with its float64 values directly (no fixed
    point): sampled ciphertexts against the oracle, the result within the
    tolerance."""
    logn, L, K, dnum, _ = synth.RING["c3"]
    ctx, orc = pair(logn, L, K, dnum, scale=40, mscale=30)
    A, x = synth.workload("c3")
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    ctx.keygen(1, [])
    orc.keygen(1, [])
    ca = ctx.encrypt_real(m, B.HESPMV_MATRIX, A.vals, seed=2)
    cx = ctx.encrypt_real(m, B.HESPMV_VECTOR, x, seed=3)
    plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, orc.p.slots)
    ga = ca.download()
    for k in (0, 13, len(plan.chunks) - 1):
        ch = plan.chunks[k]
        assert np.array_equal(ga[k], orc.encrypt(orc.encode(ch.values), 2, k)), k
    y = ctx.spmv(m, ca, cx)
    torch.cuda.synchronize()
    assert check_result(ctx, m, y, A, x) < 1e-6


def test_ckks_rescale_bit_exact_and_divides_the_scale():
    """hespmv_rescale of SpMV results equals the oracle's rescale residue for
    residue (two partitions at once), and the rescaled ciphertexts decrypt
    over the remaining primes to the same slot values at scale / q_{L-1}."""
    ctx, orc = pair(10, 3, 1, 3, scale=36, mscale=24, slots=250)
    A, _ = synth.small_matrix(12, 400, 300, 2000)
    A, x = real_workload(A, 13)
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    keys(ctx, orc, m, 7)
    assert m.n_parts == 2
    ca = ctx.encrypt_real(m, B.HESPMV_MATRIX, A.vals, seed=4)
    cx = ctx.encrypt_real(m, B.HESPMV_VECTOR, x, seed=5)
    y = ctx.spmv(m, ca, cx)
    torch.cuda.synchronize()
    N, L = 1 << 10, 3
    out = torch.full((2 * 2 * (L - 1) * N,), -1, dtype=torch.int64, device="cuda")
    ctx.rescale(y.ptr, out.data_ptr(), n=2)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint64).reshape(2, 2, L - 1, N)
    gy = y.download()
    for p in range(2):
        assert np.array_equal(got[p], orc.rescale(gy[p])), p
    total = 2 * 36 + 24
    ql = orc.p.q[L - 1]
    for p in range(2):
        before = ctx.decrypt_real_slots(y, p, total)
        after = ctx.decrypt_real_level(out.data_ptr() + p * 2 * (L - 1) * N * 8, L - 1, 2.0 ** total / ql)
        assert np.max(np.abs(after - before)) < 1e-6 * max(1.0, np.max(np.abs(before)))
    # non-CKKS contexts and misaligned buffers are refused on the host
    with pytest.raises(B.HespmvError):
        ctx.rescale(y.ptr + 8, out.data_ptr(), n=1)
