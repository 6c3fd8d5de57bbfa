"""BFV on the GPU: keys, ciphertexts, the exact scale-and-round tensor,
HE-Mult and SpMV results bit-exact with the oracle's BFV variant from the
same seeds; decryptions equal A x exactly."""
import numpy as np
import pytest

from oracle import bfv as OB
from oracle import spmv as S
from oracle.params import Params, plain_modulus
from paper_2603_04742_gb300 import binding as B
from paper_2603_04742_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def pair(logn, L, K, dnum, t, slots=0):
    from paper_2603_04742_gb300.api import Context
    ctx = Context(logn, L, K, dnum, t, scheme="bfv", slots=slots)
    orc = OB.BfvOracle(Params(log2n=logn, L=L, K=K, dnum=dnum, t=t, scheme="bfv", slots=slots))
    return ctx, orc


def keys(ctx, orc, steps, seed):
    ctx.keygen(seed, steps)
    orc.keygen(seed, sorted({e for k in steps for e in orc.rotation_elements(k)}))


def run_pair(ctx, orc, A, x, seed_a=2, seed_x=3):
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, orc.p.slots)
    ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=seed_a)
    cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=seed_x)
    oa, ox = S.encrypt_matrix(orc, plan, seed_a), S.encrypt_vector(orc, plan, x, seed_x)
    ga, gx = ca.download(), cx.download()
    for k in range(len(oa)):
        assert np.array_equal(ga[k], oa[k]) and np.array_equal(gx[k], ox[k]), k
    return m, plan, ca, cx, oa, ox


@pytest.mark.parametrize("logn", [10, 12])
def test_bfv_tensor_and_mult_bit_exact(logn):
    # 2^10 runs the unfused key switch, 2^12 the fused one
    N = 1 << logn
    t = plain_modulus(N, 1 << 17)
    ctx, orc = pair(logn, 3, 1, 3, t)
    keys(ctx, orc, [1, 3], 7)
    assert np.array_equal(ctx.key_export(B.HESPMV_KEY_RELIN).reshape(orc.rlk.shape), orc.rlk)
    A, x = synth.small_matrix(3, N // 2, 40, N, -9, 9)
    m, plan, ca, cx, oa, ox = run_pair(ctx, orc, A, x)
    L, CT = orc.p.L, 2 * orc.p.L * N
    d = torch.zeros(3 * L * N, dtype=torch.int64, device="cuda")
    ctx.he_tensor(ca.ptr, cx.ptr, d.data_ptr())
    torch.cuda.synchronize()
    od = orc.tensor(oa[0], ox[0])
    assert np.array_equal(d.cpu().numpy().view(np.uint64).reshape(3, L, N), od)
    out = torch.zeros(CT, dtype=torch.int64, device="cuda")
    ctx.he_mult(ca.ptr, cx.ptr, out.data_ptr())
    torch.cuda.synchronize()
    om = orc.mult(oa[0], ox[0])
    assert np.array_equal(out.cpu().numpy().view(np.uint64).reshape(2, L, N), om)
    # decryption of the product: slot-wise chunk values times reorganised x
    slots = ctx.decrypt_slots(ca, 0)
    assert np.array_equal(slots[:len(plan.chunks[0].values)], plan.chunks[0].values % t)


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_bfv_spmv_parity(name):
    logn, L, K, dnum, t = synth.RING[name]
    ctx, orc = pair(logn, L, K, dnum, t)
    A, x = synth.workload(name)
    probe = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    keys(ctx, orc, probe.rotation_steps(), 1)
    m, plan, ca, cx, oa, ox = run_pair(ctx, orc, A, x)
    y = ctx.spmv(m, ca, cx)
    torch.cuda.synchronize()
    ores = S.spmv(orc, plan, oa, ox)
    gy = y.download()
    for p in range(len(ores)):
        assert np.array_equal(gy[p], ores[p]), p
    assert list(ctx.decrypt(m, y)) == list(A.matvec(x)) == list(S.decrypt_result(orc, plan, ores))


def test_bfv_partitions_and_ragged_batches():
    t = plain_modulus(1 << 6, 1 << 20)
    ctx, orc = pair(6, 3, 1, 3, t, slots=32)
    A, x = synth.small_matrix(5, 960, 64, 9000, -9, 9)
    probe = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    keys(ctx, orc, probe.rotation_steps(), 4)
    m, plan, ca, cx, oa, ox = run_pair(ctx, orc, A, x)
    assert m.n_chunks > 64
    y = ctx.spmv(m, ca, cx)
    torch.cuda.synchronize()
    ores = S.spmv(orc, plan, oa, ox)
    gy = y.download()
    for p in range(len(ores)):
        assert np.array_equal(gy[p], ores[p]), p
    assert list(ctx.decrypt(m, y)) == list(A.matvec(x))
    # host-buffer paths: 64-bit words, packed (BFV groups are unpacked by
    # their own kernel before the tensor), pipelined packed
    hy = np.zeros_like(gy)
    ctx.spmv_host(m, ca.download(), cx.download(), hy)
    assert np.array_equal(hy, gy)
    words, _ = ctx.ct_packed_words()
    pA, pX = ctx.ct_pack(ca.download()), ctx.ct_pack(cx.download())
    py = np.zeros((m.n_parts, words), dtype=np.uint64)
    ctx.spmv_host_packed(m, pA, pX, py)
    assert np.array_equal(ctx.ct_unpack(py), gy)
    py[:] = 0
    stream = torch.cuda.Stream()
    for _ in range(4):
        ctx.spmv_host_packed_async(m, pA, pX, py, stream=stream)
    stream.synchronize()
    ctx.device_status()
    assert np.array_equal(ctx.ct_unpack(py), gy)


def test_bfv_c3_stencil_full_size():
    """The large configuration under BFV: sampled tensors bit-exact, the
    whole SpMV decrypting to the exact integer result."""
    logn, L, K, dnum, t = synth.RING["c3"]
    ctx, orc = pair(logn, L, K, dnum, t)
    A, xf = synth.workload("c3")
    A.vals = synth.quantize(A.vals)
    x = synth.quantize(xf)
    ctx.keygen(1, [])
    orc.keygen(1, [])
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, orc.p.slots)
    ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=2)
    cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=3)
    N = 1 << logn
    CT = 2 * L * N
    reorg = S.reorg_vector(x, plan.chunks)
    for k in (0, len(plan.chunks) - 1):
        oa = orc.encrypt(orc.encode(plan.chunks[k].values), 2, k)
        ox = orc.encrypt(orc.encode(reorg[k]), 3, k)
        assert np.array_equal(ca.download()[k], oa) and np.array_equal(cx.download()[k], ox)
        d = torch.zeros(3 * L * N, dtype=torch.int64, device="cuda")
        ctx.he_tensor(ca.ptr + 8 * k * CT, cx.ptr + 8 * k * CT, d.data_ptr())
        torch.cuda.synchronize()
        assert np.array_equal(d.cpu().numpy().view(np.uint64).reshape(3, L, N), orc.tensor(oa, ox)), k
    y = ctx.spmv(m, ca, cx)
    torch.cuda.synchronize()
    assert list(ctx.decrypt(m, y)) == list(A.matvec(x))


def test_bfv_generic_word_counts():
    """A ring whose multi-word widths (Q: 5 words, B: 5 words) take the
    kernels' runtime-width path rather than a specialised one."""
    t = plain_modulus(1 << 6, 1 << 20)
    ctx, orc = pair(6, 4, 2, 2, t, slots=24)
    A, x = synth.small_matrix(8, 80, 40, 500, -9, 9)
    probe = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    keys(ctx, orc, probe.rotation_steps(), 5)
    m, plan, ca, cx, oa, ox = run_pair(ctx, orc, A, x)
    y = ctx.spmv(m, ca, cx)
    torch.cuda.synchronize()
    ores = S.spmv(orc, plan, oa, ox)
    gy = y.download()
    for p in range(len(ores)):
        assert np.array_equal(gy[p], ores[p]), p
    assert list(ctx.decrypt(m, y)) == list(A.matvec(x))


def test_bfv_plain_matrix_mode():
    logn, L, K, dnum, t = synth.RING["c1"]
    ctx, orc = pair(logn, L, K, dnum, t)
    A, x = synth.workload("c1")
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    keys(ctx, orc, m.rotation_steps(), 3)
    plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, orc.p.slots)
    pa = ctx.encode_matrix_plain(m)
    cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=9)
    y = ctx.spmv_ptmatrix(m, pa, cx)
    torch.cuda.synchronize()
    ores = S.spmv_plain_matrix(orc, plan, S.encode_matrix_plain(orc, plan),
                               S.encrypt_vector(orc, plan, x, 9))
    gy = y.download()
    for p in range(len(ores)):
        assert np.array_equal(gy[p], ores[p]), p
    assert list(ctx.decrypt(m, y)) == list(A.matvec(x))
