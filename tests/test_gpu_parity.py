"""GPU parity: every RNS residue of every intermediate the C ABI exposes
(NTT, keys, ciphertexts, tensor, relinearisation, key switch, rotation,
mask multiply, the SpMV result) equals the oracle's from the same seeds, and
decryption equals the plaintext SpMV.  Integer work: bit-exact."""
import numpy as np
import pytest

from oracle import native
from oracle import spmv as S
from oracle.bgv import Oracle
from oracle.params import Params, plain_modulus
from paper_2603_04742_gb300 import binding as B
from paper_2603_04742_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


def make_pair(logn, L, K, dnum, t, seed=1, steps=None, policy="pow2", slots=0):
    from paper_2603_04742_gb300.api import Context
    ctx = Context(logn, L, K, dnum, t, rot_policy=policy, slots=slots)
    p = Params(log2n=logn, L=L, K=K, dnum=dnum, t=t, slots=slots)
    orc = Oracle(p)
    ctx.keygen(seed, steps)
    gels = set()
    if steps is None:
        if policy == "pow2":
            b = 1
            while b < p.N // 2:
                gels.add(pow(5, b, 2 * p.N))
                b *= 2
    else:
        for k in steps:
            gels.update(orc.rotation_elements(k, policy))
    orc.keygen(seed, sorted(gels))
    return ctx, orc


@pytest.mark.parametrize("logn", [4, 6, 10, 12, 13, 14, 15])
def test_ntt_parity_all_moduli(logn):
    from paper_2603_04742_gb300.api import Context
    N = 1 << logn
    t = plain_modulus(N, 1 << 20)
    ctx = Context(logn, 3, 2, 3, t)
    q, psi, zeta = ctx.moduli()
    moduli = q + [t]
    roots = psi + [zeta]
    rng = np.random.default_rng(logn)
    a = np.stack([rng.integers(0, m, size=N, dtype=np.uint64) for m in moduli])
    d = dev(a)
    ctx.ntt(d.data_ptr(), 0, len(moduli))
    got = host(d)
    for k in range(len(moduli)):
        assert np.array_equal(got[k], native.ntt(a[k], moduli[k], roots[k])), k
    ctx.ntt(d.data_ptr(), 0, len(moduli), inverse=True)
    assert np.array_equal(host(d), a)
    # batched items: 4 items x 3 Q limbs
    b = np.concatenate([np.stack([rng.integers(0, m, size=N, dtype=np.uint64) for m in q[:3]])
                        for _ in range(4)])
    d = dev(b)
    ctx.ntt(d.data_ptr(), 0, 3, n_items=4)
    got = host(d)
    for r in range(12):
        assert np.array_equal(got[r], native.ntt(b[r], q[r % 3], psi[r % 3]))


def test_keys_parity_c1():
    logn, L, K, dnum, t = synth.RING["c1"]
    ctx, orc = make_pair(logn, L, K, dnum, t, seed=77)
    N, LK = 1 << logn, L + K
    assert np.array_equal(ctx.key_export(B.HESPMV_KEY_SECRET).reshape(LK, N), orc.s)
    pk = ctx.key_export(B.HESPMV_KEY_PUBLIC).reshape(2, L, N)
    assert np.array_equal(pk[0], orc.pk[0]) and np.array_equal(pk[1], orc.pk[1])
    assert np.array_equal(ctx.key_export(B.HESPMV_KEY_RELIN).reshape(orc.rlk.shape), orc.rlk)
    for g, key in orc.gk.items():
        assert np.array_equal(ctx.key_export(B.HESPMV_KEY_GALOIS, g).reshape(key.shape), key), g


def test_keys_parity_two_special_primes():
    # alpha = 2 digits and K = 2, small ring
    N = 1 << 8
    t = plain_modulus(N, 1 << 16)
    ctx, orc = make_pair(8, 8, 2, 4, t, seed=5, steps=[1, 3, 7])
    assert np.array_equal(ctx.key_export(B.HESPMV_KEY_RELIN).reshape(orc.rlk.shape), orc.rlk)
    for g, key in orc.gk.items():
        assert np.array_equal(ctx.key_export(B.HESPMV_KEY_GALOIS, g).reshape(key.shape), key)


def _random_slot_ciphertexts(ctx, orc, n, seed):
    """n ciphertexts of random slot vectors, encrypted by the library through
    a one-chunk-per-ciphertext plan; the oracle encrypts the same values."""
    N = orc.p.N
    rng = np.random.default_rng(seed)
    h = N // 2
    rows = n * h
    # a diagonal-like matrix whose CSSC has n aligned columns of height h ...
    # simpler: encrypt the vector operand of a plan with n chunks of h x 1
    vals = rng.integers(0, orc.p.t, size=(n, h), dtype=np.int64)
    # build a CSR with h rows and n columns fully dense: chunk k = column k
    rowptr = np.arange(0, h * n + 1, n, dtype=np.int64)
    colidx = np.tile(np.arange(n, dtype=np.int32), h)
    m = ctx.encode_cssc(h, n, rowptr, colidx, vals.T.reshape(-1))
    assert m.n_chunks == n and all(c == 1 for c in m.chunks()[1])
    A = ctx.encrypt(m, B.HESPMV_MATRIX, seed=seed)
    oc = [orc.encrypt(orc.encode(vals[k]), seed, k) for k in range(n)]
    got = A.download()
    for k in range(n):
        assert np.array_equal(got[k], oc[k]), k
    return A, oc, vals


@pytest.fixture(scope="module", params=[10, 12])
def pair_small(request):
    # 2^10 runs the unfused key switch, 2^12 the fused one (alpha = 2, K = 2)
    logn = request.param
    N = 1 << logn
    t = plain_modulus(N, 1 << 20)
    return make_pair(logn, 5, 2, 3, t, seed=11, steps=[1, 2, 5, 100, 511])


def test_encrypt_and_ops_parity(pair_small):
    ctx, orc = pair_small
    A, oc, vals = _random_slot_ciphertexts(ctx, orc, 3, 21)
    L, N = orc.p.L, orc.p.N
    CT = 2 * L * N
    a_ptr = A.ptr
    b_ptr = A.ptr + CT * 8
    # add
    out = torch.zeros(CT, dtype=torch.int64, device="cuda")
    ctx.he_add(a_ptr, b_ptr, out.data_ptr())
    assert np.array_equal(host(out).reshape(2, L, N), orc.add(oc[0], oc[1]))
    # tensor
    d = torch.zeros(3 * L * N, dtype=torch.int64, device="cuda")
    ctx.he_tensor(a_ptr, b_ptr, d.data_ptr())
    od = orc.tensor(oc[0], oc[1])
    assert np.array_equal(host(d).reshape(3, L, N), od)
    # key switch of d2 with the relinearisation key
    ks = torch.zeros(CT, dtype=torch.int64, device="cuda")
    ctx.keyswitch(d.data_ptr() + 2 * L * N * 8, 0, ks.data_ptr())
    assert np.array_equal(host(ks).reshape(2, L, N), orc.keyswitch(od[2], orc.rlk))
    # relinearisation and HE-Mult
    ctx.he_relin(d.data_ptr(), out.data_ptr())
    om = orc.relinearize(od)
    assert np.array_equal(host(out).reshape(2, L, N), om)
    out2 = torch.zeros(CT, dtype=torch.int64, device="cuda")
    ctx.he_mult(a_ptr, b_ptr, out2.data_ptr())
    assert np.array_equal(host(out2).reshape(2, L, N), om)
    # rotations (power-of-two chains)
    for k in (1, 2, 5, 100, 511):
        ctx.he_rotate(a_ptr, k, out.data_ptr())
        assert np.array_equal(host(out).reshape(2, L, N), orc.rotate(oc[0], k)), k
    # mask multiply
    for r in (1, 37, N // 2):
        ctx.he_cmult_mask(a_ptr, r, out.data_ptr())
        assert np.array_equal(host(out).reshape(2, L, N), orc.cmult(oc[0], S.mask_ntt(orc, r)))
    # decryption of a product
    slots = ctx.decrypt_slots(A, 0)
    assert np.array_equal(slots[:N // 2], vals[0] % orc.p.t)


def test_rotation_exact_policy_parity():
    N = 1 << 9
    t = plain_modulus(N, 1 << 18)
    ctx, orc = make_pair(9, 3, 1, 3, t, seed=3, steps=[3, 17, 200], policy="exact")
    A, oc, vals = _random_slot_ciphertexts(ctx, orc, 1, 4)
    CT = 2 * 3 * N
    out = torch.zeros(CT, dtype=torch.int64, device="cuda")
    for k in (3, 17, 200):
        ctx.he_rotate(A.ptr, k, out.data_ptr())
        assert np.array_equal(host(out).reshape(2, 3, N), orc.rotate(oc[0], k, "exact"))


def run_spmv_pair(ctx, orc, A, x, kseed=1, policy="pow2"):
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, orc.p.slots)
    ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=2)
    cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=3)
    y = ctx.spmv(m, ca, cx)
    torch.cuda.synchronize()
    oa = S.encrypt_matrix(orc, plan, 2)
    ox = S.encrypt_vector(orc, plan, x, 3)
    ga, gx = ca.download(), cx.download()
    for k in range(len(oa)):
        assert np.array_equal(ga[k], oa[k]) and np.array_equal(gx[k], ox[k]), k
    ores = S.spmv(orc, plan, oa, ox, policy)
    gy = y.download()
    for p_ in range(len(ores)):
        assert np.array_equal(gy[p_], ores[p_]), p_
    out = ctx.decrypt(m, y)
    return m, y, out, S.decrypt_result(orc, plan, ores)


def test_spmv_small_partitions_parity():
    N = 1 << 6
    t = plain_modulus(N, 1 << 20)
    A, x = synth.small_matrix(9, 70, 50, 400, -9, 9)
    from paper_2603_04742_gb300.api import Context
    ctx = Context(6, 3, 1, 3, t, slots=24)
    orc = Oracle(Params(log2n=6, L=3, K=1, dnum=3, t=t, slots=24))
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    steps = m.rotation_steps()
    ctx.keygen(4, steps)
    gels = set()
    for k in steps:
        gels.update(orc.rotation_elements(k))
    orc.keygen(4, sorted(gels))
    m2, y, out, oout = run_spmv_pair(ctx, orc, A, x)
    assert m2.n_parts == 3
    assert list(out) == list(A.matvec(x)) == list(oout)


@pytest.mark.parametrize("logn,rows,nnz,slots", [(6, 960, 9000, 32), (12, 640, 3000, 16)])
def test_spmv_many_chunks_ragged_batches_parity(logn, rows, nnz, slots):
    """More chunks than one batch of every stage holds (encryption 64, HE-Mult
    32, totalSum rounds 64 ciphertexts), with a ragged last batch in each;
    2^6 runs the unfused key switch, 2^12 the fused one."""
    t = plain_modulus(1 << logn, 1 << 20)
    A, x = synth.small_matrix(5 if logn == 6 else 6, rows, 64 if logn == 6 else 96, nnz, -9, 9)
    from paper_2603_04742_gb300.api import Context
    ctx = Context(logn, 3, 1, 3, t, slots=slots)
    orc = Oracle(Params(log2n=logn, L=3, K=1, dnum=3, t=t, slots=slots))
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    h, c, _ = m.chunks()
    assert m.n_chunks > 64 and m.n_chunks % 64 and m.n_chunks % 32 and int((c > 1).sum()) > 64
    steps = m.rotation_steps()
    ctx.keygen(4, steps)
    orc.keygen(4, sorted({g for k in steps for g in orc.rotation_elements(k)}))
    m2, y, out, oout = run_spmv_pair(ctx, orc, A, x)
    assert list(out) == list(A.matvec(x)) == list(oout)
    # HE-Mult groups and totalSum rotation groups alternating over two streams
    want = y.download()
    ctx.set_tuning(7, 10, 0, 0, 0, 0, 2)
    ca = ctx.encrypt(m2, B.HESPMV_MATRIX, seed=2)
    cx = ctx.encrypt(m2, B.HESPMV_VECTOR, x=x, seed=3)
    for _ in range(2):   # capture, then replay
        assert np.array_equal(ctx.spmv(m2, ca, cx).download(), want)
    ctx.set_tuning(0, 0, 0, 0)


@pytest.mark.parametrize("policy", ["pow2", "exact"])
def test_spmv_c1_parity(policy):
    logn, L, K, dnum, t = synth.RING["c1"]
    A, x = synth.workload("c1")
    from paper_2603_04742_gb300.api import Context
    probe = Context(logn, L, K, dnum, t, device=-1, torch_alloc=False)
    steps = probe.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals).rotation_steps()
    ctx, orc = make_pair(logn, L, K, dnum, t, seed=1, steps=steps, policy=policy)
    m, y, out, oout = run_spmv_pair(ctx, orc, A, x, policy=policy)
    assert list(out) == list(A.matvec(x))


def test_spmv_c2_parity():
    logn, L, K, dnum, t = synth.RING["c2"]
    A, x = synth.workload("c2")
    from paper_2603_04742_gb300.api import Context
    probe = Context(logn, L, K, dnum, t, device=-1, torch_alloc=False)
    steps = probe.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals).rotation_steps()
    ctx, orc = make_pair(logn, L, K, dnum, t, seed=1, steps=steps)
    m, y, out, oout = run_spmv_pair(ctx, orc, A, x)
    assert list(out) == list(A.matvec(x))


def test_spmv_c3_full_size_parity_and_tolerance():
    """The bench's workload: 27-point stencil, N = 2^15, 8 + 2 primes."""
    logn, L, K, dnum, t = synth.RING["c3"]
    A, xf = synth.workload("c3")
    Af = A.vals.copy()
    A.vals = synth.quantize(Af)
    x = synth.quantize(xf)
    ctx, orc = make_pair(logn, L, K, dnum, t, seed=1, steps=[])
    m, y, out, oout = run_spmv_pair(ctx, orc, A, x)
    exact = A.matvec(x)
    assert list(out) == list(exact)
    # the autotuned schedule of this workload: groups of 14 and 13 on two streams
    ref = y.download()
    ctx.set_tuning(14, 0, 0, 0, 0, 0, 2)
    ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=2)
    cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=3)
    for _ in range(2):
        assert np.array_equal(ctx.spmv(m, ca, cx).download(), ref)
    ctx.set_tuning(0, 0, 0, 0)
    # fixed point: result scale 2^30, tolerance 1e-3 relative in the max norm
    A.vals = Af
    yref = A.matvec(xf)
    yhat = np.asarray(out, dtype=np.float64) / float(1 << 30)
    assert np.max(np.abs(yhat - yref)) <= 1e-3 * np.max(np.abs(yref))


def _uniform_rows_matrix(seed, rows, cols, per_row):
    """Every row holds exactly per_row non-zeros: all chunks are one column
    wide (c = 1) when rows fill whole partitions, so no rotation runs."""
    g = np.random.default_rng(seed)
    colidx = np.concatenate([np.sort(g.choice(cols, per_row, replace=False)) for _ in range(rows)])
    vals = g.integers(-15, 16, size=rows * per_row)
    vals[vals == 0] = 7
    rowptr = np.arange(rows + 1, dtype=np.int64) * per_row
    x = g.integers(-15, 16, size=cols)
    return synth.CSR(rows, cols, rowptr, colidx.astype(np.int32), vals.astype(np.int64)), x


def test_spmv_no_rotation_partitions_parity():
    """A matrix whose chunks are all one column wide (no rotation anywhere)
    over two partitions: the result matches the oracle's sequential
    Algorithm 4 bit for bit on the device path, the graph replay and every
    host-buffer path."""
    logn, L, K, dnum, t = synth.RING["c1"]
    A, x = _uniform_rows_matrix(77, 2 * (1 << (logn - 1)), 3000, 5)   # two partitions
    ctx, orc = make_pair(logn, L, K, dnum, t, seed=1, steps=[])
    m, y, out, oout = run_spmv_pair(ctx, orc, A, x)
    assert m.n_rot == 0 and m.n_parts == 2
    assert list(out) == list(A.matvec(x)) == list(oout)
    ref = y.download()
    # two streams: HE-Mult groups alternating between them, one group
    # spanning the partition boundary (G = 3), one not (G = 5)
    for G in (3, 5):
        ctx.set_tuning(G, 0, 0, 0, 0, 0, 2)
        for _ in range(2):
            assert np.array_equal(ctx.spmv(m, ctx.encrypt(m, B.HESPMV_MATRIX, seed=2),
                                           ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=3)).download(), ref), G
    ctx.set_tuning(0, 0, 0, 0)
    ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=2)
    cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=3)
    for _ in range(2):   # capture, then replay
        assert np.array_equal(ctx.spmv(m, ca, cx).download(), ref)
    words, _ = ctx.ct_packed_words()
    pA, pX = ctx.ct_pack(ca.download()), ctx.ct_pack(cx.download())
    py = np.zeros((m.n_parts, words), dtype=np.uint64)
    hy = np.zeros_like(ref)
    for groups in (1, 3, 0):
        ctx.set_upload_groups(groups)
        ctx.spmv_host(m, ca.download(), cx.download(), hy)
        assert np.array_equal(hy, ref), groups
        ctx.spmv_host_packed(m, pA, pX, py)
        assert np.array_equal(ctx.ct_unpack(py), ref), groups
        stream = torch.cuda.Stream()
        for _ in range(3):
            ctx.spmv_host_packed_async(m, pA, pX, py, stream=stream)
        stream.synchronize()
        assert np.array_equal(ctx.ct_unpack(py), ref), groups
    ctx.device_status()


def test_spmv_host_buffers_and_batched_match():
    logn, L, K, dnum, t = synth.RING["c1"]
    from paper_2603_04742_gb300.api import Context
    ctx = Context(logn, L, K, dnum, t)
    ctx.keygen(9)
    insts = [synth.small_matrix(s, 300, 280, 900 + 200 * s) for s in range(3)]
    ms, As, Xs, ys = [], [], [], []
    for A, x in insts:
        m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
        ms.append(m)
        As.append(ctx.encrypt(m, B.HESPMV_MATRIX, seed=5))
        Xs.append(ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=6))
        ys.append(ctx.spmv(m, As[-1], Xs[-1]))
    yb = ctx.spmv_batched(ms, As, Xs)
    for i, (A, x) in enumerate(insts):
        assert np.array_equal(yb[i].download(), ys[i].download())
        assert list(ctx.decrypt(ms[i], yb[i])) == list(A.matvec(x))
        hA, hX = As[i].download(), Xs[i].download()
        hy = np.zeros((ms[i].n_parts, 2, L, 1 << logn), dtype=np.uint64)
        ctx.spmv_host(ms[i], hA, hX, hy)
        assert np.array_equal(hy, ys[i].download())


def _set_packed_residue(packed, limb_words, limb, k, W, v):
    """Overwrite residue k of limb `limb` in one packed ciphertext with v."""
    lo = limb * limb_words * 64 + k * W
    for w in range(lo // 64, (lo + W - 1) // 64 + 1):
        sh = lo - 64 * w
        m = (((1 << W) - 1) << sh if sh >= 0 else ((1 << W) - 1) >> -sh) & ((1 << 64) - 1)
        part = (v << sh if sh >= 0 else v >> -sh) & m
        packed[w] = np.uint64((int(packed[w]) & ~m & ((1 << 64) - 1)) | part)


def test_spmv_host_packed_matches_device_path():
    """The packed host path (upload of W-bit residues, unpack kernels per
    upload group, pack kernel for the result) gives the packed form of the
    device path's result ciphertexts, bit for bit, on chunk counts that leave
    ragged upload groups; a residue >= q is reported and leaves the context
    usable."""
    logn, L, K, dnum, t = synth.RING["c1"]
    from paper_2603_04742_gb300.api import Context
    ctx = Context(logn, L, K, dnum, t, slots=256)
    ctx.keygen(12)
    words, W = ctx.ct_packed_words()
    for seed, (rows, cols, nnz) in enumerate([(300, 280, 900), (700, 640, 5000), (1, 1, 1)]):
        A, x = synth.small_matrix(seed, rows, cols, nnz)
        m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
        ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=21 + seed)
        cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=31 + seed)
        y = ctx.spmv(m, ca, cx).download()
        pA, pX = ctx.ct_pack(ca.download()), ctx.ct_pack(cx.download())
        py = np.zeros((m.n_parts, words), dtype=np.uint64)
        hy = np.zeros_like(y)
        # upload groups: one, ragged, more groups than chunks, the default
        for groups in (1, 3, 64, 0):
            ctx.set_upload_groups(groups)
            py[:] = 0
            ctx.spmv_host_packed(m, pA, pX, py)
            assert np.array_equal(py, ctx.ct_pack(y)), (seed, m.n_chunks, groups)
            ctx.spmv_host(m, ca.download(), cx.download(), hy)
            assert np.array_equal(hy, y), (seed, m.n_chunks, groups)
        assert np.array_equal(ctx.ct_unpack(py), y)
        assert list(ctx.decrypt(m, ctx.spmv(m, ca, cx))) == list(A.matvec(x))
    # an unreduced residue in the last chunk's vector ciphertext
    q = ctx.moduli()[0]
    bad = pX.copy()
    _set_packed_residue(bad[-1], words // (2 * L), 2 * L - 1, 3, W, q[L - 1])
    with pytest.raises(B.HespmvError) as ei:
        ctx.spmv_host_packed(m, pA, bad, py)
    assert ei.value.code == B.HESPMV_E_INVALID
    ctx.device_status()
    ctx.spmv_host_packed(m, pA, pX, py)
    assert np.array_equal(py, ctx.ct_pack(y))


def test_spmv_host_packed_async_pipeline():
    """Pipelined packed evaluations: calls on two instances in flight at once
    (every staging slot reused, uploads overlapping earlier
    calls' compute) give the device path's results bit for bit; a bad residue
    shows up in the device status."""
    logn, L, K, dnum, t = synth.RING["c1"]
    from paper_2603_04742_gb300.api import Context
    ctx = Context(logn, L, K, dnum, t, slots=256)
    ctx.keygen(13)
    words, W = ctx.ct_packed_words()
    inst = []
    for seed, (rows, cols, nnz) in enumerate([(700, 640, 5000), (300, 280, 900)]):
        A, x = synth.small_matrix(40 + seed, rows, cols, nnz)
        m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
        ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=51 + seed)
        cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=61 + seed)
        y = ctx.spmv(m, ca, cx).download()
        inst.append((m, ctx.ct_pack(ca.download()), ctx.ct_pack(cx.download()), ctx.ct_pack(y)))
    stream = torch.cuda.Stream()
    outs = []
    for r in range(6):
        m, pA, pX, py = inst[r % 2]
        out = np.zeros((m.n_parts, words), dtype=np.uint64)
        outs.append((out, py))
        ctx.spmv_host_packed_async(m, pA, pX, out, stream=stream)
    stream.synchronize()
    for r, (out, py) in enumerate(outs):
        assert np.array_equal(out, py), r
    ctx.device_status()
    # a synchronous call in between keeps its own staging
    m, pA, pX, py = inst[0]
    out = np.zeros_like(py)
    ctx.spmv_host_packed(m, pA, pX, out)
    assert np.array_equal(out, py)
    bad = pX.copy()
    _set_packed_residue(bad[0], words // (2 * L), L, 9, W, ctx.moduli()[0][0])
    ctx.spmv_host_packed_async(m, pA, bad, out, stream=stream)
    stream.synchronize()
    with pytest.raises(B.HespmvError) as ei:
        ctx.device_status()
    assert ei.value.code == B.HESPMV_E_INVALID
    ctx.spmv_host_packed_async(m, pA, pX, out, stream=stream)
    stream.synchronize()
    ctx.device_status()
    assert np.array_equal(out, py)


def test_spmv_edge_cases():
    logn, L, K, dnum, t = synth.RING["c1"]
    from paper_2603_04742_gb300.api import Context
    ctx = Context(logn, L, K, dnum, t, slots=64)
    ctx.keygen(2)
    N = 1 << logn
    cases = []
    # one non-zero; an empty row block in the middle; a full row; rows == slots
    cases.append((synth.CSR(3, 3, np.array([0, 0, 1, 1]), np.array([2], np.int32),
                            np.array([7])), np.array([1, 2, 3])))
    r = np.zeros(129, dtype=np.int64)
    r[65:] = 1
    rowptr = np.concatenate([[0], np.cumsum(r)])
    cases.append((synth.CSR(129, 5, rowptr, np.zeros(64, np.int32), np.arange(64)),
                  np.array([3, 0, 0, 0, 0])))
    cases.append((synth.CSR(2, 64, np.array([0, 64, 64]), np.arange(64, dtype=np.int32),
                            np.ones(64, dtype=np.int64)), np.arange(64)))
    A, x = synth.small_matrix(1, 64, 64, 64 * 64)   # dense 64 x 64: c spans several blocks
    cases.append((A, x))
    for A, x in cases:
        m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
        ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=1)
        cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=2)
        y = ctx.spmv(m, ca, cx)
        assert list(ctx.decrypt(m, y)) == list(A.matvec(x))
    # an all-zero matrix gives zero ciphertexts and zero rows
    m = ctx.encode_cssc(4, 4, [0, 0, 0, 0, 0], [], [])
    ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=1)
    cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=np.zeros(4, np.int64), seed=2)
    y = ctx.spmv(m, ca, cx)
    assert list(ctx.decrypt(m, y)) == [0, 0, 0, 0]
    assert not np.any(y.download())


def test_graph_replay_matches_eager():
    """Evaluations replayed from a CUDA graph equal eager launches, also when
    the input ciphertexts in the same buffers change between replays."""
    logn, L, K, dnum, t = synth.RING["c1"]
    from paper_2603_04742_gb300.api import Context
    ctx = Context(logn, L, K, dnum, t)
    ctx.keygen(4)
    A, x = synth.small_matrix(12, 400, 300, 2500)
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=1)
    cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=2)
    ctx.set_graphs(False)
    y_eager = ctx.spmv(m, ca, cx).download()
    ctx.set_graphs(True)
    y = ctx.spmv(m, ca, cx)
    for _ in range(3):
        ctx.spmv(m, ca, cx, y=y)
        assert np.array_equal(y.download(), y_eager)
    # new inputs in the same device buffers: the replay reads them
    x2 = (x * 3 + 1) % 7 - 3
    cx2 = ctx.encrypt(m, B.HESPMV_VECTOR, x=x2, seed=9)
    cx.upload(cx2.download())
    ctx.spmv(m, ca, cx, y=y)
    assert list(ctx.decrypt(m, y)) == list(A.matvec(x2))


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_spmv_plain_matrix_parity(name):
    """Plaintext-matrix mode: the trivial ciphertexts equal the oracle's
    plaintexts, the result ciphertexts equal the oracle's, and decrypt = A.x."""
    logn, L, K, dnum, t = synth.RING[name]
    A, x = synth.workload(name)
    from paper_2603_04742_gb300.api import Context
    probe = Context(logn, L, K, dnum, t, device=-1, torch_alloc=False)
    steps = probe.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals).rotation_steps()
    ctx, orc = make_pair(logn, L, K, dnum, t, seed=2, steps=steps)
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    pa = ctx.encode_matrix_plain(m)
    cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=3)
    y = ctx.spmv_ptmatrix(m, pa, cx)
    torch.cuda.synchronize()
    plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, orc.p.slots)
    pts = S.encode_matrix_plain(orc, plan)
    gp = pa.download()
    for k in range(len(pts)):
        assert np.array_equal(gp[k][0], pts[k]) and not np.any(gp[k][1])
    ores = S.spmv_plain_matrix(orc, plan, pts, S.encrypt_vector(orc, plan, x, 3))
    gy = y.download()
    for p_ in range(len(ores)):
        assert np.array_equal(gy[p_], ores[p_])
    assert list(ctx.decrypt(m, y)) == list(A.matvec(x))


def test_outputs_fully_written_over_poisoned_buffers():
    """Every output word is written: result buffers start filled with the
    sentinel 2^64 - 1 (never a residue) and must hold the oracle's values."""
    logn, L, K, dnum, t = synth.RING["c1"]
    A, x = synth.workload("c1")
    from paper_2603_04742_gb300.api import Context, CtBatch
    probe = Context(logn, L, K, dnum, t, device=-1, torch_alloc=False)
    steps = probe.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals).rotation_steps()
    ctx, orc = make_pair(logn, L, K, dnum, t, seed=1, steps=steps)
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=2)
    cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=3)
    N, CT = 1 << logn, 2 * L * (1 << logn)
    sentinel = np.full(m.n_parts * CT, np.iinfo(np.uint64).max, dtype=np.uint64)
    y = CtBatch.create(ctx, m.n_parts)
    y.upload(sentinel)
    ctx.set_graphs(False)
    ctx.spmv(m, ca, cx, y=y)
    torch.cuda.synchronize()
    plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, orc.p.slots)
    ores = S.spmv(orc, plan, S.encrypt_matrix(orc, plan, 2), S.encrypt_vector(orc, plan, x, 3))
    got = y.download()
    for p_ in range(len(ores)):
        assert np.array_equal(got[p_], ores[p_]), p_
    # the primitives' outputs too
    out = torch.from_numpy(np.full(3 * L * N, -1, dtype=np.int64)).cuda()
    ctx.he_tensor(ca.ptr, cx.ptr, out.data_ptr())
    assert np.array_equal(host(out).reshape(3, L, N), orc.tensor(*[S.encrypt_matrix(orc, plan, 2)[0],
                                                                   S.encrypt_vector(orc, plan, x, 3)[0]]))
    out.fill_(-1)
    ctx.he_mult(ca.ptr, cx.ptr, out.data_ptr())
    got = host(out)
    assert np.all(got[:CT] != np.iinfo(np.uint64).max) and np.all(got[CT:] == np.iinfo(np.uint64).max)


@pytest.mark.parametrize("split,rows_tma", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_fused_keyswitch_both_splits_n2048(split, rows_tma):
    """N = 2^11, the smallest fused ring, under both NTT splits (2^5 x 2^6 and
    2^6 x 2^5): HE-Mult and a rotation bit-exact with the oracle."""
    N = 1 << 11
    t = plain_modulus(N, 1 << 18)
    ctx, orc = make_pair(11, 4, 2, 2, t, seed=5, steps=[1, 9])
    ctx.set_tuning(0, 0, split, rows_tma)
    A, oc, vals = _random_slot_ciphertexts(ctx, orc, 2, 13)
    L, CT = 4, 2 * 4 * N
    out = torch.zeros(CT, dtype=torch.int64, device="cuda")
    ctx.he_mult(A.ptr, A.ptr + CT * 8, out.data_ptr())
    assert np.array_equal(host(out).reshape(2, L, N), orc.mult(oc[0], oc[1]))
    ctx.he_rotate(A.ptr, 9, out.data_ptr())
    assert np.array_equal(host(out).reshape(2, L, N), orc.rotate(oc[0], 9))
    ctx.device_status()


def test_row_pass_forms_identical_n32768():
    """At the stencil ring the TMA-fed row pass (both NTT splits) gives the
    same HE-Mult as the oracle-checked default form."""
    from paper_2603_04742_gb300.api import Context
    logn, L, K, dnum, t = synth.RING["c3"]
    A, xf = synth.workload("c3")
    A.vals = synth.quantize(A.vals)
    x = synth.quantize(xf)
    ctx = Context(logn, L, K, dnum, t)
    ctx.keygen(1, [])
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=2)
    cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=3)
    outs = []
    for split, tma in ((0, 0), (0, 1), (1, 1)):
        ctx.set_tuning(0, 0, split, tma)
        y = ctx.spmv(m, ca, cx)
        torch.cuda.synchronize()
        outs.append(y.download())
    ctx.device_status()
    assert all(np.array_equal(outs[0], o) for o in outs[1:])
    assert list(ctx.decrypt(m, y)) == list(A.matvec(x))
