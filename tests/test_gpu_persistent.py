"""The persistent evaluation: one launch per SpMV (or batch) whose CTAs take
work tiles from a device queue and wait, bounded in time, for the tiles they
depend on.  Its result ciphertexts must equal the oracle's (Algorithms 1 and
4) bit for bit, whatever the number of CTAs (one CTA exercises the ordering
argument: every dependency is a lower tile), the HE-Mult group size and the
rotation-key policy; a wait that cannot complete is reported as
HESPMV_E_TIMEOUT and leaves the context usable."""
import numpy as np
import pytest

from oracle import spmv as S
from oracle.bgv import Oracle
from oracle.params import Params, plain_modulus
from paper_2603_04742_gb300 import binding as B
from paper_2603_04742_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _pair(logn, L, K, dnum, t, steps, policy="pow2", slots=0, seed=3):
    from paper_2603_04742_gb300.api import Context
    ctx = Context(logn, L, K, dnum, t, rot_policy=policy, slots=slots)
    orc = Oracle(Params(log2n=logn, L=L, K=K, dnum=dnum, t=t, slots=slots))
    ctx.keygen(seed, steps)
    orc.keygen(seed, sorted({g for k in steps for g in orc.rotation_elements(k, policy)}))
    return ctx, orc


def _oracle_result(orc, A, x, policy, sa=2, sx=3):
    plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, orc.p.slots)
    return np.stack(S.spmv(orc, plan, S.encrypt_matrix(orc, plan, sa),
                           S.encrypt_vector(orc, plan, x, sx), policy))


def _steps(logn, L, K, dnum, t, mats, slots=0):
    from paper_2603_04742_gb300.api import Context
    probe = Context(logn, L, K, dnum, t, device=-1, torch_alloc=False, slots=slots)
    return sorted({s for A in mats for s in probe.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx,
                                                              A.vals).rotation_steps()})


@pytest.mark.parametrize("policy", ["pow2", "exact"])
def test_persistent_c1_matches_oracle_any_cta_count(policy):
    """c1 (N = 2^12, 3 chunks with rotations) under both rotation-key
    policies; 1, 3 and all resident CTAs; HE-Mult groups of 1, 2 and 16."""
    logn, L, K, dnum, t = synth.RING["c1"]
    A, x = synth.workload("c1")
    ctx, orc = _pair(logn, L, K, dnum, t, _steps(logn, L, K, dnum, t, [A]), policy)
    want = _oracle_result(orc, A, x, policy)
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    assert m.n_rot > 0
    ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=2)
    cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=3)
    for G, blocks in [(0, 0), (1, 1), (2, 3), (16, 0)]:
        ctx.set_tuning(G, 0, 0, 0, 1, blocks)
        y = ctx.spmv(m, ca, cx)
        torch.cuda.synchronize()
        assert np.array_equal(y.download(), want), (G, blocks)
    ctx.device_status()
    assert list(ctx.decrypt(m, y)) == list(A.matvec(x))


def test_persistent_partitions_ragged_groups_and_graph_replay():
    """Several partitions (one of them empty), HE-Mult groups that do not
    divide the chunk count, both NTT splits, eager launches and graph
    replays over poisoned result buffers: all equal the oracle."""
    from paper_2603_04742_gb300.api import CtBatch
    logn, slots = 12, 160
    t = plain_modulus(1 << logn, 1 << 20)
    A, x = synth.small_matrix(21, 500, 400, 4000, -9, 9)
    # rows 160 .. 319 empty: the second partition has no chunk
    keep = (np.repeat(np.arange(A.rows), np.diff(A.rowptr)) // slots) != 1
    rows = np.repeat(np.arange(A.rows), np.diff(A.rowptr))[keep]
    A = synth.CSR(A.rows, A.cols, np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=A.rows))]),
                  A.colidx[keep], A.vals[keep])
    ctx, orc = _pair(logn, 3, 1, 3, t, _steps(logn, 3, 1, 3, t, [A], slots), slots=slots)
    want = _oracle_result(orc, A, x, "pow2")
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    assert m.n_parts == 4 and m.n_chunks > 7
    ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=2)
    cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=3)
    y = CtBatch.create(ctx, m.n_parts)
    sentinel = np.full(want.size, np.iinfo(np.uint64).max, dtype=np.uint64)
    for split in (0, 1):
        for graphs in (False, True):
            ctx.set_graphs(graphs)
            ctx.set_tuning(3, 0, split, 0, 1, 0)
            for _ in range(2):   # capture, then replay
                y.upload(sentinel)
                ctx.spmv(m, ca, cx, y=y)
                torch.cuda.synchronize()
                assert np.array_equal(y.download(), want), (split, graphs)
    ctx.device_status()
    assert list(ctx.decrypt(m, y)) == list(A.matvec(x))


def test_persistent_batched_uneven_instances_equal_staged():
    """A batch of uneven SpMVs at N = 2^13 in one persistent launch equals the
    staged batched evaluation (itself oracle-checked) ciphertext for
    ciphertext, and decrypts to A.x."""
    from paper_2603_04742_gb300.api import Context
    g = np.random.default_rng(5)
    t = 114689
    ctx = Context(13, 4, 2, 2, t)
    insts = []
    for _ in range(7):
        n = int(g.integers(100, 2500))
        A = synth.uniform_positions(g, n, n, int(g.integers(n, 8 * n)), -15, 15)
        insts.append((A, g.integers(-15, 16, size=n, dtype=np.int64)))
    ms = [ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals) for A, _ in insts]
    ctx.keygen(4, sorted({s for m in ms for s in m.rotation_steps()}))
    As = [ctx.encrypt(m, B.HESPMV_MATRIX, seed=10 + i) for i, m in enumerate(ms)]
    Xs = [ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=40 + i) for i, (m, (_, x)) in enumerate(zip(ms, insts))]
    ref = [y.download() for y in ctx.spmv_batched(ms, As, Xs)]
    for G in (4, 64):
        ctx.set_tuning(G, 0, 0, 0, 1, 0)
        ys = ctx.spmv_batched(ms, As, Xs)
        torch.cuda.synchronize()
        for i, (y, r) in enumerate(zip(ys, ref)):
            assert np.array_equal(y.download(), r), (G, i)
    for m, y, (A, x) in zip(ms, ys, insts):
        assert list(ctx.decrypt(m, y)) == list(A.matvec(x))


def test_persistent_dependency_wait_times_out_and_context_survives():
    from paper_2603_04742_gb300.api import Context
    logn, L, K, dnum, t = synth.RING["c1"]
    ctx = Context(logn, L, K, dnum, t)
    ctx.keygen(1)
    rc, code = ctx.selftest_persist_timeout()
    assert rc == B.HESPMV_E_TIMEOUT and code == 3
    ctx.device_status()   # cleared
    A, x = synth.small_matrix(3, 300, 300, 1500)
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    ctx.set_tuning(0, 0, 0, 0, 1, 0)
    ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=1)
    cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=2)
    assert list(ctx.decrypt(m, ctx.spmv(m, ca, cx))) == list(A.matvec(x))


def test_persistent_degenerate_matrices():
    """The persistent program of an all-zero matrix (no chunk: zero result
    ciphertexts), of a single non-zero, and a batch mixing them with an
    ordinary matrix, over poisoned result buffers."""
    from paper_2603_04742_gb300.api import Context, CtBatch
    logn, L, K, dnum, t = synth.RING["c1"]
    ctx = Context(logn, L, K, dnum, t, slots=64)
    ctx.keygen(2)
    ctx.set_tuning(0, 0, 0, 0, 1, 0)
    zero = synth.CSR(4, 4, np.zeros(5, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int64))
    one = synth.CSR(3, 3, np.array([0, 0, 1, 1]), np.array([2], np.int32), np.array([7]))
    big, xb = synth.small_matrix(4, 200, 150, 900)
    cases = [(zero, np.zeros(4, np.int64)), (one, np.array([1, 2, 3])), (big, xb)]
    ms, As, Xs = [], [], []
    for A, x in cases:
        m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
        ms.append(m)
        As.append(ctx.encrypt(m, B.HESPMV_MATRIX, seed=1))
        Xs.append(ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=2))
    CT = 2 * L * (1 << logn)
    for single in (True, False):
        ys = [CtBatch.create(ctx, m.n_parts) for m in ms]
        for y, m in zip(ys, ms):
            y.upload(np.full(m.n_parts * CT, np.iinfo(np.uint64).max, dtype=np.uint64))
        if single:
            for m, a, xx, y in zip(ms, As, Xs, ys):
                ctx.spmv(m, a, xx, y=y)
        else:
            ctx.spmv_batched(ms, As, Xs, ys)
        torch.cuda.synchronize()
        assert not np.any(ys[0].download())
        for (A, x), m, y in zip(cases, ms, ys):
            assert list(ctx.decrypt(m, y)) == list(A.matvec(x)), single
    ctx.device_status()
