"""Oracle parity on the rings of the batched and serving workloads.

The batched ring (N = 2^14, 5 + 1 primes, dnum 5, t = 1146881) and the serving
ring (N = 2^15, 8 + 2 primes, dnum 4, t = 1179649, power-of-two Galois keys)
are checked against the CPU oracle's Algorithms 1 and 4, residue for residue:

* a batched evaluation of uneven instances, some with chunks of several
  columns, so that totalSum rotations (Algorithm 4) run on the batched ring;
* every schedule the autotuner times on that batch;
* one SpMV on the serving ring whose chunks span three or more column blocks,
  so that rotations by power-of-two chains run at N = 2^15;
* a served mix on the serving ring (continuous batching), every result
  compared with the oracle, not with another device evaluation.

Instances are shaped like the workloads (uniform positions, integers in
[-15, 15]) but small enough that the oracle finishes each in well under a
minute."""
import time

import numpy as np
import pytest

from oracle import spmv as S
from oracle.bgv import Oracle
from oracle.params import Params
from paper_2603_04742_gb300 import binding as B
from paper_2603_04742_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _oracle(ring, steps, seed):
    logn, L, K, dnum, t = ring
    orc = Oracle(Params(log2n=logn, L=L, K=K, dnum=dnum, t=t))
    orc.keygen(seed, sorted({g for k in steps for g in orc.rotation_elements(k)}))
    return orc


def _instances(seed, shapes):
    g = np.random.default_rng(seed)
    out = []
    for n, nnz in shapes:
        A = synth.uniform_positions(g, n, n, nnz, -15, 15)
        x = g.integers(-15, 16, size=n, dtype=np.int64)
        out.append((A, x))
    return out


def _oracle_results(orc, insts, seeds):
    """Oracle ciphertexts of each instance's result (the same encryption
    seeds as the library's)."""
    res = []
    for (A, x), (sa, sx) in zip(insts, seeds):
        plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, orc.p.slots)
        res.append(np.stack(S.spmv(orc, plan, S.encrypt_matrix(orc, plan, sa),
                                   S.encrypt_vector(orc, plan, x, sx))))
    return res


def _assert_equal_results(ys, want, what):
    for i, (y, w) in enumerate(zip(ys, want)):
        got = y.download()
        assert got.shape == w.shape, (what, i)
        assert np.array_equal(got, w), (what, i)


@pytest.fixture(scope="module")
def batched_ring():
    """Three uneven instances on the batched ring, their library handles and
    the oracle's result ciphertexts."""
    from paper_2603_04742_gb300.api import Context
    ring = synth.RING["c4"]
    logn, L, K, dnum, t = ring
    insts = _instances(7, [(300, 2500), (800, 6000), (5000, 15000)])
    ctx = Context(logn, L, K, dnum, t)
    ms = [ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals) for A, _ in insts]
    steps = sorted({s for m in ms for s in m.rotation_steps()})
    ctx.keygen(5, steps)
    seeds = [(30 + i, 60 + i) for i in range(len(insts))]
    As = [ctx.encrypt(m, B.HESPMV_MATRIX, seed=sa) for m, (sa, _) in zip(ms, seeds)]
    Xs = [ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=sx) for m, (_, x), (_, sx) in zip(ms, insts, seeds)]
    assert any(c > 1 for m in ms for c in m.chunks()[1]), "no rotating chunk"
    want = _oracle_results(_oracle(ring, steps, 5), insts, seeds)
    return ctx, insts, ms, As, Xs, want


def test_batched_ring_parity(batched_ring):
    ctx, insts, ms, As, Xs, want = batched_ring
    ys = ctx.spmv_batched(ms, As, Xs)
    torch.cuda.synchronize()
    _assert_equal_results(ys, want, "batched")
    for m, y, (A, x) in zip(ms, ys, insts):
        assert list(ctx.decrypt(m, y)) == list(A.matvec(x))
    # the plain per-instance calls too
    _assert_equal_results([ctx.spmv(m, a, x) for m, a, x in zip(ms, As, Xs)], want, "plain")
    # one persistent launch for the whole batch (HE-Mult groups of 16, then of 1)
    try:
        for G in (16, 1):
            ctx.set_tuning(G, 0, 0, 0, 1)
            _assert_equal_results(ctx.spmv_batched(ms, As, Xs), want, ("persistent", G))
    finally:
        ctx.set_tuning(0, 0, 0, 0)
    ctx.device_status()


def test_batched_ring_every_autotuned_schedule_matches_oracle(batched_ring):
    ctx, insts, ms, As, Xs, want = batched_ring
    res = ctx.autotune(ms, As, Xs, reps=1)
    timed = [r for r in res["tried"] if r["ms"] >= 0]
    assert len(timed) >= 3
    try:
        for r in timed:
            ctx.set_tuning(r["mult_batch"], r["rot_batch"], r["ntt_split"], r["rows_tma"], r["persistent"], 0,
                           r["streams"])
            ys = ctx.spmv_batched(ms, As, Xs)
            torch.cuda.synchronize()
            _assert_equal_results(ys, want, r)
    finally:
        ctx.set_tuning(0, 0, 0, 0)
    ctx.device_status()


@pytest.fixture(scope="module")
def serving_ring():
    """The serving ring with the keys the instances below need."""
    from paper_2603_04742_gb300.api import Context
    ring = synth.RING["c5"]
    logn, L, K, dnum, t = ring
    insts = _instances(11, [(5000, 20000), (600, 1500), (1200, 3000)])
    ctx = Context(logn, L, K, dnum, t)
    ms = [ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals) for A, _ in insts]
    steps = sorted({s for m in ms for s in m.rotation_steps()})
    ctx.keygen(9, steps)
    seeds = [(70 + i, 90 + i) for i in range(len(insts))]
    As = [ctx.encrypt(m, B.HESPMV_MATRIX, seed=sa) for m, (sa, _) in zip(ms, seeds)]
    Xs = [ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=sx) for m, (_, x), (_, sx) in zip(ms, insts, seeds)]
    want = _oracle_results(_oracle(ring, steps, 9), insts, seeds)
    return ctx, insts, ms, As, Xs, want


def test_serving_ring_rotations_parity(serving_ring):
    """One SpMV at N = 2^15 whose chunks need three or more column blocks:
    power-of-two rotation chains (least significant bit first) at the
    serving ring, bit-exact with the oracle."""
    ctx, insts, ms, As, Xs, want = serving_ring
    m = ms[0]
    h, c, _ = m.chunks()
    assert int(c.max()) >= 3 and m.n_rot >= 6
    y = ctx.spmv(m, As[0], Xs[0])
    torch.cuda.synchronize()
    _assert_equal_results([y], want[:1], "c>=3 at N=2^15")
    A, x = insts[0]
    assert list(ctx.decrypt(m, y)) == list(A.matvec(x))
    # the persistent launch: the chunks' rotation chains run concurrently
    try:
        ctx.set_tuning(0, 0, 0, 0, 1)
        _assert_equal_results([ctx.spmv(m, As[0], Xs[0])], want[:1], "persistent at N=2^15")
    finally:
        ctx.set_tuning(0, 0, 0, 0)
    ctx.device_status()


def test_serving_ring_served_mix_matches_oracle(serving_ring):
    """Requests for three instances interleaved, submitted while earlier ones
    run (continuous batching over two slots): every result equals the
    oracle's ciphertext for its instance."""
    from paper_2603_04742_gb300.api import CtBatch, Server
    ctx, insts, ms, As, Xs, want = serving_ring
    reqs = [1, 2, 0, 2, 1, 1, 0, 2, 2, 1]
    ys = [CtBatch.create(ctx, ms[i].n_parts) for i in reqs]
    torch.cuda.synchronize()
    srv = Server(ctx, slots=2, mem_budget_bytes=8 << 30, max_batch=3)
    tickets = []
    for k, i in enumerate(reqs):
        tickets.append(srv.submit(ms[i], As[i], Xs[i], ys[k]))
        if k % 3 == 2:
            time.sleep(0.003)
    t0 = time.time()
    while srv.stats()["completed"] < len(reqs):
        assert time.time() - t0 < 120, "serving did not finish"
        time.sleep(0.002)
    done = [srv.poll(tk)[0] for tk in tickets]
    st = srv.stats()
    assert srv.stop(10000) == B.HESPMV_OK
    assert all(d == 1 for d in done) and st["batches"] >= 2
    _assert_equal_results(ys, [want[i] for i in reqs], "served")


def _smallest(ms, k):
    """Indices of the k instances with the fewest key switches."""
    cost = [m.n_chunks + m.n_keyswitch for m in ms]
    return sorted(range(len(ms)), key=lambda i: (cost[i], i))[:k]


def test_c4_full_batch_sampled_oracle_parity():
    """The whole batched workload (64 uneven SpMVs at N = 2^14) in the launch
    configuration the bench times -- HE-Mult groups of 226, rotation rounds
    of 119 chunks, two streams, the alternative NTT split -- with the three
    instances of fewest key switches compared residue for residue with the
    oracle's evaluation of each alone."""
    from paper_2603_04742_gb300.api import Context
    ring = synth.RING["c4"]
    logn, L, K, dnum, t = ring
    insts = synth.workload("c4", count=64)
    ctx = Context(logn, L, K, dnum, t)
    ms = [ctx.encode_cssc(a.rows, a.cols, a.rowptr, a.colidx, a.vals) for a, _ in insts]
    ctx.keygen(1, sorted({s for m in ms for s in m.rotation_steps()}))
    seeds = [(2 + i, 3 + i) for i in range(len(insts))]
    As = [ctx.encrypt(m, B.HESPMV_MATRIX, seed=sa) for m, (sa, _) in zip(ms, seeds)]
    Xs = [ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=sx) for m, (_, x), (_, sx) in zip(ms, insts, seeds)]
    ctx.set_tuning(226, 119, 1, 0, 0, 0, 2)
    ys = ctx.spmv_batched(ms, As, Xs)
    torch.cuda.synchronize()
    pick = _smallest(ms, 3)
    assert all(ms[i].n_rot > 0 for i in pick)   # rotations run in each sampled instance
    steps = sorted({s for i in pick for s in ms[i].rotation_steps()})
    want = _oracle_results(_oracle(ring, steps, 1), [insts[i] for i in pick], [seeds[i] for i in pick])
    _assert_equal_results([ys[i] for i in pick], want, "c4 full batch")
    for m, y, (A, x) in zip(ms, ys, insts):   # and every instance decrypts to A.x
        assert list(ctx.decrypt(m, y)) == list(A.matvec(x))
    ctx.set_tuning(0, 0, 0, 0)


def test_c5_full_pool_served_sampled_oracle_parity():
    """The serving pool (32 distinct instances, n up to 16384, at N = 2^15
    with 8 + 2 primes) served with continuous batching as the bench serves it
    (3 slots, batches of up to 16), two rounds of every instance; the two
    instances of fewest key switches compared residue for residue with the
    oracle, every result decrypted to A.x."""
    from paper_2603_04742_gb300.api import Context, CtBatch, Server
    ring = synth.RING["c5"]
    logn, L, K, dnum, t = ring
    pool = synth.workload("c5", pool=32)
    ctx = Context(logn, L, K, dnum, t)
    ms = [ctx.encode_cssc(a.rows, a.cols, a.rowptr, a.colidx, a.vals) for a, _ in pool]
    ctx.keygen(1, sorted({s for m in ms for s in m.rotation_steps()}))
    seeds = [(2 + i, 500 + i) for i in range(len(pool))]
    As = [ctx.encrypt(m, B.HESPMV_MATRIX, seed=sa) for m, (sa, _) in zip(ms, seeds)]
    Xs = [ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=sx) for m, (_, x), (_, sx) in zip(ms, pool, seeds)]
    reqs = list(range(len(pool))) * 2
    ys = [CtBatch.create(ctx, ms[i].n_parts) for i in reqs]
    torch.cuda.synchronize()
    srv = Server(ctx, slots=3, mem_budget_bytes=3 * (6 << 30), max_batch=16)
    tickets = [srv.submit(ms[i], As[i], Xs[i], y) for i, y in zip(reqs, ys)]
    t0 = time.time()
    while srv.stats()["completed"] < len(reqs):
        assert time.time() - t0 < 300, "serving did not finish"
        time.sleep(0.005)
    assert all(srv.poll(tk)[0] == 1 for tk in tickets)
    assert srv.stop(10000) == B.HESPMV_OK
    pick = _smallest(ms, 2)
    assert all(ms[i].n_rot > 0 for i in pick)
    steps = sorted({s for i in pick for s in ms[i].rotation_steps()})
    want = _oracle_results(_oracle(ring, steps, 1), [pool[i] for i in pick], [seeds[i] for i in pick])
    for j, i in enumerate(pick):
        for k, r in enumerate(reqs):
            if r == i:
                _assert_equal_results([ys[k]], [want[j]], ("c5 served", i, k))
    for k, i in enumerate(reqs):
        A, x = pool[i]
        assert list(ctx.decrypt(ms[i], ys[k])) == list(A.matvec(x)), k
