"""Serving loop: continuous batching returns, for every request, exactly the
ciphertext the request gives alone; admission rejects requests larger than a
slot; stopping with a deadline is bounded and reports the timeout."""
import time

import numpy as np
import pytest

from paper_2603_04742_gb300 import binding as B
from paper_2603_04742_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _pool(ctx, n, seed):
    out = []
    for i in range(n):
        A, x = synth.small_matrix(seed + i, 200 + 150 * i, 180 + 90 * i, 600 + 900 * i)
        m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
        ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=10 + i)
        cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=20 + i)
        out.append((A, x, m, ca, cx))
    return out


def _wait(server, tickets, limit_s=120.0):
    t0 = time.time()
    res = {}
    while len(res) < len(tickets):
        for tk in tickets:
            if tk not in res:
                d, lat = server.poll(tk)
                if d != 0:
                    res[tk] = (d, lat)
        assert time.time() - t0 < limit_s, "serving did not finish"
        time.sleep(0.001)
    return res


def test_serving_results_same_alone_and_in_the_mix():
    from paper_2603_04742_gb300.api import Context, CtBatch, Server
    logn, L, K, dnum, t = synth.RING["c1"]
    ctx = Context(logn, L, K, dnum, t, slots=256)   # several partitions per matrix
    ctx.keygen(7)
    pool = _pool(ctx, 5, 300)
    alone = [ctx.spmv(m, ca, cx).download() for (_, _, m, ca, cx) in pool]
    reqs = [i % len(pool) for i in range(23)]
    ys = [CtBatch.create(ctx, pool[i][2].n_parts) for i in reqs]
    torch.cuda.synchronize()
    srv = Server(ctx, slots=3, mem_budget_bytes=3 << 30, max_batch=4)
    tickets = []
    for k, i in enumerate(reqs):
        _, _, m, ca, cx = pool[i]
        tickets.append(srv.submit(m, ca, cx, ys[k]))
        if k % 5 == 4:
            time.sleep(0.002)   # later requests arrive while earlier ones run
    res = _wait(srv, tickets)
    st = srv.stats()
    assert srv.stop(10000) == B.HESPMV_OK
    assert all(d == 1 and lat > 0 for d, lat in res.values())
    assert st["completed"] == st["submitted"] == len(reqs) and st["batches"] >= 2
    for k, i in enumerate(reqs):
        assert np.array_equal(ys[k].download(), alone[i]), k
    A, x, m, _, _ = pool[reqs[-1]]
    assert list(ctx.decrypt(m, ys[-1])) == list(A.matvec(x))


def test_serving_rejects_requests_larger_than_a_slot():
    from paper_2603_04742_gb300.api import Context, Server
    logn, L, K, dnum, t = synth.RING["c1"]
    ctx = Context(logn, L, K, dnum, t)
    ctx.keygen(3)
    (_, _, m, ca, cx), = _pool(ctx, 1, 5)
    srv = Server(ctx, slots=1, mem_budget_bytes=1 << 20, max_batch=2)
    with pytest.raises(B.HespmvError) as e:
        srv.submit(m, ca, cx)
    assert e.value.code == B.HESPMV_E_REJECTED
    assert srv.stats()["rejected"] == 1
    assert srv.stop(1000) == B.HESPMV_OK


def test_serving_stop_deadline_is_reported():
    from paper_2603_04742_gb300.api import Context, Server
    logn, L, K, dnum, t = synth.RING["c3"]
    ctx = Context(logn, L, K, dnum, t)
    ctx.keygen(3, [])
    A, x, _ = (lambda a: (a[0], a[1], None))(synth.workload("c3"))
    A.vals = synth.quantize(A.vals)
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=1)
    cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=synth.quantize(x), seed=2)
    srv = Server(ctx, slots=1, mem_budget_bytes=4 << 30, max_batch=1)
    for _ in range(8):
        srv.submit(m, ca, cx)
    # eight N = 2^15 SpMVs take milliseconds: a zero deadline must expire
    assert srv.stop(0) == B.HESPMV_E_TIMEOUT
