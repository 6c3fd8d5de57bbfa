"""The schedule autotuner on a batch of uneven SpMVs: every schedule it times
gives bit-identical results, the one it applies is the fastest it measured,
and a JSON cache replays the choice without timing."""
import os

import numpy as np
import pytest

from paper_2603_04742_gb300 import binding as B
from paper_2603_04742_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _batch(ctx, n, seed):
    g = np.random.default_rng(seed)
    insts = []
    for _ in range(n):
        rows = int(g.integers(100, 1500))
        nnz = int(g.integers(rows, rows * 12))
        A = synth.uniform_positions(g, rows, rows, nnz, -15, 15)
        x = g.integers(-15, 16, size=rows, dtype=np.int64)
        insts.append((A, x))
    ms = [ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals) for A, _ in insts]
    steps = sorted({s for m in ms for s in m.rotation_steps()})
    return insts, ms, steps


@pytest.mark.parametrize("logn", [12, 13])
def test_autotune_results_identical_and_cached(logn, tmp_path):
    from paper_2603_04742_gb300.api import Context
    t = {12: 65537, 13: 114689}[logn]
    ctx = Context(logn, 4, 2, 2, t)
    insts, ms, steps = _batch(ctx, 6, 40 + logn)
    ctx.keygen(3, steps)
    As = [ctx.encrypt(m, B.HESPMV_MATRIX, seed=10 + i) for i, m in enumerate(ms)]
    Xs = [ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=50 + i) for i, (m, (_, x)) in enumerate(zip(ms, insts))]
    ref = ctx.spmv_batched(ms, As, Xs)
    torch.cuda.synchronize()
    ref_bytes = [y.download() for y in ref]
    for m, y, (A, x) in zip(ms, ref, insts):
        assert list(ctx.decrypt(m, y)) == list(A.matvec(x))
    cache = str(tmp_path / "tune.json")
    res = ctx.autotune(ms, As, Xs, reps=2, cache=cache)
    assert not res["cached"]
    timed = [r for r in res["tried"] if r["ms"] >= 0]
    assert len(timed) >= 3
    assert res["best"]["ms"] == min(r["ms"] for r in timed)
    assert {r["ntt_split"] for r in timed} == {0, 1}
    assert {r["rows_tma"] for r in timed} == {0, 1}
    assert {r["persistent"] for r in timed} == {0, 1}
    assert {r["streams"] for r in timed} == {1, 2}
    # every schedule timed gives the same ciphertexts
    for r in timed:
        ctx.set_tuning(r["mult_batch"], r["rot_batch"], r["ntt_split"], r["rows_tma"], r["persistent"], 0,
                       r["streams"])
        ys = ctx.spmv_batched(ms, As, Xs)
        torch.cuda.synchronize()
        for y, z in zip(ys, ref_bytes):
            assert np.array_equal(y.download(), z), r
    # the cache replays the choice
    ctx.set_tuning(0, 0, 0)
    res2 = ctx.autotune(ms, As, Xs, reps=2, cache=cache)
    assert res2["cached"] and res2["best"] == res["best"]
    b = res["best"]
    assert ctx.get_tuning() == {"mult_batch": b["mult_batch"], "rot_batch": b["rot_batch"],
                                "ntt_split": b["ntt_split"], "rows_tma": b["rows_tma"],
                                "persistent": b["persistent"], "persist_blocks": b["persist_blocks"],
                                "streams": b["streams"]}
    ctx.device_status()
    assert os.path.exists(cache)
