"""Key-switch decomposition and rotation-key policy as tuned choices.

The exact-step rotation-key policy (one Galois key per distinct rotation,
instead of power-of-two chains) on the batched ring is checked against the
oracle residue for residue in a batched evaluation; the tuner over dnum and
the policy returns only correct candidates, counts keys and key bytes, and
the exact-step policy needs no more key switches than power-of-two chains."""
import numpy as np
import pytest

from oracle import spmv as S
from oracle.bgv import Oracle
from oracle.params import Params, plain_modulus
from paper_2603_04742_gb300 import binding as B
from paper_2603_04742_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _instances(seed, shapes):
    g = np.random.default_rng(seed)
    out = []
    for n, nnz in shapes:
        A = synth.uniform_positions(g, n, n, nnz, -15, 15)
        out.append((A, g.integers(-15, 16, size=n, dtype=np.int64)))
    return out


def test_exact_policy_batched_ring_matches_oracle():
    from paper_2603_04742_gb300.api import Context
    logn, L, K, dnum, t = synth.RING["c4"]
    insts = _instances(7, [(300, 2500), (800, 6000), (5000, 15000)])
    ctx = Context(logn, L, K, dnum, t, rot_policy="exact")
    ms = [ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals) for A, _ in insts]
    steps = sorted({s for m in ms for s in m.rotation_steps()})
    ctx.keygen(5, steps)
    As = [ctx.encrypt(m, B.HESPMV_MATRIX, seed=30 + i) for i, m in enumerate(ms)]
    Xs = [ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=60 + i) for i, (m, (_, x)) in enumerate(zip(ms, insts))]
    assert all(m.n_keyswitch == m.n_rot for m in ms)   # one key switch per rotation
    ys = ctx.spmv_batched(ms, As, Xs)
    torch.cuda.synchronize()
    orc = Oracle(Params(log2n=logn, L=L, K=K, dnum=dnum, t=t))
    orc.keygen(5, sorted({g for k in steps for g in orc.rotation_elements(k, "exact")}))
    for i, ((A, x), y) in enumerate(zip(insts, ys)):
        plan = S.SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, orc.p.slots)
        want = np.stack(S.spmv(orc, plan, S.encrypt_matrix(orc, plan, 30 + i),
                               S.encrypt_vector(orc, plan, x, 60 + i), "exact"))
        assert np.array_equal(y.download(), want), i
        assert list(ctx.decrypt(ms[i], y)) == list(A.matvec(x))


def test_tune_keyswitch_candidates_are_correct_and_counted():
    from paper_2603_04742_gb300.api import tune_keyswitch
    logn, L, K = 12, 4, 2
    t = plain_modulus(1 << logn, 1 << 20)
    insts = _instances(3, [(400, 3000), (900, 2500)])
    res = tune_keyswitch((logn, L, K, 2, t), insts, reps=2, schedule=False)
    assert {(r["dnum"], r["policy"]) for r in res} == {(2, "pow2"), (2, "exact"), (4, "pow2"), (4, "exact")}
    assert all(r["correct"] for r in res)
    assert [r["ms"] for r in res] == sorted(r["ms"] for r in res)
    by = {(r["dnum"], r["policy"]): r for r in res}
    for d in (2, 4):
        assert by[(d, "exact")]["keyswitches"] <= by[(d, "pow2")]["keyswitches"]
        for pol in ("pow2", "exact"):
            r = by[(d, pol)]
            assert r["key_bytes"] == (1 + r["galois_keys"]) * d * 2 * (L + K) * (1 << logn) * 8
    # dnum with alpha > K (noise) is not offered
    assert tune_keyswitch((logn, L, K, 2, t), insts, dnums=[1], reps=1, schedule=False) == []
