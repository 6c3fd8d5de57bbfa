"""C-ABI library: builds, loads, exports every declared symbol, and its host
logic (parameter tables, CSSC, partitions, chunks, rotation schedule) is
bit-exact with the oracle.  No GPU needed: host-only contexts (device -1)."""
import os
import re

import numpy as np
import pytest

from oracle.cssc import csr_to_cssc, generate_chunks, partition_rows
from oracle.params import min_primitive_root_2n, ntt_primes
from oracle.spmv import rotation_steps
from paper_2603_04742_gb300 import binding as B
from paper_2603_04742_gb300 import synth
from paper_2603_04742_gb300.api import Context

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                   "hespmv.h")


def declared_functions():
    text = open(HDR).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hespmv_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = B.load()
    names = declared_functions()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares exactly the header's functions
    assert sorted(B.SIGNATURES) == names
    assert lib.hespmv_version().decode().startswith("hespmv")


def host_ctx(name="c1", **kw):
    logn, L, K, dnum, t = synth.RING[name]
    return Context(logn, L, K, dnum, t, device=-1, torch_alloc=False, **kw)


@pytest.mark.parametrize("name", ["c1", "c2", "c3", "c4", "c5"])
def test_moduli_and_roots_match_oracle(name):
    ctx = host_ctx(name)
    logn, L, K, dnum, t = synth.RING[name]
    N = 1 << logn
    q, psi, zeta = ctx.moduli()
    assert q == ntt_primes(N, 50, L + K)
    assert psi == [min_primitive_root_2n(x, N) for x in q]
    assert zeta == min_primitive_root_2n(t, N)


def test_bad_parameters_rejected():
    with pytest.raises(B.HespmvError) as e:
        Context(12, 3, 1, 3, 65539, device=-1, torch_alloc=False)   # t not = 1 mod 2N
    assert e.value.code == B.HESPMV_E_UNSUPPORTED
    with pytest.raises(B.HespmvError):
        Context(12, 4, 1, 3, 65537, device=-1, torch_alloc=False)   # dnum leaves a digit empty


def _compare_plan(ctx, A, s):
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    parts = partition_rows(A.rows, A.rowptr, A.colidx, A.vals, s)
    assert m.n_parts == len(parts)
    hs, cs, ps = m.chunks()
    o_chunks = [(ch.h, ch.c, k) for k, p in enumerate(parts) for ch in p.chunks]
    assert list(zip(hs.tolist(), cs.tolist(), ps.tolist())) == o_chunks
    ci = m.colindex()
    assert np.array_equal(ci, np.concatenate([ch.colidx for p in parts for ch in p.chunks])
                          if o_chunks else np.zeros(0))
    for k, p in enumerate(parts):
        va, cci, cp, rm, row0 = m.arrays(k)
        assert row0 == p.row0
        assert np.array_equal(va, p.cssc.VA) and np.array_equal(cci, p.cssc.CI)
        assert np.array_equal(cp, p.cssc.CP) and np.array_equal(rm, p.cssc.RM)
    steps = sorted({k for p in parts for ch in p.chunks for k in rotation_steps(ch.c, ch.h)})
    assert m.rotation_steps() == steps
    assert m.n_rot == sum(len(rotation_steps(ch.c, ch.h)) for p in parts for ch in p.chunks)
    return m


@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
def test_cssc_plan_matches_oracle(name):
    ctx = host_ctx(name)
    A, x = synth.workload(name)
    if name == "c3":
        A.vals = synth.quantize(A.vals)
    _compare_plan(ctx, A, (1 << synth.RING[name][0]) // 2)


def test_cssc_plan_small_slots_and_partitions():
    # slots < N/2 exercise partitions and many chunk shapes
    ctx = Context(12, 3, 1, 3, 65537, slots=100, device=-1, torch_alloc=False)
    for seed in range(4):
        A, _ = synth.small_matrix(seed, 333, 217, 1500)
        _compare_plan(ctx, A, 100)


def test_cssc_plan_batched_instances():
    ctx = host_ctx("c4")
    for A, x in synth.workload("c4", count=6):
        _compare_plan(ctx, A, (1 << 14) // 2)


def test_rotation_keyswitch_count_pow2_vs_exact():
    A, _ = synth.small_matrix(3, 300, 300, 3000)
    c_pow2 = Context(12, 3, 1, 3, 65537, slots=64, device=-1, torch_alloc=False)
    c_exact = Context(12, 3, 1, 3, 65537, slots=64, rot_policy="exact", device=-1, torch_alloc=False)
    m1 = c_pow2.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    m2 = c_exact.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    assert m1.n_rot == m2.n_rot == m2.n_keyswitch
    parts = partition_rows(A.rows, A.rowptr, A.colidx, A.vals, 64)
    want = sum(bin(k).count("1") for p in parts for ch in p.chunks
               for k in rotation_steps(ch.c, ch.h))
    assert m1.n_keyswitch == want


def test_malformed_csr_and_range_errors():
    ctx = host_ctx("c1")
    with pytest.raises(B.HespmvError) as e:      # unsorted columns
        ctx.encode_cssc(2, 4, [0, 2, 3], [2, 1, 0], [1, 1, 1])
    assert e.value.code == B.HESPMV_E_INVALID
    with pytest.raises(B.HespmvError) as e:      # column out of range
        ctx.encode_cssc(1, 4, [0, 1], [4], [1])
    assert e.value.code == B.HESPMV_E_INVALID
    with pytest.raises(B.HespmvError) as e:      # rowptr inconsistent
        ctx.encode_cssc(2, 4, [0, 2, 1], [0, 1], [1, 1])
    assert e.value.code == B.HESPMV_E_INVALID
    # range: row sum 2000 * |x| 20 >= t/2 = 32768
    with pytest.raises(B.HespmvError) as e:
        ctx.encode_cssc(1, 2, [0, 2], [0, 1], [1000, -1000], max_abs_x=20)
    assert e.value.code == B.HESPMV_E_RANGE
    ctx.encode_cssc(1, 2, [0, 2], [0, 1], [1000, -1000], max_abs_x=16)   # 32000 < 32768.5


def test_empty_matrix_and_empty_rows():
    ctx = host_ctx("c1")
    m = ctx.encode_cssc(5, 3, [0, 0, 0, 0, 0, 0], [], [])
    assert m.n_parts == 1 and m.n_chunks == 0
    m = ctx.encode_cssc(0, 3, [0], [], [])
    assert m.n_parts == 0 and m.n_chunks == 0


def test_host_only_context_refuses_device_calls():
    ctx = host_ctx("c1")
    with pytest.raises(B.HespmvError) as e:
        ctx.keygen(1)
    assert e.value.code == B.HESPMV_E_INVALID


def test_server_needs_a_device_context():
    from paper_2603_04742_gb300.api import Server
    ctx = host_ctx("c1")
    with pytest.raises(B.HespmvError) as e:
        Server(ctx, slots=1, mem_budget_bytes=1 << 20, max_batch=1)
    assert e.value.code == B.HESPMV_E_INVALID


def test_tuning_round_trip_and_validation():
    ctx = host_ctx("c3")
    zero = {"mult_batch": 0, "rot_batch": 0, "ntt_split": 0, "rows_tma": 0, "persistent": 0,
            "persist_blocks": 0, "streams": 1}
    assert ctx.get_tuning() == zero
    ctx.set_tuning(8, 16, 1, 1)
    want = dict(zero, mult_batch=8, rot_batch=16, ntt_split=1, rows_tma=1)
    assert ctx.get_tuning() == want
    for bad in [(-1, 0, 0), (0, -2, 0), (0, 0, 2), (5000, 0, 0), (0, 0, 0, 2), (0, 0, 0, 0, 2),
                (0, 0, 0, 0, 1, -1), (0, 0, 0, 0, 0, 0, 3)]:
        with pytest.raises(B.HespmvError) as e:
            ctx.set_tuning(*bad)
        assert e.value.code == B.HESPMV_E_INVALID
    assert ctx.get_tuning() == want
    ctx.set_tuning(16, 0, 0, 0, 1, 7)   # the persistent form (alpha = 2, K = 2: supported)
    assert ctx.get_tuning() == dict(zero, mult_batch=16, persistent=1, persist_blocks=7)
    ctx.set_tuning(14, 0, 0, 0, 0, 0, 2)   # HE-Mult groups over two streams
    assert ctx.get_tuning() == dict(zero, mult_batch=14, streams=2)
    small = Context(10, 3, 1, 3, 40961, device=-1, torch_alloc=False)   # unfused key switch
    with pytest.raises(B.HespmvError):
        small.set_tuning(0, 0, 1)
    with pytest.raises(B.HespmvError):
        small.set_tuning(0, 0, 0, 1)
    with pytest.raises(B.HespmvError):
        small.set_tuning(0, 0, 0, 0, 1)   # no persistent form below N = 2^11


def test_autotune_needs_a_device():
    ctx = host_ctx("c1")
    with pytest.raises(B.HespmvError) as e:
        ctx.autotune([], [], [])
    assert e.value.code == B.HESPMV_E_INVALID


def test_bfv_context_tables():
    from oracle.params import ntt_primes
    logn, L, K, dnum, t = synth.RING["c3"]
    ctx = Context(logn, L, K, dnum, t, device=-1, torch_alloc=False, scheme="bfv")
    q, psi, zeta = ctx.moduli()
    assert q == ntt_primes(1 << logn, 50, L + K)
    with pytest.raises(B.HespmvError):        # K < alpha
        Context(6, 4, 1, 2, 12289, device=-1, torch_alloc=False, scheme="bfv")
