"""Ciphertext and plan serialization across the parties of Algorithm 1 on
the GPU: Client A keeps the full CSSC, the cloud rebuilds the chunk shapes
from the shape-only stream, evaluates on deserialized ciphertexts, and the
serialized result decrypts at the client to A*x, bit-identical to a local
evaluation.  Malformed streams are refused."""
import struct

import numpy as np
import pytest

from oracle.params import plain_modulus
from paper_2603_04742_gb300 import binding as B
from paper_2603_04742_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_cloud_evaluates_deserialized_inputs():
    from paper_2603_04742_gb300.api import Context
    logn, L, K, dnum, t = synth.RING["c2"]
    A, x = synth.workload("c2")
    client = Context(logn, L, K, dnum, t)
    cloud = Context(logn, L, K, dnum, t)
    m = client.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    client.keygen(5, m.rotation_steps())
    # the cloud receives the evaluation keys only
    cloud.keys_deserialize(client.keys_serialize(B.HESPMV_KEYS_EVAL))
    ca = client.encrypt(m, B.HESPMV_MATRIX, seed=2)
    cx = client.encrypt(m, B.HESPMV_VECTOR, x=x, seed=3)
    mc = cloud.cssc_from_bytes(m.serialize(B.HESPMV_SER_SHAPE))
    ca2 = cloud.ctbatch_from_bytes(ca.serialize())
    cx2 = cloud.ctbatch_from_bytes(cx.serialize())
    assert np.array_equal(ca2.download(), ca.download())
    assert np.array_equal(cx2.download(), cx.download())
    y = cloud.spmv(mc, ca2, cx2)
    torch.cuda.synchronize()
    y_back = client.ctbatch_from_bytes(y.serialize())
    assert list(client.decrypt(m, y_back)) == list(A.matvec(x))
    y_local = client.spmv(m, ca, cx)
    torch.cuda.synchronize()
    assert np.array_equal(y_local.download(), y_back.download())
    # the cloud's plan has no values, indices or row map, and it has no secret key
    with pytest.raises(B.HespmvError) as e:
        cloud.decrypt_slots(y)
    assert e.value.code == B.HESPMV_E_INVALID
    for call in (lambda: cloud.decrypt(mc, y), lambda: cloud.encrypt(mc, B.HESPMV_MATRIX)):
        with pytest.raises(B.HespmvError) as e:
            call()
        assert e.value.code == B.HESPMV_E_INVALID


def test_malformed_ciphertext_streams_refused():
    from paper_2603_04742_gb300.api import Context
    logn, L, K, dnum, t = synth.RING["c1"]
    A, x = synth.workload("c1")
    ctx = Context(logn, L, K, dnum, t)
    ctx.keygen(1)
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    blob = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=9).serialize()
    head = 32
    assert len(blob) == head + m.n_chunks * 2 * L * (1 << logn) * 8
    other = Context(logn, L, K, dnum, plain_modulus(1 << logn, 1 << 17))
    bad_cases = [blob[:-8], blob + b"\0" * 8, blob[:head], b"", b"\0" * 64]
    q0 = ctx.moduli()[0][0]
    bad = bytearray(blob)
    struct.pack_into("<Q", bad, head, q0)          # residue == q_0
    bad_cases.append(bytes(bad))
    bad = bytearray(blob)
    struct.pack_into("<Q", bad, 16, m.n_chunks + 1)  # count vs length
    bad_cases.append(bytes(bad))
    for data in bad_cases:
        with pytest.raises(B.HespmvError) as e:
            ctx.ctbatch_from_bytes(data)
        assert e.value.code == B.HESPMV_E_INVALID
    with pytest.raises(B.HespmvError) as e:
        other.ctbatch_from_bytes(blob)             # another plaintext modulus
    assert e.value.code == B.HESPMV_E_INVALID
    # and the context still works afterwards
    back = ctx.ctbatch_from_bytes(blob)
    assert back.n == m.n_chunks


def test_key_streams_round_trip_and_refusals():
    from paper_2603_04742_gb300.api import Context
    logn, L, K, dnum, t = synth.RING["c1"]
    a = Context(logn, L, K, dnum, t)
    a.keygen(3, [1, 2, 7])
    full = a.keys_serialize(B.HESPMV_KEYS_ALL)
    b = Context(logn, L, K, dnum, t)
    b.keys_deserialize(full)
    for kind in (B.HESPMV_KEY_SECRET, B.HESPMV_KEY_PUBLIC, B.HESPMV_KEY_RELIN):
        assert np.array_equal(a.key_export(kind), b.key_export(kind))
    assert b.keys_serialize(B.HESPMV_KEYS_ALL) == full
    ev = a.keys_serialize(B.HESPMV_KEYS_EVAL)
    assert len(ev) < len(full)
    head = 24
    bad_cases = [ev[:-8], ev + b"\0" * 8, ev[:head], b"\0" * 32]
    bad = bytearray(ev)
    struct.pack_into("<Q", bad, head, a.moduli()[0][0])   # pk residue == q_0
    bad_cases.append(bytes(bad))
    bad = bytearray(ev)
    struct.pack_into("<I", bad, 8, 5)                        # unknown kind
    bad_cases.append(bytes(bad))
    other = Context(logn, L, K, dnum, plain_modulus(1 << logn, 1 << 17))
    for data, ctx in [(d, b) for d in bad_cases] + [(ev, other)]:
        with pytest.raises(B.HespmvError) as e:
            ctx.keys_deserialize(data)
        assert e.value.code == B.HESPMV_E_INVALID
