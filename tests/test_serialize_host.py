"""CSSC plan serialization (hespmv_cssc_serialize / _deserialize) on the host:
round trips are exact, the shape-only form carries exactly the chunk shapes
the cloud evaluates, and every malformed stream is refused with E_INVALID
rather than read out of bounds."""
import struct

import numpy as np
import pytest

from paper_2603_04742_gb300 import binding as B
from paper_2603_04742_gb300 import synth
from paper_2603_04742_gb300.api import Context


def host_ctx(name="c1", **kw):
    logn, L, K, dnum, t = synth.RING[name]
    return Context(logn, L, K, dnum, t, device=-1, torch_alloc=False, **kw)


def plans():
    out = []
    for name in ("c1", "c2"):
        A, _ = synth.workload(name)
        out.append((host_ctx(name), A))
    ctx = Context(12, 3, 1, 3, 65537, slots=100, device=-1, torch_alloc=False)
    A, _ = synth.small_matrix(3, 333, 217, 1500)
    out.append((ctx, A))
    return out


def same_plan(a, b, values=True):
    assert (a.n_parts, a.n_chunks, a.n_rot, a.n_keyswitch, a.rows, a.cols, a.nnz) == \
        (b.n_parts, b.n_chunks, b.n_rot, b.n_keyswitch, b.rows, b.cols, b.nnz)
    for x, y in zip(a.chunks(), b.chunks()):
        assert np.array_equal(x, y)
    assert a.rotation_steps() == b.rotation_steps()
    if values:
        assert np.array_equal(a.colindex(), b.colindex())
        for p in range(a.n_parts):
            for x, y in zip(a.arrays(p), b.arrays(p)):
                assert np.array_equal(x, y)


@pytest.mark.parametrize("i", range(3))
def test_full_round_trip(i):
    ctx, A = plans()[i]
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    data = m.serialize(B.HESPMV_SER_FULL)
    m2 = ctx.cssc_from_bytes(data)
    same_plan(m, m2)
    assert m2.serialize(B.HESPMV_SER_FULL) == data


@pytest.mark.parametrize("i", range(3))
def test_shape_only_round_trip(i):
    ctx, A = plans()[i]
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    shape = m.serialize(B.HESPMV_SER_SHAPE)
    assert len(shape) < len(m.serialize(B.HESPMV_SER_FULL)) or A.nnz == 0
    ms = ctx.cssc_from_bytes(shape)
    same_plan(m, ms, values=False)
    assert ms.serialize(B.HESPMV_SER_SHAPE) == shape
    for call in (lambda: ms.colindex(), lambda: ms.arrays(0),
                 lambda: ms.serialize(B.HESPMV_SER_FULL)):
        with pytest.raises(B.HespmvError) as e:
            call()
        assert e.value.code == B.HESPMV_E_INVALID


def test_empty_matrix_round_trip():
    ctx = host_ctx("c1")
    m = ctx.encode_cssc(0, 0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int64))
    same_plan(m, ctx.cssc_from_bytes(m.serialize()))
    rows = 5
    m = ctx.encode_cssc(rows, 3, np.zeros(rows + 1, np.int64), np.zeros(0, np.int32),
                        np.zeros(0, np.int64))
    same_plan(m, ctx.cssc_from_bytes(m.serialize()))


def _refused(ctx, data):
    with pytest.raises(B.HespmvError) as e:
        ctx.cssc_from_bytes(data)
    assert e.value.code == B.HESPMV_E_INVALID


def _small():
    ctx = Context(10, 3, 1, 3, 40961, slots=8, device=-1, torch_alloc=False)
    A, _ = synth.small_matrix(1, 20, 12, 60, -5, 5)
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    return ctx, A, m, m.serialize()


def test_truncated_and_extended_streams_refused():
    ctx, A, m, data = _small()
    for cut in range(0, len(data), 4):
        _refused(ctx, data[:cut])
    _refused(ctx, data + b"\0" * 8)


def test_header_fields_checked():
    ctx, A, m, data = _small()
    bad = bytearray(data)
    bad[0] ^= 1                                    # magic
    _refused(ctx, bytes(bad))
    bad = bytearray(data)
    struct.pack_into("<I", bad, 4, 2)              # version
    _refused(ctx, bytes(bad))
    bad = bytearray(data)
    struct.pack_into("<I", bad, 8, 7)              # kind
    _refused(ctx, bytes(bad))
    other = Context(10, 3, 1, 3, 40961, slots=16, device=-1, torch_alloc=False)
    _refused(other, data)                          # chunk capacity differs
    bad = bytearray(data)
    struct.pack_into("<i", bad, 16, A.rows + 9)    # rows vs partitions
    _refused(ctx, bytes(bad))


def _first_part_offsets(data):
    # header 40 bytes; partition: row0, rows (i32), nnz_part, |CP| (i64), CP[]
    nnz_part, cp_len = struct.unpack_from("<qq", data, 48)
    cp_off = 64
    va_off = cp_off + 8 * cp_len
    ci_off = va_off + 8 * nnz_part
    rm_off = ci_off + ((4 * nnz_part + 7) // 8) * 8
    return nnz_part, cp_len, cp_off, va_off, ci_off, rm_off


def test_structural_corruptions_refused():
    ctx, A, m, data = _small()
    nnz_part, cp_len, cp_off, va_off, ci_off, rm_off = _first_part_offsets(data)
    cp = list(struct.unpack_from("<%dq" % cp_len, data, cp_off))
    assert cp_len >= 3
    # column heights must not increase
    bad = bytearray(data)
    struct.pack_into("<q", bad, cp_off + 8, cp[1] - 1)
    _refused(ctx, bytes(bad))
    # a height above the partition's rows (it would never fit a chunk)
    bad = bytearray(data)
    struct.pack_into("<q", bad, cp_off + 8, cp[1] + 100)
    _refused(ctx, bytes(bad))
    # CI out of range, and a row whose columns stop ascending
    bad = bytearray(data)
    struct.pack_into("<i", bad, ci_off, A.cols)
    _refused(ctx, bytes(bad))
    bad = bytearray(data)
    c0 = struct.unpack_from("<i", data, ci_off)[0]
    struct.pack_into("<i", bad, ci_off + 4 * cp[1], c0)   # row 0, column 1 := column 0's index
    _refused(ctx, bytes(bad))
    # RM not a permutation
    bad = bytearray(data)
    r0 = struct.unpack_from("<i", data, rm_off)[0]
    struct.pack_into("<i", bad, rm_off + 4, r0)
    _refused(ctx, bytes(bad))


def test_random_byte_flips_never_crash():
    ctx, A, m, data = _small()
    g = np.random.default_rng(7)
    accepted = 0
    for _ in range(300):
        bad = bytearray(data)
        for _ in range(int(g.integers(1, 4))):
            bad[int(g.integers(0, len(bad)))] ^= int(g.integers(1, 256))
        try:
            ctx.cssc_from_bytes(bytes(bad))
            accepted += 1          # e.g. a changed value: still a valid plan
        except B.HespmvError as e:
            assert e.code == B.HESPMV_E_INVALID
    assert accepted < 300
