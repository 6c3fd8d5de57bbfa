"""Pins of the oracle's format layer (Algorithms 5, 2, 3, Section 4.7) and of
the aggregation logic of Algorithm 4, using dense round trips, the paper's
worked-example fragments and a plaintext slot simulation."""
import json
import os

import numpy as np
import pytest

from oracle.cssc import (csr_to_cssc, generate_chunks, num_bits, partition_rows,
                         reorg_vector)
from oracle.spmv import SpmvPlan, rotation_steps
from paper_2603_04742_gb300 import synth
from tests import mock_he

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_cssc_dense_roundtrip():
    A, _ = synth.small_matrix(1, 37, 23, 160)
    cs = csr_to_cssc(A.rows, A.rowptr, A.colidx, A.vals)
    nnz_row = np.diff(A.rowptr)
    # RM orders rows by descending nnz, ties in ascending row order
    assert sorted(cs.RM.tolist()) == list(range(A.rows))
    keys = [(-nnz_row[i], i) for i in cs.RM]
    assert keys == sorted(keys)
    # CP: prefix sums of non-increasing column heights, length Lmax + 1
    heights = np.diff(cs.CP)
    assert len(cs.CP) == nnz_row.max() + 1 and cs.CP[0] == 0 and cs.CP[-1] == A.nnz
    assert np.all(heights[:-1] >= heights[1:])
    # rebuild the dense matrix from (VA, CI, RM, CP)
    D = np.zeros((A.rows, A.cols), dtype=np.int64)
    for j in range(len(cs.CP) - 1):
        for p in range(heights[j]):
            k = cs.CP[j] + p
            D[cs.RM[p], cs.CI[k]] = cs.VA[k]
    assert np.array_equal(D, A.dense())
    # each sorted row keeps its original column order (left alignment)
    for p in range(A.rows):
        cols = [cs.CI[cs.CP[j] + p] for j in range(len(cs.CP) - 1) if p < heights[j]]
        assert cols == sorted(cols)


def test_cssc_empty_rows_and_matrix():
    cs = csr_to_cssc(3, [0, 0, 0, 0], [], [])
    assert len(cs.VA) == 0 and cs.CP.tolist() == [0]
    assert generate_chunks(cs, 8) == []
    cs = csr_to_cssc(4, [0, 0, 2, 2, 3], [1, 3, 0], [5, 6, 7])
    assert cs.RM.tolist() == [1, 3, 0, 2] and cs.CP.tolist() == [0, 2, 3]


def test_figure5_reorganisation():
    g = json.load(open(os.path.join(GOLD, "fig5_reorg.json")))

    class Ch:  # one chunk whose slot k carries column index 1
        colidx = np.array([0, 2, -1, g["column_index_at_k"], 0])
    v = np.array([1, g["vector_at_column"], 3])
    out = reorg_vector(v, [Ch])[0]
    assert out[g["k"]] == g["expected_reorganized_at_k"]
    assert out[2] == 0   # padding (-1) maps to 0


def test_numbits_examples():
    g = json.load(open(os.path.join(GOLD, "numbits.json")))
    for c, n in g["cases"]:
        assert num_bits(c) == n


def test_figure4_chunk_example():
    g = json.load(open(os.path.join(GOLD, "fig4_chunks.json")))
    rows = len(g["row_nnz"])
    rowptr = np.concatenate([[0], np.cumsum(g["row_nnz"])])
    colidx = np.concatenate([np.arange(n) for n in g["row_nnz"]])
    cs = csr_to_cssc(rows, rowptr, colidx, np.ones(len(colidx), dtype=np.int64))
    chunks = generate_chunks(cs, g["s"])
    assert [c.h for c in chunks] == g["rList"]
    assert all(c.h * c.c <= g["s"] for c in chunks)
    assert [len(rotation_steps(c.c, c.h)) for c in chunks] == g["rotations_per_chunk"]


def test_chunk_invariants_and_capacity():
    A, _ = synth.small_matrix(7, 300, 200, 2000)
    for s in (16, 64, 150, 300):
        for part in partition_rows(A.rows, A.rowptr, A.colidx, A.vals, s):
            cs = part.cssc
            heights = np.diff(cs.CP)
            col = 0
            for ch in part.chunks:
                assert ch.h == heights[col] and ch.h * ch.c <= s
                # the next column would not have fitted
                if col + ch.c < len(heights):
                    assert ch.h * (ch.c + 1) > s
                for qc in range(ch.c):
                    n = heights[col + qc]
                    seg = slice(qc * ch.h, qc * ch.h + n)
                    assert np.array_equal(ch.values[seg], cs.VA[cs.CP[col + qc]:cs.CP[col + qc] + n])
                    assert np.all(ch.colidx[qc * ch.h + n:(qc + 1) * ch.h] == -1)
                col += ch.c
            assert col == len(heights)


def test_partition_rows_blocks():
    A, _ = synth.small_matrix(8, 50, 40, 300)
    parts = partition_rows(A.rows, A.rowptr, A.colidx, A.vals, 16)
    assert [p.row0 for p in parts] == [0, 16, 32, 48]
    assert sum(len(p.cssc.VA) for p in parts) == A.nnz


@pytest.mark.parametrize("c", [3, 5, 6, 7])
def test_printed_totalsum_double_counts(c):
    """The extra step as printed (Rot(w, r)) gives wrong row sums; the
    Halevi-Shoup form (Rot(ctV, e*r)) is right, for every c."""
    r = 4
    v = np.arange(1, r * c + 1, dtype=object)
    want = [sum(v[q * r + p] for q in range(c)) for p in range(r)]
    nsl = 64
    assert list(mock_he.total_sum_corrected(mock_he.slots(v, nsl), r, c)[:r]) == want
    assert list(mock_he.total_sum_as_printed(mock_he.slots(v, nsl), r, c)[:r]) != want


@pytest.mark.parametrize("c", range(1, 20))
def test_totalsum_rotation_count(c):
    steps = rotation_steps(c, 3)
    assert len(steps) == (num_bits(c) - 1) + (bin(c).count("1") - 1)
    v = np.arange(1, 3 * c + 1, dtype=object)
    w = mock_he.total_sum_corrected(mock_he.slots(v, 128), 3, c)
    assert [w[p] for p in range(3)] == [sum(v[q * 3 + p] for q in range(c)) for p in range(3)]


@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
def test_slot_simulation_equals_spmv(name):
    A, x = synth.workload(name)
    if name == "c3":
        A.vals = synth.quantize(A.vals)
        x = synth.quantize(x)
    logn = synth.RING[name][0]
    s = (1 << logn) // 2
    plan = SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, s)
    y = mock_he.spmv_slots(plan, x, s)
    assert list(y) == list(A.matvec(x))
    if name == "c3":
        assert [(c.h, c.c) for c in plan.chunks] == \
            [(16384, 1)] * 8 + [(16376, 1)] * 4 + [(16080, 1)] * 6 + [(12600, 1)] * 9
        assert A.nnz == 406456


def test_slot_simulation_partitions_and_batched_instances():
    for k, (A, x) in enumerate(synth.workload("c4", count=3)):
        plan = SpmvPlan(A.rows, A.cols, A.rowptr, A.colidx, A.vals, 1024)
        assert list(mock_he.spmv_slots(plan, x, 1024)) == list(A.matvec(x))
