"""CSSC format, chunking and vector reorganisation (TEST INFRASTRUCTURE ONLY).

* csr_to_cssc: Algorithm 5 (Appendix B), CSR -> (VA, CI, CP, RM).  Rows are
  ordered by descending non-zero count with ties kept in ascending original
  row order (a stable sort; the paper does not say how ties break).  CP has
  L+1 entries, L the longest row, as Algorithm 5 allocates it (the format
  definition in Section 4.3 writes c+1).
* partition_rows: Section 4.7, contiguous blocks of at most s rows.
* generate_chunks: Algorithm 2.  Reading of its capacity test: a chunk of
  consecutive CSSC columns start..i-1 occupies h*(i-start) slots with
  h = NNZ[start] (the padded rectangle of Figure 4), so the chunk grows while
  i < n_C and h*(i-start+1) <= s.  Slot q*h + p holds sorted row p of local
  column q; padding is value 0 and column index -1.
* reorg_vector: Algorithm 3, reorg[k] = v[CI[k]] or 0 where CI[k] = -1.
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np


@dataclass
class CSSC:
    VA: np.ndarray   # values, column-major over the left-aligned sorted rows
    CI: np.ndarray   # original column index of each value
    CP: np.ndarray   # CP[j] = start of aligned column j, length Lmax+1
    RM: np.ndarray   # RM[p] = original (local) row of sorted row p
    rows: int


def csr_to_cssc(rows, rowptr, colidx, vals) -> CSSC:
    rowptr = [int(x) for x in rowptr]
    nnz_row = [rowptr[i + 1] - rowptr[i] for i in range(rows)]
    Lmax = max(nnz_row) if rows else 0
    # stable sort by descending nnz: ties keep ascending row order
    RM = sorted(range(rows), key=lambda i: (-nnz_row[i], i))
    real = np.asarray(vals).dtype.kind == "f"   # real values (CKKS) or integers
    V, C = [], []
    CP = [0] * (Lmax + 1)
    for j in range(Lmax):
        CP[j] = len(V)
        for p in range(rows):
            i = RM[p]
            if j < nnz_row[i]:
                k = rowptr[i] + j
                V.append(float(vals[k]) if real else int(vals[k]))
                C.append(int(colidx[k]))
    CP[Lmax] = len(V)
    return CSSC(np.array(V, dtype=np.float64 if real else np.int64), np.array(C, dtype=np.int64),
                np.array(CP, dtype=np.int64), np.array(RM, dtype=np.int64), rows)


@dataclass
class Chunk:
    values: np.ndarray   # h*c slots
    colidx: np.ndarray   # h*c slots, -1 = padding
    h: int               # rows (rList entry)
    c: int               # columns (cList entry)


def generate_chunks(cssc: CSSC, s: int) -> List[Chunk]:
    CP = cssc.CP
    nC = len(CP) - 1
    NNZ = [int(CP[j + 1] - CP[j]) for j in range(nC)]
    chunks = []
    i = 0
    while i < nC:
        start = i
        h = NNZ[start]
        while i < nC and h * (i - start + 1) <= s:
            i += 1
        c = i - start
        vals = np.zeros(h * c, dtype=cssc.VA.dtype)
        cis = np.full(h * c, -1, dtype=np.int64)
        for qcol in range(c):
            col = start + qcol
            for p in range(NNZ[col]):
                vals[qcol * h + p] = cssc.VA[CP[col] + p]
                cis[qcol * h + p] = cssc.CI[CP[col] + p]
        chunks.append(Chunk(vals, cis, h, c))
    return chunks


def reorg_vector(v, chunks: List[Chunk]) -> List[np.ndarray]:
    out = []
    for ch in chunks:
        one = np.zeros(len(ch.colidx), dtype=np.float64 if np.asarray(v).dtype.kind == "f"
                       else np.int64)
        for k, idx in enumerate(ch.colidx):
            if idx >= 0:
                one[k] = v[idx]
        out.append(one)
    return out


@dataclass
class Partition:
    row0: int                   # first original row of this block
    cssc: CSSC
    chunks: List[Chunk] = field(default_factory=list)


def partition_rows(rows, rowptr, colidx, vals, s) -> List[Partition]:
    """Split the CSR matrix into blocks of <= s consecutive rows (Section 4.7)
    and build each block's CSSC and chunks."""
    parts = []
    for r0 in range(0, rows, s):
        r1 = min(rows, r0 + s)
        base = int(rowptr[r0])
        rp = [int(rowptr[i]) - base for i in range(r0, r1 + 1)]
        ci = colidx[base:int(rowptr[r1])]
        va = vals[base:int(rowptr[r1])]
        cs = csr_to_cssc(r1 - r0, rp, ci, va)
        parts.append(Partition(r0, cs, generate_chunks(cs, s)))
    return parts


def num_bits(c: int) -> int:
    """Bit length of c (Section 4.5: numBits(5) = 3, numBits(21) = 5)."""
    return int(c).bit_length()
