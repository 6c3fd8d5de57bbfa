"""Encrypted SpMV of the oracle: Algorithms 1 and 4 (TEST INFRASTRUCTURE ONLY).

Algorithm 1 (cloud lines): one HE-Mult per chunk pair.  Algorithm 4: per
chunk (r, c) the totalSum rotate-and-add, then res = sum_i intraRes_i x
mask_{r_i}.  Reading of the totalSum loop (the printed extra step adds
Rot(w, r), which double-counts whenever c is not a power of two): following
the Halevi-Shoup totalSums the paper cites,

    w = ctV; e = 1
    for j = numBits(c)-2 down to 0:
        w = w + Rot(w, e*r); e = 2e
        if bit_j(c): w = w + Rot(ctV, e*r); e = e + 1

which keeps w = sum of the first e column blocks.  The mask is always
applied, also when it is all ones.  Row 1 of the batching slots is unused.
"""
import numpy as np

from .bgv import Oracle
from .cssc import Chunk, num_bits, partition_rows, reorg_vector


def total_sum(orc: Oracle, ctV, r: int, c: int, policy="pow2"):
    w = ctV
    e = 1
    for j in range(num_bits(c) - 2, -1, -1):
        w = orc.add(w, orc.rotate(w, e * r, policy))
        e = 2 * e
        if (c >> j) & 1:
            w = orc.add(w, orc.rotate(ctV, e * r, policy))
            e = e + 1
    return w


def rotation_steps(c: int, r: int):
    """Rotation amounts used by total_sum for a chunk (r, c), in order."""
    steps = []
    e = 1
    for j in range(num_bits(c) - 2, -1, -1):
        steps.append(e * r)
        e *= 2
        if (c >> j) & 1:
            steps.append(e * r)
            e += 1
    return steps


def mask_ntt(orc: Oracle, r: int):
    return orc.plaintext_ntt([1] * r + [0] * (orc.p.N // 2 - r))


def aggregation(orc: Oracle, ct_list, r_list, c_list, policy="pow2"):
    """Algorithm 4 -> the encrypted result of one partition."""
    intra = [total_sum(orc, ct, r, c, policy) for ct, r, c in zip(ct_list, r_list, c_list)]
    res = np.zeros_like(ct_list[0])
    for i, w in enumerate(intra):
        res = orc.add(res, orc.cmult(w, mask_ntt(orc, r_list[i])))
    return res


def cloud(orc: Oracle, chunks, ct_values, ct_vectors, policy="pow2"):
    """Cloud lines of Algorithm 1 for one partition."""
    prods = [orc.mult(a, x) for a, x in zip(ct_values, ct_vectors)]
    return aggregation(orc, prods, [ch.h for ch in chunks], [ch.c for ch in chunks], policy)


def cloud_plain_matrix(orc: Oracle, chunks, pt_values, ct_vectors, policy="pow2"):
    """Algorithm 1 cloud lines when the evaluator holds the matrix in the
    clear (the Rhombus trust model of Section 5): HE-CMult per chunk, then
    Algorithm 4 unchanged."""
    prods = [orc.cmult(x, pt) for pt, x in zip(pt_values, ct_vectors)]
    return aggregation(orc, prods, [ch.h for ch in chunks], [ch.c for ch in chunks], policy)


class SpmvPlan:
    """Client-side preparation: partitions, CSSC, chunks (Algorithms 5, 2)."""

    def __init__(self, rows, cols, rowptr, colidx, vals, s):
        self.rows, self.cols, self.s = rows, cols, s
        self.parts = partition_rows(rows, rowptr, colidx, vals, s)

    @property
    def chunks(self):
        return [ch for p in self.parts for ch in p.chunks]


def encrypt_matrix(orc: Oracle, plan: SpmvPlan, seed: int):
    out = []
    for k, ch in enumerate(plan.chunks):
        out.append(orc.encrypt(orc.encode(ch.values), seed, k))
    return out


def encrypt_vector(orc: Oracle, plan: SpmvPlan, x, seed: int):
    out = []
    reorg = reorg_vector(x, plan.chunks)
    for k, v in enumerate(reorg):
        out.append(orc.encrypt(orc.encode(v), seed, k))
    return out


def encode_matrix_plain(orc: Oracle, plan: SpmvPlan):
    """Chunk values as plaintexts in the NTT domain over Q (no encryption)."""
    return [orc.plaintext_ntt(ch.values) for ch in plan.chunks]


def spmv_plain_matrix(orc: Oracle, plan: SpmvPlan, pt_values, ct_vectors, policy="pow2"):
    res = []
    k = 0
    for part in plan.parts:
        n = len(part.chunks)
        if n == 0:
            res.append(np.zeros((2, orc.p.L, orc.p.N), dtype=np.uint64))
        else:
            res.append(cloud_plain_matrix(orc, part.chunks, pt_values[k:k + n],
                                          ct_vectors[k:k + n], policy))
        k += n
    return res


def spmv(orc: Oracle, plan: SpmvPlan, ct_values, ct_vectors, policy="pow2"):
    """All partitions: one result ciphertext per partition."""
    res = []
    k = 0
    for part in plan.parts:
        n = len(part.chunks)
        if n == 0:
            res.append(np.zeros((2, orc.p.L, orc.p.N), dtype=np.uint64))
        else:
            res.append(cloud(orc, part.chunks, ct_values[k:k + n], ct_vectors[k:k + n], policy))
        k += n
    return res


def decrypt_result(orc: Oracle, plan: SpmvPlan, results):
    """Decrypt and undo the row permutation (Algorithm 1, last lines)."""
    t = orc.p.t
    out = np.zeros(plan.rows, dtype=object)
    for part, ct in zip(plan.parts, results):
        slots, _ = orc.decode(orc.decrypt(ct))
        for idx, rm in enumerate(part.cssc.RM):
            v = int(slots[idx])
            out[part.row0 + int(rm)] = v - t if 2 * v > t else v
    return out


def decrypt_result_real(orc, plan: SpmvPlan, results):
    """CKKS: decrypt, decode at the product scale (matrix x vector x mask)
    and undo the row permutation."""
    p = orc.p
    total_bits = 2 * p.scale_bits + p.mask_scale_bits
    out = np.zeros(plan.rows, dtype=np.float64)
    for part, ct in zip(plan.parts, results):
        z = orc.decode_ct(ct, len(part.cssc.RM), total_bits)
        for idx, rm in enumerate(part.cssc.RM):
            out[part.row0 + int(rm)] = z[idx]
    return out
