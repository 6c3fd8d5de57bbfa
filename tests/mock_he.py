"""Plaintext slot simulator of Algorithms 1 and 4 (test helper).

Ciphertexts are replaced by their slot vectors (row 0, N/2 slots): HE-Mult
is the slotwise product, HE-Rot(v, k) is a cyclic left shift np.roll(v, -k),
HE-CMult multiplies by the 0/1 mask.  Used to pin the chunk layout, the
totalSum loop and the masking at full workload sizes without encryption.
"""
import numpy as np

from oracle.cssc import num_bits


def rot(v, k):
    return np.roll(v, -k)


def total_sum_corrected(v, r, c):
    w, e = v.copy(), 1
    for j in range(num_bits(c) - 2, -1, -1):
        w = w + rot(w, e * r)
        e *= 2
        if (c >> j) & 1:
            w = w + rot(v, e * r)
            e += 1
    return w


def total_sum_as_printed(v, r, c):
    """Algorithm 4 exactly as printed (extra step adds Rot(w, 1*r))."""
    w, e = v.copy(), 1
    for j in range(num_bits(c) - 2, -1, -1):
        w = w + rot(w, e * r)
        e *= 2
        if (c >> j) & 1:
            w = w + rot(w, 1 * r)
            e += 1
    return w


def slots(vals, nslots):
    out = np.zeros(nslots, dtype=object)
    out[:len(vals)] = vals
    return out


def spmv_slots(plan, x, nslots, total_sum=total_sum_corrected):
    from oracle.cssc import reorg_vector
    y = np.zeros(plan.rows, dtype=object)
    for part in plan.parts:
        res = np.zeros(nslots, dtype=object)
        reorg = reorg_vector(x, part.chunks)
        for ch, xv in zip(part.chunks, reorg):
            prod = slots(ch.values.astype(object), nslots) * slots(xv.astype(object), nslots)
            w = total_sum(prod, ch.h, ch.c)
            mask = slots([1] * ch.h, nslots)
            res = res + w * mask
        for idx, rm in enumerate(part.cssc.RM):
            y[part.row0 + int(rm)] = res[idx]
    return y
