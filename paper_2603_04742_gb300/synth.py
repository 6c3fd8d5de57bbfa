"""Seeded synthetic workloads (inputs only, no scheme arithmetic).

The paper measures on SuiteSparse matrices (Section 5), which are not
available here; these generators stand in for them with the shapes, value
ranges and sparsity structures of the five benchmark configurations.  Every
generator is seeded (numpy PCG64) and returns CSR arrays with strictly
ascending column indices inside each row.

Configurations (ring parameters beside each):
  c1  512 x 512, 2,621 nnz at uniform positions, a, x integers in [-15, 15];
      N = 2^12, 3 ciphertext primes + 1 special prime, dnum 3, t = 65537
  c2  4096 x 4096, 16,777 nnz, power-law (exponent 1.5) column counts,
      integers in [-127, 127]; N = 2^14, 5 + 1 primes, dnum 5, t = 17006593
  c3  27-point stencil on a 16 x 32 x 32 grid (16,384 rows, 406,456 nnz),
      a, x uniform in [-1, 1] (fixed point, scale 2^15 each);
      N = 2^15, 8 + 2 primes, dnum 4, t = 1099512938497
  c4  64 square matrices, n log-uniform in [256, 8192], density log-uniform
      in [5e-4, 2e-2], integers in [-15, 15]; N = 2^14, 5 + 1 primes, dnum 5,
      t = 1146881
  c5  request pool: n log-uniform in [512, 16384], density log-uniform in
      [5e-4, 1e-2], integers in [-15, 15]; N = 2^15, 8 + 2 primes, dnum 4,
      t = 1179649
The plaintext moduli are the smallest primes t = 1 mod 2N at or above 2^16
(c1 uses the paper's 65537), 2^24, 2^40, 2^20 and 2^20.
"""
from dataclasses import dataclass

import numpy as np

RING = {
    # name: (log2n, L, K, dnum, t)
    "c1": (12, 3, 1, 3, 65537),
    "c2": (14, 5, 1, 5, 17006593),
    "c3": (15, 8, 2, 4, 1099512938497),
    "c4": (14, 5, 1, 5, 1146881),
    "c5": (15, 8, 2, 4, 1179649),
}

SEEDS = {"c1": 101, "c2": 102, "c3": 103, "c4": 104, "c5": 105}

FIXED_POINT_BITS = 15


@dataclass
class CSR:
    rows: int
    cols: int
    rowptr: np.ndarray   # int64, rows+1
    colidx: np.ndarray   # int32
    vals: np.ndarray     # int64 (or float64 before quantisation)

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def dense(self):
        d = np.zeros((self.rows, self.cols), dtype=self.vals.dtype)
        for i in range(self.rows):
            s, e = self.rowptr[i], self.rowptr[i + 1]
            d[i, self.colidx[s:e]] = self.vals[s:e]
        return d

    def matvec(self, x):
        """Exact integer (object) or float64 A.x, for checking results."""
        if self.vals.dtype.kind == "f":
            y = np.zeros(self.rows)
            for i in range(self.rows):
                s, e = self.rowptr[i], self.rowptr[i + 1]
                y[i] = np.dot(self.vals[s:e], np.asarray(x, dtype=np.float64)[self.colidx[s:e]])
            return y
        xo = np.asarray(x, dtype=object)
        y = np.zeros(self.rows, dtype=object)
        vo = self.vals.astype(object)
        for i in range(self.rows):
            s, e = self.rowptr[i], self.rowptr[i + 1]
            y[i] = int(np.dot(vo[s:e], xo[self.colidx[s:e]])) if e > s else 0
        return y


def _from_coo(rows, cols, r, c, v):
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(rows + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(rows, cols, rowptr, c.astype(np.int32), v)


def uniform_positions(g, rows, cols, nnz, lo, hi):
    """nnz distinct positions uniformly at random, integer values in [lo, hi]."""
    total = rows * cols
    nnz = min(nnz, total)
    flat = g.choice(total, size=nnz, replace=False)
    r = (flat // cols).astype(np.int64)
    c = (flat % cols).astype(np.int64)
    v = g.integers(lo, hi + 1, size=nnz, dtype=np.int64)
    return _from_coo(rows, cols, r, c, v)


def powerlaw_columns(g, rows, cols, nnz, exponent, lo, hi, transpose=False):
    """Per-column counts proportional to rank^-exponent over a random column
    permutation, rows uniform (without replacement) inside each column."""
    w = np.arange(1, cols + 1, dtype=np.float64) ** (-exponent)
    base = nnz * w / w.sum()
    counts = np.minimum(rows, np.floor(base)).astype(np.int64)
    frac = base - np.floor(base)
    order = np.argsort(-frac, kind="stable")
    k = 0
    while counts.sum() < nnz:
        j = order[k % cols]
        if counts[j] < rows:
            counts[j] += 1
        k += 1
    perm = g.permutation(cols)
    rr, cc = [], []
    for rank in range(cols):
        n = int(counts[rank])
        if n == 0:
            continue
        col = int(perm[rank])
        rr.append(g.choice(rows, size=n, replace=False).astype(np.int64))
        cc.append(np.full(n, col, dtype=np.int64))
    r = np.concatenate(rr)
    c = np.concatenate(cc)
    v = g.integers(lo, hi + 1, size=len(r), dtype=np.int64)
    if transpose:
        r, c = c, r
        rows, cols = cols, rows
    return _from_coo(rows, cols, r, c, v)


def stencil27(g, nz, ny, nx):
    """27-point stencil pattern on an nz x ny x nx grid, values U[-1, 1]."""
    rr, cc = [], []
    idx = np.arange(nz * ny * nx).reshape(nz, ny, nx)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                z0, z1 = max(0, -dz), min(nz, nz - dz)
                y0, y1 = max(0, -dy), min(ny, ny - dy)
                x0, x1 = max(0, -dx), min(nx, nx - dx)
                src = idx[z0:z1, y0:y1, x0:x1].ravel()
                dst = idx[z0 + dz:z1 + dz, y0 + dy:y1 + dy, x0 + dx:x1 + dx].ravel()
                rr.append(src)
                cc.append(dst)
    r = np.concatenate(rr).astype(np.int64)
    c = np.concatenate(cc).astype(np.int64)
    n = nz * ny * nx
    csr = _from_coo(n, n, r, c, np.zeros(len(r)))
    csr.vals = g.uniform(-1.0, 1.0, size=len(r))
    return csr


def quantize(x, bits=FIXED_POINT_BITS):
    """Fixed point: round(x * 2^bits) with ties away from zero, as int64."""
    x = np.asarray(x, dtype=np.float64)
    return (np.sign(x) * np.floor(np.abs(x) * (1 << bits) + 0.5)).astype(np.int64)


def loguniform_int(g, lo, hi):
    return int(round(float(np.exp(g.uniform(np.log(lo), np.log(hi))))))


def loguniform(g, lo, hi):
    return float(np.exp(g.uniform(np.log(lo), np.log(hi))))


def random_square(g, n_lo, n_hi, d_lo, d_hi, lo=-15, hi=15):
    n = loguniform_int(g, n_lo, n_hi)
    d = loguniform(g, d_lo, d_hi)
    nnz = max(1, int(round(d * n * n)))
    a = uniform_positions(g, n, n, nnz, lo, hi)
    x = g.integers(lo, hi + 1, size=n, dtype=np.int64)
    return a, x


def workload(name, seed=None, **kw):
    """(A, x) for one configuration; c4 returns a list of 64 pairs and c5 the
    request pool of distinct instances (kw: pool)."""
    g = np.random.default_rng(SEEDS[name] if seed is None else seed)
    if name == "c1":
        a = uniform_positions(g, 512, 512, 2621, -15, 15)
        return a, g.integers(-15, 16, size=512, dtype=np.int64)
    if name == "c2":
        a = powerlaw_columns(g, 4096, 4096, 16777, 1.5, -127, 127,
                             transpose=kw.get("transpose", False))
        return a, g.integers(-127, 128, size=4096, dtype=np.int64)
    if name == "c3":
        a = stencil27(g, 16, 32, 32)
        return a, g.uniform(-1.0, 1.0, size=a.cols)
    if name == "c4":
        return [random_square(g, 256, 8192, 5e-4, 2e-2) for _ in range(kw.get("count", 64))]
    if name == "c5":
        return [random_square(g, 512, 16384, 5e-4, 1e-2) for _ in range(kw.get("pool", 32))]
    raise KeyError(name)


def small_matrix(seed, rows, cols, nnz, lo=-15, hi=15):
    """A small random integer instance (tests)."""
    g = np.random.default_rng(seed)
    a = uniform_positions(g, rows, cols, nnz, lo, hi)
    return a, g.integers(lo, hi + 1, size=cols, dtype=np.int64)
