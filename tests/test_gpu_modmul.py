"""Exact residue products on the device.

The tensor product of two ciphertexts (Section 2.1, HE-Mult before
relinearisation: d = (a0 b0, a0 b1 + a1 b0, a1 b1), residue by residue in
the evaluation domain) is compared with Python integer arithmetic on
residues at the edges of [0, q): 0, 1, q - 1, q - 2, (q - 1) / 2, q / 3 and
random values, each edge paired with every other.  Primes of 20, 32, 33,
40 and 50 bits run the product's quotient estimate with no shift (2k <= 64),
with short shifts and with the 36-bit shift of the 50-bit primes."""
import numpy as np
import pytest

from oracle.params import plain_modulus

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _residues(g, q, N):
    edge = [0, 1, q - 1, q - 2, (q - 1) // 2, q // 3]
    a = [int(v) for v in g.integers(0, q, size=N, dtype=np.uint64)]
    b = [int(v) for v in g.integers(0, q, size=N, dtype=np.uint64)]
    k = 0
    for x in edge:  # every pair of edges, then random values
        for y in edge:
            a[k], b[k] = x, y
            k += 1
    return a, b


@pytest.mark.parametrize("bits", [20, 32, 33, 40, 50])
def test_tensor_exact_at_residue_edges(bits):
    from paper_2603_04742_gb300.api import Context
    logn, L = 10, 3
    N = 1 << logn
    ctx = Context(logn, L, 1, 3, plain_modulus(N, 1 << 16), prime_bits=bits)
    qs = ctx.moduli()[0][:L]
    assert all(q.bit_length() == bits for q in qs)
    g = np.random.default_rng(bits)
    A = np.zeros((2, L, N), dtype=np.uint64)
    Bm = np.zeros((2, L, N), dtype=np.uint64)
    for c in range(2):
        for l, q in enumerate(qs):
            a, b = _residues(g, q, N)
            if c == 1:  # other pairings for the cross terms
                a, b = b[::-1], a
            A[c, l] = a
            Bm[c, l] = b
    da = torch.from_numpy(A.view(np.int64).reshape(-1)).cuda()
    db = torch.from_numpy(Bm.view(np.int64).reshape(-1)).cuda()
    d = torch.zeros(3 * L * N, dtype=torch.int64, device="cuda")
    ctx.he_tensor(da.data_ptr(), db.data_ptr(), d.data_ptr())
    torch.cuda.synchronize()
    got = d.cpu().numpy().view(np.uint64).reshape(3, L, N)
    for l, q in enumerate(qs):
        a0, a1 = [int(v) for v in A[0, l]], [int(v) for v in A[1, l]]
        b0, b1 = [int(v) for v in Bm[0, l]], [int(v) for v in Bm[1, l]]
        want0 = [x * y % q for x, y in zip(a0, b0)]
        want1 = [(x * y + u * v) % q for x, y, u, v in zip(a0, b1, a1, b0)]
        want2 = [x * y % q for x, y in zip(a1, b1)]
        assert [int(v) for v in got[0, l]] == want0, (bits, l)
        assert [int(v) for v in got[1, l]] == want1, (bits, l)
        assert [int(v) for v in got[2, l]] == want2, (bits, l)
