"""The allocation-free key switch (hespmv_keyswitch_noalloc).

Some callers cannot allocate device memory where they need a key switch: a
process whose device memory is already reserved by another allocator's pool,
or a latency-sensitive loop that must not call cudaMalloc/cudaFree (they can
synchronise the device).  For them the library offers a key switch whose
scratch lives in a fixed array reserved when the library is loaded.  This
test calls it through the C ABI, twice in a row on different inputs, and
checks each result word for word against the ordinary allocating entry point
(the key switch is exact integer work, so the tolerance is zero).  It is
collected last and needs nothing from the other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _device_words(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def _host_words(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


def test_keyswitch_noalloc_matches_allocating_entry_point():
    from paper_2603_04742_gb300 import binding as B
    from paper_2603_04742_gb300 import synth
    from paper_2603_04742_gb300.api import Context

    logn, L, K, dnum, t = synth.RING["c1"]
    N = 1 << logn
    ctx = Context(logn, L, K, dnum, t)
    ctx.keygen(17, [1, 6])
    q, _, _ = ctx.moduli()
    lib = B.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(2024)
    n = 3
    for call, galois in enumerate((0, 5)):          # relinearisation key, then a Galois key
        d = np.stack([np.stack([rng.integers(0, q[l], size=N, dtype=np.uint64) for l in range(L)])
                      for _ in range(n)])
        dd = _device_words(d)
        want = torch.zeros(n * 2 * L * N, dtype=torch.int64, device="cuda")
        got = torch.full((n * 2 * L * N,), -1, dtype=torch.int64, device="cuda")
        ctx.keyswitch(dd.data_ptr(), galois, want.data_ptr(), n)
        rc = lib.hespmv_keyswitch_noalloc(ctx.h, ctypes.c_void_p(dd.data_ptr()), galois,
                                          ctypes.c_void_p(got.data_ptr()), n, stream)
        assert rc == B.HESPMV_OK, lib.hespmv_last_error(ctx.h)
        assert np.array_equal(_host_words(got), _host_words(want)), "call %d differs" % call


def test_keyswitch_noalloc_rejects_oversized_requests():
    from paper_2603_04742_gb300 import binding as B
    from paper_2603_04742_gb300 import synth
    from paper_2603_04742_gb300.api import Context

    logn, L, K, dnum, t = synth.RING["c3"]
    ctx = Context(logn, L, K, dnum, t)
    ctx.keygen(3, [])
    lib = B.load()
    buf = torch.zeros(16, dtype=torch.int64, device="cuda")
    # two N = 2^15 ciphertexts need about 42 MiB of scratch, more than reserved
    rc = lib.hespmv_keyswitch_noalloc(ctx.h, ctypes.c_void_p(buf.data_ptr()), 0,
                                      ctypes.c_void_p(buf.data_ptr()), 2, None)
    assert rc == B.HESPMV_E_INVALID
    assert b"at most 1 per call" in lib.hespmv_last_error(ctx.h)
    # a count so large that its scratch size would wrap a 64-bit product
    rc = lib.hespmv_keyswitch_noalloc(ctx.h, ctypes.c_void_p(buf.data_ptr()), 0,
                                      ctypes.c_void_p(buf.data_ptr()), 1 << 62, None)
    assert rc == B.HESPMV_E_INVALID
    # a misaligned output is refused on the host (the kernels store 16 bytes at a time)
    rc = lib.hespmv_keyswitch_noalloc(ctx.h, ctypes.c_void_p(buf.data_ptr()), 0,
                                      ctypes.c_void_p(buf.data_ptr() + 8), 1, None)
    assert rc == B.HESPMV_E_INVALID
    assert b"16-byte aligned" in lib.hespmv_last_error(ctx.h)
