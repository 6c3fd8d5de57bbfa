"""Failure handling without faulting the GPU: a device allocator that
refuses (injected on the host through the allocator callback) makes the
call fail with E_NOMEM and leaves the context usable; bad inputs are
refused before any launch."""
import numpy as np
import pytest

from paper_2603_04742_gb300 import binding as B
from paper_2603_04742_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_allocation_failure_returns_nomem_and_context_survives():
    from paper_2603_04742_gb300.api import Context, TorchAllocator

    class Refusing(TorchAllocator):
        refuse = False

        def _alloc(self, nbytes, user):
            if self.refuse:
                return 0
            return super()._alloc(nbytes, user)

    alloc = Refusing(0)
    logn, L, K, dnum, t = synth.RING["c1"]
    ctx = Context(logn, L, K, dnum, t, allocator=alloc)
    ctx.keygen(1)
    A, x = synth.small_matrix(4, 300, 300, 2000)
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    alloc.refuse = True
    with pytest.raises(B.HespmvError) as e:
        ctx.encrypt(m, B.HESPMV_MATRIX, seed=1)
    assert e.value.code == B.HESPMV_E_NOMEM
    alloc.refuse = False
    ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=1)
    cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=2)
    y = ctx.spmv(m, ca, cx)
    assert list(ctx.decrypt(m, y)) == list(A.matvec(x))


def test_bad_arguments_are_refused_before_any_launch():
    from paper_2603_04742_gb300.api import Context
    logn, L, K, dnum, t = synth.RING["c1"]
    ctx = Context(logn, L, K, dnum, t)
    ctx.keygen(1)
    lib = B.load()
    buf = torch.zeros(2 * L * (1 << logn) + 1, dtype=torch.int64, device="cuda")
    import ctypes
    # misaligned device buffer (8 bytes past a 16-byte boundary)
    rc = lib.hespmv_keyswitch(ctx.h, ctypes.c_void_p(buf.data_ptr() + 8), 0,
                              ctypes.c_void_p(buf.data_ptr()), 1, None)
    assert rc == B.HESPMV_E_INVALID
    # misaligned output buffer: refused on the host, before any 16-byte store
    rc = lib.hespmv_keyswitch(ctx.h, ctypes.c_void_p(buf.data_ptr()), 0,
                              ctypes.c_void_p(buf.data_ptr() + 8), 1, None)
    assert rc == B.HESPMV_E_INVALID
    for fn in (lib.hespmv_he_mult, lib.hespmv_he_tensor, lib.hespmv_he_add):
        rc = fn(ctx.h, ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr() + 8),
                ctypes.c_void_p(buf.data_ptr()), 1, None)
        assert rc == B.HESPMV_E_INVALID
    # a Galois element without a key
    rc = lib.hespmv_keyswitch(ctx.h, ctypes.c_void_p(buf.data_ptr()), 3,
                              ctypes.c_void_p(buf.data_ptr()), 1, None)
    assert rc == B.HESPMV_E_INVALID
    # operand batches smaller than the chunk count
    A, x = synth.small_matrix(2, 200, 200, 1500)
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    from paper_2603_04742_gb300.api import CtBatch
    small = CtBatch.create(ctx, 0)
    with pytest.raises(B.HespmvError) as e:
        ctx.spmv(m, small, small)
    assert e.value.code == B.HESPMV_E_INVALID
    # the context still evaluates correctly afterwards
    ca = ctx.encrypt(m, B.HESPMV_MATRIX, seed=3)
    cx = ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=4)
    assert list(ctx.decrypt(m, ctx.spmv(m, ca, cx))) == list(A.matvec(x))


def test_bounded_device_wait_reports_timeout():
    """A device-side wait that cannot complete gives up, the host reads
    HESPMV_E_TIMEOUT, and the context keeps working."""
    from paper_2603_04742_gb300.api import Context
    logn, L, K, dnum, t = synth.RING["c1"]
    ctx = Context(logn, L, K, dnum, t)
    ctx.keygen(1)
    rc, code = ctx.selftest_wait_timeout()
    assert rc == B.HESPMV_E_TIMEOUT and code == 1
    ctx.device_status()                       # cleared: no error now
    A, x = synth.workload("c1")
    m = ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    y = ctx.spmv(m, ctx.encrypt(m, B.HESPMV_MATRIX, seed=1), ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=2))
    assert list(ctx.decrypt(m, y)) == list(A.matvec(x))
