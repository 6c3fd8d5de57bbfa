"""Build and load the oracle's C arithmetic (TEST INFRASTRUCTURE ONLY)."""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "he_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libhe_oracle.so")

_lib = None


def build(force=False):
    """Compile he_oracle.c with the host C compiler (portable flags only)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.or_mulmod_vec.argtypes = [u64p, u64p, u64p, ctypes.c_int64, ctypes.c_uint64]
        L.or_mulmod_scalar.argtypes = [u64p, ctypes.c_uint64, u64p, ctypes.c_int64,
                                       ctypes.c_uint64]
        L.or_ntt_forward.argtypes = [u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]
        L.or_ntt_inverse.argtypes = [u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a


def mulmod(a, b, q):
    """Elementwise a*b mod q (exact)."""
    a = _u64(a)
    b = _u64(b)
    out = np.empty_like(a)
    lib().or_mulmod_vec(_p(a), _p(b), _p(out), a.size, int(q))
    return out


def mulmod_scalar(a, s, q):
    """Elementwise a*s mod q (exact)."""
    a = _u64(a)
    out = np.empty_like(a)
    lib().or_mulmod_scalar(_p(a), int(s) % (1 << 64), _p(out), a.size, int(q))
    return out


def ntt(a, q, psi):
    """Forward negacyclic NTT of one polynomial (copy)."""
    a = _u64(a).copy()
    logn = a.size.bit_length() - 1
    lib().or_ntt_forward(_p(a), logn, int(q), int(psi))
    return a


def intt(a, q, psi):
    """Inverse negacyclic NTT of one polynomial (copy)."""
    a = _u64(a).copy()
    logn = a.size.bit_length() - 1
    lib().or_ntt_inverse(_p(a), logn, int(q), int(psi))
    return a
