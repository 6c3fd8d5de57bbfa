"""ctypes binding of the hespmv C ABI (include/hespmv.h).

Argument marshalling only: every function below calls the entry point of the
same name in ``libhespmv.so``.  There is no fallback path: if the library
cannot be built or loaded, loading raises.
"""
import ctypes
import os
from ctypes import (CFUNCTYPE, POINTER, c_char_p, c_int, c_int32, c_int64, c_size_t, c_uint32,
                    c_uint64, c_void_p)

from . import build as _build

HESPMV_OK = 0
HESPMV_E_INVALID = 1
HESPMV_E_NOMEM = 2
HESPMV_E_CUDA = 3
HESPMV_E_RANGE = 4
HESPMV_E_UNSUPPORTED = 5
HESPMV_E_TIMEOUT = 6
HESPMV_E_REJECTED = 7
HESPMV_ROT_POW2 = 0
HESPMV_ROT_EXACT = 1
HESPMV_MATRIX = 0
HESPMV_VECTOR = 1
HESPMV_SCHEME_BGV = 0
HESPMV_SCHEME_CKKS = 1
HESPMV_SCHEME_BFV = 2
HESPMV_KEYS_EVAL = 0
HESPMV_KEYS_ALL = 1
HESPMV_SER_FULL = 0
HESPMV_SER_SHAPE = 1
HESPMV_KEY_SECRET = 0
HESPMV_KEY_PUBLIC = 1
HESPMV_KEY_RELIN = 2
HESPMV_KEY_GALOIS = 3

ERRORS = {1: "E_INVALID", 2: "E_NOMEM", 3: "E_CUDA", 4: "E_RANGE", 5: "E_UNSUPPORTED",
          6: "E_TIMEOUT", 7: "E_REJECTED"}

ALLOC_FN = CFUNCTYPE(c_void_p, c_size_t, c_void_p)
FREE_FN = CFUNCTYPE(None, c_void_p, c_void_p)


class hespmv_params(ctypes.Structure):
    _fields_ = [("log2n", c_int32), ("L", c_int32), ("K", c_int32), ("dnum", c_int32),
                ("t", c_uint64), ("prime_bits", c_int32), ("rot_policy", c_int32),
                ("slots", c_int32), ("device", c_int32), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_user", c_void_p), ("scheme", c_int32),
                ("scale_bits", c_int32), ("mask_scale_bits", c_int32), ("reserved", c_int32)]


class hespmv_tuning(ctypes.Structure):
    _fields_ = [("mult_batch", c_int32), ("rot_batch", c_int32), ("ntt_split", c_int32),
                ("rows_tma", c_int32), ("persistent", c_int32), ("persist_blocks", c_int32),
                ("streams", c_int32), ("ms", ctypes.c_double)]


u64p = POINTER(c_uint64)
i64p = POINTER(c_int64)
i32p = POINTER(c_int32)
szp = POINTER(c_size_t)
f64p = POINTER(ctypes.c_double)

# name -> (restype, argtypes); mirrors include/hespmv.h
SIGNATURES = {
    "hespmv_last_error": (c_char_p, [c_void_p]),
    "hespmv_version": (c_char_p, []),
    "hespmv_create": (c_int, [POINTER(hespmv_params), POINTER(c_void_p)]),
    "hespmv_destroy": (None, [c_void_p]),
    "hespmv_ctx_moduli": (c_int, [c_void_p, u64p, u64p, u64p]),
    "hespmv_ctx_device_bytes": (c_int, [c_void_p, szp]),
    "hespmv_keygen": (c_int, [c_void_p, c_uint64, i32p, c_size_t]),
    "hespmv_key_export": (c_int, [c_void_p, c_int32, c_uint32, u64p, c_size_t]),
    "hespmv_encode_cssc": (c_int, [c_void_p, c_int32, c_int32, c_int64, i64p, i32p, i64p, c_int64,
                                   POINTER(c_void_p)]),
    "hespmv_cssc_free": (None, [c_void_p]),
    "hespmv_cssc_info": (c_int, [c_void_p, i32p, i32p, i64p, i64p, i32p, i32p, i64p]),
    "hespmv_cssc_chunks": (c_int, [c_void_p, i32p, i32p, i32p]),
    "hespmv_cssc_colindex": (c_int, [c_void_p, POINTER(i32p), szp]),
    "hespmv_cssc_arrays": (c_int, [c_void_p, c_int32, POINTER(i64p), POINTER(i32p), szp,
                                   POINTER(i64p), szp, POINTER(i32p), szp, i32p]),
    "hespmv_cssc_rotation_steps": (c_int, [c_void_p, i32p, c_size_t, szp]),
    "hespmv_cssc_serialize": (c_int, [c_void_p, c_int32, c_void_p, c_size_t, szp]),
    "hespmv_cssc_deserialize": (c_int, [c_void_p, c_void_p, c_size_t, POINTER(c_void_p)]),
    "hespmv_ctbatch_create": (c_int, [c_void_p, c_size_t, POINTER(c_void_p)]),
    "hespmv_ctbatch_free": (None, [c_void_p]),
    "hespmv_ctbatch_data": (c_int, [c_void_p, POINTER(u64p), szp]),
    "hespmv_ctbatch_upload": (c_int, [c_void_p, u64p, c_size_t, c_void_p]),
    "hespmv_ctbatch_download": (c_int, [c_void_p, u64p, c_size_t, c_void_p]),
    "hespmv_ctbatch_serialize": (c_int, [c_void_p, c_void_p, c_size_t, szp]),
    "hespmv_keys_serialize": (c_int, [c_void_p, c_int32, c_void_p, c_size_t, szp]),
    "hespmv_device_status": (c_int, [c_void_p, i32p]),
    "hespmv_selftest_wait_timeout": (c_int, [c_void_p, i32p]),
    "hespmv_selftest_persist_timeout": (c_int, [c_void_p, i32p]),
    "hespmv_rescale": (c_int, [c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "hespmv_decrypt_real_level": (c_int, [c_void_p, c_void_p, c_int32, ctypes.c_double, f64p]),
    "hespmv_keys_deserialize": (c_int, [c_void_p, c_void_p, c_size_t]),
    "hespmv_encrypt_real": (c_int, [c_void_p, c_void_p, c_int32, f64p, c_uint64, POINTER(c_void_p)]),
    "hespmv_encode_matrix_plain_real": (c_int, [c_void_p, c_void_p, f64p, POINTER(c_void_p)]),
    "hespmv_ckks_encode": (c_int, [c_void_p, f64p, c_size_t, c_int32, i64p]),
    "hespmv_decrypt_real_slots": (c_int, [c_void_p, c_void_p, c_size_t, c_int32, f64p]),
    "hespmv_decrypt_real": (c_int, [c_void_p, c_void_p, c_void_p, f64p]),
    "hespmv_set_tuning": (c_int, [c_void_p, POINTER(hespmv_tuning)]),
    "hespmv_get_tuning": (c_int, [c_void_p, POINTER(hespmv_tuning)]),
    "hespmv_autotune": (c_int, [c_void_p, c_size_t, POINTER(c_void_p), POINTER(c_void_p),
                                POINTER(c_void_p), c_int32, POINTER(hespmv_tuning),
                                POINTER(hespmv_tuning), c_size_t, szp]),
    "hespmv_ctbatch_deserialize": (c_int, [c_void_p, c_void_p, c_size_t, POINTER(c_void_p)]),
    "hespmv_encrypt": (c_int, [c_void_p, c_void_p, c_int32, i64p, c_uint64, POINTER(c_void_p)]),
    "hespmv_spmv": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_void_p), c_void_p]),
    "hespmv_spmv_host": (c_int, [c_void_p, c_void_p, u64p, u64p, u64p, c_void_p]),
    "hespmv_ct_packed_words": (c_int, [c_void_p, szp, i32p]),
    "hespmv_ct_pack": (c_int, [c_void_p, u64p, c_size_t, u64p]),
    "hespmv_ct_unpack": (c_int, [c_void_p, u64p, c_size_t, u64p]),
    "hespmv_spmv_host_packed": (c_int, [c_void_p, c_void_p, u64p, u64p, u64p, c_void_p]),
    "hespmv_spmv_host_packed_async": (c_int, [c_void_p, c_void_p, u64p, u64p, u64p, c_void_p]),
    "hespmv_set_upload_groups": (c_int, [c_void_p, c_int32]),
    "hespmv_get_upload_groups": (c_int, [c_void_p, i32p]),
    "hespmv_encode_matrix_plain": (c_int, [c_void_p, c_void_p, POINTER(c_void_p)]),
    "hespmv_spmv_ptmatrix": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_void_p),
                                     c_void_p]),
    "hespmv_spmv_batched": (c_int, [c_void_p, c_size_t, POINTER(c_void_p), POINTER(c_void_p),
                                    POINTER(c_void_p), POINTER(c_void_p), c_void_p]),
    "hespmv_decrypt": (c_int, [c_void_p, c_void_p, c_void_p, i64p]),
    "hespmv_decrypt_slots": (c_int, [c_void_p, c_void_p, c_size_t, u64p]),
    "hespmv_ntt_forward": (c_int, [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_void_p]),
    "hespmv_ntt_inverse": (c_int, [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_void_p]),
    "hespmv_he_add": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "hespmv_he_tensor": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "hespmv_he_relin": (c_int, [c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "hespmv_he_mult": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "hespmv_he_rotate": (c_int, [c_void_p, c_void_p, c_int32, c_void_p, c_size_t, c_void_p]),
    "hespmv_he_cmult_mask": (c_int, [c_void_p, c_void_p, c_int32, c_void_p, c_size_t, c_void_p]),
    "hespmv_keyswitch": (c_int, [c_void_p, c_void_p, c_uint32, c_void_p, c_size_t, c_void_p]),
    "hespmv_keyswitch_noalloc": (c_int, [c_void_p, c_void_p, c_uint32, c_void_p, c_size_t,
                                         c_void_p]),
    "hespmv_set_graphs": (c_int, [c_void_p, c_int32]),
    "hespmv_server_start": (c_int, [c_void_p, c_int32, c_size_t, c_int32, POINTER(c_void_p)]),
    "hespmv_server_submit": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                     POINTER(c_uint64)]),
    "hespmv_server_poll": (c_int, [c_void_p, c_uint64, i32p, i64p]),
    "hespmv_server_stats": (c_int, [c_void_p, i64p, i64p, i64p, i64p, i64p]),
    "hespmv_server_stop": (c_int, [c_void_p, c_int64]),
    "hespmv_profile_enable": (c_int, [c_void_p, c_int32]),
    "hespmv_profile_count": (c_int, [c_void_p, i32p]),
    "hespmv_profile_entry": (c_int, [c_void_p, c_int32, POINTER(c_char_p), i64p,
                                     POINTER(ctypes.c_double)]),
    "hespmv_mulmod_rate": (c_int, [c_void_p, c_int32, POINTER(ctypes.c_double)]),
}

_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libhespmv.so (building it first if it is absent); raises on failure."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        _build.build()   # incremental: only stale translation units recompile
    elif not os.path.exists(path):
        raise RuntimeError("hespmv library not built: %s" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class HespmvError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (ERRORS.get(code, code), msg))
        self.code = code


def check(code, ctx=None):
    if code != HESPMV_OK:
        msg = ""
        if ctx is not None:
            m = load().hespmv_last_error(ctx)
            msg = m.decode() if m else ""
        raise HespmvError(code, msg)
