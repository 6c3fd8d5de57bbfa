"""Python front end of the hespmv C ABI.

Thin wrappers that marshal arguments to the entry points of the same names
(``hespmv_create``, ``hespmv_keygen``, ``hespmv_encode_cssc``,
``hespmv_encrypt``, ``hespmv_spmv``, ``hespmv_decrypt`` ...).  PyTorch is
used only as the device allocator (the caching allocator backs every device
buffer the library asks for) and as the source of CUDA streams.
"""
import ctypes
from ctypes import byref, c_int32, c_int64, c_size_t, c_uint64, c_void_p

import numpy as np

from . import binding as B


def _u64p(a):
    return a.ctypes.data_as(B.u64p)


def _i64p(a):
    return a.ctypes.data_as(B.i64p)


def _f64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i32p(a):
    return a.ctypes.data_as(B.i32p)


def _stream_handle(stream):
    if stream is None:
        import torch
        return c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return c_void_p(stream)
    return c_void_p(stream.cuda_stream)


class TorchAllocator:
    """Device allocations through PyTorch's caching allocator."""

    def __init__(self, device):
        import torch
        self._torch = torch
        self.device = device
        self.live = {}
        self.alloc_fn = B.ALLOC_FN(self._alloc)
        self.free_fn = B.FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        t = self._torch.empty(int(nbytes), dtype=self._torch.uint8, device="cuda:%d" % self.device)
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ptr, user):
        self.live.pop(ptr, None)


class Context:
    """Scheme parameters, tables and keys on one GPU (hespmv_create)."""

    def __init__(self, log2n, L, K, dnum, t, rot_policy="pow2", slots=0, device=0,
                 torch_alloc=True, prime_bits=0, allocator=None, scheme="bgv", scale_bits=40,
                 mask_scale_bits=30):
        self.lib = B.load()
        if allocator is not None:
            self.allocator = allocator
        else:
            self.allocator = TorchAllocator(device) if torch_alloc else None
        p = B.hespmv_params()
        p.log2n, p.L, p.K, p.dnum, p.t = log2n, L, K, dnum, t
        p.prime_bits = prime_bits
        p.rot_policy = B.HESPMV_ROT_EXACT if rot_policy == "exact" else B.HESPMV_ROT_POW2
        p.slots = slots
        p.device = device
        p.scheme = {"bgv": B.HESPMV_SCHEME_BGV, "ckks": B.HESPMV_SCHEME_CKKS,
                    "bfv": B.HESPMV_SCHEME_BFV}[scheme]
        p.scale_bits, p.mask_scale_bits = scale_bits, mask_scale_bits
        if self.allocator is not None:
            p.alloc = self.allocator.alloc_fn
            p.free = self.allocator.free_fn
        self._params = p
        h = c_void_p()
        rc = self.lib.hespmv_create(byref(p), byref(h))
        self.h = h
        if rc != B.HESPMV_OK:
            msg = self.lib.hespmv_last_error(h).decode() if h else ""
            if h:
                self.lib.hespmv_destroy(h)
                self.h = None
            raise B.HespmvError(rc, msg)
        self.N = 1 << log2n
        self.L, self.K, self.dnum, self.t = L, K, dnum, t
        self.device = device
        self.scheme = scheme
        self.scale_bits, self.mask_scale_bits = scale_bits, mask_scale_bits

    def close(self):
        if getattr(self, "h", None):
            self.lib.hespmv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc):
        B.check(rc, self.h)

    def moduli(self):
        n = self.L + self.K
        q = np.zeros(n, dtype=np.uint64)
        psi = np.zeros(n, dtype=np.uint64)
        z = np.zeros(1, dtype=np.uint64)
        self.check(self.lib.hespmv_ctx_moduli(self.h, _u64p(q), _u64p(psi), _u64p(z)))
        return [int(v) for v in q], [int(v) for v in psi], int(z[0])

    def device_bytes(self):
        n = c_size_t()
        self.check(self.lib.hespmv_ctx_device_bytes(self.h, byref(n)))
        return n.value

    def keygen(self, seed, rot_steps=None):
        if rot_steps is None:
            self.check(self.lib.hespmv_keygen(self.h, c_uint64(seed), None, 0))
        else:
            a = np.ascontiguousarray(list(rot_steps) + [0], dtype=np.int32)   # never NULL
            self.check(self.lib.hespmv_keygen(self.h, c_uint64(seed), _i32p(a), len(a) - 1))

    def key_export(self, which, galois=0):
        N, L, LK = self.N, self.L, self.L + self.K
        size = {B.HESPMV_KEY_SECRET: LK * N, B.HESPMV_KEY_PUBLIC: 2 * L * N,
                B.HESPMV_KEY_RELIN: self.dnum * 2 * LK * N,
                B.HESPMV_KEY_GALOIS: self.dnum * 2 * LK * N}[which]
        out = np.zeros(size, dtype=np.uint64)
        self.check(self.lib.hespmv_key_export(self.h, which, galois, _u64p(out), size))
        return out

    def encode_cssc(self, csr_rows, csr_cols, rowptr, colidx, vals, max_abs_x=0):
        return Cssc(self, csr_rows, csr_cols, rowptr, colidx, vals, max_abs_x)

    def keys_serialize(self, what=B.HESPMV_KEYS_EVAL):
        """Evaluation keys (or, HESPMV_KEYS_ALL, every key) as bytes."""
        n = c_size_t()
        self.check(self.lib.hespmv_keys_serialize(self.h, what, None, 0, byref(n)))
        buf = ctypes.create_string_buffer(max(1, n.value))
        self.check(self.lib.hespmv_keys_serialize(self.h, what, buf, n.value, byref(n)))
        return buf.raw[:n.value]

    def keys_deserialize(self, data):
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        self.check(self.lib.hespmv_keys_deserialize(self.h, buf, len(data)))

    def cssc_from_bytes(self, data):
        """A plan from Cssc.serialize output (hespmv_cssc_deserialize)."""
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        h = c_void_p()
        self.check(self.lib.hespmv_cssc_deserialize(self.h, buf, len(data), byref(h)))
        return Cssc.from_handle(self, h)

    def ctbatch_from_bytes(self, data):
        """A device batch from CtBatch.serialize output."""
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        h = c_void_p()
        self.check(self.lib.hespmv_ctbatch_deserialize(self.h, buf, len(data), byref(h)))
        return CtBatch(self, h)

    def encrypt(self, m, which, x=None, seed=0):
        out = c_void_p()
        xp = None
        if x is not None:
            xa = np.ascontiguousarray(x, dtype=np.int64)
            xp = _i64p(xa)
        self.check(self.lib.hespmv_encrypt(self.h, m.h, which, xp, c_uint64(seed), byref(out)))
        return CtBatch(self, out)

    # ---- CKKS ----
    def encrypt_real(self, m, which, values, seed=0):
        out = c_void_p()
        v = np.ascontiguousarray(values, dtype=np.float64)
        self.check(self.lib.hespmv_encrypt_real(self.h, m.h, which, _f64p(v), c_uint64(seed),
                                                byref(out)))
        return CtBatch(self, out)

    def encode_matrix_plain_real(self, m, vals):
        out = c_void_p()
        v = np.ascontiguousarray(vals, dtype=np.float64)
        self.check(self.lib.hespmv_encode_matrix_plain_real(self.h, m.h, _f64p(v), byref(out)))
        return CtBatch(self, out)

    def ckks_encode(self, z, scale_bits):
        zz = np.ascontiguousarray(z, dtype=np.float64)
        out = np.zeros(self.N, dtype=np.int64)
        self.check(self.lib.hespmv_ckks_encode(self.h, _f64p(zz), len(zz), scale_bits, _i64p(out)))
        return out

    def decrypt_real(self, m, y):
        out = np.zeros(m.rows, dtype=np.float64)
        self.check(self.lib.hespmv_decrypt_real(self.h, m.h, y.h, _f64p(out)))
        return out

    def decrypt_real_slots(self, b, index, scale_bits):
        out = np.zeros(self.N // 2, dtype=np.float64)
        self.check(self.lib.hespmv_decrypt_real_slots(self.h, b.h, index, scale_bits, _f64p(out)))
        return out

    def spmv(self, m, A, X, y=None, stream=None):
        yh = c_void_p(y.h.value if y is not None else None)
        self.check(self.lib.hespmv_spmv(self.h, m.h, A.h, X.h, byref(yh), _stream_handle(stream)))
        return y if y is not None else CtBatch(self, yh)

    def encode_matrix_plain(self, m):
        out = c_void_p()
        self.check(self.lib.hespmv_encode_matrix_plain(self.h, m.h, byref(out)))
        return CtBatch(self, out)

    def spmv_ptmatrix(self, m, Aplain, X, y=None, stream=None):
        yh = c_void_p(y.h.value if y is not None else None)
        self.check(self.lib.hespmv_spmv_ptmatrix(self.h, m.h, Aplain.h, X.h, byref(yh),
                                                 _stream_handle(stream)))
        return y if y is not None else CtBatch(self, yh)

    def spmv_batched(self, ms, As, Xs, ys=None, stream=None):
        n = len(ms)
        arr = c_void_p * n
        mh = arr(*[m.h for m in ms])
        ah = arr(*[a.h for a in As])
        xh = arr(*[x.h for x in Xs])
        yh = arr(*[(y.h if y is not None else None) for y in (ys or [None] * n)])
        self.check(self.lib.hespmv_spmv_batched(self.h, n, mh, ah, xh, yh, _stream_handle(stream)))
        if ys is not None and all(y is not None for y in ys):
            return ys
        return [CtBatch(self, c_void_p(yh[i])) for i in range(n)]

    def spmv_host(self, m, A_host, X_host, y_host, stream=None):
        self.check(self.lib.hespmv_spmv_host(self.h, m.h, _u64p(A_host), _u64p(X_host),
                                             _u64p(y_host), _stream_handle(stream)))

    def spmv_host_packed_async(self, m, A_packed, X_packed, y_packed, stream=None):
        """Enqueue only: the buffers must outlive the stream's progress past
        this call (synchronise the stream before reading y_packed)."""
        self.check(self.lib.hespmv_spmv_host_packed_async(self.h, m.h, _u64p(A_packed), _u64p(X_packed),
                                                          _u64p(y_packed), _stream_handle(stream)))

    def set_upload_groups(self, groups):
        """Upload groups of the host-buffer evaluations (0: the defaults)."""
        self.check(self.lib.hespmv_set_upload_groups(self.h, groups))

    def get_upload_groups(self):
        g = c_int32()
        self.check(self.lib.hespmv_get_upload_groups(self.h, byref(g)))
        return g.value

    # ---- packed ciphertexts (W bits per residue) ----
    def ct_packed_words(self):
        """(u64 words of one packed ciphertext, bits per residue W)."""
        w, b = c_size_t(0), c_int32(0)
        self.check(self.lib.hespmv_ct_packed_words(self.h, byref(w), byref(b)))
        return w.value, b.value

    def ct_pack(self, cts):
        cts = np.ascontiguousarray(cts, dtype=np.uint64)
        n = cts.size // (2 * self.L * self.N)
        assert cts.size == n * 2 * self.L * self.N
        out = np.zeros((n, self.ct_packed_words()[0]), dtype=np.uint64)
        self.check(self.lib.hespmv_ct_pack(self.h, _u64p(cts), n, _u64p(out)))
        return out

    def ct_unpack(self, packed):
        packed = np.ascontiguousarray(packed, dtype=np.uint64)
        w = self.ct_packed_words()[0]
        n = packed.size // w
        assert packed.size == n * w
        out = np.zeros((n, 2, self.L, self.N), dtype=np.uint64)
        self.check(self.lib.hespmv_ct_unpack(self.h, _u64p(packed), n, _u64p(out)))
        return out

    def spmv_host_packed(self, m, A_packed, X_packed, y_packed, stream=None):
        self.check(self.lib.hespmv_spmv_host_packed(self.h, m.h, _u64p(A_packed), _u64p(X_packed),
                                                    _u64p(y_packed), _stream_handle(stream)))

    def decrypt(self, m, y):
        out = np.zeros(m.rows, dtype=np.int64)
        self.check(self.lib.hespmv_decrypt(self.h, m.h, y.h, _i64p(out)))
        return out

    def decrypt_slots(self, b, index=0):
        out = np.zeros(self.N, dtype=np.uint64)
        self.check(self.lib.hespmv_decrypt_slots(self.h, b.h, index, _u64p(out)))
        return out

    # ---- schedule tuning ----
    def set_tuning(self, mult_batch=0, rot_batch=0, ntt_split=0, rows_tma=0, persistent=0,
                   persist_blocks=0, streams=1):
        t = B.hespmv_tuning(mult_batch, rot_batch, ntt_split, rows_tma, persistent, persist_blocks, streams,
                            0.0)
        self.check(self.lib.hespmv_set_tuning(self.h, byref(t)))

    def get_tuning(self):
        t = B.hespmv_tuning()
        self.check(self.lib.hespmv_get_tuning(self.h, byref(t)))
        return {"mult_batch": t.mult_batch, "rot_batch": t.rot_batch, "ntt_split": t.ntt_split,
                "rows_tma": t.rows_tma, "persistent": t.persistent, "persist_blocks": t.persist_blocks,
                "streams": t.streams}

    def tuning_key(self, ms):
        """Cache key of a workload: device, ring and the stage sizes that the
        schedule depends on (chunks, rotation chunks, instances)."""
        import torch
        name = torch.cuda.get_device_name(self.device) if self.device >= 0 else "host"
        chunks = sum(m.n_chunks for m in ms)
        rot = sum(int((m.chunks()[1] > 1).sum()) for m in ms)
        return "%s|N=%d|L=%d|K=%d|dnum=%d|inst=%d|chunks=%d|rot=%d" % (
            name, self.N, self.L, self.K, self.dnum, len(ms), chunks, rot)

    def autotune(self, ms, As, Xs, reps=3, cache=None):
        """Time candidate schedules on these SpMVs (hespmv_autotune), apply the
        fastest and return {"best": ..., "tried": [...], "cached": bool}.
        With `cache` (a JSON file path) a result stored under the same
        tuning_key is applied without timing, and new results are stored."""
        import json
        import os
        key = self.tuning_key(ms)
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
            if key in table:
                b = table[key]["best"]
                self.set_tuning(b["mult_batch"], b["rot_batch"], b["ntt_split"], b.get("rows_tma", 0),
                                b.get("persistent", 0), b.get("persist_blocks", 0), b.get("streams", 1))
                return {"best": b, "tried": table[key].get("tried", []), "cached": True}
        n = len(ms)
        arr = c_void_p * n
        mh = arr(*[m.h for m in ms])
        ah = arr(*[a.h for a in As])
        xh = arr(*[x.h for x in Xs])
        best = B.hespmv_tuning()
        cap = 64
        tried = (B.hespmv_tuning * cap)()
        nt = c_size_t()
        self.check(self.lib.hespmv_autotune(self.h, n, mh, ah, xh, reps, byref(best), tried, cap,
                                            byref(nt)))

        def as_dict(t):
            return {"mult_batch": t.mult_batch, "rot_batch": t.rot_batch,
                    "ntt_split": t.ntt_split, "rows_tma": t.rows_tma, "persistent": t.persistent,
                    "persist_blocks": t.persist_blocks, "streams": t.streams, "ms": t.ms}
        out = {"best": as_dict(best), "tried": [as_dict(tried[i]) for i in range(min(cap, nt.value))],
               "cached": False}
        if cache:
            table[key] = {"best": out["best"], "tried": out["tried"]}
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return out

    def device_status(self):
        """Raises HespmvError(E_TIMEOUT) if a device-side wait ran out."""
        code = c_int32()
        self.check(self.lib.hespmv_device_status(self.h, byref(code)))

    def selftest_wait_timeout(self):
        code = c_int32()
        rc = self.lib.hespmv_selftest_wait_timeout(self.h, byref(code))
        return rc, code.value

    def rescale(self, ct_ptr, out_ptr, n=1, stream=None):
        """CKKS: out = ct divided by the last prime (hespmv_rescale); device
        addresses of [n][2][L][N] and [n][2][L-1][N] words."""
        self.check(self.lib.hespmv_rescale(self.h, c_void_p(ct_ptr), c_void_p(out_ptr), n,
                                           _stream_handle(stream)))

    def decrypt_real_level(self, ct_ptr, limbs, scale):
        """CKKS: the N/2 slot values of one ciphertext over its first `limbs`
        primes, divided by `scale`."""
        out = np.zeros(self.N // 2, dtype=np.float64)
        self.check(self.lib.hespmv_decrypt_real_level(self.h, c_void_p(ct_ptr), limbs, float(scale), _f64p(out)))
        return out

    def selftest_persist_timeout(self):
        code = c_int32()
        rc = self.lib.hespmv_selftest_persist_timeout(self.h, byref(code))
        return rc, code.value

    def set_graphs(self, on=True):
        self.check(self.lib.hespmv_set_graphs(self.h, 1 if on else 0))

    # ---- measurement ----
    def profile_enable(self, on=True):
        self.check(self.lib.hespmv_profile_enable(self.h, 1 if on else 0))

    def profile_read(self):
        """{kernel name: (launches, device ms)} since profile_enable (synchronises)."""
        n = c_int32()
        self.check(self.lib.hespmv_profile_count(self.h, byref(n)))
        out = {}
        for i in range(n.value):
            name = ctypes.c_char_p()
            cnt = c_int64()
            ms = ctypes.c_double()
            self.check(self.lib.hespmv_profile_entry(self.h, i, byref(name), byref(cnt), byref(ms)))
            out[name.value.decode()] = (cnt.value, ms.value)
        return out

    def mulmod_rate(self, kind=0):
        r = ctypes.c_double()
        self.check(self.lib.hespmv_mulmod_rate(self.h, kind, byref(r)))
        return r.value

    # ---- primitives on device pointers (ints) ----
    def ntt(self, ptr, prime0, n_limbs, n_items=1, inverse=False, stream=None):
        fn = self.lib.hespmv_ntt_inverse if inverse else self.lib.hespmv_ntt_forward
        self.check(fn(self.h, c_void_p(ptr), prime0, n_limbs, n_items, _stream_handle(stream)))

    def he_add(self, a, b, out, n=1, stream=None):
        self.check(self.lib.hespmv_he_add(self.h, c_void_p(a), c_void_p(b), c_void_p(out), n,
                                          _stream_handle(stream)))

    def he_tensor(self, a, b, d, n=1, stream=None):
        self.check(self.lib.hespmv_he_tensor(self.h, c_void_p(a), c_void_p(b), c_void_p(d), n,
                                             _stream_handle(stream)))

    def he_relin(self, d, out, n=1, stream=None):
        self.check(self.lib.hespmv_he_relin(self.h, c_void_p(d), c_void_p(out), n,
                                            _stream_handle(stream)))

    def he_mult(self, a, b, out, n=1, stream=None):
        self.check(self.lib.hespmv_he_mult(self.h, c_void_p(a), c_void_p(b), c_void_p(out), n,
                                           _stream_handle(stream)))

    def he_rotate(self, ct, k, out, n=1, stream=None):
        self.check(self.lib.hespmv_he_rotate(self.h, c_void_p(ct), k, c_void_p(out), n,
                                             _stream_handle(stream)))

    def he_cmult_mask(self, ct, r, out, n=1, stream=None):
        self.check(self.lib.hespmv_he_cmult_mask(self.h, c_void_p(ct), r, c_void_p(out), n,
                                                 _stream_handle(stream)))

    def keyswitch(self, d, galois, out, n=1, stream=None):
        self.check(self.lib.hespmv_keyswitch(self.h, c_void_p(d), galois, c_void_p(out), n,
                                             _stream_handle(stream)))


class Server:
    """Continuous-batching serving loop (hespmv_server_*)."""

    def __init__(self, ctx, slots=2, mem_budget_bytes=8 << 30, max_batch=16):
        self.ctx = ctx
        self.lib = ctx.lib
        h = c_void_p()
        ctx.check(self.lib.hespmv_server_start(ctx.h, slots, mem_budget_bytes, max_batch, byref(h)))
        self.h = h

    def submit(self, m, A, X, y=None):
        t = c_uint64()
        rc = self.lib.hespmv_server_submit(self.h, m.h, A.h, X.h, y.h if y is not None else None,
                                           byref(t))
        self.ctx.check(rc)
        return t.value

    def poll(self, ticket):
        """(done, latency_ns): done 1 finished, 0 pending, -1 failed."""
        d = c_int32()
        lat = c_int64()
        rc = self.lib.hespmv_server_poll(self.h, ticket, byref(d), byref(lat))
        if rc != B.HESPMV_OK and d.value != -1:
            self.ctx.check(rc)
        return d.value, lat.value

    def stats(self):
        v = [c_int64() for _ in range(5)]
        self.ctx.check(self.lib.hespmv_server_stats(self.h, *[byref(x) for x in v]))
        return dict(zip(["submitted", "completed", "batches", "rejected", "max_inflight"],
                        [x.value for x in v]))

    def stop(self, timeout_ms=-1):
        if getattr(self, "h", None):
            h, self.h = self.h, None
            return self.lib.hespmv_server_stop(h, timeout_ms)
        return B.HESPMV_OK

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


class Cssc:
    """Client-side CSSC form, partitions and chunk plan (hespmv_encode_cssc)."""

    def __init__(self, ctx, rows, cols, rowptr, colidx, vals, max_abs_x=0):
        self.ctx = ctx
        self.lib = ctx.lib
        rp = np.ascontiguousarray(rowptr, dtype=np.int64)
        ci = np.ascontiguousarray(colidx, dtype=np.int32)
        # real values (CKKS) are given to encrypt_real: the plan records positions only
        real = vals is None or np.asarray(vals).dtype.kind == "f"
        va = None if real else np.ascontiguousarray(vals, dtype=np.int64)
        h = c_void_p()
        ctx.check(self.lib.hespmv_encode_cssc(ctx.h, rows, cols, int(rp[-1]) if len(rp) else 0,
                                              _i64p(rp), _i32p(ci),
                                              _i64p(va) if va is not None else None,
                                              c_int64(max_abs_x), byref(h)))
        self._attach(h)

    @classmethod
    def from_handle(cls, ctx, h):
        self = cls.__new__(cls)
        self.ctx = ctx
        self.lib = ctx.lib
        self._attach(h)
        return self

    def _attach(self, h):
        self.h = h
        info = [c_int32(), c_int32(), c_int64(), c_int64(), c_int32(), c_int32(), c_int64()]
        self.ctx.check(self.lib.hespmv_cssc_info(h, *[byref(v) for v in info]))
        (self.n_parts, self.n_chunks, self.n_rot, self.n_keyswitch, self.rows, self.cols,
         self.nnz) = [v.value for v in info]

    def serialize(self, kind=B.HESPMV_SER_FULL):
        """Bytes of hespmv_cssc_serialize (FULL: every array; SHAPE: chunk shapes only)."""
        n = c_size_t()
        self.ctx.check(self.lib.hespmv_cssc_serialize(self.h, kind, None, 0, byref(n)))
        buf = ctypes.create_string_buffer(max(1, n.value))
        self.ctx.check(self.lib.hespmv_cssc_serialize(self.h, kind, buf, n.value, byref(n)))
        return buf.raw[:n.value]

    def chunks(self):
        n = self.n_chunks
        h = np.zeros(n, dtype=np.int32)
        c = np.zeros(n, dtype=np.int32)
        p = np.zeros(n, dtype=np.int32)
        self.ctx.check(self.lib.hespmv_cssc_chunks(self.h, _i32p(h), _i32p(c), _i32p(p)))
        return h, c, p

    def colindex(self):
        ptr = B.i32p()
        n = c_size_t()
        self.ctx.check(self.lib.hespmv_cssc_colindex(self.h, byref(ptr), byref(n)))
        return np.ctypeslib.as_array(ptr, shape=(n.value,)).copy() if n.value else np.zeros(0, np.int32)

    def arrays(self, part):
        va, ci, cp, rm = B.i64p(), B.i32p(), B.i64p(), B.i32p()
        nv, ncp, nrm = c_size_t(), c_size_t(), c_size_t()
        row0 = c_int32()
        self.ctx.check(self.lib.hespmv_cssc_arrays(self.h, part, byref(va), byref(ci), byref(nv),
                                                   byref(cp), byref(ncp), byref(rm), byref(nrm),
                                                   byref(row0)))

        def arr(p, n, dt):
            return np.ctypeslib.as_array(p, shape=(n,)).copy() if n else np.zeros(0, dt)
        return (arr(va, nv.value, np.int64), arr(ci, nv.value, np.int32),
                arr(cp, ncp.value, np.int64), arr(rm, nrm.value, np.int32), row0.value)

    def rotation_steps(self):
        n = c_size_t()
        self.ctx.check(self.lib.hespmv_cssc_rotation_steps(self.h, None, 0, byref(n)))
        out = np.zeros(max(1, n.value), dtype=np.int32)
        self.ctx.check(self.lib.hespmv_cssc_rotation_steps(self.h, _i32p(out), n.value, byref(n)))
        return [int(v) for v in out[:n.value]]

    def close(self):
        if getattr(self, "h", None):
            self.lib.hespmv_cssc_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CtBatch:
    """Device ciphertexts [n][2][L][N] (hespmv_ctbatch)."""

    def __init__(self, ctx, h):
        self.ctx = ctx
        self.h = h if isinstance(h, c_void_p) else c_void_p(h)
        p = B.u64p()
        n = c_size_t()
        ctx.check(ctx.lib.hespmv_ctbatch_data(self.h, byref(p), byref(n)))
        self.ptr = ctypes.cast(p, c_void_p).value
        self.n = n.value

    @classmethod
    def create(cls, ctx, n):
        h = c_void_p()
        ctx.check(ctx.lib.hespmv_ctbatch_create(ctx.h, n, byref(h)))
        return cls(ctx, h)

    @property
    def words_per_ct(self):
        return 2 * self.ctx.L * self.ctx.N

    def download(self, stream=None):
        out = np.zeros(self.n * self.words_per_ct, dtype=np.uint64)
        self.ctx.check(self.ctx.lib.hespmv_ctbatch_download(self.h, _u64p(out), self.n,
                                                            _stream_handle(stream)))
        return out.reshape(self.n, 2, self.ctx.L, self.ctx.N)

    def serialize(self):
        """Bytes of hespmv_ctbatch_serialize."""
        n = c_size_t()
        self.ctx.check(self.ctx.lib.hespmv_ctbatch_serialize(self.h, None, 0, byref(n)))
        buf = ctypes.create_string_buffer(max(1, n.value))
        self.ctx.check(self.ctx.lib.hespmv_ctbatch_serialize(self.h, buf, n.value, byref(n)))
        return buf.raw[:n.value]

    def upload(self, host, stream=None):
        a = np.ascontiguousarray(host, dtype=np.uint64)
        n = a.size // self.words_per_ct
        self.ctx.check(self.ctx.lib.hespmv_ctbatch_upload(self.h, _u64p(a), n, _stream_handle(stream)))

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.ctx.lib.hespmv_ctbatch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def galois_key_count(N, steps, policy):
    """Galois keys a set of rotation steps needs: one per power of two
    present in any step (power-of-two chains), or one per distinct step."""
    half = N // 2
    ks = {s % half for s in steps} - {0}
    if policy == "exact":
        return len(ks)
    return len({b for s in ks for b in range(s.bit_length()) if (s >> b) & 1})


def tune_keyswitch(ring, insts, dnums=None, policies=("pow2", "exact"), reps=3, seed=1, device=0,
                   schedule=True):
    """Key-switch decomposition (dnum digits of alpha = ceil(L / dnum) primes)
    and rotation-key policy for a workload of SpMVs, chosen by measurement.

    Both are the key holder's choices: each candidate gets its own keys and
    ciphertexts (which differ between candidates; their decryptions do not).
    For every candidate this creates a context, generates the keys the
    workload's rotations need, encrypts the instances, applies the schedule
    autotuner (`schedule`), times the batched evaluation (`reps` runs after a
    warm-up, CUDA events) and checks that every result decrypts to A.x.
    Candidates whose alpha exceeds K (the special primes must cover a digit
    to keep the key-switching noise small) are skipped.  Returns the
    candidates, fastest first: dnum, alpha, policy, Galois keys, key bytes on
    the device, ms per batch, SpMV/s, correct."""
    import torch
    logn, L, K, dnum0, t = ring
    N = 1 << logn
    if dnums is None:
        dnums = sorted({d for d in range(1, L + 1) if -(-L // d) <= K and -(-L // -(-L // d)) == d} | {dnum0})
    out = []
    for d in dnums:
        alpha = -(-L // d)
        if alpha > K:
            continue
        for pol in policies:
            ctx = Context(logn, L, K, d, t, rot_policy=pol, device=device)
            ms_ = [ctx.encode_cssc(A.rows, A.cols, A.rowptr, A.colidx, A.vals) for A, _ in insts]
            steps = sorted({s for m in ms_ for s in m.rotation_steps()})
            ctx.keygen(seed, steps)
            As = [ctx.encrypt(m, B.HESPMV_MATRIX, seed=seed + 1 + i) for i, m in enumerate(ms_)]
            Xs = [ctx.encrypt(m, B.HESPMV_VECTOR, x=x, seed=seed + 1001 + i)
                  for i, (m, (_, x)) in enumerate(zip(ms_, insts))]
            if schedule:
                ctx.autotune(ms_, As, Xs, reps=2)
            stream = torch.cuda.current_stream()
            ys = ctx.spmv_batched(ms_, As, Xs, stream=stream)
            torch.cuda.synchronize()
            ok = all(list(ctx.decrypt(m, y)) == list(A.matvec(x)) for m, y, (A, x) in zip(ms_, ys, insts))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                ctx.spmv_batched(ms_, As, Xs, ys, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_batch = e0.elapsed_time(e1) / reps
            n_gk = galois_key_count(N, steps, pol)
            key_bytes = (1 + n_gk) * d * 2 * (L + K) * N * 8
            out.append({"dnum": d, "alpha": alpha, "policy": pol, "galois_keys": n_gk,
                        "key_bytes": key_bytes, "ms": ms_batch, "spmv_per_s": len(insts) * 1e3 / ms_batch,
                        "keyswitches": sum(m.n_chunks + m.n_keyswitch for m in ms_),
                        "schedule": ctx.get_tuning(), "correct": bool(ok)})
            del ctx, As, Xs, ys
    out.sort(key=lambda r: r["ms"])
    return out
