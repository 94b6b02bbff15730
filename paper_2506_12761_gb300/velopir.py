"""Thin ctypes binding of libvelopir.so (include/velopir.h) and of the
host-only client library libvelopir_client.so (include/velopir_client.h),
same names.

Argument marshalling only: every step of gate bootstrapping and of the mode
circuits runs in the library's CUDA kernels.  Buffers may be numpy arrays
(host memory) or torch tensors (host or CUDA memory); torch is used only
for device memory and streams.  There is no CPU fallback: if the compiled
library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libvelopir.so")
CLIENT_LIB = os.path.join(HERE, "libvelopir_client.so")

VELOPIR_OK = 0
ERRORS = {-1: "ERR_ARG", -2: "ERR_NOKEY", -3: "ERR_OOM", -4: "ERR_CUDA", -5: "ERR_TIMEOUT", -6: "ERR_BUSY",
          -7: "ERR_NOCUDA", -8: "ERR_PLAN", -9: "ERR_CANCELLED"}
ERRORS_BY_NAME = {v: k for k, v in ERRORS.items()}
(VP_AND, VP_NAND, VP_OR, VP_NOR, VP_XOR, VP_XNOR, VP_ANDNY, VP_ANDYN, VP_ORNY, VP_ORYN, VP_MUX) = range(11)
VP_PATH_INT32_DENSE, VP_PATH_NTT, VP_PATH_TENSOR_F16 = 0, 1, 2
VP_QUERY_INTV, VP_QUERY_COV, VP_QUERY_IDM = 0, 1, 2
VP_PLAN_INTV_ENCDB, VP_PLAN_COV_ENCDB, VP_PLAN_IDM_ENCDB = 3, 4, 5   # velopir_plan_query only
LWE_WORDS = 631
BK_WORDS = 630 * 6 * 2 * 1024
KSK_WORDS = 1024 * 8 * 4 * 631

# Every symbol include/velopir.h declares (the GPU library).
EXPORTS = [
    "velopir_create", "velopir_destroy", "velopir_load_cloud_key", "velopir_set_path",
    "velopir_bootstrap_batch", "velopir_bootstrap_plain", "velopir_interval_query",
    "velopir_coordinate_query", "velopir_id_match", "velopir_submit", "velopir_poll",
    "velopir_queue_depth", "velopir_sync", "velopir_last_error", "velopir_launch_count",
    "velopir_profile", "velopir_profile_read", "velopir_query_batch", "velopir_graph_replays",
    "velopir_bootstrap_batch_noalloc", "velopir_autotune", "velopir_tuned_shape", "velopir_progress",
    "velopir_selftest_wait_timeout", "velopir_plan_query",
    "velopir_interval_query_encdb", "velopir_coordinate_query_encdb", "velopir_id_match_encdb", "velopir_cancel",
    "velopir_plan_batch", "velopir_trace_start", "velopir_trace_stop", "velopir_set_launch_limit",
    "velopir_serve_start", "velopir_serve_stop", "velopir_set_encdb_fanin",
    "velopir_gpu_keygen", "velopir_gpu_encrypt_bits", "velopir_gpu_pubkeygen", "velopir_gpu_server_encrypt",
]
# Every symbol include/velopir_client.h declares (the host-only client library).
CLIENT_EXPORTS = [
    "velopir_client_keygen", "velopir_client_encrypt_bits", "velopir_client_decrypt_bits",
    "velopir_client_pubkeygen", "velopir_server_encrypt",
]
NOALLOC_MAX_GATES = 256
NTT_TILE_SHAPES = (6, 8, 9, 10, 12)
VP_KERNEL_BLIND_ROTATE, VP_KERNEL_KEY_SWITCH, VP_KERNEL_FREE, VP_KERNEL_SUM, VP_KERNEL_TRACE = 0, 1, 2, 3, 4
MAX_FANIN = 8
TRACE_MAX_IN = 8
# velopir_trace_rec
TRACE_DTYPE = np.dtype([("nrot", "<u4"), ("nin", "<u4"), ("ks_cst", "<u4"), ("cst", "<u4", (2,)),
                        ("coef", "<i4", (2, TRACE_MAX_IN)), ("inp", "<u4", (TRACE_MAX_IN, LWE_WORDS)),
                        ("out", "<u4", (LWE_WORDS,))])
assert TRACE_DTYPE.itemsize == 22800


class VelopirError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in ("n", "N", "k", "l", "bg_bits", "ks_t", "ks_base_bits")]


def paper_params() -> Params:
    return Params(630, 1024, 1, 3, 7, 8, 2)


class Query(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("id_bits", ctypes.c_int32), ("payload_bits", ctypes.c_int32),
                ("agg_fanin", ctypes.c_int32), ("enc_a", ctypes.c_void_p), ("enc_b", ctypes.c_void_p),
                ("db", ctypes.c_void_p), ("payload", ctypes.c_void_p), ("D", ctypes.c_size_t),
                ("out", ctypes.c_void_p)]


_lib = None
_clib = None


def clib() -> ctypes.CDLL:
    """The host-only client library (no CUDA runtime is loaded)."""
    global _clib
    if _clib is None:
        if not os.path.exists(CLIENT_LIB):
            raise ImportError(f"{CLIENT_LIB} is missing: build it with paper_2506_12761_gb300.build.build()")
        L = ctypes.CDLL(CLIENT_LIB)
        vp, sz, i = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
        sig = {
            "velopir_client_keygen": (i, [ctypes.POINTER(Params), vp, vp, vp, vp, vp, vp, vp, vp]),
            "velopir_client_encrypt_bits": (i, [vp, vp, vp, vp, sz, vp]),
            "velopir_client_decrypt_bits": (i, [vp, vp, sz, vp]),
            "velopir_client_pubkeygen": (i, [vp, vp, vp, sz, vp]),
            "velopir_server_encrypt": (i, [vp, vp, sz, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _clib = L
    return _clib


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError(f"{LIB} is missing: build it with paper_2506_12761_gb300.build.build()")
        L = ctypes.CDLL(LIB)
        vp, sz, i, u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint64
        sig = {
            "velopir_create": (i, [ctypes.POINTER(vp), i, sz, vp]),
            "velopir_destroy": (i, [vp]),
            "velopir_load_cloud_key": (i, [vp, ctypes.POINTER(Params), vp, sz, vp, sz]),
            "velopir_set_path": (i, [vp, i]),
            "velopir_set_launch_limit": (i, [vp, sz]),
            "velopir_set_encdb_fanin": (i, [vp, i]),
            "velopir_serve_start": (i, [vp]),
            "velopir_serve_stop": (i, [vp]),
            "velopir_bootstrap_batch": (i, [vp, i, vp, vp, sz]),
            "velopir_bootstrap_plain": (i, [vp, i, vp, vp, sz]),
            "velopir_bootstrap_batch_noalloc": (i, [vp, i, vp, vp, sz]),
            "velopir_interval_query": (i, [vp, vp, vp, vp, sz, vp]),
            "velopir_coordinate_query": (i, [vp, vp, vp, sz, vp]),
            "velopir_id_match": (i, [vp, vp, i, vp, sz, vp, i, vp]),
            "velopir_submit": (i, [vp, ctypes.POINTER(Query), ctypes.POINTER(u64)]),
            "velopir_poll": (i, [vp, u64, ctypes.POINTER(i)]),
            "velopir_cancel": (i, [vp, u64]),
            "velopir_queue_depth": (i, [vp, ctypes.POINTER(sz), ctypes.POINTER(sz)]),
            "velopir_progress": (i, [vp, ctypes.POINTER(u64), sz, ctypes.POINTER(sz)]),
            "velopir_sync": (i, [vp]),
            "velopir_last_error": (ctypes.c_char_p, [vp]),
            "velopir_launch_count": (u64, [vp]),
            "velopir_selftest_wait_timeout": (i, [vp]),
            "velopir_profile": (i, [vp, i]),
            "velopir_query_batch": (i, [vp, ctypes.POINTER(Query), sz, i]),
            "velopir_graph_replays": (u64, [vp]),
            "velopir_autotune": (i, [vp, ctypes.POINTER(ctypes.c_double), i]),
            "velopir_tuned_shape": (i, [vp, sz]),
            "velopir_plan_query": (i, [ctypes.POINTER(Query), i, vp, vp, vp, ctypes.POINTER(sz), i]),
            "velopir_plan_batch": (i, [ctypes.POINTER(Query), sz, i, i, vp, vp, vp, ctypes.POINTER(sz), i]),
            "velopir_interval_query_encdb": (i, [vp, vp, vp, i, vp, sz, vp, i, vp]),
            "velopir_coordinate_query_encdb": (i, [vp, vp, i, vp, sz, vp, i, vp]),
            "velopir_id_match_encdb": (i, [vp, vp, i, vp, sz, vp, i, vp]),
            "velopir_profile_read": (i, [vp, i, ctypes.POINTER(u64), ctypes.POINTER(u64),
                                         ctypes.POINTER(ctypes.c_double)]),
            "velopir_trace_start": (i, [vp, u64, ctypes.c_uint32, ctypes.c_uint32, sz]),
            "velopir_trace_stop": (i, [vp, vp, sz, ctypes.POINTER(sz)]),
            "velopir_gpu_keygen": (i, [vp, ctypes.POINTER(Params), vp, vp, vp, vp, vp, vp, vp, vp]),
            "velopir_gpu_encrypt_bits": (i, [vp, vp, vp, vp, vp, sz, vp]),
            "velopir_gpu_pubkeygen": (i, [vp, vp, vp, vp, sz, vp]),
            "velopir_gpu_server_encrypt": (i, [vp, vp, vp, sz, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def ptr(buf) -> int | None:
    """Address of a numpy array or torch tensor (contiguous uint32 / int32 data)."""
    if buf is None:
        return None
    if isinstance(buf, np.ndarray):
        assert buf.flags["C_CONTIGUOUS"] and buf.dtype.itemsize == 4, "need a contiguous 32-bit array"
        return buf.ctypes.data
    assert buf.is_contiguous() and buf.element_size() == 4, "need a contiguous 32-bit tensor"
    return buf.data_ptr()


def _check(ctx, rc: int):
    if rc != VELOPIR_OK:
        msg = lib().velopir_last_error(ctx)
        raise VelopirError(rc, msg.decode() if msg else "")


def _check_client(rc: int):
    if rc != VELOPIR_OK:
        raise VelopirError(rc, "invalid argument to the client library")


# ---- the C ABI, one function each -----------------------------------------

def velopir_create(device: int = 0, hbm_budget_bytes: int = 0, cuda_stream: int | None = None):
    h = ctypes.c_void_p()
    rc = lib().velopir_create(ctypes.byref(h), device, hbm_budget_bytes, cuda_stream)
    _check(None, rc)
    return h.value


def velopir_destroy(ctx) -> None:
    _check(ctx, lib().velopir_destroy(ctx))


def velopir_load_cloud_key(ctx, bk, ksk, params: Params | None = None) -> None:
    p = params or paper_params()
    _check(ctx, lib().velopir_load_cloud_key(ctx, ctypes.byref(p), ptr(bk), BK_WORDS, ptr(ksk), KSK_WORDS))


def velopir_set_path(ctx, path: int) -> None:
    _check(ctx, lib().velopir_set_path(ctx, path))


def velopir_set_launch_limit(ctx, max_rotations: int) -> None:
    """Blind rotations per launch at most (1: one bootstrap per launch; 0: default)."""
    _check(ctx, lib().velopir_set_launch_limit(ctx, max_rotations))


def velopir_set_encdb_fanin(ctx, fanin: int) -> None:
    """Fan-in of the *_encdb calls' XOR aggregation tree (2: pairwise HomSum; 0: default)."""
    _check(ctx, lib().velopir_set_encdb_fanin(ctx, fanin))


def velopir_bootstrap_batch(ctx, gate: int, lwe_in, lwe_out, count: int) -> None:
    _check(ctx, lib().velopir_bootstrap_batch(ctx, gate, ptr(lwe_in), ptr(lwe_out), count))


def velopir_bootstrap_batch_noalloc(ctx, gate: int, lwe_in, lwe_out, count: int) -> None:
    """Allocation-free variant of velopir_bootstrap_batch (device buffers, count <= NOALLOC_MAX_GATES)."""
    _check(ctx, lib().velopir_bootstrap_batch_noalloc(ctx, gate, ptr(lwe_in), ptr(lwe_out), count))


def velopir_bootstrap_plain(ctx, gate: int, lwe_in, lwe_out, count: int) -> None:
    _check(ctx, lib().velopir_bootstrap_plain(ctx, gate, ptr(lwe_in), ptr(lwe_out), count))


def velopir_interval_query(ctx, enc_x, enc_y, rects, D: int, out_bits) -> None:
    _check(ctx, lib().velopir_interval_query(ctx, ptr(enc_x), ptr(enc_y), ptr(rects), D, ptr(out_bits)))


def velopir_coordinate_query(ctx, enc_cell, cells, D: int, out_bits) -> None:
    _check(ctx, lib().velopir_coordinate_query(ctx, ptr(enc_cell), ptr(cells), D, ptr(out_bits)))


def velopir_id_match(ctx, enc_id, id_bits: int, ids, D: int, payload, payload_bits: int, out) -> None:
    _check(ctx, lib().velopir_id_match(ctx, ptr(enc_id), id_bits, ptr(ids), D, ptr(payload), payload_bits, ptr(out)))


def velopir_query_batch(ctx, queries, use_graph: bool = False) -> None:
    arr = (Query * len(queries))(*queries)
    _check(ctx, lib().velopir_query_batch(ctx, arr, len(queries), int(use_graph)))


def velopir_graph_replays(ctx) -> int:
    return int(lib().velopir_graph_replays(ctx))


def velopir_autotune(ctx) -> list[float]:
    """Measured full-wave times (ms) of the blind-rotation tile shapes (6, 8, 9, 10, 12 bootstraps per CTA)."""
    out = (ctypes.c_double * 8)()
    _check(ctx, lib().velopir_autotune(ctx, out, 8))
    return [x for x in out if x > 0]


def velopir_tuned_shape(ctx, count: int) -> int:
    rc = lib().velopir_tuned_shape(ctx, count)
    if rc < 0:
        _check(ctx, rc)
    return rc


def make_query(kind: int, enc_a, db, D: int, out, enc_b=None, id_bits: int = 0, payload=None,
               payload_bits: int = 0, agg_fanin: int = 0) -> Query:
    """A velopir_query record; the caller keeps every buffer alive until the query finishes."""
    return Query(kind, id_bits, payload_bits if payload is not None else 0, agg_fanin, ptr(enc_a), ptr(enc_b),
                 ptr(db), ptr(payload), D, ptr(out))


def velopir_submit(ctx, query: Query) -> int:
    t = ctypes.c_uint64()
    _check(ctx, lib().velopir_submit(ctx, ctypes.byref(query), ctypes.byref(t)))
    return t.value


def velopir_poll(ctx, ticket: int) -> bool:
    d = ctypes.c_int()
    _check(ctx, lib().velopir_poll(ctx, ticket, ctypes.byref(d)))
    return bool(d.value)


def velopir_cancel(ctx, ticket: int) -> None:
    _check(ctx, lib().velopir_cancel(ctx, ticket))


def velopir_progress(ctx, cap: int = 256) -> list[int]:
    """One serving step; the tickets that finished since the last report."""
    buf = (ctypes.c_uint64 * cap)()
    n = ctypes.c_size_t()
    _check(ctx, lib().velopir_progress(ctx, buf, cap, ctypes.byref(n)))
    return [int(buf[i]) for i in range(n.value)]


def velopir_serve_start(ctx) -> None:
    """Start the library's issue thread (serving steps back to back)."""
    _check(ctx, lib().velopir_serve_start(ctx))


def velopir_serve_stop(ctx) -> None:
    _check(ctx, lib().velopir_serve_stop(ctx))


def velopir_queue_depth(ctx) -> tuple[int, int]:
    a, w = ctypes.c_size_t(), ctypes.c_size_t()
    _check(ctx, lib().velopir_queue_depth(ctx, ctypes.byref(a), ctypes.byref(w)))
    return a.value, w.value


def velopir_sync(ctx) -> None:
    _check(ctx, lib().velopir_sync(ctx))


def velopir_last_error(ctx) -> str:
    m = lib().velopir_last_error(ctx)
    return m.decode() if m else ""


def velopir_launch_count(ctx) -> int:
    return int(lib().velopir_launch_count(ctx))


def velopir_selftest_wait_timeout(ctx) -> int:
    """Raw status of the bounded-wait self-test (VELOPIR_ERR_TIMEOUT = -5 is the expected result)."""
    return int(lib().velopir_selftest_wait_timeout(ctx))


def velopir_profile(ctx, enable: bool) -> None:
    _check(ctx, lib().velopir_profile(ctx, int(enable)))


def velopir_profile_read(ctx, kernel: int) -> tuple[int, int, float]:
    """(launches, units, device ms) accumulated for one kernel kind."""
    n, u, ms = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_double()
    _check(ctx, lib().velopir_profile_read(ctx, kernel, ctypes.byref(n), ctypes.byref(u), ctypes.byref(ms)))
    return n.value, u.value, ms.value


def velopir_trace_start(ctx, seed: int, per_launch: int, one_in: int, cap: int) -> None:
    """Record max(min(per_launch, G), ceil(G / one_in)) sampled gates of every launch of G, at most cap in all."""
    _check(ctx, lib().velopir_trace_start(ctx, seed, per_launch, one_in, cap))


def velopir_trace_stop(ctx, cap: int) -> np.ndarray:
    """Stop tracing; the first min(cap, recorded) records as a TRACE_DTYPE array."""
    n = ctypes.c_size_t()
    out = np.zeros(max(1, cap), dtype=TRACE_DTYPE)
    _check(ctx, lib().velopir_trace_stop(ctx, out.ctypes.data if cap else None, cap, ctypes.byref(n)))
    return out[: min(cap, n.value)]


def velopir_client_keygen(km, params: Params | None = None):
    """Cloud key (bk, ksk) as numpy arrays from synth.KeyMaterial."""
    p = params or paper_params()
    c = {k: np.ascontiguousarray(getattr(km, k), dtype=np.uint32) for k in ("s", "K", "bk_a", "bk_e", "ksk_a", "ksk_e")}
    bk = np.empty(BK_WORDS, dtype=np.uint32)
    ksk = np.empty(KSK_WORDS, dtype=np.uint32)
    rc = clib().velopir_client_keygen(ctypes.byref(p), ptr(c["s"]), ptr(c["K"]), ptr(c["bk_a"]), ptr(c["bk_e"]),
                                     ptr(c["ksk_a"]), ptr(c["ksk_e"]), ptr(bk), ptr(ksk))
    _check_client(rc)
    return bk, ksk


def velopir_client_encrypt_bits(s, bits, lwe_mat) -> np.ndarray:
    bits = np.ascontiguousarray(np.asarray(bits, dtype=np.uint32).reshape(-1))
    n = len(bits)
    a = np.ascontiguousarray(lwe_mat.a[:n], dtype=np.uint32)
    e = np.ascontiguousarray(lwe_mat.e[:n], dtype=np.uint32)
    out = np.empty((n, LWE_WORDS), dtype=np.uint32)
    _check_client(clib().velopir_client_encrypt_bits(ptr(np.ascontiguousarray(s, dtype=np.uint32)), ptr(bits),
                                                   ptr(a), ptr(e), n, ptr(out)))
    return out


def velopir_client_decrypt_bits(s, ct) -> np.ndarray:
    ct = np.ascontiguousarray(np.asarray(ct, dtype=np.uint32).reshape(-1, LWE_WORDS))
    out = np.empty(ct.shape[0], dtype=np.uint32)
    _check_client(clib().velopir_client_decrypt_bits(ptr(np.ascontiguousarray(s, dtype=np.uint32)), ptr(ct),
                                                   ct.shape[0], ptr(out)))
    return out


def _u32c(x):
    """numpy arrays as contiguous uint32; torch tensors pass through (they must be contiguous 32-bit)."""
    return np.ascontiguousarray(x, dtype=np.uint32) if isinstance(x, np.ndarray) else x


def velopir_gpu_keygen(ctx, km, bk_out, ksk_out, params: Params | None = None) -> None:
    """Cloud key on the GPU from synth.KeyMaterial-like fields (numpy arrays or
    torch tensors, host or device) into bk_out / ksk_out (host or device)."""
    p = params or paper_params()
    c = {k: _u32c(getattr(km, k)) for k in ("s", "K", "bk_a", "bk_e", "ksk_a", "ksk_e")}
    _check(ctx, lib().velopir_gpu_keygen(ctx, ctypes.byref(p), ptr(c["s"]), ptr(c["K"]), ptr(c["bk_a"]),
                                         ptr(c["bk_e"]), ptr(c["ksk_a"]), ptr(c["ksk_e"]), ptr(bk_out), ptr(ksk_out)))


def velopir_gpu_encrypt_bits(ctx, s, bits, a, e, out) -> None:
    """Section 2.2 Enc of len(bits) bits on the GPU into out[count][631] (host or device buffers)."""
    bits, a, e, s = _u32c(bits), _u32c(a), _u32c(e), _u32c(s)
    count = int(np.prod(bits.shape))
    _check(ctx, lib().velopir_gpu_encrypt_bits(ctx, ptr(s), ptr(bits), ptr(a), ptr(e), count, ptr(out)))


def velopir_gpu_pubkeygen(ctx, s, a, e, out) -> None:
    """Alg. PubKeyGen on the GPU: encryptions of zero, one per noise word of e."""
    a, e, s = _u32c(a), _u32c(e), _u32c(s)
    count = int(np.prod(e.shape))
    _check(ctx, lib().velopir_gpu_pubkeygen(ctx, ptr(s), ptr(a), ptr(e), count, ptr(out)))


def velopir_gpu_server_encrypt(ctx, pk, bits, out) -> None:
    """Alg. ServerEnc on the GPU: (0, Ecd(bit)) + pk, one ciphertext per bit."""
    pk, bits = _u32c(pk), _u32c(bits)
    count = int(np.prod(bits.shape))
    _check(ctx, lib().velopir_gpu_server_encrypt(ctx, ptr(pk), ptr(bits), count, ptr(out)))


class Context:
    """Owning wrapper: one velopir_ctx on one device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, cuda_stream: int | None = None):
        self.h = velopir_create(device, hbm_budget_bytes, cuda_stream)

    def close(self):
        if self.h:
            velopir_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def velopir_plan_query(kind: int, db, D: int, bits_a, bits_b=None, wave: int = 0, id_bits: int = 0,
                       payload=None, payload_bits: int = 0, max_launches: int = 4096, agg_fanin: int = 0):
    """Host-only dry run of a query's launch plan on plaintext bits.  For the
    VP_PLAN_*_ENCDB kinds id_bits is the width (l, w or id_bits) and db /
    payload are plaintext values the dry run encrypts.

    Returns (result bits, blind rotations per launch).  Raises VelopirError
    (ERR_PLAN) if the plan reads a value before it is written or after its
    pool slot was reused."""
    db = np.ascontiguousarray(db, dtype=np.uint32)
    a = np.ascontiguousarray(bits_a, dtype=np.uint32)
    b = None if bits_b is None else np.ascontiguousarray(bits_b, dtype=np.uint32)
    pay = None if payload is None else np.ascontiguousarray(payload, dtype=np.uint32)
    q = Query(kind, id_bits, payload_bits, agg_fanin, None, None, ptr(db), ptr(pay), D, None)
    nout = payload_bits if payload is not None else D
    out = np.zeros(max(1, nout), dtype=np.uint32)
    sizes = (ctypes.c_size_t * max_launches)()
    rc = lib().velopir_plan_query(ctypes.byref(q), wave, ptr(a), ptr(b), ptr(out), sizes, max_launches)
    if rc < 0:
        raise VelopirError(rc, "velopir_plan_query")
    return out[:nout], [int(sizes[k]) for k in range(min(rc, max_launches))]


def velopir_client_pubkeygen(s, lwe_mat_zero) -> np.ndarray:
    """Alg. PubKeyGen: encryptions of zero from (a, e) material (synth.lwe_material)."""
    s = np.ascontiguousarray(s, dtype=np.uint32)
    a = np.ascontiguousarray(lwe_mat_zero.a, dtype=np.uint32)
    e = np.ascontiguousarray(lwe_mat_zero.e, dtype=np.uint32)
    count = e.shape[0]
    out = np.zeros((count, LWE_WORDS), dtype=np.uint32)
    _check_client(clib().velopir_client_pubkeygen(ptr(s), ptr(a), ptr(e), count, ptr(out)))
    return out


def velopir_server_encrypt(pk, bits) -> np.ndarray:
    """Alg. ServerEnc: (0, Ecd(bit)) + pk, one ciphertext per bit (any leading shape)."""
    pk = np.ascontiguousarray(pk, dtype=np.uint32).reshape(-1, LWE_WORDS)
    b = np.ascontiguousarray(bits, dtype=np.uint32).reshape(-1)
    assert pk.shape[0] == b.shape[0]
    out = np.zeros_like(pk)
    _check_client(clib().velopir_server_encrypt(ptr(pk), ptr(b), b.shape[0], ptr(out)))
    return out.reshape(np.shape(bits) + (LWE_WORDS,))


def velopir_interval_query_encdb(ctx, enc_x, enc_y, l: int, enc_rects, D: int, enc_payload, payload_bits: int,
                                 out) -> None:
    _check(ctx, lib().velopir_interval_query_encdb(ctx, ptr(enc_x), ptr(enc_y), l, ptr(enc_rects), D,
                                                   ptr(enc_payload), payload_bits, ptr(out)))


def velopir_coordinate_query_encdb(ctx, enc_cell, w: int, enc_cells, D: int, enc_payload, payload_bits: int,
                                   out) -> None:
    _check(ctx, lib().velopir_coordinate_query_encdb(ctx, ptr(enc_cell), w, ptr(enc_cells), D, ptr(enc_payload),
                                                     payload_bits, ptr(out)))


def velopir_id_match_encdb(ctx, enc_id, id_bits: int, enc_ids, D: int, enc_payload, payload_bits: int, out) -> None:
    _check(ctx, lib().velopir_id_match_encdb(ctx, ptr(enc_id), id_bits, ptr(enc_ids), D, ptr(enc_payload),
                                             payload_bits, ptr(out)))


def velopir_plan_batch(queries, wave: int = 0, chunk_rows: int = 0, max_launches: int = 4096):
    """Host-only dry run of a query batch (velopir_query_batch's program) on
    plaintext bits.  queries: dicts with kind, db, D, bits_a, optional bits_b
    (IntV), id_bits, payload, payload_bits.  Returns (per-query result bits,
    blind rotations per launch)."""
    keep, recs, a, b, nout = [], [], [], [], []
    for q in queries:
        db = np.ascontiguousarray(q["db"], dtype=np.uint32)
        pay = None if q.get("payload") is None else np.ascontiguousarray(q["payload"], dtype=np.uint32)
        keep += [db, pay]
        recs.append(Query(q["kind"], q.get("id_bits", 0), q.get("payload_bits", 0) if pay is not None else 0,
                          q.get("agg_fanin", 0), None, None, ptr(db), ptr(pay), q["D"], None))
        a.append(np.asarray(q["bits_a"], dtype=np.uint32))
        if q["kind"] == VP_QUERY_INTV:
            b.append(np.asarray(q["bits_b"], dtype=np.uint32))
        nout.append(q["payload_bits"] if pay is not None else q["D"])
    A = np.ascontiguousarray(np.concatenate(a))
    Bb = np.ascontiguousarray(np.concatenate(b)) if b else None
    out = np.zeros(max(1, sum(nout)), dtype=np.uint32)
    sizes = (ctypes.c_size_t * max_launches)()
    arr = (Query * len(recs))(*recs)
    rc = lib().velopir_plan_batch(arr, len(recs), wave, chunk_rows, ptr(A), ptr(Bb), ptr(out), sizes, max_launches)
    if rc < 0:
        raise VelopirError(rc, "velopir_plan_batch")
    splits = np.cumsum([0] + nout)
    return [out[splits[k]:splits[k + 1]] for k in range(len(nout))], [int(sizes[k]) for k in range(min(rc, max_launches))]
