"""Thin ctypes binding of libpt2 (include/pt2.h): same names, argument
marshalling only.  Every step of the PT2 path runs in the CUDA library; this
module converts numpy arrays to pointers and status codes to exceptions.

The library is built in-tree (paper_1808_02049_gb300/_build/libpt2.so) by
``paper_1808_02049_gb300.build``; loading fails loudly when it is missing.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpt2.so")

PT2_OK = 0
PT2_ERR_INVALID = -1
PT2_ERR_OOM = -2
PT2_ERR_CUDA = -3
PT2_ERR_TIMEOUT = -4
PT2_ERR_BUSY = -5
PT2_ERR_NOT_FOUND = -6
PT2_ERR_UNSUPPORTED = -7
PT2_FLAG_PROFILE = 1
PT2_FLAG_AUTOTUNE = 2
PT2_FLAG_SPIN_SYMMETRIC = 4
PT2_FLAG_SUBTRACT_REF = 8
PT2_FLAG_HASHED_KEYS = 16
PT2_DEBUG_NARROW_SORT_HASH = 1
PT2_DEBUG_SHORT_COPY_WAIT = 2

EXPORTS = ["pt2_create", "pt2_destroy", "pt2_last_error", "pt2_load_system", "pt2_load_reference",
           "pt2_unload", "pt2_diagonal", "pt2_run", "pt2_dump_external", "pt2_batch_create", "pt2_batch_run",
           "pt2_batch_info", "pt2_batch_destroy", "pt2_autotune", "pt2_submit", "pt2_poll", "pt2_wait",
           "pt2_server_stats", "pt2_det_terms", "pt2_det_terms_noalloc", "pt2_eval_terms", "pt2_phase_times",
           "pt2_memory_info", "pt2_stream"]

PHASES = ["class_count", "tile_count", "scan", "emit", "ref_partition", "tile_sort_reduce",
          "oversize_tiles", "pass_reduce"]


class Pt2Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libpt2 error {code}: {msg}")
        self.code = code


class pt2_opts(ctypes.Structure):
    _fields_ = [("constraint_mod", ctypes.c_uint64), ("constraint_rem", ctypes.c_uint64),
                ("pass_budget_bytes", ctypes.c_uint64), ("tile_target", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("numerator_cutoff", ctypes.c_double),
                ("debug_flags", ctypes.c_uint32), ("class_slices", ctypes.c_uint32),
                ("class_slice", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("top_alpha", ctypes.c_uint64)]


class pt2_result(ctypes.Structure):
    _fields_ = [("e2", ctypes.c_double), ("n_terms", ctypes.c_uint64), ("n_unique", ctypes.c_uint64),
                ("n_in_ref", ctypes.c_uint64), ("n_external", ctypes.c_uint64),
                ("digest_sum", ctypes.c_uint64), ("digest_xor", ctypes.c_uint64),
                ("min_abs_denom", ctypes.c_double), ("n_pos_denom", ctypes.c_uint64),
                ("n_passes", ctypes.c_uint32), ("n_tiles", ctypes.c_uint32),
                ("n_oversize", ctypes.c_uint32), ("n_hash_collisions", ctypes.c_uint32),
                ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libpt2.so and declare the C signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libpt2.so not found at {path}: run paper_1808_02049_gb300.build.build_library()")
    lib = ctypes.CDLL(path)
    P, u32, u64, i32, dbl = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
    pu32, pu64 = ctypes.POINTER(u32), ctypes.POINTER(u64)
    sig = {
        "pt2_create": (i32, [ctypes.POINTER(P), i32, u64]),
        "pt2_destroy": (None, [P]),
        "pt2_last_error": (ctypes.c_char_p, [P]),
        "pt2_load_system": (i32, [P, i32, P, P, pu32]),
        "pt2_load_reference": (i32, [P, u32, u64, P, P, dbl, pu32]),
        "pt2_unload": (i32, [P, u32]),
        "pt2_diagonal": (i32, [P, u32, u64, P, P]),
        "pt2_run": (i32, [P, u32, ctypes.POINTER(pt2_opts), ctypes.POINTER(pt2_result)]),
        "pt2_dump_external": (i32, [P, u32, ctypes.POINTER(pt2_opts), P, P, P, u64, pu64]),
        "pt2_det_terms": (i32, [P, u32, u64, P, P, P, u64, pu64]),
        "pt2_batch_create": (i32, [P, u32, P, ctypes.POINTER(pt2_opts), pu32]),
        "pt2_batch_run": (i32, [P, u32, ctypes.POINTER(pt2_result)]),
        "pt2_batch_info": (i32, [P, u32, pu32, pu64, pu64]),
        "pt2_batch_destroy": (i32, [P, u32]),
        "pt2_autotune": (i32, [P, u32, ctypes.POINTER(pt2_opts), pu32]),
        "pt2_submit": (i32, [P, u32, ctypes.POINTER(pt2_opts), pu64]),
        "pt2_poll": (i32, [P, u64, ctypes.POINTER(pt2_result)]),
        "pt2_wait": (i32, [P, u64, u64, ctypes.POINTER(pt2_result)]),
        "pt2_server_stats": (i32, [P, pu64, pu64, pu64]),
        "pt2_det_terms_noalloc": (i32, [P, u32, u64, P, P, P, u64, pu64]),
        "pt2_eval_terms": (i32, [P, u64, P, P, P]),
        "pt2_phase_times": (i32, [P, P, i32, pu64]),
        "pt2_memory_info": (i32, [P, pu64, pu64, pu64]),
        "pt2_stream": (P, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(ctx, rc):
    if rc != PT2_OK:
        msg = load_library().pt2_last_error(ctx)
        raise Pt2Error(rc, msg.decode() if msg else "")
    return rc


def make_opts(constraint=(1, 0), pass_budget_bytes=0, tile_target=0, profile=False, autotune=False,
              spin_symmetric=False, cutoff=0.0, subtract_ref=False, narrow_sort_hash=False,
              short_copy_wait=False, class_slice=(0, 1), top_alpha=0, hashed_keys=False) -> pt2_opts:
    o = pt2_opts()
    o.constraint_mod, o.constraint_rem = int(constraint[0]), int(constraint[1])
    o.pass_budget_bytes = int(pass_budget_bytes)
    o.tile_target = int(tile_target)
    o.flags = ((PT2_FLAG_PROFILE if profile else 0) | (PT2_FLAG_AUTOTUNE if autotune else 0) |
               (PT2_FLAG_SPIN_SYMMETRIC if spin_symmetric else 0) |
               (PT2_FLAG_SUBTRACT_REF if subtract_ref else 0) | (PT2_FLAG_HASHED_KEYS if hashed_keys else 0))
    o.numerator_cutoff = float(cutoff)
    o.debug_flags = ((PT2_DEBUG_NARROW_SORT_HASH if narrow_sort_hash else 0) |
                     (PT2_DEBUG_SHORT_COPY_WAIT if short_copy_wait else 0))
    o.class_slice, o.class_slices = int(class_slice[0]), int(class_slice[1])
    o.top_alpha = int(top_alpha)
    return o


def pt2_create(device: int = 0, hbm_budget_bytes: int = 0):
    lib = load_library()
    h = ctypes.c_void_p()
    rc = lib.pt2_create(ctypes.byref(h), int(device), int(hbm_budget_bytes))
    if rc != PT2_OK:
        raise Pt2Error(rc, lib.pt2_last_error(None).decode())
    return h


def pt2_destroy(ctx):
    load_library().pt2_destroy(ctx)


def pt2_last_error(ctx) -> str:
    m = load_library().pt2_last_error(ctx)
    return m.decode() if m else ""


def pt2_load_system(ctx, h: np.ndarray, eri: np.ndarray) -> int:
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    sid = ctypes.c_uint32()
    _check(ctx, load_library().pt2_load_system(ctx, h.shape[0], _ptr(h), _ptr(eri), ctypes.byref(sid)))
    return sid.value


def pt2_load_reference(ctx, system_id: int, keys: np.ndarray, coef: np.ndarray, e0: float) -> int:
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    if keys.shape[0] != 2 * coef.shape[0]:
        raise ValueError("keys must hold 2 words per determinant")
    rid = ctypes.c_uint32()
    _check(ctx, load_library().pt2_load_reference(ctx, int(system_id), coef.shape[0], _ptr(keys), _ptr(coef),
                                                  float(e0), ctypes.byref(rid)))
    return rid.value


def pt2_unload(ctx, obj_id: int):
    _check(ctx, load_library().pt2_unload(ctx, int(obj_id)))


def pt2_diagonal(ctx, system_id: int, keys: np.ndarray) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    n = keys.shape[0] // 2
    out = np.empty(n)
    _check(ctx, load_library().pt2_diagonal(ctx, int(system_id), n, _ptr(keys), _ptr(out)))
    return out


def pt2_run(ctx, ref_id: int, opts: pt2_opts | None = None) -> dict:
    res = pt2_result()
    _check(ctx, load_library().pt2_run(ctx, int(ref_id), ctypes.byref(opts) if opts else None,
                                       ctypes.byref(res)))
    return res.as_dict()


def pt2_dump_external(ctx, ref_id: int, cap: int, opts: pt2_opts | None = None):
    keys = np.zeros(2 * max(cap, 1), dtype=np.uint64)
    num = np.zeros(max(cap, 1))
    haa = np.zeros(max(cap, 1))
    n = ctypes.c_uint64()
    _check(ctx, load_library().pt2_dump_external(ctx, int(ref_id), ctypes.byref(opts) if opts else None,
                                                 _ptr(keys), _ptr(num), _ptr(haa), int(cap), ctypes.byref(n)))
    m = n.value
    return keys[: 2 * m].reshape(m, 2), num[:m], haa[:m]


def pt2_batch_create(ctx, ref_ids, opts: pt2_opts | None = None) -> int:
    ids = np.ascontiguousarray(ref_ids, dtype=np.uint32)
    bid = ctypes.c_uint32()
    _check(ctx, load_library().pt2_batch_create(ctx, ids.shape[0], _ptr(ids), ctypes.byref(opts) if opts else None,
                                                ctypes.byref(bid)))
    return bid.value


def pt2_batch_run(ctx, batch_id: int, n: int) -> list:
    res = (pt2_result * n)()
    _check(ctx, load_library().pt2_batch_run(ctx, int(batch_id), res))
    return [r.as_dict() for r in res]


def pt2_batch_info(ctx, batch_id: int) -> dict:
    st, te, la = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(ctx, load_library().pt2_batch_info(ctx, int(batch_id), ctypes.byref(st), ctypes.byref(te),
                                              ctypes.byref(la)))
    return {"steps": st.value, "n_terms": te.value, "launches": la.value}


def pt2_batch_destroy(ctx, batch_id: int):
    _check(ctx, load_library().pt2_batch_destroy(ctx, int(batch_id)))


def pt2_autotune(ctx, ref_id: int, opts: pt2_opts | None = None) -> int:
    best = ctypes.c_uint32()
    _check(ctx, load_library().pt2_autotune(ctx, int(ref_id), ctypes.byref(opts) if opts else None,
                                            ctypes.byref(best)))
    return best.value


def pt2_submit(ctx, ref_id: int, opts: pt2_opts | None = None) -> int:
    t = ctypes.c_uint64()
    _check(ctx, load_library().pt2_submit(ctx, int(ref_id), ctypes.byref(opts) if opts else None, ctypes.byref(t)))
    return t.value


def pt2_poll(ctx, ticket: int):
    """The result dict once the request finished, None while it runs."""
    res = pt2_result()
    rc = load_library().pt2_poll(ctx, int(ticket), ctypes.byref(res))
    if rc == PT2_ERR_BUSY:
        return None
    _check(ctx, rc)
    return res.as_dict()


def pt2_wait(ctx, ticket: int, timeout_s: float = 3600.0) -> dict:
    res = pt2_result()
    _check(ctx, load_library().pt2_wait(ctx, int(ticket), int(timeout_s * 1e9), ctypes.byref(res)))
    return res.as_dict()


def pt2_server_stats(ctx) -> dict:
    p, a, s_ = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(ctx, load_library().pt2_server_stats(ctx, ctypes.byref(p), ctypes.byref(a), ctypes.byref(s_)))
    return {"pending": p.value, "active": a.value, "steps": s_.value}


def pt2_det_terms(ctx, ref_id: int, det_index: int, cap: int):
    keys = np.zeros(2 * max(cap, 1), dtype=np.uint64)
    val = np.zeros(max(cap, 1))
    haa = np.zeros(max(cap, 1))
    n = ctypes.c_uint64()
    _check(ctx, load_library().pt2_det_terms(ctx, int(ref_id), int(det_index), _ptr(keys), _ptr(val), _ptr(haa),
                                             int(cap), ctypes.byref(n)))
    m = n.value
    return keys[: 2 * m].reshape(m, 2), val[:m], haa[:m]


def pt2_det_terms_noalloc(ctx, ref_id: int, det_index: int, keys_dev: int, val_dev: int, haa_dev: int,
                          cap: int) -> int:
    """Terms of one determinant into caller-owned DEVICE buffers (addresses as
    integers), without any device allocation; returns the number of terms."""
    n = ctypes.c_uint64()
    _check(ctx, load_library().pt2_det_terms_noalloc(ctx, int(ref_id), int(det_index), ctypes.c_void_p(keys_dev),
                                                     ctypes.c_void_p(val_dev), ctypes.c_void_p(haa_dev), int(cap),
                                                     ctypes.byref(n)))
    return n.value


def pt2_eval_terms(ctx, num: np.ndarray, denom: np.ndarray) -> np.ndarray:
    """num^2 / denom (denom = E0 - H_aa in Hartree) with the tile kernels' arithmetic."""
    num = np.ascontiguousarray(num, dtype=np.float64)
    denom = np.ascontiguousarray(denom, dtype=np.float64)
    if num.shape != denom.shape:
        raise ValueError("num and denom must have the same shape")
    out = np.zeros_like(num)
    _check(ctx, load_library().pt2_eval_terms(ctx, num.size, _ptr(num), _ptr(denom), _ptr(out)))
    return out


def pt2_phase_times(ctx):
    out = np.zeros(8)
    launches = ctypes.c_uint64()
    _check(ctx, load_library().pt2_phase_times(ctx, _ptr(out), 8, ctypes.byref(launches)))
    return dict(zip(PHASES, out.tolist())), launches.value


def pt2_memory_info(ctx) -> dict:
    b, u, f = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(ctx, load_library().pt2_memory_info(ctx, ctypes.byref(b), ctypes.byref(u), ctypes.byref(f)))
    return {"budget": b.value, "used": u.value, "device_free": f.value}


def pt2_stream(ctx) -> int:
    return load_library().pt2_stream(ctx) or 0


class Context:
    """Owns one pt2 context; the methods are the C calls above."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.handle = pt2_create(device, hbm_budget_bytes)

    def close(self):
        if self.handle:
            pt2_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_system(self, h, eri):
        return pt2_load_system(self.handle, h, eri)

    def load_reference(self, system_id, keys, coef, e0):
        return pt2_load_reference(self.handle, system_id, keys, coef, e0)

    def unload(self, obj_id):
        pt2_unload(self.handle, obj_id)

    def diagonal(self, system_id, keys):
        return pt2_diagonal(self.handle, system_id, keys)

    def run(self, ref_id, **kw):
        return pt2_run(self.handle, ref_id, make_opts(**kw) if kw else None)

    def dump_external(self, ref_id, cap, **kw):
        return pt2_dump_external(self.handle, ref_id, cap, make_opts(**kw) if kw else None)

    def det_terms(self, ref_id, det_index, cap):
        return pt2_det_terms(self.handle, ref_id, det_index, cap)

    def batch_create(self, ref_ids, **kw):
        return pt2_batch_create(self.handle, ref_ids, make_opts(**kw) if kw else None)

    def batch_run(self, batch_id, n):
        return pt2_batch_run(self.handle, batch_id, n)

    def batch_info(self, batch_id):
        return pt2_batch_info(self.handle, batch_id)

    def batch_destroy(self, batch_id):
        pt2_batch_destroy(self.handle, batch_id)

    def autotune(self, ref_id, **kw):
        return pt2_autotune(self.handle, ref_id, make_opts(**kw) if kw else None)

    def submit(self, ref_id, **kw):
        return pt2_submit(self.handle, ref_id, make_opts(**kw) if kw else None)

    def poll(self, ticket):
        return pt2_poll(self.handle, ticket)

    def wait(self, ticket, timeout_s=3600.0):
        return pt2_wait(self.handle, ticket, timeout_s)

    def server_stats(self):
        return pt2_server_stats(self.handle)

    def eval_terms(self, num, denom):
        return pt2_eval_terms(self.handle, num, denom)

    def phase_times(self):
        return pt2_phase_times(self.handle)

    def memory_info(self):
        return pt2_memory_info(self.handle)

    @property
    def stream(self):
        return pt2_stream(self.handle)
