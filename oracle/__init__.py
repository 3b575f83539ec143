"""CPU oracle for the Epstein-Nesbet PT2 energy (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
binding) never calls it and shares no code with it.

The arithmetic lives in ``pt2_oracle.c`` (plain C, FP64, hash-map
accumulation, direct diagonal, sorted Neumaier sum); this module compiles it
with gcc on first use and marshals numpy arrays through ctypes.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pt2_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OracleResult(ctypes.Structure):
    _fields_ = [
        ("e2", ctypes.c_double),
        ("e2_ref_like", ctypes.c_double),
        ("n_terms", ctypes.c_uint64),
        ("n_unique", ctypes.c_uint64),
        ("n_in_ref", ctypes.c_uint64),
        ("n_external", ctypes.c_uint64),
        ("digest_sum", ctypes.c_uint64),
        ("digest_xor", ctypes.c_uint64),
        ("min_abs_denom", ctypes.c_double),
        ("n_pos_denom", ctypes.c_uint64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.oracle_pt2.restype = ctypes.c_int64
            lib.oracle_pt2.argtypes = [ctypes.c_int, P, P, ctypes.c_int64, P, P, ctypes.c_double,
                                       ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                       ctypes.c_double,
                                       ctypes.POINTER(OracleResult), P, P, P, ctypes.c_int64]
            lib.oracle_diagonals.restype = None
            lib.oracle_diagonals.argtypes = [ctypes.c_int, P, P, ctypes.c_int64, P, P]
            lib.oracle_det_terms.restype = ctypes.c_int64
            lib.oracle_det_terms.argtypes = [ctypes.c_int, P, P, ctypes.c_uint64, ctypes.c_uint64,
                                             ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
                                             P, P, P, ctypes.c_int64]
            lib.oracle_digest_mix1.restype = ctypes.c_uint64
            lib.oracle_digest_mix1.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.oracle_digest_mix2.restype = ctypes.c_uint64
            lib.oracle_digest_mix2.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _prep(h, eri, keys=None, coef=None):
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    out = [h, eri]
    if keys is not None:
        out.append(np.ascontiguousarray(keys, dtype=np.uint64))
    if coef is not None:
        out.append(np.ascontiguousarray(coef, dtype=np.float64))
    return out


def pt2(h, eri, keys, coef, e0, constraint=(1, 0), include_ref=False, cutoff=0.0, top_alpha=0) -> dict:
    """E2 and the connected-set statistics (see pt2_oracle.c); contributions
    |c_i H_ai| below `cutoff` are ignored."""
    lib = _load()
    h, eri, keys, coef = _prep(h, eri, keys, coef)
    n = h.shape[0]
    res = OracleResult()
    rc = lib.oracle_pt2(n, _p(h), _p(eri), coef.shape[0], _p(keys), _p(coef), float(e0),
                        int(constraint[0]), int(constraint[1]), int(top_alpha), int(bool(include_ref)),
                        float(cutoff),
                        ctypes.byref(res), None, None, None, 0)
    if rc < 0:
        raise ValueError(f"oracle_pt2 failed with code {rc}")
    return res.as_dict()


def dump_external(h, eri, keys, coef, e0, constraint=(1, 0), cutoff=0.0, top_alpha=0):
    """Sorted external keys (n, 2) uint64 with summed numerators and direct diagonals."""
    lib = _load()
    h, eri, keys, coef = _prep(h, eri, keys, coef)
    n = h.shape[0]
    res = OracleResult()
    rc = lib.oracle_pt2(n, _p(h), _p(eri), coef.shape[0], _p(keys), _p(coef), float(e0),
                        int(constraint[0]), int(constraint[1]), int(top_alpha), 0, float(cutoff), ctypes.byref(res),
                        None, None, None, 0)
    if rc < 0:
        raise ValueError(f"oracle_pt2 failed with code {rc}")
    m = int(res.n_external)
    k = np.zeros(2 * max(m, 1), dtype=np.uint64)
    num = np.zeros(max(m, 1))
    haa = np.zeros(max(m, 1))
    rc = lib.oracle_pt2(n, _p(h), _p(eri), coef.shape[0], _p(keys), _p(coef), float(e0),
                        int(constraint[0]), int(constraint[1]), int(top_alpha), 0, float(cutoff), ctypes.byref(res),
                        _p(k), _p(num), _p(haa), m)
    if rc != m:
        raise ValueError(f"oracle dump returned {rc}, expected {m}")
    return k[: 2 * m].reshape(m, 2), num[:m], haa[:m], res.as_dict()


def diagonals(h, eri, keys) -> np.ndarray:
    """Direct diagonal H_kk of each determinant of keys (alpha, beta interleaved)."""
    lib = _load()
    h, eri, keys = _prep(h, eri, keys)
    m = keys.shape[0] // 2
    out = np.empty(m)
    lib.oracle_diagonals(h.shape[0], _p(h), _p(eri), m, _p(keys), _p(out))
    return out


def det_terms(h, eri, alpha, beta, c, constraint=(1, 0)):
    """Terms (keys (m,2), H_ai c, direct H_aa) one determinant generates, in enumeration order."""
    lib = _load()
    h, eri = _prep(h, eri)
    n = h.shape[0]
    total = lib.oracle_det_terms(n, _p(h), _p(eri), int(alpha), int(beta), float(c),
                                 int(constraint[0]), int(constraint[1]), None, None, None, 0)
    k = np.zeros(2 * max(total, 1), dtype=np.uint64)
    v = np.zeros(max(total, 1))
    d = np.zeros(max(total, 1))
    lib.oracle_det_terms(n, _p(h), _p(eri), int(alpha), int(beta), float(c),
                         int(constraint[0]), int(constraint[1]), _p(k), _p(v), _p(d), total)
    return k[: 2 * total].reshape(total, 2), v[:total], d[:total]


def digest(keys2: np.ndarray):
    """(sum mix1 mod 2^64, xor mix2) of a set of keys given as an (m, 2) array."""
    lib = _load()
    s = 0
    x = 0
    for a, b in keys2.tolist():
        s = (s + lib.oracle_digest_mix1(a, b)) & 0xFFFFFFFFFFFFFFFF
        x ^= lib.oracle_digest_mix2(a, b)
    return s, x


def e0_of(h, eri, keys, shift=0.1) -> float:
    """E0 of the synthetic recipe: lowest reference diagonal minus shift."""
    return float(diagonals(h, eri, keys).min() - shift)
