"""Plain CPU oracle of the SF-sketch (SF_F form) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package.  It wraps ``sf_oracle.c`` (plain sequential C, compiled with gcc) through
ctypes and shares no code with the CUDA library.

Semantics (see ``sf_oracle.c`` for the full statement):
  * ``seq_apply``   -- the paper's one-update-at-a-time insertion (Sec. 3.4, SF_4 = SF_F
                       insertion) and SF_F deletion (Sec. 3.5), literal or clamp form; or, with
                       ``delete_rule="sf4"``, the SF_4 deletion (Sec. 3.4: decrement by 1 above
                       the bucket sum), kept for the ablation against SF_F.
  * ``chunk_apply`` -- the chunked schedule CHUNK(S), stream order inside each chunk.
  * ``query``       -- min over the d hashed Slim counters (Sec. 3.1 "Query").
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile sf_oracle.c into oracle/_build/liboracle.so (plain gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


class use_library:
    """Context manager that swaps in another build of sf_oracle.c (used by the mutation
    tests, which compile deliberately broken copies to check that the pins catch them)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        lib()
        self.prev = _lib
        _lib = _configure(ctypes.CDLL(self.path))
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.prev
        return False


def _configure(L):
    u32p = ctypes.POINTER(ctypes.c_uint32)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    i8p = ctypes.POINTER(ctypes.c_int8)
    L.osf_mix64.restype = ctypes.c_uint64
    L.osf_mix64.argtypes = [ctypes.c_uint64]
    L.osf_splitmix64_next.restype = ctypes.c_uint64
    L.osf_splitmix64_next.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
    L.osf_row_seeds.restype = None
    L.osf_row_seeds.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64)]
    L.osf_index_keys.restype = None
    L.osf_index_keys.argtypes = [u8p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                 ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, u32p, u32p]
    L.osf_seq_apply.restype = None
    L.osf_seq_apply.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, u32p, u32p,
                                u32p, u32p, i8p, ctypes.c_uint64, ctypes.c_int]
    L.osf_chunk_apply_rule.restype = ctypes.c_int
    L.osf_chunk_apply_rule.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, u32p, u32p,
                                       u32p, u32p, i8p, ctypes.c_uint64, ctypes.c_uint64,
                                       u8p, ctypes.c_uint32, ctypes.c_int]
    L.osf_chunk_apply.restype = ctypes.c_int
    L.osf_chunk_apply.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, u32p, u32p,
                                  u32p, u32p, i8p, ctypes.c_uint64, ctypes.c_uint64,
                                  u8p, ctypes.c_uint32]
    L.osf_query_idx.restype = None
    L.osf_query_idx.argtypes = [ctypes.c_uint32, ctypes.c_uint32, u32p, u32p, ctypes.c_uint64, u32p]
    return L


def _p(a: np.ndarray, ct):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.POINTER(ct))


def mix64(x: int) -> int:
    return int(lib().osf_mix64(ctypes.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def splitmix64_sequence(seed: int, n: int) -> list[int]:
    st = ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF)
    return [int(lib().osf_splitmix64_next(ctypes.byref(st))) for _ in range(n)]


def row_seeds(seed: int, d: int) -> np.ndarray:
    out = np.zeros(d, dtype=np.uint64)
    lib().osf_row_seeds(ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), d, _p(out, ctypes.c_uint64))
    return out


def index_keys(keys: np.ndarray, seed: int, d: int, w: int, z: int):
    """h, f of every key: arrays of shape (n, d), uint32.  keys: uint8 (n, key_bytes)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint8)
    n, kb = keys.shape
    h = np.zeros((n, d), dtype=np.uint32)
    f = np.zeros((n, d), dtype=np.uint32)
    if n:
        lib().osf_index_keys(_p(keys, ctypes.c_uint8), kb, n, ctypes.c_uint64(seed & (2**64 - 1)),
                             d, w, z, _p(h, ctypes.c_uint32), _p(f, ctypes.c_uint32))
    return h, f


class Sketch:
    """Oracle state: Slim A (d, w) and Fat B (d, w, z), uint32, all zero at init (Sec. 3.1).
    delete_rule: "sff" (Sec. 3.5, the final design) or "sf4" (Sec. 3.4)."""

    def __init__(self, d: int, w: int, z: int, key_bytes: int = 4, seed: int = 0, delete_rule: str = "sff"):
        if delete_rule not in ("sff", "sf4"):
            raise ValueError("delete_rule must be 'sff' or 'sf4'")
        self.d, self.w, self.z, self.key_bytes, self.seed = d, w, z, key_bytes, seed
        self.delete_rule = delete_rule
        self.A = np.zeros((d, w), dtype=np.uint32)
        self.B = np.zeros((d, w, z), dtype=np.uint32)

    def copy(self) -> "Sketch":
        s = Sketch(self.d, self.w, self.z, self.key_bytes, self.seed, self.delete_rule)
        s.A[...] = self.A
        s.B[...] = self.B
        return s

    # -- index-level calls -------------------------------------------------------
    def seq_apply(self, h, f, ops, literal: bool = True) -> None:
        """SEQ semantics.  SF_F deletes: literal rule or the clamp form; SF_4: its literal rule."""
        h, f, ops = _prep(h, f, ops, self.d)
        rule = 2 if self.delete_rule == "sf4" else (1 if literal else 0)
        lib().osf_seq_apply(self.d, self.w, self.z, _p(self.A, ctypes.c_uint32), _p(self.B, ctypes.c_uint32),
                            _p(h, ctypes.c_uint32), _p(f, ctypes.c_uint32), _p(ops, ctypes.c_int8),
                            len(ops), rule)

    def chunk_apply(self, h, f, ops, S: int, ident: np.ndarray) -> None:
        h, f, ops = _prep(h, f, ops, self.d)
        if len(ops) == 0:
            return
        ident = np.ascontiguousarray(ident).view(np.uint8).reshape(len(ops), -1)
        ident = np.ascontiguousarray(ident)
        rc = lib().osf_chunk_apply_rule(self.d, self.w, self.z, _p(self.A, ctypes.c_uint32),
                                        _p(self.B, ctypes.c_uint32), _p(h, ctypes.c_uint32),
                                        _p(f, ctypes.c_uint32), _p(ops, ctypes.c_int8), len(ops), S,
                                        _p(ident, ctypes.c_uint8), ident.shape[1] if len(ops) else 1,
                                        1 if self.delete_rule == "sf4" else 0)
        if rc != 0:
            raise ValueError("osf_chunk_apply failed (bad arguments or out of memory)")

    def query_idx(self, h) -> np.ndarray:
        h = np.ascontiguousarray(h, dtype=np.uint32).reshape(-1, self.d)
        out = np.zeros(len(h), dtype=np.uint32)
        if len(h):
            lib().osf_query_idx(self.d, self.w, _p(self.A, ctypes.c_uint32), _p(h, ctypes.c_uint32),
                                len(h), _p(out, ctypes.c_uint32))
        return out

    # -- key-level calls -----------------------------------------------------------
    def index(self, keys: np.ndarray):
        return index_keys(_as_key_bytes(keys, self.key_bytes), self.seed, self.d, self.w, self.z)

    def update(self, keys: np.ndarray, ops: np.ndarray, S: int | None = None, literal: bool = True) -> None:
        """One call of the stream.  S=None: SEQ semantics; S>=1: CHUNK(S) semantics."""
        kb = _as_key_bytes(keys, self.key_bytes)
        h, f = index_keys(kb, self.seed, self.d, self.w, self.z)
        ops = np.ascontiguousarray(ops, dtype=np.int8)
        if S is None:
            self.seq_apply(h, f, ops, literal=literal)
        else:
            self.chunk_apply(h, f, ops, S, kb)

    def insert(self, keys, S=None):
        n = len(_as_key_bytes(keys, self.key_bytes))
        self.update(keys, np.ones(n, dtype=np.int8), S)

    def delete(self, keys, S=None, literal: bool = True):
        n = len(_as_key_bytes(keys, self.key_bytes))
        self.update(keys, -np.ones(n, dtype=np.int8), S, literal=literal)

    def query(self, keys: np.ndarray) -> np.ndarray:
        h, _ = self.index(keys)
        return self.query_idx(h)


def _prep(h, f, ops, d):
    h = np.ascontiguousarray(h, dtype=np.uint32).reshape(-1, d)
    f = np.ascontiguousarray(f, dtype=np.uint32).reshape(-1, d)
    ops = np.ascontiguousarray(ops, dtype=np.int8).reshape(-1)
    if not (len(h) == len(f) == len(ops)):
        raise ValueError("h, f and ops must describe the same number of updates")
    return h, f, ops


def _as_key_bytes(keys: np.ndarray, key_bytes: int) -> np.ndarray:
    """Packed little-endian key bytes, shape (n, key_bytes)."""
    keys = np.asarray(keys)
    if keys.dtype == np.uint8 and keys.ndim == 2:
        if keys.shape[1] != key_bytes:
            raise ValueError(f"keys have {keys.shape[1]} bytes, sketch expects {key_bytes}")
        return np.ascontiguousarray(keys)
    if key_bytes == 4:
        return np.ascontiguousarray(keys.astype("<u4")).view(np.uint8).reshape(-1, 4)
    if key_bytes == 8:
        return np.ascontiguousarray(keys.astype("<u8")).view(np.uint8).reshape(-1, 8)
    raise ValueError("keys must be uint8 (n, key_bytes) for this key width")


def explicit_indices(table: np.ndarray, ids: np.ndarray):
    """Explicit-index mode: table (n_keys, d, 2) holds (h_i, f_i) per key id.
    Returns h, f of the id stream and the identity bytes (the ids) for CHUNK(S)."""
    table = np.asarray(table, dtype=np.uint32)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    h = np.ascontiguousarray(table[ids, :, 0])
    f = np.ascontiguousarray(table[ids, :, 1])
    return h, f, ids.view(np.uint8).reshape(-1, 4)
