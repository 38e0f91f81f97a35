"""GB300 (sm_103a) SF-sketch: Python binding of the C ABI in include/sf.h.

Argument marshalling only: every step of insert, delete, export and query runs in the CUDA
library ``_build/libsfgb300.so``.  PyTorch supplies device memory and streams.  There is no
CPU fallback: ``load()`` raises if the library is missing or no GPU is present.

    import torch, paper_1701_04148_gb300 as sf
    sk = sf.Sketch(d=4, w=1 << 18, z=16, key_bytes=13, seed=2, chunk=65536)
    sk.insert(keys_u8_on_gpu)          # (n, 13) uint8 device tensor
    slim, hdr = sk.export_slim()
    est = sf.query(slim, hdr, flows_u8_on_gpu)
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsfgb300.so")
BENCH_LIB_PATH = os.path.join(_HERE, "_build", "libsfbench.so")

SF_OK = 0
SF_ERR_INVALID = -1
SF_ERR_OOM = -2
SF_ERR_CUDA = -3
SF_ERR_TIMEOUT = -4
SF_ERR_UNDERFLOW = -5
SF_ERR_BUDGET = -6
SF_ERR_VERSION = -7
SF_PENDING = 1
SF_FLAG_EXPLICIT_INDEX = 1
SF_FLAG_SF4_DELETE = 2
SF_FLAG_SHARED_DICT = 4
SF_SLIM_MAGIC = 0x4D494C53
SF_HASH_SPLITMIX_LEMIRE = 1
SF_HASH_EXPLICIT = 2


class SFError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_str(status)} ({status})")


class Params(ctypes.Structure):
    _fields_ = [("d", ctypes.c_uint32), ("w", ctypes.c_uint32), ("z", ctypes.c_uint32),
                ("key_bytes", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("chunk", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class SlimHeader(ctypes.Structure):
    _fields_ = [("magic", ctypes.c_uint32), ("version", ctypes.c_uint32), ("d", ctypes.c_uint32),
                ("w", ctypes.c_uint32), ("key_bytes", ctypes.c_uint32), ("hash_id", ctypes.c_uint32),
                ("seed", ctypes.c_uint64)]


class SlimView(ctypes.Structure):
    _fields_ = [("counters", ctypes.c_void_p), ("hdr", SlimHeader), ("index_table", ctypes.c_void_p),
                ("n_index_keys", ctypes.c_uint32)]


class CollectorConfig(ctypes.Structure):
    _fields_ = [("arena_dev", ctypes.c_void_p), ("arena_bytes", ctypes.c_uint64), ("staging_dev", ctypes.c_void_p),
                ("staging_bytes", ctypes.c_uint64), ("max_sketches", ctypes.c_uint32), ("n_streams", ctypes.c_uint32),
                ("max_batch_keys", ctypes.c_uint32), ("max_batch_reqs", ctypes.c_uint32),
                ("max_wait_us", ctypes.c_uint32)]


class CollectorStats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_uint64), ("keys", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("uploads", ctypes.c_uint64), ("rejected_uploads", ctypes.c_uint64), ("evictions", ctypes.c_uint64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("qps", ctypes.c_double), ("arena_used_bytes", ctypes.c_uint64)]


_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes)
_SIGS = {
    "sf_status_str": (ctypes.c_char_p, [ctypes.c_int32]),
    "sf_required_bytes": (ctypes.c_int32, [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_uint64),
                                           ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "sf_create": (ctypes.c_int32, [ctypes.POINTER(Params), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "sf_destroy": (ctypes.c_int32, [ctypes.c_void_p]),
    "sf_reset": (ctypes.c_int32, [ctypes.c_void_p]),
    "sf_set_index_table": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32]),
    "sf_insert_batch": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64]),
    "sf_delete_batch": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64]),
    "sf_update_batch": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64]),
    "sf_export_slim": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                        ctypes.POINTER(SlimHeader)]),
    "sf_query_batch": (ctypes.c_int32, [ctypes.POINTER(SlimView), ctypes.c_void_p, ctypes.c_uint64,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "sf_sync": (ctypes.c_int32, [ctypes.c_void_p]),
    "sf_update_pipelined": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                             ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]),
    "sf_query_pipelined": (ctypes.c_int32, [ctypes.POINTER(SlimView), ctypes.c_void_p, ctypes.c_uint64,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                            ctypes.c_void_p]),
    "sf_batch_required_bytes": (ctypes.c_int32, [ctypes.c_uint32, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]),
    "sf_batch_create": (ctypes.c_int32, [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p)]),
    "sf_batch_update": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]),
    "sf_batch_sync": (ctypes.c_int32, [ctypes.c_void_p]),
    "sf_batch_set_group_bytes": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64]),
    "sf_batch_set_block_threads": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32]),
    "sf_batch_set_dictionary_arena": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64]),
    "sf_dictionary_bytes": (ctypes.c_int32, [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_uint64)]),
    "sf_set_dictionary": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64]),
    "sf_pipeline_create": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_void_p)]),
    "sf_update_pipeline": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int32, ctypes.c_uint64]),
    "sf_pipeline_destroy": (ctypes.c_int32, [ctypes.c_void_p]),
    "sf_batch_groups": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32),
                                         ctypes.POINTER(ctypes.c_uint64)]),
    "sf_batch_info": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32),
                                       ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64)]),
    "sf_batch_destroy": (ctypes.c_int32, [ctypes.c_void_p]),
    "sfc_required_staging_bytes": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "sfc_create": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "sfc_upload": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.POINTER(SlimHeader)]),
    "sfc_evict": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32]),
    "sfc_query_submit": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint64,
                                          ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "sfc_poll": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64]),
    "sfc_wait": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64]),
    "sfc_stats_get": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "sfc_destroy": (ctypes.c_int32, [ctypes.c_void_p]),
    "sf_update_batch_noalloc": (ctypes.c_int32, [ctypes.POINTER(Params), ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                                 ctypes.c_void_p]),
}

# The measurement library (include/sf_bench.h): roofline denominators and the bounded-wait test kernel.
_BENCH_SIGS = {
    "sf_bench_random_access": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                                ctypes.c_uint32, ctypes.c_void_p]),
    "sf_bench_grid_barrier": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]),
    "sf_bench_wait_timeout": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p]),
}
_bench_lib = None


def exported_symbols() -> list[str]:
    return list(_SIGS)


def exported_bench_symbols() -> list[str]:
    return list(_BENCH_SIGS)


def load_bench(path: str | None = None):
    """Load the measurement library libsfbench.so (raises if it was not built)."""
    global _bench_lib
    with _lock:
        if _bench_lib is None:
            p = path or BENCH_LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"measurement library not built ({p}); run "
                                   "`python -m paper_1701_04148_gb300.build` on a machine with nvcc")
            L = ctypes.CDLL(p)
            for name, (res, args) in _BENCH_SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _bench_lib = L
    return _bench_lib


def load(path: str | None = None):
    """Load the CUDA library (raises if it was not built: there is no CPU path)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"SF-sketch CUDA library not built ({p}); run "
                                   "`python -m paper_1701_04148_gb300.build` on a machine with nvcc")
            L = ctypes.CDLL(p)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def status_str(st: int) -> str:
    try:
        return load().sf_status_str(st).decode()
    except Exception:  # library not loadable: still name the code
        return {0: "ok", -1: "invalid argument", -2: "buffer too small", -3: "CUDA runtime error",
                -4: "device wait timed out", -5: "underflow", -6: "budget", -7: "version"}.get(st, "?")


def check(st: int, what: str) -> int:
    if st < 0:
        raise SFError(st, what)
    return st


def _torch():
    import torch
    return torch


def _stream_handle(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dev_ptr(t, what: str) -> int:
    if t is None:
        return 0
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return int(t.data_ptr())


def _host_ptr(a) -> int:
    """Address of a contiguous host numpy array or CPU tensor (the collector's per-request path:
    __array_interface__ is about twice as fast as ndarray.ctypes)."""
    dp = getattr(a, "data_ptr", None)
    if dp is not None:
        return int(dp())
    return a.__array_interface__["data"][0]


def _io_ptr(t, what: str) -> int:
    """Keys, operations and query answers: a CUDA tensor, or a pinned (page-locked) CPU tensor
    that the kernels read or write over the host link themselves (the library checks it)."""
    if t is None:
        return 0
    if not t.is_cuda and not t.is_pinned():
        raise ValueError(f"{what} must be a CUDA tensor or a pinned CPU tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return int(t.data_ptr())


def make_params(d, w, z, key_bytes, seed, chunk, flags=0) -> Params:
    return Params(d, w, z, key_bytes, seed & (2**64 - 1), chunk, flags)


def dictionary_bytes(d, w, z, key_bytes, seed, chunk) -> int:
    """sf_dictionary_bytes: the chunk dictionary of a sketch with these parameters."""
    out = ctypes.c_uint64()
    check(load().sf_dictionary_bytes(ctypes.byref(make_params(d, w, z, key_bytes, seed, chunk)), ctypes.byref(out)),
          "sf_dictionary_bytes")
    return out.value


def required_bytes(p: Params):
    fb, sb, xb = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    check(load().sf_required_bytes(ctypes.byref(p), ctypes.byref(fb), ctypes.byref(sb), ctypes.byref(xb)),
          "sf_required_bytes")
    return fb.value, sb.value, xb.value


class Sketch:
    """One SF-sketch on the current CUDA device, buffers owned by torch tensors."""

    def __init__(self, d: int, w: int, z: int, key_bytes: int = 4, seed: int = 0, chunk: int = 1,
                 explicit_index: bool = False, stream=None, device=None, delete_rule: str = "sff",
                 shared_dict: bool = False):
        """delete_rule: "sff" (Sec. 3.5, the final design) or "sf4" (Sec. 3.4, the ablation).
        shared_dict: the chunk dictionary is not in the sketch's scratch (SF_FLAG_SHARED_DICT): a
        Batch with a dictionary arena supplies it, or set_dictionary for standalone updates."""
        torch = _torch()
        L = load()
        if delete_rule not in ("sff", "sf4"):
            raise ValueError("delete_rule must be 'sff' or 'sf4'")
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the SF-sketch library has no CPU path")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        flags = ((SF_FLAG_EXPLICIT_INDEX if explicit_index else 0) | (SF_FLAG_SF4_DELETE if delete_rule == "sf4" else 0)
                 | (SF_FLAG_SHARED_DICT if shared_dict else 0))
        self.params = make_params(d, w, z, key_bytes, seed, chunk, flags)
        fb, sb, xb = required_bytes(self.params)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            self.fat = torch.empty(fb // 4, dtype=torch.int32, device=self.device)
            self.slim = torch.empty(sb // 4, dtype=torch.int32, device=self.device)
            self.scratch = torch.empty(max(xb, 16) // 4 + 4, dtype=torch.int32, device=self.device)
            h = ctypes.c_void_p()
            check(L.sf_create(ctypes.byref(self.params), self.fat.data_ptr(), self.slim.data_ptr(),
                              self.scratch.data_ptr(), _stream_handle(self.stream), ctypes.byref(h)), "sf_create")
        self.handle = h
        self._index_table = None
        self._held = []  # host tensors of calls in flight: the copies and kernels read them later

    def _hold(self, *tensors):
        for t in tensors:
            if t is not None and t.device.type == "cpu":
                self._held.append(t)

    def reset(self):
        """Initialisation again (Sec. 3.1: all counters zero) on the same device buffers (sf_reset)."""
        check(load().sf_reset(self.handle), "sf_reset")

    # shapes of the caller-visible views
    @property
    def d(self):
        return self.params.d

    @property
    def w(self):
        return self.params.w

    @property
    def z(self):
        return self.params.z

    def fat_view(self):
        return self.fat.view(self.d, self.w, self.z)

    def slim_view(self):
        return self.slim.view(self.d, self.w)

    def set_dictionary(self, buf):
        """sf_set_dictionary: a device uint8/int32 tensor of at least dictionary_bytes(...) bytes,
        shared with other sketches whose updates never run at the same time (zeroed here)."""
        nbytes = buf.numel() * buf.element_size()
        check(load().sf_set_dictionary(self.handle, _dev_ptr(buf, "dictionary"), nbytes), "sf_set_dictionary")
        self._dict = buf

    def set_index_table(self, table):
        """Explicit-index mode: table (n_keys, d, 2) uint32/int32 of (h_i, f_i) on the device."""
        torch = _torch()
        t = table.to(device=self.device, dtype=torch.int32).contiguous()
        self._index_table = t
        check(load().sf_set_index_table(self.handle, t.data_ptr(), t.shape[0]), "sf_set_index_table")

    def _keys(self, keys):
        if keys.dim() == 2 and keys.dtype == _torch().uint8:
            if keys.shape[1] != self.params.key_bytes:
                raise ValueError("key width mismatch")
            return keys, keys.shape[0]
        return keys, keys.numel() * keys.element_size() // self.params.key_bytes

    def insert(self, keys):
        k, n = self._keys(keys)
        check(load().sf_insert_batch(self.handle, _io_ptr(k, "keys"), n), "sf_insert_batch")
        self._hold(k)

    def delete(self, keys):
        k, n = self._keys(keys)
        check(load().sf_delete_batch(self.handle, _io_ptr(k, "keys"), n), "sf_delete_batch")
        self._hold(k)

    def update(self, keys, ops):
        k, n = self._keys(keys)
        if ops.numel() != n:
            raise ValueError("ops must have one entry per key")
        check(load().sf_update_batch(self.handle, _io_ptr(k, "keys"), _io_ptr(ops, "ops"), n), "sf_update_batch")
        self._hold(k, ops)

    def update_pipelined(self, keys_host, ops_host=None, op_const: int = 1, staging=None, copy_stream=None):
        """sf_update_pipelined: host keys (pinned CPU tensor) copied in chunk-aligned pieces on
        copy_stream while the previous piece is applied.  staging: device uint8 tensor (default: two
        pieces of 2^22 updates); keep the tensors alive until sync()."""
        torch = _torch()
        k, n = self._keys(keys_host)
        if staging is None:
            per = self.params.key_bytes + (1 if ops_host is not None else 0)
            piece = max(1, (1 << 22) // self.params.chunk) * self.params.chunk
            staging = torch.empty(2 * (piece * per + 32), dtype=torch.uint8, device=self.device)
        if copy_stream is None:
            copy_stream = torch.cuda.Stream(device=self.device)
        self._pipeline = (k, ops_host, staging, copy_stream)
        check(load().sf_update_pipelined(self.handle, k.data_ptr(), ops_host.data_ptr() if ops_host is not None else 0,
                                         op_const, n, _dev_ptr(staging, "staging"), staging.numel(),
                                         int(copy_stream.cuda_stream)), "sf_update_pipelined")

    def update_through(self, pipe: "Pipeline", keys_host, ops_host=None, op_const: int = 1):
        """sf_update_pipeline: host keys (pinned CPU tensor) through a Pipeline kept across calls and
        sketches; keep keys_host (and ops_host) alive until sync()."""
        k, n = self._keys(keys_host)
        if not k.is_pinned() or (ops_host is not None and not ops_host.is_pinned()):
            raise ValueError("keys_host and ops_host must be pinned CPU tensors")
        if ops_host is not None and ops_host.numel() != n:
            raise ValueError("ops must have one entry per key")
        pipe._inputs.append((k, ops_host))
        check(load().sf_update_pipeline(self.handle, pipe.handle, k.data_ptr(),
                                        ops_host.data_ptr() if ops_host is not None else 0, op_const, n),
              "sf_update_pipeline")

    def sync(self) -> int:
        st = load().sf_sync(self.handle)
        self._held = []
        return check(st, "sf_sync")

    def sync_status(self) -> int:
        st = load().sf_sync(self.handle)
        self._held = []
        return st

    def export_slim(self, out=None):
        torch = _torch()
        n = self.d * self.w
        if out is None:
            out = torch.empty(n, dtype=torch.int32, device=self.device)
        hdr = SlimHeader()
        check(load().sf_export_slim(self.handle, _dev_ptr(out, "out"), out.numel(), ctypes.byref(hdr)),
              "sf_export_slim")
        return out, hdr

    def close(self):
        if getattr(self, "handle", None):
            load().sf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pipeline:
    """sf_pipeline: a device staging buffer and a copy stream kept across sf_update_pipeline calls, on
    one sketch or several (the first copy of a call overlaps the previous call's last update)."""

    def __init__(self, staging_bytes: int = 2 * ((1 << 22) * 16 + 16), copy_stream=None, device=None):
        torch = _torch()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            self.staging = torch.empty(int(staging_bytes), dtype=torch.uint8, device=self.device)
            self.copy_stream = copy_stream if copy_stream is not None else torch.cuda.Stream(device=self.device)
            h = ctypes.c_void_p()
            check(load().sf_pipeline_create(self.staging.data_ptr(), self.staging.numel(),
                                            int(self.copy_stream.cuda_stream), ctypes.byref(h)), "sf_pipeline_create")
        self.handle = h
        self._inputs = []  # host tensors of calls in flight (dropped by release_inputs after a sync)

    def release_inputs(self):
        """Forget the host inputs of earlier calls (call after the sketches that used them synced)."""
        self._inputs = []

    def close(self):
        if getattr(self, "handle", None):
            load().sf_pipeline_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchItem(ctypes.Structure):
    _fields_ = [("sketch", ctypes.c_void_p), ("keys_dev", ctypes.c_void_p), ("ops_dev", ctypes.c_void_p),
                ("n", ctypes.c_uint64)]


SF_BATCH_GRAPH = 1


class Batch:
    """Many sketches updated by one persistent launch (sf_batch_*), CUDA graph replay by default."""

    def __init__(self, max_sketches: int, graph: bool = True, stream=None, device=None,
                 max_round_slots: int = 1 << 22, group_bytes: int | None = None, block_threads: int | None = None,
                 dict_arena_bytes: int | None = None):
        """group_bytes: counter footprint per launch group (None: the library default, 3/4 of L2;
        0: every sketch of a call in one launch).  block_threads: threads per block of the launches,
        512 (default), 256 or 128.  dict_arena_bytes: a dictionary arena for shared_dict sketches
        (sf_batch_set_dictionary_arena)."""
        torch = _torch()
        L = load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        xb = ctypes.c_uint64()
        check(L.sf_batch_required_bytes(max_sketches, max_round_slots, ctypes.byref(xb)), "sf_batch_required_bytes")
        self.scratch = torch.empty(xb.value // 4 + 4, dtype=torch.int32, device=self.device)
        h = ctypes.c_void_p()
        check(L.sf_batch_create(max_sketches, max_round_slots, self.scratch.data_ptr(), _stream_handle(self.stream),
                                SF_BATCH_GRAPH if graph else 0, ctypes.byref(h)), "sf_batch_create")
        self.handle = h
        self.max_sketches = max_sketches
        self._keep = None
        if group_bytes is not None:
            check(L.sf_batch_set_group_bytes(self.handle, int(group_bytes)), "sf_batch_set_group_bytes")
        if block_threads is not None:
            check(L.sf_batch_set_block_threads(self.handle, int(block_threads)), "sf_batch_set_block_threads")
        self.arena = None
        if dict_arena_bytes:
            self.arena = torch.empty(int(dict_arena_bytes), dtype=torch.uint8, device=self.device)
            check(L.sf_batch_set_dictionary_arena(self.handle, self.arena.data_ptr(), self.arena.numel()),
                  "sf_batch_set_dictionary_arena")

    def update(self, items):
        """items: list of (Sketch, keys tensor, ops tensor or None)."""
        arr = (BatchItem * len(items))()
        keep = []
        for i, (sk, keys, ops) in enumerate(items):
            k, n = sk._keys(keys)
            arr[i] = BatchItem(sk.handle.value, _io_ptr(k, "keys") if n else 0, _io_ptr(ops, "ops"), n)
            keep.append((k, ops))
        self._keep = keep
        check(load().sf_batch_update(self.handle, len(items), ctypes.cast(arr, ctypes.c_void_p)), "sf_batch_update")

    def sync(self) -> int:
        return check(load().sf_batch_sync(self.handle), "sf_batch_sync")

    def sync_status(self) -> int:
        return load().sf_batch_sync(self.handle)

    def info(self):
        gl, gc, rl = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint64()
        check(load().sf_batch_info(self.handle, ctypes.byref(gl), ctypes.byref(gc), ctypes.byref(rl)), "sf_batch_info")
        ng, gb = ctypes.c_uint32(), ctypes.c_uint64()
        check(load().sf_batch_groups(self.handle, ctypes.byref(ng), ctypes.byref(gb)), "sf_batch_groups")
        return {"graph_launches": gl.value, "graph_captures": gc.value, "rounds_last": rl.value,
                "groups_last": ng.value, "group_bytes": gb.value}

    def close(self):
        if getattr(self, "handle", None):
            load().sf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def query(slim, hdr: SlimHeader, keys, out=None, stream=None, index_table=None):
    """Point queries on an exported Slim; keys and out may be CUDA tensors or pinned CPU tensors.
    Returns int32 estimates (bit pattern u32); a new out is allocated where the keys live (pinned
    when the keys are pinned)."""
    torch = _torch()
    kb = hdr.key_bytes
    n = keys.shape[0] if (keys.dim() == 2 and keys.dtype == torch.uint8) else keys.numel() * keys.element_size() // kb
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=keys.device, pin_memory=not keys.is_cuda)
    v = SlimView(_dev_ptr(slim, "slim"), hdr, _dev_ptr(index_table, "index_table") if index_table is not None else 0,
                 index_table.shape[0] if index_table is not None else 0)
    check(load().sf_query_batch(ctypes.byref(v), _io_ptr(keys, "keys") if n else 0, n,
                                _io_ptr(out, "out") if n else 0, _stream_handle(stream)), "sf_query_batch")
    return out


def as_u32(t):
    """View an int32 tensor of counters as int64 holding the unsigned values."""
    return t.to(_torch().int64) & 0xFFFFFFFF


def update_batch_noalloc(params: Params, fat, slim, keys, ops=None, err=None, stream=None) -> None:
    """sf_update_batch_noalloc: the chunked update with the library's fixed scratch array
    (no scratch buffer from the caller).  fat/slim: caller tensors laid out as required_bytes says."""
    torch = _torch()
    n = keys.shape[0] if (keys.dim() == 2 and keys.dtype == torch.uint8) else \
        keys.numel() * keys.element_size() // params.key_bytes
    check(load().sf_update_batch_noalloc(ctypes.byref(params), _dev_ptr(fat, "fat"), _dev_ptr(slim, "slim"),
                                         _io_ptr(keys, "keys") if n else 0, _io_ptr(ops, "ops"), n,
                                         _dev_ptr(err, "err"), _stream_handle(stream)), "sf_update_batch_noalloc")



class Collector:
    """The collector serving loop (sfc_*): resident Slims in a device arena of `budget_bytes`,
    continuous batching of host-side point-query requests over `n_streams` CUDA streams."""

    def __init__(self, budget_bytes: int, max_sketches: int, n_streams: int = 4, max_batch_keys: int = 1 << 17,
                 max_batch_reqs: int = 1024, max_wait_us: int = 50, device=None):
        torch = _torch()
        L = load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.arena = torch.empty(max(budget_bytes, 256) // 4, dtype=torch.int32, device=self.device)
        cfg = CollectorConfig(self.arena.data_ptr(), self.arena.numel() * 4, 0, 0, max_sketches, n_streams,
                              max_batch_keys, max_batch_reqs, max_wait_us)
        need = ctypes.c_uint64()
        check(L.sfc_required_staging_bytes(ctypes.byref(cfg), ctypes.byref(need)), "sfc_required_staging_bytes")
        self.staging = torch.empty(need.value // 4 + 64, dtype=torch.int32, device=self.device)
        cfg.staging_dev = self.staging.data_ptr()
        cfg.staging_bytes = self.staging.numel() * 4
        self.cfg = cfg
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(L.sfc_create(ctypes.byref(cfg), ctypes.byref(h)), "sfc_create")
        self.handle = h
        self._live = {}

    def upload(self, sketch_id: int, counters, hdr: SlimHeader) -> int:
        """Returns the status (SF_OK, SF_ERR_BUDGET, ...); counters: device or host tensor."""
        ptr = counters.data_ptr()
        return load().sfc_upload(self.handle, sketch_id, ptr, ctypes.byref(hdr))

    def evict(self, sketch_id: int) -> int:
        return load().sfc_evict(self.handle, sketch_id)

    def submit(self, sketch_id: int, keys_np, out_np) -> int:
        """keys_np: contiguous numpy array (or CPU tensor) of packed keys (host); out_np: uint32 numpy
        array (or CPU tensor) of one answer per key."""
        t = ctypes.c_uint64()
        n = len(out_np)
        check(load().sfc_query_submit(self.handle, sketch_id, _host_ptr(keys_np) if n else None, n,
                                      _host_ptr(out_np) if n else None, ctypes.byref(t)), "sfc_query_submit")
        self._live[t.value] = (keys_np, out_np)
        return t.value

    def poll(self, ticket: int) -> int:
        st = load().sfc_poll(self.handle, ticket)
        if st != SF_PENDING:
            self._live.pop(ticket, None)
        return st

    def wait(self, ticket: int) -> int:
        st = load().sfc_wait(self.handle, ticket)
        self._live.pop(ticket, None)
        return st

    def stats(self, reset: bool = False) -> dict:
        s = CollectorStats()
        check(load().sfc_stats_get(self.handle, ctypes.byref(s), 1 if reset else 0), "sfc_stats_get")
        return {f: getattr(s, f) for f, _ in CollectorStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            load().sfc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def query_pipelined(slim, hdr: SlimHeader, keys_host, out_host, keys_dev, out_dev, streams) -> None:
    """sf_query_pipelined: the batch split over len(streams) CUDA streams (copy in, query, copy out
    per part).  keys_host/out_host: pinned CPU tensors; keys_dev/out_dev: device staging tensors."""
    n = out_host.numel()
    arr = (ctypes.c_void_p * len(streams))(*[int(s.cuda_stream) for s in streams])
    v = SlimView(_dev_ptr(slim, "slim"), hdr, 0, 0)
    check(load().sf_query_pipelined(ctypes.byref(v), keys_host.data_ptr(), n, out_host.data_ptr(),
                                    _dev_ptr(keys_dev, "keys_dev"), _dev_ptr(out_dev, "out_dev"), len(streams),
                                    ctypes.cast(arr, ctypes.c_void_p)), "sf_query_pipelined")
