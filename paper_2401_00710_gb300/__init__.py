"""Python binding of the dtsort C-ABI (include/dtsort.h).

Functions keep the C names and only marshal arguments (integers for device
pointers and streams); every step of the sort runs in the CUDA library
``_build/libdtsort.so``.  There is no fallback: if the library is missing or a
call fails, an exception is raised.

``Sorter`` is a small convenience layer over the same calls for PyTorch
tensors: it owns a handle and a workspace tensor and sorts in place.
"""
import ctypes
import os

from . import _build_ext

_lib = None

DTSORT_OK = 0
DTSORT_ERR_INVALID_ARG = 1
DTSORT_ERR_WORKSPACE_TOO_SMALL = 2
DTSORT_ERR_CUDA = 3
DTSORT_ERR_DEVICE_TIMEOUT = 4
DTSORT_ERR_UNSUPPORTED = 5
DTSORT_ERR_INTERNAL = 6

DTSORT_OP_U32, DTSORT_OP_U32_KV, DTSORT_OP_U64, DTSORT_OP_U64_KV = 0, 1, 2, 3
DTSORT_BUCKETING_DIGIT, DTSORT_BUCKETING_LEARNED, DTSORT_BUCKETING_LEARNED_ALWAYS = 0, 1, 2
DTSORT_MERGE_DOVETAIL, DTSORT_MERGE_GENERIC = 0, 1

# C symbols declared in include/dtsort.h
EXPORTED = [
    "dtsort_status_string", "dtsort_create", "dtsort_destroy",
    "dtsort_default_options", "dtsort_set_options", "dtsort_get_options",
    "dtsort_workspace_bytes", "dtsort_u32", "dtsort_u32_kv", "dtsort_u64",
    "dtsort_u64_kv", "dtsort_sort_host", "dtsort_segmented_u32", "dtsort_segmented_u32_kv",
    "dtsort_segmented_u64", "dtsort_segmented_u64_kv",
    "dtsort_last_device_error", "dtsort_get_stats", "dtsort_debug_sample",
    "dtsort_u32_kv_noalloc", "dtsort_autotune", "dtsort_autotune_scratch_bytes",
    "dtsort_mlp_forward", "dtsort_mlp_grad", "dtsort_mlp_adam", "dtsort_mlp_train",
    "dtsort_shard_sample", "dtsort_shard_splitters", "dtsort_shard_partition_workspace_bytes",
    "dtsort_shard_partition",
]

# most ranges of a sharded sort (DTSORT_SHARD_MAX_PARTS in dtsort.h)
DTSORT_SHARD_MAX_PARTS = 64

# largest n of dtsort_u32_kv_noalloc (DTSORT_NOALLOC_MAX_N in dtsort.h)
DTSORT_NOALLOC_MAX_N = 1 << 20


class DtsortError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        msg = status_string(status) if _lib is not None else str(status)
        super().__init__("%s%s" % (where + ": " if where else "", msg))


class dtsort_options(ctypes.Structure):
    _fields_ = [("gamma_max", ctypes.c_int32),
                ("finisher_capacity", ctypes.c_int32),
                ("heavy_detection", ctypes.c_int32),
                ("bucketing", ctypes.c_int32),
                ("seed", ctypes.c_uint64),
                ("sample_log_factor", ctypes.c_int32),
                ("autotune", ctypes.c_int32),
                ("learned_segments", ctypes.c_int32),
                ("learned_train_steps", ctypes.c_int32),
                ("wait_limit_ms", ctypes.c_int32),
                ("debug_fault", ctypes.c_int32),
                ("launch_mode", ctypes.c_int32),
                ("block_tiles", ctypes.c_int32),
                ("merge", ctypes.c_int32),
                ("heavy_min_share", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class dtsort_stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32),
                ("status", ctypes.c_int32),
                ("segments", ctypes.c_int64 * 16),
                ("records", ctypes.c_int64 * 16),
                ("heavy_keys", ctypes.c_int64 * 16),
                ("heavy_records", ctypes.c_int64 * 16),
                ("overflow_records", ctypes.c_int64 * 16),
                ("finisher_tasks", ctypes.c_int64),
                ("finisher_records", ctypes.c_int64),
                ("copy_records", ctypes.c_int64),
                ("merge_zones", ctypes.c_int64),
                ("merge_records", ctypes.c_int64),
                ("learned_fixup_records", ctypes.c_int64),
                ("learned_fixup_steps", ctypes.c_int64),
                ("learned_bucket_cv", ctypes.c_double),
                ("learned_bucket_max_over_mean", ctypes.c_double),
                ("phase_ms", ctypes.c_double * 8),
                ("check_site", ctypes.c_int64),
                ("check_values", ctypes.c_int64 * 2),
                ("finisher_lsd_tasks", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64),
                ("learned_zones_used", ctypes.c_int64),
                ("learned_estimate", ctypes.c_double * 2),
                ("merge_free_zones", ctypes.c_int64)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            if hasattr(v, "__len__"):
                v = list(v)
            if name != "reserved":
                out[name] = v
        return out


def library_path():
    return _build_ext.LIB


def build(force=False, verbose=False):
    """Compile the CUDA library for sm_103a (nvcc), in-tree."""
    return _build_ext.build(force=force, verbose=verbose)


def lib():
    """The loaded C library; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = _build_ext.LIB
        if not os.path.exists(path):
            raise RuntimeError(
                "dtsort CUDA library not built (%s missing); run "
                "paper_2401_00710_gb300.build()" % path)
        L = ctypes.CDLL(path)
        _declare(L)
        _lib = L
    return _lib


_H = ctypes.c_void_p
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SZ = ctypes.c_size_t
_ST = ctypes.c_int


def _declare(L):
    L.dtsort_status_string.argtypes = [_ST]
    L.dtsort_status_string.restype = ctypes.c_char_p
    L.dtsort_create.argtypes = [ctypes.POINTER(_H), ctypes.c_int]
    L.dtsort_destroy.argtypes = [_H]
    L.dtsort_default_options.argtypes = [ctypes.POINTER(dtsort_options)]
    L.dtsort_set_options.argtypes = [_H, ctypes.POINTER(dtsort_options)]
    L.dtsort_get_options.argtypes = [_H, ctypes.POINTER(dtsort_options)]
    L.dtsort_workspace_bytes.argtypes = [_H, ctypes.c_int, _I64, _I64,
                                         ctypes.POINTER(_SZ)]
    for name in ("dtsort_u32", "dtsort_u64"):
        getattr(L, name).argtypes = [_H, _P, _I64, _P, _SZ, _P]
    for name in ("dtsort_u32_kv", "dtsort_u64_kv"):
        getattr(L, name).argtypes = [_H, _P, _P, _I64, _P, _SZ, _P]
    for name in ("dtsort_segmented_u32", "dtsort_segmented_u64"):
        getattr(L, name).argtypes = [_H, _P, _P, _I64, _I64, _P, _SZ, _P]
    for name in ("dtsort_segmented_u32_kv", "dtsort_segmented_u64_kv"):
        getattr(L, name).argtypes = [_H, _P, _P, _P, _I64, _I64, _P, _SZ, _P]
    L.dtsort_sort_host.argtypes = [_H, ctypes.c_int, _P, _P, _I64, _P, _P, _P, _SZ, _P]
    L.dtsort_last_device_error.argtypes = [_H, _P]
    L.dtsort_get_stats.argtypes = [_H, ctypes.POINTER(dtsort_stats)]
    L.dtsort_debug_sample.argtypes = [_H, _P, ctypes.c_int, _I64, _I64,
                                      ctypes.c_int, ctypes.c_uint64, _I64, _I64,
                                      _P, _P, _P, _P]
    L.dtsort_u32_kv_noalloc.argtypes = [_P, _P, _I64, _P, _P]
    L.dtsort_mlp_forward.argtypes = [_P, _P, _I64, _P, _P]
    L.dtsort_mlp_grad.argtypes = [_P, _P, _P, _I64, _P, _P, _P]
    L.dtsort_mlp_adam.argtypes = [_P, _P, _P, _P, ctypes.c_int, ctypes.c_float, _P]
    L.dtsort_mlp_train.argtypes = [_P, _P, _P, _P, _P, _I64, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_float, _P, _P]
    L.dtsort_autotune_scratch_bytes.argtypes = [_H, ctypes.c_int, _I64, _I64,
                                                ctypes.POINTER(_SZ)]
    L.dtsort_autotune.argtypes = [_H, ctypes.c_int, _P, _P, _P, _I64, _I64, _P, _SZ,
                                  _P, ctypes.POINTER(dtsort_options)]
    L.dtsort_shard_sample.argtypes = [_P, ctypes.c_int, _I64, _I64, ctypes.c_uint64, _I64,
                                      _P, _P, _P]
    L.dtsort_shard_splitters.argtypes = [_P, _P, _I64, ctypes.c_int, _P, _P]
    L.dtsort_shard_partition_workspace_bytes.argtypes = [_I64, ctypes.c_int,
                                                         ctypes.POINTER(_SZ)]
    L.dtsort_shard_partition.argtypes = [_P, _P, ctypes.c_int, _I64, _I64, _P, _P,
                                         ctypes.c_int, _P, _P, _P, _P, _SZ, _P, _P]
    for name in EXPORTED:
        if name != "dtsort_status_string":
            getattr(L, name).restype = _ST


def _check(st, where):
    if st != DTSORT_OK:
        raise DtsortError(st, where)
    return st


# ---- the C-ABI, one function per entry point --------------------------------
def status_string(status):
    return lib().dtsort_status_string(int(status)).decode()


def dtsort_status_string(status):
    return status_string(status)


def dtsort_create(device=0):
    h = _H()
    _check(lib().dtsort_create(ctypes.byref(h), int(device)), "dtsort_create")
    return h.value


def dtsort_destroy(h):
    return _check(lib().dtsort_destroy(h), "dtsort_destroy")


def dtsort_default_options():
    o = dtsort_options()
    _check(lib().dtsort_default_options(ctypes.byref(o)), "dtsort_default_options")
    return o


def dtsort_set_options(h, opt=None):
    return _check(lib().dtsort_set_options(h, None if opt is None else ctypes.byref(opt)),
                  "dtsort_set_options")


def dtsort_get_options(h):
    o = dtsort_options()
    _check(lib().dtsort_get_options(h, ctypes.byref(o)), "dtsort_get_options")
    return o


def dtsort_workspace_bytes(h, op, n, num_segments=1):
    b = _SZ(0)
    _check(lib().dtsort_workspace_bytes(h, int(op), int(n), int(num_segments),
                                        ctypes.byref(b)), "dtsort_workspace_bytes")
    return b.value


def dtsort_u32(h, keys, n, ws, ws_bytes, stream=0):
    return lib().dtsort_u32(h, keys, n, ws, ws_bytes, stream or None)


def dtsort_u32_kv(h, keys, values, n, ws, ws_bytes, stream=0):
    return lib().dtsort_u32_kv(h, keys, values, n, ws, ws_bytes, stream or None)


def dtsort_u64(h, keys, n, ws, ws_bytes, stream=0):
    return lib().dtsort_u64(h, keys, n, ws, ws_bytes, stream or None)


def dtsort_u64_kv(h, keys, values, n, ws, ws_bytes, stream=0):
    return lib().dtsort_u64_kv(h, keys, values, n, ws, ws_bytes, stream or None)


def dtsort_sort_host(h, op, keys_host, values_host, n, dev_keys, dev_values, ws, ws_bytes,
                     stream=0):
    return lib().dtsort_sort_host(h, op, keys_host, values_host, n, dev_keys, dev_values, ws,
                                  ws_bytes, stream or None)


def dtsort_segmented_u32(h, keys, offsets, num_segments, n, ws, ws_bytes, stream=0):
    return lib().dtsort_segmented_u32(h, keys, offsets, num_segments, n, ws,
                                      ws_bytes, stream or None)


def dtsort_segmented_u32_kv(h, keys, values, offsets, num_segments, n, ws,
                            ws_bytes, stream=0):
    return lib().dtsort_segmented_u32_kv(h, keys, values, offsets, num_segments,
                                         n, ws, ws_bytes, stream or None)


def dtsort_segmented_u64(h, keys, offsets, num_segments, n, ws, ws_bytes, stream=0):
    return lib().dtsort_segmented_u64(h, keys, offsets, num_segments, n, ws,
                                      ws_bytes, stream or None)


def dtsort_segmented_u64_kv(h, keys, values, offsets, num_segments, n, ws,
                            ws_bytes, stream=0):
    return lib().dtsort_segmented_u64_kv(h, keys, values, offsets, num_segments,
                                         n, ws, ws_bytes, stream or None)


def dtsort_last_device_error(h, stream=0):
    return lib().dtsort_last_device_error(h, stream or None)


def dtsort_get_stats(h):
    s = dtsort_stats()
    _check(lib().dtsort_get_stats(h, ctypes.byref(s)), "dtsort_get_stats")
    return s


def dtsort_debug_sample(h, keys, key_bytes, start, size, hi, seed, count, L,
                        heavy_out, nheavy_out, max_out, stream=0):
    return lib().dtsort_debug_sample(h, keys, key_bytes, start, size, hi, seed,
                                     count, L, heavy_out, nheavy_out, max_out,
                                     stream or None)


def dtsort_mlp_forward(params, x, n, y, stream=0):
    return lib().dtsort_mlp_forward(params, x, n, y, stream or None)


def dtsort_mlp_grad(params, x, t, n, partial, grad_out, stream=0):
    return lib().dtsort_mlp_grad(params, x, t, n, partial, grad_out, stream or None)


def dtsort_mlp_adam(params, m, v, grad, step, lr, stream=0):
    return lib().dtsort_mlp_adam(params, m, v, grad, step, lr, stream or None)


def dtsort_mlp_train(params, m, v, x, t, n, steps, batch, lr, partial, stream=0):
    return lib().dtsort_mlp_train(params, m, v, x, t, n, steps, batch, lr, partial,
                                  stream or None)


def dtsort_autotune_scratch_bytes(h, op, n, num_segments=1):
    b = _SZ(0)
    _check(lib().dtsort_autotune_scratch_bytes(h, int(op), int(n), int(num_segments),
                                               ctypes.byref(b)),
           "dtsort_autotune_scratch_bytes")
    return b.value


def dtsort_autotune(h, op, keys, values, offsets, num_segments, n, scratch,
                    scratch_bytes, stream=0):
    """Returns (status, chosen options)."""
    best = dtsort_options()
    st = lib().dtsort_autotune(h, int(op), keys, values, offsets, num_segments, n,
                               scratch, scratch_bytes, stream or None,
                               ctypes.byref(best))
    return st, best


def dtsort_u32_kv_noalloc(keys, values, n, device_status=None, stream=0):
    """The allocation-free 32-bit key/value sort (n <= DTSORT_NOALLOC_MAX_N)."""
    return lib().dtsort_u32_kv_noalloc(keys, values, n, device_status, stream or None)


def dtsort_shard_sample(keys, key_bytes, n_local, gidx0, seed, count, sample_keys,
                        sample_gidx, stream=0):
    return lib().dtsort_shard_sample(keys, key_bytes, n_local, gidx0, seed, count,
                                     sample_keys, sample_gidx, stream or None)


def dtsort_shard_splitters(sample_keys, sample_gidx, m, parts, split_keys, split_gidx):
    """Host arrays (pointers) in and out."""
    return lib().dtsort_shard_splitters(sample_keys, sample_gidx, m, parts, split_keys,
                                        split_gidx)


def dtsort_shard_partition_workspace_bytes(n_local, parts):
    b = _SZ(0)
    _check(lib().dtsort_shard_partition_workspace_bytes(int(n_local), int(parts),
                                                        ctypes.byref(b)),
           "dtsort_shard_partition_workspace_bytes")
    return b.value


def dtsort_shard_partition(keys, values, key_bytes, n_local, gidx0, split_keys, split_gidx,
                           parts, out_keys, out_values, counts, ws, ws_bytes,
                           device_status=None, stream=0):
    return lib().dtsort_shard_partition(keys, values, key_bytes, n_local, gidx0, split_keys,
                                        split_gidx, parts, out_keys, out_values, counts, ws,
                                        ws_bytes, device_status, stream or None)


# ---- PyTorch convenience ----------------------------------------------------
class Sorter:
    """Owns a dtsort handle and a workspace; sorts torch CUDA tensors in place.

    keys: torch.int32/uint32 (32-bit keys) or torch.int64/uint64 (64-bit keys),
    compared as UNSIGNED integers; values (optional) of the same width are
    carried along bit for bit.  offsets (optional, int64 on the device) makes
    the call segmented.
    """

    def __init__(self, device=0, options=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device) if isinstance(device, int) else device
        self.h = dtsort_create(self.device.index or 0)
        if options is not None:
            self.set_options(**options)
        self.ws = None

    def set_options(self, **kw):
        o = dtsort_get_options(self.h)
        for k, v in kw.items():
            setattr(o, k, v)
        dtsort_set_options(self.h, o)

    def close(self):
        if self.h:
            dtsort_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def op_for(keys, values):
        wide = keys.element_size() == 8
        if values is not None and values.element_size() != keys.element_size():
            raise ValueError("values must have the key's width")
        if wide:
            return DTSORT_OP_U64_KV if values is not None else DTSORT_OP_U64
        return DTSORT_OP_U32_KV if values is not None else DTSORT_OP_U32

    def workspace(self, op, n, num_segments=1):
        need = dtsort_workspace_bytes(self.h, op, n, num_segments)
        if self.ws is None or self.ws.numel() < need:
            self.ws = self.torch.empty(max(need, 256), dtype=self.torch.uint8,
                                       device=self.device)
        return self.ws

    def sort_(self, keys, values=None, offsets=None, stream=None):
        torch = self.torch
        if not keys.is_cuda or not keys.is_contiguous():
            raise ValueError("keys must be a contiguous CUDA tensor")
        n = keys.numel()
        op = self.op_for(keys, values)
        nseg = 1 if offsets is None else offsets.numel() - 1
        ws = self.workspace(op, n, nseg)
        s = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        k = keys.data_ptr()
        v = values.data_ptr() if values is not None else None
        wsp, wsb = ws.data_ptr(), ws.numel()
        if offsets is None:
            fn = {DTSORT_OP_U32: lambda: dtsort_u32(self.h, k, n, wsp, wsb, s),
                  DTSORT_OP_U64: lambda: dtsort_u64(self.h, k, n, wsp, wsb, s),
                  DTSORT_OP_U32_KV: lambda: dtsort_u32_kv(self.h, k, v, n, wsp, wsb, s),
                  DTSORT_OP_U64_KV: lambda: dtsort_u64_kv(self.h, k, v, n, wsp, wsb, s)}[op]
        else:
            if offsets.dtype != torch.int64 or not offsets.is_cuda:
                raise ValueError("offsets must be an int64 CUDA tensor")
            o = offsets.data_ptr()
            fn = {DTSORT_OP_U32: lambda: dtsort_segmented_u32(self.h, k, o, nseg, n, wsp, wsb, s),
                  DTSORT_OP_U64: lambda: dtsort_segmented_u64(self.h, k, o, nseg, n, wsp, wsb, s),
                  DTSORT_OP_U32_KV: lambda: dtsort_segmented_u32_kv(self.h, k, v, o, nseg, n, wsp, wsb, s),
                  DTSORT_OP_U64_KV: lambda: dtsort_segmented_u64_kv(self.h, k, v, o, nseg, n, wsp, wsb, s)}[op]
        _check(fn(), "sort")
        return keys, values

    def last_device_error(self, stream=None):
        s = (stream or self.torch.cuda.current_stream(self.device)).cuda_stream
        return dtsort_last_device_error(self.h, s)

    def stats(self):
        return dtsort_get_stats(self.h).as_dict()
