"""CPU oracle for the stable integer sort (DovetailSort, PPoPP'24).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import this
package.  It shares no code with the CUDA path (``paper_2401_00710_gb300``) and
never imports it.

The arithmetic lives in ``oracle.c`` (plain C, built here with gcc); this
module only marshals numpy arrays.  What each function follows:

* ``stable_sort`` / ``stable_sort_segmented`` -- Sec. 2.3 problem statement:
  records reordered into non-decreasing key order, stably.  The unique answer
  is the lexicographic order of (key, original index).
* ``stable_positions`` -- the same definition for single records.
* ``check_sorted_keys`` -- the same definition for key-only output, where
  stability is unobservable: the input's multiset in non-decreasing order.
* ``splitmix64_*`` -- SplitMix64 (Steele, Lea, Flood 2014), the sampler's draws.
* ``sample_positions`` / ``heavy_from_sample`` / ``sample_heavy`` -- Alg. 2
  step 1 (Sec. 3.1): sample, sort, subsample every (log n)-th key, keys seen
  twice or more in the subsample are heavy; App. "Overflow bucket": the largest
  sample sets the key range.
* ``zone_layout`` / ``bucket_ids`` -- Alg. 2 bucket numbering and GetBucketId.
* ``dtmerge`` -- Alg. 3 (DTMerge) in both of its cases.

The learned-bucketing oracle (fp64 MLP forward/backward, piecewise-linear CDF
fit) is in ``oracle/learned.py``.
"""
import contextlib
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force=False):
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, portable flags)."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                           "-pthread", _SRC, "-o", tmp])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


@contextlib.contextmanager
def using_library(path):
    """Temporarily route every call through another build of oracle.c (the
    pin tests use this to check that planted mistakes are caught)."""
    global _lib
    old = _lib
    L = ctypes.CDLL(path)
    _declare(L)
    _lib = L
    try:
        yield
    finally:
        _lib = old


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_INT = ctypes.c_int


def _declare(L):
    L.oracle_default_threads.restype = _INT
    for name in ("oracle_sort_u32", "oracle_sort_u64"):
        f = getattr(L, name)
        f.argtypes = [_P, _P, _I64, _P, _P, _INT]
        f.restype = _INT
    for name in ("oracle_sort_segmented_u32", "oracle_sort_segmented_u64"):
        f = getattr(L, name)
        f.argtypes = [_P, _P, _P, _I64, _P, _P, _INT]
        f.restype = _INT
    L.oracle_stable_positions.argtypes = [_P, _INT, _I64, _P, _I64, _P, _INT]
    L.oracle_stable_positions.restype = _INT
    L.oracle_check_stable.argtypes = [_P, _P, _P, _INT, _INT, _I64, _INT]
    L.oracle_check_stable.restype = _I64
    L.oracle_check_sorted_keys.argtypes = [_P, _P, _INT, _I64, _INT]
    L.oracle_check_sorted_keys.restype = _I64
    L.oracle_splitmix64_next.argtypes = [ctypes.POINTER(_U64)]
    L.oracle_splitmix64_next.restype = _U64
    L.oracle_splitmix64_at.argtypes = [_U64, _U64]
    L.oracle_splitmix64_at.restype = _U64
    L.oracle_sample_stream.argtypes = [_U64, _I64, _I64, _INT]
    L.oracle_sample_stream.restype = _U64
    L.oracle_sample_positions.argtypes = [_U64, _I64, _I64, _INT, _I64, _P]
    L.oracle_sample_positions.restype = _INT
    L.oracle_heavy_from_sample.argtypes = [_P, _I64, _I64, _P, _P]
    L.oracle_heavy_from_sample.restype = _I64
    L.oracle_sample_heavy.argtypes = [_P, _INT, _U64, _I64, _I64, _INT, _I64,
                                      _I64, _P, _P]
    L.oracle_sample_heavy.restype = _I64
    L.oracle_zone_layout.argtypes = [_U64, _INT, _INT, ctypes.POINTER(_INT),
                                     ctypes.POINTER(_INT)]
    L.oracle_zone_layout.restype = None
    L.oracle_bucket_ids.argtypes = [_P, _I64, _U64, _INT, _INT, _P, _INT, _I64, _P]
    L.oracle_bucket_ids.restype = _I64
    L.oracle_dtmerge_u64.argtypes = [_P, _P, _I64, _I64, _P, _P, _P]
    L.oracle_dtmerge_u64.restype = _INT


def _ptr(a):
    return None if a is None else a.ctypes.data


def _kbytes(keys):
    if keys.dtype == np.uint32:
        return 4
    if keys.dtype == np.uint64:
        return 8
    raise TypeError("keys must be uint32 or uint64, got %s" % keys.dtype)


def default_threads():
    return lib().oracle_default_threads()


def stable_sort(keys, vals=None, nthreads=0):
    """Stable sort of (keys, vals) by unsigned key.  Returns new arrays."""
    keys = np.ascontiguousarray(keys)
    kb = _kbytes(keys)
    if vals is not None:
        vals = np.ascontiguousarray(vals)
        if vals.dtype.itemsize != kb or len(vals) != len(keys):
            raise ValueError("values must match keys in length and width")
    ok = np.empty_like(keys)
    ov = None if vals is None else np.empty_like(vals)
    f = lib().oracle_sort_u32 if kb == 4 else lib().oracle_sort_u64
    if f(_ptr(keys), _ptr(vals), len(keys), _ptr(ok), _ptr(ov), nthreads):
        raise MemoryError("oracle sort failed")
    return ok, ov


def stable_sort_segmented(keys, vals, offsets, nthreads=0):
    """Stable sort of every segment [offsets[s], offsets[s+1]) on its own."""
    keys = np.ascontiguousarray(keys)
    kb = _kbytes(keys)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    if vals is not None:
        vals = np.ascontiguousarray(vals)
    ok = np.empty_like(keys)
    ov = None if vals is None else np.empty_like(vals)
    f = (lib().oracle_sort_segmented_u32 if kb == 4
         else lib().oracle_sort_segmented_u64)
    if f(_ptr(keys), _ptr(vals), _ptr(offsets), len(offsets) - 1, _ptr(ok),
         _ptr(ov), nthreads):
        raise ValueError("oracle segmented sort failed")
    return ok, ov


def check_stable(keys_in, keys_out, idx_out, nthreads=0):
    """-1 if (keys_out, idx_out) is the stable sort of keys_in (idx_out[i] =
    original index of output record i), else the first failing output slot
    (len(keys_in) if some index is missing)."""
    keys_in = np.ascontiguousarray(keys_in)
    keys_out = np.ascontiguousarray(keys_out)
    idx_out = np.ascontiguousarray(idx_out)
    assert keys_in.dtype == keys_out.dtype and len(keys_in) == len(keys_out) == len(idx_out)
    assert idx_out.dtype.itemsize in (4, 8)
    return int(lib().oracle_check_stable(_ptr(keys_in), _ptr(keys_out), _ptr(idx_out),
                                         _kbytes(keys_in), idx_out.dtype.itemsize,
                                         len(keys_in), nthreads))


def check_sorted_keys(keys_in, keys_out, nthreads=0):
    """-1 if keys_out is the key-only sort of keys_in (the input's multiset of
    keys in non-decreasing order), else the first failing output slot."""
    keys_in = np.ascontiguousarray(keys_in)
    keys_out = np.ascontiguousarray(keys_out)
    assert keys_in.dtype == keys_out.dtype and len(keys_in) == len(keys_out)
    r = int(lib().oracle_check_sorted_keys(_ptr(keys_in), _ptr(keys_out), _kbytes(keys_in),
                                           len(keys_in), nthreads))
    if r == -2:
        raise MemoryError("oracle_check_sorted_keys: out of memory")
    return r


def stable_positions(keys, js, nthreads=0):
    """Stable-sorted output position of each input record js[q]."""
    keys = np.ascontiguousarray(keys)
    js = np.ascontiguousarray(js, dtype=np.int64)
    out = np.empty(len(js), dtype=np.int64)
    if lib().oracle_stable_positions(_ptr(keys), _kbytes(keys), len(keys),
                                     _ptr(js), len(js), _ptr(out), nthreads):
        raise ValueError("bad record index")
    return out


def splitmix64_sequence(seed, count):
    st = _U64(seed)
    return [lib().oracle_splitmix64_next(ctypes.byref(st)) for _ in range(count)]


def splitmix64_at(state, i):
    return lib().oracle_splitmix64_at(state, i)


def sample_stream(seed, start, size, hi):
    return lib().oracle_sample_stream(seed, start, size, hi)


def sample_positions(seed, start, size, hi, count):
    out = np.empty(count, dtype=np.int64)
    if lib().oracle_sample_positions(seed, start, size, hi, count, _ptr(out)):
        raise ValueError("bad sample request")
    return out


def heavy_from_sample(sample, L):
    """(heavy keys increasing as uint64, max sample) for a given sample."""
    s = np.ascontiguousarray(sample, dtype=np.uint64)
    out = np.empty(max(len(s), 1), dtype=np.uint64)
    mx = _U64(0)
    nh = lib().oracle_heavy_from_sample(_ptr(s), len(s), L, _ptr(out),
                                        ctypes.addressof(mx))
    return out[:nh].copy(), int(mx.value)


def sample_heavy(keys, seed, start, size, hi, count, L):
    keys = np.ascontiguousarray(keys)
    out = np.empty(max(count, 1), dtype=np.uint64)
    mx = _U64(0)
    nh = lib().oracle_sample_heavy(_ptr(keys), _kbytes(keys), seed, start, size,
                                   hi, count, L, _ptr(out), ctypes.addressof(mx))
    return out[:nh].copy(), int(mx.value)


def zone_layout(rmax, hi, gamma):
    t, lo = _INT(0), _INT(0)
    lib().oracle_zone_layout(rmax, hi, gamma, ctypes.byref(t), ctypes.byref(lo))
    return t.value, lo.value


def bucket_ids(heavy, rmax, hi, gamma, keys):
    """Bucket id of every key (Alg. 2 numbering); returns (ids, nbuckets)."""
    keys = np.ascontiguousarray(keys)
    h = np.ascontiguousarray(heavy, dtype=np.uint64)
    ids = np.empty(len(keys), dtype=np.int32)
    nb = lib().oracle_bucket_ids(_ptr(h), len(h), rmax, hi, gamma, _ptr(keys),
                                 _kbytes(keys), len(keys), _ptr(ids))
    if nb < 0:
        raise MemoryError
    return ids, int(nb)


def dtmerge(b0_keys, b0_vals, heavy_keys, heavy_sizes, heavy_vals=None):
    """Alg. 3 on one zone.  b0 sorted light records; heavy bucket i holds
    heavy_sizes[i] copies of heavy_keys[i] with values heavy_vals (concatenated).
    Returns (keys, vals, records copied out of place)."""
    b0k = np.asarray(b0_keys, dtype=np.uint64)
    hk = np.ascontiguousarray(heavy_keys, dtype=np.uint64)
    hs = np.ascontiguousarray(heavy_sizes, dtype=np.int64)
    keys = np.concatenate([b0k, np.repeat(hk, hs)]).astype(np.uint64)
    vals = None
    if b0_vals is not None:
        vals = np.concatenate([np.asarray(b0_vals, dtype=np.uint64),
                               np.asarray(heavy_vals, dtype=np.uint64)])
        vals = np.ascontiguousarray(vals)
    copied = _I64(0)
    if lib().oracle_dtmerge_u64(_ptr(keys), _ptr(vals), len(b0k), len(hk),
                                _ptr(hk), _ptr(hs), ctypes.addressof(copied)):
        raise MemoryError
    return keys, vals, int(copied.value)
