"""Seeded synthetic inputs for the stable integer sort.

Shared by the oracle side and the CUDA side (tests, smoke check, benchmark);
holds none of the sort's arithmetic.  Values are a pure function of
(seed, record index) -- see ``gen.c`` for the families -- so every input is
reproducible on any machine and with any thread count.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_SO = os.path.join(_HERE, "_build", "libgen.so")
_lib = None

UNIFORM, ZIPF, ZIPF_HASHED, EXP, BITEXP, DISTINCT, HEAVYMIX, SKEWMIX, \
    BEXP_PAPER, UNIF_MU, EDGES = range(11)
EDGE_VERTICES = 1 << 26  # power-law edge lists: 2^26 vertices


def build(force=False):
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                           "-pthread", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.gen_keys.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                               ctypes.c_double, ctypes.c_uint64, ctypes.c_int64,
                               ctypes.c_int64, ctypes.c_void_p, ctypes.c_int]
        L.gen_keys.restype = ctypes.c_int
        L.gen_iota.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                               ctypes.c_void_p]
        L.gen_iota.restype = ctypes.c_int
        L.gen_rng.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        L.gen_rng.restype = ctypes.c_uint64
        L.gen_segment_sizes.argtypes = [ctypes.c_uint64, ctypes.c_int64,
                                        ctypes.c_double, ctypes.c_double,
                                        ctypes.c_void_p, ctypes.c_void_p]
        L.gen_segment_sizes.restype = ctypes.c_int
        L.gen_edge_src.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
        L.gen_edge_src.restype = ctypes.c_int
        _lib = L
    return _lib


def fill_keys(out_ptr, n, kind, kbytes, seed, p1=0.0, p2=0.0, first=0,
              nthreads=0):
    """Write n keys of the family into host memory at out_ptr."""
    if lib().gen_keys(kind, kbytes, float(p1), float(p2), seed, first, n,
                      out_ptr, nthreads):
        raise ValueError("bad generator request")


def keys(n, kind, dtype=np.uint32, seed=1, p1=0.0, p2=0.0, first=0,
         nthreads=0):
    dtype = np.dtype(dtype)
    out = np.empty(n, dtype=dtype)
    fill_keys(out.ctypes.data, n, kind, dtype.itemsize, seed, p1, p2, first,
              nthreads)
    return out


def iota(n, dtype=np.uint32, first=0):
    dtype = np.dtype(dtype)
    out = np.empty(n, dtype=dtype)
    lib().gen_iota(dtype.itemsize, first, n, out.ctypes.data)
    return out


def fill_iota(out_ptr, n, vbytes, first=0):
    lib().gen_iota(vbytes, first, n, out_ptr)


def fill_edge_src(out_ptr, n, vbytes, E=None, V=EDGE_VERTICES, first=0):
    """Sources of edges [first, first+n) of a list of E (default n) edges over
    V vertices ordered by source: src_i = floor(i V / E)."""
    if lib().gen_edge_src(vbytes, first, n, n if E is None else E, V, out_ptr):
        raise ValueError("bad edge-list request")


def edge_src(n, dtype=np.uint32, E=None, V=EDGE_VERTICES, first=0):
    dtype = np.dtype(dtype)
    out = np.empty(n, dtype=dtype)
    fill_edge_src(out.ctypes.data, n, dtype.itemsize, E, V, first)
    return out


def rng(seed, stream, i):
    return lib().gen_rng(seed, stream, i)


def segment_sizes(nseg, lo, hi, seed=1):
    sizes = np.empty(nseg, dtype=np.int64)
    fam = np.empty(nseg, dtype=np.int32)
    lib().gen_segment_sizes(seed, nseg, float(lo), float(hi), sizes.ctypes.data,
                            fam.ctypes.data)
    return sizes, fam


# ---- the benchmark configurations ------------------------------------------
# (name -> (kind, key dtype, p1, p2)); N = 1e9 universe for Zipf families.
U32_FAMILIES = {
    "uniform": (UNIFORM, np.uint32, 0.0, 0.0),
    "zipf0.8": (ZIPF, np.uint32, 0.8, 1e9),
    "zipf1.0": (ZIPF, np.uint32, 1.0, 1e9),
    "zipf1.2": (ZIPF, np.uint32, 1.2, 1e9),
    "zipf1.5": (ZIPF, np.uint32, 1.5, 1e9),
    "zipf1.2hash": (ZIPF_HASHED, np.uint32, 1.2, 1e9),
    "exp": (EXP, np.uint32, None, 0.0),       # rate = 10 / n, filled per n
    "bitexp": (BITEXP, np.uint32, 0.0, 0.0),
    "distinct10": (DISTINCT, np.uint32, 10, 0.0),
    "bexp30": (BEXP_PAPER, np.uint32, 30, 0.0),
    "unif1e3": (UNIF_MU, np.uint32, 1e3, 0.0),
    # graph transpose: destinations of a power-law edge list (in-degree
    # Zipf 1.0 over 2^26 vertices); the values are the edges' sources
    "edges": (EDGES, np.uint32, 1.0, float(EDGE_VERTICES)),
}
U64_FAMILIES = {
    "uniform": (UNIFORM, np.uint64, 0.0, 0.0),
    "zipf1.2hash": (ZIPF_HASHED, np.uint64, 1.2, 1e9),
    "heavymix": (HEAVYMIX, np.uint64, 0.5, 100),
    "skewmix": (SKEWMIX, np.uint64, 0.0, 0.0),
    "bitexp": (BITEXP, np.uint64, 0.0, 0.0),
}


def family(name, n, dtype=np.uint32, seed=1, nthreads=0):
    table = U32_FAMILIES if np.dtype(dtype) == np.uint32 else U64_FAMILIES
    kind, dt, p1, p2 = table[name]
    if p1 is None:
        p1 = 10.0 / max(n, 1)
    return keys(n, kind, dt, seed, p1, p2, nthreads=nthreads)


def fill_family(name, out_ptr, n, dtype=np.uint32, seed=1, nthreads=0):
    table = U32_FAMILIES if np.dtype(dtype) == np.uint32 else U64_FAMILIES
    kind, dt, p1, p2 = table[name]
    if p1 is None:
        p1 = 10.0 / max(n, 1)
    fill_keys(out_ptr, n, kind, np.dtype(dt).itemsize, seed, p1, p2,
              nthreads=nthreads)


# ---- the batched segmented configuration ------------------------------------
def segmented_layout(nseg=4096, lo=100.0, hi=1e7, seed=1, total=None):
    """Sizes log-uniform in [lo, hi] (seeded), one family flag per array
    (0 uniform, 1 Zipf s=1.0 over 10^9) with probability 1/2.  With `total`,
    sizes are scaled so that they sum to about `total` (each at least lo).
    Returns (offsets int64[nseg+1], family int32[nseg])."""
    sizes, fam = segment_sizes(nseg, lo, hi, seed)
    if total is not None:
        sizes = np.maximum(np.floor(sizes * (float(total) / sizes.sum())), lo).astype(np.int64)
    off = np.zeros(nseg + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    return off, fam


def fill_segmented_u32(keys_ptr, vals_ptr, offsets, family, seed=1, nthreads=0,
                       first_segment=0, last_segment=None):
    """Keys of array s: uniform u32 or Zipf(1.0) ranks - 1, from the stream
    seeded with seed*65536 + s; values: index within the array.  With
    first_segment / last_segment only arrays [first, last) are filled, and
    keys_ptr / vals_ptr point at the first one's first record."""
    if last_segment is None:
        last_segment = len(offsets) - 1
    a0 = int(offsets[first_segment])
    for s in range(first_segment, last_segment):
        a, b = int(offsets[s]) - a0, int(offsets[s + 1]) - a0
        if b <= a:
            continue
        if family[s]:
            kind, p1, p2 = ZIPF, 1.0, 1e9
        else:
            kind, p1, p2 = UNIFORM, 0.0, 0.0
        fill_keys(keys_ptr + 4 * a, b - a, kind, 4, seed * 65536 + s, p1, p2,
                  nthreads=nthreads if b - a > (1 << 16) else 1)
        if vals_ptr is not None:
            lib().gen_iota(4, 0, b - a, vals_ptr + 4 * a)
