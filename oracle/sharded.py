"""Oracle for the rank-local partition of the sharded sort.

TEST INFRASTRUCTURE ONLY: only tests/ may import this module.  It shares no
code with the CUDA path and never imports it.

The sharded sort cuts the array at splitters in the order of the pairs
(key, global index), which is the stable order of the whole array (Sec. 2.3
problem statement): range p of a shard holds, in index order, its records
with exactly p splitters at or below (key, global index).  Keys compare as
unsigned integers.  This is the distribution step of the paper's counting
sort (preliminaries, "Counting Sort") with one bucket per rank.
"""
import numpy as np


def range_of(keys, gidx, split_keys, split_gidx):
    """Range of every record: the number of splitters (sk, sg) with
    sk < key, or sk == key and sg <= gidx."""
    k = np.asarray(keys).astype(np.uint64)
    g = np.asarray(gidx, dtype=np.int64)
    d = np.zeros(len(k), dtype=np.int64)
    for sk, sg in zip(np.asarray(split_keys, dtype=np.uint64), np.asarray(split_gidx,
                                                                          dtype=np.int64)):
        d += (sk < k) | ((sk == k) & (sg <= g))
    return d


def partition(keys, values, gidx0, split_keys, split_gidx, parts):
    """(keys by range, values by range or None, range sizes): each range in
    index order."""
    keys = np.asarray(keys)
    gidx = gidx0 + np.arange(len(keys), dtype=np.int64)
    d = range_of(keys, gidx, split_keys, split_gidx)
    order = np.argsort(d, kind="stable")
    vals = None if values is None else np.asarray(values)[order]
    return keys[order], vals, np.bincount(d, minlength=parts).astype(np.int64)
