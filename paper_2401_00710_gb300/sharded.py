"""Stable sort of one array sharded over several GPUs, with one exchange.

Rank r of a torch.distributed group holds a contiguous, index-ordered shard
of the array (global records [gidx0_r, gidx0_r + n_r), gidx0_r = the sizes of
the lower ranks).  ``sharded_sort`` runs the steps that include/dtsort.h
describes under "sorting an array sharded over several GPUs":

1. every rank samples (key, global index) pairs of its shard
   (``dtsort_shard_sample``), and the samples are gathered on every rank;
2. P-1 splitters are picked from the gathered sample (``dtsort_shard_splitters``,
   host code; every rank computes the same ones);
3. every rank partitions its shard stably into P ranges by (key, global
   index) (``dtsort_shard_partition``);
4. one all-to-all sends range p to rank p; the runs arrive in source-rank
   order, i.e. in global index order;
5. rank p sorts its runs with the single-GPU stable sort and then holds the
   p-th consecutive part of the sorted array.

The stable order of the whole array is the order of the pairs (key, global
index) (the problem statement of Sec. 2.3), so the ranges are consecutive
pieces of it and the result is the stable sort.  A key duplicated across a
splitter is split by global index, which keeps the ranges balanced.

Only collectives and argument marshalling happen here; the rank-local steps
are the ``ops`` object's: ``GpuShardOps`` calls the library's kernels on the
rank's GPU (the collectives then go through NCCL).  Tests on CPU ranks (gloo)
pass an object with the same four methods.
"""
import numpy as np

from . import (DTSORT_OK, DtsortError, Sorter, dtsort_shard_partition,
               dtsort_shard_partition_workspace_bytes, dtsort_shard_sample,
               dtsort_shard_splitters, status_string)

# samples per rank per range: enough that the ranges come out within a few
# percent of n / P
SAMPLES_PER_PART = 1024


def pick_splitters(sample_keys, sample_gidx, parts):
    """Host: P-1 splitters (uint64 keys, int64 global indices) from the
    gathered sample, through the library's host routine."""
    sk = np.ascontiguousarray(sample_keys, dtype=np.uint64)
    sg = np.ascontiguousarray(sample_gidx, dtype=np.int64)
    out_k = np.zeros(max(parts - 1, 1), dtype=np.uint64)
    out_g = np.zeros(max(parts - 1, 1), dtype=np.int64)
    st = dtsort_shard_splitters(sk.ctypes.data if len(sk) else None,
                                sg.ctypes.data if len(sg) else None, len(sk), parts,
                                out_k.ctypes.data, out_g.ctypes.data)
    if st != DTSORT_OK:
        raise DtsortError(st, "dtsort_shard_splitters")
    return out_k[:parts - 1].copy(), out_g[:parts - 1].copy()


class GpuShardOps:
    """The rank-local steps on this rank's GPU, through the C-ABI."""

    def __init__(self, device, sorter=None):
        import torch
        self.torch = torch
        self.device = device
        self.sorter = sorter or Sorter(device)

    def _stream(self):
        return self.torch.cuda.current_stream(self.device).cuda_stream

    def sample(self, keys, gidx0, count, seed):
        torch = self.torch
        sk = torch.empty(count, dtype=torch.int64, device=self.device)
        sg = torch.empty(count, dtype=torch.int64, device=self.device)
        if count:
            st = dtsort_shard_sample(keys.data_ptr(), keys.element_size(), keys.numel(), gidx0,
                                     seed, count, sk.data_ptr(), sg.data_ptr(), self._stream())
            if st != DTSORT_OK:
                raise DtsortError(st, "dtsort_shard_sample")
        return sk, sg

    def splitters(self, sample_keys, sample_gidx, parts):
        return pick_splitters(sample_keys, sample_gidx, parts)

    def partition(self, keys, values, gidx0, split_keys, split_gidx, parts):
        """Returns (keys by range, values by range, host list of range sizes)."""
        torch = self.torch
        n = keys.numel()
        ok = torch.empty_like(keys)
        ov = torch.empty_like(values) if values is not None else None
        counts = torch.zeros(parts, dtype=torch.int64, device=self.device)
        status = torch.zeros(1, dtype=torch.int32, device=self.device)
        wsb = dtsort_shard_partition_workspace_bytes(n, parts)
        ws = torch.empty(wsb, dtype=torch.uint8, device=self.device)
        skd = torch.from_numpy(np.asarray(split_keys, dtype=np.uint64).view(np.int64)).to(
            self.device)
        sgd = torch.from_numpy(np.asarray(split_gidx, dtype=np.int64)).to(self.device)
        st = dtsort_shard_partition(
            keys.data_ptr() if n else None, values.data_ptr() if values is not None and n else None,
            keys.element_size(), n, gidx0, skd.data_ptr() if parts > 1 else None,
            sgd.data_ptr() if parts > 1 else None, parts, ok.data_ptr() if n else None,
            ov.data_ptr() if ov is not None and n else None, counts.data_ptr(),
            ws.data_ptr(), wsb, status.data_ptr(), self._stream())
        if st != DTSORT_OK:
            raise DtsortError(st, "dtsort_shard_partition")
        dst = int(status.item())  # synchronises the stream
        if dst != DTSORT_OK:
            raise DtsortError(dst, "dtsort_shard_partition (device)")
        return ok, ov, [int(c) for c in counts.cpu().tolist()]

    def sort(self, keys, values):
        if keys.numel():
            self.sorter.sort_(keys, values)
            st = self.sorter.last_device_error()
            if st != DTSORT_OK:
                raise RuntimeError("sort: " + status_string(st))
        return keys, values


def _all_gather_int64(torch, dist, group, values, device):
    """All ranks' int64 vectors of equal length, stacked (world x len)."""
    t = torch.as_tensor(values, dtype=torch.int64).to(device)
    out = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(out, t, group=group)
    return torch.stack(out).cpu().numpy()


def sharded_sort(keys, values, ops, group=None, seed=1, samples_per_part=SAMPLES_PER_PART):
    """Stable sort of the array whose shard this rank holds (keys, values:
    1-D tensors on the ops' device, values None for key-only; 32-bit keys as
    int32 bit patterns, 64-bit as int64, compared as unsigned).

    Returns a dict: "keys"/"values" = this rank's part of the sorted array,
    "offset" = its first global position, "n" = the array's length,
    "sizes" = every rank's part size, "sent" = records this rank sent to each
    rank."""
    import torch
    import torch.distributed as dist

    P = dist.get_world_size(group)
    r = dist.get_rank(group)
    dev = keys.device
    n_local = keys.numel()
    sizes = _all_gather_int64(torch, dist, group, [n_local], dev)[:, 0]
    gidx0 = int(sizes[:r].sum())
    n = int(sizes.sum())
    # 1. samples in proportion to the shard sizes, gathered everywhere
    total = samples_per_part * P
    counts = [0 if n == 0 else int(-(-total * int(s) // n)) for s in sizes]
    sk, sg = ops.sample(keys, gidx0, counts[r], seed)
    smax = max(counts) if counts else 0
    pad_k = torch.zeros(smax, dtype=torch.int64, device=dev)
    pad_g = torch.zeros(smax, dtype=torch.int64, device=dev)
    pad_k[:counts[r]] = sk
    pad_g[:counts[r]] = sg
    gk = [torch.empty_like(pad_k) for _ in range(P)]
    gg = [torch.empty_like(pad_g) for _ in range(P)]
    dist.all_gather(gk, pad_k, group=group)
    dist.all_gather(gg, pad_g, group=group)
    all_k = np.concatenate([gk[q][:counts[q]].cpu().numpy() for q in range(P)]).view(np.uint64)
    all_g = np.concatenate([gg[q][:counts[q]].cpu().numpy() for q in range(P)])
    # 2. splitters (identical on every rank)
    split_k, split_g = ops.splitters(all_k, all_g, P)
    # 3. stable partition of the shard into P ranges
    pk, pv, send = ops.partition(keys, values, gidx0, split_k, split_g, P)
    # 4. one exchange: the range sizes, then the records
    recv = torch.empty(P, dtype=torch.int64, device=dev)
    dist.all_to_all_single(recv, torch.as_tensor(send, dtype=torch.int64).to(dev),
                           group=group)
    recv = [int(x) for x in recv.cpu().tolist()]
    rk = torch.empty(sum(recv), dtype=keys.dtype, device=dev)
    dist.all_to_all_single(rk, pk, recv, send, group=group)
    rv = None
    if values is not None:
        rv = torch.empty(sum(recv), dtype=values.dtype, device=dev)
        dist.all_to_all_single(rv, pv, recv, send, group=group)
    # 5. the runs are in global index order: one stable sort finishes the part
    rk, rv = ops.sort(rk, rv)
    part = _all_gather_int64(torch, dist, group, [rk.numel()], dev)[:, 0]
    return {"keys": rk, "values": rv, "offset": int(part[:r].sum()), "n": n,
            "sizes": [int(x) for x in part], "sent": send}
