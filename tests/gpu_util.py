"""Helpers for the GPU tests: run the CUDA sort through the C-ABI on numpy
inputs and compare with the oracle."""
import numpy as np

import paper_2401_00710_gb300 as dts

_SIGNED = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64}


def to_dev(a, torch, dev):
    if a is None:
        return None
    a = np.ascontiguousarray(a)
    if a.dtype in _SIGNED:
        a = a.view(_SIGNED[a.dtype])
    return torch.from_numpy(a).to(dev)


def from_dev(t, dtype):
    if t is None:
        return None
    return t.cpu().numpy().view(dtype)


def op_of(keys, vals):
    if keys.dtype == np.uint32:
        return dts.DTSORT_OP_U32_KV if vals is not None else dts.DTSORT_OP_U32
    return dts.DTSORT_OP_U64_KV if vals is not None else dts.DTSORT_OP_U64


class GpuSort:
    """One handle + a growing workspace on cuda:0."""

    def __init__(self, torch):
        self.torch = torch
        self.dev = torch.device("cuda", 0)
        self.h = dts.dtsort_create(0)
        self.ws = None

    def close(self):
        dts.dtsort_destroy(self.h)

    def set_options(self, **kw):
        o = dts.dtsort_default_options()
        for k, v in kw.items():
            setattr(o, k, v)
        dts.dtsort_set_options(self.h, o)

    def reset_options(self):
        dts.dtsort_set_options(self.h, None)

    def workspace(self, op, n, nseg=1):
        need = dts.dtsort_workspace_bytes(self.h, op, n, nseg)
        if self.ws is None or self.ws.numel() < need:
            self.ws = None
            self.torch.cuda.empty_cache()
            self.ws = self.torch.empty(max(need, 256), dtype=self.torch.uint8,
                                       device=self.dev)
        return self.ws

    def launch(self, k, v, n, op, offsets=None, nseg=1):
        """Enqueue one sort of device tensors k (and v); returns the status."""
        ws = self.workspace(op, n, nseg)
        s = self.torch.cuda.current_stream(self.dev).cuda_stream
        kp = k.data_ptr() if k is not None and n > 0 else None
        vp = v.data_ptr() if v is not None and n > 0 else None
        wp, wb = ws.data_ptr(), ws.numel()
        if offsets is None:
            if op == dts.DTSORT_OP_U32:
                return dts.dtsort_u32(self.h, kp, n, wp, wb, s)
            if op == dts.DTSORT_OP_U32_KV:
                return dts.dtsort_u32_kv(self.h, kp, vp, n, wp, wb, s)
            if op == dts.DTSORT_OP_U64:
                return dts.dtsort_u64(self.h, kp, n, wp, wb, s)
            return dts.dtsort_u64_kv(self.h, kp, vp, n, wp, wb, s)
        op_ = offsets.data_ptr()
        if op == dts.DTSORT_OP_U32:
            return dts.dtsort_segmented_u32(self.h, kp, op_, nseg, n, wp, wb, s)
        if op == dts.DTSORT_OP_U32_KV:
            return dts.dtsort_segmented_u32_kv(self.h, kp, vp, op_, nseg, n, wp, wb, s)
        if op == dts.DTSORT_OP_U64:
            return dts.dtsort_segmented_u64(self.h, kp, op_, nseg, n, wp, wb, s)
        return dts.dtsort_segmented_u64_kv(self.h, kp, vp, op_, nseg, n, wp, wb, s)

    def device_status(self):
        s = self.torch.cuda.current_stream(self.dev).cuda_stream
        return dts.dtsort_last_device_error(self.h, s)

    def sort(self, keys, vals=None, offsets=None):
        """Sort numpy arrays on the GPU; returns (keys, vals) as numpy."""
        torch = self.torch
        n = len(keys)
        op = op_of(keys, vals)
        k = to_dev(keys, torch, self.dev)
        v = to_dev(vals, torch, self.dev)
        off = None
        nseg = 1
        if offsets is not None:
            off = torch.from_numpy(np.ascontiguousarray(offsets, dtype=np.int64)).to(self.dev)
            nseg = len(offsets) - 1
        st = self.launch(k, v, n, op, off, nseg)
        assert st == dts.DTSORT_OK, dts.status_string(st)
        dst = self.device_status()
        assert dst == dts.DTSORT_OK, dts.status_string(dst)
        return from_dev(k, keys.dtype), from_dev(v, keys.dtype)

    def stats(self):
        return dts.dtsort_get_stats(self.h).as_dict()


def assert_same(got_k, got_v, exp_k, exp_v):
    if not np.array_equal(got_k, exp_k):
        i = int(np.nonzero(got_k != exp_k)[0][0])
        raise AssertionError("keys differ first at %d: got %d expected %d (of %d)"
                             % (i, got_k[i], exp_k[i], len(exp_k)))
    if exp_v is not None and not np.array_equal(got_v, exp_v):
        i = int(np.nonzero(got_v != exp_v)[0][0])
        raise AssertionError("values differ first at %d: got %d expected %d (of %d)"
                             % (i, got_v[i], exp_v[i], len(exp_v)))
