"""The allocation-free entry point dtsort_u32_kv_noalloc.

It exists for callers that may not allocate device memory when they sort:
plugin or callback code handed a stream by a host framework that owns all
device memory, or real-time pipelines that forbid allocation after start-up.
Its temporaries live in a static device array inside the library.  Here it
must give exactly what the regular entry point dtsort_u32_kv gives, and what
the CPU oracle gives, on two calls in a row (the static array keeps the
previous call's contents), and refuse sizes above its maximum.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2401_00710_gb300 as dts  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dts.build()
    return torch.device("cuda", 0)


def _regular(keys, vals, dev):
    """The existing entry point dtsort_u32_kv with a caller workspace."""
    h = dts.dtsort_create(0)
    try:
        n = len(keys)
        k = torch.from_numpy(keys.view(np.int32)).to(dev)
        v = torch.from_numpy(vals.view(np.int32)).to(dev)
        wsb = dts.dtsort_workspace_bytes(h, dts.DTSORT_OP_U32_KV, n)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        s = torch.cuda.current_stream(dev).cuda_stream
        assert dts.dtsort_u32_kv(h, k.data_ptr(), v.data_ptr(), n, ws.data_ptr(), wsb,
                                 s) == dts.DTSORT_OK
        assert dts.dtsort_last_device_error(h, s) == dts.DTSORT_OK
        return k.cpu().numpy().view(np.uint32), v.cpu().numpy().view(np.uint32)
    finally:
        dts.dtsort_destroy(h)


def _noalloc(keys, vals, dev):
    n = len(keys)
    k = torch.from_numpy(keys.view(np.int32)).to(dev)
    v = torch.from_numpy(vals.view(np.int32)).to(dev)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    s = torch.cuda.current_stream(dev).cuda_stream
    st = dts.dtsort_u32_kv_noalloc(k.data_ptr(), v.data_ptr(), n, status.data_ptr(), s)
    assert st == dts.DTSORT_OK, dts.status_string(st)
    torch.cuda.synchronize(dev)
    assert int(status.item()) == 0
    return k.cpu().numpy().view(np.uint32), v.cpu().numpy().view(np.uint32)


def test_noalloc_matches_regular_entry_point_and_oracle_twice(dev):
    cases = [("zipf1.2", dts.DTSORT_NOALLOC_MAX_N, 3),
             ("uniform", 777_777, 4)]
    for name, n, seed in cases:  # two calls in a row share the static array
        keys = gen.family(name, n, np.uint32, seed=seed)
        vals = gen.iota(n, np.uint32)
        rk, rv = _regular(keys, vals, dev)
        nk, nv = _noalloc(keys, vals, dev)
        np.testing.assert_array_equal(nk, rk)
        np.testing.assert_array_equal(nv, rv)
        ek, ev = oracle.stable_sort(keys, vals)
        np.testing.assert_array_equal(nk, ek)
        np.testing.assert_array_equal(nv, ev)


def test_noalloc_refuses_sizes_above_its_maximum(dev):
    n = dts.DTSORT_NOALLOC_MAX_N + 1
    k = torch.zeros(n, dtype=torch.int32, device=dev)
    v = torch.zeros(n, dtype=torch.int32, device=dev)
    st = dts.dtsort_u32_kv_noalloc(k.data_ptr(), v.data_ptr(), n, None, 0)
    assert st == dts.DTSORT_ERR_INVALID_ARG
    assert dts.dtsort_u32_kv_noalloc(k.data_ptr(), v.data_ptr(), 0, None, 0) == dts.DTSORT_OK
