"""pdd_interface_solve_static: the interface solve for callers that cannot
allocate device memory (hosts whose memory pool owns the device, plug-ins
handed pre-allocated buffers, loops that cannot take an allocation's latency
or failure).

Called through the C ABI with caller-provided buffers; its output must match
pdd_interface_solve's on the same inputs, on two calls in a row (the static
scratch keeps the previous call's contents, so the second call checks that
everything that must start at zero is cleared), for every problem family it
takes, and the second call must leave the device's free memory unchanged.
This file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1705_03666_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1705_03666_gb300 import _lib
    return _lib


def _problem(lib, prob):
    params = np.ascontiguousarray(prob["params"] if prob["params"].size else np.zeros(1))
    p = lib.Problem(lib.PROBLEM[prob["problem"]], lib.GEOMETRY[prob["geometry"]],
                    int(prob["dim"]), int(prob["params"].size),
                    params.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(prob["sigma"]))
    return p, params


def _static_call(lib, prob, nodes, mc, out=None):
    cdll = lib.load()
    p, keep = _problem(lib, prob)
    n = nodes.shape[0]
    if out is None:
        out = (torch.empty(n, dtype=torch.float64, device="cuda"),
               torch.empty(n, dtype=torch.float64, device="cuda"),
               torch.empty(n, dtype=torch.int64, device="cuda"))
    mean, se, cnt = out
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = cdll.pdd_interface_solve_static(ctypes.byref(p), 0, stream, nodes.data_ptr(), n,
                                         ctypes.byref(mc), mean.data_ptr(), se.data_ptr(),
                                         cnt.data_ptr())
    torch.cuda.synchronize()
    return st, mean, se, cnt


CASES = [(2, "fp32", 16, 3001), (1, "fp64", 1, 2000), (5, "fp32", 32, 1500),
         (5, "fp64", 128, 500), (2, "fp64", 2, 2100), ("pf", "fp32", 1, 4000),
         ("pf", "fp64", 1, 1000)]


def _workload(k):
    if k == "pf":   # the random-coefficient Poisson family on workload 1's 16 square nodes
        w = dict(W.workload(1))
        w["prob"] = W.poisson_fourier(5)
        return w
    return W.workload(k)


@pytest.mark.parametrize("k,precision,stride,n_paths", CASES)
def test_static_matches_context_solve_twice(lib, k, precision, stride, n_paths):
    from paper_1705_03666_gb300 import api
    w = _workload(k)
    nodes = torch.from_numpy(np.ascontiguousarray(w["nodes"][::stride])).cuda()
    kw = dict(seed=w["seed"], dt=1e-3, n_paths=n_paths, precision=precision)
    with api.Context(w["prob"]) as ctx:
        ref = ctx.interface_solve(nodes, **kw)
        ref_mean, ref_se, ref_n = (t.cpu().numpy() for t in (ref["mean"], ref["se"], ref["n"]))
    mc = lib.MCParams(w["seed"], 1e-3, n_paths, 2**31 - 1, 0, lib.PRECISION[precision], 1)
    n = nodes.shape[0]
    out = (torch.empty(n, dtype=torch.float64, device="cuda"),
           torch.empty(n, dtype=torch.float64, device="cuda"),
           torch.empty(n, dtype=torch.int64, device="cuda"))
    for call in range(2):
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st, mean, se, cnt = _static_call(lib, w["prob"], nodes, mc, out)
        free_after = torch.cuda.mem_get_info()[0]
        assert st == lib.PDD_OK
        # the same exact per-node sums as the context solve: the same bits
        np.testing.assert_array_equal(mean.cpu().numpy(), ref_mean)
        np.testing.assert_array_equal(se.cpu().numpy(), ref_se)
        assert np.array_equal(cnt.cpu().numpy(), ref_n)
        if call == 1:
            assert free_after == free_before   # nothing allocated on the device


def test_static_node_offset_matches_context_solve(lib):
    from paper_1705_03666_gb300 import api
    w = W.workload(2)
    nodes = torch.from_numpy(np.ascontiguousarray(w["nodes"][100:140])).cuda()
    with api.Context(w["prob"]) as ctx:
        ref = ctx.interface_solve(nodes, seed=w["seed"], dt=1e-3, n_paths=800, node_offset=100)
    mc = lib.MCParams(w["seed"], 1e-3, 800, 2**31 - 1, 0, lib.PRECISION["fp32"], 1, 100)
    st, mean, se, cnt = _static_call(lib, w["prob"], nodes, mc)
    assert st == lib.PDD_OK
    assert torch.equal(mean, ref["mean"]) and torch.equal(se, ref["se"])


def test_static_rejects_too_many_nodes(lib):
    w = W.workload(2)
    nodes = torch.full((65537, 3), 0.5, dtype=torch.float64, device="cuda")
    mc = lib.MCParams(1, 1e-3, 1, 100, 0, 0, 1)
    st, *_ = _static_call(lib, w["prob"], nodes, mc)
    assert st == lib.PDD_EINVAL
