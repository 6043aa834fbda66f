"""GPU parity of pdd_interface_grad (Poisson-Fourier family) against the
oracle's derivative estimators on shared streams, plus the autograd wrapper.

theta part: exact pathwise derivative, must equal a common-random-number
difference of the forward solve.  phi part: likelihood-ratio sums per path,
compared path by path with the oracle (FP32 vs FP64 rounding), and node-level
Jacobians within 1e-5 of scale plus the reach of counted exit flips.
"""
import numpy as np
import pytest
import torch

from paper_1705_03666_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1705_03666_gb300 import api as a
    return a


def test_records_and_jacobian_match_oracle(api, orc):
    w = W.workload(5)
    nodes = w["nodes"][::128]
    kw = dict(seed=w["seed"], dt=1e-3, n_paths=1500)
    with api.Context(w["prob"]) as ctx:
        g = ctx.interface_grad(torch.from_numpy(nodes), dump_paths=True, **kw)
    J, Jse, rec, steps = orc.interface_jacobian(w["prob"], nodes, dump_paths=True, **kw)
    gs, gst, gaux = g["score"].cpu().numpy(), g["steps"].cpu().numpy(), g["aux"].cpu().numpy()
    matched = (gst == steps) & (np.abs(gs - rec[:, :, 0]) <= 1e-4 * np.maximum(1, np.abs(rec[:, :, 0])))
    flip = 1.0 - matched.mean()
    assert flip <= 2e-3
    # per-path exit points and likelihood-ratio sums on matched paths
    m = matched
    assert np.max(np.abs(gaux[m][:, 0] - rec[m][:, 1])) < 1e-5
    assert np.max(np.abs(gaux[m][:, 1] - rec[m][:, 2])) < 1e-5
    L_o = rec[m][:, 4:]
    assert np.max(np.abs(gaux[m][:, 2:] - L_o) / np.maximum(1.0, np.abs(L_o))) < 1e-4
    # node-level Jacobian: 1e-5 of the component scale plus what the flipped
    # paths can move (their fraction times the largest per-path value)
    Jg = g["jac"].cpu().numpy()
    nflip = (~matched).sum(1)[:, None] / matched.shape[1]
    vmax = np.maximum(1.0, np.abs(rec[:, :, :1]).max(1) * np.abs(rec[:, :, 4:]).max(1).max(1, keepdims=True))
    scale = np.maximum(np.abs(J), Jse)
    assert np.all(np.abs(Jg - J) <= 1e-5 * scale + 2.0 * nflip * vmax + 1e-7)
    np.testing.assert_allclose(g["jac_se"].cpu().numpy(), Jse, rtol=0.05, atol=1e-6)


def test_grad_paths_are_forward_paths(api):
    w = W.workload(5)
    nodes = torch.from_numpy(w["nodes"][::256])
    kw = dict(seed=w["seed"], dt=1e-3, n_paths=777)
    with api.Context(w["prob"]) as ctx:
        f = ctx.interface_solve(nodes, precision="fp32", dump_paths=True, **kw)
        g = ctx.interface_grad(nodes, dump_paths=True, **kw)
    assert torch.equal(f["steps"], g["steps"])
    assert torch.equal(f["score"], g["score"])


def test_theta_gradient_equals_crn_difference(api):
    w = W.workload(5)
    nodes = torch.from_numpy(w["nodes"][::64])
    kw = dict(seed=w["seed"], dt=1e-3, n_paths=2000)
    prob = w["prob"]
    with api.Context(prob) as ctx:
        J = ctx.interface_grad(nodes, **kw)["jac"].cpu().numpy()
        h = 0.25
        for k in (0, 9, 36, 63):
            pp, pm = prob["params"].copy(), prob["params"].copy()
            pp[k] += h
            pm[k] -= h
            ctx.set_params(pp)
            up = ctx.interface_solve(nodes, precision="fp32", **kw)["mean"].cpu().numpy()
            ctx.set_params(pm)
            um = ctx.interface_solve(nodes, precision="fp32", **kw)["mean"].cpu().numpy()
            np.testing.assert_allclose((up - um) / (2 * h), J[:, k], rtol=2e-4, atol=2e-6)
        ctx.set_params(prob["params"])


def test_autograd_vjp(api):
    w = W.workload(5)
    nodes = torch.from_numpy(w["nodes"][::32]).cuda()
    mc = dict(seed=w["seed"], dt=1e-3, n_paths=1000)
    prm = torch.from_numpy(w["prob"]["params"])
    theta = prm[:64].clone().requires_grad_(True)
    phi = prm[64:].clone().requires_grad_(True)
    with api.Context(w["prob"]) as ctx:
        u = api.interface_values(theta, phi, ctx, nodes, **mc)
        wgt = torch.linspace(-1.0, 1.0, u.numel(), dtype=torch.float64, device=u.device)
        (u * wgt).sum().backward()
        J = ctx.interface_grad(nodes, **mc)["jac"]
    ref = (wgt[:, None] * J).sum(0).cpu()
    np.testing.assert_allclose(theta.grad.numpy(), ref[:64].numpy(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(phi.grad.numpy(), ref[64:].numpy(), rtol=1e-10, atol=1e-12)
