"""GPU parity of pdd_interface_grad (Poisson-Fourier family) against the
oracle's derivative estimators on shared streams, plus the autograd wrapper.

theta part: exact pathwise derivative, must equal a common-random-number
difference of the forward solve.  phi part: likelihood-ratio sums per path,
compared path by path with the oracle: exit-step and exit-face flips counted
apart, every same-exit path's score and sums within their binary32 bounds,
and node-level Jacobians within 1e-5 of scale plus the reach of the counted
flips.
"""
import numpy as np
import pytest
import torch

from paper_1705_03666_gb300 import workloads as W
from tests import parity

pytestmark = pytest.mark.gpu

FLIP_MAX_FP32 = 2e-4
LR_FACTOR = 2.0  # bound on the sums' binary32 error, in units of 2^-22 (n + 8)(1 + |L|); measured 0.40


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
    # the forward part of each record (score, exit step, exit point): exit
    # flips counted apart, every same-exit path within its binary32 bound
    c = parity.compare_paths({"score": gs, "steps": gst, "exit": gaux[..., 0:2]},
                             {"score": rec[..., 0], "steps": steps, "exit": rec[..., 1:3]},
                             prob=w["prob"], geometry="unit_square")
    parity.check("poisson_fourier gradient records fp32", c, flip_max=FLIP_MAX_FP32)
    m = c["same"]
    # likelihood-ratio sums of the same-exit paths: each is a sum over the
    # path's n steps of a binary32 drift derivative times a normal, so it
    # carries the steps' rounding (n + 8) 2^-22 of its magnitude scale
    L_o = rec[m][:, 4:]
    n_m = np.abs(steps[m]).astype(np.float64)[:, None]
    lr_unit = 2.0 ** -22 * (n_m + 8.0) * (1.0 + np.abs(L_o).max(1, keepdims=True))
    lr_ratio = np.abs(gaux[m][:, 2:] - L_o) / lr_unit
    print(f"[parity] likelihood-ratio sums: max |dL| / (2^-22 (n + 8)(1 + |L|)) = "
          f"{lr_ratio.max():.3f}")
    assert lr_ratio.max() <= LR_FACTOR, lr_ratio.max()
    # node-level Jacobian.  A row is the mean over the node's paths of the
    # per-path contributions: cos(m pi x) cos(n pi y) at the exit point for
    # theta_{8m+n} (Y = 1 in this family), s L_j for phi_j.  The oracle's
    # rows are that mean of its records (checked to rounding); the kernel's
    # rows must be the mean of the contributions of its own records, up to
    # their binary32 evaluation (the records themselves are checked path by
    # path above), and lie within 1e-5 of the scale plus the mean per-path
    # difference of the contributions from the oracle's.
    def contrib(sc, xe, L):
        k = np.arange(8) * np.pi
        cx, cy = np.cos(xe[..., 0, None] * k), np.cos(xe[..., 1, None] * k)
        th = (cx[..., :, None] * cy[..., None, :]).reshape(cx.shape[:-1] + (64,))
        return np.concatenate([th, sc[..., None] * L], -1)
    c_o = contrib(rec[..., 0], rec[..., 1:3], rec[..., 4:])
    np.testing.assert_allclose(c_o.mean(1), J, rtol=1e-10, atol=1e-13)
    c_g = contrib(gs, gaux[..., 0:2], gaux[..., 2:])
    Jg = g["jac"].cpu().numpy()
    red_unit = 2.0 ** -20 * np.abs(c_g).mean(1) + 1e-12
    red_ratio = np.abs(Jg - c_g.mean(1)) / red_unit
    print(f"[parity] Jacobian rows against the mean of the kernel's own records: "
          f"{red_ratio.max():.3f} of 2^-20 mean |c|")
    assert red_ratio.max() <= 1.0, red_ratio.max()
    scale = np.maximum(np.abs(J), Jse)
    assert np.all(np.abs(Jg - J) <= 1e-5 * scale + np.abs(c_g - c_o).mean(1) + red_unit)
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


def _contributions(sc, xe, L):
    """Per-path contributions of the Poisson-Fourier Jacobian row: cos(m pi x)
    cos(n pi y) at the exit point for theta_{8m+n}, s L_j for phi_j."""
    k = np.arange(8) * np.pi
    cx, cy = np.cos(xe[..., 0, None] * k), np.cos(xe[..., 1, None] * k)
    th = (cx[..., :, None] * cy[..., None, :]).reshape(cx.shape[:-1] + (64,))
    return np.concatenate([th, sc[..., None] * L], -1)


def test_jacobian_reduction_in_parts(api):
    # 40 000 paths per node: each node's records are reduced in four parts
    # and merged in part order; with a wave of 50 000 paths the nodes also
    # straddle waves.  Either way a row is the mean of the kernel's own
    # records' contributions (to 2^-20 of their mean magnitude, the binary32
    # evaluation) and its standard error theirs.
    w = W.workload(5)
    nodes = torch.from_numpy(w["nodes"][::700])
    kw = dict(seed=w["seed"], dt=1e-3, n_paths=40000)
    rows = []
    with api.Context(w["prob"]) as ctx:
        for wave in (0, 8 * 50000):
            ctx.set_tuning(0, wave)
            g = ctx.interface_grad(nodes, dump_paths=True, **kw)
            aux = g["aux"].cpu().numpy()
            c = _contributions(g["score"].cpu().numpy(), aux[..., 0:2], aux[..., 2:])
            J = g["jac"].cpu().numpy()
            unit = 2.0 ** -20 * np.abs(c).mean(1) + 1e-12
            ratio = np.abs(J - c.mean(1)) / unit
            print(f"[parity] Jacobian in parts (wave {wave or 'default'}): "
                  f"{ratio.max():.3f} of 2^-20 mean |c|")
            assert ratio.max() <= 1.0, ratio.max()
            se = c.std(1, ddof=1) / np.sqrt(c.shape[1])
            np.testing.assert_allclose(g["jac_se"].cpu().numpy(), se, rtol=1e-3, atol=1e-12)
            rows.append((J, unit))
        ctx.set_tuning(0, 0)
    # the same paths either way (records are per path), so the two rows are
    # within both reductions' bounds of each other
    assert np.all(np.abs(rows[0][0] - rows[1][0]) <= rows[0][1] + rows[1][1])
