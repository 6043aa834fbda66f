"""GPU checks of the 3-D stage two (Sec. 2.1, Fig. 2.2): the interface
interpolation on the cube's internal planes (pdd_interface_interp) and the
7-point elliptic subdomain solve (pdd_subdomain_solve with a 3-D grid),
against the FP64 oracle (SciPy's cubic RBF interpolant, a sparse direct solve
of the same finite-difference system) and the manufactured solution."""
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
    assert torch.cuda.is_available()
    return a


def _exact(x):
    x = np.asarray(x)
    return np.sin(np.pi * x[..., 0]) * np.sin(np.pi * x[..., 1]) * np.exp(x[..., 2])


def _plane_nodes(axis, pos):
    nodes = W.nodes_cube_planes(4096)
    sel = (np.arange(4096) % 3 == axis) & (nodes[:, axis] == pos)
    return nodes[sel]


def test_interface_interp_matches_oracle(api, orc):
    prob = W.elliptic_manufactured()
    rng = np.random.default_rng(5)
    planes, queries, ref = [], [], []
    for axis, pos in ((0, 0.25), (1, 0.5), (2, 0.75)):
        nd = _plane_nodes(axis, pos)
        v = _exact(nd) + 2e-3 * rng.standard_normal(len(nd))    # Monte Carlo-like noise
        q = rng.uniform(0, 1, (700, 3))
        q[:, axis] = pos
        planes.append((axis, pos, nd, v))
        queries.append(q)
        ref.append(orc.plane_interface(prob, axis, pos, nd, v, q, n_bnd=32))
    with api.Context(prob) as ctx:
        out = ctx.interface_interp(planes, queries, n_bnd=32)
    for o, r in zip(out, ref):
        np.testing.assert_allclose(o.cpu().numpy(), r, rtol=0, atol=1e-9)
    # at the nodes the interpolant returns the node values
    with api.Context(prob) as ctx:
        at = ctx.interface_interp([planes[0]], [planes[0][2]], n_bnd=32)[0].cpu().numpy()
    np.testing.assert_allclose(at, planes[0][3], atol=1e-9)


def _box_data(lo, hi, n, mask, rng):
    faces = {}
    for fc in range(6):
        if (mask >> fc) & 1:
            a = fc // 2
            o = [b for b in range(3) if b != a]
            faces[fc] = rng.uniform(-1, 1, (n[o[1]], n[o[0]]))
    return faces


def _oracle_box(orc, prob, lo, hi, n, faces):
    t = [np.linspace(lo[a], hi[a], n[a]) for a in range(3)]
    Z, Y, X = np.meshgrid(t[2], t[1], t[0], indexing="ij")
    ub = orc.eval_coeffs_many(prob, np.stack([X, Y, Z], -1).reshape(-1, 3))[:, 5].reshape(Z.shape)
    # interface faces (the first one in bit order wins on shared edges, and
    # a face without interface data wins over any interface face)
    phys = np.zeros(Z.shape, bool)
    for fc in range(6):
        a, side = fc // 2, fc % 2
        idx = [slice(None)] * 3
        idx[2 - a] = -1 if side else 0
        if fc not in faces:
            phys[tuple(idx)] = True
    for fc in sorted(faces, reverse=True):
        a, side = fc // 2, fc % 2
        idx = [slice(None)] * 3
        idx[2 - a] = -1 if side else 0
        sub = ub[tuple(idx)]
        keep = phys[tuple(idx)]
        sub[~keep] = faces[fc][~keep]
        ub[tuple(idx)] = sub
    return orc.elliptic_box_solve(prob, ub, lo, hi)


@pytest.mark.parametrize("n,mask", [((17, 17, 17), 0b010101), ((13, 17, 9), 0b111111),
                                    ((9, 9, 9), 0)])
def test_box_solve_matches_oracle(api, orc, n, mask):
    prob = W.elliptic_manufactured()
    rng = np.random.default_rng(int(mask) + n[0])
    lo, hi = (0.25, 0.5, 0.0), (0.5, 0.75, 0.25)
    faces = _box_data(lo, hi, n, mask, rng)
    ref = _oracle_box(orc, prob, lo, hi, n, faces)
    with api.Context(prob) as ctx:
        r = ctx.subdomain_solve3d(lo, hi, n, faces, method="dst", tol=1e-13)
    u = r["u"].cpu().numpy()
    print(f"3-D box {n} mask {mask:06b}: {r['iters']} corrections, relative residual "
          f"{r['resid']:.1e}, max |u - oracle| {np.abs(u - ref).max():.1e}")
    assert r["status"] == 0 and r["resid"] <= 1e-13 and r["iters"] <= 30
    np.testing.assert_allclose(u, ref, rtol=0, atol=1e-10 * max(1.0, np.abs(ref).max()))


def test_jacobi_matches_oracle_on_a_small_box(api, orc):
    prob = W.elliptic_manufactured()
    n = (9, 7, 11)
    lo, hi = (0.0, 0.25, 0.5), (0.25, 0.5, 0.75)
    faces = _box_data(lo, hi, n, 0b100001, np.random.default_rng(9))
    ref = _oracle_box(orc, prob, lo, hi, n, faces)
    with api.Context(prob) as ctx:
        r = ctx.subdomain_solve3d(lo, hi, n, faces, method="jacobi", tol=1e-15, max_iter=20000)
    assert r["status"] == 0
    np.testing.assert_allclose(r["u"].cpu().numpy(), ref, rtol=0, atol=1e-11)


def test_box_solve_second_order_to_the_manufactured_solution(api):
    """Exact face data on a subdomain of the 4x4x4 split: the solve converges
    to u at O(h^2) (17, 33, 65 points per axis)."""
    prob = W.elliptic_manufactured()
    lo, hi = (0.5, 0.25, 0.75), (0.75, 0.5, 1.0)
    errs = []
    with api.Context(prob) as ctx:
        for m in (17, 33, 65):
            t = [np.linspace(lo[a], hi[a], m) for a in range(3)]
            faces = {}
            for fc in (0, 1, 2, 3, 4):      # every face but z = 1 carries interface data
                a, side = fc // 2, fc % 2
                o = [b for b in range(3) if b != a]
                G1, G0 = np.meshgrid(t[o[1]], t[o[0]], indexing="ij")
                x = np.zeros(G0.shape + (3,))
                x[..., a] = hi[a] if side else lo[a]
                x[..., o[0]] = G0
                x[..., o[1]] = G1
                faces[fc] = _exact(x)
            r = ctx.subdomain_solve3d(lo, hi, (m, m, m), faces, tol=1e-13)
            Z, Y, X = np.meshgrid(t[2], t[1], t[0], indexing="ij")
            errs.append(np.abs(r["u"].cpu().numpy() - _exact(np.stack([X, Y, Z], -1))).max())
    print(f"3-D box errors against u: {errs}")
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


def test_two_stage_cube_with_exact_node_values(api):
    """The whole stage two on the 4x4x4 split (9 planes of the 4096-node
    recipe, 64 subdomains of 33^3 points, h = 1/128) with exact node values:
    what remains is the interpolation and discretisation error."""
    prob = W.elliptic_manufactured()
    nodes = W.nodes_cube_planes(4096)
    with api.Context(prob) as ctx:
        r = api.elliptic3d_pdd_solve(ctx, nodes, _exact(nodes), np.arange(4096) % 3)
    t = np.linspace(0, 1, 129)
    Z, Y, X = np.meshgrid(t, t, t, indexing="ij")
    err = np.abs(r["u"].cpu().numpy() - _exact(np.stack([X, Y, Z], -1))).max()
    print(f"two-stage cube, exact node values: max error {err:.2e}, {r['iters']} corrections")
    assert err < 2e-3 and r["resid"] <= 1e-12


def test_rejections(api):
    prob = W.elliptic_manufactured()
    from paper_1705_03666_gb300._lib import PDDError
    with api.Context(prob) as ctx:
        with pytest.raises(PDDError):   # too many points per axis
            ctx.subdomain_solve3d((0, 0, 0), (0.25, 0.25, 0.25), (129, 9, 9), {})
        with pytest.raises(PDDError):   # box outside the cube
            ctx.subdomain_solve3d((0.5, 0, 0), (1.5, 0.25, 0.25), (9, 9, 9), {})
        with pytest.raises(PDDError):   # wrong method for 3-D
            ctx.subdomain_solve3d((0, 0, 0), (0.25, 0.25, 0.25), (9, 9, 9), {}, method="cg")
        with pytest.raises(PDDError):   # a plane outside (0, 1)
            ctx.interface_interp([(0, 1.0, np.zeros((3, 3)), np.zeros(3))], [np.zeros((2, 3))])
    with api.Context(W.laplace_expcos()) as ctx:
        with pytest.raises(PDDError):   # 3-D grids need the 3-D family
            ctx.subdomain_solve3d((0, 0, 0), (0.25, 0.25, 0.25), (9, 9, 9), {})


@pytest.mark.parametrize("method,tol", [("dst", 1e-13), ("jacobi", 1e-13)])
def test_batch_equals_single_solves(api, method, tol):
    """pdd_subdomain_solve_batch: each box of a batch (own position, own
    interface mask) gets the bits of its own pdd_subdomain_solve, and the
    boxes stop at their own iteration counts."""
    prob = W.elliptic_manufactured()
    rng = np.random.default_rng(21)
    n = (11, 9, 13) if method == "dst" else (7, 7, 9)
    boxes = []
    for b, (mask, lo) in enumerate([(0b000000, (0.0, 0.0, 0.0)), (0b101010, (0.25, 0.5, 0.0)),
                                    (0b010101, (0.5, 0.25, 0.5)), (0b111111, (0.75, 0.75, 0.75))]):
        hi = tuple(v + 0.25 for v in lo)
        boxes.append((lo, hi, _box_data(lo, hi, n, mask, rng)))
    kw = dict(method=method, tol=tol, max_iter=20000 if method == "jacobi" else 200)
    with api.Context(prob) as ctx:
        rb = ctx.subdomain_solve3d_batch(boxes, n, **kw)
        singles = [ctx.subdomain_solve3d(lo, hi, n, faces, **kw) for lo, hi, faces in boxes]
    assert rb["status"] == 0
    for b, r in enumerate(singles):
        assert torch.equal(rb["u"][b], r["u"]), b
        assert rb["iters_each"][b] == r["iters"] and rb["resid_each"][b] == r["resid"]
    assert rb["iters"] == max(r["iters"] for r in singles)
    print(f"batch of 4 boxes ({method}): iterations {rb['iters_each']}")


def test_batch_rejections(api):
    import ctypes
    prob = W.elliptic_manufactured()
    from paper_1705_03666_gb300 import _lib
    with api.Context(prob) as ctx:
        boxes = [((0, 0, 0), (0.25, 0.25, 0.25), {}), ((0.25, 0, 0), (0.5, 0.25, 0.25), {})]
        r = ctx.subdomain_solve3d_batch(boxes, (9, 9, 9))
        assert r["status"] == 0 and r["u"].shape == (2, 9, 9, 9)
        with pytest.raises(_lib.PDDError):   # a box outside the cube
            ctx.subdomain_solve3d_batch([((0.5, 0, 0), (1.5, 0.25, 0.25), {})], (9, 9, 9))
        # two grid sizes, or two methods, in one batch (through the C ABI)
        u = torch.empty(2 * 11 * 11 * 11, dtype=torch.float64, device="cuda")
        for second in ((9, 9, 9, "dst"), (11, 11, 11, "jacobi")):
            sds = (_lib.Subdomain * 2)()
            for b, (nn, meth) in enumerate([((11, 11, 11), "dst"), (second[:3], second[3])]):
                sds[b] = _lib.Subdomain((ctypes.c_double * 3)(0.25 * b, 0, 0),
                                        (ctypes.c_double * 3)(0.25 * b + 0.25, 0.25, 0.25),
                                        (ctypes.c_int32 * 3)(*nn), 0, 0, _lib.STENCIL[meth],
                                        200, 1e-12)
            it, res = ctypes.c_int64(0), ctypes.c_double(0.0)
            st = ctx.lib.pdd_subdomain_solve_batch(ctx.handle, sds, 2, None, 0, u.data_ptr(),
                                                   ctypes.byref(it), ctypes.byref(res), None,
                                                   None)
            assert st == _lib.PDD_EINVAL
