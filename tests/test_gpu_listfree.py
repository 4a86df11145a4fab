"""The list-free near-pair correction (Sec. 3.3 step 4, Eq. er, recomputed by
every apply from the region's points and box moments instead of read from a
stored list) against the FP64 oracle, through the C ABI.  A list-free box
sums its pairs with the region's boxes that have moments; its pairs with the
other boxes stay in its points' stored rows.

The oracle computes the correction pair by pair (oracle.pim.correction_values);
the list-free kernels sum the same terms regrouped per observer box, so the
bars are the method's: relative L2 <= 1e-12 for FP64 plans, <= 2e-5 for FP32
plans.  `listfree=1` makes every box list-free; larger thresholds split the
boxes between the two forms."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import pim as opim  # noqa: E402
from paper_2312_02376_gb300 import inputs, pim  # noqa: E402

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


# name: (D, pdims, k, k0, n, N, b, nf, pf, p, layers)
CASES = {
    "helmholtz3d_bloch": ((1, 1, 1), (0, 1, 2), 2 * np.pi * 0.7, (0.9, 0.9, 0.0), (13, 13, 13), 500, 4, (8, 8, 8), 3, 4,
                          1),
    "helmholtz2d_bloch": ((1, 1, 0.5), (0, 1), 2 * np.pi * 0.8, (1.5, 0.5, 0.0), (17, 17, 9), 700, 4, (10, 10, 6), 4,
                          4, 1),
    "helmholtz1d_z": ((1, 0.5, 0.5), (2,), 2 * np.pi * 0.5, (0, 0, 0.0), (9, 9, 17), 500, 3, (6, 6, 10), 3, 4, 1),
    "helmholtz1d_x_two_layers": ((1, 0.5, 0.5), (0,), 3.0, (1.2, 0, 0), (17, 9, 9), 400, 3, (10, 6, 6), 3, 4, 2),
    "npsp3d": ((1, 1, 1), (0, 1, 2), 0.0, (0, 0, 0), (13, 13, 13), 600, 4, (8, 8, 8), 4, 4, 1),
    "static_phase3d": ((1, 1, 1), (0, 1, 2), 0.0, (1.0, 0.4, 0.3), (13, 13, 13), 400, 4, (8, 8, 8), 4, 4, 1),
    "free_space": ((1, 1, 0.5), (), 4.0, (0, 0, 0), (17, 17, 9), 600, 4, (10, 10, 10), 4, 4, 1),
    "odd_p3_bloch": ((1, 1, 0.5), (0, 1), 5.0, (0.7, -0.3, 0.0), (15, 15, 9), 500, 3, (8, 8, 6), 3, 3, 1),
    "p2_helmholtz3d": ((1, 1, 1), (0, 1, 2), 3.0, (0.5, 0.0, 0.2), (11, 11, 11), 400, 2, (8, 8, 8), 2, 2, 1),
}


def make_case(name, seed=0):
    """Half the points uniform, half in three tight clusters: boxes with
    moments (which the list-free kernels sum) and boxes without (whose pairs
    stay in the stored rows)."""
    D, pdims, k, k0, n, N, b, nf, pf, p, layers = CASES[name]
    npsp = len(pdims) > 0 and k == 0 and not any(k0)
    real = k == 0 and not any(k0)
    return inputs.random_clustered_case(N, D, pdims, k, k0, n, p=p, layers=layers, b=b, nf=nf, pf=pf,
                                        seed=seed + 11, complex_q=not real, neutral=npsp)


def oracle_plan(W):
    P = opim.Params(D=W.D, pdims=W.pdims, k=W.k, k0=W.k0, n=W.n, p=W.p, layers=W.layers, b=W.b, nf=W.nf, pf=W.pf)
    return opim.Plan(P, W.points)


def gpu_plan(W, precision, **kw):
    pl = pim.Plan(W.D, W.pdims, W.k, W.k0, W.n, p=W.p, layers=W.layers, precision=precision, b=W.b, nf=W.nf,
                  pf=W.pf, **kw)
    pl.set_points(torch.tensor(W.points, dtype=torch.float64, device="cuda"))
    return pl


def to_dev(x, precision, real):
    if real:
        return torch.tensor(np.real(x), dtype=torch.float64 if precision == "fp64" else torch.float32, device="cuda")
    return torch.tensor(x, dtype=torch.complex128 if precision == "fp64" else torch.complex64, device="cuda")


def is_real(W):
    return W.k == 0 and not any(W.k0)


@pytest.fixture(scope="module")
def cache():
    return {}


def oracle_results(name, cache):
    if name not in cache:
        W = make_case(name)
        o = oracle_plan(W)
        cache[name] = (W, o.apply(W.q), o.apply_adjoint(W.q))
    return cache[name]


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_every_box_listfree(name, cache):
    W, ue, we = oracle_results(name, cache)
    pl = gpu_plan(W, "fp64", listfree=1)
    info = pl.info()
    assert info.lf_points == W.N and info.lf_pairs > 0, (info.lf_points, info.lf_pairs)
    q = to_dev(W.q, "fp64", is_real(W))
    u = pl.apply(q).cpu().numpy()
    w = pl.apply_adjoint(q).cpu().numpy()
    assert pl.device_status() == pim.PIM_OK
    assert rel(u, ue) < FP64_TOL, rel(u, ue)
    assert rel(w, we) < FP64_TOL, rel(w, we)
    pl.close()


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_every_box_listfree(name, cache):
    W, ue, we = oracle_results(name, cache)
    pl = gpu_plan(W, "fp32", listfree=1)
    assert pl.info().lf_pairs > 0
    q = to_dev(W.q, "fp32", is_real(W))
    u = pl.apply(q).cpu().numpy()
    w = pl.apply_adjoint(q).cpu().numpy()
    assert pl.device_status() == pim.PIM_OK
    assert rel(u, ue) < FP32_TOL, rel(u, ue)
    assert rel(w, we) < FP32_TOL, rel(w, we)
    pl.close()


def clustered_case(seed=5, N=1500):
    """3D Helmholtz with a Bloch phase: a third of the points uniform, the rest
    in three tight clusters (some boxes with tens of points), the shape of the
    sphere-surface workload at a size the oracle finishes in seconds."""
    rng = np.random.default_rng(seed)
    D = np.array([1.0, 1.0, 1.0])
    nu = N // 3
    cl = [np.clip(c + 0.015 * rng.standard_normal(((N - nu) // 3, 3)), 0.0, 1.0)
          for c in (np.array([0.3, 0.4, 0.5]), np.array([0.7, 0.2, 0.8]), np.array([0.02, 0.5, 0.97]))]
    pts = np.concatenate([rng.random((nu, 3))] + cl)
    q = (rng.standard_normal(len(pts)) + 1j * rng.standard_normal(len(pts))) * np.sqrt(0.5)
    k = 2 * np.pi * 1.2
    return inputs.Workload("clusters", tuple(D), (0, 1, 2), k, (0.3 * k, -0.2 * k, 0.1 * k), (21, 21, 21), 4, 1, 4,
                           (9, 9, 9), 4, "fp64", len(pts), 1, pts, q)


@pytest.fixture(scope="module")
def clusters():
    W = clustered_case()
    o = oracle_plan(W)
    return W, o.apply(W.q), o.apply_adjoint(W.q)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_clusters_split_between_stored_and_listfree(precision, clusters):
    W, ue, we = clusters
    pl = gpu_plan(W, precision, listfree=3000)
    info = pl.info()
    assert 0 < info.lf_points < W.N and info.nnz > 0, (info.lf_points, info.nnz)
    q = to_dev(W.q, precision, False)
    u = pl.apply(q).cpu().numpy()
    w = pl.apply_adjoint(q).cpu().numpy()
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    assert pl.device_status() == pim.PIM_OK
    assert rel(u, ue) < tol, rel(u, ue)
    assert rel(w, we) < tol, rel(w, we)
    pl.close()


def test_listfree_equals_stored_list_fp64(clusters):
    """The two forms of the correction are one operator: the stored-list plan
    and the all-list-free plan agree to FP64 rounding."""
    W, _, _ = clusters
    q = to_dev(W.q, "fp64", False)
    a = gpu_plan(W, "fp64", listfree=0)
    b = gpu_plan(W, "fp64", listfree=1)
    assert a.info().lf_boxes == 0 and b.info().lf_pairs > 0
    ua, ub = a.apply(q).cpu().numpy(), b.apply(q).cpu().numpy()
    wa, wb = a.apply_adjoint(q).cpu().numpy(), b.apply_adjoint(q).cpu().numpy()
    assert rel(ub, ua) < 1e-13 and rel(wb, wa) < 1e-13, (rel(ub, ua), rel(wb, wa))
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_listfree_several_rhs(precision, clusters):
    """Three right-hand sides in one call equal three single applies."""
    W, _, _ = clusters
    rng = np.random.default_rng(3)
    Q = (rng.standard_normal((W.N, 3)) + 1j * rng.standard_normal((W.N, 3))) * np.sqrt(0.5)
    pl = gpu_plan(W, precision, listfree=3000)
    qd = to_dev(Q, precision, False)
    U = pl.apply(qd.contiguous()).cpu().numpy()
    single = np.stack([pl.apply(qd[:, r].contiguous()).cpu().numpy() for r in range(3)], axis=1)
    tol = 1e-13 if precision == "fp64" else 1e-6
    assert rel(U, single) < tol, rel(U, single)
    pl.close()


def test_listfree_rejects_coincident_points():
    """Two points equal modulo the lattice make Eq. 1 singular: set-points
    returns PIM_ERR_ARG whichever form holds their correction."""
    rng = np.random.default_rng(9)
    pts = np.concatenate([rng.random((200, 3)), 0.5 + 0.004 * rng.random((30, 3))])
    pts[-1] = pts[-2]
    for lf in (0, 1):
        pl = pim.Plan((1, 1, 1), (0, 1, 2), 3.0, (0.4, 0, 0), (13, 13, 13), p=4, layers=1, precision="fp64", b=3,
                      nf=(8, 8, 8), pf=4, listfree=lf)
        with pytest.raises(pim.PimError) as e:
            pl.set_points(torch.tensor(pts, dtype=torch.float64, device="cuda"))
        assert e.value.status == pim.PIM_ERR_ARG
        pl.close()


@pytest.mark.parametrize("name", ["helmholtz3d_bloch", "npsp3d", "helmholtz2d_bloch", "p2_helmholtz3d"])
def test_fp32_grid_part_on_tensor_cores_equals_cuda_cores(name, cache):
    """The interior boxes' grid part as one TF32-split matrix product on the
    tensor cores against the CUDA-core kernel, forward and adjoint: the same
    sums in FP32 (bar 2e-6)."""
    W, _, _ = oracle_results(name, cache)
    a = gpu_plan(W, "fp32", listfree=1)
    b = gpu_plan(W, "fp32", listfree=1, lf_tensor_cores=False)
    assert a.info().lf_tc_boxes > 0 and b.info().lf_tc_boxes == 0
    q = to_dev(W.q, "fp32", is_real(W))
    ua, ub = a.apply(q).cpu().numpy(), b.apply(q).cpu().numpy()
    wa, wb = a.apply_adjoint(q).cpu().numpy(), b.apply_adjoint(q).cpu().numpy()
    assert a.device_status() == pim.PIM_OK
    assert rel(ua, ub) < 2e-6 and rel(wa, wb) < 2e-6, (rel(ua, ub), rel(wa, wb))
    a.close()
    b.close()
