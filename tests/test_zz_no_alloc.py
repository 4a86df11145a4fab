"""pim_apply_noalloc: the apply for callers that cannot allocate device
memory when they apply the operator (its scratch is a fixed array the
library holds).  Its results must equal those of pim_apply /
pim_apply_adjoint, call after call, and the plan's device memory must not
change.  This file is collected last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_02376_gb300 import inputs, pim  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()


def rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def helmholtz2d_plan(precision, N=700, seed=21):
    W = inputs.random_case(N, (1, 1, 0.5), (0, 1), 2 * np.pi * 0.8, (1.5, 0.5, 0.0), (17, 17, 9), b=4,
                           nf=(10, 10, 6), seed=seed)
    pl = pim.Plan(W.D, W.pdims, W.k, W.k0, W.n, p=4, layers=1, precision=precision, b=W.b, nf=W.nf, pf=4)
    pl.set_points(torch.tensor(W.points, device="cuda"))
    return pl, W


def coulomb3d_plan(precision):
    W = inputs.random_case(600, (1, 1, 1), (0, 1, 2), 0.0, (0, 0, 0), (13, 13, 13), b=4, nf=(8, 8, 8), seed=4,
                           complex_q=False, neutral=True)
    pl = pim.Plan(W.D, W.pdims, 0.0, (0, 0, 0), W.n, p=4, layers=1, precision=precision, b=W.b, nf=W.nf, pf=4)
    pl.set_points(torch.tensor(W.points, device="cuda"))
    return pl, W


def free_space_plan(precision):
    W = inputs.random_case(500, (1, 1, 0.5), (), 4.0, (0, 0, 0), (17, 17, 9), b=4, seed=8)
    pl = pim.Plan(W.D, (), 4.0, (0, 0, 0), W.n, p=4, layers=1, precision=precision, b=W.b, pf=4)
    pl.set_points(torch.tensor(W.points, device="cuda"))
    return pl, W


def clustered_plan(precision):
    """Points in tight clusters, every box's correction list-free."""
    rng = np.random.default_rng(2)
    pts = np.concatenate([rng.random((300, 3)), np.clip(0.5 + 0.02 * rng.standard_normal((500, 3)), 0, 1)])
    pl = pim.Plan((1, 1, 1), (0, 1, 2), 5.0, (1.0, -0.5, 0.3), (17, 17, 17), p=4, layers=1, precision=precision, b=3,
                  nf=(8, 8, 8), pf=4, listfree=1)
    pl.set_points(torch.tensor(pts, device="cuda"))
    assert pl.info().lf_points == len(pts)
    return pl, inputs.Workload("clusters", (1, 1, 1), (0, 1, 2), 5.0, (1.0, -0.5, 0.3), (17, 17, 17), 4, 1, 3,
                               (8, 8, 8), 4, precision, len(pts), 1, pts, None)


def sources(W, nrhs, real, precision, rng):
    shape = (W.N,) if nrhs == 1 else (W.N, nrhs)
    if real:
        x = rng.standard_normal(shape)
        x = x - x.mean(axis=0, keepdims=True)
        return torch.tensor(x, dtype=torch.float64 if precision == "fp64" else torch.float32, device="cuda")
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return torch.tensor(x, dtype=torch.complex128 if precision == "fp64" else torch.complex64, device="cuda")


PLANS = {"helmholtz2d": (helmholtz2d_plan, False, 1), "coulomb3d_3rhs": (coulomb3d_plan, True, 3),
         "free_space": (free_space_plan, False, 1), "clusters_listfree": (clustered_plan, False, 2)}


@pytest.mark.parametrize("name", list(PLANS))
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_noalloc_matches_apply_on_two_calls_in_a_row(name, precision, tol):
    make, real, nrhs = PLANS[name]
    pl, W = make(precision)
    rng = np.random.default_rng(3)
    for call in range(2):
        q = sources(W, nrhs, real, precision, rng)
        u_ref = pl.apply(q)
        w_ref = pl.apply_adjoint(q)
        before = pl.info().device_bytes
        u = torch.empty_like(q)
        w = torch.empty_like(q)
        pim.pim_apply_noalloc(pl._h, q, u, nrhs, adjoint=False)
        pim.pim_apply_noalloc(pl._h, q, w, nrhs, adjoint=True)
        torch.cuda.synchronize()
        assert pl.info().device_bytes == before
        assert rel(u, u_ref) < tol, (call, rel(u, u_ref))
        assert rel(w, w_ref) < tol, (call, rel(w, w_ref))
    assert pl.device_status() == pim.PIM_OK
    pl.close()


def test_noalloc_plans_of_different_sizes_in_turn():
    """A larger plan's call between two calls of a smaller one: every call
    writes the scratch it reads, whatever the last call left there."""
    small, Ws = helmholtz2d_plan("fp32", N=400, seed=5)
    big, Wb = helmholtz2d_plan("fp32", N=3000, seed=6)
    rng = np.random.default_rng(11)
    qs = sources(Ws, 1, False, "fp32", rng)
    qb = sources(Wb, 1, False, "fp32", rng)
    ref_s, ref_b = small.apply(qs), big.apply(qb)
    for pl, q, ref in ((small, qs, ref_s), (big, qb, ref_b), (small, qs, ref_s)):
        u = torch.empty_like(q)
        pim.pim_apply_noalloc(pl._h, q, u, 1, adjoint=False)
        torch.cuda.synchronize()
        assert rel(u, ref) < 1e-6, rel(u, ref)
    small.close()
    big.close()


def test_noalloc_rejects_plans_beyond_the_limit_and_host_buffers():
    # FP64 grids of 96 x 96 x 48 nodes: the padded FFT work grids alone exceed the 32 MiB scratch
    W = inputs.helmholtz2d(N=65536, n=(96, 96, 48), nf=(12, 12, 8), b=3)
    pl = pim.Plan(W.D, W.pdims, W.k, W.k0, W.n, p=4, layers=1, precision="fp64", b=W.b, nf=W.nf, pf=4)
    pl.set_points(torch.tensor(W.points, device="cuda"))
    q = torch.tensor(W.q, dtype=torch.complex128, device="cuda")
    with pytest.raises(pim.PimError) as e:
        pim.pim_apply_noalloc(pl._h, q, torch.empty_like(q), 1)
    assert e.value.status == pim.PIM_ERR_ARG
    with pytest.raises(pim.PimError) as e:
        pim.pim_apply_noalloc(pl._h, q.cpu().numpy(), np.empty(W.N, np.complex128), 1)
    assert e.value.status == pim.PIM_ERR_ARG
    pl.close()
