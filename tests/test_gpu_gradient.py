"""GPU position gradient, frozen-topology update and autograd against the
FP64 oracle and against finite differences."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import pim as opim  # noqa: E402
from paper_2312_02376_gb300 import inputs, pim  # noqa: E402
from paper_2312_02376_gb300.autograd import pim_apply  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


CASES = {
    "helmholtz2d_bloch": dict(D=(1, 1, 0.5), pdims=(0, 1), k=4.0, k0=(1.2, 0.4, 0.0), n=(9, 9, 6), p=3, b=3,
                              nf=(7, 7, 5), pf=3),
    "npsp3d": dict(D=(1, 1, 1), pdims=(0, 1, 2), k=0.0, k0=(0, 0, 0), n=(9, 9, 9), p=4, b=4, nf=(6, 6, 6), pf=4),
    "helmholtz3d": dict(D=(1, 1, 1), pdims=(0, 1, 2), k=3.0, k0=(0.7, 0.0, 0.5), n=(9, 9, 9), p=4, b=4,
                        nf=(6, 6, 6), pf=4),
}


def setup(name, N=120, seed=0):
    c = CASES[name]
    rng = np.random.default_rng(seed)
    D = np.asarray(c["D"], float)
    pts = rng.random((N, 3)) * D * 0.98 + 0.01 * D
    real = c["k"] == 0 and not any(c["k0"])
    if real:
        q = rng.standard_normal(N)
        q -= q.mean()
        g = rng.standard_normal(N)
    else:
        q = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        g = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    P = opim.Params(D=c["D"], pdims=c["pdims"], k=c["k"], k0=c["k0"], n=c["n"], p=c["p"], layers=1, b=c["b"],
                    nf=c["nf"], pf=c["pf"])
    pl = pim.Plan(c["D"], c["pdims"], c["k"], c["k0"], c["n"], p=c["p"], layers=1, precision="fp64", b=c["b"],
                  nf=c["nf"], pf=c["pf"], with_gradient=True)
    pl.set_points(torch.tensor(pts, device="cuda"))
    return P, pl, pts, q, g, real


def dev(x, real):
    return torch.tensor(np.real(x) if real else x, dtype=torch.float64 if real else torch.complex128, device="cuda")


@pytest.mark.parametrize("name", list(CASES))
def test_position_grad_matches_oracle(name):
    P, pl, pts, q, g, real = setup(name)
    G = pl.position_grad(dev(q, real), dev(g, real)).cpu().numpy()
    Go = opim.Plan(P, pts).position_grad(q.astype(complex), g.astype(complex))
    assert rel(G, Go) < 1e-11, rel(G, Go)
    pl.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("mode", ["double_float", "compact", "fp64"])
def test_position_grad_fp32_matches_oracle(name, mode):
    # FP32 bulk (grid sums in FP32); the correction list in double-float,
    # compact or FP64: rel-L2 within the FP32 path's bound
    c = CASES[name]
    P, _, pts, q, g, real = setup(name)
    cm = {"double_float": pim.PIM_CORR_DOUBLE_FLOAT, "compact": pim.PIM_CORR_COMPACT, "fp64": pim.PIM_CORR_FP64}[mode]
    pl = pim.Plan(c["D"], c["pdims"], c["k"], c["k0"], c["n"], p=c["p"], layers=1, precision="fp32", b=c["b"],
                  nf=c["nf"], pf=c["pf"], corr_mode=cm, with_gradient=True)
    pl.set_points(torch.tensor(pts, device="cuda"))
    if real:
        qd = torch.tensor(np.real(q), dtype=torch.float32, device="cuda")
        gd = torch.tensor(np.real(g), dtype=torch.float32, device="cuda")
    else:
        qd = torch.tensor(q, dtype=torch.complex64, device="cuda")
        gd = torch.tensor(g, dtype=torch.complex64, device="cuda")
    G = pl.position_grad(qd, gd).cpu().numpy()
    qo = qd.cpu().numpy().astype(complex)
    go = gd.cpu().numpy().astype(complex)
    Go = opim.Plan(P, pts).position_grad(qo, go)
    assert rel(G, Go) < 2e-5, rel(G, Go)
    pl.close()


@pytest.mark.parametrize("name", ["helmholtz2d_bloch", "npsp3d"])
def test_update_positions_is_frozen_topology_apply(name):
    P, pl, pts, q, g, real = setup(name)
    base = opim.Plan(P, pts)
    moved = pts + 1e-3 * np.random.default_rng(1).standard_normal(pts.shape) * np.asarray(P.D)
    moved = np.clip(moved, 0, np.asarray(P.D))
    pl.update_positions(torch.tensor(moved, device="cuda"))
    u = pl.apply(dev(q, real)).cpu().numpy()
    uo = opim.Plan(P, moved, K=base.K, F=base.F, frozen=base).apply(q.astype(complex))
    assert rel(u, uo) < 1e-12
    pl.close()


@pytest.mark.parametrize("name", ["helmholtz2d_bloch", "npsp3d"])
def test_update_positions_compact_fp32(name):
    # FP32 plan with compact rows: the refilled values are split again by
    # magnitude; the apply at the moved points matches the frozen-topology
    # oracle within the FP32 path's bound
    c = CASES[name]
    P, _, pts, q, g, real = setup(name)
    pl = pim.Plan(c["D"], c["pdims"], c["k"], c["k0"], c["n"], p=c["p"], layers=1, precision="fp32", b=c["b"],
                  nf=c["nf"], pf=c["pf"], corr_mode=pim.PIM_CORR_COMPACT, corr_split=4)
    pl.set_points(torch.tensor(pts, device="cuda"))
    base = opim.Plan(P, pts)
    moved = pts + 1e-3 * np.random.default_rng(1).standard_normal(pts.shape) * np.asarray(P.D)
    moved = np.clip(moved, 0, np.asarray(P.D))
    pl.update_positions(torch.tensor(moved, device="cuda"))
    rp, val, nb = pl.debug(4), pl.debug(6), pl.debug(7)
    for r in range(len(rp) - 1):
        a, b = rp[r], rp[r + 1]
        if b > a:
            mag = np.abs(val[a:b])
            big = mag > 2.0 ** -4 * mag.max()
            assert nb[r] == big.sum() and big[:nb[r]].all()
    qd = torch.tensor(np.real(q) if real else q, dtype=torch.float32 if real else torch.complex64, device="cuda")
    u = pl.apply(qd).cpu().numpy()
    uo = opim.Plan(P, moved, K=base.K, F=base.F, frozen=base).apply(qd.cpu().numpy().astype(complex))
    assert rel(u, uo) < 2e-5, rel(u, uo)
    pl.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["helmholtz2d_bloch", "npsp3d", "helmholtz3d"])
def test_position_grad_reuse_equals_full(name, precision):
    # after apply(q) and apply_adjoint(g) the gradient kernel alone, on the
    # potentials those applies kept, equals the full gradient; the state
    # rules: none before both applies, none after a multi-RHS apply or new points
    c = CASES[name]
    P, _, pts, q, g, real = setup(name)
    pl = pim.Plan(c["D"], c["pdims"], c["k"], c["k0"], c["n"], p=c["p"], layers=1, precision=precision, b=c["b"],
                  nf=c["nf"], pf=c["pf"], with_gradient=True)
    pl.set_points(torch.tensor(pts, device="cuda"))
    if precision == "fp64":
        qd, gd = dev(q, real), dev(g, real)
    else:
        dt = torch.float32 if real else torch.complex64
        qd = torch.tensor(np.real(q) if real else q, dtype=dt, device="cuda")
        gd = torch.tensor(np.real(g) if real else g, dtype=dt, device="cuda")
    with pytest.raises(pim.PimError):
        pl.position_grad_reuse(qd, gd)
    pl.apply(qd)
    with pytest.raises(pim.PimError):
        pl.position_grad_reuse(qd, gd)
    pl.apply_adjoint(gd)
    G1 = pl.position_grad_reuse(qd, gd).cpu().numpy()
    G0 = pl.position_grad(qd, gd).cpu().numpy()
    tol = 1e-13 if precision == "fp64" else 1e-6
    assert rel(G1, G0) < tol, rel(G1, G0)
    with pytest.raises(pim.PimError):      # the full gradient replaced the kept potentials
        pl.position_grad_reuse(qd, gd)
    pl.apply_adjoint(gd)
    pl.apply(qd)
    assert rel(pl.position_grad_reuse(qd, gd).cpu().numpy(), G0) < tol
    pl.apply(torch.stack([qd, qd], dim=1).contiguous())
    with pytest.raises(pim.PimError):
        pl.position_grad_reuse(qd, gd)
    pl.close()


def test_position_grad_finite_differences_on_gpu():
    # central differences of Re <g, A q> through pim_update_positions (FP64)
    P, pl, pts, q, g, real = setup("helmholtz2d_bloch", N=200)
    qd, gd = dev(q, real), dev(g, real)
    G = pl.position_grad(qd, gd).cpu().numpy()
    h = 1e-5
    for k in (3, 77, 150):
        for d in range(3):
            vals = []
            for sgn in (1, -1):
                x = pts.copy()
                x[k, d] += sgn * h
                pl.update_positions(torch.tensor(x, device="cuda"))
                vals.append(np.real(np.vdot(g, pl.apply(qd).cpu().numpy())))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - G[k, d]) < 1e-6 * np.abs(G).max()
    pl.close()


def test_autograd_energy_gradients_coulomb3d_twin():
    # differentiated 3D Coulomb: E = 1/2 q^T phi, phi = A(x) q, gradients with
    # respect to q and x by autograd; central differences (h = 1e-4) on
    # sampled points with the discrete structure frozen
    W = inputs.coulomb3d_big(N=20000, n=32)
    pl = pim.Plan(W.D, W.pdims, 0.0, W.k0, W.n, p=4, layers=1, precision="fp64", b=W.b, nf=W.nf, pf=4,
                  with_gradient=True)
    x0 = torch.tensor(W.points, device="cuda")
    pl.set_points(x0)
    q = torch.tensor(W.q.astype(np.float64), device="cuda", requires_grad=True)
    x = x0.clone().requires_grad_(True)
    phi = pim_apply(q, x, pl)
    E = 0.5 * torch.dot(q, phi)
    E.backward()
    gq, gx = q.grad.cpu().numpy(), x.grad.cpu().numpy()
    # dE/dq = (A q + A^T q) / 2 (the far zone's shifted grids make A only
    # approximately symmetric)
    ref = 0.5 * (phi.detach() + pl.apply_adjoint(q.detach())).cpu().numpy()
    assert rel(gq, ref) < 1e-10
    idx = np.random.default_rng(2).choice(W.N, 64, replace=False)
    h = 1e-4
    qn = q.detach()
    worst = 0.0
    for k in idx[:16]:
        for d in range(3):
            e = []
            for sgn in (1, -1):
                xx = W.points.copy()
                xx[k, d] += sgn * h
                pl.update_positions(torch.tensor(xx, device="cuda"))
                e.append(0.5 * torch.dot(qn, pl.apply(qn)).item())
            fd = (e[0] - e[1]) / (2 * h)
            worst = max(worst, abs(fd - gx[k, d]) / np.abs(gx).max())
    assert worst < 1e-5, worst
    pl.close()
