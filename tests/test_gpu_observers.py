"""Observer points apart from the sources (Sec. 4.1's accuracy test; Sec. 4's
coax) through the C ABI: pim_set_points_observers, pim_apply_observers and
its adjoint against the FP64 oracle (oracle.pim.apply_observers,
apply_observers_adjoint), and the coax's analytic potentials computed on the
GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import pim as opim  # noqa: E402
from paper_2312_02376_gb300 import inputs, pim  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


# name: (D, pdims, k, k0, n, b, nf, pf, p, N, M)
CASES = {
    "helmholtz3d_bloch": ((1, 1, 1), (0, 1, 2), 2 * np.pi * 0.7, (0.9, 0.9, 0.0), (13, 13, 13), 4, (8, 8, 8), 4, 4, 500,
                          60),
    "npsp3d": ((1, 1, 1), (0, 1, 2), 0.0, (0, 0, 0), (13, 13, 13), 4, (8, 8, 8), 4, 4, 500, 40),
    "helmholtz1d_complex_k0": ((0.5, 0.5, 1), (2,), 3.0 - 0.3j, (0, 0, 1.2 - 0.2j), (9, 9, 17), 3, (6, 6, 10), 3, 4,
                               400, 30),
    "free_space": ((1, 1, 0.5), (), 4.0, (0, 0, 0), (17, 17, 9), 4, (10, 10, 10), 4, 4, 500, 50),
}


def make(name):
    D, pdims, k, k0, n, b, nf, pf, p, N, M = CASES[name]
    rng = np.random.default_rng(77)
    D = np.asarray(D, np.float64)
    src, obs = rng.random((N, 3)) * D, rng.random((M, 3)) * D
    real = k == 0 and not any(k0)
    q = rng.standard_normal(N) if real else (rng.standard_normal(N) + 1j * rng.standard_normal(N)) * np.sqrt(0.5)
    if real:
        q = q - q.mean()
    v = (rng.standard_normal(M) + 1j * rng.standard_normal(M)) * np.sqrt(0.5)
    if real:
        v = v.real.copy()
    P = opim.Params(D=tuple(D), pdims=pdims, k=k, k0=k0, n=n, p=p, layers=1, b=b, nf=nf, pf=pf)
    return P, src, obs, q, v, real


@pytest.fixture(scope="module")
def cache():
    return {}


def oracle_results(name, cache):
    if name not in cache:
        P, src, obs, q, v, real = make(name)
        cache[name] = (P, src, obs, q, v, real, opim.apply_observers(P, src, obs, q),
                       opim.apply_observers_adjoint(P, src, obs, v))
    return cache[name]


def gpu_plan(P, src, obs, precision):
    pl = pim.Plan(P.D, P.pdims, P.k, P.k0, P.n, p=P.p, layers=1, precision=precision, b=P.b,
                  nf=P.nf if P.pdims else None, pf=P.pf)
    pl.set_points_observers(torch.tensor(src, device="cuda"), torch.tensor(obs, device="cuda"))
    return pl


def dev(x, precision, real):
    if real:
        return torch.tensor(np.real(x), dtype=torch.float64 if precision == "fp64" else torch.float32, device="cuda")
    return torch.tensor(x, dtype=torch.complex128 if precision == "fp64" else torch.complex64, device="cuda")


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_observers_forward_and_adjoint(name, precision, tol, cache):
    P, src, obs, q, v, real, ue, we = oracle_results(name, cache)
    pl = gpu_plan(P, src, obs, precision)
    assert pl.info().N == len(src) + len(obs)
    u = pl.apply_observers(dev(q, precision, real)).cpu().numpy()
    w = pl.apply_observers(dev(v, precision, real), adjoint=True).cpu().numpy()
    assert pl.device_status() == pim.PIM_OK
    assert rel(u, ue) < tol, rel(u, ue)
    assert rel(w, we) < tol, rel(w, we)
    pl.close()


def test_observers_several_rhs_and_host_buffers(cache):
    P, src, obs, q, v, real, _, _ = oracle_results("helmholtz3d_bloch", cache)
    rng = np.random.default_rng(8)
    Q = (rng.standard_normal((len(src), 3)) + 1j * rng.standard_normal((len(src), 3))) * np.sqrt(0.5)
    pl = gpu_plan(P, src, obs, "fp64")
    U = pl.apply_observers(torch.tensor(Q, device="cuda")).cpu().numpy()
    Uh = pl.apply_observers(np.ascontiguousarray(Q))                  # host buffers
    for r in range(3):
        ur = pl.apply_observers(torch.tensor(Q[:, r].copy(), device="cuda")).cpu().numpy()
        assert rel(U[:, r], ur) < 1e-13 and rel(Uh[:, r], ur) < 1e-13
    pl.close()


def test_observers_neutrality_is_checked_on_the_sources(cache):
    P, src, obs, q, v, real, _, _ = oracle_results("npsp3d", cache)
    pl = gpu_plan(P, src, obs, "fp64")
    pl.apply_observers(torch.tensor(q, device="cuda"))
    assert pl.device_status() == pim.PIM_OK
    pl.apply_observers(torch.tensor(q + 1.0, device="cuda"))
    assert pl.device_status() == pim.PIM_ERR_NOT_NEUTRAL
    pl.close()


def test_observers_state_errors():
    pl = pim.Plan((1, 1, 1), (0, 1, 2), 3.0, (0, 0, 0), (9, 9, 9), precision="fp64", b=3, nf=(6, 6, 6))
    rng = np.random.default_rng(2)
    pts = torch.tensor(rng.random((50, 3)), device="cuda")
    q = torch.zeros(50, dtype=torch.complex128, device="cuda")
    pl.set_points(pts)
    pl.N_src, pl.M_obs = 50, 5
    with pytest.raises(pim.PimError) as e:
        pl.apply_observers(q)
    assert e.value.status == pim.PIM_ERR_STATE
    pl.set_points_observers(pts, torch.tensor(rng.random((5, 3)), device="cuda"))
    pl.apply_observers(q)
    pl.set_points(pts)                      # drops the observers
    with pytest.raises(pim.PimError) as e:
        pl.apply_observers(q)
    assert e.value.status == pim.PIM_ERR_STATE
    pl.close()


def coax_plan(k, k0, precision="fp64"):
    src, q, obs = inputs.coax()
    pl = pim.Plan((5.0, 5.0, 1.0), (2,), k, k0, (51, 51, 11), p=4, layers=1, precision=precision, b=5,
                  nf=(24, 24, 10), pf=4)
    pl.set_points_observers(torch.tensor(src, device="cuda"), torch.tensor(obs, device="cuda"))
    return pl, src, q, obs


def test_coax_neutral_static_on_the_gpu():
    """The neutral static coax (Sec. 4): potential flat on the axis and
    outside the outer cylinder, their difference ln(r2/r1) / (2 pi)."""
    pl, src, q, obs = coax_plan(0.0, (0, 0, 0))
    u = pl.apply_observers(torch.tensor(q, device="cuda")).cpu().numpy()
    assert pl.device_status() == pim.PIM_OK
    ua, uo = u[:8], u[8:]
    dv = ua.mean() - uo.mean()
    exact = np.log(2.0) / (2 * np.pi)
    assert np.ptp(ua) < 2e-5 * dv and np.ptp(uo) < 2e-5 * dv, (np.ptp(ua) / dv, np.ptp(uo) / dv)
    assert abs(dv - exact) < 1e-5 * exact, (dv, exact)
    pl.close()


def test_coax_dynamic_complex_phase_on_the_gpu():
    """The dynamic coax (k = 1, k0 = 1 - j, sources with the Bloch phase
    exp(-j k0 z)): the potential on the axis is C exp(-j k0 z), so that
    u(z) exp(j k0 z) is constant along it."""
    k0 = 1.0 - 1.0j
    pl, src, q, obs = coax_plan(1.0, (0, 0, k0))
    qd = q * np.exp(-1j * k0 * src[:, 2])
    u = pl.apply_observers(torch.tensor(qd, device="cuda")).cpu().numpy()
    assert pl.device_status() == pim.PIM_OK
    ua = u[:8] * np.exp(1j * k0 * obs[:8, 2])
    assert np.max(np.abs(ua - ua.mean())) < 5e-5 * abs(ua.mean()), np.max(np.abs(ua - ua.mean())) / abs(ua.mean())
    pl.close()
