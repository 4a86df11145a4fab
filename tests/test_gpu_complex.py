"""Complex wavenumber and complex phase shift (Sec. 2: a lossy medium has
Im k < 0; the Bloch phase shift k0 may be complex) on the GPU path, against
the FP64 oracle through the C ABI.

With a complex k0 the image phases exp(-j k0.(i o L)) have modulus != 1 and
the adjoint's phases exp(-j conj(k0).(i o L)) differ from them; with a
complex k the far series (Eq. pgf) are summed in complex arithmetic (the 1D
series through K0 of a complex argument) and the correction is stored for
every box.  Bars as for real k: FP64 <= 1e-12, FP32 <= 2e-5 relative L2."""
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


# name: (D, pdims, k, k0, n, N, b, nf, pf, p, clustered, listfree)
CASES = {
    "lossy3d_complex_k0": ((1, 1, 1), (0, 1, 2), 2 * np.pi * 0.7 - 0.5j, (0.9 - 0.2j, 0.9 + 0.1j, 0.0), (13, 13, 13), 500,
                           4, (8, 8, 8), 4, 4, False, None),
    "lossy2d_complex_k0": ((1, 1, 0.5), (0, 1), 2 * np.pi * 0.8 - 0.8j, (1.5 - 0.3j, 0.5 + 0.2j, 0.0), (17, 17, 9), 700,
                           4, (10, 10, 6), 4, 4, False, None),
    "lossy1d_complex_k0": ((0.5, 0.5, 1), (2,), 3.0 - 0.5j, (0.0, 0.0, 1.2 - 0.2j), (9, 9, 17), 500, 3, (6, 6, 10), 3,
                           4, False, None),
    "lossy_free_space": ((1, 1, 0.5), (), 4.0 - 1.0j, (0.0, 0.0, 0.0), (17, 17, 9), 600, 4, (10, 10, 10), 4, 4, False,
                         None),
    # real k, complex phase shift: the list-free correction stays on (every box)
    "complex_k0_listfree3d": ((1, 1, 1), (0, 1, 2), 2 * np.pi * 0.7, (0.9 - 0.3j, 0.4j, 0.0), (13, 13, 13), 500, 4,
                              (8, 8, 8), 4, 4, True, 1),
}


def make_case(name):
    D, pdims, k, k0, n, N, b, nf, pf, p, clustered, _ = CASES[name]
    mk = inputs.random_clustered_case if clustered else inputs.random_case
    return mk(N, D, pdims, k, k0, n, p=p, b=b, nf=nf, pf=pf, seed=31)


@pytest.fixture(scope="module")
def cache():
    return {}


def oracle_results(name, cache):
    if name not in cache:
        W = make_case(name)
        P = opim.Params(D=W.D, pdims=W.pdims, k=W.k, k0=W.k0, n=W.n, p=W.p, layers=W.layers, b=W.b, nf=W.nf,
                        pf=W.pf)
        o = opim.Plan(P, W.points)
        cache[name] = (W, o, o.apply(W.q), o.apply_adjoint(W.q))
    return cache[name]


def gpu_plan(name, W, precision):
    lf = CASES[name][-1]
    pl = pim.Plan(W.D, W.pdims, W.k, W.k0, W.n, p=W.p, layers=W.layers, precision=precision, b=W.b,
                  nf=W.nf if W.pdims else None, pf=W.pf, listfree=lf)
    pl.set_points(torch.tensor(W.points, dtype=torch.float64, device="cuda"))
    return pl


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("fp32", FP32_TOL)])
def test_forward_and_adjoint(name, precision, tol, cache):
    W, o, ue, we = oracle_results(name, cache)
    pl = gpu_plan(name, W, precision)
    if CASES[name][-1]:
        assert pl.info().lf_points == W.N
    elif np.imag(W.k) != 0:
        assert pl.info().lf_pairs == 0  # a complex k stores every correction
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    q = torch.tensor(W.q, dtype=dt, device="cuda")
    u = pl.apply(q).cpu().numpy()
    w = pl.apply_adjoint(q).cpu().numpy()
    assert pl.device_status() == pim.PIM_OK
    assert rel(u, ue) < tol, rel(u, ue)
    assert rel(w, we) < tol, rel(w, we)
    pl.close()


@pytest.mark.parametrize("name", ["lossy3d_complex_k0", "lossy2d_complex_k0", "lossy1d_complex_k0"])
def test_far_table_stage(name, cache):
    """The far table G^p - G_near on the shifted far grids (Eq. pgf minus the
    near images) entry by entry."""
    W, o, _, _ = oracle_results(name, cache)
    pl = gpu_plan(name, W, "fp64")
    F = pl.debug(0)
    Fo = np.transpose(o.F, (2, 1, 0))
    assert np.max(np.abs(F - Fo)) < 1e-12 * np.max(np.abs(Fo)), np.max(np.abs(F - Fo)) / np.max(np.abs(Fo))
    pl.close()


def test_complex_parameters_rejected_where_unsupported():
    """Im k > 0 (a gain medium) is an argument error; the position gradient
    needs a real k and k0."""
    with pytest.raises(pim.PimError) as e:
        pim.Plan((1, 1, 1), (0, 1, 2), 3.0 + 0.1j, (0, 0, 0), (9, 9, 9), precision="fp64", b=3, nf=(6, 6, 6))
    assert e.value.status == pim.PIM_ERR_ARG
    for k, k0 in ((3.0 - 0.2j, (0, 0, 0)), (3.0, (0.5 - 0.1j, 0, 0))):
        with pytest.raises(pim.PimError) as e:
            pim.Plan((1, 1, 1), (0, 1, 2), k, k0, (9, 9, 9), precision="fp64", b=3, nf=(6, 6, 6), with_gradient=True)
        assert e.value.status == pim.PIM_ERR_UNSUPPORTED


def test_1d_weakly_lossy_propagating_modes_beyond_the_evaluated_regimes():
    """1D lattice, k = 10 - 0.01j on a unit cell: propagating modes reach
    H0^(2) arguments k_rho rho of modulus about 14 within 0.17 rad of the real
    axis, which the complex series does not evaluate: plan creation reports
    PIM_ERR_UNSUPPORTED (the real k = 10 plan is fine)."""
    with pytest.raises(pim.PimError) as e:
        pim.Plan((1, 1, 1), (2,), 10.0 - 0.01j, (0, 0, 0), (9, 9, 9), precision="fp64", b=3, nf=(12, 12, 12))
    assert e.value.status == pim.PIM_ERR_UNSUPPORTED
    pim.Plan((1, 1, 1), (2,), 10.0, (0, 0, 0), (9, 9, 9), precision="fp64", b=3, nf=(12, 12, 12)).close()
