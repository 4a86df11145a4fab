"""pim_apply_noalloc: the apply for callers that cannot allocate device
memory when they apply the operator (its scratch is a fixed array the
library holds).  Its results must equal those of pim_apply /
pim_apply_adjoint, call after call.  This file is collected last."""
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


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_noalloc_matches_apply_on_two_calls_in_a_row(precision, tol):
    W = inputs.random_case(700, (1, 1, 0.5), (0, 1), 2 * np.pi * 0.8, (1.5, 0.5, 0.0), (17, 17, 9), b=4,
                           nf=(10, 10, 6), seed=21)
    pl = pim.Plan(W.D, W.pdims, W.k, W.k0, W.n, p=4, layers=1, precision=precision, b=W.b, nf=W.nf, pf=4)
    pl.set_points(torch.tensor(W.points, device="cuda"))
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    rng = np.random.default_rng(3)
    for call in range(2):
        q = torch.tensor(rng.standard_normal(W.N) + 1j * rng.standard_normal(W.N), dtype=dt, device="cuda")
        u_ref = pl.apply(q)
        w_ref = pl.apply_adjoint(q)
        u = torch.empty_like(q)
        w = torch.empty_like(q)
        pim.pim_apply_noalloc(pl._h, q, u, 1, adjoint=False)
        pim.pim_apply_noalloc(pl._h, q, w, 1, adjoint=True)
        torch.cuda.synchronize()
        assert rel(u, u_ref) < tol, (call, rel(u, u_ref))
        assert rel(w, w_ref) < tol, (call, rel(w, w_ref))
    assert pl.device_status() == pim.PIM_OK
    pl.close()


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
