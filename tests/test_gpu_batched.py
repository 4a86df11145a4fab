"""Several right-hand sides and several point sets (batched, graph-captured)
against single applies and against the oracle."""
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
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    b = b.cpu().numpy() if hasattr(b, "cpu") else b
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


SETS = [
    # (D, pdims, k, k0, n, N, b, nf)
    ((1, 0.25, 0.25), (2,), 2 * np.pi * 0.5, (0, 0, 0), (33, 9, 9), 900, 3, (13, 10, 10)),
    ((1, 1, 0.5), (0, 1), 2 * np.pi * 0.8, (1.5, 0.5, 0), (17, 17, 9), 700, 3, (10, 10, 6)),
    ((1, 1, 1), (0, 1, 2), 0.0, (0, 0, 0), (13, 13, 13), 600, 3, (8, 8, 8)),
]


def make(i, precision="fp64", nrhs=1, seed=0):
    D, pdims, k, k0, n, N, b, nf = SETS[i]
    real = k == 0 and not any(k0)
    W = inputs.random_case(N, D, pdims, k, k0, n, b=b, nf=nf, seed=40 + i + seed, complex_q=not real,
                           neutral=real, nrhs=nrhs)
    pl = pim.Plan(D, pdims, k, k0, n, p=4, layers=1, precision=precision, b=b, nf=nf, pf=4)
    pl.set_points(torch.tensor(W.points, device="cuda"))
    return W, pl, real


def tens(x, precision, real):
    if real:
        return torch.tensor(np.real(x), dtype=torch.float64 if precision == "fp64" else torch.float32, device="cuda")
    return torch.tensor(x, dtype=torch.complex128 if precision == "fp64" else torch.complex64, device="cuda")


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("i", [0, 1, 2])
@pytest.mark.parametrize("nrhs", [5, 40])
def test_multi_rhs_equals_columns(i, nrhs, precision, tol):
    W, pl, real = make(i, precision, nrhs=nrhs)
    Q = tens(W.q, precision, real).contiguous()
    for adj in (False, True):
        U = pl.apply(Q, adjoint=adj)
        for r in (0, nrhs // 2, nrhs - 1):
            ur = pl.apply(Q[:, r].contiguous(), adjoint=adj)
            assert rel(U[:, r], ur) < tol, (adj, r, rel(U[:, r], ur))
    pl.close()


def test_multi_rhs_against_oracle():
    W, pl, real = make(0, "fp64", nrhs=6)
    U = pl.apply(tens(W.q, "fp64", real)).cpu().numpy()
    D, pdims, k, k0, n, N, b, nf = SETS[0]
    o = opim.Plan(opim.Params(D=D, pdims=pdims, k=k, k0=k0, n=n, p=4, layers=1, b=b, nf=nf, pf=4), W.points)
    for r in range(6):
        assert rel(U[:, r], o.apply(W.q[:, r])) < 1e-12
    pl.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_batched_graph_equals_single_applies(precision, tol):
    made = [make(i, precision, nrhs=4, seed=1) for i in range(3)]
    qs = [tens(W.q, precision, real).contiguous() for (W, _, real) in made]
    plans = [pl for (_, pl, _) in made]
    for adj in (False, True):
        refs = [pl.apply(q, adjoint=adj) for pl, q in zip(plans, qs)]
        us = [torch.empty_like(q) for q in qs]
        stream = torch.cuda.Stream()
        for rep in range(3):                       # capture, then two replays
            for u in us:
                u.zero_()
            torch.cuda.synchronize()
            pim.pim_apply_batched(plans, qs, us, 4, adjoint=adj, stream=stream)
            stream.synchronize()
            for u, ref in zip(us, refs):
                assert rel(u, ref) < tol
    # new sources written into the same buffers are picked up by a replay
    # (same pointers: the cached graph of the last adjoint=False call)
    with torch.no_grad():
        qs[1].mul_(2.0)
    pim.pim_apply_batched(plans, qs, us, 4)        # library stream, synchronous
    assert rel(us[1], plans[1].apply(qs[1])) < tol
    for pl in plans:
        pl.close()
