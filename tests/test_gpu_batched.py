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


@pytest.fixture(scope="module")
def helmholtz1d_batch_run():
    """The batched 1D-periodic Helmholtz workload (16 sets, 64 right-hand
    sides, FP32 bulk) through one batched graph, as bench.py runs it."""
    sets = inputs.helmholtz1d_batch()
    plans, qs, us = [], [], []
    for W in sets:
        pl = pim.Plan(W.D, W.pdims, W.k, W.k0, W.n, p=W.p, layers=W.layers, precision="fp32", b=W.b, nf=W.nf,
                      pf=W.pf)
        pl.set_points(torch.tensor(W.points, dtype=torch.float64, device="cuda"))
        plans.append(pl)
        qs.append(torch.tensor(W.q, device="cuda"))
        us.append(torch.empty_like(qs[-1]))
    stream = torch.cuda.Stream()
    pim.pim_apply_batched(plans, qs, us, sets[0].nrhs, adjoint=False, stream=stream)
    stream.synchronize()
    out = [u.cpu().numpy() for u in us]
    infos = [pl.info() for pl in plans]
    for pl in plans:
        pl.close()
    return sets, out, infos


def test_helmholtz1d_batch_graph_vs_ewald_rows(helmholtz1d_batch_run):
    """Rows of the smallest and the largest set, first and last right-hand
    side, of the batched graph's output against the committed 1D-lattice
    Ewald ground truth, within the stated method error (1e-4 at p = 4)."""
    import os
    sets, out, _ = helmholtz1d_batch_run
    d = np.loadtxt(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                "helmholtz1d_batch_ewald_rows.txt"), comments="#")
    for si in np.unique(d[:, 0].astype(int)):
        for r in np.unique(d[d[:, 0] == si, 1].astype(int)):
            sel = (d[:, 0] == si) & (d[:, 1] == r)
            rows = d[sel, 2].astype(np.int64)
            ref = d[sel, 3] + 1j * d[sel, 4]
            e = rel(out[si][rows, r], ref)
            assert e < 1e-4, (si, r, e)


def test_helmholtz1d_batch_graph_vs_oracle_rows(helmholtz1d_batch_run):
    """The batched graph's output of the smallest and the largest set against
    the FP64 oracle's rows (FP32 bar), first and last right-hand side."""
    sets, out, infos = helmholtz1d_batch_run
    Ns = [W.N for W in sets]
    for si in (int(np.argmin(Ns)), int(np.argmax(Ns))):
        W = sets[si]
        P = opim.Params(D=W.D, pdims=W.pdims, k=W.k, k0=W.k0, n=W.n, p=W.p, layers=W.layers, b=W.b,
                        nf=tuple(infos[si].nf), pf=W.pf)
        o = opim.Plan(P, W.points)
        rows = np.random.default_rng(31 + si).choice(W.N, 6, replace=False)
        for r in (0, W.nrhs - 1):
            ue = o.apply_rows(W.q[:, r].astype(np.complex128), rows)
            assert rel(out[si][rows, r], ue) < 2e-5, (si, r, rel(out[si][rows, r], ue))
