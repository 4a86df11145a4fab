"""GPU parity: libpim (through its C ABI) against the FP64 oracle, element by
element, on seeded inputs.  Tolerances: relative L2 <= 1e-12 for FP64 plans
and <= 2e-5 for FP32-mixed plans (the bars stated for this method)."""
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


def oracle_plan(W, p=4, layers=1):
    P = opim.Params(D=W.D, pdims=W.pdims, k=W.k, k0=W.k0, n=W.n, p=p, layers=layers, b=W.b, nf=W.nf, pf=W.pf)
    return opim.Plan(P, W.points)


def gpu_plan(W, precision, p=4, layers=1, **kw):
    pl = pim.Plan(W.D, W.pdims, W.k, W.k0, W.n, p=p, layers=layers, precision=precision, b=W.b, nf=W.nf, pf=W.pf,
                  **kw)
    pl.set_points(torch.tensor(W.points, dtype=torch.float64, device="cuda"))
    return pl


def to_dev(x, precision, real):
    if real:
        dt = torch.float64 if precision == "fp64" else torch.float32
        return torch.tensor(np.real(x), dtype=dt, device="cuda")
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    return torch.tensor(x, dtype=dt, device="cuda")


CASES = {
    # name: (D, pdims, k, k0, n, N, b, nf, pf)
    "helmholtz2d_bloch": ((1, 1, 0.5), (0, 1), 2 * np.pi * 0.8, (1.5, 0.5, 0.0), (17, 17, 9), 700, 4, (10, 10, 6), 4),
    "helmholtz2d_dense": ((1, 1, 0.5), (0, 1), 2 * np.pi * 0.8, (1.5, 0.5, 0.0), (17, 17, 9), 1600, 4, (10, 10, 6),
                          4),
    "helmholtz3d_bloch": ((1, 1, 1), (0, 1, 2), 2 * np.pi * 0.7, (0.9, 0.9, 0.0), (13, 13, 13), 500, 4, (8, 8, 8), 3),
    "helmholtz1d_z": ((1, 0.5, 0.5), (2,), 2 * np.pi * 0.5, (0, 0, 0.0), (9, 9, 17), 500, 3, (6, 6, 10), 3),
    "helmholtz1d_x_phase": ((1, 0.5, 0.5), (0,), 3.0, (1.2, 0, 0), (17, 9, 9), 400, 3, (10, 6, 6), 3),
    "npsp3d": ((1, 1, 1), (0, 1, 2), 0.0, (0, 0, 0), (13, 13, 13), 600, 4, (8, 8, 8), 4),
    "npsp2d": ((1, 1, 0.5), (0, 1), 0.0, (0, 0, 0), (13, 13, 7), 400, 4, (8, 8, 6), 4),
    "npsp1d": ((0.5, 0.5, 1), (2,), 0.0, (0, 0, 0), (7, 7, 13), 300, 3, (6, 6, 8), 3),
    "static_phase3d": ((1, 1, 1), (0, 1, 2), 0.0, (1.0, 0.4, 0.3), (13, 13, 13), 400, 4, (8, 8, 8), 4),
    "free_space": ((1, 1, 0.5), (), 4.0, (0, 0, 0), (17, 17, 9), 600, 4, (10, 10, 10), 4),
}


def make_case(name, seed=0):
    D, pdims, k, k0, n, N, b, nf, pf = CASES[name]
    npsp = len(pdims) > 0 and k == 0 and not any(k0)
    real = k == 0 and not any(k0)
    return inputs.random_case(N, D, pdims, k, k0, n, b=b, nf=nf, pf=pf, seed=seed + 3,
                              complex_q=not real, neutral=npsp)


@pytest.fixture(scope="module")
def oracle_cache():
    return {}


def oracle_results(name, cache):
    if name not in cache:
        W = make_case(name)
        o = oracle_plan(W)
        cache[name] = (W, o, o.apply(W.q), o.apply_adjoint(W.q))
    return cache[name]


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_forward_and_adjoint(name, oracle_cache):
    W, o, ue, we = oracle_results(name, oracle_cache)
    real = W.k == 0 and not any(W.k0)
    pl = gpu_plan(W, "fp64")
    q = to_dev(W.q, "fp64", real)
    u = pl.apply(q).cpu().numpy()
    w = pl.apply_adjoint(q).cpu().numpy()
    assert pl.device_status() == pim.PIM_OK
    assert rel(u, ue) < FP64_TOL, rel(u, ue)
    assert rel(w, we) < FP64_TOL, rel(w, we)
    pl.close()


@pytest.mark.parametrize("mode", [pim.PIM_CORR_FP64, pim.PIM_CORR_DOUBLE_FLOAT, pim.PIM_CORR_FP32,
                                  pim.PIM_CORR_COMPACT])
@pytest.mark.parametrize("name", ["helmholtz2d_bloch", "npsp3d", "helmholtz1d_z"])
def test_fp32_mixed_forward_and_adjoint(name, mode, oracle_cache):
    W, o, ue, we = oracle_results(name, oracle_cache)
    real = W.k == 0 and not any(W.k0)
    pl = gpu_plan(W, "fp32", corr_mode=mode)
    q = to_dev(W.q, "fp32", real)
    u = pl.apply(q).cpu().numpy()
    w = pl.apply_adjoint(q).cpu().numpy()
    assert rel(u, ue) < FP32_TOL, rel(u, ue)
    assert rel(w, we) < FP32_TOL, rel(w, we)
    pl.close()


@pytest.mark.parametrize("precision,mode", [("fp32", pim.PIM_CORR_DOUBLE_FLOAT), ("fp32", pim.PIM_CORR_FP32),
                                            ("fp32", pim.PIM_CORR_COMPACT), ("fp64", pim.PIM_CORR_FP64)])
@pytest.mark.parametrize("name", ["helmholtz2d_dense", "npsp3d"])
def test_every_gather_launch_shape(name, precision, mode, oracle_cache):
    """Each launch shape of the gather kernel the autotuner may pick, forced
    through the options, on rows long enough for every unrolled trip count
    and tail."""
    W, o, ue, we = oracle_results(name, oracle_cache)
    real = W.k == 0 and not any(W.k0)
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    nvar = None
    v = 0
    while nvar is None or v < nvar:
        pl = gpu_plan(W, precision, corr_mode=mode, gather_variant=v)
        info = pl.info()
        nvar = info.gather_variants
        assert info.gather_variant == v
        q = to_dev(W.q, precision, real)
        u = pl.apply(q).cpu().numpy()
        w = pl.apply_adjoint(q).cpu().numpy()
        assert pl.device_status() == pim.PIM_OK
        assert rel(u, ue) < tol, (v, rel(u, ue))
        assert rel(w, we) < tol, (v, rel(w, we))
        pl.close()
        v += 1
    assert nvar == 5
    with pytest.raises(Exception):
        gpu_plan(W, precision, corr_mode=mode, gather_variant=nvar)


def test_stage_parity_far_table_spread_and_correction(oracle_cache):
    W, o, ue, we = oracle_results("helmholtz2d_bloch", oracle_cache)
    pl = gpu_plan(W, "fp64")
    q = to_dev(W.q, "fp64", False)
    pl.apply(q)
    # far table (x fastest on the GPU, oracle indexed [x, y, z])
    F = pl.debug(0)
    Fo = np.transpose(o.F, (2, 1, 0))
    assert np.max(np.abs(F - Fo)) < 1e-12 * np.max(np.abs(Fo))
    # grid charges of step 1
    Q = pl.debug(1)
    Qo = opim.spread(tuple(o.P.n), o.s, o.w, o.P.p, o.regularise(W.q))
    assert np.max(np.abs(Q - np.transpose(Qo, (2, 1, 0)))) < 1e-13 * np.max(np.abs(Qo))
    # correction list: same pairs, same values (compare as sets per row)
    perm = pl.debug(3)
    rp = pl.debug(4)
    col = pl.debug(5)
    val = pl.debug(6)
    m, n, ii, c = o.corrections()
    assert len(col) == len(m)
    imgs = o.P.images()
    # GPU image order: iz, iy, ix nested -> same enumeration as the oracle's meshgrid(ij) on (x,y,z)? map by vector
    gpu_imgs = [(ix, iy, iz) for iz in range(-1 if 2 in W.pdims else 0, 2 if 2 in W.pdims else 1)
                for iy in range(-1 if 1 in W.pdims else 0, 2 if 1 in W.pdims else 1)
                for ix in range(-1 if 0 in W.pdims else 0, 2 if 0 in W.pdims else 1)]
    key_o = {}
    for mm, nn, i, cc in zip(m, n, ii, c):
        key_o[(int(mm), int(nn), tuple(imgs[i]))] = cc
    ph = {tuple(v): np.exp(-1j * np.dot(W.k0, np.array(v) * np.array(W.D))) for v in gpu_imgs}
    worst = 0.0
    scale = np.max(np.abs(c))
    for r in range(len(perm)):
        for t in range(rp[r], rp[r + 1]):
            nn = col[t] & ((1 << 25) - 1)
            img = gpu_imgs[col[t] >> 25]
            cc = key_o[(int(perm[r]), int(perm[nn]), img)]
            worst = max(worst, abs(ph[img] * val[t] - cc))
    assert worst < 1e-12 * scale
    pl.close()


@pytest.mark.parametrize("split", [0, 10, 20])
def test_compact_rows_split_by_magnitude(split, oracle_cache):
    """Compact mode: each row starts with its entries above 2^-split of the
    row's largest |d| (summed in double-float), the rest follow; the pairs and
    their FP64 values are those of the FP64 plan, and the apply matches the
    oracle."""
    W, o, ue, we = oracle_results("helmholtz2d_dense", oracle_cache)
    ref = gpu_plan(W, "fp64")
    rp, col, val = ref.debug(4), ref.debug(5), ref.debug(6)
    pl = gpu_plan(W, "fp32", corr_mode=pim.PIM_CORR_COMPACT, corr_split=split)
    assert np.array_equal(pl.debug(4), rp)
    col2, val2, nb = pl.debug(5), pl.debug(6), pl.debug(7)
    thr = 2.0 ** -split
    nsmall = 0
    for r in range(len(rp) - 1):
        a, b = rp[r], rp[r + 1]
        order = np.argsort(col[a:b], kind="stable")
        order2 = np.argsort(col2[a:b], kind="stable")
        assert np.array_equal(col[a:b][order], col2[a:b][order2])
        assert np.array_equal(val[a:b][order], val2[a:b][order2])
        mag = np.abs(val2[a:b])
        if b > a:
            big = mag > thr * mag.max() if split > 0 else np.ones(b - a, bool)
            assert nb[r] == big.sum()
            assert big[:nb[r]].all() and not big[nb[r]:].any()
            nsmall += (b - a) - nb[r]
    if split == 0:
        assert nsmall == 0
    else:
        assert nsmall > 0
    real = W.k == 0 and not any(W.k0)
    q = to_dev(W.q, "fp32", real)
    assert rel(pl.apply(q).cpu().numpy(), ue) < FP32_TOL
    assert rel(pl.apply_adjoint(q).cpu().numpy(), we) < FP32_TOL
    with pytest.raises(Exception):
        gpu_plan(W, "fp32", corr_mode=pim.PIM_CORR_COMPACT, corr_split=31)
    pl.close()
    ref.close()


def test_multiple_rhs_and_host_pointers(oracle_cache):
    W, o, ue, we = oracle_results("helmholtz2d_bloch", oracle_cache)
    pl = gpu_plan(W, "fp64")
    rng = np.random.default_rng(11)
    Q2 = np.stack([W.q, rng.standard_normal(W.N) + 1j * rng.standard_normal(W.N)], axis=1)
    u2 = pl.apply(np.ascontiguousarray(Q2))       # host numpy in, host out
    assert rel(u2[:, 0], ue) < FP64_TOL
    assert rel(u2[:, 1], o.apply(Q2[:, 1])) < FP64_TOL
    pl.close()


def test_full_size_coulomb3d_4k_fp64():
    # 3D-periodic static Coulomb, N = 4096, grid 32^3, p = 4, one near layer, FP64
    W = inputs.coulomb3d()
    o = oracle_plan(W)
    ue = o.apply(W.q)
    pl = gpu_plan(W, "fp64")
    u = pl.apply(torch.tensor(W.q, device="cuda")).cpu().numpy()
    assert rel(u, ue) < FP64_TOL
    pl.close()


def test_full_size_helmholtz2d_262k_sampled_rows():
    # 2D-periodic Helmholtz + Bloch, N = 262144, grid 128 x 128 x 64, FP32 bulk:
    # 256 sampled rows of the oracle (which the oracle computes one by one)
    W = inputs.helmholtz2d(nf=(21, 21, 11))
    pl = gpu_plan(W, "fp32")
    u = pl.apply(torch.tensor(W.q, device="cuda")).cpu().numpy()
    rows = np.random.default_rng(5).choice(W.N, 256, replace=False)
    o = oracle_plan(W)
    ue = o.apply_rows(W.q.astype(np.complex128), rows)
    assert rel(u[rows], ue) < FP32_TOL
    pl.close()


def test_edge_cases_faces_single_box_and_tiny():
    rng = np.random.default_rng(4)
    D = np.array([1.0, 1.0, 0.5])
    # points on the cell faces and corners, a cluster inside one box, ragged grid vs tiles
    pts = np.concatenate([
        np.array([[0, 0, 0], [1, 1, 0.5], [1, 0, 0.25], [0, 1, 0.4], [0.5, 0, 0.5]]),
        0.31 + 0.001 * rng.random((40, 3)) * D,
        rng.random((60, 3)) * D,
    ])
    W = inputs.Workload("edges", tuple(D), (0, 1), 5.0, (0.7, -0.3, 0.0), (11, 19, 6), 4, 1, 3, (7, 9, 5), 3,
                        "fp64", len(pts), 1, pts, rng.standard_normal(len(pts)) + 1j * rng.standard_normal(len(pts)))
    o = oracle_plan(W)
    ue = o.apply(W.q)
    pl = gpu_plan(W, "fp64")
    u = pl.apply(torch.tensor(W.q, device="cuda")).cpu().numpy()
    assert rel(u, ue) < FP64_TOL
    # a single point: only self images remain
    W1 = inputs.Workload("one", tuple(D), (0, 1), 5.0, (0.7, -0.3, 0.0), (11, 19, 6), 4, 1, 3, (7, 9, 5), 3,
                         "fp64", 1, 1, np.array([[0.3, 0.4, 0.2]]), np.array([1.0 + 0.5j]))
    o1 = oracle_plan(W1)
    pl1 = gpu_plan(W1, "fp64")
    u1 = pl1.apply(torch.tensor(W1.q, device="cuda")).cpu().numpy()
    assert rel(u1, o1.apply(W1.q)) < FP64_TOL
    pl.close()
    pl1.close()


def test_errors_are_status_codes():
    D = (1.0, 1.0, 1.0)
    pl = pim.Plan(D, (0, 1, 2), 0.0, (0, 0, 0), (9, 9, 9), p=4, precision="fp64", b=3, nf=(6, 6, 6))
    # apply before set_points
    with pytest.raises(pim.PimError) as e:
        pl.apply(torch.zeros(4, dtype=torch.float64, device="cuda"))
    assert e.value.status == pim.PIM_ERR_STATE
    # a point outside the cell
    with pytest.raises(pim.PimError) as e:
        pl.set_points(torch.tensor([[0.5, 0.5, 1.2]], dtype=torch.float64, device="cuda"))
    assert e.value.status == pim.PIM_ERR_OUT_OF_CELL
    # non-neutral charges in the neutral static case: device flag
    pts = torch.rand(50, 3, dtype=torch.float64, device="cuda")
    pl.set_points(pts)
    pl.apply(torch.ones(50, dtype=torch.float64, device="cuda"))
    assert pl.device_status() == pim.PIM_ERR_NOT_NEUTRAL
    assert pl.device_status() == pim.PIM_OK
    pl.close()
    # Wood anomaly: k L / (2 pi) = 1 with no phase shift in 2D -> k_z(1,0) = 0
    with pytest.raises(pim.PimError) as e:
        pim.Plan((1, 1, 0.5), (0, 1), 2 * np.pi, (0, 0, 0), (9, 9, 5), p=4, precision="fp64", b=2, nf=(6, 6, 5))
    assert e.value.status == pim.PIM_ERR_ANOMALY
    # unsupported p, non-integer D/h
    with pytest.raises(pim.PimError) as e:
        pim.Plan(D, (0,), 1.0, (0, 0, 0), (9, 9, 9), p=6, precision="fp64")
    assert e.value.status == pim.PIM_ERR_UNSUPPORTED
    with pytest.raises(pim.PimError) as e:
        pim.pim_plan_create(np.diag(D), 1, 1.0, (0, 0, 0), (0.3, 0.125, 0.125), 4, 1, pim.PIM_FP64)
    assert e.value.status == pim.PIM_ERR_ARG
    # two points that coincide modulo the lattice make Eq. 1 singular
    pl2 = pim.Plan((1, 1, 1), (0, 1, 2), 0.0, (0, 0, 0), (9, 9, 9), p=4, precision="fp64", b=3, nf=(6, 6, 6))
    with pytest.raises(pim.PimError) as e:
        pl2.set_points(torch.tensor([[0.2, 0.3, 0.4], [1.0, 0.5, 0.5], [0.0, 0.5, 0.5]], dtype=torch.float64,
                                    device="cuda"))
    assert e.value.status == pim.PIM_ERR_ARG
    pl2.close()
    # memory cap
    with pytest.raises(pim.PimError) as e:
        pim.Plan(D, (0, 1, 2), 1.0, (0, 0, 0), (33, 33, 33), p=4, precision="fp64", mem_cap=1 << 20)
    assert e.value.status == pim.PIM_ERR_OOM
