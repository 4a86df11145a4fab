"""Pins for oracle.pim, the FFT-PIM operator of Sec. 3 with a direct grid
convolution.  Each test checks the oracle against something other than
itself: the plain O(N^2) definition (Eq. 1-2), Ewald ground truth, the exact
near-zone sum that the correction must reproduce when every pair is
corrected (Eq. er), a dense conjugate transpose, an FFT convolution, and the
method's error trend in the interpolation order (Sec. 4.1)."""
import numpy as np
import pytest

from oracle import ewald, greens, pim
from paper_2312_02376_gb300 import inputs


def _dense_exact(pts, k, D=None, pdims=(), k0=(0, 0, 0), images=None):
    """sum over the given images of exp(-jk0.iL) G0(r_m - r_n - iL), self term dropped."""
    N = len(pts)
    if images is None:
        images = np.zeros((1, 3), np.int64)
    A = np.zeros((N, N), np.complex128)
    for i in images:
        sh = i * np.asarray(D if D is not None else np.ones(3))
        d = pts[:, None, :] - pts[None, :, :] - sh
        R = np.linalg.norm(d, axis=-1)
        if not i.any():
            np.fill_diagonal(R, 1.0)
        G = np.exp(-1j * np.dot(np.asarray(k0, complex), sh)) * greens.G0(R, k)
        if not i.any():
            np.fill_diagonal(G, 0.0)
        A += G
    return A


@pytest.mark.parametrize("k", [0.0, 4.0])
def test_all_pairs_corrected_equals_exact_sum_nonperiodic(k):
    # With every pair corrected, Eq. er replaces the whole grid interaction
    # by the exact kernel: the result is Eq. 1 with G0, to round-off.
    rng = np.random.default_rng(1)
    pts = rng.random((90, 3)) * np.array([1, 1, 0.5])
    q = rng.standard_normal(90) + 1j * rng.standard_normal(90)
    P = pim.Params(D=(1, 1, 0.5), pdims=(), k=k, k0=(0, 0, 0), n=(12, 12, 7), p=4, layers=0, b=100)
    u = pim.Plan(P, pts).apply(q)
    ex = _dense_exact(pts, k) @ q
    assert np.linalg.norm(u - ex) / np.linalg.norm(ex) < 1e-12


def test_all_pairs_corrected_periodic_near_part_exact():
    # 2D-periodic, Bloch phase: with every (pair, near image) corrected, the
    # near part is the exact truncated image sum of Eq. 4.
    rng = np.random.default_rng(2)
    pts = rng.random((70, 3)) * np.array([1, 1, 0.5])
    q = rng.standard_normal(70) + 1j * rng.standard_normal(70)
    k = 2 * np.pi * 0.8
    k0 = (0.3 * k, 0.1 * k, 0.0)
    P = pim.Params(D=(1, 1, 0.5), pdims=(0, 1), k=k, k0=k0, n=(10, 10, 6), p=4, layers=1, b=100,
                   nf=(8, 8, 6), pf=4)
    pl = pim.Plan(P, pts)
    u = pl.apply(q)
    far = pim.far_apply(P, pl.F, pl.ss, pl.ws, pl.so, pl.wo, q)
    ex = _dense_exact(pts, k, P.D, P.pdims, k0, P.images()) @ q
    assert np.linalg.norm(u - far - ex) / np.linalg.norm(ex) < 1e-12


def test_separable_correction_equals_explicit_double_sum():
    rng = np.random.default_rng(3)
    pts = rng.random((120, 3))
    P = pim.Params(D=(1, 1, 1), pdims=(0, 1, 2), k=3.0, k0=(1.0, 0.5, 0.2), n=(12, 12, 12), p=4, layers=1, b=4)
    s, w, B, _ = pim.near_stencils(P, pts)
    m, n, ii = pim.correction_pairs(P, B)
    sel = np.random.default_rng(0).choice(len(m), 1500, replace=False)
    a = pim.correction_values_explicit(P, pts, s, w, m[sel], n[sel], ii[sel])
    b = pim.correction_values(P, pts, s, w, m[sel], n[sel], ii[sel])
    assert np.max(np.abs(a - b)) < 1e-14 * np.max(np.abs(a))


def test_direct_convolution_matches_fft_convolution():
    P = pim.Params(D=(1, 1, 1), pdims=(0, 1, 2), k=2.0, k0=(0.5, 0.0, 0.3), n=(9, 7, 6), p=2, layers=1)
    K = pim.near_table(P)
    rng = np.random.default_rng(4)
    Q = rng.standard_normal(tuple(P.n)) + 1j * rng.standard_normal(tuple(P.n))
    U = pim.conv_direct_full(P, K, Q)
    # linear convolution by zero-padded FFT, sizes 3n-2
    sh = tuple(3 * P.n - 2)
    full = np.fft.ifftn(np.fft.fftn(K, sh, axes=(0, 1, 2)) * np.fft.fftn(Q, sh, axes=(0, 1, 2)))
    n = P.n
    assert np.allclose(U, full[n[0] - 1:2 * n[0] - 1, n[1] - 1:2 * n[1] - 1, n[2] - 1:2 * n[2] - 1], atol=1e-12)
    nodes = np.array([[0, 0, 0], [8, 6, 5], [3, 2, 4]])
    assert np.allclose(pim.conv_direct_at(P, K, Q, nodes), U[nodes[:, 0], nodes[:, 1], nodes[:, 2]], atol=1e-12)


def test_apply_rows_equals_apply():
    W = inputs.random_case(150, (1, 1, 0.5), (0, 1), 5.0, (1.0, 0.5, 0.0), (10, 10, 6), b=3, nf=(8, 8, 6))
    P = pim.Params(D=W.D, pdims=W.pdims, k=W.k, k0=W.k0, n=W.n, p=W.p, layers=1, b=W.b, nf=W.nf, pf=4)
    pl = pim.Plan(P, W.points)
    u = pl.apply(W.q)
    rows = np.array([0, 17, 99, 149])
    assert np.allclose(pl.apply_rows(W.q, rows), u[rows], rtol=1e-12, atol=1e-12 * np.abs(u).max())


@pytest.mark.parametrize("case", ["helmholtz2d", "npsp3d", "helmholtz1d", "lossy2d", "lossy1d", "lossy3d"])
def test_adjoint_is_conjugate_transpose(case):
    # the lossy cases have complex k and complex phase shifts (Sec. 2): the
    # image phases then have modulus != 1 and the adjoint's differ from them
    rng = np.random.default_rng(5)
    N = 30
    if case == "helmholtz2d":
        P = pim.Params(D=(1, 1, 0.5), pdims=(0, 1), k=4.0, k0=(1.2, 0.4, 0.0), n=(8, 8, 6), p=3, layers=1, b=2,
                       nf=(6, 6, 5), pf=3)
    elif case == "lossy2d":
        P = pim.Params(D=(1, 1, 0.5), pdims=(0, 1), k=4.0 - 0.6j, k0=(1.2 - 0.3j, 0.4 + 0.2j, 0.0), n=(8, 8, 6), p=3,
                       layers=1, b=2, nf=(6, 6, 5), pf=3)
    elif case == "lossy1d":
        P = pim.Params(D=(0.5, 0.5, 1.0), pdims=(2,), k=3.0 - 0.4j, k0=(0, 0, 0.8 - 0.2j), n=(6, 6, 8), p=2, layers=1,
                       b=2, nf=(5, 5, 6), pf=2)
    elif case == "lossy3d":
        P = pim.Params(D=(1, 1, 1), pdims=(0, 1, 2), k=3.0 - 0.5j, k0=(1.0 - 0.2j, 0.5 + 0.1j, -0.3j), n=(8, 8, 8),
                       p=2, layers=1, b=2, nf=(5, 5, 5), pf=2)
    elif case == "helmholtz1d":
        P = pim.Params(D=(0.5, 0.5, 1.0), pdims=(2,), k=3.0, k0=(0, 0, 0.0), n=(6, 6, 8), p=2, layers=1, b=2,
                       nf=(5, 5, 6), pf=2)
    else:
        P = pim.Params(D=(1, 1, 1), pdims=(0, 1, 2), k=0.0, k0=(0, 0, 0), n=(8, 8, 8), p=2, layers=1, b=2,
                       nf=(5, 5, 5), pf=2)
    pts = rng.random((N, 3)) * P.D
    pl = pim.Plan(P, pts)
    E = np.eye(N, dtype=complex)
    if P.npsp:
        # the forward operator is defined on neutral inputs: use the basis of
        # the neutral subspace e_j - mean
        cols = [pl.apply(E[:, j] - 1.0 / N) for j in range(N)]
    else:
        cols = [pl.apply(E[:, j]) for j in range(N)]
    A = np.array(cols).T
    AH = np.array([pl.apply_adjoint(E[:, j]) for j in range(N)]).T
    if P.npsp:
        Pm = np.eye(N) - 1.0 / N
        assert np.allclose(AH, Pm @ A.conj().T, atol=1e-12 * np.abs(A).max())
    else:
        assert np.allclose(AH, A.conj().T, atol=1e-12 * np.abs(A).max())


def _dense(pl, N):
    E = np.eye(N, dtype=complex)
    return np.array([pl.apply(E[:, j]) for j in range(N)]).T


def test_reciprocity_free_space_is_exact():
    # G0(r) = G0(-r) and the spread and gather share their weights, so the
    # discrete free-space operator W K W^T + C is complex symmetric to
    # round-off (reciprocity; a sign slip in the grid kernel's offsets or in
    # the correction's pair order breaks it)
    rng = np.random.default_rng(8)
    N = 40
    P = pim.Params(D=(1, 1, 0.5), pdims=(), k=5.0, k0=(0, 0, 0), n=(9, 9, 6), p=3, layers=0, b=2)
    pts = rng.random((N, 3)) * P.D
    A = _dense(pim.Plan(P, pts), N)
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()


def test_reciprocity_bloch_swaps_the_phase():
    # periodic with a Bloch phase: A(k0)^T = A(-k0) (the image phase
    # exp(-j k0.(iL)) of pair (m, n) is that of (n, m) with -i).  The near
    # part and the corrections satisfy it exactly; the far part, whose source
    # and observer grids are half a step apart (Eq. grid), only up to its
    # interpolation error, which falls as the far grid is refined.  A wrong
    # phase sign would leave an O(1) difference.
    N = 40
    pts = np.random.default_rng(9).random((N, 3)) * np.array([1, 1, 0.5])

    def asym(nf, pf):
        kw = dict(D=(1, 1, 0.5), pdims=(0, 1), k=4.0, n=(9, 9, 6), p=3, layers=1, b=3, nf=nf, pf=pf)
        A = _dense(pim.Plan(pim.Params(k0=(1.1, 0.5, 0.0), **kw), pts), N)
        B = _dense(pim.Plan(pim.Params(k0=(-1.1, -0.5, 0.0), **kw), pts), N)
        nA = np.linalg.norm(A)
        return np.linalg.norm(A.T - B) / nA, np.linalg.norm(A.T - A) / nA

    coarse, _ = asym((8, 8, 6), 3)
    fine, unswapped = asym((16, 16, 10), 4)
    assert fine < 1e-4 and fine < coarse / 20, (coarse, fine)
    assert unswapped > 0.1


def test_method_error_falls_with_order_lossy_periodic():
    # Sec. 4.1: the error falls with interpolation order; reference = Eq. 2
    # summed by brute force (converges for Im k < 0).
    rng = np.random.default_rng(6)
    N = 220
    D = np.array([1.0, 1.0, 0.5])
    pts = rng.random((N, 3)) * D
    q = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    k = 6.0 - 2.5j
    k0 = (0.8, -0.5, 0.0)
    imgs = greens.image_offsets((0, 1), 14)
    ref = _dense_exact(pts, k, D, (0, 1), k0, imgs) @ q
    errs = []
    for p in (2, 4):
        P = pim.Params(D=D, pdims=(0, 1), k=k, k0=k0, n=(17, 17, 9), p=p, layers=1, b=p + 1,
                       nf=(14, 14, 8), pf=p)
        u = pim.Plan(P, pts).apply(q)
        errs.append(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    assert errs[1] < 0.2 * errs[0]
    assert errs[1] < 3e-4


def test_npsp3d_vs_ewald_within_method_error():
    W = inputs.coulomb3d(N=512, n=16)
    P = pim.Params(D=W.D, pdims=W.pdims, k=0.0, k0=W.k0, n=W.n, p=4, layers=1, b=5, nf=W.nf, pf=4)
    u = pim.Plan(P, W.points).apply(W.q)
    ref = ewald.potential(W.points, W.q.astype(complex), np.arange(W.N), W.D, W.pdims, 0.0, np.zeros(3), 6.0)
    e = u - ref
    e -= e.mean()          # Eq. lgf and the Ewald sum differ by a constant
    assert np.linalg.norm(e) / np.linalg.norm(ref - ref.mean()) < 2e-4


def test_helmholtz1d_vs_1d_ewald_error_falls_with_correction_radius():
    # The batched 1D-periodic workload's recipe (smallest of its sets, p = 4,
    # grid step half the mean point spacing): sampled rows of the operator
    # against the 1D-lattice Ewald ground truth.  The method error falls with
    # the correction radius b and is below 1e-4 at the recipe's b = 5 (7e-5;
    # on a grid with one node per point b = 5 is needed as well, with a
    # correction list about eight times longer).
    pytest.importorskip("mpmath")
    W = inputs.helmholtz1d_set(11294, rng=np.random.default_rng(17))
    q = (W.q[:, 0] if W.q.ndim == 2 else W.q).astype(complex)
    rows = np.random.default_rng(3).choice(W.N, 12, replace=False)
    ref = ewald.potential(W.points, q, rows, W.D, W.pdims, W.k, W.k0, 2.0)
    err = []
    for b in (2, 3, 5):
        P = pim.Params(D=W.D, pdims=W.pdims, k=W.k, k0=W.k0, n=W.n, p=4, layers=1, b=b, nf=W.nf, pf=4)
        u = pim.Plan(P, W.points).apply_rows(q, rows)
        err.append(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    assert err[0] > err[1] > err[2], err
    assert err[2] < 1e-4, err


def test_coulomb3d_4k_recipe_vs_ewald_rows():
    # The 3D Coulomb workload at full size (N = 4096, 32^3, p = 4, b = 5):
    # sampled rows of the operator against the Ewald sum, within the method
    # error target 1e-4 (the charges are exactly neutral, so Eq. lgf's free
    # constant drops out)
    W = inputs.coulomb3d()
    P = pim.Params(D=W.D, pdims=W.pdims, k=0.0, k0=W.k0, n=W.n, p=W.p, layers=W.layers, b=W.b, nf=W.nf, pf=W.pf)
    rows = np.random.default_rng(4).choice(W.N, 48, replace=False)
    u = pim.Plan(P, W.points).apply_rows(W.q.astype(complex), rows)
    ref = ewald.potential(W.points, W.q.astype(complex), rows, W.D, W.pdims, 0.0, np.zeros(3), 6.0)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-4


def test_error_converges_in_near_image_layers():
    # Sec. 3.3: the near kernel sums the images |i| <= i_d, the far series the
    # rest (Eq. 4).  Against the Ewald sum the 2D Helmholtz recipe's error
    # drops by more than an order of magnitude from i_d = 0 to 1 and then
    # settles at the grid's level (convergence in image count)
    W = inputs.helmholtz2d(N=3000, n=(24, 24, 12), nf=(14, 14, 8), b=5)
    q = W.q.astype(complex)
    rows = np.random.default_rng(5).choice(W.N, 24, replace=False)
    ref = ewald.potential(W.points, q, rows, W.D, W.pdims, W.k, W.k0, 4.0)
    err = []
    for layers in (0, 1, 2):
        P = pim.Params(D=W.D, pdims=W.pdims, k=W.k, k0=W.k0, n=W.n, p=4, layers=layers, b=W.b, nf=W.nf, pf=4)
        u = pim.Plan(P, W.points).apply_rows(q, rows)
        err.append(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    assert err[1] < err[0] / 10, err
    assert abs(err[2] - err[1]) < 0.3 * err[1] and err[2] < 1e-3, err


def test_far_table_against_ewald():
    # F(delta) = G^p - G_near at delta*Delta + Delta/2, checked pointwise
    # against the Ewald sum minus the same near images.
    P = pim.Params(D=(1, 1, 0.5), pdims=(0, 1), k=2 * np.pi * 0.8, k0=(1.5, 0.5, 0.0), n=(8, 8, 6), p=4,
                   layers=1, nf=(6, 6, 4), pf=3)
    F = pim.far_table(P)
    dF = P.delta_f
    for dl in [(0, 0, 0), (-5, 3, -3), (5, -5, 3), (2, 1, -1)]:
        r = np.array(dl) * dF + 0.5 * dF
        e = ewald.greens_function(r, P.D, P.pdims, P.k, P.k0, 3.0)[0]
        e -= greens.image_sum(r[None], P.D, P.pdims, P.k, P.k0, P.images())[0]
        got = F[tuple(np.array(dl) + P.nf - 1)]
        assert abs(got - e) < 1e-12 * max(1.0, abs(e))


def test_npsp_neutrality_and_constant_invariance():
    W = inputs.coulomb3d(N=64, n=8)
    P = pim.Params(D=W.D, pdims=W.pdims, k=0.0, k0=W.k0, n=W.n, p=2, layers=1, b=3, nf=(5, 5, 5), pf=2)
    pl = pim.Plan(P, W.points)
    u = pl.apply(W.q)
    with pytest.raises(ValueError):
        pl.apply(W.q + 0.01)
    # Eq. lgf is defined up to a constant: shifting the far table by one does
    # not change the potential of a neutral source set.
    pl2 = pim.Plan(P, W.points, F=pl.F + 7.25)
    assert np.allclose(pl2.apply(W.q), u, atol=1e-12 * np.abs(u).max())


def test_bloch_phase_when_a_source_crosses_the_cell():
    # Eq. 2: moving a source by a lattice vector a with its amplitude scaled
    # by exp(-j k0.a) leaves every other potential unchanged, and the
    # potential at the moved point scales by exp(-j k0.a); exact for the
    # definition, at method-error level for FFT-PIM.
    rng = np.random.default_rng(8)
    N = 200
    D = np.array([1.0, 1.0, 0.5])
    pts = rng.random((N, 3)) * D
    pts[0, 0] = 0.0
    q = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    k = 2 * np.pi * 0.8
    k0 = np.array([0.3 * k, 0.1 * k, 0.0])
    P = pim.Params(D=D, pdims=(0, 1), k=k, k0=k0, n=(17, 17, 9), p=4, layers=1, b=5, nf=(14, 14, 8), pf=4)
    u1 = pim.Plan(P, pts).apply(q)
    pts2 = pts.copy()
    pts2[0, 0] = 1.0
    q2 = q.copy()
    ph = np.exp(-1j * k0[0] * 1.0)
    q2[0] *= ph
    u2 = pim.Plan(P, pts2).apply(q2)
    scale = np.linalg.norm(u1)
    assert np.linalg.norm(u2[1:] - u1[1:]) / scale < 3e-4
    assert abs(u2[0] - ph * u1[0]) / np.abs(u1).mean() < 3e-3


@pytest.mark.parametrize("case", ["helmholtz2d", "npsp3d"])
def test_position_gradient_matches_finite_differences(case):
    # d/dr Re <g, A(r) q> with the stencils, boxes and pair list frozen at r
    rng = np.random.default_rng(13)
    N = 50
    if case == "helmholtz2d":
        P = pim.Params(D=(1, 1, 0.5), pdims=(0, 1), k=4.0, k0=(1.2, 0.4, 0.0), n=(9, 9, 6), p=3, layers=1, b=3,
                       nf=(7, 7, 5), pf=3)
        q = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    else:
        P = pim.Params(D=(1, 1, 1), pdims=(0, 1, 2), k=0.0, k0=(0, 0, 0), n=(9, 9, 9), p=4, layers=1, b=4,
                       nf=(6, 6, 6), pf=4)
        q = rng.standard_normal(N)
        q = (q - q.mean()).astype(complex)
    pts = rng.random((N, 3)) * P.D * 0.98 + 0.01 * P.D
    g = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    base = pim.Plan(P, pts)
    G = base.position_grad(q, g)
    eps = 1e-6
    for k in (0, 17, 41):
        for d in range(3):
            pp = pts.copy()
            pp[k, d] += eps
            up = pim.Plan(P, pp, K=base.K, F=base.F, frozen=base).apply(q)
            pp[k, d] -= 2 * eps
            um = pim.Plan(P, pp, K=base.K, F=base.F, frozen=base).apply(q)
            fd = np.real(np.vdot(g, up) - np.vdot(g, um)) / (2 * eps)
            assert abs(fd - G[k, d]) < 1e-7 * np.abs(G).max()


def test_position_gradient_all_pairs_equals_exact_gradient():
    # every pair corrected, no periodicity: A is the exact kernel matrix, so
    # the gradient is the closed form of d/dr_k Re sum conj(g_m) G0(r_m-r_n) q_n
    rng = np.random.default_rng(14)
    N, k = 40, 3.0
    pts = rng.random((N, 3)) * np.array([1, 1, 0.5])
    q = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    g = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    P = pim.Params(D=(1, 1, 0.5), pdims=(), k=k, k0=(0, 0, 0), n=(10, 10, 6), p=4, layers=0, b=100)
    G = pim.Plan(P, pts).position_grad(q, g)
    d = pts[:, None, :] - pts[None, :, :]
    R = np.linalg.norm(d, axis=-1)
    np.fill_diagonal(R, 1.0)
    dG = (greens.G0(R, k) * (-1j * k - 1.0 / R) / R)[..., None] * d   # grad wrt r_m of G0(r_m - r_n)
    dG[np.arange(N), np.arange(N)] = 0
    # observer side: conj(g_k) dG[k, n] q_n; source side: conj(g_m) d/dr_k G0(r_m - r_k) q_k = -dG[m, k]
    ref2 = np.zeros((N, 3))
    for kk in range(N):
        for dd in range(3):
            ref2[kk, dd] = np.real(np.sum(np.conj(g[kk]) * dG[kk, :, dd] * q)) + \
                np.real(np.sum(np.conj(g) * (-dG[:, kk, dd]) * q[kk]))
    assert np.allclose(G, ref2, rtol=0, atol=1e-10 * np.abs(ref2).max())


def test_full_size_helmholtz2d_rows_vs_ewald_golden():
    # the 262144-point 2D Helmholtz workload: FFT-PIM rows vs the committed
    # Ewald ground truth (tests/golden/make_helmholtz2d_262k_ewald_rows.py)
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "helmholtz2d_262k_ewald_rows.txt")
    d = np.loadtxt(path, comments="#")
    rows, ref = d[:, 0].astype(np.int64), d[:, 1] + 1j * d[:, 2]
    W = inputs.helmholtz2d()
    P = pim.Params(D=W.D, pdims=W.pdims, k=W.k, k0=W.k0, n=W.n, p=W.p, layers=W.layers, b=W.b, nf=W.nf, pf=W.pf)
    u = pim.Plan(P, W.points).apply_rows(W.q.astype(np.complex128), rows)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 5e-5


def test_far_sum_equals_the_dense_operator():
    """Eq. 8 as the oracle sums it (directly, and by FFT convolution for large
    far grids) equals the dense matrix A[a, b] = F(a - b) applied to the
    source-grid charges, forward and adjoint."""
    rng = np.random.default_rng(4)
    P = pim.Params(D=(1, 1, 0.5), pdims=(0, 1), k=5.0, k0=(0.7, -0.3, 0), n=(9, 9, 5), nf=(7, 6, 5), pf=3)
    nf = tuple(int(v) for v in P.nf)
    F = rng.standard_normal(tuple(2 * v - 1 for v in nf)) + 1j * rng.standard_normal(tuple(2 * v - 1 for v in nf))
    qg = rng.standard_normal(nf) + 1j * rng.standard_normal(nf)
    A = pim.far_matrix(P, F)
    u = (A @ qg.ravel()).reshape(nf)
    w = (A.conj().T @ qg.ravel()).reshape(nf)
    for direct in (True, False):
        assert np.abs(pim.far_sum(P, F, qg, direct=direct) - u).max() < 1e-12 * np.abs(u).max()
        assert np.abs(pim.far_sum(P, F, qg, adjoint=True, direct=direct) - w).max() < 1e-12 * np.abs(w).max()



def test_lossy_operator_vs_direct_lattice_sum():
    """A lossy wavenumber with a complex phase shift (2D lattice): the image
    sum of Eq. 2 converges absolutely, so the operator's rows can be checked
    against the lattice summed directly (the n = m, image-0 term left out,
    reading of Eq. 5), within the method error at p = 4."""
    rng = np.random.default_rng(23)
    N = 60
    D = np.array([1.0, 1.0, 0.5])
    k = 2 * np.pi * 0.8 - 1.0j
    k0 = np.array([1.0 - 0.3j, 0.5 + 0.2j, 0.0])
    P = pim.Params(D=tuple(D), pdims=(0, 1), k=k, k0=tuple(k0), n=(17, 17, 9), p=4, layers=1, b=4, nf=(12, 12, 8),
                   pf=4)
    pts = rng.random((N, 3)) * D
    q = (rng.standard_normal(N) + 1j * rng.standard_normal(N)) * np.sqrt(0.5)
    u = pim.Plan(P, pts).apply(q)
    # net decay of an image term: exp(Im k |iL|) |exp(-j k0.iL)| <= exp(-(1.0 - 0.3 sqrt 2)|i|)
    I = 40
    ref = np.zeros(N, complex)
    d = pts[:, None, :] - pts[None, :, :]
    for ix in range(-I, I + 1):
        for iy in range(-I, I + 1):
            sh = np.array([ix, iy, 0.0]) * D
            R = np.linalg.norm(d - sh, axis=-1)
            if ix == 0 and iy == 0:
                np.fill_diagonal(R, np.inf)
            ref += np.exp(-1j * np.dot(k0, sh)) * (np.exp(-1j * k * R) / (4 * np.pi * R)) @ q
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-3


def test_observers_vs_ewald_same_error_as_the_sources_rows():
    """Potentials at observer points apart from the sources (Sec. 4.1's
    accuracy test) against the Ewald sum at those points: the method error
    there is that of the sources' own rows (both fall with the grid step)."""
    rng = np.random.default_rng(1)
    N, M = 400, 24
    D = np.array([1.0, 1.0, 1.0])
    k, k0 = 2 * np.pi * 0.7, np.array([0.9, 0.5, 0.0])
    src, obs = rng.random((N, 3)), rng.random((M, 3))
    q = (rng.standard_normal(N) + 1j * rng.standard_normal(N)) * np.sqrt(0.5)
    P = pim.Params(D=tuple(D), pdims=(0, 1, 2), k=k, k0=tuple(k0), n=(33, 33, 33), p=4, layers=1, b=5,
                   nf=(16, 16, 16), pf=4)
    u = pim.apply_observers(P, src, obs, q)
    ref = ewald.potential(np.vstack([src, obs]), np.concatenate([q, np.zeros(M)]), np.arange(N, N + M), D,
                          (0, 1, 2), k, k0, 3.0)
    us = pim.Plan(P, src).apply_rows(q, np.arange(M))
    ref_s = ewald.potential(src, q, np.arange(M), D, (0, 1, 2), k, k0, 3.0)
    e_obs = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    e_src = np.linalg.norm(us - ref_s) / np.linalg.norm(ref_s)
    assert e_obs < 3e-4 and e_obs < 1.5 * e_src, (e_obs, e_src)


def test_observers_adjoint_is_conjugate_transpose():
    rng = np.random.default_rng(4)
    N, M = 25, 7
    for P in (pim.Params(D=(1, 1, 0.5), pdims=(0, 1), k=4.0 - 0.3j, k0=(1.2 - 0.2j, 0.4, 0.0), n=(8, 8, 6), p=3,
                         layers=1, b=2, nf=(6, 6, 5), pf=3),
              pim.Params(D=(1, 1, 1), pdims=(0, 1, 2), k=0.0, k0=(0, 0, 0), n=(8, 8, 8), p=2, layers=1, b=2,
                         nf=(5, 5, 5), pf=2)):
        src, obs = rng.random((N, 3)) * P.D, rng.random((M, 3)) * P.D
        E = np.eye(N)
        if P.npsp:
            A = np.array([pim.apply_observers(P, src, obs, E[:, j] - 1.0 / N) for j in range(N)]).T
            proj = np.eye(N) - 1.0 / N
        else:
            A = np.array([pim.apply_observers(P, src, obs, E[:, j]) for j in range(N)]).T
            proj = np.eye(N)
        AH = np.array([pim.apply_observers_adjoint(P, src, obs, np.eye(M)[:, j]) for j in range(M)]).T
        assert np.allclose(AH, proj @ A.conj().T, atol=1e-12 * np.abs(A).max())


def test_coax_neutral_static_axis_is_flat_at_the_coax_voltage():
    """The 1D-periodic neutral coax (inner radius 1, charge +1 per period;
    outer radius 2, charge -1): the potential is constant on the axis and
    outside the outer cylinder, and their difference is the coax voltage
    ln(r2/r1) / (2 pi) per unit charge per period (the exact values for
    uniformly charged cylinders, which the regular lattices of charges
    reproduce to exponentially small ripple at these distances)."""
    src, q, obs = inputs.coax()
    P = pim.Params(D=(5.0, 5.0, 1.0), pdims=(2,), k=0.0, k0=(0, 0, 0), n=(51, 51, 11), p=4, layers=1, b=5,
                   nf=(24, 24, 10), pf=4)
    u = pim.apply_observers(P, src, obs, q).real
    ua, uo = u[:8], u[8:]
    dv = ua.mean() - uo.mean()
    exact = np.log(2.0) / (2 * np.pi)
    assert np.ptp(ua) < 2e-5 * dv and np.ptp(uo) < 2e-5 * dv, (np.ptp(ua) / dv, np.ptp(uo) / dv)
    assert abs(dv - exact) < 1e-5 * exact, (dv, exact)
