"""The compact correction-value representation (host arithmetic, no GPU).

Compact rows keep, per row, the entries with |d| > 2^-s max_row |d| as an
FP32 head plus a bf16 tail of the FP64 remainder, and the others as their
FP32 head alone.  This checks, on the oracle's FP64 values (Eq. er) of a small
2D-periodic Helmholtz case, the bound the library states (every stored
component within 2^-33 of its row's largest |d| for s = 10) and the size of
the change in u it causes when summed exactly, against the error of plain
complex64 values.  The emulation uses numpy/torch roundings only (FP64 ->
FP32 and FP32 -> bf16, both to nearest even), not the library."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import pim as opim  # noqa: E402
from paper_2312_02376_gb300 import inputs  # noqa: E402


def _compact(c, m, split):
    """stored values of the compact rows for FP64 values c in rows m"""
    a = np.abs(c)
    rmax = np.zeros(m.max() + 1)
    np.maximum.at(rmax, m, a)
    big = a > 2.0 ** -split * rmax[m] if split > 0 else np.ones(len(c), bool)

    def part(x):
        head = x.astype(np.float32).astype(np.float64)
        tail = torch.tensor((x - head).astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
        return head, tail

    hr, tr = part(c.real)
    hi, ti = part(c.imag)
    stored = np.where(big, (hr + tr) + 1j * (hi + ti), hr + 1j * hi)
    return stored, rmax, big


@pytest.fixture(scope="module")
def case():
    W = inputs.random_case(500, (1.0, 1.0, 0.5), (0, 1), 2 * np.pi * 0.8, (1.5, 0.5, 0.0), (17, 17, 9), b=4,
                           nf=(10, 10, 6), pf=4, seed=21)
    P = opim.Params(D=W.D, pdims=W.pdims, k=W.k, k0=W.k0, n=W.n, p=4, layers=1, b=W.b, nf=W.nf, pf=W.pf)
    o = opim.Plan(P, W.points)
    m, n, ii, c = o.corrections()
    q = o.regularise(W.q.astype(complex))
    return W, o, m, n, c, q


def _corr(c, m, n, q, N):
    t = c * q[n]
    return np.bincount(m, weights=t.real, minlength=N) + 1j * np.bincount(m, weights=t.imag, minlength=N)


def test_stored_values_within_two_to_minus_33_of_the_row_maximum(case):
    W, o, m, n, c, q = case
    stored, rmax, big = _compact(c, m, 10)
    err = np.maximum(np.abs(stored.real - c.real), np.abs(stored.imag - c.imag))
    assert np.all(err <= 2.0 ** -33 * rmax[m] * (1 + 1e-12))
    # the small entries alone would break the bound at FP32 without the split
    assert 0.3 < 1 - big.mean() < 0.99


def test_compact_rows_change_u_far_less_than_complex64_values(case):
    W, o, m, n, c, q = case
    N = len(q)
    u = o.apply(W.q.astype(complex))
    exact = _corr(c, m, n, q, N)
    e_compact = np.linalg.norm(_corr(_compact(c, m, 10)[0], m, n, q, N) - exact) / np.linalg.norm(u)
    c32 = c.real.astype(np.float32).astype(np.float64) + 1j * c.imag.astype(np.float32).astype(np.float64)
    e_fp32 = np.linalg.norm(_corr(c32, m, n, q, N) - exact) / np.linalg.norm(u)
    e_all12 = np.linalg.norm(_corr(_compact(c, m, 0)[0], m, n, q, N) - exact) / np.linalg.norm(u)
    assert e_compact < 1e-9
    assert e_all12 <= e_compact < e_fp32 / 10
