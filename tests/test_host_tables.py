"""The 1D tables of the CUDA library, built on the host by libdgx.so
(dgx_basis_tables; no GPU needed), against numpy's Gauss-Legendre rule and
Legendre polynomials: the nodal GLL basis of Sec. 2 evaluated at the 2r+1
Gauss points of the consistent integrals and at the r+1 Gauss points of the
fast inverse of Sec. 3.3, the inverse of the latter, the weights, and the
centro-symmetry the kernels' even-odd storage relies on."""
import numpy as np
import pytest

from paper_2505_00384_gb300 import dgx


def _gll(n):
    # end points and the roots of P'_{n-1}, mapped to [0, 1]
    inner = np.polynomial.legendre.Legendre.basis(n - 1).deriv().roots()
    return 0.5 * (1.0 + np.concatenate([[-1.0], np.sort(inner.real), [1.0]]))


def _gauss(q):
    t, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (1.0 + t), 0.5 * w


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5, 6])
def test_basis_tables_against_numpy(r):
    T = dgx.dgx_basis_tables(r)
    N, Q = r + 1, 2 * r + 1
    xn = _gll(N)
    gq, wq = _gauss(Q)
    ga, wa = _gauss(N)
    assert np.allclose(T["gq"], gq, rtol=0, atol=1e-15) and np.allclose(T["wq"], wq, rtol=0, atol=1e-15)
    assert np.allclose(T["wa"], wa, rtol=0, atol=1e-15)
    # interpolation and differentiation of the nodal basis are exact on x^k, k <= r
    for k in range(N):
        assert np.abs(T["I"] @ xn ** k - gq ** k).max() <= 1e-13
        assert np.abs(T["Ia"] @ xn ** k - ga ** k).max() <= 1e-13
        dk = k * gq ** (k - 1) if k else np.zeros(Q)
        assert np.abs(T["D"] @ xn ** k - dk).max() <= 1e-11 * max(1, k)
    assert np.array_equal(T["IT"], T["I"].T) and np.array_equal(T["DT"], T["D"].T)
    assert np.array_equal(T["IIT"], T["IT"] ** 2) and np.array_equal(T["DDT"], T["DT"] ** 2)
    assert np.array_equal(T["IDT"], T["IT"] * T["DT"])
    assert np.abs(T["Ia"] @ T["P"] - np.eye(N)).max() <= 1e-12 and np.array_equal(T["PT"], T["P"].T)
    # centro-symmetry: interpolation even, differentiation odd under x -> 1 - x
    assert np.abs(T["I"][::-1, ::-1] - T["I"]).max() <= 1e-14
    assert np.abs(T["D"][::-1, ::-1] + T["D"]).max() <= 1e-11
    assert np.abs(T["P"][::-1, ::-1] - T["P"]).max() <= 1e-12


def test_basis_tables_arguments():
    for bad in (0, 7, -1):
        with pytest.raises(dgx.DgxError):
            dgx.dgx_basis_tables(bad)
    assert dgx.load().dgx_basis_tables(4, None, 0) == 7 * 9 * 5 + 3 * 25 + 2 * 9 + 5
