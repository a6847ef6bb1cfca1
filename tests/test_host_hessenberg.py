"""The solver's host-side GMRES least-squares update (csrc/dgx_hess.h: Givens
rotations on the Arnoldi Hessenberg matrix, rotated right-hand side, back
substitution), compiled here with g++ on its own, against numpy's dense least
squares: after k columns, y minimises ||beta e_1 - H_k y|| and the running
estimate |g_k| equals that minimum (Saad's GMRES)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2505_00384_gb300", "csrc", "dgx_hess.h")

HARNESS = r'''
#include "dgx_hess.h"
extern "C" int hess_lsq(int m, int k, const double *Hin, double beta, double *y, double *est) {
  dgx::Hess H(m);
  H.g.assign(m + 1, 0.0);
  H.g[0] = beta;
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i <= j + 1; ++i) H.h(i, j) = Hin[i * m + j];
    est[j] = H.add_column(j);
  }
  H.solve(k);
  for (int j = 0; j < k; ++j) y[j] = H.y[j];
  return 0;
}
'''


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("hess")
    src = d / "harness.cpp"
    src.write_text(HARNESS)
    so = d / "libhess.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I", os.path.dirname(HEADER), "-o", str(so),
                    str(src)], check=True)
    return C.CDLL(str(so))


def _run(lib, H, k, beta):
    m = H.shape[1]
    y, est = np.zeros(m), np.zeros(m)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    Hc = np.ascontiguousarray(H)
    lib.hess_lsq(m, k, dp(Hc), C.c_double(beta), dp(y), dp(est))
    return y[:k], est[:k]


@pytest.mark.parametrize("m", [1, 5, 20])
def test_least_squares_matches_numpy(lib, m):
    rng = np.random.default_rng(m)
    H = np.triu(rng.standard_normal((m + 1, m)), -1)  # upper Hessenberg
    beta = 2.5
    for k in range(1, m + 1):
        y, est = _run(lib, H, k, beta)
        rhs = np.zeros(k + 1)
        rhs[0] = beta
        yref, *_ = np.linalg.lstsq(H[:k + 1, :k], rhs, rcond=None)
        rmin = np.linalg.norm(rhs - H[:k + 1, :k] @ yref)
        assert np.abs(y - yref).max() <= 1e-10 * max(1.0, np.abs(yref).max())
        assert abs(est[-1] - rmin) <= 1e-12 * beta


def test_happy_breakdown_column(lib):
    """A zero subdiagonal (invariant Krylov space) gives a zero residual
    estimate and the exact solution of the square system."""
    m = 4
    rng = np.random.default_rng(7)
    H = np.triu(rng.standard_normal((m + 1, m)), -1)
    H[4, 3] = 0.0
    y, est = _run(lib, H, 4, 1.0)
    rhs = np.zeros(4)
    rhs[0] = 1.0
    assert est[-1] <= 1e-14 and np.allclose(H[:4, :4] @ y, rhs, atol=1e-12)
