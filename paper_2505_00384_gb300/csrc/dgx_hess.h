// Host-side least-squares update of (F)GMRES (Saad, Iterative Methods for
// Sparse Linear Systems, Sec. 6.5.3): the Hessenberg matrix of the Arnoldi
// process reduced column by column by Givens rotations, the rotated
// right-hand side g = beta e_1 and the back substitution for y.  Pure C++ (no
// CUDA), included by the solver translation unit and compiled on its own by
// the CPU tests.
#pragma once

#include <cmath>
#include <vector>

namespace dgx {

struct Hess {
  int m;
  std::vector<double> H, cs, sn, g, y;
  explicit Hess(int m_) : m(m_), H((m_ + 1) * m_, 0.0), cs(m_), sn(m_), g(m_ + 1), y(m_) {}
  double &h(int i, int j) { return H[i * m + j]; }
  // new column j holds h(0..j+1, j); returns |residual estimate|
  double add_column(int j) {
    for (int i = 0; i < j; ++i) {
      const double a = h(i, j), b = h(i + 1, j);
      h(i, j) = cs[i] * a + sn[i] * b;
      h(i + 1, j) = -sn[i] * a + cs[i] * b;
    }
    const double a = h(j, j), b = h(j + 1, j);
    const double r = std::hypot(a, b);
    cs[j] = r == 0.0 ? 1.0 : a / r;
    sn[j] = r == 0.0 ? 0.0 : b / r;
    h(j, j) = r;
    h(j + 1, j) = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    return std::fabs(g[j + 1]);
  }
  void solve(int k) {
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int l = i + 1; l < k; ++l) s -= h(i, l) * y[l];
      y[i] = s / h(i, i);
    }
  }
};

}  // namespace dgx
