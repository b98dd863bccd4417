// 1D GLL / Gauss-Legendre tables and the Lagrange basis on GLL nodes (Sec. 3:
// spectral elements on GLL nodes; Sec. 5: Gauss-Legendre interface quadrature),
// shared by the host setup of the box and the general-hexahedron paths.
#pragma once

#include <cmath>
#include <vector>

namespace dgtab {

// ---------------------------------------------------------------------------
// 1D tables
// ---------------------------------------------------------------------------
// Legendre P_n at x (three-term recurrence); also returns P_{n-1}.
inline void legendre(int n, double x, double* pn, double* pnm1) {
  double a = 1.0, b = x;
  if (n == 0) { *pn = 1.0; *pnm1 = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    const double c = ((2.0 * k - 1.0) * x * b - (k - 1.0) * a) / k;
    a = b;
    b = c;
  }
  *pn = b;
  *pnm1 = a;
}

// GLL nodes by the Lobatto fixed-point Newton step
//   x <- x - (x P_N - P_{N-1}) / ((N+1) P_N),
// whose fixed points are the roots of (1 - x^2) P_N'; weights 2/(N(N+1)P_N^2).
inline void gll(int N, std::vector<double>& x, std::vector<double>& w) {
  x.assign(N + 1, 0.0);
  w.assign(N + 1, 0.0);
  for (int i = 0; i <= N; ++i) {
    double xi = -std::cos(M_PI * i / N);
    for (int it = 0; it < 200; ++it) {
      double pn, pm;
      legendre(N, xi, &pn, &pm);
      const double dx = (xi * pn - pm) / ((N + 1) * pn);
      xi -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    x[i] = xi;
  }
  x[0] = -1.0;
  x[N] = 1.0;
  if (N % 2 == 0) x[N / 2] = 0.0;
  for (int i = 0; i <= N; ++i) {
    double pn, pm;
    legendre(N, x[i], &pn, &pm);
    w[i] = 2.0 / (N * (N + 1.0) * pn * pn);
  }
}

// Gauss-Legendre nodes/weights (Newton on P_q, P_q' from P_q, P_{q-1}).
inline void gauss(int q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    double xi = -std::cos(M_PI * (i + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 200; ++it) {
      double pn, pm;
      legendre(q, xi, &pn, &pm);
      dp = q * (xi * pn - pm) / (xi * xi - 1.0);
      const double dx = pn / dp;
      xi -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    double pn, pm;
    legendre(q, xi, &pn, &pm);
    dp = q * (xi * pn - pm) / (xi * xi - 1.0);
    x[i] = xi;
    w[i] = 2.0 / ((1.0 - xi * xi) * dp * dp);
  }
}

struct Basis1D {
  int N;
  std::vector<double> x, w, bw;   // nodes, GLL weights, barycentric weights
  std::vector<double> D;          // D[i*(N+1)+j] = l_j'(x_i)
  std::vector<double> A;          // A[a*(N+1)+b] = sum_q w_q l_a'(x_q) l_b'(x_q)
  explicit Basis1D(int n) : N(n) {
    gll(N, x, w);
    bw.assign(N + 1, 1.0);
    for (int j = 0; j <= N; ++j)
      for (int k = 0; k <= N; ++k)
        if (k != j) bw[j] /= (x[j] - x[k]);
    D.assign((N + 1) * (N + 1), 0.0);
    for (int i = 0; i <= N; ++i) {
      double diag = 0.0;
      for (int j = 0; j <= N; ++j) {
        if (j == i) continue;
        const double d = (bw[j] / bw[i]) / (x[i] - x[j]);
        D[i * (N + 1) + j] = d;
        diag -= d;
      }
      D[i * (N + 1) + i] = diag;
    }
    A.assign((N + 1) * (N + 1), 0.0);
    for (int a = 0; a <= N; ++a)
      for (int b = 0; b <= N; ++b) {
        double s = 0.0;
        for (int q = 0; q <= N; ++q) s += w[q] * D[q * (N + 1) + a] * D[q * (N + 1) + b];
        A[a * (N + 1) + b] = s;
      }
  }
  // Lagrange basis values at an arbitrary point (barycentric form)
  void values(double t, double* out) const {
    for (int j = 0; j <= N; ++j)
      if (t == x[j]) {
        for (int k = 0; k <= N; ++k) out[k] = (k == j) ? 1.0 : 0.0;
        return;
      }
    double den = 0.0;
    for (int j = 0; j <= N; ++j) den += bw[j] / (t - x[j]);
    for (int j = 0; j <= N; ++j) out[j] = (bw[j] / (t - x[j])) / den;
  }
  // assembled 1D weight of lattice line i in a box of ne elements
  double assembled_weight(int i, int ne) const {
    const int e = i / N, a = i - e * N;
    if (a != 0) return w[a];
    double s = 0.0;
    if (e > 0) s += w[N];
    if (e < ne) s += w[0];
    return s;
  }
};

}  // namespace dgtab

// Records the calling thread's last error message (read by dgsem_last_error)
// and returns code.
int dg_fail_msg(int code, const char* msg);
