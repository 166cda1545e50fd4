// 1D tables of the Q_k element: Gauss-Lobatto nodes (solution/geometry nodes),
// Gauss-Legendre points and weights (quadrature), and the interpolation and
// differentiation matrices between them.  Computed on the host from the
// Legendre recurrence by Newton iteration; uploaded to constant memory.
#pragma once
#include <cmath>

#define MF_KMAX 5
#define MF_NMAX (MF_KMAX + 1)

template <typename T>
struct MfTab {
  T B[MF_NMAX][MF_NMAX];    // B[q][a]  = l_a(s_q): nodal basis at Gauss points
  T Dn[MF_NMAX][MF_NMAX];   // Dn[q][a] = l_a'(s_q)
  T Hn[MF_NMAX][MF_NMAX];   // Hn[q][a] = l_a''(s_q)
  T Dg[MF_NMAX][MF_NMAX];   // Dg[q][p] = d/ds of the Gauss-point Lagrange polynomial p at s_q
  T s[MF_NMAX];             // Gauss points on [0,1]
  T w[MF_NMAX];             // Gauss weights on [0,1] (sum 1)
  T gll[MF_NMAX];           // Gauss-Lobatto nodes on [0,1]
  T bw[MF_NMAX];            // 1 / prod_{b != a} (gll_a - gll_b)
  T dLe[2][MF_NMAX];        // dLe[e][a] = l_a'(e): nodal-basis derivatives at the ends xi = 0, 1
};

namespace mfhost {

// Legendre P_n and P_n' at x in [-1,1] by the three-term recurrence.
inline void legendre(int n, double x, double& p, double& dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { p = 1.0; dp = 0.0; return; }
  for (int j = 2; j <= n; ++j) {
    double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
    p0 = p1; p1 = p2;
  }
  p = p1;
  dp = (std::fabs(x) < 1.0) ? n * (x * p1 - p0) / (x * x - 1.0) : 0.5 * n * (n + 1) * (x > 0 ? 1.0 : (n % 2 ? 1.0 : -1.0));
}

// q Gauss-Legendre points/weights on [0,1]: roots of P_q.
inline void gauss01(int q, double* s, double* w) {
  for (int i = 0; i < q; ++i) {
    double x = std::cos(M_PI * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp; legendre(q, x, p, dp);
      double dx = p / dp; x -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    double p, dp; legendre(q, x, p, dp);
    s[q - 1 - i] = 0.5 * (x + 1.0);
    w[q - 1 - i] = 1.0 / ((1.0 - x * x) * dp * dp);   // 2/((1-x^2)P'^2) scaled by 1/2
  }
}

// k+1 Gauss-Lobatto points on [0,1]: the ends and the roots of P_k'.
inline void gll01(int k, double* x01) {
  int n = k + 1;
  double x[MF_NMAX];
  x[0] = -1.0; x[k] = 1.0;
  for (int i = 1; i < k; ++i) {
    double y = -std::cos(M_PI * i / k);
    for (int it = 0; it < 100; ++it) {
      // f = P_k'(y); f' = P_k''(y) = (2y P_k' - k(k+1) P_k)/(1-y^2)
      double p, dp; legendre(k, y, p, dp);
      double d2 = (2.0 * y * dp - k * (k + 1.0) * p) / (1.0 - y * y);
      double dy = dp / d2; y -= dy;
      if (std::fabs(dy) < 1e-17) break;
    }
    x[i] = y;
  }
  for (int i = 0; i < n; ++i) x01[i] = 0.5 * (x[i] - x[k - i]) * 0.5 + 0.5;  // symmetrised
}

// Lagrange polynomial a on nodes z[0..n) and its first two derivatives at t.
inline void lagrange(const double* z, int n, int a, double t, double& v, double& d1, double& d2) {
  double den = 1.0;
  for (int b = 0; b < n; ++b) if (b != a) den *= (z[a] - z[b]);
  v = 1.0; d1 = 0.0; d2 = 0.0;
  for (int b = 0; b < n; ++b) if (b != a) v *= (t - z[b]);
  for (int c = 0; c < n; ++c) {
    if (c == a) continue;
    double pc = 1.0;
    for (int b = 0; b < n; ++b) if (b != a && b != c) pc *= (t - z[b]);
    d1 += pc;
    for (int e = 0; e < n; ++e) {
      if (e == a || e == c) continue;
      double pe = 1.0;
      for (int b = 0; b < n; ++b) if (b != a && b != c && b != e) pe *= (t - z[b]);
      d2 += pe;
    }
  }
  v /= den; d1 /= den; d2 /= den;
}

inline void build_tab(int k, MfTab<double>& T) {
  int n = k + 1;
  double s[MF_NMAX], w[MF_NMAX], g[MF_NMAX];
  gauss01(n, s, w);
  gll01(k, g);
  for (int i = 0; i < MF_NMAX; ++i) {
    T.s[i] = i < n ? s[i] : 0; T.w[i] = i < n ? w[i] : 0; T.gll[i] = i < n ? g[i] : 0;
    for (int j = 0; j < MF_NMAX; ++j) T.B[i][j] = T.Dn[i][j] = T.Hn[i][j] = T.Dg[i][j] = 0;
    T.dLe[0][i] = T.dLe[1][i] = 0;
  }
  for (int e = 0; e < 2; ++e)
    for (int a = 0; a < n; ++a) {
      double v, d1, d2;
      lagrange(g, n, a, (double)e, v, d1, d2);
      T.dLe[e][a] = d1;
    }
  for (int a = 0; a < n; ++a) {
    double den = 1.0;
    for (int b = 0; b < n; ++b) if (b != a) den *= (g[a] - g[b]);
    T.bw[a] = 1.0 / den;
  }
  for (int q = 0; q < n; ++q)
    for (int a = 0; a < n; ++a) {
      double v, d1, d2;
      lagrange(g, n, a, s[q], v, d1, d2);
      T.B[q][a] = v; T.Dn[q][a] = d1; T.Hn[q][a] = d2;
      lagrange(s, n, a, s[q], v, d1, d2);
      T.Dg[q][a] = d1;
    }
}

template <typename T> inline T cast_to(double x) { return (T)x; }

template <typename T>
inline void cast_tab(const MfTab<double>& A, MfTab<T>& B) {
  for (int i = 0; i < MF_NMAX; ++i) {
    B.s[i] = T(A.s[i]); B.w[i] = T(A.w[i]); B.gll[i] = T(A.gll[i]); B.bw[i] = T(A.bw[i]);
    B.dLe[0][i] = T(A.dLe[0][i]); B.dLe[1][i] = T(A.dLe[1][i]);
    for (int j = 0; j < MF_NMAX; ++j) {
      B.B[i][j] = T(A.B[i][j]); B.Dn[i][j] = T(A.Dn[i][j]); B.Hn[i][j] = T(A.Hn[i][j]); B.Dg[i][j] = T(A.Dg[i][j]);
    }
  }
}

}  // namespace mfhost
