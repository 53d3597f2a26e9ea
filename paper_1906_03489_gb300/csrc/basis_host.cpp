// Host FP64 construction of the basis tables (§2.1 modified basis; GLL
// quadrature of §3.5, Listing lst:python).
//
// GLL points: the end points -1, 1 and the Q-2 zeros of the Jacobi
// polynomial P^{(1,1)}_{Q-2}, obtained as the eigenvalues of its symmetric
// tridiagonal Jacobi matrix (Golub-Welsch) and polished by Newton steps on the
// three-term recurrence.  Weights w_i = 2 / (N (N+1) L_N(x_i)^2), N = Q-1.
// The collocation derivative uses barycentric weights.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "spx_internal.h"

namespace spx {
namespace {

// P^{(1,1)}_m(x) and its derivative by the recurrence and its x-derivative.
void jacobi11(int m, double x, double* val, double* der) {
  double p0 = 1.0, d0 = 0.0;
  if (m == 0) {
    *val = p0;
    *der = d0;
    return;
  }
  double p1 = 2.0 * x, d1 = 2.0;  // (a+b+2) x / 2 with a = b = 1
  for (int k = 2; k <= m; ++k) {
    // 2k(k+2)(2k) P_k = (2k+1)(2k+2)(2k) x P_{k-1} - 2k(k)(2k+2) P_{k-2}, a = b = 1
    const double c = 2.0 * k + 2.0;               // 2k + a + b
    const double a1 = 2.0 * k * (k + 2.0) * (c - 2.0);
    const double a2 = (c - 1.0) * c * (c - 2.0);  // coefficient of x P_{k-1}
    const double a3 = 2.0 * k * k * c;            // 2 (k+a-1)(k+b-1) c
    const double p2 = (a2 * x * p1 - a3 * p0) / a1;
    const double d2 = (a2 * (p1 + x * d1) - a3 * d0) / a1;
    p0 = p1; d0 = d1; p1 = p2; d1 = d2;
  }
  *val = p1;
  *der = d1;
}

double legendre_val(int N, double x) {
  double a = 1.0, b = x;
  if (N == 0) return a;
  for (int k = 1; k < N; ++k) {
    const double c = ((2.0 * k + 1.0) * x * b - k * a) / (k + 1.0);
    a = b;
    b = c;
  }
  return b;
}

// Eigenvalues of a symmetric tridiagonal matrix (diag d, off-diag e) by
// implicit QL iterations with Wilkinson shifts; d is overwritten.
void tridiag_eigenvalues(std::vector<double>& d, std::vector<double> e) {
  const int n = static_cast<int>(d.size());
  e.push_back(0.0);
  for (int l = 0; l < n; ++l) {
    for (int iter = 0; iter < 100; ++iter) {
      int m = l;
      for (; m < n - 1; ++m) {
        const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
        if (std::fabs(e[m]) <= 1e-17 * dd) break;
      }
      if (m == l) break;
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0 ? std::fabs(r) : -std::fabs(r)));
      double s = 1.0, c = 1.0, p = 0.0;
      int i = m - 1;
      for (; i >= l; --i) {
        double f = s * e[i], b = c * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= p;
          e[m] = 0.0;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
      }
      if (r == 0.0 && i >= l) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
}

void gll_points(int Q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(Q, 0.0);
  w.assign(Q, 0.0);
  const int N = Q - 1;
  x[0] = -1.0;
  x[N] = 1.0;
  const int m = Q - 2;  // interior points: zeros of P^{(1,1)}_m
  if (m > 0) {
    // Jacobi matrix of the weight (1-x)(1+x): zero diagonal, off-diagonal
    // b_k = sqrt(k (k+2) / ((2k+1)(2k+3))), k = 1..m-1
    std::vector<double> d(m, 0.0), e(m > 1 ? m - 1 : 0);
    for (int k = 1; k < m; ++k) e[k - 1] = std::sqrt(k * (k + 2.0) / ((2.0 * k + 1.0) * (2.0 * k + 3.0)));
    tridiag_eigenvalues(d, e);
    std::sort(d.begin(), d.end());
    for (int i = 0; i < m; ++i) {
      double z = d[i];
      for (int it = 0; it < 8; ++it) {  // Newton polish
        double v, dv;
        jacobi11(m, z, &v, &dv);
        z -= v / dv;
      }
      x[i + 1] = z;
    }
    for (int i = 1; i <= m / 2; ++i) {  // exact symmetry
      const double a = 0.5 * (x[N - i] - x[i]);
      x[i] = -a;
      x[N - i] = a;
    }
    if (m % 2 == 1) x[Q / 2] = 0.0;
  }
  for (int i = 0; i < Q; ++i) {
    const double L = legendre_val(N, x[i]);
    w[i] = 2.0 / (N * (N + 1.0) * L * L);
  }
}

// P^{(a,b)}_m(x) by the three-term recurrence (standard normalisation).
double jacobi_ab(int m, double a, double b, double x) {
  if (m < 0) return 0.0;
  double p0 = 1.0;
  if (m == 0) return p0;
  double p1 = 0.5 * ((a + b + 2.0) * x + a - b);
  for (int k = 2; k <= m; ++k) {
    const double c = 2.0 * k + a + b;
    const double lhs = 2.0 * k * (k + a + b) * (c - 2.0);
    const double t1 = (c - 1.0) * (c * (c - 2.0) * x + a * a - b * b);
    const double t2 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * c;
    const double p2 = (t1 * p1 - t2 * p0) / lhs;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// Collocation derivative of the Lagrange interpolant through points x (barycentric weights).
void collocation(const std::vector<double>& x, double* D) {
  const int Q = static_cast<int>(x.size());
  std::vector<double> lam(Q, 1.0);
  for (int j = 0; j < Q; ++j)
    for (int k = 0; k < Q; ++k)
      if (k != j) lam[j] /= (x[j] - x[k]);
  for (int i = 0; i < Q; ++i) {
    double diag = 0.0;
    for (int j = 0; j < Q; ++j) {
      if (j == i) continue;
      const double v = (lam[j] / lam[i]) / (x[i] - x[j]);
      D[i * Q + j] = v;
      diag -= v;
    }
    D[i * Q + i] = diag;
  }
}

}  // namespace

// Gauss-Radau-Legendre points including -1 (ascending, all < 1) and weights:
// the zeros of P_{Q-1} + P_Q by Newton's method from the Chebyshev-Radau
// points -cos(2 pi i / (2Q - 1)), weights 2 / Q^2 at -1 and
// (1 - x_i) / (Q^2 P_{Q-1}(x_i)^2) elsewhere (exact for degree 2Q - 2).
spx_status gauss_radau(int Q, double* x, double* w) {
  if (Q < 2 || Q > 16) return fail(SPX_ERR_INVALID_ARG, "Gauss-Radau points need 2 <= Q <= 16");
  const double pi = 3.14159265358979323846;
  x[0] = -1.0;
  for (int i = 1; i < Q; ++i) {
    double z = -std::cos(2.0 * pi * i / (2.0 * Q - 1.0));
    for (int it = 0; it < 100; ++it) {
      // f = P_{Q-1} + P_Q, f' = P'_{Q-1} + P'_Q by the Legendre recurrence
      double a = 1.0, b = z, da = 0.0, db = 1.0;
      for (int k = 1; k < Q; ++k) {
        const double c = ((2.0 * k + 1.0) * z * b - k * a) / (k + 1.0);
        const double dc = ((2.0 * k + 1.0) * (b + z * db) - k * da) / (k + 1.0);
        a = b;
        b = c;
        da = db;
        db = dc;
      }
      const double dz = (a + b) / (da + db);
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
  std::sort(x, x + Q);
  for (int i = 0; i < Q; ++i) {
    const double L = legendre_val(Q - 1, x[i]);
    w[i] = i == 0 ? 2.0 / (Q * Q) : (1.0 - x[i]) / (Q * Q * L * L);
  }
  return SPX_OK;
}

// Tables of the collapsed-coordinate kernels (order P, Q points per direction):
//   B1[Q][n]     modified basis psi^a at the Q GLL points;
//   Bb[n][Q][n]  psi^b_{pq} at the Q Gauss-Radau points, [p][k][q] for the q of
//                mode range of p (p = 0: psi^a_q, q <= P; p = P: psi^a_q, q < P;
//                0 < p < P: ((1-z)/2)^(p+1) for q = 0 and
//                ((1-z)/2)^(p+1) (1+z)/2 P^{(2p+1,1)}_{q-1}(z) for 0 < q < P - p),
//                zero elsewhere;
//   D1[Q][Q], D2[Q][Q]  collocation derivatives on the GLL / Gauss-Radau points;
//   xg, wg, xr, wr      the two point sets and their weights;
//   Bc[n][Q][n]  tetrahedra: ((1-z)/2)^k (r = 0) and ((1-z)/2)^k (1+z)/2
//                P^{(2k-1,1)}_{r-1}(z) (0 < r <= P - k) at the Gauss-Radau
//                points, [k][k3][r] for k = 1..P; [0][k3][0] = (1+z)/2 (apex).
spx_status collapsed_tables(int P, int Q, double* B1, double* Bb, double* D1, double* D2, double* xg, double* wg,
                            double* xr, double* wr, double* Bc) {
  if (P < 1 || P > 8 || Q < P + 1 || Q > 16) return fail(SPX_ERR_INVALID_ARG, "collapsed tables: bad P or Q");
  std::vector<double> g, gw, r(Q), rw(Q);
  gll_points(Q, g, gw);
  spx_status st = gauss_radau(Q, r.data(), rw.data());
  if (st != SPX_OK) return st;
  const int n = P + 1;
  std::vector<double> A(Q * n), Ar(Q * n);
  basis_tables(P, Q, nullptr, nullptr, A.data(), nullptr, nullptr);
  for (int k = 0; k < Q; ++k) {   // psi^a at the Radau points
    const double z = r[k];
    for (int q = 0; q < n; ++q) {
      double v;
      if (q == 0) v = 0.5 * (1.0 - z);
      else if (q == P) v = 0.5 * (1.0 + z);
      else v = 0.25 * (1.0 - z) * (1.0 + z) * jacobi_ab(q - 1, 1.0, 1.0, z);
      Ar[k * n + q] = v;
    }
  }
  if (B1) std::copy(A.begin(), A.end(), B1);
  if (Bb) {
    std::fill(Bb, Bb + n * Q * n, 0.0);
    for (int p = 0; p <= P; ++p)
      for (int k = 0; k < Q; ++k) {
        const double z = r[k], L = 0.5 * (1.0 - z), R = 0.5 * (1.0 + z);
        if (p == 0 || p == P) {
          const int nq = p == 0 ? n : P;
          for (int q = 0; q < nq; ++q) Bb[(p * Q + k) * n + q] = Ar[k * n + q];
        } else {
          const double Lp = std::pow(L, p + 1);
          for (int q = 0; q < P - p; ++q)
            Bb[(p * Q + k) * n + q] = q == 0 ? Lp : Lp * R * jacobi_ab(q - 1, 2.0 * p + 1.0, 1.0, z);
        }
      }
  }
  if (Bc) {   // tetrahedra: [k][k3][r], k = 1..P, r <= P - k; [0][k3][0] = (1 + z)/2 (apex)
    std::fill(Bc, Bc + n * Q * n, 0.0);
    for (int k3 = 0; k3 < Q; ++k3) {
      const double z = r[k3], L = 0.5 * (1.0 - z), R = 0.5 * (1.0 + z);
      Bc[k3 * n] = R;
      for (int k = 1; k <= P; ++k) {
        const double Lk = std::pow(L, k);
        for (int rr = 0; rr <= P - k; ++rr)
          Bc[(k * Q + k3) * n + rr] = rr == 0 ? Lk : Lk * R * jacobi_ab(rr - 1, 2.0 * k - 1.0, 1.0, z);
      }
    }
  }
  if (D1) collocation(g, D1);
  if (D2) collocation(r, D2);
  if (xg) std::copy(g.begin(), g.end(), xg);
  if (wg) std::copy(gw.begin(), gw.end(), wg);
  if (xr) std::copy(r.begin(), r.end(), xr);
  if (wr) std::copy(rw.begin(), rw.end(), wr);
  return SPX_OK;
}

spx_status basis_tables(int P, int Q, double* xi, double* w, double* B, double* dB, double* D) {
  if (P < 1 || Q < 2 || Q > 16) return fail(SPX_ERR_INVALID_ARG, "basis tables need 1 <= P and 2 <= Q <= 16");
  std::vector<double> x, ww;
  gll_points(Q, x, ww);
  if (xi) std::memcpy(xi, x.data(), Q * sizeof(double));
  if (w) std::memcpy(w, ww.data(), Q * sizeof(double));
  const int n = P + 1;
  for (int i = 0; i < Q; ++i) {
    const double z = x[i];
    for (int p = 0; p < n; ++p) {
      double v, dv;
      if (p == 0) {
        v = 0.5 * (1.0 - z);
        dv = -0.5;
      } else if (p == P) {
        v = 0.5 * (1.0 + z);
        dv = 0.5;
      } else {
        double j, dj;
        jacobi11(p - 1, z, &j, &dj);
        const double bub = 0.25 * (1.0 - z) * (1.0 + z);
        v = bub * j;
        dv = -0.5 * z * j + bub * dj;
      }
      if (B) B[i * n + p] = v;
      if (dB) dB[i * n + p] = dv;
    }
  }
  if (D) {
    std::vector<double> lam(Q, 1.0);  // barycentric weights
    for (int j = 0; j < Q; ++j)
      for (int k = 0; k < Q; ++k)
        if (k != j) lam[j] /= (x[j] - x[k]);
    for (int i = 0; i < Q; ++i) {
      double diag = 0.0;
      for (int j = 0; j < Q; ++j) {
        if (j == i) continue;
        const double v = (lam[j] / lam[i]) / (x[i] - x[j]);
        D[i * Q + j] = v;
        diag -= v;
      }
      D[i * Q + i] = diag;
    }
  }
  return SPX_OK;
}

// Nodal (Lagrange) basis of order P through the P + 1 GLL points z_m,
// evaluated at the Q GLL points x_i (§2.1: the classical spectral element
// basis): B[i][m] = l_m(x_i) = prod_{k != m} (x_i - z_k) / (z_m - z_k) and
// its derivative, the sum over l != m of the same product without factor l
// divided by (z_m - z_l).  With Q = P + 1 the points coincide: B = I, dB = D.
spx_status nodal_basis_tables(int P, int Q, double* B, double* dB) {
  if (P < 1 || Q < 2 || Q > 16) return fail(SPX_ERR_INVALID_ARG, "nodal basis tables need 1 <= P and 2 <= Q <= 16");
  std::vector<double> z, wz, x, wx;
  gll_points(P + 1, z, wz);
  gll_points(Q, x, wx);
  const int n = P + 1;
  for (int i = 0; i < Q; ++i)
    for (int m = 0; m < n; ++m) {
      double v = 1.0, dv = 0.0;
      for (int k = 0; k < n; ++k) {
        if (k == m) continue;
        v *= (x[i] - z[k]) / (z[m] - z[k]);
      }
      for (int l = 0; l < n; ++l) {
        if (l == m) continue;
        double t = 1.0 / (z[m] - z[l]);
        for (int k = 0; k < n; ++k)
          if (k != m && k != l) t *= (x[i] - z[k]) / (z[m] - z[k]);
        dv += t;
      }
      if (B) B[i * n + m] = v;
      if (dB) dB[i * n + m] = dv;
    }
  return SPX_OK;
}

// Even-odd coefficients of order P (layout: EOLayout in kernel_params.h),
// appended after B, dB, D of `tab`.
void eo_tables(int P, int Q, double* tab) {
  const int n = P + 1, H = Q / 2, Hc = (Q + 1) / 2;
  const double* B = tab;
  const double* D = tab + 2 * Q * n;
  double* Bs = tab + 2 * Q * n + Q * Q;
  double* Bd = Bs + Hc;
  double* Dp = Bd + Hc;
  double* Dm = Dp + H * H;
  double* Tp = Dm + H * H;
  double* Tm = Tp + H * H;
  double* Gs = Tm + H * H;
  double* Gd = Gs + Hc;
  const double* dB = tab + Q * n;
  for (int i = 0; i < Hc; ++i) {
    Bs[i] = 0.5 * (B[i * n] + B[i * n + P]);
    Bd[i] = 0.5 * (B[i * n] - B[i * n + P]);
    Gs[i] = 0.5 * (dB[i * n] + dB[i * n + P]);
    Gd[i] = 0.5 * (dB[i * n] - dB[i * n + P]);
  }
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < H; ++j) {
      Dp[i * H + j] = 0.5 * (D[i * Q + j] + D[i * Q + Q - 1 - j]);
      Dm[i * H + j] = 0.5 * (D[i * Q + j] - D[i * Q + Q - 1 - j]);
      Tp[i * H + j] = 0.5 * (D[j * Q + i] + D[(Q - 1 - j) * Q + i]);
      Tm[i * H + j] = 0.5 * (D[j * Q + i] - D[(Q - 1 - j) * Q + i]);
    }
}

// Inverse of the 1D mass matrix M1 = B^T diag(w) B (n x n, SPD) of the basis
// tables B [Q][n] of order P on Q GLL points (weights w), by Cholesky
// factorisation and two triangular solves per column.  Row-major [n][n] into
// minv.
void mass1d_inverse(int P, int Q, const double* B, double* minv, bool restricted) {
  const int nf = P + 1;
  std::vector<double> w(Q);
  basis_tables(P, Q, nullptr, w.data(), nullptr, nullptr, nullptr);
  std::fill(minv, minv + nf * nf, 0.0);
  // kept modes: all, or all but the degree-P bubble (index P - 1)
  std::vector<int> keep;
  for (int a = 0; a < nf; ++a)
    if (!restricted || a != P - 1) keep.push_back(a);
  const int n = static_cast<int>(keep.size());
  std::vector<double> M(n * n, 0.0), L(n * n, 0.0), Mi(n * n, 0.0);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      double s = 0.0;
      for (int i = 0; i < Q; ++i) s += B[i * nf + keep[a]] * w[i] * B[i * nf + keep[b]];
      M[a * n + b] = s;
    }
  for (int j = 0; j < n; ++j) {
    double d = M[j * n + j];
    for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
    L[j * n + j] = std::sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      double s = M[i * n + j];
      for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = s / L[j * n + j];
    }
  }
  std::vector<double> y(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) {  // L y = e_c
      double s = i == c ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
      y[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {  // L^T x = y
      double s = y[i];
      for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * Mi[k * n + c];
      Mi[i * n + c] = s / L[i * n + i];
    }
  }
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) minv[keep[a] * nf + keep[b]] = Mi[a * n + b];
}

}  // namespace spx
