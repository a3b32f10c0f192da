// Quadrature rules and basis tables of the library (host side, computed once
// per context and uploaded to the device).
//
// The discretisation is fixed by the C ABI (include/hdg.h):
//   * orthonormal Dubiner basis on the reference triangle (0,0),(1,0),(0,1),
//     modes ordered k = 0..p, j = 0..k, i = k-j;
//   * collapsed Gauss rule with (p+2) Gauss-Legendre x (p+2) Gauss-Jacobi(1,0)
//     points on elements, (p_e+2)-point Gauss-Legendre rule on edges;
//   * orthonormal Legendre trace basis on [0,1].
// Gauss nodes are found here by Newton's method on the orthogonal polynomial
// (with deflation by the roots already found), weights from the closed-form
// Christoffel numbers; the triangle basis is evaluated through the homogeneous
// ("scaled") Legendre recurrence in (t, s) = (2 xi + eta - 1, 1 - eta), which
// is polynomial everywhere on the triangle.
#include "hdg_internal.h"

#include <cmath>
#include <vector>

namespace hdg {

// P_n^{(a,b)}(x) and its derivative by differentiating the three-term recurrence.
static void jacobi_and_deriv(int n, double a, double b, double x, double* P, double* dP) {
  double p0 = 1.0, d0 = 0.0;
  if (n == 0) { *P = p0; *dP = d0; return; }
  double p1 = 0.5 * (a - b) + 0.5 * (a + b + 2.0) * x;
  double d1 = 0.5 * (a + b + 2.0);
  for (int k = 1; k < n; ++k) {
    // 2(k+1)(k+a+b+1)(2k+a+b) P_{k+1} = (2k+a+b+1)[(2k+a+b+2)(2k+a+b) x + a^2 - b^2] P_k
    //                                   - 2(k+a)(k+b)(2k+a+b+2) P_{k-1}
    double c = 2.0 * k + a + b;
    double den = 2.0 * (k + 1) * (k + a + b + 1) * c;
    double t1 = (c + 1.0) * ((c + 2.0) * c * x + a * a - b * b);
    double t2 = 2.0 * (k + a) * (k + b) * (c + 2.0);
    double p2 = (t1 * p1 - t2 * p0) / den;
    double d2 = (t1 * d1 + (c + 1.0) * (c + 2.0) * c * p1 - t2 * d0) / den;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *P = p1; *dP = d1;
}

// n-point Gauss rule for weight (1-x)^a (1+x)^b, a, b in {0,1} x {0}: Newton
// with deflation, starting from Chebyshev-Gauss points.
static void gauss_rule(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0); w.assign(n, 0.0);
  for (int k = 0; k < n; ++k) {
    double r = -std::cos((2.0 * k + 1.0) * M_PI / (2.0 * n));
    if (k > 0) r = 0.5 * (r + x[k - 1]);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      jacobi_and_deriv(n, a, b, r, &P, &dP);
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += 1.0 / (r - x[j]);
      double delta = -P / (dP - s * P);
      r += delta;
      if (std::fabs(delta) < 1e-17) break;
    }
    x[k] = r;
  }
  // Christoffel numbers: w = G 2^{a+b+1} / ((1-x^2) P_n'(x)^2) with
  // G = Gamma(n+a+1) Gamma(n+b+1) / (Gamma(n+a+b+1) n!); G = 1 for b = 0.
  double G = std::tgamma(n + a + 1.0) * std::tgamma(n + b + 1.0) /
             (std::tgamma(n + a + b + 1.0) * std::tgamma(n + 1.0));
  for (int k = 0; k < n; ++k) {
    double P, dP;
    jacobi_and_deriv(n, a, b, x[k], &P, &dP);
    w[k] = G * std::pow(2.0, a + b + 1.0) / ((1.0 - x[k] * x[k]) * dP * dP);
  }
}

// Dubiner modes and reference gradients at (xi, eta).
static void dubiner_eval(int p, double xi, double eta, double* phi, double* gxi, double* geta) {
  const double t = 2.0 * xi + eta - 1.0, s = 1.0 - eta;
  // Q_i = s^i P_i(t/s) and its derivatives (dt/dxi = 2, dt/deta = 1, ds/deta = -1)
  double Q[8], Qx[8], Qe[8];
  Q[0] = 1.0; Qx[0] = 0.0; Qe[0] = 0.0;
  Q[1] = t; Qx[1] = 2.0; Qe[1] = 1.0;
  for (int m = 1; m < p; ++m) {
    double a = 2.0 * m + 1.0, b = (double)m;
    Q[m + 1] = (a * t * Q[m] - b * s * s * Q[m - 1]) / (m + 1.0);
    Qx[m + 1] = (a * (2.0 * Q[m] + t * Qx[m]) - b * s * s * Qx[m - 1]) / (m + 1.0);
    Qe[m + 1] = (a * (Q[m] + t * Qe[m]) - b * (-2.0 * s * Q[m - 1] + s * s * Qe[m - 1])) / (m + 1.0);
  }
  const double y = 2.0 * eta - 1.0;
  int idx = 0;
  for (int k = 0; k <= p; ++k)
    for (int j = 0; j <= k; ++j) {
      int i = k - j;
      double c = std::sqrt(2.0 * (2 * i + 1) * (i + j + 1));
      double R, dR;
      jacobi_and_deriv(j, 2.0 * i + 1.0, 0.0, y, &R, &dR);
      phi[idx] = c * Q[i] * R;
      if (gxi) {
        gxi[idx] = c * Qx[i] * R;
        geta[idx] = c * (Qe[i] * R + Q[i] * 2.0 * dR);
      }
      ++idx;
    }
}

static void legendre01_eval(int pe, double s, double* psi) {
  double P, dP;
  for (int k = 0; k <= pe; ++k) {
    jacobi_and_deriv(k, 0.0, 0.0, 2.0 * s - 1.0, &P, &dP);
    psi[k] = std::sqrt(2.0 * k + 1.0) * P;
  }
}

void build_tables(Tables& T) {
  std::vector<double>& d = T.data;
  d.clear();
  auto reserve = [&](size_t n) { size_t off = d.size(); d.resize(off + n, 0.0); return (int)off; };
  for (int p = 1; p <= kMaxP; ++p) {
    const int np = n_basis(p), n1 = p + 2, nq = n1 * n1;
    std::vector<double> xa, wa, xb, wb;
    gauss_rule(n1, 0.0, 0.0, xa, wa);
    gauss_rule(n1, 1.0, 0.0, xb, wb);
    T.off.vol_w[p] = reserve(nq);
    T.off.vol_phi[p] = reserve(nq * np);
    T.off.vol_gxi[p] = reserve(nq * np);
    T.off.vol_geta[p] = reserve(nq * np);
    for (int i = 0; i < n1; ++i)
      for (int j = 0; j < n1; ++j) {
        int q = i * n1 + j;
        double xi = 0.25 * (1.0 + xa[i]) * (1.0 - xb[j]);
        double eta = 0.5 * (1.0 + xb[j]);
        d[T.off.vol_w[p] + q] = 0.125 * wa[i] * wb[j];
        dubiner_eval(p, xi, eta, &d[T.off.vol_phi[p] + q * np], &d[T.off.vol_gxi[p] + q * np],
                     &d[T.off.vol_geta[p] + q * np]);
      }
  }
  for (int pe = 1; pe <= kMaxP; ++pe) {
    const int ne = pe + 2, nk = pe + 1;
    std::vector<double> x, w;
    gauss_rule(ne, 0.0, 0.0, x, w);
    T.off.edge_s[pe] = reserve(ne);
    T.off.edge_w[pe] = reserve(ne);
    T.off.edge_psi[pe] = reserve(ne * nk);
    for (int g = 0; g < ne; ++g) {
      double s = 0.5 * (1.0 + x[g]);
      d[T.off.edge_s[pe] + g] = s;
      d[T.off.edge_w[pe] + g] = 0.5 * w[g];
      legendre01_eval(pe, s, &d[T.off.edge_psi[pe] + g * nk]);
    }
    for (int p = 1; p <= pe; ++p) {
      const int np = n_basis(p);
      for (int lf = 0; lf < 3; ++lf)
        for (int fl = 0; fl < 2; ++fl) {
          int o = reserve(ne * np);
          T.off.edge_phi[p][pe][lf][fl] = o;
          for (int g = 0; g < ne; ++g) {
            double s = d[T.off.edge_s[pe] + g];
            double t = fl ? 1.0 - s : s;
            double xi = (lf == 0) ? t : (lf == 1 ? 1.0 - t : 0.0);
            double eta = (lf == 0) ? 0.0 : (lf == 1 ? t : 1.0 - t);
            dubiner_eval(p, xi, eta, &d[o + g * np], nullptr, nullptr);
          }
        }
    }
  }
  // derived matrices (products of the tables above, summed in double)
  for (int p = 1; p <= kMaxP; ++p) {
    const int np = n_basis(p), nq = (p + 2) * (p + 2);
    int o = reserve(2 * np * np);
    T.off.vol_dref[p] = o;
    for (int r = 0; r < 2; ++r)
      for (int i = 0; i < np; ++i)
        for (int j = 0; j < np; ++j) {
          double acc = 0.0;
          const int g = r == 0 ? T.off.vol_gxi[p] : T.off.vol_geta[p];
          for (int q = 0; q < nq; ++q) acc += d[T.off.vol_w[p] + q] * d[g + q * np + i] * d[T.off.vol_phi[p] + q * np + j];
          d[o + (r * np + i) * np + j] = acc;
        }
    o = reserve(3 * np * np);
    T.off.vol_stiff[p] = o;
    for (int i = 0; i < np; ++i)
      for (int j = 0; j < np; ++j) {
        double s00 = 0.0, s01 = 0.0, s11 = 0.0;
        for (int q = 0; q < nq; ++q) {
          const double w = d[T.off.vol_w[p] + q];
          const double xi = d[T.off.vol_gxi[p] + q * np + i], ei = d[T.off.vol_geta[p] + q * np + i];
          const double xj = d[T.off.vol_gxi[p] + q * np + j], ej = d[T.off.vol_geta[p] + q * np + j];
          s00 += w * xi * xj;
          s01 += w * (xi * ej + ei * xj);
          s11 += w * ei * ej;
        }
        d[o + i * np + j] = s00;
        d[o + np * np + i * np + j] = s01;
        d[o + 2 * np * np + i * np + j] = s11;
      }
    for (int pe = p; pe <= kMaxP; ++pe) {
      const int ne = pe + 2, nk = pe + 1;
      for (int lf = 0; lf < 3; ++lf) {
        o = reserve(np * np);
        T.off.face_mass[p][pe][lf] = o;
        const int ph = T.off.edge_phi[p][pe][lf][0];
        for (int i = 0; i < np; ++i)
          for (int j = 0; j < np; ++j) {
            double acc = 0.0;
            for (int g = 0; g < ne; ++g) acc += d[T.off.edge_w[pe] + g] * d[ph + g * np + i] * d[ph + g * np + j];
            d[o + i * np + j] = acc;
          }
        for (int fl = 0; fl < 2; ++fl) {
          o = reserve(nk * np);
          T.off.edge_cross[p][pe][lf][fl] = o;
          const int phf = T.off.edge_phi[p][pe][lf][fl];
          for (int k = 0; k < nk; ++k)
            for (int j = 0; j < np; ++j) {
              double acc = 0.0;
              for (int g = 0; g < ne; ++g)
                acc += d[T.off.edge_w[pe] + g] * d[T.off.edge_psi[pe] + g * nk + k] * d[phf + g * np + j];
              d[o + k * np + j] = acc;
            }
        }
      }
    }
  }
}

// exported for the table cross-check tests (host only, no device needed)
extern "C" int hdg_debug_tables(int which, int p, int pe, int lf, int fl, double* out, int cap) {
  Tables T;
  build_tables(T);
  int off = -1, len = 0;
  const int np = (p >= 1 && p <= kMaxP) ? n_basis(p) : 0;
  const int nq = (p + 2) * (p + 2), ne = pe + 2;
  switch (which) {
    case 0: off = T.off.vol_w[p]; len = nq; break;
    case 1: off = T.off.vol_phi[p]; len = nq * np; break;
    case 2: off = T.off.vol_gxi[p]; len = nq * np; break;
    case 3: off = T.off.vol_geta[p]; len = nq * np; break;
    case 4: off = T.off.edge_s[pe]; len = ne; break;
    case 5: off = T.off.edge_w[pe]; len = ne; break;
    case 6: off = T.off.edge_psi[pe]; len = ne * (pe + 1); break;
    case 7: off = T.off.edge_phi[p][pe][lf][fl]; len = ne * np; break;
    case 8: off = T.off.vol_stiff[p]; len = 3 * np * np; break;
    default: return -1;
  }
  if (off < 0 || len > cap) return -1;
  for (int i = 0; i < len; ++i) out[i] = T.data[off + i];
  return len;
}

}  // namespace hdg
