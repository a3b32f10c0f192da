// HDG oracle: plain, slow, obviously-correct FP64 CPU implementation of one
// hybridized-DG Newton step for steady 2D Euler / mixed-form Navier-Stokes
// (Woopen, Balan, May, Schuetz, arXiv:1308.3995).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, import or
// call this file; only the tests, the smoke check and the CPU-baseline leg of
// the benchmark do.  It shares no code, header, table or constant generator
// with the CUDA library.
//
// What it computes (section / equation of the paper):
//   * physics: Euler convective flux and ideal-gas pressure (Sec. 2.1), viscous
//     flux, temperature, Newtonian stress and Sutherland viscosity (Sec. 2.2);
//   * the HDG residual N_h of Eq. (hdg_ls1)-(hdg_cont) with the combined
//     Lax-Friedrichs/LDG-type numerical flux of Sec. 3.2 (source s: zero, or a
//     state-independent s_h given by its projection coefficients), the
//     boundary operator of Sec. 3.2 on tagged boundary faces (Euler: slip wall
//     and characteristic far field; Navier-Stokes: no-slip adiabatic wall and
//     characteristic far field with the viscous flux at the far-field state;
//     boundary states and wall viscous flux of Sec. 2.1/2.2), optionally with the
//     shock-capturing volume term of Sec. 3.2 (artificial viscosity eps_K from
//     the L1 norm of the strong convective residual, effective size h_K / p_K);
//   * the Newton matrix N'_h (Eq. linearsystem) as the exact complex-step
//     derivative of that residual, column by column (eps_K frozen at the
//     current state: it is evaluated from the real part only), plus the optional
//     backward-Euler pseudo-time mass term with the local time step of Sec. 3.3;
//   * static condensation of Sec. 3.4: K = N - [L M][A B;C D]^{-1}[R;S],
//     E = H - [L M][A B;C D]^{-1}[F;G], assembled element by element, the
//     local solves stored for reconstruction, and the reconstruction of
//     (dQ, dW) from dLambda by Eq. (ls);
//   * for tiny meshes, the monolithic linearised system solved densely.
//
// Readings of points the paper leaves open are fixed
// here: orthonormal Dubiner basis in the order (k=0..p, j=0..k, i=k-j);
// collapsed Gauss volume rule with (p+2)x(p+2) points; (p_e+2)-point
// Gauss-Legendre edge rule; orthonormal Legendre trace basis with the edge
// parameter running from the lower to the higher global vertex id; the jump
// in Eq. (hdg_cont) is the sum of both sides' outward fluxes; momentum flux
// rho v (x) v + p Id; Sutherland's law non-dimensionalised with
// rho_inf = c_inf = 1 and T = gamma p / rho.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <limits>
#include <mutex>
#include <thread>
#include <vector>

// Scalar type of the arithmetic.  The default build computes in binary64.  The
// same source compiled with -DORC_EXTENDED computes in long double (80-bit
// extended on x86-64, binary128 on aarch64): a higher-precision evaluation of
// the same definition, used to measure the rounding error of binary64 results.
#ifdef ORC_EXTENDED
typedef long double real;
#define RLIT(x) x##L
#else
typedef double real;
#define RLIT(x) x
#endif
typedef std::complex<real> cplx;

extern "C" {
typedef struct {
  int32_t model;     // 0 = Euler (4 fields), 1 = Navier-Stokes mixed form (12 fields)
  int32_t reserved;
  double gamma;      // ratio of specific heats (Sec. 2.1)
  double prandtl;    // Pr (Sec. 2.2)
  double reynolds;   // Re based on free-stream speed, rho_inf = 1, L = 1
  double mach;       // free-stream Mach number (c_inf = 1) -> mu_inf = mach / reynolds
  double alpha;      // constant scalar stabilisation alpha = alpha_c + alpha_v (Sec. 3.2)
  double cfl;        // <= 0: pure Newton (dt = inf); else backward-Euler pseudo time (Sec. 3.3)
  double t_inf;      // dimensional free-stream temperature [K] for Sutherland's C2
  double sc_eps0;    // shock capturing factor eps_0 (Sec. 3.2); <= 0: no shock capturing
  double sc_beta;    // exponent beta of the effective mesh size h_K / p_K
  double aoa;        // free-stream angle of attack [degrees] (the far-field state of Sec. 2.1)
} orc_params;
}

// ---------------------------------------------------------------------------
// Gauss quadrature by the Golub-Welsch method: the nodes are the eigenvalues
// of the symmetric tridiagonal Jacobi matrix of the orthogonal polynomials,
// the weights mu0 * (first eigenvector component)^2.
// ---------------------------------------------------------------------------
// squared off-diagonal norm at which the Jacobi iteration stops
#ifdef ORC_EXTENDED
static const real kJacobiOffTol = 1e-70L;
#else
static const real kJacobiOffTol = 1e-34;
#endif
static void sym_eig_jacobi(int n, std::vector<real>& a, std::vector<real>& v) {
  // cyclic Jacobi rotations on a symmetric n x n row-major matrix a;
  // on exit the diagonal holds eigenvalues and the columns of v eigenvectors.
  v.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) v[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    real off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += a[i * n + j] * a[i * n + j];
    if (off < kJacobiOffTol) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        real apq = a[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        real theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
        real t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        real c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          real akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          real apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          real vkp = v[k * n + p], vkq = v[k * n + q];
          v[k * n + p] = c * vkp - s * vkq;
          v[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
}

// n-point Gauss-Jacobi rule for weight (1-x)^al (1+x)^be on [-1,1], ascending nodes.
static void gauss_jacobi(int n, real al, real be, real* x, real* w) {
  std::vector<real> J(n * n, 0.0), V;
  for (int k = 0; k < n; ++k) {
    real s = 2.0 * k + al + be;
    J[k * n + k] = (k == 0) ? (be - al) / (al + be + 2.0) : (be * be - al * al) / (s * (s + 2.0));
    if (k >= 1) {
      real kk = k;
      real num = 4.0 * kk * (kk + al) * (kk + be) * (kk + al + be);
      real den = s * s * (s + 1.0) * (s - 1.0);
      J[k * n + k - 1] = J[(k - 1) * n + k] = std::sqrt(num / den);
    }
  }
  sym_eig_jacobi(n, J, V);
  real mu0 = std::pow(2.0, al + be + 1.0) * std::tgamma(al + 1.0) * std::tgamma(be + 1.0) /
               std::tgamma(al + be + 2.0);
  std::vector<std::pair<real, real>> xw(n);
  for (int k = 0; k < n; ++k) xw[k] = {J[k * n + k], mu0 * V[0 * n + k] * V[0 * n + k]};
  std::sort(xw.begin(), xw.end());
  for (int k = 0; k < n; ++k) { x[k] = xw[k].first; w[k] = xw[k].second; }
}

// ---------------------------------------------------------------------------
// Jacobi polynomials P_n^{(a,b)}(x) by the three-term recurrence, and their
// derivative d/dx P_n^{(a,b)} = (n+a+b+1)/2 P_{n-1}^{(a+1,b+1)}.
// ---------------------------------------------------------------------------
static real jacobi_p(int n, real a, real b, real x) {
  if (n == 0) return 1.0;
  real p0 = 1.0, p1 = (a + 1.0) + (a + b + 2.0) * (x - 1.0) / 2.0;
  for (int m = 2; m <= n; ++m) {
    real c = 2.0 * m + a + b;
    real a1 = 2.0 * m * (m + a + b) * (c - 2.0);
    real a2 = (c - 1.0) * (c * (c - 2.0) * x + a * a - b * b);
    real a3 = 2.0 * (m + a - 1.0) * (m + b - 1.0) * c;
    real p2 = (a2 * p1 - a3 * p0) / a1;
    p0 = p1; p1 = p2;
  }
  return p1;
}
static real jacobi_dp(int n, real a, real b, real x) {
  if (n == 0) return 0.0;
  return 0.5 * (n + a + b + 1.0) * jacobi_p(n - 1, a + 1.0, b + 1.0, x);
}

static inline int n_basis(int p) { return (p + 1) * (p + 2) / 2; }

// Orthonormal Dubiner basis on the reference triangle (0,0),(1,0),(0,1):
//   phi_ij = c_ij P_i(a) ((1-b)/2)^i P_j^{(2i+1,0)}(b),
//   a = 2 xi/(1-eta) - 1, b = 2 eta - 1, c_ij = sqrt(2 (2i+1)(i+j+1)),
// ordered k = 0..p, j = 0..k, i = k-j.  Gradients by the chain rule through
// the collapsed coordinates (valid for eta < 1, i.e. away from vertex (0,1)).
static void dubiner(int p, real xi, real eta, real* phi, real* dxi, real* deta) {
  real om = 1.0 - eta;           // (1-b)/2
  real a = 2.0 * xi / om - 1.0;  // collapsed coordinate
  real b = 2.0 * eta - 1.0;
  int m = 0;
  for (int k = 0; k <= p; ++k)
    for (int j = 0; j <= k; ++j) {
      int i = k - j;
      real c = std::sqrt(2.0 * (2 * i + 1) * (i + j + 1));
      real Pa = jacobi_p(i, 0, 0, a), dPa = jacobi_dp(i, 0, 0, a);
      real Pb = jacobi_p(j, 2 * i + 1, 0, b), dPb = jacobi_dp(j, 2 * i + 1, 0, b);
      real omi = std::pow(om, i);
      phi[m] = c * Pa * omi * Pb;
      if (dxi) {
        // d/dxi: da/dxi = 2/(1-eta)
        real omi1 = (i >= 1) ? std::pow(om, i - 1) : 0.0;
        dxi[m] = c * dPa * 2.0 * omi1 * Pb;
        // d/deta: da/deta = (1+a)/(1-eta); d(om^i)/deta = -i om^(i-1); db/deta = 2
        real t1 = (i >= 1) ? dPa * (1.0 + a) * omi1 * Pb : 0.0;
        real t2 = (i >= 1) ? -Pa * i * omi1 * Pb : 0.0;
        real t3 = Pa * omi * dPb * 2.0;
        deta[m] = c * (t1 + t2 + t3);
      }
      ++m;
    }
}

// Orthonormal Legendre trace basis on [0,1]: psi_k(s) = sqrt(2k+1) P_k(2s-1).
static void legendre01(int pe, real s, real* psi) {
  for (int k = 0; k <= pe; ++k) psi[k] = std::sqrt(2.0 * k + 1.0) * jacobi_p(k, 0, 0, 2.0 * s - 1.0);
}

// Reference point on local face lf at local parameter t (face lf runs from
// local vertex lf to lf+1 mod 3).
static void face_point(int lf, real t, real* xi, real* eta) {
  if (lf == 0) { *xi = t; *eta = 0.0; }
  else if (lf == 1) { *xi = 1.0 - t; *eta = t; }
  else { *xi = 0.0; *eta = 1.0 - t; }
}

// ---------------------------------------------------------------------------
// Cached tables per degree (filled once, read-only afterwards).
// ---------------------------------------------------------------------------
struct VolTab {
  int p = 0, np = 0, nq = 0;
  std::vector<real> w, phi, dxi, deta;  // [nq], [nq][np]
};
struct EdgeTab {  // element degree p, edge degree pe
  int np = 0, nk = 0, ne = 0;
  std::vector<real> s, w, psi;          // [ne], [ne], [ne][nk]
  std::vector<real> phi[3][2];          // [lf][flip] -> [ne][np]
};
static VolTab g_vol[6];
static EdgeTab g_edge[6][6];
static std::once_flag g_once;

static void tri_rule(int p, std::vector<real>& xi, std::vector<real>& eta, std::vector<real>& w) {
  int n = p + 2;
  std::vector<real> xa(n), wa(n), xb(n), wb(n);
  gauss_jacobi(n, 0.0, 0.0, xa.data(), wa.data());
  gauss_jacobi(n, 1.0, 0.0, xb.data(), wb.data());
  xi.clear(); eta.clear(); w.clear();
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      xi.push_back((1.0 + xa[i]) * (1.0 - xb[j]) / 4.0);
      eta.push_back((1.0 + xb[j]) / 2.0);
      w.push_back(wa[i] * wb[j] / 8.0);
    }
}
static void edge_rule(int pe, std::vector<real>& s, std::vector<real>& w) {
  int n = pe + 2;
  std::vector<real> x(n), wx(n);
  gauss_jacobi(n, 0.0, 0.0, x.data(), wx.data());
  s.resize(n); w.resize(n);
  for (int i = 0; i < n; ++i) { s[i] = (1.0 + x[i]) / 2.0; w[i] = wx[i] / 2.0; }
}

static void init_tables() {
  for (int p = 1; p <= 5; ++p) {
    VolTab& V = g_vol[p];
    std::vector<real> xi, eta;
    tri_rule(p, xi, eta, V.w);
    V.p = p; V.np = n_basis(p); V.nq = (int)V.w.size();
    V.phi.resize(V.nq * V.np); V.dxi.resize(V.nq * V.np); V.deta.resize(V.nq * V.np);
    for (int q = 0; q < V.nq; ++q)
      dubiner(p, xi[q], eta[q], &V.phi[q * V.np], &V.dxi[q * V.np], &V.deta[q * V.np]);
  }
  for (int p = 1; p <= 5; ++p)
    for (int pe = p; pe <= 5; ++pe) {
      EdgeTab& E = g_edge[p][pe];
      E.np = n_basis(p); E.nk = pe + 1;
      edge_rule(pe, E.s, E.w);
      E.ne = (int)E.s.size();
      E.psi.resize(E.ne * E.nk);
      for (int g = 0; g < E.ne; ++g) legendre01(pe, E.s[g], &E.psi[g * E.nk]);
      for (int lf = 0; lf < 3; ++lf)
        for (int fl = 0; fl < 2; ++fl) {
          E.phi[lf][fl].resize(E.ne * E.np);
          for (int g = 0; g < E.ne; ++g) {
            real t = fl ? 1.0 - E.s[g] : E.s[g], xi, eta;
            face_point(lf, t, &xi, &eta);
            dubiner(p, xi, eta, &E.phi[lf][fl][g * E.np], nullptr, nullptr);
          }
        }
    }
}
static void ensure_tables() { std::call_once(g_once, init_tables); }

// ---------------------------------------------------------------------------
// Physics (Sec. 2), templated so that the complex-step derivative works.
// w = (rho, rho u, rho v, E); f[k][f] = flux in direction k of field f.
// ---------------------------------------------------------------------------
static const real CS_H_SC = 1e-30;  // complex step of the divergence in sc_epsilon
template <class T>
static void euler_flux(const T* w, real gam, T f[2][4]) {
  T rho = w[0], mx = w[1], my = w[2], E = w[3];
  T u = mx / rho, v = my / rho;
  T p = (gam - 1.0) * (E - real(0.5) * (mx * u + my * v));
  f[0][0] = mx;      f[0][1] = mx * u + p; f[0][2] = mx * v;     f[0][3] = u * (E + p);
  f[1][0] = my;      f[1][1] = my * u;     f[1][2] = my * v + p; f[1][3] = v * (E + p);
}

// viscous flux f_v(w, q) with q[k][f] = d w_f / d x_k (conserved-variable gradient)
template <class T>
static void ns_viscous_flux(const T* w, const T q[2][4], const orc_params& P, T fv[2][4]) {
  const real gam = P.gamma;
  T rho = w[0], u = w[1] / w[0], v = w[2] / w[0], E = w[3];
  T p = (gam - 1.0) * (E - real(0.5) * rho * (u * u + v * v));
  T dudx[2], dvdx[2], dTdx[2];
  for (int k = 0; k < 2; ++k) {
    T dr = q[k][0];
    dudx[k] = (q[k][1] - u * dr) / rho;
    dvdx[k] = (q[k][2] - v * dr) / rho;
    T dp = (gam - 1.0) * (q[k][3] - (u * q[k][1] + v * q[k][2]) + real(0.5) * (u * u + v * v) * dr);
    dTdx[k] = gam * (dp / rho - p * dr / (rho * rho));
  }
  T Tt = gam * p / rho;                                // T / T_inf
  real S = RLIT(110.4) / P.t_inf;                          // Sutherland C2 / T_inf
  real mu_inf = P.mach / P.reynolds;
  T mu = mu_inf * Tt * std::sqrt(Tt) * (1.0 + S) / (Tt + S);
  T kappa = mu / ((gam - 1.0) * P.prandtl);
  T div = dudx[0] + dvdx[1];
  T txx = mu * (real(2) * dudx[0] - (real(2) / 3) * div);
  T tyy = mu * (real(2) * dvdx[1] - (real(2) / 3) * div);
  T txy = mu * (dudx[1] + dvdx[0]);
  fv[0][0] = 0.0; fv[0][1] = txx; fv[0][2] = txy; fv[0][3] = txx * u + txy * v + kappa * dTdx[0];
  fv[1][0] = 0.0; fv[1][1] = txy; fv[1][2] = tyy; fv[1][3] = txy * u + tyy * v + kappa * dTdx[1];
}

// ---------------------------------------------------------------------------
// Mesh: topology, faces and layouts (the layouts are the library's documented
// conventions, re-derived here from their definition).
// ---------------------------------------------------------------------------
struct OMesh {
  int ne = 0, nf = 0, nfield = 4;
  std::vector<real> xy;        // [ne][3][2]
  std::vector<int> vid, p;       // [ne][3], [ne]
  std::vector<int> face_lo, face_hi, face_el0, face_el1, face_lf0, face_lf1, face_p;
  std::vector<int> elem_face;    // [ne][3], -1 on a boundary face
  std::vector<int> bc;           // [ne][3] boundary kind of local face (0 interior, 1 slip wall, 2 far field)
  std::vector<int64_t> u_off, lam_off, x_off, k_blkoff;
  std::vector<int> k_col;        // [nf][5]
  int64_t u_len = 0, lam_len = 0, x_len = 0, k_len = 0;
  std::vector<real> src;       // [u_len] source s_h in U's layout (w part), empty: s = 0
};

struct Geom {
  real J[2][2], Jinv[2][2], detJ, nrm[3][2], len[3], area, perim;
};
static void elem_geom(const OMesh& M, int K, Geom& g) {
  const real* c = &M.xy[K * 6];
  real x0 = c[0], y0 = c[1], x1 = c[2], y1 = c[3], x2 = c[4], y2 = c[5];
  g.J[0][0] = x1 - x0; g.J[0][1] = x2 - x0;
  g.J[1][0] = y1 - y0; g.J[1][1] = y2 - y0;
  g.detJ = g.J[0][0] * g.J[1][1] - g.J[0][1] * g.J[1][0];
  g.Jinv[0][0] = g.J[1][1] / g.detJ;  g.Jinv[0][1] = -g.J[0][1] / g.detJ;
  g.Jinv[1][0] = -g.J[1][0] / g.detJ; g.Jinv[1][1] = g.J[0][0] / g.detJ;
  g.perim = 0;
  for (int lf = 0; lf < 3; ++lf) {
    int a = lf, b = (lf + 1) % 3;
    real dx = c[2 * b] - c[2 * a], dy = c[2 * b + 1] - c[2 * a + 1];
    g.len[lf] = std::sqrt(dx * dx + dy * dy);
    g.nrm[lf][0] = dy / g.len[lf];
    g.nrm[lf][1] = -dx / g.len[lf];
    g.perim += g.len[lf];
  }
  g.area = 0.5 * g.detJ;
}

static inline int face_len(const OMesh& M, int e) { return e < 0 ? 0 : 4 * (M.face_p[e] + 1); }
static int elem_nt(const OMesh& M, int K) {
  int nt = 0;
  for (int lf = 0; lf < 3; ++lf) nt += face_len(M, M.elem_face[K * 3 + lf]);
  return nt;
}
static int elem_n(const OMesh& M, int K) { return M.nfield * n_basis(M.p[K]); }
static inline int elem_flip(const OMesh& M, int K, int lf) {
  return M.vid[K * 3 + lf] > M.vid[K * 3 + (lf + 1) % 3] ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Element residual (Eqs. hdg_ls1-hdg_ls3 and the element's share of
// hdg_cont), for element K with its coefficient vectors U (Q then W) and the
// traces L of its three faces in local order.  Nu has the layout of U, Nl of L.
// ---------------------------------------------------------------------------
// Shock-capturing viscosity of Sec. 3.2, from the real state U of element K:
//   eps_K = eps_0 (h_K / p_K)^(2 - beta) / |K| * int_K d(w) dx,
//   d(w) = sum over the 4 fields of |(div f_c(w))_f|,
// with h_K the longest edge of K.  The divergence of the convective flux of
// the polynomial w_h is the chain rule sum_k (d f_k / d w)(w) d w / d x_k,
// each term taken as the complex-step derivative of f_k along d w / d x_k.
// For Navier-Stokes the gradient d w / d x_k is the q_h unknown.
static real sc_epsilon(const OMesh& M, const orc_params& P, int K, const Geom& g, const real* U) {
  if (!(P.sc_eps0 > 0.0)) return 0.0;
  const int p = M.p[K], np = n_basis(p);
  const bool ns = (M.nfield == 12);
  const int woff = ns ? 8 * np : 0;
  const VolTab& V = g_vol[p];
  real integral = 0.0;
  for (int q = 0; q < V.nq; ++q) {
    const real* phi = &V.phi[q * np];
    real w[4], grad[2][4];
    for (int f = 0; f < 4; ++f) {
      w[f] = 0.0;
      grad[0][f] = 0.0;
      grad[1][f] = 0.0;
      for (int j = 0; j < np; ++j) {
        const real dx = V.dxi[q * np + j], de = V.deta[q * np + j];
        w[f] += U[woff + f * np + j] * phi[j];
        if (ns) {
          grad[0][f] += U[f * np + j] * phi[j];
          grad[1][f] += U[(4 + f) * np + j] * phi[j];
        } else {
          grad[0][f] += U[f * np + j] * (g.Jinv[0][0] * dx + g.Jinv[1][0] * de);
          grad[1][f] += U[f * np + j] * (g.Jinv[0][1] * dx + g.Jinv[1][1] * de);
        }
      }
    }
    real div[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < 2; ++k) {
      cplx wc[4], fc[2][4];
      for (int f = 0; f < 4; ++f) wc[f] = cplx(w[f], CS_H_SC * grad[k][f]);
      euler_flux(wc, P.gamma, fc);
      for (int f = 0; f < 4; ++f) div[f] += fc[k][f].imag() / CS_H_SC;
    }
    real d = 0.0;
    for (int f = 0; f < 4; ++f) d += std::fabs(div[f]);
    integral += V.w[q] * g.detJ * d;
  }
  const real hK = std::max(g.len[0], std::max(g.len[1], g.len[2]));
  return P.sc_eps0 * std::pow(hK / p, 2.0 - P.sc_beta) / g.area * integral;
}

// Boundary states of Sec. 2.1 (Euler), for the outward unit normal n:
//   slip wall: w_b = (rho, m - (m . n) n, E), so that v_b . n = 0;
//   far field (characteristic upwinding): with f_c'(w) . n = Q Lambda Q^{-1},
//     w_b = Q (P+ Q^{-1} w + P- Q^{-1} w_inf), P+ / P- selecting the
//     characteristics with eigenvalue >= 0 / < 0 (outgoing from the interior /
//     incoming from the far field); equivalently w_b = w + Q P- Q^{-1}(w_inf - w).
// Q holds the right eigenvectors of the normal flux Jacobian at w:
//   (1, u - c n, H - c v_n), (1, u, v, |v|^2/2), (0, t, v_t), (1, u + c n, H + c v_n),
// t = (-n_y, n_x), eigenvalues v_n - c, v_n, v_n, v_n + c.  The upwinding
// decision uses the real part (it is not differentiated).
static real re(real x) { return x; }
static real re(const cplx& x) { return x.real(); }
template <class T>
static void boundary_state(int kind, const T* w, real nx, real ny, const orc_params& P, T* wb) {
  if (kind == 3) {  // no-slip wall (Sec. 2.2): w_b = (rho, 0, 0, E)
    wb[0] = w[0]; wb[1] = 0.0; wb[2] = 0.0; wb[3] = w[3];
    return;
  }
  if (kind == 1) {
    T mn = w[1] * nx + w[2] * ny;
    wb[0] = w[0]; wb[1] = w[1] - mn * nx; wb[2] = w[2] - mn * ny; wb[3] = w[3];
    return;
  }
  const real gam = P.gamma, a = P.aoa * RLIT(3.14159265358979323846264338327950288) / 180.0;
  const real ui = P.mach * std::cos(a), vi = P.mach * std::sin(a), pi = 1.0 / gam;
  const real winf[4] = {1.0, ui, vi, pi / (gam - 1.0) + 0.5 * (ui * ui + vi * vi)};
  T rho = w[0], u = w[1] / rho, v = w[2] / rho;
  T p = (gam - 1.0) * (w[3] - real(0.5) * rho * (u * u + v * v));
  T c = std::sqrt(gam * p / rho), H = (w[3] + p) / rho;
  T vn = u * nx + v * ny, vt = -u * ny + v * nx;
  T Q[4][4] = {{1.0, 1.0, 0.0, 1.0},
               {u - c * nx, u, -ny, u + c * nx},
               {v - c * ny, v, nx, v + c * ny},
               {H - c * vn, real(0.5) * (u * u + v * v), vt, H + c * vn}};
  const real lam[4] = {re(vn - c), re(vn), re(vn), re(vn + c)};
  // y = Q^{-1} (w_inf - w): Gaussian elimination with partial pivoting (by real part)
  T A[4][5];
  for (int i = 0; i < 4; ++i) {
    for (int j = 0; j < 4; ++j) A[i][j] = Q[i][j];
    A[i][4] = winf[i] - w[i];
  }
  for (int k = 0; k < 4; ++k) {
    int pv = k;
    for (int i = k + 1; i < 4; ++i)
      if (std::fabs(re(A[i][k])) > std::fabs(re(A[pv][k]))) pv = i;
    for (int j = 0; j < 5; ++j) std::swap(A[k][j], A[pv][j]);
    for (int i = k + 1; i < 4; ++i) {
      T f = A[i][k] / A[k][k];
      for (int j = k; j < 5; ++j) A[i][j] -= f * A[k][j];
    }
  }
  T y[4];
  for (int i = 3; i >= 0; --i) {
    T sacc = A[i][4];
    for (int j = i + 1; j < 4; ++j) sacc -= A[i][j] * y[j];
    y[i] = sacc / A[i][i];
  }
  for (int i = 0; i < 4; ++i) {
    wb[i] = w[i];
    for (int j = 0; j < 4; ++j)
      if (lam[j] < 0.0) wb[i] += Q[i][j] * y[j];
  }
}

// eps is the element's shock-capturing viscosity (0: none), a constant here.
template <class T>
static void element_residual(const OMesh& M, const orc_params& P, int K, const Geom& g,
                             const T* U, const T* L, T* Nu, T* Nl, real eps) {
  const int p = M.p[K], np = n_basis(p);
  const bool ns = (M.nfield == 12);
  const int woff = ns ? 8 * np : 0;
  const int n = M.nfield * np;
  int nt = elem_nt(M, K);
  for (int r = 0; r < n; ++r) Nu[r] = 0.0;
  for (int r = 0; r < nt; ++r) Nl[r] = 0.0;
  const VolTab& V = g_vol[p];
  std::vector<real> gx(np), gy(np);
  // volume terms
  for (int q = 0; q < V.nq; ++q) {
    const real* phi = &V.phi[q * np];
    const real wq = V.w[q] * g.detJ;
    for (int j = 0; j < np; ++j) {
      real dx = V.dxi[q * np + j], de = V.deta[q * np + j];
      gx[j] = g.Jinv[0][0] * dx + g.Jinv[1][0] * de;
      gy[j] = g.Jinv[0][1] * dx + g.Jinv[1][1] * de;
    }
    T w[4], qv[2][4], fc[2][4], fv[2][4];
    for (int f = 0; f < 4; ++f) {
      w[f] = 0.0;
      for (int j = 0; j < np; ++j) w[f] += U[woff + f * np + j] * phi[j];
    }
    euler_flux(w, P.gamma, fc);
    if (ns) {
      for (int k = 0; k < 2; ++k)
        for (int f = 0; f < 4; ++f) {
          qv[k][f] = 0.0;
          for (int j = 0; j < np; ++j) qv[k][f] += U[(k * 4 + f) * np + j] * phi[j];
        }
      ns_viscous_flux(w, qv, P, fv);
    } else {
      for (int k = 0; k < 2; ++k) for (int f = 0; f < 4; ++f) fv[k][f] = 0.0;
    }
    // -(grad phi_i, f_c(w) - f_v(w,q))_K
    for (int f = 0; f < 4; ++f)
      for (int i = 0; i < np; ++i)
        Nu[woff + f * np + i] -= wq * (gx[i] * (fc[0][f] - fv[0][f]) + gy[i] * (fc[1][f] - fv[1][f]));
    // shock capturing: + eps (grad phi_i, grad w_f)_K (Euler) or (grad phi_i, q_f)_K (NS)
    if (eps != 0.0)
      for (int f = 0; f < 4; ++f) {
        T gwx = 0.0, gwy = 0.0;
        if (ns) {
          gwx = qv[0][f];
          gwy = qv[1][f];
        } else {
          for (int j = 0; j < np; ++j) {
            gwx += U[woff + f * np + j] * gx[j];
            gwy += U[woff + f * np + j] * gy[j];
          }
        }
        for (int i = 0; i < np; ++i) Nu[woff + f * np + i] += wq * eps * (gx[i] * gwx + gy[i] * gwy);
      }
    // (tau, q)_K + (div tau, w)_K
    if (ns)
      for (int k = 0; k < 2; ++k)
        for (int f = 0; f < 4; ++f)
          for (int i = 0; i < np; ++i) {
            real gk = (k == 0) ? gx[i] : gy[i];
            Nu[(k * 4 + f) * np + i] += wq * (phi[i] * qv[k][f] + gk * w[f]);
          }
  }
  // source: -(phi_i, s_h)_K = -det J S_i for the orthonormal basis (Eq. hdg_ls3)
  if (!M.src.empty())
    for (int r = woff; r < n; ++r) Nu[r] -= g.detJ * M.src[M.u_off[K] + r];
  // face terms
  int loff = 0;
  for (int lf = 0; lf < 3; ++lf) {
    int e = M.elem_face[K * 3 + lf];
    if (e < 0) {  // boundary operator of Sec. 3.2: <tau.n, w_b> + <phi, (f_c(w_b) - f_v(w_b, q_b)).n>, no lambda
      const EdgeTab& Eb = g_edge[p][p];
      const int fl = elem_flip(M, K, lf);
      const real nx = g.nrm[lf][0], ny = g.nrm[lf][1];
      for (int gq = 0; gq < Eb.ne; ++gq) {
        const real we = Eb.w[gq] * g.len[lf];
        const real* phi = &Eb.phi[lf][fl][gq * np];
        T w[4], wb[4], fc[2][4], fv[2][4];
        for (int f = 0; f < 4; ++f) {
          w[f] = 0.0;
          for (int j = 0; j < np; ++j) w[f] += U[woff + f * np + j] * phi[j];
        }
        boundary_state(M.bc[K * 3 + lf], w, nx, ny, P, wb);
        euler_flux(wb, P.gamma, fc);
        for (int k = 0; k < 2; ++k) for (int f = 0; f < 4; ++f) fv[k][f] = 0.0;
        if (ns) {
          // q_b = q_h (the interior gradient); at a no-slip adiabatic wall the
          // viscous flux is (0, tau, 0): the energy row (tau.v_b + k grad T)
          // vanishes as v_b = 0 and grad T . n = 0; at a far-field face it is
          // f_v(w_b, q_h) whole
          T qv[2][4];
          for (int k = 0; k < 2; ++k)
            for (int f = 0; f < 4; ++f) {
              qv[k][f] = 0.0;
              for (int j = 0; j < np; ++j) qv[k][f] += U[(k * 4 + f) * np + j] * phi[j];
            }
          ns_viscous_flux(wb, qv, P, fv);
          if (M.bc[K * 3 + lf] == 3) {  // adiabatic no-slip wall: (0, tau, 0)
            fv[0][3] = 0.0;
            fv[1][3] = 0.0;
          }
          // -<tau.n, w_b>_dK in the q equations
          for (int k = 0; k < 2; ++k) {
            const real nk_ = (k == 0) ? nx : ny;
            for (int f = 0; f < 4; ++f)
              for (int j = 0; j < np; ++j) Nu[(k * 4 + f) * np + j] -= we * phi[j] * nk_ * wb[f];
          }
        }
        for (int f = 0; f < 4; ++f)
          for (int j = 0; j < np; ++j)
            Nu[woff + f * np + j] += we * phi[j] * (nx * (fc[0][f] - fv[0][f]) + ny * (fc[1][f] - fv[1][f]));
      }
      continue;
    }
    int pe = M.face_p[e], nk = pe + 1;
    int fl = elem_flip(M, K, lf);
    const EdgeTab& Et = g_edge[p][pe];
    const real nx = g.nrm[lf][0], ny = g.nrm[lf][1];
    for (int gq = 0; gq < Et.ne; ++gq) {
      const real we = Et.w[gq] * g.len[lf];
      const real* phi = &Et.phi[lf][fl][gq * np];
      const real* psi = &Et.psi[gq * nk];
      T w[4], lam[4], qv[2][4], fc[2][4], fv[2][4], fh[4];
      for (int f = 0; f < 4; ++f) {
        w[f] = 0.0;
        for (int j = 0; j < np; ++j) w[f] += U[woff + f * np + j] * phi[j];
        lam[f] = 0.0;
        for (int k = 0; k < nk; ++k) lam[f] += L[loff + f * nk + k] * psi[k];
      }
      euler_flux(lam, P.gamma, fc);
      if (ns) {
        for (int k = 0; k < 2; ++k)
          for (int f = 0; f < 4; ++f) {
            qv[k][f] = 0.0;
            for (int j = 0; j < np; ++j) qv[k][f] += U[(k * 4 + f) * np + j] * phi[j];
          }
        ns_viscous_flux(lam, qv, P, fv);
      } else {
        for (int k = 0; k < 2; ++k) for (int f = 0; f < 4; ++f) fv[k][f] = 0.0;
      }
      // numerical flux  (f_c(lam) - f_v(lam, q)).n - alpha (lam - w)
      for (int f = 0; f < 4; ++f)
        fh[f] = nx * (fc[0][f] - fv[0][f]) + ny * (fc[1][f] - fv[1][f]) - real(P.alpha) * (lam[f] - w[f]);
      for (int f = 0; f < 4; ++f)
        for (int j = 0; j < np; ++j) Nu[woff + f * np + j] += we * phi[j] * fh[f];
      if (ns)  // -<tau.n, lambda>_dK
        for (int k = 0; k < 2; ++k) {
          real nk_ = (k == 0) ? nx : ny;
          for (int f = 0; f < 4; ++f)
            for (int j = 0; j < np; ++j) Nu[(k * 4 + f) * np + j] -= we * phi[j] * nk_ * lam[f];
        }
      // this element's share of <mu, [[f_hat]]>_e
      for (int f = 0; f < 4; ++f)
        for (int k = 0; k < nk; ++k) Nl[loff + f * nk + k] += we * psi[k] * fh[f];
    }
    loff += 4 * nk;
  }
}

// local time step of Sec. 3.3 from the element-mean state (real part of U)
static real local_dt(const OMesh& M, const orc_params& P, int K, const Geom& g, const real* U) {
  const int np = n_basis(M.p[K]);
  const int woff = (M.nfield == 12) ? 8 * np : 0;
  const real c0 = std::sqrt(real(2));  // value of the constant orthonormal mode
  real rho = c0 * U[woff], u = c0 * U[woff + np] / rho, v = c0 * U[woff + 2 * np] / rho,
         E = c0 * U[woff + 3 * np];
  real p = (P.gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v));
  real c = std::sqrt(P.gamma * p / rho);
  real lam_c = (std::sqrt(u * u + v * v) + c) * g.perim;
  real lam_v = 0.0;
  if (M.nfield == 12) {
    real Tt = P.gamma * p / rho, S = RLIT(110.4) / P.t_inf;
    real mu = (P.mach / P.reynolds) * Tt * std::sqrt(Tt) * (1.0 + S) / (Tt + S);
    lam_v = P.gamma * mu / (P.prandtl * rho) * g.perim * g.perim / g.area;
  }
  return P.cfl * g.area / (lam_c + 4.0 * lam_v);
}

// Element blocks: A = dNu/dU, B = dNu/dL, C = dNl/dU, D = dNl/dL (complex
// step, exact to rounding), F = -Nu, H = -Nl; pseudo-time mass on the W block.
static const real CS_H = 1e-30;
static void element_blocks(const OMesh& M, const orc_params& P, int K, const real* U, const real* L,
                           std::vector<real>& A, std::vector<real>& B, std::vector<real>& C,
                           std::vector<real>& D, std::vector<real>& F, std::vector<real>& H) {
  Geom g;
  elem_geom(M, K, g);
  const int n = elem_n(M, K), nt = elem_nt(M, K);
  A.assign(n * n, 0.0); B.assign(n * nt, 0.0); C.assign(nt * n, 0.0); D.assign(nt * nt, 0.0);
  F.assign(n, 0.0); H.assign(nt, 0.0);
  std::vector<cplx> Uc(n), Lc(nt), Nu(n), Nl(nt);
  for (int r = 0; r < n; ++r) Uc[r] = U[r];
  for (int r = 0; r < nt; ++r) Lc[r] = L[r];
  const real eps = sc_epsilon(M, P, K, g, U);  // frozen: not differentiated
  element_residual<cplx>(M, P, K, g, Uc.data(), Lc.data(), Nu.data(), Nl.data(), eps);
  for (int r = 0; r < n; ++r) F[r] = -Nu[r].real();
  for (int r = 0; r < nt; ++r) H[r] = -Nl[r].real();
  for (int c = 0; c < n + nt; ++c) {
    if (c < n) Uc[c] += cplx(0.0, CS_H); else Lc[c - n] += cplx(0.0, CS_H);
    element_residual<cplx>(M, P, K, g, Uc.data(), Lc.data(), Nu.data(), Nl.data(), eps);
    if (c < n) Uc[c] = U[c]; else Lc[c - n] = L[c - n];
    for (int r = 0; r < n; ++r) {
      real d = Nu[r].imag() / CS_H;
      if (c < n) A[r * n + c] = d; else B[r * nt + (c - n)] = d;
    }
    for (int r = 0; r < nt; ++r) {
      real d = Nl[r].imag() / CS_H;
      if (c < n) C[r * n + c] = d; else D[r * nt + (c - n)] = d;
    }
  }
  if (P.cfl > 0.0) {
    real dt = local_dt(M, P, K, g, U);
    const int np = n_basis(M.p[K]);
    const int woff = (M.nfield == 12) ? 8 * np : 0;
    for (int r = woff; r < n; ++r) A[r * n + r] += g.detJ / dt;
  }
}

// dense LU with partial pivoting (first maximal |pivot| wins), in place
static int lu_factor(int n, std::vector<real>& A, std::vector<int>& piv) {
  piv.resize(n);
  for (int k = 0; k < n; ++k) {
    int r = k;
    real best = std::fabs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > best) { best = std::fabs(A[i * n + k]); r = i; }
    piv[k] = r;
    if (best == 0.0) return 1;
    if (r != k)
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[r * n + j]);
    for (int i = k + 1; i < n; ++i) {
      A[i * n + k] /= A[k * n + k];
      real lik = A[i * n + k];
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= lik * A[k * n + j];
    }
  }
  return 0;
}
// solve A x = b for nrhs columns of the row-major n x nrhs matrix X (in place)
static void lu_solve(int n, const std::vector<real>& LU, const std::vector<int>& piv, int nrhs, real* X) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k)
      for (int c = 0; c < nrhs; ++c) std::swap(X[k * nrhs + c], X[piv[k] * nrhs + c]);
  for (int c = 0; c < nrhs; ++c) {
    for (int i = 0; i < n; ++i) {
      real s = X[i * nrhs + c];
      for (int j = 0; j < i; ++j) s -= LU[i * n + j] * X[j * nrhs + c];
      X[i * nrhs + c] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
      real s = X[i * nrhs + c];
      for (int j = i + 1; j < n; ++j) s -= LU[i * n + j] * X[j * nrhs + c];
      X[i * nrhs + c] = s / LU[i * n + i];
    }
  }
}

// gather of element K's trace vector from the global Lambda (faces in local order)
static void gather_trace(const OMesh& M, int K, const real* Lam, std::vector<real>& L) {
  L.clear();
  for (int lf = 0; lf < 3; ++lf) {
    int e = M.elem_face[K * 3 + lf];
    if (e < 0) continue;  // boundary face: no trace unknowns
    int len = face_len(M, e);
    for (int r = 0; r < len; ++r) L.push_back(Lam[M.lam_off[e] + r]);
  }
}

// Condensation of one element: X = A^{-1}[B | F] (n x (nt+1), row-major),
// S = D - C X_B (nt x nt), Ek = H - C X_F (nt).  Returns 1 on a zero pivot.
static int element_condense(const OMesh& M, const orc_params& P, int K, const real* U, const real* Lam,
                            std::vector<real>& X, std::vector<real>& S, std::vector<real>& Ek,
                            std::vector<real>* Nu_out, std::vector<real>* Nl_out) {
  std::vector<real> L, A, B, C, D, F, H;
  gather_trace(M, K, Lam, L);
  const real* UK = U + M.u_off[K];
  element_blocks(M, P, K, UK, L.data(), A, B, C, D, F, H);
  const int n = elem_n(M, K), nt = elem_nt(M, K), nr = nt + 1;
  if (Nu_out) { Nu_out->resize(n); for (int r = 0; r < n; ++r) (*Nu_out)[r] = -F[r]; }
  if (Nl_out) { Nl_out->resize(nt); for (int r = 0; r < nt; ++r) (*Nl_out)[r] = -H[r]; }
  X.assign(n * nr, 0.0);
  for (int r = 0; r < n; ++r) {
    for (int c = 0; c < nt; ++c) X[r * nr + c] = B[r * nt + c];
    X[r * nr + nt] = F[r];
  }
  std::vector<int> piv;
  int st = lu_factor(n, A, piv);
  S.assign(nt * nt, 0.0);
  Ek.assign(nt, 0.0);
  if (st) return st;
  lu_solve(n, A, piv, nr, X.data());
  for (int r = 0; r < nt; ++r) {
    for (int c = 0; c < nt; ++c) {
      real s = D[r * nt + c];
      for (int k = 0; k < n; ++k) s -= C[r * n + k] * X[k * nr + c];
      S[r * nt + c] = s;
    }
    real s = H[r];
    for (int k = 0; k < n; ++k) s -= C[r * n + k] * X[k * nr + nt];
    Ek[r] = s;
  }
  return 0;
}

// ---------------------------------------------------------------------------
// C interface (ctypes)
// ---------------------------------------------------------------------------
extern "C" {
#ifndef ORC_EXTENDED

// n-point Gauss-Jacobi rule, weight (1-x)^alpha (1+x)^beta on [-1,1]
int orc_gauss_jacobi(int n, double alpha, double beta, double* x, double* w) {
  if (n < 1 || n > 64) return 1;
  gauss_jacobi(n, alpha, beta, x, w);
  return 0;
}
// collapsed Gauss rule on the reference triangle: (p+2)^2 points
int orc_tri_rule(int p, double* xi, double* eta, double* w) {
  if (p < 0 || p > 20) return 1;
  std::vector<double> a, b, c;
  tri_rule(p, a, b, c);
  std::copy(a.begin(), a.end(), xi); std::copy(b.begin(), b.end(), eta); std::copy(c.begin(), c.end(), w);
  return 0;
}
// (pe+2)-point Gauss-Legendre rule on [0,1]
int orc_edge_rule(int pe, double* s, double* w) {
  if (pe < 0 || pe > 40) return 1;
  std::vector<double> a, b;
  edge_rule(pe, a, b);
  std::copy(a.begin(), a.end(), s); std::copy(b.begin(), b.end(), w);
  return 0;
}
// Dubiner basis values/gradients at npts points: out arrays [npts][n_basis(p)]
int orc_dubiner(int p, int npts, const double* xi, const double* eta, double* phi, double* dxi, double* deta) {
  if (p < 0 || p > 12) return 1;
  int np = n_basis(p);
  for (int q = 0; q < npts; ++q)
    dubiner(p, xi[q], eta[q], phi + q * np, dxi ? dxi + q * np : nullptr, deta ? deta + q * np : nullptr);
  return 0;
}
int orc_legendre01(int pe, int npts, const double* s, double* psi) {
  for (int q = 0; q < npts; ++q) legendre01(pe, s[q], psi + q * (pe + 1));
  return 0;
}
// physics at one state: f[2][4]
void orc_euler_flux(const double* w, double gamma, double* f) {
  double ff[2][4];
  euler_flux(w, gamma, ff);
  std::memcpy(f, ff, sizeof(ff));
}
void orc_ns_viscous_flux(const double* w, const double* q, const orc_params* P, double* fv) {
  double qq[2][4], ff[2][4];
  std::memcpy(qq, q, sizeof(qq));
  ns_viscous_flux(w, qq, *P, ff);
  std::memcpy(fv, ff, sizeof(ff));
}

#endif  // ORC_EXTENDED

// Build the mesh.  Returns 0 ok, 2 bad input (non-positive det J, p out of
// range, a face not shared by exactly two elements, two elements sharing two faces).
// elem_bc (may be null: every face interior) [n_elem][3]: 0 interior, 1 slip
// wall (Euler), 2 far field (both models), 3 no-slip adiabatic wall
// (Navier-Stokes);
// boundary faces carry no trace unknowns.
int orc_mesh_create(int n_elem, int nfield, const double* elem_xy, const int32_t* elem_vid,
                    const int8_t* elem_p, const int8_t* elem_bc, void** out) {
  ensure_tables();
  if (n_elem < 1 || (nfield != 4 && nfield != 12)) return 2;
  OMesh* M = new OMesh();
  M->ne = n_elem; M->nfield = nfield;
  M->xy.assign(elem_xy, elem_xy + 6 * n_elem);
  M->vid.assign(elem_vid, elem_vid + 3 * n_elem);
  M->p.resize(n_elem);
  M->bc.assign(3 * n_elem, 0);
  for (int t = 0; elem_bc && t < 3 * n_elem; ++t) {
    M->bc[t] = elem_bc[t];
    const int b = M->bc[t];
    const bool ok = b == 0 || (nfield == 4 && (b == 1 || b == 2)) || (nfield == 12 && (b == 2 || b == 3));
    if (!ok) { delete M; return 2; }
  }
  for (int K = 0; K < n_elem; ++K) {
    M->p[K] = elem_p[K];
    Geom g;
    elem_geom(*M, K, g);
    if (M->p[K] < 1 || M->p[K] > 4 || !(g.detJ > 0.0)) { delete M; return 2; }
  }
  struct Ent { int lo, hi, K, lf; };
  std::vector<Ent> ents;
  for (int K = 0; K < n_elem; ++K)
    for (int lf = 0; lf < 3; ++lf) {
      if (M->bc[K * 3 + lf]) continue;  // boundary face: no partner, no trace
      int a = M->vid[K * 3 + lf], b = M->vid[K * 3 + (lf + 1) % 3];
      ents.push_back({std::min(a, b), std::max(a, b), K, lf});
    }
  std::sort(ents.begin(), ents.end(), [](const Ent& x, const Ent& y) {
    if (x.lo != y.lo) return x.lo < y.lo;
    if (x.hi != y.hi) return x.hi < y.hi;
    return x.K < y.K;
  });
  M->elem_face.assign(3 * n_elem, -1);
  for (size_t i = 0; i < ents.size(); i += 2) {
    if (i + 1 >= ents.size() || ents[i + 1].lo != ents[i].lo || ents[i + 1].hi != ents[i].hi ||
        (i + 2 < ents.size() && ents[i + 2].lo == ents[i].lo && ents[i + 2].hi == ents[i].hi) ||
        ents[i].K == ents[i + 1].K) {
      delete M; return 2;
    }
    int f = M->nf++;
    M->face_lo.push_back(ents[i].lo); M->face_hi.push_back(ents[i].hi);
    M->face_el0.push_back(ents[i].K); M->face_lf0.push_back(ents[i].lf);
    M->face_el1.push_back(ents[i + 1].K); M->face_lf1.push_back(ents[i + 1].lf);
    M->face_p.push_back(std::max(M->p[ents[i].K], M->p[ents[i + 1].K]));
    M->elem_face[ents[i].K * 3 + ents[i].lf] = f;
    M->elem_face[ents[i + 1].K * 3 + ents[i + 1].lf] = f;
  }
  // layouts
  M->u_off.resize(n_elem + 1); M->x_off.resize(n_elem + 1);
  M->u_off[0] = 0; M->x_off[0] = 0;
  for (int K = 0; K < n_elem; ++K) {
    int n = elem_n(*M, K), nt = elem_nt(*M, K);
    M->u_off[K + 1] = M->u_off[K] + n;
    M->x_off[K + 1] = M->x_off[K] + (int64_t)n * (nt + 1);
  }
  M->u_len = M->u_off[n_elem]; M->x_len = M->x_off[n_elem];
  M->lam_off.resize(M->nf + 1);
  M->lam_off[0] = 0;
  for (int f = 0; f < M->nf; ++f) M->lam_off[f + 1] = M->lam_off[f] + 4 * (M->face_p[f] + 1);
  M->lam_len = M->lam_off[M->nf];
  M->k_col.resize(5 * M->nf);
  M->k_blkoff.resize(5 * M->nf + 1);
  M->k_blkoff[0] = 0;
  for (int f = 0; f < M->nf; ++f) {
    std::vector<int> cols = {f};
    for (int s = 0; s < 2; ++s) {
      int K = s ? M->face_el1[f] : M->face_el0[f];
      for (int lf = 0; lf < 3; ++lf) {
        int e = M->elem_face[K * 3 + lf];
        if (e != f && e >= 0) cols.push_back(e);
      }
    }
    std::sort(cols.begin(), cols.end());
    if (std::adjacent_find(cols.begin(), cols.end()) != cols.end()) { delete M; return 2; }
    // columns ascending, then unused slots (-1, empty blocks) next to boundary faces
    for (int b = 0; b < 5; ++b) {
      const int cb = b < (int)cols.size() ? cols[b] : -1;
      M->k_col[5 * f + b] = cb;
      int64_t sz = (int64_t)(4 * (M->face_p[f] + 1)) * face_len(*M, cb);
      M->k_blkoff[5 * f + b + 1] = M->k_blkoff[5 * f + b] + sz;
    }
  }
  M->k_len = M->k_blkoff[5 * M->nf];
  *out = M;
  return 0;
}
void orc_mesh_destroy(void* h) { delete (OMesh*)h; }

// Source term s of Eq. (hdg_ls3), given as the coefficients of its L2
// projection in U's layout [u_len] (only the w part is read); NULL: s = 0.
void orc_mesh_set_source(void* h, const double* S) {
  OMesh* M = (OMesh*)h;
  if (S) M->src.assign(S, S + M->u_len);
  else M->src.clear();
}

// sizes: [n_face, u_len, lam_len, x_len, k_len]
void orc_mesh_sizes(void* h, int64_t* out) {
  OMesh* M = (OMesh*)h;
  out[0] = M->nf; out[1] = M->u_len; out[2] = M->lam_len; out[3] = M->x_len; out[4] = M->k_len;
}
// layout arrays; any pointer may be null
void orc_mesh_arrays(void* h, int32_t* face_vid, int32_t* face_el, int32_t* face_lf, int32_t* face_p,
                     int32_t* elem_face, int64_t* u_off, int64_t* lam_off, int64_t* x_off, int32_t* k_col,
                     int64_t* k_blkoff) {
  OMesh* M = (OMesh*)h;
  for (int f = 0; f < M->nf; ++f) {
    if (face_vid) { face_vid[2 * f] = M->face_lo[f]; face_vid[2 * f + 1] = M->face_hi[f]; }
    if (face_el) { face_el[2 * f] = M->face_el0[f]; face_el[2 * f + 1] = M->face_el1[f]; }
    if (face_lf) { face_lf[2 * f] = M->face_lf0[f]; face_lf[2 * f + 1] = M->face_lf1[f]; }
    if (face_p) face_p[f] = M->face_p[f];
  }
  if (elem_face) std::copy(M->elem_face.begin(), M->elem_face.end(), elem_face);
  if (u_off) std::copy(M->u_off.begin(), M->u_off.end(), u_off);
  if (lam_off) std::copy(M->lam_off.begin(), M->lam_off.end(), lam_off);
  if (x_off) std::copy(M->x_off.begin(), M->x_off.end(), x_off);
  if (k_col) std::copy(M->k_col.begin(), M->k_col.end(), k_col);
  if (k_blkoff) std::copy(M->k_blkoff.begin(), M->k_blkoff.end(), k_blkoff);
}

#ifndef ORC_EXTENDED
// Residual of element K (real): Nu [n], Nl [nt] (this element's share of the trace rows).
int orc_element_residual(void* h, const orc_params* P, int K, const double* U, const double* Lam,
                         double* Nu, double* Nl) {
  OMesh* M = (OMesh*)h;
  Geom g;
  elem_geom(*M, K, g);
  std::vector<double> L;
  gather_trace(*M, K, Lam, L);
  element_residual<double>(*M, *P, K, g, U + M->u_off[K], L.data(), Nu, Nl,
                           sc_epsilon(*M, *P, K, g, U + M->u_off[K]));
  return 0;
}

// Element blocks of element K (row-major): A [n][n], B [n][nt], C [nt][n], D [nt][nt], F [n], H [nt]
int orc_element_blocks(void* h, const orc_params* P, int K, const double* U, const double* Lam, double* A,
                       double* B, double* C, double* D, double* F, double* H) {
  OMesh* M = (OMesh*)h;
  std::vector<double> L, a, b, c, d, f, hh;
  gather_trace(*M, K, Lam, L);
  element_blocks(*M, *P, K, U + M->u_off[K], L.data(), a, b, c, d, f, hh);
  std::copy(a.begin(), a.end(), A); std::copy(b.begin(), b.end(), B);
  std::copy(c.begin(), c.end(), C); std::copy(d.begin(), d.end(), D);
  std::copy(f.begin(), f.end(), F); std::copy(hh.begin(), hh.end(), H);
  return 0;
}

// Condensation of one element K: X [n][nt+1], S [nt][nt], Ek [nt]; status 0 ok / 1 zero pivot
int orc_element_condense(void* h, const orc_params* P, int K, const double* U, const double* Lam, double* X,
                         double* S, double* Ek) {
  OMesh* M = (OMesh*)h;
  std::vector<double> x, s, e;
  int st = element_condense(*M, *P, K, U, Lam, x, s, e, nullptr, nullptr);
  std::copy(x.begin(), x.end(), X); std::copy(s.begin(), s.end(), S); std::copy(e.begin(), e.end(), Ek);
  return st;
}

// Assembly of one element's condensed blocks into K, E and the trace residual
// (the element's 3x3 face-pair blocks of S_K into the 5-block rows of its faces).
static void scatter_element(const OMesh& M, int K, const std::vector<double>& s, const std::vector<double>& ek,
                            const std::vector<double>& nl, double* Kv, double* E, double* resLam) {
  const int nt = elem_nt(M, K);
  int roff = 0;
  for (int a = 0; a < 3; ++a) {
    int ea = M.elem_face[K * 3 + a], na = face_len(M, ea);
    if (ea < 0) continue;
    for (int r = 0; r < na; ++r) {
      E[M.lam_off[ea] + r] += ek[roff + r];
      resLam[M.lam_off[ea] + r] += nl[roff + r];
    }
    int coff = 0;
    for (int b = 0; b < 3; ++b) {
      int eb = M.elem_face[K * 3 + b], nb = face_len(M, eb);
      if (eb < 0) continue;
      int slot = -1;
      for (int t = 0; t < 5; ++t)
        if (M.k_col[5 * ea + t] == eb) slot = t;
      double* blk = Kv + M.k_blkoff[5 * ea + slot];
      for (int r = 0; r < na; ++r)
        for (int c = 0; c < nb; ++c) blk[r * nb + c] += s[(roff + r) * nt + coff + c];
      coff += nb;
    }
    roff += na;
  }
}

// Same, with the per-element work of [k0, k1) spread over nthreads threads
// (std::thread; each element's arithmetic is unchanged); the assembly runs
// afterwards in ascending element order, so every output is bitwise the same
// as with one thread.
int orc_condense_mt(void* h, const orc_params* P, const double* U, const double* Lam, double* X, double* Kv,
                    double* E, double* resU, double* resLam, int32_t* status, int k0, int k1, int nthreads) {
  OMesh* M = (OMesh*)h;
  if (k1 <= k0) { k0 = 0; k1 = M->ne; }
  if (nthreads < 1) nthreads = 1;
  std::fill(Kv, Kv + M->k_len, 0.0);
  std::fill(E, E + M->lam_len, 0.0);
  std::fill(resLam, resLam + M->lam_len, 0.0);
  const int cnt = k1 - k0;
  std::vector<std::vector<double>> S(cnt), EK(cnt), NL(cnt);
  auto work = [&](int t) {
    for (int i = t; i < cnt; i += nthreads) {
      const int K = k0 + i;
      std::vector<double> x, nu;
      status[K] = element_condense(*M, *P, K, U, Lam, x, S[i], EK[i], &nu, &NL[i]);
      std::copy(x.begin(), x.end(), X + M->x_off[K]);
      std::copy(nu.begin(), nu.end(), resU + M->u_off[K]);
    }
  };
  if (nthreads == 1) {
    work(0);
  } else {
    std::vector<std::thread> th;
    for (int t = 0; t < nthreads; ++t) th.emplace_back(work, t);
    for (auto& t : th) t.join();
  }
  int bad = 0;
  for (int i = 0; i < cnt; ++i) {
    bad |= status[k0 + i];
    scatter_element(*M, k0 + i, S[i], EK[i], NL[i], Kv, E, resLam);
  }
  return bad ? 1 : 0;
}

// Whole-mesh condensation and assembly: X [x_len], K [k_len], E [lam_len],
// resU [u_len], resLam [lam_len] (sum over both sides), status [n_elem].
// Elements are processed in ascending id, so every diagonal block and every
// entry of E is (lower element's contribution) + (higher element's).
// Elements [k0, k1) only if k1 > k0 (then K/E/resLam hold partial sums).
int orc_condense(void* h, const orc_params* P, const double* U, const double* Lam, double* X, double* Kv,
                 double* E, double* resU, double* resLam, int32_t* status, int k0, int k1) {
  return orc_condense_mt(h, P, U, Lam, X, Kv, E, resU, resLam, status, k0, k1, 1);
}

// Reconstruction, Eq. (ls): dU_K = X_F - X_B dLambda_K for every element.
int orc_recover(void* h, const double* X, const double* dLam, double* dU) {
  OMesh* M = (OMesh*)h;
  for (int K = 0; K < M->ne; ++K) {
    std::vector<double> L;
    gather_trace(*M, K, dLam, L);
    const int n = elem_n(*M, K), nt = elem_nt(*M, K), nr = nt + 1;
    const double* XK = X + M->x_off[K];
    for (int r = 0; r < n; ++r) {
      double s = XK[r * nr + nt];
      for (int c = 0; c < nt; ++c) s -= XK[r * nr + c] * L[c];
      dU[M->u_off[K] + r] = s;
    }
  }
  return 0;
}

// Global residual (U rows then Lambda rows summed over both sides), real.
int orc_global_residual(void* h, const orc_params* P, const double* U, const double* Lam, double* R) {
  OMesh* M = (OMesh*)h;
  std::fill(R, R + M->u_len + M->lam_len, 0.0);
  for (int K = 0; K < M->ne; ++K) {
    Geom g;
    elem_geom(*M, K, g);
    std::vector<double> L;
    gather_trace(*M, K, Lam, L);
    std::vector<double> nu(elem_n(*M, K)), nl(elem_nt(*M, K));
    element_residual<double>(*M, *P, K, g, U + M->u_off[K], L.data(), nu.data(), nl.data(),
                             sc_epsilon(*M, *P, K, g, U + M->u_off[K]));
    std::copy(nu.begin(), nu.end(), R + M->u_off[K]);
    int roff = 0;
    for (int a = 0; a < 3; ++a) {
      int ea = M->elem_face[K * 3 + a], na = face_len(*M, ea);
      for (int r = 0; r < na; ++r) R[M->u_len + M->lam_off[ea] + r] += nl[roff + r];
      roff += na;
    }
  }
  return 0;
}

// Monolithic linearised system for tiny meshes: the Jacobian of the global
// residual by complex step on every global unknown (U then Lambda), the
// pseudo-time mass on each element's W block, solved densely:
//   J [dU; dLam] = -R.   Returns 1 if the dense matrix is singular.
// Jout (optional) receives the (u_len+lam_len)^2 row-major matrix.
int orc_monolithic(void* h, const orc_params* P, const double* U, const double* Lam, double* dU,
                   double* dLam, double* Jout) {
  OMesh* M = (OMesh*)h;
  const int64_t N = M->u_len + M->lam_len;
  if (N > 4000) return 2;
  std::vector<double> J(N * N, 0.0), R(N);
  std::vector<cplx> Uc(U, U + M->u_len), Lc(Lam, Lam + M->lam_len);
  orc_global_residual(h, P, U, Lam, R.data());
  for (int64_t c = 0; c < N; ++c) {
    if (c < M->u_len) Uc[c] += cplx(0.0, CS_H); else Lc[c - M->u_len] += cplx(0.0, CS_H);
    std::vector<cplx> Rc(N, 0.0);
    for (int K = 0; K < M->ne; ++K) {
      Geom g;
      elem_geom(*M, K, g);
      std::vector<cplx> L;
      for (int lf = 0; lf < 3; ++lf) {
        int e = M->elem_face[K * 3 + lf];
        for (int r = 0; r < face_len(*M, e); ++r) L.push_back(Lc[M->lam_off[e] + r]);
      }
      std::vector<cplx> nu(elem_n(*M, K)), nl(elem_nt(*M, K));
      element_residual<cplx>(*M, *P, K, g, Uc.data() + M->u_off[K], L.data(), nu.data(), nl.data(),
                             sc_epsilon(*M, *P, K, g, U + M->u_off[K]));
      for (size_t r = 0; r < nu.size(); ++r) Rc[M->u_off[K] + r] = nu[r];
      int roff = 0;
      for (int a = 0; a < 3; ++a) {
        int ea = M->elem_face[K * 3 + a], na = face_len(*M, ea);
        for (int r = 0; r < na; ++r) Rc[M->u_len + M->lam_off[ea] + r] += nl[roff + r];
        roff += na;
      }
    }
    if (c < M->u_len) Uc[c] = U[c]; else Lc[c - M->u_len] = Lam[c - M->u_len];
    for (int64_t r = 0; r < N; ++r) J[r * N + c] = Rc[r].imag() / CS_H;
  }
  if (P->cfl > 0.0)
    for (int K = 0; K < M->ne; ++K) {
      Geom g;
      elem_geom(*M, K, g);
      double dt = local_dt(*M, *P, K, g, U + M->u_off[K]);
      const int np = n_basis(M->p[K]), woff = (M->nfield == 12) ? 8 * np : 0;
      for (int r = woff; r < elem_n(*M, K); ++r) {
        int64_t gr = M->u_off[K] + r;
        J[gr * N + gr] += g.detJ / dt;
      }
    }
  if (Jout) std::copy(J.begin(), J.end(), Jout);
  std::vector<double> x(N);
  for (int64_t r = 0; r < N; ++r) x[r] = -R[r];
  std::vector<int> piv;
  if (lu_factor((int)N, J, piv)) return 1;
  lu_solve((int)N, J, piv, 1, x.data());
  std::copy(x.begin(), x.begin() + M->u_len, dU);
  std::copy(x.begin() + M->u_len, x.end(), dLam);
  return 0;
}

// The CFL law of Eq. (cfl) (Sec. 3.3): a smooth ramp up to c0 over n0 steps,
// then growth by 1 + c1 max(0, log(||N^{n-1}|| / ||N^n||)) per step.
double orc_cfl_law(int n, double c0, double c1, int n0, double cfl_prev, double res_prev, double res_cur) {
  if (n <= n0) {
    const double t = (double)n / (double)n0;
    return c0 * (3.0 * t * t - 2.0 * t * t * t);
  }
  return cfl_prev * (1.0 + c1 * std::max(0.0, std::log(res_prev / res_cur)));
}

// Boundary state w_b(w) of Sec. 2.1 for kind 1 (slip wall) or 2 (far field), normal n.
void orc_boundary_state(int kind, const double* w, double nx, double ny, const orc_params* P, double* wb) {
  boundary_state(kind, w, nx, ny, *P, wb);
}

// Shock-capturing viscosity eps_K of element K (0 when P->sc_eps0 <= 0).
double orc_sc_epsilon(void* h, const orc_params* P, int K, const double* U) {
  OMesh* M = (OMesh*)h;
  Geom g;
  elem_geom(*M, K, g);
  return sc_epsilon(*M, *P, K, g, U + M->u_off[K]);
}

// ---------------------------------------------------------------------------
// Adaptation decisions (Sec. 4): smoothness sensor, element indicator, Doerfler
// marking, choice between h- and p-refinement.
// ---------------------------------------------------------------------------
// S_K = (w - w*, w - w*)_K / (w, w)_K, w* the L2 projection of w onto degree
// p_K - 1 (Sec. 4.4).  The inner product of the vector w sums its four
// conserved components; with the orthonormal hierarchical basis (mass det J * I)
// w - w* is the part of w on the degree-p_K modes, so S_K is a ratio of sums of
// squared coefficients.  Written here as the quotient of the two L2 norms
// integrated by the element's volume rule (the same number, by orthonormality).
double orc_smoothness(void* h, int K, const double* U) {
  OMesh* M = (OMesh*)h;
  const int p = M->p[K], np = n_basis(p), npl = n_basis(p - 1);
  const int woff = (M->nfield == 12) ? 8 * np : 0;
  const double* c = U + M->u_off[K] + woff;
  const VolTab& V = g_vol[p];
  double num = 0.0, den = 0.0;
  for (int q = 0; q < V.nq; ++q) {
    const double* phi = &V.phi[q * np];
    for (int f = 0; f < 4; ++f) {
      double w = 0.0, wh = 0.0;
      for (int j = 0; j < np; ++j) {
        w += c[f * np + j] * phi[j];
        if (j >= npl) wh += c[f * np + j] * phi[j];
      }
      num += V.w[q] * wh * wh;
      den += V.w[q] * w * w;
    }
  }
  return den > 0.0 ? num / den : 0.0;
}

// Doerfler marking (Sec. 4.3): the smallest set M with eta_M >= (1 - theta) eta_T,
// eta_M^2 = sum_{K in M} eta_K^2.  Order-independent sums: each eta_K^2 is taken
// in fixed point, v_K = floor(eta_K^2 / max eta^2 * 2^bits), bits = 62 -
// ceil(log2(n + 1)); the set is the first elements in the order (v descending,
// index ascending) whose cumulative v reaches ceil((1 - theta)^2 sum v).
// Then (Sec. 4.4) marked elements with S_K < eps_s get p-enrichment (1), the
// others mesh refinement (2); unmarked 0.  Returns the number marked.
static int fixed_bits(int n) {
  int lg = 0;
  while ((1LL << lg) < (long long)n + 1) ++lg;
  return 62 - lg;
}
int orc_adapt_mark(int n, const double* eta2, const double* sensor, double theta, double eps_s, int8_t* code) {
  double mx = 0.0;
  for (int K = 0; K < n; ++K) mx = std::max(mx, eta2[K]);
  std::vector<long long> v(n, 0);
  const int bits = fixed_bits(n);
  if (mx > 0.0)
    for (int K = 0; K < n; ++K) v[K] = (long long)std::floor(std::ldexp(eta2[K] / mx, bits));
  unsigned long long tot = 0;
  for (int K = 0; K < n; ++K) tot += (unsigned long long)v[K];
  // target = ceil(tot * q), q = (1 - theta)^2 in binary64, exactly: q = mant * 2^ex
  const double q = (1.0 - theta) * (1.0 - theta);
  unsigned long long target = 0;
  if (q > 0.0 && tot > 0) {
    int ex = 0;
    const double fr = std::frexp(q, &ex);                                  // q = fr 2^ex, fr in [0.5, 1)
    const unsigned long long mant = (unsigned long long)std::ldexp(fr, 53);  // q = mant 2^(ex - 53)
    const unsigned __int128 prod = (unsigned __int128)tot * mant;
    const int sh = 53 - ex;                                                  // >= 52 for q <= 1
    const unsigned __int128 one = 1;
    target = sh >= 120 ? 1ULL : (unsigned long long)((prod + (one << sh) - 1) >> sh);
  }
  std::vector<int> idx(n);
  for (int K = 0; K < n; ++K) idx[K] = K;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return v[a] > v[b]; });
  for (int K = 0; K < n; ++K) code[K] = 0;
  unsigned long long cum = 0;
  int marked = 0;
  for (int t = 0; t < n && cum < target; ++t) {
    const int K = idx[t];
    cum += (unsigned long long)v[K];
    code[K] = sensor[K] < eps_s ? 1 : 2;
    ++marked;
  }
  return marked;
}

// Dense LU solve helper for tests (A n x n row-major, b -> x in place).
int orc_dense_solve(int n, const double* A, double* b) {
  std::vector<double> a(A, A + (int64_t)n * n);
  std::vector<int> piv;
  if (lu_factor(n, a, piv)) return 1;
  lu_solve(n, a, piv, 1, b);
  return 0;
}

#else  // ORC_EXTENDED
// The extended-precision build exposes the mesh calls above and the local
// condensation of chosen elements: inputs are binary64 (as given to the
// binary64 oracle), everything else -- tables, geometry, residual, complex-step
// Jacobian, LU, Schur -- runs in long double; the results are returned rounded
// to binary64 (relative 1.1e-16, far below the errors this build measures).

// Condensation of element K: X [n][nt+1], S [nt][nt], Ek [nt] (as orc_element_condense),
// and the reconstruction dU_K = X_F - X_B dLambda_K [n] (Eq. ls).  Returns 0 ok / 1 zero pivot.
int orcx_element_condense(void* h, const orc_params* P, int K, const double* U, const double* Lam,
                          const double* dLam, double* X, double* S, double* Ek, double* dU) {
  OMesh* M = (OMesh*)h;
  const int n = elem_n(*M, K), nt = elem_nt(*M, K), nr = nt + 1;
  std::vector<real> Ur(M->u_len), Lr(M->lam_len), dLr(M->lam_len), x, s, e;
  for (int64_t i = 0; i < M->u_len; ++i) Ur[i] = U[i];
  for (int64_t i = 0; i < M->lam_len; ++i) { Lr[i] = Lam[i]; dLr[i] = dLam[i]; }
  const int st = element_condense(*M, *P, K, Ur.data(), Lr.data(), x, s, e, nullptr, nullptr);
  for (size_t i = 0; i < x.size(); ++i) X[i] = (double)x[i];
  for (size_t i = 0; i < s.size(); ++i) S[i] = (double)s[i];
  for (size_t i = 0; i < e.size(); ++i) Ek[i] = (double)e[i];
  std::vector<real> dl;
  gather_trace(*M, K, dLr.data(), dl);
  for (int r = 0; r < n; ++r) {
    real acc = x[r * nr + nt];
    for (int c = 0; c < nt; ++c) acc -= x[r * nr + c] * dl[c];
    dU[r] = (double)acc;
  }
  return st;
}

// Assembled condensed right-hand side of face f, E_f = sum over its two sides of
// the element contributions E_K (Sec. 3.4), summed in long double: Ef [4(p_e+1)].
int orcx_face_E(void* h, const orc_params* P, int f, const double* U, const double* Lam, double* Ef) {
  OMesh* M = (OMesh*)h;
  if (f < 0 || f >= M->nf) return 2;
  const int len = face_len(*M, f);
  std::vector<real> Ur(M->u_len), Lr(M->lam_len), acc(len, 0.0L);
  for (int64_t i = 0; i < M->u_len; ++i) Ur[i] = U[i];
  for (int64_t i = 0; i < M->lam_len; ++i) Lr[i] = Lam[i];
  int st = 0;
  for (int sd = 0; sd < 2; ++sd) {
    const int K = sd ? M->face_el1[f] : M->face_el0[f];
    std::vector<real> x, s, e;
    st |= element_condense(*M, *P, K, Ur.data(), Lr.data(), x, s, e, nullptr, nullptr);
    int roff = 0;
    for (int a = 0; a < 3; ++a) {
      const int ea = M->elem_face[K * 3 + a];
      if (ea < 0) continue;
      if (ea == f)
        for (int r = 0; r < len; ++r) acc[r] += e[roff + r];
      roff += face_len(*M, ea);
    }
  }
  for (int r = 0; r < len; ++r) Ef[r] = (double)acc[r];
  return st;
}

// Number of significand bits of the build's scalar type (64 on x86-64, 113 on aarch64).
int orcx_mantissa_bits(void) { return std::numeric_limits<real>::digits; }
#endif  // ORC_EXTENDED
}  // extern "C"
