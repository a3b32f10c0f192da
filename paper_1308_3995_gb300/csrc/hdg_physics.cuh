// Physics of the HDG element kernels (paper Sec. 2): Euler convective flux and
// its Jacobians (binary64 or float-float), written once for both arithmetics.
#pragma once

#include "hdg_arith.cuh"

namespace hdg {

// --------------------------------------------------------------------------
// Euler physics (Sec. 2.1): flux f_c = (rho v, rho v (x) v + p Id, v (E + p)),
// p = (gamma - 1)(E - rho |v|^2 / 2), and the flux Jacobians dF_x/dw, dF_y/dw
// (row-major 4x4), derived by hand from those formulas.
// --------------------------------------------------------------------------
template <class T>
struct EulerConst {  // constants of the physics in the kernel's arithmetic
  T gam, g1, three_m_gam, half, one;
};

template <class T>
__device__ __forceinline__ void euler_flux_jac(const T* w, const EulerConst<T>& C, T* fx, T* fy, T* Ax, T* Ay) {
  using A = Ar<T>;
  const T rho = w[0], ir = A::rcp(rho), u = A::mul(w[1], ir), v = A::mul(w[2], ir), E = w[3];
  const T uu = A::mul(u, u), vv = A::mul(v, v), uv = A::mul(u, v);
  const T q2 = A::add(uu, vv);
  const T p = A::mul(C.g1, A::sub(E, A::mul(A::mul(C.half, rho), q2)));
  const T Ep = A::add(E, p);
  const T H = A::mul(Ep, ir);
  const T ph2 = A::mul(A::mul(C.half, C.g1), q2);
  const T z = A::zero();
  fx[0] = w[1]; fx[1] = A::add(A::mul(w[1], u), p); fx[2] = A::mul(w[1], v); fx[3] = A::mul(u, Ep);
  fy[0] = w[2]; fy[1] = A::mul(w[2], u); fy[2] = A::add(A::mul(w[2], v), p); fy[3] = A::mul(v, Ep);
  const T g1u = A::mul(C.g1, u), g1v = A::mul(C.g1, v), g1uv = A::mul(C.g1, uv);
  const T phH = A::sub(ph2, H);
  Ax[0] = z;                 Ax[1] = C.one;                      Ax[2] = z;                        Ax[3] = z;
  Ax[4] = A::sub(ph2, uu);   Ax[5] = A::mul(C.three_m_gam, u);   Ax[6] = A::neg(g1v);              Ax[7] = C.g1;
  Ax[8] = A::neg(uv);        Ax[9] = v;                          Ax[10] = u;                       Ax[11] = z;
  Ax[12] = A::mul(u, phH);   Ax[13] = A::sub(H, A::mul(g1u, u)); Ax[14] = A::neg(g1uv);            Ax[15] = A::mul(C.gam, u);
  Ay[0] = z;                 Ay[1] = z;                          Ay[2] = C.one;                    Ay[3] = z;
  Ay[4] = A::neg(uv);        Ay[5] = v;                          Ay[6] = u;                        Ay[7] = z;
  Ay[8] = A::sub(ph2, vv);   Ay[9] = A::neg(g1u);                Ay[10] = A::mul(C.three_m_gam, v); Ay[11] = C.g1;
  Ay[12] = A::mul(v, phH);   Ay[13] = A::neg(g1uv);              Ay[14] = A::sub(H, A::mul(g1v, v)); Ay[15] = A::mul(C.gam, v);
}


// --------------------------------------------------------------------------
// Navier-Stokes viscous flux (Sec. 2.2), non-dimensional with rho_inf = c_inf = 1:
//   T = gamma p / rho, mu = mu_inf (1+S) T^{3/2} / (T+S) (Sutherland), k = mu/((gamma-1) Pr),
//   tau = mu (grad v + grad v^T - 2/3 div v Id),  f_v = (0, tau, tau v + k grad T),
// with q = grad w of the conserved variables and grad v, grad T from q by the chain rule.
// f_v is linear in q: f_v(w, q) = M(w) q.  The code is written once over a
// generic number type N (plain T, or a forward-mode dual number over T).
// --------------------------------------------------------------------------
__device__ __forceinline__ double nadd(double a, double b) { return a + b; }
__device__ __forceinline__ double nsub(double a, double b) { return a - b; }
__device__ __forceinline__ double nmul(double a, double b) { return a * b; }
__device__ __forceinline__ double nscale(double a, double s) { return a * s; }
__device__ __forceinline__ double nrcp(double a) { return Ar<double>::rcp(a); }
__device__ __forceinline__ double nsqrt(double a) { return ar_sqrt(a); }
__device__ __forceinline__ double nlift(double a) { return a; }
__device__ __forceinline__ ff nadd(ff a, ff b) { return Ar<ff>::add(a, b); }
__device__ __forceinline__ ff nsub(ff a, ff b) { return Ar<ff>::sub(a, b); }
__device__ __forceinline__ ff nmul(ff a, ff b) { return Ar<ff>::mul(a, b); }
__device__ __forceinline__ ff nscale(ff a, ff s) { return Ar<ff>::mul(a, s); }
__device__ __forceinline__ ff nrcp(ff a) { return Ar<ff>::rcp(a); }
__device__ __forceinline__ ff nsqrt(ff a) { return ar_sqrt(a); }
__device__ __forceinline__ ff nlift(ff a) { return a; }
template <class T, int ND>
__device__ __forceinline__ Dual<T, ND> nadd(const Dual<T, ND>& a, const Dual<T, ND>& b) { return dadd(a, b); }
template <class T, int ND>
__device__ __forceinline__ Dual<T, ND> nsub(const Dual<T, ND>& a, const Dual<T, ND>& b) { return dsub(a, b); }
template <class T, int ND>
__device__ __forceinline__ Dual<T, ND> nmul(const Dual<T, ND>& a, const Dual<T, ND>& b) { return dmul(a, b); }
template <class T, int ND>
__device__ __forceinline__ Dual<T, ND> nscale(const Dual<T, ND>& a, T s) { return dscale(a, s); }
template <class T, int ND>
__device__ __forceinline__ Dual<T, ND> nrcp(const Dual<T, ND>& a) { return drcp(a); }
template <class T, int ND>
__device__ __forceinline__ Dual<T, ND> nsqrt(const Dual<T, ND>& a) { return dsqrt(a); }

template <class T>
struct NsConst {  // constants of the viscous flux in the kernel's arithmetic
  T half, g1, gam, two, twothirds, suth, mu_fac, kfac;
};

template <class N>
struct ViscCoef {  // w-dependent coefficients of the linear map q -> f_v
  N ir, u, v, hq2, pir, mu, kap;
};

template <class N, class T>
__device__ __forceinline__ void visc_coef(const N* w, const NsConst<T>& C, ViscCoef<N>& c) {
  c.ir = nrcp(w[0]);
  c.u = nmul(w[1], c.ir);
  c.v = nmul(w[2], c.ir);
  c.hq2 = nscale(nadd(nmul(c.u, c.u), nmul(c.v, c.v)), C.half);   // |v|^2 / 2
  const N p = nscale(nsub(w[3], nmul(w[0], c.hq2)), C.g1);        // (gamma-1)(E - rho |v|^2/2)
  c.pir = nmul(p, c.ir);                                          // p / rho
  const N Tt = nscale(c.pir, C.gam);                              // T = gamma p / rho
  const N t32 = nmul(Tt, nsqrt(Tt));
  N den = Tt;
  den.v = Ar<T>::add(den.v, C.suth);
  c.mu = nscale(nmul(t32, nrcp(den)), C.mu_fac);
  c.kap = nscale(c.mu, C.kfac);
}
// plain-number specialisation of the "+ S" in the Sutherland denominator
template <class T>
__device__ __forceinline__ void visc_coef_plain(const T* w, const NsConst<T>& C, ViscCoef<T>& c) {
  c.ir = nrcp(w[0]);
  c.u = nmul(w[1], c.ir);
  c.v = nmul(w[2], c.ir);
  c.hq2 = nscale(nadd(nmul(c.u, c.u), nmul(c.v, c.v)), C.half);
  const T p = nscale(nsub(w[3], nmul(w[0], c.hq2)), C.g1);
  c.pir = nmul(p, c.ir);
  const T Tt = nscale(c.pir, C.gam);
  const T t32 = nmul(Tt, nsqrt(Tt));
  c.mu = nscale(nmul(t32, nrcp(nadd(Tt, C.suth))), C.mu_fac);
  c.kap = nscale(c.mu, C.kfac);
}

// f_v[k][f] for the gradient q[k][f] (k = x, y)
template <class N, class T>
__device__ __forceinline__ void visc_flux(const ViscCoef<N>& c, const N (*q)[4], const NsConst<T>& C, N (*fv)[4]) {
  N du[2], dv[2], dT[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const N dr = q[k][0];
    du[k] = nmul(nsub(q[k][1], nmul(c.u, dr)), c.ir);
    dv[k] = nmul(nsub(q[k][2], nmul(c.v, dr)), c.ir);
    const N dp = nscale(nadd(nsub(q[k][3], nadd(nmul(c.u, q[k][1]), nmul(c.v, q[k][2]))), nmul(c.hq2, dr)), C.g1);
    dT[k] = nscale(nmul(nsub(dp, nmul(c.pir, dr)), c.ir), C.gam);
  }
  const N dv2 = nscale(nadd(du[0], dv[1]), C.twothirds);
  const N txx = nmul(c.mu, nsub(nscale(du[0], C.two), dv2));
  const N tyy = nmul(c.mu, nsub(nscale(dv[1], C.two), dv2));
  const N txy = nmul(c.mu, nadd(du[1], dv[0]));
  fv[0][1] = txx;
  fv[0][2] = txy;
  fv[0][3] = nadd(nadd(nmul(c.u, txx), nmul(c.v, txy)), nmul(c.kap, dT[0]));
  fv[1][1] = txy;
  fv[1][2] = tyy;
  fv[1][3] = nadd(nadd(nmul(c.u, txy), nmul(c.v, tyy)), nmul(c.kap, dT[1]));
  fv[0][0] = nsub(fv[0][1], fv[0][1]);  // zero of the right type
  fv[1][0] = fv[0][0];
}

// Viscous flux with its derivatives at one state: fv[k][f], dw[k][f][g] = d fv/d w_g,
// dq[k][f][k'*4+g] = d fv/d q_{k'g} (f = 1..3 rows; row 0 is identically zero).
template <class T>
__device__ __forceinline__ void visc_all(const T* w, const T (*q)[4], const NsConst<T>& C, T (*fv)[4],
                                         T (*dw)[4][4], T (*dq)[4][8]) {
  using D = Dual<T, 4>;
  D wd[4], qd[2][4], fd[2][4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    wd[g] = dconst<T, 4>(w[g]);
    wd[g].d[g] = Ar<T>::from_d(1.0);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int f = 0; f < 4; ++f) qd[k][f] = dconst<T, 4>(q[k][f]);
  ViscCoef<D> cd;
  visc_coef(wd, C, cd);
  visc_flux(cd, qd, C, fd);
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      fv[k][f] = fd[k][f].v;
#pragma unroll
      for (int g = 0; g < 4; ++g) dw[k][f][g] = fd[k][f].d[g];
    }
  // linear in q: the column for q_{k'g} is f_v at the unit gradient e_{k'g}
  ViscCoef<T> cp;
  cp.ir = cd.ir.v; cp.u = cd.u.v; cp.v = cd.v.v; cp.hq2 = cd.hq2.v; cp.pir = cd.pir.v; cp.mu = cd.mu.v;
  cp.kap = cd.kap.v;
  const T z = Ar<T>::zero(), one = Ar<T>::from_d(1.0);
#pragma unroll
  for (int kg = 0; kg < 8; ++kg) {
    T qe[2][4], fe[2][4];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int f = 0; f < 4; ++f) qe[k][f] = (k * 4 + f == kg) ? one : z;
    visc_flux(cp, qe, C, fe);
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int f = 0; f < 4; ++f) dq[k][f][kg] = fe[k][f];
  }
}

// Boundary state of Sec. 2.1 and its derivative d w_b / d w (forward mode, four
// directions), for kind 1 (slip wall: w_b = (rho, m - (m . n) n, E)) or 2 (far
// field, characteristic upwinding: w_b = w + sum over negative eigenvalues of
// r_j (l_j . (w_inf - w)), with r_j / l_j the right / left eigenvectors of
// f_c'(w) . n -- r: (1, u - c n, H - c v_n), (1, u, v, |v|^2/2), (0, t, v_t),
// (1, u + c n, H + c v_n), t = (-n_y, n_x); eigenvalues v_n - c, v_n, v_n,
// v_n + c; the left eigenvectors in closed form; the selection is taken at the
// current state and not differentiated).
// Not inlined: its forward-mode elimination needs many registers, and only
// boundary points call it, so it keeps its own frame instead of raising the
// register pressure of the element kernel around it.
template <class T>
__device__ __noinline__ void boundary_state_jac(int kind, const T* w, T nx, T ny, const T* winf,
                                                const EulerConst<T>& C, T* wb, T (*dwb)[4]) {
  using A = Ar<T>;
  using D = Dual<T, 4>;
  D wd[4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    wd[g] = dconst<T, 4>(w[g]);
    wd[g].d[g] = A::from_d(1.0);
  }
  D out[4];
  if (kind == 1) {
    const D mn = dadd(dscale(wd[1], nx), dscale(wd[2], ny));
    out[0] = wd[0];
    out[1] = dsub(wd[1], dscale(mn, nx));
    out[2] = dsub(wd[2], dscale(mn, ny));
    out[3] = wd[3];
  } else {
    const D ir = drcp(wd[0]);
    const D u = dmul(wd[1], ir), v = dmul(wd[2], ir);
    const D q2h = dscale(dadd(dmul(u, u), dmul(v, v)), C.half);
    const D p = dscale(dsub(wd[3], dmul(wd[0], q2h)), C.g1);
    const D c2 = dscale(dmul(p, ir), C.gam);
    const D c = dsqrt(c2), ic = drcp(c);
    const D H = dmul(dadd(wd[3], p), ir);
    const D vn = dadd(dscale(u, nx), dscale(v, ny));
    const D vt = dsub(dscale(v, nx), dscale(u, ny));
    // left eigenvectors (rows of Q^{-1}) in closed form: b1 = (gamma-1)/c^2, b2 = b1 |v|^2/2
    const D b1 = dscale(drcp(c2), C.g1), b2 = dmul(b1, q2h);
    const T lam0 = A::sub(vn.v, c.v), lam1 = vn.v, lam3 = A::add(vn.v, c.v);
    D dw[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) dw[f] = dsub(dconst<T, 4>(winf[f]), wd[f]);   // w_inf - w
#pragma unroll
    for (int f = 0; f < 4; ++f) out[f] = wd[f];
    const D bu = dmul(b1, u), bv = dmul(b1, v), vnc = dmul(vn, ic);
    const D nxc = dscale(ic, nx), nyc = dscale(ic, ny);
    if (A::to_d(lam0) < 0.0) {  // eigenvalue v_n - c: l = (b2 + v_n/c, -b1 u - n_x/c, -b1 v - n_y/c, b1) / 2
      D y = dmul(dadd(b2, vnc), dw[0]);
      y = dsub(y, dmul(dadd(bu, nxc), dw[1]));
      y = dsub(y, dmul(dadd(bv, nyc), dw[2]));
      y = dscale(dadd(y, dmul(b1, dw[3])), C.half);
      const D cn = dscale(c, nx), cm = dscale(c, ny);
      out[0] = dadd(out[0], y);
      out[1] = dadd(out[1], dmul(dsub(u, cn), y));
      out[2] = dadd(out[2], dmul(dsub(v, cm), y));
      out[3] = dadd(out[3], dmul(dsub(H, dmul(c, vn)), y));
    }
    if (A::to_d(lam1) < 0.0) {  // eigenvalue v_n (twice): l2 = (1 - b2, b1 u, b1 v, -b1), l3 = (-v_t, -n_y, n_x, 0)
      D y2 = dmul(dsub(dconst<T, 4>(C.one), b2), dw[0]);
      y2 = dadd(y2, dmul(bu, dw[1]));
      y2 = dadd(y2, dmul(bv, dw[2]));
      y2 = dsub(y2, dmul(b1, dw[3]));
      D y3 = dmul(vt, dw[0]);
      y3 = dsub(dsub(dscale(dw[2], nx), dscale(dw[1], ny)), y3);
      out[0] = dadd(out[0], y2);
      out[1] = dadd(out[1], dsub(dmul(u, y2), dscale(y3, ny)));
      out[2] = dadd(out[2], dadd(dmul(v, y2), dscale(y3, nx)));
      out[3] = dadd(out[3], dadd(dmul(q2h, y2), dmul(vt, y3)));
    }
    if (A::to_d(lam3) < 0.0) {  // eigenvalue v_n + c: l = (b2 - v_n/c, -b1 u + n_x/c, -b1 v + n_y/c, b1) / 2
      D y = dmul(dsub(b2, vnc), dw[0]);
      y = dadd(y, dmul(dsub(nxc, bu), dw[1]));
      y = dadd(y, dmul(dsub(nyc, bv), dw[2]));
      y = dscale(dadd(y, dmul(b1, dw[3])), C.half);
      const D cn = dscale(c, nx), cm = dscale(c, ny);
      out[0] = dadd(out[0], y);
      out[1] = dadd(out[1], dmul(dadd(u, cn), y));
      out[2] = dadd(out[2], dmul(dadd(v, cm), y));
      out[3] = dadd(out[3], dmul(dadd(H, dmul(c, vn)), y));
    }
  }
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    wb[f] = out[f].v;
#pragma unroll
    for (int g = 0; g < 4; ++g) dwb[f][g] = out[f].d[g];
  }
}

}  // namespace hdg
