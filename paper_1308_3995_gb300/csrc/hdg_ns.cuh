// Navier-Stokes mixed-form element kernel (12 fields: q_x, q_y, w; paper
// Eq. strmixed and Eqs. hdg_ls1-hdg_cont with the viscous numerical flux of
// Sec. 3.2).  Same outputs as the Euler kernel: X = A^{-1}[B | F] over the
// element's [Q; W] unknowns, S = D - C X_B, E = H - C X_F, the residuals, and
// the assembly into the trace system.
//
// Structure exploited (exact in exact arithmetic, so the outputs are the same
// linear-algebra objects the oracle forms densely):
//   * dN_q/dQ = (phi_i, phi_j)_K = det J * I for the orthonormal basis on an
//     affine element, so the q unknowns are eliminated first (block Gaussian
//     elimination with the pivot block det J * I):
//       A' = A_ww - A_wq A_qw / det,  R'_w = R_w - A_wq R_q / det,
//       A' X_w = R'_w (LU with partial pivoting, 4 n_p unknowns),
//       X_q = (R_q - A_qw X_w) / det,
//       S = D - C_q B_q / det - (C_w - C_q A_qw / det) X_w,B,
//       E = H - C_q F_q / det - (C_w - C_q A_qw / det) X_w,F;
//   * A_qw = (d_k phi_i, phi_j) delta_fg, B_q = -<phi_i n_k, psi_l> delta_fg and
//     C_w = alpha <psi_l, phi_j> delta_fg come from reference tables;
//   * A_wq and C_q are produced one (direction k', field g) block column at a
//     time and consumed at once, so they are never stored whole.
// Adjoint mode (Sec. 4.2, ph.adjoint): X~ = A^{-T} [C^T | F~] by the same
// elimination transposed: A'^T X~_w = G_w - A_qw^T G_q / det (G = [C^T | F~],
// A' the Schur matrix above), then X~_q = (G_q - A_wq^T X~_w) / det with the
// block columns of A_wq and C_q produced a second time after the LU.
// No-slip adiabatic walls (Sec. 2.2, boundary operator of Sec. 3.2): a wall
// face has no trace unknowns; its flux is (f_c(w_b) - f_v(w_b, q)) . n with
// w_b = (rho, 0, 0, E) and the energy row of f_v zero, and the gradient
// equations see -<tau.n, w_b>, so A_qw of the fields rho and E gains
// -n_k |e| <phi_i, phi_j>_e (D_k^wall below) and A_ww gains the wall flux's
// Jacobian in its columns rho and E.
// Characteristic far field (Sec. 2.1, viscous flux at the far-field state):
// w_b(w) by characteristic upwinding against the free stream, the flux
// (f_c(w_b) - f_v(w_b, q)) . n whole, its Jacobian (d f / d w_b)(d w_b / d w)
// in all four columns of A_ww; the gradient equations see -<tau.n, w_b(w)>, so
// A_qw gains -n_k sum_x phi_i(x) (we d w_b / d w)_fg(x) phi_j(x) over the edge
// points x, which couples the fields: its products in the q elimination, in
// C', in X_q and in the adjoint's transposed elimination run through the
// values at those points (a low-rank update of the field-diagonal blocks).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <type_traits>

#include "hdg_arith.cuh"
#include "hdg_internal.h"
#include "hdg_lu.cuh"
#include "hdg_physics.cuh"

namespace hdg {

// threads per element CTA: 128 for p = 1, so that four CTAs (four elements)
// share an SM within the register file (uniform p = 1: 2.67 -> 3.85 M elements/s
// in binary64, 2.48 -> 4.25 M in float-float, against two CTAs of 256); 256 for
// p = 2 (the smaller CTA measured no better in binary64 and worse in
// float-float, its shared memory allowing only two per SM on mixed meshes);
// 512 for p >= 3, one CTA per SM
// One far-field edge point of the Navier-Stokes kernel (Sec. 2.1): w_b(w) by
// characteristic upwinding against the free stream and d w_b / d w, the flux
// (f_c(w_b) - f_v(w_b, q)) . n whole (we times it into fhat[4]), d fhat / d w =
// (d f / d w_b)(d w_b / d w) (al[16]), -n . d f_v / d q at w_b (aq[24], rows
// 1..3), and for the gradient equations we w_b and we d w_b / d w (fb[20]).
// Not inlined: only far-field points call it, so its registers stay out of
// the element kernel's allocation.
template <class T>
__device__ __noinline__ void ns_farfield_point(const T* w, const T (*qv)[4], T nx, T ny, T we, const double* winf_d,
                                               const EulerConst<T>& C, const NsConst<T>& V, T* fhat, T* al, T* aq,
                                               T* fb) {
  using A = Ar<T>;
  const T zero = A::zero();
  T winf[4], wb[4], dwb[4][4], fx[4], fy[4], Ax[16], Ay[16], fv[2][4], dw[2][4][4], dq[2][4][8], q2[2][4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    winf[f] = A::from_d(winf_d[f]);
    q2[0][f] = qv[0][f];
    q2[1][f] = qv[1][f];
  }
  boundary_state_jac(2, w, nx, ny, winf, C, wb, dwb);
  euler_flux_jac(wb, C, fx, fy, Ax, Ay);
  visc_all(wb, q2, V, fv, dw, dq);
#pragma unroll
  for (int f = 0; f < 4; ++f)
    fhat[f] = A::mul(we, A::add(A::mul(nx, A::sub(fx[f], fv[0][f])), A::mul(ny, A::sub(fy[f], fv[1][f]))));
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    T an[4];
#pragma unroll
    for (int g = 0; g < 4; ++g)
      an[g] = A::add(A::mul(nx, A::sub(Ax[f * 4 + g], dw[0][f][g])), A::mul(ny, A::sub(Ay[f * 4 + g], dw[1][f][g])));
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      T v = zero;
#pragma unroll
      for (int h = 0; h < 4; ++h) A::madd(v, an[h], dwb[h][g]);
      al[f * 4 + g] = A::mul(we, A::norm(v));
    }
  }
#pragma unroll
  for (int f = 1; f < 4; ++f)
#pragma unroll
    for (int kg = 0; kg < 8; ++kg)
      aq[(f - 1) * 8 + kg] = A::neg(A::mul(we, A::add(A::mul(nx, dq[0][f][kg]), A::mul(ny, dq[1][f][kg]))));
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    fb[f] = A::mul(we, wb[f]);
#pragma unroll
    for (int g = 0; g < 4; ++g) fb[4 + f * 4 + g] = A::mul(we, dwb[f][g]);
  }
}

template <int P>
constexpr int ns_threads() { return P == 1 ? 128 : (P >= 3 ? 512 : 256); }
constexpr int kNsPt = 6;   // edge point slots per face

template <int P>
struct NsLayout {
  static constexpr int NP = n_basis(P), NQ = (P + 2) * (P + 2), NW4 = 4 * NP, N = 12 * NP, LDA = NW4 + 1;
  int ldr, lds, ldc;
  int oA, oR, oCp, oS, oU, oNu, oL, oNl, oE, oDk, oPv, oPf, oW, oZ, oBc, oCc, oFb, oYf, nyf, total;
  HDG_HD NsLayout(int ntmax) {
    ldr = (ntmax + 1) | 1;
    lds = (ntmax + 1) | 1;
    ldc = (NW4 + 1) | 1;
    oA = 0;
    oR = oA + NW4 * LDA;
    oCp = oR + NW4 * ldr;
    oS = oCp + ntmax * ldc;
    oU = oS + ntmax * lds;
    oNu = oU + N;
    oL = oNu + N;
    oNl = oL + kMaxNt;
    oE = oNl + kMaxNt;
    oDk = oE + kMaxNt;
    oPv = oDk + 2 * NP * NP;
    oPf = oPv + NQ * (12 + 8 + 24 + 48);   // point values (12) + Fh (8) + Aww (24) + Awq (48)
    oW = oPf + 3 * kNsPt * (4 + 16 + 24);
    oZ = oW + 3 * kNsPt * 16 * 5;
    oBc = oZ + 4 * NP * NQ;
    oCc = oBc + NW4 * NP;
    oFb = oCc + ntmax * NP;
    oYf = oFb + 3 * kNsPt * 20;   // far-field point data: weighted w_b (4) and weighted d w_b / d w (16)
    nyf = (NW4 > ntmax + 1 ? NW4 : ntmax + 1) * 3 * kNsPt;  // values at the far-field points of rows or columns
    total = oYf + nyf;
  }
};

// Two CTAs per SM for p <= 2 (registers capped at 128, a few hundred bytes of
// spills in the pointwise Jacobians): at one CTA of 8 warps per SM those
// buckets stall on block barriers with the binary64 pipe 40-55 % busy; the
// second CTA hides them (Navier-Stokes p mix: 101.7 -> 86.0 ms per step in
// binary64, 76.3 -> 70.5 ms in float-float).  For p >= 3 shared memory allows
// one CTA per SM anyway; there the CTA has 16 warps (registers capped at 128
// the same way), which hide more of the latency inside each phase than 8 warps
// with 248-254 registers (p mix: 84.1 -> 82.9 ms binary64, 77.2 -> 75.5 ms
// float-float).
// BATCH: the launch walks the work list `bt` over the elements of several
// systems (hdg_batch_condense); otherwise m_, s_, ph_, U_, Lam_ and elems.
// FAR: the far-field boundary code is compiled in (meshes with far-field
// faces, and every batch); without it the kernel is the one of periodic and
// wall-bounded meshes, with none of that code's registers.
template <int P, class T, bool ADJ, bool BATCH = false, bool FAR = BATCH>
__global__ void __launch_bounds__(ns_threads<P>(), (P == 1 ? 4 : (P == 2 ? 2 : 1))) k_condense_ns(DevMesh m_, DevSys s_, Phys ph_, const T* __restrict__ tab,
                                                             TabOff to, const double* __restrict__ U_,
                                                             const double* __restrict__ Lam_,
                                                             const int* __restrict__ elems, int n_elems, int ntmax,
                                                             BatchRef bt) {
  using L = NsLayout<P>;
  using A = Ar<T>;
  constexpr int NP = L::NP, NQ = L::NQ, NW4 = L::NW4, N = L::N, LDA = L::LDA;
  constexpr int NT = ns_threads<P>(), NW = NT / 32;
  extern __shared__ double smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const L lay(ntmax);
  const int ldr = lay.ldr, lds = lay.lds, ldc = lay.ldc;
  T* sA = smem + lay.oA;     // A' (4 n_p x 4 n_p)
  T* sR = smem + lay.oR;     // R'_w = [B_w | F_w] - A_wq R_q / det, then X_w
  T* sCp = smem + lay.oCp;   // C' = C_w - C_q A_qw / det  (nt x 4 n_p)
  T* sS = smem + lay.oS;     // S0 = D - C_q B_q / det, then S  (nt x nt)
  T* sU = smem + lay.oU;     // element coefficients [Q; W]
  T* sNu = smem + lay.oNu;   // interior residual [N_q; N_w]
  T* sL = smem + lay.oL;     // traces of the three faces
  T* sNl = smem + lay.oNl;   // this element's share of the trace residual
  T* sE = smem + lay.oE;     // E0 = H - C_q F_q / det, then E
  T* sDk = smem + lay.oDk;   // D_k[i][j] = (d_k phi_i, phi_j)_K, k = x, y
  T* sPv = smem + lay.oPv;   // volume point data
  T* sVal = sPv;             // [12][NQ] w and q at the points (fields q_x(4), q_y(4), w(4))
  T* sFh = sVal + 12 * NQ;   // [2][4][NQ]   contravariant (f_c - f_v), weighted
  T* sAww = sFh + 8 * NQ;    // [2][12][NQ]  contravariant d(f_c - f_v)/dw, rows 1..3
  T* sAwq = sAww + 24 * NQ;  // [2][24][NQ]  contravariant d f_v/dq, rows 1..3
  T* sPf = smem + lay.oPf;   // face point data per slot t = a*6 + g
  T* sFhat = sPf;            // [18][4]  weighted numerical flux
  T* sAl = sFhat + 18 * 4;   // [18][16] weighted d f_hat/d lambda
  T* sAq = sAl + 18 * 16;    // [18][24] weighted d f_hat/d q, rows 1..3
  T* sW = smem + lay.oW;     // [18][16][5] sAl * psi_l
  T* sZ = smem + lay.oZ;     // [4][NP][NQ]
  T* sBc = smem + lay.oBc;   // A_wq block column [4 n_p][n_p]
  T* sCc = smem + lay.oCc;   // C_q block column [nt][n_p]
  T* sFb = smem + lay.oFb;   // [18][20] far-field points: we w_b (4), we d w_b / d w (16)
  T* sYf = smem + lay.oYf;   // [rows or columns][far-field points] products with phi at those points

  __shared__ T g_det, g_ic, g_Ji[2][2], g_n[3][2], g_len[3], g_mt;
  __shared__ int g_e[3], g_pe[3], g_nk[3], g_toff[4], g_fl[3], g_side[3], g_old[3], g_bc[3], g_wall, g_bnd, g_nff;
  __shared__ unsigned char g_ffa[3 * kNsPt], g_ffq[3 * kNsPt];  // far-field point x: face, point
  __shared__ unsigned char g_cf[kMaxNt], g_cg[kMaxNt], g_cl[kMaxNt];
  __shared__ T s_pinv[64];
  __shared__ int s_bad;

  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const T* vw = tab + to.vol_w[P];
  const T* vphi = tab + to.vol_phi[P];
  const T* vgx = tab + to.vol_gxi[P];
  const T* vge = tab + to.vol_geta[P];
  const T* dref = tab + to.vol_dref[P];
  const T zero = A::zero();

  int seg = 0;
  for (int it = blockIdx.x; it < n_elems; it += gridDim.x) {
    const ReqDesc* D = nullptr;
    int K;
    if constexpr (BATCH) K = batch_item(bt, it, seg, D);
    else K = elems[it];
    const DevMesh& m = pick_ref<BATCH>(D, &ReqDesc::m, m_);
    const DevSys& s = pick_ref<BATCH>(D, &ReqDesc::s, s_);
    const Phys& ph = pick_ref<BATCH>(D, &ReqDesc::ph, ph_);
    const double* __restrict__ U = BATCH ? D->U : U_;
    const double* __restrict__ Lam = BATCH ? D->Lam : Lam_;
    EulerConst<T> C;
    C.gam = A::from_d(ph.gamma);
    C.g1 = A::from_d(ph.gamma - 1.0);
    C.three_m_gam = A::from_d(3.0 - ph.gamma);
    C.half = A::from_d(0.5);
    C.one = A::from_d(1.0);
    NsConst<T> V;
    V.half = C.half;
    V.g1 = C.g1;
    V.gam = C.gam;
    V.two = A::from_d(2.0);
    V.twothirds = A::from_d(2.0 / 3.0);
    V.suth = A::from_d(ph.suth_s);
    V.mu_fac = A::from_d(ph.mu_inf * (1.0 + ph.suth_s));
    V.kfac = A::from_d(1.0 / ((ph.gamma - 1.0) * ph.prandtl));
    const T alpha = A::from_d(ph.alpha);
    // ---------------- a1: geometry, faces, state ----------------
    if (tid < 3) {
      const double* c = m.xy + 6 * (size_t)K;
      const int a = tid, b = (tid + 1) % 3;
      const double dx = c[2 * b] - c[2 * a], dy = c[2 * b + 1] - c[2 * a + 1];
      const double len = sqrt(dx * dx + dy * dy);
      const double il = __drcp_rn(len);
      g_len[a] = A::from_d(len);
      g_n[a][0] = A::from_d(dy * il);
      g_n[a][1] = A::from_d(-dx * il);
      const int e = m.elem_face[3 * (size_t)K + a];
      const int info = m.elem_info[K];
      g_e[a] = e;
      g_pe[a] = e >= 0 ? m.face_p[e] : P;  // a wall face: the element's own edge rule,
      g_nk[a] = e >= 0 ? g_pe[a] + 1 : 0;   // and no trace unknowns
      g_fl[a] = (info >> a) & 1;
      g_side[a] = (info >> (3 + a)) & 1;
      g_bc[a] = e >= 0 ? 0 : (m.elem_bc ? (m.elem_bc[K] >> (2 * a)) & 3 : 3);  // boundary: 2 far field, 3 wall
      if (tid == 0) {
        const double J00 = c[2] - c[0], J01 = c[4] - c[0], J10 = c[3] - c[1], J11 = c[5] - c[1];
        const double det = J00 * J11 - J01 * J10;
        const double inv = __drcp_rn(det);
        g_det = A::from_d(det);
        g_ic = A::from_d(inv);
        g_Ji[0][0] = A::from_d(J11 * inv); g_Ji[0][1] = A::from_d(-J01 * inv);
        g_Ji[1][0] = A::from_d(-J10 * inv); g_Ji[1][1] = A::from_d(J00 * inv);
        double mt = 0.0;
        if (ph.cfl > 0.0) {  // pseudo-time mass det(J)/dt_K (Sec. 3.3), element-mean state
          const double* u0 = U + m.u_off[K] + 8 * NP;
          const double c0 = 1.4142135623730951;  // value of the constant orthonormal mode
          const double rho = c0 * u0[0], uu = c0 * u0[NP] / rho, vv = c0 * u0[2 * NP] / rho;
          const double E = c0 * u0[3 * NP];
          const double p = (ph.gamma - 1.0) * (E - 0.5 * rho * (uu * uu + vv * vv));
          double perim = 0.0;
          for (int l = 0; l < 3; ++l) {
            const int l2 = (l + 1) % 3;
            const double ex = c[2 * l2] - c[2 * l], ey = c[2 * l2 + 1] - c[2 * l + 1];
            perim += sqrt(ex * ex + ey * ey);
          }
          const double Tt = ph.gamma * p / rho;
          const double mu = ph.mu_inf * Tt * sqrt(Tt) * (1.0 + ph.suth_s) / (Tt + ph.suth_s);
          const double lam_c = (sqrt(uu * uu + vv * vv) + sqrt(ph.gamma * p / rho)) * perim;
          const double lam_v = ph.gamma * mu / (ph.prandtl * rho) * perim * perim / (0.5 * det);
          const double dt = ph.cfl * 0.5 * det / (lam_c + 4.0 * lam_v);
          mt = det / dt;
        }
        g_mt = A::from_d(mt);
        s_bad = 0;
      }
    }
    __syncthreads();
    if (tid == 0) {
      g_toff[0] = 0;
      g_toff[1] = 4 * g_nk[0];
      g_toff[2] = 4 * (g_nk[0] + g_nk[1]);
      g_toff[3] = 4 * (g_nk[0] + g_nk[1] + g_nk[2]);
      g_wall = (g_bc[0] == 3) || (g_bc[1] == 3) || (g_bc[2] == 3);
      g_bnd = (g_e[0] < 0) || (g_e[1] < 0) || (g_e[2] < 0);
      int nff = 0;
      for (int a = 0; FAR && a < 3; ++a)
        if (g_bc[a] == 2)
          for (int q = 0; q < P + 2; ++q) {
            g_ffa[nff] = (unsigned char)a;
            g_ffq[nff] = (unsigned char)q;
            ++nff;
          }
      g_nff = nff;
    }
    {
      const double* uk = U + m.u_off[K];
      for (int t = tid; t < N; t += NT) sU[t] = A::from_d(uk[t]);
    }
    // D_k = det * sum_r Ji[r][k] Dref_r
    for (int t = tid; t < NP * NP; t += NT) {
      const T d0 = dref[t], d1 = dref[NP * NP + t];
      sDk[t] = A::mul(g_det, A::add(A::mul(g_Ji[0][0], d0), A::mul(g_Ji[1][0], d1)));
      sDk[NP * NP + t] = A::mul(g_det, A::add(A::mul(g_Ji[0][1], d0), A::mul(g_Ji[1][1], d1)));
    }
    __syncthreads();
    const int nt = g_toff[3], nr1 = nt + 1;
    for (int c = tid; c < nt; c += NT) {
      const int a = (c >= g_toff[2]) ? 2 : (c >= g_toff[1] ? 1 : 0);
      const int nk = g_nk[a], cl = c - g_toff[a], g = cl / nk;
      g_cf[c] = (unsigned char)a;
      g_cg[c] = (unsigned char)g;
      g_cl[c] = (unsigned char)(cl - g * nk);
    }
    for (int a = 0; a < 3; ++a) {
      if (g_e[a] < 0) continue;  // wall face
      const double* lk = Lam + m.lam_off[g_e[a]];
      for (int t = tid; t < 4 * g_nk[a]; t += NT) sL[g_toff[a] + t] = A::from_d(lk[t]);
    }
    // values of q (fields 0..7) and w (8..11) at the volume points
    for (int t = tid; t < 12 * NQ; t += NT) {
      const int f = t / NQ, q = t - f * NQ;
      T acc = zero;
#pragma unroll
      for (int j = 0; j < NP; ++j) A::madd(acc, sU[f * NP + j], vphi[q * NP + j]);
      sVal[t] = A::norm(acc);
    }
    __syncthreads();

    // ---------------- a2: pointwise fluxes and Jacobians at the volume points ----------------
    for (int q = tid; q < NQ; q += NT) {
      T w[4], qv[2][4], fx[4], fy[4], Ax[16], Ay[16], fv[2][4], dw[2][4][4], dq[2][4][8];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        w[f] = sVal[(8 + f) * NQ + q];
        qv[0][f] = sVal[f * NQ + q];
        qv[1][f] = sVal[(4 + f) * NQ + q];
      }
      euler_flux_jac(w, C, fx, fy, Ax, Ay);
      visc_all(w, qv, V, fv, dw, dq);
      const T c = A::mul(vw[q], g_det);
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const T a0 = A::mul(c, g_Ji[r][0]), a1 = A::mul(c, g_Ji[r][1]);
#pragma unroll
        for (int f = 0; f < 4; ++f)
          sFh[(r * 4 + f) * NQ + q] = A::add(A::mul(a0, A::sub(fx[f], fv[0][f])), A::mul(a1, A::sub(fy[f], fv[1][f])));
#pragma unroll
        for (int f = 1; f < 4; ++f)
#pragma unroll
          for (int g = 0; g < 4; ++g)
            sAww[(r * 12 + (f - 1) * 4 + g) * NQ + q] =
                A::add(A::mul(a0, A::sub(Ax[f * 4 + g], dw[0][f][g])), A::mul(a1, A::sub(Ay[f * 4 + g], dw[1][f][g])));
#pragma unroll
        for (int f = 1; f < 4; ++f)
#pragma unroll
          for (int kg = 0; kg < 8; ++kg)
            sAwq[(r * 24 + (f - 1) * 8 + kg) * NQ + q] = A::add(A::mul(a0, dq[0][f][kg]), A::mul(a1, dq[1][f][kg]));
      }
    }
    // ---------------- a3: pointwise data at the face points ----------------
    // (on warps 2 and 3, while warps 0 and 1 work on the volume points above: NQ <= 64)
    static_assert(NQ <= 64 && 64 + 3 * kNsPt <= NT, "volume and face point threads must not overlap");
    for (int t = tid - 64; t >= 0 && t < 3 * kNsPt; t += NT) {
      const int a = t / kNsPt, g = t - a * kNsPt;
      const int pe = g_pe[a], nk = pe + 1;
      if (g < pe + 2) {
        const T* phe = tab + to.edge_phi[P][pe][a][g_fl[a]] + g * NP;
        const T* ps = tab + to.edge_psi[pe] + g * nk;
        const T we = A::mul(tab[to.edge_w[pe] + g], g_len[a]);
        T w[4], lam[4], qv[2][4], fx[4], fy[4], Ax[16], Ay[16], fv[2][4], dw[2][4][4], dq[2][4][8];
#pragma unroll
        for (int f = 0; f < 12; ++f) {
          T acc = zero;
#pragma unroll
          for (int j = 0; j < NP; ++j) A::madd(acc, sU[f * NP + j], phe[j]);
          acc = A::norm(acc);
          if (f < 4) qv[0][f] = acc; else if (f < 8) qv[1][f - 4] = acc; else w[f - 8] = acc;
        }
        const T nx = g_n[a][0], ny = g_n[a][1];
        if (FAR && g_e[a] < 0 && g_bc[a] == 2) {
          // characteristic far field (Sec. 2.1): its own frame (see ns_farfield_point)
          ns_farfield_point(w, qv, nx, ny, we, ph.winf, C, V, sFhat + t * 4, sAl + t * 16, sAq + t * 24, sFb + t * 20);
          continue;
        }
        if (g_e[a] < 0) {
          // no-slip adiabatic wall: w_b = (rho, 0, 0, E), f_v(w_b, q) with its energy row zero
          const T wb[4] = {w[0], zero, zero, w[3]};
          euler_flux_jac(wb, C, fx, fy, Ax, Ay);
          visc_all(wb, qv, V, fv, dw, dq);
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            fv[k][3] = zero;
#pragma unroll
            for (int g2 = 0; g2 < 4; ++g2) dw[k][3][g2] = zero;
#pragma unroll
            for (int kg = 0; kg < 8; ++kg) dq[k][3][kg] = zero;
          }
#pragma unroll
          for (int f = 0; f < 4; ++f)
            sFhat[t * 4 + f] = A::mul(we, A::add(A::mul(nx, A::sub(fx[f], fv[0][f])), A::mul(ny, A::sub(fy[f], fv[1][f]))));
          // d f_hat / d w = (d f / d w_b) diag(1, 0, 0, 1): columns rho and E (slot of d f_hat / d lambda)
#pragma unroll
          for (int f = 0; f < 4; ++f)
#pragma unroll
            for (int g2 = 0; g2 < 4; ++g2) {
              const T an = A::add(A::mul(nx, A::sub(Ax[f * 4 + g2], dw[0][f][g2])), A::mul(ny, A::sub(Ay[f * 4 + g2], dw[1][f][g2])));
              sAl[t * 16 + f * 4 + g2] = (g2 == 0 || g2 == 3) ? A::mul(we, an) : zero;
            }
#pragma unroll
          for (int f = 1; f < 4; ++f)
#pragma unroll
            for (int kg = 0; kg < 8; ++kg)
              sAq[t * 24 + (f - 1) * 8 + kg] = A::neg(A::mul(we, A::add(A::mul(nx, dq[0][f][kg]), A::mul(ny, dq[1][f][kg]))));
          continue;
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          T al = zero;
          for (int k = 0; k < nk; ++k) A::madd(al, sL[g_toff[a] + f * nk + k], ps[k]);
          lam[f] = A::norm(al);
        }
        euler_flux_jac(lam, C, fx, fy, Ax, Ay);
        visc_all(lam, qv, V, fv, dw, dq);  // f_v(lambda, q_K) and its derivatives
#pragma unroll
        for (int f = 0; f < 4; ++f)
          sFhat[t * 4 + f] = A::mul(we, A::sub(A::add(A::mul(nx, A::sub(fx[f], fv[0][f])), A::mul(ny, A::sub(fy[f], fv[1][f]))),
                                               A::mul(alpha, A::sub(lam[f], w[f]))));
#pragma unroll
        for (int f = 0; f < 4; ++f)
#pragma unroll
          for (int g2 = 0; g2 < 4; ++g2) {
            T an = A::add(A::mul(nx, A::sub(Ax[f * 4 + g2], dw[0][f][g2])), A::mul(ny, A::sub(Ay[f * 4 + g2], dw[1][f][g2])));
            if (f == g2) an = A::sub(an, alpha);
            const T at = A::mul(we, an);
            sAl[t * 16 + f * 4 + g2] = at;
            for (int l = 0; l < nk; ++l) sW[(t * 16 + f * 4 + g2) * 5 + l] = A::mul(at, ps[l]);
          }
#pragma unroll
        for (int f = 1; f < 4; ++f)
#pragma unroll
          for (int kg = 0; kg < 8; ++kg)
            sAq[t * 24 + (f - 1) * 8 + kg] = A::neg(A::mul(we, A::add(A::mul(nx, dq[0][f][kg]), A::mul(ny, dq[1][f][kg]))));
      }
    }
    __syncthreads();
    // shock-capturing viscosity (Sec. 3.2) with q in place of grad w, held fixed in the Jacobian:
    //   eps_K = eps_0 (h_K/p)^(2-beta) / |K| int_K sum_f |(A_x q_x + A_y q_y)_f|
    T eps = zero;
    const bool shock = ph.sc_eps0 > 0.0;
    if (shock) {
      for (int q = tid; q < NQ; q += NT) {
        T w[4], fx[4], fy[4], Ax[16], Ay[16];
#pragma unroll
        for (int f = 0; f < 4; ++f) w[f] = sVal[(8 + f) * NQ + q];
        euler_flux_jac(w, C, fx, fy, Ax, Ay);
        T d = zero;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          T v = zero;
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            A::madd(v, Ax[f * 4 + g], sVal[g * NQ + q]);
            A::madd(v, Ay[f * 4 + g], sVal[(4 + g) * NQ + q]);
          }
          d = A::add(d, A::abs(A::norm(v)));
        }
        sNl[q] = A::mul(A::mul(vw[q], g_det), d);  // sNl is free until the residuals
      }
      __syncthreads();
      T sum = zero;
      for (int q = 0; q < NQ; ++q) sum = A::add(sum, sNl[q]);
      const double l0 = A::to_d(g_len[0]), l1 = A::to_d(g_len[1]), l2 = A::to_d(g_len[2]);
      const double hk = fmax(l0, fmax(l1, l2)) / P;
      const double fac = ph.sc_eps0 * pow(hk, 2.0 - ph.sc_beta) * 2.0 / A::to_d(g_det);  // 1/|K| = 2/det J
      eps = A::mul(sum, A::from_d(fac));
      __syncthreads();
    }

    // ---------------- residuals ----------------
    // N_q[(k,f),i] = det Q[(k,f),i] + sum_j D_k[i][j] W[f][j] - sum_a n_k |e_a| sum_l Me_a[l][i] Lam_a[f][l]
    for (int t = tid; t < 8 * NP; t += NT) {
      const int kf = t / NP, i = t - kf * NP, k = kf >> 2, f = kf & 3;
      T acc = zero;
      A::madd(acc, g_det, sU[t]);
      for (int j = 0; j < NP; ++j) A::madd(acc, sDk[k * NP * NP + i * NP + j], sU[(8 + f) * NP + j]);
      for (int a = 0; a < 3; ++a) {
        const T sc = A::mul(g_n[a][k], g_len[a]);
        if (FAR && g_bc[a] == 2) {  // far field: -n_k <phi_i, w_b,f(w)>_e at the edge points
          const T* phe = tab + to.edge_phi[P][P][a][g_fl[a]];
          T s2 = zero;
          for (int q = 0; q < P + 2; ++q) A::madd(s2, phe[q * NP + i], sFb[(a * kNsPt + q) * 20 + f]);
          A::msub(acc, g_n[a][k], A::norm(s2));
          continue;
        }
        if (g_e[a] < 0) {  // wall: -n_k <phi_i, w_b,f>_e, w_b = (rho, 0, 0, E)
          if (f == 0 || f == 3) {
            const T* fm = tab + to.face_mass[P][P][a];
            T s2 = zero;
            for (int j = 0; j < NP; ++j) A::madd(s2, fm[i * NP + j], sU[(8 + f) * NP + j]);
            A::msub(acc, sc, A::norm(s2));
          }
          continue;
        }
        const int nk = g_nk[a];
        const T* me = tab + to.edge_cross[P][g_pe[a]][a][g_fl[a]];
        T s2 = zero;
        for (int l = 0; l < nk; ++l) A::madd(s2, me[l * NP + i], sL[g_toff[a] + f * nk + l]);
        A::msub(acc, sc, A::norm(s2));
      }
      sNu[t] = A::norm(acc);
    }
    // N_w = -(grad phi, f_c - f_v)_K + <phi, f_hat>_dK
    for (int t = tid; t < NW4; t += NT) {
      const int f = t / NP, i = t - f * NP;
      T acc0 = zero, acc1 = zero;
      for (int q = 0; q < NQ; ++q) {
        A::msub(acc0, vgx[q * NP + i], sFh[f * NQ + q]);
        A::msub(acc1, vge[q * NP + i], sFh[(4 + f) * NQ + q]);
      }
      T acc = A::add(A::norm(acc0), A::norm(acc1));
      for (int a = 0; a < 3; ++a) {
        const T* phe = tab + to.edge_phi[P][g_pe[a]][a][g_fl[a]];
        for (int q = 0; q < g_pe[a] + 2; ++q) A::madd(acc, phe[q * NP + i], sFhat[(a * kNsPt + q) * 4 + f]);
      }
      if (shock) {  // + eps (grad phi_i, q_f)_K = eps sum_k D_k Q_(k,f)
        T v = zero;
        for (int k = 0; k < 2; ++k)
          for (int j = 0; j < NP; ++j) A::madd(v, sDk[k * NP * NP + i * NP + j], sU[(k * 4 + f) * NP + j]);
        A::madd(acc, eps, A::norm(v));
      }
      if (s.src) A::msub(acc, g_det, A::from_d(s.src[m.u_off[K] + 8 * NP + t]));  // -(phi_i, s_h)_K
      sNu[8 * NP + t] = A::norm(acc);
    }
    for (int t = tid; t < nt; t += NT) {
      const int a = g_cf[t], f = g_cg[t], k = g_cl[t], nk = g_nk[a];
      const T* ps = tab + to.edge_psi[g_pe[a]];
      T acc = zero;
      for (int q = 0; q < nk + 1; ++q) A::madd(acc, ps[q * nk + k], sFhat[(a * kNsPt + q) * 4 + f]);
      acc = A::norm(acc);
      sNl[t] = acc;
      sE[t] = A::neg(acc);  // H
    }
    // ---------------- A_ww (volume), B_w, D, C_w ----------------
    // constant row 0: A_00 = A_03 = 0, A_01 = -D_x, A_02 = -D_y (the mass flux has no viscous part)
    for (int t = tid; t < NP * NP; t += NT) {
      const int i = t / NP, j = t - i * NP;
      T* a0 = sA + i * LDA + j;
      a0[0] = zero;
      a0[NP] = A::neg(sDk[t]);
      a0[2 * NP] = A::neg(sDk[NP * NP + t]);
      a0[3 * NP] = zero;
    }
    // B_w: rows (f,i) over warps, trace columns over lanes; in adjoint mode C_w^T instead,
    // C_w^T[(f,i), (a,g,l)] = alpha |e_a| <psi_l, phi_i> delta_fg
    constexpr bool adjoint = ADJ;  // a separate instantiation: the primal kernel carries none of it
    for (int r = ty; r < NW4; r += NW) {
      const int f = r / NP, i = r - f * NP;
      for (int c = tx; c < nt; c += 32) {
        const int a = g_cf[c], g = g_cg[c], l = g_cl[c], nk = g_nk[a];
        T acc = zero;
        if (adjoint) {
          if (g == f) acc = A::mul(A::mul(alpha, g_len[a]), tab[to.edge_cross[P][g_pe[a]][a][g_fl[a]] + l * NP + i]);
        } else {
          const T* phe = tab + to.edge_phi[P][g_pe[a]][a][g_fl[a]];
          for (int q = 0; q < nk + 1; ++q) A::madd(acc, phe[q * NP + i], sW[((a * kNsPt + q) * 16 + f * 4 + g) * 5 + l]);
        }
        sR[r * ldr + c] = A::norm(acc);
      }
    }
    // S0 = D (block diagonal over faces), zero elsewhere
    for (int r = ty; r < nt; r += NW) {
      const int a = g_cf[r], f = g_cg[r], k = g_cl[r], nk = g_nk[a];
      const T* ps = tab + to.edge_psi[g_pe[a]];
      for (int c = tx; c < nt; c += 32) {
        T acc = zero;
        if (g_cf[c] == a) {
          const int g = g_cg[c], l = g_cl[c];
          for (int q = 0; q < nk + 1; ++q) A::madd(acc, ps[q * nk + k], sW[((a * kNsPt + q) * 16 + f * 4 + g) * 5 + l]);
          acc = A::norm(acc);
        }
        sS[r * lds + c] = acc;
      }
    }
    // C' starts as C_w = alpha |e_a| <psi_l, phi_j> delta_fg
    for (int r = ty; r < nt; r += NW) {
      const int a = g_cf[r], f = g_cg[r], l = g_cl[r];
      const T* me = tab + to.edge_cross[P][g_pe[a]][a][g_fl[a]];
      const T sc = A::mul(alpha, g_len[a]);
      for (int c = tx; c < NW4; c += 32) {
        const int g = c / NP, j = c - g * NP;
        sCp[r * ldc + c] = (g == f) ? A::mul(sc, me[l * NP + j]) : zero;
      }
    }
    // state-dependent rows f = 1..3 of A_ww: Z_g[i][q] = sum_r dphi_i/dxi_r Ahat_r,fg; A_fg = -Z phi^T
    for (int f = 1; f < 4; ++f) {
      for (int t = tid; t < 4 * NP * NQ; t += NT) {
        const int g = t / (NP * NQ), rem = t - g * NP * NQ, i = rem / NQ, q = rem - i * NQ;
        sZ[t] = A::add(A::mul(vgx[q * NP + i], sAww[((f - 1) * 4 + g) * NQ + q]),
                       A::mul(vge[q * NP + i], sAww[(12 + (f - 1) * 4 + g) * NQ + q]));
      }
      __syncthreads();
      for (int t = tid; t < 4 * NP * NP; t += NT) {
        const int g = t / (NP * NP), rem = t - g * NP * NP, i = rem / NP, j = rem - i * NP;
        const T* z = sZ + (g * NP + i) * NQ;
        T acc0 = zero, acc1 = zero;
        for (int q = 0; q + 1 < NQ; q += 2) {
          A::msub(acc0, z[q], vphi[q * NP + j]);
          A::msub(acc1, z[q + 1], vphi[(q + 1) * NP + j]);
        }
        if (NQ & 1) A::msub(acc0, z[NQ - 1], vphi[(NQ - 1) * NP + j]);
        sA[(f * NP + i) * LDA + g * NP + j] = A::add(A::norm(acc0), A::norm(acc1));
      }
      __syncthreads();
    }
    // face mass alpha <phi_i, phi_j>_dK and the pseudo-time mass on the diagonal blocks; F_w
    T* sDw = sW;  // D_k^wall = D_k - sum over wall faces n_k |e| <phi_i, phi_j>_e (sW is dead here)
    for (int t = tid; t < NP * NP; t += NT) {
      const int i = t / NP, j = t - i * NP;
      T v = zero;
      for (int a = 0; a < 3; ++a)
        if (g_e[a] >= 0) A::madd(v, g_len[a], tab[to.face_mass[P][g_pe[a]][a] + t]);  // no alpha on walls
      v = A::mul(alpha, A::norm(v));
      if (i == j) v = A::add(v, g_mt);
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        T* p = &sA[(f * NP + i) * LDA + f * NP + j];
        *p = A::add(*p, v);
      }
      if (g_bnd) {
        // boundary flux Jacobian <phi_i, (d f_hat_b / d w)_fg phi_j>_e: walls fill the columns
        // g = rho, E (the others are zero in sAl), the far field all four
        T wv[4][4], b0 = zero, b1 = zero;
#pragma unroll
        for (int f = 0; f < 4; ++f)
#pragma unroll
          for (int g = 0; g < 4; ++g) wv[f][g] = zero;
        for (int a = 0; a < 3; ++a) {
          if (g_e[a] >= 0) continue;
          const T* phe = tab + to.edge_phi[P][P][a][g_fl[a]];
          for (int q = 0; q < P + 2; ++q) {
            const T pp = A::mul(phe[q * NP + i], phe[q * NP + j]);
            const T* al = sAl + (a * kNsPt + q) * 16;
#pragma unroll
            for (int f = 0; f < 4; ++f)
#pragma unroll
              for (int g = 0; g < 4; ++g) A::madd(wv[f][g], pp, al[f * 4 + g]);
          }
          if (g_bc[a] == 3) {  // D_k^wall: the wall term of the gradient equations
            const T fmv = A::mul(g_len[a], tab[to.face_mass[P][P][a] + t]);
            A::madd(b0, g_n[a][0], fmv);
            A::madd(b1, g_n[a][1], fmv);
          }
        }
#pragma unroll
        for (int f = 0; f < 4; ++f)
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            T* pg = &sA[(f * NP + i) * LDA + g * NP + j];
            *pg = A::norm(A::add(*pg, A::norm(wv[f][g])));
          }
        if (g_wall) {
          sDw[t] = A::norm(A::sub(sDk[t], A::norm(b0)));
          sDw[NP * NP + t] = A::norm(A::sub(sDk[NP * NP + t], A::norm(b1)));
        }
      }
    }
    for (int t = tid; t < NW4; t += NT)  // F_w, or the adjoint right-hand side F~_w
      sR[t * ldr + nt] = adjoint ? A::from_d(s.ftilde[m.u_off[K] + 8 * NP + t]) : A::neg(sNu[8 * NP + t]);
    __syncthreads();

    // ---------------- q elimination, one (k', g) block column at a time ----------------
    // Every product below runs over its (row, column) pairs flattened across the
    // CTA.  Rows of field 0 of A_wq and C_q vanish (the mass flux has no viscous
    // part), so they are skipped unless shock capturing adds eps D_k there.  The
    // trace columns of field g are enumerated directly (nt / 4 of them: face a,
    // mode l -> column toff[a] + g nk_a + l) instead of being filtered.
    const T ic = g_ic;
    const int nq4 = nt / 4;  // trace columns per field
    // Pass 0: the q elimination of the primal (or the transposed one of the adjoint mode), the
    // LU and X_w.  Pass 1 (adjoint mode only): X~_q = (G_q - A_wq^T X~_w) / det.  Each pass
    // produces the A_wq block column kk = (k', g) into sBc [4 n_p][n_p] and the C_q block column
    // into sCc [nt][n_p] from the resident point data (sZ is free again after the LU).
    int bad = 0;
    for (int pass = 0; pass < 2; ++pass) {
      if (pass == 1 && !adjoint) break;
      for (int kk = 0; kk < 8; ++kk) {
        const int kd = kk >> 2, gq = kk & 3;
        const int r0 = (shock && gq == 0) ? 0 : NP;  // first row of A_wq that can be nonzero
        // Z'_f[i][q] = sum_r dphi_i/dxi_r Ahat^wq_r,f,kk (rows f = 1..3)
        for (int t = tid; t < 3 * NP * NQ; t += NT) {
          const int f1 = t / (NP * NQ), rem = t - f1 * NP * NQ, i = rem / NQ, q = rem - i * NQ;
          sZ[t] = A::add(A::mul(vgx[q * NP + i], sAwq[(f1 * 8 + kk) * NQ + q]),
                         A::mul(vge[q * NP + i], sAwq[(24 + f1 * 8 + kk) * NQ + q]));
        }
        // C_q block column: rows (a, f, l), C_q = <psi_l, (-n.df_v/dq)_f,kk phi_j>_e
        for (int t = tid; t < nt * NP; t += NT) {
          const int r = t / NP, jj = t - r * NP;
          const int a = g_cf[r], f = g_cg[r], l = g_cl[r], nk = g_nk[a];
          T acc = zero;
          if (f > 0) {
            const T* phe = tab + to.edge_phi[P][g_pe[a]][a][g_fl[a]];
            const T* ps = tab + to.edge_psi[g_pe[a]];
            for (int q = 0; q < nk + 1; ++q)
              A::madd(acc, A::mul(ps[q * nk + l], sAq[(a * kNsPt + q) * 24 + (f - 1) * 8 + kk]), phe[q * NP + jj]);
          }
          sCc[t] = A::norm(acc);
        }
        __syncthreads();
        // A_wq block column: volume (Z' phi^T) + face <phi_i, (-n.df_v/dq) phi_j>_dK; rows of field 0
        // are zero (plus eps D_k on field gq under shock capturing)
        for (int t = tid; t < NW4 * NP; t += NT) {
          const int r = t / NP, jj = t - r * NP, f = r / NP, i = r - f * NP;
          T acc0 = zero, acc1 = zero;
          if (f > 0) {
            const T* z = sZ + ((f - 1) * NP + i) * NQ;
            for (int q = 0; q < NQ; ++q) A::madd(acc0, z[q], vphi[q * NP + jj]);
            for (int a = 0; a < 3; ++a) {
              const T* phe = tab + to.edge_phi[P][g_pe[a]][a][g_fl[a]];
              for (int q = 0; q < g_pe[a] + 2; ++q)
                A::madd(acc1, A::mul(phe[q * NP + i], sAq[(a * kNsPt + q) * 24 + (f - 1) * 8 + kk]), phe[q * NP + jj]);
            }
          }
          T acc = A::add(A::norm(acc0), A::norm(acc1));
          if (shock && f == gq) A::madd(acc, eps, sDk[kd * NP * NP + i * NP + jj]);  // frozen shock capturing
          sBc[t] = A::norm(acc);
        }
        __syncthreads();
        if (pass == 1) {
          double* xk = s.X + m.x_off[K];
          const double* ftq = s.ftilde + m.u_off[K] + kk * NP;
          for (int t = tid; t < NP * nr1; t += NT) {
            const int c = t / NP, i = t - c * NP;
            T acc = (c < nt) ? sCc[c * NP + i] : A::from_d(ftq[i]);
            for (int r = 0; r < NW4; ++r) A::msub(acc, sBc[r * NP + i], sR[r * ldr + c]);
            const T v = A::mul(A::norm(acc), ic);
            xk[(size_t)c * N + kk * NP + i] = A::to_d(v);
            bad |= A::bad(v);
          }
          __syncthreads();
          continue;
        }
        // A_qw block of field gq: D_k, or D_k^wall for rho and E on a wall element
        const T* Dk = ((g_wall && (gq == 0 || gq == 3)) ? sDw : sDk) + kd * NP * NP;
        // (i) A'[(f,i),(g,j)] -= 1/det sum_i' A_wq[(f,i),i'] D_k'[i'][j]
        for (int t = r0 * NP + tid; t < NW4 * NP; t += NT) {
          const int r = t / NP, jj = t - r * NP;
          T acc = zero;
          for (int i2 = 0; i2 < NP; ++i2) A::madd(acc, sBc[r * NP + i2], Dk[i2 * NP + jj]);
          T* p = &sA[r * LDA + gq * NP + jj];
          A::msub(*p, ic, A::norm(acc));
          *p = A::norm(*p);
        }
        if (adjoint) {
          // transposed system: G'_w = G_w - A_qw^T G_q / det on the rows of field g, with
          // G_q = [C_q^T | F~_q] of this block: A_qw^T G_q = D_k'^T [C_q^T | F~_q]
          const double* ftq = s.ftilde + m.u_off[K] + kk * NP;
          for (int t = tid; t < NP * nr1; t += NT) {
            const int i = t / nr1, c = t - i * nr1;
            T acc = zero;
            for (int i2 = 0; i2 < NP; ++i2)
              A::madd(acc, Dk[i2 * NP + i], (c < nt) ? sCc[c * NP + i2] : A::from_d(ftq[i2]));
            T* p = &sR[(gq * NP + i) * ldr + c];
            A::msub(*p, ic, A::norm(acc));
            *p = A::norm(*p);
          }
        } else {
          // (ii)+(iii) R'_w -= 1/det A_wq R_q on the columns of field g and the F column,
          // B_q = -n_k' |e_a| <phi_i', psi_l>
          {
            const int ncol = nq4 + 1;
            for (int t = tid; t < (NW4 - r0) * ncol; t += NT) {
              const int r = r0 + t / ncol, cc = t - (t / ncol) * ncol;
              T acc = zero;
              int c;
              if (cc == nq4) {
                c = nt;
                for (int i2 = 0; i2 < NP; ++i2) A::msub(acc, sBc[r * NP + i2], sNu[kk * NP + i2]);  // F_q = -N_q
              } else {
                const int a = (cc < g_nk[0]) ? 0 : (cc < g_nk[0] + g_nk[1] ? 1 : 2);
                const int l = cc - (a > 0 ? g_nk[0] : 0) - (a > 1 ? g_nk[1] : 0);
                c = g_toff[a] + gq * g_nk[a] + l;
                const T* me = tab + to.edge_cross[P][g_pe[a]][a][g_fl[a]];
                T s2 = zero;
                for (int i2 = 0; i2 < NP; ++i2) A::madd(s2, sBc[r * NP + i2], me[l * NP + i2]);
                acc = A::neg(A::mul(A::mul(g_n[a][kd], g_len[a]), A::norm(s2)));   // A_wq B_q
              }
              T* p = &sR[r * ldr + c];
              A::msub(*p, ic, A::norm(acc));
              *p = A::norm(*p);
            }
          }
          // (iv) C' -= 1/det C_q A_qw
          for (int t = tid; t < nt * NP; t += NT) {
            const int r = t / NP, cc = t - r * NP;
            if (g_cg[r] == 0) continue;  // C_q row of field 0 is zero
            T acc = zero;
            for (int i2 = 0; i2 < NP; ++i2) A::madd(acc, sCc[r * NP + i2], Dk[i2 * NP + cc]);
            T* p = &sCp[r * ldc + gq * NP + cc];
            A::msub(*p, ic, A::norm(acc));
            *p = A::norm(*p);
          }
          // (v)+(vi) S0 -= 1/det C_q B_q on the columns of field g, E0 -= 1/det C_q F_q
          {
            const int ncol = nq4 + 1;
            for (int t = tid; t < nt * ncol; t += NT) {
              const int r = t / ncol, cc = t - r * ncol;
              if (g_cg[r] == 0) continue;  // C_q row of field 0 is zero
              T acc = zero;
              if (cc == nq4) {
                for (int i2 = 0; i2 < NP; ++i2) A::msub(acc, sCc[r * NP + i2], sNu[kk * NP + i2]);
                T* p = &sE[r];
                A::msub(*p, ic, A::norm(acc));
                *p = A::norm(*p);
              } else {
                const int a = (cc < g_nk[0]) ? 0 : (cc < g_nk[0] + g_nk[1] ? 1 : 2);
                const int l = cc - (a > 0 ? g_nk[0] : 0) - (a > 1 ? g_nk[1] : 0);
                const int c = g_toff[a] + gq * g_nk[a] + l;
                const T* me = tab + to.edge_cross[P][g_pe[a]][a][g_fl[a]];
                T s2 = zero;
                for (int i2 = 0; i2 < NP; ++i2) A::madd(s2, sCc[r * NP + i2], me[l * NP + i2]);
                acc = A::neg(A::mul(A::mul(g_n[a][kd], g_len[a]), A::norm(s2)));   // C_q B_q
                T* p = &sS[r * lds + c];
                A::msub(*p, ic, A::norm(acc));
                *p = A::norm(*p);
              }
            }
          }
        }
        __syncthreads();
        if (FAR && g_nff) {
          // far field: A_qw of block (k', g) also holds -n_k' sum_x phi_i(x) (we J)_{g,g2}(x) phi_j(x)
          // for every field g2 (the characteristic state couples the fields).  Its products go
          // through the far-field points x: Y[r][x] = sum_i' M[r][i'] phi_i'(x) for the block
          // column M = A_wq (then C_q), and the update sum_x Y[r][x] coef(x, g2) phi_j(x).
          const int nff = g_nff;
          for (int t = tid; t < NW4 * nff; t += NT) {  // Y from the A_wq block column
            const int r = t / nff, x = t - r * nff, a = g_ffa[x];
            const T* phx = tab + to.edge_phi[P][P][a][g_fl[a]] + g_ffq[x] * NP;
            T acc = zero;
            for (int i2 = 0; i2 < NP; ++i2) A::madd(acc, sBc[r * NP + i2], phx[i2]);
            sYf[t] = A::norm(acc);
          }
          __syncthreads();
          // (i') A'[r][(g2, j)] -= 1/det sum_x Y[r][x] (-n_k' (we J)_{g,g2}(x)) phi_j(x)
          for (int t = tid; t < NW4 * NW4; t += NT) {
            const int r = t / NW4, c = t - r * NW4, g2 = c / NP, jj = c - g2 * NP;
            T acc = zero;
            for (int x = 0; x < nff; ++x) {
              const int a = g_ffa[x], pt = a * kNsPt + g_ffq[x];
              const T phj = tab[to.edge_phi[P][P][a][g_fl[a]] + g_ffq[x] * NP + jj];
              const T coef = A::mul(A::neg(g_n[a][kd]), sFb[pt * 20 + 4 + gq * 4 + g2]);
              A::madd(acc, A::mul(coef, phj), sYf[r * nff + x]);
            }
            T* p = &sA[r * LDA + c];
            A::msub(*p, ic, A::norm(acc));
            *p = A::norm(*p);
          }
          __syncthreads();
          if (adjoint) {
            // G'_w[(g2, j)][c] -= 1/det sum_x (-n_k' (we J)_{g,g2}(x)) phi_j(x) sum_i' phi_i'(x) G_q[i'][c]
            const double* ftq = s.ftilde + m.u_off[K] + kk * NP;
            for (int t = tid; t < nff * nr1; t += NT) {
              const int x = t / nr1, c = t - x * nr1, a = g_ffa[x];
              const T* phx = tab + to.edge_phi[P][P][a][g_fl[a]] + g_ffq[x] * NP;
              T acc = zero;
              for (int i2 = 0; i2 < NP; ++i2)
                A::madd(acc, phx[i2], (c < nt) ? sCc[c * NP + i2] : A::from_d(ftq[i2]));
              sYf[t] = A::norm(acc);
            }
            __syncthreads();
            for (int t = tid; t < NW4 * nr1; t += NT) {
              const int rr = t / nr1, c = t - rr * nr1, g2 = rr / NP, jj = rr - g2 * NP;
              T acc = zero;
              for (int x = 0; x < nff; ++x) {
                const int a = g_ffa[x], pt = a * kNsPt + g_ffq[x];
                const T phj = tab[to.edge_phi[P][P][a][g_fl[a]] + g_ffq[x] * NP + jj];
                const T coef = A::mul(A::neg(g_n[a][kd]), sFb[pt * 20 + 4 + gq * 4 + g2]);
                A::madd(acc, A::mul(coef, phj), sYf[x * nr1 + c]);
              }
              T* p = &sR[rr * ldr + c];
              A::msub(*p, ic, A::norm(acc));
              *p = A::norm(*p);
            }
          } else {
            // (iv') C'[r][(g2, j)] -= 1/det sum_x Yc[r][x] (-n_k' (we J)_{g,g2}(x)) phi_j(x)
            for (int t = tid; t < nt * nff; t += NT) {
              const int r = t / nff, x = t - r * nff, a = g_ffa[x];
              const T* phx = tab + to.edge_phi[P][P][a][g_fl[a]] + g_ffq[x] * NP;
              T acc = zero;
              if (g_cg[r] != 0)
                for (int i2 = 0; i2 < NP; ++i2) A::madd(acc, sCc[r * NP + i2], phx[i2]);
              sYf[t] = A::norm(acc);
            }
            __syncthreads();
            for (int t = tid; t < nt * NW4; t += NT) {
              const int r = t / NW4, c = t - r * NW4, g2 = c / NP, jj = c - g2 * NP;
              if (g_cg[r] == 0) continue;  // C_q row of field 0 is zero
              T acc = zero;
              for (int x = 0; x < nff; ++x) {
                const int a = g_ffa[x], pt = a * kNsPt + g_ffq[x];
                const T phj = tab[to.edge_phi[P][P][a][g_fl[a]] + g_ffq[x] * NP + jj];
                const T coef = A::mul(A::neg(g_n[a][kd]), sFb[pt * 20 + 4 + gq * 4 + g2]);
                A::madd(acc, A::mul(coef, phj), sYf[r * nff + x]);
              }
              T* p = &sCp[r * ldc + c];
              A::msub(*p, ic, A::norm(acc));
              *p = A::norm(*p);
            }
          }
          __syncthreads();
        }
      }
      if (pass == 1) break;
      if (adjoint) {  // the adjoint solves with the transposed Schur matrix A'^T (Sec. 4.2)
        for (int t = tid; t < NW4 * NW4; t += NT) {
          const int i = t / NW4, j = t - i * NW4;
          if (i < j) {
            const T v = sA[i * LDA + j];
            sA[i * LDA + j] = sA[j * LDA + i];
            sA[j * LDA + i] = v;
          }
        }
        __syncthreads();
      }

      // ---------------- a4/a5: LU with partial pivoting on [A' | R'_w] ----------------
      lu_solve<T, NW4, NT>(sA, LDA, sR, ldr, nr1, reinterpret_cast<int*>(sZ), s_pinv, &s_bad, tid);  // sZ is dead here
      // X_w (renormalised in place) and the interior residual
      {
        double* xk = s.X + m.x_off[K];
        for (int t = tid; t < NW4 * nr1; t += NT) {
          const int c = t / NW4, r = t - c * NW4;
          const T v = A::norm(sR[r * ldr + c]);
          sR[r * ldr + c] = v;
          xk[(size_t)c * N + 8 * NP + r] = A::to_d(v);
          bad |= A::bad(v);
        }
        double* ru = s.res_u + m.u_off[K];
        for (int t = tid; t < N; t += NT) ru[t] = A::to_d(sNu[t]);
      }
      __syncthreads();
    }
    if (adjoint) {  // the adjoint needs only the local solves
      if (bad) atomicOr(&s_bad, 2);
      __syncthreads();
      if (tid == 0) s.status[K] = (s_bad & 1) ? 1 : ((s_bad & 2) ? 2 : 0);
      __syncthreads();
      continue;
    }
    // X_q = (R_q - A_qw X_w) / det; with far-field faces A_qw also holds
    // -n_k sum_x phi_i(x) (we J)_fg(x) phi_j(x), applied through the points in column chunks:
    // Tf[x][f][c] = sum_g (we J)_fg(x) X_w,g(x, c)
    const int nff = FAR ? g_nff : 0;
    const int cch = nff ? max(1, lay.nyf / (4 * nff)) : nr1;
    for (int c0 = 0; c0 < nr1; c0 += cch) {
      const int nc = min(cch, nr1 - c0);
      if (nff) {
        for (int t = tid; t < nff * 4 * nc; t += NT) {
          const int x = t / (4 * nc), rem = t - x * 4 * nc, f = rem / nc, cc = rem - f * nc;
          const int a = g_ffa[x], pt = a * kNsPt + g_ffq[x];
          const T* phx = tab + to.edge_phi[P][P][a][g_fl[a]] + g_ffq[x] * NP;
          T acc = zero;
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            T xw = zero;
            for (int j = 0; j < NP; ++j) A::madd(xw, phx[j], sR[(g * NP + j) * ldr + c0 + cc]);
            A::madd(acc, sFb[pt * 20 + 4 + f * 4 + g], A::norm(xw));
          }
          sYf[t] = A::norm(acc);
        }
        __syncthreads();
      }
      double* xk = s.X + m.x_off[K];
      for (int t = tid; t < 8 * NP * nc; t += NT) {
        const int c = c0 + t / (8 * NP), r = t - (t / (8 * NP)) * (8 * NP), kf = r / NP, i = r - kf * NP, k = kf >> 2,
                  f = kf & 3;
        T acc = zero;
        if (c == nt) {
          acc = A::neg(sNu[r]);                           // F_q
        } else if (g_cg[c] == f) {
          const int a = g_cf[c], l = g_cl[c];
          const T* me = tab + to.edge_cross[P][g_pe[a]][a][g_fl[a]];
          acc = A::neg(A::mul(A::mul(g_n[a][k], g_len[a]), me[l * NP + i]));   // B_q
        }
        const T* Dq = ((g_wall && (f == 0 || f == 3)) ? sDw : sDk) + k * NP * NP;
        for (int j = 0; j < NP; ++j) A::msub(acc, Dq[i * NP + j], sR[(f * NP + j) * ldr + c]);
        for (int x = 0; x < nff; ++x) {  // - (far-field part of A_qw) X_w
          const int a = g_ffa[x];
          const T phi_i = tab[to.edge_phi[P][P][a][g_fl[a]] + g_ffq[x] * NP + i];
          A::madd(acc, A::mul(g_n[a][k], phi_i), sYf[(x * 4 + f) * nc + (c - c0)]);
        }
        const T v = A::mul(A::norm(acc), ic);
        xk[(size_t)c * N + r] = A::to_d(v);
        bad |= A::bad(v);
      }
      if (nff) __syncthreads();  // the next chunk rewrites sYf
    }
    // ---------------- a6/a7: S = S0 - C' X_w,B, E = E0 - C' X_w,F, assembly ----------------
    for (int r = ty; r < nt; r += NW) {
      const int a = g_cf[r], rl = r - g_toff[a];
      for (int c = tx; c < nr1; c += 32) {
        T v = (c == nt) ? sE[r] : sS[r * lds + c];
        for (int j = 0; j < NW4; ++j) A::msub(v, sCp[r * ldc + j], sR[j * ldr + c]);
        v = A::norm(v);
        bad |= A::bad(v);
        if (c == nt) {
          sE[r] = v;
        } else {
          const int b = g_cf[c];
          if (b == a) sS[r * lds + c] = v;
          else s.K[m.kblk[9 * (size_t)K + 3 * a + b] + rl * (4 * g_nk[b]) + (c - g_toff[b])] = A::to_d(v);
        }
      }
    }
    if (bad) atomicOr(&s_bad, 2);
    __syncthreads();
    // two-sided sums: side 0 parks its halves in K/E/res_lam, side 1 in the work space
    for (int a = 0; a < 3; ++a) {
      const int e = g_e[a], m4 = 4 * g_nk[a], o = g_toff[a];
      if (e < 0) continue;  // wall face: nothing to assemble
      const int64_t lo = m.lam_off[e];
      double* dd = g_side[a] ? s.dhalf1 + m.dblk_off[e] : s.K + m.kblk[9 * (size_t)K + 4 * a];
      double* de = g_side[a] ? s.ehalf1 + lo : s.E + lo;
      double* dr = g_side[a] ? s.rhalf1 + lo : s.res_lam + lo;
      for (int t = tid; t < m4 * m4; t += NT) {
        const int r = t / m4, c = t - r * m4;
        dd[t] = A::to_d(sS[(o + r) * lds + o + c]);
      }
      for (int t = tid; t < m4; t += NT) {
        de[t] = A::to_d(sE[o + t]);
        dr[t] = A::to_d(sNl[o + t]);
      }
    }
    __threadfence();
    __syncthreads();
    if (tid < 3) {
      g_old[tid] = g_e[tid] >= 0 ? atomicAdd(&s.face_cnt[g_e[tid]], 1) : 0;
      __threadfence();
    }
    __syncthreads();
    for (int a = 0; a < 3; ++a) {
      if (g_old[a] != 1) continue;
      const int e = g_e[a], m4 = 4 * g_nk[a], o = g_toff[a];
      const int64_t lo = m.lam_off[e];
      double* k0 = s.K + m.kblk[9 * (size_t)K + 4 * a];
      const double* k1 = s.dhalf1 + m.dblk_off[e];
      const int side = g_side[a];
      for (int t = tid; t < m4 * m4; t += NT) {
        const int r = t / m4, c = t - r * m4;
        const double mine = A::to_d(sS[(o + r) * lds + o + c]);
        const double other = side ? __ldcg(k0 + t) : __ldcg(k1 + t);
        k0[t] = side ? other + mine : mine + other;
      }
      for (int t = tid; t < m4; t += NT) {
        const double me_ = A::to_d(sE[o + t]), mr = A::to_d(sNl[o + t]);
        const double oe = side ? __ldcg(s.E + lo + t) : __ldcg(s.ehalf1 + lo + t);
        const double orr = side ? __ldcg(s.res_lam + lo + t) : __ldcg(s.rhalf1 + lo + t);
        s.E[lo + t] = side ? oe + me_ : me_ + oe;
        s.res_lam[lo + t] = side ? orr + mr : mr + orr;
      }
      if (tid == 0) s.face_cnt[e] = 0;
    }
    if (tid == 0) s.status[K] = (s_bad & 1) ? 1 : ((s_bad & 2) ? 2 : 0);
    __syncthreads();
  }
}

template <int P, class T, bool ADJ, bool BATCH = false, bool FAR = BATCH>
inline bool launch_ns_bucket(const DevMesh& m, const DevSys& s, const Phys& ph, const T* tab, const TabOff& to,
                             const double* U, const double* Lam, const int* elems, int n, int ntmax, cudaStream_t st,
                             std::string* err, const BatchRef& bt = BatchRef{}) {
  const NsLayout<P> lay(ntmax);
  // the far-field regions close the layout: an instance without far-field code leaves them out
  const size_t bytes = sizeof(T) * (size_t)(FAR ? lay.total : lay.oFb);
  const NsLayout<P> big(kMaxNt);
  const size_t cap = sizeof(T) * (size_t)(FAR ? big.total : big.oFb);
  cudaError_t ce = set_smem_cap(k_condense_ns<P, T, ADJ, BATCH, FAR>, cap, bytes);
  if (ce != cudaSuccess) { *err = std::string("NS kernel shared memory: ") + cudaGetErrorString(ce); return false; }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_condense_ns<P, T, ADJ, BATCH, FAR>, ns_threads<P>(), bytes);
  if (per_sm < 1) { *err = "NS condensation kernel does not fit on an SM"; return false; }
  const long grid = condense_grid(ph, P, sms, per_sm, n);
  k_condense_ns<P, T, ADJ, BATCH, FAR><<<(int)grid, ns_threads<P>(), bytes, st>>>(m, s, ph, tab, to, U, Lam, elems, n,
                                                                              ntmax, bt);
  ce = cudaGetLastError();
  if (ce != cudaSuccess) { *err = cudaGetErrorString(ce); return false; }
  return true;
}

template <int P, class T>
inline int ns_occ(int ntmax) {  // the instance without far-field code
  const NsLayout<P> lay(ntmax);
  const size_t bytes = sizeof(T) * (size_t)lay.oFb;
  const size_t cap = sizeof(T) * (size_t)NsLayout<P>(kMaxNt).oFb;
  if (set_smem_cap(k_condense_ns<P, T, false, false>, cap, bytes) != cudaSuccess) return 0;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_condense_ns<P, T, false, false>, ns_threads<P>(), bytes);
  return per_sm;
}

template <class T>
inline int ns_occ_p(int p, int ntmax) {
  switch (p) {
    case 1: return ns_occ<1, T>(ntmax);
    case 2: return ns_occ<2, T>(ntmax);
    case 3: return ns_occ<3, T>(ntmax);
    case 4: return ns_occ<4, T>(ntmax);
  }
  return 0;
}

template <class T, bool ADJ = false, bool FAR = false>
inline bool launch_ns_p(int p, const DevMesh& m, const DevSys& s, const Phys& ph, const T* tab, const TabOff& to,
                        const double* U, const double* Lam, const int* elems, int n, int ntmax, cudaStream_t st,
                        std::string* err) {
  switch (p) {
    case 1: return launch_ns_bucket<1, T, ADJ, false, FAR>(m, s, ph, tab, to, U, Lam, elems, n, ntmax, st, err);
    case 2: return launch_ns_bucket<2, T, ADJ, false, FAR>(m, s, ph, tab, to, U, Lam, elems, n, ntmax, st, err);
    case 3: return launch_ns_bucket<3, T, ADJ, false, FAR>(m, s, ph, tab, to, U, Lam, elems, n, ntmax, st, err);
    case 4: return launch_ns_bucket<4, T, ADJ, false, FAR>(m, s, ph, tab, to, U, Lam, elems, n, ntmax, st, err);
  }
  *err = "degree out of range";
  return false;
}

}  // namespace hdg
