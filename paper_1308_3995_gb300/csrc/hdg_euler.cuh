// Euler element kernel of the HDG Newton-step hot path (sm_103a): the
// condensation of one element per CTA iteration (steps a1-a7), and its
// launcher.  A header so that more than one translation unit can instantiate
// it (the binary64 / float-float kernels in hdg_kernels.cu, the
// mixed-precision local-solve variants in hdg_kernels_mixed.cu).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <type_traits>

#include "hdg_arith.cuh"
#include "hdg_internal.h"
#include "hdg_lu.cuh"
#include "hdg_lu_tc.cuh"
#include "hdg_physics.cuh"

namespace hdg {

// --------------------------------------------------------------------------
// Shared-memory layout of the Euler element kernel (offsets in doubles).
// --------------------------------------------------------------------------
constexpr int kPtSlots = 6;            // edge points per face slot (p_e + 2 <= 6)
template <int P>
struct EulerLayout {
  static constexpr int NP = n_basis(P), NQ = (P + 2) * (P + 2), N = 4 * NP, LDA = N + 1;
  static constexpr int SCR_VOL = NQ * (4 + 8 + 32) + 4 * NP * NQ;
  static constexpr int SCR_FACE = 3 * kPtSlots * (4 + 16 * 5);
  static constexpr int SCR = SCR_VOL > SCR_FACE ? SCR_VOL : SCR_FACE;
  int ldr, dstride, oA, oR, oU, oL, oNu, oNl, oEh, oMe, oD, oScr, total;
  int oTc = -1, oR0 = -1;  // mixed-precision local solve: binary32 work space, copy of [B | F]
  HDG_HD EulerLayout(int ldr_, int nkmax, bool tc = false) : ldr(ldr_), dstride(16 * nkmax * nkmax) {
    oA = 0;
    oR = oA + N * LDA;
    oU = oR + N * ldr;
    oL = oU + N;
    oNu = oL + kMaxNt;
    oNl = oNu + N;
    oEh = oNl + kMaxNt;
    oMe = oEh + kMaxNt;
    oD = oMe + 3 * 5 * NP;
    oScr = oD + 3 * dstride;
    total = oScr + SCR;
    if (tc) {  // binary32 fA [N][LDA], fW [N][ldr], pinv [N] and int piv [N], in 8-byte units
      oTc = total;
      total += (N * LDA + N * ldr + 2 * N + 1) / 2;
      if (N * ldr <= SCR) {
        oR0 = oScr;  // the scratch is dead during the local solve
      } else {
        oR0 = total;
        total += N * ldr;
      }
    }
  }
};

inline int ldr_for(int ntmax) { return (ntmax + 1) | 1; }  // odd leading dimension
// largest single-face trace size in a bucket of degree p: every face has p_e >= p
inline int nkmax_for(int p, int ntmax, bool bounded = false) {
  // on a mesh with boundary faces one face of the element may carry all of nt
  int nk = bounded ? ntmax / 4 : ntmax / 4 - 2 * (p + 1);
  return nk > kMaxP + 1 ? kMaxP + 1 : nk;
}

// --------------------------------------------------------------------------
// Condensation kernel, Euler: one element per CTA iteration, in the
// arithmetic T (binary64, or float-float on the FP32 pipe).  `tab` holds the
// library's tables in that arithmetic.  Inputs and outputs are binary64.
// --------------------------------------------------------------------------
// CTAs per SM: at low degree the element's binary64 work is small and the
// block barriers dominate, so more resident CTAs pay even with some spills:
// p = 1 at 8 (64 registers; 16.6 M instead of 11.0 M elements/s in binary64,
// 18.1 M instead of 11.0 M in float-float), p = 2 at 6 in binary64 (80
// registers; 6.78 M instead of 5.82 M; float-float p = 2 is a little slower
// there and stays at 4), p >= 3 at 4 (shared memory allows no more).
// BATCH: the launch walks the work list `bt` over the elements of several
// systems (hdg_batch_condense), each item reading its own system's mesh plan,
// buffers, parameters and inputs; otherwise m_, s_, ph_, U_, Lam_ and elems.
// The two are separate instantiations of the same source: an element's
// arithmetic is the same, up to the compiler's contraction of multiply-adds.
// LS: the local solve, 0 partial-pivot LU in T (lu_solve), or kTcTF32x3 / kTcBF16:
// binary32 LU with tensor-core updates and refinement against residuals in T
// (tc_refine_solve).
template <int P, class T, int LS = 0, bool BATCH = false>
__global__ void __launch_bounds__(kCondThreads, (P == 1 ? 8 : ((P == 2 && std::is_same<T, double>::value) ? 6 : 4)))
k_condense_euler(
    DevMesh m_, DevSys s_, Phys ph_, const T* __restrict__ tab, TabOff to, const double* __restrict__ U_,
    const double* __restrict__ Lam_, const int* __restrict__ elems, int n_elems, int ldr, int nkmax, BatchRef bt) {
  using L = EulerLayout<P>;
  using A = Ar<T>;
  constexpr int NP = L::NP, NQ = L::NQ, N = L::N, LDA = L::LDA;
  constexpr int NT = kCondThreads;
  extern __shared__ double smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const L lay(ldr, nkmax, LS != 0);
  const int DS = lay.dstride;
  T* sA = smem + lay.oA;
  T* sR = smem + lay.oR;
  T* sU = smem + lay.oU;
  T* sL = smem + lay.oL;
  T* sNu = smem + lay.oNu;
  T* sNl = smem + lay.oNl;
  T* sEh = smem + lay.oEh;
  T* sMe = smem + lay.oMe;
  T* sD = smem + lay.oD;
  T* scr = smem + lay.oScr;
  // volume scratch
  T* sWq = scr;                  // [4][NQ]
  T* sFh = sWq + 4 * NQ;         // [2][4][NQ]
  T* sAh = sFh + 8 * NQ;         // [2][16][NQ]
  T* sZ = sAh + 32 * NQ;         // [4][NP][NQ]
  // face scratch (aliases the volume scratch)
  T* sFhat = scr;                // [3*6][4]
  T* sW = sFhat + 3 * kPtSlots * 4;  // [3*6][16][5]

  __shared__ T g_det, g_Ji[2][2], g_n[3][2], g_len[3], g_mt;
  __shared__ int g_e[3], g_pe[3], g_nk[3], g_toff[4], g_fl[3], g_side[3], g_old[3], g_bc[3];
  // per trace index c < nt of the element: local face, field, mode
  __shared__ unsigned char g_cf[kMaxNt], g_cg[kMaxNt], g_cl[kMaxNt];
  __shared__ T s_pinv[64];
  __shared__ int s_bad;
  __shared__ unsigned s_red[2];

  const int tid = threadIdx.x;
  const int tx = tid & 31, ty = tid >> 5;   // lane, warp: 2-D layouts without index division
  constexpr int NW = NT / 32;
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
    const T alpha = A::from_d(ph.alpha);
    // ---------------- a1: geometry (binary64, three lanes), faces, state ----------------
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
      g_bc[a] = m.elem_bc ? (m.elem_bc[K] >> (2 * a)) & 3 : 0;
      g_pe[a] = e >= 0 ? m.face_p[e] : P;   // boundary face: the element's own degree, no traces
      g_nk[a] = e >= 0 ? g_pe[a] + 1 : 0;
      g_fl[a] = (info >> a) & 1;
      g_side[a] = (info >> (3 + a)) & 1;
      if (tid == 0) {
        const double J00 = c[2] - c[0], J01 = c[4] - c[0], J10 = c[3] - c[1], J11 = c[5] - c[1];
        const double det = J00 * J11 - J01 * J10;
        const double inv = __drcp_rn(det);
        g_det = A::from_d(det);
        g_Ji[0][0] = A::from_d(J11 * inv); g_Ji[0][1] = A::from_d(-J01 * inv);
        g_Ji[1][0] = A::from_d(-J10 * inv); g_Ji[1][1] = A::from_d(J00 * inv);
        // pseudo-time mass det(J)/dt_K (Sec. 3.3), from the element-mean state
        double mt = 0.0;
        if (ph.cfl > 0.0) {
          const double* u0 = U + m.u_off[K];
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
          const double lam_c = (sqrt(uu * uu + vv * vv) + sqrt(ph.gamma * p / rho)) * perim;
          const double dt = ph.cfl * 0.5 * det / lam_c;
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
    }
    {
      const double* uk = U + m.u_off[K];
      for (int t = tid; t < N; t += NT) sU[t] = A::from_d(uk[t]);
    }
    __syncthreads();
    const int nt = g_toff[3];
    for (int c = tid; c < nt; c += NT) {
      const int a = (c >= g_toff[2]) ? 2 : (c >= g_toff[1] ? 1 : 0);
      const int nk = g_nk[a], cl = c - g_toff[a], g = cl / nk;
      g_cf[c] = (unsigned char)a;
      g_cg[c] = (unsigned char)g;
      g_cl[c] = (unsigned char)(cl - g * nk);
    }
    for (int a = 0; a < 3; ++a) {
      if (g_e[a] < 0) continue;  // boundary face: no trace
      const double* lk = Lam + m.lam_off[g_e[a]];
      for (int t = tid; t < 4 * g_nk[a]; t += NT) sL[g_toff[a] + t] = A::from_d(lk[t]);
    }
    __syncthreads();

    // ---------------- a2: volume quadrature ----------------
    for (int t = tid; t < 4 * NQ; t += NT) {
      const int f = t / NQ, q = t - f * NQ;
      T acc = zero;
#pragma unroll
      for (int j = 0; j < NP; ++j) A::madd(acc, sU[f * NP + j], vphi[q * NP + j]);
      sWq[t] = A::norm(acc);
    }
    __syncthreads();
    for (int q = tid; q < NQ; q += NT) {
      T w[4], fx[4], fy[4], Ax[16], Ay[16];
#pragma unroll
      for (int f = 0; f < 4; ++f) w[f] = sWq[f * NQ + q];
      euler_flux_jac(w, C, fx, fy, Ax, Ay);
      const T c = A::mul(vw[q], g_det);
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const T a0 = A::mul(c, g_Ji[r][0]), a1 = A::mul(c, g_Ji[r][1]);
#pragma unroll
        for (int f = 0; f < 4; ++f) sFh[(r * 4 + f) * NQ + q] = A::add(A::mul(a0, fx[f]), A::mul(a1, fy[f]));
        // rows 1..3 only: row 0 of both flux Jacobians is constant
#pragma unroll
        for (int fg = 4; fg < 16; ++fg) sAh[(r * 16 + fg) * NQ + q] = A::add(A::mul(a0, Ax[fg]), A::mul(a1, Ay[fg]));
      }
    }
    __syncthreads();
    // shock-capturing viscosity (Sec. 3.2), held fixed in the Jacobian:
    //   eps_K = eps_0 (h_K/p)^(2-beta) / |K| int_K sum_f |(div f_c(w))_f|.
    // With Ahat_r = c (Ji[r][0] A_x + Ji[r][1] A_y), c = w_q det J, and the reference
    // gradients g_r of w: c div f_c = sum_r Ahat_r g_r (row 0 of A_x, A_y is constant).
    T eps = zero;
    const bool shock = ph.sc_eps0 > 0.0;
    if (shock) {
      for (int q = tid; q < NQ; q += NT) {
        T gr[2][4];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          T a0 = zero, a1 = zero;
#pragma unroll
          for (int j = 0; j < NP; ++j) {
            A::madd(a0, sU[f * NP + j], vgx[q * NP + j]);
            A::madd(a1, sU[f * NP + j], vge[q * NP + j]);
          }
          gr[0][f] = A::norm(a0);
          gr[1][f] = A::norm(a1);
        }
        const T c = A::mul(vw[q], g_det);
        T d0 = zero;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          A::madd(d0, A::mul(c, g_Ji[r][0]), gr[r][1]);
          A::madd(d0, A::mul(c, g_Ji[r][1]), gr[r][2]);
        }
        T d = A::abs(A::norm(d0));
#pragma unroll
        for (int f = 1; f < 4; ++f) {
          T v = zero;
#pragma unroll
          for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int g = 0; g < 4; ++g) A::madd(v, sAh[(r * 16 + f * 4 + g) * NQ + q], gr[r][g]);
          d = A::add(d, A::abs(A::norm(v)));
        }
        sEh[q] = d;  // sEh and sNl are free until the face quadrature
      }
      __syncthreads();
      if (tid == 0) {
        T sum = zero;
        for (int q = 0; q < NQ; ++q) sum = A::add(sum, sEh[q]);
        const double l0 = A::to_d(g_len[0]), l1 = A::to_d(g_len[1]), l2 = A::to_d(g_len[2]);
        const double hk = fmax(l0, fmax(l1, l2)) / P;
        const double fac = ph.sc_eps0 * pow(hk, 2.0 - ph.sc_beta) * 2.0 / A::to_d(g_det);  // 1/|K| = 2/det J
        sNl[0] = A::mul(sum, A::from_d(fac));
      }
      __syncthreads();
      eps = sNl[0];
    }
    // interior residual, volume part: N_w = -(grad phi, f_c(w))_K
    for (int t = tid; t < N; t += NT) {
      const int f = t / NP, i = t - f * NP;
      T acc0 = zero, acc1 = zero;
      for (int q = 0; q < NQ; ++q) {
        A::msub(acc0, vgx[q * NP + i], sFh[f * NQ + q]);
        A::msub(acc1, vge[q * NP + i], sFh[(4 + f) * NQ + q]);
      }
      sNu[t] = A::add(A::norm(acc0), A::norm(acc1));
    }
    // volume Jacobian A_fg = -sum_k (dF_k/dw)_fg D_k.  Blocks whose flux-Jacobian
    // entries are constants (row 0: (0,1) = -D_x, (0,2) = -D_y, (0,0) = (0,3) = 0;
    // (1,3) = -(gamma-1) D_x; (2,3) = -(gamma-1) D_y) use D_k = det J sum_r Ji[r][k] Dref_r.
    for (int t = tid; t < NP * NP; t += NT) {
      const int i = t / NP, j = t - i * NP;
      const T d0 = dref[t], d1 = dref[NP * NP + t];
      const T Dx = A::mul(g_det, A::add(A::mul(g_Ji[0][0], d0), A::mul(g_Ji[1][0], d1)));
      const T Dy = A::mul(g_det, A::add(A::mul(g_Ji[0][1], d0), A::mul(g_Ji[1][1], d1)));
      T* a0 = sA + i * LDA + j;  // block row 0
      a0[0] = zero;
      a0[NP] = A::neg(Dx);
      a0[2 * NP] = A::neg(Dy);
      a0[3 * NP] = zero;
      sA[(NP + i) * LDA + 3 * NP + j] = A::neg(A::mul(C.g1, Dx));
      sA[(2 * NP + i) * LDA + 3 * NP + j] = A::neg(A::mul(C.g1, Dy));
    }
    // state-dependent blocks, one block row f = 1..3 at a time (row 3 has four):
    //   Z_g[i][q] = sum_r dphi_i/dxi_r (q) Ahat_r,fg(q);  A_fg[i][j] = -sum_q Z_g[i][q] phi_j(q)
    for (int f = 1; f < 4; ++f) {
      const int ng = (f == 3) ? 4 : 3;
      for (int t = tid; t < ng * NP * NQ; t += NT) {
        const int g = t / (NP * NQ), rem = t - g * NP * NQ, i = rem / NQ, q = rem - i * NQ;
        sZ[t] = A::add(A::mul(vgx[q * NP + i], sAh[(f * 4 + g) * NQ + q]),
                       A::mul(vge[q * NP + i], sAh[(16 + f * 4 + g) * NQ + q]));
      }
      __syncthreads();
      for (int t = tid; t < ng * NP * NP; t += NT) {
        const int g = t / (NP * NP), rem = t - g * NP * NP, i = rem / NP, j = rem - i * NP;
        const T* z = sZ + (g * NP + i) * NQ;
        T acc0 = zero, acc1 = zero;
#pragma unroll 4
        for (int q = 0; q + 1 < NQ; q += 2) {
          A::msub(acc0, z[q], vphi[q * NP + j]);
          A::msub(acc1, z[q + 1], vphi[(q + 1) * NP + j]);
        }
        if (NQ & 1) A::msub(acc0, z[NQ - 1], vphi[(NQ - 1) * NP + j]);
        sA[(f * NP + i) * LDA + g * NP + j] = A::add(A::norm(acc0), A::norm(acc1));
      }
      __syncthreads();
    }

    // ---------------- a3: face quadrature ----------------
    for (int t = tid; t < 3 * kPtSlots; t += NT) {
      const int a = t / kPtSlots, g = t - a * kPtSlots;
      const int pe = g_pe[a], nk = pe + 1;
      if (g < pe + 2 && g_bc[a]) {
        // boundary operator of Sec. 3.2: <phi, f_c(w_b(w)) . n> and its Jacobian
        // (A_n(w_b) d w_b / d w) on every field pair, kept in slot 0 of sW
        const T* phe = tab + to.edge_phi[P][pe][a][g_fl[a]] + g * NP;
        const T we = A::mul(tab[to.edge_w[pe] + g], g_len[a]);
        T w[4], wb[4], dwb[4][4], fx[4], fy[4], Ax[16], Ay[16];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          T acc = zero;
#pragma unroll
          for (int j = 0; j < NP; ++j) A::madd(acc, sU[f * NP + j], phe[j]);
          w[f] = A::norm(acc);
        }
        T winf[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) winf[f] = A::from_d(ph.winf[f]);
        const T nx = g_n[a][0], ny = g_n[a][1];
        boundary_state_jac(g_bc[a], w, nx, ny, winf, C, wb, dwb);
        euler_flux_jac(wb, C, fx, fy, Ax, Ay);
#pragma unroll
        for (int f = 0; f < 4; ++f) sFhat[t * 4 + f] = A::mul(we, A::add(A::mul(nx, fx[f]), A::mul(ny, fy[f])));
#pragma unroll
        for (int f = 0; f < 4; ++f)
#pragma unroll
          for (int gg = 0; gg < 4; ++gg) {
            T jb = zero;
#pragma unroll
            for (int h = 0; h < 4; ++h)
              A::madd(jb, A::add(A::mul(nx, Ax[f * 4 + h]), A::mul(ny, Ay[f * 4 + h])), dwb[h][gg]);
            sW[(t * 16 + f * 4 + gg) * 5] = A::mul(we, A::norm(jb));
          }
      } else if (g < pe + 2) {
        const T* phe = tab + to.edge_phi[P][pe][a][g_fl[a]] + g * NP;
        const T* ps = tab + to.edge_psi[pe] + g * nk;
        const T we = A::mul(tab[to.edge_w[pe] + g], g_len[a]);
        T w[4], lam[4], fx[4], fy[4], Ax[16], Ay[16];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          T acc = zero;
#pragma unroll
          for (int j = 0; j < NP; ++j) A::madd(acc, sU[f * NP + j], phe[j]);
          w[f] = A::norm(acc);
          T al = zero;
          for (int k = 0; k < nk; ++k) A::madd(al, sL[g_toff[a] + f * nk + k], ps[k]);
          lam[f] = A::norm(al);
        }
        euler_flux_jac(lam, C, fx, fy, Ax, Ay);
        const T nx = g_n[a][0], ny = g_n[a][1];
#pragma unroll
        for (int f = 0; f < 4; ++f)
          sFhat[t * 4 + f] = A::mul(we, A::sub(A::add(A::mul(nx, fx[f]), A::mul(ny, fy[f])),
                                               A::mul(alpha, A::sub(lam[f], w[f]))));
#pragma unroll
        for (int fg = 0; fg < 16; ++fg) {
          T an = A::add(A::mul(nx, Ax[fg]), A::mul(ny, Ay[fg]));
          if (fg % 5 == 0) an = A::sub(an, alpha);
          const T at = A::mul(we, an);
          for (int l = 0; l < nk; ++l) sW[(t * 16 + fg) * 5 + l] = A::mul(at, ps[l]);
        }
      }
    }
    __syncthreads();
    const bool adjoint = ph.adjoint != 0;
    // B = d N_w / d Lambda: the (row (f,i), column (face a; g, l)) pairs flattened over the CTA
    for (int t = tid; t < (adjoint ? 0 : N * nt); t += NT) {
      const int r = t / nt, c = t - r * nt;
      const int f = r / NP, i = r - f * NP;
      const int a = g_cf[c], g = g_cg[c], l = g_cl[c], nk = g_nk[a];
      const T* phe = tab + to.edge_phi[P][g_pe[a]][a][g_fl[a]];
      T acc = zero;
      for (int q = 0; q < nk + 1; ++q) A::madd(acc, phe[q * NP + i], sW[((a * kPtSlots + q) * 16 + f * 4 + g) * 5 + l]);
      sR[r * ldr + c] = A::norm(acc);
    }
    // D_a = d N_lambda,a / d Lambda_a (block diagonal in faces): the entries of the three
    // diagonal blocks flattened over the CTA
    {
      const int s1 = 16 * g_nk[0] * g_nk[0], s2 = s1 + 16 * g_nk[1] * g_nk[1];
      const int tot = s2 + 16 * g_nk[2] * g_nk[2];
      for (int t = tid; t < (adjoint ? 0 : tot); t += NT) {
        const int a = (t >= s2) ? 2 : (t >= s1 ? 1 : 0);
        const int nk = g_nk[a], m4 = 4 * nk, o = g_toff[a];
        const int tl = t - (a == 0 ? 0 : (a == 1 ? s1 : s2));
        const int r = tl / m4, c = tl - r * m4;
        const int f = g_cg[o + r], k = g_cl[o + r], g = g_cg[o + c], l = g_cl[o + c];
        const T* ps = tab + to.edge_psi[g_pe[a]];
        T acc = zero;
        for (int q = 0; q < nk + 1; ++q) A::madd(acc, ps[q * nk + k], sW[((a * kPtSlots + q) * 16 + f * 4 + g) * 5 + l]);
        sD[a * DS + r * m4 + c] = A::norm(acc);
      }
    }
    // C_a = alpha |e_a| <psi_k, phi_j> delta_fg, kept as the scalar edge matrix
    for (int t = tid; t < 3 * 5 * NP; t += NT) {
      const int a = t / (5 * NP), rem = t - a * 5 * NP, k = rem / NP;
      if (k < g_nk[a]) sMe[t] = A::mul(A::mul(alpha, g_len[a]), tab[to.edge_cross[P][g_pe[a]][a][g_fl[a]] + rem]);
    }
    // face parts of the residuals, and the source term -(phi_i, s_h)_K = -det J S_i (Eq. hdg_ls3)
    for (int t = tid; t < N; t += NT) {
      const int f = t / NP, i = t - f * NP;
      T acc = sNu[t];
      for (int a = 0; a < 3; ++a) {
        const T* phe = tab + to.edge_phi[P][g_pe[a]][a][g_fl[a]];
        for (int q = 0; q < g_pe[a] + 2; ++q) A::madd(acc, phe[q * NP + i], sFhat[(a * kPtSlots + q) * 4 + f]);
      }
      if (s.src) A::msub(acc, g_det, A::from_d(s.src[m.u_off[K] + t]));
      sNu[t] = A::norm(acc);
    }
    for (int t = tid; t < nt; t += NT) {
      const int a = (t >= g_toff[2]) ? 2 : (t >= g_toff[1] ? 1 : 0);
      const int nk = g_nk[a], tl = t - g_toff[a], f = tl / nk, k = tl - f * nk;
      const T* ps = tab + to.edge_psi[g_pe[a]];
      T acc = zero;
      for (int q = 0; q < nk + 1; ++q) A::madd(acc, ps[q * nk + k], sFhat[(a * kPtSlots + q) * 4 + f]);
      acc = A::norm(acc);
      sNl[t] = acc;
      sEh[t] = A::neg(acc);  // H
    }
    __syncthreads();
    if (g_bc[0] | g_bc[1] | g_bc[2]) {
      // boundary Jacobian, before the face-mass loop reuses the face scratch:
      // A[(f,i),(g,j)] += sum over boundary faces, points q of phi_i phi_j (w_e A_n(w_b) dw_b/dw)_fg
      for (int t = tid; t < 16 * NP * NP; t += NT) {
        const int fg = t / (NP * NP), rem = t - fg * NP * NP, i = rem / NP, j = rem - i * NP;
        T acc = zero;
        for (int a = 0; a < 3; ++a) {
          if (!g_bc[a]) continue;
          const T* phe = tab + to.edge_phi[P][P][a][g_fl[a]];
          for (int q = 0; q < P + 2; ++q)
            A::madd(acc, A::mul(phe[q * NP + i], phe[q * NP + j]), sW[((a * kPtSlots + q) * 16 + fg) * 5]);
        }
        T* pa = &sA[((fg >> 2) * NP + i) * LDA + (fg & 3) * NP + j];
        *pa = A::add(*pa, A::norm(acc));
      }
      __syncthreads();
    }
    // face mass alpha <phi_i, phi_j>_dK on every field's diagonal block, plus the pseudo-time
    // mass and the frozen shock-capturing stiffness eps (grad phi_i, grad phi_j)_K
    T* sSt = scr;  // [NP][NP] eps * stiffness (the face scratch is dead here)
    for (int t = tid; t < NP * NP; t += NT) {
      const int i = t / NP, j = t - i * NP;
      T v = zero;
      for (int a = 0; a < 3; ++a)
        if (!g_bc[a]) A::madd(v, g_len[a], tab[to.face_mass[P][g_pe[a]][a] + t]);
      v = A::mul(alpha, A::norm(v));
      if (i == j) v = A::add(v, g_mt);
      if (shock) {  // grad phi_i . grad phi_j = sum_rs G_rs d_r phi_i d_s phi_j, G = Ji Ji^T
        const T G00 = A::add(A::mul(g_Ji[0][0], g_Ji[0][0]), A::mul(g_Ji[0][1], g_Ji[0][1]));
        const T G01 = A::add(A::mul(g_Ji[0][0], g_Ji[1][0]), A::mul(g_Ji[0][1], g_Ji[1][1]));
        const T G11 = A::add(A::mul(g_Ji[1][0], g_Ji[1][0]), A::mul(g_Ji[1][1], g_Ji[1][1]));
        const T* sref = tab + to.vol_stiff[P];  // reference stiffness parts (rr, rs + sr, ss)
        T st = A::mul(G00, sref[t]);
        A::madd(st, G01, sref[NP * NP + t]);
        A::madd(st, G11, sref[2 * NP * NP + t]);
        st = A::mul(A::mul(eps, g_det), A::norm(st));
        sSt[t] = st;
        v = A::add(v, st);
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        T* p = &sA[(f * NP + i) * LDA + f * NP + j];
        *p = A::add(*p, v);
      }
    }
    if (shock) {  // N_w += eps (grad phi_i, grad w_f)_K
      __syncthreads();
      for (int t = tid; t < N; t += NT) {
        const int f = t / NP, i = t - f * NP;
        T acc = sNu[t];
        for (int j = 0; j < NP; ++j) A::madd(acc, sSt[i * NP + j], sU[f * NP + j]);
        sNu[t] = A::norm(acc);
      }
    }
    for (int t = tid; t < N; t += NT)  // F, or the adjoint right-hand side F~
      sR[t * ldr + nt] = adjoint ? A::from_d(s.ftilde[m.u_off[K] + t]) : A::neg(sNu[t]);
    __syncthreads();
    if (adjoint) {
      // transposed local system (Sec. 4.2): A^T against [C^T | F~],
      // C^T[(f,i), (a,g,l)] = alpha |e_a| <psi_l, phi_i> delta_fg
      for (int t = tid; t < N * N; t += NT) {
        const int i = t / N, j = t - i * N;
        if (i < j) {
          const T v = sA[i * LDA + j];
          sA[i * LDA + j] = sA[j * LDA + i];
          sA[j * LDA + i] = v;
        }
      }
      for (int r = ty; r < N; r += NW) {
        const int f = r / NP, i = r - f * NP;
        for (int c = tx; c < nt; c += 32) {
          const int a = g_cf[c], g = g_cg[c], l = g_cl[c];
          sR[r * ldr + c] = (g == f) ? sMe[(a * 5 + l) * NP + i] : zero;
        }
      }
      __syncthreads();
    }

    // ---------------- a4/a5: LU with partial pivoting on [A | B | F] ----------------
    const int nr1 = nt + 1;
    if constexpr (LS == 0) {
      lu_solve<T, N, NT>(sA, LDA, sR, ldr, nr1, reinterpret_cast<int*>(scr), s_pinv, &s_bad, tid);  // scratch is dead here
    } else {
      float* fA = reinterpret_cast<float*>(smem + lay.oTc);
      float* fW = fA + N * LDA;
      float* pinv32 = fW + N * ldr;
      int* piv = reinterpret_cast<int*>(pinv32 + N);
      tc_refine_solve<T, N, NT, LS>(sA, LDA, sR, ldr, nr1, smem + lay.oR0, fA, fW, piv, pinv32, s_red,
                                    ph.refine_max, ph.refine_tol, &s_bad, tid);
    }
    // X (column-major n x (nt+1)) and the interior residual; X renormalised in place
    int bad = 0;
    {
      double* xk = s.X + m.x_off[K];
      for (int t = tid; t < N * nr1; t += NT) {
        const int c = t / N, r = t - c * N;
        const T v = A::norm(sR[r * ldr + c]);
        sR[r * ldr + c] = v;
        xk[t] = A::to_d(v);
        bad |= A::bad(v);
      }
      double* ru = s.res_u + m.u_off[K];
      for (int t = tid; t < N; t += NT) ru[t] = A::to_d(sNu[t]);
    }
    __syncthreads();
    if (adjoint) {  // the adjoint needs only the local solves
      if (bad) atomicOr(&s_bad, 2);
      __syncthreads();
      if (tid == 0) s.status[K] = (s_bad & 1) ? 1 : ((s_bad & 2) ? 2 : ((s_bad & 4) ? 3 : 0));
      continue;
    }

    // ---------------- a6/a7: Schur complement, E_K, assembly ----------------
    // the (row, column) pairs -- rows (face a; f, k), columns (face b; g, l | E) -- flattened
    // over the CTA, two per thread (independent chains, full warps)
    {
      const int cnt = nt * nr1;
      for (int e0 = tid; e0 < cnt; e0 += 2 * NT) {
        T v[2];
        int rr[2], cc[2];
        const bool two = e0 + NT < cnt;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int e = (u == 1 && two) ? e0 + NT : e0;
          const int r = e / nr1, c = e - r * nr1;
          rr[u] = r;
          cc[u] = c;
          const int a = g_cf[r], rl = r - g_toff[a];
          if (c == nt) {
            v[u] = sEh[r];
          } else {
            const int b = g_cf[c];
            v[u] = (b == a) ? sD[a * DS + rl * 4 * g_nk[b] + c - g_toff[b]] : zero;
          }
        }
        const T* me0 = sMe + (g_cf[rr[0]] * 5 + g_cl[rr[0]]) * NP;
        const T* me1 = sMe + (g_cf[rr[1]] * 5 + g_cl[rr[1]]) * NP;
        const T* x0 = sR + g_cg[rr[0]] * NP * ldr + cc[0];
        const T* x1 = sR + g_cg[rr[1]] * NP * ldr + cc[1];
#pragma unroll
        for (int jj = 0; jj < NP; ++jj) {
          A::msub(v[0], me0[jj], x0[jj * ldr]);
          A::msub(v[1], me1[jj], x1[jj * ldr]);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          if (u == 1 && !two) break;
          const int r = rr[u], c = cc[u], a = g_cf[r], rl = r - g_toff[a];
          const T w = A::norm(v[u]);
          bad |= A::bad(w);
          if (c == nt) {
            sEh[r] = w;
          } else {
            const int b = g_cf[c], cl = c - g_toff[b], m4b = 4 * g_nk[b];
            if (b == a) sD[a * DS + rl * m4b + cl] = w;
            else s.K[m.kblk[9 * (size_t)K + 3 * a + b] + rl * m4b + cl] = A::to_d(w);
          }
        }
      }
    }
    if (bad) atomicOr(&s_bad, 2);
    __syncthreads();
    // two-sided sums: side 0 parks its halves in K/E/res_lam, side 1 in the work space
    for (int a = 0; a < 3; ++a) {
      const int e = g_e[a], m4 = 4 * g_nk[a];
      if (e < 0) continue;  // boundary face
      const int64_t lo = m.lam_off[e];
      double* dd = g_side[a] ? s.dhalf1 + m.dblk_off[e] : s.K + m.kblk[9 * (size_t)K + 4 * a];
      double* de = g_side[a] ? s.ehalf1 + lo : s.E + lo;
      double* dr = g_side[a] ? s.rhalf1 + lo : s.res_lam + lo;
      for (int t = tid; t < m4 * m4; t += NT) dd[t] = A::to_d(sD[a * DS + t]);
      for (int t = tid; t < m4; t += NT) {
        de[t] = A::to_d(sEh[g_toff[a] + t]);
        dr[t] = A::to_d(sNl[g_toff[a] + t]);
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
      if (g_old[a] != 1) continue;  // the other side arrives later and sums
      const int e = g_e[a], m4 = 4 * g_nk[a];
      const int64_t lo = m.lam_off[e];
      double* k0 = s.K + m.kblk[9 * (size_t)K + 4 * a];
      const double* k1 = s.dhalf1 + m.dblk_off[e];
      const int side = g_side[a];
      // sum in binary64, in the fixed order side 0 + side 1
      for (int t = tid; t < m4 * m4; t += NT) {
        const double mine = A::to_d(sD[a * DS + t]);
        const double other = side ? __ldcg(k0 + t) : __ldcg(k1 + t);
        k0[t] = side ? other + mine : mine + other;
      }
      for (int t = tid; t < m4; t += NT) {
        const double me_ = A::to_d(sEh[g_toff[a] + t]), mr = A::to_d(sNl[g_toff[a] + t]);
        const double oe = side ? __ldcg(s.E + lo + t) : __ldcg(s.ehalf1 + lo + t);
        const double orr = side ? __ldcg(s.res_lam + lo + t) : __ldcg(s.rhalf1 + lo + t);
        s.E[lo + t] = side ? oe + me_ : me_ + oe;
        s.res_lam[lo + t] = side ? orr + mr : mr + orr;
      }
      if (tid == 0) s.face_cnt[e] = 0;
    }
    if (tid == 0) s.status[K] = (s_bad & 1) ? 1 : ((s_bad & 2) ? 2 : ((s_bad & 4) ? 3 : 0));
    __syncthreads();
  }
}


template <int P, class T, int LS = 0, bool BATCH = false>
inline bool launch_euler_bucket(const DevMesh& m, const DevSys& s, const Phys& ph, const T* tab, const TabOff& to,
                                const double* U, const double* Lam, const int* elems, int n, int ntmax,
                                cudaStream_t st, std::string* err, const BatchRef& bt = BatchRef{},
                                bool bounded = false) {
  const int ldr = ldr_for(ntmax), nkmax = nkmax_for(P, ntmax, BATCH ? bounded : m.elem_bc != nullptr);
  const EulerLayout<P> lay(ldr, nkmax, LS != 0);
  const size_t bytes = sizeof(T) * (size_t)lay.total;
  const size_t cap = sizeof(T) * (size_t)EulerLayout<P>(ldr_for(kMaxNt), kMaxP + 1, LS != 0).total;
  cudaError_t ce = set_smem_cap(k_condense_euler<P, T, LS, BATCH>, cap, bytes);
  if (ce != cudaSuccess) { *err = cudaGetErrorString(ce); return false; }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_condense_euler<P, T, LS, BATCH>, kCondThreads, bytes);
  if (per_sm < 1) { *err = "condensation kernel does not fit on an SM"; return false; }
  const long grid = condense_grid(ph, P, sms, per_sm, n);
  k_condense_euler<P, T, LS, BATCH><<<(int)grid, kCondThreads, bytes, st>>>(m, s, ph, tab, to, U, Lam, elems, n, ldr,
                                                                         nkmax, bt);
  ce = cudaGetLastError();
  if (ce != cudaSuccess) { *err = cudaGetErrorString(ce); return false; }
  return true;
}

}  // namespace hdg
