// CUDA kernels of the HDG Newton-step hot path (sm_103a).
//
// Steps (arXiv:1308.3995):
//   a1 gather of the element state, traces and affine geometry;
//   a2 volume quadrature: -(grad phi, f_c(w))_K and its Jacobian (Eq. hdg_ls2);
//   a3 face quadrature: <phi, f_hat>_dK (Eq. hdg_ls3) and the element's share
//      of <mu, [[f_hat]]>_e (Eq. hdg_cont) with their Jacobians, numerical flux
//      f_c(lambda).n - alpha (lambda - w) (Sec. 3.2);
//   a4 LU of the local block with partial pivoting;
//   a5 X = A^{-1}[B | F], the local solves stored for reconstruction (Sec. 3.4);
//   a6 S = D - C X_B, E_K = H - C X_F (Eq. hybridsystem, element-wise);
//   a7 assembly into the block-sparse trace matrix;
//   a8 reconstruction dU = X_F - X_B dLambda (Eq. ls).
//
// Precision: IEEE binary64 throughout.  On this part the binary64 pipe is
// about 1/60 of the binary32 one, so the kernels are arranged to spend binary64
// instructions only on the method's arithmetic: full warps in every loop,
// pivots inverted once, no shuffle reductions in binary64.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "hdg_internal.h"

namespace hdg {

// --------------------------------------------------------------------------
// Euler physics (Sec. 2.1): flux f_c = (rho v, rho v (x) v + p Id, v (E + p)),
// p = (gamma - 1)(E - rho |v|^2 / 2), and the flux Jacobians dF_x/dw, dF_y/dw
// (row-major 4x4), derived by hand from those formulas.
// --------------------------------------------------------------------------
__device__ __forceinline__ void euler_flux_jac(const double* w, double gam, double* fx, double* fy, double* Ax,
                                               double* Ay) {
  const double rho = w[0], ir = __drcp_rn(rho), u = w[1] * ir, v = w[2] * ir, E = w[3];
  const double g1 = gam - 1.0;
  const double q2 = u * u + v * v;
  const double p = g1 * (E - 0.5 * rho * q2);
  const double Ep = E + p;
  const double H = Ep * ir;
  const double ph2 = 0.5 * g1 * q2;
  fx[0] = w[1]; fx[1] = w[1] * u + p; fx[2] = w[1] * v; fx[3] = u * Ep;
  fy[0] = w[2]; fy[1] = w[2] * u;     fy[2] = w[2] * v + p; fy[3] = v * Ep;
  Ax[0] = 0.0;            Ax[1] = 1.0;              Ax[2] = 0.0;              Ax[3] = 0.0;
  Ax[4] = ph2 - u * u;    Ax[5] = (3.0 - gam) * u;  Ax[6] = -g1 * v;          Ax[7] = g1;
  Ax[8] = -u * v;         Ax[9] = v;                Ax[10] = u;               Ax[11] = 0.0;
  Ax[12] = u * (ph2 - H); Ax[13] = H - g1 * u * u;  Ax[14] = -g1 * u * v;     Ax[15] = gam * u;
  Ay[0] = 0.0;            Ay[1] = 0.0;              Ay[2] = 1.0;              Ay[3] = 0.0;
  Ay[4] = -u * v;         Ay[5] = v;                Ay[6] = u;                Ay[7] = 0.0;
  Ay[8] = ph2 - v * v;    Ay[9] = -g1 * u;          Ay[10] = (3.0 - gam) * v; Ay[11] = g1;
  Ay[12] = v * (ph2 - H); Ay[13] = -g1 * u * v;     Ay[14] = H - g1 * v * v;  Ay[15] = gam * v;
}

// --------------------------------------------------------------------------
// Bit-level helpers that keep pivot search and finiteness checks off the
// binary64 pipe: for non-negative doubles, IEEE order is the order of the bit
// patterns as unsigned integers.
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long abs_key(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ int not_finite(double v) {
  return (__double2hiint(v) & 0x7ff00000) == 0x7ff00000;
}

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
  HDG_HD EulerLayout(int ldr_, int nkmax) : ldr(ldr_), dstride(16 * nkmax * nkmax) {
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
  }
};

inline int ldr_for(int ntmax) { return (ntmax + 1) | 1; }  // odd leading dimension
// largest single-face trace size in a bucket of degree p: every face has p_e >= p
inline int nkmax_for(int p, int ntmax) {
  int nk = ntmax / 4 - 2 * (p + 1);
  return nk > kMaxP + 1 ? kMaxP + 1 : nk;
}

// --------------------------------------------------------------------------
// Condensation kernel, Euler, binary64: one element per CTA iteration.
// --------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kCondThreads) k_condense_euler_f64(
    DevMesh m, DevSys s, Phys ph, const double* __restrict__ tab, TabOff to, const double* __restrict__ U,
    const double* __restrict__ Lam, const int* __restrict__ elems, int n_elems, int ldr, int nkmax) {
  using L = EulerLayout<P>;
  constexpr int NP = L::NP, NQ = L::NQ, N = L::N, LDA = L::LDA;
  constexpr int NT = kCondThreads;
  extern __shared__ double smem[];
  const L lay(ldr, nkmax);
  const int DS = lay.dstride;
  double* sA = smem + lay.oA;
  double* sR = smem + lay.oR;
  double* sU = smem + lay.oU;
  double* sL = smem + lay.oL;
  double* sNu = smem + lay.oNu;
  double* sNl = smem + lay.oNl;
  double* sEh = smem + lay.oEh;
  double* sMe = smem + lay.oMe;
  double* sD = smem + lay.oD;
  double* scr = smem + lay.oScr;
  // volume scratch
  double* sWq = scr;                  // [4][NQ]
  double* sFh = sWq + 4 * NQ;         // [2][4][NQ]
  double* sAh = sFh + 8 * NQ;         // [2][16][NQ]
  double* sZ = sAh + 32 * NQ;         // [4][NP][NQ]
  // face scratch (aliases the volume scratch)
  double* sFhat = scr;                // [3*6][4]
  double* sW = sFhat + 3 * kPtSlots * 4;  // [3*6][16][5]

  __shared__ double g_det, g_Ji[2][2], g_n[3][2], g_len[3], g_mt;
  __shared__ int g_e[3], g_pe[3], g_nk[3], g_toff[4], g_fl[3], g_side[3], g_old[3];
  __shared__ double s_pinv[64];
  __shared__ int s_piv, s_bad;

  const int tid = threadIdx.x;
  const double* vw = tab + to.vol_w[P];
  const double* vphi = tab + to.vol_phi[P];
  const double* vgx = tab + to.vol_gxi[P];
  const double* vge = tab + to.vol_geta[P];
  const double* dref = tab + to.vol_dref[P];
  const double alpha = ph.alpha;
  const double g1 = ph.gamma - 1.0;

  for (int it = blockIdx.x; it < n_elems; it += gridDim.x) {
    const int K = elems[it];
    // ---------------- a1: geometry, faces, state ----------------
    if (tid < 3) {  // one lane per local face, one warp instruction for all three
      const double* c = m.xy + 6 * (size_t)K;
      const int a = tid, b = (tid + 1) % 3;
      const double dx = c[2 * b] - c[2 * a], dy = c[2 * b + 1] - c[2 * a + 1];
      const double len = sqrt(dx * dx + dy * dy);
      const double il = __drcp_rn(len);
      g_len[a] = len;
      g_n[a][0] = dy * il;
      g_n[a][1] = -dx * il;
      const int e = m.elem_face[3 * (size_t)K + a];
      const int info = m.elem_info[K];
      g_e[a] = e;
      g_pe[a] = m.face_p[e];
      g_nk[a] = g_pe[a] + 1;
      g_fl[a] = (info >> a) & 1;
      g_side[a] = (info >> (3 + a)) & 1;
      if (tid == 0) {
        const double J00 = c[2] - c[0], J01 = c[4] - c[0], J10 = c[3] - c[1], J11 = c[5] - c[1];
        const double det = J00 * J11 - J01 * J10;
        const double inv = __drcp_rn(det);
        g_det = det;
        g_Ji[0][0] = J11 * inv; g_Ji[0][1] = -J01 * inv;
        g_Ji[1][0] = -J10 * inv; g_Ji[1][1] = J00 * inv;
        s_bad = 0;
      }
    }
    __syncthreads();
    if (tid == 0) {
      g_toff[0] = 0;
      g_toff[1] = 4 * g_nk[0];
      g_toff[2] = 4 * (g_nk[0] + g_nk[1]);
      g_toff[3] = 4 * (g_nk[0] + g_nk[1] + g_nk[2]);
      // pseudo-time mass det(J)/dt_K (Sec. 3.3), from the element-mean state
      g_mt = 0.0;
      if (ph.cfl > 0.0) {
        const double* u0 = U + m.u_off[K];
        const double c0 = 1.4142135623730951;  // value of the constant orthonormal mode
        const double rho = c0 * u0[0], uu = c0 * u0[NP] / rho, vv = c0 * u0[2 * NP] / rho;
        const double E = c0 * u0[3 * NP];
        const double p = g1 * (E - 0.5 * rho * (uu * uu + vv * vv));
        const double perim = g_len[0] + g_len[1] + g_len[2];
        const double lam_c = (sqrt(uu * uu + vv * vv) + sqrt(ph.gamma * p / rho)) * perim;
        const double dt = ph.cfl * 0.5 * g_det / lam_c;
        g_mt = g_det / dt;
      }
    }
    __syncthreads();
    const int nt = g_toff[3];
    {
      const double* uk = U + m.u_off[K];
      for (int t = tid; t < N; t += NT) sU[t] = uk[t];
      for (int a = 0; a < 3; ++a) {
        const double* lk = Lam + m.lam_off[g_e[a]];
        for (int t = tid; t < 4 * g_nk[a]; t += NT) sL[g_toff[a] + t] = lk[t];
      }
    }
    __syncthreads();

    // ---------------- a2: volume quadrature ----------------
    for (int t = tid; t < 4 * NQ; t += NT) {
      const int f = t / NQ, q = t - f * NQ;
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < NP; ++j) acc += sU[f * NP + j] * vphi[q * NP + j];
      sWq[t] = acc;
    }
    __syncthreads();
    for (int q = tid; q < NQ; q += NT) {
      double w[4], fx[4], fy[4], Ax[16], Ay[16];
#pragma unroll
      for (int f = 0; f < 4; ++f) w[f] = sWq[f * NQ + q];
      euler_flux_jac(w, ph.gamma, fx, fy, Ax, Ay);
      const double c = vw[q] * g_det;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const double a0 = c * g_Ji[r][0], a1 = c * g_Ji[r][1];
#pragma unroll
        for (int f = 0; f < 4; ++f) sFh[(r * 4 + f) * NQ + q] = a0 * fx[f] + a1 * fy[f];
        // rows 1..3 only: row 0 of both flux Jacobians is constant
#pragma unroll
        for (int fg = 4; fg < 16; ++fg) sAh[(r * 16 + fg) * NQ + q] = a0 * Ax[fg] + a1 * Ay[fg];
      }
    }
    __syncthreads();
    // interior residual, volume part: N_w = -(grad phi, f_c(w))_K
    for (int t = tid; t < N; t += NT) {
      const int f = t / NP, i = t - f * NP;
      double acc = 0.0;
      for (int q = 0; q < NQ; ++q) {
        acc -= vgx[q * NP + i] * sFh[f * NQ + q];
        acc -= vge[q * NP + i] * sFh[(4 + f) * NQ + q];
      }
      sNu[t] = acc;
    }
    // volume Jacobian A_fg = -sum_k (dF_k/dw)_fg D_k.  Blocks whose flux-Jacobian
    // entries are constants (row 0: (0,1) = -D_x, (0,2) = -D_y, (0,0) = (0,3) = 0;
    // (1,3) = -(gamma-1) D_x; (2,3) = -(gamma-1) D_y) use D_k = det J sum_r Ji[r][k] Dref_r.
    for (int t = tid; t < NP * NP; t += NT) {
      const int i = t / NP, j = t - i * NP;
      const double d0 = dref[t], d1 = dref[NP * NP + t];
      const double Dx = g_det * (g_Ji[0][0] * d0 + g_Ji[1][0] * d1);
      const double Dy = g_det * (g_Ji[0][1] * d0 + g_Ji[1][1] * d1);
      double* a0 = sA + i * LDA + j;  // block row 0
      a0[0] = 0.0;
      a0[NP] = -Dx;
      a0[2 * NP] = -Dy;
      a0[3 * NP] = 0.0;
      sA[(NP + i) * LDA + 3 * NP + j] = -g1 * Dx;
      sA[(2 * NP + i) * LDA + 3 * NP + j] = -g1 * Dy;
    }
    // state-dependent blocks, one block row f = 1..3 at a time (row 3 has four):
    //   Z_g[i][q] = sum_r dphi_i/dxi_r (q) Ahat_r,fg(q);  A_fg[i][j] = -sum_q Z_g[i][q] phi_j(q)
    for (int f = 1; f < 4; ++f) {
      const int ng = (f == 3) ? 4 : 3;
      for (int t = tid; t < ng * NP * NQ; t += NT) {
        const int g = t / (NP * NQ), rem = t - g * NP * NQ, i = rem / NQ, q = rem - i * NQ;
        sZ[t] = vgx[q * NP + i] * sAh[(f * 4 + g) * NQ + q] + vge[q * NP + i] * sAh[(16 + f * 4 + g) * NQ + q];
      }
      __syncthreads();
      for (int t = tid; t < ng * NP * NP; t += NT) {
        const int g = t / (NP * NP), rem = t - g * NP * NP, i = rem / NP, j = rem - i * NP;
        const double* z = sZ + (g * NP + i) * NQ;
        double acc = 0.0;
#pragma unroll 5
        for (int q = 0; q < NQ; ++q) acc -= z[q] * vphi[q * NP + j];
        sA[(f * NP + i) * LDA + g * NP + j] = acc;
      }
      __syncthreads();
    }

    // ---------------- a3: face quadrature ----------------
    for (int t = tid; t < 3 * kPtSlots; t += NT) {
      const int a = t / kPtSlots, g = t - a * kPtSlots;
      const int pe = g_pe[a], nk = pe + 1;
      if (g < pe + 2) {
        const double* phe = tab + to.edge_phi[P][pe][a][g_fl[a]] + g * NP;
        const double* ps = tab + to.edge_psi[pe] + g * nk;
        const double we = tab[to.edge_w[pe] + g] * g_len[a];
        double w[4], lam[4], fx[4], fy[4], Ax[16], Ay[16];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          double acc = 0.0;
#pragma unroll
          for (int j = 0; j < NP; ++j) acc += sU[f * NP + j] * phe[j];
          w[f] = acc;
          double al = 0.0;
          for (int k = 0; k < nk; ++k) al += sL[g_toff[a] + f * nk + k] * ps[k];
          lam[f] = al;
        }
        euler_flux_jac(lam, ph.gamma, fx, fy, Ax, Ay);
        const double nx = g_n[a][0], ny = g_n[a][1];
#pragma unroll
        for (int f = 0; f < 4; ++f) sFhat[t * 4 + f] = we * (nx * fx[f] + ny * fy[f] - alpha * (lam[f] - w[f]));
#pragma unroll
        for (int fg = 0; fg < 16; ++fg) {
          const double at = we * (nx * Ax[fg] + ny * Ay[fg] - ((fg % 5 == 0) ? alpha : 0.0));
          for (int l = 0; l < nk; ++l) sW[(t * 16 + fg) * 5 + l] = at * ps[l];
        }
      }
    }
    __syncthreads();
    // B = d N_w / d Lambda: rows (f,i), columns (face a; g, l)
    for (int t = tid; t < N * nt; t += NT) {
      const int r = t / nt, c = t - r * nt;
      const int f = r / NP, i = r - f * NP;
      const int a = (c >= g_toff[2]) ? 2 : (c >= g_toff[1] ? 1 : 0);
      const int nk = g_nk[a], cl = c - g_toff[a], g = cl / nk, l = cl - g * nk;
      const double* phe = tab + to.edge_phi[P][g_pe[a]][a][g_fl[a]];
      double acc = 0.0;
      for (int q = 0; q < nk + 1; ++q) acc += phe[q * NP + i] * sW[((a * kPtSlots + q) * 16 + f * 4 + g) * 5 + l];
      sR[r * ldr + c] = acc;
    }
    // D_a = d N_lambda,a / d Lambda_a (block diagonal in faces)
    for (int a = 0; a < 3; ++a) {
      const int nk = g_nk[a], m4 = 4 * nk;
      const double* ps = tab + to.edge_psi[g_pe[a]];
      for (int t = tid; t < m4 * m4; t += NT) {
        const int r = t / m4, c = t - r * m4, f = r / nk, k = r - f * nk, g = c / nk, l = c - g * nk;
        double acc = 0.0;
        for (int q = 0; q < nk + 1; ++q) acc += ps[q * nk + k] * sW[((a * kPtSlots + q) * 16 + f * 4 + g) * 5 + l];
        sD[a * DS + t] = acc;
      }
    }
    // C_a = alpha |e_a| <psi_k, phi_j> delta_fg, kept as the scalar edge matrix
    for (int t = tid; t < 3 * 5 * NP; t += NT) {
      const int a = t / (5 * NP), rem = t - a * 5 * NP, k = rem / NP;
      if (k < g_nk[a]) sMe[t] = alpha * g_len[a] * tab[to.edge_cross[P][g_pe[a]][a][g_fl[a]] + rem];
    }
    // face parts of the residuals
    for (int t = tid; t < N; t += NT) {
      const int f = t / NP, i = t - f * NP;
      double acc = 0.0;
      for (int a = 0; a < 3; ++a) {
        const double* phe = tab + to.edge_phi[P][g_pe[a]][a][g_fl[a]];
        for (int q = 0; q < g_pe[a] + 2; ++q) acc += phe[q * NP + i] * sFhat[(a * kPtSlots + q) * 4 + f];
      }
      sNu[t] += acc;
    }
    for (int t = tid; t < nt; t += NT) {
      const int a = (t >= g_toff[2]) ? 2 : (t >= g_toff[1] ? 1 : 0);
      const int nk = g_nk[a], tl = t - g_toff[a], f = tl / nk, k = tl - f * nk;
      const double* ps = tab + to.edge_psi[g_pe[a]];
      double acc = 0.0;
      for (int q = 0; q < nk + 1; ++q) acc += ps[q * nk + k] * sFhat[(a * kPtSlots + q) * 4 + f];
      sNl[t] = acc;
      sEh[t] = -acc;  // H
    }
    __syncthreads();
    // face mass alpha <phi_i, phi_j>_dK on every field's diagonal block, plus the pseudo-time mass
    for (int t = tid; t < NP * NP; t += NT) {
      const int i = t / NP, j = t - i * NP;
      double v = 0.0;
      for (int a = 0; a < 3; ++a) v += g_len[a] * tab[to.face_mass[P][g_pe[a]][a] + t];
      v = alpha * v + ((i == j) ? g_mt : 0.0);
#pragma unroll
      for (int f = 0; f < 4; ++f) sA[(f * NP + i) * LDA + f * NP + j] += v;
    }
    for (int t = tid; t < N; t += NT) sR[t * ldr + nt] = -sNu[t];  // F
    __syncthreads();

    // ---------------- a4/a5: LU with partial pivoting on [A | B | F] ----------------
    const int nr1 = nt + 1;
    for (int k = 0; k < N; ++k) {
      if (tid < 32) {
        unsigned long long best = 0ull;
        int bi = k;
        for (int i = k + tid; i < N; i += 32) {
          const unsigned long long v = abs_key(sA[i * LDA + k]);
          if (v > best) { best = v; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const unsigned long long ob = __shfl_down_sync(0xffffffffu, best, o);
          const int oi = __shfl_down_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (tid == 0) {
          s_piv = bi;
          if (best == 0ull) { s_bad |= 1; s_pinv[k] = 0.0; } else { s_pinv[k] = __drcp_rn(sA[bi * LDA + k]); }
        }
      }
      __syncthreads();
      // swap rows k and piv (columns k..N-1 of A and all of [B|F]); scale the new row k by 1/pivot
      {
        const int piv = s_piv;
        const double pinv = s_pinv[k];
        const int wa = N - k;
        for (int t = tid; t < wa + nr1; t += NT) {
          double* pk = (t < wa) ? &sA[k * LDA + k + t] : &sR[k * ldr + (t - wa)];
          double* pp = (t < wa) ? &sA[piv * LDA + k + t] : &sR[piv * ldr + (t - wa)];
          const double vk = *pk, vp = *pp;
          if (piv != k) *pp = vk;
          *pk = vp * pinv;
        }
      }
      __syncthreads();
      {
        const int nr = N - k - 1, wa = N - k - 1, nc = wa + nr1;
        for (int t = tid; t < nr * nc; t += NT) {
          const int ii = t / nc, c = t - ii * nc, i = k + 1 + ii;
          const double l = sA[i * LDA + k];
          if (c < wa) sA[i * LDA + k + 1 + c] -= l * sA[k * LDA + k + 1 + c];
          else sR[i * ldr + (c - wa)] -= l * sR[k * ldr + (c - wa)];
        }
      }
      __syncthreads();
    }
    // back substitution with the unit upper triangle
    for (int k = N - 1; k > 0; --k) {
      for (int t = tid; t < k * nr1; t += NT) {
        const int i = t / nr1, c = t - i * nr1;
        sR[i * ldr + c] -= sA[i * LDA + k] * sR[k * ldr + c];
      }
      __syncthreads();
    }

    // ---------------- a6/a7: Schur complement, E_K, assembly ----------------
    int bad = 0;
    for (int t = tid; t < nt * nr1; t += NT) {
      const int r = t / nr1, c = t - r * nr1;
      const int a = (r >= g_toff[2]) ? 2 : (r >= g_toff[1] ? 1 : 0);
      const int nka = g_nk[a], rl = r - g_toff[a], f = rl / nka, k = rl - f * nka;
      const double* me = sMe + (a * 5 + k) * NP;
      if (c == nt) {
        double v = sEh[r];
#pragma unroll
        for (int j = 0; j < NP; ++j) v -= me[j] * sR[(f * NP + j) * ldr + c];
        sEh[r] = v;
        bad |= not_finite(v);
      } else {
        const int b = (c >= g_toff[2]) ? 2 : (c >= g_toff[1] ? 1 : 0);
        const int cl = c - g_toff[b], m4b = 4 * g_nk[b];
        double v = (b == a) ? sD[a * DS + rl * m4b + cl] : 0.0;
#pragma unroll
        for (int j = 0; j < NP; ++j) v -= me[j] * sR[(f * NP + j) * ldr + c];
        if (b == a) sD[a * DS + rl * m4b + cl] = v;
        else s.K[m.kblk[9 * (size_t)K + 3 * a + b] + rl * m4b + cl] = v;
        bad |= not_finite(v);
      }
    }
    // X (column-major n x (nt+1)) and the interior residual
    {
      double* xk = s.X + m.x_off[K];
      for (int t = tid; t < N * nr1; t += NT) {
        const int c = t / N, r = t - c * N;
        const double v = sR[r * ldr + c];
        xk[t] = v;
        bad |= not_finite(v);
      }
      double* ru = s.res_u + m.u_off[K];
      for (int t = tid; t < N; t += NT) ru[t] = sNu[t];
    }
    if (bad) atomicOr(&s_bad, 2);
    __syncthreads();
    // two-sided sums: side 0 parks its halves in K/E/res_lam, side 1 in the work space
    for (int a = 0; a < 3; ++a) {
      const int e = g_e[a], m4 = 4 * g_nk[a];
      const int64_t lo = m.lam_off[e];
      double* dd = g_side[a] ? s.dhalf1 + m.dblk_off[e] : s.K + m.kblk[9 * (size_t)K + 4 * a];
      double* de = g_side[a] ? s.ehalf1 + lo : s.E + lo;
      double* dr = g_side[a] ? s.rhalf1 + lo : s.res_lam + lo;
      for (int t = tid; t < m4 * m4; t += NT) dd[t] = sD[a * DS + t];
      for (int t = tid; t < m4; t += NT) { de[t] = sEh[g_toff[a] + t]; dr[t] = sNl[g_toff[a] + t]; }
    }
    __threadfence();
    __syncthreads();
    if (tid < 3) {
      g_old[tid] = atomicAdd(&s.face_cnt[g_e[tid]], 1);
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
      // sum in the fixed order side 0 + side 1
      for (int t = tid; t < m4 * m4; t += NT) {
        const double mine = sD[a * DS + t];
        const double other = side ? __ldcg(k0 + t) : __ldcg(k1 + t);
        k0[t] = side ? other + mine : mine + other;
      }
      for (int t = tid; t < m4; t += NT) {
        const double me_ = sEh[g_toff[a] + t], mr = sNl[g_toff[a] + t];
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

// --------------------------------------------------------------------------
// Reconstruction, Eq. (ls): dU_K = X_F - X_B dLambda_K.  One thread per
// (element, interior row); X is column-major per element, so the rows of one
// element are contiguous for every column and each warp load is coalesced.
// --------------------------------------------------------------------------
__global__ void k_recover_f64(DevMesh m, const double* __restrict__ X, const double* __restrict__ dLam,
                              double* __restrict__ dU, const int* __restrict__ elems, int n_elems, int n) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n_elems * n) return;
  const int e = (int)(idx / n), r = (int)(idx - (int64_t)e * n);
  const int K = elems[e];
  const double* xk = X + m.x_off[K];
  int c = 0;
  double acc = 0.0;
  for (int a = 0; a < 3; ++a) {
    const int f = m.elem_face[3 * (size_t)K + a];
    const int len = 4 * (m.face_p[f] + 1);
    const double* dl = dLam + m.lam_off[f];
    for (int t = 0; t < len; ++t, ++c) acc += xk[(size_t)c * n + r] * dl[t];
  }
  dU[m.u_off[K] + r] = xk[(size_t)c * n + r] - acc;
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------
template <int P>
static bool launch_euler_bucket(const DevMesh& m, const DevSys& s, const Phys& ph, const double* tab,
                                const TabOff& to, const double* U, const double* Lam, const int* elems, int n,
                                int ntmax, cudaStream_t st, std::string* err) {
  const int ldr = ldr_for(ntmax), nkmax = nkmax_for(P, ntmax);
  const EulerLayout<P> lay(ldr, nkmax);
  const size_t bytes = sizeof(double) * (size_t)lay.total;
  cudaError_t ce = cudaFuncSetAttribute(k_condense_euler_f64<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)bytes);
  if (ce != cudaSuccess) { *err = cudaGetErrorString(ce); return false; }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_condense_euler_f64<P>, kCondThreads, bytes);
  if (per_sm < 1) { *err = "condensation kernel does not fit on an SM"; return false; }
  long grid = (long)sms * per_sm;
  if (grid > n) grid = n;
  k_condense_euler_f64<P><<<(int)grid, kCondThreads, bytes, st>>>(m, s, ph, tab, to, U, Lam, elems, n, ldr, nkmax);
  ce = cudaGetLastError();
  if (ce != cudaSuccess) { *err = cudaGetErrorString(ce); return false; }
  return true;
}

int launch_condense(const DevMesh& m, const DevSys& s, const Phys& ph, const double* tab, const TabOff& to,
                    const double* U, const double* Lam, const int* const* bucket, const int* bucket_n,
                    const int* bucket_ntmax, void* stream, std::string* err) {
  cudaStream_t st = (cudaStream_t)stream;
  int launches = 0;
  for (int p = 1; p <= kMaxP; ++p) {
    if (bucket_n[p] == 0) continue;
    bool ok = false;
    if (ph.model != 0) { *err = "model not supported by this kernel set"; return -1; }
    switch (p) {
      case 1: ok = launch_euler_bucket<1>(m, s, ph, tab, to, U, Lam, bucket[p], bucket_n[p], bucket_ntmax[p], st, err); break;
      case 2: ok = launch_euler_bucket<2>(m, s, ph, tab, to, U, Lam, bucket[p], bucket_n[p], bucket_ntmax[p], st, err); break;
      case 3: ok = launch_euler_bucket<3>(m, s, ph, tab, to, U, Lam, bucket[p], bucket_n[p], bucket_ntmax[p], st, err); break;
      case 4: ok = launch_euler_bucket<4>(m, s, ph, tab, to, U, Lam, bucket[p], bucket_n[p], bucket_ntmax[p], st, err); break;
    }
    if (!ok) return -1;
    ++launches;
  }
  return launches;
}

int launch_recover_buckets(const DevMesh& m, const double* X, const double* dLam, double* dU,
                           const int* const* bucket, const int* bucket_n, void* stream, std::string* err) {
  cudaStream_t st = (cudaStream_t)stream;
  int launches = 0;
  for (int p = 1; p <= kMaxP; ++p) {
    if (bucket_n[p] == 0) continue;
    const int n = m.nfield * n_basis(p);
    const int64_t total = (int64_t)bucket_n[p] * n;
    const int threads = 256;
    const int64_t grid = (total + threads - 1) / threads;
    k_recover_f64<<<(unsigned)grid, threads, 0, st>>>(m, X, dLam, dU, bucket[p], bucket_n[p], n);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) { *err = cudaGetErrorString(ce); return -1; }
    ++launches;
  }
  return launches;
}

}  // namespace hdg
