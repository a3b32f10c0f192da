// Global trace solve K dLambda = E (paper Sec. 3.4, Eq. hybridsystem) and the
// pseudo-transient Newton update (Sec. 3.3) on the GPU.
//
// The paper uses ILU(n)-preconditioned GMRES from PETSc on the CPU.  Here:
// restarted GMRES, left-preconditioned, with one of
//   0 block Jacobi (the inverses of K's diagonal face blocks),
//   1 multicolor block symmetric Gauss-Seidel,
//   2 block ILU(0) in the multicolor order of the faces (faces of one color
//     share no element, so their rows are uncoupled: each color is factored,
//     and swept in the triangular solves, by one launch),
//   3 the same with binary32 factors,
// and one of two arithmetics for the products and Krylov updates:
//   0 binary64 (the FP64 pipe), vectors in binary64;
//   1 double-word (float-float) arithmetic on the binary32 pipe, on a
//     float-float copy of K (and of the factors) made once per solve, vectors
//     stored as float-float pairs in the same 8 bytes per value.
// Kernels:
//   k_bj_invert   one warp per face: Gauss-Jordan with partial pivoting of the
//                 face's diagonal block (m = 4 (p_e + 1) <= 20 rows);
//   k_ilu_row     one warp per face of one color: the face's block row of the
//                 incomplete factors, then the inverse of its pivot block;
//   k_face_op     one warp per face: t = (K x)_e (each block staged through
//   (_ff)         shared memory with coalesced loads, the five blocks of the
//                 face row in column order; optionally only the blocks of
//                 earlier or of later colors), then, by mode, y_e = t,
//                 Dinv_e t, Dinv_e (b_e - t), Dinv_e b_e or b_e - t;
//   hdg_krylov.cuh  the Arnoldi process as delayed classical Gram-Schmidt
//                 with re-orthogonalisation: per iteration one reduction
//                 pass and one update pass over the basis (the Hessenberg
//                 column, its Givens rotation and the residual estimate in
//                 an extra block of the update launch); the triangular
//                 least-squares solve k_lsq and x += V y, all on the device
//                 (the state is read back once per chunk of iterations).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "hdg_arith.cuh"
#include "hdg_internal.h"
#include "hdg_krylov.cuh"
#include "hdg_objects.h"

using namespace hdg;
using namespace hdg::krylov;

namespace {

constexpr int kFaceWarps = 4;          // faces per CTA in the per-face kernels
constexpr int kMaxM = 4 * (kMaxP + 1);  // largest face block (20)
constexpr int kDotChunk = 8;           // vectors per k_dots block row

// MT: value type of the stored matrix and pivot inverses (binary64, or binary32
// for the mixed-precision ILU(0) factors; products always run in binary64)
template <class MT>
struct FaceDevT {
  int n_face;
  const int* face_p;
  const int64_t* lam_off;
  const int* k_col;         // [5 n_face]
  const int64_t* k_blkoff;  // [5 n_face + 1]
  const int64_t* dinv_off;  // [n_face]
  const int64_t* k_tblk;    // [5 n_face]: offset of block (k_col[5e+b], e), for products with K^T
  const int* fcolor;        // [n_face] color of each face in the multicolor order
  const MT* K;              // the matrix (K, or the incomplete factors of the ILU preconditioner)
  MT* dinv;
  int* bad;                 // set to 1 if a diagonal block is singular
};
using FaceDev = FaceDevT<double>;

// Lane order of the double-word face operator's matrix copies: a face with m
// rows splits a warp into nseg segments (32 / m rounded down to a power of
// two); lane r + m sg takes row r and the columns sg, sg + nseg, ...; entry
// (r, c) of one of its blocks sits at lane_order(r, c, m) within the block.
__host__ __device__ __forceinline__ int lane_segments(int m) { return m <= 8 ? 4 : (m <= 16 ? 2 : 1); }
__host__ __device__ __forceinline__ int64_t lane_order(int r, int c, int m) {
  const int ns = lane_segments(m);
  return (int64_t)(c / ns) * (m * ns) + r + m * (c % ns);
}

// ---------------------------------------------------------------- block Jacobi
// Gauss-Jordan inversion with partial pivoting (largest |a_rk|, first on ties)
// of the m x m block in the left half of a (the identity in the right half);
// the inverse is left in columns m .. 2m-1.  One warp, m <= 32; false if the
// block is singular (the result is then warp-uniform).
template <class VT>
__device__ bool warp_gj_invert(VT (*a)[2 * kMaxM + 1], int m, int lane) {
  const int m2 = 2 * m;
  for (int k = 0; k < m; ++k) {
    VT best = (lane >= k && lane < m) ? (VT)fabs(a[lane][k]) : (VT)-1.0;
    int bi = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const VT ob = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    best = __shfl_sync(0xffffffffu, best, 0);
    bi = __shfl_sync(0xffffffffu, bi, 0);
    if (!(best > (VT)0)) return false;
    for (int c = lane; c < m2; c += 32) {
      const VT t = a[k][c];
      a[k][c] = a[bi][c];
      a[bi][c] = t;
    }
    __syncwarp();
    const VT pinv = (VT)1 / a[k][k];
    __syncwarp();
    for (int c = lane; c < m2; c += 32) a[k][c] *= pinv;
    __syncwarp();
    VT fr[kMaxM];
#pragma unroll
    for (int r = 0; r < kMaxM; ++r) fr[r] = (r < m) ? a[r][k] : (VT)0;
    __syncwarp();
    for (int c = lane; c < m2; c += 32) {
      const VT akc = a[k][c];
#pragma unroll
      for (int r = 0; r < kMaxM; ++r)
        if (r < m && r != k) a[r][c] = fma(-fr[r], akc, a[r][c]);
    }
    __syncwarp();
  }
  return true;
}

template <class VT, class DT>
__device__ void load_aug(VT (*a)[2 * kMaxM + 1], const DT* D, int m, int lane) {
  const int m2 = 2 * m;
  for (int t = lane; t < m * m2; t += 32) {
    const int r = t / m2, c = t - r * m2;
    a[r][c] = (c < m) ? (VT)D[r * m + c] : (c - m == r ? (VT)1 : (VT)0);
  }
  __syncwarp();
}

__device__ __forceinline__ double out_value(double v, double*) { return v; }
__device__ __forceinline__ float out_value(float v, float*) { return v; }
__device__ __forceinline__ float2 out_value(float v, float2*) { return make_float2(v, 0.0f); }

// order: -1 row-major; 0 the lane order of k_face_op_ff; 1 the lane order of the transpose
template <class VT, class OT>
__device__ void store_inverse(VT (*a)[2 * kMaxM + 1], OT* out, int m, int lane, int order = -1) {
  for (int t = lane; t < m * m; t += 32) {
    const int r = t / m, c = t - r * m;
    const int64_t at = order < 0 ? t : (order == 0 ? lane_order(r, c, m) : lane_order(c, r, m));
    out[at] = out_value(a[r][m + c], out);
  }
}

// VT: arithmetic of the inversion, OT: the stored inverses (dinv, at
// f.dinv_off, in the given order).  binary64, row-major, for the binary64
// solve; binary32 arithmetic stored as float-float pairs (lo = 0) in the lane
// order of k_face_op_ff for the double-word solve, whose preconditioner is
// then a fixed binary32 operator (it changes the iteration's convergence
// rate, not the system solved).
template <class VT, class OT>
__global__ void __launch_bounds__(32 * kFaceWarps) k_bj_invert(FaceDev f, OT* dinv, int order) {
  __shared__ VT s_aug[kFaceWarps][kMaxM][2 * kMaxM + 1];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * kFaceWarps + w;
  if (e >= f.n_face) return;
  const int m = 4 * (f.face_p[e] + 1);
  int b = 0;
  while (b < 4 && f.k_col[5 * e + b] != e) ++b;
  VT(*a)[2 * kMaxM + 1] = s_aug[w];
  load_aug(a, f.K + f.k_blkoff[5 * e + b], m, lane);
  if (!warp_gj_invert(a, m, lane)) {
    if (lane == 0) *f.bad = 1;
    return;  // the whole warp leaves together
  }
  store_inverse(a, dinv + f.dinv_off[e], m, lane, order);
}

// ---------------------------------------------------------------- block ILU(0)
// One block row of the incomplete factorization per warp, for the faces of one
// color (rows of earlier colors are final; rows of one color share no block).
// F holds K's values before the first color.  For the faces k of earlier
// colors in row e, in ascending color: L_ek = F_ek U_kk^{-1}, then
// F_ej -= L_ek F_kj for every block (e, j) whose (k, j) is in the pattern and
// whose j comes after k (fill outside the pattern is dropped).  Last, the
// inverse of the modified pivot block F_ee goes to dinv.  Same-color faces k
// update disjoint blocks of row e, so the order among them does not matter.
template <class VT>
__global__ void __launch_bounds__(32 * kFaceWarps) k_ilu_row(FaceDevT<VT> f, VT* F, const int* __restrict__ faces,
                                                             int nfaces) {
  __shared__ VT s_aug[kFaceWarps][kMaxM][2 * kMaxM + 1];
  __shared__ VT s_l[kFaceWarps][kMaxM * kMaxM];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ei = blockIdx.x * kFaceWarps + w;
  if (ei >= nfaces) return;
  const int e = faces[ei];
  const int m = 4 * (f.face_p[e] + 1);
  const int ce = f.fcolor[e];
  int lk[4], lb[4], nl = 0, bd = 0;
  for (int b = 0; b < 5; ++b) {
    const int c = f.k_col[5 * e + b];
    if (c < 0) break;
    if (c == e) {
      bd = b;
      continue;
    }
    const int cc = f.fcolor[c];
    if (cc < ce && nl < 4) {  // insertion by ascending color
      int t = nl++;
      while (t > 0 && f.fcolor[lk[t - 1]] > cc) {
        lk[t] = lk[t - 1];
        lb[t] = lb[t - 1];
        --t;
      }
      lk[t] = c;
      lb[t] = b;
    }
  }
  VT* su = &s_aug[w][0][0];           // U_kk^{-1} (mk x mk)
  VT* sf = su + kMaxM * kMaxM;        // F_ek, then F_kj
  VT* sl = s_l[w];                    // L_ek (m x mk)
  for (int t = 0; t < nl; ++t) {
    const int k = lk[t], mk = 4 * (f.face_p[k] + 1), ck = f.fcolor[k];
    VT* Fek = F + f.k_blkoff[5 * e + lb[t]];
    const VT* Uk = f.dinv + f.dinv_off[k];
    for (int i = lane; i < mk * mk; i += 32) su[i] = Uk[i];
    for (int i = lane; i < m * mk; i += 32) sf[i] = Fek[i];
    __syncwarp();
    for (int i = lane; i < m * mk; i += 32) {
      const int r = i / mk, c = i - r * mk;
      VT s = 0;
      for (int q = 0; q < mk; ++q) s = fma(sf[r * mk + q], su[q * mk + c], s);
      sl[i] = s;
      Fek[i] = s;
    }
    __syncwarp();
    for (int b = 0; b < 5; ++b) {
      const int j = f.k_col[5 * e + b];
      if (j < 0) break;
      if (f.fcolor[j] <= ck) continue;  // k itself and faces before it
      int tk = 0;                        // slot of j in row k
      while (tk < 5 && f.k_col[5 * k + tk] != j) ++tk;
      if (tk == 5) continue;             // (k, j) outside the pattern
      const int mj = 4 * (f.face_p[j] + 1);
      const VT* Fkj = F + f.k_blkoff[5 * k + tk];
      VT* Fej = F + f.k_blkoff[5 * e + b];
      for (int i = lane; i < mk * mj; i += 32) sf[i] = Fkj[i];
      __syncwarp();
      for (int i = lane; i < m * mj; i += 32) {
        const int r = i / mj, c = i - r * mj;
        VT s = Fej[i];
        for (int q = 0; q < mk; ++q) s = fma(-sl[r * mk + q], sf[q * mj + c], s);
        Fej[i] = s;
      }
      __syncwarp();
    }
  }
  VT(*a)[2 * kMaxM + 1] = s_aug[w];
  load_aug(a, (const VT*)(F + f.k_blkoff[5 * e + bd]), m, lane);
  if (!warp_gj_invert(a, m, lane)) {
    if (lane == 0) *f.bad = 1;
    return;
  }
  store_inverse(a, f.dinv + f.dinv_off[e], m, lane);
}

// binary64 -> binary32 copy of K's values (the mixed-precision ILU(0) starts from it)
__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __double2float_rn(a[i]);
}

// mode: 0 y = Dinv K x, 1 y = Dinv (b - K x), 2 y = K x, 3 y = Dinv b, 4 y = b - K x.
// faces (may be null): the list of faces to process (one warp each), else all;
// skip_diag: leave the diagonal block out of K x (a Gauss-Seidel sweep over
// one color, in place: x and y may be the same vector, as no two faces of a
// color are coupled); tri: 1 only the blocks of faces of earlier colors, 2
// only those of later colors (the triangular solves of the ILU
// preconditioner, in place over one color as well).
// Each block of the face row is staged through shared memory with coalesced
// loads (the warp reads the m x mb row-major block as one contiguous run; rows
// padded to mb + 1 against bank conflicts).  The products then use every lane
// the face size allows: lane l < m * nseg takes row l % m and every nseg-th
// column from l / m (nseg = 32 / m rounded down to a power of two), and the
// nseg partial sums of a row meet by shuffles.  On this part the binary64 pipe,
// not HBM, bounds a binary64 product of 0.25 flop per byte, so idle lanes
// would cost time directly.
// TR: the same with K^T (block (k_col[5e+b], e) transposed) and Dinv^T.
template <bool TR, bool INPLACE, class MT>
__global__ void __launch_bounds__(32 * kFaceWarps) k_face_op(FaceDevT<MT> f, const double* x,
                                                               const double* __restrict__ bvec, double* y,
                                                               int mode, const int* __restrict__ faces, int nfaces,
                                                               int skip_diag, int tri) {
  __shared__ double s_blk[kFaceWarps][kMaxM * (kMaxM + 1)];
  __shared__ double s_t[kFaceWarps][kMaxM];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ei = blockIdx.x * kFaceWarps + w;
  if (ei >= (faces ? nfaces : f.n_face)) return;
  const int e = faces ? faces[ei] : ei;
  const int m = 4 * (f.face_p[e] + 1);
  const int nseg = (m <= 8) ? 4 : ((m <= 16) ? 2 : 1);
  const int r = lane % m, sg = lane / m;
  const bool act = sg < nseg;
  const int64_t lo = f.lam_off[e];
  const int ce = tri ? f.fcolor[e] : 0;
  double* sb = s_blk[w];
  double t = 0.0;
  if (mode != 3) {
    // metadata of the five slots fetched in parallel, lane b for slot b (one round of
    // dependent loads instead of one per slot): column, its size, block and x offsets
    int mcol = -1, mmb = 0;
    long long moff = 0, mxo = 0;
    if (lane < 5) {
      const int col = f.k_col[5 * e + lane];
      bool ok = col >= 0 && !(skip_diag && col == e);  // unused slots (next to boundary faces) are -1
      if (ok && tri) {
        const int cc = f.fcolor[col];
        ok = (tri == 1) ? cc < ce : cc > ce;
      }
      if (ok) {
        mcol = col;
        mmb = 4 * (f.face_p[col] + 1);
        moff = TR ? f.k_tblk[5 * e + lane] : f.k_blkoff[5 * e + lane];
        mxo = f.lam_off[col];
      }
    }
    for (int b = 0; b < 5; ++b) {
      const int col = __shfl_sync(0xffffffffu, mcol, b);
      if (col < 0) continue;
      const int mb = __shfl_sync(0xffffffffu, mmb, b), n = m * mb;
      // stored block: K (e, col) is m x mb; for K^T, block (col, e) is mb x m
      const MT* blk = f.K + __shfl_sync(0xffffffffu, moff, b);
      const double* xc = x + __shfl_sync(0xffffffffu, mxo, b);
      const int rl = TR ? m : mb, ld = rl + 1;  // stored row length and padded stride
      // (row, column) of entry lane + 32 k, stepped without division
      const int q = 32 / rl, qr = 32 - q * rl;
      int rr = lane / rl, cc = lane - rr * rl;
      for (int idx = lane; idx < n; idx += 32) {
        sb[rr * ld + cc] = (double)__ldcs(blk + idx);  // streamed: each value is used once per product
        rr += q;
        cc += qr;
        if (cc >= rl) { cc -= rl; ++rr; }
      }
      __syncwarp();
      if (act) {
        // in place (a Gauss-Seidel sweep) x is written by this launch: no read-only cache path
        if (TR) {
          for (int c = sg; c < mb; c += nseg) t = fma(sb[c * ld + r], INPLACE ? xc[c] : __ldg(xc + c), t);
        } else {
          const double* row = sb + r * ld;
          for (int c = sg; c < mb; c += nseg) t = fma(row[c], INPLACE ? xc[c] : __ldg(xc + c), t);
        }
      }
      __syncwarp();
    }
  }
  // the nseg partial sums of row r sit in lanes r, r + m, ...
  for (int o = m * (nseg >> 1); o >= m; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (lane < m) {
    if (mode == 1 || mode == 4) t = bvec[lo + lane] - t;
    if (mode == 3) t = bvec[lo + lane];
    s_t[w][lane] = t;
  }
  __syncwarp();
  if (mode == 2 || mode == 4) {
    if (lane < m) y[lo + lane] = t;
    return;
  }
  double v = 0.0;
  if (act) {
    const MT* di = f.dinv + f.dinv_off[e];
    for (int c = sg; c < m; c += nseg) v = fma((double)(TR ? di[c * m + r] : di[r * m + c]), s_t[w][c], v);
  }
  for (int o = m * (nseg >> 1); o >= m; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane < m) y[lo + lane] = v;
}

// ---------------------------------------------------------------- reductions
// partial[j][blockIdx.x] = sum over this block's slice of V_j . w, j in the
// chunk blockIdx.y (vectors V_j at V + j * ldv)
__global__ void __launch_bounds__(kDotThreads) k_multidot(const double* __restrict__ V, int64_t ldv, int nvec,
                                                          const double* __restrict__ w, int64_t n,
                                                          double* __restrict__ partial) {
  __shared__ double s_red[kDotChunk][kDotThreads];
  const int j0 = blockIdx.y * kDotChunk;
  const int nj = min(kDotChunk, nvec - j0);
  double acc[kDotChunk];
#pragma unroll
  for (int j = 0; j < kDotChunk; ++j) acc[j] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kDotThreads) {
    const double wi = __ldg(w + i);
#pragma unroll
    for (int j = 0; j < kDotChunk; ++j)
      if (j < nj) acc[j] = fma(__ldg(V + (int64_t)(j0 + j) * ldv + i), wi, acc[j]);
  }
#pragma unroll
  for (int j = 0; j < kDotChunk; ++j) s_red[j][threadIdx.x] = acc[j];
  __syncthreads();
  for (int s = kDotThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int j = 0; j < kDotChunk; ++j) s_red[j][threadIdx.x] += s_red[j][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < nj) partial[(int64_t)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = s_red[threadIdx.x][0];
}

// out[j] = sum_b partial[j][b] (fixed tree order), one block per j
__global__ void __launch_bounds__(kDotThreads) k_reduce(const double* __restrict__ partial, int nb,
                                                        double* __restrict__ out) {
  __shared__ double s[kDotThreads];
  double a = 0.0;
  for (int b = threadIdx.x; b < nb; b += kDotThreads) a += partial[(int64_t)blockIdx.x * nb + b];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int st = kDotThreads / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = s[0];
}

// ---------------------------------------------------------------- float-float face operator
// k_face_op with every vector stored as float-float pairs (float2: hi, lo) and
// the matrix as the solver's double-word copy of K (or of the ILU factors;
// MT = float2) or its binary32 ILU factors (MT = float), products and sums in
// compensated double-word multiply-adds on the binary32 pipe.
// The copy is stored in lane order: a face with m rows splits its 32 lanes
// into nseg = 32 / m (rounded down to a power of two) segments, lane
// r + m sg taking row r and the columns c = sg, sg + nseg, ...; entry (r, c)
// of each block in the face's row (of K, or of K^T for products with K^T:
// block (col, e) transposed) and of its pivot inverse sits at
// (c / nseg) (m nseg) + r + m (c % nseg) within the block.  Every load of the
// warp is then one contiguous run straight into registers: no staging, no
// index arithmetic.  Relative error of a product ~2^-46 of the magnitudes
// summed.
using AF = Ar<ff>;

__device__ __forceinline__ float2 to_mt(double v, float2*) {
  const ff p = ff_split_double(v);
  return make_float2(p.hi, p.lo);
}
__device__ __forceinline__ float to_mt(float v, float*) { return v; }

__device__ __forceinline__ ff to_ff(float2 v) { return ff{v.x, v.y}; }
__device__ __forceinline__ ff to_ff(float v) { return ff{v, 0.0f}; }
__device__ __forceinline__ ff shfl_down_ff(ff v, int o) {
  return ff{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ float2 from_ff(ff v) { return make_float2(v.hi, v.lo); }

// acc += the lane's share of one block's product: NT = MB / NSEG columns per
// lane (compile-time: every load is a constant offset from one base, issued
// in batches of up to eight before their multiply-adds), two accumulation
// chains.  x of the block's column face is loaded once, one value per lane
// (coalesced), and handed to the lanes that need it by shuffles, so the
// batch's registers hold only the matrix values.
// Every lane of the warp takes part (the shuffles); a lane past the segments
// (sg >= NSEG) loads no matrix value and its sums are never read.
template <int M, int MB, bool INPLACE, class MT>
__device__ __forceinline__ void lane_block_product(const MT* __restrict__ blk, const float2* xcol, int lane, int sg,
                                                   ff& t, ff& t2) {
  constexpr int NSEG = (M <= 8 ? 4 : (M <= 16 ? 2 : 1)), NT = MB / NSEG, MN = M * NSEG, NB = 8;
  const bool act = sg < NSEG;
  // in place (a Gauss-Seidel sweep) x is written by this launch: no read-only cache path
  const float2 xl = lane < MB ? (INPLACE ? xcol[lane] : __ldg(xcol + lane)) : make_float2(0.0f, 0.0f);
#pragma unroll
  for (int k0 = 0; k0 < NT; k0 += NB) {
    MT a[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u)
      if (k0 + u < NT) a[u] = act ? __ldcs(blk + (k0 + u) * MN) : MT{};
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      if (k0 + u < NT) {
        const int c = sg + (k0 + u) * NSEG;
        const ff xv{__shfl_sync(0xffffffffu, xl.x, c), __shfl_sync(0xffffffffu, xl.y, c)};
        AF::madd(((k0 + u) & 1) ? t2 : t, to_ff(a[u]), xv);
      }
    }
  }
}

template <int M, bool TR, bool INPLACE, class MT>
__device__ __forceinline__ void face_op_ff_body(const FaceDevT<MT>& f, const float2* x, const float2* __restrict__ bvec,
                                                float2* y, int mode, int e, int skip_diag, int tri, ff* s_t) {
  constexpr int NSEG = (M <= 8 ? 4 : (M <= 16 ? 2 : 1)), MN = M * NSEG;
  const int lane = threadIdx.x & 31;
  const int sg = lane / M;
  const bool act = sg < NSEG;
  const int64_t lo = f.lam_off[e];
  const int ce = tri ? f.fcolor[e] : 0;
  ff t = AF::zero(), t2 = AF::zero();
  if (mode != 3) {
    int mcol = -1, mmb = 0;
    long long moff = 0, mxo = 0;
    if (lane < 5) {
      const int col = f.k_col[5 * e + lane];
      bool ok = col >= 0 && !(skip_diag && col == e);
      if (ok && tri) {
        const int cc = f.fcolor[col];
        ok = (tri == 1) ? cc < ce : cc > ce;
      }
      if (ok) {
        mcol = col;
        mmb = 4 * (f.face_p[col] + 1);
        moff = TR ? f.k_tblk[5 * e + lane] : f.k_blkoff[5 * e + lane];
        mxo = f.lam_off[col];
      }
    }
    for (int b = 0; b < 5; ++b) {
      const int col = __shfl_sync(0xffffffffu, mcol, b);
      if (col < 0) continue;
      const int mb = __shfl_sync(0xffffffffu, mmb, b);
      const MT* blk = f.K + __shfl_sync(0xffffffffu, moff, b) + lane;
      const float2* xcol = x + __shfl_sync(0xffffffffu, mxo, b);
      // the whole warp takes part (the shuffles); lanes past the segments compute and drop
      switch (mb) {
        case 8: lane_block_product<M, 8, INPLACE>(blk, xcol, lane, sg, t, t2); break;
        case 12: lane_block_product<M, 12, INPLACE>(blk, xcol, lane, sg, t, t2); break;
        case 16: lane_block_product<M, 16, INPLACE>(blk, xcol, lane, sg, t, t2); break;
        default: lane_block_product<M, 20, INPLACE>(blk, xcol, lane, sg, t, t2); break;
      }
    }
  }
  t = AF::add(AF::norm(t), AF::norm(t2));
  // the NSEG partial sums of row r sit in lanes r, r + M, ...
#pragma unroll
  for (int o = M * (NSEG >> 1); o >= M; o >>= 1) t = AF::add(t, shfl_down_ff(t, o));
  if (lane < M) {
    if (mode == 1 || mode == 4) t = AF::sub(to_ff(bvec[lo + lane]), t);
    if (mode == 3) t = AF::norm(to_ff(bvec[lo + lane]));
    s_t[lane] = t;
  }
  __syncwarp();
  if (mode == 2 || mode == 4) {
    if (lane < M) y[lo + lane] = from_ff(t);
    return;
  }
  ff v = AF::zero(), v2 = AF::zero();
  if (act) {  // the pivot inverse (or its transpose) in the same lane order
    constexpr int NT = M / NSEG;
    const MT* di = f.dinv + f.dinv_off[e] + lane;
    MT a[NT];
#pragma unroll
    for (int u = 0; u < NT; ++u) a[u] = __ldg(di + u * MN);
#pragma unroll
    for (int u = 0; u < NT; ++u) AF::madd((u & 1) ? v2 : v, to_ff(a[u]), s_t[sg + u * NSEG]);
  }
  v = AF::add(AF::norm(v), AF::norm(v2));
#pragma unroll
  for (int o = M * (NSEG >> 1); o >= M; o >>= 1) v = AF::add(v, shfl_down_ff(v, o));
  if (lane < M) y[lo + lane] = from_ff(v);
}

template <bool TR, bool INPLACE, class MT>
__global__ void __launch_bounds__(32 * kFaceWarps) k_face_op_ff(FaceDevT<MT> f, const float2* x,
                                                                  const float2* __restrict__ bvec, float2* y,
                                                                  int mode, const int* __restrict__ faces, int nfaces,
                                                                  int skip_diag, int tri) {
  __shared__ ff s_t[kFaceWarps][kMaxM];
  const int w = threadIdx.x >> 5;
  const int ei = blockIdx.x * kFaceWarps + w;
  if (ei >= (faces ? nfaces : f.n_face)) return;
  const int e = faces ? faces[ei] : ei;
  switch (f.face_p[e]) {  // m = 4 (p + 1): the face's rows fix the lane order
    case 1: face_op_ff_body<8, TR, INPLACE>(f, x, bvec, y, mode, e, skip_diag, tri, s_t[w]); break;
    case 2: face_op_ff_body<12, TR, INPLACE>(f, x, bvec, y, mode, e, skip_diag, tri, s_t[w]); break;
    case 3: face_op_ff_body<16, TR, INPLACE>(f, x, bvec, y, mode, e, skip_diag, tri, s_t[w]); break;
    default: face_op_ff_body<20, TR, INPLACE>(f, x, bvec, y, mode, e, skip_diag, tri, s_t[w]); break;
  }
}

// dst = the face blocks of src (K's layout: K, or the ILU factors) converted
// to MT and placed in the lane order of k_face_op_ff, for products with K
// (tr = 0: face e's blocks (e, col)) or with K^T (tr = 1: blocks (col, e)
// transposed).  One warp per face; every stored block is written once.
template <class IT, class MT>
__global__ void __launch_bounds__(32 * kFaceWarps) k_lane_order_blocks(FaceDevT<double> f, const IT* __restrict__ src,
                                                                       MT* __restrict__ dst, int tr) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * kFaceWarps + w;
  if (e >= f.n_face) return;
  const int me = 4 * (f.face_p[e] + 1);
  for (int b = 0; b < 5; ++b) {
    const int col = f.k_col[5 * e + b];
    if (col < 0) continue;
    const int mc = 4 * (f.face_p[col] + 1);
    const int64_t o = tr ? f.k_tblk[5 * e + b] : f.k_blkoff[5 * e + b];
    const int N = tr ? me : mc;  // stored columns (rows: tr ? mc : me)
    for (int idx = lane; idx < me * mc; idx += 32) {
      const int i = idx / N, j = idx - i * N;
      dst[o + (tr ? lane_order(j, i, me) : lane_order(i, j, me))] = to_mt(__ldcs(src + o + idx), (MT*)nullptr);
    }
  }
}

// the same for the pivot inverses (m x m at dinv_off[e]; tr: transposed)
template <class IT, class MT>
__global__ void __launch_bounds__(32 * kFaceWarps) k_lane_order_dinv(FaceDevT<double> f, const IT* __restrict__ src,
                                                                     MT* __restrict__ dst, int tr) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * kFaceWarps + w;
  if (e >= f.n_face) return;
  const int m = 4 * (f.face_p[e] + 1);
  const int64_t o = f.dinv_off[e];
  for (int idx = lane; idx < m * m; idx += 32) {
    const int i = idx / m, j = idx - i * m;
    dst[o + (tr ? lane_order(j, i, m) : lane_order(i, j, m))] = to_mt(__ldcs(src + o + idx), (MT*)nullptr);
  }
}

__global__ void k_axpy2(double* __restrict__ U, const double* __restrict__ dU, int64_t nu, double* __restrict__ L,
                        const double* __restrict__ dL, int64_t nl) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nu + nl; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nu) U[i] += dU[i];
    else L[i - nu] += dL[i - nu];
  }
}

hdg_status fail(hdg_ctx* ctx, hdg_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

int grid_for(int64_t n, int threads, int cap) {
  const int64_t g = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

}  // namespace

struct hdg_solver {
  hdg_sys* sys = nullptr;
  int restart = 0;
  int64_t n = 0;
  int sms = 0;
  int dot_blocks = 0;
  FaceDev f{};
  double* V = nullptr;        // [restart + 1][n] (float-float pairs in the same bytes under arith 1)
  double* partial = nullptr;  // [2 (restart + 1)][dot_blocks] per-block partial sums
  double* gpart = nullptr;    // [2 (restart + 1)][groups] group sums of the two-level finish
  unsigned* ticket = nullptr; // [1 + groups] tickets of the two-level finish (zero between launches)
  double* h = nullptr;        // Arnoldi state (ArnoldiViews)
  double* coef = nullptr;     // [restart + 1] spare
  double* zero = nullptr;     // [n] zeros
  double* tmp = nullptr;      // [n] work vector of the Gauss-Seidel and ILU preconditioners
  double* tmp2 = nullptr;     // [n] second work vector of the ILU preconditioner
  double* hpin = nullptr;     // pinned host mirror of h / coef
  int precond = 0;            // 0 block Jacobi, 1 multicolor block SGS, 2 block ILU(0), 3 ILU(0) in binary32
  int arith = 0;              // GMRES products and Krylov updates: 0 binary64, 1 double-word on the binary32 pipe
  bool factored = false;      // a setup has been enqueued for the current kind
  int* colors = nullptr;      // faces grouped by color
  std::vector<int> color_off; // [n_colors + 1]
  std::vector<int> fcolor;    // host copy of the face colors
  FaceDev fi{};               // the ILU factors: values F (K's layout) and pivot inverses
  double* F = nullptr;
  FaceDevT<float> fi32{};     // the same in binary32 (mixed-precision ILU(0), kind 3)
  float* F32 = nullptr;
  // arith 1: float-float copies of K and its pivot inverses, of the binary64
  // ILU factors, and of the solution and right-hand side of a solve
  FaceDevT<float2> fff{};
  FaceDevT<float2> fiff{};
  FaceDevT<float> fi32ff{};   // kind 3: the binary32 factors in lane order (in fiff's buffers)
  float2* xff = nullptr;      // [n]
  float2* eff = nullptr;      // [n]
  // CUDA graphs of the GMRES chunks, captured on first use: key (chunk start,
  // arithmetic, preconditioner kind, transpose); chunk launches replay them
  cudaStream_t cap = nullptr;
  std::map<long long, cudaGraphExec_t> chunk_graphs;
  bool graphs_off = false;    // a capture failed once: launch directly
  bool external_ws = false;   // device buffers carved from the caller's workspace
  bool hpin_pageable = false; // host mirror from new[] (caller's workspace) or pinned
  int64_t k_vals = 0;         // doubles in K
  int64_t dinv_len = 0;       // doubles in the pivot inverses
  std::vector<void*> allocs;
};

namespace {

hdg_status ck(hdg_ctx* ctx, cudaError_t e, const char* what) {
  if (e != cudaSuccess) return fail(ctx, HDG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return HDG_OK;
}

// y by mode from K x (see k_face_op), binary64 vectors: the binary64 kernels
template <class MT>
void face_op(const FaceDevT<MT>& fd, bool tr, const double* x, const double* b, double* y, int mode, cudaStream_t st,
             const int* faces = nullptr, int nfaces = 0, int skip_diag = 0, int tri = 0) {
  const int nf = faces ? nfaces : fd.n_face;
  if (nf == 0) return;
  const int fb = (nf + kFaceWarps - 1) / kFaceWarps;
  const bool inplace = x == y;
  if (tr) {
    if (inplace) k_face_op<true, true, MT><<<fb, 32 * kFaceWarps, 0, st>>>(fd, x, b, y, mode, faces, nfaces, skip_diag, tri);
    else k_face_op<true, false, MT><<<fb, 32 * kFaceWarps, 0, st>>>(fd, x, b, y, mode, faces, nfaces, skip_diag, tri);
  } else {
    if (inplace) k_face_op<false, true, MT><<<fb, 32 * kFaceWarps, 0, st>>>(fd, x, b, y, mode, faces, nfaces, skip_diag, tri);
    else k_face_op<false, false, MT><<<fb, 32 * kFaceWarps, 0, st>>>(fd, x, b, y, mode, faces, nfaces, skip_diag, tri);
  }
}
// the same with float-float vectors: the double-word kernels
template <class MT>
void face_op(const FaceDevT<MT>& fd, bool tr, const float2* x, const float2* b, float2* y, int mode, cudaStream_t st,
             const int* faces = nullptr, int nfaces = 0, int skip_diag = 0, int tri = 0) {
  const int nf = faces ? nfaces : fd.n_face;
  if (nf == 0) return;
  const int fb = (nf + kFaceWarps - 1) / kFaceWarps;
  const bool inplace = x == y;
  if (tr) {
    if (inplace) k_face_op_ff<true, true, MT><<<fb, 32 * kFaceWarps, 0, st>>>(fd, x, b, y, mode, faces, nfaces, skip_diag, tri);
    else k_face_op_ff<true, false, MT><<<fb, 32 * kFaceWarps, 0, st>>>(fd, x, b, y, mode, faces, nfaces, skip_diag, tri);
  } else {
    if (inplace) k_face_op_ff<false, true, MT><<<fb, 32 * kFaceWarps, 0, st>>>(fd, x, b, y, mode, faces, nfaces, skip_diag, tri);
    else k_face_op_ff<false, false, MT><<<fb, 32 * kFaceWarps, 0, st>>>(fd, x, b, y, mode, faces, nfaces, skip_diag, tri);
  }
}

// The solver's views for a vector storage VS: K (and the pivot inverses of
// block Jacobi / SGS), the binary64 ILU factors, and its work vectors.
inline const FaceDev& kview(const hdg_solver* S, const double*) { return S->f; }
inline const FaceDevT<float2>& kview(const hdg_solver* S, const float2*) { return S->fff; }
inline const FaceDev& iview(const hdg_solver* S, const double*) { return S->fi; }
inline const FaceDevT<float2>& iview(const hdg_solver* S, const float2*) { return S->fiff; }
inline const FaceDevT<float>& i32view(const hdg_solver* S, const double*) { return S->fi32; }
inline const FaceDevT<float>& i32view(const hdg_solver* S, const float2*) { return S->fi32ff; }
template <class VS>
VS* vec(double* p) {
  return reinterpret_cast<VS*>(p);
}

// z = M^{-1} r for the multicolor block symmetric Gauss-Seidel preconditioner:
// from z = 0, a forward sweep over the colors, then a backward one; each color
// is one launch (its faces are mutually uncoupled, so the sweep is exact Gauss-Seidel).
template <class VS>
void sgs_apply(hdg_solver* S, bool tr, const VS* r, VS* z, cudaStream_t st) {
  cudaMemsetAsync(z, 0, sizeof(VS) * S->n, st);  // all-zero bytes: 0 in both storages
  const int nc = (int)S->color_off.size() - 1;
  for (int pass = 0; pass < 2; ++pass)
    for (int k = 0; k < nc; ++k) {
      const int c = pass == 0 ? k : nc - 1 - k;
      const int o0 = S->color_off[c], o1 = S->color_off[c + 1];
      face_op(kview(S, z), tr, z, r, z, 1, st, S->colors + o0, o1 - o0, 1, 0);
    }
}

// z = (L U)^{-1} r, or (L U)^{-T} r, with the block ILU(0) factors: a forward
// sweep over the colors into tmp2 (L y = r: y_e = r_e - sum of L_ek y_k over
// earlier colors; transposed, U^T y = r), then a backward one into z
// (U z = y: z_e = U_ee^{-1} (y_e - sum of U_ej z_j over later colors;
// transposed, L^T z = y).  r and z must not be tmp2.
template <class MT, class VS>
void ilu_sweeps(hdg_solver* S, const FaceDevT<MT>& fi, bool tr, const VS* r, VS* z, cudaStream_t st) {
  VS* t2 = vec<VS>(S->tmp2);
  const int nc = (int)S->color_off.size() - 1;
  for (int c = 0; c < nc; ++c) {
    const int o0 = S->color_off[c], o1 = S->color_off[c + 1];
    face_op(fi, tr, t2, r, t2, tr ? 1 : 4, st, S->colors + o0, o1 - o0, 0, 1);
  }
  for (int c = nc - 1; c >= 0; --c) {
    const int o0 = S->color_off[c], o1 = S->color_off[c + 1];
    face_op(fi, tr, z, t2, z, tr ? 4 : 1, st, S->colors + o0, o1 - o0, 0, 2);
  }
}
template <class VS>
void ilu_apply(hdg_solver* S, bool tr, const VS* r, VS* z, cudaStream_t st) {
  if (S->precond == 3) ilu_sweeps(S, i32view(S, z), tr, r, z, st);  // binary32 factors
  else ilu_sweeps(S, iview(S, z), tr, r, z, st);
}

// w = M^{-1} b for the solver's preconditioner
template <class VS>
void prec_rhs(hdg_solver* S, bool tr, const VS* b, VS* w, cudaStream_t st) {
  if (S->precond == 0) face_op(kview(S, w), tr, vec<VS>(S->zero), b, w, 3, st);
  else if (S->precond == 1) sgs_apply(S, tr, b, w, st);
  else ilu_apply(S, tr, b, w, st);
}
// w = M^{-1} K v (block Jacobi: one fused launch)
template <class VS>
void prec_op(hdg_solver* S, bool tr, const VS* v, VS* w, cudaStream_t st) {
  if (S->precond == 0) {
    face_op(kview(S, w), tr, v, (const VS*)nullptr, w, 0, st);
  } else {
    face_op(kview(S, w), tr, v, (const VS*)nullptr, vec<VS>(S->tmp), 2, st);
    prec_rhs(S, tr, (const VS*)vec<VS>(S->tmp), w, st);
  }
}
// w = M^{-1} (b - K x)
template <class VS>
void prec_res(hdg_solver* S, bool tr, const VS* x, const VS* b, VS* w, cudaStream_t st) {
  if (S->precond == 0) {
    face_op(kview(S, w), tr, x, b, w, 1, st);
  } else {
    face_op(kview(S, w), tr, x, b, vec<VS>(S->tmp), 4, st);
    prec_rhs(S, tr, (const VS*)vec<VS>(S->tmp), w, st);
  }
}

// the binary32 factor view: K's layout and tables, values and pivot inverses in binary32
template <class MT>
void set_view(FaceDevT<MT>& v, const FaceDev& f, const MT* K, MT* dinv) {
  v.n_face = f.n_face;
  v.face_p = f.face_p;
  v.lam_off = f.lam_off;
  v.k_col = f.k_col;
  v.k_blkoff = f.k_blkoff;
  v.dinv_off = f.dinv_off;
  v.k_tblk = f.k_tblk;
  v.fcolor = f.fcolor;
  v.K = K;
  v.dinv = dinv;
  v.bad = f.bad;
}
void set_fi32(hdg_solver* S, float* dinv32) { set_view(S->fi32, S->f, (const float*)S->F32, dinv32); }

void split_copy(const hdg_solver* S, const double* a, float2* b, int64_t n, cudaStream_t st) {
  if (n > 0) k_split<<<grid_for(n, 256, 8 * S->sms), 256, 0, st>>>(a, b, n);
}

// enqueue the factorization of the preconditioner for the current K (a
// singular pivot block sets f.bad, cleared first); for arith 1 the
// lane-ordered double-word copies of K and of the factors the sweeps use, for
// products with K (tr = 0) or K^T (block Jacobi / SGS: pivot inverses
// computed in binary32, stored as pairs)
hdg_status setup_enqueue(hdg_solver* S, cudaStream_t st, int arith, int tr = 0) {
  hdg_ctx* ctx = S->sys->ctx;
  const int nf = (S->f.n_face + kFaceWarps - 1) / kFaceWarps;
  hdg_status rs;
  if ((rs = ck(ctx, cudaMemsetAsync(S->f.bad, 0, sizeof(int), st), "cudaMemsetAsync")) != HDG_OK) return rs;
  if (S->precond == 2 || S->precond == 3) {
    const bool f32 = S->precond == 3;
    if (f32) {
      k_to_float<<<grid_for(S->k_vals, 256, 8 * S->sms), 256, 0, st>>>(S->f.K, S->F32, S->k_vals);
    } else if ((rs = ck(ctx, cudaMemcpyAsync(S->F, S->f.K, sizeof(double) * S->k_vals, cudaMemcpyDeviceToDevice, st),
                        "cudaMemcpyAsync")) != HDG_OK) {
      return rs;
    }
    const int nc = (int)S->color_off.size() - 1;
    for (int c = 0; c < nc; ++c) {
      const int o0 = S->color_off[c], n = S->color_off[c + 1] - o0;
      if (n == 0) continue;
      const int nb = (n + kFaceWarps - 1) / kFaceWarps;
      if (f32) k_ilu_row<float><<<nb, 32 * kFaceWarps, 0, st>>>(S->fi32, S->F32, S->colors + o0, n);
      else k_ilu_row<double><<<nb, 32 * kFaceWarps, 0, st>>>(S->fi, S->F, S->colors + o0, n);
    }
  } else if (arith == 1) {
    k_bj_invert<float, float2><<<nf, 32 * kFaceWarps, 0, st>>>(S->f, S->fff.dinv, tr);
  } else {
    k_bj_invert<double, double><<<nf, 32 * kFaceWarps, 0, st>>>(S->f, S->f.dinv, -1);
  }
  if (arith == 1) {  // the lane-ordered copies k_face_op_ff reads
    k_lane_order_blocks<double, float2><<<nf, 32 * kFaceWarps, 0, st>>>(S->f, S->f.K, const_cast<float2*>(S->fff.K), tr);
    if (S->precond == 2) {
      k_lane_order_blocks<double, float2><<<nf, 32 * kFaceWarps, 0, st>>>(S->f, S->F, const_cast<float2*>(S->fiff.K), tr);
      k_lane_order_dinv<double, float2><<<nf, 32 * kFaceWarps, 0, st>>>(S->f, S->fi.dinv, S->fiff.dinv, tr);
    } else if (S->precond == 3) {
      k_lane_order_blocks<float, float><<<nf, 32 * kFaceWarps, 0, st>>>(S->f, S->F32, const_cast<float*>(S->fi32ff.K), tr);
      k_lane_order_dinv<float, float><<<nf, 32 * kFaceWarps, 0, st>>>(S->f, S->fi32.dinv, S->fi32ff.dinv, tr);
    }
  }
  if ((rs = ck(ctx, cudaGetLastError(), "preconditioner setup")) != HDG_OK) return rs;
  // the binary64 factors (hdg_solver_precond_apply) are current unless the
  // pivot inverses were computed for the double-word solve only
  S->factored = !(arith == 1 && S->precond <= 1);
  return HDG_OK;
}

// out[j] = V_j . w for j < nvec (device), one launch
template <class VS>
void dots(hdg_solver* S, const VS* V, int nvec, const VS* w, double* out, cudaStream_t st) {
  k_dots<VS><<<S->dot_blocks, kDotThreads, 0, st>>>(V, S->n, nvec, w, S->n, S->partial, S->gpart, out, S->ticket);
}

}  // namespace

namespace {

// Byte offsets of the solver's device buffers in one workspace (256-byte aligned).
struct SolverPlan {
  int64_t n = 0, dinv_len = 0, k_vals = 0;
  int dot_blocks = 0;
  size_t kc, kb, kt, dof, dinv, bad, ticket, V, part, h, coef, zero, tmp, cols, fcol, F, dinv2, tmp2;
  size_t kff, dinvff, xff, eff, fff, dinv2ff;  // arith 1: the double-word copies (0 when not planned)
  size_t total;
};

SolverPlan plan_solver(const hdg_mesh* M, int restart, int precond, int sms, int arith = 0) {
  SolverPlan p{};
  size_t o = 0;
  auto take = [&o](size_t bytes) {
    const size_t at = o;
    o += (std::max<size_t>(bytes, 16) + 255) / 256 * 256;
    return at;
  };
  const size_t nf = (size_t)M->n_face, nr = (size_t)restart + 1;
  p.n = M->lam_len;
  for (int e = 0; e < M->n_face; ++e) p.dinv_len += (int64_t)(4 * (M->face_p[e] + 1)) * (4 * (M->face_p[e] + 1));
  p.k_vals = M->k_blkoff.empty() ? 0 : M->k_blkoff.back();
  // one wave of the Krylov kernels (two 256-thread blocks per SM at <= 128 registers), grid-stride beyond
  p.dot_blocks = std::max(1, std::min<int>(2 * std::max(sms, 1), (int)((p.n / 2 + 2 * kDotThreads - 1) / (2 * kDotThreads))));
  p.kc = take(sizeof(int) * 5 * nf);
  p.kb = take(sizeof(int64_t) * M->k_blkoff.size());
  p.kt = take(sizeof(int64_t) * 5 * nf);
  p.dof = take(sizeof(int64_t) * nf);
  p.dinv = take(sizeof(double) * p.dinv_len);
  p.bad = take(sizeof(int));
  p.ticket = take(sizeof(unsigned) * (1 + fin_groups(p.dot_blocks)));
  p.V = take(sizeof(double) * nr * p.n);
  // two rows per basis vector in an Arnoldi reduction; then the group sums of the two-level finish
  p.part = take(sizeof(double) * 2 * nr * (p.dot_blocks + fin_groups(p.dot_blocks)));
  p.h = take(sizeof(double) * arnoldi_doubles(restart));
  p.coef = take(sizeof(double) * nr);
  p.zero = take(sizeof(double) * p.n);
  p.tmp = take(sizeof(double) * p.n);
  p.cols = take(sizeof(int) * nf);
  p.fcol = take(sizeof(int) * nf);
  p.F = p.dinv2 = p.tmp2 = 0;
  if (precond == 2 || precond == 3) {  // the incomplete factors, in binary64 or binary32
    const size_t vs = precond == 2 ? sizeof(double) : sizeof(float);
    p.F = take(vs * p.k_vals);
    p.dinv2 = take(vs * p.dinv_len);
    p.tmp2 = take(sizeof(double) * p.n);
  }
  p.kff = p.dinvff = p.xff = p.eff = p.fff = p.dinv2ff = 0;
  if (arith == 1) {  // the double-word copies of the float-float solve
    p.kff = take(sizeof(float2) * p.k_vals);
    p.dinvff = take(sizeof(float2) * p.dinv_len);
    p.xff = take(sizeof(float2) * p.n);
    p.eff = take(sizeof(float2) * p.n);
    if (precond == 2 || precond == 3) {
      p.fff = take(sizeof(float2) * p.k_vals);
      p.dinv2ff = take(sizeof(float2) * p.dinv_len);
    }
  }
  p.total = o;
  return p;
}

}  // namespace

extern "C" hdg_status hdg_solver_destroy(hdg_solver* S);

namespace {

// Plan, place (one cudaMalloc, or the caller's workspace) and fill the solver's state.
hdg_status solver_build(hdg_sys* sys, int32_t restart, int32_t precond, int32_t arith, void* ws, int64_t ws_bytes,
                        hdg_solver** out) {
  if (!sys || !out) return HDG_EINVAL;
  *out = nullptr;
  hdg_ctx* ctx = sys->ctx;
  if (restart < 1 || restart > kMaxRestart) return fail(ctx, HDG_EINVAL, "hdg_solver_create: restart must be in 1..64");
  if (precond < 0 || precond > 3) return fail(ctx, HDG_EINVAL, "hdg_solver_create: preconditioner kind must be 0..3");
  const hdg_mesh* M = sys->mesh;
  HDG_ON_DEVICE(ctx, ctx->device);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (arith < 0 || arith > 1) return fail(ctx, HDG_EINVAL, "hdg_solver_create_ws_arith: arithmetic must be 0 or 1");
  const SolverPlan P = plan_solver(M, restart, precond, sms, arith);
  if (ws && ((uintptr_t)ws % 256 != 0 || ws_bytes < (int64_t)P.total))
    return fail(ctx, HDG_EINVAL,
                "hdg_solver_create_ws: workspace smaller than hdg_solver_workspace_bytes or not 256-byte aligned");
  // tables: block of (col, e) for products with K^T, pivot-inverse offsets, the multicolor order
  std::vector<int64_t> tblk(5 * (size_t)M->n_face, -1);
  for (int e = 0; e < M->n_face; ++e)
    for (int b = 0; b < 5; ++b) {
      const int f = M->k_col[5 * e + b];
      if (f < 0) continue;
      for (int t = 0; t < 5; ++t)
        if (M->k_col[5 * f + t] == e) tblk[5 * e + b] = M->k_blkoff[5 * f + t];
    }
  std::vector<int64_t> dinv_off(M->n_face);
  int64_t tot = 0;
  for (int e = 0; e < M->n_face; ++e) {
    const int m = 4 * (M->face_p[e] + 1);
    dinv_off[e] = tot;
    tot += (int64_t)m * m;
  }
  // greedy coloring: faces of one element (the nonzero blocks of a K row) get different colors
  std::vector<int> color(M->n_face, -1);
  int ncol = 0;
  for (int e = 0; e < M->n_face; ++e) {
    unsigned used = 0;
    for (int b = 0; b < 5; ++b) {
      const int f = M->k_col[5 * e + b];
      if (f >= 0 && f != e && color[f] >= 0) used |= 1u << color[f];
    }
    int c = 0;
    while (used & (1u << c)) ++c;
    color[e] = c;
    ncol = std::max(ncol, c + 1);
  }
  hdg_solver* S = new hdg_solver();
  S->sys = sys;
  S->restart = restart;
  S->n = P.n;
  S->sms = sms;
  S->dot_blocks = P.dot_blocks;
  S->color_off.assign(1, 0);
  std::vector<int> by_color;
  for (int c = 0; c < ncol; ++c) {
    for (int e = 0; e < M->n_face; ++e)
      if (color[e] == c) by_color.push_back(e);
    S->color_off.push_back((int)by_color.size());
  }
  char* base = (char*)ws;
  if (!base) {
    void* p = nullptr;
    if (cudaMalloc(&p, P.total) != cudaSuccess) {
      delete S;
      return fail(ctx, HDG_ENOMEM, "hdg_solver_create: device allocation failed");
    }
    S->allocs.push_back(p);
    base = (char*)p;
  } else {
    S->external_ws = true;
  }
  const size_t nr = (size_t)restart + 1;
  if (S->external_ws) {  // no pinned allocation (its release may synchronise the device)
    S->hpin = new double[std::max<size_t>(2 * nr + 2, 16)];
    S->hpin_pageable = true;
  } else if (cudaMallocHost((void**)&S->hpin, sizeof(double) * std::max<size_t>(2 * nr + 2, 16)) != cudaSuccess) {
    S->hpin = nullptr;
    hdg_solver_destroy(S);
    return fail(ctx, HDG_ENOMEM, "hdg_solver_create: pinned host allocation failed");
  }
  int *kc = (int*)(base + P.kc), *cols = (int*)(base + P.cols), *fcol = (int*)(base + P.fcol);
  int64_t *kb = (int64_t*)(base + P.kb), *kt = (int64_t*)(base + P.kt), *dof = (int64_t*)(base + P.dof);
  hdg_status st = HDG_OK;
  if (st == HDG_OK) st = ck(ctx, cudaMemcpy(kc, M->k_col.data(), sizeof(int) * M->k_col.size(), cudaMemcpyHostToDevice), "cudaMemcpy");
  if (st == HDG_OK) st = ck(ctx, cudaMemcpy(kb, M->k_blkoff.data(), sizeof(int64_t) * M->k_blkoff.size(), cudaMemcpyHostToDevice), "cudaMemcpy");
  if (st == HDG_OK) st = ck(ctx, cudaMemcpy(dof, dinv_off.data(), sizeof(int64_t) * dinv_off.size(), cudaMemcpyHostToDevice), "cudaMemcpy");
  if (st == HDG_OK) st = ck(ctx, cudaMemcpy(kt, tblk.data(), sizeof(int64_t) * tblk.size(), cudaMemcpyHostToDevice), "cudaMemcpy");
  if (st == HDG_OK) st = ck(ctx, cudaMemset(base + P.zero, 0, sizeof(double) * S->n), "cudaMemset");
  if (st == HDG_OK) st = ck(ctx, cudaMemset(base + P.ticket, 0, sizeof(unsigned) * (1 + fin_groups(P.dot_blocks))), "cudaMemset");
  if (st == HDG_OK && !by_color.empty())
    st = ck(ctx, cudaMemcpy(cols, by_color.data(), sizeof(int) * by_color.size(), cudaMemcpyHostToDevice), "cudaMemcpy");
  if (st == HDG_OK && !color.empty())
    st = ck(ctx, cudaMemcpy(fcol, color.data(), sizeof(int) * color.size(), cudaMemcpyHostToDevice), "cudaMemcpy");
  if (st != HDG_OK) {
    hdg_solver_destroy(S);
    return st;
  }
  S->f.n_face = M->n_face;
  S->f.face_p = M->dm.face_p;
  S->f.lam_off = M->dm.lam_off;
  S->f.k_col = kc;
  S->f.k_blkoff = kb;
  S->f.dinv_off = dof;
  S->f.k_tblk = kt;
  S->f.fcolor = fcol;
  S->f.K = sys->ds.K;
  S->f.dinv = (double*)(base + P.dinv);
  S->f.bad = (int*)(base + P.bad);
  S->V = (double*)(base + P.V);
  S->partial = (double*)(base + P.part);
  S->gpart = S->partial + (size_t)2 * nr * P.dot_blocks;
  S->ticket = (unsigned*)(base + P.ticket);
  S->h = (double*)(base + P.h);
  S->coef = (double*)(base + P.coef);
  S->zero = (double*)(base + P.zero);
  S->tmp = (double*)(base + P.tmp);
  S->colors = cols;
  S->fcolor = color;
  S->k_vals = P.k_vals;
  S->dinv_len = tot;
  if (precond == 2) {
    S->F = (double*)(base + P.F);
    S->tmp2 = (double*)(base + P.tmp2);
    S->fi = S->f;
    S->fi.K = S->F;
    S->fi.dinv = (double*)(base + P.dinv2);
  } else if (precond == 3) {
    S->F32 = (float*)(base + P.F);
    S->tmp2 = (double*)(base + P.tmp2);
    set_fi32(S, (float*)(base + P.dinv2));
  }
  S->precond = precond;
  if (arith == 1) {  // the planned double-word copies (ensure_ff finds them in place)
    set_view(S->fff, S->f, (const float2*)(base + P.kff), (float2*)(base + P.dinvff));
    S->xff = (float2*)(base + P.xff);
    S->eff = (float2*)(base + P.eff);
    if (precond == 2 || precond == 3) {
      set_view(S->fiff, S->f, (const float2*)(base + P.fff), (float2*)(base + P.dinv2ff));
      set_view(S->fi32ff, S->f, (const float*)(base + P.fff), (float*)(base + P.dinv2ff));
    }
    S->arith = 1;
  }
  *out = S;
  return HDG_OK;
}

// The double-word copies of arith 1, allocated on first use: K and its pivot
// inverses, the solution and right-hand side of a solve, and (block ILU(0))
// the factors and their pivot inverses.
hdg_status ensure_ff(hdg_solver* S, int kind) {
  hdg_ctx* ctx = S->sys->ctx;
  const bool need_k = !S->fff.K, need_i = (kind == 2 || kind == 3) && !S->fiff.K;
  if (!need_k && !need_i) return HDG_OK;
  if (S->external_ws)
    return fail(ctx, HDG_ENOMEM, "hdg_solver_set_arithmetic: the caller's workspace was planned without the float-float copies");
  HDG_ON_DEVICE(ctx, ctx->device);
  const size_t kv = sizeof(float2) * std::max<int64_t>(S->k_vals, 2), dv = sizeof(float2) * std::max<int64_t>(S->dinv_len, 2);
  auto up = [](size_t sz) { return (sz + 255) / 256 * 256; };
  const size_t bytes = up(kv) + up(dv) + (need_k ? 2 * up(sizeof(float2) * (size_t)S->n) : 0);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess)
    return fail(ctx, HDG_ENOMEM, "hdg_solver_set_arithmetic: device allocation of the float-float copies failed");
  S->allocs.push_back(p);
  char* b = (char*)p;
  auto take = [&b](size_t sz) {
    char* at = b;
    b += (sz + 255) / 256 * 256;
    return (void*)at;
  };
  if (need_k) {
    float2* K = (float2*)take(kv);
    float2* di = (float2*)take(dv);
    set_view(S->fff, S->f, (const float2*)K, di);
    S->xff = (float2*)take(sizeof(float2) * S->n);
    S->eff = (float2*)take(sizeof(float2) * S->n);
  } else {
    float2* K = (float2*)take(kv);
    float2* di = (float2*)take(dv);
    set_view(S->fiff, S->f, (const float2*)K, di);
    set_view(S->fi32ff, S->f, (const float*)K, (float*)di);
  }
  return need_k && need_i ? ensure_ff(S, kind) : HDG_OK;
}

// Steps j0 .. j1 - 1 of a GMRES cycle, enqueued on st: z = M^{-1} K u_j, the
// reduction, the update with the bookkeeping block (the last step R of a
// cycle: the reduction and the bookkeeping alone).
template <class VS>
void enqueue_chunk(hdg_solver* S, bool tr, int j0, int j1, cudaStream_t st) {
  const int64_t n = S->n;
  const int R = S->restart;
  VS* V = vec<VS>(S->V);
  for (int j = j0; j < j1; ++j) {
    const bool prod = j < R;
    if (prod) prec_op(S, tr, (const VS*)(V + (int64_t)j * n), V + (int64_t)(j + 1) * n, st);
    k_dcgs_reduce<VS><<<S->dot_blocks, kDotThreads, 0, st>>>(V, n, j, prod ? 1 : 0, n, S->partial, S->gpart,
                                                             S->ticket);
    k_dcgs_update<VS><<<(prod ? S->dot_blocks : 0) + 1, kDotThreads, 0, st>>>(
        V, n, j, prod ? 1 : 0, n, S->gpart, fin_groups(S->dot_blocks), S->h, R);
  }
}

// The chunk's launches as an instantiated CUDA graph (captured on the
// solver's own stream on first use, kept until the solver is destroyed), or
// null: a solver in a caller's workspace launches directly (instantiation may
// allocate), and so does every solver after a capture that failed.  The
// graph's arguments are the solver's own buffers, fixed for its lifetime.
template <class VS>
cudaGraphExec_t chunk_graph(hdg_solver* S, bool tr, int j0, int j1) {
  if (S->external_ws || S->graphs_off) return nullptr;
  const int arith = std::is_same<VS, float2>::value ? 1 : 0;
  const long long key = (long long)j0 | ((long long)arith << 8) | ((long long)S->precond << 9) | ((long long)tr << 12);
  auto it = S->chunk_graphs.find(key);
  if (it != S->chunk_graphs.end()) return it->second;
  if (!S->cap && cudaStreamCreateWithFlags(&S->cap, cudaStreamNonBlocking) != cudaSuccess) {
    S->cap = nullptr;
    S->graphs_off = true;
    cudaGetLastError();
    return nullptr;
  }
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  bool ok = cudaStreamBeginCapture(S->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    enqueue_chunk<VS>(S, tr, j0, j1, S->cap);
    ok = cudaStreamEndCapture(S->cap, &g) == cudaSuccess && g;
  }
  if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    if (ge) cudaGraphExecDestroy(ge);
    S->graphs_off = true;
    cudaGetLastError();  // the failure is handled: direct launches from now on
    return nullptr;
  }
  S->chunk_graphs[key] = ge;
  return ge;
}

// Restarted, left-preconditioned GMRES on vectors of storage VS (binary64, or
// float-float pairs under arith 1): x += the solution of M^{-1} K dx =
// M^{-1} (E - K x) to rtol of ||M^{-1} E||.  Each restart forms the true
// residual r0 = M^{-1} (E - K x) and its norm on the host's side of the
// loop; the cycle then runs the Arnoldi process as delayed classical
// Gram-Schmidt with re-orthogonalisation (hdg_krylov.cuh), step j being
//   z = M^{-1} K u_j (prec_op), one reduction pass (k_dcgs_reduce), one
//   update pass with the Hessenberg bookkeeping in an extra block (k_dcgs_update),
// and a last reduction-only step R that finishes column R - 1.  The host
// launches kChunk steps at a time (a captured graph per chunk) and reads the
// state back once per chunk (at most kChunk - 1 steps past convergence are
// computed and discarded: their columns are not part of the solution update).
template <class VS>
hdg_status gmres(hdg_solver* S, bool tr, const VS* E, VS* x, double rtol, int max_iter, int& it, double& rel,
                 cudaStream_t st) {
  hdg_ctx* ctx = S->sys->ctx;
  const int64_t n = S->n;
  const int R = S->restart;
  const int vb = grid_for(n, 256, 8 * S->sms);
  VS* V = vec<VS>(S->V);
  hdg_status rs;
  // the preconditioner's factors of the current K
  if ((rs = setup_enqueue(S, st, std::is_same<VS, float2>::value ? 1 : 0, tr ? 1 : 0)) != HDG_OK) return rs;
  // ||M^-1 E||
  prec_rhs(S, tr, E, V, st);
  dots(S, (const VS*)V, 1, (const VS*)V, S->h, st);
  if ((rs = ck(ctx, cudaMemcpyAsync(S->hpin, S->h, sizeof(double), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync")) != HDG_OK) return rs;
  if ((rs = ck(ctx, cudaMemcpyAsync(&S->hpin[1], S->f.bad, sizeof(int), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync")) != HDG_OK) return rs;
  if ((rs = ck(ctx, cudaStreamSynchronize(st), "cudaStreamSynchronize")) != HDG_OK) return rs;
  int bad = 0;
  std::memcpy(&bad, &S->hpin[1], sizeof(int));
  if (bad) {
    S->factored = false;
    return fail(ctx, HDG_ESINGULAR, "hdg_trace_solve: a pivot block of the preconditioner is singular");
  }
  const double bnorm = std::sqrt(S->hpin[0]);
  it = 0;
  rel = 0.0;
  if (!(bnorm > 0.0)) {  // E = 0: the solution is 0
    if ((rs = ck(ctx, cudaMemsetAsync(x, 0, sizeof(VS) * n, st), "cudaMemsetAsync")) != HDG_OK) return rs;
    return ck(ctx, cudaStreamSynchronize(st), "cudaStreamSynchronize");
  }
  constexpr int kChunk = 4;
  const ArnoldiViews av = arnoldi_views(S->h, R);
  rel = 1.0;
  while (true) {
    // r0 = M^-1 (E - K x) (the candidate u_0), beta = ||r0||
    prec_res(S, tr, (const VS*)x, E, V, st);
    dots(S, (const VS*)V, 1, (const VS*)V, S->h, st);
    if ((rs = ck(ctx, cudaMemcpyAsync(S->hpin, S->h, sizeof(double), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync")) != HDG_OK) return rs;
    if ((rs = ck(ctx, cudaStreamSynchronize(st), "cudaStreamSynchronize")) != HDG_OK) return rs;
    const double beta = std::sqrt(S->hpin[0]);
    rel = beta / bnorm;
    if (!(rel > rtol) || it >= max_iter) break;
    k_cycle_init<<<1, 1, 0, st>>>(S->h, R, beta, bnorm, rtol, it, max_iter);
    for (int j0 = 0; j0 <= R; j0 += kChunk) {
      const int j1 = std::min(R + 1, j0 + kChunk);
      cudaGraphExec_t ge = chunk_graph<VS>(S, tr, j0, j1);
      if (ge) {
        if ((rs = ck(ctx, cudaGraphLaunch(ge, st), "cudaGraphLaunch")) != HDG_OK) return rs;
      } else {
        enqueue_chunk<VS>(S, tr, j0, j1, st);
      }
      if ((rs = ck(ctx, cudaMemcpyAsync(S->hpin, av.sc, sizeof(double) * kArnoldiScalars, cudaMemcpyDeviceToHost, st),
                   "cudaMemcpyAsync")) != HDG_OK)
        return rs;
      if ((rs = ck(ctx, cudaStreamSynchronize(st), "cudaStreamSynchronize")) != HDG_OK) return rs;
      it = (int)S->hpin[6];
      rel = S->hpin[1];
      if (S->hpin[4] != 0.0) break;
    }
    // x += V y, H y = g (upper triangular), on the device
    k_lsq<<<1, 256, 0, st>>>(S->h, R);
    k_update_x<VS><<<vb, kDotThreads, 0, st>>>(V, n, av.y, av.sc + 5, x, n);
  }
  if ((rs = ck(ctx, cudaGetLastError(), "trace solve kernels")) != HDG_OK) return rs;
  return (rel > rtol) ? fail(ctx, HDG_ETIMEOUT, "hdg_trace_solve: max_iter reached before rtol") : HDG_OK;
}

}  // namespace

extern "C" {

hdg_status hdg_solver_create(hdg_sys* sys, int32_t restart, hdg_solver** out) {
  return solver_build(sys, restart, 0, 0, nullptr, 0, out);
}

hdg_status hdg_solver_create_ws(hdg_sys* sys, int32_t restart, int32_t precond, void* workspace, int64_t bytes,
                                hdg_solver** out) {
  if (!workspace) return HDG_EINVAL;
  return solver_build(sys, restart, precond, 0, workspace, bytes, out);
}

int64_t hdg_solver_workspace_bytes(const hdg_mesh* mesh, int32_t restart, int32_t precond) {
  if (!mesh || restart < 1 || restart > kMaxRestart || precond < 0 || precond > 3) return -1;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, mesh->ctx->device) != cudaSuccess) return -1;
  return (int64_t)plan_solver(mesh, restart, precond, sms).total;
}

hdg_status hdg_solver_create_ws_arith(hdg_sys* sys, int32_t restart, int32_t precond, int32_t arith, void* workspace,
                                      int64_t bytes, hdg_solver** out) {
  if (!workspace) return HDG_EINVAL;
  return solver_build(sys, restart, precond, arith, workspace, bytes, out);
}

int64_t hdg_solver_workspace_bytes_arith(const hdg_mesh* mesh, int32_t restart, int32_t precond, int32_t arith) {
  if (!mesh || restart < 1 || restart > kMaxRestart || precond < 0 || precond > 3 || arith < 0 || arith > 1) return -1;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, mesh->ctx->device) != cudaSuccess) return -1;
  return (int64_t)plan_solver(mesh, restart, precond, sms, arith).total;
}

hdg_status hdg_solver_destroy(hdg_solver* S) {
  if (!S) return HDG_EINVAL;
  hdg::DeviceGuard dg(S->sys->ctx->device);
  for (auto& kv : S->chunk_graphs) cudaGraphExecDestroy(kv.second);
  if (S->cap) cudaStreamDestroy(S->cap);
  for (void* p : S->allocs) cudaFree(p);
  if (S->hpin) {
    if (S->hpin_pageable) delete[] S->hpin;
    else cudaFreeHost(S->hpin);
  }
  delete S;
  return HDG_OK;
}

hdg_status hdg_solver_set_preconditioner(hdg_solver* S, int32_t kind) {
  if (!S || kind < 0 || kind > 3) return HDG_EINVAL;
  const bool need64 = kind == 2 && !S->F, need32 = kind == 3 && !S->F32;
  if (need64 || need32) {  // the incomplete factors: a copy of K's values, pivot inverses, a work vector
    hdg_ctx* ctx = S->sys->ctx;
    if (S->external_ws)
      return fail(ctx, HDG_ENOMEM, "hdg_solver_set_preconditioner: the caller's workspace was planned without these factors");
    HDG_ON_DEVICE(ctx, ctx->device);
    const size_t vs = need64 ? sizeof(double) : sizeof(float);
    void *F = nullptr, *di = nullptr, *t2 = nullptr;
    if (cudaMalloc(&F, vs * std::max<int64_t>(S->k_vals, 2)) != cudaSuccess) F = nullptr;
    if (F && cudaMalloc(&di, vs * std::max<int64_t>(S->dinv_len, 2)) != cudaSuccess) di = nullptr;
    if (di && !S->tmp2 && cudaMalloc(&t2, sizeof(double) * std::max<int64_t>(S->n, 2)) != cudaSuccess) t2 = nullptr;
    if (!di || (!S->tmp2 && !t2)) {
      if (F) cudaFree(F);
      if (di) cudaFree(di);
      return fail(ctx, HDG_ENOMEM, "hdg_solver_set_preconditioner: device allocation of the ILU factors failed");
    }
    S->allocs.push_back(F);
    S->allocs.push_back(di);
    if (t2) {
      S->allocs.push_back(t2);
      S->tmp2 = (double*)t2;
    }
    if (need64) {
      S->F = (double*)F;
      S->fi = S->f;
      S->fi.K = S->F;
      S->fi.dinv = (double*)di;
    } else {
      S->F32 = (float*)F;
      set_fi32(S, (float*)di);
    }
  }
  if (S->arith == 1) {
    hdg_status rs = ensure_ff(S, kind);
    if (rs != HDG_OK) return rs;
  }
  if (kind != S->precond) S->factored = false;
  S->precond = kind;
  return HDG_OK;
}

hdg_status hdg_solver_set_arithmetic(hdg_solver* S, int32_t arith) {
  if (!S || arith < 0 || arith > 1) return HDG_EINVAL;
  if (arith == 1) {
    hdg_status rs = ensure_ff(S, S->precond);
    if (rs != HDG_OK) return rs;
  }
  S->arith = arith;
  return HDG_OK;
}

hdg_status hdg_solver_setup(hdg_solver* S, void* stream) {
  hdg::NvtxRange nvtx_range_("hdg::solver_setup");
  if (!S) return HDG_EINVAL;
  hdg_ctx* ctx = S->sys->ctx;
  HDG_ON_DEVICE(ctx, ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  hdg_status rs;
  if ((rs = setup_enqueue(S, st, 0)) != HDG_OK) return rs;
  if ((rs = ck(ctx, cudaMemcpyAsync(S->hpin, S->f.bad, sizeof(int), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync")) != HDG_OK)
    return rs;
  if ((rs = ck(ctx, cudaStreamSynchronize(st), "cudaStreamSynchronize")) != HDG_OK) return rs;
  int bad = 0;
  std::memcpy(&bad, S->hpin, sizeof(int));
  if (bad) {
    S->factored = false;
    return fail(ctx, HDG_ESINGULAR, "hdg_solver_setup: a pivot block of the preconditioner is singular");
  }
  return HDG_OK;
}

hdg_status hdg_solver_precond_apply(hdg_solver* S, const double* r, double* z, int32_t transpose, void* stream) {
  if (!S || !r || !z || r == z) return HDG_EINVAL;
  hdg_ctx* ctx = S->sys->ctx;
  if (!S->factored) return fail(ctx, HDG_EINVAL, "hdg_solver_precond_apply: no preconditioner set up for this kind");
  if (r == S->tmp2 || z == S->tmp2) return HDG_EINVAL;
  HDG_ON_DEVICE(ctx, ctx->device);
  prec_rhs<double>(S, transpose != 0, r, z, (cudaStream_t)stream);  // binary64: the public apply
  return ck(ctx, cudaGetLastError(), "preconditioner apply");
}

hdg_status hdg_solver_colors(const hdg_solver* S, int32_t* face_color, int32_t* n_colors) {
  if (!S) return HDG_EINVAL;
  if (face_color) std::memcpy(face_color, S->fcolor.data(), sizeof(int32_t) * S->fcolor.size());
  if (n_colors) *n_colors = (int32_t)S->color_off.size() - 1;
  return HDG_OK;
}

hdg_status hdg_trace_matvec(hdg_solver* S, const double* x, double* y, int32_t transpose, void* stream) {
  if (!S || !x || !y) return HDG_EINVAL;
  HDG_ON_DEVICE(S->sys->ctx, S->sys->ctx->device);
  face_op(S->f, transpose != 0, x, nullptr, y, 2, (cudaStream_t)stream);
  return ck(S->sys->ctx, cudaGetLastError(), "k_face_op");
}

hdg_status hdg_trace_solve(hdg_solver* S, double* x, double rtol, int32_t max_iter, int32_t* iters_out,
                           double* rel_out, void* stream) {
  return hdg_trace_solve_ex(S, nullptr, 0, x, rtol, max_iter, iters_out, rel_out, stream);
}

hdg_status hdg_trace_solve_ex(hdg_solver* S, const double* rhs, int32_t transpose, double* x, double rtol,
                              int32_t max_iter, int32_t* iters_out, double* rel_out, void* stream) {
  hdg::NvtxRange nvtx_range_("hdg::trace_solve");
  if (!S || !x || !(rtol > 0.0) || max_iter < 1) return HDG_EINVAL;
  hdg_ctx* ctx = S->sys->ctx;
  HDG_ON_DEVICE(ctx, ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (iters_out) *iters_out = 0;
  if (rel_out) *rel_out = 0.0;
  const double* E = rhs ? rhs : S->sys->ds.E;
  int it = 0;
  double rel = 1.0;
  hdg_status rs;
  if (S->arith == 1) {
    // the solve runs on float-float copies of E and x; x is written back at the end
    split_copy(S, E, S->eff, S->n, st);
    split_copy(S, x, S->xff, S->n, st);
    rs = gmres<float2>(S, transpose != 0, S->eff, S->xff, rtol, max_iter, it, rel, st);
    if (rs == HDG_OK || rs == HDG_ETIMEOUT) {
      k_join<<<grid_for(S->n, 256, 8 * S->sms), 256, 0, st>>>(S->xff, x, S->n);
      hdg_status r2 = ck(ctx, cudaStreamSynchronize(st), "cudaStreamSynchronize");
      if (r2 != HDG_OK) return r2;
    }
  } else {
    rs = gmres<double>(S, transpose != 0, E, x, rtol, max_iter, it, rel, st);
  }
  if (rs != HDG_OK && rs != HDG_ETIMEOUT) return rs;
  if (iters_out) *iters_out = it;
  if (rel_out) *rel_out = rel;
  return rs;
}

hdg_status hdg_solve_step_host(hdg_sys* sys, hdg_solver* S, const double* U, const double* Lam, double* dU,
                               double* dLam, double rtol, int32_t max_iter, int32_t* iters, double* rel_res,
                               void* stream) {
  hdg::NvtxRange nvtx_range_("hdg::solve_step_host");
  if (!sys || !S) return HDG_EINVAL;
  hdg_ctx* ctx = sys->ctx;
  if (S->sys != sys) return fail(ctx, HDG_EINVAL, "hdg_solve_step_host: the solver belongs to another system");
  if (!U || !Lam || !dU || !dLam) return fail(ctx, HDG_EINVAL, "hdg_solve_step_host: null argument");
  HDG_ON_DEVICE(ctx, ctx->device);
  const hdg_mesh* M = sys->mesh;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t d = sizeof(double);
  hdg_status rs;
  if ((rs = ck(ctx, cudaMemcpyAsync(sys->d_U, U, d * M->u_len, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync")) != HDG_OK)
    return rs;
  if ((rs = ck(ctx, cudaMemcpyAsync(sys->d_Lam, Lam, d * M->lam_len, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync")) != HDG_OK)
    return rs;
  if ((rs = hdg_condense(sys, sys->d_U, sys->d_Lam, stream)) != HDG_OK) return rs;
  if ((rs = ck(ctx, cudaMemsetAsync(sys->d_dLam, 0, d * M->lam_len, st), "cudaMemsetAsync")) != HDG_OK) return rs;
  if ((rs = hdg_trace_solve_ex(S, nullptr, 0, sys->d_dLam, rtol, max_iter, iters, rel_res, stream)) != HDG_OK)
    return rs;
  if ((rs = hdg_recover(sys, sys->d_dLam, sys->d_dU, stream)) != HDG_OK) return rs;
  if ((rs = ck(ctx, cudaMemcpyAsync(dU, sys->d_dU, d * M->u_len, cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync")) != HDG_OK)
    return rs;
  if ((rs = ck(ctx, cudaMemcpyAsync(dLam, sys->d_dLam, d * M->lam_len, cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync")) != HDG_OK)
    return rs;
  return ck(ctx, cudaStreamSynchronize(st), "cudaStreamSynchronize");
}

hdg_status hdg_newton_update(hdg_sys* sys, double* U, double* Lam, const double* dU, const double* dLam,
                             void* stream) {
  if (!sys || !U || !Lam || !dU || !dLam) return HDG_EINVAL;
  HDG_ON_DEVICE(sys->ctx, sys->ctx->device);
  const hdg_mesh* M = sys->mesh;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, sys->ctx->device);
  k_axpy2<<<grid_for(M->u_len + M->lam_len, 256, 8 * sms), 256, 0, (cudaStream_t)stream>>>(U, dU, M->u_len, Lam,
                                                                                               dLam, M->lam_len);
  return ck(sys->ctx, cudaGetLastError(), "k_axpy2");
}

hdg_status hdg_residual_norm(hdg_sys* sys, double* norm, void* stream) {
  if (!sys || !norm) return HDG_EINVAL;
  hdg_ctx* ctx = sys->ctx;
  HDG_ON_DEVICE(ctx, ctx->device);
  const hdg_mesh* M = sys->mesh;
  cudaStream_t st = (cudaStream_t)stream;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  const int64_t nmax = std::max(M->u_len, M->lam_len);
  const int nb = std::max(1, std::min<int>(2 * sms, (int)((nmax + kDotThreads - 1) / kDotThreads)));
  double *part = nullptr, *out = nullptr, hout[2];
  hdg_status rs;
  if ((rs = ck(ctx, cudaMallocAsync((void**)&part, sizeof(double) * (2 * nb + 2), st), "cudaMallocAsync")) != HDG_OK) return rs;
  out = part + 2 * nb;
  k_multidot<<<dim3(nb, 1), kDotThreads, 0, st>>>(sys->ds.res_u, M->u_len, 1, sys->ds.res_u, M->u_len, part);
  k_reduce<<<1, kDotThreads, 0, st>>>(part, nb, out);
  k_multidot<<<dim3(nb, 1), kDotThreads, 0, st>>>(sys->ds.res_lam, M->lam_len, 1, sys->ds.res_lam, M->lam_len, part + nb);
  k_reduce<<<1, kDotThreads, 0, st>>>(part + nb, nb, out + 1);
  rs = ck(ctx, cudaMemcpyAsync(hout, out, sizeof(hout), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
  cudaFreeAsync(part, st);
  if (rs != HDG_OK) return rs;
  if ((rs = ck(ctx, cudaStreamSynchronize(st), "cudaStreamSynchronize")) != HDG_OK) return rs;
  *norm = std::sqrt(hout[0] + hout[1]);
  return HDG_OK;
}

hdg_status hdg_sys_set_cfl(hdg_sys* sys, double cfl) {
  if (!sys || !std::isfinite(cfl)) return HDG_EINVAL;
  if (sys->gexec) return fail(sys->ctx, HDG_EINVAL, "hdg_sys_set_cfl: a captured graph holds the parameters");
  sys->prm.cfl = cfl;
  sys->ph.cfl = cfl;
  return HDG_OK;
}

hdg_status hdg_sys_set_source(hdg_sys* sys, const double* S) {
  if (!sys) return HDG_EINVAL;
  if (sys->gexec) return fail(sys->ctx, HDG_EINVAL, "hdg_sys_set_source: a captured graph holds the parameters");
  sys->ds.src = S;
  return HDG_OK;
}

double hdg_cfl_law(int32_t n, double c0, double c1, int32_t n0, double cfl_prev, double res_prev, double res_cur) {
  if (n < 0 || n0 < 1) return -1.0;
  if (n <= n0) {
    const double t = (double)n / (double)n0;
    return c0 * (3.0 * t * t - 2.0 * t * t * t);
  }
  if (!(res_prev > 0.0) || !(res_cur > 0.0)) return -1.0;
  return cfl_prev * (1.0 + c1 * std::max(0.0, std::log(res_prev / res_cur)));
}

}  // extern "C"
