// Global trace solve K dLambda = E (paper Sec. 3.4, Eq. hybridsystem) and the
// pseudo-transient Newton update (Sec. 3.3) on the GPU.
//
// The paper uses ILU(n)-preconditioned GMRES from PETSc on the CPU.  Here:
// restarted GMRES, left-preconditioned, binary64 throughout, with one of
//   0 block Jacobi (the inverses of K's diagonal face blocks),
//   1 multicolor block symmetric Gauss-Seidel,
//   2 block ILU(0) in the multicolor order of the faces (faces of one color
//     share no element, so their rows are uncoupled: each color is factored,
//     and swept in the triangular solves, by one launch).
// Kernels:
//   k_bj_invert   one warp per face: Gauss-Jordan with partial pivoting of the
//                 face's diagonal block (m = 4 (p_e + 1) <= 20 rows);
//   k_ilu_row     one warp per face of one color: the face's block row of the
//                 incomplete factors, then the inverse of its pivot block;
//   k_face_op     one warp per face: t = (K x)_e (each block staged through
//                 shared memory with coalesced loads, one lane per row, the
//                 five blocks of the face row in column order; optionally only
//                 the blocks of earlier or of later colors), then, by mode,
//                 y_e = t, Dinv_e t, Dinv_e (b_e - t), Dinv_e b_e or b_e - t;
//   k_dots_slab   dot products of one vector with the Krylov vectors, one
//                 contiguous slab of rows per block, vectors over its warps;
//                 k_reduce sums the per-block partials in a fixed order
//                 (bitwise reproducible);
//   k_axpy_v      w -= V c (c on the device), fused with ||w||^2 for the
//                 second Gram-Schmidt pass (reduced by the last block to
//                 finish, in a fixed order);
//   k_multiaxpy   x += V y at the end of a restart cycle.
// The Arnoldi process uses classical Gram-Schmidt with one
// re-orthogonalisation pass; the small Hessenberg
// least-squares problem (Givens rotations) is solved on the host, one residual
// estimate read back per iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "hdg_internal.h"
#include "hdg_objects.h"

using namespace hdg;

namespace {

constexpr int kMaxRestart = 64;
constexpr int kFaceWarps = 4;          // faces per CTA in the per-face kernels
constexpr int kMaxM = 4 * (kMaxP + 1);  // largest face block (20)
constexpr int kDotThreads = 256;
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

template <class VT>
__device__ void load_aug(VT (*a)[2 * kMaxM + 1], const VT* D, int m, int lane) {
  const int m2 = 2 * m;
  for (int t = lane; t < m * m2; t += 32) {
    const int r = t / m2, c = t - r * m2;
    a[r][c] = (c < m) ? D[r * m + c] : (c - m == r ? (VT)1 : (VT)0);
  }
  __syncwarp();
}

template <class VT>
__device__ void store_inverse(VT (*a)[2 * kMaxM + 1], VT* out, int m, int lane) {
  for (int t = lane; t < m * m; t += 32) {
    const int r = t / m, c = t - r * m;
    out[t] = a[r][m + c];
  }
}

__global__ void __launch_bounds__(32 * kFaceWarps) k_bj_invert(FaceDev f) {
  __shared__ double s_aug[kFaceWarps][kMaxM][2 * kMaxM + 1];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * kFaceWarps + w;
  if (e >= f.n_face) return;
  const int m = 4 * (f.face_p[e] + 1);
  int b = 0;
  while (b < 4 && f.k_col[5 * e + b] != e) ++b;
  double(*a)[2 * kMaxM + 1] = s_aug[w];
  load_aug(a, f.K + f.k_blkoff[5 * e + b], m, lane);
  if (!warp_gj_invert(a, m, lane)) {
    if (lane == 0) *f.bad = 1;
    return;  // the whole warp leaves together
  }
  store_inverse(a, f.dinv + f.dinv_off[e], m, lane);
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

// w[i] += sgn * sum_j c[j] V_j[i]
__global__ void k_multiaxpy(const double* __restrict__ V, int64_t ldv, int nvec, const double* __restrict__ c,
                            double sgn, double* __restrict__ w, int64_t n) {
  __shared__ double s_c[kMaxRestart + 1];
  for (int j = threadIdx.x; j < nvec; j += blockDim.x) s_c[j] = sgn * c[j];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double a = w[i];
    for (int j = 0; j < nvec; ++j) a = fma(s_c[j], V[(int64_t)j * ldv + i], a);
    w[i] = a;
  }
}

__global__ void k_scale(double* __restrict__ v, double s, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] *= s;
}

// ---------------------------------------------------------------- Krylov kernels
// Vectors of the trace space have an even length (4 (p_e + 1) per face) and
// start 32-byte aligned, so they are read as double2.  The norm fused into
// the second Gram-Schmidt update is reduced in one launch: warp shuffles, the
// warps of a block in order, one partial per block, and the last block to
// finish (a ticket taken after a fence) sums the partials in a fixed order and
// resets the ticket -- bitwise reproducible.

// out[j] = sum over blocks of part[j][b], j < nout (called by the last block only):
// every thread takes a strided share of the partials, then a fixed-order tree
__device__ void finish_reduction(const double* part, int nout, int nblk, double* out, unsigned* ticket) {
  __shared__ double s_fin[kDotThreads];
  for (int j = 0; j < nout; ++j) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) v += __ldcg(part + (int64_t)j * nblk + b);
    s_fin[threadIdx.x] = v;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) s_fin[threadIdx.x] += s_fin[threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = s_fin[0];
    __syncthreads();
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

// block-wide sum of acc[0..nj) into part[j0 + j][blockIdx] (blockIdx flattened over x), then
// the last block finishes every output; returns nothing useful to the caller
template <int NA>
__device__ void block_partials(const double (&acc)[NA], int nj, int j0, double* part, int nout, int nblk,
                               double* out, unsigned* ticket) {
  __shared__ double s_red[NA][kDotThreads / 32];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    double v = acc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[j][wp] = v;
  }
  __syncthreads();
  if (threadIdx.x < nj) {
    double v = 0.0;
    for (int k = 0; k < nw; ++k) v += s_red[threadIdx.x][k];
    part[(int64_t)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x * gridDim.y - 1;
  __syncthreads();
  if (s_last) {
    __threadfence();
    finish_reduction(part, nout, nblk, out, ticket);
  }
}

// part[j][block] = V_j . w over the block's slab of rows, j < nvec: each block
// owns a contiguous slab (its slice of w stays in L1 while its warps stream
// their vectors: warp k takes vectors k, k + 8, ..., four at a time, two
// double2 rows per lane in flight for each); k_reduce sums the partials.
__global__ void __launch_bounds__(kDotThreads) k_dots_slab(const double* __restrict__ V, int64_t ldv, int nvec,
                                                           const double* __restrict__ w, int64_t n,
                                                           double* __restrict__ part) {
  constexpr int NW = kDotThreads / 32, VPW = 4;  // warps per block, vectors per warp per sweep
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int64_t n2 = n >> 1;
  const int64_t per = (n2 + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = min(n2, (int64_t)blockIdx.x * per), b1 = min(n2, b0 + per);
  const double2* w2 = reinterpret_cast<const double2*>(w);
  for (int jb = wp; jb < nvec; jb += NW * VPW) {
    const double2* v2[VPW];
    double acc[VPW];
#pragma unroll
    for (int k = 0; k < VPW; ++k) {
      const int j = min(jb + k * NW, nvec - 1);
      v2[k] = reinterpret_cast<const double2*>(V + (int64_t)j * ldv);
      acc[k] = 0.0;
    }
    for (int64_t i = b0 + lane; i < b1; i += 64) {
      const bool two = i + 32 < b1;
      const double2 wa = __ldg(w2 + i);
      const double2 wb = two ? __ldg(w2 + i + 32) : make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < VPW; ++k) {
        if (jb + k * NW >= nvec) break;  // slot without a vector (warp-uniform): no loads, no FMAs
        const double2 a = __ldg(v2[k] + i);
        const double2 b = two ? __ldg(v2[k] + i + 32) : make_double2(0.0, 0.0);
        acc[k] = fma(a.x, wa.x, acc[k]);
        acc[k] = fma(a.y, wa.y, acc[k]);
        acc[k] = fma(b.x, wb.x, acc[k]);
        acc[k] = fma(b.y, wb.y, acc[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < VPW; ++k) {
      double v = acc[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      const int j = jb + k * NW;
      if (lane == 0 && j < nvec) {
        if (blockIdx.x == 0 && (n & 1)) v = fma(V[(int64_t)j * ldv + n - 1], w[n - 1], v);  // odd tail
        part[(int64_t)j * gridDim.x + blockIdx.x] = v;
      }
    }
  }
}

// w -= V c (j < nvec, c on the device); with NORM, out[0] = ||w||^2 of the updated w
template <bool NORM>
__global__ void __launch_bounds__(kDotThreads) k_axpy_v(const double* __restrict__ V, int64_t ldv, int nvec,
                                                        const double* __restrict__ c, double* __restrict__ w,
                                                        int64_t n, double* __restrict__ part,
                                                        double* __restrict__ out, unsigned* ticket) {
  __shared__ double s_c[kMaxRestart + 1];
  for (int j = threadIdx.x; j < nvec; j += blockDim.x) s_c[j] = c[j];
  __syncthreads();
  double acc[1] = {0.0};
  const int64_t n2 = n >> 1;
  double2* w2 = reinterpret_cast<double2*>(w);
  for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < n2; i += (int64_t)gridDim.x * kDotThreads) {
    double2 a = w2[i];
    for (int j = 0; j < nvec; ++j) {
      const double2 v = __ldg(reinterpret_cast<const double2*>(V + (int64_t)j * ldv) + i);
      a.x = fma(-s_c[j], v.x, a.x);
      a.y = fma(-s_c[j], v.y, a.y);
    }
    w2[i] = a;
    if (NORM) {
      acc[0] = fma(a.x, a.x, acc[0]);
      acc[0] = fma(a.y, a.y, acc[0]);
    }
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    double a = w[n - 1];
    for (int j = 0; j < nvec; ++j) a = fma(-s_c[j], V[(int64_t)j * ldv + n - 1], a);
    w[n - 1] = a;
    if (NORM) acc[0] = fma(a, a, acc[0]);
  }
  if (NORM) block_partials<1>(acc, 1, 0, part, 1, gridDim.x, out, ticket);
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
  double* V = nullptr;        // [restart + 1][n]
  double* partial = nullptr;  // [restart + 1][dot_blocks]
  unsigned* ticket = nullptr; // last-block ticket of the fused reductions (zero between launches)
  double* h = nullptr;        // [2 (restart + 1) + 2] device results of the reductions
  double* coef = nullptr;     // [restart + 1] coefficients from the host
  double* zero = nullptr;     // [n] zeros
  double* tmp = nullptr;      // [n] work vector of the Gauss-Seidel and ILU preconditioners
  double* tmp2 = nullptr;     // [n] second work vector of the ILU preconditioner
  double* hpin = nullptr;     // pinned host mirror of h / coef
  int precond = 0;            // 0 block Jacobi, 1 multicolor block SGS, 2 block ILU(0), 3 ILU(0) in binary32
  bool factored = false;      // a setup has been enqueued for the current kind
  int* colors = nullptr;      // faces grouped by color
  std::vector<int> color_off; // [n_colors + 1]
  std::vector<int> fcolor;    // host copy of the face colors
  FaceDev fi{};               // the ILU factors: values F (K's layout) and pivot inverses
  double* F = nullptr;
  FaceDevT<float> fi32{};     // the same in binary32 (mixed-precision ILU(0), kind 3)
  float* F32 = nullptr;
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

// z = M^{-1} r for the multicolor block symmetric Gauss-Seidel preconditioner:
// from z = 0, a forward sweep over the colors, then a backward one; each color
// is one launch (its faces are mutually uncoupled, so the sweep is exact Gauss-Seidel).
void sgs_apply(hdg_solver* S, bool tr, const double* r, double* z, cudaStream_t st) {
  cudaMemsetAsync(z, 0, sizeof(double) * S->n, st);
  const int nc = (int)S->color_off.size() - 1;
  for (int pass = 0; pass < 2; ++pass)
    for (int k = 0; k < nc; ++k) {
      const int c = pass == 0 ? k : nc - 1 - k;
      const int o0 = S->color_off[c], o1 = S->color_off[c + 1];
      face_op(S->f, tr, z, r, z, 1, st, S->colors + o0, o1 - o0, 1);
    }
}

// z = (L U)^{-1} r, or (L U)^{-T} r, with the block ILU(0) factors: a forward
// sweep over the colors into tmp2 (L y = r: y_e = r_e - sum of L_ek y_k over
// earlier colors; transposed, U^T y = r), then a backward one into z
// (U z = y: z_e = U_ee^{-1} (y_e - sum of U_ej z_j over later colors;
// transposed, L^T z = y).  r and z must not be tmp2.
template <class MT>
void ilu_sweeps(hdg_solver* S, const FaceDevT<MT>& fi, bool tr, const double* r, double* z, cudaStream_t st) {
  const int nc = (int)S->color_off.size() - 1;
  for (int c = 0; c < nc; ++c) {
    const int o0 = S->color_off[c], o1 = S->color_off[c + 1];
    face_op(fi, tr, S->tmp2, r, S->tmp2, tr ? 1 : 4, st, S->colors + o0, o1 - o0, 0, 1);
  }
  for (int c = nc - 1; c >= 0; --c) {
    const int o0 = S->color_off[c], o1 = S->color_off[c + 1];
    face_op(fi, tr, z, S->tmp2, z, tr ? 4 : 1, st, S->colors + o0, o1 - o0, 0, 2);
  }
}
void ilu_apply(hdg_solver* S, bool tr, const double* r, double* z, cudaStream_t st) {
  if (S->precond == 3) ilu_sweeps(S, S->fi32, tr, r, z, st);  // binary32 factors, binary64 products
  else ilu_sweeps(S, S->fi, tr, r, z, st);
}

// w = M^{-1} b for the solver's preconditioner
void prec_rhs(hdg_solver* S, bool tr, const double* b, double* w, cudaStream_t st) {
  if (S->precond == 0) face_op(S->f, tr, S->zero, b, w, 3, st);
  else if (S->precond == 1) sgs_apply(S, tr, b, w, st);
  else ilu_apply(S, tr, b, w, st);
}
// w = M^{-1} K v (block Jacobi: one fused launch)
void prec_op(hdg_solver* S, bool tr, const double* v, double* w, cudaStream_t st) {
  if (S->precond == 0) {
    face_op(S->f, tr, v, nullptr, w, 0, st);
  } else {
    face_op(S->f, tr, v, nullptr, S->tmp, 2, st);
    prec_rhs(S, tr, S->tmp, w, st);
  }
}
// w = M^{-1} (b - K x)
void prec_res(hdg_solver* S, bool tr, const double* x, const double* b, double* w, cudaStream_t st) {
  if (S->precond == 0) {
    face_op(S->f, tr, x, b, w, 1, st);
  } else {
    face_op(S->f, tr, x, b, S->tmp, 4, st);
    prec_rhs(S, tr, S->tmp, w, st);
  }
}

// the binary32 factor view: K's layout and tables, values and pivot inverses in binary32
void set_fi32(hdg_solver* S, float* dinv32) {
  const FaceDev& f = S->f;
  S->fi32.n_face = f.n_face;
  S->fi32.face_p = f.face_p;
  S->fi32.lam_off = f.lam_off;
  S->fi32.k_col = f.k_col;
  S->fi32.k_blkoff = f.k_blkoff;
  S->fi32.dinv_off = f.dinv_off;
  S->fi32.k_tblk = f.k_tblk;
  S->fi32.fcolor = f.fcolor;
  S->fi32.K = S->F32;
  S->fi32.dinv = dinv32;
  S->fi32.bad = f.bad;
}

// enqueue the factorization of the preconditioner for the current K; a
// singular pivot block sets f.bad (cleared first)
hdg_status setup_enqueue(hdg_solver* S, cudaStream_t st) {
  hdg_ctx* ctx = S->sys->ctx;
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
  } else {
    k_bj_invert<<<(S->f.n_face + kFaceWarps - 1) / kFaceWarps, 32 * kFaceWarps, 0, st>>>(S->f);
  }
  if ((rs = ck(ctx, cudaGetLastError(), "preconditioner setup")) != HDG_OK) return rs;
  S->factored = true;
  return HDG_OK;
}

// out[0..nvec) = V_j . w for j < nvec (device), one launch, enqueued on st
void multidot(hdg_solver* S, const double* V, int nvec, const double* w, int64_t n, double* out, cudaStream_t st) {
  k_dots_slab<<<S->dot_blocks, kDotThreads, 0, st>>>(V, S->n, nvec, w, n, S->partial);
  k_reduce<<<nvec, kDotThreads, 0, st>>>(S->partial, S->dot_blocks, out);
}
// w -= V c (nvec columns); with norm2 != null also norm2[0] = ||w||^2 afterwards
void axpy_v(hdg_solver* S, const double* V, int nvec, const double* c, double* w, int64_t n, double* norm2,
            cudaStream_t st) {
  if (norm2) k_axpy_v<true><<<S->dot_blocks, kDotThreads, 0, st>>>(V, S->n, nvec, c, w, n, S->partial, norm2, S->ticket);
  else k_axpy_v<false><<<S->dot_blocks, kDotThreads, 0, st>>>(V, S->n, nvec, c, w, n, S->partial, nullptr, S->ticket);
}

}  // namespace

namespace {

// Byte offsets of the solver's device buffers in one workspace (256-byte aligned).
struct SolverPlan {
  int64_t n = 0, dinv_len = 0, k_vals = 0;
  int dot_blocks = 0;
  size_t kc, kb, kt, dof, dinv, bad, ticket, V, part, h, coef, zero, tmp, cols, fcol, F, dinv2, tmp2, total;
};

SolverPlan plan_solver(const hdg_mesh* M, int restart, int precond, int sms) {
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
  p.dot_blocks = std::max(1, std::min<int>(2 * std::max(sms, 1), (int)((p.n / 2 + kDotThreads - 1) / kDotThreads)));
  p.kc = take(sizeof(int) * 5 * nf);
  p.kb = take(sizeof(int64_t) * M->k_blkoff.size());
  p.kt = take(sizeof(int64_t) * 5 * nf);
  p.dof = take(sizeof(int64_t) * nf);
  p.dinv = take(sizeof(double) * p.dinv_len);
  p.bad = take(sizeof(int));
  p.ticket = take(sizeof(unsigned));
  p.V = take(sizeof(double) * nr * p.n);
  p.part = take(sizeof(double) * nr * p.dot_blocks);
  p.h = take(sizeof(double) * (2 * nr + 2));
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
  p.total = o;
  return p;
}

}  // namespace

extern "C" hdg_status hdg_solver_destroy(hdg_solver* S);

namespace {

// Plan, place (one cudaMalloc, or the caller's workspace) and fill the solver's state.
hdg_status solver_build(hdg_sys* sys, int32_t restart, int32_t precond, void* ws, int64_t ws_bytes,
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
  const SolverPlan P = plan_solver(M, restart, precond, sms);
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
    S->hpin = new double[2 * nr + 2];
    S->hpin_pageable = true;
  } else if (cudaMallocHost((void**)&S->hpin, sizeof(double) * (2 * nr + 2)) != cudaSuccess) {
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
  if (st == HDG_OK) st = ck(ctx, cudaMemset(base + P.ticket, 0, sizeof(unsigned)), "cudaMemset");
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
  *out = S;
  return HDG_OK;
}

}  // namespace

extern "C" {

hdg_status hdg_solver_create(hdg_sys* sys, int32_t restart, hdg_solver** out) {
  return solver_build(sys, restart, 0, nullptr, 0, out);
}

hdg_status hdg_solver_create_ws(hdg_sys* sys, int32_t restart, int32_t precond, void* workspace, int64_t bytes,
                                hdg_solver** out) {
  if (!workspace) return HDG_EINVAL;
  return solver_build(sys, restart, precond, workspace, bytes, out);
}

int64_t hdg_solver_workspace_bytes(const hdg_mesh* mesh, int32_t restart, int32_t precond) {
  if (!mesh || restart < 1 || restart > kMaxRestart || precond < 0 || precond > 3) return -1;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, mesh->ctx->device) != cudaSuccess) return -1;
  return (int64_t)plan_solver(mesh, restart, precond, sms).total;
}

hdg_status hdg_solver_destroy(hdg_solver* S) {
  if (!S) return HDG_EINVAL;
  hdg::DeviceGuard dg(S->sys->ctx->device);
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
  if (kind != S->precond) S->factored = false;
  S->precond = kind;
  return HDG_OK;
}

hdg_status hdg_solver_setup(hdg_solver* S, void* stream) {
  hdg::NvtxRange nvtx_range_("hdg::solver_setup");
  if (!S) return HDG_EINVAL;
  hdg_ctx* ctx = S->sys->ctx;
  HDG_ON_DEVICE(ctx, ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  hdg_status rs;
  if ((rs = setup_enqueue(S, st)) != HDG_OK) return rs;
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
  prec_rhs(S, transpose != 0, r, z, (cudaStream_t)stream);
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
  const bool tr = transpose != 0;
  hdg_ctx* ctx = S->sys->ctx;
  HDG_ON_DEVICE(ctx, ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = S->n;
  const int R = S->restart;
  const int vb = grid_for(n, 256, 8 * S->sms);
  hdg_status rs;
  if (iters_out) *iters_out = 0;
  if (rel_out) *rel_out = 0.0;
  // the preconditioner's factors of the current K
  if ((rs = setup_enqueue(S, st)) != HDG_OK) return rs;
  // ||M^-1 E||
  const double* E = rhs ? rhs : S->sys->ds.E;
  prec_rhs(S, tr, E, S->V, st);
  multidot(S, S->V, 1, S->V, n, S->h, st);
  int bad = 0;
  if ((rs = ck(ctx, cudaMemcpyAsync(S->hpin, S->h, sizeof(double), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync")) != HDG_OK) return rs;
  if ((rs = ck(ctx, cudaMemcpyAsync(&S->hpin[1], S->f.bad, sizeof(int), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync")) != HDG_OK) return rs;
  if ((rs = ck(ctx, cudaStreamSynchronize(st), "cudaStreamSynchronize")) != HDG_OK) return rs;
  std::memcpy(&bad, &S->hpin[1], sizeof(int));
  if (bad) {
    S->factored = false;
    return fail(ctx, HDG_ESINGULAR, "hdg_trace_solve: a pivot block of the preconditioner is singular");
  }
  const double bnorm = std::sqrt(S->hpin[0]);
  if (!(bnorm > 0.0)) {  // E = 0: the solution is 0
    if ((rs = ck(ctx, cudaMemsetAsync(x, 0, sizeof(double) * n, st), "cudaMemsetAsync")) != HDG_OK) return rs;
    return ck(ctx, cudaStreamSynchronize(st), "cudaStreamSynchronize");
  }
  std::vector<double> H((size_t)(R + 1) * R), cs(R), sn(R), g(R + 1), y(R);
  int it = 0;
  double rel = 1.0;
  while (true) {
    // r0 = M^-1 (E - K x), beta = ||r0||
    prec_res(S, tr, x, E, S->V, st);
    multidot(S, S->V, 1, S->V, n, S->h, st);
    if ((rs = ck(ctx, cudaMemcpyAsync(S->hpin, S->h, sizeof(double), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync")) != HDG_OK) return rs;
    if ((rs = ck(ctx, cudaStreamSynchronize(st), "cudaStreamSynchronize")) != HDG_OK) return rs;
    const double beta = std::sqrt(S->hpin[0]);
    rel = beta / bnorm;
    if (!(rel > rtol) || it >= max_iter) break;
    k_scale<<<vb, 256, 0, st>>>(S->V, 1.0 / beta, n);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jn = 0;  // columns of H built in this cycle
    for (int j = 0; j < R && it < max_iter; ++j) {
      double* vj = S->V + (int64_t)j * n;
      double* w = S->V + (int64_t)(j + 1) * n;
      prec_op(S, tr, vj, w, st);
      // classical Gram-Schmidt, twice (the second pass fused with ||w||^2); a
      // reorthogonalise-when-needed test (Daniel et al., ||w'||^2 < ||w||^2 / 2)
      // fires in almost every iteration of these trace systems, so both passes
      // always run and one read-back per iteration suffices
      multidot(S, S->V, j + 1, w, n, S->h, st);
      axpy_v(S, S->V, j + 1, S->h, w, n, nullptr, st);
      multidot(S, S->V, j + 1, w, n, S->h + (R + 1), st);
      axpy_v(S, S->V, j + 1, S->h + (R + 1), w, n, S->h + 2 * (R + 1), st);
      if ((rs = ck(ctx, cudaMemcpyAsync(S->hpin, S->h, sizeof(double) * (2 * (R + 1) + 1), cudaMemcpyDeviceToHost, st),
                   "cudaMemcpyAsync")) != HDG_OK)
        return rs;
      if ((rs = ck(ctx, cudaStreamSynchronize(st), "cudaStreamSynchronize")) != HDG_OK) return rs;
      ++it;
      double* col = &H[(size_t)j * (R + 1)];  // column j of H, rows 0..j+1
      for (int i = 0; i <= j; ++i) col[i] = S->hpin[i] + S->hpin[(R + 1) + i];
      const double hn = std::sqrt(S->hpin[2 * (R + 1)]);
      col[j + 1] = hn;
      for (int i = 0; i < j; ++i) {  // earlier rotations
        const double a = col[i], b = col[i + 1];
        col[i] = cs[i] * a + sn[i] * b;
        col[i + 1] = -sn[i] * a + cs[i] * b;
      }
      const double den = std::hypot(col[j], col[j + 1]);
      cs[j] = den > 0.0 ? col[j] / den : 1.0;
      sn[j] = den > 0.0 ? col[j + 1] / den : 0.0;
      col[j] = den;
      col[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      jn = j + 1;
      rel = std::fabs(g[j + 1]) / bnorm;
      if (!(rel > rtol) || !(hn > 0.0)) break;
      k_scale<<<vb, 256, 0, st>>>(w, 1.0 / hn, n);
    }
    // x += V y, H y = g (upper triangular)
    for (int i = jn - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < jn; ++k) s -= H[(size_t)k * (R + 1) + i] * y[k];
      y[i] = s / H[(size_t)i * (R + 1) + i];
    }
    std::memcpy(S->hpin, y.data(), sizeof(double) * jn);
    if ((rs = ck(ctx, cudaMemcpyAsync(S->coef, S->hpin, sizeof(double) * jn, cudaMemcpyHostToDevice, st),
                 "cudaMemcpyAsync")) != HDG_OK)
      return rs;
    k_multiaxpy<<<vb, 256, 0, st>>>(S->V, n, jn, S->coef, 1.0, x, n);
    // the pinned buffer is reused next cycle: wait for the copy
    if ((rs = ck(ctx, cudaStreamSynchronize(st), "cudaStreamSynchronize")) != HDG_OK) return rs;
  }
  if ((rs = ck(ctx, cudaGetLastError(), "trace solve kernels")) != HDG_OK) return rs;
  if (iters_out) *iters_out = it;
  if (rel_out) *rel_out = rel;
  return (rel > rtol) ? fail(ctx, HDG_ETIMEOUT, "hdg_trace_solve: max_iter reached before rtol") : HDG_OK;
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
