// Mixed-precision local solve of one element (Sec. 3.4, X = A^{-1}[B | F]):
// LU with partial pivoting of a binary32 copy of A whose rank-8 updates run on
// the tensor cores (warp-level mma.sync, binary32 accumulation), and iterative
// refinement of X against residuals [B | F] - A X formed in the element's own
// arithmetic T (binary64), so the refined X reaches the accuracy of T.
//
// Tensor-core forms of the rank-8 update C -= L U (16 x 8 output tiles, K = 8):
//   kTcTF32x3: each binary32 operand split as hi + lo, hi = its TF32 rounding and
//              lo = the TF32 rounding of the rest; C -= Lhi Uhi + Lhi Ulo + Llo Uhi
//              (three TF32 MMAs, about binary32 accuracy);
//   kTcBF16:   one BF16 MMA (8-bit significands): the cheapest and least accurate
//              update; refinement then needs many more sweeps.
// Why mma.sync and not tcgen05: the operands are one element's 12..60-row
// blocks resident in shared memory and consumed at once; tcgen05.mma needs
// M >= 64 tiles, descriptors over canonical shared-memory layouts and a TMEM
// round trip per update, for matrices that a warp-level 16 x 8 tile covers.
//
// Refinement (classical mixed-precision iterative refinement): X_0 = 0;
// sweep s: W = fl32(R - A X_s) (the residual in T), W <- LU^{-1} W (binary32,
// tensor cores), X_{s+1} = X_s + W (in T); it stops after the first sweep
// s >= 1 whose correction is below tol * max|X|, or after refine_max
// corrections (then bit 4 of *s_bad: element status 3, not converged).
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "hdg_arith.cuh"

namespace hdg {

constexpr int kTcTF32x3 = 1;
constexpr int kTcBF16 = 2;

__device__ __forceinline__ uint32_t tc_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void tc_mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void tc_mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(b0));
}

// two binary32 values as a bf16x2 register: `lo` in the low half (the smaller index)
__device__ __forceinline__ uint32_t tc_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// C[m x n] -= L[m x kw] * B[kw x n] (row-major, strides ldc, ldl, ldb; kw <= 8) by
// 16 x 8 tiles, warps `warp` of `nwarps` taking tiles in turn.  Operands outside
// [0, m) x [0, kw) / [0, kw) x [0, n) read as zero; C outside [0, m) x [0, n)
// is neither read nor written.  Fragment layouts of mma.m16n8k8 (lane = 4 g + t):
// A(g|g+8, t|t+4) (tf32) or A(g|g+8, 2t..2t+1) (bf16), B(t|t+4, g) (tf32) or
// B(2t..2t+1, g) (bf16), C(g|g+8, 2t..2t+1).
template <int MODE>
__device__ __forceinline__ void tc_update(float* C, int ldc, int m, int n, const float* L, int ldl, const float* B,
                                          int ldb, int kw, int warp, int nwarps, int lane) {
  const int g = lane >> 2, t = lane & 3;
  const int tr = (m + 15) >> 4, tcn = (n + 7) >> 3;
  for (int tile = warp; tile < tr * tcn; tile += nwarps) {
    const int r0 = (tile / tcn) << 4, c0 = (tile % tcn) << 3;
    const int ra = r0 + g, rb = ra + 8, ca = c0 + 2 * t, cb = ca + 1;
    // -L (so that the MMA's D = A B + C subtracts), zero outside the block
    auto lv = [&](int r, int k) -> float { return (r < m && k < kw) ? -L[r * ldl + k] : 0.0f; };
    auto bv = [&](int k, int c) -> float { return (k < kw && c < n) ? B[k * ldb + c] : 0.0f; };
    float c[4];
    c[0] = (ra < m && ca < n) ? C[ra * ldc + ca] : 0.0f;
    c[1] = (ra < m && cb < n) ? C[ra * ldc + cb] : 0.0f;
    c[2] = (rb < m && ca < n) ? C[rb * ldc + ca] : 0.0f;
    c[3] = (rb < m && cb < n) ? C[rb * ldc + cb] : 0.0f;
    if constexpr (MODE == kTcTF32x3) {
      const float av[4] = {lv(ra, t), lv(rb, t), lv(ra, t + 4), lv(rb, t + 4)};
      const float bw[2] = {bv(t, c0 + g), bv(t + 4, c0 + g)};
      uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ah[i] = tc_tf32(av[i]);
        al[i] = tc_tf32(av[i] - __uint_as_float(ah[i]));
      }
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        bh[i] = tc_tf32(bw[i]);
        bl[i] = tc_tf32(bw[i] - __uint_as_float(bh[i]));
      }
      tc_mma_tf32(c, al, bh);  // the small terms first
      tc_mma_tf32(c, ah, bl);
      tc_mma_tf32(c, ah, bh);
    } else {
      const uint32_t a0 = tc_bf16x2(lv(ra, 2 * t), lv(ra, 2 * t + 1));
      const uint32_t a1 = tc_bf16x2(lv(rb, 2 * t), lv(rb, 2 * t + 1));
      const uint32_t b0 = tc_bf16x2(bv(2 * t, c0 + g), bv(2 * t + 1, c0 + g));
      tc_mma_bf16(c, a0, a1, b0);
    }
    if (ra < m && ca < n) C[ra * ldc + ca] = c[0];
    if (ra < m && cb < n) C[ra * ldc + cb] = c[1];
    if (rb < m && ca < n) C[rb * ldc + ca] = c[2];
    if (rb < m && cb < n) C[rb * ldc + cb] = c[3];
  }
}

constexpr int kTcNB = 8;  // panel width = the MMA's K

// LU with partial pivoting of fA (N x N binary32, stride lda) in place: L unit
// lower, U upper; piv[k] = the row exchanged with row k at step k; pinv[k] =
// 1 / U(k, k).  Panels of 8 columns factored by one warp (pivot search on |a|
// as integer keys, first maximal row on ties), the panel's exchanges and
// U12 = L11^{-1} A12 one thread per column, the trailing update on the tensor
// cores.  A zero pivot sets bit 1 of *s_bad.
template <int N, int NT, int MODE>
__device__ void tc_lu_factor(float* fA, int lda, int* piv, float* pinv, int* s_bad, int tid) {
  static_assert(N <= 64, "the pivot search holds at most two rows per lane");
  constexpr int NW = NT / 32;
  const int tx = tid & 31, ty = tid >> 5;
  for (int k0 = 0; k0 < N; k0 += kTcNB) {
    const int nb = (N - k0 < kTcNB) ? N - k0 : kTcNB, kend = k0 + nb;
    if (ty == (k0 / kTcNB) % NW) {
      for (int j = k0; j < kend; ++j) {
        const int i1 = j + tx, i2 = j + tx + 32;
        const unsigned k1 = i1 < N ? __float_as_uint(fabsf(fA[i1 * lda + j])) : 0u;
        const unsigned k2 = i2 < N ? __float_as_uint(fabsf(fA[i2 * lda + j])) : 0u;
        const unsigned best = __reduce_max_sync(0xffffffffu, k1 > k2 ? k1 : k2);
        const unsigned b1 = __ballot_sync(0xffffffffu, i1 < N && k1 == best);
        const unsigned b2 = __ballot_sync(0xffffffffu, i2 < N && k2 == best);
        const int bi = b1 ? j + __ffs(b1) - 1 : j + 32 + __ffs(b2) - 1;
        __syncwarp();
        const float pv = fA[bi * lda + j];
        __syncwarp();
        if (tx < nb && bi != j) {
          const int c = k0 + tx;
          const float a = fA[j * lda + c];
          fA[j * lda + c] = fA[bi * lda + c];
          fA[bi * lda + c] = a;
        }
        const float pi = best == 0u ? 0.0f : 1.0f / pv;
        __syncwarp();
        if (tx == 0) {
          piv[j] = bi;
          pinv[j] = pi;
          if (best == 0u) atomicOr(s_bad, 1);
        }
        for (int i = j + 1 + tx; i < N; i += 32) {
          const float l = fA[i * lda + j] * pi;
          fA[i * lda + j] = l;
          for (int c = j + 1; c < kend; ++c) fA[i * lda + c] -= l * fA[j * lda + c];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // the panel's exchanges on the other columns (left of the panel too: L keeps
    // the final row order), then U12 = L11^{-1} A12, one thread per column
    for (int c = tid; c < N; c += NT) {
      if (c >= k0 && c < kend) continue;
      for (int t = 0; t < nb; ++t) {
        const int p = piv[k0 + t], r = k0 + t;
        if (p != r) {
          const float a = fA[r * lda + c];
          fA[r * lda + c] = fA[p * lda + c];
          fA[p * lda + c] = a;
        }
      }
      if (c >= kend)
        for (int t = 1; t < nb; ++t) {
          float v = fA[(k0 + t) * lda + c];
          for (int s2 = 0; s2 < t; ++s2) v -= fA[(k0 + t) * lda + k0 + s2] * fA[(k0 + s2) * lda + c];
          fA[(k0 + t) * lda + c] = v;
        }
    }
    __syncthreads();
    if (kend < N) {
      tc_update<MODE>(fA + kend * lda + kend, lda, N - kend, N - kend, fA + kend * lda + k0, lda,
                      fA + k0 * lda + kend, lda, nb, ty, NW, tx);
      __syncthreads();
    }
  }
}

// W <- (P L U)^{-1} W for ncol right-hand sides (W: N x ncol binary32, stride ldw):
// the exchanges, forward substitution with L and back substitution with U in
// 8-row blocks, the blocks' updates of the other rows on the tensor cores.
template <int N, int NT, int MODE>
__device__ void tc_lu_apply(const float* fA, int lda, const int* piv, const float* pinv, float* W, int ldw, int ncol,
                            int tid) {
  constexpr int NW = NT / 32;
  const int tx = tid & 31, ty = tid >> 5;
  for (int c = tid; c < ncol; c += NT)
    for (int k = 0; k < N; ++k) {
      const int p = piv[k];
      if (p != k) {
        const float a = W[k * ldw + c];
        W[k * ldw + c] = W[p * ldw + c];
        W[p * ldw + c] = a;
      }
    }
  __syncthreads();
  for (int k0 = 0; k0 < N; k0 += kTcNB) {
    const int nb = (N - k0 < kTcNB) ? N - k0 : kTcNB, kend = k0 + nb;
    for (int c = tid; c < ncol; c += NT)
      for (int t = 1; t < nb; ++t) {
        float v = W[(k0 + t) * ldw + c];
        for (int s2 = 0; s2 < t; ++s2) v -= fA[(k0 + t) * lda + k0 + s2] * W[(k0 + s2) * ldw + c];
        W[(k0 + t) * ldw + c] = v;
      }
    __syncthreads();
    if (kend < N) {
      tc_update<MODE>(W + kend * ldw, ldw, N - kend, ncol, fA + kend * lda + k0, lda, W + k0 * ldw, ldw, nb, ty, NW,
                      tx);
      __syncthreads();
    }
  }
  const int nblk = (N + kTcNB - 1) / kTcNB;
  for (int b = nblk - 1; b >= 0; --b) {
    const int k0 = b * kTcNB, nb = (N - k0 < kTcNB) ? N - k0 : kTcNB;
    for (int c = tid; c < ncol; c += NT)
      for (int t = nb - 1; t >= 0; --t) {
        const int i = k0 + t;
        float v = W[i * ldw + c];
        for (int s2 = t + 1; s2 < nb; ++s2) v -= fA[i * lda + k0 + s2] * W[(k0 + s2) * ldw + c];
        W[i * ldw + c] = v * pinv[i];
      }
    __syncthreads();
    if (k0 > 0) {
      tc_update<MODE>(W, ldw, k0, ncol, fA + k0, lda, W + k0 * ldw, ldw, nb, ty, NW, tx);
      __syncthreads();
    }
  }
}

// The local solve X = A^{-1} R of the element kernel in mixed precision.
// sA (T, N x N, stride lda) and sR (T, R = [B | F], N x nr1, stride ldr) hold the
// assembled blocks; on return sR holds X (and sA is unchanged).  sR0 (T, N x
// ldr) keeps R; fA (N x lda) and fW (N x ldr) are binary32 work space; piv,
// pinv (N), s_red (2 unsigned) shared.  Returns the number of corrections.
template <class T, int N, int NT, int MODE>
__device__ int tc_refine_solve(const T* sA, int lda, T* sR, int ldr, int nr1, T* sR0, float* fA, float* fW, int* piv,
                               float* pinv, unsigned* s_red, int refine_max, double tol, int* s_bad, int tid) {
  using A = Ar<T>;
  for (int e = tid; e < N * N; e += NT) {
    const int i = e / N, j = e - i * N;
    fA[i * lda + j] = (float)A::to_d(sA[i * lda + j]);
  }
  for (int e = tid; e < N * nr1; e += NT) {
    const int i = e / nr1, c = e - i * nr1;
    const T r = sR[i * ldr + c];
    sR0[i * ldr + c] = r;
    fW[i * ldr + c] = (float)A::to_d(r);
    sR[i * ldr + c] = A::zero();
  }
  __syncthreads();
  tc_lu_factor<N, NT, MODE>(fA, lda, piv, pinv, s_bad, tid);
  int sweeps = 0;
  for (int s = 0;; ++s) {
    tc_lu_apply<N, NT, MODE>(fA, lda, piv, pinv, fW, ldr, nr1, tid);
    if (tid == 0) { s_red[0] = 0u; s_red[1] = 0u; }
    __syncthreads();
    unsigned dmax = 0u, xmax = 0u;
    for (int e = tid; e < N * nr1; e += NT) {
      const int i = e / nr1, c = e - i * nr1;
      const float w = fW[i * ldr + c];
      const T x = A::norm(A::add(sR[i * ldr + c], A::from_d((double)w)));
      sR[i * ldr + c] = x;
      dmax = max(dmax, __float_as_uint(fabsf(w)));
      xmax = max(xmax, __float_as_uint(fabsf((float)A::to_d(x))));
    }
    atomicMax(&s_red[0], dmax);
    atomicMax(&s_red[1], xmax);
    __syncthreads();
    const float dm = __uint_as_float(s_red[0]), xm = __uint_as_float(s_red[1]);
    if (s >= 1 && (double)dm <= tol * (double)xm) break;  // converged
    if (s >= refine_max) {
      if (tid == 0 && refine_max > 0) atomicOr(s_bad, 4);
      break;
    }
    ++sweeps;
    // residual R - A X in T, rounded to binary32 for the next correction
    for (int e = tid; e < N * nr1; e += NT) {
      const int i = e / nr1, c = e - i * nr1;
      T acc = sR0[i * ldr + c];
      for (int j = 0; j < N; ++j) A::msub(acc, sA[i * lda + j], sR[j * ldr + c]);
      fW[i * ldr + c] = (float)A::to_d(A::norm(acc));
    }
    __syncthreads();
  }
  __syncthreads();
  return sweeps;
}

}  // namespace hdg
