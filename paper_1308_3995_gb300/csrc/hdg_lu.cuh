// Dense LU with partial pivoting of one element's local block, applied to its
// right-hand sides at the same time (Gaussian elimination on [A | R]), then
// back substitution: on return the rows of R hold X = A^{-1} R.  Shared
// memory, one CTA, arithmetic T (binary64 or float-float).
//
// Per elimination step k (three barriers):
//   warp 0: renormalise column k (float-float) and find the pivot (largest
//     |a|, first on ties; compared as integer keys off the FP pipes);
//   all threads: exchange rows k and pivot over columns k.. of A and all of R,
//     and scale the new row k by the inverse pivot (unit upper triangle);
//   all threads: a_ij -= a_ik a_kj on the trailing block and on R, rows over
//     warps and columns over lanes.
// (Keeping the exchanges in a permutation and letting warp 0 scale the pivot
// row and form multipliers saves one barrier per step but lengthens each
// step's serial chain; measured slower on GB300.)
#pragma once

#include <type_traits>

#include "hdg_arith.cuh"

namespace hdg {

template <class T, int NROWS, int NT>
__device__ __forceinline__ void lu_solve(T* sA, int lda, T* sR, int ldr, int nr1, int* s_piv, T* s_pinv,
                                         int* s_bad, int tid) {
  using A = Ar<T>;
  constexpr int NW = NT / 32;
  const int tx = tid & 31, ty = tid >> 5;
  for (int k = 0; k < NROWS; ++k) {
    if (tid < 32) {
      unsigned long long best = 0ull;
      int bi = k;
      for (int i = k + tx; i < NROWS; i += 32) {
        const T v = A::norm(sA[i * lda + k]);
        sA[i * lda + k] = v;
        const unsigned long long kv = A::key(v);
        if (kv > best) { best = kv; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tx == 0) {
        *s_piv = bi;
        if (best == 0ull) { *s_bad |= 1; s_pinv[k] = A::zero(); } else { s_pinv[k] = A::rcp(sA[bi * lda + k]); }
      }
    }
    __syncthreads();
    {
      const int piv = *s_piv;
      const T pinv = s_pinv[k];
      const int wa = NROWS - k;
      for (int t = tid; t < wa + nr1; t += NT) {
        T* pk = (t < wa) ? &sA[k * lda + k + t] : &sR[k * ldr + (t - wa)];
        T* pp = (t < wa) ? &sA[piv * lda + k + t] : &sR[piv * ldr + (t - wa)];
        const T vk = *pk, vp = *pp;
        if (piv != k) *pp = vk;
        *pk = A::mul(A::norm(vp), pinv);
      }
    }
    __syncthreads();
    {
      const int wa = NROWS - k - 1, nc = wa + nr1;
      if constexpr (std::is_same<T, double>::value) {
        for (int i = k + 1 + ty; i < NROWS; i += NW) {
          const T l = sA[i * lda + k];
          for (int c = tx; c < nc; c += 32) {
            const bool inA = c < wa;
            T* dst = inA ? &sA[i * lda + k + 1 + c] : &sR[i * ldr + (c - wa)];
            const T* src = inA ? &sA[k * lda + k + 1 + c] : &sR[k * ldr + (c - wa)];
            A::msub(*dst, l, *src);
          }
        }
      } else {  // float-float: four independent update chains per thread
        for (int i = k + 1 + ty; i < NROWS; i += NW) {
          const T l = sA[i * lda + k];
          for (int c0 = 0; c0 < nc; c0 += 128) {
            T dv[4], sv[4];
            T* dp[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int c = c0 + tx + 32 * u;
              const bool inA = c < wa;
              dp[u] = inA ? &sA[i * lda + k + 1 + c] : &sR[i * ldr + (c - wa)];
              if (c < nc) {
                dv[u] = *dp[u];
                sv[u] = inA ? sA[k * lda + k + 1 + c] : sR[k * ldr + (c - wa)];
              }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (c0 + tx + 32 * u < nc) A::msub(dv[u], l, sv[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (c0 + tx + 32 * u < nc) *dp[u] = dv[u];
          }
        }
      }
    }
    __syncthreads();
  }
  // back substitution with the unit upper triangle (row k renormalised before use)
  for (int k = NROWS - 1; k > 0; --k) {
    if constexpr (!std::is_same<T, double>::value) {
      for (int t = tid; t < nr1; t += NT) sR[k * ldr + t] = A::norm(sR[k * ldr + t]);
      __syncthreads();
    }
    for (int i = ty; i < k; i += NW) {  // two independent update chains per thread
      const T u = sA[i * lda + k];
      for (int c0 = 0; c0 < nr1; c0 += 64) {
        const int ca = c0 + tx, cb = c0 + tx + 32;
        T da, db, sa, sb;
        if (ca < nr1) { da = sR[i * ldr + ca]; sa = sR[k * ldr + ca]; }
        if (cb < nr1) { db = sR[i * ldr + cb]; sb = sR[k * ldr + cb]; }
        if (ca < nr1) A::msub(da, u, sa);
        if (cb < nr1) A::msub(db, u, sb);
        if (ca < nr1) sR[i * ldr + ca] = da;
        if (cb < nr1) sR[i * ldr + cb] = db;
      }
    }
    __syncthreads();
  }
}

}  // namespace hdg
