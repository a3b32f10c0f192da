// Dense LU with partial pivoting of one element's local block, applied to its
// right-hand sides at the same time (Gaussian elimination on [A | R]), then
// back substitution: on return the rows of R hold X = A^{-1} R.  Shared
// memory, one CTA, arithmetic T (binary64 or float-float).
//
// Blocked right-looking form with panels of kLuNB columns (few block-wide
// barriers; the per-column work stays inside one warp):
//   1. one warp (rotating from panel to panel) factors the panel: per column, pivot search (largest |a|, first
//      on ties; compared as integer keys), row exchange inside the panel,
//      multipliers l = a / pivot and the rank-1 update of the panel's later
//      columns (warp-synchronous);
//   2. every column right of the panel (A and all of R), one thread each:
//      the panel's row exchanges in order, then U12 = L11^{-1} A12;
//   3. trailing update A22 -= L21 U12 (rank-kLuNB), the (row, column) pairs
//      flattened over the whole CTA, two per thread (independent accumulation
//      chains, full warps whatever the column count);
//   back substitution U X = Y in blocks of kLuNB rows from the bottom: the
//   diagonal block one thread per right-hand side, then the rank-kLuNB update
//   of the rows above.
// L is unit lower, U keeps the pivots (their inverses in s_pinv).  In
// float-float every value is renormalised before it is used as a factor.
#pragma once

#include <type_traits>

#include "hdg_arith.cuh"

namespace hdg {

constexpr int kLuNB = 8;

// s_pv: scratch for kLuNB pivot indices (shared memory not otherwise live during the LU)
template <class T, int NROWS, int NT>
__device__ __forceinline__ void lu_solve(T* sA, int lda, T* sR, int ldr, int nr1, int* s_pv, T* s_pinv, int* s_bad,
                                         int tid) {
  static_assert(NROWS <= 64, "the pivot search holds at most two rows per lane");
  using A = Ar<T>;
  constexpr int NW = NT / 32;
  const int tx = tid & 31, ty = tid >> 5;
  for (int k0 = 0; k0 < NROWS; k0 += kLuNB) {
    const int nb = (NROWS - k0 < kLuNB) ? NROWS - k0 : kLuNB;
    const int kend = k0 + nb;
    // the serial parts rotate over the warps (and so over the SM's schedulers) from panel to panel
    const int pw = (k0 / kLuNB) % NW;
    const int rt = (tid + NT - 32 * pw) % NT;
    // ---- 1. panel factorisation (warp pw) ----
    if (ty == pw) {
      for (int j = k0; j < kend; ++j) {
        // pivot search over rows j.. (at most two per lane): the largest |a| as an integer
        // key, by two warp max-reductions (high, then low 32 bits), the first row on ties
        // by ballots over the lanes' first, then second, rows
        const int i1 = j + tx, i2 = j + tx + 32;
        unsigned long long k1 = 0ull, k2 = 0ull;
        if (i1 < NROWS) {
          const T v = A::norm(sA[i1 * lda + j]);
          sA[i1 * lda + j] = v;
          k1 = A::key(v);
        }
        if (i2 < NROWS) {
          const T v = A::norm(sA[i2 * lda + j]);
          sA[i2 * lda + j] = v;
          k2 = A::key(v);
        }
        const unsigned long long km = k1 > k2 ? k1 : k2;
        const unsigned mhi = __reduce_max_sync(0xffffffffu, (unsigned)(km >> 32));
        const unsigned mlo = __reduce_max_sync(0xffffffffu, (unsigned)(km >> 32) == mhi ? (unsigned)km : 0u);
        const unsigned long long best = ((unsigned long long)mhi << 32) | mlo;
        const unsigned b1 = __ballot_sync(0xffffffffu, i1 < NROWS && k1 == best);
        const unsigned b2 = __ballot_sync(0xffffffffu, i2 < NROWS && k2 == best);
        const int bi = b1 ? j + __ffs(b1) - 1 : j + 32 + __ffs(b2) - 1;
        __syncwarp();
        const T piv = sA[bi * lda + j];
        __syncwarp();
        // exchange rows j and bi inside the panel; U row j of the panel renormalised
        if (tx < nb) {
          const int c = k0 + tx;
          const T vj = sA[j * lda + c], vp = sA[bi * lda + c];
          if (bi != j) sA[bi * lda + c] = vj;
          sA[j * lda + c] = (c > j) ? A::norm(vp) : vp;
        }
        const T pinv = (best == 0ull) ? A::zero() : A::rcp(piv);
        __syncwarp();
        if (tx == 0) {
          s_pv[j - k0] = bi;
          s_pinv[j] = pinv;
          if (best == 0ull) *s_bad |= 1;
        }
        // multipliers and the rank-1 update of the panel's later columns
        for (int i = j + 1 + tx; i < NROWS; i += 32) {
          const T l = A::mul(sA[i * lda + j], pinv);
          sA[i * lda + j] = l;
          for (int c = j + 1; c < kend; ++c) A::msub(sA[i * lda + c], l, sA[j * lda + c]);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // ---- 2. row exchanges and U12 = L11^{-1} A12, one thread per column right of the panel ----
    const int wa = NROWS - kend, total = wa + nr1;
    for (int cc = rt; cc < total; cc += NT) {
      T* col = (cc < wa) ? sA + kend + cc : sR + (cc - wa);
      const int ld = (cc < wa) ? lda : ldr;
#pragma unroll
      for (int t = 0; t < kLuNB; ++t) {
        if (t < nb) {
          const int p = s_pv[t], r = k0 + t;
          if (p != r) {
            const T a = col[r * ld], b = col[p * ld];
            col[r * ld] = b;
            col[p * ld] = a;
          }
        }
      }
      T u[kLuNB];
#pragma unroll
      for (int t = 0; t < kLuNB; ++t) {
        if (t < nb) {
          T v = col[(k0 + t) * ld];
#pragma unroll
          for (int s2 = 0; s2 < t; ++s2) A::msub(v, sA[(k0 + t) * lda + k0 + s2], u[s2]);
          u[t] = A::norm(v);
          col[(k0 + t) * ld] = u[t];
        }
      }
    }
    __syncthreads();
    // ---- 3. trailing update A22 -= L21 U12: the (row, column) pairs flattened over the CTA,
    //      two per thread (independent chains, full warps) ----
    {
      const int cnt = (NROWS - kend) * total;
      const int dq = (2 * NT) / (total > 0 ? total : 1), dr = (2 * NT) - dq * (total > 0 ? total : 1);
      int r = tid / (total > 0 ? total : 1), c = tid - r * total;        // element tid
      int r2 = (tid + NT) / (total > 0 ? total : 1), c2 = (tid + NT) - r2 * total;  // element tid + NT
      for (int e = tid; e < cnt; e += 2 * NT) {
        const bool has2 = e + NT < cnt;
        const int i0 = kend + r, i1 = kend + (has2 ? r2 : r);
        const int cb = has2 ? c2 : c;
        T* pa = (c < wa) ? sA + i0 * lda + kend + c : sR + i0 * ldr + (c - wa);
        T* pb = (cb < wa) ? sA + i1 * lda + kend + cb : sR + i1 * ldr + (cb - wa);
        const T* ua = (c < wa) ? sA + k0 * lda + kend + c : sR + k0 * ldr + (c - wa);
        const T* ub = (cb < wa) ? sA + k0 * lda + kend + cb : sR + k0 * ldr + (cb - wa);
        const int la = (c < wa) ? lda : ldr, lb = (cb < wa) ? lda : ldr;
        T a = *pa, b = *pb;
#pragma unroll
        for (int t = 0; t < kLuNB; ++t) {
          if (t < nb) {
            A::msub(a, sA[i0 * lda + k0 + t], ua[t * la]);
            A::msub(b, sA[i1 * lda + k0 + t], ub[t * lb]);
          }
        }
        *pa = a;
        if (has2) *pb = b;
        r += dq; c += dr;
        if (c >= total) { c -= total; ++r; }
        r2 += dq; c2 += dr;
        if (c2 >= total) { c2 -= total; ++r2; }
      }
    }
    __syncthreads();
  }
  // ---- back substitution U X = Y, blocks of kLuNB rows from the bottom ----
  const int nblk = (NROWS + kLuNB - 1) / kLuNB;
  for (int b = nblk - 1; b >= 0; --b) {
    const int kb = b * kLuNB;
    const int nb = (NROWS - kb < kLuNB) ? NROWS - kb : kLuNB;
    for (int c = (tid + NT - 32 * (b % NW)) % NT; c < nr1; c += NT) {
      T x[kLuNB];
#pragma unroll
      for (int t = kLuNB - 1; t >= 0; --t) {
        if (t < nb) {
          const int i = kb + t;
          T v = sR[i * ldr + c];
#pragma unroll
          for (int s2 = t + 1; s2 < kLuNB; ++s2)
            if (s2 < nb) A::msub(v, sA[i * lda + kb + s2], x[s2]);
          x[t] = A::mul(A::norm(v), s_pinv[i]);
          sR[i * ldr + c] = x[t];
        }
      }
    }
    __syncthreads();
    if (kb == 0) break;
    // rows above the block: Y -= U(:, block) X(block), (row, column) pairs flattened, two per thread
    {
      const int cnt = kb * nr1;
      const int dq = (2 * NT) / nr1, dr = (2 * NT) - dq * nr1;
      int r = tid / nr1, c = tid - r * nr1;
      int r2 = (tid + NT) / nr1, c2 = (tid + NT) - r2 * nr1;
      for (int e = tid; e < cnt; e += 2 * NT) {
        const bool has2 = e + NT < cnt;
        const int rb = has2 ? r2 : r, cb = has2 ? c2 : c;
        T a = sR[r * ldr + c], b = sR[rb * ldr + cb];
#pragma unroll
        for (int t = 0; t < kLuNB; ++t) {
          if (t < nb) {
            A::msub(a, sA[r * lda + kb + t], sR[(kb + t) * ldr + c]);
            A::msub(b, sA[rb * lda + kb + t], sR[(kb + t) * ldr + cb]);
          }
        }
        sR[r * ldr + c] = a;
        if (has2) sR[rb * ldr + cb] = b;
        r += dq; c += dr;
        if (c >= nr1) { c -= nr1; ++r; }
        r2 += dq; c2 += dr;
        if (c2 >= nr1) { c2 -= nr1; ++r2; }
      }
    }
    __syncthreads();
  }
}

}  // namespace hdg
