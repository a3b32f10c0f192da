// Dense LU with partial pivoting of one element's local block, applied to its
// right-hand sides at the same time (Gaussian elimination on [A | R]), then
// back substitution: on return the rows of R hold X = A^{-1} R.  Shared
// memory, one CTA, arithmetic T (binary64 or float-float).
//
// Blocked right-looking form with panels of kLuNB columns and look-ahead:
//   1. one warp factors a panel: per column, pivot search (largest |a|, first
//      on ties; compared as integer keys), row exchange inside the panel,
//      multipliers l = a / pivot and the rank-1 update of the panel's later
//      columns (warp-synchronous);
//   2. every column right of the panel (A and all of R), one thread each:
//      the panel's row exchanges in order, then U12 = L11^{-1} A12;
//   3. trailing update A22 -= L21 U12 (rank-kLuNB): the next panel's columns
//      by the warp that factors it right after (look-ahead), the rest by the
//      other warps, (row, column) pairs flattened, two per thread;
//   back substitution U X = Y in blocks of kLuNB rows from the bottom: the
//   diagonal block one thread per right-hand side, then the rank-kLuNB update
//   of the rows above.
// L is unit lower (its rows are not exchanged by later panels: only U and the
// transformed R are used afterwards), U keeps the pivots (their inverses in
// s_pinv).  In float-float every value is renormalised before it is used as a
// factor.
#pragma once

#include <type_traits>

#include "hdg_arith.cuh"

namespace hdg {

constexpr int kLuNB = 8;

// Back substitution U X = Y in blocks of kLuNB rows from the bottom: the
// diagonal block one thread per right-hand side, then the rank-kLuNB update of
// the rows above, (row, column) pairs flattened, two per thread.
template <class T, int NROWS, int NT>
__device__ __forceinline__ void lu_back_substitute(T* sA, int lda, T* sR, int ldr, int nr1, const T* s_pinv, int tid) {
  using A = Ar<T>;
  constexpr int NW = NT / 32;
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

// One warp factors the panel of columns k0 .. k0 + nb - 1 (rows k0.. of
// those columns up to date): per column, the pivot search (largest |a|, first
// on ties, compared as integer keys), the row exchange inside the panel, the
// multipliers and the rank-1 update of the panel's later columns.  Pivot rows
// go to s_pv[0..nb), pivot inverses to s_pinv[k0..].
template <class T, int NROWS>
__device__ __forceinline__ void lu_factor_panel(T* sA, int lda, int k0, int nb, int* s_pv, T* s_pinv, int* s_bad,
                                                int tx) {
  using A = Ar<T>;
  const int kend = k0 + nb;
  for (int j = k0; j < kend; ++j) {
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
    for (int i = j + 1 + tx; i < NROWS; i += 32) {
      const T l = A::mul(sA[i * lda + j], pinv);
      sA[i * lda + j] = l;
      for (int c = j + 1; c < kend; ++c) A::msub(sA[i * lda + c], l, sA[j * lda + c]);
    }
    __syncwarp();
  }
}

// The blocked LU with look-ahead: after panel k's row exchanges and U12, the
// warp that will factor panel k + 1 applies panel k's trailing update to that
// panel's own columns and factors it at once, while the other warps apply the
// trailing update to every column right of it (A and all of R) -- the serial
// panel factorisation overlaps the parallel update, and each panel costs two
// block barriers.  s_pv: 2 kLuNB ints of scratch (the pivots of the panel
// being applied and of the one being factored).
template <class T, int NROWS, int NT>
__device__ __forceinline__ void lu_solve(T* sA, int lda, T* sR, int ldr, int nr1, int* s_pv, T* s_pinv, int* s_bad,
                                         int tid) {
  static_assert(NROWS <= 64, "the pivot search holds at most two rows per lane");
  static_assert(NT >= 64, "look-ahead needs a panel warp and at least one update warp");
  using A = Ar<T>;
  constexpr int NW = NT / 32, NP = (NROWS + kLuNB - 1) / kLuNB;
  const int tx = tid & 31, ty = tid >> 5;
  if (ty == 0) lu_factor_panel<T, NROWS>(sA, lda, 0, NROWS < kLuNB ? NROWS : kLuNB, s_pv, s_pinv, s_bad, tx);
  __syncthreads();
  for (int k = 0; k < NP; ++k) {
    const int k0 = k * kLuNB;
    const int nb = (NROWS - k0 < kLuNB) ? NROWS - k0 : kLuNB;
    const int kend = k0 + nb;
    const int* pv = s_pv + (k & 1) * kLuNB;
    // ---- row exchanges of panel k and U12 = L11^{-1} A12, one thread per column right of the panel ----
    const int wa = NROWS - kend, total = wa + nr1;
    for (int cc = tid; cc < total; cc += NT) {
      T* col = (cc < wa) ? sA + kend + cc : sR + (cc - wa);
      const int ld = (cc < wa) ? lda : ldr;
#pragma unroll
      for (int t = 0; t < kLuNB; ++t) {
        if (t < nb) {
          const int p = pv[t], r = k0 + t;
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
    if (kend >= NROWS) break;  // no trailing rows: the elimination is complete
    // ---- panel k + 1: its warp updates its columns and factors it; the others update the rest ----
    const int k1 = kend, nb1 = (NROWS - k1 < kLuNB) ? NROWS - k1 : kLuNB, kend1 = k1 + nb1;
    const int pw = (k + 1) % NW;
    if (ty == pw) {
      for (int e = tx; e < (NROWS - kend) * nb1; e += 32) {
        const int i = kend + e / nb1, c = k1 + e % nb1;
        T a = sA[i * lda + c];
#pragma unroll
        for (int t = 0; t < kLuNB; ++t)
          if (t < nb) A::msub(a, sA[i * lda + k0 + t], sA[(k0 + t) * lda + c]);
        sA[i * lda + c] = a;
      }
      __syncwarp();
      lu_factor_panel<T, NROWS>(sA, lda, k1, nb1, s_pv + ((k + 1) & 1) * kLuNB, s_pinv, s_bad, tx);
    } else {
      // columns right of panel k + 1 (A) and all of R; the (row, column) pairs flattened over the
      // update warps' threads, two per thread (independent accumulation chains)
      constexpr int NU = NT - 32;
      const int rid = (ty < pw) ? tid : tid - 32;
      const int wa1 = NROWS - kend1, tot1 = wa1 + nr1;
      const int cnt = (NROWS - kend) * tot1;
      for (int e = rid; e < cnt; e += 2 * NU) {
        const int e2 = e + NU;
        const bool has2 = e2 < cnt;
        const int r0 = e / tot1, c0 = e - r0 * tot1;
        const int r1 = has2 ? e2 / tot1 : r0, c1 = has2 ? e2 - r1 * tot1 : c0;
        const int i0 = kend + r0, i1 = kend + r1;
        T* pa = (c0 < wa1) ? sA + i0 * lda + kend1 + c0 : sR + i0 * ldr + (c0 - wa1);
        T* pb = (c1 < wa1) ? sA + i1 * lda + kend1 + c1 : sR + i1 * ldr + (c1 - wa1);
        const T* ua = (c0 < wa1) ? sA + k0 * lda + kend1 + c0 : sR + k0 * ldr + (c0 - wa1);
        const T* ub = (c1 < wa1) ? sA + k0 * lda + kend1 + c1 : sR + k0 * ldr + (c1 - wa1);
        const int la = (c0 < wa1) ? lda : ldr, lb = (c1 < wa1) ? lda : ldr;
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
      }
    }
    __syncthreads();
  }
  lu_back_substitute<T, NROWS, NT>(sA, lda, sR, ldr, nr1, s_pinv, tid);
}

}  // namespace hdg
