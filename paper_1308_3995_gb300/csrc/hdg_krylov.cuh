// Krylov-vector kernels of the GMRES trace solve (Sec. 3.4): dot products
// with the basis, the Arnoldi process as delayed classical Gram-Schmidt with
// re-orthogonalisation (one reduction and one update pass per iteration, the
// Hessenberg bookkeeping on the device), and the solution update.  Every
// kernel is written once over the storage type ST of the vectors:
//   double  binary64 values, binary64 arithmetic (the FP64 pipe);
//   float2  float-float pairs (hi, lo) in the same 8 bytes per value,
//           double-word arithmetic Ar<ff> on the binary32 pipe.
// Trace-space vectors have a length that is a multiple of 4 (4 (p_e + 1)
// values per face) and start 16-byte aligned, so two consecutive values move
// as one 16-byte load (double2 / float4).
//
// Dot products: every thread takes its own pair rows (a grid-stride loop) for
// a group of up to eight vectors, all their loads in flight together; the
// block sums each vector's values through shared memory into one partial per
// block in part[row][block]; the partials are then summed in two levels by
// the last blocks to finish (tickets taken after fences) in a fixed order --
// the results are bitwise reproducible.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "hdg_arith.cuh"

namespace hdg {
namespace krylov {

constexpr int kMaxRestart = 64;
constexpr int kDotThreads = 256;
constexpr int kDotWarps = kDotThreads / 32;

template <class ST>
struct KV;

template <>
struct KV<double> {
  using A = double;
  using P = double2;
  static __device__ __forceinline__ A x(const P& p) { return p.x; }
  static __device__ __forceinline__ A y(const P& p) { return p.y; }
  static __device__ __forceinline__ P pack(A a, A b) { return make_double2(a, b); }
  static __device__ __forceinline__ P zero2() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ A from_d(double d) { return d; }
  static __device__ __forceinline__ double to_d(A a) { return a; }
};

template <>
struct KV<float2> {
  using A = ff;
  using P = float4;
  static __device__ __forceinline__ A x(const P& p) { return ff{p.x, p.y}; }
  static __device__ __forceinline__ A y(const P& p) { return ff{p.z, p.w}; }
  static __device__ __forceinline__ P pack(A a, A b) { return make_float4(a.hi, a.lo, b.hi, b.lo); }
  static __device__ __forceinline__ P zero2() { return make_float4(0.0f, 0.0f, 0.0f, 0.0f); }
  static __device__ __forceinline__ A from_d(double d) { return ff_split_double(d); }
  static __device__ __forceinline__ double to_d(A a) { return ff_to_double(a); }
};

template <class ST>
__device__ __forceinline__ const typename KV<ST>::P* pairs(const ST* v) {
  return reinterpret_cast<const typename KV<ST>::P*>(v);
}
template <class ST>
__device__ __forceinline__ typename KV<ST>::P* pairs(ST* v) {
  return reinterpret_cast<typename KV<ST>::P*>(v);
}

// one value of a vector as its arithmetic type, and back
__device__ __forceinline__ double ld1(const double* p) { return *p; }
__device__ __forceinline__ ff ld1(const float2* p) {
  const float2 v = *p;
  return ff{v.x, v.y};
}
__device__ __forceinline__ void st1(double* p, double a) { *p = a; }
__device__ __forceinline__ void st1(float2* p, ff a) { *p = make_float2(a.hi, a.lo); }

__device__ __forceinline__ double KV_shfl_down(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ ff KV_shfl_down(ff v, int o) {
  return ff{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(ff v) { return ff_to_double(v); }

// Sum of part[j][0..nblk) for j < nrows: tpr threads per row (a power of two
// <= 32, as many as the block holds for all rows at once), each taking every
// tpr-th partial in block order in eight independent chains (their loads in
// flight together), then a shuffle tree over the tpr lanes -- a fixed order.
// Row nrows - 1 goes to *last_out when last_out is given, the others to
// out[j].  Called by the last block only; it re-arms the ticket.
__device__ __forceinline__ void finish_rows(const double* part, int nrows, int nblk, double* out, double* last_out,
                                            unsigned* ticket) {
  int tpr = 32;
  while (tpr > 1 && tpr * nrows > (int)blockDim.x) tpr >>= 1;
  const int sub = threadIdx.x & (tpr - 1);
  for (int r0 = 0; r0 < nrows; r0 += blockDim.x / tpr) {
    const int j = r0 + threadIdx.x / tpr;
    double c[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (j < nrows) {
      const double* pj = part + (int64_t)j * nblk;
      int b = sub;
      for (; b + 7 * tpr < nblk; b += 8 * tpr) {
#pragma unroll
        for (int q = 0; q < 8; ++q) c[q] += __ldcg(pj + b + q * tpr);
      }
      for (; b < nblk; b += tpr) c[0] += __ldcg(pj + b);
    }
    double v = ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
    for (int o = tpr >> 1; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (sub == 0 && j < nrows) {
      if (last_out && j == nrows - 1) *last_out = v;
      else out[j] = v;
    }
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

// Two-level finish.  After every block has written its partials
// part[j][blockIdx.x], j < nrows: the last block of each group of kFinGroup
// consecutive blocks (a ticket per group, taken after a fence) sums its
// group's partials into gpart[j][group] (group_finish); for a complete sum
// the last group to finish (ticket[0]) then sums those into out
// (finish_rows).  Each level is one round of loads and at most kFinGroup (or
// the number of groups) blocks contend for one ticket.  ticket: 1 + groups
// counters, zero between launches (re-armed here).
constexpr int kFinGroup = 16;
__host__ __device__ __forceinline__ int fin_groups(int nblk) { return (nblk + kFinGroup - 1) / kFinGroup; }

// The first level: true in the block that wrote its group's sums.
__device__ __forceinline__ bool group_finish(const double* part, int nrows, double* gpart, unsigned* ticket) {
  __shared__ bool s_glast;
  const int nblk = gridDim.x, grp = blockIdx.x / kFinGroup, ng = fin_groups(nblk);
  const int b0 = grp * kFinGroup, gsize = min(kFinGroup, nblk - b0);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_glast = atomicAdd(ticket + 1 + grp, 1u) == (unsigned)gsize - 1u;
  __syncthreads();
  if (!s_glast) return false;
  __threadfence();
  int tpr = 16;
  while (tpr > 1 && tpr * nrows > (int)blockDim.x) tpr >>= 1;
  const int sub = threadIdx.x & (tpr - 1);
  for (int r0 = 0; r0 < nrows; r0 += blockDim.x / tpr) {
    const int j = r0 + threadIdx.x / tpr;
    double v = 0.0;
    if (j < nrows)
      for (int b = sub; b < gsize; b += tpr) v += __ldcg(part + (int64_t)j * nblk + b0 + b);
    for (int o = tpr >> 1; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (sub == 0 && j < nrows) gpart[(int64_t)j * ng + grp] = v;
  }
  if (threadIdx.x == 0) ticket[1 + grp] = 0u;
  return true;
}

// Both levels: true in the one block that wrote the complete sums.
__device__ __forceinline__ bool last_block_finish(const double* part, int nrows, double* gpart, double* out,
                                                  double* last_out, unsigned* ticket) {
  __shared__ bool s_last;
  if (!group_finish(part, nrows, gpart, ticket)) return false;
  __threadfence();
  __syncthreads();
  const int ng = fin_groups(gridDim.x);
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == (unsigned)ng - 1u;
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  finish_rows(gpart, nrows, ng, out, last_out, ticket);
  return true;
}

constexpr int kGroup = 8;  // vectors per pass of the dot-product kernels (one per warp in the block reduction)

// part[row[k]][blockIdx.x] = the block's sum of acc[k] for the k set in
// valid: every thread stores its kGroup accumulators in shared memory; warp k
// then sums column k (each lane eight threads' values in thread order, then a
// shuffle tree) -- a fixed order.
template <class A>
__device__ __forceinline__ void block_rows_partial(const A (&acc)[kGroup], unsigned valid, const int (&row)[kGroup],
                                                   double* part) {
  using AR = Ar<A>;
  static_assert(kGroup == kDotWarps, "one warp per accumulator column");
  __shared__ A s_acc[kGroup][kDotThreads + 1];
#pragma unroll
  for (int k = 0; k < kGroup; ++k) s_acc[k][threadIdx.x] = acc[k];
  __syncthreads();
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  if ((valid >> wp) & 1u) {
    A v = AR::zero();
#pragma unroll
    for (int t = 0; t < kDotThreads / 32; ++t) v = AR::add(v, s_acc[wp][lane * (kDotThreads / 32) + t]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = AR::add(v, KV_shfl_down(v, o));
    int r = row[0];
#pragma unroll
    for (int k = 1; k < kGroup; ++k) r = (wp == k) ? row[k] : r;
    if (lane == 0) part[(int64_t)r * gridDim.x + blockIdx.x] = to_double(v);
  }
  __syncthreads();  // s_acc is reused by the next group
}

// acc[k] += V_{g+k}[i] . w[i] over this thread's pair rows i (i0, i0 + stride,
// ...), k < ng <= kGroup: two rows' loads of every vector in flight at a time.
// RO: w is not written by this launch (read through the read-only path).
template <class ST, bool RO>
__device__ __forceinline__ void rows_dots(const ST* __restrict__ V, int64_t ldv, int g, int ng, const ST* w,
                                          int64_t n2, typename KV<ST>::A (&acc)[kGroup]) {
  using K = KV<ST>;
  using AR = Ar<typename K::A>;
  using P = typename K::P;
  const P* w2 = pairs(w);
  const int64_t stride = (int64_t)gridDim.x * kDotThreads;
  for (int64_t i = (int64_t)blockIdx.x * kDotThreads + threadIdx.x; i < n2; i += 2 * stride) {
    const int64_t i2 = i + stride;
    const bool two = i2 < n2;
    const P wa = RO ? __ldg(w2 + i) : w2[i];
    const P wb = two ? (RO ? __ldg(w2 + i2) : w2[i2]) : K::zero2();
    P va[kGroup], vb[kGroup];
#pragma unroll
    for (int k = 0; k < kGroup; ++k) {
      if (k < ng) {
        const P* vk = pairs(V + (int64_t)(g + k) * ldv);
        va[k] = __ldg(vk + i);
        vb[k] = two ? __ldg(vk + i2) : K::zero2();
      }
    }
#pragma unroll
    for (int k = 0; k < kGroup; ++k) {
      if (k < ng) {
        AR::madd(acc[k], K::x(va[k]), K::x(wa));
        AR::madd(acc[k], K::y(va[k]), K::y(wa));
        AR::madd(acc[k], K::x(vb[k]), K::x(wb));
        AR::madd(acc[k], K::y(vb[k]), K::y(wb));
      }
    }
  }
}

// part[j][block] = this block's share of V_j . w, j < nvec, in groups of kGroup vectors
template <class ST, bool RO>
__device__ __forceinline__ void block_dots(const ST* __restrict__ V, int64_t ldv, int nvec, const ST* w, int64_t n2,
                                           double* part) {
  using A = typename KV<ST>::A;
  for (int g = 0; g < nvec; g += kGroup) {
    const int ng = min(kGroup, nvec - g);
    A acc[kGroup];
#pragma unroll
    for (int k = 0; k < kGroup; ++k) acc[k] = Ar<A>::zero();
    rows_dots<ST, RO>(V, ldv, g, ng, w, n2, acc);
    int row[kGroup];
#pragma unroll
    for (int q = 0; q < kGroup; ++q) row[q] = g + q;
    block_rows_partial(acc, (1u << ng) - 1u, row, part);
  }
}

// out[j] = V_j . w, j < nvec (vectors V_j at V + j ldv, length n)
template <class ST>
__global__ void __launch_bounds__(kDotThreads, 2) k_dots(const ST* __restrict__ V, int64_t ldv, int nvec,
                                                      const ST* __restrict__ w, int64_t n, double* __restrict__ part,
                                                      double* gpart, double* __restrict__ out, unsigned* ticket) {
  block_dots<ST, true>(V, ldv, nvec, w, n >> 1, part);
  last_block_finish(part, nvec, gpart, out, nullptr, ticket);
}

// ---------------------------------------------------------------- device-side Arnoldi bookkeeping
// The Arnoldi process runs as delayed classical Gram-Schmidt with one
// re-orthogonalisation (DCGS2; Swirydowicz et al. 2021, Bielich et al. 2022):
// step j receives u_j = A v_{j-1} - V_j h1 (v_{j-1}'s product once projected,
// not yet normalised), forms z = A u_j, and one reduction pass gives
//   s = V_j^T u_j, alpha = u_j^T u_j, c = V_j^T z, gamma = u_j^T z.
// s is the second projection of u_j (that of classical Gram-Schmidt twice),
// so column j-1 of the Hessenberg matrix is h1 + s with h_{j,j-1} = rho =
// ||u_j - V_j s|| = sqrt(alpha - s^T s), and v_j = (u_j - V_j s) / rho.  The
// product of v_j follows from z and the Arnoldi relation A V_j = V_{j+1} H:
//   A v_j = (z - V_{j+1} H s) / rho, so its first projection is
//   h1_j = [(c - H_top s) / rho; d / rho - s_{j-1}], d = v_j^T z = (gamma - s^T c) / rho,
// and the next candidate is u_{j+1} = (z - V_j c - v_j d) / rho.  One
// update pass writes v_j and u_{j+1}: two passes over the basis per
// iteration instead of four.  The norms come from the Pythagorean identity
// (V orthonormal).  Everything but the two passes runs on the device in one
// extra block of the update launch, alongside the update; the host reads the
// state back once per chunk of iterations.
// Views into the solver's h buffer:
//   red [2 (R+1)] the reduction's outputs (a_k = V_k . u, k <= j, then b_k = V_k . z),
//   h1 [R+1] the first projection of the column being built,
//   Hraw [(R+1) R] the Hessenberg matrix (column-major), H [(R+1) R] its
//   rotated (triangular) form, cs, sn [R], g [R+1], y [R], sc [kArnoldiScalars]:
//   sc[1] residual estimate, sc[2] ||M^-1 E||, sc[3] rtol, sc[4] 0 running /
//   1 converged or breakdown / 2 out of iterations, sc[5] columns of H built
//   in the cycle, sc[6] iterations so far, sc[7] max_iter (sc[0], sc[8], sc[9]
//   unused: every block of the update derives 1 / rho and d from the sums).
constexpr int kArnoldiScalars = 10;
struct ArnoldiViews {
  double *red, *h1, *Hraw, *H, *cs, *sn, *g, *y, *sc;
};
__host__ __device__ __forceinline__ ArnoldiViews arnoldi_views(double* h, int R) {
  ArnoldiViews a;
  const int nr = R + 1;
  a.red = h;
  a.h1 = h + 2 * nr;
  a.Hraw = a.h1 + nr;
  a.H = a.Hraw + nr * R;
  a.cs = a.H + nr * R;
  a.sn = a.cs + R;
  a.g = a.sn + R;
  a.y = a.g + nr;
  a.sc = a.y + R;
  return a;
}
inline size_t arnoldi_doubles(int R) { return (size_t)(3 * (R + 1) + 2 * (R + 1) * R + 2 * R + (R + 1) + R + kArnoldiScalars); }

__global__ void k_cycle_init(double* h, int R, double beta, double bnorm, double rtol, int it, int max_iter) {
  ArnoldiViews a = arnoldi_views(h, R);
  for (int i = 0; i <= R; ++i) a.g[i] = 0.0;
  a.g[0] = beta;
  a.sc[0] = 0.0;
  a.sc[1] = beta / bnorm;
  a.sc[2] = bnorm;
  a.sc[3] = rtol;
  a.sc[4] = 0.0;
  a.sc[5] = 0.0;
  a.sc[6] = it;
  a.sc[7] = max_iter;
  a.sc[8] = 0.0;
}

// The sums of step j's reduction in one block's shared memory (every block
// of the update computes the same values in the same order): s_k = V_k . u
// and c_k = V_k . z (k < j), alpha = u . u, gamma = u . z, rho =
// sqrt(alpha - s^T s) (0 when that is not positive), d = (gamma - s^T c) / rho.
struct DcgsSums {
  double s[kMaxRestart + 1], c[kMaxRestart + 1];
  double alpha, gamma, rho, d;
};

// Sum the group partials gpart[row][0..ng) (rows: a_0..a_j, then b_0..b_j
// with_z) into t, tpr threads per row in group order; then s^T s and s^T c by
// warp 0 (strided lane shares, a shuffle tree).
__device__ __forceinline__ void dcgs_sums(const double* __restrict__ gpart, int ng, int j, int with_z, DcgsSums& t) {
  const int nv = j + 1, nrows = with_z ? 2 * nv : nv;
  int tpr = 32;
  while (tpr > 1 && tpr * nrows > (int)blockDim.x) tpr >>= 1;
  const int sub = threadIdx.x & (tpr - 1);
  for (int r0 = 0; r0 < nrows; r0 += blockDim.x / tpr) {
    const int r = r0 + threadIdx.x / tpr;
    double v = 0.0;
    if (r < nrows)
      for (int b = sub; b < ng; b += tpr) v += __ldcg(gpart + (int64_t)r * ng + b);
    for (int o = tpr >> 1; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (sub == 0 && r < nrows) {
      if (r < j) t.s[r] = v;
      else if (r == j) t.alpha = v;
      else if (r < nv + j) t.c[r - nv] = v;
      else t.gamma = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double ss = 0.0, scv = 0.0;
    for (int q = threadIdx.x; q < j; q += 32) {
      ss = fma(t.s[q], t.s[q], ss);
      if (with_z) scv = fma(t.s[q], t.c[q], scv);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ss += __shfl_down_sync(0xffffffffu, ss, o);
      scv += __shfl_down_sync(0xffffffffu, scv, o);
    }
    if (threadIdx.x == 0) {
      const double rho2 = t.alpha - ss;
      t.rho = rho2 > 0.0 ? sqrt(rho2) : 0.0;
      t.d = (with_z && t.rho > 0.0) ? (t.gamma - scv) / t.rho : 0.0;
    }
  }
  __syncthreads();
}

// Step j's bookkeeping, run by one whole block from the sums t: finish
// column j - 1 (j >= 1) -- raw column h1 + s with h_{j,j-1} = rho, its
// Givens rotation, the residual estimate |g_j| / ||M^-1 E|| and the stopping
// test --, then (with_z: a product z was formed) start column j: h1_j.  The
// recurrence over the rotations runs in one thread, in registers, on operands
// the block loaded into shared memory.
__device__ __forceinline__ void dcgs_step(double* h, int R, int j, int with_z, const DcgsSums& t) {
  __shared__ double s_col[kMaxRestart + 1], s_cs[kMaxRestart], s_sn[kMaxRestart], s_stat;
  ArnoldiViews a = arnoldi_views(h, R);
  double* sc = a.sc;
  const double st = sc[4], its = sc[6], itmax = sc[7];
  if (st != 0.0) return;
  if (j >= 1 && its >= itmax) {  // iteration budget spent before this column
    if (threadIdx.x == 0) sc[4] = 2.0;
    return;
  }
  const int nr = R + 1;
  const double rho = t.rho;
  for (int k = threadIdx.x; k < j; k += blockDim.x) s_col[k] = a.h1[k] + t.s[k];
  for (int k = threadIdx.x; k + 1 < j; k += blockDim.x) {
    s_cs[k] = a.cs[k];
    s_sn[k] = a.sn[k];
  }
  if (j >= 1) {  // the raw column, written in parallel
    double* raw = a.Hraw + (size_t)(j - 1) * nr;
    for (int k = threadIdx.x; k <= j; k += blockDim.x) raw[k] = k < j ? a.h1[k] + t.s[k] : rho;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double stat = 0.0;
    if (j == 0) {
      a.g[0] = rho;
      if (!(rho > 0.0)) stat = 1.0;
    } else {
      double x = s_col[0];
      for (int k = 0; k + 1 < j; ++k) {  // earlier rotations, carried in registers
        const double z = s_col[k + 1];
        s_col[k] = s_cs[k] * x + s_sn[k] * z;
        x = -s_sn[k] * x + s_cs[k] * z;
      }
      const double den = hypot(x, rho);
      const double cr = den > 0.0 ? x / den : 1.0, sr = den > 0.0 ? rho / den : 0.0;
      a.cs[j - 1] = cr;
      a.sn[j - 1] = sr;
      s_col[j - 1] = den;
      s_col[j] = 0.0;
      const double gj = a.g[j - 1];
      a.g[j] = -sr * gj;
      a.g[j - 1] = cr * gj;
      sc[5] = j;
      sc[6] = its + 1.0;
      const double rel = fabs(a.g[j]) / sc[2];
      sc[1] = rel;
      if (!(rel > sc[3]) || !(rho > 0.0)) stat = 1.0;
    }
    if (stat != 0.0) sc[4] = stat;
    s_stat = stat;
  }
  __syncthreads();
  if (j >= 1) {
    double* col = a.H + (size_t)(j - 1) * nr;
    for (int k = threadIdx.x; k <= j; k += blockDim.x) col[k] = s_col[k];
  }
  if (s_stat != 0.0 || !with_z) return;
  // start column j: its first projection h1_j
  const double rinv = 1.0 / rho;
  for (int k = threadIdx.x; k < j; k += blockDim.x) {
    double hs = 0.0;  // (H_top s)_k: column i has rows <= i + 1
    for (int i = (k > 0 ? k - 1 : 0); i < j; ++i) hs = fma(a.Hraw[(size_t)i * nr + k], t.s[i], hs);
    a.h1[k] = (t.c[k] - hs) * rinv;
  }
  if (threadIdx.x == 0) a.h1[j] = t.d * rinv - (j >= 1 ? t.s[j - 1] : 0.0);
}

// H y = g (upper triangular, the cycle's columns): H and g loaded into shared
// memory by the block, the back substitution column by column (y_i, then
// every thread removes column i from the rows above it)
__global__ void k_lsq(double* h, int R) {
  __shared__ double s_h[(kMaxRestart + 1) * kMaxRestart], s_y[kMaxRestart + 1];
  ArnoldiViews a = arnoldi_views(h, R);
  const int jn = (int)a.sc[5];
  for (int t = threadIdx.x; t < jn * (R + 1); t += blockDim.x) s_h[t] = a.H[t];
  for (int t = threadIdx.x; t < jn; t += blockDim.x) s_y[t] = a.g[t];
  __syncthreads();
  for (int i = jn - 1; i >= 0; --i) {
    const double* col = s_h + (size_t)i * (R + 1);
    const double yi = s_y[i] / col[i];  // every thread, the same value
    __syncthreads();
    if (threadIdx.x == 0) s_y[i] = yi;
    for (int q = threadIdx.x; q < i; q += blockDim.x) s_y[q] -= col[q] * yi;
    __syncthreads();
  }
  for (int t = threadIdx.x; t < jn; t += blockDim.x) a.y[t] = s_y[t];
}

// DCGS2 reduction of step j: a_k = V_k . u and b_k = V_k . z for k <= j
// (u = V_j, the candidate; z = V_{j+1} = A u, with_z; without it only the
// a_k: the last step of a cycle, which finishes its last column), summed to
// one value per group of kFinGroup blocks (gpart; the update sums those).
// Every thread takes its own pair rows, four basis vectors and both
// right-hand vectors at a time (two rows' loads in flight).
template <class ST>
__global__ void __launch_bounds__(kDotThreads, 2) k_dcgs_reduce(const ST* __restrict__ V, int64_t ldv, int j,
                                                                int with_z, int64_t n, double* __restrict__ part,
                                                                double* gpart, unsigned* ticket) {
  using K = KV<ST>;
  using A = typename K::A;
  using AR = Ar<A>;
  using P = typename K::P;
  constexpr int NQ = kGroup / 2;  // basis vectors per pass: accumulators (a, b) per vector
  const int nv = j + 1;
  const int64_t n2 = n >> 1, stride = (int64_t)gridDim.x * kDotThreads;
  const P* u2 = pairs(V + (int64_t)j * ldv);
  const P* z2 = pairs(V + (int64_t)(j + 1) * ldv);
  for (int g = 0; g < nv; g += NQ) {
    const int ng = min(NQ, nv - g);
    A acc[kGroup];
#pragma unroll
    for (int q = 0; q < kGroup; ++q) acc[q] = AR::zero();
    for (int64_t i = (int64_t)blockIdx.x * kDotThreads + threadIdx.x; i < n2; i += 2 * stride) {
      const int64_t i2 = i + stride;
      const bool two = i2 < n2;
      const P ua = __ldg(u2 + i), ub = two ? __ldg(u2 + i2) : K::zero2();
      const P za = with_z ? __ldg(z2 + i) : K::zero2();
      const P zb = (with_z && two) ? __ldg(z2 + i2) : K::zero2();
      P va[NQ], vb[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        if (q < ng) {
          const P* vq = pairs(V + (int64_t)(g + q) * ldv);
          va[q] = __ldg(vq + i);
          vb[q] = two ? __ldg(vq + i2) : K::zero2();
        }
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        if (q < ng) {
          AR::madd(acc[2 * q], K::x(va[q]), K::x(ua));
          AR::madd(acc[2 * q], K::y(va[q]), K::y(ua));
          AR::madd(acc[2 * q], K::x(vb[q]), K::x(ub));
          AR::madd(acc[2 * q], K::y(vb[q]), K::y(ub));
          if (with_z) {
            AR::madd(acc[2 * q + 1], K::x(va[q]), K::x(za));
            AR::madd(acc[2 * q + 1], K::y(va[q]), K::y(za));
            AR::madd(acc[2 * q + 1], K::x(vb[q]), K::x(zb));
            AR::madd(acc[2 * q + 1], K::y(vb[q]), K::y(zb));
          }
        }
      }
    }
    int row[kGroup];
    unsigned valid = 0u;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      row[2 * q] = g + q;
      row[2 * q + 1] = nv + g + q;
      if (q < ng) valid |= (with_z ? 3u : 1u) << (2 * q);
    }
    block_rows_partial(acc, valid, row, part);
  }
  group_finish(part, with_z ? 2 * nv : nv, gpart, ticket);
}

// DCGS2 update of step j, one launch of nupd + 1 blocks: every block sums
// the reduction's group partials itself (dcgs_sums: the same values in every
// block); blocks below nupd write v_j = (u - V_j s) / rho into slot j and
// u_{j+1} = (z - V_j c - v_j d) / rho into slot j + 1 (with_z; one pass over
// the basis), while block nupd runs the step's Hessenberg bookkeeping
// (dcgs_step) alongside.  The update is skipped once the cycle has stopped
// or at a breakdown (rho = 0); a stop decided by this very step may or may
// not skip it, and the two slots are then not part of the solution either
// way.  Slots below j are only read.
template <class ST>
__global__ void __launch_bounds__(kDotThreads) k_dcgs_update(ST* V, int64_t ldv, int j, int with_z, int64_t n,
                                                             const double* __restrict__ gpart, int ng, double* h,
                                                             int R) {
  using K = KV<ST>;
  using A = typename K::A;
  using AR = Ar<A>;
  using P = typename K::P;
  __shared__ DcgsSums t;
  __shared__ A s_s[kMaxRestart + 1], s_c[kMaxRestart + 1];
  const ArnoldiViews av = arnoldi_views(h, R);
  const int nupd = gridDim.x - 1;
  if (av.sc[4] != 0.0) return;
  dcgs_sums(gpart, ng, j, with_z, t);
  if ((int)blockIdx.x == nupd) {
    dcgs_step(h, R, j, with_z, t);
    return;
  }
  if (!with_z || !(t.rho > 0.0)) return;
  for (int q = threadIdx.x; q < j; q += blockDim.x) {
    s_s[q] = K::from_d(t.s[q]);
    s_c[q] = K::from_d(t.c[q]);
  }
  __syncthreads();
  const A rinv = K::from_d(1.0 / t.rho), d = K::from_d(t.d);
  const ST* Vr = V;  // slots < j: read-only in this launch
  P* u2 = pairs(V + (int64_t)j * ldv);
  P* z2 = pairs(V + (int64_t)(j + 1) * ldv);
  const int64_t n2 = n >> 1;
  for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < n2; i += (int64_t)nupd * kDotThreads) {
    const P ui = u2[i], zi = z2[i];
    A ux = K::x(ui), uy = K::y(ui), zx = K::x(zi), zy = K::y(zi);
    for (int k0 = 0; k0 < j; k0 += kGroup) {
      const int nk = min(kGroup, j - k0);
      P v[kGroup];
#pragma unroll
      for (int q = 0; q < kGroup; ++q)
        if (q < nk) v[q] = __ldg(pairs(Vr + (int64_t)(k0 + q) * ldv) + i);
#pragma unroll
      for (int q = 0; q < kGroup; ++q) {
        if (q < nk) {
          AR::msub(ux, s_s[k0 + q], K::x(v[q]));
          AR::msub(uy, s_s[k0 + q], K::y(v[q]));
          AR::msub(zx, s_c[k0 + q], K::x(v[q]));
          AR::msub(zy, s_c[k0 + q], K::y(v[q]));
        }
      }
    }
    const A vx = AR::mul(AR::norm(ux), rinv), vy = AR::mul(AR::norm(uy), rinv);
    u2[i] = K::pack(vx, vy);
    AR::msub(zx, d, vx);
    AR::msub(zy, d, vy);
    z2[i] = K::pack(AR::mul(AR::norm(zx), rinv), AR::mul(AR::norm(zy), rinv));
  }
}

// v *= s
template <class ST>
__global__ void k_scale(ST* __restrict__ v, double s, int64_t n) {
  using K = KV<ST>;
  using AR = Ar<typename K::A>;
  const typename K::A sa = K::from_d(s);
  typename K::P* v2 = pairs(v);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n >> 1); i += (int64_t)gridDim.x * blockDim.x) {
    const typename K::P a = v2[i];
    v2[i] = K::pack(AR::mul(K::x(a), sa), AR::mul(K::y(a), sa));
  }
}

// x += V y over the cycle's jn columns (y and jn on the device), one value
// per thread (x is the caller's vector: only its element alignment is assumed)
template <class ST>
__global__ void __launch_bounds__(kDotThreads) k_update_x(const ST* __restrict__ V, int64_t ldv,
                                                          const double* __restrict__ y, const double* __restrict__ jn_d,
                                                          ST* __restrict__ x, int64_t n) {
  using K = KV<ST>;
  using A = typename K::A;
  using AR = Ar<A>;
  __shared__ A s_c[kMaxRestart + 1];
  const int jn = (int)*jn_d;
  for (int j = threadIdx.x; j < jn; j += blockDim.x) s_c[j] = K::from_d(y[j]);
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    A a = ld1(x + i);
    int j = 0;
    for (; j + 4 <= jn; j += 4) {
      A v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = ld1(V + (int64_t)(j + k) * ldv + i);
#pragma unroll
      for (int k = 0; k < 4; ++k) AR::madd(a, s_c[j + k], v[k]);
    }
    for (; j < jn; ++j) AR::madd(a, s_c[j], ld1(V + (int64_t)j * ldv + i));
    st1(x + i, AR::norm(a));
  }
}

// binary64 <-> float-float copies, one value per thread (integer split and
// join: no FP64 pipe work)
__global__ void k_split(const double* __restrict__ a, float2* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const ff p = ff_split_double(__ldcs(a + i));
    b[i] = make_float2(p.hi, p.lo);
  }
}
__global__ void k_join(const float2* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = a[i];
    b[i] = ff_to_double(ff{v.x, v.y});
  }
}

}  // namespace krylov
}  // namespace hdg
