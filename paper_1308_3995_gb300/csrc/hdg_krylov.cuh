// Krylov-vector kernels of the GMRES trace solve (Sec. 3.4): dot products
// with the basis, the Arnoldi process as delayed classical Gram-Schmidt with
// re-orthogonalisation (one reduction and one update pass per iteration, the
// Hessenberg bookkeeping on the device), and the solution update.  Every kernel is written once over the storage type ST of
// the vectors:
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
// block in part[row][block]; the last block to finish (a ticket taken after a
// fence) sums every row, one warp per row, in a fixed order -- the results are
// bitwise reproducible.
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

// After every block has written its partials part[j][blockIdx.x], j < nrows,
// the last block to finish sums them.
__device__ __forceinline__ bool last_block_finish(const double* part, int nrows, double* out, double* last_out,
                                                  unsigned* ticket) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (s_last) {
    __threadfence();
    finish_rows(part, nrows, gridDim.x, out, last_out, ticket);
  }
  return s_last;
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
                                                      double* __restrict__ out, unsigned* ticket) {
  block_dots<ST, true>(V, ldv, nvec, w, n >> 1, part);
  last_block_finish(part, nvec, out, nullptr, ticket);
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
// (V orthonormal).  Everything but the two passes runs here, on the device,
// in the last block of the reduction; the host reads the state back once per
// chunk of iterations.
// Views into the solver's h buffer:
//   red [2 (R+1)] the reduction's outputs (a_k = V_k . u, k <= j, then b_k = V_k . z),
//   h1 [R+1] the first projection of the column being built,
//   Hraw [(R+1) R] the Hessenberg matrix (column-major), H [(R+1) R] its
//   rotated (triangular) form, cs, sn [R], g [R+1], y [R], sc [kArnoldiScalars]:
//   sc[0] 1 / rho, sc[1] residual estimate, sc[2] ||M^-1 E||, sc[3] rtol,
//   sc[4] 0 running / 1 converged or breakdown / 2 out of iterations, sc[5]
//   columns of H built in the cycle, sc[6] iterations so far, sc[7] max_iter,
//   sc[8] d = v_j^T z.
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

// Step j's bookkeeping, run by one whole block after the reduction: finish
// column j - 1 (j >= 1) with its Givens rotation and the residual estimate
// |g_j| / ||M^-1 E||, then (with_z: a product z was formed) start column j.
// The recurrences over the rotations run in one thread on operands the block
// loaded into shared memory.
__device__ __forceinline__ void dcgs_step(double* h, int R, int j, int with_z) {
  __shared__ double s_s[kMaxRestart + 1], s_c[kMaxRestart + 1], s_col[kMaxRestart + 1];
  __shared__ double s_cs[kMaxRestart], s_sn[kMaxRestart], s_rho, s_stat;
  ArnoldiViews a = arnoldi_views(h, R);
  double* sc = a.sc;
  const double st = sc[4], its = sc[6], itmax = sc[7];
  if (st != 0.0) return;
  if (j >= 1 && its >= itmax) {  // iteration budget spent before this column
    if (threadIdx.x == 0) sc[4] = 2.0;
    return;
  }
  const int nr = R + 1;
  for (int k = threadIdx.x; k < j; k += blockDim.x) {
    s_s[k] = a.red[k];
    if (with_z) s_c[k] = a.red[j + 1 + k];
    s_col[k] = a.h1[k] + s_s[k];
  }
  for (int k = threadIdx.x; k + 1 < j; k += blockDim.x) {
    s_cs[k] = a.cs[k];
    s_sn[k] = a.sn[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ss = 0.0;
    for (int k = 0; k < j; ++k) ss = fma(s_s[k], s_s[k], ss);
    const double rho = sqrt(fmax(a.red[j] - ss, 0.0));
    double stat = 0.0;
    if (j == 0) {
      a.g[0] = rho;
      if (!(rho > 0.0)) stat = 1.0;
    } else {
      // column j - 1: raw, then rotated by the earlier rotations and a new one
      double* raw = a.Hraw + (size_t)(j - 1) * nr;
      for (int k = 0; k < j; ++k) raw[k] = s_col[k];
      raw[j] = rho;
      s_col[j] = rho;
      for (int k = 0; k + 1 < j; ++k) {
        const double x = s_col[k], z = s_col[k + 1];
        s_col[k] = s_cs[k] * x + s_sn[k] * z;
        s_col[k + 1] = -s_sn[k] * x + s_cs[k] * z;
      }
      const double den = hypot(s_col[j - 1], s_col[j]);
      const double cr = den > 0.0 ? s_col[j - 1] / den : 1.0, sr = den > 0.0 ? s_col[j] / den : 0.0;
      a.cs[j - 1] = cr;
      a.sn[j - 1] = sr;
      s_col[j - 1] = den;
      s_col[j] = 0.0;
      const double gj = a.g[j - 1];
      a.g[j] = -sr * gj;
      a.g[j - 1] = cr * gj;
      double* col = a.H + (size_t)(j - 1) * nr;
      for (int k = 0; k <= j; ++k) col[k] = s_col[k];
      sc[5] = j;
      sc[6] = its + 1.0;
      const double rel = fabs(a.g[j]) / sc[2];
      sc[1] = rel;
      if (!(rel > sc[3]) || !(rho > 0.0)) stat = 1.0;
    }
    if (stat != 0.0) sc[4] = stat;
    s_rho = rho;
    s_stat = stat;
  }
  __syncthreads();
  if (s_stat != 0.0 || !with_z) return;
  // start column j: its first projection h1_j
  const double rho = s_rho, rinv = 1.0 / rho;
  for (int k = threadIdx.x; k < j; k += blockDim.x) {
    double hs = 0.0;  // (H_top s)_k: column i has rows <= i + 1
    for (int i = (k > 0 ? k - 1 : 0); i < j; ++i) hs = fma(a.Hraw[(size_t)i * nr + k], s_s[i], hs);
    a.h1[k] = (s_c[k] - hs) * rinv;
  }
  if (threadIdx.x == 0) {
    double sdotc = 0.0;
    for (int k = 0; k < j; ++k) sdotc = fma(s_s[k], s_c[k], sdotc);
    const double d = (a.red[2 * j + 1] - sdotc) * rinv;
    a.h1[j] = d * rinv - (j >= 1 ? s_s[j - 1] : 0.0);
    sc[0] = rinv;
    sc[8] = d;
  }
}

// H y = g (upper triangular, the cycle's columns): H and g loaded into shared
// memory by the block, the back substitution by one thread on them
__global__ void k_lsq(double* h, int R) {
  __shared__ double s_h[(kMaxRestart + 1) * kMaxRestart], s_y[kMaxRestart + 1];
  ArnoldiViews a = arnoldi_views(h, R);
  const int jn = (int)a.sc[5];
  for (int t = threadIdx.x; t < jn * (R + 1); t += blockDim.x) s_h[t] = a.H[t];
  for (int t = threadIdx.x; t < jn; t += blockDim.x) s_y[t] = a.g[t];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = jn - 1; i >= 0; --i) {
      double v = s_y[i];
      for (int k = i + 1; k < jn; ++k) v -= s_h[(size_t)k * (R + 1) + i] * s_y[k];
      s_y[i] = v / s_h[(size_t)i * (R + 1) + i];
    }
  __syncthreads();
  for (int t = threadIdx.x; t < jn; t += blockDim.x) a.y[t] = s_y[t];
}

// DCGS2 reduction of step j: a_k = V_k . u and b_k = V_k . z for k <= j
// (u = V_j, the candidate; z = V_{j+1} = A u, with_z; without it only the
// a_k: the last step of a cycle, which finishes its last column), then the
// step's bookkeeping (dcgs_step) by the last block to finish.  Every thread
// takes its own pair rows, four basis vectors and both right-hand vectors at
// a time (two rows' loads in flight).
template <class ST>
__global__ void __launch_bounds__(kDotThreads, 2) k_dcgs_reduce(const ST* __restrict__ V, int64_t ldv, int j,
                                                                int with_z, int64_t n, double* __restrict__ part,
                                                                double* h, int R, unsigned* ticket) {
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
  const ArnoldiViews av = arnoldi_views(h, R);
  if (last_block_finish(part, with_z ? 2 * nv : nv, av.red, nullptr, ticket)) {
    __syncthreads();  // the outputs written by the block's warps
    dcgs_step(h, R, j, with_z);
  }
}

// DCGS2 update of step j: v_j = (u - V_j s) / rho into slot j and
// u_{j+1} = (z - V_j c - v_j d) / rho into slot j + 1 (s, c from the
// reduction, 1 / rho and d from dcgs_step), one pass over the basis;
// skipped once the cycle has stopped.  Slots below j are only read.
template <class ST>
__global__ void __launch_bounds__(kDotThreads) k_dcgs_update(ST* V, int64_t ldv, int j, int64_t n, const double* h,
                                                             int R) {
  using K = KV<ST>;
  using A = typename K::A;
  using AR = Ar<A>;
  using P = typename K::P;
  const ArnoldiViews av = arnoldi_views(const_cast<double*>(h), R);
  if (av.sc[4] != 0.0) return;
  __shared__ A s_s[kMaxRestart + 1], s_c[kMaxRestart + 1];
  for (int k = threadIdx.x; k < j; k += blockDim.x) {
    s_s[k] = K::from_d(av.red[k]);
    s_c[k] = K::from_d(av.red[j + 1 + k]);
  }
  __syncthreads();
  const A rinv = K::from_d(av.sc[0]), d = K::from_d(av.sc[8]);
  const ST* Vr = V;  // slots < j: read-only in this launch
  P* u2 = pairs(V + (int64_t)j * ldv);
  P* z2 = pairs(V + (int64_t)(j + 1) * ldv);
  const int64_t n2 = n >> 1;
  for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < n2; i += (int64_t)gridDim.x * kDotThreads) {
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
