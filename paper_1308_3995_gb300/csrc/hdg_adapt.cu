// Adaptation decisions (paper Sec. 4): per-element smoothness sensor and
// adjoint-weighted residual indicator, Doerfler marking and the choice between
// h- and p-refinement.
//
//   S_K = |w - w*|^2_K / |w|^2_K (Sec. 4.4), w* the projection of w onto degree
//         p_K - 1: with the orthonormal hierarchical basis, the share of the
//         squared degree-p_K coefficients of the four conserved fields;
//   eta_K = |N_h(x_h; q~, w~, 0)|_K| (Sec. 4.1) evaluated in the discrete space:
//         the interior residual rows of K weighted by the adjoint's interior
//         coefficients, |res_u,K . U~_K|;
//   marking (Sec. 4.3): the smallest set M with eta_M >= (1 - theta) eta_T,
//         eta^2 summed, taken in the order (eta descending, index ascending);
//         the sums are exact integer sums of v_K = floor(eta_K^2 / max eta^2 *
//         2^bits), bits = 62 - ceil(log2(n + 1)), so the set does not depend on
//         any summation order;
//   decision (Sec. 4.4): marked elements with S_K < eps_s get p-enrichment (1),
//         the others mesh refinement (2).
// The threshold value is found by bisection on integer partial sums (each a
// kernel pass), the tied elements at the threshold by a second bisection on
// the element index.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "hdg_internal.h"
#include "hdg_objects.h"

using namespace hdg;

namespace {

__global__ void k_indicators(int n_elem, int nfield, const int64_t* __restrict__ u_off, const double* __restrict__ U,
                             const double* __restrict__ res_u, const double* __restrict__ Uadj,
                             double* __restrict__ eta2, double* __restrict__ sensor) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= n_elem) return;
  const int64_t o = u_off[K];
  const int n = (int)(u_off[K + 1] - o);
  const int nb = n / nfield;
  int p = 0;
  while ((p + 1) * (p + 2) / 2 < nb) ++p;
  const int nl = p * (p + 1) / 2;                 // modes of degree < p
  const int woff = (nfield == 12) ? 8 * nb : 0;   // w after q_x, q_y in the mixed form
  double num = 0.0, den = 0.0;
  for (int f = 0; f < 4; ++f)
    for (int j = 0; j < nb; ++j) {
      const double c = U[o + woff + f * nb + j];
      den = fma(c, c, den);
      if (j >= nl) num = fma(c, c, num);
    }
  if (sensor) sensor[K] = den > 0.0 ? num / den : 0.0;
  if (eta2 && Uadj) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s = fma(res_u[o + j], Uadj[o + j], s);
    eta2[K] = s * s;
  }
}

__global__ void k_max(const double* __restrict__ x, int n, unsigned long long* out) {
  double m = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = fmax(m, x[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  // non-negative doubles order like their bit patterns
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_quantize(const double* __restrict__ eta2, int n, double mx, int bits, long long* __restrict__ v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = mx > 0.0 ? (long long)floor(ldexp(eta2[i] / mx, bits)) : 0LL;
}

// mode 0: sum of v_i with v_i >= t;  mode 1: count of i < lim with v_i == t;  mode 2: count of v_i > t
__global__ void k_partial(const long long* __restrict__ v, int n, long long t, int mode, int lim,
                          unsigned long long* out) {
  unsigned long long a = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const long long x = v[i];
    if (mode == 0) a += (x >= t) ? (unsigned long long)x : 0ull;
    else if (mode == 1) a += (i < lim && x == t) ? 1ull : 0ull;
    else a += (x > t) ? 1ull : 0ull;
  }
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0 && a) atomicAdd(out, a);  // integer sums: exact in any order
}

__global__ void k_mark(const long long* __restrict__ v, const double* __restrict__ sensor, int n, long long t,
                       int lim, double eps_s, int8_t* __restrict__ code) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long x = v[i];
  const bool mk = t > 0 && (x > t || (x == t && i < lim));
  code[i] = mk ? (int8_t)(sensor[i] < eps_s ? 1 : 2) : (int8_t)0;
}

hdg_status fail(hdg_ctx* ctx, hdg_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

struct Red {
  hdg_ctx* ctx;
  cudaStream_t st;
  unsigned long long* d;
  unsigned long long* h;
  int grid;
  hdg_status rs = HDG_OK;
  unsigned long long run(const long long* v, int n, long long t, int mode, int lim) {
    if (rs != HDG_OK) return 0;
    if (cudaMemsetAsync(d, 0, sizeof(unsigned long long), st) != cudaSuccess) { rs = HDG_ECUDA; return 0; }
    k_partial<<<grid, 256, 0, st>>>(v, n, t, mode, lim, d);
    if (cudaMemcpyAsync(h, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rs = HDG_ECUDA;
      return 0;
    }
    return *h;
  }
};

}  // namespace

extern "C" {

hdg_status hdg_adapt_indicators(hdg_sys* sys, const double* U, const double* Uadj, double* eta2, double* sensor,
                                void* stream) {
  hdg::NvtxRange nvtx_range_("hdg::adapt_indicators");
  if (!sys) return HDG_EINVAL;
  if (!U || (!sensor && !(eta2 && Uadj))) return fail(sys->ctx, HDG_EINVAL, "hdg_adapt_indicators: null argument");
  HDG_ON_DEVICE(sys->ctx, sys->ctx->device);
  const hdg_mesh* M = sys->mesh;
  k_indicators<<<(M->n_elem + 255) / 256, 256, 0, (cudaStream_t)stream>>>(M->n_elem, M->nfield, M->dm.u_off, U,
                                                                          sys->ds.res_u, Uadj, eta2, sensor);
  const cudaError_t ce = cudaGetLastError();
  return ce == cudaSuccess ? HDG_OK : fail(sys->ctx, HDG_ECUDA, std::string("k_indicators: ") + cudaGetErrorString(ce));
}

hdg_status hdg_adapt_mark(hdg_ctx* ctx, int32_t n, const double* eta2, const double* sensor, double theta,
                          double eps_s, int8_t* code, int32_t* n_marked, void* stream) {
  hdg::NvtxRange nvtx_range_("hdg::adapt_mark");
  if (!ctx) return HDG_EINVAL;
  if (n < 1 || !eta2 || !sensor || !code || !(theta >= 0.0 && theta <= 1.0))
    return fail(ctx, HDG_EINVAL, "hdg_adapt_mark: bad arguments");
  HDG_ON_DEVICE(ctx, ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  long long* v = nullptr;
  unsigned long long *dsum = nullptr, *hsum = nullptr;
  if (cudaMallocAsync((void**)&v, sizeof(long long) * (size_t)n + 64, st) != cudaSuccess)
    return fail(ctx, HDG_ENOMEM, "hdg_adapt_mark: cudaMallocAsync failed");
  dsum = (unsigned long long*)(v + n);
  if (cudaMallocHost((void**)&hsum, sizeof(unsigned long long)) != cudaSuccess) {
    cudaFreeAsync(v, st);
    return fail(ctx, HDG_ENOMEM, "hdg_adapt_mark: cudaMallocHost failed");
  }
  Red red{ctx, st, dsum, hsum, std::max(1, std::min(4 * sms, (n + 255) / 256))};
  // max eta^2, then the fixed-point values
  cudaMemsetAsync(dsum, 0, sizeof(unsigned long long), st);
  k_max<<<red.grid, 256, 0, st>>>(eta2, n, dsum);
  cudaMemcpyAsync(hsum, dsum, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
  hdg_status rs = cudaStreamSynchronize(st) == cudaSuccess ? HDG_OK : HDG_ECUDA;
  double mx = 0.0;
  std::memcpy(&mx, hsum, sizeof(double));
  int lg = 0;
  while ((1LL << lg) < (long long)n + 1) ++lg;
  const int bits = 62 - lg;
  long long t_star = 0;
  int lim = 0;
  unsigned long long j = 0;
  if (rs == HDG_OK) {
    k_quantize<<<(n + 255) / 256, 256, 0, st>>>(eta2, n, mx, bits, v);
    const unsigned long long tot = red.run(v, n, 0, 0, 0);
    // target = ceil(tot * (1 - theta)^2), exactly (q = mant 2^(ex - 53))
    const double q = (1.0 - theta) * (1.0 - theta);
    unsigned long long target = 0;
    if (q > 0.0 && tot > 0) {
      int ex = 0;
      const double fr = std::frexp(q, &ex);
      const unsigned long long mant = (unsigned long long)std::ldexp(fr, 53);
      const unsigned __int128 prod = (unsigned __int128)tot * mant;
      const int sh = 53 - ex;
      const unsigned __int128 one = 1;
      target = sh >= 120 ? 1ULL : (unsigned long long)((prod + (one << sh) - 1) >> sh);
    }
    if (target > 0) {
      // largest t with sum_{v >= t} v >= target (t is then a value of some v)
      long long lo = 1, hi = (1LL << bits) + 1;
      while (hi - lo > 1 && red.rs == HDG_OK) {
        const long long mid = lo + (hi - lo) / 2;
        if (red.run(v, n, mid, 0, 0) >= target) lo = mid;
        else hi = mid;
      }
      t_star = lo;
      const unsigned long long above = red.run(v, n, t_star + 1, 0, 0);
      j = (target - above + (unsigned long long)t_star - 1) / (unsigned long long)t_star;  // tied elements needed
      // smallest index bound with j tied elements below it
      int ilo = 0, ihi = n;
      while (ihi - ilo > 0 && red.rs == HDG_OK) {
        const int mid = ilo + (ihi - ilo) / 2;
        if (red.run(v, n, t_star, 1, mid) >= j) ihi = mid;
        else ilo = mid + 1;
      }
      lim = ilo;
    }
    rs = red.rs;
  }
  if (rs == HDG_OK) {
    k_mark<<<(n + 255) / 256, 256, 0, st>>>(v, sensor, n, t_star, lim, eps_s, code);
    if (cudaGetLastError() != cudaSuccess) rs = HDG_ECUDA;
  }
  if (rs == HDG_OK && n_marked) {
    const unsigned long long n_above = t_star > 0 ? red.run(v, n, t_star, 2, 0) : 0ull;
    rs = red.rs;
    *n_marked = (int32_t)(n_above + j);
  }
  cudaFreeAsync(v, st);
  cudaStreamSynchronize(st);
  cudaFreeHost(hsum);
  return rs == HDG_OK ? HDG_OK : fail(ctx, rs, "hdg_adapt_mark: CUDA call failed");
}

}  // extern "C"
