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
#include <type_traits>

#include "hdg_euler.cuh"

namespace hdg {

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
    if (f < 0) continue;  // boundary face: no trace unknowns
    const int len = 4 * (m.face_p[f] + 1);
    const double* dl = dLam + m.lam_off[f];
    for (int t = 0; t < len; ++t, ++c) acc += xk[(size_t)c * n + r] * dl[t];
  }
  dU[m.u_off[K] + r] = xk[(size_t)c * n + r] - acc;
}

// Reconstruction over the work list of a batched launch: one thread per
// (item, interior row) of the items of one degree; the item's system gives X,
// dLambda, dU and the mesh plan.
__global__ void k_recover_batch(BatchRef bt, int n_items, int n) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n_items * n) return;
  const int it = (int)(idx / n), r = (int)(idx - (int64_t)it * n);
  int lo = 0, hi = bt.n_segs - 1;  // last segment with first <= it
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bt.segs[mid].first <= it) lo = mid;
    else hi = mid - 1;
  }
  const BatchSeg sg = bt.segs[lo];
  const ReqDesc* d = bt.descs + sg.desc;
  const int K = sg.elems[it - sg.first];
  const DevMesh& m = d->m;
  const double* xk = d->s.X + m.x_off[K];
  int c = 0;
  double acc = 0.0;
  for (int a = 0; a < 3; ++a) {
    const int f = m.elem_face[3 * (size_t)K + a];
    if (f < 0) continue;
    const int len = 4 * (m.face_p[f] + 1);
    const double* dl = d->dLam + m.lam_off[f];
    for (int t = 0; t < len; ++t, ++c) acc += xk[(size_t)c * n + r] * dl[t];
  }
  d->dU[m.u_off[K] + r] = xk[(size_t)c * n + r] - acc;
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------

template <class T>
static bool launch_euler_p(int p, const DevMesh& m, const DevSys& s, const Phys& ph, const T* tab, const TabOff& to,
                           const double* U, const double* Lam, const int* elems, int n, int ntmax, cudaStream_t st,
                           std::string* err) {
  switch (p) {
    case 1: return launch_euler_bucket<1, T>(m, s, ph, tab, to, U, Lam, elems, n, ntmax, st, err);
    case 2: return launch_euler_bucket<2, T>(m, s, ph, tab, to, U, Lam, elems, n, ntmax, st, err);
    case 3: return launch_euler_bucket<3, T>(m, s, ph, tab, to, U, Lam, elems, n, ntmax, st, err);
    case 4: return launch_euler_bucket<4, T>(m, s, ph, tab, to, U, Lam, elems, n, ntmax, st, err);
  }
  *err = "degree out of range";
  return false;
}

template <int P, class T>
static int euler_occupancy(int ntmax) {
  const EulerLayout<P> lay(ldr_for(ntmax), nkmax_for(P, ntmax));
  const size_t bytes = sizeof(T) * (size_t)lay.total;
  const size_t cap = sizeof(T) * (size_t)EulerLayout<P>(ldr_for(kMaxNt), kMaxP + 1).total;
  if (set_smem_cap(k_condense_euler<P, T>, cap, bytes) != cudaSuccess) return 0;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_condense_euler<P, T>, kCondThreads, bytes);
  return per_sm;
}

int condense_occupancy(const Phys& ph, int p, int ntmax) {
  if (ph.model == HDG_NS_MIXED) return ns_occupancy(ph, p, ntmax);
  if (ph.precision == HDG_MIXED_TF32 || ph.precision == HDG_MIXED_BF16) return euler_mixed_occupancy(ph, p, ntmax, false);
  const bool d = ph.precision == HDG_FP64;
  switch (p) {
    case 1: return d ? euler_occupancy<1, double>(ntmax) : euler_occupancy<1, ff>(ntmax);
    case 2: return d ? euler_occupancy<2, double>(ntmax) : euler_occupancy<2, ff>(ntmax);
    case 3: return d ? euler_occupancy<3, double>(ntmax) : euler_occupancy<3, ff>(ntmax);
    case 4: return d ? euler_occupancy<4, double>(ntmax) : euler_occupancy<4, ff>(ntmax);
  }
  return 0;
}

int launch_condense(const DevMesh& m, const DevSys& s, const Phys& ph, const double* tab, const void* tab_ff,
                    const TabOff& to, const double* U, const double* Lam, const int* const* bucket,
                    const int* bucket_n, const int* bucket_ntmax, void* stream, std::string* err,
                    void* const* bucket_streams, const BucketNt* bucket_nt) {
  if (ph.model == HDG_NS_MIXED)
    return launch_condense_ns(m, s, ph, tab, tab_ff, to, U, Lam, bucket, bucket_n, bucket_ntmax, stream, err,
                              bucket_streams, bucket_nt);
  int launches = 0;
  for (int p = 1; p <= kMaxP; ++p) {
    if (bucket_n[p] == 0) continue;
    cudaStream_t st = (cudaStream_t)(bucket_streams ? bucket_streams[p] : stream);
    const int* el = bucket[p];
    const int k = launch_groups(ph, p, bucket_n[p], bucket_ntmax[p], bucket_nt, [&](int off, int n, int ntmax) {
      if (ph.precision == HDG_MIXED_TF32 || ph.precision == HDG_MIXED_BF16)
        return launch_euler_mixed(p, m, s, ph, tab, to, U, Lam, el + off, n, ntmax, st, err, BatchRef{},
                                  m.elem_bc != nullptr);
      if (ph.precision == HDG_FP64)
        return launch_euler_p<double>(p, m, s, ph, tab, to, U, Lam, el + off, n, ntmax, st, err);
      return launch_euler_p<ff>(p, m, s, ph, (const ff*)tab_ff, to, U, Lam, el + off, n, ntmax, st, err);
    });
    if (k < 0) return -1;
    launches += k;
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

// batched launches (hdg_batch_*)
template <class T>
static bool launch_euler_batch_p(int p, const Phys& ph, const T* tab, const TabOff& to, const BatchRef& bt,
                                 int n, int ntmax, bool bounded, cudaStream_t st, std::string* err) {
  const DevMesh m{};
  const DevSys s{};
  switch (p) {
    case 1: return launch_euler_bucket<1, T, 0, true>(m, s, ph, tab, to, nullptr, nullptr, nullptr, n, ntmax, st, err, bt, bounded);
    case 2: return launch_euler_bucket<2, T, 0, true>(m, s, ph, tab, to, nullptr, nullptr, nullptr, n, ntmax, st, err, bt, bounded);
    case 3: return launch_euler_bucket<3, T, 0, true>(m, s, ph, tab, to, nullptr, nullptr, nullptr, n, ntmax, st, err, bt, bounded);
    case 4: return launch_euler_bucket<4, T, 0, true>(m, s, ph, tab, to, nullptr, nullptr, nullptr, n, ntmax, st, err, bt, bounded);
  }
  *err = "degree out of range";
  return false;
}

bool launch_condense_batch(int p, const Phys& ph, const double* tab, const void* tab_ff, const TabOff& to,
                           const BatchRef& bt, int n_items, int ntmax, bool bounded, void* stream, std::string* err) {
  if (ph.model == HDG_NS_MIXED) return launch_ns_batch(p, ph, tab, tab_ff, to, bt, n_items, ntmax, stream, err);
  cudaStream_t st = (cudaStream_t)stream;
  if (ph.precision == HDG_FP64) return launch_euler_batch_p<double>(p, ph, tab, to, bt, n_items, ntmax, bounded, st, err);
  return launch_euler_batch_p<ff>(p, ph, (const ff*)tab_ff, to, bt, n_items, ntmax, bounded, st, err);
}

template <int P, class T>
static int euler_batch_occupancy(int ntmax, bool bounded) {
  const EulerLayout<P> lay(ldr_for(ntmax), nkmax_for(P, ntmax, bounded));
  const size_t bytes = sizeof(T) * (size_t)lay.total;
  const size_t cap = sizeof(T) * (size_t)EulerLayout<P>(ldr_for(kMaxNt), kMaxP + 1).total;
  if (set_smem_cap(k_condense_euler<P, T, 0, true>, cap, bytes) != cudaSuccess) return 0;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_condense_euler<P, T, 0, true>, kCondThreads, bytes);
  return per_sm;
}

int batch_occupancy(const Phys& ph, int p, int ntmax, bool bounded) {
  if (ph.model == HDG_NS_MIXED) return ns_occupancy(ph, p, ntmax);
  const bool d = ph.precision == HDG_FP64;
  switch (p) {
    case 1: return d ? euler_batch_occupancy<1, double>(ntmax, bounded) : euler_batch_occupancy<1, ff>(ntmax, bounded);
    case 2: return d ? euler_batch_occupancy<2, double>(ntmax, bounded) : euler_batch_occupancy<2, ff>(ntmax, bounded);
    case 3: return d ? euler_batch_occupancy<3, double>(ntmax, bounded) : euler_batch_occupancy<3, ff>(ntmax, bounded);
    case 4: return d ? euler_batch_occupancy<4, double>(ntmax, bounded) : euler_batch_occupancy<4, ff>(ntmax, bounded);
  }
  return 0;
}

bool launch_recover_batch(int p, int nfield, const BatchRef& bt, int n_items, void* stream, std::string* err) {
  const int n = nfield * n_basis(p);
  const int64_t total = (int64_t)n_items * n;
  const int threads = 256;
  k_recover_batch<<<(unsigned)((total + threads - 1) / threads), threads, 0, (cudaStream_t)stream>>>(bt, n_items, n);
  const cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) { *err = cudaGetErrorString(ce); return false; }
  return true;
}

}  // namespace hdg
