// Euler element kernel with the mixed-precision local solve (precisions
// HDG_MIXED_TF32 and HDG_MIXED_BF16): residual and Jacobian assembled in
// binary64, the local LU and solves in binary32 on the tensor cores, the
// solves refined against binary64 residuals (hdg_lu_tc.cuh).  A translation
// unit of its own so the library builds in parallel.
#include "hdg_euler.cuh"

namespace hdg {

template <int LS>
static bool launch_mixed_p(int p, const DevMesh& m, const DevSys& s, const Phys& ph, const double* tab,
                           const TabOff& to, const double* U, const double* Lam, const int* elems, int n, int ntmax,
                           cudaStream_t st, std::string* err, const BatchRef& bt, bool bounded) {
  switch (p) {
    case 1: return launch_euler_bucket<1, double, LS>(m, s, ph, tab, to, U, Lam, elems, n, ntmax, st, err, bt, bounded);
    case 2: return launch_euler_bucket<2, double, LS>(m, s, ph, tab, to, U, Lam, elems, n, ntmax, st, err, bt, bounded);
    case 3: return launch_euler_bucket<3, double, LS>(m, s, ph, tab, to, U, Lam, elems, n, ntmax, st, err, bt, bounded);
    case 4: return launch_euler_bucket<4, double, LS>(m, s, ph, tab, to, U, Lam, elems, n, ntmax, st, err, bt, bounded);
  }
  *err = "degree out of range";
  return false;
}

bool launch_euler_mixed(int p, const DevMesh& m, const DevSys& s, const Phys& ph, const double* tab, const TabOff& to,
                        const double* U, const double* Lam, const int* elems, int n, int ntmax, void* stream,
                        std::string* err, const BatchRef& bt, bool bounded) {
  cudaStream_t st = (cudaStream_t)stream;
  if (ph.precision == HDG_MIXED_TF32)
    return launch_mixed_p<kTcTF32x3>(p, m, s, ph, tab, to, U, Lam, elems, n, ntmax, st, err, bt, bounded);
  if (ph.precision == HDG_MIXED_BF16)
    return launch_mixed_p<kTcBF16>(p, m, s, ph, tab, to, U, Lam, elems, n, ntmax, st, err, bt, bounded);
  *err = "not a mixed-precision local solve";
  return false;
}

template <int P, int LS>
static int mixed_occ(int ntmax, bool bounded) {
  const EulerLayout<P> lay(ldr_for(ntmax), nkmax_for(P, ntmax, bounded), true);
  const size_t bytes = sizeof(double) * (size_t)lay.total;
  const size_t cap = sizeof(double) * (size_t)EulerLayout<P>(ldr_for(kMaxNt), kMaxP + 1, true).total;
  if (set_smem_cap(k_condense_euler<P, double, LS>, cap, bytes) != cudaSuccess) return 0;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_condense_euler<P, double, LS>, kCondThreads, bytes);
  return per_sm;
}

template <int LS>
static int mixed_occ_p(int p, int ntmax, bool bounded) {
  switch (p) {
    case 1: return mixed_occ<1, LS>(ntmax, bounded);
    case 2: return mixed_occ<2, LS>(ntmax, bounded);
    case 3: return mixed_occ<3, LS>(ntmax, bounded);
    case 4: return mixed_occ<4, LS>(ntmax, bounded);
  }
  return 0;
}

int euler_mixed_occupancy(const Phys& ph, int p, int ntmax, bool bounded) {
  return ph.precision == HDG_MIXED_TF32 ? mixed_occ_p<kTcTF32x3>(p, ntmax, bounded)
                                        : mixed_occ_p<kTcBF16>(p, ntmax, bounded);
}

}  // namespace hdg
