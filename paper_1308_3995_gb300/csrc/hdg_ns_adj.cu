// Navier-Stokes element kernel, adjoint mode (Sec. 4.2: X~ = A^{-T} [C^T | F~]):
// binary64 instantiations and the dispatcher over the arithmetic.
#include "hdg_ns.cuh"

namespace hdg {

bool launch_ns_adjoint_ff(int p, const DevMesh& m, const DevSys& s, const Phys& ph, const void* tab,
                          const TabOff& to, const double* U, const double* Lam, const int* elems, int n, int ntmax,
                          cudaStream_t st, std::string* err);

bool launch_ns_adjoint_far(int p, const DevMesh& m, const DevSys& s, const Phys& ph, const double* tab,
                           const TabOff& to, const double* U, const double* Lam, const int* elems, int n, int ntmax,
                           cudaStream_t st, std::string* err);

bool launch_ns_adjoint(int p, const DevMesh& m, const DevSys& s, const Phys& ph, const double* tab,
                       const void* tab_ff, const TabOff& to, const double* U, const double* Lam, const int* elems,
                       int n, int ntmax, cudaStream_t st, std::string* err) {
  if (ph.precision == HDG_FP64)
    return m.far ? launch_ns_adjoint_far(p, m, s, ph, tab, to, U, Lam, elems, n, ntmax, st, err)
                 : launch_ns_p<double, true>(p, m, s, ph, tab, to, U, Lam, elems, n, ntmax, st, err);
  return launch_ns_adjoint_ff(p, m, s, ph, tab_ff, to, U, Lam, elems, n, ntmax, st, err);
}

}  // namespace hdg
