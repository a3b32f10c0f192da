// Navier-Stokes element kernel: float-float instantiations.
#include "hdg_ns.cuh"

namespace hdg {

bool launch_ns_far_ff(int p, const DevMesh& m, const DevSys& s, const Phys& ph, const void* tab, const TabOff& to,
                      const double* U, const double* Lam, const int* elems, int n, int ntmax, cudaStream_t st,
                      std::string* err);

bool launch_ns_ff(int p, const DevMesh& m, const DevSys& s, const Phys& ph, const void* tab, const TabOff& to,
                  const double* U, const double* Lam, const int* elems, int n, int ntmax, cudaStream_t st,
                  std::string* err) {
  if (m.far) return launch_ns_far_ff(p, m, s, ph, tab, to, U, Lam, elems, n, ntmax, st, err);
  return launch_ns_p<ff>(p, m, s, ph, (const ff*)tab, to, U, Lam, elems, n, ntmax, st, err);
}

int ns_occupancy_ff(int p, int ntmax) { return ns_occ_p<ff>(p, ntmax); }

}  // namespace hdg
