// Navier-Stokes element kernel: binary64 instantiations with the far-field
// boundary code (meshes with far-field faces), in a translation unit of their
// own to keep the build's longest unit short.
#include "hdg_ns.cuh"

namespace hdg {

bool launch_ns_far(int p, const DevMesh& m, const DevSys& s, const Phys& ph, const double* tab, const TabOff& to,
                   const double* U, const double* Lam, const int* elems, int n, int ntmax, cudaStream_t st,
                   std::string* err) {
  return launch_ns_p<double, false, true>(p, m, s, ph, tab, to, U, Lam, elems, n, ntmax, st, err);
}

}  // namespace hdg
