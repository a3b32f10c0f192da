// Navier-Stokes element kernel: float-float adjoint-mode instantiations with the far-field
// boundary code (meshes with far-field faces), in a translation unit of their
// own to keep the build's longest unit short.
#include "hdg_ns.cuh"

namespace hdg {

bool launch_ns_adjoint_far_ff(int p, const DevMesh& m, const DevSys& s, const Phys& ph, const void* tab,
                              const TabOff& to, const double* U, const double* Lam, const int* elems, int n,
                              int ntmax, cudaStream_t st, std::string* err) {
  return launch_ns_p<ff, true, true>(p, m, s, ph, (const ff*)tab, to, U, Lam, elems, n, ntmax, st, err);
}

}  // namespace hdg
