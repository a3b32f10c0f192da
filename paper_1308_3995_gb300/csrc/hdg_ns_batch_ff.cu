// Navier-Stokes element kernel over a batch work list: float-float instantiations.
#include "hdg_ns.cuh"

namespace hdg {

bool launch_ns_batch_ff(int p, const Phys& ph, const void* tab, const TabOff& to, const BatchRef& bt, int n,
                        int ntmax, cudaStream_t st, std::string* err) {
  const DevMesh m{};
  const DevSys s{};
  const ff* t = (const ff*)tab;
  switch (p) {
    case 1: return launch_ns_bucket<1, ff, false, true>(m, s, ph, t, to, nullptr, nullptr, nullptr, n, ntmax, st, err, bt);
    case 2: return launch_ns_bucket<2, ff, false, true>(m, s, ph, t, to, nullptr, nullptr, nullptr, n, ntmax, st, err, bt);
    case 3: return launch_ns_bucket<3, ff, false, true>(m, s, ph, t, to, nullptr, nullptr, nullptr, n, ntmax, st, err, bt);
    case 4: return launch_ns_bucket<4, ff, false, true>(m, s, ph, t, to, nullptr, nullptr, nullptr, n, ntmax, st, err, bt);
  }
  *err = "degree out of range";
  return false;
}

}  // namespace hdg
