// Navier-Stokes element kernel over a batch work list (hdg_batch_condense):
// binary64 instantiations and the dispatcher over the arithmetic.  A
// translation unit of its own so the library builds in parallel.
#include "hdg_ns.cuh"

namespace hdg {

bool launch_ns_batch_ff(int p, const Phys& ph, const void* tab, const TabOff& to, const BatchRef& bt, int n,
                        int ntmax, cudaStream_t st, std::string* err);

bool launch_ns_batch(int p, const Phys& ph, const double* tab, const void* tab_ff, const TabOff& to,
                     const BatchRef& bt, int n_items, int ntmax, void* stream, std::string* err) {
  cudaStream_t st = (cudaStream_t)stream;
  if (ph.precision != HDG_FP64) return launch_ns_batch_ff(p, ph, tab_ff, to, bt, n_items, ntmax, st, err);
  const DevMesh m{};
  const DevSys s{};
  switch (p) {
    case 1: return launch_ns_bucket<1, double, false, true>(m, s, ph, tab, to, nullptr, nullptr, nullptr, n_items, ntmax, st, err, bt);
    case 2: return launch_ns_bucket<2, double, false, true>(m, s, ph, tab, to, nullptr, nullptr, nullptr, n_items, ntmax, st, err, bt);
    case 3: return launch_ns_bucket<3, double, false, true>(m, s, ph, tab, to, nullptr, nullptr, nullptr, n_items, ntmax, st, err, bt);
    case 4: return launch_ns_bucket<4, double, false, true>(m, s, ph, tab, to, nullptr, nullptr, nullptr, n_items, ntmax, st, err, bt);
  }
  *err = "degree out of range";
  return false;
}

}  // namespace hdg
