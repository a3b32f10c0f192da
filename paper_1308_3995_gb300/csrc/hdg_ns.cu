// Navier-Stokes element kernel: binary64 instantiations and the dispatcher.
#include "hdg_ns.cuh"

namespace hdg {

bool launch_ns_far(int p, const DevMesh& m, const DevSys& s, const Phys& ph, const double* tab, const TabOff& to,
                   const double* U, const double* Lam, const int* elems, int n, int ntmax, cudaStream_t st,
                   std::string* err);

bool launch_ns_ff(int p, const DevMesh& m, const DevSys& s, const Phys& ph, const void* tab, const TabOff& to,
                  const double* U, const double* Lam, const int* elems, int n, int ntmax, cudaStream_t st,
                  std::string* err);

int ns_occupancy_ff(int p, int ntmax);

// adjoint-mode instantiations (Sec. 4.2), in translation units of their own
bool launch_ns_adjoint(int p, const DevMesh& m, const DevSys& s, const Phys& ph, const double* tab,
                       const void* tab_ff, const TabOff& to, const double* U, const double* Lam, const int* elems,
                       int n, int ntmax, cudaStream_t st, std::string* err);

int ns_occupancy(const Phys& ph, int p, int ntmax) {
  return ph.precision == HDG_FP64 ? ns_occ_p<double>(p, ntmax) : ns_occupancy_ff(p, ntmax);
}

int launch_condense_ns(const DevMesh& m, const DevSys& s, const Phys& ph, const double* tab, const void* tab_ff,
                       const TabOff& to, const double* U, const double* Lam, const int* const* bucket,
                       const int* bucket_n, const int* bucket_ntmax, void* stream, std::string* err,
                       void* const* bucket_streams, const BucketNt* bucket_nt) {
  int launches = 0;
  for (int p = 1; p <= kMaxP; ++p) {
    if (bucket_n[p] == 0) continue;
    cudaStream_t st = (cudaStream_t)(bucket_streams ? bucket_streams[p] : stream);
    const int* el = bucket[p];
    const int k = launch_groups(ph, p, bucket_n[p], bucket_ntmax[p], bucket_nt, [&](int off, int n, int ntmax) {
      if (ph.adjoint) return launch_ns_adjoint(p, m, s, ph, tab, tab_ff, to, U, Lam, el + off, n, ntmax, st, err);
      if (ph.precision == HDG_FP64)
        return m.far ? launch_ns_far(p, m, s, ph, tab, to, U, Lam, el + off, n, ntmax, st, err)
                     : launch_ns_p<double>(p, m, s, ph, tab, to, U, Lam, el + off, n, ntmax, st, err);
      return launch_ns_ff(p, m, s, ph, tab_ff, to, U, Lam, el + off, n, ntmax, st, err);
    });
    if (k < 0) return -1;
    launches += k;
  }
  return launches;
}

}  // namespace hdg
