// hdg_condense_noalloc: the condensation of hdg_condense for callers that
// cannot allocate device memory when they call it -- serving loops with a
// latency budget (cudaMalloc and cudaFree can synchronise the whole device and
// take unbounded time) and hosts whose device memory is owned by another
// allocator or fixed at start-up.  The caller passes the inputs and every
// output buffer; the only work space the kernel needs (for each face, the
// side-1 element's half of the diagonal block, of E and of the trace residual,
// plus an int32 arrival counter) lives in the fixed array below, so this entry
// point calls no cudaMalloc, cudaFree or other allocating routine.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "hdg_internal.h"

using namespace hdg;

namespace {

constexpr size_t kWorkBytes = size_t(64) << 20;  // 64 MiB: the largest work space accepted
constexpr int kMaxDevices = 64;

// The work space.  Every GPU that loads this library holds these 64 MiB until
// the process exits.  In host code the name is only a host-side stand-in; the
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_work[kWorkBytes];

std::mutex g_mu;
void* g_work_addr[kMaxDevices] = {};

// Device address of the work array on `device`, resolved once per device.
// The caller has made `device` current (DeviceGuard), so the lookup leaves the
// thread's current device as it found it.
hdg_status work_address(int device, void** out, std::string* err) {
  if (device < 0 || device >= kMaxDevices) {
    *err = "hdg_condense_noalloc: device ordinal out of range";
    return HDG_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_work_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_work);
    if (e != cudaSuccess || !p) {
      *err = std::string("hdg_condense_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
      return HDG_ECUDA;
    }
    g_work_addr[device] = p;
  }
  *out = g_work_addr[device];
  return HDG_OK;
}

inline size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" hdg_status hdg_condense_noalloc(const hdg_mesh* mesh, const hdg_params* P, const double* U,
                                           const double* Lam, double* X, double* K_vals, double* E, double* res_u,
                                           double* res_lam, int32_t* elem_status, void* stream) {
  if (!mesh || !P) return HDG_EINVAL;
  PlanRef pr = plan_ref(mesh);
  if (!U || !Lam || !X || !K_vals || !E || !res_u || !res_lam || !elem_status) {
    *pr.err = "hdg_condense_noalloc: null argument";
    return HDG_EINVAL;
  }
  if ((P->model == HDG_EULER) != (pr.nfield == 4)) {
    *pr.err = "hdg_condense_noalloc: model does not match the mesh's field count";
    return HDG_EINVAL;
  }
  if (P->model != HDG_EULER || P->precision != HDG_FP64) {
    *pr.err = "hdg_condense_noalloc: only the FP64 Euler path has an allocation-free variant";
    return HDG_ENOTSUP;
  }
  if (!(P->gamma > 1.0) || !(P->alpha > 0.0) || !(P->mach > 0.0)) {
    *pr.err = "hdg_condense_noalloc: need gamma > 1, alpha > 0, mach > 0";
    return HDG_EINVAL;
  }
  // work space layout: counters | diagonal halves | E halves | residual halves
  const size_t b_cnt = round256(sizeof(int32_t) * (size_t)pr.n_face);
  const size_t b_dh = round256(sizeof(double) * (size_t)pr.dh_len);
  const size_t b_lam = round256(sizeof(double) * (size_t)pr.lam_len);
  const size_t need = b_cnt + b_dh + 2 * b_lam;
  if (need > kWorkBytes) {
    *pr.err = "hdg_condense_noalloc: this mesh needs " + std::to_string(need) +
              " bytes of work space, more than the fixed limit of " + std::to_string(kWorkBytes) +
              " bytes (64 MiB); use hdg_sys_create + hdg_condense for it";
    return HDG_EINVAL;
  }
  // the mesh's device is current for the memset and the launches; the
  // caller's current device is restored on every return path
  hdg::DeviceGuard dg(pr.device);
  if (!dg.ok()) {
    *pr.err = "hdg_condense_noalloc: cudaSetDevice failed";
    return HDG_ECUDA;
  }
  void* base = nullptr;
  hdg_status st = work_address(pr.device, &base, pr.err);
  if (st != HDG_OK) return st;
  unsigned char* w = (unsigned char*)base;
  DevSys ds{};
  ds.X = X;
  ds.K = K_vals;
  ds.E = E;
  ds.res_u = res_u;
  ds.res_lam = res_lam;
  ds.status = elem_status;
  ds.face_cnt = (int32_t*)w;
  ds.dhalf1 = (double*)(w + b_cnt);
  ds.ehalf1 = (double*)(w + b_cnt + b_dh);
  ds.rhalf1 = (double*)(w + b_cnt + b_dh + b_lam);
  // the arrival counters must start at zero; the array keeps the last call's contents
  cudaError_t e = cudaMemsetAsync(ds.face_cnt, 0, sizeof(int32_t) * (size_t)pr.n_face, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    *pr.err = std::string("hdg_condense_noalloc: ") + cudaGetErrorString(e);
    return HDG_ECUDA;
  }
  Phys ph{};
  ph.gamma = P->gamma;
  ph.alpha = P->alpha;
  ph.prandtl = P->prandtl;
  ph.mu_inf = P->mach / P->reynolds;
  ph.suth_s = 110.4 / P->t_inf;
  ph.cfl = P->cfl;
  ph.sc_eps0 = P->sc_eps0 > 0.0 ? P->sc_eps0 : 0.0;
  ph.sc_beta = P->sc_beta;
  far_field_state(*P, ph.winf);
  ph.model = P->model;
  ph.precision = P->precision;
  ph.persistent = 1;
  phys_default_grid(ph);
  std::string err;
  const int n = launch_condense(*pr.dm, ds, ph, pr.tab, pr.tab_ff, *pr.off, U, Lam, pr.bucket, pr.bucket_n, pr.bucket_ntmax,
                                stream, &err, nullptr, pr.bucket_nt);
  if (n < 0) {
    *pr.err = "hdg_condense_noalloc: " + err;
    return HDG_ECUDA;
  }
  return HDG_OK;
}
