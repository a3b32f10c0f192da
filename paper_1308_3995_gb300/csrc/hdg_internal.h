// Internal declarations shared by the host planner and the CUDA kernels.
#pragma once

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/hdg.h"

#ifdef __CUDACC__
#define HDG_HD __host__ __device__
#else
#define HDG_HD
#endif

namespace hdg {

// Named range around a host API call for timeline tools (NVTX; a no-op unless a
// tool is attached): the library's phases show up as hdg::condense, ... .
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Makes `device` current for the lifetime of the guard and restores the
// calling thread's current device afterwards, so that no entry point leaves a
// multi-GPU host thread on another GPU.  ok() is false when the switch failed.
class DeviceGuard {
 public:
  explicit DeviceGuard(int device) {
    if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
    if (prev_ != device) {
      ok_ = cudaSetDevice(device) == cudaSuccess;
      switched_ = ok_ && prev_ >= 0;
    }
  }
  ~DeviceGuard() {
    if (switched_) cudaSetDevice(prev_);
  }
  bool ok() const { return ok_; }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;

 private:
  int prev_ = -1;
  bool ok_ = true, switched_ = false;
};

// Entry-point prologue: `dev` current until the enclosing function returns;
// `fail` is the calling translation unit's error helper.  A pending
// non-sticky error left by an earlier call outside this entry point (the
// caller's, or another library's) is discarded first, so that the launch
// checks below report only this call's own errors (a sticky error -- a
// kernel fault -- cannot be cleared and still surfaces).
#define HDG_ON_DEVICE(ctx, dev)                                                     \
  ::hdg::DeviceGuard hdg_device_guard_(dev);                                        \
  if (!hdg_device_guard_.ok()) return fail(ctx, HDG_ECUDA, "cudaSetDevice failed"); \
  (void)cudaGetLastError()

constexpr int kMaxP = 4;          // element degrees 1..4
constexpr int kMaxNt = 60;        // 3 faces x 4 fields x (4 + 1) modes
constexpr int kNtSlots = kMaxNt / 4 + 1;  // element trace sizes 0, 4, ..., kMaxNt

// Elements of each degree bucket per trace size (slot s: nt = 4 s), each
// bucket's element list sorted by trace size.
struct BucketNt {
  int cnt[kMaxP + 1][kNtSlots];
};
constexpr int kCondThreads = 128; // threads per element CTA of the condensation kernels

HDG_HD constexpr inline int n_basis(int p) { return (p + 1) * (p + 2) / 2; }

// offsets (in doubles) of every table inside one device buffer
struct TabOff {
  int vol_w[kMaxP + 1], vol_phi[kMaxP + 1], vol_gxi[kMaxP + 1], vol_geta[kMaxP + 1];
  int edge_s[kMaxP + 1], edge_w[kMaxP + 1], edge_psi[kMaxP + 1];
  int edge_phi[kMaxP + 1][kMaxP + 1][3][2];   // [p][pe][local face][flip]
  // derived reference matrices (unit edge length, unit det J):
  int vol_dref[kMaxP + 1];                    // [2][np][np]: sum_q w_q dphi_i/dxi_r phi_j
  int vol_stiff[kMaxP + 1];                   // [3][np][np]: sum_q w_q of d0i d0j, d0i d1j + d1i d0j, d1i d1j
  int face_mass[kMaxP + 1][kMaxP + 1][3];     // [np][np]: sum_g w_g phi_i phi_j on local face lf
  int edge_cross[kMaxP + 1][kMaxP + 1][3][2]; // [pe+1][np]: sum_g w_g psi_k phi_j
};

struct Tables {
  TabOff off{};
  std::vector<double> data;
};
void build_tables(Tables& T);

// Flow parameters as the kernels use them.
struct Phys {
  double gamma, alpha, prandtl, mu_inf, suth_s, cfl;
  double sc_eps0, sc_beta;  // shock capturing (Sec. 3.2); off unless sc_eps0 > 0
  double winf[4];           // far-field conserved state (Sec. 2.1)
  int model, precision;
  int refine_max;      // mixed-precision local solves: at most this many corrections,
  double refine_tol;   // stopping when the correction is below refine_tol * max|X|
  int persistent;  // 1: grid = SMs x resident CTAs (loop over elements); 0: one CTA per element
  int adjoint;     // 1: adjoint local solves X~ = A^{-T} [C^T | F~] only (Sec. 4.2)
  // launch shape per degree (autotuned): -1 default (by `persistent`), 0 one CTA per element,
  // k > 0 persistent grid of k CTAs per SM (capped by the occupancy)
  int grid[kMaxP + 1];
};

// far-field conserved state of Sec. 2.1: rho = 1, |v| = mach at angle aoa, p = 1/gamma
inline void far_field_state(const hdg_params& P, double* w) {
  const double a = P.aoa * 3.14159265358979323846 / 180.0;
  const double u = P.mach * std::cos(a), v = P.mach * std::sin(a), p = 1.0 / P.gamma;
  w[0] = 1.0;
  w[1] = u;
  w[2] = v;
  w[3] = p / (P.gamma - 1.0) + 0.5 * (u * u + v * v);
}

inline void phys_default_grid(Phys& ph) {
  for (int p = 0; p <= kMaxP; ++p) ph.grid[p] = -1;
}

// Dynamic shared-memory cap of a kernel instance (cudaFuncAttributeMaxDynamicSharedMemorySize).
// The attribute belongs to the instance, not to a launch, so host threads that launch or query
// the instance at once must not lower it under one another: every launch and occupancy query
// sets the same value, the instance's largest layout (trace size kMaxNt), and passes its own
// size, which is below it.  Only if the device refuses that value is the caller's size set.
template <class K>
inline cudaError_t set_smem_cap(K* kernel, size_t max_bytes, size_t bytes) {
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_bytes) == cudaSuccess)
    return cudaSuccess;
  (void)cudaGetLastError();
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// number of CTAs of a condensation launch of n elements of degree p
inline long condense_grid(const Phys& ph, int p, int sms, int per_sm, int n) {
  const int g = ph.grid[p];
  long grid;
  if (g < 0) grid = ph.persistent ? (long)sms * per_sm : (long)n;
  else if (g == 0) grid = n;
  else grid = (long)sms * (g < per_sm ? g : per_sm);
  return grid > n ? n : grid;
}

// Device-resident mesh plan handed to kernels by value.
struct DevMesh {
  int n_elem, n_face, nfield;
  const double* xy;          // [n_elem][6]
  const int* elem_face;      // [n_elem][3]
  const uint8_t* elem_info;  // bits 0-2: flip of local face l; bits 3-5: side of this element on face l
  const int* face_p;         // [n_face]
  const int64_t* u_off;      // [n_elem+1]
  const int64_t* lam_off;    // [n_face+1]
  const int64_t* x_off;      // [n_elem+1]
  const int64_t* kblk;       // [n_elem][9]: offset in K of block (face a, face b), a,b local
  const int64_t* dblk_off;   // [n_face]: offset of a face's diagonal block in the half-1 scratch
  const uint8_t* elem_bc;    // [n_elem] or null: bits 2l..2l+1 boundary kind of local face l
                             // (0 interior, 1 slip wall, 2 far field); elem_face is -1 there
  int far;                   // 1 if any face is a far-field boundary (kind 2)
};

// Per-system output and work buffers handed to kernels by value.
struct DevSys {
  double* X;
  double* K;
  double* E;
  double* res_u;
  double* res_lam;
  int32_t* status;
  // work space for the two-sided sums of diagonal blocks, E and res_lam:
  // the side-1 element parks its half here; whichever side arrives second sums.
  double* dhalf1;            // [sum_e (4(p_e+1))^2]
  double* ehalf1;            // [lam_len]
  double* rhalf1;            // [lam_len]
  int32_t* face_cnt;         // [n_face], zero between calls
  const double* ftilde;      // [u_len] adjoint right-hand side (adjoint mode only)
  const double* src;         // [u_len] source coefficients in U's layout (w part), or null
};

// One system of a batch (hdg_batch_*) as the element kernels read it: its mesh
// plan, output and work buffers, physical parameters and device inputs.
struct ReqDesc {
  DevMesh m;
  DevSys s;
  Phys ph;
  const double* U;
  const double* Lam;
  const double* dLam;  // reconstruction input and output (hdg_batch_recover)
  double* dU;
};
// A run of consecutive work items of one batched launch taken from one system:
// items [first, next segment's first) are the elements elems[0 ..] of descs[desc].
struct BatchSeg {
  int desc;
  int first;
  const int* elems;
};
// Work list of a batched launch (null descs: a plain single-system launch).
struct BatchRef {
  const ReqDesc* descs;
  const BatchSeg* segs;
  int n_segs;
};

#ifdef __CUDACC__
// The current work item's system in a batched launch, or the launch's own
// arguments in a plain one.
template <bool BATCH, class M>
__device__ __forceinline__ const M& pick_ref(const ReqDesc* d, M ReqDesc::*mp, const M& single) {
  if constexpr (BATCH) return d->*mp;
  else return single;
}
// Cursor over the segments of a batched launch: item `it` (non-decreasing per CTA)
// -> its element and system.
__device__ __forceinline__ int batch_item(const BatchRef& bt, int it, int& seg, const ReqDesc*& d) {
  while (seg + 1 < bt.n_segs && it >= bt.segs[seg + 1].first) ++seg;
  const BatchSeg sg = bt.segs[seg];
  d = bt.descs + sg.desc;
  return sg.elems[it - sg.first];
}
#endif

// Read-only view of a mesh plan and its context, for translation units other
// than the one that owns the opaque structs (hdg_api.cu).
struct PlanRef {
  int device;
  const double* tab;
  const void* tab_ff;
  const TabOff* off;
  const DevMesh* dm;
  const int* const* bucket;
  const int* bucket_n;
  const int* bucket_ntmax;
  const BucketNt* bucket_nt;
  int n_face, nfield;
  int64_t lam_len, dh_len;
  std::string* err;
};
PlanRef plan_ref(const hdg_mesh* mesh);

// kernel launchers (hdg_kernels.cu); return the number of launches enqueued
// bucket_streams (optional, indexed by degree p): stream of each degree bucket's launch
// resident CTAs per SM of the condensation kernel for degree p (model and precision from ph)
int condense_occupancy(const Phys& ph, int p, int ntmax);
int ns_occupancy(const Phys& ph, int p, int ntmax);

// bucket_nt (optional): trace-size counts of the buckets, whose element lists are sorted by trace
// size; a bucket is then launched in groups (launch_groups)
int launch_condense(const DevMesh& m, const DevSys& s, const Phys& ph, const double* tab, const void* tab_ff,
                    const TabOff& off, const double* U, const double* Lam, const int* const* bucket,
                    const int* bucket_n, const int* bucket_ntmax, void* stream, std::string* err,
                    void* const* bucket_streams = nullptr, const BucketNt* bucket_nt = nullptr);
int launch_condense_ns(const DevMesh& m, const DevSys& s, const Phys& ph, const double* tab, const void* tab_ff,
                       const TabOff& off, const double* U, const double* Lam, const int* const* bucket,
                       const int* bucket_n, const int* bucket_ntmax, void* stream, std::string* err,
                       void* const* bucket_streams = nullptr, const BucketNt* bucket_nt = nullptr);

// The launches of degree bucket p.  Shared memory is sized by the largest trace size
// of a launch, so one launch over a bucket whose trace sizes differ (faces of a
// mixed-degree mesh take the larger degree of their two sides) holds every element
// to the resident CTAs per SM of the largest.  With bucket_nt the bucket is cut into
// runs of trace sizes at which the kernel keeps the same number of resident CTAs
// per SM, one launch each, sized by the run's largest trace size.  launch(offset,
// count, ntmax) enqueues one launch over elements offset .. offset + count - 1 of
// the bucket's list.  Returns the launches enqueued, or -1.
template <class F>
inline int launch_groups(const Phys& ph, int p, int n, int ntmax, const BucketNt* bucket_nt, F&& launch) {
  const int* c = bucket_nt ? bucket_nt->cnt[p] : nullptr;
  int used = 0;
  for (int t = 0; c && t < kNtSlots; ++t) used += c[t] > 0;
  if (used <= 1) return launch(0, n, ntmax) ? 1 : -1;
  int occ[kNtSlots];
  for (int t = 0; t < kNtSlots; ++t) occ[t] = c[t] ? condense_occupancy(ph, p, 4 * t) : 0;
  int launches = 0, off = 0, t = 0;
  while (t < kNtSlots) {
    if (!c[t]) { ++t; continue; }
    int cnt = 0, top = 4 * t, e = t;
    for (; e < kNtSlots; ++e) {
      if (!c[e]) continue;
      if (occ[e] != occ[t]) break;
      cnt += c[e];
      top = 4 * e;
    }
    if (!launch(off, cnt, top)) return -1;
    ++launches;
    off += cnt;
    t = e;
  }
  return launches;
}
// batched launches (hdg_batch_*): one launch over the items of every system of
// the work list `bt` whose elements have degree p (model and precision from ph)
// mixed-precision local solves (precision HDG_MIXED_TF32 / HDG_MIXED_BF16, Euler)
bool launch_euler_mixed(int p, const DevMesh& m, const DevSys& s, const Phys& ph, const double* tab, const TabOff& to,
                        const double* U, const double* Lam, const int* elems, int n, int ntmax, void* stream,
                        std::string* err, const BatchRef& bt, bool bounded);
int euler_mixed_occupancy(const Phys& ph, int p, int ntmax, bool bounded);
bool launch_condense_batch(int p, const Phys& ph, const double* tab, const void* tab_ff, const TabOff& to,
                           const BatchRef& bt, int n_items, int ntmax, bool bounded, void* stream, std::string* err);
bool launch_ns_batch(int p, const Phys& ph, const double* tab, const void* tab_ff, const TabOff& to,
                     const BatchRef& bt, int n_items, int ntmax, void* stream, std::string* err);
bool launch_recover_batch(int p, int nfield, const BatchRef& bt, int n_items, void* stream, std::string* err);
int batch_occupancy(const Phys& ph, int p, int ntmax, bool bounded);

int launch_recover_buckets(const DevMesh& m, const double* X, const double* dLam, double* dU,
                           const int* const* bucket, const int* bucket_n, void* stream, std::string* err);

}  // namespace hdg
