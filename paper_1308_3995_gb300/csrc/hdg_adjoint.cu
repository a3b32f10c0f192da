// Hybridized adjoint (paper Sec. 4.2): the adjoint system is the transpose of
// the Newton matrix, [A B R; C D S; L M N]^T [Q~; W~; Lambda~] = [F~; G~; 0].
// Static condensation gives K^T Lambda~ = E~ with the primal K, and per element
//   E~_K = -B_K^T A_K^{-T} F~_K = -X_B,K^T F~_K      (X_B = A_K^{-1} B_K, the
//          primal local solves already stored by hdg_condense),
//   U~_K = A_K^{-T} (F~_K - C_K^T Lambda~_K) = X~_F - X~_C Lambda~_K,
// X~ = A_K^{-T} [C_K^T | F~_K] from the element kernel's adjoint mode.
// k_adjoint_rhs: one warp per face, one lane per trace unknown of the face,
// the two sides' contributions in side order (no atomics, reproducible).
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "hdg_internal.h"
#include "hdg_objects.h"

using namespace hdg;

namespace {

constexpr int kRhsWarps = 4;

struct AdjRhs {
  int n_face;
  const int* face_el;       // [n_face][2]
  const int* elem_face;     // [n_elem][3]
  const int* face_p;
  const int64_t* u_off;
  const int64_t* lam_off;
  const int64_t* x_off;
  const double* X;          // primal local solves (column-major n x (nt+1) per element)
  const double* ft;         // F~ [u_len]
  double* E;                // E~ [lam_len]
};

__global__ void __launch_bounds__(32 * kRhsWarps) k_adjoint_rhs(AdjRhs a) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * kRhsWarps + w;
  if (e >= a.n_face) return;
  const int m = 4 * (a.face_p[e] + 1);
  if (lane >= m) return;
  double tot = 0.0;
  for (int side = 0; side < 2; ++side) {
    const int K = a.face_el[2 * e + side];
    int toff = 0;  // offset of face e in K's trace unknowns
    for (int l = 0; l < 3; ++l) {
      const int f = a.elem_face[3 * K + l];
      if (f == e) break;
      if (f >= 0) toff += 4 * (a.face_p[f] + 1);  // boundary faces carry no trace unknowns
    }
    const int64_t n = a.u_off[K + 1] - a.u_off[K];
    const double* xc = a.X + a.x_off[K] + (int64_t)(toff + lane) * n;  // column toff + lane of X_B
    const double* ft = a.ft + a.u_off[K];
    double s = 0.0;
    for (int64_t r = 0; r < n; ++r) s = fma(xc[r], ft[r], s);
    tot += s;
  }
  a.E[a.lam_off[e] + lane] = -tot;
}

hdg_status fail(hdg_ctx* ctx, hdg_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

}  // namespace

extern "C" {

hdg_status hdg_adjoint_condense(hdg_sys* adj, const hdg_sys* primal, const double* U, const double* Lam,
                                const double* Ftilde, void* stream) {
  hdg::NvtxRange nvtx_range_("hdg::adjoint_condense");
  if (!adj || !primal) return HDG_EINVAL;
  hdg_ctx* ctx = adj->ctx;
  if (!U || !Lam || !Ftilde) return fail(ctx, HDG_EINVAL, "hdg_adjoint_condense: null input");
  HDG_ON_DEVICE(ctx, ctx->device);
  if (adj->ph.precision != HDG_FP64 && adj->ph.precision != HDG_FLOAT2)
    return fail(ctx, HDG_ENOTSUP, "hdg_adjoint_condense: the adjoint runs in binary64 or float-float");
  const hdg_mesh* M = adj->mesh;
  if (primal->mesh != M) return fail(ctx, HDG_EINVAL, "hdg_adjoint_condense: systems on different meshes");
  if (primal->ph.precision != adj->ph.precision || primal->ph.cfl != adj->ph.cfl ||
      primal->ph.sc_eps0 != adj->ph.sc_eps0)
    return fail(ctx, HDG_EINVAL, "hdg_adjoint_condense: primal and adjoint systems have different parameters");
  cudaStream_t st = (cudaStream_t)stream;
  if (!adj->d_face_el) {  // face -> (side 0, side 1) element, uploaded once
    std::vector<int> fe(2 * (size_t)M->n_face);
    for (int e = 0; e < M->n_face; ++e) {
      fe[2 * e] = M->face_el0[e];
      fe[2 * e + 1] = M->face_el1[e];
    }
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(int) * fe.size()) != cudaSuccess)
      return fail(ctx, HDG_ENOMEM, "hdg_adjoint_condense: cudaMalloc failed");
    adj->allocs.push_back(p);
    if (cudaMemcpy(p, fe.data(), sizeof(int) * fe.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(ctx, HDG_ECUDA, "hdg_adjoint_condense: cudaMemcpy failed");
    adj->d_face_el = (int*)p;
  }
  // adjoint local solves X~ = A^{-T} [C^T | F~] into adj's X
  Phys ph = adj->ph;
  ph.adjoint = 1;
  DevSys ds = adj->ds;
  ds.ftilde = Ftilde;
  std::string err;
  const int n = launch_condense(M->dm, ds, ph, ctx->d_tab, ctx->d_tab_ff, ctx->tab.off, U, Lam, M->d_bucket,
                                M->bucket_n, M->bucket_ntmax, stream, &err, nullptr, &M->bucket_nt);
  if (n < 0) return fail(ctx, HDG_ECUDA, "hdg_adjoint_condense: " + err);
  // E~ = -X_B^T F~ from the primal local solves
  AdjRhs a{M->n_face, adj->d_face_el, M->dm.elem_face, M->dm.face_p, M->dm.u_off, M->dm.lam_off, M->dm.x_off,
           primal->ds.X, Ftilde, adj->ds.E};
  k_adjoint_rhs<<<(M->n_face + kRhsWarps - 1) / kRhsWarps, 32 * kRhsWarps, 0, st>>>(a);
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return fail(ctx, HDG_ECUDA, std::string("k_adjoint_rhs: ") + cudaGetErrorString(ce));
  adj->launches = n + 1;
  return HDG_OK;
}

}  // extern "C"
