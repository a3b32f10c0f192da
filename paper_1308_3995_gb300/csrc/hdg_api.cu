// C ABI of the HDG hot path (declared in include/hdg.h): contexts, mesh
// planning (faces, sides, layouts, degree buckets), system allocation and the
// enqueue calls.  Host planning is O(n log n) in the element count and is
// done once per mesh; every per-step call only enqueues kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "hdg_internal.h"
#include "hdg_objects.h"

using namespace hdg;

namespace {

hdg_status fail(hdg_ctx* ctx, hdg_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

#define HDG_CK(ctx, call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return fail(ctx, HDG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <class T>
hdg_status upload(hdg_ctx* ctx, std::vector<void*>& allocs, const std::vector<T>& h, T** d) {
  void* p = nullptr;
  size_t bytes = std::max<size_t>(sizeof(T) * h.size(), 16);
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) return fail(ctx, HDG_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  allocs.push_back(p);
  if (!h.empty()) HDG_CK(ctx, cudaMemcpy(p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  *d = (T*)p;
  return HDG_OK;
}

hdg_status dalloc(hdg_ctx* ctx, std::vector<void*>& allocs, size_t bytes, void** d) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) return fail(ctx, HDG_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  allocs.push_back(p);
  *d = p;
  return HDG_OK;
}

void free_all(std::vector<void*>& allocs) {
  for (void* p : allocs) cudaFree(p);
  allocs.clear();
}

int face_len(const hdg_mesh* M, int e) { return e < 0 ? 0 : 4 * (M->face_p[e] + 1); }

int elem_nt(const hdg_mesh* M, int K) {
  int nt = 0;
  for (int a = 0; a < 3; ++a) nt += face_len(M, M->elem_face[3 * K + a]);
  return nt;
}

}  // namespace

namespace hdg {
PlanRef plan_ref(const hdg_mesh* M) {
  PlanRef r;
  r.device = M->ctx->device;
  r.tab = M->ctx->d_tab;
  r.tab_ff = M->ctx->d_tab_ff;
  r.off = &M->ctx->tab.off;
  r.dm = &M->dm;
  r.bucket = M->d_bucket;
  r.bucket_n = M->bucket_n;
  r.bucket_ntmax = M->bucket_ntmax;
  r.bucket_nt = &M->bucket_nt;
  r.n_face = M->n_face;
  r.nfield = M->nfield;
  r.lam_len = M->lam_len;
  r.dh_len = M->dh_len;
  r.err = &M->ctx->err;
  return r;
}
}  // namespace hdg

extern "C" {

hdg_status hdg_create(hdg_ctx** out, int device) {
  if (!out) return HDG_EINVAL;
  *out = nullptr;
  hdg_ctx* ctx = new hdg_ctx();
  ctx->device = device;
  hdg::DeviceGuard dg(device);
  if (!dg.ok()) { delete ctx; return HDG_ECUDA; }
  cudaError_t e;
  build_tables(ctx->tab);
  e = cudaMalloc(&ctx->d_tab, sizeof(double) * ctx->tab.data.size());
  if (e != cudaSuccess) { delete ctx; return HDG_ENOMEM; }
  e = cudaMemcpy(ctx->d_tab, ctx->tab.data.data(), sizeof(double) * ctx->tab.data.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { cudaFree(ctx->d_tab); delete ctx; return HDG_ECUDA; }
  std::vector<float> split(2 * ctx->tab.data.size());
  for (size_t i = 0; i < ctx->tab.data.size(); ++i) {
    const double d = ctx->tab.data[i];
    const float h = (float)d;
    split[2 * i] = h;
    split[2 * i + 1] = (float)(d - (double)h);
  }
  e = cudaMalloc(&ctx->d_tab_ff, sizeof(float) * split.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(ctx->d_tab_ff, split.data(), sizeof(float) * split.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { cudaFree(ctx->d_tab); cudaFree(ctx->d_tab_ff); delete ctx; return HDG_ECUDA; }
  *out = ctx;
  return HDG_OK;
}

hdg_status hdg_destroy(hdg_ctx* ctx) {
  if (!ctx) return HDG_EINVAL;
  hdg::DeviceGuard dg(ctx->device);
  cudaFree(ctx->d_tab);
  cudaFree(ctx->d_tab_ff);
  delete ctx;
  return HDG_OK;
}

const char* hdg_last_error(const hdg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

hdg_status hdg_mesh_create(hdg_ctx* ctx, int32_t n_elem, int32_t nfield, const double* elem_xy,
                           const int32_t* elem_vid, const int8_t* elem_p, hdg_mesh** out) {
  return hdg_mesh_create_bc(ctx, n_elem, nfield, elem_xy, elem_vid, elem_p, nullptr, out);
}

hdg_status hdg_mesh_create_bc(hdg_ctx* ctx, int32_t n_elem, int32_t nfield, const double* elem_xy,
                              const int32_t* elem_vid, const int8_t* elem_p, const int8_t* elem_bc,
                              hdg_mesh** out) {
  if (!ctx || !out) return HDG_EINVAL;
  *out = nullptr;
  if (n_elem < 1 || (nfield != 4 && nfield != 12) || !elem_xy || !elem_vid || !elem_p)
    return fail(ctx, HDG_EINVAL, "hdg_mesh_create: bad arguments");
  bool any_bc = false;
  for (int t = 0; elem_bc && t < 3 * n_elem; ++t) {
    const int b = elem_bc[t];
    if (b < 0 || b > 3) return fail(ctx, HDG_EINVAL, "hdg_mesh_create_bc: boundary kind not in 0..3");
    if (b == 3 && nfield == 4)
      return fail(ctx, HDG_EINVAL, "hdg_mesh_create_bc: the no-slip wall (kind 3) is a Navier-Stokes boundary");
    if (b == 1 && nfield == 12)
      return fail(ctx, HDG_ENOTSUP,
                  "hdg_mesh_create_bc: Navier-Stokes boundaries are no-slip adiabatic walls (kind 3) or far field (kind 2)");
    any_bc |= b != 0;
  }
  HDG_ON_DEVICE(ctx, ctx->device);
  hdg_mesh* M = new hdg_mesh();
  M->ctx = ctx;
  M->n_elem = n_elem;
  M->nfield = nfield;
  M->has_bc = any_bc;
  std::vector<double> xy(elem_xy, elem_xy + 6 * (size_t)n_elem);
  for (int K = 0; K < n_elem; ++K) {
    const double* c = &xy[6 * (size_t)K];
    const double det = (c[2] - c[0]) * (c[5] - c[1]) - (c[4] - c[0]) * (c[3] - c[1]);
    if (elem_p[K] < 1 || elem_p[K] > kMaxP || !(det > 0.0)) {
      delete M;
      return fail(ctx, HDG_EINVAL, "hdg_mesh_create: element " + std::to_string(K) +
                                       " has p outside 1..4 or a non-positive Jacobian");
    }
  }
  // faces: unordered vertex pairs, numbered by ascending (lo, hi); side 0 = lower element id
  struct Ent { int lo, hi, K, l; };
  std::vector<Ent> ents;
  ents.reserve(3 * (size_t)n_elem);
  for (int K = 0; K < n_elem; ++K)
    for (int l = 0; l < 3; ++l) {
      if (any_bc && elem_bc[3 * K + l]) continue;  // boundary face: no partner, no trace unknowns
      const int a = elem_vid[3 * K + l], b = elem_vid[3 * K + (l + 1) % 3];
      ents.push_back({std::min(a, b), std::max(a, b), K, l});
    }
  std::sort(ents.begin(), ents.end(), [](const Ent& x, const Ent& y) {
    return x.lo != y.lo ? x.lo < y.lo : (x.hi != y.hi ? x.hi < y.hi : x.K < y.K);
  });
  M->elem_face.assign(3 * (size_t)n_elem, -1);
  std::vector<uint8_t> info(n_elem, 0);
  for (size_t i = 0; i < ents.size(); i += 2) {
    const bool ok = i + 1 < ents.size() && ents[i + 1].lo == ents[i].lo && ents[i + 1].hi == ents[i].hi &&
                    ents[i + 1].K != ents[i].K &&
                    !(i + 2 < ents.size() && ents[i + 2].lo == ents[i].lo && ents[i + 2].hi == ents[i].hi);
    if (!ok) {
      delete M;
      return fail(ctx, HDG_EINVAL, "hdg_mesh_create: an untagged face is not shared by exactly two elements");
    }
    const int f = M->n_face++;
    M->face_lo.push_back(ents[i].lo);
    M->face_hi.push_back(ents[i].hi);
    M->face_el0.push_back(ents[i].K);
    M->face_el1.push_back(ents[i + 1].K);
    M->face_p.push_back(std::max<int>(elem_p[ents[i].K], elem_p[ents[i + 1].K]));
    M->elem_face[3 * (size_t)ents[i].K + ents[i].l] = f;
    M->elem_face[3 * (size_t)ents[i + 1].K + ents[i + 1].l] = f;
    info[ents[i + 1].K] |= (uint8_t)(1u << (3 + ents[i + 1].l));
  }
  for (int K = 0; K < n_elem; ++K)
    for (int l = 0; l < 3; ++l)
      if (elem_vid[3 * K + l] > elem_vid[3 * K + (l + 1) % 3]) info[K] |= (uint8_t)(1u << l);
  // layouts
  M->u_off.assign(n_elem + 1, 0);
  M->x_off.assign(n_elem + 1, 0);
  for (int K = 0; K < n_elem; ++K) {
    const int n = nfield * n_basis(elem_p[K]), nt = elem_nt(M, K);
    M->u_off[K + 1] = M->u_off[K] + n;
    M->x_off[K + 1] = M->x_off[K] + (int64_t)n * (nt + 1);
    M->max_nt = std::max(M->max_nt, nt);
  }
  M->u_len = M->u_off[n_elem];
  M->x_len = M->x_off[n_elem];
  M->lam_off.assign(M->n_face + 1, 0);
  std::vector<int64_t> dblk(M->n_face, 0);
  for (int f = 0; f < M->n_face; ++f) {
    const int m4 = 4 * (M->face_p[f] + 1);
    M->lam_off[f + 1] = M->lam_off[f] + m4;
    dblk[f] = M->dh_len;
    M->dh_len += (int64_t)m4 * m4;
  }
  M->lam_len = M->lam_off[M->n_face];
  M->k_col.assign(5 * (size_t)M->n_face, 0);
  M->k_blkoff.assign(5 * (size_t)M->n_face + 1, 0);
  for (int f = 0; f < M->n_face; ++f) {
    int cols[5], nc = 0;
    cols[nc++] = f;
    for (int sd = 0; sd < 2; ++sd) {
      const int K = sd ? M->face_el1[f] : M->face_el0[f];
      for (int l = 0; l < 3; ++l) {
        const int e = M->elem_face[3 * (size_t)K + l];
        if (e != f && e >= 0) cols[nc++] = e;
      }
    }
    std::sort(cols, cols + nc);
    for (int b = 1; b < nc; ++b)
      if (cols[b] == cols[b - 1]) {
        delete M;
        return fail(ctx, HDG_EINVAL, "hdg_mesh_create: two elements share two faces");
      }
    for (int b = nc; b < 5; ++b) cols[b] = -1;  // unused slots next to boundary faces: empty blocks
    for (int b = 0; b < 5; ++b) {
      M->k_col[5 * (size_t)f + b] = cols[b];
      M->k_blkoff[5 * (size_t)f + b + 1] =
          M->k_blkoff[5 * (size_t)f + b] + (int64_t)(4 * (M->face_p[f] + 1)) * face_len(M, cols[b]);
    }
  }
  M->k_len = M->k_blkoff[5 * (size_t)M->n_face];
  std::vector<int64_t> kblk(9 * (size_t)n_elem);
  for (int K = 0; K < n_elem; ++K)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const int ea = M->elem_face[3 * (size_t)K + a], eb = M->elem_face[3 * (size_t)K + b];
        if (ea < 0 || eb < 0) {  // a boundary face: no block
          kblk[9 * (size_t)K + 3 * a + b] = -1;
          continue;
        }
        int slot = 0;
        while (M->k_col[5 * (size_t)ea + slot] != eb) ++slot;
        kblk[9 * (size_t)K + 3 * a + b] = M->k_blkoff[5 * (size_t)ea + slot];
      }
  // degree buckets, each sorted by trace size (launch_groups)
  std::vector<int> bucket[kMaxP + 1];
  std::vector<int> nt_of(n_elem);
  for (int K = 0; K < n_elem; ++K) {
    nt_of[K] = elem_nt(M, K);
    bucket[elem_p[K]].push_back(K);
    M->bucket_ntmax[elem_p[K]] = std::max(M->bucket_ntmax[elem_p[K]], nt_of[K]);
    ++M->bucket_nt.cnt[elem_p[K]][nt_of[K] / 4];
  }
  for (int p = 1; p <= kMaxP; ++p)
    std::stable_sort(bucket[p].begin(), bucket[p].end(), [&](int a, int b) { return nt_of[a] < nt_of[b]; });
  // upload
  hdg_status st = HDG_OK;
  DevMesh& d = M->dm;
  d.n_elem = n_elem;
  d.n_face = M->n_face;
  d.nfield = nfield;
  double* dxy;
  int *def, *dfp;
  uint8_t* dinfo;
  uint8_t* dbc = nullptr;
  std::vector<uint8_t> bcbits;
  if (any_bc) {
    bcbits.assign(n_elem, 0);
    for (int K = 0; K < n_elem; ++K)
      for (int l = 0; l < 3; ++l) bcbits[K] |= (uint8_t)((elem_bc[3 * K + l] & 3) << (2 * l));
  }
  int64_t *duo, *dlo, *dxo, *dkb, *ddb;
  if ((st = upload(ctx, M->allocs, xy, &dxy)) || (st = upload(ctx, M->allocs, M->elem_face, &def)) ||
      (st = upload(ctx, M->allocs, info, &dinfo)) || (st = upload(ctx, M->allocs, M->face_p, &dfp)) ||
      (st = upload(ctx, M->allocs, M->u_off, &duo)) || (st = upload(ctx, M->allocs, M->lam_off, &dlo)) ||
      (st = upload(ctx, M->allocs, M->x_off, &dxo)) || (st = upload(ctx, M->allocs, kblk, &dkb)) ||
      (st = upload(ctx, M->allocs, dblk, &ddb)) || (any_bc && (st = upload(ctx, M->allocs, bcbits, &dbc)))) {
    free_all(M->allocs);
    delete M;
    return st;
  }
  d.xy = dxy; d.elem_face = def; d.elem_info = dinfo; d.face_p = dfp;
  d.u_off = duo; d.lam_off = dlo; d.x_off = dxo; d.kblk = dkb; d.dblk_off = ddb;
  d.elem_bc = dbc;
  d.far = 0;
  for (int t = 0; elem_bc && t < 3 * n_elem; ++t) d.far |= elem_bc[t] == 2;
  for (int p = 1; p <= kMaxP; ++p) {
    M->bucket_n[p] = (int)bucket[p].size();
    if (M->bucket_n[p] && (st = upload(ctx, M->allocs, bucket[p], &M->d_bucket[p]))) {
      free_all(M->allocs);
      delete M;
      return st;
    }
  }
  *out = M;
  return HDG_OK;
}

hdg_status hdg_mesh_destroy(hdg_mesh* M) {
  if (!M) return HDG_EINVAL;
  hdg::DeviceGuard dg(M->ctx->device);
  free_all(M->allocs);
  delete M;
  return HDG_OK;
}

hdg_status hdg_mesh_sizes(const hdg_mesh* M, int64_t* s) {
  if (!M || !s) return HDG_EINVAL;
  s[0] = M->n_elem; s[1] = M->n_face; s[2] = M->u_len; s[3] = M->lam_len;
  s[4] = M->x_len; s[5] = M->k_len; s[6] = M->max_nt;
  return HDG_OK;
}

hdg_status hdg_mesh_layout(const hdg_mesh* M, int32_t* face_vid, int32_t* face_el, int32_t* face_p,
                           int32_t* elem_face, int64_t* u_off, int64_t* lam_off, int64_t* x_off, int32_t* k_col,
                           int64_t* k_blkoff) {
  if (!M) return HDG_EINVAL;
  for (int f = 0; f < M->n_face; ++f) {
    if (face_vid) { face_vid[2 * f] = M->face_lo[f]; face_vid[2 * f + 1] = M->face_hi[f]; }
    if (face_el) { face_el[2 * f] = M->face_el0[f]; face_el[2 * f + 1] = M->face_el1[f]; }
    if (face_p) face_p[f] = M->face_p[f];
  }
  if (elem_face) std::copy(M->elem_face.begin(), M->elem_face.end(), elem_face);
  if (u_off) std::copy(M->u_off.begin(), M->u_off.end(), u_off);
  if (lam_off) std::copy(M->lam_off.begin(), M->lam_off.end(), lam_off);
  if (x_off) std::copy(M->x_off.begin(), M->x_off.end(), x_off);
  if (k_col) std::copy(M->k_col.begin(), M->k_col.end(), k_col);
  if (k_blkoff) std::copy(M->k_blkoff.begin(), M->k_blkoff.end(), k_blkoff);
  return HDG_OK;
}

int64_t hdg_footprint_bytes(const hdg_mesh* M, const hdg_params* P) { return hdg_sys_workspace_bytes(M, P); }

}  // extern "C"

namespace {

constexpr int kSysBufs = 14;  // X, K, E, res_u, res_lam, status, dhalf1, ehalf1, rhalf1, face_cnt, U, Lam, dLam, dU

void sys_sizes(const hdg_mesh* M, size_t* sz) {
  const size_t d = sizeof(double);
  const size_t v[kSysBufs] = {d * M->x_len,   d * M->k_len,   d * M->lam_len, d * M->u_len,   d * M->lam_len,
                              4 * (size_t)M->n_elem, d * M->dh_len, d * M->lam_len, d * M->lam_len,
                              4 * (size_t)M->n_face, d * M->u_len,  d * M->lam_len, d * M->lam_len, d * M->u_len};
  for (int i = 0; i < kSysBufs; ++i) sz[i] = v[i];
}
inline size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

hdg_status sys_validate(hdg_ctx* ctx, const hdg_mesh* M, const hdg_params* P, const char* who) {
  if (M->has_bc && !std::isfinite(P->aoa))
    return fail(ctx, HDG_EINVAL, std::string(who) + ": boundary faces need a finite aoa");
  const std::string w(who);
  if ((P->model == HDG_EULER) != (M->nfield == 4) || (P->model != HDG_EULER && P->model != HDG_NS_MIXED))
    return fail(ctx, HDG_EINVAL, w + ": model does not match the mesh's field count");
  if (P->precision != HDG_FP64 && P->precision != HDG_FLOAT2 && P->precision != HDG_MIXED_TF32 &&
      P->precision != HDG_MIXED_BF16)
    return fail(ctx, HDG_ENOTSUP, w + ": precision not supported by this library");
  if ((P->precision == HDG_MIXED_TF32 || P->precision == HDG_MIXED_BF16) && P->model != HDG_EULER)
    return fail(ctx, HDG_ENOTSUP, w + ": the tensor-core local solves are built for the Euler kernel only");
  if ((P->precision == HDG_MIXED_TF32 || P->precision == HDG_MIXED_BF16) &&
      (P->refine_max < 0 || P->refine_max > 64 || !(P->refine_tol >= 0.0)))
    return fail(ctx, HDG_EINVAL, w + ": refine_max must be in 0..64 and refine_tol >= 0");
  if (P->model == HDG_NS_MIXED && !(P->reynolds > 0.0 && P->prandtl > 0.0 && P->t_inf > 0.0))
    return fail(ctx, HDG_EINVAL, w + ": Navier-Stokes needs reynolds, prandtl, t_inf > 0");
  if (!(P->gamma > 1.0) || !(P->alpha > 0.0) || !(P->mach > 0.0))
    return fail(ctx, HDG_EINVAL, w + ": need gamma > 1, alpha > 0, mach > 0");
  if (P->sc_eps0 > 0.0 && !(std::isfinite(P->sc_eps0) && std::isfinite(P->sc_beta)))
    return fail(ctx, HDG_EINVAL, w + ": shock capturing needs finite sc_eps0 and sc_beta");
  return HDG_OK;
}

hdg_sys* sys_new(hdg_ctx* ctx, const hdg_mesh* M, const hdg_params* P) {
  hdg_sys* S = new hdg_sys();
  S->ctx = ctx;
  S->mesh = M;
  S->prm = *P;
  S->ph.gamma = P->gamma;
  S->ph.alpha = P->alpha;
  S->ph.prandtl = P->prandtl;
  S->ph.mu_inf = P->mach / P->reynolds;
  S->ph.suth_s = 110.4 / P->t_inf;
  S->ph.cfl = P->cfl;
  S->ph.sc_eps0 = P->sc_eps0 > 0.0 ? P->sc_eps0 : 0.0;
  S->ph.sc_beta = P->sc_beta;
  far_field_state(*P, S->ph.winf);
  S->ph.model = P->model;
  S->ph.precision = P->precision;
  S->ph.refine_max = P->refine_max;
  S->ph.refine_tol = P->refine_tol;
  S->ph.persistent = 1;
  phys_default_grid(S->ph);
  return S;
}

int n_buckets(const hdg_mesh* M) {
  int nb = 0;
  for (int p = 1; p <= kMaxP; ++p) nb += M->bucket_n[p] > 0;
  return nb;
}

hdg_status ensure_streams(hdg_sys* S) {
  if (S->have_streams) return HDG_OK;
  for (int p = 1; p <= kMaxP; ++p) {
    HDG_CK(S->ctx, cudaStreamCreateWithFlags(&S->bstream[p], cudaStreamNonBlocking));
    HDG_CK(S->ctx, cudaEventCreateWithFlags(&S->bevent[p], cudaEventDisableTiming));
    HDG_CK(S->ctx, cudaEventCreate(&S->tbeg[p]));
    HDG_CK(S->ctx, cudaEventCreate(&S->tend[p]));
  }
  HDG_CK(S->ctx, cudaEventCreateWithFlags(&S->fork, cudaEventDisableTiming));
  S->have_streams = true;
  return HDG_OK;
}

void sys_bind(hdg_sys* S, void* const* p) {
  S->ds.X = (double*)p[0];
  S->ds.K = (double*)p[1];
  S->ds.E = (double*)p[2];
  S->ds.res_u = (double*)p[3];
  S->ds.res_lam = (double*)p[4];
  S->ds.status = (int32_t*)p[5];
  S->ds.dhalf1 = (double*)p[6];
  S->ds.ehalf1 = (double*)p[7];
  S->ds.rhalf1 = (double*)p[8];
  S->ds.face_cnt = (int32_t*)p[9];
  S->d_U = (double*)p[10];
  S->d_Lam = (double*)p[11];
  S->d_dLam = (double*)p[12];
  S->d_dU = (double*)p[13];
  S->need_zero = true;  // arrival counters are cleared on the stream of the first condensation
}

}  // namespace

extern "C" {

int64_t hdg_sys_workspace_bytes(const hdg_mesh* M, const hdg_params* P) {
  if (!M || !P) return -1;
  size_t sz[kSysBufs], tot = 0;
  sys_sizes(M, sz);
  for (int i = 0; i < kSysBufs; ++i) tot += round256(sz[i]);
  return (int64_t)tot;
}

hdg_status hdg_sys_create(hdg_ctx* ctx, const hdg_mesh* M, const hdg_params* P, hdg_sys** out) {
  if (!ctx || !M || !P || !out) return HDG_EINVAL;
  *out = nullptr;
  HDG_ON_DEVICE(ctx, ctx->device);
  hdg_status st = sys_validate(ctx, M, P, "hdg_sys_create");
  if (st != HDG_OK) return st;
  hdg_sys* S = sys_new(ctx, M, P);
  size_t sz[kSysBufs];
  sys_sizes(M, sz);
  void* p[kSysBufs];
  for (int i = 0; i < kSysBufs; ++i)
    if ((st = dalloc(ctx, S->allocs, sz[i], &p[i]))) { free_all(S->allocs); delete S; return st; }
  sys_bind(S, p);
  *out = S;
  return HDG_OK;
}

hdg_status hdg_sys_create_in(hdg_ctx* ctx, const hdg_mesh* M, const hdg_params* P, void* workspace,
                             int64_t workspace_bytes, hdg_sys** out) {
  if (!ctx || !M || !P || !out) return HDG_EINVAL;
  *out = nullptr;
  HDG_ON_DEVICE(ctx, ctx->device);
  hdg_status st = sys_validate(ctx, M, P, "hdg_sys_create_in");
  if (st != HDG_OK) return st;
  const int64_t need = hdg_sys_workspace_bytes(M, P);
  if (!workspace || ((uintptr_t)workspace & 255u) != 0 || workspace_bytes < need)
    return fail(ctx, HDG_EINVAL, "hdg_sys_create_in: workspace must be 256-byte aligned and hold " +
                                     std::to_string(need) + " bytes");
  hdg_sys* S = sys_new(ctx, M, P);
  size_t sz[kSysBufs];
  sys_sizes(M, sz);
  void* p[kSysBufs];
  unsigned char* w = (unsigned char*)workspace;
  for (int i = 0; i < kSysBufs; ++i) {
    p[i] = w;
    w += round256(sz[i]);
  }
  sys_bind(S, p);
  *out = S;
  return HDG_OK;
}

hdg_status hdg_sys_destroy(hdg_sys* S) {
  if (!S) return HDG_EINVAL;
  hdg::DeviceGuard dg(S->ctx->device);
  if (S->gexec) cudaGraphExecDestroy(S->gexec);
  if (S->graph) cudaGraphDestroy(S->graph);
  if (S->have_streams) {
    for (int p = 1; p <= kMaxP; ++p) {
      cudaStreamDestroy(S->bstream[p]);
      cudaEventDestroy(S->bevent[p]);
      cudaEventDestroy(S->tbeg[p]);
      cudaEventDestroy(S->tend[p]);
    }
    cudaEventDestroy(S->fork);
  }
  free_all(S->allocs);
  delete S;
  return HDG_OK;
}

hdg_status hdg_condense(hdg_sys* S, const double* U, const double* Lam, void* stream) {
  hdg::NvtxRange nvtx_range_("hdg::condense");
  if (!S) return HDG_EINVAL;
  hdg_ctx* ctx = S->ctx;
  if (!U || !Lam) return fail(ctx, HDG_EINVAL, "hdg_condense: null input");
  HDG_ON_DEVICE(ctx, ctx->device);
  const hdg_mesh* M = S->mesh;
  cudaStream_t st = (cudaStream_t)stream;
  if (S->need_zero) {
    HDG_CK(ctx, cudaMemsetAsync(S->ds.face_cnt, 0, 4 * (size_t)M->n_face, st));
    S->need_zero = false;
  }
  std::string err;
  int n;
  if (n_buckets(M) > 1) {
    // degree buckets run concurrently: fork onto one stream per degree, join back;
    // one CTA per element so the CTAs of the buckets interleave on the SMs
    hdg_status rs = ensure_streams(S);
    if (rs != HDG_OK) return rs;
    HDG_CK(ctx, cudaEventRecord(S->fork, st));
    // per-bucket timing events, except inside a graph capture
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    HDG_CK(ctx, cudaStreamIsCapturing(st, &cap));
    S->timed = cap == cudaStreamCaptureStatusNone;
    void* bs[kMaxP + 1] = {};
    for (int p = 1; p <= kMaxP; ++p) {
      bs[p] = S->bstream[p];
      if (M->bucket_n[p]) {
        HDG_CK(ctx, cudaStreamWaitEvent(S->bstream[p], S->fork, 0));
        if (S->timed) HDG_CK(ctx, cudaEventRecord(S->tbeg[p], S->bstream[p]));
      }
    }
    Phys ph = S->ph;
    ph.persistent = 0;
    n = launch_condense(M->dm, S->ds, ph, ctx->d_tab, ctx->d_tab_ff, ctx->tab.off, U, Lam, M->d_bucket, M->bucket_n,
                        M->bucket_ntmax, stream, &err, bs, &M->bucket_nt);
    if (n >= 0)
      for (int p = 1; p <= kMaxP; ++p)
        if (M->bucket_n[p]) {
          if (S->timed) HDG_CK(ctx, cudaEventRecord(S->tend[p], S->bstream[p]));
          HDG_CK(ctx, cudaEventRecord(S->bevent[p], S->bstream[p]));
          HDG_CK(ctx, cudaStreamWaitEvent(st, S->bevent[p], 0));
        }
  } else {
    S->timed = false;
    n = launch_condense(M->dm, S->ds, S->ph, ctx->d_tab, ctx->d_tab_ff, ctx->tab.off, U, Lam, M->d_bucket,
                        M->bucket_n, M->bucket_ntmax, stream, &err, nullptr, &M->bucket_nt);
  }
  if (n < 0) return fail(ctx, HDG_ECUDA, "hdg_condense: " + err);
  S->launches = n;
  return HDG_OK;
}

hdg_status hdg_sys_bucket_times(const hdg_sys* S, float* ms) {
  if (!S || !ms) return HDG_EINVAL;
  for (int p = 0; p <= kMaxP; ++p) ms[p] = -1.0f;
  if (!S->timed) return HDG_OK;
  HDG_ON_DEVICE(S->ctx, S->ctx->device);
  const hdg_mesh* M = S->mesh;
  for (int p = 1; p <= kMaxP; ++p) {
    if (!M->bucket_n[p]) continue;
    if (cudaEventSynchronize(S->tend[p]) != cudaSuccess ||
        cudaEventElapsedTime(&ms[p], S->tbeg[p], S->tend[p]) != cudaSuccess)
      return fail(S->ctx, HDG_ECUDA, "hdg_sys_bucket_times: event query failed");
  }
  return HDG_OK;
}

hdg_status hdg_recover(hdg_sys* S, const double* dLam, double* dU, void* stream) {
  hdg::NvtxRange nvtx_range_("hdg::recover");
  if (!S) return HDG_EINVAL;
  hdg_ctx* ctx = S->ctx;
  if (!dLam || !dU) return fail(ctx, HDG_EINVAL, "hdg_recover: null argument");
  HDG_ON_DEVICE(ctx, ctx->device);
  const hdg_mesh* M = S->mesh;
  std::string err;
  const int n = launch_recover_buckets(M->dm, S->ds.X, dLam, dU, M->d_bucket, M->bucket_n, stream, &err);
  if (n < 0) return fail(ctx, HDG_ECUDA, "hdg_recover: " + err);
  S->launches += n;
  return HDG_OK;
}

hdg_status hdg_step_host_async(hdg_sys* S, const double* U, const double* Lam, const double* dLam, double* dU,
                               void* stream) {
  hdg::NvtxRange nvtx_range_("hdg::step_host");
  if (!S) return HDG_EINVAL;
  hdg_ctx* ctx = S->ctx;
  if (!U || !Lam || !dLam || !dU) return fail(ctx, HDG_EINVAL, "hdg_step_host_async: null argument");
  HDG_ON_DEVICE(ctx, ctx->device);
  const hdg_mesh* M = S->mesh;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t d = sizeof(double);
  HDG_CK(ctx, cudaMemcpyAsync(S->d_U, U, d * M->u_len, cudaMemcpyHostToDevice, st));
  HDG_CK(ctx, cudaMemcpyAsync(S->d_Lam, Lam, d * M->lam_len, cudaMemcpyHostToDevice, st));
  HDG_CK(ctx, cudaMemcpyAsync(S->d_dLam, dLam, d * M->lam_len, cudaMemcpyHostToDevice, st));
  hdg_status rc = hdg_condense(S, S->d_U, S->d_Lam, stream);
  if (rc != HDG_OK) return rc;
  rc = hdg_recover(S, S->d_dLam, S->d_dU, stream);
  if (rc != HDG_OK) return rc;
  HDG_CK(ctx, cudaMemcpyAsync(dU, S->d_dU, d * M->u_len, cudaMemcpyDeviceToHost, st));
  return HDG_OK;
}

hdg_status hdg_step_host(hdg_sys* S, const double* U, const double* Lam, const double* dLam, double* dU,
                         void* stream) {
  if (!S) return HDG_EINVAL;
  HDG_ON_DEVICE(S->ctx, S->ctx->device);
  const hdg_status rc = hdg_step_host_async(S, U, Lam, dLam, dU, stream);
  if (rc != HDG_OK) return rc;
  HDG_CK(S->ctx, cudaStreamSynchronize((cudaStream_t)stream));
  return HDG_OK;
}

hdg_status hdg_autotune(hdg_sys* S, const double* U, const double* Lam, int32_t* grid_out, void* stream) {
  hdg::NvtxRange nvtx_range_("hdg::autotune");
  if (!S) return HDG_EINVAL;
  hdg_ctx* ctx = S->ctx;
  if (!U || !Lam) return fail(ctx, HDG_EINVAL, "hdg_autotune: null input");
  HDG_ON_DEVICE(ctx, ctx->device);
  if (S->gexec) return fail(ctx, HDG_EINVAL, "hdg_autotune: a captured graph holds the launch shapes");
  const hdg_mesh* M = S->mesh;
  cudaStream_t st = (cudaStream_t)stream;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  cudaEvent_t e0, e1;
  HDG_CK(ctx, cudaEventCreate(&e0));
  HDG_CK(ctx, cudaEventCreate(&e1));
  std::string err;
  hdg_status rs = HDG_OK;
  for (int p = 1; p <= kMaxP && rs == HDG_OK; ++p) {
    if (grid_out) grid_out[p] = S->ph.grid[p];
    if (M->bucket_n[p] == 0) continue;
    if (condense_occupancy(S->ph, p, M->bucket_ntmax[p]) < 1) {
      rs = fail(ctx, HDG_ECUDA, "hdg_autotune: kernel does not fit on an SM");
      break;
    }
    // persistent candidates up to the occupancy at the bucket's smallest trace size (its
    // launch groups with smaller traces may hold more CTAs per SM than the largest)
    int ntmin = M->bucket_ntmax[p];
    for (int t = 0; t < kNtSlots; ++t)
      if (M->bucket_nt.cnt[p][t]) { ntmin = 4 * t; break; }
    const int occ = condense_occupancy(S->ph, p, ntmin);
    int bn[kMaxP + 1] = {};
    bn[p] = M->bucket_n[p];
    float best_ms = 0.0f;
    int best = -1;
    // candidates: one CTA per element, or a persistent grid of k CTAs per SM, k = 1..occupancy
    for (int cand = 0; cand <= occ && rs == HDG_OK; ++cand) {
      Phys ph = S->ph;
      ph.grid[p] = cand;
      float t_min = 0.0f;
      for (int rep = 0; rep < 4; ++rep) {
        if (cudaMemsetAsync(S->ds.face_cnt, 0, 4 * (size_t)M->n_face, st) != cudaSuccess ||
            cudaEventRecord(e0, st) != cudaSuccess) {
          rs = fail(ctx, HDG_ECUDA, "hdg_autotune: enqueue failed");
          break;
        }
        if (launch_condense(M->dm, S->ds, ph, ctx->d_tab, ctx->d_tab_ff, ctx->tab.off, U, Lam, M->d_bucket, bn,
                            M->bucket_ntmax, stream, &err, nullptr, &M->bucket_nt) < 0) {
          rs = fail(ctx, HDG_ECUDA, "hdg_autotune: " + err);
          break;
        }
        float ms = 0.0f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          rs = fail(ctx, HDG_ECUDA, "hdg_autotune: timing failed");
          break;
        }
        if (rep > 0 && (rep == 1 || ms < t_min)) t_min = ms;  // first launch is a warm-up
      }
      if (rs == HDG_OK && (best < 0 || t_min < best_ms)) { best = cand; best_ms = t_min; }
    }
    if (rs == HDG_OK) {
      S->ph.grid[p] = best;
      if (grid_out) grid_out[p] = best;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  S->need_zero = true;  // the single-bucket launches leave shared faces half counted
  return rs;
}

hdg_status hdg_graph_create(hdg_sys* S, const double* U, const double* Lam, const double* dLam, double* dU) {
  if (!S) return HDG_EINVAL;
  hdg_ctx* ctx = S->ctx;
  if (!U || !Lam || !dLam || !dU) return fail(ctx, HDG_EINVAL, "hdg_graph_create: null argument");
  HDG_ON_DEVICE(ctx, ctx->device);
  const hdg_mesh* M = S->mesh;
  if (S->gexec) { cudaGraphExecDestroy(S->gexec); S->gexec = nullptr; }
  if (S->graph) { cudaGraphDestroy(S->graph); S->graph = nullptr; }
  cudaStream_t cs;
  HDG_CK(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  // one plain step first: kernel attributes are set outside the capture
  hdg_status rc = hdg_condense(S, U, Lam, cs);
  if (rc == HDG_OK) rc = hdg_recover(S, dLam, dU, cs);
  cudaError_t e = cudaStreamSynchronize(cs);
  if (rc == HDG_OK && e != cudaSuccess) rc = fail(ctx, HDG_ECUDA, std::string("hdg_graph_create: ") + cudaGetErrorString(e));
  if (rc == HDG_OK) {
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->ds.face_cnt, 0, 4 * (size_t)M->n_face, cs);
    if (e == cudaSuccess) {
      rc = hdg_condense(S, U, Lam, cs);
      if (rc == HDG_OK) rc = hdg_recover(S, dLam, dU, cs);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && rc == HDG_OK) e = cudaGraphInstantiate(&S->gexec, g, 0);
    S->graph = g;
    if (rc == HDG_OK && e != cudaSuccess)
      rc = fail(ctx, HDG_ECUDA, std::string("hdg_graph_create: ") + cudaGetErrorString(e));
  }
  cudaStreamDestroy(cs);
  return rc;
}

hdg_status hdg_graph_launch(hdg_sys* S, void* stream) {
  if (!S) return HDG_EINVAL;
  if (!S->gexec) return fail(S->ctx, HDG_EINVAL, "hdg_graph_launch: no graph (call hdg_graph_create)");
  HDG_ON_DEVICE(S->ctx, S->ctx->device);
  HDG_CK(S->ctx, cudaGraphLaunch(S->gexec, (cudaStream_t)stream));
  return HDG_OK;
}

hdg_status hdg_sys_get(const hdg_sys* S, double** X, double** K_vals, double** E, double** res_u, double** res_lam,
                       int32_t** elem_status) {
  if (!S) return HDG_EINVAL;
  if (X) *X = S->ds.X;
  if (K_vals) *K_vals = S->ds.K;
  if (E) *E = S->ds.E;
  if (res_u) *res_u = S->ds.res_u;
  if (res_lam) *res_lam = S->ds.res_lam;
  if (elem_status) *elem_status = S->ds.status;
  return HDG_OK;
}

int32_t hdg_sys_launches(const hdg_sys* S) { return S ? S->launches : -1; }

hdg_status hdg_sys_io(const hdg_sys* S, double** U, double** Lam, double** dLam, double** dU) {
  if (!S) return HDG_EINVAL;
  if (U) *U = S->d_U;
  if (Lam) *Lam = S->d_Lam;
  if (dLam) *dLam = S->d_dLam;
  if (dU) *dU = S->d_dU;
  return HDG_OK;
}

}  // extern "C"
