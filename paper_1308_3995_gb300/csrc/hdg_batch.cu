// Batched condensation across systems (hdg_batch_*): the elements of several
// systems -- different meshes, degree maps, flow parameters, Euler or
// Navier-Stokes -- are condensed by one launch per (model, degree) group (one
// per run of trace sizes with equal occupancy, where they differ) over a work
// list of (system, element) segments, instead of one launch per system and
// degree.  Each element's arithmetic is that of hdg_condense (the same
// kernel source, instantiated for the work list), so every system's results
// are those of condensing it alone up to the compiler's contraction of
// multiply-adds.  The step of a batch can be captured into one CUDA graph and
// replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "hdg_internal.h"
#include "hdg_objects.h"

using namespace hdg;

namespace {

// one launch of a group: its segments are d_seg[seg_off .. seg_off + n_segs), items
// numbered from 0, shared memory sized by trace size ntmax
struct Run {
  int seg_off, n_segs, n_items, ntmax;
};
// one (model, degree) group of a batch, launched as runs of trace sizes at which the
// batched kernel keeps the same resident CTAs per SM (as launch_groups does for the
// degree buckets of one system; each system's bucket list is sorted by trace size)
struct Group {
  int model, p, n_items, nfield;
  bool bounded;
  std::vector<Run> runs;
};

hdg_status fail(hdg_ctx* ctx, hdg_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

#define HDG_BCK(ctx, call)                                                                                   \
  do {                                                                                                       \
    cudaError_t e_ = (call);                                                                                 \
    if (e_ != cudaSuccess) return fail(ctx, HDG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

struct hdg_batch {
  hdg_ctx* ctx = nullptr;
  bool own_mem = true;        // d_desc / d_seg cudaMalloc'd (else in the caller's workspace)
  std::vector<unsigned char> staging;  // host copy of the work list while its upload is in flight
  std::vector<hdg_sys*> sys;
  int precision = 0;
  std::vector<Group> groups;
  ReqDesc* d_desc = nullptr;  // [n_sys]
  BatchSeg* d_seg = nullptr;  // all groups' segments
  int grid[2][kMaxP + 1];     // launch shape per (model, degree): -1 default, 0 one CTA per item, k persistent
  int launches = 0;
  cudaStream_t gstream[2 * kMaxP] = {};
  cudaEvent_t gevent[2 * kMaxP] = {};
  cudaEvent_t fork = nullptr;
  bool have_streams = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
};

namespace {

Phys group_phys(const hdg_batch* B, const Group& g) {
  Phys ph = B->sys[0]->ph;  // only model, precision and the launch shape are read on the host
  ph.model = g.model;
  ph.precision = B->precision;
  phys_default_grid(ph);
  ph.grid[g.p] = B->grid[g.model][g.p];
  ph.persistent = B->groups.size() > 1 ? 0 : 1;
  return ph;
}

BatchRef run_ref(const hdg_batch* B, const Run& r) { return BatchRef{B->d_desc, B->d_seg + r.seg_off, r.n_segs}; }

hdg_status ensure_streams(hdg_batch* B) {
  if (B->have_streams) return HDG_OK;
  for (int i = 0; i < 2 * kMaxP; ++i) {
    HDG_BCK(B->ctx, cudaStreamCreateWithFlags(&B->gstream[i], cudaStreamNonBlocking));
    HDG_BCK(B->ctx, cudaEventCreateWithFlags(&B->gevent[i], cudaEventDisableTiming));
  }
  HDG_BCK(B->ctx, cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming));
  B->have_streams = true;
  return HDG_OK;
}

hdg_status condense_groups(hdg_batch* B, cudaStream_t st) {
  hdg_ctx* ctx = B->ctx;
  for (hdg_sys* S : B->sys)
    if (S->need_zero) {  // arrival counters start at zero; the kernels leave them at zero
      HDG_BCK(ctx, cudaMemsetAsync(S->ds.face_cnt, 0, 4 * (size_t)S->mesh->n_face, st));
      S->need_zero = false;
    }
  std::string err;
  int launches = 0;
  const bool fork = B->groups.size() > 1;
  if (fork) {
    // the (model, degree) groups run concurrently, one CTA per item, like the
    // degree buckets of hdg_condense; the counter protocol orders shared faces
    hdg_status rs = ensure_streams(B);
    if (rs != HDG_OK) return rs;
    HDG_BCK(ctx, cudaEventRecord(B->fork, st));
  }
  for (size_t i = 0; i < B->groups.size(); ++i) {
    const Group& g = B->groups[i];
    cudaStream_t gs = fork ? B->gstream[i] : st;
    if (fork) HDG_BCK(ctx, cudaStreamWaitEvent(gs, B->fork, 0));
    const Phys ph = group_phys(B, g);
    for (const Run& r : g.runs) {
      if (!launch_condense_batch(g.p, ph, ctx->d_tab, ctx->d_tab_ff, ctx->tab.off, run_ref(B, r), r.n_items, r.ntmax,
                                 g.bounded, gs, &err))
        return fail(ctx, HDG_ECUDA, "hdg_batch_condense: " + err);
      ++launches;
    }
    if (fork) {
      HDG_BCK(ctx, cudaEventRecord(B->gevent[i], gs));
      HDG_BCK(ctx, cudaStreamWaitEvent(st, B->gevent[i], 0));
    }
  }
  B->launches = launches;
  return HDG_OK;
}

hdg_status recover_groups(hdg_batch* B, cudaStream_t st) {
  std::string err;
  for (const Group& g : B->groups)
    for (const Run& r : g.runs) {
      if (!launch_recover_batch(g.p, g.nfield, run_ref(B, r), r.n_items, st, &err))
        return fail(B->ctx, HDG_ECUDA, "hdg_batch_recover: " + err);
      ++B->launches;
    }
  return HDG_OK;
}

hdg_status step_host(hdg_batch* B, const double* const* U, const double* const* Lam, const double* const* dLam,
                     double* const* dU, cudaStream_t st) {
  hdg_ctx* ctx = B->ctx;
  const size_t d = sizeof(double);
  for (size_t i = 0; i < B->sys.size(); ++i) {
    hdg_sys* S = B->sys[i];
    const hdg_mesh* M = S->mesh;
    if (!U[i] || !Lam[i] || !dLam[i] || !dU[i]) return fail(ctx, HDG_EINVAL, "hdg_batch_step_host_async: null array");
    HDG_BCK(ctx, cudaMemcpyAsync(S->d_U, U[i], d * M->u_len, cudaMemcpyHostToDevice, st));
    HDG_BCK(ctx, cudaMemcpyAsync(S->d_Lam, Lam[i], d * M->lam_len, cudaMemcpyHostToDevice, st));
    HDG_BCK(ctx, cudaMemcpyAsync(S->d_dLam, dLam[i], d * M->lam_len, cudaMemcpyHostToDevice, st));
  }
  hdg_status rs = condense_groups(B, st);
  if (rs == HDG_OK) rs = recover_groups(B, st);
  if (rs != HDG_OK) return rs;
  for (size_t i = 0; i < B->sys.size(); ++i) {
    hdg_sys* S = B->sys[i];
    HDG_BCK(ctx, cudaMemcpyAsync(dU[i], S->d_dU, d * S->mesh->u_len, cudaMemcpyDeviceToHost, st));
  }
  return HDG_OK;
}

void batch_free(hdg_batch* B) {
  if (B->gexec) cudaGraphExecDestroy(B->gexec);
  if (B->graph) cudaGraphDestroy(B->graph);
  if (B->have_streams) {
    for (int i = 0; i < 2 * kMaxP; ++i) {
      cudaStreamDestroy(B->gstream[i]);
      cudaEventDestroy(B->gevent[i]);
    }
    cudaEventDestroy(B->fork);
  }
  if (B->own_mem) {
    cudaFree(B->d_desc);
    cudaFree(B->d_seg);
  }
  delete B;
}

inline size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

// Validation, descriptors and the (model, degree) groups of a batch; no device work.
hdg_status batch_plan(hdg_ctx* ctx, int32_t n_sys, hdg_sys* const* systems, hdg_batch** out,
                      std::vector<ReqDesc>* desc, std::vector<BatchSeg>* segs) {
  for (int i = 0; i < n_sys; ++i) {
    const hdg_sys* S = systems[i];
    if (!S || S->ctx != ctx) return fail(ctx, HDG_EINVAL, "hdg_batch_create: a system is null or of another context");
    if (S->ph.precision != systems[0]->ph.precision)
      return fail(ctx, HDG_EINVAL, "hdg_batch_create: the systems of a batch share one precision");
    if (S->ph.precision != HDG_FP64 && S->ph.precision != HDG_FLOAT2)
      return fail(ctx, HDG_ENOTSUP, "hdg_batch_create: batches run in binary64 or float-float");
    for (int j = 0; j < i; ++j)
      if (systems[j] == S) return fail(ctx, HDG_EINVAL, "hdg_batch_create: a system appears twice");
  }
  hdg_batch* B = new hdg_batch();
  B->ctx = ctx;
  B->sys.assign(systems, systems + n_sys);
  B->precision = systems[0]->ph.precision;
  for (int md = 0; md < 2; ++md)
    for (int p = 0; p <= kMaxP; ++p) B->grid[md][p] = -1;
  desc->assign(n_sys, ReqDesc{});
  for (int i = 0; i < n_sys; ++i) {
    const hdg_sys* S = systems[i];
    ReqDesc& d = (*desc)[i];
    d.m = S->mesh->dm;
    d.s = S->ds;
    d.ph = S->ph;
    d.ph.adjoint = 0;
    d.U = S->d_U;
    d.Lam = S->d_Lam;
    d.dLam = S->d_dLam;
    d.dU = S->d_dU;
  }
  segs->clear();
  for (int md = 0; md < 2; ++md)
    for (int p = 1; p <= kMaxP; ++p) {
      Group g{md, p, 0, md == HDG_NS_MIXED ? 12 : 4, false, {}};
      int cnt[kNtSlots] = {};
      for (int i = 0; i < n_sys; ++i) {
        const hdg_sys* S = systems[i];
        const hdg_mesh* M = S->mesh;
        if (S->ph.model != md || M->bucket_n[p] == 0) continue;
        for (int t = 0; t < kNtSlots; ++t) cnt[t] += M->bucket_nt.cnt[p][t];
        g.n_items += M->bucket_n[p];
        g.bounded |= M->has_bc;
      }
      if (!g.n_items) continue;
      // runs of trace sizes with equal resident CTAs per SM of the batched kernel
      Phys ph = systems[0]->ph;
      ph.model = md;
      int occ[kNtSlots];
      for (int t = 0; t < kNtSlots; ++t) occ[t] = cnt[t] ? batch_occupancy(ph, p, 4 * t, g.bounded) : 0;
      for (int t = 0; t < kNtSlots;) {
        if (!cnt[t]) { ++t; continue; }
        int e = t, top = 4 * t;
        for (; e < kNtSlots; ++e) {
          if (!cnt[e]) continue;
          if (occ[e] != occ[t]) break;
          top = 4 * e;
        }
        Run r{(int)segs->size(), 0, 0, top};
        for (int i = 0; i < n_sys; ++i) {
          const hdg_sys* S = systems[i];
          const hdg_mesh* M = S->mesh;
          if (S->ph.model != md || M->bucket_n[p] == 0) continue;
          int off = 0, n = 0;
          for (int u = 0; u < t; ++u) off += M->bucket_nt.cnt[p][u];
          for (int u = t; u < e; ++u) n += M->bucket_nt.cnt[p][u];
          if (n == 0) continue;
          segs->push_back(BatchSeg{i, r.n_items, M->d_bucket[p] + off});
          r.n_items += n;
          ++r.n_segs;
        }
        g.runs.push_back(r);
        t = e;
      }
      B->groups.push_back(g);
    }
  *out = B;
  return HDG_OK;
}

size_t work_list_bytes(size_t n_desc, size_t n_seg) {
  return round256(sizeof(ReqDesc) * n_desc) + round256(sizeof(BatchSeg) * std::max<size_t>(n_seg, 1));
}

}  // namespace

extern "C" {

hdg_status hdg_batch_create(hdg_ctx* ctx, int32_t n_sys, hdg_sys* const* systems, hdg_batch** out) {
  if (!ctx || !systems || !out || n_sys < 1) return HDG_EINVAL;
  *out = nullptr;
  HDG_ON_DEVICE(ctx, ctx->device);
  std::vector<ReqDesc> desc;
  std::vector<BatchSeg> segs;
  hdg_batch* B = nullptr;
  hdg_status st = batch_plan(ctx, n_sys, systems, &B, &desc, &segs);
  if (st != HDG_OK) return st;
  cudaError_t e = cudaMalloc(&B->d_desc, sizeof(ReqDesc) * desc.size());
  if (e == cudaSuccess) e = cudaMalloc(&B->d_seg, sizeof(BatchSeg) * std::max<size_t>(segs.size(), 1));
  if (e != cudaSuccess) {
    batch_free(B);
    return fail(ctx, HDG_ENOMEM, std::string("hdg_batch_create: cudaMalloc: ") + cudaGetErrorString(e));
  }
  e = cudaMemcpy(B->d_desc, desc.data(), sizeof(ReqDesc) * desc.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(B->d_seg, segs.data(), sizeof(BatchSeg) * segs.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    batch_free(B);
    return fail(ctx, HDG_ECUDA, std::string("hdg_batch_create: cudaMemcpy: ") + cudaGetErrorString(e));
  }
  *out = B;
  return HDG_OK;
}

int64_t hdg_batch_workspace_bytes(int32_t n_sys, hdg_sys* const* systems) {
  if (!systems || n_sys < 1) return -1;
  size_t n_seg = 0;  // at most one segment per (system, degree, trace size)
  for (int i = 0; i < n_sys; ++i) {
    if (!systems[i]) return -1;
    for (int p = 1; p <= kMaxP; ++p)
      for (int t = 0; t < kNtSlots; ++t) n_seg += systems[i]->mesh->bucket_nt.cnt[p][t] > 0;
  }
  return (int64_t)work_list_bytes((size_t)n_sys, n_seg);
}

hdg_status hdg_batch_create_in(hdg_ctx* ctx, int32_t n_sys, hdg_sys* const* systems, void* workspace,
                               int64_t workspace_bytes, void* stream, hdg_batch** out) {
  if (!ctx || !systems || !out || n_sys < 1) return HDG_EINVAL;
  *out = nullptr;
  HDG_ON_DEVICE(ctx, ctx->device);
  const int64_t need = hdg_batch_workspace_bytes(n_sys, systems);
  if (!workspace || ((uintptr_t)workspace & 255u) != 0 || need < 0 || workspace_bytes < need)
    return fail(ctx, HDG_EINVAL, "hdg_batch_create_in: workspace must be 256-byte aligned and hold " +
                                     std::to_string(need) + " bytes");
  std::vector<ReqDesc> desc;
  std::vector<BatchSeg> segs;
  hdg_batch* B = nullptr;
  hdg_status st = batch_plan(ctx, n_sys, systems, &B, &desc, &segs);
  if (st != HDG_OK) return st;
  B->own_mem = false;
  const size_t bd = round256(sizeof(ReqDesc) * desc.size());
  B->d_desc = (ReqDesc*)workspace;
  B->d_seg = (BatchSeg*)((unsigned char*)workspace + bd);
  // one asynchronous upload of the work list from a host copy the batch keeps
  B->staging.resize(bd + sizeof(BatchSeg) * segs.size());
  std::memcpy(B->staging.data(), desc.data(), sizeof(ReqDesc) * desc.size());
  std::memcpy(B->staging.data() + bd, segs.data(), sizeof(BatchSeg) * segs.size());
  const cudaError_t e = cudaMemcpyAsync(workspace, B->staging.data(), B->staging.size(), cudaMemcpyHostToDevice,
                                        (cudaStream_t)stream);
  if (e != cudaSuccess) {
    batch_free(B);
    return fail(ctx, HDG_ECUDA, std::string("hdg_batch_create_in: cudaMemcpyAsync: ") + cudaGetErrorString(e));
  }
  *out = B;
  return HDG_OK;
}

hdg_status hdg_batch_destroy(hdg_batch* B) {
  if (!B) return HDG_EINVAL;
  hdg::DeviceGuard dg(B->ctx->device);
  batch_free(B);
  return HDG_OK;
}

int32_t hdg_batch_groups(const hdg_batch* B, int32_t* model, int32_t* p, int32_t* n_items) {
  if (!B) return -1;
  for (size_t i = 0; i < B->groups.size(); ++i) {
    if (model) model[i] = B->groups[i].model;
    if (p) p[i] = B->groups[i].p;
    if (n_items) n_items[i] = B->groups[i].n_items;
  }
  return (int32_t)B->groups.size();
}

hdg_status hdg_batch_condense(hdg_batch* B, void* stream) {
  hdg::NvtxRange nvtx_range_("hdg::batch_condense");
  if (!B) return HDG_EINVAL;
  HDG_ON_DEVICE(B->ctx, B->ctx->device);
  return condense_groups(B, (cudaStream_t)stream);
}

hdg_status hdg_batch_recover(hdg_batch* B, void* stream) {
  hdg::NvtxRange nvtx_range_("hdg::batch_recover");
  if (!B) return HDG_EINVAL;
  HDG_ON_DEVICE(B->ctx, B->ctx->device);
  return recover_groups(B, (cudaStream_t)stream);
}

hdg_status hdg_batch_step_host_async(hdg_batch* B, const double* const* U, const double* const* Lam,
                                     const double* const* dLam, double* const* dU, void* stream) {
  hdg::NvtxRange nvtx_range_("hdg::batch_step_host");
  if (!B || !U || !Lam || !dLam || !dU) return HDG_EINVAL;
  HDG_ON_DEVICE(B->ctx, B->ctx->device);
  return step_host(B, U, Lam, dLam, dU, (cudaStream_t)stream);
}

hdg_status hdg_batch_autotune(hdg_batch* B, int32_t* grid_out, void* stream) {
  hdg::NvtxRange nvtx_range_("hdg::batch_autotune");
  if (!B) return HDG_EINVAL;
  hdg_ctx* ctx = B->ctx;
  if (B->gexec) return fail(ctx, HDG_EINVAL, "hdg_batch_autotune: a captured graph holds the launch shapes");
  HDG_ON_DEVICE(ctx, ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  HDG_BCK(ctx, cudaEventCreate(&e0));
  HDG_BCK(ctx, cudaEventCreate(&e1));
  std::string err;
  hdg_status rs = HDG_OK;
  for (size_t gi = 0; gi < B->groups.size() && rs == HDG_OK; ++gi) {
    const Group& g = B->groups[gi];
    Phys ph = group_phys(B, g);
    int occ = 0;  // persistent candidates up to the largest occupancy of the group's runs
    for (const Run& r : g.runs) {
      const int o = batch_occupancy(ph, g.p, r.ntmax, g.bounded);
      if (o < 1) { occ = 0; break; }
      occ = std::max(occ, o);
    }
    if (occ < 1) { rs = fail(ctx, HDG_ECUDA, "hdg_batch_autotune: kernel does not fit on an SM"); break; }
    float best_ms = 0.0f;
    int best = -1;
    // candidates: one CTA per item, or a persistent grid of k CTAs per SM, k = 1..occupancy
    for (int cand = 0; cand <= occ && rs == HDG_OK; ++cand) {
      ph.grid[g.p] = cand;
      float t_min = 0.0f;
      for (int rep = 0; rep < 4 && rs == HDG_OK; ++rep) {
        for (hdg_sys* S : B->sys)
          if (cudaMemsetAsync(S->ds.face_cnt, 0, 4 * (size_t)S->mesh->n_face, st) != cudaSuccess)
            rs = fail(ctx, HDG_ECUDA, "hdg_batch_autotune: memset failed");
        if (rs != HDG_OK || cudaEventRecord(e0, st) != cudaSuccess) break;
        for (const Run& r : g.runs)
          if (rs == HDG_OK && !launch_condense_batch(g.p, ph, ctx->d_tab, ctx->d_tab_ff, ctx->tab.off, run_ref(B, r),
                                                     r.n_items, r.ntmax, g.bounded, st, &err))
            rs = fail(ctx, HDG_ECUDA, "hdg_batch_autotune: " + err);
        if (rs != HDG_OK) break;
        float ms = 0.0f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          rs = fail(ctx, HDG_ECUDA, "hdg_batch_autotune: timing failed");
          break;
        }
        if (rep > 0 && (rep == 1 || ms < t_min)) t_min = ms;  // first launch is a warm-up
      }
      if (rs == HDG_OK && (best < 0 || t_min < best_ms)) { best = cand; best_ms = t_min; }
    }
    if (rs == HDG_OK) B->grid[g.model][g.p] = best;
  }
  for (int md = 0; md < 2 && grid_out; ++md)
    for (int p = 0; p <= kMaxP; ++p) grid_out[md * (kMaxP + 1) + p] = B->grid[md][p];
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (hdg_sys* S : B->sys) S->need_zero = true;  // a single group's launch leaves shared faces half counted
  return rs;
}

hdg_status hdg_batch_graph_create(hdg_batch* B, const double* const* U, const double* const* Lam,
                                  const double* const* dLam, double* const* dU) {
  if (!B || !U || !Lam || !dLam || !dU) return HDG_EINVAL;
  hdg_ctx* ctx = B->ctx;
  HDG_ON_DEVICE(ctx, ctx->device);
  if (B->gexec) { cudaGraphExecDestroy(B->gexec); B->gexec = nullptr; }
  if (B->graph) { cudaGraphDestroy(B->graph); B->graph = nullptr; }
  cudaStream_t cs;
  HDG_BCK(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  // kernel attributes, streams and events are set up outside the capture by one plain step
  hdg_status rc = step_host(B, U, Lam, dLam, dU, cs);
  cudaError_t e = cudaStreamSynchronize(cs);
  if (rc == HDG_OK && e != cudaSuccess) rc = fail(ctx, HDG_ECUDA, std::string("hdg_batch_graph_create: ") + cudaGetErrorString(e));
  if (rc == HDG_OK) {
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) rc = step_host(B, U, Lam, dLam, dU, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && rc == HDG_OK) e = cudaGraphInstantiate(&B->gexec, g, 0);
    B->graph = g;
    if (rc == HDG_OK && e != cudaSuccess)
      rc = fail(ctx, HDG_ECUDA, std::string("hdg_batch_graph_create: ") + cudaGetErrorString(e));
  }
  cudaStreamDestroy(cs);
  return rc;
}

hdg_status hdg_batch_graph_launch(hdg_batch* B, void* stream) {
  if (!B) return HDG_EINVAL;
  if (!B->gexec) return fail(B->ctx, HDG_EINVAL, "hdg_batch_graph_launch: no graph (call hdg_batch_graph_create)");
  HDG_ON_DEVICE(B->ctx, B->ctx->device);
  HDG_BCK(B->ctx, cudaGraphLaunch(B->gexec, (cudaStream_t)stream));
  return HDG_OK;
}

int32_t hdg_batch_launches(const hdg_batch* B) { return B ? B->launches : -1; }

}  // extern "C"
