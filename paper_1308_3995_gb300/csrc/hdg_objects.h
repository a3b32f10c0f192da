// Definitions of the opaque objects of the C ABI (context, mesh plan,
// system), shared by the translation units that implement the ABI.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "hdg_internal.h"  // includes the public header

struct hdg_ctx {
  int device = 0;
  std::string err;
  hdg::Tables tab;
  double* d_tab = nullptr;   // tables in binary64
  void* d_tab_ff = nullptr;  // the same tables split into float-float pairs (hi, lo)
};

struct hdg_mesh {
  hdg_ctx* ctx = nullptr;
  int n_elem = 0, n_face = 0, nfield = 4, max_nt = 0;
  bool has_bc = false;
  int64_t u_len = 0, lam_len = 0, x_len = 0, k_len = 0, dh_len = 0;
  std::vector<int> face_lo, face_hi, face_el0, face_el1, face_p, elem_face, k_col;
  std::vector<int64_t> u_off, lam_off, x_off, k_blkoff;
  std::vector<void*> allocs;
  int* d_bucket[hdg::kMaxP + 1] = {};
  int bucket_n[hdg::kMaxP + 1] = {};
  int bucket_ntmax[hdg::kMaxP + 1] = {};
  hdg::BucketNt bucket_nt{};  // trace-size counts; each d_bucket list sorted by trace size
  hdg::DevMesh dm{};
};

struct hdg_sys {
  hdg_ctx* ctx = nullptr;
  const hdg_mesh* mesh = nullptr;
  hdg_params prm{};
  hdg::Phys ph{};
  hdg::DevSys ds{};
  double *d_U = nullptr, *d_Lam = nullptr, *d_dLam = nullptr, *d_dU = nullptr;
  int* d_face_el = nullptr;  // [n_face][2], uploaded by the first hdg_adjoint_condense
  std::vector<void*> allocs;
  int launches = 0;
  bool need_zero = true;
  // degree buckets launched concurrently: one stream and one event per degree, a fork event
  cudaStream_t bstream[hdg::kMaxP + 1] = {};
  cudaEvent_t bevent[hdg::kMaxP + 1] = {};
  cudaEvent_t tbeg[hdg::kMaxP + 1] = {};  // timing events around each bucket's launches
  cudaEvent_t tend[hdg::kMaxP + 1] = {};
  bool timed = false;                      // the last hdg_condense recorded them
  cudaEvent_t fork = nullptr;
  bool have_streams = false;
  // captured step (hdg_graph_create)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
};

