/*
 * hdg.h -- C ABI of the GB300 (sm_103a) hot path of one hybridized-DG (HDG)
 * Newton step for steady 2D compressible Euler and mixed-form Navier-Stokes
 * flow, after Woopen, Balan, May, Schuetz, "A comparison of hybridized and
 * standard DG methods for target-based hp-adaptive simulation of compressible
 * flow" (arXiv:1308.3995).
 *
 * The problem statement (mesh + per-element degree p + state in; condensed
 * trace system and reconstructed update out) is Sec. 3.4 of the paper:
 *   the linearised system [A B R; C D S; L M N][dQ; dW; dLambda] = [F; G; H]
 *   (Eq. linearsystem in block form) is reduced element by element to
 *   K dLambda = E (Eq. hybridsystem) with
 *   K = N - [L M][A B; C D]^{-1}[R; S],  E = H - [L M][A B; C D]^{-1}[F; G],
 *   the local solves [A B; C D]^{-1}[R S F G] are stored, and (dQ, dW) is
 *   reconstructed from dLambda by Eq. (ls).
 * In this header, per element K: A_K = local interior block [A B; C D]
 * restricted to K, B_K = [R; S] (interior rows, trace columns of K's three
 * faces), C_K = [L M] (trace rows, interior columns), D_K = N (trace-trace),
 * F_K = -residual of the interior rows, H_K = -element share of the trace rows.
 *
 * Discretisation (fixed; identical in every call):
 *   - Triangles with vertices given counter-clockwise; affine map
 *     x = x0 + J xi from the reference triangle (0,0),(1,0),(0,1).
 *   - Interior basis: orthonormal Dubiner basis on the reference triangle,
 *     n_p = (p+1)(p+2)/2 modes ordered k = 0..p, j = 0..k, i = k-j.
 *   - Faces: local face l of an element runs from local vertex l to l+1 (mod 3).
 *     A global face is an unordered pair of topological vertex ids; faces are
 *     numbered by ascending (lo id, hi id).  Its trace lives in the orthonormal
 *     Legendre basis psi_k(s) = sqrt(2k+1) P_k(2s-1), k = 0..p_e, with the
 *     edge parameter s running from the lower to the higher vertex id, and
 *     p_e = max(p of both sides) (Sec. 3.1).  Side 0 of a face is the element
 *     with the lower id.  Only closed (periodic) meshes: every face has two sides.
 *   - Quadrature: collapsed Gauss (p+2) x (p+2) on elements, (p_e+2)-point
 *     Gauss-Legendre on edges.
 *   - Numerical flux (Sec. 3.2): (f_c(lambda) - f_v(lambda, q)).n - alpha (lambda - w),
 *     with the jump of Eq. (hdg_cont) read as the sum over both sides.
 *
 * Layouts (all FP64, little-endian, contiguous):
 *   U      element K at u_off[K]: n_K = nfield * n_p(p_K) values, fields
 *          major, modes minor.  Euler: nfield = 4, fields (rho, rho u, rho v, E).
 *          Navier-Stokes: nfield = 12, fields q_x(4), q_y(4), w(4) with
 *          q = grad w of the conserved variables (Eq. strmixed).
 *   Lambda face e at lam_off[e]: 4 (p_e+1) values, [field][mode].
 *   X      element K at x_off[K]: the n_K x (nt_K + 1) matrix X = A_K^{-1}[B_K | F_K]
 *          (the stored local solves of Sec. 3.4) in COLUMN-major order: entry
 *          (r, c) at x_off[K] + c n_K + r, column nt_K being X_F; nt_K = sum over
 *          K's faces in local order of 4 (p_e+1).
 *   K      block-sparse trace matrix: block row e has 5 blocks (itself and the
 *          other two faces of each neighbour, Sec. 3.4 last paragraph), column
 *          face ids ascending in k_col[5e .. 5e+4]; block b of row e starts at
 *          k_blkoff[5e+b] (in doubles) and is 4(p_e+1) x 4(p_col+1) row-major.
 *   E      layout of Lambda.
 *
 * Conventions:
 *   - Every call returns an hdg_status; hdg_last_error() gives the text of the
 *     last failure on that context.
 *   - Calls taking a `stream` (a cudaStream_t, e.g. torch's current stream) are
 *     asynchronous: results are valid after that stream is synchronised.
 *   - Pointers documented "device" must be device memory of the context's
 *     device, 8-byte aligned; "host" pointers are read before the call returns
 *     unless stated otherwise.  The library never frees caller memory; objects
 *     it creates are freed by the matching destroy call.
 *   - A context is used from one host thread at a time.  Calls on different
 *     systems may run on different streams concurrently.
 *   - Every call that touches the GPU makes its context's device current for
 *     the duration of the call and restores the calling thread's current
 *     device before it returns.
 *   - A call reports the CUDA errors of its own work: a pending non-sticky
 *     error (cudaGetLastError) left by an earlier call of the caller or of
 *     another library is discarded on entry.  Sticky errors (a faulted
 *     context) are not cleared and fail the call.
 */
#ifndef HDG_H_
#define HDG_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hdg_ctx hdg_ctx;
typedef struct hdg_mesh hdg_mesh;
typedef struct hdg_sys hdg_sys;

typedef enum {
  HDG_OK = 0,
  HDG_EINVAL = 1,     /* bad argument, layout or mesh */
  HDG_ENOMEM = 2,     /* device allocation failed or footprint over the limit */
  HDG_ECUDA = 3,      /* a CUDA runtime call failed */
  HDG_ESINGULAR = 4,  /* some element's local block had a zero pivot (see elem_status) */
  HDG_ETIMEOUT = 5,   /* a bounded device wait ran out */
  HDG_ENOTSUP = 6     /* combination not supported by this library */
} hdg_status;

typedef enum { HDG_EULER = 0, HDG_NS_MIXED = 1 } hdg_model;

typedef enum {
  HDG_FP64 = 0,    /* element work in IEEE binary64 (the FP64 pipe) */
  HDG_FLOAT2 = 1   /* element work in float-float arithmetic: every value a pair of
                      binary32 words (hi + lo, ~48-bit significand) computed with
                      error-free transformations on the binary32 pipe; inputs and
                      outputs stay binary64; accuracy ~1e-13 relative (FP64-class),
                      far above binary32 */,
  HDG_MIXED_TF32 = 2, /* Euler only: residual and Jacobian assembled in binary64; the
                      local LU and solves of Sec. 3.4 in binary32 on the tensor cores
                      (rank-8 updates as three TF32 MMAs on hi/lo splits, binary32
                      accumulation), refined against binary64 residuals [B | F] - A X
                      (params refine_max, refine_tol); Schur complement, assembly and
                      reconstruction in binary64 */
  HDG_MIXED_BF16 = 3  /* as HDG_MIXED_TF32 with one BF16 MMA per update (8-bit
                      significands): the refinement needs many more sweeps */
} hdg_precision;

/* Flow and discretisation parameters (paper Sec. 2 and 3).  Non-dimensional
 * with rho_inf = 1, c_inf = 1, L = 1: p_inf = 1/gamma, |v_inf| = mach,
 * T = gamma p / rho, mu = (mach/reynolds) T^{3/2} (1+S)/(T+S), S = 110.4/t_inf,
 * heat conductivity mu / ((gamma-1) prandtl). */
typedef struct {
  int32_t model;       /* hdg_model */
  int32_t precision;   /* hdg_precision */
  double gamma;        /* ratio of specific heats, Sec. 2.1 (1.4) */
  double prandtl;      /* Sec. 2.2 (0.72) */
  double reynolds;     /* Sec. 2.2 */
  double mach;         /* free-stream Mach number */
  double alpha;        /* constant scalar stabilisation alpha = alpha_c + alpha_v, Sec. 3.2 */
  double cfl;          /* <= 0: pure Newton; > 0: pseudo-time mass |K|-scaled by the local
                          time step CFL |K| / (lambda_c + 4 lambda_v) of Sec. 3.3 */
  double t_inf;        /* dimensional free-stream temperature [K] for Sutherland (288.15) */
  double refine_tol;   /* HDG_MIXED_*: stop refining once a correction is below
                          refine_tol * max|X| of the element (e.g. 1e-13) */
  int32_t refine_max;  /* HDG_MIXED_*: at most this many corrections after the first
                          solve; an element that has not met refine_tol then gets
                          elem_status 3 (its X is still the last iterate) */
  int32_t reserved;
  /* Shock capturing, Sec. 3.2 (artificial viscosity, volume term only):
   *   N_w += eps_K (grad phi, grad w)_K   (Euler)   or   eps_K (grad phi, q)_K   (NS),
   *   eps_K = sc_eps0 (h_K / p_K)^(2 - sc_beta) / |K| * int_K sum_f |(div f_c(w))_f| dx,
   * h_K the longest edge of K; for NS the gradient in div f_c is q.  eps_K is
   * evaluated at the given state and held fixed in the Newton matrix (the
   * Jacobian does not differentiate it).  sc_eps0 <= 0 disables the term
   * (paper's values when needed: sc_eps0 = 0.2, sc_beta = 0). */
  double sc_eps0;
  double sc_beta;
  /* Free-stream angle of attack [degrees]: the far-field state of boundary
   * faces (Sec. 2.1) is rho = 1, |v| = mach at this angle, p = 1/gamma. */
  double aoa;
} hdg_params;

/* Create a context on CUDA device `device` (makes it current on this thread). */
hdg_status hdg_create(hdg_ctx** out, int device);
hdg_status hdg_destroy(hdg_ctx* ctx);
/* Text of the last error on ctx (never NULL; empty if none). */
const char* hdg_last_error(const hdg_ctx* ctx);

/* Build a device-resident mesh plan (faces, sides, degree buckets, layouts,
 * basis/quadrature tables).  All pointers are HOST arrays, copied:
 *   elem_xy  [n_elem][3][2] vertex coordinates, counter-clockwise, periodic
 *            images already resolved so each element is a proper triangle;
 *   elem_vid [n_elem][3]    topological vertex ids (periodic images identified);
 *   elem_p   [n_elem]       degree p_K in 1..4.
 * nfield = 4 (Euler) or 12 (Navier-Stokes mixed form).
 * Fails with HDG_EINVAL if det J <= 0, p out of range, a face is not shared by
 * exactly two distinct elements, or two elements share two faces. */
hdg_status hdg_mesh_create(hdg_ctx* ctx, int32_t n_elem, int32_t nfield, const double* elem_xy,
                           const int32_t* elem_vid, const int8_t* elem_p, hdg_mesh** out);

/* hdg_mesh_create for a bounded domain (Sec. 2.1, 2.2, 3.2).  elem_bc (HOST,
 * may be NULL = every face interior) [n_elem][3]: boundary kind of local face
 * l of each element -- 0 interior; Euler (nfield = 4): 1 slip wall, 2 far
 * field (characteristic upwinding against the free stream of hdg_params.mach /
 * aoa); Navier-Stokes (nfield = 12): 3 no-slip adiabatic wall (w_b = (rho, 0,
 * 0, E), wall viscous flux (0, tau, 0)), 2 far field (the same characteristic
 * state, the viscous flux f_v(w_b, q) at it whole, q the interior gradient;
 * the gradient equations' boundary term -<tau.n, w_b(w)> couples the fields
 * through d w_b / d w).  A boundary face carries no trace
 * unknowns: the element gets the boundary operator of Sec. 3.2 and its
 * Jacobian instead, elem_face is -1 there, and rows of K next to a boundary
 * keep their five slots with the unused ones marked k_col = -1 (empty blocks,
 * after the used columns).  Every untagged face must be shared by exactly two
 * elements.  HDG_EINVAL for a kind outside 0..3 or kind 3 on an Euler mesh;
 * HDG_ENOTSUP for kind 1 (slip wall) on a Navier-Stokes mesh. */
hdg_status hdg_mesh_create_bc(hdg_ctx* ctx, int32_t n_elem, int32_t nfield, const double* elem_xy,
                              const int32_t* elem_vid, const int8_t* elem_p, const int8_t* elem_bc,
                              hdg_mesh** out);
hdg_status hdg_mesh_destroy(hdg_mesh* mesh);

/* sizes[7] = {n_elem, n_face, u_len, lam_len, x_len, k_len, max_nt} */
hdg_status hdg_mesh_sizes(const hdg_mesh* mesh, int64_t* sizes);

/* Layout arrays into HOST buffers (each may be NULL):
 * face_vid[n_face][2] (lo, hi), face_el[n_face][2] (side 0, side 1 element),
 * face_p[n_face], elem_face[n_elem][3], u_off[n_elem+1], lam_off[n_face+1],
 * x_off[n_elem+1], k_col[5 n_face], k_blkoff[5 n_face + 1]. */
hdg_status hdg_mesh_layout(const hdg_mesh* mesh, int32_t* face_vid, int32_t* face_el, int32_t* face_p,
                           int32_t* elem_face, int64_t* u_off, int64_t* lam_off, int64_t* x_off,
                           int32_t* k_col, int64_t* k_blkoff);

/* Device bytes a system on this mesh holds (X, K, E, residuals, status,
 * work space), for admission control.  Returns -1 on bad arguments. */
int64_t hdg_footprint_bytes(const hdg_mesh* mesh, const hdg_params* params);

/* Allocate a system (X, K, E, residuals, per-element status, work space) on
 * the mesh's device.  params->model must match the mesh's nfield. */
hdg_status hdg_sys_create(hdg_ctx* ctx, const hdg_mesh* mesh, const hdg_params* params, hdg_sys** out);

/* Bytes of device workspace a system on this mesh needs (the same figure as
 * hdg_footprint_bytes): every buffer of the system rounded up to 256 bytes. */
int64_t hdg_sys_workspace_bytes(const hdg_mesh* mesh, const hdg_params* params);

/* Like hdg_sys_create, but every buffer of the system is carved out of the
 * caller's DEVICE workspace (256-byte aligned, at least
 * hdg_sys_workspace_bytes); the library allocates no device memory for it and
 * hdg_sys_destroy frees nothing of it.  The workspace must outlive the system.
 * Lets a scheduler admit requests against its own pre-allocated arena (and
 * never call cudaMalloc/cudaFree, which synchronise the device, while other
 * requests are running). */
hdg_status hdg_sys_create_in(hdg_ctx* ctx, const hdg_mesh* mesh, const hdg_params* params, void* workspace,
                             int64_t workspace_bytes, hdg_sys** out);
hdg_status hdg_sys_destroy(hdg_sys* sys);

/* One Newton step's element work (Sec. 3.4, paper's Eqs. hdg_ls1-hdg_cont,
 * linearsystem, ls, hybridsystem), enqueued on `stream`:
 *   residual and Jacobian blocks of every element by quadrature, LU of A_K
 *   with partial pivoting, X_K = A_K^{-1}[B_K | F_K], S_K = D_K - C_K X_B,
 *   E_K = H_K - C_K X_F, assembly K = sum_K P^T S_K P, E = sum_K P^T E_K.
 * U [u_len] and Lam [lam_len] are DEVICE pointers in the layouts above.
 * Outputs stay in `sys` (see hdg_sys_get).  Every diagonal block of K and
 * every entry of E / res_lam is the sum of exactly two element contributions,
 * so results are bitwise reproducible.  elem_status[K] is set to 0 (ok),
 * 1 (zero pivot) or 2 (non-finite result).
 * Launches: one per degree bucket, the buckets of a mixed-degree mesh on their
 * own streams (forked from and joined back to `stream`); a bucket whose trace
 * sizes differ (a face takes the larger degree of its two sides) is launched in
 * groups of trace sizes at which the kernel keeps the same number of resident
 * CTAs per SM, each group's shared memory sized by its largest trace. */
hdg_status hdg_condense(hdg_sys* sys, const double* U, const double* Lam, void* stream);

/* Reconstruction, Eq. (ls): dU_K = X_F - X_B dLambda_K for every element,
 * from the local solves stored by the last hdg_condense on this system.
 * dLam [lam_len] and dU [u_len] are DEVICE pointers. */
hdg_status hdg_recover(hdg_sys* sys, const double* dLam, double* dU, void* stream);

/* Whole step from HOST buffers: copies U, Lam, dLam host->device, runs
 * hdg_condense and hdg_recover, and copies dU device->host, all on `stream`;
 * returns after the stream has synchronised.  Host buffers should be pinned
 * for full copy bandwidth.  dLam stands in for the trace update of the global
 * solve, which is outside this library. */
hdg_status hdg_step_host(hdg_sys* sys, const double* U, const double* Lam, const double* dLam, double* dU,
                         void* stream);

/* hdg_step_host without the final synchronisation: everything is enqueued on
 * `stream` and the call returns at once; dU is valid (and U, Lam, dLam may be
 * reused) only after the stream has synchronised.  The host buffers must be
 * page-locked (pinned) for the copies to be asynchronous.  This is the call a
 * scheduler uses to keep several requests in flight on several streams. */
hdg_status hdg_step_host_async(hdg_sys* sys, const double* U, const double* Lam, const double* dLam, double* dU,
                               void* stream);

/* Capture one whole step on this system -- arrival-counter reset, the
 * condensation of every degree bucket (buckets on their own streams, joined),
 * and the reconstruction -- into a CUDA graph owned by sys, for the DEVICE
 * buffers U, Lam, dLam, dU given here (their addresses are baked into the
 * graph).  Runs the step once outside the capture first (results valid after
 * the call).  A later call replaces the graph. */
hdg_status hdg_graph_create(hdg_sys* sys, const double* U, const double* Lam, const double* dLam, double* dU);
/* Replay the captured step on `stream` (asynchronous); inputs are read from the
 * buffers given to hdg_graph_create. */
hdg_status hdg_graph_launch(hdg_sys* sys, void* stream);

/* Device views of the outputs (owned by sys, valid until hdg_sys_destroy):
 * X [x_len], K_vals [k_len], E [lam_len], res_u [u_len] = interior residual
 * [N_q; N_w] per element, res_lam [lam_len] = trace residual summed over both
 * sides, elem_status [n_elem].  Any pointer may be NULL. */
hdg_status hdg_sys_get(const hdg_sys* sys, double** X, double** K_vals, double** E, double** res_u,
                       double** res_lam, int32_t** elem_status);

/* Autotuner of the condensation launch shape (no counterpart in the paper).
 * For every degree bucket of the mesh, times the bucket's kernel alone on the
 * given state (device U, Lam; one warm-up and three timed launches each, CUDA
 * events on `stream`) for every candidate shape -- one CTA per element, or a
 * persistent grid of k CTAs per SM for k = 1 .. the kernel's occupancy -- and
 * keeps the fastest for the following hdg_condense calls of this system.
 * The shape changes no arithmetic: results stay bitwise the same.  Synchronises
 * `stream`; leaves the system's outputs undefined until the next hdg_condense.
 * grid_out (may be NULL) receives [kMaxP+1 = 5] entries: per degree p the
 * chosen shape (0 one CTA per element, k > 0 persistent with k CTAs per SM,
 * -1 no elements of that degree).  Not allowed while a captured graph exists. */
hdg_status hdg_autotune(hdg_sys* sys, const double* U, const double* Lam, int32_t* grid_out, void* stream);

/* ---- Adaptation decisions (Sec. 4) ----
 * Per element, into DEVICE arrays [n_elem] (either output may be NULL):
 *   sensor[K] = S_K = |w - w*|^2_K / |w|^2_K (Sec. 4.4): w* the L2 projection
 *     of the element's conserved state onto degree p_K - 1; the inner product
 *     of the vector w sums its four components; with the orthonormal
 *     hierarchical basis this is the share of the squared degree-p_K
 *     coefficients;
 *   eta2[K] = eta_K^2, eta_K = |N_h(x_h; q~, w~, 0)|_K| (Sec. 4.1): the interior
 *     residual rows of K (res_u of the last hdg_condense of sys) weighted by the
 *     adjoint's interior coefficients Uadj [u_len], in the discrete space itself
 *     (the paper evaluates it in an enriched space, which this library does not
 *     build).  Needs Uadj (else eta2 is left alone).
 * U and Uadj are DEVICE vectors [u_len]; enqueued on `stream`. */
hdg_status hdg_adapt_indicators(hdg_sys* sys, const double* U, const double* Uadj, double* eta2, double* sensor,
                                void* stream);

/* Doerfler marking and the h/p choice (Sec. 4.3, 4.4) on DEVICE eta2, sensor
 * [n]: the smallest set M with eta_M >= (1 - theta) eta_T (eta^2 summed),
 * taken in the order eta descending, index ascending; the sums are exact
 * integer sums of v_K = floor(eta_K^2 / max_K eta_K^2 * 2^bits), bits =
 * 62 - ceil(log2(n + 1)), so the set does not depend on a summation order.
 * code[K] (DEVICE int8 [n]) = 0 unmarked, 1 p-enrichment (marked and
 * S_K < eps_s), 2 mesh refinement (marked, S_K >= eps_s); *n_marked (may be
 * NULL) the size of M.  The paper's values: theta = 0.05, eps_s = 1e-6.
 * Uses a stream-ordered temporary of 8 n bytes; synchronises `stream`. */
hdg_status hdg_adapt_mark(hdg_ctx* ctx, int32_t n, const double* eta2, const double* sensor, double theta,
                          double eps_s, int8_t* code, int32_t* n_marked, void* stream);

/* Number of kernel launches the last hdg_condense + hdg_recover enqueued. */
int32_t hdg_sys_launches(const hdg_sys* sys);

/* Per-degree time of the last hdg_condense on a mesh with more than one degree
 * bucket (the buckets run concurrently on forked streams): ms[p], p = 1..4,
 * the milliseconds between the start and the end of bucket p's launches on
 * its stream (CUDA events; waits for them), -1 for an empty bucket; ms[0] is
 * -1.  All -1 after a single-bucket hdg_condense or one captured into a graph.
 * HOST array ms[5]. */
hdg_status hdg_sys_bucket_times(const hdg_sys* sys, float* ms);

/* ---- Batched condensation across systems ----
 * The element work of Sec. 3.4 is independent per element, whatever mesh the
 * element belongs to.  A batch condenses the elements of several systems --
 * different meshes, degree maps, flow parameters (alpha, Mach, CFL, far field),
 * Euler or Navier-Stokes -- with ONE kernel launch per (model, degree) group
 * (one per run of trace sizes with equal occupancy, where the group's trace
 * sizes differ) over a work list of (system, element) segments, instead of one
 * launch per system and degree: many small requests then fill the GPU like one
 * large one.  Each
 * element's arithmetic is that of hdg_condense (the same kernel source compiled
 * for the work list), so every system's X, K, E, residuals and status are
 * those of condensing it alone, up to the rounding of multiply-adds that the
 * compiler contracts differently (measured <= 1e-13 relative).
 * Requirements: the systems belong to ctx, share one precision (HDG_FP64 or
 * HDG_FLOAT2; else HDG_ENOTSUP) and are distinct; the batch refers to them (and to their mesh plans), which must
 * outlive it.  A system may belong to several batches, but batches that share
 * a system must not run concurrently.  Inputs and outputs are each system's
 * own device buffers: U, Lam, dLam and dU in the system's staging buffers
 * (filled by hdg_batch_step_host_async, or through hdg_sys_io), results in
 * hdg_sys_get's views.
 * hdg_batch_create uploads the work list (two small cudaMalloc'd arrays);
 * hdg_batch_destroy frees it (and any captured graph). */
typedef struct hdg_batch hdg_batch;
hdg_status hdg_batch_create(hdg_ctx* ctx, int32_t n_sys, hdg_sys* const* systems, hdg_batch** out);
/* The same batch with its work list in a caller DEVICE workspace (256-byte
 * aligned, hdg_batch_workspace_bytes(n_sys, systems) bytes; -1 on bad
 * arguments), uploaded by one cudaMemcpyAsync on `stream` (the batch keeps the
 * host copy until it is destroyed): no cudaMalloc, for schedulers that form a
 * batch while other work runs.  Use the batch on `stream` or after it. */
int64_t hdg_batch_workspace_bytes(int32_t n_sys, hdg_sys* const* systems);
hdg_status hdg_batch_create_in(hdg_ctx* ctx, int32_t n_sys, hdg_sys* const* systems, void* workspace,
                               int64_t workspace_bytes, void* stream, hdg_batch** out);
hdg_status hdg_batch_destroy(hdg_batch* batch);
/* The (model, degree) groups of the batch: returns their number G (<= 8) and
 * fills model[G] (HDG_EULER / HDG_NS_MIXED), p[G] and n_items[G] (elements
 * over all systems); any array may be NULL.  A group whose trace sizes differ
 * is launched in runs of trace sizes at which the kernel keeps the same number
 * of resident CTAs per SM (as hdg_condense does for a system's buckets). */
int32_t hdg_batch_groups(const hdg_batch* batch, int32_t* model, int32_t* p, int32_t* n_items);
/* a1-a7 for every element of every system, from each system's device U and Lam
 * staging buffers; groups run concurrently on forked streams, joined back
 * into `stream`.  Asynchronous. */
hdg_status hdg_batch_condense(hdg_batch* batch, void* stream);
/* a8 for every system: dU = X_F - X_B dLambda from its device dLam staging
 * buffer into its dU staging buffer, one launch per run of each group.
 * Asynchronous. */
hdg_status hdg_batch_recover(hdg_batch* batch, void* stream);
/* A whole step of every system from HOST arrays (arrays of n_sys pointers, one
 * per system, in the order given to hdg_batch_create; pinned memory for
 * asynchronous copies): H2D of U, Lam, dLam, hdg_batch_condense,
 * hdg_batch_recover, D2H of dU.  Enqueued on `stream`; returns at once. */
hdg_status hdg_batch_step_host_async(hdg_batch* batch, const double* const* U, const double* const* Lam,
                                     const double* const* dLam, double* const* dU, void* stream);
/* Autotuner of the batched launch shape, as hdg_autotune for one system: per
 * group, every candidate (one CTA per element, persistent k CTAs per SM) timed
 * alone on the current staging inputs; the fastest is kept.  grid_out (may be
 * NULL) receives [2][5] entries (model, degree).  Synchronises `stream`; the
 * systems' outputs are undefined until the next condensation.  Not allowed
 * while a captured graph exists. */
hdg_status hdg_batch_autotune(hdg_batch* batch, int32_t* grid_out, void* stream);
/* Capture hdg_batch_step_host_async for the HOST arrays given here (their
 * addresses are baked into the graph) into one CUDA graph owned by the batch,
 * after one plain step outside the capture (results valid after the call);
 * hdg_batch_graph_launch replays it on `stream`.  A later create replaces it. */
hdg_status hdg_batch_graph_create(hdg_batch* batch, const double* const* U, const double* const* Lam,
                                  const double* const* dLam, double* const* dU);
hdg_status hdg_batch_graph_launch(hdg_batch* batch, void* stream);
/* Kernel launches of the last batched condensation + reconstruction. */
int32_t hdg_batch_launches(const hdg_batch* batch);
/* Device addresses of a system's staging buffers: U [u_len], Lam [lam_len],
 * dLam [lam_len], dU [u_len] (owned by sys); any pointer may be NULL. */
hdg_status hdg_sys_io(const hdg_sys* sys, double** U, double** Lam, double** dLam, double** dU);

/* ---- Global trace solve and pseudo-transient Newton update (Sec. 3.3, 3.4) ----
 * The paper solves K dLambda = E (Eq. hybridsystem) with preconditioned GMRES
 * (an ILU(n) preconditioner through PETSc).  This library solves it on the GPU
 * with restarted GMRES, left-preconditioned by block Jacobi (default: M = the
 * diagonal face blocks of K, inverted once per solve by Gauss-Jordan with
 * partial pivoting), multicolor block SGS or block ILU(0) (see
 * hdg_solver_set_preconditioner).  Arnoldi uses classical Gram-Schmidt with
 * one re-orthogonalisation pass, run delayed (one reduction and one update
 * pass over the basis per iteration); the Hessenberg columns, their Givens
 * rotations and the least-squares solve run on the device, the residual
 * estimate is read back once per chunk of four iterations.  Binary64 by
 * default; double-word arithmetic on the binary32 pipe with
 * hdg_solver_set_arithmetic. */
typedef struct hdg_solver hdg_solver;

/* Allocate the solver's device state for `sys` (Krylov basis of restart+1
 * vectors of lam_len doubles, block inverses, reduction buffers).
 * restart in 1..64.  The solver reads K and E of `sys` as left by the last
 * hdg_condense; it must be destroyed before sys. */
hdg_status hdg_solver_create(hdg_sys* sys, int32_t restart, hdg_solver** out);
hdg_status hdg_solver_destroy(hdg_solver* solver);

/* The same solver with every device buffer in the caller's DEVICE workspace
 * (256-byte aligned, at least hdg_solver_workspace_bytes(mesh, restart,
 * precond) bytes, owned by the caller and untouched after
 * hdg_solver_destroy), preconditioner kind `precond` (0..3 as for
 * hdg_solver_set_preconditioner; switching to an ILU(0) kind later needs a
 * workspace planned with that kind).  Creating and destroying it allocates and frees
 * no device memory, so neither synchronises the device.  HDG_EINVAL for a
 * short or misaligned workspace. */
hdg_status hdg_solver_create_ws(hdg_sys* sys, int32_t restart, int32_t precond, void* workspace, int64_t bytes,
                                hdg_solver** out);

/* Bytes of device workspace hdg_solver_create_ws needs for a system on `mesh`
 * (-1 for invalid arguments). */
int64_t hdg_solver_workspace_bytes(const hdg_mesh* mesh, int32_t restart, int32_t precond);

/* hdg_solver_create_ws with the GMRES arithmetic `arith` of
 * hdg_solver_set_arithmetic (0 binary64, 1 float-float) planned into the
 * caller's workspace: with arith 1 the workspace also holds the double-word
 * copies (8 bytes per value of K and of the pivot inverses, twice that for
 * kinds 2 and 3, plus two vectors), the solver starts in arith 1 and creating
 * it still allocates no device memory.  Sizes from
 * hdg_solver_workspace_bytes_arith (-1 for invalid arguments); arith 0 is
 * hdg_solver_create_ws / hdg_solver_workspace_bytes.  HDG_EINVAL for another
 * arith or a short or misaligned workspace.  (No counterpart in the paper,
 * which solves in binary64.) */
hdg_status hdg_solver_create_ws_arith(hdg_sys* sys, int32_t restart, int32_t precond, int32_t arith, void* workspace,
                                      int64_t bytes, hdg_solver** out);
int64_t hdg_solver_workspace_bytes_arith(const hdg_mesh* mesh, int32_t restart, int32_t precond, int32_t arith);

/* Solve K dLam = E for the DEVICE vector dLam [lam_len] (its input value is
 * the initial guess; pass zeros for none), on `stream`.  Stops when the
 * preconditioned residual ||M^-1 (E - K dLam)||_2 <= rtol ||M^-1 E||_2 or after
 * max_iter iterations.  The call synchronises `stream` (it reads the
 * residual estimate back once per chunk of four iterations; the Arnoldi
 * bookkeeping runs on the device) and returns the iteration count and the
 * final preconditioned relative residual in *iters / *rel_res (either may be
 * NULL).  Returns HDG_OK when converged, HDG_ETIMEOUT when max_iter was
 * reached first, HDG_ESINGULAR when a pivot block of the preconditioner (a
 * diagonal block of K; for ILU(0), a modified one) is singular. */
hdg_status hdg_trace_solve(hdg_solver* solver, double* dLam, double rtol, int32_t max_iter, int32_t* iters,
                           double* rel_res, void* stream);

/* Preconditioner of the trace solve: 0 block Jacobi (default), 1 multicolor
 * block symmetric Gauss-Seidel -- faces colored greedily so that no two faces
 * of one element share a color, then one forward and one backward sweep over
 * the colors, each color's block rows updated in parallel with the diagonal
 * inverses of block Jacobi (about three times the work of a block-Jacobi
 * application) -- or 2 block ILU(0), the paper's incomplete LU with no fill
 * level (Sec. 3.4), eliminated in the same multicolor order: rows of one color
 * are factored in parallel, L_ek = F_ek U_kk^{-1} for the faces k of earlier
 * colors, F_ej -= L_ek F_kj inside K's block pattern; M = L U is applied by a
 * forward and a backward sweep over the colors (about twice the work of a
 * block-Jacobi application), or 3 the same block ILU(0) with binary32
 * factors (a mixed-precision preconditioner: the factorization runs on the
 * binary32 pipe from a binary32 copy of K, the sweeps stream half the bytes
 * and form their products in binary64, so M = L U stays one fixed linear
 * operator and the binary64 GMRES loses no accuracy).  Kinds 2 and 3
 * allocate a copy of K's values, the pivot inverses and one vector here
 * (HDG_ENOMEM if that fails).  All kinds apply to both K and K^T (M^{-T} from
 * the same factors).  Returns HDG_EINVAL for any other kind. */
hdg_status hdg_solver_set_preconditioner(hdg_solver* solver, int32_t kind);

/* Arithmetic of the GMRES iterations of hdg_trace_solve / hdg_trace_solve_ex /
 * hdg_solve_step_host (no counterpart in the paper, which solves in binary64):
 * 0 binary64 throughout (default); 1 double-word ("float-float") arithmetic on
 * the binary32 pipe for the preconditioned products, the preconditioner
 * sweeps, the Gram-Schmidt dot products and updates and the solution update.
 * Under 1 every solve first copies K (and, for kind 2, the binary64 ILU
 * factors and their pivot inverses) into float-float pairs (hi, lo: the
 * leading 24 and next 23 significand bits, integer split,
 * |hi + lo - v| < 2^-46 |v|), kind 3's binary32 factors as they are, each
 * block reordered for the product kernel (for K or for K^T, by the solve's
 * transpose flag); kinds 0 and 1 compute their block pivot inverses in
 * binary32 (a fixed preconditioner: the system solved and the accuracy
 * reached are unchanged, only the convergence rate may differ).  The solve
 * then runs on float-float copies of E and x, the Krylov basis stored as
 * pairs in the same 8 bytes per value; x is rounded back to binary64 at the
 * end.  Relative error of a product or dot product ~2^-46 of the magnitudes
 * summed.  On GB300 a binary64 product of 0.25 flop per byte is bound by the
 * binary64 pipe before HBM; in arith 1 it streams the same bytes on the
 * binary32 pipe.  The first call with arith 1 (and a later change to kind 2
 * or 3) allocates the copies: 8 bytes per value of K and of the pivot
 * inverses (twice that for kinds 2 and 3) plus two vectors; HDG_ENOMEM if
 * that fails or if the solver lives in a caller's workspace planned without
 * them (hdg_solver_create_ws; hdg_solver_create_ws_arith plans them).  After a solve in arith 1
 * with kind 0 or 1 the binary64 pivot inverses are not current:
 * hdg_solver_precond_apply then needs hdg_solver_setup first.  The
 * Hessenberg least-squares problem and hdg_trace_matvec stay binary64.
 * HDG_EINVAL for any other value. */
hdg_status hdg_solver_set_arithmetic(hdg_solver* solver, int32_t arith);

/* Factor the preconditioner of the solver's kind for the system's current K
 * (enqueued on `stream`, then `stream` is synchronised).  hdg_trace_solve*
 * does this itself at every call; it is needed before
 * hdg_solver_precond_apply.  HDG_ESINGULAR if a pivot block is singular. */
hdg_status hdg_solver_setup(hdg_solver* solver, void* stream);

/* z = M^{-1} r, or M^{-T} r when transpose != 0, with the preconditioner of the
 * last hdg_solver_setup or solve (DEVICE vectors [lam_len], r != z; enqueued on
 * `stream`).  HDG_EINVAL if no factorization of the current kind exists. */
hdg_status hdg_solver_precond_apply(hdg_solver* solver, const double* r, double* z, int32_t transpose,
                                    void* stream);

/* The multicolor order: face_color[n_face] (HOST, may be NULL) receives each
 * face's color (0-based; no two faces of one element share one), *n_colors
 * (may be NULL) the number of colors. */
hdg_status hdg_solver_colors(const hdg_solver* solver, int32_t* face_color, int32_t* n_colors);

/* Like hdg_trace_solve, with a right-hand side other than the system's E
 * (DEVICE rhs [lam_len]; NULL: E) and, when transpose != 0, the transposed
 * system K^T x = rhs (block Jacobi then uses the transposed diagonal blocks):
 * the hybridized adjoint system of Sec. 4.2. */
hdg_status hdg_trace_solve_ex(hdg_solver* solver, const double* rhs, int32_t transpose, double* dLam, double rtol,
                              int32_t max_iter, int32_t* iters, double* rel_res, void* stream);

/* One pseudo-transient Newton step of Sec. 3.3 from HOST buffers, blocking:
 * copy U [u_len] and Lam [lam_len] to the system's device staging, condense
 * (hdg_condense), solve K dLam = E with `solver` (built on this system) to
 * `rtol` as hdg_trace_solve, reconstruct dU = X_F - X_B dLam (hdg_recover),
 * copy dU [u_len] and dLam [lam_len] back, synchronise `stream`.  Statuses as
 * the calls it makes (HDG_ETIMEOUT when the solve stops at max_iter: dU and
 * dLam are then not written). */
hdg_status hdg_solve_step_host(hdg_sys* sys, hdg_solver* solver, const double* U, const double* Lam, double* dU,
                               double* dLam, double rtol, int32_t max_iter, int32_t* iters, double* rel_res,
                               void* stream);

/* y = K x, or y = K^T x when transpose != 0, for DEVICE vectors x, y
 * [lam_len] (K of the last hdg_condense). */
hdg_status hdg_trace_matvec(hdg_solver* solver, const double* x, double* y, int32_t transpose, void* stream);

/* Hybridized adjoint (Sec. 4.2; Euler and Navier-Stokes).  The adjoint system is
 * the transpose of the Newton matrix of `primal` (same mesh and parameters,
 * pseudo-time mass included), right-hand side [F~; 0] (F~ = J'(U) for a target
 * functional J of the interior unknowns; the trace part is zero in the
 * paper's formulation).  Given DEVICE U, Lam (the state of the primal's last
 * hdg_condense) and Ftilde [u_len], this enqueues on `stream`:
 *   X~_K = A_K^{-T} [C_K^T | F~_K] into adj's X (the adjoint local solves),
 *   E~ = sum_K -X_B,K^T F~_K into adj's E (from primal's stored local solves).
 * Then solve K^T Lambda~ = E~ with hdg_trace_solve_ex(solver of primal,
 * E~ of adj, transpose = 1, ...) and reconstruct U~ = X~_F - X~_C Lambda~ with
 * hdg_recover(adj, Lambda~, U~).  adj must be a separate system on the same
 * mesh with the same parameters (HDG_EINVAL otherwise).  For Navier-Stokes
 * F~ covers all of [Q; W] (a functional of the gradient, e.g. a wall shear,
 * has a q part). */
hdg_status hdg_adjoint_condense(hdg_sys* adj, const hdg_sys* primal, const double* U, const double* Lam,
                                const double* Ftilde, void* stream);

/* Source term s of Eq. (hdg_ls3): the residual's w rows get -(phi_i, s_h)_K =
 * -det J_K S_K,i (orthonormal basis), s_h the L2 projection of s with
 * coefficients S (DEVICE [u_len], U's layout; only the w part is read, the
 * caller keeps it alive and unchanged while it is set).  s does not depend on
 * the state, so the Newton matrix is unchanged.  NULL removes it.  Used for
 * manufactured solutions.  HDG_EINVAL once a graph has been captured. */
hdg_status hdg_sys_set_source(hdg_sys* sys, const double* S);

/* Newton update on DEVICE vectors: U += dU [u_len], Lam += dLam [lam_len]. */
hdg_status hdg_newton_update(hdg_sys* sys, double* U, double* Lam, const double* dU, const double* dLam,
                             void* stream);

/* ||N_h||_2 of the state given to the last hdg_condense: the 2-norm of the
 * interior residual [N_q; N_w] and the two-sided trace residual together,
 * computed on the device; synchronises `stream`. */
hdg_status hdg_residual_norm(hdg_sys* sys, double* norm, void* stream);

/* Change the pseudo-time CFL number of a system (Sec. 3.3; <= 0: pure Newton)
 * for the following hdg_condense calls.  Not allowed while a captured graph
 * exists (HDG_EINVAL): the graph bakes the parameters in. */
hdg_status hdg_sys_set_cfl(hdg_sys* sys, double cfl);

/* The CFL law of Eq. (cfl), host only: for n <= n0,
 * CFL^n = c0 (3 (n/n0)^2 - 2 (n/n0)^3); afterwards
 * CFL^n = CFL^{n-1} (1 + c1 max(0, log(res_prev / res_cur))) with res_prev =
 * ||N^{n-1}||, res_cur = ||N^n||.  The paper's values: c0 = 1e6, c1 = 1e3,
 * n0 = 4.  Returns a negative value for n < 0, n0 < 1 or non-positive norms. */
double hdg_cfl_law(int32_t n, double c0, double c1, int32_t n0, double cfl_prev, double res_prev, double res_cur);

/* Allocation-free condensation.  The paper has no counterpart: this is an
 * interface for callers that cannot allocate device memory when they call --
 * serving loops with a latency budget (cudaMalloc and cudaFree can synchronise
 * the whole device and take unbounded time) and hosts whose device memory is
 * owned by another allocator or fixed at start-up.  It does the work of
 * hdg_condense for a system without a source term (same kernels, bitwise the
 * same results; a source set on some system with hdg_sys_set_source is not
 * seen here: s = 0) on the mesh's device, enqueued on `stream`, but writes to
 * CALLER device buffers: X [x_len],
 * K_vals [k_len], E [lam_len], res_u [u_len], res_lam [lam_len],
 * elem_status [n_elem] (sizes from hdg_mesh_sizes; U, Lam as in hdg_condense).
 * It calls no cudaMalloc, cudaFree or other allocating routine: the per-face
 * work space lives in one fixed 64 MiB device array inside the library, which
 * every GPU that loads the library holds until the process exits.
 *   - Meshes whose work space is larger than 64 MiB are rejected with
 *     HDG_EINVAL and a message naming the size (per face: 4 bytes + 8 (4(p_e+1))^2
 *     + 16 * 4(p_e+1) bytes, each part of the array rounded up to 256 bytes;
 *     about 19,000 faces at p_e = 4, 29,000 at p_e = 3).  Only the FP64 Euler
 *     path is supported (else HDG_ENOTSUP).
 *   - The first call on a device resolves the array's device address
 *     (cudaGetSymbolAddress, with that device made current) and keeps it for
 *     the life of the process; make that first call before any stream capture
 *     on the device.  A cudaDeviceReset of that device invalidates the kept
 *     address: the call is not supported after one.
 *   - The mesh's device is made current for the call; the calling thread's
 *     current device is restored before it returns.
 *   - Every call shares the one array, which keeps the last call's contents;
 *     the call clears the part that must start at zero (the arrival counters)
 *     on `stream` before its kernels.  Calls whose work overlaps on the GPU
 *     (other streams, other host threads, or another mesh) race on the array
 *     and give wrong results: serialise them. */
hdg_status hdg_condense_noalloc(const hdg_mesh* mesh, const hdg_params* params, const double* U,
                                const double* Lam, double* X, double* K_vals, double* E, double* res_u,
                                double* res_lam, int32_t* elem_status, void* stream);

/* Diagnostic, host only (no device needed): copy one of the library's own
 * quadrature/basis tables into out[cap]; returns its length or -1.
 * which: 0 volume weights [(p+2)^2], 1 basis values, 2 d/dxi, 3 d/deta
 * [(p+2)^2][n_p] at the volume points (xi-major collapsed ordering), 4 edge
 * points s, 5 edge weights [p_e+2], 6 trace basis [p_e+2][p_e+1], 7 basis of
 * degree p on local face lf at the edge points, flip = 1 if the face runs
 * from the higher to the lower vertex id [p_e+2][n_p], 8 reference stiffness
 * parts [3][n_p][n_p] (sum_q w_q of dxi phi_i dxi phi_j, dxi phi_i deta phi_j +
 * deta phi_i dxi phi_j, deta phi_i deta phi_j). */
int hdg_debug_tables(int which, int p, int pe, int lf, int flip, double* out, int cap);

#ifdef __cplusplus
}
#endif

#endif  // HDG_H_
