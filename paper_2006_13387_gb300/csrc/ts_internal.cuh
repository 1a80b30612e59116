// Internal declarations of libtopsolve (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <memory>
#include <vector>

#include "../../include/topsolve.h"

#define TS_MAXMODES 16   // hard upper bound for ts_options.max_modes
#define TS_EL_MAXMODES 48  // modes per coarse node of the elasticity coarse space (M_EE, coarse_method 2)
#define TS_VEC_KIND 8      // cdof_kind of an M_EE mode (both components)
// Element stiffness matrices (E = 1) live in constant memory, one slot per
// distinct (dimension, nu) among the live designs: 8 slots of 24 x 24.
#define TS_KE_SLOTS 8
#define TS_KE_SIZE 576
#define TS_LANCZOS_MAX 96
#define TS_RAND_MAX 31      // random loads per heat problem of the randomized basis (+1 constant <= 32)
#define TS_OC_STEPS 80      // bisection steps of the OC multiplier (log scale, 80 decades)

// ---------------------------------------------------------------------------
// geometry shared by host and device (POD, passed to kernels by value)
// ---------------------------------------------------------------------------
struct Geom {
  int dim, nx, ny, nz;
  int n[3];        // elements per axis
  int H[3];        // coarse block width per axis
  int ov;          // overlap delta (-1: omega geometry)
  int nsub[3];     // subdomains per axis
  int ncn[3];      // coarse nodes per axis (= blocks + 1)
  int ke;          // slot of the element stiffness in constant memory
  int64_t n_nodes, ndof, n_el;
  __host__ __device__ int nn(int a) const { return n[a] + 1; }
};

// Per-axis subdomain tables: node range [lo, hi] (inclusive, strict interior
// plus domain-boundary nodes) and the element range [elo, ehi).  cand[i] holds
// up to two subdomain axis-indices whose node range contains node coordinate i.
struct AxisTables {
  int* sub_lo[3];
  int* sub_hi[3];
  int* sub_elo[3];
  int* sub_ehi[3];
  int2* cand[3];
};

// Block-line factor of one SPD/indefinite block-tridiagonal matrix:
// nb diagonal blocks of width w; storage per block k at off + k*(2*w*w + w):
//   W_k = L_k^{-1} (w*w, row-major, unit lower), G_k (w*w, row-major; block
//   row k couples to k-1, G_0 unused), dinv_k (w).
struct BLDesc {
  int w, nb;     // line width (unknowns per line) and number of lines
  int64_t coff;  // offset of the subdomain's per-line solve blocks in the level-1 pool
};

// One heat eigenproblem: coarse node l, component c (c = -1 never stored)
struct HeatProb {
  int l;          // coarse node (linear index)
  int c;          // displacement component whose Dirichlet set applies
  int lo[3];      // closed omega box node range [lo, hi]
  int hi[3];
  int nloc;       // number of nodes in the closed box
  int w, nb;      // block-line shape (w nodes per line/plane, nb lines)
  int64_t fac_off;   // offset of its (K + sigma M) factor in the heat pool
  int64_t vec_off;   // offset of its selected eigenvectors [max_modes][nloc]
  int dedup_of;      // index of an identical earlier problem, or -1
};

struct CoarseNodeInfo {
  int idx[3];        // coarse grid index
  int first_dof;     // first coarse DOF of this node
  int nmodes[3];     // heat modes per component (0 if dropped)
  int prob[3];       // heat problem id per component (-1 if dropped)
  int nrot;          // rotation DOFs (0, 1 or 3)
  int ndof;          // total coarse DOFs of this node
  int lo[3], hi[3];  // closed omega box (node range) of this coarse node
  int nbox;          // nodes in that box
  int64_t boff;      // offset of its basis block B_l [nbox][dim][ndof] in the pool
  int nh;            // rows of W: heat DOFs (sum of nmodes, numbered first) + 2 per M_EE mode
  int64_t woff;      // offset of its hat-weighted eigenvectors chi_l psi [nh][round_up(nbox, 4)]
  int nvec;          // M_EE modes (both components; numbered after the heat DOFs, W rows x then y)
};

struct DevScalars;  // PCG scalars on the device (ts_pcg.cu)

// A context runs its work on a private non-blocking stream (so that it can be
// captured into CUDA graphs even when the caller uses the legacy default
// stream) and orders it after / before the caller's stream with events.
struct Server;  // request loop of ts_submit / ts_poll (ts_serve.cu)

// A context made by ts_ctx_create, or the private execution lane of one
// handle (parent set): every handle runs on its own streams, so solves of
// different handles issued from different host threads (the request loop's
// workers) overlap on the device.
struct ts_ctx_s {
  cudaStream_t stream = nullptr;       // private work stream
  cudaStream_t user_stream = nullptr;  // caller's stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // second work stream: the coarse correction runs on it while the level-1
  // solves run on `stream` (the two parts of the additive preconditioner are
  // independent); joined before the prolongation
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int device = 0;
  int n_sm = 1;                        // streaming multiprocessors of the device
  int prio_hi = 0;                     // greatest launch priority of the device
  ts_ctx_s* parent = nullptr;          // lanes: the user's context
  std::mutex err_mu;
  std::string err;
  std::atomic<int64_t> launches{0};    // kernels launched (graph nodes included); user contexts only
  Server* server = nullptr;            // request loop, started by the first ts_submit
  int slots = 4;                       // concurrent requests of the request loop
};

// One task of a coarse solve stage of the block path (TS_NB columns):
// out = base + sgn (op(M0) v0 + op(M1) v1) with FP32 matrices, FP32 input
// vectors [n][TS_NB] and products, the result in FP64 (out) and FP32 (out32).
// The matrices are addressed through tensor maps of the three stored arrays
// (map 0: Ainv, 1: Qlt, 2: Qrt; [lines][cw][cw] FP32) and a line index.
struct BcrTaskB {
  double* out;
  float* out32;
  const double* base;   // may be null
  const float* v0;
  const float* v1;
  int m0_map, m0_line;  // M0
  int m1_map, m1_line;  // M1 (map -1: none)
  int rows, n0, n1;
  int trans;            // 0: rows of M times v;  1: M^T v
  double sgn;
};

struct BcrTask;    // one GEMV task of a coarse solve stage, FP64 matrices (ts_cfactor.cu)
struct BcrTask32;  // the same with FP32 matrices

struct NdData;                 // nested-dissection factor of K_0 (ts_cnd.cu)
constexpr int ND_AUTO_LINES = 48;  // coarse_layout 0 takes nested dissection from this many coarse lines

struct ts_handle_s {
  ts_ctx ctx;                   // the handle's execution lane
  ts_ctx root = nullptr;        // the user's context it was created on
  std::vector<uint8_t> fm_h;    // free mask (host), kept for density updates
  int ke_slot = -1;             // element stiffness slot held (g.ke), or -1
  int64_t bytes = 0;            // device memory owned
  bool capturing = false;       // launches are being captured into a graph
  int64_t cap_launches = 0;
  Geom g;
  ts_options opt;
  double E0, Emin, p, nu;
  // device data ------------------------------------------------------------
  double* E = nullptr;          // [n_el]
  double* kst = nullptr;        // 2D: [36][n_nodes] masked nodal stencil of K
  uint8_t* freemask = nullptr;  // [ndof]
  AxisTables ax{};
  std::vector<void*> owned;     // everything cudaMalloc'd by this handle
  std::vector<void*> scratch;   // setup-only buffers (stream-ordered, freed when the setup ends)
  int64_t scratch_bytes = 0;    // scratch held now
  int64_t scratch_peak = 0;     // most scratch held at once by the last setup
  // level 1
  int nsub = 0;
  BLDesc* sub_desc = nullptr;   // [nsub]
  std::vector<BLDesc> sub_desc_h;
  double* pv64 = nullptr;       // per line: S_k^{-1} (M form) + coupling stencils, FP64 path
  float* pv32 = nullptr;        // per line: V_k (packed Gram form) + coupling stencils, mixed
  int64_t pv_len = 0;
  int pv_stride_max = 0;        // largest per-line block
  int lv1_max_nel = 0;          // largest subdomain element box
  int64_t* zloc_off = nullptr;  // [nsub] offset of the local solution in zloc
  std::vector<int64_t> zloc_off_h;
  double* zloc = nullptr;       // local solutions (FP64 path)
  float* zloc32 = nullptr;      // local solutions (FP32 path)
  int64_t zloc_len = 0;
  int max_w = 0;
  // coarse
  int n_cnodes = 0;
  CoarseNodeInfo* cn = nullptr;   // [n_cnodes]
  std::vector<CoarseNodeInfo> cn_h;
  int n_hprob = 0;
  HeatProb* hp = nullptr;         // [n_hprob]
  std::vector<HeatProb> hp_h;
  std::vector<int> hp_inertia_h;  // [n_hprob] eigenvalues below tau of the last build (distinct problems)
  size_t heat_smem = 0;           // dynamic shared memory of a k_heat_eig launch
  // rebuild policy of density updates (ts_update_density)
  int precond_age = 0;            // density updates applied since the preconditioner was built
  int iters_ref = -1;             // iterations of the first solve after the last build (-1: none yet)
  bool rebuild_pending = false;   // a solve exceeded rebuild_factor x iters_ref: rebuild at the next update
  int* hp_count = nullptr;        // [n_hprob] eigenvalues below tau
  int* hp_found = nullptr;        // [n_hprob] converged Ritz pairs stored
  double* hp_lambda = nullptr;    // [n_hprob][lam_stride]
  int lam_stride = TS_MAXMODES;   // TS_EL_MAXMODES for the M_EE problems
  double* heat_fac = nullptr;     // heat (K + sigma M) factors
  double* psi = nullptr;          // eigenvectors
  double* lanczos_ws = nullptr;   // Lanczos workspace
  int64_t lanczos_ws_per = 0;
  int nc = 0;                     // coarse dimension
  int* cdof_node = nullptr;       // [nc] coarse node of each coarse DOF
  int* cdof_kind = nullptr;       // [nc] 0..dim-1 heat component, dim.. rotation axis
  int* cdof_mode = nullptr;       // [nc] mode index within (node, component)
  // Galerkin K_0, assembled straight into the line blocks of its factor
  // (setup only): per non-empty coarse line q its diagonal block and its
  // coupling to line q + 1, each cw x cw row-major (zero padded)
  std::vector<int> cl_off, cl_wid, cl_line;  // non-empty lines: first DOF, width, coarse line index
  double* K0A = nullptr;          // [n_lines][cw][cw] diagonal blocks
  double* K0C = nullptr;          // [n_lines - 1][cw][cw] couplings A_{q,q+1}
  int K0_ld = 0;                  // padded length of the coarse vectors
  double* r0 = nullptr;           // [nc]
  double* u0 = nullptr;           // [nc]
  int cap_hits = 0, eig_unconv = 0;
  double* rho = nullptr;          // [n_el] the design's densities
  double* to_ws = nullptr;        // workspace of ts_sensitivity / ts_oc_update
  double* dc_tmp = nullptr;       // [2 n_el] sensitivities and densities of the kernel timings
  int64_t to_ws_len = 0;
  double heat_ms = 0.0;           // heat eigenproblem launch of the last setup (CUDA events)
  double heat_flops = 0.0;        // its FP64 operations (counted by the kernel)
  double cfac_ms = 0.0;           // K_0 factor of the last setup (CUDA events)
  double cfac_flops = 0.0;        // its FP64 operations (GEMM tiles counted by the kernel)
  double cfac_method_flops = 0.0; // FP64 operations of the block-tridiagonal Cholesky of K_0 by lines
  unsigned long long* cfac_cnt = nullptr;  // device counter of the factor's GEMM FLOPs
  cudaEvent_t cfac_ev[2] = {nullptr, nullptr};
  // PCG workspace (per rhs, allocated lazily)
  double *x = nullptr, *r = nullptr, *z = nullptr, *zold = nullptr, *pvec = nullptr, *q = nullptr,
         *fvec = nullptr;
  double* partials = nullptr;   // reduction partials
  double* partials_s = nullptr; // SpMV dot partials inside the PCG iteration
  double* partials_xr = nullptr;// x/r update partials inside the PCG iteration
  unsigned* counters = nullptr; // last-block counters of the PCG iteration kernels
  float* r32 = nullptr;         // FP32 copy of the preconditioner's input (mixed precision)
  double* pvec2 = nullptr;      // second search-direction buffer (fused update, 2D)
  float* u0f = nullptr;         // FP32 copy of the coarse solution (mixed precision)
  DevScalars* sc = nullptr;
  int* dstatus = nullptr;       // device error word
  int* done_flag = nullptr;     // PCG stop flag read by every iteration kernel (nullptr outside PCG)
  bool pdl = false;             // launching the PCG iteration: chain its kernels programmatically
  int prio = 0;                 // launch priority of the next launches (0: the stream's)
  double setup_ms = 0;
  int hist_cap = 0;
  double* alpha_hist = nullptr;
  double* beta_hist = nullptr;
  int* done_dev = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int* chunk_flag_h = nullptr;                      // pinned stop flags of two queued chunks
  cudaEvent_t chunk_ev[2] = {nullptr, nullptr};     // recorded after each chunk's flag copy
  double* forig = nullptr;   // right-hand side of the current solve
  double* xacc = nullptr;    // solution accumulated over refinement rounds
  double* rtrue = nullptr;   // double-double true residual of a round
  int coarse_dropped = 0;
  int64_t graph_kernels = 0; // kernel nodes in the captured PCG chunk
  // coarse basis blocks and line structure of K_0
  int line_axis = 0, n_lines = 0, max_cdof = 0;
  std::vector<int> line_off_h;   // first coarse DOF of each line (+ total)
  int64_t B_len = 0;
  double* B64 = nullptr;         // chi_l * (psi | rotation) per omega box node, FP64
  int64_t W_len = 0;
  size_t restrict_smem = 0;      // shared memory of a restriction CTA
  double* W64 = nullptr;         // chi_l psi per heat DOF over its box, FP64 (FP64 path)
  float* W32 = nullptr;          // the same in FP32 (mixed precision)
  // block cyclic reduction factor of K_0 (ts_cfactor.cu)
  bool coarse_blockline = false; // more than one coarse line
  // mixed path: the coarse solve applies the FP64 stage matrices (no block
  // path); set by coarse_needs_fp64
  bool coarse64 = false;
  int cw = 0;                    // padded line width (multiple of 32)
  int bcr_lines = 0;             // non-empty coarse lines
  double* bcr_Ainv = nullptr;    // per line: inverse of its reduced diagonal block
  double* bcr_Qlt = nullptr;     // per eliminated line: C_l Ainv_j
  double* bcr_Qrt = nullptr;     // per eliminated line: C_j^T Ainv_j
  double* bcr_ys = nullptr;      // [nc] forward results of eliminated lines
  double* bcr_bs = nullptr;      // [nc] reduced right-hand sides
  BcrTask* bcr_tasks = nullptr;
  BcrTask32* bcr_tasks32 = nullptr;  // mixed precision: FP32 stage matrices
  size_t bcr_smem = 0;
  bool bcr_stage_mats = false;       // stage CTAs copy their matrix slices to shared memory
  int2* bcr_ctas = nullptr;
  std::vector<int> bcr_stage_task, bcr_stage_cta;  // per solve stage: first task / CTA (+ end)
  double bcr_fmas = 0.0;         // FMAs of one coarse solve
  std::shared_ptr<NdData> nd;    // set: K_0 is factored by nested dissection (ts_cnd.cu), not by lines
  // block path (TS_NB columns): coarse vectors [nc][TS_NB] and the stage tasks on them
  double* r0b = nullptr;
  double* u0b = nullptr;
  float* u0fb = nullptr;
  double* bcr_ysb = nullptr;
  double* bcr_bsb = nullptr;
  float* r0b32 = nullptr;                 // FP32 copies of r0b, ysb, bsb (the stage inputs)
  float* bcr_ysb32 = nullptr;
  float* bcr_bsb32 = nullptr;
  BcrTaskB* bcr_btasks = nullptr;
  // tensor maps (CUtensorMap, 128 bytes each) of the FP32 stage arrays for
  // the block stages: [0..2] row tiles (128 columns x 32 rows), [3..5]
  // transposed tiles (32 columns x 128 rows)
  alignas(64) unsigned char bcr_tmaps[6][128];
  int2* bcr_bctas = nullptr;              // CTAs of the block stages (32 outputs each)
  std::vector<int> bcr_bstage_cta;        // per block stage: first CTA (+ end)
  // block PCG state (ts_bpcg.cu), allocated by the first block solve
  double *xb = nullptr, *rb = nullptr, *zb = nullptr, *zoldb = nullptr, *qb = nullptr, *fb = nullptr;
  double* pb[2] = {nullptr, nullptr};
  float* r32b = nullptr;        // [ndof][TS_NB]
  float* zloc32b = nullptr;     // [local][TS_NB]
  double* bpart_s = nullptr;    // SpMV partials [blocks][TS_NB]
  double* bpart_xr = nullptr;   // x/r update partials [blocks][3][TS_NB]
  double* bpart_p = nullptr;    // prolongation partials [blocks][TS_NB]
  unsigned* bcounters = nullptr;
  struct BScalars* bsc = nullptr;
  double* bhist_a = nullptr;    // [hist_cap][TS_NB]
  double* bhist_b = nullptr;
  int* bdone = nullptr;
  cudaGraphExec_t bgraph_exec = nullptr;
  int64_t bgraph_kernels = 0;
  double* red2 = nullptr;    // two reduction results
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
#define TS_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      throw TsError(TS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    }                                                                                    \
  } while (0)

struct TsError {
  ts_status st;
  std::string msg;
  TsError(ts_status s, std::string m) : st(s), msg(std::move(m)) {}
};

template <class T>
T* dalloc(ts_handle h, size_t n) {
  void* p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc(&p, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw TsError(TS_ERR_OOM, "cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes failed");
  }
  h->owned.push_back(p);
  h->bytes += (int64_t)(n * sizeof(T));
  return static_cast<T*>(p);
}

// The library's stream-ordered memory pool on a device (created on first
// use; it keeps the memory freed into it for the next setups instead of
// returning it to the driver at every synchronisation), and its memory held
// but not in use (ts_api.cu).
cudaMemPool_t ts_scratch_pool(int device);
int64_t ts_scratch_pool_idle(int device);

// Setup-only device buffer, allocated in stream order on the handle's work
// stream from the library's pool and released by sfree_all() when the setup
// ends, so that a design keeps only what its solves read.
template <class T>
T* salloc(ts_handle h, size_t n) {
  void* p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMallocFromPoolAsync(&p, n * sizeof(T), ts_scratch_pool(h->ctx->device), h->ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw TsError(TS_ERR_OOM, "cudaMallocAsync of " + std::to_string(n * sizeof(T)) + " bytes failed");
  }
  h->scratch.push_back(p);
  h->scratch_bytes += (int64_t)(n * sizeof(T));
  h->scratch_peak = std::max(h->scratch_peak, h->scratch_bytes);
  return static_cast<T*>(p);
}

// Releases every setup-only buffer after the work queued on the handle's
// stream so far.
inline void sfree_all(ts_handle h) {
  for (void* p : h->scratch) cudaFreeAsync(p, h->ctx->stream);
  h->scratch.clear();
  h->scratch_bytes = 0;
}

template <class T>
T* dupload(ts_handle h, const std::vector<T>& v) {
  T* p = dalloc<T>(h, v.size());
  if (!v.empty())
    TS_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->ctx->stream));
  return p;
}

// setup-only copy of a host array (freed with the setup scratch)
template <class T>
T* supload(ts_handle h, const std::vector<T>& v) {
  T* p = salloc<T>(h, v.size());
  if (!v.empty())
    TS_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->ctx->stream));
  return p;
}

inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Lets a kernel take as much dynamic shared memory as the device allows next
// to its static shared memory, and returns that limit (bytes).  Every call
// sets the same value, so that setups and solves of different designs on
// different host threads (the request loop) never lower the limit under
// another's launch; a launch still takes only the memory it asks for.
template <class K>
inline size_t ts_allow_dynamic_smem(K kernel, int device) {
  cudaFuncAttributes a;
  TS_CUDA(cudaFuncGetAttributes(&a, (const void*)kernel));
  int optin = 0;
  TS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  const int lim = optin - (int)a.sharedSizeBytes;
  TS_CUDA(cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  return (size_t)lim;
}

// counts kernel launches issued for a handle (reported by ts_ctx_kernel_launches
// of its user context; launches captured into a graph are counted apart)
inline void tsl(ts_handle h, int64_t n = 1) {
  if (h->capturing)
    h->cap_launches += n;
  else
    h->root->launches += n;
}

// records the reason of a failure on a context (and on the user's context of
// a lane); thread-safe
void ts_set_error(ts_ctx c, const std::string& m);

// Runs an entry point's body: a TsError or std::exception thrown inside
// becomes its status and the reason recorded on ctx, so that nothing is thrown
// across the C ABI.
template <class F>
ts_status ts_guarded(ts_ctx ctx, F&& f) {
  try {
    return f();
  } catch (const TsError& e) {
    ts_set_error(ctx, e.msg);
    return e.st;
  } catch (const std::bad_alloc&) {
    ts_set_error(ctx, "host allocation failed");
    return TS_ERR_OOM;
  } catch (const std::exception& e) {
    ts_set_error(ctx, e.what());
    return TS_ERR_INVALID;
  } catch (...) {
    ts_set_error(ctx, "unknown exception");
    return TS_ERR_INVALID;
  }
}

// design rebuild for new densities and one solve on a handle's lane (ts_api.cu)
void ts_rebuild_density(ts_handle h, const double* rho);
void ts_update_by_policy(ts_handle h, const double* rho);  // ts_update_density's rebuild policy
ts_status ts_solve_impl(ts_handle h, const double* f, double* u, int nrhs, double rtol, ts_stats* stats,
                        cudaEvent_t after);
// request loop (ts_serve.cu): stops and joins the workers of a user context
// (requests still queued end with TS_ERR_INVALID); whether a handle has a
// queued or running request
void stop_server(ts_ctx ctx);
bool server_holds(ts_ctx ctx, ts_handle h);

// 16-byte vector of FP32 / FP64 values and its dot product with 16 aligned bytes
template <class TF>
struct Vec16;
template <>
struct Vec16<float> {
  using T = float4;
  static constexpr int N = 4;
  __device__ static float dot(const float4 a, const float4 y) { return a.x * y.x + a.y * y.y + a.z * y.z + a.w * y.w; }
};
template <>
struct Vec16<double> {
  using T = double2;
  static constexpr int N = 2;
  __device__ static double dot(const double2 a, const double2 y) { return a.x * y.x + a.y * y.y; }
};

// Programmatic dependent launch.  A kernel launched with the programmatic
// stream-serialisation attribute may be scheduled before its predecessor on
// the stream has finished: every kernel of the PCG iteration waits for its
// predecessor's results (pdl_wait) before it reads anything that kernel
// wrote, and lets its own successor be scheduled (pdl_trigger) once a block
// has done its main work, so that the successor's waiting blocks do not take
// the resources the current kernel still needs.  Both instructions are
// no-ops in an ordinary launch.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// launch with the programmatic attribute when pdl is set
template <typename... KArgs, typename... Args>
inline void ts_launch(ts_handle h, bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                      cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[2];
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  int na = 0;
  if (pdl) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  if (h->prio != 0) {
    attr[na].id = cudaLaunchAttributePriority;
    attr[na].val.priority = h->prio;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  tsl(h);
  TS_CUDA(cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...));
}

// element stiffness matrices computed on the host (ts_fem.cu)
void ts_element_matrices(int dim, double nu, std::vector<double>& KE);
// element stiffness slots (ts_fem.cu): the slot for the handle's (dim, nu),
// uploaded to every translation unit's table on first use; released when
// the handle is freed
void ts_ke_acquire(ts_handle h);
void ts_ke_release(ts_handle h);
void upload_KE_local(int slot, const std::vector<double>& KE);
void upload_KE_coarse(int slot, const std::vector<double>& KE);

// kernels / launchers (ts_fem.cu)
void launch_simp(ts_handle h, const double* rho, double* E = nullptr);  // E: output (default h->E)
bool heat_counts_changed(ts_handle h, const double* E);  // ts_coarse.cu
void launch_stencil(ts_handle h, double* St);
void launch_sensitivity(ts_handle h, const double* u, double* dc, double** out);   // Eq. 1003
void launch_oc_update(ts_handle h, const double* dc, double volfrac, double move, double* rho_new);
// y = K x; optional per-block partials of dotvec.y; inside the PCG iteration
// (S, counter given) the last block turns them into alpha
void launch_spmv(ts_handle h, const double* x, double* y, double* dot_partial, const double* dotvec,
                 DevScalars* S = nullptr, unsigned* counter = nullptr);
void launch_spmv_fused_p(ts_handle h, const double* z, const double* p_old, double* p_new, double* z_old,
                         double* q, double* partial, DevScalars* S, unsigned* counter);
int spmv_blocks(const Geom& g);  // blocks (and dot partials) of launch_spmv
int node_blocks(const Geom& g);  // blocks of one-thread-per-node kernels (256 threads)
// level 1 (ts_local.cu)
void build_level1(ts_handle h);
void launch_local_solve(ts_handle h, const double* r);
// coarse (ts_coarse.cu)
void build_coarse(ts_handle h, const std::vector<uint8_t>& fm_h);
void build_coarse_basis(ts_handle h);   // ts_cbasis.cu
// Whether the mixed path must keep the coarse solve in FP64: the M_EE
// coarse space above contrast 1e6, whose diagonally scaled K_0 reaches a
// condition near the contrast itself (rigid motions of stiff islands cut by
// several partition-of-unity functions), beyond what FP32 copies of the
// stage matrices resolve.
bool coarse_needs_fp64(ts_handle h);
void build_coarse_factor(ts_handle h);  // ts_cfactor.cu
bool coarse_uses_nd(ts_handle h);            // ts_cnd.cu: the nested-dissection factor applies
void build_coarse_factor_nd(ts_handle h);
void launch_coarse_solve_nd(ts_handle h);    // u0 = K_0^{-1} r0 (one column)
void launch_bcoarse_solve_nd(ts_handle h);   // the block path's TS_NB columns
// the line blocks of K_0 (h->cl_*, h->cw, h->coarse_blockline): one line for
// small coarse spaces (the dense inverse), else the non-empty coarse lines
void coarse_line_layout(ts_handle h);   // ts_cfactor.cu
void launch_coarse_solve(ts_handle h);  // u0 = K_0^{-1} r0 (ts_cfactor.cu)
void upload_KE_cbasis(int slot, const std::vector<double>& KE);
void launch_coarse_apply(ts_handle h, const double* r);
// prolongation z = sum R_i^T zloc_i + R_0^T u0 (+ optional parts), ts_local.cu
// Inside the PCG iteration the prolongation's last block runs the
// convergence test (from the x/r update's partials) and forms beta.
struct PcgTail {
  DevScalars* S = nullptr;
  unsigned* counter = nullptr;
  const double* xr_partials = nullptr;  // 3 per block of the x/r update
  int n_xr = 0;
};
void launch_prolong(ts_handle h, double* z, int which, double* dot_partials, const double* dotvec1,
                    const double* dotvec2, PcgTail tail = PcgTail{});
