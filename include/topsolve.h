/*
 * topsolve -- C ABI of the GB300 (sm_103a) state solver for SIMP linear
 * elasticity, K(rho) u = f, by PCG preconditioned with the two-level
 * overlapping additive Schwarz method M_EH(+Rot) of Zambrano, Serrano,
 * Lazarov & Galvis (arXiv 2006.13387).
 *
 *   K(rho) u = f ........................................ Eq. 2 (eq1002)
 *   E_e = Emin + rho_e^p (E0 - Emin) .................... Eq. 4 (eq1002a1)
 *   elasticity, plane stress Q4 / Hex8 weak form ........ Sec. 1.1, Eqs. 6-9
 *   M^{-1} = sum_i R_i^T K_i^{-1} R_i  (level 1) ........ Eq. localproblemsE
 *          + [R_H(+Rot)] K_{E,0}^{-1} [R_H(+Rot)]^T ..... Eqs. juan001/juan002
 *   coarse space from heat eigenproblems per omega_l .... Sec. 4.1, Eq.
 *     juaneheateigenproblem, V_{0,H}; rotations ......... Sec. 4.2
 *   PCG with relative-residual stop ..................... Sec. 2, Sec. 5
 *
 * Conventions shared by every entry point
 *   - 2D: nodes (i, j), id = j*(nx+1) + i; 3D: id = (k*(ny+1) + j)*(nx+1) + i.
 *     DOF = dim*node + c (interleaved).  Elements row-major (x fastest).
 *     Unit element size.
 *   - Vectors f and u are FP64, [nrhs][ndof] row-major, zero at Dirichlet DOFs
 *     (f's Dirichlet entries are ignored; u's are written as 0).
 *   - Every call returns a ts_status; nothing is thrown or aborted across the
 *     ABI.  A failed call leaves no partial object behind.  ts_last_error()
 *     gives a one-line reason for the last failure on that context.
 *   - Device pointers (when ts_options.mem_is_device = 1) must be cudaMalloc'd
 *     (or torch) memory on the context's device; work is ordered on the
 *     context's stream.
 */
#ifndef TOPSOLVE_H
#define TOPSOLVE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ts_ctx_s* ts_ctx;
typedef struct ts_handle_s* ts_handle;
typedef int64_t ts_ticket;  /* a request of the request loop (ts_submit) */

typedef enum {
  TS_OK = 0,
  TS_PENDING = 1,
  TS_NOT_CONVERGED = 2,     /* max_iter reached; u holds the last iterate */
  TS_ERR_INVALID = -1,      /* bad argument; nothing was changed */
  TS_ERR_OOM = -2,          /* device allocation failed */
  TS_ERR_CUDA = -3,         /* a CUDA call failed (message in ts_last_error) */
  TS_ERR_BREAKDOWN = -4,    /* PCG p^T K p <= 0 or NaN */
  TS_ERR_TIMEOUT = -5,
  TS_ERR_NOT_SPD = -6,      /* a local or coarse factor met a non-positive pivot */
  TS_ERR_BUSY = -7
} ts_status;

enum { TS_FP64 = 0, TS_MIXED_FP32 = 1, TS_MIXED_TF32 = 2, TS_MIXED_3XTF32 = 3 };

typedef struct {
  int dim;          /* 2 (Q4, plane stress) or 3 (Hex8) */
  int nx, ny, nz;   /* elements per axis (nz ignored in 2D) */
  int blk_x, blk_y, blk_z;  /* coarse block D_i size in elements; must divide n */
  int overlap;      /* delta: D'_i = D_i grown by this many element layers
                       (box distance, clipped); -1 = D'_i = omega_i (Sec. 5).
                       Must satisfy 0 <= 2*overlap < blk (or -1). */
} ts_mesh;

typedef struct {
  int64_t n;            /* number of Dirichlet DOFs */
  const int64_t* dofs;  /* HOST array of DOF ids with u = 0 (any order, duplicates ok) */
} ts_bcs;

typedef struct {
  int precision;      /* TS_FP64: everything FP64, plain PCG.
                         TS_MIXED_FP32: level-1 local factors stored/applied in
                         FP32 inside an FP64 flexible PCG (FCG(1) beta); SpMV,
                         dots, updates and the coarse factor stay FP64, the
                         coarse solve stages and the coarse basis rows are
                         applied in FP32.
                         TS_MIXED_TF32 / TS_MIXED_3XTF32: as TS_MIXED_FP32;
                         a 2D solve of several right-hand sides (the block
                         path, see ts_solve) applies the level-1 factors on
                         the tensor cores, one TF32 product per tile or the
                         3xTF32 split (near FP32 accuracy); TS_MIXED_FP32
                         uses the 3xTF32 split there too.  One right-hand
                         side runs the FP32 sweeps in every mixed mode. */
  double tau_scale;   /* eigenvalue threshold tau = tau_scale / H^2 (default 2) */
  int max_modes;      /* cap on heat modes per (omega_l, component), 1..16,
                         default 16: the threshold tau picks the modes and
                         the cap only bounds storage (Sec. 4.1) */
  int rotations;      /* 1: M_EH+Rot (default); 0: M_EH */
  int coarse;         /* 1: two-level (default); 0: level 1 only */
  int max_iter;       /* default 5000 */
  int warm_start;     /* 1: u is read as the initial iterate */
  int mem_is_device;  /* 1: rho, f, u are device pointers; 0: host pointers */
  double energy_tol;  /* relative K-norm error target of the stopping estimate;
                         < 0 means 0.1*rtol, 0 disables it */
  int refine;         /* refinement rounds after the first PCG (default 0):
                         the true residual f - K u is formed in double-double
                         arithmetic and K d = r solved to 1e-3; u += d.  Stops
                         early once d^T r <= energy_tol^2 f^T u.  0 disables. */
  int coarse_layout;  /* K_0 factor: 0 = automatic (dense up to 2048 coarse DOFs,
                         block cyclic reduction over coarse lines up to 47
                         lines, nested dissection of the coarse grid from 48),
                         1 = dense, 2 = block cyclic reduction over coarse
                         lines, 3 = nested dissection (multifrontal: the
                         coarse grid split recursively by layers of coarse
                         nodes, dense fronts) */
  int coarse_method;  /* coarse basis: 0 = eigenpairs of the local heat
                         problems (Sec. 4.1, default); 1 = the randomized
                         basis of the paper's randomized algorithm (M_EH+Rot;Rand):
                         zero-mean random loads (SplitMix64 counters: coarse
                         node << 40 | snapshot << 32 | box node), local
                         solves, the constant mode, Rayleigh-Ritz in that
                         span; the modes are the Ritz pairs below tau;
                         2 = the elasticity coarse space M_EE (Eq. 3001, 2D):
                         per coarse node the smallest eigenpairs of the
                         elasticity operator on omega_l against the
                         E-weighted vector mass, 3 per face-connected region
                         of elements with E_e >= sqrt(E0 Emin) (at least 3,
                         at most 48), no rotations; tau_scale, max_modes and
                         rotations do not apply, and a density update
                         rebuilds only by rebuild_factor.  Above contrast
                         E0/Emin = 1e6 the mixed precisions keep the M_EE
                         coarse solve in FP64 (its scaled K_0 is too
                         ill-conditioned for FP32 copies) and solve the
                         columns one at a time, without the block path */
  int rand_snapshots; /* random loads per problem with coarse_method 1:
                         max(rand_snapshots, selected modes + 5), at most
                         31; default 15 */
  int rebuild_policy; /* what ts_update_density / ts_submit_update rebuild
                         (Sec. 1.4: the preconditioner of an earlier design
                         step may serve later ones):
                         0 = everything, for every update;
                         1 (default) = the operator only (SIMP moduli and
                         stiffness stencil; the preconditioner of the last
                         build is kept), unless the eigenvalue threshold
                         would give another coarse dimension for the new
                         moduli (the total over the neighbourhoods of the
                         heat modes below tau changes), or a solve since the last
                         build took more than rebuild_factor times the
                         iterations of the first solve after that build;
                         then everything is rebuilt */
  double rebuild_factor; /* iteration-growth trigger of policy 1, >= 1
                            (default 1.5) */
} ts_options;

typedef struct {
  int iters;             /* PCG iterations over all rounds (SpMVs with the search direction) */
  int converged;         /* first PCG met rtol and the energy estimate */
  double rel_res;        /* ||f - K u|| / ||f||: the double-double true residual
                            when refinement ran, else the recursive residual */
  double energy_est;     /* delayed estimate of ||u* - u_k||_K^2 / f^T u_k */
  double cond_est;       /* Lanczos estimate of cond(M^{-1} K) */
  int coarse_dim;        /* dimension of the coarse space */
  int cap_hits;          /* neighbourhoods with more than max_modes modes below tau */
  int eig_unconverged;   /* eigenproblems whose Ritz pairs missed the tolerance */
  double setup_ms, solve_ms;
  int precision;
  int first_iters;       /* iterations of the first PCG alone */
  int refine_rounds;     /* refinement rounds run */
  int precond_age;       /* density updates applied since the preconditioner
                            was built (0: built for these densities) */
} ts_stats;

/* Fills *o with the defaults listed above. */
void ts_options_default(ts_options* o);

/* Creates a context bound to the current CUDA device and the given stream
 * (cudaStream_t cast to void*; NULL = the legacy default stream).  The
 * context owns no device memory itself. */
ts_status ts_ctx_create(void* cuda_stream, ts_ctx* out);
ts_status ts_ctx_destroy(ts_ctx ctx);
const char* ts_last_error(ts_ctx ctx);
/* Number of kernels this context has launched so far (graph-replayed kernel
 * nodes included); for launch accounting in benchmarks. */
int64_t ts_ctx_kernel_launches(ts_ctx ctx);

/* Builds the preconditioner for one design: SIMP moduli (Eq. 4), level-1
 * twisted block LU factors of every K_i (Eq. localproblemsE), heat
 * eigenproblems with the threshold count (Sec. 4.1), the coarse basis with
 * rotations (Sec. 4.2), K_0 = R_0 K R_0^T and its factor (Sec. 2.1).
 * rho: [n_el] in [0,1] (host or device per opts->mem_is_device).
 * Rejects (TS_ERR_INVALID) rho outside [0,1] or NaN, Emin <= 0, Emin >= E0,
 * nu outside (-1, 0.5), blocks not dividing the mesh, bad overlap, an empty
 * free-DOF set.  The handle owns all device buffers it creates. */
ts_status ts_setup(ts_ctx ctx, const ts_mesh* mesh, const double* rho, double E0, double Emin,
                   double p, double nu, const ts_bcs* bcs, const ts_options* opts, ts_handle* out);

/* Solves K(rho) u = f for nrhs right-hand sides (each with its own PCG),
 * stopping when ||r||/||f|| <= rtol and the energy estimate is met.
 * f, u: [nrhs][ndof] FP64 (host or device per the handle's options).
 * stats: array of nrhs entries or NULL.  Returns TS_NOT_CONVERGED if any
 * column hit max_iter, TS_ERR_BREAKDOWN on a non-positive curvature.
 * Block path: a 2D design in a mixed precision (refine = 0; not the M_EE
 * coarse space above contrast 1e6, see coarse_method) solves nrhs >= 2
 * columns in groups of 8 that share every kernel launch -- one flexible PCG
 * per column in lock step, the stiffness stencil, level-1 factors (applied
 * on the tensor cores, see ts_options.precision), coarse basis rows and
 * coarse factor read once per iteration for the group; a column that meets
 * its test stops (its iterate is kept) while the others go on.  solve_ms is
 * then the time of the whole group.  Other designs solve the columns one
 * after another. */
ts_status ts_solve(ts_handle h, const double* f, double* u, int nrhs, double rtol, ts_stats* stats);

/* Moves the design to new densities rho (the next optimisation step, Sec.
 * 1.4) by the handle's rebuild_policy.  Policy 0: rebuilds SIMP moduli,
 * level-1 factors, heat eigenproblems (the threshold may change the coarse
 * dimension), coarse basis, K_0 and its factor.  Policy 1 (default): updates
 * the operator (moduli, stiffness stencil) and keeps the preconditioner --
 * solves then run PCG on the new K with the earlier design's two-level
 * preconditioner, which is still SPD -- unless the coarse dimension the
 * threshold gives changes for the new moduli (the heat modes below tau,
 * counted by the inertia of K - tau M, the first step of the eigensolve,
 * summed over the neighbourhoods) or the iteration trigger of
 * ts_options.rebuild_factor fired since the last build; then everything is
 * rebuilt.  Mesh, Dirichlet set, material constants and options are kept.
 * A rebuild builds the new design beside the old one (twice the handle's
 * device memory meanwhile); on any failure the handle is unchanged.
 * ts_stats.precond_age of later solves counts the updates since the last
 * build.  Returns TS_ERR_BUSY while the request loop holds requests of this
 * handle.  A later solve with warm_start = 1 starts from the u the caller
 * passes (e.g. the previous step's solution). */
ts_status ts_update_density(ts_handle h, const double* rho);

/* Request loop (continuous batching of solves on one GPU).
 * Every handle runs on its own streams.  ts_submit queues a solve of handle h
 * (created on ctx) and returns at once with a ticket; worker threads of the
 * context (ts_ctx_set_slots, default 4) take the oldest request whose handle
 * is idle -- one request per handle at a time, in submission order -- so
 * requests of different handles run concurrently and their kernels overlap
 * on the device; a request arriving while others run starts as soon as a
 * slot (and, for ts_submit_update, the memory of the rebuild) is free.  The
 * request's device work is ordered after the caller's stream as it was at
 * submission.  f and u (and rho) must stay valid and unmodified until ts_poll
 * returns something other than TS_PENDING.  A request computes exactly what
 * ts_solve would compute for the same handle and inputs.
 * ts_submit_update first moves the design to rho (as ts_update_density);
 * it returns TS_ERR_BUSY if that rebuild can never fit in the device memory.
 * ts_poll: TS_PENDING while queued or running; otherwise the request's
 * status (that of ts_solve; the reason in ts_last_error(ctx)), its stats
 * (nrhs entries, if stats is non-NULL) and the ticket is released.  An
 * unknown ticket gives TS_ERR_INVALID.  ts_submit, ts_submit_update and
 * ts_poll are thread-safe on a context; while a handle has requests in the
 * loop, ts_solve, ts_update_density and ts_destroy on it return TS_ERR_BUSY.
 * ts_ctx_destroy waits for running requests and ends queued ones. */
ts_status ts_ctx_set_slots(ts_ctx ctx, int slots);  /* 1..64, before the first ts_submit */
ts_status ts_submit(ts_ctx ctx, ts_handle h, const double* f, double* u, int nrhs, double rtol, ts_ticket* ticket);
ts_status ts_submit_update(ts_ctx ctx, ts_handle h, const double* rho, const double* f, double* u, int nrhs,
                           double rtol, ts_ticket* ticket);
ts_status ts_poll(ts_ctx ctx, ts_ticket ticket, ts_stats* stats);

/* Primitive operators on the handle's design, for verification.  x, y are
 * DEVICE arrays of ndof FP64 on the context's stream. */
ts_status ts_apply_K(ts_handle h, const double* x, double* y);   /* y = K x (Dirichlet rows/cols masked) */
ts_status ts_apply_M(ts_handle h, const double* r, double* z);   /* z = M^{-1} r */
ts_status ts_apply_M_parts(ts_handle h, const double* r, double* z_local, double* z_coarse);
/* The preconditioner of the block path on nrhs <= 8 columns at once (DEVICE
 * arrays [nrhs][ndof]): z = M^{-1} r with which = 3, the level-1 part alone
 * with which = 1, the coarse part alone with which = 2 (Eq. localproblemsE,
 * Sec. 2.1), through the same kernels as a block solve.  Mixed-precision 2D
 * designs only (else TS_ERR_INVALID). */
ts_status ts_apply_M_block(ts_handle h, const double* r, double* z, int nrhs, int which);

/* Compliance sensitivities of the handle's design (Eq. 1003, minimum
 * compliance):
 *   dc[e] = -u^T (dK/drho_e) u = -p rho_e^(p-1) (E0 - Emin) u_e^T KE u_e,
 * and *compliance = sum_e E_e u_e^T KE u_e (= f^T u when u solves K u = f).
 * u: DEVICE array of ndof FP64 (zero at Dirichlet DOFs, e.g. from ts_solve);
 * dc: DEVICE array of n_el FP64 (written); compliance: HOST double or NULL
 * (when given, the call waits for the result).  Element order is row-major
 * (x fastest), as for rho. */
ts_status ts_sensitivity(ts_handle h, const double* u, double* dc, double* compliance);

/* Optimality-criteria update of the handle's densities rho (the density
 * update of the topology-optimisation loop this solve serves, Sec. 1):
 *   rho_new[e] = clamp(rho_e sqrt(max(-dc_e, 0) / lam),
 *                      max(0, rho_e - move), min(1, rho_e + move)),
 * with the multiplier lam found by 80 halvings of log(lam) over [1e-40, 1e40]
 * so that mean(rho_new) = volfrac (elements of equal volume).
 * dc, rho_new: DEVICE arrays of n_el FP64.  volfrac in (0, 1), move in
 * (0, 1]; otherwise TS_ERR_INVALID.  The handle is not changed (apply the
 * result with ts_update_density or ts_submit_update); the call waits. */
ts_status ts_oc_update(ts_handle h, const double* dc, double volfrac, double move, double* rho_new);

/* y = K x and *out = x^T K x (device pointers), like ts_apply_K plus the
 * energy dot, but allocating nothing at call time.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * when they call -- e.g. code recorded into a CUDA graph, or a serving loop
 * running under a fixed memory budget -- and it keeps the dot's per-block
 * partial sums in a fixed device array inside the library (512 KiB, held by
 * every GPU that loads the library until the process exits) instead of a
 * buffer.
 *   - Limit: the product's launch may use at most 65536 blocks of 256 nodes
 *     (2D: ceil((nx+1)/32) * ceil((ny+1)/8) tiles; 3D: ceil(nodes/256)),
 *     i.e. meshes of up to about 16.7 million nodes; larger meshes get
 *     TS_ERR_INVALID with the reason in ts_last_error().
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls in the process share the one array: calls that overlap on
 *     the GPU (other streams, other threads, other handles) race and must be
 *     serialised by the caller.  Every call rewrites every slot it reads, so
 *     nothing carries over from one call to the next.
 *   - Calls no cudaMalloc/cudaFree or allocating library routine.
 *   - Returns TS_ERR_BUSY while the request loop holds requests of h (the
 *     call would share the handle's streams with a running request).
 * x, y: ndof FP64; out: one FP64, all on the handle's device. */
ts_status ts_apply_K_dot_static(ts_handle h, const double* x, double* y, double* out);

/* Times one kernel of the path on the handle's stream with CUDA events:
 * `reps` launches after 3 warm-ups on internal, fixed inputs (the state left
 * by the last solve, or zeros), each launch timed alone after a read of a
 * zeroed 256 MB buffer that leaves the L2 cold and clean (a transient scratch
 * allocation from the library's pool).  kernel: "spmv" (y = K x), "local_solve"
 * (level-1 twisted block LU sweeps of every subdomain), "coarse_solve" (all stages
 * of u0 = K_0^{-1} r0), "coarse_restrict" (r0 = R_0 r), "prolong",
 * "update_xr" / "update_p" (the PCG vector updates), "sensitivity" and
 * "oc_update" (Eq. 1003 and the OC update on the last solution); the kernels
 * of the block path over 8 columns (mixed-precision 2D designs, state of the
 * last block solve): "bspmv", "bupdate_xr", "blocal_solve" (level 1 on the
 * tensor cores), "brestrict", "bcoarse_solve", "bprolong"; "iteration" (one PCG
 * iteration of the captured graph: a chunk's time divided by its
 * iterations; needs one earlier ts_solve).  The vector updates and
 * "iteration" overwrite the handle's PCG state (run them after the solves
 * whose results are kept).  "heat_eig" launches nothing: it reports the heat
 * eigenproblem launch of the handle's last setup (Sec. 4.1), timed with CUDA
 * events around it on the work stream, and the FP64 operations (FMA = 2) its
 * algorithm performed as counted by the kernel (line factors, mass
 * products, line solves, Lanczos recurrences, re-orthogonalisation, Ritz
 * vectors); reps is ignored.  "coarse_factor" likewise reports the K_0 factor
 * of the last setup (block cyclic reduction: batched tile Cholesky, inverse
 * and GEMM launches), timed with events around it, and the algorithmic FP64
 * operations of factoring K_0 (block-tridiagonal Cholesky by coarse lines:
 * w^3/3 + w^2 w'/2 + w'^2 w/2 multiply-adds per line of width w, next line
 * w'); "coarse_factor_bcr" the same launch with the operations the reduction
 * performs (GEMM tiles counted by the kernel, 32^3 per Cholesky-and-inverse
 * tile).
 * Outputs: average ms per launch, and the algorithmic FLOPs and bytes of one
 * launch (what the step must compute / move, not what the kernel re-reads).
 * Returns TS_ERR_INVALID for an unknown name or a kernel the handle does not
 * use (e.g. coarse_solve without a coarse space). */
ts_status ts_time_kernel(ts_handle h, const char* kernel, int reps, double* ms_per_launch, double* flops,
                         double* bytes);

/* Introspection (host outputs). */
int64_t ts_ndof(ts_handle h);
/* Level-1 sizes: subdomains, stored solve-factor entries (per block line of
 * every subdomain's twisted block LU: the S_k^{-1} form -- the packed Gram
 * factor V_k in mixed precision, the dense S_k^{-1} in FP64 -- and the
 * coupling stencils to both neighbouring lines, rows padded to 4 entries)
 * and local unknowns summed over subdomains. */
ts_status ts_level1_info(ts_handle h, int* n_sub, int64_t* factor_entries, int64_t* local_unknowns);
int ts_coarse_dim(ts_handle h);
/* Per (coarse node, component) heat eigenproblem: counts below tau and the
 * selected eigenvalues.  Arrays sized by ts_coarse_problems(); eigvals is
 * [n_problems][max_modes] (unused slots NaN).  With coarse_method 2 (M_EE)
 * there is one problem per coarse node: component -1, n_below = the modes
 * the stiff regions ask for (3 per region, at least 3), eigvals
 * [n_problems][48]. */
int ts_coarse_problems(ts_handle h);
ts_status ts_coarse_info(ts_handle h, int* node_index, int* component, int* n_below, int* n_selected,
                         double* eigvals);
ts_status ts_destroy(ts_handle h);

#ifdef __cplusplus
}
#endif
#endif
