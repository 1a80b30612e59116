// Preconditioned conjugate gradients on the device (Sec. 2, Sec. 5), FP64.
//
// Scalars live on the device; each iteration is a fixed sequence of kernels
// that read the stop flag first, so a chunk of iterations is captured once as
// a CUDA graph and replayed until the flag is set.  Reductions are two-stage
// (fixed per-block partials, then one block sums them in a fixed order), so a
// run is bitwise repeatable.
//
// Plain PCG:     beta = r_{k+1}.z_{k+1} / r_k.z_k
// Flexible PCG:  beta = r_{k+1}.(z_{k+1} - z_k) / r_k.z_k   (Notay's FCG(1), used
//                with the FP32 local solves, whose rounding makes M^{-1} vary)
// Stopping:      ||r|| <= rtol ||f||  and the delayed energy estimate
//                sum_{j=k-d+1}^{k} alpha_j r_j.z_j <= etol^2 f.x  (d = 4).
//
// Accurate finish: the recursively updated residual of CG drifts from the true
// one by about eps * |K| * max ||x_k||, and with contrast 1e6-1e8 that drift
// hides errors along soft (low-energy) modes that still weigh 1e-8..1e-7 in the
// K-norm.  After the first solve the true residual f - K x is formed in
// double-double arithmetic (exact products by FMA, compensated sums) and
// K d = r is solved again to a loose tolerance; x += d.  Rounds stop when the
// correction's energy d.r falls below (etol)^2 f.x.
#include <cmath>

#include "ts_internal.cuh"
#include "ts_pcg.cuh"
#include "ts_reduce.cuh"

constexpr int VEC_THREADS = 256;


// x += alpha p, r -= alpha q (alpha from the SpMV's last block); FP32 copy
// of r for the mixed path; partials of r.r, f.p and r.z_old (the
// prolongation's last block turns their sums into the convergence test)
__global__ void __launch_bounds__(VEC_THREADS) k_update_xr(DevScalars* S, int64_t n, double* __restrict__ x,
                                                           double* __restrict__ r, const double* __restrict__ p,
                                                           const double* __restrict__ q, const double* __restrict__ f,
                                                           const double* __restrict__ zold, float* __restrict__ r32,
                                                           double* __restrict__ partials) {
  pdl_wait();
  if (S->done) return;
  const double a = S->alpha;
  double rr = 0.0, fp = 0.0, rzo = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double pi = p[i];
    x[i] = fma(a, pi, x[i]);
    const double ri = fma(-a, q[i], r[i]);
    r[i] = ri;
    if (r32) r32[i] = (float)ri;
    rr = fma(ri, ri, rr);
    fp = fma(f[i], pi, fp);
    if (zold) rzo = fma(ri, zold[i], rzo);
  }
  pdl_trigger();
  double v[3] = {rr, fp, rzo};
  block_sum_n<VEC_THREADS, 3>(v);
  if (threadIdx.x == 0) {
    partials[3 * blockIdx.x] = v[0];
    partials[3 * blockIdx.x + 1] = v[1];
    partials[3 * blockIdx.x + 2] = v[2];
  }
}

// p = z + beta p (beta from the prolongation's last block), and z_old = z
// for the flexible variant
__global__ void __launch_bounds__(VEC_THREADS) k_update_p(DevScalars* S, int64_t n, double* __restrict__ p,
                                                          const double* __restrict__ z, double* __restrict__ zold) {
  pdl_wait();
  if (S->done) return;
  const double b = S->beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = z[i];
    p[i] = fma(b, p[i], zi);
    if (zold) zold[i] = zi;
  }
  pdl_trigger();
}

// initial: r = f - K x (or f); partials of f.f and f.x
__global__ void __launch_bounds__(VEC_THREADS) k_init_r(int64_t n, const double* __restrict__ f,
                                                        const double* __restrict__ Kx, double* __restrict__ r,
                                                        float* __restrict__ r32, const double* __restrict__ x,
                                                        double* __restrict__ partials) {
  double ff = 0.0, fx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double fi = f[i];
    const double ri = Kx ? fi - Kx[i] : fi;
    r[i] = ri;
    if (r32) r32[i] = (float)ri;
    ff += fi * fi;
    fx += fi * x[i];
  }
  double s1 = block_sum<VEC_THREADS>(ff);
  double s2 = block_sum<VEC_THREADS>(fx);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s1;
    partials[2 * blockIdx.x + 1] = s2;
  }
}

__global__ void k_init_scalars(DevScalars* S, const double* __restrict__ partials, int n) {
  double ff = 0.0, fx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    ff += partials[2 * i];
    fx += partials[2 * i + 1];
  }
  ff = block_sum<VEC_THREADS>(ff);
  fx = block_sum<VEC_THREADS>(fx);
  if (threadIdx.x == 0) {
    S->ff = ff;
    S->fx = fx;
    S->rel = 1.0;
    if (!(ff > 0.0)) {
      S->converged = 1;
      S->rel = 0.0;
      pcg_set_done(S);
    } else if (S->done_out) {
      *S->done_out = 0;
    }
  }
}

// rz = r.z (first iteration)
__global__ void k_init_rz(DevScalars* S, const double* __restrict__ partials, int n) {
  double rz = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) rz += partials[2 * i];
  rz = block_sum<VEC_THREADS>(rz);
  if (threadIdx.x == 0) S->rzs[0] = rz;
}

__global__ void k_copy(int64_t n, const double* __restrict__ a, double* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

__global__ void k_mask(int64_t n, const uint8_t* __restrict__ fm, double* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!fm[i]) v[i] = 0.0;
}

// x += d; partials of d.r (correction energy), f.x
__global__ void __launch_bounds__(VEC_THREADS) k_refine_add(int64_t n, double* __restrict__ x,
                                                            const double* __restrict__ d, const double* __restrict__ r,
                                                            const double* __restrict__ f,
                                                            double* __restrict__ partials) {
  double dr = 0.0, fx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double di = d[i];
    double xi = x[i] + di;
    x[i] = xi;
    dr += di * r[i];
    fx += f[i] * xi;
  }
  double s1 = block_sum<VEC_THREADS>(dr);
  double s2 = block_sum<VEC_THREADS>(fx);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s1;
    partials[2 * blockIdx.x + 1] = s2;
  }
}

__global__ void k_sum2(const double* __restrict__ partials, int n, double* __restrict__ out) {
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    a += partials[2 * i];
    b += partials[2 * i + 1];
  }
  a = block_sum<VEC_THREADS>(a);
  b = block_sum<VEC_THREADS>(b);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
  }
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
// vector kernels: two blocks per SM, several entries per thread (their
// reductions then cost little next to the streaming)
static int g_vec_blocks = 2 * 152;
static int vec_blocks() { return g_vec_blocks; }

void pcg_alloc(ts_handle h) {
  g_vec_blocks = 2 * h->ctx->n_sm;
  if (h->x) return;
  const int64_t n = h->g.ndof;
  h->x = dalloc<double>(h, n);
  h->r = dalloc<double>(h, n);
  h->z = dalloc<double>(h, n);
  h->zold = dalloc<double>(h, n);
  h->pvec = dalloc<double>(h, n);
  h->q = dalloc<double>(h, n);
  h->fvec = dalloc<double>(h, n);
  for (double* v : {h->x, h->r, h->z, h->zold, h->pvec, h->q, h->fvec})
    TS_CUDA(cudaMemsetAsync(v, 0, sizeof(double) * n, h->ctx->stream));
  h->forig = dalloc<double>(h, n);
  h->xacc = dalloc<double>(h, n);
  h->rtrue = dalloc<double>(h, n);
  int np = std::max(std::max(std::max(spmv_blocks(h->g), node_blocks(h->g)), prolong_blocks(h->g)), vec_blocks());
  h->partials = dalloc<double>(h, 3 * (size_t)np + 64);
  h->partials_s = dalloc<double>(h, (size_t)spmv_blocks(h->g) + 64);
  h->partials_xr = dalloc<double>(h, 3 * (size_t)vec_blocks() + 64);
  h->pvec2 = dalloc<double>(h, n);
  TS_CUDA(cudaMemsetAsync(h->pvec2, 0, sizeof(double) * n, h->ctx->stream));
  h->counters = dalloc<unsigned>(h, 4);
  TS_CUDA(cudaMemsetAsync(h->counters, 0, 4 * sizeof(unsigned), h->ctx->stream));
  if (h->opt.precision != TS_FP64) {
    h->r32 = dalloc<float>(h, n);
    TS_CUDA(cudaMemsetAsync(h->r32, 0, sizeof(float) * n, h->ctx->stream));
  }
  h->sc = dalloc<DevScalars>(h, 1);
  h->hist_cap = std::max(h->opt.max_iter, 1);
  h->alpha_hist = dalloc<double>(h, h->hist_cap);
  h->beta_hist = dalloc<double>(h, h->hist_cap);
  h->done_dev = dalloc<int>(h, 1);
  h->red2 = dalloc<double>(h, 2);
}

// z = M^{-1} r: the coarse correction (restriction, K_0 solve) is forked onto
// the context's second stream and runs concurrently with the level-1 solves;
// the prolongation joins both.  Under stream capture the fork and join
// become graph edges.
void ts_launch_apply_M(ts_handle h, const double* r, double* z, double* partials, const double* dv1,
                       const double* dv2, bool r32_ready, PcgTail tail);

__global__ void k_to_r32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

void prepare_r32(ts_handle h, const double* r) {
  if (!h->r32) return;
  tsl(h), k_to_r32<<<vec_blocks(), VEC_THREADS, 0, h->ctx->stream>>>(h->g.ndof, r, h->r32);
  TS_CUDA(cudaGetLastError());
}

void launch_apply_M(ts_handle h, const double* r, double* z, double* partials, const double* dv1, const double* dv2,
                    bool r32_ready) {
  ts_launch_apply_M(h, r, z, partials, dv1, dv2, r32_ready, PcgTail{});
}

// the same inside the PCG iteration: the prolongation's last block runs the
// convergence test and forms beta
void ts_launch_apply_M(ts_handle h, const double* r, double* z, double* partials, const double* dv1,
                       const double* dv2, bool r32_ready, PcgTail tail) {
  ts_ctx c = h->ctx;
  if (!r32_ready) prepare_r32(h, r);
  const bool coarse = h->opt.coarse && h->nc > 0;
  if (coarse) {
    TS_CUDA(cudaEventRecord(c->ev_fork, c->stream));
    TS_CUDA(cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
    cudaStream_t main = c->stream;
    const bool keep = h->pdl;
    c->stream = c->aux;
    h->pdl = false;  // the branch starts after a cross-stream fork
    try {
      launch_coarse_apply(h, r);
    } catch (...) {
      c->stream = main;
      h->pdl = keep;
      throw;
    }
    c->stream = main;
    h->pdl = keep;
    TS_CUDA(cudaEventRecord(c->ev_join, c->aux));
  }
  // the level-1 solves are the longer branch: their blocks go first
  h->prio = coarse ? c->prio_hi : 0;
  launch_local_solve(h, r);
  h->prio = 0;
  if (coarse) TS_CUDA(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  // after a join from the other stream the prolongation is an ordinary launch
  const bool keep = h->pdl;
  if (coarse) h->pdl = false;
  launch_prolong(h, z, h->opt.coarse ? 3 : 1, partials, dv1, dv2, tail);
  h->pdl = keep;
}

// one PCG iteration (all kernels check the stop flag):
//   2D: q = K p with p = z + beta p_old formed in the SpMV (last block: alpha)
//   3D: q = K p (last block: alpha)
//   x, r update         (partials of r.r, f.p, r.z_old)
//   z = M^{-1} r        (prolongation's last block: convergence test, stop
//                        flag, beta)
//   3D: p = z + beta p
// par: the iteration's parity; in 2D the search direction alternates
// between two buffers (p_old is read around each tile while p is written)
static void pcg_iteration(ts_handle h, int par) {
  cudaStream_t st = h->ctx->stream;
  const int64_t n = h->g.ndof;
  const int nbv = vec_blocks();
  DevScalars* S = h->sc;
  const bool flex = (h->opt.precision != TS_FP64);
  const bool fused = h->g.dim == 2;
  double* pb[2] = {h->pvec, h->pvec2};
  double* p = fused ? pb[par ^ 1] : h->pvec;
  h->pdl = true;
  if (fused)
    launch_spmv_fused_p(h, h->z, pb[par], p, flex ? h->zold : nullptr, h->q, h->partials_s, S, h->counters + 0);
  else
    launch_spmv(h, h->pvec, h->q, h->partials_s, h->pvec, S, h->counters + 0);
  ts_launch(h, true, k_update_xr, nbv, VEC_THREADS, 0, st, S, n, h->x, h->r, (const double*)p, (const double*)h->q,
            (const double*)h->fvec, (const double*)(flex ? h->zold : nullptr), h->r32, h->partials_xr);
  ts_launch_apply_M(h, h->r, h->z, h->partials, h->r, nullptr, true, PcgTail{S, h->counters + 2, h->partials_xr, nbv});
  if (!fused)
    ts_launch(h, true, k_update_p, nbv, VEC_THREADS, 0, st, S, n, h->pvec, (const double*)h->z,
              flex ? h->zold : nullptr);
  h->pdl = false;
  TS_CUDA(cudaGetLastError());
}

// --- timing support: kernels of the iteration run alone ---------------------
// PCG scalars that never stop (no tolerance, no iteration limit), so that
// the iteration kernels run their full work when timed one by one.
void pcg_timing_state(ts_handle h) {
  DevScalars hs{};
  TS_CUDA(cudaMemcpyAsync(&hs, h->sc, sizeof(hs), cudaMemcpyDeviceToHost, h->ctx->stream));
  TS_CUDA(cudaStreamSynchronize(h->ctx->stream));
  hs.done = 0;
  hs.converged = 0;
  hs.status = 0;
  hs.rtol = 0.0;
  hs.etol = 0.0;
  hs.maxit = 1 << 30;
  hs.hist_cap = 0;
  hs.done_out = nullptr;
  if (!(hs.rzs[0] > 0.0)) hs.rzs[0] = hs.rzs[1] = 1.0;
  hs.iter = 0;
  if (!(hs.ff > 0.0)) hs.ff = 1.0;
  TS_CUDA(cudaMemcpyAsync(h->sc, &hs, sizeof(hs), cudaMemcpyHostToDevice, h->ctx->stream));
  // the stop flag the captured kernels read
  if (h->done_dev) TS_CUDA(cudaMemsetAsync(h->done_dev, 0, sizeof(int), h->ctx->stream));
}

void launch_update_xr_alone(ts_handle h) {
  const bool flex = (h->opt.precision != TS_FP64);
  ts_launch(h, false, k_update_xr, vec_blocks(), VEC_THREADS, 0, h->ctx->stream, h->sc, h->g.ndof, h->x, h->r,
            (const double*)h->pvec, (const double*)h->q, (const double*)h->fvec,
            (const double*)(flex ? h->zold : nullptr), h->r32, h->partials_xr);
}

void launch_update_p_alone(ts_handle h) {
  const bool flex = (h->opt.precision != TS_FP64);
  ts_launch(h, false, k_update_p, vec_blocks(), VEC_THREADS, 0, h->ctx->stream, h->sc, h->g.ndof, h->pvec,
            (const double*)h->z, flex ? h->zold : nullptr);
}

// one replay of the captured chunk of iterations; returns its iteration count
int launch_iteration_chunk(ts_handle h) {
  if (!h->graph_exec) throw TsError(TS_ERR_INVALID, "no captured PCG iteration yet (solve once first)");
  TS_CUDA(cudaGraphLaunch(h->graph_exec, h->ctx->stream));
  tsl(h, h->graph_kernels);
  return 8;
}

// Runs PCG for the right-hand side in h->fvec (device); x0 in h->x when warm.
ts_status pcg_run(ts_handle h, bool warm, double rtol, double etol, PcgResult* res) {
  cudaStream_t st = h->ctx->stream;
  const int64_t n = h->g.ndof;
  const int nbv = vec_blocks(), nbp = prolong_blocks(h->g);
  DevScalars hs{};
  hs.rtol = rtol;
  hs.etol = etol;
  hs.maxit = h->opt.max_iter;
  hs.flexible = (h->opt.precision != TS_FP64) ? 1 : 0;
  hs.hist_cap = h->hist_cap;
  hs.alpha_hist = h->alpha_hist;
  hs.beta_hist = h->beta_hist;
  hs.done_out = h->done_dev;
  TS_CUDA(cudaMemcpyAsync(h->sc, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
  h->done_flag = nullptr;
  tsl(h), k_mask<<<nbv, VEC_THREADS, 0, st>>>(n, h->freemask, h->fvec);
  if (warm) {
    tsl(h), k_mask<<<nbv, VEC_THREADS, 0, st>>>(n, h->freemask, h->x);
    launch_spmv(h, h->x, h->q, nullptr, nullptr);
    tsl(h), k_init_r<<<nbv, VEC_THREADS, 0, st>>>(n, h->fvec, h->q, h->r, h->r32, h->x, h->partials);
  } else {
    TS_CUDA(cudaMemsetAsync(h->x, 0, sizeof(double) * n, st));
    tsl(h), k_init_r<<<nbv, VEC_THREADS, 0, st>>>(n, h->fvec, nullptr, h->r, h->r32, h->x, h->partials);
  }
  tsl(h), k_init_scalars<<<1, VEC_THREADS, 0, st>>>(h->sc, h->partials, nbv);
  launch_apply_M(h, h->r, h->z, h->partials, h->r, nullptr, true);
  tsl(h), k_init_rz<<<1, VEC_THREADS, 0, st>>>(h->sc, h->partials, nbp);
  if (h->g.dim == 2) {
    // first iteration: beta = 0, so the SpMV forms p = z (p_old only needs
    // finite entries)
    TS_CUDA(cudaMemsetAsync(h->pvec, 0, sizeof(double) * n, st));
  } else {
    tsl(h), k_copy<<<nbv, VEC_THREADS, 0, st>>>(n, h->z, h->pvec);
  }
  tsl(h), k_copy<<<nbv, VEC_THREADS, 0, st>>>(n, h->z, h->zold);
  TS_CUDA(cudaGetLastError());
  // iterate in chunks captured as a graph
  const int chunk = 8;
  if (!h->graph_exec) {
    h->done_flag = h->done_dev;
    cudaGraph_t graph;
    TS_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    h->cap_launches = 0;
    try {
      for (int i = 0; i < chunk; ++i) pcg_iteration(h, i & 1);
    } catch (...) {
      cudaStreamEndCapture(st, &graph);
      h->done_flag = nullptr;
      h->capturing = false;
      throw;
    }
    h->capturing = false;
    h->graph_kernels = h->cap_launches;  // captured, not launched
    TS_CUDA(cudaStreamEndCapture(st, &graph));
    TS_CUDA(cudaGraphInstantiate(&h->graph_exec, graph, 0));
    TS_CUDA(cudaGraphDestroy(graph));
    h->done_flag = nullptr;
  }
  int done = 0;
  int launched = 0;
  TS_CUDA(cudaMemcpyAsync(&done, h->done_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  TS_CUDA(cudaStreamSynchronize(st));
  // Chunks are queued one ahead of the host's check of the stop flag, so
  // that the GPU does not idle while the host reads a flag and launches the
  // next chunk; the chunk queued after convergence only reads the flag.
  if (!h->chunk_flag_h) {
    TS_CUDA(cudaMallocHost(&h->chunk_flag_h, 2 * sizeof(int)));
    TS_CUDA(cudaEventCreateWithFlags(&h->chunk_ev[0], cudaEventDisableTiming));
    TS_CUDA(cudaEventCreateWithFlags(&h->chunk_ev[1], cudaEventDisableTiming));
  }
  auto queue_chunk = [&](int slot) {
    TS_CUDA(cudaGraphLaunch(h->graph_exec, st));
    tsl(h, h->graph_kernels);
    launched += chunk;
    TS_CUDA(cudaMemcpyAsync(h->chunk_flag_h + slot, h->done_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    TS_CUDA(cudaEventRecord(h->chunk_ev[slot], st));
  };
  if (!done) {
    int k = 0;
    queue_chunk(0);
    for (;;) {
      // the device flag must have been set by then
      const bool more = launched <= h->opt.max_iter + 2 * chunk;
      if (more) queue_chunk((k + 1) & 1);
      TS_CUDA(cudaEventSynchronize(h->chunk_ev[k & 1]));
      if (h->chunk_flag_h[k & 1] || !more) break;
      ++k;
    }
  }
  TS_CUDA(cudaMemcpyAsync(&hs, h->sc, sizeof(hs), cudaMemcpyDeviceToHost, st));
  TS_CUDA(cudaStreamSynchronize(st));
  res->iters = hs.iter;
  res->converged = hs.converged;
  // relative residual and delayed energy estimate from the scalars the
  // device kept (its stopping test compares them without dividing)
  res->rel = (hs.iter > 0 && hs.ff > 0.0) ? std::sqrt(hs.rr / hs.ff) : hs.rel;
  {
    double e = 0.0;
    for (int d = 0; d < TS_EDELAY; ++d) e += hs.terms[d];
    res->energy_est = (hs.iter >= TS_EDELAY) ? e / std::max(hs.fx, 1e-300) : hs.energy_est;
  }
  res->status = hs.status;
  res->ff = hs.ff;
  if (res->want_cond) {
    int k = std::min(hs.iter, h->hist_cap);
    std::vector<double> al(k), be(k);
    if (k > 0) {
      TS_CUDA(cudaMemcpy(al.data(), h->alpha_hist, sizeof(double) * k, cudaMemcpyDeviceToHost));
      TS_CUDA(cudaMemcpy(be.data(), h->beta_hist, sizeof(double) * k, cudaMemcpyDeviceToHost));
    }
    res->cond = lanczos_cond_host(al, be, k);
  }
  if (hs.status == TS_ERR_BREAKDOWN) return TS_ERR_BREAKDOWN;
  if (!hs.converged) return TS_NOT_CONVERGED;
  return TS_OK;
}

// Full solve of one right-hand side in h->forig: PCG, then refinement rounds
// with a double-double true residual.  Result in h->xacc.
ts_status solve_one(ts_handle h, bool warm, double rtol, ts_stats* stats) {
  cudaStream_t st = h->ctx->stream;
  const int64_t n = h->g.ndof;
  const int nbv = vec_blocks();
  const double etol = (h->opt.energy_tol < 0.0) ? 0.1 * rtol : h->opt.energy_tol;
  cudaEvent_t e0, e1;
  TS_CUDA(cudaEventCreate(&e0));
  TS_CUDA(cudaEventCreate(&e1));
  TS_CUDA(cudaEventRecord(e0, st));
  tsl(h), k_mask<<<nbv, VEC_THREADS, 0, st>>>(n, h->freemask, h->forig);
  tsl(h), k_copy<<<nbv, VEC_THREADS, 0, st>>>(n, h->forig, h->fvec);
  if (warm) tsl(h), k_copy<<<nbv, VEC_THREADS, 0, st>>>(n, h->xacc, h->x);
  PcgResult r0{};
  r0.want_cond = stats != nullptr;
  ts_status s = pcg_run(h, warm, rtol, etol, &r0);
  int iters = r0.iters;
  tsl(h), k_copy<<<nbv, VEC_THREADS, 0, st>>>(n, h->x, h->xacc);
  double true_rel = r0.rel;
  int rounds = 0;
  const double ff = r0.ff;
  if (s == TS_OK && h->opt.refine > 0 && ff > 0.0) {
    for (int round = 0; round < h->opt.refine; ++round) {
      // r = f - K x in double-double; new right-hand side
      launch_residual_dd(h, h->forig, h->xacc, h->fvec, h->partials);
      tsl(h), k_sum2<<<1, VEC_THREADS, 0, st>>>(h->partials, node_blocks(h->g), h->red2);
      double rr[2];
      TS_CUDA(cudaMemcpyAsync(rr, h->red2, sizeof(rr), cudaMemcpyDeviceToHost, st));
      TS_CUDA(cudaStreamSynchronize(st));
      true_rel = std::sqrt(rr[0] / ff);
      if (!(rr[0] > 0.0)) break;
      // correction solve K d = r to 1e-3 of ||r|| (no energy test on the correction)
      PcgResult rc{};
      tsl(h), k_copy<<<nbv, VEC_THREADS, 0, st>>>(n, h->fvec, h->rtrue);  // keep r for d.r
      ts_status sc = pcg_run(h, false, 1e-3, 0.0, &rc);
      iters += rc.iters;
      ++rounds;
      if (sc == TS_ERR_BREAKDOWN) break;
      // x += d; energy of the correction d.r relative to f.x
      tsl(h), k_refine_add<<<nbv, VEC_THREADS, 0, st>>>(n, h->xacc, h->x, h->rtrue, h->forig, h->partials);
      tsl(h), k_sum2<<<1, VEC_THREADS, 0, st>>>(h->partials, nbv, h->red2);
      double de[2];
      TS_CUDA(cudaMemcpyAsync(de, h->red2, sizeof(de), cudaMemcpyDeviceToHost, st));
      TS_CUDA(cudaStreamSynchronize(st));
      if (de[0] <= etol * etol * std::fabs(de[1])) break;
    }
  }
  TS_CUDA(cudaEventRecord(e1, st));
  TS_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  TS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (stats) {
    stats->iters = iters;
    stats->converged = r0.converged;
    stats->rel_res = true_rel;
    stats->energy_est = r0.energy_est;
    stats->cond_est = r0.cond;
    stats->coarse_dim = h->nc;
    stats->cap_hits = h->cap_hits;
    stats->eig_unconverged = h->eig_unconv;
    stats->setup_ms = h->setup_ms;
    stats->solve_ms = ms;
    stats->precision = h->opt.precision;
    stats->first_iters = r0.iters;
    stats->refine_rounds = rounds;
  }
  return s;
}

// tridiagonal T_jj = 1/a_j + b_{j-1}/a_{j-1}, T_{j,j+1} = sqrt(b_j)/a_j;
// extreme eigenvalues by Sturm bisection
static int sturm_host(const std::vector<double>& d, const std::vector<double>& e, double x) {
  int c = 0;
  double q = 1.0;
  for (size_t i = 0; i < d.size(); ++i) {
    q = (d[i] - x) - (i > 0 ? e[i - 1] * e[i - 1] / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0) ++c;
  }
  return c;
}

double lanczos_cond_host(const std::vector<double>& al, const std::vector<double>& be, int k) {
  if (k <= 0) return NAN;
  std::vector<double> d(k), e(k > 1 ? k - 1 : 0);
  for (int j = 0; j < k; ++j) {
    d[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
    if (j + 1 < k) e[j] = std::sqrt(std::max(be[j], 0.0)) / al[j];
  }
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < k; ++i) {
    double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - r);
    hi = std::max(hi, d[i] + r);
  }
  auto kth = [&](int idx) {
    double a = lo, b = hi;
    for (int it = 0; it < 200; ++it) {
      double m = 0.5 * (a + b);
      if (m <= a || m >= b) break;
      if (sturm_host(d, e, m) > idx)
        b = m;
      else
        a = m;
    }
    return 0.5 * (a + b);
  };
  double lmin = kth(0), lmax = kth(k - 1);
  return lmax / lmin;
}
