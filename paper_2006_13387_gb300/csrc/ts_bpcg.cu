// Block PCG: TS_NB right-hand sides solved together, every kernel launch
// shared by the columns (Sec. 2 PCG, Sec. 5 stopping rule, per column).
//
// A solve of several load cases of one design (2D, mixed precision) packs
// them into block vectors [ndof][TS_NB] and runs one flexible PCG per column
// in lock step: one block SpMV (the stencil read once for every column), one
// x/r update, one application of the two-level preconditioner (level 1 on the
// tensor cores, coarse restriction, the coarse solve's stages -- block
// cyclic reduction over coarse lines or the nested-dissection levels -- and
// prolongation, each reading its stored data once for every column).  Each
// column keeps its own scalars, stopping test and energy estimate; a column
// that has stopped keeps its iterate (alpha = beta = 0) while the others
// continue, and the launch sequence ends when every column has stopped.  As in
// the one-column iteration, a chunk of iterations is captured as a CUDA graph
// and replayed until the device stop flag is set.
#include <cmath>
#include <functional>
#include <string>

#include "ts_bpcg.cuh"
#include "ts_internal.cuh"
#include "ts_pcg.cuh"
#include "ts_reduce.cuh"

constexpr int BV_THREADS = 256;

// ABI [nrhs][ndof] -> block [ndof][TS_NB] (columns past nrhs zero), masked
__global__ void k_bpack(int64_t n, int nrhs, const double* __restrict__ f, const uint8_t* __restrict__ fm,
                        double* __restrict__ fb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * TS_NB;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = i / TS_NB;
    const int c = (int)(i % TS_NB);
    fb[i] = (c < nrhs && fm[d]) ? f[(int64_t)c * n + d] : 0.0;
  }
}

// block [ndof][TS_NB] -> ABI [nrhs][ndof]
__global__ void k_bunpack(int64_t n, int nrhs, const double* __restrict__ xb, double* __restrict__ u) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * nrhs;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / n);
    const int64_t d = i % n;
    u[i] = xb[d * TS_NB + c];
  }
}

// x += alpha_c p, r -= alpha_c q; FP32 copy of r; per-column partials of
// r.r, f.p and r.z_old ([block][3][TS_NB])
__global__ void __launch_bounds__(BV_THREADS) k_bupdate_xr(BScalars* S, int64_t n8, double* __restrict__ x,
                                                            double* __restrict__ r, const double* __restrict__ p,
                                                            const double* __restrict__ q,
                                                            const double* __restrict__ f,
                                                            const double* __restrict__ zold, float* __restrict__ r32,
                                                            double* __restrict__ partials) {
  pdl_wait();
  if (S->done) return;
  const double a = S->alpha[threadIdx.x % TS_NB];
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n8; i += (int64_t)gridDim.x * blockDim.x) {
    const double pi = p[i];
    x[i] = fma(a, pi, x[i]);
    const double ri = fma(-a, q[i], r[i]);
    r[i] = ri;
    r32[i] = (float)ri;
    v[0] = fma(ri, ri, v[0]);
    v[1] = fma(f[i], pi, v[1]);
    v[2] = fma(ri, zold[i], v[2]);
  }
  pdl_trigger();
  bsum_by_col<BV_THREADS, 3>(v);
  if (threadIdx.x < TS_NB)
#pragma unroll
    for (int j = 0; j < 3; ++j) partials[((int64_t)blockIdx.x * 3 + j) * TS_NB + threadIdx.x] = v[j];
}

// r = f - Kx (or f); FP32 copy; per-column partials of f.f, f.x ([block][2][TS_NB])
__global__ void __launch_bounds__(BV_THREADS) k_binit_r(int64_t n8, const double* __restrict__ f,
                                                         const double* __restrict__ Kx, double* __restrict__ r,
                                                         float* __restrict__ r32, const double* __restrict__ x,
                                                         double* __restrict__ partials) {
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n8; i += (int64_t)gridDim.x * blockDim.x) {
    const double fi = f[i];
    const double ri = Kx ? fi - Kx[i] : fi;
    r[i] = ri;
    r32[i] = (float)ri;
    v[0] = fma(fi, fi, v[0]);
    v[1] = fma(fi, x[i], v[1]);
  }
  bsum_by_col<BV_THREADS, 2>(v);
  if (threadIdx.x < TS_NB)
#pragma unroll
    for (int j = 0; j < 2; ++j) partials[((int64_t)blockIdx.x * 2 + j) * TS_NB + threadIdx.x] = v[j];
}

__global__ void __launch_bounds__(BV_THREADS) k_binit_scalars(BScalars* S, const double* __restrict__ partials,
                                                               int n) {
  double v[2];
  bsum_partials<BV_THREADS, 2, 2>(partials, n, v);
  if (threadIdx.x < TS_NB) {
    const int c = threadIdx.x;
    S->ff[c] = v[0];
    S->fx[c] = v[1];
    S->rr[c] = v[0];
    if (!(v[0] > 0.0) || c >= S->ncols) {  // a zero (or padding) column is solved by x = 0
      S->converged[c] = 1;
      S->cdone[c] = 1;
      S->it[c] = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int live = 0;
    for (int c = 0; c < TS_NB; ++c) live += S->cdone[c] ? 0 : 1;
    S->done = live == 0;
    if (S->done_out) *S->done_out = S->done;
  }
}

// r_0.z_0 per column from the prolongation's partials ([block][TS_NB])
__global__ void __launch_bounds__(BV_THREADS) k_binit_rz(BScalars* S, const double* __restrict__ partials, int n) {
  double v[1];
  bsum_partials<BV_THREADS, 1, 1>(partials, n, v);
  if (threadIdx.x < TS_NB) S->rzs[0][threadIdx.x] = v[0];
}

__global__ void k_bmask_copy(int64_t n, const uint8_t* __restrict__ fm, const double* __restrict__ a,
                             double* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * TS_NB;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = fm[i / TS_NB] ? a[i] : 0.0;
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
static int bvec_blocks(ts_handle h) { return 4 * h->ctx->n_sm; }

bool block_path_applies(ts_handle h, int nrhs) {
  return nrhs >= 2 && h->g.dim == 2 && h->opt.precision != TS_FP64 && h->kst != nullptr && h->opt.refine == 0 &&
         (!(h->opt.coarse && h->nc > 0) || h->bcr_btasks != nullptr || (h->nd && h->u0fb != nullptr));
}

static void balloc(ts_handle h) {
  if (h->xb) return;
  cudaStream_t st = h->ctx->stream;
  const int64_t n8 = h->g.ndof * TS_NB;
  for (double** v : {&h->xb, &h->rb, &h->zb, &h->zoldb, &h->qb, &h->fb, &h->pb[0], &h->pb[1]}) {
    *v = dalloc<double>(h, n8);
    TS_CUDA(cudaMemsetAsync(*v, 0, sizeof(double) * n8, st));
  }
  h->r32b = dalloc<float>(h, n8);
  TS_CUDA(cudaMemsetAsync(h->r32b, 0, sizeof(float) * n8, st));
  h->zloc32b = dalloc<float>(h, h->zloc_len * TS_NB);
  h->bpart_s = dalloc<double>(h, (size_t)bspmv_blocks(h->g) * TS_NB);
  h->bpart_xr = dalloc<double>(h, (size_t)std::max(bvec_blocks(h), 1) * 3 * TS_NB);
  h->bpart_p = dalloc<double>(h, (size_t)std::max(bprolong_blocks(h->g), bvec_blocks(h)) * 2 * TS_NB);
  h->bcounters = dalloc<unsigned>(h, 4);
  TS_CUDA(cudaMemsetAsync(h->bcounters, 0, 4 * sizeof(unsigned), st));
  h->bsc = dalloc<BScalars>(h, 1);
  h->bhist_a = dalloc<double>(h, (size_t)h->hist_cap * TS_NB);
  h->bhist_b = dalloc<double>(h, (size_t)h->hist_cap * TS_NB);
  h->bdone = dalloc<int>(h, 1);
}

// z = M^{-1} r for the block: the coarse branch (restriction, stages) on the
// second stream, concurrent with the level-1 solves; the prolongation joins
// both (and, inside the iteration, runs the stopping test and beta)
static void bapply_M(ts_handle h, double* z, double* partials, const double* dv, BPcgTail tail) {
  ts_ctx c = h->ctx;
  const bool coarse = h->opt.coarse && h->nc > 0;
  if (coarse) {
    TS_CUDA(cudaEventRecord(c->ev_fork, c->stream));
    TS_CUDA(cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
    cudaStream_t main = c->stream;
    const bool keep = h->pdl;
    c->stream = c->aux;
    h->pdl = false;
    try {
      launch_brestrict(h, h->r32b, h->r0b);
      launch_bcoarse_solve(h);
    } catch (...) {
      c->stream = main;
      h->pdl = keep;
      throw;
    }
    c->stream = main;
    h->pdl = keep;
    TS_CUDA(cudaEventRecord(c->ev_join, c->aux));
  }
  h->prio = coarse ? c->prio_hi : 0;
  launch_blocal_solve(h, h->r32b, h->zloc32b);
  h->prio = 0;
  if (coarse) TS_CUDA(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  const bool keep = h->pdl;
  if (coarse) h->pdl = false;
  launch_bprolong(h, h->zloc32b, h->u0fb, z, partials, dv, tail);
  h->pdl = keep;
}

// one block iteration; par: which search-direction buffer is p_old
static void bpcg_iteration(ts_handle h, int par) {
  cudaStream_t st = h->ctx->stream;
  BScalars* S = h->bsc;
  double* p_old = h->pb[par];
  double* p_new = h->pb[par ^ 1];
  h->pdl = true;
  launch_bspmv(h, nullptr, h->zb, p_old, p_new, h->zoldb, h->qb, h->bpart_s, S, h->bcounters + 0);
  ts_launch(h, true, k_bupdate_xr, bvec_blocks(h), BV_THREADS, 0, st, S, h->g.ndof * TS_NB, h->xb, h->rb,
            (const double*)p_new, (const double*)h->qb, (const double*)h->fb, (const double*)h->zoldb, h->r32b,
            h->bpart_xr);
  bapply_M(h, h->zb, h->bpart_p, h->rb, BPcgTail{S, h->bcounters + 2, h->bpart_xr, bvec_blocks(h)});
  h->pdl = false;
  TS_CUDA(cudaGetLastError());
}

struct BResult {
  BScalars s;
  std::vector<double> cond;
};

// Runs the block PCG on h->fb (x0 in h->xb when warm); fills res.
static void bpcg_run(ts_handle h, bool warm, int ncols, double rtol, double etol, bool want_cond, BResult* res) {
  cudaStream_t st = h->ctx->stream;
  const int64_t n = h->g.ndof, n8 = n * TS_NB;
  const int nbv = bvec_blocks(h);
  BScalars hs{};
  hs.rtol = rtol;
  hs.etol = etol;
  hs.maxit = h->opt.max_iter;
  hs.flexible = 1;
  hs.ncols = ncols;
  hs.hist_cap = h->hist_cap;
  hs.alpha_hist = h->bhist_a;
  hs.beta_hist = h->bhist_b;
  hs.done_out = h->bdone;
  TS_CUDA(cudaMemcpyAsync(h->bsc, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
  h->done_flag = nullptr;
  if (warm) {
    tsl(h), k_bmask_copy<<<nbv, BV_THREADS, 0, st>>>(n, h->freemask, h->xb, h->xb);
    launch_bspmv(h, h->xb, nullptr, nullptr, nullptr, nullptr, h->qb, nullptr, nullptr, nullptr);
    tsl(h), k_binit_r<<<nbv, BV_THREADS, 0, st>>>(n8, h->fb, h->qb, h->rb, h->r32b, h->xb, h->bpart_xr);
  } else {
    TS_CUDA(cudaMemsetAsync(h->xb, 0, sizeof(double) * n8, st));
    tsl(h), k_binit_r<<<nbv, BV_THREADS, 0, st>>>(n8, h->fb, nullptr, h->rb, h->r32b, h->xb, h->bpart_xr);
  }
  tsl(h), k_binit_scalars<<<1, BV_THREADS, 0, st>>>(h->bsc, h->bpart_xr, nbv);
  bapply_M(h, h->zb, h->bpart_p, h->rb, BPcgTail{});
  tsl(h), k_binit_rz<<<1, BV_THREADS, 0, st>>>(h->bsc, h->bpart_p, bprolong_blocks(h->g));
  // first iteration: beta = 0, p_old only needs finite entries
  TS_CUDA(cudaMemsetAsync(h->pb[0], 0, sizeof(double) * n8, st));
  TS_CUDA(cudaGetLastError());
  const int chunk = 8;
  if (!h->bgraph_exec) {
    h->done_flag = h->bdone;
    cudaGraph_t graph;
    TS_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    h->cap_launches = 0;
    try {
      for (int i = 0; i < chunk; ++i) bpcg_iteration(h, i & 1);
    } catch (...) {
      cudaStreamEndCapture(st, &graph);
      h->done_flag = nullptr;
      h->capturing = false;
      throw;
    }
    h->capturing = false;
    h->bgraph_kernels = h->cap_launches;
    TS_CUDA(cudaStreamEndCapture(st, &graph));
    TS_CUDA(cudaGraphInstantiate(&h->bgraph_exec, graph, 0));
    TS_CUDA(cudaGraphDestroy(graph));
    h->done_flag = nullptr;
  }
  int done = 0, launched = 0;
  TS_CUDA(cudaMemcpyAsync(&done, h->bdone, sizeof(int), cudaMemcpyDeviceToHost, st));
  TS_CUDA(cudaStreamSynchronize(st));
  if (!h->chunk_flag_h) {
    TS_CUDA(cudaMallocHost(&h->chunk_flag_h, 2 * sizeof(int)));
    TS_CUDA(cudaEventCreateWithFlags(&h->chunk_ev[0], cudaEventDisableTiming));
    TS_CUDA(cudaEventCreateWithFlags(&h->chunk_ev[1], cudaEventDisableTiming));
  }
  auto queue_chunk = [&](int slot) {
    TS_CUDA(cudaGraphLaunch(h->bgraph_exec, st));
    tsl(h, h->bgraph_kernels);
    launched += chunk;
    TS_CUDA(cudaMemcpyAsync(h->chunk_flag_h + slot, h->bdone, sizeof(int), cudaMemcpyDeviceToHost, st));
    TS_CUDA(cudaEventRecord(h->chunk_ev[slot], st));
  };
  if (!done) {
    int k = 0;
    queue_chunk(0);
    for (;;) {
      const bool more = launched <= h->opt.max_iter + 2 * chunk;
      if (more) queue_chunk((k + 1) & 1);
      TS_CUDA(cudaEventSynchronize(h->chunk_ev[k & 1]));
      if (h->chunk_flag_h[k & 1] || !more) break;
      ++k;
    }
  }
  TS_CUDA(cudaMemcpyAsync(&res->s, h->bsc, sizeof(BScalars), cudaMemcpyDeviceToHost, st));
  TS_CUDA(cudaStreamSynchronize(st));
  res->cond.assign(TS_NB, NAN);
  if (want_cond) {
    const int k = std::min(res->s.iter, h->hist_cap);
    std::vector<double> al((size_t)k * TS_NB), be((size_t)k * TS_NB);
    if (k > 0) {
      TS_CUDA(cudaMemcpy(al.data(), h->bhist_a, sizeof(double) * al.size(), cudaMemcpyDeviceToHost));
      TS_CUDA(cudaMemcpy(be.data(), h->bhist_b, sizeof(double) * be.size(), cudaMemcpyDeviceToHost));
    }
    for (int c = 0; c < ncols; ++c) {
      const int kc = std::min(res->s.cdone[c] ? res->s.it[c] : res->s.iter, k);
      std::vector<double> a(kc), b(kc);
      for (int j = 0; j < kc; ++j) {
        a[j] = al[(size_t)j * TS_NB + c];
        b[j] = be[(size_t)j * TS_NB + c];
      }
      res->cond[c] = lanczos_cond_host(a, b, kc);
    }
  }
}

// Solves nrhs >= 2 right-hand sides ([nrhs][ndof], host or device per the
// handle's options) in chunks of TS_NB columns; u is read as the initial
// iterate when warm_start is set.  The caller has ordered the lane's stream.
ts_status block_solve(ts_handle h, const double* f, double* u, int nrhs, double rtol, ts_stats* stats) {
  cudaStream_t st = h->ctx->stream;
  const int64_t n = h->g.ndof;
  const bool dev = h->opt.mem_is_device != 0;
  const double etol = (h->opt.energy_tol < 0.0) ? 0.1 * rtol : h->opt.energy_tol;
  const int nbv = bvec_blocks(h);
  balloc(h);
  ts_status worst = TS_OK;
  for (int c0 = 0; c0 < nrhs; c0 += TS_NB) {
    const int nc = std::min(TS_NB, nrhs - c0);
    cudaEvent_t e0, e1;
    TS_CUDA(cudaEventCreate(&e0));
    TS_CUDA(cudaEventCreate(&e1));
    TS_CUDA(cudaEventRecord(e0, st));
    // the columns go through the library's scratch copy in the ABI layout
    const double* fsrc = f + (int64_t)c0 * n;
    double* usrc = u + (int64_t)c0 * n;
    double* stage = h->qb;  // [nc][ndof] fits in one block vector
    TS_CUDA(cudaMemcpyAsync(stage, fsrc, sizeof(double) * n * nc,
                            dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    tsl(h), k_bpack<<<nbv, BV_THREADS, 0, st>>>(n, nc, stage, h->freemask, h->fb);
    const bool warm = h->opt.warm_start != 0;
    if (warm) {
      TS_CUDA(cudaMemcpyAsync(stage, usrc, sizeof(double) * n * nc,
                              dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
      tsl(h), k_bpack<<<nbv, BV_THREADS, 0, st>>>(n, nc, stage, h->freemask, h->xb);
    }
    TS_CUDA(cudaGetLastError());
    BResult res;
    bpcg_run(h, warm, nc, rtol, etol, stats != nullptr, &res);
    tsl(h), k_bunpack<<<nbv, BV_THREADS, 0, st>>>(n, nc, h->xb, stage);
    TS_CUDA(cudaGetLastError());
    TS_CUDA(cudaMemcpyAsync(usrc, stage, sizeof(double) * n * nc,
                            dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    TS_CUDA(cudaEventRecord(e1, st));
    TS_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    TS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const BScalars& S = res.s;
    for (int c = 0; c < nc; ++c) {
      const int it = S.cdone[c] ? S.it[c] : S.iter;
      ts_status sc = TS_OK;
      if (S.status[c] == TS_ERR_BREAKDOWN) sc = TS_ERR_BREAKDOWN;
      else if (!S.converged[c]) sc = TS_NOT_CONVERGED;
      if (sc == TS_ERR_BREAKDOWN) worst = sc;
      else if (sc == TS_NOT_CONVERGED && worst == TS_OK) worst = sc;
      if (stats) {
        ts_stats& o = stats[c0 + c];
        o.iters = it;
        o.converged = S.converged[c];
        o.rel_res = (S.ff[c] > 0.0) ? std::sqrt(S.rr[c] / S.ff[c]) : 0.0;
        double e = 0.0;
        for (int d = 0; d < TS_EDELAY; ++d) e += S.terms[d][c];
        o.energy_est = (it >= TS_EDELAY) ? e / std::max(S.fx[c], 1e-300) : NAN;
        o.cond_est = res.cond[c];
        o.coarse_dim = h->nc;
        o.cap_hits = h->cap_hits;
        o.eig_unconverged = h->eig_unconv;
        o.setup_ms = h->setup_ms;
        o.solve_ms = ms;  // the whole block of columns
        o.precision = h->opt.precision;
        o.first_iters = it;
        o.refine_rounds = 0;
      }
    }
  }
  int status[4];
  TS_CUDA(cudaMemcpy(status, h->dstatus, sizeof(status), cudaMemcpyDeviceToHost));
  if (status[0] & 16) throw TsError(TS_ERR_TIMEOUT, "block level 1: a staged line block did not arrive");
  return worst;
}

// z = M^{-1} r for nrhs <= TS_NB columns through the block kernels (device
// arrays [nrhs][ndof]); which: 1 level 1, 2 coarse part, 3 both
void block_apply_M(ts_handle h, const double* r, double* z, int nrhs, int which) {
  cudaStream_t st = h->ctx->stream;
  const int64_t n = h->g.ndof;
  const int nbv = bvec_blocks(h);
  balloc(h);
  h->done_flag = nullptr;
  tsl(h), k_bpack<<<nbv, BV_THREADS, 0, st>>>(n, nrhs, r, h->freemask, h->rb);
  tsl(h), k_binit_r<<<nbv, BV_THREADS, 0, st>>>(n * TS_NB, h->rb, nullptr, h->qb, h->r32b, h->rb, h->bpart_xr);
  const bool keep_coarse = h->opt.coarse != 0;
  if (!(which & 2)) h->opt.coarse = 0;
  try {
    if (which & 1) {
      bapply_M(h, h->zb, nullptr, nullptr, BPcgTail{});
    } else {
      // coarse part alone: zero local solutions
      TS_CUDA(cudaMemsetAsync(h->zloc32b, 0, sizeof(float) * h->zloc_len * TS_NB, st));
      if (h->nc > 0) {
        launch_brestrict(h, h->r32b, h->r0b);
        launch_bcoarse_solve(h);
      }
      launch_bprolong(h, h->zloc32b, h->u0fb, h->zb, nullptr, nullptr, BPcgTail{});
    }
  } catch (...) {
    h->opt.coarse = keep_coarse;
    throw;
  }
  h->opt.coarse = keep_coarse;
  tsl(h), k_bunpack<<<nbv, BV_THREADS, 0, st>>>(n, nrhs, h->zb, z);
  TS_CUDA(cudaGetLastError());
}

extern "C" ts_status ts_apply_M_block(ts_handle h, const double* r, double* z, int nrhs, int which) {
  if (!h || !r || !z) return TS_ERR_INVALID;
  return ts_guarded(h->ctx, [&]() -> ts_status {
    if (nrhs < 1 || nrhs > TS_NB) throw TsError(TS_ERR_INVALID, "nrhs must lie in [1, 8]");
    if (which < 1 || which > 3) throw TsError(TS_ERR_INVALID, "which must be 1, 2 or 3");
    if (!block_path_applies(h, 2)) throw TsError(TS_ERR_INVALID, "the block path needs a mixed-precision 2D design");
    if (server_holds(h->root, h)) throw TsError(TS_ERR_BUSY, "the handle has requests in the request loop");
    TS_CUDA(cudaEventRecord(h->ctx->ev_in, h->ctx->user_stream));
    TS_CUDA(cudaStreamWaitEvent(h->ctx->stream, h->ctx->ev_in, 0));
    block_apply_M(h, r, z, nrhs, which);
    int status[4];
    TS_CUDA(cudaMemcpyAsync(status, h->dstatus, sizeof(status), cudaMemcpyDeviceToHost, h->ctx->stream));
    TS_CUDA(cudaStreamSynchronize(h->ctx->stream));
    if (status[0] & 16) throw TsError(TS_ERR_TIMEOUT, "block level 1: a staged line block did not arrive");
    TS_CUDA(cudaEventRecord(h->ctx->ev_out, h->ctx->stream));
    TS_CUDA(cudaStreamWaitEvent(h->ctx->user_stream, h->ctx->ev_out, 0));
    return TS_OK;
  });
}

// Kernels of the block path for ts_time_kernel: the launch `run` performs,
// with its algorithmic FLOPs and bytes per launch (every stored array read
// once for all TS_NB columns; FP64 block vectors 8 B x TS_NB per DOF, FP32
// copies 4 B x TS_NB).  The state is that of the handle's last block solve
// (balloc'd zeros before any).  Returns false for a name it does not know.
double coarse_solve_flops(ts_handle h);
bool block_time_kernel(ts_handle h, const std::string& k, std::function<void()>& run, double& fl, double& by) {
  if (k.size() < 2 || k[0] != 'b') return false;
  if (!block_path_applies(h, 2)) throw TsError(TS_ERR_INVALID, "the block path needs a mixed-precision 2D design");
  balloc(h);
  {
    // scalars that never stop, so that every launch does its full work
    BScalars hs{};
    TS_CUDA(cudaMemcpyAsync(&hs, h->bsc, sizeof(hs), cudaMemcpyDeviceToHost, h->ctx->stream));
    TS_CUDA(cudaStreamSynchronize(h->ctx->stream));
    hs.done = 0;
    hs.maxit = 1 << 30;
    hs.rtol = hs.etol = 0.0;
    hs.hist_cap = 0;
    hs.done_out = nullptr;
    for (int c = 0; c < TS_NB; ++c) {
      hs.cdone[c] = 0;
      if (!(hs.ff[c] > 0.0)) hs.ff[c] = 1.0;
    }
    TS_CUDA(cudaMemcpyAsync(h->bsc, &hs, sizeof(hs), cudaMemcpyHostToDevice, h->ctx->stream));
  }
  const Geom& g = h->g;
  const double nd = (double)g.ndof, nn = (double)g.n_nodes, V8 = 8.0 * TS_NB, V4 = 4.0 * TS_NB;
  if (k == "bspmv") {
    // q = K p for every column with p = z + beta p_old formed on the fly;
    // alpha is left to the iteration (no scalars here)
    run = [h]() {
      launch_bspmv(h, nullptr, h->zb, h->pb[0], h->pb[1], h->zoldb, h->qb, nullptr, h->bsc, nullptr);
    };
    fl = TS_NB * (2.0 * 36.0 * nn + 2.0 * nd);
    by = 8.0 * 36.0 * nn + nd + V8 * nd * 5.0;  // stencil, mask; z, p_old read, p, z_old, q written
  } else if (k == "bupdate_xr") {
    run = [h]() {
      ts_launch(h, false, k_bupdate_xr, bvec_blocks(h), BV_THREADS, 0, h->ctx->stream, h->bsc, h->g.ndof * TS_NB,
                h->xb, h->rb, (const double*)h->pb[1], (const double*)h->qb, (const double*)h->fb,
                (const double*)h->zoldb, h->r32b, h->bpart_xr);
    };
    fl = TS_NB * 10.0 * nd;
    by = V8 * nd * 8.0 + V4 * nd;  // x, r, p, q, f, z_old read; x, r written; r32 written
  } else if (k == "blocal_solve") {
    run = [h]() { launch_blocal_solve(h, h->r32b, h->zloc32b); };
    const double NC = 6.0;
    for (const BLDesc& d : h->sub_desc_h) {
      const double w = d.w, nb = d.nb;
      const double a = (double)(d.w / 4);
      const double vpk = 8.0 * a * (a + 1) + (w - 4.0 * a) * 4.0 * (a + 1);
      by += nb * (vpk + 2.0 * w * NC) * 4.0 + 2.0 * nb * w * V4;
      fl += TS_NB * 2.0 * ((2.0 * nb - 1.0) * w * (w + 1) + 2.0 * (nb - 1) * w * NC);
    }
  } else if (k == "brestrict" || k == "bcoarse_solve" || k == "bprolong") {
    if (h->nc == 0) throw TsError(TS_ERR_INVALID, "no coarse space");
    if (k == "brestrict") {
      run = [h]() { launch_brestrict(h, h->r32b, h->r0b); };
      fl = TS_NB * 2.0 * (double)h->W_len;
      by = 4.0 * (double)h->W_len + V4 * nd + V8 * h->nc;
    } else if (k == "bcoarse_solve") {
      run = [h]() { launch_bcoarse_solve(h); };
      fl = TS_NB * coarse_solve_flops(h);
      by = coarse_solve_flops(h) / 2.0 * 4.0 + 4.0 * V8 * h->nc;
    } else {
      run = [h]() { launch_bprolong(h, h->zloc32b, h->u0fb, h->zb, h->bpart_p, h->rb, BPcgTail{}); };
      fl = TS_NB * 2.0 * (double)h->W_len;
      by = 4.0 * (double)h->W_len + V4 * (double)h->zloc_len + V4 * h->nc + 2.0 * V8 * nd;
    }
  } else {
    throw TsError(TS_ERR_INVALID, "unknown kernel name " + k);
  }
  return true;
}
