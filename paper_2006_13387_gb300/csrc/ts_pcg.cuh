// PCG scalars kept on the device and host entry points of ts_pcg.cu.
#pragma once
#include <vector>

#include "ts_internal.cuh"
#include "ts_reduce.cuh"

#define TS_EDELAY 4

struct DevScalars {
  double rzs[2];  // r_k.z_k in slot k & 1 (read and written in the same kernel)
  double rzo, pq, alpha, beta, rr, ff, fx, rel, energy_est;
  double rtol, etol;
  double terms[TS_EDELAY];
  int iter, done, converged, status, maxit, flexible, hist_cap;
  double* alpha_hist;
  double* beta_hist;
  int* done_out;
};

// ---------------------------------------------------------------------------
// Scalar steps of the PCG iteration, run by the last block of the kernel that
// produced their per-block partial sums (a block learns that it is last from
// an atomic counter after a memory fence; it sums the partials in a fixed
// order, so the result is the same on every run, and resets the counter).
// ---------------------------------------------------------------------------
// Only thread 0 of a block writes its partials, so its counter increment
// with release-acquire semantics at GPU scope orders them; the block that
// sees the final count acquires every other block's partials, and the
// barrier passes that on to its other threads (which read the partials
// through L2).
__device__ __forceinline__ bool pcg_last_block(unsigned* counter) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned total = gridDim.x * gridDim.y * gridDim.z;
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;\n" : "=r"(old) : "l"(counter) : "memory");
    s_last = (old == total - 1) ? 1 : 0;
  }
  __syncthreads();
  return s_last != 0;
}

__device__ __forceinline__ void pcg_set_done(DevScalars* S) {
  S->done = 1;
  if (S->done_out) *S->done_out = 1;
}

// the partial sums of n blocks, STRIDE values per block: every thread loads
// up to PU of them at once (all loads in flight), then one block reduction
template <int NT, int N, int STRIDE>
__device__ __forceinline__ void pcg_sum_partials(const double* partials, int n, double (&v)[N], int first = 0) {
  constexpr int PU = 4;
  for (int i0 = 0; i0 < n; i0 += NT * PU) {
    double buf[PU][N];
#pragma unroll
    for (int u = 0; u < PU; ++u) {
      const int i = i0 + u * NT + threadIdx.x;
#pragma unroll
      for (int j = 0; j < N; ++j) buf[u][j] = (i < n) ? __ldcg(partials + (int64_t)STRIDE * i + first + j) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < PU; ++u)
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] += buf[u][j];
  }
}

// alpha = r_k.z_k / p.Kp from the SpMV's partials of p.Kp
template <int NT>
__device__ void pcg_alpha_last(DevScalars* S, const double* partials, int n, unsigned* counter) {
  double v[1] = {0.0};
  pcg_sum_partials<NT, 1, 1>(partials, n, v);
  block_sum_n<NT, 1>(v);
  if (threadIdx.x == 0) {
    const double pq = v[0];
    const int k = S->iter;
    const double rz = S->rzs[k & 1];
    S->pq = pq;
    if (!(pq > 0.0) || !(rz == rz)) {
      S->status = TS_ERR_BREAKDOWN;
      S->alpha = 0.0;
      pcg_set_done(S);
    } else {
      S->alpha = rz / pq;
      if (k < S->hist_cap) S->alpha_hist[k] = S->alpha;
    }
    *counter = 0u;
  }
}

// The prolongation's last block: convergence test from the x/r update's
// partials of r.r, f.p, r.z_old (3 per block, n_xr blocks), then beta from
// its own partials of r.z (2 per block, n_pro blocks).  The decisions avoid
// divisions (||r||^2 <= rtol^2 ||f||^2, energy sum <= etol^2 f.x); the
// reported relative residual and energy estimate are formed on the host.
template <int NT>
__device__ void pcg_conv_beta_last(DevScalars* S, const double* xr_partials, int n_xr, const double* pro_partials,
                                   int n_pro, unsigned* counter) {
  if (S->done) {
    if (threadIdx.x == 0) *counter = 0u;
    return;
  }
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  {
    double a[3] = {0.0, 0.0, 0.0}, b[1] = {0.0};
    pcg_sum_partials<NT, 3, 3>(xr_partials, n_xr, a);
    pcg_sum_partials<NT, 1, 2>(pro_partials, n_pro, b);
    v[0] = a[0];
    v[1] = a[1];
    v[2] = a[2];
    v[3] = b[0];
  }
  block_sum_n<NT, 4>(v);
  if (threadIdx.x == 0) {
    const double rr = v[0], fp = v[1], rzo = v[2], rz = v[3];
    S->rr = rr;
    S->rzo = rzo;
    S->fx += S->alpha * fp;
    const int k = S->iter;
    S->terms[k % TS_EDELAY] = S->alpha * S->rzs[k & 1];
    S->iter = k + 1;
    bool ok_e = true;
    if (S->etol > 0.0) {
      if (k + 1 >= TS_EDELAY) {
        double e = 0.0;
        for (int d = 0; d < TS_EDELAY; ++d) e += S->terms[d];
        ok_e = e <= S->etol * S->etol * fmax(S->fx, 1e-300);
      } else {
        ok_e = false;
      }
    }
    if (!(rr == rr)) {
      S->status = TS_ERR_BREAKDOWN;
      pcg_set_done(S);
    } else if (rr <= S->rtol * S->rtol * S->ff && ok_e) {
      S->converged = 1;
      pcg_set_done(S);
    } else if (S->iter >= S->maxit) {
      S->status = TS_NOT_CONVERGED;
      pcg_set_done(S);
    }
    // beta (iteration count now k+1: r_{k+1}.z_{k+1} goes to slot (k+1) & 1)
    const double rz_old = S->rzs[k & 1];
    S->beta = (S->flexible ? (rz - rzo) : rz) / rz_old;
    S->rzs[(k + 1) & 1] = rz;
    if (k < S->hist_cap) S->beta_hist[k] = rz / rz_old;
    *counter = 0u;
  }
}

struct PcgResult {
  int iters, converged, status;
  double rel, energy_est, cond, ff;
  bool want_cond;
};

void pcg_alloc(ts_handle h);
ts_status pcg_run(ts_handle h, bool warm, double rtol, double etol, PcgResult* res);
ts_status solve_one(ts_handle h, bool warm, double rtol, ts_stats* stats);
// z = M^{-1} r (r32_ready: the FP32 copy of r used by the mixed path is current)
void launch_apply_M(ts_handle h, const double* r, double* z, double* partials, const double* dv1, const double* dv2,
                    bool r32_ready = false);
void ts_launch_apply_M(ts_handle h, const double* r, double* z, double* partials, const double* dv1,
                       const double* dv2, bool r32_ready, PcgTail tail);
// FP32 copy of r into h->r32 (mixed precision: the level-1 gather and the
// coarse restriction read it)
void prepare_r32(ts_handle h, const double* r);
double lanczos_cond_host(const std::vector<double>& al, const std::vector<double>& be, int k);
int prolong_blocks(const Geom& g);
// r = f - K x in double-double arithmetic, rounded to FP64; partials[2*b] of r.r
void launch_residual_dd(ts_handle h, const double* f, const double* x, double* r, double* partials);
