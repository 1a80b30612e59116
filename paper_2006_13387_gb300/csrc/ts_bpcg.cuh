// Block PCG over TS_NB right-hand sides that share every kernel launch: each
// column runs its own PCG (own alpha, beta, stopping test and energy
// estimate, Sec. 2 and Sec. 5) while the stiffness stencil, the level-1
// factors, the coarse basis rows and the coarse factor are read once per
// iteration for all columns.  Block vectors are DOF-major, [ndof][TS_NB]
// (the TS_NB values of one DOF are contiguous), FP64 unless stated.
#pragma once
#include <functional>
#include <string>
#include "ts_internal.cuh"
#include "ts_pcg.cuh"

#define TS_NB 8  // columns of the block path

struct BScalars {
  double rzs[2][TS_NB];  // r_k.z_k per column, slot k & 1
  double rzo[TS_NB], pq[TS_NB], alpha[TS_NB], beta[TS_NB], rr[TS_NB], ff[TS_NB], fx[TS_NB];
  double terms[TS_EDELAY][TS_NB];
  double rtol, etol;
  int iter;                // iterations run by the block
  int it[TS_NB];           // iterations of each column when it stopped
  int cdone[TS_NB];        // column stopped (converged, breakdown or max_iter)
  int converged[TS_NB], status[TS_NB];
  int ncols;               // live columns (the rest are zero padding)
  int done, maxit, flexible, hist_cap;
  double* alpha_hist;      // [hist_cap][TS_NB] (Lanczos estimate per column)
  double* beta_hist;
  int* done_out;
};

// Per-column sums of K values held by every thread of a block of NT threads,
// where thread t's values belong to column t % TS_NB (the grid-stride kernels
// over [n][TS_NB] keep each thread on one column): lanes of one column are
// added by shuffles, the warps in a fixed order.  Results in threads
// 0 .. TS_NB-1 (thread c holds column c's K sums).
template <int NT, int K>
__device__ __forceinline__ void bsum_by_col(double (&v)[K]) {
  static_assert(TS_NB == 8, "lane grouping assumes 8 columns");
  __shared__ double sh[NT / 32][K][TS_NB];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    double s = v[j];
    s += __shfl_down_sync(0xffffffffu, s, 16);
    s += __shfl_down_sync(0xffffffffu, s, 8);
    v[j] = s;
  }
  __syncthreads();
  if (lane < TS_NB)
#pragma unroll
    for (int j = 0; j < K; ++j) sh[wid][j][lane] = v[j];
  __syncthreads();
  if (threadIdx.x < TS_NB) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < NT / 32; ++w) s += sh[w][j][threadIdx.x];
      v[j] = s;
    }
  }
  __syncthreads();
}

// Per-column sums when every thread holds all TS_NB columns (v[j][c]):
// fixed shuffle tree per value, warps in a fixed order; results in thread 0.
template <int NT, int K>
__device__ __forceinline__ void bsum_all_cols(double (&v)[K][TS_NB]) {
  __shared__ double sh[NT / 32][K][TS_NB];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < K; ++j)
#pragma unroll
    for (int c = 0; c < TS_NB; ++c) v[j][c] = warp_sum(v[j][c]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < K; ++j)
#pragma unroll
      for (int c = 0; c < TS_NB; ++c) sh[wid][j][c] = v[j][c];
  __syncthreads();
  if (threadIdx.x < K * TS_NB) {
    const int j = threadIdx.x / TS_NB, c = threadIdx.x % TS_NB;
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) s += sh[w][j][c];
    sh[0][j][c] = s;  // (each (j, c) read and written by its own thread)
  }
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < K; ++j)
#pragma unroll
      for (int c = 0; c < TS_NB; ++c) v[j][c] = sh[0][j][c];
  __syncthreads();
}

// Sum over the blocks of per-column partials laid out [n][STRIDE][TS_NB]
// (value j of block b, column c at (b * STRIDE + j) * TS_NB + c) by all NT
// threads of the last block: thread t takes column t % TS_NB and blocks
// t / TS_NB, t / TS_NB + NT / TS_NB, ...; then the per-column tree of
// bsum_by_col.  Results in threads 0 .. TS_NB-1.
template <int NT, int K, int STRIDE>
__device__ __forceinline__ void bsum_partials(const double* partials, int n, double (&v)[K], int first = 0) {
  const int c = threadIdx.x % TS_NB, g = threadIdx.x / TS_NB;
  constexpr int NG = NT / TS_NB;
#pragma unroll
  for (int j = 0; j < K; ++j) v[j] = 0.0;
  for (int b0 = 0; b0 < n; b0 += 4 * NG) {
    double buf[4][K];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int b = b0 + u * NG + g;
#pragma unroll
      for (int j = 0; j < K; ++j)
        buf[u][j] = (b < n) ? __ldcg(partials + ((int64_t)b * STRIDE + first + j) * TS_NB + c) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int j = 0; j < K; ++j) v[j] += buf[u][j];
  }
  bsum_by_col<NT, K>(v);
}

// alpha_c = r_c.z_c / p_c.Kp_c for every column from the SpMV's partials
// ([n][TS_NB]); a stopped column gets alpha = 0 (its x and r stay).
template <int NT>
__device__ void bpcg_alpha_last(BScalars* S, const double* partials, int n, unsigned* counter) {
  double v[1];
  bsum_partials<NT, 1, 1>(partials, n, v);
  if (threadIdx.x < TS_NB) {
    const int c = threadIdx.x;
    const double s = v[0];
    const int k = S->iter;
    const double rz = S->rzs[k & 1][c];
    S->pq[c] = s;
    if (S->cdone[c]) {
      S->alpha[c] = 0.0;
    } else if (!(s > 0.0) || !(rz == rz)) {
      S->status[c] = TS_ERR_BREAKDOWN;
      S->alpha[c] = 0.0;
      S->cdone[c] = 1;
      S->it[c] = k;
    } else {
      S->alpha[c] = rz / s;
      if (k < S->hist_cap) S->alpha_hist[(int64_t)k * TS_NB + c] = S->alpha[c];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
}

// The prolongation's last block: per column the convergence test from the x/r
// update's partials (rr, fp, rzo: [n_xr][3][TS_NB]) and beta from its own
// partials of r.z ([n_pro][TS_NB]); sets the block's stop flag once every
// column has stopped.  The decisions avoid divisions, as in the one-column
// iteration.
template <int NT>
__device__ void bpcg_conv_beta_last(BScalars* S, const double* xr_partials, int n_xr, const double* pro_partials,
                                    int n_pro, unsigned* counter) {
  if (S->done) {
    if (threadIdx.x == 0) *counter = 0u;
    return;
  }
  __shared__ int s_live;
  double a[3], b1[1];
  bsum_partials<NT, 3, 3>(xr_partials, n_xr, a);
  bsum_partials<NT, 1, 1>(pro_partials, n_pro, b1);
  if (threadIdx.x == 0) s_live = 0;
  __syncthreads();
  if (threadIdx.x < TS_NB) {
    const int c = threadIdx.x;
    const double rr = a[0], fp = a[1], rzo = a[2], rz = b1[0];
    const int k = S->iter;
    if (!S->cdone[c]) {
      S->rr[c] = rr;
      S->rzo[c] = rzo;
      S->fx[c] += S->alpha[c] * fp;
      S->terms[k % TS_EDELAY][c] = S->alpha[c] * S->rzs[k & 1][c];
      bool ok_e = true;
      if (S->etol > 0.0) {
        if (k + 1 >= TS_EDELAY) {
          double e = 0.0;
          for (int d = 0; d < TS_EDELAY; ++d) e += S->terms[d][c];
          ok_e = e <= S->etol * S->etol * fmax(S->fx[c], 1e-300);
        } else {
          ok_e = false;
        }
      }
      if (!(rr == rr)) {
        S->status[c] = TS_ERR_BREAKDOWN;
        S->cdone[c] = 1;
      } else if (rr <= S->rtol * S->rtol * S->ff[c] && ok_e) {
        S->converged[c] = 1;
        S->cdone[c] = 1;
      } else if (k + 1 >= S->maxit) {
        S->status[c] = TS_NOT_CONVERGED;
        S->cdone[c] = 1;
      }
      if (S->cdone[c]) S->it[c] = k + 1;
      const double rz_old = S->rzs[k & 1][c];
      S->beta[c] = S->cdone[c] ? 0.0 : (S->flexible ? (rz - rzo) : rz) / rz_old;
      S->rzs[(k + 1) & 1][c] = rz;
      if (k < S->hist_cap) S->beta_hist[(int64_t)k * TS_NB + c] = rz / rz_old;
    } else {
      S->beta[c] = 0.0;
      S->rzs[(k + 1) & 1][c] = S->rzs[k & 1][c];
    }
    if (!S->cdone[c]) atomicAdd(&s_live, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    S->iter = S->iter + 1;
    if (s_live == 0) {
      S->done = 1;
      if (S->done_out) *S->done_out = 1;
    }
    *counter = 0u;
  }
}

struct BPcgTail {
  BScalars* S = nullptr;
  unsigned* counter = nullptr;
  const double* xr_partials = nullptr;  // [n_xr][3][TS_NB]
  int n_xr = 0;
};

// host entry points (ts_bpcg.cu and the kernels' translation units)
bool block_path_applies(ts_handle h, int nrhs);
// ts_time_kernel names of the block path ("bspmv", "bupdate_xr",
// "blocal_solve", "brestrict", "bcoarse_solve", "bprolong"): the launch and
// its algorithmic FLOPs and bytes; false when k is not one of them
bool block_time_kernel(ts_handle h, const std::string& k, std::function<void()>& run, double& fl, double& by);
ts_status block_solve(ts_handle h, const double* f, double* u, int nrhs, double rtol, ts_stats* stats);
// q = K p (2D stencil), p = z + beta p_old per column formed while staging
// (z_old = z for the flexible variant), partials of p.q and alpha from the
// last block; with z == nullptr the product of x alone (no scalars)
void launch_bspmv(ts_handle h, const double* x, const double* z, const double* p_old, double* p_new, double* z_old,
                  double* q, double* partials, BScalars* S, unsigned* counter);
int bspmv_blocks(const Geom& g);
// level 1 over TS_NB columns: zloc (FP32, [local][TS_NB]) from r32 ([ndof][TS_NB])
void launch_blocal_solve(ts_handle h, const float* r32, float* zloc);
// coarse restriction r0 = R_0 r ([nc][TS_NB] FP64) from r32, and the BCR
// stages with TS_NB columns
void launch_brestrict(ts_handle h, const float* r32, double* r0);
void launch_bcoarse_solve(ts_handle h);  // h->r0b -> h->u0b, h->u0fb
// prolongation z = sum R_i^T zloc_i + R_0^T u0 with the partials of dv.z per
// column; inside the iteration the last block runs the stopping test and beta
int bprolong_blocks(const Geom& g);
void launch_bprolong(ts_handle h, const float* zloc, const float* u0f, double* z, double* partials, const double* dv,
                     BPcgTail tail);
