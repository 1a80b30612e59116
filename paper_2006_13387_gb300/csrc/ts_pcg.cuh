// PCG scalars kept on the device and host entry points of ts_pcg.cu.
#pragma once
#include <vector>

#include "ts_internal.cuh"

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

struct PcgResult {
  int iters, converged, status;
  double rel, energy_est, cond, ff;
  bool want_cond;
};

void pcg_alloc(ts_handle h);
ts_status pcg_run(ts_handle h, bool warm, double rtol, double etol, PcgResult* res);
ts_status solve_one(ts_handle h, bool warm, double rtol, ts_stats* stats);
void launch_apply_M(ts_handle h, const double* r, double* z, double* partials, const double* dv1, const double* dv2);
double lanczos_cond_host(const std::vector<double>& al, const std::vector<double>& be, int k);
int prolong_blocks(const Geom& g);
// r = f - K x in double-double arithmetic, rounded to FP64; partials[2*b] of r.r
void launch_residual_dd(ts_handle h, const double* f, const double* x, double* r, double* partials);
