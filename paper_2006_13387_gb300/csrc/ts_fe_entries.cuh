// Device helpers shared by the level-1 and heat-eigenproblem kernels:
// entries of the FE matrices restricted to an element box (assembled on the
// fly: elasticity of Sec. 1.1, heat operator of Sec. 4.1), 16-byte asynchronous copies
// (cp.async) into shared memory, and the quad (4-lane) sum.
#pragma once
#include "ts_internal.cuh"

// ---------------------------------------------------------------------------
// Entries of the FE matrices restricted to an element box.
// Node coordinates are global; the box [elo, ehi) bounds the elements that
// contribute (Neumann on the box boundary for the heat problems; for the
// level-1 blocks every contributing element lies inside the box anyway).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int q4_local(int ox, int oy) { return oy == 0 ? ox : 3 - ox; }
__device__ __forceinline__ int hex8_local(int ox, int oy, int oz) { return 4 * oz + (oy == 0 ? ox : 3 - ox); }

// K entry between (node a, comp ca) and (node b, comp cb) of the elasticity
// matrix with element stiffness KE (dofs per node DIM), elements in [elo, ehi).
template <int DIM>
__device__ double elas_entry(const Geom& g, const double* __restrict__ E, const double* __restrict__ KE,
                             const int* a, int ca, const int* b, int cb, const int* elo, const int* ehi) {
  int lo[3], hi[3];
  for (int d = 0; d < DIM; ++d) {
    int dd = a[d] - b[d];
    if (dd > 1 || dd < -1) return 0.0;
    lo[d] = max(max(a[d], b[d]) - 1, elo[d]);
    hi[d] = min(min(a[d], b[d]), ehi[d] - 1);
    if (lo[d] > hi[d]) return 0.0;
  }
  double s = 0.0;
  if (DIM == 2) {
    for (int ey = lo[1]; ey <= hi[1]; ++ey)
      for (int ex = lo[0]; ex <= hi[0]; ++ex) {
        int la = q4_local(a[0] - ex, a[1] - ey), lb = q4_local(b[0] - ex, b[1] - ey);
        s += E[(int64_t)ey * g.nx + ex] * KE[(2 * la + ca) * 8 + 2 * lb + cb];
      }
  } else {
    for (int ez = lo[2]; ez <= hi[2]; ++ez)
      for (int ey = lo[1]; ey <= hi[1]; ++ey)
        for (int ex = lo[0]; ex <= hi[0]; ++ex) {
          int la = hex8_local(a[0] - ex, a[1] - ey, a[2] - ez), lb = hex8_local(b[0] - ex, b[1] - ey, b[2] - ez);
          s += E[((int64_t)ez * g.ny + ey) * g.nx + ex] * KE[(3 * la + ca) * 24 + 3 * lb + cb];
        }
  }
  return s;
}

// Heat (scalar Q1) entry of  kc * (kappa-stiffness) + mc * (kappa-mass),
// kappa = E_e, elements in [elo, ehi).  The unit Q1 element matrices are
// tensor products of the 1D matrices k1 = [1,-1;-1,1] and m1 = [2,1;1,2]/6:
// stiffness = sum_d k1_d prod_{e!=d} m1_e, mass = prod_d m1_d, and each
// factor only depends on whether the two nodes share that coordinate.
template <int DIM>
__device__ double heat_entry(const Geom& g, const double* __restrict__ E, const int* a, const int* b, double kc,
                             double mc, const int* elo, const int* ehi) {
  int lo[3], hi[3];
  for (int d = 0; d < DIM; ++d) {
    int dd = a[d] - b[d];
    if (dd > 1 || dd < -1) return 0.0;
    lo[d] = max(max(a[d], b[d]) - 1, elo[d]);
    hi[d] = min(min(a[d], b[d]), ehi[d] - 1);
    if (lo[d] > hi[d]) return 0.0;
  }
  double k1[DIM], m1[DIM];
  for (int d = 0; d < DIM; ++d) {
    bool same = (a[d] == b[d]);
    k1[d] = same ? 1.0 : -1.0;
    m1[d] = same ? (1.0 / 3.0) : (1.0 / 6.0);
  }
  double ks = 0.0, ms = 1.0;
  for (int d = 0; d < DIM; ++d) {
    double t = k1[d];
    for (int e2 = 0; e2 < DIM; ++e2)
      if (e2 != d) t *= m1[e2];
    ks += t;
    ms *= m1[d];
  }
  const double ent = kc * ks + mc * ms;
  double s = 0.0;
  if (DIM == 2) {
    for (int ey = lo[1]; ey <= hi[1]; ++ey)
      for (int ex = lo[0]; ex <= hi[0]; ++ex) s += E[(int64_t)ey * g.nx + ex];
  } else {
    for (int ez = lo[2]; ez <= hi[2]; ++ez)
      for (int ey = lo[1]; ey <= hi[1]; ++ey)
        for (int ex = lo[0]; ex <= hi[0]; ++ex) s += E[((int64_t)ez * g.ny + ey) * g.nx + ex];
  }
  return s * ent;
}

// 16-byte asynchronous global -> shared copies (cp.async, L2 only)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// four threads per row: sum over the lane's residue class, then two shuffles
template <class TF>
__device__ __forceinline__ TF quad_sum(TF s) {
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  return s;
}
