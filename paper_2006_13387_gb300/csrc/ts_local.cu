// Level 1 of the preconditioner (Sec. 2, local Dirichlet problems):
//   M_1^{-1} r = sum_i R_i^T K_i^{-1} R_i r,  K_i = R_i K R_i^T,
// with R_i the 0/1 restriction to the free DOFs of the nodes of D'_i.
// Each K_i is block-tridiagonal by node lines (2D rows, 3D planes; A_kk the
// line blocks, A_{k,k+-1} the sparse couplings of neighbouring lines).  The
// factor is a twisted block LU: the top half is eliminated downwards and the
// bottom half upwards toward the middle line m,
//   S_k  = A_kk - A_{k,k-1} S_{k-1}^{-1} A_{k-1,k}   (k < m)
//   S'_k = A_kk - A_{k,k+1} S'_{k+1}^{-1} A_{k+1,k}  (k > m)
//   S_m  = A_mm - both neighbours' terms,
// so that the solve runs both halves at once (two thread groups) and its
// chain of dependent line steps is about nb + 1 long instead of 2 nb - 1:
//   forward   u_k = S_k^{-1} (r_k - A_{k,k-/+1} u_{k-/+1})      (each half)
//   middle    x_m = S_m^{-1} (r_m - A_{m,m-1} u_{m-1} - A_{m,m+1} u_{m+1})
//   backward  x_k = u_k - S_k^{-1} A_{k,k+/-1} x_{k+/-1}          (each half)
// Stored per line: the S_k^{-1} form and the coupling stencils of the line's
// rows to both neighbouring lines (A_{k,k-1}, A_{k,k+1} restricted to the
// 3 (2D) or 9 (3D) neighbouring nodes of each row's node):
//  * FP64 path: the dense inverse M_k (one GEMV a step);
//  * mixed path: V_k = L_k^{-1} from S_k = L_k L_k^T, packed lower triangle,
//    applied as V_k^T (V_k y).  The Gram form keeps the FP32 operator
//    positive definite even when cond(S_k) exceeds 1/eps_32 (high contrast),
//    where rounding the explicit inverse to FP32 does not.
// The factor runs in FP64, one CTA per subdomain with all threads busy.  A
// node-owner gather adds the overlapping local solutions (no atomics, fixed
// sum order).
#include <algorithm>

#include "ts_fe_entries.cuh"
#include "ts_internal.cuh"
#include "ts_reduce.cuh"
#include "ts_bpcg.cuh"
#include "ts_bulk.cuh"

// element stiffness (E = 1), this translation unit's copy
static __constant__ double c_KE[TS_KE_SLOTS * TS_KE_SIZE];

void upload_KE_local(int slot, const std::vector<double>& KE) {
  TS_CUDA(cudaMemcpyToSymbol(c_KE, KE.data(), KE.size() * sizeof(double), sizeof(double) * TS_KE_SIZE * slot,
                             cudaMemcpyHostToDevice));
}

// ---------------------------------------------------------------------------
// box helpers (device)
// ---------------------------------------------------------------------------
struct SubBox {
  int nlo[3], nhi[3], elo[3], ehi[3], nb3[3];
};

__device__ __forceinline__ void sub_box(const Geom& g, const AxisTables& ax, int s, SubBox& b) {
  int sx = s % g.nsub[0];
  int t = s / g.nsub[0];
  int sy = (g.dim == 2) ? t : t % g.nsub[1];
  int sz = (g.dim == 2) ? 0 : t / g.nsub[1];
  int si[3] = {sx, sy, sz};
  for (int d = 0; d < g.dim; ++d) {
    b.nlo[d] = ax.sub_lo[d][si[d]];
    b.nhi[d] = ax.sub_hi[d][si[d]];
    b.elo[d] = ax.sub_elo[d][si[d]];
    b.ehi[d] = ax.sub_ehi[d][si[d]];
    b.nb3[d] = b.nhi[d] - b.nlo[d] + 1;
  }
}

// the same with the dimension known at compile time (registers, no stack)
template <int DIM>
__device__ __forceinline__ void sub_box_t(const Geom& g, const AxisTables& ax, int s, SubBox& b) {
  const int sx = s % g.nsub[0];
  const int t = s / g.nsub[0];
  const int si[3] = {sx, (DIM == 2) ? t : t % g.nsub[1], (DIM == 2) ? 0 : t / g.nsub[1]};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (d < DIM) {
      b.nlo[d] = ax.sub_lo[d][si[d]];
      b.nhi[d] = ax.sub_hi[d][si[d]];
      b.elo[d] = ax.sub_elo[d][si[d]];
      b.ehi[d] = ax.sub_ehi[d][si[d]];
      b.nb3[d] = b.nhi[d] - b.nlo[d] + 1;
    } else {
      b.nlo[d] = b.nhi[d] = b.elo[d] = 0;
      b.ehi[d] = b.nb3[d] = 1;
    }
  }
}

__device__ __forceinline__ int64_t node_id(const Geom& g, const int* a) {
  if (g.dim == 2) return (int64_t)a[1] * (g.nx + 1) + a[0];
  return ((int64_t)a[2] * (g.ny + 1) + a[1]) * (g.nx + 1) + a[0];
}

template <int DIM>
struct ElasAsm {
  Geom g;
  const double* E;
  const uint8_t* fm;
  SubBox b;
  __device__ void node_of(int k, int p, int* a, int& c) const {
    c = p % DIM;
    int t = p / DIM;
    if (DIM == 2) {
      a[0] = b.nlo[0] + t;
      a[1] = b.nlo[1] + k;
    } else {
      a[0] = b.nlo[0] + t % b.nb3[0];
      a[1] = b.nlo[1] + t / b.nb3[0];
      a[2] = b.nlo[2] + k;
    }
  }
  __device__ double entry(int kr, int p, int kc, int q) const {
    int a[3], bb[3], ca, cb;
    node_of(kr, p, a, ca);
    node_of(kc, q, bb, cb);
    bool fa = fm[DIM * node_id(g, a) + ca], fb = fm[DIM * node_id(g, bb) + cb];
    if (!fa || !fb) return (kr == kc && p == q) ? 1.0 : 0.0;
    return elas_entry<DIM>(g, E, c_KE + g.ke * TS_KE_SIZE, a, ca, bb, cb, b.elo, b.ehi);
  }
};

// ---------------------------------------------------------------------------
// Stored solve factors per line block (rows start on 16-byte boundaries in
// FP32 and FP64; padding is zero):
//  * M form: w rows of lv1_ld(w) = round_up(w, 4) entries;
//  * V form: row i holds round_up(i+1, 4) entries from column 0, at
//    lv1_vrow(i).
// ---------------------------------------------------------------------------
__host__ __device__ inline int lv1_ld(int w) { return (w + 3) & ~3; }
__host__ __device__ inline int64_t lv1_vrow(int i) {
  const int64_t a = i >> 2;
  return 8 * a * (a + 1) + (int64_t)(i - 4 * a) * 4 * (a + 1);
}
// the S^{-1} form of a line block (V packed or M dense)
__host__ __device__ inline int64_t lv1_sform(int w, bool vform) {
  return vform ? lv1_vrow(w) : (int64_t)w * lv1_ld(w);
}
// a stored line block: the S^{-1} form, then the coupling stencils of its
// rows to the previous and to the next line (w x NC each, NC = 6 in 2D and
// 27 in 3D: in-line node offsets times components), rounded to 4 elements
__host__ __device__ inline int64_t lv1_stride(int w, bool vform, int dim) {
  const int NC = (dim == 2) ? 6 : 27;
  return (lv1_sform(w, vform) + 2 * (int64_t)w * NC + 3) & ~(int64_t)3;
}

// ---------------------------------------------------------------------------
// twisted block LU factor, FP64, one CTA per subdomain
// ---------------------------------------------------------------------------
// couplings of a line row to the neighbouring line: in-line node offsets
// (2D: dx in -1..1; 3D: (dx, dy) in -1..1^2) times the DIM components
template <int DIM>
struct Lv1Cpl {
  static constexpr int NO = (DIM == 2) ? 3 : 9;
  static constexpr int NC = NO * DIM;
};
// column (line position) of slot s of row p, or -1 outside the line box
template <int DIM>
__device__ __forceinline__ int lv1_cpl_col(int p, int s, int nbx, int nby) {
  const int o = s / DIM, c = s % DIM, t = p / DIM;
  if (DIM == 2) {
    const int x = t + o - 1;
    return (x >= 0 && x < nbx) ? DIM * x + c : -1;
  }
  const int x = t % nbx + o % 3 - 1, y = t / nbx + o / 3 - 1;
  return (x >= 0 && x < nbx && y >= 0 && y < nby) ? DIM * (x + nbx * y) + c : -1;
}

// shared memory (doubles) of the factor: S, T (= V), M_top, M_bottom (w^2
// each) and the coupling stencil (w * NC)
__host__ inline size_t lv1_factor_smem(int w, int dim) {
  const int NC = (dim == 2) ? 6 : 27;
  return ((size_t)4 * w * w + (size_t)w * NC) * sizeof(double);
}

template <int DIM>
__global__ void __launch_bounds__(256) k_local_factor(Geom g, AxisTables ax, const double* __restrict__ E,
                                                      const uint8_t* __restrict__ fm, const BLDesc* __restrict__ desc,
                                                      double* __restrict__ pv64, float* __restrict__ pv32,
                                                      int* __restrict__ status) {
  extern __shared__ double fsm[];
  constexpr int NC = Lv1Cpl<DIM>::NC;
  __shared__ int bad;
  __shared__ double s_inv;
  const int s = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  ElasAsm<DIM> A;
  A.g = g;
  A.E = E;
  A.fm = fm;
  sub_box_t<DIM>(g, ax, s, A.b);
  const BLDesc d = desc[s];
  const int w = d.w, nb = d.nb, ld = lv1_ld(w), m = nb / 2;
  const int nbx = A.b.nb3[0], nby = A.b.nb3[1];
  const bool vf = pv32 != nullptr;
  const int64_t ps = lv1_stride(w, vf, DIM), pform = lv1_sform(w, vf);
  double* S = fsm;
  double* T = S + w * w;  // Schur product, then V = L^{-1}
  double* Mt = T + w * w;
  double* Mb = Mt + w * w;
  double* C = Mb + w * w;
  if (tid == 0) bad = 0;
  // S -= A_{k,kp} Mp A_{kp,k}
  auto schur = [&](int k, int kp, const double* Mp) {
    for (int e = tid; e < w * NC; e += nt) {
      const int p = e / NC, q = lv1_cpl_col<DIM>(p, e % NC, nbx, nby);
      C[e] = (q >= 0) ? A.entry(k, p, kp, q) : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < w * w; e += nt) {
      const int p = e / w, c = e % w;
      double t = 0.0;
#pragma unroll
      for (int sl = 0; sl < NC; ++sl) {
        const int q = lv1_cpl_col<DIM>(p, sl, nbx, nby);
        if (q >= 0) t = fma(C[p * NC + sl], Mp[q * w + c], t);
      }
      T[e] = t;
    }
    __syncthreads();
    for (int e = tid; e < w * w; e += nt) {
      const int p = e / w, p2 = e % w;
      double t = 0.0;
#pragma unroll
      for (int sl = 0; sl < NC; ++sl) {
        const int q = lv1_cpl_col<DIM>(p2, sl, nbx, nby);
        if (q >= 0) t = fma(T[p * w + q], C[p2 * NC + sl], t);
      }
      S[e] -= t;
    }
    __syncthreads();
  };
  // factor line k: S = A_kk - (Schur terms of its predecessors); store its
  // S^{-1} form and leave M = S^{-1} in Mout
  auto line = [&](int k, int kp0, const double* Mp0, int kp1, const double* Mp1, double* Mout) {
    __syncthreads();
    for (int e = tid; e < w * w; e += nt) {
      const int i = e / w, j = e % w;
      S[e] = (j <= i) ? A.entry(k, i, k, j) : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < w * w; e += nt) {
      const int i = e / w, j = e % w;
      if (j > i) S[e] = S[j * w + i];
    }
    __syncthreads();
    if (kp0 >= 0) schur(k, kp0, Mp0);
    if (kp1 >= 0) schur(k, kp1, Mp1);
    // Cholesky S = L L^T in place (lower triangle)
    for (int j = 0; j < w; ++j) {
      if (tid == 0) {
        double pj = S[j * w + j];
        if (!(pj > 0.0)) {
          bad = 1;
          pj = 1.0;
        }
        pj = sqrt(pj);
        S[j * w + j] = pj;
        s_inv = 1.0 / pj;
      }
      __syncthreads();
      const double inv = s_inv;
      for (int i = j + 1 + tid; i < w; i += nt) S[i * w + j] *= inv;
      __syncthreads();
      const int r = w - j - 1;
      for (int e = tid; e < r * r; e += nt) {
        const int i = j + 1 + e / r, c = j + 1 + e % r;
        if (c <= i) S[i * w + c] -= S[i * w + j] * S[c * w + j];
      }
      __syncthreads();
    }
    // V = L^{-1} (row by row: row i needs rows < i)
    for (int i = 0; i < w; ++i) {
      const double li = 1.0 / S[i * w + i];
      for (int c = tid; c < w; c += nt) {
        double t = 0.0;
        if (c < i) {
          for (int q = c; q < i; ++q) t = fma(S[i * w + q], T[q * w + c], t);
          t = -t * li;
        } else if (c == i) {
          t = li;
        }
        T[i * w + c] = t;
      }
      __syncthreads();
    }
    // M = V^T V
    for (int e = tid; e < w * w; e += nt) {
      const int a = e / w, b2 = e % w;
      double t = 0.0;
      for (int q = max(a, b2); q < w; ++q) t = fma(T[q * w + a], T[q * w + b2], t);
      Mout[e] = t;
    }
    __syncthreads();
    // stored form, then the coupling stencils to lines k-1 and k+1
    const int64_t o = d.coff + (int64_t)k * ps;
    for (int e = tid; e < 2 * w * NC; e += nt) {
      const int dn = e / (w * NC), r = e % (w * NC);
      const int p = r / NC, q = lv1_cpl_col<DIM>(p, r % NC, nbx, nby);
      const int kn = dn ? k + 1 : k - 1;
      const double cv = (q >= 0 && kn >= 0 && kn < nb) ? A.entry(k, p, kn, q) : 0.0;
      if (vf)
        pv32[o + pform + e] = (float)cv;
      else
        pv64[o + pform + e] = cv;
    }
    if (vf) {
      for (int64_t e = tid; e < pform; e += nt) {
        int i = (int)sqrt(2.0 * (double)e);
        while (i > 0 && lv1_vrow(i) > e) --i;
        while (i + 1 < w && lv1_vrow(i + 1) <= e) ++i;
        const int j = (int)(e - lv1_vrow(i));
        pv32[o + e] = (j <= i) ? (float)T[i * w + j] : 0.0f;
      }
    } else {
      for (int64_t e = tid; e < pform; e += nt) {
        const int i = (int)(e / ld), j = (int)(e % ld);
        pv64[o + e] = (j < w) ? Mout[i * w + j] : 0.0;
      }
    }
    for (int64_t e = pform + 2 * w * NC + tid; e < ps; e += nt) {
      if (vf)
        pv32[o + e] = 0.0f;
      else
        pv64[o + e] = 0.0;
    }
  };
  // top half downwards, bottom half upwards, then the middle line
  for (int k = 0; k < m; ++k) line(k, k > 0 ? k - 1 : -1, Mt, -1, nullptr, Mt);
  for (int k = nb - 1; k > m; --k) line(k, k < nb - 1 ? k + 1 : -1, Mb, -1, nullptr, Mb);
  line(m, m > 0 ? m - 1 : -1, Mt, m + 1 < nb ? m + 1 : -1, Mb, Mt);  // (M of the middle line is unused)
  __syncthreads();
  if (tid == 0 && bad) atomicOr(status, 1);  // non-SPD local matrix
}

// sum_{m < len} row[m] y[m] by the 4 threads of a quad: 16-byte chunks
// c = part, part+4, ... (len a multiple of 4); the quad's sum in every lane
template <class TF>
__device__ __forceinline__ TF quad_row_dot(const TF* row, const TF* y, int len, int part) {
  using VT = typename Vec16<TF>::T;
  constexpr int N = Vec16<TF>::N;
  TF s = 0;
  for (int m = part * N; m < len; m += 4 * N)
    s += Vec16<TF>::dot(*reinterpret_cast<const VT*>(row + m), *reinterpret_cast<const VT*>(y + m));
  return quad_sum(s);
}

// column j of the packed V (rows i >= j) against z, by the 4 threads of a quad
template <class TF>
__device__ __forceinline__ TF quad_col_dot(const TF* V, const TF* z, int w, int j, int part) {
  TF s = 0;
  int i = j + part;
  // row offsets by increments: lv1_vrow(i + 4) = lv1_vrow(i) + 16 (i/4 + 1) + 4 (i % 4)
  int64_t ro = lv1_vrow(i);
  const int inc_r = 4 * (i & 3);
  int a = i >> 2;
#pragma unroll 4
  for (; i < w; i += 4) {
    s += V[ro + j] * z[i];
    ro += 16 * (a + 1) + inc_r;
    ++a;
  }
  return quad_sum(s);
}

// ---------------------------------------------------------------------------
// local solve kernel: one CTA per subdomain, two thread groups of G threads
// (the top and the bottom half of the twisted factor); the couplings take one
// thread per line row, the products four threads (a quad) per row.  Each
// group streams its half's line blocks through its own ring of DEPTH shared
// slots (16-byte cp.async, one commit group per step, DEPTH-1 in flight) and
// synchronises on its own named barrier; its last DEPTH blocks of the
// forward sweep are reused by its backward sweep.  The middle line, loaded
// up front, is solved by the whole CTA between the sweeps.
// ---------------------------------------------------------------------------
template <class TF, bool VF, class Sync>
__device__ __forceinline__ void lv1_apply(const TF* M, TF* out, bool sub, const TF* y, TF* z, int w, int ld, int part,
                                          int rq, int nq, Sync sync) {
  if (VF) {
    // (the quad shuffles need every lane: rows past w run empty loops)
    for (int i0 = 0; i0 < w; i0 += nq) {
      const int i = i0 + rq;
      const bool on = i < w;
      const TF t = quad_row_dot<TF>(M + (on ? lv1_vrow(i) : 0), y, on ? (((i + 1) + 3) & ~3) : 0, part);
      if (on && part == 0) z[i] = t;
    }
    sync();
    for (int j0 = 0; j0 < w; j0 += nq) {
      const int j = j0 + rq;
      const TF t = quad_col_dot<TF>(M, z, w, j, part);  // empty for j >= w
      if (j < w && part == 0) out[j] = sub ? out[j] - t : t;
    }
  } else {
    for (int i0 = 0; i0 < w; i0 += nq) {
      const int i = i0 + rq;
      const bool on = i < w;
      const TF t = quad_row_dot<TF>(M + (on ? (int64_t)i * ld : 0), y, on ? ld : 0, part);
      if (on && part == 0) out[i] = sub ? out[i] - t : t;
    }
  }
}

// MAXT: block size bound of the instantiation (320: four CTAs per SM, so that
// a subdomain per CTA for 152 x 4 subdomains runs in one wave)
template <int DIM, class TF, int DEPTH, bool VF, int MAXT>
__global__ void __launch_bounds__(MAXT, (MAXT <= 320) ? 4 : 2)
    k_local_solve(Geom g, AxisTables ax, const TF* __restrict__ r, const BLDesc* __restrict__ desc,
                  const TF* __restrict__ pv, const uint8_t* __restrict__ fm, const int64_t* __restrict__ zoff,
                  TF* __restrict__ zloc, int ring_stride, const int* __restrict__ done) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  constexpr int NC = Lv1Cpl<DIM>::NC;
  const int s = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int G = nt >> 1, grp = tid / G, gt = tid - grp * G;
  SubBox b;
  sub_box_t<DIM>(g, ax, s, b);
  const int nbx = b.nb3[0], nby = b.nb3[1];
  const BLDesc d = desc[s];
  const int w = d.w, nb = d.nb, ld = lv1_ld(w), m = nb / 2;
  const int cnt = (grp == 0) ? m : nb - 1 - m;  // lines of this group's half
  const int64_t ps = lv1_stride(w, VF, DIM), pform = lv1_sform(w, VF);
  const TF* F = pv + d.coff;
  // DEPTH > 0: line blocks staged in shared memory (a ring per group and the
  // middle block); DEPTH == 0 (blocks too large for the rings): read in place
  constexpr bool STAGED = DEPTH > 0;
  TF* base = reinterpret_cast<TF*>(sm_raw);
  TF* ring = base + (int64_t)grp * DEPTH * ring_stride;
  TF* mids = base + (int64_t)2 * DEPTH * ring_stride;
  const TF* midb = STAGED ? mids : F + (int64_t)m * ps;
  TF* ybuf = STAGED ? mids + ring_stride : base;  // y, z of group 0, then of group 1
  TF* y = ybuf + (int64_t)grp * 2 * ld;
  TF* z = y + ld;
  TF* v = ybuf + 4 * ld;
  // line of the j-th step of this group's forward sweep
  auto line_of = [&](int j) { return (grp == 0) ? j : nb - 1 - j; };
  auto fetch = [&](int j) {
    if constexpr (STAGED) {
      if (j >= 0 && j < cnt) {
        const char* src = reinterpret_cast<const char*>(F + (int64_t)line_of(j) * ps);
        char* dst = reinterpret_cast<char*>(ring + (int64_t)(j % DEPTH) * ring_stride);
        const int chunks = (int)(ps * (int64_t)sizeof(TF) / 16);
        for (int c = gt; c < chunks; c += G) cp_async16(dst + 16 * c, src + 16 * c);
      }
      cp_async_commit();
    }
  };
  // the block of step j, once it has arrived
  auto block_of = [&](int j) -> const TF* {
    if constexpr (STAGED) {
      cp_async_wait<(STAGED ? DEPTH - 1 : 0)>();
      return ring + (int64_t)(j % (STAGED ? DEPTH : 1)) * ring_stride;
    } else {
      return F + (int64_t)line_of(j) * ps;
    }
  };
  auto gsync = [&]() { asm volatile("bar.sync %0, %1;\n" ::"r"(1 + grp), "r"(G) : "memory"); };
  auto csync = [&]() { __syncthreads(); };
  // independent of the predecessor kernel (the factors are fixed during a
  // solve): issued before the dependency wait
  for (int q = 0; q < DEPTH; ++q) fetch(q);
  if constexpr (STAGED)
    for (int64_t e = tid; e < ps; e += nt) mids[e] = F[(int64_t)m * ps + e];
  for (int i = tid; i < 4 * ld; i += nt) ybuf[i] = TF(0);  // y, z of both groups; padding stays zero
  pdl_wait();
  if (done && *done) {
    cp_async_wait<0>();
    return;
  }
  // gather R_i r (free DOFs; zero elsewhere)
  for (int e = tid; e < nb * w; e += nt) {
    const int k = e / w, p = e % w;
    const int c = p % DIM, t = p / DIM;
    int a[3];
    if (DIM == 2) {
      a[0] = b.nlo[0] + t;
      a[1] = b.nlo[1] + k;
    } else {
      a[0] = b.nlo[0] + t % nbx;
      a[1] = b.nlo[1] + t / nbx;
      a[2] = b.nlo[2] + k;
    }
    const int64_t dof = DIM * node_id(g, a) + c;
    v[e] = fm[dof] ? r[dof] : TF(0);
  }
  __syncthreads();
  // (A_{k,k+-1} xs)_p from the stored coupling stencil Cs (row p: NC
  // coefficients of the neighbouring line's nodes and components)
  auto couple = [&](const TF* Cs, int p, const TF* xs) -> TF {
    const TF* c = Cs + p * NC;
    TF t = 0;
#pragma unroll
    for (int sl = 0; sl < NC; ++sl) {
      const int q = lv1_cpl_col<DIM>(p, sl, nbx, nby);
      t = fma(c[sl], xs[q < 0 ? 0 : q], t);
    }
    return t;
  };
  const int part = gt & 3, rq = gt >> 2, nq = G >> 2;
  // forward sweeps: top u_k = S_k^{-1}(r_k - A_{k,k-1} u_{k-1}), bottom with k+1
  {
    const int dir = (grp == 0) ? -1 : +1;
    for (int j = 0; j < cnt; ++j) {
      const int k = line_of(j);
      TF* vk = v + (int64_t)k * w;
      const TF* blk = block_of(j);
      gsync();
      const TF* Cs = blk + pform + ((dir > 0) ? w * NC : 0);
      for (int p = gt; p < w; p += G) y[p] = vk[p] - ((j > 0) ? couple(Cs, p, vk + dir * w) : TF(0));
      gsync();
      lv1_apply<TF, VF>(blk, vk, false, y, z, w, ld, part, rq, nq, gsync);
      gsync();
      fetch(j + DEPTH);
    }
  }
  __syncthreads();
  // middle line, whole CTA
  {
    TF* vm = v + (int64_t)m * w;
    TF* ym = ybuf;
    TF* zm = ybuf + ld;
    for (int p = tid; p < w; p += nt) {
      TF t = vm[p];
      if (m > 0) t -= couple(midb + pform, p, vm - w);
      if (m + 1 < nb) t -= couple(midb + pform + w * NC, p, vm + w);
      ym[p] = t;
    }
    __syncthreads();
    lv1_apply<TF, VF>(midb, vm, false, ym, zm, w, ld, tid & 3, tid >> 2, nt >> 2, csync);
    __syncthreads();
  }
  // backward sweeps toward the ends: x_k = u_k - S_k^{-1} A_{k,k+/-1} x_{k+/-1}
  {
    const int dir = (grp == 0) ? +1 : -1;
    for (int j = cnt - 1; j >= 0; --j) {
      const int k = line_of(j);
      TF* vk = v + (int64_t)k * w;
      const TF* blk = block_of(j);
      gsync();
      const TF* Cs = blk + pform + ((dir > 0) ? w * NC : 0);
      for (int p = gt; p < w; p += G) y[p] = couple(Cs, p, vk + dir * w);
      gsync();
      lv1_apply<TF, VF>(blk, vk, true, y, z, w, ld, part, rq, nq, gsync);
      gsync();
      fetch(j - DEPTH);
    }
  }
  pdl_trigger();
  cp_async_wait<0>();
  __syncthreads();
  TF* out = zloc + zoff[s];
  for (int e = tid; e < nb * w; e += nt) out[e] = v[e];
}

// ---------------------------------------------------------------------------
// Level 1 over TS_NB right-hand sides on the tensor cores (mixed precision,
// 2D).  The twisted block LU sweeps of k_local_solve, with every line step a
// small GEMM over the TS_NB columns: y = r_k - A_{k,k-/+1} u (the coupling
// stencil), t = V_k y, u_k = V_k^T t, where V_k (the packed FP32 Gram factor
// of S_k^{-1}) is the A operand of mma.m16n8k8 TF32 (16 x 8 tiles of V or of
// V^T read from the staged packed rows, zero above the diagonal) and the
// block [w][TS_NB] the B operand (N = 8 = TS_NB columns).  MODE 1: one TF32
// product per tile; MODE 3: 3xTF32 (V = V_hi + V_lo, y = y_hi + y_lo split in
// TF32, products V_hi y_hi + V_hi y_lo + V_lo y_hi), close to FP32 accuracy.
// Line blocks are staged per group through a ring of DEPTH slots by bulk
// asynchronous copies (cp.async.bulk, one per block, completion on an
// mbarrier per slot), issued before the dependency wait.  Vectors in shared
// memory: the local block v [nb][w][TS_NB], per group y and t [rows][TS_NB].
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t f2tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// d += A b for FP32 fragments a (4) and b (2): MODE 1 TF32, MODE 3 3xTF32
template <int MODE>
__device__ __forceinline__ void mma_frag(float (&d)[4], const float (&a)[4], const float (&b)[2]) {
  uint32_t ah[4], bh[2];
#pragma unroll
  for (int q = 0; q < 4; ++q) ah[q] = f2tf32(a[q]);
#pragma unroll
  for (int q = 0; q < 2; ++q) bh[q] = f2tf32(b[q]);
  if (MODE == 3) {
    uint32_t al[4], bl[2];
#pragma unroll
    for (int q = 0; q < 4; ++q) al[q] = f2tf32(a[q] - __uint_as_float(ah[q]));
#pragma unroll
    for (int q = 0; q < 2; ++q) bl[q] = f2tf32(b[q] - __uint_as_float(bh[q]));
    mma_tf32(d, al, bh);
    mma_tf32(d, ah, bl);
  }
  mma_tf32(d, ah, bh);
}

// V(i, j) of a packed lower-triangular V_k (row i: round_up(i + 1, 4) stored
// entries from column 0, zero above the diagonal); zero outside
__device__ __forceinline__ float vpk(const float* V, int w, int i, int j) {
  return (i < w && j < ((i + 4) & ~3)) ? V[lv1_vrow(i) + j] : 0.f;
}

// out (=, or -= when sub) V^T (V y) for the [w][TS_NB] block y (rows w ..
// KT*8 - 1 zero); t: [MT*16][TS_NB] scratch.  Warps wi = 0 .. nw - 1 of the
// calling group take the M tiles in turn; sync() is the group's barrier.
template <int MODE, class Sync>
__device__ __forceinline__ void bls_apply(const float* V, int w, const float* y, float* t, float* out, bool sub, int wi,
                                          int nw, Sync sync) {
  const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const int MT = (w + 15) >> 4, KT = (w + 7) >> 3;
  for (int mt = wi; mt < MT; mt += nw) {
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    const int r0 = 16 * mt + gid, r1 = r0 + 8;
    const int kmax = min(KT, (16 * mt + 15) / 8 + 1);
    // rows r0, r1 of the packed V: start and stored length (0 past w)
    const float* v0 = V + lv1_vrow(r0);
    const float* v1 = V + lv1_vrow(r1);
    const int l0 = (r0 < w) ? ((r0 + 4) & ~3) : 0, l1 = (r1 < w) ? ((r1 + 4) & ~3) : 0;
    for (int kt = 0; kt < kmax; ++kt) {
      const int c0 = 8 * kt + tig;
      const float a[4] = {(c0 < l0) ? v0[c0] : 0.f, (c0 < l1) ? v1[c0] : 0.f, (c0 + 4 < l0) ? v0[c0 + 4] : 0.f,
                          (c0 + 4 < l1) ? v1[c0 + 4] : 0.f};
      const float b[2] = {y[c0 * TS_NB + gid], y[(c0 + 4) * TS_NB + gid]};
      mma_frag<MODE>(d, a, b);
    }
    t[r0 * TS_NB + 2 * tig] = d[0];
    t[r0 * TS_NB + 2 * tig + 1] = d[1];
    t[r1 * TS_NB + 2 * tig] = d[2];
    t[r1 * TS_NB + 2 * tig + 1] = d[3];
  }
  sync();
  for (int mt = wi; mt < MT; mt += nw) {
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    const int r0 = 16 * mt + gid, r1 = r0 + 8;
    for (int kt = 2 * mt; kt < KT; ++kt) {
      const int c0 = 8 * kt + tig;
      // A' = V^T: A'(i, k) = V(k, i)
      const float a[4] = {vpk(V, w, c0, r0), vpk(V, w, c0, r1), vpk(V, w, c0 + 4, r0), vpk(V, w, c0 + 4, r1)};
      const float b[2] = {t[c0 * TS_NB + gid], t[(c0 + 4) * TS_NB + gid]};
      mma_frag<MODE>(d, a, b);
    }
    if (r0 < w) {
      float* o = out + r0 * TS_NB + 2 * tig;
      o[0] = sub ? o[0] - d[0] : d[0];
      o[1] = sub ? o[1] - d[1] : d[1];
    }
    if (r1 < w) {
      float* o = out + r1 * TS_NB + 2 * tig;
      o[0] = sub ? o[0] - d[2] : d[2];
      o[1] = sub ? o[1] - d[3] : d[3];
    }
  }
}

constexpr int BLS_GW = 4;                       // warps per group
constexpr int BLS_THREADS = 2 * 32 * BLS_GW;    // two groups

template <int MODE, int DEPTH>
__global__ void __launch_bounds__(BLS_THREADS, 3)
    k_blocal_solve(Geom g, AxisTables ax, const float* __restrict__ r, const BLDesc* __restrict__ desc,
                   const float* __restrict__ pv, const uint8_t* __restrict__ fm, const int64_t* __restrict__ zoff,
                   float* __restrict__ zloc, int ring_stride, int ypad, const int* __restrict__ done,
                   int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char bls_sm[];
  constexpr int NC = Lv1Cpl<2>::NC;
  __shared__ __align__(8) uint64_t bars[2 * DEPTH + 1];
  const int s = blockIdx.x, tid = threadIdx.x;
  constexpr int G = 32 * BLS_GW;
  const int grp = tid / G, gt = tid - grp * G, wi = gt >> 5;
  SubBox b;
  sub_box_t<2>(g, ax, s, b);
  const int nbx = b.nb3[0];
  const BLDesc d = desc[s];
  const int w = d.w, nb = d.nb, m = nb / 2;
  const int cnt = (grp == 0) ? m : nb - 1 - m;
  const int64_t ps = lv1_stride(w, true, 2), pform = lv1_sform(w, true);
  const float* F = pv + d.coff;
  float* ring = reinterpret_cast<float*>(bls_sm) + (int64_t)grp * DEPTH * ring_stride;
  float* midb = reinterpret_cast<float*>(bls_sm) + (int64_t)2 * DEPTH * ring_stride;
  float* yb = midb + ring_stride;                 // [2 groups][ypad][TS_NB] y, then t
  float* y = yb + (int64_t)grp * 2 * ypad * TS_NB;
  float* t = y + (int64_t)ypad * TS_NB;
  float* v = yb + (int64_t)4 * ypad * TS_NB;      // [nb * w][TS_NB]
  uint64_t* gbar = bars + grp * DEPTH;
  uint64_t* mbar = bars + 2 * DEPTH;
  const uint32_t bytes = (uint32_t)(ps * sizeof(float));
  auto line_of = [&](int j) { return (grp == 0) ? j : nb - 1 - j; };
  auto fetch = [&](int j) {
    if (gt == 0 && j >= 0 && j < cnt)
      bulk_load(ring + (int64_t)(j % DEPTH) * ring_stride, F + (int64_t)line_of(j) * ps, bytes, gbar + j % DEPTH);
  };
  uint32_t phase = 0;  // bit q: parity of the next completion of slot q
  // the block of step j; wait: its copy was issued since the slot was last
  // read (every forward step, and the backward steps below cnt - DEPTH: the
  // last DEPTH blocks of the forward sweep are still in their slots)
  auto block_of = [&](int j, bool wait) -> const float* {
    const int q = j % DEPTH;
    if (wait) {
      mbar_wait(gbar + q, (phase >> q) & 1u, status);
      phase ^= 1u << q;
    }
    return ring + (int64_t)q * ring_stride;
  };
  auto gsync = [&]() { asm volatile("bar.sync %0, %1;\n" ::"r"(1 + grp), "r"(G) : "memory"); };
  auto csync = [&]() { __syncthreads(); };
  if (tid == 0) {
    for (int q = 0; q < 2 * DEPTH + 1; ++q) mbar_init(bars + q, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  // the factors are fixed during a solve: staged before the dependency wait
  for (int q = 0; q < DEPTH; ++q) fetch(q);
  if (tid == 0) bulk_load(midb, F + (int64_t)m * ps, bytes, mbar);
  for (int i = tid; i < 4 * ypad * TS_NB; i += blockDim.x) yb[i] = 0.f;  // padding rows stay zero
  pdl_wait();
  const bool stop = done && *done;
  if (!stop) {
    // gather R_i r for every column (r is zero at Dirichlet DOFs): one local
    // unknown's TS_NB values per thread as two 16-byte loads, four in flight
    const int nl = nb * w;
    for (int e0 = tid; e0 < nl; e0 += 4 * BLS_THREADS) {
      float4 x[4][2];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int row = e0 + BLS_THREADS * u;
        x[u][0] = x[u][1] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < nl) {
          const int k = row / w, p = row % w;
          const int64_t dof = 2 * ((int64_t)(b.nlo[1] + k) * (g.nx + 1) + b.nlo[0] + p / 2) + (p & 1);
          const float4* src = reinterpret_cast<const float4*>(r + dof * TS_NB);
          x[u][0] = src[0];
          x[u][1] = src[1];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int row = e0 + BLS_THREADS * u;
        if (row < nl) {
          float4* dst = reinterpret_cast<float4*>(v + (int64_t)row * TS_NB);
          dst[0] = x[u][0];
          dst[1] = x[u][1];
        }
      }
    }
  }
  __syncthreads();
  // (A_{k,k+-1} xs)_p for column col from the stored coupling stencil Cs
  auto couple = [&](const float* Cs, int p, int col, const float* xs) -> float {
    const float* c = Cs + p * NC;
    float acc = 0.f;
#pragma unroll
    for (int sl = 0; sl < NC; ++sl) {
      const int q = lv1_cpl_col<2>(p, sl, nbx, 1);
      acc = fmaf(c[sl], xs[(q < 0 ? 0 : q) * TS_NB + col], acc);
    }
    return acc;
  };
  // forward sweeps
  {
    const int dir = (grp == 0) ? -1 : +1;
    for (int j = 0; j < cnt; ++j) {
      const int k = line_of(j);
      float* vk = v + (int64_t)k * w * TS_NB;
      const float* blk = block_of(j, true);
      gsync();
      if (!stop) {
        const float* Cs = blk + pform + ((dir > 0) ? w * NC : 0);
        for (int e = gt; e < w * TS_NB; e += G) {
          const int p = e / TS_NB, col = e % TS_NB;
          y[e] = vk[e] - ((j > 0) ? couple(Cs, p, col, vk + dir * w * TS_NB) : 0.f);
        }
        gsync();
        bls_apply<MODE>(blk, w, y, t, vk, false, wi, BLS_GW, gsync);
      }
      gsync();
      fetch(j + DEPTH);
    }
  }
  __syncthreads();
  // middle line, whole CTA
  mbar_wait(mbar, 0u, status);
  if (!stop) {
    float* vm = v + (int64_t)m * w * TS_NB;
    float* ym = yb;
    float* tm = yb + (int64_t)ypad * TS_NB;
    for (int e = tid; e < w * TS_NB; e += blockDim.x) {
      const int p = e / TS_NB, col = e % TS_NB;
      float tt = vm[e];
      if (m > 0) tt -= couple(midb + pform, p, col, vm - w * TS_NB);
      if (m + 1 < nb) tt -= couple(midb + pform + w * NC, p, col, vm + w * TS_NB);
      ym[e] = tt;
    }
    __syncthreads();
    bls_apply<MODE>(midb, w, ym, tm, vm, false, tid >> 5, 2 * BLS_GW, csync);
  }
  __syncthreads();
  // the middle group's y/t of group 0 were used as scratch: rows past w must
  // be zero again for the group sweeps (t rows past w are rewritten as zero)
  for (int i = w * TS_NB + tid; i < ypad * TS_NB; i += blockDim.x) yb[i] = 0.f;
  __syncthreads();
  // backward sweeps toward the ends
  {
    const int dir = (grp == 0) ? +1 : -1;
    for (int j = cnt - 1; j >= 0; --j) {
      const int k = line_of(j);
      float* vk = v + (int64_t)k * w * TS_NB;
      const float* blk = block_of(j, j < cnt - DEPTH);
      gsync();
      if (!stop) {
        const float* Cs = blk + pform + ((dir > 0) ? w * NC : 0);
        for (int e = gt; e < w * TS_NB; e += G) {
          const int p = e / TS_NB, col = e % TS_NB;
          y[e] = couple(Cs, p, col, vk + dir * w * TS_NB);
        }
        gsync();
        bls_apply<MODE>(blk, w, y, t, vk, true, wi, BLS_GW, gsync);
      }
      gsync();
      fetch(j - DEPTH);
    }
  }
  pdl_trigger();
  __syncthreads();
  if (stop) return;
  float4* out = reinterpret_cast<float4*>(zloc + zoff[s] * TS_NB);
  const float4* vv = reinterpret_cast<const float4*>(v);
  for (int e = tid; e < nb * w * TS_NB / 4; e += blockDim.x) out[e] = vv[e];
}

// ---------------------------------------------------------------------------
// host: subdomain tables, factor storage, launch
// ---------------------------------------------------------------------------
static void axis_subdomains(const Geom& g, int a, std::vector<int>& lo, std::vector<int>& hi,
                            std::vector<int>& elo, std::vector<int>& ehi) {
  const int n = g.n[a], H = g.H[a], nb = n / H;
  lo.clear(); hi.clear(); elo.clear(); ehi.clear();
  int cnt = (g.ov >= 0) ? nb : nb + 1;
  for (int s = 0; s < cnt; ++s) {
    int e0, e1;
    if (g.ov >= 0) {
      e0 = std::max(0, s * H - g.ov);
      e1 = std::min(n, (s + 1) * H + g.ov);
    } else {
      e0 = std::max(0, (s - 1) * H);
      e1 = std::min(n, (s + 1) * H);
    }
    elo.push_back(e0);
    ehi.push_back(e1);
    lo.push_back(e0 + (e0 > 0 ? 1 : 0));
    hi.push_back(e1 - (e1 < n ? 1 : 0));
  }
}

void build_level1(ts_handle h) {
  Geom& g = h->g;
  cudaStream_t st = h->ctx->stream;
  std::vector<int> lo[3], hi[3], elo[3], ehi[3];
  for (int a = 0; a < g.dim; ++a) {
    axis_subdomains(g, a, lo[a], hi[a], elo[a], ehi[a]);
    g.nsub[a] = (int)lo[a].size();
    // candidate table: node coordinate -> up to two subdomains
    std::vector<int2> cand(g.n[a] + 1, make_int2(-1, -1));
    for (int s = 0; s < g.nsub[a]; ++s)
      for (int i = lo[a][s]; i <= hi[a][s]; ++i) {
        if (cand[i].x < 0)
          cand[i].x = s;
        else if (cand[i].y < 0)
          cand[i].y = s;
        else
          throw TsError(TS_ERR_INVALID, "overlap too large: a node lies in more than two subdomains per axis");
      }
    h->ax.sub_lo[a] = dupload(h, lo[a]);
    h->ax.sub_hi[a] = dupload(h, hi[a]);
    h->ax.sub_elo[a] = dupload(h, elo[a]);
    h->ax.sub_ehi[a] = dupload(h, ehi[a]);
    h->ax.cand[a] = dupload(h, cand);
  }
  for (int a = g.dim; a < 3; ++a) g.nsub[a] = 1;
  const int nsub = g.nsub[0] * g.nsub[1] * g.nsub[2];
  h->nsub = nsub;
  // block-line shapes: lines along the last axis
  std::vector<BLDesc> desc(nsub);
  std::vector<int64_t> zoff(nsub);
  int64_t zo = 0;
  int maxw = 0, maxn = 0;
  for (int s = 0; s < nsub; ++s) {
    int sx = s % g.nsub[0], t = s / g.nsub[0];
    int sy = (g.dim == 2) ? t : t % g.nsub[1];
    int sz = (g.dim == 2) ? 0 : t / g.nsub[1];
    int nbx = hi[0][sx] - lo[0][sx] + 1, nby = hi[1][sy] - lo[1][sy] + 1;
    BLDesc d;
    if (g.dim == 2) {
      d.w = 2 * nbx;
      d.nb = nby;
    } else {
      int nbz = hi[2][sz] - lo[2][sz] + 1;
      d.w = 3 * nbx * nby;
      d.nb = nbz;
    }
    zoff[s] = zo;
    zo += (int64_t)d.w * d.nb;
    maxw = std::max(maxw, d.w);
    maxn = std::max(maxn, d.w * d.nb);
    desc[s] = d;
  }
  // largest element box
  {
    int mx[3] = {1, 1, 1};
    for (int a = 0; a < g.dim; ++a)
      for (size_t q = 0; q < elo[a].size(); ++q) mx[a] = std::max(mx[a], ehi[a][q] - elo[a][q]);
    h->lv1_max_nel = mx[0] * mx[1] * mx[2];
  }
  // stored solve factor offsets (V form in mixed precision, M form in FP64)
  const bool vform = h->opt.precision != TS_FP64;
  int64_t coff = 0;
  int rs = 0;
  for (int s = 0; s < nsub; ++s) {
    desc[s].coff = coff;
    coff += (int64_t)desc[s].nb * lv1_stride(desc[s].w, vform, g.dim);
    rs = std::max(rs, (int)lv1_stride(desc[s].w, vform, g.dim));
  }
  h->pv_len = coff;
  h->pv_stride_max = rs;
  h->sub_desc_h = desc;
  h->zloc_off_h = zoff;
  h->max_w = maxw;
  h->zloc_len = zo;
  const size_t smem = lv1_factor_smem(maxw, g.dim);
  if (smem > 227 * 1024)
    throw TsError(TS_ERR_INVALID, "local block line too wide for shared memory (w=" + std::to_string(maxw) + ")");
  h->sub_desc = dupload(h, desc);
  h->zloc_off = dupload(h, zoff);
  const bool mixed = h->opt.precision != TS_FP64;
  if (mixed) {
    h->pv32 = dalloc<float>(h, coff);
    h->zloc32 = dalloc<float>(h, zo);
  } else {
    h->pv64 = dalloc<double>(h, coff);
    h->zloc = dalloc<double>(h, zo);
  }
  if (g.dim == 2) {
    if (smem > ts_allow_dynamic_smem(k_local_factor<2>, h->ctx->device))
      throw TsError(TS_ERR_INVALID, "local block line too wide for shared memory");
    tsl(h), k_local_factor<2><<<nsub, 256, smem, st>>>(g, h->ax, h->E, h->freemask, h->sub_desc, h->pv64, h->pv32,
                                                       h->dstatus);
  } else {
    if (smem > ts_allow_dynamic_smem(k_local_factor<3>, h->ctx->device))
      throw TsError(TS_ERR_INVALID, "local block line too wide for shared memory");
    tsl(h), k_local_factor<3><<<nsub, 256, smem, st>>>(g, h->ax, h->E, h->freemask, h->sub_desc, h->pv64, h->pv32,
                                                       h->dstatus);
  }
  TS_CUDA(cudaGetLastError());
  (void)maxn;
}

template <int DIM, class TF, int DEPTH, bool VF, int MAXT>
static void launch_ls_t(ts_handle h, const TF* r, const TF* pv, TF* zloc, size_t smem, int threads) {
  // the limits are set once per process, outside any stream capture (the
  // first call of each instantiation precedes the capture of the PCG
  // iteration; other threads wait for it): all of the SM's shared memory
  // may serve the CTAs
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, []() {
    attr_err = cudaFuncSetAttribute(k_local_solve<DIM, TF, DEPTH, VF, MAXT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (attr_err == cudaSuccess)
      attr_err = cudaFuncSetAttribute(k_local_solve<DIM, TF, DEPTH, VF, MAXT>,
                                      cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  });
  TS_CUDA(attr_err);
  ts_launch(h, h->pdl, k_local_solve<DIM, TF, DEPTH, VF, MAXT>, h->nsub, threads, smem, h->ctx->stream, h->g, h->ax,
            r, (const BLDesc*)h->sub_desc, pv, (const uint8_t*)h->freemask, (const int64_t*)h->zloc_off, zloc,
            h->pv_stride_max, (const int*)h->done_flag);
}

template <int DIM, class TF, int DEPTH, bool VF>
static void launch_ls(ts_handle h, const TF* r, const TF* pv, TF* zloc, size_t smem, int threads) {
  if (threads <= 320)
    launch_ls_t<DIM, TF, DEPTH, VF, 320>(h, r, pv, zloc, smem, threads);
  else
    launch_ls_t<DIM, TF, DEPTH, VF, 512>(h, r, pv, zloc, smem, threads);
}

template <int DIM, class TF, bool VF>
static void launch_ls_depth(ts_handle h, const TF* r, const TF* pv, TF* zloc) {
  int maxn = 0, maxwp = 0;
  for (auto& d : h->sub_desc_h) {
    maxn = std::max(maxn, d.w * d.nb);
    maxwp = std::max(maxwp, (d.w + 3) & ~3);
  }
  // two rings of `depth` line blocks, the middle block, y and z of both groups,
  // the local vector
  auto need = [&](int depth) {
    return ((size_t)(2 * depth + 1) * h->pv_stride_max + 4 * (size_t)maxwp + (size_t)maxn) * sizeof(TF);
  };
  // two groups of G threads, a quad per line row
  const int G = std::min(256, 32 * ((4 * h->max_w + 31) / 32));
  // the deeper rings only while every subdomain's CTA stays resident in one
  // wave (CTAs per SM x shared memory within the SM's 228 KB)
  const int per_sm = (h->nsub + h->ctx->n_sm - 1) / h->ctx->n_sm;
  // without rings: the vectors alone
  const size_t need0 = (4 * (size_t)maxwp + (size_t)maxn) * sizeof(TF);
  if (need(4) * per_sm <= 220 * 1024)
    launch_ls<DIM, TF, 4, VF>(h, r, pv, zloc, need(4), 2 * G);
  else if (need(2) <= 227 * 1024)
    launch_ls<DIM, TF, 2, VF>(h, r, pv, zloc, need(2), 2 * G);
  else if (need0 <= 227 * 1024)
    launch_ls<DIM, TF, 0, VF>(h, r, pv, zloc, need0, 2 * G);
  else
    throw TsError(TS_ERR_INVALID, "local solve needs too much shared memory");
}

void launch_local_solve(ts_handle h, const double* r) {
  if (h->opt.precision != TS_FP64) {
    // the mixed path reads the FP32 copy of r (kept current by the caller)
    const float* r32 = h->r32;
    if (h->g.dim == 2) launch_ls_depth<2, float, true>(h, r32, h->pv32, h->zloc32);
    else launch_ls_depth<3, float, true>(h, r32, h->pv32, h->zloc32);
  } else {
    if (h->g.dim == 2) launch_ls_depth<2, double, false>(h, r, h->pv64, h->zloc);
    else launch_ls_depth<3, double, false>(h, r, h->pv64, h->zloc);
  }
  TS_CUDA(cudaGetLastError());
}

template <int MODE, int DEPTH>
static void launch_bls_t(ts_handle h, const float* r32, float* zloc, size_t smem, int ypad) {
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, []() {
    attr_err = cudaFuncSetAttribute(k_blocal_solve<MODE, DEPTH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    200 * 1024);
    if (attr_err == cudaSuccess)
      attr_err = cudaFuncSetAttribute(k_blocal_solve<MODE, DEPTH>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  });
  TS_CUDA(attr_err);
  ts_launch(h, h->pdl, k_blocal_solve<MODE, DEPTH>, h->nsub, BLS_THREADS, smem, h->ctx->stream, h->g, h->ax, r32,
            (const BLDesc*)h->sub_desc, (const float*)h->pv32, (const uint8_t*)h->freemask,
            (const int64_t*)h->zloc_off, zloc, h->pv_stride_max, ypad, (const int*)h->done_flag, h->dstatus);
}

// Level 1 for TS_NB columns: zloc [local][TS_NB] (FP32) from r32 [ndof][TS_NB]
// (mixed precision, 2D).  TS_MIXED_TF32 runs one TF32 product per tile,
// TS_MIXED_FP32 and TS_MIXED_3XTF32 the 3xTF32 split.
void launch_blocal_solve(ts_handle h, const float* r32, float* zloc) {
  if (h->g.dim != 2 || !h->pv32) throw TsError(TS_ERR_INVALID, "internal: block level 1 needs a mixed 2D design");
  int maxn = 0, maxw = 0;
  for (auto& d : h->sub_desc_h) {
    maxn = std::max(maxn, d.w * d.nb);
    maxw = std::max(maxw, d.w);
  }
  const int ypad = 16 * ((maxw + 15) / 16);
  auto need = [&](int depth) {
    return ((size_t)(2 * depth + 1) * h->pv_stride_max + (size_t)4 * ypad * TS_NB + (size_t)maxn * TS_NB) *
           sizeof(float);
  };
  const bool tf32 = h->opt.precision == TS_MIXED_TF32;
  if (need(4) <= 110 * 1024) {
    if (tf32) launch_bls_t<1, 4>(h, r32, zloc, need(4), ypad);
    else launch_bls_t<3, 4>(h, r32, zloc, need(4), ypad);
  } else if (need(2) <= 200 * 1024) {
    if (tf32) launch_bls_t<1, 2>(h, r32, zloc, need(2), ypad);
    else launch_bls_t<3, 2>(h, r32, zloc, need(2), ypad);
  } else {
    throw TsError(TS_ERR_INVALID, "block level 1: subdomain too large for shared memory");
  }
  TS_CUDA(cudaGetLastError());
}
