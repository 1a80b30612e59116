// Coarse level of M_EH(+Rot) (Sec. 4.1-4.3, Eqs. juan001/juan002):
//   V_{0,H} = span{ chi_l [psi,0], chi_l [0,psi] } (+ chi_l r, Sec. 4.2),
//   psi: eigenfunctions of the heat operator -div(kappa grad psi) = lambda kappa psi
//        on each coarse-node neighbourhood omega_l (Eq. juaneheateigenproblem),
//        kappa = E_e, Neumann on the boundary of omega_l except where the
//        component is Dirichlet; those with lambda < tau = tau_scale/H^2 are kept
//        (at least one, at most max_modes).
//   K_0 = R_0 K R_0^T,  correction R_0^T K_0^{-1} R_0 r  (Sec. 2.1).
//
// Device pipeline, all FP64:
//   k_heat_eig     one CTA per (omega_l, component): inertia of K - tau M by a
//                  block-line LDL^T (Sylvester: number of negative pivots =
//                  number of eigenvalues below tau), factor of K + tau M, then
//                  shift-invert Lanczos in the M inner product with full
//                  re-orthogonalisation and deflated restarts (for repeated
//                  eigenvalues) until that many Ritz pairs have converged.
//   k_k0_column    one CTA per coarse DOF k: v = K Phi_k on omega_l, then
//                  K_0[j][k] = Phi_j . v for the DOFs of the neighbouring nodes.
//   dense blocked Cholesky of K_0, explicit L^{-1} (applied as two GEMVs).
#include <algorithm>
#include <cmath>

#include "ts_blockline.cuh"
#include "ts_internal.cuh"
#include "ts_reduce.cuh"

// element stiffness (E = 1), this translation unit's copy
static __constant__ double c_KE[24 * 24];

void upload_KE_coarse(ts_handle h, const std::vector<double>& KE) {
  TS_CUDA(cudaMemcpyToSymbolAsync(c_KE, KE.data(), KE.size() * sizeof(double), 0, cudaMemcpyHostToDevice,
                                  h->ctx->stream));
}

__device__ __forceinline__ int64_t node_id_c(const Geom& g, const int* a) {
  if (g.dim == 2) return (int64_t)a[1] * (g.nx + 1) + a[0];
  return ((int64_t)a[2] * (g.ny + 1) + a[1]) * (g.nx + 1) + a[0];
}

// local node index p within a closed box -> global coordinates
template <int DIM>
__device__ __forceinline__ void box_coords(const HeatProb& P, int idx, int* a) {
  const int bx = P.hi[0] - P.lo[0] + 1;
  if (DIM == 2) {
    a[0] = P.lo[0] + idx % bx;
    a[1] = P.lo[1] + idx / bx;
  } else {
    const int by = P.hi[1] - P.lo[1] + 1;
    a[0] = P.lo[0] + idx % bx;
    a[1] = P.lo[1] + (idx / bx) % by;
    a[2] = P.lo[2] + idx / (bx * by);
  }
}

template <int DIM>
struct HeatAsm {
  Geom g;
  const double* E;
  const uint8_t* fm;
  HeatProb P;
  double kc, mc;
  __device__ double entry(int kr, int p, int kc_, int q) const {
    int a[3], b[3];
    box_coords<DIM>(P, kr * P.w + p, a);
    box_coords<DIM>(P, kc_ * P.w + q, b);
    bool fa = fm[DIM * node_id_c(g, a) + P.c], fb = fm[DIM * node_id_c(g, b) + P.c];
    if (!fa || !fb) return (kr == kc_ && p == q) ? 1.0 : 0.0;
    return heat_entry<DIM>(g, E, a, b, kc, mc, P.lo, P.hi);
  }
};

// y = M x on the closed box (kappa-weighted consistent mass, Dirichlet rows
// and columns of component c removed).  x, y in shared memory.
template <int DIM>
__device__ void mass_apply(const Geom& g, const double* __restrict__ E, const uint8_t* __restrict__ fm,
                           const HeatProb& P, const double* x, double* y) {
  const int n = P.nloc;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int a[3];
    box_coords<DIM>(P, i, a);
    double s = 0.0;
    if (fm[DIM * node_id_c(g, a) + P.c]) {
      int lo[3], hi[3];
      for (int d = 0; d < DIM; ++d) {
        lo[d] = max(a[d] - 1, P.lo[d]);
        hi[d] = min(a[d] + 1, P.hi[d]);
      }
      const int bx = P.hi[0] - P.lo[0] + 1, by = (DIM == 3) ? P.hi[1] - P.lo[1] + 1 : 1;
      for (int bz = (DIM == 3 ? lo[2] : 0); bz <= (DIM == 3 ? hi[2] : 0); ++bz)
        for (int byy = lo[1]; byy <= hi[1]; ++byy)
          for (int bxx = lo[0]; bxx <= hi[0]; ++bxx) {
            int b[3] = {bxx, byy, bz};
            int j = (bxx - P.lo[0]) + bx * ((byy - P.lo[1]) + (DIM == 3 ? by * (bz - P.lo[2]) : 0));
            double xv = x[j];
            if (xv != 0.0) s += heat_entry<DIM>(g, E, a, b, 0.0, 1.0, P.lo, P.hi) * xv;
          }
    }
    y[i] = s;
  }
}

// --- small symmetric tridiagonal helpers (one thread each) -----------------
// number of eigenvalues of T (diag al[0..k), off be[1..k)) below x
__device__ int sturm_count(const double* al, const double* be, int k, double x) {
  int cnt = 0;
  double q = 1.0;
  for (int i = 0; i < k; ++i) {
    double b2 = (i > 0) ? be[i] * be[i] : 0.0;
    q = (al[i] - x) - ((i > 0) ? b2 / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// idx-th smallest eigenvalue of T by bisection
__device__ double tri_eig_bisect(const double* al, const double* be, int k, int idx) {
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < k; ++i) {
    double r = ((i > 0) ? fabs(be[i]) : 0.0) + ((i + 1 < k) ? fabs(be[i + 1]) : 0.0);
    lo = fmin(lo, al[i] - r);
    hi = fmax(hi, al[i] + r);
  }
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(al, be, k, mid) > idx)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

// eigenvector of T for eigenvalue th by inverse iteration with a partial-
// pivoting tridiagonal LU; s[0..k) on output (unit 2-norm)
__device__ void tri_eigvec(const double* al, const double* be, int k, double th, double* s, double* D, double* C,
                           double* F, double* L, unsigned char* pv) {
  double nrm = 0.0;
  for (int i = 0; i < k; ++i) nrm = fmax(nrm, fabs(al[i]) + ((i > 0) ? fabs(be[i]) : 0.0));
  const double tiny = 1e-15 * fmax(nrm, 1e-300);
  // factor T - th I: subdiag a_i = be[i+1], diag b_i = al[i]-th, super c_i = be[i+1]
  for (int i = 0; i < k; ++i) {
    D[i] = al[i] - th;
    C[i] = (i + 1 < k) ? be[i + 1] : 0.0;
    F[i] = 0.0;
  }
  for (int i = 0; i + 1 < k; ++i) {
    double a = be[i + 1];
    if (fabs(a) > fabs(D[i])) {
      double b1 = D[i + 1], c1 = C[i + 1];
      double m = D[i] / a;
      double cold = C[i];
      D[i] = a;
      C[i] = b1;
      F[i] = c1;
      D[i + 1] = cold - m * b1;
      C[i + 1] = -m * c1;
      L[i] = m;
      pv[i] = 1;
    } else {
      if (D[i] == 0.0) D[i] = tiny;
      double m = a / D[i];
      D[i + 1] -= m * C[i];
      L[i] = m;
      pv[i] = 0;
    }
  }
  for (int i = 0; i < k; ++i)
    if (fabs(D[i]) < tiny) D[i] = (D[i] < 0 ? -tiny : tiny);
  for (int i = 0; i < k; ++i) s[i] = 1.0 / sqrt((double)k) * (1.0 + 0.01 * ((i * 7919) % 13));
  for (int it = 0; it < 3; ++it) {
    for (int i = 0; i + 1 < k; ++i) {
      if (pv[i]) {
        double t = s[i];
        s[i] = s[i + 1];
        s[i + 1] = t;
      }
      s[i + 1] -= L[i] * s[i];
    }
    for (int i = k - 1; i >= 0; --i) {
      double v = s[i];
      if (i + 1 < k) v -= C[i] * s[i + 1];
      if (i + 2 < k) v -= F[i] * s[i + 2];
      s[i] = v / D[i];
    }
    double q = 0.0;
    for (int i = 0; i < k; ++i) q += s[i] * s[i];
    q = 1.0 / sqrt(q);
    for (int i = 0; i < k; ++i) s[i] *= q;
  }
}

__device__ __forceinline__ double hash01(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t x = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u ^ (c + 0x165667B1u) * 0xC2B2AE3Du;
  x ^= x >> 15;
  x *= 0x2C1B3C6Du;
  x ^= x >> 12;
  x *= 0x297A2D39u;
  x ^= x >> 15;
  return (double)(x & 0xFFFFFF) / 16777216.0 - 0.5;
}

constexpr int EIG_THREADS = 256;
constexpr int EIG_MAXLOCK = TS_MAXMODES;

// Lanczos workspace per problem (global): V [(kmax+1) * n] + locked [EIG_MAXLOCK * n]
template <int DIM>
__global__ void __launch_bounds__(EIG_THREADS) k_heat_eig(Geom g, const double* __restrict__ E,
                                                          const uint8_t* __restrict__ fm, const HeatProb* __restrict__ hp,
                                                          int p0, int pend, double tau, double sigma, int max_modes,
                                                          int kmax, double* __restrict__ heat_fac,
                                                          double* __restrict__ psi, double* __restrict__ lam_out,
                                                          int* __restrict__ count_out, int* __restrict__ found_out,
                                                          double* __restrict__ ws, int64_t ws_per, int* status) {
  extern __shared__ double sm[];
  __shared__ int bad;
  __shared__ double al[TS_LANCZOS_MAX + 1], be[TS_LANCZOS_MAX + 2];
  __shared__ double theta[EIG_MAXLOCK + 2], resid[EIG_MAXLOCK + 2];
  __shared__ double hcoef[TS_LANCZOS_MAX + EIG_MAXLOCK + 2];
  __shared__ double lockval[EIG_MAXLOCK];
  __shared__ int s_flag, s_nlock, s_kdim;
  __shared__ double red[32];
  __shared__ double tD[TS_LANCZOS_MAX], tC[TS_LANCZOS_MAX], tF[TS_LANCZOS_MAX], tL[TS_LANCZOS_MAX],
      tS[TS_LANCZOS_MAX];
  __shared__ unsigned char tP[TS_LANCZOS_MAX];
  const int pi = p0 + blockIdx.x;
  if (pi >= pend) return;
  const HeatProb P = hp[pi];
  if (P.dedup_of >= 0) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int n = P.nloc;
  HeatAsm<DIM> A;
  A.g = g;
  A.E = E;
  A.fm = fm;
  A.P = P;
  // (1) inertia of K - tau M
  if (tid == 0) bad = 0;
  A.kc = 1.0;
  A.mc = -tau;
  __syncthreads();
  int neg = bl_factor(A, P.nb, P.w, nullptr, false, false, sm, &bad);
  if (tid == 0 && bad) atomicOr(status, 4);  // zero pivot in the inertia count
  // (2) factor of K + sigma M (SPD)
  __syncthreads();
  if (tid == 0) bad = 0;
  A.mc = sigma;
  __syncthreads();
  double* F = heat_fac + P.fac_off;
  bl_factor(A, P.nb, P.w, F, true, true, sm, &bad);
  if (tid == 0 && bad) atomicOr(status, 8);
  __syncthreads();
  // targets
  int nfree_loc = 0;
  // count free nodes (kmax must not exceed it)
  {
    int cnt = 0;
    for (int i = tid; i < n; i += nt) {
      int a[3];
      box_coords<DIM>(P, i, a);
      cnt += fm[DIM * node_id_c(g, a) + P.c] ? 1 : 0;
    }
    double c = block_sum_dyn((double)cnt, red);
    if (tid == 0) s_kdim = (int)c;
    __syncthreads();
    nfree_loc = s_kdim;
    __syncthreads();
  }
  const int target = min(max(neg, 1), min(max_modes, nfree_loc));
  const int km = min(kmax, nfree_loc);
  double* V = ws + (int64_t)blockIdx.x * ws_per;       // (km+1) x n
  double* LK = V + (int64_t)(kmax + 1) * n;             // EIG_MAXLOCK x n (locked vectors)
  double* u = sm;            // n
  double* w = u + n;         // n
  double* tmp = w + n;       // 2*w_line
  const double th_tau = 1.0 / (tau + sigma);
  if (tid == 0) s_nlock = 0;
  __syncthreads();
  for (int restart = 0; restart < 6; ++restart) {
    const int need = target - s_nlock;
    if (need <= 0) break;
    // start vector: hashed values at free nodes, M-orthogonal to locked ones
    for (int i = tid; i < n; i += nt) {
      int a[3];
      box_coords<DIM>(P, i, a);
      w[i] = fm[DIM * node_id_c(g, a) + P.c] ? (1.0 + hash01(pi, i, restart)) : 0.0;
    }
    __syncthreads();
    int nl = s_nlock;
    for (int pass = 0; pass < 2 && nl > 0; ++pass) {
      mass_apply<DIM>(g, E, fm, P, w, u);
      __syncthreads();
      for (int q = tid >> 5; q < nl; q += nt >> 5) {
        double s = 0.0;
        for (int i = tid & 31; i < n; i += 32) s += u[i] * LK[(int64_t)q * n + i];
        s = warp_sum(s);
        if ((tid & 31) == 0) hcoef[q] = s;
      }
      __syncthreads();
      for (int i = tid; i < n; i += nt) {
        double s = w[i];
        for (int q = 0; q < nl; ++q) s -= hcoef[q] * LK[(int64_t)q * n + i];
        w[i] = s;
      }
      __syncthreads();
    }
    mass_apply<DIM>(g, E, fm, P, w, u);
    __syncthreads();
    double nn = 0.0;
    for (int i = tid; i < n; i += nt) nn += w[i] * u[i];
    nn = block_sum_dyn(nn, red);
    if (tid == 0) red[31] = nn;
    __syncthreads();
    nn = red[31];
    __syncthreads();
    double inv = 1.0 / sqrt(nn);
    for (int i = tid; i < n; i += nt) V[i] = w[i] * inv;
    if (tid == 0) {
      be[0] = 0.0;
      s_flag = 0;
      s_kdim = 0;
    }
    __syncthreads();
    int kdim = 0;
    for (int j = 0; j < km; ++j) {
      const double* vj = V + (int64_t)j * n;
      for (int i = tid; i < n; i += nt) w[i] = vj[i];
      __syncthreads();
      mass_apply<DIM>(g, E, fm, P, w, u);  // u = M v_j
      __syncthreads();
      for (int i = tid; i < n; i += nt) w[i] = u[i];
      __syncthreads();
      bl_solve<double, double>(F, P.nb, P.w, w, tmp);  // w = (K + sigma M)^{-1} M v_j
      double a = 0.0;
      for (int i = tid; i < n; i += nt) a += u[i] * w[i];
      a = block_sum_dyn(a, red);
      if (tid == 0) al[j] = a;
      __syncthreads();
      a = al[j];
      const double bj = be[j];
      for (int i = tid; i < n; i += nt) w[i] -= a * vj[i] + ((j > 0) ? bj * vj[i - n] : 0.0);
      __syncthreads();
      // full re-orthogonalisation against V[0..j] and the locked vectors (twice)
      for (int pass = 0; pass < 2; ++pass) {
        mass_apply<DIM>(g, E, fm, P, w, u);
        __syncthreads();
        const int nq = j + 1 + nl;
        for (int q = tid >> 5; q < nq; q += nt >> 5) {
          const double* vq = (q <= j) ? V + (int64_t)q * n : LK + (int64_t)(q - j - 1) * n;
          double s = 0.0;
          for (int i = tid & 31; i < n; i += 32) s += u[i] * vq[i];
          s = warp_sum(s);
          if ((tid & 31) == 0) hcoef[q] = s;
        }
        __syncthreads();
        for (int i = tid; i < n; i += nt) {
          double s = w[i];
          for (int q = 0; q <= j; ++q) s -= hcoef[q] * V[(int64_t)q * n + i];
          for (int q = 0; q < nl; ++q) s -= hcoef[j + 1 + q] * LK[(int64_t)q * n + i];
          w[i] = s;
        }
        __syncthreads();
      }
      mass_apply<DIM>(g, E, fm, P, w, u);
      __syncthreads();
      double b2 = 0.0;
      for (int i = tid; i < n; i += nt) b2 += w[i] * u[i];
      b2 = block_sum_dyn(b2, red);
      if (tid == 0) be[j + 1] = sqrt(fmax(b2, 0.0));
      __syncthreads();
      const double bn = be[j + 1];
      kdim = j + 1;
      const bool breakdown = !(bn > 1e-13 * fabs(a));
      if (!breakdown && j + 1 < km) {
        double* vn = V + (int64_t)(j + 1) * n;
        for (int i = tid; i < n; i += nt) vn[i] = w[i] / bn;
      }
      // convergence test of the top `need` Ritz pairs
      const bool check = breakdown || (j + 1 == km) || ((kdim >= need + 2) && ((kdim % 4) == 0));
      if (check) {
        const int nchk = min(need, kdim);
        if (tid < nchk) {
          double th = tri_eig_bisect(al, be, kdim, kdim - 1 - tid);
          theta[tid] = th;
        }
        __syncthreads();
        if (tid == 0) {
          for (int q = 0; q < nchk; ++q) {
            tri_eigvec(al, be, kdim, theta[q], tS, tD, tC, tF, tL, tP);
            resid[q] = fabs(bn * tS[kdim - 1]);
          }
        }
        __syncthreads();
        if (tid == 0) {
          int ok = 1;
          for (int q = 0; q < nchk; ++q)
            if (!(resid[q] <= 1e-10 * fabs(theta[q]))) ok = 0;
          s_flag = (ok || breakdown || (j + 1 == km)) ? 1 : 0;
        }
        __syncthreads();
        if (s_flag) break;
      }
      __syncthreads();
    }
    // lock converged Ritz pairs below tau (or the first one, if none is)
    {
      const int nchk = min(need, kdim);
      if (tid < nchk) {
        theta[tid] = tri_eig_bisect(al, be, kdim, kdim - 1 - tid);
      }
      __syncthreads();
      for (int q = 0; q < nchk; ++q) {
        // Ritz vector coefficients (computed by thread 0 into hcoef)
        if (tid == 0) {
          tri_eigvec(al, be, kdim, theta[q], hcoef, tD, tC, tF, tL, tP);
          resid[q] = fabs(be[kdim] * hcoef[kdim - 1]);
        }
        __syncthreads();
        const bool conv = resid[q] <= 1e-8 * fabs(theta[q]);
        const bool below = theta[q] > th_tau;
        const int nlk = s_nlock;
        if (conv && (below || nlk == 0) && nlk < EIG_MAXLOCK && nlk < target) {
          double* dst = LK + (int64_t)nlk * n;
          for (int i = tid; i < n; i += nt) {
            double s = 0.0;
            for (int m = 0; m < kdim; ++m) s += hcoef[m] * V[(int64_t)m * n + i];
            dst[i] = s;
          }
          __syncthreads();
          if (tid == 0) {
            lockval[nlk] = 1.0 / theta[q] - sigma;
            s_nlock = nlk + 1;
          }
        }
        __syncthreads();
      }
    }
    __syncthreads();
    if (s_nlock == 0) break;  // no progress possible
  }
  // store the selected eigenpairs, sorted by eigenvalue
  const int nlock = s_nlock;
  __syncthreads();
  if (tid == 0) {
    count_out[pi] = neg;
    found_out[pi] = nlock;
  }
  // order
  __shared__ int order[EIG_MAXLOCK];
  if (tid == 0) {
    for (int q = 0; q < nlock; ++q) order[q] = q;
    for (int a = 1; a < nlock; ++a)
      for (int b = a; b > 0 && lockval[order[b]] < lockval[order[b - 1]]; --b) {
        int t = order[b];
        order[b] = order[b - 1];
        order[b - 1] = t;
      }
    for (int q = 0; q < TS_MAXMODES; ++q) lam_out[(int64_t)pi * TS_MAXMODES + q] = (q < nlock) ? lockval[order[q]] : __longlong_as_double(0x7ff8000000000000LL);
  }
  __syncthreads();
  const int nst = min(nlock, max_modes);
  for (int q = 0; q < nst; ++q) {
    const double* src = LK + (int64_t)order[q] * n;
    double* dst = psi + P.vec_off + (int64_t)q * n;
    for (int i = tid; i < n; i += nt) dst[i] = src[i];
  }
}

// ---------------------------------------------------------------------------
// coarse basis evaluation
// ---------------------------------------------------------------------------
struct CoarseView {
  Geom g;
  const uint8_t* fm;
  const CoarseNodeInfo* cn;
  const HeatProb* hp;
  const double* psi;
  const int* cdof_node;
  const int* cdof_kind;
  const int* cdof_mode;
};

__device__ __forceinline__ double chi_at(const Geom& g, const int* cidx, const int* a) {
  double v = 1.0;
  for (int d = 0; d < g.dim; ++d) {
    double t = 1.0 - fabs((double)(a[d] - cidx[d] * g.H[d])) / (double)g.H[d];
    v *= (t > 0.0) ? t : 0.0;
  }
  return v;
}

// value of coarse basis DOF k at node a (global coords), component c
__device__ double phi_at(const CoarseView& V, int k, const int* a, int c) {
  const Geom& g = V.g;
  const int l = V.cdof_node[k], kind = V.cdof_kind[k];
  const CoarseNodeInfo& N = V.cn[l];
  const double ch = chi_at(g, N.idx, a);
  if (ch == 0.0) return 0.0;
  const int64_t node = node_id_c(g, a);
  if (!V.fm[g.dim * node + c]) return 0.0;
  if (kind < g.dim) {
    if (kind != c) return 0.0;
    const HeatProb& P = V.hp[N.prob[c]];
    int li = 0, stride = 1;
    for (int d = 0; d < g.dim; ++d) {
      int off = a[d] - P.lo[d];
      if (off < 0 || a[d] > P.hi[d]) return 0.0;
      li += off * stride;
      stride *= P.hi[d] - P.lo[d] + 1;
    }
    return ch * V.psi[P.vec_off + (int64_t)V.cdof_mode[k] * P.nloc + li];
  }
  // rotation about y_l
  double rel[3] = {0, 0, 0};
  for (int d = 0; d < g.dim; ++d) rel[d] = (double)(a[d] - N.idx[d] * g.H[d]);
  const int r = kind - g.dim;
  double val;
  if (g.dim == 2) {
    val = (c == 0) ? -rel[1] : rel[0];
  } else {
    // r = 0: (0, -z, y); r = 1: (z, 0, -x); r = 2: (-y, x, 0)
    const double R[3][3] = {{0.0, -rel[2], rel[1]}, {rel[2], 0.0, -rel[0]}, {-rel[1], rel[0], 0.0}};
    val = R[r][c];
  }
  return ch * val;
}

// ---------------------------------------------------------------------------
// K_0 column k: v = K Phi_k on the closed omega box, K_0[j][k] = Phi_j . v
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(256) k_k0_column(CoarseView V, const double* __restrict__ E, int nc, int ldk,
                                                   double* __restrict__ K0) {
  extern __shared__ double sm[];
  __shared__ double red[32];
  const Geom& g = V.g;
  const int k = blockIdx.x;
  const int l = V.cdof_node[k];
  const CoarseNodeInfo N = V.cn[l];
  // closed omega box of node l
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, bn[3] = {1, 1, 1};
  int nloc = 1;
  for (int d = 0; d < DIM; ++d) {
    lo[d] = max(0, (N.idx[d] - 1) * g.H[d]);
    hi[d] = min(g.n[d], (N.idx[d] + 1) * g.H[d]);
    bn[d] = hi[d] - lo[d] + 1;
    nloc *= bn[d];
  }
  double* phi = sm;               // nloc * DIM
  double* v = phi + nloc * DIM;   // nloc * DIM
  for (int e = threadIdx.x; e < nloc * DIM; e += blockDim.x) {
    int i = e / DIM, c = e % DIM;
    int a[3] = {lo[0] + i % bn[0], lo[1] + (i / bn[0]) % bn[1], (DIM == 3) ? lo[2] + i / (bn[0] * bn[1]) : 0};
    phi[e] = phi_at(V, k, a, c);
  }
  __syncthreads();
  // v = K phi restricted to elements of the box (phi vanishes outside)
  for (int i = threadIdx.x; i < nloc; i += blockDim.x) {
    int a[3] = {lo[0] + i % bn[0], lo[1] + (i / bn[0]) % bn[1], (DIM == 3) ? lo[2] + i / (bn[0] * bn[1]) : 0};
    double acc[DIM];
    for (int r = 0; r < DIM; ++r) acc[r] = 0.0;
    for (int q = 0; q < (1 << DIM); ++q) {
      int ee[3];
      bool ok = true;
      for (int d = 0; d < DIM; ++d) {
        ee[d] = a[d] - 1 + ((q >> d) & 1);
        if (ee[d] < lo[d] || ee[d] >= hi[d]) ok = false;
      }
      if (!ok) continue;
      double Ee = (DIM == 2) ? E[(int64_t)ee[1] * g.nx + ee[0]] : E[((int64_t)ee[2] * g.ny + ee[1]) * g.nx + ee[0]];
      int la;
      if (DIM == 2)
        la = q4_local(a[0] - ee[0], a[1] - ee[1]);
      else
        la = hex8_local(a[0] - ee[0], a[1] - ee[1], a[2] - ee[2]);
      for (int b = 0; b < (1 << DIM); ++b) {
        // local node b of the element in the q4/hex8 numbering
        int bx, by, bz;
        if (DIM == 2) {
          int lb = b;  // iterate local node ids directly
          bx = (lb == 1 || lb == 2) ? 1 : 0;
          by = (lb >= 2) ? 1 : 0;
          bz = 0;
        } else {
          int lb = b;
          int f = lb & 3;
          bx = (f == 1 || f == 2) ? 1 : 0;
          by = (f >= 2) ? 1 : 0;
          bz = lb >> 2;
        }
        int nbx = ee[0] + bx - lo[0], nby = ee[1] + by - lo[1], nbz = (DIM == 3) ? ee[2] + bz - lo[2] : 0;
        int j = nbx + bn[0] * (nby + bn[1] * nbz);
        for (int r = 0; r < DIM; ++r) {
          double s = 0.0;
          for (int c = 0; c < DIM; ++c) s += c_KE[(DIM * la + r) * (DIM == 2 ? 8 : 24) + DIM * b + c] * phi[j * DIM + c];
          acc[r] += Ee * s;
        }
      }
    }
    for (int r = 0; r < DIM; ++r) v[i * DIM + r] = acc[r];
  }
  __syncthreads();
  // dots with the basis functions of the neighbouring coarse nodes
  double* col = K0 + (int64_t)k * ldk;  // K_0 is symmetric: write column k as row k
  for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int ci[3] = {N.idx[0] + dx, N.idx[1] + dy, N.idx[2] + dz};
        bool ok = true;
        for (int d = 0; d < DIM; ++d)
          if (ci[d] < 0 || ci[d] >= g.ncn[d]) ok = false;
        if (!ok) continue;
        int l2 = ci[0] + g.ncn[0] * (ci[1] + g.ncn[1] * ((DIM == 3) ? ci[2] : 0));
        const CoarseNodeInfo N2 = V.cn[l2];
        for (int jj = 0; jj < N2.ndof; ++jj) {
          const int j = N2.first_dof + jj;
          double s = 0.0;
          for (int e = threadIdx.x; e < nloc * DIM; e += blockDim.x) {
            double vv = v[e];
            if (vv == 0.0) continue;
            int i = e / DIM, c = e % DIM;
            int a[3] = {lo[0] + i % bn[0], lo[1] + (i / bn[0]) % bn[1],
                        (DIM == 3) ? lo[2] + i / (bn[0] * bn[1]) : 0};
            s += phi_at(V, j, a, c) * vv;
          }
          s = block_sum_dyn(s, red);
          if (threadIdx.x == 0) col[j] = s;
          __syncthreads();
        }
      }
}

// ---------------------------------------------------------------------------
// dense blocked Cholesky (lower) and triangular inverse, FP64, tile 64
// ---------------------------------------------------------------------------
constexpr int TB = 64;

// factor the diagonal tile kk in place; write its inverse to Linv (TB x TB).
// A pivot below 1e-12 of its original diagonal marks a coarse basis vector
// that depends on the earlier ones (e.g. the rotations chi_l r_l sum to zero
// when every coarse node keeps one): it is dropped -- unit pivot, zero column
// -- which leaves span(R_0^T) and hence the Galerkin correction unchanged.
__global__ void __launch_bounds__(256) k_potrf_tile(double* __restrict__ A, int ld, int kk, double* __restrict__ Linv,
                                                    const double* __restrict__ diag0, int* __restrict__ dropped,
                                                    int* status) {
  __shared__ double T[TB][TB + 1];
  __shared__ double I[TB][TB + 1];
  __shared__ int s_drop;
  const int tid = threadIdx.x;
  double* base = A + (int64_t)kk * TB * ld + (int64_t)kk * TB;
  for (int e = tid; e < TB * TB; e += blockDim.x) T[e / TB][e % TB] = base[(int64_t)(e / TB) * ld + e % TB];
  __syncthreads();
  for (int j = 0; j < TB; ++j) {
    if (tid == 0) {
      double d = T[j][j];
      const double d0 = diag0[kk * TB + j];
      s_drop = 0;
      if (!(d > 1e-12 * d0)) {
        if (!(d > -1e-8 * d0)) atomicOr(status, 2);  // clearly negative: K_0 not SPD
        dropped[kk * TB + j] = 1;
        s_drop = 1;
        T[j][j] = 1.0;
      } else {
        T[j][j] = sqrt(d);
      }
    }
    __syncthreads();
    double djj = T[j][j];
    const bool drop = s_drop != 0;
    for (int i = j + 1 + tid; i < TB; i += blockDim.x) T[i][j] = drop ? 0.0 : T[i][j] / djj;
    __syncthreads();
    const int m = TB - j - 1;
    for (int e = tid; e < m * m; e += blockDim.x) {
      int i = j + 1 + e / m, c = j + 1 + e % m;
      if (c <= i) T[i][c] -= T[i][j] * T[c][j];
    }
    __syncthreads();
  }
  // inverse of the lower triangle, one column per thread
  for (int c = tid; c < TB; c += blockDim.x) {
    for (int i = 0; i < TB; ++i) I[i][c] = 0.0;
    I[c][c] = 1.0 / T[c][c];
    for (int i = c + 1; i < TB; ++i) {
      double s = 0.0;
      for (int m = c; m < i; ++m) s += T[i][m] * I[m][c];
      I[i][c] = -s / T[i][i];
    }
  }
  __syncthreads();
  for (int e = tid; e < TB * TB; e += blockDim.x) {
    int i = e / TB, c = e % TB;
    base[(int64_t)i * ld + c] = (c <= i) ? T[i][c] : 0.0;
    Linv[e] = I[i][c];
  }
}

// panel: A_ik <- A_ik * Linv^T for tiles i > kk
__global__ void __launch_bounds__(256) k_trsm_tiles(double* __restrict__ A, int ld, int kk, int nt,
                                                    const double* __restrict__ Linv, const int* __restrict__ dropped) {
  __shared__ double X[TB][TB + 1];
  __shared__ double Li[TB][TB + 1];
  const int i = kk + 1 + blockIdx.x;
  if (i >= nt) return;
  double* base = A + (int64_t)i * TB * ld + (int64_t)kk * TB;
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    X[e / TB][e % TB] = base[(int64_t)(e / TB) * ld + e % TB];
    Li[e / TB][e % TB] = Linv[e];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    int r = e / TB, c = e % TB;
    double s = 0.0;
    for (int m = 0; m <= c; ++m) s += X[r][m] * Li[c][m];
    base[(int64_t)r * ld + c] = dropped[kk * TB + c] ? 0.0 : s;
  }
}

__global__ void k_get_diag(const double* __restrict__ A, int ld, double* __restrict__ d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ld) d[i] = A[(int64_t)i * ld + i];
}

// rows of dropped coarse DOFs of X = L^{-1} are zeroed: those DOFs then take
// no part in u0 = X^T X r0
__global__ void k_zero_dropped_rows(double* __restrict__ X, int ld, const int* __restrict__ dropped) {
  const int row = blockIdx.x;
  if (!dropped[row]) return;
  for (int c = threadIdx.x; c < ld; c += blockDim.x) X[(int64_t)row * ld + c] = 0.0;
}

// trailing update: A_ij -= A_ik A_jk^T for kk < j <= i < nt
__global__ void __launch_bounds__(256) k_syrk_tiles(double* __restrict__ A, int ld, int kk, int nt) {
  __shared__ double Pi[TB][TB + 1];
  __shared__ double Pj[TB][TB + 1];
  const int m = nt - kk - 1;
  int t = blockIdx.x;
  // map t -> (i, j) in the lower triangle of an m x m tile grid
  int ii = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
  while (ii * (ii + 1) / 2 > t) --ii;
  int jj = t - ii * (ii + 1) / 2;
  if (ii >= m) return;
  const int i = kk + 1 + ii, j = kk + 1 + jj;
  const double* ai = A + (int64_t)i * TB * ld + (int64_t)kk * TB;
  const double* aj = A + (int64_t)j * TB * ld + (int64_t)kk * TB;
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    Pi[e / TB][e % TB] = ai[(int64_t)(e / TB) * ld + e % TB];
    Pj[e / TB][e % TB] = aj[(int64_t)(e / TB) * ld + e % TB];
  }
  __syncthreads();
  double* c = A + (int64_t)i * TB * ld + (int64_t)j * TB;
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    int r = e / TB, q = e % TB;
    double s = 0.0;
#pragma unroll 8
    for (int mm = 0; mm < TB; ++mm) s += Pi[r][mm] * Pj[q][mm];
    c[(int64_t)r * ld + q] -= s;
  }
}

// X = L^{-1} block row by block row:  X_ij = -Linv_ii * sum_{m=j}^{i-1} L_im X_mj  (j < i)
// launched for one block row i; blockIdx.x = j in [0, i)
__global__ void __launch_bounds__(256) k_trtri_row(const double* __restrict__ L, double* __restrict__ X, int ld, int i,
                                                   const double* __restrict__ Linv_ii) {
  __shared__ double Acc[TB][TB + 1];
  __shared__ double Pa[TB][TB + 1];
  __shared__ double Pb[TB][TB + 1];
  const int j = blockIdx.x;
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) Acc[e / TB][e % TB] = 0.0;
  __syncthreads();
  for (int m = j; m < i; ++m) {
    const double* lim = L + (int64_t)i * TB * ld + (int64_t)m * TB;
    const double* xmj = X + (int64_t)m * TB * ld + (int64_t)j * TB;
    for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
      Pa[e / TB][e % TB] = lim[(int64_t)(e / TB) * ld + e % TB];
      Pb[e / TB][e % TB] = xmj[(int64_t)(e / TB) * ld + e % TB];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
      int r = e / TB, c = e % TB;
      double s = 0.0;
#pragma unroll 8
      for (int q = 0; q < TB; ++q) s += Pa[r][q] * Pb[q][c];
      Acc[r][c] += s;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) Pa[e / TB][e % TB] = Linv_ii[e];
  __syncthreads();
  double* out = X + (int64_t)i * TB * ld + (int64_t)j * TB;
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    int r = e / TB, c = e % TB;
    double s = 0.0;
    for (int q = 0; q <= r; ++q) s += Pa[r][q] * Acc[q][c];
    out[(int64_t)r * ld + c] = -s;
  }
}

__global__ void k_copy_tile(const double* __restrict__ src, double* __restrict__ X, int ld, int i) {
  double* out = X + (int64_t)i * TB * ld + (int64_t)i * TB;
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) out[(int64_t)(e / TB) * ld + e % TB] = src[e];
}

__global__ void k_transpose(const double* __restrict__ X, double* __restrict__ XT, int n) {
  __shared__ double t[32][33];
  int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) t[r][threadIdx.x] = X[(int64_t)(by + r) * n + bx + threadIdx.x];
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) XT[(int64_t)(bx + r) * n + by + threadIdx.x] = t[threadIdx.x][r];
}

__global__ void k_pad_identity(double* __restrict__ A, int ld, int nc) {
  int i = nc + blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ld) A[(int64_t)i * ld + i] = 1.0;
}

// ---------------------------------------------------------------------------
// per-iteration coarse kernels
// ---------------------------------------------------------------------------
// r0[k] = Phi_k . r   (one warp per coarse DOF)
template <int DIM>
__global__ void __launch_bounds__(256) k_coarse_restrict(CoarseView V, const double* __restrict__ r, int nc,
                                                         double* __restrict__ r0, const int* done) {
  if (done && *done) return;
  const Geom& g = V.g;
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= nc) return;
  const int l = V.cdof_node[k];
  const CoarseNodeInfo& N = V.cn[l];
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, bn[3] = {1, 1, 1};
  int nloc = 1;
  for (int d = 0; d < DIM; ++d) {
    lo[d] = max(0, (N.idx[d] - 1) * g.H[d]);
    hi[d] = min(g.n[d], (N.idx[d] + 1) * g.H[d]);
    bn[d] = hi[d] - lo[d] + 1;
    nloc *= bn[d];
  }
  const int kind = V.cdof_kind[k];
  double s = 0.0;
  for (int i = lane; i < nloc; i += 32) {
    int a[3] = {lo[0] + i % bn[0], lo[1] + (i / bn[0]) % bn[1], (DIM == 3) ? lo[2] + i / (bn[0] * bn[1]) : 0};
    int64_t node = node_id_c(g, a);
    if (kind < DIM) {
      s += phi_at(V, k, a, kind) * r[DIM * node + kind];
    } else {
      for (int c = 0; c < DIM; ++c) s += phi_at(V, k, a, c) * r[DIM * node + c];
    }
  }
  s = warp_sum(s);
  if (lane == 0) r0[k] = s;
}

// y = A x for a dense row-major n x n matrix restricted to a triangle
// (lower: columns <= row; upper: columns >= row).  One warp per row.
__global__ void __launch_bounds__(256) k_tri_gemv(const double* __restrict__ A, int ld, int n, bool lower,
                                                  const double* __restrict__ x, double* __restrict__ y,
                                                  const int* done) {
  if (done && *done) return;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* a = A + (int64_t)row * ld;
  int c0 = lower ? 0 : row, c1 = lower ? row + 1 : n;
  double s = 0.0;
  for (int c = c0 + lane; c < c1; c += 32) s += a[c] * x[c];
  s = warp_sum(s);
  if (lane == 0) y[row] = s;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static CoarseView coarse_view(ts_handle h) {
  CoarseView V;
  V.g = h->g;
  V.fm = h->freemask;
  V.cn = h->cn;
  V.hp = h->hp;
  V.psi = h->psi;
  V.cdof_node = h->cdof_node;
  V.cdof_kind = h->cdof_kind;
  V.cdof_mode = h->cdof_mode;
  return V;
}

void build_coarse(ts_handle h, const std::vector<uint8_t>& fm_h) {
  Geom& g = h->g;
  cudaStream_t st = h->ctx->stream;
  const int dim = g.dim;
  for (int a = 0; a < dim; ++a) g.ncn[a] = g.n[a] / g.H[a] + 1;
  for (int a = dim; a < 3; ++a) g.ncn[a] = 1;
  const int ncn = g.ncn[0] * g.ncn[1] * g.ncn[2];
  h->n_cnodes = ncn;
  const double H = (double)std::max(std::max(g.H[0], g.H[1]), dim == 3 ? g.H[2] : 0);
  const double tau = h->opt.tau_scale / (H * H);
  // Shift of the spectral transformation (K + sigma M)^{-1} M.  The
  // contrast-dependent eigenvalues are O(Emin/E0) * tau; a shift of that size
  // keeps them apart after the transformation (a shift near tau would map
  // them all to ~1/tau and Lanczos could not resolve their order).
  const double sigma = tau * std::max(h->Emin / h->E0, 1e-10);
  auto nid = [&](const int* a) -> int64_t {
    if (dim == 2) return (int64_t)a[1] * (g.nx + 1) + a[0];
    return ((int64_t)a[2] * (g.ny + 1) + a[1]) * (g.nx + 1) + a[0];
  };
  std::vector<CoarseNodeInfo> cn(ncn);
  std::vector<HeatProb> hp;
  int64_t fac_off = 0, vec_off = 0;
  int max_w = 0, max_n = 0;
  for (int l = 0; l < ncn; ++l) {
    CoarseNodeInfo& N = cn[l];
    N.idx[0] = l % g.ncn[0];
    N.idx[1] = (l / g.ncn[0]) % g.ncn[1];
    N.idx[2] = (dim == 3) ? l / (g.ncn[0] * g.ncn[1]) : 0;
    int y[3] = {N.idx[0] * g.H[0], N.idx[1] * g.H[1], N.idx[2] * (dim == 3 ? g.H[2] : 0)};
    int64_t ynode = nid(y);
    HeatProb P{};
    int nloc = 1;
    for (int d = 0; d < dim; ++d) {
      P.lo[d] = std::max(0, (N.idx[d] - 1) * g.H[d]);
      P.hi[d] = std::min(g.n[d], (N.idx[d] + 1) * g.H[d]);
      nloc *= P.hi[d] - P.lo[d] + 1;
    }
    P.nloc = nloc;
    P.l = l;
    if (dim == 2) {
      P.w = P.hi[0] - P.lo[0] + 1;
      P.nb = P.hi[1] - P.lo[1] + 1;
    } else {
      P.w = (P.hi[0] - P.lo[0] + 1) * (P.hi[1] - P.lo[1] + 1);
      P.nb = P.hi[2] - P.lo[2] + 1;
    }
    bool any_free = false;
    for (int c = 0; c < dim; ++c) {
      N.nmodes[c] = 0;
      N.prob[c] = -1;
      if (!fm_h[dim * ynode + c]) continue;  // y_l on Gamma_D,c: no component-c basis
      any_free = true;
      P.c = c;
      P.dedup_of = -1;
      // identical Dirichlet pattern as an earlier component of this node?
      for (int c2 = 0; c2 < c; ++c2) {
        int pj = N.prob[c2];
        if (pj < 0) continue;
        bool same = true;
        for (int i = 0; i < nloc && same; ++i) {
          int a[3];
          int bx = P.hi[0] - P.lo[0] + 1, by = (dim == 3) ? P.hi[1] - P.lo[1] + 1 : 1;
          a[0] = P.lo[0] + i % bx;
          a[1] = P.lo[1] + (i / bx) % by;
          a[2] = (dim == 3) ? P.lo[2] + i / (bx * by) : 0;
          if (dim == 2) a[1] = P.lo[1] + i / bx;
          int64_t nd = nid(a);
          if (fm_h[dim * nd + c] != fm_h[dim * nd + c2]) same = false;
        }
        if (same) {
          P.dedup_of = hp[pj].dedup_of >= 0 ? hp[pj].dedup_of : pj;
          break;
        }
      }
      if (P.dedup_of < 0) {
        P.fac_off = fac_off;
        fac_off += bl_size(P.w, P.nb);
        P.vec_off = vec_off;
        vec_off += (int64_t)h->opt.max_modes * nloc;
        max_w = std::max(max_w, P.w);
        max_n = std::max(max_n, nloc);
      } else {
        P.fac_off = hp[P.dedup_of].fac_off;
        P.vec_off = hp[P.dedup_of].vec_off;
      }
      N.prob[c] = (int)hp.size();
      hp.push_back(P);
    }
    N.nrot = (h->opt.rotations && any_free) ? (dim == 2 ? 1 : 3) : 0;
  }
  const int nprob = (int)hp.size();
  h->n_hprob = nprob;
  h->hp_h = hp;
  h->hp = dupload(h, hp);
  h->hp_count = dalloc<int>(h, nprob);
  h->hp_found = dalloc<int>(h, nprob);
  h->hp_lambda = dalloc<double>(h, (size_t)nprob * TS_MAXMODES);
  h->heat_fac = dalloc<double>(h, fac_off);
  h->psi = dalloc<double>(h, vec_off);
  TS_CUDA(cudaMemsetAsync(h->hp_count, 0, sizeof(int) * std::max(nprob, 1), st));
  TS_CUDA(cudaMemsetAsync(h->hp_found, 0, sizeof(int) * std::max(nprob, 1), st));
  const int kmax = std::min(TS_LANCZOS_MAX - 1, 80);
  // Lanczos workspace, processed in batches of problems
  const int batch = std::max(1, std::min(nprob, 4096));
  const int64_t ws_per = (int64_t)(kmax + 1 + TS_MAXMODES) * max_n;
  double* ws = dalloc<double>(h, (size_t)batch * ws_per);
  size_t smem = std::max(bl_factor_smem(max_w), (size_t)(2 * max_n + 2 * max_w) * sizeof(double) + 64);
  if (smem > 227 * 1024) throw TsError(TS_ERR_INVALID, "coarse neighbourhood too large for shared memory");
  if (nprob > 0) {
    if (dim == 2) {
      TS_CUDA(cudaFuncSetAttribute(k_heat_eig<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    } else {
      TS_CUDA(cudaFuncSetAttribute(k_heat_eig<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    for (int p0 = 0; p0 < nprob; p0 += batch) {
      int cnt = std::min(batch, nprob - p0);
      if (dim == 2)
        tsl(h), k_heat_eig<2><<<cnt, EIG_THREADS, smem, st>>>(g, h->E, h->freemask, h->hp, p0, p0 + cnt, tau, sigma,
                                                      h->opt.max_modes, kmax, h->heat_fac, h->psi, h->hp_lambda,
                                                      h->hp_count, h->hp_found, ws, ws_per, h->dstatus);
      else
        tsl(h), k_heat_eig<3><<<cnt, EIG_THREADS, smem, st>>>(g, h->E, h->freemask, h->hp, p0, p0 + cnt, tau, sigma,
                                                      h->opt.max_modes, kmax, h->heat_fac, h->psi, h->hp_lambda,
                                                      h->hp_count, h->hp_found, ws, ws_per, h->dstatus);
      TS_CUDA(cudaGetLastError());
    }
  }
  // read back counts to number the coarse DOFs
  std::vector<int> count(nprob), found(nprob);
  if (nprob) {
    TS_CUDA(cudaMemcpyAsync(count.data(), h->hp_count, sizeof(int) * nprob, cudaMemcpyDeviceToHost, st));
    TS_CUDA(cudaMemcpyAsync(found.data(), h->hp_found, sizeof(int) * nprob, cudaMemcpyDeviceToHost, st));
  }
  TS_CUDA(cudaStreamSynchronize(st));
  h->cap_hits = 0;
  h->eig_unconv = 0;
  std::vector<int> cdof_node, cdof_kind, cdof_mode;
  int nc = 0;
  for (int l = 0; l < ncn; ++l) {
    CoarseNodeInfo& N = cn[l];
    N.first_dof = nc;
    for (int c = 0; c < dim; ++c) {
      int pi = N.prob[c];
      if (pi < 0) continue;
      int src = hp[pi].dedup_of >= 0 ? hp[pi].dedup_of : pi;
      int cntb = count[src];
      int want = std::min(std::max(cntb, 1), h->opt.max_modes);
      if (cntb > h->opt.max_modes) h->cap_hits++;
      int got = std::min(found[src], want);
      if (got < want) h->eig_unconv++;
      N.nmodes[c] = got;
      N.prob[c] = src;  // the problem that holds the eigenvectors
      for (int m = 0; m < got; ++m) {
        cdof_node.push_back(l);
        cdof_kind.push_back(c);
        cdof_mode.push_back(m);
      }
      nc += got;
    }
    for (int r = 0; r < N.nrot; ++r) {
      cdof_node.push_back(l);
      cdof_kind.push_back(dim + r);
      cdof_mode.push_back(0);
    }
    nc += N.nrot;
    N.ndof = nc - N.first_dof;
  }
  // keep per-problem counts for introspection (counts of deduplicated problems)
  for (int pi = 0; pi < nprob; ++pi) {
    int src = hp[pi].dedup_of >= 0 ? hp[pi].dedup_of : pi;
    count[pi] = count[src];
    found[pi] = found[src];
  }
  TS_CUDA(cudaMemcpyAsync(h->hp_count, count.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice, st));
  TS_CUDA(cudaMemcpyAsync(h->hp_found, found.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice, st));
  h->cn_h = cn;
  h->cn = dupload(h, cn);
  h->nc = nc;
  if (nc == 0) return;
  h->cdof_node = dupload(h, cdof_node);
  h->cdof_kind = dupload(h, cdof_kind);
  h->cdof_mode = dupload(h, cdof_mode);
  // K_0 (padded to a multiple of TB)
  const int ld = ((nc + TB - 1) / TB) * TB;
  const int nt = ld / TB;
  h->K0 = dalloc<double>(h, (size_t)ld * ld);
  h->K0inv_L = dalloc<double>(h, (size_t)ld * ld);
  double* XT = dalloc<double>(h, (size_t)ld * ld);
  h->K0_ld = ld;
  h->K0inv_LT = XT;
  double* Linv = dalloc<double>(h, (size_t)nt * TB * TB);
  h->r0 = dalloc<double>(h, ld);
  h->y0 = dalloc<double>(h, ld);
  h->u0 = dalloc<double>(h, ld);
  TS_CUDA(cudaMemsetAsync(h->K0, 0, sizeof(double) * (size_t)ld * ld, st));
  TS_CUDA(cudaMemsetAsync(h->K0inv_L, 0, sizeof(double) * (size_t)ld * ld, st));
  TS_CUDA(cudaMemsetAsync(h->r0, 0, sizeof(double) * ld, st));
  TS_CUDA(cudaMemsetAsync(h->y0, 0, sizeof(double) * ld, st));
  TS_CUDA(cudaMemsetAsync(h->u0, 0, sizeof(double) * ld, st));
  CoarseView V = coarse_view(h);
  int max_box = 1;
  for (int d = 0; d < dim; ++d) max_box *= 2 * g.H[d] + 1;
  size_t smk = (size_t)2 * max_box * dim * sizeof(double);
  if (smk > 227 * 1024) throw TsError(TS_ERR_INVALID, "coarse neighbourhood too large for the K_0 assembly");
  if (dim == 2) {
    TS_CUDA(cudaFuncSetAttribute(k_k0_column<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smk));
    tsl(h), k_k0_column<2><<<nc, 256, smk, st>>>(V, h->E, nc, ld, h->K0);
  } else {
    TS_CUDA(cudaFuncSetAttribute(k_k0_column<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smk));
    tsl(h), k_k0_column<3><<<nc, 256, smk, st>>>(V, h->E, nc, ld, h->K0);
  }
  TS_CUDA(cudaGetLastError());
  if (ld > nc) tsl(h), k_pad_identity<<<cdiv(ld - nc, 128), 128, 0, st>>>(h->K0, ld, nc);
  // Cholesky
  double* diag0 = dalloc<double>(h, ld);
  h->K0_dropped = dalloc<int>(h, ld);
  TS_CUDA(cudaMemsetAsync(h->K0_dropped, 0, sizeof(int) * ld, st));
  tsl(h), k_get_diag<<<cdiv(ld, 128), 128, 0, st>>>(h->K0, ld, diag0);
  for (int kk = 0; kk < nt; ++kk) {
    tsl(h), k_potrf_tile<<<1, 256, 0, st>>>(h->K0, ld, kk, Linv + (size_t)kk * TB * TB, diag0, h->K0_dropped, h->dstatus);
    if (kk + 1 < nt) {
      tsl(h), k_trsm_tiles<<<nt - kk - 1, 256, 0, st>>>(h->K0, ld, kk, nt, Linv + (size_t)kk * TB * TB, h->K0_dropped);
      int m = nt - kk - 1;
      tsl(h), k_syrk_tiles<<<m * (m + 1) / 2, 256, 0, st>>>(h->K0, ld, kk, nt);
    }
  }
  TS_CUDA(cudaGetLastError());
  // X = L^{-1}: diagonal tiles from the potrf inverses, then block rows in order
  for (int i = 0; i < nt; ++i) {
    tsl(h), k_copy_tile<<<1, 256, 0, st>>>(Linv + (size_t)i * TB * TB, h->K0inv_L, ld, i);
    if (i > 0) tsl(h), k_trtri_row<<<i, 256, 0, st>>>(h->K0, h->K0inv_L, ld, i, Linv + (size_t)i * TB * TB);
  }
  tsl(h), k_zero_dropped_rows<<<ld, 256, 0, st>>>(h->K0inv_L, ld, h->K0_dropped);
  tsl(h), k_transpose<<<dim3(ld / 32, ld / 32), dim3(32, 8), 0, st>>>(h->K0inv_L, XT, ld);
  TS_CUDA(cudaGetLastError());
  std::vector<int> dr(nc);
  TS_CUDA(cudaMemcpyAsync(dr.data(), h->K0_dropped, sizeof(int) * nc, cudaMemcpyDeviceToHost, st));
  TS_CUDA(cudaStreamSynchronize(st));
  h->coarse_dropped = 0;
  for (int v : dr) h->coarse_dropped += v;
}

void launch_coarse_apply(ts_handle h, const double* r) {
  if (h->nc == 0) return;
  cudaStream_t st = h->ctx->stream;
  CoarseView V = coarse_view(h);
  const int* done = h->done_flag;
  const int wpb = 8;
  if (h->g.dim == 2)
    tsl(h), k_coarse_restrict<2><<<cdiv(h->nc, wpb), 32 * wpb, 0, st>>>(V, r, h->nc, h->r0, done);
  else
    tsl(h), k_coarse_restrict<3><<<cdiv(h->nc, wpb), 32 * wpb, 0, st>>>(V, r, h->nc, h->r0, done);
  tsl(h), k_tri_gemv<<<cdiv(h->nc, wpb), 32 * wpb, 0, st>>>(h->K0inv_L, h->K0_ld, h->nc, true, h->r0, h->y0, done);
  tsl(h), k_tri_gemv<<<cdiv(h->nc, wpb), 32 * wpb, 0, st>>>(h->K0inv_LT, h->K0_ld, h->nc, false, h->y0, h->u0, done);
  TS_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// prolongation: z = sum_i R_i^T zloc_i (which & 1) + R_0^T u0 (which & 2),
// node-owner gather; fused partial dots sum dv1.z and sum dv2.z
// ---------------------------------------------------------------------------
constexpr int PRO_THREADS = 256;

template <int DIM, class TZ>
__global__ void __launch_bounds__(PRO_THREADS) k_prolong(CoarseView V, AxisTables ax, const BLDesc* __restrict__ desc,
                                                         const int64_t* __restrict__ zoff, const TZ* __restrict__ zloc,
                                                         const double* __restrict__ u0, int which, double* __restrict__ z,
                                                         double* __restrict__ partials, const double* __restrict__ dv1,
                                                         const double* __restrict__ dv2, const int* done) {
  if (done && *done) return;
  const Geom& g = V.g;
  const int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc1 = 0.0, acc2 = 0.0;
  if (node < g.n_nodes) {
    int a[3];
    a[0] = (int)(node % (g.nx + 1));
    if (DIM == 2) {
      a[1] = (int)(node / (g.nx + 1));
      a[2] = 0;
    } else {
      a[1] = (int)((node / (g.nx + 1)) % (g.ny + 1));
      a[2] = (int)(node / ((int64_t)(g.nx + 1) * (g.ny + 1)));
    }
    double zc[DIM];
    for (int c = 0; c < DIM; ++c) zc[c] = 0.0;
    if (which & 1) {
      int2 cx = ax.cand[0][a[0]], cy = ax.cand[1][a[1]];
      int2 cz = (DIM == 3) ? ax.cand[2][a[2]] : make_int2(0, -1);
      int sx[2] = {cx.x, cx.y}, sy[2] = {cy.x, cy.y}, sz[2] = {cz.x, cz.y};
      for (int iz = 0; iz < 2; ++iz) {
        if (sz[iz] < 0) continue;
        for (int iy = 0; iy < 2; ++iy) {
          if (sy[iy] < 0) continue;
          for (int ix = 0; ix < 2; ++ix) {
            if (sx[ix] < 0) continue;
            int s = sx[ix] + g.nsub[0] * (sy[iy] + g.nsub[1] * sz[iz]);
            const BLDesc d = desc[s];
            int lx = a[0] - ax.sub_lo[0][sx[ix]], ly = a[1] - ax.sub_lo[1][sy[iy]];
            int64_t base;
            if (DIM == 2) {
              base = zoff[s] + (int64_t)ly * d.w + 2 * lx;
            } else {
              int nbx = ax.sub_hi[0][sx[ix]] - ax.sub_lo[0][sx[ix]] + 1;
              int lz = a[2] - ax.sub_lo[2][sz[iz]];
              base = zoff[s] + (int64_t)lz * d.w + 3 * (ly * nbx + lx);
            }
            for (int c = 0; c < DIM; ++c) zc[c] += (double)zloc[base + c];
          }
        }
      }
    }
    if ((which & 2) && u0) {
      // coarse nodes whose hat is nonzero here: per axis floor(a/H) and +1
      int ci[3][2], nci[3];
      for (int d = 0; d < 3; ++d) {
        if (d >= DIM) {
          ci[d][0] = 0;
          nci[d] = 1;
          continue;
        }
        int b = a[d] / g.H[d];
        nci[d] = 0;
        ci[d][nci[d]++] = b;
        if (a[d] % g.H[d] != 0) ci[d][nci[d]++] = b + 1;
      }
      for (int iz = 0; iz < nci[2]; ++iz)
        for (int iy = 0; iy < nci[1]; ++iy)
          for (int ix = 0; ix < nci[0]; ++ix) {
            int l = ci[0][ix] + g.ncn[0] * (ci[1][iy] + g.ncn[1] * ci[2][iz]);
            const CoarseNodeInfo& N = V.cn[l];
            for (int jj = 0; jj < N.ndof; ++jj) {
              const int k = N.first_dof + jj;
              const double uk = u0[k];
              const int kind = V.cdof_kind[k];
              if (kind < DIM)
                zc[kind] += uk * phi_at(V, k, a, kind);
              else
                for (int c = 0; c < DIM; ++c) zc[c] += uk * phi_at(V, k, a, c);
            }
          }
    }
    for (int c = 0; c < DIM; ++c) {
      if (!V.fm[DIM * node + c]) zc[c] = 0.0;
      z[DIM * node + c] = zc[c];
      if (dv1) acc1 += dv1[DIM * node + c] * zc[c];
      if (dv2) acc2 += dv2[DIM * node + c] * zc[c];
    }
  }
  if (partials) {
    double s1 = block_sum<PRO_THREADS>(acc1);
    double s2 = block_sum<PRO_THREADS>(acc2);
    if (threadIdx.x == 0) {
      partials[2 * blockIdx.x] = s1;
      partials[2 * blockIdx.x + 1] = s2;
    }
  }
}

int prolong_blocks(const Geom& g) { return cdiv(g.n_nodes, PRO_THREADS); }

void launch_prolong(ts_handle h, double* z, int which, double* partials, const double* dv1, const double* dv2) {
  const Geom& g = h->g;
  cudaStream_t st = h->ctx->stream;
  CoarseView V = coarse_view(h);
  const double* u0 = (h->nc > 0) ? h->u0 : nullptr;
  const int nb = prolong_blocks(g);
  const int* done = h->done_flag;
  if (h->opt.precision == TS_MIXED_FP32) {
    if (g.dim == 2)
      tsl(h), k_prolong<2, float><<<nb, PRO_THREADS, 0, st>>>(V, h->ax, h->sub_desc, h->zloc_off, h->zloc32, u0, which, z,
                                                      partials, dv1, dv2, done);
    else
      tsl(h), k_prolong<3, float><<<nb, PRO_THREADS, 0, st>>>(V, h->ax, h->sub_desc, h->zloc_off, h->zloc32, u0, which, z,
                                                      partials, dv1, dv2, done);
  } else {
    if (g.dim == 2)
      tsl(h), k_prolong<2, double><<<nb, PRO_THREADS, 0, st>>>(V, h->ax, h->sub_desc, h->zloc_off, h->zloc, u0, which, z,
                                                       partials, dv1, dv2, done);
    else
      tsl(h), k_prolong<3, double><<<nb, PRO_THREADS, 0, st>>>(V, h->ax, h->sub_desc, h->zloc_off, h->zloc, u0, which, z,
                                                       partials, dv1, dv2, done);
  }
  TS_CUDA(cudaGetLastError());
}
