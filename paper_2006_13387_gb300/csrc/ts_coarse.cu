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
//                  block LU over node lines (Sylvester: number of negative
//                  pivots = number of eigenvalues below tau), factor of
//                  K + sigma M, then shift-invert Lanczos in the M inner
//                  product (DGKS re-orthogonalisation, a second pass only when
//                  the first lost too much) with deflated restarts (for
//                  repeated eigenvalues) until that many Ritz pairs converged.
//   k_k0_column    one CTA per coarse DOF k: v = K Phi_k on omega_l, then
//                  K_0[j][k] = Phi_j . v for the DOFs of the neighbouring nodes.
// The factor and solve of K_0 are in ts_cfactor.cu (block cyclic reduction).
#include <algorithm>
#include <cmath>

#include "ts_fe_entries.cuh"
#include "ts_heatline.cuh"
#include "ts_internal.cuh"
#include "ts_reduce.cuh"

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

// --- small symmetric tridiagonal helpers (one thread each) -----------------
// T: diagonal al[0..k), off-diagonal be[1..k) (b2[i] = be[i]^2).
//
// Number of eigenvalues of T below x: sign changes of the leading principal
// minors p_i = det(T_i - x I), p_{i+1} = (al_i - x) p_i - b2_i p_{i-1}
// (Sturm).  The recurrence needs no division: its steps form one short chain
// of dependent FP64 operations; the two latest minors are rescaled by a power
// of two whenever they leave [2^-256, 2^256], which changes no sign.  A zero
// minor takes the sign opposite to its predecessor (as a zero pivot of the
// LDL^T form of T - x I counts as negative).
__device__ int sturm_count(const double* al, const double* b2, int k, double x) {
  int cnt = 0;
  double pp = 1.0, pc = al[0] - x;
  if (pc == 0.0) pc = -1e-300;
  if (pc < 0.0) ++cnt;
  for (int i = 1; i < k; ++i) {
    double pn = fma(al[i] - x, pc, -b2[i] * pp);
    if (pn == 0.0) pn = (pc < 0.0) ? 1e-300 : -1e-300;
    if ((__double_as_longlong(pn) ^ __double_as_longlong(pc)) < 0) ++cnt;
    const int e = (int)((__double_as_longlong(pn) >> 52) & 0x7ff) - 1023;
    if (e > 256) {
      pn *= 0x1p-256;
      pc *= 0x1p-256;
    } else if (e < -256) {
      const int ec = (int)((__double_as_longlong(pc) >> 52) & 0x7ff) - 1023;
      if (ec < -256) {
        pn *= 0x1p256;
        pc *= 0x1p256;
      }
    }
    pp = pc;
    pc = pn;
  }
  return cnt;
}

// idx-th smallest eigenvalue of T by bisection
__device__ double tri_eig_bisect(const double* al, const double* be, const double* b2, int k, int idx) {
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < k; ++i) {
    double r = ((i > 0) ? fabs(be[i]) : 0.0) + ((i + 1 < k) ? fabs(be[i + 1]) : 0.0);
    lo = fmin(lo, al[i] - r);
    hi = fmax(hi, al[i] + r);
  }
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(al, b2, k, mid) > idx)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

// eigenvector of T for eigenvalue th by inverse iteration with a partial-
// pivoting tridiagonal LU; s[0..k) on output (unit 2-norm).  The factor's
// scratch is the calling thread's own, so that the eigenvectors of several
// Ritz values are formed side by side, one thread each.
__device__ void tri_eigvec(const double* al, const double* be, int k, double th, double* s) {
  double D[TS_LANCZOS_MAX], C[TS_LANCZOS_MAX], F[TS_LANCZOS_MAX], L[TS_LANCZOS_MAX];
  unsigned char pv[TS_LANCZOS_MAX];
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
  // pivots replaced by their reciprocals (the solves below multiply)
  for (int i = 0; i < k; ++i) {
    if (fabs(D[i]) < tiny) D[i] = (D[i] < 0 ? -tiny : tiny);
    D[i] = 1.0 / D[i];
  }
  const double s0 = 1.0 / sqrt((double)k);
  for (int i = 0; i < k; ++i) s[i] = s0 * (1.0 + 0.01 * ((i * 7919) % 13));
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
      s[i] = v * D[i];
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

// --- randomized heat basis (the paper's randomized algorithm for the eigen-
// problems, applied to the heat problem of Sec. 4.1) --------------------------
// SplitMix64 output function (Steele, Lea & Flood): the counter-based
// generator of the random loads (counter node << 40 | load << 32 | box node)
__device__ __forceinline__ uint64_t splitmix64_dev(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// value of v broadcast to the block (after a block sum valid in thread 0)
__device__ __forceinline__ double rb_bcast(double v, double* red) {
  if (threadIdx.x == 0) red[31] = v;
  __syncthreads();
  const double r = red[31];
  __syncthreads();
  return r;
}

// M zero-mean random loads on the free nodes, local solves with the factor
// of K + sigma M, the constant mode; the span made M-orthonormal (two
// classical Gram-Schmidt passes, dependent vectors dropped), the reduced
// stiffness Q^T K Q diagonalised by cyclic Jacobi in parallel rounds (round-
// robin pairs), and the Ritz pairs below tau (at least one, at most
// max_modes) locked as the selected modes.  M = max(rand_m, wanted modes +
// 5) (the paper's rank k + 5), at most TS_RAND_MAX and nfree - 1.
template <int DIM>
__device__ void heat_rand_basis(const Geom& g, const uint8_t* __restrict__ fm, const HeatProb& P, int n, int bx,
                                int by, int bz, int neg, int nfree, int km, int rand_m, int max_modes, double tau,
                                const double* F, const double* Cg, const double* Mst, const double* Kst, double* V,
                                double* LK, double* u, double* w, double* tmp, double* sbuf, double* red,
                                double* hcoef, double (*Kr)[TS_RAND_MAX + 2], double* Z, double* Jc, double* Js,
                                int* Jp, int* Jq, int* s_nsel, int* s_nlock, double* lockval, long long& fl,
                                long long fl_mass, long long fl_solve) {
  constexpr int LDZ = TS_RAND_MAX + 2;
  const int tid = threadIdx.x, nt = blockDim.x;
  auto is_free = [&](int i) {
    int a[3];
    box_coords<DIM>(P, i, a);
    return fm[DIM * node_id_c(g, a) + P.c] != 0;
  };
  int M = max(rand_m, min(max(neg, 1), max_modes) + 5);
  M = max(0, min(M, min(TS_RAND_MAX, km - 1)));
  // snapshots u_l = (K + sigma M)^{-1} f_l, zero total load on the free nodes
  for (int l = 0; l < M; ++l) {
    double s = 0.0;
    for (int i = tid; i < n; i += nt) {
      double v = 0.0;
      if (is_free(i)) {
        const uint64_t ctr = ((uint64_t)P.l << 40) | ((uint64_t)l << 32) | (uint64_t)i;
        v = (double)(splitmix64_dev(ctr) >> 11) * 0x1p-53 - 0.5;
      }
      w[i] = v;
      s += v;
    }
    const double mean = rb_bcast(block_sum_dyn(s, red), red) / (double)nfree;
    for (int i = tid; i < n; i += nt)
      if (is_free(i)) w[i] -= mean;
    heat_line_solve<DIM>(F, Cg, P.w, P.nb, bx, by, w, tmp, sbuf);
    __syncthreads();
    for (int i = tid; i < n; i += nt) V[(int64_t)l * n + i] = w[i];
  }
  fl += (long long)M * (fl_solve + 2LL * n);
  for (int i = tid; i < n; i += nt) V[(int64_t)M * n + i] = is_free(i) ? 1.0 : 0.0;
  __syncthreads();
  // M-orthonormal basis Q in V[0 .. mq)
  int mq = 0;
  for (int j = 0; j <= M; ++j) {
    for (int i = tid; i < n; i += nt) w[i] = V[(int64_t)j * n + i];
    __syncthreads();
    hl_mass_apply<DIM>(Mst, w, u, n, bx, by, bz);
    __syncthreads();
    double d0 = 0.0;
    for (int i = tid; i < n; i += nt) d0 += w[i] * u[i];
    const double n0 = rb_bcast(block_sum_dyn(d0, red), red);
    for (int pass = 0; pass < 2 && mq > 0; ++pass) {
      if (pass == 1) {
        hl_mass_apply<DIM>(Mst, w, u, n, bx, by, bz);
        __syncthreads();
      }
      for (int q = tid >> 5; q < mq; q += nt >> 5) {
        double sq = 0.0;
        for (int i = tid & 31; i < n; i += 32) sq += u[i] * V[(int64_t)q * n + i];
        sq = warp_sum(sq);
        if ((tid & 31) == 0) hcoef[q] = sq;
      }
      __syncthreads();
      for (int i = tid; i < n; i += nt) {
        double sv = w[i];
        for (int q = 0; q < mq; ++q) sv -= hcoef[q] * V[(int64_t)q * n + i];
        w[i] = sv;
      }
      __syncthreads();
      fl += fl_mass + 4LL * n * mq;
    }
    hl_mass_apply<DIM>(Mst, w, u, n, bx, by, bz);
    __syncthreads();
    double d1 = 0.0;
    for (int i = tid; i < n; i += nt) d1 += w[i] * u[i];
    const double nn = rb_bcast(block_sum_dyn(d1, red), red);
    fl += 2 * fl_mass + 4LL * n;
    if (nn > 1e-20 * n0 && nn > 0.0) {
      const double inv = 1.0 / sqrt(nn);
      for (int i = tid; i < n; i += nt) V[(int64_t)mq * n + i] = w[i] * inv;
      ++mq;
      __syncthreads();
    }
  }
  // reduced stiffness Kr = Q^T K Q
  for (int b = 0; b < mq; ++b) {
    for (int i = tid; i < n; i += nt) w[i] = V[(int64_t)b * n + i];
    __syncthreads();
    hl_mass_apply<DIM>(Kst, w, u, n, bx, by, bz);
    __syncthreads();
    for (int a = tid >> 5; a <= b; a += nt >> 5) {
      double sa = 0.0;
      for (int i = tid & 31; i < n; i += 32) sa += u[i] * V[(int64_t)a * n + i];
      sa = warp_sum(sa);
      if ((tid & 31) == 0) {
        Kr[a][b] = sa;
        Kr[b][a] = sa;
      }
    }
    __syncthreads();
  }
  fl += (long long)mq * (fl_mass + (long long)n * (mq + 1));
  // cyclic Jacobi: rounds of mm/2 disjoint rotations (mm even; a padding
  // index has a zero row and column and never rotates)
  const int mm = (mq + 1) & ~1;
  for (int t = tid; t < mm * mm; t += nt) {
    const int r = t / mm, c = t % mm;
    if (r >= mq || c >= mq) Kr[r][c] = 0.0;
    Z[r * LDZ + c] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 40 && mm >= 2; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int t = tid; t < mm * mm; t += nt) {
      const int r = t / mm, c = t % mm;
      const double v = Kr[r][c];
      tot += v * v;
      if (r != c) off += v * v;
    }
    off = rb_bcast(block_sum_dyn(off, red), red);
    tot = rb_bcast(block_sum_dyn(tot, red), red);
    if (!(off > 1e-30 * tot)) break;
    for (int round = 0; round < mm - 1; ++round) {
      if (tid < mm / 2) {
        int p, q;
        if (tid == 0) {
          p = round;
          q = mm - 1;
        } else {
          p = (round + tid) % (mm - 1);
          q = (round - tid + (mm - 1)) % (mm - 1);
        }
        if (p > q) {
          const int t2 = p;
          p = q;
          q = t2;
        }
        const double apq = Kr[p][q];
        double c = 1.0, sn = 0.0;
        if (apq != 0.0) {
          // Golub and Van Loan, symmetric Schur decomposition of the 2 x 2 block
          const double th = (Kr[q][q] - Kr[p][p]) / (2.0 * apq);
          const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
          c = 1.0 / sqrt(1.0 + t * t);
          sn = t * c;
        }
        Jp[tid] = p;
        Jq[tid] = q;
        Jc[tid] = c;
        Js[tid] = sn;
      }
      __syncthreads();
      for (int e = tid; e < (mm / 2) * mm; e += nt) {
        const int k = e / mm, j2 = e % mm;
        const int p = Jp[k], q = Jq[k];
        const double c = Jc[k], sn = Js[k];
        const double x = Kr[p][j2], y = Kr[q][j2];
        Kr[p][j2] = c * x - sn * y;
        Kr[q][j2] = sn * x + c * y;
      }
      __syncthreads();
      for (int e = tid; e < (mm / 2) * mm; e += nt) {
        const int k = e / mm, j2 = e % mm;
        const int p = Jp[k], q = Jq[k];
        const double c = Jc[k], sn = Js[k];
        const double x = Kr[j2][p], y = Kr[j2][q];
        Kr[j2][p] = c * x - sn * y;
        Kr[j2][q] = sn * x + c * y;
        const double xz = Z[j2 * LDZ + p], yz = Z[j2 * LDZ + q];
        Z[j2 * LDZ + p] = c * xz - sn * yz;
        Z[j2 * LDZ + q] = sn * xz + c * yz;
      }
      __syncthreads();
    }
  }
  // Ritz values in ascending order; those below tau are the modes
  if (tid == 0) {
    int ord[TS_RAND_MAX + 1];
    for (int k = 0; k < mq; ++k) ord[k] = k;
    for (int a = 1; a < mq; ++a)
      for (int b = a; b > 0 && Kr[ord[b]][ord[b]] < Kr[ord[b - 1]][ord[b - 1]]; --b) {
        const int t = ord[b];
        ord[b] = ord[b - 1];
        ord[b - 1] = t;
      }
    int nsel = 0;
    for (int k = 0; k < mq; ++k) nsel += (Kr[ord[k]][ord[k]] < tau) ? 1 : 0;
    const int m = min(min(max(nsel, 1), min(max_modes, TS_MAXMODES)), mq);
    for (int q = 0; q < m; ++q) {
      lockval[q] = Kr[ord[q]][ord[q]];
      Jp[q] = ord[q];
    }
    *s_nsel = nsel;
    *s_nlock = m;
  }
  __syncthreads();
  const int m = *s_nlock;
  for (int q = 0; q < m; ++q) {
    const int col = Jp[q];
    for (int i = tid; i < n; i += nt) {
      double sv = 0.0;
      for (int a = 0; a < mq; ++a) sv += Z[a * LDZ + col] * V[(int64_t)a * n + i];
      LK[(int64_t)q * n + i] = sv;
    }
  }
  fl += 2LL * n * mq * m;
  __syncthreads();
}

constexpr int EIG_THREADS = 192;
constexpr int EIG_MAXLOCK = TS_MAXMODES;

// Lanczos workspace per problem (global): V [(kmax+1) * n] + locked [EIG_MAXLOCK * n]
template <int DIM>
__global__ void __launch_bounds__(EIG_THREADS, 4) k_heat_eig(Geom g, const double* __restrict__ E,
                                                          const uint8_t* __restrict__ fm, const HeatProb* __restrict__ hp,
                                                          const int* __restrict__ order, int p0, int pend, double tau, double sigma, int max_modes,
                                                          int kmax, double* __restrict__ heat_fac,
                                                          double* __restrict__ psi, double* __restrict__ lam_out,
                                                          int* __restrict__ count_out, int* __restrict__ found_out,
                                                          double* __restrict__ ws, int64_t ws_per, int* status,
                                                          double* __restrict__ flops_out, int rand_m,
                                                          int64_t kr_off, int* __restrict__ inertia_out,
                                                          int count_only) {
  extern __shared__ double sm[];
  __shared__ int bad;
  __shared__ double al[TS_LANCZOS_MAX + 1], be[TS_LANCZOS_MAX + 2];
  __shared__ double theta[EIG_MAXLOCK + 2], resid[EIG_MAXLOCK + 2];
  __shared__ double hcoef[TS_LANCZOS_MAX + EIG_MAXLOCK + 2];
  __shared__ double lockval[EIG_MAXLOCK];
  __shared__ int s_flag, s_nlock, s_kdim;
  __shared__ double red[32];
  __shared__ double tB2[TS_LANCZOS_MAX];                       // be[i]^2
  __shared__ double sS[EIG_MAXLOCK][TS_LANCZOS_MAX];           // eigenvectors of T (Ritz coefficients)
  __shared__ double sJc[16], sJs[16];                           // Jacobi rotations of one round
  __shared__ int sJp[16], sJq[16], s_nsel;
  __shared__ double s_scale;
  // randomized basis: reduced stiffness, in dynamic shared memory past the
  // factor / Lanczos region (allocated only for that method)
  double(*sKr)[TS_RAND_MAX + 2] = reinterpret_cast<double(*)[TS_RAND_MAX + 2]>(sm + kr_off);
  if (p0 + (int)blockIdx.x >= pend) return;
  const int pi = order ? order[p0 + blockIdx.x] : p0 + (int)blockIdx.x;
  const HeatProb P = hp[pi];
  if (P.dedup_of >= 0) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int n = P.nloc;
  HeatAsm<DIM> A;
  A.g = g;
  A.E = E;
  A.fm = fm;
  A.P = P;
  // box shape: in-line extents (bx, by) and the line count
  const int bx = P.hi[0] - P.lo[0] + 1;
  const int by = (DIM == 2) ? P.nb : P.hi[1] - P.lo[1] + 1;
  const int bz = (DIM == 2) ? 1 : P.nb;
  constexpr int NB = HeatLine<DIM>::NB, NS = HeatLine<DIM>::NS;
  // stored factor of the problem (none in the count-only mode)
  double* F = count_only ? nullptr : heat_fac + P.fac_off;  // S_k^{-1} blocks of K + sigma M
  double* Cg = count_only ? nullptr : F + (int64_t)P.nb * hl_pk(P.w);    // its coupling stencils
  double* Mst = count_only ? nullptr : Cg + (int64_t)P.nb * P.w * NB;    // mass stencil of the box
  double* Kst = count_only ? nullptr : Mst + (int64_t)n * NS;            // stiffness stencil (randomized basis)
  // FP64 operations of the algorithm (counted by thread 0, one multiply-add
  // = 2): factors, mass products, line solves, Lanczos recurrences,
  // re-orthogonalisation and Ritz vectors
  const long long fl_mass = 2LL * n * NS;
  const long long fl_solve = 2LL * ((2LL * P.nb - 1) * P.w * P.w + 2LL * (P.nb - 1) * NB * P.w);
  // factor per line: symmetric sweeps over the upper triangle (w (w - 1) / 2
  // entries per pivot), T = C_k S_{k-1}^{-1} (NB w^2) and the upper triangle
  // of T C_k^T (NB w (w + 1) / 2)
  const long long fl_factor = 2LL * ((long long)P.nb * P.w * ((long long)P.w * (P.w - 1) / 2) +
                                     (P.nb - 1LL) * NB * ((long long)P.w * P.w + (long long)P.w * (P.w + 1) / 2));
  long long fl = 2 * fl_factor;  // integer: the count costs no FP64 issue slots
  // mass stencil (rows of Dirichlet nodes are zero)
  for (int e = tid; e < (count_only ? 0 : n * NS); e += nt) {
    const int i = e / NS, t = e % NS;
    const int j = hl_snbr<DIM>(i, t, bx, by, bz);
    double v = 0.0;
    if (j >= 0) {
      int a[3], b[3];
      box_coords<DIM>(P, i, a);
      box_coords<DIM>(P, j, b);
      if (fm[DIM * node_id_c(g, a) + P.c]) v = heat_entry<DIM>(g, E, a, b, 0.0, 1.0, P.lo, P.hi);
    }
    Mst[e] = v;
    if (rand_m > 0) {
      double kv = 0.0;
      if (j >= 0) {
        int a[3], b[3];
        box_coords<DIM>(P, i, a);
        box_coords<DIM>(P, j, b);
        if (fm[DIM * node_id_c(g, a) + P.c] && fm[DIM * node_id_c(g, b) + P.c])
          kv = heat_entry<DIM>(g, E, a, b, 1.0, 0.0, P.lo, P.hi);
      }
      Kst[e] = kv;
    }
  }
  // (1) inertia of K - tau M: number of eigenvalues below tau (Sylvester)
  if (tid == 0) bad = 0;
  A.kc = 1.0;
  A.mc = -tau;
  __syncthreads();
  const int neg = heat_line_factor<DIM>(A, P.w, P.nb, bx, by, sm, nullptr, nullptr, false, &bad);
  if (tid == 0 && bad) atomicOr(status, 4);  // zero pivot in the inertia count
  if (tid == 0 && inertia_out) inertia_out[pi] = neg;
  if (count_only) return;  // the density-update check wants the count alone
  // (2) factor of K + sigma M (SPD)
  __syncthreads();
  if (tid == 0) bad = 0;
  A.mc = sigma;
  __syncthreads();
  heat_line_factor<DIM>(A, P.w, P.nb, bx, by, sm, F, Cg, true, &bad);
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
  double* tmp = w + n;       // w_line
  double* sbuf = tmp + ((2 * n + P.w + 1) & ~1) - 2 * n;  // 2 staged line blocks, 16-byte aligned
  const double th_tau = 1.0 / (tau + sigma);
  if (tid == 0) {
    s_nlock = 0;
    s_nsel = neg;
  }
  __syncthreads();
  if (rand_m > 0) {
    heat_rand_basis<DIM>(g, fm, P, n, bx, by, bz, neg, nfree_loc, km, rand_m, max_modes, tau, F, Cg, Mst, Kst, V,
                         LK, u, w, tmp, sbuf, red, hcoef, sKr, &sS[0][0], sJc, sJs, sJp, sJq, &s_nsel, &s_nlock,
                         lockval, fl, fl_mass, fl_solve);
  }
  for (int restart = 0; restart < (rand_m > 0 ? 0 : 6); ++restart) {
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
      fl += fl_mass + 4LL * n * nl;
      hl_mass_apply<DIM>(Mst, w, u, n, bx, by, bz);
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
    fl += fl_mass + 2LL * n;
    hl_mass_apply<DIM>(Mst, w, u, n, bx, by, bz);
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
      fl += fl_mass + fl_solve + 6LL * n;  // M v, solve, alpha, three-term update
      hl_mass_apply<DIM>(Mst, w, u, n, bx, by, bz);  // u = M v_j
      __syncthreads();
      for (int i = tid; i < n; i += nt) w[i] = u[i];
      __syncthreads();
      heat_line_solve<DIM>(F, Cg, P.w, P.nb, bx, by, w, tmp, sbuf);  // w = (K + sigma M)^{-1} M v_j
      double a = 0.0;
      for (int i = tid; i < n; i += nt) a += u[i] * w[i];
      a = block_sum_dyn(a, red);
      if (tid == 0) al[j] = a;
      __syncthreads();
      a = al[j];
      const double bj = be[j];
      for (int i = tid; i < n; i += nt) w[i] -= a * vj[i] + ((j > 0) ? bj * vj[i - n] : 0.0);
      __syncthreads();
      // full re-orthogonalisation (classical Gram-Schmidt in the M inner
      // product) against V[0..j] and the locked vectors; a second pass only
      // when the first removed more than half of ||w||_M^2 (the criterion of
      // Daniel, Gragg, Kaufman and Stewart), in which case one more pass
      // restores orthogonality to working precision
      double wn2 = -1.0;  // ||w||_M^2 before the current pass
      for (int pass = 0; pass < 2; ++pass) {
        fl += fl_mass + 2LL * n;
        hl_mass_apply<DIM>(Mst, w, u, n, bx, by, bz);
        __syncthreads();
        double nn = 0.0;
        for (int i = tid; i < n; i += nt) nn += w[i] * u[i];
        nn = block_sum_dyn(nn, red);
        if (tid == 0) red[31] = nn;
        __syncthreads();
        nn = red[31];
        __syncthreads();
        // after the first pass: stop when the projection kept most of w
        if (pass == 1 && nn >= 0.5 * wn2) {
          wn2 = nn;
          break;
        }
        wn2 = nn;
        const int nq = j + 1 + nl;
        fl += 4LL * n * nq;
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
        if (pass == 1) wn2 = -1.0;  // norm after two passes: measured below
      }
      double b2 = wn2;
      if (b2 < 0.0) {
        fl += fl_mass + 2LL * n;
        hl_mass_apply<DIM>(Mst, w, u, n, bx, by, bz);
        __syncthreads();
        b2 = 0.0;
        for (int i = tid; i < n; i += nt) b2 += w[i] * u[i];
        b2 = block_sum_dyn(b2, red);
        if (tid == 0) red[31] = b2;
        __syncthreads();
        b2 = red[31];
        __syncthreads();
      }
      if (tid == 0) {
        const double bb = sqrt(fmax(b2, 0.0));
        be[j + 1] = bb;
        s_scale = (bb > 0.0) ? 1.0 / bb : 0.0;
      }
      __syncthreads();
      const double bn = be[j + 1];
      kdim = j + 1;
      const bool breakdown = !(bn > 1e-13 * fabs(a));
      if (!breakdown && j + 1 < km) {
        double* vn = V + (int64_t)(j + 1) * n;
        const double ib = s_scale;
        for (int i = tid; i < n; i += nt) vn[i] = w[i] * ib;
      }
      // convergence test of the top `need` Ritz pairs: eigenvalues of T by
      // bisection and their eigenvectors, one thread per Ritz pair.  It runs
      // once need + 6 steps are taken and then every 4 steps (and at a
      // breakdown or the last step): a test costs as much as several
      // Lanczos steps.
      const bool check = breakdown || (j + 1 == km) || ((kdim >= need + 6) && (((kdim - need - 6) & 3) == 0));
      if (check) {
        const int nchk = min(need, kdim);
        for (int i = tid; i < kdim; i += nt) tB2[i] = (i > 0) ? be[i] * be[i] : 0.0;
        __syncthreads();
        if (tid < nchk) {
          const double th = tri_eig_bisect(al, be, tB2, kdim, kdim - 1 - tid);
          theta[tid] = th;
          tri_eigvec(al, be, kdim, th, sS[tid]);
          resid[tid] = fabs(bn * sS[tid][kdim - 1]);
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
    // lock converged Ritz pairs below tau (or the first one, if none is);
    // the loop above ends on a test at kdim, which left theta, sS and resid
    {
      const int nchk = min(need, kdim);
      for (int q = 0; q < nchk; ++q) {
        const bool conv = resid[q] <= 1e-8 * fabs(theta[q]);
        const bool below = theta[q] > th_tau;
        const int nlk = s_nlock;
        if (conv && (below || nlk == 0) && nlk < EIG_MAXLOCK && nlk < target) {
          double* dst = LK + (int64_t)nlk * n;
          fl += 2LL * n * kdim;
          for (int i = tid; i < n; i += nt) {
            double s = 0.0;
            for (int m = 0; m < kdim; ++m) s += sS[q][m] * V[(int64_t)m * n + i];
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
    count_out[pi] = s_nsel;  // the inertia count, or the Ritz values below tau (randomized basis)
    atomicAdd(flops_out, (double)fl);
    found_out[pi] = nlock;
  }
  // order
  __shared__ int lorder[EIG_MAXLOCK];
  if (tid == 0) {
    for (int q = 0; q < nlock; ++q) lorder[q] = q;
    for (int a = 1; a < nlock; ++a)
      for (int b = a; b > 0 && lockval[lorder[b]] < lockval[lorder[b - 1]]; --b) {
        int t = lorder[b];
        lorder[b] = lorder[b - 1];
        lorder[b - 1] = t;
      }
    for (int q = 0; q < TS_MAXMODES; ++q) lam_out[(int64_t)pi * TS_MAXMODES + q] = (q < nlock) ? lockval[lorder[q]] : __longlong_as_double(0x7ff8000000000000LL);
  }
  __syncthreads();
  const int nst = min(nlock, max_modes);
  for (int q = 0; q < nst; ++q) {
    const double* src = LK + (int64_t)lorder[q] * n;
    double* dst = psi + P.vec_off + (int64_t)q * n;
    for (int i = tid; i < n; i += nt) dst[i] = src[i];
  }
}

// ---------------------------------------------------------------------------
// M_EE coarse space (Sec. "Generalized multiscale coarse finite element
// spaces for the elasticity equation", Eq. 3001), 2D: per coarse node l the
// eigenproblem of the elasticity operator on omega_l against the E-weighted
// vector mass, K_E psi = lambda M psi (natural boundary on omega_l, the
// globally Dirichlet DOFs removed), its 3 max(regions, 1) smallest pairs,
// regions = face-connected sets of elements with E_e >= sqrt(E0 Emin).
// The same block LU over node lines as the heat problems, with the two
// components of a node interleaved in a line (lines of W = 2 bx unknowns;
// a DOF row couples to 3 nodes x 2 components of a neighbouring line), and
// the same shift-invert Lanczos.
// ---------------------------------------------------------------------------
static __constant__ double c_KE_el[TS_KE_SLOTS * TS_KE_SIZE];

void upload_KE_coarse(int slot, const std::vector<double>& KE) {
  TS_CUDA(cudaMemcpyToSymbol(c_KE_el, KE.data(), KE.size() * sizeof(double), sizeof(double) * TS_KE_SIZE * slot,
                             cudaMemcpyHostToDevice));
}

constexpr int EL_NBD = 6;  // couplings of a DOF row to a neighbouring line: 3 nodes x 2 components

// DOF q of the neighbouring line seen from DOF p of this line through slot t
// (node offset t / 2 - 1, component t % 2), or -1 outside the box
__device__ __forceinline__ int el_nbr(int p, int t, int bx) {
  const int x = p / 2 + t / 2 - 1;
  return (x >= 0 && x < bx) ? 2 * x + (t & 1) : -1;
}

// stored doubles per problem: S_k^{-1} blocks (W = 2 bx), coupling stencils,
// scalar mass stencil (9 per node), even
__host__ __device__ inline int64_t elas_line_size(int bx, int nb, int n) {
  const int W = 2 * bx;
  const int64_t s = (int64_t)nb * hl_pk(W) + (int64_t)nb * W * EL_NBD + 9LL * n;
  return (s + 1) & ~(int64_t)1;
}

struct ElasAsm {
  Geom g;
  const double* E;
  const uint8_t* fm;
  const double* KE;
  int lo[3], hi[3];
  int bx;
  double kc, mc;
  // entry between DOF p of line kr and DOF q of line kc_ (p = 2 x + component)
  __device__ double entry(int kr, int p, int kc_, int q) const {
    const int a[3] = {lo[0] + p / 2, lo[1] + kr, 0}, b[3] = {lo[0] + q / 2, lo[1] + kc_, 0};
    const int ca = p & 1, cb = q & 1;
    const bool fa = fm[2 * ((int64_t)a[1] * (g.nx + 1) + a[0]) + ca] != 0;
    const bool fb = fm[2 * ((int64_t)b[1] * (g.nx + 1) + b[0]) + cb] != 0;
    if (!fa || !fb) return (kr == kc_ && p == q) ? 1.0 : 0.0;
    double v = kc * elas_entry<2>(g, E, KE, a, ca, b, cb, lo, hi);
    if (ca == cb && mc != 0.0) v += mc * heat_entry<2>(g, E, a, b, 0.0, 1.0, lo, hi);
    return v;
  }
};

// Block LU factor of A over lines of W DOFs (heat_line_factor with DOF rows)
__device__ int el_line_factor(const ElasAsm& A, int W, int nb, double* smem, double* Minv, double* Cout, bool spd,
                              int* bad) {
  const int tid = threadIdx.x, nt = blockDim.x, bx = W / 2;
  double* S = smem;
  double* Mp = S + W * W;
  double* T = Mp + W * W;
  double* Cs = T + W * W;
  double* rowj = Cs + W * EL_NBD;
  double* colj = rowj + W;
  unsigned* tab = reinterpret_cast<unsigned*>(colj + W);
  const int nu = hl_nup(W);
  for (int i = 0; i < W; ++i) {
    const int off = i * W - i * (i - 1) / 2;
    for (int c = i + tid; c < W; c += nt) tab[off + c - i] = ((unsigned)i << 16) | (unsigned)c;
  }
  int neg = 0;
  for (int k = 0; k < nb; ++k) {
    __syncthreads();
    for (int e = tid; e < nu; e += nt) {
      const int i = (int)(tab[e] >> 16), j = (int)(tab[e] & 0xffffu);
      S[i * W + j] = A.entry(k, i, k, j);
    }
    if (k > 0) {
      for (int e = tid; e < W * EL_NBD; e += nt) {
        const int i = e / EL_NBD, t = e % EL_NBD;
        const int q = el_nbr(i, t, bx);
        Cs[e] = (q >= 0) ? A.entry(k, i, k - 1, q) : 0.0;
      }
      __syncthreads();
      if (Cout)
        for (int e = tid; e < W * EL_NBD; e += nt) Cout[(int64_t)k * W * EL_NBD + e] = Cs[e];
      for (int e = tid; e < W * W; e += nt) {
        const int i = e / W, c = e % W;
        double s = 0.0;
#pragma unroll
        for (int t = 0; t < EL_NBD; ++t) {
          const int q = el_nbr(i, t, bx);
          if (q >= 0) s = fma(Cs[i * EL_NBD + t], Mp[q * W + c], s);
        }
        T[e] = s;
      }
      __syncthreads();
      for (int e = tid; e < nu; e += nt) {
        const int i = (int)(tab[e] >> 16), j = (int)(tab[e] & 0xffffu);
        double s = 0.0;
#pragma unroll
        for (int t = 0; t < EL_NBD; ++t) {
          const int q = el_nbr(j, t, bx);
          if (q >= 0) s = fma(T[i * W + q], Cs[j * EL_NBD + t], s);
        }
        S[i * W + j] -= s;
      }
    }
    neg += hl_gj_inverse(S, W, rowj, colj, tab, spd, bad);
    if (Minv)
      for (int e = tid; e < nu; e += nt) {
        const int i = (int)(tab[e] >> 16), c = (int)(tab[e] & 0xffffu);
        Minv[(int64_t)k * hl_pk(W) + e] = S[i * W + c];
      }
    double* t = S;
    S = Mp;
    Mp = t;
  }
  __syncthreads();
  return neg;
}

// shared memory (doubles) of the factor
__host__ inline size_t elas_factor_smem(int W) {
  return ((size_t)3 * W * W + (size_t)W * EL_NBD + 2 * (size_t)W + (size_t)(hl_nup(W) + 1) / 2) * sizeof(double);
}

// (K_E + s M) x = v in place with the stored factor (heat_line_solve with DOF rows)
__device__ void el_line_solve(const double* Minv, const double* C, int W, int nb, double* v, double* y, double* buf) {
  const int tid = threadIdx.x, nt = blockDim.x, bx = W / 2;
  const int64_t ws = hl_pk(W);
  double* b[2] = {buf, buf + ws};
  __syncthreads();
  hl_stage(b[0], Minv, W);
  for (int k = 0; k < nb; ++k) {
    double* vk = v + (int64_t)k * W;
    for (int i = tid; i < W; i += nt) {
      double s = vk[i];
      if (k > 0) {
        const double* ck = C + ((int64_t)k * W + i) * EL_NBD;
#pragma unroll
        for (int t = 0; t < EL_NBD; ++t) {
          const int q = el_nbr(i, t, bx);
          if (q >= 0) s = fma(-ck[t], vk[q - W], s);
        }
      }
      y[i] = s;
    }
    if (k + 1 < nb) {
      hl_stage(b[(k + 1) & 1], Minv + (k + 1) * ws, W);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
    hl_gemv(b[k & 1], y, vk, W, false);
    __syncthreads();
  }
  if (nb >= 3) hl_stage(b[(nb - 3) & 1], Minv + (nb - 3) * ws, W);
  for (int k = nb - 2; k >= 0; --k) {
    double* vk = v + (int64_t)k * W;
    const double* ck = C + (int64_t)(k + 1) * W * EL_NBD;
    for (int i = tid; i < W; i += nt) {
      // (C_{k+1}^T x)_i: row 2 q + b of line k+1 (node q = i / 2 + t - 1) sees
      // DOF i (node offset 1 - t, component i % 2) in slot 2 (2 - t) + i % 2
      double s = 0.0;
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        const int qn = i / 2 + t - 1;
        if (qn < 0 || qn >= bx) continue;
#pragma unroll
        for (int bb = 0; bb < 2; ++bb) {
          const int row = 2 * qn + bb;
          s = fma(ck[row * EL_NBD + 2 * (2 - t) + (i & 1)], vk[W + row], s);
        }
      }
      y[i] = s;
    }
    if (k >= 1)
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    else
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    hl_gemv(b[k & 1], y, vk, W, true);
    __syncthreads();
    if (k >= 2) hl_stage(b[k & 1], Minv + (k - 2) * ws, W);
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// y = M x for the vector mass (scalar stencil Mst per node, both components;
// rows of Dirichlet DOFs zero); DOF 2 i + c
__device__ __forceinline__ void el_mass_apply(const double* Mst, const uint8_t* dfree, const double* x, double* y,
                                              int n, int bx, int by) {
  for (int e = threadIdx.x; e < 2 * n; e += blockDim.x) {
    const int i = e >> 1, c = e & 1;
    double s = 0.0;
    if (dfree[e]) {
      const double* m = Mst + (int64_t)i * 9;
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        const int j = hl_snbr<2>(i, t, bx, by, 1);
        if (j >= 0) s = fma(m[t], x[2 * j + c], s);
      }
    }
    y[e] = s;
  }
}

constexpr int EL_THREADS = 256;
constexpr int EL_MAXLOCK = TS_EL_MAXMODES;

// one CTA per problem (coarse node); workspace per problem in ws:
// V [(kmax + 1) * 2n] + locked [EL_MAXLOCK * 2n]
__global__ void __launch_bounds__(EL_THREADS, 1) k_elas_eig(Geom g, const double* __restrict__ E,
                                                         const uint8_t* __restrict__ fm, const HeatProb* __restrict__ hp,
                                                         int p0, int pend, double sigma, double stiff, int kmax,
                                                         double* __restrict__ fac, double* __restrict__ psi,
                                                         double* __restrict__ lam_out, int* __restrict__ count_out,
                                                         int* __restrict__ found_out, double* __restrict__ ws,
                                                         int64_t ws_per, int* status, double* __restrict__ flops_out) {
  extern __shared__ double sm[];
  __shared__ int bad, s_flag, s_nlock, s_kdim, s_regions;
  __shared__ double al[TS_LANCZOS_MAX + 1], be[TS_LANCZOS_MAX + 2];
  __shared__ double theta[EL_MAXLOCK + 2], resid[EL_MAXLOCK + 2];
  __shared__ double hcoef[TS_LANCZOS_MAX + EL_MAXLOCK + 2];
  __shared__ double lockval[EL_MAXLOCK];
  __shared__ double red[32];
  __shared__ double tB2[TS_LANCZOS_MAX];
  __shared__ double sS[EL_MAXLOCK][TS_LANCZOS_MAX];
  __shared__ double s_scale;
  __shared__ int lorder[EL_MAXLOCK];
  __shared__ int parent[1024];
  __shared__ uint8_t dfree[2 * 1100];
  if (p0 + (int)blockIdx.x >= pend) return;
  const int pi = p0 + blockIdx.x;
  const HeatProb P = hp[pi];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int bx = P.hi[0] - P.lo[0] + 1, by = P.hi[1] - P.lo[1] + 1;
  const int n = P.nloc, n2 = 2 * n, W = 2 * bx;
  ElasAsm A;
  A.g = g;
  A.E = E;
  A.fm = fm;
  A.KE = c_KE_el + g.ke * TS_KE_SIZE;
  for (int d = 0; d < 3; ++d) {
    A.lo[d] = P.lo[d];
    A.hi[d] = P.hi[d];
  }
  A.bx = bx;
  double* F = fac + P.fac_off;
  double* Cg = F + (int64_t)by * hl_pk(W);
  double* Mst = Cg + (int64_t)by * W * EL_NBD;
  // free DOFs of the box and the scalar E-weighted mass stencil
  for (int e = tid; e < n2; e += nt) {
    const int i = e >> 1;
    dfree[e] = fm[2 * ((int64_t)(P.lo[1] + i / bx) * (g.nx + 1) + P.lo[0] + i % bx) + (e & 1)];
  }
  for (int e = tid; e < n * 9; e += nt) {
    const int i = e / 9, t = e % 9;
    const int j = hl_snbr<2>(i, t, bx, by, 1);
    double v = 0.0;
    if (j >= 0) {
      const int a[3] = {P.lo[0] + i % bx, P.lo[1] + i / bx, 0}, b[3] = {P.lo[0] + j % bx, P.lo[1] + j / bx, 0};
      v = heat_entry<2>(g, E, a, b, 0.0, 1.0, P.lo, P.hi);
    }
    Mst[e] = v;
  }
  // stiff regions: face-connected components of the elements with E_e >= stiff
  {
    const int ex = bx - 1, ey = by - 1, ne = ex * ey;
    for (int e = tid; e < ne; e += nt) {
      const double Ee = E[(int64_t)(P.lo[1] + e / ex) * g.nx + P.lo[0] + e % ex];
      parent[e] = (Ee >= stiff) ? e : -1;
    }
    __syncthreads();
    if (tid == 0) {
      auto find = [&](int x) {
        while (parent[x] != x) {
          parent[x] = parent[parent[x]];
          x = parent[x];
        }
        return x;
      };
      for (int e = 0; e < ne; ++e) {
        if (parent[e] < 0) continue;
        const int x = e % ex, y = e / ex;
        if (x > 0 && parent[e - 1] >= 0) {
          const int ra = find(e), rb = find(e - 1);
          if (ra != rb) parent[max(ra, rb)] = min(ra, rb);
        }
        if (y > 0 && parent[e - ex] >= 0) {
          const int ra = find(e), rb = find(e - ex);
          if (ra != rb) parent[max(ra, rb)] = min(ra, rb);
        }
      }
      int r = 0;
      for (int e = 0; e < ne; ++e)
        if (parent[e] >= 0 && find(e) == e) ++r;
      s_regions = r;
    }
    __syncthreads();
  }
  const long long fl_mass = 2LL * n2 * 9;
  const long long fl_solve = 2LL * ((2LL * by - 1) * W * W + 2LL * (by - 1) * EL_NBD * W);
  const long long fl_factor = 2LL * ((long long)by * W * ((long long)W * (W - 1) / 2) +
                                     (by - 1LL) * EL_NBD * ((long long)W * W + (long long)W * (W + 1) / 2));
  long long fl = fl_factor;
  // factor of K_E + sigma M (SPD)
  if (tid == 0) bad = 0;
  A.kc = 1.0;
  A.mc = sigma;
  __syncthreads();
  el_line_factor(A, W, by, sm, F, Cg, true, &bad);
  if (tid == 0 && bad) atomicOr(status, 8);
  __syncthreads();
  int nfree = 0;
  {
    int cnt = 0;
    for (int e = tid; e < n2; e += nt) cnt += dfree[e] ? 1 : 0;
    const double c = block_sum_dyn((double)cnt, red);
    if (tid == 0) s_kdim = (int)c;
    __syncthreads();
    nfree = s_kdim;
    __syncthreads();
  }
  const int want = 3 * max(s_regions, 1);
  const int target = min(min(want, EL_MAXLOCK), nfree);
  const int km = min(kmax, nfree);
  double* V = ws + (int64_t)blockIdx.x * ws_per;      // (km + 1) x n2
  double* LK = V + (int64_t)(kmax + 1) * n2;          // EL_MAXLOCK x n2
  double* u = sm;
  double* w = u + n2;
  double* tmp = w + n2;
  double* sbuf = tmp + ((2 * n2 + W + 1) & ~1) - 2 * n2;
  if (tid == 0) s_nlock = 0;
  __syncthreads();
  for (int restart = 0; restart < 8; ++restart) {
    const int need = target - s_nlock;
    if (need <= 0) break;
    for (int e = tid; e < n2; e += nt) w[e] = dfree[e] ? (1.0 + hash01(pi, e, restart + 17)) : 0.0;
    __syncthreads();
    const int nl = s_nlock;
    for (int pass = 0; pass < 2 && nl > 0; ++pass) {
      fl += fl_mass + 4LL * n2 * nl;
      el_mass_apply(Mst, dfree, w, u, n, bx, by);
      __syncthreads();
      for (int q = tid >> 5; q < nl; q += nt >> 5) {
        double sq = 0.0;
        for (int i = tid & 31; i < n2; i += 32) sq += u[i] * LK[(int64_t)q * n2 + i];
        sq = warp_sum(sq);
        if ((tid & 31) == 0) hcoef[q] = sq;
      }
      __syncthreads();
      for (int i = tid; i < n2; i += nt) {
        double sv = w[i];
        for (int q = 0; q < nl; ++q) sv -= hcoef[q] * LK[(int64_t)q * n2 + i];
        w[i] = sv;
      }
      __syncthreads();
    }
    fl += fl_mass + 2LL * n2;
    el_mass_apply(Mst, dfree, w, u, n, bx, by);
    __syncthreads();
    double nn = 0.0;
    for (int i = tid; i < n2; i += nt) nn += w[i] * u[i];
    nn = block_sum_dyn(nn, red);
    if (tid == 0) red[31] = nn;
    __syncthreads();
    nn = red[31];
    __syncthreads();
    const double inv = 1.0 / sqrt(nn);
    for (int i = tid; i < n2; i += nt) V[i] = w[i] * inv;
    if (tid == 0) {
      be[0] = 0.0;
      s_flag = 0;
    }
    __syncthreads();
    int kdim = 0;
    for (int j = 0; j < km; ++j) {
      const double* vj = V + (int64_t)j * n2;
      for (int i = tid; i < n2; i += nt) w[i] = vj[i];
      __syncthreads();
      fl += fl_mass + fl_solve + 6LL * n2;
      el_mass_apply(Mst, dfree, w, u, n, bx, by);  // u = M v_j
      __syncthreads();
      for (int i = tid; i < n2; i += nt) w[i] = u[i];
      __syncthreads();
      el_line_solve(F, Cg, W, by, w, tmp, sbuf);  // w = (K_E + sigma M)^{-1} M v_j
      double a = 0.0;
      for (int i = tid; i < n2; i += nt) a += u[i] * w[i];
      a = block_sum_dyn(a, red);
      if (tid == 0) al[j] = a;
      __syncthreads();
      a = al[j];
      const double bj = be[j];
      for (int i = tid; i < n2; i += nt) w[i] -= a * vj[i] + ((j > 0) ? bj * vj[i - n2] : 0.0);
      __syncthreads();
      double wn2 = -1.0;
      for (int pass = 0; pass < 2; ++pass) {
        fl += fl_mass + 2LL * n2;
        el_mass_apply(Mst, dfree, w, u, n, bx, by);
        __syncthreads();
        double q2 = 0.0;
        for (int i = tid; i < n2; i += nt) q2 += w[i] * u[i];
        q2 = block_sum_dyn(q2, red);
        if (tid == 0) red[31] = q2;
        __syncthreads();
        q2 = red[31];
        __syncthreads();
        if (pass == 1 && q2 >= 0.5 * wn2) {
          wn2 = q2;
          break;
        }
        wn2 = q2;
        const int nq = j + 1 + nl;
        fl += 4LL * n2 * nq;
        for (int q = tid >> 5; q < nq; q += nt >> 5) {
          const double* vq = (q <= j) ? V + (int64_t)q * n2 : LK + (int64_t)(q - j - 1) * n2;
          double sq = 0.0;
          for (int i = tid & 31; i < n2; i += 32) sq += u[i] * vq[i];
          sq = warp_sum(sq);
          if ((tid & 31) == 0) hcoef[q] = sq;
        }
        __syncthreads();
        for (int i = tid; i < n2; i += nt) {
          double sv = w[i];
          for (int q = 0; q <= j; ++q) sv -= hcoef[q] * V[(int64_t)q * n2 + i];
          for (int q = 0; q < nl; ++q) sv -= hcoef[j + 1 + q] * LK[(int64_t)q * n2 + i];
          w[i] = sv;
        }
        __syncthreads();
        if (pass == 1) wn2 = -1.0;
      }
      double b2 = wn2;
      if (b2 < 0.0) {
        fl += fl_mass + 2LL * n2;
        el_mass_apply(Mst, dfree, w, u, n, bx, by);
        __syncthreads();
        b2 = 0.0;
        for (int i = tid; i < n2; i += nt) b2 += w[i] * u[i];
        b2 = block_sum_dyn(b2, red);
        if (tid == 0) red[31] = b2;
        __syncthreads();
        b2 = red[31];
        __syncthreads();
      }
      if (tid == 0) {
        const double bb = sqrt(fmax(b2, 0.0));
        be[j + 1] = bb;
        s_scale = (bb > 0.0) ? 1.0 / bb : 0.0;
      }
      __syncthreads();
      const double bn = be[j + 1];
      kdim = j + 1;
      const bool breakdown = !(bn > 1e-13 * fabs(a));
      if (!breakdown && j + 1 < km) {
        double* vn = V + (int64_t)(j + 1) * n2;
        const double ib = s_scale;
        for (int i = tid; i < n2; i += nt) vn[i] = w[i] * ib;
      }
      const bool check = breakdown || (j + 1 == km) || ((kdim >= need + 6) && (((kdim - need - 6) & 3) == 0));
      if (check) {
        const int nchk = min(need, kdim);
        for (int i = tid; i < kdim; i += nt) tB2[i] = (i > 0) ? be[i] * be[i] : 0.0;
        __syncthreads();
        if (tid < nchk) {
          const double th = tri_eig_bisect(al, be, tB2, kdim, kdim - 1 - tid);
          theta[tid] = th;
          tri_eigvec(al, be, kdim, th, sS[tid]);
          resid[tid] = fabs(bn * sS[tid][kdim - 1]);
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
    // lock the converged Ritz pairs (the largest theta = the smallest eigenvalues)
    {
      const int nchk = min(need, kdim);
      for (int q = 0; q < nchk; ++q) {
        const bool conv = resid[q] <= 1e-8 * fabs(theta[q]);
        const int nlk = s_nlock;
        if (conv && nlk < target) {
          double* dst = LK + (int64_t)nlk * n2;
          fl += 2LL * n2 * kdim;
          for (int i = tid; i < n2; i += nt) {
            double sv = 0.0;
            for (int m = 0; m < kdim; ++m) sv += sS[q][m] * V[(int64_t)m * n2 + i];
            dst[i] = sv;
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
    if (s_nlock == 0) break;
  }
  const int nlock = s_nlock;
  __syncthreads();
  if (tid == 0) {
    count_out[pi] = want;
    atomicAdd(flops_out, (double)fl);
    found_out[pi] = nlock;
    for (int q = 0; q < nlock; ++q) lorder[q] = q;
    for (int a = 1; a < nlock; ++a)
      for (int b = a; b > 0 && lockval[lorder[b]] < lockval[lorder[b - 1]]; --b) {
        const int t = lorder[b];
        lorder[b] = lorder[b - 1];
        lorder[b - 1] = t;
      }
    for (int q = 0; q < TS_EL_MAXMODES; ++q)
      lam_out[(int64_t)pi * TS_EL_MAXMODES + q] = (q < nlock) ? lockval[lorder[q]] : __longlong_as_double(0x7ff8000000000000LL);
  }
  __syncthreads();
  for (int q = 0; q < nlock; ++q) {
    const double* src = LK + (int64_t)lorder[q] * n2;
    double* dst = psi + P.vec_off + (int64_t)q * n2;
    for (int i = tid; i < n2; i += nt) dst[i] = src[i];
  }
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
  // coarse_method 2: the elasticity eigenproblems of M_EE, one per coarse node
  const bool elastic = h->opt.coarse_method == 2;
  if (elastic && dim != 2) throw TsError(TS_ERR_INVALID, "the M_EE coarse space (coarse_method 2) is built for 2D only");
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
    if (elastic) {
      // a coarse node Dirichlet in every component gets no basis
      for (int c = 0; c < dim; ++c) {
        N.nmodes[c] = 0;
        N.prob[c] = -1;
        if (fm_h[dim * ynode + c]) any_free = true;
      }
      N.nrot = 0;
      if (any_free) {
        if (nloc > 1100 || P.w > 33) throw TsError(TS_ERR_INVALID, "coarse neighbourhood too large for M_EE");
        P.c = -1;
        P.dedup_of = -1;
        P.fac_off = fac_off;
        fac_off += elas_line_size(P.w, P.nb, nloc);
        P.vec_off = vec_off;
        vec_off += (int64_t)TS_EL_MAXMODES * 2 * nloc;
        max_w = std::max(max_w, P.w);
        max_n = std::max(max_n, nloc);
        N.prob[0] = (int)hp.size();
        hp.push_back(P);
      }
      continue;
    }
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
        fac_off += heat_line_size(P.w, P.nb, nloc, dim);
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
  h->lam_stride = elastic ? TS_EL_MAXMODES : TS_MAXMODES;
  h->hp_lambda = dalloc<double>(h, (size_t)std::max(nprob, 1) * h->lam_stride);
  h->heat_fac = salloc<double>(h, fac_off);
  h->psi = salloc<double>(h, vec_off);
  TS_CUDA(cudaMemsetAsync(h->hp_count, 0, sizeof(int) * std::max(nprob, 1), st));
  TS_CUDA(cudaMemsetAsync(h->hp_found, 0, sizeof(int) * std::max(nprob, 1), st));
  const int kmax = std::min(TS_LANCZOS_MAX - 1, 80);
  // factor: heat_factor_smem; Lanczos: u, w (n each), y (w), two staged line blocks
  size_t smem = elastic ? std::max(elas_factor_smem(2 * max_w),
                                    (size_t)(4 * max_n + 2 * max_w + 2 + 2 * hl_pk(2 * max_w)) * sizeof(double)) + 64
                         : std::max(heat_factor_smem(max_w, dim),
                                    (size_t)(2 * max_n + max_w + 2 + 2 * hl_pk(max_w)) * sizeof(double)) + 64;
  const int rand_m = (h->opt.coarse_method == 1) ? h->opt.rand_snapshots : 0;
  const int64_t kr_off = (int64_t)(smem / sizeof(double));
  if (rand_m > 0) smem += sizeof(double) * (TS_RAND_MAX + 1) * (TS_RAND_MAX + 2);
  if (smem > 227 * 1024) throw TsError(TS_ERR_INVALID, "coarse neighbourhood too large for shared memory");
  // FP64 operation count of the eigenproblems, and CUDA events around their
  // launches on the work stream (reported by ts_time_kernel("heat_eig"))
  double* flops = salloc<double>(h, 1);
  TS_CUDA(cudaMemsetAsync(flops, 0, sizeof(double), st));
  cudaEvent_t ev[2] = {nullptr, nullptr};
  TS_CUDA(cudaEventCreate(&ev[0]));
  TS_CUDA(cudaEventCreate(&ev[1]));
  struct EvGuard {
    cudaEvent_t* e;
    ~EvGuard() {
      cudaEventDestroy(e[0]);
      cudaEventDestroy(e[1]);
    }
  } evg{ev};
  // the distinct problems (the others copy an earlier component's result),
  // largest first: the block scheduler hands consecutive CTAs to different
  // SMs, so every SM gets one problem of each size class and the SMs finish
  // together.  Cost proxy: line count x line width^2 (factor and solves).
  std::vector<int> run_order;
  for (int i = 0; i < nprob; ++i)
    if (hp[i].dedup_of < 0 && !elastic) run_order.push_back(i);
  std::stable_sort(run_order.begin(), run_order.end(), [&](int a, int b) {
    return (int64_t)hp[a].nb * hp[a].w * hp[a].w > (int64_t)hp[b].nb * hp[b].w * hp[b].w;
  });
  const int nrun = (int)run_order.size();
  const int* d_order = supload(h, run_order);
  // Lanczos workspace, processed in batches of problems
  const int batch = std::max(1, std::min(nrun, 4096));
  const int64_t ws_per = (int64_t)(kmax + 1 + TS_MAXMODES) * max_n;
  double* ws = salloc<double>(h, (size_t)batch * ws_per);
  int* inertia = salloc<int>(h, std::max(nprob, 1));
  TS_CUDA(cudaMemsetAsync(inertia, 0, sizeof(int) * std::max(nprob, 1), st));
  h->heat_smem = smem;
  TS_CUDA(cudaEventRecord(ev[0], st));
  if (elastic && nprob > 0) {
    // M_EE: every problem, in batches (Lanczos workspace of 2 n per vector)
    const size_t lim = ts_allow_dynamic_smem(k_elas_eig, h->ctx->device);
    if (smem > lim) throw TsError(TS_ERR_INVALID, "coarse neighbourhood too large for M_EE in shared memory");
    const int eb = std::min(nprob, 1024);
    const int64_t ews = (int64_t)(kmax + 1 + TS_EL_MAXMODES) * 2 * max_n;
    double* ew = salloc<double>(h, (size_t)eb * ews);
    const double stiff = std::sqrt(h->E0 * h->Emin);
    for (int p0 = 0; p0 < nprob; p0 += eb) {
      const int cnt = std::min(eb, nprob - p0);
      tsl(h), k_elas_eig<<<cnt, EL_THREADS, smem, st>>>(g, h->E, h->freemask, h->hp, p0, p0 + cnt, sigma, stiff, kmax,
                                                        h->heat_fac, h->psi, h->hp_lambda, h->hp_count, h->hp_found, ew,
                                                        ews, h->dstatus, flops);
      TS_CUDA(cudaGetLastError());
    }
  }
  if (nrun > 0) {
    const size_t lim = (dim == 2) ? ts_allow_dynamic_smem(k_heat_eig<2>, h->ctx->device)
                                  : ts_allow_dynamic_smem(k_heat_eig<3>, h->ctx->device);
    if (smem > lim) throw TsError(TS_ERR_INVALID, "coarse neighbourhood too large for shared memory");
    // four CTAs of 192 threads per SM need the largest shared-memory carveout
    TS_CUDA(cudaFuncSetAttribute(dim == 2 ? (const void*)k_heat_eig<2> : (const void*)k_heat_eig<3>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    for (int p0 = 0; p0 < nrun; p0 += batch) {
      int cnt = std::min(batch, nrun - p0);
      if (dim == 2)
        tsl(h), k_heat_eig<2><<<cnt, EIG_THREADS, smem, st>>>(g, h->E, h->freemask, h->hp, d_order, p0, p0 + cnt, tau, sigma,
                                                      h->opt.max_modes, kmax, h->heat_fac, h->psi, h->hp_lambda,
                                                      h->hp_count, h->hp_found, ws, ws_per, h->dstatus, flops,
                                                      rand_m, kr_off, inertia, 0);
      else
        tsl(h), k_heat_eig<3><<<cnt, EIG_THREADS, smem, st>>>(g, h->E, h->freemask, h->hp, d_order, p0, p0 + cnt, tau, sigma,
                                                      h->opt.max_modes, kmax, h->heat_fac, h->psi, h->hp_lambda,
                                                      h->hp_count, h->hp_found, ws, ws_per, h->dstatus, flops,
                                                      rand_m, kr_off, inertia, 0);
      TS_CUDA(cudaGetLastError());
    }
  }
  TS_CUDA(cudaEventRecord(ev[1], st));
  // read back counts to number the coarse DOFs
  std::vector<int> count(nprob), found(nprob);
  h->hp_inertia_h.assign(nprob, 0);
  if (nprob) {
    TS_CUDA(cudaMemcpyAsync(h->hp_inertia_h.data(), inertia, sizeof(int) * nprob, cudaMemcpyDeviceToHost, st));
    TS_CUDA(cudaMemcpyAsync(count.data(), h->hp_count, sizeof(int) * nprob, cudaMemcpyDeviceToHost, st));
    TS_CUDA(cudaMemcpyAsync(found.data(), h->hp_found, sizeof(int) * nprob, cudaMemcpyDeviceToHost, st));
  }
  double fl_h = 0.0;
  TS_CUDA(cudaMemcpyAsync(&fl_h, flops, sizeof(double), cudaMemcpyDeviceToHost, st));
  TS_CUDA(cudaStreamSynchronize(st));
  float heat_ms = 0.0f;
  TS_CUDA(cudaEventElapsedTime(&heat_ms, ev[0], ev[1]));
  h->heat_ms = heat_ms;
  h->heat_flops = fl_h;
  h->cap_hits = 0;
  h->eig_unconv = 0;
  // Coarse DOFs are numbered line by line along the axis with the most
  // coarse nodes (the coarse matrix is then block-tridiagonal by lines, and
  // each line holds the fewest nodes); within a line, x-fastest.
  int A = 0;
  for (int a = 1; a < dim; ++a)
    if (g.ncn[a] >= g.ncn[A]) A = a;
  h->line_axis = A;
  h->n_lines = g.ncn[A];
  std::vector<int> order;
  order.reserve(ncn);
  for (int k = 0; k < g.ncn[A]; ++k)
    for (int l = 0; l < ncn; ++l)
      if (cn[l].idx[A] == k) order.push_back(l);
  std::vector<int> cdof_node, cdof_kind, cdof_mode;
  h->line_off_h.assign(g.ncn[A] + 1, 0);
  int nc = 0;
  int64_t boff = 0, woff = 0;
  int max_ndof = 0;
  for (int l : order) {
    CoarseNodeInfo& N = cn[l];
    N.first_dof = nc;
    N.nvec = 0;
    if (elastic && N.prob[0] >= 0) {
      // M_EE: 3 max(regions, 1) modes (count), at most TS_EL_MAXMODES
      const int pi = N.prob[0];
      const int want = std::min(count[pi], TS_EL_MAXMODES);
      if (count[pi] > TS_EL_MAXMODES) h->cap_hits++;
      const int got = std::min(found[pi], want);
      if (got < want) h->eig_unconv++;
      N.nvec = got;
      for (int m = 0; m < got; ++m) {
        cdof_node.push_back(l);
        cdof_kind.push_back(TS_VEC_KIND);
        cdof_mode.push_back(m);
      }
      nc += got;
    }
    for (int c = 0; c < dim && !elastic; ++c) {
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
    max_ndof = std::max(max_ndof, N.ndof);
    // closed omega box of the node and its basis block offset
    N.nbox = 1;
    for (int d = 0; d < 3; ++d) {
      N.lo[d] = (d < dim) ? std::max(0, (N.idx[d] - 1) * g.H[d]) : 0;
      N.hi[d] = (d < dim) ? std::min(g.n[d], (N.idx[d] + 1) * g.H[d]) : 0;
      N.nbox *= N.hi[d] - N.lo[d] + 1;
    }
    N.boff = boff;
    boff += (int64_t)N.nbox * dim * N.ndof;
    N.nh = 2 * N.nvec;
    for (int c = 0; c < dim; ++c) N.nh += N.nmodes[c];
    N.woff = woff;
    woff += (int64_t)N.nh * ((N.nbox + 3) & ~3);
    h->line_off_h[N.idx[A] + 1] = nc;
  }
  for (int k = 1; k <= g.ncn[A]; ++k) h->line_off_h[k] = std::max(h->line_off_h[k], h->line_off_h[k - 1]);
  h->max_cdof = max_ndof;
  h->B_len = boff;
  h->W_len = woff;
  // keep per-problem counts for introspection (counts of deduplicated problems)
  for (int pi = 0; pi < nprob; ++pi) {
    int src = hp[pi].dedup_of >= 0 ? hp[pi].dedup_of : pi;
    count[pi] = count[src];
    found[pi] = found[src];
  }
  TS_CUDA(cudaMemcpyAsync(h->hp_count, count.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice, st));
  TS_CUDA(cudaMemcpyAsync(h->hp_found, found.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice, st));
  TS_CUDA(cudaStreamSynchronize(st));
  h->cn_h = cn;
  h->cn = dupload(h, cn);
  h->nc = nc;
  if (nc == 0) return;
  h->cdof_node = dupload(h, cdof_node);
  h->cdof_kind = dupload(h, cdof_kind);
  h->cdof_mode = dupload(h, cdof_mode);
  build_coarse_basis(h);   // Phi blocks and K_0 (ts_cbasis.cu)
  // factor of K_0 (ts_cfactor.cu), timed with events on the work stream and
  // its GEMM FLOPs counted on the device (read back when the setup ends)
  if (!h->cfac_ev[0]) {
    TS_CUDA(cudaEventCreate(&h->cfac_ev[0]));
    TS_CUDA(cudaEventCreate(&h->cfac_ev[1]));
  }
  h->cfac_cnt = dalloc<unsigned long long>(h, 1);
  TS_CUDA(cudaMemsetAsync(h->cfac_cnt, 0, sizeof(unsigned long long), h->ctx->stream));
  h->cfac_flops = 0.0;
  TS_CUDA(cudaEventRecord(h->cfac_ev[0], h->ctx->stream));
  build_coarse_factor(h);
  TS_CUDA(cudaEventRecord(h->cfac_ev[1], h->ctx->stream));
}

// Would the threshold change the coarse dimension for the moduli E (device,
// [n_el])?  The inertia of K - tau M of every heat eigenproblem (the first
// step of k_heat_eig alone, with E in place of the design's moduli), each
// count taken as the build takes it (at least one, at most max_modes), summed
// over the problems, against the same sum for the last build.
bool heat_counts_changed(ts_handle h, const double* E) {
  if (h->opt.coarse_method == 2) return false;  // M_EE: no threshold count (the iteration trigger applies)
  const int nprob = h->n_hprob;
  if (nprob == 0 || !h->hp || (int)h->hp_inertia_h.size() != nprob) return false;
  const Geom& g = h->g;
  cudaStream_t st = h->ctx->stream;
  const double H = (double)std::max(std::max(g.H[0], g.H[1]), g.dim == 3 ? g.H[2] : 0);
  const double tau = h->opt.tau_scale / (H * H);
  int* inertia = salloc<int>(h, nprob);
  TS_CUDA(cudaMemsetAsync(inertia, 0, sizeof(int) * nprob, st));
  const size_t smem = h->heat_smem;
  if (g.dim == 2)
    tsl(h), k_heat_eig<2><<<nprob, EIG_THREADS, smem, st>>>(g, E, h->freemask, h->hp, nullptr, 0, nprob, tau, 0.0,
                                                      h->opt.max_modes, 0, nullptr, nullptr, nullptr, nullptr,
                                                      nullptr, nullptr, 0, h->dstatus, nullptr, 0, 0, inertia, 1);
  else
    tsl(h), k_heat_eig<3><<<nprob, EIG_THREADS, smem, st>>>(g, E, h->freemask, h->hp, nullptr, 0, nprob, tau, 0.0,
                                                      h->opt.max_modes, 0, nullptr, nullptr, nullptr, nullptr,
                                                      nullptr, nullptr, 0, h->dstatus, nullptr, 0, 0, inertia, 1);
  TS_CUDA(cudaGetLastError());
  std::vector<int> now(nprob);
  TS_CUDA(cudaMemcpyAsync(now.data(), inertia, sizeof(int) * nprob, cudaMemcpyDeviceToHost, st));
  TS_CUDA(cudaStreamSynchronize(st));
  const int mm = h->opt.max_modes;
  int64_t before = 0, after = 0;
  for (int i = 0; i < nprob; ++i) {
    const int src = h->hp_h[i].dedup_of >= 0 ? h->hp_h[i].dedup_of : i;  // a copied component counts again
    before += std::min(std::max(h->hp_inertia_h[src], 1), mm);
    after += std::min(std::max(now[src], 1), mm);
  }
  return before != after;
}
