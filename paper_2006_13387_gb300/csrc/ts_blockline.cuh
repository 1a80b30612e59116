// Block-line LDL^T factorisation and solve for block-tridiagonal symmetric
// matrices, one CTA per matrix.
//
// Every matrix on the path has this shape once its unknowns are ordered by
// node lines (2D: node rows; 3D: node planes): elements couple only adjacent
// lines.  With A_kk the diagonal blocks and A_{k,k-1} the sub-diagonal ones:
//   S_0 = A_00,  S_k = A_kk - G_k D_{k-1}^{-1} G_k^T,  G_k = A_{k,k-1} W_{k-1}^T,
//   S_k = L_k D_k L_k^T (unit lower, no pivoting),  W_k = L_k^{-1}.
// Solve A x = r:
//   forward   y_k = W_k (r_k - G_k yt_{k-1}),  yt_k = D_k^{-1} y_k
//   backward  x_k = W_k^T (yt_k - D_k^{-1} G_{k+1}^T x_{k+1})
// The number of negative D entries is the inertia (Sylvester) of A.
// FP64 work is O(nb w^3) per factor instead of O((nb w)^3) for a dense one,
// and the solve is 2 nb small GEMV steps.
#pragma once
#include "ts_internal.cuh"

// Factor storage per block k at base + k*stride: W (w*w), G (w*w), dinv (w);
// the stride is rounded up to 4 elements so that every block starts on a
// 16-byte boundary in FP32 and FP64 (asynchronous 16-byte copies).
__host__ __device__ inline int64_t bl_block_stride(int w) { return ((2 * (int64_t)w * w + w + 3) / 4) * 4; }
__host__ __device__ inline int64_t bl_size(int w, int nb) { return nb * bl_block_stride(w); }

// Shared memory needed by bl_factor: 4 w*w doubles + 2 w doubles + 2 ints
__host__ inline size_t bl_factor_smem(int w) { return (4 * (size_t)w * w + 2 * w) * sizeof(double) + 64; }

// Asm must provide:
//   __device__ double entry(int kr, int p, int kc, int q) const : A entry
//     between unknown p of line kr and unknown q of line kc (|kr-kc|<=1)
//
// Returns (in all threads) the number of negative pivots; *bad is set
// (shared, nonzero) if a pivot was zero/NaN or, with spd, non-positive.
template <class Asm>
__device__ int bl_factor(const Asm& A, int nb, int w, double* __restrict__ out, bool store, bool spd,
                         double* smem, int* bad) {
  double* S = smem;              // w*w
  double* T = S + w * w;         // w*w  (A_{k+1,k}, then scratch)
  double* Wm = T + w * w;        // w*w
  double* G = Wm + w * w;        // w*w
  double* dinv = G + w * w;      // w
  double* colj = dinv + w;       // w
  __shared__ int s_neg;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) s_neg = 0;
  for (int k = 0; k < nb; ++k) {
    // S = A_kk (lower triangle incl. diagonal)
    for (int e = tid; e < w * w; e += nt) {
      int i = e / w, j = e % w;
      S[e] = (j <= i) ? A.entry(k, i, k, j) : 0.0;
    }
    __syncthreads();
    if (k > 0) {
      // S -= G diag(dinv) G^T   (lower triangle)
      for (int e = tid; e < w * w; e += nt) {
        int i = e / w, j = e % w;
        if (j <= i) {
          double s = 0.0;
          for (int m = 0; m < w; ++m) s += G[i * w + m] * dinv[m] * G[j * w + m];
          S[e] -= s;
        }
      }
      __syncthreads();
      if (store) {
        double* o = out + k * bl_block_stride(w) + (int64_t)w * w;
        for (int e = tid; e < w * w; e += nt) o[e] = G[e];
      }
    } else if (store) {
      double* o = out + (int64_t)w * w;
      for (int e = tid; e < w * w; e += nt) o[e] = 0.0;
    }
    // in-place LDL^T of S (right-looking, no pivoting)
    for (int j = 0; j < w; ++j) {
      double dj = S[j * w + j];
      for (int i = j + 1 + tid; i < w; i += nt) colj[i] = S[i * w + j];
      __syncthreads();
      if (tid == 0) {
        if (!(dj == dj) || dj == 0.0 || (spd && !(dj > 0.0))) *bad = 1;
        if (dj < 0.0) s_neg++;
        dinv[j] = (dj != 0.0) ? 1.0 / dj : 0.0;
      }
      double inv = (dj != 0.0) ? 1.0 / dj : 0.0;
      const int m = w - j - 1;  // trailing size
      for (int e = tid; e < m * m; e += nt) {
        int ii = j + 1 + e / m, kk = j + 1 + e % m;
        if (kk <= ii) S[ii * w + kk] -= colj[ii] * inv * colj[kk];
      }
      for (int i = j + 1 + tid; i < w; i += nt) S[i * w + j] = colj[i] * inv;
      __syncthreads();
    }
    // W = L^{-1}, one column per thread: W[i][c] = -sum_{m=c}^{i-1} L[i][m] W[m][c]
    for (int c = tid; c < w; c += nt) {
      for (int i = 0; i < c; ++i) Wm[i * w + c] = 0.0;
      Wm[c * w + c] = 1.0;
      for (int i = c + 1; i < w; ++i) {
        double s = 0.0;
        for (int m = c; m < i; ++m) s += S[i * w + m] * Wm[m * w + c];
        Wm[i * w + c] = -s;
      }
    }
    __syncthreads();
    if (store) {
      double* o = out + k * bl_block_stride(w);
      for (int e = tid; e < w * w; e += nt) o[e] = Wm[e];
      for (int i = tid; i < w; i += nt) o[2 * (int64_t)w * w + i] = dinv[i];
    }
    if (k + 1 < nb) {
      // T = A_{k+1,k};  G = T W^T  (W lower: G[i][j] = sum_{m<=j} T[i][m] W[j][m])
      for (int e = tid; e < w * w; e += nt) {
        int i = e / w, j = e % w;
        T[e] = A.entry(k + 1, i, k, j);
      }
      __syncthreads();
      for (int e = tid; e < w * w; e += nt) {
        int i = e / w, j = e % w;
        double s = 0.0;
        for (int m = 0; m <= j; ++m) s += T[i * w + m] * Wm[j * w + m];
        G[e] = s;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  return s_neg;
}

// Solve A x = r in place on a shared-memory vector v (nb*w entries, line-major)
// with a stored factor F (element type TF).  tmp: shared scratch of 2*w TA.
template <class TF, class TA>
__device__ void bl_solve(const TF* __restrict__ F, int nb, int w, TA* v, TA* tmp) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t bs = bl_block_stride(w);
  TA* t = tmp;
  // forward: v_k <- yt_k = dinv_k * W_k (r_k - G_k yt_{k-1})
  for (int k = 0; k < nb; ++k) {
    const TF* Wk = F + k * bs;
    const TF* Gk = Wk + (int64_t)w * w;
    const TF* dk = Gk + (int64_t)w * w;
    TA* vk = v + (int64_t)k * w;
    if (k > 0) {
      const TA* vp = vk - w;
      for (int i = tid; i < w; i += nt) {
        TA s = vk[i];
        const TF* gr = Gk + (int64_t)i * w;
        for (int m = 0; m < w; ++m) s -= (TA)gr[m] * vp[m];
        t[i] = s;
      }
    } else {
      for (int i = tid; i < w; i += nt) t[i] = vk[i];
    }
    __syncthreads();
    for (int i = tid; i < w; i += nt) {
      const TF* wr = Wk + (int64_t)i * w;
      TA s = 0;
      for (int m = 0; m <= i; ++m) s += (TA)wr[m] * t[m];
      vk[i] = s * (TA)dk[i];
    }
    __syncthreads();
  }
  // backward: x_k = W_k^T (yt_k - dinv_k * G_{k+1}^T x_{k+1})
  for (int k = nb - 1; k >= 0; --k) {
    const TF* Wk = F + k * bs;
    const TF* dk = Wk + 2 * (int64_t)w * w;
    TA* vk = v + (int64_t)k * w;
    if (k + 1 < nb) {
      const TF* Gn = F + (k + 1) * bs + (int64_t)w * w;
      const TA* xn = vk + w;
      for (int j = tid; j < w; j += nt) {
        TA s = 0;
        for (int i = 0; i < w; ++i) s += (TA)Gn[(int64_t)i * w + j] * xn[i];
        t[j] = vk[j] - (TA)dk[j] * s;
      }
    } else {
      for (int j = tid; j < w; j += nt) t[j] = vk[j];
    }
    __syncthreads();
    for (int j = tid; j < w; j += nt) {
      TA s = 0;
      for (int i = j; i < w; ++i) s += (TA)Wk[(int64_t)i * w + j] * t[i];
      vk[j] = s;
    }
    __syncthreads();
  }
}

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

// ---------------------------------------------------------------------------
// Solve with the factor blocks staged through shared memory.  The factor of
// line k (W_k, G_k, dinv_k: one contiguous, 16-byte aligned block) does not
// depend on the vector, so it is fetched with asynchronous 16-byte copies
// (cp.async) one step ahead into a second buffer while the current step runs
// from shared memory.  Sweeps as in bl_solve.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

template <class TF>
__device__ __forceinline__ void stage_block(TF* dst, const TF* src, int64_t elems) {
  const int64_t chunks = elems * (int64_t)sizeof(TF) / 16;
  const char* s = reinterpret_cast<const char*>(src);
  char* d = reinterpret_cast<char*>(dst);
  for (int64_t c = threadIdx.x; c < chunks; c += blockDim.x) cp_async16(d + 16 * c, s + 16 * c);
  cp_async_commit();
}

// four threads per row: sum over the lane's residue class, then two shuffles
template <class TF>
__device__ __forceinline__ TF quad_sum(TF s) {
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  return s;
}

template <class TF>
__device__ void bl_solve_staged(const TF* __restrict__ F, int nb, int w, TF* v, TF* t, TF* buf0, TF* buf1) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int p = tid & 3, rpp = nt >> 2;  // lane in the row group, rows per pass
  const int64_t bs = bl_block_stride(w);
  const int64_t ww = (int64_t)w * w;
  TF* buf[2] = {buf0, buf1};
  stage_block(buf[0], F, bs);
  // forward: v_k <- dinv_k * W_k (r_k - G_k v_{k-1})
  for (int k = 0; k < nb; ++k) {
    if (k + 1 < nb) {
      stage_block(buf[(k + 1) & 1], F + (k + 1) * bs, bs);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const TF* Wk = buf[k & 1];
    const TF* Gk = Wk + ww;
    const TF* dk = Wk + 2 * ww;
    TF* vk = v + (int64_t)k * w;
    for (int i0 = 0; i0 < w; i0 += rpp) {
      const int i = i0 + (tid >> 2);
      TF s = 0;
      if (k > 0 && i < w) {
        const TF* gr = Gk + (int64_t)i * w;
        const TF* vp = vk - w;
        for (int m = p; m < w; m += 4) s += gr[m] * vp[m];
      }
      s = quad_sum(s);
      if (p == 0 && i < w) t[i] = vk[i] - s;
    }
    __syncthreads();
    for (int i0 = 0; i0 < w; i0 += rpp) {
      const int i = i0 + (tid >> 2);
      TF s = 0;
      if (i < w) {
        const TF* wr = Wk + (int64_t)i * w;
        for (int m = p; m <= i; m += 4) s += wr[m] * t[m];
      }
      s = quad_sum(s);
      if (p == 0 && i < w) vk[i] = s * dk[i];
    }
    __syncthreads();
  }
  // backward: x_k = W_k^T (yt_k - dinv_k * G_{k+1}^T x_{k+1}); block nb-1 is resident
  for (int k = nb - 1; k >= 0; --k) {
    const TF* Wk = buf[k & 1];
    const TF* dk = Wk + 2 * ww;
    TF* vk = v + (int64_t)k * w;
    for (int j0 = 0; j0 < w; j0 += rpp) {
      const int j = j0 + (tid >> 2);
      TF s = 0;
      if (k + 1 < nb && j < w) {
        const TF* Gn = buf[(k + 1) & 1] + ww;
        const TF* xn = vk + w;
        for (int i = p; i < w; i += 4) s += Gn[(int64_t)i * w + j] * xn[i];
      }
      s = quad_sum(s);
      if (p == 0 && j < w) t[j] = vk[j] - dk[j] * s;
    }
    __syncthreads();
    // the buffer of block k+1 is free: fetch block k-1 into it
    if (k > 0) stage_block(buf[(k + 1) & 1], F + (k - 1) * bs, bs);
    for (int j0 = 0; j0 < w; j0 += rpp) {
      const int j = j0 + (tid >> 2);
      TF s = 0;
      if (j < w)
        for (int i = j + p; i < w; i += 4) s += Wk[(int64_t)i * w + j] * t[i];
      s = quad_sum(s);
      if (p == 0 && j < w) vk[j] = s;
    }
    cp_async_wait<0>();
    __syncthreads();
  }
}
