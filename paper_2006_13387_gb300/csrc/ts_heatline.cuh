// Block-line factor and solve of the heat matrices K^l + s M^l on a closed
// coarse box (Sec. 4.1), one CTA per problem, every thread busy.
//
// Unknowns are ordered by node lines (2D: rows, 3D: planes) of width w; a
// node couples to the 3 (2D) or 9 (3D) nodes of each neighbouring line whose
// in-line position differs by at most one.  Block LU:
//   S_0 = A_00,  S_k = A_kk - C_k S_{k-1}^{-1} C_k^T,   C_k = A_{k,k-1},
// with each S_k^{-1} formed by symmetric Gauss-Jordan sweeps over the upper
// triangle, all its entries at once (no pivoting: the pivots are those of the
// LDL^T factor, so the number of negative ones is the inertia of the matrix,
// Sylvester).  The solve is
//   forward   u_k = S_k^{-1} (r_k - C_k u_{k-1})
//   backward  x_k = u_k - S_k^{-1} C_{k+1}^T x_{k+1}
// one dense symmetric GEMV per line and sweep (8 threads per row).  Stored per problem:
// S_k^{-1} (its upper triangle per line), the coupling stencils C_k (w * NB per line) and the
// mass stencil of the box (n * NS) used by the Lanczos iteration.
#pragma once
#include "ts_fe_entries.cuh"
#include "ts_internal.cuh"

template <int DIM>
struct HeatLine {
  static constexpr int NB = (DIM == 2) ? 3 : 9;   // couplings to one neighbouring line
  static constexpr int NS = (DIM == 2) ? 9 : 27;  // full node stencil
};

// position q in the neighbouring line of in-line position p, offset slot t
// (2D: dx = t - 1; 3D: dx = t % 3 - 1, dy = t / 3 - 1), or -1 outside the box
template <int DIM>
__device__ __forceinline__ int hl_nbr(int p, int t, int bx, int by) {
  if (DIM == 2) {
    const int x = p + t - 1;
    return (x >= 0 && x < bx) ? x : -1;
  }
  const int x = p % bx + t % 3 - 1, y = p / bx + t / 3 - 1;
  return (x >= 0 && x < bx && y >= 0 && y < by) ? x + bx * y : -1;
}

// stored line block of S_k^{-1}: its upper triangle, row by row (row i holds
// columns i..w-1 from offset i w - i (i - 1) / 2), rounded up to an even count
// of doubles (every block starts on a 16-byte boundary)
__host__ __device__ inline int64_t hl_pk(int w) { return ((int64_t)w * (w + 1) / 2 + 1) & ~(int64_t)1; }

// stored doubles per problem: S_k^{-1} blocks, coupling stencils, mass and
// stiffness stencils (even, so that problems stay 16-byte aligned)
__host__ __device__ inline int64_t heat_line_size(int w, int nb, int n, int dim) {
  const int NB = (dim == 2) ? 3 : 9, NS = (dim == 2) ? 9 : 27;
  const int64_t s = (int64_t)nb * hl_pk(w) + (int64_t)nb * w * NB + 2 * (int64_t)n * NS;
  return (s + 1) & ~(int64_t)1;
}

// upper-triangle entries (i <= c) of a w x w line block
__host__ __device__ inline int hl_nup(int w) { return w * (w + 1) / 2; }

// shared memory (doubles) of the factor: S, S_prev^{-1}, T (w^2 each), the
// coupling stencil (w * NB), pivot row and column (2 w), and the (row, column)
// table of the upper triangle (one 32-bit word per entry)
__host__ inline size_t heat_factor_smem(int w, int dim) {
  const int NB = (dim == 2) ? 3 : 9;
  return ((size_t)3 * w * w + (size_t)w * NB + 2 * (size_t)w + (size_t)(hl_nup(w) + 1) / 2) * sizeof(double);
}

// In-place inverse of the symmetric w x w matrix S (shared; only its upper
// triangle is read) by Gauss-Jordan sweeps without pivoting.  A sweep keeps
// the matrix symmetric, so each one updates the upper triangle only (tab:
// its (row << 16 | column) pairs) and the lower one is mirrored at the end.
// Returns the number of negative pivots (valid in all threads); sets *bad on
// a zero/NaN pivot or, with spd, a non-positive one.
__device__ int hl_gj_inverse(double* S, int w, double* rowj, double* colj, const unsigned* tab, bool spd,
                             int* bad) {
  __shared__ double s_ip;
  __shared__ int s_neg;
  const int tid = threadIdx.x, nt = blockDim.x, nu = hl_nup(w);
  if (tid == 0) s_neg = 0;
  for (int j = 0; j < w; ++j) {
    __syncthreads();
    // pivot reciprocal, formed once
    if (tid == 0) {
      const double p = S[j * w + j];
      if (!(p == p) || p == 0.0 || (spd && !(p > 0.0))) *bad = 1;
      if (p < 0.0) ++s_neg;
      s_ip = (p != 0.0) ? 1.0 / p : 0.0;
    }
    __syncthreads();
    const double ip = s_ip;
    // pivot row (= column), and its copy already scaled by 1/p
    for (int c = tid; c < w; c += nt) {
      const double r = (c >= j) ? S[j * w + c] : S[c * w + j];
      rowj[c] = r;
      colj[c] = r * ip;
    }
    __syncthreads();
    for (int e = tid; e < nu; e += nt) {
      const unsigned ic = tab[e];
      const int i = (int)(ic >> 16), c = (int)(ic & 0xffffu);
      double v;
      if (i == j && c == j)
        v = -ip;
      else if (i == j || c == j)
        v = colj[i + c - j];
      else
        v = fma(-colj[i], rowj[c], S[i * w + c]);
      S[i * w + c] = v;
    }
  }
  __syncthreads();
  // the sweeps leave -S^{-1} in the upper triangle: mirror, then negate
  for (int e = tid; e < w * w; e += nt) {
    const int i = e / w, c = e % w;
    if (i > c) S[e] = -S[c * w + i];
  }
  __syncthreads();
  for (int e = tid; e < nu; e += nt) {
    const unsigned ic = tab[e];
    const int i = (int)(ic >> 16), c = (int)(ic & 0xffffu);
    S[i * w + c] = -S[i * w + c];
  }
  __syncthreads();
  return s_neg;
}

// Block LU factor of A (A.entry(kr, p, kc, q): the entry between unknown p
// of line kr and unknown q of line kc, |kr - kc| <= 1).  With Minv /
// Cout given, stores S_k^{-1} and the coupling stencils C_k (k >= 1).
// Returns the number of negative pivots in every thread.
template <int DIM, class Asm>
__device__ int heat_line_factor(const Asm& A, int w, int nb, int bx, int by, double* smem, double* Minv, double* Cout,
                                bool spd, int* bad) {
  constexpr int NB = HeatLine<DIM>::NB;
  const int tid = threadIdx.x, nt = blockDim.x;
  double* S = smem;
  double* Mp = S + w * w;
  double* T = Mp + w * w;
  double* Cs = T + w * w;
  double* rowj = Cs + w * NB;
  double* colj = rowj + w;
  unsigned* tab = reinterpret_cast<unsigned*>(colj + w);
  const int nu = hl_nup(w);
  // (row, column) pairs of the upper triangle, row by row
  for (int i = 0; i < w; ++i) {
    const int off = i * w - i * (i - 1) / 2;
    for (int c = i + tid; c < w; c += nt) tab[off + c - i] = ((unsigned)i << 16) | (unsigned)c;
  }
  int neg = 0;
  for (int k = 0; k < nb; ++k) {
    __syncthreads();
    // the line's own block, upper triangle (the sweeps read no other part)
    for (int e = tid; e < nu; e += nt) {
      const int i = (int)(tab[e] >> 16), j = (int)(tab[e] & 0xffffu);
      S[i * w + j] = A.entry(k, i, k, j);
    }
    if (k > 0) {
      // C_k stencil
      for (int e = tid; e < w * NB; e += nt) {
        const int i = e / NB, t = e % NB;
        const int q = hl_nbr<DIM>(i, t, bx, by);
        Cs[e] = (q >= 0) ? A.entry(k, i, k - 1, q) : 0.0;
      }
      __syncthreads();
      if (Cout)
        for (int e = tid; e < w * NB; e += nt) Cout[(int64_t)k * w * NB + e] = Cs[e];
      // T = C_k S_{k-1}^{-1}
      for (int e = tid; e < w * w; e += nt) {
        const int i = e / w, c = e % w;
        double s = 0.0;
#pragma unroll
        for (int t = 0; t < NB; ++t) {
          const int q = hl_nbr<DIM>(i, t, bx, by);
          if (q >= 0) s = fma(Cs[i * NB + t], Mp[q * w + c], s);
        }
        T[e] = s;
      }
      __syncthreads();
      // S -= T C_k^T (symmetric: the upper triangle)
      for (int e = tid; e < nu; e += nt) {
        const int i = (int)(tab[e] >> 16), j = (int)(tab[e] & 0xffffu);
        double s = 0.0;
#pragma unroll
        for (int t = 0; t < NB; ++t) {
          const int q = hl_nbr<DIM>(j, t, bx, by);
          if (q >= 0) s = fma(T[i * w + q], Cs[j * NB + t], s);
        }
        S[i * w + j] -= s;
      }
    }
    neg += hl_gj_inverse(S, w, rowj, colj, tab, spd, bad);
    if (Minv)
      for (int e = tid; e < nu; e += nt) {
        const int i = (int)(tab[e] >> 16), c = (int)(tab[e] & 0xffffu);
        Minv[(int64_t)k * hl_pk(w) + e] = S[i * w + c];
      }
    // S_k^{-1} becomes the previous inverse of the next line
    double* t = S;
    S = Mp;
    Mp = t;
  }
  __syncthreads();
  return neg;
}

__device__ __forceinline__ void hl_cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}

// copy one stored line block (hl_pk(w) doubles, 16-byte aligned) into buf
// with 16-byte asynchronous copies, as one commit group
__device__ __forceinline__ void hl_stage(double* buf, const double* src, int w) {
  const int64_t half = hl_pk(w) / 2;
  for (int64_t c = threadIdx.x; c < half; c += blockDim.x) hl_cp_async16(buf + 2 * c, src + 2 * c);
  asm volatile("cp.async.commit_group;\n" ::);
}

// out_i (= or -=) sum_c S[i][c] y[c] for the symmetric S stored as its packed
// upper triangle P (S[i][c] = P[i w - i (i - 1) / 2 + c - i] for c >= i, and
// S[c][i] below the diagonal), 8 threads per row
__device__ __forceinline__ void hl_gemv(const double* P, const double* y, double* out, int w, bool sub) {
  const int tid = threadIdx.x, part = tid & 7, rq = tid >> 3, nq = blockDim.x >> 3;
  for (int i0 = 0; i0 < w; i0 += nq) {
    const int i = i0 + rq;
    double s = 0.0;
    if (i < w) {
      const int ri = i * w - i * (i - 1) / 2 - i;
      for (int c = part; c < w; c += 8) {
        const int idx = (c >= i) ? ri + c : c * w - c * (c - 1) / 2 + i - c;
        s = fma(P[idx], y[c], s);
      }
    }
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    if (i < w && part == 0) out[i] = sub ? out[i] - s : s;
  }
}

// Solve (K + s M) x = v in place (v: n doubles in shared memory) with the
// stored factor; y: w doubles of scratch, buf: 2 hl_pk(w) doubles (16-byte
// aligned) in which the line blocks are staged one step ahead.
template <int DIM>
__device__ void heat_line_solve(const double* Minv, const double* C, int w, int nb, int bx, int by, double* v,
                                double* y, double* buf) {
  constexpr int NB = HeatLine<DIM>::NB;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t ws = hl_pk(w);
  double* b[2] = {buf, buf + ws};
  __syncthreads();
  hl_stage(b[0], Minv, w);
  // forward: u_k = S_k^{-1} (v_k - C_k u_{k-1})
  for (int k = 0; k < nb; ++k) {
    double* vk = v + (int64_t)k * w;
    for (int i = tid; i < w; i += nt) {
      double s = vk[i];
      if (k > 0) {
        const double* ck = C + ((int64_t)k * w + i) * NB;
#pragma unroll
        for (int t = 0; t < NB; ++t) {
          const int q = hl_nbr<DIM>(i, t, bx, by);
          if (q >= 0) s = fma(-ck[t], vk[q - w], s);
        }
      }
      y[i] = s;
    }
    if (k + 1 < nb) {
      hl_stage(b[(k + 1) & 1], Minv + (k + 1) * ws, w);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
    hl_gemv(b[k & 1], y, vk, w, false);
    __syncthreads();
  }
  // backward: x_k = u_k - S_k^{-1} C_{k+1}^T x_{k+1}.  Blocks nb-1 and nb-2
  // are staged from the forward sweep; block k-2 goes into block k's buffer
  // once block k is used, so one block is always in flight.
  if (nb >= 3) hl_stage(b[(nb - 3) & 1], Minv + (nb - 3) * ws, w);
  for (int k = nb - 2; k >= 0; --k) {
    double* vk = v + (int64_t)k * w;
    const double* ck = C + (int64_t)(k + 1) * w * NB;
    for (int i = tid; i < w; i += nt) {
      // (C_{k+1}^T x)_i: node q of line k+1 at offset t from i sees i at the
      // mirrored offset NB-1-t
      double s = 0.0;
#pragma unroll
      for (int t = 0; t < NB; ++t) {
        const int q = hl_nbr<DIM>(i, t, bx, by);
        if (q >= 0) s = fma(ck[q * NB + (NB - 1 - t)], vk[w + q], s);
      }
      y[i] = s;
    }
    if (k >= 1)
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    else
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    hl_gemv(b[k & 1], y, vk, w, true);
    __syncthreads();
    if (k >= 2) hl_stage(b[k & 1], Minv + (k - 2) * ws, w);
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Mass stencil of the box: Mst[i][t] = M(i, neighbour t) for free i (zero
// rows at Dirichlet nodes), t over the 3^DIM offsets (x fastest).
template <int DIM>
__device__ __forceinline__ int hl_snbr(int i, int t, int bx, int by, int bz) {
  const int x = i % bx + t % 3 - 1;
  const int y = (DIM == 2) ? i / bx + t / 3 - 1 : (i / bx) % by + (t / 3) % 3 - 1;
  const int z = (DIM == 2) ? 0 : i / (bx * by) + t / 9 - 1;
  if (x < 0 || x >= bx || y < 0 || y >= by || z < 0 || z >= bz) return -1;
  return x + bx * (y + by * z);
}

template <int DIM>
__device__ __forceinline__ void hl_mass_apply(const double* Mst, const double* x, double* y, int n, int bx, int by,
                                              int bz) {
  constexpr int NS = HeatLine<DIM>::NS;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double* m = Mst + (int64_t)i * NS;
    double s = 0.0;
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const int j = hl_snbr<DIM>(i, t, bx, by, bz);
      if (j >= 0) s = fma(m[t], x[j], s);
    }
    y[i] = s;
  }
}
