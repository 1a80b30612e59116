// Factor and solve of the coarse matrix K_0 = R_0 K R_0^T (Sec. 2.1), FP64.
//
// Two layouts, chosen by the coarse dimension N_c:
//  * dense (N_c <= 2048): blocked Cholesky in 64-wide tiles, explicit
//    L^{-1}, and u0 = L^{-T} (L^{-1} r0) as two triangular GEMVs over all SMs.
//  * block-line (larger N_c): coarse DOFs are numbered line by line, so K_0 is
//    block-tridiagonal with one block per coarse line.  Block Cholesky
//      S_0 = A_00, S_k = A_kk - G_k G_k^T, S_k = L_k L_k^T, W_k = L_k^{-1},
//      G_{k+1} = A_{k+1,k} W_k^T
//    runs line after line with the same tile kernels (O(lines * w^3) FP64
//    work instead of O(N_c^3)), and the solve
//      forward  y_k = W_k (r_k - G_k y_{k-1})
//      backward x_k = W_k^T (y_k - G_{k+1}^T x_{k+1})
//    runs in one launch of a 16-CTA thread-block cluster that keeps the line
//    vectors in distributed shared memory and synchronises per step with the
//    cluster barrier.
// In both, a pivot below 1e-12 of its original diagonal marks a coarse basis
// vector that depends on the earlier ones (e.g. the rotations chi_l r_l sum
// to zero when every coarse node keeps one); it is dropped (unit pivot, zero
// column, zero row of L^{-1}), which leaves span(R_0^T) and hence the Galerkin
// correction unchanged.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "ts_internal.cuh"
#include "ts_reduce.cuh"

namespace cg = cooperative_groups;

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
// block-line helpers
// ---------------------------------------------------------------------------
// S (cw x cw) = K0[r0.., c0..] (nr x nc block), zero elsewhere, optional unit
// diagonal on the padding
__global__ void k_extract_block(const double* __restrict__ K0, int ld, int r0, int c0, int nr, int ncol,
                                double* __restrict__ S, int cw, int unit_pad) {
  const int64_t n = (int64_t)cw * cw;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / cw), j = (int)(e % cw);
    double v;
    if (i < nr && j < ncol)
      v = K0[(int64_t)(r0 + i) * ld + c0 + j];
    else
      v = (unit_pad && i == j) ? 1.0 : 0.0;
    S[e] = v;
  }
}

// C = alpha A B^T (+ C if accumulate), 64x64 tiles; lower_only skips tiles
// above the diagonal.  A, B, C: cw x cw row-major.
__global__ void __launch_bounds__(256) k_gemm_nt(double* __restrict__ C, const double* __restrict__ A,
                                                 const double* __restrict__ B, int cw, double alpha, int accumulate,
                                                 int lower_only) {
  __shared__ double Pa[TB][TB + 1];
  __shared__ double Pb[TB][TB + 1];
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (lower_only && tj > ti) return;
  const int nt = cw / TB;
  double acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.0;
  for (int tk = 0; tk < nt; ++tk) {
    const double* a = A + (int64_t)ti * TB * cw + (int64_t)tk * TB;
    const double* b = B + (int64_t)tj * TB * cw + (int64_t)tk * TB;
    for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
      Pa[e / TB][e % TB] = a[(int64_t)(e / TB) * cw + e % TB];
      Pb[e / TB][e % TB] = b[(int64_t)(e / TB) * cw + e % TB];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int e = threadIdx.x + q * 256;
      const int r = e / TB, c = e % TB;
      double s = 0.0;
#pragma unroll 8
      for (int m = 0; m < TB; ++m) s += Pa[r][m] * Pb[c][m];
      acc[q] += s;
    }
    __syncthreads();
  }
  double* out = C + (int64_t)ti * TB * cw + (int64_t)tj * TB;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int e = threadIdx.x + q * 256;
    const int r = e / TB, c = e % TB;
    double* p = out + (int64_t)r * cw + c;
    *p = accumulate ? *p + alpha * acc[q] : alpha * acc[q];
  }
}

// ---------------------------------------------------------------------------
// Block-line solve.  With F_k = W_k G_k and H_k = W_k^T G_{k+1}^T (setup):
//   forward   t_k = W_k r_k (all lines at once),  y_k = t_k - F_k y_{k-1}
//   backward  s_k = W_k^T y_k (all lines at once), x_k = s_k - H_k x_{k+1}
// so the sequential part is one dense GEMV per line and sweep.
// Per-line storage (stride 3 cw^2): W_k | F_k | H_k, row-major.
// ---------------------------------------------------------------------------
// out[k][i] = sum_j W_k[i][j] in[k][j] (lower) or sum_j W_k[j][i] in[k][j]
// (upper = W^T); grid (nb, cw/16), 16 rows (outputs) per CTA.
// in_dof: if non-null, the input of line k is in_dof[off_k + j] (j < w_k).
__global__ void __launch_bounds__(256) k_cline_tri(const double* __restrict__ cfac, int cw, int transpose,
                                                   const int* __restrict__ line_off, const double* __restrict__ in_dof,
                                                   const double* __restrict__ in, double* __restrict__ out,
                                                   const int* done) {
  if (done && *done) return;
  __shared__ double v[1024];
  const int k = blockIdx.x;
  const int off = line_off[k], wk = line_off[k + 1] - off;
  for (int j = threadIdx.x; j < cw; j += blockDim.x)
    v[j] = in_dof ? ((j < wk) ? in_dof[off + j] : 0.0) : in[(int64_t)k * cw + j];
  __syncthreads();
  const double* W = cfac + (int64_t)k * 3 * cw * cw;
  if (!transpose) {
    // 16 lanes per row read the row contiguously
    const int row = blockIdx.y * 16 + threadIdx.x / 16, part = threadIdx.x % 16;
    const double* wr = W + (int64_t)row * cw;
    double s = 0.0;
    for (int j = part; j <= row; j += 16) s += wr[j] * v[j];
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (part == 0) out[(int64_t)k * cw + row] = s;
  } else {
    // 16 consecutive outputs per row of W read contiguously; 16 row groups
    __shared__ double red[16][17];
    const int j = blockIdx.y * 16 + threadIdx.x % 16, part = threadIdx.x / 16;
    double s = 0.0;
    for (int i = part; i < cw; i += 16)
      if (i >= j) s += W[(int64_t)i * cw + j] * v[i];
    red[part][threadIdx.x % 16] = s;
    __syncthreads();
    if (threadIdx.x < 16) {
      double t = 0.0;
      for (int q = 0; q < 16; ++q) t += red[q][threadIdx.x];
      out[(int64_t)k * cw + blockIdx.y * 16 + threadIdx.x] = t;
    }
  }
}

// Sequential recurrences v_k = tin_k - M_k v_prev over a run of lines, one
// thread-block cluster per run (the launch holds two clusters: the runs of the
// top and bottom halves of the twisted factorization proceed at the same
// time).  Each CTA owns R = cw/C rows, stages its row slice of the next M
// (16-byte asynchronous copies, double-buffered) while the current step runs,
// and writes its part of v_k into every CTA's shared memory before the
// cluster barrier.  The first line of a run has no coupling unless prev0 is
// given.  mat selects the per-line matrix: 1 = F (forward), 2 = H (backward).
struct RecRun {
  int k_first, dir, count, mat;
  const double* prev0;
};

__device__ __forceinline__ void cp_async16_cf(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}

__global__ void __launch_bounds__(256) k_cline_rec(const double* __restrict__ cfac, int cw,
                                                   const int* __restrict__ line_off, const double* __restrict__ tin,
                                                   double* __restrict__ vout, double* __restrict__ u0, RecRun run0,
                                                   RecRun run1, const int* done) {
  if (done && *done) return;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int C = (int)cl.num_blocks();
  const RecRun run = (blockIdx.x / C == 0) ? run0 : run1;
  if (run.count <= 0) return;  // uniform over the cluster
  const int R = cw / C, P = blockDim.x / R;
  const int stride = cw + 2;  // padded row stride of a staged slice (16-byte multiple)
  extern __shared__ double sm[];
  double* vA = sm;
  double* vB = sm + cw;
  double* slice[2] = {sm + 2 * cw, sm + 2 * cw + (size_t)R * stride};
  const int tid = threadIdx.x, ri = tid / P, p = tid % P;
  const int64_t cc = (int64_t)cw * cw;
  const int64_t lstride = 3 * cc;
  auto stage = [&](int k, int buf) {
    const double* src = cfac + (int64_t)k * lstride + (int64_t)run.mat * cc + (int64_t)rank * R * cw;
    const int chunks_per_row = cw / 2;  // 16 bytes = 2 doubles
    for (int c = tid; c < R * chunks_per_row; c += blockDim.x) {
      const int r = c / chunks_per_row, q = c % chunks_per_row;
      cp_async16_cf(slice[buf] + (size_t)r * stride + 2 * q, src + (int64_t)r * cw + 2 * q);
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };
  double* prev = vA;
  double* cur = vB;
  for (int i = tid; i < cw; i += blockDim.x) prev[i] = run.prev0 ? run.prev0[i] : 0.0;
  // matrices are used from step n0 on (step 0 has none without prev0)
  const int n0 = run.prev0 ? 0 : 1;
  int buf = 0;
  if (n0 < run.count) stage(run.k_first + run.dir * n0, 0);
  for (int n = 0; n < run.count; ++n) {
    const int k = run.k_first + run.dir * n;
    const bool coupled = (n >= n0);
    if (coupled) {
      if (n + 1 < run.count) {
        stage(k + run.dir, buf ^ 1);
        asm volatile("cp.async.wait_group 1;\n" ::);
      } else {
        asm volatile("cp.async.wait_group 0;\n" ::);
      }
    }
    __syncthreads();
    double s = 0.0;
    if (coupled) {
      const double* M = slice[buf] + (size_t)ri * stride;
      for (int j = p; j < cw; j += P) s += M[j] * prev[j];
    }
    for (int o = P / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (p == 0) {
      const int i = rank * R + ri;
      const double x = tin[(int64_t)k * cw + i] - s;
      for (int c = 0; c < C; ++c) cl.map_shared_rank(cur, c)[i] = x;
      if (u0) {
        const int off = line_off[k], wk = line_off[k + 1] - off;
        if (i < wk) u0[off + i] = x;
      } else {
        vout[(int64_t)k * cw + i] = x;
      }
    }
    cl.sync();
    if (coupled) buf ^= 1;
    double* t = prev;
    prev = cur;
    cur = t;
  }
  asm volatile("cp.async.wait_group 0;\n" ::);
}

// Middle line of the twisted factorization, in one cluster:
//   y_m = W_m (r_m - G_m y_{m-1} - G'_m y'_{m+1}),  x_m = W_m^T y_m
// G_m and G'_m sit in the F and H slots of line m.  x_m goes to u0 and xm.
__global__ void __launch_bounds__(256) k_cline_mid(const double* __restrict__ cfac, int cw, int nb, int m,
                                                   const int* __restrict__ line_off, const double* __restrict__ r0,
                                                   const double* __restrict__ y, double* __restrict__ u0,
                                                   double* __restrict__ xm, const int* done) {
  if (done && *done) return;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int C = (int)cl.num_blocks();
  const int R = cw / C, P = blockDim.x / R;
  extern __shared__ double sm[];
  double* a = sm;
  double* yy = sm + cw;
  const int tid = threadIdx.x, ri = tid / P, p = tid % P;
  const int i = rank * R + ri;
  const int64_t cc = (int64_t)cw * cw;
  const double* W = cfac + (int64_t)m * 3 * cc;
  const double* Gt = W + cc;       // G_m (couples line m-1)
  const double* Gb = W + 2 * cc;   // G'_m (couples line m+1)
  const int off = line_off[m], wm = line_off[m + 1] - off;
  double s = 0.0;
  if (m > 0) {
    const double* g = Gt + (int64_t)i * cw;
    const double* v = y + (int64_t)(m - 1) * cw;
    for (int j = p; j < cw; j += P) s += g[j] * v[j];
  }
  if (m + 1 < nb) {
    const double* g = Gb + (int64_t)i * cw;
    const double* v = y + (int64_t)(m + 1) * cw;
    for (int j = p; j < cw; j += P) s += g[j] * v[j];
  }
  for (int o = P / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (p == 0) {
    const double v = ((i < wm) ? r0[off + i] : 0.0) - s;
    for (int c = 0; c < C; ++c) cl.map_shared_rank(a, c)[i] = v;
  }
  cl.sync();
  s = 0.0;
  {
    const double* w = W + (int64_t)i * cw;
    for (int j = p; j <= i; j += P) s += w[j] * a[j];
  }
  for (int o = P / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (p == 0)
    for (int c = 0; c < C; ++c) cl.map_shared_rank(yy, c)[i] = s;
  cl.sync();
  s = 0.0;
  for (int q = i + p; q < cw; q += P) s += W[(int64_t)q * cw + i] * yy[q];
  for (int o = P / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (p == 0) {
    xm[i] = s;
    if (i < wm) u0[off + i] = s;
  }
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
static void chol_tiles(ts_handle h, double* A, int ld, double* Linv, const double* diag0, int* dropped) {
  cudaStream_t st = h->ctx->stream;
  const int nt = ld / TB;
  for (int kk = 0; kk < nt; ++kk) {
    tsl(h), k_potrf_tile<<<1, 256, 0, st>>>(A, ld, kk, Linv + (size_t)kk * TB * TB, diag0, dropped, h->dstatus);
    if (kk + 1 < nt) {
      tsl(h), k_trsm_tiles<<<nt - kk - 1, 256, 0, st>>>(A, ld, kk, nt, Linv + (size_t)kk * TB * TB, dropped);
      const int m = nt - kk - 1;
      tsl(h), k_syrk_tiles<<<m * (m + 1) / 2, 256, 0, st>>>(A, ld, kk, nt);
    }
  }
}

// X = L^{-1} (lower tiles; the caller zeroes X first)
static void inverse_tiles(ts_handle h, const double* L, double* X, int ld, const double* Linv, const int* dropped) {
  cudaStream_t st = h->ctx->stream;
  const int nt = ld / TB;
  for (int i = 0; i < nt; ++i) {
    tsl(h), k_copy_tile<<<1, 256, 0, st>>>(Linv + (size_t)i * TB * TB, X, ld, i);
    if (i > 0) tsl(h), k_trtri_row<<<i, 256, 0, st>>>(L, X, ld, i, Linv + (size_t)i * TB * TB);
  }
  tsl(h), k_zero_dropped_rows<<<ld, 256, 0, st>>>(X, ld, dropped);
}

constexpr int DENSE_MAX = 2048;
constexpr int CLUSTER = 16;

void build_coarse_factor(ts_handle h) {
  cudaStream_t st = h->ctx->stream;
  const int nc = h->nc;
  const int ld = h->K0_ld;
  h->coarse_dropped = 0;
  const bool dense = (h->opt.coarse_layout == 1) || (h->opt.coarse_layout == 0 && nc <= DENSE_MAX);
  if (dense) {
    h->coarse_blockline = false;
    h->K0inv_L = dalloc<double>(h, (size_t)ld * ld);
    h->K0inv_LT = dalloc<double>(h, (size_t)ld * ld);
    h->y0 = dalloc<double>(h, ld);
    double* Linv = dalloc<double>(h, (size_t)(ld / TB) * TB * TB);
    double* diag0 = dalloc<double>(h, ld);
    h->K0_dropped = dalloc<int>(h, ld);
    TS_CUDA(cudaMemsetAsync(h->K0inv_L, 0, sizeof(double) * (size_t)ld * ld, st));
    TS_CUDA(cudaMemsetAsync(h->y0, 0, sizeof(double) * ld, st));
    TS_CUDA(cudaMemsetAsync(h->K0_dropped, 0, sizeof(int) * ld, st));
    if (ld > nc) tsl(h), k_pad_identity<<<cdiv(ld - nc, 128), 128, 0, st>>>(h->K0, ld, nc);
    tsl(h), k_get_diag<<<cdiv(ld, 128), 128, 0, st>>>(h->K0, ld, diag0);
    chol_tiles(h, h->K0, ld, Linv, diag0, h->K0_dropped);
    inverse_tiles(h, h->K0, h->K0inv_L, ld, Linv, h->K0_dropped);
    tsl(h), k_transpose<<<dim3(ld / 32, ld / 32), dim3(32, 8), 0, st>>>(h->K0inv_L, h->K0inv_LT, ld);
    TS_CUDA(cudaGetLastError());
    std::vector<int> dr(nc);
    TS_CUDA(cudaMemcpyAsync(dr.data(), h->K0_dropped, sizeof(int) * nc, cudaMemcpyDeviceToHost, st));
    TS_CUDA(cudaStreamSynchronize(st));
    for (int v : dr) h->coarse_dropped += v;
    return;
  }
  // block-line layout: twisted block Cholesky, top half 0..m-1 from the top,
  // bottom half nb-1..m+1 from the bottom, middle line m last
  const std::vector<int>& off = h->line_off_h;
  const int nb = h->n_lines;
  int wmax = 0;
  for (int k = 0; k < nb; ++k) wmax = std::max(wmax, off[k + 1] - off[k]);
  int cw = 64;
  while (cw < wmax) cw *= 2;
  if (cw > 1024) throw TsError(TS_ERR_INVALID, "coarse line too wide for the block-line factor (" + std::to_string(wmax) + ")");
  h->coarse_blockline = true;
  h->cw = cw;
  const int m = nb / 2;
  h->cmid = m;
  const int64_t cc = (int64_t)cw * cw;
  const int64_t bs = 3 * cc;  // per line: W | F | H  (line m: W | G_m | G'_m)
  h->cfac = dalloc<double>(h, (size_t)nb * bs);
  double* S = dalloc<double>(h, cc);
  double* T = dalloc<double>(h, cc);
  double* G = dalloc<double>(h, cc);
  double* GT = dalloc<double>(h, cc);
  double* WT = dalloc<double>(h, cc);
  double* Linv = dalloc<double>(h, (size_t)(cw / TB) * TB * TB);
  double* diag0 = dalloc<double>(h, cw);
  int* dropped = dalloc<int>(h, (size_t)nb * cw);
  h->y0 = dalloc<double>(h, (size_t)nb * cw);
  h->y1 = dalloc<double>(h, (size_t)nb * cw);
  h->xm = dalloc<double>(h, cw);
  h->cline_off = dupload(h, off);
  TS_CUDA(cudaMemsetAsync(h->cfac, 0, sizeof(double) * (size_t)nb * bs, st));
  TS_CUDA(cudaMemsetAsync(dropped, 0, sizeof(int) * (size_t)nb * cw, st));
  TS_CUDA(cudaMemsetAsync(h->y0, 0, sizeof(double) * (size_t)nb * cw, st));
  TS_CUDA(cudaMemsetAsync(h->y1, 0, sizeof(double) * (size_t)nb * cw, st));
  const dim3 tiles(cw / TB, cw / TB);
  const dim3 tgrid(cw / 32, cw / 32), tblk(32, 8);
  auto W_of = [&](int k) { return h->cfac + k * bs; };
  // factor line k with S = A_kk - sum of the given couplings G G^T
  auto factor_line = [&](int k, const double* Ga, const double* Gb) {
    const int o = off[k], w = off[k + 1] - off[k];
    tsl(h), k_extract_block<<<cdiv(cc, 256), 256, 0, st>>>(h->K0, ld, o, o, w, w, S, cw, 1);
    tsl(h), k_get_diag<<<cdiv(cw, 128), 128, 0, st>>>(S, cw, diag0);
    if (Ga) tsl(h), k_gemm_nt<<<tiles, 256, 0, st>>>(S, Ga, Ga, cw, -1.0, 1, 1);
    if (Gb) tsl(h), k_gemm_nt<<<tiles, 256, 0, st>>>(S, Gb, Gb, cw, -1.0, 1, 1);
    chol_tiles(h, S, cw, Linv, diag0, dropped + (size_t)k * cw);
    inverse_tiles(h, S, W_of(k), cw, Linv, dropped + (size_t)k * cw);
  };
  // Gout = A_{kn,k} W_k^T (coupling of the next line kn to line k)
  auto coupling = [&](int kn, int k, double* Gout) {
    tsl(h), k_extract_block<<<cdiv(cc, 256), 256, 0, st>>>(h->K0, ld, off[kn], off[k], off[kn + 1] - off[kn],
                                                          off[k + 1] - off[k], T, cw, 0);
    tsl(h), k_gemm_nt<<<tiles, 256, 0, st>>>(Gout, T, W_of(k), cw, 1.0, 0, 0);
  };
  // F_k = W_k G (C = A B^T with B = G^T)
  auto make_F = [&](int k, const double* Gk) {
    tsl(h), k_transpose<<<tgrid, tblk, 0, st>>>(Gk, GT, cw);
    tsl(h), k_gemm_nt<<<tiles, 256, 0, st>>>(W_of(k) + cc, W_of(k), GT, cw, 1.0, 0, 0);
  };
  // H_k = W_k^T Gn^T (C = A B^T with A = W_k^T, B = Gn)
  auto make_H = [&](int k, const double* Gn) {
    tsl(h), k_transpose<<<tgrid, tblk, 0, st>>>(W_of(k), WT, cw);
    tsl(h), k_gemm_nt<<<tiles, 256, 0, st>>>(W_of(k) + 2 * cc, WT, Gn, cw, 1.0, 0, 0);
  };
  double* Gmid_top = W_of(m) + cc;      // G_m
  double* Gmid_bot = W_of(m) + 2 * cc;  // G'_m
  // top half
  for (int k = 0; k < m; ++k) {
    factor_line(k, k > 0 ? G : nullptr, nullptr);
    if (k > 0) make_F(k, G);
    double* Gn = (k + 1 == m) ? Gmid_top : G;
    coupling(k + 1, k, Gn);
    make_H(k, Gn);
  }
  // bottom half (reversed order: the predecessor of line k is line k+1)
  for (int k = nb - 1; k > m; --k) {
    factor_line(k, k < nb - 1 ? G : nullptr, nullptr);
    if (k < nb - 1) make_F(k, G);
    double* Gn = (k - 1 == m) ? Gmid_bot : G;
    coupling(k - 1, k, Gn);
    make_H(k, Gn);
  }
  // middle line; its F/H slots keep G_m and G'_m, factor W_m
  {
    double* keepW = W_of(m);
    (void)keepW;
    factor_line(m, m > 0 ? Gmid_top : nullptr, m + 1 < nb ? Gmid_bot : nullptr);
  }
  TS_CUDA(cudaGetLastError());
  TS_CUDA(cudaFuncSetAttribute(k_cline_rec, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  TS_CUDA(cudaFuncSetAttribute(k_cline_mid, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  const size_t smem = (size_t)(2 * cw + 2 * (cw / CLUSTER) * (cw + 2)) * sizeof(double);
  TS_CUDA(cudaFuncSetAttribute(k_cline_rec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  std::vector<int> dr((size_t)nb * cw);
  TS_CUDA(cudaMemcpyAsync(dr.data(), dropped, sizeof(int) * dr.size(), cudaMemcpyDeviceToHost, st));
  TS_CUDA(cudaStreamSynchronize(st));
  for (int v : dr) h->coarse_dropped += v;
}

static void cluster_cfg(ts_handle h, cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int clusters, size_t smem) {
  const int cw = h->cw;
  const int R = cw / CLUSTER;
  const int P = std::min(32, 256 / R);  // threads per row: one warp or less
  cfg = {};
  cfg.gridDim = dim3(CLUSTER * clusters, 1, 1);
  cfg.blockDim = dim3(R * P, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = h->ctx->stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CLUSTER;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
}

static void launch_rec(ts_handle h, RecRun a, RecRun b, const double* tin, double* vout, double* u0) {
  const int cw = h->cw;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cluster_cfg(h, cfg, attr, 2, (size_t)(2 * cw + 2 * (cw / CLUSTER) * (cw + 2)) * sizeof(double));
  tsl(h);
  TS_CUDA(cudaLaunchKernelEx(&cfg, k_cline_rec, (const double*)h->cfac, cw, (const int*)h->cline_off, tin, vout, u0,
                             a, b, (const int*)h->done_flag));
}

void launch_coarse_solve(ts_handle h) {
  cudaStream_t st = h->ctx->stream;
  const int nc = h->nc;
  if (!h->coarse_blockline) {
    const int wpb = 8;
    tsl(h), k_tri_gemv<<<cdiv(nc, wpb), 32 * wpb, 0, st>>>(h->K0inv_L, h->K0_ld, nc, true, h->r0, h->y0, h->done_flag);
    tsl(h), k_tri_gemv<<<cdiv(nc, wpb), 32 * wpb, 0, st>>>(h->K0inv_LT, h->K0_ld, nc, false, h->y0, h->u0,
                                                          h->done_flag);
    TS_CUDA(cudaGetLastError());
    return;
  }
  const int cw = h->cw, nb = h->n_lines, m = h->cmid;
  const dim3 grid(nb, cw / 16);
  // t_k = W_k r_k
  tsl(h), k_cline_tri<<<grid, 256, 0, st>>>(h->cfac, cw, 0, h->cline_off, h->r0, nullptr, h->y0, h->done_flag);
  // forward runs: top 0..m-1, bottom nb-1..m+1  ->  y (in y1)
  launch_rec(h, RecRun{0, 1, m, 1, nullptr}, RecRun{nb - 1, -1, nb - 1 - m, 1, nullptr}, h->y0, h->y1, nullptr);
  // middle line -> x_m
  {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    cluster_cfg(h, cfg, attr, 1, (size_t)(2 * cw) * sizeof(double));
    tsl(h);
    TS_CUDA(cudaLaunchKernelEx(&cfg, k_cline_mid, (const double*)h->cfac, cw, nb, m, (const int*)h->cline_off,
                               (const double*)h->r0, (const double*)h->y1, h->u0, h->xm, (const int*)h->done_flag));
  }
  // s_k = W_k^T y_k
  tsl(h), k_cline_tri<<<grid, 256, 0, st>>>(h->cfac, cw, 1, h->cline_off, nullptr, h->y1, h->y0, h->done_flag);
  // backward runs from the middle: top m-1..0, bottom m+1..nb-1  ->  u0
  launch_rec(h, RecRun{m - 1, -1, m, 2, h->xm}, RecRun{m + 1, 1, nb - 1 - m, 2, h->xm}, h->y0, nullptr, h->u0);
  TS_CUDA(cudaGetLastError());
}

// one forward launch of the coarse recurrences (both halves), for timing
void launch_coarse_rec_once(ts_handle h) {
  const int nb = h->n_lines, m = h->cmid;
  launch_rec(h, RecRun{0, 1, m, 1, nullptr}, RecRun{nb - 1, -1, nb - 1 - m, 1, nullptr}, h->y0, h->y1, nullptr);
}

// algorithmic FLOPs of one such launch: a w_k x w_prev GEMV per coupled line
double coarse_rec_flops(ts_handle h) {
  const std::vector<int>& off = h->line_off_h;
  const int nb = h->n_lines, m = h->cmid;
  double f = 0.0;
  for (int k = 1; k < m; ++k) f += 2.0 * (off[k + 1] - off[k]) * (off[k] - off[k - 1]);
  for (int k = nb - 2; k > m; --k) f += 2.0 * (off[k + 1] - off[k]) * (off[k + 2] - off[k + 1]);
  return f;
}
