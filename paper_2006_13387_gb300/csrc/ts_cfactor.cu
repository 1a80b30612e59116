// Factor and solve of the coarse matrix K_0 = R_0 K R_0^T (Sec. 2), FP64.
//
// Coarse DOFs are numbered line by line (ts_coarse.cu), so K_0 is block
// tridiagonal with one diagonal block per coarse line and couplings only
// between neighbouring lines.  The factor is block cyclic reduction: the
// lines at odd positions of the current line list are eliminated together
// (they are coupled only to lines that stay), the Schur complement on the
// remaining lines is again block tridiagonal, and the halving repeats until
// one line is left.  For an eliminated line j with list neighbours l < j < r
// (current blocks Ahat_j, couplings C_l = A_{l,j}, C_j = A_{j,r}):
//   Ainv_j = Ahat_j^{-1}                         (Cholesky, L^{-1}, L^{-T} L^{-1})
//   Qlt_j  = C_l Ainv_j,   Qrt_j = C_j^T Ainv_j  (= (Ahat_j^{-1} A_{j,l})^T, ...)
//   Ahat_l -= Qlt_j C_l^T,  Ahat_r -= Qrt_j C_j, new coupling A_{l,r} = -Qlt_j C_j.
// The solve is then 2 log2(lines) + 1 stages of independent dense GEMVs:
//   forward   y_j = Ainv_j b_j,  b_l -= Qlt_{j+} b_{j+} + Qrt_{j-} b_{j-}
//   last line x = Ainv b
//   backward  x_j = y_j - Qlt_j^T x_l - Qrt_j^T x_r
// each stage one launch over all SMs, instead of a recurrence over the lines.
// With one line (small coarse spaces) this is the dense inverse K_0^{-1}.
//
// A pivot below 1e-9 of its original diagonal entry marks a coarse basis
// vector that depends on the others (e.g. the rotations chi_l r_l sum to
// zero when every coarse node keeps one); it is dropped -- unit pivot, zero
// column of L, zero row of L^{-1} -- which leaves span(R_0^T) and hence the
// Galerkin correction unchanged.  The margin above the rounding level
// matters for the reduction: an exactly dependent vector's pivot comes out
// of the tiled elimination as rounding noise of either sign, around 1e-12 of
// its diagonal, and a kept noise pivot would poison the Schur complements of
// the next levels.  Only a pivot below -1e-6 of its diagonal is taken as a
// K_0 that is not positive semi-definite.
//
// All dense block work runs in batched FP64 tile kernels (32 x 32 tiles, one
// launch per step for all lines of a level).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <cmath>
#include <mutex>
#include <vector>

#include "ts_internal.cuh"
#include "ts_bpcg.cuh"
#include "ts_bulk.cuh"
#include "ts_tiles.cuh"

constexpr int T32 = TILE;   // tile edge of the batched dense kernels
constexpr int DENSE_MAX = 2048;
constexpr int BR = 16;      // output rows per CTA in a solve stage

// ---------------------------------------------------------------------------
// batched FP64 tile GEMM:  C = alpha op(A) op(B) + beta C
// ---------------------------------------------------------------------------

// One CTA per 32 x 32 output tile of one task; blockIdx.y selects the task.
// Every operand tile is staged in shared memory before C is written, and a
// CTA writes only its own tile, so C may alias A when k == 32 (in-place
// panel update).
// Split k (gridDim.z = splits > 1, launches with fewer tiles than the GPU
// holds CTAs and no aliasing): slice z of a tile forms the product over its
// share of the tile's k range and stores it in part; the slice that arrives
// last (per-tile counter in cnt, reset by it) adds the partial tiles in slice
// order, so the result does not depend on the arrival order, and writes C.
__global__ void __launch_bounds__(256, 5) k_bgemm(const GemmTask* __restrict__ tasks, double* __restrict__ part,
                                              unsigned* __restrict__ cnt) {
  const GemmTask t = tasks[blockIdx.y];
  const int tn = t.n / T32;
  const int ti = blockIdx.x / tn, tj = blockIdx.x % tn;
  if (ti * T32 >= t.m) return;
  if ((t.mode & 1) && tj > ti) return;
  __shared__ double As[T32][T32 + 1];
  __shared__ double Bs[T32][T32 + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  int k0 = 0, k1 = t.k;
  if (t.mode & 2) k0 = max(ti, tj) * T32;
  if (t.mode & 4) k0 = tj * T32;
  if (t.kr) {
    // tiles of the sparse operand outside this range are zero
    const int2 r = t.kr[t.kr_by == 1 ? ti : tj];
    k0 = max(k0, r.x * T32);
    k1 = min(k1, (r.y + 1) * T32);
  }
  const int splits = gridDim.z;
  if (splits > 1) {
    const int per = ((max(k1 - k0, 0) / T32 + splits - 1) / splits) * T32;
    const int s0 = k0 + (int)blockIdx.z * per;
    k1 = min(k1, s0 + per);
    k0 = s0;
  }
  if (t.flops && threadIdx.x == 0 && k1 > k0) atomicAdd(t.flops, 2ull * T32 * T32 * (unsigned long long)(k1 - k0));
  const int i0 = ti * T32, j0 = tj * T32;
  for (int kk = k0; kk < k1; kk += T32) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = ty + 8 * q;
      if (!t.ta)
        As[r][tx] = t.A[(int64_t)(i0 + r) * t.lda + kk + tx];
      else
        As[tx][r] = t.A[(int64_t)(kk + r) * t.lda + i0 + tx];
      if (!t.tb)
        Bs[r][tx] = t.B[(int64_t)(kk + r) * t.ldb + j0 + tx];
      else
        Bs[tx][r] = t.B[(int64_t)(j0 + r) * t.ldb + kk + tx];
    }
    __syncthreads();
#pragma unroll 8
    for (int p = 0; p < T32; ++p) {
      const double b = Bs[p][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fma(As[ty + 8 * q][p], b, acc[q]);
    }
    __syncthreads();
  }
  if (splits > 1) {
    __shared__ int s_last;
    const int64_t tile = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    double* mine = part + (tile * splits + blockIdx.z) * (T32 * T32);
#pragma unroll
    for (int q = 0; q < 4; ++q) mine[(ty + 8 * q) * T32 + tx] = acc[q];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&cnt[tile], 1u) == (unsigned)splits - 1u) ? 1 : 0;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double v = 0.0;
      for (int z = 0; z < splits; ++z) v += __ldcg(part + (tile * splits + z) * (T32 * T32) + (ty + 8 * q) * T32 + tx);
      acc[q] = v;
    }
    if (threadIdx.x == 0) cnt[tile] = 0u;  // ready for the next launch
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double* c = t.C + (int64_t)(i0 + ty + 8 * q) * t.ldc + j0 + tx;
    *c = (t.beta != 0.0) ? t.alpha * acc[q] + t.beta * *c : t.alpha * acc[q];
  }
}

// ---------------------------------------------------------------------------
// batched Cholesky of one 32 x 32 diagonal tile (in place) and its inverse
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_bpotrf(const PotrfTask* __restrict__ tasks, int ld_all, int* status) {
  const PotrfTask t = tasks[blockIdx.x];
  const int ld = t.ld > 0 ? t.ld : ld_all;
  __shared__ double T[T32][T32 + 1];
  __shared__ double I[T32][T32 + 1];
  __shared__ double rd[T32];   // reciprocals of the factor's diagonal
  __shared__ int s_drop[T32];
  const int tid = threadIdx.x;
  for (int e = tid; e < T32 * T32; e += blockDim.x) T[e / T32][e % T32] = t.A[(int64_t)(e / T32) * ld + e % T32];
  __syncthreads();
  for (int j = 0; j < T32; ++j) {
    if (tid == 0) {
      const double d = T[j][j], d0 = t.diag0[j];
      int drop = 0;
      if (!(d > 1e-9 * d0)) {
        if (!(d > -1e-6 * d0)) atomicOr(status, 2);  // clearly negative: K_0 not SPD
        drop = 1;
        T[j][j] = 1.0;
        rd[j] = 0.0;   // the column below a dropped pivot becomes zero
      } else {
        const double r = sqrt(d);
        T[j][j] = r;
        rd[j] = 1.0 / r;
      }
      s_drop[j] = drop;
    }
    __syncthreads();
    const double rj = rd[j];
    const bool dropj = s_drop[j] != 0;
    for (int i = j + 1 + tid; i < T32; i += blockDim.x) T[i][j] = dropj ? 0.0 : T[i][j] * rj;
    __syncthreads();
    const int m = T32 - j - 1;
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int i = j + 1 + e / m, c = j + 1 + e % m;
      if (c <= i) T[i][c] = fma(-T[i][j], T[c][j], T[i][c]);
    }
    __syncthreads();
  }
  // inverse of the lower triangle by forward substitution, column c by the 8
  // lanes (tid & 7) of its group: I[i][c] = -(sum_{m=c}^{i-1} T[i][m] I[m][c]) / T[i][i]
  for (int i = tid; i < T32; i += blockDim.x) rd[i] = 1.0 / T[i][i];
  __syncthreads();
  {
    const int c = tid >> 3, part = tid & 7;
    for (int i = 0; i < T32; ++i) {
      double s = 0.0;
      if (i > c)
        for (int mm = c + part; mm < i; mm += 8) s = fma(T[i][mm], I[mm][c], s);
      s += __shfl_xor_sync(0xffffffffu, s, 4);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      if (part == 0) I[i][c] = (i < c) ? 0.0 : (i == c) ? rd[c] : -s * rd[i];
      __syncwarp();
    }
  }
  __syncthreads();
  // rows of dropped DOFs are zeroed (the factor's column below a dropped
  // pivot is zero, so no other row uses them)
  for (int e = tid; e < T32 * T32; e += blockDim.x) {
    const int i = e / T32, c = e % T32;
    t.A[(int64_t)i * ld + c] = (c <= i) ? T[i][c] : 0.0;
    t.Linv[e] = s_drop[i] ? 0.0 : I[i][c];
  }
  if (tid < T32) t.dropped[tid] = s_drop[tid];
}

// the 32 x 32 inverse tiles become the diagonal tiles of W = L^{-1}
__global__ void k_bdiag_tiles(double* const* __restrict__ W, const double* const* __restrict__ Linv, int cw) {
  const int line = blockIdx.y, tile = blockIdx.x;
  double* w = W[line] + (int64_t)tile * T32 * cw + tile * T32;
  const double* s = Linv[line] + (int64_t)tile * T32 * T32;
  for (int e = threadIdx.x; e < T32 * T32; e += blockDim.x) w[(int64_t)(e / T32) * cw + e % T32] = s[e];
}

__global__ void k_get_diag(const double* __restrict__ A, int ld, int n, double* __restrict__ d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = A[(int64_t)i * ld + i];
}

// ---------------------------------------------------------------------------
// solve stage: out[i] = base[i] + sgn * (op(M0) v0 + op(M1) v1)[i]
// ---------------------------------------------------------------------------
template <class TM>
struct BcrTaskT {
  double* out;
  float* out32;         // optional FP32 copy of out (the coarse solution in the mixed path)
  const double* base;   // may be null
  const TM* M0;
  const double* v0;
  const TM* M1;         // may be null
  const double* v1;
  int rows, n0, n1;
  int trans;            // 0: (M v)[i] = sum_c M[i][c] v[c];  1: (M^T v)[i] = sum_a M[a][i] v[a]
  double sgn;
};
struct BcrTask : BcrTaskT<double> {};
struct BcrTask32 : BcrTaskT<float> {};

__device__ __forceinline__ void cf_cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}

// One CTA per BR = 16 outputs of one task.  Stages are chained with
// programmatic dependent launch: a stage CTA starts while the previous stage
// still runs, copies its matrix slice (16 rows, or 16 columns, of M0 and M1;
// the matrices are fixed after setup) into shared memory with 16-byte
// asynchronous copies, and only then waits for the previous grid
// (griddepcontrol.wait), whose results it reads as input vectors.  Row form:
// 16 lanes per output.  Transposed form: 16 consecutive outputs, 16 row
// groups reduced in shared memory.  FP64 path: FP64 arithmetic; mixed path:
// FP32 matrices and products, FP64 result.  stage_mats = 0 (very wide lines)
// reads the matrices from global memory instead.
template <class TM>
__global__ void __launch_bounds__(256) k_bcr_stage(const BcrTaskT<TM>* __restrict__ tasks, const int2* __restrict__ cta,
                                                   int ld, int stage_mats, const int* done) {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  extern __shared__ __align__(16) unsigned char bcr_sm[];
  constexpr int E = 16 / sizeof(TM);  // elements per 16-byte copy
  const int2 cr = cta[blockIdx.x];
  const BcrTaskT<TM> t = tasks[cr.x];
  const int row0 = cr.y;
  const int tid = threadIdx.x;
  const int n1 = t.M1 ? t.n1 : 0;
  const int n0p = (t.n0 + E - 1) / E * E, n1p = (n1 + E - 1) / E * E;
  TM* vs = reinterpret_cast<TM*>(bcr_sm);
  TM* ms0 = vs + 2 * ld;
  TM* ms1 = ms0 + 16 * n0p;
  if (stage_mats) {
    if (!t.trans) {
      const int c0 = n0p / E, c1 = n1p / E;
      for (int c = tid; c < 16 * c0; c += blockDim.x) {
        const int r = c / c0, q = c % c0;
        if (row0 + r < t.rows) cf_cp_async16(ms0 + r * n0p + q * E, t.M0 + (int64_t)(row0 + r) * ld + q * E);
      }
      for (int c = tid; c < 16 * c1; c += blockDim.x) {
        const int r = c / c1, q = c % c1;
        if (row0 + r < t.rows) cf_cp_async16(ms1 + r * n1p + q * E, t.M1 + (int64_t)(row0 + r) * ld + q * E);
      }
    } else {
      constexpr int CPR = 16 / E;  // copies per matrix row slice of 16 outputs
      for (int c = tid; c < t.n0 * CPR; c += blockDim.x) {
        const int a = c / CPR, q = c % CPR;
        cf_cp_async16(ms0 + a * 16 + q * E, t.M0 + (int64_t)a * ld + row0 + q * E);
      }
      for (int c = tid; c < n1 * CPR; c += blockDim.x) {
        const int a = c / CPR, q = c % CPR;
        cf_cp_async16(ms1 + a * 16 + q * E, t.M1 + (int64_t)a * ld + row0 + q * E);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::);
  }
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  const bool stop = done && *done;
  if (!stop) {
    for (int c = tid; c < t.n0; c += blockDim.x) vs[c] = (TM)t.v0[c];
    for (int c = tid; c < n1; c += blockDim.x) vs[n0p + c] = (TM)t.v1[c];
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  if (stop) return;
  const TM* w0 = vs;
  const TM* w1 = vs + n0p;
  if (!t.trans) {
    const int r = tid / 16, i = row0 + r, part = tid % 16;
    TM s = 0;
    if (i < t.rows) {
      const TM* m0 = stage_mats ? ms0 + r * n0p : t.M0 + (int64_t)i * ld;
      for (int c = part; c < t.n0; c += 16) s = fma(m0[c], w0[c], s);
      if (n1) {
        const TM* m1 = stage_mats ? ms1 + r * n1p : t.M1 + (int64_t)i * ld;
        for (int c = part; c < n1; c += 16) s = fma(m1[c], w1[c], s);
      }
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (part == 0 && i < t.rows) {
      const double o = (t.base ? t.base[i] : 0.0) + t.sgn * (double)s;
      t.out[i] = o;
      if (t.out32) t.out32[i] = (float)o;
    }
  } else {
    __shared__ TM red[16][17];
    const int il = tid % 16, i = row0 + il, part = tid / 16;
    TM s = 0;
    if (i < t.rows) {
      if (stage_mats) {
        for (int a = part; a < t.n0; a += 16) s = fma(ms0[a * 16 + il], w0[a], s);
        for (int a = part; a < n1; a += 16) s = fma(ms1[a * 16 + il], w1[a], s);
      } else {
        for (int a = part; a < t.n0; a += 16) s = fma(t.M0[(int64_t)a * ld + i], w0[a], s);
        for (int a = part; a < n1; a += 16) s = fma(t.M1[(int64_t)a * ld + i], w1[a], s);
      }
    }
    red[part][il] = s;
    __syncthreads();
    if (tid < 16) {
      const int o = row0 + tid;
      TM v = 0;
#pragma unroll
      for (int q = 0; q < 16; ++q) v += red[q][tid];
      if (o < t.rows) {
        const double ov = (t.base ? t.base[o] : 0.0) + t.sgn * (double)v;
        t.out[o] = ov;
        if (t.out32) t.out32[o] = (float)ov;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Block solve stage over TS_NB columns (mixed precision): the tasks of the
// one-column stages on block vectors [n][TS_NB], FP32 matrices, input
// vectors and products, the result in FP64 and FP32.  A CTA forms BRB = 32
// outputs of a task for every column, so each stored matrix entry is read
// once for all columns.  Its slice of M streams through a ring of BDEPTH
// shared-memory tiles of BCK reduction indices, each filled by one tiled
// tensor copy (TMA, a 3D tensor map over the stored [lines][cw][cw] array)
// and a bulk copy of the matching rows of the input vector, completing on one
// mbarrier per tile, which run ahead of the arithmetic.
//   Row form (out = M v): a tile is 32 rows x BCK columns of M; warp w takes
//   rows 4w .. 4w+3, its lanes four columns each, every lane all TS_NB sums;
//   one butterfly per warp at the end.
//   Transposed form (out = M^T v): a tile is BCK rows x the 32 columns of M
//   whose outputs the CTA forms; warp w takes rows 16w .. 16w+15 of it, lane
//   l output l; the 8 warps' sums are added through shared memory in order.
// ---------------------------------------------------------------------------
constexpr int BRB = 32, BCK = 128, BDEPTH = 3;
constexpr int BTILE = BRB * BCK + BCK * TS_NB;  // a tile of M and its rows of v (floats)

__device__ __forceinline__ void bfma8(float (&acc)[TS_NB], float m, const float4 v0, const float4 v1) {
  acc[0] = fmaf(m, v0.x, acc[0]); acc[1] = fmaf(m, v0.y, acc[1]);
  acc[2] = fmaf(m, v0.z, acc[2]); acc[3] = fmaf(m, v0.w, acc[3]);
  acc[4] = fmaf(m, v1.x, acc[4]); acc[5] = fmaf(m, v1.y, acc[5]);
  acc[6] = fmaf(m, v1.z, acc[6]); acc[7] = fmaf(m, v1.w, acc[7]);
}

struct BcrMaps {
  CUtensorMap m[6];
};

__global__ void __launch_bounds__(256, 3) k_bbcr_stage(const BcrTaskB* __restrict__ tasks,
                                                       const int2* __restrict__ cta, int ld, const int* done,
                                                       int* status, const __grid_constant__ BcrMaps maps) {
  extern __shared__ __align__(128) float tile[];  // [BDEPTH][BTILE]
  __shared__ __align__(8) uint64_t bar[BDEPTH];
  __shared__ float red[8][BRB][TS_NB + 1];
  const int2 cr = cta[blockIdx.x];
  const BcrTaskB t = tasks[cr.x];
  const int row0 = cr.y, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) {
    for (int q = 0; q < BDEPTH; ++q) mbar_init(bar + q, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  if (done && *done) return;  // (no copy issued yet)
  const int n1 = (t.m1_map >= 0) ? t.n1 : 0;
  const int c0 = (t.n0 + BCK - 1) / BCK, c1 = (n1 + BCK - 1) / BCK, nch = c0 + c1;
  // chunk k: matrix (map, line), first reduction index a0
  auto chunk = [&](int k, int& map, int& line, int& n, int& a0) {
    const bool second = k >= c0;
    map = second ? t.m1_map : t.m0_map;
    line = second ? t.m1_line : t.m0_line;
    n = second ? n1 : t.n0;
    a0 = (second ? k - c0 : k) * BCK;
  };
  // thread 0 fills tile k % BDEPTH with chunk k: one tiled tensor copy (a
  // box of BRB x BCK or BCK x BRB FP32 entries; entries past the array edge
  // arrive as zeros)
  auto issue = [&](int k) {
    if (tid != 0 || k >= nch) return;
    int map, line, n, a0;
    chunk(k, map, line, n, a0);
    float* dst = tile + (k % BDEPTH) * BTILE;
    uint64_t* b = bar + k % BDEPTH;
    const CUtensorMap* tm = &maps.m[map + (t.trans ? 3 : 0)];
    const int x = t.trans ? row0 : a0, y = t.trans ? a0 : row0;
    // the chunk's rows of the input vector ride along: [min(BCK, n - a0)][TS_NB]
    const float* v = (k >= c0) ? t.v1 : t.v0;
    const uint32_t vbytes = (uint32_t)(min(BCK, n - a0) * TS_NB * sizeof(float));
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect(b, (uint32_t)(BRB * BCK * sizeof(float)) + vbytes);
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(line), "r"(smem_u32(b))
        : "memory");
    bulk_copy(dst + BRB * BCK, v + (int64_t)a0 * TS_NB, vbytes, b);
  };
  for (int k = 0; k < BDEPTH; ++k) issue(k);
  float acc[4][TS_NB];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int c = 0; c < TS_NB; ++c) acc[q][c] = 0.f;
  const int hf = (lane >> 2) & 1;  // row form: this lane's first vector half
  for (int k = 0; k < nch; ++k) {
    int map, line, n, a0;
    chunk(k, map, line, n, a0);
    mbar_wait(bar + k % BDEPTH, (uint32_t)((k / BDEPTH) & 1), status);
    const float* T = tile + (k % BDEPTH) * BTILE;
    const float4* v = reinterpret_cast<const float4*>(T + BRB * BCK);  // two float4 per row, row a at v + 2 (a - a0)
    if (!t.trans) {
      // lane l takes the reduction indices a0 + l + 32 u: the warp's reads of
      // a matrix row are consecutive words, and its reads of the vector rows
      // (32 bytes each) are conflict-free because lanes 4..7 of every group
      // of eight read the two 16-byte halves of their row in the opposite
      // order (hf); their accumulator halves are swapped back at the end.
      // Rows past t.rows hold stale tile data: their sums are never written.
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int a = a0 + lane + 32 * u;
        if (a >= n) break;
        const float4 vh = v[2 * (a - a0) + hf], vl = v[2 * (a - a0) + (hf ^ 1)];
#pragma unroll
        for (int q = 0; q < 4; ++q) bfma8(acc[q], T[(4 * wid + q) * BCK + lane + 32 * u], vh, vl);
      }
    } else {
#pragma unroll 4
      for (int r = 16 * wid; r < 16 * wid + 16; ++r) {
        const int a = a0 + r;
        if (a >= n) break;
        const float4 v0 = v[2 * r], v1 = v[2 * r + 1];
        bfma8(acc[0], T[r * BRB + lane], v0, v1);
      }
    }
    __syncthreads();  // every warp is done with the tile
    issue(k + BDEPTH);
  }
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  if (!t.trans) {
    // columns 4..7 came first in the lanes with hf = 1
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < TS_NB / 2; ++c) {
        const float lo = acc[q][c], hi = acc[q][c + TS_NB / 2];
        acc[q][c] = hf ? hi : lo;
        acc[q][c + TS_NB / 2] = hf ? lo : hi;
      }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < TS_NB; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[q][c] += __shfl_xor_sync(0xffffffffu, acc[q][c], o);
    // lane l writes (row l / 8, column l % 8) of the warp's four rows
    const int q = lane / TS_NB, c = lane % TS_NB, i = row0 + 4 * wid + q;
    float sv = 0.f;
#pragma unroll
    for (int qq = 0; qq < 4; ++qq)
#pragma unroll
      for (int cc = 0; cc < TS_NB; ++cc)
        if (qq == q && cc == c) sv = acc[qq][cc];
    if (i < t.rows) {
      const int64_t o = (int64_t)i * TS_NB + c;
      const double ov = (t.base ? t.base[o] : 0.0) + t.sgn * (double)sv;
      t.out[o] = ov;
      t.out32[o] = (float)ov;
    }
  } else {
#pragma unroll
    for (int c = 0; c < TS_NB; ++c) red[wid][lane][c] = acc[0][c];
    __syncthreads();
    const int il = tid / TS_NB, c = tid % TS_NB, i = row0 + il;
    float sv = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) sv += red[w][il][c];
    if (i < t.rows) {
      const int64_t o = (int64_t)i * TS_NB + c;
      const double ov = (t.base ? t.base[o] : 0.0) + t.sgn * (double)sv;
      t.out[o] = ov;
      t.out32[o] = (float)ov;
    }
  }
}

__global__ void k_cf_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
void tiles_gemm(ts_handle h, const std::vector<GemmTask>& ts, TileScratch& sc) {
  if (ts.empty()) return;
  std::vector<GemmTask> tc(ts);
  for (GemmTask& t : tc) t.flops = h->cfac_cnt;
  GemmTask* d = supload(h, tc);
  int tiles = 0, min_kt = 1 << 30;
  bool alias = false;
  for (const GemmTask& t : ts) {
    if (t.m % T32 || t.n % T32 || t.k % T32 || t.m <= 0 || t.n <= 0 || t.k <= 0)
      throw TsError(TS_ERR_INVALID, "internal: batched GEMM shape not a positive multiple of 32");
    tiles = std::max(tiles, (t.m / T32) * (t.n / T32));
    min_kt = std::min(min_kt, t.k / T32);
    alias = alias || t.C == t.A || t.C == t.B;
  }
  if (ts.size() > 65535) throw TsError(TS_ERR_INVALID, "internal: too many batched GEMM tasks");
  // launches with fewer output tiles than 4 resident CTAs per SM split k
  const int64_t ctas = (int64_t)tiles * (int64_t)ts.size();
  const int64_t want = 4LL * h->ctx->n_sm;
  int splits = 1;
  if (!alias && min_kt >= 4 && ctas < want)
    splits = (int)std::min<int64_t>({8, (want + ctas - 1) / ctas, (int64_t)min_kt / 2});
  if (splits > 1) {
    if (ctas * splits > sc.part_tiles) {
      sc.part_tiles = ctas * splits;
      sc.part = salloc<double>(h, (size_t)sc.part_tiles * T32 * T32);
    }
    if (ctas > sc.cnt_tiles) {
      sc.cnt_tiles = ctas;
      sc.cnt = salloc<unsigned>(h, (size_t)sc.cnt_tiles);
      TS_CUDA(cudaMemsetAsync(sc.cnt, 0, sizeof(unsigned) * (size_t)sc.cnt_tiles, h->ctx->stream));
    }
  }
  tsl(h), k_bgemm<<<dim3(tiles, (unsigned)ts.size(), (unsigned)splits), 256, 0, h->ctx->stream>>>(
      d, splits > 1 ? sc.part : nullptr, splits > 1 ? sc.cnt : nullptr);
  TS_CUDA(cudaGetLastError());
}

void tiles_potrf(ts_handle h, const std::vector<PotrfTask>& ts) {
  if (ts.empty()) return;
  PotrfTask* d = supload(h, ts);
  h->cfac_flops += (double)ts.size() * T32 * T32 * T32;  // Cholesky (n^3/3 FMA) and triangular inverse (n^3/6 FMA)
  tsl(h), k_bpotrf<<<(unsigned)ts.size(), 256, 0, h->ctx->stream>>>(d, 0, h->dstatus);
  TS_CUDA(cudaGetLastError());
}

namespace {

struct Level {
  std::vector<int> elim, left, right;        // eliminated lines and their list neighbours (-1: none)
  std::vector<int> remain, jm, jp, rnext;    // remaining lines, eliminated neighbours, next remaining line
};

template <class T>
T* upload_vec(ts_handle h, const std::vector<T>& v) {
  return v.empty() ? nullptr : dupload(h, v);
}

// Batched launches of the setup, issued on the handle's stream.
struct Setup {
  ts_handle h;
  int cw, nt;
  double *Ab, *Wb, *Tb, *Linvb, *diag0;
  int* dropped;

  double* A(int q) const { return Ab + (int64_t)q * cw * cw; }
  double* W(int q) const { return Wb + (int64_t)q * cw * cw; }
  double* T(int q) const { return Tb + (int64_t)q * T32 * cw; }
  double* Linv(int q, int kb) const { return Linvb + ((int64_t)q * nt + kb) * T32 * T32; }

  // split-k scratch: partial tiles and per-tile arrival counters (zeroed
  // once; the last slice of a tile resets its counter)
  TileScratch sc;

  void gemm(const std::vector<GemmTask>& ts) {
    for (const GemmTask& t : ts)
      if ((t.m / T32) * (t.n / T32) != (ts[0].m / T32) * (ts[0].n / T32))
        throw TsError(TS_ERR_INVALID, "internal: mismatched batched GEMM shapes");
    tiles_gemm(h, ts, sc);
  }

  // Cholesky, W = L^{-1} and Ainv = W^T W of the diagonal blocks of the given lines
  void invert(const std::vector<int>& lines, double* Ainv_base) {
    if (lines.empty()) return;
    cudaStream_t st = h->ctx->stream;
    const int nl = (int)lines.size();
    for (int kb = 0; kb < nt; ++kb) {
      std::vector<PotrfTask> pt;
      for (int q : lines)
        pt.push_back(PotrfTask{A(q) + (int64_t)kb * T32 * cw + kb * T32, Linv(q, kb), diag0 + (int64_t)q * cw + kb * T32,
                               dropped + (int64_t)q * cw + kb * T32});
      for (PotrfTask& t : pt) t.ld = cw;
      tiles_potrf(h, pt);
      const int rest = nt - kb - 1;
      if (rest == 0) break;
      std::vector<GemmTask> tr, sy;
      for (int q : lines) {
        double* panel = A(q) + (int64_t)(kb + 1) * T32 * cw + kb * T32;
        // panel <- panel Linv^T (in place: k = 32)
        tr.push_back(GemmTask{panel, Linv(q, kb), panel, rest * T32, T32, T32, cw, T32, cw, 0, 1, 1.0, 0.0, 0});
        // trailing lower tiles -= panel panel^T
        double* trail = A(q) + (int64_t)(kb + 1) * T32 * cw + (kb + 1) * T32;
        sy.push_back(GemmTask{panel, panel, trail, rest * T32, rest * T32, T32, cw, cw, cw, 0, 1, -1.0, 1.0, 1});
      }
      gemm(tr);
      gemm(sy);
    }
    // W = L^{-1}: diagonal tiles, then block row i from the rows above it
    {
      std::vector<double*> wp, lp;
      for (int q : lines) {
        wp.push_back(W(q));
        lp.push_back(Linv(q, 0));
      }
      double** dw = supload(h, wp);
      double** dl = supload(h, lp);
      for (int q : lines) TS_CUDA(cudaMemsetAsync(W(q), 0, sizeof(double) * (size_t)cw * cw, st));
      tsl(h), k_bdiag_tiles<<<dim3(nt, nl), 256, 0, st>>>(dw, (const double* const*)dl, cw);
      TS_CUDA(cudaGetLastError());
    }
    for (int i = 1; i < nt; ++i) {
      std::vector<GemmTask> g1, g2;
      for (int q : lines) {
        // T = L[i, 0:i] W[0:i, 0:i]
        g1.push_back(GemmTask{A(q) + (int64_t)i * T32 * cw, W(q), T(q), T32, i * T32, i * T32, cw, cw, cw, 0, 0, 1.0,
                              0.0, 4});
        // W[i, 0:i] = -Linv_ii T
        g2.push_back(GemmTask{Linv(q, i), T(q), W(q) + (int64_t)i * T32 * cw, T32, i * T32, T32, T32, cw, cw, 0, 0,
                              -1.0, 0.0, 0});
      }
      gemm(g1);
      gemm(g2);
    }
    std::vector<GemmTask> gi;
    for (int q : lines)
      gi.push_back(GemmTask{W(q), W(q), Ainv_base + (int64_t)q * cw * cw, cw, cw, cw, cw, cw, cw, 1, 0, 1.0, 0.0, 2});
    gemm(gi);
  }
};

}  // namespace

// A 3D tiled tensor map over an FP32 array [nl][cw][cw] (x: column, y: row,
// z: line) with boxes of bx columns x by rows; entries past the edges read as
// zeros.
static void encode_stage_map(unsigned char* out, const float* base, int cw, int nl, int bx, int by) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  static cudaError_t err = cudaSuccess;
  std::call_once(once, []() {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    err = cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q);
    if (err == cudaSuccess && q != cudaDriverEntryPointSuccess) err = cudaErrorNotSupported;
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  TS_CUDA(err);
  const cuuint64_t dims[3] = {(cuuint64_t)cw, (cuuint64_t)cw, (cuuint64_t)nl};
  const cuuint64_t strides[2] = {(cuuint64_t)cw * sizeof(float), (cuuint64_t)cw * cw * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(reinterpret_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base),
                  dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw TsError(TS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
}

void coarse_line_layout(ts_handle h) {
  const int nc = h->nc;
  const bool dense = (h->opt.coarse_layout == 1) || (h->opt.coarse_layout == 0 && nc <= DENSE_MAX);
  h->cl_off.clear();
  h->cl_wid.clear();
  h->cl_line.clear();
  if (dense) {
    h->cl_off = {0};
    h->cl_wid = {nc};
    h->cl_line = {-1};
  } else {
    const std::vector<int>& lo = h->line_off_h;
    for (int k = 0; k + 1 < (int)lo.size(); ++k)
      if (lo[k + 1] > lo[k]) {
        h->cl_off.push_back(lo[k]);
        h->cl_wid.push_back(lo[k + 1] - lo[k]);
        h->cl_line.push_back(k);
      }
  }
  int wmax = 0;
  for (int w : h->cl_wid) wmax = std::max(wmax, w);
  h->cw = ((wmax + T32 - 1) / T32) * T32;
  h->coarse_blockline = !dense;
  h->bcr_lines = (int)h->cl_off.size();
}

// unit diagonal on the padding rows of the diagonal blocks (the padded
// unknowns decouple and stay zero)
__global__ void k_unit_pad(double* __restrict__ A, const int* __restrict__ wid, int cw) {
  const int q = blockIdx.y;
  const int w = wid[q];
  for (int i = w + blockIdx.x * blockDim.x + threadIdx.x; i < cw; i += gridDim.x * blockDim.x)
    A[(int64_t)q * cw * cw + (int64_t)i * cw + i] = 1.0;
}

bool coarse_needs_fp64(ts_handle h) {
  // contrast E0 / Emin above 1e6 (a contrast of exactly 1e6, however rounded, stays FP32)
  return h->opt.precision != TS_FP64 && h->opt.coarse_method == 2 && h->E0 > 1.000001e6 * h->Emin;
}

void build_coarse_factor(ts_handle h) {
  h->nd.reset();
  h->coarse64 = coarse_needs_fp64(h);
  if (coarse_uses_nd(h)) {
    build_coarse_factor_nd(h);
    return;
  }
  cudaStream_t st = h->ctx->stream;
  const int nc = h->nc;
  h->coarse_dropped = 0;
  const std::vector<int>& off = h->cl_off;
  const std::vector<int>& wid = h->cl_wid;
  const std::vector<int>& cline = h->cl_line;
  const int nl = (int)off.size();
  const int cw = h->cw;
  // the algorithmic work of the step: block-tridiagonal Cholesky by lines,
  // per line its Cholesky (w^3/3 multiply-adds), L^{-1} times the coupling
  // to the next line (w^2 w'/2) and the Schur update of the next line
  // (w'^2 w/2), FMA = 2 FLOP
  h->cfac_method_flops = 0.0;
  for (int q = 0; q < nl; ++q) {
    const double w = wid[q], wn = (q + 1 < nl) ? wid[q + 1] : 0.0;
    h->cfac_method_flops += 2.0 * (w * w * w / 3.0 + w * w * wn / 2.0 + wn * wn * w / 2.0);
  }
  const int64_t cc = (int64_t)cw * cw;
  // level structure
  std::vector<Level> levels;
  std::vector<int> list(nl);
  for (int q = 0; q < nl; ++q) list[q] = q;
  while (list.size() > 1) {
    Level L;
    const int n = (int)list.size();
    for (int p = 0; p < n; ++p) {
      if (p & 1) {
        L.elim.push_back(list[p]);
        L.left.push_back(list[p - 1]);
        L.right.push_back(p + 1 < n ? list[p + 1] : -1);
      } else {
        L.remain.push_back(list[p]);
        L.jm.push_back(p >= 1 ? list[p - 1] : -1);
        L.jp.push_back(p + 1 < n ? list[p + 1] : -1);
        L.rnext.push_back(p + 2 < n ? list[p + 2] : -1);
      }
    }
    std::vector<int> next;
    for (int p = 0; p < n; p += 2) next.push_back(list[p]);
    list.swap(next);
    levels.push_back(std::move(L));
  }
  const int last = list[0];
  // storage
  Setup S{h, cw, cw / T32, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  S.Ab = h->K0A;  // assembled in place (ts_cbasis.cu); factored in place
  S.Wb = salloc<double>(h, (size_t)nl * cc);
  S.Tb = salloc<double>(h, (size_t)nl * T32 * cw);
  S.Linvb = salloc<double>(h, (size_t)nl * S.nt * T32 * T32);
  S.diag0 = salloc<double>(h, (size_t)nl * cw);
  S.dropped = salloc<int>(h, (size_t)nl * cw);
  h->bcr_Ainv = dalloc<double>(h, (size_t)nl * cc);
  double *Cin = nullptr, *Cout = nullptr;
  if (nl > 1) {
    h->bcr_Qlt = dalloc<double>(h, (size_t)nl * cc);
    h->bcr_Qrt = dalloc<double>(h, (size_t)nl * cc);
    Cin = h->K0C;
    Cout = salloc<double>(h, (size_t)nl * cc);
    TS_CUDA(cudaMemsetAsync(h->bcr_Qrt, 0, sizeof(double) * (size_t)nl * cc, st));
  }
  TS_CUDA(cudaMemsetAsync(S.dropped, 0, sizeof(int) * (size_t)nl * cw, st));
  // padding of the diagonal blocks, original diagonals
  {
    const int* wd = supload(h, wid);
    tsl(h), k_unit_pad<<<dim3(1, nl), 256, 0, st>>>(S.A(0), wd, cw);
    TS_CUDA(cudaGetLastError());
    for (int q = 0; q < nl; ++q) tsl(h), k_get_diag<<<cdiv(cw, 128), 128, 0, st>>>(S.A(q), cw, cw, S.diag0 + (int64_t)q * cw);
    TS_CUDA(cudaGetLastError());
  }
  // Tiles of the couplings C_q = A_{q,q+1} that can be nonzero: a coarse
  // node couples only to the coarse nodes of the next line within one coarse
  // step in every direction.  rowR[q][ti]: k-tile range of row tile ti;
  // colR[q][tj]: row-tile range of column tile tj (empty: x = nt, y = -1).
  // The first reduction level multiplies by these couplings and skips the
  // zero tiles; later levels see the filled-in Schur couplings.
  int2* rowR_d = nullptr;
  int2* colR_d = nullptr;
  if (nl > 1) {
    const int A = h->line_axis, dim = h->g.dim, nt = S.nt;
    std::vector<int2> rowR((size_t)nl * nt, make_int2(nt, -1)), colR((size_t)nl * nt, make_int2(nt, -1));
    std::vector<std::vector<int>> in_line(nl);
    {
      std::vector<int> q_of(h->n_lines + 1, -1);
      for (int q = 0; q < nl; ++q) q_of[cline[q]] = q;
      for (int l = 0; l < h->n_cnodes; ++l) {
        const CoarseNodeInfo& N = h->cn_h[l];
        if (N.ndof == 0) continue;
        const int q = q_of[N.idx[A]];
        if (q >= 0) in_line[q].push_back(l);
      }
    }
    for (int q = 0; q + 1 < nl; ++q) {
      for (int u : in_line[q])
        for (int v : in_line[q + 1]) {
          const CoarseNodeInfo &U = h->cn_h[u], &Vn = h->cn_h[v];
          bool nb = true;
          for (int d = 0; d < dim; ++d)
            if (std::abs(U.idx[d] - Vn.idx[d]) > 1) nb = false;
          if (!nb) continue;
          const int r0 = U.first_dof - off[q], r1 = r0 + U.ndof - 1;
          const int c0 = Vn.first_dof - off[q + 1], c1 = c0 + Vn.ndof - 1;
          for (int ti = r0 / T32; ti <= r1 / T32; ++ti) {
            int2& r = rowR[(size_t)q * nt + ti];
            r.x = std::min(r.x, c0 / T32);
            r.y = std::max(r.y, c1 / T32);
          }
          for (int tj = c0 / T32; tj <= c1 / T32; ++tj) {
            int2& r = colR[(size_t)q * nt + tj];
            r.x = std::min(r.x, r0 / T32);
            r.y = std::max(r.y, r1 / T32);
          }
        }
    }
    rowR_d = salloc<int2>(h, rowR.size());
    colR_d = salloc<int2>(h, colR.size());
    TS_CUDA(cudaMemcpyAsync(rowR_d, rowR.data(), sizeof(int2) * rowR.size(), cudaMemcpyHostToDevice, st));
    TS_CUDA(cudaMemcpyAsync(colR_d, colR.data(), sizeof(int2) * colR.size(), cudaMemcpyHostToDevice, st));
  }
  auto rowR = [&](int q) { return rowR_d + (int64_t)q * S.nt; };
  auto colR = [&](int q) { return colR_d + (int64_t)q * S.nt; };
  // reduction levels
  bool first_level = true;
  for (const Level& L : levels) {
    S.invert(L.elim, h->bcr_Ainv);
    std::vector<GemmTask> ql, qr, s1, s2, cn;
    for (size_t e = 0; e < L.elim.size(); ++e) {
      const int j = L.elim[e], l = L.left[e], r = L.right[e];
      const double* Aj = h->bcr_Ainv + (int64_t)j * cc;
      ql.push_back(GemmTask{Cin + (int64_t)l * cc, Aj, h->bcr_Qlt + (int64_t)j * cc, cw, cw, cw, cw, cw, cw, 0, 0, 1.0,
                            0.0, 0});
      if (first_level) {  // A = C_l: its row tile's k range
        ql.back().kr = rowR(l);
        ql.back().kr_by = 1;
      }
      if (r >= 0) {
        qr.push_back(GemmTask{Cin + (int64_t)j * cc, Aj, h->bcr_Qrt + (int64_t)j * cc, cw, cw, cw, cw, cw, cw, 1, 0,
                              1.0, 0.0, 0});
        if (first_level) {  // A = C_j^T: the row range of C_j's column tile
          qr.back().kr = colR(j);
          qr.back().kr_by = 1;
        }
      }
    }
    S.gemm(ql);
    S.gemm(qr);
    for (size_t e = 0; e < L.remain.size(); ++e) {
      const int l = L.remain[e], jm = L.jm[e], jp = L.jp[e], rn = L.rnext[e];
      if (jp >= 0) {
        // Ahat_l -= Qlt_jp C_l^T (full block: the lower-tile factor reads only the lower part)
        s1.push_back(GemmTask{h->bcr_Qlt + (int64_t)jp * cc, Cin + (int64_t)l * cc, S.A(l), cw, cw, cw, cw, cw, cw, 0,
                              1, -1.0, 1.0, 1});
        if (first_level) {  // B = C_l^T: the k range of C_l's row tile tj
          s1.back().kr = rowR(l);
          s1.back().kr_by = 2;
        }
        if (rn >= 0) {
          cn.push_back(GemmTask{h->bcr_Qlt + (int64_t)jp * cc, Cin + (int64_t)jp * cc, Cout + (int64_t)l * cc, cw, cw,
                                cw, cw, cw, cw, 0, 0, -1.0, 0.0, 0});
          if (first_level) {  // B = C_jp: the row range of its column tile
            cn.back().kr = colR(jp);
            cn.back().kr_by = 2;
          }
        }
      }
      if (jm >= 0) {
        s2.push_back(GemmTask{h->bcr_Qrt + (int64_t)jm * cc, Cin + (int64_t)jm * cc, S.A(l), cw, cw, cw, cw, cw, cw, 0,
                              0, -1.0, 1.0, 1});
        if (first_level) {  // B = C_jm: the row range of its column tile
          s2.back().kr = colR(jm);
          s2.back().kr_by = 2;
        }
      }
    }
    S.gemm(s1);
    S.gemm(s2);
    S.gemm(cn);
    std::swap(Cin, Cout);
    first_level = false;
  }
  S.invert({last}, h->bcr_Ainv);
  TS_CUDA(cudaGetLastError());

  // solve stages
  std::vector<BcrTask> tasks;
  std::vector<int2> ctas;
  h->bcr_stage_task.clear();
  h->bcr_stage_cta.clear();
  h->bcr_fmas = 0.0;
  h->bcr_ys = dalloc<double>(h, std::max(nc, 1));
  h->bcr_bs = dalloc<double>(h, std::max(nc, 1));
  double* ys = h->bcr_ys;
  double* bs = h->bcr_bs;
  auto begin_stage = [&]() {
    h->bcr_stage_task.push_back((int)tasks.size());
    h->bcr_stage_cta.push_back((int)ctas.size());
  };
  auto add = [&](const BcrTask& t, int stage_task0) {
    const int id = (int)tasks.size() - stage_task0;
    tasks.push_back(t);
    for (int r = 0; r < t.rows; r += BR) ctas.push_back(make_int2(id, r));
    h->bcr_fmas += (double)t.rows * (t.n0 + (t.M1 ? t.n1 : 0));
  };
  const int nlev = (int)levels.size();
  for (int lv = 0; lv < nlev; ++lv) {
    const Level& L = levels[lv];
    begin_stage();
    const int t0 = (int)tasks.size();
    const double* vin = (lv == 0) ? h->r0 : bs;
    for (size_t e = 0; e < L.elim.size(); ++e) {
      const int j = L.elim[e];
      add(BcrTask{ys + off[j], nullptr, nullptr, h->bcr_Ainv + (int64_t)j * cc, vin + off[j], nullptr, nullptr, wid[j],
                  wid[j], 0, 0, 1.0},
          t0);
    }
    for (size_t e = 0; e < L.remain.size(); ++e) {
      const int l = L.remain[e], jm = L.jm[e], jp = L.jp[e];
      BcrTask t{bs + off[l], nullptr, vin + off[l], nullptr, nullptr, nullptr, nullptr, wid[l], 0, 0, 0, -1.0};
      if (jp >= 0) {
        t.M0 = h->bcr_Qlt + (int64_t)jp * cc;
        t.v0 = vin + off[jp];
        t.n0 = wid[jp];
      }
      if (jm >= 0) {
        const double* M = h->bcr_Qrt + (int64_t)jm * cc;
        if (!t.M0) {
          t.M0 = M;
          t.v0 = vin + off[jm];
          t.n0 = wid[jm];
        } else {
          t.M1 = M;
          t.v1 = vin + off[jm];
          t.n1 = wid[jm];
        }
      }
      add(t, t0);
    }
  }
  {
    begin_stage();
    const int t0 = (int)tasks.size();
    const double* vin = (nlev == 0) ? h->r0 : bs;
    add(BcrTask{h->u0 + off[last], h->u0f ? h->u0f + off[last] : nullptr, nullptr, h->bcr_Ainv + (int64_t)last * cc,
                vin + off[last], nullptr, nullptr, wid[last], wid[last], 0, 0, 1.0},
        t0);
  }
  for (int lv = nlev - 1; lv >= 0; --lv) {
    const Level& L = levels[lv];
    begin_stage();
    const int t0 = (int)tasks.size();
    for (size_t e = 0; e < L.elim.size(); ++e) {
      const int j = L.elim[e], l = L.left[e], r = L.right[e];
      BcrTask t{h->u0 + off[j], h->u0f ? h->u0f + off[j] : nullptr, ys + off[j], h->bcr_Qlt + (int64_t)j * cc,
                h->u0 + off[l], nullptr, nullptr, wid[j], wid[l], 0, 1, -1.0};
      if (r >= 0) {
        t.M1 = h->bcr_Qrt + (int64_t)j * cc;
        t.v1 = h->u0 + off[r];
        t.n1 = wid[r];
      }
      add(t, t0);
    }
  }
  h->bcr_stage_task.push_back((int)tasks.size());
  h->bcr_stage_cta.push_back((int)ctas.size());
  h->bcr_tasks = upload_vec(h, tasks);
  h->bcr_ctas = upload_vec(h, ctas);
  h->bcr_tasks32 = nullptr;
  if (h->opt.precision != TS_FP64 && !h->coarse64) {
    // FP32 copies of the (FP64-computed) stage matrices; same task list
    const size_t nA = (size_t)nl * cc, nQ = (nl > 1) ? (size_t)nl * cc : 0;
    float* A32 = dalloc<float>(h, nA);
    float* Ql32 = nQ ? dalloc<float>(h, nQ) : nullptr;
    float* Qr32 = nQ ? dalloc<float>(h, nQ) : nullptr;
    tsl(h), k_cf_to_f32<<<1024, 256, 0, st>>>(h->bcr_Ainv, A32, (int64_t)nA);
    if (nQ) {
      tsl(h), k_cf_to_f32<<<1024, 256, 0, st>>>(h->bcr_Qlt, Ql32, (int64_t)nQ);
      tsl(h), k_cf_to_f32<<<1024, 256, 0, st>>>(h->bcr_Qrt, Qr32, (int64_t)nQ);
    }
    TS_CUDA(cudaGetLastError());
    auto map = [&](const double* p) -> const float* {
      if (!p) return nullptr;
      if (p >= h->bcr_Ainv && p < h->bcr_Ainv + nA) return A32 + (p - h->bcr_Ainv);
      if (nQ && p >= h->bcr_Qlt && p < h->bcr_Qlt + nQ) return Ql32 + (p - h->bcr_Qlt);
      if (nQ && p >= h->bcr_Qrt && p < h->bcr_Qrt + nQ) return Qr32 + (p - h->bcr_Qrt);
      throw TsError(TS_ERR_INVALID, "internal: coarse stage matrix outside the factor");
    };
    std::vector<BcrTask32> t32(tasks.size());
    for (size_t i = 0; i < tasks.size(); ++i) {
      const BcrTask& t = tasks[i];
      BcrTask32& u = t32[i];
      u.out = t.out;
      u.out32 = t.out32;
      u.base = t.base;
      u.M0 = map(t.M0);
      u.v0 = t.v0;
      u.M1 = map(t.M1);
      u.v1 = t.v1;
      u.rows = t.rows;
      u.n0 = t.n0;
      u.n1 = t.n1;
      u.trans = t.trans;
      u.sgn = t.sgn;
    }
    h->bcr_tasks32 = upload_vec(h, t32);
    // the block path's copy of the task list: the same stages and CTAs on
    // block vectors [n][TS_NB]
    if (h->g.dim == 2) {
      const int64_t nb = (int64_t)std::max(nc, 1) * TS_NB;
      const int64_t ldb = (int64_t)h->K0_ld * TS_NB;
      h->r0b = dalloc<double>(h, ldb);
      h->u0b = dalloc<double>(h, ldb);
      h->u0fb = dalloc<float>(h, ldb);
      h->r0b32 = dalloc<float>(h, ldb);
      h->bcr_ysb = dalloc<double>(h, nb);
      h->bcr_bsb = dalloc<double>(h, nb);
      h->bcr_ysb32 = dalloc<float>(h, nb);
      h->bcr_bsb32 = dalloc<float>(h, nb);
      TS_CUDA(cudaMemsetAsync(h->r0b, 0, sizeof(double) * ldb, st));
      TS_CUDA(cudaMemsetAsync(h->u0b, 0, sizeof(double) * ldb, st));
      TS_CUDA(cudaMemsetAsync(h->u0fb, 0, sizeof(float) * ldb, st));
      TS_CUDA(cudaMemsetAsync(h->r0b32, 0, sizeof(float) * ldb, st));
      // a one-column vector pointer -> its block vector (FP64) and FP32 copy
      auto bmap = [&](const double* p, float** p32) -> double* {
        if (!p) {
          if (p32) *p32 = nullptr;
          return nullptr;
        }
        struct V { const double* one; int64_t len; double* b; float* b32; };
        const V vs[4] = {{h->r0, h->K0_ld, h->r0b, h->r0b32}, {h->u0, h->K0_ld, h->u0b, h->u0fb},
                         {ys, std::max(nc, 1), h->bcr_ysb, h->bcr_ysb32}, {bs, std::max(nc, 1), h->bcr_bsb, h->bcr_bsb32}};
        for (const V& x : vs)
          if (p >= x.one && p < x.one + x.len) {
            if (p32) *p32 = x.b32 + (p - x.one) * TS_NB;
            return x.b + (p - x.one) * TS_NB;
          }
        throw TsError(TS_ERR_INVALID, "internal: coarse stage vector outside the solve buffers");
      };
      // tensor maps over the three FP32 stage arrays, row and transposed tiles
      const float* arrays[3] = {A32, Ql32, Qr32};
      for (int a = 0; a < 3; ++a)
        for (int tr = 0; tr < 2; ++tr) {
          if (!arrays[a]) {
            std::memset(h->bcr_tmaps[3 * tr + a], 0, 128);
            continue;
          }
          encode_stage_map(h->bcr_tmaps[3 * tr + a], arrays[a], cw, nl, tr ? BRB : BCK, tr ? BCK : BRB);
        }
      auto mid = [&](const float* m, int& map, int& line) {
        map = -1;
        line = 0;
        if (!m) return;
        for (int a = 0; a < 3; ++a)
          if (arrays[a] && m >= arrays[a] && m < arrays[a] + (int64_t)nl * cc) {
            map = a;
            line = (int)((m - arrays[a]) / cc);
            if ((m - arrays[a]) % cc != 0) break;
            return;
          }
        throw TsError(TS_ERR_INVALID, "internal: coarse stage matrix outside the factor");
      };
      std::vector<BcrTaskB> tb(t32.size());
      for (size_t i = 0; i < t32.size(); ++i) {
        const BcrTask32& u = t32[i];
        BcrTaskB& b = tb[i];
        b.out = bmap(u.out, &b.out32);
        b.base = bmap(u.base, nullptr);
        float* f0 = nullptr;
        float* f1 = nullptr;
        bmap(u.v0, &f0);
        bmap(u.v1, &f1);
        b.v0 = f0;
        b.v1 = f1;
        mid(u.M0, b.m0_map, b.m0_line);
        mid(u.M1, b.m1_map, b.m1_line);
        b.rows = u.rows;
        b.n0 = u.n0;
        b.n1 = u.n1;
        b.trans = u.trans;
        b.sgn = u.sgn;
      }
      h->bcr_btasks = upload_vec(h, tb);
      // CTAs of the block stages: BRB outputs of a task each
      std::vector<int2> bc;
      h->bcr_bstage_cta.clear();
      const int ns = (int)h->bcr_stage_task.size() - 1;
      for (int st2 = 0; st2 < ns; ++st2) {
        h->bcr_bstage_cta.push_back((int)bc.size());
        for (int ti = h->bcr_stage_task[st2]; ti < h->bcr_stage_task[st2 + 1]; ++ti)
          for (int r = 0; r < tasks[ti].rows; r += BRB) bc.push_back(make_int2(ti - h->bcr_stage_task[st2], r));
      }
      h->bcr_bstage_cta.push_back((int)bc.size());
      h->bcr_bctas = upload_vec(h, bc);
    }
  }
  // shared memory of a stage CTA: the two input vectors and, when they fit,
  // the two staged matrix slices (16 x n each), in the element type of the
  // stage matrices the one-column solve applies (FP32 copies, else FP64)
  {
    const size_t es = h->bcr_tasks32 ? sizeof(float) : sizeof(double);
    const size_t with = (size_t)(2 * cw + 32 * cw) * es;
    h->bcr_stage_mats = with <= 110 * 1024;
    h->bcr_smem = h->bcr_stage_mats ? with : (size_t)2 * cw * es;
    const size_t lim = std::min(ts_allow_dynamic_smem(k_bcr_stage<double>, h->ctx->device),
                                ts_allow_dynamic_smem(k_bcr_stage<float>, h->ctx->device));
    if (h->bcr_smem > lim) throw TsError(TS_ERR_INVALID, "coarse line too wide for the coarse solve");
  }
  // dropped coarse DOFs
  std::vector<int> dr((size_t)nl * cw);
  TS_CUDA(cudaMemcpyAsync(dr.data(), S.dropped, sizeof(int) * dr.size(), cudaMemcpyDeviceToHost, st));
  TS_CUDA(cudaStreamSynchronize(st));
  for (int q = 0; q < nl; ++q)
    for (int i = 0; i < wid[q]; ++i) h->coarse_dropped += dr[(size_t)q * cw + i];
}

template <class TM>
static void launch_stage(ts_handle h, const BcrTaskT<TM>* tasks, const int2* ctas, int nct, bool pdl) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3(nct, 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = h->bcr_smem;
  cfg.stream = h->ctx->stream;
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  tsl(h);
  TS_CUDA(cudaLaunchKernelEx(&cfg, k_bcr_stage<TM>, tasks, ctas, h->cw, h->bcr_stage_mats ? 1 : 0,
                             (const int*)h->done_flag));
}

void launch_coarse_solve(ts_handle h) {
  if (h->nd) {
    launch_coarse_solve_nd(h);
    return;
  }
  const int ns = (int)h->bcr_stage_task.size() - 1;
  bool first = true;
  for (int s = 0; s < ns; ++s) {
    const int nct = h->bcr_stage_cta[s + 1] - h->bcr_stage_cta[s];
    if (nct == 0) continue;
    const int2* ctas = h->bcr_ctas + h->bcr_stage_cta[s];
    if (h->bcr_tasks32)
      launch_stage<float>(h, h->bcr_tasks32 + h->bcr_stage_task[s], ctas, nct, !first);
    else
      launch_stage<double>(h, h->bcr_tasks + h->bcr_stage_task[s], ctas, nct, !first);
    first = false;
  }
}

// u0 = K_0^{-1} r0 for the TS_NB columns of the block path (h->r0b -> h->u0b,
// h->u0fb): the stages of launch_coarse_solve with block vectors
void launch_bcoarse_solve(ts_handle h) {
  if (h->nd) {
    launch_bcoarse_solve_nd(h);
    return;
  }
  if (!h->bcr_btasks) throw TsError(TS_ERR_INVALID, "internal: no block coarse solve (mixed 2D designs only)");
  const int ns = (int)h->bcr_stage_task.size() - 1;
  const size_t smem = (size_t)BDEPTH * BTILE * sizeof(float);
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [smem]() {
    attr_err = cudaFuncSetAttribute(k_bbcr_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  TS_CUDA(attr_err);
  BcrMaps maps;
  std::memcpy(&maps, h->bcr_tmaps, sizeof(maps));
  bool first = true;
  for (int s = 0; s < ns; ++s) {
    const int nct = h->bcr_bstage_cta[s + 1] - h->bcr_bstage_cta[s];
    if (nct == 0) continue;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(nct, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = h->ctx->stream;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = first ? 0 : 1;
    tsl(h);
    TS_CUDA(cudaLaunchKernelEx(&cfg, k_bbcr_stage, (const BcrTaskB*)(h->bcr_btasks + h->bcr_stage_task[s]),
                               (const int2*)(h->bcr_bctas + h->bcr_bstage_cta[s]), h->cw, (const int*)h->done_flag,
                               h->dstatus, maps));
    first = false;
  }
}

// algorithmic FLOPs of one coarse solve: one FMA per stored matrix entry used
double coarse_solve_flops(ts_handle h) { return 2.0 * h->bcr_fmas; }
