// Nested-dissection factor and solve of the coarse matrix K_0 = R_0 K R_0^T
// (Sec. 2.1), the FP64 alternative to the block cyclic reduction of
// ts_cfactor.cu for large coarse grids.
//
// K_0 couples a coarse node only to its neighbours (a node's basis functions
// live on omega_l), so its graph is the coarse grid with the 9-point (2D) or
// 27-point (3D) stencil, each node a block of its ndof coarse DOFs.  The grid
// box is split recursively: the middle layer of nodes across its longest axis
// is a separator, the two halves are split in turn; boxes of at most four
// nodes are leaves.  Every separator (or leaf) is the pivot set P of a front
// F; its update set U holds the nodes outside F's box next to it (they lie on
// the separators of F's ancestors).  Fronts are eliminated deepest level
// first (the multifrontal method):
//   assemble   F = [F11 F12; F21 F22] over P u U from the K_0 entries of the
//              rows of P and the children's update matrices (extend-add);
//   factor     F11 = L L^T (dependent pivots dropped as in the reduction),
//              Ainv = F11^{-1} = L^{-T} L^{-1},  Q = F21 Ainv,
//              update matrix S = F22 - Q F12 for the parent.
// Compared with block cyclic reduction over coarse lines -- whose Schur
// complements fill whole lines of width w, O(lines w^3) -- the dense work
// concentrates in the few long separators near the root.
//
// Solve (every level one launch per step, all its fronts at once; stored per
// front Ainv and Q, FP32 copies in the mixed path):
//   forward, deepest level first
//     v_F = [b_P; 0] + children's update vectors (extend-add)
//     w_F = v_U - Q v_P                        (kept in place of v_U)
//   backward, root first
//     x_P = Ainv v_P - Q^T x_U                 (x_U: the ancestors' results)
// Every sum is formed in a fixed order: results do not depend on timing.
#include <algorithm>
#include <cstring>
#include <memory>
#include <vector>

#include "ts_bpcg.cuh"
#include "ts_internal.cuh"
#include "ts_tiles.cuh"

namespace {

constexpr int ND_ROWS = 32;   // outputs per solve CTA
constexpr int ND_THREADS = 256;
constexpr int ND_G8_LP = 512; // rows of at most this many entries: eight lanes per row

// a front as the solve sees it
struct NdFrontD {
  int np, nu;        // pivots and update DOFs
  int lp, lu;        // np and nu rounded up to 4: row lengths of the stored matrices
  int64_t aoff;      // Ainv: np rows of lp (zero past np)
  int64_t qoff;      // Q: nu rows of lp
  int64_t toff;      // Q^T: np rows of lu (zero past nu)
  int64_t voff;      // front vector rows [voff, voff + np + nu)
  int64_t ioff;      // index lists: P at ioff, U at ioff + np (coarse DOFs)
};

// a front of the level being factored
struct NdAsmF {
  int np, nu, npp, nup;          // sizes and their multiples of 32
  int64_t a11, a21, a22, d0;     // offsets in the level buffers
  int64_t ioff;                  // index lists (as NdFrontD)
  int64_t upos;                  // positions of the U entries in the parent front
  int child[2];                  // children (index into the child level's NdAsmF), -1 none
};

// entry (gi, gj) of K_0 from the assembled line blocks (diagonal blocks A and
// couplings C_q = A_{q,q+1}, each cw x cw)
struct K0Lines {
  const double* A;
  const double* C;
  const int* qline;
  const int* qoff;
  int cw;
  __device__ double get(int gi, int gj) const {
    const int qi = qline[gi], qj = qline[gj];
    const int64_t cc = (int64_t)cw * cw;
    if (qi == qj) return A[qi * cc + (int64_t)(gi - qoff[qi]) * cw + (gj - qoff[qj])];
    if (qj == qi + 1) return C[qi * cc + (int64_t)(gi - qoff[qi]) * cw + (gj - qoff[qj])];
    if (qi == qj + 1) return C[qj * cc + (int64_t)(gj - qoff[qj]) * cw + (gi - qoff[qi])];
    return 0.0;
  }
};

// F11 and F21 of every front of the level from K_0 (padding pivots get a unit
// diagonal and decouple), F22 zero, original diagonal entries of the pivots.
__global__ void k_nd_assemble(const NdAsmF* __restrict__ fr, const int* __restrict__ idx, K0Lines K0,
                              double* __restrict__ A11, double* __restrict__ A21, double* __restrict__ A22,
                              double* __restrict__ d0) {
  const NdAsmF F = fr[blockIdx.y];
  const int* pd = idx + F.ioff;
  const int* ud = pd + F.np;
  const int64_t n11 = (int64_t)F.npp * F.npp, n21 = (int64_t)F.nup * F.npp, n22 = (int64_t)F.nup * F.nup;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n11; e += stride) {
    const int i = (int)(e / F.npp), j = (int)(e % F.npp);
    double v;
    if (i < F.np && j < F.np)
      v = K0.get(pd[i], pd[j]);
    else
      v = (i == j) ? 1.0 : 0.0;
    A11[F.a11 + e] = v;
    if (i == j) d0[F.d0 + i] = v;
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n21; e += stride) {
    const int u = (int)(e / F.npp), j = (int)(e % F.npp);
    A21[F.a21 + e] = (u < F.nu && j < F.np) ? K0.get(ud[u], pd[j]) : 0.0;
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n22; e += stride) A22[F.a22 + e] = 0.0;
}

// Extend-add of child slot `slot`'s update matrix (lower triangle stored)
// into its parent: every entry (i, j) of the child's U x U lands at the
// parent positions (pi, pj); F11 takes both triangles, F21 its rows, F22 its
// lower triangle.  Positions within one child are distinct, so the threads
// of a launch never add to the same entry.
__global__ void k_nd_extend(const NdAsmF* __restrict__ fr, const NdAsmF* __restrict__ cfr,
                            const int* __restrict__ upos, const double* __restrict__ cA22, int slot,
                            double* __restrict__ A11, double* __restrict__ A21, double* __restrict__ A22) {
  const NdAsmF F = fr[blockIdx.y];
  if (F.child[slot] < 0) return;
  const NdAsmF C = cfr[F.child[slot]];
  const int* pos = upos + C.upos;
  const int64_t n = (int64_t)C.nu * C.nu;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / C.nu), j = (int)(e % C.nu);
    const double v = cA22[C.a22 + (int64_t)max(i, j) * C.nup + min(i, j)];
    const int pi = pos[i], pj = pos[j];
    if (pi < F.np && pj < F.np)
      A11[F.a11 + (int64_t)pi * F.npp + pj] += v;
    else if (pi >= F.np && pj < F.np)
      A21[F.a21 + (int64_t)(pi - F.np) * F.npp + pj] += v;
    else if (pi >= F.np && pj >= F.np && pi >= pj)
      A22[F.a22 + (int64_t)(pi - F.np) * F.nup + (pj - F.np)] += v;
  }
}

// the 32 x 32 inverse tiles of the factor's diagonal become the diagonal
// tiles of W = L^{-1} (per front: W at a11 offsets, Linv tiles at d0 * 32)
__global__ void k_nd_diag_tiles(const NdAsmF* __restrict__ fr, double* __restrict__ W,
                                const double* __restrict__ Linv) {
  const NdAsmF F = fr[blockIdx.y];
  const int t = blockIdx.x;
  if (t * TILE >= F.npp) return;
  double* w = W + F.a11 + (int64_t)t * TILE * F.npp + t * TILE;
  const double* s = Linv + F.d0 * TILE + (int64_t)t * TILE * TILE;
  for (int e = threadIdx.x; e < TILE * TILE; e += blockDim.x) w[(int64_t)(e / TILE) * F.npp + e % TILE] = s[e];
}

// the solve matrices of the level's fronts: Ainv (np rows of lp), Q (nu rows
// of lp) and Q^T (np rows of lu), zero in the padding columns
template <class T>
__global__ void k_nd_store(const NdAsmF* __restrict__ fr, const NdFrontD* __restrict__ sf, int f0,
                           const double* __restrict__ Ainv, const double* __restrict__ Q, T* __restrict__ As,
                           T* __restrict__ Qs, T* __restrict__ Ts) {
  const NdAsmF F = fr[blockIdx.y];
  const NdFrontD S = sf[f0 + blockIdx.y];
  const int64_t na = (int64_t)F.np * S.lp, nq = (int64_t)F.nu * S.lp, nt = (int64_t)F.np * S.lu;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < na; e += stride) {
    const int64_t i = e / S.lp, j = e % S.lp;
    As[S.aoff + e] = (j < F.np) ? (T)Ainv[F.a11 + i * F.npp + j] : (T)0;
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nq; e += stride) {
    const int64_t u = e / S.lp, j = e % S.lp;
    Qs[S.qoff + e] = (j < F.np) ? (T)Q[F.a21 + u * F.npp + j] : (T)0;
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt; e += stride) {
    const int64_t i = e / S.lu, u = e % S.lu;
    Ts[S.toff + e] = (u < F.nu) ? (T)Q[F.a21 + u * F.npp + i] : (T)0;
  }
}

__global__ void k_nd_count(const NdAsmF* __restrict__ fr, int nf, const int* __restrict__ dropped,
                           int* __restrict__ total) {
  int s = 0;
  for (int f = 0; f < nf; ++f)
    for (int i = threadIdx.x; i < fr[f].np; i += blockDim.x) s += dropped[fr[f].d0 + i];
  s = __reduce_add_sync(0xffffffffu, s);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(total, s);
}

// ---------------------------------------------------------------------------
// solve kernels; NC columns (1, or TS_NB in the block path), T the matrix,
// vector and arithmetic type (FP32 mixed, FP64)
// ---------------------------------------------------------------------------

// front-vector rows of the level: b at the pivots plus the children's update
// vectors, added in child order
template <int NC, class TB, class T>
__global__ void __launch_bounds__(ND_THREADS) k_nd_gather(const int4* __restrict__ grow, int64_t r0, int64_t r1,
                                                         const TB* __restrict__ b, T* __restrict__ v,
                                                         const int* done) {
  pdl_wait();
  if (done && *done) return;
  for (int64_t r = r0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < r1; r += (int64_t)gridDim.x * blockDim.x) {
    const int4 g = grow[r];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T s = (g.x >= 0) ? (T)b[(int64_t)g.x * NC + c] : (T)0;
      if (g.y >= 0) s += v[(int64_t)g.y * NC + c];
      if (g.z >= 0) s += v[(int64_t)g.z * NC + c];
      v[r * NC + c] = s;
    }
  }
  pdl_trigger();
}

// A vector of n rows (NC values each) staged in shared memory for products
// whose lanes take four consecutive rows k = 4 k4 .. 4 k4 + 3 each:
//  NC = 8 (FP32): eight planes of float4, plane (h, s) holding columns
//    4h .. 4h + 3 of the rows k = 4 k4 + s at index k4 -- lanes with
//    consecutive k4 read consecutive 16-byte words;
//  NC = 1: the n values, rows past n zero.
// n4 = ceil(n / 4); rows past n are zero (the matrices' padding columns are
// zero too, and 0 * 0 stays 0).
template <int NC, class T>
__device__ __forceinline__ size_t nd_vec_len(int n) {
  return (size_t)((n + 3) / 4) * 4 * NC;
}

template <int NC, class T, class F>
__device__ __forceinline__ void nd_stage(int n, T* sm, F row) {
  const int n4 = (n + 3) / 4;
  for (int k = threadIdx.x; k < 4 * n4; k += blockDim.x) {
    T y[NC];
    if (k < n) {
      row(k, y);
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) y[c] = (T)0;
    }
    if constexpr (NC == 8) {
      float4* pl = reinterpret_cast<float4*>(sm);
      pl[(0 * 4 + (k & 3)) * n4 + (k >> 2)] = make_float4(y[0], y[1], y[2], y[3]);
      pl[(1 * 4 + (k & 3)) * n4 + (k >> 2)] = make_float4(y[4], y[5], y[6], y[7]);
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) sm[(int64_t)k * NC + c] = y[c];
    }
  }
}

// acc[q][c] += sgn * sum_k M[row_q][k] y_k[c] over the warp's four rows
// (row_q = row0 + q < nrows; M row-major with leading dimension ld, a
// multiple of 4, zero past n): lane l takes k = 4 k4 .. 4 k4 + 3 for
// k4 = l, l + 32, ... as 16-byte loads of each row.  Not reduced over lanes.
template <int NC, class T>
__device__ __forceinline__ void nd_rows4(const T* __restrict__ M, int ld, int n, int row0, int nrows, const T* sm,
                                         T sgn, T (&acc)[4][NC]) {
  const int lane = threadIdx.x & 31, n4 = (n + 3) / 4;
  const T* m[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) m[q] = M + (int64_t)min(row0 + q, max(nrows - 1, 0)) * ld;
#pragma unroll 2
  for (int k4 = lane; k4 < n4; k4 += 32) {
    T mv[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if constexpr (sizeof(T) == 4) {
        const float4 x = (row0 + q < nrows) ? *reinterpret_cast<const float4*>(m[q] + 4 * k4)
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
        mv[q][0] = x.x; mv[q][1] = x.y; mv[q][2] = x.z; mv[q][3] = x.w;
      } else {
        double2 x0 = make_double2(0.0, 0.0), x1 = x0;
        if (row0 + q < nrows) {
          x0 = *reinterpret_cast<const double2*>(m[q] + 4 * k4);
          x1 = *reinterpret_cast<const double2*>(m[q] + 4 * k4 + 2);
        }
        mv[q][0] = x0.x; mv[q][1] = x0.y; mv[q][2] = x1.x; mv[q][3] = x1.y;
      }
      if (sgn < (T)0)
#pragma unroll
        for (int s = 0; s < 4; ++s) mv[q][s] = -mv[q][s];
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      T y[NC];
      if constexpr (NC == 8) {
        const float4* pl = reinterpret_cast<const float4*>(sm);
        const float4 a = pl[(0 * 4 + s) * n4 + k4], b = pl[(1 * 4 + s) * n4 + k4];
        y[0] = a.x; y[1] = a.y; y[2] = a.z; y[3] = a.w;
        y[4] = b.x; y[5] = b.y; y[6] = b.z; y[7] = b.w;
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) y[c] = sm[(int64_t)(4 * k4 + s) * NC + c];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[q][c] = fma(mv[q][s], y[c], acc[q][c]);
    }
  }
}

template <int NC, class T>
__device__ __forceinline__ void nd_reduce4(T (&acc)[4][NC]) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[q][c] += __shfl_xor_sync(0xffffffffu, acc[q][c], o);
}

// the lane's share of the warp's four-row result: lane q * NC + c holds
// (row q, column c); returns false for lanes without one
template <int NC, class T>
__device__ __forceinline__ bool nd_pick(const T (&acc)[4][NC], int lane, int& q, int& c, T& val) {
  if (lane >= 4 * NC) return false;
  q = lane / NC;
  c = lane % NC;
  val = (T)0;
#pragma unroll
  for (int qq = 0; qq < 4; ++qq)
#pragma unroll
    for (int cc = 0; cc < NC; ++cc)
      if (qq == q && cc == c) val = acc[qq][cc];
  return true;
}

// Fronts with few pivots: eight lanes per row (lane group g = lane / 8 takes
// row row0 + g), k4 = lane % 8, lane % 8 + 8, ...; the row's sums are added
// over the eight lanes only (three butterfly steps instead of five for four
// rows per lane).
template <int NC, class T>
__device__ __forceinline__ void nd_row8(const T* __restrict__ M, int ld, int n, int row, int nrows, const T* sm,
                                        T sgn, T (&a)[NC]) {
  if (row >= nrows) return;
  const int n4 = (n + 3) / 4;
  const T* m = M + (int64_t)row * ld;
#pragma unroll 2
  for (int k4 = threadIdx.x & 7; k4 < n4; k4 += 8) {
    T mv[4];
    if constexpr (sizeof(T) == 4) {
      const float4 x = *reinterpret_cast<const float4*>(m + 4 * k4);
      mv[0] = x.x; mv[1] = x.y; mv[2] = x.z; mv[3] = x.w;
    } else {
      const double2 x0 = *reinterpret_cast<const double2*>(m + 4 * k4);
      const double2 x1 = *reinterpret_cast<const double2*>(m + 4 * k4 + 2);
      mv[0] = x0.x; mv[1] = x0.y; mv[2] = x1.x; mv[3] = x1.y;
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const T mm = sgn * mv[s];
      T y[NC];
      if constexpr (NC == 8) {
        const float4* pl = reinterpret_cast<const float4*>(sm);
        const float4 u = pl[(0 * 4 + s) * n4 + k4], w = pl[(1 * 4 + s) * n4 + k4];
        y[0] = u.x; y[1] = u.y; y[2] = u.z; y[3] = u.w;
        y[4] = w.x; y[5] = w.y; y[6] = w.z; y[7] = w.w;
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) y[c] = sm[(int64_t)(4 * k4 + s) * NC + c];
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) a[c] = fma(mm, y[c], a[c]);
    }
  }
}

template <int NC, class T>
__device__ __forceinline__ void nd_reduce8(T (&a)[NC]) {
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) a[c] += __shfl_xor_sync(0xffffffffu, a[c], o);
}

// lane (g, j) with j < NC holds column j of row g's sum
template <int NC, class T>
__device__ __forceinline__ bool nd_pick8(const T (&a)[NC], int lane, int& c, T& val) {
  c = lane & 7;
  if (c >= NC) return false;
  val = (T)0;
#pragma unroll
  for (int cc = 0; cc < NC; ++cc)
    if (cc == c) val = a[cc];
  return true;
}

// forward: w = v_U - Q v_P for ND_ROWS update rows of a front per CTA
template <int NC, class T, int G>
__global__ void __launch_bounds__(ND_THREADS) k_nd_fwd(const NdFrontD* __restrict__ fr, const int2* __restrict__ cta,
                                                      const T* __restrict__ Q, T* __restrict__ v, const int* done) {
  extern __shared__ __align__(16) unsigned char nd_sm[];
  T* sm = reinterpret_cast<T*>(nd_sm);
  pdl_wait();
  if (done && *done) return;
  const int2 cr = cta[blockIdx.x];
  const NdFrontD F = fr[cr.x];
  const T* vp = v + F.voff * NC;
  nd_stage<NC, T>(F.np, sm, [&](int k, T (&y)[NC]) {
#pragma unroll
    for (int c = 0; c < NC; ++c) y[c] = vp[(int64_t)k * NC + c];
  });
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = cr.y + 4 * w;
  if constexpr (G == 8) {
    T a[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) a[c] = (T)0;
    const int r = row0 + (lane >> 3);
    nd_row8<NC, T>(Q + F.qoff, F.lp, F.np, r, F.nu, sm, (T)1, a);
    nd_reduce8<NC, T>(a);
    pdl_trigger();
    int c;
    T s;
    if (nd_pick8<NC, T>(a, lane, c, s) && r < F.nu) {
      T* o = v + (F.voff + F.np + r) * NC + c;
      *o = *o - s;
    }
  } else {
    T acc[4][NC];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[q][c] = (T)0;
    nd_rows4<NC, T>(Q + F.qoff, F.lp, F.np, row0, F.nu, sm, (T)1, acc);
    nd_reduce4<NC, T>(acc);
    pdl_trigger();
    int q, c;
    T s;
    if (nd_pick<NC, T>(acc, lane, q, c, s) && row0 + q < F.nu) {
      T* o = v + (F.voff + F.np + row0 + q) * NC + c;
      *o = *o - s;
    }
  }
}

// backward: x_P = Ainv v_P - Q^T x_U for ND_ROWS pivots of a front per CTA
// (Q^T stored); x: FP64 [nc][NC], read at U and written at P; x32 its FP32
// copy (optional; the staged x_U is read from it when T is FP32)
template <int NC, class T, int G>
__global__ void __launch_bounds__(ND_THREADS) k_nd_bwd(const NdFrontD* __restrict__ fr, const int2* __restrict__ cta,
                                                      const T* __restrict__ A, const T* __restrict__ QT,
                                                      const T* __restrict__ v, const int* __restrict__ idx,
                                                      double* __restrict__ x, float* __restrict__ x32,
                                                      const int* done) {
  extern __shared__ __align__(16) unsigned char nd_sm[];
  pdl_wait();
  if (done && *done) return;
  const int2 cr = cta[blockIdx.x];
  const NdFrontD F = fr[cr.x];
  const int* pd = idx + F.ioff;
  const int* ud = pd + F.np;
  T* sv = reinterpret_cast<T*>(nd_sm);
  T* sx = sv + nd_vec_len<NC, T>(F.np);
  const T* vp = v + F.voff * NC;
  nd_stage<NC, T>(F.np, sv, [&](int k, T (&y)[NC]) {
#pragma unroll
    for (int c = 0; c < NC; ++c) y[c] = vp[(int64_t)k * NC + c];
  });
  nd_stage<NC, T>(F.nu, sx, [&](int k, T (&y)[NC]) {
    const int64_t g = (int64_t)ud[k] * NC;
    if (sizeof(T) == 4 && x32) {
#pragma unroll
      for (int c = 0; c < NC; ++c) y[c] = (T)x32[g + c];
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) y[c] = (T)x[g + c];
    }
  });
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = cr.y + 4 * w;
  if constexpr (G == 8) {
    T a[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) a[c] = (T)0;
    const int r = row0 + (lane >> 3);
    nd_row8<NC, T>(A + F.aoff, F.lp, F.np, r, F.np, sv, (T)1, a);
    nd_row8<NC, T>(QT + F.toff, F.lu, F.nu, r, F.np, sx, (T)-1, a);
    nd_reduce8<NC, T>(a);
    pdl_trigger();
    int c;
    T s;
    if (nd_pick8<NC, T>(a, lane, c, s) && r < F.np) {
      const int64_t gi = (int64_t)pd[r] * NC + c;
      x[gi] = (double)s;
      if (x32) x32[gi] = (float)s;
    }
  } else {
    T acc[4][NC];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[q][c] = (T)0;
    nd_rows4<NC, T>(A + F.aoff, F.lp, F.np, row0, F.np, sv, (T)1, acc);
    nd_rows4<NC, T>(QT + F.toff, F.lu, F.nu, row0, F.np, sx, (T)-1, acc);
    nd_reduce4<NC, T>(acc);
    pdl_trigger();
    int q, c;
    T s;
    if (nd_pick<NC, T>(acc, lane, q, c, s) && row0 + q < F.np) {
      const int64_t gi = (int64_t)pd[row0 + q] * NC + c;
      x[gi] = (double)s;
      if (x32) x32[gi] = (float)s;
    }
  }
}

}  // namespace

// host data of the factor
struct NdData {
  int nfront = 0, nlev = 0, max_np = 0;
  std::vector<size_t> lev_fsm, lev_bsm;  // per level: the largest staged v_P (forward) and v_P + x_U
                                         // (backward), in vector rows rounded to 4
  std::vector<int> lev_f0;            // fronts of solve level l: [lev_f0[l], lev_f0[l + 1]), l = 0 deepest
  std::vector<int64_t> lev_r0;        // their front-vector rows
  std::vector<int> lev_fwd, lev_bwd;  // their solve CTAs (+ end)
  std::vector<char> lev_fw8, lev_bw8; // the level's products run eight lanes per row (few pivots)
  NdFrontD* fronts = nullptr;
  int* idx = nullptr;
  int4* grow = nullptr;
  int2* fwd_cta = nullptr;
  int2* bwd_cta = nullptr;
  int64_t nrows = 0;
  float *A32 = nullptr, *Q32 = nullptr, *T32 = nullptr;
  double *A64 = nullptr, *Q64 = nullptr, *T64 = nullptr;
  float* vb = nullptr;    // [nrows][TS_NB] block path
  float* v1f = nullptr;   // [nrows] one column, mixed precision
  double* v1d = nullptr;  // [nrows] one column, FP64
};

namespace {

struct HostFront {
  int depth = 0, parent = -1;
  int child[2] = {-1, -1};
  std::vector<int> pn, un;  // pivot and update coarse nodes
};

// the nested-dissection tree of the coarse grid
struct NdTree {
  const ts_handle h;
  int dim, n[3];
  std::vector<HostFront> f;
  explicit NdTree(ts_handle hh) : h(hh) {
    dim = h->g.dim;
    for (int a = 0; a < 3; ++a) n[a] = (a < dim) ? h->g.ncn[a] : 1;
  }
  int node(int x, int y, int z) const { return x + n[0] * (y + n[1] * z); }
  int ndof(int l) const { return h->cn_h[l].ndof; }
  int build(const int* lo, const int* hi, int depth, int parent) {
    const int id = (int)f.size();
    f.emplace_back();
    f[id].depth = depth;
    f[id].parent = parent;
    int ext[3], cnt = 1, ax = 0;
    for (int a = 0; a < 3; ++a) {
      ext[a] = hi[a] - lo[a];
      cnt *= ext[a];
      if (ext[a] > ext[ax]) ax = a;
    }
    std::vector<int> piv;
    const bool leaf = cnt <= 4;
    const int mid = lo[ax] + ext[ax] / 2;
    for (int z = lo[2]; z < hi[2]; ++z)
      for (int y = lo[1]; y < hi[1]; ++y)
        for (int x = lo[0]; x < hi[0]; ++x) {
          const int c[3] = {x, y, z};
          if ((leaf || c[ax] == mid) && ndof(node(x, y, z)) > 0) piv.push_back(node(x, y, z));
        }
    // update set: nodes next to the box, outside it
    std::vector<int> upd;
    int l2[3], h2[3];
    for (int a = 0; a < 3; ++a) {
      l2[a] = std::max(lo[a] - 1, 0);
      h2[a] = std::min(hi[a] + 1, n[a]);
    }
    for (int z = l2[2]; z < h2[2]; ++z)
      for (int y = l2[1]; y < h2[1]; ++y)
        for (int x = l2[0]; x < h2[0]; ++x) {
          const bool in = x >= lo[0] && x < hi[0] && y >= lo[1] && y < hi[1] && z >= lo[2] && z < hi[2];
          if (!in && ndof(node(x, y, z)) > 0) upd.push_back(node(x, y, z));
        }
    f[id].pn = piv;
    f[id].un = upd;
    if (!leaf) {
      int clo[3], chi[3];
      for (int s = 0; s < 2; ++s) {
        for (int a = 0; a < 3; ++a) {
          clo[a] = lo[a];
          chi[a] = hi[a];
        }
        if (s == 0)
          chi[ax] = mid;
        else
          clo[ax] = mid + 1;
        if (chi[ax] > clo[ax]) {
          const int c = build(clo, chi, depth + 1, id);
          f[id].child[s] = c;
        }
      }
    }
    return id;
  }
};

int r32(int x) { return ((x + TILE - 1) / TILE) * TILE; }

// stream-ordered setup memory freed level by level (counted in the handle's
// scratch peak like salloc)
struct LevelMem {
  ts_handle h;
  std::vector<std::pair<void*, size_t>> held;
  template <class T>
  T* get(size_t n) {
    void* p = nullptr;
    const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, ts_scratch_pool(h->ctx->device), h->ctx->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw TsError(TS_ERR_OOM, "cudaMallocAsync of " + std::to_string(bytes) + " bytes failed");
    }
    held.emplace_back(p, bytes);
    h->scratch_bytes += (int64_t)bytes;
    h->scratch_peak = std::max(h->scratch_peak, h->scratch_bytes);
    return static_cast<T*>(p);
  }
  void release() {
    for (auto& pb : held) {
      cudaFreeAsync(pb.first, h->ctx->stream);
      h->scratch_bytes -= (int64_t)pb.second;
    }
    held.clear();
  }
  ~LevelMem() { release(); }
};

}  // namespace

bool coarse_uses_nd(ts_handle h) {
  if (h->cl_off.size() < 2) return false;  // one dense line
  if (h->opt.coarse_layout == 3) return true;
  return h->opt.coarse_layout == 0 && (int)h->cl_off.size() >= ND_AUTO_LINES;
}

void build_coarse_factor_nd(ts_handle h) {
  cudaStream_t st = h->ctx->stream;
  const int nc = h->nc;
  auto nd = std::make_shared<NdData>();
  // (1) the tree and its fronts, deepest level first
  NdTree T(h);
  {
    const int lo[3] = {0, 0, 0};
    const int hi[3] = {T.n[0], T.n[1], T.n[2]};
    T.build(lo, hi, 0, -1);
  }
  const int nf = (int)T.f.size();
  int maxd = 0;
  for (const HostFront& F : T.f) maxd = std::max(maxd, F.depth);
  std::vector<int> order;  // solve order: deepest level first
  std::vector<int> lev_of;
  nd->lev_f0.clear();
  for (int d = maxd; d >= 0; --d) {
    nd->lev_f0.push_back((int)order.size());
    for (int i = 0; i < nf; ++i)
      if (T.f[i].depth == d) order.push_back(i);
  }
  nd->lev_f0.push_back(nf);
  nd->nlev = maxd + 1;
  nd->nfront = nf;
  std::vector<int> rank(nf);
  for (int i = 0; i < nf; ++i) rank[order[i]] = i;
  // the pivot front of every coarse node: each node with basis functions is
  // a pivot exactly once, and every update node is a pivot of an ancestor
  std::vector<int> owner(h->n_cnodes, -1);
  for (int i = 0; i < nf; ++i)
    for (int l : T.f[i].pn) {
      if (owner[l] >= 0) throw TsError(TS_ERR_INVALID, "internal: nested dissection pivots a coarse node twice");
      owner[l] = i;
    }
  for (int l = 0; l < h->n_cnodes; ++l)
    if (h->cn_h[l].ndof > 0 && owner[l] < 0) throw TsError(TS_ERR_INVALID, "internal: coarse node left out");
  for (int i = 0; i < nf; ++i)
    for (int l : T.f[i].un) {
      int a = T.f[i].parent;
      while (a >= 0 && a != owner[l]) a = T.f[a].parent;
      if (a < 0) throw TsError(TS_ERR_INVALID, "internal: update node outside the ancestors");
    }
  // DOF lists, sizes, offsets (in solve order)
  std::vector<NdFrontD> fd(nf);
  std::vector<int> idx;
  std::vector<std::vector<int>> pd(nf), ud(nf);
  int64_t aoff = 0, qoff = 0, toff = 0, voff = 0;
  double mflops = 0.0, fmas = 0.0;
  for (int r = 0; r < nf; ++r) {
    const HostFront& F = T.f[order[r]];
    for (int l : F.pn)
      for (int k = 0; k < h->cn_h[l].ndof; ++k) pd[r].push_back(h->cn_h[l].first_dof + k);
    for (int l : F.un)
      for (int k = 0; k < h->cn_h[l].ndof; ++k) ud[r].push_back(h->cn_h[l].first_dof + k);
    NdFrontD& D = fd[r];
    D.np = (int)pd[r].size();
    D.nu = (int)ud[r].size();
    D.lp = (D.np + 3) & ~3;
    D.lu = (D.nu + 3) & ~3;
    D.aoff = aoff;
    D.qoff = qoff;
    D.toff = toff;
    D.voff = voff;
    D.ioff = (int64_t)idx.size();
    idx.insert(idx.end(), pd[r].begin(), pd[r].end());
    idx.insert(idx.end(), ud[r].begin(), ud[r].end());
    aoff += (int64_t)D.np * D.lp;
    qoff += (int64_t)D.nu * D.lp;
    toff += (int64_t)D.np * D.lu;
    voff += D.np + D.nu;
    nd->max_np = std::max(nd->max_np, D.np);
    const double p = D.np, u = D.nu;
    // multifrontal Cholesky: factor (p^3/3), L21 (p^2 u), Schur update (p u^2) FLOP
    mflops += p * p * p / 3.0 + p * p * u + p * u * u;
    fmas += p * p + 2.0 * u * p;  // Ainv, Q (forward) and Q^T (backward) entries, one FMA each
  }
  nd->nrows = voff;
  // front-vector rows: b index at the pivots, the children's contributions,
  // and the U positions of every front in its parent
  std::vector<int4> grow(voff, make_int4(-1, -1, -1, 0));
  std::vector<int64_t> upos_off(nf, 0);
  std::vector<int> upos_all;
  {
    std::vector<int> pos(nc, -1);
    for (int r = 0; r < nf; ++r) {
      const HostFront& F = T.f[order[r]];
      const NdFrontD& D = fd[r];
      for (int i = 0; i < D.np; ++i) {
        grow[D.voff + i].x = pd[r][i];
        pos[pd[r][i]] = i;
      }
      for (int j = 0; j < D.nu; ++j) pos[ud[r][j]] = D.np + j;
      for (int s = 0; s < 2; ++s) {
        if (F.child[s] < 0) continue;
        const int c = rank[F.child[s]];
        const NdFrontD& C = fd[c];
        upos_off[c] = (int64_t)upos_all.size();
        for (int j = 0; j < C.nu; ++j) {
          const int p = pos[ud[c][j]];
          if (p < 0) throw TsError(TS_ERR_INVALID, "internal: child update outside its parent front");
          upos_all.push_back(p);
          int4& g = grow[D.voff + p];
          if (s == 0)
            g.y = (int)(C.voff + C.np + j);
          else
            g.z = (int)(C.voff + C.np + j);
        }
      }
      for (int i = 0; i < D.np; ++i) pos[pd[r][i]] = -1;
      for (int j = 0; j < D.nu; ++j) pos[ud[r][j]] = -1;
    }
  }
  if (voff >= (int64_t)1 << 31) throw TsError(TS_ERR_INVALID, "internal: coarse front vectors too long");
  nd->fronts = dupload(h, fd);
  nd->idx = dupload(h, idx);
  nd->grow = dupload(h, grow);
  const int* upos_d = supload(h, upos_all);
  // solve CTAs per level
  {
    std::vector<int2> fw, bw;
    nd->lev_fwd.clear();
    nd->lev_bwd.clear();
    nd->lev_r0.clear();
    for (int lv = 0; lv < nd->nlev; ++lv) {
      nd->lev_fwd.push_back((int)fw.size());
      nd->lev_bwd.push_back((int)bw.size());
      nd->lev_r0.push_back(fd[nd->lev_f0[lv]].voff);
      size_t fsm = 0, bsm = 0;
      for (int r = nd->lev_f0[lv]; r < nd->lev_f0[lv + 1]; ++r) {
        fsm = std::max(fsm, (size_t)fd[r].lp);
        bsm = std::max(bsm, (size_t)(fd[r].lp + fd[r].lu));
      }
      nd->lev_fsm.push_back(fsm);
      nd->lev_bsm.push_back(bsm);
      // eight lanes per row while a row takes at most ND_G8_LP / 4 16-byte loads
      nd->lev_fw8.push_back(fsm <= (size_t)ND_G8_LP ? 1 : 0);
      nd->lev_bw8.push_back(bsm <= (size_t)ND_G8_LP ? 1 : 0);
      for (int r = nd->lev_f0[lv]; r < nd->lev_f0[lv + 1]; ++r) {
        for (int j = 0; j < fd[r].nu; j += ND_ROWS)
          if (fd[r].np > 0) fw.push_back(make_int2(r, j));
        for (int i = 0; i < fd[r].np; i += ND_ROWS) bw.push_back(make_int2(r, i));
      }
    }
    nd->lev_fwd.push_back((int)fw.size());
    nd->lev_bwd.push_back((int)bw.size());
    nd->lev_r0.push_back(voff);
    nd->fwd_cta = fw.empty() ? nullptr : dupload(h, fw);
    nd->bwd_cta = bw.empty() ? nullptr : dupload(h, bw);
  }
  const bool mixed = h->opt.precision != TS_FP64 && !h->coarse64;
  if (mixed) {
    nd->A32 = dalloc<float>(h, std::max<int64_t>(aoff, 1));
    nd->Q32 = dalloc<float>(h, std::max<int64_t>(qoff, 1));
    nd->T32 = dalloc<float>(h, std::max<int64_t>(toff, 1));
    nd->v1f = dalloc<float>(h, voff);
    if (h->g.dim == 2) nd->vb = dalloc<float>(h, voff * TS_NB);
  } else {
    nd->A64 = dalloc<double>(h, std::max<int64_t>(aoff, 1));
    nd->Q64 = dalloc<double>(h, std::max<int64_t>(qoff, 1));
    nd->T64 = dalloc<double>(h, std::max<int64_t>(toff, 1));
    nd->v1d = dalloc<double>(h, voff);
  }
  h->cfac_method_flops = mflops;
  h->bcr_fmas = fmas;
  // (2) numeric factor, level by level
  K0Lines K0;
  {
    std::vector<int> qline(nc);
    for (size_t q = 0; q < h->cl_off.size(); ++q)
      for (int i = 0; i < h->cl_wid[q]; ++i) qline[h->cl_off[q] + i] = (int)q;
    K0.A = h->K0A;
    K0.C = h->K0C;
    K0.qline = supload(h, qline);
    K0.qoff = supload(h, h->cl_off);
    K0.cw = h->cw;
  }
  int* dropped_total = salloc<int>(h, 1);
  TS_CUDA(cudaMemsetAsync(dropped_total, 0, sizeof(int), st));
  TileScratch sc;
  std::unique_ptr<LevelMem> child_mem;
  std::vector<NdAsmF> child_af;
  NdAsmF* child_af_d = nullptr;
  double* child_A22 = nullptr;
  for (int lv = 0; lv < nd->nlev; ++lv) {
    const int f0 = nd->lev_f0[lv], f1 = nd->lev_f0[lv + 1], nl = f1 - f0;
    auto mem = std::make_unique<LevelMem>();
    mem->h = h;
    std::vector<NdAsmF> af(nl);
    int64_t n11 = 0, n21 = 0, n22 = 0, nd0 = 0;
    int max_nt = 0;
    int64_t max_e = 1;
    for (int k = 0; k < nl; ++k) {
      const NdFrontD& D = fd[f0 + k];
      NdAsmF& A = af[k];
      A.np = D.np;
      A.nu = D.nu;
      A.npp = r32(D.np);
      A.nup = r32(D.nu);
      A.a11 = n11;
      A.a21 = n21;
      A.a22 = n22;
      A.d0 = nd0;
      A.ioff = D.ioff;
      A.upos = upos_off[f0 + k];
      n11 += (int64_t)A.npp * A.npp;
      n21 += (int64_t)A.nup * A.npp;
      n22 += (int64_t)A.nup * A.nup;
      nd0 += A.npp;
      max_nt = std::max(max_nt, A.npp / TILE);
      max_e = std::max({max_e, (int64_t)A.npp * A.npp, (int64_t)A.nup * A.npp, (int64_t)A.nup * A.nup});
      const HostFront& F = T.f[order[f0 + k]];
      for (int s = 0; s < 2; ++s) A.child[s] = (F.child[s] >= 0) ? rank[F.child[s]] - nd->lev_f0[lv - 1] : -1;
    }
    NdAsmF* af_d = supload(h, af);
    double* A11 = mem->get<double>(n11);
    double* A21 = mem->get<double>(n21);
    double* A22 = mem->get<double>(n22);
    double* d0 = mem->get<double>(nd0);
    int* drop = mem->get<int>(nd0);
    TS_CUDA(cudaMemsetAsync(drop, 0, sizeof(int) * std::max<int64_t>(nd0, 1), st));
    const unsigned gx = (unsigned)std::min<int64_t>((max_e + 255) / 256, 64);
    tsl(h), k_nd_assemble<<<dim3(gx, nl), 256, 0, st>>>(af_d, nd->idx, K0, A11, A21, A22, d0);
    TS_CUDA(cudaGetLastError());
    if (lv > 0) {
      int64_t cmax = 1;
      for (const NdAsmF& C : child_af) cmax = std::max(cmax, (int64_t)C.nu * C.nu);
      const unsigned cx = (unsigned)std::min<int64_t>((cmax + 255) / 256, 64);
      for (int s = 0; s < 2; ++s)
        tsl(h), k_nd_extend<<<dim3(cx, nl), 256, 0, st>>>(af_d, child_af_d, upos_d, child_A22, s, A11, A21, A22);
      TS_CUDA(cudaGetLastError());
      child_mem.reset();  // the children's update matrices are consumed
    }
    // Cholesky with dropping, W = L^{-1}, Ainv = W^T W (per front, tiled)
    double* W = mem->get<double>(n11);
    double* Ainv = mem->get<double>(n11);
    double* Tt = mem->get<double>(nd0 * TILE);
    double* Linv = mem->get<double>(nd0 * TILE);
    for (int kb = 0; kb < max_nt; ++kb) {
      std::vector<PotrfTask> pt;
      std::vector<GemmTask> tr, sy;
      for (const NdAsmF& A : af) {
        const int nt = A.npp / TILE;
        if (nt <= kb) continue;
        const int ld = A.npp;
        pt.push_back(PotrfTask{A11 + A.a11 + (int64_t)kb * TILE * ld + kb * TILE,
                               Linv + (A.d0 + kb * TILE) * TILE, d0 + A.d0 + kb * TILE, drop + A.d0 + kb * TILE, ld});
        const int rest = nt - kb - 1;
        if (rest == 0) continue;
        double* panel = A11 + A.a11 + (int64_t)(kb + 1) * TILE * ld + kb * TILE;
        const double* li = Linv + (A.d0 + kb * TILE) * TILE;
        tr.push_back(GemmTask{panel, li, panel, rest * TILE, TILE, TILE, ld, TILE, ld, 0, 1, 1.0, 0.0, 0});
        double* trail = A11 + A.a11 + (int64_t)(kb + 1) * TILE * ld + (kb + 1) * TILE;
        sy.push_back(GemmTask{panel, panel, trail, rest * TILE, rest * TILE, TILE, ld, ld, ld, 0, 1, -1.0, 1.0, 1});
      }
      tiles_potrf(h, pt);
      tiles_gemm(h, tr, sc);
      tiles_gemm(h, sy, sc);
    }
    if (max_nt > 0) {
      TS_CUDA(cudaMemsetAsync(W, 0, sizeof(double) * std::max<int64_t>(n11, 1), st));
      tsl(h), k_nd_diag_tiles<<<dim3(max_nt, nl), 256, 0, st>>>(af_d, W, Linv);
      TS_CUDA(cudaGetLastError());
    }
    for (int i = 1; i < max_nt; ++i) {
      std::vector<GemmTask> g1, g2;
      for (const NdAsmF& A : af) {
        if (A.npp / TILE <= i) continue;
        const int ld = A.npp;
        double* Tf = Tt + A.d0 * TILE;
        g1.push_back(GemmTask{A11 + A.a11 + (int64_t)i * TILE * ld, W + A.a11, Tf, TILE, i * TILE, i * TILE, ld, ld, ld,
                              0, 0, 1.0, 0.0, 4});
        g2.push_back(GemmTask{Linv + (A.d0 + i * TILE) * TILE, Tf, W + A.a11 + (int64_t)i * TILE * ld, TILE, i * TILE,
                              TILE, TILE, ld, ld, 0, 0, -1.0, 0.0, 0});
      }
      tiles_gemm(h, g1, sc);
      tiles_gemm(h, g2, sc);
    }
    {
      std::vector<GemmTask> gi, gq, gs;
      for (const NdAsmF& A : af) {
        if (A.npp == 0) continue;
        const int ld = A.npp;
        gi.push_back(GemmTask{W + A.a11, W + A.a11, Ainv + A.a11, ld, ld, ld, ld, ld, ld, 1, 0, 1.0, 0.0, 2});
      }
      tiles_gemm(h, gi, sc);
      // Q = F21 Ainv takes W's place (W is not read once Ainv is formed) when it fits
      double* Q = (n21 <= n11) ? W : mem->get<double>(n21);
      for (const NdAsmF& A : af) {
        if (A.npp == 0 || A.nup == 0) continue;
        gq.push_back(GemmTask{A21 + A.a21, Ainv + A.a11, Q + A.a21, A.nup, A.npp, A.npp, A.npp, A.npp, A.npp, 0, 0,
                              1.0, 0.0, 0});
        // S = F22 - Q F21^T (lower tiles)
        gs.push_back(GemmTask{Q + A.a21, A21 + A.a21, A22 + A.a22, A.nup, A.nup, A.npp, A.npp, A.npp, A.nup, 0, 1,
                              -1.0, 1.0, 1});
      }
      tiles_gemm(h, gq, sc);
      tiles_gemm(h, gs, sc);
      const unsigned sx = (unsigned)std::min<int64_t>((max_e + 255) / 256, 64);
      if (mixed)
        tsl(h), k_nd_store<float><<<dim3(sx, nl), 256, 0, st>>>(af_d, nd->fronts, f0, Ainv, Q, nd->A32, nd->Q32,
                                                                nd->T32);
      else
        tsl(h), k_nd_store<double><<<dim3(sx, nl), 256, 0, st>>>(af_d, nd->fronts, f0, Ainv, Q, nd->A64, nd->Q64,
                                                                 nd->T64);
      TS_CUDA(cudaGetLastError());
    }
    tsl(h), k_nd_count<<<1, 256, 0, st>>>(af_d, nl, drop, dropped_total);
    TS_CUDA(cudaGetLastError());
    // this level's update matrices stay for its parents
    child_af = af;
    child_af_d = af_d;
    child_A22 = A22;
    child_mem = std::move(mem);
  }
  child_mem.reset();
  int dr = 0;
  TS_CUDA(cudaMemcpyAsync(&dr, dropped_total, sizeof(int), cudaMemcpyDeviceToHost, st));
  TS_CUDA(cudaStreamSynchronize(st));
  h->coarse_dropped = dr;
  // the block path's coarse vectors
  if (mixed && h->g.dim == 2) {
    const int64_t ldb = (int64_t)h->K0_ld * TS_NB;
    h->r0b = dalloc<double>(h, ldb);
    h->u0b = dalloc<double>(h, ldb);
    h->u0fb = dalloc<float>(h, ldb);
    h->r0b32 = dalloc<float>(h, ldb);
    TS_CUDA(cudaMemsetAsync(h->r0b, 0, sizeof(double) * ldb, st));
    TS_CUDA(cudaMemsetAsync(h->u0b, 0, sizeof(double) * ldb, st));
    TS_CUDA(cudaMemsetAsync(h->u0fb, 0, sizeof(float) * ldb, st));
    TS_CUDA(cudaMemsetAsync(h->r0b32, 0, sizeof(float) * ldb, st));
  }
  // shared memory of the solve kernels: the largest staged v_P + x_U
  {
    size_t mb = 1;
    for (size_t b : nd->lev_bsm) mb = std::max(mb, b);
    const size_t sb = mb * TS_NB * sizeof(float);
    const size_t s1 = mb * sizeof(double);
    const int dev = h->ctx->device;
    const size_t lim = std::min({ts_allow_dynamic_smem(k_nd_fwd<TS_NB, float, 32>, dev),
                                 ts_allow_dynamic_smem(k_nd_bwd<TS_NB, float, 32>, dev),
                                 ts_allow_dynamic_smem(k_nd_fwd<1, float, 32>, dev),
                                 ts_allow_dynamic_smem(k_nd_bwd<1, float, 32>, dev),
                                 ts_allow_dynamic_smem(k_nd_fwd<1, double, 32>, dev),
                                 ts_allow_dynamic_smem(k_nd_bwd<1, double, 32>, dev),
                                 ts_allow_dynamic_smem(k_nd_fwd<TS_NB, float, 8>, dev),
                                 ts_allow_dynamic_smem(k_nd_bwd<TS_NB, float, 8>, dev),
                                 ts_allow_dynamic_smem(k_nd_fwd<1, float, 8>, dev),
                                 ts_allow_dynamic_smem(k_nd_bwd<1, float, 8>, dev),
                                 ts_allow_dynamic_smem(k_nd_fwd<1, double, 8>, dev),
                                 ts_allow_dynamic_smem(k_nd_bwd<1, double, 8>, dev)});
    if (std::max(sb, s1) > lim) throw TsError(TS_ERR_INVALID, "coarse separator too large for the nested-dissection solve");
  }
  h->nd = nd;
}

namespace {

template <class K, class... Args>
void nd_launch(ts_handle h, bool pdl, K kernel, unsigned grid, size_t smem, Args... args) {
  if (grid == 0) return;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(ND_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = h->ctx->stream;
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  tsl(h);
  TS_CUDA(cudaLaunchKernelEx(&cfg, kernel, args...));
}

// x = K_0^{-1} b (NC columns): the forward and backward level sweeps
template <int NC, class TB, class T>
void nd_solve(ts_handle h, const TB* b, T* v, const T* A, const T* Q, const T* QT, double* x, float* x32) {
  const NdData& nd = *h->nd;
  const int* done = h->done_flag;
  bool pdl = false;
  for (int lv = 0; lv < nd.nlev; ++lv) {
    const int64_t r0 = nd.lev_r0[lv], r1 = nd.lev_r0[lv + 1];
    const unsigned g = (unsigned)std::min<int64_t>((r1 - r0 + ND_THREADS - 1) / ND_THREADS, 8 * h->ctx->n_sm);
    nd_launch(h, pdl, k_nd_gather<NC, TB, T>, g, 0, (const int4*)nd.grow, r0, r1, b, v, done);
    pdl = true;
    const int c0 = nd.lev_fwd[lv], c1 = nd.lev_fwd[lv + 1];
    auto kf = nd.lev_fw8[lv] ? k_nd_fwd<NC, T, 8> : k_nd_fwd<NC, T, 32>;
    nd_launch(h, pdl, kf, (unsigned)(c1 - c0), nd.lev_fsm[lv] * NC * sizeof(T), (const NdFrontD*)nd.fronts,
              (const int2*)(nd.fwd_cta + c0), Q, v, done);
  }
  for (int lv = nd.nlev - 1; lv >= 0; --lv) {
    const int c0 = nd.lev_bwd[lv], c1 = nd.lev_bwd[lv + 1];
    auto kb = nd.lev_bw8[lv] ? k_nd_bwd<NC, T, 8> : k_nd_bwd<NC, T, 32>;
    nd_launch(h, pdl, kb, (unsigned)(c1 - c0), nd.lev_bsm[lv] * NC * sizeof(T), (const NdFrontD*)nd.fronts,
              (const int2*)(nd.bwd_cta + c0), A, QT, (const T*)v, (const int*)nd.idx, x, x32, done);
    pdl = true;
  }
}

}  // namespace

void launch_coarse_solve_nd(ts_handle h) {
  const NdData& nd = *h->nd;
  if (nd.A32)
    nd_solve<1, double, float>(h, h->r0, nd.v1f, nd.A32, nd.Q32, nd.T32, h->u0, h->u0f);
  else
    nd_solve<1, double, double>(h, h->r0, nd.v1d, nd.A64, nd.Q64, nd.T64, h->u0, h->u0f);
}

void launch_bcoarse_solve_nd(ts_handle h) {
  const NdData& nd = *h->nd;
  if (!nd.vb) throw TsError(TS_ERR_INVALID, "internal: no block coarse solve (mixed 2D designs only)");
  nd_solve<TS_NB, float, float>(h, h->r0b32, nd.vb, nd.A32, nd.Q32, nd.T32, h->u0b, h->u0fb);
}
