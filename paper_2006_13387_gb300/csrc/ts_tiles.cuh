// Batched FP64 32 x 32 tile kernels of the coarse factors (defined in
// ts_cfactor.cu), shared by the block cyclic reduction (ts_cfactor.cu) and
// the nested-dissection factor (ts_cnd.cu).
#pragma once
#include <vector>

#include "ts_internal.cuh"

constexpr int TILE = 32;  // tile edge of the batched dense kernels

// C = alpha op(A) op(B) + beta C for one task; a launch runs many tasks.
struct GemmTask {
  const double* A;
  const double* B;
  double* C;
  int m, n, k;        // op(A): m x k, op(B): k x n; all multiples of 32
  int lda, ldb, ldc;
  int ta, tb;         // 1: the operand is stored transposed (row-major k x m / n x k)
  double alpha, beta;
  int mode;           // bit 0: lower output tiles only; bit 1: k from max(ti,tj)*32
                      // (A^T B with both lower); bit 2: k from tj*32 (B lower)
  const int2* kr;     // optional: k-tile range [x, y] of the nonzero operand tiles,
  int kr_by;          // indexed by the output row tile (1) or column tile (2)
  unsigned long long* flops;  // optional: FLOPs of the tiles formed are added here
};

// Cholesky of one 32 x 32 diagonal tile in place, with dropping of dependent
// pivots (below 1e-9 of the original diagonal entry), and its inverse.
struct PotrfTask {
  double* A;             // the diagonal tile, leading dimension ld
  double* Linv;          // 32 x 32 output: inverse of the factor tile
  const double* diag0;   // original diagonal entries of these 32 DOFs
  int* dropped;          // 32 flags
  int ld;                // leading dimension of A (0: the launch's)
};

// Split-k scratch of a sequence of batched GEMM launches (stream-ordered
// setup memory of the handle, grown on demand).
struct TileScratch {
  double* part = nullptr;
  unsigned* cnt = nullptr;
  int64_t part_tiles = 0, cnt_tiles = 0;
};

// One launch of the tasks (shapes may differ between tasks; each task's own
// m, n, k and leading dimensions are used).  Adds the formed tiles' FLOPs to
// h->cfac_cnt.  Launches with fewer output tiles than four resident CTAs per
// SM split k when no task's output aliases an operand.
void tiles_gemm(ts_handle h, const std::vector<GemmTask>& ts, TileScratch& sc);
// One launch of the tile Cholesky tasks (status bit 2 on a clearly negative pivot).
void tiles_potrf(ts_handle h, const std::vector<PotrfTask>& ts);
