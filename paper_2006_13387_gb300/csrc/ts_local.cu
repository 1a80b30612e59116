// Level 1 of the preconditioner (Sec. 2, local Dirichlet problems):
//   M_1^{-1} r = sum_i R_i^T K_i^{-1} R_i r,  K_i = R_i K R_i^T,
// with R_i the 0/1 restriction to the free DOFs of the nodes of D'_i.
// Each K_i is block-tridiagonal by node lines (2D rows, 3D planes).  Setup:
// FP64 block-line LDL^T (one CTA per subdomain), S_k = L_k D_k L_k^T,
// W_k = L_k^{-1}.  Solve, block LU:
//   forward   y_k = r_k - A_{k,k-1} u_{k-1},  u_k = S_k^{-1} y_k
//   backward  x_k = u_k - S_k^{-1} (A_{k,k+1} x_{k+1})
// where the couplings A_{k,k+-1} between neighbouring lines are applied
// matrix-free from E_e and KE, so only S_k^{-1} is stored per line:
//  * FP64 path: the dense inverse M_k = W_k^T D_k^{-1} W_k (one GEMV a step);
//  * mixed path: V_k = D_k^{-1/2} W_k, packed lower triangle, applied as
//    V_k^T (V_k y).  The Gram form keeps the FP32 operator positive definite
//    even when cond(S_k) exceeds 1/eps_32 (high contrast), where rounding the
//    explicit inverse to FP32 does not.
// A node-owner gather adds the overlapping local solutions (no atomics,
// fixed sum order).
#include <algorithm>

#include "ts_blockline.cuh"
#include "ts_internal.cuh"
#include "ts_reduce.cuh"

// element stiffness (E = 1), this translation unit's copy
static __constant__ double c_KE[24 * 24];
static __constant__ float c_KEf[24 * 24];

void upload_KE_local(ts_handle h, const std::vector<double>& KE) {
  static std::vector<float> kf;
  kf.assign(KE.begin(), KE.end());
  TS_CUDA(cudaMemcpyToSymbolAsync(c_KE, KE.data(), KE.size() * sizeof(double), 0, cudaMemcpyHostToDevice,
                                  h->ctx->stream));
  TS_CUDA(cudaMemcpyToSymbolAsync(c_KEf, kf.data(), kf.size() * sizeof(float), 0, cudaMemcpyHostToDevice,
                                  h->ctx->stream));
  TS_CUDA(cudaStreamSynchronize(h->ctx->stream));
}

template <class TF>
__device__ __forceinline__ const TF* ke_const();
template <>
__device__ __forceinline__ const double* ke_const<double>() { return c_KE; }
template <>
__device__ __forceinline__ const float* ke_const<float>() { return c_KEf; }

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
    return elas_entry<DIM>(g, E, c_KE, a, ca, bb, cb, b.elo, b.ehi);
  }
};

// ---------------------------------------------------------------------------
// factor kernel: one CTA per subdomain
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(256) k_local_factor(Geom g, AxisTables ax, const double* __restrict__ E,
                                                      const uint8_t* __restrict__ fm, const BLDesc* __restrict__ desc,
                                                      double* __restrict__ fac, int* __restrict__ status) {
  extern __shared__ double smem[];
  __shared__ int bad;
  const int s = blockIdx.x;
  if (threadIdx.x == 0) bad = 0;
  ElasAsm<DIM> A;
  A.g = g;
  A.E = E;
  A.fm = fm;
  sub_box(g, ax, s, A.b);
  __syncthreads();
  const BLDesc d = desc[s];
  bl_factor(A, d.nb, d.w, fac + d.off, true, true, smem, &bad);
  if (threadIdx.x == 0 && bad) atomicOr(status, 1);  // non-SPD local matrix
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (; i < n; i += st) b[i] = (float)a[i];
}

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
__host__ __device__ inline int64_t lv1_stride(int w, bool vform) {
  return vform ? lv1_vrow(w) : (int64_t)w * lv1_ld(w);
}

// From the block-line factor (W_k unit lower), W_k and dinv_k staged in
// shared memory, one CTA per subdomain:
//   M form: M[i][j] = sum_{m >= max(i,j)} dinv[m] W[m][i] W[m][j]
//   V form: V[i][m] = sqrt(dinv[i]) W[i][m], m <= i
template <bool VF>
__global__ void __launch_bounds__(256) k_pack_level1(const BLDesc* __restrict__ desc, const double* __restrict__ fac,
                                                     double* __restrict__ pv64, float* __restrict__ pv32) {
  extern __shared__ double pk_sm[];
  const BLDesc d = desc[blockIdx.x];
  const int w = d.w, ld = lv1_ld(w);
  const int64_t ps = lv1_stride(w, VF), bs = bl_block_stride(w);
  double* Ws = pk_sm;
  double* dv = Ws + (int64_t)w * w;
  for (int k = 0; k < d.nb; ++k) {
    const double* W = fac + d.off + k * bs;
    __syncthreads();
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) Ws[e] = W[e];
    for (int e = threadIdx.x; e < w; e += blockDim.x) dv[e] = W[2 * (int64_t)w * w + e];
    __syncthreads();
    const int64_t o = d.coff + k * ps;
    for (int64_t e = threadIdx.x; e < ps; e += blockDim.x) {
      double v = 0.0;
      if (VF) {
        int i = (int)sqrt(2.0 * (double)e);
        while (i > 0 && lv1_vrow(i) > e) --i;
        while (i + 1 < w && lv1_vrow(i + 1) <= e) ++i;
        const int m = (int)(e - lv1_vrow(i));
        if (m <= i) v = sqrt(dv[i]) * Ws[i * w + m];
      } else {
        const int i = (int)(e / ld), j = (int)(e % ld);
        if (j < w)
          for (int m = max(i, j); m < w; ++m) v += dv[m] * Ws[m * w + i] * Ws[m * w + j];
      }
      if (pv64) pv64[o + e] = v;
      if (pv32) pv32[o + e] = (float)v;
    }
  }
}

// (A_{k,k+dir} x)_p for local row p of line k; x: local values of line k+dir.
// Elements in the subdomain's element box, source nodes in its node box
// (other nodes carry no local unknown); rows of non-free DOFs are zero.
// Everything comes from shared memory: KE (ks), the box's moduli (es, element
// (ex,ey[,ez]) at its box-relative position) and free flags (fs, per local
// DOF of the node box).
template <class TF>
__device__ __forceinline__ TF couple_q4(const SubBox& b, const TF* ks, const TF* es, const uint8_t* fs, int k, int dir,
                                        int p, const TF* xs) {
  const int c = p & 1, t = p >> 1;
  const int x = b.nlo[0] + t, y = b.nlo[1] + k, y2 = y + dir;
  const int ey = (dir < 0) ? y - 1 : y;
  if (ey < b.elo[1] || ey >= b.ehi[1]) return TF(0);
  if (!fs[k * 2 * b.nb3[0] + p]) return TF(0);
  const int nex = b.ehi[0] - b.elo[0];
  TF s = 0;
#pragma unroll
  for (int ex = x - 1; ex <= x; ++ex) {
    if (ex < b.elo[0] || ex >= b.ehi[0]) continue;
    const int row = (2 * q4_local(x - ex, y - ey) + c) * 8;
    TF se = 0;
#pragma unroll
    for (int x2 = ex; x2 <= ex + 1; ++x2) {
      if (x2 < b.nlo[0] || x2 > b.nhi[0]) continue;
      const int lb = q4_local(x2 - ex, y2 - ey), t2 = x2 - b.nlo[0];
      se += ks[row + 2 * lb] * xs[2 * t2] + ks[row + 2 * lb + 1] * xs[2 * t2 + 1];
    }
    s += es[(ey - b.elo[1]) * nex + (ex - b.elo[0])] * se;
  }
  return s;
}

template <class TF>
__device__ __forceinline__ TF couple_hex8(const SubBox& b, const TF* ks, const TF* es, const uint8_t* fs, int k,
                                          int dir, int p, const TF* xs) {
  const int c = p % 3, t = p / 3, nbx = b.nb3[0];
  const int x = b.nlo[0] + t % nbx, y = b.nlo[1] + t / nbx, z = b.nlo[2] + k, z2 = z + dir;
  const int ez = (dir < 0) ? z - 1 : z;
  if (ez < b.elo[2] || ez >= b.ehi[2]) return TF(0);
  if (!fs[k * 3 * nbx * b.nb3[1] + p]) return TF(0);
  const int nex = b.ehi[0] - b.elo[0], ney = b.ehi[1] - b.elo[1];
  TF s = 0;
#pragma unroll
  for (int ey = y - 1; ey <= y; ++ey) {
    if (ey < b.elo[1] || ey >= b.ehi[1]) continue;
#pragma unroll
    for (int ex = x - 1; ex <= x; ++ex) {
      if (ex < b.elo[0] || ex >= b.ehi[0]) continue;
      const int row = (3 * hex8_local(x - ex, y - ey, z - ez) + c) * 24;
      TF se = 0;
#pragma unroll
      for (int y2 = ey; y2 <= ey + 1; ++y2) {
        if (y2 < b.nlo[1] || y2 > b.nhi[1]) continue;
#pragma unroll
        for (int x2 = ex; x2 <= ex + 1; ++x2) {
          if (x2 < b.nlo[0] || x2 > b.nhi[0]) continue;
          const int col = 3 * hex8_local(x2 - ex, y2 - ey, z2 - ez);
          const int t2 = 3 * ((x2 - b.nlo[0]) + nbx * (y2 - b.nlo[1]));
          se += ks[row + col] * xs[t2] + ks[row + col + 1] * xs[t2 + 1] + ks[row + col + 2] * xs[t2 + 2];
        }
      }
      s += es[((ez - b.elo[2]) * ney + (ey - b.elo[1])) * nex + (ex - b.elo[0])] * se;
    }
  }
  return s;
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
#pragma unroll 4
  for (int i = j + part; i < w; i += 4) s += V[lv1_vrow(i) + j] * z[i];
  return quad_sum(s);
}

// ---------------------------------------------------------------------------
// local solve kernel: one CTA per subdomain; the couplings take one thread
// per line row, the products four threads (a quad) per row.  The stored
// line blocks stream through a ring of DEPTH shared-memory slots (16-byte
// cp.async, one commit group per step, DEPTH-1 groups in flight); the last
// DEPTH blocks of the forward sweep are reused by the backward sweep.
// ---------------------------------------------------------------------------
template <int DIM, class TF, int DEPTH, bool VF>
__global__ void __launch_bounds__(256) k_local_solve(Geom g, AxisTables ax, const TF* __restrict__ r,
                                                     const BLDesc* __restrict__ desc, const TF* __restrict__ pv,
                                                     const TF* __restrict__ E, const uint8_t* __restrict__ fm,
                                                     const int64_t* __restrict__ zoff, TF* __restrict__ zloc,
                                                     int ring_stride, const int* __restrict__ done) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  constexpr int NKE = (DIM == 2) ? 64 : 576;
  const int s = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int part = tid & 3, rq = tid >> 2, nq = nt >> 2;  // quad lane, quad row, quads
  SubBox b;
  sub_box_t<DIM>(g, ax, s, b);
  const BLDesc d = desc[s];
  const int w = d.w, nb = d.nb, ld = lv1_ld(w);
  const int64_t ps = lv1_stride(w, VF);
  const TF* F = pv + d.coff;
  TF* ring = reinterpret_cast<TF*>(sm_raw);
  TF* y = ring + (int64_t)DEPTH * ring_stride;
  TF* z = y + ld;
  TF* v = z + ld;
  TF* ks = v + ((nb * w + 3) & ~3);
  TF* es = ks + NKE;
  int nel = 1;
#pragma unroll
  for (int q = 0; q < DIM; ++q) nel *= b.ehi[q] - b.elo[q];
  uint8_t* fs = reinterpret_cast<uint8_t*>(es + ((nel + 3) & ~3));
  auto fetch = [&](int blk) {
    if (blk >= 0 && blk < nb) {
      const char* src = reinterpret_cast<const char*>(F + (int64_t)blk * ps);
      char* dst = reinterpret_cast<char*>(ring + (int64_t)(blk % DEPTH) * ring_stride);
      const int chunks = (int)(ps * (int64_t)sizeof(TF) / 16);
      for (int c = tid; c < chunks; c += nt) cp_async16(dst + 16 * c, src + 16 * c);
    }
    cp_async_commit();
  };
  // independent of the predecessor kernel (the factors, moduli, free flags
  // and KE are fixed during a solve): issued before the dependency wait
  for (int q = 0; q < DEPTH; ++q) fetch(q);
  auto dof_of = [&](int e) -> int64_t {
    const int k = e / w, p = e % w;
    const int c = p % DIM, t = p / DIM;
    int a[3];
    if (DIM == 2) {
      a[0] = b.nlo[0] + t;
      a[1] = b.nlo[1] + k;
    } else {
      a[0] = b.nlo[0] + t % b.nb3[0];
      a[1] = b.nlo[1] + t / b.nb3[0];
      a[2] = b.nlo[2] + k;
    }
    return DIM * node_id(g, a) + c;
  };
  for (int e = tid; e < nb * w; e += nt) fs[e] = fm[dof_of(e)];
  for (int i = tid; i < NKE; i += nt) ks[i] = ke_const<TF>()[i];
  {
    const int nex = b.ehi[0] - b.elo[0], ney = (DIM == 3) ? b.ehi[1] - b.elo[1] : 1;
    for (int e = tid; e < nel; e += nt) {
      const int ex = b.elo[0] + e % nex;
      const int ey = b.elo[1] + (DIM == 2 ? e / nex : (e / nex) % ney);
      const int64_t ge = (DIM == 2) ? (int64_t)ey * g.nx + ex
                                    : ((int64_t)(b.elo[2] + e / (nex * ney)) * g.ny + ey) * g.nx + ex;
      es[e] = E[ge];
    }
  }
  for (int i = tid; i < 2 * ld; i += nt) y[i] = TF(0);  // y and z; padding stays zero
  pdl_wait();
  if (done && *done) {
    cp_async_wait<0>();
    return;
  }
  __syncthreads();
  // gather R_i r (free DOFs; zero elsewhere)
  for (int e = tid; e < nb * w; e += nt) v[e] = fs[e] ? r[dof_of(e)] : TF(0);
  __syncthreads();
  auto couple = [&](int k, int dir, int p, const TF* xs) -> TF {
    if (DIM == 2) return couple_q4<TF>(b, ks, es, fs, k, dir, p, xs);
    return couple_hex8<TF>(b, ks, es, fs, k, dir, p, xs);
  };
  // out (= or -=) S_k^{-1} y for the line block M in shared memory
  auto apply = [&](const TF* M, TF* out, bool sub) {
    if (VF) {
      // (the quad shuffles need every lane: rows past w run empty loops)
      for (int i0 = 0; i0 < w; i0 += nq) {
        const int i = i0 + rq;
        const bool on = i < w;
        const TF t = quad_row_dot<TF>(M + (on ? lv1_vrow(i) : 0), y, on ? (((i + 1) + 3) & ~3) : 0, part);
        if (on && part == 0) z[i] = t;
      }
      __syncthreads();
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
  };
  // forward: y_k = r_k - A_{k,k-1} u_{k-1};  u_k = S_k^{-1} y_k  (in place)
  for (int k = 0; k < nb; ++k) {
    TF* vk = v + (int64_t)k * w;
    for (int p = tid; p < w; p += nt) y[p] = vk[p] - ((k > 0) ? couple(k, -1, p, vk - w) : TF(0));
    cp_async_wait<DEPTH - 1>();
    __syncthreads();
    apply(ring + (int64_t)(k % DEPTH) * ring_stride, vk, false);
    __syncthreads();
    fetch(k + DEPTH);
  }
  // backward: x_k = u_k - S_k^{-1} (A_{k,k+1} x_{k+1});  x_{nb-1} = u_{nb-1}
  fetch(nb - 1 - DEPTH);
  for (int k = nb - 2; k >= 0; --k) {
    TF* vk = v + (int64_t)k * w;
    for (int p = tid; p < w; p += nt) y[p] = couple(k, +1, p, vk + w);
    cp_async_wait<DEPTH - 1>();
    __syncthreads();
    apply(ring + (int64_t)(k % DEPTH) * ring_stride, vk, true);
    __syncthreads();
    fetch(k - DEPTH);
  }
  pdl_trigger();
  cp_async_wait<0>();
  TF* out = zloc + zoff[s];
  for (int e = tid; e < nb * w; e += nt) out[e] = v[e];
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
  int64_t off = 0, zo = 0;
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
    d.off = off;
    off += bl_size(d.w, d.nb);
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
  const bool vform = h->opt.precision == TS_MIXED_FP32;
  int64_t coff = 0;
  int rs = 0;
  for (int s = 0; s < nsub; ++s) {
    desc[s].coff = coff;
    coff += (int64_t)desc[s].nb * lv1_stride(desc[s].w, vform);
    rs = std::max(rs, (int)lv1_stride(desc[s].w, vform));
  }
  h->pv_len = coff;
  h->pv_stride_max = rs;
  h->sub_desc_h = desc;
  h->zloc_off_h = zoff;
  h->max_w = maxw;
  h->fac_len = off;
  h->zloc_len = zo;
  size_t smem = bl_factor_smem(maxw);
  if (smem > 227 * 1024)
    throw TsError(TS_ERR_INVALID, "local block line too wide for shared memory (w=" + std::to_string(maxw) + ")");
  h->sub_desc = dupload(h, desc);
  h->zloc_off = dupload(h, zoff);
  h->fac64 = dalloc<double>(h, off);
  const bool mixed = h->opt.precision == TS_MIXED_FP32;
  if (mixed) {
    h->pv32 = dalloc<float>(h, coff);
    h->zloc32 = dalloc<float>(h, zo);
    h->E32 = dalloc<float>(h, g.n_el);
  } else {
    h->pv64 = dalloc<double>(h, coff);
    h->zloc = dalloc<double>(h, zo);
  }
  if (g.dim == 2) {
    TS_CUDA(cudaFuncSetAttribute(k_local_factor<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tsl(h), k_local_factor<2><<<nsub, 256, smem, st>>>(g, h->ax, h->E, h->freemask, h->sub_desc, h->fac64, h->dstatus);
  } else {
    TS_CUDA(cudaFuncSetAttribute(k_local_factor<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tsl(h), k_local_factor<3><<<nsub, 256, smem, st>>>(g, h->ax, h->E, h->freemask, h->sub_desc, h->fac64, h->dstatus);
  }
  TS_CUDA(cudaGetLastError());
  {
    const size_t psm = ((size_t)maxw * maxw + maxw) * sizeof(double);
    if (vform) {
      if (psm > 48 * 1024)
        TS_CUDA(cudaFuncSetAttribute(k_pack_level1<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
      tsl(h), k_pack_level1<true><<<nsub, 256, psm, st>>>(h->sub_desc, h->fac64, h->pv64, h->pv32);
    } else {
      if (psm > 48 * 1024)
        TS_CUDA(cudaFuncSetAttribute(k_pack_level1<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
      tsl(h), k_pack_level1<false><<<nsub, 256, psm, st>>>(h->sub_desc, h->fac64, h->pv64, h->pv32);
    }
  }
  if (mixed) tsl(h), k_to_f32<<<256, 256, 0, st>>>(h->E, h->E32, g.n_el);
  TS_CUDA(cudaGetLastError());
  (void)maxn;
}

template <int DIM, class TF, int DEPTH, bool VF>
static void launch_ls(ts_handle h, const TF* r, const TF* pv, const TF* E, TF* zloc, size_t smem) {
  // the limit is raised once, to the maximum, outside any stream capture
  // (the first call of each instantiation precedes the capture of the PCG
  // iteration)
  static bool attr_set = false;
  if (!attr_set) {
    TS_CUDA(cudaFuncSetAttribute(k_local_solve<DIM, TF, DEPTH, VF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 227 * 1024));
    attr_set = true;
  }
  const int threads = std::min(256, 32 * ((4 * h->max_w + 31) / 32));
  ts_launch(h, h->pdl, k_local_solve<DIM, TF, DEPTH, VF>, h->nsub, threads, smem, h->ctx->stream, h->g, h->ax, r,
            (const BLDesc*)h->sub_desc, pv, E, (const uint8_t*)h->freemask, (const int64_t*)h->zloc_off, zloc,
            h->pv_stride_max, (const int*)h->done_flag);
}

template <int DIM, class TF, bool VF>
static void launch_ls_depth(ts_handle h, const TF* r, const TF* pv, const TF* E, TF* zloc) {
  int maxn = 0, maxwp = 0;
  for (auto& d : h->sub_desc_h) {
    maxn = std::max(maxn, d.w * d.nb);
    maxwp = std::max(maxwp, (d.w + 3) & ~3);
  }
  const int nel = h->lv1_max_nel;  // largest element box of a subdomain
  const size_t extra = (size_t)(((maxn + 3) & ~3) - maxn) + ((DIM == 2) ? 64 : 576) + ((nel + 3) & ~3);
  auto need = [&](int depth) {
    return ((size_t)depth * h->pv_stride_max + 2 * (size_t)maxwp + (size_t)maxn + extra) * sizeof(TF) +
           (size_t)maxn;
  };
  // the deeper ring only while every subdomain's CTA stays resident in one
  // wave (CTAs per SM x shared memory within the SM's 228 KB)
  const int per_sm = (h->nsub + h->ctx->n_sm - 1) / h->ctx->n_sm;
  if (need(4) * per_sm <= 220 * 1024)
    launch_ls<DIM, TF, 4, VF>(h, r, pv, E, zloc, need(4));
  else if (need(2) <= 227 * 1024)
    launch_ls<DIM, TF, 2, VF>(h, r, pv, E, zloc, need(2));
  else
    throw TsError(TS_ERR_INVALID, "local solve needs too much shared memory");
}

void launch_local_solve(ts_handle h, const double* r) {
  if (h->opt.precision == TS_MIXED_FP32) {
    // the mixed path reads the FP32 copy of r (kept current by the caller)
    const float* r32 = h->r32;
    if (h->g.dim == 2) launch_ls_depth<2, float, true>(h, r32, h->pv32, h->E32, h->zloc32);
    else launch_ls_depth<3, float, true>(h, r32, h->pv32, h->E32, h->zloc32);
  } else {
    if (h->g.dim == 2) launch_ls_depth<2, double, false>(h, r, h->pv64, h->E, h->zloc);
    else launch_ls_depth<3, double, false>(h, r, h->pv64, h->E, h->zloc);
  }
  TS_CUDA(cudaGetLastError());
}
