// Level 1 of the preconditioner (Eq. localproblemsE):
//   M_1^{-1} r = sum_i R_i^T K_i^{-1} R_i r,  K_i = R_i K R_i^T,
// with R_i the 0/1 restriction to the free DOFs of the nodes of D'_i
// (Eq. def:overlapping-subdomains).  Each K_i is block-tridiagonal by node
// lines and is factored once (FP64 block-line LDL^T, one CTA per subdomain);
// every application gathers R_i r, runs the two sweeps and writes the local
// solution, and a node-owner gather adds the overlapping pieces (no atomics,
// so the sum order is fixed).
#include <algorithm>

#include "ts_blockline.cuh"
#include "ts_internal.cuh"
#include "ts_reduce.cuh"

// element stiffness (E = 1), this translation unit's copy
static __constant__ double c_KE[24 * 24];

void upload_KE_local(ts_handle h, const std::vector<double>& KE) {
  TS_CUDA(cudaMemcpyToSymbolAsync(c_KE, KE.data(), KE.size() * sizeof(double), 0, cudaMemcpyHostToDevice,
                                  h->ctx->stream));
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
// local solve kernel: gather R_i r, block-line sweeps, store local solution
// ---------------------------------------------------------------------------
template <int DIM, class TF>
__global__ void __launch_bounds__(256) k_local_solve(Geom g, AxisTables ax, const double* __restrict__ r,
                                                     const BLDesc* __restrict__ desc, const TF* __restrict__ fac,
                                                     const int64_t* __restrict__ zoff, TF* __restrict__ zloc,
                                                     const int* __restrict__ done) {
  if (done && *done) return;
  extern __shared__ unsigned char sm_raw[];
  TF* v = reinterpret_cast<TF*>(sm_raw);
  const int s = blockIdx.x;
  SubBox b;
  sub_box(g, ax, s, b);
  const BLDesc d = desc[s];
  const int n = d.nb * d.w;
  TF* tmp = v + n;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    int k = e / d.w, p = e % d.w;
    int c = p % DIM, t = p / DIM;
    int a[3];
    if (DIM == 2) {
      a[0] = b.nlo[0] + t;
      a[1] = b.nlo[1] + k;
    } else {
      a[0] = b.nlo[0] + t % b.nb3[0];
      a[1] = b.nlo[1] + t / b.nb3[0];
      a[2] = b.nlo[2] + k;
    }
    v[e] = (TF)r[DIM * node_id(g, a) + c];
  }
  __syncthreads();
  // staging buffers for two factor blocks, 16-byte aligned after v and tmp
  const size_t head = (((size_t)(n + 2 * d.w) * sizeof(TF) + 15) / 16) * 16;
  TF* buf0 = reinterpret_cast<TF*>(sm_raw + head);
  TF* buf1 = buf0 + bl_block_stride(d.w);
  bl_solve_staged<TF>(fac + d.off, d.nb, d.w, v, tmp, buf0, buf1);
  TF* out = zloc + zoff[s];
  for (int e = threadIdx.x; e < n; e += blockDim.x) out[e] = v[e];
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
  h->zloc = dalloc<double>(h, zo);
  if (h->opt.precision == TS_MIXED_FP32) {
    h->fac32 = dalloc<float>(h, off);
    h->zloc32 = dalloc<float>(h, zo);
  }
  if (g.dim == 2) {
    TS_CUDA(cudaFuncSetAttribute(k_local_factor<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tsl(h), k_local_factor<2><<<nsub, 256, smem, st>>>(g, h->ax, h->E, h->freemask, h->sub_desc, h->fac64, h->dstatus);
  } else {
    TS_CUDA(cudaFuncSetAttribute(k_local_factor<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tsl(h), k_local_factor<3><<<nsub, 256, smem, st>>>(g, h->ax, h->E, h->freemask, h->sub_desc, h->fac64, h->dstatus);
  }
  TS_CUDA(cudaGetLastError());
  if (h->fac32) {
    tsl(h), k_to_f32<<<1024, 256, 0, st>>>(h->fac64, h->fac32, off);
    TS_CUDA(cudaGetLastError());
  }
  (void)maxn;
}

template <int DIM, class TF>
static void launch_ls(ts_handle h, const double* r, const TF* fac, TF* zloc, int maxn) {
  const size_t smem = ((((size_t)maxn + 2 * h->max_w) * sizeof(TF) + 15) / 16) * 16 +
                      2 * (size_t)bl_block_stride(h->max_w) * sizeof(TF);
  if (smem > 227 * 1024) throw TsError(TS_ERR_INVALID, "local solve needs too much shared memory");
  // the limit is raised once, to the maximum, outside any stream capture
  // (the first call of each instantiation precedes the capture of the PCG
  // iteration)
  static bool attr_set = false;
  if (!attr_set) {
    TS_CUDA(cudaFuncSetAttribute(k_local_solve<DIM, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr_set = true;
  }
  tsl(h), k_local_solve<DIM, TF><<<h->nsub, 256, smem, h->ctx->stream>>>(h->g, h->ax, r, h->sub_desc, fac,
                                                                         h->zloc_off, zloc, h->done_flag);
}

void launch_local_solve(ts_handle h, const double* r) {
  int maxn = 0;
  for (auto& d : h->sub_desc_h) maxn = std::max(maxn, d.w * d.nb);
  if (h->opt.precision == TS_MIXED_FP32) {
    if (h->g.dim == 2) launch_ls<2, float>(h, r, h->fac32, h->zloc32, maxn);
    else launch_ls<3, float>(h, r, h->fac32, h->zloc32, maxn);
  } else {
    if (h->g.dim == 2) launch_ls<2, double>(h, r, h->fac64, h->zloc, maxn);
    else launch_ls<3, double>(h, r, h->fac64, h->zloc, maxn);
  }
  TS_CUDA(cudaGetLastError());
}
