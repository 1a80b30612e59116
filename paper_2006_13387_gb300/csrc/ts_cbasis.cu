// Coarse basis of M_EH(+Rot) as stored blocks, and the per-iteration coarse
// restriction / prolongation (Sec. 2.1: R_0^T = [Phi_1 ... Phi_Nc]; Sec. 4.1,
// V_{0,H}: chi_l [psi,0], chi_l [0,psi]; Sec. 4.2: chi_l r).
//
// Every basis function of coarse node l lives on the closed box of omega_l.
// A heat basis function chi_l psi e_c has one nonzero component, a rotation
// chi_l (-(y-Y_l), x-X_l) is a closed form.  Per iteration only the products
// W_k = chi_l psi_k over the box (one row per heat DOF, FP32 in the mixed
// path) are streamed:
//   r0_k = sum_i W_k[i] r_c(i)            one CTA per coarse node, r over
//                                         the box staged in shared memory
//   z    += sum_l sum_k Phi_k u0_k        node-owner gather over the <= 2^dim
//                                         coarse nodes whose hat covers it
// with the rotation terms evaluated in place.  The dense blocks
// B_l[i][c][k] = Phi_{first_l + k}(node i, component c) (FP64, setup only)
// serve the Galerkin product K_0 = R_0 K R_0^T, formed block by block for
// pairs of neighbouring coarse nodes.
#include <algorithm>
#include <cmath>

#include "ts_fe_entries.cuh"
#include "ts_internal.cuh"
#include "ts_pcg.cuh"
#include "ts_bpcg.cuh"
#include "ts_reduce.cuh"

// element stiffness (E = 1), this translation unit's copy
static __constant__ double c_KE[TS_KE_SLOTS * TS_KE_SIZE];

void upload_KE_cbasis(int slot, const std::vector<double>& KE) {
  TS_CUDA(cudaMemcpyToSymbol(c_KE, KE.data(), KE.size() * sizeof(double), sizeof(double) * TS_KE_SIZE * slot,
                             cudaMemcpyHostToDevice));
}

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

__device__ __forceinline__ int64_t gnode(const Geom& g, const int* a) {
  if (g.dim == 2) return (int64_t)a[1] * (g.nx + 1) + a[0];
  return ((int64_t)a[2] * (g.ny + 1) + a[1]) * (g.nx + 1) + a[0];
}

// global coordinates of box node i of coarse node N (x fastest)
template <int DIM>
__device__ __forceinline__ void box_node(const CoarseNodeInfo& N, int i, int* a) {
  const int bx = N.hi[0] - N.lo[0] + 1;
  a[0] = N.lo[0] + i % bx;
  if (DIM == 2) {
    a[1] = N.lo[1] + i / bx;
    a[2] = 0;
  } else {
    const int by = N.hi[1] - N.lo[1] + 1;
    a[1] = N.lo[1] + (i / bx) % by;
    a[2] = N.lo[2] + i / (bx * by);
  }
}

template <int DIM>
__device__ __forceinline__ int box_index(const CoarseNodeInfo& N, const int* a) {
  const int bx = N.hi[0] - N.lo[0] + 1;
  if (DIM == 2) return (a[0] - N.lo[0]) + bx * (a[1] - N.lo[1]);
  const int by = N.hi[1] - N.lo[1] + 1;
  return (a[0] - N.lo[0]) + bx * ((a[1] - N.lo[1]) + by * (a[2] - N.lo[2]));
}

// ---------------------------------------------------------------------------
// setup: B_l blocks (FP64, for K_0) and the W rows, one CTA per coarse node.
// The node's record, the kind and mode of its coarse DOFs and the boxes of
// its heat problems are staged in shared memory; the hat is the integer
// product prod_d max(0, H_d - |a_d - Y_d|) times 1 / prod_d H_d.
// ---------------------------------------------------------------------------
struct BasisStage {
  CoarseNodeInfo N;
  int kind[64], mode[64];
  int plo[3][3], pbx[3], pby[3], pnloc[3];
  int64_t pvec[3];
};

template <int DIM>
__device__ void stage_basis(const CoarseView& V, BasisStage& S) {
  if (threadIdx.x == 0) S.N = V.cn[blockIdx.x];
  __syncthreads();
  const int m = S.N.ndof;
  for (int k = threadIdx.x; k < m && k < 64; k += blockDim.x) {
    S.kind[k] = V.cdof_kind[S.N.first_dof + k];
    S.mode[k] = V.cdof_mode[S.N.first_dof + k];
  }
  if (threadIdx.x < DIM) {
    const int c = threadIdx.x;
    if (S.N.prob[c] >= 0) {
      const HeatProb& P = V.hp[S.N.prob[c]];
      for (int d = 0; d < 3; ++d) S.plo[c][d] = P.lo[d];
      S.pbx[c] = P.hi[0] - P.lo[0] + 1;
      S.pby[c] = P.hi[1] - P.lo[1] + 1;
      S.pvec[c] = P.vec_off;
      S.pnloc[c] = P.nloc;
    }
  }
  __syncthreads();
}

// hat numerator of node N at a (0 outside its support)
template <int DIM>
__device__ __forceinline__ int chi_num(const Geom& g, const CoarseNodeInfo& N, const int* a) {
  int v = 1;
#pragma unroll
  for (int d = 0; d < DIM; ++d) v *= max(0, g.H[d] - abs(a[d] - N.idx[d] * g.H[d]));
  return v;
}

template <int DIM>
__global__ void __launch_bounds__(256) k_build_B(CoarseView V, double* __restrict__ B64) {
  __shared__ BasisStage S;
  stage_basis<DIM>(V, S);
  const Geom& g = V.g;
  const CoarseNodeInfo& N = S.N;
  const int m = N.ndof;
  const int per = N.nbox * DIM;
  const int tot = per * m;
  int hprod = 1;
  for (int d = 0; d < DIM; ++d) hprod *= g.H[d];
  const double ih = 1.0 / (double)hprod;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int k = e % m;
    const int t = e / m;
    const int c = t % DIM, i = t / DIM;
    int a[3];
    box_node<DIM>(N, i, a);
    const int num = chi_num<DIM>(g, N, a);
    double v = 0.0;
    if (num != 0 && V.fm[DIM * gnode(g, a) + c]) {
      const double ch = (double)num * ih;
      const int kind = S.kind[k];
      if (kind == TS_VEC_KIND) {
        // M_EE mode: both components, psi stored [mode][box node][component]
        const int li = (a[0] - S.plo[0][0]) +
                       S.pbx[0] * ((a[1] - S.plo[0][1]) + ((DIM == 3) ? S.pby[0] * (a[2] - S.plo[0][2]) : 0));
        v = ch * V.psi[S.pvec[0] + (int64_t)S.mode[k] * DIM * S.pnloc[0] + (int64_t)DIM * li + c];
      } else if (kind < DIM) {
        if (kind == c) {
          const int li = (a[0] - S.plo[c][0]) +
                         S.pbx[c] * ((a[1] - S.plo[c][1]) + ((DIM == 3) ? S.pby[c] * (a[2] - S.plo[c][2]) : 0));
          v = ch * V.psi[S.pvec[c] + (int64_t)S.mode[k] * S.pnloc[c] + li];
        }
      } else {
        double rel[3] = {0, 0, 0};
        for (int d = 0; d < DIM; ++d) rel[d] = (double)(a[d] - N.idx[d] * g.H[d]);
        const int r = kind - DIM;
        double val;
        if (DIM == 2) {
          val = (c == 0) ? -rel[1] : rel[0];
        } else {
          // axis rotations about y_l: x: (0, -z, y); y: (z, 0, -x); z: (-y, x, 0)
          const double R[3][3] = {{0.0, -rel[2], rel[1]}, {rel[2], 0.0, -rel[0]}, {-rel[1], rel[0], 0.0}};
          val = R[r][c];
        }
        v = ch * val;
      }
    }
    B64[N.boff + e] = v;
  }
}

// W[woff + j*nbp + i] = chi_l(i) psi_j(i) for the heat DOFs j of the node
// (components in order), zero padding up to nbp = round_up(nbox, 4)
template <int DIM>
__global__ void __launch_bounds__(256) k_build_W(CoarseView V, double* __restrict__ W64, float* __restrict__ W32) {
  __shared__ BasisStage S;
  stage_basis<DIM>(V, S);
  const Geom& g = V.g;
  const CoarseNodeInfo& N = S.N;
  const int nbp = (N.nbox + 3) & ~3;
  const int tot = N.nh * nbp;
  int hprod = 1;
  for (int d = 0; d < DIM; ++d) hprod *= g.H[d];
  const double ih = 1.0 / (double)hprod;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int j = e / nbp, i = e % nbp;
    double v = 0.0;
    if (i < N.nbox) {
      int a[3];
      box_node<DIM>(N, i, a);
      const int nheat = N.nh - 2 * N.nvec;
      if (j >= nheat) {
        // M_EE mode md: rows x then y
        const int md = (j - nheat) / 2, c = (j - nheat) % 2;
        const int li = (a[0] - S.plo[0][0]) +
                       S.pbx[0] * ((a[1] - S.plo[0][1]) + ((DIM == 3) ? S.pby[0] * (a[2] - S.plo[0][2]) : 0));
        v = ((double)chi_num<DIM>(g, N, a) * ih) *
            V.psi[S.pvec[0] + (int64_t)md * DIM * S.pnloc[0] + (int64_t)DIM * li + c];
      } else {
        int c = 0, md = j;
        while (c < DIM - 1 && md >= N.nmodes[c]) md -= N.nmodes[c++];
        const int li = (a[0] - S.plo[c][0]) +
                       S.pbx[c] * ((a[1] - S.plo[c][1]) + ((DIM == 3) ? S.pby[c] * (a[2] - S.plo[c][2]) : 0));
        v = ((double)chi_num<DIM>(g, N, a) * ih) * V.psi[S.pvec[c] + (int64_t)md * S.pnloc[c] + li];
      }
    }
    if (W64) W64[N.woff + e] = v;
    if (W32) W32[N.woff + e] = (float)v;
  }
}

// hat and rotation of coarse node N at node a in type T (per-iteration use);
// ih[d] = 1 / H_d, so that no division runs per node
template <int DIM, class T>
__device__ __forceinline__ T chi_t(const Geom& g, const CoarseNodeInfo& N, const int* a, const T* ih, T* rel) {
  T v = 1;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int dd = a[d] - N.idx[d] * g.H[d];
    rel[d] = (T)dd;
    const T t = T(1) - (T)abs(dd) * ih[d];
    v *= (t > T(0)) ? t : T(0);
  }
  return v;
}
// component c of rotation q (2D: (-y, x); 3D axis rotations x, y, z)
template <int DIM, class T>
__device__ __forceinline__ T rot_t(int q, int c, const T* rel) {
  if (DIM == 2) return (c == 0) ? -rel[1] : rel[0];
  if (q == 0) return (c == 0) ? T(0) : (c == 1) ? -rel[2] : rel[1];
  if (q == 1) return (c == 0) ? rel[2] : (c == 1) ? T(0) : -rel[0];
  return (c == 0) ? -rel[1] : (c == 1) ? rel[0] : T(0);
}

// ---------------------------------------------------------------------------
// Galerkin product K_0 = R_0 K R_0^T (Sec. 2.1), in three setup kernels:
//   k_stencil  the nodal stencil of K: S[i][nb][r][c] = sum over the elements
//              holding node i and its neighbour nb of E_e KE(i r, nb c)
//   k_kphi     V_l = K B_l for every coarse node l, all its basis columns at
//              once, over the closed box of omega_l (B_l vanishes outside it
//              and on its boundary inside the domain, where chi_l = 0, so
//              neighbours outside the box contribute nothing)
//   k_k0_pair  for each pair of neighbouring coarse nodes (l, l2) taken once,
//              the block K_0[l][l2] = V_l^T B_l2 summed over the nodes the two
//              boxes share, written with its mirror K_0[l2][l]; a heat basis
//              column chi psi e_c has one nonzero component, so its sum runs
//              over component c alone, and the diagonal block of a node is
//              formed as its upper triangle only.
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(256) k_stencil(Geom g, const double* __restrict__ E, double* __restrict__ S) {
  constexpr int NN = (DIM == 2) ? 9 : 27, NE = 1 << DIM, NKE = DIM * NE;
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.n_nodes) return;
  int a[3];
  a[0] = (int)(node % (g.nx + 1));
  if (DIM == 2) {
    a[1] = (int)(node / (g.nx + 1));
    a[2] = 0;
  } else {
    a[1] = (int)((node / (g.nx + 1)) % (g.ny + 1));
    a[2] = (int)(node / ((int64_t)(g.nx + 1) * (g.ny + 1)));
  }
  const double* KE = c_KE + g.ke * TS_KE_SIZE;
  double* out = S + node * (NN * DIM * DIM);
  for (int nb = 0; nb < NN; ++nb) {
    const int o[3] = {nb % 3 - 1, (nb / 3) % 3 - 1, (DIM == 3) ? nb / 9 - 1 : 0};
    double blk[DIM * DIM];
#pragma unroll
    for (int t = 0; t < DIM * DIM; ++t) blk[t] = 0.0;
    for (int q = 0; q < NE; ++q) {
      int ee[3] = {0, 0, 0}, la3[3] = {0, 0, 0}, lb3[3] = {0, 0, 0};
      bool ok = true;
      for (int d = 0; d < DIM; ++d) {
        ee[d] = a[d] - 1 + ((q >> d) & 1);
        la3[d] = a[d] - ee[d];
        lb3[d] = a[d] + o[d] - ee[d];
        if (ee[d] < 0 || ee[d] >= g.n[d] || lb3[d] < 0 || lb3[d] > 1) ok = false;
      }
      if (!ok) continue;
      const double Ee = (DIM == 2) ? E[(int64_t)ee[1] * g.nx + ee[0]] : E[((int64_t)ee[2] * g.ny + ee[1]) * g.nx + ee[0]];
      const int la = (DIM == 2) ? q4_local(la3[0], la3[1]) : hex8_local(la3[0], la3[1], la3[2]);
      const int lb = (DIM == 2) ? q4_local(lb3[0], lb3[1]) : hex8_local(lb3[0], lb3[1], lb3[2]);
#pragma unroll
      for (int r = 0; r < DIM; ++r)
#pragma unroll
        for (int c = 0; c < DIM; ++c) blk[r * DIM + c] += Ee * KE[(DIM * la + r) * NKE + DIM * lb + c];
    }
#pragma unroll
    for (int t = 0; t < DIM * DIM; ++t) out[nb * DIM * DIM + t] = blk[t];
  }
}

// V_l = K B_l in the layout of B ([nbox][DIM][m], m = ndof of node l).
// Block (32, 8): threadIdx.x runs over 32 box nodes, threadIdx.y over the
// basis columns, so that a warp handles one column (one kind of basis
// function) at consecutive nodes.
template <int DIM>
__global__ void __launch_bounds__(256) k_kphi(CoarseView V, const double* __restrict__ S, const double* __restrict__ B,
                                              double* __restrict__ VK) {
  constexpr int NN = (DIM == 2) ? 9 : 27;
  const CoarseNodeInfo& N = V.cn[blockIdx.x];
  const int nbox = N.nbox;
  const int i = blockIdx.y * 32 + threadIdx.x;
  if (i >= nbox) return;
  const int m = N.ndof;
  int a[3];
  box_node<DIM>(N, i, a);
  const double* Si = S + gnode(V.g, a) * (NN * DIM * DIM);
  const double* Bl = B + N.boff;
  for (int k = threadIdx.y; k < m; k += 8) {
    const int kind = V.cdof_kind[N.first_dof + k];
    const int c0 = (kind < DIM) ? kind : 0, c1 = (kind < DIM) ? kind + 1 : DIM;
    double acc[DIM];
#pragma unroll
    for (int r = 0; r < DIM; ++r) acc[r] = 0.0;
    for (int nb = 0; nb < NN; ++nb) {
      const int o[3] = {nb % 3 - 1, (nb / 3) % 3 - 1, (DIM == 3) ? nb / 9 - 1 : 0};
      int b[3] = {a[0] + o[0], a[1] + o[1], a[2] + o[2]};
      bool in = true;
      for (int d = 0; d < DIM; ++d)
        if (b[d] < N.lo[d] || b[d] > N.hi[d]) in = false;
      if (!in) continue;
      const double* Bj = Bl + (int64_t)box_index<DIM>(N, b) * DIM * m + k;
      for (int c = c0; c < c1; ++c) {
        const double bv = Bj[c * m];
#pragma unroll
        for (int r = 0; r < DIM; ++r) acc[r] += Si[(nb * DIM + r) * DIM + c] * bv;
      }
    }
#pragma unroll
    for (int r = 0; r < DIM; ++r) VK[N.boff + ((int64_t)i * DIM + r) * m + k] = acc[r];
  }
}

constexpr int K0_PC = 16;     // shared nodes staged per step in k_k0_pair
constexpr int K0_MAXO = 16;   // outputs per thread (64 x 64 / 256)

// node t of the box [olo, olo + on) (x fastest)
template <int DIM>
__device__ __forceinline__ void overlap_node(const int* olo, const int* on, int t, int* a) {
  a[0] = olo[0] + t % on[0];
  a[1] = olo[1] + (t / on[0]) % on[1];
  a[2] = (DIM == 3) ? olo[2] + t / (on[0] * on[1]) : 0;
}

// Destination of the K_0 entries: the line blocks of the coarse factor.
// Entry (gi, gj) with gi on line qi and gj on line qj lies in the diagonal
// block of qi when qi = qj and in the coupling A_{qi,qi+1} when qj = qi + 1;
// the block below the diagonal (qj = qi - 1) is the transpose of a stored
// coupling and is not kept.
struct K0Out {
  double* A;           // [lines][cw][cw]
  double* C;           // [lines][cw][cw] (lines > 1)
  const int* qline;    // [nc] line of each coarse DOF
  const int* qoff;     // [lines] first DOF of each line
  int cw;
  __device__ __forceinline__ void put(int gi, int gj, double v) const {
    const int qi = qline[gi], qj = qline[gj];
    const int64_t cc = (int64_t)cw * cw;
    const int64_t e = (int64_t)(gi - qoff[qi]) * cw + (gj - qoff[qj]);
    if (qi == qj)
      A[qi * cc + e] = v;
    else if (qj == qi + 1)
      C[qi * cc + e] = v;
  }
};

template <int DIM>
__global__ void __launch_bounds__(256, 2) k_k0_pair(CoarseView V, const int2* __restrict__ pairs,
                                                 const double* __restrict__ B, const double* __restrict__ VK,
                                                 K0Out K0) {
  extern __shared__ double k0s[];
  const int2 pr = pairs[blockIdx.x];
  const CoarseNodeInfo& N = V.cn[pr.x];
  const CoarseNodeInfo& N2 = V.cn[pr.y];
  const int m = N.ndof, m2 = N2.ndof;
  const bool self = pr.x == pr.y;
  double* Vs = k0s;                      // [K0_PC][DIM][m]
  double* Bs = k0s + K0_PC * DIM * m;    // [K0_PC][DIM][m2]
  int olo[3] = {0, 0, 0}, on[3] = {1, 1, 1};
  int ocount = 1;
  for (int d = 0; d < DIM; ++d) {
    olo[d] = max(N.lo[d], N2.lo[d]);
    on[d] = min(N.hi[d], N2.hi[d]) - olo[d] + 1;
    ocount *= on[d];
  }
  // outputs of this thread: (i, j) with i fastest; the diagonal block of a
  // node runs over its upper triangle (j >= i) in packed order
  const int nout = self ? m * (m + 1) / 2 : m * m2;
  // per output: i | j << 8 | c0 << 16 | c1 << 20 (components summed: [c0, c1))
  int code[K0_MAXO];
  double acc[K0_MAXO];
#pragma unroll
  for (int q = 0; q < K0_MAXO; ++q) {
    const int o = threadIdx.x + q * 256;
    int i = 0, j = 0;
    if (self) {
      j = (int)((sqrt(8.0 * o + 1.0) - 1.0) * 0.5);
      while ((j + 1) * (j + 2) / 2 <= o) ++j;
      while (j * (j + 1) / 2 > o) --j;
      i = o - j * (j + 1) / 2;
    } else {
      j = o / max(m, 1);
      i = o - j * m;
    }
    int c0 = 0, c1 = 0;
    if (o < nout) {
      const int kind = V.cdof_kind[N2.first_dof + j];
      c0 = (kind < DIM) ? kind : 0;
      c1 = (kind < DIM) ? kind + 1 : DIM;
    } else {
      i = j = 0;
    }
    code[q] = i | (j << 8) | (c0 << 16) | (c1 << 20);
    acc[q] = 0.0;
  }
  const int sv = DIM * m, sb = DIM * m2;
  for (int p0 = 0; p0 < ocount; p0 += K0_PC) {
    const int pc = min(K0_PC, ocount - p0);
    __syncthreads();
    for (int t = threadIdx.x; t < pc * sv; t += blockDim.x) {
      const int p = t / sv, e = t - p * sv;
      int a[3];
      overlap_node<DIM>(olo, on, p0 + p, a);
      Vs[t] = VK[N.boff + (int64_t)box_index<DIM>(N, a) * sv + e];
    }
    for (int t = threadIdx.x; t < pc * sb; t += blockDim.x) {
      const int p = t / sb, e = t - p * sb;
      int a[3];
      overlap_node<DIM>(olo, on, p0 + p, a);
      Bs[t] = B[N2.boff + (int64_t)box_index<DIM>(N2, a) * sb + e];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < K0_MAXO; ++q) {
      if (threadIdx.x + q * 256 < nout) {
        const int cd = code[q];
        const int i = cd & 0xff, j = (cd >> 8) & 0xff, c0 = (cd >> 16) & 0xf, c1 = (cd >> 20) & 0xf;
        double s = acc[q];
        for (int p = 0; p < pc; ++p)
          for (int c = c0; c < c1; ++c) s += Vs[p * sv + c * m + i] * Bs[p * sb + c * m2 + j];
        acc[q] = s;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < K0_MAXO; ++q) {
    if (threadIdx.x + q * 256 < nout) {
      const int gi = N.first_dof + (code[q] & 0xff), gj = N2.first_dof + ((code[q] >> 8) & 0xff);
      K0.put(gi, gj, acc[q]);
      K0.put(gj, gi, acc[q]);
    }
  }
}

// ---------------------------------------------------------------------------
// r0 = R_0 r: one CTA per coarse node.  r over the node's box (free DOFs,
// component-planar, zero padded) is staged in shared memory in the
// arithmetic type T (FP32 in the mixed path); a warp per heat DOF streams its
// W row with 16-byte loads; rotations are summed from the closed form.
// ---------------------------------------------------------------------------
template <int DIM, class T>
__global__ void __launch_bounds__(256) k_coarse_restrict(CoarseView V, const T* __restrict__ W,
                                                         const T* __restrict__ r, double* __restrict__ r0,
                                                         const int* done) {
  pdl_wait();
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char rs_sm[];
  T* rb = reinterpret_cast<T*>(rs_sm);
  const Geom& g = V.g;
  const CoarseNodeInfo N = V.cn[blockIdx.x];
  if (N.ndof == 0) return;
  const int nbox = N.nbox, nbp = (nbox + 3) & ~3;
  for (int i = threadIdx.x; i < nbp; i += blockDim.x) {
    if (i < nbox) {
      int a[3];
      box_node<DIM>(N, i, a);
      const int64_t dof = DIM * gnode(g, a);
#pragma unroll
      for (int c = 0; c < DIM; ++c) rb[c * nbp + i] = V.fm[dof + c] ? r[dof + c] : T(0);
    } else {
#pragma unroll
      for (int c = 0; c < DIM; ++c) rb[c * nbp + i] = T(0);
    }
  }
  __syncthreads();
  using VT = typename Vec16<T>::T;
  constexpr int NV = Vec16<T>::N;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nheat = N.nh - 2 * N.nvec;
  for (int j = wid; j < N.ndof; j += nw) {
    T s = 0;
    if (j < nheat) {
      int c = 0, m = j;
      while (c < DIM - 1 && m >= N.nmodes[c]) m -= N.nmodes[c++];
      const T* w = W + N.woff + (int64_t)j * nbp;
      const T* x = rb + c * nbp;
      for (int i = lane * NV; i < nbp; i += 32 * NV)
        s += Vec16<T>::dot(*reinterpret_cast<const VT*>(w + i), *reinterpret_cast<const VT*>(x + i));
    } else if (j < nheat + N.nvec) {
      // M_EE mode: its x and y rows against the two components
      const int r = nheat + 2 * (j - nheat);
#pragma unroll
      for (int c = 0; c < DIM && c < 2; ++c) {
        const T* w = W + N.woff + (int64_t)(r + c) * nbp;
        const T* x = rb + c * nbp;
        for (int i = lane * NV; i < nbp; i += 32 * NV)
          s += Vec16<T>::dot(*reinterpret_cast<const VT*>(w + i), *reinterpret_cast<const VT*>(x + i));
      }
    } else {
      const int q = j - nheat - N.nvec;
      T ih[3];
#pragma unroll
      for (int d = 0; d < DIM; ++d) ih[d] = T(1) / (T)g.H[d];
      for (int i = lane; i < nbox; i += 32) {
        int a[3];
        box_node<DIM>(N, i, a);
        T rel[3] = {0, 0, 0};
        const T ch = chi_t<DIM, T>(g, N, a, ih, rel);
        T t = 0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) t += rot_t<DIM, T>(q, c, rel) * rb[c * nbp + i];
        s += ch * t;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) r0[N.first_dof + j] = (double)s;
  }
  pdl_trigger();
}

// ---------------------------------------------------------------------------
// prolongation: z = sum_i R_i^T zloc_i (which & 1) + R_0^T u0 (which & 2),
// node-owner gather (fixed summation order); fused partial dots dv1.z, dv2.z
// ---------------------------------------------------------------------------
constexpr int PRO_THREADS = 256;

template <int DIM, class TZ, class TB>
__global__ void __launch_bounds__(PRO_THREADS, 4) k_prolong(CoarseView V, AxisTables ax, const BLDesc* __restrict__ desc,
                                                         const int64_t* __restrict__ zoff, const TZ* __restrict__ zloc,
                                                         const TB* __restrict__ B, const TB* __restrict__ u0,
                                                         int which, double* __restrict__ z,
                                                         double* __restrict__ partials, const double* __restrict__ dv1,
                                                         const double* __restrict__ dv2, const int* done,
                                                         PcgTail tail) {
  pdl_wait();
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
    // sums in the basis type (FP32 in the mixed path), rounded to FP64 once
    TB zc[DIM];
    for (int c = 0; c < DIM; ++c) zc[c] = TB(0);
    if (which & 1) {
      const int2 cx = ax.cand[0][a[0]], cy = ax.cand[1][a[1]];
      const int2 cz = (DIM == 3) ? ax.cand[2][a[2]] : make_int2(0, -1);
      const int sx[2] = {cx.x, cx.y}, sy[2] = {cy.x, cy.y}, sz[2] = {cz.x, cz.y};
      for (int iz = 0; iz < 2; ++iz) {
        if (sz[iz] < 0) continue;
        for (int iy = 0; iy < 2; ++iy) {
          if (sy[iy] < 0) continue;
          for (int ix = 0; ix < 2; ++ix) {
            if (sx[ix] < 0) continue;
            const int s = sx[ix] + g.nsub[0] * (sy[iy] + g.nsub[1] * sz[iz]);
            const BLDesc d = desc[s];
            const int lx = a[0] - ax.sub_lo[0][sx[ix]], ly = a[1] - ax.sub_lo[1][sy[iy]];
            int64_t base;
            if (DIM == 2) {
              base = zoff[s] + (int64_t)ly * d.w + 2 * lx;
            } else {
              const int nbx = ax.sub_hi[0][sx[ix]] - ax.sub_lo[0][sx[ix]] + 1;
              const int lz = a[2] - ax.sub_lo[2][sz[iz]];
              base = zoff[s] + (int64_t)lz * d.w + 3 * (ly * nbx + lx);
            }
            for (int c = 0; c < DIM; ++c) zc[c] += (TB)zloc[base + c];
          }
        }
      }
    }
    if ((which & 2) && u0) {
      TB ih[3];
#pragma unroll
      for (int d = 0; d < DIM; ++d) ih[d] = TB(1) / (TB)g.H[d];
      int ci[3][2], nci[3];
      for (int d = 0; d < 3; ++d) {
        if (d >= DIM) {
          ci[d][0] = 0;
          nci[d] = 1;
          continue;
        }
        const int b = a[d] / g.H[d];
        nci[d] = 0;
        ci[d][nci[d]++] = b;
        if (a[d] % g.H[d] != 0) ci[d][nci[d]++] = b + 1;
      }
      for (int iz = 0; iz < nci[2]; ++iz)
        for (int iy = 0; iy < nci[1]; ++iy)
          for (int ix = 0; ix < nci[0]; ++ix) {
            const int l = ci[0][ix] + g.ncn[0] * (ci[1][iy] + g.ncn[1] * ci[2][iz]);
            const CoarseNodeInfo& N = V.cn[l];
            if (N.ndof == 0) continue;
            const int i = box_index<DIM>(N, a);
            const int nbp = (N.nbox + 3) & ~3;
            const TB* uu = u0 + N.first_dof;
            const TB* w = B + N.woff + i;
            // eight W entries and coarse values loaded ahead of their
            // multiply-adds (the sums keep their order), so that a warp
            // has several loads in flight
            int j = 0;
            for (int c = 0; c < DIM; ++c) {
              const int nm = N.nmodes[c];
              int m = 0;
              for (; m + 8 <= nm; m += 8, j += 8) {
                TB wv[8], uv[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                  wv[t] = w[(int64_t)(j + t) * nbp];
                  uv[t] = uu[j + t];
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) zc[c] = fma(wv[t], uv[t], zc[c]);
              }
              for (; m < nm; ++m, ++j) zc[c] = fma(w[(int64_t)j * nbp], uu[j], zc[c]);
            }
            // M_EE modes: rows x, y per mode after the heat rows
            for (int md = 0; md < N.nvec; ++md) {
              const TB um = uu[j + md];
              for (int c = 0; c < DIM && c < 2; ++c) zc[c] = fma(w[(int64_t)(j + 2 * md + c) * nbp], um, zc[c]);
            }
            if (N.nrot) {
              TB rel[3] = {0, 0, 0};
              const TB ch = chi_t<DIM, TB>(g, N, a, ih, rel);
              const int r0q = N.nh - N.nvec;  // first rotation DOF: heat DOFs + M_EE modes
              for (int q = 0; q < N.nrot; ++q) {
                const TB uq = ch * uu[r0q + q];
                for (int c = 0; c < DIM; ++c) zc[c] = fma(rot_t<DIM, TB>(q, c, rel), uq, zc[c]);
              }
            }
          }
    }
    for (int c = 0; c < DIM; ++c) {
      const double zd = V.fm[DIM * node + c] ? (double)zc[c] : 0.0;
      z[DIM * node + c] = zd;
      if (dv1) acc1 = fma(dv1[DIM * node + c], zd, acc1);
      if (dv2) acc2 = fma(dv2[DIM * node + c], zd, acc2);
    }
  }
  pdl_trigger();
  if (partials) {
    double v[2] = {acc1, acc2};
    block_sum_n<PRO_THREADS, 2>(v);
    if (threadIdx.x == 0) {
      partials[2 * blockIdx.x] = v[0];
      partials[2 * blockIdx.x + 1] = v[1];
    }
    if (tail.counter && pcg_last_block(tail.counter))
      pcg_conv_beta_last<PRO_THREADS>(tail.S, tail.xr_partials, tail.n_xr, partials, gridDim.x, tail.counter);
  }
}

// ---------------------------------------------------------------------------
// host
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

void build_coarse_basis(ts_handle h) {
  const Geom& g = h->g;
  cudaStream_t st = h->ctx->stream;
  const int dim = g.dim;
  if (h->max_cdof > 64) throw TsError(TS_ERR_INVALID, "more than 64 coarse DOFs at one coarse node");
  h->B64 = salloc<double>(h, h->B_len);
  if (h->opt.precision != TS_FP64)
    h->W32 = dalloc<float>(h, h->W_len);
  else
    h->W64 = dalloc<double>(h, h->W_len);
  CoarseView V = coarse_view(h);
  if (dim == 2) {
    tsl(h), k_build_B<2><<<h->n_cnodes, 256, 0, st>>>(V, h->B64);
    tsl(h), k_build_W<2><<<h->n_cnodes, 256, 0, st>>>(V, h->W64, h->W32);
  } else {
    tsl(h), k_build_B<3><<<h->n_cnodes, 256, 0, st>>>(V, h->B64);
    tsl(h), k_build_W<3><<<h->n_cnodes, 256, 0, st>>>(V, h->W64, h->W32);
  }
  TS_CUDA(cudaGetLastError());
  // shared memory of the restriction: r over the largest box, per component
  {
    int mb = 0;
    for (const CoarseNodeInfo& N : h->cn_h) mb = std::max(mb, (N.nbox + 3) & ~3);
    const size_t es = (h->opt.precision != TS_FP64) ? sizeof(float) : sizeof(double);
    h->restrict_smem = (size_t)mb * dim * es;
    if (h->restrict_smem > 227 * 1024) throw TsError(TS_ERR_INVALID, "coarse neighbourhood too large");
    size_t lim = ts_allow_dynamic_smem(k_coarse_restrict<2, float>, h->ctx->device);
    lim = std::min(lim, ts_allow_dynamic_smem(k_coarse_restrict<2, double>, h->ctx->device));
    lim = std::min(lim, ts_allow_dynamic_smem(k_coarse_restrict<3, float>, h->ctx->device));
    lim = std::min(lim, ts_allow_dynamic_smem(k_coarse_restrict<3, double>, h->ctx->device));
    if (h->restrict_smem > lim) throw TsError(TS_ERR_INVALID, "coarse neighbourhood too large");
  }
  // K_0 goes straight into the line blocks of its factor: the diagonal
  // block of every coarse line and its coupling to the next line (a coarse
  // node couples only to its neighbours, so nothing else is nonzero)
  const int ld = ((h->nc + 63) / 64) * 64;
  h->K0_ld = ld;
  coarse_line_layout(h);
  K0Out k0o;
  {
    const int nl = (int)h->cl_off.size();
    const size_t cc = (size_t)h->cw * h->cw;
    h->K0A = salloc<double>(h, (size_t)nl * cc);
    TS_CUDA(cudaMemsetAsync(h->K0A, 0, sizeof(double) * (size_t)nl * cc, st));
    h->K0C = nullptr;
    if (nl > 1) {
      h->K0C = salloc<double>(h, (size_t)nl * cc);
      TS_CUDA(cudaMemsetAsync(h->K0C, 0, sizeof(double) * (size_t)nl * cc, st));
    }
    std::vector<int> qline(h->nc);
    for (int q = 0; q < nl; ++q)
      for (int i = 0; i < h->cl_wid[q]; ++i) qline[h->cl_off[q] + i] = q;
    k0o.A = h->K0A;
    k0o.C = h->K0C;
    k0o.qline = supload(h, qline);
    k0o.qoff = supload(h, h->cl_off);
    k0o.cw = h->cw;
  }
  // K_0 = R_0 K R_0^T: nodal stencil of K, V_l = K B_l, pair blocks
  {
    const int NN = (dim == 2) ? 9 : 27;
    double* S = salloc<double>(h, (size_t)g.n_nodes * NN * dim * dim);
    double* VK = salloc<double>(h, h->B_len);
    const int nb_st = cdiv(g.n_nodes, 256);
    int max_nbox = 1;
    for (const CoarseNodeInfo& N : h->cn_h) max_nbox = std::max(max_nbox, N.nbox);
    const dim3 gk(h->n_cnodes, cdiv(max_nbox, 32)), bk(32, 8);
    // neighbouring coarse-node pairs, each once (l2 at a lexicographically
    // non-negative offset from l), both with basis functions
    std::vector<int2> pairs;
    for (int l = 0; l < h->n_cnodes; ++l) {
      const CoarseNodeInfo& N = h->cn_h[l];
      if (N.ndof == 0) continue;
      for (int dz = (dim == 3 ? -1 : 0); dz <= (dim == 3 ? 1 : 0); ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            if (dz < 0 || (dz == 0 && (dy < 0 || (dy == 0 && dx < 0)))) continue;
            const int ci[3] = {N.idx[0] + dx, N.idx[1] + dy, N.idx[2] + dz};
            bool ok = true;
            for (int d = 0; d < dim; ++d)
              if (ci[d] < 0 || ci[d] >= g.ncn[d]) ok = false;
            if (!ok) continue;
            const int l2 = ci[0] + g.ncn[0] * (ci[1] + g.ncn[1] * ((dim == 3) ? ci[2] : 0));
            if (h->cn_h[l2].ndof == 0) continue;
            pairs.push_back(make_int2(l, l2));
          }
    }
    int2* dpairs = nullptr;
    if (!pairs.empty()) {
      dpairs = salloc<int2>(h, pairs.size());
      TS_CUDA(cudaMemcpyAsync(dpairs, pairs.data(), sizeof(int2) * pairs.size(), cudaMemcpyHostToDevice, st));
    }
    const size_t smk = (size_t)K0_PC * dim * 2 * h->max_cdof * sizeof(double);
    if (dim == 2) {
      tsl(h), k_stencil<2><<<nb_st, 256, 0, st>>>(g, h->E, S);
      tsl(h), k_kphi<2><<<gk, bk, 0, st>>>(V, S, h->B64, VK);
      if (!pairs.empty()) {
        if (smk > ts_allow_dynamic_smem(k_k0_pair<2>, h->ctx->device))
          throw TsError(TS_ERR_INVALID, "coarse neighbourhood too large for the K_0 assembly");
        tsl(h), k_k0_pair<2><<<(unsigned)pairs.size(), 256, smk, st>>>(V, dpairs, h->B64, VK, k0o);
      }
    } else {
      tsl(h), k_stencil<3><<<nb_st, 256, 0, st>>>(g, h->E, S);
      tsl(h), k_kphi<3><<<gk, bk, 0, st>>>(V, S, h->B64, VK);
      if (!pairs.empty()) {
        if (smk > ts_allow_dynamic_smem(k_k0_pair<3>, h->ctx->device))
          throw TsError(TS_ERR_INVALID, "coarse neighbourhood too large for the K_0 assembly");
        tsl(h), k_k0_pair<3><<<(unsigned)pairs.size(), 256, smk, st>>>(V, dpairs, h->B64, VK, k0o);
      }
    }
  }
  TS_CUDA(cudaGetLastError());
  h->r0 = dalloc<double>(h, ld);
  h->u0 = dalloc<double>(h, ld);
  TS_CUDA(cudaMemsetAsync(h->r0, 0, sizeof(double) * ld, st));
  TS_CUDA(cudaMemsetAsync(h->u0, 0, sizeof(double) * ld, st));
  if (h->opt.precision != TS_FP64) {
    h->u0f = dalloc<float>(h, ld);
    TS_CUDA(cudaMemsetAsync(h->u0f, 0, sizeof(float) * ld, st));
  }
}

template <int DIM, class T>
static void launch_restrict(ts_handle h, const CoarseView& V, const T* W, const T* r) {
  ts_launch(h, h->pdl, k_coarse_restrict<DIM, T>, h->n_cnodes, 256, h->restrict_smem, h->ctx->stream, V, W, r, h->r0,
            (const int*)h->done_flag);
}

void launch_coarse_restrict(ts_handle h, const double* r) {
  if (h->nc == 0) return;
  CoarseView V = coarse_view(h);
  // the mixed path reads the FP32 copy of r (kept current by the caller)
  const bool f32 = h->W32 != nullptr;
  if (h->g.dim == 2) {
    if (f32) launch_restrict<2, float>(h, V, h->W32, (const float*)h->r32);
    else launch_restrict<2, double>(h, V, h->W64, r);
  } else {
    if (f32) launch_restrict<3, float>(h, V, h->W32, (const float*)h->r32);
    else launch_restrict<3, double>(h, V, h->W64, r);
  }
  TS_CUDA(cudaGetLastError());
}

void launch_coarse_apply(ts_handle h, const double* r) {
  if (h->nc == 0) return;
  launch_coarse_restrict(h, r);
  launch_coarse_solve(h);
}

int prolong_blocks(const Geom& g) { return cdiv(g.n_nodes, PRO_THREADS); }

template <int DIM, class TZ, class TB>
static void launch_pro(ts_handle h, const CoarseView& V, const TZ* zloc, const TB* B, const TB* u0, double* z,
                       int which, double* partials, const double* dv1, const double* dv2, PcgTail tail) {
  if (h->nc == 0) u0 = nullptr;
  ts_launch(h, h->pdl, k_prolong<DIM, TZ, TB>, prolong_blocks(h->g), PRO_THREADS, 0, h->ctx->stream, V, h->ax,
            (const BLDesc*)h->sub_desc, (const int64_t*)h->zloc_off, zloc, B, u0, which, z, partials, dv1, dv2,
            (const int*)h->done_flag, tail);
}

void launch_prolong(ts_handle h, double* z, int which, double* partials, const double* dv1, const double* dv2,
                    PcgTail tail) {
  CoarseView V = coarse_view(h);
  const bool mixed = (h->opt.precision != TS_FP64);
  if (h->g.dim == 2) {
    if (mixed) launch_pro<2, float, float>(h, V, h->zloc32, h->W32, h->u0f, z, which, partials, dv1, dv2, tail);
    else launch_pro<2, double, double>(h, V, h->zloc, h->W64, h->u0, z, which, partials, dv1, dv2, tail);
  } else {
    if (mixed) launch_pro<3, float, float>(h, V, h->zloc32, h->W32, h->u0f, z, which, partials, dv1, dv2, tail);
    else launch_pro<3, double, double>(h, V, h->zloc, h->W64, h->u0, z, which, partials, dv1, dv2, tail);
  }
  TS_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Block path (TS_NB columns, 2D, mixed precision): r0 = R_0 r and
// z = sum_i R_i^T zloc_i + R_0^T u0 for every column, each W row read once
// for all columns.  r32, zloc and u0f are FP32 [n][TS_NB]; r0 and z FP64.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_brestrict(CoarseView V, const float* __restrict__ W,
                                                   const float* __restrict__ r, double* __restrict__ r0,
                                                   float* __restrict__ r0f, const int* done) {
  pdl_wait();
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char brs_sm[];
  // r over the box in four planes [component][column half][nbp] of float4
  // (columns 0..3 and 4..7): a warp's reads of consecutive box nodes are
  // consecutive 16-byte words
  float4* rb = reinterpret_cast<float4*>(brs_sm);
  const Geom& g = V.g;
  const CoarseNodeInfo N = V.cn[blockIdx.x];
  if (N.ndof == 0) return;
  const int nbox = N.nbox, nbp = (nbox + 3) & ~3;
  auto plane = [&](int c, int half) { return rb + (int64_t)(2 * c + half) * nbp; };
  // one (box node, component) pair per thread: its TS_NB values as two
  // 16-byte loads
  // (r is zero at Dirichlet DOFs: no mask needed); four pairs in flight
  for (int e0 = threadIdx.x; e0 < nbp * 2; e0 += 4 * 256) {
    float4 v[4][2];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + 256 * u, i = e >> 1, c = e & 1;
      v[u][0] = v[u][1] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < nbox) {
        int a[3];
        box_node<2>(N, i, a);
        const float4* src = reinterpret_cast<const float4*>(r + (2 * gnode(g, a) + c) * TS_NB);
        v[u][0] = src[0];
        v[u][1] = src[1];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + 256 * u, i = e >> 1, c = e & 1;
      if (e < nbp * 2) {
        plane(c, 0)[i] = v[u][0];
        plane(c, 1)[i] = v[u][1];
      }
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nheat = N.nh - 2 * N.nvec;
  for (int j = wid; j < N.ndof; j += nw) {
    float s[TS_NB];
#pragma unroll
    for (int q = 0; q < TS_NB; ++q) s[q] = 0.f;
    if (j < nheat + N.nvec) {
      // a heat DOF: its W row against its component; an M_EE mode: its x
      // and y rows against the two components
      const bool vec = j >= nheat;
      const int r = vec ? nheat + 2 * (j - nheat) : j;
      const int c0 = vec ? 0 : ((j < N.nmodes[0]) ? 0 : 1), c1 = vec ? 2 : c0 + 1;
      for (int c = c0; c < c1; ++c) {
        const float* w = W + N.woff + (int64_t)(r + c - c0) * nbp;
        const float4* p0 = plane(c, 0);
        const float4* p1 = plane(c, 1);
        for (int i = lane; i < nbox; i += 32) {
          const float wv = w[i];
          const float4 a = p0[i];
          const float4 b = p1[i];
          s[0] = fmaf(wv, a.x, s[0]); s[1] = fmaf(wv, a.y, s[1]); s[2] = fmaf(wv, a.z, s[2]); s[3] = fmaf(wv, a.w, s[3]);
          s[4] = fmaf(wv, b.x, s[4]); s[5] = fmaf(wv, b.y, s[5]); s[6] = fmaf(wv, b.z, s[6]); s[7] = fmaf(wv, b.w, s[7]);
        }
      }
    } else {
      const int q = j - nheat - N.nvec;
      const float ih[3] = {1.f / (float)g.H[0], 1.f / (float)g.H[1], 1.f};
      for (int i = lane; i < nbox; i += 32) {
        int a[3];
        box_node<2>(N, i, a);
        float rel[3] = {0, 0, 0};
        const float ch = chi_t<2, float>(g, N, a, ih, rel);
        const float wx = ch * rot_t<2, float>(q, 0, rel), wy = ch * rot_t<2, float>(q, 1, rel);
        const float4 xa = plane(0, 0)[i], xb = plane(0, 1)[i], ya = plane(1, 0)[i], yb = plane(1, 1)[i];
        const float xs[TS_NB] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
        const float ys[TS_NB] = {ya.x, ya.y, ya.z, ya.w, yb.x, yb.y, yb.z, yb.w};
#pragma unroll
        for (int t = 0; t < TS_NB; ++t) s[t] = fmaf(wx, xs[t], fmaf(wy, ys[t], s[t]));
      }
    }
#pragma unroll
    for (int t = 0; t < TS_NB; ++t)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s[t] += __shfl_xor_sync(0xffffffffu, s[t], o);
    if (lane < TS_NB) {
      float v = s[0];
#pragma unroll
      for (int t = 1; t < TS_NB; ++t)
        if (lane == t) v = s[t];
      r0[(int64_t)(N.first_dof + j) * TS_NB + lane] = (double)v;
      r0f[(int64_t)(N.first_dof + j) * TS_NB + lane] = v;
    }
  }
  pdl_trigger();
}

__global__ void __launch_bounds__(PRO_THREADS, 3) k_bprolong(CoarseView V, AxisTables ax,
                                                          const BLDesc* __restrict__ desc,
                                                          const int64_t* __restrict__ zoff,
                                                          const float* __restrict__ zloc, const float* __restrict__ W,
                                                          const float* __restrict__ u0, double* __restrict__ z,
                                                          double* __restrict__ partials,
                                                          const double* __restrict__ dv, const int* done,
                                                          BPcgTail tail) {
  pdl_wait();
  if (done && *done) return;
  const Geom& g = V.g;
  const int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc[1][TS_NB];
#pragma unroll
  for (int t = 0; t < TS_NB; ++t) acc[0][t] = 0.0;
  if (node < g.n_nodes) {
    const int a[3] = {(int)(node % (g.nx + 1)), (int)(node / (g.nx + 1)), 0};
    float zc[2][TS_NB];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int t = 0; t < TS_NB; ++t) zc[c][t] = 0.f;
    // level 1: the local solutions of the <= 4 subdomains holding the node
    {
      const int2 cx = ax.cand[0][a[0]], cy = ax.cand[1][a[1]];
      const int sx[2] = {cx.x, cx.y}, sy[2] = {cy.x, cy.y};
      for (int iy = 0; iy < 2; ++iy) {
        if (sy[iy] < 0) continue;
        for (int ix = 0; ix < 2; ++ix) {
          if (sx[ix] < 0) continue;
          const int s = sx[ix] + g.nsub[0] * sy[iy];
          const int lx = a[0] - ax.sub_lo[0][sx[ix]], ly = a[1] - ax.sub_lo[1][sy[iy]];
          const float4* src = reinterpret_cast<const float4*>(zloc + (zoff[s] + (int64_t)ly * desc[s].w + 2 * lx) * TS_NB);
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const float4 p = src[2 * c], q = src[2 * c + 1];
            zc[c][0] += p.x; zc[c][1] += p.y; zc[c][2] += p.z; zc[c][3] += p.w;
            zc[c][4] += q.x; zc[c][5] += q.y; zc[c][6] += q.z; zc[c][7] += q.w;
          }
        }
      }
    }
    // coarse: the <= 4 coarse nodes whose hat covers the node
    if (u0) {
      const float ih[3] = {1.f / (float)g.H[0], 1.f / (float)g.H[1], 1.f};
      int ci[2][2], nci[2];
      for (int d = 0; d < 2; ++d) {
        const int b = a[d] / g.H[d];
        nci[d] = 0;
        ci[d][nci[d]++] = b;
        if (a[d] % g.H[d] != 0) ci[d][nci[d]++] = b + 1;
      }
      for (int iy = 0; iy < nci[1]; ++iy)
        for (int ix = 0; ix < nci[0]; ++ix) {
          const int l = ci[0][ix] + g.ncn[0] * ci[1][iy];
          const CoarseNodeInfo& N = V.cn[l];
          if (N.ndof == 0) continue;
          const int i = box_index<2>(N, a);
          const int nbp = (N.nbox + 3) & ~3;
          const float* w = W + N.woff + i;
          int j = 0;
          for (int c = 0; c < 2; ++c) {
#pragma unroll 4
            for (int m = 0; m < N.nmodes[c]; ++m, ++j) {
              const float wv = w[(int64_t)j * nbp];
              const float4* up = reinterpret_cast<const float4*>(u0 + (int64_t)(N.first_dof + j) * TS_NB);
              const float4 p = up[0], q = up[1];
              zc[c][0] = fmaf(wv, p.x, zc[c][0]); zc[c][1] = fmaf(wv, p.y, zc[c][1]);
              zc[c][2] = fmaf(wv, p.z, zc[c][2]); zc[c][3] = fmaf(wv, p.w, zc[c][3]);
              zc[c][4] = fmaf(wv, q.x, zc[c][4]); zc[c][5] = fmaf(wv, q.y, zc[c][5]);
              zc[c][6] = fmaf(wv, q.z, zc[c][6]); zc[c][7] = fmaf(wv, q.w, zc[c][7]);
            }
          }
          // M_EE modes: rows x, y per mode after the heat rows (j = the heat DOFs)
          for (int md = 0; md < N.nvec; ++md) {
            const float wx = w[(int64_t)(j + 2 * md) * nbp], wy = w[(int64_t)(j + 2 * md + 1) * nbp];
            const float4* up = reinterpret_cast<const float4*>(u0 + (int64_t)(N.first_dof + j + md) * TS_NB);
            const float4 p = up[0], q = up[1];
            const float uv[TS_NB] = {p.x, p.y, p.z, p.w, q.x, q.y, q.z, q.w};
#pragma unroll
            for (int t = 0; t < TS_NB; ++t) {
              zc[0][t] = fmaf(wx, uv[t], zc[0][t]);
              zc[1][t] = fmaf(wy, uv[t], zc[1][t]);
            }
          }
          if (N.nrot) {
            float rel[3] = {0, 0, 0};
            const float ch = chi_t<2, float>(g, N, a, ih, rel);
            const float wx = ch * rot_t<2, float>(0, 0, rel), wy = ch * rot_t<2, float>(0, 1, rel);
            const float* uq = u0 + (int64_t)(N.first_dof + N.nh - N.nvec) * TS_NB;
#pragma unroll
            for (int t = 0; t < TS_NB; ++t) {
              zc[0][t] = fmaf(wx, uq[t], zc[0][t]);
              zc[1][t] = fmaf(wy, uq[t], zc[1][t]);
            }
          }
        }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const bool fr = V.fm[2 * node + c] != 0;
      double2* zo = reinterpret_cast<double2*>(z + (2 * node + c) * TS_NB);
      const double2* dvp = dv ? reinterpret_cast<const double2*>(dv + (2 * node + c) * TS_NB) : nullptr;
#pragma unroll
      for (int t = 0; t < TS_NB; t += 2) {
        const double z0 = fr ? (double)zc[c][t] : 0.0, z1 = fr ? (double)zc[c][t + 1] : 0.0;
        zo[t / 2] = make_double2(z0, z1);
        if (dvp) {
          const double2 d = dvp[t / 2];
          acc[0][t] = fma(d.x, z0, acc[0][t]);
          acc[0][t + 1] = fma(d.y, z1, acc[0][t + 1]);
        }
      }
    }
  }
  pdl_trigger();
  if (partials) {
    bsum_all_cols<PRO_THREADS, 1>(acc);
    if (threadIdx.x == 0)
#pragma unroll
      for (int t = 0; t < TS_NB; ++t) partials[(int64_t)blockIdx.x * TS_NB + t] = acc[0][t];
    if (tail.counter && pcg_last_block(tail.counter))
      bpcg_conv_beta_last<PRO_THREADS>(tail.S, tail.xr_partials, tail.n_xr, partials, gridDim.x, tail.counter);
  }
}

int bprolong_blocks(const Geom& g) { return cdiv(g.n_nodes, PRO_THREADS); }

void launch_brestrict(ts_handle h, const float* r32, double* r0) {
  if (h->nc == 0) return;
  if (h->g.dim != 2 || !h->W32) throw TsError(TS_ERR_INVALID, "internal: block restriction needs a mixed 2D design");
  int mb = 0;
  for (const CoarseNodeInfo& N : h->cn_h) mb = std::max(mb, (N.nbox + 3) & ~3);
  const size_t smem = (size_t)mb * 2 * TS_NB * sizeof(float);
  if (smem > ts_allow_dynamic_smem(k_brestrict, h->ctx->device))
    throw TsError(TS_ERR_INVALID, "coarse neighbourhood too large for the block restriction");
  ts_launch(h, h->pdl, k_brestrict, h->n_cnodes, 256, smem, h->ctx->stream, coarse_view(h), (const float*)h->W32, r32,
            r0, h->r0b32, (const int*)h->done_flag);
  TS_CUDA(cudaGetLastError());
}

void launch_bprolong(ts_handle h, const float* zloc, const float* u0f, double* z, double* partials, const double* dv,
                     BPcgTail tail) {
  if (h->g.dim != 2) throw TsError(TS_ERR_INVALID, "internal: block prolongation is 2D only");
  const bool coarse = h->opt.coarse && h->nc > 0;
  ts_launch(h, h->pdl, k_bprolong, bprolong_blocks(h->g), PRO_THREADS, 0, h->ctx->stream, coarse_view(h), h->ax,
            (const BLDesc*)h->sub_desc, (const int64_t*)h->zloc_off, zloc, (const float*)h->W32,
            coarse ? u0f : (const float*)nullptr, z, partials, dv, (const int*)h->done_flag, tail);
  TS_CUDA(cudaGetLastError());
}
