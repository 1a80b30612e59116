// Finite-element operators on the device: SIMP moduli (Eq. 4) and the
// matrix-free stiffness product y = K(rho) x (Eq. 2 with the Q4 / Hex8
// discretisation of Sec. 1.1), Dirichlet rows and columns masked.
#include <cmath>
#include <map>

#include "ts_fe_entries.cuh"
#include "ts_internal.cuh"
#include "ts_pcg.cuh"
#include "ts_bpcg.cuh"
#include "ts_reduce.cuh"

// element stiffness slots (E = 1); one copy per translation unit (no
// relocatable device code), each filled by its own upload function
static __constant__ double c_KE[TS_KE_SLOTS * TS_KE_SIZE];

// ---------------------------------------------------------------------------
// host: element stiffness E = 1 by 2-point Gauss quadrature per axis
// ---------------------------------------------------------------------------
void ts_element_matrices(int dim, double nu, std::vector<double>& KE) {
  const double gp[2] = {-1.0 / std::sqrt(3.0), 1.0 / std::sqrt(3.0)};
  if (dim == 2) {
    // plane stress D = 1/(1-nu^2) [[1,nu,0],[nu,1,0],[0,0,(1-nu)/2]]
    double D[3][3] = {{1, nu, 0}, {nu, 1, 0}, {0, 0, 0.5 * (1 - nu)}};
    for (auto& r : D)
      for (double& v : r) v /= (1 - nu * nu);
    const int sx[4] = {-1, 1, 1, -1}, sy[4] = {-1, -1, 1, 1};
    KE.assign(64, 0.0);
    for (double xi : gp)
      for (double eta : gp) {
        double B[3][8] = {};
        for (int a = 0; a < 4; ++a) {
          // dN/dx = 2 * dN/dxi on the unit element
          double dx = 2.0 * 0.25 * sx[a] * (1 + sy[a] * eta);
          double dy = 2.0 * 0.25 * sy[a] * (1 + sx[a] * xi);
          B[0][2 * a] = dx;
          B[1][2 * a + 1] = dy;
          B[2][2 * a] = dy;
          B[2][2 * a + 1] = dx;
        }
        for (int i = 0; i < 8; ++i)
          for (int j = 0; j < 8; ++j) {
            double s = 0;
            for (int p = 0; p < 3; ++p)
              for (int q = 0; q < 3; ++q) s += B[p][i] * D[p][q] * B[q][j];
            KE[i * 8 + j] += 0.25 * s;
          }
      }
  } else {
    double lam = nu / ((1 + nu) * (1 - 2 * nu)), mu = 1.0 / (2 * (1 + nu));
    double D[6][6] = {};
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) D[i][j] = lam;
      D[i][i] += 2 * mu;
      D[3 + i][3 + i] = mu;
    }
    const int sx[8] = {-1, 1, 1, -1, -1, 1, 1, -1}, sy[8] = {-1, -1, 1, 1, -1, -1, 1, 1},
              sz[8] = {-1, -1, -1, -1, 1, 1, 1, 1};
    KE.assign(576, 0.0);
    for (double xi : gp)
      for (double eta : gp)
        for (double zeta : gp) {
          double B[6][24] = {};
          for (int a = 0; a < 8; ++a) {
            double dx = 2.0 * 0.125 * sx[a] * (1 + sy[a] * eta) * (1 + sz[a] * zeta);
            double dy = 2.0 * 0.125 * sy[a] * (1 + sx[a] * xi) * (1 + sz[a] * zeta);
            double dz = 2.0 * 0.125 * sz[a] * (1 + sx[a] * xi) * (1 + sy[a] * eta);
            B[0][3 * a] = dx;
            B[1][3 * a + 1] = dy;
            B[2][3 * a + 2] = dz;
            B[3][3 * a + 1] = dz;
            B[3][3 * a + 2] = dy;
            B[4][3 * a] = dz;
            B[4][3 * a + 2] = dx;
            B[5][3 * a] = dy;
            B[5][3 * a + 1] = dx;
          }
          for (int i = 0; i < 24; ++i)
            for (int j = 0; j < 24; ++j) {
              double s = 0;
              for (int p = 0; p < 6; ++p)
                for (int q = 0; q < 6; ++q) s += B[p][i] * D[p][q] * B[q][j];
              KE[i * 24 + j] += 0.125 * s;
            }
        }
  }
}

static void upload_KE_fem(int slot, const std::vector<double>& KE) {
  TS_CUDA(cudaMemcpyToSymbol(c_KE, KE.data(), KE.size() * sizeof(double), sizeof(double) * TS_KE_SIZE * slot,
                             cudaMemcpyHostToDevice));
}

namespace {
struct KeSlot {
  int dim = 0;
  double nu = 0.0;
  int refs = 0;
};
std::mutex g_ke_mu;
std::map<int, std::vector<KeSlot>> g_ke;  // per device
}  // namespace

void ts_ke_acquire(ts_handle h) {
  std::lock_guard<std::mutex> lk(g_ke_mu);
  std::vector<KeSlot>& t = g_ke[h->ctx->device];
  t.resize(TS_KE_SLOTS);
  int slot = -1;
  for (int i = 0; i < TS_KE_SLOTS && slot < 0; ++i)
    if (t[i].refs > 0 && t[i].dim == h->g.dim && t[i].nu == h->nu) slot = i;
  if (slot < 0) {
    for (int i = 0; i < TS_KE_SLOTS && slot < 0; ++i)
      if (t[i].refs == 0) slot = i;
    if (slot < 0)
      throw TsError(TS_ERR_BUSY, "more than 8 distinct element matrices (dimension, nu) in use at once");
    // a free slot is read by no kernel in flight (its last design has been
    // destroyed after its streams drained); the copies are synchronous
    std::vector<double> KE;
    ts_element_matrices(h->g.dim, h->nu, KE);
    upload_KE_fem(slot, KE);
    upload_KE_local(slot, KE);
    upload_KE_cbasis(slot, KE);
    upload_KE_coarse(slot, KE);
    t[slot].dim = h->g.dim;
    t[slot].nu = h->nu;
  }
  t[slot].refs += 1;
  h->ke_slot = slot;
  h->g.ke = slot;
}

void ts_ke_release(ts_handle h) {
  if (h->ke_slot < 0) return;
  std::lock_guard<std::mutex> lk(g_ke_mu);
  g_ke[h->ctx->device][h->ke_slot].refs -= 1;
  h->ke_slot = -1;
}

// ---------------------------------------------------------------------------
// SIMP: E_e = Emin + rho_e^p (E0 - Emin)        (Eq. 4)
// ---------------------------------------------------------------------------
__global__ void k_simp(const double* __restrict__ rho, double* __restrict__ E, int64_t n, double E0, double Emin,
                       double p) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    double r = rho[i];
    double rp = (p == 3.0) ? r * r * r : pow(r, p);
    E[i] = Emin + rp * (E0 - Emin);
  }
}

// Nodal stencil of K, masked at Dirichlet DOFs, coefficient-major:
// St[((nb * DIM + r) * DIM + c) * n_nodes + node] = sum over the elements
// holding the node and its neighbour nb (offsets x fastest in {-1,0,1}^DIM)
// of E_e KE(node r, nb c); zero when either DOF is Dirichlet.
template <int DIM>
__global__ void __launch_bounds__(256) k_stencil_soa(Geom g, const double* __restrict__ E,
                                                     const uint8_t* __restrict__ fm, double* __restrict__ St) {
  constexpr int NN = (DIM == 2) ? 9 : 27, NE = 1 << DIM, NKE = DIM * NE;
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.n_nodes) return;
  const int64_t nn = g.n_nodes;
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
  for (int nb = 0; nb < NN; ++nb) {
    const int o[3] = {nb % 3 - 1, (nb / 3) % 3 - 1, (DIM == 3) ? nb / 9 - 1 : 0};
    double blk[DIM * DIM];
#pragma unroll
    for (int t = 0; t < DIM * DIM; ++t) blk[t] = 0.0;
    bool nb_in = true;
    for (int d = 0; d < DIM; ++d)
      if (a[d] + o[d] < 0 || a[d] + o[d] > g.n[d]) nb_in = false;
    int64_t nbn = -1;
    if (nb_in) {
      nbn = (DIM == 2) ? (int64_t)(a[1] + o[1]) * (g.nx + 1) + a[0] + o[0]
                       : ((int64_t)(a[2] + o[2]) * (g.ny + 1) + a[1] + o[1]) * (g.nx + 1) + a[0] + o[0];
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
    }
#pragma unroll
    for (int r = 0; r < DIM; ++r)
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        const bool free_rc = fm[DIM * node + r] && nbn >= 0 && fm[DIM * nbn + c];
        St[(int64_t)((nb * DIM + r) * DIM + c) * nn + node] = free_rc ? blk[r * DIM + c] : 0.0;
      }
  }
}

void launch_stencil(ts_handle h, double* St) {
  const Geom& g = h->g;
  if (g.dim == 2)
    tsl(h), k_stencil_soa<2><<<cdiv(g.n_nodes, 256), 256, 0, h->ctx->stream>>>(g, h->E, h->freemask, St);
  else
    tsl(h), k_stencil_soa<3><<<cdiv(g.n_nodes, 256), 256, 0, h->ctx->stream>>>(g, h->E, h->freemask, St);
  TS_CUDA(cudaGetLastError());
}

void launch_simp(ts_handle h, const double* rho, double* E) {
  int64_t n = h->g.n_el;
  tsl(h), k_simp<<<cdiv(n, 256), 256, 0, h->ctx->stream>>>(rho, E ? E : h->E, n, h->E0, h->Emin, h->p);
  TS_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// y = K x, node-centric gather: each thread owns one node, sums E_e KE_e x_e
// over the elements around it.  Dirichlet DOFs: x is read as 0 there and
// y is written as 0.  Optional fused partial dot sum_i dotvec_i * y_i.
// ---------------------------------------------------------------------------
constexpr int SPMV_THREADS = 256;

// Q4: one CTA per tile of SX x SY nodes.  x (zero at Dirichlet DOFs) over
// the tile plus a one-node halo and E over the tile's elements (zero outside
// the mesh) are staged in shared memory, so each node's 64 FMAs read shared
// memory only and need no bounds tests.
constexpr int SX = 32, SY = SPMV_THREADS / 32;

// Optional fused search-direction update of the PCG iteration: the vector
// multiplied is p = z + beta p_old (beta from the PCG scalars), computed while
// staging; the tile's own nodes write p to p_new (and z to z_old for the
// flexible variant), and the dot partial is p.Kp.
struct PUpdate {
  const double* z;      // null: multiply x as given
  const double* p_old;
  double* p_new;
  double* z_old;        // may be null
};

// ST: the node's 9-point stencil of K (36 FP64 coefficients, masked at
// Dirichlet DOFs, stored coefficient-major: St[k * n_nodes + node]) replaces
// the element products: 36 FMAs per node and coalesced coefficient loads.
template <bool ST>
__global__ void __launch_bounds__(SPMV_THREADS) k_spmv_q4(Geom g, const double* __restrict__ E,
                                                           const uint8_t* __restrict__ fm,
                                                           const double* __restrict__ x, double* __restrict__ y,
                                                           double* __restrict__ partial,
                                                           const double* __restrict__ dotvec, const int* done,
                                                           DevScalars* S, unsigned* counter, PUpdate pu,
                                                           const double* __restrict__ St) {
  __shared__ double xs[SY + 2][SX + 2][2];
  __shared__ double es[ST ? 1 : SY + 1][ST ? 1 : SX + 1];
  const int nx = g.nx, ny = g.ny, nnx = nx + 1;
  const int x0 = blockIdx.x * SX, y0 = blockIdx.y * SY, tid = threadIdx.x;
  const int ko = g.ke * TS_KE_SIZE;  // this design's element stiffness
  // moduli do not change during a solve: staged before the dependency wait
  if (!ST)
    for (int e = tid; e < (SY + 1) * (SX + 1); e += SPMV_THREADS) {
      const int ly = e / (SX + 1), lx = e % (SX + 1);
      const int ex = x0 - 1 + lx, ey = y0 - 1 + ly;
      es[ly][lx] = (ex >= 0 && ex < nx && ey >= 0 && ey < ny) ? __ldg(&E[(int64_t)ey * nx + ex]) : 0.0;
    }
  pdl_wait();
  if (done && *done) return;
  const bool fused = pu.z != nullptr;
  const double beta = fused ? S->beta : 0.0;
  for (int e = tid; e < (SY + 2) * (SX + 2); e += SPMV_THREADS) {
    const int ly = e / (SX + 2), lx = e % (SX + 2);
    const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
    double ux = 0.0, uy = 0.0;
    if (gx >= 0 && gx <= nx && gy >= 0 && gy <= ny) {
      const int64_t nd = (int64_t)gy * nnx + gx;
      if (fused) {
        const double zx = pu.z[2 * nd], zy = pu.z[2 * nd + 1];
        if (fm[2 * nd]) ux = fma(beta, pu.p_old[2 * nd], zx);
        if (fm[2 * nd + 1]) uy = fma(beta, pu.p_old[2 * nd + 1], zy);
        if (lx >= 1 && lx <= SX && ly >= 1 && ly <= SY) {  // a node of this tile
          pu.p_new[2 * nd] = ux;
          pu.p_new[2 * nd + 1] = uy;
          if (pu.z_old) {
            pu.z_old[2 * nd] = zx;
            pu.z_old[2 * nd + 1] = zy;
          }
        }
      } else {
        if (fm[2 * nd]) ux = x[2 * nd];
        if (fm[2 * nd + 1]) uy = x[2 * nd + 1];
      }
    }
    xs[ly][lx][0] = ux;
    xs[ly][lx][1] = uy;
  }
  __syncthreads();
  const int lx = tid % SX, ly = tid / SX;
  const int i = x0 + lx, j = y0 + ly;
  double acc = 0.0;
  if (ST && i <= nx && j <= ny) {
    const int64_t nn = g.n_nodes, node = (int64_t)j * nnx + i;
    double yx = 0.0, yy = 0.0;
#pragma unroll
    for (int nb = 0; nb < 9; ++nb) {
      const double* xv = xs[ly + 1 + nb / 3 - 1][lx + 1 + nb % 3 - 1];
      const double* sc = St + (int64_t)(4 * nb) * nn + node;
      yx = fma(__ldg(sc), xv[0], yx);
      yx = fma(__ldg(sc + nn), xv[1], yx);
      yy = fma(__ldg(sc + 2 * nn), xv[0], yy);
      yy = fma(__ldg(sc + 3 * nn), xv[1], yy);
    }
    if (!fm[2 * node]) yx = 0.0;
    if (!fm[2 * node + 1]) yy = 0.0;
    y[2 * node] = yx;
    y[2 * node + 1] = yy;
    if (fused)
      acc = fma(xs[ly + 1][lx + 1][0], yx, xs[ly + 1][lx + 1][1] * yy);
    else if (dotvec)
      acc = fma(dotvec[2 * node], yx, dotvec[2 * node + 1] * yy);
  } else if (!ST && i <= nx && j <= ny) {
    double yx = 0.0, yy = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      // element (i-1+(q&1), j-1+(q>>1)); its nodes sit at xs[ly+(q>>1)+{0,1}][lx+(q&1)+{0,1}]
      const int ox = lx + (q & 1), oy = ly + (q >> 1);
      const int la = (q == 0) ? 2 : (q == 1) ? 3 : (q == 2) ? 1 : 0;
      const double Ee = es[oy][ox];
      const double* n0 = xs[oy][ox];
      const double* n1 = xs[oy][ox + 1];
      const double* n2 = xs[oy + 1][ox + 1];
      const double* n3 = xs[oy + 1][ox];
      const double* nb[4] = {n0, n1, n2, n3};
      // two FMA chains per element (one DFMA per matrix entry)
      double sx = 0.0, sy = 0.0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const double ux = nb[b][0], uy = nb[b][1];
        sx = fma(c_KE[ko + (2 * la) * 8 + 2 * b], ux, sx);
        sx = fma(c_KE[ko + (2 * la) * 8 + 2 * b + 1], uy, sx);
        sy = fma(c_KE[ko + (2 * la + 1) * 8 + 2 * b], ux, sy);
        sy = fma(c_KE[ko + (2 * la + 1) * 8 + 2 * b + 1], uy, sy);
      }
      yx = fma(Ee, sx, yx);
      yy = fma(Ee, sy, yy);
    }
    const int64_t node = (int64_t)j * nnx + i;
    if (!fm[2 * node]) yx = 0.0;
    if (!fm[2 * node + 1]) yy = 0.0;
    y[2 * node] = yx;
    y[2 * node + 1] = yy;
    if (fused)
      acc = fma(xs[ly + 1][lx + 1][0], yx, xs[ly + 1][lx + 1][1] * yy);
    else if (dotvec)
      acc = fma(dotvec[2 * node], yx, dotvec[2 * node + 1] * yy);
  }
  // the successor may be scheduled once this block has done its main work
  pdl_trigger();
  if (partial) {
    double v[1] = {acc};
    block_sum_n<SPMV_THREADS, 1>(v);
    const double s = v[0];
    if (tid == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = s;
    if (counter && pcg_last_block(counter)) pcg_alpha_last<SPMV_THREADS>(S, partial, gridDim.x * gridDim.y, counter);
  }
}

__global__ void __launch_bounds__(SPMV_THREADS) k_spmv_hex8(Geom g, const double* __restrict__ E,
                                                             const uint8_t* __restrict__ fm,
                                                             const double* __restrict__ x, double* __restrict__ y,
                                                             double* __restrict__ partial,
                                                             const double* __restrict__ dotvec, const int* done, DevScalars* S,
                                                             unsigned* counter) {
  pdl_wait();
  if (done && *done) return;
  const int nx = g.nx, ny = g.ny, nz = g.nz, nnx = nx + 1, nny = ny + 1;
  const int ko = g.ke * TS_KE_SIZE;  // this design's element stiffness
  int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (node < g.n_nodes) {
    int i = (int)(node % nnx);
    int j = (int)((node / nnx) % nny);
    int k = (int)(node / ((int64_t)nnx * nny));
    double yv[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < 8; ++q) {
      int ex = i - 1 + (q & 1), ey = j - 1 + ((q >> 1) & 1), ez = k - 1 + (q >> 2);
      if (ex < 0 || ex >= nx || ey < 0 || ey >= ny || ez < 0 || ez >= nz) continue;
      // local index of this node: offsets (i-ex, j-ey, k-ez) in {0,1}^3
      int ox = i - ex, oy = j - ey, oz = k - ez;
      int la = (oz ? 4 : 0) + (oy ? (ox ? 2 : 3) : (ox ? 1 : 0));
      double Ee = __ldg(&E[((int64_t)ez * ny + ey) * nx + ex]);
      int64_t n0 = ((int64_t)ez * nny + ey) * nnx + ex;
      int64_t nd[8] = {n0, n0 + 1, n0 + nnx + 1, n0 + nnx};
      int64_t pl = (int64_t)nnx * nny;
      for (int b = 0; b < 4; ++b) nd[4 + b] = nd[b] + pl;
      double s[3] = {0.0, 0.0, 0.0};
      for (int b = 0; b < 8; ++b) {
        double u[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) u[c] = fm[3 * nd[b] + c] ? __ldg(&x[3 * nd[b] + c]) : 0.0;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c) s[r] += c_KE[ko + (3 * la + r) * 24 + 3 * b + c] * u[c];
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) yv[r] += Ee * s[r];
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (!fm[3 * node + r]) yv[r] = 0.0;
      y[3 * node + r] = yv[r];
      if (dotvec) acc += dotvec[3 * node + r] * yv[r];
    }
  }
  pdl_trigger();
  if (partial) {
    double s = block_sum<SPMV_THREADS>(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
    if (counter && pcg_last_block(counter)) pcg_alpha_last<SPMV_THREADS>(S, partial, gridDim.x, counter);
  }
}

// SpMV grid: 2D tiles of SX x SY nodes, 3D one thread per node
static dim3 spmv_grid(const Geom& g) {
  if (g.dim == 2) return dim3(cdiv(g.nx + 1, SX), cdiv(g.ny + 1, SY), 1);
  return dim3(cdiv(g.n_nodes, SPMV_THREADS), 1, 1);
}
int spmv_blocks(const Geom& g) {
  const dim3 d = spmv_grid(g);
  return (int)(d.x * d.y);
}
int node_blocks(const Geom& g) { return cdiv(g.n_nodes, SPMV_THREADS); }

void launch_spmv(ts_handle h, const double* x, double* y, double* partial, const double* dotvec, DevScalars* S,
                 unsigned* counter) {
  const Geom& g = h->g;
  const dim3 nb = spmv_grid(g);
  if (g.dim == 2 && h->kst)
    ts_launch(h, h->pdl, k_spmv_q4<true>, nb, SPMV_THREADS, 0, h->ctx->stream, g, (const double*)h->E,
              (const uint8_t*)h->freemask, x, y, partial, dotvec, (const int*)h->done_flag, S, counter,
              PUpdate{nullptr, nullptr, nullptr, nullptr}, (const double*)h->kst);
  else if (g.dim == 2)
    ts_launch(h, h->pdl, k_spmv_q4<false>, nb, SPMV_THREADS, 0, h->ctx->stream, g, (const double*)h->E,
              (const uint8_t*)h->freemask, x, y, partial, dotvec, (const int*)h->done_flag, S, counter,
              PUpdate{nullptr, nullptr, nullptr, nullptr}, (const double*)nullptr);
  else
    ts_launch(h, h->pdl, k_spmv_hex8, nb, SPMV_THREADS, 0, h->ctx->stream, g, (const double*)h->E,
              (const uint8_t*)h->freemask, x, y, partial, dotvec, (const int*)h->done_flag, S, counter);
  TS_CUDA(cudaGetLastError());
}

// q = K p with p = z + beta p_old formed on the fly (2D Q4 only): p to
// p_new, z to z_old (if given), partials of p.q and alpha from the last block
void launch_spmv_fused_p(ts_handle h, const double* z, const double* p_old, double* p_new, double* z_old, double* q,
                         double* partial, DevScalars* S, unsigned* counter) {
  const Geom& g = h->g;
  if (g.dim != 2) throw TsError(TS_ERR_INVALID, "internal: fused search-direction update is 2D only");
  if (h->kst)
    ts_launch(h, h->pdl, k_spmv_q4<true>, spmv_grid(g), SPMV_THREADS, 0, h->ctx->stream, g, (const double*)h->E,
              (const uint8_t*)h->freemask, (const double*)nullptr, q, partial, (const double*)nullptr,
              (const int*)h->done_flag, S, counter, PUpdate{z, p_old, p_new, z_old}, (const double*)h->kst);
  else
    ts_launch(h, h->pdl, k_spmv_q4<false>, spmv_grid(g), SPMV_THREADS, 0, h->ctx->stream, g, (const double*)h->E,
              (const uint8_t*)h->freemask, (const double*)nullptr, q, partial, (const double*)nullptr,
              (const int*)h->done_flag, S, counter, PUpdate{z, p_old, p_new, z_old}, (const double*)nullptr);
  TS_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// r = f - K x with every product formed exactly (FMA two-product) and every
// sum compensated (two-sum): a double-double accumulator per output, rounded
// to FP64 at the end.  Used once or twice per solve to see the true residual
// below FP64's own summation noise.
// ---------------------------------------------------------------------------
struct DD {
  double hi, lo;
};

__device__ __forceinline__ DD dd_two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

// acc += a * b * c (a, b, c FP64), the product a*b kept as a double-double
__device__ __forceinline__ void dd_add_prod3(DD& acc, double a, double b, double c) {
  double p = a * b;
  double pe = fma(a, b, -p);      // a*b = p + pe exactly
  double q = p * c;
  double qe = fma(p, c, -q);      // p*c = q + qe exactly
  double tail = qe + pe * c;      // second-order part
  DD s = dd_two_sum(acc.hi, q);
  double lo = s.lo + acc.lo + tail;
  double hi = s.hi + lo;
  acc.lo = lo - (hi - s.hi);
  acc.hi = hi;
}

template <int DIM>
__global__ void __launch_bounds__(SPMV_THREADS) k_residual_dd(Geom g, const double* __restrict__ E,
                                                               const uint8_t* __restrict__ fm,
                                                               const double* __restrict__ f,
                                                               const double* __restrict__ x, double* __restrict__ r,
                                                               double* __restrict__ partial) {
  const int nx = g.nx, ny = g.ny, nz = (DIM == 3) ? g.nz : 1, nnx = nx + 1, nny = ny + 1;
  constexpr int NE = (DIM == 2) ? 4 : 8, KD = (DIM == 2) ? 8 : 24;
  int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc2 = 0.0;
  if (node < g.n_nodes) {
    int a[3];
    a[0] = (int)(node % nnx);
    a[1] = (int)((node / nnx) % nny);
    a[2] = (DIM == 3) ? (int)(node / ((int64_t)nnx * nny)) : 0;
    DD acc[DIM];
    for (int c = 0; c < DIM; ++c) acc[c] = {0.0, 0.0};
    for (int q = 0; q < NE; ++q) {
      int e[3] = {a[0] - 1 + (q & 1), a[1] - 1 + ((q >> 1) & 1), (DIM == 3) ? a[2] - 1 + (q >> 2) : 0};
      if (e[0] < 0 || e[0] >= nx || e[1] < 0 || e[1] >= ny || (DIM == 3 && (e[2] < 0 || e[2] >= nz))) continue;
      int ox = a[0] - e[0], oy = a[1] - e[1], oz = a[2] - e[2];
      int la = 4 * oz + (oy == 0 ? ox : 3 - ox);
      double Ee = E[((int64_t)e[2] * ny + e[1]) * nx + e[0]];
      for (int b = 0; b < NE; ++b) {
        int f4 = b & 3;
        int bx = e[0] + ((f4 == 1 || f4 == 2) ? 1 : 0), by = e[1] + ((f4 >= 2) ? 1 : 0), bz = e[2] + (b >> 2);
        int64_t nb = ((int64_t)bz * nny + by) * nnx + bx;
        for (int cc = 0; cc < DIM; ++cc) {
          if (!fm[DIM * nb + cc]) continue;
          double xv = x[DIM * nb + cc];
          if (xv == 0.0) continue;
          for (int r0 = 0; r0 < DIM; ++r0) dd_add_prod3(acc[r0], Ee, c_KE[g.ke * TS_KE_SIZE + (DIM * la + r0) * KD + DIM * b + cc], xv);
        }
      }
    }
    for (int c = 0; c < DIM; ++c) {
      double out = 0.0;
      if (fm[DIM * node + c]) {
        DD s = dd_two_sum(f[DIM * node + c], -acc[c].hi);
        out = s.hi + (s.lo - acc[c].lo);
      }
      r[DIM * node + c] = out;
      acc2 += out * out;
    }
  }
  double s = block_sum<SPMV_THREADS>(acc2);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = s;
    partial[2 * blockIdx.x + 1] = 0.0;
  }
}

void launch_residual_dd(ts_handle h, const double* f, const double* x, double* r, double* partials) {
  const Geom& g = h->g;
  int nb = node_blocks(g);
  if (g.dim == 2)
    tsl(h), k_residual_dd<2><<<nb, SPMV_THREADS, 0, h->ctx->stream>>>(g, h->E, h->freemask, f, x, r, partials);
  else
    tsl(h), k_residual_dd<3><<<nb, SPMV_THREADS, 0, h->ctx->stream>>>(g, h->E, h->freemask, f, x, r, partials);
  TS_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the stiffness product with its energy dot:
//   y = K x  and  out[0] = x^T K x,
// for callers that may not allocate device memory at call time.  The
// per-block partial sums of the dot, which the regular path keeps in a buffer
// the handle allocated, live here in a fixed file-scope device array.
// ---------------------------------------------------------------------------
#define TS_STATIC_PARTIALS 65536  // 512 KiB: one slot per SpMV block (256 nodes)

static __device__ __align__(256) double g_static_partials[TS_STATIC_PARTIALS];

// device address of g_static_partials per device, looked up once per device
// (std::call_once: request-loop workers and caller threads may make their
// first call on a device at the same time)
static std::once_flag g_static_once[64];
static double* g_static_partials_addr[64];
static cudaError_t g_static_partials_err[64];

static cudaError_t static_partials_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::call_once(g_static_once[dev], [dev]() {
    void* p = nullptr;
    g_static_partials_err[dev] = cudaGetSymbolAddress(&p, g_static_partials);
    g_static_partials_addr[dev] = static_cast<double*>(p);
  });
  if (g_static_partials_err[dev] != cudaSuccess) return g_static_partials_err[dev];
  *out = g_static_partials_addr[dev];
  return cudaSuccess;
}

__global__ void __launch_bounds__(SPMV_THREADS) k_sum_partials(const double* __restrict__ partials, int n,
                                                                double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
  s = block_sum<SPMV_THREADS>(s);
  if (threadIdx.x == 0) *out = s;
}

extern "C" ts_status ts_apply_K_dot_static(ts_handle h, const double* x, double* y, double* out) {
  if (!h || !x || !y || !out) return TS_ERR_INVALID;
  return ts_guarded(h->ctx, [&]() -> ts_status {
    // the handle's lane (streams, events) belongs to the request loop while
    // it holds requests of this handle
    if (server_holds(h->root, h)) throw TsError(TS_ERR_BUSY, "the handle has requests in the request loop");
    const Geom& g = h->g;
    const int nb = spmv_blocks(g);
    if (nb > TS_STATIC_PARTIALS)
      throw TsError(TS_ERR_INVALID, "ts_apply_K_dot_static: the product needs " + std::to_string(nb) +
                                        " blocks of 256 nodes; the fixed scratch holds " +
                                        std::to_string(TS_STATIC_PARTIALS));
    double* partials = nullptr;
    cudaError_t e = static_partials_address(&partials);
    if (e != cudaSuccess) throw TsError(TS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    cudaStream_t st = h->ctx->stream;
    TS_CUDA(cudaEventRecord(h->ctx->ev_in, h->ctx->user_stream));
    TS_CUDA(cudaStreamWaitEvent(st, h->ctx->ev_in, 0));
    // every block writes its own slot, so no slot needs clearing first
    if (g.dim == 2 && h->kst)
      k_spmv_q4<true><<<spmv_grid(g), SPMV_THREADS, 0, st>>>(g, h->E, h->freemask, x, y, partials, x, nullptr,
                                                            nullptr, nullptr,
                                                            PUpdate{nullptr, nullptr, nullptr, nullptr}, h->kst);
    else if (g.dim == 2)
      k_spmv_q4<false><<<spmv_grid(g), SPMV_THREADS, 0, st>>>(g, h->E, h->freemask, x, y, partials, x, nullptr,
                                                             nullptr, nullptr,
                                                             PUpdate{nullptr, nullptr, nullptr, nullptr}, nullptr);
    else
      k_spmv_hex8<<<spmv_grid(g), SPMV_THREADS, 0, st>>>(g, h->E, h->freemask, x, y, partials, x, nullptr, nullptr,
                                                        nullptr);
    k_sum_partials<<<1, SPMV_THREADS, 0, st>>>(partials, nb, out);
    tsl(h, 2);
    TS_CUDA(cudaGetLastError());
    TS_CUDA(cudaEventRecord(h->ctx->ev_out, st));
    TS_CUDA(cudaStreamWaitEvent(h->ctx->user_stream, h->ctx->ev_out, 0));
    return TS_OK;
  });
}

// ---------------------------------------------------------------------------
// Compliance sensitivities (Eq. 1003) and the optimality-criteria density
// update of the topology-optimisation loop the state solve serves (Sec. 1)
// ---------------------------------------------------------------------------
// dc_e = -p rho_e^(p-1) (E0 - Emin) u_e^T KE u_e, one thread per element;
// block partials of the compliance sum_e E_e u_e^T KE u_e
template <int DIM>
__global__ void __launch_bounds__(256) k_sensitivity(Geom g, const double* __restrict__ rho,
                                                     const double* __restrict__ E, const double* __restrict__ u,
                                                     double p, double dE, double* __restrict__ dc,
                                                     double* __restrict__ partials) {
  constexpr int NE = 1 << DIM, ND = DIM * NE;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double ce = 0.0;
  if (e < g.n_el) {
    const int ex = (int)(e % g.nx);
    const int ey = (DIM == 2) ? (int)(e / g.nx) : (int)((e / g.nx) % g.ny);
    const int ez = (DIM == 2) ? 0 : (int)(e / ((int64_t)g.nx * g.ny));
    double ue[ND];
#pragma unroll
    for (int b = 0; b < NE; ++b) {
      // local node b of the element (the numbering of KE)
      const int f4 = b & 3;
      const int ox = (f4 == 1 || f4 == 2) ? 1 : 0, oy = (f4 >= 2) ? 1 : 0, oz = b >> 2;
      const int64_t node = (DIM == 2) ? (int64_t)(ey + oy) * (g.nx + 1) + ex + ox
                                      : ((int64_t)(ez + oz) * (g.ny + 1) + ey + oy) * (g.nx + 1) + ex + ox;
#pragma unroll
      for (int c = 0; c < DIM; ++c) ue[DIM * b + c] = u[DIM * node + c];
    }
    const double* KE = c_KE + g.ke * TS_KE_SIZE;
    double q = 0.0;
    for (int i = 0; i < ND; ++i) {
      double t = 0.0;
#pragma unroll
      for (int j = 0; j < ND; ++j) t = fma(KE[i * ND + j], ue[j], t);
      q = fma(ue[i], t, q);
    }
    // rho^(p-1): repeated products for the usual integer penalties
    const double r = rho[e];
    double rp;
    if (p == 3.0)
      rp = r * r;
    else if (p == 2.0)
      rp = r;
    else if (p == 4.0)
      rp = r * r * r;
    else
      rp = pow(r, p - 1.0);
    dc[e] = -p * rp * dE * q;
    ce = E[e] * q;
  }
  ce = block_sum<256>(ce);
  if (threadIdx.x == 0) partials[blockIdx.x] = ce;
}

struct OcState {
  double lo, hi;    // bracket of the multiplier
  unsigned count;   // blocks done in the current step
};

// rho_e(lam) = clamp(rho_e sqrt(max(-dc_e, 0) / lam), max(0, rho_e - move), min(1, rho_e + move))
__device__ __forceinline__ double oc_rho(double r, double d, double move, double lam) {
  const double v = r * sqrt(fmax(-d, 0.0) / lam);
  return fmin(fmin(1.0, r + move), fmax(fmax(0.0, r - move), v));
}

// one bisection step of log(lam): the mean density at lam = sqrt(lo hi) is
// summed over the grid (block partials added in block order by the last
// block), which then keeps the half of the bracket holding the target
__global__ void __launch_bounds__(256) k_oc_step(int64_t n, const double* __restrict__ rho,
                                                 const double* __restrict__ dc, double move, double target,
                                                 double* __restrict__ partials, OcState* st) {
  __shared__ bool last;
  const double lam = sqrt(st->lo * st->hi);
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    s += oc_rho(rho[e], dc[e], move, lam);
  s = block_sum<256>(s);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(&st->count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(partials + i);
    t = block_sum<256>(t);
    if (threadIdx.x == 0) {
      if (t > target)
        st->lo = lam;
      else
        st->hi = lam;
      st->count = 0;
    }
  }
}

__global__ void __launch_bounds__(256) k_oc_apply(int64_t n, const double* __restrict__ rho,
                                                  const double* __restrict__ dc, double move, const OcState* st,
                                                  double* __restrict__ rho_new) {
  const double lam = sqrt(st->lo * st->hi);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    rho_new[e] = oc_rho(rho[e], dc[e], move, lam);
}

// per-handle workspace of the two calls below: block partials and the OC state
static double* to_workspace(ts_handle h, int64_t nblk) {
  const int64_t need = nblk + 8;
  if (!h->to_ws || h->to_ws_len < need) {
    h->to_ws = dalloc<double>(h, need);
    h->to_ws_len = need;
  }
  return h->to_ws;
}

// dc (device, n_el) and the compliance at out (device) for displacements u
void launch_sensitivity(ts_handle h, const double* u, double* dc, double** out) {
  const Geom& g = h->g;
  cudaStream_t st = h->ctx->stream;
  const int nblk = cdiv(g.n_el, 256);
  double* ws = to_workspace(h, nblk);
  *out = ws + nblk;
  if (g.dim == 2)
    tsl(h), k_sensitivity<2><<<nblk, 256, 0, st>>>(g, h->rho, h->E, u, h->p, h->E0 - h->Emin, dc, ws);
  else
    tsl(h), k_sensitivity<3><<<nblk, 256, 0, st>>>(g, h->rho, h->E, u, h->p, h->E0 - h->Emin, dc, ws);
  tsl(h), k_sum_partials<<<1, SPMV_THREADS, 0, st>>>(ws, nblk, *out);
  TS_CUDA(cudaGetLastError());
}

// rho_new = OC update of the handle's densities for sensitivities dc; the
// host waits for it (the initial bracket is copied from the host stack)
void launch_oc_update(ts_handle h, const double* dc, double volfrac, double move, double* rho_new) {
  const Geom& g = h->g;
  cudaStream_t st = h->ctx->stream;
  const int nblk = std::min(cdiv(g.n_el, 256), 4 * h->ctx->n_sm);
  double* ws = to_workspace(h, nblk + 4);
  OcState* S = reinterpret_cast<OcState*>(ws + nblk);
  const OcState init{1e-40, 1e40, 0u};
  TS_CUDA(cudaMemcpyAsync(S, &init, sizeof(init), cudaMemcpyHostToDevice, st));
  const double target = volfrac * (double)g.n_el;
  for (int it = 0; it < TS_OC_STEPS; ++it)
    tsl(h), k_oc_step<<<nblk, 256, 0, st>>>(g.n_el, h->rho, dc, move, target, ws, S);
  tsl(h), k_oc_apply<<<nblk, 256, 0, st>>>(g.n_el, h->rho, dc, move, S, rho_new);
  TS_CUDA(cudaGetLastError());
  TS_CUDA(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------------------
// Block SpMV over TS_NB columns (2D stencil): q = K p for every column, with
// p = z + beta_c p_old formed while staging (z_old = z for the flexible
// variant) and the per-column partials of p.q; the last block forms alpha.
// The 36 stencil coefficients of a node are read once for all columns.
// Block vectors are [ndof][TS_NB].  Shared memory holds the tile of SBX x SBY
// nodes plus a one-node halo as [component][column][y][x], so that the lanes
// of a warp (consecutive x) read consecutive words.
// ---------------------------------------------------------------------------
constexpr int SBX = 32, SBY = 8, BSP_THREADS = SBX * SBY;

__global__ void __launch_bounds__(BSP_THREADS) k_bspmv(Geom g, const uint8_t* __restrict__ fm,
                                                        const double* __restrict__ x, const double* __restrict__ z,
                                                        const double* __restrict__ p_old, double* __restrict__ p_new,
                                                        double* __restrict__ z_old, double* __restrict__ q,
                                                        double* __restrict__ partial, const int* done, BScalars* S,
                                                        unsigned* counter, const double* __restrict__ St) {
  extern __shared__ __align__(16) double bxs[];  // [2][TS_NB][SBY + 2][SBX + 2]
  constexpr int PL = (SBY + 2) * (SBX + 2);
  const int nx = g.nx, ny = g.ny, nnx = nx + 1;
  const int x0 = blockIdx.x * SBX, y0 = blockIdx.y * SBY, tid = threadIdx.x;
  pdl_wait();
  if (done && *done) return;
  const bool fused = z != nullptr;
  __shared__ double beta_s[TS_NB];
  if (tid < TS_NB) beta_s[tid] = fused ? S->beta[tid] : 0.0;
  __syncthreads();
  // staging: consecutive threads take consecutive values of a node's 16
  // (2 components x TS_NB columns), so the global loads are contiguous
  for (int e = tid; e < PL * 2 * TS_NB; e += BSP_THREADS) {
    const int k = e % (2 * TS_NB), pos = e / (2 * TS_NB);
    const int ly = pos / (SBX + 2), lx = pos % (SBX + 2);
    const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
    const int comp = k / TS_NB, col = k % TS_NB;
    double u = 0.0;
    if (gx >= 0 && gx <= nx && gy >= 0 && gy <= ny) {
      const int64_t nd = (int64_t)gy * nnx + gx;
      const int64_t idx = (2 * nd + comp) * TS_NB + col;
      if (fused) {
        const double zv = z[idx];
        if (fm[2 * nd + comp]) u = fma(beta_s[col], p_old[idx], zv);
        if (lx >= 1 && lx <= SBX && ly >= 1 && ly <= SBY) {
          p_new[idx] = u;
          if (z_old) z_old[idx] = zv;
        }
      } else if (fm[2 * nd + comp]) {
        u = x[idx];
      }
    }
    bxs[(comp * TS_NB + col) * PL + pos] = u;
  }
  __syncthreads();
  const int lx = tid % SBX, ly = tid / SBX;
  const int i = x0 + lx, j = y0 + ly;
  double acc[TS_NB];
#pragma unroll
  for (int c = 0; c < TS_NB; ++c) acc[c] = 0.0;
  if (i <= nx && j <= ny) {
    const int64_t nn = g.n_nodes, node = (int64_t)j * nnx + i;
    double yx[TS_NB], yy[TS_NB];
#pragma unroll
    for (int c = 0; c < TS_NB; ++c) yx[c] = yy[c] = 0.0;
#pragma unroll
    for (int nb = 0; nb < 9; ++nb) {
      const int pos = (ly + nb / 3) * (SBX + 2) + lx + nb % 3;
      const double* sc = St + (int64_t)(4 * nb) * nn + node;
      const double kxx = __ldg(sc), kxy = __ldg(sc + nn), kyx = __ldg(sc + 2 * nn), kyy = __ldg(sc + 3 * nn);
#pragma unroll
      for (int c = 0; c < TS_NB; ++c) {
        const double ux = bxs[c * PL + pos], uy = bxs[(TS_NB + c) * PL + pos];
        yx[c] = fma(kxx, ux, yx[c]);
        yx[c] = fma(kxy, uy, yx[c]);
        yy[c] = fma(kyx, ux, yy[c]);
        yy[c] = fma(kyy, uy, yy[c]);
      }
    }
    const bool fx_ = fm[2 * node] != 0, fy_ = fm[2 * node + 1] != 0;
    const int pos0 = (ly + 1) * (SBX + 2) + lx + 1;
    double2* qx = reinterpret_cast<double2*>(q + 2 * node * TS_NB);
    double2* qy = reinterpret_cast<double2*>(q + (2 * node + 1) * TS_NB);
#pragma unroll
    for (int c = 0; c < TS_NB; c += 2) {
      const double ax = fx_ ? yx[c] : 0.0, bx = fx_ ? yx[c + 1] : 0.0;
      const double ay = fy_ ? yy[c] : 0.0, by = fy_ ? yy[c + 1] : 0.0;
      qx[c / 2] = make_double2(ax, bx);
      qy[c / 2] = make_double2(ay, by);
      acc[c] = fma(bxs[c * PL + pos0], ax, bxs[(TS_NB + c) * PL + pos0] * ay);
      acc[c + 1] = fma(bxs[(c + 1) * PL + pos0], bx, bxs[(TS_NB + c + 1) * PL + pos0] * by);
    }
  }
  pdl_trigger();
  if (partial) {
    double v[1][TS_NB];
#pragma unroll
    for (int c = 0; c < TS_NB; ++c) v[0][c] = acc[c];
    bsum_all_cols<BSP_THREADS, 1>(v);
    const int b = blockIdx.y * gridDim.x + blockIdx.x;
    if (tid == 0)
#pragma unroll
      for (int c = 0; c < TS_NB; ++c) partial[(int64_t)b * TS_NB + c] = v[0][c];
    if (counter && pcg_last_block(counter)) bpcg_alpha_last<BSP_THREADS>(S, partial, gridDim.x * gridDim.y, counter);
  }
}

static dim3 bspmv_grid(const Geom& g) { return dim3(cdiv(g.nx + 1, SBX), cdiv(g.ny + 1, SBY), 1); }
int bspmv_blocks(const Geom& g) {
  const dim3 d = bspmv_grid(g);
  return (int)(d.x * d.y);
}

void launch_bspmv(ts_handle h, const double* x, const double* z, const double* p_old, double* p_new, double* z_old,
                  double* q, double* partials, BScalars* S, unsigned* counter) {
  const Geom& g = h->g;
  if (g.dim != 2 || !h->kst) throw TsError(TS_ERR_INVALID, "internal: the block product needs the 2D stencil");
  const size_t smem = (size_t)2 * TS_NB * (SBY + 2) * (SBX + 2) * sizeof(double);
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [smem]() {
    attr_err = cudaFuncSetAttribute(k_bspmv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  TS_CUDA(attr_err);
  ts_launch(h, h->pdl, k_bspmv, bspmv_grid(g), BSP_THREADS, smem, h->ctx->stream, g, (const uint8_t*)h->freemask, x,
            z, p_old, p_new, z_old, q, partials, (const int*)h->done_flag, S, counter, (const double*)h->kst);
  TS_CUDA(cudaGetLastError());
}
