// FEM kernels: element tables, rigid-body modes, traction loads, the return
// mapping with its Clarke derivative (Sec. 2.4, Sec. 3.1), the element
// tangent corrections and the assembly of Algorithm 5 into banded subdomain
// matrices, the lumped-preconditioner blocks and the internal force.
#include <cfloat>

#include "dev.h"

namespace tfeti {

namespace {

constexpr double kSqrt32 = 1.2247448713915890491;   // sqrt(3/2), correctly rounded
constexpr double kSqrt23 = 0.81649658092772603273;  // sqrt(2/3), correctly rounded
constexpr double kTie = 1e-12;                       // exact-tie band of the elastic predictor test
constexpr double kThird = 1.0 / 3.0;

// element local node of offset (ox, oy, oz) -> index ox + 2 oy + 4 oz
__constant__ int c_off2local[8] = {0, 1, 3, 2, 4, 5, 7, 6};
__constant__ int c_local_off[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                                      {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};

__device__ __forceinline__ int tri_index(int i, int j) {  // packed lower triangle
  return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i;
}

__device__ __forceinline__ int find_sub(const SubDev* subs, int n_sub, long long dof) {
  int lo = 0, hi = n_sub - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (subs[mid].dof_off <= dof) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Element tables: physical shape-function gradients at the 8 Gauss points,
// the elastic brick stiffness and w detJ B_g^T E_eps B_g (eq. (K_def) pieces).
// ---------------------------------------------------------------------------
__global__ void k_tables(double h0, double h1, double h2, double lam, double mu, double* dN, double* Kel,
                         double* Q) {
  __shared__ double B[8][6][24];
  __shared__ double dn[8][8][3];
  const double hh[3] = {h0, h1, h2};
  const double a = 1.0 / sqrt(3.0);
  const int t = threadIdx.x;
  if (t < 64 * 3) {
    const int g = t / 24, rem = t % 24, node = rem / 3, d = rem % 3;
    const double xi[3] = {(2 * (g & 1) - 1) * a, (2 * ((g >> 1) & 1) - 1) * a, (2 * ((g >> 2) & 1) - 1) * a};
    double v = (2 * c_local_off[node][d] - 1) / 8.0;
    for (int e = 0; e < 3; ++e)
      if (e != d) v *= 1.0 + (2 * c_local_off[node][e] - 1) * xi[e];
    dn[g][node][d] = v * (2.0 / hh[d]);
  }
  __syncthreads();
  for (int i = t; i < 8 * 8 * 3; i += blockDim.x) dN[i] = (&dn[0][0][0])[i];
  for (int i = t; i < 8 * 6 * 24; i += blockDim.x) (&B[0][0][0])[i] = 0.0;
  __syncthreads();
  if (t < 64) {
    const int g = t / 8, nd = t % 8;
    const double dx = dn[g][nd][0], dy = dn[g][nd][1], dz = dn[g][nd][2];
    const int c = 3 * nd;
    B[g][0][c] = dx;
    B[g][1][c + 1] = dy;
    B[g][2][c + 2] = dz;
    B[g][3][c] = dy;
    B[g][3][c + 1] = dx;
    B[g][4][c + 1] = dz;
    B[g][4][c + 2] = dy;
    B[g][5][c] = dz;
    B[g][5][c + 2] = dx;
  }
  __syncthreads();
  double C[6][6], E[6][6];
  for (int r = 0; r < 6; ++r)
    for (int s = 0; s < 6; ++s) {
      C[r][s] = 0.0;
      E[r][s] = 0.0;
    }
  for (int r = 0; r < 3; ++r) {
    for (int s = 0; s < 3; ++s) {
      C[r][s] = lam;
      E[r][s] = -1.0 / 3.0;
    }
    C[r][r] = lam + 2.0 * mu;
    C[3 + r][3 + r] = mu;
    E[r][r] = 2.0 / 3.0;
    E[3 + r][3 + r] = 0.5;
  }
  const double wdet = h0 * h1 * h2 / 8.0;
  for (int idx = t; idx < 9 * 576; idx += blockDim.x) {
    const int which = idx / 576, i = (idx % 576) / 24, j = idx % 24;
    double s = 0.0;
    if (which == 0) {
      for (int g = 0; g < 8; ++g)
        for (int r = 0; r < 6; ++r)
          for (int q = 0; q < 6; ++q) s += B[g][r][i] * C[r][q] * B[g][q][j];
      Kel[i * 24 + j] = wdet * s;
    } else {
      const int g = which - 1;
      for (int r = 0; r < 6; ++r)
        for (int q = 0; q < 6; ++q) s += B[g][r][i] * E[r][q] * B[g][q][j];
      Q[(size_t)g * 576 + i * 24 + j] = wdet * s;
    }
  }
}

// ---------------------------------------------------------------------------
// Rigid-body modes of one subdomain shape: translations, rotations about the
// centroid, modified Gram-Schmidt (Sec. 4.2, orthonormal basis of Ker K_p).
// ---------------------------------------------------------------------------
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    red[32] = s;
  }
  __syncthreads();
  return red[32];
}

__global__ void k_rigid(SubDev S, double h0, double h1, double h2, double* R) {
  __shared__ double red[33];
  const int n = S.n_dof;
  const double hh[3] = {h0, h1, h2};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int node = i / 3, c = i % 3;
    const int li = node % S.nn[0], lj = (node / S.nn[0]) % S.nn[1], lk = node / (S.nn[0] * S.nn[1]);
    const double X[3] = {(li - 0.5 * S.dims[0]) * hh[0], (lj - 0.5 * S.dims[1]) * hh[1],
                         (lk - 0.5 * S.dims[2]) * hh[2]};
    double* row = R + (size_t)i * 6;
    row[0] = c == 0;
    row[1] = c == 1;
    row[2] = c == 2;
    // e_x x X = (0, -Xz, Xy); e_y x X = (Xz, 0, -Xx); e_z x X = (-Xy, Xx, 0)
    row[3] = c == 0 ? 0.0 : (c == 1 ? -X[2] : X[1]);
    row[4] = c == 0 ? X[2] : (c == 1 ? 0.0 : -X[0]);
    row[5] = c == 0 ? -X[1] : (c == 1 ? X[0] : 0.0);
  }
  __syncthreads();
  for (int j = 0; j < 6; ++j) {
    for (int q = 0; q < j; ++q) {
      double s = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) s += R[(size_t)i * 6 + q] * R[(size_t)i * 6 + j];
      s = block_sum(s, red);
      for (int i = threadIdx.x; i < n; i += blockDim.x) R[(size_t)i * 6 + j] -= s * R[(size_t)i * 6 + q];
      __syncthreads();
    }
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += R[(size_t)i * 6 + j] * R[(size_t)i * 6 + j];
    s = block_sum(s, red);
    const double inv = 1.0 / sqrt(s);
    for (int i = threadIdx.x; i < n; i += blockDim.x) R[(size_t)i * 6 + j] *= inv;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Uniform traction on a face: t * area / 4 per element face and node.
// ---------------------------------------------------------------------------
__global__ void k_traction(DevMesh M, int face, int nel0, int nel1, int nel2, double t0, double t1, double t2,
                           double h0, double h1, double h2, double* f) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= M.n_dof) return;
  const int p = find_sub(M.subs, M.n_sub, i);
  const SubDev& S = M.subs[p];
  const int ld = (int)(i - S.dof_off);
  const int node = ld / 3, c = ld % 3;
  const int l[3] = {node % S.nn[0], (node / S.nn[0]) % S.nn[1], node / (S.nn[0] * S.nn[1])};
  const int axis = face / 2, side = face % 2;
  const int nel[3] = {nel0, nel1, nel2};
  const double hh[3] = {h0, h1, h2};
  double v = 0.0;
  const bool touches = side == 0 ? S.origin[axis] == 0 : S.origin[axis] + S.dims[axis] == nel[axis];
  const int lface = side == 0 ? 0 : S.dims[axis];
  if (touches && l[axis] == lface) {
    const int o1 = (axis + 1) % 3, o2 = (axis + 2) % 3;
    const int cnt = ((l[o1] > 0) + (l[o1] < S.dims[o1])) * ((l[o2] > 0) + (l[o2] < S.dims[o2]));
    const double tc = c == 0 ? t0 : (c == 1 ? t1 : t2);
    v = cnt * (tc * (hh[o1] * hh[o2]) / 4.0);
  }
  f[i] = v;
}

// ---------------------------------------------------------------------------
// Trilinear gradients by sum factorisation over the 8 lanes of an element (lane bits x + 2y + 4z
// give both the lane's Gauss point and the element node it loads).  For one displacement
// component u (the lane's node value) the lane receives grad u at its Gauss point:
//   along x: I = interpolant at the point's x, D = u(x=1) - u(x=0) on each x-edge;
//   along y: DX = D interpolated in y, E = I(y=1) - I(y=0), J = I interpolated in y (/ h_z);
//   along z: du/dx = DX interpolated in z / h_x, du/dy = E interpolated in z / h_y,
//            du/dz = J(z=1) - J(z=0);
// each interpolation step takes the lane's own value with weight (1 + 1/sqrt 3)/2 and its
// partner's with (1 - 1/sqrt 3)/2 (the 2-point Gauss abscissae +-1/sqrt 3).  13 FP64 operations
// per component and point instead of the 24 of the direct sum over the 8 nodes.
// All 32 lanes of the warp take part.
constexpr double kGa = 0.78867513459481288225;   // (1 + 1/sqrt 3) / 2
constexpr double kGb = 0.21132486540518711775;   // (1 - 1/sqrt 3) / 2

__device__ __forceinline__ void grad_lanes(const DevMesh& M, double u, int bx, int by, int bz, double& gx,
                                           double& gy, double& gz) {
  const unsigned all = 0xffffffffu;
  const double up = __shfl_xor_sync(all, u, 1);
  const double I1 = kGa * u + kGb * up;
  const double D1 = (bx ? u : up) - (bx ? up : u);
  const double D1p = __shfl_xor_sync(all, D1, 2), I1p = __shfl_xor_sync(all, I1, 2);
  const double DX2 = kGa * D1 + kGb * D1p;
  const double E2 = (by ? I1 : I1p) - (by ? I1p : I1);
  const double J2 = M.ga[2] * I1 + M.gb[2] * I1p;
  const double DX2p = __shfl_xor_sync(all, DX2, 4), E2p = __shfl_xor_sync(all, E2, 4),
               J2p = __shfl_xor_sync(all, J2, 4);
  gx = M.ga[0] * DX2 + M.gb[0] * DX2p;
  gy = M.ga[1] * E2 + M.gb[1] * E2p;
  gz = (bz ? J2 : J2p) - (bz ? J2p : J2);
}

// The transpose of grad_lanes: given (fx, fy, fz) at the lane's Gauss point, returns at the
// lane's node sum over the element's points of grad N_node . (fx, fy, fz).
__device__ __forceinline__ double grad_lanes_t(const DevMesh& M, double fx, double fy, double fz, int bx, int by,
                                               int bz) {
  const unsigned all = 0xffffffffu;
  const double sx = bx ? 1.0 : -1.0, sy = by ? 1.0 : -1.0, sz = bz ? 1.0 : -1.0;
  const double fxp = __shfl_xor_sync(all, fx, 4), fyp = __shfl_xor_sync(all, fy, 4), fzp = __shfl_xor_sync(all, fz, 4);
  const double bDX2 = M.ga[0] * fx + M.gb[0] * fxp;
  const double bE2 = M.ga[1] * fy + M.gb[1] * fyp;
  const double bJ2 = sz * (fz + fzp);
  const double bDX2p = __shfl_xor_sync(all, bDX2, 2), bE2p = __shfl_xor_sync(all, bE2, 2),
               bJ2p = __shfl_xor_sync(all, bJ2, 2);
  const double bD1 = kGa * bDX2 + kGb * bDX2p;
  const double bI1 = sy * (bE2 + bE2p) + (M.ga[2] * bJ2 + M.gb[2] * bJ2p);
  const double bD1p = __shfl_xor_sync(all, bD1, 1), bI1p = __shfl_xor_sync(all, bI1, 1);
  return sx * (bD1 + bD1p) + (kGa * bI1 + kGb * bI1p);
}

// ---------------------------------------------------------------------------
// Return mapping and Clarke derivative at one Gauss point.
// eta = B_g u_e; tau = sigma_k + C eta; Phi = sqrt(3/2)||dev tau|| - (sigma_y + H kappa_k).
// Phi <= 0: dsigma = C eta, dkappa = 0, D = C.
// Phi > 0 : dsigma = C eta - c sqrt(2/3) Phi n, dkappa = Phi/(3mu+H),
// A point returned to the yield surface has Phi = 0 in exact arithmetic (elastic by
// the rule above) but +-1 ulp after rounding: |Phi| <= kTie (sigma_y + H kappa_k)
// is read as that tie, i.e. elastic.
//           D = C - 2mu c (1 - rho) E_eps - 2mu c rho n n^T, rho = sqrt(2/3)(sigma_y+H kappa)/||dev tau||,
//           c = 3mu/(3mu+H)  (the Sec. 3.1 form of eq. (stress_op_deriv_plast)).
// ---------------------------------------------------------------------------
// One thread per Gauss point, the 8 points of an element in 8 consecutive lanes (blockDim and n_gp
// multiples of 8); lanes past n_gp compute on the last element and store nothing.
__global__ void k_return_map(DevMesh M, const double* __restrict__ du, const double* __restrict__ sig_k,
                             const double* __restrict__ kap_k, double* dsig, double* dkap, uint8_t* plastic,
                             double* Dtan, double* pa, double* pb, double* pn) {
  const long long gp_t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const bool live = gp_t < M.n_gp;
  const long long gp = live ? gp_t : M.n_gp - 8 + (gp_t & 7);
  const long long e = gp >> 3;
  const int g = (int)(gp & 7);
  const int bx = g & 1, by = (g >> 1) & 1, bz = (g >> 2) & 1;
  const int p = M.elem_sub[e];
  const SubDev& S = M.subs[p];
  const int le = (int)(e - S.elem_off);
  const int ex = le % S.dims[0], ey = (le / S.dims[0]) % S.dims[1], ez = le / (S.dims[0] * S.dims[1]);
  const int ln = (ex + bx) + S.nn[0] * ((ey + by) + S.nn[1] * (ez + bz));
  const double* u = du + S.dof_off + 3LL * ln;
  double gr[3][3];   // gr[c][d] = d u_c / d x_d at the lane's Gauss point
#pragma unroll
  for (int c = 0; c < 3; ++c) grad_lanes(M, u[c], bx, by, bz, gr[c][0], gr[c][1], gr[c][2]);
  if (!live) return;
  const double eta[6] = {gr[0][0], gr[1][1], gr[2][2], gr[0][1] + gr[1][0], gr[1][2] + gr[2][1],
                         gr[0][2] + gr[2][0]};
  const double lam = M.lam, mu = M.mu;
  const double tr = eta[0] + eta[1] + eta[2];
  double ce[6];
  ce[0] = lam * tr + 2.0 * mu * eta[0];
  ce[1] = lam * tr + 2.0 * mu * eta[1];
  ce[2] = lam * tr + 2.0 * mu * eta[2];
  ce[3] = mu * eta[3];
  ce[4] = mu * eta[4];
  ce[5] = mu * eta[5];
  double tau[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) tau[c] = sig_k[c * M.n_gp + gp] + ce[c];
  const double kap = kap_k[gp];
  const double mean = (tau[0] + tau[1] + tau[2]) * kThird;
  double dev[6] = {tau[0] - mean, tau[1] - mean, tau[2] - mean, tau[3], tau[4], tau[5]};
  const double nrm2 =
      dev[0] * dev[0] + dev[1] * dev[1] + dev[2] * dev[2] + 2.0 * (dev[3] * dev[3] + dev[4] * dev[4] + dev[5] * dev[5]);
  const double yield = M.sigma_y + M.H * kap;
  // (3/2) |dev tau|^2 <= yield^2 (yield > 0) puts Phi within rounding of <= 0, far inside the
  // tie band: elastic without the square root; otherwise Phi and the test as stated above
  double nrm = 0.0, phi = 0.0;
  bool pl = false;
  if (1.5 * nrm2 > yield * yield) {
    nrm = sqrt(nrm2);
    phi = kSqrt32 * nrm - yield;
    pl = phi > kTie * yield;
  }
  double ds[6];
  double a = 0.0, b = 0.0, nb[6] = {0, 0, 0, 0, 0, 0};
  if (pl) {
    const double c = 3.0 * mu / (3.0 * mu + M.H);
    const double inv = 1.0 / nrm;
    const double corr = c * kSqrt23 * phi;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      nb[q] = dev[q] * inv;
      ds[q] = ce[q] - corr * nb[q];
    }
    const double rho = kSqrt23 * yield * inv;
    a = 2.0 * mu * c * (1.0 - rho);
    b = 2.0 * mu * c * rho;
    if (dkap) dkap[gp] = phi / (3.0 * mu + M.H);
  } else {
#pragma unroll
    for (int q = 0; q < 6; ++q) ds[q] = ce[q];
    if (dkap) dkap[gp] = 0.0;
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) dsig[q * M.n_gp + gp] = ds[q];
  if (plastic) plastic[gp] = pl ? 1 : 0;
  if (pa) {
    pa[gp] = a;
    pb[gp] = b;
#pragma unroll
    for (int q = 0; q < 6; ++q) pn[q * M.n_gp + gp] = nb[q];
  }
  if (Dtan) {
    int idx = 0;
    for (int r = 0; r < 6; ++r)
      for (int s = r; s < 6; ++s, ++idx) {
        double C = 0.0, E = 0.0;
        if (r < 3 && s < 3) {
          C = lam + (r == s ? 2.0 * mu : 0.0);
          E = r == s ? 2.0 / 3.0 : -1.0 / 3.0;
        } else if (r == s) {
          C = mu;
          E = 0.5;
        }
        Dtan[idx * M.n_gp + gp] = pl ? C - a * E - b * nb[r] * nb[s] : C;
      }
  }
}

// ---------------------------------------------------------------------------
// Element tangent correction dK_e = sum_{plastic g} (a_g Q_g + w detJ b_g v_g v_g^T),
// v_g = B_g^T n_g.  K_e = K_el - dK_e.  One warp per element.
// ---------------------------------------------------------------------------
__global__ void k_elem_correction(DevMesh M, GPData gd, int* elem_np, int* sub_np, double* dKe) {
  __shared__ double v[8][8][24];  // [warp][g][i]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long e = blockIdx.x * (long long)(blockDim.x >> 5) + warp;
  if (e >= M.n_elem) return;
  const long long gp0 = e * 8;
  int flag = 0;
  if (lane < 8) flag = gd.plastic[gp0 + lane];
  const unsigned mask = __ballot_sync(0xffffffffu, flag != 0);
  const int cnt = __popc(mask);
  if (lane == 0) {
    elem_np[e] = cnt;
    if (cnt) atomicAdd(&sub_np[M.elem_sub[e]], cnt);
  }
  if (!cnt) return;
  if (lane < 8 && flag) {
    const long long gp = gp0 + lane;
    double n[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) n[q] = gd.pn[q * M.n_gp + gp];
    const double* dn = M.dN + lane * 24;
    for (int a = 0; a < 8; ++a) {
      const double dx = dn[3 * a], dy = dn[3 * a + 1], dz = dn[3 * a + 2];
      v[warp][lane][3 * a + 0] = dx * n[0] + dy * n[3] + dz * n[5];
      v[warp][lane][3 * a + 1] = dy * n[1] + dx * n[3] + dz * n[4];
      v[warp][lane][3 * a + 2] = dz * n[2] + dy * n[4] + dx * n[5];
    }
  }
  __syncwarp();
  double ag[8], bg[8];
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    const bool pl = (mask >> g) & 1u;
    ag[g] = pl ? gd.pa[gp0 + g] : 0.0;
    bg[g] = pl ? M.wdet * gd.pb[gp0 + g] : 0.0;
  }
  for (int idx = lane; idx < kTri24; idx += 32) {
    int i = 0;
    while ((i + 1) * (i + 2) / 2 <= idx) ++i;
    const int j = idx - i * (i + 1) / 2;
    double s = 0.0;
#pragma unroll
    for (int g = 0; g < 8; ++g)
      if ((mask >> g) & 1u) s += ag[g] * M.Q[g * 576 + i * 24 + j] + bg[g] * v[warp][g][i] * v[warp][g][j];
    dKe[e * kTri24 + idx] = s;
  }
}

// K entry (true tangent) between local dofs r and c of subdomain S.
__device__ double stiffness_entry(const DevMesh& M, const SubDev& S, const int* elem_np, const double* dKe, int r,
                                  int c, bool elastic_only) {
  const int nr = r / 3, ar = r % 3, nc = c / 3, ac = c % 3;
  const int ri = nr % S.nn[0], rj = (nr / S.nn[0]) % S.nn[1], rk = nr / (S.nn[0] * S.nn[1]);
  const int ci = nc % S.nn[0], cj = (nc / S.nn[0]) % S.nn[1], ck = nc / (S.nn[0] * S.nn[1]);
  if (abs(ri - ci) > 1 || abs(rj - cj) > 1 || abs(rk - ck) > 1) return 0.0;
  double sum = 0.0;
  const int ex0 = max(max(ri, ci) - 1, 0), ex1 = min(min(ri, ci), S.dims[0] - 1);
  const int ey0 = max(max(rj, cj) - 1, 0), ey1 = min(min(rj, cj), S.dims[1] - 1);
  const int ez0 = max(max(rk, ck) - 1, 0), ez1 = min(min(rk, ck), S.dims[2] - 1);
  for (int ez = ez0; ez <= ez1; ++ez)
    for (int ey = ey0; ey <= ey1; ++ey)
      for (int ex = ex0; ex <= ex1; ++ex) {
        const int a = c_off2local[(ri - ex) + 2 * (rj - ey) + 4 * (rk - ez)];
        const int b = c_off2local[(ci - ex) + 2 * (cj - ey) + 4 * (ck - ez)];
        const int i = 3 * a + ar, j = 3 * b + ac;
        double v = M.Kel[i * 24 + j];
        if (!elastic_only) {
          const long long ge = S.elem_off + ex + S.dims[0] * (ey + S.dims[1] * ez);
          if (elem_np[ge]) v -= dKe[ge * kTri24 + tri_index(i, j)];
        }
        sum += v;
      }
  return sum;
}

// Band storage of subdomain K_p with the fixing dofs replaced by identity rows:
// band[r*(bw+1) + k] = K[r][r - bw + k] (lower band, row-major).
// With bmask == null the six fixing dofs of Remark 1 get identity rows and columns
// (K_rr of the generalised inverse); with bmask the dofs marked in it do (K_ii of the
// Dirichlet preconditioner: the constrained nodes eliminated, Sec. 4.2).
__global__ void k_band_fill(DevMesh M, const int* __restrict__ sub_list, const int* elem_np, const double* dKe,
                            double* band, const long long* __restrict__ band_off_list, int elastic_only,
                            const uint8_t* __restrict__ bmask) {
  const int item = blockIdx.y;
  const int p = sub_list[item];
  const SubDev& S = M.subs[p];
  const long long total = (long long)S.n_dof * (S.bw + 1);
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int r = (int)(idx / (S.bw + 1)), k = (int)(idx % (S.bw + 1));
  const int c = r - S.bw + k;
  double v = 0.0;
  if (c >= 0) {
    bool fixed = false;
    if (bmask) {
      fixed = bmask[S.dof_off + r] | bmask[S.dof_off + c];
    } else {
#pragma unroll
      for (int t = 0; t < 6; ++t) fixed |= (S.fix[t] == r) | (S.fix[t] == c);
    }
    if (fixed) v = (r == c) ? 1.0 : 0.0;
    else v = stiffness_entry(M, S, elem_np, dKe, r, c, elastic_only != 0);
  }
  band[band_off_list[item] + idx] = v;
}

// Lumped-preconditioner blocks of one subdomain (or its shape's elastic template):
// K[3 ln(b) + a][3 ln(nu) + c] for every box-boundary node b and its 27 stencil neighbours nu.
__global__ void k_kbb_fill(DevMesh M, const int* __restrict__ sub_list, const long long* __restrict__ dst_off,
                           const int* elem_np, const double* dKe, double* kbb, float* kbb32, int elastic_only) {
  const int p = sub_list[blockIdx.y];
  const SubDev& S = M.subs[p];
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)S.n_bnd * 243) return;
  // layout [t][cc][3 b + a]: for a fixed neighbour t and column cc the rows of all boundary
  // nodes are contiguous, so the lumped kernel's threads (consecutive rows) read coalesced
  const long long nr = 3LL * S.n_bnd;
  const int tc = (int)(idx / nr), ra = (int)(idx % nr);
  const int t = tc / 3, cc = tc % 3, b = ra / 3, a = ra % 3;
  const int nu = M.shape_tnbr[(S.bnd_off + b) * 27 + t];
  double v = 0.0;
  if (nu >= 0) {
    const int r = 3 * M.shape_bln[S.bnd_off + b] + a;
    const int c = 3 * M.shape_bln[S.bnd_off + nu] + cc;
    v = stiffness_entry(M, S, elem_np, dKe, r, c, elastic_only != 0);
  }
  kbb[dst_off[blockIdx.y] + idx] = v;
  if (kbb32) kbb32[dst_off[blockIdx.y] + idx] = (float)v;
}

// Internal force of eq. (F_def), element part: for every element node a (bit order x + 2y + 4z)
// and component c, fe = sum over the element's Gauss points of grad N_a . sigma_c (sigma_c the
// row c of the stress dsig), by the transposed sum factorisation over the element's 8 lanes.
__global__ void k_elem_force(DevMesh M, const double* __restrict__ dsig, double* fe) {
  const long long gp_t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const bool live = gp_t < M.n_gp;
  const long long gp = live ? gp_t : M.n_gp - 8 + (gp_t & 7);
  const int g = (int)(gp & 7);
  const int bx = g & 1, by = (g >> 1) & 1, bz = (g >> 2) & 1;
  double sg[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) sg[q] = dsig[q * M.n_gp + gp];
  // Voigt order xx, yy, zz, xy, yz, xz
  const double f0 = grad_lanes_t(M, sg[0], sg[3], sg[5], bx, by, bz);
  const double f1 = grad_lanes_t(M, sg[3], sg[1], sg[4], bx, by, bz);
  const double f2 = grad_lanes_t(M, sg[5], sg[4], sg[2], bx, by, bz);
  if (!live) return;
  double* o = fe + 3 * gp;   // element e = gp / 8, node g
  o[0] = f0;
  o[1] = f1;
  o[2] = f2;
}

// f = df - w detJ (sum of the element parts at the dof), the adjacent elements in (z, y, x) order.
__global__ void k_gather_force(DevMesh M, const double* __restrict__ fe, const double* __restrict__ df, double* f) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= M.n_dof) return;
  const int p = find_sub(M.subs, M.n_sub, i);
  const SubDev& S = M.subs[p];
  const int ld = (int)(i - S.dof_off);
  const int node = ld / 3, c = ld % 3;
  const int li = node % S.nn[0], lj = (node / S.nn[0]) % S.nn[1], lk = node / (S.nn[0] * S.nn[1]);
  double s = 0.0;
  for (int ez = max(lk - 1, 0); ez <= min(lk, S.dims[2] - 1); ++ez)
    for (int ey = max(lj - 1, 0); ey <= min(lj, S.dims[1] - 1); ++ey)
      for (int ex = max(li - 1, 0); ex <= min(li, S.dims[0] - 1); ++ex) {
        const int a = (li - ex) + 2 * (lj - ey) + 4 * (lk - ez);
        const long long ge = S.elem_off + ex + S.dims[0] * (ey + S.dims[1] * ez);
        s += fe[(ge * 8 + a) * 3 + c];
      }
  f[i] = (df ? df[i] : 0.0) - M.wdet * s;
}

// y = K x per subdomain with the assembled tangent (27-node stencil).
__global__ void k_apply_K(DevMesh M, const int* elem_np, const double* dKe, const double* __restrict__ x,
                          double* y) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= M.n_dof) return;
  const int p = find_sub(M.subs, M.n_sub, i);
  const SubDev& S = M.subs[p];
  const int r = (int)(i - S.dof_off);
  const int node = r / 3;
  const int li = node % S.nn[0], lj = (node / S.nn[0]) % S.nn[1], lk = node / (S.nn[0] * S.nn[1]);
  double s = 0.0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int a = li + dx, b = lj + dy, c = lk + dz;
        if (a < 0 || b < 0 || c < 0 || a >= S.nn[0] || b >= S.nn[1] || c >= S.nn[2]) continue;
        const int nn = a + S.nn[0] * (b + S.nn[1] * c);
        for (int q = 0; q < 3; ++q)
          s += stiffness_entry(M, S, elem_np, dKe, r, 3 * nn + q, false) * x[S.dof_off + 3 * nn + q];
      }
  y[i] = s;
}

__global__ void k_commit(long long n_dof, long long n_gp, const double* du, const double* dsig,
                         const double* dkap, double* u, double* sig, double* kap) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n_dof) u[i] += du[i];
  if (i < 6 * n_gp) sig[i] += dsig[i];
  if (i < n_gp) kap[i] += dkap[i];
}

__global__ void k_vm_partial(long long n_gp, const double* __restrict__ s, double* partial) {
  __shared__ double red[256];
  double m = 0.0;
  for (long long gp = blockIdx.x * (long long)blockDim.x + threadIdx.x; gp < n_gp;
       gp += (long long)gridDim.x * blockDim.x) {
    const double t0 = s[gp], t1 = s[n_gp + gp], t2 = s[2 * n_gp + gp];
    const double mean = (t0 + t1 + t2) / 3.0;
    const double d0 = t0 - mean, d1 = t1 - mean, d2 = t2 - mean;
    const double t3 = s[3 * n_gp + gp], t4 = s[4 * n_gp + gp], t5 = s[5 * n_gp + gp];
    const double q = kSqrt32 * sqrt(d0 * d0 + d1 * d1 + d2 * d2 + 2.0 * (t3 * t3 + t4 * t4 + t5 * t5));
    m = fmax(m, q);
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_max_final(const double* partial, int n, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < n; ++i) m = fmax(m, partial[i]);
    *out = m;
  }
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void launch_tables(const double* h, double lam, double mu, double* dN, double* Kel, double* Q, cudaStream_t st) {
  k_tables<<<1, 256, 0, st>>>(h[0], h[1], h[2], lam, mu, dN, Kel, Q);
}

void launch_rigid_for_shape(const SubDev& S, const double* h, double* R_shape, cudaStream_t st) {
  k_rigid<<<1, 256, 0, st>>>(S, h[0], h[1], h[2], R_shape);
}

void launch_traction(const DevMesh& M, int face, const int* nel, const double* t, const double* h, double* f,
                     cudaStream_t st) {
  k_traction<<<blocks_for(M.n_dof, 256), 256, 0, st>>>(M, face, nel[0], nel[1], nel[2], t[0], t[1], t[2], h[0],
                                                          h[1], h[2], f);
}

void launch_return_map(const DevMesh& M, const double* du, const double* sig_k, const double* kap_k,
                       double* dsig, double* dkap, uint8_t* plastic, double* Dtan, double* pa, double* pb,
                       double* pn, cudaStream_t st) {
  k_return_map<<<blocks_for(M.n_gp, 128), 128, 0, st>>>(M, du, sig_k, kap_k, dsig, dkap, plastic, Dtan, pa, pb,
                                                           pn);
}

void launch_elem_correction(const DevMesh& M, GPData gp, int* elem_np, int* sub_np, double* dKe, cudaStream_t st) {
  k_elem_correction<<<blocks_for(M.n_elem, 8), 256, 0, st>>>(M, gp, elem_np, sub_np, dKe);
}

void launch_band_fill(const DevMesh& M, const int* sub_list, int n_list, const int* elem_np, const double* dKe,
                      double* band, const long long* band_off_list, int elastic_only, int max_rows, int max_bw,
                      cudaStream_t st, const uint8_t* bmask) {
  if (n_list <= 0) return;
  dim3 grid(blocks_for((long long)max_rows * (max_bw + 1), 256), n_list);
  k_band_fill<<<grid, 256, 0, st>>>(M, sub_list, elem_np, dKe, band, band_off_list, elastic_only, bmask);
}

void launch_kbb_fill(const DevMesh& M, const int* sub_list, const long long* dst_off, int n_list, int max_bnd,
                     const int* elem_np, const double* dKe, double* kbb, float* kbb32, int elastic_only,
                     cudaStream_t st) {
  if (n_list <= 0) return;
  dim3 grid(blocks_for((long long)max_bnd * 243, 256), n_list);
  k_kbb_fill<<<grid, 256, 0, st>>>(M, sub_list, dst_off, elem_np, dKe, kbb, kbb32, elastic_only);
}

void launch_internal_force(const DevMesh& M, const double* dsig, const double* df, double* fe, double* f,
                           cudaStream_t st) {
  if (M.n_gp > 0) k_elem_force<<<blocks_for(M.n_gp, 128), 128, 0, st>>>(M, dsig, fe);
  k_gather_force<<<blocks_for(M.n_dof, 128), 128, 0, st>>>(M, fe, df, f);
}

void launch_apply_K(const DevMesh& M, const int* elem_np, const double* dKe, const double* x, double* y,
                    cudaStream_t st) {
  k_apply_K<<<blocks_for(M.n_dof, 128), 128, 0, st>>>(M, elem_np, dKe, x, y);
}

void launch_commit(const DevMesh& M, const double* du, const double* dsig, const double* dkap, double* u,
                   double* sig, double* kap, cudaStream_t st) {
  const long long n = 6 * M.n_gp > M.n_dof ? 6 * M.n_gp : M.n_dof;
  k_commit<<<blocks_for(n, 256), 256, 0, st>>>(M.n_dof, M.n_gp, du, dsig, dkap, u, sig, kap);
}

void launch_vm_max(const DevMesh& M, const double* dsig, double* partial, double* out, cudaStream_t st) {
  k_vm_partial<<<kRedBlocks, 256, 0, st>>>(M.n_gp, dsig, partial);
  k_max_final<<<1, 32, 0, st>>>(partial, kRedBlocks, out);
}

}  // namespace tfeti
