// Inner (FP32) F-apply of plastic subdomains through their shape's elastic dual Schur block
// plus a low-rank correction (Sherman-Morrison-Woodbury), instead of banded solves.
//
// The assembled tangent of a subdomain with plastic Gauss points differs from its shape's
// elastic matrix by the element corrections of Algorithm 5's Clarke tangent (Sec. 3.1):
//   K_p = K_el - sum_{plastic g} |T| B_g^T (a_g E_eps + b_g n_g n_g^T) B_g = K_el - U U^T,
// with six columns per plastic point, U_g = sqrt(a_g |T|) B_g^T F and sqrt(b_g |T|) B_g^T n_g,
// F F^T = E_eps (F: an orthonormal basis of the deviatoric plane, and sqrt(1/2) on the shear
// components).  a_g, b_g >= 0 and the tangent stays positive definite, so with the fixing-dof
// generalised inverse K^+ of the elastic matrix (zero rows and columns at the fixing dofs):
//   K_p^+ = K^+ + Z C^{-1} Z^T,  Z = K^+ U,  C = I - U^T K^+ U  (symmetric positive definite),
// and on the box boundary  S_p = S_el + Z_b C^{-1} Z_b^T,  Z_b the boundary rows of Z.  The
// subdomain's slots then come from the shape's tensor-core GEMM (as for elastic subdomains)
// plus the correction  Z_b (Y x_b),  Y = C^{-1} Z_b^T,  two skinny products per subdomain.
//
// All of it in FP32, the precision of the inner iterations.  Per subdomain (one CTA each):
// the plastic points in order (k_wood_points), C and Z_b from the shape's dense K^+ (k_wood_C,
// k_wood_Zb), the blocked Cholesky factor of C (k_wood_chol_*) and Y by blocked substitution
// (k_wood_subst); per inner F-apply k_wood_x, k_wood_t and k_wood_y.
#include "dev.h"
#include "dual_common.cuh"

namespace tfeti {

namespace {

// element node offsets (same order as the shape-function gradient table dN)
__constant__ int c_wnode[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                                  {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};

// The 24 local dofs of plastic point `pt` (element-local index * 8 + g) of subdomain S and its six
// U columns u[j][t] (t: element dof).
__device__ void wood_point(const DevMesh& M, const SubDev& S, int pt, const double* __restrict__ pa,
                           const double* __restrict__ pb, const double* __restrict__ pn, int dofs[24],
                           float u[6][24]) {
  const int le = pt >> 3, g = pt & 7;
  const int ax = S.dims[0], ay = S.dims[1];
  const int ex = le % ax, ey = (le / ax) % ay, ez = le / (ax * ay);
  const long long gp = 8 * (S.elem_off + le) + g;
  const double sa = sqrt(fmax(pa[gp], 0.0) * M.wdet), sb = sqrt(fmax(pb[gp], 0.0) * M.wdet);
  double n[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) n[q] = pn[q * M.n_gp + gp];
  // columns of F: deviatoric plane basis, then sqrt(1/2) e_4, e_5, e_6
  const double r2 = 0.70710678118654752440, r6 = 0.40824829046386301637;
  const double F[5][6] = {{r2, -r2, 0, 0, 0, 0},
                          {r6, r6, -2 * r6, 0, 0, 0},
                          {0, 0, 0, r2, 0, 0},
                          {0, 0, 0, 0, r2, 0},
                          {0, 0, 0, 0, 0, r2}};
  for (int a = 0; a < 8; ++a) {
    const int ln = (ex + c_wnode[a][0]) + S.nn[0] * ((ey + c_wnode[a][1]) + S.nn[1] * (ez + c_wnode[a][2]));
    const double dx = M.dN[(g * 8 + a) * 3], dy = M.dN[(g * 8 + a) * 3 + 1], dz = M.dN[(g * 8 + a) * 3 + 2];
    for (int c = 0; c < 3; ++c) dofs[3 * a + c] = 3 * ln + c;
    for (int j = 0; j < 6; ++j) {
      const double* v = j < 5 ? F[j] : n;
      const double s = j < 5 ? sa : sb;
      u[j][3 * a + 0] = (float)(s * (dx * v[0] + dy * v[3] + dz * v[5]));
      u[j][3 * a + 1] = (float)(s * (dy * v[1] + dx * v[3] + dz * v[4]));
      u[j][3 * a + 2] = (float)(s * (dz * v[2] + dy * v[4] + dx * v[5]));
    }
  }
}

// Plastic points of subdomain list[w] in Gauss-point order -> pts + pt_off[w] (a block-wide scan).
__global__ void k_wood_points(DevMesh M, const int* __restrict__ list, const long long* __restrict__ pt_off,
                              const int* __restrict__ n_pts, const uint8_t* __restrict__ plastic, int* pts) {
  __shared__ int wsum[32];
  __shared__ int base;
  const SubDev S = M.subs[list[blockIdx.x]];
  const long long g0 = 8 * S.elem_off;
  const int n = 8 * S.n_elem;
  int* out = pts + pt_off[blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int c = 0; c < n; c += blockDim.x) {
    const int i = c + threadIdx.x;
    const bool f = i < n && plastic[g0 + i] != 0;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int before = base;
    for (int k = 0; k < warp; ++k) before += wsum[k];
    const int at = before + __popc(bal & ((1u << lane) - 1u));
    if (f && at < n_pts[blockIdx.x]) out[at] = i;   // the count equals n_pts (same flags)
    __syncthreads();
    if (threadIdx.x == 0)
      for (int k = 0; k < nw; ++k) base += wsum[k];
    __syncthreads();
  }
}

// C = I - U^T K^+ U for subdomain list[blockIdx.x], rows 6i..6i+5 (i = blockIdx.y): for every point
// j, the 6 x 6 block U_i^T K^+[D_i, D_j] U_j.  C row-major r x r at c_pool + c_off[w].
__global__ void __launch_bounds__(256) k_wood_C(DevMesh M, const int* __restrict__ list,
                                                const long long* __restrict__ pt_off, const int* __restrict__ pts,
                                                const int* __restrict__ n_pts, const float* __restrict__ kinv,
                                                const long long* __restrict__ kinv_off, const double* __restrict__ pa,
                                                const double* __restrict__ pb, const double* __restrict__ pn,
                                                const long long* __restrict__ c_off, float* c_pool) {
  __shared__ int di[24], dj[24];
  __shared__ float ui[6][24], uj[6][24], kb[24][25], ku[24][6];
  const int w = blockIdx.x, i = blockIdx.y;
  const int np = n_pts[w];
  if (i >= np) return;
  const SubDev S = M.subs[list[w]];
  const int n = S.n_dof, r = 6 * np;
  const float* K = kinv + kinv_off[S.shape];
  const int* P = pts + pt_off[w];
  float* C = c_pool + c_off[w];
  if (threadIdx.x == 0) {
    int d[24];
    float u[6][24];
    wood_point(M, S, P[i], pa, pb, pn, d, u);
    for (int t = 0; t < 24; ++t) {
      di[t] = d[t];
      for (int j = 0; j < 6; ++j) ui[j][t] = u[j][t];
    }
  }
  __syncthreads();
  for (int j = 0; j < np; ++j) {
    if (threadIdx.x == 0) {
      int d[24];
      float u[6][24];
      wood_point(M, S, P[j], pa, pb, pn, d, u);
      for (int t = 0; t < 24; ++t) {
        dj[t] = d[t];
        for (int q = 0; q < 6; ++q) uj[q][t] = u[q][t];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 576; e += blockDim.x) {
      const int s = e / 24, t = e % 24;
      kb[s][t] = K[(long long)di[s] * n + dj[t]];
    }
    __syncthreads();
    if (threadIdx.x < 144) {   // ku = K^+[D_i, D_j] u_j
      const int s = threadIdx.x / 6, q = threadIdx.x % 6;
      float v = 0.f;
      for (int t = 0; t < 24; ++t) v += kb[s][t] * uj[q][t];
      ku[s][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 36) {
      const int a = threadIdx.x / 6, q = threadIdx.x % 6;
      float v = 0.f;
      for (int s = 0; s < 24; ++s) v += ui[a][s] * ku[s][q];
      C[(long long)(6 * i + a) * r + 6 * j + q] = (i == j && a == q ? 1.f : 0.f) - v;
    }
    __syncthreads();
  }
}

// Z_b^T for point i = blockIdx.y of subdomain list[blockIdx.x]: rows 6i..6i+5 of the r x n_bd
// array at z_pool + z_off[w]:  Zt[6i + q][k] = sum_t u_q[t] K^+[D_i[t], boundary dof k].
__global__ void __launch_bounds__(256) k_wood_Zb(DevMesh M, const int* __restrict__ list,
                                                 const long long* __restrict__ pt_off, const int* __restrict__ pts,
                                                 const int* __restrict__ n_pts, const float* __restrict__ kinv,
                                                 const long long* __restrict__ kinv_off, const double* __restrict__ pa,
                                                 const double* __restrict__ pb, const double* __restrict__ pn,
                                                 const long long* __restrict__ z_off, float* z_pool) {
  __shared__ int di[24];
  __shared__ float ui[6][24];
  const int w = blockIdx.x, i = blockIdx.y;
  const int np = n_pts[w];
  if (i >= np) return;
  const SubDev S = M.subs[list[w]];
  const int n = S.n_dof, n_bd = 3 * S.n_bnd;
  const float* K = kinv + kinv_off[S.shape];
  float* Zt = z_pool + z_off[w];
  if (threadIdx.x == 0) {
    int d[24];
    float u[6][24];
    wood_point(M, S, pts[pt_off[w] + i], pa, pb, pn, d, u);
    for (int t = 0; t < 24; ++t) {
      di[t] = d[t];
      for (int q = 0; q < 6; ++q) ui[q][t] = u[q][t];
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n_bd; k += blockDim.x) {
    const int dof = 3 * M.shape_bln[S.bnd_off + k / 3] + k % 3;
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int t = 0; t < 24; ++t) {
      const float kv = K[(long long)di[t] * n + dof];   // K^+ is symmetric
#pragma unroll
      for (int q = 0; q < 6; ++q) acc[q] += ui[q][t] * kv;
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) Zt[(long long)(6 * i + q) * n_bd + k] = acc[q];
  }
}

// Blocked Cholesky C = L L^T in place (lower triangle), panels of kBlk columns, all subdomains
// in each launch: for panel p, k_wood_chol_diag factors the diagonal block (one CTA per
// subdomain, in shared memory) and stores the inverse of its factor in dinv (kBlk x kBlk per
// panel); k_wood_chol_trsm forms the panel below it, L_ip = C_ip L_pp^-T; k_wood_chol_syrk
// updates the trailing lower triangle, C_ij -= L_ip L_jp^T, one kBlk x kBlk tile per CTA.
// A non-positive pivot sets *err bit 8 (the host then keeps the banded solves).
constexpr int kBlk = 32;

__device__ __forceinline__ int wood_nblk(int r) { return (r + kBlk - 1) / kBlk; }

__global__ void __launch_bounds__(256) k_wood_chol_diag(const int* __restrict__ n_pts,
                                                        const long long* __restrict__ c_off, float* c_pool,
                                                        const long long* __restrict__ d_off, float* d_pool, int p,
                                                        int* err) {
  __shared__ float A[kBlk][kBlk + 1], Li[kBlk][kBlk + 1];
  const int w = blockIdx.x, r = 6 * n_pts[w];
  const int k0 = p * kBlk;
  if (k0 >= r) return;
  const int jb = min(kBlk, r - k0);
  float* C = c_pool + c_off[w];
  for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
    const int i = e / kBlk, j = e % kBlk;
    A[i][j] = (i < jb && j < jb) ? C[(long long)(k0 + i) * r + k0 + j] : (i == j ? 1.f : 0.f);
    Li[i][j] = i == j ? 1.f : 0.f;
  }
  __syncthreads();
  for (int k = 0; k < kBlk; ++k) {   // right-looking in shared memory
    if (threadIdx.x == 0) {
      if (!(A[k][k] > 0.f)) atomicOr(err, 8);
      A[k][k] = sqrtf(fmaxf(A[k][k], 1e-30f));
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < kBlk; i += blockDim.x) A[i][k] /= A[k][k];
    __syncthreads();
    for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
      const int i = e / kBlk, j = e % kBlk;
      if (i > k && j > k && j <= i) A[i][j] -= A[i][k] * A[j][k];
    }
    __syncthreads();
  }
  // inverse of the lower factor, one column per thread (forward substitution of unit vectors)
  if (threadIdx.x < kBlk) {
    const int c = threadIdx.x;
    for (int i = 0; i < kBlk; ++i) {
      float v = i == c ? 1.f : 0.f;
      for (int q = c; q < i; ++q) v -= A[i][q] * Li[q][c];
      Li[i][c] = i >= c ? v / A[i][i] : 0.f;
    }
  }
  __syncthreads();
  float* D = d_pool + d_off[w] + (long long)p * kBlk * kBlk;
  for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
    const int i = e / kBlk, j = e % kBlk;
    D[e] = Li[i][j];
    if (i < jb && j < jb && j <= i) C[(long long)(k0 + i) * r + k0 + j] = A[i][j];
  }
}

__global__ void __launch_bounds__(256) k_wood_chol_trsm(const int* __restrict__ n_pts,
                                                        const long long* __restrict__ c_off, float* c_pool,
                                                        const long long* __restrict__ d_off,
                                                        const float* __restrict__ d_pool, int p) {
  __shared__ float X[kBlk][kBlk + 1], Li[kBlk][kBlk + 1];
  const int w = blockIdx.x, r = 6 * n_pts[w];
  const int k0 = p * kBlk, i0 = (p + 1 + blockIdx.y) * kBlk;
  if (i0 >= r) return;
  const int ib = min(kBlk, r - i0), jb = min(kBlk, r - k0);
  float* C = c_pool + c_off[w];
  const float* D = d_pool + d_off[w] + (long long)p * kBlk * kBlk;
  for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
    const int i = e / kBlk, j = e % kBlk;
    X[i][j] = (i < ib && j < jb) ? C[(long long)(i0 + i) * r + k0 + j] : 0.f;
    Li[i][j] = D[e];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {   // L_ip = X Li^T
    const int i = e / kBlk, j = e % kBlk;
    if (i >= ib || j >= jb) continue;
    float v = 0.f;
    for (int q = 0; q <= j; ++q) v += X[i][q] * Li[j][q];
    C[(long long)(i0 + i) * r + k0 + j] = v;
  }
}

__global__ void __launch_bounds__(256) k_wood_chol_syrk(const int* __restrict__ n_pts,
                                                        const long long* __restrict__ c_off, float* c_pool, int p) {
  __shared__ float Li[kBlk][kBlk + 1], Lj[kBlk][kBlk + 1];
  const int w = blockIdx.x, r = 6 * n_pts[w];
  const int nb = wood_nblk(r) - p - 1;            // trailing blocks
  // tile t of the trailing lower triangle: (bi, bj), bj <= bi
  int t = blockIdx.y, bi = 0;
  while (bi < nb && t > bi) t -= ++bi;
  if (bi >= nb) return;
  const int bj = t;
  const int k0 = p * kBlk, i0 = (p + 1 + bi) * kBlk, j0 = (p + 1 + bj) * kBlk;
  const int ib = min(kBlk, r - i0), jb = min(kBlk, r - j0), kb = min(kBlk, r - k0);
  float* C = c_pool + c_off[w];
  for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
    const int i = e / kBlk, q = e % kBlk;
    Li[i][q] = (i < ib && q < kb) ? C[(long long)(i0 + i) * r + k0 + q] : 0.f;
    Lj[i][q] = (i < jb && q < kb) ? C[(long long)(j0 + i) * r + k0 + q] : 0.f;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
    const int i = e / kBlk, j = e % kBlk;
    if (i >= ib || j >= jb || (bi == bj && j > i)) continue;
    float v = 0.f;
#pragma unroll 8
    for (int q = 0; q < kBlk; ++q) v += Li[i][q] * Lj[j][q];
    C[(long long)(i0 + i) * r + j0 + j] -= v;
  }
}

// Y = C^-1 Z_b^T in place of the r x n_bd array Y (a copy of Z_b^T), for 32 boundary columns per
// CTA (blockIdx.y): forward Y_b = Li_b (Y_b - sum_{a<b} L_ba Y_a), then backward
// Y_b = Li_b^T (Y_b - sum_{a>b} L_ab^T Y_a), with the stored inverses Li_b of the diagonal blocks.
// The column chunk of Y sits in shared memory (r x 32 floats).
__global__ void __launch_bounds__(256) k_wood_subst(const SubDev* __restrict__ subs, const int* __restrict__ list,
                                                    const int* __restrict__ n_pts, const long long* __restrict__ c_off,
                                                    const float* __restrict__ c_pool, const long long* __restrict__ d_off,
                                                    const float* __restrict__ d_pool,
                                                    const long long* __restrict__ z_off, float* y_pool) {
  extern __shared__ float ys[];     // [r][kBlk]
  __shared__ float T[kBlk][kBlk + 1];
  const int w = blockIdx.x, r = 6 * n_pts[w];
  const int n_bd = 3 * subs[list[w]].n_bnd;
  const int col0 = blockIdx.y * kBlk;
  if (col0 >= n_bd) return;
  const int cb = min(kBlk, n_bd - col0);
  const float* C = c_pool + c_off[w];
  const float* D = d_pool + d_off[w];
  float* Y = y_pool + z_off[w];
  for (int e = threadIdx.x; e < r * kBlk; e += blockDim.x) {
    const int i = e / kBlk, j = e % kBlk;
    ys[e] = j < cb ? Y[(long long)i * n_bd + col0 + j] : 0.f;
  }
  __syncthreads();
  const int nbk = wood_nblk(r);
  for (int pass = 0; pass < 2; ++pass) {
    for (int s = 0; s < nbk; ++s) {
      const int b = pass == 0 ? s : nbk - 1 - s;
      const int b0 = b * kBlk, bb = min(kBlk, r - b0);
      // T = Y_b - sum over the solved blocks (forward: a < b, L_ba; backward: a > b, L_ab^T)
      for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
        const int i = e / kBlk, j = e % kBlk;
        float v = i < bb ? ys[(b0 + i) * kBlk + j] : 0.f;
        if (i < bb) {
          if (pass == 0) {
            for (int q = 0; q < b0; ++q) v -= C[(long long)(b0 + i) * r + q] * ys[q * kBlk + j];
          } else {
            for (int q = b0 + bb; q < r; ++q) v -= C[(long long)q * r + b0 + i] * ys[q * kBlk + j];
          }
        }
        T[i][j] = v;
      }
      __syncthreads();
      const float* Li = D + (long long)b * kBlk * kBlk;
      for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
        const int i = e / kBlk, j = e % kBlk;
        if (i >= bb) continue;
        float v = 0.f;
        if (pass == 0)
          for (int q = 0; q <= i; ++q) v += Li[i * kBlk + q] * T[q][j];
        else
          for (int q = i; q < bb; ++q) v += Li[q * kBlk + i] * T[q][j];
        ys[(b0 + i) * kBlk + j] = v;
      }
      __syncthreads();
    }
  }
  for (int e = threadIdx.x; e < r * kBlk; e += blockDim.x) {
    const int i = e / kBlk, j = e % kBlk;
    if (j < cb) Y[(long long)i * n_bd + col0 + j] = ys[e];
  }
}

// Correction of the inner F-apply, in three launches spread over many CTAs (the per-subdomain
// products are a few MB each and one CTA per subdomain would leave them latency-bound):
// k_wood_x: x_b = B^T lam at the boundary dofs of subdomain list[blockIdx.x] -> xbuf + w * xstride;
// k_wood_t: t = Y x_b, one row per warp, kWoodRows rows per CTA (blockIdx.y) -> tbuf + w * tstride;
// k_wood_y: cbuf[slots] += Z_b t for 64 boundary dofs per CTA (blockIdx.y), four threads per dof
// splitting the sum over the rows, combined in shared memory in a fixed order.
constexpr int kWoodRows = 8;

__global__ void __launch_bounds__(256) k_wood_x(DevMesh M, const int* __restrict__ list, const double* __restrict__ lam,
                                                float* xbuf, int xstride) {
  const int w = blockIdx.x;
  const SubDev S = M.subs[list[w]];
  const int n_bd = 3 * S.n_bnd;
  const int k = blockIdx.y * blockDim.x + threadIdx.x;
  if (k >= n_bd) return;
  const int sl = M.sub_b2s[S.b2s_off + k / 3];
  xbuf[(long long)w * xstride + k] = sl >= 0 ? (float)bt_at_slot(M, lam, (long long)sl + k % 3) : 0.f;
}

__global__ void __launch_bounds__(256) k_wood_t(const SubDev* __restrict__ subs, const int* __restrict__ list,
                                                const int* __restrict__ n_pts, const long long* __restrict__ y_off,
                                                const float* __restrict__ y_pool, const float* __restrict__ xbuf,
                                                int xstride, float* tbuf, int tstride) {
  const int w = blockIdx.x;
  const int r = 6 * n_pts[w];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.y * kWoodRows + warp;
  if (c >= r) return;
  const int n_bd = 3 * subs[list[w]].n_bnd;
  const float* yr = y_pool + y_off[w] + (long long)c * n_bd;
  const float* xb = xbuf + (long long)w * xstride;
  float v = 0.f;
#pragma unroll 8
  for (int k = lane; k < n_bd; k += 32) v += __ldg(yr + k) * __ldg(xb + k);
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) tbuf[(long long)w * tstride + c] = v;
}

__global__ void __launch_bounds__(256) k_wood_y(DevMesh M, const int* __restrict__ list, const int* __restrict__ n_pts,
                                                const long long* __restrict__ z_off, const float* __restrict__ z_pool,
                                                const float* __restrict__ tbuf, int tstride, double* cbuf) {
  __shared__ float part[4][64];
  const int w = blockIdx.x;
  const int r = 6 * n_pts[w];
  const SubDev S = M.subs[list[w]];
  const int n_bd = 3 * S.n_bnd;
  const int k0 = blockIdx.y * 64;
  if (k0 >= n_bd) return;
  const int kk = threadIdx.x & 63, q = threadIdx.x >> 6, k = k0 + kk;
  const float* Zt = z_pool + z_off[w];
  const float* t = tbuf + (long long)w * tstride;
  float v = 0.f;
  if (k < n_bd) {
    const int c0 = q * ((r + 3) / 4), c1 = min(r, c0 + (r + 3) / 4);
#pragma unroll 4
    for (int c = c0; c < c1; ++c) v += __ldg(Zt + (long long)c * n_bd + k) * __ldg(t + c);
  }
  part[q][kk] = v;
  __syncthreads();
  if (q == 0 && k < n_bd) {
    const int sl = M.sub_b2s[S.b2s_off + k / 3];
    if (sl >= 0) cbuf[(long long)sl + k % 3] += (double)(((part[0][kk] + part[1][kk]) + part[2][kk]) + part[3][kk]);
  }
}

}  // namespace

void launch_wood_setup(const DevMesh& M, const WoodArgs& a, cudaStream_t st) {
  if (a.n <= 0) return;
  k_wood_points<<<a.n, 256, 0, st>>>(M, a.list, a.pt_off, a.n_pts, a.plastic, a.pts);
  k_wood_C<<<dim3((unsigned)a.n, (unsigned)a.max_pts), 256, 0, st>>>(M, a.list, a.pt_off, a.pts, a.n_pts, a.kinv,
                                                                     a.kinv_off, a.pa, a.pb, a.pn, a.c_off,
                                                                     a.c_pool);
  k_wood_Zb<<<dim3((unsigned)a.n, (unsigned)a.max_pts), 256, 0, st>>>(M, a.list, a.pt_off, a.pts, a.n_pts, a.kinv,
                                                                      a.kinv_off, a.pa, a.pb, a.pn, a.z_off,
                                                                      a.z_pool);
  // Zt is copied to the Y pool, which the substitution overwrites with C^{-1} Z_b^T
  cudaMemcpyAsync(a.y_pool, a.z_pool, sizeof(float) * (size_t)a.z_total, cudaMemcpyDeviceToDevice, st);
  const int rmax = 6 * a.max_pts, nb = (rmax + kBlk - 1) / kBlk;
  for (int p = 0; p < nb; ++p) {
    k_wood_chol_diag<<<a.n, 256, 0, st>>>(a.n_pts, a.c_off, a.c_pool, a.d_off, a.d_pool, p, a.err);
    if (p + 1 < nb) {
      const int t = nb - p - 1;
      k_wood_chol_trsm<<<dim3((unsigned)a.n, (unsigned)t), 256, 0, st>>>(a.n_pts, a.c_off, a.c_pool, a.d_off,
                                                                          a.d_pool, p);
      k_wood_chol_syrk<<<dim3((unsigned)a.n, (unsigned)(t * (t + 1) / 2)), 256, 0, st>>>(a.n_pts, a.c_off,
                                                                                          a.c_pool, p);
    }
  }
  const size_t smem = sizeof(float) * (size_t)rmax * kBlk;
  cudaFuncSetAttribute(k_wood_subst, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_wood_subst<<<dim3((unsigned)a.n, (unsigned)((a.max_bd + kBlk - 1) / kBlk)), 256, smem, st>>>(
      M.subs, a.list, a.n_pts, a.c_off, a.c_pool, a.d_off, a.d_pool, a.z_off, a.y_pool);
}

int wood_setup_launches(const WoodArgs& a) {
  const int nb = (6 * a.max_pts + kBlk - 1) / kBlk;
  return 5 + 3 * nb - 2;
}

void launch_wood_apply(const DevMesh& M, const WoodArgs& a, const double* lam, double* cbuf, cudaStream_t st) {
  if (a.n <= 0) return;
  const int rmax = 6 * a.max_pts;
  k_wood_x<<<dim3((unsigned)a.n, (unsigned)((a.max_bd + 255) / 256)), 256, 0, st>>>(M, a.list, lam, a.xbuf, a.max_bd);
  k_wood_t<<<dim3((unsigned)a.n, (unsigned)((rmax + kWoodRows - 1) / kWoodRows)), 256, 0, st>>>(
      M.subs, a.list, a.n_pts, a.z_off, a.y_pool, a.xbuf, a.max_bd, a.tbuf, rmax);
  k_wood_y<<<dim3((unsigned)a.n, (unsigned)((a.max_bd + 63) / 64)), 256, 0, st>>>(M, a.list, a.n_pts, a.z_off,
                                                                                   a.z_pool, a.tbuf, rmax, cbuf);
}

}  // namespace tfeti
