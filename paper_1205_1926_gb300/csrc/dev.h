// Device-side data structures and kernel entry points of the TFETI library.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace tfeti {

constexpr int kMaxNB = 32;     // row block of the banded factor / solves
constexpr int kTri24 = 300;    // packed lower triangle of a 24x24 element matrix

struct SubDev {
  int origin[3], dims[3], nn[3];
  int n_dof, n_elem, bw, nb, shape, n_copy;
  int fix[6];
  int nblk, rec;              // factor row blocks; doubles per off-diagonal panel record
  int n_bnd;                  // box-boundary nodes of its shape
  long long dof_off, elem_off, band_off, copy_off, r_off;
  long long bnd_off;          // its shape's boundary tables (shape_bln, 27 x for shape_tnbr)
  long long b2s_off;          // its boundary index -> first copy slot table
};

constexpr int kMaxRHS = 4;     // right-hand sides one solve CTA carries
constexpr int kSchurMinCount = 4;   // shapes with fewer subdomains never form their dual Schur block

// One CTA of the subdomain solve: up to kMaxRHS subdomains of one shape that
// share the factor record at `fac` (the elastic template) or a single
// subdomain with its own factor.
// A work item's factor record: an offset into the shape-template pool, or, with the
// kOwnFac bit set, into the pool of records of subdomains with plastic points.
constexpr long long kOwnFac = 1LL << 62;
struct SolveItem {
  long long fac;
  int count;
  int sub[kMaxRHS];
};

struct GroupDev {
  int row0, k, nrows, dirichlet;
  int slot[8];
  int sub[8];
};
// kernels read the header (row0, k, nrows, dirichlet) of a group as one 16-byte load
static_assert(sizeof(GroupDev) % 16 == 0 && offsetof(GroupDev, dirichlet) == 12, "GroupDev header layout");

// Everything a kernel needs to know about the mesh and the decomposition.
struct DevMesh {
  const SubDev* subs;
  int n_sub;
  const GroupDev* groups;
  const int* slot_group;
  const int* slot_j;
  const int* slot_ldof;
  const int* slot_sub;
  const int* row_group;
  const int* row_r;
  const int* shape_bln;     // box-boundary node -> local node, per shape
  const int* shape_tnbr;    // [boundary node][27] neighbour boundary index or -1, per shape
  const int* sub_b2s;       // boundary index -> first copy slot or -1, per subdomain
  const int* slot_bnd;      // copy slot -> boundary index of its node
  const int* sub_nbr;       // [interface node][28] first slot of each stencil neighbour or -1
  const int* bt_ptr;        // B^T by copy slot (CSR over multiplier rows): bt_ptr[n_copy + 1],
  const int* bt_row;        //   rows bt_row[e] and coefficients bt_val[e]
  const double* bt_val;
  const int* elem_sub;     // subdomain of every element
  const double* R;         // rigid-body bases per shape, [n_dof][6] row-major
  const double* dN;        // [8 g][8 a][3] physical shape-function gradients
  const double* Kel;       // [24][24] elastic brick stiffness
  const double* Q;         // [8 g][24][24] w detJ B_g^T E_eps B_g
  const double* helm;      // [8 r][8 j] Helmert coefficients (row r = 1..7, copy j)
  // G = R^T B^T explicitly (it depends only on B and R): one entry per (multiplier
  // row, copy slot) with B[row][slot] != 0, value B[row][slot] * R[slot dof][0..5].
  // Subdomain order: entries gp_ptr[p]..gp_ptr[p+1] of subdomain p, their rows gp_row,
  // values Gv / Gv32 [entry][6].  Row order: entries gt_ptr[row]..gt_ptr[row+1],
  // subdomain gt_p, values GTv / GTv32 [entry][6].
  const long long* gp_ptr;
  const int* gp_row;
  const double* Gv;
  const float* Gv32;
  const long long* gt_ptr;
  const int* gt_p;
  const double* GTv;
  const float* GTv32;
  long long n_gpairs;
  double wdet;
  // trilinear gradient weights on the uniform bricks: ga[d] = (1 + 1/sqrt 3) / (2 h_d) and
  // gb[d] = (1 - 1/sqrt 3) / (2 h_d), the nodal weights of a Gauss point on the same and on the
  // other side of the element along direction d, divided by h_d
  double ga[3], gb[3];
  double lam, mu, sigma_y, H;
  long long n_dof, n_gp, n_mult, n_copy, n_elem;
  long long n_groups;
};

// Per-Newton-iterate Gauss-point data used by the assembly.
struct GPData {
  const double* dsig;      // [6][n_gp]
  const double* pa;        // [n_gp] 2 mu c (1 - rho)  (0 if elastic)
  const double* pb;        // [n_gp] 2 mu c rho
  const double* pn;        // [6][n_gp] n-bar
  const uint8_t* plastic;  // [n_gp]
};

// ---- launchers (all enqueue on `st`) -------------------------------------
void launch_tables(const double* h, double lam, double mu, double* dN, double* Kel, double* Q, cudaStream_t st);
void launch_rigid_for_shape(const SubDev& S, const double* h, double* R_shape, cudaStream_t st);
void launch_traction(const DevMesh& M, int face, const int* nel, const double* t, const double* h, double* f,
                     cudaStream_t st);
// Internal force f = df - F(dsig) of eq. (F_def): element contributions into fe
// ([element][8 nodes, bit order x + 2y + 4z][3]), then gathered per dof in a fixed order.
void launch_internal_force(const DevMesh& M, const double* dsig, const double* df, double* fe, double* f,
                           cudaStream_t st);
void launch_return_map(const DevMesh& M, const double* du, const double* sig_k, const double* kap_k,
                       double* dsig, double* dkap, uint8_t* plastic, double* Dtan, double* pa, double* pb,
                       double* pn, cudaStream_t st);
void launch_elem_correction(const DevMesh& M, GPData gp, int* elem_np, int* sub_np, double* dKe, cudaStream_t st);
void launch_band_fill(const DevMesh& M, const int* sub_list, int n_list, const int* elem_np, const double* dKe,
                      double* band, const long long* band_off_list, int elastic_only, int max_rows, int max_bw,
                      cudaStream_t st,
                      const uint8_t* bmask = nullptr);
// Boundary 3x3 blocks of K for the listed subdomains (elastic_only: the shape's elastic template);
// also rounded to FP32 into kbb32 at the same offsets when kbb32 != null.  Per subdomain the
// 27 x 9 values of its n_bnd boundary nodes are stored [t][cc][3 b + a]: K[3 node_b + a][3 nbr_t + cc].
void launch_kbb_fill(const DevMesh& M, const int* sub_list, const long long* dst_off, int n_list, int max_bnd,
                     const int* elem_np, const double* dKe, double* kbb, float* kbb32, int elastic_only,
                     cudaStream_t st);
void launch_apply_K(const DevMesh& M, const int* elem_np, const double* dKe, const double* x, double* y,
                    cudaStream_t st);
void launch_commit(const DevMesh& M, const double* du, const double* dsig, const double* dkap, double* u,
                   double* sig, double* kap, cudaStream_t st);
void launch_vm_max(const DevMesh& M, const double* dsig, double* partial, double* out, cudaStream_t st);

// Banded Cholesky of K_rr in the band workspace, writing the factor record
// (off-diagonal panels M_b = L_bb^{-1} L_b,off and the inverted diagonal blocks).
void launch_band_chol(const DevMesh& M, const int* sub_list, int n_list, const long long* band_off_list,
                      double* band, const long long* fac_off_list, double* fac, int* err, int max_bw,
                      int n_sm, cudaStream_t st);

// Subdomain K^+ solve.  in_mode 0: x = B^T lam at the interface slots (zero
// elsewhere); 1: x = src - B^T lam (lam nullable); 4: see bmask.  out_mode 0: interface slots
// to cbuf; 1: full local vector to dst (+ R alpha if alpha != null); 3: both.
struct SolveArgs {
  const double* lam;
  const double* src;
  double* cbuf;
  double* dst;
  const double* alpha;
  const double* fac;           // factor pool (FP64)
  const float* fac32;          // the same records rounded to FP32 (used when fp32 != 0)
  const double* fac_own;       // records of subdomains with plastic points (items with kOwnFac)
  const float* fac32_own;
  int fp32;                    // 1: FP32 arithmetic (inner solves of the mixed-precision PCGP)
  const SolveItem* items;
  int n_items;
  int in_mode, out_mode;
  int* err;                    // bit 2 set if a bounded wait on a panel copy gives up
  int rec_max;                 // largest panel record of the launch (doubles, even)
  int npad;                    // vector stride in shared memory (largest n, even)
  int rcap;                    // vectors allocated per CTA (>= every item's count)
  // in_mode 2 / out_mode 2 (dual Schur block formation of one shape): item.sub[] hold
  // boundary-dof columns j; the geometry is subdomain rep_sub; column j of
  // S = (K^+)_{boundary, boundary} goes to S32 + s_off + j * n_bd.
  // in_mode 5 / out_mode 4 (dense K^+ of one shape): item.sub[] hold local dofs j; column j
  // of K^+ (all n rows, zero at the fixing dofs) goes to S64 + s_off + j * n
  int rep_sub;
  float* S32;
  double* S64;                 // nullable: the same columns in FP64
  long long s_off;
  // in_mode 4 (Dirichlet preconditioner): x = src with the dofs marked in bmask zeroed;
  // no_fix: the factor has no fixing dofs (they are not zeroed before and after)
  const uint8_t* bmask;
  int no_fix;
};
int smem_optin_max();
int dyn_smem_limit(const void* fn);
void launch_sub_solve(const DevMesh& M, const SolveArgs& a, size_t smem_bytes, cudaStream_t st);
size_t sub_solve_smem(int rec_max, int npad, int rcap, int elem_bytes);
// FP64 dual Schur block applied to the elastic subdomains of one shape: X[k][i] =
// (B^T lam) at boundary dof i of subdomain sub_list[k] (row-major [n_list][n_bd]),
// then cbuf at the interface slots = (X S)[k][i], S64[j * n_bd + i] = S[i][j].
void launch_schur_gather64(const DevMesh& M, const int* sub_list, int n_list, int n_bd, const double* lam, double* X,
                           cudaStream_t st);
void launch_schur_dgemm_scatter(const DevMesh& M, const int* sub_list, int n_list, int n_bd, const double* X,
                                const double* S, double* cbuf, cudaStream_t st);
// Dual Schur block applied to the elastic subdomains of one shape on the tensor
// cores: X[k][i] = (B^T lam) at boundary dof i of subdomain sub_list[k] (0 off the
// interface), split into hi/lo tiles (TF32 floats, or BF16 halves with bf16); then
// cbuf at the interface slots = (X S)[k][i].  S tiles (TF32 hi/lo, or one BF16 copy)
// are formed once from the FP32 block S32 (S32[j * n_bd + i] = S[i][j]).  The GEMM's
// output tiles (with splits > 1, one partial per split of the K range) go to `part`
// (schur_part_floats), from which a second kernel sums the splits in order and writes
// the slots.  err: bit 4 set if a bounded wait gives up.
int schur_nk(int n_bd);
int schur_tiles(int n_list, int n_bd);
int schur_splits(int n_list, int n_bd, int n_sm);
long long schur_x_tile_elems(int n_list, int n_bd);   // elements of each of Xhi, Xlo
long long schur_s_tile_elems(int n_bd);               // elements of each of Shi, Slo (Slo unused with BF16)
long long schur_part_floats(int n_list, int n_bd, int splits);
void launch_schur_tile_S(const float* S32, int n_bd, bool bf16, void* Shi, void* Slo, cudaStream_t st);
void launch_schur_gather(const DevMesh& M, const int* sub_list, int n_list, int n_bd, bool bf16, const double* lam,
                         void* Xhi, void* Xlo, cudaStream_t st);
void launch_schur_gemm_scatter(const DevMesh& M, const int* sub_list, int n_list, int n_bd, bool bf16, int splits,
                               const void* Xhi, const void* Xlo, const void* Shi, const void* Slo, float* part,
                               double* cbuf, int* err, cudaStream_t st);
// Plastic subdomains on their shape's elastic factor plus a Woodbury correction
// (kernels_woodbury.cu).  list: the n subdomains (r = 6 n_pts[w] correction columns each, n dofs,
// n_bd boundary dofs).  Per subdomain w: pts + pt_off[w] its plastic points; u_pool +
// 144 pt_off[w] the r x 24 U and dof_pool + 24 pt_off[w] the points' 24 local dofs; zt_pool +
// zt_off[w] Z^T = (K^+ U)^T (r x n, FP64); c_pool + c_off[w] C = I - U^T Z, then its lower
// Cholesky factor (r x r, FP64), d_pool + d_off[w] the inverses of its 32 x 32 diagonal blocks;
// c32_pool / d32_pool the same rounded to FP32; z_pool + z_off[w] Z_b^T (r x n_bd, FP32) and
// y_pool + z_off[w] Y = C^-1 Z_b^T.  kinv: dense FP64 K^+ per shape at kinv_off[shape].
// err: bit 8 set if a Cholesky pivot of C is not positive.
constexpr int kWoodMaxN = 3072;    // shapes with at most this many dofs keep a dense K^+
constexpr int kWoodMaxPts = 96;    // subdomains with more plastic points keep the banded solve
struct WoodArgs {
  int n = 0, max_pts = 0, max_bd = 0, max_n = 0, max_copy = 0;
  bool fp64 = false;                 // the FP64 solves run on the elastic factor + correction
  const int* list = nullptr;
  const long long* pt_off = nullptr;
  const int* n_pts = nullptr;
  int* pts = nullptr;
  const uint8_t* plastic = nullptr;
  const double *pa = nullptr, *pb = nullptr, *pn = nullptr;
  const double* kinv = nullptr;
  const long long* kinv_off = nullptr;
  double* u_pool = nullptr;
  int* dof_pool = nullptr;
  const long long* zt_off = nullptr;
  double* zt_pool = nullptr;
  const long long* c_off = nullptr;
  double* c_pool = nullptr;
  float* c32_pool = nullptr;
  long long c_total = 0;
  const long long* d_off = nullptr;
  double* d_pool = nullptr;
  float* d32_pool = nullptr;
  long long d_total = 0;
  const long long* z_off = nullptr;
  float *z_pool = nullptr, *y_pool = nullptr;
  long long z_total = 0;
  float* tbuf = nullptr;             // [n][6 max_pts]: t = Y x_b of the inner apply
  double* vbuf = nullptr;            // [n][max_n]: v of the FP64 correction
  double* tbuf64 = nullptr;          // [n][6 max_pts]: t = Z^T v, then C^-1 t
  double* ybuf = nullptr;            // [n][max_n]: y = Z C^-1 t
  int* err = nullptr;
};
void launch_wood_setup(const DevMesh& M, const WoodArgs& a, cudaStream_t st);
int wood_setup_launches(const WoodArgs& a);
// Inner (FP32) F-apply correction: cbuf at the subdomains' interface slots += Z_b Y x_b.
void launch_wood_apply(const DevMesh& M, const WoodArgs& a, const double* lam, double* cbuf, cudaStream_t st);
// FP64 correction after a subdomain solve of the list's subdomains on the elastic factor with
// right-hand side v = src + sign B^T lam (src, lam nullable; sign -1 for in_mode 1, +1 for in_mode
// 0): y = Z C^-1 Z^T v is added to dst (the decomposed vector, nullable) and to cbuf at the
// interface slots (nullable).  Returns the number of launches.
int launch_wood_apply64(const DevMesh& M, const WoodArgs& a, const double* src, const double* lam, double sign,
                        double* cbuf, double* dst, cudaStream_t st);
// The same correction in two parts, so that the first can run beside the subdomain solve (it
// reads only the solve's inputs): launch_wood_corr64 forms y = Z C^-1 Z^T v in ybuf;
// launch_wood_add64 then adds it to dst and to cbuf at the copy slots (each nullable).
// Both return their launch counts.
int launch_wood_corr64(const DevMesh& M, const WoodArgs& a, const double* src, const double* lam, double sign,
                       cudaStream_t st);
int launch_wood_add64(const DevMesh& M, const WoodArgs& a, double* cbuf, double* dst, cudaStream_t st);

// dst[i] = (float) src[i], i < n.
void launch_to_f32(const double* src, float* dst, long long n, cudaStream_t st);
// FP32 copies of factor records (offsets in entries, same for both pools)
void launch_fac_to_f32(const double* fac, float* fac32, const long long* off_list, int n_list, long long len,
                       cudaStream_t st);

void launch_contract(const DevMesh& M, const double* cbuf, double* y, cudaStream_t st);
void launch_G_apply(const DevMesh& M, const double* x_lam, const double* x_full, double* gx, double scale,
                    cudaStream_t st);
void launch_GT_update(const DevMesh& M, const double* x, double ax, const double* h, double bh, double* out,
                      cudaStream_t st);
void launch_gemv(const double* A, long long n, const double* x, double alpha, double* y, cudaStream_t st);
// out = v + R alpha per subdomain (u = K^+(f - B^T lambda) + R alpha); device [n_dof].
void launch_add_R_alpha(const DevMesh& M, const double* v, const double* alpha, double* out, int max_ndof,
                       cudaStream_t st);
void launch_lumped(const DevMesh& M, const double* w, const double* kbb, const long long* kbb_off, double* cbuf,
                   cudaStream_t st, int max_copy);
// The coarse solve h = H g, H = (G G^T)^-1 (Sec. 4.2's projector).  Dense: the explicit
// inverse H (l x l, and its FP32 copy H32 with rows padded to h32_ld(l)), one GEMV.  Planes:
// G G^T is block tridiagonal over the planes of subdomains with equal z index (a subdomain
// couples only to the 26 boxes around it), n_planes blocks of n_pl = 6 x (subdomains per
// plane); a block LDL^T with explicit inverses W_k of the pivots and the products V_k, U_k
// turns the solve into 2 n_planes - 1 dependent GEMVs of n_pl x n_pl (coarse_planes_factor).
constexpr int kCoarseDense = 0, kCoarsePlanes = 1;
constexpr long long kCoarseDenseMax = 6144;   // TFETI_COARSE_AUTO: dense H up to this n_coarse
struct CoarseOp {
  int mode = kCoarseDense;
  long long l = 0;
  const double* H = nullptr;
  const float* H32 = nullptr;
  int n_pl = 0, n_planes = 0;
  const double *W = nullptr, *V = nullptr, *U = nullptr;      // [n_planes][n_pl][n_pl]
  const float *W32 = nullptr, *V32 = nullptr, *U32 = nullptr;
};
// y = alpha H x in FP64 (x and y distinct).
void coarse_apply(const CoarseOp& C, const double* x, double alpha, double* y, cudaStream_t st);
// y = H x with the FP32 copies (FP32 products and sums), and y8, its FP32 copy padded to 8
// values per subdomain.
// x32 (nullable): x already rounded to FP32 (the dense GEMV then reads it instead of converting x).
void coarse_apply32(const CoarseOp& C, const double* x, const float* x32, double* y, float* y8, cudaStream_t st);
int coarse_launches(const CoarseOp& C);
void launch_coarse_assemble_planes(const DevMesh& M, const int* pair_p, const int* pair_q, const long long* pair_start,
                                   const int* trip_group, const int* trip_i, const int* trip_j, long long n_pairs,
                                   double* Adiag, double* Aoff, int per_plane, int n_pl, int n_planes,
                                   cudaStream_t st);
void coarse_planes_factor(double* W, const double* Aoff, double* V, double* U, int n, int np, double* T,
                          double* work, int* err, cudaStream_t st);

// FP32 operators of the inner iterations of the mixed mode (FP64 vectors in and out):
// P x with the FP32 copies of R and of the coarse solve, and the lumped preconditioner with
// the FP32 copy of the boundary blocks.  gx, hx: coarse work vectors [l].
// hx8: FP32 copy of H g padded to 8 values per subdomain (entries 6, 7 zero), [n_sub][8].
// G values in FP32 (M.Gv32, M.GTv32) are stored 8 per entry (6 and two zeros).
void launch_project32(const DevMesh& M, const CoarseOp& C, const double* x, double* gx, float* gx32, double* hx,
                      float* hx8, double* out, cudaStream_t st);
inline long long h32_ld(long long l) { return (l + 3) & ~3LL; }
void launch_h_to_f32(const double* H, long long l, float* H32, cudaStream_t st);
// Values of the explicit G from R and the (row, slot, coefficient) entries (set-up).
void launch_fill_G(const DevMesh& M, const int* gp_slot, const double* gp_coef, const int* gt_e, double* Gv,
                   float* Gv32, double* GTv, float* GTv32, cudaStream_t st);
// Dirichlet preconditioner pieces: xfull = B^T w on the copy-slot dofs, 0 elsewhere
// (xfull zeroed by the caller); cbuf[slot] = v[dof] - t[dof] on the copy slots.
void launch_slots_to_full(const DevMesh& M, const double* w, double* xfull, cudaStream_t st);
void launch_slots_diff(const DevMesh& M, const double* v, const double* t, double* cbuf, cudaStream_t st);
void launch_lumped32(const DevMesh& M, const double* w, const float* kbb32, const long long* kbb_off, double* cbuf,
                     cudaStream_t st, int max_copy);

// The inner PCGP iteration between two F-applies as one cooperative launch (kernels_inner.cu):
// contraction of F p and p.Fp, the lambda and r updates (body launches), then w = P r, the lumped
// preconditioner, y = P z and the new search direction, with grid barriers between the phases.
// The lumped preconditioner runs by tasks: up to kLumpR subdomains that share their boundary
// blocks (kbb32 + kbb; the elastic subdomains of a shape share its template) and a range
// [row0, row1) of those blocks' rows.
constexpr int kLumpR = 4;
struct LumpTask {
  long long kbb;
  int count, row0, row1, pad;
  int sub[kLumpR];
};
struct InnerArgs {
  DevMesh M;
  const float* H32 = nullptr;        // dense FP32 H, rows padded to ld
  long long l = 0, ld = 0;
  const float* kbb32 = nullptr;
  const LumpTask* tasks = nullptr;
  int n_tasks = 0, max_nr = 0;       // max_nr: largest 3 n_bnd of the tasks' shapes
  double *r = nullptr, *w = nullptr, *z = nullptr, *y = nullptr, *p = nullptr, *Fp = nullptr, *lam = nullptr;
  double* cbuf = nullptr;
  float* xslot = nullptr;            // [n_copy]: B^T w at the copy slots
  double *gx = nullptr, *hx = nullptr;
  float* hx8 = nullptr;
  double* sc = nullptr;
  double* partial = nullptr;         // [3][grid]
  unsigned* bar = nullptr;           // grid barrier (count, generation), count zero between launches
  int* err = nullptr;                // bit 32: a grid-barrier wait gave up
  unsigned long long cond = 0;       // WHILE handle of the graph body (has_cond)
  int has_cond = 0;
  int body = 0;                      // 1: starts with the contraction and the updates
};
size_t inner_smem(const InnerArgs& a);
int inner_grid(int n_sm, size_t smem);   // CTAs of the launch (one per SM), 0 if it cannot run
cudaError_t launch_inner(const InnerArgs& a, int grid, size_t smem, cudaStream_t st);

// Deterministic reductions and PCG vector updates
constexpr int kRedBlocks = 304;

// History start of the dual PCGP: at most kRecMax stored solutions.  Gram system
// out[i * kRecMax + j] = L_i . FL_j, out[kRecMax^2 + i] = L_i . d (L, FL: q vectors
// of length m, stride m); partial: kRedBlocks * (kRecMax^2 + kRecMax) doubles.
constexpr int kRecMax = 8;

// Per-interface MLP of the learned start (kernels_mlp.cu).  scal (device, 5 floats):
// 1/s, 1/s_d, rho, s, the Newton-index feature, with s = RMS of the previous step's
// lambda and s_d = RMS of d~.  kMlpIdx: Newton iterations with their own histories.
constexpr int kMlpIn = 8, kMlpHid = 64, kMlpBatch = 128, kMlpIdx = 4;
constexpr int kMlpParams = kMlpHid * kMlpIn + kMlpHid + kMlpHid * kMlpHid + kMlpHid + kMlpHid + 1;
size_t mlp_grad_smem();
void launch_mlp_infer(const DevMesh& M, const void* w16, const double* la, const double* lb, const double* d,
                      const float* pf_now, const float* pf_prev, const float* scal, double* y, cudaStream_t st);
// One Adam step on nblocks x kMlpBatch rows (start + i * stride mod n_mult); partial:
// nblocks x kMlpParams floats.
void launch_mlp_train_step(const DevMesh& M, const float* wm, const double* la, const double* lb, const double* d,
                           const float* pf_now, const float* pf_prev, const float* scal, const double* target,
                           long long start, long long stride, int nblocks, float* partial, float* wm_out, float* m1,
                           float* m2, void* w16, float lr, int t, cudaStream_t st);
void launch_plastic_fraction(const DevMesh& M, const int* sub_np, float* pf, cudaStream_t st);
void launch_mlp_cast(const float* wm, void* w16, cudaStream_t st);
void launch_rec_gram(const double* L, const double* FL, const double* d, int q, long long m, double* partial,
                     double* out, cudaStream_t st);
// out = (base ? base : 0) + sign * sum_j c_j X_j, c device [q].
void launch_rec_combine(const double* X, const double* c, int q, long long m, const double* base, double sign,
                        double* out, cudaStream_t st);

// Device scalars of the graph-driven PCGP (indices into the context's scalar array)
enum PcgScalar {
  kYW = 0, kYWPrev = 1, kPFP = 2, kWW = 3,
  kDone = 20, kStatus = 21, kStopAfter = 22, kFirst = 23, kTol2 = 24, kIter = 25, kMaxit = 26, kLastWW = 27,
  kBodyRuns = 28, kDeflK = 29, kMu0 = 32, kNumScalars = 48
};
// Deflated inner PCGP: at most kDeflMax deflation vectors W (in range(P)), their products
// A W with the inner operator, and E^-1 = (W^T A W)^-1 ([kDeflMax][kDeflMax]); the size in
// use is sc[kDeflK] (0: plain PCGP) and mu = E^-1 (AW)^T y sits at sc[kMu0 ..].
constexpr int kDeflMax = 8;
void launch_pcg_init(double* sc, double tol2, int maxit, cudaStream_t st);
void launch_dot2(const double* x1, const double* y1, const double* x2, const double* y2, long long n,
                 double* partial, double* out1, double* out2, cudaStream_t st);
// Fused kernels of the graph-driven inner iteration (grid kFusedBlocks; each dot is summed by the
// block that arrives last, in block order; ctr: one zeroed int per kernel, left zero; partial:
// (1 + kDeflMax) x kFusedBlocks doubles).  With deflation (AW, Einv, W given and sc[kDeflK] > 0)
// GT32_dot mode 1 also forms mu = E^-1 (AW)^T y and p_update subtracts W mu.  GT32_dot: out = x - G^T h8 and sc[kWW] = out.out (mode 0) or
// sc[kYW] = out.v plus the stop test (mode 1).  contract_dot: Fp = B cbuf, sc[kPFP] = p.Fp plus
// the breakdown test.  lam_r_update_post: the guarded updates, then the body run is closed and,
// with has_h, the WHILE condition h set.  G32_coarse32: gx = G x and hx = H gx in FP32 (+ padded hx8).
constexpr int kFusedBlocks = 608;
void launch_G32_coarse32(const DevMesh& M, const CoarseOp& C, const double* x, double* gx, float* gx32, double* hx,
                         float* hx8, cudaStream_t st);
void launch_GT32_dot(const DevMesh& M, const double* x, const float* h8, double* out, const double* v, int mode,
                     double* sc, double* partial, int* ctr, cudaStream_t st, const double* AW = nullptr,
                     const double* Einv = nullptr);
void launch_contract_dot(const DevMesh& M, const double* cbuf, double* Fp, const double* p, double* sc,
                         double* partial, int* ctr, cudaStream_t st);
void launch_lam_r_update_post(long long n, const double* p, const double* Fp, double* lam, double* r, double* sc,
                              int* ctr, unsigned long long h, int has_h, cudaStream_t st);
void launch_pcg_pre(double* sc, cudaStream_t st);
void launch_pcg_mid(double* sc, cudaStream_t st);
void launch_pcg_post(double* sc, unsigned long long cond_handle, cudaStream_t st);
// guarded updates: no-ops once sc[kDone] is set
void launch_p_update_g(long long n, const double* y, double* p, const double* sc, cudaStream_t st,
                       const double* W = nullptr);
void launch_lam_r_update_g(long long n, const double* p, const double* Fp, double* lam, double* r, const double* sc,
                           cudaStream_t st);
void launch_dot(const double* x, const double* y, long long n, double* partial, double* out, cudaStream_t st);
void launch_axpby(long long n, double a, const double* x, double b, const double* y, double* out, cudaStream_t st);
void launch_p_update(long long n, const double* y, double* p, const double* sc, int first, cudaStream_t st);
void launch_lam_r_update(long long n, const double* p, const double* Fp, double* lam, double* r, double* sc,
                         cudaStream_t st);

// Coarse problem
void launch_coarse_assemble(const DevMesh& M, const int* pair_p, const int* pair_q, const long long* pair_start,
                            const int* trip_group, const int* trip_i, const int* trip_j, long long n_pairs,
                            double* A, long long l, cudaStream_t st);
long long dense_inverse_work(long long l);
int dense_cholesky_inverse(double* A, double* work, long long l, int* err, cudaStream_t st);

}  // namespace tfeti
