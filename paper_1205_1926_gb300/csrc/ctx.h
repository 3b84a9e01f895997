// Internal definition of the device context (shared by the library's host
// translation units; not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "dev.h"
#include "plan.h"

struct tfeti_ctx {
  // all members are owned by the context and released by tfeti_destroy
  tfeti::Plan plan;
  cudaStream_t st = nullptr;
  bool owns_stream = false;          // st was created by the context (case contexts without a stream)
  int device = 0;                    // CUDA device current at set-up (the context's device)
  // case context (tfeti_setup_case): the context whose read-only set-up this one shares
  tfeti_ctx* base = nullptr;
  std::string err;
  std::vector<void*> allocs;
  size_t bytes = 0;
  tfeti::DevMesh M{};
  long long l = 0;
  // tables and maps
  tfeti::SubDev* d_subs = nullptr;
  std::vector<tfeti::SubDev> h_subs;
  // state
  double *u = nullptr, *sig = nullptr, *kap = nullptr;
  // Newton iterate
  double *du = nullptr, *df = nullptr, *dsig = nullptr, *dkap = nullptr, *pa = nullptr, *pb = nullptr, *pn = nullptr;
  double* fe = nullptr;   // [n_elem][8][3] element parts of the internal force
  uint8_t* plastic = nullptr;
  int *elem_np = nullptr, *sub_np = nullptr;
  double* dKe = nullptr;
  double* band = nullptr;            // band matrices of the shape templates
  std::vector<long long> tmpl_off;   // per shape
  double* fac = nullptr;             // factor records of the shape templates
  float* fac32 = nullptr;            // the same records rounded to FP32 (mixed-precision inner solves)
  // factor records of the subdomains with plastic points: one slot each (slot_size
  // values, the largest record), taken when a subdomain first has plastic points and
  // given back when it is elastic again; the pools grow on demand and keep their
  // records.  The Dirichlet K_ii factors use the same slot numbers in their own pools.
  double* fac_own = nullptr;
  float* fac32_own = nullptr;
  double* dfac_own = nullptr;
  float* dfac32_own = nullptr;
  long long slot_size = 0;
  int slot_cap = 0;
  std::vector<int> slot_of, free_slots;
  double* band_ws = nullptr;         // band workspace of the refactorisations (grows on demand)
  long long band_ws_cap = 0;
  std::vector<tfeti::SolveItem> h_items32;
  tfeti::SolveItem* d_items32 = nullptr;
  int n_items32 = 0;
  int rcap32 = 1;
  size_t solve_smem32 = 0;
  int precision = 0;                 // TFETI_PRECISION_*
  double inner_rtol = 1e-3;
  double *dlt = nullptr, *rin = nullptr;
  long long f32_launches = 0;
  // dual Schur blocks of the shapes' elastic templates (mixed precision)
  float* S32 = nullptr;
  // FP64 Schur F-apply (tfeti_set_fapply): S in FP64 [s_total], gathered X [n_sub][max n_bd],
  // FP64 items of the subdomains with plastic points (their banded solves on st2)
  int fapply = 0;                            // TFETI_FAPPLY_*
  // per shape: S formed (shapes with at least kSchurMinCount subdomains), compact offsets
  // of S and its tiles, and whether the inner F-apply uses it (count >= schur_threshold,
  // the threshold picked by timing the FP32 F-apply for a few candidates)
  std::vector<char> schur_formed, schur_use;
  std::vector<long long> s_off_c;
  int schur_threshold = 0;
  std::vector<float> schur_tune_ms;          // measured FP32 F-apply per candidate threshold
  std::vector<int> h_np;                     // plastic points per subdomain at the last assembly
  double *S64 = nullptr, *X64 = nullptr;
  tfeti::SolveItem* d_items_pl64 = nullptr;
  int n_items_pl64 = 0;
  double g_ms = 0.0, g_flops = 0.0, g_bytes = 0.0;
  long long g_launches = 0;
  // tensor-core operand tiles (TF32 hi/lo parts): S per shape at s_tile_off[shape] (elements),
  // the gathered interface vectors of one shape's elastic subdomains (TF32 hi/lo, or BF16
  // hi/lo in the same buffers); Sbf: the BF16 copy of the S tiles (same element offsets),
  // formed when the BF16 format is first chosen
  float *Shi = nullptr, *Slo = nullptr, *Xhi = nullptr, *Xlo = nullptr;
  void* Sbf = nullptr;
  bool schur_bf16 = false;                   // inner Schur apply with BF16 S (else TF32 x 3)
  bool schur_manual = false;                 // threshold set by tfeti_set_schur_threshold (no re-tuning)
  // Plastic subdomains on their shape's elastic factor plus a Woodbury correction
  // (kernels_woodbury.cu): dense FP64 K^+ per shape (kinv_off[shape] >= 0 where formed; a case
  // context shares the base's), the subdomains handled that way after the last assembly and
  // their pools (grown on demand, contents not kept).  wood_mode: 0 off, 1 the inner FP32
  // F-apply only (the subdomains are still refactorised for the FP64 solves), 2 also the FP64
  // solves (no refactorisation).
  int wood_mode = 2;
  double* kinv = nullptr;
  std::vector<long long> kinv_off;
  long long* d_kinv_off = nullptr;
  std::vector<char> h_wood;                  // per subdomain: on the Woodbury correction
  std::vector<int> h_np_all;                 // plastic points per subdomain at the last assembly
  tfeti::WoodArgs wood;
  int* d_wood_list = nullptr;
  int* d_wood_np = nullptr;
  long long *d_wood_pt_off = nullptr, *d_wood_c_off = nullptr, *d_wood_z_off = nullptr, *d_wood_d_off = nullptr,
            *d_wood_zt_off = nullptr;
  int *d_wood_pts = nullptr, *wood_dofs = nullptr;
  double *wood_u = nullptr, *wood_zt = nullptr, *wood_c64 = nullptr, *wood_d64 = nullptr;
  double *wood_v = nullptr, *wood_t64 = nullptr, *wood_yb = nullptr;
  float *wood_c = nullptr, *wood_d = nullptr, *wood_z = nullptr, *wood_y = nullptr, *wood_t = nullptr;
  long long wood_pts_cap = 0, wood_dofs_cap = 0, wood_u_cap = 0, wood_zt_cap = 0, wood_c64_cap = 0,
            wood_d64_cap = 0, wood_c_cap = 0, wood_d_cap = 0, wood_z_cap = 0, wood_y_cap = 0,
            wood_v_cap = 0, wood_yb_cap = 0;
  long long wood_subs = 0, wood_fallbacks = 0, wood_fac_saved = 0;
  // set-up inside a load step: on st_wood beside the first residual solve; the context stream waits
  // for ev_wood_done before the first use (wood_pending) and the host reads the pivots' status at its
  // next synchronisation (wood_check_pending)
  cudaStream_t st_wood = nullptr;
  cudaEvent_t ev_wood_fork = nullptr, ev_wood_done = nullptr;
  // the FP64 Woodbury correction of a timed subdomain-solve pass runs on st_wc beside the pass (it
  // reads only the pass's inputs); the context stream waits for ev_wc_done before adding it
  cudaStream_t st_wc = nullptr;
  cudaEvent_t ev_wc_fork = nullptr, ev_wc_done = nullptr;
  int* d_err_wood = nullptr;
  int* h_err_wood = nullptr;
  bool wood_pending = false, wood_check_pending = false;
  // fused inner iteration (kernels_inner.cu): one cooperative launch between two F-applies
  bool fused_req = false;                    // tfeti_set_fused_inner
  bool g_inner_fused = false;                // the built graph body uses it
  bool in_cases = false;                     // inside ssn_time_step_cases with other contexts
  tfeti::LumpTask* d_lump = nullptr;
  int n_lump = 0, lump_cap = 0, lump_max_nr = 0;
  bool lump_stale = true;
  float* xslot = nullptr;
  unsigned* d_bar = nullptr;
  int inner_grid_n = -1;                     // CTAs of the fused launch (0: not possible, -1: not asked)
  size_t inner_smem_b = 0;
  float* s_part = nullptr;                   // output tiles of the Schur apply, one set per K split
  std::vector<long long> s_tile_off;
  bool schur_ready = false;
  int* d_el = nullptr;                       // elastic subdomains grouped by shape
  std::vector<int> h_el, el_off, el_cnt;     // per shape: offset and count into d_el
  tfeti::SolveItem* d_items_pl = nullptr;    // FP32 items of the subdomains with plastic points
  int n_items_pl = 0;
  tfeti::SolveItem* d_items_s = nullptr;     // column items for forming S
  cudaStream_t st2 = nullptr;
  // refactorisation of the plastic subdomains inside a load step runs on st_fac while the
  // elastic items of the next residual solve run on st; st joins at ev_fac_done before the
  // first item that reads an own record (fac_pending), the host checks the pivots afterwards
  cudaStream_t st_fac = nullptr;
  cudaEvent_t ev_fac_fork = nullptr, ev_fac_done = nullptr;
  bool fac_pending = false, fac_check_pending = false, fac_timed = false;
  int* d_err_fac = nullptr;
  int* h_err_fac = nullptr;          // pinned
  int n_items_el = 0;                // FP64 items on shape templates (they come first in d_items)
  long long f_split = 0;             // FP64 passes split around a deferred refactorisation (untimed)
  cudaStream_t st_cap = nullptr;     // private stream used only to capture graphs
  // CUDA graph of the mixed-precision inner PCGP: a WHILE node whose body is one iteration
  cudaGraph_t g_inner = nullptr;
  cudaGraphExec_t g_inner_exec = nullptr;
  bool g_inner_stale = true;
  int g_body_kernels = 0;
  bool use_graphs = true;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::vector<long long> tmpl_fac_off;   // per shape
  tfeti::SolveItem* d_items = nullptr;   // solve work items (device), rebuilt after each assembly
  std::vector<tfeti::SolveItem> h_items;
  int n_items = 0;
  int rec_max = 0, npad = 0, rcap = 1;
  size_t solve_smem = 0;
  int n_sm = 1;
  int* d_list = nullptr;
  long long* d_list_off = nullptr;
  long long* d_list_fac = nullptr;
  double* kbb = nullptr;               // boundary 3x3 blocks: template pool then per-subdomain pool
  long long own_kbb_base = 0;
  long long* d_kbb_off = nullptr;      // per subdomain: template or own offset
  std::vector<long long> h_kbb_off;
  long long* d_kbb_off32 = nullptr;    // the same for the inner FP32 lumped preconditioner: the template
  std::vector<long long> h_kbb_off32;  //   for subdomains on the Woodbury path
  long long* d_list_kbb = nullptr;
  int* d_klist = nullptr;                    // plastic subdomains of the last assembly (K_bb refresh)
  int max_bnd = 0;
  // dual
  double *cbuf = nullptr, *lam = nullptr, *lam_im = nullptr, *lamk = nullptr, *r = nullptr, *w = nullptr,
         *z = nullptr, *y = nullptr, *pdir = nullptr, *Fp = nullptr, *tm = nullptr;
  double* vsol = nullptr;   // K^+(f - B^T lambda) of the last residual solve, device [n_dof]
  // Dirichlet preconditioner (Sec. 4.2): factors of K_p with the constrained-node dofs
  // replaced by identity rows and columns (K_ii), one template per (shape, pattern of
  // constrained dofs) class for elastic subdomains, own ones for plastic subdomains
  bool dirichlet = false;
  uint8_t* d_bmask = nullptr;               // 1 at the local dofs of constrained nodes, [n_dof]
  std::vector<int> dclass, dclass_rep;      // class of each subdomain; a representative of each class
  std::vector<long long> dtmpl_off;         // per class: offset of its factor in dfac
  double* dfac = nullptr;
  float* dfac32 = nullptr;
  std::vector<tfeti::SolveItem> h_items_d, h_items_d32;
  tfeti::SolveItem *d_items_d = nullptr, *d_items_d32 = nullptr;
  int n_items_d = 0, n_items_d32 = 0;
  double *dx_a = nullptr, *dx_b = nullptr, *dx_c = nullptr;   // [n_dof] work vectors
  // history start (tfeti_set_recycling): ring of the last rec_q solutions lambda_Ker and
  // their products F lambda_Ker, [rec_q][n_mult] each
  int rec_q = 0, rec_n = 0, rec_head = 0;
  // deflated inner PCGP (tfeti_set_deflation): W (up to kDeflMax vectors in range(P_N)), A W with
  // the inner FP32 operator, E^-1 = (W^T A W)^-1 over the independent vectors; defl_req: the
  // requested size, defl_k: the size formed for the current dual solve (0 until its first inner
  // solve); mlp_slot_valid: the last start formed the network's prediction in slot rec_n
  int defl_req = 0, defl_k = 0;
  bool defl_formed = false, mlp_slot_valid = false;
  bool mlp_consulted = false;   // this solve's start consulted the network
  double *defl_W = nullptr, *defl_AW = nullptr, *defl_Einv = nullptr;
  long long defl_setups = 0, defl_vectors = 0, defl_fallbacks = 0;
  double *rec_L = nullptr, *rec_FL = nullptr, *rec_partial = nullptr, *rec_out = nullptr, *rec_c = nullptr;
  double* dtil = nullptr;        // d~ of the current solve (kept when the history start is on)
  double rec_accept = 0.5;       // try the start if the predicted ||P r|| < rec_accept ||P d~||
  long long rec_tried = 0, rec_used = 0, rec_exact = 0;
  // operator versions: 0 for the all-elastic tangent, a new number for every other assembly; a stored
  // solution whose version equals the current one has its exact FP64 products F lambda_j and
  // w_j = K^+ B^T lambda_j ([rec_q + 1][n_dof] in rec_W), so a start built from such solutions alone
  // gets its residual and primal vector by linear combination instead of a residual solve
  long long op_ver = 0, ver_counter = 0;
  std::vector<long long> rec_ver;
  double* rec_W = nullptr;
  double* vsol_im = nullptr;                 // K^+ (f - B^T lambda_Im) of the current dual solve
  // per-interface MLP of the learned start (tfeti_set_learned): FP32 master weights and
  // Adam moments, FP16 copy for inference, the first-Newton-solve solutions of the last
  // two load steps, per-subdomain plastic fractions, the previous load increment
  // (histories per Newton index 1..kMlpIdx: [kMlpIdx][n_mult] and [kMlpIdx][n_sub])
  bool mlp_on = false, have_dfprev = false, mlp_missed = false;   // missed: the history alone fell short
  int newton_idx = 0;                 // Newton iteration of the running dual solve (0: not inside Newton)
  int mlp_epochs = 8, mlp_t = 0, mlp_blocks = 64;
  int mlp_seen[tfeti::kMlpIdx] = {0, 0, 0, 0};
  float mlp_lr = 1e-3f;
  float *mlp_w = nullptr, *mlp_m1 = nullptr, *mlp_m2 = nullptr, *mlp_partial = nullptr, *mlp_scal = nullptr;
  void* mlp_w16 = nullptr;
  double *mlp_la = nullptr, *mlp_lb = nullptr, *mlp_dfprev = nullptr;
  float *pf_now = nullptr, *pf_prev = nullptr;
  double mlp_rho = 1.0;
  float h_scal[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  bool mlp_scal_valid = false;
  // training runs on its own low-priority stream, beside the next Newton iteration: the inputs that
  // the next solve overwrites (d~, lambda_Ker, the plastic fractions, the scalings) are copied first,
  // and every later reader of the network's weights or histories waits for ev_mlp_done
  cudaStream_t st_mlp = nullptr;
  cudaEvent_t ev_mlp_fork = nullptr, ev_mlp_done = nullptr;
  bool mlp_pending = false;
  double *mlp_d = nullptr, *mlp_tgt = nullptr;
  float *mlp_pf = nullptr, *mlp_scal_t = nullptr;
  long long mlp_used = 0, mlp_skipped = 0, mlp_probe = 0;
  int mlp_nogain[tfeti::kMlpIdx] = {0, 0, 0, 0};   // consecutive solves where the network added < 10 %
  // FP32 copies for the inner iterations of the mixed mode (allocated by tfeti_set_precision)
  float *H32 = nullptr, *kbb32 = nullptr;
  double *H = nullptr, *gx = nullptr, *hx = nullptr, *ev = nullptr, *alpha = nullptr;
  float* hx8 = nullptr;              // FP32 H g padded to 8 per subdomain (FP32 projector)
  float* gx32 = nullptr;             // FP32 G x of the FP32 projector (the coarse GEMV's input)
  double *f_full = nullptr, *tn = nullptr, *tn2 = nullptr;
  // coarse solve (dense explicit H or the plane solver's blocks; a case context shares the base's)
  tfeti::CoarseOp coarse;
  double *cW = nullptr, *cV = nullptr, *cU = nullptr, *cAoff = nullptr;
  float *cW32 = nullptr, *cV32 = nullptr, *cU32 = nullptr;
  double *partial = nullptr, *sc = nullptr, *h_sc = nullptr;
  int* d_ctr = nullptr;                      // arrival counters of the fused inner-iteration kernels
  int* d_err = nullptr;
  int max_copy = 0;
  // timing
  bool events = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<uint8_t> ev_kind;             // per event pair: 0 banded F-apply, 1 Schur F-apply
  size_t ev_used = 0;
  cudaEvent_t fac_e0 = nullptr, fac_e1 = nullptr;
  cudaEvent_t in_e0 = nullptr, in_e1 = nullptr;   // around each inner-solve graph launch (timing on)
  double inner_ms = 0.0;                           // device time of the timed inner solves
  long long inner_its = 0, inner_runs = 0;         // their PCGP iterations and body runs
  double f_ms = 0.0, factor_ms = 0.0;
  long long f_launches = 0, factor_launches = 0, launches = 0;
  std::vector<int> last_refactored;
};
