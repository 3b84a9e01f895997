// Host-side plan: mesh numbering, box subdomains, copies of nodes, the
// orthonormal constraint matrix B (Sec. 4.1) as groups of copies, interface
// copy slots, fixing dofs (Remark 1) and the index lists the kernels use.
// Pure integer/index work plus the closed-form Helmert coefficients; no GPU.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tfeti.h"

namespace tfeti {

struct SubInfo {
  int origin[3];      // element index of the lower corner
  int dims[3];        // elements per axis
  int nn[3];          // nodes per axis
  int n_nodes, n_dof, n_elem;
  int bw;             // half bandwidth in dofs of the lexicographic local order
  int shape;          // shape class (subdomains with equal dims share one)
  int64_t dof_off, elem_off;
  int64_t band_off;   // offset (doubles) of this subdomain's band storage
  int64_t copy_off;   // first interface copy slot
  int n_copy;         // interface copy slots (3 per interface node)
  int fix[6];         // fixing dofs (local)
  int nb, nblk;       // factor block size and number of row blocks
  int rec;            // entries per off-diagonal panel record (nb * bw, rounded to a multiple of 4)
  int64_t fac_off;    // offset (doubles) of this subdomain's factor record in the own pool
  int64_t fac_size;   // doubles of one factor record: nblk * rec + nblk * nb * nb
  int64_t b2s_off;    // offset into Plan::sub_b2s (n_bnd of its shape entries)
  int64_t kbb_off;    // offset of its own boundary blocks in the per-subdomain pool
};

struct ShapeInfo {
  int dims[3];
  int n_dof, bw, n_elem;
  int64_t band_off;   // template (elastic) band storage offset in the template pool
  int64_t r_off;      // offset of R (n_dof x 6, row-major) in the R pool
  int rep_sub;        // a subdomain of this shape
  int64_t fac_off;    // offset of the shape's elastic factor record in the template pool
  int n_bnd;          // nodes on the box boundary
  int64_t bnd_off;    // offset into Plan::shape_bln (and 27 x into Plan::shape_tnbr)
  int64_t kbb_off;    // offset of the shape's elastic boundary blocks in the template pool
  int64_t s_off;      // offset of the shape's elastic dual Schur block (3 n_bnd)^2 in the S pool
};

// One (global node, component) with its copies.  rows = k (Dirichlet), k-1
// (free, k >= 2) or 0.
struct Group {
  int64_t row0;
  int k;
  int nrows;
  int dirichlet;
  int64_t slot[8];    // interface copy slots of the k copies (subdomain order)
  int sub[8];
};

struct Plan {
  tfeti_problem prob{};
  std::vector<int> cuts[3];
  int nsub[3];
  double h[3];
  int64_t n_nodes = 0, n_elem = 0, n_gp = 0, n_dof = 0, n_mult = 0, n_copy = 0;
  int max_bw = 0, max_ndof = 0;
  int64_t band_total = 0, template_band_total = 0, r_total = 0;
  int64_t fac_total = 0, template_fac_total = 0;
  std::vector<SubInfo> subs;
  std::vector<ShapeInfo> shapes;
  std::vector<Group> groups;
  // per copy slot: group index, index j within group, local dof, subdomain
  std::vector<int32_t> slot_group, slot_j, slot_ldof, slot_sub;
  // per row: group index and row index within group
  std::vector<int32_t> row_group, row_r;
  // lumped preconditioner structure.  Per shape: the box-boundary nodes (local
  // node ids) and, for each, its 27 stencil neighbours as boundary indices (or -1).
  // Per subdomain: boundary index -> first copy slot of that node (or -1).
  // Per copy slot: the boundary index of its node.  Blocks of K are stored per
  // boundary node and neighbour as 3x3 (27 x 9 doubles per boundary node).
  std::vector<int32_t> shape_bln, shape_tnbr, sub_b2s, slot_bnd;
  // per interface node (3 slots): first slot of each of its 27 stencil neighbours
  // that is an interface node of the same subdomain, or -1; padded to 28 entries
  std::vector<int32_t> sub_nbr;
  int64_t kbb_template_total = 0, kbb_total = 0;
  int64_t s_total = 0;       // floats of all shapes' dual Schur blocks
  // coarse matrix pairs (p, q) with p >= q that share at least one group,
  // and per pair the list of (group, i, j) triples
  std::vector<int32_t> pair_p, pair_q;
  std::vector<int64_t> pair_start;
  std::vector<int32_t> trip_group, trip_i, trip_j;
  std::string error;
};

int plan_build(const tfeti_problem* prob, Plan& plan);
double helmert_coef(int r, int j);   // coefficient of copy j (0-based) in Helmert row r (1-based)

}  // namespace tfeti
