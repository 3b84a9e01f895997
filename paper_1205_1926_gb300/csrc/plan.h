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
};

struct ShapeInfo {
  int dims[3];
  int n_dof, bw, n_elem;
  int64_t band_off;   // template (elastic) band storage offset in the template pool
  int64_t r_off;      // offset of R (n_dof x 6, row-major) in the R pool
  int rep_sub;        // a subdomain of this shape
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
  std::vector<SubInfo> subs;
  std::vector<ShapeInfo> shapes;
  std::vector<Group> groups;
  // per copy slot: group index, index j within group, local dof, subdomain
  std::vector<int32_t> slot_group, slot_j, slot_ldof, slot_sub;
  // per row: group index and row index within group
  std::vector<int32_t> row_group, row_r;
  // lumped preconditioner structure: per interface node (3 slots), up to 27
  // neighbour interface nodes of the same subdomain (slot base, or -1)
  std::vector<int32_t> ell_nbr;   // [n_copy/3][27]: neighbour's first slot or -1
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
