// Device helpers for the orthonormal constraint matrix B (Sec. 4.1) acting
// between multiplier space and the interface copy slots of the subdomains.
#pragma once
#include "dev.h"

namespace tfeti {

// (B^T x) at one copy slot: Dirichlet groups carry one identity row per copy;
// free groups carry Helmert rows r = 1..k-1, whose coefficient for copy j is
// helm[r][j] (non-zero for j <= r).
__device__ __forceinline__ double bt_at_slot(const DevMesh& M, const double* __restrict__ x, long long slot) {
  const GroupDev& g = M.groups[M.slot_group[slot]];
  const int j = M.slot_j[slot];
  if (g.nrows == 0) return 0.0;
  if (g.dirichlet) return x[g.row0 + j];
  double s = 0.0;
  for (int r = (j > 1 ? j : 1); r < g.k; ++r) s += M.helm[r * 8 + j] * x[g.row0 + r - 1];
  return s;
}

// (B v)[row] for copy-slot values v.
__device__ __forceinline__ double b_at_row(const DevMesh& M, const double* __restrict__ v, long long row) {
  const GroupDev& g = M.groups[M.row_group[row]];
  const int rr = M.row_r[row];
  if (g.dirichlet) return v[g.slot[rr]];
  const int r = rr + 1;
  double s = 0.0;
  for (int j = 0; j <= r; ++j) s += M.helm[r * 8 + j] * v[g.slot[j]];
  return s;
}

}  // namespace tfeti
