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

// Scalar logic of the inner PCGP (state in sc, see PcgScalar): pre -- after y.w of the
// iteration: the finiteness and stop tests; mid -- after p.Fp: the breakdown test; post -- at the
// end of a body run: the counters and the done flag; returns whether another body run follows.
__device__ __forceinline__ void pcg_pre_logic(double* sc) {
  if (sc[kDone] != 0.0) return;
  const double ww = sc[kWW], yw = sc[kYW];
  sc[kLastWW] = ww;
  if (!isfinite(ww) || !isfinite(yw)) {
    sc[kDone] = 1.0;
    sc[kStatus] = 8.0;
    return;
  }
  if (sc[kFirst] != 0.0 && !(ww > 0.0)) {   // w^0 = 0: nothing to do
    sc[kDone] = 1.0;
    sc[kStopAfter] = 1.0;
    return;
  }
  sc[kStopAfter] = ww <= sc[kTol2] ? 1.0 : 0.0;
}

__device__ __forceinline__ void pcg_mid_logic(double* sc) {
  if (sc[kDone] != 0.0) return;
  if (!(sc[kPFP] > 0.0)) {
    sc[kDone] = 1.0;
    sc[kStatus] = 7.0;
  }
}

// Closes one body run; returns whether the WHILE loop goes on.
__device__ __forceinline__ bool pcg_post_logic(double* sc) {
  sc[kBodyRuns] += 1.0;
  if (sc[kDone] == 0.0) {
    sc[kYWPrev] = sc[kYW];
    sc[kIter] += 1.0;
    sc[kFirst] = 0.0;
    if (sc[kStopAfter] != 0.0 || sc[kIter] >= sc[kMaxit]) sc[kDone] = 1.0;
  }
  return sc[kDone] == 0.0 && sc[kBodyRuns] < 2.0 * sc[kMaxit] + 4.0;
}

}  // namespace tfeti
