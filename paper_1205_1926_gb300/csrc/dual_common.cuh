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

// (B^T x) at U copy slots at once (slot < 0 gives 0), each value summed as bt_at_slot sums it.
// The loads run stage by stage over the U slots (their groups, the groups' headers, then each
// value's first Helmert term), so that the U chains of dependent loads overlap; the further
// terms (copies shared by more than two subdomains) follow in a loop.
template <int U>
__device__ __forceinline__ void bt_at_slots(const DevMesh& M, const double* __restrict__ x, const long long* slot,
                                            double* out) {
  int g[U], j[U];
#pragma unroll
  for (int k = 0; k < U; ++k) {
    g[k] = slot[k] >= 0 ? __ldg(M.slot_group + slot[k]) : -1;
    j[k] = slot[k] >= 0 ? __ldg(M.slot_j + slot[k]) : 0;
  }
  int4 hd[U];   // GroupDev header: row0, k, nrows, dirichlet
#pragma unroll
  for (int k = 0; k < U; ++k)
    hd[k] = g[k] >= 0 ? __ldg(reinterpret_cast<const int4*>(M.groups + g[k])) : make_int4(0, 0, 0, 0);
  double xv[U], hv[U];
  int r0[U];
#pragma unroll
  for (int k = 0; k < U; ++k) {
    r0[k] = hd[k].w ? j[k] : (j[k] > 1 ? j[k] : 1);
    const bool any = hd[k].z != 0 && (hd[k].w || r0[k] < hd[k].y);
    xv[k] = any ? x[hd[k].x + r0[k] - (hd[k].w ? 0 : 1)] : 0.0;
    hv[k] = any && !hd[k].w ? __ldg(M.helm + r0[k] * 8 + j[k]) : 0.0;
  }
#pragma unroll
  for (int k = 0; k < U; ++k) {
    if (hd[k].z == 0) {
      out[k] = 0.0;
    } else if (hd[k].w) {
      out[k] = xv[k];
    } else {
      double s = 0.0;
      if (r0[k] < hd[k].y) {
        s += hv[k] * xv[k];
        for (int r = r0[k] + 1; r < hd[k].y; ++r) s += M.helm[r * 8 + j[k]] * x[hd[k].x + r - 1];
      }
      out[k] = s;
    }
  }
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
