// Host plan construction (Sec. 4.1 tearing; Remark 1 fixing dofs).  See plan.h.
#include "plan.h"

#include <algorithm>
#include <array>
#include <new>
#include <cmath>
#include <map>
#include <utility>

namespace tfeti {

double helmert_coef(int r, int j) {
  // Helmert row r (1-based): copies 0..r-1 get 1/sqrt(r(r+1)), copy r gets -r/sqrt(r(r+1)).
  const double s = 1.0 / std::sqrt((double)r * (r + 1.0));
  if (j < r) return s;
  if (j == r) return -r * s;
  return 0.0;
}

static bool bad(Plan& plan, const char* msg) {
  plan.error = msg;
  return true;
}

int plan_build(const tfeti_problem* prob, Plan& plan) {
  if (!prob) { plan.error = "null problem"; return TFETI_ERR_ARG; }
  plan.prob = *prob;
  for (int d = 0; d < 3; ++d) plan.prob.cuts[d] = nullptr;
  for (int d = 0; d < 3; ++d) {
    if (prob->nel[d] < 1 || prob->nsub[d] < 1 || prob->nsub[d] > prob->nel[d] || !(prob->length[d] > 0))
      return bad(plan, "bad nel/nsub/length"), TFETI_ERR_ARG;
    auto& c = plan.cuts[d];
    c.resize(prob->nsub[d] + 1);
    if (prob->cuts[d]) {
      for (int i = 0; i <= prob->nsub[d]; ++i) c[i] = prob->cuts[d][i];
    } else {
      if (prob->nel[d] % prob->nsub[d]) return bad(plan, "nel not divisible by nsub"), TFETI_ERR_ARG;
      for (int i = 0; i <= prob->nsub[d]; ++i) c[i] = i * (prob->nel[d] / prob->nsub[d]);
    }
    if (c[0] != 0 || c.back() != prob->nel[d]) return bad(plan, "cuts must span 0..nel"), TFETI_ERR_ARG;
    for (int i = 0; i < prob->nsub[d]; ++i)
      if (c[i + 1] <= c[i]) return bad(plan, "cuts must increase"), TFETI_ERR_ARG;
    plan.nsub[d] = prob->nsub[d];
    plan.h[d] = prob->length[d] / prob->nel[d];
  }
  if (!(prob->young > 0) || !(prob->poisson > 0 && prob->poisson < 0.5) || !(prob->sigma_y > 0) ||
      !(prob->hardening > 0))
    return bad(plan, "bad material (need E>0, 0<nu<0.5, sigma_y>0, H>0)"), TFETI_ERR_ARG;
  for (int f = 0; f < 6; ++f)
    if (prob->dirichlet[f] < 0 || prob->dirichlet[f] > 7) return bad(plan, "bad dirichlet mask"), TFETI_ERR_ARG;
  if (prob->traction_face < 0 || prob->traction_face > 5) return bad(plan, "bad traction face"), TFETI_ERR_ARG;
  if (prob->precond != TFETI_PRECOND_NONE && prob->precond != TFETI_PRECOND_LUMPED &&
      prob->precond != TFETI_PRECOND_DIRICHLET)
    return bad(plan, "bad preconditioner"), TFETI_ERR_ARG;
  if (prob->coarse < TFETI_COARSE_AUTO || prob->coarse > TFETI_COARSE_PLANES)
    return bad(plan, "bad coarse mode"), TFETI_ERR_ARG;

  const int nx = prob->nel[0], ny = prob->nel[1], nz = prob->nel[2];
  const int64_t nx1 = nx + 1, ny1 = ny + 1, nz1 = nz + 1;
  plan.n_nodes = nx1 * ny1 * nz1;
  plan.n_elem = (int64_t)nx * ny * nz;
  plan.n_gp = 8 * plan.n_elem;

  // ---- subdomains (x-fastest) and shape classes
  const int sx = plan.nsub[0], sy = plan.nsub[1], sz = plan.nsub[2];
  std::map<std::vector<int>, int> shape_of;
  int64_t dof_off = 0, elem_off = 0, band_off = 0;
  for (int K = 0; K < sz; ++K)
    for (int J = 0; J < sy; ++J)
      for (int I = 0; I < sx; ++I) {
        SubInfo s{};
        const int idx[3] = {I, J, K};
        for (int d = 0; d < 3; ++d) {
          s.origin[d] = plan.cuts[d][idx[d]];
          s.dims[d] = plan.cuts[d][idx[d] + 1] - s.origin[d];
          s.nn[d] = s.dims[d] + 1;
        }
        s.n_nodes = s.nn[0] * s.nn[1] * s.nn[2];
        s.n_dof = 3 * s.n_nodes;
        s.n_elem = s.dims[0] * s.dims[1] * s.dims[2];
        s.bw = 3 * (s.nn[0] * s.nn[1] + s.nn[0] + 1) + 2;   // node offset 1 + nx1 + nx1*ny1, 3 dofs
        if (s.bw > s.n_dof - 1) s.bw = s.n_dof - 1;
        s.dof_off = dof_off;
        s.elem_off = elem_off;
        s.band_off = band_off;
        dof_off += s.n_dof;
        elem_off += s.n_elem;
        band_off += (int64_t)s.n_dof * (s.bw + 1);
        std::vector<int> key = {s.dims[0], s.dims[1], s.dims[2]};
        auto it = shape_of.find(key);
        if (it == shape_of.end()) {
          ShapeInfo sh{};
          for (int d = 0; d < 3; ++d) sh.dims[d] = s.dims[d];
          sh.n_dof = s.n_dof;
          sh.bw = s.bw;
          sh.n_elem = s.n_elem;
          sh.rep_sub = (int)plan.subs.size();
          shape_of[key] = (int)plan.shapes.size();
          s.shape = (int)plan.shapes.size();
          plan.shapes.push_back(sh);
        } else {
          s.shape = it->second;
        }
        // 3-2-1 fixing dofs: node (0,0,0) xyz, node (ax,0,0) yz, node (0,ay,0) z
        const int a = 0, b = s.dims[0], c = s.nn[0] * s.dims[1];
        int fx[6] = {3 * a, 3 * a + 1, 3 * a + 2, 3 * b + 1, 3 * b + 2, 3 * c + 2};
        std::sort(fx, fx + 6);
        for (int t = 0; t < 6; ++t) s.fix[t] = fx[t];
        plan.max_bw = std::max(plan.max_bw, s.bw);
        plan.max_ndof = std::max(plan.max_ndof, s.n_dof);
        plan.subs.push_back(s);
      }
  plan.n_dof = dof_off;
  plan.band_total = band_off;
  // factor blocks: 32 rows unless two panels of 32 x bw and one local vector exceed 200 KB
  // of shared memory; the solve launch sizes its shared memory by the largest record and
  // the largest local vector of all subdomains, so the test uses the largest n
  for (auto& s : plan.subs) {
    s.nb = std::min(32, s.bw + 1);
    if ((2LL * s.nb * s.bw + plan.max_ndof) * 8 > 200 * 1024) s.nb = std::min(16, s.bw + 1);
    s.nblk = (s.n_dof + s.nb - 1) / s.nb;
    s.rec = ((s.nb * s.bw) + 3) & ~3;                  // 16-byte records in FP64 and FP32
    s.fac_size = (int64_t)s.nblk * s.rec + (int64_t)s.nblk * s.nb * s.nb;
  }
  int64_t fo = 0;
  for (auto& s : plan.subs) {
    s.fac_off = fo;
    fo += (s.fac_size + 3) & ~3LL;        // keep every record 16-byte aligned (FP64 and FP32 copies)
  }
  plan.fac_total = fo;
  int64_t tb = 0, rt = 0, tf = 0;
  for (auto& sh : plan.shapes) {
    sh.band_off = tb;
    tb += (int64_t)sh.n_dof * (sh.bw + 1);
    sh.r_off = rt;
    rt += (int64_t)sh.n_dof * 6;
    sh.fac_off = tf;
    tf += (plan.subs[sh.rep_sub].fac_size + 3) & ~3LL;
  }
  plan.template_fac_total = tf;
  plan.template_band_total = tb;
  plan.r_total = rt;
  const int ns = (int)plan.subs.size();

  // ---- copies of every global node, in subdomain order
  std::vector<int32_t> ncopy(plan.n_nodes, 0);
  auto gnode_of = [&](const SubInfo& s, int li, int lj, int lk) -> int64_t {
    return (int64_t)(s.origin[0] + li) + nx1 * ((int64_t)(s.origin[1] + lj) + ny1 * (s.origin[2] + lk));
  };
  for (const auto& s : plan.subs)
    for (int lk = 0; lk < s.nn[2]; ++lk)
      for (int lj = 0; lj < s.nn[1]; ++lj)
        for (int li = 0; li < s.nn[0]; ++li) ncopy[gnode_of(s, li, lj, lk)]++;
  std::vector<int64_t> cstart(plan.n_nodes + 1, 0);
  for (int64_t n = 0; n < plan.n_nodes; ++n) cstart[n + 1] = cstart[n] + ncopy[n];
  std::vector<int32_t> copy_sub(cstart.back()), copy_lnode(cstart.back());
  std::vector<int64_t> fillp(cstart.begin(), cstart.end() - 1);
  for (int p = 0; p < ns; ++p) {
    const auto& s = plan.subs[p];
    int ln = 0;
    for (int lk = 0; lk < s.nn[2]; ++lk)
      for (int lj = 0; lj < s.nn[1]; ++lj)
        for (int li = 0; li < s.nn[0]; ++li, ++ln) {
          int64_t g = gnode_of(s, li, lj, lk);
          copy_sub[fillp[g]] = p;
          copy_lnode[fillp[g]] = ln;
          fillp[g]++;
        }
  }
  auto node_mask = [&](int64_t g) -> int {
    int64_t i = g % nx1, j = (g / nx1) % ny1, k = g / (nx1 * ny1);
    int m = 0;
    if (i == 0) m |= prob->dirichlet[0];
    if (i == nx) m |= prob->dirichlet[1];
    if (j == 0) m |= prob->dirichlet[2];
    if (j == ny) m |= prob->dirichlet[3];
    if (k == 0) m |= prob->dirichlet[4];
    if (k == nz) m |= prob->dirichlet[5];
    return m;
  };
  auto has_rows = [&](int64_t g) { return ncopy[g] >= 2 || node_mask(g) != 0; };

  // ---- interface nodes and copy slots per subdomain (local node order)
  std::vector<std::vector<int32_t>> iface_index(ns);   // local node -> interface index or -1
  int64_t slot_off = 0;
  for (int p = 0; p < ns; ++p) {
    auto& s = plan.subs[p];
    auto& ix = iface_index[p];
    ix.assign(s.n_nodes, -1);
    int cnt = 0, ln = 0;
    for (int lk = 0; lk < s.nn[2]; ++lk)
      for (int lj = 0; lj < s.nn[1]; ++lj)
        for (int li = 0; li < s.nn[0]; ++li, ++ln)
          if (has_rows(gnode_of(s, li, lj, lk))) ix[ln] = cnt++;
    s.copy_off = slot_off;
    s.n_copy = 3 * cnt;
    slot_off += s.n_copy;
  }
  plan.n_copy = slot_off;
  plan.slot_group.assign(plan.n_copy, -1);
  plan.slot_j.assign(plan.n_copy, 0);
  plan.slot_ldof.assign(plan.n_copy, 0);
  plan.slot_sub.assign(plan.n_copy, 0);
  for (int p = 0; p < ns; ++p) {
    const auto& s = plan.subs[p];
    for (int ln = 0; ln < s.n_nodes; ++ln) {
      int ii = iface_index[p][ln];
      if (ii < 0) continue;
      for (int c = 0; c < 3; ++c) {
        int64_t sl = s.copy_off + 3 * ii + c;
        plan.slot_ldof[sl] = 3 * ln + c;
        plan.slot_sub[sl] = p;
      }
    }
  }

  // ---- groups and rows in (global node, component) order
  int64_t row = 0;
  for (int64_t g = 0; g < plan.n_nodes; ++g) {
    if (!has_rows(g)) continue;
    const int k = ncopy[g];
    if (k > 8) return bad(plan, "more than 8 copies of a node"), TFETI_ERR_ARG;
    const int mask = node_mask(g);
    for (int c = 0; c < 3; ++c) {
      Group gr{};
      gr.k = k;
      gr.dirichlet = (mask >> c) & 1;
      gr.nrows = gr.dirichlet ? k : (k >= 2 ? k - 1 : 0);
      gr.row0 = row;
      for (int j = 0; j < k; ++j) {
        const int p = copy_sub[cstart[g] + j];
        const int ln = copy_lnode[cstart[g] + j];
        gr.sub[j] = p;
        gr.slot[j] = plan.subs[p].copy_off + 3 * iface_index[p][ln] + c;
        plan.slot_group[gr.slot[j]] = (int32_t)plan.groups.size();
        plan.slot_j[gr.slot[j]] = j;
      }
      for (int r = 0; r < gr.nrows; ++r) {
        plan.row_group.push_back((int32_t)plan.groups.size());
        plan.row_r.push_back(r);
      }
      row += gr.nrows;
      plan.groups.push_back(gr);
    }
  }
  plan.n_mult = row;
  for (int64_t sl = 0; sl < plan.n_copy; ++sl)
    if (plan.slot_group[sl] < 0) return bad(plan, "internal: copy slot without group"), TFETI_ERR_ARG;

  // ---- lumped preconditioner tables (box-boundary nodes of each shape)
  {
    int64_t boff = 0, kt = 0;
    for (auto& sh : plan.shapes) {
      const int nx_ = sh.dims[0] + 1, ny_ = sh.dims[1] + 1, nz_ = sh.dims[2] + 1;
      std::vector<int32_t> ln2b(nx_ * ny_ * nz_, -1);
      sh.bnd_off = boff;
      sh.n_bnd = 0;
      for (int lk = 0; lk < nz_; ++lk)
        for (int lj = 0; lj < ny_; ++lj)
          for (int li = 0; li < nx_; ++li) {
            const bool on = li == 0 || lj == 0 || lk == 0 || li == nx_ - 1 || lj == ny_ - 1 || lk == nz_ - 1;
            if (!on) continue;
            const int ln = li + nx_ * (lj + ny_ * lk);
            ln2b[ln] = sh.n_bnd++;
            plan.shape_bln.push_back(ln);
          }
      for (int b = 0; b < sh.n_bnd; ++b) {
        const int ln = plan.shape_bln[boff + b];
        const int li = ln % nx_, lj = (ln / nx_) % ny_, lk = ln / (nx_ * ny_);
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              const int a = li + dx, bb = lj + dy, cc = lk + dz;
              int v = -1;
              if (a >= 0 && bb >= 0 && cc >= 0 && a < nx_ && bb < ny_ && cc < nz_) v = ln2b[a + nx_ * (bb + ny_ * cc)];
              plan.shape_tnbr.push_back(v);
            }
      }
      sh.kbb_off = kt;
      kt += (int64_t)sh.n_bnd * 243;
      boff += sh.n_bnd;
      sh.s_off = plan.s_total;
      plan.s_total += (9LL * sh.n_bnd * sh.n_bnd + 3) & ~3LL;
    }
    plan.kbb_template_total = kt;
    plan.slot_bnd.assign(plan.n_copy, -1);
    int64_t b2 = 0, kown = 0;
    for (int p = 0; p < ns; ++p) {
      auto& s = plan.subs[p];
      const auto& sh = plan.shapes[s.shape];
      s.b2s_off = b2;
      s.kbb_off = kown;
      kown += (int64_t)sh.n_bnd * 243;
      for (int b = 0; b < sh.n_bnd; ++b) {
        const int ln = plan.shape_bln[sh.bnd_off + b];
        const int ii = iface_index[p][ln];
        plan.sub_b2s.push_back(ii >= 0 ? (int32_t)(s.copy_off + 3 * ii) : -1);
        if (ii >= 0)
          for (int c = 0; c < 3; ++c) plan.slot_bnd[s.copy_off + 3 * ii + c] = b;
      }
      b2 += sh.n_bnd;
    }
    plan.kbb_total = kown;
    plan.sub_nbr.assign((size_t)(plan.n_copy / 3) * 28, -1);
    for (int p = 0; p < ns; ++p) {
      const auto& s = plan.subs[p];
      int ln = 0;
      for (int lk = 0; lk < s.nn[2]; ++lk)
        for (int lj = 0; lj < s.nn[1]; ++lj)
          for (int li = 0; li < s.nn[0]; ++li, ++ln) {
            const int ii = iface_index[p][ln];
            if (ii < 0) continue;
            const int64_t base = (s.copy_off / 3 + ii) * 28;
            for (int dz = -1; dz <= 1; ++dz)
              for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                  const int t = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
                  const int a = li + dx, b = lj + dy, c = lk + dz;
                  if (a < 0 || b < 0 || c < 0 || a >= s.nn[0] || b >= s.nn[1] || c >= s.nn[2]) continue;
                  const int jj = iface_index[p][a + s.nn[0] * (b + s.nn[1] * c)];
                  if (jj >= 0) plan.sub_nbr[base + t] = (int32_t)(s.copy_off + 3 * jj);
                }
          }
    }
    for (int64_t sl = 0; sl < plan.n_copy; ++sl)
      if (plan.slot_bnd[sl] < 0) return bad(plan, "internal: interface node off the box boundary"), TFETI_ERR_ARG;
  }

  // ---- coarse pairs: GG^T[p][q] (p >= q) = sum over groups with copies in p and q
  std::map<std::pair<int, int>, std::vector<std::array<int32_t, 3>>> pairs;
  for (size_t gi = 0; gi < plan.groups.size(); ++gi) {
    const auto& gr = plan.groups[gi];
    if (gr.nrows == 0) continue;
    for (int i = 0; i < gr.k; ++i)
      for (int j = 0; j <= i; ++j)   // subdomain order: sub[i] >= sub[j]
        pairs[{gr.sub[i], gr.sub[j]}].push_back({(int32_t)gi, i, j});
  }
  plan.pair_start.push_back(0);
  for (auto& kv : pairs) {
    plan.pair_p.push_back(kv.first.first);
    plan.pair_q.push_back(kv.first.second);
    for (auto& t : kv.second) {
      plan.trip_group.push_back(t[0]);
      plan.trip_i.push_back(t[1]);
      plan.trip_j.push_back(t[2]);
    }
    plan.pair_start.push_back((int64_t)plan.trip_group.size());
  }
  return TFETI_OK;
}

}  // namespace tfeti

// ---------------------------------------------------------------------------
// C ABI of the host plan
// ---------------------------------------------------------------------------
struct tfeti_plan {
  tfeti::Plan plan;
};

extern "C" int tfeti_plan_create(const tfeti_problem* prob, tfeti_plan** out) {
  if (!out) return TFETI_ERR_ARG;
  *out = nullptr;
  tfeti_plan* p = new (std::nothrow) tfeti_plan();
  if (!p) return TFETI_ERR_OOM;
  int st;
  try {
    st = tfeti::plan_build(prob, p->plan);
  } catch (const std::bad_alloc&) {
    st = TFETI_ERR_OOM;
  }
  if (st != TFETI_OK) {
    delete p;
    return st;
  }
  *out = p;
  return TFETI_OK;
}

extern "C" int tfeti_plan_destroy(tfeti_plan* plan) {
  delete plan;
  return TFETI_OK;
}

extern "C" int tfeti_plan_sizes(const tfeti_plan* plan, tfeti_sizes* out) {
  if (!plan || !out) return TFETI_ERR_ARG;
  const auto& P = plan->plan;
  out->n_sub = (int64_t)P.subs.size();
  out->n_dof = P.n_dof;
  out->n_elements = P.n_elem;
  out->n_gp = P.n_gp;
  out->n_mult = P.n_mult;
  out->n_coarse = 6 * (int64_t)P.subs.size();
  out->n_nodes = P.n_nodes;
  out->n_copy = P.n_copy;
  out->max_band = P.max_bw;
  out->device_bytes = 0;
  return TFETI_OK;
}

extern "C" int tfeti_plan_export_B(const tfeti_plan* plan, int64_t* rows, int64_t* cols, double* vals,
                                   int64_t* nnz) {
  if (!plan || !nnz) return TFETI_ERR_ARG;
  const auto& P = plan->plan;
  int64_t cnt = 0;
  for (int64_t r = 0; r < P.n_mult; ++r) {
    const auto& g = P.groups[P.row_group[r]];
    const int rr = P.row_r[r];
    for (int j = 0; j < g.k; ++j) {
      double v;
      if (g.dirichlet) v = (j == rr) ? 1.0 : 0.0;
      else v = tfeti::helmert_coef(rr + 1, j);
      if (v == 0.0) continue;
      if (rows) {
        const auto& s = P.subs[g.sub[j]];
        rows[cnt] = r;
        cols[cnt] = s.dof_off + P.slot_ldof[g.slot[j]];
        vals[cnt] = v;
      }
      ++cnt;
    }
  }
  *nnz = cnt;
  return TFETI_OK;
}

extern "C" int tfeti_plan_export_subdomains(const tfeti_plan* plan, int64_t* out) {
  if (!plan || !out) return TFETI_ERR_ARG;
  const auto& P = plan->plan;
  for (size_t p = 0; p < P.subs.size(); ++p) {
    const auto& s = P.subs[p];
    int64_t* o = out + 9 * p;
    for (int d = 0; d < 3; ++d) {
      o[d] = s.origin[d];
      o[3 + d] = s.dims[d];
    }
    o[6] = s.dof_off;
    o[7] = s.elem_off;
    o[8] = s.bw;
  }
  return TFETI_OK;
}

extern "C" int tfeti_plan_export_fixing(const tfeti_plan* plan, int32_t* out) {
  if (!plan || !out) return TFETI_ERR_ARG;
  const auto& P = plan->plan;
  for (size_t p = 0; p < P.subs.size(); ++p)
    for (int t = 0; t < 6; ++t) out[6 * p + t] = P.subs[p].fix[t];
  return TFETI_OK;
}
