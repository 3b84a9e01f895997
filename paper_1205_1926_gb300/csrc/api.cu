// C ABI of the GB300 TFETI solver: context set-up (Sec. 4.1-4.2), assembly
// (Algorithm 5), PCGP (Algorithm 3) and one semismooth-Newton time step
// (Algorithm 4).  Host code only orchestrates; every arithmetic step of the
// solver runs in the kernels of kernels_*.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include "../../include/tfeti.h"
#include "ctx.h"
#include "dev.h"
#include "plan.h"

using namespace tfeti;


namespace {

int fail(tfeti_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_check(tfeti_ctx* c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, TFETI_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return TFETI_OK;
}

template <class T>
T* dalloc(tfeti_ctx* c, size_t n) {
  void* p = nullptr;
  if (n == 0) n = 1;
  if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    throw std::bad_alloc();
  }
  c->allocs.push_back(p);
  c->bytes += n * sizeof(T);
  return static_cast<T*>(p);
}

template <class T>
T* upload(tfeti_ctx* c, const std::vector<T>& v) {
  T* d = dalloc<T>(c, v.size());
  if (!v.empty()) cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->st);
  return d;
}

void sync(tfeti_ctx* c) { cudaStreamSynchronize(c->st); }

template <class T>
void dfree(tfeti_ctx* c, T*& p, size_t n) {
  if (!p) return;
  auto it = std::find(c->allocs.begin(), c->allocs.end(), static_cast<void*>(p));
  if (it != c->allocs.end()) {
    c->allocs.erase(it);
    c->bytes -= std::max<size_t>(n, 1) * sizeof(T);
  }
  cudaFree(p);
  p = nullptr;
}

// Grow an own-record pool from old_n to new_n values, keeping the first old_n.
template <class T>
void grow_pool(tfeti_ctx* c, T*& p, long long old_n, long long new_n) {
  T* q = dalloc<T>(c, (size_t)new_n);
  if (p && old_n > 0) cudaMemcpyAsync(q, p, sizeof(T) * old_n, cudaMemcpyDeviceToDevice, c->st);
  sync(c);
  dfree(c, p, (size_t)old_n);
  p = q;
}

// Give every subdomain with plastic points (np[p] > 0) an own-record slot and take the
// slots of the others back; the pools grow (to at least twice their size, at most one
// slot per subdomain) when the free slots do not suffice.  Slots are handed out lowest
// first in subdomain order.  Throws std::bad_alloc when the device is full.
void update_slots(tfeti_ctx* c, const std::vector<int>& np) {
  const int ns = (int)np.size();
  for (int p = 0; p < ns; ++p)
    if (np[p] == 0 && c->slot_of[p] >= 0) {
      c->free_slots.push_back(c->slot_of[p]);
      c->slot_of[p] = -1;
    }
  int need = 0;
  for (int p = 0; p < ns; ++p) need += np[p] > 0 && c->slot_of[p] < 0;
  if (need > (int)c->free_slots.size()) {
    const int want = c->slot_cap + need - (int)c->free_slots.size();
    const int cap = std::min(ns, std::max(want, std::max(8, 2 * c->slot_cap)));
    // slack of one record after the last slot: whole-record bulk copies may read past it
    const long long old_n = c->slot_cap ? (long long)(c->slot_cap + 1) * c->slot_size : 0;
    const long long new_n = (long long)(cap + 1) * c->slot_size;
    grow_pool(c, c->fac_own, old_n, new_n);
    grow_pool(c, c->fac32_own, old_n, new_n);
    if (c->dirichlet) {
      grow_pool(c, c->dfac_own, old_n, new_n);
      grow_pool(c, c->dfac32_own, old_n, new_n);
    }
    for (int k = c->slot_cap; k < cap; ++k) c->free_slots.push_back(k);
    c->slot_cap = cap;
  }
  std::sort(c->free_slots.begin(), c->free_slots.end(), std::greater<int>());
  for (int p = 0; p < ns; ++p)
    if (np[p] > 0 && c->slot_of[p] < 0) {
      c->slot_of[p] = c->free_slots.back();
      c->free_slots.pop_back();
    }
}

long long own_off(const tfeti_ctx* c, int p) { return (long long)c->slot_of[p] * c->slot_size; }

// Band workspaces for factorising the subdomains of `list`: offsets (16-byte aligned)
// into band_ws, which grows (without keeping its contents) when it is too small.
std::vector<long long> band_workspace(tfeti_ctx* c, const std::vector<int>& list) {
  std::vector<long long> offs;
  long long tot = 0;
  for (int p : list) {
    offs.push_back(tot);
    tot += ((long long)c->h_subs[p].n_dof * (c->h_subs[p].bw + 1) + 3) & ~3LL;
  }
  if (tot > c->band_ws_cap) {
    sync(c);
    dfree(c, c->band_ws, (size_t)c->band_ws_cap);
    c->band_ws_cap = std::max(tot, c->band_ws_cap + c->band_ws_cap / 2);
    c->band_ws = dalloc<double>(c, (size_t)c->band_ws_cap);
  }
  return offs;
}

double dot_host(tfeti_ctx* c, const double* x, const double* y, long long n) {
  launch_dot(x, y, n, c->partial, c->sc + 8, c->st);
  c->launches += 2;
  double v = 0.0;
  cudaMemcpyAsync(&v, c->sc + 8, sizeof(double), cudaMemcpyDeviceToHost, c->st);
  sync(c);
  return v;
}

// Largest work first: CTAs start roughly in index order, so with uneven subdomains the
// long solves begin early and the short ones fill in behind them (a stable order, so
// the items, and therefore the results, do not depend on anything but the inputs).
void sort_items_by_cost(const tfeti_ctx* c, std::vector<SolveItem>& items) {
  auto cost = [c](const SolveItem& it) {
    const SubDev& S = c->h_subs[it.sub[0]];
    return (double)it.count * S.n_dof * (S.bw + 1);
  };
  std::stable_sort(items.begin(), items.end(),
                   [&cost](const SolveItem& a, const SolveItem& b) { return cost(a) > cost(b); });
}

// Solve work items: elastic subdomains of one shape share the shape's template
// factor and are grouped R to a CTA so that the items fit one wave of SMs;
// subdomains with plastic points carry their own factor, one per CTA.
void build_item_list(tfeti_ctx* c, const std::vector<int>& plastic_count, int R, std::vector<SolveItem>& items) {
  const int ns = (int)c->h_subs.size();
  items.clear();
  for (size_t sh = 0; sh < c->plan.shapes.size(); ++sh) {
    SolveItem it{};
    it.fac = c->tmpl_fac_off[sh];
    for (int p = 0; p < ns; ++p) {
      if (plastic_count[p] > 0 || c->h_subs[p].shape != (int)sh) continue;
      it.sub[it.count++] = p;
      if (it.count == R) {
        items.push_back(it);
        it.count = 0;
      }
    }
    if (it.count) items.push_back(it);
  }
  // template items first, then the subdomains with their own records (each group by cost):
  // a residual solve can start the first group while the own records are still being
  // factorised (results do not depend on the order: every item writes its own subdomains)
  std::vector<SolveItem> own;
  for (int p = 0; p < ns; ++p)
    if (plastic_count[p] > 0) {
      SolveItem it{};
      it.fac = kOwnFac | own_off(c, p);
      it.count = 1;
      it.sub[0] = p;
      own.push_back(it);
    }
  sort_items_by_cost(c, items);
  sort_items_by_cost(c, own);
  items.insert(items.end(), own.begin(), own.end());
}

// Items of the Dirichlet-preconditioner solves: elastic subdomains grouped R to a CTA
// per template class, subdomains with plastic points on their own factors.
void build_dir_item_list(tfeti_ctx* c, const std::vector<int>& plastic_count, int R, std::vector<SolveItem>& items) {
  const int ns = (int)c->h_subs.size();
  items.clear();
  for (size_t k = 0; k < c->dtmpl_off.size(); ++k) {
    SolveItem it{};
    it.fac = c->dtmpl_off[k];
    for (int p = 0; p < ns; ++p) {
      if (plastic_count[p] > 0 || c->dclass[p] != (int)k) continue;
      it.sub[it.count++] = p;
      if (it.count == R) {
        items.push_back(it);
        it.count = 0;
      }
    }
    if (it.count) items.push_back(it);
  }
  for (int p = 0; p < ns; ++p)
    if (plastic_count[p] > 0) {
      SolveItem it{};
      it.fac = kOwnFac | own_off(c, p);
      it.count = 1;
      it.sub[0] = p;
      items.push_back(it);
    }
}

void build_items(tfeti_ctx* c, const std::vector<int>& plastic_count) {
  const int ns = (int)c->h_subs.size();
  int n_pl = 0;
  for (int v : plastic_count) n_pl += v > 0;
  const int n_el = ns - n_pl;
  // FP64: one CTA per SM, so at most n_sm items; FP32: two CTAs per SM fit in shared memory
  const int slots64 = std::max(1, c->n_sm - n_pl), slots32 = std::max(1, 2 * c->n_sm - n_pl);
  const int R64 = std::max(1, std::min((n_el + slots64 - 1) / slots64, c->rcap));
  const int R32 = std::max(1, std::min((n_el + slots32 - 1) / slots32, c->rcap32));
  build_item_list(c, plastic_count, R64, c->h_items);
  build_item_list(c, plastic_count, R32, c->h_items32);
  // for the Schur-block inner F-apply: elastic subdomains per shape, FP32 items of the plastic ones
  c->h_el.clear();
  c->el_off.assign(c->plan.shapes.size(), 0);
  c->el_cnt.assign(c->plan.shapes.size(), 0);
  c->h_np = plastic_count;
  const bool have_use = c->schur_use.size() == c->plan.shapes.size();
  auto uses_schur = [&](int sh) { return have_use && c->schur_use[sh]; };
  const bool have_wood = c->h_wood.size() == (size_t)ns;
  auto wood = [&](int p) { return have_wood && c->h_wood[p] && uses_schur(c->h_subs[p].shape); };
  for (size_t sh = 0; sh < c->plan.shapes.size(); ++sh) {
    c->el_off[sh] = (int)c->h_el.size();
    if (uses_schur((int)sh))
      for (int p = 0; p < ns; ++p)
        if ((plastic_count[p] == 0 || wood(p)) && c->h_subs[p].shape == (int)sh) c->h_el.push_back(p);
    c->el_cnt[sh] = (int)c->h_el.size() - c->el_off[sh];
  }
  // banded items beside the Schur GEMMs: subdomains with plastic points (unless their inner apply
  // goes through the Schur block and a Woodbury correction) and the elastic subdomains of shapes
  // without a Schur block in use
  std::vector<SolveItem> pl, pl64;
  for (const SolveItem& it : c->h_items32)
    if (((it.fac & kOwnFac) && !wood(it.sub[0])) || !uses_schur(c->h_subs[it.sub[0]].shape)) pl.push_back(it);
  for (const SolveItem& it : c->h_items)
    if ((it.fac & kOwnFac) || !uses_schur(c->h_subs[it.sub[0]].shape)) pl64.push_back(it);
  c->n_items_pl = (int)pl.size();
  c->n_items_pl64 = (int)pl64.size();
  if (!pl64.empty())
    cudaMemcpyAsync(c->d_items_pl64, pl64.data(), sizeof(SolveItem) * pl64.size(), cudaMemcpyHostToDevice, c->st);
  if (!c->h_el.empty())
    cudaMemcpyAsync(c->d_el, c->h_el.data(), sizeof(int) * c->h_el.size(), cudaMemcpyHostToDevice, c->st);
  if (!pl.empty())
    cudaMemcpyAsync(c->d_items_pl, pl.data(), sizeof(SolveItem) * pl.size(), cudaMemcpyHostToDevice, c->st);
  c->n_items = (int)c->h_items.size();
  c->n_items32 = (int)c->h_items32.size();
  c->n_items_el = 0;
  for (const SolveItem& it : c->h_items) c->n_items_el += (it.fac & kOwnFac) ? 0 : 1;
  c->g_inner_stale = true;
  c->lump_stale = true;
  if (c->dirichlet) {
    build_dir_item_list(c, plastic_count, R64, c->h_items_d);
    build_dir_item_list(c, plastic_count, R32, c->h_items_d32);
    c->n_items_d = (int)c->h_items_d.size();
    c->n_items_d32 = (int)c->h_items_d32.size();
    cudaMemcpyAsync(c->d_items_d, c->h_items_d.data(), sizeof(SolveItem) * c->h_items_d.size(),
                    cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(c->d_items_d32, c->h_items_d32.data(), sizeof(SolveItem) * c->h_items_d32.size(),
                    cudaMemcpyHostToDevice, c->st);
  }
  cudaMemcpyAsync(c->d_items, c->h_items.data(), sizeof(SolveItem) * c->h_items.size(), cudaMemcpyHostToDevice,
                  c->st);
  cudaMemcpyAsync(c->d_items32, c->h_items32.data(), sizeof(SolveItem) * c->h_items32.size(),
                  cudaMemcpyHostToDevice, c->st);
}

SolveArgs solve_args(tfeti_ctx* c, bool fp32 = false) {
  SolveArgs a{};
  a.fac = c->fac;
  a.fac32 = c->fac32;
  a.fac_own = c->fac_own;
  a.fac32_own = c->fac32_own;
  a.fp32 = fp32 ? 1 : 0;
  a.items = fp32 ? c->d_items32 : c->d_items;
  a.n_items = fp32 ? c->n_items32 : c->n_items;
  a.err = c->d_err;
  a.rec_max = c->rec_max;
  a.npad = c->npad;
  a.rcap = fp32 ? c->rcap32 : c->rcap;
  return a;
}

// ---- dual operators ---------------------------------------------------------
void collect_events(tfeti_ctx* c);

// One FP64 subdomain-solve pass over all subdomains, bracketed by timing events
// when timing is on (every counted pass is timed: a full event pool is drained first).
// Start a timed region on the context stream (kind 0: banded F-apply, 1: Schur
// F-apply); returns the closing event or null when timing is off.
cudaEvent_t timed_begin(tfeti_ctx* c, int kind) {
  if (!c->events) return nullptr;
  if (c->ev_used + 2 > c->ev_pool.size()) {
    sync(c);
    collect_events(c);
  }
  if (c->ev_used + 2 > c->ev_pool.size()) return nullptr;
  c->ev_kind[c->ev_used / 2] = (uint8_t)kind;
  cudaEventRecord(c->ev_pool[c->ev_used++], c->st);
  return c->ev_pool[c->ev_used++];
}

// The context stream waits for a deferred refactorisation (no host wait).
void join_factorisation(tfeti_ctx* c) {
  if (!c->fac_pending) return;
  cudaStreamWaitEvent(c->st, c->ev_fac_done, 0);
  c->fac_pending = false;
}

// After the context stream has been synchronised past the join: the pivots' status and
// the factorisation time of a deferred refactorisation.
int check_factorisation(tfeti_ctx* c) {
  if (!c->fac_check_pending) return TFETI_OK;
  join_factorisation(c);
  cudaStreamSynchronize(c->st_fac);
  c->fac_check_pending = false;
  if (c->fac_timed) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->fac_e0, c->fac_e1);
    c->factor_ms += ms;
    c->fac_timed = false;
  }
  if (*c->h_err_fac) return fail(c, TFETI_ERR_NUMERIC, "non-positive pivot in a subdomain factorisation");
  return TFETI_OK;
}

void wood_correct_solve(tfeti_ctx* c, const SolveArgs& a, cudaStream_t st);
void wood_join(tfeti_ctx* c);

// FP64 Woodbury correction of a subdomain-solve pass in two halves: y = Z C^-1 Z^T v from the
// pass's inputs on st_wc, launched before the pass so that it runs beside it, and its addition
// to the pass's outputs on the context stream afterwards.  Returns whether a correction is pending.
bool wood_correct_begin(tfeti_ctx* c, const SolveArgs& a) {
  if (a.fp32 || (a.in_mode != 0 && a.in_mode != 1) || c->wood.n <= 0 || !c->wood.fp64) return false;
  if (!c->st_wc) {
    cudaStreamCreateWithFlags(&c->st_wc, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&c->ev_wc_fork, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&c->ev_wc_done, cudaEventDisableTiming);
  }
  cudaEventRecord(c->ev_wc_fork, c->st);
  cudaStreamWaitEvent(c->st_wc, c->ev_wc_fork, 0);
  if (c->wood_pending) cudaStreamWaitEvent(c->st_wc, c->ev_wood_done, 0);   // the set-up's data
  c->launches += launch_wood_corr64(c->M, c->wood, a.in_mode == 1 ? a.src : nullptr, a.lam,
                                    a.in_mode == 0 ? 1.0 : -1.0, c->st_wc);
  cudaEventRecord(c->ev_wc_done, c->st_wc);
  return true;
}

void wood_correct_end(tfeti_ctx* c, const SolveArgs& a) {
  const bool to_c = a.out_mode == 0 || a.out_mode == 3, to_d = a.out_mode == 1 || a.out_mode == 3;
  wood_join(c);
  cudaStreamWaitEvent(c->st, c->ev_wc_done, 0);
  c->launches += launch_wood_add64(c->M, c->wood, to_c ? a.cbuf : nullptr, to_d ? a.dst : nullptr, c->st);
}

void timed_sub_solve(tfeti_ctx* c, const SolveArgs& a) {
  // subdomains on their elastic factor + Woodbury correction
  const bool corr = wood_correct_begin(c, a);
  cudaEvent_t e1 = timed_begin(c, 0);
  launch_sub_solve(c->M, a, c->solve_smem, c->st);
  if (e1) cudaEventRecord(e1, c->st);
  if (corr) wood_correct_end(c, a);
  c->launches += 1;
  c->f_launches += 1;
}

void op_F(tfeti_ctx* c, const double* x, double* yv) {
  SolveArgs a = solve_args(c);
  a.lam = x;
  a.cbuf = c->cbuf;
  a.in_mode = 0;
  a.out_mode = 0;
  if (c->fapply == TFETI_FAPPLY_SCHUR && c->schur_ready) {
    // elastic subdomains: one DGEMM with the shape's FP64 dual Schur block; the ones with
    // plastic points: their banded solves, concurrently on the second stream
    if (c->n_items_pl64 > 0) {
      cudaEventRecord(c->ev_fork, c->st);
      cudaStreamWaitEvent(c->st2, c->ev_fork, 0);
      a.items = c->d_items_pl64;
      a.n_items = c->n_items_pl64;
      launch_sub_solve(c->M, a, c->solve_smem, c->st2);
      cudaEventRecord(c->ev_join, c->st2);
      c->launches += 1;
    }
    cudaEvent_t ge1 = timed_begin(c, 1);
    for (size_t sh = 0; sh < c->plan.shapes.size(); ++sh) {
      const int cnt = c->el_cnt[sh];
      if (!cnt) continue;
      const int n_bd = 3 * c->plan.shapes[sh].n_bnd;
      launch_schur_gather64(c->M, c->d_el + c->el_off[sh], cnt, n_bd, x, c->X64, c->st);
      launch_schur_dgemm_scatter(c->M, c->d_el + c->el_off[sh], cnt, n_bd, c->X64, c->S64 + c->s_off_c[sh],
                                 c->cbuf, c->st);
      c->launches += 2;
      c->g_flops += 2.0 * cnt * (double)n_bd * n_bd;
      c->g_bytes += 8.0 * ((double)n_bd * n_bd + 2.0 * cnt * n_bd);
    }
    wood_correct_solve(c, a, c->st);   // plastic subdomains on the Schur block + correction
    if (ge1) cudaEventRecord(ge1, c->st);
    c->g_launches += 1;
    if (c->n_items_pl64 > 0) cudaStreamWaitEvent(c->st, c->ev_join, 0);
  } else {
    timed_sub_solve(c, a);
  }
  launch_contract(c->M, c->cbuf, yv, c->st);
  c->launches += 1;
}

// F x with FP32 subdomain solves (inner iterations of the mixed-precision PCGP).
// With the shapes' dual Schur blocks formed, subdomains on the elastic template are
// applied as one FP32 GEMM per shape while the subdomains with plastic points run
// their FP32 banded solves concurrently on the second stream.
void op_F32(tfeti_ctx* c, const double* x, double* yv, bool contract = true) {
  SolveArgs a = solve_args(c, true);
  a.lam = x;
  a.cbuf = c->cbuf;
  a.in_mode = 0;
  a.out_mode = 0;
  if (!c->schur_ready) {
    launch_sub_solve(c->M, a, c->solve_smem32, c->st);
    c->launches += 1;
  } else {
    if (c->n_items_pl > 0) {
      cudaEventRecord(c->ev_fork, c->st);
      cudaStreamWaitEvent(c->st2, c->ev_fork, 0);
      a.items = c->d_items_pl;
      a.n_items = c->n_items_pl;
      launch_sub_solve(c->M, a, c->solve_smem32, c->st2);
      cudaEventRecord(c->ev_join, c->st2);
      c->launches += 1;
    }
    for (size_t sh = 0; sh < c->plan.shapes.size(); ++sh) {
      const int cnt = c->el_cnt[sh];
      if (!cnt) continue;
      const int n_bd = 3 * c->plan.shapes[sh].n_bnd;
      const bool bf = c->schur_bf16;
      launch_schur_gather(c->M, c->d_el + c->el_off[sh], cnt, n_bd, bf, x, c->Xhi, c->Xlo, c->st);
      const void* s_hi = bf ? static_cast<const void*>(static_cast<const unsigned char*>(c->Sbf) + 2 * c->s_tile_off[sh])
                            : static_cast<const void*>(c->Shi + c->s_tile_off[sh]);
      launch_schur_gemm_scatter(c->M, c->d_el + c->el_off[sh], cnt, n_bd, bf, schur_splits(cnt, n_bd, c->n_sm),
                                c->Xhi, c->Xlo, s_hi, c->Slo + c->s_tile_off[sh], c->s_part, c->cbuf, c->d_err, c->st);
      c->launches += 3;
    }
    if (c->wood.n > 0) {   // plastic subdomains on their shape's block: + Z_b C^-1 Z_b^T x_b
      wood_join(c);
      launch_wood_apply(c->M, c->wood, x, c->cbuf, c->st);
      c->launches += 3;
    }
    if (c->n_items_pl > 0) cudaStreamWaitEvent(c->st, c->ev_join, 0);
  }
  if (contract) {
    launch_contract(c->M, c->cbuf, yv, c->st);
    c->launches += 1;
  }
  c->f32_launches += 1;
}

// Dual Schur block S = (K^+)_{boundary,boundary} of every shape's elastic template,
// formed in FP64 by the panel solve with unit right-hand sides and stored in FP32.
int form_schur_blocks(tfeti_ctx* c) {
  const Plan& P = c->plan;
  for (size_t sh = 0; sh < P.shapes.size(); ++sh) {
    if (!c->schur_formed[sh]) continue;
    const int n_bd = 3 * P.shapes[sh].n_bnd;
    std::vector<SolveItem> items;
    for (int j = 0; j < n_bd; j += c->rcap) {
      SolveItem it{};
      it.fac = c->tmpl_fac_off[sh];
      for (int r = 0; r < c->rcap && j + r < n_bd; ++r) it.sub[it.count++] = j + r;
      items.push_back(it);
    }
    cudaMemcpyAsync(c->d_items_s, items.data(), sizeof(SolveItem) * items.size(), cudaMemcpyHostToDevice, c->st);
    SolveArgs a = solve_args(c);
    a.items = c->d_items_s;
    a.n_items = (int)items.size();
    a.in_mode = 2;
    a.out_mode = 2;
    a.rep_sub = P.shapes[sh].rep_sub;
    a.S32 = c->S32;
    a.S64 = c->S64;
    a.s_off = c->s_off_c[sh];
    launch_sub_solve(c->M, a, c->solve_smem, c->st);
    launch_schur_tile_S(c->S32 + c->s_off_c[sh], n_bd, false, c->Shi + c->s_tile_off[sh], c->Slo + c->s_tile_off[sh],
                        c->st);
    c->launches += 2;
    sync(c);
  }
  c->schur_ready = true;
  return cuda_check(c, "forming dual Schur blocks");
}

// Per-context work space of the tensor-core Schur apply: the gathered operand tiles and the
// output tiles of the K splits (each context's own: case contexts run concurrently).
void alloc_schur_work(tfeti_ctx* c, int max_bd) {
  const int ns = (int)c->h_subs.size();
  const long long x_tiles = schur_x_tile_elems(ns, max_bd);
  c->Xhi = dalloc<float>(c, (size_t)std::max(1LL, x_tiles));
  c->Xlo = dalloc<float>(c, (size_t)std::max(1LL, x_tiles));
  c->X64 = dalloc<double>(c, (size_t)ns * (size_t)std::max(1, max_bd));
  c->s_part = dalloc<float>(c, (size_t)std::max(1LL, schur_part_floats(ns, max_bd, 2)));
}

// The shapes' dual Schur blocks in FP32 (tensor-core tiles) and FP64, formed once.
int ensure_schur(tfeti_ctx* c) {
  if (c->schur_ready) return TFETI_OK;
  if (c->base) {
    // the Schur blocks depend only on the shapes' elastic templates: share the base's
    int st = ensure_schur(c->base);
    if (st != TFETI_OK) return fail(c, st, c->base->err);
    tfeti_ctx* b = c->base;
    c->schur_formed = b->schur_formed;
    c->s_off_c = b->s_off_c;
    c->s_tile_off = b->s_tile_off;
    c->S32 = b->S32;
    c->S64 = b->S64;
    c->Shi = b->Shi;
    c->Slo = b->Slo;
    int max_bd = 0;
    for (size_t sh = 0; sh < c->plan.shapes.size(); ++sh)
      if (c->schur_formed[sh]) max_bd = std::max(max_bd, 3 * c->plan.shapes[sh].n_bnd);
    try {
      alloc_schur_work(c, max_bd);
    } catch (const std::bad_alloc&) {
      return fail(c, TFETI_ERR_OOM, "device allocation failed");
    }
    c->schur_use = c->schur_formed;
    c->schur_ready = true;
    return TFETI_OK;
  }
  const size_t nsh = c->plan.shapes.size();
  std::vector<int> count(nsh, 0);
  for (const SubDev& sd : c->h_subs) ++count[sd.shape];
  c->schur_formed.assign(nsh, 0);
  c->s_off_c.assign(nsh, 0);
  try {
    int max_bd = 0;
    long long s_tiles = 0, s_tot = 0;
    c->s_tile_off.assign(nsh, 0);
    for (size_t sh = 0; sh < nsh; ++sh) {
      if (count[sh] < kSchurMinCount) continue;
      c->schur_formed[sh] = 1;
      const int n_bd = 3 * c->plan.shapes[sh].n_bnd;
      max_bd = std::max(max_bd, n_bd);
      c->s_off_c[sh] = s_tot;
      s_tot += (long long)n_bd * n_bd;
      c->s_tile_off[sh] = s_tiles;
      s_tiles += schur_s_tile_elems(n_bd);
    }
    c->S32 = dalloc<float>(c, (size_t)std::max(1LL, s_tot));
    c->S64 = dalloc<double>(c, (size_t)std::max(1LL, s_tot));
    c->Shi = dalloc<float>(c, (size_t)std::max(1LL, s_tiles));
    c->Slo = dalloc<float>(c, (size_t)std::max(1LL, s_tiles));
    alloc_schur_work(c, max_bd);
  } catch (const std::bad_alloc&) {
    return fail(c, TFETI_ERR_OOM, "device allocation failed");
  }
  c->schur_use = c->schur_formed;
  return form_schur_blocks(c);
}

// The BF16 copy of the shapes' S tiles (formed once from the FP32 blocks; a case context
// shares its base's).
int ensure_schur_bf16(tfeti_ctx* c) {
  if (c->Sbf) return TFETI_OK;
  if (c->base) {
    const int st = ensure_schur_bf16(c->base);
    if (st != TFETI_OK) return fail(c, st, c->base->err);
    c->Sbf = c->base->Sbf;
    return TFETI_OK;
  }
  long long s_tiles = 0;
  for (size_t sh = 0; sh < c->plan.shapes.size(); ++sh)
    if (c->schur_formed[sh]) s_tiles = std::max(s_tiles, c->s_tile_off[sh] + schur_s_tile_elems(3 * c->plan.shapes[sh].n_bnd));
  try {
    c->Sbf = dalloc<uint16_t>(c, (size_t)std::max(1LL, s_tiles));
  } catch (const std::bad_alloc&) {
    return fail(c, TFETI_ERR_OOM, "device allocation failed");
  }
  for (size_t sh = 0; sh < c->plan.shapes.size(); ++sh) {
    if (!c->schur_formed[sh]) continue;
    launch_schur_tile_S(c->S32 + c->s_off_c[sh], 3 * c->plan.shapes[sh].n_bnd, true,
                        static_cast<unsigned char*>(c->Sbf) + 2 * c->s_tile_off[sh], nullptr, c->st);
    c->launches += 1;
  }
  sync(c);
  return cuda_check(c, "forming BF16 Schur tiles");
}

// Dense FP64 K^+ (fixing-dof generalised inverse of the elastic template) of every shape with a
// formed dual Schur block and at most kWoodMaxN dofs, from unit right-hand sides through the FP64
// banded solve; formed once (a case context shares its base's).  Used by the Woodbury set-up.
int ensure_kinv(tfeti_ctx* c) {
  if (c->kinv) return TFETI_OK;
  if (c->base) {
    const int st = ensure_kinv(c->base);
    if (st != TFETI_OK) return fail(c, st, c->base->err);
    c->kinv = c->base->kinv;
    c->kinv_off = c->base->kinv_off;
    c->d_kinv_off = c->base->d_kinv_off;
    return TFETI_OK;
  }
  const Plan& P = c->plan;
  const size_t nsh = P.shapes.size();
  std::vector<long long> off(nsh, -1);
  long long tot = 0;
  for (size_t sh = 0; sh < nsh; ++sh) {
    const int n = (int)P.shapes[sh].n_dof;
    if (!c->schur_formed[sh] || n > kWoodMaxN) continue;
    off[sh] = tot;
    tot += (long long)n * n;
  }
  double* kinv = nullptr;
  try {
    kinv = dalloc<double>(c, (size_t)std::max(1LL, tot));
    c->d_kinv_off = upload(c, off);
  } catch (const std::bad_alloc&) {
    dfree(c, kinv, (size_t)std::max(1LL, tot));
    return fail(c, TFETI_ERR_OOM, "device allocation failed");
  }
  for (size_t sh = 0; sh < nsh; ++sh) {
    if (off[sh] < 0) continue;
    const int n = (int)P.shapes[sh].n_dof;
    std::vector<SolveItem> items;
    for (int j = 0; j < n; j += c->rcap) {
      SolveItem it{};
      it.fac = c->tmpl_fac_off[sh];
      for (int r = 0; r < c->rcap && j + r < n; ++r) it.sub[it.count++] = j + r;
      items.push_back(it);
    }
    SolveItem* d_items = nullptr;
    try {
      d_items = upload(c, items);
    } catch (const std::bad_alloc&) {
      return fail(c, TFETI_ERR_OOM, "device allocation failed");
    }
    SolveArgs a = solve_args(c);
    a.items = d_items;
    a.n_items = (int)items.size();
    a.in_mode = 5;
    a.out_mode = 4;
    a.rep_sub = P.shapes[sh].rep_sub;
    a.S64 = kinv;
    a.s_off = off[sh];
    launch_sub_solve(c->M, a, c->solve_smem, c->st);
    c->launches += 1;
    sync(c);
    dfree(c, d_items, items.size());
  }
  c->kinv = kinv;
  c->kinv_off = off;
  return cuda_check(c, "forming dense K^+ blocks");
}

// Grows a scratch pool (contents not kept) to at least `need` elements, doubling.
template <typename T>
void ensure_cap(tfeti_ctx* c, T*& p, long long& cap, long long need) {
  if (need <= cap && p) return;
  sync(c);
  dfree(c, p, (size_t)std::max(1LL, cap));
  cap = std::max(need, 2 * cap);
  p = dalloc<T>(c, (size_t)std::max(1LL, cap));
}

// Woodbury set-up of the plastic subdomains chosen in c->h_wood (after an assembly in the mixed
// mode): their plastic points, U, Z^T, C and its Cholesky factor in FP64, and the inner apply's
// FP32 Z_b^T and Y = C^-1 Z_b^T.  fp64: the FP64 solves of these subdomains will run on the
// elastic factor plus the correction (no refactorisation).  If a pivot of some C is not
// positive (not expected: C is positive definite) no subdomain keeps the correction and the
// function returns TFETI_OK with c->wood.n == 0 and h_wood cleared.
int wood_setup(tfeti_ctx* c, const std::vector<int>& np, bool fp64, bool async = false) {
  wood_join(c);   // an earlier set-up still in flight finishes before its pools are reused
  c->wood.n = 0;
  std::vector<int> list, npts;
  std::vector<long long> pt_off, c_off, z_off, d_off, zt_off;
  long long pts_tot = 0, c_tot = 0, z_tot = 0, d_tot = 0, zt_tot = 0;
  int max_pts = 0, max_bd = 0, max_n = 0, max_copy = 0;
  for (size_t p = 0; p < c->h_wood.size(); ++p) {
    if (!c->h_wood[p]) continue;
    const SubDev& S = c->h_subs[p];
    const int k = np[p], r = 6 * k, n_bd = 3 * S.n_bnd;
    list.push_back((int)p);
    npts.push_back(k);
    pt_off.push_back(pts_tot);
    c_off.push_back(c_tot);
    z_off.push_back(z_tot);
    d_off.push_back(d_tot);
    zt_off.push_back(zt_tot);
    pts_tot += k;
    c_tot += (long long)r * r;
    z_tot += (long long)r * n_bd;
    d_tot += (long long)((r + 31) / 32) * 32 * 32;
    zt_tot += (long long)r * S.n_dof;
    max_pts = std::max(max_pts, k);
    max_bd = std::max(max_bd, n_bd);
    max_n = std::max(max_n, S.n_dof);
    max_copy = std::max(max_copy, S.n_copy);
  }
  if (list.empty()) return TFETI_OK;
  const int nl = (int)list.size();
  try {
    if (!c->d_wood_list) {
      const int ns = (int)c->h_subs.size();
      c->d_wood_list = dalloc<int>(c, ns);
      c->d_wood_np = dalloc<int>(c, ns);
      c->d_wood_pt_off = dalloc<long long>(c, ns);
      c->d_wood_c_off = dalloc<long long>(c, ns);
      c->d_wood_z_off = dalloc<long long>(c, ns);
      c->d_wood_d_off = dalloc<long long>(c, ns);
      c->d_wood_zt_off = dalloc<long long>(c, ns);
      c->wood_t = dalloc<float>(c, (size_t)ns * 6 * kWoodMaxPts);
      c->wood_t64 = dalloc<double>(c, (size_t)ns * 6 * kWoodMaxPts);
    }
    ensure_cap(c, c->d_wood_pts, c->wood_pts_cap, pts_tot);
    ensure_cap(c, c->wood_dofs, c->wood_dofs_cap, 24 * pts_tot);
    ensure_cap(c, c->wood_u, c->wood_u_cap, 144 * pts_tot);
    ensure_cap(c, c->wood_zt, c->wood_zt_cap, zt_tot);
    ensure_cap(c, c->wood_c64, c->wood_c64_cap, c_tot);
    ensure_cap(c, c->wood_d64, c->wood_d64_cap, d_tot);
    ensure_cap(c, c->wood_c, c->wood_c_cap, c_tot);
    ensure_cap(c, c->wood_d, c->wood_d_cap, d_tot);
    ensure_cap(c, c->wood_z, c->wood_z_cap, z_tot);
    ensure_cap(c, c->wood_y, c->wood_y_cap, z_tot);
    if (fp64) {
      ensure_cap(c, c->wood_v, c->wood_v_cap, (long long)nl * max_n);
      ensure_cap(c, c->wood_yb, c->wood_yb_cap, (long long)nl * max_n);
    }
    cudaMemcpyAsync(c->d_wood_list, list.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(c->d_wood_np, npts.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(c->d_wood_pt_off, pt_off.data(), sizeof(long long) * nl, cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(c->d_wood_c_off, c_off.data(), sizeof(long long) * nl, cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(c->d_wood_z_off, z_off.data(), sizeof(long long) * nl, cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(c->d_wood_d_off, d_off.data(), sizeof(long long) * nl, cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(c->d_wood_zt_off, zt_off.data(), sizeof(long long) * nl, cudaMemcpyHostToDevice, c->st);
  } catch (const std::bad_alloc&) {
    return fail(c, TFETI_ERR_OOM, "device allocation failed (Woodbury pools)");
  }
  WoodArgs& w = c->wood;
  w = WoodArgs{};
  w.n = nl;
  w.max_pts = max_pts;
  w.max_bd = max_bd;
  w.max_n = max_n;
  w.max_copy = max_copy;
  w.fp64 = fp64;
  w.list = c->d_wood_list;
  w.pt_off = c->d_wood_pt_off;
  w.n_pts = c->d_wood_np;
  w.pts = c->d_wood_pts;
  w.plastic = c->plastic;
  w.pa = c->pa;
  w.pb = c->pb;
  w.pn = c->pn;
  w.kinv = c->kinv;
  w.kinv_off = c->d_kinv_off;
  w.u_pool = c->wood_u;
  w.dof_pool = c->wood_dofs;
  w.zt_off = c->d_wood_zt_off;
  w.zt_pool = c->wood_zt;
  w.c_off = c->d_wood_c_off;
  w.c_pool = c->wood_c64;
  w.c32_pool = c->wood_c;
  w.c_total = c_tot;
  w.d_off = c->d_wood_d_off;
  w.d_pool = c->wood_d64;
  w.d32_pool = c->wood_d;
  w.d_total = d_tot;
  w.z_off = c->d_wood_z_off;
  w.z_pool = c->wood_z;
  w.y_pool = c->wood_y;
  w.z_total = z_tot;
  w.tbuf = c->wood_t;
  w.vbuf = c->wood_v;
  w.tbuf64 = c->wood_t64;
  w.ybuf = c->wood_yb;
  if (async) {
    // beside the first residual solve of the Newton iteration (its template items do not need it)
    if (!c->st_wood) {
      try {
        c->d_err_wood = dalloc<int>(c, 1);
      } catch (const std::bad_alloc&) {
        return fail(c, TFETI_ERR_OOM, "device allocation failed");
      }
      if (cudaMallocHost(&c->h_err_wood, sizeof(int)) != cudaSuccess) return fail(c, TFETI_ERR_OOM, "host allocation failed");
      cudaStreamCreateWithFlags(&c->st_wood, cudaStreamNonBlocking);
      cudaEventCreateWithFlags(&c->ev_wood_fork, cudaEventDisableTiming);
      cudaEventCreateWithFlags(&c->ev_wood_done, cudaEventDisableTiming);
    }
    w.err = c->d_err_wood;
    cudaEventRecord(c->ev_wood_fork, c->st);
    cudaStreamWaitEvent(c->st_wood, c->ev_wood_fork, 0);
    cudaMemsetAsync(c->d_err_wood, 0, sizeof(int), c->st_wood);
    launch_wood_setup(c->M, w, c->st_wood);
    cudaMemcpyAsync(c->h_err_wood, c->d_err_wood, sizeof(int), cudaMemcpyDeviceToHost, c->st_wood);
    cudaEventRecord(c->ev_wood_done, c->st_wood);
    c->launches += wood_setup_launches(w);
    c->wood_pending = c->wood_check_pending = true;
    c->wood_subs += w.n;
    if (fp64) c->wood_fac_saved += w.n;
    return cuda_check(c, "Woodbury set-up");
  }
  w.err = c->d_err;
  cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st);
  launch_wood_setup(c->M, w, c->st);
  c->launches += wood_setup_launches(w);
  int herr = 0;
  cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st);
  sync(c);
  if (herr & 8) {   // keep the refactorisation and the banded solves for this assembly
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st);
    std::fill(c->h_wood.begin(), c->h_wood.end(), 0);
    c->wood.n = 0;
    c->wood_fallbacks += 1;
    return cuda_check(c, "Woodbury set-up");
  }
  c->wood_subs += w.n;
  if (fp64) c->wood_fac_saved += w.n;
  return cuda_check(c, "Woodbury set-up");
}

// After an FP64 subdomain-solve pass whose items put the Woodbury subdomains on their elastic
// factor (right-hand side src + sign B^T lam): add Z C^-1 Z^T v to dst and the slots in cbuf.
// The context stream waits for an asynchronous Woodbury set-up (no host wait).
void wood_join(tfeti_ctx* c) {
  if (!c->wood_pending) return;
  cudaStreamWaitEvent(c->st, c->ev_wood_done, 0);
  c->wood_pending = false;
}

void wood_correct64(tfeti_ctx* c, const double* src, const double* lam, double sign, double* cbuf, double* dst,
                    cudaStream_t st) {
  if (c->wood.n <= 0 || !c->wood.fp64) return;
  wood_join(c);
  c->launches += launch_wood_apply64(c->M, c->wood, src, lam, sign, cbuf, dst, st);
}

// Gives the subdomains that the last assembly put on the FP64 Woodbury correction their own
// factor records (from the element corrections kept since), so that they no longer depend on
// the inner apply's Schur block; called before the Schur blocks in use change.
int wood_materialize(tfeti_ctx* c) {
  if (c->wood.n <= 0 || !c->wood.fp64) return TFETI_OK;
  wood_join(c);
  const int fst = check_factorisation(c);
  if (fst != TFETI_OK) return fst;
  const DevMesh& M = c->M;
  const std::vector<int>& np = c->h_np_all;
  std::vector<int> list;
  std::vector<long long> offs, facs;
  try {
    update_slots(c, np);
    for (int p = 0; p < M.n_sub; ++p)
      if (c->h_wood[p]) list.push_back(p);
    offs = band_workspace(c, list);
  } catch (const std::bad_alloc&) {
    return fail(c, TFETI_ERR_OOM, "device allocation failed (own factor records)");
  }
  int max_rows = 0;
  long long len = 0;
  for (int p : list) {
    facs.push_back(own_off(c, p));
    max_rows = std::max(max_rows, c->h_subs[p].n_dof);
    len = std::max<long long>(len, c->plan.subs[p].fac_size);
  }
  cudaMemcpyAsync(c->d_list, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->d_list_off, offs.data(), sizeof(long long) * offs.size(), cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->d_list_fac, facs.data(), sizeof(long long) * facs.size(), cudaMemcpyHostToDevice, c->st);
  launch_band_fill(M, c->d_list, (int)list.size(), c->elem_np, c->dKe, c->band_ws, c->d_list_off, 0, max_rows,
                   c->plan.max_bw, c->st);
  cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st);
  launch_band_chol(M, c->d_list, (int)list.size(), c->d_list_off, c->band_ws, c->d_list_fac, c->fac_own, c->d_err,
                   c->plan.max_bw, c->n_sm, c->st);
  launch_fac_to_f32(c->fac_own, c->fac32_own, c->d_list_fac, (int)list.size(), len, c->st);
  c->launches += 3;
  c->factor_launches += 1;
  int herr = 0;
  cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st);
  sync(c);
  if (herr) return fail(c, TFETI_ERR_NUMERIC, "non-positive pivot in a subdomain factorisation");
  c->wood.fp64 = false;
  c->wood_fac_saved -= (long long)list.size();
  build_items(c, np);
  return cuda_check(c, "Woodbury subdomains refactorised");
}

// After a synchronisation of the context stream that followed wood_join: the pivots of an
// asynchronous set-up.  A failed Cholesky (not expected: C is positive definite) drops the correction
// for this assembly: its subdomains get their own factor records, and *redo = 1 tells the caller to
// repeat the residual solve it made with the correction.
int wood_check(tfeti_ctx* c, int* redo) {
  *redo = 0;
  if (!c->wood_check_pending) return TFETI_OK;
  c->wood_check_pending = false;
  if (!(*c->h_err_wood & 8)) return TFETI_OK;
  c->wood_fallbacks += 1;
  if (c->wood.fp64) {
    const int st = wood_materialize(c);
    if (st != TFETI_OK) return st;
  }
  std::fill(c->h_wood.begin(), c->h_wood.end(), 0);
  c->wood.n = 0;
  build_items(c, c->h_np_all);
  *redo = 1;
  return cuda_check(c, "Woodbury set-up");
}

// The same for the outputs of the FP64 solve pass `a` (in_mode 0 or 1; out_mode 0, 1 or 3).
void wood_correct_solve(tfeti_ctx* c, const SolveArgs& a, cudaStream_t st) {
  if (a.fp32 || (a.in_mode != 0 && a.in_mode != 1)) return;
  const bool to_c = a.out_mode == 0 || a.out_mode == 3, to_d = a.out_mode == 1 || a.out_mode == 3;
  wood_correct64(c, a.in_mode == 1 ? a.src : nullptr, a.lam, a.in_mode == 0 ? 1.0 : -1.0, to_c ? a.cbuf : nullptr,
                 to_d ? a.dst : nullptr, st);
}

void op_F32(tfeti_ctx* c, const double* x, double* yv, bool contract);

// Autotuner of the inner F-apply: a shape uses its dual Schur block (one tensor-core
// GEMM over its elastic subdomains) only if it has at least T subdomains, the others
// run FP32 banded solves.  T is picked among a few candidates by timing the FP32
// F-apply once per distinct choice (after one warm-up application each).
int tune_schur_threshold(tfeti_ctx* c) {
  {
    const int wst = wood_materialize(c);
    if (wst != TFETI_OK) return wst;
  }
  const size_t nsh = c->plan.shapes.size();
  std::vector<int> count(nsh, 0);
  for (const SubDev& sd : c->h_subs) ++count[sd.shape];
  const std::vector<int> np = c->h_np.size() == c->h_subs.size() ? c->h_np : std::vector<int>(c->h_subs.size(), 0);
  const int cands[] = {kSchurMinCount, 16, 64, 1 << 30};
  const long long m = c->M.n_mult;
  cudaMemsetAsync(c->tm, 0, sizeof(double) * m, c->st);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  c->schur_tune_ms.clear();
  float best = 0.f;
  int best_t = cands[3];
  std::vector<char> last;
  for (int t : cands) {
    std::vector<char> use(nsh, 0);
    for (size_t sh = 0; sh < nsh; ++sh) use[sh] = c->schur_formed[sh] && count[sh] >= t;
    if (use == last) {
      c->schur_tune_ms.push_back(c->schur_tune_ms.back());
      continue;
    }
    last = use;
    c->schur_use = use;
    build_items(c, np);
    op_F32(c, c->tm, c->Fp);
    cudaEventRecord(e0, c->st);
    for (int r = 0; r < 3; ++r) op_F32(c, c->tm, c->Fp);
    cudaEventRecord(e1, c->st);
    sync(c);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= 3.f;
    c->schur_tune_ms.push_back(ms);
    if (best_t == cands[3] && c->schur_tune_ms.size() == 1) best = ms, best_t = t;
    else if (ms < best) best = ms, best_t = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->schur_threshold = best_t;
  for (size_t sh = 0; sh < nsh; ++sh) c->schur_use[sh] = c->schur_formed[sh] && count[sh] >= best_t;
  build_items(c, np);
  return cuda_check(c, "tuning the inner F-apply");
}

void op_project(tfeti_ctx* c, const double* x, double* out) {
  launch_G_apply(c->M, x, nullptr, c->gx, 1.0, c->st);
  coarse_apply(c->coarse, c->gx, 1.0, c->hx, c->st);
  launch_GT_update(c->M, x, 1.0, c->hx, -1.0, out, c->st);
  c->launches += 2 + coarse_launches(c->coarse);
}

// Dirichlet preconditioner (Sec. 4.2): z = Bbar Sbar Bbar^T w with
// Sbar x_b = (K [x_b; -K_ii^-1 (K [x_b; 0])_i])_b, the K_ii solves on the masked
// factors (FP32 copies in the inner iterations of the mixed mode), K applied in FP64.
void op_precond_dirichlet(tfeti_ctx* c, const double* w, double* out, bool fp32) {
  const DevMesh& M = c->M;
  cudaMemsetAsync(c->dx_a, 0, sizeof(double) * M.n_dof, c->st);
  launch_slots_to_full(M, w, c->dx_a, c->st);                        // [x_b; 0]
  launch_apply_K(M, c->elem_np, c->dKe, c->dx_a, c->dx_b, c->st);    // v = K [x_b; 0]
  SolveArgs a = solve_args(c, fp32);
  a.fac = c->dfac;
  a.fac32 = c->dfac32;
  a.fac_own = c->dfac_own;
  a.fac32_own = c->dfac32_own;
  a.items = fp32 ? c->d_items_d32 : c->d_items_d;
  a.n_items = fp32 ? c->n_items_d32 : c->n_items_d;
  a.src = c->dx_b;
  a.bmask = c->d_bmask;
  a.no_fix = 1;
  a.dst = c->dx_c;
  a.in_mode = 4;
  a.out_mode = 1;
  launch_sub_solve(M, a, fp32 ? c->solve_smem32 : c->solve_smem, c->st);   // y = K_ii^-1 v_i, 0 on b
  launch_apply_K(M, c->elem_np, c->dKe, c->dx_c, c->dx_a, c->st);    // t = K [0; y]
  launch_slots_diff(M, c->dx_b, c->dx_a, c->cbuf, c->st);            // (v - t)_b
  launch_contract(M, c->cbuf, out, c->st);
  c->launches += 6;
}

// FP32 projector and preconditioner of the inner iterations of the mixed mode.
void op_project32(tfeti_ctx* c, const double* x, double* out) {
  launch_project32(c->M, c->coarse, x, c->gx, c->gx32, c->hx, c->hx8, out, c->st);
  c->launches += 2 + coarse_launches(c->coarse);
}

void op_precond32(tfeti_ctx* c, const double* x, double* out) {
  if (c->dirichlet) {
    op_precond_dirichlet(c, x, out, true);
  } else if (c->plan.prob.precond == TFETI_PRECOND_LUMPED) {
    launch_lumped32(c->M, x, c->kbb32, c->d_kbb_off32, c->cbuf, c->st, c->max_copy);
    launch_contract(c->M, c->cbuf, out, c->st);
    c->launches += 2;
  } else {
    cudaMemcpyAsync(out, x, sizeof(double) * c->M.n_mult, cudaMemcpyDeviceToDevice, c->st);
  }
}

void op_precond(tfeti_ctx* c, const double* x, double* out) {
  if (c->dirichlet) {
    op_precond_dirichlet(c, x, out, false);
  } else if (c->plan.prob.precond == TFETI_PRECOND_LUMPED) {
    launch_lumped(c->M, x, c->kbb, c->d_kbb_off, c->cbuf, c->st, c->max_copy);
    launch_contract(c->M, c->cbuf, out, c->st);
    c->launches += 2;
  } else {
    cudaMemcpyAsync(out, x, sizeof(double) * c->M.n_mult, cudaMemcpyDeviceToDevice, c->st);
  }
}

void collect_events(tfeti_ctx* c) {
  if (!c->events) return;
  for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev_pool[i], c->ev_pool[i + 1]) == cudaSuccess) {
      if (c->ev_kind[i / 2]) c->g_ms += ms;
      else c->f_ms += ms;
    }
  }
  c->ev_used = 0;
}

int assemble(tfeti_ctx* c, const double* du, const double* df, double* f_out, bool defer = false) {
  const DevMesh& M = c->M;
  {
    const int fst = check_factorisation(c);   // a previous deferred one must be finished
    if (fst != TFETI_OK) return fst;
  }
  launch_return_map(M, du, c->sig, c->kap, c->dsig, c->dkap, c->plastic, nullptr, c->pa, c->pb, c->pn, c->st);
  cudaMemsetAsync(c->sub_np, 0, sizeof(int) * M.n_sub, c->st);
  GPData gd{c->dsig, c->pa, c->pb, c->pn, c->plastic};
  launch_elem_correction(M, gd, c->elem_np, c->sub_np, c->dKe, c->st);
  c->launches += 2;
  std::vector<int> np(M.n_sub);
  cudaMemcpyAsync(np.data(), c->sub_np, sizeof(int) * M.n_sub, cudaMemcpyDeviceToHost, c->st);
  sync(c);
  c->h_np_all = np;
  {
    long long npl = 0;
    for (int v : np) npl += v;
    c->op_ver = npl == 0 ? 0 : ++c->ver_counter;   // the all-elastic tangent is always the same operator
  }
  // plastic subdomains on their shape's elastic factor plus a Woodbury correction, where the shape
  // keeps a dense K^+ and the subdomain has at most kWoodMaxPts plastic points: in the inner FP32
  // F-apply (through the shape's Schur block) and, with wood_mode 2, in the FP64 solves as well,
  // which leaves them out of the refactorisation
  c->h_wood.assign(M.n_sub, 0);
  c->wood.n = 0;
  const bool wood_ok = c->wood_mode > 0 && c->precision == TFETI_PRECISION_MIXED && c->schur_ready && c->kinv &&
                       c->schur_use.size() == c->plan.shapes.size();
  if (wood_ok) {
    for (int p = 0; p < M.n_sub; ++p) {
      const int sh = c->h_subs[p].shape;
      c->h_wood[p] = np[p] > 0 && np[p] <= kWoodMaxPts && c->kinv_off[sh] >= 0 && c->schur_use[sh];
    }
    const int wst = wood_setup(c, np, c->wood_mode >= 2 && !c->dirichlet, defer && !c->dirichlet);
    if (wst != TFETI_OK) return wst;
  }
  std::vector<int> npf = np;   // plastic points of the subdomains that are refactorised
  if (c->wood.n > 0 && c->wood.fp64)
    for (int p = 0; p < M.n_sub; ++p)
      if (c->h_wood[p]) npf[p] = 0;
  std::vector<int> list, klist;
  std::vector<long long> offs, facs, kbbs;
  try {
    update_slots(c, npf);
    for (int p = 0; p < M.n_sub; ++p)
      if (npf[p] > 0) list.push_back(p);
    offs = band_workspace(c, list);
  } catch (const std::bad_alloc&) {
    return fail(c, TFETI_ERR_OOM, "device allocation failed (own factor records)");
  }
  for (int p = 0; p < M.n_sub; ++p) {
    const SubDev& S = c->h_subs[p];
    if (npf[p] > 0) facs.push_back(own_off(c, p));
    if (np[p] > 0) {   // the lumped preconditioner's K_bb of every plastic subdomain
      klist.push_back(p);
      kbbs.push_back(c->own_kbb_base + c->plan.subs[p].kbb_off);
      c->h_kbb_off[p] = kbbs.back();
    } else {
      c->h_kbb_off[p] = c->plan.shapes[S.shape].kbb_off;
    }
  }
  cudaMemcpyAsync(c->d_kbb_off, c->h_kbb_off.data(), sizeof(long long) * M.n_sub, cudaMemcpyHostToDevice, c->st);
  // The inner FP32 iterations precondition the subdomains on the Woodbury path with their shape's
  // elastic K_bb: their few plastic points change K_bb only by the terms of U U^T at the box
  // boundary, and an inner preconditioner need only be symmetric positive definite (the FP64
  // residual and stopping test, and the FP64 preconditioner, keep the tangent's K_bb).  The
  // template stays in L2 where the own blocks (about 1 MB each for an 8^3 box) would stream from
  // HBM at every inner iteration.
  for (int p = 0; p < M.n_sub; ++p)
    c->h_kbb_off32[p] = (c->wood.n > 0 && c->h_wood[p]) ? c->plan.shapes[c->h_subs[p].shape].kbb_off : c->h_kbb_off[p];
  cudaMemcpyAsync(c->d_kbb_off32, c->h_kbb_off32.data(), sizeof(long long) * M.n_sub, cudaMemcpyHostToDevice, c->st);
  if (!klist.empty()) {
    cudaMemcpyAsync(c->d_klist, klist.data(), sizeof(int) * klist.size(), cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(c->d_list_kbb, kbbs.data(), sizeof(long long) * kbbs.size(), cudaMemcpyHostToDevice, c->st);
  }
  c->last_refactored.push_back((int)list.size());
  build_items(c, npf);
  if (!list.empty()) {
    cudaMemcpyAsync(c->d_list, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(c->d_list_off, offs.data(), sizeof(long long) * offs.size(), cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(c->d_list_fac, facs.data(), sizeof(long long) * facs.size(), cudaMemcpyHostToDevice, c->st);
    int max_rows = 0;
    for (int p : list) max_rows = std::max(max_rows, c->h_subs[p].n_dof);
    launch_band_fill(M, c->d_list, (int)list.size(), c->elem_np, c->dKe, c->band_ws, c->d_list_off, 0, max_rows,
                     c->plan.max_bw, c->st);
    if (defer && !c->dirichlet) {
      // factorise on st_fac; the residual solve joins before it reads an own record and
      // the host checks the pivots after its next synchronisation (check_factorisation)
      cudaEventRecord(c->ev_fac_fork, c->st);
      cudaStreamWaitEvent(c->st_fac, c->ev_fac_fork, 0);
      cudaMemsetAsync(c->d_err_fac, 0, sizeof(int), c->st_fac);
      c->fac_timed = c->events;
      if (c->fac_timed) cudaEventRecord(c->fac_e0, c->st_fac);
      launch_band_chol(M, c->d_list, (int)list.size(), c->d_list_off, c->band_ws, c->d_list_fac, c->fac_own,
                       c->d_err_fac, c->plan.max_bw, c->n_sm, c->st_fac);
      if (c->fac_timed) cudaEventRecord(c->fac_e1, c->st_fac);
      c->launches += 2;
      c->factor_launches += 1;
      if (c->precision == TFETI_PRECISION_MIXED) {
        long long len = 0;
        for (int p : list) len = std::max<long long>(len, c->plan.subs[p].fac_size);
        launch_fac_to_f32(c->fac_own, c->fac32_own, c->d_list_fac, (int)list.size(), len, c->st_fac);
        c->launches += 1;
      }
      cudaMemcpyAsync(c->h_err_fac, c->d_err_fac, sizeof(int), cudaMemcpyDeviceToHost, c->st_fac);
      cudaEventRecord(c->ev_fac_done, c->st_fac);
      c->fac_pending = c->fac_check_pending = true;
      launch_kbb_fill(M, c->d_klist, c->d_list_kbb, (int)klist.size(), c->max_bnd, c->elem_np, c->dKe, c->kbb,
                      c->kbb32, 0, c->st);
      launch_internal_force(M, c->dsig, df, c->fe, c->f_full, c->st);
      c->launches += 2 + (klist.empty() ? 0 : 1);
      if (f_out && f_out != c->f_full)
        cudaMemcpyAsync(f_out, c->f_full, sizeof(double) * M.n_dof, cudaMemcpyDeviceToDevice, c->st);
      return cuda_check(c, "assemble");
    }
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st);
    cudaEvent_t e0 = c->events ? c->fac_e0 : nullptr, e1 = c->events ? c->fac_e1 : nullptr;
    if (e0) cudaEventRecord(e0, c->st);
    launch_band_chol(M, c->d_list, (int)list.size(), c->d_list_off, c->band_ws, c->d_list_fac, c->fac_own,
                     c->d_err, c->plan.max_bw, c->n_sm, c->st);
    if (e1) cudaEventRecord(e1, c->st);
    c->launches += 2;
    c->factor_launches += 1;
    int herr = 0;
    cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    sync(c);
    if (e0) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      c->factor_ms += ms;
    }
    if (herr) return fail(c, TFETI_ERR_NUMERIC, "non-positive pivot in a subdomain factorisation");
    if (c->precision == TFETI_PRECISION_MIXED) {
      long long len = 0;
      for (int p : list) len = std::max<long long>(len, c->plan.subs[p].fac_size);
      launch_fac_to_f32(c->fac_own, c->fac32_own, c->d_list_fac, (int)list.size(), len, c->st);
      c->launches += 1;
    }
    if (c->dirichlet) {
      // K_ii factors of the plastic subdomains (same slots), on the same band workspaces
      launch_band_fill(M, c->d_list, (int)list.size(), c->elem_np, c->dKe, c->band_ws, c->d_list_off, 0, max_rows,
                       c->plan.max_bw, c->st, c->d_bmask);
      cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st);
      launch_band_chol(M, c->d_list, (int)list.size(), c->d_list_off, c->band_ws, c->d_list_fac, c->dfac_own,
                       c->d_err, c->plan.max_bw, c->n_sm, c->st);
      c->launches += 2;
      c->factor_launches += 1;
      if (c->precision == TFETI_PRECISION_MIXED) {
        long long len = 0;
        for (int p : list) len = std::max<long long>(len, c->plan.subs[p].fac_size);
        launch_fac_to_f32(c->dfac_own, c->dfac32_own, c->d_list_fac, (int)list.size(), len, c->st);
        c->launches += 1;
      }
      int derr = 0;
      cudaMemcpyAsync(&derr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st);
      sync(c);
      if (derr) return fail(c, TFETI_ERR_NUMERIC, "non-positive pivot in a Dirichlet-preconditioner factorisation");
    }
  }
  if (!klist.empty()) {
    launch_kbb_fill(M, c->d_klist, c->d_list_kbb, (int)klist.size(), c->max_bnd, c->elem_np, c->dKe, c->kbb,
                    c->kbb32, 0, c->st);
    c->launches += 1;
  }
  launch_internal_force(M, c->dsig, df, c->fe, c->f_full, c->st);
  c->launches += 2;
  if (f_out && f_out != c->f_full)
    cudaMemcpyAsync(f_out, c->f_full, sizeof(double) * M.n_dof, cudaMemcpyDeviceToDevice, c->st);
  return cuda_check(c, "assemble");
}

struct PcgOut {
  int it = 0, converged = 0, status = TFETI_OK;
  double w_norm = 0.0;
};

// The PCGP loop of Algorithm 3 on P F x = P r: x (in Ker N) and its residual r are
// updated in place; stops after the updates of the iteration whose ||w^{j-1}|| =
// ||P r^{j-1}|| <= tol_abs, or at maxit.  fp32: F-applies with FP32 subdomain solves.
PcgOut pcg_core(tfeti_ctx* c, double* x, double* r, double tol_abs, int maxit, bool fp32) {
  const long long m = c->M.n_mult;
  PcgOut o;
  for (int j = 1; j <= maxit; ++j) {
    if (fp32) {                                      // inner iterations of the mixed mode
      op_project32(c, r, c->w);
      launch_dot(c->w, c->w, m, c->partial, c->sc + 3, c->st);
      op_precond32(c, c->w, c->z);
      op_project32(c, c->z, c->y);
    } else {
      op_project(c, r, c->w);                        // w = P r
      launch_dot(c->w, c->w, m, c->partial, c->sc + 3, c->st);
      op_precond(c, c->w, c->z);                     // z = F^-1 w
      op_project(c, c->z, c->y);                     // y = P z
    }
    launch_dot(c->y, c->w, m, c->partial, c->sc + 0, c->st);
    c->launches += 4;
    cudaMemcpyAsync(c->h_sc, c->sc, sizeof(double) * 8, cudaMemcpyDeviceToHost, c->st);
    cudaEvent_t ready = nullptr;
    if (j == 1) {
      sync(c);
      if (!(c->h_sc[3] > 0.0)) {                     // ||w^0|| = 0: nothing to do
        o.w_norm = std::sqrt(std::max(0.0, c->h_sc[3]));
        o.converged = 1;
        break;
      }
    } else {
      cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
      cudaEventRecord(ready, c->st);
    }
    launch_p_update(m, c->y, c->pdir, c->sc, j == 1, c->st);   // p = y + beta p
    if (fp32) op_F32(c, c->pdir, c->Fp);
    else op_F(c, c->pdir, c->Fp);                              // F p
    launch_dot(c->pdir, c->Fp, m, c->partial, c->sc + 2, c->st);
    launch_lam_r_update(m, c->pdir, c->Fp, x, r, c->sc, c->st);
    cudaMemcpyAsync(c->sc + 1, c->sc + 0, sizeof(double), cudaMemcpyDeviceToDevice, c->st);
    c->launches += 5;
    if (ready) {
      cudaEventSynchronize(ready);
      cudaEventDestroy(ready);
    }
    o.it = j;
    const double ww = c->h_sc[3];
    if (!std::isfinite(ww) || !std::isfinite(c->h_sc[0])) {
      o.status = fail(c, TFETI_ERR_NONFINITE, "non-finite residual in PCGP");
      break;
    }
    if (c->h_sc[6] != 0.0) {
      o.status = fail(c, TFETI_ERR_BREAKDOWN, "p^T F p <= 0 in PCGP");
      break;
    }
    o.w_norm = std::sqrt(ww);
    if (o.w_norm <= tol_abs) {
      o.converged = 1;
      break;
    }
  }
  // the breakdown flag of the last iteration, read on the context stream
  cudaMemcpyAsync(c->h_sc + 6, c->sc + 6, sizeof(double), cudaMemcpyDeviceToHost, c->st);
  sync(c);
  if (o.status == TFETI_OK && c->h_sc[6] != 0.0) o.status = fail(c, TFETI_ERR_BREAKDOWN, "p^T F p <= 0 in PCGP");
  return o;
}

void destroy_inner_graph(tfeti_ctx* c) {
  if (c->g_inner_exec) cudaGraphExecDestroy(c->g_inner_exec);
  if (c->g_inner) cudaGraphDestroy(c->g_inner);
  c->g_inner_exec = nullptr;
  c->g_inner = nullptr;
}

// One PCGP iteration on x = dlt, r = rin with FP32 F-applies and device-side scalars.  The
// dot products and scalar steps ride in the kernels that produce their vectors (w, y, F p),
// and the last kernel closes the body run; inside a graph (has_h) it also sets the WHILE
// condition `h` of the enclosing node.
// Tasks of the fused inner iteration's lumped preconditioner: the subdomains that share their
// boundary blocks (the elastic ones of a shape share its template), kLumpR to a task in index
// order; a block's rows are split only when there are fewer such groups than SMs.
int build_lump_tasks(tfeti_ctx* c) {
  std::map<long long, std::vector<int>> by;
  for (size_t p = 0; p < c->h_subs.size(); ++p) by[c->h_kbb_off32[p]].push_back((int)p);
  long long n_grp = 0;
  for (const auto& kv : by) n_grp += ((long long)kv.second.size() + kLumpR - 1) / kLumpR;
  const int split = (int)std::max(1LL, std::min(8LL, c->n_sm / std::max(1LL, n_grp)));
  std::vector<LumpTask> t;
  int max_nr = 0;
  for (const auto& kv : by) {
    const std::vector<int>& v = kv.second;
    const int nr = 3 * c->h_subs[v[0]].n_bnd;
    max_nr = std::max(max_nr, nr);
    const int chunk = ((nr + split - 1) / split + 31) / 32 * 32;
    for (size_t i0 = 0; i0 < v.size(); i0 += kLumpR)
      for (int r0 = 0; r0 < nr; r0 += chunk) {
        LumpTask T{};
        T.kbb = kv.first;
        T.count = (int)std::min<size_t>(kLumpR, v.size() - i0);
        for (int k = 0; k < T.count; ++k) T.sub[k] = v[i0 + k];
        T.row0 = r0;
        T.row1 = std::min(nr, r0 + chunk);
        t.push_back(T);
      }
  }
  try {
    if ((int)t.size() > c->lump_cap) {
      sync(c);
      dfree(c, c->d_lump, (size_t)std::max(1, c->lump_cap));
      c->lump_cap = std::max((int)t.size(), 2 * c->lump_cap);
      c->d_lump = dalloc<LumpTask>(c, (size_t)c->lump_cap);
    }
  } catch (const std::bad_alloc&) {
    return fail(c, TFETI_ERR_OOM, "device allocation failed");
  }
  cudaMemcpyAsync(c->d_lump, t.data(), sizeof(LumpTask) * t.size(), cudaMemcpyHostToDevice, c->st);
  c->n_lump = (int)t.size();
  c->lump_max_nr = max_nr;
  c->lump_stale = false;
  return TFETI_OK;
}

// The fused inner iteration applies to the lumped preconditioner with the dense coarse solve and
// no deflation, outside ssn_time_step_cases runs with other contexts (two cooperative launches of
// the whole device must not run at once).
bool fused_usable(tfeti_ctx* c) {
  if (!c->fused_req || c->in_cases || c->dirichlet || c->plan.prob.precond != TFETI_PRECOND_LUMPED) return false;
  if (c->coarse.mode != kCoarseDense || !c->coarse.H32 || c->defl_req > 0) return false;
  if (c->lump_stale && build_lump_tasks(c) != TFETI_OK) return false;
  if (c->inner_grid_n < 0) {
    try {
      c->xslot = dalloc<float>(c, (size_t)std::max(1LL, c->M.n_copy));
      c->d_bar = dalloc<unsigned>(c, 2);
    } catch (const std::bad_alloc&) {
      c->inner_grid_n = 0;
      return false;
    }
    cudaMemsetAsync(c->d_bar, 0, 2 * sizeof(unsigned), c->st);
    InnerArgs a;
    a.max_nr = c->lump_max_nr;
    a.ld = h32_ld(c->coarse.l);
    c->inner_smem_b = inner_smem(a);
    c->inner_grid_n = inner_grid(c->n_sm, c->inner_smem_b);
  }
  return c->inner_grid_n > 0 && c->n_lump > 0;
}

InnerArgs inner_args(tfeti_ctx* c, int body, unsigned long long h, bool has_h) {
  InnerArgs a;
  a.M = c->M;
  a.H32 = c->coarse.H32;
  a.l = c->coarse.l;
  a.ld = h32_ld(c->coarse.l);
  a.kbb32 = c->kbb32;
  a.tasks = c->d_lump;
  a.n_tasks = c->n_lump;
  a.max_nr = c->lump_max_nr;
  a.r = c->rin;
  a.w = c->w;
  a.z = c->z;
  a.y = c->y;
  a.p = c->pdir;
  a.Fp = c->Fp;
  a.lam = c->dlt;
  a.cbuf = c->cbuf;
  a.xslot = c->xslot;
  a.gx = c->gx;
  a.hx = c->hx;
  a.hx8 = c->hx8;
  a.sc = c->sc;
  a.partial = c->partial;
  a.bar = c->d_bar;
  a.err = c->d_err;
  a.cond = h;
  a.has_cond = has_h ? 1 : 0;
  a.body = body;
  return a;
}

int launch_inner_fused(tfeti_ctx* c, int body, unsigned long long h, bool has_h) {
  const cudaError_t e = launch_inner(inner_args(c, body, h, has_h), c->inner_grid_n, c->inner_smem_b, c->st);
  c->launches += 1;
  if (e != cudaSuccess) return fail(c, TFETI_ERR_CUDA, cudaGetErrorString(e));
  return TFETI_OK;
}

// Body of the fused inner iteration: F p onto the slots, then the fused launch.
int enqueue_inner_fused_body(tfeti_ctx* c, unsigned long long h, bool has_h) {
  op_F32(c, c->pdir, c->Fp, false);   // slots of F p
  return launch_inner_fused(c, 1, h, has_h);
}

void enqueue_inner_iteration(tfeti_ctx* c, unsigned long long h, bool has_h) {
  const long long m = c->M.n_mult;
  launch_G32_coarse32(c->M, c->coarse, c->rin, c->gx, c->gx32, c->hx, c->hx8, c->st);
  launch_GT32_dot(c->M, c->rin, c->hx8, c->w, nullptr, 0, c->sc, c->partial, c->d_ctr, c->st);   // w = P r, w.w
  op_precond32(c, c->w, c->z);                                                                   // z = F^-1 w
  launch_G32_coarse32(c->M, c->coarse, c->z, c->gx, c->gx32, c->hx, c->hx8, c->st);
  launch_GT32_dot(c->M, c->z, c->hx8, c->y, c->w, 1, c->sc, c->partial, c->d_ctr + 1, c->st,   // y = P z, y.w
                  c->defl_AW, c->defl_Einv);                                                     // (and mu)
  launch_p_update_g(m, c->y, c->pdir, c->sc, c->st, c->defl_W);                               // p = y + beta p - W mu
  op_F32(c, c->pdir, c->Fp, false);                                                              // slots of F p
  launch_contract_dot(c->M, c->cbuf, c->Fp, c->pdir, c->sc, c->partial, c->d_ctr + 2, c->st);  // F p, p.Fp
  launch_lam_r_update_post(m, c->pdir, c->Fp, c->dlt, c->rin, c->sc, c->d_ctr + 3, h, has_h ? 1 : 0, c->st);
  c->launches += 6 + 2 * coarse_launches(c->coarse);
}

int build_inner_graph(tfeti_ctx* c) {
  destroy_inner_graph(c);
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return cuda_check(c, "cudaGraphCreate");
  cudaGraphConditionalHandle h;
  if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_check(c, "cudaGraphConditionalHandleCreate");
  }
  cudaGraphNodeParams params{};
  params.type = cudaGraphNodeTypeConditional;
  params.conditional.handle = h;
  params.conditional.type = cudaGraphCondTypeWhile;
  params.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &params) != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_check(c, "cudaGraphAddNode(while)");
  }
  cudaGraph_t body = params.conditional.phGraph_out[0];
  const long long before = c->launches;
  // capture on the private stream (the context's stream may be the legacy default stream)
  if (cudaStreamBeginCaptureToGraph(c->st_cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
      cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_check(c, "cudaStreamBeginCaptureToGraph");
  }
  cudaStream_t saved = c->st;
  c->st = c->st_cap;
  const bool fused = fused_usable(c);
  int fst = TFETI_OK;
  if (fused) fst = enqueue_inner_fused_body(c, (unsigned long long)h, true);
  else enqueue_inner_iteration(c, (unsigned long long)h, true);
  c->st = saved;
  cudaGraph_t captured = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->st_cap, &captured);
  if (fused && (fst != TFETI_OK || e != cudaSuccess)) {
    // the cooperative launch could not be captured: build the body from separate kernels
    cudaGetLastError();
    if (captured) cudaGraphDestroy(captured);
    cudaGraphDestroy(g);
    c->launches = before;
    c->inner_grid_n = 0;
    return build_inner_graph(c);
  }
  c->g_inner_fused = fused;
  c->g_body_kernels = (int)(c->launches - before);
  c->launches = before;
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_check(c, "cudaStreamEndCapture");
  }
  if (cudaGraphInstantiate(&c->g_inner_exec, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    c->g_inner_exec = nullptr;
    return cuda_check(c, "cudaGraphInstantiate");
  }
  c->g_inner = g;
  c->g_inner_stale = false;
  return TFETI_OK;
}

// Inner PCGP of the mixed-precision refinement on (dlt, rin), run as one graph launch.
PcgOut pcg_inner_graph(tfeti_ctx* c, double tol_abs, int maxit) {
  PcgOut o;
  const bool fused = fused_usable(c);
  if (c->g_inner_stale || !c->g_inner_exec || c->g_inner_fused != fused) {
    o.status = build_inner_graph(c);
    if (o.status != TFETI_OK) return o;
  }
  launch_pcg_init(c->sc, tol_abs * tol_abs, maxit, c->st);
  if (c->events) cudaEventRecord(c->in_e0, c->st);
  if (c->g_inner_fused) {   // the first w, z, y and p, before the loop
    o.status = launch_inner_fused(c, 0, 0ULL, false);
    if (o.status != TFETI_OK) return o;
  }
  cudaGraphLaunch(c->g_inner_exec, c->st);
  if (c->events) cudaEventRecord(c->in_e1, c->st);
  cudaMemcpyAsync(c->h_sc, c->sc, sizeof(double) * kNumScalars, cudaMemcpyDeviceToHost, c->st);
  sync(c);
  const double* h = c->h_sc;
  o.it = (int)h[kIter];
  if (c->events) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->in_e0, c->in_e1) == cudaSuccess) c->inner_ms += ms;
    c->inner_its += o.it;
    c->inner_runs += (long long)h[kBodyRuns];
  }
  c->launches += 1 + (long long)c->g_body_kernels * (long long)h[kBodyRuns];
  c->f32_launches += (long long)h[kBodyRuns];
  o.w_norm = std::sqrt(std::max(0.0, h[kLastWW]));
  o.converged = h[kStopAfter] != 0.0 ? 1 : 0;
  if (h[kStatus] == 7.0) o.status = fail(c, TFETI_ERR_BREAKDOWN, "p^T F p <= 0 in PCGP");
  if (h[kStatus] == 8.0) o.status = fail(c, TFETI_ERR_NONFINITE, "non-finite residual in PCGP");
  const int st = cuda_check(c, "inner PCGP graph");
  if (st != TFETI_OK) o.status = st;
  return o;
}

// Deflation space of the inner PCGP for the current dual solve (formed at its first inner
// solve): the network's prediction when the start formed one, then the most recent stored
// solutions, up to defl_req vectors; each projected by P_N in FP64 and scaled to unit length,
// A W = P F P W with the inner FP32 operators, and E = W^T A W inverted on the host over its
// independent columns (a Cholesky that drops columns whose pivot shows them dependent on those
// kept, at the accuracy of the FP32 products).
int deflation_setup(tfeti_ctx* c) {
  c->defl_formed = true;
  c->defl_k = 0;
  const long long m = c->M.n_mult;
  std::vector<const double*> src;
  if (c->mlp_slot_valid) src.push_back(c->rec_L + (long long)c->rec_n * m);
  for (int i = 0; i < c->rec_n && (int)src.size() < c->defl_req; ++i) {
    const int slot = ((c->rec_head - 1 - i) % c->rec_q + c->rec_q) % c->rec_q;
    src.push_back(c->rec_L + (long long)slot * m);
  }
  const int k = (int)src.size();
  double zero = 0.0;
  if (k == 0) {
    cudaMemcpyAsync(c->sc + kDeflK, &zero, sizeof(double), cudaMemcpyHostToDevice, c->st);
    sync(c);
    return cuda_check(c, "deflation set-up");
  }
  for (int j = 0; j < k; ++j) {
    double* Wj = c->defl_W + (long long)j * m;
    op_project(c, src[j], Wj);
    const double nrm = std::sqrt(std::max(0.0, dot_host(c, Wj, Wj, m)));
    launch_axpby(m, nrm > 0.0 ? 1.0 / nrm : 0.0, Wj, 0.0, nullptr, Wj, c->st);   // unit vectors
    op_F32(c, Wj, c->tm);
    op_project32(c, c->tm, c->defl_AW + (long long)j * m);
  }
  launch_rec_gram(c->defl_W, c->defl_AW, c->defl_W, k, m, c->rec_partial, c->rec_out, c->st);
  double g[kRecMax * kRecMax + kRecMax];
  cudaMemcpyAsync(g, c->rec_out, sizeof(g), cudaMemcpyDeviceToHost, c->st);
  sync(c);
  c->launches += 2;
  // E (symmetrised), its Cholesky over the kept columns, and E^-1 on them (zero elsewhere)
  std::vector<double> E(k * k), L(k * k, 0.0), Einv(kDeflMax * kDeflMax, 0.0);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) E[i * k + j] = 0.5 * (g[i * kRecMax + j] + g[j * kRecMax + i]);
  std::vector<int> kept;
  for (int j = 0; j < k; ++j) {
    std::vector<double> row(kept.size());
    double d = E[j * k + j];
    for (size_t a = 0; a < kept.size(); ++a) {
      double v = E[j * k + kept[a]];
      for (size_t b = 0; b < a; ++b) v -= row[b] * L[a * k + b];
      row[a] = v / L[a * k + a];
      d -= row[a] * row[a];
    }
    // A W comes from FP32 operators (~1e-7 relative), so a pivot below 1e-4 of its diagonal would
    // amplify rounding into the search directions: such a vector counts as dependent
    if (!(d > 1e-4 * E[j * k + j]) || !std::isfinite(d)) continue;
    const size_t a = kept.size();
    for (size_t b = 0; b < a; ++b) L[a * k + b] = row[b];
    L[a * k + a] = std::sqrt(d);
    kept.push_back(j);
  }
  const int kk = (int)kept.size();
  for (int col = 0; col < kk; ++col) {   // column col of (L L^T)^-1 by two triangular solves
    std::vector<double> y(kk, 0.0), x(kk, 0.0);
    for (int a = 0; a < kk; ++a) {
      double v = a == col ? 1.0 : 0.0;
      for (int b = 0; b < a; ++b) v -= L[a * k + b] * y[b];
      y[a] = v / L[a * k + a];
    }
    for (int a = kk - 1; a >= 0; --a) {
      double v = y[a];
      for (int b = a + 1; b < kk; ++b) v -= L[b * k + a] * x[b];
      x[a] = v / L[a * k + a];
    }
    for (int a = 0; a < kk; ++a) Einv[kept[a] * kDeflMax + kept[col]] = x[a];
  }
  cudaMemcpyAsync(c->defl_Einv, Einv.data(), sizeof(double) * Einv.size(), cudaMemcpyHostToDevice, c->st);
  const double kd = kk > 0 ? (double)k : 0.0;
  cudaMemcpyAsync(c->sc + kDeflK, &kd, sizeof(double), cudaMemcpyHostToDevice, c->st);
  sync(c);
  c->defl_k = kk > 0 ? k : 0;
  c->defl_setups += 1;
  c->defl_vectors += kk;
  return cuda_check(c, "deflation set-up");
}

// Deflated start of one inner solve on (dlt = 0, rin): dlt = W E^-1 W^T rin, rin -= A W E^-1 W^T rin.
void deflation_start(tfeti_ctx* c) {
  const long long m = c->M.n_mult;
  const int k = c->defl_k;
  launch_rec_gram(c->defl_W, c->defl_AW, c->rin, k, m, c->rec_partial, c->rec_out, c->st);
  double g[kRecMax * kRecMax + kRecMax];
  std::vector<double> Ei(kDeflMax * kDeflMax);
  cudaMemcpyAsync(g, c->rec_out, sizeof(g), cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(Ei.data(), c->defl_Einv, sizeof(double) * Ei.size(), cudaMemcpyDeviceToHost, c->st);
  sync(c);
  std::vector<double> coef(k, 0.0);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) coef[i] += Ei[i * kDeflMax + j] * g[kRecMax * kRecMax + j];
  cudaMemcpyAsync(c->rec_c, coef.data(), sizeof(double) * k, cudaMemcpyHostToDevice, c->st);
  launch_rec_combine(c->defl_W, c->rec_c, k, m, nullptr, 1.0, c->dlt, c->st);
  launch_rec_combine(c->defl_AW, c->rec_c, k, m, c->rin, -1.0, c->rin, c->st);
  c->launches += 4;
}

// The same inner PCGP launched body by body from the host (no graph): the host reads the
// device scalars after every body run; used when graphs are off, e.g. for profilers, which
// do not see into conditional graph bodies.
PcgOut pcg_inner_eager(tfeti_ctx* c, double tol_abs, int maxit) {
  PcgOut o;
  launch_pcg_init(c->sc, tol_abs * tol_abs, maxit, c->st);
  const bool fused = fused_usable(c);
  if (fused) {
    o.status = launch_inner_fused(c, 0, 0ULL, false);
    if (o.status != TFETI_OK) return o;
  }
  for (int run = 0; run < 2 * maxit + 4; ++run) {
    if (fused) {
      o.status = enqueue_inner_fused_body(c, 0ULL, false);
      if (o.status != TFETI_OK) return o;
    } else {
      enqueue_inner_iteration(c, 0ULL, false);
    }
    c->f32_launches += 1;
    cudaMemcpyAsync(c->h_sc, c->sc, sizeof(double) * kNumScalars, cudaMemcpyDeviceToHost, c->st);
    sync(c);
    if (c->h_sc[kDone] != 0.0) break;
  }
  const double* hs = c->h_sc;
  o.it = (int)hs[kIter];
  o.w_norm = std::sqrt(std::max(0.0, hs[kLastWW]));
  o.converged = hs[kStopAfter] != 0.0 ? 1 : 0;
  if (hs[kStatus] == 7.0) o.status = fail(c, TFETI_ERR_BREAKDOWN, "p^T F p <= 0 in PCGP");
  if (hs[kStatus] == 8.0) o.status = fail(c, TFETI_ERR_NONFINITE, "non-finite residual in PCGP");
  const int st = cuda_check(c, "inner PCGP");
  if (st != TFETI_OK) o.status = st;
  return o;
}

// Residual solve: vsol = K^+(f - B^T lam) per subdomain and r_out = B vsol.  By
// linearity B K^+(f - B^T lam) = d - F lam, so one subdomain-solve pass gives both
// the dual residual of Algorithm 3 and the primal part of the recovered u.
void residual_solve(tfeti_ctx* c, const double* f, const double* lam, double* r_out) {
  SolveArgs a = solve_args(c);
  a.src = f;
  a.lam = lam;
  a.cbuf = c->cbuf;
  a.dst = c->vsol;
  a.in_mode = 1;
  a.out_mode = 3;
  if (c->fac_pending && c->n_items_el < c->n_items) {
    // template items while the own records are factorised on st_fac, then the others; such a
    // split pass is not among the timed F-apply passes (its span includes the factorisation)
    SolveArgs e = a;
    e.n_items = c->n_items_el;
    launch_sub_solve(c->M, e, c->solve_smem, c->st);
    join_factorisation(c);
    SolveArgs o = a;
    o.items = a.items + c->n_items_el;
    o.n_items = c->n_items - c->n_items_el;
    launch_sub_solve(c->M, o, c->solve_smem, c->st);
    wood_correct_solve(c, a, c->st);
    c->launches += 2;
    c->f_split += 1;
  } else {
    join_factorisation(c);
    timed_sub_solve(c, a);
  }
  launch_contract(c->M, c->cbuf, r_out, c->st);
  c->launches += 1;
}

// Solve the Gram system (L^T F L) c = L^T d~ of the history start on the host:
// Cholesky of the symmetrised matrix over the stored vectors in order, skipping any
// whose pivot shows it (numerically) dependent on those kept; skipped ones get c = 0.
std::vector<double> history_coefficients(const double* g, int n) {
  std::vector<double> A(n * n), b(n), Lc(n * n, 0.0), c(n, 0.0), y(n, 0.0);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) A[i * n + j] = 0.5 * (g[i * kRecMax + j] + g[j * kRecMax + i]);
    b[i] = g[kRecMax * kRecMax + i];
  }
  std::vector<int> kept;
  for (int j = 0; j < n; ++j) {
    if (!(A[j * n + j] > 0.0)) continue;
    double piv = A[j * n + j];
    for (int t = 0; t < (int)kept.size(); ++t) {
      const int kk = kept[t];
      double v = A[j * n + kk];
      for (int u = 0; u < t; ++u) v -= Lc[j * n + kept[u]] * Lc[kk * n + kept[u]];
      v /= Lc[kk * n + kk];
      Lc[j * n + kk] = v;
      piv -= v * v;
    }
    if (piv > 1e-10 * A[j * n + j]) {
      Lc[j * n + j] = std::sqrt(piv);
      kept.push_back(j);
    } else {
      for (int t = 0; t < (int)kept.size(); ++t) Lc[j * n + kept[t]] = 0.0;
    }
  }
  for (int t = 0; t < (int)kept.size(); ++t) {
    const int j = kept[t];
    double v = b[j];
    for (int u = 0; u < t; ++u) v -= Lc[j * n + kept[u]] * y[kept[u]];
    y[j] = v / Lc[j * n + j];
  }
  for (int t = (int)kept.size() - 1; t >= 0; --t) {
    const int j = kept[t];
    double v = y[j];
    for (int u = t + 1; u < (int)kept.size(); ++u) v -= Lc[kept[u] * n + j] * c[kept[u]];
    c[j] = v / Lc[j * n + j];
  }
  return c;
}

bool mlp_index_ok(const tfeti_ctx* c) { return c->mlp_on && c->newton_idx >= 1 && c->newton_idx <= kMlpIdx; }
bool mlp_ready(const tfeti_ctx* c) { return mlp_index_ok(c) && c->mlp_seen[c->newton_idx - 1] >= 1; }
double* mlp_la_of(tfeti_ctx* c) { return c->mlp_la + (long long)(c->newton_idx - 1) * c->M.n_mult; }
double* mlp_lb_of(tfeti_ctx* c) { return c->mlp_lb + (long long)(c->newton_idx - 1) * c->M.n_mult; }
float* pf_prev_of(tfeti_ctx* c) { return c->pf_prev + (long long)(c->newton_idx - 1) * c->M.n_sub; }

// Scalars of the MLP features: 1/s, 1/s_d, rho, s, index feature, with s the RMS of
// the previous step's lambda_Ker at this Newton iteration and s_d the RMS of d~
// (||d~|| = r0).  False if s = 0.
// The context stream waits for the network's last training (no host wait).
void mlp_join(tfeti_ctx* c) {
  if (!c->mlp_pending) return;
  cudaStreamWaitEvent(c->st, c->ev_mlp_done, 0);
  c->mlp_pending = false;
}

bool mlp_scalars(tfeti_ctx* c, double r0) {
  mlp_join(c);
  const long long m = c->M.n_mult;
  const double s = std::sqrt(std::max(0.0, dot_host(c, mlp_la_of(c), mlp_la_of(c), m)) / (double)m);
  const double sd = r0 / std::sqrt((double)m);
  c->mlp_scal_valid = s > 0.0 && sd > 0.0;
  if (!c->mlp_scal_valid) return false;
  c->h_scal[0] = (float)(1.0 / s);
  c->h_scal[1] = (float)(1.0 / sd);
  c->h_scal[2] = (float)c->mlp_rho;
  c->h_scal[3] = (float)s;
  c->h_scal[4] = (float)(c->newton_idx - 1) / (float)(kMlpIdx - 1);
  cudaMemcpyAsync(c->mlp_scal, c->h_scal, sizeof(c->h_scal), cudaMemcpyHostToDevice, c->st);
  sync(c);
  return true;
}

// History start (extension of Algorithm 3): on entry r = d~ and lambda_Ker = o.
// The basis is the stored solutions and, for the first Newton solve of a load step
// with the learned start on, the projected MLP prediction (its F-product by one FP64
// F-apply) when the stored solutions alone do not meet the stopping test.  Returns 0 if not applied (state unchanged), 1
// if lambda_Ker = P(sum c_j lambda_j) was taken (r = d~ - F lambda_Ker by a residual
// solve), 3 if so with a nonzero coefficient on the MLP vector, 2 if it was tried and
// rejected because ||P r|| did not fall below ||P d~|| (state reset to d~, the
// residual-solve vector no longer matches).
int history_start(tfeti_ctx* c, const double* f, double tol_abs, double r0) {
  const long long m = c->M.n_mult;
  const int n = c->rec_n;
  c->mlp_slot_valid = false;
  op_project(c, c->r, c->w);
  const double w0 = std::sqrt(std::max(0.0, dot_host(c, c->w, c->w, m)));
  if (w0 <= tol_abs) return 0;   // the zero start already meets the stopping test
  // Galerkin coefficients over the first nb stored vectors and the projected residual
  // they predict with the stored products; pred = inf if no vector is usable
  auto galerkin = [&](int nb, std::vector<double>& coef) -> double {
    launch_rec_gram(c->rec_L, c->rec_FL, c->r, nb, m, c->rec_partial, c->rec_out, c->st);
    double g[kRecMax * kRecMax + kRecMax];
    cudaMemcpyAsync(g, c->rec_out, sizeof(g), cudaMemcpyDeviceToHost, c->st);
    sync(c);
    c->launches += 2;
    coef = history_coefficients(g, nb);
    bool any = false;
    for (double v : coef) any = any || (v != 0.0 && std::isfinite(v));
    if (!any) return HUGE_VAL;
    cudaMemcpyAsync(c->rec_c, coef.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, c->st);
    launch_rec_combine(c->rec_FL, c->rec_c, nb, m, c->r, -1.0, c->tm, c->st);   // d~ - sum c_j F lambda_j
    op_project(c, c->tm, c->z);
    c->launches += 1;
    return std::sqrt(std::max(0.0, dot_host(c, c->z, c->z, m)));
  };
  std::vector<double> coef;
  int nb = n;
  double pred = n > 0 ? galerkin(n, coef) : HUGE_VAL;
  bool with_mlp = false;
  // the MLP vector joins only where the stored solutions alone miss the stopping test
  // (there the start is refined anyway, so the mixed mode takes its product in FP32)
  c->mlp_missed = pred > tol_abs;
  // the network's own gate: a solve where its vector lowered the predicted residual by less than
  // 10 % counts against it, and after two such solves in a row at this Newton index it is consulted
  // only every fourth time (it keeps training meanwhile)
  bool consult = true;
  if (mlp_index_ok(c) && c->mlp_nogain[c->newton_idx - 1] >= 2) consult = (c->mlp_probe++ % 4) == 0;
  if (pred > tol_abs && mlp_ready(c) && !consult) ++c->mlp_skipped;
  if (pred > tol_abs && mlp_ready(c) && consult && mlp_scalars(c, r0)) {
    const double pred0 = pred;
    double* Ln = c->rec_L + (long long)n * m;   // slot n is free: rec_q solutions in rec_q + 1 slots
    double* FLn = c->rec_FL + (long long)n * m;
    launch_mlp_infer(c->M, c->mlp_w16, mlp_la_of(c), mlp_lb_of(c), c->r, c->pf_now, pf_prev_of(c), c->mlp_scal,
                     c->y, c->st);
    op_project(c, c->y, Ln);
    if (c->precision == TFETI_PRECISION_MIXED) op_F32(c, Ln, FLn);   // the solve is refined in FP64 anyway
    else op_F(c, Ln, FLn);
    c->launches += 1;
    // the Galerkin start over the larger span has the smaller F-norm error, so it is kept
    std::vector<double> coef2;
    pred = galerkin(n + 1, coef2);
    coef = coef2;
    nb = n + 1;
    with_mlp = coef2[n] != 0.0;
    c->mlp_slot_valid = true;
    c->mlp_consulted = true;
    int& ng = c->mlp_nogain[c->newton_idx - 1];
    ng = pred > 0.9 * pred0 ? ng + 1 : 0;
  }
  if (nb == 0 || !(pred < c->rec_accept * w0)) return 0;
  ++c->rec_tried;
  launch_rec_combine(c->rec_L, c->rec_c, nb, m, nullptr, 1.0, c->y, c->st);
  op_project(c, c->y, c->lamk);
  launch_axpby(m, 1.0, c->lam_im, 1.0, c->lamk, c->lam, c->st);
  c->launches += 2;
  // with every contributing solution stored under the current operator, F and K^+ B^T are linear
  // in it: r = d~ - sum_j c_j F lambda_j (formed above) and K^+ (f - B^T lambda) = K^+ (f - B^T
  // lambda_Im) - sum_j c_j w_j replace the residual solve (the stored lambda_j lie in Ker N, so the
  // projection of their combination changes it only by rounding)
  bool exact = true;
  for (int j = 0; j < nb && exact; ++j)
    if (coef[j] != 0.0) exact = j < n && c->rec_ver[j] == c->op_ver;
  double w1;
  if (exact) {
    const long long nd = c->M.n_dof;
    launch_rec_combine(c->rec_W, c->rec_c, std::min(nb, n), nd, c->vsol_im, -1.0, c->vsol, c->st);
    cudaMemcpyAsync(c->r, c->tm, sizeof(double) * m, cudaMemcpyDeviceToDevice, c->st);
    c->launches += 1;
    ++c->rec_exact;
    w1 = pred;
  } else {
    residual_solve(c, f, c->lam, c->r);   // r = d~ - F lambda_Ker
    op_project(c, c->r, c->w);
    w1 = std::sqrt(std::max(0.0, dot_host(c, c->w, c->w, m)));
  }
  if (!(w1 < w0)) {
    cudaMemsetAsync(c->lamk, 0, sizeof(double) * m, c->st);
    cudaMemcpyAsync(c->r, c->dtil, sizeof(double) * m, cudaMemcpyDeviceToDevice, c->st);
    return 2;
  }
  ++c->rec_used;
  if (with_mlp) {
    ++c->mlp_used;
    return 3;
  }
  return 1;
}

// Online training of the MLP after the first Newton solve of a load step: target
// lambda_Ker of this solve, features from the two previous steps' solutions, this
// solve's d~, the plastic fractions and rho; then the histories move on by one step.
void mlp_train(tfeti_ctx* c, double r0) {
  if (!mlp_index_ok(c)) return;
  const long long m = c->M.n_mult;
  // training only after solves that the stored solutions alone could not start well, and while the
  // gate has the network benched at this Newton index (two solves in a row where it added less than
  // 10 %) only after the solves that consulted it
  const bool benched = c->mlp_nogain[c->newton_idx - 1] >= 2 && !c->mlp_consulted;
  const bool train = !benched && c->mlp_missed && c->mlp_seen[c->newton_idx - 1] >= 1 &&
                     (c->mlp_scal_valid || mlp_scalars(c, r0));
  // the next Newton iteration overwrites d~, lambda_Ker and the plastic fractions on the context stream
  cudaMemcpyAsync(c->mlp_d, c->dtil, sizeof(double) * m, cudaMemcpyDeviceToDevice, c->st);
  cudaMemcpyAsync(c->mlp_tgt, c->lamk, sizeof(double) * m, cudaMemcpyDeviceToDevice, c->st);
  cudaMemcpyAsync(c->mlp_pf, c->pf_now, sizeof(float) * c->M.n_sub, cudaMemcpyDeviceToDevice, c->st);
  cudaMemcpyAsync(c->mlp_scal_t, c->mlp_scal, sizeof(float) * 8, cudaMemcpyDeviceToDevice, c->st);
  cudaEventRecord(c->ev_mlp_fork, c->st);
  cudaStreamWaitEvent(c->st_mlp, c->ev_mlp_fork, 0);
  if (train) {
    for (int e = 0; e < c->mlp_epochs; ++e) {
      ++c->mlp_t;
      const long long start = (104729LL * c->mlp_t + 7919LL * e) % m;
      launch_mlp_train_step(c->M, c->mlp_w, mlp_la_of(c), mlp_lb_of(c), c->mlp_d, c->mlp_pf, pf_prev_of(c),
                            c->mlp_scal_t, c->mlp_tgt, start, 7919, c->mlp_blocks, c->mlp_partial, c->mlp_w,
                            c->mlp_m1, c->mlp_m2, c->mlp_w16, c->mlp_lr, c->mlp_t, c->st_mlp);
      c->launches += 2;
    }
  }
  cudaMemcpyAsync(mlp_lb_of(c), mlp_la_of(c), sizeof(double) * m, cudaMemcpyDeviceToDevice, c->st_mlp);
  cudaMemcpyAsync(mlp_la_of(c), c->mlp_tgt, sizeof(double) * m, cudaMemcpyDeviceToDevice, c->st_mlp);
  cudaMemcpyAsync(pf_prev_of(c), c->mlp_pf, sizeof(float) * c->M.n_sub, cudaMemcpyDeviceToDevice, c->st_mlp);
  cudaEventRecord(c->ev_mlp_done, c->st_mlp);
  c->mlp_pending = true;
  c->mlp_scal_valid = false;
  ++c->mlp_seen[c->newton_idx - 1];
}

// Store the solution of the finished solve: lambda_Ker and F lambda_Ker = d~ - r.
void history_push(tfeti_ctx* c) {
  const long long m = c->M.n_mult;
  double* Lj = c->rec_L + (long long)c->rec_head * m;
  double* FLj = c->rec_FL + (long long)c->rec_head * m;
  cudaMemcpyAsync(Lj, c->lamk, sizeof(double) * m, cudaMemcpyDeviceToDevice, c->st);
  launch_axpby(m, 1.0, c->dtil, -1.0, c->r, FLj, c->st);
  // w_j = K^+ B^T lambda_Ker = K^+ (f - B^T lambda_Im) - K^+ (f - B^T lambda)
  const long long nd = c->M.n_dof;
  launch_axpby(nd, 1.0, c->vsol_im, -1.0, c->vsol, c->rec_W + (long long)c->rec_head * nd, c->st);
  c->rec_ver[c->rec_head] = c->op_ver;
  c->launches += 2;
  c->rec_head = (c->rec_head + 1) % c->rec_q;
  c->rec_n = std::min(c->rec_n + 1, c->rec_q);
}

int dual_pcg(tfeti_ctx* c, const double* f, double* u_out, double* lambda_out, const double* lambda0, double rtol,
             int maxit, tfeti_pcg_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  const DevMesh& M = c->M;
  const long long m = M.n_mult;
  const long long f_before = c->f_launches + c->f_split, f32_before = c->f32_launches;
  // e = -R^T f ; lambda_Im = N^T H e = -B R (H e)
  launch_G_apply(M, nullptr, f, c->ev, -1.0, c->st);
  coarse_apply(c->coarse, c->ev, 1.0, c->hx, c->st);
  launch_GT_update(M, nullptr, 0.0, c->hx, -1.0, c->lam_im, c->st);
  c->launches += 3;
  // d~ = d - F lambda_Im = B K^+(f - B^T lambda_Im) ; r^0 = d~
  residual_solve(c, f, c->lam_im, c->r);
  wood_join(c);   // the inner solves read the set-up's FP32 part
  double r0 = std::sqrt(std::max(0.0, dot_host(c, c->r, c->r, m)));
  {
    const int fst = check_factorisation(c);   // pivots of a deferred refactorisation
    if (fst != TFETI_OK) return fst;
    int redo = 0;
    const int wst = wood_check(c, &redo);      // pivots of an asynchronous Woodbury set-up
    if (wst != TFETI_OK) return wst;
    if (redo) {
      residual_solve(c, f, c->lam_im, c->r);
      r0 = std::sqrt(std::max(0.0, dot_host(c, c->r, c->r, m)));
    }
  }
  if (c->rec_q > 0 && c->vsol_im)
    cudaMemcpyAsync(c->vsol_im, c->vsol, sizeof(double) * M.n_dof, cudaMemcpyDeviceToDevice, c->st);
  cudaMemsetAsync(c->lamk, 0, sizeof(double) * m, c->st);
  bool v_current = true;   // vsol and r belong to lambda = lambda_Im + lambda_Ker
  int used_l0 = 0;
  const bool history = c->rec_q > 0 && m > 0;
  if (history) cudaMemcpyAsync(c->dtil, c->r, sizeof(double) * m, cudaMemcpyDeviceToDevice, c->st);
  c->mlp_missed = c->rec_n == 0;   // set by the history start when it runs
  c->mlp_consulted = false;
  c->defl_formed = false;          // the deflation space is formed again for this solve
  c->defl_k = 0;
  cudaMemsetAsync(c->sc + kDeflK, 0, sizeof(double), c->st);
  if (lambda0) {
    op_project(c, lambda0, c->lamk);
    launch_axpby(m, 1.0, c->lam_im, 1.0, c->lamk, c->lam, c->st);
    residual_solve(c, f, c->lam, c->r);      // r = d~ - F lambda_Ker
    c->launches += 1;
    used_l0 = 1;
  } else if (history && (c->rec_n > 0 || mlp_ready(c)) && r0 > 0.0) {
    const int h = history_start(c, f, rtol * r0, r0);
    if (h == 1) used_l0 = 2;
    if (h == 3) used_l0 = 3;
    if (h == 2) v_current = false;
  }
  int it = 0, converged = 0, status = TFETI_OK, outer = 0;
  double w_norm = 0.0;
  if (m > 0 && r0 > 0.0) {
    if (c->precision == TFETI_PRECISION_MIXED) {
      // FP64 iterative refinement of the dual problem: the true residual
      // r = d~ - F lambda_Ker (FP64 solves) is corrected by inner PCGP solves whose
      // F-applies are FP32; the stopping test is Algorithm 3's, on the FP64 residual.
      double wn_prev = HUGE_VAL;
      for (outer = 0; outer < 100;) {
        op_project(c, c->r, c->w);
        const double wn = std::sqrt(std::max(0.0, dot_host(c, c->w, c->w, m)));
        w_norm = wn;
        if (c->defl_k > 0 && !(wn < wn_prev)) {
          // a deflated inner solve did not reduce the FP64 residual: plain inner PCGP from here on
          c->defl_k = 0;
          c->defl_fallbacks += 1;
          cudaMemsetAsync(c->sc + kDeflK, 0, sizeof(double), c->st);
        }
        wn_prev = wn;
        if (!std::isfinite(wn)) {
          status = fail(c, TFETI_ERR_NONFINITE, "non-finite residual in PCGP");
          break;
        }
        if (wn <= rtol * r0) {
          converged = 1;
          break;
        }
        if (it >= maxit) break;
        cudaMemsetAsync(c->dlt, 0, sizeof(double) * m, c->st);
        // the inner right-hand side is P r (same correction equation: P F P delta = P r), so
        // the FP32 projections inside work relative to ||P r||, not to ||r||
        cudaMemcpyAsync(c->rin, c->w, sizeof(double) * m, cudaMemcpyDeviceToDevice, c->st);
        if (c->defl_req > 0 && history) {
          if (!c->defl_formed) {
            const int dst = deflation_setup(c);
            if (dst != TFETI_OK) {
              status = dst;
              break;
            }
          }
          if (c->defl_k > 0) deflation_start(c);
        }
        const double tol_in = std::max(c->inner_rtol * wn, 0.5 * rtol * r0);
        PcgOut in = c->use_graphs ? pcg_inner_graph(c, tol_in, std::min(maxit - it, 1000))
                                  : pcg_inner_eager(c, tol_in, std::min(maxit - it, 1000));
        it += in.it;
        ++outer;
        if (in.status != TFETI_OK) {
          status = in.status;
          v_current = false;
          break;
        }
        // the correction comes from FP32 projections: project it in FP64 so that
        // lambda_Ker stays in Ker N to FP64 accuracy
        op_project(c, c->dlt, c->tm);
        launch_axpby(m, 1.0, c->lamk, 1.0, c->tm, c->lamk, c->st);
        launch_axpby(m, 1.0, c->lam_im, 1.0, c->lamk, c->lam, c->st);
        residual_solve(c, f, c->lam, c->r);    // r = d~ - F lambda_Ker
        v_current = true;
        c->launches += 2;
      }
    } else {
      PcgOut o = pcg_core(c, c->lamk, c->r, rtol * r0, maxit, false);
      it = o.it;
      converged = o.converged;
      status = o.status;
      w_norm = o.w_norm;
      v_current = false;
    }
  } else {
    converged = 1;
  }
  // lambda = lambda_Im + lambda_Ker ; alpha = H N (d - F lambda) ; u = K^+(f - B^T lambda) + R alpha
  launch_axpby(m, 1.0, c->lam_im, 1.0, c->lamk, c->lam, c->st);
  c->launches += 1;
  if (!v_current) residual_solve(c, f, c->lam, c->r);
  if (history && r0 > 0.0 && status == TFETI_OK) {   // r is the true residual here
    if (c->mlp_on) mlp_train(c, r0);
    history_push(c);
  }
  launch_G_apply(M, c->r, nullptr, c->gx, -1.0, c->st);
  coarse_apply(c->coarse, c->gx, 1.0, c->alpha, c->st);
  c->launches += 2;
  if (u_out) {
    launch_add_R_alpha(M, c->vsol, c->alpha, u_out, (int)c->plan.max_ndof, c->st);
    c->launches += 1;
  }
  if (lambda_out) cudaMemcpyAsync(lambda_out, c->lam, sizeof(double) * m, cudaMemcpyDeviceToDevice, c->st);
  cudaMemsetAsync(c->sc + 6, 0, sizeof(double), c->st);
  int herr = 0;
  cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st);
  sync(c);
  collect_events(c);
  int cst = cuda_check(c, "tfeti_dual_pcg");
  if (cst != TFETI_OK) return cst;
  if (herr & 38) {
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st);
    if (herr & 32) cudaMemsetAsync(c->d_bar, 0, 2 * sizeof(unsigned), c->st);   // the barrier restarts at zero
    return fail(c, TFETI_ERR_TIMEOUT, (herr & 2)    ? "a factor-panel copy did not complete within its time limit"
                                      : (herr & 4) ? "a Schur-tile copy or MMA did not complete within its time limit"
                                                   : "a grid-barrier wait of the fused inner iteration gave up");
  }
  if (status == TFETI_OK && !converged) status = fail(c, TFETI_ERR_NOT_CONVERGED, "PCGP iteration limit reached");
  if (info) {
    info->iterations = it;
    info->converged = converged;
    info->used_lambda0 = used_l0;
    info->f_applies = (int)(c->f_launches + c->f_split - f_before);
    info->f32_applies = (int)(c->f32_launches - f32_before);
    info->outer_iterations = outer;
    info->r0_norm = r0;
    info->w_norm = w_norm;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return status;
}

void fill_sizes(const tfeti_ctx* c, tfeti_sizes* out) {
  const Plan& P = c->plan;
  out->n_sub = (int64_t)P.subs.size();
  out->n_dof = P.n_dof;
  out->n_elements = P.n_elem;
  out->n_gp = P.n_gp;
  out->n_mult = P.n_mult;
  out->n_coarse = 6 * (int64_t)P.subs.size();
  out->n_nodes = P.n_nodes;
  out->n_copy = P.n_copy;
  out->max_band = P.max_bw;
  out->device_bytes = (int64_t)c->bytes;
}

// Set-up of a context.  With `base` (a case context, tfeti_setup_case) the read-only
// device set-up is taken from base instead of being built: subdomain descriptors, index
// maps, R, G, the coarse inverse H, the shape templates' factors and boundary blocks and
// the Dirichlet templates; everything the case writes is its own.
int setup_impl(tfeti_ctx* c, tfeti_ctx* base = nullptr) {
  Plan& P = c->plan;
  cudaGetDevice(&c->device);
  const int ns = (int)P.subs.size();
  c->l = 6LL * ns;
  // subdomain descriptors
  c->h_subs.resize(ns);
  for (int p = 0; p < ns; ++p) {
    const SubInfo& s = P.subs[p];
    SubDev d{};
    for (int k = 0; k < 3; ++k) {
      d.origin[k] = s.origin[k];
      d.dims[k] = s.dims[k];
      d.nn[k] = s.nn[k];
    }
    d.n_dof = s.n_dof;
    d.n_elem = s.n_elem;
    d.bw = s.bw;
    d.nb = s.nb;
    d.nblk = s.nblk;
    d.rec = s.rec;
    d.shape = s.shape;
    d.n_copy = s.n_copy;
    for (int t = 0; t < 6; ++t) d.fix[t] = s.fix[t];
    d.n_bnd = P.shapes[s.shape].n_bnd;
    d.bnd_off = P.shapes[s.shape].bnd_off;
    d.b2s_off = s.b2s_off;
    d.dof_off = s.dof_off;
    d.elem_off = s.elem_off;
    d.band_off = s.band_off;
    d.copy_off = s.copy_off;
    d.r_off = P.shapes[s.shape].r_off;
    c->h_subs[p] = d;
    c->max_copy = std::max(c->max_copy, s.n_copy);
  }
  DevMesh& M = c->M;
  const tfeti_problem& pr = P.prob;
  if (base) {
    c->d_subs = base->d_subs;
    M = base->M;
    M.sigma_y = pr.sigma_y;
    M.H = pr.hardening;
  } else {
  c->d_subs = upload(c, c->h_subs);
  std::vector<GroupDev> gd(P.groups.size());
  for (size_t g = 0; g < P.groups.size(); ++g) {
    const Group& s = P.groups[g];
    GroupDev d{};
    d.row0 = (int)s.row0;
    d.k = s.k;
    d.nrows = s.nrows;
    d.dirichlet = s.dirichlet;
    for (int j = 0; j < 8; ++j) {
      d.slot[j] = j < s.k ? (int)s.slot[j] : 0;
      d.sub[j] = j < s.k ? s.sub[j] : 0;
    }
    gd[g] = d;
  }
  std::vector<int> elem_sub(P.n_elem);
  for (int p = 0; p < ns; ++p)
    for (int e = 0; e < P.subs[p].n_elem; ++e) elem_sub[P.subs[p].elem_off + e] = p;
  std::vector<double> helm(64, 0.0);
  for (int r = 1; r < 8; ++r)
    for (int j = 0; j <= r; ++j) helm[r * 8 + j] = helmert_coef(r, j);
  // B^T by copy slot (CSR): slot j of a free group takes helm[r][j] x[row0 + r - 1] for
  // r = max(j, 1) .. k - 1, of a Dirichlet group x[row0 + j] (the fused inner iteration gathers with it)
  std::vector<int> bt_ptr((size_t)P.n_copy + 1, 0), bt_row;
  std::vector<double> bt_val;
  for (const Group& g : P.groups)
    for (int j = 0; j < g.k; ++j)
      bt_ptr[(size_t)g.slot[j] + 1] = g.nrows == 0 ? 0 : (g.dirichlet ? 1 : g.k - std::max(j, 1));
  for (size_t i = 0; i < (size_t)P.n_copy; ++i) bt_ptr[i + 1] += bt_ptr[i];
  bt_row.resize((size_t)bt_ptr[(size_t)P.n_copy]);
  bt_val.resize(bt_row.size());
  for (const Group& g : P.groups)
    for (int j = 0; j < g.k; ++j) {
      int e = bt_ptr[(size_t)g.slot[j]];
      if (g.nrows == 0) continue;
      if (g.dirichlet) {
        bt_row[e] = (int)g.row0 + j;
        bt_val[e] = 1.0;
        continue;
      }
      for (int r = std::max(j, 1); r < g.k; ++r, ++e) {
        bt_row[e] = (int)g.row0 + r - 1;
        bt_val[e] = helmert_coef(r, j);
      }
    }
  M.subs = c->d_subs;
  M.n_sub = ns;
  M.groups = upload(c, gd);
  M.bt_ptr = upload(c, bt_ptr);
  M.bt_row = upload(c, bt_row);
  M.bt_val = upload(c, bt_val);
  M.slot_group = upload(c, P.slot_group);
  M.slot_j = upload(c, P.slot_j);
  M.slot_ldof = upload(c, P.slot_ldof);
  M.slot_sub = upload(c, P.slot_sub);
  M.row_group = upload(c, P.row_group);
  M.row_r = upload(c, P.row_r);
  M.shape_bln = upload(c, P.shape_bln);
  M.shape_tnbr = upload(c, P.shape_tnbr);
  M.sub_b2s = upload(c, P.sub_b2s);
  M.slot_bnd = upload(c, P.slot_bnd);
  M.sub_nbr = upload(c, P.sub_nbr);
  M.elem_sub = upload(c, elem_sub);
  M.helm = upload(c, helm);
  double* dN = dalloc<double>(c, 8 * 8 * 3);
  double* Kel = dalloc<double>(c, 576);
  double* Q = dalloc<double>(c, 8 * 576);
  double* R = dalloc<double>(c, P.r_total);
  M.dN = dN;
  M.Kel = Kel;
  M.Q = Q;
  M.R = R;
  const double lam = pr.young * pr.poisson / ((1.0 + pr.poisson) * (1.0 - 2.0 * pr.poisson));
  const double mu = pr.young / (2.0 * (1.0 + pr.poisson));
  M.lam = lam;
  M.mu = mu;
  M.sigma_y = pr.sigma_y;
  M.H = pr.hardening;
  M.wdet = P.h[0] * P.h[1] * P.h[2] / 8.0;
  for (int d = 0; d < 3; ++d) {
    M.ga[d] = 0.5 * (1.0 + 1.0 / std::sqrt(3.0)) / P.h[d];
    M.gb[d] = 0.5 * (1.0 - 1.0 / std::sqrt(3.0)) / P.h[d];
  }
  M.n_dof = P.n_dof;
  M.n_gp = P.n_gp;
  M.n_mult = P.n_mult;
  M.n_copy = P.n_copy;
  M.n_groups = (long long)gd.size();
  M.n_elem = P.n_elem;
  launch_tables(P.h, lam, mu, dN, Kel, Q, c->st);
  for (const ShapeInfo& sh : P.shapes) launch_rigid_for_shape(c->h_subs[sh.rep_sub], P.h, R + sh.r_off, c->st);
  c->launches += 1 + (long long)P.shapes.size();
  {
    // explicit G = R^T B^T: entries (row, slot, B coefficient) in subdomain order, and
    // the permutation into row order (a counting sort; subdomain order within a row)
    std::vector<long long> gp_ptr(ns + 1, 0);
    std::vector<int> gp_row, gp_slot;
    std::vector<double> gp_coef;
    for (int p = 0; p < ns; ++p) {
      gp_ptr[p] = (long long)gp_row.size();
      const SubInfo& sb = P.subs[p];
      for (long long sl = sb.copy_off; sl < sb.copy_off + sb.n_copy; ++sl) {
        const Group& g = P.groups[P.slot_group[sl]];
        const int j = P.slot_j[sl];
        if (g.nrows == 0) continue;
        if (g.dirichlet) {
          gp_row.push_back((int)(g.row0 + j));
          gp_slot.push_back((int)sl);
          gp_coef.push_back(1.0);
        } else {
          for (int r = std::max(j, 1); r < g.k; ++r) {
            gp_row.push_back((int)(g.row0 + r - 1));
            gp_slot.push_back((int)sl);
            gp_coef.push_back(helmert_coef(r, j));
          }
        }
      }
    }
    const long long ne = (long long)gp_row.size();
    gp_ptr[ns] = ne;
    std::vector<long long> gt_ptr(P.n_mult + 1, 0);
    for (long long e = 0; e < ne; ++e) ++gt_ptr[gp_row[e] + 1];
    for (long long r = 0; r < P.n_mult; ++r) gt_ptr[r + 1] += gt_ptr[r];
    std::vector<long long> fill(gt_ptr.begin(), gt_ptr.end() - 1);
    std::vector<int> gt_e(ne), gt_p(ne);
    for (long long e = 0; e < ne; ++e) {
      const long long et = fill[gp_row[e]]++;
      gt_e[et] = (int)e;
      gt_p[et] = P.slot_sub[gp_slot[e]];
    }
    M.n_gpairs = ne;
    M.gp_ptr = upload(c, gp_ptr);
    M.gp_row = upload(c, gp_row);
    M.gt_ptr = upload(c, gt_ptr);
    M.gt_p = upload(c, gt_p);
    double* Gv = dalloc<double>(c, (size_t)std::max(1LL, 6 * ne));
    double* GTv = dalloc<double>(c, (size_t)std::max(1LL, 6 * ne));
    float* Gv32 = dalloc<float>(c, (size_t)std::max(1LL, 8 * ne));
    float* GTv32 = dalloc<float>(c, (size_t)std::max(1LL, 8 * ne));
    M.Gv = Gv;
    M.GTv = GTv;
    M.Gv32 = Gv32;
    M.GTv32 = GTv32;
    int* d_slot = upload(c, gp_slot);
    double* d_coef = upload(c, gp_coef);
    int* d_gte = upload(c, gt_e);
    launch_fill_G(M, d_slot, d_coef, d_gte, Gv, Gv32, GTv, GTv32, c->st);
    c->launches += 1;
    sync(c);
  }
  }   // shared tables
  // state and iterate buffers
  c->u = dalloc<double>(c, P.n_dof);
  c->sig = dalloc<double>(c, 6 * P.n_gp);
  c->kap = dalloc<double>(c, P.n_gp);
  c->du = dalloc<double>(c, P.n_dof);
  c->df = dalloc<double>(c, P.n_dof);
  c->dsig = dalloc<double>(c, 6 * P.n_gp);
  c->fe = dalloc<double>(c, 3 * P.n_gp);
  c->dkap = dalloc<double>(c, P.n_gp);
  c->pa = dalloc<double>(c, P.n_gp);
  c->pb = dalloc<double>(c, P.n_gp);
  c->pn = dalloc<double>(c, 6 * P.n_gp);
  c->plastic = dalloc<uint8_t>(c, P.n_gp);
  c->elem_np = dalloc<int>(c, P.n_elem);
  c->sub_np = dalloc<int>(c, ns);
  c->dKe = dalloc<double>(c, (size_t)P.n_elem * kTri24);
  long long max_fac = 0;
  for (const SubInfo& s : P.subs) max_fac = std::max<long long>(max_fac, s.fac_size);
  c->slot_size = (max_fac + 3) & ~3LL;
  c->slot_of.assign(ns, -1);
  if (base) {
    c->band = base->band;
    c->fac = base->fac;
    c->fac32 = base->fac32;
  } else {
    c->band = dalloc<double>(c, P.template_band_total);
    c->fac = dalloc<double>(c, P.template_fac_total + max_fac);   // slack for whole-record copies
    c->fac32 = dalloc<float>(c, P.template_fac_total + max_fac);
  }
  c->d_items = dalloc<SolveItem>(c, ns);
  c->d_items32 = dalloc<SolveItem>(c, ns);
  c->d_items_pl = dalloc<SolveItem>(c, ns);
  c->d_items_pl64 = dalloc<SolveItem>(c, ns);
  c->d_el = dalloc<int>(c, ns);
  {
    int max_bd = 0;
    for (const ShapeInfo& sh : P.shapes) max_bd = std::max(max_bd, 3 * sh.n_bnd);
    c->d_items_s = dalloc<SolveItem>(c, max_bd);
  }
  c->d_list = dalloc<int>(c, ns);
  c->d_list_off = dalloc<long long>(c, ns);
  c->d_list_fac = dalloc<long long>(c, ns);
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, dev);
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    for (const SubInfo& s : P.subs) c->rec_max = std::max(c->rec_max, s.rec);
    c->npad = (P.max_ndof + 1) & ~1;
    const long long room = (long long)max_smem - 1024 - 16LL * c->rec_max;   // static smem and barriers
    c->rcap = (int)std::min<long long>(kMaxRHS, room / (8LL * c->npad));
    if (c->rcap < 1) return fail(c, TFETI_ERR_ARG, "subdomain too large for the shared-memory solve");
    c->solve_smem = sub_solve_smem(c->rec_max, c->npad, c->rcap, 8);
    const long long room32 = (long long)max_smem - 1024 - 8LL * c->rec_max;
    c->rcap32 = (int)std::min<long long>(kMaxRHS, room32 / (4LL * c->npad));
    if (c->rcap32 < 1) c->rcap32 = 1;
    c->solve_smem32 = sub_solve_smem(c->rec_max, c->npad, c->rcap32, 4);
  }
  c->kbb = dalloc<double>(c, P.kbb_template_total + P.kbb_total);
  c->own_kbb_base = P.kbb_template_total;
  if (base)
    cudaMemcpyAsync(c->kbb, base->kbb, sizeof(double) * P.kbb_template_total, cudaMemcpyDeviceToDevice, c->st);
  c->d_kbb_off = dalloc<long long>(c, ns);
  c->h_kbb_off.assign(ns, 0);
  c->d_kbb_off32 = dalloc<long long>(c, ns);
  c->h_kbb_off32.assign(ns, 0);
  c->d_list_kbb = dalloc<long long>(c, ns);
  c->d_klist = dalloc<int>(c, ns);
  for (const ShapeInfo& sh : P.shapes) c->max_bnd = std::max(c->max_bnd, sh.n_bnd);
  c->cbuf = dalloc<double>(c, P.n_copy);
  const size_t m = (size_t)P.n_mult;
  for (double** v : {&c->lam, &c->lam_im, &c->lamk, &c->r, &c->w, &c->z, &c->y, &c->pdir, &c->Fp, &c->tm, &c->dlt,
                     &c->rin})
    *v = dalloc<double>(c, m);
  c->vsol = dalloc<double>(c, (size_t)P.n_dof);
  c->gx = dalloc<double>(c, c->l);
  c->hx = dalloc<double>(c, c->l);
  c->hx8 = dalloc<float>(c, 8 * (size_t)ns);
  c->gx32 = dalloc<float>(c, (size_t)std::max(1LL, c->l));
  cudaMemsetAsync(c->hx8, 0, sizeof(float) * 8 * (size_t)ns, c->st);
  c->ev = dalloc<double>(c, c->l);
  c->alpha = dalloc<double>(c, c->l);
  c->f_full = dalloc<double>(c, P.n_dof);
  c->tn = dalloc<double>(c, P.n_dof);
  c->tn2 = dalloc<double>(c, P.n_dof);
  c->partial = dalloc<double>(c, std::max(2 * kRedBlocks, (1 + kDeflMax) * kFusedBlocks));   // dot2, fused kernels
  c->d_ctr = dalloc<int>(c, 4);                                              // arrival counters of the fused kernels
  cudaMemsetAsync(c->d_ctr, 0, sizeof(int) * 4, c->st);
  c->sc = dalloc<double>(c, kNumScalars);
  c->d_err = dalloc<int>(c, 1);
  if (cudaMallocHost(&c->h_sc, kNumScalars * sizeof(double)) != cudaSuccess) throw std::bad_alloc();
  cudaMemsetAsync(c->u, 0, sizeof(double) * P.n_dof, c->st);
  cudaMemsetAsync(c->sig, 0, sizeof(double) * 6 * P.n_gp, c->st);
  cudaMemsetAsync(c->kap, 0, sizeof(double) * P.n_gp, c->st);
  cudaMemsetAsync(c->elem_np, 0, sizeof(int) * P.n_elem, c->st);
  cudaMemsetAsync(c->sc, 0, sizeof(double) * kNumScalars, c->st);
  // coarse problem: G G^T assembled once and factorised (G depends only on B and R)
  if (base) {
    c->H = base->H;
    c->cW = base->cW;
    c->cV = base->cV;
    c->cU = base->cU;
    c->coarse = base->coarse;
  } else {
    const int per_plane = (int)(P.nsub[0] * P.nsub[1]);
    const int n_planes = (int)P.nsub[2];
    const int mode = P.prob.coarse == TFETI_COARSE_DENSE ? kCoarseDense
                     : P.prob.coarse == TFETI_COARSE_PLANES ? kCoarsePlanes
                     : (c->l > kCoarseDenseMax ? kCoarsePlanes : kCoarseDense);
    int* pp = upload(c, P.pair_p);
    int* pq = upload(c, P.pair_q);
    long long* ps = upload(c, std::vector<long long>(P.pair_start.begin(), P.pair_start.end()));
    int* tg = upload(c, P.trip_group);
    int* ti = upload(c, P.trip_i);
    int* tj = upload(c, P.trip_j);
    double* work = nullptr;
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st);
    c->coarse = CoarseOp{};
    c->coarse.mode = mode;
    c->coarse.l = c->l;
    if (mode == kCoarseDense) {
      c->H = dalloc<double>(c, (size_t)c->l * c->l);
      launch_coarse_assemble(M, pp, pq, ps, tg, ti, tj, (long long)P.pair_p.size(), c->H, c->l, c->st);
      if (cudaMalloc(&work, sizeof(double) * dense_inverse_work(c->l)) != cudaSuccess) {
        cudaGetLastError();
        throw std::bad_alloc();
      }
      dense_cholesky_inverse(c->H, work, c->l, c->d_err, c->st);
      c->coarse.H = c->H;
    } else {
      const int n_pl = 6 * per_plane;
      const size_t blk = (size_t)n_pl * n_pl;
      c->cW = dalloc<double>(c, blk * n_planes);
      c->cAoff = dalloc<double>(c, blk * n_planes);
      c->cV = dalloc<double>(c, blk * n_planes);
      c->cU = dalloc<double>(c, blk * n_planes);
      launch_coarse_assemble_planes(M, pp, pq, ps, tg, ti, tj, (long long)P.pair_p.size(), c->cW, c->cAoff, per_plane,
                                    n_pl, n_planes, c->st);
      if (cudaMalloc(&work, sizeof(double) * (dense_inverse_work(n_pl) + blk)) != cudaSuccess) {
        cudaGetLastError();
        throw std::bad_alloc();
      }
      coarse_planes_factor(c->cW, c->cAoff, c->cV, c->cU, n_pl, n_planes, work + dense_inverse_work(n_pl), work,
                           c->d_err, c->st);
      c->coarse.n_pl = n_pl;
      c->coarse.n_planes = n_planes;
      c->coarse.W = c->cW;
      c->coarse.V = c->cV;
      c->coarse.U = c->cU;
    }
    int herr = 0;
    cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    sync(c);
    cudaFree(work);
    if (herr) return fail(c, TFETI_ERR_SINGULAR, "coarse matrix G G^T is not positive definite");
  }
  // Dirichlet preconditioner: constrained-dof mask, template classes, factor pools
  if (P.prob.precond == TFETI_PRECOND_DIRICHLET && base) {
    c->dirichlet = true;
    c->d_bmask = base->d_bmask;
    c->dclass = base->dclass;
    c->dclass_rep = base->dclass_rep;
    c->dtmpl_off = base->dtmpl_off;
    c->dfac = base->dfac;
    c->dfac32 = base->dfac32;
    c->d_items_d = dalloc<SolveItem>(c, ns);
    c->d_items_d32 = dalloc<SolveItem>(c, ns);
    c->dx_a = dalloc<double>(c, P.n_dof);
    c->dx_b = dalloc<double>(c, P.n_dof);
    c->dx_c = dalloc<double>(c, P.n_dof);
  } else if (P.prob.precond == TFETI_PRECOND_DIRICHLET) {
    c->dirichlet = true;
    std::vector<uint8_t> mask(P.n_dof, 0);
    for (long long sl = 0; sl < P.n_copy; ++sl) mask[P.subs[P.slot_sub[sl]].dof_off + P.slot_ldof[sl]] = 1;
    c->d_bmask = upload(c, mask);
    std::map<std::pair<int, std::vector<int>>, int> classes;
    c->dclass.assign(ns, 0);
    long long tmpl = 0;
    for (int p = 0; p < ns; ++p) {
      const SubInfo& sb = P.subs[p];
      std::vector<int> key(P.slot_ldof.begin() + sb.copy_off, P.slot_ldof.begin() + sb.copy_off + sb.n_copy);
      auto it = classes.find({sb.shape, key});
      if (it == classes.end()) {
        it = classes.emplace(std::make_pair(sb.shape, std::move(key)), (int)c->dclass_rep.size()).first;
        c->dclass_rep.push_back(p);
        c->dtmpl_off.push_back(tmpl);
        tmpl += (sb.fac_size + 3) & ~3LL;     // 16-byte aligned records (bulk copies)
      }
      c->dclass[p] = it->second;
    }
    long long max_fac = 0;
    for (const SubInfo& sb : P.subs) max_fac = std::max<long long>(max_fac, sb.fac_size);
    c->dfac = dalloc<double>(c, tmpl + max_fac);
    c->dfac32 = dalloc<float>(c, tmpl + max_fac);
    c->d_items_d = dalloc<SolveItem>(c, ns);
    c->d_items_d32 = dalloc<SolveItem>(c, ns);
    c->dx_a = dalloc<double>(c, P.n_dof);
    c->dx_b = dalloc<double>(c, P.n_dof);
    c->dx_c = dalloc<double>(c, P.n_dof);
    // template factors on the representatives' own band workspaces (unused at set-up)
    std::vector<long long> boffs = band_workspace(c, c->dclass_rep), foffs;
    int max_rows = 0;
    for (size_t k = 0; k < c->dclass_rep.size(); ++k) {
      const int rp = c->dclass_rep[k];
      foffs.push_back(c->dtmpl_off[k]);
      max_rows = std::max(max_rows, P.subs[rp].n_dof);
    }
    int* dl = upload(c, c->dclass_rep);
    long long* dbo = upload(c, boffs);
    long long* dfo = upload(c, foffs);
    launch_band_fill(M, dl, (int)boffs.size(), c->elem_np, c->dKe, c->band_ws, dbo, 1, max_rows, P.max_bw, c->st,
                     c->d_bmask);
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st);
    launch_band_chol(M, dl, (int)boffs.size(), dbo, c->band_ws, dfo, c->dfac, c->d_err, P.max_bw, c->n_sm, c->st);
    int herr = 0;
    cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    sync(c);
    if (herr) return fail(c, TFETI_ERR_NUMERIC, "non-positive pivot in a Dirichlet-preconditioner factorisation");
    long long len = 0;
    for (int rp : c->dclass_rep) len = std::max<long long>(len, P.subs[rp].fac_size);
    launch_fac_to_f32(c->dfac, c->dfac32, dfo, (int)foffs.size(), len, c->st);
    c->launches += 3;
  }
  // shared elastic factor per subdomain shape
  {
    std::vector<int> reps;
    std::vector<long long> offs, facs;
    int max_rows = 0;
    for (size_t s = 0; s < P.shapes.size(); ++s) {
      reps.push_back(P.shapes[s].rep_sub);
      offs.push_back(P.shapes[s].band_off);
      facs.push_back(P.shapes[s].fac_off);
      c->tmpl_off.push_back(P.shapes[s].band_off);
      c->tmpl_fac_off.push_back(P.shapes[s].fac_off);
      max_rows = std::max(max_rows, P.shapes[s].n_dof);
    }
    if (!base) {
    int* dl = upload(c, reps);
    long long* dof = upload(c, offs);
    long long* dfac = upload(c, facs);
    launch_band_fill(M, dl, (int)reps.size(), c->elem_np, c->dKe, c->band, dof, 1, max_rows, P.max_bw, c->st);
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st);
    launch_band_chol(M, dl, (int)reps.size(), dof, c->band, dfac, c->fac, c->d_err, P.max_bw, c->n_sm, c->st);
    int herr = 0;
    cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    sync(c);
    if (herr) return fail(c, TFETI_ERR_NUMERIC, "non-positive pivot in an elastic template factorisation");
    long long len = 0;
    for (const ShapeInfo& sh : P.shapes) len = std::max<long long>(len, P.subs[sh.rep_sub].fac_size);
    launch_fac_to_f32(c->fac, c->fac32, dfac, (int)reps.size(), len, c->st);
    build_items(c, std::vector<int>(ns, 0));
    std::vector<long long> kt;
    for (const ShapeInfo& sh : P.shapes) kt.push_back(sh.kbb_off);
    long long* dkt = upload(c, kt);
    launch_kbb_fill(M, dl, dkt, (int)reps.size(), c->max_bnd, c->elem_np, c->dKe, c->kbb, nullptr, 1, c->st);
    } else {
      build_items(c, std::vector<int>(ns, 0));
    }
    for (int p = 0; p < ns; ++p) c->h_kbb_off[p] = c->h_kbb_off32[p] = P.shapes[c->h_subs[p].shape].kbb_off;
    cudaMemcpyAsync(c->d_kbb_off, c->h_kbb_off.data(), sizeof(long long) * ns, cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(c->d_kbb_off32, c->h_kbb_off32.data(), sizeof(long long) * ns, cudaMemcpyHostToDevice, c->st);
  }
  c->launches += 4;
  cudaEventCreate(&c->fac_e0);
  cudaEventCreate(&c->in_e0);
  cudaEventCreate(&c->in_e1);
  cudaEventCreate(&c->fac_e1);
  cudaStreamCreateWithFlags(&c->st2, cudaStreamNonBlocking);
  cudaStreamCreateWithFlags(&c->st_fac, cudaStreamNonBlocking);
  cudaEventCreateWithFlags(&c->ev_fac_fork, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&c->ev_fac_done, cudaEventDisableTiming);
  c->d_err_fac = dalloc<int>(c, 1);
  if (cudaMallocHost(&c->h_err_fac, sizeof(int)) != cudaSuccess) throw std::bad_alloc();
  *c->h_err_fac = 0;
  cudaStreamCreateWithFlags(&c->st_cap, cudaStreamNonBlocking);
  cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
  for (int i = 0; i < 8192; ++i) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) break;
    c->ev_pool.push_back(e);
  }
  c->ev_kind.assign(c->ev_pool.size() / 2 + 1, 0);
  sync(c);
  return cuda_check(c, "tfeti_setup");
}

}  // namespace

// ===========================================================================
extern "C" {

const char* tfeti_status_str(int s) {
  switch (s) {
    case TFETI_OK: return "ok";
    case TFETI_ERR_ARG: return "invalid argument";
    case TFETI_ERR_CUDA: return "CUDA error";
    case TFETI_ERR_OOM: return "out of memory";
    case TFETI_ERR_NUMERIC: return "non-positive pivot";
    case TFETI_ERR_SINGULAR: return "singular coarse problem";
    case TFETI_ERR_NOT_CONVERGED: return "not converged";
    case TFETI_ERR_BREAKDOWN: return "PCGP breakdown";
    case TFETI_ERR_NONFINITE: return "non-finite value";
    case TFETI_ERR_TIMEOUT: return "bounded device wait gave up";
    default: return "unknown status";
  }
}

const char* tfeti_last_error(const tfeti_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int tfeti_setup(const tfeti_problem* prob, void* cuda_stream, tfeti_ctx** out) {
  if (!out) return TFETI_ERR_ARG;
  *out = nullptr;
  tfeti_ctx* c = new (std::nothrow) tfeti_ctx();
  if (!c) return TFETI_ERR_OOM;
  c->st = static_cast<cudaStream_t>(cuda_stream);
  int st = plan_build(prob, c->plan);
  if (st == TFETI_OK) {
    try {
      st = setup_impl(c);
    } catch (const std::bad_alloc&) {
      st = fail(c, TFETI_ERR_OOM, "device allocation failed");
    }
  }
  if (st != TFETI_OK) {
    tfeti_destroy(c);
    return st;
  }
  *out = c;
  return TFETI_OK;
}

int tfeti_setup_case(tfeti_ctx* base, double sigma_y, double hardening, void* cuda_stream, tfeti_ctx** out) {
  if (!out) return TFETI_ERR_ARG;
  *out = nullptr;
  if (!base || base->base) return TFETI_ERR_ARG;
  if (!(sigma_y > 0.0) || !(hardening > 0.0)) return fail(base, TFETI_ERR_ARG, "case: sigma_y and H must be > 0");
  tfeti_ctx* c = new (std::nothrow) tfeti_ctx();
  if (!c) return TFETI_ERR_OOM;
  c->base = base;
  if (cuda_stream) {
    c->st = static_cast<cudaStream_t>(cuda_stream);
  } else if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) == cudaSuccess) {
    c->owns_stream = true;
  } else {
    delete c;
    cudaGetLastError();
    return TFETI_ERR_CUDA;
  }
  int st = TFETI_OK;
  try {
    c->plan = base->plan;
    c->plan.prob.sigma_y = sigma_y;
    c->plan.prob.hardening = hardening;
    for (int a = 0; a < 3; ++a) c->plan.prob.cuts[a] = nullptr;   // already applied in the plan
    sync(base);
    st = setup_impl(c, base);
  } catch (const std::bad_alloc&) {
    st = fail(c, TFETI_ERR_OOM, "device allocation failed");
  }
  if (st != TFETI_OK) {
    tfeti_destroy(c);
    return st;
  }
  *out = c;
  return TFETI_OK;
}

int ssn_time_step_cases(tfeti_ctx* const* ctxs, int32_t n_cases, const double* const* df, int32_t df_on_host,
                        double newton_tol, double pcg_rtol, int32_t newton_maxit, int32_t pcg_maxit,
                        tfeti_step_info* info) {
  if (!ctxs || !df || n_cases < 1) return TFETI_ERR_ARG;
  for (int k = 0; k < n_cases; ++k) {
    if (!ctxs[k] || !df[k]) return TFETI_ERR_ARG;
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return fail(ctxs[k], TFETI_ERR_ARG, "ssn_time_step_cases: a context appears twice");
  }
  std::vector<int> status(n_cases, TFETI_OK);
  for (int k = 0; k < n_cases; ++k) ctxs[k]->in_cases = n_cases > 1;
  auto run = [&](int k) {
    // a new host thread starts on device 0: make the context's device current
    if (cudaSetDevice(ctxs[k]->device) != cudaSuccess) {
      cudaGetLastError();
      status[k] = fail(ctxs[k], TFETI_ERR_CUDA, "ssn_time_step_cases: cudaSetDevice failed");
      return;
    }
    try {
      status[k] = ssn_time_step(ctxs[k], df[k], df_on_host, newton_tol, pcg_rtol, newton_maxit, pcg_maxit,
                                info ? info + k : nullptr);
    } catch (const std::bad_alloc&) {
      status[k] = fail(ctxs[k], TFETI_ERR_OOM, "host allocation failed");
    } catch (...) {
      status[k] = fail(ctxs[k], TFETI_ERR_ARG, "unexpected exception");
    }
  };
  std::vector<std::thread> threads;
  try {
    for (int k = 1; k < n_cases; ++k) threads.emplace_back(run, k);
  } catch (const std::system_error&) {
    for (std::thread& t : threads) t.join();
    return fail(ctxs[0], TFETI_ERR_ARG, "ssn_time_step_cases: could not start a host thread");
  }
  int prev_device = 0;
  cudaGetDevice(&prev_device);
  run(0);
  cudaSetDevice(prev_device);   // the caller's current device is left as it was
  for (std::thread& t : threads) t.join();
  for (int k = 0; k < n_cases; ++k) ctxs[k]->in_cases = false;
  for (int k = 0; k < n_cases; ++k)
    if (status[k] != TFETI_OK) return status[k];
  return TFETI_OK;
}

int tfeti_destroy(tfeti_ctx* c) {
  if (!c) return TFETI_OK;
  if (c->st) cudaStreamSynchronize(c->st);
  else cudaDeviceSynchronize();
  if (c->st_fac) cudaStreamSynchronize(c->st_fac);
  if (c->st_mlp) cudaStreamSynchronize(c->st_mlp);
  if (c->st_wood) cudaStreamSynchronize(c->st_wood);
  if (c->st_wc) cudaStreamSynchronize(c->st_wc);
  for (void* p : c->allocs) cudaFree(p);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->fac_e0) cudaEventDestroy(c->fac_e0);
  if (c->in_e0) cudaEventDestroy(c->in_e0);
  if (c->in_e1) cudaEventDestroy(c->in_e1);
  if (c->fac_e1) cudaEventDestroy(c->fac_e1);
  destroy_inner_graph(c);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->st_fac) cudaStreamDestroy(c->st_fac);
  if (c->ev_fac_fork) cudaEventDestroy(c->ev_fac_fork);
  if (c->ev_fac_done) cudaEventDestroy(c->ev_fac_done);
  if (c->h_err_fac) cudaFreeHost(c->h_err_fac);
  if (c->st2) cudaStreamDestroy(c->st2);
  if (c->st_mlp) cudaStreamDestroy(c->st_mlp);
  if (c->st_wood) cudaStreamDestroy(c->st_wood);
  if (c->st_wc) cudaStreamDestroy(c->st_wc);
  if (c->ev_wc_fork) cudaEventDestroy(c->ev_wc_fork);
  if (c->ev_wc_done) cudaEventDestroy(c->ev_wc_done);
  if (c->ev_wood_fork) cudaEventDestroy(c->ev_wood_fork);
  if (c->ev_wood_done) cudaEventDestroy(c->ev_wood_done);
  if (c->h_err_wood) cudaFreeHost(c->h_err_wood);
  if (c->ev_mlp_fork) cudaEventDestroy(c->ev_mlp_fork);
  if (c->ev_mlp_done) cudaEventDestroy(c->ev_mlp_done);
  if (c->st_cap) cudaStreamDestroy(c->st_cap);
  if (c->h_sc) cudaFreeHost(c->h_sc);
  if (c->owns_stream && c->st) cudaStreamDestroy(c->st);
  delete c;
  return TFETI_OK;
}

int tfeti_sizes_get(const tfeti_ctx* c, tfeti_sizes* out) {
  if (!c || !out) return TFETI_ERR_ARG;
  fill_sizes(c, out);
  return TFETI_OK;
}

int tfeti_traction_load(tfeti_ctx* c, const double* t, double* f_out) {
  if (!c || !t || !f_out) return fail(c, TFETI_ERR_ARG, "null argument");
  launch_traction(c->M, c->plan.prob.traction_face, c->plan.prob.nel, t, c->plan.h, f_out, c->st);
  c->launches += 1;
  return cuda_check(c, "tfeti_traction_load");
}

int tfeti_return_map(tfeti_ctx* c, const double* du, double* dsigma, double* dkappa, uint8_t* plastic,
                     double* Dtan) {
  if (!c || !du || !dsigma || !dkappa || !plastic) return fail(c, TFETI_ERR_ARG, "null argument");
  launch_return_map(c->M, du, c->sig, c->kap, dsigma, dkappa, plastic, Dtan, nullptr, nullptr, nullptr, c->st);
  c->launches += 1;
  return cuda_check(c, "tfeti_return_map");
}

int tfeti_assemble_tangent(tfeti_ctx* c, const double* du, const double* df, double* f_out) {
  if (!c || !du || !df) return fail(c, TFETI_ERR_ARG, "null argument");
  int st = assemble(c, du, df, f_out);
  sync(c);
  return st;
}

int tfeti_dual_pcg(tfeti_ctx* c, const double* f, double* u_out, double* lambda_out, const double* lambda0,
                   double rtol, int32_t maxit, tfeti_pcg_info* info) {
  if (!c || !f || !u_out || !(rtol >= 0.0) || maxit < 0) return fail(c, TFETI_ERR_ARG, "bad argument");
  return dual_pcg(c, f, u_out, lambda_out, lambda0, rtol, maxit, info);
}

int ssn_time_step(tfeti_ctx* c, const double* df, int32_t df_on_host, double newton_tol, double pcg_rtol,
                  int32_t newton_maxit, int32_t pcg_maxit, tfeti_step_info* info) {
  if (!c || !df || !(newton_tol >= 0.0) || newton_maxit < 1 || newton_maxit > TFETI_MAX_NEWTON)
    return fail(c, TFETI_ERR_ARG, "bad argument");
  const auto t0 = std::chrono::steady_clock::now();
  const DevMesh& M = c->M;
  const long long n = M.n_dof;
  tfeti_step_info loc{};
  c->last_refactored.clear();
  cudaMemcpyAsync(c->df, df, sizeof(double) * n, df_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                  c->st);
  cudaMemsetAsync(c->du, 0, sizeof(double) * n, c->st);
  if (c->mlp_on) {
    // load-increment ratio of the MLP features: (df . df_prev) / ||df_prev||^2
    double den = c->have_dfprev ? dot_host(c, c->mlp_dfprev, c->mlp_dfprev, n) : 0.0;
    c->mlp_rho = den > 0.0 ? dot_host(c, c->df, c->mlp_dfprev, n) / den : 1.0;
  }
  int status = TFETI_OK;
  double nrm_old = 0.0;
  for (int i = 1; i <= newton_maxit; ++i) {
    status = assemble(c, c->du, c->df, nullptr, true);
    if (status != TFETI_OK) break;
    if (c->mlp_on) launch_plastic_fraction(M, c->sub_np, c->pf_now, c->st);
    c->newton_idx = i;
    std::vector<int> np(M.n_sub);
    cudaMemcpyAsync(np.data(), c->sub_np, sizeof(int) * M.n_sub, cudaMemcpyDeviceToHost, c->st);
    tfeti_pcg_info pi{};
    status = dual_pcg(c, c->f_full, c->tn, nullptr, nullptr, pcg_rtol, pcg_maxit, &pi);
    c->newton_idx = 0;
    {
      const int fst = check_factorisation(c);   // no-op unless the solve ended before its join
      if (status == TFETI_OK) status = fst;
    }
    if (status != TFETI_OK) break;
    const double nd = std::sqrt(dot_host(c, c->tn, c->tn, n));
    launch_axpby(n, 1.0, c->du, 1.0, c->tn, c->du, c->st);
    c->launches += 1;
    const double nrm_new = std::sqrt(dot_host(c, c->du, c->du, n));
    const double den = nrm_new + nrm_old;
    const double crit = den == 0.0 ? 0.0 : nd / den;
    nrm_old = nrm_new;
    long long npl = 0;
    for (int v : np) npl += v;
    loc.newton = i;
    loc.pcg[i - 1] = pi.iterations;
    loc.outer[i - 1] = pi.outer_iterations;
    loc.history[i - 1] = pi.used_lambda0 == 2 ? 1 : (pi.used_lambda0 == 3 ? 2 : 0);
    loc.plastic[i - 1] = npl;
    loc.criterion[i - 1] = crit;
    loc.refactored[i - 1] = c->last_refactored.empty() ? 0 : c->last_refactored.back();
    if (!std::isfinite(crit)) {
      status = fail(c, TFETI_ERR_NONFINITE, "non-finite Newton increment");
      break;
    }
    if (crit <= newton_tol) {
      loc.converged = 1;
      break;
    }
  }
  {
    // a refactorisation queued on st_fac by an assembly whose step then failed is joined here, so
    // that no later call reads own factors (or the list buffers) while it may still run
    const int fst = check_factorisation(c);
    if (status == TFETI_OK) status = fst;
  }
  if (c->mlp_on) {
    cudaMemcpyAsync(c->mlp_dfprev, c->df, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st);
    c->have_dfprev = true;
  }
  if (status == TFETI_OK && !loc.converged) status = fail(c, TFETI_ERR_NOT_CONVERGED, "Newton iteration limit");
  if (status == TFETI_OK) {
    // commit at the converged increment (Algorithm 1 evaluates T_k at the solution)
    launch_return_map(M, c->du, c->sig, c->kap, c->dsig, c->dkap, c->plastic, nullptr, nullptr, nullptr, nullptr,
                      c->st);
    cudaMemsetAsync(c->sub_np, 0, sizeof(int) * M.n_sub, c->st);
    GPData gd{c->dsig, c->pa, c->pb, c->pn, c->plastic};
    launch_elem_correction(M, gd, c->elem_np, c->sub_np, c->dKe, c->st);
    std::vector<int> np(M.n_sub);
    cudaMemcpyAsync(np.data(), c->sub_np, sizeof(int) * M.n_sub, cudaMemcpyDeviceToHost, c->st);
    launch_commit(M, c->du, c->dsig, c->dkap, c->u, c->sig, c->kap, c->st);
    c->launches += 3;
    sync(c);
    for (int v : np) loc.plastic_committed += v;
  }
  sync(c);
  loc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = loc;
  int cst = cuda_check(c, "ssn_time_step");
  return cst != TFETI_OK ? cst : status;
}

int tfeti_set_precision(tfeti_ctx* c, int32_t mode, double inner_rtol) {
  if (!c || (mode != TFETI_PRECISION_FP64 && mode != TFETI_PRECISION_MIXED) || !(inner_rtol > 0.0 && inner_rtol < 1.0))
    return fail(c, TFETI_ERR_ARG, "bad precision mode or inner tolerance");
  if (mode == TFETI_PRECISION_MIXED && c->precision != TFETI_PRECISION_MIXED) {
    // bring the FP32 copies of the per-subdomain factors in use up to date
    std::vector<long long> offs;
    long long len = 0;
    for (const SolveItem& it : c->h_items)
      if (it.fac & kOwnFac) {
        offs.push_back(it.fac & ~kOwnFac);
        len = std::max<long long>(len, c->plan.subs[it.sub[0]].fac_size);
      }
    if (!offs.empty()) {
      cudaMemcpyAsync(c->d_list_fac, offs.data(), sizeof(long long) * offs.size(), cudaMemcpyHostToDevice, c->st);
      launch_fac_to_f32(c->fac_own, c->fac32_own, c->d_list_fac, (int)offs.size(), len, c->st);
      sync(c);
    }
    if (c->dirichlet) {
      std::vector<long long> doffs;
      for (const SolveItem& it : c->h_items_d)
        if (it.fac & kOwnFac) doffs.push_back(it.fac & ~kOwnFac);
      if (!doffs.empty()) {
        cudaMemcpyAsync(c->d_list_fac, doffs.data(), sizeof(long long) * doffs.size(), cudaMemcpyHostToDevice,
                        c->st);
        launch_fac_to_f32(c->dfac_own, c->dfac32_own, c->d_list_fac, (int)doffs.size(), len, c->st);
        sync(c);
      }
    }
  }
  c->precision = mode;
  c->inner_rtol = inner_rtol;
  c->g_inner_stale = true;
  if (mode == TFETI_PRECISION_MIXED && !c->kbb32) {
    // FP32 copies of the coarse solve and the boundary blocks for the inner projector and
    // preconditioner (the FP32 values of G are formed at set-up)
    // (a case context shares the base's FP32 coarse blocks, formed here if the base has none)
    tfeti_ctx* hown = c->base ? c->base : c;
    try {
      if (hown->coarse.mode == kCoarseDense && !hown->H32) {
        hown->H32 = dalloc<float>(hown, (size_t)c->l * (size_t)h32_ld(c->l));
        launch_h_to_f32(hown->H, c->l, hown->H32, c->st);
        hown->coarse.H32 = hown->H32;
        sync(c);
      }
      if (hown->coarse.mode == kCoarsePlanes && !hown->cW32) {
        const long long n = (long long)hown->coarse.n_pl * hown->coarse.n_pl * hown->coarse.n_planes;
        hown->cW32 = dalloc<float>(hown, (size_t)n);
        hown->cV32 = dalloc<float>(hown, (size_t)n);
        hown->cU32 = dalloc<float>(hown, (size_t)n);
        launch_to_f32(hown->cW, hown->cW32, n, c->st);
        launch_to_f32(hown->cV, hown->cV32, n, c->st);
        launch_to_f32(hown->cU, hown->cU32, n, c->st);
        hown->coarse.W32 = hown->cW32;
        hown->coarse.V32 = hown->cV32;
        hown->coarse.U32 = hown->cU32;
        sync(c);
      }
      c->H32 = hown->H32;
      c->coarse = hown->coarse;
      c->kbb32 = dalloc<float>(c, c->plan.kbb_template_total + c->plan.kbb_total);
    } catch (const std::bad_alloc&) {
      return fail(c, TFETI_ERR_OOM, "device allocation failed");
    }
    launch_to_f32(c->kbb, c->kbb32, c->plan.kbb_template_total + c->plan.kbb_total, c->st);
    c->launches += 2;
  }
  if (mode == TFETI_PRECISION_MIXED) {
    const bool fresh = !c->schur_ready;
    int st = ensure_schur(c);
    if (st != TFETI_OK) return st;
    if (c->wood_mode > 0) {
      st = ensure_kinv(c);
      if (st != TFETI_OK) return st;
    }
    if (fresh || c->schur_threshold == 0) {
      st = tune_schur_threshold(c);
      if (st != TFETI_OK) return st;
    }
  }
  return cuda_check(c, "tfeti_set_precision");
}

int tfeti_set_fapply(tfeti_ctx* c, int32_t mode) {
  if (!c || (mode != TFETI_FAPPLY_BANDED && mode != TFETI_FAPPLY_SCHUR)) return fail(c, TFETI_ERR_ARG, "bad F-apply mode");
  if (mode == TFETI_FAPPLY_SCHUR) {
    const int st = ensure_schur(c);
    if (st != TFETI_OK) return st;
  }
  c->fapply = mode;
  return cuda_check(c, "tfeti_set_fapply");
}

int tfeti_set_schur_format(tfeti_ctx* c, int32_t format) {
  if (!c || (format != TFETI_SCHUR_TF32X3 && format != TFETI_SCHUR_BF16))
    return fail(c, TFETI_ERR_ARG, "bad Schur operand format");
  if (c->precision != TFETI_PRECISION_MIXED) return fail(c, TFETI_ERR_ARG, "the Schur operand format needs the mixed mode");
  if (format == TFETI_SCHUR_BF16) {
    const int st = ensure_schur_bf16(c);
    if (st != TFETI_OK) return st;
  }
  const bool bf = format == TFETI_SCHUR_BF16;
  if (bf != c->schur_bf16) {
    c->schur_bf16 = bf;
    c->g_inner_stale = true;
    if (!c->schur_manual) {
      const int st = tune_schur_threshold(c);   // the faster BF16 apply may move the threshold
      if (st != TFETI_OK) return st;
    }
  }
  return cuda_check(c, "tfeti_set_schur_format");
}

int tfeti_set_schur_threshold(tfeti_ctx* c, int32_t threshold) {
  if (!c || threshold < 0) return fail(c, TFETI_ERR_ARG, "bad Schur threshold");
  if (c->precision != TFETI_PRECISION_MIXED) return fail(c, TFETI_ERR_ARG, "the Schur threshold needs the mixed mode");
  c->schur_manual = threshold != 0;
  if (threshold == 0) return tune_schur_threshold(c);
  {
    const int wst = wood_materialize(c);
    if (wst != TFETI_OK) return wst;
  }
  const size_t nsh = c->plan.shapes.size();
  std::vector<int> count(nsh, 0);
  for (const SubDev& sd : c->h_subs) ++count[sd.shape];
  c->schur_threshold = threshold;
  for (size_t sh = 0; sh < nsh; ++sh) c->schur_use[sh] = c->schur_formed[sh] && count[sh] >= threshold;
  build_items(c, c->h_np.size() == c->h_subs.size() ? c->h_np : std::vector<int>(c->h_subs.size(), 0));
  c->g_inner_stale = true;
  return cuda_check(c, "tfeti_set_schur_threshold");
}

int tfeti_get_tuning(tfeti_ctx* c, int32_t* schur_threshold, int32_t* n_schur_shapes, float* tune_ms) {
  if (!c) return TFETI_ERR_ARG;
  int n = 0;
  for (char u : c->schur_use) n += u != 0;
  if (schur_threshold) *schur_threshold = c->schur_threshold;
  if (n_schur_shapes) *n_schur_shapes = n;
  if (tune_ms)
    for (int i = 0; i < 4; ++i) tune_ms[i] = i < (int)c->schur_tune_ms.size() ? c->schur_tune_ms[i] : -1.f;
  return TFETI_OK;
}

int tfeti_set_graphs(tfeti_ctx* c, int32_t enable) {
  if (!c) return TFETI_ERR_ARG;
  c->use_graphs = enable != 0;
  c->g_inner_stale = true;
  return TFETI_OK;
}

int tfeti_set_recycling(tfeti_ctx* c, int32_t q) {
  if (!c || q < 0 || q > kRecMax) return fail(c, TFETI_ERR_ARG, "history size must be in 0..8");
  if (c->mlp_on && (q < 1 || q > kRecMax - 1))
    return fail(c, TFETI_ERR_ARG, "with the learned start the history size must be in 1..7");
  const long long m = c->M.n_mult;
  if (q > 0 && q > c->rec_q) {
    try {
      // one spare slot for the MLP vector of the learned start
      const long long nd = std::max(1LL, c->M.n_dof);
      dfree(c, c->rec_L, (size_t)(c->rec_q + 1) * (size_t)std::max(1LL, m));
      dfree(c, c->rec_FL, (size_t)(c->rec_q + 1) * (size_t)std::max(1LL, m));
      dfree(c, c->rec_W, (size_t)(c->rec_q + 1) * (size_t)nd);
      c->rec_L = dalloc<double>(c, (size_t)(q + 1) * (size_t)std::max(1LL, m));
      c->rec_FL = dalloc<double>(c, (size_t)(q + 1) * (size_t)std::max(1LL, m));
      c->rec_W = dalloc<double>(c, (size_t)(q + 1) * (size_t)nd);
      if (!c->vsol_im) c->vsol_im = dalloc<double>(c, (size_t)nd);
      if (!c->rec_partial) {
        c->rec_partial = dalloc<double>(c, (size_t)kRedBlocks * (kRecMax * kRecMax + kRecMax));
        c->rec_out = dalloc<double>(c, kRecMax * kRecMax + kRecMax);
        c->rec_c = dalloc<double>(c, kRecMax);
        c->dtil = dalloc<double>(c, (size_t)std::max(1LL, m));
      }
    } catch (const std::bad_alloc&) {
      return fail(c, TFETI_ERR_OOM, "device allocation failed");
    }
  }
  c->rec_q = q;
  c->rec_n = 0;
  c->rec_head = 0;
  c->rec_tried = c->rec_used = c->rec_exact = 0;
  c->rec_ver.assign((size_t)q + 1, -1);
  return cuda_check(c, "tfeti_set_recycling");
}

int tfeti_set_woodbury(tfeti_ctx* c, int32_t mode) {
  if (!c) return TFETI_ERR_ARG;
  if (mode < 0 || mode > 2) return fail(c, TFETI_ERR_ARG, "Woodbury mode must be 0, 1 or 2");
  c->wood_mode = mode;
  if (mode > 0 && c->precision == TFETI_PRECISION_MIXED && c->schur_ready) {
    const int st = ensure_kinv(c);
    if (st != TFETI_OK) return st;
  }
  return TFETI_OK;   // takes effect at the next assembly
}

int tfeti_set_fused_inner(tfeti_ctx* c, int32_t enable) {
  if (!c) return TFETI_ERR_ARG;
  c->fused_req = enable != 0;
  return TFETI_OK;   // the inner graph is rebuilt at the next inner solve if the choice changes
}

int tfeti_get_fused_inner(tfeti_ctx* c, int32_t* active) {
  if (!c || !active) return TFETI_ERR_ARG;
  *active = c->precision == TFETI_PRECISION_MIXED && fused_usable(c) ? 1 : 0;
  return cuda_check(c, "tfeti_get_fused_inner");
}

int tfeti_get_woodbury_stats(tfeti_ctx* c, int64_t* subdomains, int64_t* fallbacks) {
  if (!c) return TFETI_ERR_ARG;
  if (subdomains) *subdomains = c->wood_subs;
  if (fallbacks) *fallbacks = c->wood_fallbacks;
  return TFETI_OK;
}

int tfeti_set_deflation(tfeti_ctx* c, int32_t k) {
  if (!c || k < 0 || k > kDeflMax) return fail(c, TFETI_ERR_ARG, "deflation size must be in 0..8");
  if (k > 0 && c->rec_q < 1) return fail(c, TFETI_ERR_ARG, "deflation needs the history start (tfeti_set_recycling)");
  const long long m = c->M.n_mult;
  if (k > 0 && !c->defl_W) {
    try {
      c->defl_W = dalloc<double>(c, (size_t)kDeflMax * (size_t)std::max(1LL, m));
      c->defl_AW = dalloc<double>(c, (size_t)kDeflMax * (size_t)std::max(1LL, m));
      c->defl_Einv = dalloc<double>(c, kDeflMax * kDeflMax);
    } catch (const std::bad_alloc&) {
      return fail(c, TFETI_ERR_OOM, "device allocation failed");
    }
    c->g_inner_stale = true;   // the graph body takes the deflation buffers
  }
  c->defl_req = k;
  c->defl_setups = c->defl_vectors = c->defl_fallbacks = 0;
  return cuda_check(c, "tfeti_set_deflation");
}

int tfeti_get_deflation_stats(tfeti_ctx* c, int64_t* setups, int64_t* vectors, int64_t* fallbacks) {
  if (!c) return TFETI_ERR_ARG;
  if (setups) *setups = c->defl_setups;
  if (vectors) *vectors = c->defl_vectors;
  if (fallbacks) *fallbacks = c->defl_fallbacks;
  return TFETI_OK;
}

int tfeti_set_learned(tfeti_ctx* c, int32_t enable, int32_t epochs, double lr) {
  if (!c || epochs < 0 || epochs > 1000 || !(lr > 0.0 && lr < 1.0)) return fail(c, TFETI_ERR_ARG, "bad argument");
  if (enable && (c->rec_q < 1 || c->rec_q > kRecMax - 1))
    return fail(c, TFETI_ERR_ARG, "the learned start needs a history of 1..7 (tfeti_set_recycling)");
  const long long m = c->M.n_mult;
  if (enable && !c->mlp_w) {
    try {
      c->mlp_w = dalloc<float>(c, kMlpParams);
      c->mlp_m1 = dalloc<float>(c, kMlpParams);
      c->mlp_m2 = dalloc<float>(c, kMlpParams);
      c->mlp_partial = dalloc<float>(c, (size_t)c->mlp_blocks * kMlpParams);
      c->mlp_scal = dalloc<float>(c, 8);
      c->mlp_w16 = dalloc<uint16_t>(c, kMlpParams);
      c->mlp_la = dalloc<double>(c, (size_t)kMlpIdx * (size_t)std::max(1LL, m));
      c->mlp_lb = dalloc<double>(c, (size_t)kMlpIdx * (size_t)std::max(1LL, m));
      c->mlp_dfprev = dalloc<double>(c, (size_t)std::max(1LL, c->M.n_dof));
      c->pf_now = dalloc<float>(c, c->M.n_sub);
      c->pf_prev = dalloc<float>(c, (size_t)kMlpIdx * c->M.n_sub);
      c->mlp_d = dalloc<double>(c, (size_t)std::max(1LL, m));
      c->mlp_tgt = dalloc<double>(c, (size_t)std::max(1LL, m));
      c->mlp_pf = dalloc<float>(c, (size_t)std::max(1, c->M.n_sub));
      c->mlp_scal_t = dalloc<float>(c, 8);
      int lo = 0, hi = 0;
      cudaDeviceGetStreamPriorityRange(&lo, &hi);
      cudaStreamCreateWithPriority(&c->st_mlp, cudaStreamNonBlocking, lo);
      cudaEventCreateWithFlags(&c->ev_mlp_fork, cudaEventDisableTiming);
      cudaEventCreateWithFlags(&c->ev_mlp_done, cudaEventDisableTiming);
    } catch (const std::bad_alloc&) {
      return fail(c, TFETI_ERR_OOM, "device allocation failed");
    }
  }
  if (c->st_mlp) cudaStreamSynchronize(c->st_mlp);
  if (c->st_wood) cudaStreamSynchronize(c->st_wood);   // no training in flight while the network is reset
  c->mlp_pending = false;
  if (enable) {
    // seeded initialisation: uniform(-a, a), a = sqrt(6 / (fan_in + fan_out)) for the two
    // hidden layers, zero biases and a zero last layer (the untrained predictor is the
    // previous step's value)
    std::vector<float> w(kMlpParams, 0.0f);
    unsigned long long st = 0x9E3779B97F4A7C15ULL;
    auto uni = [&st]() {
      st = st * 6364136223846793005ULL + 1442695040888963407ULL;
      return (double)(st >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    };
    const double a1 = std::sqrt(6.0 / (kMlpIn + kMlpHid)), a2 = std::sqrt(6.0 / (2 * kMlpHid));
    for (int i = 0; i < kMlpHid * kMlpIn; ++i) w[i] = (float)(a1 * uni());
    const int w2 = kMlpHid * kMlpIn + kMlpHid;
    for (int i = 0; i < kMlpHid * kMlpHid; ++i) w[w2 + i] = (float)(a2 * uni());
    cudaMemcpyAsync(c->mlp_w, w.data(), sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, c->st);
    cudaMemsetAsync(c->mlp_m1, 0, sizeof(float) * kMlpParams, c->st);
    cudaMemsetAsync(c->mlp_m2, 0, sizeof(float) * kMlpParams, c->st);
    cudaMemsetAsync(c->mlp_la, 0, sizeof(double) * kMlpIdx * m, c->st);
    cudaMemsetAsync(c->mlp_lb, 0, sizeof(double) * kMlpIdx * m, c->st);
    cudaMemsetAsync(c->pf_now, 0, sizeof(float) * c->M.n_sub, c->st);
    cudaMemsetAsync(c->pf_prev, 0, sizeof(float) * kMlpIdx * c->M.n_sub, c->st);
    launch_mlp_cast(c->mlp_w, c->mlp_w16, c->st);
    sync(c);
  }
  c->mlp_on = enable != 0;
  c->mlp_epochs = epochs;
  c->mlp_lr = (float)lr;
  c->mlp_t = 0;
  for (int& v : c->mlp_seen) v = 0;
  c->mlp_used = c->mlp_skipped = c->mlp_probe = 0;
  for (int& v : c->mlp_nogain) v = 0;
  c->have_dfprev = false;
  return cuda_check(c, "tfeti_set_learned");
}

int tfeti_mlp_predict(tfeti_ctx* c, const double* la, const double* lb, const double* d, const float* pf_now,
                      const float* pf_prev, const float* scal, double* y) {
  if (!c || !la || !lb || !d || !pf_now || !pf_prev || !scal || !y) return fail(c, TFETI_ERR_ARG, "null argument");
  if (!c->mlp_w) return fail(c, TFETI_ERR_ARG, "the learned start is not set up");
  const float sc[5] = {scal[0], scal[1], scal[2], scal[3], 0.0f};
  cudaMemcpyAsync(c->mlp_scal, sc, sizeof(sc), cudaMemcpyHostToDevice, c->st);
  sync(c);
  mlp_join(c);
  launch_mlp_infer(c->M, c->mlp_w16, la, lb, d, pf_now, pf_prev, c->mlp_scal, y, c->st);
  c->launches += 1;
  sync(c);
  c->mlp_scal_valid = false;
  return cuda_check(c, "tfeti_mlp_predict");
}

int tfeti_mlp_train(tfeti_ctx* c, const double* la, const double* lb, const double* d, const float* pf_now,
                    const float* pf_prev, const float* scal, const double* target, int32_t steps) {
  if (!c || !la || !lb || !d || !pf_now || !pf_prev || !scal || !target || steps < 0)
    return fail(c, TFETI_ERR_ARG, "bad argument");
  if (!c->mlp_w) return fail(c, TFETI_ERR_ARG, "the learned start is not set up");
  const long long m = c->M.n_mult;
  const float sc[5] = {scal[0], scal[1], scal[2], scal[3], 0.0f};
  cudaMemcpyAsync(c->mlp_scal, sc, sizeof(sc), cudaMemcpyHostToDevice, c->st);
  sync(c);
  for (int e = 0; e < steps && m > 0; ++e) {
    ++c->mlp_t;
    const long long start = (104729LL * c->mlp_t + 7919LL * e) % m;
    launch_mlp_train_step(c->M, c->mlp_w, la, lb, d, pf_now, pf_prev, c->mlp_scal, target, start, 7919,
                          c->mlp_blocks, c->mlp_partial, c->mlp_w, c->mlp_m1, c->mlp_m2, c->mlp_w16, c->mlp_lr,
                          c->mlp_t, c->st);
    c->launches += 2;
  }
  sync(c);
  c->mlp_scal_valid = false;
  return cuda_check(c, "tfeti_mlp_train");
}

int tfeti_mlp_weights(tfeti_ctx* c, float* out) {
  if (!c || !out) return fail(c, TFETI_ERR_ARG, "null argument");
  if (!c->mlp_w) return fail(c, TFETI_ERR_ARG, "the learned start is not set up");
  cudaMemcpyAsync(out, c->mlp_w, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, c->st);
  sync(c);
  return cuda_check(c, "tfeti_mlp_weights");
}

int tfeti_first_yield_traction(tfeti_ctx* c, const double* dir, double rtol, double* t_y) {
  if (!c || !dir || !t_y) return fail(c, TFETI_ERR_ARG, "null argument");
  const long long n = c->M.n_dof;
  launch_traction(c->M, c->plan.prob.traction_face, c->plan.prob.nel, dir, c->plan.h, c->tn2, c->st);
  cudaMemsetAsync(c->du, 0, sizeof(double) * n, c->st);
  int st = assemble(c, c->du, c->tn2, nullptr);
  if (st != TFETI_OK) return st;
  st = dual_pcg(c, c->f_full, c->tn, nullptr, nullptr, rtol, 100000, nullptr);
  if (st != TFETI_OK) return st;
  launch_return_map(c->M, c->tn, c->sig, c->kap, c->dsig, c->dkap, c->plastic, nullptr, nullptr, nullptr, nullptr,
                    c->st);
  launch_vm_max(c->M, c->dsig, c->partial, c->sc + 9, c->st);
  c->launches += 4;
  double q = 0.0;
  cudaMemcpyAsync(&q, c->sc + 9, sizeof(double), cudaMemcpyDeviceToHost, c->st);
  sync(c);
  if (!(q > 0.0)) return fail(c, TFETI_ERR_NUMERIC, "zero elastic response");
  *t_y = c->plan.prob.sigma_y / q;
  return cuda_check(c, "tfeti_first_yield_traction");
}

int tfeti_get_state(tfeti_ctx* c, double* u, double* sigma, double* kappa) {
  if (!c) return TFETI_ERR_ARG;
  if (u) cudaMemcpyAsync(u, c->u, sizeof(double) * c->M.n_dof, cudaMemcpyDeviceToDevice, c->st);
  if (sigma) cudaMemcpyAsync(sigma, c->sig, sizeof(double) * 6 * c->M.n_gp, cudaMemcpyDeviceToDevice, c->st);
  if (kappa) cudaMemcpyAsync(kappa, c->kap, sizeof(double) * c->M.n_gp, cudaMemcpyDeviceToDevice, c->st);
  sync(c);
  return cuda_check(c, "tfeti_get_state");
}

int tfeti_set_state(tfeti_ctx* c, const double* u, const double* sigma, const double* kappa) {
  if (!c) return TFETI_ERR_ARG;
  if (u) cudaMemcpyAsync(c->u, u, sizeof(double) * c->M.n_dof, cudaMemcpyDeviceToDevice, c->st);
  if (sigma) cudaMemcpyAsync(c->sig, sigma, sizeof(double) * 6 * c->M.n_gp, cudaMemcpyDeviceToDevice, c->st);
  if (kappa) cudaMemcpyAsync(c->kap, kappa, sizeof(double) * c->M.n_gp, cudaMemcpyDeviceToDevice, c->st);
  sync(c);
  return cuda_check(c, "tfeti_set_state");
}

int tfeti_apply_F(tfeti_ctx* c, const double* x, double* y) {
  if (!c || !x || !y) return fail(c, TFETI_ERR_ARG, "null argument");
  op_F(c, x, y);
  sync(c);
  collect_events(c);
  return cuda_check(c, "tfeti_apply_F");
}

int tfeti_apply_F32(tfeti_ctx* c, const double* x, double* y) {
  if (!c || !x || !y) return fail(c, TFETI_ERR_ARG, "null argument");
  if (c->precision != TFETI_PRECISION_MIXED) return fail(c, TFETI_ERR_ARG, "FP32 F-apply needs the mixed mode");
  op_F32(c, x, y);
  int herr = 0;
  cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st);
  sync(c);
  const int cst = cuda_check(c, "tfeti_apply_F32");
  if (cst != TFETI_OK) return cst;
  if (herr & 6) {
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st);
    return fail(c, TFETI_ERR_TIMEOUT, "a bounded device wait gave up in the FP32 F-apply");
  }
  return TFETI_OK;
}

int tfeti_apply_projector(tfeti_ctx* c, const double* x, double* y) {
  if (!c || !x || !y) return fail(c, TFETI_ERR_ARG, "null argument");
  op_project(c, x, y);
  sync(c);
  return cuda_check(c, "tfeti_apply_projector");
}

int tfeti_apply_precond(tfeti_ctx* c, const double* x, double* y) {
  if (!c || !x || !y) return fail(c, TFETI_ERR_ARG, "null argument");
  op_precond(c, x, y);
  sync(c);
  return cuda_check(c, "tfeti_apply_precond");
}

int tfeti_apply_N(tfeti_ctx* c, const double* x, double* y) {
  if (!c || !x || !y) return fail(c, TFETI_ERR_ARG, "null argument");
  launch_G_apply(c->M, x, nullptr, y, -1.0, c->st);
  c->launches += 1;
  sync(c);
  return cuda_check(c, "tfeti_apply_N");
}

int tfeti_apply_kdag(tfeti_ctx* c, const double* x, double* y) {
  if (!c || !x || !y) return fail(c, TFETI_ERR_ARG, "null argument");
  SolveArgs a = solve_args(c);
  a.src = x;
  a.dst = y;
  a.in_mode = 1;
  a.out_mode = 1;
  launch_sub_solve(c->M, a, c->solve_smem, c->st);
  wood_correct_solve(c, a, c->st);
  c->launches += 1;
  sync(c);
  return cuda_check(c, "tfeti_apply_kdag");
}

int tfeti_apply_K(tfeti_ctx* c, const double* x, double* y) {
  if (!c || !x || !y) return fail(c, TFETI_ERR_ARG, "null argument");
  launch_apply_K(c->M, c->elem_np, c->dKe, x, y, c->st);
  c->launches += 1;
  sync(c);
  return cuda_check(c, "tfeti_apply_K");
}

int tfeti_timing_get(tfeti_ctx* c, tfeti_timing* out) {
  if (!c || !out) return TFETI_ERR_ARG;
  collect_events(c);
  out->f_apply_ms_total = c->f_ms;
  out->f_apply_launches = c->f_launches;
  double bytes = 0.0, flops = 0.0;
  for (const SubDev& s : c->h_subs) {
    // two sweeps over the panels (nb x bw per block) and the inverted diagonal blocks
    const double panel = (double)s.nblk * s.nb * s.bw, diag = (double)s.nblk * s.nb * (s.nb + 1) / 2.0;
    bytes += 2.0 * 8.0 * (panel + (double)s.nblk * s.nb * s.nb);
    flops += 2.0 * 2.0 * (panel + diag);
  }
  out->f_apply_bytes = bytes;
  out->f_apply_flops = flops;
  out->factor_ms_total = c->factor_ms;
  out->factor_launches = c->factor_launches;
  out->kernel_launches = c->launches;
  out->schur_ms_total = c->g_ms;
  out->schur_launches = c->g_launches;
  out->schur_flops_total = c->g_flops;
  out->schur_bytes_total = c->g_bytes;
  out->inner_ms_total = c->inner_ms;
  out->inner_iterations = c->inner_its;
  out->inner_body_runs = c->inner_runs;
  return TFETI_OK;
}

int tfeti_timing_reset(tfeti_ctx* c, int32_t enable_events) {
  if (!c) return TFETI_ERR_ARG;
  collect_events(c);
  c->events = enable_events != 0;
  c->f_ms = c->factor_ms = 0.0;
  c->f_launches = c->factor_launches = c->launches = 0;
  c->g_ms = c->g_flops = c->g_bytes = 0.0;
  c->g_launches = 0;
  c->inner_ms = 0.0;
  c->inner_its = c->inner_runs = 0;
  return TFETI_OK;
}

}  // extern "C"
