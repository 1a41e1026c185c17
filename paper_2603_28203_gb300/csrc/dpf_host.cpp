// Host-only part of libdpf: grid validation, Y_bus assembly in CSR, bridge
// detection for N-1 outages, and the locality ordering of buses used on the
// device.  No CUDA call is made here, so all of it runs without a GPU.
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <queue>
#include <set>
#include <utility>

#include "dpf_internal.h"

namespace dpf {

static thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

void clear_error() { g_err.clear(); }

// Branch pi-model (the MATPOWER branch model the paper's Eq. powerbalance
// footnote refers to): y_s = 1/(r + jx) = (r - jx)/(r^2 + x^2), charging
// b_ch split half to each end, ideal transformer of ratio tap at the from-bus.
// out = {Re y_ff, Im y_ff, Re y_ft, Im y_ft, Re y_tt, Im y_tt}; y_tf = y_ft.
void branch_block(double r, double x, double b_ch, double tap, double out[6]) {
  const double tau = (tap == 0.0) ? 1.0 : tap;
  const double d = r * r + x * x;
  const double gs = r / d, bs = -x / d;
  const double t2 = tau * tau;
  out[0] = gs / t2;
  out[1] = (bs + 0.5 * b_ch) / t2;
  out[2] = -gs / tau;
  out[3] = -bs / tau;
  out[4] = gs;
  out[5] = bs + 0.5 * b_ch;
}

// Bridges by iterative Tarjan low-link (one DFS per component).
static void find_bridges(int n, const std::vector<int32_t>& f, const std::vector<int32_t>& t,
                         std::vector<uint8_t>& is_bridge) {
  const int m = (int)f.size();
  std::vector<int32_t> head(n + 1, 0), adj_v(2 * m), adj_e(2 * m);
  for (int e = 0; e < m; ++e) { head[f[e] + 1]++; head[t[e] + 1]++; }
  for (int i = 0; i < n; ++i) head[i + 1] += head[i];
  std::vector<int32_t> fill(head.begin(), head.end() - 1);
  for (int e = 0; e < m; ++e) {
    adj_v[fill[f[e]]] = t[e]; adj_e[fill[f[e]]++] = e;
    adj_v[fill[t[e]]] = f[e]; adj_e[fill[t[e]]++] = e;
  }
  is_bridge.assign(m, 0);
  std::vector<int32_t> disc(n, -1), low(n, 0), it(n, 0), pedge(n, -1);
  std::vector<int32_t> stack;
  int timer = 0;
  for (int root = 0; root < n; ++root) {
    if (disc[root] != -1) continue;
    disc[root] = low[root] = timer++;
    it[root] = head[root];
    stack.push_back(root);
    while (!stack.empty()) {
      const int u = stack.back();
      if (it[u] < head[u + 1]) {
        const int k = it[u]++;
        const int v = adj_v[k], e = adj_e[k];
        if (e == pedge[u]) continue;
        if (disc[v] == -1) {
          disc[v] = low[v] = timer++;
          pedge[v] = e;
          it[v] = head[v];
          stack.push_back(v);
        } else {
          low[u] = std::min(low[u], disc[v]);
        }
      } else {
        stack.pop_back();
        if (!stack.empty()) {
          const int p = stack.back();
          low[p] = std::min(low[p], low[u]);
          if (low[u] > disc[p]) is_bridge[pedge[u]] = 1;
        }
      }
    }
  }
}

// Reverse Cuthill-McKee ordering: BFS from a low-degree pseudo-peripheral
// bus, neighbours visited by increasing degree, order reversed.  Neighbouring
// buses get nearby indices, so the gathers of one CTA hit the same cache
// lines.  perm[new] = old.
static void rcm_order(int n, const std::vector<int32_t>& rp, const std::vector<int32_t>& col,
                      std::vector<int32_t>& perm) {
  std::vector<int32_t> deg(n);
  for (int i = 0; i < n; ++i) deg[i] = rp[i + 1] - rp[i];
  std::vector<uint8_t> seen(n, 0);
  perm.clear();
  perm.reserve(n);
  auto bfs_last = [&](int s, std::vector<int32_t>* order) {
    std::vector<int32_t> lev(n, -1);
    std::queue<int32_t> q;
    q.push(s);
    lev[s] = 0;
    int last = s;
    while (!q.empty()) {
      const int u = q.front();
      q.pop();
      last = u;
      if (order) order->push_back(u);
      std::vector<int32_t> nb;
      for (int p = rp[u]; p < rp[u + 1]; ++p)
        if (col[p] != u && lev[col[p]] == -1) nb.push_back(col[p]);
      std::sort(nb.begin(), nb.end(), [&](int a, int b) { return deg[a] != deg[b] ? deg[a] < deg[b] : a < b; });
      for (int v : nb) { lev[v] = lev[u] + 1; q.push(v); }
    }
    return last;
  };
  for (int s0 = 0; s0 < n; ++s0) {
    if (seen[s0]) continue;
    // one BFS to find a far bus of this component, then order from it
    const int s = bfs_last(s0, nullptr);
    std::vector<int32_t> comp;
    bfs_last(s, &comp);
    for (int v : comp) seen[v] = 1;
    std::reverse(comp.begin(), comp.end());
    perm.insert(perm.end(), comp.begin(), comp.end());
  }
}

static bool is_finite(double v) { return std::isfinite(v); }

}  // namespace dpf

using namespace dpf;

extern "C" int dpf_build_ybus_host(const dpf_grid* g, dpf_ybus** out) {
  clear_error();
  if (!g || !out) return fail(DPF_E_INVALID, "dpf_build_ybus_host: NULL argument");
  *out = nullptr;
  const int n = g->n_bus, m = g->n_branch;
  if (n < 1 || m < 0) return fail(DPF_E_INVALID, "n_bus must be >= 1 and n_branch >= 0 (got %d, %d)", n, m);
  if (!g->bus_type || !g->p_spec || !g->q_spec || !g->vm_set)
    return fail(DPF_E_INVALID, "bus arrays must not be NULL");
  if (m > 0 && (!g->f_bus || !g->t_bus || !g->r || !g->x || !g->b_ch || !g->tap))
    return fail(DPF_E_INVALID, "branch arrays must not be NULL");
  if (!is_finite(g->va_slack)) return fail(DPF_E_INVALID, "va_slack is not finite");
  int n_slack = 0, slack = -1, n_pv = 0, n_pq = 0;
  for (int i = 0; i < n; ++i) {
    const int ty = g->bus_type[i];
    if (ty == DPF_SLACK) { ++n_slack; slack = i; }
    else if (ty == DPF_PV) ++n_pv;
    else if (ty == DPF_PQ) ++n_pq;
    else return fail(DPF_E_INVALID, "bus %d has unknown type %d", i, ty);
    if (!is_finite(g->p_spec[i]) || !is_finite(g->q_spec[i]) || !is_finite(g->vm_set[i]))
      return fail(DPF_E_INVALID, "bus %d has a non-finite specified value", i);
    if (ty != DPF_PQ && !(g->vm_set[i] > 0.0))
      return fail(DPF_E_INVALID, "bus %d: |V| set-point must be > 0", i);
  }
  if (n_slack < 1) return fail(DPF_E_INVALID, "need a slack bus");
  std::set<std::pair<int, int>> pairs;
  for (int e = 0; e < m; ++e) {
    const int f = g->f_bus[e], t = g->t_bus[e];
    if (f < 0 || f >= n || t < 0 || t >= n || f == t)
      return fail(DPF_E_INVALID, "branch %d has invalid buses (%d, %d)", e, f, t);
    if (!is_finite(g->r[e]) || !is_finite(g->x[e]) || !is_finite(g->b_ch[e]) || !is_finite(g->tap[e]))
      return fail(DPF_E_INVALID, "branch %d has a non-finite parameter", e);
    if (g->r[e] * g->r[e] + g->x[e] * g->x[e] <= 0.0)
      return fail(DPF_E_INVALID, "branch %d has zero impedance", e);
    if (g->tap[e] < 0.0) return fail(DPF_E_INVALID, "branch %d has a negative tap", e);
    if (g->shift && g->shift[e] != 0.0)
      return fail(DPF_E_UNSUPPORTED, "branch %d: phase-shifting transformers are not supported", e);
    if (!pairs.insert({std::min(f, t), std::max(f, t)}).second)
      return fail(DPF_E_UNSUPPORTED, "branch %d is parallel to an earlier branch", e);
  }

  {  // a block-diagonal batch of grids (Sec. 4.2) has several islands: one slack each
    std::vector<int32_t> parent(n);
    for (int i = 0; i < n; ++i) parent[i] = i;
    auto find = [&](int v) {
      while (parent[v] != v) v = parent[v] = parent[parent[v]];
      return v;
    };
    for (int e = 0; e < m; ++e) parent[find(g->f_bus[e])] = find(g->t_bus[e]);
    std::vector<int32_t> slacks(n, 0);
    for (int i = 0; i < n; ++i)
      if (g->bus_type[i] == DPF_SLACK) slacks[find(i)]++;
    for (int i = 0; i < n; ++i)
      if (find(i) == i && slacks[i] != 1)
        return fail(DPF_E_INVALID, "each island needs exactly one slack bus (island of bus %d has %d)", i,
                    slacks[i]);
  }
  dpf_ybus* y = new (std::nothrow) dpf_ybus();
  if (!y) return fail(DPF_E_OOM, "out of host memory");
  y->n = n;
  y->m = m;
  y->n_pv = n_pv;
  y->n_pq = n_pq;
  y->m_loss = n_pv + 2 * n_pq;
  y->slack = slack;
  y->va_slack = g->va_slack;
  y->bus_type.assign(g->bus_type, g->bus_type + n);
  y->p_spec.assign(g->p_spec, g->p_spec + n);
  y->q_spec.assign(g->q_spec, g->q_spec + n);
  y->vm_set.assign(g->vm_set, g->vm_set + n);
  if (m > 0) {
    y->f_bus.assign(g->f_bus, g->f_bus + m);
    y->t_bus.assign(g->t_bus, g->t_bus + m);
    y->r.assign(g->r, g->r + m);
    y->x.assign(g->x, g->x + m);
    y->b_ch.assign(g->b_ch, g->b_ch + m);
    y->tap.assign(g->tap, g->tap + m);
  }

  // CSR pattern: every diagonal plus (f,t) and (t,f) of every branch.
  std::vector<int32_t> cnt(n, 1);
  for (int e = 0; e < m; ++e) { cnt[y->f_bus[e]]++; cnt[y->t_bus[e]]++; }
  y->row_ptr.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) y->row_ptr[i + 1] = y->row_ptr[i] + cnt[i];
  const int nnz = y->row_ptr[n];
  y->nnz = nnz;
  y->col.assign(nnz, 0);
  y->ebr.assign(nnz, -1);
  {
    std::vector<int32_t> fill(y->row_ptr.begin(), y->row_ptr.end() - 1);
    for (int i = 0; i < n; ++i) { y->col[fill[i]] = i; y->ebr[fill[i]++] = -1; }
    for (int e = 0; e < m; ++e) {
      const int f = y->f_bus[e], t = y->t_bus[e];
      y->col[fill[f]] = t; y->ebr[fill[f]++] = e;
      y->col[fill[t]] = f; y->ebr[fill[t]++] = e;
    }
    for (int i = 0; i < n; ++i) {  // sort each row by column
      std::vector<std::pair<int32_t, int32_t>> row;
      for (int p = y->row_ptr[i]; p < y->row_ptr[i + 1]; ++p) row.push_back({y->col[p], y->ebr[p]});
      std::sort(row.begin(), row.end());
      for (int p = y->row_ptr[i], k = 0; p < y->row_ptr[i + 1]; ++p, ++k) {
        y->col[p] = row[k].first;
        y->ebr[p] = row[k].second;
      }
    }
  }
  y->dpos.assign(n, -1);
  for (int i = 0; i < n; ++i)
    for (int p = y->row_ptr[i]; p < y->row_ptr[i + 1]; ++p)
      if (y->col[p] == i) y->dpos[i] = p;
  // values: branch contributions summed in branch order
  y->val_re.assign(nnz, 0.0);
  y->val_im.assign(nnz, 0.0);
  for (int e = 0; e < m; ++e) {
    double blk[6];
    branch_block(y->r[e], y->x[e], y->b_ch[e], y->tap[e], blk);
    const int f = y->f_bus[e], t = y->t_bus[e];
    y->val_re[y->dpos[f]] += blk[0];
    y->val_im[y->dpos[f]] += blk[1];
    y->val_re[y->dpos[t]] += blk[4];
    y->val_im[y->dpos[t]] += blk[5];
    for (int p = y->row_ptr[f]; p < y->row_ptr[f + 1]; ++p)
      if (y->ebr[p] == e) { y->val_re[p] = blk[2]; y->val_im[p] = blk[3]; }
    for (int p = y->row_ptr[t]; p < y->row_ptr[t + 1]; ++p)
      if (y->ebr[p] == e) { y->val_re[p] = blk[2]; y->val_im[p] = blk[3]; }
  }
  find_bridges(n, y->f_bus, y->t_bus, y->bridge);

  // internal (device) order
  rcm_order(n, y->row_ptr, y->col, y->perm);
  y->iperm.assign(n, 0);
  for (int i = 0; i < n; ++i) y->iperm[y->perm[i]] = i;
  y->irow_ptr.assign(n + 1, 0);
  y->icol.assign(nnz, 0);
  y->iebr.assign(nnz, -1);
  y->ival_re.assign(nnz, 0.0);
  y->ival_im.assign(nnz, 0.0);
  y->idpos.assign(n, -1);
  for (int ni = 0; ni < n; ++ni) {
    const int oi = y->perm[ni];
    std::vector<std::pair<int32_t, int32_t>> row;  // (new col, old position)
    for (int p = y->row_ptr[oi]; p < y->row_ptr[oi + 1]; ++p) row.push_back({y->iperm[y->col[p]], p});
    std::sort(row.begin(), row.end());
    y->irow_ptr[ni + 1] = y->irow_ptr[ni] + (int)row.size();
    for (size_t k = 0; k < row.size(); ++k) {
      const int q = y->irow_ptr[ni] + (int)k;
      y->icol[q] = row[k].first;
      y->iebr[q] = y->ebr[row[k].second];
      y->ival_re[q] = y->val_re[row[k].second];
      y->ival_im[q] = y->val_im[row[k].second];
      if (row[k].first == ni) y->idpos[ni] = q;
    }
  }
  // Padded rows for the shared-memory SpMV: each row's entries rounded up to
  // a multiple of 4 by zero-weight entries on the row's own bus, so the
  // device loop runs whole groups of four with no per-entry predicate.
  // ippos maps a padded slot to its CSR position, or holds -(row + 1).
  y->iprow_ptr.assign(n + 1, 0);
  for (int i = 0; i < n; ++i)
    y->iprow_ptr[i + 1] = y->iprow_ptr[i] + ((y->irow_ptr[i + 1] - y->irow_ptr[i] + 3) & ~3);
  y->ippos.assign(y->iprow_ptr[n], 0);
  for (int i = 0; i < n; ++i) {
    int q = y->iprow_ptr[i];
    for (int p = y->irow_ptr[i]; p < y->irow_ptr[i + 1]; ++p) y->ippos[q++] = p;
    for (; q < y->iprow_ptr[i + 1]; ++q) y->ippos[q] = -(i + 1);
  }
  *out = y;
  return DPF_OK;
}

extern "C" int dpf_ybus_info(const dpf_ybus* y, int32_t* n_bus, int32_t* n_branch, int32_t* nnz) {
  if (!y) return fail(DPF_E_INVALID, "dpf_ybus_info: NULL handle");
  if (n_bus) *n_bus = y->n;
  if (n_branch) *n_branch = y->m;
  if (nnz) *nnz = y->nnz;
  return DPF_OK;
}

extern "C" int dpf_ybus_export(const dpf_ybus* y, int32_t* row_ptr, int32_t* col, double* val_re,
                               double* val_im) {
  if (!y) return fail(DPF_E_INVALID, "dpf_ybus_export: NULL handle");
  if (row_ptr) std::copy(y->row_ptr.begin(), y->row_ptr.end(), row_ptr);
  if (col) std::copy(y->col.begin(), y->col.end(), col);
  if (val_re) std::copy(y->val_re.begin(), y->val_re.end(), val_re);
  if (val_im) std::copy(y->val_im.begin(), y->val_im.end(), val_im);
  return DPF_OK;
}

extern "C" int dpf_ybus_bridges(const dpf_ybus* y, uint8_t* bridge) {
  if (!y || (!bridge && y->m > 0)) return fail(DPF_E_INVALID, "dpf_ybus_bridges: NULL argument");
  std::copy(y->bridge.begin(), y->bridge.end(), bridge);
  return DPF_OK;
}

extern "C" const char* dpf_last_error(void) { return dpf::g_err.c_str(); }

extern "C" const char* dpf_status_str(int s) {
  switch (s) {
    case DPF_OK: return "ok";
    case DPF_E_INVALID: return "invalid argument";
    case DPF_E_ISLANDED: return "outage islands the grid";
    case DPF_E_CUDA: return "CUDA error";
    case DPF_E_OOM: return "out of memory";
    case DPF_E_UNSUPPORTED: return "unsupported grid feature";
    case DPF_E_STATE: return "call out of order";
    default: return "unknown status";
  }
}

extern "C" void dpf_default_opts(dpf_solve_opts* o) {
  if (!o) return;
  o->lr = 1e-2;
  o->beta1 = 0.979;
  o->beta2 = 0.963;
  o->eps = 1e-8;
  o->optimizer = DPF_OPT_ADAM;
  o->momentum = 0.0;
  o->alpha = 0.99;
  o->sched = DPF_SCHED_PLATEAU;
  o->factor = 0.547;
  o->threshold = 0.0673;
  o->min_lr = 0.0;
  o->patience = 41;
  o->cooldown = 97;
  o->step_size = 100;
  o->gamma = 0.773;
  o->max_iter = 1000;
  o->check_every = 25;
  o->tol = 1e-6;
  o->gate = 1e-3;
  o->flat_start = 1;
  o->precision = DPF_FP32;
  o->lanes = 0;
  o->warps = 0;
  o->row_blocks = 0;
  o->use_graph = 1;
  o->pair_cases = 1;  /* forward pass two cases per thread */
  o->stage_v = 0;
  o->pdl = 1;
  o->plain = 0;
  o->dc_start = 0;
  o->stage_y = 0;
  o->dc_tol = 1e-10;
  o->dc_max_iter = 10000;
  o->refresh_every = 0;
}
