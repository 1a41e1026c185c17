// Host analysis of the batched Newton-Raphson solver (Alg. 2): elimination
// order, filled block pattern, elimination-tree levels and the update lists
// the GPU factorisation walks.  Plain C++, no CUDA call.
#include <string.h>

#include <algorithm>
#include <functional>
#include <queue>
#include <utility>
#include <vector>

#include "dpf_nr.h"

namespace dpf {

int nr_symbolic(const dpf_ybus* y, int64_t max_pairs, NrSymbolic* s) {
  const int n = y->n;
  s->n = n;
  // graph of Y_bus (off-diagonal pattern), internal bus order, sorted lists
  std::vector<std::vector<int32_t>> adj(n);
  for (int i = 0; i < n; ++i)
    for (int p = y->irow_ptr[i]; p < y->irow_ptr[i + 1]; ++p)
      if (y->icol[p] != i) adj[i].push_back(y->icol[p]);
  for (auto& a : adj) std::sort(a.begin(), a.end());

  // Minimum degree on the elimination graph: eliminate a live vertex of
  // least degree (ties: lowest index), turning its live neighbours into a
  // clique.  Its neighbours at that moment are the off-diagonal pattern of
  // its row of U (and column of L).
  s->order.assign(n, 0);
  s->rank.assign(n, 0);
  std::vector<std::vector<int32_t>> nb_at(n);  // live neighbours when eliminated (bus ids)
  std::vector<char> gone(n, 0);
  using QE = std::pair<int, int>;
  std::priority_queue<QE, std::vector<QE>, std::greater<QE>> pq;
  for (int i = 0; i < n; ++i) pq.push({(int)adj[i].size(), i});
  std::vector<int32_t> merged;
  for (int r = 0; r < n;) {
    const QE top = pq.top();
    pq.pop();
    const int v = top.second;
    if (gone[v] || top.first != (int)adj[v].size()) continue;  // stale entry
    gone[v] = 1;
    s->order[r] = v;
    s->rank[v] = r;
    ++r;
    const std::vector<int32_t>& nb = adj[v];
    for (int u : nb) {
      merged.clear();
      std::set_union(adj[u].begin(), adj[u].end(), nb.begin(), nb.end(), std::back_inserter(merged));
      merged.erase(std::remove_if(merged.begin(), merged.end(), [&](int w) { return w == u || w == v; }),
                   merged.end());
      adj[u].swap(merged);
      pq.push({(int)adj[u].size(), u});
    }
    nb_at[v] = nb;
    std::vector<int32_t>().swap(adj[v]);
  }

  // U pattern of every row in elimination steps, sorted
  std::vector<std::vector<int32_t>> up(n);
  for (int r = 0; r < n; ++r) {
    for (int u : nb_at[s->order[r]]) up[r].push_back(s->rank[u]);
    std::sort(up[r].begin(), up[r].end());
    std::vector<int32_t>().swap(nb_at[s->order[r]]);
  }
  // L pattern: row r has column c < r wherever r is in U row c
  std::vector<std::vector<int32_t>> low(n);
  for (int c = 0; c < n; ++c)
    for (int r : up[c]) low[r].push_back(c);  // c ascending: sorted

  // positions, row-major
  s->row_ptr.assign(n + 1, 0);
  for (int r = 0; r < n; ++r) s->row_ptr[r + 1] = s->row_ptr[r] + (int)low[r].size() + 1 + (int)up[r].size();
  const int64_t npos = s->row_ptr[n];
  s->col.resize(npos);
  s->diag.resize(n);
  for (int r = 0; r < n; ++r) {
    int q = s->row_ptr[r];
    for (int c : low[r]) s->col[q++] = c;
    s->diag[r] = q;
    s->col[q++] = r;
    for (int c : up[r]) s->col[q++] = c;
  }
  auto pos = [&](int r, int c) -> int {
    const int32_t* b = s->col.data() + s->row_ptr[r];
    const int32_t* e = s->col.data() + s->row_ptr[r + 1];
    const int32_t* it = std::lower_bound(b, e, c);
    return (it != e && *it == c) ? (int)(it - s->col.data()) : -1;
  };

  // Y_bus entries: every one lies in the filled pattern
  s->ymap.assign(npos, -1);
  for (int i = 0; i < n; ++i)
    for (int p = y->irow_ptr[i]; p < y->irow_ptr[i + 1]; ++p) {
      const int q = pos(s->rank[i], s->rank[y->icol[p]]);
      if (q < 0) return fail(DPF_E_INVALID, "Newton analysis: Y_bus entry outside the filled pattern");
      s->ymap[q] = p;
    }

  // elimination tree (parent = first U column) and its heights
  s->level.assign(n, 0);
  for (int c = 0; c < n; ++c)
    if (!up[c].empty()) {
      const int p = up[c][0];
      s->level[p] = std::max(s->level[p], s->level[c] + 1);
    }
  int nl = 0;
  for (int r = 0; r < n; ++r) nl = std::max(nl, s->level[r] + 1);
  s->n_levels = n ? nl : 0;

  // Update lists.  Left-looking: position (i, j) with pivot p = min(i, j)
  // receives -L(i,k) U(k,j) from every earlier pivot k whose U row holds
  // both i and j; all such k are descendants of p in the tree (lower levels).
  std::vector<int64_t> cnt(npos + 1, 0);
  int64_t total = 0;
  for (int k = 0; k < n; ++k) {
    const int64_t d = (int64_t)up[k].size();
    total += d * d;
    if (total > max_pairs)
      return fail(DPF_E_UNSUPPORTED, "Newton analysis: %lld block updates exceed the limit %lld",
                  (long long)total, (long long)max_pairs);
    for (int i : up[k])
      for (int j : up[k]) cnt[pos(i, j) + 1] += 1;
  }
  for (int64_t q = 0; q < npos; ++q) cnt[q + 1] += cnt[q];
  s->pairs.assign(2 * (size_t)total, 0);
  std::vector<int64_t> cur(cnt.begin(), cnt.end() - 1);
  for (int k = 0; k < n; ++k)
    for (int i : up[k]) {
      const int lik = pos(i, k);
      for (int j : up[k]) {
        const int64_t q = cur[pos(i, j)]++;
        s->pairs[2 * q] = lik;
        s->pairs[2 * q + 1] = pos(k, j);
      }
    }

  // targets by pivot level, then pivot, then position
  std::vector<std::vector<int32_t>> by_level(s->n_levels);
  for (int r = 0; r < n; ++r) by_level[s->level[r]].push_back(r);
  s->lvl_ptr.assign(s->n_levels + 1, 0);
  s->targets.clear();
  s->targets.reserve(8 * (size_t)npos);
  s->rlvl_ptr.assign(s->n_levels + 1, 0);
  s->rows.clear();
  for (int l = 0; l < s->n_levels; ++l) {
    for (int p : by_level[l]) {
      const int dq = s->diag[p];
      const int32_t rw[4] = {p, dq + 1, s->row_ptr[p + 1], 0};
      s->rows.insert(s->rows.end(), rw, rw + 4);
      auto add = [&](int q, int kind) {
        const int32_t t[8] = {q, (int32_t)cnt[q], (int32_t)cnt[q + 1], kind,
                              kind == NR_DIAG ? s->row_ptr[p] : dq, (int32_t)cnt[dq], (int32_t)cnt[dq + 1], p};
        s->targets.insert(s->targets.end(), t, t + 8);
      };
      add(dq, NR_DIAG);
      for (int i : up[p]) add(pos(i, p), NR_L);
      for (int j : up[p]) add(pos(p, j), NR_U);
    }
    s->lvl_ptr[l + 1] = (int32_t)(s->targets.size() / 8);
    s->rlvl_ptr[l + 1] = (int32_t)(s->rows.size() / 4);
  }
  if ((int64_t)s->targets.size() / 8 != npos) return fail(DPF_E_INVALID, "Newton analysis: target count");
  return DPF_OK;
}

}  // namespace dpf

using namespace dpf;

// Default limit on the update lists of the host analysis (8 bytes each).
static const int64_t kMaxPairs = (int64_t)1 << 28;

extern "C" int dpf_nr_analyze(const dpf_ybus* y, int64_t* n_pos, int64_t* n_pairs, int32_t* n_levels) {
  clear_error();
  if (!y) return fail(DPF_E_INVALID, "dpf_nr_analyze: NULL Y_bus");
  NrSymbolic s;
  const int rc = nr_symbolic(y, kMaxPairs, &s);
  if (rc != DPF_OK) return rc;
  if (n_pos) *n_pos = s.row_ptr[s.n];
  if (n_pairs) *n_pairs = (int64_t)s.pairs.size() / 2;
  if (n_levels) *n_levels = s.n_levels;
  return DPF_OK;
}

extern "C" int dpf_nr_pattern(const dpf_ybus* y, int32_t* order, int32_t* row_ptr, int32_t* col, int32_t* level) {
  clear_error();
  if (!y) return fail(DPF_E_INVALID, "dpf_nr_pattern: NULL Y_bus");
  NrSymbolic s;
  const int rc = nr_symbolic(y, kMaxPairs, &s);
  if (rc != DPF_OK) return rc;
  const int n = s.n;
  if (order)
    for (int r = 0; r < n; ++r) order[r] = y->perm[s.order[r]];  // user bus index
  if (row_ptr) memcpy(row_ptr, s.row_ptr.data(), (size_t)(n + 1) * 4);
  if (col) memcpy(col, s.col.data(), (size_t)s.row_ptr[n] * 4);
  if (level) memcpy(level, s.level.data(), (size_t)n * 4);
  return DPF_OK;
}
