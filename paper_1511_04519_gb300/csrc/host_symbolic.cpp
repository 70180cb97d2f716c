// Host setup, part 1: fill-reducing ordering and supernodal symbolic analysis
// of the SPD matrices that Alg. 2 factors once, X1 = C + gamma G and G: for
// R-MATEX X1 = C + gamma G (Sec. 3.3.2), and G itself for F, P and the DC
// state (Eq. 6).  C is diagonal, so both share one sparsity pattern and one
// symbolic analysis.
//
// Ordering: recursive nested dissection with breadth-first level-structure
// separators (no coordinates are needed, only the graph of G).
#include <algorithm>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace matex {

namespace {

struct Graph {
  int64_t n;
  std::vector<int64_t> ptr;
  std::vector<int32_t> adj;
};

Graph build_graph(const CsrSym& A) {
  Graph g;
  g.n = A.n;
  g.ptr.assign(A.n + 1, 0);
  for (int64_t i = 0; i < A.n; ++i) {
    int64_t cnt = 0;
    for (int64_t p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p)
      if (A.col[p] != i) ++cnt;
    g.ptr[i + 1] = g.ptr[i] + cnt;
  }
  g.adj.resize(g.ptr[A.n]);
  for (int64_t i = 0; i < A.n; ++i) {
    int64_t q = g.ptr[i];
    for (int64_t p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p)
      if (A.col[p] != i) g.adj[q++] = A.col[p];
  }
  return g;
}

struct NdState {
  const Graph* g;
  std::vector<int32_t> tag;     // subset membership tag per node
  std::vector<int32_t> level;   // BFS level per node
  std::vector<int32_t> queue;
  int32_t next_tag = 1;
  std::vector<int32_t>* out;
};

// BFS from root over nodes carrying tag t; fills st.queue with the visit order
// and st.level; returns the number of levels.
int32_t bfs(NdState& st, int32_t root, int32_t t) {
  const Graph& g = *st.g;
  st.queue.clear();
  st.queue.push_back(root);
  st.level[root] = 0;
  int32_t lvl_tag = -t;  // visited nodes carry -t while the BFS runs
  st.tag[root] = lvl_tag;
  size_t head = 0;
  int32_t maxl = 0;
  while (head < st.queue.size()) {
    int32_t v = st.queue[head++];
    int32_t lv = st.level[v];
    for (int64_t p = g.ptr[v]; p < g.ptr[v + 1]; ++p) {
      int32_t u = g.adj[p];
      if (st.tag[u] == t) {
        st.tag[u] = lvl_tag;
        st.level[u] = lv + 1;
        maxl = std::max(maxl, lv + 1);
        st.queue.push_back(u);
      }
    }
  }
  for (int32_t v : st.queue) st.tag[v] = t;  // restore membership
  return maxl + 1;
}

const int32_t kLeaf = 48;

void nd_rec(NdState& st, std::vector<int32_t>& nodes) {
  if ((int64_t)nodes.size() <= kLeaf) {
    st.out->insert(st.out->end(), nodes.begin(), nodes.end());
    return;
  }
  const Graph& g = *st.g;
  int32_t t = st.next_tag++;
  for (int32_t v : nodes) st.tag[v] = t;
  // pseudo-peripheral root: repeat BFS from the last-visited node
  int32_t root = nodes[0];
  int32_t nl = bfs(st, root, t);
  if (st.queue.size() < nodes.size()) {
    // disconnected subset: order the reached component, then the rest
    std::vector<int32_t> comp(st.queue.begin(), st.queue.end());
    int32_t ct = st.next_tag++;
    for (int32_t v : comp) st.tag[v] = ct;
    std::vector<int32_t> rest;
    rest.reserve(nodes.size() - comp.size());
    for (int32_t v : nodes)
      if (st.tag[v] == t) rest.push_back(v);
    nodes.clear();
    nodes.shrink_to_fit();
    nd_rec(st, comp);
    nd_rec(st, rest);
    return;
  }
  for (int it = 0; it < 4; ++it) {
    int32_t cand = st.queue.back();
    int32_t nl2 = bfs(st, cand, t);
    if (nl2 <= nl && it > 0) {
      if (nl2 < nl) bfs(st, root, t);
      break;
    }
    root = cand;
    nl = nl2;
  }
  if (nl < 3) {  // no proper separator (clique-like); keep as a leaf block
    st.out->insert(st.out->end(), nodes.begin(), nodes.end());
    return;
  }
  std::vector<int64_t> cnt(nl, 0);
  for (int32_t v : st.queue) cnt[st.level[v]]++;
  int64_t half = (int64_t)nodes.size() / 2, acc = 0;
  int32_t mid = 1;
  for (int32_t l = 0; l < nl; ++l) {
    if (acc + cnt[l] > half) { mid = l; break; }
    acc += cnt[l];
  }
  mid = std::max(1, std::min(mid, nl - 2));
  std::vector<int32_t> A, B, S;
  for (int32_t v : st.queue) {
    int32_t lv = st.level[v];
    if (lv < mid) A.push_back(v);
    else if (lv > mid) B.push_back(v);
    else {
      // a separator node with no neighbour beyond the separator joins A
      bool touches_b = false;
      for (int64_t p = g.ptr[v]; p < g.ptr[v + 1]; ++p) {
        int32_t u = g.adj[p];
        if (st.tag[u] == t && st.level[u] == mid + 1) { touches_b = true; break; }
      }
      if (touches_b) S.push_back(v); else A.push_back(v);
    }
  }
  nodes.clear();
  nodes.shrink_to_fit();
  nd_rec(st, A);
  nd_rec(st, B);
  st.out->insert(st.out->end(), S.begin(), S.end());
}

}  // namespace

std::string nested_dissection(const CsrSym& A, std::vector<int32_t>& perm) {
  Graph g = build_graph(A);
  NdState st;
  st.g = &g;
  st.tag.assign(A.n, 0);
  st.level.assign(A.n, 0);
  std::vector<int32_t> out;
  out.reserve(A.n);
  st.out = &out;
  std::vector<int32_t> all(A.n);
  std::iota(all.begin(), all.end(), 0);
  nd_rec(st, all);
  if ((int64_t)out.size() != A.n) return "nested dissection lost nodes";
  perm.swap(out);
  return "";
}

std::string symbolic_analysis(const CsrSym& A, const std::vector<int32_t>& nd_perm,
                              int32_t max_width, Symbolic& S) {
  const int64_t n = A.n;
  std::vector<int32_t> ip(n);
  for (int64_t k = 0; k < n; ++k) ip[nd_perm[k]] = (int32_t)k;
  // lower pattern by rows (new numbering): row j lists k < j with A[j,k] != 0
  auto row_lower = [&](const std::vector<int32_t>& perm, const std::vector<int32_t>& iperm,
                       std::vector<int64_t>& rp, std::vector<int32_t>& ci) {
    rp.assign(n + 1, 0);
    for (int64_t j = 0; j < n; ++j) {
      int32_t o = perm[j];
      int64_t c = 0;
      for (int64_t p = A.rowptr[o]; p < A.rowptr[o + 1]; ++p)
        if (iperm[A.col[p]] < j) ++c;
      rp[j + 1] = rp[j] + c;
    }
    ci.resize(rp[n]);
    for (int64_t j = 0; j < n; ++j) {
      int32_t o = perm[j];
      int64_t q = rp[j];
      for (int64_t p = A.rowptr[o]; p < A.rowptr[o + 1]; ++p) {
        int32_t k = iperm[A.col[p]];
        if (k < j) ci[q++] = k;
      }
    }
  };
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  row_lower(nd_perm, ip, rp, ci);
  // elimination tree (Liu, with path compression)
  std::vector<int32_t> parent(n, -1), anc(n, -1);
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t p = rp[j]; p < rp[j + 1]; ++p) {
      int32_t i = ci[p];
      while (i != -1 && i < j) {
        int32_t nx = anc[i];
        anc[i] = (int32_t)j;
        if (nx == -1) { parent[i] = (int32_t)j; break; }
        i = nx;
      }
    }
  }
  // postorder of the etree (children visited in increasing order)
  std::vector<int32_t> head(n, -1), nxt(n, -1), post;
  post.reserve(n);
  for (int64_t j = n - 1; j >= 0; --j)
    if (parent[j] != -1) { nxt[j] = head[parent[j]]; head[parent[j]] = (int32_t)j; }
  std::vector<int32_t> stk;
  for (int64_t r = 0; r < n; ++r) {
    if (parent[r] != -1) continue;
    stk.push_back((int32_t)r);
    while (!stk.empty()) {
      int32_t v = stk.back();
      if (head[v] != -1) {
        int32_t c = head[v];
        head[v] = nxt[c];
        stk.push_back(c);
      } else {
        post.push_back(v);
        stk.pop_back();
      }
    }
  }
  if ((int64_t)post.size() != n) return "etree postorder failed";
  S.n = n;
  S.perm.resize(n);
  S.iperm.resize(n);
  for (int64_t k = 0; k < n; ++k) S.perm[k] = nd_perm[post[k]];
  for (int64_t k = 0; k < n; ++k) S.iperm[S.perm[k]] = (int32_t)k;
  // everything again in the final numbering
  row_lower(S.perm, S.iperm, rp, ci);
  std::fill(parent.begin(), parent.end(), -1);
  std::fill(anc.begin(), anc.end(), -1);
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t p = rp[j]; p < rp[j + 1]; ++p) {
      int32_t i = ci[p];
      while (i != -1 && i < j) {
        int32_t nx = anc[i];
        anc[i] = (int32_t)j;
        if (nx == -1) { parent[i] = (int32_t)j; break; }
        i = nx;
      }
    }
  }
  // column counts through row subtrees
  std::vector<int64_t> cc(n, 1);
  std::vector<int32_t> mark(n, -1);
  for (int64_t i = 0; i < n; ++i) {
    mark[i] = (int32_t)i;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int32_t k = ci[p];
      while (k != -1 && mark[k] != i) {
        cc[k]++;
        mark[k] = (int32_t)i;
        k = parent[k];
      }
    }
  }
  // the fill of L itself: what the method needs, before amalgamation pads it
  S.nnz_L_exact = 0;
  for (int64_t j = 0; j < n; ++j) S.nnz_L_exact += cc[j] - 1;
  // supernodes: j joins j-1 when parent[j-1] == j and the structures nest
  S.sup_first.clear();
  for (int64_t j = 0; j < n; ++j) {
    bool start = (j == 0) || parent[j - 1] != j || cc[j - 1] != cc[j] + 1 ||
                 (j - S.sup_first.back()) >= max_width;
    if (start) S.sup_first.push_back((int32_t)j);
  }
  S.nsup = (int32_t)S.sup_first.size();
  S.sup_first.push_back((int32_t)n);
  std::vector<int32_t> col2sup(n);
  for (int32_t s = 0; s < S.nsup; ++s)
    for (int32_t j = S.sup_first[s]; j < S.sup_first[s + 1]; ++j) col2sup[j] = s;
  // row structures: own columns, then A's rows below plus children's rows
  std::vector<std::vector<int32_t>> offrows(S.nsup);
  std::vector<std::vector<int32_t>> kids(S.nsup);
  // column pattern (lower) of A in the final numbering, from the row lists
  std::vector<int64_t> cp(n + 1, 0);
  for (int64_t p = 0; p < rp[n]; ++p) cp[ci[p] + 1]++;
  for (int64_t j = 0; j < n; ++j) cp[j + 1] += cp[j];
  std::vector<int32_t> cr(rp[n]);
  {
    std::vector<int64_t> fill(cp.begin(), cp.end() - 1);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) cr[fill[ci[p]]++] = (int32_t)i;
  }
  std::fill(mark.begin(), mark.end(), -1);
  S.sup_parent.assign(S.nsup, -1);
  for (int32_t s = 0; s < S.nsup; ++s) {
    int32_t f = S.sup_first[s], l = S.sup_first[s + 1];
    std::vector<int32_t>& rows = offrows[s];
    for (int32_t j = f; j < l; ++j)
      for (int64_t p = cp[j]; p < cp[j + 1]; ++p) {
        int32_t i = cr[p];
        if (i >= l && mark[i] != s) { mark[i] = s; rows.push_back(i); }
      }
    for (int32_t c : kids[s])
      for (int32_t i : offrows[c])
        if (i >= l && mark[i] != s) { mark[i] = s; rows.push_back(i); }
    std::sort(rows.begin(), rows.end());
    if (!rows.empty()) {
      int32_t par = col2sup[rows[0]];
      S.sup_parent[s] = par;
      kids[par].push_back(s);
    }
    if ((int64_t)rows.size() + (l - f) != cc[f]) return "supernode structure mismatch";
  }
  // Relaxed amalgamation: a supernode joins its parent when it is the parent's
  // last child (adjacent columns) and the explicit zeros of the merged dense
  // block stay small; fewer, wider supernodes mean fewer tree levels and
  // denser panels for the solves.  Thresholds: merged width <= 4 always;
  // <= 16 with < 80% zeros; <= 48 with < 10%; otherwise < 5%.
  {
    const int32_t ns = S.nsup;
    std::vector<int32_t> first(ns), last(ns);
    std::vector<int64_t> zeros(ns, 0);
    std::vector<char> gone(ns, 0);
    for (int32_t t = 0; t < ns; ++t) {
      first[t] = S.sup_first[t];
      last[t] = S.sup_first[t + 1];
    }
    for (int32_t t = 0; t < ns; ++t) {
      const int32_t par = S.sup_parent[t];
      if (par < 0 || last[t] != first[par]) continue;
      const int64_t ws = last[t] - first[t], wp = last[par] - first[par];
      const int64_t rt = (int64_t)offrows[t].size(), rpar = (int64_t)offrows[par].size();
      const int64_t w = ws + wp;
      if (w > max_width) continue;
      const int64_t z = zeros[t] + zeros[par] + ws * (wp + rpar - rt);
      const double dense = (double)w * (double)(w + 1) / 2.0 + (double)w * (double)rpar;
      const double zf = (double)z / dense;
      const bool merge = w <= 4 || (w <= 16 && zf < 0.8) || (w <= 48 && zf < 0.1) || zf < 0.05;
      if (!merge) continue;
      first[par] = first[t];
      zeros[par] = z;
      gone[t] = 1;
    }
    std::vector<int32_t> keep;
    for (int32_t t = 0; t < ns; ++t)
      if (!gone[t]) keep.push_back(t);
    std::sort(keep.begin(), keep.end(), [&](int32_t a, int32_t b) { return first[a] < first[b]; });
    std::vector<std::vector<int32_t>> rows2(keep.size());
    S.sup_first.assign(keep.size() + 1, 0);
    for (size_t k = 0; k < keep.size(); ++k) {
      S.sup_first[k] = first[keep[k]];
      rows2[k].swap(offrows[keep[k]]);
    }
    S.nsup = (int32_t)keep.size();
    S.sup_first[S.nsup] = (int32_t)n;
    for (int32_t t = 0; t < S.nsup; ++t)
      for (int32_t j = S.sup_first[t]; j < S.sup_first[t + 1]; ++j) col2sup[j] = t;
    S.sup_parent.assign(S.nsup, -1);
    for (int32_t t = 0; t < S.nsup; ++t)
      if (!rows2[t].empty()) S.sup_parent[t] = col2sup[rows2[t][0]];
    offrows.swap(rows2);
  }
  S.sup_rowptr.assign(S.nsup + 1, 0);
  S.pan_off.assign(S.nsup + 1, 0);
  S.nnz_L = 0;
  S.flops_factor = 0;
  for (int32_t s = 0; s < S.nsup; ++s) {
    int64_t w = S.sup_first[s + 1] - S.sup_first[s];
    int64_t r = (int64_t)offrows[s].size();
    S.sup_rowptr[s + 1] = S.sup_rowptr[s] + w + r;
    S.pan_off[s + 1] = S.pan_off[s] + (w + r) * w;
    S.nnz_L += w * (w - 1) / 2 + w * r;
    double nr = (double)(w + r);
    S.flops_factor += (double)w * nr * nr;  // order of the partial factorisation cost
  }
  S.sup_rows.resize(S.sup_rowptr[S.nsup]);
  for (int32_t s = 0; s < S.nsup; ++s) {
    int64_t q = S.sup_rowptr[s];
    for (int32_t j = S.sup_first[s]; j < S.sup_first[s + 1]; ++j) S.sup_rows[q++] = j;
    for (int32_t i : offrows[s]) S.sup_rows[q++] = i;
  }
  // levels of the supernodal tree, leaves first
  std::vector<int32_t> lev(S.nsup, 0);
  int32_t maxlev = 0;
  for (int32_t s = 0; s < S.nsup; ++s) {
    int32_t p = S.sup_parent[s];
    if (p >= 0) lev[p] = std::max(lev[p], lev[s] + 1);
    maxlev = std::max(maxlev, lev[s]);
  }
  S.level_ptr.assign(maxlev + 2, 0);
  for (int32_t s = 0; s < S.nsup; ++s) S.level_ptr[lev[s] + 1]++;
  for (int32_t l = 0; l <= maxlev; ++l) S.level_ptr[l + 1] += S.level_ptr[l];
  S.level_sups.resize(S.nsup);
  {
    std::vector<int32_t> fill(S.level_ptr.begin(), S.level_ptr.end() - 1);
    for (int32_t s = 0; s < S.nsup; ++s) S.level_sups[fill[lev[s]]++] = s;
  }
  return "";
}

}  // namespace matex
