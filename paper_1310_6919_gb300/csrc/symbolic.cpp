// Host symbolic analysis (Sec. 2.1 "permute ... generate a chordal graph ... extract cliques",
// Sec. 3.1 "row/column sets of CHOLMOD supernodes have the running intersection property").
// Everything here is integer work done once before the main loop.
#include "symbolic.h"

#include <algorithm>
#include <cstdint>
#include <array>
#include <map>
#include <numeric>
#include <set>
#include <sstream>

namespace mcsdp {
namespace {

// Binary min-heap of the live vertices keyed by (degree, vertex), with each vertex's position
// in the heap kept so that a degree change moves the vertex in place.  The key order is total,
// so the minimum is unique: the vertex of least degree, ties going to the smallest index.
class DegreeHeap {
 public:
  explicit DegreeHeap(const std::vector<int> &deg) : deg_(deg), h_(deg.size()), pos_(deg.size()) {
    const int n = (int)deg.size();
    for (int v = 0; v < n; ++v) h_[v] = pos_[v] = v;
    for (int i = n / 2 - 1; i >= 0; --i) down(i);
  }
  bool empty() const { return h_.empty(); }
  int pop() {
    const int v = h_[0];
    pos_[v] = -1;
    const int last = h_.back();
    h_.pop_back();
    if (!h_.empty()) {
      h_[0] = last;
      pos_[last] = 0;
      down(0);
    }
    return v;
  }
  void changed(int v) {  // deg[v] changed; v is still in the heap
    up(pos_[v]);
    down(pos_[v]);
  }

 private:
  bool less(int a, int b) const { return deg_[a] != deg_[b] ? deg_[a] < deg_[b] : a < b; }
  void up(int i) {
    const int v = h_[i];
    while (i > 0) {
      const int p = (i - 1) / 2;
      if (!less(v, h_[p])) break;
      h_[i] = h_[p];
      pos_[h_[i]] = i;
      i = p;
    }
    h_[i] = v;
    pos_[v] = i;
  }
  void down(int i) {
    const int v = h_[i], n = (int)h_.size();
    for (;;) {
      int c = 2 * i + 1;
      if (c >= n) break;
      if (c + 1 < n && less(h_[c + 1], h_[c])) ++c;
      if (!less(h_[c], v)) break;
      h_[i] = h_[c];
      pos_[h_[i]] = i;
      i = c;
    }
    h_[i] = v;
    pos_[v] = i;
  }
  const std::vector<int> &deg_;
  std::vector<int> h_, pos_;
};

// Exact minimum-degree ordering on the elimination graph (ties: smallest caller index).
// Returns the elimination order and, for each step, the neighbours at elimination time
// (= the row structure of that column of the Cholesky factor).  The candidates sit in a
// DegreeHeap, updated in place when an elimination changes a neighbour's degree.
// Up to MD_BITSET_N vertices the elimination graph is held as adjacency bitsets (n^2/8 bytes:
// 128 MiB at the bound): a step is then one word-wise OR per neighbour plus a popcount, instead
// of a merge of two sorted lists (the same graph, so the same order).  Once fill makes the
// neighbour sets dense (separator cliques of thousands of vertices in random sparse graphs) the
// merge costs O(|adj u| + |N|) per neighbour and step against O(n/64) for the OR, so the bitsets
// win by the clique size over 64.
constexpr int MD_BITSET_N = 32768;

void min_degree_bits(int n, const std::vector<std::vector<int>> &adj, std::vector<int> &order,
                     std::vector<std::vector<int>> &elim_struct) {
  const int W = (n + 63) / 64;
  std::vector<uint64_t> bits((size_t)n * W, 0);
  std::vector<int> deg(n);
  for (int v = 0; v < n; ++v) {
    uint64_t *b = bits.data() + (size_t)v * W;
    for (int u : adj[v]) b[u >> 6] |= 1ull << (u & 63);
    deg[v] = (int)adj[v].size();
  }
  DegreeHeap heap(deg);
  order.clear();
  order.reserve(n);
  elim_struct.assign(n, {});
  std::vector<uint64_t> nb(W);
  std::vector<int> nzw;  // words of nb that hold a neighbour
  nzw.reserve(W);
  int last = -1;         // the vertex eliminated in the previous step
  while (!heap.empty()) {
    const int v = heap.pop();
    order.push_back(v);
    uint64_t *bv = bits.data() + (size_t)v * W;
    std::vector<int> &N = elim_struct[v];  // ascending
    // After eliminating `last` with neighbours P, every u in P is adjacent to all of P \ {u}.
    // If v is in P with degree |P| - 1, its neighbours are exactly P \ {v} and each of them
    // already holds P \ {v} minus itself: eliminating v adds no fill, and the update reduces to
    // taking v out of their rows (one degree less each) -- the same graph and degrees the
    // general step below would produce, so the same order.  This is the common case inside a
    // supernode, where the general step's word-wise OR would add nothing.
    if (last >= 0) {
      const std::vector<int> &P = elim_struct[last];
      if (deg[v] == (int)P.size() - 1 && ((nb[v >> 6] >> (v & 63)) & 1)) {
        for (int u : P)
          if (u != v) N.push_back(u);
        nb[v >> 6] &= ~(1ull << (v & 63));  // nb becomes the bitset of N
        std::fill(bv, bv + W, 0ull);
        for (int u : N) {
          bits[(size_t)u * W + (v >> 6)] &= ~(1ull << (v & 63));
          deg[u] -= 1;
          heap.changed(u);
        }
        last = v;
        continue;
      }
    }
    last = v;
    std::copy(bv, bv + W, nb.begin());
    nzw.clear();
    for (int w = 0; w < W; ++w) {
      if (nb[w]) nzw.push_back(w);
      for (uint64_t x = nb[w]; x; x &= x - 1) N.push_back(w * 64 + __builtin_ctzll(x));
    }
    std::fill(bv, bv + W, 0ull);
    for (int u : N) {
      // adj[u] := (adj[u] ∪ N) \ {u, v}; deg[u] is the popcount of row u, so only the bits
      // that N adds are counted (v ∈ adj[u] drops out; u's own bit is held set meanwhile so
      // that it is never counted as new)
      uint64_t *bu = bits.data() + (size_t)u * W;
      const uint64_t ubit = 1ull << (u & 63);
      bu[v >> 6] &= ~(1ull << (v & 63));
      bu[u >> 6] |= ubit;
      int d = deg[u] - 1;
      for (int w : nzw) {
        const uint64_t add = nb[w] & ~bu[w];
        if (add) {
          bu[w] |= add;
          d += __builtin_popcountll(add);
        }
      }
      bu[u >> 6] &= ~ubit;
      if (d != deg[u]) {
        deg[u] = d;
        heap.changed(u);
      }
    }
  }
}

void min_degree(int n, std::vector<std::vector<int>> adj, std::vector<int> &order,
                std::vector<std::vector<int>> &elim_struct) {
  if (n <= MD_BITSET_N) {
    min_degree_bits(n, adj, order, elim_struct);
    return;
  }
  std::vector<int> deg(n);
  for (int v = 0; v < n; ++v) deg[v] = (int)adj[v].size();
  DegreeHeap heap(deg);
  order.clear();
  order.reserve(n);
  elim_struct.assign(n, {});
  std::vector<int> tmp;
  int last = -1;  // the vertex eliminated in the previous step
  while (!heap.empty()) {
    const int v = heap.pop();
    std::vector<int> N;
    N.swap(adj[v]);  // all live
    order.push_back(v);
    // the no-fill step of min_degree_bits: v's neighbours are exactly the previous step's
    // neighbours minus v, each already adjacent to all the others, so only v leaves their lists
    if (last >= 0) {
      const std::vector<int> &P = elim_struct[last];
      if (deg[v] == (int)P.size() - 1 && std::binary_search(P.begin(), P.end(), v)) {
        for (int u : N) {
          auto &a = adj[u];
          a.erase(std::lower_bound(a.begin(), a.end(), v));
          deg[u] = (int)a.size();
          heap.changed(u);
        }
        elim_struct[v] = std::move(N);
        last = v;
        continue;
      }
    }
    last = v;
    for (int u : N) {
      // adj[u] := (adj[u] ∪ N) \ {u, v}
      tmp.clear();
      const auto &a = adj[u];
      size_t i = 0, j = 0;
      while (i < a.size() || j < N.size()) {
        int x;
        if (j >= N.size() || (i < a.size() && a[i] < N[j])) x = a[i++];
        else if (i >= a.size() || N[j] < a[i]) x = N[j++];
        else { x = a[i]; ++i; ++j; }
        if (x != u && x != v) tmp.push_back(x);
      }
      adj[u].swap(tmp);
      if ((int)adj[u].size() != deg[u]) {
        deg[u] = (int)adj[u].size();
        heap.changed(u);
      }
    }
    elim_struct[v] = std::move(N);
  }
}

}  // namespace

std::string analyze(const ProblemData &P, const SymbolicOptions &o, Symbolic &S) {
  const int n = P.n, m = P.m;
  S = Symbolic();
  S.n = n;
  S.m = m;
  // ---- aggregate sparsity pattern (Sec. 1) ----
  std::vector<std::vector<int>> adj(n);
  {
    // neighbour lists by counting, each sorted and deduplicated on its own
    std::vector<int> deg(n, 0);
    for (size_t t = 0; t < P.row.size(); ++t)
      if (P.row[t] != P.col[t]) { ++deg[P.row[t]]; ++deg[P.col[t]]; }
    for (int v = 0; v < n; ++v) adj[v].reserve(deg[v]);
    for (size_t t = 0; t < P.row.size(); ++t) {
      const int i = P.row[t], j = P.col[t];
      if (i != j) { adj[i].push_back(j); adj[j].push_back(i); }
    }
    for (int v = 0; v < n; ++v) {
      std::sort(adj[v].begin(), adj[v].end());
      adj[v].erase(std::unique(adj[v].begin(), adj[v].end()), adj[v].end());
    }
  }
  // ---- ordering + filled structure ----
  std::vector<int> order;
  std::vector<std::vector<int>> est;
  min_degree(n, std::move(adj), order, est);
  std::vector<int> pos(n);
  for (int p = 0; p < n; ++p) pos[order[p]] = p;
  std::vector<std::vector<int>> st(n);  // struct in elimination positions
  std::vector<int> parent(n, -1);
  for (int p = 0; p < n; ++p) {
    auto &s = st[p];
    for (int u : est[order[p]]) s.push_back(pos[u]);
    std::sort(s.begin(), s.end());
    if (!s.empty()) parent[p] = s[0];
  }
  // ---- postorder of the elimination tree ----
  std::vector<std::vector<int>> kids(n);
  for (int p = 0; p < n; ++p)
    if (parent[p] >= 0) kids[parent[p]].push_back(p);
  std::vector<int> post(n, -1);
  {
    int cnt = 0;
    std::vector<std::pair<int, size_t>> stack;
    for (int r = 0; r < n; ++r) {
      if (parent[r] >= 0) continue;
      stack.push_back({r, 0});
      while (!stack.empty()) {
        auto &top = stack.back();
        if (top.second < kids[top.first].size()) {
          int c = kids[top.first][top.second++];
          stack.push_back({c, 0});
        } else {
          post[top.first] = cnt++;
          stack.pop_back();
        }
      }
    }
  }
  S.perm.assign(n, 0);
  S.iperm.assign(n, 0);
  std::vector<std::vector<int>> sn_struct(n);  // struct in new indices
  std::vector<int> par(n, -1);
  for (int p = 0; p < n; ++p) {
    int q = post[p];
    S.perm[q] = order[p];
    S.iperm[order[p]] = q;
    auto &s = sn_struct[q];
    for (int x : st[p]) s.push_back(post[x]);
    std::sort(s.begin(), s.end());
    par[q] = parent[p] >= 0 ? post[parent[p]] : -1;
  }
  // ---- fundamental supernodes ----
  std::vector<int> nchild(n, 0);
  for (int q = 0; q < n; ++q)
    if (par[q] >= 0) nchild[par[q]]++;
  struct SN {
    int c0, c1;
    double truenz;
    bool alive;
  };
  std::vector<SN> F;
  std::vector<int> col2f(n, 0);
  for (int q = 0; q < n;) {
    int v = q;
    while (v + 1 < n && par[v] == v + 1 && nchild[v + 1] == 1 &&
           sn_struct[v].size() == sn_struct[v + 1].size() + 1)
      ++v;
    double t = 0;
    for (int c = q; c <= v; ++c) t += 1.0 + (double)sn_struct[c].size();
    for (int c = q; c <= v; ++c) col2f[c] = (int)F.size();
    F.push_back({q, v + 1, t, true});
    q = v + 1;
  }
  // ---- relaxed amalgamation: merge a supernode into its parent when it is the parent's last
  // child (columns contiguous) and the explicit zeros this adds stay small.  The merged clique is
  // S_child ∪ S_parent ∪ U_parent (U_child \ S_parent ⊆ U_parent by the clique-tree property), so
  // E grows by the zeros counted here and stays chordal with the same ordering.
  if (o.relax) {
    for (size_t f = 0; f + 1 < F.size(); ++f) {
      SN &a = F[f];
      const auto &Ua = sn_struct[a.c1 - 1];
      if (Ua.empty()) continue;
      const int pf = col2f[Ua[0]];
      SN &p = F[pf];
      if (p.c0 != a.c1) continue;  // not the contiguous (last) child
      const double k = p.c1 - a.c0;
      const double nu = (double)sn_struct[p.c1 - 1].size();
      if (k + nu > o.max_clique) continue;
      const double stored = k * (k + 1) / 2 + nu * k;
      const double z = (stored - (a.truenz + p.truenz)) / stored;
      const bool merge = k <= 4 || (k <= 16 && z < 0.8) || (k <= 48 && z < 0.1) || z < 0.05;
      if (!merge) continue;
      p.c0 = a.c0;
      p.truenz += a.truenz;
      a.alive = false;
      for (int c = a.c0; c < a.c1; ++c) col2f[c] = pf;
    }
  }
  // ---- dense root: every clique with more than root_rows rows or root_cols columns goes, with
  // all its ancestors, into one root supernode whose clique is the union R of their columns.
  // The merged set is closed under taking parents, so the other supernodes keep their columns,
  // their relative order (still a postorder of the forest that remains) and their cliques; R is
  // numbered last.  E grows by the pairs of R that were not yet in it: it stays chordal, with
  // the new order as a perfect elimination order (a vertex outside R keeps its later
  // neighbours, which are its etree ancestors and already a clique; R is a clique).  The clique
  // kernels for small cliques then serve every supernode but the root, and the root is one dense
  // block handled by dense kernels. ----
  if (o.root_rows > 0 || o.root_cols > 0) {
    const int nf = (int)F.size();
    std::vector<int> fpar(nf, -1);
    std::vector<char> big(nf, 0);
    for (int f = 0; f < nf; ++f) {
      if (!F[f].alive) continue;
      const auto &U = sn_struct[F[f].c1 - 1];
      if (!U.empty()) fpar[f] = col2f[U[0]];
      const int ncol = F[f].c1 - F[f].c0, nrow = ncol + (int)U.size();
      if ((o.root_rows > 0 && nrow > o.root_rows) || (o.root_cols > 0 && ncol > o.root_cols))
        big[f] = 1;
    }
    for (int f = 0; f < nf; ++f)
      if (big[f])
        for (int a = fpar[f]; a >= 0 && !big[a]; a = fpar[a]) big[a] = 1;
    int nroot = 0;
    for (int f = 0; f < nf; ++f)
      if (F[f].alive && big[f]) nroot += F[f].c1 - F[f].c0;
    if (nroot > 0) {
      // new number of every column: the columns outside R in order, then those of R in order
      std::vector<char> inR(n, 0);
      for (int f = 0; f < nf; ++f)
        if (F[f].alive && big[f])
          for (int c = F[f].c0; c < F[f].c1; ++c) inR[c] = 1;
      std::vector<int> nq(n);
      int a = 0, b = n - nroot;
      for (int q = 0; q < n; ++q) nq[q] = inR[q] ? b++ : a++;
      std::vector<int> perm2(n);
      for (int q = 0; q < n; ++q) perm2[nq[q]] = S.perm[q];
      S.perm = perm2;
      for (int q = 0; q < n; ++q) S.iperm[S.perm[q]] = q;
      std::vector<std::vector<int>> st2(n);
      std::vector<SN> F2;
      std::vector<int> col2f2(n, 0);
      for (int f = 0; f < nf; ++f) {
        if (!F[f].alive || big[f]) continue;
        auto U = sn_struct[F[f].c1 - 1];
        for (int &x : U) x = nq[x];
        std::sort(U.begin(), U.end());
        const int c0 = nq[F[f].c0], c1 = nq[F[f].c1 - 1] + 1;
        if (c1 - c0 != F[f].c1 - F[f].c0) return "internal: a supernode outside the root split";
        st2[c1 - 1] = std::move(U);
        for (int c = c0; c < c1; ++c) col2f2[c] = (int)F2.size();
        F2.push_back({c0, c1, 0.0, true});
      }
      for (int c = n - nroot; c < n; ++c) col2f2[c] = (int)F2.size();
      F2.push_back({n - nroot, n, 0.0, true});
      F.swap(F2);
      col2f.swap(col2f2);
      sn_struct.swap(st2);
      S.dense_root = true;
    }
  }
  S.sn_col.push_back(0);
  std::vector<std::pair<int, int>> sns;  // (c0, c1) of the surviving supernodes
  for (auto &f : F)
    if (f.alive) sns.push_back({f.c0, f.c1});
  std::sort(sns.begin(), sns.end());
  for (auto &pr : sns) S.sn_col.push_back(pr.second);
  S.ns = (int)sns.size();
  S.col2sn.assign(n, 0);
  S.sn_rowptr.assign(S.ns + 1, 0);
  S.sn_valptr.assign(S.ns + 1, 0);
  S.sn_dptr.assign(S.ns + 1, 0);
  for (int s = 0; s < S.ns; ++s) {
    int c0 = S.sn_col[s], c1 = S.sn_col[s + 1];
    // (the dense root keeps no inverse of its diagonal block in this table: its dense kernels
    // hold their own 32 x 32 block inverses)
    const bool droot = S.dense_root && s == S.ns - 1;
    S.sn_dptr[s + 1] = S.sn_dptr[s] + (droot ? 0 : (int64_t)(c1 - c0) * (c1 - c0));
    if (c0 != sns[s].first) return "internal: supernode partition not contiguous";
    for (int c = c0; c < c1; ++c) S.col2sn[c] = s;
    for (int c = c0; c < c1; ++c) S.rows.push_back(c);
    for (int x : sn_struct[c1 - 1]) S.rows.push_back(x);
    int nrow = (c1 - c0) + (int)sn_struct[c1 - 1].size();
    int ncol = c1 - c0;
    S.sn_rowptr[s + 1] = S.sn_rowptr[s] + nrow;
    S.sn_valptr[s + 1] = S.sn_valptr[s] + (int64_t)nrow * ncol;
    S.max_nrow = std::max(S.max_nrow, nrow);
    S.max_ncol = std::max(S.max_ncol, ncol);
    S.nnz_lower_E += (int64_t)nrow * ncol - (int64_t)ncol * (ncol - 1) / 2;
  }
  S.sn_parent.assign(S.ns, -1);
  for (int s = 0; s < S.ns; ++s) {
    int nrow = (int)(S.sn_rowptr[s + 1] - S.sn_rowptr[s]);
    int ncol = S.sn_col[s + 1] - S.sn_col[s];
    if (nrow > ncol) S.sn_parent[s] = S.col2sn[S.rows[S.sn_rowptr[s] + ncol]];
  }
  S.sn_fdesc.resize(S.ns);
  for (int s = 0; s < S.ns; ++s) S.sn_fdesc[s] = s;
  for (int s = 0; s < S.ns; ++s)
    if (S.sn_parent[s] >= 0) S.sn_fdesc[S.sn_parent[s]] = std::min(S.sn_fdesc[S.sn_parent[s]], S.sn_fdesc[s]);
  // ---- height levels ----
  {
    std::vector<int> h(S.ns, 0);
    for (int s = 0; s < S.ns; ++s)  // children precede parents
      if (S.sn_parent[s] >= 0) h[S.sn_parent[s]] = std::max(h[S.sn_parent[s]], h[s] + 1);
    // the dense root (the last supernode) alone in the top level, so the level-scheduled
    // small-clique kernels can stop one level short of it
    if (S.dense_root && S.ns > 1)
      h[S.ns - 1] = *std::max_element(h.begin(), h.end() - 1) + 1;
    S.height = S.ns ? *std::max_element(h.begin(), h.end()) + 1 : 0;
    S.lvl_ptr.assign(S.height + 1, 0);
    for (int s = 0; s < S.ns; ++s) S.lvl_ptr[h[s] + 1]++;
    for (int l = 0; l < S.height; ++l) S.lvl_ptr[l + 1] += S.lvl_ptr[l];
    S.lvl_sn.assign(S.ns, 0);
    std::vector<int> fill(S.lvl_ptr.begin(), S.lvl_ptr.end() - 1);
    for (int s = 0; s < S.ns; ++s) S.lvl_sn[fill[h[s]]++] = s;
  }
  // ---- left-looking update lists ----
  {
    std::vector<std::vector<std::array<int, 3>>> lists(S.ns);  // (src, p1, p2)
    for (int s = 0; s < S.ns; ++s) {
      int64_t r0 = S.sn_rowptr[s];
      int nrow = (int)(S.sn_rowptr[s + 1] - r0);
      int ncol = S.sn_col[s + 1] - S.sn_col[s];
      int p = ncol;
      while (p < nrow) {
        int t = S.col2sn[S.rows[r0 + p]];
        int q = p;
        while (q < nrow && S.rows[r0 + q] < S.sn_col[t + 1]) ++q;
        lists[t].push_back({s, p, q});
        p = q;
      }
    }
    S.upd_ptr.assign(S.ns + 1, 0);
    S.upd_relptr.push_back(0);
    std::vector<int> at_in_t(n, -1);  // position of a row inside the current target's clique
    for (int t = 0; t < S.ns; ++t) {
      int64_t tr0 = S.sn_rowptr[t];
      int tnrow = (int)(S.sn_rowptr[t + 1] - tr0);
      for (int k = 0; k < tnrow; ++k) at_in_t[S.rows[tr0 + k]] = k;
      for (auto &e : lists[t]) {
        int s = e[0];
        S.upd_src.push_back(s);
        S.upd_p1.push_back(e[1]);
        S.upd_p2.push_back(e[2]);
        int64_t r0 = S.sn_rowptr[s];
        int nrow = (int)(S.sn_rowptr[s + 1] - r0);
        for (int p = e[1]; p < nrow; ++p) {
          const int k = at_in_t[S.rows[r0 + p]];
          if (k < 0) return "internal: update rows not in target clique";
          S.upd_rel.push_back(k);
        }
        S.upd_relptr.push_back((int64_t)S.upd_rel.size());
      }
      for (int k = 0; k < tnrow; ++k) at_in_t[S.rows[tr0 + k]] = -1;
      S.upd_ptr[t + 1] = (int)S.upd_src.size();
    }
  }
  // ---- layout offset of a lower position (new indices r >= c) ----
  auto layout_off = [&](int r, int c) -> int64_t {
    int s = S.col2sn[c];
    int64_t r0 = S.sn_rowptr[s];
    int nrow = (int)(S.sn_rowptr[s + 1] - r0);
    const int *b = S.rows.data() + r0;
    const int *it = std::lower_bound(b, b + nrow, r);
    if (it == b + nrow || *it != r) return -1;
    return S.sn_valptr[s] + (int64_t)(it - b) + (int64_t)(c - S.sn_col[s]) * nrow;
  };
  // ---- aggregate-pattern slots ----
  {
    size_t ne = P.row.size();
    std::vector<int64_t> off(ne);
    for (size_t t = 0; t < ne; ++t) {
      int p = S.iperm[P.row[t]], q = S.iperm[P.col[t]];
      int r = std::max(p, q), c = std::min(p, q);
      off[t] = layout_off(r, c);
      if (off[t] < 0) return "internal: aggregate entry not covered by E";
    }
    // entries in (layout offset, matrix, input index) order.  Layout offsets increase with the
    // column of the lower position (supernodes are contiguous column ranges in order, each block
    // column-major), so a counting sort on that column followed by a sort of each column's
    // entries gives the full order without one sort over every entry.
    std::vector<size_t> idx(ne);
    {
      std::vector<int64_t> colptr(n + 1, 0);
      std::vector<int> colof(ne);
      for (size_t t = 0; t < ne; ++t) {
        colof[t] = std::min(S.iperm[P.row[t]], S.iperm[P.col[t]]);
        colptr[colof[t] + 1]++;
      }
      for (int c = 0; c < n; ++c) colptr[c + 1] += colptr[c];
      std::vector<int64_t> at(colptr.begin(), colptr.end() - 1);
      for (size_t t = 0; t < ne; ++t) idx[at[colof[t]]++] = t;
      for (int c = 0; c < n; ++c)
        std::sort(idx.begin() + colptr[c], idx.begin() + colptr[c + 1], [&](size_t a, size_t b) {
          if (off[a] != off[b]) return off[a] < off[b];
          if (P.mat[a] != P.mat[b]) return P.mat[a] < P.mat[b];
          return a < b;
        });
    }
    S.slot_ptr.push_back(0);
    for (size_t u = 0; u < ne;) {
      size_t v = u;
      double a0 = 0.0;
      while (v < ne && off[idx[v]] == off[idx[u]]) {
        size_t t = idx[v];
        S.slot_k.push_back(P.mat[t]);
        S.slot_val.push_back(P.val[t]);
        if (P.mat[t] == 0) a0 += P.val[t];
        ++v;
      }
      size_t t = idx[u];
      int p = S.iperm[P.row[t]], q = S.iperm[P.col[t]];
      S.slot_i.push_back(std::max(p, q));
      S.slot_j.push_back(std::min(p, q));
      S.slot_off.push_back(off[t]);
      S.slot_a0.push_back(a0);
      S.slot_ptr.push_back((int)S.slot_k.size());
      u = v;
    }
    S.nslot = (int64_t)S.slot_off.size();
    // constraint lists
    std::vector<std::vector<std::array<double, 3>>> cl(m);  // (offset, weight, value)
    for (size_t t = 0; t < ne; ++t) {
      if (P.mat[t] == 0) continue;
      double w = P.row[t] == P.col[t] ? P.val[t] : 2.0 * P.val[t];
      cl[P.mat[t] - 1].push_back({(double)off[t], w, P.val[t]});
    }
    S.con_ptr.assign(m + 1, 0);
    S.con_disjoint = true;
    for (int k = 0; k < m; ++k) {
      std::sort(cl[k].begin(), cl[k].end());
      for (auto &e : cl[k]) {
        S.con_off.push_back((int64_t)e[0]);
        S.con_w.push_back(e[1]);
        S.con_v.push_back(e[2]);
      }
      S.con_ptr[k + 1] = (int)S.con_off.size();
    }
    {
      std::vector<int64_t> offs(S.con_off.begin(), S.con_off.end());
      std::sort(offs.begin(), offs.end());
      S.con_disjoint = std::adjacent_find(offs.begin(), offs.end()) == offs.end();
    }
    // symmetric row lists over slots
    std::vector<std::vector<std::pair<int, int64_t>>> rl(n);
    for (int64_t s = 0; s < S.nslot; ++s) {
      rl[S.slot_i[s]].push_back({S.slot_j[s], S.slot_off[s]});
      if (S.slot_i[s] != S.slot_j[s]) rl[S.slot_j[s]].push_back({S.slot_i[s], S.slot_off[s]});
    }
    S.arow_ptr.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) {
      std::sort(rl[i].begin(), rl[i].end());
      for (auto &e : rl[i]) { S.arow_col.push_back(e.first); S.arow_off.push_back(e.second); }
      S.arow_ptr[i + 1] = (int)S.arow_col.size();
    }
  }
  // ---- strict-lower row structures ----
  {
    std::vector<int> cnt(n + 1, 0);
    for (int s = 0; s < S.ns; ++s) {
      int64_t r0 = S.sn_rowptr[s];
      int nrow = (int)(S.sn_rowptr[s + 1] - r0), c0 = S.sn_col[s], ncol = S.sn_col[s + 1] - c0;
      for (int lc = 0; lc < ncol; ++lc)
        for (int p = lc + 1; p < nrow; ++p) cnt[S.rows[r0 + p] + 1]++;
    }
    for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    S.rs_ptr = cnt;
    S.rs_col.assign(cnt[n], 0);
    S.rs_off.assign(cnt[n], 0);
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    for (int s = 0; s < S.ns; ++s) {
      int64_t r0 = S.sn_rowptr[s];
      int nrow = (int)(S.sn_rowptr[s + 1] - r0), c0 = S.sn_col[s], ncol = S.sn_col[s + 1] - c0;
      for (int lc = 0; lc < ncol; ++lc)
        for (int p = lc + 1; p < nrow; ++p) {
          int r = S.rows[r0 + p];
          int at = fill[r]++;
          S.rs_col[at] = c0 + lc;
          S.rs_off[at] = S.sn_valptr[s] + p + (int64_t)lc * nrow;
        }
    }
  }
  // ---- SCM groups ----
  {
    std::vector<std::vector<int>> supp(m);
    S.unit_diag_constraints = true;
    S.diag_constraints = true;
    for (size_t t = 0; t < P.row.size(); ++t) {
      if (P.mat[t] == 0) continue;
      int k = P.mat[t] - 1;
      supp[k].push_back(S.iperm[P.row[t]]);
      supp[k].push_back(S.iperm[P.col[t]]);
    }
    std::vector<int> cnt_entries(m, 0);
    for (size_t t = 0; t < P.row.size(); ++t) {
      if (P.mat[t] == 0) continue;
      int k = P.mat[t] - 1;
      cnt_entries[k]++;
      if (P.row[t] != P.col[t] || P.row[t] != k || P.val[t] != 1.0) S.unit_diag_constraints = false;
      if (P.row[t] != P.col[t]) S.diag_constraints = false;
    }
    for (int k = 0; k < m; ++k) {
      if (cnt_entries[k] != 1) S.unit_diag_constraints = false;
      auto &s = supp[k];
      std::sort(s.begin(), s.end());
      s.erase(std::unique(s.begin(), s.end()), s.end());
      if (s.empty()) return "constraint matrix A_" + std::to_string(k + 1) + " is empty";
      if ((int)s.size() > o.panel_max)
        return "constraint A_" + std::to_string(k + 1) + " touches " + std::to_string(s.size()) +
               " rows/columns; the SCM panel limit is " + std::to_string(o.panel_max);
    }
    // connected components of the SCM's nonzero structure: union-find over every input entry
    // (elimination numbering) and over each constraint's support (an A_k with only diagonal
    // entries, on rows of different pattern components, couples them through B_kq)
    std::vector<int> uf(n);
    std::iota(uf.begin(), uf.end(), 0);
    auto find = [&](int x) {
      while (uf[x] != x) {
        uf[x] = uf[uf[x]];
        x = uf[x];
      }
      return x;
    };
    for (size_t t = 0; t < P.row.size(); ++t) {
      const int a = find(S.iperm[P.row[t]]), b = find(S.iperm[P.col[t]]);
      if (a != b) uf[std::max(a, b)] = std::min(a, b);
    }
    for (int k = 0; k < m; ++k)
      for (size_t q = 1; q < supp[k].size(); ++q) {
        const int a = find(supp[k][0]), b = find(supp[k][q]);
        if (a != b) uf[std::max(a, b)] = std::min(a, b);
      }
    std::vector<int> ccomp(m);
    for (int k = 0; k < m; ++k) ccomp[k] = find(supp[k][0]);
    std::vector<int> ord(m);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) {
      if (ccomp[a] != ccomp[b]) return ccomp[a] < ccomp[b];
      if (supp[a][0] != supp[b][0]) return supp[a][0] < supp[b][0];
      return a < b;
    });
    S.comp_cptr.assign(1, 0);
    for (int i = 1; i <= m; ++i)
      if (i == m || ccomp[ord[i]] != ccomp[ord[i - 1]]) S.comp_cptr.push_back(i);
    S.ncomp = (int)S.comp_cptr.size() - 1;
    S.con_order = ord;
    S.con_internal.assign(m, 0);
    for (int i = 0; i < m; ++i) S.con_internal[ord[i]] = i;
    S.grp_cptr.push_back(0);
    S.grp_pptr.push_back(0);
    std::vector<int> U, tmp;
    int gstart = 0;
    auto close_group = [&](int end) {
      S.grp_cptr.push_back(end);
      for (int x : U) S.grp_cols.push_back(x);
      S.grp_pptr.push_back((int)S.grp_cols.size());
      U.clear();
      gstart = end;
    };
    for (int i = 0; i < m; ++i) {
      const auto &s = supp[ord[i]];
      tmp.clear();
      std::set_union(U.begin(), U.end(), s.begin(), s.end(), std::back_inserter(tmp));
      const bool new_comp = i > gstart && ccomp[ord[i]] != ccomp[ord[i - 1]];
      if (i > gstart && ((int)tmp.size() > o.panel_max || i - gstart >= o.group_max || new_comp)) {
        close_group(i);
        U = s;
      } else {
        U.swap(tmp);
      }
    }
    close_group(m);
    S.ngroup = (int)S.grp_cptr.size() - 1;
    S.grp_comp.assign(S.ngroup, 0);
    for (int g = 0, cc = 0; g < S.ngroup; ++g) {
      while (S.comp_cptr[cc + 1] <= S.grp_cptr[g]) ++cc;
      S.grp_comp[g] = cc;
    }
    S.grp_rowoff.assign(S.ngroup + 1, 0);
    for (int g = 0; g < S.ngroup; ++g)
      S.grp_rowoff[g + 1] = S.grp_rowoff[g] + (S.grp_pptr[g + 1] - S.grp_pptr[g]);
    // local nonzero lists per internal constraint (both triangles: an off-diagonal entry is
    // followed by its mirror), each in input order; counted first, then filled in place
    std::vector<int> grp_of(m);
    for (int g = 0; g < S.ngroup; ++g)
      for (int i = S.grp_cptr[g]; i < S.grp_cptr[g + 1]; ++i) grp_of[i] = g;
    S.anz_ptr.assign(m + 1, 0);
    for (size_t t = 0; t < P.row.size(); ++t)
      if (P.mat[t] != 0) S.anz_ptr[S.con_internal[P.mat[t] - 1] + 1] += P.row[t] != P.col[t] ? 2 : 1;
    for (int i = 0; i < m; ++i) S.anz_ptr[i + 1] += S.anz_ptr[i];
    S.anz_a.assign(S.anz_ptr[m], 0);
    S.anz_b.assign(S.anz_ptr[m], 0);
    S.anz_v.assign(S.anz_ptr[m], 0.0);
    {
      std::vector<int> at(S.anz_ptr.begin(), S.anz_ptr.end() - 1);
      for (size_t t = 0; t < P.row.size(); ++t) {
        if (P.mat[t] == 0) continue;
        int i = S.con_internal[P.mat[t] - 1];
        int g = grp_of[i];
        const int *pb = S.grp_cols.data() + S.grp_pptr[g];
        const int *pe = S.grp_cols.data() + S.grp_pptr[g + 1];
        int a = (int)(std::lower_bound(pb, pe, S.iperm[P.row[t]]) - pb);
        int b = (int)(std::lower_bound(pb, pe, S.iperm[P.col[t]]) - pb);
        if ((a != b) != (P.row[t] != P.col[t])) return "internal: constraint entry outside its panel";
        S.anz_a[at[i]] = (int16_t)a;
        S.anz_b[at[i]] = (int16_t)b;
        S.anz_v[at[i]++] = P.val[t];
        if (a != b) {
          S.anz_a[at[i]] = (int16_t)b;
          S.anz_b[at[i]] = (int16_t)a;
          S.anz_v[at[i]++] = P.val[t];
        }
      }
    }
    // reach (forward) and need (backward) supernode lists per group
    std::vector<char> mark(S.ns, 0);
    S.reach_ptr.push_back(0);
    for (int g = 0; g < S.ngroup; ++g) {
      std::fill(mark.begin(), mark.end(), 0);
      for (int p = S.grp_pptr[g]; p < S.grp_pptr[g + 1]; ++p)
        for (int s = S.col2sn[S.grp_cols[p]]; s >= 0 && !mark[s]; s = S.sn_parent[s]) mark[s] = 1;
      for (int s = 0; s < S.ns; ++s)
        if (mark[s]) S.reach_sn.push_back(s);
      S.reach_ptr.push_back((int64_t)S.reach_sn.size());
    }
    std::vector<std::vector<int>> need(S.ngroup);
    std::fill(mark.begin(), mark.end(), 0);
    for (int g = S.ngroup - 1; g >= 0; --g) {
      for (int p = S.grp_pptr[g]; p < S.grp_pptr[g + 1]; ++p)
        for (int s = S.col2sn[S.grp_cols[p]]; s >= 0 && !mark[s]; s = S.sn_parent[s]) mark[s] = 1;
      for (int s = 0; s < S.ns; ++s)
        if (mark[s]) need[g].push_back(s);
    }
    S.need_ptr.push_back(0);
    for (int g = 0; g < S.ngroup; ++g) {
      for (int s : need[g]) S.need_sn.push_back(s);
      S.need_ptr.push_back((int64_t)S.need_sn.size());
    }
  }
  return "";
}

}  // namespace mcsdp
