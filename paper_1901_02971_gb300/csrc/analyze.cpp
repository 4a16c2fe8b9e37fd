// Host-side analysis for spaND: modified nested-dissection ordering and
// clustering (Algorithm 3, Sec. 2.3), cluster formation, and the symbolic
// per-step structure the numeric factorization runs on (elimination sets,
// fill pattern of Sec. 2.4, colouring of the sparsification order, merge maps
// of Sec. 2.7).  Integer work only; deterministic.
//
// Readings of the paper (identical in the test oracle):
//  * separator (l,k) <-> heap index h = 2^(l-1)+k-1, none = -1;
//  * geometric bisection of U = I u B: dimension of largest span (lowest on
//    ties), order U by (coordinate, id), threshold = coordinate at 0-based
//    position floor((|U|-1)/2), P1 = {x <= threshold}, P2 = rest (if P2 is
//    empty: P1 = first ceil(|U|/2) of the order), |U| < 2: all left;
//    separator M = vertices of P1 adjacent to P2;
//  * no coordinates: BFS distance from the vertex farthest from the smallest
//    id (smallest id on ties) is the single coordinate, unreached vertices get
//    the largest finite distance + 1;
//  * clusters ordered by (step, S, L, R), vertices by id; step t = L+1-level(S);
//  * merge after step t: labels at level L+1-t replaced by their parent;
//  * greedy colouring of the remaining clusters after the step's fill.
#include "spand_internal.h"

#include <algorithm>
#include <numeric>
#include <stdexcept>
#include <tuple>

namespace spand {

static inline int level_of(int32_t h) {
  int l = 0;
  while (h > 0) { ++l; h >>= 1; }
  return l;
}

namespace {

struct Graph {
  int64_t n;
  const int64_t* rowptr;
  const int32_t* colind;
};

// Split U (ascending ids) into left / mid / right; writes membership into
// part[] (0 left, 1 mid, 2 right) for the vertices of U.
void bisect(const Graph& g, const std::vector<int32_t>& U, const std::vector<double>& x, int dim,
            std::vector<int8_t>& part, std::vector<uint8_t>& flag) {
  const size_t m = U.size();
  if (m < 2) {
    for (int32_t v : U) part[v] = 0;
    return;
  }
  int dbest = 0;
  double sbest = -1.0;
  for (int d = 0; d < dim; ++d) {
    double lo = x[(size_t)0 * dim + d], hi = lo;
    for (size_t i = 1; i < m; ++i) {
      double c = x[i * dim + d];
      lo = std::min(lo, c);
      hi = std::max(hi, c);
    }
    double s = hi - lo;
    if (s > sbest) { sbest = s; dbest = d; }
  }
  std::vector<int32_t> ord(m);
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) {
    double ca = x[(size_t)a * dim + dbest], cb = x[(size_t)b * dim + dbest];
    if (ca != cb) return ca < cb;
    return U[a] < U[b];
  });
  const double t = x[(size_t)ord[(m - 1) / 2] * dim + dbest];
  size_t n1 = 0;
  for (size_t i = 0; i < m; ++i) {
    bool in1 = x[i * dim + dbest] <= t;
    part[U[i]] = in1 ? 0 : 2;
    n1 += in1;
  }
  if (n1 == m) {
    for (size_t i = 0; i < m; ++i) part[U[ord[i]]] = (i < (m + 1) / 2) ? 0 : 2;
  }
  for (int32_t v : U) flag[v] = (part[v] == 2);
  for (int32_t v : U) {
    if (part[v] != 0) continue;
    for (int64_t e = g.rowptr[v]; e < g.rowptr[v + 1]; ++e) {
      int32_t w = g.colind[e];
      if (w != v && flag[w]) { part[v] = 1; break; }
    }
  }
  for (int32_t v : U) flag[v] = 0;
}

// BFS distances inside U (inU flags set by the caller), from src.
void bfs(const Graph& g, int32_t src, const std::vector<uint8_t>& inU, std::vector<int32_t>& dist,
         std::vector<int32_t>& queue) {
  queue.clear();
  dist[src] = 0;
  queue.push_back(src);
  for (size_t head = 0; head < queue.size(); ++head) {
    int32_t v = queue[head];
    for (int64_t e = g.rowptr[v]; e < g.rowptr[v + 1]; ++e) {
      int32_t w = g.colind[e];
      if (inU[w] && dist[w] < 0) {
        dist[w] = dist[v] + 1;
        queue.push_back(w);
      }
    }
  }
}

}  // namespace

int analyze_tree(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* coords,
                 int dim, int L, Tree& T, std::string& err) {
  Graph g{n, rowptr, colind};
  T.n = n;
  T.L = L;
  std::vector<int32_t> S(n, 1), Lb(n, -1), Rb(n, -1);
  std::vector<int8_t> part(n, 0);
  std::vector<uint8_t> flag(n, 0), inU(n, 0);
  std::vector<int32_t> dist(n, -1), queue;
  queue.reserve(n);
  // ---------------- Algorithm 3
  for (int lvl = 1; lvl < L; ++lvl) {
    const int32_t first = 1 << (lvl - 1);
    std::vector<std::vector<int32_t>> Ib(first), Bb(first);
    for (int64_t v = 0; v < n; ++v) {
      if (level_of(S[v]) == lvl) Ib[S[v] - first].push_back((int32_t)v);
      bool inl = Lb[v] >= 0 && level_of(Lb[v]) == lvl;
      bool inr = Rb[v] >= 0 && level_of(Rb[v]) == lvl;
      if (inl) Bb[Lb[v] - first].push_back((int32_t)v);
      if (inr && !(inl && Rb[v] == Lb[v])) Bb[Rb[v] - first].push_back((int32_t)v);
    }
    for (int32_t k = 0; k < first; ++k) {
      const int32_t h = first + k;
      const auto& I = Ib[k];
      const auto& B = Bb[k];
      std::vector<int32_t> U;
      U.reserve(I.size() + B.size());
      std::merge(I.begin(), I.end(), B.begin(), B.end(), std::back_inserter(U));
      std::vector<double> x;
      int xd = dim;
      if (coords) {
        x.resize(U.size() * (size_t)dim);
        for (size_t i = 0; i < U.size(); ++i)
          for (int d = 0; d < dim; ++d) x[i * dim + d] = coords[(size_t)U[i] * dim + d];
      } else {
        xd = 1;
        x.assign(U.size(), 0.0);
        if (U.size() >= 2) {
          for (int32_t v : U) inU[v] = 1;
          bfs(g, U[0], inU, dist, queue);
          int32_t far = -1, r1 = U[0];
          for (int32_t v : U)
            if (dist[v] > far) { far = dist[v]; r1 = v; }
          for (int32_t v : U) dist[v] = -1;
          bfs(g, r1, inU, dist, queue);
          int32_t dmax = 0;
          for (int32_t v : U) dmax = std::max(dmax, dist[v]);
          for (size_t i = 0; i < U.size(); ++i) {
            int32_t d = dist[U[i]];
            x[i] = (double)(d >= 0 ? d : dmax + 1);
          }
          for (int32_t v : U) { dist[v] = -1; inU[v] = 0; }
        }
      }
      bisect(g, U, x, xd, part, flag);
      // updates (I and B are disjoint: interior vertices carry no L/R label)
      for (int32_t v : I) {
        if (part[v] == 0) S[v] = 2 * h;
        else if (part[v] == 2) S[v] = 2 * h + 1;
        else { Lb[v] = 2 * h; Rb[v] = 2 * h + 1; }
      }
      for (int32_t v : B) {
        if (part[v] == 1) continue;
        int32_t child = part[v] == 0 ? 2 * h : 2 * h + 1;
        if (Lb[v] == h) Lb[v] = child;
        else Rb[v] = child;
      }
    }
  }
  // ---------------- clusters
  auto step_of = [&](int32_t s) { return L + 1 - level_of(s); };
  std::vector<int32_t> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) {
    auto ka = std::make_tuple(step_of(S[a]), S[a], Lb[a], Rb[a], a);
    auto kb = std::make_tuple(step_of(S[b]), S[b], Lb[b], Rb[b], b);
    return ka < kb;
  });
  T.perm.assign(ord.begin(), ord.end());
  T.cluster_ptr.clear();
  T.keys.clear();
  std::vector<int32_t> cl_of(n);
  for (int64_t i = 0; i < n; ++i) {
    int32_t v = ord[i];
    if (i == 0 || S[v] != S[ord[i - 1]] || Lb[v] != Lb[ord[i - 1]] || Rb[v] != Rb[ord[i - 1]]) {
      T.cluster_ptr.push_back((int32_t)i);
      T.keys.push_back(S[v]);
      T.keys.push_back(Lb[v]);
      T.keys.push_back(Rb[v]);
    }
    cl_of[v] = (int32_t)T.cluster_ptr.size() - 1;
  }
  T.cluster_ptr.push_back((int32_t)n);
  const int nc = (int)T.cluster_ptr.size() - 1;
  // ---------------- symbolic steps
  std::vector<std::vector<int32_t>> adj(nc);
  for (int64_t v = 0; v < n; ++v)
    for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
      int32_t a = cl_of[v], b = cl_of[colind[e]];
      if (a != b) adj[a].push_back(b);
    }
  auto uniq = [](std::vector<int32_t>& l) {
    std::sort(l.begin(), l.end());
    l.erase(std::unique(l.begin(), l.end()), l.end());
  };
  for (auto& l : adj) uniq(l);
  std::vector<std::array<int32_t, 3>> cur(nc);
  for (int c = 0; c < nc; ++c) cur[c] = {T.keys[3 * c], T.keys[3 * c + 1], T.keys[3 * c + 2]};
  std::vector<std::vector<int32_t>> children(nc);
  for (int c = 0; c < nc; ++c) children[c] = {c};
  T.steps.clear();
  for (int t = 1; t <= L; ++t) {
    const int lam = L + 1 - t;
    const int nt = (int)cur.size();
    StepStruct st;
    st.n = nt;
    st.elim.resize(nt);
    for (int i = 0; i < nt; ++i) st.elim[i] = level_of(cur[i][0]) == lam ? 1 : 0;
    for (int i = 0; i < nt; ++i)
      if (st.elim[i])
        for (int32_t j : adj[i])
          if (st.elim[j]) {
            err = "two separators of one level are adjacent";
            return 1;
          }
    std::vector<std::vector<int32_t>> adjf(nt);
    for (int i = 0; i < nt; ++i)
      if (!st.elim[i])
        for (int32_t j : adj[i])
          if (!st.elim[j]) adjf[i].push_back(j);
    for (int s = 0; s < nt; ++s)
      if (st.elim[s])
        for (int32_t a : adj[s])
          for (int32_t b : adj[s])
            if (a != b) adjf[a].push_back(b);
    for (auto& l : adjf) uniq(l);
    st.colour.assign(nt, -1);
    std::vector<int32_t> mark;
    for (int i = 0; i < nt; ++i) {
      if (st.elim[i]) continue;
      mark.clear();
      for (int32_t j : adjf[i])
        if (j < i) mark.push_back(st.colour[j]);
      std::sort(mark.begin(), mark.end());
      int32_t c = 0;
      for (int32_t m : mark) {
        if (m == c) ++c;
        else if (m > c) break;
      }
      st.colour[i] = c;
    }
    for (int i = 0; i < nt; ++i)
      for (int q = 0; q < 3; ++q) st.keys.push_back(cur[i][q]);
    st.child_ptr.push_back(0);
    for (auto& ch : children) {
      st.child_idx.insert(st.child_idx.end(), ch.begin(), ch.end());
      st.child_ptr.push_back((int32_t)st.child_idx.size());
    }
    st.adj_ptr.push_back(0);
    for (auto& l : adj) {
      st.adj_idx.insert(st.adj_idx.end(), l.begin(), l.end());
      st.adj_ptr.push_back((int32_t)st.adj_idx.size());
    }
    st.adjf_ptr.push_back(0);
    for (auto& l : adjf) {
      st.adjf_idx.insert(st.adjf_idx.end(), l.begin(), l.end());
      st.adjf_ptr.push_back((int32_t)st.adjf_idx.size());
    }
    T.steps.push_back(std::move(st));
    // merge
    auto coarsen = [&](int32_t h) { return (h >= 0 && level_of(h) == lam) ? h / 2 : h; };
    std::vector<int32_t> rem;
    for (int i = 0; i < nt; ++i)
      if (!T.steps.back().elim[i]) rem.push_back(i);
    std::vector<std::array<int32_t, 3>> nk(nt);
    for (int32_t i : rem) nk[i] = {cur[i][0], coarsen(cur[i][1]), coarsen(cur[i][2])};
    std::vector<std::array<int32_t, 3>> parents;
    for (int32_t i : rem) parents.push_back(nk[i]);
    auto pless = [&](const std::array<int32_t, 3>& a, const std::array<int32_t, 3>& b) {
      return std::make_tuple(step_of(a[0]), a[0], a[1], a[2]) < std::make_tuple(step_of(b[0]), b[0], b[1], b[2]);
    };
    std::sort(parents.begin(), parents.end(), pless);
    parents.erase(std::unique(parents.begin(), parents.end()), parents.end());
    std::vector<int32_t> pof(nt, -1);
    for (int32_t i : rem)
      pof[i] = (int32_t)(std::lower_bound(parents.begin(), parents.end(), nk[i], pless) - parents.begin());
    std::vector<std::vector<int32_t>> nch(parents.size()), nadj(parents.size());
    for (int32_t i : rem) nch[pof[i]].push_back(i);
    for (int32_t i : rem)
      for (int32_t j : adjf[i])
        if (pof[i] != pof[j]) nadj[pof[i]].push_back(pof[j]);
    for (auto& l : nadj) uniq(l);
    cur = std::move(parents);
    children = std::move(nch);
    adj = std::move(nadj);
  }
  if (!cur.empty()) {
    err = "clusters left after the root step";
    return 1;
  }
  return 0;
}

int validate_csr(int64_t n, const int64_t* rowptr, const int32_t* colind, std::string& err) {
  if (n < 0) { err = "n < 0"; return 1; }
  if (n > 0 && (!rowptr || !colind)) { err = "null CSR array"; return 1; }
  if (n == 0) return 0;
  if (rowptr[0] != 0) { err = "rowptr[0] != 0"; return 1; }
  for (int64_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) { err = "rowptr not monotone"; return 1; }
  const int64_t nnz = rowptr[n];
  std::vector<int64_t> cnt(n, 0);
  for (int64_t i = 0; i < n; ++i) {
    bool diag = false;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      int32_t j = colind[e];
      if (j < 0 || j >= n) { err = "column index out of range"; return 1; }
      if (e > rowptr[i] && colind[e - 1] >= j) { err = "columns not strictly increasing in a row"; return 1; }
      diag |= (j == i);
      cnt[j]++;
    }
    if (!diag) { err = "missing diagonal entry"; return 1; }
  }
  // symmetric pattern: every (i,j) has (j,i)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      int32_t j = colind[e];
      const int32_t* b = colind + rowptr[j];
      const int32_t* en = colind + rowptr[j + 1];
      if (!std::binary_search(b, en, (int32_t)i)) { err = "pattern is not symmetric"; return 1; }
    }
  (void)nnz;
  return 0;
}

}  // namespace spand
