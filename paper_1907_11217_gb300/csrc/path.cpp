// Contraction trees: analysis, the greedy builder, the cost model and the
// slice selector. The paper defers its own contraction algorithm to its
// earlier work; these are the library's own.
#include <algorithm>
#include <functional>
#include <limits>
#include <cmath>
#include <queue>
#include <unordered_map>

#include "tz_internal.h"

namespace tz {

void validate_tree(const Network &net, const Pairs &pairs) {
  const int L = (int)net.leaves.size();
  if (L == 0) fail(TZ_EINVAL, "network has no tensors");
  if ((int)pairs.size() != L - 1)
    fail(TZ_EINVAL, "tree must have exactly n_tensors-1 pairs (got " + std::to_string(pairs.size()) + ", want " +
                        std::to_string(L - 1) + ")");
  std::vector<char> used(2 * L, 0);
  for (size_t s = 0; s < pairs.size(); s++) {
    int a = pairs[s].first, b = pairs[s].second, c = L + (int)s;
    if (a < 0 || b < 0 || a >= c || b >= c || a == b) fail(TZ_EINVAL, "tree pair " + std::to_string(s) + " is invalid");
    if (used[a] || used[b]) fail(TZ_EINVAL, "tree uses a node twice (pair " + std::to_string(s) + ")");
    used[a] = used[b] = 1;
  }
}

static std::vector<int> set_union(const std::vector<int> &a, const std::vector<int> &b) {
  std::vector<int> r;
  std::set_union(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(r));
  return r;
}

TreeInfo analyse_tree(const Network &net, const Pairs &pairs, const std::vector<char> &sliced) {
  TreeInfo ti;
  const int L = (int)net.leaves.size();
  const int I = (int)net.indices.size();
  std::vector<int> cnt(I, 0);
  ti.sets.resize(L + pairs.size());
  ti.var.assign(L + pairs.size(), 0);
  for (int l = 0; l < L; l++) {
    const Leaf &lf = net.leaves[l];
    bool var = lf.kind == LEAF_OUTPUT;
    for (int i : lf.idx) {
      if (!sliced.empty() && sliced[i]) {
        var = true;
        continue;
      }
      ti.sets[l].push_back(i);
      cnt[i]++;
    }
    std::sort(ti.sets[l].begin(), ti.sets[l].end());
    ti.var[l] = var;
    ti.max_bits = std::max(ti.max_bits, (int)ti.sets[l].size());
  }
  ti.steps.reserve(pairs.size());
  for (size_t s = 0; s < pairs.size(); s++) {
    StepInfo st;
    st.a = pairs[s].first;
    st.b = pairs[s].second;
    st.c = L + (int)s;
    const auto &A = ti.sets[st.a], &B = ti.sets[st.b];
    std::vector<int> C;
    size_t ia = 0, ib = 0;
    while (ia < A.size() || ib < B.size()) {
      int i;
      bool inA, inB;
      if (ib >= B.size() || (ia < A.size() && A[ia] < B[ib])) {
        i = A[ia++];
        inA = true;
        inB = false;
      } else if (ia >= A.size() || B[ib] < A[ia]) {
        i = B[ib++];
        inA = false;
        inB = true;
      } else {
        i = A[ia];
        ia++;
        ib++;
        inA = inB = true;
      }
      if (inA && inB) {
        cnt[i]--;
        if (cnt[i] > 1 || net.is_open(i)) {
          st.batch.push_back(i);
          C.push_back(i);
        } else {
          st.contr.push_back(i);
          cnt[i] = 0;
        }
      } else {
        if (cnt[i] <= 1 && !net.is_open(i)) fail(TZ_EINVAL, "index held by one tensor only (dangling)");
        (inA ? st.freeA : st.freeB).push_back(i);
        C.push_back(i);
      }
    }
    st.var = ti.var[st.a] || ti.var[st.b];
    ti.var[st.c] = st.var;
    ti.sets[st.c] = C;
    ti.max_bits = std::max(ti.max_bits, (int)C.size());
    ti.steps.push_back(std::move(st));
  }
  return ti;
}

// The estimate depends only on the sizes of the four index classes.
double CostModel::step_time_sizes(int nb, int nc, int na, int nf) const {
  const int all = nb + nc + na + nf;
  const double macs = std::ldexp(1.0, all);
  const bool c128 = precision == TZ_C128_SIMT;
  const double esz = c128 ? 16.0 : 8.0;
  const double bytes =
      esz * (std::ldexp(1.0, nb + nc + na) + std::ldexp(1.0, nb + nc + nf) + std::ldexp(1.0, nb + na + nf));
  const double simt = c128 ? simt_fp64_flops : simt_flops;
  if (all <= small_log2) return small_step_s + bytes / hbm_bps + 8.0 * macs / simt * 0.5;
  double rate = simt;
  if (precision == TZ_TF32X3 || precision == TZ_BF16X3 || precision == TZ_FP16X3) {
    // the tensor-core path needs a real contraction (k >= 2 complex, m >= 64)
    const int mk = std::max(na, nf);
    if (nc >= 1 && mk >= 6) rate = tc_useful_flops;
  }
  return 3.0e-6 + std::max(8.0 * macs / rate, bytes / hbm_bps);
}

double CostModel::step_time(const StepInfo &s) const {
  return step_time_sizes((int)s.batch.size(), (int)s.contr.size(), (int)s.freeA.size(), (int)s.freeB.size());
}

double group_time(const TreeInfo &ti, const CostModel &cm) {
  double t = 0;
  for (const StepInfo &s : ti.steps)
    if (s.var) t += cm.step_time(s);
  return t;
}

// ------------------------------------------------------------------ greedy
Pairs greedy_tree(const Network &net, double alpha, double temperature, uint64_t seed) {
  const int L = (int)net.leaves.size();
  const int I = (int)net.indices.size();
  std::vector<std::vector<int>> sets(L);
  std::vector<std::vector<int>> holders(I);
  std::vector<int> cnt(I, 0);
  for (int l = 0; l < L; l++) {
    sets[l] = net.leaves[l].idx;
    std::sort(sets[l].begin(), sets[l].end());
    for (int i : sets[l]) {
      cnt[i]++;
      holders[i].push_back(l);
    }
  }
  std::vector<char> alive(L, 1);
  uint64_t rng = seed;
  auto gumbel = [&]() {
    double u = ((splitmix64_next(rng) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    return -std::log(-std::log(u));
  };
  auto out_bits = [&](int a, int b) {
    const auto &A = sets[a], &B = sets[b];
    int n = 0;
    size_t ia = 0, ib = 0;
    while (ia < A.size() || ib < B.size()) {
      if (ib >= B.size() || (ia < A.size() && A[ia] < B[ib])) {
        n++;
        ia++;
      } else if (ia >= A.size() || B[ib] < A[ia]) {
        n++;
        ib++;
      } else {
        int i = A[ia];
        if (cnt[i] - 1 > 1 || net.is_open(i)) n++;
        ia++;
        ib++;
      }
    }
    return n;
  };
  struct Cand {
    double score;
    int a, b;
    bool operator<(const Cand &o) const {
      if (score != o.score) return score > o.score;  // min-heap
      if (a != o.a) return a > o.a;
      return b > o.b;
    }
  };
  std::priority_queue<Cand> heap;
  auto push = [&](int a, int b) {
    if (a > b) std::swap(a, b);
    double sc = std::ldexp(1.0, out_bits(a, b)) - alpha * (std::ldexp(1.0, (int)sets[a].size()) +
                                                           std::ldexp(1.0, (int)sets[b].size()));
    double lg = (sc >= 0 ? 1.0 : -1.0) * std::log2(1.0 + std::fabs(sc));
    if (temperature > 0) lg -= temperature * gumbel();
    heap.push({lg, a, b});
  };
  for (int i = 0; i < I; i++) {
    if (net.is_open(i)) continue;
    auto &h = holders[i];
    for (size_t x = 0; x < h.size(); x++)
      for (size_t y = x + 1; y < h.size(); y++) push(h[x], h[y]);
  }
  Pairs pairs;
  pairs.reserve(L);
  while (!heap.empty()) {
    Cand cd_ = heap.top();
    heap.pop();
    int a = cd_.a, b = cd_.b;
    if (!alive[a] || !alive[b]) continue;
    // merge
    const auto &A = sets[a], &B = sets[b];
    std::vector<int> C;
    size_t ia = 0, ib = 0;
    while (ia < A.size() || ib < B.size()) {
      if (ib >= B.size() || (ia < A.size() && A[ia] < B[ib])) {
        C.push_back(A[ia++]);
      } else if (ia >= A.size() || B[ib] < A[ia]) {
        C.push_back(B[ib++]);
      } else {
        int i = A[ia];
        cnt[i]--;
        if (cnt[i] > 1 || net.is_open(i))
          C.push_back(i);
        else
          cnt[i] = 0;
        ia++;
        ib++;
      }
    }
    int c = (int)sets.size();
    alive[a] = alive[b] = 0;
    alive.push_back(1);
    sets.push_back(C);
    pairs.push_back({a, b});
    for (int i : C) {
      auto &h = holders[i];
      h.erase(std::remove_if(h.begin(), h.end(), [&](int x) { return !alive[x]; }), h.end());
      h.push_back(c);
    }
    std::vector<int> nb;
    for (int i : C) {
      if (net.is_open(i)) continue;
      for (int d : holders[i])
        if (d != c) nb.push_back(d);
    }
    std::sort(nb.begin(), nb.end());
    nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
    for (int d : nb) push(c, d);
  }
  // components left (joined only through open indices): smallest first
  std::vector<int> rest;
  for (int x = 0; x < (int)sets.size(); x++)
    if (alive[x]) rest.push_back(x);
  while (rest.size() > 1) {
    std::sort(rest.begin(), rest.end(), [&](int x, int y) {
      if (sets[x].size() != sets[y].size()) return sets[x].size() < sets[y].size();
      return x < y;
    });
    int a = rest[0], b = rest[1];
    std::vector<int> C = set_union(sets[a], sets[b]);
    int c = (int)sets.size();
    sets.push_back(C);
    alive[a] = alive[b] = 0;
    alive.push_back(1);
    pairs.push_back({a, b});
    rest.erase(rest.begin(), rest.begin() + 2);
    rest.push_back(c);
  }
  return pairs;
}

// ------------------------------------------------------ variable elimination
// Bucket elimination: repeatedly pick an index, merge every tensor that holds
// it (two smallest first) so that it is summed out, and continue. The index
// picked is the one whose merged tensor would be smallest (min-degree
// order), with Gumbel noise of the given temperature to randomise ties.
Pairs elimination_tree(const Network &net, double temperature, uint64_t seed) {
  const int L = (int)net.leaves.size();
  const int I = (int)net.indices.size();
  std::vector<std::vector<int>> sets(L);
  std::vector<std::vector<int>> holders(I);
  std::vector<int> cnt(I, 0);
  std::vector<char> alive(L, 1);
  for (int l = 0; l < L; l++) {
    sets[l] = net.leaves[l].idx;
    std::sort(sets[l].begin(), sets[l].end());
    for (int i : sets[l]) {
      cnt[i]++;
      holders[i].push_back(l);
    }
  }
  uint64_t rng = seed;
  auto gumbel = [&]() {
    double u = ((splitmix64_next(rng) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    return -std::log(-std::log(u));
  };
  auto live_holders = [&](int v) {
    auto &h = holders[v];
    h.erase(std::remove_if(h.begin(), h.end(), [&](int x) { return !alive[x]; }), h.end());
    return h;
  };
  auto score = [&](int v) {
    std::vector<int> u;
    for (int t : live_holders(v)) u = set_union(u, sets[t]);
    return (double)u.size() - 1.0;
  };
  std::vector<int> version(I, 0);
  struct Cand {
    double key;
    int v, ver;
    bool operator<(const Cand &o) const {
      if (key != o.key) return key > o.key;
      return v > o.v;
    }
  };
  std::priority_queue<Cand> heap;
  auto push = [&](int v) {
    version[v]++;
    double k = score(v);
    if (temperature > 0) k -= temperature * gumbel();
    heap.push({k, v, version[v]});
  };
  for (int v = 0; v < I; v++)
    if (!net.is_open(v) && cnt[v] > 0) push(v);
  Pairs pairs;
  auto merge = [&](int a, int b) {
    const auto &A = sets[a], &B = sets[b];
    std::vector<int> C;
    size_t ia = 0, ib = 0;
    while (ia < A.size() || ib < B.size()) {
      if (ib >= B.size() || (ia < A.size() && A[ia] < B[ib])) {
        C.push_back(A[ia++]);
      } else if (ia >= A.size() || B[ib] < A[ia]) {
        C.push_back(B[ib++]);
      } else {
        int i = A[ia];
        cnt[i]--;
        if (cnt[i] > 1 || net.is_open(i))
          C.push_back(i);
        else
          cnt[i] = 0;
        ia++;
        ib++;
      }
    }
    int c = (int)sets.size();
    alive[a] = alive[b] = 0;
    alive.push_back(1);
    sets.push_back(C);
    for (int i : C) holders[i].push_back(c);
    pairs.push_back({a, b});
    return c;
  };
  while (!heap.empty()) {
    Cand cd_ = heap.top();
    heap.pop();
    int v = cd_.v;
    if (cd_.ver != version[v] || cnt[v] == 0) continue;
    std::vector<int> H = live_holders(v);
    if (H.size() < 2) continue;
    // merge the bucket, two smallest first
    while (H.size() > 1) {
      std::sort(H.begin(), H.end(), [&](int x, int y) {
        if (sets[x].size() != sets[y].size()) return sets[x].size() < sets[y].size();
        return x < y;
      });
      int c = merge(H[0], H[1]);
      H.erase(H.begin(), H.begin() + 2);
      H.push_back(c);
    }
    int c = H[0];
    for (int u : sets[c])
      if (!net.is_open(u) && cnt[u] > 0) push(u);
  }
  std::vector<int> rest;
  for (int x = 0; x < (int)sets.size(); x++)
    if (alive[x]) rest.push_back(x);
  while (rest.size() > 1) {
    std::sort(rest.begin(), rest.end(), [&](int x, int y) {
      if (sets[x].size() != sets[y].size()) return sets[x].size() < sets[y].size();
      return x < y;
    });
    int c = merge(rest[0], rest[1]);
    rest.erase(rest.begin(), rest.begin() + 2);
    rest.push_back(c);
  }
  return pairs;
}

// ------------------------------------------------------- local rotations
// Three tensors S, Y1, Y2 can be combined as ((S Y1) Y2), ((S Y2) Y1) or
// ((Y1 Y2) S); the result is the same, the intermediate differs. A pass
// visits every node whose child is an internal node and keeps the cheapest
// of the three under the time model (steps that run once at bind time cost
// nothing per group). Typical win: a large stem absorbing two small branches
// one after the other is read once instead of twice.
namespace {
struct Node {
  int l = -1, r = -1;
};
// Estimated cost of ((X Y) Z) -> O (steps that run once at bind time cost
// nothing), and in *wbits the size of W = (X Y). W keeps the indices of X and
// Y that are open or also held by Z or O. The step classes (those classify()
// gives) come from one merge over the sorted sets, without allocation.
double two_step_cost(const std::vector<int> &X, const std::vector<int> &Y, const std::vector<int> &Z,
                     const std::vector<int> &O, bool vxy, bool vz, const Network &net, const CostModel &cm,
                     int *wbits) {
  constexpr int kEnd = std::numeric_limits<int>::max();
  size_t ix = 0, iy = 0, iz = 0, io = 0;
  int b1 = 0, c1 = 0, a1 = 0, f1 = 0, b2 = 0, c2 = 0, a2 = 0, f2 = 0, w = 0;
  for (;;) {
    const int hx = ix < X.size() ? X[ix] : kEnd, hy = iy < Y.size() ? Y[iy] : kEnd, hz = iz < Z.size() ? Z[iz] : kEnd;
    const int i = std::min(hx, std::min(hy, hz));
    if (i == kEnd) break;
    const bool inX = hx == i, inY = hy == i, inZ = hz == i;
    ix += inX;
    iy += inY;
    iz += inZ;
    while (io < O.size() && O[io] < i) io++;
    const bool inO = io < O.size() && O[io] == i;
    bool inW = false;
    if (inX || inY) {
      inW = net.is_open(i) || inZ || inO;
      if (inX && inY)
        (inW ? b1 : c1)++;
      else if (inX)
        a1++;
      else
        f1++;
    }
    if (inW) {
      w++;
      if (inZ)
        (inO ? b2 : c2)++;
      else
        a2++;
    } else if (inZ) {
      f2++;
    }
  }
  *wbits = w;
  return (vxy ? cm.step_time_sizes(b1, c1, a1, f1) : 0.0) + ((vxy || vz) ? cm.step_time_sizes(b2, c2, a2, f2) : 0.0);
}

StepInfo classify(const std::vector<int> &x, const std::vector<int> &y, const std::vector<int> &c, bool var) {
  StepInfo st;
  for (int i : x) {
    bool iny = std::binary_search(y.begin(), y.end(), i), inc = std::binary_search(c.begin(), c.end(), i);
    if (iny)
      (inc ? st.batch : st.contr).push_back(i);
    else
      st.freeA.push_back(i);
  }
  for (int i : y)
    if (!std::binary_search(x.begin(), x.end(), i)) st.freeB.push_back(i);
  st.var = var;
  return st;
}
}  // namespace

Pairs rotate_tree(const Network &net, const Pairs &pairs, const std::vector<char> &sliced, const CostModel &cm,
                  int max_passes) {
  const int L = (int)net.leaves.size();
  Pairs cur = pairs;
  for (int pass = 0; pass < max_passes; pass++) {
    TreeInfo ti = analyse_tree(net, cur, sliced);
    const int NS = (int)cur.size();
    std::vector<Node> nd(L + NS);
    for (int s = 0; s < NS; s++) nd[L + s] = {cur[s].first, cur[s].second};
    std::vector<char> touched(L + NS, 0);
    bool changed = false;
    for (int q = L; q < L + NS; q++) {
      if (touched[q]) continue;
      for (int side = 0; side < 2; side++) {
        const int p = side == 0 ? nd[q].l : nd[q].r;
        const int y2 = side == 0 ? nd[q].r : nd[q].l;
        if (p < L || touched[p]) continue;
        const int s0 = nd[p].l, y1 = nd[p].r;
        const auto &Out = ti.sets[q];
        // the three ways: first pair, then the third tensor (k = 0 is the
        // current arrangement)
        const int first[3][2] = {{s0, y1}, {s0, y2}, {y1, y2}};
        const int third[3] = {y2, y1, s0};
        double best = 0, c0 = 0;
        int best_k = 0;
        for (int k = 0; k < 3; k++) {
          const auto &X = ti.sets[first[k][0]], &Y = ti.sets[first[k][1]], &Z = ti.sets[third[k]];
          const bool vxy = ti.var[first[k][0]] || ti.var[first[k][1]];
          int wbits = 0;
          const double c = two_step_cost(X, Y, Z, Out, vxy, ti.var[third[k]] != 0, net, cm, &wbits);
          if (k == 0) c0 = c;
          if (k > 0 && wbits > ti.max_bits) continue;  // never raise the memory peak
          if (k == 0 || c < best) {
            best = c;
            best_k = k;
          }
        }
        if (best_k == 0) continue;
        // keep it only if clearly cheaper than the current arrangement
        if (best >= 0.98 * c0) continue;
        nd[p] = {first[best_k][0], first[best_k][1]};
        if (side == 0)
          nd[q] = {p, third[best_k]};
        else
          nd[q] = {third[best_k], p};
        touched[p] = touched[q] = 1;
        changed = true;
        break;
      }
    }
    if (!changed) break;
    // re-linearise: post-order from the root
    Pairs out;
    std::vector<int> newid(L + NS, -1);
    for (int l = 0; l < L; l++) newid[l] = l;
    std::vector<std::pair<int, int>> stack;  // (node, state)
    stack.push_back({L + NS - 1, 0});
    while (!stack.empty()) {
      auto [n, st] = stack.back();
      stack.pop_back();
      if (n < L) continue;
      if (st == 0) {
        stack.push_back({n, 1});
        stack.push_back({nd[n].r, 0});
        stack.push_back({nd[n].l, 0});
      } else {
        out.push_back({newid[nd[n].l], newid[nd[n].r]});
        newid[n] = L + (int)out.size() - 1;
      }
    }
    cur = out;
  }
  return cur;
}

// ------------------------------------------------- subtree reconfiguration
// A window is a node v and the subtrees below it down to a frontier of at
// most `window` nodes (grown by opening the largest internal frontier node
// first). The contraction of the frontier nodes into v is re-solved exactly:
// dynamic programming over all subsets of the frontier, each subset's tensor
// holding the indices that some tensor outside the subset still holds, at the
// cost of the time model (steps that run once at bind time cost nothing per
// group), never exceeding the tree's largest intermediate. The cheapest order
// replaces the window when it saves at least 1 %. A pass skips windows that
// overlap one already rewritten; passes repeat until nothing improves.
Pairs reconfigure_tree(const Network &net, const Pairs &pairs, const std::vector<char> &sliced, const CostModel &cm,
                       int window, int max_passes) {
  const int L = (int)net.leaves.size();
  const int I = (int)net.indices.size();
  window = std::max(3, std::min(window, 10));
  Pairs cur = pairs;
  // leaves holding each index (sliced indices are not held)
  std::vector<int> total(I, 0);
  for (int l = 0; l < L; l++)
    for (int i : net.leaves[l].idx)
      if (sliced.empty() || !sliced[i]) total[i]++;
  for (int pass = 0; pass < max_passes; pass++) {
    TreeInfo ti = analyse_tree(net, cur, sliced);
    const int NS = (int)cur.size();
    std::vector<Node> nd(L + NS);
    for (int s = 0; s < NS; s++) nd[L + s] = {cur[s].first, cur[s].second};
    // leaves under each node holding each index of its set (same order as
    // the set)
    std::vector<std::vector<int>> cnt(L + NS);
    for (int l = 0; l < L; l++) cnt[l].assign(ti.sets[l].size(), 1);
    for (int s = 0; s < NS; s++) {
      const int c = L + s, a = nd[c].l, b = nd[c].r;
      const auto &C = ti.sets[c];
      cnt[c].assign(C.size(), 0);
      for (int side = 0; side < 2; side++) {
        const int u = side ? b : a;
        const auto &U = ti.sets[u];
        size_t q = 0;
        for (size_t j = 0; j < U.size(); j++) {
          while (q < C.size() && C[q] < U[j]) q++;
          if (q < C.size() && C[q] == U[j]) cnt[c][q] += cnt[u][j];
        }
      }
    }
    auto step_cost = [&](const std::vector<int> &x, const std::vector<int> &y, const std::vector<int> &out, bool var) {
      return var ? cm.step_time(classify(x, y, out, var)) : 0.0;
    };
    std::vector<char> touched(L + NS, 0);
    bool changed = false;
    const int M = window;
    for (int v = L + NS - 1; v >= L; v--) {
      if (touched[v]) continue;
      // grow the frontier
      std::vector<int> front = {nd[v].l, nd[v].r}, inner = {v};
      while ((int)front.size() < M) {
        int pick = -1;
        for (int j = 0; j < (int)front.size(); j++) {
          const int u = front[j];
          if (u < L || touched[u]) continue;
          if (pick < 0 || ti.sets[u].size() > ti.sets[front[pick]].size() ||
              (ti.sets[u].size() == ti.sets[front[pick]].size() && u > front[pick]))
            pick = j;
        }
        if (pick < 0) break;
        const int u = front[pick];
        front[pick] = nd[u].l;
        front.push_back(nd[u].r);
        inner.push_back(u);
      }
      const int m = (int)front.size();
      if (m < 3) continue;
      bool skip = false;
      for (int u : inner) skip |= touched[u] != 0;
      if (skip) continue;
      // current cost of the window's steps
      double cur_cost = 0;
      for (int u : inner) cur_cost += step_cost(ti.sets[nd[u].l], ti.sets[nd[u].r], ti.sets[u], ti.var[u]);
      // subset tensors: index j of the local universe survives when some
      // leaf outside the subset holds it, or it is open
      std::vector<int> uni;
      for (int u : front) uni.insert(uni.end(), ti.sets[u].begin(), ti.sets[u].end());
      std::sort(uni.begin(), uni.end());
      uni.erase(std::unique(uni.begin(), uni.end()), uni.end());
      const int U = (int)uni.size();
      std::vector<std::vector<int>> fc(m, std::vector<int>(U, 0));
      for (int k = 0; k < m; k++) {
        const auto &S = ti.sets[front[k]];
        for (size_t j = 0; j < S.size(); j++)
          fc[k][std::lower_bound(uni.begin(), uni.end(), S[j]) - uni.begin()] = cnt[front[k]][j];
      }
      const int full = (1 << m) - 1;
      std::vector<std::vector<int>> sub(1 << m);
      std::vector<char> svar(1 << m, 0);
      std::vector<int> scount(U);
      for (int mask = 1; mask <= full; mask++) {
        std::fill(scount.begin(), scount.end(), 0);
        bool var = false;
        for (int k = 0; k < m; k++)
          if (mask >> k & 1) {
            for (int j = 0; j < U; j++) scount[j] += fc[k][j];
            var |= ti.var[front[k]] != 0;
          }
        for (int j = 0; j < U; j++)
          if (scount[j] > 0 && (scount[j] < total[uni[j]] || net.is_open(uni[j]))) sub[mask].push_back(uni[j]);
        svar[mask] = var;
      }
      const double INF = 1e300;
      std::vector<double> best(1 << m, INF);
      std::vector<int> split(1 << m, 0);
      for (int k = 0; k < m; k++) best[1 << k] = 0;
      for (int mask = 1; mask <= full; mask++) {
        if ((mask & (mask - 1)) == 0) continue;
        if (mask != full && (int)sub[mask].size() > ti.max_bits) continue;  // never raise the memory peak
        const int low = mask & -mask;
        for (int a = (mask - 1) & mask; a > 0; a = (a - 1) & mask) {
          if (!(a & low)) continue;  // each unordered split once
          const int b = mask ^ a;
          if (best[a] >= INF || best[b] >= INF) continue;
          const double c = best[a] + best[b] + step_cost(sub[a], sub[b], sub[mask], svar[a] || svar[b]);
          if (c < best[mask]) {
            best[mask] = c;
            split[mask] = a;
          }
        }
      }
      if (best[full] >= 0.99 * cur_cost) continue;
      // rebuild the window on its own internal node ids, v as the root
      std::vector<int> ids(inner.begin() + 1, inner.end());
      size_t next_id = 0;
      std::function<int(int, int)> emit = [&](int mask, int as) -> int {
        if ((mask & (mask - 1)) == 0) return front[__builtin_ctz(mask)];
        const int node = as >= 0 ? as : ids[next_id++];
        const int a = split[mask];
        const int l = emit(a, -1), r = emit(mask ^ a, -1);
        nd[node] = {l, r};
        return node;
      };
      emit(full, v);
      for (int u : inner) touched[u] = 1;
      changed = true;
    }
    if (!changed) break;
    // re-linearise: post-order from the root
    Pairs out;
    std::vector<int> newid(L + NS, -1);
    for (int l = 0; l < L; l++) newid[l] = l;
    std::vector<std::pair<int, int>> stack;
    stack.push_back({L + NS - 1, 0});
    while (!stack.empty()) {
      auto [n, st] = stack.back();
      stack.pop_back();
      if (n < L) continue;
      if (st == 0) {
        stack.push_back({n, 1});
        stack.push_back({nd[n].r, 0});
        stack.push_back({nd[n].l, 0});
      } else {
        out.push_back({newid[nd[n].l], newid[nd[n].r]});
        newid[n] = L + (int)out.size() - 1;
      }
    }
    cur = out;
  }
  return cur;
}

// ------------------------------------------------------------------ slicing
std::vector<int> select_slices(const Network &net, const Pairs &pairs, int log2_max, int k_max,
                               const CostModel &cm) {
  std::vector<char> sliced(net.indices.size(), 0);
  std::vector<int> out;
  while ((int)out.size() < k_max) {
    TreeInfo ti = analyse_tree(net, pairs, sliced);
    if (ti.max_bits <= log2_max) break;
    std::vector<int> cands;
    for (const auto &s : ti.sets)
      if ((int)s.size() == ti.max_bits)
        for (int i : s)
          if (!net.is_open(i)) cands.push_back(i);
    std::sort(cands.begin(), cands.end());
    cands.erase(std::unique(cands.begin(), cands.end()), cands.end());
    if (cands.empty()) break;
    int best = -1;
    int best_max = 1 << 30;
    double best_cost = 0;
    // each step's estimate without slicing, reused for the steps a
    // candidate does not touch (summed in step order)
    const int NQ = (int)ti.steps.size();
    std::vector<double> base(NQ);
    for (int q = 0; q < NQ; q++) base[q] = cm.step_time(ti.steps[q]);
    // per candidate: the largest tensors holding it, and the steps holding
    // it with its class there (0 batch, 1 summed, 2 A only, 3 B only; the
    // classes of a step are disjoint)
    std::vector<char> is_cand(net.indices.size(), 0);
    for (int e : cands) is_cand[e] = 1;
    int n_top = 0;
    std::vector<int> top_holders(net.indices.size(), 0);
    for (const auto &st_set : ti.sets)
      if ((int)st_set.size() == ti.max_bits) {
        n_top++;
        for (int i : st_set) top_holders[i]++;
      }
    std::vector<std::vector<std::pair<int, int>>> held(net.indices.size());
    for (int q = 0; q < NQ; q++) {
      const StepInfo &st = ti.steps[q];
      const std::vector<int> *cls[4] = {&st.batch, &st.contr, &st.freeA, &st.freeB};
      for (int c = 0; c < 4; c++)
        for (int i : *cls[c])
          if (is_cand[i]) held[i].push_back({q, c});
    }
    for (int e : cands) {
      // slicing e shrinks every tensor holding it by one bit: the peak stays
      // unless every largest tensor holds e
      const int mx = top_holders[e] < n_top ? ti.max_bits : ti.max_bits - 1;
      double cost = 0;
      const auto &lst = held[e];
      size_t p = 0;
      for (int q = 0; q < NQ; q++) {
        const StepInfo &st = ti.steps[q];
        const bool has_e = p < lst.size() && lst[p].first == q;
        if (!st.var && !has_e) continue;  // stays a bind-time step
        if (!has_e) {
          cost += base[q];
          continue;
        }
        const int where = lst[p++].second;
        cost += cm.step_time_sizes((int)st.batch.size() - (where == 0), (int)st.contr.size() - (where == 1),
                                   (int)st.freeA.size() - (where == 2), (int)st.freeB.size() - (where == 3));
      }
      cost *= 2.0;  // twice as many slices
      if (best < 0 || mx < best_max || (mx == best_max && cost < best_cost)) {
        best = e;
        best_max = mx;
        best_cost = cost;
      }
    }
    sliced[best] = 1;
    out.push_back(best);
  }
  return out;
}

}  // namespace tz
