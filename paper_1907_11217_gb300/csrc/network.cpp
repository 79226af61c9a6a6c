// Hypergraph tensor network of a circuit (Sec. 1: each node holds a tensor,
// each hyperedge is a running index), with exact simplifications.
#include <algorithm>
#include <cmath>
#include <set>

#include "tz_internal.h"

namespace tz {

namespace {

// Gate matrices U[out][in] (standard definitions; principal square roots).
void gate_matrix(int type, cd U[2][2]) {
  const double s = 1.0 / std::sqrt(2.0);
  const cd p(0.5, 0.5), m(0.5, -0.5);
  switch (type) {
    case G_H: U[0][0] = s; U[0][1] = s; U[1][0] = s; U[1][1] = -s; break;
    case G_SX: U[0][0] = p; U[0][1] = m; U[1][0] = m; U[1][1] = p; break;
    case G_SY: U[0][0] = p; U[0][1] = -p; U[1][0] = p; U[1][1] = p; break;
    default: fail(TZ_EINVAL, "not a non-diagonal one-qubit gate");
  }
}

struct Builder {
  Network net;
  std::vector<char> live;
  std::vector<std::set<int>> holders;

  int add_index(int q, int seg) {
    net.indices.push_back({q, seg});
    holders.emplace_back();
    return (int)net.indices.size() - 1;
  }
  int add_leaf(Leaf L) {
    int id = (int)net.leaves.size();
    for (int i : L.idx) holders[i].insert(id);
    net.leaves.push_back(std::move(L));
    live.push_back(1);
    return id;
  }
  void kill(int id) {
    for (int i : net.leaves[id].idx) holders[i].erase(id);
    live[id] = 0;
  }
  int rank_circuit(int id) const {
    const Leaf &L = net.leaves[id];
    return L.kind == LEAF_OUTPUT ? L.rc : (int)L.idx.size();
  }

  // Contract CONST leaf B into CONST leaf P (P keeps its storage order,
  // minus indices held by nobody else afterwards).
  void merge_const(int P, int B) {
    Leaf &lp = net.leaves[P];
    const Leaf &lb = net.leaves[B];
    std::vector<int> uni = lp.idx;
    for (int i : lb.idx)
      if (std::find(uni.begin(), uni.end(), i) == uni.end()) uni.push_back(i);
    std::vector<int> out;
    for (int i : uni) {
      bool inP = std::count(lp.idx.begin(), lp.idx.end(), i) > 0;
      bool inB = std::count(lb.idx.begin(), lb.idx.end(), i) > 0;
      int after = (int)holders[i].size() - (inP ? 1 : 0) - (inB ? 1 : 0) + 1;
      if (after > 1 || net.is_open(i)) out.push_back(i);
    }
    std::vector<cd> data(size_t(1) << out.size(), cd(0, 0));
    const int u = (int)uni.size();
    for (uint64_t v = 0; v < (uint64_t(1) << u); v++) {
      auto off = [&](const std::vector<int> &idx) {
        uint64_t o = 0;
        for (size_t p = 0; p < idx.size(); p++) {
          int pos = (int)(std::find(uni.begin(), uni.end(), idx[p]) - uni.begin());
          o |= ((v >> pos) & 1) << p;
        }
        return o;
      };
      data[off(out)] += lp.data[off(lp.idx)] * lb.data[off(lb.idx)];
    }
    for (int i : lp.idx) holders[i].erase(P);
    lp.idx = out;
    lp.data = std::move(data);
    for (int i : lp.idx) holders[i].insert(P);
  }
};

}  // namespace

Network build_network(const Circuit &c, int batch_log2, const std::vector<int> &open_qubits) {
  if (batch_log2 < 0 || batch_log2 > 8) fail(TZ_EINVAL, "batch_log2 must be in 0..8");
  Builder b;
  b.net.n_qubits = c.n;
  b.net.batch_log2 = batch_log2;
  const int n = c.n;
  std::vector<int> opened(open_qubits);
  std::sort(opened.begin(), opened.end());
  if ((int)opened.size() > kMaxOpenQubits)
    fail(TZ_EINVAL, "at most " + std::to_string(kMaxOpenQubits) + " open output qubits");
  for (size_t j = 0; j < opened.size(); j++) {
    if (opened[j] < 0 || opened[j] >= n) fail(TZ_EINVAL, "open qubit out of range");
    if (j && opened[j] == opened[j - 1]) fail(TZ_EINVAL, "open qubit listed twice");
  }
  if (n > 0 && (int)opened.size() >= n) fail(TZ_EINVAL, "at least one output qubit must stay closed");
  std::vector<char> is_opened(n, 0);
  for (int q : opened) is_opened[q] = 1;
  std::vector<int> cur(n), seg(n, 0);
  for (int q = 0; q < n; q++) {
    cur[q] = b.add_index(q, 0);
    Leaf L;
    L.idx = {cur[q]};
    L.data = {cd(1, 0), cd(0, 0)};  // |0>
    b.add_leaf(L);
  }
  const cd w = std::polar(1.0, M_PI / 4.0);
  for (const Gate &g : c.gates) {
    if (g.type == G_CZ) {
      Leaf L;
      L.idx = {cur[g.q0], cur[g.q1]};
      L.data = {cd(1, 0), cd(1, 0), cd(1, 0), cd(-1, 0)};
      b.add_leaf(L);
    } else if (g.type == G_T) {
      Leaf L;
      L.idx = {cur[g.q0]};
      L.data = {cd(1, 0), w};
      b.add_leaf(L);
    } else {
      cd U[2][2];
      gate_matrix(g.type, U);
      int q = g.q0;
      int nw = b.add_index(q, ++seg[q]);
      Leaf L;
      L.idx = {cur[q], nw};  // storage: old is bit 0, new is bit 1
      L.data.resize(4);
      for (int o = 0; o < 2; o++)
        for (int i = 0; i < 2; i++) L.data[i + 2 * o] = U[o][i];
      b.add_leaf(L);
      cur[q] = nw;
    }
  }
  // An open output qubit has no output tensor: its last wire index stays
  // open to the end, and its value is the qubit's output bit.
  for (size_t j = 0; j < opened.size(); j++) b.net.indices[cur[opened[j]]] = Index{-2, (int)j};
  std::vector<int> beta;
  for (int k = 0; k < batch_log2; k++) beta.push_back(b.add_index(-1, k));
  for (int q = 0; q < n; q++) {
    if (is_opened[q]) continue;
    Leaf L;
    L.kind = LEAF_OUTPUT;
    L.qubit = q;
    L.rc = 1;
    L.idx = {cur[q]};
    for (int k : beta) L.idx.push_back(k);
    L.data = {cd(1, 0), cd(0, 0), cd(0, 0), cd(1, 0)};  // M[x*2+e] = [x == e]
    b.add_leaf(L);
  }

  // Simplify: fold rank-1 constant tensors into a neighbour, and the last
  // gate of each wire into its output tensor, until nothing changes.
  bool changed = true;
  while (changed) {
    changed = false;
    for (int id = 0; id < (int)b.net.leaves.size(); id++) {
      if (!b.live[id]) continue;
      Leaf &L = b.net.leaves[id];
      if (L.kind != LEAF_CONST) continue;
      if (L.idx.empty()) {
        b.net.scalar *= L.data[0];
        b.kill(id);
        changed = true;
        continue;
      }
      if (L.idx.size() != 1) continue;
      int i = L.idx[0];
      int best = -1;
      for (int p : b.holders[i]) {
        if (p == id) continue;
        const Leaf &P = b.net.leaves[p];
        auto key = [&](int x) {
          const Leaf &X = b.net.leaves[x];
          return std::make_pair(X.kind == LEAF_OUTPUT ? 1 : 0, (int)X.idx.size() * 100000 + x);
        };
        (void)P;
        if (best < 0 || key(p) < key(best)) best = p;
      }
      if (best < 0) {  // index held by nobody else: sum it out
        if (b.net.is_open(i)) continue;  // unless it is open: the factor stays
        b.net.scalar *= L.data[0] + L.data[1];
        b.kill(id);
        changed = true;
        continue;
      }
      Leaf &P = b.net.leaves[best];
      if (P.kind == LEAF_CONST) {
        b.merge_const(best, id);
      } else {  // output tensor: scale its table along e, or sum e out
        std::vector<cd> v = L.data;
        bool last = b.holders[i].size() == 2;
        std::vector<cd> M(2);
        if (last) {
          for (int x = 0; x < 2; x++) M[x] = P.data[x * 2 + 0] * v[0] + P.data[x * 2 + 1] * v[1];
          b.holders[i].erase(best);
          P.idx.erase(P.idx.begin());
          P.rc = 0;
          P.data = M;
        } else {
          for (int x = 0; x < 2; x++)
            for (int e = 0; e < 2; e++) P.data[x * 2 + e] *= v[e];
        }
      }
      b.kill(id);
      changed = true;
    }
    for (int id = 0; id < (int)b.net.leaves.size(); id++) {
      if (!b.live[id]) continue;
      Leaf &O = b.net.leaves[id];
      if (O.kind != LEAF_OUTPUT || O.rc != 1) continue;
      int e = O.idx[0];
      if (b.holders[e].size() != 2) continue;
      int u = *b.holders[e].begin() == id ? *b.holders[e].rbegin() : *b.holders[e].begin();
      Leaf &U = b.net.leaves[u];
      if (U.kind != LEAF_CONST || U.idx.size() != 2) continue;
      int pe = U.idx[0] == e ? 0 : 1;
      int e2 = U.idx[1 - pe];
      std::vector<cd> M(4, cd(0, 0));
      for (int x = 0; x < 2; x++)
        for (int v2 = 0; v2 < 2; v2++)
          for (int v = 0; v < 2; v++) {
            int off = pe == 0 ? (v | (v2 << 1)) : (v2 | (v << 1));
            M[x * 2 + v2] += O.data[x * 2 + v] * U.data[off];
          }
      b.kill(u);
      b.holders[e].erase(id);
      O.idx[0] = e2;
      O.data = M;
      b.holders[e2].insert(id);
      changed = true;
    }
  }

  // Compact: keep live leaves, renumber the indices they use (and the batch
  // indices) in order of first appearance.
  Network out;
  out.n_qubits = n;
  out.batch_log2 = batch_log2;
  out.n_open = (int)opened.size();
  out.open_qubits = opened;
  out.scalar = b.net.scalar;
  std::vector<int> remap(b.net.indices.size(), -1);
  auto map_index = [&](int i) {
    if (remap[i] < 0) {
      remap[i] = (int)out.indices.size();
      out.indices.push_back(b.net.indices[i]);
    }
    return remap[i];
  };
  for (int k : beta) map_index(k);
  for (size_t id = 0; id < b.net.leaves.size(); id++) {
    if (!b.live[id]) continue;
    Leaf L = b.net.leaves[id];
    for (int &i : L.idx) i = map_index(i);
    out.leaves.push_back(std::move(L));
  }
  return out;
}

}  // namespace tz
