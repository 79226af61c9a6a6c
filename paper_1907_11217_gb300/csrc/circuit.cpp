// Circuits: spec parsing, the Sec. 1 prescription generator, spec writing.
#include <algorithm>
#include <cstring>
#include <map>
#include <set>
#include <sstream>

#include "tz_internal.h"

namespace tz {

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): Weyl step then finaliser.
uint64_t splitmix64_next(uint64_t &state) {
  state += 0x9E3779B97F4A7C15ULL;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static const char *kGateName[] = {"h", "cz", "t", "x_1_2", "y_1_2"};

static int gate_type(const std::string &s) {
  for (int i = 0; i < 5; i++)
    if (s == kGateName[i]) return i;
  return -1;
}

Circuit parse_spec(const char *text, size_t len) {
  if (!text) fail(TZ_EINVAL, "spec text is NULL");
  std::string s(text, len);
  std::istringstream in(s);
  std::string line;
  Circuit c;
  bool have_n = false;
  int lineno = 0;
  while (std::getline(in, line)) {
    lineno++;
    size_t p = line.find_first_not_of(" \t\r");
    if (p == std::string::npos || line[p] == '#') continue;
    std::istringstream ls(line);
    std::vector<std::string> tok;
    std::string t;
    while (ls >> t) tok.push_back(t);
    auto as_int = [&](const std::string &x) -> long {
      char *end = nullptr;
      long v = std::strtol(x.c_str(), &end, 10);
      if (end == x.c_str() || *end) fail(TZ_EINVAL, "line " + std::to_string(lineno) + ": not an integer: " + x);
      return v;
    };
    if (!have_n) {
      if (tok.size() != 1) fail(TZ_EINVAL, "first line must hold the qubit count");
      long n = as_int(tok[0]);
      if (n < 1 || n > 4096) fail(TZ_EINVAL, "qubit count out of range");
      c.n = (int)n;
      have_n = true;
      continue;
    }
    if (tok.size() < 3) fail(TZ_EINVAL, "line " + std::to_string(lineno) + ": expected `cycle name q0 [q1]`");
    Gate g{};
    g.cycle = (int)as_int(tok[0]);
    g.type = gate_type(tok[1]);
    if (g.type < 0) fail(TZ_EINVAL, "line " + std::to_string(lineno) + ": unknown gate " + tok[1]);
    size_t want = g.type == G_CZ ? 4 : 3;
    if (tok.size() != want) fail(TZ_EINVAL, "line " + std::to_string(lineno) + ": wrong qubit count for " + tok[1]);
    g.q0 = (int)as_int(tok[2]);
    g.q1 = g.type == G_CZ ? (int)as_int(tok[3]) : -1;
    if (g.q0 < 0 || g.q0 >= c.n || (g.type == G_CZ && (g.q1 < 0 || g.q1 >= c.n)))
      fail(TZ_EINVAL, "line " + std::to_string(lineno) + ": qubit out of range");
    if (g.type == G_CZ && g.q0 == g.q1) fail(TZ_EINVAL, "line " + std::to_string(lineno) + ": cz on one qubit");
    c.gates.push_back(g);
  }
  if (!have_n) fail(TZ_EINVAL, "empty spec");
  return c;
}

std::string circuit_spec(const Circuit &c) {
  std::ostringstream o;
  o << c.n << "\n";
  for (const Gate &g : c.gates) {
    o << g.cycle << " " << kGateName[g.type] << " " << g.q0;
    if (g.type == G_CZ) o << " " << g.q1;
    o << "\n";
  }
  return o.str();
}

// Lattice sites in row-major order.
static std::vector<std::pair<int, int>> lattice_sites(const tz_lattice &lat) {
  std::vector<std::pair<int, int>> s;
  if (lat.kind == TZ_LATTICE_GRID) {
    if (lat.rows < 1 || lat.cols < 1 || (long)lat.rows * lat.cols > 4096) fail(TZ_EINVAL, "bad grid size");
    for (int r = 0; r < lat.rows; r++)
      for (int c = 0; c < lat.cols; c++) s.push_back({r, c});
  } else if (lat.kind == TZ_LATTICE_BRISTLECONE) {
    if (lat.n_qubits != 70 && lat.n_qubits != 72) fail(TZ_EINVAL, "bristlecone lattice has 70 or 72 qubits");
    for (int r = 0; r < 11; r++) {
      int m = std::min(r, 10 - r);
      for (int c = 5 - m; c < 7 + m; c++) {
        if (lat.n_qubits == 70 && r == 5 && (c == 0 || c == 11)) continue;
        s.push_back({r, c});
      }
    }
  } else {
    fail(TZ_EINVAL, "unknown lattice kind");
  }
  return s;
}

static int pymod(int a, int m) { return ((a % m) + m) % m; }

Circuit generate_circuit(const tz_lattice &lat, int depth_t, uint64_t seed) {
  if (depth_t < 0 || depth_t > 100000) fail(TZ_EINVAL, "depth out of range");
  auto sites = lattice_sites(lat);
  std::map<std::pair<int, int>, int> index;
  for (size_t q = 0; q < sites.size(); q++) index[sites[q]] = (int)q;
  const int n = (int)sites.size();
  // pattern order H0 V0 H2 V2 H1 V1 H3 V3
  static const int kind[8] = {0, 1, 0, 1, 0, 1, 0, 1};
  static const int off[8] = {0, 0, 2, 2, 1, 1, 3, 3};
  Circuit c;
  c.n = n;
  for (int q = 0; q < n; q++) c.gates.push_back({0, G_H, q, -1});
  std::vector<int> prev(n, G_H), cur(n);
  uint64_t rng = seed;
  for (int t = 1; t <= depth_t; t++) {
    int p = (t - 1) % 8;
    std::vector<std::pair<int, int>> edges;
    for (auto &s : sites) {
      int r = s.first, col = s.second;
      if (kind[p] == 0) {
        if (pymod(col - off[p] - 2 * (r % 2), 4) == 0 && index.count({r, col + 1}))
          edges.push_back({index[s], index[{r, col + 1}]});
      } else {
        if (pymod(r - off[p] - 2 * (col % 2), 4) == 0 && index.count({r + 1, col}))
          edges.push_back({index[s], index[{r + 1, col}]});
      }
    }
    for (auto &e : edges)
      if (e.first > e.second) std::swap(e.first, e.second);
    std::sort(edges.begin(), edges.end());
    std::vector<char> in_cz(n, 0);
    for (auto &e : edges) {
      in_cz[e.first] = in_cz[e.second] = 1;
      c.gates.push_back({t, G_CZ, e.first, e.second});
    }
    for (int q = 0; q < n; q++) {
      if (in_cz[q]) {
        cur[q] = G_CZ;
        continue;
      }
      int g = -1;
      if (prev[q] == G_CZ)
        g = (splitmix64_next(rng) >> 63) ? G_SY : G_SX;
      else if (prev[q] == G_H || prev[q] == G_SX || prev[q] == G_SY)
        g = G_T;
      if (g >= 0) c.gates.push_back({t, g, q, -1});
      cur[q] = g;
    }
    prev = cur;
  }
  for (int q = 0; q < n; q++) c.gates.push_back({depth_t + 1, G_H, q, -1});
  return c;
}

}  // namespace tz
