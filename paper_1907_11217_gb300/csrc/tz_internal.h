// Internal declarations of the amplitude library (host side).
#pragma once
#include <complex>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "tz.h"

namespace tz {

using cd = std::complex<double>;

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};
[[noreturn]] inline void fail(int code, const std::string &msg) { throw Error(code, msg); }

// ------------------------------------------------------------------ circuits
enum GateType { G_H = 0, G_CZ = 1, G_T = 2, G_SX = 3, G_SY = 4 };
struct Gate {
  int cycle, type, q0, q1;
};
struct Circuit {
  int n = 0;
  std::vector<Gate> gates;
};
Circuit parse_spec(const char *text, size_t len);
Circuit generate_circuit(const tz_lattice &lat, int depth_t, uint64_t seed);
std::string circuit_spec(const Circuit &c);

// ------------------------------------------------------------------ networks
struct Index {
  int qubit;    // -1 for a batch (bitstring) index, -2 for an open output qubit
  int segment;  // wire segment, batch bit number, or open bit number
};
enum LeafKind { LEAF_CONST = 0, LEAF_OUTPUT = 1 };
struct Leaf {
  int kind = LEAF_CONST;
  // Storage order: idx[p] is bit p of the linear element offset. OUTPUT
  // leaves list their circuit index (0 or 1 of them) first, then the batch
  // indices in bit order.
  std::vector<int> idx;
  // CONST: 2^rank values. OUTPUT: table M[x * 2^rc + e], x the output bit of
  // the leaf's qubit, e the value of its circuit index (rc = 0 or 1).
  std::vector<cd> data;
  int qubit = -1;
  int rc = 0;  // OUTPUT: number of circuit indices (0 or 1)
};
struct Network {
  int n_qubits = 0, batch_log2 = 0;
  // Open output qubits: bit j of an amplitude's open value is the output bit
  // of qubit open_qubits[j] (ascending); every bitstring yields 2^n_open
  // amplitudes, its own bits on those qubits ignored.
  int n_open = 0;
  std::vector<int> open_qubits;
  std::vector<Index> indices;
  std::vector<Leaf> leaves;
  cd scalar{1.0, 0.0};  // global factor of the amplitude
  // kept to the end of the contraction: batch indices and open output qubits
  bool is_open(int i) const { return indices[i].qubit < 0; }
  bool is_batch(int i) const { return indices[i].qubit == -1; }
};
constexpr int kMaxOpenQubits = 12;
Network build_network(const Circuit &c, int batch_log2, const std::vector<int> &open_qubits = {});

// ------------------------------------------------------- trees and analysis
using Pairs = std::vector<std::pair<int, int>>;

// One contraction step of a tree, with its index classes (sliced indices
// removed). Index ids are sorted in each list.
struct StepInfo {
  int a, b, c;
  std::vector<int> batch, contr, freeA, freeB;  // a∩b kept, a∩b summed, a only, b only
  bool var;                                     // depends on the group (slice or bitstrings)
  int bitsA() const { return (int)(batch.size() + contr.size() + freeA.size()); }
  int bitsB() const { return (int)(batch.size() + contr.size() + freeB.size()); }
  int bitsC() const { return (int)(batch.size() + freeA.size() + freeB.size()); }
  int bitsAll() const { return (int)(batch.size() + contr.size() + freeA.size() + freeB.size()); }
};
struct TreeInfo {
  std::vector<std::vector<int>> sets;  // index set of every node (leaves then steps)
  std::vector<char> var;               // per node
  std::vector<StepInfo> steps;
  int max_bits = 0;                    // largest node (var nodes and const nodes)
};
// sliced: flag per index (may be empty).
TreeInfo analyse_tree(const Network &net, const Pairs &pairs, const std::vector<char> &sliced);
void validate_tree(const Network &net, const Pairs &pairs);

// Estimated GB300 time (seconds) of one group of a plan (var steps) and of
// the bind-time part (const steps).
struct CostModel {
  int precision = TZ_C64_SIMT;
  double hbm_bps = 6.8e12;
  double simt_flops = 60e12;        // complex64 useful flop rate on CUDA cores
  double simt_fp64_flops = 1.0e12;  // complex128 useful flop rate (GB300's FP64 units)
  double tc_useful_flops = 300e12;  // useful flop rate of the split tensor-core product
  double small_step_s = 2.0e-6;     // fixed cost of a small step
  int small_log2 = 22;
  double step_time(const StepInfo &s) const;
  double step_time_sizes(int n_batch, int n_contr, int n_freeA, int n_freeB) const;
};
double group_time(const TreeInfo &ti, const CostModel &cm);

Pairs greedy_tree(const Network &net, double alpha, double temperature, uint64_t seed);
Pairs elimination_tree(const Network &net, double temperature, uint64_t seed);
Pairs rotate_tree(const Network &net, const Pairs &pairs, const std::vector<char> &sliced, const CostModel &cm,
                  int max_passes);
// Exact re-optimisation of windows of at most `window` subtrees (3..10).
Pairs reconfigure_tree(const Network &net, const Pairs &pairs, const std::vector<char> &sliced, const CostModel &cm,
                       int window, int max_passes);
std::vector<int> select_slices(const Network &net, const Pairs &pairs, int log2_max, int k_max,
                               const CostModel &cm);

uint64_t splitmix64_next(uint64_t &state);

}  // namespace tz
