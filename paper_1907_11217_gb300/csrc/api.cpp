// C ABI entry points (include/tz.h): argument checks, error codes, handles.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <memory>
#include <mutex>
#include <new>
#include <thread>

#include "plan.h"

struct tz_circuit {
  tz::Circuit c;
};
struct tz_network {
  tz::Network n;
};
struct tz_tree {
  tz::Pairs pairs;
};

namespace {
thread_local std::string g_err;
void set_error(const std::string &m) { g_err = m; }
bool is_tc_precision(int p) { return p == TZ_TF32X3 || p == TZ_BF16X3 || p == TZ_FP16X3; }
// tz_op_cgemm scratch of the split-precision modes: the error word of the
// call in the first 256 bytes, then the product's own scratch
constexpr size_t kOpErrBytes = 256;
}  // namespace

// shared with the other translation units that export C entry points
void tz_set_error_message(const std::string &m) { set_error(m); }

#define TZ_TRY try {
#define TZ_CATCH                           \
  }                                        \
  catch (const tz::Error &e) {             \
    set_error(e.what());                   \
    return e.code;                         \
  }                                        \
  catch (const std::bad_alloc &) {         \
    set_error("host allocation failed");   \
    return TZ_ENOMEM;                      \
  }                                        \
  catch (const std::exception &e) {        \
    set_error(e.what());                   \
    return TZ_EINVAL;                      \
  }                                        \
  return TZ_OK;

#define REQUIRE(cond, msg) \
  if (!(cond)) tz::fail(TZ_EINVAL, msg)

extern "C" {

const char *tz_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------ circuits
int tz_circuit_from_spec(const char *text, size_t len, tz_circuit **out) {
  TZ_TRY
  REQUIRE(out, "out is NULL");
  *out = nullptr;
  auto c = std::make_unique<tz_circuit>();
  c->c = tz::parse_spec(text, len);
  *out = c.release();
  TZ_CATCH
}

int tz_circuit_generate(const tz_lattice *lat, int depth_t, uint64_t seed, tz_circuit **out) {
  TZ_TRY
  REQUIRE(lat && out, "NULL argument");
  *out = nullptr;
  auto c = std::make_unique<tz_circuit>();
  c->c = tz::generate_circuit(*lat, depth_t, seed);
  *out = c.release();
  TZ_CATCH
}

int tz_circuit_n_qubits(const tz_circuit *c) { return c ? c->c.n : TZ_EINVAL; }
int tz_circuit_n_gates(const tz_circuit *c) { return c ? (int)c->c.gates.size() : TZ_EINVAL; }

int tz_circuit_to_spec(const tz_circuit *c, char *buf, size_t cap, size_t *len) {
  TZ_TRY
  REQUIRE(c && len, "NULL argument");
  std::string s = tz::circuit_spec(c->c);
  *len = s.size();
  if (!buf || cap < s.size() + 1) tz::fail(TZ_EINVAL, "buffer too small");
  std::memcpy(buf, s.c_str(), s.size() + 1);
  TZ_CATCH
}

void tz_circuit_destroy(tz_circuit *c) { delete c; }

// ------------------------------------------------------------------ networks
int tz_network_from_circuit(const tz_circuit *c, const tz_network_opts *opts, tz_network **out) {
  TZ_TRY
  REQUIRE(c && out, "NULL argument");
  *out = nullptr;
  auto n = std::make_unique<tz_network>();
  std::vector<int> open_q;
  if (opts && opts->n_open) {
    REQUIRE(opts->n_open > 0 && opts->open_qubits, "n_open > 0 needs open_qubits");
    open_q.assign(opts->open_qubits, opts->open_qubits + opts->n_open);
  }
  n->n = tz::build_network(c->c, opts ? opts->batch_log2 : 0, open_q);
  *out = n.release();
  TZ_CATCH
}

int tz_network_n_tensors(const tz_network *net) { return net ? (int)net->n.leaves.size() : TZ_EINVAL; }
int tz_network_n_indices(const tz_network *net) { return net ? (int)net->n.indices.size() : TZ_EINVAL; }

int tz_network_index_info(const tz_network *net, int index, int *qubit, int *segment) {
  TZ_TRY
  REQUIRE(net && qubit && segment, "NULL argument");
  REQUIRE(index >= 0 && index < (int)net->n.indices.size(), "index out of range");
  *qubit = net->n.indices[index].qubit;
  *segment = net->n.indices[index].segment;
  TZ_CATCH
}

int tz_network_tensor_indices(const tz_network *net, int t, int32_t *idx, int cap, int *rank) {
  TZ_TRY
  REQUIRE(net && rank, "NULL argument");
  REQUIRE(t >= 0 && t < (int)net->n.leaves.size(), "tensor out of range");
  const auto &v = net->n.leaves[t].idx;
  *rank = (int)v.size();
  REQUIRE(idx && cap >= (int)v.size(), "buffer too small");
  for (size_t i = 0; i < v.size(); i++) idx[i] = v[i];
  TZ_CATCH
}

void tz_network_destroy(tz_network *net) { delete net; }

// ------------------------------------------------------------------ trees
static tz::CostModel cost_model(int precision) {
  tz::CostModel cm;
  cm.precision = precision;
  return cm;
}

// Score of a tree: estimated time of all 2^k groups after slicing to the
// target, plus the bind-time part once.
static double tree_score(const tz::Network &net, const tz::Pairs &pairs, int log2_max, const tz::CostModel &cm,
                         int *max_bits) {
  std::vector<int> sl;
  if (log2_max > 0) sl = tz::select_slices(net, pairs, log2_max, 40, cm);
  std::vector<char> flag(net.indices.size(), 0);
  for (int e : sl) flag[e] = 1;
  tz::TreeInfo ti = tz::analyse_tree(net, pairs, flag);
  *max_bits = ti.max_bits;
  double t = std::ldexp(tz::group_time(ti, cm), (int)sl.size());
  for (const auto &s : ti.steps)
    if (!s.var) t += cm.step_time(s);
  return t;
}

int tz_path_greedy(const tz_network *net, const tz_path_opts *opts, tz_tree **out) {
  TZ_TRY
  REQUIRE(net && out, "NULL argument");
  *out = nullptr;
  tz_path_opts o{};
  o.restarts = 1;
  if (opts) o = *opts;
  if (o.restarts < 1) o.restarts = 1;
  tz::CostModel cm = cost_model(o.precision);
  REQUIRE(o.algorithm >= TZ_PATH_AUTO && o.algorithm <= TZ_PATH_ELIMINATION, "unknown path algorithm");
  REQUIRE(o.reconfigure == 0 || (o.reconfigure >= 3 && o.reconfigure <= 10), "reconfigure must be 0 or 3..10");
  // Every trial's parameters are drawn first, in trial order, from one
  // stream; the trials then run on host threads, and the earliest trial with
  // the lowest score wins. The result does not depend on the thread count.
  struct Trial {
    int algo;
    double alpha, temp;
    uint64_t seed;
  };
  std::vector<Trial> trials(o.restarts);
  uint64_t rng = o.seed ^ 0x5DEECE66DULL;
  for (int trial = 0; trial < o.restarts; trial++) {
    Trial &tr = trials[trial];
    tr.algo = o.algorithm;
    int nth = trial;  // trial number within its algorithm
    if (tr.algo == TZ_PATH_AUTO) {
      tr.algo = (trial % 2 == 0) ? TZ_PATH_ELIMINATION : TZ_PATH_GREEDY;
      nth = trial / 2;
    }
    tr.alpha = 1.0;
    tr.temp = 0.0;
    const double u1 = (tz::splitmix64_next(rng) >> 11) * (1.0 / 9007199254740992.0);
    const double u2 = (tz::splitmix64_next(rng) >> 11) * (1.0 / 9007199254740992.0);
    if (nth > 0) {
      tr.alpha = 0.5 + 1.0 * u1;
      tr.temp = 0.05 + 1.0 * u2;
    }
    tr.seed = tz::splitmix64_next(rng);
  }
  // Only the best trees are kept: each thread keeps its `keep` best, ordered
  // by (score, trial), and the lists are merged at the end.
  struct Kept {
    double score;
    int trial;
    tz::Pairs pairs;
  };
  auto before = [](const Kept &a, const Kept &b) {
    return a.score < b.score || (a.score == b.score && a.trial < b.trial);
  };
  const int keep = o.reconfigure > 0 ? 8 : 1;
  auto run_trial = [&](int i, std::vector<Kept> &mine) {
    const Trial &tr = trials[i];
    tz::Pairs pr = tr.algo == TZ_PATH_GREEDY ? tz::greedy_tree(net->n, tr.alpha, tr.temp, tr.seed)
                                             : tz::elimination_tree(net->n, tr.temp, tr.seed);
    if (o.log2_max_intermediate > 0) {
      // local three-way rotations under the slicing this tree would get
      std::vector<int> sl = tz::select_slices(net->n, pr, o.log2_max_intermediate, 40, cm);
      std::vector<char> flag(net->n.indices.size(), 0);
      for (int e : sl) flag[e] = 1;
      pr = tz::rotate_tree(net->n, pr, flag, cm, 16);
    }
    int mb = 0;
    Kept k{tree_score(net->n, pr, o.log2_max_intermediate, cm, &mb), i, std::move(pr)};
    if ((int)mine.size() == keep && !before(k, mine.back())) return;
    mine.insert(std::upper_bound(mine.begin(), mine.end(), k, before), std::move(k));
    if ((int)mine.size() > keep) mine.pop_back();
  };
  // host threads: TZ_PATH_THREADS if set (>= 1), else one per hardware thread (at most 64)
  unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  if (const char *env = std::getenv("TZ_PATH_THREADS")) {
    const long v = std::strtol(env, nullptr, 10);
    if (v >= 1) hw = (unsigned)std::min<long>(v, 1024);
  }
  const int n_threads = (int)std::min<unsigned>({(unsigned)o.restarts, hw, 64u});
  std::vector<std::vector<Kept>> kept(std::max(1, n_threads));
  if (n_threads <= 1) {
    for (int i = 0; i < o.restarts; i++) run_trial(i, kept[0]);
  } else {
    std::atomic<int> next{0};
    std::exception_ptr err;
    std::mutex err_mu;
    std::vector<std::thread> pool;
    for (int w = 0; w < n_threads; w++)
      pool.emplace_back([&, w] {
        for (int i; (i = next.fetch_add(1)) < o.restarts;) {
          try {
            run_trial(i, kept[w]);
          } catch (...) {
            std::lock_guard<std::mutex> lk(err_mu);
            if (!err) err = std::current_exception();
          }
        }
      });
    for (auto &th : pool) th.join();
    if (err) std::rethrow_exception(err);
  }
  std::vector<Kept> top;
  for (auto &mine : kept)
    for (auto &k : mine) top.push_back(std::move(k));
  std::sort(top.begin(), top.end(), before);
  if ((int)top.size() > keep) top.resize(keep);
  Kept &best = top[0];
  if (o.reconfigure > 0) {
    // exact window re-optimisation of the best few trees (best first, ties by
    // restart order); the lowest score after it wins, ties to the earlier
    const int n_top = (int)top.size();
    std::vector<Kept> refined(n_top);
    std::vector<std::thread> pool;
    std::exception_ptr err;
    std::mutex err_mu;
    for (int q = 0; q < n_top; q++)
      pool.emplace_back([&, q] {
        try {
          const Kept &src = top[q];
          std::vector<char> flag(net->n.indices.size(), 0);
          if (o.log2_max_intermediate > 0)
            for (int e : tz::select_slices(net->n, src.pairs, o.log2_max_intermediate, 40, cm)) flag[e] = 1;
          refined[q].pairs = tz::reconfigure_tree(net->n, src.pairs, flag, cm, o.reconfigure, 8);
          int mb = 0;
          refined[q].score = tree_score(net->n, refined[q].pairs, o.log2_max_intermediate, cm, &mb);
        } catch (...) {
          std::lock_guard<std::mutex> lk(err_mu);
          if (!err) err = std::current_exception();
        }
      });
    for (auto &th : pool) th.join();
    if (err) std::rethrow_exception(err);
    int rb = -1;
    for (int q = 0; q < n_top; q++)
      if (refined[q].score < best.score && (rb < 0 || refined[q].score < refined[rb].score)) rb = q;
    if (rb >= 0) {
      best.pairs = std::move(refined[rb].pairs);
      best.score = refined[rb].score;
    }
  }
  auto t = std::make_unique<tz_tree>();
  t->pairs = std::move(best.pairs);
  *out = t.release();
  TZ_CATCH
}

int tz_tree_from_pairs(const tz_network *net, const int32_t *pairs, int n_pairs, tz_tree **out) {
  TZ_TRY
  REQUIRE(net && out && (pairs || n_pairs == 0), "NULL argument");
  *out = nullptr;
  tz::Pairs pr;
  for (int i = 0; i < n_pairs; i++) pr.push_back({pairs[2 * i], pairs[2 * i + 1]});
  tz::validate_tree(net->n, pr);
  tz::analyse_tree(net->n, pr, {});
  auto t = std::make_unique<tz_tree>();
  t->pairs = pr;
  *out = t.release();
  TZ_CATCH
}

int tz_tree_pairs(const tz_tree *tree, int32_t *pairs, int cap, int *n_pairs) {
  TZ_TRY
  REQUIRE(tree && n_pairs, "NULL argument");
  *n_pairs = (int)tree->pairs.size();
  REQUIRE(pairs && cap >= (int)tree->pairs.size(), "buffer too small");
  for (size_t i = 0; i < tree->pairs.size(); i++) {
    pairs[2 * i] = tree->pairs[i].first;
    pairs[2 * i + 1] = tree->pairs[i].second;
  }
  TZ_CATCH
}

void tz_tree_destroy(tz_tree *tree) { delete tree; }

int tz_slice_select(const tz_network *net, const tz_tree *tree, int log2_max_intermediate, int k_max,
                    int32_t *sliced_edges, int *k_out) {
  TZ_TRY
  REQUIRE(net && tree && k_out, "NULL argument");
  REQUIRE(k_max >= 0 && k_max <= 40, "k_max must be in 0..40");
  REQUIRE(sliced_edges || k_max == 0, "NULL sliced_edges");
  tz::validate_tree(net->n, tree->pairs);
  std::vector<int> sl = tz::select_slices(net->n, tree->pairs, log2_max_intermediate, k_max, cost_model(TZ_C64_SIMT));
  for (size_t i = 0; i < sl.size(); i++) sliced_edges[i] = sl[i];
  *k_out = (int)sl.size();
  TZ_CATCH
}

// ------------------------------------------------------------------ plans
int tz_plan_create(const tz_network *network, const tz_tree *contraction_tree, const int32_t *sliced_edges, int k,
                   const tz_plan_opts *opts, tz_plan **out) {
  TZ_TRY
  REQUIRE(network && contraction_tree && out, "NULL argument");
  REQUIRE(k >= 0 && (k == 0 || sliced_edges), "bad sliced edge list");
  *out = nullptr;
  tz_plan_opts o{};
  if (opts) o = *opts;
  std::vector<int> sl(sliced_edges, sliced_edges + k);
  *out = tz::plan_create(network->n, contraction_tree->pairs, sl, o);
  TZ_CATCH
}

int tz_plan_stats_get(const tz_plan *plan, tz_plan_stats *out) {
  TZ_TRY
  REQUIRE(plan && out, "NULL argument");
  *out = plan->stats;
  TZ_CATCH
}

int tz_plan_bind_workspace(tz_plan *plan, void *dev_ptr, size_t bytes) {
  TZ_TRY
  REQUIRE(plan, "NULL plan");
  tz::plan_bind(plan, dev_ptr, bytes);
  TZ_CATCH
}

int tz_plan_set_slice_range(tz_plan *plan, int64_t lo, int64_t hi) {
  TZ_TRY
  REQUIRE(plan, "NULL plan");
  const int64_t n = int64_t(1) << plan->sliced.size();
  REQUIRE(0 <= lo && lo < hi && hi <= n, "slice range must satisfy 0 <= lo < hi <= 2^k");
  plan->lo = lo;
  plan->hi = hi;
  TZ_CATCH
}

int tz_plan_sliced_segments(const tz_plan *plan, int32_t *qubit_segment, int cap, int *k) {
  TZ_TRY
  REQUIRE(plan && k, "NULL argument");
  *k = (int)plan->sliced.size();
  REQUIRE(qubit_segment || plan->sliced.empty(), "NULL buffer");
  REQUIRE(cap >= (int)plan->sliced.size(), "buffer too small");
  for (size_t j = 0; j < plan->sliced.size(); j++) {
    qubit_segment[2 * j] = plan->net.indices[plan->sliced[j]].qubit;
    qubit_segment[2 * j + 1] = plan->net.indices[plan->sliced[j]].segment;
  }
  TZ_CATCH
}

static void check_rows(const tz_plan *plan, int64_t n) {
  REQUIRE(n >= 0, "bitstring count must be >= 0");
  if (n > plan->max_rows)
    tz::fail(TZ_EINVAL, "at most " + std::to_string(plan->max_rows) + " bitstrings per call");
}

int tz_contract_amplitudes(tz_plan *plan, const uint8_t *bitstrings, int64_t n, double *out) {
  TZ_TRY
  REQUIRE(plan, "NULL argument");
  check_rows(plan, n);
  if (n == 0) return TZ_OK;  // nothing to contract, nothing written
  REQUIRE(bitstrings && out, "NULL argument");
  REQUIRE(plan->bound, "plan has no workspace bound");
  const int nq = plan->net.n_qubits;
  for (int64_t i = 0; i < n * nq; i++)
    if (bitstrings[i] > 1) tz::fail(TZ_EINVAL, "bitstring bytes must be 0 or 1");
  tz::cuda_check(cudaSetDevice(plan->opts.device), "cudaSetDevice");
  const tz::RunCtx ctx = tz::default_ctx(plan);
  cudaStream_t s = ctx.stream;
  tz::cuda_check(cudaMemcpyAsync(ctx.scratch + plan->s_bits, bitstrings, (size_t)(n * nq), cudaMemcpyHostToDevice, s),
                 "copy bitstrings in");
  tz::plan_run(plan, ctx, n, plan->lo, plan->hi);
  tz::cuda_check(cudaMemcpyAsync(out, ctx.scratch + plan->s_acc, (size_t)n * 16 << plan->net.n_open,
                                 cudaMemcpyDeviceToHost, s),
                 "copy amplitudes out");
  tz::cuda_check(cudaStreamSynchronize(s), "contract");
  if (tz::read_tc_error(plan, ctx))
    tz::fail(TZ_ETIMEOUT, "a bounded wait (tensor-core product or direct-step queue) ran out; the amplitudes are invalid (NaN)");
  TZ_CATCH
}

int tz_plan_status(tz_plan *plan) {
  TZ_TRY
  REQUIRE(plan, "NULL plan");
  REQUIRE(plan->bound, "plan has no workspace bound");
  tz::cuda_check(cudaSetDevice(plan->opts.device), "cudaSetDevice");
  const tz::RunCtx ctx = tz::default_ctx(plan);
  tz::cuda_check(cudaStreamSynchronize(ctx.stream), "synchronise the plan's stream");
  if (tz::read_tc_error(plan, ctx))
    tz::fail(TZ_ETIMEOUT, "a bounded wait (tensor-core product or direct-step queue) of the last call ran out; its amplitudes are NaN");
  TZ_CATCH
}

int tz_contract_amplitudes_device(tz_plan *plan, const uint8_t *d_bitstrings, int64_t n, double *d_out) {
  TZ_TRY
  REQUIRE(plan, "NULL argument");
  check_rows(plan, n);
  if (n == 0) return TZ_OK;  // nothing to contract, nothing written
  REQUIRE(d_bitstrings && d_out, "NULL argument");
  REQUIRE(plan->bound, "plan has no workspace bound");
  tz::cuda_check(cudaSetDevice(plan->opts.device), "cudaSetDevice");
  const tz::RunCtx ctx = tz::default_ctx(plan);
  cudaStream_t s = ctx.stream;
  tz::cuda_check(cudaMemcpyAsync(ctx.scratch + plan->s_bits, d_bitstrings, (size_t)(n * plan->net.n_qubits),
                                 cudaMemcpyDeviceToDevice, s),
                 "copy bitstrings in");
  tz::plan_run(plan, ctx, n, plan->lo, plan->hi);
  tz::cuda_check(cudaMemcpyAsync(d_out, ctx.scratch + plan->s_acc, (size_t)n * 16 << plan->net.n_open,
                                 cudaMemcpyDeviceToDevice, s),
                 "copy amplitudes out");
  TZ_CATCH
}

int tz_plan_describe(const tz_plan *plan, char *buf, size_t cap, size_t *len) {
  TZ_TRY
  REQUIRE(plan && len, "NULL argument");
  std::string s = tz::plan_describe(plan);
  *len = s.size();
  if (!buf || cap < s.size() + 1) tz::fail(TZ_EINVAL, "buffer too small");
  std::memcpy(buf, s.c_str(), s.size() + 1);
  TZ_CATCH
}

void tz_plan_destroy(tz_plan *plan) { tz::plan_destroy(plan); }

int tz_plan_profile_enable(tz_plan *plan, int on) {
  TZ_TRY
  REQUIRE(plan, "NULL plan");
  if (plan->bound) tz::plan_profile_collect(plan);
  plan->prof = tz_plan_profile{};
  plan->item_ms.clear();
  plan->item_count.clear();
  plan->profiling = on != 0;
  TZ_CATCH
}

int tz_plan_profile_items(tz_plan *plan, double *out, int cap, int *n) {
  TZ_TRY
  REQUIRE(plan && n, "NULL argument");
  if (plan->bound) tz::plan_profile_collect(plan);
  const auto &items = plan->var_items;
  *n = (int)items.size();
  REQUIRE(out && cap >= (int)items.size(), "buffer too small");
  for (size_t i = 0; i < items.size(); i++) {
    int kind = 0;
    double fl = 0, by = 0;
    tz::item_cost_public(plan, (int)i, &kind, &fl, &by);
    double *o = out + 6 * i;
    o[0] = kind;
    o[1] = i < plan->item_ms.size() ? plan->item_ms[i] : 0.0;
    o[2] = fl;
    o[3] = by;
    o[4] = items[i].kind == tz::IT_GEMM ? items[i].a : -1;
    o[5] = i < plan->item_count.size() ? (double)plan->item_count[i] : 0.0;
  }
  TZ_CATCH
}

int tz_plan_profile_get(tz_plan *plan, tz_plan_profile *out) {
  TZ_TRY
  REQUIRE(plan && out, "NULL argument");
  if (plan->bound) tz::plan_profile_collect(plan);
  *out = plan->prof;
  TZ_CATCH
}

// ------------------------------------------------------------------ ops
int tz_op_permute(const void *in, void *out, int rank, const int32_t *perm, void *stream) {
  TZ_TRY
  REQUIRE(in && out && (perm || rank == 0), "NULL argument");
  REQUIRE(rank >= 0 && rank <= tz::dev::kMaxBits, "rank must be in 0..40");
  tz::dev::PermuteArgs a{};
  a.rank = rank;
  std::vector<char> seen(rank, 0);
  for (int p = 0; p < rank; p++) {
    REQUIRE(perm[p] >= 0 && perm[p] < rank && !seen[perm[p]], "perm is not a permutation");
    seen[perm[p]] = 1;
    a.perm[p] = (int8_t)perm[p];
  }
  tz::cuda_check(tz::dev::launch_permute((const float2 *)in, (float2 *)out, a, (cudaStream_t)stream), "permute");
  TZ_CATCH
}

int tz_op_cgemm_scratch_bytes(int precision, int64_t batch, int64_t m, int64_t n, int64_t k, size_t *bytes) {
  TZ_TRY
  REQUIRE(bytes, "NULL argument");
  REQUIRE(batch >= 1 && m >= 1 && n >= 1 && k >= 1, "sizes must be >= 1");
  *bytes = 0;
  if (precision == TZ_TF32X3 || precision == TZ_BF16X3 || precision == TZ_FP16X3) {
    if (!tz::dev::cgemm_tc_supported(precision, m, n, k))
      tz::fail(TZ_EUNSUPPORTED, "shape not supported by the tensor-core product");
    *bytes = kOpErrBytes + tz::dev::cgemm_tc_scratch_bytes(precision, batch, m, n, k);
  } else if (precision != TZ_C64_SIMT && precision != TZ_C128_SIMT) {
    tz::fail(TZ_EINVAL, "unknown precision");
  }
  TZ_CATCH
}

int tz_op_cgemm(int precision, int64_t batch, int64_t m, int64_t n, int64_t k, const void *A, int64_t sa,
                const void *B, int64_t sb, void *C, int64_t sc, void *scratch, size_t scratch_bytes, void *stream) {
  TZ_TRY
  REQUIRE(A && B && C, "NULL argument");
  REQUIRE(batch >= 1 && m >= 1 && n >= 1 && k >= 1, "sizes must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == TZ_C128_SIMT) {
    tz::cuda_check(tz::dev::launch_zgemm_simt((const double2 *)A, (const double2 *)B, (double2 *)C, batch, m, n, k, sa,
                                              sb, sc, nullptr, s),
                   "complex128 gemm");
  } else if (precision == TZ_C64_SIMT) {
    tz::cuda_check(tz::dev::launch_cgemm_simt((const float2 *)A, (const float2 *)B, (float2 *)C, batch, m, n, k, sa,
                                              sb, sc, nullptr, s),
                   "simt gemm");
  } else if (precision == TZ_TF32X3 || precision == TZ_BF16X3 || precision == TZ_FP16X3) {
    if (!tz::dev::cgemm_tc_supported(precision, m, n, k))
      tz::fail(TZ_EUNSUPPORTED, "shape not supported by the tensor-core product");
    const size_t need = kOpErrBytes + tz::dev::cgemm_tc_scratch_bytes(precision, batch, m, n, k);
    REQUIRE(scratch && scratch_bytes >= need, "scratch too small (tz_op_cgemm_scratch_bytes)");
    REQUIRE((reinterpret_cast<uintptr_t>(scratch) & 255) == 0, "scratch must be 256-byte aligned");
    int *err = static_cast<int *>(scratch);
    tz::cuda_check(cudaMemsetAsync(err, 0, sizeof(int), s), "clear error word");
    tz::cuda_check(tz::dev::launch_cgemm_tc(precision, (const float2 *)A, (const float2 *)B, (float2 *)C, batch, m, n,
                                            k, sa, sb, sc, nullptr, static_cast<char *>(scratch) + kOpErrBytes,
                                            scratch_bytes - kOpErrBytes, err, s),
                   "tensor-core gemm");
  } else {
    tz::fail(TZ_EINVAL, "unknown precision");
  }
  TZ_CATCH
}

int tz_op_cgemm_status(int precision, const void *scratch, void *stream) {
  TZ_TRY
  tz::cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "synchronise the stream");
  if (!is_tc_precision(precision)) return TZ_OK;
  REQUIRE(scratch, "NULL scratch");
  int v = 0;
  tz::cuda_check(cudaMemcpy(&v, scratch, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
  if (v) tz::fail(TZ_ETIMEOUT, "the tensor-core product timed out in a bounded wait; its result is invalid");
  TZ_CATCH
}

int tz_debug_set_wait_limit(int64_t ns) {
  TZ_TRY
  REQUIRE(ns >= 0, "wait limit must be >= 0");
  tz::cuda_check(tz::dev::tc_set_wait_limit((unsigned long long)ns), "set wait limit");
  tz::cuda_check(tz::dev::direct_queue_set_wait_limit((unsigned long long)ns), "set queue wait limit");
  TZ_CATCH
}

int tz_tune_tc_pairs(int mode) {
  TZ_TRY
  tz::dev::tc_set_pairs(mode);
  TZ_CATCH
}

int tz_tune_tc_prefetch(int kblocks) {
  TZ_TRY
  tz::dev::tc_set_prefetch(kblocks);
  TZ_CATCH
}

int tz_tune_preset(int precision, int64_t batch, int64_t m, int64_t n, int64_t k, int scatter, int pair, int ksplit,
                   int simt) {
  TZ_TRY
  REQUIRE(precision == TZ_C64_SIMT || is_tc_precision(precision), "presets are for the complex64 precisions");
  tz::tune_preset(precision, batch, m, n, k, scatter, pair, ksplit, simt);
  TZ_CATCH
}

int tz_debug_stream_tile(int64_t batch, int64_t m, int64_t n, int64_t k, int scatter, const int8_t *pb,
                         const int8_t *pm, const int8_t *pn, int32_t *out, int *supported) {
  TZ_TRY
  REQUIRE(out && supported, "NULL argument");
  REQUIRE(batch >= 1 && m >= 1 && n >= 1 && k >= 1, "dimensions must be >= 1");
  tz::dev::CScatter sc{};
  if (scatter) {
    REQUIRE(pb && pm && pn, "NULL scatter positions");
    auto lg = [](int64_t v) { int b = 0; while ((int64_t(1) << b) < v) b++; return b; };
    sc.nb = lg(batch);
    sc.nm = lg(m);
    sc.nn = lg(n);
    REQUIRE(sc.nb + sc.nm + sc.nn <= tz::dev::kMaxBits, "too many index bits");
    for (int j = 0; j < sc.nb; j++) sc.pb[j] = pb[j];
    for (int j = 0; j < sc.nm; j++) sc.pm[j] = pm[j];
    for (int j = 0; j < sc.nn; j++) sc.pn[j] = pn[j];
  }
  *supported = tz::dev::cgemm_stream_describe(batch, m, n, k, scatter ? &sc : nullptr, out);
  TZ_CATCH
}

int tz_debug_tune_force_simt(int on) {
  TZ_TRY
  tz::tune_force_simt(on);
  TZ_CATCH
}

int tz_debug_stall_tensor_core(int on) {
  TZ_TRY
  tz::cuda_check(tz::dev::tc_set_stall(on), "set stall switch");
  TZ_CATCH
}

int tz_debug_stall_direct_queue(int on) {
  TZ_TRY
  tz::cuda_check(tz::dev::direct_queue_set_stall(on), "set queue stall switch");
  TZ_CATCH
}

int tz_op_accumulate(const void *part, double *acc, int64_t n, double scale_re, double scale_im, void *stream) {
  TZ_TRY
  REQUIRE(part && acc, "NULL argument");
  REQUIRE(n >= 0, "n must be >= 0");
  tz::cuda_check(tz::dev::launch_accumulate_plain((const float2 *)part, (double2 *)acc, n, scale_re, scale_im,
                                                  (cudaStream_t)stream),
                 "accumulate");
  TZ_CATCH
}

}  // extern "C"
