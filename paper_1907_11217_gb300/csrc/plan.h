// Internal plan structure (host side).
#pragma once
#include <cuda_runtime.h>

#include "kernels.h"
#include "tz_internal.h"

namespace tz {

enum Region { R_NONE = 0, R_CONST = 1, R_ARENA = 2 };
enum ItemKind { IT_LEAVES = 0, IT_DIRECT = 1, IT_PERMUTE = 2, IT_GEMM = 3, IT_ACCUM = 4 };

struct PTensor {
  std::vector<int> lay;   // index ids, lay[p] = bit p of the element offset
  bool var = false;       // recomputed every group
  bool fixed = false;     // layout decided
  int region = R_NONE;
  int64_t off = -1;       // byte offset within its region
  int birth = -1, death = -1;
  int leaf = -1;          // network leaf it holds (or the full source of)
  bool full_source = false;  // full constant source of a sliced leaf
  int64_t elems() const { return int64_t(1) << lay.size(); }
  int64_t bytes() const { return elems() * 8; }
};

struct PStep {
  int a, b, c;
  bool var = false, gemm = false, tc = false;
  int opX = -1, opY = -1;     // tensors fed to the GEMM (after permutes)
  int permX = -1, permY = -1; // permute sources (or -1)
  int64_t M = 0, N = 0, K = 0, batch = 0;
  int level = 0;
  int dstep = -1;             // index into dsteps (direct steps)
  int64_t tc_scratch = 0;     // bytes of tensor-core operand scratch
  int64_t tc_scratch_off = -1;
  int tc_pair = -1;           // tensor-core launch choice (autotuned at bind): pairs of
  int tc_ksplit = 0;          // CTAs (1/0, -1 default) and K split (1 none, 0 default)
  int tc_simt = 0;            // autotuned kernel of a small-K step: 1 the tiled CUDA-core
                              // complex64 kernel (tensor-core steps), 2 the stream kernel
                              // (any complex64 step it supports), 0 the step's own
  dev::CScatter scatter{};    // where the GEMM writes its result
  bool row_major = false;     // scatter is the plain row-major order
  int c_nat = -1;             // tensor the GEMM writes in row-major order when a
                              // permute then moves it into c's layout
  bool skinny = false;        // n <= 4, k <= 16: operands read in place
  dev::GatherMap gather{};    // skinny: where the operands' elements sit
};

struct Item {
  int kind;
  int a = -1, b = -1;         // PERMUTE: src, dst tensors; GEMM: step
  int first = 0, count = 0;   // DIRECT: dsteps range
  int64_t blocks = 0;         // DIRECT: total blocks
  bool queue = false;         // DIRECT: one queue launch over dependent steps
  int64_t ctrl_off = -1;      // DIRECT queue: its counters in the scratch part's queue area
  int64_t bmap_off = -1;      // DIRECT: its block -> step map (int32) in the resident bmap table
};

}  // namespace tz

struct tz_plan {
  tz::Network net;
  tz::Pairs pairs;
  std::vector<int> sliced;
  std::vector<int> slice_bit;  // per index: slice bit number or -1
  tz_plan_opts opts{};
  tz::TreeInfo ti;
  std::vector<tz::PTensor> T;
  std::vector<tz::PStep> S;
  std::vector<tz::Item> var_items, const_items;
  std::vector<tz::dev::DStep> dsteps;
  std::vector<int> dstep_tensors;  // 3 tensor ids per dstep (A, B, C)
  std::vector<tz::dev::LeafJob> jobs;
  std::vector<int> job_tensors;    // 2 per job (dst, src or -1)
  int root = -1;
  int64_t max_rows = 0;
  int esz = 8;                     // bytes per tensor element: 8 complex64, 16 complex128
  // workspace layout (bytes): resident part [step tables | leaf tables |
  // constants], then one scratch part [group state | bitstrings | FP64
  // accumulator | group arena]; a query can also run in another scratch part
  size_t off_dsteps = 0, off_jobs = 0, off_bmap = 0, off_const = 0, off_scratch = 0;
  std::vector<int32_t> bmap;       // direct launches: step of each block, from the launch's first step
  size_t s_gs = 0, s_bits = 0, s_acc = 0, s_arena = 0;  // offsets within a scratch part
  size_t s_queue = 0, queue_bytes = 0;  // counters of the direct-step queue launches
  size_t const_bytes = 0, arena_bytes = 0, resident_bytes = 0, scratch_bytes = 0, total_bytes = 0;
  // device state
  char *ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t stream = nullptr;
  bool bound = false;
  int64_t lo = 0, hi = 1;
  // captured launches of one group, per scratch part they run on (the
  // plan's own, or a server slot's), oldest dropped beyond kMaxGraphs
  struct Graph {
    char *scratch;
    cudaGraph_t g;
    cudaGraphExec_t e;
  };
  static constexpr size_t kMaxGraphs = 8;
  std::vector<Graph> graphs;
  tz_plan_stats stats{};
  // profiling
  bool profiling = false;
  bool capturing = false;
  struct Pending {
    int kind;
    cudaEvent_t a, b;
    double flops, bytes;
    int item;   // index in var_items, -1 for bind-time items
  };
  std::vector<double> item_ms;     // per var item, summed over profiled groups
  std::vector<int64_t> item_count;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  tz_plan_profile prof{};
};

namespace tz {
// Where one query of a plan runs: a scratch part and a stream.
struct RunCtx {
  char *scratch;
  cudaStream_t stream;
};
inline RunCtx default_ctx(const tz_plan *p) { return RunCtx{p->ws + p->off_scratch, p->stream}; }
tz_plan *plan_create(const Network &net, const Pairs &pairs, const std::vector<int> &sliced, const tz_plan_opts &o);
void plan_bind(tz_plan *p, void *ws, size_t bytes);
// Contract all groups of the slice range [lo, hi) for n rows already in the
// scratch part's bitstring buffer; leaves the FP64 sums in its accumulator
// (asynchronous on ctx.stream). With use_graph, the launches of a group are
// captured once per scratch part and replayed. fresh = false continues a
// call: the accumulator and the error word keep what earlier slice ranges
// left (a query run in several slice ranges, as the server does).
void plan_run(tz_plan *p, const RunCtx &ctx, int64_t n_rows, int64_t lo, int64_t hi, bool fresh = true);
// The error word of a scratch part: 1 when a tensor-core product of the last
// call on it (or of the bind-time steps) timed out in a bounded wait.
// Synchronous (reads device memory); call after the stream has finished.
int read_tc_error(const tz_plan *p, const RunCtx &ctx);
// test hook: autotuned steps with small K take the CUDA-core kernel
void tune_force_simt(int on);
// one autotuner cache entry for the current device (tz_tune_preset)
void tune_preset(int precision, int64_t batch, int64_t M, int64_t N, int64_t K, int scatter, int pair, int ksplit,
                 int simt);
void plan_destroy(tz_plan *p);
void plan_profile_collect(tz_plan *p);
void item_cost_public(const tz_plan *p, int var_item, int *kind, double *flops, double *bytes);
std::string plan_describe(const tz_plan *p);
inline void cuda_check(cudaError_t e, const char *what) {
  if (e != cudaSuccess) fail(TZ_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
}  // namespace tz
