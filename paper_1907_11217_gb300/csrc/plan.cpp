// Plans: from (network, tree, sliced indices) to a launch schedule over one
// device workspace. A group is one slice (Sec. 1: one subtask) for one chunk
// of 2^batch_log2 bitstrings; every group runs the same launches.
#include <chrono>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <atomic>
#include <mutex>
#include <memory>
#include <sstream>

#include "plan.h"

namespace tz {

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int pos_of(const std::vector<int> &lay, int idx) {
  for (size_t p = 0; p < lay.size(); p++)
    if (lay[p] == idx) return (int)p;
  return -1;
}

// If lay = (perm of g1) ++ (perm of g2) ++ (perm of g3), return true and the
// three orders as they appear in lay.
bool groups_ok(const std::vector<int> &lay, const std::vector<int> &g1, const std::vector<int> &g2,
               const std::vector<int> &g3, std::vector<int> *o1, std::vector<int> *o2, std::vector<int> *o3) {
  if (lay.size() != g1.size() + g2.size() + g3.size()) return false;
  size_t p = 0;
  const std::vector<int> *gs[3] = {&g1, &g2, &g3};
  std::vector<int> *os[3] = {o1, o2, o3};
  for (int g = 0; g < 3; g++) {
    std::vector<int> seg(lay.begin() + p, lay.begin() + p + gs[g]->size());
    std::vector<int> a = seg, b = *gs[g];
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    if (a != b) return false;
    if (os[g]) *os[g] = seg;
    p += gs[g]->size();
  }
  return true;
}

std::vector<int> concat3(const std::vector<int> &a, const std::vector<int> &b, const std::vector<int> &c) {
  std::vector<int> r = a;
  r.insert(r.end(), b.begin(), b.end());
  r.insert(r.end(), c.begin(), c.end());
  return r;
}

// Relative order of the members of `set` as they appear in `lay`.
std::vector<int> rel_order(const std::vector<int> &lay, const std::vector<int> &set) {
  std::vector<int> r;
  for (int i : lay)
    if (std::find(set.begin(), set.end(), i) != set.end()) r.push_back(i);
  return r;
}

// First-fit interval allocator over one region.
struct Interval {
  int64_t off, size;
  int death;
};
int64_t first_fit(std::vector<Interval> &live, int64_t size, int birth, int death, int64_t *peak) {
  live.erase(std::remove_if(live.begin(), live.end(), [&](const Interval &x) { return x.death < birth; }),
             live.end());
  std::sort(live.begin(), live.end(), [](const Interval &x, const Interval &y) { return x.off < y.off; });
  int64_t cur = 0;
  for (const Interval &x : live) {
    if (x.off - cur >= size) break;
    cur = std::max(cur, x.off + x.size);
  }
  live.push_back({cur, size, death});
  *peak = std::max(*peak, cur + size);
  return cur;
}

}  // namespace

tz_plan *plan_create(const Network &net, const Pairs &pairs, const std::vector<int> &sliced, const tz_plan_opts &o) {
  validate_tree(net, pairs);
  const int I = (int)net.indices.size();
  std::vector<char> flag(I, 0);
  std::vector<int> slice_bit(I, -1);
  for (size_t j = 0; j < sliced.size(); j++) {
    int e = sliced[j];
    if (e < 0 || e >= I) fail(TZ_EINVAL, "sliced edge id out of range");
    if (net.is_open(e)) fail(TZ_EINVAL, "a batch index cannot be sliced");
    if (flag[e]) fail(TZ_EINVAL, "sliced edge listed twice");
    flag[e] = 1;
    slice_bit[e] = (int)j;
  }
  if (sliced.size() > 40) fail(TZ_EUNSUPPORTED, "more than 40 sliced indices");
  if (o.precision < TZ_C64_SIMT || o.precision > TZ_FP16X3) fail(TZ_EINVAL, "unknown precision");

  auto p = std::make_unique<tz_plan>();
  p->net = net;
  p->pairs = pairs;
  p->sliced = sliced;
  p->slice_bit = slice_bit;
  p->opts = o;
  p->esz = o.precision == TZ_C128_SIMT ? 16 : 8;
  const int64_t esz = p->esz;
  if (p->opts.small_log2 <= 0) p->opts.small_log2 = 20;
  p->opts.small_log2 = std::min(p->opts.small_log2, 26);
  p->max_rows = o.max_bitstrings > 0 ? o.max_bitstrings : 4096;
  if (p->max_rows > (int64_t(1) << 24)) fail(TZ_EINVAL, "max_bitstrings above 2^24");
  p->ti = analyse_tree(net, pairs, flag);
  const TreeInfo &ti = p->ti;
  if (ti.max_bits > dev::kMaxBits) fail(TZ_EUNSUPPORTED, "an intermediate tensor exceeds 2^40 elements");
  const int L = (int)net.leaves.size();
  const int NS = (int)ti.steps.size();
  const int g = net.batch_log2;

  // tensors: leaves, then step outputs
  p->T.resize(L + NS);
  for (int n = 0; n < L + NS; n++) {
    p->T[n].var = ti.var[n];
    if (n < L) p->T[n].leaf = n;
  }
  std::vector<int> consumer(L + NS, -1);
  p->S.resize(NS);
  for (int s = 0; s < NS; s++) {
    const StepInfo &st = ti.steps[s];
    PStep &ps = p->S[s];
    ps.a = st.a;
    ps.b = st.b;
    ps.c = st.c;
    ps.var = st.var;
    ps.gemm = st.bitsAll() > p->opts.small_log2 || st.bitsC() > dev::kMaxDirect - 4 ||
              (int)st.contr.size() > dev::kMaxDirect - 4;
    consumer[st.a] = consumer[st.b] = s;
  }
  p->root = NS > 0 ? L + NS - 1 : 0;

  auto set_of = [&](int node) { return ti.sets[node]; };

  // ---------------------------------------------------------------- layouts
  // Every tensor is stored in the order its consumer needs, and its producer
  // (leaf builder, constant upload, direct step or GEMM epilogue) writes it
  // in that order directly: no operand permutes. Layouts are decided in
  // reverse tree order, consumer before producer. A GEMM step wants
  //   X = [summed | X-free | batch],  Y = [summed | Y-free | batch]
  // (row-major [batch][rows][k]); its result goes through a scatter map.
  // The summed-bit order favours bits its producer writes contiguously:
  // bits the producing GEMM holds as columns, then rows, then batch.
  std::vector<int> roleX(NS, -1);  // operand used as X (rows) of each GEMM step
  for (int s = 0; s < NS; s++) {
    const StepInfo &st = ti.steps[s];
    roleX[s] = st.freeA.size() >= st.freeB.size() ? st.a : st.b;
  }
  std::vector<int> producer(L + NS, -1);
  for (int s = 0; s < NS; s++) producer[ti.steps[s].c] = s;
  // class of bit i in the natural output order of node t's producer:
  // 0 = GEMM column (fastest), 1 = GEMM row, 2 = batch or no preference
  auto bit_class = [&](int t, int i) {
    int s = producer[t];
    if (s < 0 || !p->S[s].gemm) return 2;
    const StepInfo &st = ti.steps[s];
    const auto &fx = roleX[s] == st.a ? st.freeA : st.freeB;
    const auto &fy = roleX[s] == st.a ? st.freeB : st.freeA;
    if (std::find(fy.begin(), fy.end(), i) != fy.end()) return 0;
    if (std::find(fx.begin(), fx.end(), i) != fx.end()) return 1;
    return 2;
  };
  auto natural = [&](int t) {  // producer's own preferred order
    int s = producer[t];
    if (s < 0 || !p->S[s].gemm) return set_of(t);
    const StepInfo &st = ti.steps[s];
    const auto &fx = roleX[s] == st.a ? st.freeA : st.freeB;
    const auto &fy = roleX[s] == st.a ? st.freeB : st.freeA;
    return concat3(fy, fx, st.batch);
  };
  // GEMM shapes and kernels, known before any layout
  for (int s = 0; s < NS; s++) {
    const StepInfo &st = ti.steps[s];
    PStep &ps = p->S[s];
    if (!ps.gemm) continue;
    const bool xa = roleX[s] == st.a;
    ps.M = int64_t(1) << (xa ? st.freeA : st.freeB).size();
    ps.N = int64_t(1) << (xa ? st.freeB : st.freeA).size();
    ps.K = int64_t(1) << st.contr.size();
    ps.batch = int64_t(1) << st.batch.size();
    // skinny products are memory-bound: the streaming SIMT kernel serves them
    ps.tc = (o.precision == TZ_TF32X3 || o.precision == TZ_BF16X3 || o.precision == TZ_FP16X3) &&
            dev::cgemm_tc_supported(o.precision, ps.M, ps.N, ps.K) &&
            !(ps.N <= 4 && ps.K <= 16);
    ps.skinny = !ps.tc && ps.N <= 4 && ps.K <= 16 && ps.M >= 256;
    if (ps.tc) ps.tc_scratch = (int64_t)dev::cgemm_tc_scratch_bytes(o.precision, ps.batch, ps.M, ps.N, ps.K);
  }
  p->T[p->root].lay = natural(p->root);
  p->T[p->root].fixed = true;
  for (int s = NS - 1; s >= 0; s--) {
    const StepInfo &st = ti.steps[s];
    PStep &ps = p->S[s];
    if (!p->T[st.c].fixed) {
      p->T[st.c].lay = natural(st.c);
      p->T[st.c].fixed = true;
    }
    if (!ps.gemm) continue;
    if (ps.skinny) {
      // operands are read in place: their producers keep their own order
      ps.opX = roleX[s];
      ps.opY = roleX[s] == st.a ? st.b : st.a;
      continue;
    }
    const std::vector<int> &Lc = p->T[st.c].lay;
    const int X = roleX[s], Y = X == st.a ? st.b : st.a;
    const std::vector<int> &fX = X == st.a ? st.freeA : st.freeB;
    const std::vector<int> &fY = X == st.a ? st.freeB : st.freeA;
    // summed bits: ordered for the larger operand's producer
    const int big = p->T[X].var == p->T[Y].var ? (fX.size() >= fY.size() ? X : Y) : (p->T[X].var ? X : Y);
    std::vector<int> ko = st.contr;
    std::stable_sort(ko.begin(), ko.end(), [&](int u, int v) { return bit_class(big, u) < bit_class(big, v); });
    std::vector<int> fxo = rel_order(Lc, fX), fyo = rel_order(Lc, fY), bo = rel_order(Lc, st.batch);
    p->T[X].lay = concat3(ko, fxo, bo);
    p->T[Y].lay = concat3(ko, fyo, bo);
    p->T[X].fixed = p->T[Y].fixed = true;
    ps.opX = X;
    ps.opY = Y;
    // where canonical (z, m, n) lands in C
    dev::CScatter &sc = ps.scatter;
    std::memset(&sc, 0, sizeof(sc));
    sc.nm = (int)fxo.size();
    sc.nn = (int)fyo.size();
    sc.nb = (int)bo.size();
    for (int j = 0; j < sc.nm; j++) sc.pm[j] = (int8_t)pos_of(Lc, fxo[j]);
    for (int j = 0; j < sc.nn; j++) sc.pn[j] = (int8_t)pos_of(Lc, fyo[j]);
    for (int j = 0; j < sc.nb; j++) sc.pb[j] = (int8_t)pos_of(Lc, bo[j]);
    ps.row_major = true;
    for (int j = 0; j < sc.nn; j++) ps.row_major &= sc.pn[j] == j;
    for (int j = 0; j < sc.nm; j++) ps.row_major &= sc.pm[j] == sc.nn + j;
    for (int j = 0; j < sc.nb; j++) ps.row_major &= sc.pb[j] == sc.nn + sc.nm + j;
  }
  for (int n = 0; n < L + NS; n++)
    if (!p->T[n].fixed) {
      p->T[n].lay = set_of(n);
      p->T[n].fixed = true;
    }
  // skinny steps: rows numbered in the order of X's storage (so a warp's loads
  // stay together), then the gather maps of both operands and the scatter map
  for (int s = 0; s < NS; s++) {
    PStep &ps = p->S[s];
    if (!ps.gemm || !ps.skinny) continue;
    const StepInfo &st = ti.steps[s];
    const std::vector<int> &LX = p->T[ps.opX].lay, &LY = p->T[ps.opY].lay, &Lc = p->T[ps.c].lay;
    const std::vector<int> &fX = ps.opX == st.a ? st.freeA : st.freeB;
    const std::vector<int> &fY = ps.opX == st.a ? st.freeB : st.freeA;
    const std::vector<int> fxo = rel_order(LX, fX), ko = rel_order(LX, st.contr), bo = rel_order(LX, st.batch);
    const std::vector<int> fyo = rel_order(LY, fY);
    dev::GatherMap &g = ps.gather;
    std::memset(&g, 0, sizeof(g));
    g.nm = (int)fxo.size();
    g.nn = (int)fyo.size();
    g.nk = (int)ko.size();
    g.nb = (int)bo.size();
    for (int j = 0; j < g.nm; j++) g.xm[j] = (int8_t)pos_of(LX, fxo[j]);
    for (int j = 0; j < g.nk; j++) {
      g.xk[j] = (int8_t)pos_of(LX, ko[j]);
      g.yk[j] = (int8_t)pos_of(LY, ko[j]);
    }
    for (int j = 0; j < g.nb; j++) {
      g.xb[j] = (int8_t)pos_of(LX, bo[j]);
      g.yb[j] = (int8_t)pos_of(LY, bo[j]);
    }
    for (int j = 0; j < g.nn; j++) g.yn[j] = (int8_t)pos_of(LY, fyo[j]);
    dev::CScatter &sc = ps.scatter;
    std::memset(&sc, 0, sizeof(sc));
    sc.nm = g.nm;
    sc.nn = g.nn;
    sc.nb = g.nb;
    for (int j = 0; j < sc.nm; j++) sc.pm[j] = (int8_t)pos_of(Lc, fxo[j]);
    for (int j = 0; j < sc.nn; j++) sc.pn[j] = (int8_t)pos_of(Lc, fyo[j]);
    for (int j = 0; j < sc.nb; j++) sc.pb[j] = (int8_t)pos_of(Lc, bo[j]);
    ps.row_major = true;
    for (int j = 0; j < sc.nn; j++) ps.row_major &= sc.pn[j] == j;
    for (int j = 0; j < sc.nm; j++) ps.row_major &= sc.pm[j] == sc.nn + j;
    for (int j = 0; j < sc.nb; j++) ps.row_major &= sc.pb[j] == sc.nn + sc.nm + j;
  }
  // A GEMM epilogue writes its consumer's layout directly only when the two
  // lowest bits of that layout are bits it writes contiguously (rows across a
  // warp, or a thread's run of columns); otherwise whole sectors would be
  // assembled from several CTAs' 8-byte stores. Then it writes row-major and
  // the tiled permute moves the result (both sides in 256-byte runs).
  for (int s = 0; s < NS; s++) {
    PStep &ps = p->S[s];
    if (!ps.gemm || ps.row_major) continue;
    const std::vector<int> &Lc = p->T[ps.c].lay;
    if (Lc.size() < 2) continue;
    const dev::CScatter &sc = ps.scatter;
    std::vector<int> good;  // positions in Lc written contiguously
    const bool skinny = ps.skinny;
    const int m_run = ps.tc || skinny ? 5 : 2, n_run = ps.tc ? 3 : skinny ? sc.nn : 4;
    for (int j = 0; j < std::min(sc.nm, m_run); j++) good.push_back(sc.pm[j]);
    for (int j = 0; j < std::min(sc.nn, n_run); j++) good.push_back(sc.pn[j]);
    auto has = [&](int pos) { return std::find(good.begin(), good.end(), pos) != good.end(); };
    if (has(0) && has(1)) continue;
    PTensor t;
    t.var = p->T[ps.c].var;
    t.fixed = true;
    // row-major [batch][m][n]: n bits lowest, then m, then batch
    for (int j = 0; j < sc.nn; j++) t.lay.push_back(Lc[sc.pn[j]]);
    for (int j = 0; j < sc.nm; j++) t.lay.push_back(Lc[sc.pm[j]]);
    for (int j = 0; j < sc.nb; j++) t.lay.push_back(Lc[sc.pb[j]]);
    p->T.push_back(t);
    ps.c_nat = (int)p->T.size() - 1;
    ps.row_major = true;
  }
  // root must hold exactly the batch indices
  for (int i : p->T[p->root].lay)
    if (!net.is_open(i)) fail(TZ_EINVAL, "tree root keeps a wire index: the tree does not contract the network");

  // full constant sources of sliced constant leaves
  std::vector<int> full_src(L, -1);
  for (int l = 0; l < L; l++) {
    const Leaf &lf = net.leaves[l];
    if (lf.kind != LEAF_CONST || !p->T[l].var) continue;
    PTensor t;
    t.lay = lf.idx;
    t.var = false;
    t.fixed = true;
    t.leaf = l;
    t.full_source = true;
    p->T.push_back(t);
    full_src[l] = (int)p->T.size() - 1;
  }

  // ---------------------------------------------------------------- schedule
  std::vector<int> level(L + NS, 0);
  int max_level[2] = {0, 0};
  for (int s = 0; s < NS; s++) {
    const StepInfo &st = ti.steps[s];
    int lv = 0;
    for (int x : {st.a, st.b})
      if (x >= L && p->T[x].var == st.var) lv = std::max(lv, level[x]);
    level[st.c] = lv + 1;
    p->S[s].level = lv + 1;
    max_level[st.var] = std::max(max_level[st.var], lv + 1);
  }
  std::vector<int> late_const_permutes;  // const operands of var GEMMs: permuted at bind time
  for (int s = 0; s < NS; s++) {
    const PStep &ps = p->S[s];
    if (!ps.var || !ps.gemm) continue;
    if (ps.permX >= 0 && !p->T[ps.permX].var) late_const_permutes.insert(late_const_permutes.end(), {ps.permX, ps.opX});
    if (ps.permY >= 0 && !p->T[ps.permY].var) late_const_permutes.insert(late_const_permutes.end(), {ps.permY, ps.opY});
  }
  for (int pass = 0; pass < 2; pass++) {
    bool var = pass == 1;
    std::vector<Item> &items = var ? p->var_items : p->const_items;
    if (var) items.push_back({IT_LEAVES});
    for (int lv = 1; lv <= max_level[var]; lv++) {
      Item d{IT_DIRECT};
      d.first = (int)p->dsteps.size();
      for (int s = 0; s < NS; s++) {
        PStep &ps = p->S[s];
        if (ps.var != var || ps.level != lv || ps.gemm) continue;
        ps.dstep = (int)p->dsteps.size();
        p->dsteps.push_back(dev::DStep{});
        p->dstep_tensors.insert(p->dstep_tensors.end(), {ps.a, ps.b, ps.c});
      }
      d.count = (int)p->dsteps.size() - d.first;
      if (d.count) items.push_back(d);
      for (int s = 0; s < NS; s++) {
        PStep &ps = p->S[s];
        if (ps.var != var || ps.level != lv || !ps.gemm) continue;
        for (int k = 0; k < 2; k++) {
          int src = k == 0 ? ps.permX : ps.permY, dst = k == 0 ? ps.opX : ps.opY;
          if (src < 0) continue;
          if (var && !p->T[src].var) {
            continue;  // constant operand of a group step: permuted once at bind time
          } else {
            Item it{IT_PERMUTE};
            it.a = src;
            it.b = dst;
            items.push_back(it);
          }
        }
        Item it{IT_GEMM};
        it.a = s;
        items.push_back(it);
        if (ps.c_nat >= 0) {
          Item pm{IT_PERMUTE};
          pm.a = ps.c_nat;
          pm.b = ps.c;
          items.push_back(pm);
        }
      }
    }
    if (!var) {
      for (size_t j = 0; j < late_const_permutes.size(); j += 2) {
        Item it{IT_PERMUTE};
        it.a = late_const_permutes[j];
        it.b = late_const_permutes[j + 1];
        items.push_back(it);
      }
    } else {
      items.push_back({IT_ACCUM});
    }
  }

  // ------------------------------------------------- direct-step queues
  // Each group's direct steps move to the earliest point where their inputs
  // exist: right after the last product or permute whose result they read
  // (through other direct steps, too). The direct steps that share such a
  // point form one queue launch, in their level order, which is a
  // topological order. A direct step only moves earlier, and a product reads
  // a direct step's result at a later point than before, so every item
  // still runs after its inputs.
  if (p->opts.direct_queue) {
    std::vector<Item> &items = p->var_items;
    std::vector<int> phase(p->T.size(), 0);  // point after which a tensor exists
    std::vector<Item> bars;                  // the other items, in order
    std::vector<std::vector<int>> at;        // direct steps per point
    int v0 = -1;
    for (const Item &it : items) {
      if (it.kind == IT_DIRECT) {
        for (int d = it.first; d < it.first + it.count; d++) {
          if (v0 < 0) v0 = d;
          const int a = p->dstep_tensors[3 * d], b = p->dstep_tensors[3 * d + 1], c = p->dstep_tensors[3 * d + 2];
          const int ph = std::max(phase[a], phase[b]);
          at[ph].push_back(d);
          phase[c] = ph;
        }
        continue;
      }
      const int bi = (int)bars.size();
      bars.push_back(it);
      at.resize(bars.size());
      if (it.kind == IT_PERMUTE) phase[it.b] = bi;
      if (it.kind == IT_GEMM) {
        const PStep &ps = p->S[it.a];
        phase[ps.c_nat >= 0 ? ps.c_nat : ps.c] = bi;
      }
    }
    if (v0 >= 0) {
      std::vector<dev::DStep> nd(p->dsteps.begin(), p->dsteps.begin() + v0);
      std::vector<int> nt(p->dstep_tensors.begin(), p->dstep_tensors.begin() + 3 * (size_t)v0);
      std::vector<int> remap(p->dsteps.size(), -1);
      std::vector<Item> out;
      for (size_t bi = 0; bi < bars.size(); bi++) {
        out.push_back(bars[bi]);
        if (at[bi].empty()) continue;
        Item q{IT_DIRECT};
        q.queue = true;
        q.first = (int)nd.size();
        for (int d : at[bi]) {
          remap[d] = (int)nd.size();
          nd.push_back(p->dsteps[d]);
          nt.insert(nt.end(), {p->dstep_tensors[3 * d], p->dstep_tensors[3 * d + 1], p->dstep_tensors[3 * d + 2]});
        }
        q.count = (int)nd.size() - q.first;
        out.push_back(q);
      }
      for (PStep &ps : p->S)
        if (ps.dstep >= v0) ps.dstep = remap[ps.dstep];
      p->dsteps.swap(nd);
      p->dstep_tensors.swap(nt);
      items.swap(out);
    }
  }

  // ---------------------------------------------------------------- memory
  // lifetimes in item time; const tensors consumed by var work are persistent
  const int NT = (int)p->T.size();
  std::vector<int> birth[2], death[2];
  for (int pass = 0; pass < 2; pass++) {
    birth[pass].assign(NT, -1);
    death[pass].assign(NT, -1);
  }
  std::vector<char> persistent(NT, 0);
  auto use = [&](int pass, int t, int time) {
    death[pass][t] = std::max(death[pass][t], time);
    if (pass == 1 && !p->T[t].var) persistent[t] = 1;
  };
  for (int pass = 0; pass < 2; pass++) {
    std::vector<Item> &items = pass ? p->var_items : p->const_items;
    for (int time = 0; time < (int)items.size(); time++) {
      const Item &it = items[time];
      if (it.kind == IT_LEAVES) {
        for (int l = 0; l < L; l++)
          if (p->T[l].var) {
            birth[1][l] = time;
            if (full_src[l] >= 0) use(1, full_src[l], time);
          }
      } else if (it.kind == IT_DIRECT) {
        for (int d = it.first; d < it.first + it.count; d++) {
          use(pass, p->dstep_tensors[3 * d], time);
          use(pass, p->dstep_tensors[3 * d + 1], time);
          birth[pass][p->dstep_tensors[3 * d + 2]] = time;
        }
      } else if (it.kind == IT_PERMUTE) {
        use(pass, it.a, time);
        birth[pass][it.b] = time;
      } else if (it.kind == IT_GEMM) {
        const PStep &ps = p->S[it.a];
        use(pass, ps.opX, time);
        use(pass, ps.opY, time);
        birth[pass][ps.c_nat >= 0 ? ps.c_nat : ps.c] = time;
      } else if (it.kind == IT_ACCUM) {
        use(pass, p->root, time);
      }
    }
  }
  // the root may be a leaf (no steps): built by the leaf builder
  int64_t const_peak = 0, arena_peak = 0, arena_const_peak = 0;
  std::vector<Interval> live_var, live_const;
  // const region: constant leaves used anywhere, full sources, persistent step outputs
  for (int t = 0; t < NT; t++) {
    PTensor &pt = p->T[t];
    if (pt.var) continue;
    bool is_const_leaf = (t < L) || pt.full_source;
    bool used = death[0][t] >= 0 || death[1][t] >= 0;
    if (!used) continue;
    if (is_const_leaf || persistent[t]) {
      pt.region = R_CONST;
      pt.off = const_peak;
      const_peak = (int64_t)align256(const_peak + pt.elems() * esz);
    }
  }
  // arena: var tensors in the group pass, transient const tensors in the bind
  // pass (the two overlay each other); requests in birth order
  for (int pass = 1; pass >= 0; pass--) {
    struct Req {
      int birth, death, tensor, step;
      int64_t size;
    };
    std::vector<Req> reqs;
    for (int t = 0; t < NT; t++) {
      PTensor &pt = p->T[t];
      if (pt.region != R_NONE || birth[pass][t] < 0) continue;
      if ((pass == 1) != pt.var) continue;
      reqs.push_back(Req{birth[pass][t], std::max(death[pass][t], birth[pass][t]), t, -1,
                         (int64_t)align256((size_t)(pt.elems() * esz))});
    }
    // tensor-core operand scratch of each GEMM: lives during its item only
    std::vector<Item> &items = pass ? p->var_items : p->const_items;
    for (int time = 0; time < (int)items.size(); time++) {
      if (items[time].kind != IT_GEMM) continue;
      PStep &ps = p->S[items[time].a];
      if (ps.tc_scratch <= 0) continue;
      reqs.push_back(Req{time, time, -1, items[time].a, (int64_t)align256((size_t)ps.tc_scratch)});
    }
    std::sort(reqs.begin(), reqs.end(), [](const Req &x, const Req &y) {
      if (x.birth != y.birth) return x.birth < y.birth;
      if (x.tensor != y.tensor) return x.tensor < y.tensor;
      return x.step < y.step;
    });
    std::vector<Interval> &live = pass ? live_var : live_const;
    int64_t *peak = pass ? &arena_peak : &arena_const_peak;
    for (const Req &r : reqs) {
      int64_t at = first_fit(live, r.size, r.birth, r.death, peak);
      if (r.tensor >= 0) {
        PTensor &pt = p->T[r.tensor];
        pt.region = R_ARENA;
        pt.birth = r.birth;
        pt.death = r.death;
        pt.off = at;
      } else {
        p->S[r.step].tc_scratch_off = at;
      }
    }
  }
  for (int t = 0; t < NT; t++) {
    const PTensor &pt = p->T[t];
    bool needed = death[0][t] >= 0 || death[1][t] >= 0 || birth[0][t] >= 0 || birth[1][t] >= 0;
    if (needed && pt.region == R_NONE)
      fail(TZ_EINVAL, "internal: tensor " + std::to_string(t) + " without memory (var " + std::to_string(pt.var) +
                          ", births " + std::to_string(birth[0][t]) + "/" + std::to_string(birth[1][t]) +
                          ", deaths " + std::to_string(death[0][t]) + "/" + std::to_string(death[1][t]) + ")");
  }

  // ---------------------------------------------------------------- tables
  for (int d = 0; d < (int)p->dsteps.size(); d++) {
    dev::DStep &ds = p->dsteps[d];
    const PTensor &A = p->T[p->dstep_tensors[3 * d]];
    const PTensor &B = p->T[p->dstep_tensors[3 * d + 1]];
    const PTensor &C = p->T[p->dstep_tensors[3 * d + 2]];
    std::memset(&ds, 0, sizeof(ds));
    ds.nC = (int)C.lay.size();
    std::vector<int> contr;
    for (int i : A.lay)
      if (pos_of(C.lay, i) < 0) contr.push_back(i);
    ds.nK = (int)contr.size();
    for (int j = 0; j < dev::kMaxDirect; j++) ds.a_c[j] = ds.b_c[j] = ds.a_k[j] = ds.b_k[j] = -1;
    for (int j = 0; j < ds.nC; j++) {
      ds.a_c[j] = (int8_t)pos_of(A.lay, C.lay[j]);
      ds.b_c[j] = (int8_t)pos_of(B.lay, C.lay[j]);
    }
    for (int j = 0; j < ds.nK; j++) {
      ds.a_k[j] = (int8_t)pos_of(A.lay, contr[j]);
      ds.b_k[j] = (int8_t)pos_of(B.lay, contr[j]);
      if (ds.b_k[j] < 0) fail(TZ_EINVAL, "internal: summed index missing from one operand");
    }
    int want = std::max(0, 12 - ds.nC);
    ds.split = std::min({ds.nK, want, 8});
  }
  int64_t queue_words = 0;
  for (std::vector<Item> *items : {&p->var_items, &p->const_items})
    for (Item &it : *items) {
      if (it.kind != IT_DIRECT) continue;
      int64_t b = 0;
      for (int d = it.first; d < it.first + it.count; d++) {
        dev::DStep &ds = p->dsteps[d];
        ds.block_begin = b;
        ds.nblk = (int)std::max<int64_t>(1, ((int64_t(1) << (ds.nC + ds.split)) + 255) / 256);
        ds.dep[0] = ds.dep[1] = -1;
        ds.dep_nblk[0] = ds.dep_nblk[1] = 0;
        b += ds.nblk;
        if (!it.queue) continue;
        // steps of the same launch whose results this step reads
        for (int k = 0; k < 2; k++)
          for (int e = it.first; e < d; e++)
            if (p->dstep_tensors[3 * e + 2] == p->dstep_tensors[3 * d + k]) {
              ds.dep[k] = e - it.first;
              ds.dep_nblk[k] = p->dsteps[e].nblk;
            }
      }
      it.blocks = b;
      // the step of each block of the launch (one load instead of a search)
      it.bmap_off = (int64_t)p->bmap.size() * 4;
      for (int d = it.first; d < it.first + it.count; d++)
        p->bmap.insert(p->bmap.end(), (size_t)p->dsteps[d].nblk, d - it.first);
      if (it.queue) {
        it.ctrl_off = queue_words * 4;
        queue_words += dev::direct_queue_ctrl_words(it.count);
      }
    }
  // leaf jobs
  for (int l = 0; l < L; l++) {
    if (!p->T[l].var) continue;
    const Leaf &lf = net.leaves[l];
    const PTensor &dst = p->T[l];
    dev::LeafJob j;
    std::memset(&j, 0, sizeof(j));
    j.rank = (int)dst.lay.size();
    if (j.rank > 24) fail(TZ_EUNSUPPORTED, "leaf tensor above 2^24 elements");
    for (int x = 0; x < 24; x++) j.src_pos[x] = -1;
    for (int x = 0; x < 8; x++) j.fixed_src_pos[x] = j.fixed_slice_bit[x] = j.beta_dst_pos[x] = -1;
    j.e_dst_pos = j.e_slice_bit = -1;
    if (lf.kind == LEAF_OUTPUT) {
      j.kind = dev::LJ_OUTPUT;
      j.qubit = lf.qubit;
      j.rc = lf.rc;
      if (lf.rc == 1) {
        int e = lf.idx[0];
        if (slice_bit[e] >= 0)
          j.e_slice_bit = slice_bit[e];
        else
          j.e_dst_pos = pos_of(dst.lay, e);
      }
      for (int i : lf.idx) {
        if (!net.is_batch(i)) continue;
        j.beta_dst_pos[net.indices[i].segment] = (int8_t)pos_of(dst.lay, i);
      }
      for (int x = 0; x < 2 * (1 << lf.rc) && x < 4; x++) {
        j.M[x] = make_float2((float)lf.data[x].real(), (float)lf.data[x].imag());
        j.Md[x] = make_double2(lf.data[x].real(), lf.data[x].imag());
      }
      p->job_tensors.insert(p->job_tensors.end(), {l, -1});
    } else {
      j.kind = dev::LJ_GATHER;
      const PTensor &src = p->T[full_src[l]];
      for (int x = 0; x < j.rank; x++) j.src_pos[x] = (int8_t)pos_of(src.lay, dst.lay[x]);
      for (size_t x = 0; x < src.lay.size(); x++) {
        int e = src.lay[x];
        if (slice_bit[e] < 0) continue;
        if (j.n_fixed >= 8) fail(TZ_EUNSUPPORTED, "leaf with more than 8 sliced indices");
        j.fixed_src_pos[j.n_fixed] = (int8_t)x;
        j.fixed_slice_bit[j.n_fixed] = (int8_t)slice_bit[e];
        j.n_fixed++;
      }
      p->job_tensors.insert(p->job_tensors.end(), {l, full_src[l]});
    }
    p->jobs.push_back(j);
  }

  // workspace layout
  size_t off = 0;
  p->off_dsteps = off;
  off = align256(off + sizeof(dev::DStep) * std::max<size_t>(1, p->dsteps.size()));
  p->off_jobs = off;
  off = align256(off + sizeof(dev::LeafJob) * std::max<size_t>(1, p->jobs.size()));
  p->off_bmap = off;
  off = align256(off + sizeof(int32_t) * p->bmap.size());
  p->off_const = off;
  p->const_bytes = (size_t)const_peak;
  off = align256(off + p->const_bytes);
  p->resident_bytes = off;
  p->off_scratch = off;
  size_t so = 0;
  p->s_gs = so;
  so = align256(so + sizeof(dev::GroupState));
  p->s_bits = so;
  so = align256(so + (size_t)p->max_rows * net.n_qubits);
  p->s_acc = so;
  so = align256(so + ((size_t)p->max_rows * 16 << net.n_open));
  p->s_queue = so;
  p->queue_bytes = (size_t)queue_words * 4;
  so = align256(so + p->queue_bytes);
  p->s_arena = so;
  p->arena_bytes = (size_t)std::max(arena_peak, arena_const_peak);
  so = align256(so + p->arena_bytes);
  p->scratch_bytes = so;
  p->total_bytes = p->resident_bytes + p->scratch_bytes;

  // stats
  tz_plan_stats &stt = p->stats;
  stt.n_steps = NS;
  stt.k = (int)sliced.size();
  stt.batch_log2 = g;
  stt.n_open = net.n_open;
  stt.max_log2 = ti.max_bits;
  for (int s = 0; s < NS; s++) {
    const StepInfo &st = ti.steps[s];
    double fl = 8.0 * std::ldexp(1.0, st.bitsAll());
    if (!st.var) {
      stt.n_const_steps++;
      stt.const_flops += fl;
      continue;
    }
    stt.flops_per_group += fl;
    stt.bytes_per_group +=
        (double)esz * (std::ldexp(1.0, st.bitsA()) + std::ldexp(1.0, st.bitsB()) + std::ldexp(1.0, st.bitsC()));
    if (p->S[s].gemm) {
      stt.n_gemm_steps++;
      stt.gemm_flops_per_group += fl;
    }
  }
  for (const Item &it : p->var_items)
    if (it.kind == IT_PERMUTE) {
      stt.n_permutes++;
      stt.permute_bytes_per_group += 2.0 * esz * p->T[it.a].elems();
    }
  // kernel launches: one per item, but a tensor-core product also prepares B
  // and, when it splits K, sums the partials
  stt.n_launches_per_group = 0;
  for (const Item &it : p->var_items) {
    int n = 1;
    if (it.kind == IT_GEMM) {
      const PStep &ps = p->S[it.a];
      if (ps.tc)
        n = dev::cgemm_tc_launches(p->opts.precision, ps.batch, ps.M, ps.N, ps.K, !ps.row_major);
    } else if (it.kind == IT_ACCUM) {
      n = dev::accumulate_launches(net.batch_log2, net.n_open);
    }
    stt.n_launches_per_group += n;
  }
  stt.workspace_bytes = p->total_bytes;
  stt.const_bytes = p->const_bytes;
  stt.scratch_bytes = p->scratch_bytes;
  p->lo = 0;
  p->hi = int64_t(1) << sliced.size();
  return p.release();
}

std::string plan_describe(const tz_plan *p) {
  std::ostringstream o;
  o << "{\"tensors\": [";
  for (size_t t = 0; t < p->T.size(); t++) {
    const PTensor &x = p->T[t];
    o << (t ? "," : "") << "{\"id\":" << t << ",\"lay\":[";
    for (size_t q = 0; q < x.lay.size(); q++) o << (q ? "," : "") << x.lay[q];
    o << "],\"var\":" << (x.var ? 1 : 0) << ",\"region\":" << x.region << ",\"off\":" << x.off
      << ",\"leaf\":" << x.leaf << ",\"full\":" << (x.full_source ? 1 : 0) << "}";
  }
  o << "],\"steps\":[";
  for (size_t s = 0; s < p->S.size(); s++) {
    const PStep &x = p->S[s];
    o << (s ? "," : "") << "{\"a\":" << x.a << ",\"b\":" << x.b << ",\"c\":" << x.c << ",\"var\":" << x.var
      << ",\"gemm\":" << x.gemm << ",\"tc\":" << x.tc << ",\"opX\":" << x.opX << ",\"opY\":" << x.opY
      << ",\"M\":" << x.M << ",\"N\":" << x.N << ",\"K\":" << x.K << ",\"batch\":" << x.batch
      << ",\"level\":" << x.level << ",\"dstep\":" << x.dstep << ",\"permX\":" << x.permX << ",\"permY\":" << x.permY
      << ",\"row_major\":" << x.row_major << ",\"c_nat\":" << x.c_nat << ",\"skinny\":" << x.skinny
      << ",\"tc_pair\":" << x.tc_pair << ",\"tc_ksplit\":" << x.tc_ksplit << ",\"tc_simt\":" << x.tc_simt;
    auto arr = [&](const char *name, const int8_t *v, int n) {
      o << ",\"" << name << "\":[";
      for (int j = 0; j < n; j++) o << (j ? "," : "") << (int)v[j];
      o << "]";
    };
    arr("xm", x.gather.xm, x.gather.nm);
    arr("xk", x.gather.xk, x.gather.nk);
    arr("xb", x.gather.xb, x.gather.nb);
    arr("yn", x.gather.yn, x.gather.nn);
    arr("yk", x.gather.yk, x.gather.nk);
    arr("yb", x.gather.yb, x.gather.nb);
    o << ",\"pm\":[";
    for (int j = 0; j < x.scatter.nm; j++) o << (j ? "," : "") << (int)x.scatter.pm[j];
    o << "],\"pn\":[";
    for (int j = 0; j < x.scatter.nn; j++) o << (j ? "," : "") << (int)x.scatter.pn[j];
    o << "],\"pb\":[";
    for (int j = 0; j < x.scatter.nb; j++) o << (j ? "," : "") << (int)x.scatter.pb[j];
    o << "]}";
  }
  auto items = [&](const std::vector<Item> &v) {
    o << "[";
    for (size_t i = 0; i < v.size(); i++)
      o << (i ? "," : "") << "[" << v[i].kind << "," << v[i].a << "," << v[i].b << "," << v[i].first << ","
        << v[i].count << "," << v[i].blocks << "," << (v[i].queue ? 1 : 0) << "]";
    o << "]";
  };
  o << "],\"dsteps\":[";
  for (size_t d = 0; d < p->dsteps.size(); d++)
    o << (d ? "," : "") << "[" << p->dstep_tensors[3 * d] << "," << p->dstep_tensors[3 * d + 1] << ","
      << p->dstep_tensors[3 * d + 2] << "," << p->dsteps[d].nblk << "," << p->dsteps[d].dep[0] << ","
      << p->dsteps[d].dep[1] << "]";
  o << "],\"var_items\":";
  items(p->var_items);
  o << ",\"const_items\":";
  items(p->const_items);
  o << ",\"root\":" << p->root << ",\"sliced\":[";
  for (size_t j = 0; j < p->sliced.size(); j++) o << (j ? "," : "") << p->sliced[j];
  o << "],\"scalar\":[" << p->net.scalar.real() << "," << p->net.scalar.imag() << "],\"leaves\":[";
  o.precision(17);
  for (size_t l = 0; l < p->net.leaves.size(); l++) {
    const Leaf &lf = p->net.leaves[l];
    o << (l ? "," : "") << "{\"kind\":" << lf.kind << ",\"qubit\":" << lf.qubit << ",\"rc\":" << lf.rc
      << ",\"idx\":[";
    for (size_t q = 0; q < lf.idx.size(); q++) o << (q ? "," : "") << lf.idx[q];
    o << "],\"data\":[";
    for (size_t q = 0; q < lf.data.size(); q++)
      o << (q ? "," : "") << "[" << lf.data[q].real() << "," << lf.data[q].imag() << "]";
    o << "]}";
  }
  o << "],\"open\":[";
  bool first = true;
  for (size_t i = 0; i < p->net.indices.size(); i++)
    if (p->net.is_open((int)i)) {
      o << (first ? "" : ",") << "[" << i << "," << p->net.indices[i].qubit << "," << p->net.indices[i].segment
        << "]";
      first = false;
    }
  o << "]}";
  return o.str();
}

// ------------------------------------------------------------------ device
static void *tensor_ptr(const tz_plan *p, const RunCtx &ctx, int t) {
  const PTensor &x = p->T[t];
  if (x.region == R_CONST) return p->ws + p->off_const + x.off;
  if (x.region == R_ARENA) return ctx.scratch + p->s_arena + x.off;
  fail(TZ_EINVAL, "internal: tensor has no memory");
}

static int64_t tensor_rel(const tz_plan *p, int t) {
  const PTensor &x = p->T[t];
  if (x.region == R_CONST) return x.off;
  if (x.region == R_ARENA) return dev::kArenaTag | x.off;
  fail(TZ_EINVAL, "internal: tensor has no memory");
}

static cudaEvent_t take_event(tz_plan *p) {
  if (!p->event_pool.empty()) {
    cudaEvent_t e = p->event_pool.back();
    p->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cuda_check(cudaEventCreate(&e), "cudaEventCreate");
  return e;
}

void plan_profile_collect(tz_plan *p) {
  if (p->pending.empty()) return;
  cuda_check(cudaStreamSynchronize(p->stream), "profile sync");
  for (auto &q : p->pending) {
    float ms = 0;
    cuda_check(cudaEventElapsedTime(&ms, q.a, q.b), "event time");
    p->prof.launches[q.kind]++;
    p->prof.ms[q.kind] += ms;
    p->prof.flops[q.kind] += q.flops;
    p->prof.bytes[q.kind] += q.bytes;
    if (q.item >= 0) {
      if (p->item_ms.size() < p->var_items.size()) {
        p->item_ms.assign(p->var_items.size(), 0.0);
        p->item_count.assign(p->var_items.size(), 0);
      }
      p->item_ms[q.item] += ms;
      p->item_count[q.item]++;
    }
    p->event_pool.push_back(q.a);
    p->event_pool.push_back(q.b);
  }
  p->pending.clear();
}

// kind (profile slot), useful flops and algorithmic bytes of one item
static void item_cost(const tz_plan *p, const Item &it, int *kind, double *flops, double *bytes) {
  *flops = 0;
  *bytes = 0;
  switch (it.kind) {
    case IT_LEAVES:
      *kind = 0;
      for (size_t j = 0; j < p->jobs.size(); j++) *bytes += (double)p->esz * (int64_t(1) << p->jobs[j].rank);
      break;
    case IT_DIRECT:
      *kind = 1;
      for (int d = it.first; d < it.first + it.count; d++) {
        const PTensor &A = p->T[p->dstep_tensors[3 * d]], &B = p->T[p->dstep_tensors[3 * d + 1]],
                      &C = p->T[p->dstep_tensors[3 * d + 2]];
        *flops += 8.0 * std::ldexp(1.0, p->dsteps[d].nC + p->dsteps[d].nK);
        *bytes += (double)p->esz * (A.elems() + B.elems() + C.elems());
      }
      break;
    case IT_PERMUTE:
      *kind = 2;
      *bytes = 2.0 * p->esz * p->T[it.a].elems();
      break;
    case IT_GEMM: {
      const PStep &ps = p->S[it.a];
      const bool dot = ps.M * ps.N <= 64 && ps.K >= 64 && (ps.K % 2) == 0;
      *kind = ps.tc && !ps.tc_simt ? 4 : ps.skinny ? 6 : dot ? 7 : 3;
      *flops = 8.0 * ps.batch * (double)ps.M * (double)ps.N * (double)ps.K;
      *bytes = (double)p->esz * ps.batch * ((double)ps.M * ps.K + (double)ps.N * ps.K + (double)ps.M * ps.N);
      break;
    }
    default:
      *kind = 5;
      *bytes = 24.0 * (int64_t(1) << p->net.batch_log2);
  }
}

void item_cost_public(const tz_plan *p, int var_item, int *kind, double *flops, double *bytes) {
  item_cost(p, p->var_items[var_item], kind, flops, bytes);
}

static void run_items(tz_plan *p, const std::vector<Item> &items, const RunCtx &ctx) {
  cudaStream_t s = ctx.stream;
  auto *gs = reinterpret_cast<dev::GroupState *>(ctx.scratch + p->s_gs);
  const char *cbase = p->ws + p->off_const;
  char *abase = ctx.scratch + p->s_arena;
  const bool prof = p->profiling && !p->capturing;
  const bool is_var = &items == &p->var_items;
  for (size_t ii = 0; ii < items.size(); ii++) {
    const Item &it = items[ii];
    tz_plan::Pending pend{};
    if (prof) {
      item_cost(p, it, &pend.kind, &pend.flops, &pend.bytes);
      pend.item = is_var ? (int)ii : -1;
      pend.a = take_event(p);
      pend.b = take_event(p);
      cuda_check(cudaEventRecord(pend.a, s), "event record");
    }
    switch (it.kind) {
      case IT_LEAVES:
        if (!p->jobs.empty())
          cuda_check(dev::launch_leaf_build(reinterpret_cast<const dev::LeafJob *>(p->ws + p->off_jobs),
                                            (int)p->jobs.size(), gs,
                                            reinterpret_cast<const uint8_t *>(ctx.scratch + p->s_bits),
                                            p->net.n_qubits, p->net.batch_log2, cbase, abase, p->esz == 16, s),
                     "leaf build");
        break;
      case IT_DIRECT:
        if (it.queue)
          cuda_check(dev::launch_direct_queue(reinterpret_cast<const dev::DStep *>(p->ws + p->off_dsteps) + it.first,
                                              it.count,
                                              reinterpret_cast<const int *>(p->ws + p->off_bmap + it.bmap_off),
                                              it.blocks, cbase, abase,
                                              reinterpret_cast<unsigned *>(ctx.scratch + p->s_queue + it.ctrl_off),
                                              &gs->tc_error, p->esz == 16, s),
                     "direct step queue");
        else
          cuda_check(dev::launch_direct(reinterpret_cast<const dev::DStep *>(p->ws + p->off_dsteps) + it.first,
                                        it.count,
                                        reinterpret_cast<const int *>(p->ws + p->off_bmap + it.bmap_off),
                                        it.blocks, cbase, abase, p->esz == 16, s),
                     "direct steps");
        break;
      case IT_PERMUTE: {
        dev::PermuteArgs a{};
        const PTensor &src = p->T[it.a], &dst = p->T[it.b];
        a.rank = (int)dst.lay.size();
        for (int q = 0; q < a.rank; q++) a.perm[q] = (int8_t)pos_of(src.lay, dst.lay[q]);
        if (p->esz == 16)
          cuda_check(dev::launch_permute_z((const double2 *)tensor_ptr(p, ctx, it.a),
                                           (double2 *)tensor_ptr(p, ctx, it.b), a, s),
                     "permute");
        else
          cuda_check(dev::launch_permute((const float2 *)tensor_ptr(p, ctx, it.a), (float2 *)tensor_ptr(p, ctx, it.b),
                                         a, s),
                     "permute");
        break;
      }
      case IT_GEMM: {
        const PStep &ps = p->S[it.a];
        const float2 *X = (const float2 *)tensor_ptr(p, ctx, ps.opX);
        const float2 *Y = (const float2 *)tensor_ptr(p, ctx, ps.opY);
        float2 *C = (float2 *)tensor_ptr(p, ctx, ps.c_nat >= 0 ? ps.c_nat : ps.c);
        const dev::CScatter *sc = ps.row_major ? nullptr : &ps.scatter;
        if (p->esz == 16) {
          const double2 *Xz = (const double2 *)X, *Yz = (const double2 *)Y;
          double2 *Cz = (double2 *)C;
          if (ps.skinny)
            cuda_check(dev::launch_zskinny_gather(Xz, Yz, Cz, ps.batch, ps.M, ps.N, ps.K, ps.gather, sc, s),
                       "skinny gemm");
          else
            cuda_check(dev::launch_zgemm_simt(Xz, Yz, Cz, ps.batch, ps.M, ps.N, ps.K, ps.M * ps.K, ps.N * ps.K,
                                              ps.M * ps.N, sc, s),
                       "simt gemm");
        } else if (ps.skinny) {
          cuda_check(dev::launch_cgemm_skinny_gather(X, Y, C, ps.batch, ps.M, ps.N, ps.K, ps.gather, sc, s),
                     "skinny gemm");
        } else if (ps.tc_simt == 2) {
          cuda_check(dev::launch_cgemm_stream(X, Y, C, ps.batch, ps.M, ps.N, ps.K, ps.M * ps.K, ps.N * ps.K,
                                              ps.M * ps.N, sc, s),
                     "stream gemm");
        } else if (ps.tc && !ps.tc_simt) {
          void *scr = abase + ps.tc_scratch_off;
          cuda_check(dev::launch_cgemm_tc(p->opts.precision, X, Y, C, ps.batch, ps.M, ps.N, ps.K, ps.M * ps.K,
                                          ps.N * ps.K, ps.M * ps.N, sc, scr, (size_t)ps.tc_scratch, &gs->tc_error,
                                          s, ps.tc_pair, ps.tc_ksplit),
                     "tensor-core gemm");
        } else {
          cuda_check(dev::launch_cgemm_simt(X, Y, C, ps.batch, ps.M, ps.N, ps.K, ps.M * ps.K, ps.N * ps.K,
                                            ps.M * ps.N, sc, s),
                     "simt gemm");
        }
        break;
      }
      case IT_ACCUM: {
        dev::AccumArgs a{};
        a.root = tensor_ptr(p, ctx, p->root);
        a.dbl = p->esz == 16;
        a.acc = reinterpret_cast<double2 *>(ctx.scratch + p->s_acc);
        a.gs = gs;
        a.g = p->net.batch_log2;
        a.m = p->net.n_open;
        for (int j = 0; j < dev::kMaxBatch; j++) a.beta_pos[j] = -1;
        for (int j = 0; j < dev::kMaxOpen; j++) a.open_pos[j] = -1;
        for (size_t q = 0; q < p->T[p->root].lay.size(); q++) {
          int i = p->T[p->root].lay[q];
          if (p->net.is_batch(i))
            a.beta_pos[p->net.indices[i].segment] = (int8_t)q;
          else
            a.open_pos[p->net.indices[i].segment] = (int8_t)q;
        }
        a.scale_re = p->net.scalar.real();
        a.scale_im = p->net.scalar.imag();
        a.advance = 1;
        cuda_check(dev::launch_accumulate(a, s), "accumulate");
        break;
      }
    }
    if (prof) {
      cuda_check(cudaEventRecord(pend.b, s), "event record");
      p->pending.push_back(pend);
      if (p->pending.size() >= 4096) plan_profile_collect(p);
    }
  }
}

// ---------------------------------------------------------------- autotuner
// For every tensor-core step of the group, time the product's launch
// configurations (pairs of CTAs or single CTAs; K split or not) on the
// plan's own operand and scratch buffers, and keep the fastest. Choices are
// cached per (device, precision, product shape, output kind), so plans that
// share step shapes (other slicings, other bitstrings, server slots) reuse
// them. The buffers hold whatever the arena holds at bind time: the product
// writes only its own output buffer, which every group recomputes.
namespace {
struct TuneKey {
  int dev, prec;
  int64_t batch, M, N, K;
  int out;  // 0 row-major, 1 scatter
  bool operator<(const TuneKey &o) const {
    return std::tie(dev, prec, batch, M, N, K, out) < std::tie(o.dev, o.prec, o.batch, o.M, o.N, o.K, o.out);
  }
};
struct TuneChoice {
  int pair, ksplit, simt;
  float ms;
};
// products with at most this many complex K values also try the CUDA-core
// complex64 kernel (FP32 FMA: at least as accurate as the split products);
// with so few terms per output they are bound by writing C
constexpr int64_t kTuneSimtMaxK = 32;
std::atomic<int> g_tune_force_simt{0};  // test hook: 1 the tiled CUDA-core kernel, 2 the
                                        // stream kernel, wherever allowed
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune_cache;
}  // namespace

void tune_force_simt(int on) {
  g_tune_force_simt.store(on == 2 ? 2 : on ? 1 : 0);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache.clear();  // choices made under the other setting are not reused
}

void tune_preset(int precision, int64_t batch, int64_t M, int64_t N, int64_t K, int scatter, int pair, int ksplit,
                 int simt) {
  if (batch < 1 || M < 1 || N < 1 || K < 1 || (scatter != 0 && scatter != 1) || pair < -1 || pair > 1 ||
      (ksplit != 0 && ksplit != 1) || simt < 0 || simt > 2 || (simt && K > kTuneSimtMaxK))
    fail(TZ_EINVAL, "bad autotuner preset");
  int dev = 0;
  cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[TuneKey{dev, precision, batch, M, N, K, scatter}] = TuneChoice{simt ? -1 : pair, simt ? 0 : ksplit, simt, 0.f};
}

static void autotune_tc_steps(tz_plan *p) {
  cudaStream_t s = p->stream;
  const RunCtx ctx = default_ctx(p);
  auto *gs = reinterpret_cast<dev::GroupState *>(ctx.scratch + p->s_gs);
  char *abase = ctx.scratch + p->s_arena;
  int dev = 0;
  cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  cudaEvent_t e0, e1;
  cuda_check(cudaEventCreate(&e0), "event");
  cuda_check(cudaEventCreate(&e1), "event");
  int tuned = 0;
  try {
    for (const Item &it : p->var_items) {
      if (it.kind != IT_GEMM) continue;
      PStep &ps = p->S[it.a];
      const dev::CScatter *sc0 = ps.row_major ? nullptr : &ps.scatter;
      // the stream kernel is a candidate for every complex64 product with
      // few summed values that it supports, on the tensor-core path or not
      const bool stream_ok = p->esz == 8 && !ps.skinny && ps.K <= kTuneSimtMaxK &&
                             dev::cgemm_stream_supported(ps.batch, ps.M, ps.N, ps.K, sc0);
      if (!ps.tc && !stream_ok) continue;
      const TuneKey key{dev, p->opts.precision, ps.batch, ps.M, ps.N, ps.K, ps.row_major ? 0 : 1};
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto f = g_tune_cache.find(key);
        // (a preset of the stream kernel for a product it does not support
        // is not taken: the step is timed instead)
        if (f != g_tune_cache.end() && (f->second.simt != 2 || stream_ok)) {
          ps.tc_pair = f->second.pair;
          ps.tc_ksplit = f->second.ksplit;
          ps.tc_simt = f->second.simt;
          tuned++;
          continue;
        }
      }
      std::vector<int> pairs;
      if (ps.tc) pairs.push_back(0);
      if (ps.tc && dev::tc_pair_supported(p->opts.precision, ps.M, ps.N)) pairs.push_back(1);
      std::vector<int> splits = {0};
      if (ps.tc && ps.row_major && dev::cgemm_tc_split(p->opts.precision, ps.batch, ps.M, ps.N, ps.K) > 1)
        splits.push_back(1);
      const float2 *X = (const float2 *)tensor_ptr(p, ctx, ps.opX);
      const float2 *Y = (const float2 *)tensor_ptr(p, ctx, ps.opY);
      float2 *C = (float2 *)tensor_ptr(p, ctx, ps.c_nat >= 0 ? ps.c_nat : ps.c);
      const dev::CScatter *sc = ps.row_major ? nullptr : &ps.scatter;
      void *scr = abase + ps.tc_scratch_off;
      TuneChoice best{-1, 0, 0, 1e30f};
      auto time_it = [&](auto launch) {
        launch();  // warm-up
        cuda_check(cudaEventRecord(e0, s), "event");
        for (int r = 0; r < 3; r++) launch();
        cuda_check(cudaEventRecord(e1, s), "event");
        cuda_check(cudaEventSynchronize(e1), "event");
        float ms = 0;
        cuda_check(cudaEventElapsedTime(&ms, e0, e1), "event");
        return ms;
      };
      for (int pr : pairs)
        for (int ks : splits) {
          const float ms = time_it([&] {
            cuda_check(dev::launch_cgemm_tc(p->opts.precision, X, Y, C, ps.batch, ps.M, ps.N, ps.K, ps.M * ps.K,
                                            ps.N * ps.K, ps.M * ps.N, sc, scr, (size_t)ps.tc_scratch, &gs->tc_error,
                                            s, pr, ks),
                       "autotune launch");
          });
          if (ms < best.ms) best = TuneChoice{pr, ks, 0, ms};
        }
      const int force = g_tune_force_simt.load();
      if (ps.K <= kTuneSimtMaxK) {
        // the tiled CUDA-core kernel: simt = 1 on the tensor-core path, the
        // step's own kernel (0) otherwise
        const float ms = time_it([&] {
          cuda_check(dev::launch_cgemm_simt(X, Y, C, ps.batch, ps.M, ps.N, ps.K, ps.M * ps.K, ps.N * ps.K,
                                            ps.M * ps.N, sc, s),
                     "autotune launch");
        });
        if (ms < best.ms || (force == 1 && ps.tc)) best = TuneChoice{-1, 0, ps.tc ? 1 : 0, ms};
      }
      if (stream_ok) {
        const float ms = time_it([&] {
          cuda_check(dev::launch_cgemm_stream(X, Y, C, ps.batch, ps.M, ps.N, ps.K, ps.M * ps.K, ps.N * ps.K,
                                              ps.M * ps.N, sc, s),
                     "autotune launch");
        });
        if ((ms < best.ms && force != 1) || force == 2) best = TuneChoice{-1, 0, 2, ms};
      }
      ps.tc_pair = best.pair;
      ps.tc_ksplit = best.ksplit;
      ps.tc_simt = best.simt;
      tuned++;
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[key] = best;
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->stats.n_tuned_steps = tuned;
  // the launch count per group follows the choices
  int n = 0;
  for (const Item &it : p->var_items) {
    int c = 1;
    if (it.kind == IT_GEMM && p->S[it.a].tc && !p->S[it.a].tc_simt) {
      const PStep &ps = p->S[it.a];
      c = dev::cgemm_tc_launches(p->opts.precision, ps.batch, ps.M, ps.N, ps.K, !ps.row_major, ps.tc_ksplit);
    } else if (it.kind == IT_ACCUM) {
      c = dev::accumulate_launches(p->net.batch_log2, p->net.n_open);
    }
    n += c;
  }
  p->stats.n_launches_per_group = n;
}

static void clear_graphs(tz_plan *p) {
  // an executable graph still in flight is freed when it completes
  for (auto &g : p->graphs) {
    cudaGraphExecDestroy(g.e);
    cudaGraphDestroy(g.g);
  }
  p->graphs.clear();
}

void plan_bind(tz_plan *p, void *ws, size_t bytes) {
  const auto t_bind = std::chrono::steady_clock::now();
  if (!ws) fail(TZ_EINVAL, "workspace pointer is NULL");
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) fail(TZ_EINVAL, "workspace must be 256-byte aligned");
  if (bytes < p->total_bytes)
    fail(TZ_ENOMEM, "workspace too small: need " + std::to_string(p->total_bytes) + " bytes");
  cuda_check(cudaSetDevice(p->opts.device), "cudaSetDevice");
  clear_graphs(p);  // they hold pointers into the old workspace
  p->ws = static_cast<char *>(ws);
  p->ws_bytes = bytes;
  p->stream = static_cast<cudaStream_t>(p->opts.stream);
  cudaStream_t s = p->stream;
  // tables with resolved pointers
  std::vector<dev::DStep> ds = p->dsteps;
  for (size_t d = 0; d < ds.size(); d++) {
    ds[d].A = tensor_rel(p, p->dstep_tensors[3 * d]);
    ds[d].B = tensor_rel(p, p->dstep_tensors[3 * d + 1]);
    ds[d].C = tensor_rel(p, p->dstep_tensors[3 * d + 2]);
  }
  std::vector<dev::LeafJob> js = p->jobs;
  for (size_t j = 0; j < js.size(); j++) {
    js[j].dst = tensor_rel(p, p->job_tensors[2 * j]);
    js[j].src = p->job_tensors[2 * j + 1] >= 0 ? tensor_rel(p, p->job_tensors[2 * j + 1]) : 0;
  }
  if (!ds.empty())
    cuda_check(cudaMemcpyAsync(p->ws + p->off_dsteps, ds.data(), ds.size() * sizeof(dev::DStep),
                               cudaMemcpyHostToDevice, s),
               "upload step tables");
  if (!js.empty())
    cuda_check(cudaMemcpyAsync(p->ws + p->off_jobs, js.data(), js.size() * sizeof(dev::LeafJob),
                               cudaMemcpyHostToDevice, s),
               "upload leaf tables");
  if (!p->bmap.empty())
    cuda_check(cudaMemcpyAsync(p->ws + p->off_bmap, p->bmap.data(), p->bmap.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, s),
               "upload queue block maps");
  // constant leaves, in their planned storage order
  std::vector<float2> host;
  std::vector<double2> hostz;
  for (size_t t = 0; t < p->T.size(); t++) {
    const PTensor &x = p->T[t];
    if (x.region != R_CONST || x.leaf < 0) continue;
    if (x.var) continue;
    const Leaf &lf = p->net.leaves[x.leaf];
    host.assign(x.elems(), make_float2(0, 0));
    hostz.assign(x.elems(), make_double2(0, 0));
    std::vector<int> srcpos(x.lay.size());
    for (size_t q = 0; q < x.lay.size(); q++) srcpos[q] = pos_of(lf.idx, x.lay[q]);
    for (int64_t e = 0; e < x.elems(); e++) {
      int64_t so = 0;
      for (size_t q = 0; q < x.lay.size(); q++) so |= ((e >> q) & 1) << srcpos[q];
      host[e] = make_float2((float)lf.data[so].real(), (float)lf.data[so].imag());
      hostz[e] = make_double2(lf.data[so].real(), lf.data[so].imag());
    }
    if (p->esz == 16)
      cuda_check(cudaMemcpyAsync(tensor_ptr(p, default_ctx(p), (int)t), hostz.data(), hostz.size() * sizeof(double2),
                                 cudaMemcpyHostToDevice, s),
                 "upload constants");
    else
      cuda_check(cudaMemcpyAsync(tensor_ptr(p, default_ctx(p), (int)t), host.data(), host.size() * sizeof(float2),
                                 cudaMemcpyHostToDevice, s),
                 "upload constants");
    cuda_check(cudaStreamSynchronize(s), "sync");  // host buffer is reused
  }
  auto *gs = reinterpret_cast<dev::GroupState *>(default_ctx(p).scratch + p->s_gs);
  cuda_check(cudaMemsetAsync(&gs->tc_error, 0, sizeof(int), s), "clear error word");
  run_items(p, p->const_items, default_ctx(p));
  cuda_check(cudaStreamSynchronize(s), "bind-time steps");
  if (p->opts.autotune) autotune_tc_steps(p);
  if (read_tc_error(p, default_ctx(p)))
    fail(TZ_ETIMEOUT, "a tensor-core product of the bind-time steps timed out in a bounded wait");
  p->stats.bind_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_bind).count();
  p->bound = true;
}

int read_tc_error(const tz_plan *p, const RunCtx &ctx) {
  int v = 0;
  const auto *gs = reinterpret_cast<const dev::GroupState *>(ctx.scratch + p->s_gs);
  cuda_check(cudaMemcpy(&v, &gs->tc_error, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
  return v;
}

void plan_run(tz_plan *p, const RunCtx &ctx, int64_t n_rows, int64_t lo, int64_t hi, bool fresh) {
  if (!p->bound) fail(TZ_EINVAL, "plan has no workspace bound (tz_plan_bind_workspace)");
  cuda_check(cudaSetDevice(p->opts.device), "cudaSetDevice");
  cudaStream_t s = ctx.stream;
  auto *gs = reinterpret_cast<dev::GroupState *>(ctx.scratch + p->s_gs);
  if (fresh)
    cuda_check(cudaMemsetAsync(ctx.scratch + p->s_acc, 0, (size_t)n_rows * 16 << p->net.n_open, s),
               "clear accumulator");
  // queue launches leave their counters zeroed; this covers a scratch part
  // the plan has not run on before
  if (p->queue_bytes)
    cuda_check(cudaMemsetAsync(ctx.scratch + p->s_queue, 0, p->queue_bytes, s), "clear queue counters");
  cuda_check(dev::launch_init_state(gs, lo, hi, n_rows, s, fresh ? 0 : 1), "init group state");
  const int64_t chunk = int64_t(1) << p->net.batch_log2;
  const int64_t n_chunks = (n_rows + chunk - 1) / chunk;
  const int64_t n_groups = n_chunks * (hi - lo);
  cudaGraphExec_t exec = nullptr;
  if (p->opts.use_graph && s != nullptr && !p->profiling) {
    for (auto &g : p->graphs)
      if (g.scratch == ctx.scratch) exec = g.e;
    if (!exec) {
      cuda_check(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
      p->capturing = true;
      try {
        run_items(p, p->var_items, ctx);
      } catch (...) {
        p->capturing = false;
        cudaGraph_t g2 = nullptr;
        cudaStreamEndCapture(s, &g2);
        if (g2) cudaGraphDestroy(g2);
        throw;
      }
      p->capturing = false;
      tz_plan::Graph g{ctx.scratch, nullptr, nullptr};
      cuda_check(cudaStreamEndCapture(s, &g.g), "end capture");
      if (cudaGraphInstantiate(&g.e, g.g, 0) != cudaSuccess) {
        cudaGraphDestroy(g.g);
        fail(TZ_ECUDA, "instantiate graph");
      }
      if (p->graphs.size() >= tz_plan::kMaxGraphs) {
        cudaGraphExecDestroy(p->graphs.front().e);
        cudaGraphDestroy(p->graphs.front().g);
        p->graphs.erase(p->graphs.begin());
      }
      p->graphs.push_back(g);
      exec = g.e;
    }
  }
  for (int64_t gi = 0; gi < n_groups; gi++) {
    if (exec)
      cuda_check(cudaGraphLaunch(exec, s), "graph launch");
    else
      run_items(p, p->var_items, ctx);
  }
}

void plan_destroy(tz_plan *p) {
  if (!p) return;
  for (auto &q : p->pending) {
    cudaEventDestroy(q.a);
    cudaEventDestroy(q.b);
  }
  for (auto e : p->event_pool) cudaEventDestroy(e);
  clear_graphs(p);
  delete p;
}

}  // namespace tz
