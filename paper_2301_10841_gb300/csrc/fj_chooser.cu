// The learned plan chooser (no counterpart in the paper; the paper converts
// the binary plan a conventional optimizer picks, Section 4.1, and chooses
// covers per tuple by key counts, Section 4.4).
//
// A candidate is a left-deep join order -- converted by binary2fj and
// factored into the Free Join plan that runs -- together with a cover
// policy (the static first subatom, or the fewest-keys dynamic cover).  Its
// features describe the data the order meets:
//   * for each of the first kPositions relations of the order: log2 of its
//     row count / 32, and the 32-bucket histogram of log2 key degrees of the
//     column it joins on (fj_degree_histogram: a counter-based 1% sample of
//     the column, on the GPU);
//   * the number of atoms / 8, of variables / 32, whether the query is
//     cyclic, a constant 1, and the cover policy (0 static, 1 fewest).
// The network (fj_model) predicts the standardized log2 of the engine's work
// for a candidate; the chooser takes the candidate with the smallest
// prediction.  Every valid plan and policy gives the same result, so a wrong
// prediction costs time, never exactness; with no model the declared order
// with the static cover (the plain converted binary plan) is chosen.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/fj.h"
#include "fj_ctx_access.h"
#include "fj_plan.h"

using namespace fj;

namespace {

constexpr int kPositions = 4;
constexpr int kBuckets = 32;
static_assert(kPositions * (kBuckets + 1) + 5 == FJ_CHOOSER_IN_DIM, "feature layout");

thread_local std::string g_ch_err;

fj_status ch_fail(fj_status st, const std::string& m) {
  g_ch_err = m;
  return st;
}

// SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
// generators", 2014): the candidate sampler's generator.
uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

uint64_t atom_mask(const PQuery& q, int a) {
  uint64_t m = 0;
  for (int v : q.atom_vars[a]) m |= 1ull << v;
  return m;
}

// Every left-deep order whose prefixes are connected (no Cartesian
// product), enumerated depth first; stops after `cap` orders.
void connected_orders(const PQuery& q, std::vector<int>& cur, uint64_t used, uint64_t bound,
                      size_t cap, std::vector<std::vector<int>>& out) {
  const int n = int(q.atom_vars.size());
  if (out.size() >= cap) return;
  if (int(cur.size()) == n) {
    out.push_back(cur);
    return;
  }
  for (int a = 0; a < n; ++a) {
    if (used >> a & 1) continue;
    const uint64_t m = atom_mask(q, a);
    if (!cur.empty() && !(m & bound)) continue;
    cur.push_back(a);
    connected_orders(q, cur, used | (1ull << a), bound | m, cap, out);
    cur.pop_back();
  }
}

// The candidate orders: the declared order 0..n-1 first, then at most
// limit - 1 others drawn without replacement (seeded) from the connected
// orders.
std::vector<std::vector<int>> candidate_orders(const PQuery& q, int limit, uint64_t seed) {
  const int n = int(q.atom_vars.size());
  std::vector<int> declared(n);
  for (int i = 0; i < n; ++i) declared[i] = i;
  std::vector<std::vector<int>> all;
  std::vector<int> cur;
  connected_orders(q, cur, 0, 0, 40320, all);
  std::vector<std::vector<int>> rest;
  for (auto& o : all)
    if (o != declared) rest.push_back(o);
  uint64_t s = seed;
  const size_t want = size_t(std::max(0, limit - 1));
  for (size_t i = 0; i < rest.size() && i < want; ++i) {  // partial Fisher-Yates
    const size_t j = i + size_t(splitmix64(s) % (rest.size() - i));
    std::swap(rest[i], rest[j]);
  }
  if (rest.size() > want) rest.resize(want);
  std::vector<std::vector<int>> out{declared};
  for (auto& o : rest) out.push_back(o);
  return out;
}

struct Features {
  fj_ctx* ctx;
  const fj_query* query;
  PQuery q;
  std::map<std::pair<int, int>, std::vector<float>> hist;  // (atom, var index)

  fj_status histogram(int a, int j, const float** out) {
    auto key = std::make_pair(a, j);
    auto it = hist.find(key);
    if (it == hist.end()) {
      const fj_atom& at = query->atoms[a];
      const int col = at.cols ? at.cols[j] : j;
      const int32_t* d = fj_internal_rel_col(at.rel, col);
      if (!d) return ch_fail(FJ_ERR_INVALID_ARG, "atom column out of range");
      std::vector<float> h(kBuckets, 0.f);
      fj_status st = fj_degree_histogram(ctx, d, fj_relation_rows(at.rel), 100,
                                         uint32_t(31 * a + j), h.data());
      if (st != FJ_OK) return ch_fail(st, std::string("features: ") + fj_stats_last_error());
      it = hist.emplace(key, std::move(h)).first;
    }
    *out = it->second.data();
    return FJ_OK;
  }

  fj_status of(const std::vector<int>& order, int policy, float* f) {
    const int n = int(q.atom_vars.size());
    uint64_t all = 0, bound = 0;
    int arity = 0;
    for (int a = 0; a < n; ++a) {
      all |= atom_mask(q, a);
      arity += int(q.atom_vars[a].size());
    }
    const int n_vars = __builtin_popcountll(all);
    const bool cyclic = arity - n_vars >= n;
    int w = 0;
    for (int pos = 0; pos < kPositions; ++pos) {
      if (pos >= int(order.size())) {
        for (int b = 0; b < kBuckets + 1; ++b) f[w++] = 0.f;
        continue;
      }
      const int a = order[pos];
      const auto& vs = q.atom_vars[a];
      // The column it joins on: for the first relation, its first variable
      // shared with the second; otherwise its first variable already bound.
      const uint64_t with = pos == 0 ? (order.size() > 1 ? atom_mask(q, order[1]) : 0) : bound;
      int j = 0;
      for (int k = 0; k < int(vs.size()); ++k)
        if (with >> vs[k] & 1) {
          j = k;
          break;
        }
      const float* h = nullptr;
      fj_status st = histogram(a, j, &h);
      if (st != FJ_OK) return st;
      f[w++] = float(std::log2(double(fj_relation_rows(query->atoms[a].rel)) + 1.0) / 32.0);
      for (int b = 0; b < kBuckets; ++b) f[w++] = h[b];
      bound |= atom_mask(q, a);
    }
    f[w++] = float(order.size()) / 8.f;
    f[w++] = float(n_vars) / 32.f;
    f[w++] = cyclic ? 1.f : 0.f;
    f[w++] = 1.f;
    f[w++] = policy == FJ_COVER_FEWEST ? 1.f : 0.f;
    return FJ_OK;
  }
};

fj_status init_features(Features& F, fj_ctx* ctx, const fj_query* query) {
  F.ctx = ctx;
  F.query = query;
  if (!ctx || !query) return ch_fail(FJ_ERR_INVALID_ARG, "NULL context or query");
  if (!load_query(query, F.q)) return ch_fail(FJ_ERR_INVALID_ARG, get_error());
  for (int a = 0; a < query->n_atoms; ++a)
    if (!query->atoms[a].rel) return ch_fail(FJ_ERR_INVALID_ARG, "atom without a relation");
  return FJ_OK;
}

// The order in which a plan's subatoms first reach each atom.
std::vector<int> appearance_order(const PPlan& plan, int n_atoms) {
  std::vector<int> order;
  uint64_t seen = 0;
  for (const PNode& node : plan)
    for (const PSub& s : node)
      if (!(seen >> s.atom & 1)) {
        seen |= 1ull << s.atom;
        order.push_back(s.atom);
      }
  for (int a = 0; a < n_atoms; ++a)
    if (!(seen >> a & 1)) order.push_back(a);
  return order;
}

}  // namespace

extern "C" {

const char* fj_chooser_last_error(void) { return g_ch_err.c_str(); }

fj_status fj_plan_features(fj_ctx* ctx, const fj_query* query, int n_candidates,
                           const int* orders, const int* cover_policies, float* host_out) {
  g_ch_err.clear();
  Features F;
  fj_status st = init_features(F, ctx, query);
  if (st != FJ_OK) return st;
  if (n_candidates < 0 || (n_candidates && (!orders || !cover_policies || !host_out)))
    return ch_fail(FJ_ERR_INVALID_ARG, "NULL candidate arrays");
  const int n = query->n_atoms;
  for (int c = 0; c < n_candidates; ++c) {
    std::vector<int> o(orders + size_t(c) * n, orders + size_t(c + 1) * n), chk(o);
    std::sort(chk.begin(), chk.end());
    for (int i = 0; i < n; ++i)
      if (chk[i] != i)
        return ch_fail(FJ_ERR_INVALID_ARG,
                       "candidate " + std::to_string(c) + ": the order must list every atom once");
    const int pol = cover_policies[c];
    if (pol != FJ_COVER_STATIC && pol != FJ_COVER_FEWEST)
      return ch_fail(FJ_ERR_INVALID_ARG, "cover policy must be static or fewest");
    st = F.of(o, pol, host_out + size_t(c) * FJ_CHOOSER_IN_DIM);
    if (st != FJ_OK) return st;
  }
  return FJ_OK;
}

fj_status fj_choose_plan(fj_ctx* ctx, const fj_query* query, const fj_model* model,
                         int max_candidates, uint64_t seed, fj_plan** out_plan,
                         int* out_cover_policy, int* out_order) {
  g_ch_err.clear();
  if (!out_plan || !out_cover_policy) return ch_fail(FJ_ERR_INVALID_ARG, "NULL output");
  *out_plan = nullptr;
  Features F;
  fj_status st = init_features(F, ctx, query);
  if (st != FJ_OK) return st;
  const int n = query->n_atoms;
  std::vector<std::vector<int>> orders =
      candidate_orders(F.q, std::max(1, max_candidates), seed);
  std::vector<int> best = orders[0];
  int policy = FJ_COVER_STATIC;
  if (model) {
    const int nc = int(orders.size()) * 2;
    std::vector<float> x(size_t(nc) * FJ_CHOOSER_IN_DIM), y(nc);
    for (int c = 0; c < nc; ++c) {
      st = F.of(orders[c / 2], c % 2 ? FJ_COVER_FEWEST : FJ_COVER_STATIC,
                x.data() + size_t(c) * FJ_CHOOSER_IN_DIM);
      if (st != FJ_OK) return st;
    }
    st = fj_internal_model_predict(const_cast<fj_model*>(model), x.data(), nc,
                                   FJ_CHOOSER_IN_DIM, y.data());
    if (st != FJ_OK) return ch_fail(st, std::string("chooser: ") + fj_model_last_error());
    int arg = 0;
    for (int c = 1; c < nc; ++c)
      if (y[c] < y[arg]) arg = c;
    best = orders[arg / 2];
    policy = arg % 2 ? FJ_COVER_FEWEST : FJ_COVER_STATIC;
  }
  PPlan plan = factor(binary2fj(F.q, best));
  *out_plan = export_plan(plan);
  *out_cover_policy = policy;
  if (out_order)
    for (int i = 0; i < n; ++i) out_order[i] = best[i];
  return FJ_OK;
}

}  // extern "C"

// The learned cover policy of a prepared plan (FJ_COVER_LEARNED): the
// policy the network predicts cheaper for the plan's appearance order.
fj_status fj_internal_learned_policy(fj_ctx* ctx, const fj_query* query, const PPlan& plan,
                                     const fj_model* model, int* policy) {
  Features F;
  fj_status st = init_features(F, ctx, query);
  if (st != FJ_OK) return st;
  if (!model) return ch_fail(FJ_ERR_INVALID_ARG, "FJ_COVER_LEARNED needs a model");
  const std::vector<int> order = appearance_order(plan, query->n_atoms);
  float x[2 * FJ_CHOOSER_IN_DIM], y[2];
  if ((st = F.of(order, FJ_COVER_STATIC, x)) != FJ_OK ||
      (st = F.of(order, FJ_COVER_FEWEST, x + FJ_CHOOSER_IN_DIM)) != FJ_OK)
    return st;
  st = fj_internal_model_predict(const_cast<fj_model*>(model), x, 2, FJ_CHOOSER_IN_DIM, y);
  if (st != FJ_OK) return ch_fail(st, std::string("learned cover: ") + fj_model_last_error());
  *policy = y[1] < y[0] ? FJ_COVER_FEWEST : FJ_COVER_STATIC;
  return FJ_OK;
}

const char* fj_internal_chooser_error() { return g_ch_err.c_str(); }
