// Free Join oracle: plain, slow, obviously-correct CPU evaluation of a full
// conjunctive query under bag semantics.
//
// TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
// call this file; only the test suite, the smoke check and the CPU-baseline
// leg of the benchmark do.  It shares no code, header or constant with the
// CUDA library.
//
// What is computed (paper Section 2.1, Eq. 1, with the bag-semantics
// footnotes of Sections 2.2 and 2.3): for Q(x) :- R1(x1), ..., Rm(xm), the
// result is the multiset of head tuples obtained from every combination of one
// row per atom whose values agree on every shared variable.  Selections are
// pushed to the atoms (Section 2.1): an atom only contributes rows that pass
// all of its predicates.
//
// Two independent evaluations of that definition are given:
//   * oracle_binary_join  -- a left-deep pipelined hash join in the order the
//     caller gives (Section 2.2, Fig. 2a, Example 2.2): one hash table per
//     right-hand relation keyed on the variables it shares with everything
//     to its left, probed tuple by tuple.
//   * oracle_generic_join -- textbook Generic Join (Section 2.3, Fig. 2b):
//     one full hash trie per atom following a total variable order, one loop
//     per variable, intersecting by iterating the smallest key set and
//     probing the others; leaf multiplicities are multiplied for bags.
// Both report COUNT(*) (uint64), MIN of requested variables (int32, with a
// validity flag for the empty result), and optionally the full output as
// head-ordered int32 tuples sorted lexicographically (signed order),
// duplicates kept.
//
// Error returns: 0 ok; -1 invalid argument; -4 output buffer too small (the
// count and n_out are still exact); -5 count overflow (not reachable at the
// sizes used).

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <unordered_map>
#include <vector>

namespace {

constexpr int kMaxVars = 64;

struct OAtom {
  int n_vars;
  const int32_t* const* cols;  // cols[j] = column holding variable vars[j]
  uint64_t n_rows;
  const int* vars;
  int n_preds;
  const int* pred_col;  // index j into cols
  const int* pred_op;   // 0 <, 1 <=, 2 >, 3 >=, 4 ==, 5 !=
  const int32_t* pred_val;
};

bool passes(const OAtom& a, uint64_t r) {
  for (int p = 0; p < a.n_preds; ++p) {
    int32_t v = a.cols[a.pred_col[p]][r];
    int32_t c = a.pred_val[p];
    bool ok = false;
    switch (a.pred_op[p]) {
      case 0: ok = v < c; break;
      case 1: ok = v <= c; break;
      case 2: ok = v > c; break;
      case 3: ok = v >= c; break;
      case 4: ok = v == c; break;
      case 5: ok = v != c; break;
      default: ok = false;
    }
    if (!ok) return false;
  }
  return true;
}

// Hash of a vector<int32_t> key for std::unordered_map (any hash is correct;
// equality decides membership).
struct VecHash {
  size_t operator()(const std::vector<int32_t>& k) const {
    size_t h = 1469598103934665603ull;
    for (int32_t v : k) {
      h ^= static_cast<uint32_t>(v);
      h *= 1099511628211ull;
    }
    return h;
  }
};

// Collects the result: count, mins and (optionally) materialized tuples.
struct Sink {
  int n_head;
  const int* head;
  int n_min;
  const int* min_vars;
  uint64_t count = 0;
  bool overflow = false;
  std::vector<int32_t> mins;
  std::vector<uint8_t> min_valid;
  int32_t* out;  // may be null
  uint64_t out_cap;

  void init() {
    mins.assign(n_min, INT32_MAX);
    min_valid.assign(n_min, 0);
  }
  // Emit the current binding `mult` times.
  void emit(const int32_t* bind, uint64_t mult) {
    if (mult == 0) return;
    uint64_t before = count;
    count += mult;
    if (count < before) overflow = true;
    for (int i = 0; i < n_min; ++i) {
      int32_t v = bind[min_vars[i]];
      if (!min_valid[i] || v < mins[i]) mins[i] = v;
      min_valid[i] = 1;
    }
    if (out) {
      for (uint64_t m = 0; m < mult; ++m) {
        uint64_t row = before + m;
        if (row >= out_cap) break;
        for (int h = 0; h < n_head; ++h) out[row * n_head + h] = bind[head[h]];
      }
    }
  }
  int finish(uint64_t* count_out, int32_t* mins_out, uint8_t* valid_out,
             uint64_t* n_out) {
    *count_out = count;
    for (int i = 0; i < n_min; ++i) {
      mins_out[i] = mins[i];
      valid_out[i] = min_valid[i];
    }
    if (n_out) *n_out = count;
    if (out) {
      uint64_t n = std::min(count, out_cap);
      // Sort the rows lexicographically under signed int32 order.
      std::vector<uint64_t> idx(n);
      for (uint64_t i = 0; i < n; ++i) idx[i] = i;
      int w = n_head;
      const int32_t* base = out;
      std::sort(idx.begin(), idx.end(), [base, w](uint64_t a, uint64_t b) {
        for (int h = 0; h < w; ++h) {
          int32_t x = base[a * w + h], y = base[b * w + h];
          if (x != y) return x < y;
        }
        return false;
      });
      std::vector<int32_t> tmp(static_cast<size_t>(n) * w);
      for (uint64_t i = 0; i < n; ++i)
        std::memcpy(&tmp[i * w], &base[idx[i] * w], sizeof(int32_t) * w);
      if (n) std::memcpy(out, tmp.data(), sizeof(int32_t) * n * w);
      if (count > out_cap) return -4;
    }
    if (overflow) return -5;
    return 0;
  }
};

bool check_query(int n_atoms, const OAtom* atoms, int n_head, const int* head,
                 int n_min, const int* min_vars) {
  if (n_atoms <= 0) return false;
  std::vector<int> seen(kMaxVars, 0);
  for (int i = 0; i < n_atoms; ++i) {
    const OAtom& a = atoms[i];
    if (a.n_vars <= 0) return false;
    std::vector<int> local(kMaxVars, 0);
    for (int j = 0; j < a.n_vars; ++j) {
      int v = a.vars[j];
      if (v < 0 || v >= kMaxVars || local[v]) return false;  // distinct vars
      local[v] = 1;
      seen[v] = 1;
    }
    for (int p = 0; p < a.n_preds; ++p)
      if (a.pred_col[p] < 0 || a.pred_col[p] >= a.n_vars) return false;
  }
  // The query is full: the head lists every variable exactly once.
  std::vector<int> inhead(kMaxVars, 0);
  for (int h = 0; h < n_head; ++h) {
    int v = head[h];
    if (v < 0 || v >= kMaxVars || !seen[v] || inhead[v]) return false;
    inhead[v] = 1;
  }
  for (int v = 0; v < kMaxVars; ++v)
    if (seen[v] && !inhead[v]) return false;
  for (int i = 0; i < n_min; ++i)
    if (min_vars[i] < 0 || min_vars[i] >= kMaxVars || !seen[min_vars[i]])
      return false;
  return true;
}

// ---------------------------------------------------------------------------
// O1: left-deep pipelined hash join (Section 2.2).
// ---------------------------------------------------------------------------
struct BinaryJoin {
  const OAtom* atoms;
  std::vector<int> order;
  // For position s >= 1: key variable positions (indices j into atom columns)
  // and the remaining (new) variable positions.
  std::vector<std::vector<int>> key_pos, new_pos;
  std::vector<std::unordered_map<std::vector<int32_t>, std::vector<uint64_t>,
                                 VecHash>>
      tables;
  int32_t bind[kMaxVars];
  Sink* sink;

  void build() {
    int m = static_cast<int>(order.size());
    std::vector<int> bound(kMaxVars, 0);
    key_pos.assign(m, {});
    new_pos.assign(m, {});
    tables.resize(m);
    const OAtom& r1 = atoms[order[0]];
    for (int j = 0; j < r1.n_vars; ++j) bound[r1.vars[j]] = 1;
    for (int s = 1; s < m; ++s) {
      const OAtom& a = atoms[order[s]];
      for (int j = 0; j < a.n_vars; ++j) {
        if (bound[a.vars[j]])
          key_pos[s].push_back(j);
        else
          new_pos[s].push_back(j);
      }
      for (int j = 0; j < a.n_vars; ++j) bound[a.vars[j]] = 1;
      // Hash table: key = values of the shared variables -> rows.
      for (uint64_t r = 0; r < a.n_rows; ++r) {
        if (!passes(a, r)) continue;
        std::vector<int32_t> key;
        for (int j : key_pos[s]) key.push_back(a.cols[j][r]);
        tables[s][key].push_back(r);
      }
    }
  }

  void probe(int s) {
    int m = static_cast<int>(order.size());
    if (s == m) {
      sink->emit(bind, 1);
      return;
    }
    const OAtom& a = atoms[order[s]];
    std::vector<int32_t> key;
    for (int j : key_pos[s]) key.push_back(bind[a.vars[j]]);
    auto it = tables[s].find(key);
    if (it == tables[s].end()) return;
    for (uint64_t r : it->second) {
      for (int j : new_pos[s]) bind[a.vars[j]] = a.cols[j][r];
      probe(s + 1);
    }
  }

  void run() {
    build();
    const OAtom& r1 = atoms[order[0]];
    for (uint64_t r = 0; r < r1.n_rows; ++r) {
      if (!passes(r1, r)) continue;
      for (int j = 0; j < r1.n_vars; ++j) bind[r1.vars[j]] = r1.cols[j][r];
      probe(1);
    }
  }
};

// ---------------------------------------------------------------------------
// O2: Generic Join over full hash tries (Section 2.3).
// ---------------------------------------------------------------------------
struct TrieNode {
  // Interior: value -> child.  Leaf (all variables consumed): multiplicity.
  std::unordered_map<int32_t, std::unique_ptr<TrieNode>> child;
  uint64_t mult = 0;
};

struct GenericJoin {
  const OAtom* atoms;
  int n_atoms;
  std::vector<int> var_order;            // total order of variables
  std::vector<std::vector<int>> levels;  // per atom: column index per level
  std::vector<std::unique_ptr<TrieNode>> roots;
  int32_t bind[kMaxVars];
  Sink* sink;

  void build() {
    levels.assign(n_atoms, {});
    roots.clear();
    for (int i = 0; i < n_atoms; ++i) {
      const OAtom& a = atoms[i];
      // The atom's trie levels follow the global variable order.
      for (int v : var_order)
        for (int j = 0; j < a.n_vars; ++j)
          if (a.vars[j] == v) levels[i].push_back(j);
      roots.emplace_back(new TrieNode());
      for (uint64_t r = 0; r < a.n_rows; ++r) {
        if (!passes(a, r)) continue;
        TrieNode* n = roots[i].get();
        for (int j : levels[i]) {
          auto& c = n->child[a.cols[j][r]];
          if (!c) c.reset(new TrieNode());
          n = c.get();
        }
        n->mult += 1;
      }
    }
  }

  // cur[i] = current trie node of atom i.
  void recurse(size_t depth, std::vector<TrieNode*>& cur) {
    if (depth == var_order.size()) {
      uint64_t mult = 1;
      for (int i = 0; i < n_atoms; ++i) {
        uint64_t m = cur[i]->mult;
        if (m != 0 && mult > UINT64_MAX / m) sink->overflow = true;
        mult *= m;
      }
      sink->emit(bind, mult);
      return;
    }
    int x = var_order[depth];
    std::vector<int> rel;  // atoms containing x
    for (int i = 0; i < n_atoms; ++i)
      for (int j = 0; j < atoms[i].n_vars; ++j)
        if (atoms[i].vars[j] == x) rel.push_back(i);
    // Iterate the smallest key set, probe the rest.
    int best = rel[0];
    for (int i : rel)
      if (cur[i]->child.size() < cur[best]->child.size()) best = i;
    for (auto& kv : cur[best]->child) {
      int32_t val = kv.first;
      std::vector<TrieNode*> saved(rel.size());
      bool ok = true;
      for (size_t t = 0; t < rel.size(); ++t) {
        int i = rel[t];
        saved[t] = cur[i];
        auto it = cur[i]->child.find(val);
        if (it == cur[i]->child.end()) {
          ok = false;
          break;
        }
      }
      if (!ok) continue;
      for (size_t t = 0; t < rel.size(); ++t) {
        int i = rel[t];
        cur[i] = cur[i]->child.find(val)->second.get();
      }
      bind[x] = val;
      recurse(depth + 1, cur);
      for (size_t t = 0; t < rel.size(); ++t) cur[rel[t]] = saved[t];
    }
  }

  void run() {
    build();
    std::vector<TrieNode*> cur(n_atoms);
    for (int i = 0; i < n_atoms; ++i) cur[i] = roots[i].get();
    recurse(0, cur);
  }
};

}  // namespace

extern "C" {

// Atom descriptor shared with the Python wrapper (ctypes).
typedef struct {
  int n_vars;
  const int32_t* const* cols;
  uint64_t n_rows;
  const int* vars;
  int n_preds;
  const int* pred_col;
  const int* pred_op;
  const int32_t* pred_val;
} oracle_atom;

int oracle_binary_join(int n_atoms, const oracle_atom* atoms, const int* order,
                       int n_head, const int* head, int n_min,
                       const int* min_vars, uint64_t* count, int32_t* mins,
                       uint8_t* min_valid, int32_t* out, uint64_t out_cap,
                       uint64_t* n_out) {
  static_assert(sizeof(oracle_atom) == sizeof(OAtom), "layout");
  const OAtom* a = reinterpret_cast<const OAtom*>(atoms);
  if (!check_query(n_atoms, a, n_head, head, n_min, min_vars)) return -1;
  std::vector<int> ord(order, order + n_atoms);
  {
    std::vector<int> chk(ord);
    std::sort(chk.begin(), chk.end());
    for (int i = 0; i < n_atoms; ++i)
      if (chk[i] != i) return -1;
  }
  Sink sink{n_head, head, n_min, min_vars};
  sink.out = out;
  sink.out_cap = out_cap;
  sink.init();
  BinaryJoin bj;
  bj.atoms = a;
  bj.order = ord;
  bj.sink = &sink;
  bj.run();
  return sink.finish(count, mins, min_valid, n_out);
}

int oracle_generic_join(int n_atoms, const oracle_atom* atoms,
                        const int* var_order, int n_order, int n_head,
                        const int* head, int n_min, const int* min_vars,
                        uint64_t* count, int32_t* mins, uint8_t* min_valid,
                        int32_t* out, uint64_t out_cap, uint64_t* n_out) {
  const OAtom* a = reinterpret_cast<const OAtom*>(atoms);
  if (!check_query(n_atoms, a, n_head, head, n_min, min_vars)) return -1;
  // The variable order must list each head variable exactly once.
  if (n_order != n_head) return -1;
  {
    std::vector<int> x(var_order, var_order + n_order), y(head, head + n_head);
    std::sort(x.begin(), x.end());
    std::sort(y.begin(), y.end());
    if (x != y) return -1;
  }
  Sink sink{n_head, head, n_min, min_vars};
  sink.out = out;
  sink.out_cap = out_cap;
  sink.init();
  GenericJoin gj;
  gj.atoms = a;
  gj.n_atoms = n_atoms;
  gj.var_order.assign(var_order, var_order + n_order);
  gj.sink = &sink;
  gj.run();
  return sink.finish(count, mins, min_valid, n_out);
}

}  // extern "C"
