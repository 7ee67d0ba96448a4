// Free Join plans on the host: loading and checking queries and plans
// (Section 2.1 Eq. 1; Section 3.2 Def. 3.4-3.7), converting a left-deep
// binary plan (Section 4.1 Fig. 9, binary2fj), and factoring it (Section 4.1
// Fig. 10, factor).
//
// Readings of passages the paper leaves open:
//  * binary2fj: the variables "available" while the current node is built
//    are all variables bound so far, including the current node's own;
//    otherwise the chain example of Section 4.1 would not convert as printed.
//    A relation whose variables are all bound already becomes the empty
//    subatom s(), which iterates its leaf vector (the bag multiplicity).
//  * factor: only non-cover subatoms may move, in node order, and the first
//    that cannot move ends the node (the conservative rule); nodes are
//    visited from the last to the second and a moved subatom is appended to
//    the previous node, where it may move again.  This reproduces the
//    optimized clover plan printed in Section 4.1.
#include <algorithm>
#include <cstring>
#include <memory>

#include "fj_plan.h"

namespace fj {

namespace {
thread_local std::string g_error;
}

void set_error(const std::string& msg) { g_error = msg; }
const char* get_error() { return g_error.c_str(); }

bool load_query(const fj_query* q, PQuery& out) {
  if (!q || q->n_atoms <= 0 || q->n_atoms > FJ_MAX_ATOMS || !q->atoms) {
    set_error("query: need 1..FJ_MAX_ATOMS atoms");
    return false;
  }
  out.atom_vars.assign(q->n_atoms, {});
  uint64_t seen = 0;
  std::vector<int> first_order;
  for (int i = 0; i < q->n_atoms; ++i) {
    const fj_atom& a = q->atoms[i];
    if (a.n_vars <= 0 || a.n_vars > FJ_MAX_ARITY || !a.vars) {
      set_error("query: atom " + std::to_string(i) + " needs 1..FJ_MAX_ARITY vars");
      return false;
    }
    uint64_t local = 0;
    for (int j = 0; j < a.n_vars; ++j) {
      int v = a.vars[j];
      if (v < 0 || v >= FJ_MAX_VARS) {
        set_error("query: variable id out of range in atom " + std::to_string(i));
        return false;
      }
      if (local >> v & 1) {
        set_error("query: repeated variable in atom " + std::to_string(i));
        return false;
      }
      local |= 1ull << v;
      if (!(seen >> v & 1)) first_order.push_back(v);
      seen |= 1ull << v;
      out.atom_vars[i].push_back(v);
    }
    if (a.n_preds < 0 || a.n_preds > FJ_MAX_PREDS || (a.n_preds && !a.preds)) {
      set_error("query: bad predicate list in atom " + std::to_string(i));
      return false;
    }
    for (int p = 0; p < a.n_preds; ++p) {
      if (a.preds[p].col < 0 || a.preds[p].col >= a.n_vars || a.preds[p].op < FJ_LT ||
          a.preds[p].op > FJ_NE) {
        set_error("query: bad predicate in atom " + std::to_string(i));
        return false;
      }
    }
  }
  if (q->head_vars) {
    if (q->n_head != int(first_order.size())) {
      set_error("query: the head must list every variable exactly once (full query)");
      return false;
    }
    uint64_t h = 0;
    for (int k = 0; k < q->n_head; ++k) {
      int v = q->head_vars[k];
      if (v < 0 || v >= FJ_MAX_VARS || !(seen >> v & 1) || (h >> v & 1)) {
        set_error("query: the head must list every variable exactly once (full query)");
        return false;
      }
      h |= 1ull << v;
      out.head.push_back(v);
    }
  } else {
    out.head = first_order;
  }
  return true;
}

bool load_plan(const PQuery& q, const fj_plan* p, PPlan& out) {
  if (!p || p->n_nodes <= 0 || p->n_nodes > FJ_MAX_NODES || !p->nodes) {
    set_error("plan: need 1..FJ_MAX_NODES nodes");
    return false;
  }
  out.assign(p->n_nodes, {});
  for (int k = 0; k < p->n_nodes; ++k) {
    const fj_node& n = p->nodes[k];
    if (n.n_sub <= 0 || n.n_sub > FJ_MAX_SUB || !n.sub) {
      set_error("plan: node " + std::to_string(k) + " needs 1..FJ_MAX_SUB subatoms");
      return false;
    }
    for (int s = 0; s < n.n_sub; ++s) {
      const fj_subatom& sa = n.sub[s];
      if (sa.atom < 0 || sa.atom >= int(q.atom_vars.size()) || sa.n_vars < 0 ||
          (sa.n_vars && !sa.vars)) {
        set_error("plan: bad subatom in node " + std::to_string(k));
        return false;
      }
      uint64_t m = 0;
      for (int j = 0; j < sa.n_vars; ++j) {
        int v = sa.vars[j];
        const auto& av = q.atom_vars[sa.atom];
        if (v < 0 || v >= FJ_MAX_VARS || std::find(av.begin(), av.end(), v) == av.end() ||
            (m >> v & 1)) {
          set_error("plan: subatom variables must be distinct variables of its atom (node " +
                    std::to_string(k) + ")");
          return false;
        }
        m |= 1ull << v;
      }
      PSub ps{sa.atom, {}};
      for (int v : q.atom_vars[sa.atom])
        if (m >> v & 1) ps.vars.push_back(v);
      out[k].push_back(ps);
    }
  }
  return true;
}

uint64_t vs_mask(const PNode& node) {
  uint64_t m = 0;
  for (const PSub& s : node)
    for (int v : s.vars) m |= 1ull << v;
  return m;
}

uint64_t avs_mask(const PPlan& plan, int k) {
  uint64_t m = 0;
  for (int j = 0; j < k; ++j) m |= vs_mask(plan[j]);
  return m;
}

std::vector<int> covers(const PPlan& plan, int k) {
  uint64_t need = vs_mask(plan[k]) & ~avs_mask(plan, k);
  std::vector<int> out;
  for (int s = 0; s < int(plan[k].size()); ++s) {
    uint64_t m = 0;
    for (int v : plan[k][s].vars) m |= 1ull << v;
    if ((need & ~m) == 0) out.push_back(s);
  }
  return out;
}

bool validate(const PQuery& q, const PPlan& plan) {
  int na = int(q.atom_vars.size());
  std::vector<uint64_t> got(na, 0);
  std::vector<int> appears(na, 0);
  for (int k = 0; k < int(plan.size()); ++k) {
    uint64_t atoms_here = 0;
    for (const PSub& s : plan[k]) {
      if (atoms_here >> s.atom & 1) {
        set_error("invalid plan: node " + std::to_string(k) +
                  " has two subatoms of one atom (Def. 3.7 a)");
        return false;
      }
      atoms_here |= 1ull << s.atom;
      for (int v : s.vars) {
        if (got[s.atom] >> v & 1) {
          set_error("invalid plan: a variable of atom " + std::to_string(s.atom) +
                    " appears in two subatoms (Def. 3.5)");
          return false;
        }
        got[s.atom] |= 1ull << v;
      }
      appears[s.atom] = 1;
    }
    auto cv = covers(plan, k);
    if (cv.empty()) {
      set_error("invalid plan: node " + std::to_string(k) + " has no cover (Def. 3.7 b)");
      return false;
    }
    if (cv[0] != 0) {
      set_error("invalid plan: the first subatom of node " + std::to_string(k) +
                " must be a cover");
      return false;
    }
  }
  for (int a = 0; a < na; ++a) {
    uint64_t want = 0;
    for (int v : q.atom_vars[a]) want |= 1ull << v;
    if (!appears[a] || got[a] != want) {
      set_error("invalid plan: the subatoms of atom " + std::to_string(a) +
                " do not partition its variables (Def. 3.5)");
      return false;
    }
  }
  return true;
}

PPlan binary2fj(const PQuery& q, const std::vector<int>& order) {
  PPlan plan;
  int r = order[0];
  PNode phi{PSub{r, q.atom_vars[r]}};  // iterate over the left relation
  uint64_t bound = 0;
  for (int v : q.atom_vars[r]) bound |= 1ull << v;
  for (size_t i = 1; i < order.size(); ++i) {
    int s = order[i];
    PSub probe{s, {}}, rest{s, {}};
    for (int v : q.atom_vars[s]) (bound >> v & 1 ? probe : rest).vars.push_back(v);
    phi.push_back(probe);  // probe with the available variables
    plan.push_back(phi);
    phi = PNode{rest};     // iterate over the probe result
    for (int v : q.atom_vars[s]) bound |= 1ull << v;
  }
  plan.push_back(phi);
  return plan;
}

PPlan factor(const PPlan& in) {
  PPlan plan = in;
  int n = int(plan.size());
  for (int i = n - 1; i >= 1; --i) {
    uint64_t avail = avs_mask(plan, i);
    PNode& phi = plan[i];
    PNode& prev = plan[i - 1];
    while (phi.size() > 1) {
      const PSub alpha = phi[1];
      uint64_t m = 0;
      for (int v : alpha.vars) m |= 1ull << v;
      bool in_prev = false;
      for (const PSub& p : prev) in_prev |= p.atom == alpha.atom;
      if ((m & ~avail) == 0 && !in_prev) {
        phi.erase(phi.begin() + 1);
        prev.push_back(alpha);
      } else {
        break;  // conservative: keep the optimizer's lookup order
      }
    }
  }
  return plan;
}

PPlan generic_join(const PQuery& q, const std::vector<int>& var_order) {
  PPlan plan;
  for (int x : var_order) {
    PNode node;
    for (int a = 0; a < int(q.atom_vars.size()); ++a)
      for (int v : q.atom_vars[a])
        if (v == x) node.push_back(PSub{a, {x}});
    plan.push_back(node);
  }
  return plan;
}

std::vector<std::vector<int>> ght_schema(const PPlan& plan, int atom) {
  std::vector<std::vector<int>> levels;
  bool last_is_cover = false;
  for (const PNode& node : plan)
    for (size_t s = 0; s < node.size(); ++s)
      if (node[s].atom == atom) {
        levels.push_back(node[s].vars);
        last_is_cover = s == 0;
      }
  if (!last_is_cover) levels.push_back({});
  return levels;
}

namespace {
struct PlanStore {
  fj_plan plan;  // first member: fj_plan* <-> PlanStore*
  std::vector<fj_node> nodes;
  std::vector<std::vector<fj_subatom>> subs;
  std::vector<std::vector<std::vector<int>>> vars;
};
}  // namespace

fj_plan* export_plan(const PPlan& p) {
  auto* st = new PlanStore();
  st->subs.resize(p.size());
  st->vars.resize(p.size());
  for (size_t k = 0; k < p.size(); ++k) {
    st->vars[k].resize(p[k].size());
    for (size_t s = 0; s < p[k].size(); ++s) st->vars[k][s] = p[k][s].vars;
  }
  for (size_t k = 0; k < p.size(); ++k) {
    for (size_t s = 0; s < p[k].size(); ++s)
      st->subs[k].push_back(fj_subatom{p[k][s].atom, int(st->vars[k][s].size()),
                                       st->vars[k][s].empty() ? nullptr : st->vars[k][s].data()});
    st->nodes.push_back(fj_node{int(st->subs[k].size()), st->subs[k].data()});
  }
  st->plan.n_nodes = int(st->nodes.size());
  st->plan.nodes = st->nodes.data();
  return &st->plan;
}

}  // namespace fj

using namespace fj;

extern "C" {

const char* fj_last_error(void) { return get_error(); }

fj_status fj_validate_plan(const fj_query* query, const fj_plan* plan) {
  PQuery q;
  PPlan p;
  if (!load_query(query, q)) return FJ_ERR_INVALID_ARG;
  if (!load_plan(q, plan, p)) return FJ_ERR_INVALID_PLAN;
  if (!validate(q, p)) return FJ_ERR_INVALID_PLAN;
  set_error("");
  return FJ_OK;
}

fj_status fj_binary_to_free_plan(const fj_query* query, const int* order, int n, int apply_factor,
                                 fj_plan** out) {
  if (!out) {
    set_error("fj_binary_to_free_plan: out is NULL");
    return FJ_ERR_INVALID_ARG;
  }
  *out = nullptr;
  PQuery q;
  if (!load_query(query, q)) return FJ_ERR_INVALID_ARG;
  if (!order || n != int(q.atom_vars.size())) {
    set_error("fj_binary_to_free_plan: order must list every atom once");
    return FJ_ERR_INVALID_ARG;
  }
  std::vector<int> ord(order, order + n), chk(ord);
  std::sort(chk.begin(), chk.end());
  for (int i = 0; i < n; ++i)
    if (chk[i] != i) {
      set_error("fj_binary_to_free_plan: order must be a permutation of the atoms");
      return FJ_ERR_INVALID_ARG;
    }
  PPlan p = binary2fj(q, ord);
  if (apply_factor) p = factor(p);
  if (int(p.size()) > FJ_MAX_NODES) {
    set_error("fj_binary_to_free_plan: plan exceeds FJ_MAX_NODES");
    return FJ_ERR_UNSUPPORTED;
  }
  *out = export_plan(p);
  set_error("");
  return FJ_OK;
}

fj_status fj_generic_join_plan(const fj_query* query, const int* var_order, int n,
                               fj_plan** out) {
  if (!out) {
    set_error("fj_generic_join_plan: out is NULL");
    return FJ_ERR_INVALID_ARG;
  }
  *out = nullptr;
  PQuery q;
  if (!load_query(query, q)) return FJ_ERR_INVALID_ARG;
  uint64_t all = 0, seen = 0;
  for (const auto& vs : q.atom_vars)
    for (int v : vs) all |= 1ull << v;
  if (!var_order || n != __builtin_popcountll(all)) {
    set_error("fj_generic_join_plan: the order must list every variable once");
    return FJ_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n; ++i) {
    const int v = var_order[i];
    if (v < 0 || v >= FJ_MAX_VARS || !(all >> v & 1) || (seen >> v & 1)) {
      set_error("fj_generic_join_plan: the order must list every variable once");
      return FJ_ERR_INVALID_ARG;
    }
    seen |= 1ull << v;
  }
  if (n > FJ_MAX_NODES) {
    set_error("fj_generic_join_plan: more variables than FJ_MAX_NODES");
    return FJ_ERR_UNSUPPORTED;
  }
  *out = export_plan(generic_join(q, std::vector<int>(var_order, var_order + n)));
  set_error("");
  return FJ_OK;
}

void fj_plan_free(fj_plan* plan) { delete reinterpret_cast<PlanStore*>(plan); }

fj_status fj_ght_schema(const fj_query* query, const fj_plan* plan, int atom, int* n_levels,
                        int* level_sizes, int* vars_out) {
  PQuery q;
  PPlan p;
  if (!load_query(query, q)) return FJ_ERR_INVALID_ARG;
  if (!load_plan(q, plan, p)) return FJ_ERR_INVALID_PLAN;
  if (atom < 0 || atom >= int(q.atom_vars.size()) || !n_levels || !level_sizes || !vars_out) {
    set_error("fj_ght_schema: bad argument");
    return FJ_ERR_INVALID_ARG;
  }
  auto levels = ght_schema(p, atom);
  *n_levels = int(levels.size());
  int w = 0;
  for (size_t l = 0; l < levels.size(); ++l) {
    level_sizes[l] = int(levels[l].size());
    for (int v : levels[l]) vars_out[w++] = v;
  }
  set_error("");
  return FJ_OK;
}

fj_status fj_node_covers(const fj_query* query, const fj_plan* plan, int k, int* n_covers,
                         int* covers_out) {
  PQuery q;
  PPlan p;
  if (!load_query(query, q)) return FJ_ERR_INVALID_ARG;
  if (!load_plan(q, plan, p)) return FJ_ERR_INVALID_PLAN;
  if (k < 0 || k >= int(p.size()) || !n_covers || !covers_out) {
    set_error("fj_node_covers: bad argument");
    return FJ_ERR_INVALID_ARG;
  }
  auto c = covers(p, k);
  *n_covers = int(c.size());
  for (size_t i = 0; i < c.size(); ++i) covers_out[i] = c[i];
  set_error("");
  return FJ_OK;
}

}  // extern "C"
