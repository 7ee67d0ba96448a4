// Host-side Free Join plan logic (paper Section 3.2 and Section 4.1).
#pragma once

#include <string>
#include <vector>

#include "../../include/fj.h"

namespace fj {

// A subatom with its variables in the atom's column order.
struct PSub {
  int atom;
  std::vector<int> vars;
};
using PNode = std::vector<PSub>;
using PPlan = std::vector<PNode>;

struct PQuery {
  std::vector<std::vector<int>> atom_vars;  // per atom, in column order
  std::vector<int> head;                    // output variable order
};

// Thread-local error message shared by every entry point.
void set_error(const std::string& msg);
const char* get_error();

bool load_query(const fj_query* q, PQuery& out);
bool load_plan(const PQuery& q, const fj_plan* p, PPlan& out);

uint64_t vs_mask(const PNode& node);
uint64_t avs_mask(const PPlan& plan, int k);
std::vector<int> covers(const PPlan& plan, int k);

// Def. 3.5 / Def. 3.7, plus: sub[0] of every node is a cover.
bool validate(const PQuery& q, const PPlan& plan);

PPlan binary2fj(const PQuery& q, const std::vector<int>& order);
PPlan factor(const PPlan& plan);
// The Generic Join plan of a total variable order (Section 3.2, Eq. 3).
PPlan generic_join(const PQuery& q, const std::vector<int>& var_order);

// GHT schema of one atom (Section 3.3): levels and whether the trailing
// empty level is present.
std::vector<std::vector<int>> ght_schema(const PPlan& plan, int atom);

fj_plan* export_plan(const PPlan& plan);

}  // namespace fj

// The cover policy (FJ_COVER_STATIC or FJ_COVER_FEWEST) the chooser's
// network predicts cheaper for `plan` (fj_chooser.cu); the reason of a
// failure in fj_internal_chooser_error().
fj_status fj_internal_learned_policy(fj_ctx* ctx, const fj_query* query, const fj::PPlan& plan,
                                     const fj_model* model, int* policy);
const char* fj_internal_chooser_error();
