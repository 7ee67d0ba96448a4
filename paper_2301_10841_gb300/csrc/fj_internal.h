// Internal device-side structures of libfj (shared by the host driver and the
// kernels).  Not part of the public ABI.
//
// COLT layout in HBM (paper Section 4.2, Def. 4.2 and Fig. 12).  For every
// atom the library keeps one array of row offsets `perm` and a stack of levels
// L[0..n_levels).  L[0] is a virtual level with a single entry standing for
// the whole relation; L[i] (i >= 1) holds the hash-map nodes of schema level
// i-1.  An entry e of L[i] is one key of one map node: it owns the contiguous
// offsets perm[begin[e] .. begin[e]+count[e]) -- the COLT child vector -- and,
// once that vector is forced into a map of L[i+1], the contiguous entries
// child_first[e] .. child_first[e]+child_nkeys[e].  Forcing regroups the
// parent's offsets in place, so a child vector is always a sub-range of its
// parent's range.  A level's hash table maps the pair (parent entry, key
// tuple) to the entry, so all map nodes of one level share one table.
#pragma once

#include <cstdint>

#include "../../include/fj.h"

namespace fj {

constexpr int kMaxLevels = FJ_MAX_NODES + 1;  // virtual root + schema levels
constexpr uint64_t kEmptyKey = ~0ull;
constexpr uint32_t kNone = 0xffffffffu;

// Child-state of an entry: has its child vector been turned into a map?
constexpr uint32_t kUnforced = 0;
constexpr uint32_t kRequested = 1;
constexpr uint32_t kForced = 2;

// Status bits set on the device.
constexpr uint32_t kStOutputOverflow = 1u << 0;
constexpr uint32_t kStCountOverflow = 1u << 1;
constexpr uint32_t kStTableFull = 1u << 2;
constexpr uint32_t kStItemsOverflow = 1u << 3;
constexpr uint32_t kStTimeout = 1u << 4;
constexpr uint32_t kStDrainTimeout = 1u << 5;  // after a timeout, copies in flight did not land

// States of a level's hash table between executions (LevelDev::ht_state).
constexpr uint32_t kHtListed = 1;
constexpr uint32_t kHtUnknown = 2;

struct LevelDev {
  // Entries of this level.
  uint32_t* begin = nullptr;
  uint32_t* count = nullptr;
  uint32_t* fill = nullptr;
  uint64_t* key = nullptr;
  uint32_t* child_state = nullptr;
  uint32_t* child_first = nullptr;
  uint32_t* child_nkeys = nullptr;
  uint32_t entries_cap = 0;
  // Hash table (level >= 1): (cap + 1) 16-byte slots {key lo, key hi, entry,
  // count}; slot `cap` is reserved for the one key equal to kEmptyKey.
  uint4* ht = nullptr;
  uint32_t ht_cap_max = 0;
  // Root levels: per slot, the first offset of its entry's range (written
  // by the root build, read by its scatter).
  uint32_t* sbegin = nullptr;
  // Root levels: per entry, its slot.  The root build leaves its table
  // dirty and lists the slots it used here, so that the next build clears
  // only those instead of the whole table (ht_state below).
  uint32_t* slot_of = nullptr;
  // Root levels whose entries' vectors a plan folds into COUNT/MIN as a
  // trailing node (a tail): per entry, the MIN of column `tmin_col` over the
  // entry's vector, computed by the root build (a partial aggregate of the
  // vector, so the aggregate epilogue reads one word instead of walking it).
  int32_t* tmin = nullptr;
  int tmin_col = -1;
  // Key columns: indices into AtomDev::cols (0 to 3 of them).
  int nk = 0;
  int kcol[3] = {0, 0, 0};
  // Blocked Bloom filter over this level's keys (narrow levels): one 32-bit
  // word per key hash, two bits set.  Probes test it before touching the
  // table; it is switched off on the device when the level holds too many
  // keys for its size.
  uint32_t* filter = nullptr;
  uint32_t filter_words = 0;  // power of two
  // Root levels keyed by one column: one bit per key value in
  // [0, 32 filter_words), set by the root build next to the Bloom filter.
  // When every key falls in that range (`exact`, set by the build) the
  // bitmap answers membership exactly: the node-0 scan then needs no hash
  // lookup for the rows it keeps and fetches their entries only for the
  // final survivors.
  uint32_t* bitmap = nullptr;
  // Wide levels (more than one key value below the root, or three values)
  // use 32-byte slots {parent, k0, k1, k2 | entry, count, -, -} claimed with
  // a 16-byte compare-and-swap; their entries keep only the parent in key[]
  // and read key values from a representative row.
  int wide = 0;
  // Forcing work list: parents of L[i-1] whose child vectors must become
  // maps of this level, and their row-offset prefix sums.
  uint32_t* req = nullptr;
  uint32_t* rowoff = nullptr;  // n_req + 1 entries
  uint32_t req_cap = 0;
  // Device-side counters (written by kernels).
  uint32_t mask;       // ht capacity - 1 once cleared
  uint32_t cleared;    // table cleared for this execution
  uint32_t n_entries;  // entries created so far
  uint32_t n_req;      // parents requested in the current force
  uint32_t n_new;      // entries created by the current force
  uint32_t n_rows;     // offsets regrouped by the current force
  uint32_t base;       // first entry id of the current force
  uint32_t pos_total;  // offsets placed by the current force
  uint32_t n_in;       // rows that reach this level's table (sizing)
  uint32_t filter_on;  // the filter is built and selective
  uint32_t exact;      // the bitmap holds every key of the level
  uint32_t n_tmp;      // (row, slot) pairs staged by the current force
  // State of the table between executions (kept across resets):
  // kHtListed: empty except the slots slot_of[0, n_listed) (and, for a
  // tail level, sbegin is INT32_MAX except there); kHtUnknown: any slot may
  // be dirty.
  uint32_t ht_state = kHtUnknown;
  uint32_t n_listed = 0;
};

struct AtomDev {
  const int32_t* cols[FJ_MAX_ARITY];  // column of the atom's j-th variable
  uint32_t n_rows;
  int n_vars;
  int n_preds;
  int pred_col[FJ_MAX_PREDS];
  int pred_op[FJ_MAX_PREDS];
  int32_t pred_val[FJ_MAX_PREDS];
  uint32_t* perm;      // row offsets, grouped level by level
  uint32_t* tmp_row;   // per forced row: its offset
  uint32_t* tmp_slot;  // per forced row: its hash slot
  uint32_t* newslots;  // slots claimed by the current force
  uint32_t root_mat;   // perm[0..n_pass) holds the passing rows
  uint32_t n_pass;
  float load;
  int n_levels;
  LevelDev L[kMaxLevels];
};

// One subatom of a node, as the expansion kernel sees it.
struct SubDev {
  int atom;
  int lvl;        // level index of the parent handle; entries live in L[lvl+1]
  int last;       // this subatom is its atom's last schema level
  int nv;
  int var[FJ_MAX_ARITY];
  int col[FJ_MAX_ARITY];  // index into AtomDev::cols per variable
  int hslot;      // input handle array of this atom (-1: root, handle 0)
  int is_cover;   // cover candidate of its node
  uint32_t bound_mask;  // bit j: var[j] was bound by an earlier node; when
                        // this subatom is iterated as the cover its elements
                        // must agree with those values
};

// A tail node: a single-subatom node that iterates the last level of its
// atom after the last expanded node.  In aggregate modes it contributes the
// length of its vector as a product factor and the MIN of its variables.
struct TailDev {
  int atom;
  int lvl;   // the vector is the range of the handle's entry in L[lvl]
  int hsrc;  // >= 0: the new handle of that subatom; -1: the input handle
  int n_min;
  int min_idx[FJ_MAX_ARITY];  // index into the result MIN array
  int min_col[FJ_MAX_ARITY];  // column index into AtomDev::cols
  const int32_t* tmin;        // per-entry MIN of min_col[0] (n_min == 1), or null
};

// Where one variable's value comes from for a batch element of a node whose
// cover is fixed (static): the input tuples (by item), a base-table column
// of the cover (by row), or the cover's map key (by entry).
constexpr int kSrcItem = 0;
constexpr int kSrcRow = 1;
constexpr int kSrcKey = 2;      // narrow map level: unpack key[entry]
constexpr int kSrcKeyWide = 3;  // wide map level: column at perm[begin[entry]]
struct VarSrc {
  int kind;
  int pos;                  // position in the key (kSrcKey)
  int nk;                   // key arity (kSrcKey)
  const int32_t* col;       // kSrcItem: input array; kSrcRow/kSrcKeyWide: column
  const uint64_t* key;      // kSrcKey
  const uint32_t* perm;     // kSrcKeyWide
  const uint32_t* begin;    // kSrcKeyWide
};

// One probe phase of a static-cover node, resolved on the host.
struct ProbeDev {
  int sub;                  // subatom index in the node
  int nv;
  int var[3];
  const uint4* ht;
  const uint32_t* mask;     // device-side table mask (read once per block)
  const uint32_t* filter;   // Bloom filter words (null: none)
  uint32_t filter_words;
  const uint32_t* filter_on;  // device-side switch (read once per block)
  int nk;
  int wide;
  int last;                 // ends its atom: multiply by the vector length
  const uint32_t* hsrc;     // parent handles by item (null: the root)
};

constexpr int kModeItems = 0;
constexpr int kModeAggregate = 1;
constexpr int kModeMaterialize = 2;
constexpr int kModeFactorized = 3;

struct NodeDev {
  int n_sub;
  int dynamic;
  int tile;                               // cover elements per batch
  SubDev sub[FJ_MAX_SUB];
  int8_t vpos[FJ_MAX_SUB][FJ_MAX_VARS];   // position of a variable in sub s
  uint32_t avs_mask;                      // bit v: variable v bound before
  // Static-cover fast path (dynamic == 0): resolved sources and probes.
  VarSrc src[FJ_MAX_VARS];
  int n_probe;
  ProbeDev probe[FJ_MAX_SUB];
  const uint32_t* cover_root_mat;         // &atoms[cover].root_mat
  const uint32_t* cover_perm;
  const uint32_t* cover_begin;            // L[lvl].begin of the cover
  const uint32_t* cover_first;            // L[lvl].child_first of the cover
  const uint32_t* cover_hsrc;             // cover parent handles by item
  // Input partial tuples (structure of arrays).
  const int32_t* in_var[FJ_MAX_VARS];     // by variable id
  const uint32_t* in_h[FJ_MAX_ATOMS];     // by atom
  const uint64_t* in_mult;                // null: all 1
  uint8_t* choice;                        // cover choice per item
  const uint32_t* n_items;                // device count of input items
  uint32_t single_item;                   // the input is the one root item
  uint64_t* fan;                          // per item fanout
  uint64_t* scan;                         // exclusive fanout prefix (n+1)
  uint64_t* total;                        // scan[n] copy for the host
  uint64_t chunk_begin;
  uint64_t chunk_end;
  int check_total;                        // the host did not read the node's total:
                                          // a total above chunk_end is an overflow
  int mode;
  int track_mult;                         // some probe ends an atom at a leaf
  // kModeItems.
  int n_out_vars;
  int out_var_id[FJ_MAX_VARS];
  int32_t* out_var[FJ_MAX_VARS];
  uint32_t* out_h[FJ_MAX_ATOMS];          // by atom; null: not carried
  int out_h_src[FJ_MAX_ATOMS];            // >= 0: sub index; -1: pass input
  uint64_t* out_mult;
  uint32_t* out_n;
  uint32_t out_cap;
  // kModeAggregate.
  int n_tail;
  TailDev tail[FJ_MAX_NODES];
  int n_min;
  int min_var[FJ_MAX_VARS];
  int min_idx[FJ_MAX_VARS];
  // kModeMaterialize (and kModeFactorized: out_tuples, out_rows_cap).
  int n_head;
  int head_var[FJ_MAX_VARS];
  int32_t* out_tuples;
  uint64_t out_rows_cap;
  // kModeFactorized: one row per surviving partial tuple of the last
  // expanded node -- its head variables bound so far (n_pre, in head
  // order), its multiplicity (two words, low first), and per tail the
  // (first offset, length) of the vector the tail iterates; row width
  // n_pre + 2 + 2 n_tail.
  int n_pre;
  int pre_var[FJ_MAX_VARS];
};

struct ResultDev {
  unsigned long long count;
  int32_t mins[FJ_MAX_VARS];
  unsigned long long n_out;
  uint32_t status;
  uint32_t pad;
  unsigned long long ctr[16];
};

}  // namespace fj
