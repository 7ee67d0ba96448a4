// Device kernels of libfj.
//
//  * COLT forcing (paper Section 4.2, Fig. 12 `force`): turn the child
//    vectors of a list of parent entries into hash-map nodes of the next
//    level, regrouping their offsets in place.  The root level is the same
//    operation on the single virtual root entry, with the atom's pushed-down
//    selections (Section 2.1) applied while scanning the base table.
//  * Node expansion (Section 3.3 Fig. 7 with the batching of Section 4.3
//    Fig. 13): iterate a batch of cover elements, probe every other subatom
//    for the whole batch, drop misses, and hand the survivors to the next
//    node, or aggregate / materialize them at the end of the plan.
//  * Cover choice (Section 4.4): per partial tuple, the cover whose trie has
//    the fewest keys; an unforced COLT vector is estimated by its length.
//
// Hashing uses the 64-bit finalizer of MurmurHash3 (Austin Appleby, public
// domain) on a packed 64-bit key word (parent entry, key values).
#pragma once

#include <cstdint>

#include "fj_internal.h"

namespace fj {

constexpr int kThreads = 256;

__device__ __forceinline__ uint64_t mix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

// 32-bit finalizer of MurmurHash3 (Austin Appleby, public domain).
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// Hash of a narrow key word (parent entry in the high half).
__device__ __forceinline__ uint32_t hash_key(uint64_t kw) {
  return fmix32(uint32_t(kw) ^ fmix32(uint32_t(kw >> 32) + 0x9e3779b9u));
}

// Blocked Bloom filter hash of a narrow key word: the high half of a
// multiplicative (Fibonacci) hash of both halves of the word, so a key of
// the root (parent 0) costs one wide multiply.  Independent of hash_key,
// which places keys in the table.
constexpr uint64_t kFibLo = 0x9e3779b97f4a7c15ull;  // 2^64 / golden ratio
constexpr uint64_t kFibHi = 0xc2b2ae3d27d4eb4full;
__device__ __forceinline__ uint32_t filter_hash(uint64_t kw) {
  return uint32_t((uint64_t(uint32_t(kw)) * kFibLo + uint64_t(uint32_t(kw >> 32)) * kFibHi) >>
                  32);
}
__device__ __forceinline__ uint32_t filter_hash_root1(int32_t k) {
  return uint32_t((uint64_t(uint32_t(k)) * kFibLo) >> 32);
}

// Filter word: (fh mod words); two bits from the top ten bits of fh.
__device__ __forceinline__ uint32_t bloom_bits(uint32_t fh) {
  return (1u << (fh >> 27)) | (1u << ((fh >> 22) & 31u));
}

// True when the filter rules the key out (no false negatives).
__device__ __forceinline__ bool bloom_rejects(const uint32_t* __restrict__ f, uint32_t words,
                                              uint32_t fh) {
  uint32_t m = bloom_bits(fh);
  return (__ldg(&f[fh & (words - 1)]) & m) != m;
}

// Key word of (parent, key tuple).  One level's keys all have the same arity:
// 0 or 1 values are packed beside the parent; 2 values fill the word and are
// only used where the parent is the single root entry.
__device__ __forceinline__ uint64_t pack_key(uint32_t parent, int nk, int32_t v0, int32_t v1) {
  if (nk == 2) return (uint64_t(uint32_t(v0)) << 32) | uint32_t(v1);
  uint64_t w = uint64_t(parent) << 32;
  if (nk == 1) w |= uint32_t(v0);
  return w;
}

__device__ __forceinline__ uint32_t key_parent(uint64_t kw, int nk) {
  return nk == 2 ? 0u : uint32_t(kw >> 32);
}

__device__ __forceinline__ int32_t key_value(uint64_t kw, int nk, int pos) {
  if (nk == 2) return pos == 0 ? int32_t(uint32_t(kw >> 32)) : int32_t(uint32_t(kw));
  return int32_t(uint32_t(kw));
}

__device__ __forceinline__ bool row_passes(const AtomDev& a, uint32_t row) {
  for (int p = 0; p < a.n_preds; ++p) {
    int32_t v = a.cols[a.pred_col[p]][row];
    int32_t c = a.pred_val[p];
    bool ok;
    switch (a.pred_op[p]) {
      case FJ_LT: ok = v < c; break;
      case FJ_LE: ok = v <= c; break;
      case FJ_GT: ok = v > c; break;
      case FJ_GE: ok = v >= c; break;
      case FJ_EQ: ok = v == c; break;
      default: ok = v != c; break;
    }
    if (!ok) return false;
  }
  return true;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ uint32_t lanemask_lt() {
  return (1u << lane_id()) - 1u;
}

// Hash-table slot access.  A slot is {key lo, key hi, entry, count}.
__device__ __forceinline__ unsigned long long* slot_key(uint4* ht, uint32_t s) {
  return reinterpret_cast<unsigned long long*>(&ht[s]);
}

// Insert kw; returns the slot and whether this thread claimed it.  Linear
// probing bounded by the capacity (a full table sets kStTableFull).
__device__ __forceinline__ uint32_t ht_insert(uint4* ht, uint32_t mask, uint64_t kw, bool& claimed,
                                              uint32_t* status) {
  claimed = false;
  if (kw == kEmptyKey) {
    uint32_t s = mask + 1;
    claimed = atomicCAS(&ht[s].z, kNone, 0u) == kNone;
    return s;
  }
  uint32_t h = hash_key(kw) & mask;
  for (uint32_t it = 0; it <= mask; ++it) {
    unsigned long long* kp = slot_key(ht, h);
    unsigned long long cur = *reinterpret_cast<volatile unsigned long long*>(kp);
    if (cur == kw) return h;
    if (cur == kEmptyKey) {
      unsigned long long old = atomicCAS(kp, kEmptyKey, kw);
      if (old == kEmptyKey) {
        claimed = true;
        return h;
      }
      if (old == kw) return h;
    }
    h = (h + 1) & mask;
  }
  atomicOr(status, kStTableFull);
  return kNone;
}

// Read-only lookup: returns the slot contents' entry and count, or false.
__device__ __forceinline__ bool ht_find(const uint4* __restrict__ ht, uint32_t mask, uint64_t kw,
                                        uint32_t& e, uint32_t& cnt) {
  if (kw == kEmptyKey) {
    uint4 s = ht[mask + 1];
    e = s.z;
    cnt = s.w;
    return s.w != 0;
  }
  uint32_t h = hash_key(kw) & mask;
  for (uint32_t it = 0; it <= mask; ++it) {
    uint4 s = __ldg(&ht[h]);
    uint64_t k = (uint64_t(s.y) << 32) | s.x;
    if (k == kw) {
      e = s.z;
      cnt = s.w;
      return true;
    }
    if (k == kEmptyKey) return false;
    h = (h + 1) & mask;
  }
  return false;
}

// Wide slots: slot s occupies ht[2s] (key: parent, k0, k1, k2) and ht[2s+1]
// (entry, count).  The parent word is below 2^32 - 1, so no real key equals
// the all-ones empty marker.
struct alignas(16) Key128 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ bool key128_eq(const uint4& a, const uint4& b) {
  return a.x == b.x && a.y == b.y && a.z == b.z && a.w == b.w;
}

__device__ __forceinline__ uint64_t mix128(const uint4& k) {
  return mix64((uint64_t(k.x) << 32 | k.y) ^ mix64(uint64_t(k.z) << 32 | k.w));
}

// Insert into a wide level.  Every probe of a slot is a 16-byte CAS, so a
// half-written key is never observed.
__device__ __forceinline__ uint32_t ht_insert_wide(uint4* ht, uint32_t mask, uint4 kw, bool& claimed,
                                                   uint32_t* status) {
  claimed = false;
  uint32_t h = uint32_t(mix128(kw)) & mask;
  const Key128 empty{kNone, kNone, kNone, kNone};
  const Key128 want{kw.x, kw.y, kw.z, kw.w};
  for (uint32_t it = 0; it <= mask; ++it) {
    Key128* kp = reinterpret_cast<Key128*>(&ht[2 * size_t(h)]);
    Key128 old = atomicCAS(kp, empty, want);
    if (old.x == kNone && old.y == kNone && old.z == kNone && old.w == kNone) {
      claimed = true;
      return h;
    }
    if (old.x == kw.x && old.y == kw.y && old.z == kw.z && old.w == kw.w) return h;
    h = (h + 1) & mask;
  }
  atomicOr(status, kStTableFull);
  return kNone;
}

__device__ __forceinline__ bool ht_find_wide(const uint4* __restrict__ ht, uint32_t mask, uint4 kw,
                                             uint32_t& e, uint32_t& cnt) {
  uint32_t h = uint32_t(mix128(kw)) & mask;
  for (uint32_t it = 0; it <= mask; ++it) {
    uint4 k = __ldg(&ht[2 * size_t(h)]);
    if (key128_eq(k, kw)) {
      uint4 v = __ldg(&ht[2 * size_t(h) + 1]);
      e = v.x;
      cnt = v.y;
      return true;
    }
    if (k.x == kNone && k.y == kNone && k.z == kNone && k.w == kNone) return false;
    h = (h + 1) & mask;
  }
  return false;
}

// Entry / count fields of slot s of a level.
__device__ __forceinline__ uint32_t* slot_e(uint4* ht, int wide, uint32_t s) {
  return wide ? &ht[2 * size_t(s) + 1].x : &ht[s].z;
}
__device__ __forceinline__ uint32_t* slot_cnt(uint4* ht, int wide, uint32_t s) {
  return wide ? &ht[2 * size_t(s) + 1].y : &ht[s].w;
}
// Empty a slot.
__device__ __forceinline__ void slot_clear(uint4* ht, int wide, uint32_t s) {
  if (wide) {
    ht[2 * size_t(s)] = make_uint4(kNone, kNone, kNone, kNone);
    ht[2 * size_t(s) + 1] = make_uint4(kNone, 0u, 0u, 0u);
  } else {
    ht[s] = make_uint4(0xffffffffu, 0xffffffffu, kNone, 0u);
  }
}

// ---------------------------------------------------------------------------
// Block-level helpers.
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane_id() >= uint32_t(o)) v += n;
  }
  return v;
}

// Exclusive block scan of one value per thread; returns the prefix and
// writes the block total to *total.  Uses `sh` (>= 33 elements).
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* sh, T* total) {
  T inc = warp_incl_scan(v);
  int w = threadIdx.x >> 5;
  if (lane_id() == 31) sh[w] = inc;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    T x = lane_id() < uint32_t(nw) ? sh[lane_id()] : T(0);
    T xi = warp_incl_scan(x);
    if (lane_id() < uint32_t(nw)) sh[lane_id()] = xi - x;
    if (lane_id() == uint32_t(nw - 1)) sh[32] = xi;
  }
  __syncthreads();
  T out = sh[w] + inc - v;
  *total = sh[32];
  __syncthreads();
  return out;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  T tot;
  block_excl_scan(v, sh, &tot);
  return tot;
}

// ---------------------------------------------------------------------------
// Device-wide exclusive scans (three passes, device-side lengths, one scan
// per blockIdx.y job).  The Op supplies n(job), load(job, i) and
// store(job, i, prefix) and receives the total.
// ---------------------------------------------------------------------------

constexpr int kScanBlocks = 608;  // 4 per SM

template <typename T, typename Op>
__global__ void __launch_bounds__(kThreads) k_scan_reduce(Op op, T* partials) {
  int job = blockIdx.y;
  uint64_t n = op.n(job);
  uint64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  uint64_t lo = chunk * blockIdx.x, hi = min(n, lo + chunk);
  T acc = 0;
  for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += op.load(job, i);
  __shared__ T sh[33];
  T tot = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[size_t(job) * kScanBlocks + blockIdx.x] = tot;
}

template <typename T, typename Op>
__global__ void __launch_bounds__(1024) k_scan_mid(Op op, T* partials, int nb) {
  int job = blockIdx.y;
  __shared__ T sh[33];
  T* p = partials + size_t(job) * kScanBlocks;
  T carry = 0;
  for (int base = 0; base < nb; base += blockDim.x) {
    int i = base + threadIdx.x;
    T v = i < nb ? p[i] : T(0);
    T tot;
    T ex = block_excl_scan(v, sh, &tot);
    if (i < nb) p[i] = ex + carry;
    carry += tot;
  }
  if (threadIdx.x == 0) op.total(job, carry);
}

template <typename T, typename Op>
__global__ void __launch_bounds__(kThreads) k_scan_down(Op op, const T* partials) {
  int job = blockIdx.y;
  uint64_t n = op.n(job);
  uint64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  uint64_t lo = chunk * blockIdx.x, hi = min(n, lo + chunk);
  __shared__ T sh[33];
  T carry = partials[size_t(job) * kScanBlocks + blockIdx.x];
  for (uint64_t base = lo; base < hi; base += blockDim.x) {
    uint64_t i = base + threadIdx.x;
    T v = i < hi ? op.load(job, i) : T(0);
    T tot;
    T ex = block_excl_scan(v, sh, &tot);
    if (i < hi) op.store(job, i, ex + carry);
    carry += tot;
  }
}

// ---------------------------------------------------------------------------
// COLT forcing.  A job is (atom, level i >= 1): build the map nodes of L[i]
// for the parents of L[i-1] listed in L[i].req.
// ---------------------------------------------------------------------------

struct ForceJobs {
  AtomDev* atoms;
  const int2* jobs;  // (atom, level)
  int n_jobs;
};

// Rows a job regroups: the root (level 1, relation not yet materialized)
// scans the whole base table; otherwise the parents' ranges of perm.
__device__ __forceinline__ bool job_identity(const AtomDev& a, int lvl) {
  return lvl == 1 && !a.root_mat;
}

// Pass 0a: rows that will be inserted (identity root jobs count the rows
// passing the selection; deeper levels use the root's passing-row count).
__global__ void __launch_bounds__(kThreads) k_force_count(ForceJobs fj) {
  int2 jb = fj.jobs[blockIdx.y];
  AtomDev& a = fj.atoms[jb.x];
  LevelDev& L = a.L[jb.y];
  if (L.n_req == 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // Per-force counters (the parent scans below overwrite n_rows for
    // non-root jobs).
    L.n_new = 0;
    L.n_tmp = 0;
    L.base = L.n_entries;
    if (job_identity(a, jb.y)) L.n_rows = a.n_rows;
  }
  // The requested parents' fill cursors start this force's bump allocation
  // of their children's ranges (the root build leaves them past the end).
  if (jb.y > 1) {
    LevelDev& P = a.L[jb.y - 1];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < L.n_req;
         i += gridDim.x * blockDim.x)
      P.fill[L.req[i]] = 0;
  }
  if (L.cleared) return;
  if (!job_identity(a, jb.y)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) L.n_in = a.n_pass;
    return;
  }
  if (a.n_preds == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) L.n_in = a.n_rows;
    return;
  }
  __shared__ uint32_t sh[33];
  uint32_t c = 0;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < a.n_rows; r += gridDim.x * blockDim.x)
    c += row_passes(a, r);
  uint32_t tot = block_sum(c, sh);
  if (threadIdx.x == 0 && tot) atomicAdd(&L.n_in, tot);
}

// Pass 0b: size the table of a level the first time it is forced.
__global__ void k_force_prepare(ForceJobs fj) {
  int2 jb = fj.jobs[blockIdx.x];
  AtomDev& a = fj.atoms[jb.x];
  LevelDev& L = a.L[jb.y];
  if (L.n_req == 0 || L.cleared || threadIdx.x != 0) return;
  float want = float(L.n_in) / (a.load > 0.f ? a.load : 0.5f);
  uint32_t cap = 16;
  while (float(cap) < want && cap < L.ht_cap_max) cap <<= 1;
  L.mask = cap - 1;
  // This build leaves no list of the slots it writes, and no bitmap.
  L.ht_state = kHtUnknown;
  L.exact = 0;
  // Keep the filter only with at least 4 bits per key.
  L.filter_on = L.filter && uint64_t(L.n_in) * 4 <= uint64_t(L.filter_words) * 32;
}

// Pass 1: clear a level's table the first time it is forced.
__global__ void k_force_clear(ForceJobs fj) {
  int2 jb = fj.jobs[blockIdx.y];
  AtomDev& a = fj.atoms[jb.x];
  LevelDev& L = a.L[jb.y];
  if (L.n_req == 0 || L.cleared) return;
  uint32_t n = L.mask + 2;
  if (L.filter_on)
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < L.filter_words;
         i += gridDim.x * blockDim.x)
      L.filter[i] = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (L.wide) {
      L.ht[2 * size_t(i)] = make_uint4(kNone, kNone, kNone, kNone);
      L.ht[2 * size_t(i) + 1] = make_uint4(kNone, 0u, 0u, 0u);
    } else {
      L.ht[i] = make_uint4(0xffffffffu, 0xffffffffu, kNone, 0u);
    }
  }
}

// Scan op: row offsets of the requested parents.
struct RowOffOp {
  AtomDev* atoms;
  const int2* jobs;
  __device__ uint64_t n(int job) const {
    int2 jb = jobs[job];
    return atoms[jb.x].L[jb.y].n_req;
  }
  __device__ uint32_t load(int job, uint64_t i) const {
    int2 jb = jobs[job];
    const AtomDev& a = atoms[jb.x];
    const LevelDev& L = a.L[jb.y];
    if (job_identity(a, jb.y)) return a.n_rows;
    return a.L[jb.y - 1].count[L.req[i]];
  }
  __device__ void store(int job, uint64_t i, uint32_t v) const {
    int2 jb = jobs[job];
    atoms[jb.x].L[jb.y].rowoff[i] = v;
  }
  __device__ void total(int job, uint32_t v) const {
    int2 jb = jobs[job];
    LevelDev& L = atoms[jb.x].L[jb.y];
    L.n_rows = v;
    L.rowoff[L.n_req] = v;
  }
};

__device__ __forceinline__ uint32_t upper_bound_u32(const uint32_t* a, uint32_t n, uint32_t x) {
  // first index i in [0, n) with a[i] > x
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Pass 2: insert every row's (parent, key) and count it.  Each block walks
// its rows 256 at a time; the counters every row group appends to (new
// slots, staged rows, and the root's key count) are summed per block in
// shared memory and advanced with one global atomic per counter.
__global__ void __launch_bounds__(kThreads) k_force_insert(ForceJobs fj, ResultDev* res) {
  int2 jb = fj.jobs[blockIdx.y];
  AtomDev& a = fj.atoms[jb.x];
  LevelDev& L = a.L[jb.y];
  LevelDev& P = a.L[jb.y - 1];
  uint32_t nreq = L.n_req;
  if (nreq == 0) return;
  const uint32_t n = L.n_rows;
  const bool ident = job_identity(a, jb.y);
  const uint32_t mask = L.mask;
  const int nk = L.nk;
  const int wide = L.wide;
  const bool fon = L.filter_on;
  const bool root = jb.y == 1;  // single parent: entry 0 of the virtual level
  const int32_t* c0 = a.cols[L.kcol[0]];
  const int32_t* c1 = a.cols[L.kcol[1]];
  const int32_t* c2 = a.cols[L.kcol[2]];
  __shared__ uint32_t s_cnt[3];   // claimed (new slots), staged rows, -
  __shared__ uint32_t s_base[3];
  const uint32_t warp = threadIdx.x >> 5;
  for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    uint32_t t = base + threadIdx.x;
    bool active = t < n;
    uint32_t row = 0, parent = 0, slot = kNone;
    bool claimed = false;
    if (active) {
      if (ident) {
        row = t;
        active = row_passes(a, row);
      } else {
        uint32_t pi = upper_bound_u32(L.rowoff, nreq, t) - 1;
        parent = L.req[pi];
        row = a.perm[P.begin[parent] + (t - L.rowoff[pi])];
      }
    }
    if (active) {
      if (wide) {
        uint4 kw = make_uint4(parent, nk > 0 ? uint32_t(c0[row]) : 0u,
                              nk > 1 ? uint32_t(c1[row]) : 0u, nk > 2 ? uint32_t(c2[row]) : 0u);
        slot = ht_insert_wide(L.ht, mask, kw, claimed, &res->status);
      } else {
        uint64_t kw = pack_key(parent, nk, nk > 0 ? c0[row] : 0, nk > 1 ? c1[row] : 0);
        slot = ht_insert(L.ht, mask, kw, claimed, &res->status);
        if (claimed && fon) {
          uint32_t fh = filter_hash(kw);
          atomicOr(&L.filter[fh & (L.filter_words - 1)], bloom_bits(fh));
        }
      }
      if (slot == kNone) active = false;
    }
    if (active) atomicAdd(slot_cnt(L.ht, wide, slot), 1u);
    // Per-warp ranks, per-block offsets.
    uint32_t cmask = __ballot_sync(0xffffffffu, claimed);
    uint32_t amask = __ballot_sync(0xffffffffu, active);
    uint32_t cw = 0, aw = 0;
    if (lane_id() == 0) {
      if (cmask) cw = atomicAdd(&s_cnt[0], __popc(cmask));
      if (amask) aw = atomicAdd(&s_cnt[1], __popc(amask));
    }
    cw = __shfl_sync(0xffffffffu, cw, 0);
    aw = __shfl_sync(0xffffffffu, aw, 0);
    __syncthreads();
    if (threadIdx.x == 0) {
      s_base[0] = s_cnt[0] ? atomicAdd(&L.n_new, s_cnt[0]) : 0u;
      s_base[1] = s_cnt[1] ? atomicAdd(&L.n_tmp, s_cnt[1]) : 0u;
      // Root: local key indices are the new-slot positions themselves.
      s_base[2] = (root && s_cnt[0]) ? atomicAdd(&P.child_nkeys[0], s_cnt[0]) : 0u;
    }
    __syncthreads();
    if (claimed) {
      uint32_t cpos = cw + __popc(cmask & lanemask_lt());
      a.newslots[s_base[0] + cpos] = slot;
      if (root) *slot_e(L.ht, wide, slot) = s_base[2] + cpos;
    }
    if (!root) {
      // Below the root: one local index per parent (grouped per warp).
      if (claimed) {
        uint32_t grp = __match_any_sync(cmask, parent);
        uint32_t leader = __ffs(grp) - 1;
        uint32_t first = 0;
        if (lane_id() == leader) first = atomicAdd(&P.child_nkeys[parent], __popc(grp));
        first = __shfl_sync(grp, first, leader);
        *slot_e(L.ht, wide, slot) = first + __popc(grp & lanemask_lt());
      }
    }
    if (active) {
      uint32_t o = s_base[1] + aw + __popc(amask & lanemask_lt());
      a.tmp_row[o] = row;
      a.tmp_slot[o] = slot;
    }
    (void)warp;
    __syncthreads();
  }
}

// Scan op: first child entry of each requested parent.
struct ChildFirstOp {
  AtomDev* atoms;
  const int2* jobs;
  __device__ uint64_t n(int job) const {
    int2 jb = jobs[job];
    return atoms[jb.x].L[jb.y].n_req;
  }
  __device__ uint32_t load(int job, uint64_t i) const {
    int2 jb = jobs[job];
    const AtomDev& a = atoms[jb.x];
    return a.L[jb.y - 1].child_nkeys[a.L[jb.y].req[i]];
  }
  __device__ void store(int job, uint64_t i, uint32_t v) const {
    int2 jb = jobs[job];
    AtomDev& a = atoms[jb.x];
    a.L[jb.y - 1].child_first[a.L[jb.y].req[i]] = a.L[jb.y].base + v;
  }
  __device__ void total(int job, uint32_t) const {}
};

// Pass 3: give each new slot its entry id, fill the entry arrays, and
// allocate the entry's vector inside its parent's range (the parent's fill
// cursor, zero at the start; one atomic per warp when the warp's entries
// share a parent, as at the root).
__global__ void __launch_bounds__(kThreads) k_force_assign(ForceJobs fj) {
  int2 jb = fj.jobs[blockIdx.y];
  AtomDev& a = fj.atoms[jb.x];
  LevelDev& L = a.L[jb.y];
  LevelDev& P = a.L[jb.y - 1];
  if (L.n_req == 0) return;
  uint32_t nnew = L.n_new;
  bool ident = jb.y == 1 && !a.root_mat;
  uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < nnew;
       base += stride) {
    uint32_t i = base + lane_id();
    bool active = i < nnew;
    uint32_t parent = 0, cnt = 0, e = 0;
    if (active) {
      uint32_t s = a.newslots[i];
      uint64_t kw;
      uint32_t local;
      if (L.wide) {
        uint4 k = L.ht[2 * size_t(s)];
        uint4 v = L.ht[2 * size_t(s) + 1];
        parent = k.x;
        kw = uint64_t(parent) << 32;  // wide entries keep only the parent
        local = v.x;
        cnt = v.y;
      } else {
        uint4 sl = L.ht[s];
        kw = s == L.mask + 1 ? kEmptyKey : ((uint64_t(sl.y) << 32) | sl.x);
        parent = key_parent(kw, L.nk);
        local = sl.z;
        cnt = sl.w;
      }
      e = P.child_first[parent] + local;
      *slot_e(L.ht, L.wide, s) = e;
      L.key[e] = kw;
      L.count[e] = cnt;
      if (L.child_state) L.child_state[e] = kUnforced;
      if (L.child_nkeys) L.child_nkeys[e] = 0;
      if (L.child_first) L.child_first[e] = 0;
    }
    uint32_t amask = __ballot_sync(0xffffffffu, active);
    if (!amask) continue;
    uint32_t lead = __ffs(amask) - 1;
    uint32_t p0 = __shfl_sync(0xffffffffu, parent, lead);
    uint32_t off;
    if (__all_sync(0xffffffffu, !active || parent == p0)) {
      uint32_t inc = warp_incl_scan(active ? cnt : 0u);
      uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
      uint32_t b = 0;
      if (lane_id() == lead) b = atomicAdd(&P.fill[p0], tot);
      b = __shfl_sync(0xffffffffu, b, lead);
      off = b + inc - (active ? cnt : 0u);
    } else {
      off = active ? atomicAdd(&P.fill[parent], cnt) : 0u;
    }
    if (active) {
      uint32_t pstart = ident ? 0u : P.begin[parent];
      L.begin[e] = pstart + off;
      L.fill[e] = pstart + off;  // scatter cursor
    }
  }
}

// Pass 5: move every staged row to its entry's range (fill[] is the cursor).
__global__ void __launch_bounds__(kThreads) k_force_scatter(ForceJobs fj) {
  int2 jb = fj.jobs[blockIdx.y];
  AtomDev& a = fj.atoms[jb.x];
  LevelDev& L = a.L[jb.y];
  if (L.n_req == 0) return;
  uint32_t n = L.n_tmp;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    uint32_t e = *slot_e(L.ht, L.wide, a.tmp_slot[t]);
    a.perm[atomicAdd(&L.fill[e], 1u)] = a.tmp_row[t];
  }
}

// Pass 6: bookkeeping.  begin[e] = cursor - count; requested parents are
// forced; the root range is now materialized (perm[0..n_pass) holds exactly
// the rows that pass the selection).
__global__ void __launch_bounds__(kThreads) k_force_finish(ForceJobs fj, ResultDev* res) {
  int2 jb = fj.jobs[blockIdx.y];
  AtomDev& a = fj.atoms[jb.x];
  LevelDev& L = a.L[jb.y];
  LevelDev& P = a.L[jb.y - 1];
  uint32_t nreq = L.n_req;
  if (nreq == 0) return;
  uint32_t nnew = L.n_new;
  uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (uint32_t i = tid; i < nnew; i += stride) L.fill[L.base + i] = 0;  // child cursor
  for (uint32_t i = tid; i < nreq; i += stride) P.child_state[L.req[i]] = kForced;
  if (tid == 0) {
    if (jb.y == 1) {
      a.n_pass = L.n_tmp;
      a.root_mat = 1;
      P.begin[0] = 0;
      P.count[0] = L.n_tmp;
      atomicAdd(&res->ctr[FJ_CTR_ROOTS_BUILT], 1ull);
      atomicOr(reinterpret_cast<unsigned long long*>(&res->ctr[FJ_CTR_ATOM_BUILT_MASK]),
               1ull << jb.x);
    } else {
      atomicAdd(&res->ctr[FJ_CTR_SUBTRIES_FORCED], (unsigned long long)nreq);
    }
    atomicAdd(&res->ctr[FJ_CTR_ROWS_REGROUPED], (unsigned long long)L.n_tmp);
    L.n_entries = L.base + nnew;
    L.cleared = 1;
  }
}

// The next force of this level starts with an empty request list.  Runs after
// k_force_finish (a separate launch so no block still reads n_req).
__global__ void k_force_reset_req(ForceJobs fj) {
  int2 jb = fj.jobs[blockIdx.x];
  if (threadIdx.x == 0) {
    fj.atoms[jb.x].L[jb.y].n_req = 0;
    fj.atoms[jb.x].L[jb.y].n_in = 0;
  }
}

// ---------------------------------------------------------------------------
// Root levels in one cooperative launch.  Forcing the root of an atom (its
// first schema level) reads the whole base table; for a node whose jobs are
// all roots, the passes of a force run in one kernel whose blocks are all
// resident (cudaLaunchCooperativeKernel), separated by grid barriers:
//   A  clear each Bloom filter, and each table's slots the previous build
//      listed (a table is cleared whole only when no build left a list),
//   C  select the rows, insert their keys, count rows per key, list the
//      slots, stage (row, slot, rank) per passing row,
//   D  make each listed slot an entry with its range of offsets; place the
//      row of every key that has one; record the level as forced,
//   E  (only when some key repeats) scatter the staged rows.
// A table spans its whole allocation, so C need not wait for the count of
// passing rows to size it.  Each pass splits the work of all jobs into one
// contiguous range per block and takes several independent elements per
// thread at a time (the passes are chains of dependent L2 accesses);
// offsets come from counters per job, advanced once per block sweep.
// Every barrier wait is bounded: on expiry the kernel sets kStTimeout and
// its blocks return; the host reports FJ_ERR_TIMEOUT.
// ---------------------------------------------------------------------------

constexpr int kRootThreads = 512;
constexpr int kRootRows = 12;  // rows per thread per sweep of C
// Dynamic shared memory of k_force_roots: per warp a queue of 32 x kRootRows
// (row, key then slot, rank) entries.
constexpr size_t kRootSmem = size_t(kRootThreads) * kRootRows * 3 * sizeof(uint32_t);

struct RootsState {        // zero at the start of each execution (k_reset)
  unsigned int bar_count;  // block arrivals at grid barriers this execution
  unsigned int bar_gen;    // unused (kept for the layout k_reset zeroes)
  // Per job: rows passing, keys; per launch: some key has more than one
  // row.  Launches alternate between the two sets; a launch zeroes the set
  // the next launch uses.
  unsigned int n_pass[2][FJ_MAX_ATOMS];
  unsigned int n_new[2][FJ_MAX_ATOMS];
  unsigned int dup[2];
  unsigned int oor[2][FJ_MAX_ATOMS];  // per job: some key outside the bitmap's range
};

constexpr uint32_t kGridSpinLimit = 1u << 22;  // polls of a grid barrier (about a second)

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier among all blocks of a cooperative launch.  The arrival
// counter only grows (k_reset zeroes it at the start of an execution): each
// block adds one with a release reduction, and waits, polling with acquire
// loads, until the count reaches `target` (the caller's count of arrivals
// at the end of this barrier) -- the releases and the acquire order the
// blocks' writes around the barrier, and nobody has to publish the barrier's
// end.  Returns false (in every thread of the block) when the wait ran out;
// `never` (the test of the bounded wait) makes the barrier wait for an
// arrival that never comes.
__device__ __forceinline__ bool grid_sync(RootsState* cs, uint32_t* status, uint32_t spin,
                                          uint32_t target, bool never = false) {
  const uint32_t limit = spin ? spin : kGridSpinLimit;
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&cs->bar_count) : "memory");
    const uint32_t want = never ? target + 1 : target;
    uint32_t it = 0;
    while (ld_acquire_gpu(&cs->bar_count) < want) {
      if (++it > limit) {
        atomicOr(status, kStTimeout);
        ok = 0;
        break;
      }
    }
  }
  return __syncthreads_and(ok);
}

// s_off[0..n] = prefix sums of size(j) over the jobs; all threads call it.
template <typename F>
__device__ __forceinline__ void jobs_prefix(int n, uint32_t* s_off, F size) {
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int j = 0; j < n; ++j) {
      s_off[j] = acc;
      acc += size(j);
    }
    s_off[n] = acc;
  }
  __syncthreads();
}

__device__ __forceinline__ int job_at(const uint32_t* s_off, int n, uint32_t x) {
  int j = 0;
  while (j + 1 < n && s_off[j + 1] <= x) ++j;
  return j;
}

// This block's contiguous part [lo, hi) of `total` elements.
__device__ __forceinline__ void block_range(uint32_t total, uint32_t& lo, uint32_t& hi) {
  lo = uint32_t(uint64_t(total) * blockIdx.x / gridDim.x);
  hi = uint32_t(uint64_t(total) * (blockIdx.x + 1) / gridDim.x);
}

// A root job's descriptors, copied once into shared memory so the passes
// do not chase the atom descriptors in global memory per element.
struct RootJob {
  uint4* ht;
  uint32_t* filter;
  uint32_t* bitmap;  // exact key bitmap (one-column narrow levels) or null
  uint32_t filter_words;
  uint32_t ht_cap_max;
  const int32_t* kc[3];
  int nk;
  int wide;
  int ident;     // rows are the base table's, filtered by the selection
  int act;       // the level is requested and not yet built
  uint32_t src;  // rows to read (base table, or perm[0, n_pass))
  uint32_t base_e;
  uint32_t* tmp_row;
  uint32_t* tmp_slot;
  uint32_t* newslots;  // the root build keeps each passing row's rank here
  uint32_t* sbegin;    // per slot: its entry's first offset
  uint32_t* slot_of;   // per entry: its slot (the list the next build clears)
  uint32_t state;      // the table's state when the launch began (LevelDev::ht_state)
  uint32_t n_listed;   // ... and its listed slots
  int32_t* tmin;       // per entry: MIN of tcol over its rows (or null)
  const int32_t* tcol;
  uint32_t* perm;
  uint64_t* key;
  uint32_t* count;
  uint32_t* begin;
  uint32_t* fill;
  uint32_t* cstate;
  uint32_t* cfirst;
  uint32_t* cnkeys;
  uint32_t* pfill;  // the root's fill cursor
  int n_preds;
  const int32_t* pcol[FJ_MAX_PREDS];
  int pop[FJ_MAX_PREDS];
  int32_t pval[FJ_MAX_PREDS];
};

__device__ __forceinline__ bool pred_holds(int op, int32_t v, int32_t c) {
  switch (op) {
    case FJ_LT: return v < c;
    case FJ_LE: return v <= c;
    case FJ_GT: return v > c;
    case FJ_GE: return v >= c;
    case FJ_EQ: return v == c;
    default: return v != c;
  }
}

// Pass bits of rows r0 + k * blockDim + tid (k < RPT, below r1) of a root
// job.
template <int RPT>
__device__ __forceinline__ uint32_t root_rows_pass(const RootJob& J, uint32_t r0, uint32_t r1,
                                                   uint32_t (&row)[RPT]) {
  uint32_t pass = 0;
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const uint32_t i = r0 + k * blockDim.x + threadIdx.x;
    row[k] = i;
    if (i < r1) {
      if (!J.ident) row[k] = J.perm[i];
      pass |= 1u << k;
    }
  }
  if (J.ident) {
    // One selection at a time, its column for all the rows at once.
    for (int p = 0; p < J.n_preds; ++p) {
      int32_t v[RPT];
#pragma unroll
      for (int k = 0; k < RPT; ++k) v[k] = (pass >> k & 1u) ? __ldg(J.pcol[p] + row[k]) : 0;
#pragma unroll
      for (int k = 0; k < RPT; ++k)
        if ((pass >> k & 1u) && !pred_holds(J.pop[p], v[k], J.pval[p])) pass &= ~(1u << k);
    }
  }
  return pass;
}

// Insert a narrow key: a compare-and-swap at its home slot `h` was
// answered with `old`; continue probing after it when the slot holds
// another key.
__device__ __forceinline__ uint32_t ht_insert_from(uint4* ht, uint32_t mask, uint64_t kw,
                                                   uint32_t h, unsigned long long old,
                                                   bool& claimed, uint32_t* status) {
  claimed = false;
  for (uint32_t it = 0; it <= mask; ++it) {
    if (old == kEmptyKey) {
      claimed = true;
      return h;
    }
    if (old == kw) return h;
    h = (h + 1) & mask;
    old = atomicCAS(slot_key(ht, h), kEmptyKey, kw);
  }
  atomicOr(status, kStTableFull);
  return kNone;
}

__global__ void __launch_bounds__(kRootThreads, 2) k_force_roots(ForceJobs fj, RootsState* cs,
                                                                 int set, int request_all,
                                                                 int test_timeout,
                                                                 ResultDev* res, uint32_t spin) {
  constexpr int E = 4;  // independent elements per thread in C's inserts, D and E
  constexpr uint32_t NT = kRootThreads, NW = NT / 32, QW = 32 * kRootRows;
  const int nj = fj.n_jobs;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  // Per warp, C's queue of the rows of a sweep that pass the selection:
  // QW rows, QW one-column keys (then the rows' slots), QW ranks.
  extern __shared__ __align__(16) uint32_t s_queue[];
  uint32_t* q_row = s_queue + size_t(warp) * 3 * QW;
  uint32_t* q_key = q_row + QW;
  uint32_t* q_slot = q_key;
  uint32_t* q_rank = q_key + QW;
  __shared__ RootJob s_job[FJ_MAX_ATOMS];
  __shared__ uint32_t s_off[FJ_MAX_ATOMS + 1];
  __shared__ uint32_t s_mask[FJ_MAX_ATOMS];
  __shared__ uint32_t s_np[FJ_MAX_ATOMS], s_nn[FJ_MAX_ATOMS];  // rows passing, keys
  __shared__ uint32_t s_wq[NW], s_wc[NW];  // per warp: queued rows, new keys
  __shared__ uint32_t s_scan[33];
  __shared__ uint32_t s_base2;
  // Arrivals at grid barriers before this launch (an execution may launch
  // the build more than once): whole barriers of the same grid -- a block of
  // this launch may already have arrived at the first one, so round down.
  // Only thread 0 takes part in the barriers.
  uint32_t bar_target = tid == 0 ? ld_acquire_gpu(&cs->bar_count) / gridDim.x * gridDim.x : 0u;
  if (tid < uint32_t(nj)) {
    const int2 jb = fj.jobs[tid];
    const AtomDev& a = fj.atoms[jb.x];
    const LevelDev& L = a.L[jb.y];
    const LevelDev& P = a.L[jb.y - 1];
    RootJob& J = s_job[tid];
    J.ht = L.ht;
    J.filter = L.filter;
    J.bitmap = L.bitmap;
    J.filter_words = L.filter_words;
    J.ht_cap_max = L.ht_cap_max;
    J.nk = L.nk;
    for (int k = 0; k < 3; ++k) J.kc[k] = a.cols[L.kcol[k]];
    J.wide = L.wide;
    J.ident = !a.root_mat;
    // request_all: node 0 of a single root tuple reaches every root of its
    // jobs (what k_choose would request); otherwise the requests decide.
    J.act = (request_all || L.n_req > 0) && !L.cleared;
    J.src = a.root_mat ? a.n_pass : a.n_rows;
    J.base_e = L.n_entries;
    J.tmp_row = a.tmp_row;
    J.tmp_slot = a.tmp_slot;
    J.newslots = a.newslots;
    J.sbegin = L.sbegin;
    J.slot_of = L.slot_of;
    J.state = L.ht_state;
    J.n_listed = L.n_listed;
    J.tmin = L.tmin;
    J.tcol = L.tmin ? a.cols[L.tmin_col] : nullptr;
    J.perm = a.perm;
    J.key = L.key;
    J.count = L.count;
    J.begin = L.begin;
    J.fill = L.fill;
    J.cstate = L.child_state;
    J.cfirst = L.child_first;
    J.cnkeys = L.child_nkeys;
    J.pfill = P.fill;
    J.n_preds = a.n_preds;
    for (int p = 0; p < a.n_preds; ++p) {
      J.pcol[p] = a.cols[a.pred_col[p]];
      J.pop[p] = a.pred_op[p];
      J.pval[p] = a.pred_val[p];
    }
    // The table spans its whole allocation (sized for every row of the
    // atom at its load factor): it is never cleared as a whole once built,
    // so a larger span costs nothing, and its size need not wait for the
    // count of passing rows.
    s_mask[tid] = L.ht_cap_max - 1;
  }
  if (blockIdx.x == 0 && tid < uint32_t(FJ_MAX_ATOMS)) {
    cs->n_pass[set ^ 1][tid] = 0;
    cs->n_new[set ^ 1][tid] = 0;
    cs->oor[set ^ 1][tid] = 0;
    if (tid == 0) cs->dup[set ^ 1] = 0;
  }
  __syncthreads();
  uint32_t lo, hi;

  // A: every active job's Bloom filter to zero; its table back to empty --
  // the slots its previous build listed (and a tail level's running MINs
  // there back to INT32_MAX), or, when no build left a list, every slot.
  jobs_prefix(nj, s_off, [&](int j) {
    const RootJob& J = s_job[j];
    return J.act && J.filter ? J.filter_words / 4 * (J.bitmap ? 2u : 1u) : 0u;
  });
  for (uint32_t x = blockIdx.x * NT + tid; x < s_off[nj]; x += gridDim.x * NT) {
    const int j = job_at(s_off, nj, x);
    const RootJob& J = s_job[j];
    const uint32_t u = x - s_off[j], fq = J.filter_words / 4;
    uint32_t* w = u < fq ? J.filter : J.bitmap;  // the filter's words, then the bitmap's
    reinterpret_cast<uint4*>(w)[u < fq ? u : u - fq] = make_uint4(0u, 0u, 0u, 0u);
  }
  // One contiguous part of the slots per block (equal parts), two per
  // thread at a time with their list loads in flight together.
  jobs_prefix(nj, s_off, [&](int j) {
    const RootJob& J = s_job[j];
    if (!J.act) return 0u;
    return J.state == kHtListed ? J.n_listed : J.ht_cap_max + 1;
  });
  block_range(s_off[nj], lo, hi);
  for (uint32_t x0 = lo + tid; x0 < hi; x0 += 2 * NT) {
    uint32_t sl[2];
    int jj[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint32_t x = x0 + u * NT;
      jj[u] = -1;
      if (x >= hi) continue;
      jj[u] = job_at(s_off, nj, x);
      const RootJob& J = s_job[jj[u]];
      sl[u] = J.state == kHtListed ? J.slot_of[x - s_off[jj[u]]] : x - s_off[jj[u]];
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (jj[u] < 0) continue;
      const RootJob& J = s_job[jj[u]];
      slot_clear(J.ht, J.wide, sl[u]);
      if (J.tmin) J.sbegin[sl[u]] = uint32_t(INT32_MAX);
    }
  }
  if (!grid_sync(cs, &res->status, spin, bar_target += gridDim.x, test_timeout != 0)) return;
  // From here on a failed launch leaves the tables in an unknown state; a
  // complete one lists the slots it used.
  if (blockIdx.x == 0 && tid < uint32_t(nj) && s_job[tid].act) {
    LevelDev& L = fj.atoms[fj.jobs[tid].x].L[fj.jobs[tid].y];
    L.mask = s_mask[tid];
    L.ht_state = kHtUnknown;
  }

  // C: per sweep, kRootRows rows per thread: the selection and key loads of
  // all of them in flight together, the passing rows into the warp's queue,
  // then the queue's keys inserted E per lane with their first
  // compare-and-swaps in flight together, each row counted in its key's
  // slot.  The count before a row's increment is its rank among the rows
  // of its key (its place in the entry's range); the rank-0 row leaves
  // itself in the slot (D places it when it is the key's only row, and a
  // tail level's MIN starts from its value; the other rows fold theirs into
  // the slot's running MIN) and puts the slot on the table's list, whose
  // order numbers the entries.  Per sweep one advance of the job's row and
  // key counters: the queues go to the staging arrays (for E) and the list
  // at those offsets.
  // The work split: when every active job's rows fit in whole sweeps of
  // the grid's blocks, each block takes at most one sweep of one job (no
  // block waits on two chains); otherwise one contiguous part of all rows
  // per block.
  constexpr uint32_t SW = kRootRows * NT;  // rows per block sweep
  jobs_prefix(nj, s_off, [&](int j) { return s_job[j].act ? (s_job[j].src + SW - 1) / SW : 0u; });
  const bool per_job = s_off[nj] <= gridDim.x;
  int jsel = -1;
  uint32_t jr0 = 0, jr1 = 0;
  if (per_job && blockIdx.x < s_off[nj]) {
    jsel = job_at(s_off, nj, blockIdx.x);
    jr0 = (blockIdx.x - s_off[jsel]) * SW;
    jr1 = min(s_job[jsel].src, jr0 + SW);
  }
  jobs_prefix(nj, s_off, [&](int j) { return s_job[j].act ? s_job[j].src : 0u; });
  block_range(s_off[nj], lo, hi);
  bool dup = false;  // some key of this block's rows has another row before it
  bool oor = false;  // some key of this block's sweep falls outside its job's bitmap
  for (int j = 0; j < nj; ++j) {
    uint32_t r0 = jr0, r1 = jr1;  // this block's rows of job j
    if (per_job) {
      if (j != jsel) continue;
    } else {
      const uint32_t a0 = max(lo, s_off[j]), a1 = min(hi, s_off[j + 1]);
      if (a0 >= a1) continue;
      r0 = a0 - s_off[j];
      r1 = a1 - s_off[j];
    }
    const RootJob& J = s_job[j];
    const bool k1 = !J.wide && J.nk == 1;
    const uint32_t mask = s_mask[j];
    for (uint32_t r = r0; r < r1; r += SW) {
      uint32_t qn;
      {
        uint32_t row[kRootRows];
        int32_t key[kRootRows];
        // Base-table rows: every key load goes out with the selection loads
        // (one round trip to memory instead of two).
        const bool early = k1 && J.ident;
#pragma unroll
        for (int k = 0; k < kRootRows; ++k) {
          const uint32_t i = r + k * NT + tid;
          key[k] = (early && i < r1) ? __ldg(J.kc[0] + i) : 0;
        }
        const uint32_t pass = root_rows_pass<kRootRows>(J, r, r1, row);
        if (k1 && !early) {
#pragma unroll
          for (int k = 0; k < kRootRows; ++k)
            key[k] = (pass >> k & 1u) ? __ldg(J.kc[0] + row[k]) : 0;
        }
        const uint32_t np = __popc(pass);
        const uint32_t incl = warp_incl_scan(np);
        qn = __shfl_sync(0xffffffffu, incl, 31);
        uint32_t qp = incl - np;
#pragma unroll
        for (int k = 0; k < kRootRows; ++k)
          if (pass >> k & 1u) {
            q_row[qp] = row[k];
            q_key[qp] = uint32_t(key[k]);
            ++qp;
          }
      }
      __syncwarp();
      uint32_t n_first = 0;  // this lane's rank-0 rows
      for (uint32_t i0 = 0; i0 < qn; i0 += E * 32) {
        uint32_t slot[E], rw[E];
#pragma unroll
        for (int u = 0; u < E; ++u) {
          const uint32_t i = i0 + u * 32 + lane;
          rw[u] = i < qn ? q_row[i] : 0u;
        }
        if (!J.wide) {
          uint64_t kw[E];
          uint32_t h[E];
          unsigned long long old[E];
#pragma unroll
          for (int u = 0; u < E; ++u) {
            const uint32_t i = i0 + u * 32 + lane;
            kw[u] = 0;
            if (i >= qn) continue;
            if (k1) {
              kw[u] = q_key[i];
            } else {
              const uint32_t row = rw[u];
              kw[u] = pack_key(0u, J.nk, J.nk > 0 ? __ldg(J.kc[0] + row) : 0,
                               J.nk > 1 ? __ldg(J.kc[1] + row) : 0);
            }
          }
#pragma unroll
          for (int u = 0; u < E; ++u) {
            const uint32_t i = i0 + u * 32 + lane;
            if (i >= qn || kw[u] == kEmptyKey) continue;
            h[u] = hash_key(kw[u]) & mask;
            old[u] = atomicCAS(slot_key(J.ht, h[u]), kEmptyKey, kw[u]);
          }
#pragma unroll
          for (int u = 0; u < E; ++u) {
            const uint32_t i = i0 + u * 32 + lane;
            slot[u] = kNone;
            if (i >= qn) continue;
            bool cl = false;
            if (kw[u] == kEmptyKey)
              slot[u] = ht_insert(J.ht, mask, kw[u], cl, &res->status);
            else
              slot[u] = ht_insert_from(J.ht, mask, kw[u], h[u], old[u], cl, &res->status);
            if (cl && J.filter) {
              const uint32_t fh = filter_hash(kw[u]);
              atomicOr(&J.filter[fh & (J.filter_words - 1)], bloom_bits(fh));
              if (J.bitmap) {
                if (kw[u] < 32ull * J.filter_words)
                  atomicOr(&J.bitmap[kw[u] >> 5], 1u << (kw[u] & 31u));
                else
                  oor = true;
              }
            }
          }
        } else {
#pragma unroll
          for (int u = 0; u < E; ++u) {
            const uint32_t i = i0 + u * 32 + lane;
            slot[u] = kNone;
            if (i >= qn) continue;
            const uint32_t row = rw[u];
            uint4 kw = make_uint4(0u, J.nk > 0 ? uint32_t(__ldg(J.kc[0] + row)) : 0u,
                                  J.nk > 1 ? uint32_t(__ldg(J.kc[1] + row)) : 0u,
                                  J.nk > 2 ? uint32_t(__ldg(J.kc[2] + row)) : 0u);
            bool cl = false;
            slot[u] = ht_insert_wide(J.ht, mask, kw, cl, &res->status);
          }
        }
#pragma unroll
        for (int u = 0; u < E; ++u) {
          const uint32_t i = i0 + u * 32 + lane;
          if (i >= qn) continue;
          uint32_t rank = 0;
          if (slot[u] != kNone) {
            rank = atomicAdd(slot_cnt(J.ht, J.wide, slot[u]), 1u);
            if (rank == 0) {
              ++n_first;
            } else {
              dup = true;
              if (J.tmin)
                atomicMin(reinterpret_cast<int*>(&J.sbegin[slot[u]]), __ldg(J.tcol + rw[u]));
            }
          }
          q_slot[i] = slot[u];
          q_rank[i] = rank;
        }
      }
      if (__syncthreads_or(oor) && tid == 0) atomicOr(&cs->oor[set][j], 1u);
      oor = false;
      // Offsets of this sweep's rows and keys: one advance of each counter
      // per block.
      n_first = __reduce_add_sync(0xffffffffu, n_first);
      if (lane == 0) {
        s_wq[warp] = qn;
        s_wc[warp] = n_first;
      }
      __syncthreads();
      if (warp == 0) {
        const uint32_t vq = lane < NW ? s_wq[lane] : 0u, vc = lane < NW ? s_wc[lane] : 0u;
        const uint32_t iq = warp_incl_scan(vq), ic = warp_incl_scan(vc);
        const uint32_t tq = __shfl_sync(0xffffffffu, iq, 31), tc = __shfl_sync(0xffffffffu, ic, 31);
        uint32_t bq = 0, bc = 0;
        if (lane == 0) {
          bq = tq ? atomicAdd(&cs->n_pass[set][j], tq) : 0u;
          bc = tc ? atomicAdd(&cs->n_new[set][j], tc) : 0u;
        }
        bq = __shfl_sync(0xffffffffu, bq, 0);
        bc = __shfl_sync(0xffffffffu, bc, 0);
        if (lane < NW) {
          s_wq[lane] = bq + iq - vq;
          s_wc[lane] = bc + ic - vc;
        }
      }
      __syncthreads();
      const uint32_t pb = s_wq[warp];
      uint32_t eb = s_wc[warp];
      // Two queue entries per lane at a time, every global load (the key
      // word from the slot, a tail level's value) issued before any store.
      for (uint32_t i0 = 0; i0 < qn; i0 += 64) {
        uint32_t sl[2], rk[2], row[2];
        uint64_t kw[2];
        int32_t tv[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const uint32_t i = i0 + u * 32 + lane;
          sl[u] = kNone;
          rk[u] = 0;
          row[u] = 0;
          if (i < qn) {
            sl[u] = q_slot[i];
            rk[u] = q_rank[i];
            row[u] = q_row[i];
          }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          kw[u] = 0;  // wide entries keep only the parent (the root: 0)
          tv[u] = 0;
          if (sl[u] == kNone || rk[u] != 0) continue;
          if (!J.wide) {
            if (sl[u] == mask + 1) {
              kw[u] = kEmptyKey;
            } else {  // the key word from its slot
              const uint4 v = J.ht[sl[u]];
              kw[u] = (uint64_t(v.y) << 32) | v.x;
            }
          }
          if (J.tmin) tv[u] = __ldg(J.tcol + row[u]);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const uint32_t i = i0 + u * 32 + lane;
          if (i < qn) {
            J.tmp_row[pb + i] = row[u];
            J.tmp_slot[pb + i] = sl[u];
            J.newslots[pb + i] = rk[u];
          }
          const bool first = sl[u] != kNone && rk[u] == 0;
          const uint32_t fm = __ballot_sync(0xffffffffu, first);
          if (first) {
            // The entry, as if its key had only this row (D corrects the
            // ranges when some key repeats): list position er, offset er.
            const uint32_t er = eb + __popc(fm & lanemask_lt()), e = J.base_e + er;
            J.slot_of[er] = sl[u];
            *slot_e(J.ht, J.wide, sl[u]) = e;
            J.key[e] = kw[u];
            J.count[e] = 1;
            J.begin[e] = er;
            J.fill[e] = J.ident ? er : row[u];  // a row read from perm: D places it
            if (J.ident) J.perm[er] = row[u];
            if (J.cstate) J.cstate[e] = kUnforced;
            if (J.cnkeys) J.cnkeys[e] = 0;
            if (J.cfirst) J.cfirst[e] = 0;
            if (J.tmin) J.tmin[e] = tv[u];
          }
          eb += __popc(fm);
        }
      }
      __syncthreads();  // the queues are reused by the next sweep
    }
  }
  if (__syncthreads_or(dup) && tid == 0) cs->dup[set] = 1u;
  if (!grid_sync(cs, &res->status, spin, bar_target += gridDim.x)) return;
  // Every key has exactly one row: no E.
  const bool scatter = ld_acquire_gpu(&cs->dup[set]) != 0;
  if (tid < uint32_t(nj)) {
    s_np[tid] = ld_acquire_gpu(&cs->n_pass[set][tid]);
    s_nn[tid] = ld_acquire_gpu(&cs->n_new[set][tid]);
  }
  __syncthreads();

  // The level's bookkeeping (block 0, while the others go on; nothing in
  // D or E reads it).  The table's dirty slots are the listed ones from
  // here on; the Bloom filter is used when it has at least four bits per
  // key.  The entries' fill cursors stay at their first offsets: forcing
  // the next level resets the cursors of the parents it regroups.
  if (blockIdx.x == 0 && tid < uint32_t(nj)) {
    const int j = tid;
    const RootJob& J = s_job[j];
    AtomDev& a = fj.atoms[fj.jobs[j].x];
    LevelDev& L = a.L[fj.jobs[j].y];
    LevelDev& P = a.L[fj.jobs[j].y - 1];
    if (!J.act) {  // nothing to build: the request list starts empty again
      L.n_req = 0;
      L.n_in = 0;
    } else {
      const uint32_t np = s_np[j], nn = s_nn[j];
      if (request_all) P.child_state[0] = kForced;
      for (uint32_t r = 0; r < L.n_req; ++r) P.child_state[L.req[r]] = kForced;
      P.child_first[0] = J.base_e;
      P.child_nkeys[0] = nn;
      if (J.ident) {
        a.n_pass = np;
        a.root_mat = 1;
        P.begin[0] = 0;
        P.count[0] = np;
      }
      if (!scatter) *J.pfill = np;  // the rows were placed without the cursor
      atomicAdd(&res->ctr[FJ_CTR_ROOTS_BUILT], 1ull);
      atomicOr(reinterpret_cast<unsigned long long*>(&res->ctr[FJ_CTR_ATOM_BUILT_MASK]),
               1ull << fj.jobs[j].x);
      atomicAdd(&res->ctr[FJ_CTR_ROWS_REGROUPED], (unsigned long long)np);
      L.filter_on = J.filter && uint64_t(nn) * 4 <= uint64_t(J.filter_words) * 32;
      L.exact = J.bitmap && !ld_acquire_gpu(&cs->oor[set][j]);
      L.n_rows = J.src;
      L.n_tmp = np;
      L.n_new = nn;
      L.base = J.base_e;
      L.n_entries = J.base_e + nn;
      L.cleared = 1;
      L.n_req = 0;
      L.n_in = 0;
      L.n_listed = nn;
      L.ht_state = kHtListed;
    }
  }

  // The entries C wrote are final when every key has one row and every
  // job's rows are the base table's.
  bool fix = scatter;
  for (int j = 0; j < nj; ++j) fix |= s_job[j].act && !s_job[j].ident;
  if (!fix) return;

  // D: each entry's range inside the root's range, ED consecutive entries
  // per thread: when some key repeats, its count from the slot and its
  // first offset from a block scan of the counts (one advance of the root's
  // fill cursor per sweep), and a tail level's MIN folds the slot's running
  // MIN in; otherwise offset = list position, and a row that came from perm
  // (kept in the entry's fill cursor by C) is placed here.
  jobs_prefix(nj, s_off, [&](int j) { return s_job[j].act ? s_nn[j] : 0u; });
  block_range(s_off[nj], lo, hi);
  for (int j = 0; j < nj; ++j) {
    const uint32_t a0 = max(lo, s_off[j]), a1 = min(hi, s_off[j + 1]);
    if (a0 >= a1) continue;
    const RootJob& J = s_job[j];
    const uint32_t r1 = a1 - s_off[j];
    constexpr int ED = E;  // entries per thread per sweep
    for (uint32_t r = a0 - s_off[j]; r < r1; r += ED * NT) {
      uint32_t sl[ED], cnt[ED], prow[ED], sum = 0;
      int32_t smin[ED];
      const uint32_t i0 = r + tid * ED;
#pragma unroll
      for (int u = 0; u < ED; ++u) sl[u] = i0 + u < r1 ? J.slot_of[i0 + u] : kNone;
#pragma unroll
      for (int u = 0; u < ED; ++u) {
        const uint32_t e = J.base_e + i0 + u;
        cnt[u] = 0;
        prow[u] = 0;
        smin[u] = 0;
        if (sl[u] == kNone) continue;
        cnt[u] = 1;
        if (scatter) {
          cnt[u] = *slot_cnt(J.ht, J.wide, sl[u]);
          if (J.tmin) smin[u] = min(J.tmin[e], int32_t(J.sbegin[sl[u]]));
        } else if (!J.ident) {
          prow[u] = J.fill[e];
        }
        sum += cnt[u];
      }
      uint32_t b = i0;  // the root's range starts at 0
      if (scatter) {
        uint32_t tot;
        const uint32_t pre = block_excl_scan<uint32_t>(sum, s_scan, &tot);
        if (tid == 0) s_base2 = tot ? atomicAdd(J.pfill, tot) : 0u;
        __syncthreads();
        b = s_base2 + pre;
      }
#pragma unroll
      for (int u = 0; u < ED; ++u) {
        if (sl[u] == kNone) continue;
        const uint32_t e = J.base_e + i0 + u;
        if (scatter) {
          J.count[e] = cnt[u];
          J.begin[e] = b;
          J.fill[e] = b;
          J.sbegin[sl[u]] = b;
          if (J.tmin) J.tmin[e] = smin[u];
        } else {  // a row from perm, placed at its entry's offset
          J.perm[b] = prow[u];
          J.fill[e] = b;
        }
        b += cnt[u];
      }
      if (scatter) __syncthreads();
    }
  }

  if (!scatter) return;
  if (!grid_sync(cs, &res->status, spin, bar_target += gridDim.x)) return;

  // E: every passing row to its place in its entry's range (the entry's
  // first offset, kept per slot by D, plus the row's rank from C).
  jobs_prefix(nj, s_off, [&](int j) { return s_job[j].act ? s_np[j] : 0u; });
  block_range(s_off[nj], lo, hi);
  for (uint32_t x0 = lo; x0 < hi; x0 += E * NT) {
    uint32_t t[E], rk[E], rw[E], b[E];
    int jj[E];
#pragma unroll
    for (int u = 0; u < E; ++u) {
      const uint32_t x = x0 + u * NT + tid;
      t[u] = kNone;
      jj[u] = 0;
      if (x >= hi) continue;
      jj[u] = job_at(s_off, nj, x);
      const RootJob& J = s_job[jj[u]];
      t[u] = J.tmp_slot[x - s_off[jj[u]]];
      rk[u] = J.newslots[x - s_off[jj[u]]];
      rw[u] = J.tmp_row[x - s_off[jj[u]]];
    }
#pragma unroll
    for (int u = 0; u < E; ++u)
      if (t[u] != kNone) b[u] = s_job[jj[u]].sbegin[t[u]];
#pragma unroll
    for (int u = 0; u < E; ++u)
      if (t[u] != kNone) s_job[jj[u]].perm[b[u] + rk[u]] = rw[u];
  }
}

}  // namespace fj
