// Node execution kernels: cover choice, fanout, and the vectorized expansion
// (paper Section 3.3 Fig. 7, Section 4.3 Fig. 11, Section 4.4).
//
// A node's input is a set of partial tuples ("items"): the variables bound by
// earlier nodes, one COLT handle per atom (an entry of the atom's level that
// earlier nodes reached), and a bag multiplicity.  Every item contributes as
// many cover elements as its chosen cover has: the offsets of a COLT vector
// when the cover is the atom's last level (iterated without forcing, as the
// `is_suffix` case of Fig. 10), or the keys of a forced map otherwise.  A
// prefix sum of these fanouts maps a flat position space onto
// (item, element), which is cut into batches of `tile` elements -- the
// paper's batch of cover tuples -- each handled by one thread block: the
// block binds the batch, then probes one subatom at a time for the whole
// batch, compacting the survivors in shared memory after every probe.
#pragma once

#include "fj_kernels.cuh"

namespace fj {

__device__ __forceinline__ uint32_t item_handle(const NodeDev& nd, const SubDev& s, uint32_t it) {
  return s.hslot < 0 ? 0u : nd.in_h[s.hslot][it];
}

// Estimated number of keys of a subatom's trie for one item (Section 4.4): a
// forced map knows its key count; an unforced COLT vector uses its length.
__device__ __forceinline__ uint64_t cover_estimate(const AtomDev& a, const SubDev& s, uint32_t h) {
  const LevelDev& P = a.L[s.lvl];
  if (P.child_state[h] == kForced) return P.child_nkeys[h];
  if (s.lvl == 0 && !a.root_mat) return a.n_rows;
  return P.count[h];
}

// Per item: pick the cover and request forcing of every trie the item will
// probe, or iterate as a map.
__global__ void __launch_bounds__(kThreads) k_choose(const __grid_constant__ NodeDev nd,
                                                     AtomDev* atoms) {
  uint32_t n = nd.single_item ? 1u : *nd.n_items;
  for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < n; it += gridDim.x * blockDim.x) {
    int c = 0;
    if (nd.dynamic) {
      uint64_t best = ~0ull;
      for (int s = 0; s < nd.n_sub; ++s) {
        const SubDev& S = nd.sub[s];
        if (!S.is_cover) continue;
        uint64_t est = cover_estimate(atoms[S.atom], S, item_handle(nd, S, it));
        if (est < best) {
          best = est;
          c = s;
        }
      }
    }
    nd.choice[it] = uint8_t(c);
    for (int s = 0; s < nd.n_sub; ++s) {
      const SubDev& S = nd.sub[s];
      if (s == c && S.last) continue;  // iterated as a vector: nothing to build
      AtomDev& a = atoms[S.atom];
      uint32_t h = item_handle(nd, S, it);
      LevelDev& P = a.L[S.lvl];
      if (P.child_state[h] == kUnforced &&
          atomicCAS(&P.child_state[h], kUnforced, kRequested) == kUnforced) {
        LevelDev& L = a.L[S.lvl + 1];
        uint32_t idx = atomicAdd(&L.n_req, 1u);
        L.req[idx] = h;
      }
    }
  }
}

// Per item: number of cover elements (after forcing).
__global__ void __launch_bounds__(kThreads) k_fanout(const __grid_constant__ NodeDev nd,
                                                     AtomDev* atoms) {
  uint32_t n = nd.single_item ? 1u : *nd.n_items;
  for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < n; it += gridDim.x * blockDim.x) {
    const SubDev& S = nd.sub[nd.choice[it]];
    const AtomDev& a = atoms[S.atom];
    uint32_t h = item_handle(nd, S, it);
    const LevelDev& P = a.L[S.lvl];
    uint64_t f;
    if (S.last)
      f = (S.lvl == 0 && !a.root_mat) ? a.n_rows : P.count[h];
    else
      f = P.child_nkeys[h];
    nd.fan[it] = f;
  }
}

struct FanScanOp {
  const uint64_t* fan;
  uint64_t* scan;
  uint64_t* total_out;
  const uint32_t* n_items;
  uint32_t single;
  __device__ uint64_t n(int) const { return single ? 1u : *n_items; }
  __device__ uint64_t load(int, uint64_t i) const { return fan[i]; }
  __device__ void store(int, uint64_t i, uint64_t v) const { scan[i] = v; }
  __device__ void total(int, uint64_t v) const {
    scan[single ? 1u : *n_items] = v;
    *total_out = v;
  }
};

__device__ __forceinline__ uint64_t upper_bound_u64(const uint64_t* a, uint64_t lo, uint64_t hi,
                                                    uint64_t x) {
  while (lo < hi) {
    uint64_t mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Shared-memory state of one batch.
struct BatchSmem {
  uint32_t* item;
  uint32_t* elem;
  uint64_t* mult;
  uint32_t* newh;  // [n_sub][tile]
  uint16_t* list[2];
};

// Value j of the key of entry e in the map level of subatom S (a wide level
// reads it from one row of the entry's vector; all its rows share the key).
__device__ __forceinline__ int32_t map_key_value(const AtomDev& a, const SubDev& S, uint32_t e,
                                                 int j) {
  const LevelDev& L = a.L[S.lvl + 1];
  if (L.wide) return __ldg(&a.cols[S.col[j]][a.perm[L.begin[e]]]);
  return key_value(L.key[e], L.nk, j);
}

// Value of variable u for batch slot i (item it, cover c): from the input
// items when bound earlier, else from the cover element (a base-table row for
// a vector cover, a map key for a map cover).
__device__ __forceinline__ int32_t load_var(const NodeDev& nd, const AtomDev* atoms,
                                            const BatchSmem& b, int u, int i, uint32_t it, int c) {
  if ((nd.avs_mask >> u) & 1u) return nd.in_var[u][it];
  const SubDev& S = nd.sub[c];
  int j = nd.vpos[c][u];
  const AtomDev& a = atoms[S.atom];
  if (S.last) return __ldg(&a.cols[S.col[j]][b.elem[i]]);
  return map_key_value(a, S, b.elem[i], j);
}

__device__ __forceinline__ uint64_t mul_sat(uint64_t a, uint64_t b, uint32_t* status) {
  if (__umul64hi(a, b) != 0) {
    atomicOr(status, kStCountOverflow);
    return ~0ull;
  }
  return a * b;
}

// Append slot i to list `dst` when keep is set (warp-aggregated).
__device__ __forceinline__ void append_keep(bool keep, uint16_t i, uint16_t* dst, uint32_t* cnt) {
  uint32_t m = __ballot_sync(0xffffffffu, keep);
  if (m == 0) return;
  uint32_t leader = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane_id() == leader) base = atomicAdd(cnt, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (keep) dst[base + __popc(m & lanemask_lt())] = i;
}

__global__ void __launch_bounds__(kThreads) k_expand(const __grid_constant__ NodeDev nd,
                                                     AtomDev* atoms, ResultDev* res) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int T = nd.tile;
  BatchSmem b;
  {
    uint8_t* p = smem;
    b.mult = reinterpret_cast<uint64_t*>(p);
    p += sizeof(uint64_t) * T;
    b.item = reinterpret_cast<uint32_t*>(p);
    p += sizeof(uint32_t) * T;
    b.elem = reinterpret_cast<uint32_t*>(p);
    p += sizeof(uint32_t) * T;
    b.newh = reinterpret_cast<uint32_t*>(p);
    p += sizeof(uint32_t) * T * nd.n_sub;
    b.list[0] = reinterpret_cast<uint16_t*>(p);
    p += sizeof(uint16_t) * T;
    b.list[1] = reinterpret_cast<uint16_t*>(p);
  }
  __shared__ uint32_t s_cnt[2];
  __shared__ uint64_t s_range[2];
  __shared__ uint32_t s_base;
  __shared__ unsigned long long s_u64[33];
  __shared__ int32_t s_min[FJ_MAX_VARS];
  __shared__ unsigned long long s_ctr[4];  // cover iters, probes, hits, survivors

  if (threadIdx.x < FJ_MAX_VARS) s_min[threadIdx.x] = INT32_MAX;
  if (threadIdx.x < 4) s_ctr[threadIdx.x] = 0;
  unsigned long long my_count = 0;
  bool any_out = false;

  uint32_t n_items = nd.single_item ? 1u : *nd.n_items;
  uint64_t end = nd.chunk_end;
  if (!nd.single_item) end = min(end, nd.scan[n_items]);
  __syncthreads();

  for (uint64_t tile = blockIdx.x;; tile += gridDim.x) {
    uint64_t tpos = nd.chunk_begin + tile * uint64_t(T);
    if (tpos >= end) break;
    uint32_t tn = uint32_t(min(uint64_t(T), end - tpos));
    if (threadIdx.x == 0) {
      s_cnt[0] = 0;
      s_cnt[1] = 0;
      if (!nd.single_item) {
        s_range[0] = upper_bound_u64(nd.scan, 0, uint64_t(n_items) + 1, tpos) - 1;
        s_range[1] = upper_bound_u64(nd.scan, 0, uint64_t(n_items) + 1, tpos + tn - 1);
      }
    }
    __syncthreads();
    // Phase 0: bind the batch of cover elements.
    for (uint32_t base = 0; base < uint32_t(T); base += blockDim.x) {
      uint32_t i = base + threadIdx.x;
      bool alive = i < tn;
      if (alive) {
        uint64_t pos = tpos + i;
        uint32_t it = 0;
        uint64_t j = pos;
        if (!nd.single_item) {
          it = uint32_t(upper_bound_u64(nd.scan, s_range[0], s_range[1], pos) - 1);
          j = pos - nd.scan[it];
        }
        int c = nd.choice[it];
        const SubDev& S = nd.sub[c];
        const AtomDev& a = atoms[S.atom];
        uint32_t h = item_handle(nd, S, it);
        uint32_t elem;
        if (S.last) {
          if (S.lvl == 0 && !a.root_mat) {
            elem = uint32_t(j);
            alive = row_passes(a, elem);
          } else {
            elem = a.perm[a.L[S.lvl].begin[h] + uint32_t(j)];
          }
        } else {
          elem = a.L[S.lvl].child_first[h] + uint32_t(j);
          b.newh[c * T + i] = elem;
        }
        b.item[i] = it;
        b.elem[i] = elem;
        b.mult[i] = nd.in_mult ? nd.in_mult[it] : 1ull;
        // A cover holding variables bound by earlier nodes only yields the
        // elements that agree with them.
        if (alive && S.bound_mask) {
          for (int j = 0; j < S.nv; ++j) {
            if (!((S.bound_mask >> j) & 1u)) continue;
            int32_t v;
            if (S.last)
              v = __ldg(&a.cols[S.col[j]][elem]);
            else
              v = map_key_value(a, S, elem, j);
            if (v != nd.in_var[S.var[j]][it]) alive = false;
          }
        }
      }
      append_keep(alive, uint16_t(i), b.list[0], &s_cnt[0]);
    }
    if (threadIdx.x == 0) atomicAdd(&s_ctr[0], (unsigned long long)tn);
    __syncthreads();
    int cur = 0;
    // Probe phases: one subatom at a time for the whole batch (Fig. 11).
    for (int s = 0; s < nd.n_sub; ++s) {
      if (!nd.dynamic && s == 0) continue;
      const SubDev& S = nd.sub[s];
      const AtomDev& a = atoms[S.atom];
      const LevelDev& L = a.L[S.lvl + 1];
      uint32_t n = s_cnt[cur];
      uint32_t probes = 0, hits = 0;
      for (uint32_t base = 0; base < n; base += blockDim.x) {
        uint32_t q = base + threadIdx.x;
        bool keep = false;
        uint16_t i = 0;
        if (q < n) {
          i = b.list[cur][q];
          uint32_t it = b.item[i];
          int c = nd.choice[it];
          keep = true;
          if (c != s) {
            uint32_t h = item_handle(nd, S, it);
            int32_t v0 = S.nv > 0 ? load_var(nd, atoms, b, S.var[0], i, it, c) : 0;
            int32_t v1 = S.nv > 1 ? load_var(nd, atoms, b, S.var[1], i, it, c) : 0;
            uint32_t e = 0, cnt = 0;
            ++probes;
            if (L.wide) {
              int32_t v2 = S.nv > 2 ? load_var(nd, atoms, b, S.var[2], i, it, c) : 0;
              keep = ht_find_wide(L.ht, L.mask,
                                  make_uint4(h, uint32_t(v0), uint32_t(v1), uint32_t(v2)), e, cnt);
            } else {
              keep = ht_find(L.ht, L.mask, pack_key(h, L.nk, v0, v1), e, cnt);
            }
            if (keep) {
              ++hits;
              if (S.last) {
                if (nd.track_mult) b.mult[i] = mul_sat(b.mult[i], cnt, &res->status);
              } else {
                b.newh[s * T + i] = e;
              }
            }
          }
        }
        append_keep(keep, i, b.list[cur ^ 1], &s_cnt[cur ^ 1]);
      }
      if (probes) atomicAdd(&s_ctr[1], (unsigned long long)probes);
      if (hits) atomicAdd(&s_ctr[2], (unsigned long long)hits);
      __syncthreads();
      if (threadIdx.x == 0) s_cnt[cur] = 0;
      cur ^= 1;
      __syncthreads();
    }
    uint32_t n = s_cnt[cur];
    if (threadIdx.x == 0) atomicAdd(&s_ctr[3], (unsigned long long)n);
    // Epilogue.
    if (nd.mode == kModeItems) {
      if (threadIdx.x == 0) {
        uint32_t bse = n ? atomicAdd(nd.out_n, n) : 0u;
        if (bse + n > nd.out_cap) atomicOr(&res->status, kStItemsOverflow);
        s_base = bse;
      }
      __syncthreads();
      uint32_t obase = s_base;
      for (uint32_t q = threadIdx.x; q < n; q += blockDim.x) {
        uint32_t o = obase + q;
        if (o >= nd.out_cap) break;
        uint16_t i = b.list[cur][q];
        uint32_t it = b.item[i];
        int c = nd.choice[it];
        for (int k = 0; k < nd.n_out_vars; ++k)
          nd.out_var[k][o] = load_var(nd, atoms, b, nd.out_var_id[k], i, it, c);
        for (int a = 0; a < FJ_MAX_ATOMS; ++a) {
          if (!nd.out_h[a]) continue;
          int src = nd.out_h_src[a];
          nd.out_h[a][o] = src >= 0 ? b.newh[src * T + i] : nd.in_h[a][it];
        }
        if (nd.out_mult) nd.out_mult[o] = b.mult[i];
      }
    } else if (nd.mode == kModeAggregate) {
      for (uint32_t q = threadIdx.x; q < n; q += blockDim.x) {
        uint16_t i = b.list[cur][q];
        uint32_t it = b.item[i];
        int c = nd.choice[it];
        uint64_t m = b.mult[i];
        for (int t = 0; t < nd.n_tail; ++t) {
          const TailDev& td = nd.tail[t];
          const AtomDev& ta = atoms[td.atom];
          uint32_t h = td.hsrc >= 0 ? b.newh[td.hsrc * T + i] : nd.in_h[td.atom][it];
          m = mul_sat(m, ta.L[td.lvl].count[h], &res->status);
        }
        if (m == 0) continue;
        unsigned long long before = my_count;
        my_count += m;
        if (my_count < before) atomicOr(&res->status, kStCountOverflow);
        any_out = true;
        for (int k = 0; k < nd.n_min; ++k)
          atomicMin(&s_min[nd.min_idx[k]], load_var(nd, atoms, b, nd.min_var[k], i, it, c));
        for (int t = 0; t < nd.n_tail; ++t) {
          const TailDev& td = nd.tail[t];
          if (!td.n_min) continue;
          const AtomDev& ta = atoms[td.atom];
          uint32_t h = td.hsrc >= 0 ? b.newh[td.hsrc * T + i] : nd.in_h[td.atom][it];
          uint32_t bg = ta.L[td.lvl].begin[h], cn = ta.L[td.lvl].count[h];
          for (int k = 0; k < td.n_min; ++k) {
            const int32_t* col = ta.cols[td.min_col[k]];
            int32_t lo = INT32_MAX;
            for (uint32_t r = 0; r < cn; ++r) lo = min(lo, col[ta.perm[bg + r]]);
            atomicMin(&s_min[td.min_idx[k]], lo);
          }
        }
      }
    } else {  // kModeMaterialize
      for (uint32_t base = 0; base < n; base += blockDim.x) {
        uint32_t q = base + threadIdx.x;
        uint64_t m = 0;
        uint16_t i = 0;
        if (q < n) {
          i = b.list[cur][q];
          m = b.mult[i];
        }
        unsigned long long tot;
        unsigned long long ex = block_excl_scan<unsigned long long>(m, s_u64, &tot);
        if (threadIdx.x == 0) s_range[0] = atomicAdd(&res->n_out, tot);
        __syncthreads();
        uint64_t row0 = s_range[0] + ex;
        if (q < n && m) {
          uint32_t it = b.item[i];
          int c = nd.choice[it];
          for (uint64_t r = 0; r < m; ++r) {
            uint64_t row = row0 + r;
            if (row >= nd.out_rows_cap) {
              atomicOr(&res->status, kStOutputOverflow);
              break;
            }
            for (int h = 0; h < nd.n_head; ++h)
              nd.out_tuples[row * nd.n_head + h] =
                  load_var(nd, atoms, b, nd.head_var[h], i, it, c);
          }
        }
        __syncthreads();
      }
    }
    __syncthreads();
  }
  // Block totals.
  if (nd.mode == kModeAggregate) {
    unsigned long long tot = block_sum<unsigned long long>(my_count, s_u64);
    int any = __syncthreads_or(any_out);
    if (threadIdx.x == 0 && tot) {
      unsigned long long old = atomicAdd(&res->count, tot);
      if (old + tot < old) atomicOr(&res->status, kStCountOverflow);
    }
    // Every MIN slot is flushed (a slot still at INT32_MAX leaves the result
    // unchanged); validity of the MINs is COUNT > 0.
    if (any && threadIdx.x < FJ_MAX_VARS) atomicMin(&res->mins[threadIdx.x], s_min[threadIdx.x]);
  }
  __syncthreads();
  if (threadIdx.x < 4 && s_ctr[threadIdx.x]) {
    const int slot[4] = {FJ_CTR_COVER_ITERS, FJ_CTR_PROBES, FJ_CTR_PROBE_HITS, FJ_CTR_SURVIVORS};
    atomicAdd(&res->ctr[slot[threadIdx.x]], s_ctr[threadIdx.x]);
  }
}

// Reset the COLT state of every atom (nothing built) and/or the result.
__global__ void k_reset(AtomDev* atoms, int n_atoms, ResultDev* res, int do_atoms) {
  int a = blockIdx.x;
  if (do_atoms && a < n_atoms && threadIdx.x == 0) {
    AtomDev& A = atoms[a];
    A.root_mat = 0;
    A.n_pass = 0;
    LevelDev& R = A.L[0];
    R.begin[0] = 0;
    R.count[0] = A.n_rows;
    R.child_state[0] = kUnforced;
    R.child_first[0] = 0;
    R.child_nkeys[0] = 0;
    for (int l = 1; l < A.n_levels; ++l) {
      LevelDev& L = A.L[l];
      L.cleared = 0;
      L.n_entries = 0;
      L.n_req = 0;
      L.n_new = 0;
      L.n_rows = 0;
      L.base = 0;
      L.pos_total = 0;
      L.mask = 0;
      L.n_in = 0;
    }
  }
  if (a == 0 && threadIdx.x == 0) {
    res->count = 0;
    res->n_out = 0;
    res->status = 0;
    for (int k = 0; k < FJ_MAX_VARS; ++k) res->mins[k] = INT32_MAX;
    for (int k = 0; k < 16; ++k) res->ctr[k] = 0;
  }
}

// Eager forcing (simple trie / simple lazy trie ablations): request every
// entry of L[lvl-1] that is not yet forced.
__global__ void k_request_all(AtomDev* atoms, int atom, int lvl) {
  AtomDev& a = atoms[atom];
  LevelDev& P = a.L[lvl - 1];
  LevelDev& L = a.L[lvl];
  uint32_t n = lvl == 1 ? 1u : a.L[lvl - 1].n_entries;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    if (P.child_state[e] == kUnforced && atomicCAS(&P.child_state[e], kUnforced, kRequested) == kUnforced) {
      uint32_t idx = atomicAdd(&L.n_req, 1u);
      L.req[idx] = e;
    }
  }
}

}  // namespace fj
