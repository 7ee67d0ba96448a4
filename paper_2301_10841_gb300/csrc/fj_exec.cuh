// Node execution kernels: cover choice, fanout, and the vectorized expansion
// (paper Section 3.3 Fig. 7, Section 4.3 Fig. 13, Section 4.4).
//
// A node's input is a set of partial tuples ("items"): the variables bound by
// earlier nodes, one COLT handle per atom (an entry of the atom's level that
// earlier nodes reached), and a bag multiplicity.  Every item contributes as
// many cover elements as its chosen cover has: the offsets of a COLT vector
// when the cover is the atom's last level (iterated without forcing, as the
// `is_suffix` case of Fig. 12), or the keys of a forced map otherwise.  A
// prefix sum of these fanouts maps a flat position space onto
// (item, element), which is cut into batches of `tile` elements -- the
// paper's batch of cover tuples -- each handled by one thread block: the
// block binds the batch, then probes one subatom at a time for the whole
// batch, compacting the survivors in shared memory after every probe.
#pragma once

#include "fj_kernels.cuh"

namespace fj {

static_assert(sizeof(NodeDev) < 32000, "node descriptor must fit the kernel parameter space");

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
// With a single input tuple (node 0) the subatoms are handled by one thread
// each, so the node's requests do not wait on each other.
__device__ __forceinline__ void request_force(AtomDev* atoms, const SubDev& S, uint32_t h) {
  AtomDev& a = atoms[S.atom];
  LevelDev& P = a.L[S.lvl];
  if (P.child_state[h] == kUnforced &&
      atomicCAS(&P.child_state[h], kUnforced, kRequested) == kUnforced) {
    LevelDev& L = a.L[S.lvl + 1];
    uint32_t idx = atomicAdd(&L.n_req, 1u);
    L.req[idx] = h;
  }
}

__global__ void __launch_bounds__(kThreads) k_choose(const __grid_constant__ NodeDev nd,
                                                     AtomDev* atoms) {
  if (nd.single_item && !nd.dynamic) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s == 0) nd.choice[0] = 0;
    if (s < nd.n_sub && !(s == 0 && nd.sub[0].last)) request_force(atoms, nd.sub[s], 0u);
    return;
  }
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

// Value j of the key of entry e in the map level of subatom S (a wide level
// reads it from one row of the entry's vector; all its rows share the key).
__device__ __forceinline__ int32_t map_key_value(const AtomDev& a, const SubDev& S, uint32_t e,
                                                 int j) {
  const LevelDev& L = a.L[S.lvl + 1];
  if (L.wide) return __ldg(&a.cols[S.col[j]][a.perm[L.begin[e]]]);
  return key_value(L.key[e], L.nk, j);
}

// Value of variable u for a batch element (item it, cover c, cover element
// elem): from the input tuples when an earlier node bound it, else from the
// cover element (a base-table row for a vector cover, a map key otherwise).
__device__ __forceinline__ int32_t load_var(const NodeDev& nd, const AtomDev* atoms, int u,
                                            uint32_t it, int c, uint32_t elem) {
  if ((nd.avs_mask >> u) & 1u) return nd.in_var[u][it];
  const SubDev& S = nd.sub[c];
  int j = nd.vpos[c][u];
  const AtomDev& a = atoms[S.atom];
  if (S.last) return __ldg(&a.cols[S.col[j]][elem]);
  return map_key_value(a, S, elem, j);
}

__device__ __forceinline__ uint64_t mul_sat(uint64_t a, uint64_t b, uint32_t* status) {
  if (__umul64hi(a, b) != 0) {
    atomicOr(status, kStCountOverflow);
    return ~0ull;
  }
  return a * b;
}

// First step of a narrow lookup: the Bloom filter (when on) and the load of
// the first hash slot.  Returns false when the filter rules the key out.
__device__ __forceinline__ bool probe_start(const uint4* __restrict__ ht, uint32_t mask,
                                            const uint32_t* __restrict__ filt, uint32_t fwords,
                                            uint64_t kw, uint32_t& hh, uint4& sl) {
  if (filt && kw != kEmptyKey && bloom_rejects(filt, fwords, filter_hash(kw))) return false;
  hh = hash_key(kw) & mask;
  sl = __ldg(&ht[hh]);
  return true;
}

// Rest of a lookup whose first slot is already loaded (narrow levels).
__device__ __forceinline__ bool ht_resolve(const uint4* __restrict__ ht, uint32_t mask,
                                           uint64_t kw, uint32_t h, uint4 sl, uint32_t& e,
                                           uint32_t& cnt) {
  for (uint32_t it = 0; it <= mask; ++it) {
    uint64_t k = (uint64_t(sl.y) << 32) | sl.x;
    if (k == kw) {
      e = sl.z;
      cnt = sl.w;
      return true;
    }
    if (k == kEmptyKey) return false;
    h = (h + 1) & mask;
    sl = __ldg(&ht[h]);
  }
  return false;
}

// Factorized output (FJ_OUT_FACTORIZED, the result in trie form of
// Section 4.4): a live element becomes one row -- the head variables bound so
// far, its multiplicity (two words, low first), and per tail the first
// offset and length of the COLT vector the tail would iterate -- unless a
// vector is empty.  `handle(t)` gives tail t's entry and `value(v)` the value
// of variable v.  The element's bag size is added to my_count.  Rows are
// appended warp-wide: every lane of the warp calls this together.
template <typename H, typename V>
__device__ __forceinline__ void factor_emit(const NodeDev& nd, const AtomDev* atoms,
                                            ResultDev* res, bool live, uint64_t mult,
                                            H handle, V value,
                                            unsigned long long& my_count) {
  uint64_t m = live ? mult : 0;
  for (int t = 0; t < nd.n_tail && m; ++t) {
    const TailDev& td = nd.tail[t];
    m = mul_sat(m, atoms[td.atom].L[td.lvl].count[handle(t)], &res->status);
  }
  const bool emit = m != 0;
  const uint32_t em = __ballot_sync(0xffffffffu, emit);
  uint64_t base = 0;
  if (lane_id() == 0 && em) base = atomicAdd(&res->n_out, (unsigned long long)__popc(em));
  base = __shfl_sync(0xffffffffu, (unsigned long long)base, 0);
  if (!emit) return;
  const unsigned long long before = my_count;
  my_count += m;
  if (my_count < before) atomicOr(&res->status, kStCountOverflow);
  const uint64_t pos = base + __popc(em & lanemask_lt());
  if (pos >= nd.out_rows_cap) {
    atomicOr(&res->status, kStOutputOverflow);
    return;
  }
  const int width = nd.n_pre + 2 + 2 * nd.n_tail;
  int32_t* row = nd.out_tuples + pos * uint64_t(width);
  for (int k = 0; k < nd.n_pre; ++k) row[k] = value(nd.pre_var[k]);
  row[nd.n_pre] = int32_t(uint32_t(mult));
  row[nd.n_pre + 1] = int32_t(uint32_t(mult >> 32));
  for (int t = 0; t < nd.n_tail; ++t) {
    const TailDev& td = nd.tail[t];
    const LevelDev& L = atoms[td.atom].L[td.lvl];
    const uint32_t h = handle(t);
    row[nd.n_pre + 2 + 2 * t] = int32_t(L.begin[h]);
    row[nd.n_pre + 3 + 2 * t] = int32_t(L.count[h]);
  }
}

// Expansion of one node over positions [chunk_begin, chunk_end): batches of
// T = R * 256 cover elements; thread t owns batch elements r * 256 + t.  Each
// probe phase first gathers the keys of all of a thread's live elements,
// then issues all their first hash-slot loads, then resolves them, so every
// thread keeps R independent gathers in flight.
// Blocks per SM the register budget is sized for (R elements per thread).
constexpr int expand_min_blocks(int r) { return r >= 8 ? 1 : (r == 4 ? 2 : 3); }

template <int R>
__global__ void __launch_bounds__(kThreads, expand_min_blocks(R))
    k_expand(const __grid_constant__ NodeDev nd, AtomDev* atoms, ResultDev* res) {
  // A root build whose bounded wait ran out left its levels unbuilt.
  if (__syncthreads_or(threadIdx.x == 0 && (res->status & kStTimeout))) return;
  extern __shared__ uint32_t s_newh[];  // [n_sub][T]: handles found by probes
  constexpr int T = R * kThreads;
  __shared__ uint64_t s_range[2];
  __shared__ unsigned long long s_red[33];
  __shared__ int32_t s_min[FJ_MAX_VARS];
  const uint32_t tid = threadIdx.x;
  if (tid < FJ_MAX_VARS) s_min[tid] = INT32_MAX;
  unsigned long long my_count = 0, c_iters = 0, c_probes = 0, c_hits = 0, c_surv = 0;
  bool any_out = false;
  uint32_t n_items = nd.single_item ? 1u : *nd.n_items;
  uint64_t end = nd.chunk_end;
  if (!nd.single_item) end = min(end, nd.scan[n_items]);
  if (nd.check_total && !nd.single_item && blockIdx.x == 0 && tid == 0 &&
      nd.scan[n_items] > nd.chunk_end)
    atomicOr(&res->status, kStItemsOverflow);
  __syncthreads();

  for (uint64_t tile = blockIdx.x;; tile += gridDim.x) {
    uint64_t tpos = nd.chunk_begin + tile * uint64_t(T);
    if (tpos >= end) break;
    uint32_t tn = uint32_t(min(uint64_t(T), end - tpos));
    uint64_t lo = 0, hi = 1;
    if (!nd.single_item) {
      __syncthreads();
      if (tid == 0) {
        s_range[0] = upper_bound_u64(nd.scan, 0, uint64_t(n_items) + 1, tpos) - 1;
        s_range[1] = upper_bound_u64(nd.scan, 0, uint64_t(n_items) + 1, tpos + tn - 1);
      }
      __syncthreads();
      lo = s_range[0];
      hi = s_range[1];
    }
    uint32_t it[R], elem[R];
    int ch[R];
    uint64_t mult[R];
    uint32_t alive = 0;
    // Phase 0: bind the cover elements of the batch.
#pragma unroll
    for (int r = 0; r < R; ++r) {
      uint32_t i = r * kThreads + tid;
      it[r] = 0;
      elem[r] = 0;
      ch[r] = 0;
      mult[r] = 1;
      if (i < tn) {
        uint64_t pos = tpos + i;
        uint64_t j = pos;
        if (!nd.single_item) {
          it[r] = uint32_t(upper_bound_u64(nd.scan, lo, hi, pos) - 1);
          j = pos - nd.scan[it[r]];
        }
        int c = nd.choice[it[r]];
        ch[r] = c;
        const SubDev& S = nd.sub[c];
        const AtomDev& a = atoms[S.atom];
        uint32_t h = item_handle(nd, S, it[r]);
        bool ok = true;
        uint32_t e;
        if (S.last) {
          if (S.lvl == 0 && !a.root_mat) {
            e = uint32_t(j);
            ok = row_passes(a, e);
          } else {
            e = a.perm[a.L[S.lvl].begin[h] + uint32_t(j)];
          }
        } else {
          e = a.L[S.lvl].child_first[h] + uint32_t(j);
          s_newh[c * T + i] = e;
        }
        elem[r] = e;
        if (nd.in_mult) mult[r] = nd.in_mult[it[r]];
        // A cover holding variables bound by earlier nodes only yields the
        // elements that agree with them.
        if (ok && S.bound_mask) {
          for (int jj = 0; jj < S.nv; ++jj) {
            if (!((S.bound_mask >> jj) & 1u)) continue;
            int32_t v = S.last ? __ldg(&a.cols[S.col[jj]][e]) : map_key_value(a, S, e, jj);
            if (v != nd.in_var[S.var[jj]][it[r]]) ok = false;
          }
        }
        if (ok) alive |= 1u << r;
      }
    }
    if (tid == 0) c_iters += tn;
    // Probe phases: one subatom at a time for the whole batch (Fig. 13).
    for (int s = 0; s < nd.n_sub; ++s) {
      if (!nd.dynamic && s == 0) continue;
      const SubDev& S = nd.sub[s];
      const AtomDev& a = atoms[S.atom];
      const LevelDev& L = a.L[S.lvl + 1];
      const uint4* ht = L.ht;
      const uint32_t mask = L.mask;
      const int nk = L.nk;
      uint32_t probing = 0;
      uint64_t kw[R];
      uint32_t par[R];
      // Key sources.  With one cover for every element (static cover) they
      // are the same for the whole batch: an input-tuple array indexed by
      // item, or a base-table column indexed by the cover row.
      const int32_t* ksrc[2] = {nullptr, nullptr};
      int kkind[2] = {2, 2};  // 0: input tuples, 1: cover column, 2: generic
      const uint32_t* hsrc = S.hslot < 0 ? nullptr : nd.in_h[S.hslot];
      if (!nd.dynamic) {
        const SubDev& C = nd.sub[0];
        for (int j = 0; j < S.nv && j < 2; ++j) {
          int u = S.var[j];
          if ((nd.avs_mask >> u) & 1u) {
            kkind[j] = 0;
            ksrc[j] = nd.in_var[u];
          } else if (C.last) {
            kkind[j] = 1;
            ksrc[j] = atoms[C.atom].cols[C.col[nd.vpos[0][u]]];
          }
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        kw[r] = 0;
        par[r] = 0;
        if ((alive >> r & 1u) && ch[r] != s) {
          probing |= 1u << r;
          par[r] = hsrc ? hsrc[it[r]] : 0u;
          int32_t v0 = 0, v1 = 0;
          if (S.nv > 0)
            v0 = kkind[0] == 0   ? ksrc[0][it[r]]
                 : kkind[0] == 1 ? __ldg(ksrc[0] + elem[r])
                                 : load_var(nd, atoms, S.var[0], it[r], ch[r], elem[r]);
          if (S.nv > 1)
            v1 = kkind[1] == 0   ? ksrc[1][it[r]]
                 : kkind[1] == 1 ? __ldg(ksrc[1] + elem[r])
                                 : load_var(nd, atoms, S.var[1], it[r], ch[r], elem[r]);
          kw[r] = pack_key(par[r], nk, v0, v1);
        }
      }
      c_probes += __popc(probing);
      if (L.wide) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (!(probing >> r & 1u)) continue;
          int32_t v0 = S.nv > 0 ? load_var(nd, atoms, S.var[0], it[r], ch[r], elem[r]) : 0;
          int32_t v1 = S.nv > 1 ? load_var(nd, atoms, S.var[1], it[r], ch[r], elem[r]) : 0;
          int32_t v2 = S.nv > 2 ? load_var(nd, atoms, S.var[2], it[r], ch[r], elem[r]) : 0;
          uint32_t e = 0, cnt = 0;
          bool hit = ht_find_wide(ht, mask, make_uint4(par[r], uint32_t(v0), uint32_t(v1),
                                                       uint32_t(v2)), e, cnt);
          if (!hit) {
            alive &= ~(1u << r);
          } else {
            ++c_hits;
            if (S.last) {
              if (nd.track_mult) mult[r] = mul_sat(mult[r], cnt, &res->status);
            } else {
              s_newh[s * T + r * kThreads + tid] = e;
            }
          }
        }
        continue;
      }
      uint4 sl[R];
      uint32_t hh[R];
      const uint32_t* filt = L.filter_on ? L.filter : nullptr;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        hh[r] = 0;
        if ((probing >> r & 1u) && kw[r] != kEmptyKey &&
            !probe_start(ht, mask, filt, L.filter_words, kw[r], hh[r], sl[r]))
          probing &= ~(1u << r), alive &= ~(1u << r);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!(probing >> r & 1u)) continue;
        uint32_t e = 0, cnt = 0;
        bool hit;
        if (kw[r] == kEmptyKey) {
          uint4 sp = __ldg(&ht[mask + 1]);
          e = sp.z;
          cnt = sp.w;
          hit = sp.w != 0;
        } else {
          hit = ht_resolve(ht, mask, kw[r], hh[r], sl[r], e, cnt);
        }
        if (!hit) {
          alive &= ~(1u << r);
        } else {
          ++c_hits;
          if (S.last) {
            if (nd.track_mult) mult[r] = mul_sat(mult[r], cnt, &res->status);
          } else {
            s_newh[s * T + r * kThreads + tid] = e;
          }
        }
      }
    }
    c_surv += __popc(alive);
    // Epilogue.
    if (nd.mode == kModeItems) {
      uint32_t mine = __popc(alive);
      uint32_t inc = warp_incl_scan(mine);
      uint32_t base = 0;
      if (lane_id() == 31 && inc) base = atomicAdd(nd.out_n, inc);
      base = __shfl_sync(0xffffffffu, base, 31) + inc - mine;
      if (base + mine > nd.out_cap && mine) atomicOr(&res->status, kStItemsOverflow);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!(alive >> r & 1u)) continue;
        uint32_t o = base++;
        if (o >= nd.out_cap) continue;
        uint32_t i = r * kThreads + tid;
        for (int k = 0; k < nd.n_out_vars; ++k)
          nd.out_var[k][o] = load_var(nd, atoms, nd.out_var_id[k], it[r], ch[r], elem[r]);
        for (int a = 0; a < FJ_MAX_ATOMS; ++a) {
          if (!nd.out_h[a]) continue;
          int src = nd.out_h_src[a];
          nd.out_h[a][o] = src >= 0 ? s_newh[src * T + i] : nd.in_h[a][it[r]];
        }
        if (nd.out_mult) nd.out_mult[o] = mult[r];
      }
    } else if (nd.mode == kModeAggregate) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!(alive >> r & 1u)) continue;
        uint32_t i = r * kThreads + tid;
        uint64_t m = mult[r];
        for (int t = 0; t < nd.n_tail; ++t) {
          const TailDev& td = nd.tail[t];
          const AtomDev& ta = atoms[td.atom];
          uint32_t h = td.hsrc >= 0 ? s_newh[td.hsrc * T + i] : nd.in_h[td.atom][it[r]];
          m = mul_sat(m, ta.L[td.lvl].count[h], &res->status);
        }
        if (m == 0) continue;
        unsigned long long before = my_count;
        my_count += m;
        if (my_count < before) atomicOr(&res->status, kStCountOverflow);
        any_out = true;
        for (int k = 0; k < nd.n_min; ++k)
          atomicMin(&s_min[nd.min_idx[k]],
                    load_var(nd, atoms, nd.min_var[k], it[r], ch[r], elem[r]));
        for (int t = 0; t < nd.n_tail; ++t) {
          const TailDev& td = nd.tail[t];
          if (!td.n_min) continue;
          const AtomDev& ta = atoms[td.atom];
          uint32_t h = td.hsrc >= 0 ? s_newh[td.hsrc * T + i] : nd.in_h[td.atom][it[r]];
          uint32_t bg = ta.L[td.lvl].begin[h], cn = ta.L[td.lvl].count[h];
          for (int k = 0; k < td.n_min; ++k) {
            const int32_t* col = ta.cols[td.min_col[k]];
            int32_t lo_v = INT32_MAX;
            for (uint32_t q = 0; q < cn; ++q) lo_v = min(lo_v, col[ta.perm[bg + q]]);
            atomicMin(&s_min[td.min_idx[k]], lo_v);
          }
        }
      }
    } else if (nd.mode == kModeFactorized) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t i = r * kThreads + tid;
        factor_emit(
            nd, atoms, res, alive >> r & 1u, mult[r],
            [&](int t) {
              const TailDev& td = nd.tail[t];
              return td.hsrc >= 0 ? s_newh[td.hsrc * T + i] : nd.in_h[td.atom][it[r]];
            },
            [&](int v) { return load_var(nd, atoms, v, it[r], ch[r], elem[r]); }, my_count);
      }
    } else {  // kModeMaterialize
      uint64_t tot = 0;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (alive >> r & 1u) tot += mult[r];
      uint64_t inc = warp_incl_scan<unsigned long long>(tot);
      uint64_t base = 0;
      if (lane_id() == 31 && inc) base = atomicAdd(&res->n_out, (unsigned long long)inc);
      base = __shfl_sync(0xffffffffu, (unsigned long long)base, 31) + inc - tot;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!(alive >> r & 1u)) continue;
        for (uint64_t q = 0; q < mult[r]; ++q) {
          uint64_t row = base++;
          if (row >= nd.out_rows_cap) {
            atomicOr(&res->status, kStOutputOverflow);
            continue;
          }
          for (int h = 0; h < nd.n_head; ++h)
            nd.out_tuples[row * nd.n_head + h] =
                load_var(nd, atoms, nd.head_var[h], it[r], ch[r], elem[r]);
        }
      }
    }
  }
  // Block totals.
  __syncthreads();
  if (nd.mode == kModeAggregate || nd.mode == kModeFactorized) {
    unsigned long long tot = block_sum<unsigned long long>(my_count, s_red);
    int any = __syncthreads_or(any_out);
    if (tid == 0 && tot) {
      unsigned long long old = atomicAdd(&res->count, tot);
      if (old + tot < old) atomicOr(&res->status, kStCountOverflow);
    }
    // Every MIN slot is flushed (a slot still at INT32_MAX leaves the result
    // unchanged); validity of the MINs is COUNT > 0.
    if (nd.mode == kModeAggregate && any && tid < FJ_MAX_VARS)
      atomicMin(&res->mins[tid], s_min[tid]);
  }
  unsigned long long v;
  v = block_sum<unsigned long long>(c_iters, s_red);
  if (tid == 0 && v) atomicAdd(&res->ctr[FJ_CTR_COVER_ITERS], v);
  v = block_sum<unsigned long long>(c_probes, s_red);
  if (tid == 0 && v) atomicAdd(&res->ctr[FJ_CTR_PROBES], v);
  v = block_sum<unsigned long long>(c_hits, s_red);
  if (tid == 0 && v) atomicAdd(&res->ctr[FJ_CTR_PROBE_HITS], v);
  v = block_sum<unsigned long long>(c_surv, s_red);
  if (tid == 0 && v) atomicAdd(&res->ctr[FJ_CTR_SURVIVORS], v);
}

__device__ __forceinline__ int32_t src_value(const VarSrc& v, uint32_t it, uint32_t elem) {
  switch (v.kind) {
    case kSrcItem: return v.col[it];
    case kSrcRow: return __ldg(v.col + elem);
    case kSrcKey: return key_value(v.key[elem], v.nk, v.pos);
    default: return __ldg(v.col + v.perm[v.begin[elem]]);
  }
}

// One probe phase over up to R batch elements held by this thread: gather
// the keys of all live elements, issue all their first hash-slot loads, then
// resolve.  `live` bit r marks element r; returns the elements that hit.
// Hits on a non-last level leave the entry in newh_out[r]; hits on a last
// level multiply mult[r] by the vector length.
template <int R>
__device__ __forceinline__ uint32_t probe_batch(const NodeDev& nd, const ProbeDev& Pd,
                                                uint32_t mask, uint32_t live,
                                                const uint32_t (&it)[R],
                                                const uint32_t (&elem)[R], uint64_t (&mult)[R],
                                                uint32_t (&newh_out)[R], uint32_t* status) {
  uint64_t kw[R];
  uint32_t par[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    kw[r] = 0;
    par[r] = 0;
    newh_out[r] = 0;
    if (live >> r & 1u) {
      par[r] = Pd.hsrc ? Pd.hsrc[it[r]] : 0u;
      int32_t v0 = Pd.nv > 0 ? src_value(nd.src[Pd.var[0]], it[r], elem[r]) : 0;
      int32_t v1 = Pd.nv > 1 ? src_value(nd.src[Pd.var[1]], it[r], elem[r]) : 0;
      kw[r] = pack_key(par[r], Pd.nk, v0, v1);
    }
  }
  if (Pd.wide) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!(live >> r & 1u)) continue;
      int32_t v0 = Pd.nv > 0 ? src_value(nd.src[Pd.var[0]], it[r], elem[r]) : 0;
      int32_t v1 = Pd.nv > 1 ? src_value(nd.src[Pd.var[1]], it[r], elem[r]) : 0;
      int32_t v2 = Pd.nv > 2 ? src_value(nd.src[Pd.var[2]], it[r], elem[r]) : 0;
      uint32_t e = 0, cnt = 0;
      bool hit = ht_find_wide(Pd.ht, mask,
                              make_uint4(par[r], uint32_t(v0), uint32_t(v1), uint32_t(v2)), e,
                              cnt);
      if (!hit) {
        live &= ~(1u << r);
      } else if (Pd.last) {
        if (nd.track_mult) mult[r] = mul_sat(mult[r], cnt, status);
      } else {
        newh_out[r] = e;
      }
    }
    return live;
  }
  uint4 sl[R];
  uint32_t hh[R];
  const uint32_t* filt = Pd.filter && *Pd.filter_on ? Pd.filter : nullptr;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    hh[r] = 0;
    if ((live >> r & 1u) && kw[r] != kEmptyKey &&
        !probe_start(Pd.ht, mask, filt, Pd.filter_words, kw[r], hh[r], sl[r]))
      live &= ~(1u << r);
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (!(live >> r & 1u)) continue;
    uint32_t e = 0, cnt = 0;
    bool hit;
    if (kw[r] == kEmptyKey) {
      uint4 sp = __ldg(&Pd.ht[mask + 1]);
      e = sp.z;
      cnt = sp.w;
      hit = sp.w != 0;
    } else {
      hit = ht_resolve(Pd.ht, mask, kw[r], hh[r], sl[r], e, cnt);
    }
    if (!hit) {
      live &= ~(1u << r);
    } else if (Pd.last) {
      if (nd.track_mult) mult[r] = mul_sat(mult[r], cnt, status);
    } else {
      newh_out[r] = e;
    }
  }
  return live;
}

// Append batch slot i to a shared list when keep is set (warp-aggregated).
__device__ __forceinline__ void list_append(bool keep, uint32_t i, uint16_t* list, uint32_t* cnt) {
  uint32_t m = __ballot_sync(0xffffffffu, keep);
  if (!m) return;
  uint32_t leader = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane_id() == leader) base = atomicAdd(cnt, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (keep) list[base + __popc(m & lanemask_lt())] = uint16_t(i);
}

// Expansion of a node whose cover is fixed (the static cover, or the only
// cover): every variable source and every probed hash level is resolved on
// the host into the node descriptor.  Batches of T = R * 256 cover elements;
// the first probe runs over the whole batch in registers, R independent
// gathers per thread; its survivors are compacted into a shared list and
// the remaining probes and the epilogue run over that list only.
template <int R>
__global__ void __launch_bounds__(kThreads, expand_min_blocks(R))
    k_expand_static(const __grid_constant__ NodeDev nd, AtomDev* atoms, ResultDev* res) {
  // A root build whose bounded wait ran out left its levels unbuilt.
  if (__syncthreads_or(threadIdx.x == 0 && (res->status & kStTimeout))) return;
  constexpr int T = R * kThreads;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  uint64_t* s_mult = reinterpret_cast<uint64_t*>(smem_raw);
  uint32_t* s_it = reinterpret_cast<uint32_t*>(s_mult + T);
  uint32_t* s_elem = s_it + T;
  uint32_t* s_newh = s_elem + T;  // [n_sub][T]
  uint16_t* s_list0 = reinterpret_cast<uint16_t*>(s_newh + size_t(nd.n_sub) * T);
  uint16_t* s_list1 = s_list0 + T;
  __shared__ uint32_t s_mask[FJ_MAX_SUB];
  __shared__ uint32_t s_root_mat;
  __shared__ uint32_t s_cnt[2];
  __shared__ uint64_t s_range[2];
  __shared__ unsigned long long s_red[33];
  __shared__ int32_t s_min[FJ_MAX_VARS];
  const uint32_t tid = threadIdx.x;
  if (tid < uint32_t(nd.n_probe)) s_mask[tid] = *nd.probe[tid].mask;
  if (tid == 0) s_root_mat = *nd.cover_root_mat;
  if (tid < FJ_MAX_VARS) s_min[tid] = INT32_MAX;
  unsigned long long my_count = 0, c_iters = 0, c_probes = 0, c_hits = 0, c_surv = 0;
  bool any_out = false;
  uint32_t n_items = nd.single_item ? 1u : *nd.n_items;
  uint64_t end = nd.chunk_end;
  if (!nd.single_item) end = min(end, nd.scan[n_items]);
  if (nd.check_total && !nd.single_item && blockIdx.x == 0 && tid == 0 &&
      nd.scan[n_items] > nd.chunk_end)
    atomicOr(&res->status, kStItemsOverflow);
  const SubDev& C = nd.sub[0];
  const AtomDev& ca = atoms[C.atom];
  __syncthreads();
  const bool ident = C.last && C.lvl == 0 && !s_root_mat;
  const int n_preds = ident ? ca.n_preds : 0;

  for (uint64_t tile = blockIdx.x;; tile += gridDim.x) {
    uint64_t tpos = nd.chunk_begin + tile * uint64_t(T);
    if (tpos >= end) break;
    uint32_t tn = uint32_t(min(uint64_t(T), end - tpos));
    __syncthreads();  // the previous batch's lists are consumed
    if (tid == 0) {
      s_cnt[0] = 0;
      s_cnt[1] = 0;
      if (!nd.single_item) {
        s_range[0] = upper_bound_u64(nd.scan, 0, uint64_t(n_items) + 1, tpos) - 1;
        s_range[1] = upper_bound_u64(nd.scan, 0, uint64_t(n_items) + 1, tpos + tn - 1);
      }
    }
    __syncthreads();
    uint64_t lo = 0, hi = 1;
    if (!nd.single_item) {
      lo = s_range[0];
      hi = s_range[1];
    }
    uint32_t it[R], elem[R], nh[R];
    uint64_t mult[R];
    uint32_t alive = 0;
    // Phase 0: bind the cover elements of the batch.
#pragma unroll
    for (int r = 0; r < R; ++r) {
      uint32_t i = r * kThreads + tid;
      it[r] = 0;
      elem[r] = 0;
      mult[r] = 1;
      if (i < tn) {
        uint64_t pos = tpos + i;
        uint64_t j = pos;
        if (!nd.single_item) {
          it[r] = uint32_t(upper_bound_u64(nd.scan, lo, hi, pos) - 1);
          j = pos - nd.scan[it[r]];
        }
        bool ok = true;
        uint32_t e;
        if (ident) {
          e = uint32_t(j);
          if (n_preds) ok = row_passes(ca, e);
        } else {
          uint32_t h = nd.cover_hsrc ? nd.cover_hsrc[it[r]] : 0u;
          if (C.last) {
            e = nd.cover_perm[nd.cover_begin[h] + uint32_t(j)];
          } else {
            e = nd.cover_first[h] + uint32_t(j);
            s_newh[i] = e;
          }
        }
        elem[r] = e;
        if (nd.in_mult) mult[r] = nd.in_mult[it[r]];
        if (ok && C.bound_mask) {
          for (int jj = 0; jj < C.nv; ++jj) {
            if (!((C.bound_mask >> jj) & 1u)) continue;
            int32_t v = C.last ? __ldg(&ca.cols[C.col[jj]][e]) : map_key_value(ca, C, e, jj);
            if (v != nd.in_var[C.var[jj]][it[r]]) ok = false;
          }
        }
        if (ok) alive |= 1u << r;
      }
    }
    if (tid == 0) c_iters += tn;
    // First probe over the whole batch, in registers.
    if (nd.n_probe > 0) {
      const ProbeDev& Pd = nd.probe[0];
      c_probes += __popc(alive);
      alive = probe_batch<R>(nd, Pd, s_mask[0], alive, it, elem, mult, nh, &res->status);
      c_hits += __popc(alive);
      if (!Pd.last)
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (alive >> r & 1u) s_newh[Pd.sub * T + r * kThreads + tid] = nh[r];
    }
    // Compact the survivors.
#pragma unroll
    for (int r = 0; r < R; ++r) {
      uint32_t i = r * kThreads + tid;
      bool keep = alive >> r & 1u;
      if (keep) {
        s_it[i] = it[r];
        s_elem[i] = elem[r];
        s_mult[i] = mult[r];
      }
      list_append(keep, i, s_list0, &s_cnt[0]);
    }
    __syncthreads();
    int cur = 0;
    // Remaining probes over the survivor list.
    for (int p = 1; p < nd.n_probe; ++p) {
      const ProbeDev& Pd = nd.probe[p];
      uint16_t* lin = cur ? s_list1 : s_list0;
      uint16_t* lout = cur ? s_list0 : s_list1;
      uint32_t n = s_cnt[cur];
      uint32_t live = 0, slot[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        uint32_t q = r * kThreads + tid;
        slot[r] = 0;
        if (q < n) {
          uint32_t i = lin[q];
          slot[r] = i;
          it[r] = s_it[i];
          elem[r] = s_elem[i];
          mult[r] = s_mult[i];
          live |= 1u << r;
        }
      }
      c_probes += __popc(live);
      uint32_t hit = probe_batch<R>(nd, Pd, s_mask[p], live, it, elem, mult, nh, &res->status);
      c_hits += __popc(hit);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        bool keep = hit >> r & 1u;
        if (keep) {
          if (Pd.last)
            s_mult[slot[r]] = mult[r];
          else
            s_newh[Pd.sub * T + slot[r]] = nh[r];
        }
        list_append(keep, slot[r], lout, &s_cnt[cur ^ 1]);
      }
      __syncthreads();
      if (tid == 0) s_cnt[cur] = 0;
      cur ^= 1;
      __syncthreads();
    }
    // Epilogue over the final list.
    const uint16_t* lfin = cur ? s_list1 : s_list0;
    uint32_t n = s_cnt[cur];
    uint32_t live = 0, slot[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      uint32_t q = r * kThreads + tid;
      slot[r] = 0;
      if (q < n) {
        uint32_t i = lfin[q];
        slot[r] = i;
        it[r] = s_it[i];
        elem[r] = s_elem[i];
        mult[r] = s_mult[i];
        live |= 1u << r;
      }
    }
    c_surv += __popc(live);
    if (nd.mode == kModeItems) {
      uint32_t mine = __popc(live);
      uint32_t inc = warp_incl_scan(mine);
      uint32_t base = 0;
      if (lane_id() == 31 && inc) base = atomicAdd(nd.out_n, inc);
      base = __shfl_sync(0xffffffffu, base, 31) + inc - mine;
      if (base + mine > nd.out_cap && mine) atomicOr(&res->status, kStItemsOverflow);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!(live >> r & 1u)) continue;
        uint32_t o = base++;
        if (o >= nd.out_cap) continue;
        uint32_t i = slot[r];
        for (int k = 0; k < nd.n_out_vars; ++k)
          nd.out_var[k][o] = src_value(nd.src[nd.out_var_id[k]], it[r], elem[r]);
        for (int a = 0; a < FJ_MAX_ATOMS; ++a) {
          if (!nd.out_h[a]) continue;
          int src = nd.out_h_src[a];
          nd.out_h[a][o] = src >= 0 ? s_newh[src * T + i] : nd.in_h[a][it[r]];
        }
        if (nd.out_mult) nd.out_mult[o] = mult[r];
      }
    } else if (nd.mode == kModeAggregate) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!(live >> r & 1u)) continue;
        uint32_t i = slot[r];
        uint64_t m = mult[r];
        for (int t = 0; t < nd.n_tail; ++t) {
          const TailDev& td = nd.tail[t];
          const AtomDev& ta = atoms[td.atom];
          uint32_t h = td.hsrc >= 0 ? s_newh[td.hsrc * T + i] : nd.in_h[td.atom][it[r]];
          m = mul_sat(m, ta.L[td.lvl].count[h], &res->status);
        }
        if (m == 0) continue;
        unsigned long long before = my_count;
        my_count += m;
        if (my_count < before) atomicOr(&res->status, kStCountOverflow);
        any_out = true;
        for (int k = 0; k < nd.n_min; ++k)
          atomicMin(&s_min[nd.min_idx[k]], src_value(nd.src[nd.min_var[k]], it[r], elem[r]));
        for (int t = 0; t < nd.n_tail; ++t) {
          const TailDev& td = nd.tail[t];
          if (!td.n_min) continue;
          const AtomDev& ta = atoms[td.atom];
          uint32_t h = td.hsrc >= 0 ? s_newh[td.hsrc * T + i] : nd.in_h[td.atom][it[r]];
          uint32_t bg = ta.L[td.lvl].begin[h], cn = ta.L[td.lvl].count[h];
          for (int k = 0; k < td.n_min; ++k) {
            const int32_t* col = ta.cols[td.min_col[k]];
            int32_t lo_v = INT32_MAX;
            for (uint32_t q = 0; q < cn; ++q) lo_v = min(lo_v, col[ta.perm[bg + q]]);
            atomicMin(&s_min[td.min_idx[k]], lo_v);
          }
        }
      }
    } else if (nd.mode == kModeFactorized) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t i = slot[r];
        factor_emit(
            nd, atoms, res, live >> r & 1u, mult[r],
            [&](int t) {
              const TailDev& td = nd.tail[t];
              return td.hsrc >= 0 ? s_newh[td.hsrc * T + i] : nd.in_h[td.atom][it[r]];
            },
            [&](int v) { return src_value(nd.src[v], it[r], elem[r]); }, my_count);
      }
    } else {  // kModeMaterialize
      uint64_t tot = 0;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (live >> r & 1u) tot += mult[r];
      uint64_t inc = warp_incl_scan<unsigned long long>(tot);
      uint64_t base = 0;
      if (lane_id() == 31 && inc) base = atomicAdd(&res->n_out, (unsigned long long)inc);
      base = __shfl_sync(0xffffffffu, (unsigned long long)base, 31) + inc - tot;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!(live >> r & 1u)) continue;
        for (uint64_t q = 0; q < mult[r]; ++q) {
          uint64_t row = base++;
          if (row >= nd.out_rows_cap) {
            atomicOr(&res->status, kStOutputOverflow);
            continue;
          }
          for (int h = 0; h < nd.n_head; ++h)
            nd.out_tuples[row * nd.n_head + h] = src_value(nd.src[nd.head_var[h]], it[r], elem[r]);
        }
      }
    }
  }
  __syncthreads();
  if (nd.mode == kModeAggregate || nd.mode == kModeFactorized) {
    unsigned long long tot = block_sum<unsigned long long>(my_count, s_red);
    int any = __syncthreads_or(any_out);
    if (tid == 0 && tot) {
      unsigned long long old = atomicAdd(&res->count, tot);
      if (old + tot < old) atomicOr(&res->status, kStCountOverflow);
    }
    if (nd.mode == kModeAggregate && any && tid < FJ_MAX_VARS)
      atomicMin(&res->mins[tid], s_min[tid]);
  }
  unsigned long long v;
  v = block_sum<unsigned long long>(c_iters, s_red);
  if (tid == 0 && v) atomicAdd(&res->ctr[FJ_CTR_COVER_ITERS], v);
  v = block_sum<unsigned long long>(c_probes, s_red);
  if (tid == 0 && v) atomicAdd(&res->ctr[FJ_CTR_PROBES], v);
  v = block_sum<unsigned long long>(c_hits, s_red);
  if (tid == 0 && v) atomicAdd(&res->ctr[FJ_CTR_PROBE_HITS], v);
  v = block_sum<unsigned long long>(c_surv, s_red);
  if (tid == 0 && v) atomicAdd(&res->ctr[FJ_CTR_SURVIVORS], v);
}

// Reset the COLT state of every atom (nothing built) and/or the result.
__global__ void k_reset(AtomDev* atoms, int n_atoms, ResultDev* res, int do_atoms,
                        unsigned int* zero, int n_zero) {
  int a = blockIdx.x;
  // Words that must start at zero (the root-build barrier and counters,
  // which leave themselves at zero only after a complete launch).
  if (a == 0 && zero)
    for (int i = threadIdx.x; i < n_zero; i += blockDim.x) zero[i] = 0;
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
    R.fill[0] = 0;
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
      L.filter_on = 0;
      L.exact = 0;
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
