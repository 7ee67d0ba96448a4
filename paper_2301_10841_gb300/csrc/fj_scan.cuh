// Node 0 of a plan whose cover is iterated straight from its base table (the
// COLT base-table case of Section 4.2: nothing is built for the cover), run
// as the batch-at-a-time probing of Section 4.3 with the whole chunk of
// cover rows as the batch.  This is node 0 of every plan produced by
// binary2fj, and the whole probe phase of a factored star join.
//
// Two kernels, each lean and fully occupied:
//  1. k_scan_first: stream the cover's rows (16-byte loads where aligned),
//     apply its selections, probe the first subatom -- Bloom filter first,
//     then the hash slot -- and append the survivors (row, entry) to a
//     buffer (one global atomic per block iteration);
//  2. k_scan_rest: take every survivor through the remaining probes, R per
//     thread with their gathers in flight together, then through the
//     node's epilogue (aggregate, partial tuples for node 1, or output).
#pragma once

#include "fj_exec.cuh"

namespace fj {

// One probe of node 0, resolved on the host: key columns of the cover row
// (node 0 binds every variable from the cover), the hash level and its
// Bloom filter.
struct ScanProbe {
  const int32_t* kcol[3];
  int nk;
  int wide;
  int last;
  int sub;                    // subatom index in the node
  const uint4* ht;
  const uint32_t* mask;       // device-side
  const uint32_t* filter;
  uint32_t filter_words;
  const uint32_t* filter_on;  // device-side
  const uint32_t* bitmap;     // exact key bitmap of a one-column root level (or null)
  const uint32_t* exact;      // device-side: the bitmap holds every key
};

// Survivor buffer: structure of arrays, device-side count.
struct ScanBuf {
  uint32_t* row;
  uint32_t* h[FJ_MAX_SUB];  // entry reached by probe p (non-last probes)
  uint64_t* mult;           // null when no probe ends an atom at a leaf
  uint32_t* n;
  uint32_t* src;            // k_scan_fused: position after the first probe
};

struct ScanDev {
  int n_probe;
  ScanProbe probe[FJ_MAX_SUB];
  int n_preds;
  const int32_t* pred_col[FJ_MAX_PREDS];
  int pred_op[FJ_MAX_PREDS];
  int32_t pred_val[FJ_MAX_PREDS];
  int k1;      // the first probe is one key column at the root, narrow level
  int vec_ok;  // its key column is 16-byte aligned (chunks start at 4k rows)
  ScanBuf buf[1];
  uint32_t cap;
  uint32_t spin;  // mbarrier waits before a copy counts as lost (0: default)
};

__device__ __forceinline__ bool scan_pred(const ScanDev& sc, uint32_t row) {
  for (int p = 0; p < sc.n_preds; ++p) {
    int32_t v = __ldg(sc.pred_col[p] + row);
    int32_t c = sc.pred_val[p];
    bool ok;
    switch (sc.pred_op[p]) {
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

// Root-level, one-column key: the key word is the value itself (parent 0),
// so the hash is one finalizer round away from it.
__device__ __forceinline__ uint32_t hash_root1(int32_t k) {
  constexpr uint32_t kC = []() {
    uint32_t h = 0x9e3779b9u;
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
  }();
  return fmix32(uint32_t(k) ^ kC);
}

// Probe R elements (rows) of one thread against probe P: keys from the
// cover columns, Bloom filter, all first slot loads, then resolve.  `live`
// bit r marks element r; returns the hits with entries in e[] and leaf
// lengths multiplied into mult[] (when tracked).
template <int R>
__device__ __forceinline__ uint32_t scan_probe_rows(const ScanProbe& P, uint32_t mask,
                                                    const uint32_t* filt, uint32_t live,
                                                    const uint32_t (&row)[R], uint32_t (&e)[R],
                                                    uint64_t* mult, uint32_t* status) {
  if (P.wide) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      e[r] = 0;
      if (!(live >> r & 1u)) continue;
      uint4 k = make_uint4(0u, P.nk > 0 ? uint32_t(__ldg(P.kcol[0] + row[r])) : 0u,
                           P.nk > 1 ? uint32_t(__ldg(P.kcol[1] + row[r])) : 0u,
                           P.nk > 2 ? uint32_t(__ldg(P.kcol[2] + row[r])) : 0u);
      uint32_t cnt = 0;
      if (!ht_find_wide(P.ht, mask, k, e[r], cnt))
        live &= ~(1u << r);
      else if (P.last && mult)
        mult[r] = mul_sat(mult[r], cnt, status);
    }
    return live;
  }
  uint64_t kw[R];
  uint32_t hh[R];
  uint4 sl[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    e[r] = 0;
    kw[r] = 0;
    hh[r] = 0;
    if (live >> r & 1u) {
      int32_t v0 = P.nk > 0 ? __ldg(P.kcol[0] + row[r]) : 0;
      int32_t v1 = P.nk > 1 ? __ldg(P.kcol[1] + row[r]) : 0;
      kw[r] = pack_key(0u, P.nk, v0, v1);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    if ((live >> r & 1u) && kw[r] != kEmptyKey &&
        !probe_start(P.ht, mask, filt, P.filter_words, kw[r], hh[r], sl[r]))
      live &= ~(1u << r);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (!(live >> r & 1u)) continue;
    uint32_t cnt = 0;
    bool hit;
    if (kw[r] == kEmptyKey) {
      uint4 sp = __ldg(&P.ht[mask + 1]);
      e[r] = sp.z;
      cnt = sp.w;
      hit = sp.w != 0;
    } else {
      hit = ht_resolve(P.ht, mask, kw[r], hh[r], sl[r], e[r], cnt);
    }
    if (!hit)
      live &= ~(1u << r);
    else if (P.last && mult)
      mult[r] = mul_sat(mult[r], cnt, status);
  }
  return live;
}

// Block-aggregated append: returns this thread's first output position for
// its `mine` elements (every thread of the block must call it).
__device__ __forceinline__ uint32_t block_append(uint32_t mine, uint32_t* counter,
                                                 uint32_t* s_cnt, uint32_t* s_base) {
  uint32_t inc = warp_incl_scan(mine);
  uint32_t wtot = __shfl_sync(0xffffffffu, inc, 31);
  uint32_t woff = 0;
  if (lane_id() == 31 && wtot) woff = atomicAdd(s_cnt, wtot);
  woff = __shfl_sync(0xffffffffu, woff, 31);
  __syncthreads();
  if (threadIdx.x == 0) {
    *s_base = *s_cnt ? atomicAdd(counter, *s_cnt) : 0u;
    *s_cnt = 0;
  }
  __syncthreads();
  return *s_base + woff + inc - mine;
}

// Step 1: stream the cover rows of [chunk_begin, chunk_end), selections and
// the first probe (if any); survivors to buf[0].
template <int R>
__global__ void __launch_bounds__(kThreads) k_scan_first(const __grid_constant__ NodeDev nd,
                                                         const __grid_constant__ ScanDev sc,
                                                         ResultDev* res) {
  // A root build whose bounded wait ran out left its levels unbuilt.
  if (__syncthreads_or(threadIdx.x == 0 && (res->status & kStTimeout))) return;
  static_assert(R % 4 == 0, "rows come in 16-byte groups");
  __shared__ uint32_t s_cnt, s_base;
  __shared__ uint32_t s_mask, s_fon;
  __shared__ unsigned long long s_red[33];
  if (threadIdx.x == 0) {
    s_cnt = 0;
    s_mask = sc.n_probe ? *sc.probe[0].mask : 0u;
    s_fon = sc.n_probe && sc.probe[0].filter ? *sc.probe[0].filter_on : 0u;
  }
  __syncthreads();
  const uint32_t mask = s_mask;
  const ScanProbe& P = sc.probe[0];
  const uint32_t* filt = s_fon ? P.filter : nullptr;
  const ScanBuf& out = sc.buf[0];
  const uint64_t begin = nd.chunk_begin, end = nd.chunk_end;
  constexpr uint64_t BT = uint64_t(R) * kThreads;  // rows per block iteration
  unsigned long long c_probe = 0, c_hit = 0;
  for (uint64_t b0 = begin + uint64_t(blockIdx.x) * BT; b0 < end;
       b0 += uint64_t(gridDim.x) * BT) {
    uint32_t row[R], e[R];
    uint64_t mult[R];
    uint32_t live = 0;
    // Thread t owns rows 4t..4t+3 of each 1024-row quarter of the block's
    // rows, so each 16-byte load of a warp is contiguous.
#pragma unroll
    for (int q = 0; q < R / 4; ++q) {
      uint64_t base = b0 + uint64_t(q) * 4 * kThreads + 4 * threadIdx.x;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        row[q * 4 + j] = uint32_t(base + j);
        mult[q * 4 + j] = 1;
        e[q * 4 + j] = 0;
        if (base + j < end) live |= 1u << (q * 4 + j);
      }
    }
    if (sc.n_preds) {
#pragma unroll
      for (int r = 0; r < R; ++r)
        if ((live >> r & 1u) && !scan_pred(sc, row[r])) live &= ~(1u << r);
    }
    if (sc.n_probe) {
      c_probe += __popc(live);
      if (sc.k1) {
        // One key column at the root: 16-byte key loads, one hash per row.
        int32_t k[R];
        uint32_t hv[R];
        uint4 sl[R];
#pragma unroll
        for (int q = 0; q < R / 4; ++q) {
          uint64_t base = b0 + uint64_t(q) * 4 * kThreads + 4 * threadIdx.x;
          if (sc.vec_ok && base + 4 <= end) {
            int4 v = __ldg(reinterpret_cast<const int4*>(P.kcol[0] + base));
            k[q * 4 + 0] = v.x;
            k[q * 4 + 1] = v.y;
            k[q * 4 + 2] = v.z;
            k[q * 4 + 3] = v.w;
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
              k[q * 4 + j] = base + j < end ? __ldg(P.kcol[0] + base + j) : 0;
          }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
          hv[r] = hash_root1(k[r]);
          if (filt && (live >> r & 1u) &&
              bloom_rejects(filt, P.filter_words, filter_hash_root1(k[r])))
            live &= ~(1u << r);
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (live >> r & 1u) sl[r] = __ldg(&P.ht[hv[r] & mask]);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (!(live >> r & 1u)) continue;
          uint32_t h = hv[r] & mask;
          uint4 s = sl[r];
          bool hit = false;
          for (uint32_t it = 0; it <= mask; ++it) {
            if (s.x == uint32_t(k[r]) && s.y == 0u) {
              hit = true;
              break;
            }
            if (s.x == kNone && s.y == kNone) break;
            h = (h + 1) & mask;
            s = __ldg(&P.ht[h]);
          }
          if (!hit) {
            live &= ~(1u << r);
          } else {
            e[r] = s.z;
            if (P.last && out.mult) mult[r] = mul_sat(mult[r], s.w, &res->status);
          }
        }
      } else {
        live = scan_probe_rows<R>(P, mask, filt, live, row, e, out.mult ? mult : nullptr,
                                  &res->status);
      }
      c_hit += __popc(live);
    }
    uint32_t pos = block_append(__popc(live), out.n, &s_cnt, &s_base);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!(live >> r & 1u)) continue;
      if (pos < sc.cap) {
        out.row[pos] = row[r];
        if (sc.n_probe && !P.last) out.h[0][pos] = e[r];
        if (out.mult) out.mult[pos] = mult[r];
      } else {
        atomicOr(&res->status, kStItemsOverflow);
      }
      ++pos;
    }
  }
  unsigned long long v = block_sum<unsigned long long>(c_probe, s_red);
  if (threadIdx.x == 0 && v) atomicAdd(&res->ctr[FJ_CTR_PROBES], v);
  v = block_sum<unsigned long long>(c_hit, s_red);
  if (threadIdx.x == 0 && v) atomicAdd(&res->ctr[FJ_CTR_PROBE_HITS], v);
  if (blockIdx.x == 0 && threadIdx.x == 0 && end > begin)
    atomicAdd(&res->ctr[FJ_CTR_COVER_ITERS], (unsigned long long)(end - begin));
}

// Entry of subatom `sub` for buffered element i.
__device__ __forceinline__ uint32_t scan_handle(const ScanDev& sc, const ScanBuf& b, int sub,
                                                uint32_t i) {
  for (int p = 0; p < sc.n_probe; ++p)
    if (sc.probe[p].sub == sub && !sc.probe[p].last) return b.h[p][i];
  return 0u;
}

// Remaining probes 1..n_probe-1 for R survivors of one thread, in plan
// order; each probe's entries are kept beside the survivor (b.h[p]) for the
// epilogue.  Returns the survivors that hit every probe.
template <int R>
__device__ __forceinline__ uint32_t scan_rest_probes(const ScanDev& sc, const ScanBuf& b,
                                                     const uint32_t* s_mask,
                                                     const uint32_t* s_fon, uint32_t live,
                                                     const uint32_t (&idx)[R],
                                                     const uint32_t (&row)[R], uint32_t (&e)[R],
                                                     uint64_t (&mult)[R], uint32_t* status,
                                                     unsigned long long& c_probe,
                                                     unsigned long long& c_hit) {
  for (int p = 1; p < sc.n_probe && live; ++p) {
    const ScanProbe& P = sc.probe[p];
    c_probe += __popc(live);
    live = scan_probe_rows<R>(P, s_mask[p], s_fon[p] ? P.filter : nullptr, live, row, e,
                              b.mult ? mult : nullptr, status);
    c_hit += __popc(live);
    if (!P.last)
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (live >> r & 1u) b.h[p][idx[r]] = e[r];
  }
  return live;
}

// Node 0's epilogue for R survivors of one thread: partial tuples for node 1,
// aggregation (COUNT, MIN, trailing product nodes), or output tuples.  The
// partial tuples are appended block-wide (every thread of the block calls
// this the same number of times) or, with WARP_APPEND, warp-wide (every lane
// of the warp does).
template <int R, bool WARP_APPEND = false>
__device__ __forceinline__ void scan_epilogue(const NodeDev& nd, const ScanDev& sc,
                                              const ScanBuf& b, AtomDev* atoms, ResultDev* res,
                                              const uint32_t (&idx)[R], const uint32_t (&row)[R],
                                              const uint64_t (&mult)[R], uint32_t live,
                                              uint32_t* s_cnt, uint32_t* s_base, int32_t* s_min,
                                              unsigned long long& my_count, bool& any) {
  if (nd.mode == kModeItems) {
    uint32_t pos;
    if (WARP_APPEND) {
      const uint32_t mine = __popc(live);
      const uint32_t inc = warp_incl_scan(mine);
      uint32_t b0 = 0;
      if (lane_id() == 31 && inc) b0 = atomicAdd(nd.out_n, inc);
      pos = __shfl_sync(0xffffffffu, b0, 31) + inc - mine;
    } else {
      pos = block_append(__popc(live), nd.out_n, s_cnt, s_base);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!(live >> r & 1u)) continue;
      uint32_t o = pos++;
      if (o >= nd.out_cap) {
        atomicOr(&res->status, kStItemsOverflow);
        continue;
      }
      for (int k = 0; k < nd.n_out_vars; ++k)
        nd.out_var[k][o] = src_value(nd.src[nd.out_var_id[k]], 0, row[r]);
      for (int a = 0; a < FJ_MAX_ATOMS; ++a)
        if (nd.out_h[a]) nd.out_h[a][o] = scan_handle(sc, b, nd.out_h_src[a], idx[r]);
      if (nd.out_mult) nd.out_mult[o] = mult[r];
    }
  } else if (nd.mode == kModeAggregate) {
    constexpr int MT = 4;  // tails whose lookups are issued together
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!(live >> r & 1u)) continue;
      uint64_t m = mult[r];
      const int nt = nd.n_tail;
      uint32_t th[MT], cn[MT], pr[MT];
      if (nt <= MT) {
        // Each tail's vector: handle, then length and first offset, then
        // the first row, every level of lookups in flight for all tails.
#pragma unroll
        for (int t = 0; t < MT; ++t)
          th[t] = t < nt ? scan_handle(sc, b, nd.tail[t].hsrc, idx[r]) : 0u;
        uint32_t bg[MT];
#pragma unroll
        for (int t = 0; t < MT; ++t) {
          cn[t] = 1;
          bg[t] = 0;
          if (t < nt) {
            const LevelDev& L = atoms[nd.tail[t].atom].L[nd.tail[t].lvl];
            cn[t] = L.count[th[t]];
            // A pre-aggregated tail: its MIN in place of the first offset.
            if (nd.tail[t].tmin)
              bg[t] = uint32_t(nd.tail[t].tmin[th[t]]);
            else if (nd.tail[t].n_min)
              bg[t] = L.begin[th[t]];
          }
        }
#pragma unroll
        for (int t = 0; t < MT; ++t) {
          pr[t] = 0;
          if (t < nt && nd.tail[t].n_min && !nd.tail[t].tmin && cn[t])
            pr[t] = atoms[nd.tail[t].atom].perm[bg[t]];
          if (t < nt) m = mul_sat(m, cn[t], &res->status);
        }
        if (!m) continue;
        unsigned long long before = my_count;
        my_count += m;
        if (my_count < before) atomicOr(&res->status, kStCountOverflow);
        any = true;
        for (int k = 0; k < nd.n_min; ++k)
          atomicMin(&s_min[nd.min_idx[k]], src_value(nd.src[nd.min_var[k]], 0, row[r]));
#pragma unroll
        for (int t = 0; t < MT; ++t) {
          if (t >= nt || !nd.tail[t].n_min) continue;
          const TailDev& td = nd.tail[t];
          if (td.tmin) {
            atomicMin(&s_min[td.min_idx[0]], int32_t(bg[t]));
            continue;
          }
          const AtomDev& ta = atoms[td.atom];
          for (int k = 0; k < td.n_min; ++k) {
            const int32_t* col = ta.cols[td.min_col[k]];
            int32_t lo = col[pr[t]];
            for (uint32_t x = 1; x < cn[t]; ++x) lo = min(lo, col[ta.perm[bg[t] + x]]);
            atomicMin(&s_min[td.min_idx[k]], lo);
          }
        }
        continue;
      }
      for (int t = 0; t < nd.n_tail && m; ++t) {
        const TailDev& td = nd.tail[t];
        const AtomDev& ta = atoms[td.atom];
        m = mul_sat(m, ta.L[td.lvl].count[scan_handle(sc, b, td.hsrc, idx[r])], &res->status);
      }
      if (!m) continue;
      unsigned long long before = my_count;
      my_count += m;
      if (my_count < before) atomicOr(&res->status, kStCountOverflow);
      any = true;
      for (int k = 0; k < nd.n_min; ++k)
        atomicMin(&s_min[nd.min_idx[k]], src_value(nd.src[nd.min_var[k]], 0, row[r]));
      for (int t = 0; t < nd.n_tail; ++t) {
        const TailDev& td = nd.tail[t];
        if (!td.n_min) continue;
        const AtomDev& ta = atoms[td.atom];
        uint32_t h = scan_handle(sc, b, td.hsrc, idx[r]);
        uint32_t bg = ta.L[td.lvl].begin[h], cn = ta.L[td.lvl].count[h];
        for (int k = 0; k < td.n_min; ++k) {
          const int32_t* col = ta.cols[td.min_col[k]];
          int32_t lo = INT32_MAX;
          for (uint32_t x = 0; x < cn; ++x) lo = min(lo, col[ta.perm[bg + x]]);
          atomicMin(&s_min[td.min_idx[k]], lo);
        }
      }
    }
  } else if (nd.mode == kModeFactorized) {
#pragma unroll
    for (int r = 0; r < R; ++r)
      factor_emit(
          nd, atoms, res, live >> r & 1u, mult[r],
          [&](int t) { return scan_handle(sc, b, nd.tail[t].hsrc, idx[r]); },
          [&](int v) { return src_value(nd.src[v], 0, row[r]); }, my_count);
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
      for (uint64_t x = 0; x < mult[r]; ++x) {
        uint64_t orow = base++;
        if (orow >= nd.out_rows_cap) {
          atomicOr(&res->status, kStOutputOverflow);
          continue;
        }
        for (int h = 0; h < nd.n_head; ++h)
          nd.out_tuples[orow * nd.n_head + h] = src_value(nd.src[nd.head_var[h]], 0, row[r]);
      }
    }
  }
}

// Block totals of node 0 into the result: COUNT and MIN (aggregate mode)
// and the probe counters.
__device__ __forceinline__ void scan_block_totals(const NodeDev& nd, ResultDev* res,
                                                  int32_t* s_min, unsigned long long* s_red,
                                                  unsigned long long my_count, bool any,
                                                  unsigned long long surv,
                                                  unsigned long long c_probe,
                                                  unsigned long long c_hit) {
  if (nd.mode == kModeAggregate || nd.mode == kModeFactorized) {
    unsigned long long tot = block_sum<unsigned long long>(my_count, s_red);
    int any_b = __syncthreads_or(any);
    if (threadIdx.x == 0 && tot) {
      unsigned long long old = atomicAdd(&res->count, tot);
      if (old + tot < old) atomicOr(&res->status, kStCountOverflow);
    }
    if (nd.mode == kModeAggregate && any_b && threadIdx.x < FJ_MAX_VARS)
      atomicMin(&res->mins[threadIdx.x], s_min[threadIdx.x]);
  }
  unsigned long long v = block_sum<unsigned long long>(surv, s_red);
  if (threadIdx.x == 0 && v) atomicAdd(&res->ctr[FJ_CTR_SURVIVORS], v);
  v = block_sum<unsigned long long>(c_probe, s_red);
  if (threadIdx.x == 0 && v) atomicAdd(&res->ctr[FJ_CTR_PROBES], v);
  v = block_sum<unsigned long long>(c_hit, s_red);
  if (threadIdx.x == 0 && v) atomicAdd(&res->ctr[FJ_CTR_PROBE_HITS], v);
}

// Step 2: every survivor of the first probe goes through the remaining
// probes in order (R survivors per thread, their gathers issued together),
// recording each entry in place, and then through the node's epilogue:
// aggregate (COUNT, MIN, trailing product nodes), write partial tuples for
// node 1, or materialize output tuples.
template <int R>
__global__ void __launch_bounds__(kThreads) k_scan_rest(const __grid_constant__ NodeDev nd,
                                                        const __grid_constant__ ScanDev sc,
                                                        AtomDev* atoms, ResultDev* res) {
  // A root build whose bounded wait ran out left its levels unbuilt.
  if (__syncthreads_or(threadIdx.x == 0 && (res->status & kStTimeout))) return;
  __shared__ uint32_t s_mask[FJ_MAX_SUB], s_fon[FJ_MAX_SUB];
  __shared__ int32_t s_min[FJ_MAX_VARS];
  __shared__ unsigned long long s_red[33];
  __shared__ uint32_t s_cnt, s_base;
  if (threadIdx.x < uint32_t(sc.n_probe)) {
    s_mask[threadIdx.x] = *sc.probe[threadIdx.x].mask;
    s_fon[threadIdx.x] = sc.probe[threadIdx.x].filter ? *sc.probe[threadIdx.x].filter_on : 0u;
  }
  if (threadIdx.x < FJ_MAX_VARS) s_min[threadIdx.x] = INT32_MAX;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  const ScanBuf& b = sc.buf[0];
  const uint32_t n = min(*b.n, sc.cap);
  unsigned long long my_count = 0, surv = 0, c_probe = 0, c_hit = 0;
  bool any = false;
  for (uint32_t b0 = blockIdx.x * (R * kThreads); b0 < n; b0 += gridDim.x * (R * kThreads)) {
    uint32_t idx[R], row[R], e[R];
    uint64_t mult[R];
    uint32_t live = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      idx[r] = b0 + r * kThreads + threadIdx.x;
      row[r] = 0;
      mult[r] = 1;
      if (idx[r] < n) {
        live |= 1u << r;
        row[r] = b.row[idx[r]];
        if (b.mult) mult[r] = b.mult[idx[r]];
      }
    }
    live = scan_rest_probes<R>(sc, b, s_mask, s_fon, live, idx, row, e, mult, &res->status,
                               c_probe, c_hit);
    surv += __popc(live);
    scan_epilogue<R>(nd, sc, b, atoms, res, idx, row, mult, live, &s_cnt, &s_base, s_min,
                     my_count, any);
  }
  scan_block_totals(nd, res, s_min, s_red, my_count, any, surv, c_probe, c_hit);
}

// ---------------------------------------------------------------------------
// Node 0 in one launch, for a cover without selections whose first probe is
// one key column at the root of a narrow level (every binary2fj plan over a
// star or chain of equi-joins).  Every warp works on its own, on a
// contiguous run of tiles of 512 cover rows:
//  * the cover's key column is streamed into the warp's shared memory by
//    bulk asynchronous copies (TMA, two stages completing on mbarriers, the
//    next tile in flight while this one is probed);
//  * every row is tested against the first probe's Bloom filter (a
//    multiplicative hash and one word), staged once per block (one block
//    per SM) in shared memory, the rows that pass are queued, and the
//    queue is resolved against the hash level with all 32 lanes busy;
//  * survivors go to a region of the survivor buffer private to the warp
//    (its own rows: no counter shared with other warps).
// Then the warp runs the remaining probes breadth-first over its survivors
// (every one a single key column at the root):
// one probe at a time over the whole list, kFuseU entries per lane with
// their key gathers and slot loads in flight together and no Bloom filter
// in the way (these levels are small and sit in L2), compacting the hits in
// place (each keeps the position it had after the first probe, where the
// entries of every probe are recorded), and finally the epilogue.  No
// block-wide barrier is taken after the prologue: warp totals go to shared
// memory and the last warp of the block publishes them, so the warps of an
// SM overlap their latency chains and never wait for one another.
// ---------------------------------------------------------------------------

constexpr uint32_t kFuseTile = 512;  // cover rows per warp tile (2 KB of keys)
constexpr uint32_t kFuseStages = 2;
constexpr int kFuseU = 4;  // list entries per lane per round of a later probe
// One block of 32 warps per SM, so that one copy of the first probe's Bloom
// filter in shared memory serves the whole SM (random words in shared
// memory cost a few bank conflicts; the same loads through L1 are
// uncoalesced and take one L1 wavefront per distinct line).
constexpr int kFuseThreads = 1024;
constexpr uint32_t kFuseFilterWords = 8192;  // the largest Bloom filter (32 KB)
constexpr size_t kFuseSmem = size_t(kFuseThreads / 32) * kFuseTile * (kFuseStages * 4 + 2) +
                             size_t(kFuseFilterWords) * 4;
constexpr uint32_t kSpinLimit = 50000;      // default mbarrier waits before giving up
constexpr uint32_t kSuspendHintNs = 20000;  // each wait sleeps at most this long

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

// Arm the barrier for `bytes` of asynchronous copies and copy them: global
// [src, src + bytes) to shared [dst, dst + bytes).  src, dst and bytes are
// multiples of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes,
                                            uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Wait for phase `parity` of the barrier to complete.  Each try suspends the
// thread until the phase completes or kSuspendHintNs pass; false after
// `limit` tries (about a second at the default).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendHintNs)
        : "memory");
    if (done) return true;
  }
  return false;
}

// The rest of a narrow root lookup of `key` whose first slot `sl` (index h)
// is loaded.
__device__ __forceinline__ bool root1_resolve(const uint4* __restrict__ ht, uint32_t mask,
                                              uint32_t key, uint32_t h, uint4 sl, uint32_t& e,
                                              uint32_t& cnt) {
  for (uint32_t it = 0; it <= mask; ++it) {
    if (sl.x == key && sl.y == 0u) {
      e = sl.z;
      cnt = sl.w;
      return true;
    }
    if (sl.x == kNone && sl.y == kNone) return false;
    h = (h + 1) & mask;
    sl = __ldg(&ht[h]);
  }
  return false;
}

// Bloom filter bits of one tile for lane `lane`: rows 128 g + 4 lane + i
// (g < G, i < 4) map to bit 4 g + i.  FULL: all T rows exist and are staged
// in `kt`; otherwise rows at or past `here` are absent and read from `kg`.
template <uint32_t G, bool FULL>
__device__ __forceinline__ uint32_t filter_bits(const int32_t* kt, const int32_t* kg,
                                                uint32_t here, const uint32_t* filt,
                                                uint32_t fw1, uint32_t lane) {
  uint32_t pass = 0;
#pragma unroll
  for (uint32_t g = 0; g < G; ++g) {
    const uint32_t j0 = g * 128 + 4 * lane;
    int32_t k[4];
    if (FULL) {
      int4 v = *reinterpret_cast<const int4*>(&kt[j0]);
      k[0] = v.x;
      k[1] = v.y;
      k[2] = v.z;
      k[3] = v.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) k[i] = j0 + i < here ? __ldg(kg + j0 + i) : 0;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      bool ok = FULL || j0 + i < here;
      if (filt) {  // the filter's copy in shared memory
        const uint32_t fh = filter_hash_root1(k[i]);
        const uint32_t m = bloom_bits(fh);
        ok = ok && (filt[fh & fw1] & m) == m;
      }
      if (ok) pass |= 1u << (4 * g + i);
    }
  }
  return pass;
}

// Exact membership bits of one tile for lane `lane` (same row-to-bit map as
// filter_bits): the key's bit in the level's key bitmap `bm` of `nbits`
// bits (keys outside it are not in the level).
template <uint32_t G, bool FULL>
__device__ __forceinline__ uint32_t bitmap_bits(const int32_t* kt, const int32_t* kg,
                                                uint32_t here, const uint32_t* bm, uint32_t nbits,
                                                uint32_t lane) {
  uint32_t pass = 0;
#pragma unroll
  for (uint32_t g = 0; g < G; ++g) {
    const uint32_t j0 = g * 128 + 4 * lane;
    uint32_t k[4];
    if (FULL) {
      int4 v = *reinterpret_cast<const int4*>(&kt[j0]);
      k[0] = uint32_t(v.x);
      k[1] = uint32_t(v.y);
      k[2] = uint32_t(v.z);
      k[3] = uint32_t(v.w);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) k[i] = j0 + i < here ? uint32_t(__ldg(kg + j0 + i)) : nbits;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (k[i] < nbits && (bm[k[i] >> 5] >> (k[i] & 31u) & 1u)) pass |= 1u << (4 * g + i);
  }
  return pass;
}

template <int R>
__global__ void __launch_bounds__(kFuseThreads, 1) k_scan_fused(const __grid_constant__ NodeDev nd,
                                                            const __grid_constant__ ScanDev sc,
                                                            AtomDev* atoms, ResultDev* res) {
  // A root build whose bounded wait ran out left its levels unbuilt.
  if (__syncthreads_or(threadIdx.x == 0 && (res->status & kStTimeout))) return;
  constexpr uint32_t T = kFuseTile, NS = kFuseStages, W = kFuseThreads / 32;
  constexpr uint32_t G = T / 128;  // groups of 4 rows per lane
  static_assert(G <= 8, "a lane's pass mask holds 32 rows");
  constexpr int QU = 2;  // queue entries per lane with slot loads in flight
  // Dynamic shared memory (kFuseSmem bytes): per warp NS key stages of T
  // rows, then per warp the queue of the rows of a tile that pass the
  // filter, then the first probe's Bloom filter.
  extern __shared__ __align__(128) unsigned char s_dyn[];
  auto s_keys = reinterpret_cast<int32_t(*)[NS][T]>(s_dyn);
  auto s_q = reinterpret_cast<uint16_t(*)[T]>(s_dyn + size_t(W) * NS * T * 4);
  uint32_t* s_filt =
      reinterpret_cast<uint32_t*>(s_dyn + size_t(W) * NS * T * 4 + size_t(W) * T * 2);
  __shared__ alignas(8) uint64_t s_bar[W][NS];
  __shared__ alignas(8) uint64_t s_fbar;  // the filter's bulk copy
  __shared__ uint32_t s_mask[FJ_MAX_SUB], s_fon[FJ_MAX_SUB];
  __shared__ int32_t s_min[FJ_MAX_VARS];
  __shared__ unsigned long long s_tot[5];  // count, survivors, probes, hits, any row
  __shared__ uint32_t s_done, s_cnt, s_base;
  const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
  const uint64_t begin = nd.chunk_begin;
  const uint32_t n_rows = uint32_t(nd.chunk_end - begin);
  const uint32_t n_tiles = (n_rows + T - 1) / T;
  const uint32_t n_warps = gridDim.x * W, gw = blockIdx.x * W + warp;
  // Balanced contiguous runs: warp gw takes tiles [gw n / N, (gw + 1) n / N).
  const uint32_t t0 = uint32_t(uint64_t(gw) * n_tiles / n_warps);
  const uint32_t t1 = uint32_t(uint64_t(gw + 1) * n_tiles / n_warps);
  const uint32_t region = t0 * T;
  const ScanProbe& P = sc.probe[0];
  const int32_t* kcol = P.kcol[0] + begin;
  const ScanBuf& out = sc.buf[0];
  const uint32_t spin = sc.spin ? sc.spin : kSpinLimit;
  int32_t(*keys)[T] = s_keys[warp];
  uint64_t* bar = s_bar[warp];
  uint16_t* q = s_q[warp];

  if (tid < uint32_t(sc.n_probe)) {
    s_mask[tid] = *sc.probe[tid].mask;
    s_fon[tid] = sc.probe[tid].filter ? *sc.probe[tid].filter_on : 0u;
  }
  if (tid < FJ_MAX_VARS) s_min[tid] = INT32_MAX;
  if (tid < 5) s_tot[tid] = 0;
  if (tid == 0) s_done = 0;
  if (lane == 0) {
    for (uint32_t i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // The first probe's filter, when it is on, into shared memory by one bulk
  // copy that lands while the warps start their first tiles -- or, when the
  // level's key bitmap holds every key (and the probe does not end its
  // atom), the bitmap: membership is then exact, the rows that pass are the
  // probe's hits, and their entries are looked up only for the final
  // survivors.
  const bool ex0 = P.bitmap && !P.last && sc.k1 && *P.exact;
  const bool fon0 = !ex0 && P.filter && *P.filter_on;
  const bool copy0 = ex0 || fon0;
  if (tid == 0 && copy0) {
    mbar_init(&s_fbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    tma_load_1d(s_filt, ex0 ? P.bitmap : P.filter, P.filter_words * 4, &s_fbar);
  }
  __syncthreads();
  // Lane 0 is the warp's producer: its first NS full tiles now, then each
  // tile NS ahead once the warp is done with the stage it reuses.
  if (lane == 0)
    for (uint32_t t = t0; t < t1 && t < t0 + NS; ++t)
      if ((t + 1) * T <= n_rows) tma_load_1d(keys[t - t0], kcol + size_t(t) * T, T * 4, &bar[t - t0]);

  const uint32_t mask = s_mask[0];
  const uint32_t* filt = fon0 ? s_filt : nullptr;
  const uint32_t fw1 = P.filter_words - 1;
  const bool keep_h = !P.last;
  const int nk1 = sc.n_probe > 1 ? sc.probe[1].nk : 0;  // second probe's key columns
  const int32_t* kc1a = sc.probe[1].kcol[0];
  const int32_t* kc1b = sc.probe[1].kcol[1];
  const int32_t* kc1c = sc.probe[1].kcol[2];
  unsigned long long c_probe = 0, c_hit = 0, my_count = 0, surv = 0;
  bool any = false, timed_out = false;
  if (copy0 && !mbar_wait(&s_fbar, 0, spin)) timed_out = true;
  uint32_t n_surv = 0;  // survivors in the warp's region (the same in every lane)
  uint32_t t = t0;
  for (; t < t1; ++t) {
    const uint32_t li = t - t0, st = li % NS;
    const uint32_t here = min(T, n_rows - t * T);
    const bool staged = here == T;
    if (staged && !mbar_wait(&bar[st], (li / NS) & 1u, spin)) timed_out = true;
    if (__any_sync(0xffffffffu, timed_out)) break;
    const int32_t* kt = keys[st];
    const int32_t* kg = kcol + size_t(t) * T;
    if (ex0) {
      // Exact: the rows that pass go straight to the warp's region.
      const uint32_t nbits = P.filter_words * 32;
      const uint32_t pass = staged ? bitmap_bits<G, true>(kt, kg, here, s_filt, nbits, lane)
                                   : bitmap_bits<G, false>(kt, kg, here, s_filt, nbits, lane);
      if (lane == 0) c_probe += here;
      const uint32_t np = __popc(pass);
      const uint32_t incl = warp_incl_scan(np);
      uint32_t pos = region + n_surv + incl - np;
      const uint32_t rbase = uint32_t(begin + size_t(t) * T);
      for (uint32_t m = pass; m; m &= m - 1) {
        const uint32_t bt = __ffs(m) - 1;
        const uint32_t row = rbase + (bt >> 2) * 128 + 4 * lane + (bt & 3);
        out.row[pos] = row;
        if (out.mult) out.mult[pos] = 1u;
        ++pos;
        // The second probe gathers this row's key later: its sector into L2.
        if (nk1 > 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(kc1a + row));
        if (nk1 > 1) asm volatile("prefetch.global.L2 [%0];" ::"l"(kc1b + row));
        if (nk1 > 2) asm volatile("prefetch.global.L2 [%0];" ::"l"(kc1c + row));
      }
      n_surv += __shfl_sync(0xffffffffu, incl, 31);
      __syncwarp();
      if (lane == 0 && t + NS < t1 && (t + NS + 1) * T <= n_rows)
        tma_load_1d(keys[st], kcol + size_t(t + NS) * T, T * 4, &bar[st]);
      continue;
    }
    const uint32_t pass = staged ? filter_bits<G, true>(kt, kg, here, filt, fw1, lane)
                                 : filter_bits<G, false>(kt, kg, here, filt, fw1, lane);
    if (lane == 0) c_probe += here;
    const uint32_t np = __popc(pass);
    const uint32_t incl = warp_incl_scan(np);
    const uint32_t qn = __shfl_sync(0xffffffffu, incl, 31);
    uint32_t qp = incl - np;
    for (uint32_t m = pass; m; m &= m - 1) {
      const uint32_t bt = __ffs(m) - 1;
      q[qp++] = uint16_t((bt >> 2) * 128 + 4 * lane + (bt & 3));
    }
    __syncwarp();
    // Resolve the queue, QU entries per lane with their first slot loads in
    // flight together; hits are appended to the warp's region.
    const uint32_t rbase = uint32_t(begin + size_t(t) * T);
    for (uint32_t i0 = 0; i0 < qn; i0 += QU * 32) {
      uint32_t key[QU], hh[QU], jj[QU];
      uint4 sl[QU];
#pragma unroll
      for (int u = 0; u < QU; ++u) {
        const uint32_t i = i0 + u * 32 + lane;
        jj[u] = i < qn ? q[i] : 0u;
        key[u] = uint32_t(staged ? kt[jj[u]] : __ldg(kg + jj[u]));
        hh[u] = hash_root1(int32_t(key[u])) & mask;
        if (i < qn) sl[u] = __ldg(&P.ht[hh[u]]);
      }
#pragma unroll
      for (int u = 0; u < QU; ++u) {
        uint32_t e = 0, cnt = 0;
        const bool hit = i0 + u * 32 + lane < qn &&
                         root1_resolve(P.ht, mask, key[u], hh[u], sl[u], e, cnt);
        const uint32_t hm = __ballot_sync(0xffffffffu, hit);
        if (hit) {
          const uint32_t pos = region + n_surv + __popc(hm & lanemask_lt());
          out.row[pos] = rbase + jj[u];
          if (keep_h) out.h[0][pos] = e;
          if (out.mult) out.mult[pos] = P.last ? cnt : 1u;
          // The second probe gathers this row's key later: bring its sector
          // into L2 now (no register waits on it).
          const uint32_t row = rbase + jj[u];
          if (nk1 > 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(kc1a + row));
          if (nk1 > 1) asm volatile("prefetch.global.L2 [%0];" ::"l"(kc1b + row));
          if (nk1 > 2) asm volatile("prefetch.global.L2 [%0];" ::"l"(kc1c + row));
        }
        n_surv += __popc(hm);
      }
    }
    __syncwarp();
    if (lane == 0 && t + NS < t1 && (t + NS + 1) * T <= n_rows)
      tma_load_1d(keys[st], kcol + size_t(t + NS) * T, T * 4, &bar[st]);
  }
  if (t < t1 || timed_out) {
    // A copy did not complete in time: record it and let the warp's copies
    // still in flight (its tiles, and the block's filter) land before its
    // shared memory can be released (a longer bounded wait; one that runs
    // out too is flagged apart).
    if (lane == 0) {
      atomicOr(&res->status, kStTimeout);
      if (copy0 && !mbar_wait(&s_fbar, 0, 64u * spin)) atomicOr(&res->status, kStDrainTimeout);
      for (uint32_t u = t; u < t1 && u < t + NS; ++u)
        if ((u + 1) * T <= n_rows &&
            !mbar_wait(&bar[(u - t0) % NS], ((u - t0) / NS) & 1u, 64u * spin))
          atomicOr(&res->status, kStDrainTimeout);
    }
    n_surv = 0;
  }
  if (lane == 0) c_hit += n_surv;

  // Remaining probes, breadth-first over the warp's list [region, region+n).
  uint32_t n_list = n_surv;
  for (int p = 1; p < sc.n_probe && n_list; ++p) {
    const ScanProbe& Pp = sc.probe[p];
    const uint32_t mp = s_mask[p];
    uint32_t n_out = 0;
    {
      // One key column at the root (the key word is the value; the host
      // uses this kernel only when every probe has that shape): kFuseU
      // entries per lane, every key gather in flight together, then every
      // first slot load.
      const int32_t* kc = Pp.kcol[0];
      for (uint32_t i0 = 0; i0 < n_list; i0 += kFuseU * 32) {
        uint32_t row[kFuseU], key[kFuseU];
        uint4 sl[kFuseU];
        uint32_t lv = 0;
#pragma unroll
        for (int u = 0; u < kFuseU; ++u) {
          const uint32_t i = i0 + u * 32 + lane;
          row[u] = 0;
          if (i < n_list) {
            lv |= 1u << u;
            row[u] = out.row[region + i];
          }
        }
#pragma unroll
        for (int u = 0; u < kFuseU; ++u) key[u] = (lv >> u & 1u) ? uint32_t(__ldg(kc + row[u])) : 0u;
#pragma unroll
        for (int u = 0; u < kFuseU; ++u)
          if (lv >> u & 1u) sl[u] = __ldg(&Pp.ht[hash_root1(int32_t(key[u])) & mp]);
        c_probe += __popc(lv);
#pragma unroll
        for (int u = 0; u < kFuseU; ++u) {
          if (!(lv >> u & 1u)) continue;
          uint32_t e = 0, cnt = 0;
          if (root1_resolve(Pp.ht, mp, key[u], hash_root1(int32_t(key[u])) & mp, sl[u], e,
                            cnt)) {
            sl[u].z = e;
            sl[u].w = cnt;
          } else {
            lv &= ~(1u << u);
          }
        }
        c_hit += __popc(lv);
        // Each hit's position after the first probe (into key[]) and
        // multiplicity (into the spent key words of its slot), read by every
        // lane before any lane compacts.
#pragma unroll
        for (int u = 0; u < kFuseU; ++u) {
          if (!(lv >> u & 1u)) continue;
          const uint32_t i = region + i0 + u * 32 + lane;
          key[u] = p > 1 ? out.src[i] : i;
          if (out.mult) {
            uint64_t m = out.mult[i];
            if (Pp.last) m = mul_sat(m, sl[u].w, &res->status);
            sl[u].x = uint32_t(m);
            sl[u].y = uint32_t(m >> 32);
          }
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < kFuseU; ++u) {
          const bool hit = lv >> u & 1u;
          const uint32_t hm = __ballot_sync(0xffffffffu, hit);
          if (hit) {
            const uint32_t pos = region + n_out + __popc(hm & lanemask_lt());
            if (!Pp.last) out.h[p][key[u]] = sl[u].z;
            if (out.mult) out.mult[pos] = (uint64_t(sl[u].y) << 32) | sl[u].x;
            out.row[pos] = row[u];
            out.src[pos] = key[u];
          }
          n_out += __popc(hm);
        }
        __syncwarp();
      }
    }
    n_list = n_out;
  }
  // The first probe's entries when its bitmap was exact, for the final
  // survivors only (their keys are in the level: every lookup hits).
  if (ex0 && keep_h) {
    for (uint32_t i0 = 0; i0 < n_list; i0 += uint32_t(R) * 32) {
      uint32_t key[R], ix[R];
      uint4 sl[R];
      uint32_t lv = 0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t i = i0 + r * 32 + lane, pos = region + i;
        key[r] = 0;
        ix[r] = pos;
        if (i < n_list) {
          lv |= 1u << r;
          key[r] = out.row[pos];
          if (sc.n_probe > 1) ix[r] = out.src[pos];
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (lv >> r & 1u) key[r] = uint32_t(__ldg(P.kcol[0] + key[r]));
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (lv >> r & 1u) sl[r] = __ldg(&P.ht[hash_root1(int32_t(key[r])) & mask]);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        uint32_t e = 0, cnt = 0;
        if ((lv >> r & 1u) &&
            root1_resolve(P.ht, mask, key[r], hash_root1(int32_t(key[r])) & mask, sl[r], e, cnt))
          out.h[0][ix[r]] = e;
      }
    }
  }
  // Epilogue over the final list.
  for (uint32_t i0 = 0; i0 < n_list; i0 += uint32_t(R) * 32) {
    uint32_t idx[R], row[R];
    uint64_t mult[R];
    uint32_t lv = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t i = i0 + r * 32 + lane, pos = region + i;
      idx[r] = pos;
      row[r] = 0;
      mult[r] = 1;
      if (i < n_list) {
        lv |= 1u << r;
        row[r] = out.row[pos];
        if (sc.n_probe > 1) idx[r] = out.src[pos];
        if (out.mult) mult[r] = out.mult[pos];
      }
    }
    surv += __popc(lv);
    scan_epilogue<R, true>(nd, sc, out, atoms, res, idx, row, mult, lv, &s_cnt, &s_base, s_min,
                           my_count, any);
  }

  // Warp totals into shared memory; the last warp of the block to arrive
  // publishes the block's totals (no block barrier).
  for (int o = 16; o; o >>= 1) {
    my_count += __shfl_xor_sync(0xffffffffu, my_count, o);
    surv += __shfl_xor_sync(0xffffffffu, surv, o);
    c_probe += __shfl_xor_sync(0xffffffffu, c_probe, o);
    c_hit += __shfl_xor_sync(0xffffffffu, c_hit, o);
  }
  const bool any_w = __any_sync(0xffffffffu, any);
  __threadfence_block();  // every lane's shared-memory MINs before the arrival
  __syncwarp();
  uint32_t last = 0;
  if (lane == 0) {
    if (my_count) {
      const unsigned long long old = atomicAdd(&s_tot[0], my_count);
      if (old + my_count < old) atomicOr(&res->status, kStCountOverflow);
    }
    if (surv) atomicAdd(&s_tot[1], surv);
    if (c_probe) atomicAdd(&s_tot[2], c_probe);
    if (c_hit) atomicAdd(&s_tot[3], c_hit);
    if (any_w) atomicOr(&s_tot[4], 1ull);
    __threadfence_block();
    last = atomicAdd(&s_done, 1u) == W - 1;
  }
  if (!__shfl_sync(0xffffffffu, last, 0)) return;
  __threadfence_block();
  const volatile unsigned long long* vt = s_tot;
  if (nd.mode == kModeAggregate || nd.mode == kModeFactorized) {
    if (lane == 0 && vt[0]) {
      const unsigned long long old = atomicAdd(&res->count, vt[0]);
      if (old + vt[0] < old) atomicOr(&res->status, kStCountOverflow);
    }
    if (nd.mode == kModeAggregate && vt[4])
      atomicMin(&res->mins[lane], reinterpret_cast<volatile int32_t*>(s_min)[lane]);
  }
  if (lane == 0) {
    if (vt[1]) atomicAdd(&res->ctr[FJ_CTR_SURVIVORS], vt[1]);
    if (vt[2]) atomicAdd(&res->ctr[FJ_CTR_PROBES], vt[2]);
    if (vt[3]) atomicAdd(&res->ctr[FJ_CTR_PROBE_HITS], vt[3]);
    if (blockIdx.x == 0 && n_rows)
      atomicAdd(&res->ctr[FJ_CTR_COVER_ITERS], (unsigned long long)n_rows);
  }
}

// The survivor count to zero before a chunk.
__global__ void k_scan_reset(const __grid_constant__ ScanDev sc) {
  if (threadIdx.x == 0) *sc.buf[0].n = 0;
}

}  // namespace fj
