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
};

// Survivor buffer: structure of arrays, device-side count.
struct ScanBuf {
  uint32_t* row;
  uint32_t* h[FJ_MAX_SUB];  // entry reached by probe p (non-last probes)
  uint64_t* mult;           // null when no probe ends an atom at a leaf
  uint32_t* n;
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
          if (filt && (live >> r & 1u)) {
            uint32_t m = bloom_bits(hv[r]);
            if ((__ldg(&filt[hv[r] & (P.filter_words - 1)]) & m) != m) live &= ~(1u << r);
          }
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

// Step 2: every survivor of the first probe goes through the remaining
// probes in order (R survivors per thread, their gathers issued together),
// recording each entry in place, and then through the node's epilogue:
// aggregate (COUNT, MIN, trailing product nodes), write partial tuples for
// node 1, or materialize output tuples.
template <int R>
__global__ void __launch_bounds__(kThreads) k_scan_rest(const __grid_constant__ NodeDev nd,
                                                        const __grid_constant__ ScanDev sc,
                                                        AtomDev* atoms, ResultDev* res) {
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
    for (int p = 1; p < sc.n_probe && live; ++p) {
      const ScanProbe& P = sc.probe[p];
      c_probe += __popc(live);
      live = scan_probe_rows<R>(P, s_mask[p], s_fon[p] ? P.filter : nullptr, live, row, e,
                                b.mult ? mult : nullptr, &res->status);
      c_hit += __popc(live);
      if (!P.last)
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (live >> r & 1u) b.h[p][idx[r]] = e[r];
    }
    surv += __popc(live);
    if (nd.mode == kModeItems) {
      uint32_t pos = block_append(__popc(live), nd.out_n, &s_cnt, &s_base);
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
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!(live >> r & 1u)) continue;
        uint64_t m = mult[r];
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
  if (nd.mode == kModeAggregate) {
    unsigned long long tot = block_sum<unsigned long long>(my_count, s_red);
    int any_b = __syncthreads_or(any);
    if (threadIdx.x == 0 && tot) {
      unsigned long long old = atomicAdd(&res->count, tot);
      if (old + tot < old) atomicOr(&res->status, kStCountOverflow);
    }
    if (any_b && threadIdx.x < FJ_MAX_VARS)
      atomicMin(&res->mins[threadIdx.x], s_min[threadIdx.x]);
  }
  unsigned long long v = block_sum<unsigned long long>(surv, s_red);
  if (threadIdx.x == 0 && v) atomicAdd(&res->ctr[FJ_CTR_SURVIVORS], v);
  v = block_sum<unsigned long long>(c_probe, s_red);
  if (threadIdx.x == 0 && v) atomicAdd(&res->ctr[FJ_CTR_PROBES], v);
  v = block_sum<unsigned long long>(c_hit, s_red);
  if (threadIdx.x == 0 && v) atomicAdd(&res->ctr[FJ_CTR_PROBE_HITS], v);
}

// The survivor count to zero before a chunk.
__global__ void k_scan_reset(const __grid_constant__ ScanDev sc) {
  if (threadIdx.x == 0) *sc.buf[0].n = 0;
}

}  // namespace fj
