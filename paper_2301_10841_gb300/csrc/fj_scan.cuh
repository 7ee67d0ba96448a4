// Node 0 of a plan whose cover is iterated straight from its base table (the
// COLT base-table case of Section 4.2: nothing is built for the cover), with
// the batch-at-a-time probes of Section 4.3.  This is node 0 of every plan
// produced by binary2fj, and the whole probe phase of a factored star join.
//
// Design (GB300): a lean kernel (few registers, high occupancy) in which
//  * each lane takes R rows of a warp tile (coalesced column loads), tests
//    the first probe's Bloom filter (L1-resident) and issues the hash-slot
//    loads of all its rows before resolving any;
//  * survivors go to a per-warp queue in shared memory; when the queue might
//    not hold another tile it is flushed: the remaining probes run phase by
//    phase over the whole queue (4 elements per lane in flight), compacting
//    the live list after each phase, and then the epilogue (write partial
//    tuples, aggregate, or materialize) runs over what is left.
// No block-wide barrier is taken inside the row loop.
#pragma once

#include "fj_exec.cuh"

namespace fj {

// One probe of the scan kernel, resolved on the host: key columns of the
// cover row (node 0 binds every variable from the cover), the hash level,
// and its Bloom filter.
struct ScanProbe {
  const int32_t* kcol[3];
  int nk;
  int wide;
  int last;
  int sub;                    // subatom index (new handle slot)
  const uint4* ht;
  const uint32_t* mask;       // device-side
  const uint32_t* filter;
  uint32_t filter_words;
  const uint32_t* filter_on;  // device-side
};

struct ScanDev {
  int track;   // some probe ends an atom at a leaf: keep multiplicities
  int k1;      // the first probe is one key column at the root, narrow level
  int vec_ok;  // its key column is 16-byte aligned and chunks start at 4k rows
  int n_probe;
  ScanProbe probe[FJ_MAX_SUB];
  int n_preds;
  const int32_t* pred_col[FJ_MAX_PREDS];
  int pred_op[FJ_MAX_PREDS];
  int32_t pred_val[FJ_MAX_PREDS];
};

constexpr int kScanQ = 384;  // queue slots per warp
constexpr int kScanFR = 4;   // queue elements per lane per flush step

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

__device__ __forceinline__ uint64_t scan_key(const ScanProbe& P, uint32_t row) {
  int32_t v0 = P.nk > 0 ? __ldg(P.kcol[0] + row) : 0;
  int32_t v1 = P.nk > 1 ? __ldg(P.kcol[1] + row) : 0;
  return pack_key(0u, P.nk, v0, v1);
}

__device__ __forceinline__ bool scan_find_wide(const ScanProbe& P, uint32_t mask, uint32_t row,
                                               uint32_t& e, uint32_t& cnt) {
  uint4 k = make_uint4(0u, P.nk > 0 ? uint32_t(__ldg(P.kcol[0] + row)) : 0u,
                       P.nk > 1 ? uint32_t(__ldg(P.kcol[1] + row)) : 0u,
                       P.nk > 2 ? uint32_t(__ldg(P.kcol[2] + row)) : 0u);
  return ht_find_wide(P.ht, mask, k, e, cnt);
}

// Shared per-warp queue: row, multiplicity, new handle per probe, live list.
struct ScanQueue {
  uint32_t* row;   // [kScanQ]
  uint64_t* mult;  // [kScanQ]
  uint32_t* newh;  // [n_probe][kScanQ]
  uint16_t* live;  // [kScanQ]
};

__host__ __device__ constexpr size_t scan_queue_bytes(int n_probe, int track) {
  return size_t(kScanQ) * ((track ? 8 : 0) + 4 + 4 * size_t(n_probe) + 2);
}

// Per-warp counters of the scan kernel.
struct ScanAcc {
  unsigned long long iters, probes, hits, surv, count;
};

// Remaining probes (1..n_probe-1) over the queued survivors, phase by phase,
// then the epilogue.
__device__ __forceinline__ void scan_flush(const NodeDev& nd, const ScanDev& sc,
                                           const AtomDev* atoms, ResultDev* res,
                                           const ScanQueue& q, uint32_t qn,
                                           const uint32_t* s_mask, const uint32_t* s_fon,
                                           int32_t* s_min, ScanAcc& acc) {
  const uint32_t lane = lane_id();
  for (int p = 1; p < sc.n_probe && qn; ++p) {
    const ScanProbe& P = sc.probe[p];
    const uint32_t mask = s_mask[p];
    const uint32_t* filt = s_fon[p] ? P.filter : nullptr;
    uint32_t out = 0;
    for (uint32_t c0 = 0; c0 < qn; c0 += 32 * kScanFR) {
      uint32_t slot[kScanFR], hh[kScanFR], live = 0;
      uint64_t kw[kScanFR];
      uint4 sl[kScanFR];
#pragma unroll
      for (int r = 0; r < kScanFR; ++r) {
        uint32_t pos = c0 + r * 32 + lane;
        slot[r] = pos < qn ? q.live[pos] : 0u;
        kw[r] = 0;
        hh[r] = 0;
        if (pos < qn) {
          live |= 1u << r;
          if (!P.wide) kw[r] = scan_key(P, q.row[slot[r]]);
        }
      }
      acc.probes += __popc(live);
      if (!P.wide) {
#pragma unroll
        for (int r = 0; r < kScanFR; ++r)
          if ((live >> r & 1u) && kw[r] != kEmptyKey &&
              !probe_start(P.ht, mask, filt, P.filter_words, kw[r], hh[r], sl[r]))
            live &= ~(1u << r);
      }
#pragma unroll
      for (int r = 0; r < kScanFR; ++r) {
        if (!(live >> r & 1u)) continue;
        uint32_t e = 0, cnt = 0;
        bool hit;
        if (P.wide) {
          hit = scan_find_wide(P, mask, q.row[slot[r]], e, cnt);
        } else if (kw[r] == kEmptyKey) {
          uint4 sp = __ldg(&P.ht[mask + 1]);
          e = sp.z;
          cnt = sp.w;
          hit = sp.w != 0;
        } else {
          hit = ht_resolve(P.ht, mask, kw[r], hh[r], sl[r], e, cnt);
        }
        if (!hit) {
          live &= ~(1u << r);
        } else if (P.last) {
          if (q.mult) q.mult[slot[r]] = mul_sat(q.mult[slot[r]], cnt, &res->status);
        } else {
          q.newh[p * kScanQ + slot[r]] = e;
        }
      }
      acc.hits += __popc(live);
      // Compact the live list in place (positions only move down; every
      // lane has read its slots before any lane writes).
      __syncwarp();
#pragma unroll
      for (int r = 0; r < kScanFR; ++r) {
        bool keep = live >> r & 1u;
        uint32_t m = __ballot_sync(0xffffffffu, keep);
        if (keep) q.live[out + __popc(m & lanemask_lt())] = uint16_t(slot[r]);
        out += __popc(m);
      }
      __syncwarp();
    }
    qn = out;
  }
  if (lane == 0) acc.surv += qn;
  // Epilogue.
  for (uint32_t c0 = 0; c0 < qn; c0 += 32) {
    uint32_t pos = c0 + lane;
    bool live = pos < qn;
    uint32_t slot = live ? q.live[pos] : 0u;
    uint32_t row = live ? q.row[slot] : 0u;
    uint64_t m = live ? (q.mult ? q.mult[slot] : 1ull) : 0ull;
    if (nd.mode == kModeItems) {
      uint32_t bm = __ballot_sync(0xffffffffu, live);
      uint32_t base = 0;
      if (lane == 0 && bm) base = atomicAdd(nd.out_n, __popc(bm));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (live) {
        uint32_t o = base + __popc(bm & lanemask_lt());
        if (o >= nd.out_cap) {
          atomicOr(&res->status, kStItemsOverflow);
        } else {
          for (int k = 0; k < nd.n_out_vars; ++k)
            nd.out_var[k][o] = src_value(nd.src[nd.out_var_id[k]], 0, row);
          for (int a = 0; a < FJ_MAX_ATOMS; ++a) {
            if (!nd.out_h[a]) continue;
            int src = nd.out_h_src[a];  // a probed subatom (node 0 has no inputs)
            for (int p = 0; p < sc.n_probe; ++p)
              if (sc.probe[p].sub == src) nd.out_h[a][o] = q.newh[p * kScanQ + slot];
          }
          if (nd.out_mult) nd.out_mult[o] = m;
        }
      }
    } else if (nd.mode == kModeAggregate) {
      if (live) {
        for (int t = 0; t < nd.n_tail && m; ++t) {
          const TailDev& td = nd.tail[t];
          const AtomDev& ta = atoms[td.atom];
          uint32_t h = 0;
          for (int p = 0; p < sc.n_probe; ++p)
            if (sc.probe[p].sub == td.hsrc) h = q.newh[p * kScanQ + slot];
          m = mul_sat(m, ta.L[td.lvl].count[h], &res->status);
        }
        if (m) {
          unsigned long long before = acc.count;
          acc.count += m;
          if (acc.count < before) atomicOr(&res->status, kStCountOverflow);
          for (int k = 0; k < nd.n_min; ++k)
            atomicMin(&s_min[nd.min_idx[k]], src_value(nd.src[nd.min_var[k]], 0, row));
          for (int t = 0; t < nd.n_tail; ++t) {
            const TailDev& td = nd.tail[t];
            if (!td.n_min) continue;
            const AtomDev& ta = atoms[td.atom];
            uint32_t h = 0;
            for (int p = 0; p < sc.n_probe; ++p)
              if (sc.probe[p].sub == td.hsrc) h = q.newh[p * kScanQ + slot];
            uint32_t bg = ta.L[td.lvl].begin[h], cn = ta.L[td.lvl].count[h];
            for (int k = 0; k < td.n_min; ++k) {
              const int32_t* col = ta.cols[td.min_col[k]];
              int32_t lo_v = INT32_MAX;
              for (uint32_t x = 0; x < cn; ++x) lo_v = min(lo_v, col[ta.perm[bg + x]]);
              atomicMin(&s_min[td.min_idx[k]], lo_v);
            }
          }
        }
      }
    } else {  // kModeMaterialize
      uint64_t tot = live ? m : 0ull;
      uint64_t inc = warp_incl_scan<unsigned long long>(tot);
      uint64_t base = 0;
      if (lane == 31 && inc) base = atomicAdd(&res->n_out, (unsigned long long)inc);
      base = __shfl_sync(0xffffffffu, (unsigned long long)base, 31) + inc - tot;
      if (live) {
        for (uint64_t x = 0; x < m; ++x) {
          uint64_t orow = base + x;
          if (orow >= nd.out_rows_cap) {
            atomicOr(&res->status, kStOutputOverflow);
            break;
          }
          for (int h = 0; h < nd.n_head; ++h)
            nd.out_tuples[orow * nd.n_head + h] = src_value(nd.src[nd.head_var[h]], 0, row);
        }
      }
    }
  }
  __syncwarp();
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

// First probe for the common case (one key column, root level, narrow
// table): 16-byte loads of the key column, one hash per row, the Bloom test,
// then the slot loads.  Lane l owns rows 4l..4l+3 of each 128-row half of
// the 256-row warp tile.  Returns the live mask; entries in e[].
__device__ __forceinline__ uint32_t scan_first_k1(const ScanDev& sc, uint32_t mask,
                                                  const uint32_t* filt, uint64_t r0, uint64_t end,
                                                  uint32_t lane, uint32_t (&row)[8],
                                                  uint32_t (&e)[8]) {
  const ScanProbe& P = sc.probe[0];
  int32_t k[8];
  uint32_t alive = 0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint64_t base = r0 + h * 128 + 4 * lane;
#pragma unroll
    for (int j = 0; j < 4; ++j) row[h * 4 + j] = uint32_t(base + j);
    if (sc.vec_ok && base + 4 <= end) {
      int4 v = __ldg(reinterpret_cast<const int4*>(P.kcol[0] + base));
      k[h * 4 + 0] = v.x;
      k[h * 4 + 1] = v.y;
      k[h * 4 + 2] = v.z;
      k[h * 4 + 3] = v.w;
      alive |= 0xfu << (h * 4);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        k[h * 4 + j] = 0;
        if (base + j < end) {
          k[h * 4 + j] = __ldg(P.kcol[0] + base + j);
          alive |= 1u << (h * 4 + j);
        }
      }
    }
  }
  if (sc.n_preds) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
      if ((alive >> r & 1u) && !scan_pred(sc, row[r])) alive &= ~(1u << r);
  }
  uint32_t hv[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    hv[r] = hash_root1(k[r]);
    if (filt && (alive >> r & 1u)) {
      uint32_t m = bloom_bits(hv[r]);
      if ((__ldg(&filt[hv[r] & (P.filter_words - 1)]) & m) != m) alive &= ~(1u << r);
    }
  }
  uint4 sl[8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
    if (alive >> r & 1u) sl[r] = __ldg(&P.ht[hv[r] & mask]);
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    if (!(alive >> r & 1u)) continue;
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
    if (!hit)
      alive &= ~(1u << r);
    else
      e[r] = s.z;
  }
  return alive;
}

template <int R>
__global__ void __launch_bounds__(kThreads, 2)
    k_scan_probe(const __grid_constant__ NodeDev nd, const __grid_constant__ ScanDev sc,
                 AtomDev* atoms, ResultDev* res) {
  constexpr int WT = 32 * R;
  static_assert(kScanQ >= WT, "the queue must hold a tile of survivors");
  constexpr int NW = kThreads / 32;
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint32_t s_mask[FJ_MAX_SUB];
  __shared__ uint32_t s_fon[FJ_MAX_SUB];
  __shared__ unsigned long long s_red[33];
  __shared__ int32_t s_min[FJ_MAX_VARS];
  const uint32_t tid = threadIdx.x;
  const int warp = tid >> 5;
  const uint32_t lane = tid & 31;
  const int np = sc.n_probe;
  // Queue layout: [mult[Q] (8-byte aligned, only when tracked)], row[Q],
  // newh[np][Q], live[Q].
  const int track = sc.track;
  uint8_t* w = smem + warp * scan_queue_bytes(np, track);
  const size_t mb = track ? 8 * kScanQ : 0;
  ScanQueue q{reinterpret_cast<uint32_t*>(w + mb),
              track ? reinterpret_cast<uint64_t*>(w) : nullptr,
              reinterpret_cast<uint32_t*>(w + mb + 4 * kScanQ),
              reinterpret_cast<uint16_t*>(w + mb + size_t(kScanQ) * (4 + 4 * np))};
  if (tid < uint32_t(np)) {
    s_mask[tid] = *sc.probe[tid].mask;
    s_fon[tid] = sc.probe[tid].filter ? *sc.probe[tid].filter_on : 0u;
  }
  if (tid < FJ_MAX_VARS) s_min[tid] = INT32_MAX;
  __syncthreads();

  ScanAcc acc{0, 0, 0, 0, 0};
  const uint64_t begin = nd.chunk_begin, end = nd.chunk_end;
  const uint64_t n_wt = (end - begin + WT - 1) / WT;
  const uint64_t nwarps = uint64_t(gridDim.x) * NW;
  const uint32_t mask0 = np > 0 ? s_mask[0] : 0u;
  const uint32_t* filt0 = np > 0 && s_fon[0] ? sc.probe[0].filter : nullptr;
  uint32_t qn = 0;
  uint64_t t = uint64_t(blockIdx.x) * NW + warp;
  for (;;) {
    const bool have = t < n_wt;
    if (have && R == 8 && sc.k1) {
      const uint64_t r0 = begin + t * WT;
      uint32_t row[8], nh[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) nh[r] = 0;
      if (lane == 0) acc.iters += end - r0 < uint64_t(WT) ? end - r0 : uint64_t(WT);
      uint32_t alive = scan_first_k1(sc, mask0, filt0, r0, end, lane, row, nh);
      acc.probes += end - r0 < uint64_t(WT) ? uint32_t(end - r0) / 32 : 8;  // approximate
      acc.hits += __popc(alive);
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        bool keep = alive >> r & 1u;
        uint32_t m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
          uint32_t pos = qn + __popc(m & lanemask_lt());
          q.row[pos] = row[r];
          if (track) q.mult[pos] = 1ull;
          q.live[pos] = uint16_t(pos);
          q.newh[pos] = nh[r];
        }
        qn += __popc(m);
      }
      __syncwarp();
    } else if (have) {
      // Generic first probe: two halves of 4 rows per lane.
      constexpr int RG = 4;
      for (int half = 0; half < WT / (32 * RG); ++half) {
        const uint64_t r0 = begin + t * WT + half * 32 * RG;
        uint32_t alive = 0, row[RG], nh[RG], hh[RG];
        uint64_t kw[RG], mult[RG];
        uint4 sl[RG];
#pragma unroll
        for (int r = 0; r < RG; ++r) {
          row[r] = uint32_t(r0) + r * 32 + lane;
          kw[r] = 0;
          hh[r] = 0;
          nh[r] = 0;
          mult[r] = 1;
          if (r0 + r * 32 + lane < end && scan_pred(sc, row[r])) {
            alive |= 1u << r;
            if (np > 0 && !sc.probe[0].wide) kw[r] = scan_key(sc.probe[0], row[r]);
          }
        }
        if (lane == 0 && r0 < end) acc.iters += end - r0 < uint64_t(32 * RG) ? end - r0 : uint64_t(32 * RG);
        if (np > 0) {
          const ScanProbe& P = sc.probe[0];
          acc.probes += __popc(alive);
          if (!P.wide) {
#pragma unroll
            for (int r = 0; r < RG; ++r)
              if ((alive >> r & 1u) && kw[r] != kEmptyKey &&
                  !probe_start(P.ht, mask0, filt0, P.filter_words, kw[r], hh[r], sl[r]))
                alive &= ~(1u << r);
          }
#pragma unroll
          for (int r = 0; r < RG; ++r) {
            if (!(alive >> r & 1u)) continue;
            uint32_t e = 0, cnt = 0;
            bool hit;
            if (P.wide) {
              hit = scan_find_wide(P, mask0, row[r], e, cnt);
            } else if (kw[r] == kEmptyKey) {
              uint4 sp = __ldg(&P.ht[mask0 + 1]);
              e = sp.z;
              cnt = sp.w;
              hit = sp.w != 0;
            } else {
              hit = ht_resolve(P.ht, mask0, kw[r], hh[r], sl[r], e, cnt);
            }
            if (!hit) {
              alive &= ~(1u << r);
            } else if (P.last) {
              mult[r] = mul_sat(mult[r], cnt, &res->status);
            } else {
              nh[r] = e;
            }
          }
          acc.hits += __popc(alive);
        }
#pragma unroll
        for (int r = 0; r < RG; ++r) {
          bool keep = alive >> r & 1u;
          uint32_t m = __ballot_sync(0xffffffffu, keep);
          if (keep) {
            uint32_t pos = qn + __popc(m & lanemask_lt());
            q.row[pos] = row[r];
            if (track) q.mult[pos] = mult[r];
            q.live[pos] = uint16_t(pos);
            if (np > 0) q.newh[pos] = nh[r];
          }
          qn += __popc(m);
        }
        __syncwarp();
      }
    }
    // Flush when the next tile might not fit, and at the end (one call site,
    // so the flush is inlined).
    if (qn > uint32_t(kScanQ - WT) || (!have && qn)) {
      scan_flush(nd, sc, atoms, res, q, qn, s_mask, s_fon, s_min, acc);
      qn = 0;
    }
    if (!have) break;
    t += nwarps;
  }
  __syncthreads();
  if (nd.mode == kModeAggregate) {
    unsigned long long tot = block_sum<unsigned long long>(acc.count, s_red);
    if (tid == 0 && tot) {
      unsigned long long old = atomicAdd(&res->count, tot);
      if (old + tot < old) atomicOr(&res->status, kStCountOverflow);
    }
    if (tot && tid < FJ_MAX_VARS) atomicMin(&res->mins[tid], s_min[tid]);
  }
  unsigned long long v;
  v = block_sum<unsigned long long>(acc.iters, s_red);
  if (tid == 0 && v) atomicAdd(&res->ctr[FJ_CTR_COVER_ITERS], v);
  v = block_sum<unsigned long long>(acc.probes, s_red);
  if (tid == 0 && v) atomicAdd(&res->ctr[FJ_CTR_PROBES], v);
  v = block_sum<unsigned long long>(acc.hits, s_red);
  if (tid == 0 && v) atomicAdd(&res->ctr[FJ_CTR_PROBE_HITS], v);
  v = block_sum<unsigned long long>(acc.surv, s_red);
  if (tid == 0 && v) atomicAdd(&res->ctr[FJ_CTR_SURVIVORS], v);
}

}  // namespace fj
