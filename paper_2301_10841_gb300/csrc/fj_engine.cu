// libfj host engine: contexts, relations, plan compilation and the node
// driver.  All compute runs in the kernels of fj_kernels.cuh / fj_exec.cuh.
//
// Execution of a prepared plan (paper Section 3.3 build + join phases, with
// COLT making the build phase lazy, Section 4.2):
//   1. reset the per-execution COLT state (nothing is built yet);
//   2. run node 0 on the single empty partial tuple;
//   3. for node k: choose a cover per partial tuple and request the COLT
//      levels it will probe or iterate as a map (k_choose); force exactly
//      those (the k_force_* sequence, batched over atoms); count each tuple's
//      cover elements and prefix-sum them (k_fanout + scan); expand the
//      position space in chunks bounded by the next node's buffer
//      (k_expand), recursing into node k+1 after every chunk;
//   4. the last expanded node aggregates (COUNT, MIN, with the remaining
//      single-vector nodes folded in as product factors) or materializes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "fj_ctx_access.h"
#include "fj_scan.cuh"
#include "fj_plan.h"

using namespace fj;

struct fj_rel {
  fj_ctx* ctx = nullptr;
  std::string name;
  std::vector<const int32_t*> cols;
  uint64_t n_rows = 0;
  std::vector<void*> owned;
};

struct fj_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;
  int n_sm = 0;
  uint64_t* h_total = nullptr;  // pinned
  void* d_partials = nullptr;   // scan partials: kMaxScanJobs x kScanBlocks x 8 B
  std::set<fj_prepared*> preps;  // live prepared plans (released by destroy)
  std::set<fj_rel*> rels;        // live relations (released by destroy)
};

namespace {

constexpr int kMaxScanJobs = FJ_MAX_ATOMS;

struct Error {
  fj_status st;
  std::string msg;
};

[[noreturn]] void fail(fj_status st, const std::string& msg) { throw Error{st, msg}; }

void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      fail(FJ_ERR_OOM, std::string(what) + ": out of device memory");
    }
    fail(FJ_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
}

#define CK(x) cuda_check((x), #x)
#define CK_LAUNCH(what) cuda_check(cudaGetLastError(), what)

template <typename T>
T* dalloc(fj_ctx* c, size_t n) {
  void* p = nullptr;
  CK(cudaMallocFromPoolAsync(&p, std::max<size_t>(n, 1) * sizeof(T), c->pool, c->stream));
  return static_cast<T*>(p);
}

void dfree(fj_ctx* c, void* p) {
  if (p) cudaFreeAsync(p, c->stream);
}

template <typename F>
fj_status guarded(F&& f) {
  try {
    f();
    set_error("");
    return FJ_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.st;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return FJ_ERR_OOM;
  }
}

uint32_t pow2_at_least(uint64_t x) {
  uint64_t c = 16;
  while (c < x) c <<= 1;
  if (c > (1ull << 31)) fail(FJ_ERR_UNSUPPORTED, "hash level too large");
  return uint32_t(c);
}

int blocks_for(uint64_t work, int per_block, int cap) {
  uint64_t b = (work + per_block - 1) / per_block;
  return int(std::max<uint64_t>(1, std::min<uint64_t>(b, uint64_t(cap))));
}

}  // namespace

// ---------------------------------------------------------------------------
// Prepared plans.
// ---------------------------------------------------------------------------

struct ItemsBuf {
  int32_t* var[FJ_MAX_VARS] = {};
  uint32_t* h[FJ_MAX_ATOMS] = {};
  uint64_t* mult = nullptr;
  uint8_t* choice = nullptr;
  uint64_t* fan = nullptr;
  uint64_t* scan = nullptr;
  uint64_t* total = nullptr;
  uint32_t* n = nullptr;
  uint32_t cap = 0;
};

struct AtomPlan {
  int n_levels = 0;                     // schema levels
  std::vector<int> level_node;          // node of each schema level
  std::vector<std::vector<int>> level_vars;
  std::vector<bool> may_force;          // per L index (1..n_levels)
};

struct fj_prepared {
  fj_ctx* ctx = nullptr;
  PQuery q;
  PPlan plan;
  fj_exec_opts opts{};
  std::vector<int> min_vars;
  std::vector<fj_rel*> rels;
  std::vector<AtomPlan> ap;
  std::vector<AtomDev> host_atoms;
  AtomDev* d_atoms = nullptr;
  std::vector<void*> allocs;
  int n_nodes = 0;
  int tail_start = 0;  // first node folded into the aggregation epilogue
  int last = 0;        // last expanded node
  std::vector<NodeDev> nd;
  std::vector<ItemsBuf> items;             // items[k]: input of node k
  std::vector<std::vector<int2>> jobs;     // force jobs per node
  std::vector<int2*> d_jobs;
  int2* d_level_jobs = nullptr;            // [atom][level] single jobs
  std::vector<uint32_t> max_rows_job;      // per node: largest atom among its jobs
  std::vector<uint32_t> max_req_job;
  std::vector<bool> roots_only;            // per node: every force job is a root
  int32_t* d_out = nullptr;
  uint64_t out_cap = 0;
  bool materialize = false;
  bool factorized = false;  // FJ_OUT_FACTORIZED
  int out_width = 0;        // int32 words per output row (either mode)
  size_t smem_expand = 0;
  int expand_blocks_per_sm = 1;
  int expand_r = 8;
  // Node 0 streamed from its cover's base table (the scan pipeline).
  bool scan0 = false;
  ScanDev sc0{};
  int fuse_blocks = 0;  // > 0: node 0 runs as one k_scan_fused launch of this many blocks
  bool device_totals = false;  // node totals stay on the device (batched runs)
  ResultDev* d_res = nullptr;  // this query's result block (device)
  void* d_partials = nullptr;  // its scan partials (queries of a batch may run concurrently)
  ResultDev* h_res = nullptr;  // and its pinned host copy
  RootsState* roots_state = nullptr;  // k_force_roots barrier
  int roots_grid = 0;                 // > 0: root-only forces run as one cooperative launch
  int roots_set = 0;                  // counter set of the next k_force_roots launch
  uint64_t kernels = 0;
  uint64_t chunks = 0;
  bool explicit_built = false;  // levels built outside the join since reset
  // FJ_FLAG_TIMING: event pool and the pairs recorded by this execution.
  std::vector<cudaEvent_t> events;
  size_t n_events = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> t_expand, t_build;
  cudaEvent_t t_first = nullptr, t_last = nullptr;

  bool timing() const { return opts.flags & FJ_FLAG_TIMING; }
  cudaEvent_t mark() {
    if (n_events == events.size()) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      events.push_back(e);
    }
    cudaEvent_t e = events[n_events++];
    // Inside a stream capture (a batch captured into a CUDA graph) the event
    // becomes an event-record node of the graph, recorded at every launch.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(ctx->stream, &cs));
    if (cs == cudaStreamCaptureStatusActive)
      CK(cudaEventRecordWithFlags(e, ctx->stream, cudaEventRecordExternal));
    else
      CK(cudaEventRecord(e, ctx->stream));
    return e;
  }

  template <typename T>
  T* alloc(size_t n) {
    T* p = dalloc<T>(ctx, n);
    allocs.push_back(p);
    return p;
  }
};

namespace {

// Scans ---------------------------------------------------------------------

template <typename T, typename Op>
void run_scan(fj_prepared* P, Op op, int n_jobs, uint64_t ub_n) {
  fj_ctx* c = P->ctx;
  int nb = blocks_for(ub_n, 4096, kScanBlocks);
  dim3 g(nb, n_jobs);
  k_scan_reduce<T, Op><<<g, kThreads, 0, c->stream>>>(op, static_cast<T*>(P->d_partials));
  k_scan_mid<T, Op><<<dim3(1, n_jobs), 1024, 0, c->stream>>>(op, static_cast<T*>(P->d_partials),
                                                             nb);
  k_scan_down<T, Op><<<g, kThreads, 0, c->stream>>>(op, static_cast<T*>(P->d_partials));
  CK_LAUNCH("scan");
  P->kernels += 3;
}

// COLT forcing of a batch of (atom, level) jobs.  `roots` says every job is
// a root level (its single parent needs no row-offset or child-first scan).
void force(fj_prepared* P, const int2* d_jobs, int n_jobs, uint32_t ub_rows, uint32_t ub_req,
           bool roots, bool request_all = false) {
  if (n_jobs == 0) return;
  fj_ctx* c = P->ctx;
  cudaStream_t s = c->stream;
  ForceJobs fj{P->d_atoms, d_jobs, n_jobs};
  cudaEvent_t t0 = P->timing() ? P->mark() : nullptr;
  if (roots && P->roots_grid > 0) {
    RootsState* cs = P->roots_state;  // zeroed by k_reset at the start of the execution
    int set = P->roots_set;
    P->roots_set ^= 1;
    int all = request_all ? 1 : 0;
    int test_timeout = (P->opts.flags & FJ_FLAG_TEST_TIMEOUT) ? 1 : 0;
    ResultDev* rd = P->d_res;
    uint32_t spin = uint32_t(std::min<uint64_t>(P->opts.spin_limit, 0xffffffffull));
    void* args[] = {&fj, &cs, &set, &all, &test_timeout, &rd, &spin};
    CK(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&k_force_roots),
                                   dim3(P->roots_grid), dim3(kRootThreads), args, kRootSmem, s));
    if (test_timeout) {
      // The test of the bounded waits stops the execution here: nothing may
      // run on the levels the build left unbuilt.
      CK(cudaMemcpyAsync(P->h_res, P->d_res, sizeof(ResultDev), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (P->h_res->status & kStTimeout) fail(FJ_ERR_TIMEOUT, "a bounded device wait ran out");
    }
    P->kernels += 1;
    if (t0) P->t_build.emplace_back(t0, P->mark());
    return;
  }
  int cap = c->n_sm * 8;
  int g_rows = blocks_for(ub_rows, kThreads * 4, cap);
  int g_ht = blocks_for(uint64_t(ub_rows) * 2 + 2, kThreads * 4, cap);
  k_force_count<<<dim3(g_rows, n_jobs), kThreads, 0, s>>>(fj);
  k_force_prepare<<<n_jobs, 32, 0, s>>>(fj);
  k_force_clear<<<dim3(g_ht, n_jobs), kThreads, 0, s>>>(fj);
  CK_LAUNCH("force prepare");
  P->kernels += 3;
  if (!roots) run_scan<uint32_t>(P, RowOffOp{P->d_atoms, d_jobs}, n_jobs, ub_req);
  k_force_insert<<<dim3(g_rows, n_jobs), kThreads, 0, s>>>(fj, P->d_res);
  CK_LAUNCH("force insert");
  P->kernels += 1;
  if (!roots) run_scan<uint32_t>(P, ChildFirstOp{P->d_atoms, d_jobs}, n_jobs, ub_req);
  k_force_assign<<<dim3(g_rows, n_jobs), kThreads, 0, s>>>(fj);
  k_force_scatter<<<dim3(g_rows, n_jobs), kThreads, 0, s>>>(fj);
  k_force_finish<<<dim3(g_rows, n_jobs), kThreads, 0, s>>>(fj, P->d_res);
  k_force_reset_req<<<n_jobs, 32, 0, s>>>(fj);
  CK_LAUNCH("force finish");
  P->kernels += 4;
  if (t0) P->t_build.emplace_back(t0, P->mark());
}

template <int R>
void launch_expand_r(fj_prepared* P, int grid, const NodeDev& nd) {
  fj_ctx* c = P->ctx;
  if (nd.dynamic)
    k_expand<R><<<grid, kThreads, P->smem_expand, c->stream>>>(nd, P->d_atoms, P->d_res);
  else
    k_expand_static<R><<<grid, kThreads, P->smem_expand, c->stream>>>(nd, P->d_atoms, P->d_res);
}

constexpr int kMaxDevicesAttr = 64;

template <int R>
void expand_attrs(size_t smem, int* blocks) {
  const void* fns[2] = {reinterpret_cast<const void*>(&k_expand<R>),
                        reinterpret_cast<const void*>(&k_expand_static<R>)};
  // The dynamic shared memory limit is one setting per kernel (and device)
  // for the whole process: only ever raise it, so a prepared plan needing
  // less never lowers it under one needing more.
  static std::mutex mu;
  static size_t limit[kMaxDevicesAttr] = {};
  int dev = 0;
  CK(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = limit[dev < kMaxDevicesAttr && dev >= 0 ? dev : 0];
    if (smem > cur) {
      for (const void* fn : fns)
        CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
      cur = smem;
    }
  }
  *blocks = 1 << 20;
  for (const void* fn : fns) {
    int b = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kThreads, smem));
    *blocks = std::min(*blocks, std::max(1, b));
  }
}

void expand_setup(int r, size_t smem, int* blocks) {
  switch (r) {
    case 1: expand_attrs<1>(smem, blocks); break;
    case 2: expand_attrs<2>(smem, blocks); break;
    case 4: expand_attrs<4>(smem, blocks); break;
    case 8: expand_attrs<8>(smem, blocks); break;
    default: expand_attrs<16>(smem, blocks); break;
  }
}

constexpr int kScanR = 4;  // rows per thread per block iteration of k_scan_first

constexpr int kFuseR = 4;  // survivors per lane per round in k_scan_fused

// Node 0 through the scan pipeline for positions [c0, c1) of its cover.
void run_scan_chunk(fj_prepared* P, NodeDev& nd) {
  fj_ctx* c = P->ctx;
  cudaStream_t s = c->stream;
  const ScanDev& sc = P->sc0;
  if (P->fuse_blocks > 0) {
    k_scan_fused<kFuseR><<<P->fuse_blocks, kFuseThreads, kFuseSmem, s>>>(nd, sc, P->d_atoms,
                                                                         P->d_res);
    CK_LAUNCH("scan fused");
    P->kernels += 1;
    return;
  }
  int cap_blocks = c->n_sm * 8;
  k_scan_reset<<<1, 32, 0, s>>>(sc);
  int g1 = blocks_for(nd.chunk_end - nd.chunk_begin, kScanR * kThreads, cap_blocks);
  k_scan_first<kScanR><<<g1, kThreads, 0, s>>>(nd, sc, P->d_res);
  CK_LAUNCH("scan first");
  P->kernels += 2;
  // Survivors are about a tenth of the rows in a selective join; size the
  // grid for a quarter of them, the loop strides over the rest.
  uint64_t est = std::max<uint64_t>(1, (nd.chunk_end - nd.chunk_begin) / 4);
  int g2 = blocks_for(est, 4 * kThreads, cap_blocks);
  k_scan_rest<4><<<g2, kThreads, 0, s>>>(nd, sc, P->d_atoms, P->d_res);
  CK_LAUNCH("scan rest");
  P->kernels += 1;
}

void launch_expand(fj_prepared* P, int grid, const NodeDev& nd) {
  switch (P->expand_r) {
    case 1: launch_expand_r<1>(P, grid, nd); break;
    case 2: launch_expand_r<2>(P, grid, nd); break;
    case 4: launch_expand_r<4>(P, grid, nd); break;
    case 8: launch_expand_r<8>(P, grid, nd); break;
    default: launch_expand_r<16>(P, grid, nd); break;
  }
}

void sync_read_total(fj_prepared* P, const uint64_t* d_total, uint64_t* out) {
  fj_ctx* c = P->ctx;
  CK(cudaMemcpyAsync(c->h_total, d_total, sizeof(uint64_t), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *out = *c->h_total;
}

void run_node(fj_prepared* P, int k, uint64_t ub_items) {
  fj_ctx* c = P->ctx;
  cudaStream_t s = c->stream;
  NodeDev nd = P->nd[k];
  int g_items = blocks_for(ub_items, kThreads, c->n_sm * 8);
  // Node 0 over a base-table cover whose jobs are all roots: its single
  // root tuple reaches every one of them, so the root build requests them
  // itself and no choice kernel runs.
  const bool roots_direct = k == 0 && P->scan0 && nd.single_item && !nd.dynamic &&
                            P->roots_only[0] && P->roots_grid > 0 && !P->jobs[0].empty();
  if (!roots_direct) {
    k_choose<<<g_items, kThreads, 0, s>>>(nd, P->d_atoms);
    CK_LAUNCH("choose");
    P->kernels += 1;
  }
  force(P, P->d_jobs[k], int(P->jobs[k].size()), P->max_rows_job[k], P->max_req_job[k],
        P->roots_only[k], roots_direct);
  uint64_t total = 0;
  const SubDev& S0 = nd.sub[0];
  bool use_scan = k == 0 && P->scan0;
  bool host_known = use_scan || (k == 0 && !nd.dynamic && S0.last && S0.lvl == 0 &&
                                 !(P->opts.flags & (FJ_FLAG_EAGER_ALL | FJ_FLAG_EAGER_ROOT)) &&
                                 !P->explicit_built);
  bool device_total = false;  // the total stays on the device (batches)
  if (host_known) {
    // The single root tuple iterates the cover's base table directly.
    total = P->host_atoms[S0.atom].n_rows;
  } else {
    k_fanout<<<g_items, kThreads, 0, s>>>(nd, P->d_atoms);
    CK_LAUNCH("fanout");
    P->kernels += 1;
    run_scan<uint64_t>(P,
                       FanScanOp{nd.fan, nd.scan, nd.total, nd.n_items, nd.single_item},
                       1, ub_items);
    if (P->device_totals) {
      // One chunk as large as the next node's input buffer (or unbounded
      // for the last node); the kernel clamps to the device total and
      // flags a total the chunk cannot hold.
      device_total = true;
      total = nd.mode == kModeItems ? uint64_t(P->items[k + 1].cap) : ~0ull >> 1;
      nd.check_total = 1;
    } else {
      sync_read_total(P, nd.total, &total);
    }
  }
  if (total == 0) return;
  bool items_mode = nd.mode == kModeItems;
  uint64_t step = items_mode ? P->items[k + 1].cap : total;
  if (use_scan) step = std::min<uint64_t>(step, P->sc0.cap);
  for (uint64_t c0 = 0; c0 < total; c0 += step) {
    nd.chunk_begin = c0;
    nd.chunk_end = std::min(total, c0 + step);
    if (items_mode) CK(cudaMemsetAsync(P->items[k + 1].n, 0, sizeof(uint32_t), s));
    cudaEvent_t t0 = P->timing() ? P->mark() : nullptr;
    if (use_scan) {
      run_scan_chunk(P, nd);
    } else {
      int grid = device_total ? c->n_sm * P->expand_blocks_per_sm
                              : blocks_for(nd.chunk_end - c0, nd.tile,
                                           c->n_sm * P->expand_blocks_per_sm);
      launch_expand(P, grid, nd);
      CK_LAUNCH("expand");
      P->kernels += 1;
    }
    if (t0) P->t_expand.emplace_back(t0, P->mark());
    P->chunks += 1;
    if (items_mode) run_node(P, k + 1, nd.chunk_end - c0);
  }
}

}  // namespace

// Compile query + plan into device descriptors and allocate COLT storage.
static void compile(fj_prepared* P) {
  fj_ctx* c = P->ctx;
  const PQuery& q = P->q;
  const PPlan& plan = P->plan;
  const fj_exec_opts& o = P->opts;
  int na = int(q.atom_vars.size());
  int nn = int(plan.size());
  P->n_nodes = nn;
  P->materialize = o.out_mode == FJ_OUT_MATERIALIZE;
  P->factorized = o.out_mode == FJ_OUT_FACTORIZED;
  bool dyn_policy = o.cover_policy == FJ_COVER_FEWEST || o.cover_policy == FJ_COVER_LEARNED;

  // Per-atom schema levels and which of them may be forced.
  P->ap.assign(na, {});
  std::vector<std::vector<int>> lvl_of(nn);  // per node, per sub: schema level
  std::vector<std::vector<int>> cov(nn);
  for (int k = 0; k < nn; ++k) {
    cov[k] = covers(plan, k);
    for (const PSub& sa : plan[k]) {
      AtomPlan& A = P->ap[sa.atom];
      lvl_of[k].push_back(A.n_levels);
      A.level_node.push_back(k);
      A.level_vars.push_back(sa.vars);
      A.n_levels++;
    }
  }
  for (int a = 0; a < na; ++a) P->ap[a].may_force.assign(P->ap[a].n_levels + 2, false);
  std::vector<int> dynamic(nn, 0);
  for (int k = 0; k < nn; ++k) {
    dynamic[k] = dyn_policy && cov[k].size() > 1;
    for (int s = 0; s < int(plan[k].size()); ++s) {
      const PSub& sa = plan[k][s];
      AtomPlan& A = P->ap[sa.atom];
      int l = lvl_of[k][s];
      bool last = l == A.n_levels - 1;
      bool probed = dynamic[k] ? true : s != 0;
      bool map_iter = !last;
      if (probed || map_iter) A.may_force[l + 1] = true;
    }
  }
  // Eager builds (the simple trie and simple lazy trie ablations) force
  // every level (or every root) from the top down, stopping above the first
  // level of more than three variables, which stays a vector (it is then
  // only ever iterated: a probed level of that width is refused below).
  if (o.flags & (FJ_FLAG_EAGER_ALL | FJ_FLAG_EAGER_ROOT))
    for (int a = 0; a < na; ++a) {
      const int top = (o.flags & FJ_FLAG_EAGER_ALL) ? P->ap[a].n_levels : 1;
      for (int l = 1; l <= top; ++l) {
        if (P->ap[a].level_vars[l - 1].size() > 3) break;
        P->ap[a].may_force[l] = true;
      }
    }
  // A level can only be forced below an entry of the level above it.
  for (int a = 0; a < na; ++a)
    for (int l = P->ap[a].n_levels; l >= 2; --l)
      if (P->ap[a].may_force[l]) P->ap[a].may_force[l - 1] = true;
  // Key-arity limits of forced levels.
  for (int a = 0; a < na; ++a)
    for (int l = 1; l <= P->ap[a].n_levels; ++l) {
      if (!P->ap[a].may_force[l]) continue;
      int nk = int(P->ap[a].level_vars[l - 1].size());
      if (nk > 3)
        fail(FJ_ERR_UNSUPPORTED,
             "a probed (hashed) subatom holds at most 3 variables (atom " + std::to_string(a) +
                 ")");
    }

  // Atom device descriptors and COLT storage.
  float load = o.load_factor > 0.f ? o.load_factor : 0.25f;
  if (load > 0.9f) load = 0.9f;
  P->host_atoms.assign(na, AtomDev{});
  for (int a = 0; a < na; ++a) {
    fj_rel* r = P->rels[a];
    AtomDev& D = P->host_atoms[a];
    const AtomPlan& A = P->ap[a];
    D.n_rows = uint32_t(r->n_rows);
    D.n_vars = int(q.atom_vars[a].size());
    D.load = load;
    D.n_levels = A.n_levels + 1;
    if (D.n_levels > kMaxLevels) fail(FJ_ERR_UNSUPPORTED, "too many levels");
    bool any_force = false;
    for (int l = 1; l <= A.n_levels; ++l) any_force |= A.may_force[l];
    uint32_t n = std::max<uint32_t>(D.n_rows, 1);
    if (any_force) {
      D.perm = P->alloc<uint32_t>(n);
      D.tmp_row = P->alloc<uint32_t>(n);
      D.tmp_slot = P->alloc<uint32_t>(n);
      D.newslots = P->alloc<uint32_t>(n);
    }
    // L[0]: the virtual root entry.
    LevelDev& R = D.L[0];
    R.begin = P->alloc<uint32_t>(1);
    R.count = P->alloc<uint32_t>(1);
    R.child_state = P->alloc<uint32_t>(1);
    R.child_first = P->alloc<uint32_t>(1);
    R.child_nkeys = P->alloc<uint32_t>(1);
    R.fill = P->alloc<uint32_t>(1);
    R.entries_cap = 1;
    for (int l = 1; l <= A.n_levels; ++l) {
      LevelDev& L = D.L[l];
      const auto& lv = A.level_vars[l - 1];
      L.nk = int(lv.size());
      for (int j = 0; j < L.nk && j < 3; ++j) {
        const auto& av = q.atom_vars[a];
        L.kcol[j] = int(std::find(av.begin(), av.end(), lv[j]) - av.begin());
      }
      L.wide = L.nk == 3 || (L.nk == 2 && l > 1);
      if (!A.may_force[l]) continue;
      L.entries_cap = n;
      L.begin = P->alloc<uint32_t>(n);
      L.count = P->alloc<uint32_t>(n);
      L.fill = P->alloc<uint32_t>(n);
      L.key = P->alloc<uint64_t>(n);
      L.ht_cap_max = pow2_at_least(uint64_t(double(n) / load) + 1);
      L.ht = P->alloc<uint4>((size_t(L.ht_cap_max) + 1) * (L.wide ? 2 : 1));
      if (l == 1) {
        L.sbegin = P->alloc<uint32_t>(size_t(L.ht_cap_max) + 1);
        L.slot_of = P->alloc<uint32_t>(n);
      }
      L.ht_state = kHtUnknown;  // fresh memory: the first build clears it all
      L.n_listed = 0;
      if (!L.wide) {
        // Bloom filter: about 8 bits per row, 256 B to 32 KB.
        uint32_t words = 64;
        while (words < 8192 && uint64_t(words) * 32 < uint64_t(n) * 8) words <<= 1;
        L.filter_words = words;
        L.filter = P->alloc<uint32_t>(words);
      }
      L.req_cap = D.L[l - 1].entries_cap;
      L.req = P->alloc<uint32_t>(L.req_cap);
      L.rowoff = P->alloc<uint32_t>(size_t(L.req_cap) + 1);
      LevelDev& Pl = D.L[l - 1];
      if (!Pl.child_state) {
        Pl.child_state = P->alloc<uint32_t>(Pl.entries_cap);
        Pl.child_first = P->alloc<uint32_t>(Pl.entries_cap);
        Pl.child_nkeys = P->alloc<uint32_t>(Pl.entries_cap);
      }
    }
  }

  // Tail detection (aggregate modes): trailing single-subatom nodes that
  // iterate their atom's last level below the root.
  P->tail_start = nn;
  if (!P->materialize) {
    while (P->tail_start - 1 >= 1) {
      int k = P->tail_start - 1;
      const PSub& sa = plan[k][0];
      int l = lvl_of[k][0];
      bool eligible = plan[k].size() == 1 && l == P->ap[sa.atom].n_levels - 1 && l >= 1;
      if (!eligible) break;
      P->tail_start--;
    }
  }
  P->last = P->tail_start - 1;

  // Live variables and handles per node input.
  uint64_t outvars = 0;
  if (P->materialize || P->factorized)
    for (int v : q.head) outvars |= 1ull << v;
  else
    for (int v : P->min_vars) outvars |= 1ull << v;
  std::vector<uint64_t> live_in(nn + 1, 0);
  std::vector<uint32_t> hand_in(nn + 1, 0);
  for (int k = 0; k <= P->last; ++k) {
    uint64_t need = outvars;
    for (int j = k; j <= P->last; ++j) need |= vs_mask(plan[j]);
    live_in[k] = avs_mask(plan, k) & need;
    for (int a = 0; a < na; ++a) {
      int consumed = 0;
      for (int j = 0; j < k; ++j)
        for (const PSub& sa : plan[j]) consumed += sa.atom == a;
      if (consumed >= 1 && consumed < P->ap[a].n_levels) hand_in[k] |= 1u << a;
    }
  }

  // Batch tile (R batch elements per thread) and shared memory.
  uint32_t tile = o.batch_size ? o.batch_size : 1024;
  int R = 1;
  while (R < 16 && uint32_t(R * kThreads) < tile) R <<= 1;
  int max_sub = 1;
  for (int k = 0; k < nn; ++k) max_sub = std::max<int>(max_sub, int(plan[k].size()));
  // Static kernel: mult, item, element, per-subatom handles, two lists.
  auto smem_for = [&](int r) { return size_t(r) * kThreads * (8 + 4 + 4 + 4 * max_sub + 4); };
  while (R > 1 && smem_for(R) > 160 * 1024) R >>= 1;
  P->expand_r = R;
  P->smem_expand = smem_for(R);
  tile = uint32_t(R * kThreads);
  expand_setup(R, P->smem_expand, &P->expand_blocks_per_sm);

  // Item buffers.
  uint64_t max_rows = 1;
  for (fj_rel* r : P->rels) max_rows = std::max<uint64_t>(max_rows, r->n_rows);
  uint32_t cap = uint32_t(std::min<uint64_t>(1ull << 24, std::max<uint64_t>(1ull << 16, max_rows)));
  cap &= ~4095u;  // chunks start on a 16-byte boundary of every column
  P->items.assign(nn + 1, ItemsBuf{});
  for (int k = 0; k <= P->last; ++k) {
    ItemsBuf& B = P->items[k];
    uint32_t bc = k == 0 ? 1u : cap;
    B.cap = bc;
    if (k > 0) {
      for (int v = 0; v < FJ_MAX_VARS; ++v)
        if (live_in[k] >> v & 1) B.var[v] = P->alloc<int32_t>(bc);
      for (int a = 0; a < na; ++a)
        if (hand_in[k] >> a & 1) B.h[a] = P->alloc<uint32_t>(bc);
      B.mult = P->alloc<uint64_t>(bc);
    }
    B.choice = P->alloc<uint8_t>(bc);
    B.fan = P->alloc<uint64_t>(bc);
    B.scan = P->alloc<uint64_t>(size_t(bc) + 1);
    B.total = P->alloc<uint64_t>(1);
    B.n = P->alloc<uint32_t>(1);
  }

  // One force job per (atom, level), for explicit builds.
  {
    std::vector<int2> all(size_t(na) * kMaxLevels);
    for (int a = 0; a < na; ++a)
      for (int l = 0; l < kMaxLevels; ++l) all[size_t(a) * kMaxLevels + l] = make_int2(a, l);
    P->d_level_jobs = P->alloc<int2>(all.size());
    CK(cudaMemcpyAsync(P->d_level_jobs, all.data(), sizeof(int2) * all.size(),
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  // Node descriptors and force jobs.
  P->nd.assign(nn, NodeDev{});
  P->jobs.assign(nn, {});
  P->d_jobs.assign(nn, nullptr);
  P->max_rows_job.assign(nn, 1);
  P->max_req_job.assign(nn, 1);
  P->roots_only.assign(nn, true);
  for (int k = 0; k <= P->last; ++k) {
    NodeDev& N = P->nd[k];
    std::memset(&N, 0, sizeof(N));
    N.n_sub = int(plan[k].size());
    N.dynamic = dynamic[k];
    N.tile = int(tile);
    std::memset(N.vpos, -1, sizeof(N.vpos));
    for (int s = 0; s < N.n_sub; ++s) {
      const PSub& sa = plan[k][s];
      SubDev& S = N.sub[s];
      S.atom = sa.atom;
      S.lvl = lvl_of[k][s];
      S.last = S.lvl == P->ap[sa.atom].n_levels - 1;
      S.nv = int(sa.vars.size());
      for (int j = 0; j < S.nv; ++j) {
        S.var[j] = sa.vars[j];
        const auto& av = q.atom_vars[sa.atom];
        S.col[j] = int(std::find(av.begin(), av.end(), sa.vars[j]) - av.begin());
        N.vpos[s][sa.vars[j]] = int8_t(j);
      }
      S.hslot = S.lvl >= 1 ? sa.atom : -1;
      S.bound_mask = 0;
      for (int j = 0; j < S.nv; ++j)
        if (avs_mask(plan, k) >> sa.vars[j] & 1) S.bound_mask |= 1u << j;
      S.is_cover = std::find(cov[k].begin(), cov[k].end(), s) != cov[k].end();
      if (P->ap[sa.atom].may_force[S.lvl + 1] && (dynamic[k] || s != 0 || !S.last)) {
        P->jobs[k].push_back(make_int2(sa.atom, S.lvl + 1));
        if (S.lvl + 1 != 1) P->roots_only[k] = false;
        P->max_rows_job[k] = std::max<uint32_t>(P->max_rows_job[k], P->host_atoms[sa.atom].n_rows);
        P->max_req_job[k] =
            std::max<uint32_t>(P->max_req_job[k], P->host_atoms[sa.atom].L[S.lvl].entries_cap);
      }
    }
    N.avs_mask = uint32_t(avs_mask(plan, k));
    const ItemsBuf& In = P->items[k];
    for (int v = 0; v < FJ_MAX_VARS; ++v) N.in_var[v] = In.var[v];
    for (int a = 0; a < na; ++a) N.in_h[a] = In.h[a];
    N.in_mult = k == 0 ? nullptr : In.mult;
    N.choice = In.choice;
    N.n_items = In.n;
    N.single_item = k == 0;
    N.fan = In.fan;
    N.scan = In.scan;
    N.total = In.total;
    N.track_mult = 1;
    auto touching = [&](int a) {
      for (int s = 0; s < N.n_sub; ++s)
        if (plan[k][s].atom == a) return s;
      return -1;
    };
    if (k < P->last) {
      N.mode = kModeItems;
      const ItemsBuf& Out = P->items[k + 1];
      for (int v = 0; v < FJ_MAX_VARS; ++v)
        if (Out.var[v]) {
          N.out_var_id[N.n_out_vars] = v;
          N.out_var[N.n_out_vars] = Out.var[v];
          N.n_out_vars++;
        }
      for (int a = 0; a < na; ++a) {
        N.out_h[a] = Out.h[a];
        N.out_h_src[a] = touching(a);
      }
      N.out_mult = Out.mult;
      N.out_n = Out.n;
      N.out_cap = Out.cap;
    } else if (!P->materialize) {
      N.mode = kModeAggregate;
      uint64_t bound = avs_mask(plan, k) | vs_mask(plan[k]);
      for (int i = 0; i < int(P->min_vars.size()); ++i) {
        int v = P->min_vars[i];
        if (bound >> v & 1) {
          N.min_var[N.n_min] = v;
          N.min_idx[N.n_min] = i;
          N.n_min++;
        }
      }
      for (int t = P->tail_start; t < nn; ++t) {
        const PSub& sa = plan[t][0];
        TailDev& T = N.tail[N.n_tail++];
        T.atom = sa.atom;
        T.lvl = lvl_of[t][0];
        T.hsrc = touching(sa.atom);
        for (int i = 0; i < int(P->min_vars.size()); ++i) {
          int v = P->min_vars[i];
          auto it = std::find(sa.vars.begin(), sa.vars.end(), v);
          if (it == sa.vars.end()) continue;
          const auto& av = q.atom_vars[sa.atom];
          T.min_idx[T.n_min] = i;
          T.min_col[T.n_min] = int(std::find(av.begin(), av.end(), v) - av.begin());
          T.n_min++;
        }
      }
      if (P->factorized) {
        // The union of products: rows of the head variables bound here,
        // the multiplicity, and each tail's vector.
        N.mode = kModeFactorized;
        N.n_pre = 0;
        for (int v : q.head)
          if (bound >> v & 1) N.pre_var[N.n_pre++] = v;
        P->out_width = N.n_pre + 2 + 2 * N.n_tail;
      }
    } else {
      N.mode = kModeMaterialize;
      N.n_head = int(q.head.size());
      for (int h = 0; h < N.n_head; ++h) N.head_var[h] = q.head[h];
      P->out_width = N.n_head;
    }
    if (!P->jobs[k].empty()) {
      P->d_jobs[k] = P->alloc<int2>(P->jobs[k].size());
      CK(cudaMemcpyAsync(P->d_jobs[k], P->jobs[k].data(), sizeof(int2) * P->jobs[k].size(),
                         cudaMemcpyHostToDevice, c->stream));
    }
  }
}

static void upload_atoms(fj_prepared* P, const fj_query* query) {
  fj_ctx* c = P->ctx;
  int na = int(P->q.atom_vars.size());
  for (int a = 0; a < na; ++a) {
    AtomDev& D = P->host_atoms[a];
    const fj_atom& fa = query->atoms[a];
    fj_rel* r = P->rels[a];
    for (int j = 0; j < fa.n_vars; ++j) {
      int col = fa.cols ? fa.cols[j] : j;
      if (col < 0 || col >= int(r->cols.size()))
        fail(FJ_ERR_INVALID_ARG, "atom " + std::to_string(a) + ": column index out of range");
      D.cols[j] = r->cols[col];
    }
    D.n_preds = fa.n_preds;
    for (int p = 0; p < fa.n_preds; ++p) {
      D.pred_col[p] = fa.preds[p].col;
      D.pred_op[p] = fa.preds[p].op;
      D.pred_val[p] = fa.preds[p].value;
    }
  }
  P->d_atoms = P->alloc<AtomDev>(na);
  CK(cudaMemcpyAsync(P->d_atoms, P->host_atoms.data(), sizeof(AtomDev) * na,
                     cudaMemcpyHostToDevice, c->stream));
}

// Resolve the static-cover fast path of every node: variable sources, the
// cover's arrays and the probed hash levels (device addresses of the masks,
// which kernels fill when the level is first forced).
static void finalize_nodes(fj_prepared* P) {
  const PPlan& plan = P->plan;
  const PQuery& q = P->q;
  for (int k = 0; k <= P->last; ++k) {
    NodeDev& N = P->nd[k];
    if (N.dynamic) continue;
    const SubDev& C = N.sub[0];
    const AtomDev& ca = P->host_atoms[C.atom];
    const ItemsBuf& In = P->items[k];
    for (int u = 0; u < FJ_MAX_VARS; ++u) {
      VarSrc& v = N.src[u];
      std::memset(&v, 0, sizeof(v));
      v.kind = kSrcItem;
      if ((N.avs_mask >> u) & 1u) {
        v.col = In.var[u];
        continue;
      }
      int j = N.vpos[0][u];
      if (j < 0) continue;
      if (C.last) {
        v.kind = kSrcRow;
        v.col = ca.cols[C.col[j]];
      } else if (ca.L[C.lvl + 1].wide) {
        v.kind = kSrcKeyWide;
        v.col = ca.cols[C.col[j]];
        v.perm = ca.perm;
        v.begin = ca.L[C.lvl + 1].begin;
      } else {
        v.kind = kSrcKey;
        v.key = ca.L[C.lvl + 1].key;
        v.nk = ca.L[C.lvl + 1].nk;
        v.pos = j;
      }
    }
    N.cover_root_mat = &P->d_atoms[C.atom].root_mat;
    N.cover_perm = ca.perm;
    N.cover_begin = ca.L[C.lvl].begin;
    N.cover_first = ca.L[C.lvl].child_first;
    N.cover_hsrc = C.lvl >= 1 ? In.h[C.atom] : nullptr;
    N.n_probe = 0;
    for (int s = 1; s < N.n_sub; ++s) {
      const SubDev& S = N.sub[s];
      const AtomDev& a = P->host_atoms[S.atom];
      ProbeDev& Pd = N.probe[N.n_probe++];
      Pd.sub = s;
      Pd.nv = S.nv;
      for (int j = 0; j < 3; ++j) Pd.var[j] = j < S.nv ? S.var[j] : 0;
      Pd.ht = a.L[S.lvl + 1].ht;
      Pd.mask = &P->d_atoms[S.atom].L[S.lvl + 1].mask;
      Pd.filter = a.L[S.lvl + 1].filter;
      Pd.filter_words = a.L[S.lvl + 1].filter_words;
      Pd.filter_on = &P->d_atoms[S.atom].L[S.lvl + 1].filter_on;
      Pd.nk = a.L[S.lvl + 1].nk;
      Pd.wide = a.L[S.lvl + 1].wide;
      Pd.last = S.last;
      Pd.hsrc = S.lvl >= 1 ? In.h[S.atom] : nullptr;
    }
    (void)plan;
    (void)q;
  }
}

// Node 0 iterates its cover's base table: resolve every probe's key columns
// (all from the cover row) and the cover's predicates for the scan
// pipeline, and allocate its two survivor buffers.
static void setup_scan(fj_prepared* P) {
  P->scan0 = false;
  P->fuse_blocks = 0;
  if (P->opts.flags & FJ_FLAG_NO_FUSED_SCAN) return;
  NodeDev& N = P->nd[0];
  const SubDev& C = N.sub[0];
  if (N.dynamic || !C.last || C.lvl != 0) return;
  const AtomDev& ca = P->host_atoms[C.atom];
  ScanDev sc{};
  sc.n_probe = N.n_probe;
  bool track = false;
  for (int p = 0; p < N.n_probe; ++p) {
    const ProbeDev& Pd = N.probe[p];
    ScanProbe& S = sc.probe[p];
    S.nk = Pd.nv;
    for (int j = 0; j < Pd.nv && j < 3; ++j) {
      const VarSrc& v = N.src[Pd.var[j]];
      if (v.kind != kSrcRow) return;
      S.kcol[j] = v.col;
    }
    S.wide = Pd.wide;
    S.last = Pd.last;
    S.sub = Pd.sub;
    S.ht = Pd.ht;
    S.mask = Pd.mask;
    S.filter = Pd.filter;
    S.filter_words = Pd.filter_words;
    S.filter_on = Pd.filter_on;
    S.bitmap = nullptr;  // set below for the first probe of a one-launch scan
    S.exact = &P->d_atoms[N.sub[Pd.sub].atom].L[N.sub[Pd.sub].lvl + 1].exact;
    track |= Pd.last;
  }
  if (sc.n_probe > 0) {
    const ScanProbe& F = sc.probe[0];
    sc.k1 = F.nk == 1 && !F.wide;
    sc.vec_ok = sc.k1 && !(reinterpret_cast<uintptr_t>(F.kcol[0]) & 15);
  }
  sc.n_preds = ca.n_preds;
  for (int p = 0; p < ca.n_preds; ++p) {
    sc.pred_col[p] = ca.cols[ca.pred_col[p]];
    sc.pred_op[p] = ca.pred_op[p];
    sc.pred_val[p] = ca.pred_val[p];
  }
  // Survivor buffers, sized for one chunk of cover rows (a multiple of 4096
  // rows, so chunks keep 16-byte alignment).
  uint64_t rows = std::max<uint64_t>(ca.n_rows, 1);
  uint32_t cap = uint32_t(std::min<uint64_t>((rows + 4095) & ~4095ull, 1ull << 24));
  sc.cap = cap;
  sc.spin = uint32_t(std::min<uint64_t>(P->opts.spin_limit, 0xffffffffull));
  for (int b = 0; b < 1; ++b) {
    ScanBuf& B = sc.buf[b];
    B.row = P->alloc<uint32_t>(cap);
    for (int p = 0; p < sc.n_probe; ++p)
      if (!sc.probe[p].last) B.h[p] = P->alloc<uint32_t>(cap);
    B.mult = track ? P->alloc<uint64_t>(cap) : nullptr;
    B.n = P->alloc<uint32_t>(1);
    B.src = P->alloc<uint32_t>(cap);
  }
  P->sc0 = sc;
  P->scan0 = true;
  // One launch per chunk when the first probe reads one 16-byte aligned key
  // column, every later probe one key column at the root (a narrow level),
  // and the cover has no selection: one resident wave of blocks.
  P->fuse_blocks = 0;
  bool later_k1 = true;
  for (int p = 1; p < sc.n_probe; ++p) later_k1 &= sc.probe[p].nk == 1 && !sc.probe[p].wide;
  if (sc.k1 && sc.vec_ok && sc.n_preds == 0 && later_k1) {
    int b = 0;
    CK(cudaFuncSetAttribute(k_scan_fused<kFuseR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            int(kFuseSmem)));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_scan_fused<kFuseR>, kFuseThreads,
                                                     kFuseSmem));
    P->fuse_blocks = P->ctx->n_sm * std::max(1, b);
    // The first probe's root level (one key column) also gets an exact key
    // bitmap, built with the level; only this probe reads one.
    const SubDev& S0 = N.sub[N.probe[0].sub];
    AtomDev& A0 = P->host_atoms[S0.atom];
    LevelDev& L0 = A0.L[S0.lvl + 1];
    if (!P->sc0.probe[0].last && S0.lvl == 0 && L0.filter && L0.nk == 1 && !L0.wide) {
      if (!L0.bitmap) {
        L0.bitmap = P->alloc<uint32_t>(L0.filter_words);
        CK(cudaMemcpyAsync(&P->d_atoms[S0.atom], &A0, sizeof(AtomDev), cudaMemcpyHostToDevice,
                           P->ctx->stream));
      }
      P->sc0.probe[0].bitmap = L0.bitmap;
    }
  }
}

// Root-only forces as one cooperative launch: every block resident (two
// blocks of 512 threads per SM at most), where the device supports
// cooperative launches.
static void setup_roots(fj_prepared* P) {
  P->roots_grid = 0;
  int coop = 0;
  CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, P->ctx->device));
  if (!coop) return;
  CK(cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_force_roots),
                          cudaFuncAttributeMaxDynamicSharedMemorySize, int(kRootSmem)));
  int b = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_force_roots, kRootThreads, kRootSmem));
  if (b < 1) return;
  P->roots_state = P->alloc<RootsState>(1);
  P->roots_grid = P->ctx->n_sm * std::min(b, 2);
}

// Tails of the last expanded node that iterate a root level's vectors with
// one MIN variable: the root build keeps each entry's MIN of that column
// (LevelDev::tmin), so the aggregate epilogue reads it instead of walking
// the vector.  Only where that root level is always built by the
// cooperative root build (k_force_roots): its node forces roots only.
static void setup_tails(fj_prepared* P) {
  if (P->roots_grid <= 0 || P->materialize || P->last < 0) return;
  NodeDev& N = P->nd[P->last];
  if (N.mode != kModeAggregate) return;
  bool any = false;
  for (int t = 0; t < N.n_tail; ++t) {
    TailDev& T = N.tail[t];
    T.tmin = nullptr;
    if (T.lvl != 1 || T.n_min != 1) continue;
    const int k0 = P->ap[T.atom].level_node[0];
    if (!P->roots_only[k0]) continue;
    LevelDev& L = P->host_atoms[T.atom].L[1];
    if (!L.ht || L.tmin) continue;
    L.tmin = P->alloc<int32_t>(L.entries_cap);
    L.tmin_col = T.min_col[0];
    T.tmin = L.tmin;
    any = true;
  }
  if (any)
    CK(cudaMemcpyAsync(P->d_atoms, P->host_atoms.data(), sizeof(AtomDev) * P->host_atoms.size(),
                       cudaMemcpyHostToDevice, P->ctx->stream));
}

static void ensure_output(fj_prepared* P, uint64_t rows) {
  if (!P->materialize && !P->factorized) return;
  int nh = P->out_width;
  if (P->d_out && P->out_cap >= rows) return;
  if (P->d_out) dfree(P->ctx, P->d_out);
  P->out_cap = std::max<uint64_t>(rows, 1);
  P->d_out = dalloc<int32_t>(P->ctx, size_t(P->out_cap) * nh);
  P->nd[P->last].out_tuples = P->d_out;
  P->nd[P->last].out_rows_cap = P->out_cap;
}

// Reset the COLT state (every level unbuilt) and/or the result accumulators.
static void reset_state(fj_prepared* P, bool atoms) {
  fj_ctx* c = P->ctx;
  int na = int(P->q.atom_vars.size());
  k_reset<<<std::max(na, 1), 32, 0, c->stream>>>(
      P->d_atoms, na, P->d_res, atoms ? 1 : 0,
      reinterpret_cast<unsigned int*>(P->roots_state),
      P->roots_state ? int(sizeof(RootsState) / sizeof(unsigned int)) : 0);
  CK_LAUNCH("reset");
  P->kernels += 1;
}

// Force level l (L index, >= 1) of an atom for every entry of the level above.
static void build_level(fj_prepared* P, int atom, int l) {
  fj_ctx* c = P->ctx;
  k_request_all<<<blocks_for(P->host_atoms[atom].L[l - 1].entries_cap, kThreads, c->n_sm * 4),
                  kThreads, 0, c->stream>>>(P->d_atoms, atom, l);
  CK_LAUNCH("request_all");
  P->kernels += 1;
  force(P, P->d_level_jobs + size_t(atom) * kMaxLevels + l, 1, P->host_atoms[atom].n_rows,
        P->host_atoms[atom].L[l - 1].entries_cap, l == 1);
}

static void eager_builds(fj_prepared* P) {
  uint32_t fl = P->opts.flags;
  if (!(fl & (FJ_FLAG_EAGER_ALL | FJ_FLAG_EAGER_ROOT))) return;
  int na = int(P->q.atom_vars.size());
  int max_l = 1;
  if (fl & FJ_FLAG_EAGER_ALL)
    for (int a = 0; a < na; ++a) max_l = std::max(max_l, P->ap[a].n_levels);
  for (int l = 1; l <= max_l; ++l)
    for (int a = 0; a < na; ++a)
      if (l <= P->ap[a].n_levels && P->ap[a].may_force[l]) build_level(P, a, l);
}

static void run_once(fj_prepared* P) {
  if (P->timing()) P->t_first = P->mark();
  eager_builds(P);
  run_node(P, 0, 1);
  if (P->timing()) P->t_last = P->mark();
}

static uint64_t elapsed_ns(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, a, b));
  return uint64_t(double(ms) * 1e6);
}

static void interpret_result(fj_prepared* P, fj_result* out, bool* retry);

static void read_result(fj_prepared* P, fj_result* out, bool* retry) {
  fj_ctx* c = P->ctx;
  CK(cudaMemcpyAsync(P->h_res, P->d_res, sizeof(ResultDev), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  interpret_result(P, out, retry);
}

// The result of the last execution from its host copy (already fetched).
static void interpret_result(fj_prepared* P, fj_result* out, bool* retry) {
  const ResultDev& r = *P->h_res;
  *retry = false;
  if (r.status & kStTableFull) fail(FJ_ERR_CUDA, "internal: COLT hash level overfilled");
  if (r.status & kStItemsOverflow)
    fail(FJ_ERR_UNSUPPORTED, "more partial tuples than one chunk holds (in a batch, a node's "
                             "input must fit its buffer: run the query on its own)");
  if (r.status & kStCountOverflow) fail(FJ_ERR_COUNT_OVERFLOW, "COUNT(*) exceeds 2^64 - 1");
  if (r.status & kStDrainTimeout)
    fail(FJ_ERR_TIMEOUT, "a bounded device wait ran out, and so did the wait for the "
                         "copies in flight");
  if (r.status & kStTimeout) fail(FJ_ERR_TIMEOUT, "a bounded device wait ran out");
  std::memset(out, 0, sizeof(*out));
  out->n_head = int(P->q.head.size());
  if (P->materialize) {
    out->count = r.n_out;
    uint64_t lim = P->opts.list_limit;
    if (r.status & kStOutputOverflow) {
      if (lim == 0 || P->out_cap < lim) {
        *retry = true;  // grow the buffer to the exact size and run again
        return;
      }
    }
    out->n_out = std::min<uint64_t>(r.n_out, P->out_cap);
    out->d_tuples = P->d_out;
    out->tuples_owned = 0;
  } else if (P->factorized) {
    // COUNT(*) of the bag, and its factorized rows.
    if (r.status & kStOutputOverflow) {
      *retry = true;
      return;
    }
    out->count = r.count;
    out->n_head = P->out_width;
    out->n_out = std::min<uint64_t>(r.n_out, P->out_cap);
    out->d_tuples = P->d_out;
    out->tuples_owned = 0;
  } else {
    out->count = r.count;
    for (int i = 0; i < int(P->min_vars.size()); ++i) {
      out->mins[i] = r.mins[i];
      out->min_valid[i] = r.count > 0;
    }
  }
  for (int i = 0; i < 16; ++i) out->counters[i] = r.ctr[i];
  out->counters[FJ_CTR_COVER_POLICY] = uint64_t(P->opts.cover_policy);
  out->counters[FJ_CTR_CHUNKS] = P->chunks;
  out->counters[FJ_CTR_KERNELS] = P->kernels;
  if (P->timing() && P->t_first) {
    uint64_t ex = 0, bu = 0;
    for (auto& pr : P->t_expand) ex += elapsed_ns(pr.first, pr.second);
    for (auto& pr : P->t_build) bu += elapsed_ns(pr.first, pr.second);
    out->counters[FJ_CTR_EXPAND_NS] = ex;
    out->counters[FJ_CTR_EXPAND_LAUNCHES] = P->t_expand.size();
    out->counters[FJ_CTR_BUILD_NS] = bu;
    out->counters[FJ_CTR_SPAN_NS] = elapsed_ns(P->t_first, P->t_last);
  }
}

static void begin_execution(fj_prepared* P) {
  P->kernels = 0;
  P->chunks = 0;
  P->n_events = 0;
  P->t_expand.clear();
  P->t_build.clear();
  P->t_first = P->t_last = nullptr;
}

// Runs the prepared plan and fills *out; returns true when a materialized
// output has more rows than list_limit (*out then holds the exact count and
// the first list_limit rows; the caller reports FJ_ERR_OUTPUT_OVERFLOW).
static bool execute(fj_prepared* P, fj_result* out) {
  for (int attempt = 0; attempt < 3; ++attempt) {
    begin_execution(P);
    if (P->materialize) {
      uint64_t want = P->opts.list_limit ? P->opts.list_limit : (P->out_cap ? P->out_cap : 1u << 20);
      ensure_output(P, want);
    } else if (P->factorized) {
      ensure_output(P, P->out_cap ? P->out_cap : 1u << 20);
    }
    reset_state(P, false);
    run_once(P);
    bool retry = false;
    read_result(P, out, &retry);
    if (!retry) return P->materialize && P->opts.list_limit && out->count > P->opts.list_limit;
    uint64_t need = P->h_res->n_out;
    if (P->opts.list_limit && P->materialize) need = std::min<uint64_t>(need, P->opts.list_limit);
    ensure_output(P, need);
  }
  fail(FJ_ERR_CUDA, "internal: output sizing did not converge");
}

static void execute_async(fj_prepared* P) {
  begin_execution(P);
  if (P->materialize)
    ensure_output(P, P->opts.list_limit ? P->opts.list_limit : (P->out_cap ? P->out_cap : 1u << 20));
  else if (P->factorized)
    ensure_output(P, P->out_cap ? P->out_cap : 1u << 20);
  reset_state(P, false);
  run_once(P);
}

static void prepared_result(fj_prepared* P, fj_result* out) {
  bool retry = false;
  read_result(P, out, &retry);
  if (retry || (P->materialize && P->opts.list_limit && out->count > P->opts.list_limit))
    fail(FJ_ERR_OUTPUT_OVERFLOW, "more output rows than the prepared output buffer");
}

static void prepared_release(fj_prepared* P) {
  if (!P) return;
  P->ctx->preps.erase(P);
  for (cudaEvent_t e : P->events) cudaEventDestroy(e);
  for (void* p : P->allocs) dfree(P->ctx, p);
  if (P->d_out) dfree(P->ctx, P->d_out);
  cudaStreamSynchronize(P->ctx->stream);
  if (P->h_res) cudaFreeHost(P->h_res);
  delete P;
}

static fj_prepared* prepare(fj_ctx* ctx, const fj_query* query, const fj_plan* plan,
                            const fj_exec_opts* opts) {
  if (!ctx) fail(FJ_ERR_INVALID_ARG, "NULL context");
  std::unique_ptr<fj_prepared> P(new fj_prepared());
  P->ctx = ctx;
  if (!load_query(query, P->q)) fail(FJ_ERR_INVALID_ARG, get_error());
  if (!load_plan(P->q, plan, P->plan)) fail(FJ_ERR_INVALID_PLAN, get_error());
  if (!validate(P->q, P->plan)) fail(FJ_ERR_INVALID_PLAN, get_error());
  if (opts) P->opts = *opts;
  if (P->opts.out_mode < FJ_OUT_MATERIALIZE || P->opts.out_mode > FJ_OUT_FACTORIZED)
    fail(FJ_ERR_INVALID_ARG, "bad out_mode");
  if (P->opts.cover_policy < FJ_COVER_STATIC || P->opts.cover_policy > FJ_COVER_LEARNED)
    fail(FJ_ERR_INVALID_ARG, "bad cover_policy");
  if (P->opts.cover_policy == FJ_COVER_LEARNED) {
    // Decided once, here: the policy the network predicts cheaper.
    if (!P->opts.model) fail(FJ_ERR_INVALID_ARG, "FJ_COVER_LEARNED needs opts.model");
    int pol = FJ_COVER_STATIC;
    fj_status st = fj_internal_learned_policy(ctx, query, P->plan,
                                              static_cast<const fj_model*>(P->opts.model), &pol);
    if (st != FJ_OK) fail(st, fj_internal_chooser_error());
    P->opts.cover_policy = pol;
  }
  P->opts.model = nullptr;
  if (P->opts.out_mode == FJ_OUT_COUNT_MIN) {
    if (P->opts.n_min_vars < 0 || P->opts.n_min_vars > FJ_MAX_VARS ||
        (P->opts.n_min_vars && !P->opts.min_vars))
      fail(FJ_ERR_INVALID_ARG, "bad min_vars");
    for (int i = 0; i < P->opts.n_min_vars; ++i) {
      int v = P->opts.min_vars[i];
      if (std::find(P->q.head.begin(), P->q.head.end(), v) == P->q.head.end())
        fail(FJ_ERR_INVALID_ARG, "min variable not in the query");
      P->min_vars.push_back(v);
    }
  }
  P->opts.min_vars = nullptr;
  for (int a = 0; a < query->n_atoms; ++a) {
    fj_rel* r = query->atoms[a].rel;
    if (!r || r->ctx != ctx) fail(FJ_ERR_INVALID_ARG, "atom without a relation of this context");
    if (r->n_rows >= 0xffffffffull) fail(FJ_ERR_INVALID_ARG, "relation too large");
    P->rels.push_back(r);
  }
  CK(cudaSetDevice(ctx->device));
  try {
    P->d_res = P->alloc<ResultDev>(1);
    P->d_partials = P->alloc<uint64_t>(size_t(kMaxScanJobs) * kScanBlocks);
    CK(cudaMallocHost(&P->h_res, sizeof(ResultDev)));
    compile(P.get());
    upload_atoms(P.get(), query);
    finalize_nodes(P.get());
    setup_scan(P.get());
    setup_roots(P.get());
    setup_tails(P.get());
    reset_state(P.get(), true);
  } catch (...) {
    for (void* p : P->allocs) dfree(ctx, p);
    if (P->h_res) cudaFreeHost(P->h_res);
    throw;
  }
  ctx->preps.insert(P.get());
  return P.release();
}

// ---------------------------------------------------------------------------
// Batches: many prepared queries as one unit of work (no counterpart in the
// paper).  Every query runs from scratch, back to back on the context's
// stream, and the host synchronizes once for all results; with
// FJ_BATCH_GRAPH the whole sequence is captured once into a CUDA graph and
// each execution is one graph launch.
// ---------------------------------------------------------------------------

struct fj_batch {
  fj_ctx* ctx = nullptr;
  std::vector<fj_prepared*> preps;
  int flags = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<uint64_t> kernels, chunks;  // per query, as enqueued
};

// A query can be batched when nothing in its execution waits for the host:
// aggregate output, no timing or eager builds, and node 0 as its only
// expanded node with a total known on the host (its cover is a base table).
static bool batchable(const fj_prepared* P, std::string* why) {
  if (P->materialize || P->factorized) {
    *why = "materialized or factorized output (the output size is decided on the host)";
    return false;
  }
  if (P->opts.flags & (FJ_FLAG_EAGER_ALL | FJ_FLAG_EAGER_ROOT)) {
    *why = "eager-build flags";
    return false;
  }
  return true;
}

static void batch_enqueue(fj_batch* B, const std::vector<cudaStream_t>* branches = nullptr) {
  for (size_t i = 0; i < B->preps.size(); ++i) {
    fj_prepared* P = B->preps[i];
    if (branches) B->ctx->stream = (*branches)[i % branches->size()];
    begin_execution(P);
    reset_state(P, true);
    P->device_totals = true;
    try {
      run_once(P);
    } catch (...) {
      P->device_totals = false;
      throw;
    }
    P->device_totals = false;
    CK(cudaMemcpyAsync(P->h_res, P->d_res, sizeof(ResultDev), cudaMemcpyDeviceToHost,
                       B->ctx->stream));
    B->kernels[i] = P->kernels;
    B->chunks[i] = P->chunks;
  }
}

static fj_batch* batch_create(fj_ctx* ctx, int n, fj_prepared* const* preps, int flags) {
  if (!ctx || n < 0 || (n > 0 && !preps)) fail(FJ_ERR_INVALID_ARG, "bad batch arguments");
  std::unique_ptr<fj_batch> B(new fj_batch);
  B->ctx = ctx;
  B->flags = flags;
  for (int i = 0; i < n; ++i) {
    fj_prepared* P = preps[i];
    if (!P || P->ctx != ctx) fail(FJ_ERR_INVALID_ARG, "query of another context in the batch");
    std::string why;
    if (!batchable(P, &why))
      fail(FJ_ERR_UNSUPPORTED, "batch query " + std::to_string(i) + ": " + why);
    B->preps.push_back(P);
  }
  B->kernels.assign(n, 0);
  B->chunks.assign(n, 0);
  if ((flags & FJ_BATCH_CONCURRENT) && !(flags & FJ_BATCH_GRAPH))
    fail(FJ_ERR_INVALID_ARG, "FJ_BATCH_CONCURRENT needs FJ_BATCH_GRAPH");
  if (flags & FJ_BATCH_GRAPH) {
    // Capture on a private stream (the context's stream may be the legacy
    // default stream, which cannot be captured); the graph is launched on
    // the context's stream.  FJ_BATCH_CONCURRENT: the queries are spread
    // over kBranches streams forked from it and joined at the end, so the
    // graph holds independent branches the GPU runs side by side; their
    // root levels are then built by the multi-launch force (cooperative
    // launches must not share the GPU), without the per-entry tail MINs.
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    const bool conc = flags & FJ_BATCH_CONCURRENT;
    constexpr int kBranches = 8;
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> br;
    std::vector<cudaEvent_t> evs;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t saved = ctx->stream;
    struct Saved {
      int roots_grid;
      std::vector<const int32_t*> tmin;
    };
    std::vector<Saved> keep;
    auto restore = [&] {
      ctx->stream = saved;
      for (size_t i = 0; i < keep.size(); ++i) {
        fj_prepared* P = B->preps[i];
        P->roots_grid = keep[i].roots_grid;
        for (size_t t = 0; t < keep[i].tmin.size(); ++t) P->nd[P->last].tail[t].tmin = keep[i].tmin[t];
      }
      for (cudaStream_t b : br) cudaStreamDestroy(b);
      for (cudaEvent_t e : evs) cudaEventDestroy(e);
      cudaStreamDestroy(cap);
    };
    if (conc) {
      for (fj_prepared* P : B->preps) {
        Saved sv{P->roots_grid, {}};
        if (P->last >= 0)
          for (int t = 0; t < P->nd[P->last].n_tail; ++t) {
            sv.tmin.push_back(P->nd[P->last].tail[t].tmin);
            P->nd[P->last].tail[t].tmin = nullptr;
          }
        P->roots_grid = 0;
        keep.push_back(sv);
      }
      for (int i = 0; i < kBranches; ++i) {
        cudaStream_t b = nullptr;
        cudaEvent_t e = nullptr;
        CK(cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking));
        br.push_back(b);
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        evs.push_back(e);
      }
      cudaEvent_t e = nullptr;
      CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      evs.push_back(e);
    }
    ctx->stream = cap;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      try {
        if (conc) {
          cudaEvent_t fork = evs[kBranches];
          CK(cudaEventRecord(fork, cap));
          for (cudaStream_t b : br) CK(cudaStreamWaitEvent(b, fork, 0));
          batch_enqueue(B.get(), &br);
          for (int i = 0; i < kBranches; ++i) {
            CK(cudaEventRecord(evs[i], br[i]));
            CK(cudaStreamWaitEvent(cap, evs[i], 0));
          }
        } else {
          batch_enqueue(B.get());
        }
      } catch (...) {
        cudaGraph_t g = nullptr;
        ctx->stream = cap;
        cudaStreamEndCapture(cap, &g);
        if (g) cudaGraphDestroy(g);
        restore();
        throw;
      }
      e = cudaStreamEndCapture(cap, &B->graph);
    }
    restore();
    CK(e);
    CK(cudaGraphInstantiate(&B->exec, B->graph, 0));
  }
  return B.release();
}

static void batch_launch(fj_batch* B) {
  fj_ctx* c = B->ctx;
  CK(cudaSetDevice(c->device));
  if (B->exec) {
    CK(cudaGraphLaunch(B->exec, c->stream));
  } else {
    batch_enqueue(B);
  }
}

static void batch_results(fj_batch* B, fj_result* results) {
  fj_ctx* c = B->ctx;
  CK(cudaSetDevice(c->device));
  CK(cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i < B->preps.size(); ++i) {
    fj_prepared* P = B->preps[i];
    P->kernels = B->kernels[i];
    P->chunks = B->chunks[i];
    bool retry = false;
    interpret_result(P, &results[i], &retry);
  }
}

static void batch_free(fj_batch* B) {
  if (!B) return;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  delete B;
}

// ---------------------------------------------------------------------------
// Expansion of a factorized result into flat head-order tuples.
// ---------------------------------------------------------------------------

namespace {

struct FactorExpandDev {
  int width, n_pre, n_tail, n_head;
  // Per head position: the prefix column (src >= 0), or the tail (-1 - t)
  // and its atom column.
  int src[FJ_MAX_VARS];
  int tcol[FJ_MAX_VARS];
  const uint32_t* perm[FJ_MAX_NODES];
  const int32_t* cols[FJ_MAX_NODES][FJ_MAX_ARITY];
};

// Bag size of every factorized row: multiplicity times the tail lengths.
__global__ void k_factor_fan(const int32_t* __restrict__ rows, uint64_t n, FactorExpandDev fx,
                             unsigned long long* fan) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
       i += uint64_t(gridDim.x) * blockDim.x) {
    const int32_t* r = rows + i * fx.width;
    unsigned long long m = uint64_t(uint32_t(r[fx.n_pre])) | uint64_t(uint32_t(r[fx.n_pre + 1])) << 32;
    for (int t = 0; t < fx.n_tail; ++t) m *= uint32_t(r[fx.n_pre + 3 + 2 * t]);
    fan[i] = m;
  }
}

// One thread per factorized row writes its tuples at offset off[i]: the
// multiplicity copies outermost, then the tails' vectors in mixed radix.
__global__ void k_factor_expand(const int32_t* __restrict__ rows, uint64_t n, FactorExpandDev fx,
                                const unsigned long long* __restrict__ off,
                                const unsigned long long* __restrict__ fan, int32_t* out) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
       i += uint64_t(gridDim.x) * blockDim.x) {
    const int32_t* r = rows + i * fx.width;
    for (unsigned long long j = 0; j < fan[i]; ++j) {
      int32_t* o = out + (off[i] + j) * fx.n_head;
      uint32_t trow[FJ_MAX_NODES];
      unsigned long long q = j;
      for (int t = fx.n_tail - 1; t >= 0; --t) {
        const uint32_t cn = uint32_t(r[fx.n_pre + 3 + 2 * t]);
        trow[t] = fx.perm[t][uint32_t(r[fx.n_pre + 2 + 2 * t]) + uint32_t(q % cn)];
        q /= cn;
      }
      for (int h = 0; h < fx.n_head; ++h) {
        const int s = fx.src[h];
        o[h] = s >= 0 ? r[s] : fx.cols[-1 - s][fx.tcol[h]][trow[-1 - s]];
      }
    }
  }
}

}  // namespace

static void factor_layout(const fj_prepared* P, FactorExpandDev& fx) {
  if (!P->factorized) fail(FJ_ERR_INVALID_ARG, "the plan was not prepared with FJ_OUT_FACTORIZED");
  const NodeDev& N = P->nd[P->last];
  fx.width = P->out_width;
  fx.n_pre = N.n_pre;
  fx.n_tail = N.n_tail;
  fx.n_head = int(P->q.head.size());
  for (int h = 0; h < fx.n_head; ++h) {
    const int v = P->q.head[h];
    fx.src[h] = 0;
    fx.tcol[h] = 0;
    bool found = false;
    for (int k = 0; k < N.n_pre && !found; ++k)
      if (N.pre_var[k] == v) {
        fx.src[h] = k;
        found = true;
      }
    for (int t = 0; t < N.n_tail && !found; ++t) {
      const int node = P->tail_start + t;
      const PSub& sa = P->plan[node][0];
      if (std::find(sa.vars.begin(), sa.vars.end(), v) == sa.vars.end()) continue;
      const auto& av = P->q.atom_vars[sa.atom];
      fx.src[h] = -1 - t;
      fx.tcol[h] = int(std::find(av.begin(), av.end(), v) - av.begin());
      found = true;
    }
    if (!found) fail(FJ_ERR_INVALID_ARG, "internal: a head variable is in no factor");
  }
  for (int t = 0; t < N.n_tail; ++t) {
    const AtomDev& a = P->host_atoms[N.tail[t].atom];
    fx.perm[t] = a.perm;
    for (int j = 0; j < FJ_MAX_ARITY; ++j) fx.cols[t][j] = a.cols[j];
  }
}

// ---------------------------------------------------------------------------
// Bushy plans (paper Section 2.2 and Section 5.2): a binary join tree whose
// right children may be subtrees.  Its left spine is a left-deep plan; every
// right child that is not an atom is evaluated first (recursively) and its
// bag of tuples materialized as a relation with one column per variable of
// the subtree, which the spine then joins like a base table.  The spine is
// converted by binary2fj and factored (Section 4.1).
// ---------------------------------------------------------------------------

namespace {

// Row-major n x k tuples into k columns.
__global__ void k_transpose_cols(const int32_t* __restrict__ rows, uint64_t n, int k,
                                 int32_t* const* cols) {
  const uint64_t total = n * uint64_t(k);
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < total;
       i += uint64_t(gridDim.x) * blockDim.x)
    cols[i % k][i / k] = rows[i];
}

struct BushyCtx {
  fj_ctx* ctx;
  const fj_query* query;
  const fj_bushy_node* nodes;
  int n_nodes;
  const fj_exec_opts* opts;
  std::vector<fj_rel*> temps;  // materialized subtrees (released at the end)
  std::vector<void*> dbufs;    // device buffers of the same lifetime
  uint64_t kernels = 0;
};

uint64_t bushy_vars(const BushyCtx& B, int n, int depth = 0) {
  if (n < 0 || n >= B.n_nodes || depth > B.n_nodes) fail(FJ_ERR_INVALID_ARG, "bushy: bad node index");
  const fj_bushy_node& nd = B.nodes[n];
  if (nd.atom >= 0) {
    if (nd.atom >= B.query->n_atoms) fail(FJ_ERR_INVALID_ARG, "bushy: bad atom index");
    uint64_t m = 0;
    for (int j = 0; j < B.query->atoms[nd.atom].n_vars; ++j) m |= 1ull << B.query->atoms[nd.atom].vars[j];
    return m;
  }
  return bushy_vars(B, nd.left, depth + 1) | bushy_vars(B, nd.right, depth + 1);
}

// The left spine of subtree n as a list of leaves: atoms of the query, or
// materialized subtrees (their relation and variables).
struct Leaf {
  fj_atom atom;
  std::vector<int> vars, cols;
  std::vector<fj_pred> preds;
};

fj_rel* bushy_materialize(BushyCtx& B, int n);

void bushy_spine(BushyCtx& B, int n, std::vector<Leaf>& out, int depth = 0) {
  if (depth > B.n_nodes) fail(FJ_ERR_INVALID_ARG, "bushy: the tree has a cycle");
  const fj_bushy_node& nd = B.nodes[n];
  if (nd.atom >= 0) {
    const fj_atom& a = B.query->atoms[nd.atom];
    Leaf L;
    L.vars.assign(a.vars, a.vars + a.n_vars);
    if (a.cols) L.cols.assign(a.cols, a.cols + a.n_vars);
    if (a.n_preds) L.preds.assign(a.preds, a.preds + a.n_preds);
    L.atom = a;
    out.push_back(std::move(L));
    return;
  }
  bushy_spine(B, nd.left, out, depth + 1);
  const fj_bushy_node& r = B.nodes[nd.right];
  if (r.atom >= 0) {
    bushy_spine(B, nd.right, out, depth + 1);
  } else {
    // A bushy right child: evaluate it first and join its bag as a relation
    // over its variables (in increasing id order, one column each).
    fj_rel* rel = bushy_materialize(B, nd.right);
    const uint64_t m = bushy_vars(B, nd.right);
    Leaf L;
    for (int v = 0; v < FJ_MAX_VARS; ++v)
      if (m >> v & 1) L.vars.push_back(v);
    L.atom = fj_atom{rel, int(L.vars.size()), nullptr, nullptr, 0, nullptr};
    out.push_back(std::move(L));
  }
}

// Run the left spine of subtree n with `mode` over `head` (variable ids).
void bushy_run(BushyCtx& B, int n, int mode, const std::vector<int>& head,
               const fj_exec_opts* base, fj_result* res) {
  std::vector<Leaf> leaves;
  bushy_spine(B, n, leaves);
  std::vector<fj_atom> atoms(leaves.size());
  for (size_t i = 0; i < leaves.size(); ++i) {
    atoms[i] = leaves[i].atom;
    atoms[i].vars = leaves[i].vars.data();
    atoms[i].n_vars = int(leaves[i].vars.size());
    atoms[i].cols = leaves[i].cols.empty() ? nullptr : leaves[i].cols.data();
    atoms[i].preds = leaves[i].preds.empty() ? nullptr : leaves[i].preds.data();
    atoms[i].n_preds = int(leaves[i].preds.size());
  }
  fj_query q{int(atoms.size()), atoms.data(), int(head.size()), head.data()};
  PQuery pq;
  if (!load_query(&q, pq)) fail(FJ_ERR_INVALID_ARG, std::string("bushy: ") + get_error());
  std::vector<int> order(atoms.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = int(i);
  PPlan plan = factor(binary2fj(pq, order));
  std::unique_ptr<fj_plan, void (*)(fj_plan*)> ep(export_plan(plan), fj_plan_free);
  fj_exec_opts o = base ? *base : fj_exec_opts{};
  o.out_mode = mode;
  if (mode != FJ_OUT_COUNT_MIN) {
    o.n_min_vars = 0;
    o.min_vars = nullptr;
  }
  if (n != B.n_nodes - 1) o.list_limit = 0;  // intermediates are never cut short
  fj_status st = fj_execute_plan(B.ctx, &q, ep.get(), &o, res);
  if (st != FJ_OK) fail(st, std::string("bushy subplan: ") + get_error());
  B.kernels += res->counters[FJ_CTR_KERNELS];
}

fj_rel* bushy_materialize(BushyCtx& B, int n) {
  const uint64_t m = bushy_vars(B, n);
  std::vector<int> head;
  for (int v = 0; v < FJ_MAX_VARS; ++v)
    if (m >> v & 1) head.push_back(v);
  fj_result r{};
  bushy_run(B, n, FJ_OUT_MATERIALIZE, head, B.opts, &r);
  fj_ctx* c = B.ctx;
  const int k = int(head.size());
  if (r.n_out >= 0xffffffffull) fail(FJ_ERR_UNSUPPORTED, "bushy: intermediate above 2^32 - 1 rows");
  std::unique_ptr<fj_rel> rel(new fj_rel());
  rel->ctx = c;
  rel->name = "bushy intermediate";
  rel->n_rows = r.n_out;
  std::vector<int32_t*> cols(k);
  for (int j = 0; j < k; ++j) {
    cols[j] = dalloc<int32_t>(c, std::max<uint64_t>(r.n_out, 1));
    rel->owned.push_back(cols[j]);
    rel->cols.push_back(cols[j]);
  }
  if (r.n_out) {
    int32_t** d_cols = dalloc<int32_t*>(c, k);
    B.dbufs.push_back(d_cols);
    CK(cudaMemcpyAsync(d_cols, cols.data(), sizeof(int32_t*) * k, cudaMemcpyHostToDevice,
                       c->stream));
    k_transpose_cols<<<blocks_for(r.n_out * k, 256, c->n_sm * 8), 256, 0, c->stream>>>(
        r.d_tuples, r.n_out, k, d_cols);
    CK_LAUNCH("bushy transpose");
    B.kernels += 1;
  }
  fj_result_free(c, &r);
  c->rels.insert(rel.get());
  B.temps.push_back(rel.get());
  return rel.release();
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI.
// ---------------------------------------------------------------------------

extern "C" {

fj_status fj_ctx_create(int device, void* cuda_stream, fj_ctx** out) {
  return guarded([&] {
    if (!out) fail(FJ_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    CK(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) fail(FJ_ERR_INVALID_ARG, "no such CUDA device");
    CK(cudaSetDevice(device));
    auto* c = new fj_ctx();
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    CK(cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device));
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    CK(cudaMemPoolCreate(&c->pool, &props));
    uint64_t keep = ~0ull;
    CK(cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep));
    CK(cudaMallocHost(&c->h_total, sizeof(uint64_t)));
    c->d_partials = dalloc<uint64_t>(c, size_t(kMaxScanJobs) * kScanBlocks);
    CK(cudaStreamSynchronize(c->stream));
    *out = c;
  });
}

void fj_ctx_destroy(fj_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  while (!c->preps.empty()) prepared_release(*c->preps.begin());
  while (!c->rels.empty()) fj_release_relation(c, *c->rels.begin());
  dfree(c, c->d_partials);
  cudaStreamSynchronize(c->stream);
  if (c->h_total) cudaFreeHost(c->h_total);
  if (c->pool) cudaMemPoolDestroy(c->pool);
  delete c;
}

fj_status fj_ctx_set_stream(fj_ctx* c, void* cuda_stream) {
  return guarded([&] {
    if (!c) fail(FJ_ERR_INVALID_ARG, "NULL context");
    c->stream = static_cast<cudaStream_t>(cuda_stream);
  });
}

fj_status fj_load_relation(fj_ctx* c, const char* name, int n_cols, const int32_t* const* d_cols,
                           uint64_t n_rows, fj_rel** out) {
  return guarded([&] {
    if (!c || !out || !d_cols || n_cols < 1 || n_cols > FJ_MAX_ARITY * 4)
      fail(FJ_ERR_INVALID_ARG, "fj_load_relation: bad argument");
    if (n_rows >= 0xffffffffull) fail(FJ_ERR_INVALID_ARG, "fj_load_relation: too many rows");
    auto* r = new fj_rel();
    r->ctx = c;
    r->name = name ? name : "";
    r->n_rows = n_rows;
    for (int j = 0; j < n_cols; ++j) {
      if (!d_cols[j] && n_rows) {
        delete r;
        fail(FJ_ERR_INVALID_ARG, "fj_load_relation: NULL column");
      }
      r->cols.push_back(d_cols[j]);
    }
    c->rels.insert(r);
    *out = r;
  });
}

fj_status fj_load_relation_host(fj_ctx* c, const char* name, int n_cols,
                                const int32_t* const* h_cols, uint64_t n_rows, fj_rel** out) {
  return guarded([&] {
    if (!c || !out || !h_cols || n_cols < 1 || n_cols > FJ_MAX_ARITY * 4)
      fail(FJ_ERR_INVALID_ARG, "fj_load_relation_host: bad argument");
    if (n_rows >= 0xffffffffull) fail(FJ_ERR_INVALID_ARG, "fj_load_relation_host: too many rows");
    std::unique_ptr<fj_rel> r(new fj_rel());
    r->ctx = c;
    r->name = name ? name : "";
    r->n_rows = n_rows;
    try {
      for (int j = 0; j < n_cols; ++j) {
        if (!h_cols[j] && n_rows) fail(FJ_ERR_INVALID_ARG, "fj_load_relation_host: NULL column");
        int32_t* d = dalloc<int32_t>(c, n_rows);
        r->owned.push_back(d);
        r->cols.push_back(d);
        if (n_rows)
          CK(cudaMemcpyAsync(d, h_cols[j], n_rows * sizeof(int32_t), cudaMemcpyHostToDevice,
                             c->stream));
      }
    } catch (...) {
      for (void* p : r->owned) dfree(c, p);
      throw;
    }
    c->rels.insert(r.get());
    *out = r.release();
  });
}

void fj_release_relation(fj_ctx* c, fj_rel* r) {
  if (!r) return;
  fj_ctx* owner = r->ctx;
  for (void* p : r->owned) dfree(owner, p);
  owner->rels.erase(r);
  delete r;
}

uint64_t fj_relation_rows(const fj_rel* r) { return r ? r->n_rows : 0; }

fj_status fj_prepare(fj_ctx* ctx, const fj_query* query, const fj_plan* plan,
                     const fj_exec_opts* opts, fj_prepared** out) {
  return guarded([&] {
    if (!out) fail(FJ_ERR_INVALID_ARG, "out is NULL");
    *out = prepare(ctx, query, plan, opts);
  });
}

fj_status fj_build_colt_level(fj_prepared* P, int atom, int level) {
  return guarded([&] {
    if (!P || atom < 0 || atom >= int(P->q.atom_vars.size()) || level < 0 ||
        level >= P->ap[atom].n_levels)
      fail(FJ_ERR_INVALID_ARG, "fj_build_colt_level: bad atom or level");
    int l = level + 1;
    if (!P->ap[atom].may_force[l])
      fail(FJ_ERR_UNSUPPORTED,
           "fj_build_colt_level: this level is only iterated under the plan and opts; prepare "
           "with FJ_FLAG_EAGER_ALL to build every level");
    build_level(P, atom, l);
    P->explicit_built = true;
  });
}

fj_status fj_execute_prepared_async(fj_prepared* P) {
  return guarded([&] {
    if (!P) fail(FJ_ERR_INVALID_ARG, "NULL prepared plan");
    execute_async(P);
  });
}

fj_status fj_prepared_result(fj_prepared* P, fj_result* out) {
  return guarded([&] {
    if (!P || !out) fail(FJ_ERR_INVALID_ARG, "NULL argument");
    prepared_result(P, out);
  });
}

fj_status fj_execute_prepared(fj_prepared* P, fj_result* out) {
  return guarded([&] {
    if (!P || !out) fail(FJ_ERR_INVALID_ARG, "NULL argument");
    if (execute(P, out)) fail(FJ_ERR_OUTPUT_OVERFLOW, "more output rows than list_limit");
  });
}

fj_status fj_reset_prepared(fj_prepared* P) {
  return guarded([&] {
    if (!P) fail(FJ_ERR_INVALID_ARG, "NULL prepared plan");
    reset_state(P, true);
    P->explicit_built = false;
  });
}

void fj_prepared_free(fj_prepared* P) { prepared_release(P); }

fj_status fj_execute_plan(fj_ctx* ctx, const fj_query* query, const fj_plan* plan,
                          const fj_exec_opts* opts, fj_result* out) {
  fj_prepared* P = nullptr;
  fj_status st = guarded([&] {
    if (!out) fail(FJ_ERR_INVALID_ARG, "out is NULL");
    if (opts && opts->out_mode == FJ_OUT_FACTORIZED)
      fail(FJ_ERR_UNSUPPORTED, "factorized output needs a prepared plan (fj_prepare): its "
                               "vectors live in the plan's COLT storage");
    P = prepare(ctx, query, plan, opts);
    const bool over = execute(P, out);
    if (out->d_tuples) {
      // Hand the output buffer to the result.
      P->d_out = nullptr;
      out->tuples_owned = 1;
    }
    if (over) fail(FJ_ERR_OUTPUT_OVERFLOW, "more output rows than list_limit");
  });
  if (P) prepared_release(P);
  if (st != FJ_OK) set_error(get_error());
  return st;
}

fj_status fj_prepared_factor_layout(const fj_prepared* P, int* width, int* n_prefix,
                                    int* prefix_vars, int* n_tails, int* tail_atoms) {
  return guarded([&] {
    if (!P || !width || !n_prefix || !prefix_vars || !n_tails || !tail_atoms)
      fail(FJ_ERR_INVALID_ARG, "NULL argument");
    FactorExpandDev fx{};
    factor_layout(P, fx);
    const NodeDev& N = P->nd[P->last];
    *width = fx.width;
    *n_prefix = N.n_pre;
    for (int k = 0; k < N.n_pre; ++k) prefix_vars[k] = N.pre_var[k];
    *n_tails = N.n_tail;
    for (int t = 0; t < N.n_tail; ++t) tail_atoms[t] = N.tail[t].atom;
  });
}

fj_status fj_prepared_expand(fj_prepared* P, const fj_result* res, int32_t* d_dst,
                             uint64_t dst_rows) {
  return guarded([&] {
    if (!P || !res || (!d_dst && res->count)) fail(FJ_ERR_INVALID_ARG, "NULL argument");
    FactorExpandDev fx{};
    factor_layout(P, fx);
    if (res->d_tuples != P->d_out) fail(FJ_ERR_INVALID_ARG, "not this plan's last result");
    if (dst_rows < res->count) fail(FJ_ERR_INVALID_ARG, "the destination holds fewer rows than COUNT");
    const uint64_t n = res->n_out;
    if (n == 0) return;
    fj_ctx* c = P->ctx;
    cudaStream_t s = c->stream;
    unsigned long long* fan = dalloc<unsigned long long>(c, n);
    unsigned long long* off = dalloc<unsigned long long>(c, n);
    std::vector<unsigned long long> h(n);
    k_factor_fan<<<blocks_for(n, 256, c->n_sm * 8), 256, 0, s>>>(res->d_tuples, n, fx, fan);
    CK_LAUNCH("factor fan");
    CK(cudaMemcpyAsync(h.data(), fan, n * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    unsigned long long acc = 0;
    for (uint64_t i = 0; i < n; ++i) {
      const unsigned long long f = h[i];
      h[i] = acc;
      acc += f;
    }
    if (acc != res->count) fail(FJ_ERR_CUDA, "internal: factorized rows disagree with COUNT");
    CK(cudaMemcpyAsync(off, h.data(), n * 8, cudaMemcpyHostToDevice, s));
    k_factor_expand<<<blocks_for(n, 128, c->n_sm * 8), 128, 0, s>>>(res->d_tuples, n, fx, off, fan,
                                                                    d_dst);
    CK_LAUNCH("factor expand");
    CK(cudaStreamSynchronize(s));
    dfree(c, fan);
    dfree(c, off);
  });
}

fj_status fj_result_copy_tuples(fj_ctx* c, const fj_result* res, void* dst, int dst_is_device) {
  return guarded([&] {
    if (!c || !res || !dst || !res->d_tuples) fail(FJ_ERR_INVALID_ARG, "no tuples to copy");
    size_t bytes = size_t(res->n_out) * res->n_head * sizeof(int32_t);
    if (bytes)
      CK(cudaMemcpyAsync(dst, res->d_tuples, bytes,
                         dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                         c->stream));
    CK(cudaStreamSynchronize(c->stream));
  });
}

fj_status fj_execute_bushy(fj_ctx* ctx, const fj_query* query, const fj_bushy_node* nodes,
                           int n_nodes, const fj_exec_opts* opts, fj_result* out) {
  BushyCtx B{ctx, query, nodes, n_nodes, opts, {}, {}, 0};
  fj_status st = guarded([&] {
    if (!ctx || !query || !nodes || n_nodes < 1 || !out)
      fail(FJ_ERR_INVALID_ARG, "fj_execute_bushy: bad argument");
    PQuery pq;
    if (!load_query(query, pq)) fail(FJ_ERR_INVALID_ARG, get_error());
    // Every atom exactly once among the leaves.
    std::vector<int> seen(query->n_atoms, 0);
    for (int i = 0; i < n_nodes; ++i)
      if (nodes[i].atom >= 0) {
        if (nodes[i].atom >= query->n_atoms) fail(FJ_ERR_INVALID_ARG, "bushy: bad atom index");
        seen[nodes[i].atom]++;
      }
    for (int a = 0; a < query->n_atoms; ++a)
      if (seen[a] != 1) fail(FJ_ERR_INVALID_ARG, "bushy: every atom must be one leaf");
    const int root = n_nodes - 1;
    if (bushy_vars(B, root) != [&] {
          uint64_t m = 0;
          for (const auto& vs : pq.atom_vars)
            for (int v : vs) m |= 1ull << v;
          return m;
        }())
      fail(FJ_ERR_INVALID_ARG, "bushy: the tree does not cover the query");
    const int mode = opts ? opts->out_mode : FJ_OUT_COUNT;
    bushy_run(B, root, mode, pq.head, opts, out);
    out->counters[FJ_CTR_KERNELS] = B.kernels;
  });
  const std::string msg = get_error();
  for (fj_rel* r : B.temps) fj_release_relation(ctx, r);
  for (void* p : B.dbufs) dfree(ctx, p);
  set_error(msg);
  return st;
}

void fj_result_free(fj_ctx* c, fj_result* res) {
  if (!c || !res || !res->d_tuples) return;
  if (res->tuples_owned) dfree(c, res->d_tuples);
  res->d_tuples = nullptr;
  res->tuples_owned = 0;
}

}  // extern "C"

extern "C" fj_status fj_batch_create(fj_ctx* ctx, int n, fj_prepared* const* preps, int flags,
                                     fj_batch** out) {
  return guarded([&] {
    if (!out) fail(FJ_ERR_INVALID_ARG, "NULL output");
    *out = batch_create(ctx, n, preps, flags);
  });
}

extern "C" fj_status fj_batch_launch(fj_batch* batch) {
  return guarded([&] {
    if (!batch) fail(FJ_ERR_INVALID_ARG, "NULL batch");
    batch_launch(batch);
  });
}

extern "C" fj_status fj_batch_results(fj_batch* batch, fj_result* results) {
  return guarded([&] {
    if (!batch || (!results && !batch->preps.empty())) fail(FJ_ERR_INVALID_ARG, "NULL argument");
    batch_results(batch, results);
  });
}

extern "C" fj_status fj_batch_execute(fj_batch* batch, fj_result* results) {
  return guarded([&] {
    if (!batch || (!batch->preps.empty() && !results)) fail(FJ_ERR_INVALID_ARG, "NULL argument");
    batch_launch(batch);
    batch_results(batch, results);
  });
}

extern "C" void fj_batch_free(fj_batch* batch) { batch_free(batch); }


cudaStream_t fj_internal_ctx_stream(const fj_ctx* c) { return c->stream; }
const int32_t* fj_internal_rel_col(const fj_rel* r, int col) {
  return r && col >= 0 && col < int(r->cols.size()) ? r->cols[col] : nullptr;
}
int fj_internal_ctx_device(const fj_ctx* c) { return c->device; }
