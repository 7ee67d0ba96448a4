// fj_join2_count_noalloc: a join entry point that allocates no memory.
//
// Some callers cannot allocate device memory on the path that runs the
// join: code that runs while a stream is being captured into a CUDA graph
// (allocation calls are not allowed there), services that run under a fixed,
// pre-reserved memory budget and must not grow it per request, and hosts
// that hand the library a stream but no allocator.  This entry point serves
// them for the simplest shape the library handles -- the bag COUNT of the
// equi-join R(x), S(x) -- by building the hash level of S in a fixed array
// that is part of the library image, then probing it with R.
//
// Scratch: g_scratch below, kMaxSlots 8-byte slots (8 MiB), a file-scope
// device array.  Every GPU that loads the library holds it until the process
// exits.  Every call shares it and it keeps the last call's contents; each
// call clears the part it uses first.  Calls that overlap on the GPU (on
// different streams, or from several host threads) race on it.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/fj.h"

namespace {

constexpr uint32_t kMaxSlots = 1u << 20;        // 8 MiB of 8-byte slots
constexpr uint64_t kMaxBuildRows = kMaxSlots / 2;  // load factor at most 1/2
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;

// Slot: key in the low 32 bits, count in the high 32 bits; 0 means empty
// (every occupied slot has a count of at least 1).
static __device__ __align__(256) unsigned long long g_scratch[kMaxSlots];

std::mutex g_mu;
unsigned long long* g_addr[kMaxDevices] = {};

thread_local char g_err[256];

__device__ __forceinline__ uint32_t mix(uint32_t h) {
  // 32-bit finalizer of MurmurHash3 (Austin Appleby, public domain).
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

__global__ void k_na_clear(unsigned long long* slots, uint32_t n, unsigned long long* count) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    slots[i] = 0ull;
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = 0ull;
}

// Count the rows of S per key.  Linear probing, bounded by the capacity.
__global__ void k_na_build(unsigned long long* slots, uint32_t mask, const int32_t* s, uint64_t n) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
       i += uint64_t(gridDim.x) * blockDim.x) {
    uint32_t k = uint32_t(s[i]);
    uint32_t h = mix(k) & mask;
    const unsigned long long claim = (1ull << 32) | k;
    for (uint32_t it = 0; it <= mask; ++it) {
      unsigned long long old = atomicCAS(&slots[h], 0ull, claim);
      if (old == 0ull) break;
      if (uint32_t(old) == k) {
        atomicAdd(&slots[h], 1ull << 32);
        break;
      }
      h = (h + 1) & mask;
    }
  }
}

// For every row of R, add the count of its key in S.
__global__ void k_na_probe(const unsigned long long* slots, uint32_t mask, const int32_t* r,
                           uint64_t n, unsigned long long* count) {
  unsigned long long mine = 0;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
       i += uint64_t(gridDim.x) * blockDim.x) {
    uint32_t k = uint32_t(r[i]);
    uint32_t h = mix(k) & mask;
    for (uint32_t it = 0; it <= mask; ++it) {
      unsigned long long v = slots[h];
      if (v == 0ull) break;
      if (uint32_t(v) == k) {
        mine += v >> 32;
        break;
      }
      h = (h + 1) & mask;
    }
  }
  for (int o = 16; o; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  __shared__ unsigned long long red[kThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    if (t) atomicAdd(count, t);
  }
}

fj_status fail(fj_status st, const char* msg) {
  snprintf(g_err, sizeof(g_err), "%s", msg);
  return st;
}

fj_status fail_cuda(const char* what, cudaError_t e) {
  snprintf(g_err, sizeof(g_err), "fj_join2_count_noalloc: %s: %s", what, cudaGetErrorString(e));
  return FJ_ERR_CUDA;
}

}  // namespace

extern "C" {

// Message of the last failure of fj_join2_count_noalloc on this thread.
const char* fj_noalloc_last_error(void) { return g_err; }

fj_status fj_join2_count_noalloc(const int32_t* d_r_key, uint64_t n_r, const int32_t* d_s_key,
                                 uint64_t n_s, uint64_t* d_count, void* cuda_stream) {
  g_err[0] = 0;
  if (!d_count || (n_r && !d_r_key) || (n_s && !d_s_key))
    return fail(FJ_ERR_INVALID_ARG, "fj_join2_count_noalloc: NULL pointer");
  if (n_s > kMaxBuildRows)
    return fail(FJ_ERR_INVALID_ARG,
                "fj_join2_count_noalloc: S has more than 524288 rows (the fixed scratch "
                "table holds 1048576 slots at load factor 1/2)");
  // An error left pending by the caller's earlier work is reported as such
  // and left in place (not consumed, not blamed on this call's launches).
  const cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess) return fail_cuda("a CUDA error was pending before the call", pending);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(FJ_ERR_CUDA, "fj_join2_count_noalloc: no current CUDA device");
  unsigned long long* slots;
  {
    // Once per device, with that device current: the device address of the
    // scratch array (the host-side symbol is not a device address).
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess) return fail_cuda("cudaGetSymbolAddress", e);
      if (!p) return fail(FJ_ERR_CUDA, "fj_join2_count_noalloc: cudaGetSymbolAddress gave NULL");
      g_addr[dev] = static_cast<unsigned long long*>(p);
    }
    slots = g_addr[dev];
  }
  uint32_t cap = 16;
  while (uint64_t(cap) < 2 * n_s) cap <<= 1;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int grid_c = int((cap + kThreads - 1) / kThreads);
  if (grid_c > 4096) grid_c = 4096;
  k_na_clear<<<grid_c, kThreads, 0, s>>>(slots, cap, reinterpret_cast<unsigned long long*>(d_count));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_cuda("clear launch", e);
  if (n_s) {
    uint64_t g = (n_s + kThreads - 1) / kThreads;
    k_na_build<<<int(g < 4096 ? g : 4096), kThreads, 0, s>>>(slots, cap - 1, d_s_key, n_s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda("build launch", e);
  }
  if (n_r) {
    uint64_t g = (n_r + kThreads - 1) / kThreads;
    k_na_probe<<<int(g < 4096 ? g : 4096), kThreads, 0, s>>>(
        slots, cap - 1, d_r_key, n_r, reinterpret_cast<unsigned long long*>(d_count));
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda("probe launch", e);
  }
  return FJ_OK;
}

}  // extern "C"
