// Sampled key-degree histogram of one column, the chooser's feature:
// row i is sampled iff fmix32(i xor seed) % mod == 0 (the 32-bit finalizer
// of MurmurHash3, Austin Appleby, public domain); sampled keys are counted
// in an open-addressing table; a key seen c times among the m sampled rows
// of n has estimated degree c n / m and falls in the largest bucket b < 32
// with c n >= m 2^b (an exact integer form of floor(log2 degree)); the
// result is the fraction of distinct sampled keys per bucket.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "../../include/fj.h"
#include "fj_ctx_access.h"

namespace {

constexpr int kT = 256;

__device__ __forceinline__ uint32_t sample_mix(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// Slot: key in the low 32 bits, count in the high 32 bits; 0 = empty.
__global__ void k_hist_count(const int32_t* __restrict__ col, uint64_t n, uint32_t mod,
                             uint32_t seed, unsigned long long* slots, uint32_t mask,
                             unsigned long long* n_sampled, uint32_t* status) {
  unsigned long long mine = 0;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
       i += uint64_t(gridDim.x) * blockDim.x) {
    if (sample_mix(uint32_t(i) ^ seed) % mod != 0) continue;
    ++mine;
    const uint32_t k = uint32_t(__ldg(col + i));
    uint32_t h = sample_mix(k) & mask;
    const unsigned long long claim = (1ull << 32) | k;
    bool done = false;
    for (uint32_t it = 0; it <= mask && !done; ++it) {
      const unsigned long long old = atomicCAS(&slots[h], 0ull, claim);
      if (old == 0ull) {
        done = true;
      } else if (uint32_t(old) == k) {
        atomicAdd(&slots[h], 1ull << 32);
        done = true;
      } else {
        h = (h + 1) & mask;
      }
    }
    if (!done) atomicOr(status, 1u);
  }
  if (mine) atomicAdd(n_sampled, mine);
}

__global__ void k_hist_bucket(const unsigned long long* __restrict__ slots, uint32_t cap,
                              uint64_t n, const unsigned long long* n_sampled,
                              unsigned long long* hist /* 33: buckets, keys */) {
  __shared__ unsigned long long sh[33];
  if (threadIdx.x < 33) sh[threadIdx.x] = 0;
  __syncthreads();
  const unsigned long long m = *n_sampled;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < cap; s += gridDim.x * blockDim.x) {
    const unsigned long long v = slots[s];
    if (!v) continue;
    const unsigned long long cn = (v >> 32) * n;  // count * n (below 2^63 for n < 2^31)
    int b = 0;
    while (b < 31 && cn >= (m << (b + 1))) ++b;
    atomicAdd(&sh[b], 1ull);
    atomicAdd(&sh[32], 1ull);
  }
  __syncthreads();
  if (threadIdx.x < 33 && sh[threadIdx.x]) atomicAdd(&hist[threadIdx.x], sh[threadIdx.x]);
}

thread_local std::string g_stats_err;

fj_status stats_fail(fj_status st, const std::string& m) {
  g_stats_err = m;
  return st;
}

}  // namespace

extern "C" {

const char* fj_stats_last_error(void) { return g_stats_err.c_str(); }

fj_status fj_degree_histogram(fj_ctx* ctx, const int32_t* d_col, uint64_t n, uint32_t mod,
                              uint32_t seed, float* host_hist) {
  g_stats_err.clear();
  if (!ctx || !host_hist || (n && !d_col) || mod == 0)
    return stats_fail(FJ_ERR_INVALID_ARG, "bad histogram arguments");
  if (n >= (1ull << 31)) return stats_fail(FJ_ERR_INVALID_ARG, "column above 2^31 rows");
  for (int b = 0; b < 32; ++b) host_hist[b] = 0.f;
  // An error left pending by the caller's earlier work is reported and left
  // in place: the error reads below then only ever see this call's own.
  const cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess)
    return stats_fail(FJ_ERR_CUDA, std::string("a CUDA error was pending before the call: ") +
                                       cudaGetErrorString(pending));
  if (n == 0) return FJ_OK;
  cudaStream_t s = fj_internal_ctx_stream(ctx);
  const uint64_t expect = n / mod + 64;
  uint32_t cap = 64;
  while (uint64_t(cap) < 4 * expect && cap < (1u << 30)) cap <<= 1;
  unsigned long long* buf = nullptr;  // slots, n_sampled, hist[33], status
  const size_t words = size_t(cap) + 1 + 33;
  // Plain allocation: this runs once per column, outside any timed path,
  // and must leave no pending error behind for the caller's next launch.
  if (cudaMalloc(&buf, words * 8 + 8) != cudaSuccess) {
    cudaGetLastError();
    return stats_fail(FJ_ERR_OOM, "histogram scratch");
  }
  uint32_t* status = reinterpret_cast<uint32_t*>(buf + words);
  unsigned long long host[34];
  uint32_t st = 0;
  cudaError_t e = cudaMemsetAsync(buf, 0, words * 8 + 8, s);
  if (e == cudaSuccess) {
    int g = int(std::min<uint64_t>((n + kT - 1) / kT, 4096));
    k_hist_count<<<g, kT, 0, s>>>(d_col, n, mod, seed, buf, cap - 1, buf + cap, status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    int g2 = int(std::min<uint64_t>((cap + kT - 1) / kT, 1024));
    k_hist_bucket<<<g2, kT, 0, s>>>(buf, cap, n, buf + cap, buf + cap + 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, buf + cap + 1, 33 * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  const cudaError_t ef = cudaFree(buf);
  if (e == cudaSuccess) e = ef;
  cudaGetLastError();  // reported below, not left for the next launch
  if (e != cudaSuccess) return stats_fail(FJ_ERR_CUDA, cudaGetErrorString(e));
  if (st) return stats_fail(FJ_ERR_CUDA, "histogram table overfilled");
  if (host[32])
    for (int b = 0; b < 32; ++b) host_hist[b] = float(double(host[b]) / double(host[32]));
  return FJ_OK;
}

}  // extern "C"
