// Work lists built without a global counter: block b of a persistent producer
// kernel appends to its own segment [b*seg, b*seg + count[b]) through a
// shared-memory counter, and a consumer kernel maps a dense index q in
// [0, sum of counts) to an entry with the exclusive prefix of the counts.
// One global atomic per appending warp on a single address contends across
// all SMs; the shared-memory counter does not.
#pragma once

#include "pic_internal.cuh"

namespace pic {

// warp-aggregated append to the block's segment; returns the entry index of
// this lane (valid where take is true).  s_cnt: the block's shared counter.
__device__ __forceinline__ long long seg_append(int *s_cnt, bool take, int lane, long long off) {
  const unsigned full = 0xffffffffu;
  unsigned m = __ballot_sync(full, take);
  if (!m) return -1;
  int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(s_cnt, __popc(m));
  base = __shfl_sync(full, base, leader);
  return off + base + __popc(m & ((1u << lane) - 1u));
}

// exclusive prefix of count[0..nblk) into s_pre[0..nblk] (blockDim 256,
// nblk <= kMaxFastBlocks); returns the total
__device__ __forceinline__ int seg_prefix(const int *count, int nblk, int *s_pre) {
  constexpr int kPer = (kMaxFastBlocks + 255) / 256;
  __shared__ int s_w[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int loc[kPer], sum = 0;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    int idx = threadIdx.x * kPer + k;
    loc[k] = idx < nblk ? count[idx] : 0;
    sum += loc[k];
  }
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  int wpre = 0;
  for (int k = 0; k < warp; ++k) wpre += s_w[k];
  int ex = wpre + incl - sum;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    int idx = threadIdx.x * kPer + k;
    if (idx < nblk) s_pre[idx] = ex;
    ex += loc[k];
  }
  if (threadIdx.x == 255) s_pre[nblk] = ex;
  __syncthreads();
  return s_pre[nblk];
}

// entry of dense index q (0 <= q < total): segment b with s_pre[b] <= q < s_pre[b+1]
__device__ __forceinline__ long long seg_entry(const int *s_pre, int nblk, long long seg, int q) {
  int lo = 0, hi = nblk;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (s_pre[mid] <= q) lo = mid;
    else hi = mid;
  }
  return (long long)lo * seg + (q - s_pre[lo]);
}

// the same for entries appended from the back of each segment (the r-th entry
// of segment b sits at b*seg + seg - 1 - r)
__device__ __forceinline__ long long seg_entry_back(const int *s_pre, int nblk, long long seg, int q) {
  int lo = 0, hi = nblk;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (s_pre[mid] <= q) lo = mid;
    else hi = mid;
  }
  return (long long)lo * seg + seg - 1 - (q - s_pre[lo]);
}

// blocks of 256 threads of a persistent kernel: resident blocks per SM x SMs
// (at most kMaxFastBlocks)
template <typename K>
int persistent_grid(K kernel) {
  int v = 0, dev = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, 256, 0) != cudaSuccess || v < 1)
    v = 1;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
    nsm = 152;
  long long nb = (long long)v * nsm;
  return (int)(nb < kMaxFastBlocks ? nb : kMaxFastBlocks);
}

}  // namespace pic
