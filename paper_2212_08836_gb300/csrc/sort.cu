// Row a8: counting sort of the particle SoA by cell (the per-cell fine
// sorting that the paper's GPU layer keeps, Sec. 2.1, after Mertmann 2011).
// histogram (warp-aggregated atomics) -> exclusive scan -> scatter with
// warp-aggregated per-cell cursors into the second buffer.  Absorbed
// particles (cell < 0) are dropped.  Also provides the device-wide exclusive
// scan used by the MCC append.
#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int SCAN_BS = 1024;
constexpr int SCAN_IPT = 4;
constexpr int SCAN_TILE = SCAN_BS * SCAN_IPT;
static_assert(SCAN_TILE == kScanTile, "scan tile and the scratch size it implies must agree");

// block-wide exclusive scan of int64 values held one per thread
__device__ long long block_excl_scan(long long v, long long *tot) {
  __shared__ long long warp_tot[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    long long t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) warp_tot[lane] = t;
  }
  __syncthreads();
  long long base = w > 0 ? warp_tot[w - 1] : 0;
  if (tot) *tot = warp_tot[(blockDim.x >> 5) - 1];
  long long r = base + x - v;
  __syncthreads();
  return r;
}

// per tile: local exclusive scan, tile sums
__global__ void __launch_bounds__(SCAN_BS) k_scan_tiles(const int32_t *in, int32_t *out,
                                                        long long n, long long *tile_sum) {
  long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_IPT;
  int v[SCAN_IPT];
  long long s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_IPT; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    s += v[k];
  }
  long long tot;
  long long off = block_excl_scan(s, &tot);
#pragma unroll
  for (int k = 0; k < SCAN_IPT; ++k) {
    if (base + k < n) out[base + k] = (int32_t)off;
    off += v[k];
  }
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// single block: exclusive scan of tile sums (any count, serial over chunks)
__global__ void __launch_bounds__(SCAN_BS) k_scan_sums(long long *sums, long long nt,
                                                       long long *total) {
  long long carry = 0;
  for (long long c0 = 0; c0 < nt; c0 += SCAN_BS) {
    long long i = c0 + threadIdx.x;
    long long v = i < nt ? sums[i] : 0;
    long long tot;
    long long off = block_excl_scan(v, &tot);
    if (i < nt) sums[i] = carry + off;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(256) k_scan_add(int32_t *out, long long n,
                                                  const long long *tile_off) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += (int32_t)tile_off[i / SCAN_TILE];
}

__global__ void __launch_bounds__(256) k_hist(const int32_t *cell, long long n, int ncell,
                                              int32_t *counts) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int c = p < n ? cell[p] : -1;
  if (c >= ncell) c = -1;
  unsigned peers = __match_any_sync(0xffffffffu, c);
  int lane = threadIdx.x & 31;
  int leader = __ffs(peers) - 1;
  if (c >= 0 && lane == leader) atomicAdd(&counts[c], __popc(peers));
}

// the source fields are loaded before the cursor atomic, so their latency
// overlaps it (one HBM round trip per particle instead of three in a row)
template <typename T>
__global__ void __launch_bounds__(256) k_scatter(SortLaunchT<T> S) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = p < S.n;
  int c = in ? S.src.cell[p] : -1;
  T a = 0, b = 0, vr = 0, vt = 0, vz = 0, w = 0;
  uint32_t id = 0;
  if (in) {
    a = S.src.a[p];
    b = S.src.b[p];
    vr = S.src.vr[p];
    vt = S.src.vt[p];
    vz = S.src.vz[p];
    w = S.src.w[p];
    id = S.src.id[p];
  }
  if (c >= S.ncell) c = -1;
  unsigned peers = __match_any_sync(0xffffffffu, c);
  int lane = threadIdx.x & 31;
  int leader = __ffs(peers) - 1;
  int base = 0;
  if (c >= 0 && lane == leader) base = atomicAdd(&S.cursor[c], __popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (c < 0) return;
  int rank = __popc(peers & ((1u << lane) - 1u));
  long long d = (long long)S.offs[c] + base + rank;
  S.dst.cell[d] = c;
  S.dst.a[d] = a;
  S.dst.b[d] = b;
  S.dst.vr[d] = vr;
  S.dst.vt[d] = vt;
  S.dst.vz[d] = vz;
  S.dst.w[d] = w;
  S.dst.id[d] = id;
}

}  // namespace

size_t scan_scratch_bytes(long long n) {
  long long nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  return (size_t)(nt + 1) * sizeof(long long);
}

cudaError_t scan_exclusive(const int32_t *in, int32_t *out, long long n, long long *total_dev,
                           void *scratch, cudaStream_t s) {
  if (n <= 0) return cudaMemsetAsync(total_dev, 0, sizeof(long long), s);
  long long nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  long long *sums = (long long *)scratch;
  k_scan_tiles<<<(unsigned)nt, SCAN_BS, 0, s>>>(in, out, n, sums);
  k_scan_sums<<<1, SCAN_BS, 0, s>>>(sums, nt, total_dev);
  k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, sums);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sort(const SortLaunchT<T> &S, cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(S.counts, 0, sizeof(int32_t) * (S.ncell + 1), s)) != cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(S.cursor, 0, sizeof(int32_t) * S.ncell, s)) != cudaSuccess) return e;
  if (S.n > 0) k_hist<<<(unsigned)((S.n + 255) / 256), 256, 0, s>>>(S.src.cell, S.n, S.ncell, S.counts);
  if ((e = scan_exclusive(S.counts, S.offs, S.ncell + 1, S.total, S.scan_scratch, s)) !=
      cudaSuccess)
    return e;
  if (S.n > 0) k_scatter<T><<<(unsigned)((S.n + 255) / 256), 256, 0, s>>>(S);
  return cudaGetLastError();
}

template cudaError_t launch_sort<double>(const SortLaunchT<double> &, cudaStream_t);
template cudaError_t launch_sort<float>(const SortLaunchT<float> &, cudaStream_t);

}  // namespace pic
