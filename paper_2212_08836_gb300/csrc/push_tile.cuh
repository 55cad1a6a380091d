// Mover + deposit of rows a2, a3 and a6 (Sec. 2.1, Eqs. 3-4) for the FP32
// particle store of the mixed form, as one streaming kernel.
//
// The store is streamed in tiles of kTile consecutive particles.  One thread
// of each block copies a tile's seven arrays (cell, a, b, v_r, v_theta, v_z,
// w) from global into shared memory with 1-D bulk copies of the tensor memory
// accelerator, kStages tiles ahead, each stage tracked by an mbarrier; the
// threads read their particles from shared memory, so the loads cost no
// address arithmetic and no registers for prefetching.  Per tile:
//   1. in-cell phase: each thread takes kPPT particles; the in-cell CN step
//      (the scalar Newton solve of push_general.cuh) for particles that stay
//      in their cell, deposits summed per warp and added with FP64 atomics,
//      the rest appended to a shared-memory list of the tile;
//   2. crosser phase: the block's threads take the listed particles, one per
//      thread, through the general sub-step path, reading their start state
//      and the in-cell phase's converged whole-step trial from shared memory.
// Crossers are finished inside their tile: no global queue, no second launch
// and no scattered re-read of their state from the store.
#pragma once

#include <cstddef>

#include "push_kernels.cuh"

namespace pic {
namespace {

constexpr int kTileThreads = 256;
constexpr int kTileWarps = kTileThreads / 32;
constexpr int kWT = 64;                        // particles per warp tile (two per lane)
constexpr int kStages = 3;                     // warp tiles in flight per warp
constexpr int kTileArrays = 7;                 // cell, a, b, vr, vt, vz, w
// a warp's crosser lists hold fewer than 32 entries each between batches,
// plus the at most kWT a tile adds
constexpr int kListCap = 32 + kWT;
// an mbarrier wait gives up after this many polls (each after a short sleep),
// about a second: the copies of a tile normally land within microseconds
constexpr unsigned kWaitPolls = 1u << 24;

// a warp's crossers of one kind: store index and the in-cell step's converged
// whole-step trial (the start state is read back from the store, which this
// pass streamed through L2 moments before)
struct CrossList {
  unsigned idx[kListCap];
  float da[kListCap], db[kListCap];
};

// one warp's private pipeline: staged tiles, their barriers, its lists.
// Aligned so that every warp's staged arrays start on a 16-byte boundary, as
// the bulk copies require (an unaligned size would shift the next warp's)
struct __align__(128) WarpSmem {
  float st[kStages][kTileArrays][kWT];  // staged tiles (cell as int bits)
  unsigned long long bar[kStages];
  int issued[kStages];                  // tiles copied into the stage so far
  // crossers whose trial leaves the cell through a z-face only (one sub-step
  // sequence for all: a z-landing, then the next cell) and the rest; a full
  // warp of either kind runs the general path together
  CrossList zl, gl;
};
constexpr size_t kTileSmemBytes = sizeof(WarpSmem) * kTileWarps;
static_assert(sizeof(WarpSmem) % 16 == 0, "each warp's pipeline starts 16-byte aligned");
static_assert(offsetof(WarpSmem, st) % 16 == 0 && (kWT * 4) % 16 == 0,
              "every staged array starts 16-byte aligned");
static_assert(offsetof(WarpSmem, bar) % 8 == 0, "mbarriers are 8-byte aligned");

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// lane 0: bulk copies of warp tile t (particles [t kWT, ...) of n) into stage s
__device__ __forceinline__ bool issue_tile(WarpSmem &W, int s, const PartsT<float> &P, long long t,
                                           long long n) {
  const long long p0 = t * kWT;
  const long long cnt = n - p0 < kWT ? n - p0 : kWT;
  // whole 16-byte granules: the store's arrays start on 256-byte boundaries
  // and each is padded to the next one, so the granule past n stays inside
  // the array's piece of the workspace
  const uint32_t bytes = (uint32_t)((cnt * 4 + 15) & ~15ll);
  const uint32_t bar = smem_addr(&W.bar[s]);
  const void *src[kTileArrays] = {P.cell + p0, P.a + p0, P.b + p0, P.vr + p0,
                                  P.vt + p0,   P.vz + p0, P.w + p0};
  // a misaligned source or destination is never copied (the wait for it then
  // times out and the kernel reports the error)
  uintptr_t al = smem_addr(&W.st[s][0][0]);
#pragma unroll
  for (int k = 0; k < kTileArrays; ++k) al |= (uintptr_t)src[k];
  if (al & 15u) return false;
  W.issued[s] += 1;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile(
      "{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(bar),
      "r"(bytes * kTileArrays)
      : "memory");
#pragma unroll
  for (int k = 0; k < kTileArrays; ++k)
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(&W.st[s][k][0])),
        "l"(src[k]), "r"(bytes), "r"(bar)
        : "memory");
  return true;
}

// bounded wait for the given phase parity of stage s; false on time-out
__device__ __forceinline__ bool wait_tile(WarpSmem &W, int s, uint32_t parity) {
  const uint32_t bar = smem_addr(&W.bar[s]);
  for (unsigned i = 0; i < kWaitPolls; ++i) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    __nanosleep(64);
  }
  return false;
}

// the general sub-step path for the list entries [e0, e0 + m) of a warp, one
// per lane (lanes >= m idle); entries next to the axis go to the FP64 list
template <bool kZ>
__device__ __forceinline__ void run_crossers(const PushLaunchT<float> &L, const GenArgs<float> &G,
                                             const CrossList &C, int e0, int m, int lane, int nz,
                                             Tally &tl) {
  if (lane >= m) return;
  const int e = e0 + lane;
  const long long p = C.idx[e];
  const int cj = L.p.cell[p];
  const float a = L.p.a[p], b = L.p.b[p], vr = L.p.vr[p], vt = L.p.vt[p], vz = L.p.vz[p],
              w = L.p.w[p];
  const float d = C.da[e];
  // FP64 next to the axis, where the centrifugal term amplifies FP32 rounding:
  // in the first radial cells, a radius below kPromoteRho cells at the start or
  // at the end of the whole-step trial, or an angular step |u_theta| >= rho/4
  bool prom = false;
  if (L.queue && cj >= 0 && cj < kPromoteRows * nz) {
    const int ic = cj / nz;
    const float rho = L.rm.rho0(ic) + a;
    prom = rho < kPromoteRho || fabsf(vt * L.rm.crr(ic)) >= 0.25f * rho ||
           (!Num<float>::nan_bits(d) && rho + d < kPromoteRho);
  }
  const unsigned am = __activemask();
  const unsigned pm = __ballot_sync(am, prom);
  if (prom) {
    const int leader = __ffs(pm) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(L.pcnt, (unsigned)__popc(pm));
    base = __shfl_sync(pm, base, leader);
    L.queue[base + __popc(pm & ((1u << lane) - 1u))] = (int)p;
  } else if (kZ) {
    push_zcross<float>(G, p, cj, a, b, vr, vt, vz, w, d, C.db[e], tl);
  } else {
    push_general<float, false>(G, p, cj, a, b, vr, vt, vz, w, d, C.db[e], tl);
  }
}

__global__ void __launch_bounds__(kTileThreads, 3) k_push_tile32(PushLaunchT<float> L) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  typedef Num<float> N;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  WarpSmem &W = reinterpret_cast<WarpSmem *>(smem_raw)[warp];
  const int nz = L.g.nz, nz1 = nz + 1, ncell = L.g.nr * nz;
  const float zero = 0.f, one = 1.f, h = 0.5f, q = 0.25f;
  const long long n = L.n_dev ? *L.n_dev : L.n;
  const long long ntiles = (n + kWT - 1) / kWT;
  // each warp of the grid streams a contiguous range of warp tiles [t0, t1):
  // consecutive tiles share cells (the store is sorted), so the field gathers
  // of one tile find the previous tile's lines in L1
  const long long gw = (long long)blockIdx.x * kTileWarps + warp;
  const long long nw = (long long)gridDim.x * kTileWarps;
  const long long per = (ntiles + nw - 1) / nw;
  const long long t0 = gw * per < ntiles ? gw * per : ntiles;
  const long long t1 = t0 + per < ntiles ? t0 + per : ntiles;
  unsigned n_newton = 0, n_acc = 0;
  Tally tl = {0, 0, 0, 0, 0, 0};
  GenArgs<float> G;
  G.nr = L.g.nr; G.nz = nz; G.ar = L.ar; G.az = L.az;
  G.wt = L.wbt; G.icr = L.icr; G.icz = L.icz; G.cz = L.cz; G.rm = L.rm;
  G.q = L.q; G.m = L.m; G.qf = L.qf; G.ir = L.ir; G.iz = L.iz; G.write = L.write; G.p = L.p;
  G.oop = L.oop; G.dst = L.dst; G.hist = L.hist;
  G.wall_z0 = L.wall_z0; G.wall_zl = L.wall_zl; G.wall_r = L.wall_r; G.ke_lost = L.ke_lost;
  int nzl = 0, ngl = 0;  // entries in this warp's lists (warp-uniform)

  if (lane == 0) {
    for (int s = 0; s < kStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&W.bar[s])) : "memory");
      W.issued[s] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int s = 0; s < kStages; ++s) {
      const long long t = t0 + s;
      if (t < t1) issue_tile(W, s, L.p, t, n);
    }
  }
  __syncwarp();

  bool failed = false;
  for (long long k = 0;; ++k) {
    const long long t = t0 + k;
    if (t >= t1) break;
    const int s = (int)(k % kStages);
    if (!wait_tile(W, s, (uint32_t)((k / kStages) & 1))) {
      failed = true;
      break;
    }
    const long long p0 = t * kWT;
    const int cnt = (int)(n - p0 < kWT ? n - p0 : kWT);
    const int32_t *cells = reinterpret_cast<const int32_t *>(W.st[s][0]);

#pragma unroll
    for (int r = 0; r < kWT / 32; ++r) {
      const int j = r * 32 + lane;
      const long long p = p0 + j;
      const bool live = j < cnt;
      const int c0 = live ? cells[j] : -1;
      float v0 = zero, v1 = zero, v2 = zero, v3 = zero;
      bool queued = false, zc = false;
      float d = zero, e = zero;
      int key = -1, ic = 0, jc = 0;
      if (c0 >= 0 && c0 < ncell) {
        key = c0;
        ic = __float2int_rz(__int2float_rn(c0) * L.inz);
        jc = c0 - ic * nz;
        if (jc < 0) { ic -= 1; jc += nz; }
        else if (jc >= nz) { ic += 1; jc -= nz; }
        const float a = W.st[s][1][j], b = W.st[s][2][j];
        const float crr = L.rm.crr(ic);
        const float ur = W.st[s][3][j] * crr, ut = W.st[s][4][j] * crr, uz = W.st[s][5][j] * L.cz;
        const float rho = L.rm.rho0(ic) + a;
        bool acc = false, trial = false;
        if (N::in01(a) && N::in01(b) && N::lt_abs(ut, q * rho)) {
          const float ar0 = __ldg(&L.ar[ic * nz1 + jc]);
          const float gar = __ldg(&L.ar[ic * nz1 + jc + 1]) - ar0;
          const float az0 = __ldg(&L.az[ic * nz + jc]);
          const float gaz = __ldg(&L.az[(ic + 1) * nz + jc]) - az0;
          const float zb = uz + h * (az0 + gaz * a);
          const float K = ur + h * (ar0 + gar * b) + q * gar * zb;
          const float k1 = one - 0.0625f * gar * gaz;
          if (N::gt(k1, h) && fast_solve<float>(rho, ut, K, k1, d, n_newton)) {
            trial = true;
            e = zb + q * gaz * d;
            const float a1 = a + d, b1 = b + e;
            acc = N::in01(a1) && N::in01(b1);
            zc = !acc && N::in01(a1) && (b1 < zero || b1 > one);
            if (acc) {
              n_acc++;
              const float qw = L.qf * W.st[s][6][j];
              const float fr = qw * d, fz = qw * e;
              const float am = a + h * d, bm = b + h * e;
              v1 = fr * bm;
              v0 = fr - v1;
              v3 = fz * am;
              v2 = fz - v3;
              if (L.write) {
                // CN velocity relations: the displacement is the mean of u and u'
                L.dst.a[p] = a1;
                L.dst.b[p] = b1;
                const float icr = L.rm.icrr(ic);
                L.dst.vr[p] = (2.f * d - ur) * icr;
                L.dst.vz[p] = (2.f * e - uz) * L.icz;
                L.dst.vt[p] = rho * ut * N::rcp(rho + d) * icr;
                if (L.oop) {
                  L.dst.cell[p] = c0;
                  L.dst.w[p] = W.st[s][6][j];
                  L.dst.id[p] = L.p.id[p];
                }
              }
            }
          }
        }
        queued = !acc;
        if (!trial) d = __int_as_float(0x7fc00000);  // no converged trial
      } else if (live && L.write && L.oop) {
        L.dst.cell[p] = c0;  // not pushed (absorbed earlier): stays out of the store
      }
      warp_deposit<float>(key, ic, jc, v0, v1, v2, v3, lane, nz, L.ir, L.iz);
      if (L.hist) {  // in-cell pushes: one sub-step (bin 0), one count per warp
        const unsigned m = __ballot_sync(0xffffffffu, key >= 0 && !queued);
        if (lane == 0 && m) atomicAdd(&L.hist[0], (unsigned long long)__popc(m));
      }
      // the rest joins one of this warp's crosser lists
      const unsigned zm = __ballot_sync(0xffffffffu, queued && zc);
      const unsigned gm = __ballot_sync(0xffffffffu, queued && !zc);
      if (queued) {
        const unsigned lt = (1u << lane) - 1u;
        CrossList &C = zc ? W.zl : W.gl;
        const int x = zc ? nzl + __popc(zm & lt) : ngl + __popc(gm & lt);
        C.idx[x] = (unsigned)p;
        C.da[x] = d;
        C.db[x] = e;
      }
      nzl += __popc(zm);
      ngl += __popc(gm);
    }
    // stage s is free: this warp's tile kStages ahead goes there
    __syncwarp();
    if (lane == 0) {
      const long long tn = t + kStages;
      if (tn < t1) issue_tile(W, s, L.p, tn, n);
    }
    // ---- full warps of crossers of one kind, taken from the top of a list
    while (nzl >= 32) {
      nzl -= 32;
      run_crossers<true>(L, G, W.zl, nzl, 32, lane, nz, tl);
      __syncwarp();
    }
    while (ngl >= 32) {
      ngl -= 32;
      run_crossers<false>(L, G, W.gl, ngl, 32, lane, nz, tl);
      __syncwarp();
    }
  }
  if (failed) {
    // a copy did not land in time: count it, and wait (again bounded) for the
    // last copy into each stage before the warp's shared memory is released
    if (lane == 0) {
      atomicAdd(L.kerr, 1ull);
      for (int s = 0; s < kStages; ++s)
        if (W.issued[s] > 0) wait_tile(W, s, (uint32_t)((W.issued[s] - 1) & 1));
    }
  } else {
    run_crossers<true>(L, G, W.zl, 0, nzl, lane, nz, tl);
    __syncwarp();
    run_crossers<false>(L, G, W.gl, 0, ngl, lane, nz, tl);
  }
  __syncwarp();
  flush_tally(L.counters, tl, lane, n_newton, n_acc);
}

// the listed near-axis crossers of one FP32 pass in FP64 arithmetic: state
// and accelerations read from the FP32 store, every sub-step solved in
// double, the end state rounded to FP32 once
__global__ void __launch_bounds__(128) k_push_promoted32(PushLaunchT<float> L) {
  const int lane = threadIdx.x & 31;
  const long long cnt = *L.pcnt;
  GenArgs<double, float> G;
  G.nr = L.g.nr; G.nz = L.g.nz; G.ar = L.ar; G.az = L.az;
  G.wt = 0.0; G.icr = L.icr64; G.icz = L.icz64; G.cz = L.cz64; G.rm = L.rm64;
  G.q = L.q; G.m = L.m; G.qf = L.q; G.ir = L.ir; G.iz = L.iz; G.write = L.write; G.p = L.p;
  G.oop = L.oop; G.dst = L.dst; G.hist = L.hist;
  G.wall_z0 = L.wall_z0; G.wall_zl = L.wall_zl; G.wall_r = L.wall_r; G.ke_lost = L.ke_lost;
  Tally tl = {0, 0, 0, 0, 0, 0};
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += stride) {
    const long long p = L.queue[k];
    push_general<double, false, float>(G, p, L.p.cell[p], (double)L.p.a[p], (double)L.p.b[p],
                                       (double)L.p.vr[p], (double)L.p.vt[p], (double)L.p.vz[p],
                                       (double)L.p.w[p], (double)NAN, (double)NAN, tl);
  }
  flush_tally(L.counters, tl, lane, 0, 0);
}

// resident blocks of the tile kernel (its shared memory set up once)
int tile_grid32() {
  static int nb = 0;
  if (nb == 0) {
    if (cudaFuncSetAttribute(k_push_tile32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kTileSmemBytes) != cudaSuccess)
      return 0;
    int v = 0, dev = 0, nsm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_push_tile32, kTileThreads,
                                                      kTileSmemBytes) != cudaSuccess || v < 1)
      v = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      nsm = 152;
    nb = v * nsm;
  }
  return nb;
}

}  // namespace

// FP32 store without B_z: one streaming launch per species and pass (the
// near-axis list's count is cleared first; launch_push_promoted32 follows)
inline cudaError_t launch_push_tile32(const PushLaunchT<float> &L, cudaStream_t s) {
  const long long nsz = L.n_dev ? L.cap : L.n;
  if (nsz <= 0) return cudaSuccess;
  const int wave = tile_grid32();
  if (wave <= 0) return cudaErrorInvalidConfiguration;
  const long long nb = ((nsz + kWT - 1) / kWT + kTileWarps - 1) / kTileWarps;
  long long g = L.fgrid > 0 ? L.fgrid : wave;
  if (g > nb) g = nb;
  if (L.queue && cudaMemsetAsync(L.pcnt, 0, sizeof(unsigned), s) != cudaSuccess)
    return cudaErrorInvalidValue;
  k_push_tile32<<<(unsigned)g, kTileThreads, kTileSmemBytes, s>>>(L);
  return cudaGetLastError();
}

// the near-axis crossers the tile kernel listed, in FP64 arithmetic
inline cudaError_t launch_push_promoted32(const PushLaunchT<float> &L, cudaStream_t s) {
  const long long nsz = L.n_dev ? L.cap : L.n;
  if (nsz <= 0 || !L.queue) return cudaSuccess;
  k_push_promoted32<<<304, 128, 0, s>>>(L);
  return cudaGetLastError();
}

}  // namespace pic
