// Learned Picard start: a stack of 3x3 convolutions trained on the fields
// the method itself produces, used only as the initial iterate of the
// nonlinear iteration of Sec. 2.1.
//
// Activations and gradients are BF16 in planes of 8 channels: plane k holds
// channels 8k..8k+7 of every position (16 bytes per position), the channel
// count padded to a multiple of 16, on the grid with a one-point zero halo:
// positions run over batch x (nr+3) x (nz+3), and the halo points hold zeros,
// so every tap of a 3x3 convolution is a fixed offset in the position index
// (no boundary tests).  The network output is FP32, position-major, without
// the halo.
//
// Convolutions (forward and data gradient) run on the fifth-generation tensor
// cores: per tile of 128 positions, three bands of 130 input positions (the
// rows above, at and below the tile, one position either side) are copied by
// the tensor memory accelerator (one 3-D box per band: contiguous 2080-byte
// runs of every plane) into shared memory, where a plane of a band is exactly
// the no-swizzle K-major operand layout (8 rows x 16 bytes per core matrix);
// each tap is the band shifted by one row (a different start address of the
// same shared-memory descriptor), and tcgen05.mma accumulates the 9 taps in
// tensor memory; the epilogue reads it back with tcgen05.ld and stores each
// plane coalesced.  Weight gradients use mma.sync (positions as the reduction
// dimension).
//   forward      out[q][o] = b[o] + sum_{tap, c} W[tap][o][c] in[q + off(tap)][c]
//   data grad    dIn[q][c] = sum_{tap, o} W[8 - tap][o][c] dOut[q + off(tap)][o]
//                (the same kernel with the flipped, transposed weights), times
//                the ReLU derivative of the layer below
//   weight grad  dW[tap][o][c] = sum_q dOut[q][o] in[q + off(tap)][c]
// with off(tap) the neighbour (dy, dx) = (tap / 3 - 1, tap % 3 - 1).  FP32
// master weights and Adam state (Kingma & Ba 2015).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <vector>

#include "../../include/pic_guess.h"
#include "pic_internal.cuh"

namespace pic {
namespace {

typedef __nv_bfloat16 bf16;
constexpr int kBM = 64;        // positions per step of the weight-gradient kernel
constexpr int kMaxL = 8;       // most layers
constexpr int kWChunk = 2048;  // positions per block of the weight-gradient kernel
constexpr int kTM = 128;       // positions per tile of the tensor-core convolution (MMA M)
constexpr int kBand = kTM + 2; // input rows per band

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}

struct Geo {
  int H, W;             // grid points along r and z
  int Hp, Wp;           // with the halo
  int P, Pp;            // points per sample without / with the halo
  int npos, npp;        // batch x P, batch x Pp
  long long ps;         // elements between the planes of an activation buffer (capacity x 8)
};

// position q of the haloed grid: interior?  (*qu: its index without the halo)
__device__ __forceinline__ bool interior(const Geo &g, int q, int *qu) {
  const int b = q / g.Pp;
  const int r = q - b * g.Pp;
  const int yp = r / g.Wp, xp = r - yp * g.Wp;
  *qu = b * g.P + (yp - 1) * g.W + (xp - 1);
  return yp >= 1 && yp <= g.H && xp >= 1 && xp <= g.W;
}

// ---- tensor-core convolution ------------------------------------------------

// A band is copied as whole 128-byte rows of its planes (8 positions x 8
// channels): kGroups rows from the row holding its first position, so the
// band starts (first position mod 8) positions into each plane copy, an
// offset folded into the descriptors' start addresses like the taps' shifts.
constexpr int kGroups = 18;  // 144 positions >= 7 + kBand

// Shared memory of one CTA: kStages buffers of three bands (each CIN/8 planes
// of kGroups x 128 bytes, as the 3-D box lands), the nine taps' weights (CIN/8
// planes of COUT 16-byte rows each), the bias, the mbarriers (per stage: bands
// landed / stage free; per accumulator: MMAs done / epilogue done), an abort
// flag and the tensor-memory address.  As many stages (up to 4) as fit.
template <int CIN, int COUT>
struct TcLayout {
  static constexpr int kPlanes = CIN / 8;
  static constexpr int kLboA = kGroups * 128;
  static constexpr int kBandBytes = kPlanes * kLboA;
  static constexpr int kStageBytes = 3 * kBandBytes;
  static constexpr int kLboB = COUT * 16;
  static constexpr int kTapBytes = kPlanes * kLboB;
  static constexpr int kFixed = 9 * kTapBytes + COUT * 4 + 112;
  static constexpr int kStages = (227 * 1024 - kFixed) / kStageBytes > 4 ? 4
                                                                         : (227 * 1024 - kFixed) / kStageBytes;
  static constexpr int kOffW = kStages * kStageBytes;
  static constexpr int kOffBias = kOffW + 9 * kTapBytes;
  static constexpr int kOffBar = kOffBias + COUT * 4;
  static constexpr int kBytes = kOffBar + 112;
  static constexpr int kTmemCols = 2 * COUT < 32 ? 32 : 2 * COUT;  // two accumulators
  static constexpr uint32_t kTxBytes = 3u * kPlanes * kGroups * 128u;
  static constexpr int kEpiWarps = COUT >= 32 ? 8 : 4;  // two per TMEM lane quarter for 64 columns
  static constexpr int kThreads = 64 + 32 * kEpiWarps;   // warp 0 copies, warp 1 issues MMAs
  static_assert(kBandBytes % 128 == 0 && kTapBytes % 128 == 0 && kOffBar % 8 == 0, "alignment");
  static_assert(kTmemCols == 32 || kTmemCols == 64 || kTmemCols == 128 || kTmemCols == 256, "TMEM");
  static_assert(kStages >= 2 && kBytes <= 227 * 1024, "shared memory");
};

struct ConvArgs {
  Geo g;
  const bf16 *w;       // [9][COUT][CIN]
  const float *bias;   // [COUT] (modes 0, 1)
  const bf16 *mask;    // mode 2: ReLU output of the layer below, BF16 planes
  void *out;           // modes 0, 2: BF16 planes [COUT/8][ps]; mode 1: FP32 [npos][COUT]
  int ntiles;
  int *err;            // bit 0: a wait gave up; bit 2: misaligned shared memory
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: no swizzle, K-major core matrices of 8 rows
// x 16 bytes; lbo = bytes between core matrices along K, sbo = along M/N
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// bounded wait on an mbarrier phase (about a second at most); gives up early
// when another role has raised the abort flag, and raises it when it gives up
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, volatile int *abort) {
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 255) == 255 && *abort) return false;
  }
  *abort = 1;
  return false;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// first position of band dy of tile t, and the 128-byte row (8 positions)
// holding it (floor division: the first bands start before position 0)
__device__ __forceinline__ int band_start(const Geo &g, int t, int dy) {
  return t * kTM + (dy - 1) * g.Wp - 1;
}
__device__ __forceinline__ int band_group(const Geo &g, int t, int dy) {
  const int s = band_start(g, t, dy);
  return s >= 0 ? s >> 3 : -((7 - s) >> 3);
}

// the three bands of tile t into stage st (one thread)
template <int CIN, int COUT>
__device__ __forceinline__ void load_bands(const CUtensorMap *tm, const Geo &g, int t, int st,
                                           uint32_t base, uint32_t bar) {
  using Lt = TcLayout<CIN, COUT>;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
               "r"(Lt::kTxBytes)
               : "memory");
#pragma unroll
  for (int dy = 0; dy < 3; ++dy) {
    const uint32_t dst = base + st * Lt::kStageBytes + dy * Lt::kBandBytes;
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(tm), "r"(0), "r"(band_group(g, t, dy)), "r"(0), "r"(bar)
        : "memory");
  }
}

// the 9 taps x CIN/16 MMAs of the tile in stage st into accumulator j (one
// thread); the descriptors differ only in their start addresses, which stay
// below 256 KB, so each is the first one plus a constant
template <int CIN, int COUT>
__device__ __forceinline__ void issue_mmas(const Geo &g, int t, uint32_t base, int st, int j,
                                           uint32_t tmem) {
  using Lt = TcLayout<CIN, COUT>;
  int off[3];  // positions from the start of each plane copy to the band's first
#pragma unroll
  for (int dy = 0; dy < 3; ++dy) off[dy] = band_start(g, t, dy) - 8 * band_group(g, t, dy);
  constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(COUT >> 3) << 17) |
                             ((uint32_t)(kTM >> 4) << 24);  // f32 += bf16 x bf16, K-major A and B
  const uint32_t d = tmem + (uint32_t)(j * COUT);
  const uint64_t a0 = smem_desc(base + st * Lt::kStageBytes, Lt::kLboA, 128);
  const uint64_t b0 = smem_desc(base + Lt::kOffW, Lt::kLboB, 128);
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
#pragma unroll
    for (int kk = 0; kk < Lt::kPlanes / 2; ++kk) {
      const uint64_t ad = a0 + (uint64_t)(((tap / 3) * Lt::kBandBytes +
                                           (off[tap / 3] + tap % 3) * 16 + 2 * kk * Lt::kLboA) >> 4);
      const uint64_t bd = b0 + (uint64_t)((tap * Lt::kTapBytes + 2 * kk * Lt::kLboB) >> 4);
      const uint32_t acc = (tap | kk) != 0;
      asm volatile(
          "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
          "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
          "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
  }
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// N FP32 columns (16 or 32) of this thread's TMEM lane, waited for inside the
// same statement (the registers are not valid before tcgen05.wait::ld)
template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t ta, float *v) {
  uint32_t r[N];
  if constexpr (N == 16)
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta)
        : "memory");
  else
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(ta)
        : "memory");
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = __uint_as_float(r[i]);
}

// tile t's results from accumulator j: thread = one position (TMEM lane
// 32 quarter + lane), columns cbeg .. cbeg + N - 1
template <int COUT, int MODE, int N>
__device__ __forceinline__ void epilogue(const ConvArgs &a, const float *sbias, int t, int j,
                                         uint32_t tmem, int quarter, int cbeg) {
  const int lane = threadIdx.x & 31;
  const int q = t * kTM + 32 * quarter + lane;
  int qu = 0;
  const bool live = q < a.g.npp;
  const bool in = live && interior(a.g, q, &qu);
  float v[N];
  tmem_ld<N>(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(j * COUT + cbeg), v);
  if (MODE == 1) {
    if (in) {
      float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(a.out) + (long long)qu * COUT + cbeg);
#pragma unroll
      for (int i = 0; i < N / 4; ++i)
        o[i] = make_float4(v[4 * i] + sbias[cbeg + 4 * i], v[4 * i + 1] + sbias[cbeg + 4 * i + 1],
                           v[4 * i + 2] + sbias[cbeg + 4 * i + 2], v[4 * i + 3] + sbias[cbeg + 4 * i + 3]);
    }
    return;
  }
  if (!live) return;
  // mode 2: every plane's mask loaded before any store (the stores could alias
  // it as far as the compiler knows, which would serialise load and store)
  uint4 mk[N / 8];
  if (MODE == 2) {
#pragma unroll
    for (int k = 0; k < N / 8; ++k)
      mk[k] = __ldg(reinterpret_cast<const uint4 *>(a.mask + (long long)((cbeg >> 3) + k) * a.g.ps +
                                                    (long long)q * 8));
  }
#pragma unroll
  for (int k = 0; k < N / 8; ++k) {
    const long long off = (long long)((cbeg >> 3) + k) * a.g.ps + (long long)q * 8;
    float *w = v + 8 * k;
    if (MODE == 0) {
#pragma unroll
      for (int i = 0; i < 8; ++i) w[i] = in ? fmaxf(w[i] + sbias[cbeg + 8 * k + i], 0.f) : 0.f;
    } else {
      const bf16 *mb = reinterpret_cast<const bf16 *>(&mk[k]);
#pragma unroll
      for (int i = 0; i < 8; ++i) w[i] = (in && __bfloat162float(mb[i]) > 0.f) ? w[i] : 0.f;
    }
    *reinterpret_cast<uint4 *>(static_cast<bf16 *>(a.out) + off) =
        make_uint4(pack_bf16(w[0], w[1]), pack_bf16(w[2], w[3]), pack_bf16(w[4], w[5]),
                   pack_bf16(w[6], w[7]));
  }
}

// MODE 0: + bias, ReLU, BF16 out (halo points zero); 1: + bias, FP32 out
// without the halo; 2: times (mask > 0), BF16 out (halo points zero).
// Persistent and warp-specialised: CTA b takes tiles b, b + grid, ...; warp 0
// copies the bands of the coming tiles into a ring of kStages stages, warp 1
// issues each tile's MMAs into one of two TMEM accumulators as soon as its
// bands have landed and the accumulator is drained, and the remaining warps
// drain the accumulators (two warps per TMEM lane quarter for 64 channels),
// all ordered by mbarriers.
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(TcLayout<CIN, COUT>::kThreads)
    k_conv_tc(const __grid_constant__ CUtensorMap tm, ConvArgs a) {
  using Lt = TcLayout<CIN, COUT>;
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t base = smem_u32(sm);
  if ((base & 1023u) != 0u) {  // uniform: every thread sees the same base
    if (tid == 0) atomicOr(a.err, 4);
    return;
  }
  const uint32_t bar = base + Lt::kOffBar;
  constexpr int S = Lt::kStages;
  auto full = [&](int st) { return bar + 8u * st; };
  auto empty = [&](int st) { return bar + 32u + 8u * st; };
  auto accf = [&](int j) { return bar + 64u + 8u * j; };
  auto acce = [&](int j) { return bar + 80u + 8u * j; };
  volatile int *abort = reinterpret_cast<volatile int *>(sm + Lt::kOffBar + 96);
  uint32_t *slot = reinterpret_cast<uint32_t *>(sm + Lt::kOffBar + 100);
  float *sbias = reinterpret_cast<float *>(sm + Lt::kOffBias);
  if (tid == 0) {
    for (int k = 0; k < S; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full(k)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty(k)));
    }
    for (int k = 0; k < 2; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(accf(k)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(acce(k)), "n"(Lt::kEpiWarps));
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "n"(Lt::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  for (int e = tid; e < 9 * COUT * Lt::kPlanes; e += blockDim.x) {
    const int tap = e / (COUT * Lt::kPlanes), r = e - tap * (COUT * Lt::kPlanes);
    const int o = r / Lt::kPlanes, ch = r - o * Lt::kPlanes;
    *reinterpret_cast<uint4 *>(sm + Lt::kOffW + tap * Lt::kTapBytes + ch * Lt::kLboB + o * 16) =
        *reinterpret_cast<const uint4 *>(a.w + ((long long)tap * COUT + o) * CIN + ch * 8);
  }
  if (MODE != 2)
    for (int o = tid; o < COUT; o += blockDim.x) sbias[o] = a.bias[o];
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const int G = gridDim.x;
  if (warp == 0) {
    if (lane == 0) {
      int last[4] = {-1, -1, -1, -1};  // latest tile copied into each stage
      int k = 0;
      for (int t = blockIdx.x; t < a.ntiles; t += G, ++k) {
        const int st = k % S, u = k / S;
        if (u > 0 && !bar_wait(empty(st), (u - 1) & 1, abort)) break;
        load_bands<CIN, COUT>(&tm, a.g, t, st, base, full(st));
        last[st] = k;
      }
      if (*abort)  // let the copies in flight land (bounded)
        for (int st = 0; st < S; ++st)
          if (last[st] >= 0) {
            volatile int never = 0;
            bar_wait(full(st), (last[st] / S) & 1, &never);
          }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int lastk = -1;
      int k = 0;
      for (int t = blockIdx.x; t < a.ntiles; t += G, ++k) {
        const int st = k % S, j = k & 1, v = k >> 1;
        if (!bar_wait(full(st), (k / S) & 1, abort)) break;
        if (v > 0 && !bar_wait(acce(j), (v - 1) & 1, abort)) break;
        tc_fence_after();
        issue_mmas<CIN, COUT>(a.g, t, base, st, j, tmem);
        tc_commit(empty(st));
        tc_commit(accf(j));
        lastk = k;
      }
      if (*abort && lastk >= 0) {  // let the MMAs in flight finish (bounded)
        volatile int never = 0;
        bar_wait(accf(lastk & 1), (lastk >> 1) & 1, &never);
      }
    }
  } else {
    const int ew = warp - 2, quarter = warp & 3;
    constexpr int N = COUT >= 32 ? COUT / 2 : COUT;
    const int cbeg = COUT >= 32 ? (ew >> 2) * N : 0;
    int k = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += G, ++k) {
      const int j = k & 1, v = k >> 1;
      // warp-uniform: tcgen05.ld needs the whole warp
      if (!__all_sync(0xffffffffu, bar_wait(accf(j), v & 1, abort))) break;
      tc_fence_after();
      epilogue<COUT, MODE, N>(a, sbias, t, j, tmem, quarter, cbeg);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce(j)) : "memory");
    }
  }
  __syncthreads();
  if (tid == 0 && *abort) atomicOr(a.err, 1);
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "n"(Lt::kTmemCols));
}

// dW[tap][o][c] += sum over a chunk of positions of the haloed grid (dOut is
// zero on the halo); grid (chunks, 9).  The centre tap also accumulates the
// bias gradient.
template <int CIN, int COUT>
__global__ void __launch_bounds__(128) k_wgrad(Geo g, const bf16 *__restrict__ in,
                                               const bf16 *__restrict__ dz, float *dw,
                                               float *db) {
  constexpr int MT = COUT / 16, NTT = CIN / 8;
  constexpr int WM = MT >= 4 ? MT / 4 : 1;      // m-tiles per warp
  constexpr int WN = MT >= 4 ? NTT : NTT / 4;   // n-tiles per warp
  static_assert(MT >= 4 || NTT % 4 == 0, "tile split");
  constexpr int SK = kBM + 8;
  __shared__ __align__(16) bf16 Dt[COUT * SK];  // [o][q]
  __shared__ __align__(16) bf16 It[CIN * SK];   // [c][q]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gq = lane >> 2, t4 = lane & 3;
  const int tap = blockIdx.y, dy = tap / 3 - 1, dx = tap % 3 - 1;
  const int mbase = MT >= 4 ? warp * WM : 0;
  const int nbase = MT >= 4 ? 0 : warp * WN;
  float acc[WM][WN][4];
#pragma unroll
  for (int i = 0; i < WM; ++i)
#pragma unroll
    for (int j = 0; j < WN; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.f;
  float bsum = 0.f;  // bias gradient of channel tid (centre tap, tid < COUT)
  const long long c0 = (long long)blockIdx.x * kWChunk;
  const long long off = (long long)dy * g.Wp + dx;
  for (long long s0 = c0; s0 < c0 + kWChunk && s0 < g.npp; s0 += kBM) {
    for (int e = tid; e < kBM * (COUT / 8); e += 128) {
      const int k8 = e / kBM, r = e - k8 * kBM;
      const long long q = s0 + r;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (q < g.npp) v = *reinterpret_cast<const uint4 *>(dz + k8 * g.ps + q * 8);
      const bf16 *pv = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
      for (int j = 0; j < 8; ++j) Dt[(k8 * 8 + j) * SK + r] = pv[j];
    }
    for (int e = tid; e < kBM * (CIN / 8); e += 128) {
      const int k8 = e / kBM, r = e - k8 * kBM;
      const long long q = s0 + r;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      const long long nq = q + off;
      if (q < g.npp && nq >= 0 && nq < g.npp)
        v = *reinterpret_cast<const uint4 *>(in + k8 * g.ps + nq * 8);
      const bf16 *pv = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
      for (int j = 0; j < 8; ++j) It[(k8 * 8 + j) * SK + r] = pv[j];
    }
    __syncthreads();
    if (tap == 4 && tid < COUT)
      for (int r = 0; r < kBM; ++r) bsum += __bfloat162float(Dt[tid * SK + r]);
#pragma unroll
    for (int k0 = 0; k0 < kBM; k0 += 16) {
#pragma unroll
      for (int i = 0; i < WM; ++i) {
        const int mr = (mbase + i) * 16;
        uint32_t a[4];
        a[0] = *reinterpret_cast<const uint32_t *>(Dt + (mr + gq) * SK + k0 + 2 * t4);
        a[1] = *reinterpret_cast<const uint32_t *>(Dt + (mr + gq + 8) * SK + k0 + 2 * t4);
        a[2] = *reinterpret_cast<const uint32_t *>(Dt + (mr + gq) * SK + k0 + 8 + 2 * t4);
        a[3] = *reinterpret_cast<const uint32_t *>(Dt + (mr + gq + 8) * SK + k0 + 8 + 2 * t4);
#pragma unroll
        for (int j = 0; j < WN; ++j) {
          const int nc = (nbase + j) * 8;
          uint32_t b[2];
          b[0] = *reinterpret_cast<const uint32_t *>(It + (nc + gq) * SK + k0 + 2 * t4);
          b[1] = *reinterpret_cast<const uint32_t *>(It + (nc + gq) * SK + k0 + 8 + 2 * t4);
          mma16816(acc[i][j], a, b);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < WM; ++i)
#pragma unroll
    for (int j = 0; j < WN; ++j)
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        const int o = (mbase + i) * 16 + gq + 8 * hf;
        const int c = (nbase + j) * 8 + 2 * t4;
        float *d = dw + ((long long)tap * COUT + o) * CIN + c;
        atomicAdd(d, acc[i][j][2 * hf]);
        atomicAdd(d + 1, acc[i][j][2 * hf + 1]);
      }
  if (tap == 4 && tid < COUT) atomicAdd(&db[tid], bsum);
}

// NCHW FP32 [B][c_real][H][W] -> BF16 planes of the haloed grid (zero on the
// halo and in the padding channels); thread = (position, plane)
__global__ void k_pack(Geo g, int c_real, int cp, const float *x, bf16 *out) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)g.npp * (cp / 8)) return;
  const int k = (int)(t / g.npp), q = (int)(t - (long long)k * g.npp);
  int qu;
  const bool in = interior(g, q, &qu);
  const int b = qu / g.P, p = qu - b * g.P;
  float v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int c = 8 * k + i;
    v[i] = in && c < c_real ? x[((long long)b * c_real + c) * g.P + p] : 0.f;
  }
  *reinterpret_cast<uint4 *>(out + k * g.ps + (long long)q * 8) =
      make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                 pack_bf16(v[6], v[7]));
}

// position-major FP32 [B*P][cp] -> NCHW [B][c_real][H][W]
__global__ void k_unpack(Geo g, int c_real, int cp, const float *y, float *out) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.npos * c_real) return;
  long long b = t / (c_real * g.P);
  long long r = t - b * c_real * g.P;
  int c = (int)(r / g.P);
  long long p = r - (long long)c * g.P;
  out[t] = y[((long long)b * g.P + p) * cp + c];
}

// loss = mean over the batch of sum_valid (y - t)^2 / nvalid; dZ of the last
// layer (BF16, cp channels, haloed grid, zero on the halo) = d loss / d y.
// Valid: channel 0 on rows < H-1 (E_r), channel 1 on columns < W-1 (E_z).
__global__ void k_loss(Geo g, int cp, const float *y, const float *t, int batch, double nvalid,
                       bf16 *dz, double *acc) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (q < g.npp) {
    int qu;
    const bool in = interior(g, q, &qu);
    const int b = qu / g.P;
    const int p = qu - b * g.P;
    int yy = p / g.W, xx = p - (p / g.W) * g.W;
    const float sc = (float)(2.0 / ((double)batch * nvalid));
    for (int c = 0; c < cp; ++c) {
      float d = 0.f;
      bool valid = in && ((c == 0 && yy < g.H - 1) || (c == 1 && xx < g.W - 1));
      if (valid) {
        float r = y[(long long)qu * cp + c] - t[((long long)b * 2 + c) * g.P + p];
        l += (double)r * (double)r;
        d = sc * r;
      }
      dz[(c >> 3) * g.ps + (long long)q * 8 + (c & 7)] = __float2bfloat16_rn(d);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(acc, l / ((double)batch * nvalid));
}

struct LayerMeta {
  int L;
  int cin[kMaxL], cout[kMaxL], cinp[kMaxL], coutp[kMaxL];
  long long offw[kMaxL], offb[kMaxL];  // master layout: w (o, c, ky, kx) then b
  long long offdw[kMaxL];              // padded gradient buffer: [tap][op][cp] then b [op]
};

// master FP32 -> forward weights W[tap][op][cp], flipped data-grad weights
// Wb[tap][cp][op] = W[8 - tap][o][c], padded biases
__global__ void k_publish(LayerMeta M, int layer, const float *master, bf16 *wf, bf16 *wb,
                          float *bias) {
  const int ci = M.cin[layer], co = M.cout[layer], cp = M.cinp[layer], op = M.coutp[layer];
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long n = 9LL * op * cp;
  if (t < n) {
    int tap = (int)(t / ((long long)op * cp));
    int r = (int)(t - (long long)tap * op * cp);
    int o = r / cp, c = r - (r / cp) * cp;
    float v = 0.f;
    if (o < co && c < ci) v = master[M.offw[layer] + ((long long)(o * ci + c) * 9) + tap];
    wf[t] = __float2bfloat16_rn(v);
    wb[((long long)(8 - tap) * cp + c) * op + o] = __float2bfloat16_rn(v);
  }
  if (t < op) bias[t] = t < co ? master[M.offb[layer] + t] : 0.f;
}

// gradient in the master layout from the padded buffers, then Adam
__global__ void k_adam(LayerMeta M, long long nparam, const float *gpad, float *master, float *m,
                       float *v, float *gout, float lr, float bc1, float bc2, int update) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nparam) return;
  int l = 0;
  while (l + 1 < M.L && k >= M.offw[l + 1]) ++l;
  const int ci = M.cin[l], cp = M.cinp[l], op = M.coutp[l];
  float g;
  if (k < M.offb[l]) {
    long long r = k - M.offw[l];
    int tap = (int)(r % 9);
    long long oc = r / 9;
    int c = (int)(oc % ci), o = (int)(oc / ci);
    g = gpad[M.offdw[l] + ((long long)tap * op + o) * cp + c];
  } else {
    int o = (int)(k - M.offb[l]);
    g = gpad[M.offdw[l] + 9LL * op * cp + o];
  }
  if (gout) gout[k] = g;
  if (!update) return;
  float mm = 0.9f * m[k] + 0.1f * g;
  float vv = 0.999f * v[k] + 0.001f * g * g;
  m[k] = mm;
  v[k] = vv;
  master[k] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + 1e-8f);
}

int pad16(int c) { return (c + 15) / 16 * 16; }

}  // namespace
}  // namespace pic

using namespace pic;

struct pic_cnn {
  CUtensorMap tm_act[kMaxL];  // band copies of act[l] (cinp[l] channels)
  CUtensorMap tm_dz[2][2];    // of dz[k] with 16 / 64 channels
  pic_cnn_config cfg;
  cudaStream_t s;
  int nsm;
  int *err;            // set by the tensor-core kernels when a wait gives up
  LayerMeta M;
  long long nparam, ngpad;
  float *master, *m, *v, *gpad, *gtmp;
  bf16 *wf[kMaxL], *wb[kMaxL];
  float *bias[kMaxL];
  bf16 *act[kMaxL];    // act[0]: packed input; act[l]: output of layer l-1 (hidden);
                       // haloed grid [bmax*Pp][cinp[l]]
  float *out;          // [bmax*P][coutp(last)], without the halo
  bf16 *dz[2];         // gradient ping-pong, haloed grid [bmax*Pp][64]
  double *lossacc;
  int t;               // Adam steps taken
};

namespace {

struct Carve {
  char *base;
  size_t off, cap;
  void *take(size_t b) {
    off = (off + 255) & ~(size_t)255;
    void *p = base ? base + off : nullptr;
    off += b;
    return p;
  }
};

// positions of an activation plane: the haloed grid of the largest batch,
// rounded up to whole 128-byte rows of the tensor maps
long long cap_rows(const pic_cnn_config *c) {
  return ((long long)(c->nr + 3) * (c->nz + 3) * c->batch + 7) / 8 * 8;
}

bool cfg_ok(const pic_cnn_config *c) {
  return c && c->nr >= 1 && c->nz >= 1 && c->width == 64 && c->depth >= 2 && c->depth <= kMaxL &&
         c->batch >= 1 && c->batch <= 64;
}

void meta(const pic_cnn_config *c, LayerMeta &M, long long &np, long long &ng) {
  M.L = c->depth;
  np = 0;
  ng = 0;
  for (int l = 0; l < M.L; ++l) {
    M.cin[l] = l == 0 ? PIC_CNN_IN : c->width;
    M.cout[l] = l + 1 == M.L ? PIC_CNN_OUT : c->width;
    M.cinp[l] = pad16(M.cin[l]);
    M.coutp[l] = pad16(M.cout[l]);
    M.offw[l] = np;
    np += (long long)M.cout[l] * M.cin[l] * 9;
    M.offb[l] = np;
    np += M.cout[l];
    M.offdw[l] = ng;
    ng += 9LL * M.coutp[l] * M.cinp[l] + M.coutp[l];
  }
}

bool layout(pic_cnn *x, const pic_cnn_config *c, char *base, size_t *used) {
  Carve K{base, 0, 0};
  meta(c, x->M, x->nparam, x->ngpad);
  const long long P = (long long)(c->nr + 1) * (c->nz + 1);
  const long long NP = P * c->batch;
  const long long NPP = cap_rows(c);
  x->master = (float *)K.take(x->nparam * 4);
  x->m = (float *)K.take(x->nparam * 4);
  x->v = (float *)K.take(x->nparam * 4);
  x->gtmp = (float *)K.take(x->nparam * 4);
  x->gpad = (float *)K.take(x->ngpad * 4);
  for (int l = 0; l < x->M.L; ++l) {
    size_t nw = 9ull * x->M.coutp[l] * x->M.cinp[l];
    x->wf[l] = (bf16 *)K.take(nw * 2);
    x->wb[l] = (bf16 *)K.take(nw * 2);
    x->bias[l] = (float *)K.take(x->M.coutp[l] * 4);
    x->act[l] = (bf16 *)K.take((size_t)NPP * x->M.cinp[l] * 2);
  }
  x->out = (float *)K.take((size_t)NP * x->M.coutp[x->M.L - 1] * 4);
  x->dz[0] = (bf16 *)K.take((size_t)NPP * 64 * 2);
  x->dz[1] = (bf16 *)K.take((size_t)NPP * 64 * 2);
  x->lossacc = (double *)K.take(256);
  x->err = (int *)K.take(256);
  *used = K.off + 256;
  return true;
}

Geo geo(const pic_cnn *x, int batch) {
  Geo g;
  g.H = x->cfg.nr + 1;
  g.W = x->cfg.nz + 1;
  g.Hp = g.H + 2;
  g.Wp = g.W + 2;
  g.P = g.H * g.W;
  g.Pp = g.Hp * g.Wp;
  g.npos = g.P * batch;
  g.npp = g.Pp * batch;
  g.ps = 8LL * cap_rows(&x->cfg);
  return g;
}

// 3-D tensor map of a plane buffer (64 elements = 8 positions x 8 channels per
// 128-byte row, rows / 8 rows, cin / 8 planes): one box = kGroups rows of
// every plane, no swizzle, zero outside
cudaError_t encode_rows(CUtensorMap *m, void *ptr, int cin, long long rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return (PFN_cuTensorMapEncodeTiled_v12000)f;
  }();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dim[3] = {64, (cuuint64_t)(rows / 8), (cuuint64_t)(cin / 8)};
  cuuint64_t str[2] = {128, (cuuint64_t)rows * 16};
  cuuint32_t box[3] = {64, (cuuint32_t)kGroups, (cuuint32_t)(cin / 8)}, es[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ptr, dim, str, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t encode_maps(pic_cnn *x) {
  const long long rows = cap_rows(&x->cfg);
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < x->M.L && e == cudaSuccess; ++l)
    e = encode_rows(&x->tm_act[l], x->act[l], x->M.cinp[l], rows);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = encode_rows(&x->tm_dz[k][0], x->dz[k], 16, rows);
    if (e == cudaSuccess) e = encode_rows(&x->tm_dz[k][1], x->dz[k], 64, rows);
  }
  return e;
}

// resident CTAs per SM of one tensor-core kernel (shared memory and the 512
// tensor-memory columns), with its dynamic shared memory size set once
template <int CIN, int COUT, int MODE>
int tc_blocks_per_sm() {
  static const int n = [] {
    using Lt = TcLayout<CIN, COUT>;
    auto k = k_conv_tc<CIN, COUT, MODE>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Lt::kBytes) !=
        cudaSuccess)
      return 0;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, Lt::kThreads, Lt::kBytes) != cudaSuccess)
      return 0;
    return b < 512 / Lt::kTmemCols ? b : 512 / Lt::kTmemCols;
  }();
  return n;
}

template <int CIN, int COUT, int MODE>
cudaError_t conv_tc(pic_cnn *x, const CUtensorMap &tm, const Geo &g, const bf16 *w,
                    const float *bias, const bf16 *mask, void *out) {
  using Lt = TcLayout<CIN, COUT>;
  const int per_sm = tc_blocks_per_sm<CIN, COUT, MODE>();
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  ConvArgs a{g, w, bias, mask, out, (g.npp + kTM - 1) / kTM, x->err};
  const int grid = a.ntiles < x->nsm * per_sm ? a.ntiles : x->nsm * per_sm;
  k_conv_tc<CIN, COUT, MODE><<<grid, Lt::kThreads, Lt::kBytes, x->s>>>(tm, a);
  return cudaGetLastError();
}

cudaError_t publish(pic_cnn *x) {
  for (int l = 0; l < x->M.L; ++l) {
    long long n = 9LL * x->M.coutp[l] * x->M.cinp[l];
    k_publish<<<(unsigned)((n + 255) / 256), 256, 0, x->s>>>(x->M, l, x->master, x->wf[l],
                                                             x->wb[l], x->bias[l]);
  }
  return cudaGetLastError();
}

cudaError_t conv_fwd(pic_cnn *x, int l, const Geo &g) {
  const int ci = x->M.cinp[l], co = x->M.coutp[l];
  const bool last = l + 1 == x->M.L;
  void *out = last ? (void *)x->out : (void *)x->act[l + 1];
  const CUtensorMap &tm = x->tm_act[l];
  if (ci == 16 && co == 64 && !last)
    return conv_tc<16, 64, 0>(x, tm, g, x->wf[l], x->bias[l], nullptr, out);
  if (ci == 64 && co == 64 && !last)
    return conv_tc<64, 64, 0>(x, tm, g, x->wf[l], x->bias[l], nullptr, out);
  if (ci == 64 && co == 16 && last)
    return conv_tc<64, 16, 1>(x, tm, g, x->wf[l], x->bias[l], nullptr, out);
  return cudaErrorInvalidValue;
}

cudaError_t forward(pic_cnn *x, const float *xin, int batch) {
  Geo g = geo(x, batch);
  long long n = (long long)g.npp * 2;  // positions x planes of the 16 input channels
  k_pack<<<(unsigned)((n + 255) / 256), 256, 0, x->s>>>(g, PIC_CNN_IN, 16, xin, x->act[0]);
  for (int l = 0; l < x->M.L; ++l) {
    cudaError_t e = conv_fwd(x, l, g);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// backward from the loss; gradients into gpad (zeroed here)
cudaError_t backward(pic_cnn *x, const float *t, int batch) {
  Geo g = geo(x, batch);
  const int L = x->M.L;
  cudaError_t e = cudaMemsetAsync(x->gpad, 0, x->ngpad * 4, x->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(x->lossacc, 0, 8, x->s);
  if (e != cudaSuccess) return e;
  const double nvalid = (double)x->cfg.nr * (x->cfg.nz + 1) + (double)(x->cfg.nr + 1) * x->cfg.nz;
  const int cpo = x->M.coutp[L - 1];
  k_loss<<<(unsigned)((g.npp + 255) / 256), 256, 0, x->s>>>(g, cpo, x->out, t, batch, nvalid,
                                                            x->dz[0], x->lossacc);
  int cur = 0;
  const unsigned nch = (unsigned)((g.npp + kWChunk - 1) / kWChunk);
  dim3 wg(nch, 9);
  for (int l = L - 1; l >= 0; --l) {
    const int ci = x->M.cinp[l], co = x->M.coutp[l];
    float *dw = x->gpad + x->M.offdw[l];
    float *db = dw + 9LL * co * ci;
    const bf16 *dzl = x->dz[cur];
    if (ci == 64 && co == 16) k_wgrad<64, 16><<<wg, 128, 0, x->s>>>(g, x->act[l], dzl, dw, db);
    else if (ci == 64 && co == 64) k_wgrad<64, 64><<<wg, 128, 0, x->s>>>(g, x->act[l], dzl, dw, db);
    else if (ci == 16 && co == 64) k_wgrad<16, 64><<<wg, 128, 0, x->s>>>(g, x->act[l], dzl, dw, db);
    else return cudaErrorInvalidValue;
    if (l == 0) break;
    // data gradient into the layer below, times its ReLU derivative
    bf16 *nx = x->dz[cur ^ 1];
    const CUtensorMap &tmz = x->tm_dz[cur][co == 16 ? 0 : 1];
    cudaError_t ce;
    if (co == 16 && ci == 64)
      ce = conv_tc<16, 64, 2>(x, tmz, g, x->wb[l], nullptr, x->act[l], nx);
    else if (co == 64 && ci == 64)
      ce = conv_tc<64, 64, 2>(x, tmz, g, x->wb[l], nullptr, x->act[l], nx);
    else
      return cudaErrorInvalidValue;
    if (ce != cudaSuccess) return ce;
    cur ^= 1;
  }
  return cudaGetLastError();
}

int rc(cudaError_t e) { return e == cudaSuccess ? PIC_OK : PIC_E_CUDA; }

// after a stream synchronisation: PIC_E_CUDA if a tensor-core kernel gave up
int rc_err(pic_cnn *x, cudaError_t e) {
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, x->err, sizeof(int), cudaMemcpyDeviceToHost);
  return e == cudaSuccess && h == 0 ? PIC_OK : PIC_E_CUDA;
}

}  // namespace

extern "C" {

size_t pic_cnn_workspace_size(const pic_cnn_config *c) {
  if (!cfg_ok(c)) return 0;
  pic_cnn tmp;
  tmp.cfg = *c;
  size_t used = 0;
  layout(&tmp, c, nullptr, &used);
  return used;
}

int pic_cnn_init(const pic_cnn_config *c, void *ws, size_t bytes, void *stream, pic_cnn **out) {
  if (!out) return PIC_E_CONFIG;
  *out = nullptr;
  if (!cfg_ok(c)) return PIC_E_CONFIG;
  if (!ws || bytes < pic_cnn_workspace_size(c)) return PIC_E_WORKSPACE;
  pic_cnn *x = new pic_cnn();
  x->cfg = *c;
  x->s = (cudaStream_t)stream;
  x->t = 0;
  size_t used = 0;
  layout(x, c, (char *)ws, &used);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&x->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      encode_maps(x) != cudaSuccess) {
    delete x;
    return PIC_E_CUDA;
  }
  // He-normal weights from a fixed-seed generator on the host, zero biases
  std::vector<float> h(x->nparam, 0.f);
  uint64_t st = c->seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
  auto u01 = [&]() {
    st ^= st >> 12;
    st ^= st << 25;
    st ^= st >> 27;
    return ((st * 0x2545F4914F6CDD1Dull) >> 11) * (1.0 / 9007199254740992.0);
  };
  for (int l = 0; l < x->M.L; ++l) {
    double sd = sqrt(2.0 / (9.0 * x->M.cin[l]));
    for (long long k = x->M.offw[l]; k < x->M.offb[l]; ++k) {
      double a = u01(), b = u01();
      h[k] = (float)(sd * sqrt(-2.0 * log(1.0 - a)) * cos(6.283185307179586 * b));
    }
  }
  cudaError_t e = cudaMemcpyAsync(x->master, h.data(), x->nparam * 4, cudaMemcpyHostToDevice, x->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(x->m, 0, x->nparam * 4, x->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(x->v, 0, x->nparam * 4, x->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(x->err, 0, sizeof(int), x->s);
  if (e == cudaSuccess) e = publish(x);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->s);
  if (e != cudaSuccess) {
    delete x;
    return PIC_E_CUDA;
  }
  *out = x;
  return PIC_OK;
}

void pic_cnn_destroy(pic_cnn *x) { delete x; }

long long pic_cnn_num_params(const pic_cnn *x) { return x ? x->nparam : 0; }

int pic_cnn_get_params(pic_cnn *x, float *host) {
  if (!x || !host) return PIC_E_CONFIG;
  cudaError_t e = cudaMemcpyAsync(host, x->master, x->nparam * 4, cudaMemcpyDeviceToHost, x->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->s);
  return rc(e);
}

int pic_cnn_set_params(pic_cnn *x, const float *host) {
  if (!x || !host) return PIC_E_CONFIG;
  cudaError_t e = cudaMemcpyAsync(x->master, host, x->nparam * 4, cudaMemcpyHostToDevice, x->s);
  if (e == cudaSuccess) e = publish(x);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->s);
  return rc(e);
}

int pic_cnn_forward(pic_cnn *x, const float *xin, int batch, float *y) {
  if (!x || !xin || !y || batch < 1 || batch > x->cfg.batch) return PIC_E_CONFIG;
  cudaError_t e = forward(x, xin, batch);
  if (e == cudaSuccess) {
    Geo g = geo(x, batch);
    long long n = g.npos * PIC_CNN_OUT;
    k_unpack<<<(unsigned)((n + 255) / 256), 256, 0, x->s>>>(g, PIC_CNN_OUT, x->M.coutp[x->M.L - 1],
                                                            x->out, y);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->s);
  return rc_err(x, e);
}

int pic_cnn_loss_grad(pic_cnn *x, const float *xin, const float *t, int batch, double *loss,
                      float *grad) {
  if (!x || !xin || !t || batch < 1 || batch > x->cfg.batch) return PIC_E_CONFIG;
  cudaError_t e = forward(x, xin, batch);
  if (e == cudaSuccess) e = backward(x, t, batch);
  if (e == cudaSuccess) {
    k_adam<<<(unsigned)((x->nparam + 255) / 256), 256, 0, x->s>>>(
        x->M, x->nparam, x->gpad, x->master, x->m, x->v, x->gtmp, 0.f, 1.f, 1.f, 0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && grad)
    e = cudaMemcpyAsync(grad, x->gtmp, x->nparam * 4, cudaMemcpyDeviceToHost, x->s);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, x->lossacc, 8, cudaMemcpyDeviceToHost, x->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->s);
  return rc_err(x, e);
}

int pic_cnn_train_step(pic_cnn *x, const float *xin, const float *t, int batch, float lr,
                       double *loss) {
  if (!x || !xin || !t || batch < 1 || batch > x->cfg.batch || !(lr >= 0.f)) return PIC_E_CONFIG;
  cudaError_t e = forward(x, xin, batch);
  if (e == cudaSuccess) e = backward(x, t, batch);
  if (e == cudaSuccess) {
    x->t += 1;
    float bc1 = 1.f - powf(0.9f, (float)x->t), bc2 = 1.f - powf(0.999f, (float)x->t);
    k_adam<<<(unsigned)((x->nparam + 255) / 256), 256, 0, x->s>>>(
        x->M, x->nparam, x->gpad, x->master, x->m, x->v, nullptr, lr, bc1, bc2, 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = publish(x);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, x->lossacc, 8, cudaMemcpyDeviceToHost, x->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->s);
  return rc_err(x, e);
}

}  // extern "C"

namespace pic {
// forward of one sample on the network's stream without synchronising (the
// guess of pic_step): y = network output in the position-major FP32 buffer
int cnn_forward_async(pic_cnn *x, const float *xin, const float **y_posmajor, int *cp) {
  if (forward(x, xin, 1) != cudaSuccess) return PIC_E_CUDA;
  *y_posmajor = x->out;
  *cp = x->M.coutp[x->M.L - 1];
  return PIC_OK;
}
cudaStream_t cnn_stream(const pic_cnn *x) { return x->s; }
const int *cnn_err_flag(const pic_cnn *x) { return x->err; }
int cnn_layers(const pic_cnn *x) { return x->M.L; }
int cnn_grid(const pic_cnn *x, int *nr, int *nz) {
  *nr = x->cfg.nr;
  *nz = x->cfg.nz;
  return PIC_OK;
}
}  // namespace pic
