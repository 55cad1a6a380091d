// Learned Picard start: a stack of 3x3 convolutions trained on the fields
// the method itself produces, used only as the initial iterate of the
// nonlinear iteration of Sec. 2.1.
//
// Tensors inside are channels-last (position-major) BF16 with the channel
// count padded to a multiple of 16; positions run over batch x (nr+1) x (nz+1).
// Every convolution is an implicit GEMM on the tensor cores
// (mma.sync m16n8k16, BF16 operands, FP32 accumulation):
//   forward      out[q][o] = b[o] + sum_{tap, c} W[tap][o][c] in[q + off(tap)][c]
//   data grad    dIn[q][c] = sum_{tap, o} W[8 - tap][o][c] dOut[q + off(tap)][o]
//                (the same kernel with the flipped, transposed weights), times
//                the ReLU derivative of the layer below
//   weight grad  dW[tap][o][c] = sum_q dOut[q][o] in[q + off(tap)][c]
// with off(tap) the neighbour (dy, dx) = (tap / 3 - 1, tap % 3 - 1) and zero
// outside the grid.  FP32 master weights and Adam state (Kingma & Ba 2015).
#include <cuda_bf16.h>

#include <vector>

#include "../../include/pic_guess.h"
#include "pic_internal.cuh"

namespace pic {
namespace {

typedef __nv_bfloat16 bf16;
constexpr int kBM = 64;        // positions per block of the convolution kernels
constexpr int kMaxL = 8;       // most layers
constexpr int kWChunk = 2048;  // positions per block of the weight-gradient kernel

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
  int H, W;
  long long P, npos;  // points per sample, batch x P
};

// neighbour of position q at (dy, dx), or -1 outside the grid
__device__ __forceinline__ long long neighbour(const Geo &g, long long q, int dy, int dx) {
  long long b = q / g.P;
  int p = (int)(q - b * g.P);
  int y = p / g.W, x = p - y * g.W;
  int yy = y + dy, xx = x + dx;
  if (yy < 0 || yy >= g.H || xx < 0 || xx >= g.W) return -1;
  return b * g.P + (long long)yy * g.W + xx;
}

// MODE 0: + bias, ReLU, BF16 out; 1: + bias, FP32 out; 2: times (mask > 0), BF16 out
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(128) k_conv(Geo g, const bf16 *__restrict__ in,
                                              const bf16 *__restrict__ w,
                                              const float *__restrict__ bias,
                                              const bf16 *__restrict__ mask, void *out) {
  constexpr int SA = CIN + 8;  // row stride in shared memory (conflict-free fragments)
  constexpr int CH = CIN / 8;  // 16-byte chunks per row
  constexpr int NT = COUT / 8;
  __shared__ __align__(16) bf16 As[kBM * SA];
  __shared__ __align__(16) bf16 Ws[COUT * SA];
  __shared__ long long rowq[kBM];
  __shared__ int rowy[kBM], rowx[kBM];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gq = lane >> 2, t4 = lane & 3;
  const long long m0 = (long long)blockIdx.x * kBM;
  if (tid < kBM) {
    long long q = m0 + tid;
    if (q < g.npos) {
      long long b = q / g.P;
      int p = (int)(q - b * g.P);
      rowy[tid] = p / g.W;
      rowx[tid] = p - (p / g.W) * g.W;
      rowq[tid] = q;
    } else {
      rowy[tid] = -1000000;
      rowx[tid] = 0;
      rowq[tid] = 0;
    }
  }
  float acc[NT][4];
#pragma unroll
  for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  __syncthreads();
  for (int tap = 0; tap < 9; ++tap) {
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    for (int c = tid; c < kBM * CH; c += 128) {
      const int r = c / CH, k8 = c - (c / CH) * CH;
      const int yy = rowy[r] + dy, xx = rowx[r] + dx;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (yy >= 0 && yy < g.H && xx >= 0 && xx < g.W)
        v = *reinterpret_cast<const uint4 *>(in + (rowq[r] + (long long)dy * g.W + dx) * CIN + k8 * 8);
      *reinterpret_cast<uint4 *>(As + r * SA + k8 * 8) = v;
    }
    for (int c = tid; c < COUT * CH; c += 128) {
      const int r = c / CH, k8 = c - (c / CH) * CH;
      *reinterpret_cast<uint4 *>(Ws + r * SA + k8 * 8) =
          *reinterpret_cast<const uint4 *>(w + ((long long)tap * COUT + r) * CIN + k8 * 8);
    }
    __syncthreads();
    const bf16 *Aw = As + warp * 16 * SA;
#pragma unroll
    for (int k0 = 0; k0 < CIN; k0 += 16) {
      uint32_t a[4];
      a[0] = *reinterpret_cast<const uint32_t *>(Aw + gq * SA + k0 + 2 * t4);
      a[1] = *reinterpret_cast<const uint32_t *>(Aw + (gq + 8) * SA + k0 + 2 * t4);
      a[2] = *reinterpret_cast<const uint32_t *>(Aw + gq * SA + k0 + 8 + 2 * t4);
      a[3] = *reinterpret_cast<const uint32_t *>(Aw + (gq + 8) * SA + k0 + 8 + 2 * t4);
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        uint32_t b[2];
        b[0] = *reinterpret_cast<const uint32_t *>(Ws + (n * 8 + gq) * SA + k0 + 2 * t4);
        b[1] = *reinterpret_cast<const uint32_t *>(Ws + (n * 8 + gq) * SA + k0 + 8 + 2 * t4);
        mma16816(acc[n], a, b);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int n = 0; n < NT; ++n) {
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      const int row = warp * 16 + gq + 8 * hf;
      const long long q = m0 + row;
      if (q >= g.npos) continue;
      const int col = n * 8 + 2 * t4;
      float v0 = acc[n][2 * hf], v1 = acc[n][2 * hf + 1];
      if (MODE == 0 || MODE == 1) {
        v0 += bias[col];
        v1 += bias[col + 1];
      }
      if (MODE == 0) {
        v0 = fmaxf(v0, 0.f);
        v1 = fmaxf(v1, 0.f);
      }
      if (MODE == 2) {
        __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162 *>(mask + q * COUT + col);
        if (!(__low2float(mk) > 0.f)) v0 = 0.f;
        if (!(__high2float(mk) > 0.f)) v1 = 0.f;
      }
      if (MODE == 1)
        *reinterpret_cast<float2 *>(static_cast<float *>(out) + q * COUT + col) = make_float2(v0, v1);
      else
        *reinterpret_cast<uint32_t *>(static_cast<bf16 *>(out) + q * COUT + col) = pack_bf16(v0, v1);
    }
  }
}

// dW[tap][o][c] += sum over a chunk of positions; grid (chunks, 9).  The
// centre tap also accumulates the bias gradient.
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
  for (long long s0 = c0; s0 < c0 + kWChunk && s0 < g.npos; s0 += kBM) {
    for (int e = tid; e < kBM * (COUT / 8); e += 128) {
      const int r = e / (COUT / 8), k8 = e - (e / (COUT / 8)) * (COUT / 8);
      const long long q = s0 + r;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (q < g.npos) v = *reinterpret_cast<const uint4 *>(dz + q * COUT + k8 * 8);
      const bf16 *pv = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
      for (int j = 0; j < 8; ++j) Dt[(k8 * 8 + j) * SK + r] = pv[j];
    }
    for (int e = tid; e < kBM * (CIN / 8); e += 128) {
      const int r = e / (CIN / 8), k8 = e - (e / (CIN / 8)) * (CIN / 8);
      const long long q = s0 + r;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (q < g.npos) {
        long long nq = neighbour(g, q, dy, dx);
        if (nq >= 0) v = *reinterpret_cast<const uint4 *>(in + nq * CIN + k8 * 8);
      }
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

// NCHW FP32 [B][c_real][H][W] -> position-major BF16 [B*P][cp] (zero padding channels)
__global__ void k_pack(Geo g, int c_real, int cp, const float *x, bf16 *out) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.npos * cp) return;
  long long q = t / cp;
  int c = (int)(t - q * cp);
  long long b = q / g.P, p = q - b * g.P;
  float v = c < c_real ? x[(b * c_real + c) * g.P + p] : 0.f;
  out[t] = __float2bfloat16_rn(v);
}

// position-major FP32 [B*P][cp] -> NCHW [B][c_real][H][W]
__global__ void k_unpack(Geo g, int c_real, int cp, const float *y, float *out) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.npos * c_real) return;
  long long b = t / (c_real * g.P);
  long long r = t - b * c_real * g.P;
  int c = (int)(r / g.P);
  long long p = r - (long long)c * g.P;
  out[t] = y[(b * g.P + p) * cp + c];
}

// loss = mean over the batch of sum_valid (y - t)^2 / nvalid; dZ of the last
// layer (BF16, cp channels) = d loss / d y.  Valid: channel 0 on rows < H-1
// (E_r), channel 1 on columns < W-1 (E_z).
__global__ void k_loss(Geo g, int cp, const float *y, const float *t, int batch, double nvalid,
                       bf16 *dz, double *acc) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (q < g.npos) {
    long long b = q / g.P;
    int p = (int)(q - b * g.P);
    int yy = p / g.W, xx = p - (p / g.W) * g.W;
    const float sc = (float)(2.0 / ((double)batch * nvalid));
    for (int c = 0; c < cp; ++c) {
      float d = 0.f;
      bool valid = (c == 0 && yy < g.H - 1) || (c == 1 && xx < g.W - 1);
      if (valid) {
        float r = y[q * cp + c] - t[(b * 2 + c) * g.P + p];
        l += (double)r * (double)r;
        d = sc * r;
      }
      dz[q * cp + c] = __float2bfloat16_rn(d);
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
  pic_cnn_config cfg;
  cudaStream_t s;
  Geo geo1;            // batch 1
  LayerMeta M;
  long long nparam, ngpad;
  float *master, *m, *v, *gpad, *gtmp;
  bf16 *wf[kMaxL], *wb[kMaxL];
  float *bias[kMaxL];
  bf16 *act[kMaxL];    // act[0]: packed input; act[l]: output of layer l-1 (hidden)
  float *out;          // [bmax*P][coutp(last)]
  bf16 *dz[2];         // gradient ping-pong [bmax*P][64]
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
    x->act[l] = (bf16 *)K.take((size_t)NP * x->M.cinp[l] * 2);
  }
  x->out = (float *)K.take((size_t)NP * x->M.coutp[x->M.L - 1] * 4);
  x->dz[0] = (bf16 *)K.take((size_t)NP * 64 * 2);
  x->dz[1] = (bf16 *)K.take((size_t)NP * 64 * 2);
  x->lossacc = (double *)K.take(256);
  *used = K.off + 256;
  return true;
}

Geo geo(const pic_cnn *x, int batch) {
  Geo g;
  g.H = x->cfg.nr + 1;
  g.W = x->cfg.nz + 1;
  g.P = (long long)g.H * g.W;
  g.npos = g.P * batch;
  return g;
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
  dim3 grid((unsigned)((g.npos + kBM - 1) / kBM));
  void *out = last ? (void *)x->out : (void *)x->act[l + 1];
  if (ci == 16 && co == 64 && !last)
    k_conv<16, 64, 0><<<grid, 128, 0, x->s>>>(g, x->act[l], x->wf[l], x->bias[l], nullptr, out);
  else if (ci == 64 && co == 64 && !last)
    k_conv<64, 64, 0><<<grid, 128, 0, x->s>>>(g, x->act[l], x->wf[l], x->bias[l], nullptr, out);
  else if (ci == 64 && co == 16 && last)
    k_conv<64, 16, 1><<<grid, 128, 0, x->s>>>(g, x->act[l], x->wf[l], x->bias[l], nullptr, out);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t forward(pic_cnn *x, const float *xin, int batch) {
  Geo g = geo(x, batch);
  long long n = g.npos * 16;
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
  k_loss<<<(unsigned)((g.npos + 255) / 256), 256, 0, x->s>>>(g, cpo, x->out, t, batch, nvalid,
                                                             x->dz[0], x->lossacc);
  int cur = 0;
  const unsigned nch = (unsigned)((g.npos + kWChunk - 1) / kWChunk);
  dim3 wg(nch, 9);
  dim3 cg((unsigned)((g.npos + kBM - 1) / kBM));
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
    if (co == 16 && ci == 64)
      k_conv<16, 64, 2><<<cg, 128, 0, x->s>>>(g, dzl, x->wb[l], nullptr, x->act[l], nx);
    else if (co == 64 && ci == 64)
      k_conv<64, 64, 2><<<cg, 128, 0, x->s>>>(g, dzl, x->wb[l], nullptr, x->act[l], nx);
    else
      return cudaErrorInvalidValue;
    cur ^= 1;
  }
  return cudaGetLastError();
}

int rc(cudaError_t e) { return e == cudaSuccess ? PIC_OK : PIC_E_CUDA; }

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
  x->geo1 = geo(x, 1);
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
  return rc(e);
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
  return rc(e);
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
  return rc(e);
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
int cnn_layers(const pic_cnn *x) { return x->M.L; }
int cnn_grid(const pic_cnn *x, int *nr, int *nz) {
  *nr = x->cfg.nr;
  *nz = x->cfg.nz;
  return PIC_OK;
}
}  // namespace pic
