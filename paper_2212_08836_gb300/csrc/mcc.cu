// Row a7: null-collision Monte Carlo collisions (Sec. 2.1, after Mertmann et
// al. 2011 / Vahedi & Surendra 1995) with analytic argon-like cross sections.
// Electrons: elastic, excitation (11.5 eV), ionization (15.76 eV, equal
// split, new e + Ar+ pair at the parent's position and weight).  Ar+: charge
// exchange with a constant cross section against a 300 K neutral Maxwellian.
// Philox4x64-10 with counter (id, step, block, 0), so the draws do not depend
// on the launch shape.  Two kernels: k_mcc_select tests every particle against
// the null-collision probability with integers only and lists the candidates
// (a few per cent); k_mcc_collide runs the FP64 collision physics on the
// packed list, so the narrow FP64 pipe is not spent on idle lanes of warps
// with one candidate.  The ionizing parents are ordered by their id and the
// new pairs appended in that order, so the ids they receive do not depend on
// how the store happens to be ordered inside a cell.
#include "seg_queue.cuh"

namespace pic {
namespace {

__device__ __forceinline__ double sig_el(double eps) {
  double x = eps / 12.0;
  return 1.5e-19 * x / (1.0 + x * x) + 1e-20;
}
__device__ __forceinline__ double sig_ex(double eps) {
  if (!(eps > 11.5)) return 0.0;
  double u = eps / 11.5;
  return 4e-20 * log(u) / u;
}
__device__ __forceinline__ double sig_iz(double eps) {
  if (!(eps > 15.76)) return 0.0;
  double u = eps / 15.76;
  return 8e-20 * log(u) / u;
}

__device__ __forceinline__ void iso_dir(double u2, double u3, double &nr, double &nt, double &nz) {
  double ct = 1.0 - 2.0 * u2;
  double st = sqrt(fmax(0.0, 1.0 - ct * ct));
  double ph = kTwoPi * u3;
  nr = st * cos(ph);
  nt = st * sin(ph);
  nz = ct;
}

__device__ __forceinline__ double wsumd(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// phase 1: candidates of both species, integer test on the first Philox word
template <typename T>
__global__ void __launch_bounds__(256) k_mcc_select(MccLaunchT<T> M) {
  __shared__ int s_cnt;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long off = (long long)blockIdx.x * M.cseg;
  const long long n = M.ne > M.ni ? M.ne : M.ni;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += stride) {
    const long long p = base + threadIdx.x;
    bool ce = false, ci = false;
    if (p < M.ne && M.e.cell[p] >= 0) {
      uint64_t c4[4] = {(uint64_t)M.e.id[p], M.step, 0, 0};
      philox4x64(c4, M.seed, kStreamMccE);
      ce = (c4[0] >> 11) < M.thr_e;
    }
    if (p < M.ni && M.i.cell[p] >= 0) {
      uint64_t c4[4] = {(uint64_t)M.i.id[p], M.step, 0, 0};
      philox4x64(c4, M.seed, kStreamMccI);
      ci = (c4[0] >> 11) < M.thr_i;
    }
    long long k = seg_append(&s_cnt, ce, lane, off);
    if (ce) M.cand[k] = (uint32_t)p;
    k = seg_append(&s_cnt, ci, lane, off);
    if (ci) M.cand[k] = (uint32_t)p | 0x80000000u;
  }
  __syncthreads();
  if (threadIdx.x == 0) M.cblock[blockIdx.x] = s_cnt;
}

// phase 2: the collisions of the listed candidates
template <typename T>
__global__ void __launch_bounds__(256) k_mcc_collide(MccLaunchT<T> M) {
  __shared__ int s_pre[kMaxFastBlocks + 1];
  const int total = seg_prefix(M.cblock, M.cgrid, s_pre);
  unsigned c[7] = {0, 0, 0, 0, 0, 0, 0};
  double de = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
    const uint32_t code = M.cand[seg_entry(s_pre, M.cgrid, M.cseg, (int)q)];
    const long long p = (long long)(code & 0x7fffffffu);
    if (!(code >> 31)) {
      uint64_t c4[4] = {(uint64_t)M.e.id[p], M.step, 0, 0};
      philox4x64(c4, M.seed, kStreamMccE);
      double u[4] = {u01(c4[0]), u01(c4[1]), u01(c4[2]), u01(c4[3])};
      c[0]++;
      double vr = (double)M.e.vr[p], vt = (double)M.e.vt[p], vz = (double)M.e.vz[p];
      double v2 = vr * vr + vt * vt + vz * vz;
      double v = sqrt(v2);
      double eps = 0.5 * kME * v2 / kQE;
      double nu_el = M.ng * sig_el(eps) * v;
      double nu_ex = M.ng * sig_ex(eps) * v;
      double nu_iz = M.ng * sig_iz(eps) * v;
      double x = u[1] * M.numax_e;
      double w = (double)M.e.w[p];
      double ke0 = 0.5 * kME * w * v2;
      bool hit = true;
      double nr_, nt_, nz_, v1;
      iso_dir(u[2], u[3], nr_, nt_, nz_);
      if (x < nu_el) {
        double cchi = v > 0.0 ? (nr_ * vr + nt_ * vt + nz_ * vz) / v : 1.0;
        double eps1 = eps * (1.0 - 2.0 * (kME / kMAr) * (1.0 - cchi));
        v1 = sqrt(2.0 * eps1 * kQE / kME);
        c[1]++;
      } else if (x < nu_el + nu_ex) {
        double eps1 = eps - 11.5;
        v1 = sqrt(2.0 * eps1 * kQE / kME);
        c[2]++;
      } else if (x < nu_el + nu_ex + nu_iz) {
        double eps1 = 0.5 * (eps - 15.76);
        v1 = sqrt(2.0 * eps1 * kQE / kME);
        c[3]++;
        unsigned long long slot = atomicAdd(&M.cnt->iz_slots, 1ull);
        M.keys[slot] = ((uint64_t)M.e.id[p] << 32) | (uint64_t)(uint32_t)p;
      } else {
        hit = false;
        v1 = 0.0;
      }
      if (hit) {
        T nvr = (T)(v1 * nr_), nvt = (T)(v1 * nt_), nvz = (T)(v1 * nz_);
        M.e.vr[p] = nvr;
        M.e.vt[p] = nvt;
        M.e.vz[p] = nvz;
        double r2 = (double)nvr * (double)nvr + (double)nvt * (double)nvt + (double)nvz * (double)nvz;
        de += 0.5 * kME * w * r2 - ke0;
      }
    } else {
      uint64_t c4[4] = {(uint64_t)M.i.id[p], M.step, 0, 0};
      philox4x64(c4, M.seed, kStreamMccI);
      double u[4] = {u01(c4[0]), u01(c4[1]), u01(c4[2]), u01(c4[3])};
      c[4]++;
      double u1[4];
      draw4(M.seed, kStreamMccI, M.i.id[p], M.step, 1, u1);
      double g1, g2, g3, g4;
      gauss2(u[2], u[3], g1, g2);
      gauss2(u1[0], u1[1], g3, g4);
      double vthg = sqrt(kKB * M.tg / kMAr);
      double wr = vthg * g1, wt = vthg * g2, wz = vthg * g3;
      double vr = (double)M.i.vr[p], vt = (double)M.i.vt[p], vz = (double)M.i.vz[p];
      double dr_ = vr - wr, dt_ = vt - wt, dz_ = vz - wz;
      double g = sqrt(dr_ * dr_ + dt_ * dt_ + dz_ * dz_);
      if (g > M.gmax) c[6]++;
      if (u[1] * M.gmax < g) {
        double w = (double)M.i.w[p];
        double ke0 = 0.5 * kMAr * w * (vr * vr + vt * vt + vz * vz);
        T nr = (T)wr, nt = (T)wt, nz = (T)wz;
        M.i.vr[p] = nr;
        M.i.vt[p] = nt;
        M.i.vz[p] = nz;
        double r2 = (double)nr * (double)nr + (double)nt * (double)nt + (double)nz * (double)nz;
        de += 0.5 * kMAr * w * r2 - ke0;
        c[5]++;
      }
    }
  }
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    unsigned s = __reduce_add_sync(0xffffffffu, c[k]);
    if (lane == 0 && s) atomicAdd(&M.cnt->mcc[k], (unsigned long long)s);
  }
  de = wsumd(de);
  if (lane == 0 && de != 0.0) atomicAdd(&M.cnt->de_coll, de);
}

// one-block bitonic sort of up to kSortMax keys (padded with all-ones)
constexpr int kSortMax = 4096;
__global__ void __launch_bounds__(1024) k_sort_keys_block(uint64_t *keys, int n) {
  __shared__ uint64_t sk[kSortMax];
  int m = 1;
  while (m < n) m <<= 1;
  for (int i = threadIdx.x; i < m; i += blockDim.x) sk[i] = i < n ? keys[i] : ~0ull;
  __syncthreads();
  for (int k = 2; k <= m; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        int l = i ^ j;
        if (l > i) {
          bool up = (i & k) == 0;
          uint64_t x = sk[i], y = sk[l];
          if ((x > y) == up) {
            sk[i] = y;
            sk[l] = x;
          }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < n; i += blockDim.x) keys[i] = sk[i];
}

// large counts: rank of every key by counting smaller keys (keys are unique)
__global__ void __launch_bounds__(256) k_sort_keys_rank(const uint64_t *keys, uint64_t *out,
                                                        long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    uint64_t x = keys[i];
    long long r = 0;
    for (long long j = 0; j < n; ++j) r += keys[j] < x ? 1 : 0;
    out[r] = x;
  }
}

// pair k (in order of the parent's id): electron at ne0 + k, ion at ni0 + k
template <typename T>
__global__ void __launch_bounds__(256) k_append(MccLaunchT<T> M, const uint64_t *keys,
                                                long long tot, long long ne0, long long ni0,
                                                uint32_t id_e0, uint32_t id_i0) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double de = 0.0;
  if (k < tot) {
    long long p = (long long)(uint32_t)(keys[k] & 0xffffffffull);
    double u1[4], u2[4];
    draw4(M.seed, kStreamMccE, M.e.id[p], M.step, 1, u1);
    draw4(M.seed, kStreamMccE, M.e.id[p], M.step, 2, u2);
    double vr = (double)M.e.vr[p], vt = (double)M.e.vt[p], vz = (double)M.e.vz[p];
    double v1 = sqrt(vr * vr + vt * vt + vz * vz);  // the parent's share: equal split
    double mr, mt, mz;
    iso_dir(u1[0], u1[1], mr, mt, mz);
    long long q = ne0 + k;
    int32_t cell = M.e.cell[p];
    T a = M.e.a[p], b = M.e.b[p], w = M.e.w[p];
    M.e.cell[q] = cell; M.e.a[q] = a; M.e.b[q] = b; M.e.w[q] = w;
    T er = (T)(v1 * mr), et = (T)(v1 * mt), ez = (T)(v1 * mz);
    M.e.vr[q] = er; M.e.vt[q] = et; M.e.vz[q] = ez;
    M.e.id[q] = id_e0 + (uint32_t)k;
    double g1, g2, g3, g4;
    gauss2(u1[2], u1[3], g1, g2);
    gauss2(u2[0], u2[1], g3, g4);
    double vthg = sqrt(kKB * M.tg / kMAr);
    long long s = ni0 + k;
    M.i.cell[s] = cell; M.i.a[s] = a; M.i.b[s] = b; M.i.w[s] = w;
    T ir = (T)(vthg * g1), it = (T)(vthg * g2), iz = (T)(vthg * g3);
    M.i.vr[s] = ir; M.i.vt[s] = it; M.i.vz[s] = iz;
    M.i.id[s] = id_i0 + (uint32_t)k;
    double wd = (double)w;
    double e2 = (double)er * (double)er + (double)et * (double)et + (double)ez * (double)ez;
    double i2 = (double)ir * (double)ir + (double)it * (double)it + (double)iz * (double)iz;
    de = 0.5 * kME * wd * e2 + 0.5 * kMAr * wd * i2;
  }
  de = wsumd(de);
  if ((threadIdx.x & 31) == 0 && de != 0.0) atomicAdd(&M.cnt->de_coll, de);
}

}  // namespace

namespace {
template <typename T>
int select_grid() {
  static int nb = 0;
  if (nb == 0) nb = persistent_grid(k_mcc_select<T>);
  return nb;
}
}  // namespace

template <typename T>
cudaError_t launch_mcc_collide(const MccLaunchT<T> &M, cudaStream_t s) {
  long long n = M.ne > M.ni ? M.ne : M.ni;
  if (n <= 0) return cudaSuccess;
  long long nb = (n + 255) / 256;
  long long g = select_grid<T>();
  if (g > nb) g = nb;
  MccLaunchT<T> A = M;
  A.cgrid = (int)g;
  A.cseg = 2 * ((nb + g - 1) / g) * 256;  // two species per visited slot, at most
  k_mcc_select<T><<<(unsigned)g, 256, 0, s>>>(A);
  // the candidates are a few per cent of the particles
  k_mcc_collide<T><<<(unsigned)(nb < 152 * 4 ? nb : 152 * 4), 256, 0, s>>>(A);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mcc_append(const MccLaunchT<T> &M, long long tot, long long ne0,
                              long long ni0, uint32_t id_e0, uint32_t id_i0, cudaStream_t s) {
  if (tot <= 0 || M.ne <= 0) return cudaSuccess;
  const uint64_t *sorted = M.keys;
  if (tot <= kSortMax) {
    k_sort_keys_block<<<1, 1024, 0, s>>>(M.keys, (int)tot);
  } else {
    long long nb = (tot + 255) / 256;
    k_sort_keys_rank<<<(unsigned)(nb < 152 * 8 ? nb : 152 * 8), 256, 0, s>>>(M.keys, M.keys2, tot);
    sorted = M.keys2;
  }
  k_append<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(M, sorted, tot, ne0, ni0, id_e0, id_i0);
  return cudaGetLastError();
}

template cudaError_t launch_mcc_collide<double>(const MccLaunchT<double> &, cudaStream_t);
template cudaError_t launch_mcc_collide<float>(const MccLaunchT<float> &, cudaStream_t);
template cudaError_t launch_mcc_append<double>(const MccLaunchT<double> &, long long, long long,
                                               long long, uint32_t, uint32_t, cudaStream_t);
template cudaError_t launch_mcc_append<float>(const MccLaunchT<float> &, long long, long long,
                                              long long, uint32_t, uint32_t, cudaStream_t);

}  // namespace pic
