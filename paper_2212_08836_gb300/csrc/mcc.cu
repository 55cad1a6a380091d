// Row a7: null-collision Monte Carlo collisions (Sec. 2.1, after Mertmann et
// al. 2011 / Vahedi & Surendra 1995) with analytic argon-like cross sections.
// Electrons: elastic, excitation (11.5 eV), ionization (15.76 eV, equal
// split, new e + Ar+ pair at the parent's position and weight).  Ar+: charge
// exchange with a constant cross section against a 300 K neutral Maxwellian.
// One thread per particle; Philox4x64-10 with counter (id, step, block, 0), so
// the draws do not depend on the launch shape.  Ionizing electrons set a flag;
// an exclusive scan of the flags gives the append slot in parent order.
#include "pic_internal.cuh"

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

__device__ __forceinline__ unsigned long long wsum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double wsumd(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(256) k_mcc(MccLaunch M) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long c[7] = {0, 0, 0, 0, 0, 0, 0};
  double de = 0.0;
  if (t < M.ne) {
    long long p = t;
    int32_t flag = 0;
    if (M.e.cell[p] >= 0) {
      double u[4];
      draw4(M.seed, kStreamMccE, M.e.id[p], M.step, 0, u);
      if (u[0] < M.pnull_e) {
        c[0]++;
        double vr = M.e.vr[p], vt = M.e.vt[p], vz = M.e.vz[p];
        double v2 = vr * vr + vt * vt + vz * vz;
        double v = sqrt(v2);
        double eps = 0.5 * kME * v2 / kQE;
        double nu_el = M.ng * sig_el(eps) * v;
        double nu_ex = M.ng * sig_ex(eps) * v;
        double nu_iz = M.ng * sig_iz(eps) * v;
        double x = u[1] * M.numax_e;
        double w = M.e.w[p];
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
          flag = 1;
        } else {
          hit = false;
          v1 = 0.0;
        }
        if (hit) {
          double nvr = v1 * nr_, nvt = v1 * nt_, nvz = v1 * nz_;
          M.e.vr[p] = nvr;
          M.e.vt[p] = nvt;
          M.e.vz[p] = nvz;
          de += 0.5 * kME * w * (nvr * nvr + nvt * nvt + nvz * nvz) - ke0;
        }
      }
    }
    M.flag[p] = flag;
  }
  if (t < M.ni) {
    long long p = t;
    if (M.i.cell[p] >= 0) {
      double u[4];
      draw4(M.seed, kStreamMccI, M.i.id[p], M.step, 0, u);
      if (u[0] < M.pnull_i) {
        c[4]++;
        double u1[4];
        draw4(M.seed, kStreamMccI, M.i.id[p], M.step, 1, u1);
        double g1, g2, g3, g4;
        gauss2(u[2], u[3], g1, g2);
        gauss2(u1[0], u1[1], g3, g4);
        double vthg = sqrt(kKB * M.tg / kMAr);
        double wr = vthg * g1, wt = vthg * g2, wz = vthg * g3;
        double vr = M.i.vr[p], vt = M.i.vt[p], vz = M.i.vz[p];
        double dr_ = vr - wr, dt_ = vt - wt, dz_ = vz - wz;
        double g = sqrt(dr_ * dr_ + dt_ * dt_ + dz_ * dz_);
        if (g > M.gmax) c[6]++;
        if (u[1] * M.gmax < g) {
          double w = M.i.w[p];
          double ke0 = 0.5 * kMAr * w * (vr * vr + vt * vt + vz * vz);
          M.i.vr[p] = wr;
          M.i.vt[p] = wt;
          M.i.vz[p] = wz;
          de += 0.5 * kMAr * w * (wr * wr + wt * wt + wz * wz) - ke0;
          c[5]++;
        }
      }
    }
  }
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    unsigned long long s = wsum(c[k]);
    if (lane == 0 && s) atomicAdd(&M.cnt->mcc[k], s);
  }
  de = wsumd(de);
  if (lane == 0 && de != 0.0) atomicAdd(&M.cnt->de_coll, de);
}

// new pairs for flagged electrons: electron at ne_new0 + k, ion at ni_new0 + k
__global__ void __launch_bounds__(256) k_append(MccLaunch M, long long ne0, long long ni0,
                                                uint32_t id_e0, uint32_t id_i0) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double de = 0.0;
  if (p < M.ne && M.flag[p]) {
    long long k = M.offs[p];
    double u1[4], u2[4];
    draw4(M.seed, kStreamMccE, M.e.id[p], M.step, 1, u1);
    draw4(M.seed, kStreamMccE, M.e.id[p], M.step, 2, u2);
    double vr = M.e.vr[p], vt = M.e.vt[p], vz = M.e.vz[p];
    double v1 = sqrt(vr * vr + vt * vt + vz * vz);  // the parent's share: equal split
    double mr, mt, mz;
    iso_dir(u1[0], u1[1], mr, mt, mz);
    long long q = ne0 + k;
    int32_t cell = M.e.cell[p];
    double a = M.e.a[p], b = M.e.b[p], w = M.e.w[p];
    M.e.cell[q] = cell; M.e.a[q] = a; M.e.b[q] = b; M.e.w[q] = w;
    M.e.vr[q] = v1 * mr; M.e.vt[q] = v1 * mt; M.e.vz[q] = v1 * mz;
    M.e.id[q] = id_e0 + (uint32_t)k;
    double g1, g2, g3, g4;
    gauss2(u1[2], u1[3], g1, g2);
    gauss2(u2[0], u2[1], g3, g4);
    double vthg = sqrt(kKB * M.tg / kMAr);
    long long s = ni0 + k;
    M.i.cell[s] = cell; M.i.a[s] = a; M.i.b[s] = b; M.i.w[s] = w;
    double ir = vthg * g1, it = vthg * g2, iz = vthg * g3;
    M.i.vr[s] = ir; M.i.vt[s] = it; M.i.vz[s] = iz;
    M.i.id[s] = id_i0 + (uint32_t)k;
    de = 0.5 * kME * w * (v1 * v1) + 0.5 * kMAr * w * (ir * ir + it * it + iz * iz);
  }
  de = wsumd(de);
  if ((threadIdx.x & 31) == 0 && de != 0.0) atomicAdd(&M.cnt->de_coll, de);
}

}  // namespace

cudaError_t launch_mcc_collide(const MccLaunch &M, cudaStream_t s) {
  long long n = M.ne > M.ni ? M.ne : M.ni;
  if (n <= 0) return cudaSuccess;
  k_mcc<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(M);
  return cudaGetLastError();
}

cudaError_t launch_mcc_append(const MccLaunch &M, long long ne0, long long ni0, uint32_t id_e0,
                              uint32_t id_i0, cudaStream_t s) {
  if (M.ne <= 0) return cudaSuccess;
  k_append<<<(unsigned)((M.ne + 255) / 256), 256, 0, s>>>(M, ne0, ni0, id_e0, id_i0);
  return cudaGetLastError();
}

}  // namespace pic
