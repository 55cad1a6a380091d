// Mover + deposit kernels of rows a2, a3 and a6 (Sec. 2.1, Eqs. 3-4) for a
// particle store of scalar type T (double: plain form, float: mixed form).
//
// Two phases, both in the normalised units of push_general.cuh:
//   1. k_push_fast: particles that stay inside their cell over the whole step
//      (the common case).  Without B_z the z-equation of the CN midpoint system
//      is linear in the r-displacement, so the system reduces to one scalar
//      equation g(d) = 0 for d = delta a, solved by Newton with an a-priori
//      error estimate (one iteration is usually enough).  The home-cell
//      deposits of a warp are summed with a transposed butterfly and added
//      with one FP64 atomic per edge and run of lanes with the same cell.
//      The kernel is persistent (one wave of resident blocks striding over
//      the store), which measured 20 % faster than one particle per thread.
//   2. k_push_general: the queued rest (crossings, particles on faces, near
//      the axis, no convergence) through the general sub-step path, starting
//      from the fast phase's converged whole-step trial where there is one.
#pragma once

#include "push_general.cuh"
#include "seg_queue.cuh"

namespace pic {
namespace {

// ---------------------------------------------------------------------------
// Warp sums of the home-cell deposits.  v0, v1: charge through the r-faces
// (i+1/2, j) and (i+1/2, j+1); v2, v3: through the z-faces (i, j+1/2) and
// (i+1, j+1/2) of the lane's cell `key` (ascending over the lanes, -1: none).

// lane l ends with the warp total of v[(l >> 3) & 3]
template <typename T>
__device__ __forceinline__ T bfly4(T v0, T v1, T v2, T v3, int lane) {
  const unsigned full = 0xffffffffu;
  const bool h16 = lane & 16, h8 = lane & 8;
  T k0 = h16 ? v2 : v0, k1 = h16 ? v3 : v1;
  T s0 = h16 ? v0 : v2, s1 = h16 ? v1 : v3;
  k0 += __shfl_xor_sync(full, s0, 16);
  k1 += __shfl_xor_sync(full, s1, 16);
  T k = h8 ? k1 : k0, s = h8 ? k0 : k1;
  k += __shfl_xor_sync(full, s, 8);
  k += __shfl_xor_sync(full, k, 4);
  k += __shfl_xor_sync(full, k, 2);
  k += __shfl_xor_sync(full, k, 1);
  return k;
}

// two runs (lanes below / from the second run's first lane): lane l ends with
// the total of run (l >> 4) of v[(l >> 2) & 3]
template <typename T>
__device__ __forceinline__ T bfly8(T v0, T v1, T v2, T v3, bool second, int lane) {
  const unsigned full = 0xffffffffu;
  const T z = (T)0;
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
  const bool keep = h16 == second;
  T k0 = keep ? v0 : z, k1 = keep ? v1 : z, k2 = keep ? v2 : z, k3 = keep ? v3 : z;
  T s0 = keep ? z : v0, s1 = keep ? z : v1, s2 = keep ? z : v2, s3 = keep ? z : v3;
  k0 += __shfl_xor_sync(full, s0, 16);
  k1 += __shfl_xor_sync(full, s1, 16);
  k2 += __shfl_xor_sync(full, s2, 16);
  k3 += __shfl_xor_sync(full, s3, 16);
  T m0 = h8 ? k2 : k0, m1 = h8 ? k3 : k1;
  T t0 = h8 ? k0 : k2, t1 = h8 ? k1 : k3;
  m0 += __shfl_xor_sync(full, t0, 8);
  m1 += __shfl_xor_sync(full, t1, 8);
  T k = h4 ? m1 : m0, s = h4 ? m0 : m1;
  k += __shfl_xor_sync(full, s, 4);
  k += __shfl_xor_sync(full, k, 2);
  k += __shfl_xor_sync(full, k, 1);
  return k;
}

// edge j of cell (ic, jc): 0, 1 = r-faces (ic, jc), (ic, jc+1) of the Er-layout;
// 2, 3 = z-faces (ic, jc), (ic+1, jc) of the Ez-layout
__device__ __forceinline__ double *edge_ptr(int ic, int jc, int j, int nz, double *ir, double *iz) {
  return j < 2 ? ir + ic * (nz + 1) + jc + j : iz + (ic + (j - 2)) * nz + jc;
}

// key: the lane's cell (ascending over the lanes, -1: none), (ic, jc) its
// indices
template <typename T>
__device__ __forceinline__ void warp_deposit(int key, int ic, int jc, T v0, T v1, T v2, T v3,
                                             int lane, int nz, double *ir, double *iz) {
  const unsigned full = 0xffffffffu;
  int prev = __shfl_up_sync(full, key, 1);
  unsigned heads = __ballot_sync(full, lane == 0 || prev != key);
  int nrun = __popc(heads);
  if (nrun == 1) {
    T t = bfly4(v0, v1, v2, v3, lane);
    if ((lane & 7) == 0 && key >= 0 && ir)
      atomicAdd(edge_ptr(ic, jc, (lane >> 3) & 3, nz, ir, iz), Num<T>::to_double(t));
  } else if (nrun == 2) {
    int first2 = __ffs(heads & ~1u) - 1;
    T t = bfly8(v0, v1, v2, v3, lane >= first2, lane);
    int src = (lane & 16) ? 31 : 0;
    int k = __shfl_sync(full, key, src);
    int ki = __shfl_sync(full, ic, src), kj = __shfl_sync(full, jc, src);
    if ((lane & 3) == 0 && k >= 0 && ir)
      atomicAdd(edge_ptr(ki, kj, (lane >> 2) & 3, nz, ir, iz), Num<T>::to_double(t));
  } else {
    // segmented inclusive scan; the last lane of each run adds the run's totals
    unsigned below = heads & ((2u << lane) - 1u);
    int seg_start = 31 - __clz(below);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T t0 = __shfl_up_sync(full, v0, o);
      T t1 = __shfl_up_sync(full, v1, o);
      T t2 = __shfl_up_sync(full, v2, o);
      T t3 = __shfl_up_sync(full, v3, o);
      if (lane - o >= seg_start) {
        v0 += t0; v1 += t1; v2 += t2; v3 += t3;
      }
    }
    int next = __shfl_down_sync(full, key, 1);
    if ((lane == 31 || next != key) && key >= 0 && ir) {
      atomicAdd(edge_ptr(ic, jc, 0, nz, ir, iz), Num<T>::to_double(v0));
      atomicAdd(edge_ptr(ic, jc, 1, nz, ir, iz), Num<T>::to_double(v1));
      atomicAdd(edge_ptr(ic, jc, 2, nz, ir, iz), Num<T>::to_double(v2));
      atomicAdd(edge_ptr(ic, jc, 3, nz, ir, iz), Num<T>::to_double(v3));
    }
  }
}

// ---------------------------------------------------------------------------
template <typename T>
struct PState {
  int c;
  T a, b, vr, vt, vz, w;
};

template <typename T>
__device__ __forceinline__ void load_state(const PartsT<T> &P, long long p, long long n,
                                           PState<T> &s) {
  if (p < n) {
    s.c = P.cell[p];
    s.a = P.a[p];
    s.b = P.b[p];
    s.vr = P.vr[p];
    s.vt = P.vt[p];
    s.vz = P.vz[p];
    s.w = P.w[p];
  } else {
    s.c = -1;
  }
}

// FP32 crossers that take FP64 arithmetic (the centrifugal term of Eq. 4
// grows like 1/r and amplifies FP32 rounding): in the first radial cells, a
// straight path over the step that comes closer to the axis than 1/8 of the
// start radius (the amplification grows like rho / rho_min), or a CN
// whole-step trial (d: its radial displacement, NaN: none) that ends that close
template <typename T>
__device__ __forceinline__ bool near_axis32(const PushLaunchT<T> &L, int c, T a, T vr, T vt, T d) {
  const int nz = L.g.nz;
  if (c < 0 || c >= kPromoteRows * nz) return false;
  const int ic = c / nz;
  const T crr = L.rm.crr(ic);
  const T rho = L.rm.rho0(ic) + a, ur = vr * crr, ut = vt * crr;
  const T u2 = ur * ur + ut * ut;
  bool close = false;
  if (ur < (T)0 && u2 > (T)0) {
    const T sm = fmin(-rho * ur / u2, (T)1);
    const T x = rho + ur * sm, y = ut * sm;
    close = (T)64 * (x * x + y * y) < rho * rho;
  }
  if (!Num<T>::nan_bits(d)) close = close || (T)64 * (rho + d) * (rho + d) < rho * rho;
  return close;
}

// the fast phase of block `bid` of a grid of `nblk` blocks (a launch of its
// own, or one work item of a launch over several discharges)
template <typename T>
__device__ __forceinline__ void push_fast_body(const PushLaunchT<T> &L, int bid, int nblk) {
  const int lane = threadIdx.x & 31;
  const int nz = L.g.nz, nz1 = nz + 1, ncell = L.g.nr * nz;
  const T zero = (T)0, one = (T)1, h = (T)0.5, q = (T)0.25;
  const long long stride = (long long)nblk * blockDim.x;
  unsigned n_newton = 0, n_acc = 0;
  // entries this block appended to its queue segment: [0] single z-face
  // crossings of the trial from the front, [1] the rest from the back
  __shared__ int s_qn[2];
  if (threadIdx.x < 2) s_qn[threadIdx.x] = 0;
  // the near-axis list of this pass starts empty (the general kernel, which
  // fills it, runs after this kernel on the same stream)
  if (L.pcnt && bid == 0 && threadIdx.x == 0) *L.pcnt = 0u;
  __syncthreads();
  const long long qoff = (long long)bid * L.qseg;
  const long long n = L.n_dev ? *L.n_dev : L.n;
  long long base = (long long)bid * blockDim.x;
  // FP32 form: the next tile's state is loaded while this one is pushed (the
  // kernel is issue-bound; the FP64 form is bound by its FP64 pipe instead)
  constexpr bool kPrefetch = sizeof(T) == 4;
  PState<T> nxt;
  if (kPrefetch) load_state(L.p, base + threadIdx.x, n, nxt);
  for (; base < n; base += stride) {
    const long long p = base + threadIdx.x;
    PState<T> cur;
    if (kPrefetch) {
      cur = nxt;
      load_state(L.p, base + stride + threadIdx.x, n, nxt);
    } else {
      load_state(L.p, p, n, cur);
    }
    const int c0 = cur.c;
    const T a = cur.a, b = cur.b, w = cur.w;
    T ur = zero, ut = zero, uz = zero;
    T v0 = zero, v1 = zero, v2 = zero, v3 = zero;
    bool queued = false, trial = false, zcross = false;
    T d = zero, e = zero;
    int key = -1, ic = 0, jc = 0;
    if (c0 >= 0 && c0 < ncell) {
      key = c0;
      // cell -> (ic, jc) without an integer division (c0 < 2^24 is exact in FP32)
      ic = __float2int_rz(__int2float_rn(c0) * L.inz);
      jc = c0 - ic * nz;
      if (jc < 0) { ic -= 1; jc += nz; }
      else if (jc >= nz) { ic += 1; jc -= nz; }
      // products that feed no addition go through Num<T>::mul (the FP64 form
      // computes them on the integer pipes)
      typedef Num<T> N;
      const T crr = L.rm.crr(ic);
      ur = N::mul(cur.vr, crr);
      ut = N::mul(cur.vt, crr);
      uz = N::mul(cur.vz, L.cz);
      const T rho = L.rm.rho0(ic) + a;
      bool acc = false;
      if (N::in01(a) && N::in01(b) && N::lt_abs(ut, N::mul(q, rho))) {
        const T ar0 = L.ar[ic * nz1 + jc];
        const T gar = L.ar[ic * nz1 + jc + 1] - ar0;
        const T az0 = L.az[ic * nz + jc];
        const T gaz = L.az[(ic + 1) * nz + jc] - az0;
        const T zb = uz + h * (az0 + gaz * a);
        const T K = ur + h * (ar0 + gar * b) + N::mul(q, gar) * zb;
        const T k1 = one - N::mul((T)0.0625, gar) * gaz;
        if (Num<T>::gt(k1, h) && fast_solve<T>(rho, ut, K, k1, d, n_newton)) {
          trial = true;
          e = zb + N::mul(q, gaz) * d;
          const T a1 = a + d, b1 = b + e;
          acc = Num<T>::in01(a1) && Num<T>::in01(b1);
          // FP32: an end much closer to the axis than the start is queued (it
          // may need FP64: the centrifugal term grows like 1/r)
          if (sizeof(T) == 4 && acc && ic < kPromoteRows)
            acc = !((T)64 * (rho + d) * (rho + d) < rho * rho);
          // the trial crosses one z-face (two or more: the loop)
          zcross = Num<T>::in01(a1) && ((b1 < zero && b1 > -one) || (b1 > one && b1 < (T)2));
          if (acc) {
            n_acc++;
            const T qw = N::mul(L.qf, w);
            const T fr = N::mul(qw, d), fz = N::mul(qw, e);
            const T am = a + h * d, bm = b + h * e;
            v1 = N::mul(fr, bm);
            v0 = fr - v1;
            v3 = N::mul(fz, am);
            v2 = fz - v3;
            if (L.write) {
              // CN velocity relations: the displacement is the mean of u and u'
              L.dst.a[p] = a1;
              L.dst.b[p] = b1;
              const T icr = L.rm.icrr(ic);
              L.dst.vr[p] = N::mul((T)2 * d - ur, icr);
              L.dst.vz[p] = N::mul((T)2 * e - uz, L.icz);
              L.dst.vt[p] = N::mul(N::mul(N::mul(rho, ut), N::rcp(rho + d)), icr);
              if (L.oop) {
                L.dst.cell[p] = c0;
                L.dst.w[p] = w;
                L.dst.id[p] = L.p.id[p];
              }
            }
          }
        }
      }
      queued = !acc;
    } else if (L.write && L.oop && p < n) {
      L.dst.cell[p] = c0;  // not pushed (absorbed earlier): stays out of the store
    }
    warp_deposit<T>(key, ic, jc, v0, v1, v2, v3, lane, nz, L.ir, L.iz);
    if (L.hist) {  // in-cell pushes: one sub-step (bin 0), one count per warp
      const unsigned m = __ballot_sync(0xffffffffu, key >= 0 && !queued);
      if (lane == 0 && m) atomicAdd(&L.hist[0], (unsigned long long)__popc(m));
    }
    // queue the rest for the general path (warp-aggregated append to the
    // block's segment; the shared-memory counter keeps it off global atomics),
    // in two kinds: the crossings of the trial through one z-face only from the
    // front, the rest from the back, so that the general kernel's warps take
    // one sub-step sequence at a time.  FP32 entries carry the start state
    // (written coalesced here, read coalesced there: no scattered re-read)
    const bool front = zcross && trial;
    const long long kf = seg_append(&s_qn[0], queued && front, lane, qoff);
    const long long kb = seg_append(&s_qn[1], queued && !front, lane, 0);
    const long long k = front ? kf : qoff + L.qseg - 1 - kb;
    if (queued) {
      L.queue[k] = (int)p;
      L.q_da[k] = trial ? d : (T)NAN;
      L.q_db[k] = e;
      if (L.q_cell) {
        L.q_cell[k] = c0;
        L.q_a[k] = a;
        L.q_b[k] = b;
        L.q_vr[k] = cur.vr;
        L.q_vt[k] = cur.vt;
        L.q_vz[k] = cur.vz;
        L.q_w[k] = w;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    L.qblock[bid] = s_qn[0];
    L.qblock[L.qgrid + bid] = s_qn[1];
  }
  Tally T0 = {0, 0, 0, 0, 0, 0, 0};
  flush_tally(L.counters, T0, lane, n_newton, n_acc);
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 3) k_push_fast(PushLaunchT<T> L) {
  push_fast_body<T>(L, blockIdx.x, gridDim.x);
}

// queued particles (or all of them when queue == nullptr) of block `bid` of
// `nblk`; blockDim 256
template <typename T, bool kB>
__device__ __forceinline__ void push_general_body(const PushLaunchT<T> &L, int bid, int nblk) {
  const int lane = threadIdx.x & 31;
  GenArgs<T> G;
  G.nr = L.g.nr; G.nz = L.g.nz; G.ar = L.ar; G.az = L.az;
  G.wt = L.wbt; G.icr = L.icr; G.icz = L.icz; G.cz = L.cz; G.rm = L.rm;
  G.q = L.q; G.m = L.m; G.qf = L.qf; G.ir = L.ir; G.iz = L.iz; G.write = L.write; G.p = L.p;
  G.oop = L.oop; G.dst = L.dst; G.hist = L.hist;
  G.wall_z0 = L.wall_z0; G.wall_zl = L.wall_zl; G.wall_r = L.wall_r; G.ke_lost = L.ke_lost;
  Tally tl = {0, 0, 0, 0, 0, 0, 0};
  const long long gstride = (long long)nblk * blockDim.x;
  const long long gtid = (long long)bid * blockDim.x + threadIdx.x;
  if (L.queue) {
    // the single z-face crossings first, then the rest (uniform warps)
    __shared__ int s_pre[kMaxFastBlocks + 1], s_preb[kMaxFastBlocks + 1];
    const int total_f = seg_prefix(L.qblock, L.qgrid, s_pre);
    const int total = total_f + seg_prefix(L.qblock + L.qgrid, L.qgrid, s_preb);
    auto entry = [&](long long q) {
      return q < total_f ? seg_entry(s_pre, L.qgrid, L.qseg, (int)q)
                         : seg_entry_back(s_preb, L.qgrid, L.qseg, (int)(q - total_f));
    };
    if (sizeof(T) == 4) {
      // FP32 form: the entries carry the start state; the next entry is loaded
      // while this one is pushed.  z-face crossers (the front kind) take the
      // straight-line routine; crossers next to the axis go to the FP64 list
      struct Ent {
        long long p;
        PState<T> s;
        T da, db;
      };
      auto fetch = [&](long long q, Ent &en) {
        const long long k = entry(q);
        en.p = L.queue[k];
        en.da = L.q_da[k];
        en.db = L.q_db[k];
        en.s.c = L.q_cell[k];
        en.s.a = L.q_a[k];
        en.s.b = L.q_b[k];
        en.s.vr = L.q_vr[k];
        en.s.vt = L.q_vt[k];
        en.s.vz = L.q_vz[k];
        en.s.w = L.q_w[k];
      };
      Ent nx;
      if (gtid < total) fetch(gtid, nx);
      for (long long q = gtid; q < total; q += gstride) {
        const Ent cu = nx;
        if (q + gstride < total) fetch(q + gstride, nx);
        if (L.pcnt && near_axis32(L, cu.s.c, cu.s.a, cu.s.vr, cu.s.vt, cu.da)) {
          const unsigned am = __activemask();
          const unsigned pm = __ballot_sync(am, true);
          const int leader = __ffs(pm) - 1;
          unsigned base = 0;
          if (lane == leader) base = atomicAdd(L.pcnt, (unsigned)__popc(pm));
          base = __shfl_sync(pm, base, leader);
          L.plist[base + __popc(pm & ((1u << lane) - 1u))] = (int)cu.p;
        } else if (!kB && q < total_f) {
          push_zcross<T>(G, cu.p, cu.s.c, cu.s.a, cu.s.b, cu.s.vr, cu.s.vt, cu.s.vz, cu.s.w,
                         cu.da, cu.db, tl);
        } else {
          push_general<T, kB>(G, cu.p, cu.s.c, cu.s.a, cu.s.b, cu.s.vr, cu.s.vt, cu.s.vz,
                              cu.s.w, cu.da, cu.db, tl);
        }
      }
    } else {
      // FP64 form: the start state from the store; z-face crossers (the front
      // kind) through the straight-line routine as well
      for (long long q = gtid; q < total; q += gstride) {
        long long k = entry(q);
        long long p = L.queue[k];
        if (!kB && q < total_f)
          push_zcross<T>(G, p, L.p.cell[p], L.p.a[p], L.p.b[p], L.p.vr[p], L.p.vt[p],
                         L.p.vz[p], L.p.w[p], L.q_da[k], L.q_db[k], tl);
        else
          push_general<T, kB>(G, p, L.p.cell[p], L.p.a[p], L.p.b[p], L.p.vr[p], L.p.vt[p],
                              L.p.vz[p], L.p.w[p], L.q_da[k], L.q_db[k], tl);
      }
    }
  } else {
    const long long n = L.n_dev ? *L.n_dev : L.n;
    for (long long k = gtid; k < n; k += gstride) {
      push_general<T, kB>(G, k, L.p.cell[k], L.p.a[k], L.p.b[k], L.p.vr[k], L.p.vt[k],
                          L.p.vz[k], L.p.w[k], (T)NAN, (T)NAN, tl);
    }
  }
  flush_tally(L.counters, tl, lane, 0, 0);
}

template <typename T, bool kB>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_push_general(PushLaunchT<T> L) {
  push_general_body<T, kB>(L, blockIdx.x, gridDim.x);
}

// One launch over several discharges (an ensemble's Picard round): work item
// k of first[nl] is virtual block k - first[j] of launch j, first[j] <= k <
// first[j + 1], whose grid is first[j + 1] - first[j] blocks.  The launch's
// parameters are copied into shared memory once per item.
template <typename T>
__device__ __forceinline__ const PushLaunchT<T> &multi_item(const PushLaunchT<T> *Ls,
                                                            const int *first, int nl, int k,
                                                            int &vb, int &vg) {
  __shared__ __align__(16) int s_launch[sizeof(PushLaunchT<T>) / 4];
  __shared__ int s_j;
  static_assert(sizeof(PushLaunchT<T>) % 4 == 0, "launch parameters in 4-byte words");
  __syncthreads();  // the previous item is done with s_launch
  if (threadIdx.x == 0) {
    int j = 0;
    while (j + 1 < nl && first[j + 1] <= k) ++j;
    s_j = j;
  }
  __syncthreads();
  const int j = s_j;
  const int *src = reinterpret_cast<const int *>(Ls + j);
  for (int i = threadIdx.x; i < (int)(sizeof(PushLaunchT<T>) / 4); i += blockDim.x)
    s_launch[i] = src[i];
  vb = k - first[j];
  vg = first[j + 1] - first[j];
  __syncthreads();
  return *reinterpret_cast<const PushLaunchT<T> *>(s_launch);
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 3)
    k_push_fast_multi(const PushLaunchT<T> *Ls, const int *first, int nl) {
  const int total = first[nl];
  for (int k = blockIdx.x; k < total; k += gridDim.x) {
    int vb, vg;
    const PushLaunchT<T> &L = multi_item<T>(Ls, first, nl, k, vb, vg);
    push_fast_body<T>(L, vb, vg);
  }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2)
    k_push_general_multi(const PushLaunchT<T> *Ls, const int *first, int nl) {
  const int total = first[nl];
  for (int k = blockIdx.x; k < total; k += gridDim.x) {
    int vb, vg;
    const PushLaunchT<T> &L = multi_item<T>(Ls, first, nl, k, vb, vg);
    push_general_body<T, false>(L, vb, vg);
  }
}

// grids of the persistent kernels (one wave of resident blocks)
template <typename T>
long long fast_grid() {
  static int nb = 0;
  if (nb == 0) nb = persistent_grid(k_push_fast<T>);
  return nb;
}
template <typename T>
long long general_grid() {
  static int nb = 0;
  if (nb == 0) nb = persistent_grid(k_push_general<T, false>);
  return nb;
}

}  // namespace

// every particle through the general path (external B_z, or no queue)
template <typename T>
cudaError_t launch_push_all(const PushLaunchT<T> &L, cudaStream_t s) {
  const long long nsz = L.n_dev ? L.cap : L.n;
  if (nsz <= 0) return cudaSuccess;
  const int bs = 256;
  long long nb = (nsz + bs - 1) / bs;
  PushLaunchT<T> A = L;
  A.queue = nullptr;
  if (L.wbt == (T)0)
    k_push_general<T, false><<<(unsigned)nb, bs, 0, s>>>(A);
  else
    k_push_general<T, true><<<(unsigned)nb, bs, 0, s>>>(A);
  return cudaGetLastError();
}

// the virtual grids of one discharge's fast and general phases (as
// launch_push would launch them); L.qgrid and L.qseg are set
template <typename T>
void push_shape(PushLaunchT<T> &L, int *nfast, int *ngen) {
  const long long nsz = L.n_dev ? L.cap : L.n;
  const int bs = 256;
  long long nb = (nsz + bs - 1) / bs;
  if (nb < 1) nb = 1;
  long long nf = L.fgrid > 0 ? L.fgrid : fast_grid<T>();
  if (nf > kMaxFastBlocks) nf = kMaxFastBlocks;
  if (nf > nb) nf = nb;
  L.qgrid = (int)nf;
  L.qseg = (nb + nf - 1) / nf * bs;
  long long ng = L.ggrid > 0 ? L.ggrid : general_grid<T>();
  if (ng > nb) ng = nb;
  *nfast = (int)nf;
  *ngen = (int)ng;
}

// fast then general phase of nl discharges in two launches of one resident
// wave each; Ls and first (item offsets: fast [nl + 1], then general [nl + 1])
// in device memory
template <typename T>
cudaError_t launch_push_multi(const PushLaunchT<T> *Ls, const int *first, int nl,
                              cudaStream_t s) {
  k_push_fast_multi<T><<<(unsigned)fast_grid<T>(), 256, 0, s>>>(Ls, first, nl);
  k_push_general_multi<T><<<(unsigned)general_grid<T>(), 256, 0, s>>>(Ls, first + nl + 1, nl);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_push(const PushLaunchT<T> &L, cudaStream_t s) {
  // with the count on the device the grids depend only on the capacity, so a
  // captured launch stays valid while the count changes
  const long long nsz = L.n_dev ? L.cap : L.n;
  if (nsz <= 0) return cudaSuccess;

  const int bs = 256;
  long long nb = (nsz + bs - 1) / bs;
  if (L.wbt == (T)0 && L.queue) {
    long long nf = L.fgrid > 0 ? L.fgrid : fast_grid<T>();
    if (nf > kMaxFastBlocks) nf = kMaxFastBlocks;
    if (nf > nb) nf = nb;
    PushLaunchT<T> A = L;
    A.qgrid = (int)nf;
    A.qseg = (nb + nf - 1) / nf * bs;  // particles one fast block visits, at most
    k_push_fast<T><<<(unsigned)nf, bs, 0, s>>>(A);
    // the queue holds the crossing / near-axis particles (a fraction of n);
    // one wave, so the per-block prefix of the segment counts is computed once
    // per resident block
    long long ng = L.ggrid > 0 ? L.ggrid : general_grid<T>();
    if (ng > nb) ng = nb;
    k_push_general<T, false><<<(unsigned)ng, bs, 0, s>>>(A);
    return cudaGetLastError();
  }
  return launch_push_all<T>(L, s);
}

}  // namespace pic
