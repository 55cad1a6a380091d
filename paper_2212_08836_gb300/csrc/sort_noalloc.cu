// Allocation-free variant of the counting sort by cell.
//
// Some callers cannot hand this library a device workspace: a host code that
// reserves all device memory once at start-up and forbids any allocation
// afterwards, or a plugin that only receives the particle arrays across its
// interface.  pic_sort_cells_noalloc serves them: the caller passes only the
// input and output particle arrays, and the sort's scratch (per-cell counts,
// offsets, cursors and the scan's tile sums) lives in one file-scope device
// array of fixed size that every GPU loading this library keeps until the
// process exits.
#include <mutex>

#include "pic_internal.cuh"

namespace pic {
namespace {

// largest grid the static scratch can sort: nr * nz <= kNoallocMaxCells
constexpr long long kNoallocMaxCells = 1 << 18;
constexpr size_t kAlignUp(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kCountsBytes = kAlignUp((kNoallocMaxCells + 1) * sizeof(int32_t));
constexpr size_t kCursorBytes = kAlignUp(kNoallocMaxCells * sizeof(int32_t));
constexpr size_t kTotalBytes = 256;
constexpr size_t kScanBytes =
    kAlignUp(((kNoallocMaxCells + 1 + kScanTile - 1) / kScanTile + 1) * sizeof(long long));
constexpr size_t kScratchBytes = 2 * kCountsBytes + kCursorBytes + kTotalBytes + kScanBytes;

// the scratch: shared by every call on a device, contents persist between calls
static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices];

// device address of the scratch on the current device (set up once per
// device; a context destroyed by cudaDeviceReset reloads the module, so the
// cached address is not valid across a reset)
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace pic

using namespace pic;

extern "C" int pic_sort_cells_noalloc(int nr, int nz, long long n, const int32_t *cell,
                                      const double *a, const double *b, const double *vr,
                                      const double *vt, const double *vz, const double *w,
                                      const uint32_t *id, int32_t *cell_out, double *a_out,
                                      double *b_out, double *vr_out, double *vt_out,
                                      double *vz_out, double *w_out, uint32_t *id_out,
                                      void *stream, long long *n_out) {
  if (nr < 1 || nz < 1 || n < 0 || !n_out) return PIC_E_CONFIG;
  if ((long long)nr * nz > kNoallocMaxCells) return PIC_E_CONFIG;
  // the scan's tile sums must fit the part of the array set aside for them
  if (scan_scratch_bytes((long long)nr * nz + 1) > kScanBytes) return PIC_E_CONFIG;
  if (n > 0x7FFFFFFFll) return PIC_E_CONFIG;
  if (n > 0 && (!cell || !a || !b || !vr || !vt || !vz || !w || !id || !cell_out || !a_out ||
                !b_out || !vr_out || !vt_out || !vz_out || !w_out || !id_out))
    return PIC_E_CONFIG;
  void *base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return PIC_E_CUDA;
  char *p = (char *)base;
  SortLaunch S;
  S.ncell = nr * nz;
  S.n = n;
  S.src = Parts{(int32_t *)cell, (double *)a, (double *)b, (double *)vr, (double *)vt,
                (double *)vz, (double *)w, (uint32_t *)id};
  S.dst = Parts{cell_out, a_out, b_out, vr_out, vt_out, vz_out, w_out, id_out};
  S.counts = (int32_t *)p;
  S.offs = (int32_t *)(p + kCountsBytes);
  S.cursor = (int32_t *)(p + 2 * kCountsBytes);
  S.total = (long long *)(p + 2 * kCountsBytes + kCursorBytes);
  S.scan_scratch = p + 2 * kCountsBytes + kCursorBytes + kTotalBytes;
  cudaStream_t s = (cudaStream_t)stream;
  // launch_sort zeroes the counts and cursors it needs before using them
  if (launch_sort(S, s) != cudaSuccess) return PIC_E_CUDA;
  long long tot = 0;
  if (cudaMemcpyAsync(&tot, S.total, sizeof(long long), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PIC_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PIC_E_CUDA;
  *n_out = tot;
  return PIC_OK;
}
