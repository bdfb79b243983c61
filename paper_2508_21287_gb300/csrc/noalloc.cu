// Canonical row sort that allocates no device memory.
//
// Some callers cannot allocate device memory at the moment they need a sort: cudaMalloc and
// cudaFree synchronise the whole device, which a latency-bound serving thread cannot afford;
// a host framework whose caching allocator has reserved (almost) all device memory makes a
// raw cudaMalloc fail or fragment its pool; and code that is handed only pre-reserved
// buffers by its owner is not allowed to allocate at all. dm_sort_rows_static serves them:
// it sorts caller-owned device rows into a caller-owned output buffer, and every temporary
// (two permutation arrays, the digit histograms and their scan) lives in one file-scope
// device array of fixed size, reserved when the library's device code is loaded and held by
// every GPU that loads the library until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dm.h"
#include "kernels.h"

namespace {

constexpr int64_t kMaxRows = DM_SORT_STATIC_MAX_ROWS;
constexpr int32_t kMaxWidth = 64;
constexpr int64_t kHist = dmk::radix_hist_elems(kMaxRows);
constexpr int64_t kScanTmp = dmk::scan_tmp_elems(kHist);
// the radix passes of n <= kMaxRows rows use at most these many histogram and scan words
static_assert(dmk::radix_hist_elems(kMaxRows) <= kHist, "histogram region too small");
static_assert(dmk::scan_tmp_elems(dmk::radix_hist_elems(kMaxRows)) <= kScanTmp, "scan region too small");
static_assert(kMaxRows % 2 == 0, "two int32 permutations per pair of 8-byte words");
// layout in 8-byte words: perm A | perm B | hist | hist scan (+1) | scan temporaries
constexpr int64_t kPermWords = kMaxRows / 2;
constexpr int64_t kScratchWords = 2 * kPermWords + kHist + (kHist + 1) + kScanTmp;

static __device__ __align__(256) unsigned long long g_sort_scratch[kScratchWords];

// Device address of g_sort_scratch in the current device's context. It is looked up on every
// call (a host-side lookup, no device work): an address cached across calls would go stale if
// the context were reset and the module loaded again at another address.
int scratch_for_current_device(unsigned long long **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DM_E_CUDA;
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
  if (e != cudaSuccess || !p) return DM_E_CUDA;
  *out = (unsigned long long *)p;
  return DM_OK;
}

}  // namespace

extern "C" int dm_sort_rows_static(const int32_t *rows_in, const float *scores_in, int64_t n, int32_t w,
                                   int32_t bits, int32_t *rows_out, float *scores_out, void *stream) {
  if (n < 0 || w < 1 || w > kMaxWidth || bits < 1 || bits > 31) return DM_E_INVAL;
  if (n > kMaxRows) return DM_E_CAPACITY;
  if (n > 0 && (!rows_in || !rows_out || (scores_in && !scores_out))) return DM_E_INVAL;
  unsigned long long *base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc != DM_OK || n == 0) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t *A = (int32_t *)base;
  int32_t *B = (int32_t *)(base + kPermWords);
  int64_t *hist = (int64_t *)(base + 2 * kPermWords);
  int64_t *hscan = hist + kHist;
  int64_t *tmp = hscan + kHist + 1;
  // every scratch word read below is written first in the same call (iota, histograms,
  // scans), so nothing has to be cleared between calls
  if (dmk::launch_iota(A, n, s) != cudaSuccess) return DM_E_CUDA;
  for (int col = w - 1; col >= 0; col--)
    for (int shift = 0; shift < bits; shift += 8) {
      if (dmk::radix_pass((const uint32_t *)rows_in + col, w, A, B, n, shift, hist, hscan, tmp, s) != cudaSuccess)
        return DM_E_CUDA;
      int32_t *t = A;
      A = B;
      B = t;
    }
  if (dmk::launch_gather_rows(rows_in, scores_in, A, n, w, rows_out, scores_in ? scores_out : nullptr, s) !=
      cudaSuccess)
    return DM_E_CUDA;
  return DM_OK;
}
