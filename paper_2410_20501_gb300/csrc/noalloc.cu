// pm_deposit_noalloc: the TSC deposit for callers that cannot allocate device
// memory.  Instead of a caller workspace it uses one file-scope device array.
#include <string.h>

#include <mutex>

#include "pm_internal.cuh"

namespace pmgb {

namespace {

constexpr int kNoallocMaxN = 64;
constexpr int64_t kNoallocMaxNp = (int64_t)1 << 18;
constexpr size_t kNoallocBytes = (size_t)16 << 20;   // 16 MiB: the pm_deposit workspace at the limits is 14.5 MiB
constexpr int kMaxDevices = 64;

// Shared by every call on a device; it keeps the previous call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (host code must
// not use the symbol itself: on the host it is only a stand-in).  Outside
// stream capture the address is looked up again on every call, so a device
// reset (after which the module is loaded anew and the array may move) is
// followed; during capture the address recorded by the last uncaptured call
// on this device is used, and a call that has none returns PM_EINVAL.
pm_status scratch_address(cudaStream_t s, void** out) {
  int dev = 0;
  PM_TRY(cuda_status(cudaGetDevice(&dev)));
  if (dev < 0 || dev >= kMaxDevices) return PM_EINVAL;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  PM_TRY(cuda_status(cudaStreamIsCapturing(s, &cap)));
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    PM_TRY(cuda_status(cudaGetSymbolAddress(&p, g_noalloc_scratch)));
    g_scratch_addr[dev] = p;
  }
  if (!g_scratch_addr[dev]) return PM_EINVAL;
  *out = g_scratch_addr[dev];
  return PM_OK;
}

}  // namespace

}  // namespace pmgb

using namespace pmgb;

extern "C" pm_status pm_deposit_noalloc(const uint32_t* X, int64_t np, int n, float* rho, void* stream) {
  if (!valid_n(n) || n > kNoallocMaxN || np < 0 || np > kNoallocMaxNp || (np > 0 && !X) || !rho ||
      (((uintptr_t)X | (uintptr_t)rho) & 15) != 0)
    return PM_EINVAL;
  const size_t need = layout_workspace(nullptr, nullptr, n, np, PM_WS_SORT);
  if (need > kNoallocBytes) return PM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  void* base = nullptr;
  PM_TRY(scratch_address(s, &base));
  Workspace w;
  layout_workspace(&w, base, n, np, PM_WS_SORT);
  // Nothing in the scratch has to start at zero: every buffer the deposit
  // reads (cell starts, keys, the permutation, sorted positions, block
  // partials) is fully written earlier in the same call.
  uint32_t* perm;
  PM_TRY(sort_cells(X, np, n, w, s, w.cellstart, &perm));
  PM_TRY(permute_particles(perm, np, X, nullptr, nullptr, w.Xs, nullptr, nullptr, s));
  PM_TRY(deposit_sorted(w.Xs, np, w.cellstart, n, rho, w.partials, w.scalars, s,
                        Crowded{w.runs, w.meds, w.bigs, w.smalls, w.moments}));
  return launch_status();
}
