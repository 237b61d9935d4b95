// Allocation-free dot product: ilu0dd_dot_noalloc (declared in include/ilu0dd.h).
//
// The regular entry points keep their reduction scratch in the device
// workspace that the caller allocates once. Some callers cannot make even
// that one allocation: code that runs while a CUDA graph is being captured
// (where cudaMalloc is not permitted), code whose device memory is owned by
// another framework's allocator or by a fixed memory budget, and hot loops
// that must never touch the allocator. For them the reduction scratch of this
// entry point is a file-scope __device__ array that is part of the loaded
// module: it exists on every device that loads the library and lives until the
// process exits, and nothing here allocates or frees memory.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"
#include "kernels.h"

namespace {

// Tile partials of the fixed-order reduction (one per 256 block rows, padded
// to a power of two) plus one completion counter: 16384 tiles cover
// 4,194,304 block rows (12,582,912 doubles per vector).
constexpr int64_t kNoAllocMaxTiles = 16384;
struct NoAllocScratch {
  double partials[kNoAllocMaxTiles];
  uint32_t counter;
  uint32_t pad[63];
};
static __device__ __align__(256) NoAllocScratch g_scratch;

// Device address of g_scratch per device. In host code `g_scratch` names a
// host-side stand-in, so the kernel is always given the address that
// cudaGetSymbolAddress returns with the device current.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
NoAllocScratch* g_addr[kMaxDevices] = {};

cudaError_t scratch_for_current_device(NoAllocScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<NoAllocScratch*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int ilu0dd_dot_noalloc(const double* d_x, const double* d_y, int64_t n_brows, double* d_result,
                                  void* stream) {
  if (n_brows < 0 || !d_result || (n_brows > 0 && (!d_x || !d_y))) return ILU0DD_ERR_INVALID;
  const int64_t ntiles = (n_brows + ilu0dd::kDotTile - 1) / ilu0dd::kDotTile;
  if (ntiles > kNoAllocMaxTiles) return ILU0DD_ERR_WORKSPACE;  // beyond the static scratch
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n_brows == 0) return cudaMemsetAsync(d_result, 0, sizeof(double), s) == cudaSuccess ? ILU0DD_OK : ILU0DD_ERR_CUDA;
  NoAllocScratch* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return ILU0DD_ERR_CUDA;
  int64_t m = 1;
  while (m < ntiles) m *= 2;
  // The array keeps the previous call's contents: the halving sum reads the
  // zero padding past the tile count, and the completion counter starts at 0.
  cudaError_t e = cudaSuccess;
  if (m > ntiles) e = cudaMemsetAsync(scratch->partials + ntiles, 0, sizeof(double) * (size_t)(m - ntiles), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(&scratch->counter, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess)
    e = ilu0dd::launch_dot_scratch(d_x, d_y, (int32_t)n_brows, scratch->partials, m, &scratch->counter, d_result, s);
  return e == cudaSuccess ? ILU0DD_OK : ILU0DD_ERR_CUDA;
}
