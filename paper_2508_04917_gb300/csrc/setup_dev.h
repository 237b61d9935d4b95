// Device-side numeric setup (setup_dev.cu): the same factors, factor stream
// and SpMV matrix as the host path, computed on the GPU from the host plan.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace ilu0dd {

struct DeviceSetupResult {
  int32_t bad_row = -1;     // first reordered row with a zero pivot (ILU0DD_ERR_ZERO_PIVOT)
  bool range_bad = false;   // DF64: a factor outside [2^-70, 2^100] (ILU0DD_ERR_INVALID)
  cudaError_t cuda = cudaSuccess;
  const double* w = nullptr;     // device: L below, U on and above the diagonal (dd order)
  const double* invd = nullptr;  // device: D^-1 per row
};

// Device scratch the numeric setup of plan `p` needs (bytes).
size_t device_setup_scratch_bytes(const Plan& p);

// Fill the workspace's factor stream, SpMV matrix, CtaDesc and PieceDesc
// arrays and slice offsets from the caller's natural-order values
// `aval_in` (bs * bs * nnzb doubles in host memory or in device memory of the
// current device). `scratch` is device memory of
// at least device_setup_scratch_bytes(p) bytes, 256-byte aligned; it may be
// released after the call (res->w and res->invd point into it). Synchronises
// `s`. Returns ILU0DD_OK, ILU0DD_ERR_ZERO_PIVOT, ILU0DD_ERR_INVALID (DF64
// range), ILU0DD_ERR_WORKSPACE (scratch too small or misaligned) or
// ILU0DD_ERR_CUDA.
int setup_on_device(const Plan& p, const double* aval_in, unsigned char* scratch, size_t scratch_bytes,
                    unsigned char* ws, cudaStream_t s, DeviceSetupResult* res);

// Level sets of the lower (upper = 0) or upper (upper = 1) triangle of a
// block-diagonal pattern (device CSR rp/col of the reordered dropped matrix,
// subdomain row ranges part_ptr[nsub + 1]) by Algorithm 5, one block per
// subdomain; lev[N] receives each row's level and nlev[nsub] (optional) each
// subdomain's level count. Entries outside a row's subdomain are ignored.
cudaError_t launch_levels(const int32_t* rp, const int32_t* col, const int32_t* part_ptr, int32_t nsub, int upper,
                          int32_t* lev, int32_t* nlev, cudaStream_t s);

}  // namespace ilu0dd
