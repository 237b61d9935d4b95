// Launch wrappers of the sm_103a kernels (kernels.cu), called by the C ABI.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace ilu0dd {

struct DevCtx {
  // preconditioner (fused apply)
  const unsigned char* stream;
  const CtaDesc* cta;
  const PieceDesc* pieces;
  int nsub, threads, prefetch_bytes, vec_bytes, factor_prec;
  size_t smem_bytes;
  // SpMV (sliced ELL of the reordered full matrix)
  const int32_t* slice_off;
  const int32_t* sell_col;
  const double* sell_val;
  int64_t nslices;
  // permutation
  const int32_t* perm;
  const int32_t* iperm;
  // solver state
  int32_t N;
  int64_t ntiles, ntiles_pow2;
  double* vec[kNumVec];
  double* partials;     // 5 arrays of ntiles_pow2
  uint32_t* counters;
  SolverScalars* scal;
  double* hist;
  int32_t* err;
};

// Opt the apply kernels into the context's dynamic shared memory.
cudaError_t apply_configure(const DevCtx& d);

// z = M^-1 r (mode plain), or the fused BiCGSTAB variants (modes P and S).
cudaError_t launch_apply(const DevCtx& d, int mode, const double* r, double* z, cudaStream_t s);

// y = A_p x; kind 0 plain, 1: v = A ph with (rh.v) -> alpha, 2: t = A sh with (t.s),(t.t) -> omega.
cudaError_t launch_spmv(const DevCtx& d, int kind, const double* x, double* y, cudaStream_t s);

// x += alpha ph + omega sh; r = s - omega t; (r.r), (rh.r) -> convergence test, beta.
cudaError_t launch_update(const DevCtx& d, cudaStream_t s);

// Initial state from b (reordered): x = 0, r = rh = p = b, v = 0, rho = bb = (b.b).
cudaError_t launch_init(const DevCtx& d, double rtol, int32_t maxit, cudaStream_t s);

// r = b - t (t = A x computed before); rel_true; mode 1 also restarts from it.
cudaError_t launch_residual(const DevCtx& d, int restart, cudaStream_t s);

// *out = x . y in the fixed order.
cudaError_t launch_dot(const DevCtx& d, const double* x, const double* y, double* out, cudaStream_t s);

// Same dot product on caller-provided scratch: `partials` holds m doubles
// (m = tiles padded to a power of two, entries past the tile count zero) and
// `counter` one zeroed word; used by the allocation-free entry point.
cudaError_t launch_dot_scratch(const double* x, const double* y, int32_t n_brows, double* partials, int64_t m,
                               uint32_t* counter, double* out, cudaStream_t s);

// dir 0: out = in[perm] (natural -> reordered); dir 1: inverse.
cudaError_t launch_permute(const DevCtx& d, const double* in, double* out, int dir, cudaStream_t s);

}  // namespace ilu0dd
