// Launch wrappers of the sm_103a kernels (kernels.cu), called by the C ABI.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace ilu0dd {

// Everything a kernel needs about one system (copied by value into kernel
// parameters for single-system launches, and into a device array for batched
// launches).
struct SysDesc {
  // preconditioner (fused apply)
  const unsigned char* stream;
  const CtaDesc* cta;
  const PieceDesc* pieces;
  // SpMV (sliced ELL of the reordered full matrix)
  const int32_t* slice_off;
  const int32_t* sell_col;
  const double* sell_val;
  int64_t nslices;
  // permutation
  const int32_t* perm;
  const int32_t* iperm;
  const uint8_t* row_l0;  // 1 for rows of L level 0 (the row-flag apply's initial flags)
  // solver state
  double* vec[kNumVec];
  double* partials;     // 5 arrays of ntiles_pow2
  uint32_t* counters;
  SolverScalars* scal;
  double* hist;
  int32_t* err;
  int64_t ntiles, ntiles_pow2;
  int32_t N, nsub;
  int32_t vec_bytes, prefetch_bytes;
  // apply waits: SM cycles before giving up; a piece (global index) whose
  // completion is never reached (-1: none; failure-path tests only)
  uint64_t wait_cycles;
  int32_t wait_stuck;
  // 1: the stream is in the row-thread layout (3x3 blocks, FP32 or BF16
  // factors, no row with more than kDescSlots blocks on either side)
  int32_t row_thread;
};

// Host view of one context: the system and its launch configuration.
struct DevCtx {
  SysDesc sd;
  int threads, factor_prec;
  size_t smem_bytes;
  size_t smem_rowsync;  // shared memory of the row-flag apply (0: does not fit)
  int bs = 3;  // block dimension: 3 or 1 (scalar CSR)
  int traversal = 0;  // apply traversal: 0 vertex-centric, 1 edge-centric (ilu0dd_opts.traversal)
};

// Work item of a batched launch: system index and block index inside it.
struct BatchItem {
  int32_t sys, local;
};

// Opt the apply kernels into the device's shared memory.
cudaError_t apply_configure(const DevCtx& d);

// z = M^-1 r (mode plain), or the fused BiCGSTAB variants (modes P and S).
cudaError_t launch_apply(const DevCtx& d, int mode, const double* r, double* z, cudaStream_t s);

// The same for subdomains [sub0, sub0 + nsub) only (r and z are full vectors;
// other subdomains' entries are neither read nor written).
cudaError_t launch_apply_range(const DevCtx& d, int mode, const double* r, double* z, int sub0, int nsub,
                               cudaStream_t s);

// The same z = M^-1 r in two launches (L sweep r -> z, then D^-1 and U~ sweep
// z -> z in place), the unfused variant of the fusion ablation.
cudaError_t launch_apply_unfused(const DevCtx& d, const double* r, double* z, cudaStream_t s);
// The plain apply with per-row completion flags (Algorithm 4's
// synchronization) instead of per-level mbarriers; d.smem_rowsync must be > 0.
cudaError_t launch_apply_rowsync(const DevCtx& d, const double* r, double* z, cudaStream_t s);
// The plain apply with the edge-centric traversal (one thread per block,
// shared-memory atomics); FP64, FP32 and BF16 factors only.
cudaError_t launch_apply_edge(const DevCtx& d, const double* r, double* z, cudaStream_t s);
// The plain FP64 apply with the subdomain vector in global memory (z).
cudaError_t launch_apply_vglobal(const DevCtx& d, const double* r, double* z, cudaStream_t s);

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

// ---- batched launches: one launch covers the work items of many systems.
// `sys` is a device array of SysDesc; items list (system, subdomain) for the
// apply and (system, dot tile) for the others. Systems whose solve is done are
// skipped. `grid` blocks loop over the items (persistent launch). Every
// system of one launch has block dimension `bs` (3 or 1) and the same
// row-thread flag (SysDesc.row_thread).
cudaError_t launch_apply_batched(const SysDesc* sys, const BatchItem* items, int64_t nitems, int mode,
                                 int factor_prec, int bs, int row_thread, int threads, size_t smem, int grid,
                                 cudaStream_t s);
cudaError_t launch_spmv_batched(const SysDesc* sys, const BatchItem* items, int64_t nitems, int kind, int bs,
                                int grid, cudaStream_t s);
cudaError_t launch_update_batched(const SysDesc* sys, const BatchItem* items, int64_t nitems, int bs, int grid,
                                  cudaStream_t s);
// mode 0: init from b (vec B), 1: r = b - t with rel_true, 2: restart from r
// (systems flagged in `flags`).
cudaError_t launch_vec_batched(const SysDesc* sys, const BatchItem* items, int64_t nitems, int mode, double rtol,
                               int32_t maxit, const int32_t* flags, int bs, int grid, cudaStream_t s);
// dir 0: vec B of system i <- in[i] permuted; dir 1: out[i] <- vec X of system i.
cudaError_t launch_permute_batched(const SysDesc* sys, const BatchItem* items, int64_t nitems,
                                   const double* const* ptrs, int dir, int bs, int grid, cudaStream_t s);
// out[i] = the solver scalars of system i (one small launch).
cudaError_t launch_gather_status(const SysDesc* sys, int32_t nsys, SolverScalars* out, cudaStream_t s);

// Blocks per SM of the batched kernels (for persistent grids).
int apply_blocks_per_sm(int factor_prec, int bs, int row_thread, int threads, size_t smem);
int tile_blocks_per_sm(int bs);

}  // namespace ilu0dd
