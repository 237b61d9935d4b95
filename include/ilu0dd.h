/*
 * ilu0dd — subdomain-wise ILU0 preconditioning on GB300 (sm_103a).
 *
 * C ABI of the library built from paper_2508_04917_gb300/csrc. It implements
 * the hot path of arXiv 2508.04917, "Mapping Sparse Triangular Solves to GPUs
 * via Fine-grained Domain Decomposition": a 3x3-block (BSR) or scalar (CSR)
 * system A x = b is cut into subdomains (box subdomains of a grid, Algorithm
 * 2, or the parts of a graph partition, Section 3.1), reordered so every
 * subdomain is a contiguous row range (Algorithm 3),
 * stripped of inter-subdomain blocks (Section 3.2) and factored with ILU0 /
 * ILDU0 (Algorithm 7). The preconditioner z = M^-1 r, M = LU, is then applied
 * by one fused L -> D^-1 -> U kernel with one thread block per subdomain and
 * the subdomain vector in shared memory, rows scheduled by level
 * (Sections 4.2, 4.3, 4.4), inside preconditioned BiCGSTAB (Algorithm 1).
 *
 * Conventions of every entry point:
 *  - Return value: ILU0DD_OK (0) or one of the ILU0DD_ERR_* codes below. No
 *    exception crosses the ABI; nothing is printed unless opts.trace is set.
 *  - "host" pointers are ordinary CPU memory, "device" pointers are CUDA
 *    device memory of the current device.
 *  - `stream` is a cudaStream_t passed as void*; 0 means the legacy default
 *    stream.
 *  - The library never allocates device memory. The caller allocates one
 *    device workspace of ilu0_dd_workspace_size() bytes (256-byte aligned)
 *    and keeps it alive for the lifetime of the context (and, for the device
 *    setup, a scratch buffer that is free again once setup returns). Small
 *    host-side bookkeeping (the context object, host copies for
 *    ilu0_dd_export) is allocated with malloc and released by
 *    ilu0_dd_destroy. The exceptions are the static array of
 *    ilu0dd_dot_noalloc and the streams ilu0_dd_apply_host creates.
 *  - Vectors hold bs doubles per block row (bs = the matrix's block_dim: 3
 *    or 1), entry bs*i + a; "3*N doubles" below reads bs*N for scalar
 *    matrices.
 */
#ifndef ILU0DD_H_
#define ILU0DD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define ILU0DD_OK 0
#define ILU0DD_ERR_INVALID 1        /* bad pointer, size, pattern (unsorted columns, missing diagonal) */
#define ILU0DD_ERR_ZERO_PIVOT 2     /* singular or non-finite pivot block (3x3 or 1x1) in ILU0 */
#define ILU0DD_ERR_SMEM 3           /* a subdomain vector does not fit in shared memory */
#define ILU0DD_ERR_CUDA 4           /* a CUDA call failed (see ilu0_dd_query ILU0DD_Q_CUDA_ERROR) */
#define ILU0DD_ERR_BREAKDOWN 5      /* BiCGSTAB breakdown: (r^,v)=0, rho=0, omega=0 or non-finite */
#define ILU0DD_ERR_NOT_CONVERGED 6  /* maxit reached, or the true residual misses rtol after a restart */
#define ILU0DD_ERR_NONFINITE 7      /* NaN/Inf in an input vector */
#define ILU0DD_ERR_WORKSPACE 8      /* workspace too small or misaligned */
#define ILU0DD_ERR_DEVICE_WAIT 9    /* a device-side bounded wait expired (see ilu0_dd_device_error) */

/* ---- factor storage precision (opts.factor_prec) --------------------- */
#define ILU0DD_F64 0   /* factors and apply arithmetic in FP64 */
#define ILU0DD_F32 1   /* factors stored in FP32, apply in FP32 */
#define ILU0DD_BF16 2  /* factors stored in BF16, apply in FP32 */
#define ILU0DD_DF64 3  /* factors stored as float pairs hi + lo (8 bytes, about 48
                          significant bits), apply in double-float arithmetic on
                          the FP32 pipe; every factor magnitude must lie in
                          [2^-70, 2^100] (else ILU0DD_ERR_INVALID). Not in the
                          paper: FP64-accurate to about 1e-14 relative per
                          operation where this GPU's FP64 pipe is the bound. */

/* ---- inputs ----------------------------------------------------------- */

/* Block-CSR matrix in natural cell order gidx = i + nx*(j + ny*k) (grid
 * path) or any order (partitioned path): row_ptr[n_brows+1], col_idx[nnzb]
 * (strictly ascending per row, diagonal block present), val[bs*bs*nnzb]
 * (row-major bs x bs blocks). block_dim = bs: 3 (also 0) for 3x3 blocks, 1
 * for a scalar CSR matrix; vectors then hold bs*n_brows doubles.
 * n_brows = 0 (an empty system) is accepted on the partitioned path
 * (ilu0dd_plan_create_partitioned, any nparts >= 0; the grid path needs
 * positive sides): nothing is launched, vector pointers may be null, a solve
 * returns ILU0DD_OK after no iteration, alone or in a batch.
 * Each array may be in host memory or in device memory of the current device
 * (the library tells them apart with cudaPointerGetAttributes). The
 * structural setup runs on the host, so device-resident row_ptr and col_idx
 * are copied to host memory for it (a synchronous copy); device-resident
 * values go to the device numeric setup (ilu0_dd_setup_planned with scratch)
 * by a device-to-device copy, and are copied to the host only for the host
 * numeric setup. The caller keeps ownership; nothing is kept after setup. */
typedef struct {
  int32_t n_brows;
  int32_t block_dim;
  int64_t nnzb;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const double* val;
} ilu0dd_bsr;

/* Grid (nx, ny, nz) and subdomain box (sx, sy, sz), the inputs of
 * Algorithm 2. Edge subdomains are smaller when a side does not divide. */
typedef struct {
  int32_t nx, ny, nz;
  int32_t sx, sy, sz;
} ilu0dd_geom;

typedef struct {
  int32_t factor_prec;      /* ILU0DD_F64 / ILU0DD_F32 / ILU0DD_BF16 / ILU0DD_DF64 */
  int32_t threads_per_cta;  /* apply block size, a multiple of 32; 0 = from the widest level: 3x3 FP64 / DF64
                               factors (three threads per row, ten rows per warp) one warp per row group,
                               1.5x from four groups, at most 384; 3x3 FP32 / BF16 factors with no row of
                               more than three blocks on either side (one thread per row, 32 rows per warp,
                               ILU0DD_Q_ROW_THREAD = 1) 1.5 warps per row group, at most 256; other 3x3
                               FP32 / BF16 systems (three threads per row) one warp per row group, at most
                               384; scalar rows (32 per warp) one warp per row group, at most 384 */
  int32_t prefetch_bytes;   /* apply: L2 prefetch distance per block, bytes (multiple of 16); 0 = 32768 (16384 for BF16) */
  int32_t maxit;            /* BiCGSTAB iteration limit; 0 = 10000 */
  double rtol;              /* stop when ||r||_2/||b||_2 < rtol; 0 = 1e-8 */
  int32_t check_every;      /* iterations per CUDA-graph launch between convergence polls; 0 = 8 */
  int32_t use_graphs;       /* 1 = capture iterations as CUDA graphs (default), 0 = plain launches */
  int32_t keep_host;        /* 1 = keep host copies of factors and levels for ilu0_dd_export */
  int32_t trace;            /* 1 = print per-phase timings to stderr */
  int32_t traversal;        /* apply traversal of a level (Section 4.2.3), used by ilu0_dd_apply and
                               bicgstab_solve: 0 = vertex-centric, rows in a fixed order (default,
                               deterministic); 1 = edge-centric, the blocks of a level spread over
                               threads with shared-memory atomic adds (the paper's fastest kernel on
                               MI210; its rounding order, hence the iteration count, may vary).
                               1 is not available with ILU0DD_DF64 (ILU0DD_ERR_INVALID); batched
                               solves always use 0. */
  int32_t apply_mapping;    /* threads per 3x3 block row in the apply: 0 = automatic (default: one
                               thread per row, the row-thread layout, for FP32 / BF16 factors when
                               no row has more than three blocks on either side; else three);
                               1 = three threads per row always (the row-thread layout's ablation:
                               the same bits where both apply). Any other value: ILU0DD_ERR_INVALID.
                               ILU0DD_Q_ROW_THREAD reports the mapping taken. */
} ilu0dd_opts;

typedef struct {
  int32_t status;             /* ILU0DD_OK or an error code */
  int32_t iterations;         /* BiCGSTAB iterations (j + 1 at the stopping iteration) */
  int32_t restarts;           /* 0 or 1: restarts from the true residual */
  int32_t reserved;
  double rel_res_recurrence;  /* ||r_j|| / ||b|| of the recurrence at exit */
  double rel_res_true;        /* ||b - A x|| / ||b|| recomputed at exit */
  double setup_s;             /* wall time of ilu0_dd_setup (host side included) */
  double solve_s;             /* wall time of the last bicgstab_solve */
} ilu0dd_info;

typedef struct ilu0dd_ctx ilu0dd_ctx;

/* Fill *opts with the defaults listed above; trace defaults to 1 when the
 * environment variable ILU0DD_TRACE is a positive integer. */
int ilu0dd_default_opts(ilu0dd_opts* opts);

/* Human-readable name of a return code (static string, never NULL). */
const char* ilu0dd_strerror(int code);

/*
 * Device workspace bytes needed by ilu0_dd_setup for this matrix, geometry
 * and options. Runs the structural part of the setup on the host
 * (Algorithm 2, Algorithm 3, Section 3.2 drop, Algorithm 5 levels) without
 * factoring. Errors: INVALID (pattern), SMEM (subdomain too large for shared
 * memory of the current device).
 */
int ilu0_dd_workspace_size(const ilu0dd_bsr* A, const ilu0dd_geom* geom, const ilu0dd_opts* opts,
                           size_t* bytes);

/*
 * Build the preconditioner and the solver state in d_workspace
 * (ws_bytes >= ilu0_dd_workspace_size): partition (Algorithm 2), reorder
 * (Algorithm 3), drop inter-subdomain blocks (Section 3.2), block ILU0 and
 * ILDU0 in FP64 (Algorithm 7), level sets per subdomain (Algorithm 5), pack
 * the factors for the fused apply in opts.factor_prec, and upload everything
 * on `stream`. The host-side steps run on the CPU threads of the caller's
 * process; A may be freed after return. Synchronizes `stream`.
 * On success *out owns host memory released by ilu0_dd_destroy; it refers
 * to d_workspace, which must outlive it.
 */
int ilu0_dd_setup(const ilu0dd_bsr* A, const ilu0dd_geom* geom, const ilu0dd_opts* opts,
                  void* d_workspace, size_t ws_bytes, void* stream, ilu0dd_ctx** out);

/* ---- two-phase setup: plan once on the host, factor on the device ------- */

typedef struct ilu0dd_plan ilu0dd_plan;

/*
 * The structural half of ilu0_dd_setup on the host (Algorithm 2, Algorithm 3,
 * the drop of Section 3.2, Algorithm 5 level sets, the packing layout), run
 * once. Reports the device workspace bytes (*workspace_bytes, as
 * ilu0_dd_workspace_size) and the device scratch bytes (*scratch_bytes) that
 * ilu0_dd_setup_planned needs to factor and pack on the device; either
 * pointer may be NULL. Only A's pattern is read. On success *out owns host
 * memory released by ilu0dd_plan_destroy. Errors as ilu0_dd_workspace_size.
 */
int ilu0dd_plan_create(const ilu0dd_bsr* A, const ilu0dd_geom* geom, const ilu0dd_opts* opts,
                       ilu0dd_plan** out, size_t* workspace_bytes, size_t* scratch_bytes);

/*
 * As ilu0dd_plan_create for a matrix without a grid: the subdomains are the
 * parts of a given partition (Section 3.1's graph-partition path) instead of
 * Algorithm 2's boxes. part_id: HOST array of n_brows labels in [0, nparts)
 * (any partition, e.g. from ilu0dd_partition_bfs or an external graph
 * partitioner); every part must fit the shared-memory limit of the apply.
 * Rows of a part keep their relative order (Section 3.1's stable grouping).
 * Errors: INVALID (pattern, labels out of range), SMEM (a part too large).
 */
int ilu0dd_plan_create_partitioned(const ilu0dd_bsr* A, const int32_t* part_id, int32_t nparts,
                                   const ilu0dd_opts* opts, ilu0dd_plan** out, size_t* workspace_bytes,
                                   size_t* scratch_bytes);

/*
 * Graph partition of A's pattern into parts of part_rows rows (the last may
 * be smaller), the project's stand-in for the METIS partition the paper uses
 * for matrices without a grid (Section 3.1, equal-size parts as in Section
 * 5): the vertices in breadth-first order over the pattern of A + A^T
 * (neighbours ascending), component by component, each component's order
 * started at the last vertex that a first search from its smallest vertex
 * reaches; part_id[order[t]] = t / part_rows. Host only, deterministic.
 * part_id: HOST array of n_brows int32 (written); *nparts receives the number
 * of parts. Errors: INVALID (null arrays, part_rows <= 0, column out of range).
 */
int ilu0dd_partition_bfs(const ilu0dd_bsr* A, int32_t part_rows, int32_t* part_id, int32_t* nparts);

/*
 * The numeric half: as ilu0_dd_setup, for a matrix with the pattern given to
 * ilu0dd_plan_create (n_brows and nnzb are checked, the pattern is not).
 * With d_scratch (device, >= *scratch_bytes of the plan, 256-byte aligned)
 * the block ILU0 (Algorithm 7; one thread block per subdomain, one thread per
 * row of an L level) and the packing of the factor stream and of the SpMV
 * matrix run on the device, bit-identical to the host path; with d_scratch ==
 * NULL they run on the host. The scratch is free for other use on return.
 * The plan is consumed (it may be used once) and must still be destroyed.
 * Errors: INVALID (plan already used, size mismatch, DF64 range),
 * ZERO_PIVOT, WORKSPACE (workspace or scratch too small or misaligned), CUDA.
 */
int ilu0_dd_setup_planned(ilu0dd_plan* plan, const ilu0dd_bsr* A, void* d_workspace, size_t ws_bytes,
                          void* d_scratch, size_t scratch_bytes, void* stream, ilu0dd_ctx** out);

int ilu0dd_plan_destroy(ilu0dd_plan* plan);

/*
 * z = M^-1 r = U~^-1 D^-1 L^-1 r (Sections 4.3-4.4), one fused kernel launch:
 * one thread block per subdomain, the subdomain vector in shared memory, the
 * rows in Algorithm 5's level order (a warp starts a level's rows once the
 * previous level is complete; one mbarrier per level slice, no block
 * barriers). d_r, d_z: device, bs*N doubles each, in the reordered
 * (subdomain-contiguous) numbering; they must not overlap. Asynchronous on
 * `stream`. The context is only read, so concurrent applies on one context
 * are safe. A wait that exceeds its bound (ilu0dd_set_wait_limits) sets the
 * device error word (ilu0_dd_device_error) instead of hanging.
 */
int ilu0_dd_apply(const ilu0dd_ctx* ctx, const double* d_r, double* d_z, void* stream);

/*
 * z = M^-1 r as ilu0_dd_apply, from and to HOST buffers: h_r, h_z hold 3*N
 * doubles in the reordered numbering (page-locked memory lets the copies
 * overlap; pageable memory works but serialises them). The subdomains are
 * split into up to sixteen contiguous chunks (subdomains are independent:
 * Section 3.2), each copied in, applied and copied out on its own stream of
 * the context, so one chunk's copies overlap other chunks' applies. Work is
 * ordered after earlier work on `stream`, and `stream` waits for all of it;
 * h_z is valid once `stream` has completed. Uses the context's solver
 * vectors as device staging: do not overlap with bicgstab_* calls on the same
 * context. Not const: creates the context's streams on first use.
 */
int ilu0_dd_apply_host(ilu0dd_ctx* ctx, const double* h_r, double* h_z, void* stream);

/*
 * The same z = M^-1 r as ilu0_dd_apply, unfused: two launches, the L sweep
 * (r -> z) and then the D^-1 and U~ sweep (z -> z in place), each loading
 * the subdomain vector into shared memory; the separate-kernel variant of
 * the paper's preconditioner-application comparison (Section 5, Table 4),
 * kept to measure what the fusion of Section 4.4 saves. Same arguments,
 * results bit-identical to ilu0_dd_apply for FP64, FP32 and BF16 factors
 * (DF64 rescales between the launches: equal to rounding).
 */
int ilu0_dd_apply_unfused(const ilu0dd_ctx* ctx, const double* d_r, double* d_z, void* stream);

/*
 * The same z = M^-1 r as ilu0_dd_apply with the synchronization of the
 * paper's synchronization-free triangular solve (Algorithm 4) in place of the
 * level order: one completion flag per row in shared memory, and each row
 * waits (spinning, bounded like every wait of the apply) for exactly the rows
 * it reads instead of for the whole previous level; the L and U sweeps are
 * separated by one block barrier. Same arguments; results bit-identical to
 * ilu0_dd_apply (each row's arithmetic and its order are unchanged). For the
 * synchronization ablation. Returns ILU0DD_ERR_SMEM when the subdomain vector
 * plus one flag byte per row does not fit in shared memory (the largest
 * boxes), ILU0DD_ERR_INVALID for overlapping r and z.
 */
int ilu0_dd_apply_rowsync(const ilu0dd_ctx* ctx, const double* d_r, double* d_z, void* stream);

/*
 * The same z = M^-1 r as ilu0_dd_apply with the paper's edge-centric
 * traversal (Section 4.2.3) in place of the row-wise one: within each level
 * one thread per block forms that block's product and subtracts it from its
 * row with shared-memory atomic adds (after the row's D^-1 step in the U
 * sweep). The row sums are rounded in a different order, so results agree
 * with ilu0_dd_apply to rounding, not bit for bit. For the traversal
 * ablation; FP64, FP32 and BF16 factors (ILU0DD_ERR_INVALID for DF64, whose
 * float pairs have no atomic add, and for overlapping r and z).
 */
int ilu0_dd_apply_edge(const ilu0dd_ctx* ctx, const double* d_r, double* d_z, void* stream);

/*
 * The same z = M^-1 r as ilu0_dd_apply, FP64 factors only, with the
 * subdomain vector kept in global memory (in d_z itself) instead of shared
 * memory: the vector-in-global-memory variant of the paper's lower-solve
 * comparison (Table 3), to measure what shared memory brings. Results
 * bit-identical to ilu0_dd_apply. ILU0DD_ERR_INVALID for other factor
 * precisions and for overlapping r and z.
 */
int ilu0_dd_apply_global_vector(const ilu0dd_ctx* ctx, const double* d_r, double* d_z, void* stream);

/*
 * Level sets on the device (Algorithm 5, the paper's GPU level assignment,
 * Section 4.2.2), one thread block per subdomain: a row joins level l + 1 once
 * every lower (for d_lev_u: upper) neighbour inside its subdomain sits on a
 * level <= l; rows without such neighbours are level 0. Inputs are DEVICE
 * arrays of the reordered dropped (block-diagonal) pattern: d_row_ptr[n + 1],
 * d_col[nnz] (block rows or scalar rows alike), and the subdomain row ranges
 * d_part_ptr[nsub + 1] (rows of subdomain s are d_part_ptr[s] ..
 * d_part_ptr[s+1] - 1); entries outside a row's subdomain are ignored.
 * Outputs (device, caller-owned): d_lev_l[n], d_lev_u[n], and, if not NULL,
 * d_nlev_l[nsub], d_nlev_u[nsub] (level counts per subdomain). The result
 * equals the library's host level sets (ILU0DD_X_LEVEL_L / _U). Asynchronous
 * on `stream`. ILU0DD_ERR_INVALID for nsub < 0 or null arrays (nsub > 0).
 */
int ilu0dd_levels_device(const int32_t* d_row_ptr, const int32_t* d_col, const int32_t* d_part_ptr, int32_t nsub,
                         int32_t* d_lev_l, int32_t* d_lev_u, int32_t* d_nlev_l, int32_t* d_nlev_u, void* stream);

/*
 * y = A_p x with the full reordered matrix (all inter-subdomain blocks kept,
 * Section 3.2 last paragraph). Device vectors in the reordered numbering,
 * 3*N doubles each, not overlapping. Asynchronous on `stream`.
 */
int ilu0_dd_spmv(const ilu0dd_ctx* ctx, const double* d_x, double* d_y, void* stream);

/*
 * *d_result = x . y over 3*N doubles (device pointers) in the library's fixed
 * summation order: per block row fma(x2,y2,fma(x1,y1,x0*y0)); halving sums in
 * 256-row tiles; halving sum over tiles zero-padded to a power of two.
 * Uses the context's reduction scratch: calls on one context must be
 * serialized on one stream.
 */
int ilu0_dd_dot(const ilu0dd_ctx* ctx, const double* d_x, const double* d_y, double* d_result,
                void* stream);

/*
 * Allocation-free variant of ilu0_dd_dot (the paper has no counterpart; it is
 * a deployment convenience). *d_result = x . y over n_brows block rows
 * (3*n_brows doubles, device pointers, same fixed summation order), without a
 * context and without any allocation: the reduction scratch is a static
 * device array of 16384 tile partials built into the library, present on
 * every device that loads it until the process exits. It serves callers that
 * cannot allocate device memory at the call site, e.g. code running under
 * CUDA-graph capture or under a fixed device-memory budget. Limits and rules:
 *  - n_brows <= 4,194,304 (16384 tiles of 256 block rows), else
 *    ILU0DD_ERR_WORKSPACE;
 *  - the first call on a device looks up the array's device address (with
 *    that device current); make that first call before any stream capture;
 *  - all calls share the one array: calls that may overlap on the GPU (on
 *    different streams, or from several threads) race and must be serialized
 *    by the caller;
 *  - asynchronous on `stream`; never calls cudaMalloc or cudaFree.
 */
int ilu0dd_dot_noalloc(const double* d_x, const double* d_y, int64_t n_brows, double* d_result, void* stream);

/* Permute a device vector between numberings: dir 0 natural -> reordered,
 * dir 1 reordered -> natural (Algorithm 3's perm/iperm). Asynchronous. */
int ilu0_dd_permute(const ilu0dd_ctx* ctx, const double* d_in, double* d_out, int dir, void* stream);

/*
 * Preconditioned BiCGSTAB (Algorithm 1) with K1 = I, K2 = M (right
 * preconditioning), x0 = 0, stopping when ||r_{j+1}||/||b|| < rtol, followed
 * by a true-residual check and at most one restart. d_b and d_x are device
 * vectors in the NATURAL numbering (3*N doubles); d_x receives the solution.
 * Scalars stay on the device; iterations run as CUDA graphs of
 * opts.check_every iterations. Synchronizes `stream`. The solver vectors live
 * in the workspace: solves on one context must not overlap.
 * Errors: BREAKDOWN, NOT_CONVERGED, NONFINITE, CUDA, DEVICE_WAIT.
 */
int bicgstab_solve(ilu0dd_ctx* ctx, const double* d_b, double* d_x, ilu0dd_info* info,
                   void* stream);

/*
 * Stepwise form of bicgstab_solve, for timing and for callers that drive the
 * iteration themselves. bicgstab_start permutes d_b (natural numbering,
 * device) into the workspace and sets x = 0, r = r^ = p = b, rho = (b . b)
 * on the device (asynchronous on `stream`). bicgstab_iterate then launches n
 * iterations of Algorithm 1 on `stream` (5 kernels each: fused apply with
 * the p update, SpMV with (r^ . v), fused apply with s = r - alpha v, SpMV
 * with (t . s) and (t . t), update of x and r with ||r|| and (r^ . r)).
 * Iterations after convergence or breakdown return at once. If
 * host_kernel_ms is not NULL it receives 5*n per-kernel durations in
 * milliseconds (CUDA events recorded on `stream` between the launches) and
 * the call synchronizes `stream`; otherwise it is asynchronous.
 * bicgstab_state synchronizes `stream` and reports the current iteration
 * count, status and recurrence residual (restarts = 0, rel_res_true = 1).
 */
int bicgstab_start(ilu0dd_ctx* ctx, const double* d_b, void* stream);
int bicgstab_iterate(ilu0dd_ctx* ctx, int32_t n, float* host_kernel_ms, void* stream);
int bicgstab_state(ilu0dd_ctx* ctx, ilu0dd_info* info, void* stream);

/*
 * Batched BiCGSTAB over many independent systems (the batching pattern; the
 * paper has no batched solver). Each system is an ilu0dd_ctx from
 * ilu0_dd_setup (any grid and subdomain size; all with the same block dimension,
 * 3x3 or scalar, the same factor_prec, the same apply mapping
 * (ILU0DD_Q_ROW_THREAD) and the current device; otherwise
 * ilu0dd_batch_create returns ILU0DD_ERR_INVALID). It records them in a small device
 * workspace (ilu0dd_batch_workspace_size bytes, 256-byte aligned, caller-owned)
 * and keeps pointers to the contexts: they must outlive the batch, and a
 * context must not be solved alone while a batched solve that uses it runs.
 * opts supplies rtol, maxit (capped by each context's own maxit),
 * check_every and use_graphs; the other fields are ignored.
 *
 * bicgstab_solve_batched runs Algorithm 1 on every system at once: each step
 * of an iteration is ONE kernel launch over the work items of all systems
 * ((system, subdomain) for the fused applies, (system, 256-row tile) for the
 * SpMVs and vector steps, persistent grids), with per-system scalars on the
 * device; systems that have converged are skipped by later launches; the
 * iterations run as CUDA graphs of check_every iterations. d_b[i] and d_x[i]
 * are device vectors of system i in its natural numbering (host arrays of
 * nsys pointers); infos (optional, nsys entries) receives each system's
 * result, as bicgstab_solve reports it. Returns ILU0DD_OK or the first
 * failing system's status. Synchronizes `stream`.
 */
typedef struct ilu0dd_batch ilu0dd_batch;
int ilu0dd_batch_workspace_size(ilu0dd_ctx* const* ctxs, int32_t nsys, size_t* bytes);
int ilu0dd_batch_create(ilu0dd_ctx* const* ctxs, int32_t nsys, const ilu0dd_opts* opts, void* d_workspace,
                        size_t ws_bytes, void* stream, ilu0dd_batch** out);
int bicgstab_solve_batched(ilu0dd_batch* batch, const double* const* d_b, double* const* d_x, ilu0dd_info* infos,
                           void* stream);
void ilu0dd_batch_destroy(ilu0dd_batch* batch);

/* Residual history of the last solve: hist[j] = ||r_j||/||b||, j = 0..iterations
 * (host destination of n doubles; copies min(n, iterations+1) entries). */
int ilu0_dd_history(const ilu0dd_ctx* ctx, double* host_dst, int32_t n);

/* ---- inspection ------------------------------------------------------ */
#define ILU0DD_X_PART_ID 0   /* int32[N]   Algorithm 2 label per natural cell */
#define ILU0DD_X_PERM 1      /* int32[N]   perm[new] = old */
#define ILU0DD_X_IPERM 2     /* int32[N]   iperm[old] = new */
#define ILU0DD_X_PART_PTR 3  /* int32[nsub+1] row range of each subdomain */
#define ILU0DD_X_LEVEL_L 4   /* int32[N]   L level of each reordered row (local DAG) */
#define ILU0DD_X_LEVEL_U 5   /* int32[N]   U level of each reordered row */
#define ILU0DD_X_DD_ROW_PTR 6 /* int32[N+1] pattern of the dropped matrix */
#define ILU0DD_X_DD_COL 7    /* int32[kept] */
#define ILU0DD_X_L 8         /* double[kept*9]: L blocks at strictly-lower positions, 0 elsewhere */
#define ILU0DD_X_UT 9        /* double[kept*9]: U~ = D^-1 U at strictly-upper positions, 0 elsewhere */
#define ILU0DD_X_INVD 10     /* double[N*9]: D^-1 = U_ii^-1 per row */
#define ILU0DD_X_AP_ROW_PTR 11 /* int32[N+1] reordered full matrix */
#define ILU0DD_X_AP_COL 12   /* int32[nnzb] */
#define ILU0DD_X_STREAM 13   /* uint8[Q_STREAM_BYTES]: the packed factor stream (device copy) */
#define ILU0DD_X_SELL_COL 14 /* int32[sell slots * 32]: sliced-ELL columns of the SpMV matrix (device copy) */
#define ILU0DD_X_SELL_VAL 15 /* double[sell slots * 32 * 9]: sliced-ELL values (device copy) */

/* Copy one array to host memory (`bytes` must equal its size). Arrays
 * 4..10 need opts.keep_host = 1 at setup. */
int ilu0_dd_export(const ilu0dd_ctx* ctx, int what, void* host_dst, size_t bytes);

#define ILU0DD_Q_N 0              /* block rows */
#define ILU0DD_Q_NNZB 1           /* blocks of A */
#define ILU0DD_Q_KEPT 2           /* blocks kept after the drop */
#define ILU0DD_Q_NSUB 3           /* subdomains (= apply thread blocks) */
#define ILU0DD_Q_NL 4             /* strictly-lower blocks kept */
#define ILU0DD_Q_NU 5             /* strictly-upper blocks kept */
#define ILU0DD_Q_APPLY_BYTES 6    /* algorithmic bytes of one apply */
#define ILU0DD_Q_SPMV_BYTES 7     /* algorithmic bytes of one SpMV */
#define ILU0DD_Q_STREAM_BYTES 8   /* bytes of the packed factor stream */
#define ILU0DD_Q_THREADS 9        /* apply threads per block */
#define ILU0DD_Q_SMEM 10          /* apply dynamic shared memory per block */
#define ILU0DD_Q_PIECES 11        /* pieces (level slices of a subdomain), summed over subdomains */
#define ILU0DD_Q_CUDA_ERROR 12    /* last cudaError_t recorded by the context */
#define ILU0DD_Q_MAX_LEVELS 13    /* max over subdomains of L levels + U levels */
#define ILU0DD_Q_WORKSPACE 14     /* workspace bytes in use */
#define ILU0DD_Q_APPLY_KERNELS 15 /* kernel launches per apply (always 1) */
#define ILU0DD_Q_ITER_KERNELS 16  /* kernel launches per BiCGSTAB iteration */
#define ILU0DD_Q_SELL_SLOTS 17    /* slots of the sliced-ELL SpMV matrix (32 entries each) */
#define ILU0DD_Q_BLOCK_DIM 18     /* block dimension bs (3 or 1); vectors hold bs*N doubles */
#define ILU0DD_Q_ROW_THREAD 19    /* apply mapping: 1 one thread per 3x3 row (FP32/BF16 factors, no row
                                     with more than three blocks on either side), 0 three threads per
                                     3x3 row (or one per scalar row) */

int ilu0_dd_query(const ilu0dd_ctx* ctx, int what, int64_t* value);

/* Read (and clear) the device error word: 0, or the code of a bounded wait
 * that expired inside a kernel (1: an apply warp's wait for the previous
 * level, Section 4.4's level order). Synchronizes the device. */
int ilu0_dd_device_error(const ilu0dd_ctx* ctx, int32_t* code);

/* The apply's waits (Section 4.4: a warp starts a level's rows once the
 * previous level is done) are bounded. A warp waits for the previous level's
 * pieces at most `wait_us` microseconds (at the peak SM clock; 0 restores the
 * default, 100000 = 0.1 s); then the block stops waiting, sets the device
 * error word to 1 and finishes (its z values are then not valid), so the
 * kernel always returns. bicgstab_solve then returns ILU0DD_ERR_DEVICE_WAIT, and a
 * batched solve reports it for that system. stuck_piece >= 0 (a piece
 * index in [0, ILU0DD_Q_PIECES)) makes that piece's completion count
 * unreachable, so every wait on it expires: a failure-path test of the waits
 * that needs no GPU fault; -1 (the default) disables it. Host-side only
 * (takes effect at the context's next launch, and for batches created after
 * the call). Returns ILU0DD_ERR_INVALID for a null ctx or a piece out of
 * range. */
int ilu0dd_set_wait_limits(ilu0dd_ctx* ctx, uint32_t wait_us, int32_t stuck_piece);

/* Release the host-side context (the caller frees the workspace). */
void ilu0_dd_destroy(ilu0dd_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* ILU0DD_H_ */
