// Batched BiCGSTAB over many independent systems (C ABI in include/ilu0dd.h).
//
// Every step of an iteration is ONE launch for all systems: the fused apply
// walks the (system, subdomain) items of every system, the SpMV, update and
// vector kernels walk their (system, 256-row tile) items; each system keeps
// its own scalars and reductions in its own context workspace, and a system
// whose solve has finished is skipped by every later launch. Iterations are
// captured as CUDA graphs of opts.check_every iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "ctx.h"

struct ilu0dd_batch {
  std::vector<ilu0dd_ctx*> ctxs;
  int32_t nsys = 0;
  unsigned char* ws = nullptr;
  SysDesc* d_sys = nullptr;
  BatchItem* d_apply_items = nullptr;
  BatchItem* d_tile_items = nullptr;
  const double** d_ptrs = nullptr;  // [nsys] b pointers, then [nsys] x pointers
  SolverScalars* d_status = nullptr;
  int32_t* d_flags = nullptr;
  int64_t n_apply = 0, n_tile = 0;
  int factor_prec = 0, bs = 3, threads = 0;
  int row_thread = 0;  // the systems' stream layout (SysDesc.row_thread, the same for all)
  size_t smem = 0;
  int grid_apply = 1, grid_tile = 1;
  double rtol = 1e-8;
  int32_t maxit = 10000;
  int check_every = 8;
  bool use_graphs = true;
  cudaStream_t own = nullptr;
  cudaGraphExec_t graph = nullptr;
  std::vector<SolverScalars> h_status;
};

namespace {

inline size_t align256(size_t v) { return (v + 255) / 256 * 256; }

struct BatchLayout {
  size_t sys, apply_items, tile_items, ptrs, status, flags, total;
};

BatchLayout batch_layout(ilu0dd_ctx* const* ctxs, int32_t nsys, int64_t* n_apply, int64_t* n_tile) {
  int64_t na = 0, nt = 0;
  for (int32_t i = 0; i < nsys; ++i) {
    na += ctxs[i]->plan.nsub;
    nt += ctxs[i]->plan.ntiles;
  }
  BatchLayout L{};
  size_t cur = 0;
  auto take = [&](size_t bytes) {
    size_t at = cur;
    cur = align256(cur + bytes);
    return at;
  };
  L.sys = take(sizeof(SysDesc) * (size_t)nsys);
  L.apply_items = take(sizeof(BatchItem) * (size_t)std::max<int64_t>(1, na));
  L.tile_items = take(sizeof(BatchItem) * (size_t)std::max<int64_t>(1, nt));
  L.ptrs = take(sizeof(double*) * 2 * (size_t)nsys);
  L.status = take(sizeof(SolverScalars) * (size_t)nsys);
  L.flags = take(sizeof(int32_t) * (size_t)nsys);
  L.total = cur;
  if (n_apply) *n_apply = na;
  if (n_tile) *n_tile = nt;
  return L;
}

cudaError_t batch_iteration(const ilu0dd_batch* b, cudaStream_t s) {
  cudaError_t e;
  if ((e = launch_apply_batched(b->d_sys, b->d_apply_items, b->n_apply, kModeP, b->factor_prec, b->bs, b->row_thread,
                                b->threads, b->smem, b->grid_apply, s)) != cudaSuccess)
    return e;
  if ((e = launch_spmv_batched(b->d_sys, b->d_tile_items, b->n_tile, 1, b->bs, b->grid_tile, s)) != cudaSuccess)
    return e;
  if ((e = launch_apply_batched(b->d_sys, b->d_apply_items, b->n_apply, kModeS, b->factor_prec, b->bs, b->row_thread,
                                b->threads, b->smem, b->grid_apply, s)) != cudaSuccess)
    return e;
  if ((e = launch_spmv_batched(b->d_sys, b->d_tile_items, b->n_tile, 2, b->bs, b->grid_tile, s)) != cudaSuccess)
    return e;
  return launch_update_batched(b->d_sys, b->d_tile_items, b->n_tile, b->bs, b->grid_tile, s);
}

cudaError_t batch_chunk(ilu0dd_batch* b) {
  if (!b->use_graphs) {
    for (int i = 0; i < b->check_every; ++i) {
      cudaError_t e = batch_iteration(b, b->own);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (!b->graph) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < b->check_every && e == cudaSuccess; ++i) e = batch_iteration(b, b->own);
    cudaError_t e2 = cudaStreamEndCapture(b->own, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
  }
  return cudaGraphLaunch(b->graph, b->own);
}

cudaError_t read_status(ilu0dd_batch* b) {
  cudaError_t e = launch_gather_status(b->d_sys, b->nsys, b->d_status, b->own);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->h_status.data(), b->d_status, sizeof(SolverScalars) * (size_t)b->nsys,
                        cudaMemcpyDeviceToHost, b->own);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->own);
  return e;
}

}  // namespace

extern "C" {

int ilu0dd_batch_workspace_size(ilu0dd_ctx* const* ctxs, int32_t nsys, size_t* bytes) {
  if (!ctxs || nsys <= 0 || !bytes) return ILU0DD_ERR_INVALID;
  for (int32_t i = 0; i < nsys; ++i)
    if (!ctxs[i]) return ILU0DD_ERR_INVALID;
  *bytes = batch_layout(ctxs, nsys, nullptr, nullptr).total;
  return ILU0DD_OK;
}

int ilu0dd_batch_create(ilu0dd_ctx* const* ctxs, int32_t nsys, const ilu0dd_opts* opts, void* d_workspace,
                        size_t ws_bytes, void* stream, ilu0dd_batch** out) {
  if (!ctxs || nsys <= 0 || !out) return ILU0DD_ERR_INVALID;
  *out = nullptr;
  for (int32_t i = 0; i < nsys; ++i)
    if (!ctxs[i] || ctxs[i]->dev.factor_prec != ctxs[0]->dev.factor_prec || ctxs[i]->device != ctxs[0]->device ||
        ctxs[i]->dev.bs != ctxs[0]->dev.bs || ctxs[i]->dev.sd.row_thread != ctxs[0]->dev.sd.row_thread)
      return ILU0DD_ERR_INVALID;  // one device, factor precision, block dimension and apply mapping per batch
  int64_t na = 0, nt = 0;
  const BatchLayout L = batch_layout(ctxs, nsys, &na, &nt);
  if (!d_workspace || ws_bytes < L.total || (reinterpret_cast<uintptr_t>(d_workspace) & 255))
    return ILU0DD_ERR_WORKSPACE;
  ilu0dd_batch* b = new (std::nothrow) ilu0dd_batch();
  if (!b) return ILU0DD_ERR_INVALID;
  b->ctxs.assign(ctxs, ctxs + nsys);
  b->nsys = nsys;
  b->ws = static_cast<unsigned char*>(d_workspace);
  b->d_sys = reinterpret_cast<SysDesc*>(b->ws + L.sys);
  b->d_apply_items = reinterpret_cast<BatchItem*>(b->ws + L.apply_items);
  b->d_tile_items = reinterpret_cast<BatchItem*>(b->ws + L.tile_items);
  b->d_ptrs = reinterpret_cast<const double**>(b->ws + L.ptrs);
  b->d_status = reinterpret_cast<SolverScalars*>(b->ws + L.status);
  b->d_flags = reinterpret_cast<int32_t*>(b->ws + L.flags);
  b->n_apply = na;
  b->n_tile = nt;
  b->factor_prec = ctxs[0]->dev.factor_prec;
  b->bs = ctxs[0]->dev.bs;
  b->row_thread = ctxs[0]->dev.sd.row_thread;
  ilu0dd_opts o;
  ilu0dd_default_opts(&o);
  if (opts) o = *opts;
  b->rtol = o.rtol > 0.0 ? o.rtol : 1e-8;
  b->maxit = o.maxit > 0 ? o.maxit : 10000;
  b->check_every = o.check_every > 0 ? o.check_every : 8;
  b->use_graphs = o.use_graphs != 0;
  std::vector<SysDesc> sys(nsys);
  std::vector<BatchItem> ai, ti;
  ai.reserve(na);
  ti.reserve(nt);
  for (int32_t i = 0; i < nsys; ++i) {
    const DevCtx& d = ctxs[i]->dev;
    sys[i] = d.sd;
    b->threads = std::max(b->threads, d.threads);
    b->smem = std::max(b->smem, d.smem_bytes);
    // a system's residual history must hold the batch's iteration limit
    if (ctxs[i]->maxit < b->maxit) b->maxit = ctxs[i]->maxit;
  }
  // interleave the systems' items so that each part of the persistent grid
  // sees a mix of systems
  int64_t left = na;
  std::vector<int32_t> next(nsys, 0);
  while (left > 0)
    for (int32_t i = 0; i < nsys; ++i)
      if (next[i] < ctxs[i]->plan.nsub) {
        ai.push_back(BatchItem{i, next[i]++});
        --left;
      }
  for (int32_t i = 0; i < nsys; ++i)
    for (int64_t t = 0; t < ctxs[i]->plan.ntiles; ++t) ti.push_back(BatchItem{i, (int32_t)t});
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(b->d_sys, sys.data(), sizeof(SysDesc) * sys.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !ai.empty())
    e = cudaMemcpyAsync(b->d_apply_items, ai.data(), sizeof(BatchItem) * ai.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !ti.empty())
    e = cudaMemcpyAsync(b->d_tile_items, ti.data(), sizeof(BatchItem) * ti.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int dev = 0, nsm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    if (b->own) cudaStreamDestroy(b->own);
    delete b;
    return ILU0DD_ERR_CUDA;
  }
  b->grid_apply = (int)std::min<int64_t>(std::max<int64_t>(1, na),
                                         (int64_t)nsm * apply_blocks_per_sm(b->factor_prec, b->bs, b->row_thread, b->threads, b->smem));
  b->grid_tile = (int)std::min<int64_t>(std::max<int64_t>(1, nt), (int64_t)nsm * tile_blocks_per_sm(b->bs));
  b->h_status.resize(nsys);
  *out = b;
  return ILU0DD_OK;
}

int bicgstab_solve_batched(ilu0dd_batch* b, const double* const* d_b, double* const* d_x, ilu0dd_info* infos,
                           void* stream) {
  if (!b || !d_b || !d_x) return ILU0DD_ERR_INVALID;
  for (int32_t i = 0; i < b->nsys; ++i)
    if (b->ctxs[i]->plan.N > 0 && (!d_b[i] || !d_x[i])) return ILU0DD_ERR_INVALID;
  const double t0 = wall_seconds();
  const int32_t n = b->nsys;
  std::vector<const double*> ptrs(2 * (size_t)n);
  for (int32_t i = 0; i < n; ++i) {
    ptrs[i] = d_b[i];
    ptrs[n + i] = d_x[i];
  }
  std::vector<int32_t> restarts(n, 0), flags(n, 0);
  auto fail = [&](cudaError_t) { return ILU0DD_ERR_CUDA; };
  cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  // A system with no rows has no work items, so no kernel ever sets its
  // scalars: it is finished from the start (x empty, residual 0), as
  // bicgstab_solve reports it.
  SolverScalars empty{};
  empty.done = 1;
  empty.converged = 1;
  for (int32_t i = 0; i < n && e == cudaSuccess; ++i)
    if (b->ctxs[i]->plan.N == 0)
      e = cudaMemcpyAsync(b->ctxs[i]->dev.sd.scal, &empty, sizeof empty, cudaMemcpyHostToDevice, b->own);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_ptrs, ptrs.data(), sizeof(double*) * ptrs.size(), cudaMemcpyHostToDevice, b->own);
  if (e == cudaSuccess) e = launch_permute_batched(b->d_sys, b->d_tile_items, b->n_tile, b->d_ptrs, 0, b->bs, b->grid_tile,
                                                 b->own);
  if (e == cudaSuccess)
    e = launch_vec_batched(b->d_sys, b->d_tile_items, b->n_tile, 0, b->rtol, b->maxit, nullptr, b->bs, b->grid_tile,
                           b->own);
  if (e == cudaSuccess) e = read_status(b);
  if (e != cudaSuccess) return fail(e);
  for (;;) {
    auto all_done = [&]() {
      for (int32_t i = 0; i < n; ++i)
        if (!b->h_status[i].done) return false;
      return true;
    };
    while (!all_done()) {
      if ((e = batch_chunk(b)) != cudaSuccess || (e = read_status(b)) != cudaSuccess) return fail(e);
    }
    // true residual r = b - A x of every system
    e = launch_spmv_batched(b->d_sys, b->d_tile_items, b->n_tile, 0, b->bs, b->grid_tile, b->own);
    if (e == cudaSuccess)
      e = launch_vec_batched(b->d_sys, b->d_tile_items, b->n_tile, 1, 0.0, 0, nullptr, b->bs, b->grid_tile, b->own);
    if (e == cudaSuccess) e = read_status(b);
    if (e != cudaSuccess) return fail(e);
    // restart once the systems that converged on the recurrence only
    bool any = false;
    for (int32_t i = 0; i < n; ++i) {
      const SolverScalars& h = b->h_status[i];
      flags[i] = h.converged && h.status == ILU0DD_OK && !(h.rel_true < b->rtol) && restarts[i] == 0;
      if (flags[i]) {
        restarts[i] = 1;
        any = true;
      }
    }
    if (!any) break;
    e = cudaMemcpyAsync(b->d_flags, flags.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, b->own);
    if (e == cudaSuccess)
      e = launch_vec_batched(b->d_sys, b->d_tile_items, b->n_tile, 2, 0.0, 0, b->d_flags, b->bs, b->grid_tile,
                             b->own);
    if (e == cudaSuccess) e = read_status(b);
    if (e != cudaSuccess) return fail(e);
  }
  e = launch_permute_batched(b->d_sys, b->d_tile_items, b->n_tile, b->d_ptrs + n, 1, b->bs, b->grid_tile, b->own);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->own);
  if (e != cudaSuccess) return fail(e);
  const double solve_s = wall_seconds() - t0;
  int worst = ILU0DD_OK;
  for (int32_t i = 0; i < n; ++i) {
    const SolverScalars& h = b->h_status[i];
    int st = h.status;
    if (st == ILU0DD_OK && !(h.rel_true < b->rtol)) st = ILU0DD_ERR_NOT_CONVERGED;
    if (st != ILU0DD_OK && worst == ILU0DD_OK) worst = st;
    b->ctxs[i]->last_iterations = h.iter;
    if (infos) {
      ilu0dd_info& f = infos[i];
      std::memset(&f, 0, sizeof f);
      f.status = st;
      f.iterations = h.iter;
      f.restarts = restarts[i];
      f.rel_res_recurrence = h.rel;
      f.rel_res_true = h.rel_true;
      f.setup_s = b->ctxs[i]->setup_s;
      f.solve_s = solve_s;
    }
  }
  return worst;
}

void ilu0dd_batch_destroy(ilu0dd_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->own) cudaStreamDestroy(b->own);
  delete b;
}

}  // extern "C"
