// The C ABI declared in include/ilu0dd.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ctx.h"
#include "setup_dev.h"

using namespace ilu0dd;


namespace {

int cuda_fail(ilu0dd_ctx* c, cudaError_t e, const char* what) {
  if (c) {
    c->last_cuda = e;
    c->why = std::string(what) + ": " + cudaGetErrorString(e);
    if (c->trace) std::fprintf(stderr, "[ilu0dd] %s\n", c->why.c_str());
  }
  return ILU0DD_ERR_CUDA;
}

// The apply's wait bound in SM cycles, from microseconds at the device's
// peak SM clock (a lower running clock only lengthens the bound).
cudaError_t set_wait_us(ilu0dd_ctx* c, uint32_t us) {
  int dev = 0, khz = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  if (e != cudaSuccess) return e;
  c->dev.sd.wait_cycles = (uint64_t)us * (uint64_t)(khz > 0 ? khz : 2000000) / 1000u;
  return cudaSuccess;
}

#define CK(ctx, call)                                    \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

ilu0dd_opts resolved(const ilu0dd_opts* o) {
  ilu0dd_opts r;
  ilu0dd_default_opts(&r);
  if (o) r = *o;
  if (r.maxit <= 0) r.maxit = 10000;
  if (!(r.rtol > 0.0)) r.rtol = 1e-8;
  if (r.check_every <= 0) r.check_every = 8;
  return r;
}

int max_smem_optin() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return 232448;  // sm_103 opt-in limit: lets the structural query run without a device
  }
  return v;
}

}  // namespace

namespace {

// The matrix arrays of ilu0dd_bsr may be host memory or device memory of the
// current device, each on its own (told apart by cudaPointerGetAttributes;
// without a device every pointer is host memory). The structural plan reads
// the pattern on the host, so device-resident row_ptr and col_idx are copied
// to host buffers first; device-resident values go straight to the device
// numeric setup and are copied to the host only for the host numeric setup.
bool device_resident(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice;
}

struct HostMatrix {
  ilu0dd_bsr bsr{};  // the caller's matrix with host pointers for what was copied
  std::vector<int32_t> rp, col;
  std::vector<double> val;
};

// Host view of A: the pattern always, the values when `values` is set.
int host_matrix(const ilu0dd_bsr* A, bool values, HostMatrix* h) {
  h->bsr = *A;
  if (A->n_brows < 0 || A->nnzb < 0) return ILU0DD_OK;  // make_plan reports it
  const size_t n1 = (size_t)A->n_brows + 1, nb = (size_t)A->nnzb;
  const int bs = A->block_dim == 1 ? 1 : 3;
  cudaError_t e = cudaSuccess;
  if (device_resident(A->row_ptr)) {
    h->rp.resize(n1);
    e = cudaMemcpy(h->rp.data(), A->row_ptr, sizeof(int32_t) * n1, cudaMemcpyDeviceToHost);
    h->bsr.row_ptr = h->rp.data();
  }
  if (e == cudaSuccess && nb && device_resident(A->col_idx)) {
    h->col.resize(nb);
    e = cudaMemcpy(h->col.data(), A->col_idx, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost);
    h->bsr.col_idx = h->col.data();
  }
  if (e == cudaSuccess && values && nb && device_resident(A->val)) {
    h->val.resize((size_t)bs * bs * nb);
    e = cudaMemcpy(h->val.data(), A->val, sizeof(double) * h->val.size(), cudaMemcpyDeviceToHost);
    h->bsr.val = h->val.data();
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ILU0DD_ERR_CUDA;
  }
  return ILU0DD_OK;
}

// The numeric half of setup (ILU0, ILDU0, packing, upload) for a context whose
// plan is in place. d_scratch != nullptr runs ILU0 and the packing on the
// device (setup_dev.cu); else on the host. Deletes the context on failure.
int setup_numeric(ilu0dd_ctx* c, const ilu0dd_bsr* A, const ilu0dd_opts& o, void* d_workspace, size_t ws_bytes,
                  void* d_scratch, size_t scratch_bytes, void* stream, double t0, ilu0dd_ctx** out) {
  Plan& p = c->plan;
  if (!d_workspace || ws_bytes < p.lay.total || (reinterpret_cast<uintptr_t>(d_workspace) & 255)) {
    delete c;
    return ILU0DD_ERR_WORKSPACE;
  }
  const double t1 = wall_seconds();
  const bool on_device = d_scratch != nullptr;
  int rc = ILU0DD_OK;
  int32_t bad = -1;
  std::vector<double> F, invD;
  std::vector<uint8_t> sbytes;
  std::vector<int32_t> sell_col;
  std::vector<double> sell_val;
  DeviceSetupResult dres;
  double t2 = t1, t3 = t1;
  if (on_device) {
    rc = setup_on_device(p, A->val, static_cast<unsigned char*>(d_scratch), scratch_bytes,
                         static_cast<unsigned char*>(d_workspace), reinterpret_cast<cudaStream_t>(stream), &dres);
    t2 = t3 = wall_seconds();
    if (rc == ILU0DD_ERR_CUDA) {
      int r = cuda_fail(c, dres.cuda, "device setup");
      delete c;
      return r;
    }
    if (rc) {
      if (rc == ILU0DD_ERR_ZERO_PIVOT) c->why = "zero pivot at reordered row " + std::to_string(dres.bad_row);
      else if (dres.range_bad) c->why = "a factor magnitude lies outside [2^-70, 2^100], the double-float range";
      else c->why = "device setup scratch too small or misaligned";
      if (c->trace) std::fprintf(stderr, "[ilu0dd] setup: %s\n", c->why.c_str());
      delete c;
      return rc;
    }
  } else {
    HostMatrix hv;  // the host numeric setup reads the values on the host
    if (host_matrix(A, true, &hv)) {
      c->why = "copy of the device-resident values to the host failed";
      delete c;
      return ILU0DD_ERR_CUDA;
    }
    A = &hv.bsr;
    rc = factor_ildu0(p, A->val, &F, &invD, &bad);
    if (rc) {
      if (c->trace) std::fprintf(stderr, "[ilu0dd] setup: zero pivot at reordered row %d\n", bad);
      delete c;
      return rc;
    }
    if (p.factor_prec == ILU0DD_DF64 && !df64_range_ok(F, invD)) {
      c->why = "a factor magnitude lies outside [2^-70, 2^100], the double-float range";
      if (c->trace) std::fprintf(stderr, "[ilu0dd] setup: %s\n", c->why.c_str());
      delete c;
      return ILU0DD_ERR_INVALID;
    }
    t2 = wall_seconds();
    pack_stream(p, F, invD, &sbytes);
    pack_sell(p, A->val, &sell_col, &sell_val);
    t3 = wall_seconds();
  }

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  c->ws = static_cast<unsigned char*>(d_workspace);
  c->ws_bytes = ws_bytes;
  c->rtol = o.rtol;
  c->maxit = o.maxit;
  c->check_every = o.check_every;
  c->use_graphs = o.use_graphs != 0;
  {
    auto up = [&](size_t off, const void* src, size_t bytes) -> cudaError_t {
      if (!bytes) return cudaSuccess;
      return cudaMemcpyAsync(c->ws + off, src, bytes, cudaMemcpyHostToDevice, s);
    };
    const Plan::Layout& L = p.lay;
    cudaError_t e = cudaGetDevice(&c->device);
    if (!on_device) {  // the device path wrote these already
      if (e == cudaSuccess) e = up(L.stream, sbytes.data(), sbytes.size());
      if (e == cudaSuccess) e = up(L.cta, p.cta.data(), sizeof(CtaDesc) * p.cta.size());
      if (e == cudaSuccess) e = up(L.pieces, p.pieces.data(), sizeof(PieceDesc) * p.pieces.size());
      if (e == cudaSuccess) e = up(L.sell_off, p.slice_off.data(), sizeof(int32_t) * p.slice_off.size());
      if (e == cudaSuccess) e = up(L.sell_col, sell_col.data(), sizeof(int32_t) * sell_col.size());
      if (e == cudaSuccess) e = up(L.sell_val, sell_val.data(), sizeof(double) * sell_val.size());
    }
    if (e == cudaSuccess) e = up(L.perm, p.perm.data(), sizeof(int32_t) * p.perm.size());
    if (e == cudaSuccess) e = up(L.iperm, p.iperm.data(), sizeof(int32_t) * p.iperm.size());
    if (e == cudaSuccess) e = up(L.row_l0, p.row_l0.data(), p.row_l0.size());
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.partials, 0, sizeof(double) * 5 * (size_t)p.ntiles_pow2, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.counters, 0, sizeof(uint32_t) * 16, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.scal, 0, sizeof(SolverScalars), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.err, 0, sizeof(int32_t) * 4, s);
    for (int v = 0; v < kNumVec && e == cudaSuccess; ++v)
      e = cudaMemsetAsync(c->ws + L.vec[v], 0, sizeof(double) * p.bs * (size_t)p.N, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host staging buffers die below
    if (e != cudaSuccess) {
      int r = cuda_fail(c, e, "setup upload");
      delete c;
      return r;
    }
    DevCtx& d = c->dev;
    SysDesc& S = d.sd;
    S.stream = c->ws + L.stream;
    S.cta = reinterpret_cast<const CtaDesc*>(c->ws + L.cta);
    S.pieces = reinterpret_cast<const PieceDesc*>(c->ws + L.pieces);
    S.nsub = p.nsub;
    S.prefetch_bytes = p.prefetch_bytes;
    S.vec_bytes = (int)(p.smem_bytes - kApplyTailSmem);
    S.wait_stuck = -1;
    S.row_thread = p.row_thread ? 1 : 0;
    S.slice_off = reinterpret_cast<const int32_t*>(c->ws + L.sell_off);
    S.sell_col = reinterpret_cast<const int32_t*>(c->ws + L.sell_col);
    S.sell_val = reinterpret_cast<const double*>(c->ws + L.sell_val);
    S.nslices = p.nslices;
    S.perm = reinterpret_cast<const int32_t*>(c->ws + L.perm);
    S.row_l0 = c->ws + L.row_l0;
    S.iperm = reinterpret_cast<const int32_t*>(c->ws + L.iperm);
    S.N = p.N;
    S.ntiles = p.ntiles;
    S.ntiles_pow2 = p.ntiles_pow2;
    for (int v = 0; v < kNumVec; ++v) S.vec[v] = reinterpret_cast<double*>(c->ws + L.vec[v]);
    S.partials = reinterpret_cast<double*>(c->ws + L.partials);
    S.counters = reinterpret_cast<uint32_t*>(c->ws + L.counters);
    S.scal = reinterpret_cast<SolverScalars*>(c->ws + L.scal);
    S.hist = reinterpret_cast<double*>(c->ws + L.hist);
    S.err = reinterpret_cast<int32_t*>(c->ws + L.err);
    d.threads = p.threads;
    d.factor_prec = o.factor_prec;
    d.smem_bytes = p.smem_bytes;
    d.smem_rowsync = p.smem_rowsync;
    d.bs = p.bs;
    d.traversal = o.traversal;
    e = apply_configure(d);
    if (e == cudaSuccess) e = set_wait_us(c, kApplyWaitUs);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      int r = cuda_fail(c, e, "setup configure");
      if (c->own) cudaStreamDestroy(c->own);
      delete c;
      return r;
    }
  }
  if (o.keep_host) {
    if (on_device) {  // the host copies the ILDU0 post-processing exactly as factor_ildu0 does
      const int64_t kept = p.dd_rp[p.N];
      std::vector<double> W((size_t)p.bs * p.bs * (size_t)kept);
      invD.resize((size_t)p.bs * p.bs * (size_t)p.N);
      cudaError_t e = cudaMemcpy(W.data(), dres.w, sizeof(double) * W.size(), cudaMemcpyDeviceToHost);
      if (e == cudaSuccess)
        e = cudaMemcpy(invD.data(), dres.invd, sizeof(double) * invD.size(), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        int r = cuda_fail(c, e, "setup keep_host download");
        delete c;
        return r;
      }
      ildu0_from_w(p, W, invD, &F);
    }
    c->F.swap(F);
    c->invD.swap(invD);
    c->have_factors = true;
  }
  const double t4 = wall_seconds();
  c->setup_s = t4 - t0;
  if (c->trace)
    std::fprintf(stderr,
                 "[ilu0dd] setup (%s): plan %.3fs factor %.3fs pack %.3fs upload %.3fs; N=%d nsub=%d pieces=%lld "
                 "threads=%d smem=%zu stream=%lld B\n",
                 on_device ? "device" : "host", t1 - t0, t2 - t1, t3 - t2, t4 - t3, p.N, p.nsub,
                 (long long)p.n_pieces, p.threads,
                 p.smem_bytes, (long long)p.stream_bytes);
  *out = c;
  return ILU0DD_OK;
}

}  // namespace

extern "C" {

int ilu0dd_default_opts(ilu0dd_opts* o) {
  if (!o) return ILU0DD_ERR_INVALID;
  std::memset(o, 0, sizeof *o);
  o->factor_prec = ILU0DD_F64;
  o->threads_per_cta = 0;
  o->prefetch_bytes = 0;
  o->maxit = 10000;
  o->rtol = 1e-8;
  o->check_every = 8;
  o->use_graphs = 1;
  o->keep_host = 0;
  const char* tr = std::getenv("ILU0DD_TRACE");  // per-phase timings without recompiling the caller
  o->trace = tr && std::atoi(tr) > 0 ? 1 : 0;
  return ILU0DD_OK;
}

const char* ilu0dd_strerror(int code) {
  switch (code) {
    case ILU0DD_OK: return "ok";
    case ILU0DD_ERR_INVALID: return "invalid argument or matrix pattern";
    case ILU0DD_ERR_ZERO_PIVOT: return "singular or non-finite pivot block in ILU0";
    case ILU0DD_ERR_SMEM: return "subdomain does not fit in shared memory";
    case ILU0DD_ERR_CUDA: return "CUDA error";
    case ILU0DD_ERR_BREAKDOWN: return "BiCGSTAB breakdown";
    case ILU0DD_ERR_NOT_CONVERGED: return "BiCGSTAB did not converge";
    case ILU0DD_ERR_NONFINITE: return "non-finite input";
    case ILU0DD_ERR_WORKSPACE: return "workspace too small or misaligned";
    case ILU0DD_ERR_DEVICE_WAIT: return "device-side bounded wait expired";
    default: return "unknown error code";
  }
}

int ilu0_dd_workspace_size(const ilu0dd_bsr* A, const ilu0dd_geom* geom, const ilu0dd_opts* opts,
                           size_t* bytes) {
  if (!A || !geom || !bytes) return ILU0DD_ERR_INVALID;
  ilu0dd_opts o = resolved(opts);
  Plan p;
  std::string why;
  HostMatrix hv;
  if (host_matrix(A, false, &hv)) return ILU0DD_ERR_CUDA;
  int rc = make_plan(&hv.bsr, geom, &o, max_smem_optin(), &p, &why);
  if (rc) {
    if (o.trace) std::fprintf(stderr, "[ilu0dd] workspace_size: %s\n", why.c_str());
    return rc;
  }
  *bytes = p.lay.total;
  return ILU0DD_OK;
}

int ilu0_dd_setup(const ilu0dd_bsr* A, const ilu0dd_geom* geom, const ilu0dd_opts* opts, void* d_workspace,
                  size_t ws_bytes, void* stream, ilu0dd_ctx** out) {
  if (!A || !geom || !out) return ILU0DD_ERR_INVALID;
  *out = nullptr;
  const double t0 = wall_seconds();
  ilu0dd_opts o = resolved(opts);
  ilu0dd_ctx* c = new (std::nothrow) ilu0dd_ctx();
  if (!c) return ILU0DD_ERR_INVALID;
  c->trace = o.trace != 0;
  HostMatrix hv;
  if (host_matrix(A, false, &hv)) {
    delete c;
    return ILU0DD_ERR_CUDA;
  }
  int rc = make_plan(&hv.bsr, geom, &o, max_smem_optin(), &c->plan, &c->why);
  if (rc) {
    if (c->trace) std::fprintf(stderr, "[ilu0dd] setup: %s\n", c->why.c_str());
    delete c;
    return rc;
  }
  return setup_numeric(c, A, o, d_workspace, ws_bytes, nullptr, 0, stream, t0, out);
}

int ilu0dd_plan_create(const ilu0dd_bsr* A, const ilu0dd_geom* geom, const ilu0dd_opts* opts, ilu0dd_plan** out,
                       size_t* workspace_bytes, size_t* scratch_bytes) {
  if (!A || !geom || !out) return ILU0DD_ERR_INVALID;
  *out = nullptr;
  ilu0dd_plan* pl = new (std::nothrow) ilu0dd_plan();
  if (!pl) return ILU0DD_ERR_INVALID;
  pl->t0 = wall_seconds();
  pl->opts = resolved(opts);
  HostMatrix hv;
  if (host_matrix(A, false, &hv)) {
    delete pl;
    return ILU0DD_ERR_CUDA;
  }
  int rc = make_plan(&hv.bsr, geom, &pl->opts, max_smem_optin(), &pl->plan, &pl->why);
  if (rc) {
    if (pl->opts.trace) std::fprintf(stderr, "[ilu0dd] plan: %s\n", pl->why.c_str());
    delete pl;
    return rc;
  }
  pl->scratch_bytes = device_setup_scratch_bytes(pl->plan);
  if (workspace_bytes) *workspace_bytes = pl->plan.lay.total;
  if (scratch_bytes) *scratch_bytes = pl->scratch_bytes;
  *out = pl;
  return ILU0DD_OK;
}

int ilu0dd_plan_create_partitioned(const ilu0dd_bsr* A, const int32_t* part_id, int32_t nparts,
                                   const ilu0dd_opts* opts, ilu0dd_plan** out, size_t* workspace_bytes,
                                   size_t* scratch_bytes) {
  if (!A || !out || (A->n_brows > 0 && !part_id)) return ILU0DD_ERR_INVALID;
  *out = nullptr;
  ilu0dd_plan* pl = new (std::nothrow) ilu0dd_plan();
  if (!pl) return ILU0DD_ERR_INVALID;
  pl->t0 = wall_seconds();
  pl->opts = resolved(opts);
  HostMatrix hv;
  if (host_matrix(A, false, &hv)) {
    delete pl;
    return ILU0DD_ERR_CUDA;
  }
  int rc = make_plan(&hv.bsr, nullptr, &pl->opts, max_smem_optin(), &pl->plan, &pl->why, part_id, nparts);
  if (rc) {
    if (pl->opts.trace) std::fprintf(stderr, "[ilu0dd] plan: %s\n", pl->why.c_str());
    delete pl;
    return rc;
  }
  pl->scratch_bytes = device_setup_scratch_bytes(pl->plan);
  if (workspace_bytes) *workspace_bytes = pl->plan.lay.total;
  if (scratch_bytes) *scratch_bytes = pl->scratch_bytes;
  *out = pl;
  return ILU0DD_OK;
}

int ilu0dd_partition_bfs(const ilu0dd_bsr* A, int32_t part_rows, int32_t* part_id, int32_t* nparts) {
  if (!A) return ILU0DD_ERR_INVALID;
  HostMatrix hv;
  if (host_matrix(A, false, &hv)) return ILU0DD_ERR_CUDA;
  return partition_bfs(&hv.bsr, part_rows, part_id, nparts);
}

int ilu0_dd_setup_planned(ilu0dd_plan* plan, const ilu0dd_bsr* A, void* d_workspace, size_t ws_bytes,
                          void* d_scratch, size_t scratch_bytes, void* stream, ilu0dd_ctx** out) {
  if (!plan || !A || !out || plan->consumed) return ILU0DD_ERR_INVALID;
  *out = nullptr;
  if (A->n_brows != plan->plan.N || A->nnzb != plan->plan.nnzb || (plan->plan.nnzb > 0 && !A->val))
    return ILU0DD_ERR_INVALID;
  ilu0dd_ctx* c = new (std::nothrow) ilu0dd_ctx();
  if (!c) return ILU0DD_ERR_INVALID;
  c->trace = plan->opts.trace != 0;
  c->plan = std::move(plan->plan);
  plan->consumed = true;
  return setup_numeric(c, A, plan->opts, d_workspace, ws_bytes, d_scratch, scratch_bytes, stream, plan->t0, out);
}

int ilu0dd_plan_destroy(ilu0dd_plan* plan) {
  delete plan;
  return ILU0DD_OK;
}

int ilu0_dd_apply(const ilu0dd_ctx* ctx, const double* d_r, double* d_z, void* stream) {
  if (!ctx || (ctx->plan.N > 0 && (!d_r || !d_z))) return ILU0DD_ERR_INVALID;
  const size_t n = (size_t)ctx->plan.bs * (size_t)ctx->plan.N * sizeof(double);
  const char* r = reinterpret_cast<const char*>(d_r);
  const char* z = reinterpret_cast<const char*>(d_z);
  if (r < z + n && z < r + n) return ILU0DD_ERR_INVALID;  // overlapping vectors
  cudaError_t e = launch_apply(ctx->dev, kModePlain, d_r, d_z, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(const_cast<ilu0dd_ctx*>(ctx), e, "apply launch");
  return ILU0DD_OK;
}

int ilu0_dd_apply_host(ilu0dd_ctx* ctx, const double* h_r, double* h_z, void* stream) {
  if (!ctx || (ctx->plan.N > 0 && (!h_r || !h_z))) return ILU0DD_ERR_INVALID;
  const Plan& p = ctx->plan;
  if (p.N == 0) return ILU0DD_OK;
  constexpr int kChunks = 16;
  const int nch = std::min(kChunks, p.nsub);
  if ((int)ctx->hstreams.size() != nch) {
    for (cudaStream_t x : ctx->hstreams) cudaStreamDestroy(x);
    for (cudaEvent_t x : ctx->hevents) cudaEventDestroy(x);
    ctx->hstreams.assign(nch, nullptr);
    ctx->hevents.assign(nch + 1, nullptr);
    for (int i = 0; i < nch; ++i) CK(ctx, cudaStreamCreateWithFlags(&ctx->hstreams[i], cudaStreamNonBlocking));
    for (int i = 0; i <= nch; ++i) CK(ctx, cudaEventCreateWithFlags(&ctx->hevents[i], cudaEventDisableTiming));
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // staging: the solver's s and t vectors (not in use outside bicgstab_* calls)
  double* dr = ctx->dev.sd.vec[kVecS];
  double* dz = ctx->dev.sd.vec[kVecT];
  CK(ctx, cudaEventRecord(ctx->hevents[0], s));  // after the caller's earlier work
  for (int i = 0; i < nch; ++i) {
    const int s0 = (int)((int64_t)p.nsub * i / nch), s1 = (int)((int64_t)p.nsub * (i + 1) / nch);
    const size_t r0 = (size_t)p.bs * p.part_ptr[s0], r1 = (size_t)p.bs * p.part_ptr[s1];
    cudaStream_t cs = ctx->hstreams[i];
    CK(ctx, cudaStreamWaitEvent(cs, ctx->hevents[0], 0));
    CK(ctx, cudaMemcpyAsync(dr + r0, h_r + r0, sizeof(double) * (r1 - r0), cudaMemcpyHostToDevice, cs));
    CK(ctx, launch_apply_range(ctx->dev, kModePlain, dr, dz, s0, s1 - s0, cs));
    CK(ctx, cudaMemcpyAsync(h_z + r0, dz + r0, sizeof(double) * (r1 - r0), cudaMemcpyDeviceToHost, cs));
    CK(ctx, cudaEventRecord(ctx->hevents[1 + i], cs));
  }
  for (int i = 0; i < nch; ++i) CK(ctx, cudaStreamWaitEvent(s, ctx->hevents[1 + i], 0));
  return ILU0DD_OK;
}

int ilu0_dd_apply_rowsync(const ilu0dd_ctx* ctx, const double* d_r, double* d_z, void* stream) {
  if (!ctx || (ctx->plan.N > 0 && (!d_r || !d_z))) return ILU0DD_ERR_INVALID;
  const size_t n = (size_t)ctx->plan.bs * (size_t)ctx->plan.N * sizeof(double);
  const char* r = reinterpret_cast<const char*>(d_r);
  const char* z = reinterpret_cast<const char*>(d_z);
  if (r < z + n && z < r + n) return ILU0DD_ERR_INVALID;  // overlapping vectors
  if (ctx->plan.N > 0 && ctx->dev.smem_rowsync == 0) return ILU0DD_ERR_SMEM;
  cudaError_t e = launch_apply_rowsync(ctx->dev, d_r, d_z, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(const_cast<ilu0dd_ctx*>(ctx), e, "row-flag apply launch");
  return ILU0DD_OK;
}

int ilu0_dd_apply_global_vector(const ilu0dd_ctx* ctx, const double* d_r, double* d_z, void* stream) {
  if (!ctx || (ctx->plan.N > 0 && (!d_r || !d_z)) || ctx->dev.factor_prec != ILU0DD_F64) return ILU0DD_ERR_INVALID;
  const size_t n = (size_t)ctx->plan.bs * (size_t)ctx->plan.N * sizeof(double);
  const char* r = reinterpret_cast<const char*>(d_r);
  const char* z = reinterpret_cast<const char*>(d_z);
  if (r < z + n && z < r + n) return ILU0DD_ERR_INVALID;  // overlapping vectors
  cudaError_t e = launch_apply_vglobal(ctx->dev, d_r, d_z, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(const_cast<ilu0dd_ctx*>(ctx), e, "global-vector apply launch");
  return ILU0DD_OK;
}

int ilu0_dd_apply_edge(const ilu0dd_ctx* ctx, const double* d_r, double* d_z, void* stream) {
  if (!ctx || (ctx->plan.N > 0 && (!d_r || !d_z)) || ctx->dev.factor_prec == ILU0DD_DF64) return ILU0DD_ERR_INVALID;
  const size_t n = (size_t)ctx->plan.bs * (size_t)ctx->plan.N * sizeof(double);
  const char* r = reinterpret_cast<const char*>(d_r);
  const char* z = reinterpret_cast<const char*>(d_z);
  if (r < z + n && z < r + n) return ILU0DD_ERR_INVALID;  // overlapping vectors
  cudaError_t e = launch_apply_edge(ctx->dev, d_r, d_z, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(const_cast<ilu0dd_ctx*>(ctx), e, "edge-centric apply launch");
  return ILU0DD_OK;
}

int ilu0dd_levels_device(const int32_t* d_row_ptr, const int32_t* d_col, const int32_t* d_part_ptr, int32_t nsub,
                         int32_t* d_lev_l, int32_t* d_lev_u, int32_t* d_nlev_l, int32_t* d_nlev_u, void* stream) {
  if (nsub < 0 || (nsub > 0 && (!d_row_ptr || !d_col || !d_part_ptr || !d_lev_l || !d_lev_u)))
    return ILU0DD_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = launch_levels(d_row_ptr, d_col, d_part_ptr, nsub, 0, d_lev_l, d_nlev_l, s);
  if (e == cudaSuccess) e = launch_levels(d_row_ptr, d_col, d_part_ptr, nsub, 1, d_lev_u, d_nlev_u, s);
  return e == cudaSuccess ? ILU0DD_OK : ILU0DD_ERR_CUDA;
}

int ilu0_dd_apply_unfused(const ilu0dd_ctx* ctx, const double* d_r, double* d_z, void* stream) {
  if (!ctx || (ctx->plan.N > 0 && (!d_r || !d_z))) return ILU0DD_ERR_INVALID;
  const size_t n = (size_t)ctx->plan.bs * (size_t)ctx->plan.N * sizeof(double);
  const char* r = reinterpret_cast<const char*>(d_r);
  const char* z = reinterpret_cast<const char*>(d_z);
  if (r < z + n && z < r + n) return ILU0DD_ERR_INVALID;  // overlapping vectors
  cudaError_t e = launch_apply_unfused(ctx->dev, d_r, d_z, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(const_cast<ilu0dd_ctx*>(ctx), e, "unfused apply launch");
  return ILU0DD_OK;
}

int ilu0_dd_spmv(const ilu0dd_ctx* ctx, const double* d_x, double* d_y, void* stream) {
  if (!ctx || (ctx->plan.N > 0 && (!d_x || !d_y || d_x == d_y))) return ILU0DD_ERR_INVALID;
  cudaError_t e = launch_spmv(ctx->dev, 0, d_x, d_y, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(const_cast<ilu0dd_ctx*>(ctx), e, "spmv launch");
  return ILU0DD_OK;
}

int ilu0_dd_dot(const ilu0dd_ctx* ctx, const double* d_x, const double* d_y, double* d_result, void* stream) {
  if (!ctx || !d_result || (ctx->plan.N > 0 && (!d_x || !d_y))) return ILU0DD_ERR_INVALID;
  cudaError_t e = launch_dot(ctx->dev, d_x, d_y, d_result, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(const_cast<ilu0dd_ctx*>(ctx), e, "dot launch");
  return ILU0DD_OK;
}

int ilu0_dd_permute(const ilu0dd_ctx* ctx, const double* d_in, double* d_out, int dir, void* stream) {
  if (!ctx || (dir != 0 && dir != 1) || (ctx->plan.N > 0 && (!d_in || !d_out || d_in == d_out)))
    return ILU0DD_ERR_INVALID;
  cudaError_t e = launch_permute(ctx->dev, d_in, d_out, dir, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(const_cast<ilu0dd_ctx*>(ctx), e, "permute launch");
  return ILU0DD_OK;
}

}  // extern "C"

namespace {

// One BiCGSTAB iteration of Algorithm 1 as five launches.
cudaError_t launch_iteration(const DevCtx& d, cudaStream_t s) {
  cudaError_t e;
  // p = r + beta (p - omega v); ph = M^-1 p
  if ((e = launch_apply(d, kModeP, d.sd.vec[kVecR], d.sd.vec[kVecPh], s)) != cudaSuccess) return e;
  // v = A ph; alpha = rho / (rh . v)
  if ((e = launch_spmv(d, 1, d.sd.vec[kVecPh], d.sd.vec[kVecV], s)) != cudaSuccess) return e;
  // s = r - alpha v; sh = M^-1 s
  if ((e = launch_apply(d, kModeS, d.sd.vec[kVecR], d.sd.vec[kVecSh], s)) != cudaSuccess) return e;
  // t = A sh; omega = (t . s) / (t . t)
  if ((e = launch_spmv(d, 2, d.sd.vec[kVecSh], d.sd.vec[kVecT], s)) != cudaSuccess) return e;
  // x += alpha ph + omega sh; r = s - omega t; convergence; beta
  return launch_update(d, s);
}

cudaError_t run_chunk(ilu0dd_ctx* c) {
  const DevCtx& d = c->dev;
  if (!c->use_graphs) {
    for (int i = 0; i < c->check_every; ++i) {
      cudaError_t e = launch_iteration(d, c->own);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (!c->graph) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->own, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < c->check_every && e == cudaSuccess; ++i) e = launch_iteration(d, c->own);
    cudaError_t e2 = cudaStreamEndCapture(c->own, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    c->graph_iters = c->check_every;
  }
  return cudaGraphLaunch(c->graph, c->own);
}

// The solver scalars and the device error word (an apply wait that expired).
cudaError_t read_scalars(ilu0dd_ctx* c, SolverScalars* h, int32_t* derr) {
  cudaError_t e = cudaMemcpyAsync(h, c->dev.sd.scal, sizeof *h, cudaMemcpyDeviceToHost, c->own);
  if (e == cudaSuccess) e = cudaMemcpyAsync(derr, c->dev.sd.err, sizeof *derr, cudaMemcpyDeviceToHost, c->own);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->own);
  return e;
}

}  // namespace

extern "C" {

int bicgstab_solve(ilu0dd_ctx* c, const double* d_b, double* d_x, ilu0dd_info* info, void* stream) {
  if (!c || (c->plan.N > 0 && (!d_b || !d_x))) return ILU0DD_ERR_INVALID;
  const double t0 = wall_seconds();
  const DevCtx& d = c->dev;
  cudaStream_t us = reinterpret_cast<cudaStream_t>(stream);
  SolverScalars h{};
  int32_t derr = 0;
  int status = ILU0DD_OK, restarts = 0;
  CK(c, cudaStreamSynchronize(us));
  if (c->plan.N == 0) {
    if (info) {
      std::memset(info, 0, sizeof *info);
      info->setup_s = c->setup_s;
    }
    return ILU0DD_OK;
  }
  CK(c, launch_permute(d, d_b, d.sd.vec[kVecB], 0, c->own));
  CK(c, launch_init(d, c->rtol, c->maxit, c->own));
  CK(c, read_scalars(c, &h, &derr));
  if (h.status == ILU0DD_ERR_NONFINITE) status = ILU0DD_ERR_NONFINITE;
  while (status == ILU0DD_OK && !h.converged) {
    while (!h.done && !derr) {
      CK(c, run_chunk(c));
      CK(c, read_scalars(c, &h, &derr));
    }
    if (derr) break;  // an apply wait expired: the iterates are not valid
    if (h.status != ILU0DD_OK) {
      status = h.status;
      break;
    }
    // true residual r = b - A x
    CK(c, launch_spmv(d, 0, d.sd.vec[kVecX], d.sd.vec[kVecT], c->own));
    CK(c, launch_residual(d, 0, c->own));
    CK(c, read_scalars(c, &h, &derr));
    if (h.rel_true < c->rtol) break;
    if (restarts == 0) {
      restarts = 1;
      CK(c, launch_residual(d, 1, c->own));
      CK(c, read_scalars(c, &h, &derr));
      continue;
    }
    status = ILU0DD_ERR_NOT_CONVERGED;
    break;
  }
  // a device wait that expired poisons the result, whatever else was seen
  CK(c, cudaMemcpyAsync(&derr, d.sd.err, sizeof derr, cudaMemcpyDeviceToHost, c->own));
  CK(c, launch_permute(d, d.sd.vec[kVecX], d_x, 1, c->own));
  CK(c, cudaStreamSynchronize(c->own));
  if (derr) status = ILU0DD_ERR_DEVICE_WAIT;
  c->last_iterations = h.iter;
  if (info) {
    info->status = status;
    info->iterations = h.iter;
    info->restarts = restarts;
    info->reserved = 0;
    info->rel_res_recurrence = h.rel;
    info->rel_res_true = h.rel_true;
    info->setup_s = c->setup_s;
    info->solve_s = wall_seconds() - t0;
  }
  if (c->trace)
    std::fprintf(stderr, "[ilu0dd] solve: status=%d iterations=%d restarts=%d rel=%.3e true=%.3e %.4fs\n", status,
                 h.iter, restarts, h.rel, h.rel_true, wall_seconds() - t0);
  return status;
}

int bicgstab_start(ilu0dd_ctx* c, const double* d_b, void* stream) {
  if (!c || (c->plan.N > 0 && !d_b)) return ILU0DD_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CK(c, launch_permute(c->dev, d_b, c->dev.sd.vec[kVecB], 0, s));
  CK(c, launch_init(c->dev, c->rtol, c->maxit, s));
  return ILU0DD_OK;
}

int bicgstab_iterate(ilu0dd_ctx* c, int32_t n, float* host_kernel_ms, void* stream) {
  if (!c || n < 0) return ILU0DD_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const DevCtx& d = c->dev;
  if (!host_kernel_ms) {
    for (int32_t i = 0; i < n; ++i) CK(c, launch_iteration(d, s));
    return ILU0DD_OK;
  }
  const size_t need = 5 * (size_t)n + 1;
  while (c->events.size() < need) {
    cudaEvent_t e;
    CK(c, cudaEventCreate(&e));
    c->events.push_back(e);
  }
  size_t k = 0;
  CK(c, cudaEventRecord(c->events[k++], s));
  for (int32_t i = 0; i < n; ++i) {
    CK(c, launch_apply(d, kModeP, d.sd.vec[kVecR], d.sd.vec[kVecPh], s));
    CK(c, cudaEventRecord(c->events[k++], s));
    CK(c, launch_spmv(d, 1, d.sd.vec[kVecPh], d.sd.vec[kVecV], s));
    CK(c, cudaEventRecord(c->events[k++], s));
    CK(c, launch_apply(d, kModeS, d.sd.vec[kVecR], d.sd.vec[kVecSh], s));
    CK(c, cudaEventRecord(c->events[k++], s));
    CK(c, launch_spmv(d, 2, d.sd.vec[kVecSh], d.sd.vec[kVecT], s));
    CK(c, cudaEventRecord(c->events[k++], s));
    CK(c, launch_update(d, s));
    CK(c, cudaEventRecord(c->events[k++], s));
  }
  CK(c, cudaStreamSynchronize(s));
  for (size_t j = 0; j + 1 < k; ++j) CK(c, cudaEventElapsedTime(&host_kernel_ms[j], c->events[j], c->events[j + 1]));
  return ILU0DD_OK;
}

int bicgstab_state(ilu0dd_ctx* c, ilu0dd_info* info, void* stream) {
  if (!c || !info) return ILU0DD_ERR_INVALID;
  SolverScalars h{};
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CK(c, cudaMemcpyAsync(&h, c->dev.sd.scal, sizeof h, cudaMemcpyDeviceToHost, s));
  CK(c, cudaStreamSynchronize(s));
  std::memset(info, 0, sizeof *info);
  info->status = h.status;
  info->iterations = h.iter;
  info->rel_res_recurrence = h.rel;
  info->rel_res_true = 1.0;
  info->setup_s = c->setup_s;
  return ILU0DD_OK;
}

int ilu0_dd_history(const ilu0dd_ctx* c, double* host_dst, int32_t n) {
  if (!c || !host_dst || n < 0) return ILU0DD_ERR_INVALID;
  int32_t m = std::min(n, c->last_iterations + 1);
  if (m <= 0) return ILU0DD_OK;
  cudaError_t e = cudaMemcpy(host_dst, c->dev.sd.hist, sizeof(double) * (size_t)m, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(const_cast<ilu0dd_ctx*>(c), e, "history copy");
  return ILU0DD_OK;
}

int ilu0_dd_export(const ilu0dd_ctx* c, int what, void* dst, size_t bytes) {
  if (!c || !dst) return ILU0DD_ERR_INVALID;
  const Plan& p = c->plan;
  auto put = [&](const void* src, size_t n) {
    if (n != bytes) return ILU0DD_ERR_INVALID;
    if (n) std::memcpy(dst, src, n);
    return ILU0DD_OK;
  };
  const size_t kept = (size_t)p.dd_rp[p.N];
  switch (what) {
    case ILU0DD_X_PART_ID: return put(p.part_id.data(), 4 * p.part_id.size());
    case ILU0DD_X_PERM: return put(p.perm.data(), 4 * p.perm.size());
    case ILU0DD_X_IPERM: return put(p.iperm.data(), 4 * p.iperm.size());
    case ILU0DD_X_PART_PTR: return put(p.part_ptr.data(), 4 * p.part_ptr.size());
    case ILU0DD_X_LEVEL_L: return put(p.lev_l.data(), 4 * p.lev_l.size());
    case ILU0DD_X_LEVEL_U: return put(p.lev_u.data(), 4 * p.lev_u.size());
    case ILU0DD_X_DD_ROW_PTR: return put(p.dd_rp.data(), 4 * p.dd_rp.size());
    case ILU0DD_X_DD_COL: return put(p.dd_col.data(), 4 * p.dd_col.size());
    case ILU0DD_X_AP_ROW_PTR: return put(p.ap_rp.data(), 4 * p.ap_rp.size());
    case ILU0DD_X_AP_COL: return put(p.ap_col.data(), 4 * p.ap_col.size());
    case ILU0DD_X_STREAM:
    case ILU0DD_X_SELL_COL:
    case ILU0DD_X_SELL_VAL: {  // device copies, read back
      size_t off = p.lay.stream, n = (size_t)p.stream_bytes;
      if (what == ILU0DD_X_SELL_COL) off = p.lay.sell_col, n = sizeof(int32_t) * (size_t)p.sell_slots * kSlice;
      if (what == ILU0DD_X_SELL_VAL)
        off = p.lay.sell_val, n = sizeof(double) * p.bs * p.bs * (size_t)p.sell_slots * kSlice;
      if (n != bytes) return ILU0DD_ERR_INVALID;
      if (!n) return ILU0DD_OK;
      cudaError_t e = cudaMemcpy(dst, c->ws + off, n, cudaMemcpyDeviceToHost);
      return e == cudaSuccess ? ILU0DD_OK : ILU0DD_ERR_CUDA;
    }
    case ILU0DD_X_INVD:
      if (!c->have_factors) return ILU0DD_ERR_INVALID;
      return put(c->invD.data(), 8 * c->invD.size());
    case ILU0DD_X_L:
    case ILU0DD_X_UT: {
      const size_t bb = (size_t)p.bs * p.bs;
      if (!c->have_factors || bytes != 8 * bb * kept) return ILU0DD_ERR_INVALID;
      double* o = static_cast<double*>(dst);
      for (int32_t i = 0; i < p.N; ++i)
        for (int64_t q = p.dd_rp[i]; q < p.dd_rp[i + 1]; ++q) {
          const bool take = what == ILU0DD_X_L ? p.dd_col[q] < i : p.dd_col[q] > i;
          for (size_t e = 0; e < bb; ++e) o[bb * q + e] = take ? c->F[bb * (size_t)q + e] : 0.0;
        }
      return ILU0DD_OK;
    }
    default: return ILU0DD_ERR_INVALID;
  }
}

int ilu0_dd_query(const ilu0dd_ctx* c, int what, int64_t* v) {
  if (!c || !v) return ILU0DD_ERR_INVALID;
  const Plan& p = c->plan;
  switch (what) {
    case ILU0DD_Q_N: *v = p.N; break;
    case ILU0DD_Q_NNZB: *v = p.nnzb; break;
    case ILU0DD_Q_KEPT: *v = p.dd_rp[p.N]; break;
    case ILU0DD_Q_NSUB: *v = p.nsub; break;
    case ILU0DD_Q_NL: *v = p.nL; break;
    case ILU0DD_Q_NU: *v = p.nU; break;
    case ILU0DD_Q_APPLY_BYTES: *v = p.apply_bytes; break;
    case ILU0DD_Q_SPMV_BYTES: *v = p.spmv_bytes; break;
    case ILU0DD_Q_STREAM_BYTES: *v = p.stream_bytes; break;
    case ILU0DD_Q_THREADS: *v = p.threads; break;
    case ILU0DD_Q_SMEM: *v = (int64_t)p.smem_bytes; break;
    case ILU0DD_Q_PIECES: *v = p.n_pieces; break;
    case ILU0DD_Q_CUDA_ERROR: *v = (int64_t)c->last_cuda; break;
    case ILU0DD_Q_MAX_LEVELS: *v = p.max_levels; break;
    case ILU0DD_Q_WORKSPACE: *v = (int64_t)p.lay.total; break;
    case ILU0DD_Q_APPLY_KERNELS: *v = 1; break;
    case ILU0DD_Q_ITER_KERNELS: *v = 5; break;
    case ILU0DD_Q_SELL_SLOTS: *v = p.sell_slots; break;
    case ILU0DD_Q_BLOCK_DIM: *v = p.bs; break;
    case ILU0DD_Q_ROW_THREAD: *v = p.row_thread ? 1 : 0; break;
    default: return ILU0DD_ERR_INVALID;
  }
  return ILU0DD_OK;
}

int ilu0dd_set_wait_limits(ilu0dd_ctx* c, uint32_t wait_us, int32_t stuck_piece) {
  if (!c || stuck_piece < -1 || (stuck_piece >= 0 && stuck_piece >= c->plan.n_pieces)) return ILU0DD_ERR_INVALID;
  if (cudaError_t e = set_wait_us(c, wait_us ? wait_us : kApplyWaitUs); e != cudaSuccess)
    return cuda_fail(c, e, "wait limits");
  c->dev.sd.wait_stuck = stuck_piece;
  if (c->graph) {  // captured launches hold the old kernel parameters
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return ILU0DD_OK;
}

int ilu0_dd_device_error(const ilu0dd_ctx* c, int32_t* code) {
  if (!c || !code) return ILU0DD_ERR_INVALID;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(code, c->dev.sd.err, sizeof *code, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(c->dev.sd.err, 0, sizeof *code);
  if (e != cudaSuccess) return cuda_fail(const_cast<ilu0dd_ctx*>(c), e, "device error read");
  return ILU0DD_OK;
}

void ilu0_dd_destroy(ilu0dd_ctx* c) {
  if (!c) return;
  for (cudaEvent_t e : c->events) cudaEventDestroy(e);
  for (cudaStream_t x : c->hstreams) cudaStreamDestroy(x);
  for (cudaEvent_t e : c->hevents) cudaEventDestroy(e);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->own) cudaStreamDestroy(c->own);
  delete c;
}

}  // extern "C"
