// sm_103a kernels of the hot path:
//  - ildu0_apply: fused L -> D^-1 -> U~ sweep, one thread block per subdomain
//    (Sections 4.2-4.4), subdomain vector in shared memory, factor records
//    streamed through a ring of bulk copies (cp.async.bulk + mbarrier),
//    vertex-centric rows (Section 4.2.3: one thread per block row, fixed
//    per-row order, deterministic);
//  - sell_spmv: y = A_p x on a sliced-ELL copy (coalesced, entry-major),
//    with the dot products of Algorithm 1 fused into the epilogue;
//  - update / init / residual / dot / permute: the BiCGSTAB vector steps.
// Dot products use one fixed order (per-row FMA, halving sums over 256-row
// tiles and over tiles); the last block of each reduction kernel finishes the
// sum and updates the device-resident scalars, so no scalar goes to the host
// inside an iteration.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.h"

namespace ilu0dd {

// ---------------------------------------------------------------------------
// Fused ILDU0 apply
// ---------------------------------------------------------------------------
struct ApplyArgs {
  const unsigned char* stream;
  const CtaDesc* cta;
  const PieceDesc* pieces;
  const double* r;
  double* z;
  double* p;        // mode P: search direction, updated in place
  double* s;        // mode S: s = r - alpha v (written)
  const double* v;
  const SolverScalars* scal;
  int32_t* err;
  int ring_bytes, chunk_bytes, nslot, vec_bytes;
};

template <typename TF>
__device__ __forceinline__ typename FactorLoad<TF>::compute ring_factor(const unsigned char* ring, uint32_t mask,
                                                                         uint32_t off) {
  return FactorLoad<TF>::get(ring + (off & mask));
}

__device__ __forceinline__ uint32_t ring_u16(const unsigned char* ring, uint32_t mask, uint32_t off) {
  return *reinterpret_cast<const uint16_t*>(ring + (off & mask));
}

template <typename TF, int MODE>
__global__ void __launch_bounds__(kMaxApplyThreads) ildu0_apply_kernel(ApplyArgs a) {
  using TV = typename FactorLoad<TF>::compute;
  constexpr uint32_t FE = sizeof(TF);
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxSlots];
  __shared__ int abort_flag;

  if (MODE != kModePlain && a.scal->done) return;
  const CtaDesc cd = a.cta[blockIdx.x];
  const int tid = threadIdx.x;
  TV* y = reinterpret_cast<TV*>(smem);
  unsigned char* ring = smem + a.vec_bytes;
  const unsigned char* gsrc = a.stream + cd.stream_off;
  const uint32_t CH = (uint32_t)a.chunk_bytes;
  const uint32_t mask = (uint32_t)a.ring_bytes - 1u;
  const int nslot = a.nslot;
  const int nchunks = (int)((cd.stream_len + CH - 1) / CH);

  auto issue = [&](int c) {
    const int slot = c % nslot;
    const uint32_t bytes = min(CH, (uint32_t)cd.stream_len - (uint32_t)c * CH);
    mbar_arrive_expect_tx(&bars[slot], bytes);
    bulk_g2s(ring + (uint32_t)slot * CH, gsrc + (size_t)c * CH, bytes, &bars[slot]);
  };

  if (tid == 0) {
    for (int i = 0; i < nslot; ++i) mbar_init(&bars[i], 1);
    mbar_fence_init();
    abort_flag = 0;
  }
  __syncthreads();
  int issued = 0;  // tracked by thread 0
  if (tid == 0)
    for (; issued < nchunks && issued < nslot; ++issued) issue(issued);

  // subdomain vector -> shared memory (with the fused BiCGSTAB update)
  const int64_t base = 3ll * cd.row0;
  const int nv = 3 * cd.nrows;
  double alpha = 0.0, beta = 0.0, omega = 0.0;
  if (MODE == kModeP) { beta = a.scal->beta; omega = a.scal->omega; }
  if (MODE == kModeS) alpha = a.scal->alpha;
  for (int e = tid; e < nv; e += blockDim.x) {
    double val;
    if (MODE == kModePlain) {
      val = a.r[base + e];
    } else if (MODE == kModeP) {
      val = fma(beta, fma(-omega, a.v[base + e], a.p[base + e]), a.r[base + e]);
      a.p[base + e] = val;
    } else {
      val = fma(-alpha, a.v[base + e], a.r[base + e]);
      a.s[base + e] = val;
    }
    y[e] = (TV)val;
  }
  __syncthreads();

  PieceDesc nxt = cd.npieces > 0 ? a.pieces[cd.piece0] : PieceDesc{0, 0, 0, 0};
  for (int k = 0; k < cd.npieces; ++k) {
    const PieceDesc pd = nxt;
    if (k + 1 < cd.npieces) nxt = a.pieces[cd.piece0 + k + 1];
    const int n = (int)(pd.meta & 0xFFFFu);
    const int w = (int)((pd.meta >> 16) & 0xFFu);
    const int kind = (int)(pd.meta >> 24);
    const uint32_t beg = pd.off;
    const uint32_t vend = pd.voff + ((kind ? 9u * (uint32_t)n : 0u) + 9u * pd.nb) * FE;
    const uint32_t end = beg + ((vend + 15u) & ~15u);
    const int c_first = (int)(beg / CH), c_last = (int)((end - 1) / CH);
    if (tid == 0) {
      const int lim = c_first + nslot;
      for (; issued < nchunks && issued < lim; ++issued) issue(issued);
    }
    if (tid < n) {
      bool ok = true;
      for (int c = c_first; c <= c_last; ++c)
        ok &= mbar_wait_bounded(&bars[c % nslot], (uint32_t)((c / nslot) & 1));
      if (!ok) {
        abort_flag = 1;
        atomicOr(a.err, kDevErrWaitExpired);
      } else {
        const uint32_t rb = beg;  // record base in stream bytes
        const int row = (int)ring_u16(ring, mask, rb + 2u * (uint32_t)(w + tid));
        TV acc0 = y[3 * row], acc1 = y[3 * row + 1], acc2 = y[3 * row + 2];
        uint32_t vb = rb + pd.voff;
        if (kind) {
          // D^-1 (Section 4.3): w_i = D_i^-1 y_i before the U~ updates
          TV d[9];
#pragma unroll
          for (int e = 0; e < 9; ++e) d[e] = ring_factor<TF>(ring, mask, vb + ((uint32_t)(e * n + tid)) * FE);
          TV t0 = d[0] * acc0, t1 = d[3] * acc0, t2 = d[6] * acc0;
          t0 = fma(d[1], acc1, t0);
          t1 = fma(d[4], acc1, t1);
          t2 = fma(d[7], acc1, t2);
          t0 = fma(d[2], acc2, t0);
          t1 = fma(d[5], acc2, t1);
          t2 = fma(d[8], acc2, t2);
          acc0 = t0;
          acc1 = t1;
          acc2 = t2;
          vb += 9u * (uint32_t)n * FE;
        }
        const uint32_t cb = rb + 2u * (uint32_t)(w + n);
        uint32_t c0 = 0;
        for (int sl = 0; sl < w; ++sl) {
          const uint32_t cs = ring_u16(ring, mask, rb + 2u * (uint32_t)sl);
          if ((uint32_t)tid >= cs) break;
          const int col = (int)ring_u16(ring, mask, cb + 2u * (c0 + (uint32_t)tid));
          const uint32_t vo = vb + 9u * c0 * FE + (uint32_t)tid * FE;
          TV b[9];
#pragma unroll
          for (int e = 0; e < 9; ++e) b[e] = ring_factor<TF>(ring, mask, vo + (uint32_t)e * cs * FE);
          const TV x0 = y[3 * col], x1 = y[3 * col + 1], x2 = y[3 * col + 2];
          acc0 = fma(-b[0], x0, acc0);
          acc1 = fma(-b[3], x0, acc1);
          acc2 = fma(-b[6], x0, acc2);
          acc0 = fma(-b[1], x1, acc0);
          acc1 = fma(-b[4], x1, acc1);
          acc2 = fma(-b[7], x1, acc2);
          acc0 = fma(-b[2], x2, acc0);
          acc1 = fma(-b[5], x2, acc1);
          acc2 = fma(-b[8], x2, acc2);
          c0 += cs;
        }
        y[3 * row] = acc0;
        y[3 * row + 1] = acc1;
        y[3 * row + 2] = acc2;
      }
    }
    __syncthreads();
    if (abort_flag) break;
  }
  if (abort_flag) {
    // drain copies still in flight (bounded) before the block exits
    // (only the last nslot issued chunks can be pending; each is the latest use of its slot)
    if (tid == 0)
      for (int c = max(0, issued - nslot); c < issued; ++c)
        mbar_wait_bounded(&bars[c % nslot], (uint32_t)((c / nslot) & 1));
    return;
  }
  for (int e = tid; e < nv; e += blockDim.x) a.z[base + e] = (double)y[e];
}

template <typename TF, int MODE>
static cudaError_t configure_one(size_t smem) {
  return cudaFuncSetAttribute(ildu0_apply_kernel<TF, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

// The attribute is a per-kernel permission shared by every context in the
// process, so it is raised once to the device's opt-in maximum; each launch
// still requests only its own context's shared memory.
cudaError_t apply_configure(const DevCtx& d) {
  (void)d;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)optin - kApplyStaticSmem;
  auto acc = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  acc(configure_one<double, kModePlain>(smem));
  acc(configure_one<double, kModeP>(smem));
  acc(configure_one<double, kModeS>(smem));
  acc(configure_one<float, kModePlain>(smem));
  acc(configure_one<float, kModeP>(smem));
  acc(configure_one<float, kModeS>(smem));
  acc(configure_one<bf16s, kModePlain>(smem));
  acc(configure_one<bf16s, kModeP>(smem));
  acc(configure_one<bf16s, kModeS>(smem));
  return e;
}

template <typename TF>
static cudaError_t launch_apply_t(const DevCtx& d, int mode, const ApplyArgs& a, cudaStream_t s) {
  dim3 grid(d.nsub), block(d.threads);
  if (mode == kModePlain)
    ildu0_apply_kernel<TF, kModePlain><<<grid, block, d.smem_bytes, s>>>(a);
  else if (mode == kModeP)
    ildu0_apply_kernel<TF, kModeP><<<grid, block, d.smem_bytes, s>>>(a);
  else
    ildu0_apply_kernel<TF, kModeS><<<grid, block, d.smem_bytes, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_apply(const DevCtx& d, int mode, const double* r, double* z, cudaStream_t s) {
  if (d.nsub == 0) return cudaSuccess;
  ApplyArgs a;
  a.stream = d.stream;
  a.cta = d.cta;
  a.pieces = d.pieces;
  a.r = r;
  a.z = z;
  a.p = d.vec[kVecP];
  a.s = d.vec[kVecS];
  a.v = d.vec[kVecV];
  a.scal = d.scal;
  a.err = d.err;
  a.ring_bytes = d.ring_bytes;
  a.chunk_bytes = d.chunk_bytes;
  a.nslot = d.nslot;
  a.vec_bytes = d.vec_bytes;
  if (d.factor_prec == ILU0DD_F64) return launch_apply_t<double>(d, mode, a, s);
  if (d.factor_prec == ILU0DD_F32) return launch_apply_t<float>(d, mode, a, s);
  return launch_apply_t<bf16s>(d, mode, a, s);
}

// ---------------------------------------------------------------------------
// Reductions: last-block completion
// ---------------------------------------------------------------------------

// Write this tile's partials; returns true in every thread of the block that
// arrived last (it then owns the final reduction).
template <int NV>
__device__ __forceinline__ bool publish_partials(const double (&q)[NV], double* partials, int64_t stride,
                                                 uint32_t* counter) {
  __shared__ unsigned int s_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) partials[v * stride + blockIdx.x] = q[v];
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    s_last = prev == gridDim.x - 1;
  }
  __syncthreads();
  const bool last = s_last != 0;
  if (last) __threadfence();
  return last;
}

template <int NV>
__device__ __forceinline__ void finish_sum(double* partials, int64_t stride, int64_t m, double (&out)[NV],
                                           double (*buf)[kDotTile]) {
  const double* part[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) part[v] = partials + v * stride;
  final_halving_sum<NV>(part, m, out, buf);
}

__device__ __forceinline__ double row_dot(const double* x, const double* y, int64_t i) {
  return fma(x[3 * i + 2], y[3 * i + 2], fma(x[3 * i + 1], y[3 * i + 1], x[3 * i] * y[3 * i]));
}

__device__ __forceinline__ bool finite(double v) { return isfinite(v); }

// ---------------------------------------------------------------------------
// SpMV (sliced ELL), kinds: 0 plain, 1 (rh . v) -> alpha, 2 (t . s), (t . t) -> omega
// ---------------------------------------------------------------------------
struct SpmvArgs {
  const int32_t* slice_off;
  const int32_t* cols;
  const double* vals;
  int64_t nslices;
  int32_t N;
  const double* x;
  double* y;
  const double* w;       // kind 1: rh, kind 2: s
  double* partials;
  int64_t stride, m;
  uint32_t* counter;
  SolverScalars* scal;
};

template <int KIND>
__global__ void __launch_bounds__(kDotTile) sell_spmv_kernel(SpmvArgs a) {
  if (KIND != 0 && a.scal->done) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t slice = (int64_t)blockIdx.x * (kDotTile / kSlice) + warp;
  const int64_t row = slice * kSlice + lane;
  double y0 = 0.0, y1 = 0.0, y2 = 0.0;
  if (slice < a.nslices) {
    const int64_t so = a.slice_off[slice];
    const int w = a.slice_off[slice + 1] - (int32_t)so;
    const int32_t* cp = a.cols + so * kSlice + lane;
    const double* vp = a.vals + so * 9 * kSlice + lane;
    for (int sl = 0; sl < w; ++sl) {
      const int c = __ldg(cp + sl * kSlice);
      double b[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) b[e] = __ldg(vp + (sl * 9 + e) * kSlice);
      const double x0 = a.x[3ll * c], x1 = a.x[3ll * c + 1], x2 = a.x[3ll * c + 2];
      y0 = fma(b[0], x0, y0);
      y1 = fma(b[3], x0, y1);
      y2 = fma(b[6], x0, y2);
      y0 = fma(b[1], x1, y0);
      y1 = fma(b[4], x1, y1);
      y2 = fma(b[7], x1, y2);
      y0 = fma(b[2], x2, y0);
      y1 = fma(b[5], x2, y1);
      y2 = fma(b[8], x2, y2);
    }
    if (row < a.N) {
      a.y[3 * row] = y0;
      a.y[3 * row + 1] = y1;
      a.y[3 * row + 2] = y2;
    }
  }
  if (KIND == 0) return;
  __shared__ double buf[2][kDotTile];
  const bool in = row < a.N;
  if (KIND == 1) {
    double q[1] = {in ? fma(a.w[3 * row + 2], y2, fma(a.w[3 * row + 1], y1, a.w[3 * row] * y0)) : 0.0};
    tile_halving_sum<1>(q, buf);
    if (!publish_partials<1>(q, a.partials, a.stride, a.counter)) return;
    double out[1];
    finish_sum<1>(a.partials, a.stride, a.m, out, buf);
    if (threadIdx.x == 0) {
      SolverScalars* S = a.scal;
      const double rv = out[0];
      S->rv = rv;
      if (rv == 0.0 || !finite(rv)) {
        S->status = ILU0DD_ERR_BREAKDOWN;
        S->done = 1;
      } else {
        S->alpha = S->rho / rv;
      }
      *a.counter = 0;
    }
  } else {
    // (t . s) and (t . t), t = y
    double q[2] = {in ? fma(y2, a.w[3 * row + 2], fma(y1, a.w[3 * row + 1], y0 * a.w[3 * row])) : 0.0,
                   in ? fma(y2, y2, fma(y1, y1, y0 * y0)) : 0.0};
    tile_halving_sum<2>(q, buf);
    if (!publish_partials<2>(q, a.partials, a.stride, a.counter)) return;
    double out[2];
    finish_sum<2>(a.partials, a.stride, a.m, out, buf);
    if (threadIdx.x == 0) {
      SolverScalars* S = a.scal;
      S->ts = out[0];
      S->tt = out[1];
      S->omega = out[1] == 0.0 ? 0.0 : out[0] / out[1];
      *a.counter = 0;
    }
  }
}

cudaError_t launch_spmv(const DevCtx& d, int kind, const double* x, double* y, cudaStream_t s) {
  if (d.N == 0) return cudaSuccess;
  SpmvArgs a;
  a.slice_off = d.slice_off;
  a.cols = d.sell_col;
  a.vals = d.sell_val;
  a.nslices = d.nslices;
  a.N = d.N;
  a.x = x;
  a.y = y;
  a.w = kind == 1 ? d.vec[kVecRh] : d.vec[kVecS];
  a.partials = d.partials;
  a.stride = d.ntiles_pow2;
  a.m = d.ntiles_pow2;
  a.counter = d.counters + (kind == 1 ? kCntSpmvV : kCntSpmvT);
  a.scal = d.scal;
  dim3 grid((unsigned)d.ntiles), block(kDotTile);
  if (kind == 0)
    sell_spmv_kernel<0><<<grid, block, 0, s>>>(a);
  else if (kind == 1)
    sell_spmv_kernel<1><<<grid, block, 0, s>>>(a);
  else
    sell_spmv_kernel<2><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Vector steps
// ---------------------------------------------------------------------------
struct VecArgs {
  double* v[kNumVec];
  int32_t N;
  double* partials;
  int64_t stride, m;
  uint32_t* counters;
  SolverScalars* scal;
  double* hist;
  double rtol;
  int32_t maxit;
  int restart;
};

// x += alpha ph + omega sh; r = s - omega t; then ||r||/||b|| and rho.
__global__ void __launch_bounds__(kDotTile) update_kernel(VecArgs a) {
  SolverScalars* S = a.scal;
  if (S->done) return;
  const int64_t i = (int64_t)blockIdx.x * kDotTile + threadIdx.x;
  const double alpha = S->alpha, omega = S->omega;
  double q[2] = {0.0, 0.0};
  if (i < a.N) {
    double* x = a.v[kVecX];
    double* r = a.v[kVecR];
    const double* ph = a.v[kVecPh];
    const double* sh = a.v[kVecSh];
    const double* sv = a.v[kVecS];
    const double* t = a.v[kVecT];
    const double* rh = a.v[kVecRh];
    double rr[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int64_t e = 3 * i + c;
      x[e] = fma(omega, sh[e], fma(alpha, ph[e], x[e]));
      rr[c] = fma(-omega, t[e], sv[e]);
      r[e] = rr[c];
    }
    q[0] = fma(rr[2], rr[2], fma(rr[1], rr[1], rr[0] * rr[0]));
    q[1] = fma(rh[3 * i + 2], rr[2], fma(rh[3 * i + 1], rr[1], rh[3 * i] * rr[0]));
  }
  __shared__ double buf[2][kDotTile];
  tile_halving_sum<2>(q, buf);
  uint32_t* counter = a.counters + kCntUpdate;
  if (!publish_partials<2>(q, a.partials, a.stride, counter)) return;
  double out[2];
  finish_sum<2>(a.partials, a.stride, a.m, out, buf);
  if (threadIdx.x == 0) {
    const double rr = out[0], rho_new = out[1];
    const double rel = sqrt(rr) / sqrt(S->bb);
    S->rr = rr;
    S->rhr = rho_new;
    S->rel = rel;
    S->iter += 1;
    if (S->iter <= S->maxit) a.hist[S->iter] = rel;
    if (!finite(rel)) {
      S->status = ILU0DD_ERR_BREAKDOWN;
      S->done = 1;
    } else if (rel < S->rtol) {
      S->converged = 1;
      S->done = 1;
    } else if (S->iter >= S->maxit) {
      S->status = ILU0DD_ERR_NOT_CONVERGED;
      S->done = 1;
    } else if (rho_new == 0.0 || omega == 0.0 || !finite(rho_new)) {
      S->status = ILU0DD_ERR_BREAKDOWN;
      S->done = 1;
    } else {
      S->beta = (alpha / omega) * (rho_new / S->rho);
      S->rho = rho_new;
    }
    *counter = 0;
  }
}

cudaError_t launch_update(const DevCtx& d, cudaStream_t s) {
  if (d.N == 0) return cudaSuccess;
  VecArgs a{};
  for (int v = 0; v < kNumVec; ++v) a.v[v] = d.vec[v];
  a.N = d.N;
  a.partials = d.partials;
  a.stride = d.ntiles_pow2;
  a.m = d.ntiles_pow2;
  a.counters = d.counters;
  a.scal = d.scal;
  a.hist = d.hist;
  update_kernel<<<(unsigned)d.ntiles, kDotTile, 0, s>>>(a);
  return cudaGetLastError();
}

// x = 0, r = rh = p = b, v = 0; bb = rho = (b . b).
__global__ void __launch_bounds__(kDotTile) init_kernel(VecArgs a) {
  const int64_t i = (int64_t)blockIdx.x * kDotTile + threadIdx.x;
  double q[1] = {0.0};
  if (i < a.N) {
    const double* b = a.v[kVecB];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int64_t e = 3 * i + c;
      const double be = b[e];
      a.v[kVecX][e] = 0.0;
      a.v[kVecR][e] = be;
      a.v[kVecRh][e] = be;
      a.v[kVecP][e] = be;
      a.v[kVecV][e] = 0.0;
    }
    q[0] = row_dot(b, b, i);
  }
  __shared__ double buf[1][kDotTile];
  tile_halving_sum<1>(q, buf);
  uint32_t* counter = a.counters + kCntInit;
  if (!publish_partials<1>(q, a.partials, a.stride, counter)) return;
  double out[1];
  finish_sum<1>(a.partials, a.stride, a.m, out, buf);
  if (threadIdx.x == 0) {
    SolverScalars* S = a.scal;
    const double bb = out[0];
    S->bb = bb;
    S->rho = bb;
    S->alpha = S->beta = S->omega = 0.0;
    S->rv = S->ts = S->tt = S->rr = S->rhr = 0.0;
    S->rel = 1.0;
    S->rel_true = 1.0;
    S->rtol = a.rtol;
    S->maxit = a.maxit;
    S->iter = 0;
    S->converged = 0;
    S->status = ILU0DD_OK;
    S->done = 0;
    a.hist[0] = 1.0;
    if (!finite(bb)) {
      S->status = ILU0DD_ERR_NONFINITE;
      S->done = 1;
    } else if (bb == 0.0) {
      S->converged = 1;
      S->rel = 0.0;
      S->rel_true = 0.0;
      S->done = 1;
    } else if (a.maxit <= 0) {
      S->status = ILU0DD_ERR_NOT_CONVERGED;
      S->done = 1;
    }
    *counter = 0;
  }
}

cudaError_t launch_init(const DevCtx& d, double rtol, int32_t maxit, cudaStream_t s) {
  if (d.N == 0) return cudaSuccess;
  VecArgs a{};
  for (int v = 0; v < kNumVec; ++v) a.v[v] = d.vec[v];
  a.N = d.N;
  a.partials = d.partials;
  a.stride = d.ntiles_pow2;
  a.m = d.ntiles_pow2;
  a.counters = d.counters;
  a.scal = d.scal;
  a.hist = d.hist;
  a.rtol = rtol;
  a.maxit = maxit;
  init_kernel<<<(unsigned)d.ntiles, kDotTile, 0, s>>>(a);
  return cudaGetLastError();
}

// restart 0: r = b - t (t = A x), rel_true = ||r||/||b||.
// restart 1: continue from r: rh = p = r, v = 0, rho = (r . r), done = 0.
__global__ void __launch_bounds__(kDotTile) residual_kernel(VecArgs a) {
  const int64_t i = (int64_t)blockIdx.x * kDotTile + threadIdx.x;
  SolverScalars* S = a.scal;
  if (a.restart) {
    if (i < a.N) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int64_t e = 3 * i + c;
        const double re = a.v[kVecR][e];
        a.v[kVecRh][e] = re;
        a.v[kVecP][e] = re;
        a.v[kVecV][e] = 0.0;
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      S->rho = S->rr;
      S->alpha = S->beta = S->omega = 0.0;
      S->converged = 0;
      S->done = 0;
    }
    return;
  }
  double q[1] = {0.0};
  if (i < a.N) {
    double rr[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int64_t e = 3 * i + c;
      rr[c] = a.v[kVecB][e] - a.v[kVecT][e];
      a.v[kVecR][e] = rr[c];
    }
    q[0] = fma(rr[2], rr[2], fma(rr[1], rr[1], rr[0] * rr[0]));
  }
  __shared__ double buf[1][kDotTile];
  tile_halving_sum<1>(q, buf);
  uint32_t* counter = a.counters + kCntResid;
  if (!publish_partials<1>(q, a.partials, a.stride, counter)) return;
  double out[1];
  finish_sum<1>(a.partials, a.stride, a.m, out, buf);
  if (threadIdx.x == 0) {
    S->rr = out[0];
    S->rel_true = sqrt(out[0]) / sqrt(S->bb);
    *counter = 0;
  }
}

cudaError_t launch_residual(const DevCtx& d, int restart, cudaStream_t s) {
  if (d.N == 0) return cudaSuccess;
  VecArgs a{};
  for (int v = 0; v < kNumVec; ++v) a.v[v] = d.vec[v];
  a.N = d.N;
  a.partials = d.partials;
  a.stride = d.ntiles_pow2;
  a.m = d.ntiles_pow2;
  a.counters = d.counters;
  a.scal = d.scal;
  a.restart = restart;
  residual_kernel<<<(unsigned)d.ntiles, kDotTile, 0, s>>>(a);
  return cudaGetLastError();
}

// Standalone dot product in the fixed order.
__global__ void __launch_bounds__(kDotTile) dot_kernel(const double* x, const double* y, int32_t N, double* partials,
                                                       int64_t m, uint32_t* counter, double* out_p) {
  const int64_t i = (int64_t)blockIdx.x * kDotTile + threadIdx.x;
  double q[1] = {i < N ? row_dot(x, y, i) : 0.0};
  __shared__ double buf[1][kDotTile];
  tile_halving_sum<1>(q, buf);
  if (!publish_partials<1>(q, partials, m, counter)) return;
  double out[1];
  finish_sum<1>(partials, m, m, out, buf);
  if (threadIdx.x == 0) {
    *out_p = out[0];
    *counter = 0;
  }
}

cudaError_t launch_dot(const DevCtx& d, const double* x, const double* y, double* out, cudaStream_t s) {
  if (d.N == 0) return cudaMemsetAsync(out, 0, sizeof(double), s);
  dot_kernel<<<(unsigned)d.ntiles, kDotTile, 0, s>>>(x, y, d.N, d.partials, d.ntiles_pow2,
                                                      d.counters + kCntDot, out);
  return cudaGetLastError();
}

__global__ void permute_kernel(const double* in, double* out, const int32_t* map, int32_t N, int dir) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t j = map[i];
  if (dir == 0) {
    // out[i] = in[perm[i]]
#pragma unroll
    for (int c = 0; c < 3; ++c) out[3 * i + c] = in[3 * j + c];
  } else {
    // out[old] = in[iperm[old]]
#pragma unroll
    for (int c = 0; c < 3; ++c) out[3 * i + c] = in[3 * j + c];
  }
}

cudaError_t launch_permute(const DevCtx& d, const double* in, double* out, int dir, cudaStream_t s) {
  if (d.N == 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = (unsigned)((d.N + threads - 1) / threads);
  permute_kernel<<<blocks, threads, 0, s>>>(in, out, dir == 0 ? d.perm : d.iperm, d.N, dir);
  return cudaGetLastError();
}

}  // namespace ilu0dd
