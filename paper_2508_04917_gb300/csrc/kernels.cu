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
  int prefetch_bytes, vec_bytes;
};

__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <typename TF>
__device__ __forceinline__ typename FactorLoad<TF>::compute gfactor(const unsigned char* p) {
  return FactorLoad<TF>::getg(p);
}

__device__ __forceinline__ int gu16(const unsigned char* p) {
  return (int)__ldg(reinterpret_cast<const unsigned short*>(p));
}

// One block per subdomain. The block reads its factor records straight from
// global memory (coalesced: consecutive threads read consecutive values) while
// thread 0 keeps bulk L2 prefetches (cp.async.bulk.prefetch.L2) a fixed
// distance ahead in the subdomain's stream, so the per-level loads hit L2.
// Shared memory holds only the subdomain vector. Three threads per row
// (lane = 3 * (row in warp) + a, ten rows per warp); rows of one piece are
// independent and pieces are separated by block barriers.
template <typename TF, int MODE>
__global__ void __launch_bounds__(kMaxApplyThreads, kApplyMinBlocks) ildu0_apply_kernel(ApplyArgs a) {
  using TV = typename FactorLoad<TF>::compute;
  constexpr uint32_t FE = sizeof(TF);
  extern __shared__ __align__(128) unsigned char smem[];

  if (MODE != kModePlain && a.scal->done) return;
  const CtaDesc cd = a.cta[blockIdx.x];
  const int tid = threadIdx.x;
  TV* y = reinterpret_cast<TV*>(smem);
  const unsigned char* gs = a.stream + cd.stream_off;
  const uint32_t len = (uint32_t)cd.stream_len;
  const uint32_t dist = (uint32_t)a.prefetch_bytes;
  constexpr uint32_t kPf = 16384;  // bytes per L2 prefetch instruction
  uint32_t pf_end = 0;             // prefetched prefix of the stream (thread 0)
  auto prefetch_upto = [&](uint32_t upto) {
    upto = min(upto, len);
    while (pf_end < upto) {
      const uint32_t bytes = min(kPf, len - pf_end);
      prefetch_l2(gs + pf_end, bytes);
      pf_end += bytes;
    }
  };
  if (tid == 0) prefetch_upto(dist);

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

  const int warp = tid >> 5, lane = tid & 31;
  const int comp = lane % 3;
  const int trow = warp * kRowsPerWarp + lane / 3;
  const bool lane_ok = lane < 3 * kRowsPerWarp;
  const int base_lane = lane - comp;

  PieceDesc nxt = cd.npieces > 0 ? a.pieces[cd.piece0] : PieceDesc{};
  for (int k = 0; k < cd.npieces; ++k) {
    const PieceDesc pd = nxt;
    if (k + 1 < cd.npieces) nxt = a.pieces[cd.piece0 + k + 1];
    if (tid == 0) prefetch_upto(pd.off + dist);
    const int n = (int)(pd.meta & 0xFFFFu);
    const int w = (int)((pd.meta >> 16) & 0xFFu);
    const int kind = (int)(pd.meta >> 24);
    if (warp * kRowsPerWarp < n) {  // warp-uniform: this warp has rows in the piece
      const bool active = lane_ok && trow < n;
      const unsigned char* rec = gs + pd.off;
      const unsigned char* cb = rec + 2 * (w + n);
      const unsigned char* vb = rec + pd.voff + (kind ? 9 * (size_t)n * FE : 0);
      // Issue every load of this row's slots at once: slot s starts at block
      // c0[s] = cnt[0] + .. + cnt[s-1] of the record (counts from the descriptor).
      int col[kDescSlots];
      TV bv[kDescSlots][3];
      uint32_t c0 = 0;
      int len = 0;
#pragma unroll
      for (int sl = 0; sl < kDescSlots; ++sl) {
        const uint32_t cs = pd.cnt[sl];  // 0 beyond w
        const bool has = active && sl < w && (uint32_t)trow < cs;
        len += has;
        col[sl] = has ? gu16(cb + 2 * (c0 + (uint32_t)trow)) : 0;
        const unsigned char* vo = vb + (9 * (size_t)c0 + (size_t)(3 * trow + comp)) * FE;
        const size_t cstride = 3 * (size_t)cs * FE;
#pragma unroll
        for (int c = 0; c < 3; ++c) bv[sl][c] = has ? gfactor<TF>(vo + c * cstride) : TV(0);
        c0 += cs;
      }
      TV d[3] = {TV(0), TV(0), TV(0)};
      if (kind && active) {
        const unsigned char* io = rec + pd.voff + (size_t)(3 * trow + comp) * FE;
        const size_t cstride = 3 * (size_t)n * FE;
#pragma unroll
        for (int c = 0; c < 3; ++c) d[c] = gfactor<TF>(io + c * cstride);
      }
      const int row = active ? gu16(rec + 2 * (w + trow)) : 0;
      TV acc = active ? y[3 * row + comp] : TV(0);
      if (kind) {
        // D^-1 (Section 4.3): w_i = D_i^-1 y_i; the row's three components
        // come from the neighbouring lanes
        const TV y0 = __shfl_sync(0xffffffffu, acc, base_lane);
        const TV y1 = __shfl_sync(0xffffffffu, acc, base_lane + 1);
        const TV y2 = __shfl_sync(0xffffffffu, acc, base_lane + 2);
        TV t = d[0] * y0;
        t = fma(d[1], y1, t);
        t = fma(d[2], y2, t);
        if (active) acc = t;
      }
      if (active) {
#pragma unroll
        for (int sl = 0; sl < kDescSlots; ++sl) {
          if (sl < len) {
            const int cl = col[sl];
            acc = fma(-bv[sl][0], y[3 * cl], acc);
            acc = fma(-bv[sl][1], y[3 * cl + 1], acc);
            acc = fma(-bv[sl][2], y[3 * cl + 2], acc);
          }
        }
        // rows with more than kDescSlots blocks (general patterns): remaining slots
        if (w > kDescSlots && len == kDescSlots) {
          for (int sl = kDescSlots; sl < w; ++sl) {
            const uint32_t cs = (uint32_t)gu16(rec + 2 * sl);
            if ((uint32_t)trow >= cs) break;
            const int cl = gu16(cb + 2 * (c0 + (uint32_t)trow));
            const unsigned char* vo = vb + (9 * (size_t)c0 + (size_t)(3 * trow + comp)) * FE;
            const size_t cstride = 3 * (size_t)cs * FE;
            acc = fma(-gfactor<TF>(vo), y[3 * cl], acc);
            acc = fma(-gfactor<TF>(vo + cstride), y[3 * cl + 1], acc);
            acc = fma(-gfactor<TF>(vo + 2 * cstride), y[3 * cl + 2], acc);
            c0 += cs;
          }
        }
        y[3 * row + comp] = acc;
      }
    }
    __syncthreads();
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
  const size_t smem = (size_t)optin - kApplyStaticSmem;  // the kernel's static shared memory
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
  a.prefetch_bytes = d.prefetch_bytes;
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

cudaError_t launch_dot_scratch(const double* x, const double* y, int32_t n_brows, double* partials, int64_t m,
                               uint32_t* counter, double* out, cudaStream_t s) {
  const int64_t ntiles = ((int64_t)n_brows + kDotTile - 1) / kDotTile;
  dot_kernel<<<(unsigned)ntiles, kDotTile, 0, s>>>(x, y, n_brows, partials, m, counter, out);
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
