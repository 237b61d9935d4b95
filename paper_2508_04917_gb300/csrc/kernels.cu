// sm_103a kernels of the hot path:
//  - apply_block: fused L -> D^-1 -> U~ sweep of one subdomain (Sections
//    4.2-4.4) by one thread block, subdomain vector in shared memory,
//    vertex-centric rows (Section 4.2.3) with three threads per row (3x3
//    blocks) or one (scalar CSR);
//  - spmv_block: y = A_p x on a sliced-ELL copy (coalesced, entry-major),
//    with the dot products of Algorithm 1 fused into the epilogue;
//  - update / init / residual / dot / permute: the BiCGSTAB vector steps.
// Each step is a per-block device function; the single-system kernels call it
// for their block, the batched kernels loop over a work list of
// (system, block) items of many systems in one launch.
// Dot products use one fixed order (per-row FMA, halving sums over 256-row
// tiles and over tiles); the last block of each reduction finishes the sum and
// updates the system's device-resident scalars, so no scalar goes to the host
// inside an iteration.
#include <cuda_runtime.h>

#include <type_traits>

#include "device_common.cuh"
#include "kernels.h"

namespace ilu0dd {

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

// Row i's contribution to a dot product in the fixed order: x0*y0, then
// fma(x_c, y_c, .) for c = 1..BS-1 (BS = 3: fma(x2,y2,fma(x1,y1,x0*y0))).
template <int BS>
__device__ __forceinline__ double row_dot(const double* x, const double* y, int64_t i) {
  double q = x[BS * i] * y[BS * i];
#pragma unroll
  for (int c = 1; c < BS; ++c) q = fma(x[BS * i + c], y[BS * i + c], q);
  return q;
}
template <int BS>
__device__ __forceinline__ double reg_dot(const double (&a)[BS], const double (&b)[BS]) {
  double q = a[0] * b[0];
#pragma unroll
  for (int c = 1; c < BS; ++c) q = fma(a[c], b[c], q);
  return q;
}

__device__ __forceinline__ bool finite(double v) { return isfinite(v); }

// ===========================================================================
// Fused ILDU0 apply
// ===========================================================================

// One block per subdomain. The block reads its factor records straight from
// global memory (coalesced: consecutive threads read consecutive values; the
// slot counts in the piece descriptor let every load of a level issue at
// once) while one thread keeps bulk L2 prefetches (cp.async.bulk.prefetch.L2)
// a fixed distance ahead in the subdomain's stream. Shared memory holds the
// subdomain vector, the block's piece descriptors and one mbarrier per piece.
// Rows of one piece are independent. There are no block barriers between
// pieces: a piece's row groups go to warps round-robin, a warp issues the
// loads of its row group at once and then waits (suspended, not polling)
// only until the previous level's pieces are complete, so warps with no rows
// in the current level run ahead to load for later ones.
// Two thread mappings: FP64 and float-pair 3x3 factors take three threads per
// row (lane = 3 * (row in warp) + a, ten rows per warp: apply_block), whose
// per-thread chain of multiply-adds stays short where this GPU's FP64 pipe or
// the double-float arithmetic is the bound; FP32 and BF16 factors one thread
// per row computing all three components (32 rows per warp, the row-thread
// layout: apply_block_rt), which issues a third of the instructions of the
// three-thread mapping, when no row has more than kDescSlots blocks on either
// side (else they too take three threads per row, whose general-pattern path
// loads wider rows' slots in groups); scalar rows take one thread each
// (apply_block with BS = 1). On rows of up to kDescSlots blocks a side both
// 3x3 mappings compute each output component with the same operations in the
// same order, so they give the same bits.
// In the DF64 mode the vector is held as float pairs, scaled by a power of two
// per block (exact, and the apply is linear and local to the block) so that
// the FP32 exponent range never limits it.
// Modes: plain z = M^-1 r; P: p <- r + beta (p - omega v), z = M^-1 p;
// S: s <- r - alpha v, z = M^-1 s. Modes P and S skip a finished solve.
// PART 0 runs every piece (the fused apply); 1 only the L sweep, 2 only the
// D^-1 and U~ sweep (the two launches of the unfused apply). The ablations:
// SYNC 1 orders rows by per-row flags (Algorithm 4) instead of the per-piece
// mbarriers; TRAV 1 traverses a level edge-centrically (threads over the
// blocks of a level, shared-memory atomics into the rows) instead of
// row-wise; VGLOB 1 (FP64 only) keeps the subdomain vector in global memory
// (in z) instead of shared memory, to measure what shared memory brings.

// Subdomain vector -> shared memory, with the fused BiCGSTAB update of modes P
// (p <- r + beta (p - omega v), written back to p) and S (s <- r - alpha v,
// written back to s). Entry e of the subdomain (row e / BS, component e % BS)
// goes to y[VS * row + component]. DF64: the block's largest magnitude sets a
// power-of-two scale 2^-k (applied here) and the function returns k, which
// store_vector undoes; otherwise it returns 0. The DF64 maximum and split run
// on integer and FP32 operations (df_from_double_scaled_bits), with the FP64
// operations only where that path declines.
template <typename TV, int MODE, int BS, int VS>
__device__ __forceinline__ int load_vector(const SysDesc& S, const CtaDesc& cd, const double* r, TV* y,
                                           unsigned char* smem) {
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)BS * cd.row0;
  const int nv = BS * cd.nrows;
  double alpha = 0.0, beta = 0.0, omega = 0.0;
  if (MODE == kModeP) { beta = S.scal->beta; omega = S.scal->omega; }
  if (MODE == kModeS) alpha = S.scal->alpha;
  const double* vv = S.vec[kVecV];
  double* pp = S.vec[kVecP];
  double* ss = S.vec[kVecS];
  constexpr bool kDF = std::is_same<TV, df64>::value;
  static_assert(!kDF || VS == BS, "float pairs keep the unpadded vector");
  // DF64: bits of the largest |value| this thread loads (for non-NaN values
  // the magnitude bits order like the magnitudes; NaNs are skipped, as fmax does)
  unsigned long long amax_bits = 0ull;
  for (int e = tid; e < nv; e += blockDim.x) {
    double val;
    if (MODE == kModePlain) {
      val = r[base + e];
    } else if (MODE == kModeP) {
      val = fma(beta, fma(-omega, vv[base + e], pp[base + e]), r[base + e]);
      pp[base + e] = val;
    } else {
      val = fma(-alpha, vv[base + e], r[base + e]);
      ss[base + e] = val;
    }
    if constexpr (kDF) {
      reinterpret_cast<double*>(y)[e] = val;  // same 8 bytes; converted below
      const unsigned long long mag = (unsigned long long)__double_as_longlong(val) & 0x7FFFFFFFFFFFFFFFull;
      if (mag <= 0x7FF0000000000000ull && mag > amax_bits) amax_bits = mag;
    } else if constexpr (VS == BS) {
      y[e] = to_compute<TV>(val);
    } else {
      const int row = e / BS;
      y[VS * row + (e - BS * row)] = to_compute<TV>(val);
    }
  }
  int k = 0;
  if constexpr (kDF) {
    // block maximum -> scale 2^-k with max |value| * 2^-k in [0.5, 1)
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(0xffffffffu, amax_bits, o);
      if (other > amax_bits) amax_bits = other;
    }
    unsigned long long* red = reinterpret_cast<unsigned long long*>(smem + S.vec_bytes);  // descriptor area, not yet in use
    if ((tid & 31) == 0) red[tid >> 5] = amax_bits;
    __syncthreads();
    amax_bits = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (red[w] > amax_bits) amax_bits = red[w];
    const double amax = __longlong_as_double((long long)amax_bits);
    if (amax > 0.0 && isfinite(amax)) frexp(amax, &k);
    const double scale = ldexp(1.0, -k);
    for (int e = tid; e < nv; e += blockDim.x) {
      const double v = reinterpret_cast<double*>(y)[e];
      df64 pair;
      if (!df_from_double_scaled_bits(v, k, &pair)) pair = df_from_double(v * scale);
      y[e] = pair;
    }
  }
  return k;
}

// Shared memory -> z (the subdomain's entries), undoing the DF64 scale 2^-k.
template <typename TV, int BS, int VS>
__device__ __forceinline__ void store_vector(const CtaDesc& cd, const TV* y, double* z, int k) {
  const int64_t base = (int64_t)BS * cd.row0;
  const int nv = BS * cd.nrows;
  for (int e = threadIdx.x; e < nv; e += blockDim.x) {
    const int row = VS == BS ? 0 : e / BS;
    const TV v = VS == BS ? y[e] : y[VS * row + (e - BS * row)];
    if constexpr (std::is_same<TV, df64>::value)
      z[base + e] = df_to_double_scaled(v, k);
    else
      z[base + e] = to_double(v);
  }
  (void)k;
}

// Stage the descriptors of pieces [k, k + min(kDescCache, k1 - k)) in shared
// memory and, for the mbarrier-ordered apply (SYNC 0), arm one mbarrier per
// staged piece: every thread of the piece's row groups (RPW rows each)
// arrives once its rows are written, 32 arrivals per group (the stuck piece
// of the failure-path tests expects one arrival too many). Called by every
// thread; the previous window's pieces must all be complete.
template <int RPW, int SYNC>
__device__ __forceinline__ void stage_window(const SysDesc& S, const CtaDesc& cd, int k, int k0, int k1,
                                             PieceDesc* dsm, uint64_t* mbar, volatile uint32_t* abort_flag) {
  const int tid = threadIdx.x;
  const int cnt = min(kDescCache, k1 - k);
  if (k > k0) {
    __syncthreads();  // every piece of the (full) window is done
    if constexpr (SYNC == 0)
      for (int q = tid; q < kDescCache; q += blockDim.x) mbar_inval(mbar + q);
  }
  const uint4* src = reinterpret_cast<const uint4*>(S.pieces + cd.piece0 + k);
  uint4* dst = reinterpret_cast<uint4*>(dsm);
  for (int q = tid; q < 2 * cnt; q += blockDim.x) dst[q] = __ldg(src + q);
  if (k == k0 && tid == 0) *abort_flag = 0;
  __syncthreads();
  if constexpr (SYNC == 0) {
    for (int q = tid; q < cnt; q += blockDim.x) {
      const uint32_t groups = ((dsm[q].meta & 0xFFFFu) + RPW - 1) / RPW;
      mbar_init(mbar + q, 32u * groups + (cd.piece0 + k + q == S.wait_stuck ? 1u : 0u));
    }
    __syncthreads();
  }
}

// Wait for the previous level's pieces of this window (earlier windows are
// done). Bounded: after S.wait_cycles SM cycles the block gives up, flags the
// device error word and carries on (its results are then not valid).
__device__ __forceinline__ void wait_prev_level(const SysDesc& S, const PieceDesc& pd, int win0, uint64_t* mbar,
                                                volatile uint32_t* abort_flag) {
  for (int j = max((int)pd.prev_first, win0); j < (int)pd.lvl_first; ++j) {
    uint64_t* b = mbar + (j - win0);
    if (!mbar_try_wait(b, 0)) {
      const long long t0 = clock64();
      while (!mbar_try_wait(b, 0)) {
        if (*abort_flag || clock64() - t0 > (long long)S.wait_cycles) {
          if (atomicCAS(const_cast<uint32_t*>(abort_flag), 0u, 1u) == 0u) atomicCAS(S.err, 0, kErrApplyWait);
          break;
        }
      }
    }
  }
}

// Algorithm 4's wait (SYNC 1): spin (bounded) until row rr's flag reaches ph
// (1: its L result is in the vector, 2: its final value).
__device__ __forceinline__ void wait_row_flag(const SysDesc& S, volatile uint8_t* rflag, int rr, uint8_t ph,
                                              volatile uint32_t* abort_flag) {
  if (rflag[rr] >= ph) return;
  const long long t0 = clock64();
  while (rflag[rr] < ph) {
    if (*abort_flag || clock64() - t0 > (long long)S.wait_cycles) {
      if (atomicCAS(const_cast<uint32_t*>(abort_flag), 0u, 1u) == 0u) atomicCAS(S.err, 0, kErrApplyWait);
      return;
    }
  }
}

template <typename TF, int MODE, int PART = 0, int SYNC = 0, int TRAV = 0>
__device__ __forceinline__ void apply_block_rt(const SysDesc& S, int sub, const double* r, double* z);

// RT 1: the row-thread layout (apply_block_rt); RT 0: three threads per 3x3
// row, one per scalar row.
template <typename TF, int MODE, int PART = 0, int BS = 3, int SYNC = 0, int TRAV = 0, int VGLOB = 0, int RT = 0>
__device__ __forceinline__ void apply_block(const SysDesc& S, int sub, const double* r, double* z) {
  static_assert(BS == 1 || BS == 3, "block dimension 1 or 3");
  if constexpr (RT) {
    static_assert(BS == 3 && !VGLOB, "row-thread layout: 3x3 blocks, vector in shared memory");
    apply_block_rt<TF, MODE, PART, SYNC, TRAV>(S, sub, r, z);
  } else {
  constexpr int RPW = BS == 3 ? kRowsPerWarp : 32;  // rows per warp
  using TV = typename FactorLoad<TF>::compute;
  constexpr uint32_t FE = sizeof(TF);
  extern __shared__ __align__(128) unsigned char smem[];

  if (MODE != kModePlain && S.scal->done) return;
  const CtaDesc cd = S.cta[sub];
  const int tid = threadIdx.x;
  static_assert(!VGLOB || std::is_same<TF, double>::value, "global vector: FP64 only");
  TV* y = VGLOB ? reinterpret_cast<TV*>(z + (int64_t)BS * cd.row0) : reinterpret_cast<TV*>(smem);
  const unsigned char* gs = S.stream + cd.stream_off;
  const uint32_t len = (uint32_t)cd.stream_len;
  const uint32_t dist = (uint32_t)S.prefetch_bytes;
  constexpr uint32_t kPf = 16384;  // bytes per L2 prefetch instruction
  const int k0 = PART == 2 ? cd.npieces_l : 0;             // pieces [k0, k1) run here
  const int k1 = PART == 1 ? cd.npieces_l : cd.npieces;
  uint32_t pf_end = PART == 2 && k0 < k1 ? S.pieces[cd.piece0 + k0].off : 0;  // prefetched prefix
  auto prefetch_upto = [&](uint32_t upto) {
    upto = min(upto, len);
    while (pf_end < upto) {
      const uint32_t bytes = min(kPf, len - pf_end);
      prefetch_l2(gs + pf_end, bytes);
      pf_end += bytes;
    }
  };
  // L2 prefetches come from lane 0 of the last warp, as that warp passes the
  // pieces
  const bool pf_thread = tid == (int)blockDim.x - 32;
  if (pf_thread) prefetch_upto(pf_end + dist);

  constexpr bool kDF = std::is_same<TV, df64>::value;
  const int kscale = load_vector<TV, MODE, BS, BS>(S, cd, r, y, smem);
  // SYNC 1 (Algorithm 4's synchronization): one flag per row, 1 once the
  // row's L result is in the vector (at once for rows of L level 0), 2 once
  // its final value is.
  volatile uint8_t* rflag = smem + S.vec_bytes + kApplyTailSmem;
  if constexpr (SYNC == 1)
    for (int e = tid; e < cd.nrows; e += blockDim.x) rflag[e] = S.row_l0[cd.row0 + e];
  __syncthreads();

  const int warp = tid >> 5, lane = tid & 31;
  const int nwarps = (int)(blockDim.x >> 5);
  const int comp = BS == 3 ? lane % 3 : 0;
  const bool lane_ok = BS == 3 ? lane < 3 * kRowsPerWarp : true;
  const int base_lane = lane - comp;

  PieceDesc* dsm = reinterpret_cast<PieceDesc*>(smem + S.vec_bytes);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(dsm + kDescCache);
  volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(mbar + kDescCache);
  int win0 = k0;  // first piece of the staged window
  int rot = 0;    // warp that takes row group 0 of the next piece
  for (int k = k0; k < k1; ++k) {
    // Row flags order only the reads of each row; the U sweep overwrites L
    // results that rows of the L sweep may still read (for unsymmetric
    // patterns), so with SYNC 1 the sweeps are separated by a barrier.
    if constexpr (SYNC == 1)
      if (k == cd.npieces_l && k > k0 && (k - k0) % kDescCache != 0) __syncthreads();
    if ((k - k0) % kDescCache == 0) {
      stage_window<RPW, SYNC>(S, cd, k, k0, k1, dsm, mbar, abort_flag);
      win0 = k;
    }
    const PieceDesc pd = dsm[k - win0];
    if (pf_thread) prefetch_upto(pd.off + dist);
    const int n = (int)(pd.meta & 0xFFFFu);
    const int w = (int)((pd.meta >> 16) & 0xFFu);
    const int kind = (int)(pd.meta >> 24);
    // Row groups (RPW rows each) go to warps round-robin across pieces, so a
    // warp issues the loads of its next group while the pieces before it run
    // on other warps. Without block barriers, a warp waits only for the
    // previous level's pieces (their mbarriers), and only before it reads the
    // subdomain vector.
    const int ng = (n + RPW - 1) / RPW;  // <= nwarps (pieces fit the block)
    int g = warp - rot;
    if (g < 0) g += nwarps;
    rot += ng;
    if (rot >= nwarps) rot -= nwarps;
    if (g < ng) {  // warp-uniform: this warp has a row group in the piece
      const int trow = g * RPW + (BS == 3 ? lane / 3 : lane);
      const bool active = lane_ok && trow < n;
      const uint32_t lane_voff = (uint32_t)(BS * trow + comp) * FE;  // this thread's value offset in a slot
      const uint32_t trow2 = 2u * (uint32_t)trow;
      const unsigned char* rec = gs + pd.off;
      // 32-bit byte offsets from the block's (uniform) stream base: the
      // warp-uniform part per slot plus this thread's fixed part
      const uint32_t vbase = pd.off + pd.voff + (kind ? (uint32_t)(BS * BS) * (uint32_t)n * FE : 0u);
      const uint32_t cbase = pd.off + 2u * (uint32_t)(w + n);
      int col[kDescSlots];
      TV bv[kDescSlots][BS];
      uint32_t c0 = 0;
      int nsl = 0;
      if constexpr (TRAV == 0) {
#pragma unroll
        for (int sl = 0; sl < kDescSlots; ++sl) {
          const uint32_t cs = pd.cnt[sl];  // 0 beyond w
          const bool has = active && sl < w && (uint32_t)trow < cs;
          nsl += has;
          col[sl] = has ? gu16(gs + (cbase + 2u * c0 + trow2)) : 0;
          const uint32_t vo = vbase + (uint32_t)(BS * BS) * FE * c0 + lane_voff;
          const uint32_t cstride = (uint32_t)BS * FE * cs;
#pragma unroll
          for (int c = 0; c < BS; ++c) bv[sl][c] = has ? gfactor<TF>(gs + (vo + (uint32_t)c * cstride)) : TV(0);
          c0 += cs;
        }
      }
      // Edge-centric traversal (TRAV 1): the group's blocks are tasks
      // (slot, row in group), task = 32 * round + lane; round 0's block is
      // loaded here, ahead of the wait.
      int e_row = 0, e_col = 0;
      TV ev[BS][BS];
      bool e_has = false;
      auto edge_task = [&](int task, int& rrow, int& rcol, TV (&v)[BS][BS]) -> bool {
        const int sl = task / RPW, t = task % RPW;
        const int tr = g * RPW + t;
        if (sl >= w) return false;
        uint32_t cc = 0, cs = 0;
        for (int q = 0; q <= sl; ++q) {
          cs = q < kDescSlots ? (uint32_t)pd.cnt[q] : (uint32_t)gu16(rec + 2 * q);
          if (q < sl) cc += cs;
        }
        if ((uint32_t)tr >= cs) return false;
        rrow = gu16(gs + (pd.off + 2u * (uint32_t)w + 2u * (uint32_t)tr));
        rcol = gu16(gs + (cbase + 2u * (cc + (uint32_t)tr)));
        const uint32_t vo = vbase + (uint32_t)(BS * BS) * FE * cc;
#pragma unroll
        for (int a = 0; a < BS; ++a)
#pragma unroll
          for (int c = 0; c < BS; ++c)
            v[a][c] = gfactor<TF>(gs + (vo + (((uint32_t)c * cs + (uint32_t)tr) * BS + (uint32_t)a) * FE));
        return true;
      };
      if constexpr (TRAV == 1) e_has = edge_task(lane, e_row, e_col, ev);
      TV d[BS];
#pragma unroll
      for (int c = 0; c < BS; ++c) d[c] = TV(0);
      if (kind && active) {
        const uint32_t io = pd.off + pd.voff + lane_voff;
        const uint32_t cstride = (uint32_t)BS * FE * (uint32_t)n;
#pragma unroll
        for (int c = 0; c < BS; ++c) d[c] = gfactor<TF>(gs + (io + (uint32_t)c * cstride));
      }
      const int row = active ? gu16(gs + (pd.off + 2u * (uint32_t)w + trow2)) : 0;
      if constexpr (SYNC == 0) {
        wait_prev_level(S, pd, win0, mbar, abort_flag);
      } else {
        // Algorithm 4: wait (spin, bounded) for exactly the rows this row
        // reads: its own L result in the U sweep, then each slot's column.
        if (active) {
          const uint8_t phase = kind ? 2 : 1;
          auto wait_row = [&](int rr, uint8_t ph) { wait_row_flag(S, rflag, rr, ph, abort_flag); };
          if (kind) wait_row(row, 1);
#pragma unroll
          for (int sl = 0; sl < kDescSlots; ++sl)
            if (sl < nsl) wait_row(col[sl], phase);
          // further slots of general patterns: their columns come from the record
          if (w > kDescSlots && nsl == kDescSlots) {
            uint32_t cc = (uint32_t)pd.cnt[0] + pd.cnt[1] + pd.cnt[2];
            for (int sl = kDescSlots; sl < w; ++sl) {
              const uint32_t cs = (uint32_t)gu16(rec + 2 * sl);
              if ((uint32_t)trow >= cs) break;
              wait_row(gu16(gs + (cbase + 2u * cc + trow2)), phase);
              cc += cs;
            }
          }
        }
        __threadfence_block();
      }
      __syncwarp();
      TV acc = active ? y[BS * row + comp] : TV(0);
      if (kind) {
        // D^-1 (Section 4.3): w_i = D_i^-1 y_i; with 3x3 blocks the row's
        // three components come from the neighbouring lanes
        if constexpr (BS == 3) {
          const TV y0 = shfl(acc, base_lane);
          const TV y1 = shfl(acc, base_lane + 1);
          const TV y2 = shfl(acc, base_lane + 2);
          TV t = d[0] * y0;
          t = mac(d[1], y1, t);
          t = mac(d[2], y2, t);
          if (active) acc = t;
        } else {
          if (active) acc = d[0] * acc;
        }
      }
      if constexpr (TRAV == 1) {
        // the D^-1 result first (it is what the U blocks subtract from), then
        // each task subtracts its block's product with shared-memory atomics
        if (kind && active) y[BS * row + comp] = acc;
        __syncwarp();
        auto edge_apply = [&](int rrow, int rcol, const TV (&v)[BS][BS]) {
#pragma unroll
          for (int a = 0; a < BS; ++a) {
            TV p = v[a][0] * y[BS * rcol];
#pragma unroll
            for (int c = 1; c < BS; ++c) p = mac(v[a][c], y[BS * rcol + c], p);
            atomicAdd(&y[BS * rrow + a], -p);
          }
        };
        if (e_has) edge_apply(e_row, e_col, ev);
        for (int base_t = 32; base_t < RPW * w; base_t += 32) {  // further rounds (warp-uniform)
          int rr, rc;
          TV v[BS][BS];
          if (edge_task(base_t + lane, rr, rc, v)) edge_apply(rr, rc, v);
        }
      } else if (active) {
#pragma unroll
        for (int sl = 0; sl < kDescSlots; ++sl) {
          if (sl < nsl) {
            const int cl = col[sl];
#pragma unroll
            for (int c = 0; c < BS; ++c) acc = mac(-bv[sl][c], y[BS * cl + c], acc);
          }
        }
        // Rows with more than kDescSlots blocks (general patterns): the further
        // slots, G at a time with all their loads issued first (the slot
        // counts come from the record head). FP64-arithmetic applies (FP64,
        // DF64) multiply-add them in slot (ascending column) order into the
        // one accumulator, as the first slots; FP32 arithmetic alternates
        // two accumulators, added at the end, to shorten the dependency
        // chain (measured on GB300, unstructured 128^3: FP64 0.779 -> 0.770
        // ms and DF64 0.629 -> 0.608 with one accumulator; FP32 0.336 with
        // two against 0.388 with one).
        if (w > kDescSlots && nsl == kDescSlots) {
          constexpr int G = sizeof(TV) >= 8 ? 4 : 3;
          constexpr bool two = sizeof(TV) < 8;
          TV acc_b = TV(0);
          for (int sl = kDescSlots; sl < w; sl += G) {
            uint32_t cs[G], off[G];
            bool has[G];
            uint32_t cc = c0;
#pragma unroll
            for (int u = 0; u < G; ++u) {
              cs[u] = sl + u < w ? (uint32_t)gu16(rec + 2 * (sl + u)) : 0u;
              off[u] = cc;
              cc += cs[u];
              has[u] = (uint32_t)trow < cs[u];  // counts do not grow with the slot
            }
            int cl[G];
            TV v[G][BS];
#pragma unroll
            for (int u = 0; u < G; ++u) {
              cl[u] = has[u] ? gu16(gs + (cbase + 2u * off[u] + trow2)) : 0;
              const uint32_t vo = vbase + (uint32_t)(BS * BS) * FE * off[u] + lane_voff;
#pragma unroll
              for (int c = 0; c < BS; ++c)
                v[u][c] = has[u] ? gfactor<TF>(gs + (vo + (uint32_t)c * ((uint32_t)BS * FE * cs[u]))) : TV(0);
            }
#pragma unroll
            for (int u = 0; u < G; ++u) {
              if (has[u]) {
                TV& a2 = two && (u & 1) ? acc_b : acc;
#pragma unroll
                for (int c = 0; c < BS; ++c) a2 = mac(-v[u][c], y[BS * cl[u] + c], a2);
              }
            }
            c0 = cc;
            if (!has[G - 1]) break;
          }
          if constexpr (two) acc = mac(TV(1), acc_b, acc);
        }
        y[BS * row + comp] = acc;
      }
      __syncwarp();
      if constexpr (SYNC == 0) {
        mbar_arrive(mbar + (k - win0));  // every lane: releases its own writes
      } else {
        __threadfence_block();
        __syncwarp();
        if (active && comp == 0) rflag[row] = kind ? 2 : 1;
      }
    }
  }
  __syncthreads();
  if constexpr (SYNC == 0)
    for (int q = tid; q < k1 - win0; q += blockDim.x) mbar_inval(mbar + q);
  if constexpr (!VGLOB) store_vector<TV, BS, BS>(cd, y, z, kscale);
  (void)kDF;
  }
}


// ---- row-thread mapping (3x3 blocks with FP32 or BF16 factors)

// One block (or D^-1) of one row in the row-thread layout, as loaded: entry
// e = 3a + c of the value array `arr` of `count` rows, row t, read with
// 16-byte vector loads (rt_value_offset); get(e) converts entry e to the
// compute type.
template <typename TF>
struct RtBlock;
template <>
struct RtBlock<float> {
  float4 q0, q1;
  float e8;
  __device__ __forceinline__ void load(const unsigned char* arr, uint32_t count, uint32_t t) {
    q0 = __ldg(reinterpret_cast<const float4*>(arr + 16u * t));
    q1 = __ldg(reinterpret_cast<const float4*>(arr + 16u * (count + t)));
    e8 = __ldg(reinterpret_cast<const float*>(arr + 32u * count + 4u * t));
  }
  __device__ __forceinline__ float get(int e) const {
    switch (e) {
      case 0: return q0.x;
      case 1: return q0.y;
      case 2: return q0.z;
      case 3: return q0.w;
      case 4: return q1.x;
      case 5: return q1.y;
      case 6: return q1.z;
      case 7: return q1.w;
      default: return e8;
    }
  }
};
template <>
struct RtBlock<bf16s> {
  uint4 q;  // entries 0..7, two per word (the lower half first)
  unsigned short e8;
  __device__ __forceinline__ void load(const unsigned char* arr, uint32_t count, uint32_t t) {
    q = __ldg(reinterpret_cast<const uint4*>(arr + 16u * t));
    e8 = __ldg(reinterpret_cast<const unsigned short*>(arr + 16u * count + 2u * t));
  }
  __device__ __forceinline__ float get(int e) const {
    const uint32_t wd = e < 2 ? q.x : e < 4 ? q.y : e < 6 ? q.z : q.w;
    if (e == 8) return bf16_to_f32(e8);
    return __uint_as_float((e & 1) ? (wd & 0xFFFF0000u) : (wd << 16));
  }
};

// Bytes of one value array of `count` rows (padded to 16).
template <typename TF>
__device__ __forceinline__ uint32_t rt_bytes(uint32_t count) {
  return (9u * (uint32_t)sizeof(TF) * count + 15u) & ~15u;
}

// Three components of one row of the shared-memory vector (VS entries per row).
template <typename TV, int VS>
__device__ __forceinline__ void rt_get3(const TV* y, int row, TV (&x)[3]) {
  if constexpr (std::is_same<TV, float>::value && VS == 4) {
    const float4 v = reinterpret_cast<const float4*>(y)[row];
    x[0] = v.x;
    x[1] = v.y;
    x[2] = v.z;
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) x[c] = y[VS * row + c];
  }
}
template <typename TV, int VS>
__device__ __forceinline__ void rt_put3(TV* y, int row, const TV (&x)[3]) {
  if constexpr (std::is_same<TV, float>::value && VS == 4) {
    reinterpret_cast<float4*>(y)[row] = make_float4(x[0], x[1], x[2], 0.f);
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) y[VS * row + c] = x[c];
  }
}

// acc[a] -= B x for one 3x3 block, per component a: c = 0..2 in order, each a
// multiply-add (the three-thread mapping's operations, one thread per row).
template <typename TF, typename TV>
__device__ __forceinline__ void rt_sub_block(const RtBlock<TF>& b, const TV (&x)[3], TV (&acc)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[a] = mac(-b.get(3 * a + c), x[c], acc[a]);
}

// The fused apply with one thread per row (see the comment above apply_block):
// each thread loads its row's D^-1 block and all its blocks (the plan takes
// this mapping only when no row has more than kDescSlots blocks on either
// side) before the wait for the previous level (loading the FP32 slots after
// the wait instead cost 12 % at 160^3), then forms all three components of
// the row.
template <typename TF, int MODE, int PART, int SYNC, int TRAV>
__device__ __forceinline__ void apply_block_rt(const SysDesc& S, int sub, const double* r, double* z) {
  constexpr int RPW = 32;
  using TV = typename FactorLoad<TF>::compute;
  constexpr int VS = std::is_same<TV, float>::value ? 4 : 3;  // vector entries per row in shared memory
  extern __shared__ __align__(128) unsigned char smem[];

  if (MODE != kModePlain && S.scal->done) return;
  const CtaDesc cd = S.cta[sub];
  const int tid = threadIdx.x;
  TV* y = reinterpret_cast<TV*>(smem);
  const unsigned char* gs = S.stream + cd.stream_off;
  const uint32_t len = (uint32_t)cd.stream_len;
  const uint32_t dist = (uint32_t)S.prefetch_bytes;
  constexpr uint32_t kPf = 16384;
  const int k0 = PART == 2 ? cd.npieces_l : 0;
  const int k1 = PART == 1 ? cd.npieces_l : cd.npieces;
  uint32_t pf_end = PART == 2 && k0 < k1 ? S.pieces[cd.piece0 + k0].off : 0;
  auto prefetch_upto = [&](uint32_t upto) {
    upto = min(upto, len);
    while (pf_end < upto) {
      const uint32_t bytes = min(kPf, len - pf_end);
      prefetch_l2(gs + pf_end, bytes);
      pf_end += bytes;
    }
  };
  const bool pf_thread = tid == (int)blockDim.x - 32;
  if (pf_thread) prefetch_upto(pf_end + dist);

  const int kscale = load_vector<TV, MODE, 3, VS>(S, cd, r, y, smem);
  volatile uint8_t* rflag = smem + S.vec_bytes + kApplyTailSmem;
  if constexpr (SYNC == 1)
    for (int e = tid; e < cd.nrows; e += blockDim.x) rflag[e] = S.row_l0[cd.row0 + e];
  __syncthreads();

  const int warp = tid >> 5, lane = tid & 31;
  const int nwarps = (int)(blockDim.x >> 5);
  PieceDesc* dsm = reinterpret_cast<PieceDesc*>(smem + S.vec_bytes);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(dsm + kDescCache);
  volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(mbar + kDescCache);
  int win0 = k0;
  int rot = 0;
  for (int k = k0; k < k1; ++k) {
    if constexpr (SYNC == 1)
      if (k == cd.npieces_l && k > k0 && (k - k0) % kDescCache != 0) __syncthreads();
    if ((k - k0) % kDescCache == 0) {
      stage_window<RPW, SYNC>(S, cd, k, k0, k1, dsm, mbar, abort_flag);
      win0 = k;
    }
    const PieceDesc pd = dsm[k - win0];
    if (pf_thread) prefetch_upto(pd.off + dist);
    const int n = (int)(pd.meta & 0xFFFFu);
    const int w = (int)((pd.meta >> 16) & 0xFFu);
    const int kind = (int)(pd.meta >> 24);
    const int ng = (n + RPW - 1) / RPW;
    int g = warp - rot;
    if (g < 0) g += nwarps;
    rot += ng;
    if (rot >= nwarps) rot -= nwarps;
    if (g < ng) {  // warp-uniform
      const int trow = g * RPW + lane;
      const bool active = trow < n;
      const unsigned char* rec = gs + pd.off;
      const uint32_t arr0 = pd.off + pd.voff;  // first value array (D^-1 for U pieces)
      const uint32_t cbase = pd.off + 2u * (uint32_t)(w + n);
      uint32_t sb = arr0 + (kind ? rt_bytes<TF>((uint32_t)n) : 0u);  // current slot's value array
      uint32_t c0 = 0;
      int col[kDescSlots];
      RtBlock<TF> blk[kDescSlots];
      int nsl = 0;
      if constexpr (TRAV == 0) {
#pragma unroll
        for (int sl = 0; sl < kDescSlots; ++sl) {
          const uint32_t cs = pd.cnt[sl];  // 0 beyond w
          const bool has = active && sl < w && (uint32_t)trow < cs;
          nsl += has;
          col[sl] = has ? gu16(gs + (cbase + 2u * (c0 + (uint32_t)trow))) : 0;
          if (has) blk[sl].load(gs + sb, cs, (uint32_t)trow);
          sb += rt_bytes<TF>(cs);
          c0 += cs;
        }
      }
      RtBlock<TF> dblk;
      if (kind && active) dblk.load(gs + arr0, (uint32_t)n, (uint32_t)trow);
      const int row = active ? gu16(gs + (pd.off + 2u * (uint32_t)(w + trow))) : 0;
      if constexpr (SYNC == 0) {
        wait_prev_level(S, pd, win0, mbar, abort_flag);
      } else if (active) {
        // Algorithm 4: wait for exactly the rows this row reads
        const uint8_t phase = kind ? 2 : 1;
        if (kind) wait_row_flag(S, rflag, row, 1, abort_flag);
        uint32_t cc = 0;
        for (int sl = 0; sl < w; ++sl) {
          const uint32_t cs = sl < kDescSlots ? (uint32_t)pd.cnt[sl] : (uint32_t)gu16(rec + 2 * sl);
          if ((uint32_t)trow >= cs) break;
          wait_row_flag(S, rflag, gu16(gs + (cbase + 2u * (cc + (uint32_t)trow))), phase, abort_flag);
          cc += cs;
        }
        __threadfence_block();
      }
      __syncwarp();
      if constexpr (TRAV == 0) {
        if (active) {
          TV acc[3];
          rt_get3<TV, VS>(y, row, acc);
          if (kind) {
            // D^-1 (Section 4.3): w = D_i^-1 y_i
            TV t[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              t[a] = dblk.get(3 * a) * acc[0];
              t[a] = mac(dblk.get(3 * a + 1), acc[1], t[a]);
              t[a] = mac(dblk.get(3 * a + 2), acc[2], t[a]);
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[a] = t[a];
          }
#pragma unroll
          for (int sl = 0; sl < kDescSlots; ++sl) {
            if (sl < nsl) {
              TV x[3];
              rt_get3<TV, VS>(y, col[sl], x);
              rt_sub_block<TF, TV>(blk[sl], x, acc);
            }
          }
          rt_put3<TV, VS>(y, row, acc);
        }
      } else {
        // Edge-centric traversal (TRAV 1): the row's D^-1 step first, then
        // the (row, slot) blocks of the group are tasks spread over the lanes
        // (task = row-in-group * w + slot, lanes in turn), each subtracting
        // its block's product from its row with shared-memory atomics.
        if (kind && active) {
          TV v[3], t[3];
          rt_get3<TV, VS>(y, row, v);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            t[a] = dblk.get(3 * a) * v[0];
            t[a] = mac(dblk.get(3 * a + 1), v[1], t[a]);
            t[a] = mac(dblk.get(3 * a + 2), v[2], t[a]);
          }
          rt_put3<TV, VS>(y, row, t);
        }
        __syncwarp();
        const int rows_g = min(RPW, n - g * RPW);
        for (int task = lane; task < rows_g * w; task += 32) {
          const int tg = task / w, sl = task - tg * w;  // row in group, slot
          const uint32_t tr = (uint32_t)(g * RPW + tg);
          uint32_t cs = 0, cc = 0, sbb = arr0 + (kind ? rt_bytes<TF>((uint32_t)n) : 0u);
          for (int q = 0; q <= sl; ++q) {
            cs = q < kDescSlots ? (uint32_t)pd.cnt[q] : (uint32_t)gu16(rec + 2 * q);
            if (q < sl) {
              cc += cs;
              sbb += rt_bytes<TF>(cs);
            }
          }
          if (tr >= cs) continue;
          const int rrow = gu16(gs + (pd.off + 2u * ((uint32_t)w + tr)));
          const int rcol = gu16(gs + (cbase + 2u * (cc + tr)));
          RtBlock<TF> b;
          b.load(gs + sbb, cs, tr);
          TV x[3];
          rt_get3<TV, VS>(y, rcol, x);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            TV p = b.get(3 * a) * x[0];
            p = mac(b.get(3 * a + 1), x[1], p);
            p = mac(b.get(3 * a + 2), x[2], p);
            atomicAdd(&y[VS * rrow + a], -p);
          }
        }
      }
      __syncwarp();
      if constexpr (SYNC == 0) {
        mbar_arrive(mbar + (k - win0));
      } else {
        __threadfence_block();
        __syncwarp();
        if (active) rflag[row] = kind ? 2 : 1;
      }
    }
  }
  __syncthreads();
  if constexpr (SYNC == 0)
    for (int q = tid; q < k1 - win0; q += blockDim.x) mbar_inval(mbar + q);
  store_vector<TV, 3, VS>(cd, y, z, kscale);
}

// Kernel instances come per (factor type, block dimension BS, mapping RT):
// RT 1 is the row-thread layout (3x3 blocks, FP32 or BF16 factors, rows of at
// most kDescSlots blocks a side), RT 0 three threads per 3x3 row or one per
// scalar row. The plan's row_thread flag picks the instance at launch.
template <typename TF>
constexpr bool kHasRowThread = std::is_same<TF, float>::value || std::is_same<TF, bf16s>::value;

// Launch bounds of an apply instance (see kMaxRtThreads): the row-thread
// instances at up to 256 threads and three (FP32, 80 registers) or four
// (BF16, 64) blocks per SM; the three-thread and scalar instances at up to
// 384 threads and three (56 registers; at four, 40 registers, the scalar and
// FP64 instances spill and run slower).
template <typename TF, int BS, int RT>
struct ApplyLaunch {
  static_assert(!RT || (BS == 3 && kHasRowThread<TF>), "row-thread layout: 3x3 blocks, FP32 or BF16 factors");
  static constexpr int threads = RT ? kMaxRtThreads : kMaxApplyThreads;
  static constexpr int min_blocks =
      !RT ? kApplyMinBlocks : std::is_same<TF, float>::value ? kRtMinBlocksF32 : kRtMinBlocksBF16;
};

template <typename TF, int MODE, int BS, int RT>
__global__ void __launch_bounds__(ApplyLaunch<TF, BS, RT>::threads, ApplyLaunch<TF, BS, RT>::min_blocks)
    ildu0_apply_kernel(SysDesc S, const double* r, double* z, int sub0) {
  apply_block<TF, MODE, 0, BS, 0, 0, 0, RT>(S, sub0 + blockIdx.x, r, z);
}

// The plain apply with Algorithm 4's synchronization (row flags, bounded
// spin loops) instead of the per-level mbarriers: the same arithmetic in the
// same order, for the synchronization ablation.
template <typename TF, int BS, int RT>
__global__ void __launch_bounds__(ApplyLaunch<TF, BS, RT>::threads, ApplyLaunch<TF, BS, RT>::min_blocks)
    ildu0_apply_rowsync_kernel(SysDesc S, const double* r, double* z) {
  apply_block<TF, kModePlain, 0, BS, 1, 0, 0, RT>(S, blockIdx.x, r, z);
}

// The apply with the edge-centric traversal of the paper (threads over the
// blocks of a level, shared-memory atomics into the rows) instead of the
// row-wise one: the traversal ablation and the solver's opts.traversal = 1
// (FP64, FP32 and BF16 factors; every mode).
template <typename TF, int MODE, int BS, int RT>
__global__ void __launch_bounds__(ApplyLaunch<TF, BS, RT>::threads, ApplyLaunch<TF, BS, RT>::min_blocks)
    ildu0_apply_edge_kernel(SysDesc S, const double* r, double* z, int sub0) {
  apply_block<TF, MODE, 0, BS, 0, 1, 0, RT>(S, sub0 + blockIdx.x, r, z);
}

// The plain FP64 apply with the subdomain vector in global memory (z itself)
// instead of shared memory: the same arithmetic in the same order, for the
// shared-memory ablation.
template <int BS>
__global__ void __launch_bounds__(kMaxApplyThreads, kApplyMinBlocks)
    ildu0_apply_vglobal_kernel(SysDesc S, const double* r, double* z) {
  apply_block<double, kModePlain, 0, BS, 0, 0, 1>(S, blockIdx.x, r, z);
}

// The unfused apply's two launches (plain mode): PART 1 = L sweep, r -> z;
// PART 2 = D^-1 and U~ sweep, z -> z in place.
template <typename TF, int PART, int BS, int RT>
__global__ void __launch_bounds__(ApplyLaunch<TF, BS, RT>::threads, ApplyLaunch<TF, BS, RT>::min_blocks)
    ildu0_apply_part_kernel(SysDesc S, const double* r, double* z) {
  apply_block<TF, kModePlain, PART, BS, 0, 0, 0, RT>(S, blockIdx.x, r, z);
}

// Batched apply (modes P and S): persistent blocks walk (system, subdomain)
// items; every system of a batch has the same mapping.
template <typename TF, int MODE, int BS, int RT>
__global__ void __launch_bounds__(ApplyLaunch<TF, BS, RT>::threads, ApplyLaunch<TF, BS, RT>::min_blocks)
    ildu0_apply_batched(const SysDesc* __restrict__ sys, const BatchItem* __restrict__ items, int64_t nitems) {
  for (int64_t i = blockIdx.x; i < nitems; i += gridDim.x) {
    const BatchItem it = items[i];
    const SysDesc& S = sys[it.sys];
    apply_block<TF, MODE, 0, BS, 0, 0, 0, RT>(S, it.local, S.vec[kVecR], S.vec[MODE == kModeP ? kVecPh : kVecSh]);
    __syncthreads();  // the next item reuses shared memory
  }
}

template <typename TF, int MODE, int BS, int RT>
static cudaError_t configure_layout(int sm) {
  constexpr cudaFuncAttribute kSmem = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(ildu0_apply_kernel<TF, MODE, BS, RT>, kSmem, sm);
  if (e == cudaSuccess && MODE != kModePlain) e = cudaFuncSetAttribute(ildu0_apply_batched<TF, MODE, BS, RT>, kSmem, sm);
  if constexpr (MODE == kModePlain) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(ildu0_apply_part_kernel<TF, 1, BS, RT>, kSmem, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(ildu0_apply_part_kernel<TF, 2, BS, RT>, kSmem, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(ildu0_apply_rowsync_kernel<TF, BS, RT>, kSmem, sm);
    if constexpr (std::is_same<TF, double>::value)
      if (e == cudaSuccess) e = cudaFuncSetAttribute(ildu0_apply_vglobal_kernel<BS>, kSmem, sm);
  }
  if constexpr (!std::is_same<TF, df64s>::value)
    if (e == cudaSuccess) e = cudaFuncSetAttribute(ildu0_apply_edge_kernel<TF, MODE, BS, RT>, kSmem, sm);
  return e;
}

template <typename TF, int MODE>
static cudaError_t configure_one(size_t smem) {
  const int sm = (int)smem;
  cudaError_t e = configure_layout<TF, MODE, 3, 0>(sm);
  if (e == cudaSuccess) e = configure_layout<TF, MODE, 1, 0>(sm);
  if constexpr (kHasRowThread<TF>)
    if (e == cudaSuccess) e = configure_layout<TF, MODE, 3, 1>(sm);
  return e;
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
  const size_t smem = (size_t)optin - kApplyStaticSmem;  // minus the kernel's static shared memory
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
  acc(configure_one<df64s, kModePlain>(smem));
  acc(configure_one<df64s, kModeP>(smem));
  acc(configure_one<df64s, kModeS>(smem));
  return e;
}

// Calls L.template run<BS, RT>() for the instance that fits a system with
// block dimension bs and row-thread flag rt.
template <typename TF, typename L>
static cudaError_t by_layout(int bs, int rt, const L& l) {
  if (bs == 1) return l.template run<1, 0>();
  if constexpr (kHasRowThread<TF>)
    if (rt) return l.template run<3, 1>();
  return l.template run<3, 0>();
}

template <typename TF>
struct ApplyRun {
  const DevCtx& d;
  int mode;
  const double* r;
  double* z;
  int sub0, nsub;
  cudaStream_t s;
  template <int BS, int RT>
  cudaError_t run() const {
    dim3 grid(nsub), block(d.threads);
    if constexpr (!std::is_same<TF, df64s>::value) {
      if (d.traversal == 1) {  // edge-centric (opts.traversal)
        if (mode == kModePlain)
          ildu0_apply_edge_kernel<TF, kModePlain, BS, RT><<<grid, block, d.smem_bytes, s>>>(d.sd, r, z, sub0);
        else if (mode == kModeP)
          ildu0_apply_edge_kernel<TF, kModeP, BS, RT><<<grid, block, d.smem_bytes, s>>>(d.sd, r, z, sub0);
        else
          ildu0_apply_edge_kernel<TF, kModeS, BS, RT><<<grid, block, d.smem_bytes, s>>>(d.sd, r, z, sub0);
        return cudaGetLastError();
      }
    }
    if (mode == kModePlain)
      ildu0_apply_kernel<TF, kModePlain, BS, RT><<<grid, block, d.smem_bytes, s>>>(d.sd, r, z, sub0);
    else if (mode == kModeP)
      ildu0_apply_kernel<TF, kModeP, BS, RT><<<grid, block, d.smem_bytes, s>>>(d.sd, r, z, sub0);
    else
      ildu0_apply_kernel<TF, kModeS, BS, RT><<<grid, block, d.smem_bytes, s>>>(d.sd, r, z, sub0);
    return cudaGetLastError();
  }
};

template <typename TF>
static cudaError_t launch_apply_t(const DevCtx& d, int mode, const double* r, double* z, int sub0, int nsub,
                                  cudaStream_t s) {
  return by_layout<TF>(d.bs, d.sd.row_thread, ApplyRun<TF>{d, mode, r, z, sub0, nsub, s});
}

cudaError_t launch_apply_range(const DevCtx& d, int mode, const double* r, double* z, int sub0, int nsub,
                               cudaStream_t s) {
  if (nsub <= 0) return cudaSuccess;
  if (d.factor_prec == ILU0DD_F64) return launch_apply_t<double>(d, mode, r, z, sub0, nsub, s);
  if (d.factor_prec == ILU0DD_F32) return launch_apply_t<float>(d, mode, r, z, sub0, nsub, s);
  if (d.factor_prec == ILU0DD_DF64) return launch_apply_t<df64s>(d, mode, r, z, sub0, nsub, s);
  return launch_apply_t<bf16s>(d, mode, r, z, sub0, nsub, s);
}

cudaError_t launch_apply(const DevCtx& d, int mode, const double* r, double* z, cudaStream_t s) {
  return launch_apply_range(d, mode, r, z, 0, d.sd.nsub, s);
}

template <typename TF>
struct UnfusedRun {
  const DevCtx& d;
  const double* r;
  double* z;
  cudaStream_t s;
  template <int BS, int RT>
  cudaError_t run() const {
    dim3 grid(d.sd.nsub), block(d.threads);
    ildu0_apply_part_kernel<TF, 1, BS, RT><<<grid, block, d.smem_bytes, s>>>(d.sd, r, z);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ildu0_apply_part_kernel<TF, 2, BS, RT><<<grid, block, d.smem_bytes, s>>>(d.sd, z, z);
    return cudaGetLastError();
  }
};

template <typename TF>
static cudaError_t launch_unfused_t(const DevCtx& d, const double* r, double* z, cudaStream_t s) {
  return by_layout<TF>(d.bs, d.sd.row_thread, UnfusedRun<TF>{d, r, z, s});
}

cudaError_t launch_apply_unfused(const DevCtx& d, const double* r, double* z, cudaStream_t s) {
  if (d.sd.nsub == 0) return cudaSuccess;
  if (d.factor_prec == ILU0DD_F64) return launch_unfused_t<double>(d, r, z, s);
  if (d.factor_prec == ILU0DD_F32) return launch_unfused_t<float>(d, r, z, s);
  if (d.factor_prec == ILU0DD_DF64) return launch_unfused_t<df64s>(d, r, z, s);
  return launch_unfused_t<bf16s>(d, r, z, s);
}

template <typename TF>
struct RowsyncRun {
  const DevCtx& d;
  const double* r;
  double* z;
  cudaStream_t s;
  template <int BS, int RT>
  cudaError_t run() const {
    ildu0_apply_rowsync_kernel<TF, BS, RT><<<d.sd.nsub, d.threads, d.smem_rowsync, s>>>(d.sd, r, z);
    return cudaGetLastError();
  }
};

cudaError_t launch_apply_rowsync(const DevCtx& d, const double* r, double* z, cudaStream_t s) {
  if (d.sd.nsub == 0) return cudaSuccess;
  const int bs = d.bs, rt = d.sd.row_thread;
  if (d.factor_prec == ILU0DD_F64) return by_layout<double>(bs, rt, RowsyncRun<double>{d, r, z, s});
  if (d.factor_prec == ILU0DD_F32) return by_layout<float>(bs, rt, RowsyncRun<float>{d, r, z, s});
  if (d.factor_prec == ILU0DD_DF64) return by_layout<df64s>(bs, rt, RowsyncRun<df64s>{d, r, z, s});
  return by_layout<bf16s>(bs, rt, RowsyncRun<bf16s>{d, r, z, s});
}

template <typename TF>
struct EdgeRun {
  const DevCtx& d;
  const double* r;
  double* z;
  cudaStream_t s;
  template <int BS, int RT>
  cudaError_t run() const {
    ildu0_apply_edge_kernel<TF, kModePlain, BS, RT><<<d.sd.nsub, d.threads, d.smem_bytes, s>>>(d.sd, r, z, 0);
    return cudaGetLastError();
  }
};

cudaError_t launch_apply_vglobal(const DevCtx& d, const double* r, double* z, cudaStream_t s) {
  if (d.sd.nsub == 0) return cudaSuccess;
  if (d.factor_prec != ILU0DD_F64) return cudaErrorInvalidValue;
  if (d.bs == 1)
    ildu0_apply_vglobal_kernel<1><<<d.sd.nsub, d.threads, d.smem_bytes, s>>>(d.sd, r, z);
  else
    ildu0_apply_vglobal_kernel<3><<<d.sd.nsub, d.threads, d.smem_bytes, s>>>(d.sd, r, z);
  return cudaGetLastError();
}

cudaError_t launch_apply_edge(const DevCtx& d, const double* r, double* z, cudaStream_t s) {
  if (d.sd.nsub == 0) return cudaSuccess;
  const int bs = d.bs, rt = d.sd.row_thread;
  if (d.factor_prec == ILU0DD_F64) return by_layout<double>(bs, rt, EdgeRun<double>{d, r, z, s});
  if (d.factor_prec == ILU0DD_F32) return by_layout<float>(bs, rt, EdgeRun<float>{d, r, z, s});
  if (d.factor_prec == ILU0DD_BF16) return by_layout<bf16s>(bs, rt, EdgeRun<bf16s>{d, r, z, s});
  return cudaErrorInvalidValue;  // DF64 pairs have no atomic add
}

template <typename TF>
struct BatchedRun {
  const SysDesc* sys;
  const BatchItem* items;
  int64_t nitems;
  int mode, threads;
  size_t smem;
  int grid;
  cudaStream_t s;
  template <int BS, int RT>
  cudaError_t run() const {
    if (mode == kModeP)
      ildu0_apply_batched<TF, kModeP, BS, RT><<<grid, threads, smem, s>>>(sys, items, nitems);
    else
      ildu0_apply_batched<TF, kModeS, BS, RT><<<grid, threads, smem, s>>>(sys, items, nitems);
    return cudaGetLastError();
  }
};

cudaError_t launch_apply_batched(const SysDesc* sys, const BatchItem* items, int64_t nitems, int mode,
                                 int factor_prec, int bs, int row_thread, int threads, size_t smem, int grid,
                                 cudaStream_t s) {
  if (nitems == 0) return cudaSuccess;
  const int rt = row_thread;
  if (factor_prec == ILU0DD_F64)
    return by_layout<double>(bs, rt, BatchedRun<double>{sys, items, nitems, mode, threads, smem, grid, s});
  if (factor_prec == ILU0DD_F32)
    return by_layout<float>(bs, rt, BatchedRun<float>{sys, items, nitems, mode, threads, smem, grid, s});
  if (factor_prec == ILU0DD_DF64)
    return by_layout<df64s>(bs, rt, BatchedRun<df64s>{sys, items, nitems, mode, threads, smem, grid, s});
  return by_layout<bf16s>(bs, rt, BatchedRun<bf16s>{sys, items, nitems, mode, threads, smem, grid, s});
}

template <typename TF>
struct OccupancyRun {
  int* n;
  int threads;
  size_t smem;
  template <int BS, int RT>
  cudaError_t run() const {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, ildu0_apply_batched<TF, kModeP, BS, RT>, threads, smem);
  }
};

int apply_blocks_per_sm(int factor_prec, int bs, int row_thread, int threads, size_t smem) {
  int n = 0;
  cudaError_t e;
  if (factor_prec == ILU0DD_F64)
    e = by_layout<double>(bs, row_thread, OccupancyRun<double>{&n, threads, smem});
  else if (factor_prec == ILU0DD_F32)
    e = by_layout<float>(bs, row_thread, OccupancyRun<float>{&n, threads, smem});
  else if (factor_prec == ILU0DD_DF64)
    e = by_layout<df64s>(bs, row_thread, OccupancyRun<df64s>{&n, threads, smem});
  else
    e = by_layout<bf16s>(bs, row_thread, OccupancyRun<bf16s>{&n, threads, smem});
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

// ===========================================================================
// Reductions: last-block completion
// ===========================================================================

// Write this tile's partials; returns true in every thread of the block that
// completed the `count`-th tile of the reduction (it owns the final sum).
template <int NV>
__device__ __forceinline__ bool publish_partials(const double (&q)[NV], double* partials, int64_t stride,
                                                 int64_t tile, int64_t count, uint32_t* counter) {
  __shared__ unsigned int s_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) partials[v * stride + tile] = q[v];
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    s_last = prev == (unsigned int)(count - 1);
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

// ===========================================================================
// SpMV (sliced ELL), kinds: 0 plain, 1 (rh . v) -> alpha, 2 (t . s), (t . t) -> omega
// ===========================================================================
template <int KIND, int BS = 3>
__device__ __forceinline__ void spmv_block(const SysDesc& S, int64_t tile, const double* x, double* y) {
  if (KIND != 0 && S.scal->done) return;
  constexpr int BB = BS * BS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t slice = tile * (kDotTile / kSlice) + warp;
  const int64_t row = slice * kSlice + lane;
  double yv[BS];
#pragma unroll
  for (int a = 0; a < BS; ++a) yv[a] = 0.0;
  if (slice < S.nslices) {
    const int64_t so = S.slice_off[slice];
    const int w = S.slice_off[slice + 1] - (int32_t)so;
    const int32_t* cp = S.sell_col + so * kSlice + lane;
    const double* vp = S.sell_val + so * BB * kSlice + lane;
    for (int sl = 0; sl < w; ++sl) {
      const int c = __ldg(cp + sl * kSlice);
      double b[BB];
#pragma unroll
      for (int e = 0; e < BB; ++e) b[e] = __ldg(vp + (sl * BB + e) * kSlice);
      // per output entry a: blocks in slot order, within a block c = 0..BS-1
#pragma unroll
      for (int cc = 0; cc < BS; ++cc) {
        const double xc = x[(int64_t)BS * c + cc];
#pragma unroll
        for (int a = 0; a < BS; ++a) yv[a] = fma(b[BS * a + cc], xc, yv[a]);
      }
    }
    if (row < S.N) {
#pragma unroll
      for (int a = 0; a < BS; ++a) y[BS * row + a] = yv[a];
    }
  }
  if (KIND == 0) return;
  __shared__ double buf[2][kDotTile];
  const bool in = row < S.N;
  const int64_t m = S.ntiles_pow2;
  if (KIND == 1) {
    const double* w = S.vec[kVecRh];
    double wv[BS];
#pragma unroll
    for (int a = 0; a < BS; ++a) wv[a] = in ? w[BS * row + a] : 0.0;
    double q[1] = {in ? reg_dot<BS>(wv, yv) : 0.0};
    tile_halving_sum<1>(q, buf);
    uint32_t* counter = S.counters + kCntSpmvV;
    if (!publish_partials<1>(q, S.partials, m, tile, S.ntiles, counter)) return;
    double out[1];
    finish_sum<1>(S.partials, m, m, out, buf);
    if (threadIdx.x == 0) {
      SolverScalars* sc = S.scal;
      const double rv = out[0];
      sc->rv = rv;
      if (rv == 0.0 || !finite(rv)) {
        sc->status = ILU0DD_ERR_BREAKDOWN;
        sc->done = 1;
      } else {
        sc->alpha = sc->rho / rv;
      }
      *counter = 0;
    }
  } else {
    // (t . s) and (t . t), t = y
    const double* w = S.vec[kVecS];
    double wv[BS];
#pragma unroll
    for (int a = 0; a < BS; ++a) wv[a] = in ? w[BS * row + a] : 0.0;
    double q[2] = {in ? reg_dot<BS>(yv, wv) : 0.0, in ? reg_dot<BS>(yv, yv) : 0.0};
    tile_halving_sum<2>(q, buf);
    uint32_t* counter = S.counters + kCntSpmvT;
    if (!publish_partials<2>(q, S.partials, m, tile, S.ntiles, counter)) return;
    double out[2];
    finish_sum<2>(S.partials, m, m, out, buf);
    if (threadIdx.x == 0) {
      SolverScalars* sc = S.scal;
      sc->ts = out[0];
      sc->tt = out[1];
      sc->omega = out[1] == 0.0 ? 0.0 : out[0] / out[1];
      *counter = 0;
    }
  }
}

template <int KIND, int BS>
__global__ void __launch_bounds__(kDotTile) sell_spmv_kernel(SysDesc S, const double* x, double* y) {
  spmv_block<KIND, BS>(S, blockIdx.x, x, y);
}

template <int KIND, int BS>
__global__ void __launch_bounds__(kDotTile)
    sell_spmv_batched(const SysDesc* __restrict__ sys, const BatchItem* __restrict__ items, int64_t nitems) {
  for (int64_t i = blockIdx.x; i < nitems; i += gridDim.x) {
    const BatchItem it = items[i];
    const SysDesc& S = sys[it.sys];
    if (KIND == 0)
      spmv_block<0, BS>(S, it.local, S.vec[kVecX], S.vec[kVecT]);
    else if (KIND == 1)
      spmv_block<1, BS>(S, it.local, S.vec[kVecPh], S.vec[kVecV]);
    else
      spmv_block<2, BS>(S, it.local, S.vec[kVecSh], S.vec[kVecT]);
    __syncthreads();
  }
}

template <int BS>
static cudaError_t launch_spmv_b(const DevCtx& d, int kind, const double* x, double* y, cudaStream_t s) {
  dim3 grid((unsigned)d.sd.ntiles), block(kDotTile);
  if (kind == 0)
    sell_spmv_kernel<0, BS><<<grid, block, 0, s>>>(d.sd, x, y);
  else if (kind == 1)
    sell_spmv_kernel<1, BS><<<grid, block, 0, s>>>(d.sd, x, y);
  else
    sell_spmv_kernel<2, BS><<<grid, block, 0, s>>>(d.sd, x, y);
  return cudaGetLastError();
}

cudaError_t launch_spmv(const DevCtx& d, int kind, const double* x, double* y, cudaStream_t s) {
  if (d.sd.N == 0) return cudaSuccess;
  return d.bs == 1 ? launch_spmv_b<1>(d, kind, x, y, s) : launch_spmv_b<3>(d, kind, x, y, s);
}

template <int BS>
static cudaError_t launch_spmv_batched_b(const SysDesc* sys, const BatchItem* items, int64_t nitems, int kind,
                                         int grid, cudaStream_t s) {
  if (kind == 0)
    sell_spmv_batched<0, BS><<<grid, kDotTile, 0, s>>>(sys, items, nitems);
  else if (kind == 1)
    sell_spmv_batched<1, BS><<<grid, kDotTile, 0, s>>>(sys, items, nitems);
  else
    sell_spmv_batched<2, BS><<<grid, kDotTile, 0, s>>>(sys, items, nitems);
  return cudaGetLastError();
}

cudaError_t launch_spmv_batched(const SysDesc* sys, const BatchItem* items, int64_t nitems, int kind, int bs,
                                int grid, cudaStream_t s) {
  if (nitems == 0) return cudaSuccess;
  return bs == 1 ? launch_spmv_batched_b<1>(sys, items, nitems, kind, grid, s)
                 : launch_spmv_batched_b<3>(sys, items, nitems, kind, grid, s);
}

// ===========================================================================
// Vector steps
// ===========================================================================

// x += alpha ph + omega sh; r = s - omega t; then ||r||/||b|| and rho.
template <int BS = 3>
__device__ __forceinline__ void update_block(const SysDesc& S, int64_t tile) {
  SolverScalars* sc = S.scal;
  if (sc->done) return;
  const int64_t i = tile * kDotTile + threadIdx.x;
  const double alpha = sc->alpha, omega = sc->omega;
  double q[2] = {0.0, 0.0};
  if (i < S.N) {
    double* x = S.vec[kVecX];
    double* r = S.vec[kVecR];
    const double* ph = S.vec[kVecPh];
    const double* sh = S.vec[kVecSh];
    const double* sv = S.vec[kVecS];
    const double* t = S.vec[kVecT];
    const double* rh = S.vec[kVecRh];
    double rr[BS], rhv[BS];
#pragma unroll
    for (int c = 0; c < BS; ++c) {
      const int64_t e = BS * i + c;
      x[e] = fma(omega, sh[e], fma(alpha, ph[e], x[e]));
      rr[c] = fma(-omega, t[e], sv[e]);
      r[e] = rr[c];
      rhv[c] = rh[e];
    }
    q[0] = reg_dot<BS>(rr, rr);
    q[1] = reg_dot<BS>(rhv, rr);
  }
  __shared__ double buf[2][kDotTile];
  tile_halving_sum<2>(q, buf);
  uint32_t* counter = S.counters + kCntUpdate;
  if (!publish_partials<2>(q, S.partials, S.ntiles_pow2, tile, S.ntiles, counter)) return;
  double out[2];
  finish_sum<2>(S.partials, S.ntiles_pow2, S.ntiles_pow2, out, buf);
  if (threadIdx.x == 0) {
    const double rr = out[0], rho_new = out[1];
    const double rel = sqrt(rr) / sqrt(sc->bb);
    sc->rr = rr;
    sc->rhr = rho_new;
    sc->rel = rel;
    sc->iter += 1;
    if (sc->iter <= sc->maxit) S.hist[sc->iter] = rel;
    if (!finite(rel)) {
      sc->status = ILU0DD_ERR_BREAKDOWN;
      sc->done = 1;
    } else if (rel < sc->rtol) {
      sc->converged = 1;
      sc->done = 1;
    } else if (sc->iter >= sc->maxit) {
      sc->status = ILU0DD_ERR_NOT_CONVERGED;
      sc->done = 1;
    } else if (rho_new == 0.0 || omega == 0.0 || !finite(rho_new)) {
      sc->status = ILU0DD_ERR_BREAKDOWN;
      sc->done = 1;
    } else {
      sc->beta = (alpha / omega) * (rho_new / sc->rho);
      sc->rho = rho_new;
    }
    *counter = 0;
  }
}

// x = 0, r = rh = p = b, v = 0; bb = rho = (b . b).
template <int BS = 3>
__device__ __forceinline__ void init_block(const SysDesc& S, int64_t tile, double rtol, int32_t maxit) {
  const int64_t i = tile * kDotTile + threadIdx.x;
  double q[1] = {0.0};
  if (i < S.N) {
    const double* b = S.vec[kVecB];
#pragma unroll
    for (int c = 0; c < BS; ++c) {
      const int64_t e = BS * i + c;
      const double be = b[e];
      S.vec[kVecX][e] = 0.0;
      S.vec[kVecR][e] = be;
      S.vec[kVecRh][e] = be;
      S.vec[kVecP][e] = be;
      S.vec[kVecV][e] = 0.0;
    }
    q[0] = row_dot<BS>(b, b, i);
  }
  __shared__ double buf[1][kDotTile];
  tile_halving_sum<1>(q, buf);
  uint32_t* counter = S.counters + kCntInit;
  if (!publish_partials<1>(q, S.partials, S.ntiles_pow2, tile, S.ntiles, counter)) return;
  double out[1];
  finish_sum<1>(S.partials, S.ntiles_pow2, S.ntiles_pow2, out, buf);
  if (threadIdx.x == 0) {
    SolverScalars* sc = S.scal;
    const double bb = out[0];
    sc->bb = bb;
    sc->rho = bb;
    sc->alpha = sc->beta = sc->omega = 0.0;
    sc->rv = sc->ts = sc->tt = sc->rr = sc->rhr = 0.0;
    sc->rel = 1.0;
    sc->rel_true = 1.0;
    sc->rtol = rtol;
    sc->maxit = maxit;
    sc->iter = 0;
    sc->converged = 0;
    sc->status = ILU0DD_OK;
    sc->done = 0;
    S.hist[0] = 1.0;
    if (!finite(bb)) {
      sc->status = ILU0DD_ERR_NONFINITE;
      sc->done = 1;
    } else if (bb == 0.0) {
      sc->converged = 1;
      sc->rel = 0.0;
      sc->rel_true = 0.0;
      sc->done = 1;
    } else if (maxit <= 0) {
      sc->status = ILU0DD_ERR_NOT_CONVERGED;
      sc->done = 1;
    }
    *counter = 0;
  }
}

// r = b - t (t = A x computed before), rel_true = ||r||/||b||.
template <int BS = 3>
__device__ __forceinline__ void residual_block(const SysDesc& S, int64_t tile) {
  const int64_t i = tile * kDotTile + threadIdx.x;
  double q[1] = {0.0};
  if (i < S.N) {
    double rr[BS];
#pragma unroll
    for (int c = 0; c < BS; ++c) {
      const int64_t e = BS * i + c;
      rr[c] = S.vec[kVecB][e] - S.vec[kVecT][e];
      S.vec[kVecR][e] = rr[c];
    }
    q[0] = reg_dot<BS>(rr, rr);
  }
  __shared__ double buf[1][kDotTile];
  tile_halving_sum<1>(q, buf);
  uint32_t* counter = S.counters + kCntResid;
  if (!publish_partials<1>(q, S.partials, S.ntiles_pow2, tile, S.ntiles, counter)) return;
  double out[1];
  finish_sum<1>(S.partials, S.ntiles_pow2, S.ntiles_pow2, out, buf);
  if (threadIdx.x == 0) {
    const double bb = S.scal->bb;
    S.scal->rr = out[0];
    // b = 0: x = 0 is exact (rel_true 0); otherwise ||r|| / ||b||
    S.scal->rel_true = bb > 0.0 ? sqrt(out[0]) / sqrt(bb) : (out[0] == 0.0 ? 0.0 : HUGE_VAL);
    *counter = 0;
  }
}

// Continue from r: rh = p = r, v = 0, rho = (r . r) of the true residual, done = 0.
template <int BS = 3>
__device__ __forceinline__ void restart_block(const SysDesc& S, int64_t tile) {
  const int64_t i = tile * kDotTile + threadIdx.x;
  if (i < S.N) {
#pragma unroll
    for (int c = 0; c < BS; ++c) {
      const int64_t e = BS * i + c;
      const double re = S.vec[kVecR][e];
      S.vec[kVecRh][e] = re;
      S.vec[kVecP][e] = re;
      S.vec[kVecV][e] = 0.0;
    }
  }
  if (tile == 0 && threadIdx.x == 0) {
    SolverScalars* sc = S.scal;
    sc->rho = sc->rr;
    sc->alpha = sc->beta = sc->omega = 0.0;
    sc->converged = 0;
    sc->done = 0;
  }
}

template <int BS>
__global__ void __launch_bounds__(kDotTile) update_kernel(SysDesc S) { update_block<BS>(S, blockIdx.x); }

template <int BS>
__global__ void __launch_bounds__(kDotTile) init_kernel(SysDesc S, double rtol, int32_t maxit) {
  init_block<BS>(S, blockIdx.x, rtol, maxit);
}

template <int BS>
__global__ void __launch_bounds__(kDotTile) residual_kernel(SysDesc S, int restart) {
  if (restart)
    restart_block<BS>(S, blockIdx.x);
  else
    residual_block<BS>(S, blockIdx.x);
}

template <int BS>
__global__ void __launch_bounds__(kDotTile)
    update_batched(const SysDesc* __restrict__ sys, const BatchItem* __restrict__ items, int64_t nitems) {
  for (int64_t i = blockIdx.x; i < nitems; i += gridDim.x) {
    const BatchItem it = items[i];
    update_block<BS>(sys[it.sys], it.local);
    __syncthreads();
  }
}

template <int BS>
__global__ void __launch_bounds__(kDotTile)
    vec_batched(const SysDesc* __restrict__ sys, const BatchItem* __restrict__ items, int64_t nitems, int mode,
                double rtol, int32_t maxit, const int32_t* __restrict__ flags) {
  for (int64_t i = blockIdx.x; i < nitems; i += gridDim.x) {
    const BatchItem it = items[i];
    if (flags && !flags[it.sys]) continue;  // uniform per item
    const SysDesc& S = sys[it.sys];
    if (mode == 0)
      init_block<BS>(S, it.local, rtol, maxit);
    else if (mode == 1)
      residual_block<BS>(S, it.local);
    else
      restart_block<BS>(S, it.local);
    __syncthreads();
  }
}

cudaError_t launch_update(const DevCtx& d, cudaStream_t s) {
  if (d.sd.N == 0) return cudaSuccess;
  if (d.bs == 1)
    update_kernel<1><<<(unsigned)d.sd.ntiles, kDotTile, 0, s>>>(d.sd);
  else
    update_kernel<3><<<(unsigned)d.sd.ntiles, kDotTile, 0, s>>>(d.sd);
  return cudaGetLastError();
}

cudaError_t launch_init(const DevCtx& d, double rtol, int32_t maxit, cudaStream_t s) {
  if (d.sd.N == 0) return cudaSuccess;
  if (d.bs == 1)
    init_kernel<1><<<(unsigned)d.sd.ntiles, kDotTile, 0, s>>>(d.sd, rtol, maxit);
  else
    init_kernel<3><<<(unsigned)d.sd.ntiles, kDotTile, 0, s>>>(d.sd, rtol, maxit);
  return cudaGetLastError();
}

cudaError_t launch_residual(const DevCtx& d, int restart, cudaStream_t s) {
  if (d.sd.N == 0) return cudaSuccess;
  if (d.bs == 1)
    residual_kernel<1><<<(unsigned)d.sd.ntiles, kDotTile, 0, s>>>(d.sd, restart);
  else
    residual_kernel<3><<<(unsigned)d.sd.ntiles, kDotTile, 0, s>>>(d.sd, restart);
  return cudaGetLastError();
}

cudaError_t launch_update_batched(const SysDesc* sys, const BatchItem* items, int64_t nitems, int bs, int grid,
                                  cudaStream_t s) {
  if (nitems == 0) return cudaSuccess;
  if (bs == 1)
    update_batched<1><<<grid, kDotTile, 0, s>>>(sys, items, nitems);
  else
    update_batched<3><<<grid, kDotTile, 0, s>>>(sys, items, nitems);
  return cudaGetLastError();
}

cudaError_t launch_vec_batched(const SysDesc* sys, const BatchItem* items, int64_t nitems, int mode, double rtol,
                               int32_t maxit, const int32_t* flags, int bs, int grid, cudaStream_t s) {
  if (nitems == 0) return cudaSuccess;
  if (bs == 1)
    vec_batched<1><<<grid, kDotTile, 0, s>>>(sys, items, nitems, mode, rtol, maxit, flags);
  else
    vec_batched<3><<<grid, kDotTile, 0, s>>>(sys, items, nitems, mode, rtol, maxit, flags);
  return cudaGetLastError();
}

int tile_blocks_per_sm(int bs) {
  int n = 0;
  cudaError_t e = bs == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sell_spmv_batched<2, 1>, kDotTile, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sell_spmv_batched<2, 3>, kDotTile, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

// ===========================================================================
// Standalone dot product, permutation, status
// ===========================================================================
template <int BS>
__global__ void __launch_bounds__(kDotTile) dot_kernel(const double* x, const double* y, int32_t N, double* partials,
                                                       int64_t m, uint32_t* counter, double* out_p) {
  const int64_t i = (int64_t)blockIdx.x * kDotTile + threadIdx.x;
  double q[1] = {i < N ? row_dot<BS>(x, y, i) : 0.0};
  __shared__ double buf[1][kDotTile];
  tile_halving_sum<1>(q, buf);
  if (!publish_partials<1>(q, partials, m, blockIdx.x, gridDim.x, counter)) return;
  double out[1];
  finish_sum<1>(partials, m, m, out, buf);
  if (threadIdx.x == 0) {
    *out_p = out[0];
    *counter = 0;
  }
}

cudaError_t launch_dot(const DevCtx& d, const double* x, const double* y, double* out, cudaStream_t s) {
  if (d.sd.N == 0) return cudaMemsetAsync(out, 0, sizeof(double), s);
  if (d.bs == 1)
    dot_kernel<1><<<(unsigned)d.sd.ntiles, kDotTile, 0, s>>>(x, y, d.sd.N, d.sd.partials, d.sd.ntiles_pow2,
                                                              d.sd.counters + kCntDot, out);
  else
    dot_kernel<3><<<(unsigned)d.sd.ntiles, kDotTile, 0, s>>>(x, y, d.sd.N, d.sd.partials, d.sd.ntiles_pow2,
                                                              d.sd.counters + kCntDot, out);
  return cudaGetLastError();
}

cudaError_t launch_dot_scratch(const double* x, const double* y, int32_t n_brows, double* partials, int64_t m,
                               uint32_t* counter, double* out, cudaStream_t s) {
  const int64_t ntiles = ((int64_t)n_brows + kDotTile - 1) / kDotTile;
  dot_kernel<3><<<(unsigned)ntiles, kDotTile, 0, s>>>(x, y, n_brows, partials, m, counter, out);
  return cudaGetLastError();
}

// out[i] = in[map[i]] (BS doubles per row): map = perm gathers natural -> reordered,
// map = iperm gathers reordered -> natural.
template <int BS = 3>
__device__ __forceinline__ void gather_rows(const double* in, double* out, const int32_t* map, int64_t i) {
  const int64_t j = map[i];
#pragma unroll
  for (int c = 0; c < BS; ++c) out[BS * i + c] = in[BS * j + c];
}

template <int BS>
__global__ void permute_kernel(const double* in, double* out, const int32_t* map, int32_t N) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) gather_rows<BS>(in, out, map, i);
}

cudaError_t launch_permute(const DevCtx& d, const double* in, double* out, int dir, cudaStream_t s) {
  if (d.sd.N == 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = (unsigned)((d.sd.N + threads - 1) / threads);
  if (d.bs == 1)
    permute_kernel<1><<<blocks, threads, 0, s>>>(in, out, dir == 0 ? d.sd.perm : d.sd.iperm, d.sd.N);
  else
    permute_kernel<3><<<blocks, threads, 0, s>>>(in, out, dir == 0 ? d.sd.perm : d.sd.iperm, d.sd.N);
  return cudaGetLastError();
}

// Tile items of 256 rows; dir 0: vec B <- ptrs[sys] permuted; dir 1: ptrs[sys] <- vec X natural.
template <int BS>
__global__ void __launch_bounds__(kDotTile)
    permute_batched(const SysDesc* __restrict__ sys, const BatchItem* __restrict__ items, int64_t nitems,
                    const double* const* __restrict__ ptrs, int dir) {
  for (int64_t k = blockIdx.x; k < nitems; k += gridDim.x) {
    const BatchItem it = items[k];
    const SysDesc& S = sys[it.sys];
    const int64_t i = (int64_t)it.local * kDotTile + threadIdx.x;
    if (i >= S.N) continue;
    if (dir == 0)
      gather_rows<BS>(ptrs[it.sys], S.vec[kVecB], S.perm, i);
    else
      gather_rows<BS>(S.vec[kVecX], const_cast<double*>(ptrs[it.sys]), S.iperm, i);
  }
}

cudaError_t launch_permute_batched(const SysDesc* sys, const BatchItem* items, int64_t nitems,
                                   const double* const* ptrs, int dir, int bs, int grid, cudaStream_t s) {
  if (nitems == 0) return cudaSuccess;
  if (bs == 1)
    permute_batched<1><<<grid, kDotTile, 0, s>>>(sys, items, nitems, ptrs, dir);
  else
    permute_batched<3><<<grid, kDotTile, 0, s>>>(sys, items, nitems, ptrs, dir);
  return cudaGetLastError();
}

// A system whose device error word is set (an apply wait expired) reports
// ILU0DD_ERR_DEVICE_WAIT in its gathered status.
__global__ void gather_status(const SysDesc* __restrict__ sys, int32_t nsys, SolverScalars* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nsys) {
    SolverScalars h = *sys[i].scal;
    if (*sys[i].err != 0) h.status = ILU0DD_ERR_DEVICE_WAIT;
    out[i] = h;
  }
}

cudaError_t launch_gather_status(const SysDesc* sys, int32_t nsys, SolverScalars* out, cudaStream_t s) {
  if (nsys == 0) return cudaSuccess;
  gather_status<<<(nsys + 127) / 128, 128, 0, s>>>(sys, nsys, out);
  return cudaGetLastError();
}

}  // namespace ilu0dd
