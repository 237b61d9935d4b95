// Device-side numeric setup (the alternative to factor_ildu0 + pack_stream +
// pack_sell on the host): gather of the kept blocks, block ILU0 of every
// subdomain (Algorithm 7, IKJ form) level-scheduled with one thread block per
// subdomain and one thread per row of an L level (rows of a level depend only
// on rows of earlier levels), and the packing of the factor stream and of the
// sliced-ELL SpMV matrix straight into the workspace.
//
// Every floating-point step repeats the host setup's operations in the same
// order, and this file is compiled without contraction (--fmad=false), so
// the device and host setups produce the same bits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <thread>
#include <vector>

#include "internal.h"
#include "setup_dev.h"

namespace ilu0dd {

namespace {

inline size_t align256(size_t v) { return (v + 255) / 256 * 256; }

template <typename F>
void host_parallel_for(int64_t n, F&& f) {
  unsigned hw = std::thread::hardware_concurrency();
  int64_t nt = std::max<int64_t>(1, std::min<int64_t>(hw ? hw : 1, n));
  if (nt <= 1) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::vector<std::thread> th;
  for (int64_t t = 0; t < nt; ++t)
    th.emplace_back([&, t] {
      for (int64_t i = n * t / nt; i < n * (t + 1) / nt; ++i) f(i);
    });
  for (auto& x : th) x.join();
}

// Scratch regions (byte offsets), all 256-aligned.
struct ScratchLayout {
  size_t aval, w, invd, dd_src, dd_rp, dd_col, ap_rp, ap_col, ap_src, order, lev_off, lptr, prow_off, prows,
      piece_sub, flags, total;
};

ScratchLayout scratch_layout(const Plan& p, int64_t total_levels, int64_t total_prows) {
  ScratchLayout L{};
  size_t cur = 0;
  auto take = [&](size_t bytes) {
    size_t at = cur;
    cur = align256(cur + std::max<size_t>(bytes, 1));
    return at;
  };
  const size_t kept = (size_t)p.dd_rp[p.N];
  const size_t bb = (size_t)p.bs * p.bs;
  L.aval = take(sizeof(double) * bb * (size_t)p.nnzb);
  L.w = take(sizeof(double) * bb * kept);
  L.invd = take(sizeof(double) * bb * (size_t)p.N);
  L.dd_src = take(sizeof(int64_t) * kept);
  L.dd_rp = take(sizeof(int32_t) * (size_t)(p.N + 1));
  L.dd_col = take(sizeof(int32_t) * kept);
  L.ap_rp = take(sizeof(int32_t) * (size_t)(p.N + 1));
  L.ap_col = take(sizeof(int32_t) * (size_t)p.nnzb);
  L.ap_src = take(sizeof(int64_t) * (size_t)p.nnzb);
  L.order = take(sizeof(int32_t) * (size_t)p.N);
  L.lev_off = take(sizeof(int32_t) * (size_t)(p.nsub + 1));
  L.lptr = take(sizeof(int32_t) * (size_t)(total_levels + p.nsub));
  L.prow_off = take(sizeof(int32_t) * (size_t)(p.n_pieces + 1));
  L.prows = take(sizeof(int32_t) * (size_t)total_prows);
  L.piece_sub = take(sizeof(int32_t) * (size_t)p.n_pieces);
  L.flags = take(sizeof(int32_t) * 4);
  L.total = cur;
  return L;
}

int64_t total_levels_of(const Plan& p) {
  int64_t t = 0;
  for (int s = 0; s < p.nsub; ++s) {
    int32_t m = 0;
    for (int32_t i = p.part_ptr[s]; i < p.part_ptr[s + 1]; ++i) m = std::max(m, p.lev_l[i] + 1);
    t += m;
  }
  return t;
}

int64_t total_prows_of(const Plan& p) { return (int64_t)p.piece_rows.size(); }

// ---------------------------------------------------------------- kernels

__global__ void gather_w_kernel(const double* __restrict__ aval, const int64_t* __restrict__ dd_src, int64_t kept,
                                int bb, double* __restrict__ W) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < bb * kept; e += (int64_t)gridDim.x * blockDim.x)
    W[e] = aval[bb * dd_src[e / bb] + e % bb];
}

// C = A * B (bs x bs), the host's summation order: s = 0; s += A_rk B_kc, k = 0..bs-1.
__device__ __forceinline__ void dmul_bs(int bs, const double* A, const double* B, double* C) {
  for (int r = 0; r < bs; ++r)
    for (int c = 0; c < bs; ++c) {
      double s = 0.0;
      for (int k = 0; k < bs; ++k) s += A[bs * r + k] * B[bs * k + c];
      C[bs * r + c] = s;
    }
}

// bs x bs inverse (bs <= 3) by Gauss-Jordan elimination with partial pivoting (the host's steps).
__device__ bool dinverse_bs(int bs, const double* M, double* X) {
  double a[3][6];
  for (int r = 0; r < bs; ++r)
    for (int c = 0; c < 2 * bs; ++c) a[r][c] = c < bs ? M[bs * r + c] : (c - bs == r ? 1.0 : 0.0);
  for (int c = 0; c < bs; ++c) {
    int piv = c;
    for (int r = c + 1; r < bs; ++r)
      if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
    double pv = a[piv][c];
    if (!(fabs(pv) > 0.0) || !isfinite(pv)) return false;
    if (piv != c)
      for (int q = 0; q < 2 * bs; ++q) {
        double tmp = a[c][q];
        a[c][q] = a[piv][q];
        a[piv][q] = tmp;
      }
    double inv = 1.0 / a[c][c];
    for (int q = 0; q < 2 * bs; ++q) a[c][q] *= inv;
    for (int r = 0; r < bs; ++r) {
      if (r == c) continue;
      double m = a[r][c];
      if (m == 0.0) continue;
      for (int q = 0; q < 2 * bs; ++q) a[r][q] -= m * a[c][q];
    }
  }
  for (int r = 0; r < bs; ++r)
    for (int c = 0; c < bs; ++c) {
      X[bs * r + c] = a[r][c + bs];
      if (!isfinite(X[bs * r + c])) return false;
    }
  return true;
}

// Algorithm 7 for one subdomain, one L level at a time; row i (IKJ): for each
// strictly-lower block j (ascending): L_ij = W_ij U_jj^-1, then W_it -= L_ij U_jt
// for the strictly-upper blocks t of row j present in row i (descending t);
// finally D_i^-1 = U_ii^-1. W holds L below and U on and above the diagonal.
__global__ void factor_kernel(const int32_t* __restrict__ dd_rp, const int32_t* __restrict__ dd_col,
                              const int32_t* __restrict__ order, const int32_t* __restrict__ lev_off,
                              const int32_t* __restrict__ lptr, int bs, double* W, double* invD, int32_t* bad_row) {
  const int bb = bs * bs;
  const int s = blockIdx.x;
  const int32_t l0 = lev_off[s], l1 = lev_off[s + 1];
  for (int32_t l = l0; l + 1 < l1; ++l) {
    for (int32_t idx = lptr[l] + threadIdx.x; idx < lptr[l + 1]; idx += blockDim.x) {
      const int32_t i = order[idx];
      const int32_t q0 = dd_rp[i], q1 = dd_rp[i + 1];
      int32_t diag = -1;
      for (int32_t q = q0; q < q1; ++q)
        if (dd_col[q] == i) diag = q;
      double Lij[9], prod[9];
      for (int32_t q = q0; q < q1 && dd_col[q] < i; ++q) {
        const int32_t j = dd_col[q];
        dmul_bs(bs, &W[bb * (int64_t)q], &invD[bb * (int64_t)j], Lij);
        for (int e = 0; e < bb; ++e) W[bb * (int64_t)q + e] = Lij[e];
        for (int32_t t = dd_rp[j + 1] - 1; t >= dd_rp[j] && dd_col[t] > j; --t) {
          const int32_t ct = dd_col[t];
          int32_t at = -1;
          for (int32_t u = q0; u < q1; ++u)
            if (dd_col[u] == ct) at = u;
          if (at < 0) continue;
          dmul_bs(bs, Lij, &W[bb * (int64_t)t], prod);
          for (int e = 0; e < bb; ++e) W[bb * (int64_t)at + e] -= prod[e];
        }
      }
      if (diag < 0 || !dinverse_bs(bs, &W[bb * (int64_t)diag], &invD[bb * (int64_t)i])) atomicMin(bad_row, i);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ uint16_t dev_to_bf16(float f) {
  uint32_t u = __float_as_uint(f);
  if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x7FFFFFu)) return (uint16_t)((u >> 16) | 0x40);
  u += 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even
  return (uint16_t)(u >> 16);
}

// One factor entry in the stream's precision (the host's put_factor); DF64
// also checks the double-float range.
__device__ __forceinline__ void dev_put(unsigned char* dst, int prec, double v, int32_t* range_bad) {
  if (prec == ILU0DD_F64) {
    *reinterpret_cast<double*>(dst) = v;
  } else if (prec == ILU0DD_F32) {
    *reinterpret_cast<float*>(dst) = (float)v;
  } else if (prec == ILU0DD_DF64) {
    const float hi = (float)v;
    const float lo = (float)(v - (double)hi);
    reinterpret_cast<float*>(dst)[0] = hi;
    reinterpret_cast<float*>(dst)[1] = lo;
    const double a = fabs(v);
    if (a != 0.0 && !(a >= 0x1p-70 && a <= 0x1p100)) *range_bad = 1;
  } else {
    *reinterpret_cast<uint16_t*>(dst) = dev_to_bf16((float)v);
  }
}

// One thread block per piece, its threads over the piece's rows: the record
// head (slot counts, local rows, local columns slot-major) and the values,
// interleaved by component (entry [a][c] of row t's block at
// (c * count + t) * bs + a) or, in the row-thread layout (row_thread = 1),
// in 16-byte planes per value array (rt_value_offset).
__global__ void pack_stream_kernel(const CtaDesc* __restrict__ cta, const PieceDesc* __restrict__ pieces,
                                   const int32_t* __restrict__ piece_sub, const int32_t* __restrict__ prow_off,
                                   const int32_t* __restrict__ prows, const int32_t* __restrict__ dd_rp,
                                   const int32_t* __restrict__ dd_col, const double* __restrict__ W,
                                   const double* __restrict__ invD, int fe, int prec, int bs, int row_thread,
                                   unsigned char* stream, int32_t* range_bad) {
  const int bb = bs * bs;
  __shared__ int32_t cnt[256];
  const int32_t p = blockIdx.x;
  const PieceDesc pd = pieces[p];
  const CtaDesc cd = cta[piece_sub[p]];
  const int n = (int)(pd.meta & 0xFFFFu), w = (int)((pd.meta >> 16) & 0xFFu), kind = (int)(pd.meta >> 24);
  for (int sl = threadIdx.x; sl < 256; sl += blockDim.x) cnt[sl] = 0;
  __syncthreads();
  // the blocks of row t of the piece: strictly lower ones (first in the row)
  // or strictly upper ones (after the diagonal)
  auto row_blocks = [&](int t, int32_t* i, int32_t* qa, int32_t* nblk) {
    *i = cd.row0 + prows[prow_off[p] + t];
    const int32_t q0 = dd_rp[*i], q1 = dd_rp[*i + 1];
    int32_t q = q0;
    if (kind) {
      while (q < q1 && dd_col[q] <= *i) ++q;
      *qa = q;
      *nblk = q1 - q;
    } else {
      while (q < q1 && dd_col[q] < *i) ++q;
      *qa = q0;
      *nblk = q - q0;
    }
  };
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    int32_t i, qa, nblk;
    row_blocks(t, &i, &qa, &nblk);
    for (int sl = 0; sl < nblk; ++sl) atomicAdd(&cnt[sl], 1);
  }
  __syncthreads();
  unsigned char* rec = stream + cd.stream_off + pd.off;
  uint16_t* h = reinterpret_cast<uint16_t*>(rec);
  for (int sl = threadIdx.x; sl < w; sl += blockDim.x) h[sl] = (uint16_t)cnt[sl];
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    int32_t i, qa, nblk;
    row_blocks(t, &i, &qa, &nblk);
    h[w + t] = (uint16_t)(i - cd.row0);
    unsigned char* v = rec + pd.voff;
    if (kind) {
      const double* di = &invD[bb * (int64_t)i];
      if (row_thread) {
        for (int e = 0; e < 9; ++e) dev_put(v + rt_value_offset(e, t, n, fe), prec, di[e], range_bad);
        v += rt_slot_bytes(n, fe);
      } else {
        for (int cc = 0; cc < bs; ++cc)
          for (int a = 0; a < bs; ++a)
            dev_put(v + (((int64_t)cc * n + t) * bs + a) * fe, prec, di[bs * a + cc], range_bad);
        v += (int64_t)bb * n * fe;
      }
    }
    int64_t c0 = 0;
    unsigned char* vs = v;  // this slot's value array
    for (int sl = 0; sl < nblk; ++sl) {
      const int32_t q = qa + sl;
      const int cs = cnt[sl];
      h[w + n + c0 + t] = (uint16_t)(dd_col[q] - cd.row0);
      double F[9];
      if (kind) {
        dmul_bs(bs, &invD[bb * (int64_t)i], &W[bb * (int64_t)q], F);  // U~_iq = D_i^-1 U_iq
      } else {
        for (int e = 0; e < bb; ++e) F[e] = W[bb * (int64_t)q + e];
      }
      if (row_thread) {
        for (int e = 0; e < 9; ++e) dev_put(vs + rt_value_offset(e, t, cs, fe), prec, F[e], range_bad);
        vs += rt_slot_bytes(cs, fe);
      } else {
        vs = v + bb * c0 * fe;
        for (int cc = 0; cc < bs; ++cc)
          for (int a = 0; a < bs; ++a)
            dev_put(vs + (((int64_t)cc * cs + t) * bs + a) * fe, prec, F[bs * a + cc], range_bad);
      }
      c0 += cs;
    }
  }
}

// Sliced ELL of the reordered full matrix (the host's pack_sell): slot-major,
// entry-major within a slot; padding entries are zero blocks on the row's
// own column (column 0 past the last row).
__global__ void pack_sell_kernel(const int32_t* __restrict__ slice_off, int64_t nslices, int32_t N,
                                 const int32_t* __restrict__ ap_rp, const int32_t* __restrict__ ap_col,
                                 const int64_t* __restrict__ ap_src, const double* __restrict__ aval, int bb,
                                 int32_t* __restrict__ cols, double* __restrict__ vals) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t k = g / kSlice;
  const int lane = (int)(g % kSlice);
  if (k >= nslices) return;
  const int64_t so = slice_off[k];
  const int32_t w = slice_off[k + 1] - slice_off[k];
  const int64_t r = k * kSlice + lane;
  const int32_t len = r < N ? ap_rp[r + 1] - ap_rp[r] : 0;
  for (int32_t s = 0; s < w; ++s) {
    const int64_t slot = so + s;
    int32_t col = r < N ? (int32_t)r : 0;
    const double* src = nullptr;
    if (s < len) {
      const int64_t q = ap_rp[r] + s;
      col = ap_col[q];
      src = aval + bb * ap_src[q];
    }
    cols[slot * kSlice + lane] = col;
    for (int e = 0; e < bb; ++e) vals[(slot * bb + e) * kSlice + lane] = src ? src[e] : 0.0;
  }
}

// Algorithm 5 (level sets by repeated sweeps), one block per subdomain: a row
// joins level l + 1 once all its lower (upper = 1: upper) neighbours inside
// the subdomain sit on levels <= l. lev[] is in global memory: kUnset until
// assigned, kJoining between the check and the promotion of a sweep.
constexpr int32_t kUnset = INT32_MAX, kJoining = -1;
__global__ void levels_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                              const int32_t* __restrict__ part_ptr, int upper, int32_t* lev, int32_t* nlev) {
  const int32_t r0 = part_ptr[blockIdx.x], r1 = part_ptr[blockIdx.x + 1];
  auto dep = [&](int32_t i, int32_t j) { return j >= r0 && j < r1 && (upper ? j > i : j < i); };
  for (int32_t i = r0 + (int32_t)threadIdx.x; i < r1; i += (int32_t)blockDim.x) {
    bool any = false;
    for (int32_t q = rp[i]; q < rp[i + 1] && !any; ++q) any = dep(i, col[q]);
    lev[i] = any ? kUnset : 0;
  }
  volatile int32_t* vlev = lev;  // read while other threads of the sweep mark rows
  __shared__ int joined;
  int32_t level = 0;
  // at most one sweep per row: every sweep of an acyclic pattern adds a row
  for (; level <= r1 - r0; ++level) {
    if (threadIdx.x == 0) joined = 0;
    __syncthreads();
    for (int32_t i = r0 + (int32_t)threadIdx.x; i < r1; i += (int32_t)blockDim.x) {
      if (vlev[i] != kUnset) continue;
      bool ready = true;
      for (int32_t q = rp[i]; q < rp[i + 1] && ready; ++q) {
        const int32_t j = col[q];
        if (dep(i, j)) {
          const int32_t lj = vlev[j];
          ready = lj >= 0 && lj <= level;
        }
      }
      if (ready) {
        vlev[i] = kJoining;
        joined = 1;
      }
    }
    __syncthreads();
    const int any = joined;
    for (int32_t i = r0 + (int32_t)threadIdx.x; i < r1; i += (int32_t)blockDim.x)
      if (lev[i] == kJoining) lev[i] = level + 1;
    __syncthreads();
    if (!any) break;
  }
  if (threadIdx.x == 0 && nlev) nlev[blockIdx.x] = r1 > r0 ? level + 1 : 0;
}

}  // namespace

cudaError_t launch_levels(const int32_t* rp, const int32_t* col, const int32_t* part_ptr, int32_t nsub, int upper,
                          int32_t* lev, int32_t* nlev, cudaStream_t s) {
  if (nsub <= 0) return cudaSuccess;
  levels_kernel<<<nsub, 256, 0, s>>>(rp, col, part_ptr, upper, lev, nlev);
  return cudaGetLastError();
}

size_t device_setup_scratch_bytes(const Plan& p) {
  return scratch_layout(p, total_levels_of(p), total_prows_of(p)).total;
}

int setup_on_device(const Plan& p, const double* aval_in, unsigned char* scratch, size_t scratch_bytes,
                    unsigned char* ws, cudaStream_t s, DeviceSetupResult* res) {
  res->bad_row = -1;
  res->range_bad = false;
  res->cuda = cudaSuccess;
  const int64_t total_levels = total_levels_of(p);
  const int64_t total_prows = total_prows_of(p);
  const ScratchLayout L = scratch_layout(p, total_levels, total_prows);
  if (!scratch || scratch_bytes < L.total || (reinterpret_cast<uintptr_t>(scratch) & 255)) return ILU0DD_ERR_WORKSPACE;
  const int64_t kept = p.dd_rp[p.N];

  // ---- host: index arrays the kernels read
  RawVec<int64_t> dd_src((size_t)kept);
  host_parallel_for(kept, [&](int64_t q) { dd_src[q] = p.ap_src[p.dd_ap[q]]; });
  std::vector<int32_t> order((size_t)p.N), lev_off((size_t)p.nsub + 1), lptr((size_t)(total_levels + p.nsub));
  {
    std::vector<int32_t> nl(p.nsub);
    host_parallel_for(p.nsub, [&](int64_t sub) {
      int32_t m = 0;
      for (int32_t i = p.part_ptr[sub]; i < p.part_ptr[sub + 1]; ++i) m = std::max(m, p.lev_l[i] + 1);
      nl[sub] = m;
    });
    lev_off[0] = 0;
    for (int sub = 0; sub < p.nsub; ++sub) lev_off[sub + 1] = lev_off[sub] + nl[sub] + 1;
    host_parallel_for(p.nsub, [&](int64_t sub) {
      const int32_t r0 = p.part_ptr[sub], r1 = p.part_ptr[sub + 1];
      int32_t* lp = &lptr[lev_off[sub]];
      const int32_t m = nl[sub];
      for (int32_t l = 0; l <= m; ++l) lp[l] = 0;
      for (int32_t i = r0; i < r1; ++i) lp[p.lev_l[i] + 1]++;
      lp[0] = r0;
      for (int32_t l = 0; l < m; ++l) lp[l + 1] += lp[l];
      std::vector<int32_t> next(lp, lp + m);
      for (int32_t i = r0; i < r1; ++i) order[next[p.lev_l[i]]++] = i;  // stable within a level
    });
  }
  std::vector<int32_t> prow_off((size_t)p.n_pieces + 1), piece_sub((size_t)p.n_pieces);
  for (int64_t k = 0; k <= p.n_pieces; ++k) prow_off[k] = (int32_t)p.piece_rows_off[k];
  for (int sub = 0; sub < p.nsub; ++sub)
    for (int32_t k = 0; k < p.cta[sub].npieces; ++k) piece_sub[p.cta[sub].piece0 + k] = sub;

  // ---- uploads
  cudaError_t e = cudaSuccess;
  auto up = [&](size_t off, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(scratch + off, src, bytes, cudaMemcpyHostToDevice, s);
  };
  const int bs = p.bs, bb = bs * bs;
  // the caller's values: host memory, or device memory (a device-to-device copy)
  if (e == cudaSuccess && p.nnzb)
    e = cudaMemcpyAsync(scratch + L.aval, aval_in, sizeof(double) * bb * (size_t)p.nnzb, cudaMemcpyDefault, s);
  up(L.dd_src, dd_src.data(), sizeof(int64_t) * dd_src.size());
  up(L.dd_rp, p.dd_rp.data(), sizeof(int32_t) * p.dd_rp.size());
  up(L.dd_col, p.dd_col.data(), sizeof(int32_t) * p.dd_col.size());
  up(L.ap_rp, p.ap_rp.data(), sizeof(int32_t) * p.ap_rp.size());
  up(L.ap_col, p.ap_col.data(), sizeof(int32_t) * p.ap_col.size());
  up(L.ap_src, p.ap_src.data(), sizeof(int64_t) * p.ap_src.size());
  up(L.order, order.data(), sizeof(int32_t) * order.size());
  up(L.lev_off, lev_off.data(), sizeof(int32_t) * lev_off.size());
  up(L.lptr, lptr.data(), sizeof(int32_t) * lptr.size());
  up(L.prow_off, prow_off.data(), sizeof(int32_t) * prow_off.size());
  up(L.prows, p.piece_rows.data(), sizeof(int32_t) * p.piece_rows.size());
  up(L.piece_sub, piece_sub.data(), sizeof(int32_t) * piece_sub.size());
  if (e == cudaSuccess) e = cudaMemcpyAsync(ws + p.lay.cta, p.cta.data(), sizeof(CtaDesc) * p.cta.size(),
                                            cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !p.pieces.empty())
    e = cudaMemcpyAsync(ws + p.lay.pieces, p.pieces.data(), sizeof(PieceDesc) * p.pieces.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ws + p.lay.sell_off, p.slice_off.data(), sizeof(int32_t) * p.slice_off.size(),
                        cudaMemcpyHostToDevice, s);
  const int32_t init_flags[4] = {INT32_MAX, 0, 0, 0};
  up(L.flags, init_flags, sizeof init_flags);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws + p.lay.stream, 0, (size_t)p.stream_bytes, s);
  // host staging buffers must outlive the copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    res->cuda = e;
    return ILU0DD_ERR_CUDA;
  }

  const double* aval = reinterpret_cast<const double*>(scratch + L.aval);
  double* W = reinterpret_cast<double*>(scratch + L.w);
  double* invD = reinterpret_cast<double*>(scratch + L.invd);
  int32_t* flags = reinterpret_cast<int32_t*>(scratch + L.flags);
  auto I32 = [&](size_t off) { return reinterpret_cast<const int32_t*>(scratch + off); };

  // ---- SpMV matrix
  if (p.nslices > 0)
    pack_sell_kernel<<<(unsigned)((p.nslices * kSlice + 255) / 256), 256, 0, s>>>(
        reinterpret_cast<const int32_t*>(ws + p.lay.sell_off), p.nslices, p.N, I32(L.ap_rp), I32(L.ap_col),
        reinterpret_cast<const int64_t*>(scratch + L.ap_src), aval, bb, reinterpret_cast<int32_t*>(ws + p.lay.sell_col),
        reinterpret_cast<double*>(ws + p.lay.sell_val));
  // ---- factors
  if (kept > 0)
    gather_w_kernel<<<(unsigned)std::min<int64_t>((bb * kept + 255) / 256, 152 * 64), 256, 0, s>>>(
        aval, reinterpret_cast<const int64_t*>(scratch + L.dd_src), kept, bb, W);
  if (p.nsub > 0)
    factor_kernel<<<p.nsub, 128, 0, s>>>(I32(L.dd_rp), I32(L.dd_col), I32(L.order), I32(L.lev_off), I32(L.lptr), bs,
                                         W, invD, flags);
  e = cudaGetLastError();
  int32_t hflags[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hflags, flags, sizeof hflags, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    res->cuda = e;
    return ILU0DD_ERR_CUDA;
  }
  if (hflags[0] != INT32_MAX) {
    res->bad_row = hflags[0];
    return ILU0DD_ERR_ZERO_PIVOT;
  }
  // ---- factor stream
  if (p.n_pieces > 0)
    pack_stream_kernel<<<(unsigned)p.n_pieces, 128, 0, s>>>(
        reinterpret_cast<const CtaDesc*>(ws + p.lay.cta), reinterpret_cast<const PieceDesc*>(ws + p.lay.pieces),
        I32(L.piece_sub), I32(L.prow_off), I32(L.prows), I32(L.dd_rp), I32(L.dd_col), W, invD, p.factor_elem,
        p.factor_prec, bs, p.row_thread ? 1 : 0, ws + p.lay.stream, flags + 1);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(hflags, flags, sizeof hflags, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    res->cuda = e;
    return ILU0DD_ERR_CUDA;
  }
  if (hflags[1]) {
    res->range_bad = true;
    return ILU0DD_ERR_INVALID;
  }
  res->w = W;
  res->invd = invD;
  return ILU0DD_OK;
}

}  // namespace ilu0dd
