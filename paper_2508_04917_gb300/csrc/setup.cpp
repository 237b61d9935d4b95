// Host side of ilu0_dd_setup: decomposition (Algorithm 2, Algorithm 3, the drop
// of Section 3.2), level sets (Algorithm 5), block ILU0 / ILDU0 (Algorithm 7)
// and packing of the device layouts. FP64 throughout; compiled without FMA
// contraction so x86-64 and aarch64 hosts produce the same bits.
#include <algorithm>
#include <chrono>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <thread>

#include "internal.h"

namespace ilu0dd {

double wall_seconds() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

namespace {

inline int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }
inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Run f(i) for i in [0, n) on the host's hardware threads.
template <typename F>
void parallel_for(int64_t n, F&& f) {
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

// Bytes of one piece record (see internal.h). cnt[s] (s < w) = rows with more
// than s blocks. In the row-thread layout every value array (D^-1, then each
// slot) starts on a 16-byte boundary.
int64_t record_bytes(int n, int w, int64_t nb, const int32_t* cnt, int kind, int felem, int bs, bool row_thread,
                     int64_t* voff) {
  int64_t head = 2 * (int64_t)w + 2 * (int64_t)n + 2 * nb;
  int64_t v = align_up(head, 16);
  if (voff) *voff = v;
  const int64_t bb = (int64_t)bs * bs;
  if (row_thread) {
    int64_t at = v + (kind ? rt_slot_bytes(n, felem) : 0);
    for (int s = 0; s < w; ++s) at += rt_slot_bytes(cnt[s], felem);
    return align_up(at, 16);
  }
  int64_t vals = (kind ? bb * n : 0) + bb * nb;
  return align_up(v + vals * felem, 16);
}

// bs x bs inverse (bs <= 3) by Gauss-Jordan elimination with partial pivoting.
bool inverse_bs(int bs, const double* M, double* X) {
  double a[3][6];
  for (int r = 0; r < bs; ++r)
    for (int c = 0; c < 2 * bs; ++c) a[r][c] = c < bs ? M[bs * r + c] : (c - bs == r ? 1.0 : 0.0);
  for (int c = 0; c < bs; ++c) {
    int piv = c;
    for (int r = c + 1; r < bs; ++r)
      if (std::fabs(a[r][c]) > std::fabs(a[piv][c])) piv = r;
    double pv = a[piv][c];
    if (!(std::fabs(pv) > 0.0) || !std::isfinite(pv)) return false;
    if (piv != c)
      for (int q = 0; q < 2 * bs; ++q) std::swap(a[c][q], a[piv][q]);
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
      if (!std::isfinite(X[bs * r + c])) return false;
    }
  return true;
}

// C = A * B (bs x bs).
inline void mul_bs(int bs, const double* A, const double* B, double* C) {
  for (int r = 0; r < bs; ++r)
    for (int c = 0; c < bs; ++c) {
      double s = 0.0;
      for (int k = 0; k < bs; ++k) s += A[bs * r + k] * B[bs * k + c];
      C[bs * r + c] = s;
    }
}

uint16_t to_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x7FFFFFu)) return (uint16_t)((u >> 16) | 0x40);
  u += 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even
  return (uint16_t)(u >> 16);
}

void put_factor(uint8_t* dst, int prec, double v) {
  if (prec == ILU0DD_F64) {
    std::memcpy(dst, &v, 8);
  } else if (prec == ILU0DD_F32) {
    float f = (float)v;
    std::memcpy(dst, &f, 4);
  } else if (prec == ILU0DD_DF64) {
    // hi = fl32(v), lo = fl32(v - hi); v - hi is exact in FP64
    float hl[2];
    hl[0] = (float)v;
    hl[1] = (float)(v - (double)hl[0]);
    std::memcpy(dst, hl, 8);
  } else {
    uint16_t h = to_bf16((float)v);
    std::memcpy(dst, &h, 2);
  }
}

}  // namespace

int make_plan(const ilu0dd_bsr* A, const ilu0dd_geom* g, const ilu0dd_opts* o, int max_smem,
              Plan* P, std::string* why, const int32_t* labels, int32_t nlabels) {
  if (!A || !o || !P || (!g && !labels)) return ILU0DD_ERR_INVALID;
  if (!labels && (g->nx <= 0 || g->ny <= 0 || g->nz <= 0 || g->sx <= 0 || g->sy <= 0 || g->sz <= 0)) {
    *why = "grid and subdomain sides must be positive";
    return ILU0DD_ERR_INVALID;
  }
  int64_t N64 = labels ? (int64_t)A->n_brows : (int64_t)g->nx * g->ny * g->nz;
  if (N64 != A->n_brows || N64 < 0 || N64 >= (1ll << 31)) {
    *why = "n_brows must equal nx*ny*nz (< 2^31)";
    return ILU0DD_ERR_INVALID;
  }
  if (labels && nlabels <= 0 && N64 > 0) {
    *why = "nparts must be positive";
    return ILU0DD_ERR_INVALID;
  }
  const int bs = A->block_dim == 0 ? 3 : A->block_dim;
  if (bs != 1 && bs != 3) {
    *why = "block_dim must be 1 (scalar CSR) or 3 (3x3 blocks)";
    return ILU0DD_ERR_INVALID;
  }
  if (!A->row_ptr || !A->col_idx || (A->nnzb > 0 && !A->val)) {
    *why = "null matrix array";
    return ILU0DD_ERR_INVALID;
  }
  const int32_t N = (int32_t)N64;
  const int32_t* rp = A->row_ptr;
  const int32_t* ci = A->col_idx;
  if (rp[0] != 0 || rp[N] != A->nnzb) {
    *why = "row_ptr[0] must be 0 and row_ptr[N] must equal nnzb";
    return ILU0DD_ERR_INVALID;
  }
  {
    // pattern checks in parallel; the first bad row (lowest index) is reported
    std::atomic<int32_t> bad_row{INT32_MAX};
    parallel_for(N, [&](int64_t i) {
      int kind = 0;
      if (rp[i + 1] < rp[i]) {
        kind = 1;
      } else {
        bool diag = false;
        for (int64_t q = rp[i]; q < rp[i + 1] && !kind; ++q) {
          if (ci[q] < 0 || ci[q] >= N) kind = 2;
          else if (q > rp[i] && ci[q] <= ci[q - 1]) kind = 3;
          diag |= ci[q] == i;
        }
        if (!kind && !diag) kind = 4;
      }
      if (kind) {
        int32_t cur = bad_row.load();
        while ((int32_t)i < cur && !bad_row.compare_exchange_weak(cur, (int32_t)i)) {
        }
      }
    });
    if (bad_row.load() != INT32_MAX) {
      const int32_t i = bad_row.load();
      int kind = 0;  // re-check the reported row alone for its message
      if (rp[i + 1] < rp[i]) kind = 1;
      for (int64_t q = rp[i]; !kind && q < rp[i + 1]; ++q) {
        if (ci[q] < 0 || ci[q] >= N) kind = 2;
        else if (q > rp[i] && ci[q] <= ci[q - 1]) kind = 3;
      }
      *why = kind == 1 ? "row_ptr not monotone"
             : kind == 2 ? "column out of range"
             : kind == 3 ? "columns not strictly ascending"
                         : "missing diagonal block in row " + std::to_string(i);
      return ILU0DD_ERR_INVALID;
    }
  }
  Plan& p = *P;
  p = Plan();
  p.bs = bs;
  // per-phase wall times (opts.trace)
  double tprev = wall_seconds();
  std::string tlog;
  auto tmark = [&](const char* what) {
    if (!o->trace) return;
    const double t = wall_seconds();
    tlog += std::string(" ") + what + " " + std::to_string((int)((t - tprev) * 1e3)) + "ms";
    tprev = t;
  };
  p.N = N;
  p.nnzb = A->nnzb;
  if (g) p.geom = *g;
  p.opts = *o;

  tmark("check");
  if (labels) {
    // ---- given labels (a graph partition): Section 3.1's stable grouping
    std::atomic<int> bad{0};
    parallel_for(N, [&](int64_t r) {
      if (labels[r] < 0 || labels[r] >= nlabels) bad = 1;
    });
    if (bad) {
      *why = "part_id out of [0, nparts)";
      return ILU0DD_ERR_INVALID;
    }
    p.nsub = nlabels;
    p.part_id.assign(labels, labels + N);
    p.part_ptr.assign(p.nsub + 1, 0);
    for (int32_t r = 0; r < N; ++r) p.part_ptr[p.part_id[r] + 1]++;
    for (int s = 0; s < p.nsub; ++s) p.part_ptr[s + 1] += p.part_ptr[s];
    std::vector<int32_t> next(p.part_ptr.begin(), p.part_ptr.end() - 1);
    p.perm.resize(N);
    p.iperm.resize(N);
    for (int32_t r = 0; r < N; ++r) {
      const int32_t nr = next[p.part_id[r]]++;
      p.perm[nr] = r;
      p.iperm[r] = nr;
    }
  } else {
    // ---- Algorithm 2: labels from geometric cuts (ceil-division at the edges)
    const int bx = ceil_div(g->nx, g->sx), by = ceil_div(g->ny, g->sy), bz = ceil_div(g->nz, g->sz);
    p.nsub = bx * by * bz;
    p.part_id.resize(N);
    parallel_for(g->nz, [&](int64_t k) {
      for (int j = 0; j < g->ny; ++j)
        for (int i = 0; i < g->nx; ++i)
          p.part_id[(int64_t)i + (int64_t)g->nx * (j + (int64_t)g->ny * k)] =
              i / g->sx + bx * (j / g->sy + by * ((int)k / g->sz));
    });

    // ---- Section 3.1: stable grouping by label (perm[new] = old). A label's
    // cells in natural order are its box's cells in (k, j, i) order, so each
    // subdomain's slice of perm is filled independently.
    p.part_ptr.assign(p.nsub + 1, 0);
    auto box_side = [](int n, int sd, int b) { return std::min(sd, n - b * sd); };
    for (int s = 0; s < p.nsub; ++s) {
      const int ib = s % bx, jb = (s / bx) % by, kb = s / (bx * by);
      p.part_ptr[s + 1] = p.part_ptr[s] + box_side(g->nx, g->sx, ib) * box_side(g->ny, g->sy, jb) *
                                              box_side(g->nz, g->sz, kb);
    }
    p.perm.resize(N);
    p.iperm.resize(N);
    parallel_for(p.nsub, [&](int64_t s) {
      const int ib = (int)(s % bx), jb = (int)((s / bx) % by), kb = (int)(s / ((int64_t)bx * by));
      int32_t nr = p.part_ptr[s];
      for (int k = kb * g->sz; k < std::min(g->nz, (kb + 1) * g->sz); ++k)
        for (int j = jb * g->sy; j < std::min(g->ny, (jb + 1) * g->sy); ++j)
          for (int i = ib * g->sx; i < std::min(g->nx, (ib + 1) * g->sx); ++i) {
            const int32_t r = (int32_t)((int64_t)i + (int64_t)g->nx * (j + (int64_t)g->ny * k));
            p.perm[nr] = r;
            p.iperm[r] = nr++;
          }
    });
  }
  tmark("label+perm");
  // ---- Algorithm 3 on BSR: reorder rows and columns, sort each row
  p.ap_rp.resize(N + 1);
  p.ap_rp[0] = 0;
  for (int32_t i = 0; i < N; ++i) p.ap_rp[i + 1] = p.ap_rp[i] + (rp[p.perm[i] + 1] - rp[p.perm[i]]);
  p.ap_col.resize(A->nnzb);
  p.ap_src.resize(A->nnzb);
  parallel_for(N, [&](int64_t i) {
    int32_t old = p.perm[i];
    int64_t base = p.ap_rp[i], len = rp[old + 1] - rp[old];
    std::pair<int32_t, int64_t> tmp[64];
    std::vector<std::pair<int32_t, int64_t>> big;
    auto* e = tmp;
    if (len > 64) { big.resize(len); e = big.data(); }
    for (int64_t q = 0; q < len; ++q) e[q] = {p.iperm[ci[rp[old] + q]], rp[old] + q};
    std::sort(e, e + len);
    for (int64_t q = 0; q < len; ++q) {
      p.ap_col[base + q] = e[q].first;
      p.ap_src[base + q] = e[q].second;
    }
  });

  tmark("reorder");
  // ---- Section 3.2: drop blocks whose row and column lie in different subdomains
  std::vector<int32_t> label(N);
  parallel_for(N, [&](int64_t i) { label[i] = p.part_id[p.perm[i]]; });
  p.dd_rp.assign(N + 1, 0);
  parallel_for(N, [&](int64_t i) {
    int32_t c = 0;
    for (int64_t q = p.ap_rp[i]; q < p.ap_rp[i + 1]; ++q) c += label[p.ap_col[q]] == label[i];
    p.dd_rp[i + 1] = c;
  });
  for (int32_t i = 0; i < N; ++i) p.dd_rp[i + 1] += p.dd_rp[i];
  int64_t kept = p.dd_rp[N];
  p.dd_col.resize(kept);
  p.dd_ap.resize(kept);
  parallel_for(N, [&](int64_t i) {
    int64_t d = p.dd_rp[i];
    for (int64_t q = p.ap_rp[i]; q < p.ap_rp[i + 1]; ++q)
      if (label[p.ap_col[q]] == label[i]) {
        p.dd_col[d] = p.ap_col[q];
        p.dd_ap[d++] = q;
      }
  });
  {
    std::vector<int64_t> nl(p.nsub, 0), nu(p.nsub, 0);
    parallel_for(p.nsub, [&](int64_t s) {
      for (int32_t i = p.part_ptr[s]; i < p.part_ptr[s + 1]; ++i)
        for (int64_t q = p.dd_rp[i]; q < p.dd_rp[i + 1]; ++q) {
          nl[s] += p.dd_col[q] < i;
          nu[s] += p.dd_col[q] > i;
        }
    });
    for (int s = 0; s < p.nsub; ++s) {
      p.nL += nl[s];
      p.nU += nu[s];
    }
  }

  tmark("drop");
  // ---- Algorithm 5 (level sets of each subdomain's L and U DAG)
  p.lev_l.assign(N, 0);
  p.lev_u.assign(N, 0);
  std::vector<int32_t> nlev_l(p.nsub), nlev_u(p.nsub);
  parallel_for(p.nsub, [&](int64_t s) {
    int32_t r0 = p.part_ptr[s], r1 = p.part_ptr[s + 1], ml = 0, mu = 0;
    for (int32_t i = r0; i < r1; ++i) {
      int32_t l = 0;
      for (int64_t q = p.dd_rp[i]; q < p.dd_rp[i + 1] && p.dd_col[q] < i; ++q)
        l = std::max(l, p.lev_l[p.dd_col[q]] + 1);
      p.lev_l[i] = l;
      ml = std::max(ml, l + 1);
    }
    for (int32_t i = r1 - 1; i >= r0; --i) {
      int32_t l = 0;
      for (int64_t q = p.dd_rp[i + 1] - 1; q >= p.dd_rp[i] && p.dd_col[q] > i; --q)
        l = std::max(l, p.lev_u[p.dd_col[q]] + 1);
      p.lev_u[i] = l;
      mu = std::max(mu, l + 1);
    }
    nlev_l[s] = r1 > r0 ? ml : 0;
    nlev_u[s] = r1 > r0 ? mu : 0;
  });

  tmark("levels");
  // ---- apply configuration
  const int fp = o->factor_prec;
  if (fp != ILU0DD_F64 && fp != ILU0DD_F32 && fp != ILU0DD_BF16 && fp != ILU0DD_DF64) {
    *why = "factor_prec must be ILU0DD_F64, ILU0DD_F32, ILU0DD_BF16 or ILU0DD_DF64";
    return ILU0DD_ERR_INVALID;
  }
  p.factor_prec = fp;
  if (o->traversal != 0 && o->traversal != 1) {
    *why = "traversal must be 0 (vertex-centric) or 1 (edge-centric)";
    return ILU0DD_ERR_INVALID;
  }
  if (o->traversal == 1 && fp == ILU0DD_DF64) {
    *why = "the edge-centric traversal has no float-pair form (no atomic add on pairs)";
    return ILU0DD_ERR_INVALID;
  }
  // blocks on each side of the diagonal per row (the jagged-diagonal sort key)
  std::vector<int32_t> nlo(N), nup(N);
  parallel_for(N, [&](int64_t i) {
    int32_t lo = 0, up = 0;
    for (int64_t q = p.dd_rp[i]; q < p.dd_rp[i + 1]; ++q) {
      lo += p.dd_col[q] < i;
      up += p.dd_col[q] > i;
    }
    nlo[i] = lo;
    nup[i] = up;
  });
  int32_t side_max = 0;
  for (int64_t i = 0; i < N; ++i) side_max = std::max(side_max, std::max(nlo[i], nup[i]));
  // 3x3 blocks: FP64 and float-pair factors take three threads per row (ten
  // rows per warp); FP32 and BF16 factors one thread per row (the row-thread
  // layout) when no row has more than kDescSlots blocks on either side (all
  // of a row's blocks then load ahead of the level wait; rows with more, as
  // in 27-point patterns, take the three-thread mapping, which loads their
  // further slots in groups: measured on GB300, unstructured 128^3 apply
  // with one thread per row / three: FP32 0.574 / 0.336 ms, BF16 0.407 /
  // 0.336); scalar rows one thread per row
  if (o->apply_mapping != 0 && o->apply_mapping != 1) {
    *why = "apply_mapping must be 0 (automatic) or 1 (three threads per 3x3 row)";
    return ILU0DD_ERR_INVALID;
  }
  p.row_thread = bs == 3 && (fp == ILU0DD_F32 || fp == ILU0DD_BF16) && side_max <= kDescSlots && o->apply_mapping == 0;
  p.rows_per_warp = bs == 3 && !p.row_thread ? kRowsPerWarp : 32;
  p.factor_elem = (fp == ILU0DD_F64 || fp == ILU0DD_DF64) ? 8 : fp == ILU0DD_F32 ? 4 : 2;
  p.vec_elem = (fp == ILU0DD_F64 || fp == ILU0DD_DF64) ? 8 : 4;
  // shared-memory bytes per row of the subdomain vector: FP32 arithmetic in the
  // row-thread layout pads the three entries to 16 bytes (one vector access)
  p.vec_row_bytes = p.row_thread && p.vec_elem == 4 ? 16 : bs * p.vec_elem;
  for (int s = 0; s < p.nsub; ++s) p.rmax = std::max(p.rmax, p.part_ptr[s + 1] - p.part_ptr[s]);
  if (p.rmax > 65535) {
    *why = "a subdomain has more than 65535 rows";
    return ILU0DD_ERR_SMEM;
  }
  // widest level decides the default block size
  int widest = 1;
  {
    std::vector<int32_t> cnt;
    for (int s = 0; s < p.nsub; ++s) {
      int32_t r0 = p.part_ptr[s], r1 = p.part_ptr[s + 1];
      int32_t nl = std::max(nlev_l[s], nlev_u[s]);
      cnt.assign(2 * (size_t)nl, 0);
      for (int32_t i = r0; i < r1; ++i) {
        cnt[p.lev_l[i]]++;
        cnt[nl + p.lev_u[i]]++;
      }
      for (int32_t c : cnt) widest = std::max(widest, c);
      p.max_levels = std::max(p.max_levels, nlev_l[s] + nlev_u[s]);
    }
  }
  // One warp per row group of the widest level. FP64-arithmetic applies (FP64
  // and DF64) get half as many warps again once that is four groups or more:
  // their groups compute long enough that spare warps, loading ahead for later
  // levels, pay (measured on GB300: 200^3 scalar 0.241 -> 0.222 ms, 8^3 boxes
  // 0.064 -> 0.062 ms); FP32/BF16 groups and small boxes run faster without.
  const int groups = (int)ceil_div(widest, p.rows_per_warp);
  const bool fp64_arith = o->factor_prec == ILU0DD_F64 || o->factor_prec == ILU0DD_DF64;
  // the row-thread layout (32 rows per warp): 1.5 warps per row group of the
  // widest level, the spare warps loading ahead for later levels (measured at
  // 160^3: 192 threads for the 16x16x8 box; 128 / 160 / 224 / 256 are slower
  // or within 1 %)
  const int warps = p.row_thread ? std::max(1, (3 * groups + 1) / 2) : fp64_arith && groups >= 4 ? groups + (groups + 1) / 2 : groups;
  const int max_threads = p.row_thread ? kMaxRtThreads : kMaxApplyThreads;
  p.threads = o->threads_per_cta > 0 ? o->threads_per_cta : std::min(max_threads, 32 * warps);
  if (p.threads % 32 || p.threads > max_threads || p.threads < 32) {
    *why = "threads_per_cta must be a multiple of 32 in [32, " + std::to_string(max_threads) +
           "] (256 with 3x3 FP32 or BF16 factors in the row-thread mapping, else 384)";
    return ILU0DD_ERR_INVALID;
  }
  // default L2 prefetch distance: 32 KiB of stream, 16 KiB for BF16 whose
  // levels take half the bytes (measured at 160^3: BF16 0.1886 ms at 16 KiB,
  // 0.1925 at 32; FP32 best at 32 KiB; FP64 and DF64 within 0.5 % from 16 to 64)
  p.prefetch_bytes = o->prefetch_bytes > 0 ? o->prefetch_bytes : std::min(32768, 8192 * p.factor_elem);
  if (p.prefetch_bytes % 16 || p.prefetch_bytes > (1 << 24)) {
    *why = "prefetch_bytes must be a multiple of 16 up to 16 MiB";
    return ILU0DD_ERR_INVALID;
  }
  const int rows_cap = (p.threads / 32) * p.rows_per_warp;
  const int64_t cap = 1ll << 30;  // record bytes (offsets are 32-bit)

  // ---- pieces: per subdomain, L levels 1.. then U levels 0.., rows of a level
  // sorted by block count (longest first), split by the block's row capacity
  p.cta.resize(p.nsub);
  std::vector<std::vector<int32_t>> sub_rows(p.nsub);  // local rows, piece after piece
  std::vector<std::vector<PieceDesc>> sub_desc(p.nsub);
  std::vector<int64_t> sub_len(p.nsub, 0);
  std::vector<int> sub_fail(p.nsub, 0);
  parallel_for(p.nsub, [&](int64_t s) {
    const int32_t r0 = p.part_ptr[s], r1 = p.part_ptr[s + 1];
    std::vector<int32_t>& out = sub_rows[s];
    out.reserve(2 * (size_t)(r1 - r0));
    std::vector<int32_t> start, byl;
    std::vector<std::pair<int32_t, int32_t>> key;  // (-blocks, row)
    uint32_t off = 0;
    int64_t prev_lvl = -1;  // first piece of the previous non-empty level
    for (int kind = 0; kind < 2; ++kind) {
      const int32_t nl = kind ? nlev_u[s] : nlev_l[s];
      const std::vector<int32_t>& lev = kind ? p.lev_u : p.lev_l;
      // rows grouped by level (counting sort, ascending rows within a level)
      start.assign((size_t)nl + 1, 0);
      for (int32_t i = r0; i < r1; ++i) start[lev[i] + 1]++;
      for (int32_t l = 0; l < nl; ++l) start[l + 1] += start[l];
      byl.resize((size_t)(r1 - r0));
      {
        std::vector<int32_t> next(start.begin(), start.end() - 1);
        for (int32_t i = r0; i < r1; ++i) byl[next[lev[i]]++] = i;
      }
      for (int32_t l = kind ? 0 : 1; l < nl; ++l) {
        if (start[l + 1] == start[l]) continue;
        const uint32_t first = (uint32_t)sub_desc[s].size();
        const uint32_t prev = prev_lvl < 0 ? first : (uint32_t)prev_lvl;
        prev_lvl = first;
        key.clear();
        for (int32_t x = start[l]; x < start[l + 1]; ++x) {
          const int32_t i = byl[x];
          key.push_back({-(kind ? nup[i] : nlo[i]), i});
        }
        std::sort(key.begin(), key.end());
        size_t a = 0;
        std::vector<int32_t> scnt;
        while (a < key.size()) {
          // grow the piece while it fits the block (the size bound adds the
          // row-thread layout's padding of at most 16 bytes per value array)
          size_t b = a;
          int64_t nb = 0;
          while (b < key.size() && (int)(b - a) < rows_cap) {
            int w = -key[a].first;
            int64_t bytes = record_bytes((int)(b - a + 1), w, nb - key[b].first, nullptr, kind, p.factor_elem, bs,
                                         false, nullptr) + 16 * (int64_t)(w + 1);
            if (bytes > cap && b > a) break;
            nb += -key[b].first;
            ++b;
          }
          int n = (int)(b - a), w = -key[a].first;
          scnt.assign((size_t)w, 0);
          for (size_t t = a; t < b; ++t)
            for (int sl = 0; sl < -key[t].first; ++sl) scnt[sl] += 1;
          int64_t voff;
          int64_t bytes = record_bytes(n, w, nb, scnt.data(), kind, p.factor_elem, bs, p.row_thread, &voff);
          if (bytes > cap || w > 255) sub_fail[s] = 1;
          for (size_t t = a; t < b; ++t) out.push_back(key[t].second - r0);
          PieceDesc d{};
          d.off = off;
          d.meta = (uint32_t)n | ((uint32_t)w << 16) | ((uint32_t)kind << 24);
          d.nb = (uint32_t)nb;
          d.voff = (uint32_t)voff;
          d.lvl_first = first;
          d.prev_first = prev;
          for (int sl = 0; sl < std::min(w, kDescSlots); ++sl) d.cnt[sl] = (uint16_t)scnt[sl];
          sub_desc[s].push_back(d);
          sub_len[s] += bytes;
          off += (uint32_t)bytes;
          a = b;
        }
      }
    }
  });
  for (int s = 0; s < p.nsub; ++s)
    if (sub_fail[s]) {
      *why = "a piece record exceeds 1 GiB or has more than 255 blocks per row";
      return ILU0DD_ERR_SMEM;
    }
  int64_t soff = 0, npc = 0, nrw = 0;
  std::vector<int64_t> row_at(p.nsub);
  for (int s = 0; s < p.nsub; ++s) {
    CtaDesc& c = p.cta[s];
    const int64_t len = sub_len[s];
    if (len >= (1ll << 31)) {
      *why = "subdomain stream exceeds 2 GiB";
      return ILU0DD_ERR_INVALID;
    }
    c.stream_off = soff;
    c.stream_len = (int32_t)len;
    c.row0 = p.part_ptr[s];
    c.nrows = p.part_ptr[s + 1] - p.part_ptr[s];
    c.piece0 = (int32_t)npc;
    c.npieces = (int32_t)sub_desc[s].size();
    c.npieces_l = 0;
    for (const PieceDesc& d : sub_desc[s]) c.npieces_l += (d.meta >> 24) == 0;
    p.max_pieces = std::max(p.max_pieces, c.npieces);
    row_at[s] = nrw;
    npc += c.npieces;
    nrw += (int64_t)sub_rows[s].size();
    soff = align_up(soff + len, 128);
  }
  p.pieces.resize((size_t)npc);
  p.piece_rows.resize((size_t)nrw);
  p.piece_rows_off.resize((size_t)npc + 1);
  p.piece_rows_off[npc] = nrw;
  parallel_for(p.nsub, [&](int64_t s) {
    const CtaDesc& c = p.cta[s];
    std::copy(sub_desc[s].begin(), sub_desc[s].end(), p.pieces.begin() + c.piece0);
    std::copy(sub_rows[s].begin(), sub_rows[s].end(), p.piece_rows.begin() + row_at[s]);
    int64_t at = row_at[s];
    for (int32_t k = 0; k < c.npieces; ++k) {
      p.piece_rows_off[c.piece0 + k] = at;
      at += (int64_t)(sub_desc[s][k].meta & 0xFFFFu);
    }
  });
  p.stream_bytes = soff;
  p.n_pieces = (int64_t)p.pieces.size();
  p.smem_bytes = (size_t)align_up((int64_t)p.rmax * p.vec_row_bytes, 128) + kApplyTailSmem;
  if ((int64_t)p.smem_bytes > (int64_t)max_smem - kApplyStaticSmem) {
    *why = "subdomain vector (" + std::to_string((int64_t)p.rmax * p.vec_row_bytes) + " B) exceeds the " +
           std::to_string(max_smem) +
           " B of shared memory per block";
    return ILU0DD_ERR_SMEM;
  }
  // the row-flag apply (Algorithm 4's synchronization) adds one byte per row;
  // 0 when that does not fit
  p.smem_rowsync = p.smem_bytes + (size_t)align_up(p.rmax, 16);
  if ((int64_t)p.smem_rowsync > (int64_t)max_smem - kApplyStaticSmem) p.smem_rowsync = 0;
  p.row_l0.resize((size_t)N);
  parallel_for(N, [&](int64_t i) { p.row_l0[i] = p.lev_l[i] == 0 ? 1 : 0; });

  tmark("pieces");
  // ---- sliced ELL for the SpMV
  p.nslices = (N + kSlice - 1) / kSlice;
  p.slice_off.assign(p.nslices + 1, 0);
  parallel_for(p.nslices, [&](int64_t k) {
    int32_t w = 0;
    for (int64_t r = k * kSlice; r < std::min<int64_t>(N, (k + 1) * kSlice); ++r)
      w = std::max(w, p.ap_rp[r + 1] - p.ap_rp[r]);
    p.slice_off[k + 1] = w;
  });
  for (int64_t k = 0; k < p.nslices; ++k) p.slice_off[k + 1] += p.slice_off[k];
  p.sell_slots = p.slice_off[p.nslices];

  // ---- dot tiles
  p.ntiles = (N + kDotTile - 1) / kDotTile;
  p.ntiles_pow2 = 1;
  while (p.ntiles_pow2 < p.ntiles) p.ntiles_pow2 *= 2;

  // ---- workspace layout
  size_t cur = 0;
  auto take = [&](size_t bytes) {
    size_t at = cur;
    cur = (size_t)align_up((int64_t)(cur + bytes), 256);
    return at;
  };
  Plan::Layout& L = p.lay;
  L.stream = take((size_t)p.stream_bytes);
  L.cta = take(sizeof(CtaDesc) * (size_t)p.nsub);
  L.pieces = take(sizeof(PieceDesc) * (size_t)std::max<int64_t>(1, p.n_pieces));
  L.sell_off = take(sizeof(int32_t) * (size_t)(p.nslices + 1));
  L.sell_col = take(sizeof(int32_t) * (size_t)p.sell_slots * kSlice);
  L.sell_val = take(sizeof(double) * bs * bs * (size_t)p.sell_slots * kSlice);
  L.perm = take(sizeof(int32_t) * (size_t)N);
  L.iperm = take(sizeof(int32_t) * (size_t)N);
  L.row_l0 = take((size_t)N);
  for (int v = 0; v < kNumVec; ++v) L.vec[v] = take(sizeof(double) * bs * (size_t)N);
  L.partials = take(sizeof(double) * 5 * (size_t)p.ntiles_pow2);
  L.counters = take(sizeof(uint32_t) * 16);
  L.scal = take(sizeof(SolverScalars));
  int32_t maxit = o->maxit > 0 ? o->maxit : 10000;
  L.hist = take(sizeof(double) * (size_t)(maxit + 2));
  L.err = take(sizeof(int32_t) * 4);
  L.total = cur;

  // ---- algorithmic bytes (values + int32 column indices + row pointers of L
  // and U + FP64 r in and z out; SpMV: values + columns + row pointers + x, y)
  const int64_t bb = (int64_t)bs * bs;
  p.apply_bytes = bb * p.factor_elem * (p.nL + p.nU + N) + 4 * (p.nL + p.nU) + 8ll * (N + 1) + 16ll * bs * N;
  p.spmv_bytes = (8 * bb + 4) * p.nnzb + 4ll * (N + 1) + 16ll * bs * N;
  tmark("sell+layout");
  if (o->trace) std::fprintf(stderr, "[ilu0dd] plan:%s\n", tlog.c_str());
  return ILU0DD_OK;
}

int partition_bfs(const ilu0dd_bsr* A, int32_t part_rows, int32_t* part_id, int32_t* nparts) {
  if (!A || !part_id || !nparts || part_rows <= 0 || A->n_brows < 0 || !A->row_ptr || !A->col_idx)
    return ILU0DD_ERR_INVALID;
  const int32_t N = A->n_brows;
  const int32_t* rp = A->row_ptr;
  const int32_t* ci = A->col_idx;
  for (int32_t i = 0; i < N; ++i)
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
      if (ci[q] < 0 || ci[q] >= N) return ILU0DD_ERR_INVALID;
  // neighbours: the pattern of A + A^T without the diagonal, ascending, unique
  std::vector<int64_t> off((size_t)N + 1, 0);
  for (int32_t i = 0; i < N; ++i)
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
      if (ci[q] != i) {
        off[i + 1]++;
        off[ci[q] + 1]++;
      }
  for (int32_t i = 0; i < N; ++i) off[i + 1] += off[i];
  RawVec<int32_t> nb((size_t)off[N]);
  {
    std::vector<int64_t> at(off.begin(), off.end() - 1);
    for (int32_t i = 0; i < N; ++i)
      for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
        if (ci[q] != i) {
          nb[at[i]++] = ci[q];
          nb[at[ci[q]]++] = i;
        }
  }
  std::vector<int64_t> len((size_t)N);
  parallel_for(N, [&](int64_t i) {
    int32_t* b = nb.data() + off[i];
    int32_t* e = nb.data() + off[i + 1];
    std::sort(b, e);
    len[i] = std::unique(b, e) - b;
  });
  // 1. seed order: breadth-first, component by component; a component's order
  //    starts at the last vertex that a first search from its smallest vertex reaches
  std::vector<uint8_t> done((size_t)N, 0);
  std::vector<int32_t> mark((size_t)N, -1), queue((size_t)N), order;
  order.reserve((size_t)N);
  int32_t pass = 0;
  auto bfs = [&](int32_t from, bool place) {
    size_t h = 0, t = 0;
    queue[t++] = from;
    mark[from] = pass;
    int32_t last = from;
    while (h < t) {
      const int32_t w = queue[h++];
      last = w;
      if (place) {
        done[w] = 1;
        order.push_back(w);
      }
      for (int64_t q = off[w]; q < off[w] + len[w]; ++q) {
        const int32_t x = nb[q];
        if (!done[x] && mark[x] != pass) {
          mark[x] = pass;
          queue[t++] = x;
        }
      }
    }
    ++pass;
    return last;
  };
  for (int32_t u = 0; u < N; ++u) {
    if (done[u]) continue;
    const int32_t far = bfs(u, false);
    bfs(far, true);
  }
  // 2. parts grown one after another as breadth-first balls over unassigned
  //    vertices, each from the first unassigned vertex of the seed order; a
  //    ball that runs out continues the part from the next seed
  for (int32_t i = 0; i < N; ++i) part_id[i] = -1;
  int32_t part = 0, size = 0, assigned = 0;
  size_t next = 0;
  while (assigned < N) {
    while (part_id[order[next]] >= 0) ++next;
    size_t h = 0, t = 0;
    queue[t++] = order[next];
    mark[order[next]] = pass;
    while (h < t && size < part_rows) {
      const int32_t w = queue[h++];
      part_id[w] = part;
      ++size;
      ++assigned;
      for (int64_t q = off[w]; q < off[w] + len[w]; ++q) {
        const int32_t x = nb[q];
        if (part_id[x] < 0 && mark[x] != pass) {
          mark[x] = pass;
          queue[t++] = x;
        }
      }
    }
    ++pass;
    if (size == part_rows) {
      ++part;
      size = 0;
    }
  }
  *nparts = (N + part_rows - 1) / part_rows;
  return ILU0DD_OK;
}

int factor_ildu0(const Plan& p, const double* aval, std::vector<double>* Fp, std::vector<double>* invDp,
                 int32_t* bad_row) {
  std::vector<double>& F = *Fp;
  std::vector<double>& invD = *invDp;
  const int64_t kept = p.dd_rp[p.N];
  const int bs = p.bs, bb = bs * bs;
  F.assign(bb * (size_t)kept, 0.0);
  invD.assign(bb * (size_t)p.N, 0.0);
  std::vector<int32_t> fail(p.nsub, -1);
  parallel_for(p.nsub, [&](int64_t s) {
    const int32_t r0 = p.part_ptr[s], r1 = p.part_ptr[s + 1];
    const int64_t q0 = p.dd_rp[r0], q1 = p.dd_rp[r1];
    // W: working rows of the subdomain (Algorithm 7, U <- A)
    std::vector<double> W(bb * (size_t)(q1 - q0));
    for (int64_t q = q0; q < q1; ++q)
      std::memcpy(&W[bb * (q - q0)], aval + bb * p.ap_src[p.dd_ap[q]], bb * sizeof(double));
    std::vector<int64_t> pos(r1 - r0, -1);
    std::vector<int64_t> diag(r1 - r0, -1);
    double Lij[9], prod[9];
    for (int32_t i = r0; i < r1; ++i) {
      for (int64_t q = p.dd_rp[i]; q < p.dd_rp[i + 1]; ++q) {
        pos[p.dd_col[q] - r0] = q - q0;
        if (p.dd_col[q] == i) diag[i - r0] = q - q0;
      }
      if (diag[i - r0] < 0) { fail[s] = i; return; }
      for (int64_t q = p.dd_rp[i]; q < p.dd_rp[i + 1] && p.dd_col[q] < i; ++q) {
        int32_t j = p.dd_col[q];
        // L_ij = W_ij U_jj^-1 (U_jj^-1 is invD of row j, already final)
        mul_bs(bs, &W[bb * (q - q0)], &invD[bb * (size_t)j], Lij);
        std::memcpy(&W[bb * (q - q0)], Lij, bb * sizeof(double));
        for (int64_t t = p.dd_rp[j + 1] - 1; t >= p.dd_rp[j] && p.dd_col[t] > j; --t) {
          int64_t at = pos[p.dd_col[t] - r0];
          if (at < 0) continue;
          mul_bs(bs, Lij, &W[bb * (t - q0)], prod);
          for (int e = 0; e < bb; ++e) W[bb * at + e] -= prod[e];
        }
      }
      if (!inverse_bs(bs, &W[bb * diag[i - r0]], &invD[bb * (size_t)i])) { fail[s] = i; return; }
      for (int64_t q = p.dd_rp[i]; q < p.dd_rp[i + 1]; ++q) pos[p.dd_col[q] - r0] = -1;
    }
    // ILDU0 (Algorithm 7, lower half, read as scaling the strictly-upper blocks):
    // F <- L at lower positions, U~_ik = D_i^-1 U_ik at upper positions.
    for (int32_t i = r0; i < r1; ++i)
      for (int64_t q = p.dd_rp[i]; q < p.dd_rp[i + 1]; ++q) {
        double* dst = &F[bb * (size_t)q];
        if (p.dd_col[q] < i) {
          std::memcpy(dst, &W[bb * (q - q0)], bb * sizeof(double));
        } else if (p.dd_col[q] > i) {
          mul_bs(bs, &invD[bb * (size_t)i], &W[bb * (q - q0)], dst);
        }
      }
  });
  for (int s = 0; s < p.nsub; ++s)
    if (fail[s] >= 0) {
      if (bad_row) *bad_row = fail[s];
      return ILU0DD_ERR_ZERO_PIVOT;
    }
  return ILU0DD_OK;
}

void ildu0_from_w(const Plan& p, const std::vector<double>& W, const std::vector<double>& invD,
                  std::vector<double>* Fp) {
  std::vector<double>& F = *Fp;
  F.assign(W.size(), 0.0);
  const int bs = p.bs, bb = bs * bs;
  parallel_for(p.N, [&](int64_t i) {
    for (int64_t q = p.dd_rp[i]; q < p.dd_rp[i + 1]; ++q) {
      double* dst = &F[bb * (size_t)q];
      if (p.dd_col[q] < i) {
        std::memcpy(dst, &W[bb * (size_t)q], bb * sizeof(double));
      } else if (p.dd_col[q] > i) {
        mul_bs(bs, &invD[bb * (size_t)i], &W[bb * (size_t)q], dst);
      }
    }
  });
}

bool df64_range_ok(const std::vector<double>& F, const std::vector<double>& invD) {
  const double lo = std::ldexp(1.0, -70), hi = std::ldexp(1.0, 100);
  auto ok = [&](const std::vector<double>& v) {
    for (double x : v) {
      const double a = std::fabs(x);
      if (a != 0.0 && !(a >= lo && a <= hi)) return false;
    }
    return true;
  };
  return ok(F) && ok(invD);
}

void pack_stream(const Plan& p, const std::vector<double>& F, const std::vector<double>& invD,
                 std::vector<uint8_t>* out) {
  std::vector<uint8_t>& S = *out;
  S.assign((size_t)p.stream_bytes, 0);
  const int fe = p.factor_elem, fp = p.factor_prec, bs = p.bs, bb = bs * bs;
  parallel_for(p.nsub, [&](int64_t s) {
    const CtaDesc& c = p.cta[s];
    for (int32_t k = 0; k < c.npieces; ++k) {
      const PieceDesc& d = p.pieces[c.piece0 + k];
      const int32_t* rows = &p.piece_rows[p.piece_rows_off[c.piece0 + k]];
      const int n = (int)(d.meta & 0xFFFF), w = (int)((d.meta >> 16) & 0xFF), kind = (int)(d.meta >> 24);
      uint8_t* rec = S.data() + c.stream_off + d.off;
      // blocks of each row (ascending column), strictly lower (kind 0) or upper (kind 1)
      std::vector<std::vector<int64_t>> blk(n);
      for (int t = 0; t < n; ++t) {
        int32_t i = c.row0 + rows[t];
        for (int64_t q = p.dd_rp[i]; q < p.dd_rp[i + 1]; ++q)
          if (kind ? p.dd_col[q] > i : p.dd_col[q] < i) blk[t].push_back(q);
      }
      std::vector<uint16_t> cnt(w, 0);
      for (int slot = 0; slot < w; ++slot)
        for (int t = 0; t < n; ++t) cnt[slot] += (int)blk[t].size() > slot;
      uint16_t* h = reinterpret_cast<uint16_t*>(rec);
      for (int slot = 0; slot < w; ++slot) h[slot] = cnt[slot];
      for (int t = 0; t < n; ++t) h[w + t] = (uint16_t)rows[t];
      int64_t cpos = w + n;
      for (int slot = 0; slot < w; ++slot)
        for (int t = 0; t < cnt[slot]; ++t) h[cpos++] = (uint16_t)(p.dd_col[blk[t][slot]] - c.row0);
      uint8_t* v = rec + d.voff;
      if (p.row_thread) {
        // row-thread layout: entry e = 3a + c of row t in 16-byte planes
        if (kind) {
          for (int t = 0; t < n; ++t)
            for (int e = 0; e < 9; ++e)
              put_factor(v + rt_value_offset(e, t, n, fe), fp, invD[9 * (size_t)(c.row0 + rows[t]) + e]);
          v += rt_slot_bytes(n, fe);
        }
        for (int slot = 0; slot < w; ++slot) {
          const int cs = cnt[slot];
          for (int t = 0; t < cs; ++t)
            for (int e = 0; e < 9; ++e) put_factor(v + rt_value_offset(e, t, cs, fe), fp, F[9 * (size_t)blk[t][slot] + e]);
          v += rt_slot_bytes(cs, fe);
        }
        continue;
      }
      // entry [a][c] of row t's block at (c * count + t) * bs + a
      if (kind) {
        for (int cc = 0; cc < bs; ++cc)
          for (int t = 0; t < n; ++t)
            for (int a = 0; a < bs; ++a)
              put_factor(v + (((int64_t)cc * n + t) * bs + a) * fe, fp,
                         invD[bb * (size_t)(c.row0 + rows[t]) + bs * a + cc]);
        v += (int64_t)bb * n * fe;
      }
      for (int slot = 0; slot < w; ++slot) {
        const int cs = cnt[slot];
        for (int cc = 0; cc < bs; ++cc)
          for (int t = 0; t < cs; ++t)
            for (int a = 0; a < bs; ++a)
              put_factor(v + (((int64_t)cc * cs + t) * bs + a) * fe, fp,
                         F[bb * (size_t)blk[t][slot] + bs * a + cc]);
        v += (int64_t)bb * cs * fe;
      }
    }
  });
}

void pack_sell(const Plan& p, const double* aval, std::vector<int32_t>* cols, std::vector<double>* vals) {
  const int bb = p.bs * p.bs;
  cols->assign((size_t)p.sell_slots * kSlice, 0);
  vals->assign((size_t)p.sell_slots * kSlice * bb, 0.0);
  parallel_for(p.nslices, [&](int64_t k) {
    int64_t so = p.slice_off[k];
    int32_t w = p.slice_off[k + 1] - p.slice_off[k];
    for (int lane = 0; lane < kSlice; ++lane) {
      int64_t r = k * kSlice + lane;
      for (int32_t s = 0; s < w; ++s) {
        int64_t slot = so + s;
        int32_t col = r < p.N ? (int32_t)r : 0;
        double blk[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (r < p.N && s < p.ap_rp[r + 1] - p.ap_rp[r]) {
          int64_t q = p.ap_rp[r] + s;
          col = p.ap_col[q];
          std::memcpy(blk, aval + bb * p.ap_src[q], bb * sizeof(double));
        }
        (*cols)[(size_t)slot * kSlice + lane] = col;
        for (int e = 0; e < bb; ++e) (*vals)[((size_t)slot * bb + e) * kSlice + lane] = blk[e];
      }
    }
  });
}

}  // namespace ilu0dd
