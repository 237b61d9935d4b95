/*
 * Seeded synthetic inputs: 3D 7-point stencils with 3 unknowns per cell,
 * stored as BSR with 3x3 row-major blocks in natural cell order
 * gidx = i + nx*(j + ny*k) (the ordering the geometric-cut partition of
 * Algorithm 2 assumes).
 *
 * This file holds no arithmetic of the solver or of the preconditioner. It is
 * the common input source of the CPU oracle and of the CUDA library; both
 * consume the arrays it writes.
 *
 * Random numbers: a counter-based generator. Each draw is the SplitMix64
 * output function (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014) applied to a counter derived from
 * (seed, stream, index), so any entry can be recomputed on its own.
 *
 * Two coefficient models:
 *  - "laplace": off-diagonal block of each existing face = -I + U(-0.1,0.1)
 *    per entry; diagonal block = 6.5*I + U(-0.1,0.1) per entry.
 *  - "layered": cell coefficient kappa = exp(2*g), g ~ N(0,1) drawn once per
 *    (i, j, floor(k/8)); face coupling c_ab = H(kappa_a, kappa_b)*(I + P_ab)
 *    with H the harmonic mean and P_ab a 3x3 U(-0.1,0.1) perturbation drawn per
 *    directed face; off-diagonal block = -c_ab; diagonal block = sum of the
 *    cell's face couplings + 0.01*I.
 * x* ~ U(-1,1) per unknown; b = A x* (per scalar row, blocks in ascending
 * column order, entries c = 0..2, fused multiply-add from 0).
 *
 * A third, unstructured input (synth_unstructured) stands in for the paper's
 * graph-partitioned matrices: a grid of cells where every face neighbour and,
 * with probability 0.35 per pair, each edge or corner neighbour of the
 * 27-point neighbourhood is coupled, renumbered by a seeded random
 * permutation so that the matrix order carries no geometry.
 *
 * Build: gcc -O2 -ffp-contract=off -shared -fPIC (no fast-math), so the same
 * source gives the same bits on x86-64 and aarch64 apart from libm's exp,
 * log and cos (used by the layered model only).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { STREAM_DIAG = 1, STREAM_OFF = 2, STREAM_XSTAR = 3, STREAM_FIELD = 4, STREAM_SIDES = 5, STREAM_PERM = 6,
       STREAM_EDGE = 7 };

static inline uint64_t sm64_out(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Counter -> 64 random bits. */
uint64_t synth_bits(uint64_t seed, uint64_t stream, uint64_t index) {
  uint64_t key = sm64_out(seed * 0x9E3779B97F4A7C15ULL + stream);
  return sm64_out(key + (index + 1) * 0x9E3779B97F4A7C15ULL);
}

/* Uniform double in [0, 1) with 53 random bits. */
double synth_unit(uint64_t seed, uint64_t stream, uint64_t index) {
  return (double)(synth_bits(seed, stream, index) >> 11) * 0x1.0p-53;
}

static inline double unif(uint64_t seed, uint64_t stream, uint64_t index, double lo, double hi) {
  return lo + (hi - lo) * synth_unit(seed, stream, index);
}

/* Face directions of a cell: 0:-x 1:+x 2:-y 3:+y 4:-z 5:+z. */
static inline int64_t nbr(int nx, int ny, int nz, int i, int j, int k, int dir) {
  switch (dir) {
    case 0: return i > 0 ? (int64_t)(i - 1) + (int64_t)nx * (j + (int64_t)ny * k) : -1;
    case 1: return i + 1 < nx ? (int64_t)(i + 1) + (int64_t)nx * (j + (int64_t)ny * k) : -1;
    case 2: return j > 0 ? (int64_t)i + (int64_t)nx * ((j - 1) + (int64_t)ny * k) : -1;
    case 3: return j + 1 < ny ? (int64_t)i + (int64_t)nx * ((j + 1) + (int64_t)ny * k) : -1;
    case 4: return k > 0 ? (int64_t)i + (int64_t)nx * (j + (int64_t)ny * (k - 1)) : -1;
    default: return k + 1 < nz ? (int64_t)i + (int64_t)nx * (j + (int64_t)ny * (k + 1)) : -1;
  }
}

/* Number of stored blocks: one diagonal block per cell plus two per interior face. */
int64_t synth_nnzb(int nx, int ny, int nz) {
  int64_t n = (int64_t)nx * ny * nz;
  int64_t faces = (int64_t)(nx - 1) * ny * nz + (int64_t)nx * (ny - 1) * nz + (int64_t)nx * ny * (nz - 1);
  return n + 2 * faces;
}

/* Row order of a cell's blocks in ascending column: -z, -y, -x, self, +x, +y, +z. */
static const int k_order[7] = {4, 2, 0, -1, 1, 3, 5};

/* Sparsity pattern only (row_ptr[N+1], col[nnzb]). */
void synth_pattern(int nx, int ny, int nz, int32_t* row_ptr, int32_t* col) {
  int64_t p = 0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t g = (int64_t)i + (int64_t)nx * (j + (int64_t)ny * k);
        row_ptr[g] = (int32_t)p;
        for (int o = 0; o < 7; ++o) {
          int d = k_order[o];
          int64_t c = d < 0 ? g : nbr(nx, ny, nz, i, j, k, d);
          if (c >= 0) col[p++] = (int32_t)c;
        }
      }
  row_ptr[(int64_t)nx * ny * nz] = (int32_t)p;
}

static double layered_kappa(uint64_t seed, int nx, int ny, int i, int j, int k) {
  uint64_t id = (uint64_t)i + (uint64_t)nx * ((uint64_t)j + (uint64_t)ny * (uint64_t)(k / 8));
  double u1 = synth_unit(seed, STREAM_FIELD, 2 * id);
  double u2 = synth_unit(seed, STREAM_FIELD, 2 * id + 1);
  /* Box-Muller: 1-u1 lies in (0, 1], so the logarithm is finite. */
  double g = sqrt(-2.0 * log(1.0 - u1)) * cos(6.283185307179586 * u2);
  return exp(2.0 * g);
}

/*
 * Full system with bs x bs blocks (bs = 3: the BSR inputs; bs = 1: the scalar
 * CSR form of the same stencil, whose value is the 3x3 model's (0,0) entry).
 * model 0 = laplace, 1 = layered. Writes row_ptr[N+1], col[nnzb],
 * val[nnzb*bs*bs], xstar[bs*N], b[bs*N]. Returns the number of blocks.
 */
int64_t synth_system_bs(int model, int bs, int nx, int ny, int nz, uint64_t seed, int32_t* row_ptr,
                        int32_t* col, double* val, double* xstar, double* b) {
  const int bb = bs * bs;
  int64_t n = (int64_t)nx * ny * nz;
  synth_pattern(nx, ny, nz, row_ptr, col);
  for (int64_t g = 0; g < n; ++g)
    for (int a = 0; a < bs; ++a) xstar[bs * g + a] = unif(seed, STREAM_XSTAR, (uint64_t)(bs * g + a), -1.0, 1.0);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t g = (int64_t)i + (int64_t)nx * (j + (int64_t)ny * k);
        int64_t p = row_ptr[g];
        double diag[9];
        double ka = model ? layered_kappa(seed, nx, ny, i, j, k) : 0.0;
        if (model == 0) {
          for (int e = 0; e < bb; ++e)
            diag[e] = (e % (bs + 1) == 0 ? 6.5 : 0.0) + unif(seed, STREAM_DIAG, (uint64_t)(9 * g + e), -0.1, 0.1);
        } else {
          for (int e = 0; e < bb; ++e) diag[e] = (e % (bs + 1) == 0 ? 0.01 : 0.0);
        }
        int64_t pdiag = -1;
        for (int o = 0; o < 7; ++o) {
          int d = k_order[o];
          if (d < 0) { pdiag = p++; continue; }
          int64_t c = nbr(nx, ny, nz, i, j, k, d);
          if (c < 0) continue;
          double* blk = val + bb * p;
          uint64_t base = (uint64_t)(6 * g + d) * 9;
          if (model == 0) {
            for (int e = 0; e < bb; ++e)
              blk[e] = (e % (bs + 1) == 0 ? -1.0 : 0.0) + unif(seed, STREAM_OFF, base + e, -0.1, 0.1);
          } else {
            int ci = (int)(c % nx), cj = (int)((c / nx) % ny), ck = (int)(c / ((int64_t)nx * ny));
            double kb = layered_kappa(seed, nx, ny, ci, cj, ck);
            double h = 2.0 * ka * kb / (ka + kb);
            for (int e = 0; e < bb; ++e) {
              double cpl = h * ((e % (bs + 1) == 0 ? 1.0 : 0.0) + unif(seed, STREAM_OFF, base + e, -0.1, 0.1));
              blk[e] = -cpl;
              diag[e] += cpl;
            }
          }
          ++p;
        }
        memcpy(val + bb * pdiag, diag, bb * sizeof(double));
      }
  for (int64_t g = 0; g < n; ++g)
    for (int a = 0; a < bs; ++a) {
      double acc = 0.0;
      for (int64_t p = row_ptr[g]; p < row_ptr[g + 1]; ++p)
        for (int c = 0; c < bs; ++c) acc = fma(val[bb * p + bs * a + c], xstar[bs * (int64_t)col[p] + c], acc);
      b[bs * g + a] = acc;
    }
  return row_ptr[n];
}

int64_t synth_system(int model, int nx, int ny, int nz, uint64_t seed, int32_t* row_ptr, int32_t* col,
                     double* val, double* xstar, double* b) {
  return synth_system_bs(model, 3, nx, ny, nz, seed, row_ptr, col, val, xstar, b);
}

/* Grid sides of one system of a ragged batch: integers uniform in [lo, hi]. */
void synth_sides(uint64_t seed, int lo, int hi, int32_t* sides) {
  for (int a = 0; a < 3; ++a)
    sides[a] = lo + (int)(synth_unit(seed, STREAM_SIDES, (uint64_t)a) * (double)(hi - lo + 1));
}

/* ---- unstructured input ------------------------------------------------ */

/* Offset o in [0, 27) of the 27-point neighbourhood: (di, dj, dk) in {-1,0,1}^3. */
static inline void off27(int o, int* di, int* dj, int* dk) {
  *di = o % 3 - 1;
  *dj = (o / 3) % 3 - 1;
  *dk = o / 9 - 1;
}

/* Whether cells g (at i, j, k) and its neighbour at offset o are coupled: face
 * neighbours always, the others with probability 0.35, drawn once per
 * unordered pair (from the smaller cell's side) so the pattern is symmetric. */
static int coupled(uint64_t seed, int nx, int ny, int nz, int i, int j, int k, int o, int64_t* out) {
  int di, dj, dk;
  off27(o, &di, &dj, &dk);
  if (o == 13) return 0;
  int a = i + di, b = j + dj, c = k + dk;
  if (a < 0 || a >= nx || b < 0 || b >= ny || c < 0 || c >= nz) return 0;
  int64_t g = (int64_t)i + (int64_t)nx * (j + (int64_t)ny * k);
  int64_t h = (int64_t)a + (int64_t)nx * (b + (int64_t)ny * c);
  *out = h;
  if (abs(di) + abs(dj) + abs(dk) == 1) return 1;
  int64_t lo = g < h ? g : h;
  int olo = g < h ? o : 26 - o; /* the same pair seen from the smaller cell */
  return synth_unit(seed, STREAM_EDGE, (uint64_t)(27 * lo + olo)) < 0.35;
}

/* Renumbering: new_of_old[g] from a Fisher-Yates shuffle driven by the counter generator. */
static void renumber(uint64_t seed, int64_t n, int32_t* new_of_old) {
  int32_t* old_of_new = new_of_old; /* built in place, then inverted */
  for (int64_t t = 0; t < n; ++t) old_of_new[t] = (int32_t)t;
  for (int64_t t = n - 1; t > 0; --t) {
    int64_t r = (int64_t)(synth_bits(seed, STREAM_PERM, (uint64_t)t) % (uint64_t)(t + 1));
    int32_t tmp = old_of_new[t];
    old_of_new[t] = old_of_new[r];
    old_of_new[r] = tmp;
  }
}

/* Blocks of the unstructured system (call before synth_unstructured). */
int64_t synth_unstructured_nnzb(int nx, int ny, int nz, uint64_t seed) {
  int64_t m = 0, h;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        m += 1;
        for (int o = 0; o < 27; ++o) m += coupled(seed, nx, ny, nz, i, j, k, o, &h);
      }
  return m;
}

/*
 * The unstructured system in its renumbered order: row_ptr[N+1], col[nnzb]
 * (ascending per row), val[9*nnzb], xstar[3N], b[3N]; `scratch` holds 2N
 * int32. A coupling of weight w (1 across a face, 0.5 across an edge or a
 * corner) gives the off-diagonal block -w*(I + P), P ~ U(-0.1, 0.1) per entry
 * and directed coupling; the diagonal block is (sum of the row's weights +
 * 0.5)*I + U(-0.1, 0.1) per entry, a Laplacian-like system. Returns nnzb.
 */
int64_t synth_unstructured(int nx, int ny, int nz, uint64_t seed, int32_t* row_ptr, int32_t* col, double* val,
                           double* xstar, double* b, int32_t* scratch) {
  int64_t n = (int64_t)nx * ny * nz;
  int32_t* old_of_new = scratch;
  int32_t* new_of_old = scratch + n;
  renumber(seed, n, old_of_new);
  for (int64_t t = 0; t < n; ++t) new_of_old[old_of_new[t]] = (int32_t)t;
  /* row lengths in the new order */
  row_ptr[0] = 0;
  for (int64_t t = 0; t < n; ++t) {
    int64_t g = old_of_new[t], h;
    int i = (int)(g % nx), j = (int)((g / nx) % ny), k = (int)(g / ((int64_t)nx * ny));
    int len = 1;
    for (int o = 0; o < 27; ++o) len += coupled(seed, nx, ny, nz, i, j, k, o, &h);
    row_ptr[t + 1] = row_ptr[t] + len;
  }
  for (int64_t t = 0; t < n; ++t) {
    int64_t g = old_of_new[t], h;
    int i = (int)(g % nx), j = (int)((g / nx) % ny), k = (int)(g / ((int64_t)nx * ny));
    /* (new column, source) pairs; source -1 = diagonal, else offset o */
    int32_t cc[28], src[28];
    int len = 0;
    cc[len] = (int32_t)t;
    src[len++] = -1;
    for (int o = 0; o < 27; ++o)
      if (coupled(seed, nx, ny, nz, i, j, k, o, &h)) {
        cc[len] = new_of_old[h];
        src[len++] = o;
      }
    for (int x = 1; x < len; ++x) /* insertion sort by column */
      for (int y = x; y > 0 && cc[y - 1] > cc[y]; --y) {
        int32_t tc = cc[y]; cc[y] = cc[y - 1]; cc[y - 1] = tc;
        int32_t ts = src[y]; src[y] = src[y - 1]; src[y - 1] = ts;
      }
    double wsum = 0.0; /* coupling weights of the row: 1 per face, 0.5 per edge or corner */
    for (int x = 0; x < len; ++x)
      if (src[x] >= 0) {
        int di, dj, dk;
        off27(src[x], &di, &dj, &dk);
        wsum += abs(di) + abs(dj) + abs(dk) == 1 ? 1.0 : 0.5;
      }
    for (int x = 0; x < len; ++x) {
      int64_t p = row_ptr[t] + x;
      col[p] = cc[x];
      double* blk = val + 9 * p;
      if (src[x] < 0) {
        for (int e = 0; e < 9; ++e)
          blk[e] = (e % 4 == 0 ? wsum + 0.5 : 0.0) + unif(seed, STREAM_DIAG, (uint64_t)(9 * g + e), -0.1, 0.1);
      } else {
        int di, dj, dk;
        off27(src[x], &di, &dj, &dk);
        double w = abs(di) + abs(dj) + abs(dk) == 1 ? 1.0 : 0.5;
        for (int e = 0; e < 9; ++e)
          blk[e] = -w * ((e % 4 == 0 ? 1.0 : 0.0) + unif(seed, STREAM_OFF, (uint64_t)((27 * g + src[x]) * 9 + e), -0.1, 0.1));
      }
    }
  }
  for (int64_t t = 0; t < n; ++t)
    for (int a = 0; a < 3; ++a) xstar[3 * t + a] = unif(seed, STREAM_XSTAR, (uint64_t)(3 * t + a), -1.0, 1.0);
  for (int64_t t = 0; t < n; ++t)
    for (int a = 0; a < 3; ++a) {
      double acc = 0.0;
      for (int64_t p = row_ptr[t]; p < row_ptr[t + 1]; ++p)
        for (int c = 0; c < 3; ++c) acc = fma(val[9 * p + 3 * a + c], xstar[3 * (int64_t)col[p] + c], acc);
      b[3 * t + a] = acc;
    }
  return row_ptr[n];
}
