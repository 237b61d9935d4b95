/*
 * CPU oracle for subdomain-wise ILU0-preconditioned BiCGSTAB on 3x3 BSR
 * matrices (arXiv 2508.04917). TEST INFRASTRUCTURE ONLY: the test suite, the
 * smoke check and the benchmark's CPU-baseline leg are its only callers. The
 * CUDA library never links, loads or calls it, and it shares no code with it.
 *
 * Plain FP64 loops, written for reading, not for speed. Every function says
 * which part of the paper it follows. Indices are int32 (rows, columns) and
 * int64 (block positions). Blocks are bs x bs row-major (bs*bs doubles each)
 * with bs = 3 (the BSR inputs: 3 unknowns per cell) or bs = 1 (scalar CSR,
 * the paper's other input format).
 *
 * Readings of passages the paper leaves open (the same list is kept with the
 * design notes of the project):
 *  - Algorithm 2 with ceil-division: edge subdomains may be smaller.
 *  - Algorithm 3 permutation semantics: perm[new] = old, iperm[old] = new.
 *    Rows of one subdomain keep ascending natural order (stable grouping).
 *  - Section 3.2 drop: keep block (i, j) iff rows i and j carry the same label.
 *  - Algorithm 7, block form: L unit block-lower with L_ij = W_ij * U_jj^-1,
 *    U keeps full 3x3 diagonal blocks; the update loop runs over k > j.
 *  - 3x3 solves: Gaussian elimination with partial pivoting.
 *  - ILDU0 form (Section 4.3, Algorithm 7 post-processing), block reading:
 *    inv_D_i = U_ii^-1 by Gauss-Jordan elimination with partial pivoting,
 *    L_ij = W_ij * inv_D_j (the block form of U[i,j] / U[j,j], with the
 *    stored inverse), U~_ik = inv_D_i * U_ik for k > i (the strictly-upper
 *    blocks; the algorithm's "j < i" loop is read as the text describes).
 *  - Algorithm 1 with K1 = I, K2 = M = LU (right preconditioning), x0 = 0,
 *    stop when ||r||_2 / ||b||_2 < rtol (checked on r_{j+1} only), then one
 *    restart from the true residual if the true residual misses rtol.
 *  - Dot products follow one fixed order (oracle_dot) that the GPU library
 *    implements independently; vector updates use the fused multiply-adds
 *    written below.
 *
 * Parity pins for every function are in the CPU test suite. Nothing in this
 * file is "parity unpinned".
 *
 * Loops over independent subdomains, rows and dot tiles carry OpenMP
 * pragmas. Built without -fopenmp they are ignored; built with it, every
 * result is the same bits (no loop with a pragma combines values across its
 * iterations).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Decomposition: Algorithm 2, Algorithm 3, Section 3.2                      */
/* ------------------------------------------------------------------------ */

static int ceil_div(int a, int b) { return (a + b - 1) / b; }

/* Algorithm 2: label of every cell from the grid and subdomain dimensions. */
void oracle_partition(int nx, int ny, int nz, int sx, int sy, int sz, int32_t* part_id) {
  int bx = ceil_div(nx, sx), by = ceil_div(ny, sy);
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < ny; ++j)
      for (int k = 0; k < nz; ++k) {
        int64_t gidx = (int64_t)i + (int64_t)nx * (j + (int64_t)ny * k);
        part_id[gidx] = (i / sx) + bx * ((j / sy) + by * (k / sz));
      }
}

/*
 * Graph partition for matrices without a grid (Section 3.1 partitions those
 * with METIS into parts of equal size; this is a plain stand-in with the same
 * output form): parts of part_rows rows (the last may be smaller) grown as
 * breadth-first balls. The graph is the pattern of A + A^T without the
 * diagonal; neighbours are visited in ascending index order.
 *  1. A seed order O: component by component, u = the smallest vertex not yet
 *     in O; a first search from u ends at its last visited vertex v (a far
 *     vertex of the component); a second search from v appends its visiting
 *     order to O.
 *  2. Parts one after another: the part's next seed is the first vertex of O
 *     not yet assigned; a search from it over unassigned vertices assigns
 *     them in visiting order until the part holds part_rows rows; if the
 *     search runs out first, the next seed of O continues the same part.
 * Returns the number of parts. Pinned in the CPU tests against this
 * definition on small graphs (paths, disconnected graphs, grids).
 */
int32_t oracle_partition_bfs(int32_t n, const int32_t* row_ptr, const int32_t* col, int32_t part_rows,
                             int32_t* part_id) {
  if (n <= 0 || part_rows <= 0) return 0;
  /* adjacency of A + A^T without the diagonal: count, fill, sort, drop duplicates */
  int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  for (int32_t i = 0; i < n; ++i)
    for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
      int32_t j = col[q];
      if (j == i) continue;
      deg[i + 1] += 1;
      deg[j + 1] += 1;
    }
  for (int32_t i = 0; i < n; ++i) deg[i + 1] += deg[i];
  int32_t* adj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(deg[n] > 0 ? deg[n] : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int32_t i = 0; i < n; ++i) fill[i] = deg[i];
  for (int32_t i = 0; i < n; ++i)
    for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
      int32_t j = col[q];
      if (j == i) continue;
      adj[fill[i]++] = j;
      adj[fill[j]++] = i;
    }
  int64_t* end = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int32_t i = 0; i < n; ++i) {
    int32_t* a = adj + deg[i];
    int64_t m = deg[i + 1] - deg[i];
    for (int64_t x = 1; x < m; ++x) /* insertion sort */
      for (int64_t y = x; y > 0 && a[y - 1] > a[y]; --y) {
        int32_t t = a[y];
        a[y] = a[y - 1];
        a[y - 1] = t;
      }
    int64_t u = 0;
    for (int64_t x = 0; x < m; ++x)
      if (x == 0 || a[x] != a[x - 1]) a[u++] = a[x];
    end[i] = deg[i] + u;
  }
  int32_t* stamp = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int32_t i = 0; i < n; ++i) stamp[i] = -1;
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  char* in_order = (char*)calloc((size_t)n, 1);
  int32_t placed = 0, search = 0;
  /* 1. seed order */
  for (int32_t u = 0; u < n; ++u) {
    if (in_order[u]) continue;
    int32_t head = 0, tail = 0, v = u;
    queue[tail++] = u;
    stamp[u] = search;
    while (head < tail) {
      int32_t w = queue[head++];
      v = w;
      for (int64_t q = deg[w]; q < end[w]; ++q) {
        int32_t x = adj[q];
        if (!in_order[x] && stamp[x] != search) {
          stamp[x] = search;
          queue[tail++] = x;
        }
      }
    }
    ++search;
    head = 0;
    tail = 0;
    queue[tail++] = v;
    stamp[v] = search;
    while (head < tail) {
      int32_t w = queue[head++];
      in_order[w] = 1;
      order[placed++] = w;
      for (int64_t q = deg[w]; q < end[w]; ++q) {
        int32_t x = adj[q];
        if (!in_order[x] && stamp[x] != search) {
          stamp[x] = search;
          queue[tail++] = x;
        }
      }
    }
    ++search;
  }
  /* 2. parts grown as breadth-first balls from seeds taken in that order */
  for (int32_t i = 0; i < n; ++i) part_id[i] = -1;
  int32_t part = 0, size = 0, next_seed = 0, assigned = 0;
  while (assigned < n) {
    while (part_id[order[next_seed]] >= 0) ++next_seed;
    int32_t seed = order[next_seed];
    int32_t head = 0, tail = 0;
    queue[tail++] = seed;
    stamp[seed] = search;
    while (head < tail && size < part_rows) {
      int32_t w = queue[head++];
      part_id[w] = part;
      ++size;
      ++assigned;
      for (int64_t q = deg[w]; q < end[w]; ++q) {
        int32_t x = adj[q];
        if (part_id[x] < 0 && stamp[x] != search) {
          stamp[x] = search;
          queue[tail++] = x;
        }
      }
    }
    ++search;
    if (size == part_rows) {
      ++part;
      size = 0;
    }
  }
  free(deg);
  free(adj);
  free(fill);
  free(end);
  free(stamp);
  free(queue);
  free(order);
  free(in_order);
  return (n + part_rows - 1) / part_rows;
}

/*
 * Section 3.1: rows grouped by label, in label order; inside a label the
 * original order is kept. perm[new] = old, iperm[old] = new, and
 * part_ptr[p] .. part_ptr[p+1] is the new row range of label p.
 */
void oracle_permutation(int32_t n, int32_t nparts, const int32_t* part_id, int32_t* perm,
                        int32_t* iperm, int32_t* part_ptr) {
  for (int32_t p = 0; p <= nparts; ++p) part_ptr[p] = 0;
  for (int32_t r = 0; r < n; ++r) part_ptr[part_id[r] + 1] += 1;
  for (int32_t p = 0; p < nparts; ++p) part_ptr[p + 1] += part_ptr[p];
  int32_t* next = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nparts > 0 ? nparts : 1));
  for (int32_t p = 0; p < nparts; ++p) next[p] = part_ptr[p];
  for (int32_t r = 0; r < n; ++r) {
    int32_t newr = next[part_id[r]]++;
    perm[newr] = r;
    iperm[r] = newr;
  }
  free(next);
}

/*
 * Algorithm 3 on BSR: new row i is old row perm[i]; its blocks move with
 * their columns renamed by iperm and are then sorted by new column.
 * val may be NULL (pattern only).
 */
void oracle_reorder(int32_t n, int bs, const int32_t* row_ptr, const int32_t* col, const double* val,
                    const int32_t* perm, const int32_t* iperm, int32_t* out_row_ptr,
                    int32_t* out_col, double* out_val) {
  const int bb = bs * bs;
  out_row_ptr[0] = 0;
  for (int32_t i = 0; i < n; ++i) {
    int32_t k = perm[i];
    out_row_ptr[i + 1] = row_ptr[k + 1] - row_ptr[k];
  }
  for (int32_t i = 0; i < n; ++i) out_row_ptr[i + 1] += out_row_ptr[i];
  for (int32_t i = 0; i < n; ++i) {
    int32_t m = perm[i];
    int64_t dst = out_row_ptr[i];
    for (int64_t q = row_ptr[m]; q < row_ptr[m + 1]; ++q, ++dst) {
      out_col[dst] = iperm[col[q]];
      if (val) memcpy(out_val + bb * dst, val + bb * q, bb * sizeof(double));
    }
    /* sort the row by new column (insertion sort; rows are short) */
    int64_t lo = out_row_ptr[i], hi = out_row_ptr[i + 1];
    for (int64_t a = lo + 1; a < hi; ++a) {
      int32_t c = out_col[a];
      double blk[9];
      if (val) memcpy(blk, out_val + bb * a, bb * sizeof(double));
      int64_t b = a - 1;
      while (b >= lo && out_col[b] > c) {
        out_col[b + 1] = out_col[b];
        if (val) memcpy(out_val + bb * (b + 1), out_val + bb * b, bb * sizeof(double));
        --b;
      }
      out_col[b + 1] = c;
      if (val) memcpy(out_val + bb * (b + 1), blk, bb * sizeof(double));
    }
  }
}

/*
 * Section 3.2: keep only blocks whose row and column lie in the same
 * subdomain. label[i] is the subdomain of (new) row i. With out_col == NULL
 * only the number of kept blocks is returned.
 */
int64_t oracle_drop(int32_t n, int bs, const int32_t* row_ptr, const int32_t* col, const double* val,
                    const int32_t* label, int32_t* out_row_ptr, int32_t* out_col, double* out_val) {
  const int bb = bs * bs;
  int64_t kept = 0;
  if (out_row_ptr) out_row_ptr[0] = 0;
  for (int32_t i = 0; i < n; ++i) {
    for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
      if (label[col[q]] != label[i]) continue;
      if (out_col) {
        out_col[kept] = col[q];
        if (val && out_val) memcpy(out_val + bb * kept, val + bb * q, bb * sizeof(double));
      }
      ++kept;
    }
    if (out_row_ptr) out_row_ptr[i + 1] = (int32_t)kept;
  }
  return kept;
}

/* ------------------------------------------------------------------------ */
/* bs x bs dense helpers (bs <= 3)                                            */
/* ------------------------------------------------------------------------ */

/*
 * Solve M y = f for a bs x bs row-major M by Gaussian elimination with
 * partial pivoting. Returns 0, or -1 for a zero or non-finite pivot.
 */
static int solve_bs(int bs, const double* M, const double* f, double* y) {
  double a[3][4];
  for (int r = 0; r < bs; ++r) {
    for (int c = 0; c < bs; ++c) a[r][c] = M[bs * r + c];
    a[r][bs] = f[r];
  }
  for (int c = 0; c < bs; ++c) {
    int piv = c;
    for (int r = c + 1; r < bs; ++r)
      if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
    if (!(fabs(a[piv][c]) > 0.0) || !isfinite(a[piv][c])) return -1;
    if (piv != c)
      for (int q = 0; q <= bs; ++q) {
        double t = a[c][q];
        a[c][q] = a[piv][q];
        a[piv][q] = t;
      }
    for (int r = c + 1; r < bs; ++r) {
      double m = a[r][c] / a[c][c];
      for (int q = c; q <= bs; ++q) a[r][q] = a[r][q] - m * a[c][q];
    }
  }
  for (int r = bs - 1; r >= 0; --r) {
    double s = a[r][bs];
    for (int q = r + 1; q < bs; ++q) s = s - a[r][q] * y[q];
    y[r] = s / a[r][r];
  }
  return 0;
}

/* X = W * U^-1, i.e. solve X U = W row by row: U^T x_r = w_r. */
static int right_divide_bs(int bs, const double* W, const double* U, double* X) {
  double Ut[9];
  for (int r = 0; r < bs; ++r)
    for (int c = 0; c < bs; ++c) Ut[bs * r + c] = U[bs * c + r];
  for (int r = 0; r < bs; ++r)
    if (solve_bs(bs, Ut, W + bs * r, X + bs * r)) return -1;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 7 (ILU0, block form) and the level sets of Algorithm 5         */
/* ------------------------------------------------------------------------ */

/*
 * Block ILU0 in IKJ order (Algorithm 7, upper half) on the dropped matrix.
 * lu receives L (strictly lower blocks; unit block diagonal implied) and U
 * (diagonal and upper blocks) in the pattern of the input. Returns 0, or
 * -(row+1) for a singular pivot block.
 */
int oracle_ilu0(int32_t n, int bs, const int32_t* row_ptr, const int32_t* col, const double* val, double* lu) {
  const int bb = bs * bs;
  int64_t nnzb = row_ptr[n];
  memcpy(lu, val, (size_t)nnzb * bb * sizeof(double));
  int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t* diag = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t c = 0; c < n; ++c) pos[c] = -1;
  int status = 0;
  for (int32_t i = 0; i < n && status == 0; ++i) {
    diag[i] = -1;
    for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
      pos[col[q]] = q;
      if (col[q] == i) diag[i] = q;
    }
    if (diag[i] < 0) { status = -(i + 1); break; }
    for (int64_t q = row_ptr[i]; q < row_ptr[i + 1] && col[q] < i; ++q) {
      int32_t j = col[q];
      double Lij[9];
      if (right_divide_bs(bs, lu + bb * q, lu + bb * diag[j], Lij)) { status = -(j + 1); break; }
      memcpy(lu + bb * q, Lij, bb * sizeof(double));
      /* W_ik -= L_ij U_jk for every k > j present in both rows i and j */
      for (int64_t t = row_ptr[j]; t < row_ptr[j + 1]; ++t) {
        int32_t k = col[t];
        if (k <= j || pos[k] < 0) continue;
        double* W = lu + bb * pos[k];
        const double* Ujk = lu + bb * t;
        for (int a = 0; a < bs; ++a)
          for (int c = 0; c < bs; ++c) {
            double s = 0.0;
            for (int b = 0; b < bs; ++b) s = s + Lij[bs * a + b] * Ujk[bs * b + c];
            W[bs * a + c] = W[bs * a + c] - s;
          }
      }
    }
    for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) pos[col[q]] = -1;
    if (status == 0) {
      /* the pivot block of row i must be invertible for later rows */
      double probe[9], eye[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      for (int a = 0; a < bs; ++a) eye[bs * a + a] = 1.0;
      if (right_divide_bs(bs, eye, lu + bb * diag[i], probe)) status = -(i + 1);
    }
  }
  free(pos);
  free(diag);
  return status;
}

/*
 * Level of every row in the lower-triangular DAG: 0 without a strictly-lower
 * block, else one more than the deepest strictly-lower neighbour (the fixed
 * point that Algorithm 5 reaches). Returns the number of levels.
 */
int32_t oracle_levels_lower(int32_t n, const int32_t* row_ptr, const int32_t* col, int32_t* lev) {
  int32_t nlev = 0;
  for (int32_t i = 0; i < n; ++i) {
    int32_t l = 0;
    for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q)
      if (col[q] < i && lev[col[q]] + 1 > l) l = lev[col[q]] + 1;
    lev[i] = l;
    if (l + 1 > nlev) nlev = l + 1;
  }
  return nlev;
}

/* Same on the upper-triangular DAG, solved from the last row backwards. */
int32_t oracle_levels_upper(int32_t n, const int32_t* row_ptr, const int32_t* col, int32_t* lev) {
  int32_t nlev = 0;
  for (int32_t i = n - 1; i >= 0; --i) {
    int32_t l = 0;
    for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q)
      if (col[q] > i && lev[col[q]] + 1 > l) l = lev[col[q]] + 1;
    lev[i] = l;
    if (l + 1 > nlev) nlev = l + 1;
  }
  return nlev;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 7 with the ILDU0 post-processing (Section 4.3)                  */
/* ------------------------------------------------------------------------ */

/*
 * bs x bs inverse by Gauss-Jordan elimination with partial pivoting on the
 * augmented matrix [M | I]. For each column c in turn: the row at or below
 * c with the largest |entry| in column c (the first of equals) is swapped
 * into row c; row c is multiplied by the reciprocal of its pivot; every
 * other row r with a nonzero entry m in column c has m times row c
 * subtracted from it. The right half is then M^-1. Returns 0, or -1 for a
 * zero or non-finite pivot or a non-finite entry of the result.
 */
static int inverse_gj_bs(int bs, const double* M, double* X) {
  double a[3][6];
  for (int r = 0; r < bs; ++r)
    for (int c = 0; c < 2 * bs; ++c) a[r][c] = c < bs ? M[bs * r + c] : (c - bs == r ? 1.0 : 0.0);
  for (int c = 0; c < bs; ++c) {
    int piv = c;
    for (int r = c + 1; r < bs; ++r)
      if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
    if (!(fabs(a[piv][c]) > 0.0) || !isfinite(a[piv][c])) return -1;
    if (piv != c)
      for (int q = 0; q < 2 * bs; ++q) {
        double t = a[c][q];
        a[c][q] = a[piv][q];
        a[piv][q] = t;
      }
    double recip = 1.0 / a[c][c];
    for (int q = 0; q < 2 * bs; ++q) a[c][q] = a[c][q] * recip;
    for (int r = 0; r < bs; ++r) {
      if (r == c || a[r][c] == 0.0) continue;
      double m = a[r][c];
      for (int q = 0; q < 2 * bs; ++q) a[r][q] = a[r][q] - m * a[c][q];
    }
  }
  for (int r = 0; r < bs; ++r)
    for (int c = 0; c < bs; ++c) {
      X[bs * r + c] = a[r][bs + c];
      if (!isfinite(X[bs * r + c])) return -1;
    }
  return 0;
}

/* Exported for the pins of the inverse on its own. */
int oracle_inverse_gj(int bs, const double* M, double* X) { return inverse_gj_bs(bs, M, X); }

/* C = A B for bs x bs blocks: each entry sums k = 0..bs-1 in order, from 0, without FMA. */
static void block_product(int bs, const double* A, const double* B, double* C) {
  for (int a = 0; a < bs; ++a)
    for (int c = 0; c < bs; ++c) {
      double s = 0.0;
      for (int k = 0; k < bs; ++k) s = s + A[bs * a + k] * B[bs * k + c];
      C[bs * a + c] = s;
    }
}

/*
 * Block ILU0 followed by the ILDU0 post-processing (Algorithm 7; Section
 * 4.3), the factors the fused apply uses, on the dropped matrix's pattern.
 * Row by row (ascending) with a working row W_i* = A_i* (U <- A):
 *   for each strictly-lower block j of row i, ascending:
 *     L_ij = W_ij inv_D_j                  (U[i,j] / U[j,j] in block form)
 *     W_ik = W_ik - L_ij U_jk              for every k > j present in rows i and j
 *   inv_D_i = W_ii^-1                      (Gauss-Jordan, above)
 * and afterwards, for every strictly-upper block of row i,
 *   U~_ik = inv_D_i U_ik                   (U = D U~, unit block diagonal).
 * Rows of different subdomains share no block (Section 3.2), so the
 * subdomains part_ptr[p] .. part_ptr[p+1] are factored independently.
 * f receives L at strictly-lower positions, U~ at strictly-upper positions
 * and zero on the diagonal; inv_d (bs*bs per row) receives inv_D. Returns 0,
 * or -(row+1) for the first subdomain's failing pivot block in row order.
 */
int oracle_ildu0(int32_t n, int bs, const int32_t* row_ptr, const int32_t* col, const double* val,
                 int32_t nparts, const int32_t* part_ptr, double* f, double* inv_d) {
  const int bb = bs * bs;
  int32_t* fail = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nparts > 0 ? nparts : 1));
  int32_t p;
#pragma omp parallel for schedule(dynamic, 1)
  for (p = 0; p < nparts; ++p) {
    const int32_t r0 = part_ptr[p], r1 = part_ptr[p + 1];
    const int64_t q0 = row_ptr[r0], q1 = row_ptr[r1];
    double* W = (double*)malloc(sizeof(double) * (size_t)bb * (size_t)(q1 > q0 ? q1 - q0 : 1));
    int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(r1 > r0 ? r1 - r0 : 1));
    fail[p] = -1;
    memcpy(W, val + bb * q0, sizeof(double) * (size_t)bb * (size_t)(q1 - q0));
    for (int32_t c = r0; c < r1; ++c) pos[c - r0] = -1;
    for (int32_t i = r0; i < r1 && fail[p] < 0; ++i) {
      int64_t d = -1;
      for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
        pos[col[q] - r0] = q;
        if (col[q] == i) d = q;
      }
      if (d < 0) { fail[p] = i; break; }
      for (int64_t q = row_ptr[i]; q < row_ptr[i + 1] && col[q] < i; ++q) {
        const int32_t j = col[q];
        double Lij[9], prod[9];
        block_product(bs, W + bb * (q - q0), inv_d + bb * (int64_t)j, Lij);
        memcpy(W + bb * (q - q0), Lij, sizeof(double) * bb);
        for (int64_t t = row_ptr[j]; t < row_ptr[j + 1]; ++t) {
          const int32_t k = col[t];
          if (k <= j || pos[k - r0] < 0) continue;
          block_product(bs, Lij, W + bb * (t - q0), prod);
          double* Wik = W + bb * (pos[k - r0] - q0);
          for (int e = 0; e < bb; ++e) Wik[e] = Wik[e] - prod[e];
        }
      }
      if (inverse_gj_bs(bs, W + bb * (d - q0), inv_d + bb * (int64_t)i)) fail[p] = i;
      for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) pos[col[q] - r0] = -1;
    }
    if (fail[p] < 0)
      for (int32_t i = r0; i < r1; ++i)
        for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
          double* dst = f + bb * q;
          if (col[q] < i)
            memcpy(dst, W + bb * (q - q0), sizeof(double) * bb);
          else if (col[q] > i)
            block_product(bs, inv_d + bb * (int64_t)i, W + bb * (q - q0), dst);
          else
            for (int e = 0; e < bb; ++e) dst[e] = 0.0;
        }
    free(W);
    free(pos);
  }
  int status = 0;
  for (int32_t q = 0; q < nparts && status == 0; ++q)
    if (fail[q] >= 0) status = -(fail[q] + 1);
  free(fail);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Preconditioner apply, SpMV, dot                                           */
/* ------------------------------------------------------------------------ */

/*
 * z = U^-1 L^-1 r by plain sequential substitution over all rows (Section
 * 4.2.2 computes the same result level by level). L has a unit block
 * diagonal; each U diagonal block is applied through a bs x bs solve. Within
 * a row, blocks are taken in ascending column order and, per output entry,
 * block entries c = 0..bs-1 with a fused multiply-add.
 */
int oracle_apply(int32_t n, int bs, const int32_t* row_ptr, const int32_t* col, const double* lu,
                 const double* r, double* z) {
  const int bb = bs * bs;
  double* y = (double*)malloc(sizeof(double) * bs * (size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i < n; ++i)
    for (int a = 0; a < bs; ++a) {
      double acc = r[bs * (int64_t)i + a];
      for (int64_t q = row_ptr[i]; q < row_ptr[i + 1] && col[q] < i; ++q)
        for (int c = 0; c < bs; ++c) acc = fma(-lu[bb * q + bs * a + c], y[bs * (int64_t)col[q] + c], acc);
      y[bs * (int64_t)i + a] = acc;
    }
  int status = 0;
  for (int32_t i = n - 1; i >= 0; --i) {
    double w[3];
    int64_t d = -1;
    for (int a = 0; a < bs; ++a) {
      double acc = y[bs * (int64_t)i + a];
      for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
        if (col[q] == i) d = q;
        if (col[q] <= i) continue;
        for (int c = 0; c < bs; ++c) acc = fma(-lu[bb * q + bs * a + c], z[bs * (int64_t)col[q] + c], acc);
      }
      w[a] = acc;
    }
    if (d < 0 || solve_bs(bs, lu + bb * d, w, z + bs * (int64_t)i)) status = -(i + 1);
  }
  free(y);
  return status;
}

/*
 * z = U~^-1 D^-1 L^-1 r with the ILDU0 factors of oracle_ildu0 (Section
 * 4.3; the fused kernel of Section 4.4 computes the same rows level by
 * level, Algorithm 6), by plain sequential substitution:
 *   y_i = r_i - sum_j L_ij y_j        for i ascending (strictly-lower j)
 *   w_i = inv_D_i y_i
 *   z_i = w_i - sum_k U~_ik z_k       for i descending (strictly-upper k)
 * Per output entry a, the sums take blocks in ascending column order and
 * block entries c = 0..bs-1, each with a fused multiply-add; w_i[a] =
 * inv_D[a][0] y_i[0], then fma(inv_D[a][c], y_i[c], .) for c = 1..bs-1. The
 * factors couple no two subdomains (Section 3.2), so each subdomain range
 * part_ptr[p] .. part_ptr[p+1] is substituted on its own.
 */
void oracle_apply_ildu0(int32_t n, int bs, const int32_t* row_ptr, const int32_t* col, const double* f,
                        const double* inv_d, int32_t nparts, const int32_t* part_ptr, const double* r,
                        double* z) {
  const int bb = bs * bs;
  (void)n;
  int32_t p;
#pragma omp parallel for schedule(dynamic, 1)
  for (p = 0; p < nparts; ++p) {
    const int32_t r0 = part_ptr[p], r1 = part_ptr[p + 1];
    for (int32_t i = r0; i < r1; ++i) {
      double y[3];
      for (int a = 0; a < bs; ++a) {
        double acc = r[bs * (int64_t)i + a];
        for (int64_t q = row_ptr[i]; q < row_ptr[i + 1] && col[q] < i; ++q)
          for (int c = 0; c < bs; ++c) acc = fma(-f[bb * q + bs * a + c], z[bs * (int64_t)col[q] + c], acc);
        y[a] = acc;
      }
      /* L results are kept in z until the backward sweep overwrites them */
      for (int a = 0; a < bs; ++a) z[bs * (int64_t)i + a] = y[a];
    }
    for (int32_t i = r1 - 1; i >= r0; --i) {
      const double* D = inv_d + bb * (int64_t)i;
      const double* y = z + bs * (int64_t)i;
      double w[3];
      for (int a = 0; a < bs; ++a) {
        double acc = D[bs * a] * y[0];
        for (int c = 1; c < bs; ++c) acc = fma(D[bs * a + c], y[c], acc);
        w[a] = acc;
      }
      for (int a = 0; a < bs; ++a) {
        double acc = w[a];
        for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
          if (col[q] <= i) continue;
          for (int c = 0; c < bs; ++c) acc = fma(-f[bb * q + bs * a + c], z[bs * (int64_t)col[q] + c], acc);
        }
        w[a] = acc;
      }
      for (int a = 0; a < bs; ++a) z[bs * (int64_t)i + a] = w[a];
    }
  }
}

/* y = A x: per scalar row, blocks in ascending column order, c = 0..bs-1, FMA from 0. */
void oracle_spmv(int32_t n, int bs, const int32_t* row_ptr, const int32_t* col, const double* val,
                 const double* x, double* y) {
  const int bb = bs * bs;
  int32_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < n; ++i)
    for (int a = 0; a < bs; ++a) {
      double acc = 0.0;
      for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q)
        for (int c = 0; c < bs; ++c) acc = fma(val[bb * q + bs * a + c], x[bs * (int64_t)col[q] + c], acc);
      y[bs * (int64_t)i + a] = acc;
    }
}

/* Block rows per tile of the fixed dot order. */
#define DOT_TILE 256

/* In place pairwise (halving) sum of s[0..m), m a power of two: s[i] += s[i+h]. */
static double halving_sum(double* s, int64_t m) {
  for (int64_t h = m / 2; h >= 1; h /= 2)
    for (int64_t i = 0; i < h; ++i) s[i] = s[i] + s[i + h];
  return s[0];
}

/*
 * x . y over n block rows (bs*n scalars) in one fixed order:
 *  1. per block row: q_i = x0 * y0, then q_i = fma(xc, yc, q_i) for c = 1..bs-1
 *     (for bs = 3: fma(x2, y2, fma(x1, y1, x0 * y0)));
 *  2. per tile of 256 block rows (missing rows count as 0): halving sum;
 *  3. over the tile sums, padded with zeros to a power of two: halving sum.
 */
double oracle_dot(int32_t n, int bs, const double* x, const double* y) {
  int64_t ntiles = (n + DOT_TILE - 1) / DOT_TILE;
  if (ntiles == 0) return 0.0;
  int64_t m = 1;
  while (m < ntiles) m *= 2;
  double* tile = (double*)calloc((size_t)m, sizeof(double));
  int64_t t;
#pragma omp parallel for schedule(static)
  for (t = 0; t < ntiles; ++t) {
    double q[DOT_TILE];
    for (int r = 0; r < DOT_TILE; ++r) {
      int64_t i = t * DOT_TILE + r;
      q[r] = 0.0;
      if (i < n) {
        q[r] = x[bs * i] * y[bs * i];
        for (int c = 1; c < bs; ++c) q[r] = fma(x[bs * i + c], y[bs * i + c], q[r]);
      }
    }
    tile[t] = halving_sum(q, DOT_TILE);
  }
  double s = halving_sum(tile, m);
  free(tile);
  return s;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: preconditioned BiCGSTAB                                      */
/* ------------------------------------------------------------------------ */

enum {
  ORC_OK = 0,
  ORC_BREAKDOWN = 5,
  ORC_NOT_CONVERGED = 6,
  ORC_ZERO_PIVOT = 2,
};

typedef struct {
  int32_t status, iterations, restarts, pad;
  double rel_res_recurrence, rel_res_true;
} oracle_info;

static double rel_of(double rr, double bb) { return sqrt(rr) / sqrt(bb); }

/*
 * The preconditioner M = LU of a solve, in one of two forms:
 *   form 0: lu from oracle_ilu0, applied by oracle_apply (ILU0 form);
 *   form 1: f and inv_d from oracle_ildu0, applied by oracle_apply_ildu0
 *           over the subdomains part_ptr[0..nparts] (ILDU0 form, Section 4.3).
 * Both forms are M^-1 of the same M in exact arithmetic.
 */
typedef struct {
  int32_t form, nparts;
  const int32_t* part_ptr;
  const int32_t* row_ptr;
  const int32_t* col;
  const double* lu;
  const double* f;
  const double* inv_d;
} oracle_precond;

static int precond_apply(int32_t n, int bs, const oracle_precond* M, const double* r, double* z) {
  if (M->form == 0) return oracle_apply(n, bs, M->row_ptr, M->col, M->lu, r, z);
  oracle_apply_ildu0(n, bs, M->row_ptr, M->col, M->f, M->inv_d, M->nparts, M->part_ptr, r, z);
  return 0;
}

/*
 * Algorithm 1 read as right preconditioning (K1 = I, K2 = M): solve A x = b.
 * A is the full reordered matrix. x0 is the initial guess (NULL: x0 = 0,
 * the solver runs' reading). All vectors are in the reordered numbering.
 *   r = b - A x0, r^ = r, rho = r^ . r, p = r
 *   per iteration j: p^ = M^-1 p, v = A p^, alpha = rho / (r^ . v),
 *     s = r - alpha v, s^ = M^-1 s, t = A s^, omega = (t . s) / (t . t),
 *     x = x + alpha p^ + omega s^, r = s - omega t,
 *     stop if ||r|| / ||b|| < rtol (iterations = j + 1),
 *     rho' = r^ . r, beta = (alpha / omega)(rho' / rho), p = r + beta (p - omega v).
 * After the recurrence converges, the true residual b - A x is formed; if it
 * misses rtol, the iteration restarts once from it (r = r^ = p = b - A x,
 * rho = r^ . r), the iteration count carrying on. hist (optional, maxit + 1
 * entries) receives ||r_j|| / ||b|| with hist[0] = ||r_0|| / ||b||.
 */
static int bicgstab_core(int32_t n, int bs, const int32_t* arp, const int32_t* acol, const double* aval,
                         const oracle_precond* M, const double* b, const double* x0, double* x, int32_t maxit,
                         double rtol, oracle_info* info, double* hist) {
  size_t m = bs * (size_t)(n > 0 ? n : 1);
  double *r = calloc(m, 8), *rh = calloc(m, 8), *p = calloc(m, 8), *v = calloc(m, 8);
  double *s = calloc(m, 8), *t = calloc(m, 8), *ph = calloc(m, 8), *sh = calloc(m, 8);
  int64_t len = bs * (int64_t)n, e;
  memset(info, 0, sizeof *info);
  for (e = 0; e < len; ++e) x[e] = 0.0;
  double bb = oracle_dot(n, bs, b, b);
  int status = ORC_NOT_CONVERGED;
  if (!(bb > 0.0)) {
    status = ORC_OK; /* b = 0: x = 0 is exact */
    goto done;
  }
  if (x0) {
    for (e = 0; e < len; ++e) x[e] = x0[e];
    oracle_spmv(n, bs, arp, acol, aval, x, t);
#pragma omp parallel for schedule(static)
    for (e = 0; e < len; ++e) r[e] = b[e] - t[e];
  } else {
    for (e = 0; e < len; ++e) r[e] = b[e];
  }
  if (hist) hist[0] = rel_of(oracle_dot(n, bs, r, r), bb);
  int j = 0;
  for (int restart = 0; restart < 2; ++restart) {
#pragma omp parallel for schedule(static)
    for (e = 0; e < len; ++e) rh[e] = r[e], p[e] = r[e];
    double rho = oracle_dot(n, bs, rh, r);
    int converged = 0;
    for (; j < maxit; ++j) {
      if (precond_apply(n, bs, M, p, ph)) { status = ORC_ZERO_PIVOT; goto done; }
      oracle_spmv(n, bs, arp, acol, aval, ph, v);
      double rv = oracle_dot(n, bs, rh, v);
      if (rv == 0.0 || !isfinite(rv)) { status = ORC_BREAKDOWN; goto done; }
      double alpha = rho / rv;
#pragma omp parallel for schedule(static)
      for (e = 0; e < len; ++e) s[e] = fma(-alpha, v[e], r[e]);
      if (precond_apply(n, bs, M, s, sh)) { status = ORC_ZERO_PIVOT; goto done; }
      oracle_spmv(n, bs, arp, acol, aval, sh, t);
      double ts = oracle_dot(n, bs, t, s);
      double tt = oracle_dot(n, bs, t, t);
      double omega = tt == 0.0 ? 0.0 : ts / tt;
#pragma omp parallel for schedule(static)
      for (e = 0; e < len; ++e) {
        x[e] = fma(omega, sh[e], fma(alpha, ph[e], x[e]));
        r[e] = fma(-omega, t[e], s[e]);
      }
      double rr = oracle_dot(n, bs, r, r);
      double rel = rel_of(rr, bb);
      info->rel_res_recurrence = rel;
      if (hist) hist[j + 1] = rel;
      if (!isfinite(rel)) { status = ORC_BREAKDOWN; goto done; }
      if (rel < rtol) { ++j; converged = 1; break; }
      double rho_new = oracle_dot(n, bs, rh, r);
      if (rho_new == 0.0 || omega == 0.0 || !isfinite(rho_new)) { status = ORC_BREAKDOWN; goto done; }
      double beta = (alpha / omega) * (rho_new / rho);
#pragma omp parallel for schedule(static)
      for (e = 0; e < len; ++e) p[e] = fma(beta, fma(-omega, v[e], p[e]), r[e]);
      rho = rho_new;
    }
    info->iterations = j;
    if (!converged) { status = ORC_NOT_CONVERGED; goto done; }
    /* true residual r = b - A x */
    oracle_spmv(n, bs, arp, acol, aval, x, t);
#pragma omp parallel for schedule(static)
    for (e = 0; e < len; ++e) r[e] = b[e] - t[e];
    double rel_true = rel_of(oracle_dot(n, bs, r, r), bb);
    info->rel_res_true = rel_true;
    if (rel_true < rtol) { status = ORC_OK; goto done; }
    if (restart == 0) info->restarts = 1;
  }
  status = ORC_NOT_CONVERGED;
done:
  info->status = status;
  free(r); free(rh); free(p); free(v); free(s); free(t); free(ph); free(sh);
  return status;
}

/* Algorithm 1 with the ILU0-form preconditioner (lu of oracle_ilu0), x0 = 0. */
int oracle_bicgstab(int32_t n, int bs, const int32_t* arp, const int32_t* acol, const double* aval,
                    const int32_t* lrp, const int32_t* lcol, const double* lu, const double* b,
                    double* x, int32_t maxit, double rtol, oracle_info* info, double* hist) {
  oracle_precond M = {0, 0, NULL, lrp, lcol, lu, NULL, NULL};
  return bicgstab_core(n, bs, arp, acol, aval, &M, b, NULL, x, maxit, rtol, info, hist);
}

/*
 * Algorithm 1 with either preconditioner form (oracle_precond above) and an
 * initial guess x0 (NULL: zero).
 */
int oracle_bicgstab_general(int32_t n, int bs, const int32_t* arp, const int32_t* acol, const double* aval,
                            const oracle_precond* M, const double* b, const double* x0, double* x,
                            int32_t maxit, double rtol, oracle_info* info, double* hist) {
  return bicgstab_core(n, bs, arp, acol, aval, M, b, x0, x, maxit, rtol, info, hist);
}

/* Threads of the OpenMP build (no effect without it). */
#ifdef _OPENMP
#include <omp.h>
void oracle_set_threads(int k) { omp_set_num_threads(k > 0 ? k : 1); }
int oracle_threads(void) { return omp_get_max_threads(); }
#else
void oracle_set_threads(int k) { (void)k; }
int oracle_threads(void) { return 1; }
#endif
