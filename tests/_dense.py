"""Small dense helpers for the CPU pins (tiny grids only).  Independent of oracle.c."""
import numpy as np


def bsr_to_dense(row_ptr, col, val, n):
    """Scalar dense matrix (3n x 3n) of a 3x3 BSR matrix."""
    D = np.zeros((3 * n, 3 * n))
    for i in range(n):
        for q in range(row_ptr[i], row_ptr[i + 1]):
            j = col[q]
            D[3 * i:3 * i + 3, 3 * j:3 * j + 3] = val[q]
    return D


def lu_to_dense(row_ptr, col, lu, n):
    """Split combined ILU0 storage into dense L (unit block diagonal) and U."""
    L = np.eye(3 * n)
    U = np.zeros((3 * n, 3 * n))
    for i in range(n):
        for q in range(row_ptr[i], row_ptr[i + 1]):
            j = col[q]
            if j < i:
                L[3 * i:3 * i + 3, 3 * j:3 * j + 3] = lu[q]
            else:
                U[3 * i:3 * i + 3, 3 * j:3 * j + 3] = lu[q]
    return L, U


def block_mask(row_ptr, col, n):
    M = np.zeros((n, n), bool)
    for i in range(n):
        for q in range(row_ptr[i], row_ptr[i + 1]):
            M[i, col[q]] = True
    return M


def dense_block_ilu0(Ad, mask):
    """Brute-force block ILU0 on a dense array of blocks (n, n, 3, 3) with a block mask.

    Textbook IKJ variant (Saad, Iterative Methods, Alg. 10.4), block form:
    for each row i, for each masked k < i: W_ik <- W_ik U_kk^-1, then
    W_ij -= W_ik U_kj for masked j > k.  Written with dense numpy blocks.
    """
    n = mask.shape[0]
    W = Ad.copy()
    for i in range(1, n):
        for k in range(i):
            if not mask[i, k]:
                continue
            W[i, k] = np.linalg.solve(W[k, k].T, W[i, k].T).T
            for j in range(k + 1, n):
                if mask[i, j] and mask[k, j]:
                    W[i, j] = W[i, j] - W[i, k] @ W[k, j]
    return W


def dense_scalar_ilu0(A, mask):
    """Scalar ILU0 (unit lower L, upper U) of a dense matrix restricted to a scalar mask."""
    n = A.shape[0]
    W = A.copy()
    for i in range(1, n):
        for k in range(i):
            if not mask[i, k]:
                continue
            W[i, k] = W[i, k] / W[k, k]
            js = np.nonzero(mask[i, k + 1:] & mask[k, k + 1:])[0] + k + 1
            W[i, js] -= W[i, k] * W[k, js]
    L = np.tril(W, -1) + np.eye(n)
    U = np.triu(W)
    return L, U


def blocks_dense(row_ptr, col, val, n):
    B = np.zeros((n, n, 3, 3))
    for i in range(n):
        for q in range(row_ptr[i], row_ptr[i + 1]):
            B[i, col[q]] = val[q]
    return B


def local_coords(grid, sub, perm, part_ptr):
    """Local (a, b, c) box coordinates of every reordered row."""
    nx, ny, _ = grid
    g = perm.astype(np.int64)
    i, j, k = g % nx, (g // nx) % ny, g // (nx * ny)
    return i % sub[0], j % sub[1], k % sub[2]
