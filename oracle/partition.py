"""Oracle for the quantities of the partition method itself (Sec. 2), by
their plain definitions, for small dense cases.  TEST INFRASTRUCTURE ONLY
(see the package docstring).

Partitioning (the reading used throughout for p not dividing N): partition i
(0-based) owns ``N // p`` block rows, the first ``N % p`` partitions one more;
for i < p-1 the LAST block row of partition i is the separator a^(i+1) (the
paper numbers partitions and separators from 1), the other rows form the local
block A^(i+1).  Partition p-1 has no separator (Eq. (parpart)).

For BABD systems (Eq. (parpart1) with c = 0) the separators are block row 0
(the boundary row), block row N, and the last block row of each of the first
p-1 partitions of block rows 1..N-1 (``babd_bounds``), so the reduced
system has p+1 block rows (Eq. (redmatr1)).

Every function here works on dense matrices with numpy; the reduced matrix is
the Schur complement of the local unknowns, T_p = A_ss - A_sI A_II^{-1} A_Is,
which is what the factorization A = F T G of Eqs. (parfact)-(parG) leaves in
the separator rows of T (Eq. (redmatr)), whatever local factorization
N^(i) S^(i) is used.
"""
from __future__ import annotations

import numpy as np


def btri_bounds(N: int, p: int):
    """Return ([(start, stop)] of local block rows, [separator block rows])."""
    if p < 1 or N < 2 * p - 1:
        raise ValueError("need 1 <= p and N >= 2p-1")
    base, extra = divmod(N, p)
    starts = []
    s = 0
    for i in range(p):
        cnt = base + (1 if i < extra else 0)
        starts.append((s, s + cnt))
        s += cnt
    local, seps = [], []
    for i, (a, b) in enumerate(starts):
        if i < p - 1:
            local.append((a, b - 1))
            seps.append(b - 1)
        else:
            local.append((a, b))
    return local, seps


def babd_bounds(N: int, p: int):
    """BABD partitioning of block rows 0..N: separators 0 and N plus the last
    row of each of the first p-1 partitions of rows 1..N-1 (split as in
    ``btri_bounds`` with N-1 rows and p partitions, whose separators are then
    shifted by one).  Returns ([(start, stop)] local rows, [separators])."""
    if N == 1:
        if p != 1:
            raise ValueError("N = 1 allows p = 1 only")
        return [(1, 1)], [0, 1]
    if p < 1 or N - 1 < p:
        raise ValueError("need 1 <= p <= N-1")
    M = N - 1                      # rows 1..N-1
    base, extra = divmod(M, p)
    local, seps = [], [0]
    s = 1
    for i in range(p):
        cnt = base + (1 if i < extra else 0)
        if i < p - 1:
            local.append((s, s + cnt - 1))
            seps.append(s + cnt - 1)
        else:
            local.append((s, s + cnt))
        s += cnt
    seps.append(N)
    return local, seps


def _rows(blocks, m):
    idx = []
    for j in blocks:
        idx.extend(range(j * m, (j + 1) * m))
    return np.array(idx, dtype=np.int64)


def schur_reduced(A: np.ndarray, f: np.ndarray, m: int, local, seps):
    """Reduced matrix and right-hand side by the Schur-complement definition:
    T = A_ss - A_sI A_II^{-1} A_Is,  g = f_s - A_sI A_II^{-1} f_I."""
    I = _rows([j for a, b in local for j in range(a, b)], m)
    s = _rows(seps, m)
    f2 = f.reshape(A.shape[0], -1)
    AII = A[np.ix_(I, I)]
    if I.size:
        sol = np.linalg.solve(AII, np.concatenate([A[np.ix_(I, s)], f2[I]], axis=1))
        T = A[np.ix_(s, s)] - A[np.ix_(s, I)] @ sol[:, :s.size]
        g = f2[s] - A[np.ix_(s, I)] @ sol[:, s.size:]
    else:
        T = A[np.ix_(s, s)].copy()
        g = f2[s].copy()
    return T, g


def btri_reduced_blocks(A, f, m, N, p):
    """(alpha, beta, gamma, g) of Eq. (redmatr) for a block tridiagonal A:
    alpha[s] = T[s, s], beta[s] = T[s, s-1] (s >= 1), gamma[s] = T[s, s+1]
    (s <= p-3), g[s] = reduced right-hand side; s = 0..p-2."""
    local, seps = btri_bounds(N, p)
    T, g = schur_reduced(A, f, m, local, seps)
    q = len(seps)
    blk = lambda r, c: T[r * m:(r + 1) * m, c * m:(c + 1) * m]
    alpha = np.stack([blk(s, s) for s in range(q)]) if q else np.zeros((0, m, m))
    beta = np.stack([blk(s, s - 1) if s >= 1 else np.zeros((m, m)) for s in range(q)]) if q else np.zeros((0, m, m))
    gamma = np.stack([blk(s, s + 1) if s + 1 < q else np.zeros((m, m)) for s in range(q)]) if q else np.zeros((0, m, m))
    nrhs = f.reshape(A.shape[0], -1).shape[1]
    return alpha, beta, gamma, g.reshape(q, m, nrhs), T


def unpivoted_lu(a: np.ndarray):
    """Doolittle LU without pivoting (unit lower L), plain loops."""
    n = a.shape[0]
    U = a.astype(np.float64).copy()
    L = np.eye(n)
    for k in range(n):
        for i in range(k + 1, n):
            L[i, k] = U[i, k] / U[k, k]
            U[i, k:] -= L[i, k] * U[k, k:]
            U[i, k] = 0.0
    return L, U


def partition_solve(B, D, C, F, p: int):
    """Solution of the block tridiagonal system by the partition method's
    definition, at sizes where A is not formed: the reduced matrix T_p and
    right-hand side g by the Schur complement onto the separators of
    ``btri_bounds`` (every local block A^(i) by a dense solve of its own),
    x_s = T_p^{-1} g by a banded LU with partial pivoting (T_p is block
    tridiagonal, Eq. (redmatr)), then x_I = A_II^{-1} (f_I - A_Is x_s).
    B, D, C: [N][m][m] (B[0], C[N-1] unused); F: [N m][nrhs]."""
    from scipy.linalg import solve_banded
    N, m = D.shape[0], D.shape[1]
    F2 = F.reshape(N * m, -1)
    nr = F2.shape[1]
    local, seps = btri_bounds(N, p)

    def dense(a, b):
        n = (b - a) * m
        A = np.zeros((n, n))
        for j in range(a, b):
            r = (j - a) * m
            A[r:r + m, r:r + m] = D[j]
            if j > a:
                A[r:r + m, r - m:r] = B[j]
            if j + 1 < b:
                A[r:r + m, r + m:r + 2 * m] = C[j]
        return A

    K = len(seps)
    al = np.array([D[sj].copy() for sj in seps]).reshape(K, m, m)
    be = np.zeros((K, m, m))
    ga = np.zeros((K, m, m))
    g = np.array([F2[sj * m:(sj + 1) * m].copy() for sj in seps]).reshape(K, m, nr)
    sol = []
    for i, (a, b) in enumerate(local):
        n = (b - a) * m
        if n == 0:
            sol.append(None)
            if 0 < i < K:               # adjacent separators couple directly
                be[i] = B[seps[i]]
                ga[i - 1] = C[seps[i - 1]]
            continue
        Ai = dense(a, b)
        cols = [F2[a * m:b * m]]
        if i > 0:                       # b0: coupling of the first local row to seps[i-1]
            b0 = np.zeros((n, m))
            b0[:m] = B[a]
            cols.append(b0)
        if i < K:                       # c1: coupling of the last local row to seps[i]
            c1 = np.zeros((n, m))
            c1[n - m:] = C[b - 1]
            cols.append(c1)
        Y = np.linalg.solve(Ai, np.concatenate(cols, axis=1))
        yf = Y[:, :nr]
        yb0 = Y[:, nr:nr + m] if i > 0 else None
        yc1 = Y[:, -m:] if i < K else None
        sol.append((yf, yb0, yc1))
        if i > 0:                       # row seps[i-1]: c0^T = C[seps[i-1]] on the first local row
            c0T = C[seps[i - 1]]
            al[i - 1] -= c0T @ yb0[:m]
            g[i - 1] -= c0T @ yf[:m]
            if i < K:
                ga[i - 1] -= c0T @ yc1[:m]
        if i < K:                       # row seps[i]: b1^T = B[seps[i]] on the last local row
            b1T = B[seps[i]]
            al[i] -= b1T @ yc1[n - m:]
            g[i] -= b1T @ yf[n - m:]
            if i > 0:
                be[i] -= b1T @ yb0[n - m:]
    x = np.zeros((N * m, nr))
    if K:
        q = K * m
        w = 2 * m - 1
        ab = np.zeros((2 * w + 1, q))
        for k in range(K):
            for r in range(m):
                row = k * m + r
                for blk, c0 in ((be[k], (k - 1) * m), (al[k], k * m), (ga[k], (k + 1) * m)):
                    if c0 < 0 or c0 >= q:
                        continue
                    for c in range(m):
                        ab[w + row - (c0 + c), c0 + c] = blk[r, c]
        xs = solve_banded((w, w), ab, g.reshape(q, nr)).reshape(K, m, nr)
        for k, sj in enumerate(seps):
            x[sj * m:(sj + 1) * m] = xs[k]
    for i, (a, b) in enumerate(local):
        if sol[i] is None:
            continue
        yf, yb0, yc1 = sol[i]
        xi = yf.copy()
        if i > 0:
            xi -= yb0 @ x[seps[i - 1] * m:(seps[i - 1] + 1) * m]
        if i < K:
            xi -= yc1 @ x[seps[i] * m:(seps[i] + 1) * m]
        x[a * m:b * m] = xi
    return x


def householder_qr(a: np.ndarray):
    """QR factorization by Householder reflections, plain loops: for each
    column k the reflector H_k = I - 2 u u^T / (u^T u), u = x - alpha e_1 with
    x the column's entries from the diagonal down and alpha = -sign(x_1) ||x||,
    annihilates the entries below the diagonal.  Returns (Q, R) with
    Q = H_0 H_1 ... H_{n-2} orthogonal and R upper triangular, Q R = a."""
    n = a.shape[0]
    R = a.astype(np.float64).copy()
    Q = np.eye(n)
    for k in range(n - 1):
        x = R[k:, k].copy()
        nrm = np.sqrt(np.dot(x, x))
        if nrm == 0.0:
            continue
        alpha = -nrm if x[0] >= 0.0 else nrm
        u = x.copy()
        u[0] -= alpha
        uu = np.dot(u, u)
        if uu == 0.0:
            continue
        for j in range(k, n):
            R[k:, j] -= (2.0 * np.dot(u, R[k:, j]) / uu) * u
        for i in range(n):
            Q[i, k:] -= (2.0 * np.dot(Q[i, k:], u) / uu) * u
        R[k + 1:, k] = 0.0
    return Q, R


def _parallel_factors(A, m, N, p, local_factor, n_solve, s_solve_right):
    """Eq. (parblock) for every partition with the local factorization
    A^(i) = N^(i) S^(i) given by local_factor; z = N^{-1} b0, y = N^{-1} c1
    (n_solve), w^T = c0^T S^{-1}, v^T = b1^T S^{-1} (s_solve_right),
    alpha1 = -w^T z, gamma = -w^T y, beta = -v^T z, alpha2 = a - v^T y and
    alpha = alpha2^(i) + alpha1^(i+1).  Returns (F, T, G, parts) in the
    ORIGINAL row/column order of A; ``parts`` lists per partition the dict of
    its blocks (N, S and the four vectors)."""
    n = A.shape[0]
    local, seps = btri_bounds(N, p)
    F = np.zeros((n, n))
    T = np.zeros((n, n))
    G = np.zeros((n, n))
    parts = []
    sep_rows = [_rows([s], m) for s in seps]
    for s_rows in sep_rows:
        F[np.ix_(s_rows, s_rows)] = np.eye(m)
        G[np.ix_(s_rows, s_rows)] = np.eye(m)
    alpha1 = [None] * p
    alpha2 = [None] * p
    for i, (a, b) in enumerate(local):
        I = _rows(range(a, b), m)
        Ai = A[np.ix_(I, I)]
        Nf, Sf = local_factor(Ai)
        F[np.ix_(I, I)] = Nf
        G[np.ix_(I, I)] = Sf
        T[np.ix_(I, I)] = np.eye(I.size)
        d = {"N": Nf, "S": Sf}
        if i > 0:                                   # left separator seps[i-1]
            sl = sep_rows[i - 1]
            b0 = A[np.ix_(I, sl)]
            c0T = A[np.ix_(sl, I)]
            z = n_solve(Nf, b0)
            wT = s_solve_right(Sf, c0T)
            G[np.ix_(I, sl)] = z
            F[np.ix_(sl, I)] = wT
            alpha1[i] = -wT @ z
            d.update(z=z, wT=wT, b0=b0, c0T=c0T)
        if i < p - 1:                               # right separator seps[i]
            sr = sep_rows[i]
            c1 = A[np.ix_(I, sr)]
            b1T = A[np.ix_(sr, I)]
            y = n_solve(Nf, c1)
            vT = s_solve_right(Sf, b1T)
            G[np.ix_(I, sr)] = y
            F[np.ix_(sr, I)] = vT
            alpha2[i] = A[np.ix_(sr, sr)] - vT @ y
            d.update(y=y, vT=vT, c1=c1, b1T=b1T)
        if 0 < i < p - 1:
            sl, sr = sep_rows[i - 1], sep_rows[i]
            T[np.ix_(sl, sr)] = -d["wT"] @ d["y"]          # gamma^(i), Eq. (parblock)
            T[np.ix_(sr, sl)] = -d["vT"] @ d["z"]          # beta^(i)
        parts.append(d)
    for s in range(len(seps)):
        T[np.ix_(sep_rows[s], sep_rows[s])] = alpha2[s] + alpha1[s + 1]
    return F, T, G, parts


def _upper_right_solve(S, rhsT):
    """X with X S = rhsT for upper triangular S (forward substitution)."""
    from scipy.linalg import solve_triangular
    return solve_triangular(S, rhsT.T, trans="T", lower=False).T


def parallel_factors_lu(A: np.ndarray, m: int, N: int, p: int):
    """The factors F, T, G of Eqs. (parF)-(parG) for the LU variant
    (N^(i) = L^(i), S^(i) = U^(i), Sec. 2): z = L^{-1} b0, y = L^{-1} c1,
    w^T = c0^T U^{-1}, v^T = b1^T U^{-1}.  ``parts[i]`` also carries the
    factors as "L" and "U"."""
    F, T, G, parts = _parallel_factors(A, m, N, p, unpivoted_lu, lambda L, b: np.linalg.solve(L, b),
                                       lambda U, cT: np.linalg.solve(U.T, cT.T).T)
    for d in parts:
        d["L"], d["U"] = d["N"], d["S"]
    return F, T, G, parts


def parallel_factors_qr(A: np.ndarray, m: int, N: int, p: int):
    """The factors F, T, G of Eqs. (parF)-(parG) for the QR variant
    (N^(i) = Q^(i), S^(i) = R^(i), Sec. 2): z = Q^T b0, y = Q^T c1 (Q
    orthogonal), w^T = c0^T R^{-1}, v^T = b1^T R^{-1}.  ``parts[i]`` also
    carries the factors as "Q" and "R"."""
    F, T, G, parts = _parallel_factors(A, m, N, p, householder_qr, lambda Q, b: Q.T @ b, _upper_right_solve)
    for d in parts:
        d["Q"], d["R"] = d["N"], d["S"]
    return F, T, G, parts


def babd_reduced_blocks(S, R, B0, B1, RHS, p):
    """Reduced BABD system of Eq. (redmatr1) with c = 0 (lower block bidiagonal
    plus corner) by the Schur-complement definition.  Returns
    (alpha [p+1,m,m], beta [p+1,m,m] with beta[0] = the corner block,
    g [p+1,m,nrhs], T)."""
    from gen import babd_dense   # matrix assembly only
    N, m = S.shape[0], S.shape[1]
    A = babd_dense(S, R, B0, B1)
    local, seps = babd_bounds(N, p)
    T, g = schur_reduced(A, RHS, m, local, seps)
    q = len(seps)
    blk = lambda r, c: T[r * m:(r + 1) * m, c * m:(c + 1) * m]
    alpha = np.stack([blk(s, s) for s in range(q)])
    beta = np.stack([blk(0, q - 1)] + [blk(s, s - 1) for s in range(1, q)])
    return alpha, beta, g.reshape(q, m, -1), T
