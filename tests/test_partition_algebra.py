"""The partition method's own algebra (Sec. 2 and Sec. 3), checked on small
dense cases against plain definitions: A = F T G (Eq. (parfact)), the
separator sum rule alpha = alpha2^(i) + alpha1^(i+1) (Eq. (parblock)) against
the Schur complement, the sparsity claims of the LU variant, the size of the
reduced matrix (Eqs. (redmatr), (redmatr1)), invariance of x under p, and the
IVP recurrences (D), (redsys)-(recur) and (pups)."""
import numpy as np
import pytest

import gen
import oracle
from oracle import partition as P


@pytest.mark.parametrize("N,m,p", [(5, 1, 1), (11, 2, 2), (11, 2, 3), (13, 3, 5), (15, 2, 7), (9, 1, 4)])
def test_F_T_G_reconstructs_A(N, m, p):
    s = gen.btri_random(N, m, 1, seed_rep=N + p)
    A = gen.btri_dense(s.B, s.D, s.C)
    F, T, G, parts = P.parallel_factors_lu(A, m, N, p)
    assert np.abs(F @ T @ G - A).max() <= 1e-13 * np.abs(A).max()
    # separator rows of T are the Schur complement (alpha2 + alpha1 rule)
    al, be, ga, g, Tp = P.btri_reduced_blocks(A, s.F, m, N, p)
    local, seps = P.btri_bounds(N, p)
    for k, sidx in enumerate(seps):
        rows = slice(sidx * m, (sidx + 1) * m)
        assert np.allclose(T[rows, rows], al[k], atol=1e-13)
        if k >= 1:
            assert np.allclose(T[rows, seps[k - 1] * m:(seps[k - 1] + 1) * m], be[k], atol=1e-13)
        if k + 1 < len(seps):
            assert np.allclose(T[rows, seps[k + 1] * m:(seps[k + 1] + 1) * m], ga[k], atol=1e-13)


def test_lu_variant_sparsity():
    """y, v keep the sparsity of c1, b1 (last block row only); z, w are fill-in."""
    N, m, p = 17, 2, 3
    s = gen.btri_random(N, m, 1, seed_rep=5)
    A = gen.btri_dense(s.B, s.D, s.C)
    _, _, _, parts = P.parallel_factors_lu(A, m, N, p)
    mid = parts[1]
    k = mid["L"].shape[0]
    assert np.all(mid["y"][:k - m] == 0) and np.abs(mid["y"][k - m:]).max() > 0
    assert np.all(mid["vT"][:, :k - m] == 0) and np.abs(mid["vT"][:, k - m:]).max() > 0
    assert np.count_nonzero(np.abs(mid["z"]) > 1e-300) > 0.8 * mid["z"].size
    assert np.count_nonzero(np.abs(mid["wT"]) > 1e-300) > 0.8 * mid["wT"].size


@pytest.mark.parametrize("n,zero_col", [(1, False), (2, False), (5, False), (12, False), (6, True)])
def test_householder_qr(n, zero_col):
    """Q orthogonal, R upper triangular, Q R = a; R equals LAPACK's R
    (numpy.linalg.qr) up to the signs of its rows; a zero column is skipped."""
    rng = np.random.default_rng(n)
    a = rng.standard_normal((n, n))
    if zero_col:
        a[:, 2] = 0.0
    Q, R = P.householder_qr(a)
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= 4e-15 * n
    assert np.all(np.tril(R, -1) == 0)
    assert np.abs(Q @ R - a).max() <= 4e-15 * n * np.abs(a).max()
    assert np.allclose(np.abs(R), np.abs(np.linalg.qr(a, mode="r")), atol=1e-13)


@pytest.mark.parametrize("N,m,p", [(11, 2, 3), (13, 3, 5), (15, 2, 7), (9, 1, 4), (12, 4, 1)])
def test_qr_variant_F_T_G(N, m, p):
    """The QR variant (N^(i) = Q^(i), S^(i) = R^(i)) also gives A = F T G, on
    matrices with singular diagonal blocks (where every local block A^(i)
    spans at least two block rows, so that A^(i) stays nonsingular), and its
    separator rows of T are the same Schur complement as the LU variant's."""
    zf = 0.3 if N // p >= 3 else 0.0
    s = gen.btri_nondominant(N, m, 1, seed_rep=3 * N + m, zero_frac=zf)
    A = gen.btri_dense(s.B, s.D, s.C)
    F, T, G, parts = P.parallel_factors_qr(A, m, N, p)
    assert np.abs(F @ T @ G - A).max() <= 1e-12 * np.abs(A).max()
    for d in parts:
        k = d["Q"].shape[0]
        assert np.abs(d["Q"].T @ d["Q"] - np.eye(k)).max() <= 1e-14 * k
        assert np.all(np.tril(d["R"], -1) == 0)
    al, be, ga, g, Tp = P.btri_reduced_blocks(A, s.F, m, N, p)
    local, seps = P.btri_bounds(N, p)
    scale = np.abs(Tp).max() if Tp.size else 1.0
    for k, sidx in enumerate(seps):
        rows = slice(sidx * m, (sidx + 1) * m)
        assert np.abs(T[rows, rows] - al[k]).max() <= 1e-12 * scale
        if k >= 1:
            assert np.abs(T[rows, seps[k - 1] * m:(seps[k - 1] + 1) * m] - be[k]).max() <= 1e-12 * scale
        if k + 1 < len(seps):
            assert np.abs(T[rows, seps[k + 1] * m:(seps[k + 1] + 1) * m] - ga[k]).max() <= 1e-12 * scale


@pytest.mark.parametrize("N,m,p,nr", [(11, 2, 3, 1), (40, 3, 6, 2), (9, 1, 5, 1), (30, 4, 1, 3), (64, 2, 32, 1)])
def test_partition_solve_matches_dense(N, m, p, nr):
    """The partition method by its definition (Schur complement, banded
    reduced solve, local back substitution) gives the dense solution."""
    s = gen.btri_random(N, m, nr, seed_rep=N * p + m)
    A = gen.btri_dense(s.B, s.D, s.C)
    x = P.partition_solve(s.B, s.D, s.C, s.F, p)
    ref = np.linalg.solve(A, s.F.reshape(N * m, -1))
    assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max() * np.linalg.cond(A, 1)
    # its reduced system is the one of btri_reduced_blocks: x on the separators solves it
    al, be, ga, g, T = P.btri_reduced_blocks(A, s.F, m, N, p)
    _, seps = P.btri_bounds(N, p)
    if seps:
        xs = np.concatenate([x[j * m:(j + 1) * m] for j in seps])
        assert np.abs(T @ xs - g.reshape(len(seps) * m, -1)).max() <= 1e-12 * (np.abs(T).max() * np.abs(xs).max())


def test_qr_variant_sparsity():
    """QR variant: v^T keeps the sparsity of b1^T (last block column), y = Q^T c1
    is confined to the last two block rows (R has two block superdiagonals),
    z = Q^T b0 and w^T = c0^T R^{-1} are fill-in."""
    N, m, p = 17, 2, 3
    s = gen.btri_random(N, m, 1, seed_rep=5)
    A = gen.btri_dense(s.B, s.D, s.C)
    _, _, _, parts = P.parallel_factors_qr(A, m, N, p)
    mid = parts[1]
    k = mid["Q"].shape[0]
    assert np.all(mid["vT"][:, :k - m] == 0) and np.abs(mid["vT"][:, k - m:]).max() > 0
    assert np.all(mid["y"][:k - 2 * m] == 0) and np.abs(mid["y"][k - 2 * m:k - m]).max() > 0
    R = mid["R"]
    assert all(np.all(R[r * m:(r + 1) * m, (r + 3) * m:] == 0) for r in range(k // m))
    assert np.count_nonzero(np.abs(mid["z"]) > 1e-300) > 0.8 * mid["z"].size
    assert np.count_nonzero(np.abs(mid["wT"]) > 1e-300) > 0.8 * mid["wT"].size


@pytest.mark.parametrize("N", [40, 80, 400])
def test_reduced_size_depends_on_p_only(N):
    p, m = 6, 2
    s = gen.btri_random(N, m, 1, seed_rep=1)
    A = gen.btri_dense(s.B, s.D, s.C)
    al, *_ = P.btri_reduced_blocks(A, s.F, m, N, p)
    assert al.shape[0] == p - 1
    b = gen.babd_bvp(N, m, 1)
    al2, be2, g2, T2 = P.babd_reduced_blocks(b.S, b.R, b.B0, b.B1, b.RHS, p)
    assert al2.shape[0] == p + 1


@pytest.mark.parametrize("N,m", [(23, 2), (40, 3), (7, 1)])
def test_solution_invariant_under_p(N, m):
    """Solve the reduced system, then the local blocks: same x for every p."""
    s = gen.btri_random(N, m, 2, seed_rep=N)
    A = gen.btri_dense(s.B, s.D, s.C)
    xref = oracle.btri_solve(s.B, s.D, s.C, s.F)
    for p in range(1, (N + 1) // 2 + 1):
        local, seps = P.btri_bounds(N, p)
        T, g = P.schur_reduced(A, s.F, m, local, seps)
        x = np.zeros_like(s.F)
        sr = np.concatenate([np.arange(q * m, (q + 1) * m) for q in seps]) if seps else np.zeros(0, int)
        if seps:
            x[sr] = np.linalg.solve(T, g)
        I = np.setdiff1d(np.arange(N * m), sr)
        x[I] = np.linalg.solve(A[np.ix_(I, I)], s.F[I] - A[np.ix_(I, sr)] @ x[sr])
        assert oracle.rel_err(x, xref) <= 1e-13, p


def test_babd_reduced_is_lower_bidiagonal_with_corner():
    """With c = 0 the reduced matrix keeps the form of A: alpha^(i) = a^(i),
    gamma = 0, one subdiagonal block and the corner (Eq. (redmatr1))."""
    N, m, p = 30, 3, 4
    b = gen.babd_bvp(N, m, 1, seed_rep=2)
    al, be, g, T = P.babd_reduced_blocks(b.S, b.R, b.B0, b.B1, b.RHS, p)
    local, seps = P.babd_bounds(N, p)
    q = len(seps)
    for r in range(q):
        for c in range(q):
            blk = T[r * m:(r + 1) * m, c * m:(c + 1) * m]
            allowed = (r == c) or (c == r - 1) or (r == 0 and c == q - 1)
            if not allowed:
                assert np.all(blk == 0)
    assert np.array_equal(al[0], b.B0)
    assert np.allclose(be[0], b.B1)
    for k in range(1, q):
        assert np.array_equal(al[k], b.R[seps[k] - 1])


def test_ivp_parallel_recurrences():
    """Sec. 3 with the trapezoidal rule as the local method: the global
    system (My) is solved by the parallel solves (D), the reduced system
    (redsys) as the recurrence (recur), and the parallel updates (pups)."""
    Nglob, m, p = 48, 4, 4
    b = gen.babd_bvp(Nglob, m, 1, seed_rep=9)
    y0 = b.RHS[:m, 0]
    r = b.RHS[m:, 0].reshape(Nglob, m)
    n_loc = Nglob // p
    Z, W = [], []
    for i in range(p):
        # local problem on [tau_{i-1}, tau_i]: M_i y_i = v_i y_0i + g_i with
        # M_i lower block bidiagonal (R on the diagonal, S below), v_i = -S_first
        js = range(i * n_loc, (i + 1) * n_loc)
        Mi = np.zeros((n_loc * m, n_loc * m))
        for a, j in enumerate(js):
            Mi[a * m:(a + 1) * m, a * m:(a + 1) * m] = b.R[j]
            if a > 0:
                Mi[a * m:(a + 1) * m, (a - 1) * m:a * m] = b.S[j]
        vi = np.zeros((n_loc * m, m))
        vi[:m] = -b.S[js[0]]
        gi = np.concatenate([r[j] for j in js])
        Z.append(np.linalg.solve(Mi, gi))          # (D)
        W.append(np.linalg.solve(Mi, vi))          # (Wi)
    y0i = [y0]
    for i in range(p - 1):                          # (recur)
        y0i.append(Z[i][-m:] + W[i][-m:] @ y0i[i])
    Y = np.concatenate([y0] + [Z[i] + W[i] @ y0i[i] for i in range(p)])   # (pups)
    ref = oracle.babd_solve(b.S, b.R, np.eye(m), np.zeros((m, m)), b.RHS)[:, 0]
    assert oracle.rel_err(Y, ref) <= 1e-13
