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
