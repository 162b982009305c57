"""Seeded synthetic inputs shaped like the workloads of Amodio & Brugnano,
"Parallel Factorizations in Numerical Analysis" (Sec. 3: linear ODE-BVP / IVP
discretisations giving (block) tridiagonal and BABD systems).

This module builds problem data only: matrices, right-hand sides and exact
solutions.  It holds none of the solver arithmetic (no factorization, no
elimination), so both the oracle and the CUDA path can take their inputs from
it.  Every generator is deterministic in its seed; the default seeds are
``20091234 + 1000 * workload + rep`` (numpy PCG64).

Layouts (all row-major FP64):
* scalar tridiagonal: ``dl, d, du`` of length n (``dl[0] = du[n-1] = 0``),
  right-hand sides ``f`` of shape [n, nrhs];
* block tridiagonal: ``B, D, C`` of shape [N, m, m] (``B[0] = C[N-1] = 0``),
  ``F`` of shape [N*m, nrhs];
* BABD: ``S, R`` of shape [N, m, m], ``B0, B1`` of shape [m, m], ``RHS`` of
  shape [(N+1)*m, nrhs] with the boundary row first.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20091234


def rng_for(workload: int, rep: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + 1000 * workload + rep))


# ---------------------------------------------------------------- products --

def tri_matvec(dl, d, du, x):
    """A x for the tridiagonal A (x: [n] or [n, k])."""
    x = np.asarray(x, dtype=np.float64)
    y = d.reshape(-1, *([1] * (x.ndim - 1))) * x
    if x.shape[0] > 1:
        y[1:] += dl[1:].reshape(-1, *([1] * (x.ndim - 1))) * x[:-1]
        y[:-1] += du[:-1].reshape(-1, *([1] * (x.ndim - 1))) * x[1:]
    return y


def btri_matvec(B, D, C, X):
    """A X for the block tridiagonal A; X: [N*m, k]."""
    N, m = D.shape[0], D.shape[1]
    Xb = np.asarray(X, dtype=np.float64).reshape(N, m, -1)
    Y = np.einsum("jab,jbk->jak", D, Xb)
    if N > 1:
        Y[1:] += np.einsum("jab,jbk->jak", B[1:], Xb[:-1])
        Y[:-1] += np.einsum("jab,jbk->jak", C[:-1], Xb[1:])
    return Y.reshape(N * m, -1)


def babd_matvec(S, R, B0, B1, Y):
    """A Y for the BABD A; Y: [(N+1)*m, k]; result has the boundary row first."""
    N, m = S.shape[0], S.shape[1]
    Yb = np.asarray(Y, dtype=np.float64).reshape(N + 1, m, -1)
    out = np.empty_like(Yb)
    out[0] = B0 @ Yb[0] + B1 @ Yb[N]
    out[1:] = np.einsum("jab,jbk->jak", S, Yb[:-1]) + np.einsum("jab,jbk->jak", R, Yb[1:])
    return out.reshape((N + 1) * m, -1)


def btri_dense(B, D, C):
    N, m = D.shape[0], D.shape[1]
    A = np.zeros((N * m, N * m))
    for j in range(N):
        A[j * m:(j + 1) * m, j * m:(j + 1) * m] = D[j]
        if j > 0:
            A[j * m:(j + 1) * m, (j - 1) * m:j * m] = B[j]
        if j + 1 < N:
            A[j * m:(j + 1) * m, (j + 1) * m:(j + 2) * m] = C[j]
    return A


def babd_dense(S, R, B0, B1):
    N, m = S.shape[0], S.shape[1]
    A = np.zeros(((N + 1) * m, (N + 1) * m))
    A[:m, :m] = B0
    A[:m, N * m:] += B1
    for j in range(N):
        A[(j + 1) * m:(j + 2) * m, j * m:(j + 1) * m] = S[j]
        A[(j + 1) * m:(j + 2) * m, (j + 1) * m:(j + 2) * m] = R[j]
    return A


# ------------------------------------------------------- scalar tridiagonal --

@dataclass
class TriSystem:
    dl: np.ndarray
    d: np.ndarray
    du: np.ndarray
    f: np.ndarray          # [n, nrhs]
    xstar: np.ndarray      # [n, nrhs] (the vector f was made from)


def tri_sdd(n: int, nrhs: int = 1, seed_rep: int = 0, rng=None) -> TriSystem:
    """Strictly diagonally dominant tridiagonal system: d ~ U[4,6],
    dl, du ~ U[-1,1], x* ~ N(0,1), f = A x*."""
    rng = rng if rng is not None else rng_for(1, seed_rep)
    d = rng.uniform(4.0, 6.0, n)
    dl = rng.uniform(-1.0, 1.0, n)
    du = rng.uniform(-1.0, 1.0, n)
    dl[0] = 0.0
    du[n - 1] = 0.0
    xs = rng.standard_normal((n, nrhs))
    return TriSystem(dl, d, du, tri_matvec(dl, d, du, xs), xs)


def poisson(n: int):
    """The 1-D Poisson matrix tridiag(-1, 2, -1) of order n."""
    dl = -np.ones(n)
    du = -np.ones(n)
    dl[0] = 0.0
    du[n - 1] = 0.0
    return dl, 2.0 * np.ones(n), du


# -------------------------------------------------------- block tridiagonal --

@dataclass
class BtriSystem:
    B: np.ndarray
    D: np.ndarray
    C: np.ndarray
    F: np.ndarray          # [N*m, nrhs]
    Xstar: np.ndarray


def btri_random(N: int, m: int, nrhs: int = 1, seed_rep: int = 0, rng=None,
                diag_shift: float = 4.0) -> BtriSystem:
    """Block tridiagonal system: D_j = 4 I + G/sqrt(m), B_j, C_j = G/sqrt(m),
    G ~ N(0,1) (fresh per block), X* ~ N(0,1), F = A X*."""
    rng = rng if rng is not None else rng_for(2, seed_rep)
    s = 1.0 / math.sqrt(m)
    B = rng.standard_normal((N, m, m)) * s
    D = rng.standard_normal((N, m, m)) * s + diag_shift * np.eye(m)
    C = rng.standard_normal((N, m, m)) * s
    B[0] = 0.0
    C[N - 1] = 0.0
    Xs = rng.standard_normal((N * m, nrhs))
    return BtriSystem(B, D, C, btri_matvec(B, D, C, Xs), Xs)


def btri_nondominant(N: int, m: int, nrhs: int = 1, seed_rep: int = 0, zero_frac: float = 0.1,
                     rng=None) -> BtriSystem:
    """Block tridiagonal system that is not block diagonally dominant, with a
    fraction of exactly singular diagonal blocks: B_j, C_j, D_j = G/sqrt(m),
    G ~ N(0,1), and D_j = 0 for about zero_frac of the block rows (block LU
    without interchanges breaks down there).  X* ~ N(0,1), F = A X*."""
    rng = rng if rng is not None else rng_for(7, seed_rep)
    s = 1.0 / math.sqrt(m)
    B = rng.standard_normal((N, m, m)) * s
    D = rng.standard_normal((N, m, m)) * s
    C = rng.standard_normal((N, m, m)) * s
    D[rng.random(N) < zero_frac] = 0.0
    B[0] = 0.0
    C[N - 1] = 0.0
    Xs = rng.standard_normal((N * m, nrhs))
    return BtriSystem(B, D, C, btri_matvec(B, D, C, Xs), Xs)


# ------------------------------------------------------------- heat equation --

def heat_problem(n: int, nu: float = 0.5, seed_rep: int = 0, smooth: bool = False):
    """y' = L y + g0 + t g1 with L = nu/dx^2 tridiag(1, -2, 1) on n interior
    points of [0, 1] (Dirichlet, dx = 1/(n+1)).  Data: y0, g0, g1 ~ N(0,1), or
    (smooth) a few low Fourier modes with N(0,1) amplitudes (the setting where
    a coarse propagator resolves the solution and Parareal converges fast).
    Returns (dl, d, du, y0, g0, g1) with dl[0] = du[n-1] = 0."""
    dx = 1.0 / (n + 1)
    c = nu / (dx * dx)
    dl = np.full(n, c)
    du = np.full(n, c)
    d = np.full(n, -2.0 * c)
    dl[0] = 0.0
    du[-1] = 0.0
    rng = rng_for(10, seed_rep)
    if not smooth:
        return dl, d, du, rng.standard_normal(n), rng.standard_normal(n), rng.standard_normal(n)
    x = np.arange(1, n + 1) * dx
    modes = lambda: sum(rng.standard_normal() * np.sin(k * np.pi * x) for k in range(1, 5))
    return dl, d, du, modes(), modes(), modes()


# ----------------------------------------------------- circulant-like (cyclic) --

@dataclass
class CycSystem:
    """S_j y_j + R_j y_{(j+1) mod N} = r_j, j = 0..N-1."""
    S: np.ndarray
    R: np.ndarray
    RHS: np.ndarray
    Ystar: np.ndarray


def cyc_matvec(S, R, Y):
    N, m = S.shape[0], S.shape[1]
    Y3 = Y.reshape(N, m, -1)
    out = np.einsum("jab,jbc->jac", S, Y3) + np.einsum("jab,jbc->jac", R, np.roll(Y3, -1, axis=0))
    return out.reshape(N * m, -1)


def cyc_dense(S, R):
    N, m = S.shape[0], S.shape[1]
    A = np.zeros((N * m, N * m))
    for j in range(N):
        A[j * m:(j + 1) * m, j * m:(j + 1) * m] += S[j]
        k = (j + 1) % N
        A[j * m:(j + 1) * m, k * m:(k + 1) * m] += R[j]
    return A


def cyc_random(N: int, m: int, nrhs: int = 1, seed_rep: int = 0, rng=None) -> CycSystem:
    """A cyclic block bidiagonal system with R_j = 3 I + G/sqrt(m), S_j = G/sqrt(m)."""
    rng = rng if rng is not None else rng_for(8, seed_rep)
    s = 1.0 / math.sqrt(m)
    S = rng.standard_normal((N, m, m)) * s
    R = rng.standard_normal((N, m, m)) * s + 3.0 * np.eye(m)
    Ys = rng.standard_normal((N * m, nrhs))
    return CycSystem(S, R, cyc_matvec(S, R, Ys), Ys)


def periodic_bvp(N: int, m: int, nrhs: int = 1, seed_rep: int = 0) -> CycSystem:
    """Trapezoidal rule for the periodic linear BVP y' = L(t) y + q(t) on [0,1],
    y(0) = y(1), with L(t) = S + cos(2 pi t) K (S, K as in the BVP workload) and
    the periodic exact solution y(t) = exp(sin(2 pi t)) v: rows
    S_j = -(I + h/2 L(t_j)), R_j = I - h/2 L(t_{j+1}), r_j = h/2 (q(t_j) + q(t_{j+1})),
    j = 0..N-1, with y_N identified with y_0.  Ystar holds y(t_j), j < N."""
    rng = rng_for(9, seed_rep)
    Sm = stable_matrix(m, rng)
    K = rng.standard_normal((m, m)) * 0.1
    V = rng.standard_normal((m, nrhs))
    h = 1.0 / N
    t = np.arange(N + 1) * h
    L = Sm[None] + np.cos(2 * np.pi * t)[:, None, None] * K[None]
    ys = np.exp(np.sin(2 * np.pi * t))[:, None, None] * V[None]                  # [N+1][m][nrhs]
    dys = (2 * np.pi * np.cos(2 * np.pi * t) * np.exp(np.sin(2 * np.pi * t)))[:, None, None] * V[None]
    q = dys - np.einsum("jab,jbc->jac", L, ys)
    I = np.eye(m)
    S = -(I[None] + 0.5 * h * L[:-1])
    R = I[None] - 0.5 * h * L[1:]
    rhs = 0.5 * h * (q[:-1] + q[1:])
    return CycSystem(S, R, rhs.reshape(N * m, nrhs), ys[:-1].reshape(N * m, nrhs))


# --------------------------------------------------------------------- BABD --

@dataclass
class BvpProblem:
    """Linear BVP y' = L(t) y + q(t) on [0,1], B0 y(0) + B1 y(1) = beta,
    with exact solution y(t) = exp(sin 3t) v (one v per right-hand side)."""
    Smat: np.ndarray
    K: np.ndarray
    B0: np.ndarray
    B1: np.ndarray
    V: np.ndarray          # [m, nrhs]

    def L(self, t):
        t = np.asarray(t, dtype=np.float64)
        return self.Smat[None] + np.cos(2 * np.pi * t)[:, None, None] * self.K[None]

    def y(self, t):
        t = np.asarray(t, dtype=np.float64)
        return np.exp(np.sin(3 * t))[:, None, None] * self.V[None]

    def q(self, t):
        t = np.asarray(t, dtype=np.float64)
        dy = (3 * np.cos(3 * t) * np.exp(np.sin(3 * t)))[:, None, None] * self.V[None]
        return dy - np.einsum("tab,tbk->tak", self.L(t), self.y(t))


@dataclass
class BabdSystem:
    S: np.ndarray
    R: np.ndarray
    B0: np.ndarray
    B1: np.ndarray
    RHS: np.ndarray        # [(N+1)*m, nrhs], boundary row first
    Yexact: np.ndarray     # [(N+1)*m, nrhs]: y(t_j) of the continuous problem
    problem: BvpProblem = field(repr=False)


def random_orthogonal(m: int, rng) -> np.ndarray:
    q, r = np.linalg.qr(rng.standard_normal((m, m)))
    return q * np.sign(np.diag(r))[None, :]


def stable_matrix(m: int, rng) -> np.ndarray:
    """S = Q Lam Q^T, Q random orthogonal, Lam block diagonal with 2x2 blocks
    [[a, b], [-b, a]], a ~ U[-5,-0.5], b ~ U[-3,3] (one 1x1 block a if m is
    odd): eigenvalues a +- ib with real parts in [-5, -0.5]."""
    Q = random_orthogonal(m, rng)
    lam = np.zeros((m, m))
    i = 0
    while i + 1 < m:
        a = rng.uniform(-5.0, -0.5)
        b = rng.uniform(-3.0, 3.0)
        lam[i:i + 2, i:i + 2] = [[a, b], [-b, a]]
        i += 2
    if i < m:
        lam[i, i] = rng.uniform(-5.0, -0.5)
    return Q @ lam @ Q.T


def bvp_problem(m: int, nrhs: int = 1, separated: bool = False, seed_rep: int = 0,
                rng=None, workload: int = 3) -> BvpProblem:
    """Seeded linear BVP: L(t) = S + cos(2 pi t) K, K ~ N(0, 0.1^2).

    Boundary conditions: general (non-separated) B0 = random orthogonal and
    B1 = G / (2 ||G||_2), so ||B1||_2 = 1/2; with ||Phi(1)||_2 close to 1 for
    this L, B0 + B1 Phi(1) is nonsingular and well conditioned by construction.
    ``separated=True``: B0 = [Ba; 0], B1 = [0; Bb] with ceil(m/2) rows at t=0."""
    rng = rng if rng is not None else rng_for(workload, seed_rep)
    Smat = stable_matrix(m, rng)
    K = rng.standard_normal((m, m)) * 0.1
    if separated:
        ma = (m + 1) // 2
        B0 = np.zeros((m, m))
        B1 = np.zeros((m, m))
        B0[:ma] = rng.standard_normal((ma, m))
        B1[ma:] = rng.standard_normal((m - ma, m))
    else:
        B0 = random_orthogonal(m, rng)
        G = rng.standard_normal((m, m))
        B1 = G / (2.0 * np.linalg.norm(G, 2))
    V = rng.standard_normal((m, nrhs))
    return BvpProblem(Smat, K, B0, B1, V)


def trapezoidal_babd(prob: BvpProblem, N: int) -> BabdSystem:
    """Trapezoidal rule on the uniform mesh t_j = j h, h = 1/N:
    S_j = -(I + h/2 L(t_j)), R_j = I - h/2 L(t_{j+1}), r_j = h/2 (q(t_j) + q(t_{j+1})),
    boundary row B0 y_0 + B1 y_N = beta with beta from the exact solution."""
    m = prob.Smat.shape[0]
    h = 1.0 / N
    t = np.arange(N + 1, dtype=np.float64) * h
    Lt = prob.L(t)
    I = np.eye(m)
    S = -(I[None] + 0.5 * h * Lt[:-1])
    R = I[None] - 0.5 * h * Lt[1:]
    qt = prob.q(t)
    r = 0.5 * h * (qt[:-1] + qt[1:])
    yt = prob.y(t)
    beta = prob.B0 @ yt[0] + prob.B1 @ yt[N]
    nrhs = prob.V.shape[1]
    RHS = np.concatenate([beta[None], r], axis=0).reshape((N + 1) * m, nrhs)
    return BabdSystem(np.ascontiguousarray(S), np.ascontiguousarray(R), prob.B0.copy(),
                      prob.B1.copy(), RHS, yt.reshape((N + 1) * m, nrhs), prob)


def babd_bvp(N: int, m: int, nrhs: int = 1, separated: bool = False, seed_rep: int = 0,
             rng=None) -> BabdSystem:
    return trapezoidal_babd(bvp_problem(m, nrhs, separated, seed_rep, rng), N)


def babd_random(N: int, m: int, nrhs: int = 1, seed_rep: int = 0, rng=None) -> BabdSystem:
    """A generic (non-ODE) BABD system with well conditioned diagonal blocks, for
    structure tests: R_j = 3 I + G/sqrt(m), S_j = G/sqrt(m), B0, B1 as for the
    non-separated BVP."""
    rng = rng if rng is not None else rng_for(6, seed_rep)
    s = 1.0 / math.sqrt(m)
    S = rng.standard_normal((N, m, m)) * s
    R = rng.standard_normal((N, m, m)) * s + 3.0 * np.eye(m)
    B0 = random_orthogonal(m, rng)
    G = rng.standard_normal((m, m))
    B1 = G / (2.0 * np.linalg.norm(G, 2))
    Ys = rng.standard_normal(((N + 1) * m, nrhs))
    RHS = babd_matvec(S, R, B0, B1, Ys)
    return BabdSystem(S, R, B0, B1, RHS, Ys, None)


# ------------------------------------------------------- batched and served --

@dataclass
class BatchSpec:
    n: int           # unknowns (a multiple of m)
    m: int
    lowprec: bool    # True: low-precision factor + FP64 refinement
    seed: int


def batch_specs(count: int = 4096, nmin: float = 1e3, nmax: float = 1e6,
                ms=(1, 4, 8, 16, 32), rep: int = 0) -> list:
    """Uneven independent systems: n log-uniform in [nmin, nmax], m uniform
    from ``ms``, a 50/50 precision tag; n is rounded down to a multiple of m."""
    rng = rng_for(4, rep)
    out = []
    for k in range(count):
        n = int(math.exp(rng.uniform(math.log(nmin), math.log(nmax))))
        m = int(rng.choice(ms))
        n = max(2 * m, (n // m) * m)
        out.append(BatchSpec(n, m, bool(rng.integers(0, 2)), int(SEED_BASE + 4000 * 1000 + k)))
    return out


def scalar_batch_specs(count: int = 1024, n: int = 1 << 16, rep: int = 0) -> list:
    """The scalar tridiagonal throughput workload: `count` independent systems
    of order n (the diagonally dominant scalar recipe, one seed each), all FP64."""
    return [BatchSpec(n, 1, False, int(SEED_BASE + 1000 * 1 + 100000 * (rep + 1) + k)) for k in range(count)]


def batch_systems_device(specs: list, device, seed: int = SEED_BASE + 4000) -> list:
    """The batch recipe generated on a CUDA device with torch (the sizes of the
    full batch do not fit a host round trip): per spec, m = 1 the scalar recipe
    (d ~ U[4,6], dl, du ~ U[-1,1]), m > 1 the block recipe (D = 4I + G/sqrt(m),
    B, C = G/sqrt(m)); one right-hand side F ~ N(0,1); "prec" from the spec's
    precision tag.  Returns dicts with B, D, C, F, an empty X and prec."""
    import torch
    g = torch.Generator(device=device).manual_seed(int(seed))
    out = []
    for sp in specs:
        N, m = sp.n // sp.m, sp.m
        s = 1.0 / m ** 0.5
        if m == 1:
            D = torch.rand((N, 1, 1), generator=g, device=device, dtype=torch.float64) * 2 + 4
            B = torch.rand((N, 1, 1), generator=g, device=device, dtype=torch.float64) * 2 - 1
            C = torch.rand((N, 1, 1), generator=g, device=device, dtype=torch.float64) * 2 - 1
        else:
            B = torch.randn((N, m, m), generator=g, device=device, dtype=torch.float64) * s
            C = torch.randn((N, m, m), generator=g, device=device, dtype=torch.float64) * s
            D = torch.randn((N, m, m), generator=g, device=device, dtype=torch.float64) * s
            D += 4 * torch.eye(m, device=device, dtype=torch.float64)
        F = torch.randn((N * m, 1), generator=g, device=device, dtype=torch.float64)
        out.append({"B": B, "D": D, "C": C, "F": F, "X": torch.empty_like(F),
                    "prec": "bf16_ir" if sp.lowprec else "fp64"})
    return out


def batch_system(spec: BatchSpec, nrhs: int = 1) -> BtriSystem:
    """Materialise one batched system: m = 1 follows the scalar recipe, m > 1
    the block recipe."""
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    if spec.m == 1:
        t = tri_sdd(spec.n, nrhs, rng=rng)
        N = spec.n
        return BtriSystem(t.dl.reshape(N, 1, 1), t.d.reshape(N, 1, 1), t.du.reshape(N, 1, 1),
                          t.f, t.xstar)
    return btri_random(spec.n // spec.m, spec.m, nrhs, rng=rng)


@dataclass
class ServeRequest:
    arrival_s: float
    m: int
    N: int
    nrhs: int
    problem_id: int        # requests with equal problem_id share L, B0, B1
    v_seed: int


def serve_trace(duration_s: float, rate: float = 2000.0, ms=(4, 8, 16), Nmin: float = 1e3,
                Nmax: float = 5e5, reuse: float = 0.3, rep: int = 0) -> list:
    """Poisson arrivals (exponential gaps) of BVP solve requests; a fraction
    ``reuse`` repeats an earlier problem (same L, B0, B1, N, m; new v)."""
    rng = rng_for(5, rep)
    t = 0.0
    out, problems = [], []
    k = 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration_s:
            break
        nrhs = int(rng.integers(1, 33))
        if problems and rng.uniform() < reuse:
            pid, m, N = problems[int(rng.integers(0, len(problems)))]
        else:
            m = int(rng.choice(ms))
            N = int(math.exp(rng.uniform(math.log(Nmin), math.log(Nmax))))
            pid = len(problems)
            problems.append((pid, m, N))
        out.append(ServeRequest(t, m, N, nrhs, pid, SEED_BASE + 5000 * 1000 + k))
        k += 1
    return out


def serve_system(req: ServeRequest) -> BabdSystem:
    prob_rng = np.random.Generator(np.random.PCG64(SEED_BASE + 5000 * 1000 + 7919 * (req.problem_id + 1)))
    prob = bvp_problem(req.m, 1, rng=prob_rng)
    vrng = np.random.Generator(np.random.PCG64(req.v_seed))
    prob.V = vrng.standard_normal((req.m, req.nrhs))
    return trapezoidal_babd(prob, req.N)
