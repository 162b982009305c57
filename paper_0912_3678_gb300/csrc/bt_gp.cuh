// Partition-method kernels with a group of M*M lanes per partition (or per
// separator, or per (partition, column chunk) in the solves), for block sizes
// M in {2, 4} in FP64: the same algebra and outputs as the thread-per-partition
// bodies of bt_tp.cuh, with lane q of a group holding entry (q / M, q % M) of
// every M x M block and the block products done through warp shuffles.
//
// Why: on this GPU an FP64 instruction costs a sub-partition the same time
// whether 1 or 32 of its lanes are active, so a thread that carries a whole
// block row (7 M^3 FMAs at M = 4) alone takes ~14 us per row.  Thread per
// partition is right where the partitions fill every lane (the first level of
// a large system); the recursion levels and small systems have far fewer
// partitions, are latency-bound, and there M*M lanes share each row's work.
#pragma once
#include "bt_device.cuh"
#include "bt_level.h"

namespace bt {

template <int M>
struct Grp {
    static constexpr int G = M * M;
    int q, r, c, base;
    unsigned mask;
    __device__ __forceinline__ Grp() {
        const int lane = threadIdx.x & 31;
        q = lane % G;
        r = q / M;
        c = q % M;
        base = lane - q;
        mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << base);
    }
    // entry (rr, cc) of the block whose entries the group's lanes hold
    __device__ __forceinline__ double at(double v, int rr, int cc) const {
        return __shfl_sync(mask, v, base + rr * M + cc);
    }
};

// Entry (r, c) of sgn * A B (+ acc if ACC), A and B held one entry per lane.
template <int M, bool NEG, bool ACC>
__device__ __forceinline__ double gmm(const Grp<M>& g, double A, double B, double acc) {
    double s = ACC ? acc : 0.0;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const double x = g.at(A, g.r, k), y = g.at(B, k, g.c);
        s = fma(NEG ? -x : x, y, s);
    }
    return s;
}

// In-place Gauss-Jordan inverse with partial pivoting of the block held one
// entry per lane (same pivot choice as rgj_inverse: the largest magnitude in
// the column, the first such row on ties).
template <int M>
__device__ __forceinline__ bool ggj_inverse(const Grp<M>& g, double& a, long long* st, int level, long long part,
                                            long long row) {
    int perm[M];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        // pivot row: largest |a(r, k)| over r >= k
        const double ak = g.at(a, g.r, k);
        unsigned long long best = (g.r >= k) ? abs_key(ak) : 0ull;
        int pr = (g.r >= k) ? g.r : M;   // rows above k never win (M sorts after every row)
#pragma unroll
        for (int off = M; off < M * M; off <<= 1) {
            const unsigned long long ok2 = __shfl_xor_sync(g.mask, best, off);
            const int op = __shfl_xor_sync(g.mask, pr, off);
            if (ok2 > best || (ok2 == best && op < pr)) {
                best = ok2;
                pr = op;
            }
        }
        // rows k and pr swap
        const int src = (g.r == k) ? pr : ((g.r == pr) ? k : g.r);
        a = g.at(a, src, g.c);
        perm[k] = pr;
        double pv = g.at(a, k, k);
        if (nonfinite(pv)) {
            if (g.q == 0) report(st, ST_NONFINITE, level, part, row);
            pv = 1.0;
            ok = false;
        } else if (best == 0ull) {
            if (g.q == 0) report(st, ST_SINGULAR, level, part, row);
            pv = 1.0;
            ok = false;
        }
        const double rv = rcp(pv);
        // scale row k; eliminate column k from the other rows
        // every lane takes part in both shuffles before any lane-dependent choice
        const double l = g.at(a, g.r, k);     // a(r, k) before the update
        const double akc = g.at(a, k, g.c);   // a(k, c) before the update
        const double rowk = (g.c == k) ? rv : akc * rv;   // new a(k, c)
        if (g.r == k) {
            a = rowk;
        } else {
            a = (g.c == k) ? -l * rv : fma(-l, rowk, a);
        }
    }
    // undo the row interchanges as column interchanges
#pragma unroll
    for (int k = M - 1; k >= 0; --k) {
        const int p = perm[k];
        const int src = (g.c == k) ? p : ((g.c == p) ? k : g.c);
        a = g.at(a, g.r, src);
    }
    return ok;
}

// ---------------------------------------------------------------- factor --
template <int M, int MODE>
__device__ __forceinline__ void factor_gp_body(const LevelArgs& a, const long long tid) {
    constexpr int MM = M * M;
    const Grp<M> g;
    const long long i = tid / MM;
    if (i >= a.p) return;
    const Part pt = part_bounds(a, MODE, i);
    double* gDinv = reinterpret_cast<double*>(a.Dinv);
    double* gY = reinterpret_cast<double*>(a.Y);
    double* gZ = reinterpret_cast<double*>(a.Zc);
    const int q = g.q;
    const bool wchain = (MODE == 0) && pt.hasL;
    double Yp = 0.0, Zp = 0.0, W = 0.0, CP = 0.0;
    if (wchain) W = a.C[(pt.s - 1 - a.shift) * MM + q];   // W_s = C of the left separator row
    // the blocks of row j + 1 are loaded while row j is processed
    auto needC_of = [&](long long j) { return (MODE == 0) && ((j < pt.e - 1) || pt.hasR); };
    double nD = 0.0, nB = 0.0, nC = 0.0;
    if (pt.s < pt.e) {
        nD = a.D[(pt.s - a.shift) * MM + q];
        nB = pt.hasL ? a.B[(pt.s - a.shift) * MM + q] : 0.0;
        nC = needC_of(pt.s) ? a.C[(pt.s - a.shift) * MM + q] : 0.0;
    }
    for (long long j = pt.s; j < pt.e; ++j) {
        const bool first = (j == pt.s);
        const bool needC = needC_of(j);
        double Dp = nD;
        const double Bj = nB, Cj = nC;
        if (j + 1 < pt.e) {
            nD = a.D[(j + 1 - a.shift) * MM + q];
            nB = a.B[(j + 1 - a.shift) * MM + q];
            nC = needC_of(j + 1) ? a.C[(j + 1 - a.shift) * MM + q] : 0.0;
        }
        if (MODE == 0 && !first) Dp = gmm<M, true, true>(g, Bj, Yp, Dp);
        ggj_inverse<M>(g, Dp, a.status, a.level, i, j);
        gDinv[j * MM + q] = Dp;
        if (pt.hasL) {
            if (!first) {
                const double t = gmm<M, false, false>(g, Bj, Zp, 0.0);
                Zp = gmm<M, true, false>(g, Dp, t, 0.0);
            } else {
                Zp = gmm<M, true, false>(g, Dp, Bj, 0.0);
            }
            gZ[j * MM + q] = Zp;
        }
        if (needC) {
            Yp = gmm<M, false, false>(g, Dp, Cj, 0.0);
            gY[j * MM + q] = Yp;
        }
        if (wchain) {
            // CP += W_j Zc_j ;  W_{j+1} = -W_j Y_j  (zero after the last row without x_R)
            CP = gmm<M, false, true>(g, W, Zp, CP);
            W = needC ? gmm<M, true, false>(g, W, Yp, 0.0) : 0.0;
        }
    }
    if (MODE == 0) {
        if (!pt.hasL) return;
        reinterpret_cast<double*>(a.Pf)[i * MM + q] = CP;
        reinterpret_cast<double*>(a.Qf)[i * MM + q] = W;
    } else {
        const long long e = pt.e;
        const double Be = a.B[(e - a.shift) * MM + q];
        a.Dn[i * MM + q] = a.D[(e - a.shift) * MM + q];
        const double t = gmm<M, false, false>(g, Be, Zp, 0.0);
        a.Bn[i * MM + q] = (pt.e > pt.s) ? t : Be;
    }
}

// --------------------------------------------------------------- assemble --
template <int M>
__device__ __forceinline__ void assemble_gp_body(const LevelArgs& a, const long long tid) {
    constexpr int MM = M * M;
    const Grp<M> g;
    const long long s = tid / MM;
    if (s >= a.p - 1) return;
    const int q = g.q;
    const Part pt = part_bounds(a, 0, s);
    const long long e = pt.e;
    const bool local = pt.e > pt.s;   // partition s has local rows before its separator
    const double Be = a.B[(e - a.shift) * MM + q];
    double al = a.D[(e - a.shift) * MM + q];
    const double Pf = reinterpret_cast<const double*>(a.Pf)[(s + 1) * MM + q];
    const double Yl = local ? reinterpret_cast<const double*>(a.Y)[(e - 1) * MM + q] : 0.0;
    al = gmm<M, true, true>(g, Be, Yl, al);
    a.Dn[s * MM + q] = al + Pf;
    const double Zl = local ? reinterpret_cast<const double*>(a.Zc)[(e - 1) * MM + q] : 0.0;
    const double bz = gmm<M, false, false>(g, Be, Zl, 0.0);
    const double be = (s == 0) ? 0.0 : (local ? bz : Be);   // no local rows: direct coupling
    const double ga = (s + 1 < a.p - 1) ? reinterpret_cast<const double*>(a.Qf)[(s + 1) * MM + q] : 0.0;
    a.Bn[s * MM + q] = be;
    a.Cn[s * MM + q] = ga;
}

// ----------------------------------------------------------------- solves --
// Unit = (partition, chunk of M right-hand-side columns); lane (r, c) of the
// group carries column chunk*M + c (zero, and never stored, past nr).
template <int M>
struct Cols {
    long long unit;
    int col;
    bool live;
};
template <int M>
__device__ __forceinline__ Cols<M> cols_of(const Grp<M>& g, const LevelArgs& a, long long tid) {
    const int nc = (a.nr + M - 1) / M;
    const long long u = tid / (M * M);
    Cols<M> o;
    o.unit = u / nc;
    o.col = (int)(u % nc) * M + g.c;
    o.live = o.col < a.nr;
    return o;
}

template <int M, int MODE>
__device__ __forceinline__ void solve_fwd_gp_body(const LevelArgs& a, const long long tid) {
    constexpr int MM = M * M;
    const Grp<M> g;
    const Cols<M> cl = cols_of<M>(g, a, tid);
    const long long i = cl.unit;
    if (i >= a.p) return;
    const int nr = a.nr, q = g.q;
    const long long E = (long long)M * nr;
    const long long o = (long long)g.r * nr + cl.col;   // offset of this lane's entry in a block row
    const Part pt = part_bounds(a, MODE, i);
    const double* gDinv = reinterpret_cast<const double*>(a.Dinv);
    double hp = 0.0;
    // row j + 1's data loaded while row j is processed
    double nF = 0.0, nB = 0.0, nDi = 0.0;
    if (pt.s < pt.e) {
        nF = cl.live ? a.F[pt.s * E + o] : 0.0;
        nDi = gDinv[pt.s * MM + q];
    }
    for (long long j = pt.s; j < pt.e; ++j) {
        double v = nF;
        const double Bj = nB, Di = nDi;
        if (j + 1 < pt.e) {
            nF = cl.live ? a.F[(j + 1) * E + o] : 0.0;
            nB = a.B[(j + 1 - a.shift) * MM + q];
            nDi = gDinv[(j + 1) * MM + q];
        }
        if (j != pt.s) v = gmm<M, true, true>(g, Bj, hp, v);
        hp = gmm<M, false, false>(g, Di, v, 0.0);
        if (cl.live) a.X[j * E + o] = hp;
    }
    if (MODE == 1) {
        const long long e = pt.e;
        if (i == 0 && cl.live) a.Fn[o] = a.F[o];
        double gv = cl.live ? a.F[e * E + o] : 0.0;
        if (pt.e > pt.s) gv = gmm<M, true, true>(g, a.B[(e - a.shift) * MM + q], hp, gv);
        if (cl.live) a.Fn[(i + 1) * E + o] = gv;
        return;
    }
    if (!pt.hasL) return;
    const double* gY = reinterpret_cast<const double*>(a.Y);
    for (long long j = pt.e - 2; j >= pt.s; --j) {
        const double h = cl.live ? a.X[j * E + o] : 0.0;
        hp = gmm<M, true, true>(g, gY[j * MM + q], hp, h);
    }
    if (cl.live) reinterpret_cast<double*>(a.Hf)[i * E + o] = hp;
}

template <int M>
__device__ __forceinline__ void assemble_rhs_gp_body(const LevelArgs& a, const long long tid) {
    constexpr int MM = M * M;
    const Grp<M> g;
    const Cols<M> cl = cols_of<M>(g, a, tid);
    const long long s = cl.unit;
    if (s >= a.p - 1) return;
    const int nr = a.nr, q = g.q;
    const long long E = (long long)M * nr;
    const long long o = (long long)g.r * nr + cl.col;
    const Part pt = part_bounds(a, 0, s);
    const long long e = pt.e;
    double gv = cl.live ? a.F[e * E + o] : 0.0;
    const double h = (cl.live && pt.e > pt.s) ? a.X[(e - 1) * E + o] : 0.0;
    const double H = cl.live ? reinterpret_cast<const double*>(a.Hf)[(s + 1) * E + o] : 0.0;
    gv = gmm<M, true, true>(g, a.B[(e - a.shift) * MM + q], h, gv);
    gv = gmm<M, true, true>(g, a.C[(e - a.shift) * MM + q], H, gv);
    if (cl.live) a.Fn[s * E + o] = gv;
}

template <int M, int MODE>
__device__ __forceinline__ void solve_bwd_gp_body(const LevelArgs& a, const long long tid) {
    constexpr int MM = M * M;
    const Grp<M> g;
    const Cols<M> cl = cols_of<M>(g, a, tid);
    const long long i = cl.unit;
    if (i >= a.p) return;
    const int nr = a.nr, q = g.q;
    const long long E = (long long)M * nr;
    const long long o = (long long)g.r * nr + cl.col;
    const Part pt = part_bounds(a, MODE, i);
    const long long li = (MODE == 0) ? i - 1 : i;
    const long long ri = (MODE == 0) ? i : i + 1;
    double x = 0.0, xl = 0.0;
    if (pt.hasR) {
        const double xr = cl.live ? a.Xn[ri * E + o] : 0.0;
        if (cl.live) a.X[pt.e * E + o] = xr;
        x = xr;
    }
    if (MODE == 1 && i == 0 && cl.live) a.X[o] = a.Xn[o];
    if (pt.hasL) xl = cl.live ? a.Xn[li * E + o] : 0.0;
    const double* gY = reinterpret_cast<const double*>(a.Y);
    const double* gZ = reinterpret_cast<const double*>(a.Zc);
    auto useY = [&](long long j) { return MODE == 0 && ((j < pt.e - 1) || pt.hasR); };
    // row j - 1's data loaded while row j is processed
    double nH = 0.0, nY = 0.0, nZ = 0.0;
    if (pt.e > pt.s) {
        const long long j = pt.e - 1;
        nH = cl.live ? a.X[j * E + o] : 0.0;
        nY = useY(j) ? gY[j * MM + q] : 0.0;
        nZ = pt.hasL ? gZ[j * MM + q] : 0.0;
    }
    for (long long j = pt.e - 1; j >= pt.s; --j) {
        double v = nH;
        const double Yj = nY, Zj = nZ;
        if (j - 1 >= pt.s) {
            nH = cl.live ? a.X[(j - 1) * E + o] : 0.0;
            nY = useY(j - 1) ? gY[(j - 1) * MM + q] : 0.0;
            nZ = pt.hasL ? gZ[(j - 1) * MM + q] : 0.0;
        }
        if (useY(j)) v = gmm<M, true, true>(g, Yj, x, v);
        if (pt.hasL) v = gmm<M, false, true>(g, Zj, xl, v);
        x = v;
        if (cl.live) a.X[j * E + o] = x;
    }
}

// Units [unit0, unit_end) of the launch (whole groups: both are multiples of M*M).
__device__ __forceinline__ bool gp_unit(const LevelArgs& a, long long& u) {
    u = a.unit0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    return !(a.unit_end > 0 && u >= a.unit_end);
}
template <int M, int MODE>
__global__ void __launch_bounds__(128) k_factor_gp(const LevelArgs a) {
    long long u;
    if (gp_unit(a, u)) factor_gp_body<M, MODE>(a, u);
}
template <int M>
__global__ void __launch_bounds__(128) k_assemble_gp(const LevelArgs a) {
    long long u;
    if (gp_unit(a, u)) assemble_gp_body<M>(a, u);
}
template <int M, int MODE>
__global__ void __launch_bounds__(128) k_solve_fwd_gp(const LevelArgs a) {
    long long u;
    if (gp_unit(a, u)) solve_fwd_gp_body<M, MODE>(a, u);
}
template <int M>
__global__ void __launch_bounds__(128) k_assemble_rhs_gp(const LevelArgs a) {
    long long u;
    if (gp_unit(a, u)) assemble_rhs_gp_body<M>(a, u);
}
template <int M, int MODE>
__global__ void __launch_bounds__(128) k_solve_bwd_gp(const LevelArgs a) {
    long long u;
    if (gp_unit(a, u)) solve_bwd_gp_body<M, MODE>(a, u);
}

}  // namespace bt
