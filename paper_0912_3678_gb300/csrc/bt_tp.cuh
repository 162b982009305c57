// Partition-method kernels with one thread per partition (factor) or per
// (partition, right-hand side) pair (solve), for block sizes M in {1, 2, 4}:
// the m x m blocks live in registers.  Same algorithm and outputs as the
// CTA kernels in bt_cta.cuh.
#pragma once
#include <type_traits>

#include "bt_device.cuh"
#include "bt_level.h"

namespace bt {

template <typename T, int M>
struct Reg {
    static constexpr int MM = M * M;
};

template <typename T, int M, typename G>
__device__ __forceinline__ void rld(T (&b)[M * M], const G* g) {
#pragma unroll
    for (int u = 0; u < M * M; ++u) b[u] = (T)g[u];
}
template <typename T, int M, typename G>
__device__ __forceinline__ void rst(G* g, const T (&b)[M * M]) {
#pragma unroll
    for (int u = 0; u < M * M; ++u) g[u] = (G)b[u];
}
// c = sgn * a b (+ c if ACC)
template <typename T, int M, bool NEG, bool ACC>
__device__ __forceinline__ void rmm(T (&c)[M * M], const T (&a)[M * M], const T (&b)[M * M]) {
    T out[M * M];
#pragma unroll
    for (int r = 0; r < M; ++r)
#pragma unroll
        for (int cc = 0; cc < M; ++cc) {
            T acc = ACC ? c[r * M + cc] : T(0);
#pragma unroll
            for (int k = 0; k < M; ++k) acc = fmaT<T>(NEG ? -a[r * M + k] : a[r * M + k], b[k * M + cc], acc);
            out[r * M + cc] = acc;
        }
#pragma unroll
    for (int u = 0; u < M * M; ++u) c[u] = out[u];
}

// In-place Gauss-Jordan inverse with partial pivoting, blocks in registers.
// brk != null (pivoted levels): a pivot with |pivot| <= thr marks a breakdown
// of the partition at this row (atomicMin into brk[part]) instead of an error.
template <typename T, int M>
__device__ __forceinline__ bool rgj_inverse(T (&a)[M * M], long long* st, int level, long long part,
                                            long long row, long long* brk = nullptr, T thr = T(0),
                                            long long cap = 0) {
    int perm[M];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        int p = k;
        unsigned long long best = abs_key(a[k * M + k]);
#pragma unroll
        for (int i = k + 1; i < M; ++i) {
            const unsigned long long key = abs_key(a[i * M + k]);
            if (key > best) {
                best = key;
                p = i;
            }
        }
#pragma unroll
        for (int i = k + 1; i < M; ++i) {
            if (p == i) {
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    const T t = a[k * M + c];
                    a[k * M + c] = a[i * M + c];
                    a[i * M + c] = t;
                }
            }
        }
        perm[k] = p;
        T pv = a[k * M + k];
        if (nonfinite(pv)) {
            report(st, ST_NONFINITE, level, part, row);
            pv = T(1);
            ok = false;
        } else if (brk != nullptr && !(abs_key(pv) > abs_key(thr))) {
            if (ok) record_breakdown(brk, cap, row);
            pv = T(1);
            ok = false;
        } else if (best == 0ull) {
            report(st, ST_SINGULAR, level, part, row);
            pv = T(1);
            ok = false;
        }
        const T r = rcp(pv);
#pragma unroll
        for (int c = 0; c < M; ++c) a[k * M + c] = (c == k) ? r : a[k * M + c] * r;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            if (i == k) continue;
            const T l = a[i * M + k];
#pragma unroll
            for (int c = 0; c < M; ++c) a[i * M + c] = (c == k) ? -l * r : fmaT<T>(-l, a[k * M + c], a[i * M + c]);
        }
    }
#pragma unroll
    for (int k = M - 1; k >= 0; --k) {
#pragma unroll
        for (int i = k + 1; i < M; ++i) {
            if (perm[k] == i) {
#pragma unroll
                for (int r = 0; r < M; ++r) {
                    const T t = a[r * M + k];
                    a[r * M + k] = a[r * M + i];
                    a[r * M + i] = t;
                }
            }
        }
    }
    return ok;
}

// ------------------------------------------------------- scalar partitions --
// m = 1, block tridiagonal levels: the recurrences of the bodies below with
// the rows read and the factors written four at a time (one 256-bit access
// per thread and array: whole 32-byte sectors, half the load instructions of
// 128-bit pairs), and the loads of the next chunks issued before the current
// four rows are processed.  Rows before the first multiple of 4 and after the
// last one, and arrays that are not 32-byte aligned, are taken one at a time.
template <typename P, typename Q, typename R>
__device__ __forceinline__ bool aligned32(const P* p, const Q* q, const R* r) {
    return (((uintptr_t)p | (uintptr_t)q | (uintptr_t)r) & 31u) == 0;
}
template <typename T>
__device__ __forceinline__ void st4(T* g, const T (&v)[4]) {
    if constexpr (std::is_same<T, double>::value) {
        *reinterpret_cast<double4_32a*>(g) = make_double4_32a(v[0], v[1], v[2], v[3]);
    } else {
        *reinterpret_cast<float4*>(g) = make_float4(v[0], v[1], v[2], v[3]);
    }
}
template <typename T>
__device__ __forceinline__ void ld4(T (&v)[4], const T* g) {
    if constexpr (std::is_same<T, double>::value) {
        const double4_32a p = *reinterpret_cast<const double4_32a*>(g);
        v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w;
    } else {
        const float4 p = *reinterpret_cast<const float4*>(g);
        v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w;
    }
}

template <typename T>
__device__ __forceinline__ void factor_tp_scalar(const LevelArgs& a, const long long i) {
    if (i >= a.p) return;
    const Part pt = part_bounds(a, 0, i);
    T* gDinv = reinterpret_cast<T*>(a.Dinv);
    T* gY = reinterpret_cast<T*>(a.Y);
    T* gZ = reinterpret_cast<T*>(a.Zc);
    const double* gB = a.B - a.shift;
    const double* gD = a.D - a.shift;
    const double* gC = a.C - a.shift;
    const long long s = pt.s, e = pt.e;
    const bool hasL = pt.hasL, hasR = pt.hasR;
    T yp = T(0), zp = T(0), cp = T(0);
    T w = hasL ? (T)gC[s - 1] : T(0);   // W_s = C of the left separator row
    const bool vec = aligned32(gB, gD, gC) && aligned32(gDinv, gY, gZ);
    auto step = [&](long long j, double bj, double dj, double cj, T& dinv, T& z, T& y) {
        const bool first = (j == s);
        const bool needB = !first || hasL;
        const bool needC = (j < e - 1) || hasR;
        T u = (T)dj;
        if (!first) u = fmaT<T>(-(T)bj, yp, u);
        bool ok = true;
        T pv = u;
        T thr = T(0);
        if (a.brk != nullptr) {
            unsigned long long mk = abs_key(u);
            if (needB) mk = max(mk, abs_key((T)bj));
            if (needC) mk = max(mk, abs_key((T)cj));
            thr = (T)a.tau * key_abs<T>(mk);
        }
        if (nonfinite(pv)) {
            report(a.status, ST_NONFINITE, a.level, i, j);
            pv = T(1);
            ok = false;
        } else if (a.brk != nullptr && !(abs_key(pv) > abs_key(thr))) {
            record_breakdown(a.brk, a.brk_cap, j);
            pv = T(1);
            ok = false;
        } else if (pv == T(0)) {
            report(a.status, ST_SINGULAR, a.level, i, j);
            pv = T(1);
            ok = false;
        }
        const T r = rcp(pv);
        dinv = r;
        z = T(0);
        if (hasL) z = first ? -r * (T)bj : -r * ((T)bj * zp);
        y = T(0);
        if (needC && (ok || a.brk == nullptr)) y = r * (T)cj;
        if (hasL) {
            cp = fmaT<T>(w, z, cp);
            w = needC ? -w * y : T(0);
        }
        if (needC) yp = y;
        zp = z;
    };
    long long j = s;
    for (; j < e && ((j & 3) || !vec); ++j) {
        T dv, zv, yv;
        step(j, gB[j], gD[j], gC[j], dv, zv, yv);
        gDinv[j] = dv;
        gZ[j] = zv;
        gY[j] = yv;
    }
    if (j + 4 <= e) {
        double cb[4], cd[4], cc[4];
        ld4<double>(cb, gB + j);
        ld4<double>(cd, gD + j);
        ld4<double>(cc, gC + j);
        for (; j + 4 <= e; j += 4) {
            const bool more = (j + 8 <= e);
            double nb[4], nd[4], nc[4];
            if (more) {
                ld4<double>(nb, gB + j + 4);
                ld4<double>(nd, gD + j + 4);
                ld4<double>(nc, gC + j + 4);
            }
            T dv[4], zv[4], yv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) step(j + u, cb[u], cd[u], cc[u], dv[u], zv[u], yv[u]);
            st4<T>(gDinv + j, dv);
            st4<T>(gZ + j, zv);
            st4<T>(gY + j, yv);
            if (more) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    cb[u] = nb[u];
                    cd[u] = nd[u];
                    cc[u] = nc[u];
                }
            }
        }
    }
    for (; j < e; ++j) {
        T dv, zv, yv;
        step(j, gB[j], gD[j], gC[j], dv, zv, yv);
        gDinv[j] = dv;
        gZ[j] = zv;
        gY[j] = yv;
    }
    if (!hasL) return;
    reinterpret_cast<T*>(a.Pf)[i] = cp;
    reinterpret_cast<T*>(a.Qf)[i] = w;
}

// Forward substitution h_j = D'_j^{-1}(f_j - b_j h_{j-1}) for one right-hand
// side; the top row's value after full elimination, H = sum_j w_j h_j with
// w_s = 1, w_{j+1} = -w_j Y_j, is accumulated on the way (no backward pass).
template <typename T>
__device__ __forceinline__ void solve_fwd_tp_scalar(const LevelArgs& a, const long long i) {
    if (i >= a.p) return;
    const Part pt = part_bounds(a, 0, i);
    const T* gDinv = reinterpret_cast<const T*>(a.Dinv);
    const T* gY = reinterpret_cast<const T*>(a.Y);
    const double* gB = a.B - a.shift;
    const double* F = a.F;
    double* X = a.X;
    const long long s = pt.s, e = pt.e;
    const bool hasL = pt.hasL;
    T h = T(0), H = T(0), w = T(1);
    const bool vec = aligned32(F, X, gB) && aligned32(gDinv, gY, gY);
    auto step = [&](long long j, double fj, double bj, T dinv, T yj) -> T {
        T v = (T)fj;
        if (j != s) v = fmaT<T>(-(T)bj, h, v);
        h = dinv * v;
        if (hasL) {
            H = fmaT<T>(w, h, H);
            w = -w * yj;
        }
        return h;
    };
    long long j = s;
    for (; j < e && ((j & 3) || !vec); ++j) X[j] = (double)step(j, F[j], gB[j], gDinv[j], hasL ? gY[j] : T(0));
    // chunks of four rows; the PD chunks after the one being processed are in flight
    constexpr int PD = 3;
    double qf[PD + 1][4], qb[PD + 1][4];
    T qd[PD + 1][4], qy[PD + 1][4];
    auto load = [&](long long r, int k) {
        ld4<double>(qf[k], F + r);
        ld4<double>(qb[k], gB + r);
        ld4<T>(qd[k], gDinv + r);
        if (hasL) ld4<T>(qy[k], gY + r);
    };
#pragma unroll
    for (int k = 0; k < PD; ++k)
        if (j + 4 * (k + 1) <= e) load(j + 4 * k, k);
    for (; j + 4 <= e; j += 4) {
        if (j + 4 * (PD + 1) <= e) load(j + 4 * PD, PD);
        double xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = (double)step(j + u, qf[0][u], qb[0][u], qd[0][u], hasL ? qy[0][u] : T(0));
        st4<double>(X + j, xv);
#pragma unroll
        for (int k = 0; k < PD; ++k)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                qf[k][u] = qf[k + 1][u];
                qb[k][u] = qb[k + 1][u];
                qd[k][u] = qd[k + 1][u];
                qy[k][u] = qy[k + 1][u];
            }
    }
    for (; j < e; ++j) X[j] = (double)step(j, F[j], gB[j], gDinv[j], hasL ? gY[j] : T(0));
    if (hasL) reinterpret_cast<T*>(a.Hf)[i] = H;
}

// Back substitution x_j = h_j + Zc_j x_L - Y_j x_{j+1}, one right-hand side,
// from the last local row up (chunks of four aligned rows, read backwards).
template <typename T>
__device__ __forceinline__ void solve_bwd_tp_scalar(const LevelArgs& a, const long long i) {
    if (i >= a.p) return;
    const Part pt = part_bounds(a, 0, i);
    const T* gY = reinterpret_cast<const T*>(a.Y);
    const T* gZ = reinterpret_cast<const T*>(a.Zc);
    double* X = a.X;
    const long long s = pt.s, e = pt.e;
    const bool hasL = pt.hasL, hasR = pt.hasR;
    T x = T(0), xl = T(0);
    const bool vec = aligned32(X, gY, gZ);
    if (hasR) {
        const double xr = a.Xn[i];
        X[e] = xr;
        x = (T)xr;
    }
    if (hasL) xl = (T)a.Xn[i - 1];
    auto step = [&](long long j, double hj, T yj, T zj) -> T {
        T v = (T)hj;
        if ((j < e - 1) || hasR) v = fmaT<T>(-yj, x, v);
        if (hasL) v = fmaT<T>(zj, xl, v);
        x = v;
        return v;
    };
    long long j = e - 1;
    for (; j >= s && (((j + 1) & 3) || !vec); --j) X[j] = (double)step(j, X[j], gY[j], hasL ? gZ[j] : T(0));
    // j + 1 is now a multiple of 4: chunks [j-3, j]; PD chunks below it in flight
    constexpr int PD = 3;
    double qh[PD + 1][4];
    T qy[PD + 1][4], qz[PD + 1][4];
    auto load = [&](long long r, int k) {
        ld4<double>(qh[k], X + r);
        ld4<T>(qy[k], gY + r);
        if (hasL) ld4<T>(qz[k], gZ + r);
    };
#pragma unroll
    for (int k = 0; k < PD; ++k)
        if (j - 3 - 4 * k >= s) load(j - 3 - 4 * k, k);
    for (; j - 3 >= s; j -= 4) {
        if (j - 3 - 4 * PD >= s) load(j - 3 - 4 * PD, PD);
        double xv[4];
#pragma unroll
        for (int u = 3; u >= 0; --u) xv[u] = (double)step(j - 3 + u, qh[0][u], qy[0][u], hasL ? qz[0][u] : T(0));
        st4<double>(X + j - 3, xv);
#pragma unroll
        for (int k = 0; k < PD; ++k)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                qh[k][u] = qh[k + 1][u];
                qy[k][u] = qy[k + 1][u];
                qz[k][u] = qz[k + 1][u];
            }
    }
    for (; j >= s; --j) X[j] = (double)step(j, X[j], gY[j], hasL ? gZ[j] : T(0));
}

template <typename T, int M, int MODE>
__device__ __forceinline__ void factor_tp_body(const LevelArgs& a, const long long i) {
    constexpr int MM = M * M;
    if constexpr (M == 1 && MODE == 0) {
        factor_tp_scalar<T>(a, i);
        return;
    }
    if (i >= a.p) return;
    const Part pt = part_bounds(a, MODE, i);
    T* gDinv = reinterpret_cast<T*>(a.Dinv);
    T* gY = reinterpret_cast<T*>(a.Y);
    T* gZ = reinterpret_cast<T*>(a.Zc);
    const bool wchain = (MODE == 0) && pt.hasL;
    T Yp[MM], Zp[MM], W[MM], CP[MM];
#pragma unroll
    for (int u = 0; u < MM; ++u) Yp[u] = Zp[u] = W[u] = CP[u] = T(0);
    if (wchain) rld<T, M>(W, a.C + (pt.s - 1 - a.shift) * MM);   // W_s = C of the left separator row
    for (long long j = pt.s; j < pt.e; ++j) {
        const bool first = (j == pt.s);
        const bool needB = !first || pt.hasL;
        const bool needC = (MODE == 0) && ((j < pt.e - 1) || pt.hasR);
        T Dp[MM], Bj[MM];
        rld<T, M>(Dp, a.D + (j - a.shift) * MM);
        if (needB) rld<T, M>(Bj, a.B + (j - a.shift) * MM);
        if (MODE == 0 && !first) rmm<T, M, true, true>(Dp, Bj, Yp);
        T thr = T(0);
        if (a.brk != nullptr) {
            // breakdown threshold: tau times the largest entry of B_j, D'_j, C_j
            unsigned long long mk = 0ull;
#pragma unroll
            for (int u = 0; u < MM; ++u) {
                mk = max(mk, abs_key(Dp[u]));
                if (needB) mk = max(mk, abs_key(Bj[u]));
            }
            if (needC) {
                const double* gC = a.C + (j - a.shift) * MM;
#pragma unroll
                for (int u = 0; u < MM; ++u) mk = max(mk, abs_key((T)gC[u]));
            }
            thr = (T)a.tau * key_abs<T>(mk);
        }
        const bool ok = rgj_inverse<T, M>(Dp, a.status, a.level, i, j, a.brk, thr, a.brk_cap);
        rst<T, M>(gDinv + j * MM, Dp);
        if (pt.hasL) {
            if (!first) {
                T t[MM];
                rmm<T, M, false, false>(t, Bj, Zp);
                rmm<T, M, true, false>(Zp, Dp, t);
            } else {
                rmm<T, M, true, false>(Zp, Dp, Bj);
            }
            rst<T, M>(gZ + j * MM, Zp);
        }
        if (needC) {
            T Cj[MM];
            rld<T, M>(Cj, a.C + (j - a.shift) * MM);
            rmm<T, M, false, false>(Yp, Dp, Cj);
            if (!ok && a.brk != nullptr) {
                // restart the local factorization at the next row after a breakdown
#pragma unroll
                for (int u = 0; u < MM; ++u) Yp[u] = T(0);
            }
            rst<T, M>(gY + j * MM, Yp);
        }
        if (wchain) {
            // CP += W_j Zc_j ;  W_{j+1} = -W_j Y_j  (zero after the last row without x_R)
            rmm<T, M, false, true>(CP, W, Zp);
            if (needC) {
                rmm<T, M, true, false>(W, W, Yp);
            } else {
#pragma unroll
                for (int u = 0; u < MM; ++u) W[u] = T(0);
            }
        }
    }
    if (MODE == 0) {
        if (!pt.hasL) return;
        rst<T, M>(reinterpret_cast<T*>(a.Pf) + i * MM, CP);
        rst<T, M>(reinterpret_cast<T*>(a.Qf) + i * MM, W);
    } else {
        const long long e = pt.e;
        T Be[MM];
        rld<T, M>(Be, a.B + (e - a.shift) * MM);
        double* Sn = a.Bn + i * MM;
        double* Rn = a.Dn + i * MM;
#pragma unroll
        for (int u = 0; u < MM; ++u) Rn[u] = a.D[(e - a.shift) * MM + u];
        if (pt.e > pt.s) {
            T t[MM];
            rmm<T, M, false, false>(t, Be, Zp);
            rst<T, M>(Sn, t);
        } else {
#pragma unroll
            for (int u = 0; u < MM; ++u) Sn[u] = a.B[(e - a.shift) * MM + u];
        }
    }
}

template <typename T, int M>
__device__ __forceinline__ void assemble_tp_body(const LevelArgs& a, const long long s) {
    constexpr int MM = M * M;
    if (s >= a.p - 1) return;
    const Part pt = part_bounds(a, 0, s);
    const long long e = pt.e;
    const bool local = pt.e > pt.s;   // partition s has local rows before its separator
    double Be[MM], al[MM], Pf[MM];
    rld<double, M>(Be, a.B + (e - a.shift) * MM);
    rld<double, M>(al, a.D + (e - a.shift) * MM);
    rld<double, M>(Pf, reinterpret_cast<const T*>(a.Pf) + (s + 1) * MM);
    if (local) {
        double Yl[MM];
        rld<double, M>(Yl, reinterpret_cast<const T*>(a.Y) + (e - 1) * MM);
        rmm<double, M, true, true>(al, Be, Yl);
    }
#pragma unroll
    for (int u = 0; u < MM; ++u) al[u] += Pf[u];
    rst<double, M>(a.Dn + s * MM, al);
    double be[MM], ga[MM];
#pragma unroll
    for (int u = 0; u < MM; ++u) be[u] = ga[u] = 0.0;
    if (s > 0 && local) {
        double Zl[MM];
        rld<double, M>(Zl, reinterpret_cast<const T*>(a.Zc) + (e - 1) * MM);
        rmm<double, M, false, false>(be, Be, Zl);
    } else if (s > 0) {
#pragma unroll
        for (int u = 0; u < MM; ++u) be[u] = Be[u];   // direct coupling to the previous separator
    }
    if (s + 1 < a.p - 1) rld<double, M>(ga, reinterpret_cast<const T*>(a.Qf) + (s + 1) * MM);
    rst<double, M>(a.Bn + s * MM, be);
    rst<double, M>(a.Cn + s * MM, ga);
}

// v (M) = sgn * A (M x M) x (M) (+ v if ACC)
template <typename T, int M, bool NEG, bool ACC>
__device__ __forceinline__ void rmv(T (&v)[M], const T (&A)[M * M], const T (&x)[M]) {
    T out[M];
#pragma unroll
    for (int r = 0; r < M; ++r) {
        T acc = ACC ? v[r] : T(0);
#pragma unroll
        for (int k = 0; k < M; ++k) acc = fmaT<T>(NEG ? -A[r * M + k] : A[r * M + k], x[k], acc);
        out[r] = acc;
    }
#pragma unroll
    for (int r = 0; r < M; ++r) v[r] = out[r];
}

template <int M, typename T>
__device__ __forceinline__ void vld(T (&v)[M], const double* g, int nr) {
#pragma unroll
    for (int r = 0; r < M; ++r) v[r] = (T)g[r * nr];
}
template <int M, typename T>
__device__ __forceinline__ void vst(double* g, const T (&v)[M], int nr) {
#pragma unroll
    for (int r = 0; r < M; ++r) g[r * nr] = (double)v[r];
}

template <typename T, int M, int MODE>
__device__ __forceinline__ void solve_fwd_tp_body(const LevelArgs& a, const long long tid) {
    constexpr int MM = M * M;
    if constexpr (M == 1 && MODE == 0) {
        if (a.nr == 1) {
            solve_fwd_tp_scalar<T>(a, tid);
            return;
        }
    }
    const int nr = a.nr;
    const long long i = tid / nr;
    const int c = (int)(tid % nr);
    if (i >= a.p) return;
    const Part pt = part_bounds(a, MODE, i);
    const long long E = (long long)M * nr;
    const T* gDinv = reinterpret_cast<const T*>(a.Dinv);
    T hp[M];
#pragma unroll
    for (int r = 0; r < M; ++r) hp[r] = T(0);
    for (long long j = pt.s; j < pt.e; ++j) {
        T v[M];
        vld<M, T>(v, a.F + j * E + c, nr);
        if (j != pt.s) {
            T Bj[MM];
            rld<T, M>(Bj, a.B + (j - a.shift) * MM);
            rmv<T, M, true, true>(v, Bj, hp);
        }
        T Di[MM];
        rld<T, M>(Di, gDinv + j * MM);
        rmv<T, M, false, false>(hp, Di, v);
        vst<M, T>(a.X + j * E + c, hp, nr);
    }
    if (MODE == 1) {
        const long long e = pt.e;
        if (i == 0) {
#pragma unroll
            for (int r = 0; r < M; ++r) a.Fn[r * nr + c] = a.F[r * nr + c];
        }
        double g[M];
        vld<M, double>(g, a.F + e * E + c, nr);
        if (pt.e > pt.s) {
            T Be[MM], t[M];
            rld<T, M>(Be, a.B + (e - a.shift) * MM);
            rmv<T, M, false, false>(t, Be, hp);
#pragma unroll
            for (int r = 0; r < M; ++r) g[r] -= (double)t[r];
        }
        vst<M, double>(a.Fn + (i + 1) * E + c, g, nr);
        return;
    }
    if (!pt.hasL) return;
    const T* gY = reinterpret_cast<const T*>(a.Y);
    for (long long j = pt.e - 2; j >= pt.s; --j) {
        T h[M], Yj[MM];
        vld<M, T>(h, a.X + j * E + c, nr);
        rld<T, M>(Yj, gY + j * MM);
        rmv<T, M, true, true>(h, Yj, hp);
#pragma unroll
        for (int r = 0; r < M; ++r) hp[r] = h[r];
    }
    T* Hf = reinterpret_cast<T*>(a.Hf) + i * E + c;
#pragma unroll
    for (int r = 0; r < M; ++r) Hf[r * nr] = hp[r];
}

template <typename T, int M>
__device__ __forceinline__ void assemble_rhs_tp_body(const LevelArgs& a, const long long tid) {
    constexpr int MM = M * M;
    const int nr = a.nr;
    const long long s = tid / nr;
    const int c = (int)(tid % nr);
    if (s >= a.p - 1) return;
    const Part pt = part_bounds(a, 0, s);
    const long long e = pt.e;
    const long long E = (long long)M * nr;
    double g[M], h[M], H[M], Be[MM], Ce[MM];
    vld<M, double>(g, a.F + e * E + c, nr);
    if (pt.e > pt.s) {
        vld<M, double>(h, a.X + (e - 1) * E + c, nr);
    } else {
#pragma unroll
        for (int r = 0; r < M; ++r) h[r] = 0.0;
    }
    const T* Hf = reinterpret_cast<const T*>(a.Hf) + (s + 1) * E + c;
#pragma unroll
    for (int r = 0; r < M; ++r) H[r] = (double)Hf[r * nr];
    rld<double, M>(Be, a.B + (e - a.shift) * MM);
    rld<double, M>(Ce, a.C + (e - a.shift) * MM);
    rmv<double, M, true, true>(g, Be, h);
    rmv<double, M, true, true>(g, Ce, H);
    vst<M, double>(a.Fn + s * E + c, g, nr);
}

template <typename T, int M, int MODE>
__device__ __forceinline__ void solve_bwd_tp_body(const LevelArgs& a, const long long tid) {
    constexpr int MM = M * M;
    if constexpr (M == 1 && MODE == 0) {
        if (a.nr == 1) {
            solve_bwd_tp_scalar<T>(a, tid);
            return;
        }
    }
    const int nr = a.nr;
    const long long i = tid / nr;
    const int c = (int)(tid % nr);
    if (i >= a.p) return;
    const Part pt = part_bounds(a, MODE, i);
    const long long E = (long long)M * nr;
    const long long li = (MODE == 0) ? i - 1 : i;
    const long long ri = (MODE == 0) ? i : i + 1;
    T x[M], xl[M];
#pragma unroll
    for (int r = 0; r < M; ++r) {
        x[r] = T(0);
        xl[r] = T(0);
    }
    if (pt.hasR) {
        double xr[M];
        vld<M, double>(xr, a.Xn + ri * E + c, nr);
        vst<M, double>(a.X + pt.e * E + c, xr, nr);
#pragma unroll
        for (int r = 0; r < M; ++r) x[r] = (T)xr[r];
    }
    if (MODE == 1 && i == 0) {
#pragma unroll
        for (int r = 0; r < M; ++r) a.X[r * nr + c] = a.Xn[r * nr + c];
    }
    if (pt.hasL) vld<M, T>(xl, a.Xn + li * E + c, nr);
    const T* gY = reinterpret_cast<const T*>(a.Y);
    const T* gZ = reinterpret_cast<const T*>(a.Zc);
    for (long long j = pt.e - 1; j >= pt.s; --j) {
        T v[M];
        vld<M, T>(v, a.X + j * E + c, nr);
        if (MODE == 0 && ((j < pt.e - 1) || pt.hasR)) {
            T Yj[MM];
            rld<T, M>(Yj, gY + j * MM);
            rmv<T, M, true, true>(v, Yj, x);
        }
        if (pt.hasL) {
            T Zj[MM];
            rld<T, M>(Zj, gZ + j * MM);
            rmv<T, M, false, true>(v, Zj, xl);
        }
#pragma unroll
        for (int r = 0; r < M; ++r) x[r] = v[r];
        vst<M, T>(a.X + j * E + c, x, nr);
    }
}

// ---------------------------------------------------------------- wrappers --
// Single system: global thread t handles unit t (partition, separator or
// (partition, rhs) pair).  Batched (persistent, grid-stride): item w of the
// work list is (system, unit).
#define BT_TP_KERNELS(NAME, BODY, TPL, TARGS)                                                           \
    template <TPL>                                                                                     \
    __global__ void __launch_bounds__(256) NAME(const LevelArgs a) {                                   \
        const long long u = a.unit0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;               \
        if (a.unit_end > 0 && u >= a.unit_end) return;                                                 \
        BODY<TARGS>(a, u);                                                                             \
    }                                                                                                  \
    template <TPL>                                                                                     \
    __global__ void __launch_bounds__(256)                                                             \
        NAME##_batch(const LevelArgs* __restrict__ args, const int2* __restrict__ work, int nwork) {   \
        for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nwork; w += gridDim.x * blockDim.x) {  \
            const int2 it = work[w];                                                                   \
            BODY<TARGS>(args[it.x], (long long)it.y);                                                   \
        }                                                                                              \
    }

#define BT_TP_COMMA ,
BT_TP_KERNELS(k_factor_tp, factor_tp_body, typename T BT_TP_COMMA int M BT_TP_COMMA int MODE, T BT_TP_COMMA M BT_TP_COMMA MODE)
BT_TP_KERNELS(k_assemble_tp, assemble_tp_body, typename T BT_TP_COMMA int M, T BT_TP_COMMA M)
BT_TP_KERNELS(k_solve_fwd_tp, solve_fwd_tp_body, typename T BT_TP_COMMA int M BT_TP_COMMA int MODE, T BT_TP_COMMA M BT_TP_COMMA MODE)
BT_TP_KERNELS(k_assemble_rhs_tp, assemble_rhs_tp_body, typename T BT_TP_COMMA int M, T BT_TP_COMMA M)
BT_TP_KERNELS(k_solve_bwd_tp, solve_bwd_tp_body, typename T BT_TP_COMMA int M BT_TP_COMMA int MODE, T BT_TP_COMMA M BT_TP_COMMA MODE)

}  // namespace bt
