// Device-side helpers shared by the partition-method kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "bt_level.h"

namespace bt {

enum : int { ST_OK = 0, ST_SINGULAR = 3, ST_NONFINITE = 4, ST_TIMEOUT = 6 };

// Status word (4 x int64): [0] code, [1] level, [2] partition, [3] block row.
// The first error wins; later ones are dropped.
__device__ __forceinline__ void report(long long* st, int code, long long level, long long part,
                                       long long row) {
    if (st == nullptr) return;
    if (atomicCAS(reinterpret_cast<unsigned long long*>(st), 0ull, (unsigned long long)code) == 0ull) {
        st[1] = level;
        st[2] = part;
        st[3] = row;
    }
}

// 1/x.  A hardware reciprocal seed r0 (rcp.approx.ftz.f64, relative error
// below 2^-19 over the normal range) refined by one third-order Newton step,
// r = r0 (1 + e + e^2) with e = 1 - x r0, i.e. the geometric series of
// 1/(1 - e) truncated after e^2 (relative error about e^3 before the final
// rounding).  Zero, subnormal, huge (1/x subnormal) and non-finite x take the
// IEEE division.
__device__ __forceinline__ double rcp(double x) {
    const int ex = (__double2hiint(x) >> 20) & 0x7ff;
    if (ex < 1 || ex > 2044) return 1.0 / x;
    double r0;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r0) : "d"(x));
    const double e = fma(-x, r0, 1.0);
    const double t = fma(e, e, e);
    return fma(r0, t, r0);
}
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }

// Append block row `row` to a breakdown list: brk[0] counts, brk[1..cap] hold
// the rows (a row may appear more than once; entries past cap are dropped and
// found again by the next factorization pass).
__device__ __forceinline__ void record_breakdown(long long* brk, long long cap, long long row) {
    const unsigned long long k = atomicAdd(reinterpret_cast<unsigned long long*>(brk), 1ull);
    if ((long long)k < cap) brk[1 + k] = row;
}

// |x| as an integer key that orders like |x| for finite x (sign bit cleared).
__device__ __forceinline__ unsigned long long abs_key(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long abs_key(float x) {
    return (unsigned long long)(__float_as_uint(x) & 0x7fffffffu);
}
// The magnitude back from abs_key.
template <typename T>
__device__ __forceinline__ T key_abs(unsigned long long k);
template <>
__device__ __forceinline__ double key_abs<double>(unsigned long long k) {
    return __longlong_as_double((long long)k);
}
template <>
__device__ __forceinline__ float key_abs<float>(unsigned long long k) {
    return __uint_as_float((unsigned)k);
}
__device__ __forceinline__ bool nonfinite(double x) {
    return ((__double2hiint(x) >> 20) & 0x7ff) == 0x7ff;
}
__device__ __forceinline__ bool nonfinite(float x) {
    return ((__float_as_uint(x) >> 23) & 0xff) == 0xff;
}

template <typename T> __device__ __forceinline__ T fmaT(T a, T b, T c);
template <> __device__ __forceinline__ double fmaT<double>(double a, double b, double c) { return fma(a, b, c); }
template <> __device__ __forceinline__ float fmaT<float>(float a, float b, float c) { return fmaf(a, b, c); }

// ---------------------------------------------------------------- geometry --
// Block-tridiagonal level (mode 0): rows 0..N-1 in p partitions; partition i
// owns base + (i < extra) rows, its last row is the separator for i < p-1.
// BABD level (mode 1): rows 0..N; rows 1..N-1 are split the same way, the
// separators are row 0, the last row of partitions 0..p-2, and row N.
struct Part {
    long long s, e;   // local rows [s, e); e is the right separator row if hasR
    bool hasL, hasR;
};

__device__ __forceinline__ Part part_bounds(int mode, long long N, long long p, long long base,
                                            long long extra, long long i) {
    Part q;
    const long long cnt = base + (i < extra ? 1 : 0);
    const long long start = i * base + (i < extra ? i : extra);
    if (mode == 0) {
        q.s = start;
        q.hasL = i > 0;
        q.hasR = i < p - 1;
        q.e = q.hasR ? start + cnt - 1 : start + cnt;
    } else {
        q.s = 1 + start;
        q.hasL = true;
        q.hasR = true;
        q.e = (i < p - 1) ? q.s + cnt - 1 : N;
    }
    return q;
}

// Bounds of partition i of a level: explicit starts (pivoted levels, where a
// partition may have no local rows: only its separator, or nothing at the end)
// or the uniform split.
__device__ __forceinline__ Part part_bounds(const LevelArgs& a, int mode, long long i) {
    if (a.starts != nullptr) {
        Part q;
        const long long start = a.starts[i], cnt = a.starts[i + 1] - start;
        q.s = start;
        q.hasL = i > 0;
        q.hasR = i < a.p - 1;
        q.e = q.hasR ? start + cnt - 1 : start + cnt;
        return q;
    }
    return part_bounds(mode, a.N, a.p, a.base, a.extra, i);
}

}  // namespace bt
