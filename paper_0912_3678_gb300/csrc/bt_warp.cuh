// Warp-per-partition local factorization in FP32 for blocks of order 16 (the
// low-precision local factors of the refined paths, Sec. 2 LU variant,
// Eqs. (parfact)-(parblock), with each pivot block inverted by Gauss-Jordan
// elimination with partial pivoting inside the block).
//
// One warp owns one partition.  Every block row j applies Gauss-Jordan
// elimination to the augmented 16 x 64 matrix
//     [ D'_j | C_j | T_j | I ]  ->  [ I | Y_j | Zc_j | D'_j^{-1} ],
//     D'_j = D_j - B_j Y_{j-1},   T_j = -B_j Zc_{j-1}  (T_s = -B_s),
// so the upper factor Y_j = D'_j^{-1} C_j, the left spike Zc_j and the
// inverse come out of one elimination.  Lane r (r < 16) holds row r of
// [D'|C], lane 16 + r row r of [T|I]; a column of D' lies across lanes 0-15,
// so the pivot of step k is one redux over 32-bit magnitude keys, and rows
// are never swapped: the pivot row of step k is only broadcast (through
// shared memory) and every other row eliminates against it.  Row r ends as
// the pivot row of some step k_r with pivot d_r, which makes it row k_r of
// the result after division by d_r.  No CTA barrier is involved: the warp
// synchronises with __syncwarp only.
//
// The left separator's coupling to the top row (needed by its reduced row,
// Eq. (parblock)) runs as the forward chain W_s = C_{s-1},
// Pf = sum_j W_j Zc_j, W_{j+1} = -W_j Y_j, Qf = W_e, fused with the next
// row's Schur product (both read the rows of Y_{j-1} and Zc_{j-1} once).
// Input block rows (FP64) are staged into shared memory with cp.async,
// one row ahead, and converted to FP32 by integer operations; the block
// products and the elimination updates run on paired FP32 FMAs (FFMA2).  The
// factorization also leaves the split copy of the matrix for the refinement
// residual and the forward solve: negated FP32 (hi, lo) parts by column
// pairs, (-hi_k, -hi_k+1, -lo_k, -lo_k+1) for even k, 16 bytes.
#pragma once
#include "bt_bcr.cuh"
#include "bt_misc.h"

namespace bt {

struct WarpF16 {
    static constexpr int M = 16;
    static constexpr int WARPS = 4;    // partitions (warps) per CTA
    static constexpr int SR = 18;      // row stride of the FP64 staging blocks (doubles, 144 bytes)
    static constexpr int FR = 20;      // row stride of the FP32 blocks (floats, 80 bytes)
    struct Smem {
        double stage[2][3][M * SR];    // B, D, C of two block rows (FP64)
        float cv[3][M * FR];           // B, D, C of the current row (FP32)
        float ex[2][M * FR];           // rows of Y_{j-1} (0) and Zc_{j-1} (1), by row index
        float prow[2][2][2 * M + 4];   // pivot row of step k (parity k & 1), both halves
    };
};

// 1/x from the hardware approximation (relative error below 2^-22): the
// local factors are FP32 approximations that refinement corrects.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Stage one 16 x 16 FP64 block (2 KB, 16-byte aligned) into a padded shared block:
// 4 copies of 16 bytes per lane, each instruction covering 512 contiguous bytes.
__device__ __forceinline__ void stage_blk16(double* dst, const double* src, int lane) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int g = q * 32 + lane, rr = g >> 3, cc = (g & 7) * 2;
        cp_async16(dst + rr * WarpF16::SR + cc, src + rr * 16 + cc);
    }
}

// FP64 staging block -> FP32 block (zeros when absent): lane l converts row
// l / 2, columns (l % 2) * 8 .. + 7.  With gs (the block's place in the split
// copy of the matrix) the (hi, lo) pairs of the present entries are stored too.
__device__ __forceinline__ void convert_blk16(float* dst, const double* src, bool present, int lane,
                                              float2* gs = nullptr) {
    const int rr = lane >> 1, c0 = (lane & 1) * 8;
    float o[8];
    if (present) {
        const double2* s = reinterpret_cast<const double2*>(src + rr * WarpF16::SR + c0);
        float2 sp[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double2 v = s[q];
            sp[2 * q] = split_f64(v.x);
            sp[2 * q + 1] = split_f64(v.y);
            o[2 * q] = sp[2 * q].x;
            o[2 * q + 1] = sp[2 * q + 1].x;
        }
        if (gs != nullptr) {
            // the split copy, negated, by column pairs: (-hi_k, -hi_k+1, -lo_k, -lo_k+1), k even
            float4* g4 = reinterpret_cast<float4*>(gs + rr * 16 + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                g4[q] = make_float4(-sp[2 * q].x, -sp[2 * q + 1].x, -sp[2 * q].y, -sp[2 * q + 1].y);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) o[q] = 0.f;
    }
    float4* d = reinterpret_cast<float4*>(dst + rr * WarpF16::FR + c0);
    d[0] = make_float4(o[0], o[1], o[2], o[3]);
    d[1] = make_float4(o[4], o[5], o[6], o[7]);
}

__device__ __forceinline__ void read_row16(float (&v)[16], const float* s) {
    const float4* p = reinterpret_cast<const float4*>(s);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 t = p[q];
        v[4 * q] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
    }
}
__device__ __forceinline__ void write_row16(float* s, const float* v) {
    float4* p = reinterpret_cast<float4*>(s);
#pragma unroll
    for (int q = 0; q < 4; ++q) p[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// Block tridiagonal level (mode 0), FP32 factors: partition i of the level.
__device__ __forceinline__ void factor_warp16_body(const LevelArgs& a, const long long i, WarpF16::Smem& sm) {
    constexpr int M = 16;
    constexpr int FR = WarpF16::FR;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, h = lane >> 4, r = lane & 15;
    const Part pt = part_bounds(a, 0, i);
    const long long MM = M * M;
    float* gDinv = reinterpret_cast<float*>(a.Dinv);
    float* gY = reinterpret_cast<float*>(a.Y);
    float* gZ = reinterpret_cast<float*>(a.Zc);
    const bool hasL = pt.hasL;
    auto needB = [&](long long j) { return j > pt.s || hasL; };
    auto needC = [&](long long j) { return (j < pt.e - 1) || pt.hasR; };
    long long jb = pt.s, je = pt.e;
    if (a.phases > 1) {
        const long long cnt = pt.e - pt.s;
        jb = pt.s + cnt * a.phase / a.phases;
        je = pt.s + cnt * (a.phase + 1) / a.phases;
    }
    auto issue = [&](long long j, int buf) {
        const long long o = (j - a.shift) * MM;
        if (needB(j)) stage_blk16(sm.stage[buf][0], a.B + o, lane);
        stage_blk16(sm.stage[buf][1], a.D + o, lane);
        if (needC(j)) stage_blk16(sm.stage[buf][2], a.C + o, lane);
        cp_async_commit();
    };

    float w[16], cp[16];   // W_j row r (both halves); sum_j W_j Zc_j row r (upper half)
#pragma unroll
    for (int c = 0; c < 16; ++c) cp[c] = 0.f;
    bool wpend = false;    // the W step of the previous row is still to be taken
    float amax_run = 0.f;  // largest row sum of |A| over this partition's rows (lanes 0-15)
    if (jb < je) issue(jb, 0);
    if (jb > pt.s) {
        // a later phase: resume from the stored Y_{jb-1}, Zc_{jb-1} and the running W, Pf
        const float* yb = gY + (jb - 1) * MM;
        const float* zb = gZ + (jb - 1) * MM;
        float v[16];
        read_row16(v, (h == 0) ? yb + r * M : zb + r * M);
        if (h == 1 && !hasL) {
#pragma unroll
            for (int c = 0; c < 16; ++c) v[c] = 0.f;
        }
        write_row16(&sm.ex[h][r * FR], v);
        if (hasL) {
            read_row16(w, reinterpret_cast<const float*>(a.Qf) + i * MM + r * M);
            read_row16(cp, reinterpret_cast<const float*>(a.Pf) + i * MM + r * M);
        }
    } else if (hasL) {
        // W_s = C of the left separator row
        const double* cs = a.C + (pt.s - 1 - a.shift) * MM + r * M;
#pragma unroll
        for (int c = 0; c < 16; ++c) w[c] = trunc_f32(cs[c]);
    }
    if (!hasL) {
#pragma unroll
        for (int c = 0; c < 16; ++c) w[c] = 0.f;
    }

    for (long long j = jb; j < je; ++j) {
        const int buf = (int)((j - jb) & 1);
        if (j + 1 < je) issue(j + 1, buf ^ 1);
        else cp_async_commit();
        cp_async_wait<1>();
        __syncwarp();
        const bool hB = needB(j), hC = needC(j);
        float2* gsp = reinterpret_cast<float2*>(a.As);
        const long long rows = a.N;
        convert_blk16(sm.cv[0], sm.stage[buf][0], hB, lane, gsp ? gsp + (0 * rows + j) * MM : nullptr);
        convert_blk16(sm.cv[1], sm.stage[buf][1], true, lane, gsp ? gsp + (1 * rows + j) * MM : nullptr);
        convert_blk16(sm.cv[2], sm.stage[buf][2], hC, lane, gsp ? gsp + (2 * rows + j) * MM : nullptr);
        __syncwarp();
        float bro[16], a32[32];
        read_row16(bro, &sm.cv[0][r * FR]);
        if (h == 0) {
            float t[16];
            read_row16(t, &sm.cv[1][r * FR]);
#pragma unroll
            for (int c = 0; c < 16; ++c) a32[c] = t[c];
            read_row16(t, &sm.cv[2][r * FR]);
#pragma unroll
            for (int c = 0; c < 16; ++c) a32[16 + c] = t[c];
            if (a.amax != nullptr) {
                // row r of block row j of A (entries truncated toward zero): |B| + |D| + |C|
                float rs = 0.f;
#pragma unroll
                for (int c = 0; c < 16; ++c) rs += fabsf(bro[c]) + fabsf(a32[c]) + fabsf(a32[16 + c]);
                amax_run = fmaxf(amax_run, rs);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                a32[c] = 0.f;
                a32[16 + c] = (c == r) ? 1.f : 0.f;
            }
        }
        if (j > pt.s) {
            // D'_j = D_j - B_j Y_{j-1} (lower half), T_j = -B_j Zc_{j-1} (upper half), and the
            // pending W step: W_j = -W_{j-1} Y_{j-1}, Pf += W_{j-1} Zc_{j-1}
            float acc[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[c] = 0.f;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                float srow[16];
                read_row16(srow, &sm.ex[h][k * FR]);
                const float2 nb = make_float2(-bro[k], -bro[k]), wk = make_float2(w[k], w[k]);
#pragma unroll
                for (int c = 0; c < 16; c += 2) {
                    // paired FMAs (FFMA2): each component is the scalar fmaf
                    const float2 sv = make_float2(srow[c], srow[c + 1]);
                    const float2 t = __ffma2_rn(nb, sv, make_float2(a32[c], a32[c + 1]));
                    const float2 u = __ffma2_rn(wk, sv, make_float2(acc[c], acc[c + 1]));
                    a32[c] = t.x;
                    a32[c + 1] = t.y;
                    acc[c] = u.x;
                    acc[c + 1] = u.y;
                }
            }
            if (wpend) {
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const float wn = __shfl_sync(FULL, -acc[c], r);
                    if (h == 1) cp[c] += acc[c];
                    w[c] = wn;
                }
            }
        } else if (h == 1 && hasL) {
#pragma unroll
            for (int c = 0; c < 16; ++c) a32[c] = -bro[c];   // T_s = -B_s
        }
        if (hasL && h == 0 && a.W != nullptr) write_row16(reinterpret_cast<float*>(a.W) + j * MM + r * M, w);
        __syncwarp();   // every lane has read ex before it is rewritten below

        // Gauss-Jordan elimination without row interchanges
        int bad = 0;
        bool used = false;
        float dsave = 1.f;
        int kpos = 0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const unsigned key = (h == 0 && !used) ? ((mag_key<float>(a32[k]) << 5) | (unsigned)(31 - lane)) : 0u;
            const unsigned best = __reduce_max_sync(FULL, key);
            const int p = 31 - (int)(best & 31u);
            float piv = __shfl_sync(FULL, a32[k], p);
            const float colk = __shfl_sync(FULL, a32[k], r);
            // a zero (or subnormal: its reciprocal overflows FP32) or non-finite
            // pivot is reported after the elimination (the first such step wins)
            // and replaced by 1 to keep going
            const unsigned pe = (__float_as_uint(piv) >> 23) & 0xffu;
            const int flag = (pe == 0xffu) ? ST_NONFINITE : (pe == 0u ? ST_SINGULAR : 0);
            bad = bad ? bad : flag;
            piv = flag ? 1.f : piv;
            const float rp = rcp_approx(piv);
            const bool mine = (r == p);
            const float l = mine ? 0.f : colk * rp;
            float* pb = sm.prow[k & 1][h];
            if (mine) {
                float4* d = reinterpret_cast<float4*>(pb);
#pragma unroll
                for (int q = 0; q < 8; ++q) d[q] = make_float4(a32[4 * q], a32[4 * q + 1], a32[4 * q + 2], a32[4 * q + 3]);
            }
            __syncwarp();
            const float4* s = reinterpret_cast<const float4*>(pb);
            const float2 nl = make_float2(-l, -l);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 t = s[q];
                const float2 u0 = __ffma2_rn(nl, make_float2(t.x, t.y), make_float2(a32[4 * q], a32[4 * q + 1]));
                const float2 u1 = __ffma2_rn(nl, make_float2(t.z, t.w), make_float2(a32[4 * q + 2], a32[4 * q + 3]));
                a32[4 * q] = u0.x;
                a32[4 * q + 1] = u0.y;
                a32[4 * q + 2] = u1.x;
                a32[4 * q + 3] = u1.y;
            }
            if (mine) {
                used = true;
                dsave = piv;
                kpos = k;
            }
        }
        if (bad && lane == 0) report(a.status, bad, a.level, i, j);
        // row r is row kpos of [I | Y | Zc | D'^{-1}] after division by its pivot
        const float sc = rcp_approx(dsave);
        if (h == 0) {
            float y[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) y[c] = a32[16 + c] * sc;
            if (hC) write_row16(gY + j * MM + kpos * M, y);
            write_row16(&sm.ex[0][kpos * FR], y);
        } else {
            float z[16], di[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                z[c] = a32[c] * sc;
                di[c] = a32[16 + c] * sc;
            }
            write_row16(gDinv + j * MM + kpos * M, di);
            if (hasL) write_row16(gZ + j * MM + kpos * M, z);
            write_row16(&sm.ex[1][kpos * FR], z);
        }
        wpend = hasL;
        __syncwarp();
    }
    cp_async_wait<0>();
    if (a.As != nullptr && pt.hasR && (a.phases <= 1 || a.phase == a.phases - 1)) {
        // the split copy also holds the right separator row e (read only by the residual)
        const long long e = pt.e, o = (e - a.shift) * MM;
        __syncwarp();
        stage_blk16(sm.stage[0][0], a.B + o, lane);
        stage_blk16(sm.stage[0][1], a.D + o, lane);
        stage_blk16(sm.stage[0][2], a.C + o, lane);
        cp_async_commit();
        cp_async_wait<0>();
        __syncwarp();
        float2* gsp = reinterpret_cast<float2*>(a.As);
        for (int w = 0; w < 3; ++w) convert_blk16(sm.cv[w], sm.stage[0][w], true, lane, gsp + (w * a.N + e) * MM);
        __syncwarp();
        if (a.amax != nullptr && h == 0) {
            float t0[16], t1[16], t2[16];
            read_row16(t0, &sm.cv[0][r * FR]);
            read_row16(t1, &sm.cv[1][r * FR]);
            read_row16(t2, &sm.cv[2][r * FR]);
            float rs = 0.f;
#pragma unroll
            for (int c = 0; c < 16; ++c) rs += fabsf(t0[c]) + fabsf(t1[c]) + fabsf(t2[c]);
            amax_run = fmaxf(amax_run, rs);
        }
        __syncwarp();
    }
    if (a.amax != nullptr) {
        // as a double bit pattern, like the residual maxima slots
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) amax_run = fmaxf(amax_run, __shfl_xor_sync(FULL, amax_run, off));
        if (lane == 0) {
            const unsigned u = __float_as_uint(amax_run);
            const unsigned e8 = (u >> 23) & 0xffu;
            const unsigned long long bits =
                (e8 == 0u) ? 0ull : (((unsigned long long)(e8 + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29));
            atomicMax(a.amax + 3 * ((blockIdx.x * WarpF16::WARPS + (threadIdx.x >> 5)) % kMaxSlots), bits);
        }
    }
    if (!hasL) return;
    if (wpend) {
        // the W step of the last row: Pf += W Zc_{je-1}, W_{je} = -W Y_{je-1}
        float acc[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float srow[16];
            read_row16(srow, &sm.ex[h][k * FR]);
            const float wk = w[k];
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[c] = fmaf(wk, srow[c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const float wn = __shfl_sync(FULL, -acc[c], r);
            if (h == 1) cp[c] += acc[c];
            w[c] = wn;
        }
    }
    // final: C_sep P_first (Pf) and W_e (Qf); between phases: the running sum and W
    if (h == 1) write_row16(reinterpret_cast<float*>(a.Pf) + i * MM + r * M, cp);
    else write_row16(reinterpret_cast<float*>(a.Qf) + i * MM + r * M, w);
}

template <int MODE>
__global__ void __launch_bounds__(32 * WarpF16::WARPS) k_factor_w16(const LevelArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    WarpF16::Smem& sm = reinterpret_cast<WarpF16::Smem*>(smem_raw)[warp];
    const long long u = a.unit0 + (long long)blockIdx.x * WarpF16::WARPS + warp;
    const long long end = (a.unit_end > 0) ? a.unit_end : a.p;
    if (u >= end) return;
    factor_warp16_body(a, u, sm);
}

constexpr size_t factor_w16_smem_bytes() { return sizeof(WarpF16::Smem) * WarpF16::WARPS; }

// ---------------------------------------------------------------- solves --
// Forward and back substitution with the warp kernel's FP32 factors, one warp
// per partition (block tridiagonal, order 16).  Lane (r, hc) holds entry r of
// right-hand-side columns hc*NH .. hc*NH + NH - 1 of each block row; block
// products take the other rows from a shared exchange row (broadcast loads).
//   forward   h_s = D'^{-1}_s f_s,  h_j = D'^{-1}_j (f_j - B_j h_{j-1}),
//             Hw  = sum_j W_j h_j              (the left separator's coupling),
//             g_e = f_e - B_e h_{e-1}          (right separator, partial:
//                                               k_sep_rhs_w16 subtracts Hw of the next partition)
//   backward  x_j = h_j + Zc_j x_L - Y_j x_{j+1}.
template <int NH>
struct WarpS16 {
    static constexpr int M = 16;
    static constexpr int WARPS = 4;
    static constexpr int SW = 2 * NH + 4;   // exchange row stride (floats)
    static constexpr int S = 4;             // block rows in flight (copy ring depth)
    static constexpr int NRMAX = 2 * NH;    // right-hand sides the variant takes
    struct alignas(16) Smem {
        double sB[S][M * WarpF16::SR];       // forward: B_j (FP64)
        float sA[S][M * M];                  // forward: D'^{-1}_j; backward: Y_j
        float sC[S][M * M];                  // forward: W_j; backward: Zc_j
        double sV[S][M * NRMAX];             // forward: f_j; backward: X_j (update form)
        float sH[S][M * NRMAX];              // backward: h_j
        float xa[M * SW];                    // exchange row: h_{j-1}, t_j, or x_{j+1}
        float xb[M * SW];                    // exchange row: h_j, or x_L
    };
};

// Copies of one block row's operands into ring slot b (every lane takes a
// share; 16-byte copies for the 16 x 16 blocks, 8-byte copies for the
// right-hand-side rows, whose base need not be 16-byte aligned).
__device__ __forceinline__ void ring_blk32(float* dst, const float* src, int lane) {
#pragma unroll
    for (int q = 0; q < 2; ++q) cp_async16(dst + 4 * (q * 32 + lane), src + 4 * (q * 32 + lane));
}
__device__ __forceinline__ void ring_vec64(double* dst, const double* src, int n, int lane) {
    for (int e = lane; e < n; e += 32) cp_async8(dst + e, src + e);
}
__device__ __forceinline__ void ring_vec32(float* dst, const float* src, int n, int lane) {
    // n floats, n a multiple of 4 (16 nr), src 16-byte aligned
    for (int e = lane; e < n / 4; e += 32) cp_async16(dst + 4 * e, src + 4 * e);
}

template <int NH>
__device__ __forceinline__ void load_vec(float (&v)[NH], const double* g, int cbase, int nr) {
#pragma unroll
    for (int q = 0; q < NH; ++q) v[q] = (cbase + q < nr) ? trunc_f32(g[cbase + q]) : 0.f;
}
template <int NH>
__device__ __forceinline__ void put_vec(float* s, const float (&v)[NH]) {
#pragma unroll
    for (int q = 0; q < NH; q += 4) *reinterpret_cast<float4*>(s + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
}
// acc[q] += sgn * sum_k A[k] X[k][q]  (A: 16 coefficients in registers; X rows in shared memory)
template <int NH, bool NEG>
__device__ __forceinline__ void gemv_acc(float (&acc)[NH], const float (&A)[16], const float* X, int stride) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const float ak = NEG ? -A[k] : A[k];
#pragma unroll
        for (int q = 0; q < NH; q += 4) {
            const float4 x = *reinterpret_cast<const float4*>(X + k * stride + q);
            acc[q] = fmaf(ak, x.x, acc[q]);
            acc[q + 1] = fmaf(ak, x.y, acc[q + 1]);
            acc[q + 2] = fmaf(ak, x.z, acc[q + 2]);
            acc[q + 3] = fmaf(ak, x.w, acc[q + 3]);
        }
    }
}
__device__ __forceinline__ void load_row16(float (&v)[16], const float* g) { read_row16(v, g); }

template <int NH>
__device__ __forceinline__ void solve_fwd_w16_body(const LevelArgs& a, const long long i,
                                                   typename WarpS16<NH>::Smem& sm) {
    using WS = WarpS16<NH>;
    constexpr int M = 16, SW = WS::SW, S = WS::S;
    const int lane = threadIdx.x & 31, r = lane & 15, hc = lane >> 4;
    const int nr = a.nr, E = M * nr, cb = hc * NH;
    const Part pt = part_bounds(a, 0, i);
    const long long MM = M * M;
    const float* gDi = reinterpret_cast<const float*>(a.Dinv);
    const float* gW = reinterpret_cast<const float*>(a.W);
    float* gH = reinterpret_cast<float*>(a.Hv);
    // B_j truncated to FP32: the (negated) high parts of the factorization's
    // split copy when there is one (2 KB per block, as the FP64 block), else
    // converted here
    const float2* gBs = reinterpret_cast<const float2*>(a.As);
    float* xa = sm.xa + r * SW + cb;
    float* xb = sm.xb + r * SW + cb;
    float acc[NH];
#pragma unroll
    for (int q = 0; q < NH; ++q) acc[q] = 0.f;
    // operands of local row s + t go to ring slot t % S, S - 1 rows ahead of use
    auto issue = [&](long long t) {
        const long long j = pt.s + t;
        if (j < pt.e) {
            const int b = (int)(t % S);
            if (j > pt.s)
                stage_blk16(sm.sB[b], gBs ? reinterpret_cast<const double*>(gBs + j * MM) : a.B + (j - a.shift) * MM,
                            lane);
            ring_blk32(sm.sA[b], gDi + j * MM, lane);
            if (pt.hasL) ring_blk32(sm.sC[b], gW + j * MM, lane);
            ring_vec64(sm.sV[b], a.F + j * E, E, lane);
        }
        cp_async_commit();   // one group per row, empty past the end
    };
    const long long n = pt.e - pt.s;
#pragma unroll
    for (int t = 0; t < S - 1; ++t) issue(t);
    for (long long t = 0; t < n; ++t) {
        const long long j = pt.s + t;
        const int b = (int)(t % S);
        cp_async_wait<S - 2>();
        __syncwarp();
        issue(t + S - 1);    // into the slot row t - 1 used
        float t4[NH];
#pragma unroll
        for (int q = 0; q < NH; ++q) t4[q] = (cb + q < nr) ? __double2float_rz(sm.sV[b][r * nr + cb + q]) : 0.f;
        if (j > pt.s) {
            // t = f_j - B_j h_{j-1}  (h_{j-1} in xb)
            float Br[16];
            const double* sbr = sm.sB[b] + r * WarpF16::SR;
            if (gBs) {
                // -B_j row r: entry k at float (k / 2) * 4 + k % 2 of the row
                const float4* sp = reinterpret_cast<const float4*>(sbr);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 v = sp[q];
                    Br[2 * q] = v.x;
                    Br[2 * q + 1] = v.y;
                }
                gemv_acc<NH, false>(t4, Br, sm.xb + cb, SW);
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k) Br[k] = trunc_f32(sbr[k]);
                gemv_acc<NH, true>(t4, Br, sm.xb + cb, SW);
            }
        }
        put_vec<NH>(xa, t4);
        __syncwarp();
        float Di[16], h[NH];
        read_row16(Di, sm.sA[b] + r * M);
#pragma unroll
        for (int q = 0; q < NH; ++q) h[q] = 0.f;
        gemv_acc<NH, false>(h, Di, sm.xa + cb, SW);
        __syncwarp();          // xb (h_{j-1}) and xa (t) fully read
        put_vec<NH>(xb, h);
#pragma unroll
        for (int q = 0; q < NH; ++q)
            if (cb + q < nr) gH[j * E + r * nr + cb + q] = h[q];
        __syncwarp();
        if (pt.hasL) {
            float Wr[16];
            read_row16(Wr, sm.sC[b] + r * M);
            gemv_acc<NH, false>(acc, Wr, sm.xb + cb, SW);
        }
        __syncwarp();          // slot b is refilled by the next iteration
    }
    cp_async_wait<0>();
    __syncwarp();
    if (pt.hasL) {
        float* hw = reinterpret_cast<float*>(a.Hw) + i * E + r * nr;
#pragma unroll
        for (int q = 0; q < NH; ++q)
            if (cb + q < nr) hw[cb + q] = acc[q];
    }
    if (pt.hasR) {
        // partial reduced right-hand side of the right separator e: f_e - B_e h_{e-1}
        const long long e = pt.e;
        float g[NH], Br[16];
        load_vec<NH>(g, a.F + (e * M + r) * nr, cb, nr);
        if (pt.e > pt.s) {
            if (gBs) {
                const float4* be = reinterpret_cast<const float4*>(gBs + e * MM + r * M);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 v = be[q];
                    Br[2 * q] = v.x;
                    Br[2 * q + 1] = v.y;
                }
                gemv_acc<NH, false>(g, Br, sm.xb + cb, SW);
            } else {
                const double* be = a.B + (e - a.shift) * MM + r * M;
#pragma unroll
                for (int k = 0; k < 16; ++k) Br[k] = trunc_f32(be[k]);
                gemv_acc<NH, true>(g, Br, sm.xb + cb, SW);
            }
        }
        double* fn = a.Fn + i * E + r * nr;
#pragma unroll
        for (int q = 0; q < NH; ++q)
            if (cb + q < nr) fn[cb + q] = (double)g[q];
    }
}

template <int NH>
__device__ __forceinline__ void solve_bwd_w16_body(const LevelArgs& a, const long long i,
                                                   typename WarpS16<NH>::Smem& sm) {
    using WS = WarpS16<NH>;
    constexpr int M = 16, SW = WS::SW, S = WS::S;
    const int lane = threadIdx.x & 31, r = lane & 15, hc = lane >> 4;
    const int nr = a.nr, E = M * nr, cb = hc * NH;
    const Part pt = part_bounds(a, 0, i);
    const long long MM = M * M;
    const float* gY = reinterpret_cast<const float*>(a.Y);
    const float* gZ = reinterpret_cast<const float*>(a.Zc);
    const float* gH = reinterpret_cast<const float*>(a.Hv);
    float* xa = sm.xa + r * SW + cb;   // x_{j+1}
    float* xb = sm.xb + r * SW + cb;   // x_L
    auto useY = [&](long long j) { return (j < pt.e - 1) || pt.hasR; };
    // operands of local row e - 1 - t go to ring slot t % S, S - 1 rows ahead of use
    auto issue = [&](long long t) {
        const long long j = pt.e - 1 - t;
        if (j >= pt.s) {
            const int b = (int)(t % S);
            if (useY(j)) ring_blk32(sm.sA[b], gY + j * MM, lane);
            if (pt.hasL) ring_blk32(sm.sC[b], gZ + j * MM, lane);
            ring_vec32(sm.sH[b], gH + j * E, E, lane);
            if (a.accum) ring_vec64(sm.sV[b], a.X + j * E, E, lane);
        }
        cp_async_commit();
    };
    const long long n = pt.e - pt.s;
#pragma unroll
    for (int t = 0; t < S - 1; ++t) issue(t);
    float v[NH];
    float dd = 0.f, xx = 0.f;   // update form: sums of d^2 and of the updated x^2
    if (pt.hasR) {
        const double* xr = a.Xn + i * E + r * nr;
        double* xo = a.X + pt.e * E + r * nr;
#pragma unroll
        for (int q = 0; q < NH; ++q) {
            const double d = (cb + q < nr) ? xr[cb + q] : 0.0;
            v[q] = trunc_f32(d);
            if (cb + q < nr) {
                if (a.accum) {
                    const double xn = xo[cb + q] + d;
                    xo[cb + q] = xn;
                    const float xf = trunc_f32(xn);
                    dd = fmaf(v[q], v[q], dd);
                    xx = fmaf(xf, xf, xx);
                } else {
                    xo[cb + q] = d;
                }
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < NH; ++q) v[q] = 0.f;
    }
    put_vec<NH>(xa, v);
    if (pt.hasL) {
        load_vec<NH>(v, a.Xn + (i - 1) * E + r * nr, cb, nr);
        put_vec<NH>(xb, v);
    }
    __syncwarp();
    for (long long t = 0; t < n; ++t) {
        const long long j = pt.e - 1 - t;
        const int b = (int)(t % S);
        cp_async_wait<S - 2>();
        __syncwarp();
        issue(t + S - 1);    // into the slot row j + 1 used
        float x[NH];
#pragma unroll
        for (int q = 0; q < NH; ++q) x[q] = (cb + q < nr) ? sm.sH[b][r * nr + cb + q] : 0.f;
        if (useY(j)) {
            float Yr[16];
            read_row16(Yr, sm.sA[b] + r * M);
            gemv_acc<NH, true>(x, Yr, sm.xa + cb, SW);
        }
        if (pt.hasL) {
            float Zr[16];
            read_row16(Zr, sm.sC[b] + r * M);
            gemv_acc<NH, false>(x, Zr, sm.xb + cb, SW);
        }
        __syncwarp();          // x_{j+1} fully read
        put_vec<NH>(xa, x);
        double* xo = a.X + j * E + r * nr;
        if (a.accum) {
#pragma unroll
            for (int q = 0; q < NH; ++q)
                if (cb + q < nr) {
                    const double xn = sm.sV[b][r * nr + cb + q] + (double)x[q];
                    xo[cb + q] = xn;
                    const float xf = trunc_f32(xn);
                    dd = fmaf(x[q], x[q], dd);
                    xx = fmaf(xf, xf, xx);
                }
        } else {
#pragma unroll
            for (int q = 0; q < NH; ++q)
                if (cb + q < nr) xo[cb + q] = (double)x[q];
        }
        __syncwarp();          // slot b is refilled by the next iteration
    }
    cp_async_wait<0>();
    __syncwarp();
    if (a.accum) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            dd += __shfl_xor_sync(0xffffffffu, dd, off);
            xx += __shfl_xor_sync(0xffffffffu, xx, off);
        }
        if (lane == 0) {
            a.nrm[2 * i] = (double)dd;
            a.nrm[2 * i + 1] = (double)xx;
        }
    }
}

template <int NH>
__global__ void __launch_bounds__(32 * WarpS16<NH>::WARPS) k_solve_fwd_w16(const LevelArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    auto& sm = reinterpret_cast<typename WarpS16<NH>::Smem*>(smem_raw)[warp];
    const long long u = (long long)blockIdx.x * WarpS16<NH>::WARPS + warp;
    if (u >= a.p) return;
    solve_fwd_w16_body<NH>(a, u, sm);
}
template <int NH>
__global__ void __launch_bounds__(32 * WarpS16<NH>::WARPS) k_solve_bwd_w16(const LevelArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    auto& sm = reinterpret_cast<typename WarpS16<NH>::Smem*>(smem_raw)[warp];
    const long long u = (long long)blockIdx.x * WarpS16<NH>::WARPS + warp;
    if (u >= a.p) return;
    solve_bwd_w16_body<NH>(a, u, sm);
}
// Reduced right-hand side of separator s: g_s -= Hw of partition s + 1.
template <int MODE>
__global__ void __launch_bounds__(256) k_sep_rhs_w16(const LevelArgs a) {
    const long long E = 16LL * a.nr;
    const long long n = (a.p - 1) * E;
    const float* hw = reinterpret_cast<const float*>(a.Hw);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        a.Fn[e] -= (double)hw[e + E];
}

// The warp kernel serves FP32 block tridiagonal levels of order 16 without the
// BF16 tensor-core products and without breakdown detection (pivoted plans),
// whose matrices start on 16-byte boundaries (the staging copies are 16 bytes).
inline bool use_factor_w16(const LevelArgs& a) {
    const uintptr_t al = (uintptr_t)a.B | (uintptr_t)a.D | (uintptr_t)a.C;
    return a.mode == 0 && !a.bf16 && a.brk == nullptr && a.starts == nullptr && (al & 15u) == 0;
}

}  // namespace bt
