// Block cyclic reduction (odd-even reduction) of the reduced system, the
// "cyclic reduction" variant of Sec. 2 applied to T_p with one
// synchronisation (kernel launch) per reduction step.  FP64, CTA per row
// (m >= 8).  Level l holds K active block rows (B_q, D_q, C_q, f_q); the rows
// at odd positions are eliminated:
//   alpha_q = -B_{2q} D_{2q-1}^{-1},  gamma_q = -C_{2q} D_{2q+1}^{-1}
//   D'_q = D_{2q} + alpha_q C_{2q-1} + gamma_q B_{2q+1}
//   B'_q = alpha_q B_{2q-1},  C'_q = gamma_q C_{2q+1},  f'_q = f_{2q} + alpha_q f_{2q-1} + gamma_q f_{2q+1}
// and after the single remaining row is solved the odd rows are recovered:
//   x_{2q+1} = D_{2q+1}^{-1} (f_{2q+1} - B_{2q+1} x_{2q} - C_{2q+1} x_{2q+2}).
#pragma once
#include "bt_cta.cuh"

namespace bt {

struct BcrArgs {
    long long K;          // active rows of this level
    int nr, level;
    const double* B;      // [K][m][m]
    const double* D;
    const double* C;
    double* Dinv;         // [K/2] inverses of the odd rows (the single row when K == 1)
    double* al;           // [(K+1)/2] alpha of the kept rows
    double* ga;           // [(K+1)/2] gamma of the kept rows
    double* Bn;           // next level [(K+1)/2][m][m]
    double* Dn;
    double* Cn;
    const double* F;      // [K][m][nr]
    double* Fn;           // [(K+1)/2][m][nr]
    double* X;            // [K][m][nr]
    const double* Xn;     // [(K+1)/2][m][nr]
    long long* status;
};

template <int M>
constexpr size_t bcr_smem_bytes() {
    return sizeof(double) * (4 * Cta<double, M>::BLK + M) + sizeof(int) * M;
}

// Inverse of the odd rows (q -> row 2q+1), or of the single row when K == 1.
template <int M>
__global__ void __launch_bounds__(8 * M) k_bcr_inv(const BcrArgs a) {
    using S = Cta<double, M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sD = reinterpret_cast<double*>(smem_raw);
    double* colk = sD + 4 * S::BLK;
    int* perm = reinterpret_cast<int*>(colk + M);
    const long long q = blockIdx.x;
    const long long row = (a.K == 1) ? 0 : 2 * q + 1;
    if (row >= a.K) return;
    load_blk<double, M>(sD, a.D + row * S::MM);
    __syncthreads();
    gj_inverse<double, M>(sD, colk, perm, a.status, a.level, -2, row);
    store_blk<double, M>(a.Dinv + q * S::MM, sD);
}

// Update of the kept row 2q: alpha, gamma, D', B', C'.
template <int M>
__global__ void __launch_bounds__(8 * M) k_bcr_update(const BcrArgs a) {
    using S = Cta<double, M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* s0 = reinterpret_cast<double*>(smem_raw);
    double* s1 = s0 + S::BLK;
    double* sal = s1 + S::BLK;
    double* sga = sal + S::BLK;
    const long long q = blockIdx.x;
    const long long r = 2 * q;
    const bool left = q >= 1;
    const bool right = r + 1 < a.K;
    const long long MM = S::MM;
    const Own<double, M> o;
    double al[S::R], ga[S::R];
    zero_own<double, M>(al);
    zero_own<double, M>(ga);
    if (left) {
        load_blk<double, M>(s0, a.B + r * MM);
        load_blk<double, M>(s1, a.Dinv + (q - 1) * MM);
        __syncthreads();
        gemm_acc<double, M, true>(al, s0, s1, o);
        __syncthreads();
    }
    if (right) {
        load_blk<double, M>(s0, a.C + r * MM);
        load_blk<double, M>(s1, a.Dinv + q * MM);
        __syncthreads();
        gemm_acc<double, M, true>(ga, s0, s1, o);
        __syncthreads();
    }
    write_own<double, M>(sal, al, o);
    write_own<double, M>(sga, ga, o);
    store_own<double, M>(a.al + q * MM, al, o);
    store_own<double, M>(a.ga + q * MM, ga, o);
    double d[S::R], bn[S::R], cn[S::R];
#pragma unroll
    for (int u = 0; u < S::R; ++u) d[u] = a.D[r * MM + (o.r0 + u) * M + o.c];
    zero_own<double, M>(bn);
    zero_own<double, M>(cn);
    __syncthreads();
    if (left) {
        load_blk<double, M>(s0, a.C + (r - 1) * MM);
        load_blk<double, M>(s1, a.B + (r - 1) * MM);
        __syncthreads();
        gemm_acc<double, M, false>(d, sal, s0, o);
        if (r - 1 >= 1) gemm_acc<double, M, false>(bn, sal, s1, o);
        __syncthreads();
    }
    if (right) {
        load_blk<double, M>(s0, a.B + (r + 1) * MM);
        load_blk<double, M>(s1, a.C + (r + 1) * MM);
        __syncthreads();
        gemm_acc<double, M, false>(d, sga, s0, o);
        if (r + 2 < a.K) gemm_acc<double, M, false>(cn, sga, s1, o);
    }
    store_own<double, M>(a.Dn + q * MM, d, o);
    store_own<double, M>(a.Bn + q * MM, bn, o);
    store_own<double, M>(a.Cn + q * MM, cn, o);
}

// f'_q = f_{2q} + alpha_q f_{2q-1} + gamma_q f_{2q+1}; with K == 1: x = D^{-1} f.
template <int M>
__global__ void __launch_bounds__(8 * M) k_bcr_rhs(const BcrArgs a) {
    using S = Cta<double, M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* s0 = reinterpret_cast<double*>(smem_raw);
    double* s1 = s0 + S::BLK;
    double* v0 = s1 + S::BLK;
    double* v1 = v0 + M * 32;
    const int nr = a.nr;
    const int E = M * nr;
    const long long q = blockIdx.x;
    const long long MM = S::MM;
    if (a.K == 1) {
        load_blk<double, M>(s0, a.Dinv);
        for (int el = threadIdx.x; el < E; el += S::NT) v0[el] = a.F[el];
        __syncthreads();
        for (int el = threadIdx.x; el < E; el += S::NT) {
            const int rr = el / nr, c = el % nr;
            double acc = 0.0;
            for (int k = 0; k < M; ++k) acc = fma(s0[rr * S::LD + k], v0[k * nr + c], acc);
            a.X[el] = acc;
        }
        return;
    }
    const long long r = 2 * q;
    const bool left = q >= 1, right = r + 1 < a.K;
    if (left) load_blk<double, M>(s0, a.al + q * MM);
    if (right) load_blk<double, M>(s1, a.ga + q * MM);
    for (int el = threadIdx.x; el < E; el += S::NT) {
        v0[el] = left ? a.F[(r - 1) * E + el] : 0.0;
        v1[el] = right ? a.F[(r + 1) * E + el] : 0.0;
    }
    __syncthreads();
    for (int el = threadIdx.x; el < E; el += S::NT) {
        const int rr = el / nr, c = el % nr;
        double acc = a.F[r * E + el];
        if (left)
            for (int k = 0; k < M; ++k) acc = fma(s0[rr * S::LD + k], v0[k * nr + c], acc);
        if (right)
            for (int k = 0; k < M; ++k) acc = fma(s1[rr * S::LD + k], v1[k * nr + c], acc);
        a.Fn[q * E + el] = acc;
    }
}

// x_{2q} = x'_q;  x_{2q+1} = D_{2q+1}^{-1} (f_{2q+1} - B_{2q+1} x'_q - C_{2q+1} x'_{q+1}).
template <int M>
__global__ void __launch_bounds__(8 * M) k_bcr_back(const BcrArgs a) {
    using S = Cta<double, M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* s0 = reinterpret_cast<double*>(smem_raw);
    double* s1 = s0 + S::BLK;
    double* s2 = s1 + S::BLK;
    double* v0 = s2 + S::BLK;
    double* v1 = v0 + M * 32;
    double* t = v1 + M * 32;
    const int nr = a.nr;
    const int E = M * nr;
    const long long q = blockIdx.x;
    const long long MM = S::MM;
    const long long r = 2 * q + 1;
    for (int el = threadIdx.x; el < E; el += S::NT) a.X[2 * q * E + el] = a.Xn[q * E + el];
    if (r >= a.K) return;
    const bool right = r + 1 < a.K;
    load_blk<double, M>(s0, a.B + r * MM);
    if (right) load_blk<double, M>(s1, a.C + r * MM);
    load_blk<double, M>(s2, a.Dinv + q * MM);
    for (int el = threadIdx.x; el < E; el += S::NT) {
        v0[el] = a.Xn[q * E + el];
        v1[el] = right ? a.Xn[(q + 1) * E + el] : 0.0;
    }
    __syncthreads();
    for (int el = threadIdx.x; el < E; el += S::NT) {
        const int rr = el / nr, c = el % nr;
        double acc = a.F[r * E + el];
        for (int k = 0; k < M; ++k) acc = fma(-s0[rr * S::LD + k], v0[k * nr + c], acc);
        if (right)
            for (int k = 0; k < M; ++k) acc = fma(-s1[rr * S::LD + k], v1[k * nr + c], acc);
        t[el] = acc;
    }
    __syncthreads();
    for (int el = threadIdx.x; el < E; el += S::NT) {
        const int rr = el / nr, c = el % nr;
        double acc = 0.0;
        for (int k = 0; k < M; ++k) acc = fma(s2[rr * S::LD + k], t[k * nr + c], acc);
        a.X[r * E + el] = acc;
    }
}

template <int M>
constexpr size_t bcr_vec_smem_bytes() {
    return sizeof(double) * (3 * Cta<double, M>::BLK + 3 * M * 32);
}

}  // namespace bt
