// Cyclic reduction of a whole BABD system (the method Sec. 2 recommends for
// ABD/BABD matrices, the two-row case of its partitioning applied
// recursively).  Level l holds N rows S_j y_j + R_j y_{j+1} = r_j (j < N) on
// the unknowns y_0..y_N; rows 2k and 2k+1 eliminate y_{2k+1}:
//   y_{2k+1} = R_{2k}^{-1} r_{2k} - T_k y_{2k},   T_k = R_{2k}^{-1} S_{2k},
//   (-S_{2k+1} T_k) y_{2k} + R_{2k+1} y_{2k+2} = r_{2k+1} - S_{2k+1} R_{2k}^{-1} r_{2k},
// which leaves ceil(N/2) rows of the same form on y_0, y_2, ..., y_N (for odd
// N the last row passes unchanged and y_N keeps its place at the end).  After
// ceil(log2 N) levels one row is left; with the boundary row B0 y_0 + B1 y_N =
// beta it is a 2m x 2m system, solved by elimination with partial pivoting.
// One CTA of 8m threads per pair of rows; the inverses are Gauss-Jordan with
// partial pivoting.  Right-hand sides are stored in the BABD layout
// [beta; r_0; ...; r_{N-1}] ([N+1][m][nr]) on every level.
#pragma once
#include "bt_bcr.cuh"
#include "bt_cta.cuh"

namespace bt {

struct CrbArgs {
    long long N;          // rows of this level (>= 2)
    int nr, level;
    const double* S;      // [N][m][m]
    const double* R;
    double* Rinv;         // [N/2] R_{2k}^{-1}
    double* T;            // [N/2] R_{2k}^{-1} S_{2k}
    double* Sn;           // next level [ceil(N/2)][m][m]
    double* Rn;
    const double* F;      // [N+1][m][nr]: beta, r_0 .. r_{N-1}
    double* U;            // [N/2][m][nr]: R_{2k}^{-1} r_{2k}
    double* Fn;           // next level [ceil(N/2)+1][m][nr]
    double* X;            // [N+1][m][nr]: y_0 .. y_N
    const double* Xn;     // next level [ceil(N/2)+1][m][nr]
    long long* status;
};

template <int M>
constexpr size_t crb_factor_smem_bytes() {
    return sizeof(double) * (3 * Cta<double, M>::BLK + M) + sizeof(int) * 32;
}
template <int M>
constexpr size_t crb_vec_smem_bytes() {
    return sizeof(double) * (2 * Cta<double, M>::BLK + 2 * M * 32);
}

template <int M>
__global__ void __launch_bounds__(8 * M) k_crb_factor(const CrbArgs a) {
    using S = Cta<double, M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* s0 = reinterpret_cast<double*>(smem_raw);
    double* s1 = s0 + S::BLK;
    double* s2 = s1 + S::BLK;
    double* colk = s2 + S::BLK;
    int* perm = reinterpret_cast<int*>(colk + M);
    const long long MM = S::MM;
    const long long P = a.N / 2;
    const long long k = blockIdx.x;
    const Own<double, M> o;
    if (k >= P) {
        // odd N: the last row passes to the next level unchanged
        for (int idx = threadIdx.x; idx < M * M; idx += S::NT) {
            a.Sn[k * MM + idx] = a.S[(a.N - 1) * MM + idx];
            a.Rn[k * MM + idx] = a.R[(a.N - 1) * MM + idx];
        }
        return;
    }
    load_blk<double, M>(s0, a.R + 2 * k * MM);
    load_blk<double, M>(s1, a.S + 2 * k * MM);
    load_blk<double, M>(s2, a.S + (2 * k + 1) * MM);
    for (int idx = threadIdx.x; idx < M * M; idx += S::NT) a.Rn[k * MM + idx] = a.R[(2 * k + 1) * MM + idx];
    __syncthreads();
    gj_inverse<double, M>(s0, colk, perm, a.status, a.level, k, 2 * k);
    __syncthreads();
    store_blk<double, M>(a.Rinv + k * MM, s0);
    double t[S::R];
    zero_own<double, M>(t);
    gemm_acc<double, M, false>(t, s0, s1, o);          // T_k = R_{2k}^{-1} S_{2k}
    store_own<double, M>(a.T + k * MM, t, o);
    __syncthreads();
    write_own<double, M>(s1, t, o);
    __syncthreads();
    double sn[S::R];
    zero_own<double, M>(sn);
    gemm_acc<double, M, true>(sn, s2, s1, o);          // S'_k = -S_{2k+1} T_k
    store_own<double, M>(a.Sn + k * MM, sn, o);
}

template <int M>
__global__ void __launch_bounds__(8 * M) k_crb_rhs(const CrbArgs a) {
    using S = Cta<double, M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* s0 = reinterpret_cast<double*>(smem_raw);
    double* s1 = s0 + S::BLK;
    double* v0 = s1 + S::BLK;
    double* v1 = v0 + M * 32;
    const int nr = a.nr;
    const int E = M * nr;
    const long long MM = S::MM;
    const long long P = a.N / 2;
    const long long k = blockIdx.x;
    if (k == 0)
        for (int el = threadIdx.x; el < E; el += S::NT) a.Fn[el] = a.F[el];   // beta
    if (k >= P) {
        for (int el = threadIdx.x; el < E; el += S::NT) a.Fn[(k + 1) * E + el] = a.F[a.N * E + el];
        return;
    }
    load_blk<double, M>(s0, a.Rinv + k * MM);
    load_blk<double, M>(s1, a.S + (2 * k + 1) * MM);
    for (int el = threadIdx.x; el < E; el += S::NT) v0[el] = a.F[(2 * k + 1) * E + el];   // r_{2k}
    __syncthreads();
    for (int el = threadIdx.x; el < E; el += S::NT) {
        const int rr = el / nr, c = el % nr;
        v1[el] = dot_lat<double, M>(s0 + rr * S::LD, v0 + c, nr);
    }
    __syncthreads();
    for (int el = threadIdx.x; el < E; el += S::NT) {
        const int rr = el / nr, c = el % nr;
        a.U[k * E + el] = v1[el];
        a.Fn[(k + 1) * E + el] = a.F[(2 * k + 2) * E + el] - dot_lat<double, M>(s1 + rr * S::LD, v1 + c, nr);
    }
}

template <int M>
__global__ void __launch_bounds__(8 * M) k_crb_back(const CrbArgs a) {
    using S = Cta<double, M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* s0 = reinterpret_cast<double*>(smem_raw);
    double* v0 = s0 + 2 * S::BLK;
    const int nr = a.nr;
    const int E = M * nr;
    const long long MM = S::MM;
    const long long P = a.N / 2;
    const long long Nn = a.N - P;       // rows of the next level
    const long long k = blockIdx.x;
    if (k >= P) {
        // y_N is the next level's last unknown; for odd N, y_{N-1} its unknown P
        for (int el = threadIdx.x; el < E; el += S::NT) {
            a.X[a.N * E + el] = a.Xn[Nn * E + el];
            if (a.N & 1) a.X[(a.N - 1) * E + el] = a.Xn[P * E + el];
        }
        return;
    }
    load_blk<double, M>(s0, a.T + k * MM);
    for (int el = threadIdx.x; el < E; el += S::NT) {
        const double y = a.Xn[k * E + el];
        v0[el] = y;
        a.X[2 * k * E + el] = y;
    }
    __syncthreads();
    for (int el = threadIdx.x; el < E; el += S::NT) {
        const int rr = el / nr, c = el % nr;
        a.X[(2 * k + 1) * E + el] = a.U[k * E + el] - dot_lat<double, M>(s0 + rr * S::LD, v0 + c, nr);
    }
}

}  // namespace bt
