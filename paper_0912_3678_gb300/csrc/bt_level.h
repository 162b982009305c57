// Arguments of one level of the recursive partition method (host and device).
#pragma once
#include <cstdint>

namespace bt {

// One level: a block tridiagonal system (mode 0, block rows 0..N-1) or a
// BABD system (mode 1, block rows 0..N with row 0 the boundary row and the
// corner coupling row 0 to row N).  Block row r of the level matrix is read
// at index r - shift of B/D/C (BABD: B = S, D = R, shift = 1, C unused).
struct LevelArgs {
    int mode;
    int level;
    int tpb;           // threads per CTA of the thread-per-partition kernels (m <= 4): 64, 128 or 256
    int bf16;          // Schur product B_j Y_{j-1} with BF16 operands on the tensor cores (FP32 levels, m >= 16)
    int group;         // m = 2, 4 FP64 levels: a group of m*m lanes per partition instead of one thread
    long long N, p, base, extra;
    const double* B;
    const double* D;
    const double* C;
    int shift;
    // factors of the local blocks, element type T of the level, indexed by block row
    void* Dinv;     // D'_j^{-1}
    void* Y;        // D'_j^{-1} C_j
    void* Zc;       // left spike coefficient: x_j = h_j + Zc_j x_L - Y_j x_{j+1}
    void* Pf;       // [p][m][m] top-row coefficient on x_L after full elimination
    void* Qf;       // [p][m][m] top-row coefficient on x_R
    // next level matrix (FP64)
    double* Bn;
    double* Dn;
    double* Cn;
    // solve phase
    const double* F;   // [rows][m][nr] right-hand side of this level
    double* X;         // [rows][m][nr] solution of this level (holds h_j in between)
    int nr;
    double* Fn;        // next level right-hand side
    const double* Xn;  // next level solution
    void* Hf;          // [p][m][nr] top-row right-hand side after full elimination (T)
    long long* status;
    // pivoted partitions (mode 0): explicit partition starts and breakdown rows
    const long long* starts;   // [p+1] first block row of each partition (null: uniform split)
    long long* brk;            // breakdown list: [0] count, [1..brk_cap] block rows (null: report singular)
    long long brk_cap;
    double tau;                // breakdown: |pivot| <= tau * largest entry of the row's blocks
    // a launch over part of the level: units [unit0, unit_end) (unit_end = 0: the whole level)
    long long unit0, unit_end;
    // factorization in phases (CTA kernels, mode 0): phase k of `phases` takes local rows
    // [s + L k / phases, s + L (k+1) / phases) of every partition (L = e - s); phases <= 1: all
    int phase, phases;
    // warp-per-partition FP32 kernels (order 16, bt_warp.cuh): the left separator's
    // chain W_j = -W_{j-1} Y_{j-1} per block row ([rows][m][m], null: not stored), the
    // forward-solve vectors h_j ([rows][m][nr], FP32) and sum_j W_j h_j per partition
    // ([p][m][nr], FP32)
    void* W;
    void* Hv;
    void* Hw;
    // the level matrix split into FP32 (hi, lo) parts for the double-float
    // refinement residual and the warp forward solve, negated, by column pairs:
    // float4 (-hi_k, -hi_k+1, -lo_k, -lo_k+1), k even, [3][rows][m][m/2]
    // (B, D, C; the same bytes as float2 [3][rows][m][m]); null: not kept
    void* As;
    // warp kernels: ||A||_inf maxima slots filled by the factorization (null: not
    // computed there); back substitution in update form X += d with per-partition
    // (||d||^2, ||x||^2) partials in nrm[2 i] (accum != 0)
    unsigned long long* amax;
    int accum;
    double* nrm;
};

}  // namespace bt
