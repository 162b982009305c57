// Host-side launchers of the partition-method kernels, one table per block order m.
#pragma once
#include <cuda_runtime.h>
#include "bt_level.h"

namespace bt {
struct BcrArgs;
struct CrbArgs;
}

namespace bt {

struct Launchers {
    // low = true: local factors of this level in FP32 (the level's T is float)
    cudaError_t (*factor)(const LevelArgs&, bool low, cudaStream_t);
    // the factorization of partitions [p_begin, p_end) of a level only
    cudaError_t (*factor_part)(const LevelArgs&, bool low, long long p_begin, long long p_end, cudaStream_t);
    // phase k of `phases` of a block tridiagonal level's factorization (CTA kernels; null for m <= 4)
    cudaError_t (*factor_phase)(const LevelArgs&, bool low, int k, int phases, cudaStream_t);
    cudaError_t (*assemble)(const LevelArgs&, bool low, cudaStream_t);
    cudaError_t (*solve_fwd)(const LevelArgs&, bool low, cudaStream_t);
    cudaError_t (*assemble_rhs)(const LevelArgs&, bool low, cudaStream_t);
    cudaError_t (*solve_bwd)(const LevelArgs&, bool low, cudaStream_t);
    // Batched (persistent) variants: work[w] = (index into args, unit); `grid`
    // CTAs stride over the nwork items.  mode is the same for every item.
    cudaError_t (*factor_b)(const LevelArgs* args, const int2* work, int nwork, int mode, bool low, int grid,
                            cudaStream_t);
    cudaError_t (*assemble_b)(const LevelArgs* args, const int2* work, int nwork, int mode, bool low, int grid,
                              cudaStream_t);
    cudaError_t (*solve_fwd_b)(const LevelArgs* args, const int2* work, int nwork, int mode, bool low, int grid,
                               cudaStream_t);
    cudaError_t (*assemble_rhs_b)(const LevelArgs* args, const int2* work, int nwork, int mode, bool low,
                                  int grid, cudaStream_t);
    cudaError_t (*solve_bwd_b)(const LevelArgs* args, const int2* work, int nwork, int mode, bool low, int grid,
                               cudaStream_t);
    // CTA-per-unit kernels (m >= 8) or thread-per-unit kernels (m <= 4)
    bool cta;
    // dynamic shared memory per CTA of each kernel kind (CTA kernels)
    size_t smem_factor64, smem_factor32, smem_assemble, smem_solve64, smem_solve32, smem_assemble_rhs;
    // make sure every kernel of this m has its shared-memory attribute set
    cudaError_t (*prepare)();
    // block cyclic reduction of the reduced system (m >= 8; null otherwise)
    cudaError_t (*bcr_factor)(const BcrArgs&, long long ctas, cudaStream_t);   // one reduction step
    cudaError_t (*bcr_rhs)(const BcrArgs&, long long ctas, cudaStream_t);
    cudaError_t (*bcr_back)(const BcrArgs&, long long ctas, cudaStream_t);
    // cyclic reduction of a whole BABD system: one level's factor, right-hand side and back
    // substitution (m >= 8; null otherwise)
    cudaError_t (*crb_factor)(const CrbArgs&, cudaStream_t);
    cudaError_t (*crb_rhs)(const CrbArgs&, cudaStream_t);
    cudaError_t (*crb_back)(const CrbArgs&, cudaStream_t);
    // warp-per-partition FP32 kernels (order 16; null otherwise): whether the level's
    // factorization runs on them, and their forward solve, separator right-hand side and
    // back substitution (they need the level's W, Hv and Hw buffers)
    bool (*warp_ok)(const LevelArgs&, bool low);
    cudaError_t (*solve_fwd_w)(const LevelArgs&, cudaStream_t);
    cudaError_t (*sep_rhs_w)(const LevelArgs&, cudaStream_t);
    cudaError_t (*solve_bwd_w)(const LevelArgs&, cudaStream_t);
};

const Launchers* launchers_m1();
const Launchers* launchers_m2();
const Launchers* launchers_m4();
const Launchers* launchers_m8();
const Launchers* launchers_m16();
const Launchers* launchers_m32();

inline const Launchers* launchers_for(int m) {
    switch (m) {
        case 1: return launchers_m1();
        case 2: return launchers_m2();
        case 4: return launchers_m4();
        case 8: return launchers_m8();
        case 16: return launchers_m16();
        case 32: return launchers_m32();
        default: return nullptr;
    }
}

}  // namespace bt
