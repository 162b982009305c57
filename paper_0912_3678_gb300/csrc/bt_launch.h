// Host-side launchers of the partition-method kernels, one table per block order m.
#pragma once
#include <cuda_runtime.h>
#include "bt_level.h"

namespace bt {

struct Launchers {
    // low = true: local factors of this level in FP32 (the level's T is float)
    cudaError_t (*factor)(const LevelArgs&, bool low, cudaStream_t);
    cudaError_t (*assemble)(const LevelArgs&, bool low, cudaStream_t);
    cudaError_t (*solve_fwd)(const LevelArgs&, bool low, cudaStream_t);
    cudaError_t (*assemble_rhs)(const LevelArgs&, bool low, cudaStream_t);
    cudaError_t (*solve_bwd)(const LevelArgs&, bool low, cudaStream_t);
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
