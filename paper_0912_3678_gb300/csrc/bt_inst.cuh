// Instantiates the launchers of one block order M (included by bt_inst_m*.cu).
#pragma once
#include "bt_bcr.cuh"
#include "bt_crb.cuh"
#include "bt_cta.cuh"
#include "bt_gp.cuh"
#include "bt_launch.h"
#include "bt_tp.cuh"
#include "bt_warp.cuh"

namespace bt {

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static inline unsigned grid_for(long long threads, int block) { return (unsigned)((threads + block - 1) / block); }
static inline int tpb(const LevelArgs& a) { return (a.tpb == 64 || a.tpb == 256) ? a.tpb : 128; }
// lane-group kernels (bt_gp.cuh): FP64 levels of block order 2 or 4 flagged by the planner
template <typename T, int M>
static inline bool use_gp(const LevelArgs& a) {
    return (M == 2 || M == 4) && std::is_same<T, double>::value && a.group != 0;
}
static inline long long chunks(const LevelArgs& a, int m) { return (a.nr + m - 1) / m; }

template <int M>
struct Inst {
    // FP32 block tridiagonal levels of order 16: one warp per partition (bt_warp.cuh)
    template <typename T, int MODE>
    static bool warp_factor(const LevelArgs& a) {
        if constexpr (M == 16 && MODE == 0 && std::is_same<T, float>::value) return use_factor_w16(a);
        return false;
    }
    static cudaError_t launch_w16(const LevelArgs& a, long long units, cudaStream_t s) {
        const size_t smem = factor_w16_smem_bytes();
        cudaError_t e = set_smem(k_factor_w16<0>, smem);
        if (e != cudaSuccess) return e;
        k_factor_w16<0><<<grid_for(units, WarpF16::WARPS), 32 * WarpF16::WARPS, smem, s>>>(a);
        return cudaGetLastError();
    }
    template <typename T, int MODE>
    static cudaError_t factor_t(const LevelArgs& a, cudaStream_t s) {
        if (a.p <= 0) return cudaSuccess;
        if (warp_factor<T, MODE>(a)) return launch_w16(a, a.p, s);
        if constexpr (M >= 8) {
            const size_t smem = factor_smem_bytes<T, M>();
            cudaError_t e = set_smem(k_factor_cta<T, M, MODE>, smem);
            if (e != cudaSuccess) return e;
            k_factor_cta<T, M, MODE><<<(unsigned)a.p, 8 * M, smem, s>>>(a);
        } else if (use_gp<T, M>(a)) {
            if constexpr (M == 2 || M == 4) k_factor_gp<M, MODE><<<grid_for(a.p * M * M, 128), 128, 0, s>>>(a);
        } else {
            k_factor_tp<T, M, MODE><<<grid_for(a.p, tpb(a)), tpb(a), 0, s>>>(a);
        }
        return cudaGetLastError();
    }
    static cudaError_t factor(const LevelArgs& a, bool low, cudaStream_t s) {
        if (a.mode == 0) return low ? factor_t<float, 0>(a, s) : factor_t<double, 0>(a, s);
        return low ? factor_t<float, 1>(a, s) : factor_t<double, 1>(a, s);
    }
    template <typename T, int MODE>
    static cudaError_t factor_part_t(const LevelArgs& a0, long long pb, long long pe, cudaStream_t s) {
        if (pe > a0.p) pe = a0.p;
        if (pb < 0 || pe <= pb) return cudaSuccess;
        LevelArgs a = a0;
        if (warp_factor<T, MODE>(a)) {
            a.unit0 = pb;
            a.unit_end = pe;
            return launch_w16(a, pe - pb, s);
        }
        if constexpr (M >= 8) {
            const size_t smem = factor_smem_bytes<T, M>();
            cudaError_t e = set_smem(k_factor_cta<T, M, MODE>, smem);
            if (e != cudaSuccess) return e;
            a.unit0 = pb;
            a.unit_end = pe;
            k_factor_cta<T, M, MODE><<<(unsigned)(pe - pb), 8 * M, smem, s>>>(a);
        } else if (use_gp<T, M>(a)) {
            if constexpr (M == 2 || M == 4) {
                a.unit0 = pb * M * M;
                a.unit_end = pe * M * M;
                k_factor_gp<M, MODE><<<grid_for((pe - pb) * M * M, 128), 128, 0, s>>>(a);
            }
        } else {
            a.unit0 = pb;
            a.unit_end = pe;
            k_factor_tp<T, M, MODE><<<grid_for(pe - pb, tpb(a)), tpb(a), 0, s>>>(a);
        }
        return cudaGetLastError();
    }
    static cudaError_t factor_phase(const LevelArgs& a0, bool low, int k, int phases, cudaStream_t s) {
        if (a0.mode != 0 || k < 0 || k >= phases) return cudaErrorInvalidValue;
        LevelArgs a = a0;
        a.phase = k;
        a.phases = phases;
        return low ? factor_t<float, 0>(a, s) : factor_t<double, 0>(a, s);
    }
    static cudaError_t factor_part(const LevelArgs& a, bool low, long long pb, long long pe, cudaStream_t s) {
        if (a.mode == 0) return low ? factor_part_t<float, 0>(a, pb, pe, s) : factor_part_t<double, 0>(a, pb, pe, s);
        return low ? factor_part_t<float, 1>(a, pb, pe, s) : factor_part_t<double, 1>(a, pb, pe, s);
    }
    template <typename T>
    static cudaError_t assemble_t(const LevelArgs& a, cudaStream_t s) {
        if (a.p <= 1) return cudaSuccess;
        if constexpr (M >= 8) {
            const size_t smem = assemble_smem_bytes<M>();
            cudaError_t e = set_smem(k_assemble_cta<T, M>, smem);
            if (e != cudaSuccess) return e;
            k_assemble_cta<T, M><<<(unsigned)(a.p - 1), 8 * M, smem, s>>>(a);
        } else if (use_gp<T, M>(a)) {
            if constexpr (M == 2 || M == 4) k_assemble_gp<M><<<grid_for((a.p - 1) * M * M, 128), 128, 0, s>>>(a);
        } else {
            k_assemble_tp<T, M><<<grid_for(a.p - 1, tpb(a)), tpb(a), 0, s>>>(a);
        }
        return cudaGetLastError();
    }
    static cudaError_t assemble(const LevelArgs& a, bool low, cudaStream_t s) {
        return low ? assemble_t<float>(a, s) : assemble_t<double>(a, s);
    }
    template <typename T, int MODE>
    static cudaError_t solve_fwd_t(const LevelArgs& a, cudaStream_t s) {
        if (a.p <= 0) return cudaSuccess;
        if constexpr (M >= 8) {
            const size_t smem = solve_smem_bytes<T, M>();
            cudaError_t e = set_smem(k_solve_fwd_cta<T, M, MODE>, smem);
            if (e != cudaSuccess) return e;
            k_solve_fwd_cta<T, M, MODE><<<(unsigned)a.p, 8 * M, smem, s>>>(a);
        } else if (use_gp<T, M>(a)) {
            if constexpr (M == 2 || M == 4)
                k_solve_fwd_gp<M, MODE><<<grid_for(a.p * chunks(a, M) * M * M, 128), 128, 0, s>>>(a);
        } else {
            k_solve_fwd_tp<T, M, MODE><<<grid_for(a.p * a.nr, tpb(a)), tpb(a), 0, s>>>(a);
        }
        return cudaGetLastError();
    }
    static cudaError_t solve_fwd(const LevelArgs& a, bool low, cudaStream_t s) {
        if (a.mode == 0) return low ? solve_fwd_t<float, 0>(a, s) : solve_fwd_t<double, 0>(a, s);
        return low ? solve_fwd_t<float, 1>(a, s) : solve_fwd_t<double, 1>(a, s);
    }
    template <typename T>
    static cudaError_t assemble_rhs_t(const LevelArgs& a, cudaStream_t s) {
        if (a.p <= 1) return cudaSuccess;
        if constexpr (M >= 8) {
            const size_t smem = assemble_rhs_smem_bytes<M>();
            cudaError_t e = set_smem(k_assemble_rhs_cta<T, M>, smem);
            if (e != cudaSuccess) return e;
            k_assemble_rhs_cta<T, M><<<(unsigned)(a.p - 1), 8 * M, smem, s>>>(a);
        } else if (use_gp<T, M>(a)) {
            if constexpr (M == 2 || M == 4)
                k_assemble_rhs_gp<M><<<grid_for((a.p - 1) * chunks(a, M) * M * M, 128), 128, 0, s>>>(a);
        } else {
            k_assemble_rhs_tp<T, M><<<grid_for((a.p - 1) * a.nr, tpb(a)), tpb(a), 0, s>>>(a);
        }
        return cudaGetLastError();
    }
    static cudaError_t assemble_rhs(const LevelArgs& a, bool low, cudaStream_t s) {
        return low ? assemble_rhs_t<float>(a, s) : assemble_rhs_t<double>(a, s);
    }
    template <typename T, int MODE>
    static cudaError_t solve_bwd_t(const LevelArgs& a, cudaStream_t s) {
        if (a.p <= 0) return cudaSuccess;
        if constexpr (M >= 8) {
            const size_t smem = solve_smem_bytes<T, M>();
            cudaError_t e = set_smem(k_solve_bwd_cta<T, M, MODE>, smem);
            if (e != cudaSuccess) return e;
            k_solve_bwd_cta<T, M, MODE><<<(unsigned)a.p, 8 * M, smem, s>>>(a);
        } else if (use_gp<T, M>(a)) {
            if constexpr (M == 2 || M == 4)
                k_solve_bwd_gp<M, MODE><<<grid_for(a.p * chunks(a, M) * M * M, 128), 128, 0, s>>>(a);
        } else {
            k_solve_bwd_tp<T, M, MODE><<<grid_for(a.p * a.nr, tpb(a)), tpb(a), 0, s>>>(a);
        }
        return cudaGetLastError();
    }
    static cudaError_t solve_bwd(const LevelArgs& a, bool low, cudaStream_t s) {
        if (a.mode == 0) return low ? solve_bwd_t<float, 0>(a, s) : solve_bwd_t<double, 0>(a, s);
        return low ? solve_bwd_t<float, 1>(a, s) : solve_bwd_t<double, 1>(a, s);
    }
    // ------------------------------------------------------------ batched --
    template <typename K>
    static cudaError_t launch_cta_b(K k, size_t smem, const LevelArgs* args, const int2* work, int nwork, int grid,
                                    cudaStream_t s) {
        if (nwork <= 0) return cudaSuccess;
        cudaError_t e = set_smem(k, smem);
        if (e != cudaSuccess) return e;
        k<<<grid, 8 * M, smem, s>>>(args, work, nwork);
        return cudaGetLastError();
    }
    template <typename K>
    static cudaError_t launch_tp_b(K k, const LevelArgs* args, const int2* work, int nwork, int grid,
                                   cudaStream_t s) {
        if (nwork <= 0) return cudaSuccess;
        k<<<grid, 128, 0, s>>>(args, work, nwork);
        return cudaGetLastError();
    }
    template <typename T, int MODE>
    static cudaError_t factor_bt(const LevelArgs* args, const int2* work, int nwork, int grid, cudaStream_t s) {
        if constexpr (M >= 8)
            return launch_cta_b(k_factor_cta_batch<T, M, MODE>, factor_smem_bytes<T, M>(), args, work, nwork, grid, s);
        else
            return launch_tp_b(k_factor_tp_batch<T, M, MODE>, args, work, nwork, grid, s);
    }
    template <typename T>
    static cudaError_t assemble_bt(const LevelArgs* args, const int2* work, int nwork, int grid, cudaStream_t s) {
        if constexpr (M >= 8)
            return launch_cta_b(k_assemble_cta_batch<T, M>, assemble_smem_bytes<M>(), args, work, nwork, grid, s);
        else
            return launch_tp_b(k_assemble_tp_batch<T, M>, args, work, nwork, grid, s);
    }
    template <typename T, int MODE>
    static cudaError_t solve_fwd_bt(const LevelArgs* args, const int2* work, int nwork, int grid, cudaStream_t s) {
        if constexpr (M >= 8)
            return launch_cta_b(k_solve_fwd_cta_batch<T, M, MODE>, solve_smem_bytes<T, M>(), args, work, nwork, grid, s);
        else
            return launch_tp_b(k_solve_fwd_tp_batch<T, M, MODE>, args, work, nwork, grid, s);
    }
    template <typename T>
    static cudaError_t assemble_rhs_bt(const LevelArgs* args, const int2* work, int nwork, int grid,
                                       cudaStream_t s) {
        if constexpr (M >= 8)
            return launch_cta_b(k_assemble_rhs_cta_batch<T, M>, assemble_rhs_smem_bytes<M>(), args, work, nwork,
                                grid, s);
        else
            return launch_tp_b(k_assemble_rhs_tp_batch<T, M>, args, work, nwork, grid, s);
    }
    template <typename T, int MODE>
    static cudaError_t solve_bwd_bt(const LevelArgs* args, const int2* work, int nwork, int grid, cudaStream_t s) {
        if constexpr (M >= 8)
            return launch_cta_b(k_solve_bwd_cta_batch<T, M, MODE>, solve_smem_bytes<T, M>(), args, work, nwork, grid, s);
        else
            return launch_tp_b(k_solve_bwd_tp_batch<T, M, MODE>, args, work, nwork, grid, s);
    }
    static cudaError_t factor_b(const LevelArgs* args, const int2* work, int nwork, int mode, bool low, int grid,
                                cudaStream_t s) {
        if (mode == 0)
            return low ? factor_bt<float, 0>(args, work, nwork, grid, s) : factor_bt<double, 0>(args, work, nwork, grid, s);
        return low ? factor_bt<float, 1>(args, work, nwork, grid, s) : factor_bt<double, 1>(args, work, nwork, grid, s);
    }
    static cudaError_t assemble_b(const LevelArgs* args, const int2* work, int nwork, int mode, bool low, int grid,
                                  cudaStream_t s) {
        (void)mode;
        return low ? assemble_bt<float>(args, work, nwork, grid, s) : assemble_bt<double>(args, work, nwork, grid, s);
    }
    static cudaError_t solve_fwd_b(const LevelArgs* args, const int2* work, int nwork, int mode, bool low, int grid,
                                   cudaStream_t s) {
        if (mode == 0)
            return low ? solve_fwd_bt<float, 0>(args, work, nwork, grid, s)
                       : solve_fwd_bt<double, 0>(args, work, nwork, grid, s);
        return low ? solve_fwd_bt<float, 1>(args, work, nwork, grid, s)
                   : solve_fwd_bt<double, 1>(args, work, nwork, grid, s);
    }
    static cudaError_t assemble_rhs_b(const LevelArgs* args, const int2* work, int nwork, int mode, bool low,
                                      int grid, cudaStream_t s) {
        (void)mode;
        return low ? assemble_rhs_bt<float>(args, work, nwork, grid, s)
                   : assemble_rhs_bt<double>(args, work, nwork, grid, s);
    }
    static cudaError_t solve_bwd_b(const LevelArgs* args, const int2* work, int nwork, int mode, bool low, int grid,
                                   cudaStream_t s) {
        if (mode == 0)
            return low ? solve_bwd_bt<float, 0>(args, work, nwork, grid, s)
                       : solve_bwd_bt<double, 0>(args, work, nwork, grid, s);
        return low ? solve_bwd_bt<float, 1>(args, work, nwork, grid, s)
                   : solve_bwd_bt<double, 1>(args, work, nwork, grid, s);
    }
    static bool warp_ok(const LevelArgs& a, bool low) {
        if constexpr (M == 16) return low && use_factor_w16(a);
        return false;
    }
    template <int NH>
    static cudaError_t launch_sw(void (*k)(const LevelArgs), const LevelArgs& a, cudaStream_t s) {
        const size_t smem = sizeof(typename WarpS16<NH>::Smem) * WarpS16<NH>::WARPS;
        cudaError_t e = set_smem(k, smem);
        if (e != cudaSuccess) return e;
        k<<<grid_for(a.p, WarpS16<NH>::WARPS), 32 * WarpS16<NH>::WARPS, smem, s>>>(a);
        return cudaGetLastError();
    }
    static cudaError_t solve_fwd_w(const LevelArgs& a, cudaStream_t s) {
        if (a.p <= 0) return cudaSuccess;
        if constexpr (M == 16) {
            if (a.nr <= 8) return launch_sw<4>(k_solve_fwd_w16<4>, a, s);
            return launch_sw<16>(k_solve_fwd_w16<16>, a, s);
        }
        return cudaErrorInvalidValue;
    }
    static cudaError_t solve_bwd_w(const LevelArgs& a, cudaStream_t s) {
        if (a.p <= 0) return cudaSuccess;
        if constexpr (M == 16) {
            if (a.nr <= 8) return launch_sw<4>(k_solve_bwd_w16<4>, a, s);
            return launch_sw<16>(k_solve_bwd_w16<16>, a, s);
        }
        return cudaErrorInvalidValue;
    }
    static cudaError_t sep_rhs_w(const LevelArgs& a, cudaStream_t s) {
        if (a.p <= 1) return cudaSuccess;
        const long long n = (a.p - 1) * 16LL * a.nr;
        long long blocks = (n + 255) / 256;
        if (blocks > 4096) blocks = 4096;
        k_sep_rhs_w16<0><<<(unsigned)blocks, 256, 0, s>>>(a);
        return cudaGetLastError();
    }
    static cudaError_t prepare() {
        if constexpr (M >= 8) {
            const size_t f64 = factor_smem_bytes<double, M>(), f32 = factor_smem_bytes<float, M>();
            cudaError_t e = set_smem(k_factor_cta<double, M, 0>, f64);
            if (e == cudaSuccess) e = set_smem(k_factor_cta<double, M, 1>, f64);
            if (e == cudaSuccess) e = set_smem(k_factor_cta<float, M, 0>, f32);
            if (e == cudaSuccess) e = set_smem(k_factor_cta<float, M, 1>, f32);
            if (e == cudaSuccess) e = set_smem(k_factor_cta_batch<double, M, 0>, f64);
            if (e == cudaSuccess) e = set_smem(k_factor_cta_batch<double, M, 1>, f64);
            if (e == cudaSuccess) e = set_smem(k_factor_cta_batch<float, M, 0>, f32);
            if (e == cudaSuccess) e = set_smem(k_factor_cta_batch<float, M, 1>, f32);
            if (e == cudaSuccess) e = set_smem(k_bcr_factor<double, double, double, M>, bcr_factor_smem_bytes<double, M>());
            if (e == cudaSuccess) e = set_smem(k_bcr_rhs<double, M>, bcr_vec_smem_bytes<double, M>());
            if (e == cudaSuccess) e = set_smem(k_bcr_back<double, double, M>, bcr_vec_smem_bytes<double, M>());
            if constexpr (M == 16) {
                if (e == cudaSuccess) e = set_smem(k_factor_w16<0>, factor_w16_smem_bytes());
                if (e == cudaSuccess)
                    e = set_smem(k_solve_fwd_w16<16>, sizeof(WarpS16<16>::Smem) * WarpS16<16>::WARPS);
                if (e == cudaSuccess)
                    e = set_smem(k_solve_bwd_w16<16>, sizeof(WarpS16<16>::Smem) * WarpS16<16>::WARPS);
            }
            return e;
        }
        return cudaSuccess;
    }
    // ------------------------------------------------------ cyclic reduction --
    template <typename K>
    static cudaError_t launch_bcr(K k, size_t smem, const BcrArgs& a, long long ctas, cudaStream_t s) {
        if (ctas <= 0) return cudaSuccess;
        cudaError_t e = set_smem(k, smem);
        if (e != cudaSuccess) return e;
        k<<<(unsigned)ctas, 8 * M, smem, s>>>(a);
        return cudaGetLastError();
    }
    static cudaError_t bcr_factor(const BcrArgs& a, long long ctas, cudaStream_t s) {
        if constexpr (M >= 8) {
            constexpr size_t s64 = bcr_factor_smem_bytes<double, M>(), s32 = bcr_factor_smem_bytes<float, M>();
            switch (a.mode) {
                case BCR_F64: return launch_bcr(k_bcr_factor<double, double, double, M>, s64, a, 2 * ctas, s);
                case BCR_F32_FIRST: return launch_bcr(k_bcr_factor<float, double, float, M>, s32, a, 2 * ctas, s);
                case BCR_F32: return launch_bcr(k_bcr_factor<float, float, float, M>, s32, a, 2 * ctas, s);
                case BCR_F32_LAST: return launch_bcr(k_bcr_factor<float, float, double, M>, s32, a, 2 * ctas, s);
                case BCR_F32_ONLY: return launch_bcr(k_bcr_factor<float, double, double, M>, s32, a, 2 * ctas, s);
                default: return cudaErrorInvalidValue;
            }
        }
        return cudaErrorNotSupported;
    }
    static cudaError_t bcr_rhs(const BcrArgs& a, long long ctas, cudaStream_t s) {
        if constexpr (M >= 8) {
            if (a.mode == BCR_F64) return launch_bcr(k_bcr_rhs<double, M>, bcr_vec_smem_bytes<double, M>(), a, ctas, s);
            return launch_bcr(k_bcr_rhs<float, M>, bcr_vec_smem_bytes<float, M>(), a, ctas, s);
        }
        return cudaErrorNotSupported;
    }
    static cudaError_t bcr_back(const BcrArgs& a, long long ctas, cudaStream_t s) {
        if constexpr (M >= 8) {
            constexpr size_t s64 = bcr_vec_smem_bytes<double, M>(), s32 = bcr_vec_smem_bytes<float, M>();
            if (a.mode == BCR_F64) return launch_bcr(k_bcr_back<double, double, M>, s64, a, ctas, s);
            if (a.mode == BCR_F32_FIRST || a.mode == BCR_F32_ONLY)
                return launch_bcr(k_bcr_back<float, double, M>, s32, a, ctas, s);
            return launch_bcr(k_bcr_back<float, float, M>, s32, a, ctas, s);
        }
        return cudaErrorNotSupported;
    }
    // ------------------------------------------------ BABD cyclic reduction --
    static cudaError_t crb_factor(const CrbArgs& a, cudaStream_t s) {
        if constexpr (M >= 8) {
            constexpr size_t smem = crb_factor_smem_bytes<M>();
            cudaError_t e = set_smem(k_crb_factor<M>, smem);
            if (e != cudaSuccess) return e;
            k_crb_factor<M><<<(unsigned)(a.N - a.N / 2), 8 * M, smem, s>>>(a);
            return cudaGetLastError();
        }
        return cudaErrorNotSupported;
    }
    static cudaError_t crb_rhs(const CrbArgs& a, cudaStream_t s) {
        if constexpr (M >= 8) {
            constexpr size_t smem = crb_vec_smem_bytes<M>();
            cudaError_t e = set_smem(k_crb_rhs<M>, smem);
            if (e != cudaSuccess) return e;
            k_crb_rhs<M><<<(unsigned)(a.N - a.N / 2), 8 * M, smem, s>>>(a);
            return cudaGetLastError();
        }
        return cudaErrorNotSupported;
    }
    static cudaError_t crb_back(const CrbArgs& a, cudaStream_t s) {
        if constexpr (M >= 8) {
            constexpr size_t smem = crb_vec_smem_bytes<M>();
            cudaError_t e = set_smem(k_crb_back<M>, smem);
            if (e != cudaSuccess) return e;
            k_crb_back<M><<<(unsigned)(a.N / 2 + 1), 8 * M, smem, s>>>(a);
            return cudaGetLastError();
        }
        return cudaErrorNotSupported;
    }
    static const Launchers* table() {
        static const Launchers L = {factor, factor_part, M >= 8 ? factor_phase : nullptr, assemble, solve_fwd,
                                    assemble_rhs, solve_bwd,
                                    factor_b, assemble_b, solve_fwd_b, assemble_rhs_b, solve_bwd_b,
                                    M >= 8,
                                    M >= 8 ? factor_smem_bytes<double, M>() : 0,
                                    M >= 8 ? factor_smem_bytes<float, M>() : 0,
                                    M >= 8 ? assemble_smem_bytes<M>() : 0,
                                    M >= 8 ? solve_smem_bytes<double, M>() : 0,
                                    M >= 8 ? solve_smem_bytes<float, M>() : 0,
                                    M >= 8 ? assemble_rhs_smem_bytes<M>() : 0,
                                    prepare,
                                    M >= 8 ? bcr_factor : nullptr,
                                    M >= 8 ? bcr_rhs : nullptr,
                                    M >= 8 ? bcr_back : nullptr,
                                    M >= 8 ? crb_factor : nullptr,
                                    M >= 8 ? crb_rhs : nullptr,
                                    M >= 8 ? crb_back : nullptr,
                                    warp_ok,
                                    M == 16 ? solve_fwd_w : nullptr,
                                    M == 16 ? sep_rhs_w : nullptr,
                                    M == 16 ? solve_bwd_w : nullptr};
        return &L;
    }
};

}  // namespace bt
