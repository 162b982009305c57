// C ABI: plans, the recursion over reduced systems, solves and refinement.
#include <cuda_runtime.h>
#include <cmath>
#include <cstdint>
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/bt.h"
#include "bt_launch.h"
#include "bt_level.h"
#include "bt_misc.h"
#include "bt_planner.h"
#include "bt_bcr.cuh"
#include "bt_crb.cuh"
#include "bt_qr.h"
#include "bt_rsolve.h"

namespace {

using bt::LevelArgs;

constexpr int kNrhsMax = 32;
constexpr int kSlotWords = 3 * bt::kMaxSlots;        // words of one maxima slot array
constexpr int kNormWords = 4;                        // ||d||^2, ||x||^2 of the last correction and of the one before
constexpr int kHostNorms = kNormWords + 2 * kSlotWords;   // pinned host copy: norms, rmax, amax

struct Level {
    LevelArgs a;
    bool low = false;   // local factors in FP32
    long long rows = 0; // block rows stored for this level (BABD: N+1)
    long long pcap = 0; // partitions the level's buffers hold (pivoted level 0: room for splits)
};

}  // namespace

struct bt_plan_s {
    int kind = 0;   // 0 block tridiagonal, 1 BABD
    long long N = 0;
    int m = 0;          // block order the kernels run at (1, 2, 4, 8, 16 or 32)
    int mu = 0;         // block order of the caller's arrays (m >= mu; padded when larger)
    int nrhs_max = 0;
    int prec = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    const bt::Launchers* L = nullptr;
    std::vector<Level> lv;   // lv[0..nlev-1] partitioned levels; lv[nlev] the top
    int nlev = 0;
    bool factored = false;
    // caller's matrices (kept by reference)
    const double* A0 = nullptr;  // B or S
    const double* A1 = nullptr;  // D or R
    const double* A2 = nullptr;  // C
    // device memory
    char* arena = nullptr;
    size_t arena_bytes = 0;
    bool own_arena = true;
    bool pinned = true;
    long long* status = nullptr;
    long long* status_host = nullptr;   // pinned
    double* norms = nullptr;            // [4] ||d||^2, ||x||^2 of the last correction, then of the one
                                        // before it (NaN: none)
    double* norms_host = nullptr;       // pinned: [2] norms, then the rmax and amax slots
    unsigned long long* rmax = nullptr; // [kMaxSlots][3] max |r|, |x|, |f| of the last residual (bit patterns)
    unsigned long long* amax = nullptr; // [kMaxSlots][3] ||A||_inf (bit pattern) in word 0
    bool anorm_valid = false;
    bool anorm_fac = false;             // ||A||_inf was taken by the last level-0 factorization
    int async_sweeps = 0;
    double eta_tol = -1.0;              // backward-error stopping threshold (< 0: default)
    double fwd_tol = -1.0;              // estimated forward-error stopping threshold (<= 0: not used)
    double* partial = nullptr;          // [2*1024]
    double* Rbuf = nullptr;
    double* Dbuf = nullptr;
    double* B0 = nullptr;               // BABD boundary blocks (copies)
    double* B1 = nullptr;
    double* keep = nullptr;             // BABD top-level pivot rows
    bool bcr = false;                   // reduced system by block cyclic reduction
    int local = 0;                      // level-0 local cyclic-reduction steps (plans without partition levels)
    // pivoted partitions: level 0 split at breakdown rows, reduced system by banded GEPP
    bool pivot = false;
    double pivot_tau = 1e-3;
    // partitions factored by local QR (pivot = 2): no splits, reduced system by banded GEPP
    bool qr = false;
    bt::QrArgs qa{};
    long long p_init = 0, base_init = 0, extra_init = 0;
    long long* starts_dev = nullptr;    // [pcap+1]
    long long* brk_dev = nullptr;       // [1 + brk_cap]: breakdown count and rows
    long long brk_cap = 0;
    std::vector<long long> starts_host, brk_host;
    // circulant-like plans: a BABD plan of N-1 steps with the right-hand side rotated
    bool cyclic = false;
    double* rot = nullptr;              // [(N+1)*m][nrhs_max] rotated right-hand side
    double* rot2 = nullptr;             // the same for residuals
    bool padded = false;                // caller blocks of order mu embedded in order m
    double* Ap[3] = {nullptr, nullptr, nullptr};   // padded matrices (B/S, D/R, C)
    double* Fp = nullptr;               // padded right-hand side / solution / residual
    double* Xp = nullptr;
    double* Rp = nullptr;
    const double* U[4] = {nullptr, nullptr, nullptr, nullptr};   // caller matrices of a padded plan
    std::vector<bt::BcrArgs> bl;        // its levels
    // refined plans: the reduced system's cyclic-reduction factors are also kept
    // in FP32 and the correction solves apply them in one cluster launch
    bool rs32 = false;
    // refined plans of order 16: level-0 factors and solves on the warp-per-partition
    // kernels (when the matrices start on 16-byte boundaries; bt_warp.cuh)
    bool warp = false;
    bt::RsolveArgs rsa{};
    bt::CvtArgs cva{};
    // refined plans of order 8 or 16: the reduced system's FP32 cyclic
    // reduction in one cluster launch
    bool rf = false;
    bt::RfactorArgs rfa{};
    // BABD plans solved by cyclic reduction of the whole system (no partitions)
    bool crb = false;
    std::vector<bt::CrbArgs> cl;        // its levels (N_q rows each, down to one row)
    const double* crb_top[4] = {nullptr, nullptr, nullptr, nullptr};   // S, R, F, X of the last row
    double* crb_topx = nullptr;
    // captured call sequence
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    long long graph_launches = 0;
    // captured factor+solve sequences: the factorization of levels >= 1 (and
    // the reduced system's cyclic reduction) runs on a second stream, beside
    // the level-0 forward substitution, which needs only the level-0 factors
    bool serial = false;                // captured sequences on one stream
    bool overlap = false;
    bool join_pending = false;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // host-buffer entry point: device copies of the caller's arrays, a copy
    // stream and per-chunk streams on which the level-0 factorization of each
    // chunk of partitions starts as soon as its rows have arrived
    static constexpr int kChunks = 8;
    static constexpr int kPhases = 4;   // row slabs of the block kernels' host path
    double* hb = nullptr;               // B, D, C [N m m] each, then F, X [N m nrhs_max]
    cudaStream_t copy_stream = nullptr;
    cudaStream_t chunk_stream[kChunks] = {};
    cudaEvent_t ev_in = nullptr, ev_rhs = nullptr;
    // host-array path: the solution is final (the last correction added) / copied out
    cudaEvent_t ev_xfinal = nullptr, ev_xout = nullptr;
    bool x_event = false;   // run_refine_async records ev_xfinal before the checking residual
    cudaEvent_t ev_rows[kChunks] = {}, ev_part[kChunks] = {};
    // tracing
    bool trace = false;
    struct Rec { int key; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
    long long launches = 0;
};

namespace {

struct Arena {
    size_t off = 0;
    char* base = nullptr;
    void* take(size_t bytes) {
        off = (off + 255) & ~size_t(255);
        void* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    }
};

bt_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return BT_OK;
    if (e == cudaErrorMemoryAllocation) return BT_ERR_NOMEM;
    return BT_ERR_CUDA;
}

int sm_count(int dev) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    return n;
}

// Lay out (or measure, when ar.base == nullptr) the plan's device memory.
void layout(bt_plan_s* P, Arena& ar) {
    const int m = P->m;
    const long long mm = (long long)m * m;
    const int nr = P->nrhs_max;
    P->status = (long long*)ar.take(4 * sizeof(long long));
    P->norms = (double*)ar.take(kNormWords * sizeof(double));
    P->rmax = (unsigned long long*)ar.take(kSlotWords * sizeof(unsigned long long));
    P->amax = (unsigned long long*)ar.take(kSlotWords * sizeof(unsigned long long));
    P->partial = (double*)ar.take(2 * 1024 * sizeof(double));
    const long long rows0 = P->lv[0].rows;
    P->Rbuf = (double*)ar.take(sizeof(double) * rows0 * m * nr);
    P->Dbuf = (double*)ar.take(sizeof(double) * rows0 * m * nr);
    if (P->kind == 1) {
        P->B0 = (double*)ar.take(sizeof(double) * mm);
        P->B1 = (double*)ar.take(sizeof(double) * mm);
    }
    if (P->padded) {
        for (int k = 0; k < (P->kind == 0 ? 3 : 2); ++k) P->Ap[k] = (double*)ar.take(sizeof(double) * P->N * mm);
        P->Fp = (double*)ar.take(sizeof(double) * rows0 * m * nr);
        P->Xp = (double*)ar.take(sizeof(double) * rows0 * m * nr);
        P->Rp = (double*)ar.take(sizeof(double) * rows0 * m * nr);
    }
    if (P->warp) {
        // warp-per-partition FP32 kernels at level 0: W chain, h_j and sum_j W_j h_j
        Level& v0 = P->lv[0];
        const long long pa = std::max(v0.a.p, v0.pcap);
        v0.a.W = ar.take(sizeof(float) * rows0 * mm);
        v0.a.Hv = ar.take(sizeof(float) * rows0 * m * nr);
        v0.a.Hw = ar.take(sizeof(float) * pa * m * nr);
        v0.a.As = ar.take(2 * sizeof(float) * 3 * rows0 * mm);
        v0.a.nrm = (double*)ar.take(sizeof(double) * 2 * pa);
    }
    for (int l = 0; l <= P->nlev; ++l) {
        Level& v = P->lv[l];
        const size_t ts = v.low ? sizeof(float) : sizeof(double);
        const bool top = (l == P->nlev);
        const bool holder = top && (P->bcr || P->pivot);
        if (l == 0 && P->qr) {
            // local QR factors (bt_qr.h)
            bt::QrArgs& q = P->qa;
            const long long pa = v.a.p;
            q.Qt = (double*)ar.take(sizeof(double) * v.rows * 4 * mm);
            q.R = (double*)ar.take(sizeof(double) * v.rows * 3 * mm);
            q.Z = (double*)ar.take(sizeof(double) * v.rows * mm);
            q.W = (double*)ar.take(sizeof(double) * v.rows * mm);
            q.Vb = (double*)ar.take(sizeof(double) * pa * mm);
            q.Ta = (double*)ar.take(sizeof(double) * pa * mm);
            q.Tf = (double*)ar.take(sizeof(double) * pa * m * nr);
        } else if (!(top && P->kind == 1) && !holder) {
            const long long pa = std::max(v.a.p, v.pcap);
            v.a.Dinv = ar.take(ts * v.rows * mm);
            if (P->kind == 0) v.a.Y = ar.take(ts * v.rows * mm);
            v.a.Zc = ar.take(ts * v.rows * mm);
            if (P->kind == 0) {
                v.a.Pf = ar.take(ts * pa * mm);
                v.a.Qf = ar.take(ts * pa * mm);
                v.a.Hf = ar.take(ts * pa * m * nr);
            }
        }
        if (l >= 1) {
            // this level's matrix and vectors are owned by the plan
            Level& u = P->lv[l - 1];
            if (P->kind == 0) {
                double* Bn = (double*)ar.take(sizeof(double) * v.rows * mm);
                double* Dn = (double*)ar.take(sizeof(double) * v.rows * mm);
                double* Cn = (double*)ar.take(sizeof(double) * v.rows * mm);
                u.a.Bn = Bn; u.a.Dn = Dn; u.a.Cn = Cn;
                v.a.B = Bn; v.a.D = Dn; v.a.C = Cn;
                v.a.shift = 0;
            } else {
                // reduced BABD of p rows + boundary row: S', R' hold p blocks
                double* Sn = (double*)ar.take(sizeof(double) * u.a.p * mm);
                double* Rn = (double*)ar.take(sizeof(double) * u.a.p * mm);
                u.a.Bn = Sn; u.a.Dn = Rn;
                v.a.B = Sn; v.a.D = Rn;
                v.a.shift = 1;
            }
            double* Fn = (double*)ar.take(sizeof(double) * v.rows * m * nr);
            double* Xn = (double*)ar.take(sizeof(double) * v.rows * m * nr);
            u.a.Fn = Fn;
            u.a.Xn = Xn;
            v.a.F = Fn;
            v.a.X = Xn;
        }
        if (top && P->kind == 1)
            P->keep = (double*)ar.take(sizeof(double) * (P->crb ? 1 : v.a.N) * m * (3 * m + nr) + 8);
        if (top && P->pivot) P->keep = (double*)ar.take(sizeof(double) * v.rows * m * (3 * m + nr) + 8);
    }
    if (P->crb) {
        const long long vb = (long long)m * nr;
        for (size_t q = 0; q < P->cl.size(); ++q) {
            bt::CrbArgs& c = P->cl[q];
            const long long pairs = c.N / 2, nn = c.N - pairs;
            c.Rinv = (double*)ar.take(sizeof(double) * pairs * mm);
            c.T = (double*)ar.take(sizeof(double) * pairs * mm);
            c.Sn = (double*)ar.take(sizeof(double) * nn * mm);
            c.Rn = (double*)ar.take(sizeof(double) * nn * mm);
            c.U = (double*)ar.take(sizeof(double) * pairs * vb);
            c.Fn = (double*)ar.take(sizeof(double) * (nn + 1) * vb);
            double* xn = (double*)ar.take(sizeof(double) * (nn + 1) * vb);
            c.Xn = xn;
            if (q + 1 < P->cl.size()) {
                P->cl[q + 1].S = c.Sn;
                P->cl[q + 1].R = c.Rn;
                P->cl[q + 1].F = c.Fn;
                P->cl[q + 1].X = xn;
            } else {
                P->crb_top[0] = c.Sn;
                P->crb_top[1] = c.Rn;
                P->crb_top[2] = c.Fn;
                P->crb_topx = xn;
            }
        }
    }
    if (P->kind == 1) {
        // room for a rotated right-hand side (circulant-like plans)
        P->rot = (double*)ar.take(sizeof(double) * rows0 * m * nr);
        P->rot2 = (double*)ar.take(sizeof(double) * rows0 * m * nr);
    }
    if (P->pivot && !P->qr) {
        const long long pc = P->lv[0].pcap;
        P->starts_dev = (long long*)ar.take(sizeof(long long) * (pc + 1));
        P->brk_cap = 4 * pc;
        P->brk_dev = (long long*)ar.take(sizeof(long long) * (P->brk_cap + 1));
        P->lv[0].a.starts = P->starts_dev;
    }
    if (P->bcr) {
        Level& h = P->lv[P->nlev];
        long long K = h.a.N;
        for (size_t q = 0; q < P->bl.size(); ++q) {
            bt::BcrArgs& b = P->bl[q];
            b.K = K;
            b.level = P->nlev + (int)q;
            b.nr = nr;
            // factor storage in the level's arithmetic type, the next level's
            // matrix in its input type
            const int md = b.mode;
            const size_t tsz = (md == bt::BCR_F64) ? sizeof(double) : sizeof(float);
            const size_t osz = (md == bt::BCR_F32_FIRST || md == bt::BCR_F32) ? sizeof(float) : sizeof(double);
            const long long keep = (K + 1) / 2, odd = (K == 1) ? 1 : K / 2;
            if (q == 0) {
                b.B = h.a.B; b.D = h.a.D; b.C = h.a.C;
                b.F = h.a.F; b.X = h.a.X;
            }
            b.Dinv = ar.take(tsz * odd * mm);
            if (K > 1) {
                b.al = ar.take(tsz * keep * mm);
                b.ga = ar.take(tsz * keep * mm);
                bt::BcrArgs& n = P->bl[q + 1];
                b.Bn = ar.take(osz * keep * mm);
                b.Dn = ar.take(osz * keep * mm);
                b.Cn = ar.take(osz * keep * mm);
                b.Fn = (double*)ar.take(sizeof(double) * keep * m * nr);
                double* Xn = (double*)ar.take(sizeof(double) * keep * m * nr);
                b.Xn = Xn;
                n.B = b.Bn; n.D = b.Dn; n.C = b.Cn; n.F = b.Fn; n.X = Xn;
            }
            K = keep;
        }
    }
    if (P->rs32) {
        bt::RsolveArgs& r = P->rsa;
        bt::CvtArgs& c = P->cva;
        r.nlev = (int)P->bl.size();
        r.m = m;
        r.nr = nr;
        c.nseg = 0;
        auto seg = [&](const void* src, long long n) {
            float* d = (float*)ar.take(sizeof(float) * n);
            if (c.nseg < bt::kCvtSegs) {
                c.src[c.nseg] = (const double*)src;
                c.dst[c.nseg] = d;
                c.n[c.nseg] = n;
                ++c.nseg;
            }
            return (const float*)d;
        };
        for (size_t q = 0; q < P->bl.size(); ++q) {
            const bt::BcrArgs& b = P->bl[q];
            const long long K = b.K, kept = (K + 1) / 2, odd = (K == 1) ? 1 : K / 2;
            r.K[q] = K;
            if (b.mode == bt::BCR_F64) {
                r.al[q] = (K > 1) ? seg(b.al, kept * mm) : nullptr;
                r.ga[q] = (K > 1) ? seg(b.ga, kept * mm) : nullptr;
                r.Dinv[q] = seg(b.Dinv, odd * mm);
            } else {
                // FP32 factors, used as they are
                r.al[q] = (const float*)b.al;
                r.ga[q] = (const float*)b.ga;
                r.Dinv[q] = (const float*)b.Dinv;
            }
            // the level matrix: FP64 at the first level (the partition level's
            // output), FP32 above it when the levels are FP32
            const bool in64 = (b.mode == bt::BCR_F64) || q == 0;
            r.B[q] = (K > 1) ? (in64 ? seg(b.B, K * mm) : (const float*)b.B) : nullptr;
            r.C[q] = (K > 1) ? (in64 ? seg(b.C, K * mm) : (const float*)b.C) : nullptr;
            r.f[q] = (float*)ar.take(sizeof(float) * K * m * nr);
            r.x[q] = (float*)ar.take(sizeof(float) * K * m * nr);
        }
        r.F0 = P->bl[0].F;
        r.X0 = P->bl[0].X;
        if (P->rf) {
            bt::RfactorArgs& f = P->rfa;
            f.nlev = (int)P->bl.size();
            f.m = m;
            f.level0 = P->nlev;
            f.B0 = (const double*)P->bl[0].B;
            f.D0 = (const double*)P->bl[0].D;
            f.C0 = (const double*)P->bl[0].C;
            for (size_t q = 0; q < P->bl.size(); ++q) {
                const bt::BcrArgs& b = P->bl[q];
                f.K[q] = b.K;
                f.B[q] = q ? (float*)b.B : nullptr;
                f.D[q] = q ? (float*)b.D : nullptr;
                f.C[q] = q ? (float*)b.C : nullptr;
                f.al[q] = (float*)b.al;
                f.ga[q] = (float*)b.ga;
                f.Dinv[q] = (float*)b.Dinv;
            }
            f.B0f = const_cast<float*>(r.B[0]);
            f.C0f = const_cast<float*>(r.C[0]);
        }
    }
}

bt_status plan_create(bt_plan* out, int kind, int64_t N, int m, int nrhs_max, int prec, const bt::Tuning& tune,
                      void* stream, void* workspace = nullptr, int64_t ws_bytes = 0, int64_t* need_bytes = nullptr) {
    const int64_t p = tune.p0;
    if (!out) return BT_ERR_INVALID;
    *out = nullptr;
    const int mu = m;
    if (m >= 1 && m <= 32) {
        int M = 1;
        while (M < m) M *= 2;
        m = M;
    }
    const bt::Launchers* L = bt::launchers_for(m);
    if (!L || nrhs_max < 1 || nrhs_max > kNrhsMax || prec < 0 || prec > 2 || p < 0) return BT_ERR_INVALID;
    if (kind == 0 && N < 1) return BT_ERR_INVALID;
    if (kind == 1 && N < 1) return BT_ERR_INVALID;
    if (kind == 0 && p > (N + 1) / 2 && p > 1) return BT_ERR_INVALID;
    if (kind == 1 && p > 0 && p > (N - 1) / 2 && p > 1) return BT_ERR_INVALID;
    bt_plan_s* P = new (std::nothrow) bt_plan_s();
    if (!P) return BT_ERR_NOMEM;
    P->kind = kind;
    P->N = N;
    P->m = m;
    P->mu = mu;
    P->padded = (mu != m);
    P->nrhs_max = nrhs_max;
    P->prec = prec;
    P->stream = (cudaStream_t)stream;
    P->L = L;
    cudaGetDevice(&P->device);
    const int sms = sm_count(P->device);
    std::vector<bt::LevelShape> shapes;
    P->pivot = (kind == 0 && tune.pivot > 0);
    P->qr = P->pivot && tune.pivot == 2;
    P->serial = tune.serial > 0;
    if (P->qr && prec != BT_FP64) {
        delete P;
        return BT_ERR_INVALID;
    }
    bt::Tuning tsh = tune;
    if (P->pivot) {
        tsh.reduced = 0;
        tsh.local = 0;
    }
    P->crb = (kind == 1 && tune.reduced == 1);
    if (P->crb) {
        // cyclic reduction of the whole BABD system: blocks of order 8, 16 or 32, FP64
        if (mu != m || m < 8 || prec != BT_FP64) {
            delete P;
            return BT_ERR_INVALID;
        }
        shapes.assign(1, bt::LevelShape{N, 0, 0, 0, N + 1});
        long long n = N;
        while (n > 1) {
            bt::CrbArgs c{};
            c.N = n;
            c.level = (int)P->cl.size();
            P->cl.push_back(c);
            n -= n / 2;
        }
    } else if (!bt::plan_shapes(kind, N, m, sms, tsh, shapes)) {
        delete P;
        return BT_ERR_INVALID;
    }
    long long pcap = 0;
    if (P->pivot) {
        // level 0 as planned; its reduced system (which breakdown splits may
        // enlarge up to pcap - 1 block rows) by the pivoted direct solver
        const bt::LevelShape s0 = shapes[0];
        shapes.resize(1);
        pcap = P->qr ? s0.p : std::min<long long>(N + 1, std::max<long long>(2 * s0.p, N / 16) + 16);
        shapes.push_back(bt::LevelShape{s0.p - 1, 0, 0, 0, std::max<long long>(pcap - 1, 1)});
        P->p_init = s0.p;
        P->base_init = s0.base;
        P->extra_init = s0.extra;
    }
    for (size_t l = 0; l < shapes.size(); ++l) {
        Level v;
        std::memset(&v.a, 0, sizeof(LevelArgs));
        v.a.mode = kind;
        v.a.level = (int)l;
        v.a.N = shapes[l].N;
        v.a.p = shapes[l].p;
        v.a.base = shapes[l].base;
        v.a.extra = shapes[l].extra;
        v.rows = shapes[l].rows;
        v.low = (l == 0) && (prec != BT_FP64);
        v.a.bf16 = (l == 0) && (prec == BT_BF16_IR) && (m >= 16) ? 1 : 0;
        v.a.tpb = tune.tp_block;
        // m = 2, 4 FP64 levels with fewer partitions than lanes of a full thread-per-partition
        // wave: one group of m*m lanes per partition (latency-bound levels)
        v.a.group = ((m == 2 || m == 4) && !v.low && !(P->pivot && l == 0) &&
                     v.a.p < (long long)sms * 128) ? 1 : 0;
        if (P->pivot && l == 0) v.pcap = pcap;
        P->lv.push_back(v);
    }
    P->nlev = (int)P->lv.size() - 1;
    P->warp = (kind == 0) && (m == 16) && (prec == BT_FP32_IR) && !P->pivot && tune.local == 0 && P->lv[0].low;
    P->bcr = !P->pivot && (kind == 0 && P->lv[P->nlev].a.p == 0 && (P->nlev >= 1 || tune.local > 0));
    if (P->bcr) {
        long long K = P->lv[P->nlev].a.N;
        int n = 1;
        while (K > 1) {
            K = (K + 1) / 2;
            ++n;
        }
        P->bl.assign(n, bt::BcrArgs{});
        // local cyclic-reduction steps (level 0 only): at least the last row stays FP64
        P->local = (P->nlev == 0) ? std::min(tune.local, n - 1) : 0;
        const bool lo = prec != BT_FP64;
        for (int q = 0; q < n; ++q) {
            int mode = bt::BCR_F64;
            if (lo && q < P->local) {
                if (P->local == 1) mode = bt::BCR_F32_ONLY;
                else if (q == 0) mode = bt::BCR_F32_FIRST;
                else if (q == P->local - 1) mode = bt::BCR_F32_LAST;
                else mode = bt::BCR_F32;
            }
            P->bl[q].mode = mode;
        }
        P->rs32 = (prec != BT_FP64) && P->local == 0 && P->nlev >= 1 && m >= 8 &&
                  (int)P->bl.size() <= bt::kRsMaxLevels && 5 * (int)P->bl.size() <= bt::kCvtSegs;
        if (P->rs32) {
            // the reduced system of a refined plan is factored in FP32 too: its
            // factors only enter the FP32 correction solves
            for (int q = 0; q < n; ++q)
                P->bl[q].mode = (q > 0) ? bt::BCR_F32 : (n == 1 ? bt::BCR_F32_ONLY : bt::BCR_F32_FIRST);
            P->rf = (m == 8 || m == 16) && n >= 2;
        }
    }
    if (kind == 0) {
        // the top level is a single partition; levels below it have >= 2
    }
    Arena meas;
    layout(P, meas);
    size_t bytes = meas.off + 256;
    if (need_bytes) {
        *need_bytes = (int64_t)bytes;
        delete P;
        return BT_OK;
    }
    cudaError_t e = cudaSuccess;
    if (workspace) {
        if (ws_bytes < (int64_t)bytes || ((uintptr_t)workspace & 255u)) {
            delete P;
            return BT_ERR_INVALID;
        }
        P->arena = (char*)workspace;
        P->own_arena = false;
        P->pinned = false;
    } else {
        e = cudaMalloc((void**)&P->arena, bytes);
        if (e != cudaSuccess) {
            delete P;
            cudaGetLastError();
            return from_cuda(e);
        }
    }
    P->arena_bytes = bytes;
    Arena real;
    real.base = P->arena;
    layout(P, real);
    for (auto& v : P->lv) v.a.status = P->status;
    for (auto& b : P->bl) b.status = P->status;
    for (auto& c : P->cl) c.status = P->status;
    if (P->pinned) {
        e = cudaMallocHost((void**)&P->status_host, 4 * sizeof(long long));
        if (e == cudaSuccess) e = cudaMallocHost((void**)&P->norms_host, kHostNorms * sizeof(double));
    } else {
        P->status_host = new (std::nothrow) long long[4];
        P->norms_host = new (std::nothrow) double[kHostNorms];
        if (!P->status_host || !P->norms_host) e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(P->status, 0, 4 * sizeof(long long), P->stream);
    if (e == cudaSuccess && P->qr) e = bt::qr_prepare(m);
    // the split copy of the matrix: blocks B_0 and C_{N-1} are never written and stay zero
    if (e == cudaSuccess && P->warp && P->lv[0].a.As)
        e = cudaMemsetAsync(P->lv[0].a.As, 0, 2 * sizeof(float) * 3 * P->lv[0].rows * (size_t)m * m, P->stream);
    if (e != cudaSuccess) {
        if (P->own_arena) cudaFree(P->arena);
        if (P->pinned) {
            if (P->status_host) cudaFreeHost(P->status_host);
            if (P->norms_host) cudaFreeHost(P->norms_host);
        } else {
            delete[] P->status_host;
            delete[] P->norms_host;
        }
        delete P;
        return from_cuda(e);
    }
    *out = P;
    return BT_OK;
}

enum Kind { K_FACTOR = 0, K_ASSEMBLE, K_SOLVE_FWD, K_ASSEMBLE_RHS, K_SOLVE_BWD, K_DIRECT, K_RESID, K_IR, K_BCR_FACTOR,
            K_BCR_SOLVE, K_NORM };

cudaEvent_t take_event(bt_plan_s* P) {
    if (P->pool_used == P->pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        P->pool.push_back(e);
    }
    return P->pool[P->pool_used++];
}

// Launch through f(), counting kernels and bracketing them with events when tracing.
template <typename Fn>
cudaError_t launch(bt_plan_s* P, int kind, int level, int nkernels, Fn&& f) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (P->trace) {
        a = take_event(P);
        b = take_event(P);
        if (a) cudaEventRecord(a, P->stream);
    }
    cudaError_t e = f();
    if (P->trace && a && b) {
        cudaEventRecord(b, P->stream);
        P->recs.push_back({kind * 64 + (level < 63 ? level : 63), a, b});
    }
    P->launches += nkernels;
    return e;
}

bt_status read_status(bt_plan_s* P) {
    cudaError_t e = cudaMemcpyAsync(P->status_host, P->status, 4 * sizeof(long long), cudaMemcpyDeviceToHost,
                                    P->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) return from_cuda(e);
    const long long c = P->status_host[0];
    if (c == 0) return BT_OK;
    return (bt_status)c;
}

// Factor every level: local factorizations and reduced systems.
// Pivoted partitions (the variant of Sec. 2 for matrices whose local blocks may
// be singular or ill-conditioned): factor level 0; every partition whose local
// factorization broke down at some block row (a pivot below tau times the
// largest entry of the row's blocks) is split there, that row becoming one
// more separator of the reduced system; repeat until no partition breaks
// down.  The reduced system (at most pcap - 1 block rows) is solved by banded
// GEPP at solve time.  One host synchronisation per pass.
bt_status run_factor_pivoted(bt_plan_s* P) {
    const bt::Launchers* L = P->L;
    Level& v = P->lv[0];
    Level& t = P->lv[1];
    const long long N = v.a.N, pcap = v.pcap;
    long long p = P->p_init;
    std::vector<long long>& st = P->starts_host;
    st.assign(p + 1, 0);
    for (long long i = 0; i < p; ++i) st[i] = i * P->base_init + std::min(i, P->extra_init);
    st[p] = N;
    v.a.brk = P->brk_dev;
    v.a.brk_cap = P->brk_cap;
    v.a.tau = P->pivot_tau;
    bt_status res = BT_OK;
    for (int pass = 0;; ++pass) {
        v.a.p = p;
        t.a.N = p - 1;
        cudaError_t e = cudaMemcpyAsync(P->starts_dev, st.data(), sizeof(long long) * (p + 1),
                                        cudaMemcpyHostToDevice, P->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(P->brk_dev, 0, sizeof(long long), P->stream);
        if (e == cudaSuccess) e = launch(P, K_FACTOR, 0, 1, [&] { return L->factor(v.a, v.low, P->stream); });
        P->brk_host.assign(P->brk_cap + 1, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(P->brk_host.data(), P->brk_dev, sizeof(long long) * (P->brk_cap + 1),
                                cudaMemcpyDeviceToHost, P->stream);
        if (e != cudaSuccess) return from_cuda(e);
        bt_status sst = read_status(P);   // synchronises
        if (sst != BT_OK) return sst;
        const long long cnt = std::min(P->brk_host[0], P->brk_cap);
        if (cnt == 0) break;
        std::vector<long long> rows(P->brk_host.begin() + 1, P->brk_host.begin() + 1 + cnt);
        std::sort(rows.begin(), rows.end());
        rows.erase(std::unique(rows.begin(), rows.end()), rows.end());
        // every breakdown row closes a partition as its separator: new start j + 1
        std::vector<long long> nst(st.begin(), st.end() - 1);
        for (long long j : rows) nst.push_back(j + 1);
        std::sort(nst.begin(), nst.end());
        nst.push_back(N);
        const long long np = (long long)nst.size() - 1;
        if (np > pcap || pass > 64) {
            // more breakdowns than the reduced system has room for
            res = BT_ERR_SINGULAR;
            break;
        }
        st.swap(nst);
        p = np;
    }
    v.a.brk = nullptr;
    if (res != BT_OK) {
        // the status word carries it for bt_info / the next synchronising call
        long long code[4] = {BT_ERR_SINGULAR, 0, -1, -1};
        cudaMemcpyAsync(P->status, code, sizeof(code), cudaMemcpyHostToDevice, P->stream);
        cudaStreamSynchronize(P->stream);
        return res;
    }
    cudaError_t e = launch(P, K_ASSEMBLE, 0, 1, [&] { return L->assemble(v.a, v.low, P->stream); });
    return from_cuda(e);
}

// The QR arguments of level 0 and its reduced system for nr right-hand sides.
bt::QrArgs& qr_args(bt_plan_s* P, int nr) {
    bt::QrArgs& q = P->qa;
    const Level& v = P->lv[0];
    const Level& t = P->lv[1];
    q.N = v.a.N;
    q.p = v.a.p;
    q.base = v.a.base;
    q.extra = v.a.extra;
    q.m = P->m;
    q.nr = nr;
    q.B = v.a.B;
    q.D = v.a.D;
    q.C = v.a.C;
    q.Bn = v.a.Bn;
    q.Dn = v.a.Dn;
    q.Cn = v.a.Cn;
    q.F = v.a.F;
    q.X = v.a.X;
    q.Fn = v.a.Fn;
    q.Xn = t.a.X;
    q.status = P->status;
    return q;
}

// Partitions factored by local QR: one launch for every partition, one that
// completes the reduced diagonal; no host synchronisation.
bt_status run_factor_qr(bt_plan_s* P) {
    bt::QrArgs& q = qr_args(P, 1);
    cudaError_t e = launch(P, K_FACTOR, 0, 2, [&] { return bt::launch_qr_factor(q, P->stream); });
    return from_cuda(e);
}

bt_status run_factor(bt_plan_s* P, bool level0_done = false) {
    if (P->qr) return run_factor_qr(P);
    if (P->pivot) return run_factor_pivoted(P);
    if (P->crb) {
        // cyclic reduction of the whole BABD system, level by level
        if (!P->cl.empty()) {
            P->cl[0].S = P->A0;
            P->cl[0].R = P->A1;
        }
        for (auto& c : P->cl) {
            cudaError_t e = launch(P, K_FACTOR, c.level, 1, [&] { return P->L->crb_factor(c, P->stream); });
            if (e != cudaSuccess) return from_cuda(e);
        }
        return BT_OK;
    }
    const bt::Launchers* L = P->L;
    const bool split = P->overlap && P->side && P->nlev >= 1;
    cudaStream_t main_stream = P->stream;
    // levels >= 1 on the side stream when split; rejoined by run_solve after level 0
    auto rejoin = [&](bt_status st) {
        if (P->stream != main_stream) {
            cudaError_t e = cudaEventRecord(P->ev_join, P->stream);
            P->stream = main_stream;
            if (e != cudaSuccess) return from_cuda(e);
            P->join_pending = true;
        }
        return st;
    };
    for (int l = 0; l <= P->nlev; ++l) {
        Level& v = P->lv[l];
        if (split && l == 1) {
            cudaError_t e = cudaEventRecord(P->ev_fork, main_stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(P->side, P->ev_fork, 0);
            if (e != cudaSuccess) return from_cuda(e);
            P->stream = P->side;
        }
        if (P->kind == 1 && l == P->nlev) break;   // BABD top: direct solve at solve time
        if (P->bcr && l == P->nlev) {
            // block cyclic reduction of the reduced system (or of the whole
            // matrix: local cyclic reduction, then the reduced system)
            if (P->nlev == 0) {
                P->bl[0].B = v.a.B;
                P->bl[0].D = v.a.D;
                P->bl[0].C = v.a.C;
            }
            if (P->rf) {
                P->rfa.status = P->status;
                cudaError_t e = launch(P, K_BCR_FACTOR, P->nlev, 1,
                                       [&] { return bt::launch_rfactor_f32(P->rfa, P->stream); });
                if (e != cudaSuccess) return rejoin(from_cuda(e));
                break;
            }
            for (size_t q = 0; q < P->bl.size(); ++q) {
                bt::BcrArgs& b = P->bl[q];
                const long long ctas = (b.K == 1) ? 1 : (b.K + 1) / 2;
                cudaError_t e =
                    launch(P, K_BCR_FACTOR, b.level, 1, [&] { return L->bcr_factor(b, ctas, P->stream); });
                if (e != cudaSuccess) return rejoin(from_cuda(e));
            }
            if (P->rs32) {
                cudaError_t e = launch(P, K_BCR_FACTOR, P->nlev, 1, [&] { return bt::launch_cvt_f32(P->cva, P->stream); });
                if (e != cudaSuccess) return rejoin(from_cuda(e));
            }
            break;
        }
        cudaError_t e = cudaSuccess;
        // warp kernels at level 0 take ||A||_inf while they convert the rows
        const bool wn = (l == 0) && !level0_done && P->warp && L->warp_ok && L->warp_ok(v.a, v.low);
        if (l == 0 && !level0_done) P->anorm_fac = false;
        if (wn) {
            e = cudaMemsetAsync(P->amax, 0, kSlotWords * sizeof(unsigned long long), P->stream);
            v.a.amax = P->amax;
        }
        if (e == cudaSuccess && !(l == 0 && level0_done))
            e = launch(P, K_FACTOR, l, 1, [&] { return L->factor(v.a, v.low, P->stream); });
        v.a.amax = nullptr;
        if (wn && e == cudaSuccess) {
            P->anorm_valid = true;
            P->anorm_fac = true;
        }
        if (e == cudaSuccess && P->kind == 0 && l < P->nlev)
            e = launch(P, K_ASSEMBLE, l, 1, [&] { return L->assemble(v.a, v.low, P->stream); });
        if (e != cudaSuccess) return rejoin(from_cuda(e));
    }
    return rejoin(BT_OK);
}

// Second stream for the factorization of levels >= 1 (captured sequences and
// the host-buffer entry point), created on first use.
cudaError_t ensure_side(bt_plan_s* P) {
    if (P->pivot || P->serial || P->nlev < 1 || P->side) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming);
    return e;
}

// The main stream waits for a factorization left running on the side stream.
cudaError_t join_factor(bt_plan_s* P) {
    if (!P->join_pending) return cudaSuccess;
    P->join_pending = false;
    return cudaStreamWaitEvent(P->stream, P->ev_join, 0);
}

// Solve with the factors: F (level-0 rhs) -> X.
bt_status run_solve(bt_plan_s* P, const double* F, double* X, int nr) {
    const bt::Launchers* L = P->L;
    if (P->crb) {
        cudaError_t e = cudaSuccess;
        if (!P->cl.empty()) {
            P->cl[0].F = F;
            P->cl[0].X = X;
        }
        for (auto& c : P->cl) {
            c.nr = nr;
            if (e == cudaSuccess) e = launch(P, K_SOLVE_FWD, c.level, 1, [&] { return L->crb_rhs(c, P->stream); });
        }
        // one row left: with the boundary row, a 2m x 2m system
        const double* tS = P->cl.empty() ? P->A0 : P->crb_top[0];
        const double* tR = P->cl.empty() ? P->A1 : P->crb_top[1];
        const double* tF = P->cl.empty() ? F : P->crb_top[2];
        double* tX = P->cl.empty() ? X : P->crb_topx;
        const int lt = (int)P->cl.size();
        if (e == cudaSuccess)
            e = launch(P, K_DIRECT, lt, 1, [&] {
                return bt::launch_babd_direct(1, P->m, nr, tS, tR, P->B0, P->B1, tF, tX, P->keep, P->status, lt,
                                              P->stream);
            });
        for (int q = (int)P->cl.size() - 1; q >= 0 && e == cudaSuccess; --q) {
            bt::CrbArgs& c = P->cl[q];
            e = launch(P, K_SOLVE_BWD, c.level, 1, [&] { return L->crb_back(c, P->stream); });
        }
        return from_cuda(e);
    }
    P->lv[0].a.F = F;
    P->lv[0].a.X = X;
    for (auto& v : P->lv) v.a.nr = nr;
    const bool w0 = P->warp && L->warp_ok && L->warp_ok(P->lv[0].a, P->lv[0].low);
    for (int l = 0; l < P->nlev; ++l) {
        Level& v = P->lv[l];
        const bool w = (l == 0) && w0;
        if (l == 0 && P->qr) {
            bt::QrArgs& q = qr_args(P, nr);
            cudaError_t e = launch(P, K_SOLVE_FWD, 0, 2, [&] { return bt::launch_qr_solve_fwd(q, P->stream); });
            if (e != cudaSuccess) return from_cuda(e);
            continue;
        }
        cudaError_t e = launch(P, K_SOLVE_FWD, l, 1, [&] {
            return w ? L->solve_fwd_w(v.a, P->stream) : L->solve_fwd(v.a, v.low, P->stream);
        });
        if (e == cudaSuccess && P->kind == 0)
            e = launch(P, K_ASSEMBLE_RHS, l, 1, [&] {
                return w ? L->sep_rhs_w(v.a, P->stream) : L->assemble_rhs(v.a, v.low, P->stream);
            });
        if (e == cudaSuccess && l == 0) e = join_factor(P);
        if (e != cudaSuccess) return from_cuda(e);
    }
    Level& t = P->lv[P->nlev];
    const int lt = P->nlev;
    cudaError_t e = join_factor(P);
    if (e != cudaSuccess) return from_cuda(e);
    if (P->bcr && P->rs32) {
        P->rsa.nr = nr;
        e = launch(P, K_BCR_SOLVE, P->nlev, 1, [&] { return bt::launch_rsolve_f32(P->rsa, P->stream); });
    } else if (P->bcr) {
        e = cudaSuccess;
        if (P->nlev == 0) {
            P->bl[0].F = F;
            P->bl[0].X = X;
        }
        for (size_t q = 0; q < P->bl.size() && e == cudaSuccess; ++q) {
            bt::BcrArgs& b = P->bl[q];
            b.nr = nr;
            e = launch(P, K_BCR_SOLVE, b.level, 1,
                       [&] { return L->bcr_rhs(b, b.K == 1 ? 1 : (b.K + 1) / 2, P->stream); });
        }
        for (int q = (int)P->bl.size() - 2; q >= 0 && e == cudaSuccess; --q) {
            bt::BcrArgs& b = P->bl[q];
            e = launch(P, K_BCR_SOLVE, b.level, 1, [&] { return L->bcr_back(b, (b.K + 1) / 2, P->stream); });
        }
    } else if (P->pivot) {
        e = cudaSuccess;
        if (t.a.N >= 1)
            e = launch(P, K_DIRECT, lt, 1, [&] {
                return bt::launch_btri_direct((int)t.a.N, P->m, nr, t.a.B, t.a.D, t.a.C, t.a.F, t.a.X, P->keep,
                                              P->status, t.a.level, P->stream);
            });
    } else if (P->kind == 0) {
        e = launch(P, K_SOLVE_FWD, lt, 1, [&] { return L->solve_fwd(t.a, t.low, P->stream); });
        if (e == cudaSuccess) e = launch(P, K_SOLVE_BWD, lt, 1, [&] { return L->solve_bwd(t.a, t.low, P->stream); });
    } else {
        e = launch(P, K_DIRECT, lt, 1, [&] {
            return bt::launch_babd_direct((int)t.a.N, P->m, nr, t.a.B, t.a.D, P->B0, P->B1, t.a.F, t.a.X, P->keep,
                                          P->status, t.a.level, P->stream);
        });
    }
    if (e != cudaSuccess) return from_cuda(e);
    for (int l = P->nlev - 1; l >= 0; --l) {
        Level& v = P->lv[l];
        const bool w = (l == 0) && w0;
        e = launch(P, K_SOLVE_BWD, l, 1, [&] {
            if (l == 0 && P->qr) return bt::launch_qr_solve_bwd(qr_args(P, nr), P->stream);
            return w ? L->solve_bwd_w(v.a, P->stream) : L->solve_bwd(v.a, v.low, P->stream);
        });
        if (e != cudaSuccess) return from_cuda(e);
    }
    return BT_OK;
}

// df: the refinement residual of a refined plan, in double-float arithmetic on
// the FP32 pipe (bt_resid_df.cu); otherwise plain FP64.
bt_status run_residual(bt_plan_s* P, const double* F, const double* X, double* R, int nr,
                       unsigned long long* maxout = nullptr, bool df = false) {
    if (P->join_pending) {
        cudaError_t e = join_factor(P);
        if (e != cudaSuccess) return from_cuda(e);
    }
    if (maxout) {
        cudaError_t e = cudaMemsetAsync(maxout, 0, kSlotWords * sizeof(unsigned long long), P->stream);
        if (e != cudaSuccess) return from_cuda(e);
    }
    cudaError_t e = launch(P, K_RESID, 0, 1, [&] {
        // warp-kernel plans: double-float from the split copy the factorization
        // left; other plans of order 16 with up to 8 right-hand sides: the
        // tensor-core (digit-plane) residual from the FP64 matrix; else
        // double-float from the FP64 matrix
        if (P->kind == 0 && df && P->warp && P->lv[0].a.As && P->L->warp_ok && P->L->warp_ok(P->lv[0].a, P->lv[0].low) &&
            ((((uintptr_t)X) | ((uintptr_t)F)) & 15u) == 0)
            return bt::launch_resid_btri_dfs(P->N, P->m, nr, reinterpret_cast<const float2*>(P->lv[0].a.As), X, F,
                                             R, P->stream, maxout);
        if (P->kind == 0 && df && P->m == 16 && nr <= 8 &&
            ((((uintptr_t)P->A0) | ((uintptr_t)P->A1) | ((uintptr_t)P->A2) | ((uintptr_t)X) | ((uintptr_t)F)) & 15u) == 0)
            return bt::launch_resid_btri_oz(P->N, P->m, nr, P->A0, P->A1, P->A2, X, F, R, P->stream, maxout);
        if (P->kind == 0)
            return df ? bt::launch_resid_btri_df(P->N, P->m, nr, P->A0, P->A1, P->A2, X, F, R, P->stream, maxout)
                      : bt::launch_resid_btri(P->N, P->m, nr, P->A0, P->A1, P->A2, X, F, R, P->stream, maxout);
        return df ? bt::launch_resid_babd_df(P->N, P->m, nr, P->A0, P->A1, P->B0, P->B1, X, F, R, P->stream, maxout)
                  : bt::launch_resid_babd(P->N, P->m, nr, P->A0, P->A1, P->B0, P->B1, X, F, R, P->stream, maxout);
    });
    return from_cuda(e);
}

// ||A||_inf of the factored matrices (once per factorization).
bt_status ensure_anorm(bt_plan_s* P, bool force) {
    if (P->anorm_valid && (!force || P->anorm_fac)) return BT_OK;
    cudaError_t e = cudaMemsetAsync(P->amax, 0, kSlotWords * sizeof(unsigned long long), P->stream);
    if (e == cudaSuccess)
        e = launch(P, K_NORM, 0, 1, [&] {
            return bt::launch_norm_inf(P->kind, P->N, P->m, P->A0, P->A1, P->A2, P->B0, P->B1, P->amax, P->stream);
        });
    if (e != cudaSuccess) return from_cuda(e);
    P->anorm_valid = true;
    return BT_OK;
}

double eta_threshold(const bt_plan_s* P) {
    if (P->eta_tol >= 0.0) return P->eta_tol;
    // a few units of FP64 rounding per term of a residual row (3m terms)
    return 4.0 * (3.0 * P->m + 1.0) * 1.1102230246251565e-16;
}

// Copy the correction norms (2) and the residual and ||A||_inf slots to the host (async).
cudaError_t fetch_norms(bt_plan_s* P) {
    cudaError_t e = cudaMemcpyAsync(P->norms_host, P->norms, kNormWords * sizeof(double), cudaMemcpyDeviceToHost,
                                    P->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P->norms_host + kNormWords, P->rmax, kSlotWords * sizeof(double), cudaMemcpyDeviceToHost,
                            P->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P->norms_host + kNormWords + kSlotWords, P->amax, kSlotWords * sizeof(double),
                            cudaMemcpyDeviceToHost, P->stream);
    return e;
}

// Maximum of word w over the slots of a copied slot array.
double slot_max(const double* slots, int w) {
    double v = 0.0;
    for (int q = 0; q < bt::kMaxSlots; ++q) v = std::fmax(v, slots[3 * q + w]);
    return v;
}

// Normwise backward error ||r||_inf / (||A||_inf ||x||_inf + ||f||_inf) from the host copies.
double backward_error(const bt_plan_s* P) {
    const double* rs = P->norms_host + kNormWords;
    const double* as = P->norms_host + kNormWords + kSlotWords;
    const double rm = slot_max(rs, 0), xm = slot_max(rs, 1), fm = slot_max(rs, 2), am = slot_max(as, 0);
    const double den = am * xm + fm;
    return den > 0.0 ? rm / den : (rm > 0.0 ? INFINITY : 0.0);
}

// One refinement correction from the residual in Rbuf: d = solve(r), X += d,
// and (||d||^2, ||x||^2) in P->norms.  With the warp kernels at level 0 the
// back substitution applies the update itself and leaves per-partition norm
// partials; otherwise d goes through Dbuf and the update kernel.
bt_status run_correction(bt_plan_s* P, double* X, int nr, long long n, bool first) {
    Level& v0 = P->lv[0];
    if (!first) {
        // the norms of the correction before this one, for the forward-error estimate
        cudaError_t e = cudaMemcpyAsync(P->norms + 2, P->norms, 2 * sizeof(double), cudaMemcpyDeviceToDevice,
                                        P->stream);
        if (e != cudaSuccess) return from_cuda(e);
    }
    const bool w = P->warp && P->nlev >= 1 && P->L->warp_ok && P->L->warp_ok(v0.a, v0.low) && v0.a.nrm;
    if (w) {
        v0.a.accum = 1;
        bt_status st = run_solve(P, P->Rbuf, X, nr);
        v0.a.accum = 0;
        if (st != BT_OK) return st;
        cudaError_t e = launch(P, K_IR, 0, 1,
                               [&] { return bt::launch_reduce_pairs((int)v0.a.p, v0.a.nrm, P->norms, P->stream); });
        return from_cuda(e);
    }
    bt_status st = run_solve(P, P->Rbuf, P->Dbuf, nr);
    if (st != BT_OK) return st;
    cudaError_t e = launch(P, K_IR, 0, 2,
                           [&] { return bt::launch_ir_update(n, X, P->Dbuf, P->partial, P->norms, P->stream); });
    return from_cuda(e);
}

// Estimated relative forward error of the current iterate x_k after k >= 1
// corrections, from the last two corrections under linear convergence:
// ||x_k - x*|| <= rho / (1 - rho) ||d_k|| with the contraction ratio
// rho = ||d_k|| / ||d_(k-1)|| (d_0 = x_0, taken as ||x_k||: they differ by
// ||d_1||), the error estimate of refinement by correction ratios (Demmel,
// Hida, Kahan, Li, Mukherjee and Riedy 2006).  +inf without a clear
// contraction (rho >= 1/2) or without norms.
double forward_estimate(const bt_plan_s* P) {
    const double dd = P->norms_host[0], xx = P->norms_host[1], dp = P->norms_host[2];
    if (!(xx > 0.0) || !(dd >= 0.0)) return INFINITY;
    const double rel = std::sqrt(dd / xx);
    const double rho = std::isnan(dp) ? rel : ((dp > 0.0) ? std::sqrt(dd / dp) : INFINITY);
    if (!(rho < 0.5)) return INFINITY;
    return rho / (1.0 - rho) * rel;
}

// The norms of the last and the previous correction: zero and none.
cudaError_t reset_norms(bt_plan_s* P) {
    cudaError_t e = cudaMemsetAsync(P->norms, 0, 2 * sizeof(double), P->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->norms + 2, 0xff, 2 * sizeof(double), P->stream);   // NaN
    return e;
}

bt_status run_refine(bt_plan_s* P, const double* F, double* X, int nr, double tol, int maxit, int* iters,
                     double* relcorr) {
    // x = solve(f); then repeat: r = f - A x (FP64); stop when the normwise
    // backward error of x, or the last correction relative to x, is small;
    // otherwise d = solve(r), x += d.  One host synchronisation per round.
    if (iters) *iters = 0;
    if (relcorr) *relcorr = -1.0;
    bt_status st = ensure_anorm(P, false);
    if (st == BT_OK) st = run_solve(P, F, X, nr);
    if (st != BT_OK) return st;
    const long long n = P->lv[0].rows * P->m * nr;
    const double eta_tol = eta_threshold(P);
    cudaError_t e = reset_norms(P);
    if (e != cudaSuccess) return from_cuda(e);
    for (int it = 0;; ++it) {
        st = run_residual(P, F, X, P->Rbuf, nr, P->rmax, P->prec != BT_FP64);
        if (st != BT_OK) return st;
        e = fetch_norms(P);
        if (e != cudaSuccess) return from_cuda(e);
        st = read_status(P);   // synchronises
        if (st != BT_OK) return st;
        const double eta = backward_error(P);
        const double dd = P->norms_host[0], xx = P->norms_host[1];
        const double rel = (it == 0) ? -1.0 : ((xx > 0.0) ? std::sqrt(dd / xx) : std::sqrt(dd));
        if (iters) *iters = it;
        if (relcorr) *relcorr = rel;
        if (!std::isfinite(eta) || (it > 0 && !std::isfinite(rel))) return BT_ERR_NONFINITE;
        if (eta <= eta_tol) return BT_OK;
        if (it > 0 && rel <= tol) return BT_OK;
        if (it > 0 && P->fwd_tol > 0.0 && forward_estimate(P) <= P->fwd_tol) return BT_OK;
        if (it == maxit) return BT_ERR_NOT_CONVERGED;
        st = run_correction(P, X, nr, n, it == 0);
        if (st != BT_OK) return st;
    }
}

// Enqueue X = solve(F) and `sweeps` refinement corrections; no host sync.
bt_status run_refine_async(bt_plan_s* P, const double* F, double* X, int nr, int sweeps) {
    bt_status st = ensure_anorm(P, false);
    if (st == BT_OK) st = run_solve(P, F, X, nr);
    const long long n = P->lv[0].rows * P->m * nr;
    if (st == BT_OK) {
        cudaError_t e = reset_norms(P);
        if (e != cudaSuccess) return from_cuda(e);
    }
    for (int it = 0; it < sweeps && st == BT_OK; ++it) {
        st = run_residual(P, F, X, P->Rbuf, nr, nullptr, P->prec != BT_FP64);
        if (st == BT_OK) st = run_correction(P, X, nr, n, it == 0);
        if (st != BT_OK) return st;
    }
    if (st == BT_OK && P->x_event) {
        // X is final: the host-array path copies it out beside the checking residual
        cudaError_t e = cudaEventRecord(P->ev_xfinal, P->stream);
        if (e != cudaSuccess) return from_cuda(e);
    }
    // final residual of the result: its backward error decides convergence
    if (st == BT_OK) st = run_residual(P, F, X, P->Rbuf, nr, P->rmax, P->prec != BT_FP64);
    P->async_sweeps = sweeps;
    return st;
}

}  // namespace

extern "C" {

const char* bt_status_string(bt_status s) {
    switch (s) {
        case BT_OK: return "ok";
        case BT_ERR_INVALID: return "invalid argument";
        case BT_ERR_NOMEM: return "out of device memory";
        case BT_ERR_SINGULAR: return "singular pivot block";
        case BT_ERR_NONFINITE: return "non-finite pivot";
        case BT_ERR_NOT_CONVERGED: return "refinement did not converge";
        case BT_ERR_TIMEOUT: return "device wait timed out";
        case BT_ERR_CUDA: return "CUDA error";
    }
    return "unknown status";
}

static bt::Tuning to_tuning(const bt_tuning* t, int64_t p) {
    bt::Tuning u;
    if (t) {
        u.p0 = t->p0;
        u.ctas_per_sm = t->ctas_per_sm;
        u.sub_rows = t->sub_rows;
        u.top_rows = t->top_rows;
        u.reduced = t->reduced;
        u.tp_block = t->tp_block;
        u.local = t->local;
        u.pivot = t->pivot;
        u.serial = t->serial;
    }
    if (p > 0) u.p0 = p;
    return u;
}

bt_status bt_plan_create(bt_plan* plan, int64_t nblk, int m, int nrhs_max, int prec, int64_t p, void* stream) {
    return plan_create(plan, 0, nblk, m, nrhs_max, prec, to_tuning(nullptr, p), stream);
}

bt_status bt_plan_create_tuned(bt_plan* plan, int64_t nblk, int m, int nrhs_max, int prec, const bt_tuning* tuning,
                               void* stream) {
    if (tuning && (tuning->p0 < 0 || tuning->ctas_per_sm < 0 || tuning->sub_rows < 0 || tuning->top_rows < 0 ||
                   tuning->reduced < 0 || tuning->reduced > 1 || tuning->local < 0 || tuning->local > 62 || tuning->pivot < 0 || tuning->pivot > 2 ||
                   tuning->serial < 0 || tuning->serial > 1 ||
                   !(tuning->tp_block == 0 || tuning->tp_block == 64 || tuning->tp_block == 128 ||
                     tuning->tp_block == 256)))
        return BT_ERR_INVALID;
    return plan_create(plan, 0, nblk, m, nrhs_max, prec, to_tuning(tuning, 0), stream);
}

bt_status abd_plan_create_tuned(abd_plan* plan, int64_t N, int m, int nrhs_max, int prec, const bt_tuning* tuning,
                                void* stream) {
    if (tuning && (tuning->p0 < 0 || tuning->ctas_per_sm < 0 || tuning->sub_rows < 0 || tuning->top_rows < 0 ||
                   tuning->reduced < 0 || tuning->reduced > 1 || tuning->local != 0 || tuning->pivot != 0 ||
                   tuning->serial < 0 || tuning->serial > 1))
        return BT_ERR_INVALID;
    return plan_create(plan, 1, N, m, nrhs_max, prec, to_tuning(tuning, 0), stream);
}

bt_status abd_plan_create(abd_plan* plan, int64_t N, int m, int nrhs_max, int prec, int64_t p, void* stream) {
    return plan_create(plan, 1, N, m, nrhs_max, prec, to_tuning(nullptr, p), stream);
}

bt_status cyc_plan_create(abd_plan* plan, int64_t N, int m, int nrhs_max, int prec, int64_t p, void* stream) {
    if (!plan || N < 2) return BT_ERR_INVALID;
    bt_status st = abd_plan_create(plan, N - 1, m, nrhs_max, prec, p, stream);
    if (st == BT_OK) (*plan)->cyclic = true;
    return st;
}

bt_status cyc_factor(abd_plan P, const double* S, const double* R) {
    if (!P || !P->cyclic || !S || !R) return BT_ERR_INVALID;
    // the last block row S_{N-1} y_{N-1} + R_{N-1} y_0 moves to the top
    const size_t off = (size_t)P->N * P->mu * P->mu;
    return abd_factor(P, S, R, R + off, S + off);
}

namespace {
// dst = src rotated by one block row: dst[0] = src[N-1], dst[j+1] = src[j] (Nrows = N+1 of the abd plan)
cudaError_t rotate_rhs(bt_plan_s* P, const double* src, double* dst, int nrhs, bool forward) {
    const size_t blk = (size_t)P->mu * nrhs * sizeof(double);
    const size_t rest = (size_t)P->N * blk;   // N = steps of the abd plan = cycle length - 1
    cudaError_t e;
    if (forward) {
        e = cudaMemcpyAsync(dst, (const char*)src + rest, blk, cudaMemcpyDeviceToDevice, P->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync((char*)dst + blk, src, rest, cudaMemcpyDeviceToDevice, P->stream);
    } else {
        e = cudaMemcpyAsync((char*)dst + rest, src, blk, cudaMemcpyDeviceToDevice, P->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, (const char*)src + blk, rest, cudaMemcpyDeviceToDevice, P->stream);
    }
    return e;
}
}  // namespace

bt_status cyc_solve(abd_plan P, const double* RHS, double* Y, int nrhs) {
    if (!P || !P->cyclic || !RHS || !Y || nrhs < 1 || nrhs > P->nrhs_max) return BT_ERR_INVALID;
    cudaError_t e = rotate_rhs(P, RHS, P->rot, nrhs, true);
    if (e != cudaSuccess) return from_cuda(e);
    return abd_solve(P, P->rot, Y, nrhs);
}

bt_status cyc_residual(abd_plan P, const double* RHS, const double* Y, double* Rout, int nrhs) {
    if (!P || !P->cyclic || !RHS || !Y || !Rout || nrhs < 1 || nrhs > P->nrhs_max) return BT_ERR_INVALID;
    cudaError_t e = rotate_rhs(P, RHS, P->rot, nrhs, true);
    if (e != cudaSuccess) return from_cuda(e);
    bt_status st = abd_residual(P, P->rot, Y, P->rot2, nrhs);
    if (st != BT_OK) return st;
    return from_cuda(rotate_rhs(P, P->rot2, Rout, nrhs, false));
}

bt_status cyc_refine(abd_plan P, const double* RHS, double* Y, int nrhs, double tol, int maxit, int* iters_out,
                     double* relcorr_out) {
    if (!P || !P->cyclic || !RHS || !Y || nrhs < 1 || nrhs > P->nrhs_max) return BT_ERR_INVALID;
    cudaError_t e = rotate_rhs(P, RHS, P->rot, nrhs, true);
    if (e != cudaSuccess) return from_cuda(e);
    return abd_refine(P, P->rot, Y, nrhs, tol, maxit, iters_out, relcorr_out);
}

bt_status bt_factor(bt_plan P, const double* B, const double* D, const double* C) {
    if (!P || P->kind != 0 || !D || (P->N > 1 && (!B || !C))) return BT_ERR_INVALID;
    if (P->padded) {
        P->U[0] = B;
        P->U[1] = D;
        P->U[2] = C;
        cudaError_t e = bt::launch_pad_blocks(P->N, P->mu, P->m, D, P->Ap[1], 1, P->stream);
        if (e == cudaSuccess && P->N > 1) e = bt::launch_pad_blocks(P->N, P->mu, P->m, B, P->Ap[0], 0, P->stream);
        if (e == cudaSuccess && P->N > 1) e = bt::launch_pad_blocks(P->N, P->mu, P->m, C, P->Ap[2], 0, P->stream);
        if (e != cudaSuccess) return from_cuda(e);
        P->launches += 3;
        B = P->Ap[0];
        D = P->Ap[1];
        C = P->Ap[2];
    }
    P->A0 = B;
    P->A1 = D;
    P->A2 = C;
    Level& v = P->lv[0];
    v.a.B = B;
    v.a.D = D;
    v.a.C = C;
    v.a.shift = 0;
    cudaError_t e = cudaMemsetAsync(P->status, 0, 4 * sizeof(long long), P->stream);
    if (e != cudaSuccess) return from_cuda(e);
    P->anorm_valid = false;
    bt_status st = run_factor(P);
    P->factored = (st == BT_OK);
    return st;
}

bt_status abd_factor(abd_plan P, const double* S, const double* R, const double* B0, const double* B1) {
    if (!P || P->kind != 1 || !S || !R || !B0 || !B1) return BT_ERR_INVALID;
    cudaError_t e = cudaSuccess;
    if (P->padded) {
        P->U[0] = S;
        P->U[1] = R;
        P->U[2] = B0;
        P->U[3] = B1;
        e = bt::launch_pad_blocks(P->N, P->mu, P->m, S, P->Ap[0], 0, P->stream);
        if (e == cudaSuccess) e = bt::launch_pad_blocks(P->N, P->mu, P->m, R, P->Ap[1], 1, P->stream);
        if (e == cudaSuccess) e = bt::launch_pad_blocks(1, P->mu, P->m, B0, P->B0, 1, P->stream);
        if (e == cudaSuccess) e = bt::launch_pad_blocks(1, P->mu, P->m, B1, P->B1, 0, P->stream);
        if (e != cudaSuccess) return from_cuda(e);
        P->launches += 4;
        S = P->Ap[0];
        R = P->Ap[1];
    } else {
        P->U[2] = B0;
        P->U[3] = B1;
        const size_t mm = (size_t)P->m * P->m * sizeof(double);
        e = cudaMemcpyAsync(P->B0, B0, mm, cudaMemcpyDeviceToDevice, P->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(P->B1, B1, mm, cudaMemcpyDeviceToDevice, P->stream);
    }
    P->A0 = S;
    P->A1 = R;
    if (e == cudaSuccess) e = cudaMemsetAsync(P->status, 0, 4 * sizeof(long long), P->stream);
    if (e != cudaSuccess) return from_cuda(e);
    Level& v = P->lv[0];
    v.a.B = S;
    v.a.D = R;
    v.a.C = nullptr;
    v.a.shift = 1;
    P->anorm_valid = false;
    bt_status st = run_factor(P);
    P->factored = (st == BT_OK);
    return st;
}

static bt_status check_solve(bt_plan P, int kind, const void* F, const void* X, int nrhs) {
    if (!P || P->kind != kind || !F || !X || nrhs < 1 || nrhs > P->nrhs_max) return BT_ERR_INVALID;
    if (!P->factored) return BT_ERR_INVALID;
    if (F == X) return BT_ERR_INVALID;
    return BT_OK;
}

}  // extern "C"

// Padded plans: right-hand sides are embedded before and solutions extracted
// after the run; fn(F', X') runs on the padded arrays.
template <typename Fn>
static bt_status padded_call(bt_plan P, const double* F, double* X, int nrhs, Fn&& fn) {
    if (!P->padded) return fn(F, X);
    cudaError_t e = bt::launch_pad_rhs(P->lv[0].rows, P->mu, P->m, nrhs, F, P->Fp, P->stream);
    if (e != cudaSuccess) return from_cuda(e);
    bt_status st = fn(P->Fp, P->Xp);
    if (st != BT_OK && st != BT_ERR_NOT_CONVERGED) return st;
    e = bt::launch_unpad_rhs(P->lv[0].rows, P->mu, P->m, nrhs, P->Xp, X, P->stream);
    P->launches += 2;
    return e != cudaSuccess ? from_cuda(e) : st;
}

static bt_status residual_entry(bt_plan P, const double* F, const double* X, double* R, int nrhs, bool df = false) {
    if (!P->padded) return run_residual(P, F, X, R, nrhs, nullptr, df);
    cudaError_t e = bt::launch_pad_rhs(P->lv[0].rows, P->mu, P->m, nrhs, F, P->Fp, P->stream);
    if (e == cudaSuccess) e = bt::launch_pad_rhs(P->lv[0].rows, P->mu, P->m, nrhs, X, P->Xp, P->stream);
    if (e != cudaSuccess) return from_cuda(e);
    bt_status st = run_residual(P, P->Fp, P->Xp, P->Rp, nrhs, nullptr, df);
    if (st != BT_OK) return st;
    e = bt::launch_unpad_rhs(P->lv[0].rows, P->mu, P->m, nrhs, P->Rp, R, P->stream);
    P->launches += 3;
    return from_cuda(e);
}

extern "C" {

bt_status bt_solve(bt_plan P, const double* F, double* X, int nrhs) {
    bt_status st = check_solve(P, 0, F, X, nrhs);
    if (st != BT_OK) return st;
    return padded_call(P, F, X, nrhs, [&](const double* f, double* x) { return run_solve(P, f, x, nrhs); });
}
bt_status abd_solve(abd_plan P, const double* RHS, double* Y, int nrhs) {
    bt_status st = check_solve(P, 1, RHS, Y, nrhs);
    if (st != BT_OK) return st;
    return padded_call(P, RHS, Y, nrhs, [&](const double* f, double* x) { return run_solve(P, f, x, nrhs); });
}
bt_status bt_residual(bt_plan P, const double* F, const double* X, double* R, int nrhs) {
    bt_status st = check_solve(P, 0, F, X, nrhs);
    if (st == BT_OK && !R) st = BT_ERR_INVALID;
    return st != BT_OK ? st : residual_entry(P, F, X, R, nrhs);
}
bt_status abd_residual(abd_plan P, const double* RHS, const double* Y, double* Rout, int nrhs) {
    bt_status st = check_solve(P, 1, RHS, Y, nrhs);
    if (st == BT_OK && !Rout) st = BT_ERR_INVALID;
    return st != BT_OK ? st : residual_entry(P, RHS, Y, Rout, nrhs);
}
bt_status bt_refine_residual(bt_plan P, const double* F, const double* X, double* R, int nrhs) {
    bt_status st = check_solve(P, 0, F, X, nrhs);
    if (st == BT_OK && !R) st = BT_ERR_INVALID;
    return st != BT_OK ? st : residual_entry(P, F, X, R, nrhs, P->prec != BT_FP64);
}
bt_status abd_refine_residual(abd_plan P, const double* RHS, const double* Y, double* Rout, int nrhs) {
    bt_status st = check_solve(P, 1, RHS, Y, nrhs);
    if (st == BT_OK && !Rout) st = BT_ERR_INVALID;
    return st != BT_OK ? st : residual_entry(P, RHS, Y, Rout, nrhs, P->prec != BT_FP64);
}
bt_status bt_refine(bt_plan P, const double* F, double* X, int nrhs, double tol, int maxit, int* iters_out,
                    double* relcorr_out) {
    bt_status st = check_solve(P, 0, F, X, nrhs);
    if (st == BT_OK && (maxit < 1 || !(tol >= 0.0))) st = BT_ERR_INVALID;
    if (st != BT_OK) return st;
    return padded_call(P, F, X, nrhs, [&](const double* f, double* x) {
        return run_refine(P, f, x, nrhs, tol, maxit, iters_out, relcorr_out);
    });
}
bt_status abd_refine(abd_plan P, const double* RHS, double* Y, int nrhs, double tol, int maxit, int* iters_out,
                     double* relcorr_out) {
    bt_status st = check_solve(P, 1, RHS, Y, nrhs);
    if (st == BT_OK && (maxit < 1 || !(tol >= 0.0))) st = BT_ERR_INVALID;
    if (st != BT_OK) return st;
    return padded_call(P, RHS, Y, nrhs, [&](const double* f, double* x) {
        return run_refine(P, f, x, nrhs, tol, maxit, iters_out, relcorr_out);
    });
}

bt_status bt_refine_async(bt_plan P, const double* F, double* X, int nrhs, int sweeps) {
    bt_status st = check_solve(P, P ? P->kind : 0, F, X, nrhs);
    if (st == BT_OK && (sweeps < 0 || sweeps > 30)) st = BT_ERR_INVALID;
    if (st != BT_OK) return st;
    return padded_call(P, F, X, nrhs, [&](const double* f, double* x) { return run_refine_async(P, f, x, nrhs, sweeps); });
}

bt_status bt_refine_result(bt_plan P, double tol, double* relcorr_out) {
    if (!P) return BT_ERR_INVALID;
    cudaError_t e = fetch_norms(P);
    if (e != cudaSuccess) return from_cuda(e);
    bt_status st = read_status(P);
    const double dd = P->norms_host[0], xx = P->norms_host[1];
    const double rel = (xx > 0.0) ? std::sqrt(dd / xx) : std::sqrt(dd);
    if (relcorr_out) *relcorr_out = (P->async_sweeps > 0) ? rel : -1.0;
    if (st != BT_OK) return st;
    const double eta = backward_error(P);
    if (!std::isfinite(eta)) return BT_ERR_NONFINITE;
    if (eta <= eta_threshold(P)) return BT_OK;
    if (P->async_sweeps > 0 && std::isfinite(rel) && rel <= tol) return BT_OK;
    if (P->async_sweeps > 0 && P->fwd_tol > 0.0 && forward_estimate(P) <= P->fwd_tol) return BT_OK;
    return BT_ERR_NOT_CONVERGED;
}

bt_status bt_plan_anorm(bt_plan P, double* anorm_out) {
    if (!P || !anorm_out) return BT_ERR_INVALID;
    if (!P->factored) return BT_ERR_INVALID;
    bt_status st = ensure_anorm(P, false);
    if (st != BT_OK) return st;
    cudaError_t e = fetch_norms(P);
    if (e != cudaSuccess) return from_cuda(e);
    st = read_status(P);
    if (st != BT_OK) return st;
    *anorm_out = slot_max(P->norms_host + kNormWords + kSlotWords, 0);
    return BT_OK;
}

bt_status bt_plan_set_pivot_tol(bt_plan P, double tau) {
    if (!P || !P->pivot || !(tau >= 0.0) || !(tau < 1.0)) return BT_ERR_INVALID;
    P->pivot_tau = tau;
    return BT_OK;
}

bt_status bt_plan_set_backward_tol(bt_plan P, double eta_tol) {
    if (!P) return BT_ERR_INVALID;
    P->eta_tol = eta_tol;
    return BT_OK;
}

bt_status bt_plan_set_forward_tol(bt_plan P, double fwd_tol) {
    if (!P || std::isnan(fwd_tol)) return BT_ERR_INVALID;
    P->fwd_tol = fwd_tol;
    return BT_OK;
}

bt_status bt_plan_workspace_size(int kind, int64_t n, int m, int nrhs_max, int prec, const bt_tuning* tuning,
                                 int64_t* bytes) {
    if (!bytes || (kind != 0 && kind != 1)) return BT_ERR_INVALID;
    bt_plan tmp = nullptr;
    return plan_create(&tmp, kind, n, m, nrhs_max, prec, to_tuning(tuning, 0), nullptr, nullptr, 0, bytes);
}

bt_status bt_plan_create_in(bt_plan* plan, int kind, int64_t n, int m, int nrhs_max, int prec,
                            const bt_tuning* tuning, void* workspace, int64_t bytes, void* stream) {
    if (!workspace || (kind != 0 && kind != 1)) return BT_ERR_INVALID;
    return plan_create(plan, kind, n, m, nrhs_max, prec, to_tuning(tuning, 0), stream, workspace, bytes, nullptr);
}

bt_status bt_plan_capture(bt_plan P, int what, const double* F, double* X, int nrhs, int sweeps) {
    if (!P || what < 1 || what > 3) return BT_ERR_INVALID;
    if (P->pivot && !P->qr && what != 2) return BT_ERR_INVALID;   // the pivoted factorization synchronises
    bt_status st = check_solve(P, P->kind, F, X, nrhs);
    if (st != BT_OK) return st;
    if (what == 3 && (sweeps < 0 || sweeps > 30)) return BT_ERR_INVALID;
    if (P->graph_exec) {
        cudaGraphExecDestroy(P->graph_exec);
        P->graph_exec = nullptr;
    }
    if (P->graph) {
        cudaGraphDestroy(P->graph);
        P->graph = nullptr;
    }
    cudaError_t e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) return from_cuda(e);
    // kernels with large shared memory get their attribute before capture
    e = P->L->prepare();
    if (e != cudaSuccess) return from_cuda(e);
    if (what != 2) {
        e = ensure_side(P);
        if (e != cudaSuccess) return from_cuda(e);
    }
    cudaStream_t saved = P->stream, cap = nullptr;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return from_cuda(e);
    const bool saved_trace = P->trace;
    const long long l0 = P->launches;
    P->trace = false;
    P->stream = cap;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        if (what != 2) {
            e = cudaMemsetAsync(P->status, 0, 4 * sizeof(long long), cap);
            if (e == cudaSuccess && P->padded) {
                // the graph re-embeds the caller's matrices before factoring
                if (P->kind == 0) {
                    e = bt::launch_pad_blocks(P->N, P->mu, P->m, P->U[1], P->Ap[1], 1, cap);
                    if (e == cudaSuccess && P->N > 1) e = bt::launch_pad_blocks(P->N, P->mu, P->m, P->U[0], P->Ap[0], 0, cap);
                    if (e == cudaSuccess && P->N > 1) e = bt::launch_pad_blocks(P->N, P->mu, P->m, P->U[2], P->Ap[2], 0, cap);
                } else {
                    e = bt::launch_pad_blocks(P->N, P->mu, P->m, P->U[0], P->Ap[0], 0, cap);
                    if (e == cudaSuccess) e = bt::launch_pad_blocks(P->N, P->mu, P->m, P->U[1], P->Ap[1], 1, cap);
                    if (e == cudaSuccess) e = bt::launch_pad_blocks(1, P->mu, P->m, P->U[2], P->B0, 1, cap);
                    if (e == cudaSuccess) e = bt::launch_pad_blocks(1, P->mu, P->m, P->U[3], P->B1, 0, cap);
                }
            }
            if (e == cudaSuccess && P->kind == 1 && !P->padded) {
                const size_t mm = (size_t)P->m * P->m * sizeof(double);
                e = cudaMemcpyAsync(P->B0, P->U[2], mm, cudaMemcpyDeviceToDevice, cap);
                if (e == cudaSuccess) e = cudaMemcpyAsync(P->B1, P->U[3], mm, cudaMemcpyDeviceToDevice, cap);
            }
            P->overlap = !P->serial;
            if (e == cudaSuccess) st = run_factor(P);
            P->overlap = false;
            if (e == cudaSuccess && st == BT_OK && what == 3) st = ensure_anorm(P, true);
        }
        if (e == cudaSuccess && st == BT_OK) {
            st = padded_call(P, F, X, nrhs, [&](const double* f, double* x) {
                return what == 3 ? run_refine_async(P, f, x, nrhs, sweeps) : run_solve(P, f, x, nrhs);
            });
        }
        if (P->join_pending) {
            cudaError_t ej = join_factor(P);
            if (e == cudaSuccess) e = ej;
        }
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e2;
        P->graph = g;
        if (e == cudaSuccess && st == BT_OK) e = cudaGraphInstantiate(&P->graph_exec, g, 0);
    }
    P->stream = saved;
    P->trace = saved_trace;
    P->graph_launches = P->launches - l0;
    P->launches = l0;
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return from_cuda(e);
    }
    if (st == BT_OK && what != 2) P->factored = true;
    return st;
}

// Host-buffer factor + solve (or + refinement): the caller's arrays are host
// memory.  The block rows are copied in chunks of level-0 partitions on a
// copy stream, and each chunk's local factorizations start on their own
// stream as soon as its rows (and the separator row before them) have
// arrived, so the transfer overlaps the FP64 work; the right-hand side
// follows, then the reduced systems, the solve and the copy of X back, all
// ordered on the plan's stream.
namespace {
long long part_start(const LevelArgs& a, long long i) { return i * a.base + (i < a.extra ? i : a.extra); }

cudaError_t ensure_host_path(bt_plan_s* P) {
    cudaError_t e = cudaSuccess;
    if (!P->hb) {
        const size_t mm = (size_t)P->N * P->m * P->m, v = (size_t)P->N * P->m * P->nrhs_max;
        e = cudaMalloc(&P->hb, sizeof(double) * (3 * mm + 2 * v));
    }
    if (e == cudaSuccess && !P->copy_stream) e = cudaStreamCreateWithFlags(&P->copy_stream, cudaStreamNonBlocking);
    for (int k = 0; k < bt_plan_s::kChunks && e == cudaSuccess; ++k) {
        if (!P->chunk_stream[k]) e = cudaStreamCreateWithFlags(&P->chunk_stream[k], cudaStreamNonBlocking);
        if (e == cudaSuccess && !P->ev_rows[k]) e = cudaEventCreateWithFlags(&P->ev_rows[k], cudaEventDisableTiming);
        if (e == cudaSuccess && !P->ev_part[k]) e = cudaEventCreateWithFlags(&P->ev_part[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess && !P->ev_in) e = cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess && !P->ev_rhs) e = cudaEventCreateWithFlags(&P->ev_rhs, cudaEventDisableTiming);
    if (e == cudaSuccess && !P->ev_xfinal) e = cudaEventCreateWithFlags(&P->ev_xfinal, cudaEventDisableTiming);
    if (e == cudaSuccess && !P->ev_xout) e = cudaEventCreateWithFlags(&P->ev_xout, cudaEventDisableTiming);
    return e;
}
}  // namespace

namespace {
bt_status check_host_call(bt_plan P, const double* B, const double* D, const double* C, const double* F,
                          const double* X, int nrhs, int sweeps) {
    if (!P || P->kind != 0 || !D || !F || !X || (P->N > 1 && (!B || !C)) || nrhs < 1 || nrhs > P->nrhs_max ||
        sweeps < -1 || sweeps > 30 || P->padded || P->pivot || P->local > 0)
        return BT_ERR_INVALID;
    if (P->prec == BT_FP64 && sweeps >= 0) return BT_ERR_INVALID;
    if (P->prec != BT_FP64 && sweeps < 0) return BT_ERR_INVALID;
    return BT_OK;
}

bt_status enqueue_host(bt_plan P, const double* B, const double* D, const double* C, const double* F, double* X,
                       int nrhs, int sweeps) {
    cudaError_t e = cudaSuccess;
    const size_t mm = (size_t)P->m * P->m, bmm = sizeof(double) * mm;
    double* dB = P->hb;
    double* dD = dB + (size_t)P->N * mm;
    double* dC = dD + (size_t)P->N * mm;
    double* dF = dC + (size_t)P->N * mm;
    double* dX = dF + (size_t)P->N * P->m * P->nrhs_max;
    Level& v = P->lv[0];
    P->A0 = dB;
    P->A1 = dD;
    P->A2 = dC;
    v.a.B = dB;
    v.a.D = dD;
    v.a.C = dC;
    v.a.shift = 0;
    P->anorm_valid = false;
    // warp kernels take ||A||_inf while they convert the rows, chunk by chunk too
    const bool wn = P->warp && P->L->warp_ok && P->L->warp_ok(v.a, v.low);
    if (wn) {
        e = cudaMemsetAsync(P->amax, 0, kSlotWords * sizeof(unsigned long long), P->stream);
        v.a.amax = P->amax;
    }
    // the device copies may still be read by work queued earlier on the plan's stream
    if (e == cudaSuccess) e = cudaEventRecord(P->ev_in, P->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->copy_stream, P->ev_in, 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->status, 0, 4 * sizeof(long long), P->stream);
    const long long p = v.a.p;
    const int K = (int)std::min<long long>(bt_plan_s::kChunks, std::max<long long>(p, 1));
    // CTA kernels (m >= 8): row slabs of every partition in turn, the factorization in as
    // many phases, so every partition starts as soon as the first slab is in (strided
    // copies: one per array for each class of partitions with the same row count)
    const long long base = v.a.base, extra = v.a.extra;
    const bool slabs = P->L->factor_phase != nullptr && p >= 2 && base >= 1 &&
                       (size_t)(base + 1) * bmm < ((size_t)1 << 30);
    const int KP = bt_plan_s::kPhases;
    if (slabs && e == cudaSuccess) {
        struct Cls { long long first, count, stride, local; };
        Cls cls[3];
        int nc = 0;
        const long long nA = std::min<long long>(extra, p - 1);
        if (nA > 0) cls[nc++] = {0, nA, base + 1, base};                       // base+1 rows, last is the separator
        if (p - 1 - nA > 0) cls[nc++] = {nA, p - 1 - nA, base, base - 1};      // base rows, last is the separator
        const long long lastcnt = base + ((p - 1) < extra ? 1 : 0);
        cls[nc++] = {p - 1, 1, lastcnt, lastcnt};                              // the last partition: no separator
        auto copy2d = [&](long long row0, long long stride, long long rows, long long count) {
            if (rows <= 0 || count <= 0) return cudaSuccess;
            const size_t off = (size_t)row0 * mm, pitch = (size_t)stride * bmm, width = (size_t)rows * bmm;
            cudaError_t r = cudaMemcpy2DAsync(dB + off, pitch, B + off, pitch, width, count, cudaMemcpyHostToDevice,
                                              P->copy_stream);
            if (r == cudaSuccess)
                r = cudaMemcpy2DAsync(dD + off, pitch, D + off, pitch, width, count, cudaMemcpyHostToDevice,
                                      P->copy_stream);
            if (r == cudaSuccess && C)
                r = cudaMemcpy2DAsync(dC + off, pitch, C + off, pitch, width, count, cudaMemcpyHostToDevice,
                                      P->copy_stream);
            return r;
        };
        // the separator rows first: the first phase reads the left separator's C
        for (int c = 0; c < nc && e == cudaSuccess; ++c)
            if (cls[c].local < cls[c].stride) e = copy2d(part_start(v.a, cls[c].first) + cls[c].local, cls[c].stride, 1, cls[c].count);
        for (int k = 0; k < KP && e == cudaSuccess; ++k) {
            for (int c = 0; c < nc && e == cudaSuccess; ++c) {
                const long long l0 = cls[c].local * k / KP, l1 = cls[c].local * (k + 1) / KP;
                e = copy2d(part_start(v.a, cls[c].first) + l0, cls[c].stride, l1 - l0, cls[c].count);
            }
            if (e == cudaSuccess) e = cudaEventRecord(P->ev_rows[k], P->copy_stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(P->stream, P->ev_rows[k], 0);
            if (e == cudaSuccess)
                e = launch(P, K_FACTOR, 0, 1, [&] { return P->L->factor_phase(v.a, v.low, k, KP, P->stream); });
        }
    }
    for (int k = 0; k < K && e == cudaSuccess && !slabs; ++k) {
        const long long pb = p * k / K, pe = p * (k + 1) / K;
        // rows of partitions [pb, pe) and the separator row before them (its C)
        const long long r0 = std::max<long long>(part_start(v.a, pb) - 1, 0);
        const long long r1 = (pe >= p) ? P->N : part_start(v.a, pe);
        const size_t off = (size_t)r0 * mm, bytes = (size_t)(r1 - r0) * bmm;
        e = cudaMemcpyAsync(dB + off, B + off, bytes, cudaMemcpyHostToDevice, P->copy_stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dD + off, D + off, bytes, cudaMemcpyHostToDevice, P->copy_stream);
        if (e == cudaSuccess && C) e = cudaMemcpyAsync(dC + off, C + off, bytes, cudaMemcpyHostToDevice, P->copy_stream);
        if (e == cudaSuccess) e = cudaEventRecord(P->ev_rows[k], P->copy_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(P->chunk_stream[k], P->ev_rows[k], 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(P->chunk_stream[k], P->ev_in, 0);
        if (e == cudaSuccess)
            e = launch(P, K_FACTOR, 0, 1,
                       [&] { return P->L->factor_part(v.a, v.low, pb, pe, P->chunk_stream[k]); });
        if (e == cudaSuccess) e = cudaEventRecord(P->ev_part[k], P->chunk_stream[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(P->stream, P->ev_part[k], 0);
    }
    const size_t fbytes = sizeof(double) * (size_t)P->N * P->m * nrhs;
    if (e == cudaSuccess) e = cudaMemcpyAsync(dF, F, fbytes, cudaMemcpyHostToDevice, P->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(P->ev_rhs, P->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->stream, P->ev_rhs, 0);
    v.a.amax = nullptr;
    if (e != cudaSuccess) return from_cuda(e);
    if (wn) {
        P->anorm_valid = true;
        P->anorm_fac = true;
    }
    P->overlap = !P->serial;
    bt_status st = run_factor(P, true);
    P->overlap = false;
    P->factored = (st == BT_OK);
    const bool xev = sweeps >= 0;
    P->x_event = xev;
    if (st == BT_OK) st = (sweeps < 0) ? run_solve(P, dF, dX, nrhs) : run_refine_async(P, dF, dX, nrhs, sweeps);
    P->x_event = false;
    if (P->join_pending) {
        cudaError_t ej = join_factor(P);
        if (st == BT_OK && ej != cudaSuccess) st = from_cuda(ej);
    }
    if (st != BT_OK) return st;
    if (!xev) {
        e = cudaMemcpyAsync(X, dX, fbytes, cudaMemcpyDeviceToHost, P->stream);
        return from_cuda(e);
    }
    // the copy out runs on the copy stream beside the checking residual; the plan's
    // stream waits for it
    e = cudaStreamWaitEvent(P->copy_stream, P->ev_xfinal, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(X, dX, fbytes, cudaMemcpyDeviceToHost, P->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(P->ev_xout, P->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->stream, P->ev_xout, 0);
    return from_cuda(e);
}
}  // namespace

bt_status bt_factor_solve_host(bt_plan P, const double* B, const double* D, const double* C, const double* F,
                               double* X, int nrhs, int sweeps) {
    bt_status st = check_host_call(P, B, D, C, F, X, nrhs, sweeps);
    if (st != BT_OK) return st;
    cudaError_t e = ensure_host_path(P);
    if (e == cudaSuccess) e = ensure_side(P);
    if (e != cudaSuccess) return from_cuda(e);
    return enqueue_host(P, B, D, C, F, X, nrhs, sweeps);
}

bt_status bt_plan_capture_host(bt_plan P, const double* B, const double* D, const double* C, const double* F,
                               double* X, int nrhs, int sweeps) {
    bt_status st = check_host_call(P, B, D, C, F, X, nrhs, sweeps);
    if (st != BT_OK) return st;
    cudaError_t e = ensure_host_path(P);
    if (e == cudaSuccess) e = ensure_side(P);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    if (e == cudaSuccess) e = P->L->prepare();
    if (e != cudaSuccess) return from_cuda(e);
    if (P->graph_exec) {
        cudaGraphExecDestroy(P->graph_exec);
        P->graph_exec = nullptr;
    }
    if (P->graph) {
        cudaGraphDestroy(P->graph);
        P->graph = nullptr;
    }
    cudaStream_t saved = P->stream, cap = nullptr;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return from_cuda(e);
    const bool saved_trace = P->trace;
    const long long l0 = P->launches;
    P->trace = false;
    P->stream = cap;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        st = enqueue_host(P, B, D, C, F, X, nrhs, sweeps);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e2;
        P->graph = g;
        if (e == cudaSuccess && st == BT_OK) e = cudaGraphInstantiate(&P->graph_exec, g, 0);
    }
    P->stream = saved;
    P->trace = saved_trace;
    P->graph_launches = P->launches - l0;
    P->launches = l0;
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return from_cuda(e);
    }
    return st;
}

bt_status bt_band_to_blocks(int64_t n, int s, int r, const double* band, int m, double* B, double* D, double* C,
                            void* stream) {
    if (n < 1 || s < 0 || r < 0 || m < 1 || m > 32 || m < s || m < r || !band || !B || !D || !C)
        return BT_ERR_INVALID;
    const long long N = (n + m - 1) / m;
    return from_cuda(bt::launch_band_to_blocks(n, s, r, band, N, m, B, D, C, (cudaStream_t)stream));
}

bt_status bt_plan_replay(bt_plan P) {
    if (!P || !P->graph_exec) return BT_ERR_INVALID;
    P->launches += P->graph_launches;
    return from_cuda(cudaGraphLaunch(P->graph_exec, P->stream));
}

bt_status bt_sync(bt_plan P) {
    if (!P) return BT_ERR_INVALID;
    return read_status(P);
}
bt_status abd_sync(abd_plan P) { return bt_sync(P); }

bt_status bt_info(bt_plan P, int* level, int64_t* partition, int64_t* row) {
    if (!P) return BT_ERR_INVALID;
    bt_status st = read_status(P);
    if (level) *level = (int)P->status_host[1];
    if (partition) *partition = P->status_host[2];
    if (row) *row = P->status_host[3];
    return st;
}

bt_status bt_plan_levels(bt_plan P, int* levels, int64_t* rows, int64_t* parts, int capacity) {
    if (!P) return BT_ERR_INVALID;
    if (levels) *levels = P->nlev + 1;
    for (int l = 0; l <= P->nlev && l < capacity; ++l) {
        if (rows) rows[l] = P->lv[l].a.N;
        if (parts) parts[l] = P->lv[l].a.p;
    }
    return BT_OK;
}

bt_status bt_plan_bytes(bt_plan P, int64_t* bytes) {
    if (!P || !bytes) return BT_ERR_INVALID;
    *bytes = (int64_t)P->arena_bytes;
    return BT_OK;
}

bt_status bt_reduced_export(bt_plan P, double* alpha, double* beta, double* gamma) {
    if (!P || !P->factored || !alpha || !beta || P->padded) return BT_ERR_INVALID;
    const size_t mm = (size_t)P->m * P->m * sizeof(double);
    if (P->kind == 0 && P->nlev == 0 && P->bcr && P->local > 0) {
        // local cyclic reduction: the FP64 system left on the separators
        const bt::BcrArgs& b = P->bl[P->local];
        if (!gamma || b.mode != bt::BCR_F64) return BT_ERR_INVALID;
        const size_t bytes = mm * (size_t)b.K;
        cudaError_t e = cudaMemcpyAsync(alpha, b.D, bytes, cudaMemcpyDeviceToDevice, P->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(beta, b.B, bytes, cudaMemcpyDeviceToDevice, P->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(gamma, b.C, bytes, cudaMemcpyDeviceToDevice, P->stream);
        return from_cuda(e);
    }
    if (P->nlev < 1) return BT_ERR_INVALID;
    const Level& u = P->lv[0];
    cudaError_t e;
    if (P->kind == 0) {
        if (!gamma) return BT_ERR_INVALID;
        const size_t bytes = mm * (size_t)(u.a.p - 1);
        e = cudaMemcpyAsync(alpha, u.a.Dn, bytes, cudaMemcpyDeviceToDevice, P->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(beta, u.a.Bn, bytes, cudaMemcpyDeviceToDevice, P->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(gamma, u.a.Cn, bytes, cudaMemcpyDeviceToDevice, P->stream);
    } else {
        const size_t bytes = mm * (size_t)u.a.p;
        e = cudaMemcpyAsync(alpha, P->B0, mm, cudaMemcpyDeviceToDevice, P->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(beta, P->B1, mm, cudaMemcpyDeviceToDevice, P->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((char*)alpha + mm, u.a.Dn, bytes, cudaMemcpyDeviceToDevice, P->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((char*)beta + mm, u.a.Bn, bytes, cudaMemcpyDeviceToDevice, P->stream);
    }
    return from_cuda(e);
}

bt_status bt_plan_trace(bt_plan P, int enable) {
    if (!P) return BT_ERR_INVALID;
    cudaError_t e = cudaStreamSynchronize(P->stream);
    P->recs.clear();
    P->pool_used = 0;
    P->trace = enable != 0;
    return from_cuda(e);
}

bt_status bt_plan_trace_query(bt_plan P, int kind, int level, double* total_ms, int64_t* launches) {
    if (!P) return BT_ERR_INVALID;
    cudaError_t e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) return from_cuda(e);
    double tot = 0.0;
    int64_t n = 0;
    for (const auto& r : P->recs) {
        if (r.key / 64 != kind) continue;
        if (level >= 0 && r.key % 64 != (level < 63 ? level : 63)) continue;
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) return from_cuda(e);
        tot += ms;
        ++n;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = n;
    return BT_OK;
}

bt_status bt_plan_launches(bt_plan P, int64_t* count) {
    if (!P || !count) return BT_ERR_INVALID;
    *count = P->launches;
    return BT_OK;
}

void bt_plan_destroy(bt_plan P) {
    if (!P) return;
    cudaStreamSynchronize(P->stream);
    for (auto ev : P->pool) cudaEventDestroy(ev);
    if (P->graph_exec) cudaGraphExecDestroy(P->graph_exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    if (P->side) {
        cudaStreamSynchronize(P->side);
        cudaStreamDestroy(P->side);
    }
    if (P->copy_stream) {
        cudaStreamSynchronize(P->copy_stream);
        cudaStreamDestroy(P->copy_stream);
    }
    for (int k = 0; k < bt_plan_s::kChunks; ++k) {
        if (P->chunk_stream[k]) {
            cudaStreamSynchronize(P->chunk_stream[k]);
            cudaStreamDestroy(P->chunk_stream[k]);
        }
        if (P->ev_rows[k]) cudaEventDestroy(P->ev_rows[k]);
        if (P->ev_part[k]) cudaEventDestroy(P->ev_part[k]);
    }
    if (P->ev_in) cudaEventDestroy(P->ev_in);
    if (P->ev_rhs) cudaEventDestroy(P->ev_rhs);
    if (P->ev_xfinal) cudaEventDestroy(P->ev_xfinal);
    if (P->ev_xout) cudaEventDestroy(P->ev_xout);
    if (P->hb) cudaFree(P->hb);
    if (P->ev_fork) cudaEventDestroy(P->ev_fork);
    if (P->ev_join) cudaEventDestroy(P->ev_join);
    if (P->own_arena) cudaFree(P->arena);
    if (P->pinned) {
        if (P->status_host) cudaFreeHost(P->status_host);
        if (P->norms_host) cudaFreeHost(P->norms_host);
    } else {
        delete[] P->status_host;
        delete[] P->norms_host;
    }
    delete P;
}
void abd_plan_destroy(abd_plan P) { bt_plan_destroy(P); }

}  // extern "C"
