// Batched solves of many independent block tridiagonal systems of different
// sizes, block orders and precisions (plan step A0 per system, steps A1-A7 for
// all of them together).  The partitions of every system at the same
// recursion level, block order and precision are one work list; each list is
// processed by one persistent launch (a fixed grid striding over the items),
// and the whole sequence -- factor, solve and a fixed number of FP64
// refinement sweeps for the low-precision systems -- is captured into one CUDA
// graph, so a run is a single graph launch.  Block-order classes run on
// parallel capture streams.  If the workspace of all systems exceeds the
// memory cap, the systems are split into waves that reuse the same workspace
// one after the other inside the graph.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <tuple>
#include <new>
#include <vector>

#include "../../include/bt.h"
#include "bt_launch.h"
#include "bt_level.h"
#include "bt_planner.h"

namespace bt {

struct ResidDesc {
    long long N;
    int m, nr;
    const double *B, *D, *C, *F;
    double* X;
    double* R;
    const double* Dc;
};
struct Chunk {
    int sys;
    long long start, count;
};

// r = f - A x for every chunk (FP64), one thread per entry.
__global__ void __launch_bounds__(256) k_resid_btri_batch(const ResidDesc* __restrict__ ds,
                                                          const Chunk* __restrict__ ch, int nch) {
    for (int q = blockIdx.x; q < nch; q += gridDim.x) {
        const Chunk c = ch[q];
        const ResidDesc d = ds[c.sys];
        const long long mm = (long long)d.m * d.m;
        for (long long el = c.start + threadIdx.x; el < c.start + c.count; el += blockDim.x) {
            const long long gr = el / d.nr;
            const int col = (int)(el % d.nr);
            const long long j = gr / d.m;
            const int r = (int)(gr % d.m);
            double acc = d.F[el];
            const double* xj = d.X + j * d.m * d.nr + col;
            const double* Drow = d.D + j * mm + (long long)r * d.m;
            for (int k = 0; k < d.m; ++k) acc = fma(-Drow[k], xj[(long long)k * d.nr], acc);
            if (j > 0) {
                const double* Brow = d.B + j * mm + (long long)r * d.m;
                for (int k = 0; k < d.m; ++k) acc = fma(-Brow[k], xj[(long long)(k - d.m) * d.nr], acc);
            }
            if (j + 1 < d.N) {
                const double* Crow = d.C + j * mm + (long long)r * d.m;
                for (int k = 0; k < d.m; ++k) acc = fma(-Crow[k], xj[(long long)(k + d.m) * d.nr], acc);
            }
            d.R[el] = acc;
        }
    }
}

// x += d for every chunk; partial[q] = (sum d^2, sum x^2) of chunk q.
__global__ void __launch_bounds__(256) k_ir_update_batch(const ResidDesc* __restrict__ ds,
                                                         const Chunk* __restrict__ ch, int nch,
                                                         double* __restrict__ partial) {
    __shared__ double sd[256], sx[256];
    for (int q = blockIdx.x; q < nch; q += gridDim.x) {
        const Chunk c = ch[q];
        const ResidDesc d = ds[c.sys];
        double ad = 0.0, ax = 0.0;
        for (long long el = c.start + threadIdx.x; el < c.start + c.count; el += blockDim.x) {
            const double dv = d.Dc[el];
            const double xv = d.X[el] + dv;
            d.X[el] = xv;
            ad = fma(dv, dv, ad);
            ax = fma(xv, xv, ax);
        }
        sd[threadIdx.x] = ad;
        sx[threadIdx.x] = ax;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                sd[threadIdx.x] += sd[threadIdx.x + s];
                sx[threadIdx.x] += sx[threadIdx.x + s];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            partial[2 * q] = sd[0];
            partial[2 * q + 1] = sx[0];
        }
        __syncthreads();
    }
}

// norms[2s..2s+1] = sums of the partials of system s's chunks (fixed order).
__global__ void __launch_bounds__(32) k_reduce_sys(const int* __restrict__ first, const int* __restrict__ sys_ids,
                                                   int nsys, const double* __restrict__ partial,
                                                   double* __restrict__ norms) {
    for (int t = blockIdx.x; t < nsys; t += gridDim.x) {
        if (threadIdx.x == 0) {
            double ad = 0.0, ax = 0.0;
            for (int q = first[t]; q < first[t + 1]; ++q) {
                ad += partial[2 * q];
                ax += partial[2 * q + 1];
            }
            norms[2 * sys_ids[t]] = ad;
            norms[2 * sys_ids[t] + 1] = ax;
        }
    }
}

}  // namespace bt

namespace {

using bt::LevelArgs;
constexpr long long kChunk = 1 << 16;

struct BSys {
    bt_batch_desc d;
    bool low = false;
    std::vector<bt::LevelShape> shapes;
    std::vector<LevelArgs> lv;
    LevelArgs corr0;
    size_t bytes = 0, off = 0;
    int wave = 0;
    int arg_base = 0;   // lv[l] at arg_base + l; corr0 at arg_base + nlev + 1
    double* R = nullptr;
    double* Dc = nullptr;
    int nlev() const { return (int)lv.size() - 1; }
};

struct Group {   // one persistent launch
    int kind;    // 0 factor, 1 assemble, 2 solve_fwd, 3 assemble_rhs, 4 solve_bwd
    int m;
    bool low;
    size_t work_off;
    int nwork;
};

struct Cursor {
    char* base;
    size_t off;
    void* take(size_t bytes) {
        off = (off + 255) & ~size_t(255);
        void* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    }
};

void layout_sys(BSys& s, Cursor& c) {
    const int m = s.d.m, nr = s.d.nrhs;
    const long long mm = (long long)m * m;
    for (size_t l = 0; l < s.lv.size(); ++l) {
        LevelArgs& a = s.lv[l];
        const size_t ts = (l == 0 && s.low) ? sizeof(float) : sizeof(double);
        const long long rows = s.shapes[l].rows;
        a.Dinv = c.take(ts * rows * mm);
        a.Y = c.take(ts * rows * mm);
        a.Zc = c.take(ts * rows * mm);
        a.Pf = c.take(ts * a.p * mm);
        a.Qf = c.take(ts * a.p * mm);
        a.Hf = c.take(ts * a.p * m * nr);
        if (l >= 1) {
            LevelArgs& u = s.lv[l - 1];
            double* Bn = (double*)c.take(sizeof(double) * rows * mm);
            double* Dn = (double*)c.take(sizeof(double) * rows * mm);
            double* Cn = (double*)c.take(sizeof(double) * rows * mm);
            double* Fn = (double*)c.take(sizeof(double) * rows * m * nr);
            double* Xn = (double*)c.take(sizeof(double) * rows * m * nr);
            u.Bn = Bn; u.Dn = Dn; u.Cn = Cn; u.Fn = Fn; u.Xn = Xn;
            a.B = Bn; a.D = Dn; a.C = Cn; a.F = Fn; a.X = Xn;
        }
    }
    if (s.low) {
        s.R = (double*)c.take(sizeof(double) * s.d.nblk * m * nr);
        s.Dc = (double*)c.take(sizeof(double) * s.d.nblk * m * nr);
    }
}

bt_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return BT_OK;
    if (e == cudaErrorMemoryAllocation) return BT_ERR_NOMEM;
    return BT_ERR_CUDA;
}

}  // namespace

struct bt_batch_s {
    std::vector<BSys> sys;
    cudaStream_t stream = nullptr;
    int device = 0, sms = 148, waves = 1, ir_sweeps = 0;
    char* arena = nullptr;
    size_t arena_bytes = 0, other_bytes = 0;
    LevelArgs* d_args = nullptr;
    int2* d_work = nullptr;
    long long* d_status = nullptr;
    double* d_norms = nullptr;
    bt::ResidDesc* d_rdesc = nullptr;
    bt::Chunk* d_chunks = nullptr;
    int* d_first = nullptr;
    int* d_sysids = nullptr;
    double* d_partial = nullptr;
    std::vector<cudaStream_t> cls_streams;
    std::vector<cudaEvent_t> events;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t graph_nodes = 0;
    std::vector<long long> h_status;
    std::vector<double> h_norms;
};

namespace {

void free_batch(bt_batch_s* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto s : b->cls_streams) cudaStreamDestroy(s);
    for (auto e : b->events) cudaEventDestroy(e);
    cudaFree(b->arena);
    cudaFree(b->d_args);
    cudaFree(b->d_work);
    cudaFree(b->d_status);
    cudaFree(b->d_norms);
    cudaFree(b->d_rdesc);
    cudaFree(b->d_chunks);
    cudaFree(b->d_first);
    cudaFree(b->d_sysids);
    cudaFree(b->d_partial);
    delete b;
}

int grid_for(const bt::Launchers* L, int nwork, int sms) {
    if (L->cta) return std::max(1, std::min(nwork, sms * 8));
    return std::max(1, std::min((nwork + 127) / 128, sms * 16));
}

}  // namespace

extern "C" {

bt_status bt_batch_create(bt_batch* out, const bt_batch_desc* descs, int count, int ir_sweeps,
                          int64_t mem_cap_bytes, void* stream) {
    if (!out || !descs || count < 1 || ir_sweeps < 0 || ir_sweeps > 30) return BT_ERR_INVALID;
    *out = nullptr;
    bt_batch_s* b = new (std::nothrow) bt_batch_s();
    if (!b) return BT_ERR_NOMEM;
    b->stream = (cudaStream_t)stream;
    b->ir_sweeps = ir_sweeps;
    cudaGetDevice(&b->device);
    if (cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess || b->sms <= 0)
        b->sms = 148;
    // ---- per-system levels and workspace sizes
    b->sys.resize(count);
    for (int k = 0; k < count; ++k) {
        BSys& s = b->sys[k];
        s.d = descs[k];
        const bt_batch_desc& d = s.d;
        if (!bt::launchers_for(d.m) || d.nblk < 1 || d.nrhs < 1 || d.nrhs > 32 || d.prec < 0 || d.prec > 2 ||
            !d.D || !d.F || !d.X || d.F == d.X || (d.nblk > 1 && (!d.B || !d.C))) {
            free_batch(b);
            return BT_ERR_INVALID;
        }
        s.low = d.prec != BT_FP64;
        bt::Tuning t;
        t.p0 = d.tuning.p0;
        t.ctas_per_sm = d.tuning.ctas_per_sm;
        t.sub_rows = d.tuning.sub_rows;
        t.top_rows = d.tuning.top_rows;
        if (t.p0 == 0 && t.ctas_per_sm == 0) {
            // in a batch the GPU is filled by many systems: long partitions
            const long long k0 = (d.m >= 8) ? 32 : 64;
            t.p0 = std::max<long long>(1, std::min<long long>(d.nblk / k0, (d.nblk + 1) / 2));
            if (d.nblk <= 8) t.p0 = 1;
        }
        if (!bt::plan_shapes(0, d.nblk, d.m, b->sms, t, s.shapes)) {
            free_batch(b);
            return BT_ERR_INVALID;
        }
        s.lv.resize(s.shapes.size());
        for (size_t l = 0; l < s.shapes.size(); ++l) {
            LevelArgs& a = s.lv[l];
            std::memset(&a, 0, sizeof(a));
            a.mode = 0;
            a.level = (int)l;
            a.N = s.shapes[l].N;
            a.p = s.shapes[l].p;
            a.base = s.shapes[l].base;
            a.extra = s.shapes[l].extra;
            a.nr = d.nrhs;
            a.bf16 = (l == 0 && d.prec == BT_BF16_IR && d.m >= 16) ? 1 : 0;
        }
        s.lv[0].B = d.B;
        s.lv[0].D = d.D;
        s.lv[0].C = d.C;
        s.lv[0].F = d.F;
        s.lv[0].X = d.X;
        Cursor meas{nullptr, 0};
        layout_sys(s, meas);
        s.bytes = (meas.off + 255) & ~size_t(255);
    }
    // ---- waves under the memory cap
    const size_t cap = mem_cap_bytes > 0 ? (size_t)mem_cap_bytes : SIZE_MAX;
    size_t used = 0, maxwave = 0;
    int wave = 0;
    for (auto& s : b->sys) {
        if (s.bytes > cap) {
            free_batch(b);
            return BT_ERR_NOMEM;
        }
        if (used + s.bytes > cap) {
            ++wave;
            used = 0;
        }
        s.wave = wave;
        s.off = used;
        used += s.bytes;
        maxwave = std::max(maxwave, used);
    }
    b->waves = wave + 1;
    cudaError_t e = cudaMalloc((void**)&b->arena, std::max<size_t>(maxwave, 256));
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_batch(b);
        return from_cuda(e);
    }
    b->arena_bytes = maxwave;
    e = cudaMalloc((void**)&b->d_status, sizeof(long long) * 4 * count);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_norms, sizeof(double) * 2 * count);
    if (e != cudaSuccess) {
        free_batch(b);
        return from_cuda(e);
    }
    // ---- real layout and the args array
    std::vector<LevelArgs> h_args;
    for (int k = 0; k < count; ++k) {
        BSys& s = b->sys[k];
        Cursor c{b->arena + s.off, 0};
        layout_sys(s, c);
        for (auto& a : s.lv) a.status = b->d_status + 4 * k;
        s.corr0 = s.lv[0];
        s.corr0.F = s.R;
        s.corr0.X = s.Dc;
        s.arg_base = (int)h_args.size();
        for (auto& a : s.lv) h_args.push_back(a);
        h_args.push_back(s.corr0);
    }
    // ---- work lists: groups per (wave, phase, level, kind, m, low)
    std::vector<int2> h_work;
    struct Key {
        int wave, phase, level, kind, m, low;
        bool operator<(const Key& o) const {
            return std::tie(wave, phase, level, kind, m, low) < std::tie(o.wave, o.phase, o.level, o.kind, o.m, o.low);
        }
    };
    std::map<Key, std::vector<int2>> lists;
    int maxlev = 0;
    for (int k = 0; k < count; ++k) {
        BSys& s = b->sys[k];
        const bt::Launchers* L = bt::launchers_for(s.d.m);
        const int nr = s.d.nrhs;
        maxlev = std::max(maxlev, s.nlev());
        for (int l = 0; l <= s.nlev(); ++l) {
            const LevelArgs& a = s.lv[l];
            const bool lowl = s.low && l == 0;
            const bool top = (l == s.nlev());
            for (int phase = 0; phase < (s.low ? 2 : 1); ++phase) {
                // phase 0: main factor + solve; phase 1: correction solve of a sweep
                const int arg = (phase == 1 && l == 0) ? s.arg_base + s.nlev() + 1 : s.arg_base + l;
                auto add = [&](int kind, long long units) {
                    auto& v = lists[{s.wave, phase, l, kind, s.d.m, lowl ? 1 : 0}];
                    for (long long u = 0; u < units; ++u) v.push_back(make_int2(arg, (int)u));
                };
                const long long per_rhs = L->cta ? 1 : nr;
                if (phase == 0) {
                    add(0, a.p);
                    if (!top) add(1, a.p - 1);
                }
                add(2, a.p * per_rhs);
                if (!top) add(3, (a.p - 1) * per_rhs);
                add(4, a.p * per_rhs);
            }
        }
    }
    std::map<Key, Group> groups;
    for (auto& kv : lists) {
        Group g{kv.first.kind, kv.first.m, kv.first.low != 0, h_work.size(), (int)kv.second.size()};
        h_work.insert(h_work.end(), kv.second.begin(), kv.second.end());
        groups[kv.first] = g;
    }
    // ---- refinement chunks (low-precision systems)
    std::vector<bt::ResidDesc> h_rd(count);
    std::vector<std::vector<bt::Chunk>> wave_chunks(b->waves);
    std::vector<std::vector<int>> wave_first(b->waves), wave_ids(b->waves);
    for (int k = 0; k < count; ++k) {
        BSys& s = b->sys[k];
        h_rd[k] = bt::ResidDesc{s.d.nblk, s.d.m, s.d.nrhs, s.d.B, s.d.D, s.d.C, s.d.F, s.d.X, s.R, s.Dc};
    }
    std::vector<bt::Chunk> h_chunks;
    std::vector<int> h_first, h_ids;
    std::vector<size_t> wave_chunk_off(b->waves), wave_nchunk(b->waves), wave_first_off(b->waves),
        wave_nsys(b->waves);
    for (int w = 0; w < b->waves; ++w) {
        wave_chunk_off[w] = h_chunks.size();
        wave_first_off[w] = h_first.size();
        int nsys = 0;
        for (int k = 0; k < count; ++k) {
            BSys& s = b->sys[k];
            if (s.wave != w || !s.low) continue;
            h_first.push_back((int)(h_chunks.size() - wave_chunk_off[w]));
            h_ids.push_back(k);
            const long long n = s.d.nblk * s.d.m * s.d.nrhs;
            for (long long st = 0; st < n; st += kChunk) h_chunks.push_back(bt::Chunk{k, st, std::min(kChunk, n - st)});
            ++nsys;
        }
        h_first.push_back((int)(h_chunks.size() - wave_chunk_off[w]));
        h_ids.push_back(-1);
        wave_nchunk[w] = h_chunks.size() - wave_chunk_off[w];
        wave_nsys[w] = nsys;
    }
    auto upload = [&](auto** dptr, const auto& vec) -> cudaError_t {
        using T = typename std::decay<decltype(vec)>::type::value_type;
        const size_t n = std::max<size_t>(vec.size(), 1);
        cudaError_t err = cudaMalloc((void**)dptr, n * sizeof(T));
        if (err == cudaSuccess && !vec.empty())
            err = cudaMemcpy(*dptr, vec.data(), vec.size() * sizeof(T), cudaMemcpyHostToDevice);
        b->other_bytes += n * sizeof(T);
        return err;
    };
    e = upload(&b->d_args, h_args);
    if (e == cudaSuccess) e = upload(&b->d_work, h_work);
    if (e == cudaSuccess) e = upload(&b->d_rdesc, h_rd);
    if (e == cudaSuccess) e = upload(&b->d_chunks, h_chunks);
    if (e == cudaSuccess) e = upload(&b->d_first, h_first);
    if (e == cudaSuccess) e = upload(&b->d_sysids, h_ids);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_partial, sizeof(double) * 2 * std::max<size_t>(h_chunks.size(), 1));
    if (e != cudaSuccess) {
        free_batch(b);
        return from_cuda(e);
    }
    // ---- block-order classes -> capture streams
    std::vector<int> ms;
    for (auto& s : b->sys)
        if (std::find(ms.begin(), ms.end(), s.d.m) == ms.end()) ms.push_back(s.d.m);
    std::sort(ms.begin(), ms.end());
    for (int m : ms) {
        const bt::Launchers* L = bt::launchers_for(m);
        e = L->prepare();
        if (e != cudaSuccess) {
            free_batch(b);
            return from_cuda(e);
        }
        cudaStream_t cs;
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            free_batch(b);
            return from_cuda(e);
        }
        b->cls_streams.push_back(cs);
    }
    auto new_event = [&]() {
        cudaEvent_t ev;
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        b->events.push_back(ev);
        return ev;
    };
    // ---- capture
    cudaStream_t origin = b->stream;
    cudaStream_t cap_stream = origin;
    bool own_origin = false;
    if (origin == nullptr) {   // the legacy stream cannot be captured: capture on a private stream
        e = cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking);
        own_origin = true;
    }
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeRelaxed);
    auto run_groups = [&](int w, int phase, int lo, int hi, int step, const std::vector<int>& kinds) -> cudaError_t {
        for (int l = lo; l != hi; l += step)
            for (int kind : kinds)
                for (size_t ci = 0; ci < ms.size(); ++ci)
                    for (int lowv = 0; lowv < 2; ++lowv) {
                        auto it = groups.find({w, phase, l, kind, ms[ci], lowv});
                        if (it == groups.end()) continue;
                        const Group& g = it->second;
                        const bt::Launchers* L = bt::launchers_for(g.m);
                        const int grid = grid_for(L, g.nwork, b->sms);
                        const int2* wk = b->d_work + g.work_off;
                        cudaStream_t cs = b->cls_streams[ci];
                        cudaError_t r;
                        switch (kind) {
                            case 0: r = L->factor_b(b->d_args, wk, g.nwork, 0, g.low, grid, cs); break;
                            case 1: r = L->assemble_b(b->d_args, wk, g.nwork, 0, g.low, grid, cs); break;
                            case 2: r = L->solve_fwd_b(b->d_args, wk, g.nwork, 0, g.low, grid, cs); break;
                            case 3: r = L->assemble_rhs_b(b->d_args, wk, g.nwork, 0, g.low, grid, cs); break;
                            default: r = L->solve_bwd_b(b->d_args, wk, g.nwork, 0, g.low, grid, cs); break;
                        }
                        if (r != cudaSuccess) return r;
                        ++b->graph_nodes;
                    }
        return cudaSuccess;
    };
    auto fork = [&]() {
        cudaEvent_t ev = new_event();
        cudaEventRecord(ev, cap_stream);
        for (auto cs : b->cls_streams) cudaStreamWaitEvent(cs, ev, 0);
    };
    auto join = [&]() {
        for (auto cs : b->cls_streams) {
            cudaEvent_t ev = new_event();
            cudaEventRecord(ev, cs);
            cudaStreamWaitEvent(cap_stream, ev, 0);
        }
    };
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(long long) * 4 * count, cap_stream);
    for (int w = 0; w < b->waves && e == cudaSuccess; ++w) {
        fork();
        // factor: levels ascending, each level's factor then its assembly
        for (int l = 0; l <= maxlev && e == cudaSuccess; ++l) e = run_groups(w, 0, l, l + 1, 1, {0, 1});
        // solve
        if (e == cudaSuccess) e = run_groups(w, 0, 0, maxlev + 1, 1, {2, 3});
        if (e == cudaSuccess) e = run_groups(w, 0, maxlev, -1, -1, {4});
        join();
        if (wave_nsys[w] == 0) continue;
        const bt::Chunk* ch = b->d_chunks + wave_chunk_off[w];
        const int nch = (int)wave_nchunk[w];
        const int grid = std::max(1, std::min(nch, b->sms * 8));
        for (int sweep = 0; sweep < b->ir_sweeps && e == cudaSuccess; ++sweep) {
            bt::k_resid_btri_batch<<<grid, 256, 0, cap_stream>>>(b->d_rdesc, ch, nch);
            fork();
            e = run_groups(w, 1, 0, maxlev + 1, 1, {2, 3});
            if (e == cudaSuccess) e = run_groups(w, 1, maxlev, -1, -1, {4});
            join();
            bt::k_ir_update_batch<<<grid, 256, 0, cap_stream>>>(b->d_rdesc, ch, nch, b->d_partial);
            const int nsys = (int)wave_nsys[w];
            bt::k_reduce_sys<<<std::min(nsys, 1024), 32, 0, cap_stream>>>(b->d_first + wave_first_off[w],
                                                                          b->d_sysids + wave_first_off[w], nsys,
                                                                          b->d_partial, b->d_norms);
            b->graph_nodes += 3;
            if (e == cudaSuccess) e = cudaGetLastError();
        }
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap_stream, &g);
    if (own_origin) cudaStreamDestroy(cap_stream);
    if (e == cudaSuccess) e = e2;
    b->graph = g;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_batch(b);
        return from_cuda(e);
    }
    b->h_status.assign(4 * count, 0);
    b->h_norms.assign(2 * count, 0.0);
    *out = b;
    return BT_OK;
}

bt_status bt_batch_run(bt_batch b) {
    if (!b) return BT_ERR_INVALID;
    return from_cuda(cudaGraphLaunch(b->exec, b->stream));
}

bt_status bt_batch_finish(bt_batch b, double tol, int* status, double* relcorr) {
    if (!b) return BT_ERR_INVALID;
    const int count = (int)b->sys.size();
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->h_status.data(), b->d_status, sizeof(long long) * 4 * count, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->h_norms.data(), b->d_norms, sizeof(double) * 2 * count, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return from_cuda(e);
    bt_status worst = BT_OK;
    for (int k = 0; k < count; ++k) {
        bt_status st = (bt_status)b->h_status[4 * k];
        double rel = 0.0;
        if (b->sys[k].low) {
            const double dd = b->h_norms[2 * k], xx = b->h_norms[2 * k + 1];
            rel = xx > 0 ? std::sqrt(dd / xx) : std::sqrt(dd);
            if (st == BT_OK && !std::isfinite(rel)) st = BT_ERR_NONFINITE;
            if (st == BT_OK && (b->ir_sweeps == 0 || rel > tol)) st = BT_ERR_NOT_CONVERGED;
        }
        if (status) status[k] = (int)st;
        if (relcorr) relcorr[k] = rel;
        if (st != BT_OK && worst == BT_OK) worst = st;
    }
    return worst;
}

bt_status bt_batch_info(bt_batch b, int* waves, int64_t* graph_nodes, int64_t* bytes) {
    if (!b) return BT_ERR_INVALID;
    if (waves) *waves = b->waves;
    if (graph_nodes) *graph_nodes = (int64_t)b->graph_nodes;
    if (bytes) *bytes = (int64_t)(b->arena_bytes + b->other_bytes);
    return BT_OK;
}

void bt_batch_destroy(bt_batch b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
}

}  // extern "C"
