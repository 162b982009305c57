// bt_solve_noalloc: a one-shot FP64 block tridiagonal factor + solve that
// performs no device allocation.  It exists for callers that are not allowed
// to call cudaMalloc: code running inside a host application that owns all
// device memory through its own pool or budget, or a latency-critical loop
// where cudaMalloc's implicit device synchronisation, or its possible
// failure, cannot be accepted.  Such callers pass inputs and outputs; every
// intermediate (the factors of every recursion level, the reduced systems,
// the status word) lives in one file-scope device array of fixed size.
//
// The array is part of the library's device image: every GPU that loads the
// library holds its kNoallocScratchBytes until the process exits.  All calls
// share it and it keeps the previous call's contents, so the status word is
// cleared at the start of every call (every other buffer is written before it
// is read).  Calls whose GPU work overlaps (different streams or host
// threads) race on the array: callers must serialise them.
#include <cuda_runtime.h>
#include <cstdint>
#include <mutex>

#include "../../include/bt.h"
#include "bt_launch.h"
#include "bt_level.h"

namespace {

constexpr size_t kNoallocScratchBytes = BT_NOALLOC_SCRATCH_BYTES;   // 8 MiB
constexpr int kMaxLevels = 40;
constexpr int kMaxDevices = 64;
constexpr long long kTopRows = 8;
constexpr long long kSubLevelRows = 4;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {

// Device address of g_noalloc_scratch for each device, found once per device
// (with that device current) by cudaGetSymbolAddress.  In host code the name
// g_noalloc_scratch is only a host-side stand-in, never a device address.
void* g_scratch_ptr[kMaxDevices];
cudaError_t g_scratch_err[kMaxDevices];
std::once_flag g_scratch_once[kMaxDevices];

cudaError_t scratch_for_device(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(g_scratch_once[dev], [dev] {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        g_scratch_ptr[dev] = (e == cudaSuccess) ? p : nullptr;
        g_scratch_err[dev] = e;
    });
    *out = g_scratch_ptr[dev];
    return g_scratch_err[dev];
}

long long parts_for(long long rows, int m, int level, int sms) {
    long long cap = (rows + 1) / 2;
    if (cap < 1) cap = 1;
    long long target;
    if (level == 0) {
        target = (long long)sms * ((m >= 8) ? 4 : 512);
        const long long byk = rows / ((m >= 8) ? 4 : 8);
        if (byk < target) target = byk;
    } else {
        target = rows / kSubLevelRows;
    }
    if (target < 1) target = 1;
    if (target > cap) target = cap;
    return target;
}

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

// Levels and the layout of the scratch; with c.base == nullptr only measures.
int plan_levels(bt::LevelArgs* lv, long long N, int m, int nr, int sms, Cursor& c, long long** status) {
    const long long mm = (long long)m * m;
    *status = (long long*)c.take(4 * sizeof(long long));
    long long rows = N;
    int n = 0;
    for (;;) {
        if (n >= kMaxLevels) return -1;
        bt::LevelArgs& a = lv[n];
        a = bt::LevelArgs{};
        a.mode = 0;
        a.level = n;
        a.N = rows;
        const long long parts = (rows <= kTopRows) ? 1 : parts_for(rows, m, n, sms);
        a.p = parts;
        a.base = rows / parts;
        a.extra = rows % parts;
        a.Dinv = c.take(sizeof(double) * rows * mm);
        a.Y = c.take(sizeof(double) * rows * mm);
        a.Zc = c.take(sizeof(double) * rows * mm);
        a.Pf = c.take(sizeof(double) * parts * mm);
        a.Qf = c.take(sizeof(double) * parts * mm);
        a.Hf = c.take(sizeof(double) * parts * m * nr);
        a.nr = nr;
        a.status = *status;
        if (n >= 1) {
            bt::LevelArgs& u = lv[n - 1];
            double* Bn = (double*)c.take(sizeof(double) * rows * mm);
            double* Dn = (double*)c.take(sizeof(double) * rows * mm);
            double* Cn = (double*)c.take(sizeof(double) * rows * mm);
            double* Fn = (double*)c.take(sizeof(double) * rows * m * nr);
            double* Xn = (double*)c.take(sizeof(double) * rows * m * nr);
            u.Bn = Bn; u.Dn = Dn; u.Cn = Cn; u.Fn = Fn; u.Xn = Xn;
            a.B = Bn; a.D = Dn; a.C = Cn; a.F = Fn; a.X = Xn;
        }
        ++n;
        if (parts <= 1) break;
        rows = parts - 1;
    }
    return n;
}

bt_status to_status(cudaError_t e) {
    if (e == cudaSuccess) return BT_OK;
    return BT_ERR_CUDA;
}

}  // namespace

extern "C" bt_status bt_solve_noalloc(int64_t nblk, int m, const double* B, const double* D, const double* C,
                                      const double* F, double* X, int nrhs, void* stream,
                                      int64_t* required_bytes) {
    if (required_bytes) *required_bytes = 0;
    const bt::Launchers* L = bt::launchers_for(m);
    if (!L || nblk < 1 || nrhs < 1 || nrhs > 32 || !D || !F || !X || F == X) return BT_ERR_INVALID;
    if (nblk > 1 && (!B || !C)) return BT_ERR_INVALID;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return to_status(e);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
    bt::LevelArgs lv[kMaxLevels];
    long long* status = nullptr;
    Cursor measure{nullptr, 0};
    const int nlev = plan_levels(lv, nblk, m, nrhs, sms, measure, &status);
    if (required_bytes) *required_bytes = (int64_t)measure.off;
    if (nlev < 1 || measure.off > kNoallocScratchBytes) return BT_ERR_INVALID;
    void* base = nullptr;
    e = scratch_for_device(dev, &base);
    if (e != cudaSuccess || !base) return to_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e);
    Cursor real{(char*)base, 0};
    plan_levels(lv, nblk, m, nrhs, sms, real, &status);
    cudaStream_t s = (cudaStream_t)stream;
    lv[0].B = B;
    lv[0].D = D;
    lv[0].C = C;
    lv[0].F = F;
    lv[0].X = X;
    const int top = nlev - 1;
    e = cudaMemsetAsync(status, 0, 4 * sizeof(long long), s);
    for (int l = 0; l <= top && e == cudaSuccess; ++l) {
        e = L->factor(lv[l], false, s);
        if (e == cudaSuccess && l < top) e = L->assemble(lv[l], false, s);
    }
    for (int l = 0; l < top && e == cudaSuccess; ++l) {
        e = L->solve_fwd(lv[l], false, s);
        if (e == cudaSuccess) e = L->assemble_rhs(lv[l], false, s);
    }
    if (e == cudaSuccess) e = L->solve_fwd(lv[top], false, s);
    if (e == cudaSuccess) e = L->solve_bwd(lv[top], false, s);
    for (int l = top - 1; l >= 0 && e == cudaSuccess; --l) e = L->solve_bwd(lv[l], false, s);
    long long st[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(st, status, sizeof(st), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return to_status(e);
    return st[0] == 0 ? BT_OK : (bt_status)st[0];
}
