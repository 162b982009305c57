// Host-side choice of the recursion levels (partition counts per level).
#pragma once
#include <vector>

namespace bt {

struct Tuning {
    long long p0 = 0;        // level-0 partitions (0: from ctas_per_sm)
    int ctas_per_sm = 0;     // level-0 target partitions per SM (0: 4 for CTA kernels, 512 for m <= 4)
    int sub_rows = 0;        // block rows per partition on recursion levels (0: 4)
    int top_rows = 0;        // a level with at most this many rows is one partition / direct (0: 8)
    int reduced = 0;         // reduced-system solver: 0 recursive partitions, 1 block cyclic reduction
    int tp_block = 0;        // threads per CTA of the thread-per-partition kernels (0: 128)
    int local = 0;           // level-0 local factorization: 0 block LU + spikes, L >= 1 cyclic reduction of 2^L rows
    int pivot = 0;           // 1: partitions split at breakdown rows, reduced system by banded GEPP
    int serial = 0;          // 1: captured factor+solve sequences on one stream
};

struct LevelShape {
    long long N, p, base, extra, rows;
};

// kind 0: block tridiagonal (last level: one partition); kind 1: BABD (last
// level: direct solve, p = 0).  Returns false on invalid parameters.
inline bool plan_shapes(int kind, long long N, int m, int sms, const Tuning& t, std::vector<LevelShape>& out) {
    out.clear();
    if (kind == 0 && t.local > 0) {
        // local cyclic reduction: no partition levels; the whole matrix is
        // one level handled by the cyclic-reduction kernels
        if (m < 8 || t.local > 62) return false;
        out.push_back(LevelShape{N, 0, 0, 0, N});
        return true;
    }
    const long long top_rows = t.top_rows > 0 ? t.top_rows : 8;
    const long long sub_rows = t.sub_rows >= 2 ? t.sub_rows : 4;
    // level-0 partitions per SM: enough resident warps to hide the Gauss-Jordan
    // latency (m = 8: 2 warps per CTA, m = 16: 4, m = 32: 8; m <= 4: threads)
    const long long per_sm = t.ctas_per_sm > 0 ? t.ctas_per_sm : (m >= 32 ? 3 : m >= 16 ? 4 : m >= 8 ? 12 : 512);
    const long long kmin = (m >= 8) ? 4 : 8;
    long long rows = N;
    for (int l = 0; l < 64; ++l) {
        const bool small = rows <= top_rows;
        long long cap = (kind == 0) ? (rows + 1) / 2 : (rows - 1) / 2;
        if (cap < 1) cap = 1;
        long long parts;
        if (l == 0 && t.p0 > 0) {
            parts = t.p0;
            if (kind == 0 && parts > 1 && parts > cap) return false;
            if (kind == 1 && parts > 1 && parts > cap && rows >= 3) return false;
        } else if (small) {
            parts = 1;
        } else if (l == 0) {
            parts = (long long)sms * per_sm;
            if (rows / kmin < parts) parts = rows / kmin;
        } else {
            parts = rows / sub_rows;
        }
        if (parts < 1) parts = 1;
        if (!(l == 0 && t.p0 > 0) && parts > cap) parts = cap;
        if (kind == 1) {
            if (small || rows < 3) parts = 0;
            if (parts == 1 && l > 0) parts = 0;
            if (l == 0 && t.p0 == 1 && rows >= 3) parts = 1;
        }
        LevelShape s{rows, parts, 0, 0, kind == 0 ? rows : rows + 1};
        if (parts > 0) {
            const long long span = (kind == 0) ? rows : rows - 1;
            s.base = span / parts;
            s.extra = span % parts;
        }
        out.push_back(s);
        if (kind == 0 && parts <= 1) return true;
        if (kind == 0 && t.reduced == 1 && m >= 8) {
            // the reduced system is solved by block cyclic reduction: one more
            // level that holds it, without partitions
            const long long n1 = parts - 1;
            out.push_back(LevelShape{n1, 0, 0, 0, n1});
            return true;
        }
        if (kind == 1 && parts == 0) return true;
        rows = (kind == 0) ? parts - 1 : parts;
    }
    return false;
}

}  // namespace bt
