// Host side of libgbrank: error state, device buffers, binomials, the
// staggered-table and packed-trie builders (Sec. III-B and IV of
// Wallerberger & Held).
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstring>

#include "gbr_common.h"

namespace gbr {

static thread_local char g_err[1024] = "";

int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { g_err[0] = 0; }

int DevBuf::alloc(size_t b) {
    release();
    if (b == 0) b = 16;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return set_error(GBR_ENOMEM, "cudaMalloc(%zu) failed: %s", b, cudaGetErrorString(e));
    }
    bytes = b;
    return GBR_OK;
}

int DevBuf::upload(const void *h, size_t b) {
    int rc = alloc(b);
    if (rc) return rc;
    if (b) GBR_CUDA_TRY(cudaMemcpy(p, h, b, cudaMemcpyHostToDevice));
    return GBR_OK;
}

void DevBuf::release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
void set_launch_count(int64_t v) { g_launches.store(v, std::memory_order_relaxed); }

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 152;
    return n;
}

// Pascal's triangle up to n = 64; C(64, 32) < 2^63 so every entry fits.
static struct BinomTable {
    uint64_t c[65][65];
    BinomTable() {
        memset(c, 0, sizeof(c));
        for (int n = 0; n <= 64; ++n) {
            c[n][0] = 1;
            for (int k = 1; k <= n; ++k) c[n][k] = c[n - 1][k - 1] + (k <= n - 1 ? c[n - 1][k] : 0);
        }
    }
} g_binom;

uint64_t binom(int n, int k) {
    if (n < 0 || k < 0 || k > n || n > 64) return 0;
    return g_binom.c[n][k];
}

// Fig. algr: walk the set bits from the least significant one (ctz), adding
// C(c, k) for the k-th set bit at position c.
uint64_t cns_rank_host(uint64_t a) {
    uint64_t i = 0;
    int k = 1;
    while (a) {
        int c = __builtin_ctzll(a);
        a &= a - 1;
        i += binom(c, k);
        ++k;
    }
    return i;
}

int stag_plan(int M, int N, int R, StagDesc *d) {
    if (M < 1 || M > 64) return set_error(GBR_EINVAL, "M=%d out of range 1..64", M);
    if (N < 0 || N > M) return set_error(GBR_EINVAL, "N=%d out of range 0..M", N);
    if (R < 1 || R > 12) return set_error(GBR_EINVAL, "R=%d out of range 1..12", R);
    memset(d, 0, sizeof(*d));
    d->M = M; d->N = N; d->R = R;
    d->Q = (M + R - 1) / R;
    int64_t off = 0;
    for (int q = 0; q < d->Q; ++q) {
        d->shift[q] = q * R;
        d->width[q] = std::min(R, M - q * R);
        d->lo[q] = std::max(0, N - (M - d->shift[q]));
        d->hi[q] = std::min(d->shift[q], N);
        d->off[q] = off;
        off += (int64_t)(d->hi[q] - d->lo[q] + 1) << d->width[q];
    }
    d->entries = off;
    return GBR_OK;
}

// Eq. partrank through Eq. reuse: the N' previously seen set bits are put at
// positions 0..N'-1 and the chunk's bits at M' + c; Fig. algr then yields
// sum_i C(M' + c_i, N' + i), the earlier bits contributing C(j, j+1) = 0.
void stag_fill(StagDesc &d, std::vector<uint64_t> &tab) {
    tab.assign((size_t)d.entries, 0);
    uint64_t mx = 0;
    for (int q = 0; q < d.Q; ++q) {
        int Mp = d.shift[q], w = d.width[q];
        for (int Np = d.lo[q]; Np <= d.hi[q]; ++Np) {
            uint64_t low = Np ? ((Np >= 64) ? ~0ull : ((1ull << Np) - 1)) : 0;
            for (uint64_t r = 0; r < (1ull << w); ++r) {
                uint64_t beta = (r << Mp) | low;
                uint64_t v = cns_rank_host(beta);
                tab[(size_t)(d.off[q] + ((int64_t)(Np - d.lo[q]) << w) + (int64_t)r)] = v;
                mx = std::max(mx, v);
            }
        }
    }
    d.wide = mx > 0xFFFFFFFFull ? 1 : 0;
}

uint64_t stag_rank_host(const StagDesc &d, const std::vector<uint64_t> &tab, uint64_t a) {
    uint64_t i = 0;
    int Np = 0;
    for (int q = 0; q < d.Q; ++q) {
        uint64_t r = (a >> d.shift[q]) & ((1ull << d.width[q]) - 1);
        int row = std::min(std::max(Np, d.lo[q]), d.hi[q]) - d.lo[q];
        i += tab[(size_t)(d.off[q] + ((int64_t)row << d.width[q]) + (int64_t)r)];
        Np += __builtin_popcountll(r);
    }
    return i;
}

void enumerate_combinations(int L, int N, std::vector<uint64_t> &out) {
    out.clear();
    if (N < 0 || N > L) return;
    if (N == 0) { out.push_back(0); return; }
    uint64_t a = (N == 64) ? ~0ull : ((1ull << N) - 1);
    uint64_t lim = (L == 64) ? 0 : (1ull << L);
    while (true) {
        out.push_back(a);
        // next larger number with the same popcount
        uint64_t c = a & (0 - a);
        uint64_t r = a + c;
        if (r == 0) break;                       // overflow past 64 bits
        uint64_t nxt = (((r ^ a) >> 2) / c) | r;
        if (L < 64 && nxt >= lim) break;
        if (nxt <= a) break;
        a = nxt;
    }
}

// ------------------------------------------------------------------ trie

int trie_build(const uint64_t *sorted, int64_t n, int M, int R, TriePlan *plan, std::vector<uint64_t> *t,
               int msb_first) {
    if (M < 1 || M > 64) return set_error(GBR_EINVAL, "trie: M=%d out of range 1..64", M);
    if (R < 1 || R > 16) return set_error(GBR_EINVAL, "trie: R=%d out of range 1..16", R);
    if (n < 1) return set_error(GBR_EINVAL, "trie: empty member set");
    if (!sorted) return set_error(GBR_EINVAL, "trie: NULL member list");
    for (int64_t i = 0; i < n; ++i) {
        if (M < 64 && (sorted[i] >> M)) return set_error(GBR_EINVAL, "trie: member %lld has a bit at or above M", (long long)i);
        if (i && sorted[i] <= sorted[i - 1])
            return set_error(GBR_EINVAL, "trie: members not strictly increasing at %lld", (long long)i);
    }
    TriePlan &P = *plan;
    P.M = M; P.R = R;
    int w0 = M % R ? M % R : R;
    P.H = 1 + (M - w0) / R;
    for (int d = 0, sh = 0; d < P.H; ++d) {
        P.width[d] = d ? R : w0;
        P.shift[d] = msb_first ? M - sh - P.width[d] : sh;
        sh += P.width[d];
    }
    // dispatch key: first dispatched (lowest) chunk most significant
    std::vector<std::pair<uint64_t, uint64_t>> kr((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        uint64_t a = sorted[i], k = 0;
        for (int d = 0; d < P.H; ++d) k = (k << P.width[d]) | ((a >> P.shift[d]) & ((1ull << P.width[d]) - 1));
        kr[(size_t)i] = {k, (uint64_t)i};
    }
    std::sort(kr.begin(), kr.end());
    std::vector<int> below(P.H, 0);
    for (int d = P.H - 2; d >= 0; --d) below[d] = below[d + 1] + P.width[d + 1];
    auto chunk = [&](size_t idx, int d) -> uint64_t {
        return (kr[idx].first >> below[d]) & ((1ull << P.width[d]) - 1);
    };
    // breadth-first: nodes of level d are member ranges in key order, each
    // remembering the slot of its parent that must point at it
    struct Node { int64_t lo, hi, slot; };
    std::vector<Node> cur{{0, n, -1}}, nxt;
    std::vector<uint64_t> &T = *t;
    T.clear();
    P.level_off.assign(P.H + 1, 0);
    for (int d = 0; d < P.H; ++d) {
        P.level_off[d] = (int64_t)T.size();
        nxt.clear();
        for (const Node &nd : cur) {
            uint64_t cmin = chunk((size_t)nd.lo, d), cmax = chunk((size_t)nd.hi - 1, d);
            if (d == 0) { cmin = 0; cmax = (1ull << P.width[0]) - 1; }
            int64_t start = (int64_t)T.size();
            T.resize(T.size() + (size_t)(cmax - cmin + 1), 0);
            if (nd.slot >= 0) T[(size_t)nd.slot] = (uint64_t)(start - (int64_t)cmin);
            int64_t i = nd.lo;
            while (i < nd.hi) {
                uint64_t c = chunk((size_t)i, d);
                int64_t j = i + 1;
                while (j < nd.hi && chunk((size_t)j, d) == c) ++j;
                int64_t slot = start + (int64_t)(c - cmin);
                if (d == P.H - 1) T[(size_t)slot] = kr[(size_t)i].second;
                else nxt.push_back({i, j, slot});
                i = j;
            }
        }
        cur.swap(nxt);
    }
    P.level_off[P.H] = (int64_t)T.size();
    P.size = (int64_t)T.size();
    T.resize(T.size() + ((size_t)1 << R), 0);   // trailing padding
    return GBR_OK;
}

}  // namespace gbr

using namespace gbr;

extern "C" const char *gbr_last_error(void) { return g_err; }

extern "C" int gbr_version(void) { return 1; }

extern "C" int64_t gbr_launch_count(void) { return launch_count(); }

extern "C" int gbr_trie_build_host_ordered(const uint64_t *h_sorted, int64_t n, int M, int R, int msb_first,
                                           uint64_t *h_t, int64_t cap, int64_t *size_out) {
    clear_error();
    if (msb_first != 0 && msb_first != 1) return set_error(GBR_EINVAL, "msb_first=%d must be 0 or 1", msb_first);
    TriePlan plan;
    std::vector<uint64_t> t;
    int rc = trie_build(h_sorted, n, M, R, &plan, &t, msb_first);
    if (rc) return rc;
    if (size_out) *size_out = plan.size;
    if (h_t) {
        if (cap < (int64_t)t.size())
            return set_error(GBR_EINVAL, "trie_build_host: capacity %lld < %lld", (long long)cap, (long long)t.size());
        memcpy(h_t, t.data(), t.size() * sizeof(uint64_t));
    }
    return GBR_OK;
}

extern "C" int gbr_trie_build_host(const uint64_t *h_sorted, int64_t n, int M, int R, uint64_t *h_t, int64_t cap,
                                   int64_t *size_out) {
    return gbr_trie_build_host_ordered(h_sorted, n, M, R, 0, h_t, cap, size_out);
}
