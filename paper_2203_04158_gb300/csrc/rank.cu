// Ranking and unranking kernels for fixed-popcount sectors (staggered
// lookup, Sec. III-B of Wallerberger & Held) and for packed tries (Sec. IV).
#include <algorithm>
#include <mutex>
#include <cstring>

#include "gbr_common.h"

namespace gbr {

// Per-chunk constants of the staggered tables, passed by value so that the
// unrolled chunk loop reads them from the constant bank.
struct StagK {
    int M, N, Q;
    int shift[kMaxChunks];
    int width[kMaxChunks];
    int lo[kMaxChunks];
    int hi[kMaxChunks];
    int off[kMaxChunks];
};

static StagK to_kernel(const StagDesc &d) {
    StagK k;
    memset(&k, 0, sizeof(k));
    k.M = d.M; k.N = d.N; k.Q = d.Q;
    for (int q = 0; q < d.Q; ++q) {
        k.shift[q] = d.shift[q];
        k.width[q] = d.width[q];
        k.lo[q] = d.lo[q];
        k.hi[q] = d.hi[q];
        k.off[q] = (int)d.off[q];
    }
    return k;
}

constexpr int kRankThreads = 512;
constexpr int kRankItems = 4;           // patterns per thread per tile (independent chains)
constexpr int kSmemTableMax = 96 * 1024;

template <typename E>
__device__ __forceinline__ void stage_table(E *s, const E *__restrict__ g, int64_t entries) {
    // 16-byte copies when possible (tables are allocated with cudaMalloc, so aligned)
    const int64_t bytes = entries * (int64_t)sizeof(E);
    const int64_t n16 = bytes / 16;
    const uint4 *g4 = reinterpret_cast<const uint4 *>(g);
    uint4 *s4 = reinterpret_cast<uint4 *>(s);
    for (int64_t i = threadIdx.x; i < n16; i += blockDim.x) s4[i] = __ldg(g4 + i);
    for (int64_t i = n16 * 16 / (int64_t)sizeof(E) + threadIdx.x; i < entries; i += blockDim.x) s[i] = __ldg(g + i);
    __syncthreads();
}

// Fig. fastrank for one pattern: chunk q adds rank(r_q, M'_q, N'_q), where
// N'_q (set bits below the chunk) is clamped into the admissible rows so a
// pattern outside the sector never reads outside the table.
template <typename E, int QT>
__device__ __forceinline__ E stag_rank(const StagK &d, const E *tab, uint64_t a) {
    E acc = 0;
    int np = 0;
    const int Q = QT > 0 ? QT : d.Q;
#pragma unroll
    for (int q = 0; q < (QT > 0 ? QT : kMaxChunks); ++q) {
        if (QT == 0 && q >= Q) break;
        const uint32_t r = (uint32_t)(a >> d.shift[q]) & ((1u << d.width[q]) - 1u);
        const int row = min(max(np, d.lo[q]), d.hi[q]) - d.lo[q];
        acc += tab[d.off[q] + (row << d.width[q]) + (int)r];
        np += __popc(r);
    }
    return acc;
}

template <typename E, typename RT, int QT>
__global__ void __launch_bounds__(kRankThreads) k_comb_rank(const uint64_t *__restrict__ pat, RT *__restrict__ out,
                                                            int64_t n, const StagK d, const E *__restrict__ gtab,
                                                            int64_t entries, int use_smem, int check) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const E *tab = gtab;
    if (use_smem) {
        stage_table<E>(reinterpret_cast<E *>(smem_raw), gtab, entries);
        tab = reinterpret_cast<const E *>(smem_raw);
    }
    const int64_t tile = (int64_t)kRankThreads * kRankItems;
    for (int64_t base = (int64_t)blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {
        uint64_t a[kRankItems];
#pragma unroll
        for (int j = 0; j < kRankItems; ++j) {
            const int64_t i = base + threadIdx.x + (int64_t)j * kRankThreads;
            a[j] = i < n ? __ldcs(pat + i) : 0ull;
        }
#pragma unroll
        for (int j = 0; j < kRankItems; ++j) {
            const int64_t i = base + threadIdx.x + (int64_t)j * kRankThreads;
            if (i >= n) break;
            RT r = (RT)stag_rank<E, QT>(d, tab, a[j]);
            if (check) {
                const bool ok = (d.M == 64 || (a[j] >> d.M) == 0ull) && __popcll(a[j]) == d.N;
                if (!ok) r = (RT)~(RT)0;
            }
            __stcs(out + i, r);
        }
    }
}

// Same as k_comb_rank on 16-byte aligned input: pairs of patterns per
// 16-byte load, four pairs in flight per thread, pairs of ranks per store.
template <typename RT> struct Pair;
template <> struct Pair<uint32_t> { typedef uint2 t; static __device__ __forceinline__ uint2 make(uint32_t a, uint32_t b) { return make_uint2(a, b); } };
template <> struct Pair<uint64_t> { typedef ulonglong2 t; static __device__ __forceinline__ ulonglong2 make(uint64_t a, uint64_t b) { return make_ulonglong2(a, b); } };

template <typename E, typename RT, int QT>
__global__ void __launch_bounds__(kRankThreads) k_comb_rank_pairs(const ulonglong2 *__restrict__ pat2, RT *__restrict__ out,
                                                                  int64_t n, const StagK d, const E *__restrict__ gtab,
                                                                  int64_t entries, int use_smem, int check) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const E *tab = gtab;
    if (use_smem) {
        stage_table<E>(reinterpret_cast<E *>(smem_raw), gtab, entries);
        tab = reinterpret_cast<const E *>(smem_raw);
    }
    typedef typename Pair<RT>::t P;
    P *out2 = reinterpret_cast<P *>(out);
    const int64_t np = n >> 1;
    const int64_t tile = (int64_t)kRankThreads * kRankItems;
    for (int64_t base = (int64_t)blockIdx.x * tile; base < np; base += (int64_t)gridDim.x * tile) {
        ulonglong2 a[kRankItems];
#pragma unroll
        for (int j = 0; j < kRankItems; ++j) {
            const int64_t p = base + threadIdx.x + (int64_t)j * kRankThreads;
            a[j] = p < np ? __ldcs(pat2 + p) : make_ulonglong2(0ull, 0ull);
        }
#pragma unroll
        for (int j = 0; j < kRankItems; ++j) {
            const int64_t p = base + threadIdx.x + (int64_t)j * kRankThreads;
            if (p >= np) break;
            RT r0 = (RT)stag_rank<E, QT>(d, tab, a[j].x);
            RT r1 = (RT)stag_rank<E, QT>(d, tab, a[j].y);
            if (check) {
                if (!((d.M == 64 || (a[j].x >> d.M) == 0ull) && __popcll(a[j].x) == d.N)) r0 = (RT)~(RT)0;
                if (!((d.M == 64 || (a[j].y >> d.M) == 0ull) && __popcll(a[j].y) == d.N)) r1 = (RT)~(RT)0;
            }
            __stcs(out2 + p, Pair<RT>::make(r0, r1));
        }
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        const uint64_t a = reinterpret_cast<const uint64_t *>(pat2)[n - 1];
        RT r = (RT)stag_rank<E, QT>(d, tab, a);
        if (check && !((d.M == 64 || (a >> d.M) == 0ull) && __popcll(a) == d.N)) r = (RT)~(RT)0;
        out[n - 1] = r;
    }
}

// Eq. unrank: greedy combinatorial-number-system decomposition, the k-th set
// bit at the largest c with C(c, k) <= remaining rank.
template <typename RT>
__global__ void k_comb_unrank(const RT *__restrict__ rank, uint64_t *__restrict__ pat, int64_t n, int M, int N,
                              uint64_t dim, const uint64_t *__restrict__ binom65) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t r = (uint64_t)rank[i];
        uint64_t a = 0;
        if (r >= dim) {
            a = ~0ull;
        } else {
            int c = M - 1;
            for (int k = N; k >= 1; --k) {
                while (c >= 0 && __ldg(binom65 + c * 65 + k) > r) --c;
                a |= 1ull << c;
                r -= __ldg(binom65 + c * 65 + k);
                --c;
            }
        }
        pat[i] = a;
    }
}

// ------------------------------------------------------------------ trie

struct TrieK {
    int H;
    int shift[kMaxChunks];
    int width[kMaxChunks];
};

// Loads with an L2 eviction priority: the upper levels of a trie (a few tens
// of MB, touched by every query) are kept in L2 with evict_last while the
// deep levels, read once per query at random, go with evict_first.
template <typename E> __device__ __forceinline__ E ld_policy(const E *p, uint64_t pol);
template <> __device__ __forceinline__ uint32_t ld_policy<uint32_t>(const uint32_t *p, uint64_t pol) {
    uint32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
template <> __device__ __forceinline__ uint64_t ld_policy<uint64_t>(const uint64_t *p, uint64_t pol) {
    uint64_t v;
    asm volatile("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
    return v;
}

// Fig. trielookup for kRankItems independent patterns per thread, the walks
// interleaved so that their dependent loads overlap.  Entries are unsigned
// and the pointer arithmetic wraps, so the stored (start - smallest child)
// works even where it is negative; every index is clamped into the table.
template <typename E, typename RT, int HT>
__global__ void __launch_bounds__(kRankThreads) k_trie_rank(const uint64_t *__restrict__ pat, RT *__restrict__ out,
                                                            int64_t n, const TrieK d, const E *__restrict__ t,
                                                            int64_t padded, int64_t smem_entries, int64_t hot_end,
                                                            const uint64_t *__restrict__ members, int64_t n_members,
                                                            int check) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    E *s = reinterpret_cast<E *>(smem_raw);
    if (smem_entries > 0) stage_table<E>(s, t, smem_entries);
    const E last = (E)(padded - 1);
    const E sm_end = (E)smem_entries;
    const E hot = (E)hot_end;
    uint64_t pol_last, pol_first;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol_last));
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol_first));
    const int H = HT > 0 ? HT : d.H;
    const int64_t tile = (int64_t)kRankThreads * kRankItems;
    for (int64_t base = (int64_t)blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {
        uint64_t a[kRankItems];
        E k[kRankItems];
#pragma unroll
        for (int j = 0; j < kRankItems; ++j) {
            const int64_t i = base + threadIdx.x + (int64_t)j * kRankThreads;
            a[j] = i < n ? __ldcs(pat + i) : 0ull;
            k[j] = 0;
        }
#pragma unroll
        for (int lvl = 0; lvl < (HT > 0 ? HT : kMaxChunks); ++lvl) {
            if (HT == 0 && lvl >= H) break;
            const uint32_t mask = (1u << d.width[lvl]) - 1u;
#pragma unroll
            for (int j = 0; j < kRankItems; ++j) {
                E idx = k[j] + (E)((uint32_t)(a[j] >> d.shift[lvl]) & mask);
                idx = idx > last ? last : idx;
                k[j] = idx < sm_end ? s[idx] : ld_policy<E>(t + idx, idx < hot ? pol_last : pol_first);
            }
        }
#pragma unroll
        for (int j = 0; j < kRankItems; ++j) {
            const int64_t i = base + threadIdx.x + (int64_t)j * kRankThreads;
            if (i >= n) break;
            RT r = (RT)k[j];
            if (check) {
                const bool ok = (uint64_t)k[j] < (uint64_t)n_members && ld_policy<uint64_t>(members + (uint64_t)k[j], pol_first) == a[j];
                if (!ok) r = (RT)~(RT)0;
            }
            __stcs(out + i, r);
        }
    }
}

// Bisection over the sorted member list -- the established method that the
// paper's tries replace (Sec. II, last paragraph; Sec. V-A), kept as the
// comparison point.  Fixed trip count (ceil log2(n+1) halvings) so that the
// kRankItems searches of a thread interleave.
template <typename RT>
__global__ void __launch_bounds__(kRankThreads) k_list_rank(const uint64_t *__restrict__ pat, RT *__restrict__ out,
                                                            int64_t n, const uint64_t *__restrict__ members,
                                                            int64_t nm, int steps, int check) {
    const int64_t tile = (int64_t)kRankThreads * kRankItems;
    for (int64_t base = (int64_t)blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {
        uint64_t a[kRankItems];
        int64_t lo[kRankItems], len[kRankItems];
#pragma unroll
        for (int j = 0; j < kRankItems; ++j) {
            const int64_t i = base + threadIdx.x + (int64_t)j * kRankThreads;
            a[j] = i < n ? __ldcs(pat + i) : 0ull;
            lo[j] = 0;
            len[j] = nm;
        }
        for (int s = 0; s < steps; ++s) {
#pragma unroll
            for (int j = 0; j < kRankItems; ++j) {
                // lower bound: first index whose member is >= a
                const int64_t half = len[j] >> 1;
                if (len[j] > 0) {
                    const uint64_t m = __ldg(members + lo[j] + half);
                    if (m < a[j]) { lo[j] += half + 1; len[j] -= half + 1; } else { len[j] = half; }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kRankItems; ++j) {
            const int64_t i = base + threadIdx.x + (int64_t)j * kRankThreads;
            if (i >= n) break;
            RT r = (RT)lo[j];
            if (check && !(lo[j] < nm && __ldg(members + lo[j]) == a[j])) r = (RT)~(RT)0;
            __stcs(out + i, r);
        }
    }
}

template <typename RT>
__global__ void k_list_unrank(const RT *__restrict__ rank, uint64_t *__restrict__ pat, int64_t n,
                              const uint64_t *__restrict__ members, int64_t n_members) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t r = (uint64_t)rank[i];
        pat[i] = r < (uint64_t)n_members ? __ldg(members + r) : ~0ull;
    }
}

static int grid_for(int64_t n, int64_t per_block, int blocks_per_sm) {
    int64_t b = (n + per_block - 1) / per_block;
    int64_t cap = (int64_t)sm_count() * blocks_per_sm;
    return (int)std::max<int64_t>(1, std::min(b, cap));
}

template <typename E, typename RT>
static int launch_comb_rank(const gbr_comb *c, const uint64_t *pat, RT *out, int64_t n, int check, cudaStream_t st) {
    const StagK d = to_kernel(c->desc);
    const int64_t tbytes = c->desc.entries * (int64_t)sizeof(E);
    const int use_smem = tbytes <= kSmemTableMax;
    const size_t smem = use_smem ? (size_t)tbytes : 0;
    int per_sm = use_smem ? std::max<int>(1, std::min<int>(4, (int)((200 * 1024) / std::max<int64_t>(tbytes, 1)))) : 4;
    const int grid = grid_for(n, (int64_t)kRankThreads * kRankItems, per_sm);
    const int grid2 = grid_for((n >> 1) + 1, (int64_t)kRankThreads * kRankItems, per_sm);
    const E *tab = c->table.as<E>();
    const bool pairs = (((uintptr_t)pat & 15u) == 0) && (((uintptr_t)out & (2 * sizeof(RT) - 1)) == 0);
#define GBR_COMB_CASE(QV)                                                                                  \
    case QV: {                                                                                             \
        if (pairs) {                                                                                       \
            auto kern = k_comb_rank_pairs<E, RT, QV>;                                                      \
            if (smem > 48 * 1024) GBR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
            kern<<<grid2, kRankThreads, smem, st>>>(reinterpret_cast<const ulonglong2 *>(pat), out, n, d, tab, \
                                                    c->desc.entries, use_smem, check);                     \
        } else {                                                                                           \
            auto kern = k_comb_rank<E, RT, QV>;                                                            \
            if (smem > 48 * 1024) GBR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
            kern<<<grid, kRankThreads, smem, st>>>(pat, out, n, d, tab, c->desc.entries, use_smem, check); \
        }                                                                                                  \
        break;                                                                                             \
    }
    switch (d.Q) {
        GBR_COMB_CASE(1)
        GBR_COMB_CASE(2)
        GBR_COMB_CASE(3)
        GBR_COMB_CASE(4)
        GBR_COMB_CASE(5)
        GBR_COMB_CASE(6)
        GBR_COMB_CASE(7)
        GBR_COMB_CASE(8)
        default: GBR_COMB_CASE(0)
    }
#undef GBR_COMB_CASE
    GBR_LAUNCH_CHECK();
    count_launches(1);
    return GBR_OK;
}

// The walk reads the leading ("hot") levels with the L2 evict_last policy.
// The L2 keeps such lines only inside its persisting set-aside, which is
// empty unless the context asks for one, so the hot levels were evicted by
// the random reads of the large levels.  This sizes the set-aside to the hot
// levels (at most the device's maximum), once per process and device; the
// set-aside belongs to this process's CUDA context and ends with it.
static size_t g_persist_done[64] = {0};
static std::mutex g_persist_mu;

size_t ensure_persisting_l2(size_t bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lock(g_persist_mu);
    if (g_persist_done[dev] >= bytes) return g_persist_done[dev];
    int maxp = 0;
    if (cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, dev) != cudaSuccess || maxp <= 0) {
        cudaGetLastError();
        return 0;
    }
    size_t cur = 0;
    cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
    const size_t want = std::min(bytes, (size_t)maxp);
    if (cur < want && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess) {
        cudaGetLastError();   // no set-aside on this device (e.g. a MIG slice): the walk still runs
        return 0;
    }
    g_persist_done[dev] = std::max(cur, want);
    return g_persist_done[dev];
}

template <typename E, typename RT>
static int launch_trie_rank(const gbr_trie *T, const uint64_t *pat, RT *out, int64_t n, int check, cudaStream_t st) {
    ensure_persisting_l2((size_t)T->hot_entries * sizeof(E));
    TrieK d;
    memset(&d, 0, sizeof(d));
    d.H = T->H;
    for (int l = 0; l < T->H; ++l) { d.shift[l] = T->shift[l]; d.width[l] = T->width[l]; }
    const size_t smem = (size_t)T->smem_entries * sizeof(E);
    const int grid = grid_for(n, (int64_t)kRankThreads * kRankItems, 4);
#define GBR_TRIE_CASE(HV)                                                                                  \
    case HV: {                                                                                             \
        auto kern = k_trie_rank<E, RT, HV>;                                                                \
        if (smem > 48 * 1024) GBR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        kern<<<grid, kRankThreads, smem, st>>>(pat, out, n, d, T->t.as<E>(), T->padded, T->smem_entries,   \
                                               T->hot_entries,                                             \
                                               T->members.as<uint64_t>(), T->n_members, check);            \
        break;                                                                                             \
    }
    switch (d.H) {
        GBR_TRIE_CASE(1)
        GBR_TRIE_CASE(2)
        GBR_TRIE_CASE(3)
        GBR_TRIE_CASE(4)
        GBR_TRIE_CASE(5)
        GBR_TRIE_CASE(6)
        GBR_TRIE_CASE(8)
        default: GBR_TRIE_CASE(0)
    }
#undef GBR_TRIE_CASE
    GBR_LAUNCH_CHECK();
    count_launches(1);
    return GBR_OK;
}

static int check_io(const void *a, const void *b, int64_t n, int rank_bits) {
    if (n < 0) return set_error(GBR_EINVAL, "n=%lld < 0", (long long)n);
    if (n > 0 && (!a || !b)) return set_error(GBR_EINVAL, "NULL buffer");
    if (rank_bits != 32 && rank_bits != 64) return set_error(GBR_EINVAL, "rank_bits=%d must be 32 or 64", rank_bits);
    if (n > 0 && (((uintptr_t)a | (uintptr_t)b) & 3u)) return set_error(GBR_EINVAL, "buffers must be 4-byte aligned");
    return GBR_OK;
}

}  // namespace gbr

using namespace gbr;

extern "C" int gbr_comb_create(int M, int N, int R, gbr_comb **out) {
    clear_error();
    if (!out) return set_error(GBR_EINVAL, "out is NULL");
    *out = nullptr;
    gbr_comb *c = new (std::nothrow) gbr_comb();
    if (!c) return set_error(GBR_ENOMEM, "host allocation failed");
    int rc = stag_plan(M, N, R, &c->desc);
    if (rc) { delete c; return rc; }
    if (c->desc.entries > (int64_t)1 << 30) { delete c; return set_error(GBR_EINVAL, "staggered table too large"); }
    std::vector<uint64_t> tab;
    stag_fill(c->desc, tab);
    c->dim = binom(M, N);
    if (c->desc.wide) {
        rc = c->table.upload(tab.data(), tab.size() * sizeof(uint64_t));
    } else {
        std::vector<uint32_t> t32(tab.begin(), tab.end());
        rc = c->table.upload(t32.data(), t32.size() * sizeof(uint32_t));
    }
    if (!rc) {
        std::vector<uint64_t> b(65 * 65);
        for (int i = 0; i <= 64; ++i)
            for (int k = 0; k <= 64; ++k) b[(size_t)(i * 65 + k)] = binom(i, k);
        rc = c->binom.upload(b.data(), b.size() * sizeof(uint64_t));
    }
    if (rc) { delete c; return rc; }
    *out = c;
    return GBR_OK;
}

extern "C" void gbr_comb_destroy(gbr_comb *c) { delete c; }

extern "C" int gbr_comb_info(const gbr_comb *c, uint64_t *dim, int64_t *table_bytes) {
    clear_error();
    if (!c) return set_error(GBR_EINVAL, "NULL handle");
    if (dim) *dim = c->dim;
    if (table_bytes) *table_bytes = c->desc.entries * (c->desc.wide ? 8 : 4);
    return GBR_OK;
}

extern "C" int gbr_comb_rank(const gbr_comb *c, const uint64_t *d_pat, void *d_rank, int rank_bits, int64_t n,
                             int check, void *stream) {
    clear_error();
    if (!c) return set_error(GBR_EINVAL, "NULL handle");
    int rc = check_io(d_pat, d_rank, n, rank_bits);
    if (rc) return rc;
    if (((uintptr_t)d_pat & 7u) || (rank_bits == 64 && ((uintptr_t)d_rank & 7u)))
        return set_error(GBR_EINVAL, "64-bit buffers must be 8-byte aligned");
    if (rank_bits == 32 && c->dim > 0x100000000ull)
        return set_error(GBR_EINVAL, "C(M,N)=%llu does not fit 32-bit ranks", (unsigned long long)c->dim);
    if (n == 0) return GBR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (c->desc.wide) {
        if (rank_bits == 32) return launch_comb_rank<uint64_t, uint32_t>(c, d_pat, (uint32_t *)d_rank, n, check, st);
        return launch_comb_rank<uint64_t, uint64_t>(c, d_pat, (uint64_t *)d_rank, n, check, st);
    }
    if (rank_bits == 32) return launch_comb_rank<uint32_t, uint32_t>(c, d_pat, (uint32_t *)d_rank, n, check, st);
    return launch_comb_rank<uint32_t, uint64_t>(c, d_pat, (uint64_t *)d_rank, n, check, st);
}

extern "C" int gbr_comb_unrank(const gbr_comb *c, const void *d_rank, int rank_bits, uint64_t *d_pat, int64_t n,
                               void *stream) {
    clear_error();
    if (!c) return set_error(GBR_EINVAL, "NULL handle");
    int rc = check_io(d_rank, d_pat, n, rank_bits);
    if (rc) return rc;
    if (((uintptr_t)d_pat & 7u) || (rank_bits == 64 && ((uintptr_t)d_rank & 7u)))
        return set_error(GBR_EINVAL, "64-bit buffers must be 8-byte aligned");
    if (n == 0) return GBR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = grid_for(n, 256, 16);
    if (rank_bits == 32)
        k_comb_unrank<uint32_t><<<grid, 256, 0, st>>>((const uint32_t *)d_rank, d_pat, n, c->desc.M, c->desc.N, c->dim,
                                                      c->binom.as<uint64_t>());
    else
        k_comb_unrank<uint64_t><<<grid, 256, 0, st>>>((const uint64_t *)d_rank, d_pat, n, c->desc.M, c->desc.N, c->dim,
                                                      c->binom.as<uint64_t>());
    GBR_LAUNCH_CHECK();
    count_launches(1);
    return GBR_OK;
}

namespace gbr {
// Handle from a trie plan and its table (entries as uint64, padding included).
static int trie_upload(const uint64_t *h_sorted, int64_t n, int M, int R, int msb_first, const TriePlan &plan,
                       std::vector<uint64_t> &t, gbr_trie **out) {
    int rc = GBR_OK;
    gbr_trie *T = new (std::nothrow) gbr_trie();
    if (!T) return set_error(GBR_ENOMEM, "host allocation failed");
    T->M = M; T->R = R; T->H = plan.H;
    T->msb_first = msb_first;
    for (int l = 0; l < plan.H; ++l) { T->width[l] = plan.width[l]; T->shift[l] = plan.shift[l]; }
    T->n_members = n;
    T->size = plan.size;
    T->padded = (int64_t)t.size();
    T->wide = (T->padded > (int64_t)0xFFFFFFFFll || n > (int64_t)0xFFFFFFFFll) ? 1 : 0;
    const int eb = T->wide ? 8 : 4;
    // leading whole levels that fit a 32 KiB shared-memory budget
    T->smem_levels = 0;
    T->smem_entries = 0;
    for (int l = 0; l < plan.H; ++l) {
        if (plan.level_off[l + 1] * eb > 32 * 1024) break;
        T->smem_levels = l + 1;
        T->smem_entries = plan.level_off[l + 1];
    }
    // leading whole levels that fit 96 MB (of the 126 MB L2): kept in L2 by the walk
    T->hot_entries = 0;
    for (int l = 0; l < plan.H; ++l) {
        if (plan.level_off[l + 1] * eb > ((int64_t)96 << 20)) break;
        T->hot_entries = plan.level_off[l + 1];
    }
    if (T->wide) {
        rc = T->t.upload(t.data(), t.size() * 8);
    } else {
        std::vector<uint32_t> t32(t.size());
        for (size_t i = 0; i < t.size(); ++i) t32[i] = (uint32_t)t[i];   // wraps negative offsets on purpose
        std::vector<uint64_t>().swap(t);
        rc = T->t.upload(t32.data(), t32.size() * 4);
    }
    if (!rc) rc = T->members.upload(h_sorted, (size_t)n * 8);
    if (rc) { delete T; return rc; }
    *out = T;
    return GBR_OK;
}
}  // namespace gbr

extern "C" int gbr_trie_create_ordered(const uint64_t *h_sorted, int64_t n, int M, int R, int msb_first,
                                       gbr_trie **out) {
    clear_error();
    if (!out) return set_error(GBR_EINVAL, "out is NULL");
    *out = nullptr;
    if (msb_first != 0 && msb_first != 1) return set_error(GBR_EINVAL, "msb_first=%d must be 0 or 1", msb_first);
    TriePlan plan;
    std::vector<uint64_t> t;
    int rc = trie_build(h_sorted, n, M, R, &plan, &t, msb_first);
    if (rc) return rc;
    return trie_upload(h_sorted, n, M, R, msb_first, plan, t, out);
}

extern "C" int gbr_trie_create_from_table(const uint64_t *h_sorted, int64_t n, int M, int R, int msb_first,
                                          const uint64_t *h_t, int64_t len, gbr_trie **out) {
    clear_error();
    if (!out) return set_error(GBR_EINVAL, "out is NULL");
    *out = nullptr;
    if (msb_first != 0 && msb_first != 1) return set_error(GBR_EINVAL, "msb_first=%d must be 0 or 1", msb_first);
    if (!h_t) return set_error(GBR_EINVAL, "NULL table");
    TriePlan plan;
    std::vector<uint64_t> t;
    int rc = trie_build(h_sorted, n, M, R, &plan, &t, msb_first);   // the member list's layout
    if (rc) return rc;
    if (len != (int64_t)t.size())
        return set_error(GBR_EINVAL, "table of %lld entries, the member list's trie has %lld", (long long)len,
                         (long long)t.size());
    t.assign(h_t, h_t + len);
    return trie_upload(h_sorted, n, M, R, msb_first, plan, t, out);
}

extern "C" int gbr_trie_create(const uint64_t *h_sorted, int64_t n, int M, int R, gbr_trie **out) {
    return gbr_trie_create_ordered(h_sorted, n, M, R, 0, out);
}

extern "C" void gbr_trie_destroy(gbr_trie *t) { delete t; }

extern "C" int gbr_trie_info(const gbr_trie *t, int64_t *n_members, int64_t *n_elements, int *entry_bytes, int *levels) {
    clear_error();
    if (!t) return set_error(GBR_EINVAL, "NULL handle");
    if (n_members) *n_members = t->n_members;
    if (n_elements) *n_elements = t->size;
    if (entry_bytes) *entry_bytes = t->wide ? 8 : 4;
    if (levels) *levels = t->H;
    return GBR_OK;
}

extern "C" int gbr_trie_rank(const gbr_trie *t, const uint64_t *d_pat, void *d_rank, int rank_bits, int64_t n,
                             int check, void *stream) {
    clear_error();
    if (!t) return set_error(GBR_EINVAL, "NULL handle");
    int rc = check_io(d_pat, d_rank, n, rank_bits);
    if (rc) return rc;
    if (((uintptr_t)d_pat & 7u) || (rank_bits == 64 && ((uintptr_t)d_rank & 7u)))
        return set_error(GBR_EINVAL, "64-bit buffers must be 8-byte aligned");
    if (rank_bits == 32 && t->n_members > (int64_t)0x100000000ll)
        return set_error(GBR_EINVAL, "member count does not fit 32-bit ranks");
    if (n == 0) return GBR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (t->wide) {
        if (rank_bits == 32) return launch_trie_rank<uint64_t, uint32_t>(t, d_pat, (uint32_t *)d_rank, n, check, st);
        return launch_trie_rank<uint64_t, uint64_t>(t, d_pat, (uint64_t *)d_rank, n, check, st);
    }
    if (rank_bits == 32) return launch_trie_rank<uint32_t, uint32_t>(t, d_pat, (uint32_t *)d_rank, n, check, st);
    return launch_trie_rank<uint32_t, uint64_t>(t, d_pat, (uint64_t *)d_rank, n, check, st);
}

extern "C" int gbr_trie_rank_bisect(const gbr_trie *t, const uint64_t *d_pat, void *d_rank, int rank_bits, int64_t n,
                                    int check, void *stream) {
    clear_error();
    if (!t) return set_error(GBR_EINVAL, "NULL handle");
    int rc = check_io(d_pat, d_rank, n, rank_bits);
    if (rc) return rc;
    if (((uintptr_t)d_pat & 7u) || (rank_bits == 64 && ((uintptr_t)d_rank & 7u)))
        return set_error(GBR_EINVAL, "64-bit buffers must be 8-byte aligned");
    if (rank_bits == 32 && t->n_members > (int64_t)0x100000000ll)
        return set_error(GBR_EINVAL, "member count does not fit 32-bit ranks");
    if (n == 0) return GBR_OK;
    int steps = 0;
    while (((int64_t)1 << steps) <= t->n_members) ++steps;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = grid_for(n, (int64_t)kRankThreads * kRankItems, 8);
    if (rank_bits == 32)
        k_list_rank<uint32_t><<<grid, kRankThreads, 0, st>>>(d_pat, (uint32_t *)d_rank, n, t->members.as<uint64_t>(),
                                                             t->n_members, steps, check);
    else
        k_list_rank<uint64_t><<<grid, kRankThreads, 0, st>>>(d_pat, (uint64_t *)d_rank, n, t->members.as<uint64_t>(),
                                                             t->n_members, steps, check);
    GBR_LAUNCH_CHECK();
    count_launches(1);
    return GBR_OK;
}

extern "C" int gbr_trie_unrank(const gbr_trie *t, const void *d_rank, int rank_bits, uint64_t *d_pat, int64_t n,
                               void *stream) {
    clear_error();
    if (!t) return set_error(GBR_EINVAL, "NULL handle");
    int rc = check_io(d_rank, d_pat, n, rank_bits);
    if (rc) return rc;
    if (((uintptr_t)d_pat & 7u) || (rank_bits == 64 && ((uintptr_t)d_rank & 7u)))
        return set_error(GBR_EINVAL, "64-bit buffers must be 8-byte aligned");
    if (n == 0) return GBR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = grid_for(n, 256, 16);
    if (rank_bits == 32)
        k_list_unrank<uint32_t><<<grid, 256, 0, st>>>((const uint32_t *)d_rank, d_pat, n, t->members.as<uint64_t>(),
                                                      t->n_members);
    else
        k_list_unrank<uint64_t><<<grid, 256, 0, st>>>((const uint64_t *)d_rank, d_pat, n, t->members.as<uint64_t>(),
                                                      t->n_members);
    GBR_LAUNCH_CHECK();
    count_launches(1);
    return GBR_OK;
}
