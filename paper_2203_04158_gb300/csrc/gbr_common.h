// Internal declarations shared by the translation units of libgbrank.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "gbrank.h"

namespace gbr {

// ----------------------------------------------------------------- errors

int set_error(int code, const char *fmt, ...);
void clear_error();

#define GBR_CUDA_TRY(call)                                                                      \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return ::gbr::set_error(GBR_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                    __FILE__, __LINE__);                                        \
    } while (0)

#define GBR_LAUNCH_CHECK()                                                                      \
    do {                                                                                        \
        cudaError_t e_ = cudaGetLastError();                                                    \
        if (e_ != cudaSuccess)                                                                  \
            return ::gbr::set_error(GBR_ECUDA, "kernel launch failed: %s (%s:%d)",              \
                                    cudaGetErrorString(e_), __FILE__, __LINE__);                \
    } while (0)

// Owned device allocation (freed in the destructor).
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    int alloc(size_t b);
    int upload(const void *h, size_t b);
    void release();
    template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

int sm_count();

// Process-wide count of kernel launches issued by the library.
void count_launches(int64_t n);
int64_t launch_count();
void set_launch_count(int64_t v);

// ------------------------------------------------------------- binomials

// C(n, k) for 0 <= n, k <= 64 (0 for k > n), exact in 64 bits.
uint64_t binom(int n, int k);

// --------------------------------------------------- staggered lookup tables
//
// Sector C^M_N split into chunks of R bits from the least significant end
// (Fig. fastrank).  Chunk q covers bits [shift_q, shift_q + width_q).  For the
// chunk the table holds rank(r, M' = shift_q, N') of Eq. partrank for every
// r < 2^width_q and every N' admissible for N:
//   lo_q = max(0, N - (M - shift_q)) <= N' <= hi_q = min(shift_q, N).
// Row (q, N') starts at entry off_q + (N' - lo_q) * 2^width_q, r varying
// fastest (Sec. III-B, layout remark).
constexpr int kMaxChunks = 64;

struct StagDesc {
    int M, N, R, Q;
    int shift[kMaxChunks];
    int width[kMaxChunks];
    int lo[kMaxChunks];
    int hi[kMaxChunks];
    int64_t off[kMaxChunks];
    int64_t entries;
    int wide;        // 1: 64-bit entries
};

int stag_plan(int M, int N, int R, StagDesc *d);
// Fills the table (entries as uint64) through Eq. reuse and Fig. algr.
void stag_fill(StagDesc &d, std::vector<uint64_t> &tab);
// Host reference of Fig. fastrank on the same table (used by host builders).
uint64_t stag_rank_host(const StagDesc &d, const std::vector<uint64_t> &tab, uint64_t a);
// Fig. algr (combinadics with ctz) for an arbitrary pattern.
uint64_t cns_rank_host(uint64_t a);

// Sorted list of all L-bit patterns with N bits set (Gosper's next-combination).
void enumerate_combinations(int L, int N, std::vector<uint64_t> &out);

// ------------------------------------------------------------------- trie

struct TriePlan {
    int M, R, H;                   // H = number of levels (chunks)
    int width[kMaxChunks];
    int shift[kMaxChunks];
    std::vector<int64_t> level_off; // H + 1 entries: start of each level
    int64_t size = 0;              // elements without padding
};

// Builds the breadth-first packed trie into t (uint64 entries, size + 2^R
// padding).  msb_first = 0: the paper's order (Fig. trielookup), the least
// significant chunk (width M mod R, or R) dispatched first; 1: the most
// significant chunk first (the same width at the top), so that members close
// in value share their walk down to the last levels.  Returns GBR_OK or
// GBR_EINVAL (message set).
int trie_build(const uint64_t *sorted, int64_t n, int M, int R, TriePlan *plan, std::vector<uint64_t> *t,
               int msb_first = 0);

}  // namespace gbr

// ----------------------------------------------------------------- handles

struct gbr_comb {
    gbr::StagDesc desc;
    gbr::DevBuf table;      // entries (uint32 or uint64)
    gbr::DevBuf binom;      // 65 x 65 uint64 binomials (unranking)
    uint64_t dim;
};

struct gbr_trie {
    int M, R, H;
    int msb_first;           // dispatch order of the chunks (trie_build)
    int width[gbr::kMaxChunks];
    int shift[gbr::kMaxChunks];
    int64_t n_members, size, padded;
    int wide;
    int smem_levels;         // number of leading levels copied to shared memory
    int64_t smem_entries;    // entries in those levels
    int64_t hot_entries;     // leading levels read with the L2 evict_last policy
    gbr::DevBuf t;
    gbr::DevBuf members;
};
