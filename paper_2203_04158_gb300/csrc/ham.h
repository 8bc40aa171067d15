// Hamiltonian handle: per-spin sectors, their ranking tables and hop lists.
#pragma once

#include "gbr_common.h"

namespace gbr {

constexpr int kMaxL = 32;
constexpr int kMaxUClasses = 8;

// One spin species: all L-bit patterns with N bits set, in increasing order.
struct SpinSector {
    int L = 0, N = 0;
    int64_t D = 0;
    StagDesc desc{};          // staggered tables (Fig. fastrank) for C^L_N, 8-bit chunks
    DevBuf stag;              // uint32 entries (per-spin dimensions stay below 2^32)
    StagDesc desc4{};         // the same with 4-bit chunks (more, smaller lookups)
    DevBuf stag4;
    DevBuf states;            // D uint32 patterns (unrank list, Sec. II)
    DevBuf diag;              // D doubles: sum_p h_pp n_p
    int hmax = 0;             // largest number of valid hops of one state
    int64_t hops = 0;         // total valid hops over all states
    DevBuf hop_cnt;           // D uint16: valid hops of each state (zero until the first ranking pass)
    int lists_ready = 0;      // 1 once a ranking pass has written the hop lists
    DevBuf hop_tgt;           // hmax x D uint32 (k-major): target rank | sign << 31
    DevBuf hop_bond;          // hmax x D uint16: index into the bond table
};

// Device-side description of the one-body terms and ranking method, passed
// to kernels by value.
struct HamK {
    int L;
    int nbond;                 // directed bonds (p, q), p != q, h_pq != 0
    int uniform;               // 1: every bond has the same coefficient
    double hu;                 // that coefficient
    int rank_method;           // GBR_RANK_*
    int nucls;                 // U classes
    uint32_t umask[kMaxUClasses];
    double uval[kMaxUClasses];
    uint32_t nbr[kMaxL];       // nbr[p]: sites q with h_pq != 0, q != p
};

// Fused first update of a Lanczos step on the unnormalised vectors
// u_j = g_j v_j (g_0 = 1, g_j = beta_j), done in the epilogue of the spin-up
// pass: w = H u_k / g_k - (beta_k / g_{k-1}) u_{k-1} (k read from device
// memory) and per-CTA partial sums of <w, u_k> (part may be NULL).  The two
// factors are precomputed: scal[4k] = 1/g_k, scal[4k+1] = beta_k / g_{k-1}
// (0 at k = 0).  With xt_next set (a second run of the recurrence, alpha_k
// already stored in scal[4k+2] = alpha_k / g_k) the epilogue also finishes
// the step: w - (alpha_k / g_k) u_k = u_{k+1} goes to y row-major and, through
// the CTA's Z tile, transposed to xt_next (X^T of the next H·v); no partials.
struct LzHook {
    const void *vprev;
    const double *scal;
    const int *kstate;
    double *part;
    void *xt_next = nullptr;
};

// The recurrence's two updates with their roundings spelled out, so that every
// kernel computing a step (the fused epilogue, the separate update kernels,
// the first and the second run) rounds it the same way: s * w - b * p with
// s * w rounded first, and w - a * x with one rounding.  Left to itself the
// compiler may contract s * w - b * p either way round.
__device__ __forceinline__ float lz_rec(float s, float w, float b, float p) { return __fmaf_rn(-b, p, __fmul_rn(s, w)); }
__device__ __forceinline__ double lz_rec(double s, double w, double b, double p) {
    return __fma_rn(-b, p, __dmul_rn(s, w));
}
__device__ __forceinline__ float lz_fnma(float a, float x, float w) { return __fmaf_rn(-a, x, w); }
__device__ __forceinline__ double lz_fnma(double a, double x, double w) { return __fma_rn(-a, x, w); }

// Device work buffers of a Lanczos solve, kept between calls and grown when
// needed (one set per operator handle).
struct LzWork {
    DevBuf state, alpha, beta, scal, part, coef, tri, svec, work, ritz;
    DevBuf buf[3], basis, x, hx;
};

}  // namespace gbr

struct gbr_ham {
    int L, Nup, Ndn;
    int64_t D;
    int64_t elements;
    int rank_method;
    int path;                  // GBR_HV_*
    std::vector<double> h, U;
    gbr::HamK k;
    gbr::SpinSector up, dn;
    gbr::DevBuf bonds;         // nbond x {p, q} uint8 pairs (as uint16), bond order
    gbr::DevBuf bond_coef64;   // nbond doubles
    gbr::DevBuf bond_coef32;   // nbond floats
    gbr::DevBuf hcoef64;       // L x L doubles (fused path lookups)
    gbr::DevBuf binom;         // (L+1) x (L+1) uint32 binomials (CNS ranking)
    // tuned launch shape (0 = default): rows per CTA of the gather passes
    int tune_up_rows[2] = {0, 0};
    int tune_dn_rows[2] = {0, 0};
    int tune_lz_rows[2] = {0, 0};   // the spin-up pass with the fused Lanczos update
    // windowed gathers (own rows staged in shared memory, Z written row-major):
    // win_dn < 0 = off (the untuned default), else on; the rows per CTA of the
    // spin-down, spin-up and fused-update passes (32 or 64; 0 = 64)
    int win_dn[2] = {-1, -1}, win_up[2] = {0, 0}, win_lz[2] = {0, 0};
    // chunk width R of the per-spin staggered tables (8 or 4) and threads per
    // state of the fused per-element kernel (1, 2 or 4)
    int rank_R[2] = {8, 8}, fused_tps[2] = {1, 1};
    // threads per CTA of the plain gather passes (spin-down, spin-up, fused
    // update): 128, or 64 for column chunks half as wide
    int gather_nt[3][2] = {{128, 128}, {128, 128}, {128, 128}};
    // scratch of the factored path (X^T and Z^T), grown on first use; one
    // H·v at a time per handle
    gbr::DevBuf ws_xt, ws_zt;
    // Lanczos work buffers
    gbr::LzWork lzw;
};

namespace gbr {
// ev (optional): 5 events recorded at the stage boundaries (hop lists,
// transpose, spin-down gather, spin-up gather with diagonal and combine);
// the fused path records the first four before its single kernel.
int hv_launch(const gbr_ham *H, const void *x, void *y, int fp, cudaStream_t st, cudaEvent_t *ev = nullptr);
int hv_stage(const gbr_ham *H, const void *x, void *y, int fp, int stage, cudaStream_t st);
// factored path with the two scratch vectors (dim elements each) supplied
int hv_factored_with_scratch(const gbr_ham *H, const void *x, void *y, int fp, cudaStream_t st, void *xt, void *zt);
// one-body bonds in (p, q) order, neighbour masks, U classes (shared by the
// sector and the set Hamiltonians); pairs gets (p, q) per bond, bidx the bond
// index of every (p, q)
int build_hamk(int L, const double *h, const double *U, int rank_method, HamK *k, std::vector<uint16_t> *pairs,
               std::vector<uint16_t> *bidx);
// true if gbr_hv runs the factored path on this handle
bool hv_is_factored(const gbr_ham *H);
// factored H·v with the fused Lanczos epilogue; *nparts receives the number
// of partial sums written (the grid of the spin-up pass)
// xt_ready: X^T is already in the handle's scratch (written by the previous
// step's update), so the transpose is skipped.  With hook.xt_next set,
// *updated tells whether the spin-up pass finished the step (u_{k+1} in y,
// its transpose in xt_next); when it could not (windowed passes, or a launch
// shape without full 16-byte vectors) y holds w and the caller updates.
int hv_launch_lz(const gbr_ham *H, const void *x, void *y, int fp, cudaStream_t st, cudaEvent_t *ev, const LzHook &hook,
                 int *nparts, bool xt_ready = false, bool *updated = nullptr);
// the handle's X^T scratch for precision fp (allocated if needed; NULL on failure)
void *hv_xt_scratch(const gbr_ham *H, int fp);
// upper bound of the partial sums hv_launch_lz writes for precision fp
int64_t hv_lz_parts(const gbr_ham *H, int fp);

// The operator of a Lanczos solve: the sector Hamiltonian (whose factored
// H·v carries the fused first update of each step), or any other operator
// given as y = A x in precision fp (32 or 64) on a stream.
struct LzOp {
    const gbr_ham *ham;
    const void *obj;
    int (*apply)(const void *obj, const void *x, void *y, int fp, cudaStream_t st);
    int64_t n;
    LzWork *work;
};
// The Lanczos solve of gbr_lanczos on any operator (argument checks included).
int lanczos_solve(const LzOp &op, const gbr_lanczos_opts *o, const double *d_v0, gbr_lanczos_result *res,
                  double *h_alpha, double *h_beta, double *h_ritz, void *stream);
}
