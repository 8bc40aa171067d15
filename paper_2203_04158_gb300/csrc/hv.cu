// On-the-fly H·v for Hubbard / impurity Hamiltonians in a (N_up, N_dn) sector
// (Wallerberger & Held, Sec. II: Eq. Talpha applied to every basis state,
// Eq. mvblock on one block; ranking by Fig. fastrank or Fig. algr; the spin
// factorisation of Eq. rankupdown).
//
// With the spin-down bits below the spin-up bits, a same-spin hop c^dag_p c_q
// changes only that spin's pattern, and its fermionic sign counts only that
// spin's occupied sites strictly between p and q (Eq. Talpha with
// s = the bits between p and q).  Writing x as a D_up x D_dn matrix X
// (index r_up * D_dn + r_dn):
//     Y = Dg o X + H_up X + X H_dn^T        (H_dn symmetric)
// Two implementations:
//   * fused: one thread per element does unrank, diagonal, every hop with
//     its sign and an on-the-fly rank, and the gather -- the method exactly as
//     the paper states it; used for small sectors;
//   * factored: per call, a ranking kernel walks every per-spin state once
//     (unrank, hop, sign by popcount, staggered rank) and writes its hop
//     list; two gather passes then apply H_up (row gathers of X, coalesced
//     along r_dn, column-chunked so the gathered columns stay in L2) and
//     H_dn plus the diagonal (X rows staged in shared memory).  Ranking work
//     drops from D * hops to (D_up + D_dn) * hops.
// Both are deterministic: each y element has one owner and a fixed order.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ham.h"
#include "dot.cuh"

namespace gbr {

// Per-spin ranking constants: chunks of R = 8 bits (at most 4 for L <= 32)
// or R = 4 bits (at most 8).
constexpr int kSpinChunks = 8;
struct SpinK {
    int L, N, Q;
    int shift[kSpinChunks], width[kSpinChunks], lo[kSpinChunks], hi[kSpinChunks], off[kSpinChunks];
    int64_t D;
    int tab_entries;
};

static SpinK spin_k(const SpinSector &s, int R = 8) {
    const StagDesc &d = R == 4 ? s.desc4 : s.desc;
    SpinK k;
    memset(&k, 0, sizeof(k));
    k.L = s.L; k.N = s.N; k.Q = d.Q; k.D = s.D;
    for (int q = 0; q < d.Q && q < kSpinChunks; ++q) {
        k.shift[q] = d.shift[q];
        k.width[q] = d.width[q];
        k.lo[q] = d.lo[q];
        k.hi[q] = d.hi[q];
        k.off[q] = (int)d.off[q];
    }
    k.tab_entries = (int)d.entries;
    return k;
}

static const uint32_t *spin_tab(const SpinSector &s, int R) { return (R == 4 ? s.stag4 : s.stag).as<uint32_t>(); }

// Fig. fastrank on a per-spin pattern (tables in shared memory).
__device__ __forceinline__ uint32_t spin_rank_stag(const SpinK &s, const uint32_t *tab, uint32_t a) {
    uint32_t acc = 0;
    int np = 0;
#pragma unroll
    for (int q = 0; q < kSpinChunks; ++q) {
        if (q < s.Q) {
            const uint32_t r = (a >> s.shift[q]) & ((1u << s.width[q]) - 1u);
            const int row = min(max(np, s.lo[q]), s.hi[q]) - s.lo[q];
            acc += tab[s.off[q] + (row << s.width[q]) + (int)r];
            np += __popc(r);
        }
    }
    return acc;
}

// Fig. algr: for the k-th set bit (from the least significant one, found by
// count-trailing-zeros) at position c add C(c, k).  binom is (L+1) x (L+1).
__device__ __forceinline__ uint32_t spin_rank_cns(int L, const uint32_t *binom, uint32_t a) {
    uint32_t i = 0;
    int k = 1;
    while (a) {
        const int c = __ffs(a) - 1;
        a &= a - 1u;
        i += binom[c * (L + 1) + k];
        ++k;
    }
    return i;
}

__device__ __forceinline__ uint32_t spin_rank(const SpinK &s, int method, const uint32_t *tab, const uint32_t *binom,
                                              uint32_t a) {
    return method == GBR_RANK_CNS ? spin_rank_cns(s.L, binom, a) : spin_rank_stag(s, tab, a);
}

// bits strictly between p and q
__device__ __forceinline__ uint32_t between_mask(int p, int q) {
    const int lo = min(p, q), hi = max(p, q);
    const uint32_t below_hi = (hi >= 32) ? 0xFFFFFFFFu : ((1u << hi) - 1u);
    const uint32_t upto_lo = (lo + 1 >= 32) ? 0xFFFFFFFFu : ((1u << (lo + 1)) - 1u);
    return below_hi & ~upto_lo;
}

// Loads the per-spin ranking table (staggered or binomial) into shared memory.
__device__ __forceinline__ void stage_u32(uint32_t *s, const uint32_t *__restrict__ g, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) s[i] = __ldg(g + i);
}

// ---------------------------------------------------------------- hop lists
//
// One thread per per-spin state r: unrank (list), then for every occupied
// site p (ascending) and every empty site q connected to it (ascending):
// target = rank(a ^ (2^p | 2^q)), sign = parity of the occupied sites
// strictly between p and q (Eq. Talpha, gather form Eq. Talpha2).
__global__ void k_hop_lists(const SpinK s, const HamK hk, const uint32_t *__restrict__ states,
                            const uint32_t *__restrict__ gtab, const uint32_t *__restrict__ gbinom,
                            const uint16_t *__restrict__ gbond_index, uint16_t *__restrict__ cnt,
                            uint32_t *__restrict__ tgt, uint16_t *__restrict__ bond, int hmax) {
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t *tab = sm;
    const int nb = (hk.L + 1) * (hk.L + 1);
    uint32_t *binom = sm + s.tab_entries;
    uint16_t *bidx = reinterpret_cast<uint16_t *>(binom + nb);
    stage_u32(tab, gtab, s.tab_entries);
    stage_u32(binom, gbinom, nb);
    for (int i = threadIdx.x; i < hk.L * hk.L; i += blockDim.x) bidx[i] = gbond_index[i];
    __syncthreads();
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s.D; r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = states[r];
        int k = 0;
        uint32_t occ = a;
        while (occ) {
            const int p = __ffs(occ) - 1;
            occ &= occ - 1u;
            uint32_t emp = hk.nbr[p] & ~a;
            while (emp) {
                const int q = __ffs(emp) - 1;
                emp &= emp - 1u;
                const uint32_t b = a ^ ((1u << p) | (1u << q));
                const uint32_t t = spin_rank(s, hk.rank_method, tab, binom, b);
                const uint32_t sg = (uint32_t)(__popc(a & between_mask(p, q)) & 1);
                if (k < hmax) {
                    tgt[(int64_t)k * s.D + r] = t | (sg << 31);
                    bond[(int64_t)k * s.D + r] = bidx[p * hk.L + q];
                }
                ++k;
            }
        }
        cnt[r] = (uint16_t)min(k, hmax);
    }
}

template <typename T> struct Vec;
template <> struct Vec<float> { typedef float4 v4; typedef float2 v2; };
template <> struct Vec<double> { typedef double2 v2; typedef double2 v4; };

__device__ __forceinline__ void unpack16(const float4 &p, float *o) { o[0] = p.x; o[1] = p.y; o[2] = p.z; o[3] = p.w; }
__device__ __forceinline__ void unpack16(const double2 &p, double *o) { o[0] = p.x; o[1] = p.y; }
__device__ __forceinline__ float4 pack16(const float *o) { return make_float4(o[0], o[1], o[2], o[3]); }
__device__ __forceinline__ double2 pack16(const double *o) { return make_double2(o[0], o[1]); }

template <typename T>
__device__ __forceinline__ T diag_value(const HamK &hk, const T *dup, const T *ddn, const T *uval, int64_t ru,
                                        int64_t rd, uint32_t au, uint32_t ad) {
    T d = dup[ru] + ddn[rd];
    const uint32_t both = au & ad;
#pragma unroll
    for (int c = 0; c < kMaxUClasses; ++c) {
        if (c >= hk.nucls) break;
        d += uval[c] * (T)__popc(both & hk.umask[c]);
    }
    return d;
}

// --------------------------------------------------------------- fused path
//
// One group of TPS threads per element i = r_up * D_dn + r_dn: the whole of
// Eq. Talpha for every term, with the target ranked on the fly.  With
// TPS > 1 the occupied sites of both spins are dealt round-robin to the
// group's threads (site j of the list of occupied sites, up spin first, goes
// to thread j mod TPS), whose partial sums meet in a fixed butterfly; the
// diagonal term is the first thread's.
template <typename T, int TPS>
__global__ void __launch_bounds__(256) k_hv_fused(const SpinK su, const SpinK sd, const HamK hk,
                                                  const uint32_t *__restrict__ st_up, const uint32_t *__restrict__ st_dn,
                                                  const uint32_t *__restrict__ tab_up, const uint32_t *__restrict__ tab_dn,
                                                  const uint32_t *__restrict__ gbinom, const T *__restrict__ hcoef,
                                                  const T *__restrict__ dup, const T *__restrict__ ddn,
                                                  const T *__restrict__ uval_g, const T *__restrict__ x,
                                                  T *__restrict__ y) {
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t *tu = sm;
    uint32_t *td = tu + su.tab_entries;
    const int nb = (hk.L + 1) * (hk.L + 1);
    uint32_t *binom = td + sd.tab_entries;
    T *hc = reinterpret_cast<T *>(binom + nb + (nb & 1));   // 8-byte aligned
    stage_u32(tu, tab_up, su.tab_entries);
    stage_u32(td, tab_dn, sd.tab_entries);
    stage_u32(binom, gbinom, nb);
    for (int i = threadIdx.x; i < hk.L * hk.L; i += blockDim.x) hc[i] = hcoef[i];
    T uval[kMaxUClasses];
#pragma unroll
    for (int c = 0; c < kMaxUClasses; ++c) uval[c] = c < hk.nucls ? uval_g[c] : T(0);
    __syncthreads();
    const int g = (int)(threadIdx.x % TPS);
    const int lane = threadIdx.x & 31;
    const unsigned gmask = TPS == 32 ? 0xFFFFFFFFu : (((1u << TPS) - 1u) << (lane & ~(TPS - 1)));
    const int64_t D = su.D * sd.D;
    const int64_t first = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / TPS;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x / TPS;
    for (int64_t i = first; i < D; i += stride) {
        const int64_t ru = i / sd.D, rd = i - ru * sd.D;
        const uint32_t au = st_up[ru], ad = st_dn[rd];
        T acc = g == 0 ? diag_value<T>(hk, dup, ddn, uval, ru, rd, au, ad) * x[i] : T(0);
        int j = 0;   // index of the occupied site in the list (up spin, then down)
        // spin up: changes r_up
        uint32_t occ = au;
        while (occ) {
            const int p = __ffs(occ) - 1;
            occ &= occ - 1u;
            if ((j++ % TPS) != g) continue;
            uint32_t emp = hk.nbr[p] & ~au;
            while (emp) {
                const int q = __ffs(emp) - 1;
                emp &= emp - 1u;
                const uint32_t t = spin_rank(su, hk.rank_method, tu, binom, au ^ ((1u << p) | (1u << q)));
                const T c = hc[p * hk.L + q];
                const T v = x[(int64_t)t * sd.D + rd];
                acc += (__popc(au & between_mask(p, q)) & 1) ? -c * v : c * v;
            }
        }
        // spin down: changes r_dn
        occ = ad;
        while (occ) {
            const int p = __ffs(occ) - 1;
            occ &= occ - 1u;
            if ((j++ % TPS) != g) continue;
            uint32_t emp = hk.nbr[p] & ~ad;
            while (emp) {
                const int q = __ffs(emp) - 1;
                emp &= emp - 1u;
                const uint32_t t = spin_rank(sd, hk.rank_method, td, binom, ad ^ ((1u << p) | (1u << q)));
                const T c = hc[p * hk.L + q];
                const T v = x[ru * sd.D + (int64_t)t];
                acc += (__popc(ad & between_mask(p, q)) & 1) ? -c * v : c * v;
            }
        }
#pragma unroll
        for (int o = TPS / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(gmask, acc, o);
        if (g == 0) y[i] = acc;
    }
}

// ------------------------------------------------------------ factored path
//
// Y = H_up X + Dg o X + (H_dn X^T)^T.  Both off-diagonal products are row
// gathers of the same shape, Z[r, c] = sum_k coef_k(r) W[t_k(r), c]: for
// H_up, W = X; for H_dn, W = X^T (an explicit transpose), whose result Z^T
// is added back in the epilogue of the spin-up pass.  A CTA owns TR rows and
// 128*VEC columns; its rows' hop lists are staged in shared memory, each
// thread streams VEC consecutive columns of every gathered row (coalesced),
// and consecutive CTAs share a column chunk so the gathered rows of that
// chunk stay in L2.

template <typename T, int TILE>
__global__ void __launch_bounds__(TILE * 4) k_transpose(const T *__restrict__ in, T *__restrict__ out, int64_t rows,
                                                        int64_t cols) {
    __shared__ T tile[TILE][TILE + 1];
    const int64_t c0 = (int64_t)blockIdx.x * TILE, r0 = (int64_t)blockIdx.y * TILE;
    for (int i = threadIdx.y; i < TILE; i += blockDim.y) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[i][threadIdx.x] = __ldcs(in + r * cols + c);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < TILE; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[c * rows + r] = tile[threadIdx.x][i];
    }
}

// The same transpose with 16-byte packs on both sides: a 64 x 64 tile is
// read as row packs and written as packs of V consecutive elements of one
// output row (V = 4 FP32, 2 FP64).  Needs cols and rows multiples of V and
// 16-byte aligned vectors; partial edge tiles fall back to single elements.
template <typename T>
__global__ void __launch_bounds__(256) k_transpose16(const T *__restrict__ in, T *__restrict__ out, int64_t rows,
                                                     int64_t cols) {
    constexpr int TILE = 64, V = 16 / (int)sizeof(T), RP = TILE / V, PAD = 1;
    typedef typename Vec<T>::v4 P16;
    __shared__ T tile[TILE][TILE + PAD];
    const int64_t c0 = (int64_t)blockIdx.x * TILE, r0 = (int64_t)blockIdx.y * TILE;
    const bool full = r0 + TILE <= rows && c0 + TILE <= cols;
    for (int idx = threadIdx.x; idx < TILE * RP; idx += blockDim.x) {
        const int i = idx / RP, j = idx % RP;
        const int64_t r = r0 + i, c = c0 + (int64_t)j * V;
        T o[V];
        if (full) {
            unpack16(__ldcs(reinterpret_cast<const P16 *>(in + r * cols + c)), o);
        } else {
#pragma unroll
            for (int e = 0; e < V; ++e) o[e] = (r < rows && c + e < cols) ? __ldcs(in + r * cols + c + e) : T(0);
        }
#pragma unroll
        for (int e = 0; e < V; ++e) tile[i][j * V + e] = o[e];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < TILE * RP; idx += blockDim.x) {
        const int c = idx / RP, j = idx % RP;
        T o[V];
#pragma unroll
        for (int e = 0; e < V; ++e) o[e] = tile[j * V + e][c];
        const int64_t oc = c0 + c, orow = r0 + (int64_t)j * V;
        if (full) {
            *reinterpret_cast<P16 *>(out + oc * rows + orow) = pack16(o);
        } else if (oc < cols) {
#pragma unroll
            for (int e = 0; e < V; ++e)
                if (orow + e < rows) out[oc * rows + orow + e] = o[e];
        }
    }
}

// Asynchronous copies of B = 4, 8, 16 (or twice 16) bytes from global to shared memory
// (cp.async: no registers are held while they are in flight).  The issuing
// thread waits for its own copies with cp_async_wait_all; other threads see
// them after a barrier that follows that wait.
template <int B>
__device__ __forceinline__ void cp_async(void *dst, const void *src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    if constexpr (B == 32) {
        cp_async<16>(dst, src);
        cp_async<16>((char *)dst + 16, (const char *)src + 16);
    } else if constexpr (B == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(B) : "memory");
}
// the same with an L2 cache policy (data read once: evict_first)
template <int B>
__device__ __forceinline__ void cp_async_hint(void *dst, const void *src, uint64_t pol) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    if constexpr (B == 32) {
        cp_async_hint<16>(dst, src, pol);
        cp_async_hint<16>((char *)dst + 16, (const char *)src + 16, pol);
    } else if constexpr (B == 16)
        asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, 16, %2;" ::"r"(d), "l"(src), "l"(pol)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], %2, %2, %3;" ::"r"(d), "l"(src), "n"(B),
                     "l"(pol)
                     : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Row stride padding (elements) of the staged Z tile.  The tile is written
// column by column, TR rows of one column from consecutive threads, so a warp
// covers 32 / TR columns; a padding of 32 / TR FP32 elements puts all 32 in
// different banks for TR = 4 and 8.  The rows stay 16-byte aligned for the
// vector reads, so TR = 16 keeps 4 (two-way conflicts); FP64 keeps 16 bytes.
__host__ __device__ constexpr int ztile_pad(int elem_bytes, int TR) {
    return (elem_bytes == 4 && TR == 4) ? 8 : 16 / elem_bytes;
}

struct CombineArgs {
    const uint32_t *st_up, *st_dn;   // per-spin patterns (row and column states)
    const void *dup, *ddn, *uval;     // per-spin diagonals, U class values (precision T)
    const void *zt;                   // Z^T = H_dn X^T (D_dn x D_up), or Z (D_up x D_dn) when zrow
    HamK hk;
    LzHook lz;                        // fused first Lanczos update (MODE 2)
    int zrow;                         // 1: the spin-down pass wrote Z row-major (window kernels)
};

// MODE 0: Z = H_lists W.  MODE 1: y = H_up X + Dg o X + Z (combine).  MODE 2:
// as 1, then the first update of a Lanczos step on unnormalised vectors
// u_j = g_j v_j (g_0 = 1, g_j = beta_j) in the same epilogue,
// w = y / g_k - (beta_k / g_{k-1}) u_{k-1} (k > 0; x = u_k) and the block's
// partial <w, x>.  MODE 3: as 2 on a second run of the recurrence (alpha_k
// known, no partials), then u_{k+1} = w - (alpha_k / g_k) x to y and, through
// the Z tile (each thread overwrites the values it read), transposed to
// ca.lz.xt_next once the CTA's rows are done.
// The FP32 passes are held to 1280 threads per SM (48 registers): left free
// the compiler takes up to 56-60 registers and the occupancy drops; at 12 or
// 16 CTAs of 128 threads the combine pass spills.  Measured on the 4x4
// sector: combine 1.16 ms (10 CTAs) against 1.21 ms (free) and 1.25 ms (16).
// NT threads per CTA (128, or 64 for column chunks half as wide: the
// gathered rows of a chunk then take half the L2).
template <typename T, int VEC, int MODE, int TR, int NT>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 ? 1280 / NT : 1)) k_gather(const int64_t Drows, const int64_t Dcols, const int hmax,
                                                const int64_t nrb, const uint16_t *__restrict__ cnt,
                                                const uint32_t *__restrict__ tgt, const uint16_t *__restrict__ bond,
                                                const T *__restrict__ bcoef, const int uniform, const T hu,
                                                const T *__restrict__ x, T *__restrict__ y, const CombineArgs ca) {
    constexpr bool COMBINE = MODE >= 1;
    constexpr bool LZ = MODE >= 2;
    constexpr bool UPD = MODE == 3;
    constexpr int VB = VEC * (int)sizeof(T);   // bytes of one thread's slice of a row
    constexpr int ZS = NT * VEC + ztile_pad((int)sizeof(T), TR);
    // hop-list row stride, a multiple of 4 so that four targets (and four
    // coefficients) are read with one 16-byte broadcast load
    const int hs = (hmax + 3) & ~3;
    extern __shared__ __align__(128) unsigned char smr[];
    uint32_t *st = reinterpret_cast<uint32_t *>(smr);
    T *sc = reinterpret_cast<T *>(smr + (size_t)TR * hs * 4);
    // combine epilogue: the block Z[r0..r0+TR, chunk] = (Z^T)[chunk, r0..r0+TR]
    // (TR rows of ZS), then one slot each for the current row's own x slice
    // (diagonal term) and its u_{k-1} slice (Lanczos update)
    T *zs = reinterpret_cast<T *>(smr + (size_t)TR * hs * (4 + sizeof(T)));
    T *xs = zs + (size_t)TR * ZS;
    T *vs = xs + NT * VEC;
    __shared__ int scnt[TR];
    // per-row spin-up pattern and diagonal, U class values (combine), in
    // shared memory to keep registers for occupancy
    __shared__ uint32_t sau[TR];
    __shared__ T sdu[TR];
    __shared__ T suv[kMaxUClasses];
    const int64_t rb = blockIdx.x % nrb, cc = blockIdx.x / nrb;
    const int64_t r0 = rb * TR;
    const int nrow = (int)((Drows - r0) < (int64_t)TR ? (Drows - r0) : (int64_t)TR);
    const int64_t cbase = cc * (int64_t)(NT * VEC);
    // The prologue issues every load that does not wait on another before the
    // first barrier: the Z tile goes to shared memory by asynchronous copies
    // (4 or 8 bytes each, waited for before the second barrier), so it is in
    // flight while the hop lists are staged.
    if (COMBINE && !ca.zrow) {
        const T *zt = (const T *)ca.zt;
        const uint64_t pol = l2_evict_first();
        for (int e = threadIdx.x; e < NT * VEC * TR; e += blockDim.x) {
            const int col = e / TR, i = e % TR;
            const int64_t c = cbase + col;
            if (c < Dcols && i < nrow) cp_async_hint<(int)sizeof(T)>(zs + i * ZS + col, zt + c * Drows + r0 + i, pol);
            else zs[i * ZS + col] = T(0);
        }
    }
    const int64_t c0 = cbase + (int64_t)threadIdx.x * VEC;
    const bool active = c0 < Dcols;
    DotAcc<T> dacc;
    int klz = 0;
    T slz = T(1), blz = T(0), alz = T(0);
    if (LZ) {
        klz = *ca.lz.kstate;
        slz = (T)ca.lz.scal[4 * klz];
        blz = (T)ca.lz.scal[4 * klz + 1];
        if (UPD) alz = (T)ca.lz.scal[4 * klz + 2];
    }
    // combine epilogue: column states and diagonals of this thread's columns
    uint32_t ad[VEC];
    T dd[VEC];
    if (COMBINE && active) {
        const T *ddn = (const T *)ca.ddn;
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            ad[v] = ca.st_dn[c0 + v];
            dd[v] = ddn[c0 + v];
        }
    }
    for (int i = threadIdx.x; i < TR; i += blockDim.x) {
        scnt[i] = i < nrow ? (int)cnt[r0 + i] : 0;
        if (COMBINE && i < nrow) {
            sau[i] = ca.st_up[r0 + i];
            sdu[i] = ((const T *)ca.dup)[r0 + i];
        }
    }
    if (COMBINE && threadIdx.x < kMaxUClasses)
        suv[threadIdx.x] = threadIdx.x < ca.hk.nucls ? ((const T *)ca.uval)[threadIdx.x] : T(0);
    __syncthreads();
    for (int e = threadIdx.x; e < TR * hmax; e += blockDim.x) {
        const int i = e % TR, k = e / TR;
        if (k < scnt[i]) {
            const int64_t g = (int64_t)k * Drows + r0 + i;
            const uint32_t w = tgt[g];
            const T c = uniform ? hu : bcoef[bond[g]];
            st[i * hs + k] = w & 0x7FFFFFFFu;
            sc[i * hs + k] = (w >> 31) ? -c : c;
        }
    }
    if (COMBINE && !ca.zrow) cp_async_wait_all();
    __syncthreads();
    const uint64_t pol_first = LZ ? l2_evict_first() : 0;
    for (int i = 0; i < TR && active; ++i) {
        const int64_t r = r0 + i;
        if (r >= Drows) break;
        // combine: the row's own x slice and u_{k-1} slice travel to this
        // thread's slots while the row gathers (each thread reads back only
        // what it copied, after waiting for its own copies)
        if (COMBINE) {
            cp_async<VB>(xs + threadIdx.x * VEC, x + r * Dcols + c0);
            if (LZ && klz > 0) cp_async_hint<VB>(vs + threadIdx.x * VEC, (const T *)ca.lz.vprev + r * Dcols + c0, pol_first);
        }
        const int n = scnt[i];
        const uint32_t *ti = st + i * hs;
        const T *ci = sc + i * hs;
        T acc[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] = 0;
        if (VEC == 4 && sizeof(T) == 4) {
            // the gathered rows move through the L1 data pipe at 4 wavefronts
            // a row; the hop list costs half a wavefront a row, read four at
            // a time (summed in hop order, as one at a time)
            float4 a4 = make_float4(0.f, 0.f, 0.f, 0.f);
            const float *cf = reinterpret_cast<const float *>(ci);
            int k = 0;
#pragma unroll 2
            for (; k + 4 <= n; k += 4) {
                const uint4 t4 = *reinterpret_cast<const uint4 *>(ti + k);
                const float4 c4 = *reinterpret_cast<const float4 *>(cf + k);
                const float4 v0 = __ldcg(reinterpret_cast<const float4 *>(x + (int64_t)t4.x * Dcols + c0));
                const float4 v1 = __ldcg(reinterpret_cast<const float4 *>(x + (int64_t)t4.y * Dcols + c0));
                const float4 v2 = __ldcg(reinterpret_cast<const float4 *>(x + (int64_t)t4.z * Dcols + c0));
                const float4 v3 = __ldcg(reinterpret_cast<const float4 *>(x + (int64_t)t4.w * Dcols + c0));
                a4.x += c4.x * v0.x; a4.y += c4.x * v0.y; a4.z += c4.x * v0.z; a4.w += c4.x * v0.w;
                a4.x += c4.y * v1.x; a4.y += c4.y * v1.y; a4.z += c4.y * v1.z; a4.w += c4.y * v1.w;
                a4.x += c4.z * v2.x; a4.y += c4.z * v2.y; a4.z += c4.z * v2.z; a4.w += c4.z * v2.w;
                a4.x += c4.w * v3.x; a4.y += c4.w * v3.y; a4.z += c4.w * v3.z; a4.w += c4.w * v3.w;
            }
            if (k < n) {
                // the last one to three hops as one batch of independent loads
                const bool h1 = k + 1 < n, h2 = k + 2 < n;
                const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 v0 = __ldcg(reinterpret_cast<const float4 *>(x + (int64_t)ti[k] * Dcols + c0));
                const float4 v1 = h1 ? __ldcg(reinterpret_cast<const float4 *>(x + (int64_t)ti[k + 1] * Dcols + c0)) : zero;
                const float4 v2 = h2 ? __ldcg(reinterpret_cast<const float4 *>(x + (int64_t)ti[k + 2] * Dcols + c0)) : zero;
                float c = cf[k];
                a4.x += c * v0.x; a4.y += c * v0.y; a4.z += c * v0.z; a4.w += c * v0.w;
                if (h1) {
                    c = cf[k + 1];
                    a4.x += c * v1.x; a4.y += c * v1.y; a4.z += c * v1.z; a4.w += c * v1.w;
                }
                if (h2) {
                    c = cf[k + 2];
                    a4.x += c * v2.x; a4.y += c * v2.y; a4.z += c * v2.z; a4.w += c * v2.w;
                }
            }
            acc[0] = a4.x; acc[1] = a4.y; acc[2] = a4.z; acc[3 % VEC] = a4.w;
        } else if (VEC == 2) {
            T a0 = 0, a1 = 0;
#pragma unroll 4
            for (int k = 0; k < n; ++k) {
                const typename Vec<T>::v2 v = __ldcg(reinterpret_cast<const typename Vec<T>::v2 *>(x + (int64_t)ti[k] * Dcols + c0));
                a0 += ci[k] * v.x; a1 += ci[k] * v.y;
            }
            acc[0] = a0; acc[1 % VEC] = a1;
        } else {
            T a0 = 0;
#pragma unroll 4
            for (int k = 0; k < n; ++k) a0 += ci[k] * __ldcg(x + (int64_t)ti[k] * Dcols + c0);
            acc[0] = a0;
        }
        if (COMBINE) {
            const uint32_t au = sau[i];
            const T du = sdu[i];
            cp_async_wait_all();
            T xo[VEC];
            if (VEC == 4 && sizeof(T) == 4) {
                const float4 o = *reinterpret_cast<const float4 *>(xs + threadIdx.x * VEC);
                xo[0] = o.x; xo[1 % VEC] = o.y; xo[2 % VEC] = o.z; xo[3 % VEC] = o.w;
            } else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) xo[v] = xs[threadIdx.x * VEC + v];
            }
            T zv[VEC];
            if (ca.zrow) {
                const T *zr = (const T *)ca.zt + r * Dcols + c0;
#pragma unroll
                for (int v = 0; v < VEC; ++v) zv[v] = __ldcs(zr + v);
            } else if (VEC == 4 && sizeof(T) == 4) {
                const float4 z4 = *reinterpret_cast<const float4 *>(zs + i * ZS + threadIdx.x * VEC);
                zv[0] = z4.x; zv[1 % VEC] = z4.y; zv[2 % VEC] = z4.z; zv[3 % VEC] = z4.w;
            } else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) zv[v] = zs[i * ZS + threadIdx.x * VEC + v];
            }
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const uint32_t both = au & ad[v];
                T dg = du + dd[v];
                // unrolled with a uniform exit, so no FP64 work is spent on
                // unused classes
#pragma unroll
                for (int u = 0; u < kMaxUClasses; ++u) {
                    if (u >= ca.hk.nucls) break;
                    dg += suv[u] * (T)__popc(both & ca.hk.umask[u]);
                }
                acc[v] += dg * xo[v] + zv[v];
            }
            if (LZ) {
                if (klz > 0) {
                    T vp[VEC];
                    if (VEC == 4 && sizeof(T) == 4) {
                        const float4 o = *reinterpret_cast<const float4 *>(vs + threadIdx.x * VEC);
                        vp[0] = o.x; vp[1 % VEC] = o.y; vp[2 % VEC] = o.z; vp[3 % VEC] = o.w;
                    } else {
#pragma unroll
                        for (int v = 0; v < VEC; ++v) vp[v] = vs[threadIdx.x * VEC + v];
                    }
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[v] = lz_rec(slz, acc[v], blz, vp[v]);
                }
                if (UPD) {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[v] = lz_fnma(alz, xo[v], acc[v]);
                    if (VEC == 4 && sizeof(T) == 4) {
                        *reinterpret_cast<float4 *>(zs + i * ZS + threadIdx.x * VEC) =
                            make_float4((float)acc[0], (float)acc[1 % VEC], (float)acc[2 % VEC], (float)acc[3 % VEC]);
                    } else {
#pragma unroll
                        for (int v = 0; v < VEC; ++v) zs[i * ZS + threadIdx.x * VEC + v] = acc[v];
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) dacc.add(acc[v], xo[v]);
                }
            }
        }
        if (VEC == 4 && sizeof(T) == 4) {
            __stcs(reinterpret_cast<float4 *>(y + r * Dcols + c0), make_float4((float)acc[0], (float)acc[1 % VEC], (float)acc[2 % VEC], (float)acc[3 % VEC]));
        } else if (VEC == 2) {
            typename Vec<T>::v2 o;
            o.x = acc[0]; o.y = acc[1 % VEC];
            __stcs(reinterpret_cast<typename Vec<T>::v2 *>(y + r * Dcols + c0), o);
        } else {
            y[r * Dcols + c0] = acc[0];
        }
    }
    if (UPD) {
        // u_{k+1} of the CTA's rows and columns, TR consecutive values per
        // column of the transpose (as the Z tile was read)
        __syncthreads();
        T *xt = (T *)ca.lz.xt_next;
        for (int e = threadIdx.x; e < NT * VEC * TR; e += blockDim.x) {
            const int col = e / TR, i = e % TR;
            const int64_t c = cbase + col;
            if (c < Dcols && i < nrow) __stcs(xt + c * Drows + r0 + i, zs[i * ZS + col]);
        }
    } else if (LZ && ca.lz.part) {
        const double r = block_sum(dacc.value());
        if (threadIdx.x == 0) ca.lz.part[blockIdx.x] = r;
    }
}

// ------------------------------------------------------- windowed gathers
//
// The same row gathers with the CTA's own rows staged in shared memory.  A
// CTA owns TR consecutive rows and one 512-byte column slice of the gather
// source (128 FP32 or 64 FP64 columns); those TR row slices are copied into
// shared memory with 1-D bulk copies (cp.async.bulk, completion counted on an
// mbarrier) while the CTA stages its hop lists.  A hop whose target row lies
// in the window is read from shared memory, every other hop from L2, so the
// L2-to-SM traffic falls by the share of hops that stay inside TR
// consecutive ranks (lexicographic order keeps hops on the low sites local:
// about 27 % of the 4x4 torus's hops and 40 % of the 18-site ring's at
// TR = 64).  The combine pass also takes the state's own x value (diagonal
// term) from the window.  The spin-down pass writes Z = (H_dn X^T)^T row-major
// through a shared-memory transpose of its output tile, so the spin-up pass
// reads Z with plain coalesced row loads.  8 warps; warp w handles the rows
// w, w + 8, ... of the tile, its 32 lanes 16 bytes each of the slice.

// bounded wait on an mbarrier phase: false if it did not complete within
// about a second (the caller reports GBR_ETIMEOUT through the status word)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    for (int it = 0; it < (1 << 24); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

// device status word: bit 0 = a bounded wait ran out (read and cleared by
// gbr_device_status)
__device__ int g_gbr_status = 0;

template <typename T> struct WinVec;
template <> struct WinVec<float> {
    typedef float4 V;
    __device__ static __forceinline__ void fma4(float *a, float c, const float4 &v) {
        a[0] += c * v.x; a[1] += c * v.y; a[2] += c * v.z; a[3] += c * v.w;
    }
    __device__ static __forceinline__ void get(float *o, const float4 &v) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
    __device__ static __forceinline__ float4 put(const float *o) { return make_float4(o[0], o[1], o[2], o[3]); }
    // four consecutive hop coefficients (16-byte aligned)
    __device__ static __forceinline__ void coef4(float *c, const float *p) { get(c, *reinterpret_cast<const float4 *>(p)); }
};
template <> struct WinVec<double> {
    typedef double2 V;
    __device__ static __forceinline__ void fma4(double *a, double c, const double2 &v) { a[0] += c * v.x; a[1] += c * v.y; }
    __device__ static __forceinline__ void get(double *o, const double2 &v) { o[0] = v.x; o[1] = v.y; }
    __device__ static __forceinline__ double2 put(const double *o) { return make_double2(o[0], o[1]); }
    __device__ static __forceinline__ void coef4(double *c, const double *p) {
        get(c, *reinterpret_cast<const double2 *>(p));
        get(c + 2, *reinterpret_cast<const double2 *>(p + 2));
    }
};

// bytes of the window region (also the transposed output tile of MODE 0,
// whose rows are padded by one element)
template <typename T, int TR>
__host__ __device__ constexpr size_t win_region_bytes() {
    return ((size_t)TR * (32 * (16 / sizeof(T)) + 1) * sizeof(T) + 15) & ~(size_t)15;
}

template <typename T, int MODE, int TR>
__global__ void __launch_bounds__(256, 2) k_gwin(const int64_t Drows, const int64_t Dcols, const int hmax,
                                                 const int64_t nrb, const uint16_t *__restrict__ cnt,
                                                 const uint32_t *__restrict__ tgt, const uint16_t *__restrict__ bond,
                                                 const T *__restrict__ bcoef, const int uniform, const T hu,
                                                 const T *__restrict__ x, T *__restrict__ y, const CombineArgs ca) {
    constexpr bool COMBINE = MODE >= 1;
    constexpr bool LZ = MODE == 2;
    constexpr int VEC = 16 / (int)sizeof(T);
    constexpr int WC = 32 * VEC;          // columns of the slice (512 bytes)
    constexpr int NW = 8;                 // warps
    constexpr int RPW = TR / NW;          // rows per warp
    typedef typename WinVec<T>::V V;
    // padded hop-list stride (multiple of 4: four targets per 16-byte load)
    const int hs = (hmax + 3) & ~3;
    extern __shared__ __align__(128) unsigned char smr[];
    T *win = reinterpret_cast<T *>(smr);
    uint32_t *st = reinterpret_cast<uint32_t *>(smr + win_region_bytes<T, TR>());
    T *sc = reinterpret_cast<T *>(smr + win_region_bytes<T, TR>() + (size_t)TR * hs * 4);
    __shared__ int scnt[TR];
    __shared__ T suv[kMaxUClasses];
    __shared__ __align__(8) uint64_t bar;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t rb = blockIdx.x % nrb, cc = blockIdx.x / nrb;
    const int64_t r0 = rb * TR, c0 = cc * WC;
    const int nrow = (int)((Drows - r0) < (int64_t)TR ? (Drows - r0) : (int64_t)TR);
    const int ncol = (int)((Dcols - c0) < (int64_t)WC ? (Dcols - c0) : (int64_t)WC);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // window: nrow slices of ncol * sizeof(T) bytes (a multiple of 16: the
    // launcher requires Dcols * sizeof(T) % 16 == 0 and 16-byte aligned x)
    if (warp == 0) {
        const uint32_t rowb = (uint32_t)ncol * (uint32_t)sizeof(T);
        const uint32_t ba = (uint32_t)__cvta_generic_to_shared(&bar);
        if (lane == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ba), "r"(rowb * (uint32_t)nrow)
                         : "memory");
        __syncwarp();
        for (int i = lane; i < nrow; i += 32) {
            const T *src = x + (r0 + i) * Dcols + c0;
            const uint32_t dst = (uint32_t)__cvta_generic_to_shared(win + (size_t)i * WC);
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                         "l"(src), "r"(rowb), "r"(ba)
                         : "memory");
        }
    }
    // hop lists of the tile's rows (coalesced along the rows), meanwhile
    for (int i = threadIdx.x; i < TR; i += blockDim.x) scnt[i] = (i < nrow) ? (int)cnt[r0 + i] : 0;
    if (COMBINE && threadIdx.x < kMaxUClasses)
        suv[threadIdx.x] = threadIdx.x < ca.hk.nucls ? ((const T *)ca.uval)[threadIdx.x] : T(0);
    __syncthreads();
    for (int e = threadIdx.x; e < TR * hmax; e += blockDim.x) {
        const int i = e % TR, k = e / TR;
        if (k < scnt[i]) {
            const int64_t g = (int64_t)k * Drows + r0 + i;
            const uint32_t w = tgt[g];
            const T c = uniform ? hu : bcoef[bond[g]];
            st[i * hs + k] = w & 0x7FFFFFFFu;
            sc[i * hs + k] = (w >> 31) ? -c : c;
        }
    }
    const int ok = mbar_wait_bounded(&bar, 0) ? 1 : 0;
    if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0) atomicOr(&g_gbr_status, 1);
        return;
    }
    const int cl = lane * VEC;                 // this lane's first column in the slice
    const bool active = cl < ncol;
    const T *xs = x + c0 + cl;
    DotAcc<T> dacc;
    int klz = 0;
    T slz = T(1), blz = T(0);
    if (LZ) {
        klz = *ca.lz.kstate;
        slz = (T)ca.lz.scal[4 * klz];
        blz = (T)ca.lz.scal[4 * klz + 1];
    }
    uint32_t ad[VEC];
    T dd[VEC];
    if (COMBINE && active) {
        const T *ddn = (const T *)ca.ddn;
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            ad[v] = ca.st_dn[c0 + cl + v];
            dd[v] = ddn[c0 + cl + v];
        }
    }
    T keep[MODE == 0 ? RPW : 1][VEC];
#pragma unroll
    for (int j = 0; j < RPW; ++j) {
        const int i = warp + j * NW;
        T acc[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] = T(0);
        if (i < nrow && active) {
            const int n = scnt[i];
            const uint32_t *ti = st + i * hs;
            const T *ci = sc + i * hs;
            // target row t: from the window if r0 <= t < r0 + nrow, else from L2
            auto row = [&](uint32_t t) -> const V * {
                const uint32_t tl = t - (uint32_t)r0;
                return tl < (uint32_t)nrow ? reinterpret_cast<const V *>(win + (size_t)tl * WC + cl)
                                           : reinterpret_cast<const V *>(xs + (int64_t)t * Dcols);
            };
            int k = 0;
#pragma unroll 2
            for (; k + 4 <= n; k += 4) {
                const uint4 t4 = *reinterpret_cast<const uint4 *>(ti + k);
                T c4[4];
                WinVec<T>::coef4(c4, ci + k);
                const V v0 = *row(t4.x), v1 = *row(t4.y), v2 = *row(t4.z), v3 = *row(t4.w);
                WinVec<T>::fma4(acc, c4[0], v0);
                WinVec<T>::fma4(acc, c4[1], v1);
                WinVec<T>::fma4(acc, c4[2], v2);
                WinVec<T>::fma4(acc, c4[3], v3);
            }
            for (; k < n; ++k) WinVec<T>::fma4(acc, ci[k], *row(ti[k]));
            if (COMBINE) {
                const int64_t r = r0 + i;
                const uint32_t au = ca.st_up[r];
                const T du = ((const T *)ca.dup)[r];
                T xo[VEC], zv[VEC];
                WinVec<T>::get(xo, *reinterpret_cast<const V *>(win + (size_t)i * WC + cl));
                WinVec<T>::get(zv, __ldcs(reinterpret_cast<const V *>((const T *)ca.zt + r * Dcols + c0 + cl)));
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    const uint32_t both = au & ad[v];
                    T dg = du + dd[v];
#pragma unroll
                    for (int u = 0; u < kMaxUClasses; ++u) {
                        if (u >= ca.hk.nucls) break;
                        dg += suv[u] * (T)__popc(both & ca.hk.umask[u]);
                    }
                    acc[v] += dg * xo[v] + zv[v];
                }
                if (LZ) {
                    if (klz > 0) {
                        T vp[VEC];
                        WinVec<T>::get(vp, __ldcs(reinterpret_cast<const V *>((const T *)ca.lz.vprev + r * Dcols + c0 + cl)));
#pragma unroll
                        for (int v = 0; v < VEC; ++v) acc[v] = lz_rec(slz, acc[v], blz, vp[v]);
                    }
#pragma unroll
                    for (int v = 0; v < VEC; ++v) dacc.add(acc[v], xo[v]);
                }
                __stcs(reinterpret_cast<V *>(y + r * Dcols + c0 + cl), WinVec<T>::put(acc));
            }
        }
        if (MODE == 0) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) keep[MODE == 0 ? j : 0][v] = acc[v];
        }
    }
    if (MODE == 0) {
        // transpose the TR x ncol output tile through shared memory (the
        // window is no longer read) and write Z[c0 + col][r0 + i] = tile[i][col]
        // as TR-element runs of consecutive ranks
        constexpr int TS = WC + 1;
        __syncthreads();
        if (active) {
#pragma unroll
            for (int j = 0; j < RPW; ++j) {
                const int i = warp + j * NW;
                if (i < nrow) {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) win[(size_t)i * TS + cl + v] = keep[j][v];
                }
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < TR * ncol; e += blockDim.x) {
            const int i = e % TR, col = e / TR;
            if (i < nrow) __stcs(y + (c0 + col) * Drows + r0 + i, win[(size_t)i * TS + col]);
        }
    }
    if (LZ && ca.lz.part) {
        const double r = block_sum(dacc.value());
        if (threadIdx.x == 0) ca.lz.part[blockIdx.x] = r;
    }
}

// ------------------------------------------------------------------ launch

struct HamDev {
    // precision-specific copies of the diagonal and coefficients
    const void *dup, *ddn, *uval, *bcoef, *hcoef;
};

template <typename T>
static int launch_hop_lists(const gbr_ham *H, const SpinSector &s, cudaStream_t st) {
    const int R = H->rank_R[sizeof(T) == 8 ? 1 : 0];
    const SpinK sk = spin_k(s, R);
    const int nb = (H->L + 1) * (H->L + 1);
    const size_t smem = (size_t)(sk.tab_entries + nb) * 4 + (size_t)H->L * H->L * 2 + 16;
    const int threads = 128;
    int64_t blocks = (s.D + threads - 1) / threads;
    blocks = std::min<int64_t>(blocks, (int64_t)sm_count() * 8);
    if (smem > 48 * 1024) GBR_CUDA_TRY(cudaFuncSetAttribute(k_hop_lists, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_hop_lists<<<(int)std::max<int64_t>(blocks, 1), threads, smem, st>>>(
        sk, H->k, s.states.as<uint32_t>(), spin_tab(s, R), H->binom.as<uint32_t>(),
        reinterpret_cast<const uint16_t *>(H->bonds.p) + 2 * H->k.nbond, s.hop_cnt.as<uint16_t>(),
        s.hop_tgt.as<uint32_t>(), s.hop_bond.as<uint16_t>(), s.hmax);
    GBR_LAUNCH_CHECK();
    const_cast<SpinSector &>(s).lists_ready = 1;
    count_launches(1);
    return GBR_OK;
}

template <typename T>
static int launch_fused(const gbr_ham *H, const T *x, T *y, cudaStream_t st, const HamDev &hd) {
    const int fpi = sizeof(T) == 8 ? 1 : 0;
    const int R = H->rank_R[fpi], tps = H->fused_tps[fpi];
    const SpinK su = spin_k(H->up, R), sd = spin_k(H->dn, R);
    const int nb = (H->L + 1) * (H->L + 1);
    const size_t smem = (size_t)(su.tab_entries + sd.tab_entries + nb + 1) * 4 + (size_t)H->L * H->L * sizeof(T) + 16;
    const int threads = 256;
    int64_t blocks = (H->D * tps + threads - 1) / threads;
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sm_count() * 8));
    auto kern = tps == 4 ? k_hv_fused<T, 4> : (tps == 2 ? k_hv_fused<T, 2> : k_hv_fused<T, 1>);
    if (smem > 48 * 1024) GBR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(int)blocks, threads, smem, st>>>(su, sd, H->k, H->up.states.as<uint32_t>(), H->dn.states.as<uint32_t>(),
                                             spin_tab(H->up, R), spin_tab(H->dn, R),
                                             H->binom.as<uint32_t>(), (const T *)hd.hcoef, (const T *)hd.dup,
                                             (const T *)hd.ddn, (const T *)hd.uval, x, y);
    GBR_LAUNCH_CHECK();
    count_launches(1);
    return GBR_OK;
}

// When N_up == N_dn both spin species share one sector and one set of hop
// lists (the hopping is spin independent).
static const SpinSector &dn_lists(const gbr_ham *H) { return H->Nup == H->Ndn ? H->up : H->dn; }

template <typename T>
static int stage_hop_lists(const gbr_ham *H, cudaStream_t st) {
    int rc = launch_hop_lists<T>(H, H->up, st);
    if (rc) return rc;
    if (H->Nup != H->Ndn) rc = launch_hop_lists<T>(H, H->dn, st);
    return rc;
}

// scratch of the factored path: X^T and Z^T, owned by the handle unless the
// caller supplies them (gbr_hv_static)
struct Scratch {
    void *xt, *zt;
};

static int ensure_ws(const gbr_ham *H, size_t bytes) {
    gbr_ham *h = const_cast<gbr_ham *>(H);
    if (h->ws_xt.bytes >= bytes && h->ws_zt.bytes >= bytes) return GBR_OK;
    int rc = h->ws_xt.alloc(bytes);
    if (!rc) rc = h->ws_zt.alloc(bytes);
    return rc;
}

// Vector width and rows per CTA of a gather pass (shared by the launch and
// the partial-sum sizing of the fused Lanczos epilogue).
template <typename T>
static void gather_shape(const gbr_ham *H, int64_t Drows, int64_t Dcols, bool aligned16, bool combine, bool lz,
                         int nt, int *vec_out, int *tr_out) {
    const int fpi = sizeof(T) == 8 ? 1 : 0;
    const int vmax = sizeof(T) == 4 ? 4 : 2;
    // widest vector whose column chunk (the rows one wave of CTAs gathers
    // from) stays within the cap: 128 MB for FP32, 64 MB for FP64 (measured
    // on the L=18 ring, 48,620 rows: FP32 20.7 ms with 100 MB chunks against
    // 24.5 ms with 50 MB and 37 ms with 25 MB; FP64 109 ms at 50 MB, 113 ms at 100 MB)
    const double cap = sizeof(T) == 4 ? 128e6 : 64e6;
    int vec = 1;
    for (int v = vmax; v >= 2; v /= 2)
        if (aligned16 && Dcols % v == 0 && (double)Drows * nt * v * sizeof(T) <= cap) { vec = v; break; }
    const int tuned = lz ? H->tune_lz_rows[fpi] : (combine ? H->tune_up_rows[fpi] : H->tune_dn_rows[fpi]);
    // untuned default: 4 rows for the FP32 combine pass (its registers limit
    // occupancy; the tuner's pick on the 4x4 sector), 8 otherwise
    const int tr_req = tuned ? tuned : ((combine && vec == 4) ? 4 : 8);
    *vec_out = vec;
    *tr_out = (tr_req == 4 || tr_req == 16) ? tr_req : 8;
}

// Shared memory of a windowed gather pass with TR rows per CTA.
template <typename T>
static size_t gwin_smem(int TR, int hmax) {
    const int hs = (std::max(1, hmax) + 3) & ~3;
    const size_t win = TR == 32 ? win_region_bytes<T, 32>() : win_region_bytes<T, 64>();
    return win + (size_t)TR * hs * (4 + sizeof(T));
}

// Rows per CTA of a windowed pass (knob: 0 = default 64, -1 = windows off).
static int gwin_rows(int knob) { return knob == 32 ? 32 : 64; }

// Whether this H·v runs the windowed passes (and so keeps Z row-major): the
// handle's choice, slices that are whole 16-byte packs, and shared memory
// for the hop lists of the longest per-spin list.
template <typename T>
static bool gwin_on(const gbr_ham *H) {
    const int fpi = sizeof(T) == 8 ? 1 : 0;
    if (H->win_dn[fpi] < 0) return false;
    if ((H->up.D * (int64_t)sizeof(T)) % 16 || (H->dn.D * (int64_t)sizeof(T)) % 16) return false;
    const int hmax = std::max(H->up.hmax, H->dn.hmax);
    return gwin_smem<T>(64, hmax) <= 200 * 1024;
}

// Windowed row-gather pass (k_gwin); the caller has checked gwin_on and the
// 16-byte alignment of every vector the pass reads or writes.
template <typename T, int MODE>
static int launch_gwin(const gbr_ham *H, const SpinSector &lists, int64_t Drows, int64_t Dcols, const T *w, T *z,
                       const CombineArgs &ca, cudaStream_t st, const HamDev &hd, int TR, int *grid_out) {
    constexpr int WC = 32 * (16 / (int)sizeof(T));
    const int64_t nrb = (Drows + TR - 1) / TR;
    const int64_t ncc = (Dcols + WC - 1) / WC;
    const int hmax = std::max(1, lists.hmax);
    const size_t smem = gwin_smem<T>(TR, hmax);
    const int64_t blocks = nrb * ncc;
    if (blocks > 0x7FFFFFFF) return set_error(GBR_EINVAL, "sector too large for the gather grid");
#define GBR_W(R)                                                                                                    \
    {                                                                                                               \
        auto kern = k_gwin<T, MODE, R>;                                                                             \
        GBR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));          \
        kern<<<(int)blocks, 256, smem, st>>>(Drows, Dcols, hmax, nrb, lists.hop_cnt.as<uint16_t>(),                \
                                             lists.hop_tgt.as<uint32_t>(), lists.hop_bond.as<uint16_t>(),           \
                                             (const T *)hd.bcoef, H->k.uniform, (T)H->k.hu, w, z, ca);               \
    }
    if (TR == 32) GBR_W(32) else GBR_W(64)
#undef GBR_W
    GBR_LAUNCH_CHECK();
    count_launches(1);
    if (grid_out) *grid_out = (int)blocks;
    return GBR_OK;
}

// One row-gather pass Z = H_lists W (+ the combine epilogue, + the Lanczos update).
// MODE 3 runs only with full 16-byte vectors and the Z tile (the caller has
// checked that the windowed passes are off); on any other launch shape it
// launches nothing and sets *declined.
template <typename T, int MODE>
static int launch_gather(const gbr_ham *H, const SpinSector &lists, int64_t Drows, int64_t Dcols, const T *w, T *z,
                         const CombineArgs &ca, cudaStream_t st, const HamDev &hd, int *grid_out = nullptr,
                         bool *declined = nullptr) {
    constexpr bool COMBINE = MODE >= 1;
    constexpr int VM = 16 / (int)sizeof(T);
    if (declined) *declined = false;
    if constexpr (MODE == 3) {
        if (ca.zrow || !ca.lz.xt_next) {
            if (declined) *declined = true;
            return GBR_OK;
        }
    } else if (gwin_on<T>(H)) {
        // the windowed kernels need every vector on a 16-byte boundary
        uintptr_t al = (uintptr_t)w | (uintptr_t)z;
        if (COMBINE) al |= (uintptr_t)ca.zt;
        if (MODE == 2) al |= (uintptr_t)ca.lz.vprev;
        const int fpi = sizeof(T) == 8 ? 1 : 0;
        const int knob = MODE == 0 ? H->win_dn[fpi] : (MODE == 1 ? H->win_up[fpi] : H->win_lz[fpi]);
        if ((al & 15u) == 0) return launch_gwin<T, MODE>(H, lists, Drows, Dcols, w, z, ca, st, hd, gwin_rows(knob), grid_out);
        // MODE 0 always gets the 16-byte aligned scratch; a combine pass on
        // unaligned vectors falls through to the plain kernel reading Z row-major
    }
    bool aligned16 = (((uintptr_t)w | (uintptr_t)z) & 15u) == 0;
    if (MODE >= 2) aligned16 = aligned16 && (((uintptr_t)ca.lz.vprev) & 15u) == 0;
    int vec = 1, TR = 8;
    const int fpi = sizeof(T) == 8 ? 1 : 0;
    const int NT = H->gather_nt[MODE >= 2 ? 2 : MODE][fpi] == 64 ? 64 : 128;
    gather_shape<T>(H, Drows, Dcols, aligned16, COMBINE, MODE >= 2, NT, &vec, &TR);
    if (MODE == 3 && vec != VM) {
        if (declined) *declined = true;
        return GBR_OK;
    }
    const int64_t nrb = (Drows + TR - 1) / TR;
    const int64_t ncc = (Dcols + NT * vec - 1) / (NT * vec);
    const int hmax = std::max(1, lists.hmax);
    const int hs = (hmax + 3) & ~3;   // the kernel's padded hop-list stride
    // hop lists, then (combine) the Z tile and the row slots for x and (Lanczos) u_{k-1}
    const size_t smem = (size_t)TR * hs * (4 + sizeof(T)) +
                        (COMBINE ? (size_t)TR * (NT * vec + ztile_pad((int)sizeof(T), TR)) * sizeof(T) + (MODE >= 2 ? 2 : 1) * (size_t)NT * vec * sizeof(T)
                                 : 0);
    const int64_t blocks = nrb * ncc;
    if (blocks > 0x7FFFFFFF) return set_error(GBR_EINVAL, "sector too large for the gather grid");
#define GBR_G(V, R, N)                                                                                       \
    {                                                                                                        \
        auto kern = k_gather<T, V, MODE, R, N>;                                                              \
        if (smem > 48 * 1024) GBR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        kern<<<(int)blocks, N, smem, st>>>(Drows, Dcols, hmax, nrb, lists.hop_cnt.as<uint16_t>(),            \
                                           lists.hop_tgt.as<uint32_t>(), lists.hop_bond.as<uint16_t>(),      \
                                           (const T *)hd.bcoef, H->k.uniform, (T)H->k.hu, w, z, ca);          \
    }
#define GBR_GN(V, R)                                                                                         \
    {                                                                                                        \
        if (NT == 64) GBR_G(V, R, 64) else GBR_G(V, R, 128)                                                  \
    }
#define GBR_GV(V)                                                                                            \
    {                                                                                                        \
        if (TR == 4) GBR_GN(V, 4) else if (TR == 16) GBR_GN(V, 16) else GBR_GN(V, 8)                         \
    }
    if constexpr (MODE == 3) {
        GBR_GV(VM)
    } else {
        if (vec == 4) GBR_GV(4) else if (vec == 2) GBR_GV(2) else GBR_GV(1)
    }
#undef GBR_GV
#undef GBR_GN
#undef GBR_G
    GBR_LAUNCH_CHECK();
    count_launches(1);
    if (grid_out) *grid_out = (int)blocks;
    return GBR_OK;
}

template <typename T>
static int stage_transpose(const gbr_ham *H, const T *x, cudaStream_t st, const Scratch *ws = nullptr) {
    if (!ws) {
        int rc = ensure_ws(H, (size_t)H->D * sizeof(T));
        if (rc) return rc;
    }
    T *xt = ws ? (T *)ws->xt : H->ws_xt.as<T>();
    const int64_t Dup = H->up.D, Ddn = H->dn.D;
    constexpr int TILE = 64, V = 16 / (int)sizeof(T);
    dim3 grid((unsigned)((Ddn + TILE - 1) / TILE), (unsigned)((Dup + TILE - 1) / TILE));
    if (grid.y > 65535) return set_error(GBR_EINVAL, "sector too large for the transpose grid");
    const bool packs = ((((uintptr_t)x) | ((uintptr_t)xt)) & 15u) == 0 && Dup % V == 0 && Ddn % V == 0;
    if (packs) k_transpose16<T><<<grid, 256, 0, st>>>(x, xt, Dup, Ddn);
    else k_transpose<T, TILE><<<grid, dim3(TILE, 4), 0, st>>>(x, xt, Dup, Ddn);
    GBR_LAUNCH_CHECK();
    count_launches(1);
    return GBR_OK;
}

// Z^T = H_dn X^T (rows: spin-down states, columns: spin-up states)
template <typename T>
static int stage_dn(const gbr_ham *H, cudaStream_t st, const HamDev &hd, const Scratch *ws = nullptr) {
    CombineArgs ca{};
    T *xt = ws ? (T *)ws->xt : H->ws_xt.as<T>();
    T *zt = ws ? (T *)ws->zt : H->ws_zt.as<T>();
    return launch_gather<T, 0>(H, dn_lists(H), H->dn.D, H->up.D, xt, zt, ca, st, hd);
}

// Y = H_up X + Dg o X + (Z^T)^T
template <typename T>
static int stage_up(const gbr_ham *H, const T *x, T *y, cudaStream_t st, const HamDev &hd,
                    const Scratch *ws = nullptr, const LzHook *hook = nullptr, int *nparts = nullptr,
                    bool *updated = nullptr) {
    CombineArgs ca;
    ca.lz = hook ? *hook : LzHook{nullptr, nullptr, nullptr, nullptr};
    ca.st_up = H->up.states.as<uint32_t>();
    ca.st_dn = H->dn.states.as<uint32_t>();
    ca.dup = hd.dup;
    ca.ddn = hd.ddn;
    ca.uval = hd.uval;
    ca.zt = ws ? ws->zt : H->ws_zt.p;
    ca.hk = H->k;
    ca.zrow = gwin_on<T>(H) ? 1 : 0;
    if (updated) *updated = false;
    if (hook && hook->xt_next) {
        bool declined = true;
        int rc = launch_gather<T, 3>(H, H->up, H->up.D, H->dn.D, x, y, ca, st, hd, nparts, &declined);
        if (rc || !declined) {
            if (!rc && updated) *updated = true;
            return rc;
        }
        ca.lz.xt_next = nullptr;
    }
    if (hook) return launch_gather<T, 2>(H, H->up, H->up.D, H->dn.D, x, y, ca, st, hd, nparts);
    return launch_gather<T, 1>(H, H->up, H->up.D, H->dn.D, x, y, ca, st, hd, nparts);
}

template <typename T>
static int launch_factored(const gbr_ham *H, const T *x, T *y, cudaStream_t st, const HamDev &hd,
                           cudaEvent_t *ev = nullptr, const Scratch *ws = nullptr, const LzHook *hook = nullptr,
                           int *nparts = nullptr, bool xt_ready = false, bool *updated = nullptr) {
    if (ev) cudaEventRecord(ev[0], st);
    int rc = stage_hop_lists<T>(H, st);
    if (rc) return rc;
    if (ev) cudaEventRecord(ev[1], st);
    if (!xt_ready && (rc = stage_transpose<T>(H, x, st, ws))) return rc;
    if (ev) cudaEventRecord(ev[2], st);
    if ((rc = stage_dn<T>(H, st, hd, ws))) return rc;
    if (ev) cudaEventRecord(ev[3], st);
    if ((rc = stage_up<T>(H, x, y, st, hd, ws, hook, nparts, updated))) return rc;
    if (ev) cudaEventRecord(ev[4], st);
    return GBR_OK;
}

}  // namespace gbr

// Precision-specific device arrays hang off the handle as extra buffers.
struct gbr_ham_prec {
    gbr::DevBuf dup, ddn, uval, bcoef, hcoef;
};

namespace gbr {

static gbr_ham_prec *prec_bufs(const gbr_ham *H, int fpi);

int hv_launch(const gbr_ham *H, const void *x, void *y, int fp, cudaStream_t st, cudaEvent_t *ev) {
    const int fpi = fp == 64 ? 1 : 0;
    gbr_ham_prec *pb = prec_bufs(H, fpi);
    HamDev hd{pb->dup.p, pb->ddn.p, pb->uval.p, pb->bcoef.p, pb->hcoef.p};
    int path = H->path;
    if (path == GBR_HV_AUTO) path = H->D <= (1 << 17) ? GBR_HV_FUSED : GBR_HV_FACTORED;
    if (path == GBR_HV_FUSED) {
        int rc;
        if (ev)
            for (int e = 0; e < 4; ++e) cudaEventRecord(ev[e], st);
        if (fp == 64) rc = launch_fused<double>(H, (const double *)x, (double *)y, st, hd);
        else rc = launch_fused<float>(H, (const float *)x, (float *)y, st, hd);
        if (ev) cudaEventRecord(ev[4], st);
        return rc;
    }
    if (fp == 64) return launch_factored<double>(H, (const double *)x, (double *)y, st, hd, ev);
    return launch_factored<float>(H, (const float *)x, (float *)y, st, hd, ev);
}

bool hv_is_factored(const gbr_ham *H) {
    return H->path == GBR_HV_FACTORED || (H->path == GBR_HV_AUTO && H->D > (1 << 17));
}

int hv_launch_lz(const gbr_ham *H, const void *x, void *y, int fp, cudaStream_t st, cudaEvent_t *ev, const LzHook &hook,
                 int *nparts, bool xt_ready, bool *updated) {
    const int fpi = fp == 64 ? 1 : 0;
    gbr_ham_prec *pb = prec_bufs(H, fpi);
    HamDev hd{pb->dup.p, pb->ddn.p, pb->uval.p, pb->bcoef.p, pb->hcoef.p};
    if (fp == 64)
        return launch_factored<double>(H, (const double *)x, (double *)y, st, hd, ev, nullptr, &hook, nparts, xt_ready,
                                       updated);
    return launch_factored<float>(H, (const float *)x, (float *)y, st, hd, ev, nullptr, &hook, nparts, xt_ready,
                                  updated);
}

void *hv_xt_scratch(const gbr_ham *H, int fp) {
    const size_t bytes = (size_t)H->D * (fp == 64 ? 8 : 4);
    return ensure_ws(H, bytes) ? nullptr : H->ws_xt.p;
}

int64_t hv_lz_parts(const gbr_ham *H, int fp) {
    // the smallest launch shape (vector width 1, 4 rows and 64 threads per
    // CTA) bounds every grid
    const int64_t nrb = (H->up.D + 3) / 4;
    const int64_t ncc = (H->dn.D + 63) / 64;
    (void)fp;
    return nrb * ncc;
}

int hv_factored_with_scratch(const gbr_ham *H, const void *x, void *y, int fp, cudaStream_t st, void *xt, void *zt) {
    const int fpi = fp == 64 ? 1 : 0;
    gbr_ham_prec *pb = prec_bufs(H, fpi);
    HamDev hd{pb->dup.p, pb->ddn.p, pb->uval.p, pb->bcoef.p, pb->hcoef.p};
    const Scratch ws{xt, zt};
    if (fp == 64) return launch_factored<double>(H, (const double *)x, (double *)y, st, hd, nullptr, &ws);
    return launch_factored<float>(H, (const float *)x, (float *)y, st, hd, nullptr, &ws);
}

int hv_stage(const gbr_ham *H, const void *x, void *y, int fp, int stage, cudaStream_t st) {
    const int fpi = fp == 64 ? 1 : 0;
    // the gather stages read the hop lists (stage 1) and the handle's scratch
    // (stage 2 allocates it): refuse them before those stages have run
    if (stage >= 3) {
        if (!H->up.lists_ready || !dn_lists(H).lists_ready)
            return set_error(GBR_EINVAL, "stage %d before stage 1 (hop lists) on this handle", stage);
        const size_t need = (size_t)H->D * (fp == 64 ? 8 : 4);
        if (H->ws_xt.bytes < need || H->ws_zt.bytes < need)
            return set_error(GBR_EINVAL, "stage %d before stage 2 (scratch) in this precision", stage);
    }
    gbr_ham_prec *pb = prec_bufs(H, fpi);
    HamDev hd{pb->dup.p, pb->ddn.p, pb->uval.p, pb->bcoef.p, pb->hcoef.p};
    if (fp == 64) {
        if (stage == 1) return stage_hop_lists<double>(H, st);
        if (stage == 2) return stage_transpose<double>(H, (const double *)x, st);
        if (stage == 3) return stage_dn<double>(H, st, hd);
        return stage_up<double>(H, (const double *)x, (double *)y, st, hd);
    }
    if (stage == 1) return stage_hop_lists<float>(H, st);
    if (stage == 2) return stage_transpose<float>(H, (const float *)x, st);
    if (stage == 3) return stage_dn<float>(H, st, hd);
    return stage_up<float>(H, (const float *)x, (float *)y, st, hd);
}

// ------------------------------------------------------------- host build

static std::vector<gbr_ham_prec *> g_prec_owner;   // never shared across handles

static int build_spin(gbr_ham *H, SpinSector &s, int N) {
    s.L = H->L;
    s.N = N;
    int rc = GBR_OK;
    for (int R : {8, 4}) {
        StagDesc &d = R == 8 ? s.desc : s.desc4;
        if ((rc = stag_plan(H->L, N, std::min(R, H->L), &d))) return rc;
        if (d.Q > kSpinChunks) return set_error(GBR_EINVAL, "internal: %d chunks", d.Q);
        std::vector<uint64_t> tab;
        stag_fill(d, tab);
        if (d.wide) return set_error(GBR_EINVAL, "per-spin ranks exceed 32 bits");
        std::vector<uint32_t> t32(tab.begin(), tab.end());
        if ((rc = (R == 8 ? s.stag : s.stag4).upload(t32.data(), t32.size() * 4))) return rc;
    }
    std::vector<uint64_t> st;
    enumerate_combinations(H->L, N, st);
    s.D = (int64_t)st.size();
    if (s.D != (int64_t)binom(H->L, N)) return set_error(GBR_EINVAL, "internal: enumeration size mismatch");
    if (s.D >= (int64_t)1 << 31) return set_error(GBR_EINVAL, "per-spin dimension %lld too large", (long long)s.D);
    std::vector<uint32_t> st32(st.begin(), st.end());
    rc = s.states.upload(st32.data(), st32.size() * 4);
    if (rc) return rc;
    // per-state diagonal and hop counts (host, for sizing and element counts)
    std::vector<double> dg((size_t)s.D);
    int hmax = 0;
    int64_t hops = 0;
    for (int64_t r = 0; r < s.D; ++r) {
        const uint32_t a = st32[(size_t)r];
        double d = 0.0;
        int k = 0;
        for (int p = 0; p < H->L; ++p) {
            if (!((a >> p) & 1u)) continue;
            d += H->h[(size_t)(p * H->L + p)];
            k += __builtin_popcount(H->k.nbr[p] & ~a);
        }
        dg[(size_t)r] = d;
        hmax = std::max(hmax, k);
        hops += k;
    }
    s.hmax = hmax;
    s.hops = hops;
    rc = s.diag.upload(dg.data(), dg.size() * 8);
    if (rc) return rc;
    const int64_t hm = std::max(1, hmax);
    if ((rc = s.hop_cnt.alloc((size_t)s.D * 2))) return rc;
    // no hops until the first ranking pass writes the lists: a gather pass
    // that ran before it reads empty lists, never stale targets
    GBR_CUDA_TRY(cudaMemset(s.hop_cnt.p, 0, (size_t)s.D * 2));
    if ((rc = s.hop_tgt.alloc((size_t)(hm * s.D) * 4))) return rc;
    if ((rc = s.hop_bond.alloc((size_t)(hm * s.D) * 2))) return rc;
    return GBR_OK;
}

template <typename T>
static int upload_prec(gbr_ham *H, gbr_ham_prec *pb) {
    auto conv = [](const std::vector<double> &v) { return std::vector<T>(v.begin(), v.end()); };
    std::vector<double> dup((size_t)H->up.D), ddn((size_t)H->dn.D);
    GBR_CUDA_TRY(cudaMemcpy(dup.data(), H->up.diag.p, dup.size() * 8, cudaMemcpyDeviceToHost));
    GBR_CUDA_TRY(cudaMemcpy(ddn.data(), H->dn.diag.p, ddn.size() * 8, cudaMemcpyDeviceToHost));
    std::vector<double> uv(kMaxUClasses, 0.0), bc, hc((size_t)H->L * H->L, 0.0);
    for (int c = 0; c < H->k.nucls; ++c) uv[(size_t)c] = H->k.uval[c];
    for (int p = 0; p < H->L; ++p)
        for (int q = 0; q < H->L; ++q)
            if (p != q) hc[(size_t)(p * H->L + q)] = H->h[(size_t)(p * H->L + q)];
    for (int p = 0; p < H->L; ++p)
        for (int q = 0; q < H->L; ++q)
            if (p != q && H->h[(size_t)(p * H->L + q)] != 0.0) bc.push_back(H->h[(size_t)(p * H->L + q)]);
    if (bc.empty()) bc.push_back(0.0);
    int rc;
    auto a = conv(dup), b = conv(ddn), u = conv(uv), c = conv(bc), h = conv(hc);
    if ((rc = pb->dup.upload(a.data(), a.size() * sizeof(T)))) return rc;
    if ((rc = pb->ddn.upload(b.data(), b.size() * sizeof(T)))) return rc;
    if ((rc = pb->uval.upload(u.data(), u.size() * sizeof(T)))) return rc;
    if ((rc = pb->bcoef.upload(c.data(), c.size() * sizeof(T)))) return rc;
    if ((rc = pb->hcoef.upload(h.data(), h.size() * sizeof(T)))) return rc;
    return GBR_OK;
}

int build_hamk(int L, const double *h, const double *U, int rank_method, HamK *kout, std::vector<uint16_t> *pairs,
               std::vector<uint16_t> *bidx) {
    HamK &k = *kout;
    memset(&k, 0, sizeof(k));
    k.L = L;
    k.rank_method = rank_method;
    pairs->clear();
    bidx->assign((size_t)L * L, 0);
    double first = 0.0;
    k.uniform = 1;
    for (int p = 0; p < L; ++p)
        for (int q = 0; q < L; ++q) {
            if (p == q) continue;
            const double v = h[p * L + q];
            if (v == 0.0) continue;
            if (k.nbond == 0) first = v;
            else if (v != first) k.uniform = 0;
            (*bidx)[(size_t)(p * L + q)] = (uint16_t)k.nbond;
            pairs->push_back((uint16_t)p);
            pairs->push_back((uint16_t)q);
            k.nbr[p] |= 1u << q;
            ++k.nbond;
        }
    k.hu = first;
    for (int p = 0; p < L; ++p) {
        const double u = U ? U[p] : 0.0;
        if (u == 0.0) continue;
        int c = 0;
        while (c < k.nucls && k.uval[c] != u) ++c;
        if (c == k.nucls) {
            if (k.nucls == kMaxUClasses) return set_error(GBR_EINVAL, "more than %d distinct U values", kMaxUClasses);
            k.uval[c] = u;
            ++k.nucls;
        }
        k.umask[c] |= 1u << p;
    }
    return GBR_OK;
}

}  // namespace gbr

using namespace gbr;

struct gbr_ham_ext {
    gbr_ham_prec prec[2];
};

// The handle is allocated together with its precision buffers.
struct gbr_ham_full : gbr_ham {
    gbr_ham_ext ext;
};

namespace gbr {
static gbr_ham_prec *prec_bufs(const gbr_ham *H, int fpi) {
    return &const_cast<gbr_ham_full *>(static_cast<const gbr_ham_full *>(H))->ext.prec[fpi];
}
}  // namespace gbr

extern "C" int gbr_ham_create(int L, const double *h, const double *U, int Nup, int Ndn, int rank_method,
                              gbr_ham **out) {
    clear_error();
    if (!out) return set_error(GBR_EINVAL, "out is NULL");
    *out = nullptr;
    if (L < 1 || L > kMaxL) return set_error(GBR_EINVAL, "L=%d out of range 1..%d", L, kMaxL);
    if (!h) return set_error(GBR_EINVAL, "h is NULL");
    if (Nup < 0 || Nup > L || Ndn < 0 || Ndn > L) return set_error(GBR_EINVAL, "particle numbers out of range");
    if (rank_method != GBR_RANK_STAGGERED && rank_method != GBR_RANK_CNS)
        return set_error(GBR_EINVAL, "unknown rank_method %d", rank_method);
    for (int p = 0; p < L; ++p)
        for (int q = 0; q < L; ++q) {
            const double a = h[p * L + q], b = h[q * L + p];
            if (!std::isfinite(a)) return set_error(GBR_EINVAL, "h[%d][%d] is not finite", p, q);
            if (a != b) return set_error(GBR_EINVAL, "h is not symmetric at (%d, %d)", p, q);
        }
    if (U)
        for (int p = 0; p < L; ++p)
            if (!std::isfinite(U[p])) return set_error(GBR_EINVAL, "U[%d] is not finite", p);
    gbr_ham_full *H = new (std::nothrow) gbr_ham_full();
    if (!H) return set_error(GBR_ENOMEM, "host allocation failed");
    H->L = L; H->Nup = Nup; H->Ndn = Ndn;
    H->rank_method = rank_method;
    H->path = GBR_HV_AUTO;
    H->h.assign(h, h + L * L);
    H->U.assign(L, 0.0);
    if (U) H->U.assign(U, U + L);
    // one-body bonds in (p, q) order, neighbour masks, U classes
    std::vector<uint16_t> pairs, bidx;
    {
        const int rck = build_hamk(L, h, H->U.data(), rank_method, &H->k, &pairs, &bidx);
        if (rck) { delete H; return rck; }
    }
    std::vector<uint16_t> bonds_blob(pairs);
    bonds_blob.insert(bonds_blob.end(), bidx.begin(), bidx.end());
    int rc = H->bonds.upload(bonds_blob.data(), bonds_blob.size() * 2);
    std::vector<uint32_t> bin((size_t)(L + 1) * (L + 1));
    for (int n = 0; n <= L; ++n)
        for (int kk = 0; kk <= L; ++kk) bin[(size_t)(n * (L + 1) + kk)] = (uint32_t)binom(n, kk);
    if (!rc) rc = H->binom.upload(bin.data(), bin.size() * 4);
    if (!rc) rc = build_spin(H, H->up, Nup);
    if (!rc) rc = build_spin(H, H->dn, Ndn);
    if (!rc) {
        H->D = H->up.D * H->dn.D;
        H->elements = H->D + H->up.hops * H->dn.D + H->dn.hops * H->up.D;
        rc = upload_prec<float>(H, &H->ext.prec[0]);
        if (!rc) rc = upload_prec<double>(H, &H->ext.prec[1]);
    }
    if (rc) { delete H; return rc; }
    *out = H;
    return GBR_OK;
}

extern "C" void gbr_ham_destroy(gbr_ham *H) { delete static_cast<gbr_ham_full *>(H); }

extern "C" int gbr_ham_info(const gbr_ham *H, int64_t *dim, int64_t *elements) {
    clear_error();
    if (!H) return set_error(GBR_EINVAL, "NULL handle");
    if (dim) *dim = H->D;
    if (elements) *elements = H->elements;
    return GBR_OK;
}

extern "C" int gbr_ham_set_path(gbr_ham *H, int path) {
    clear_error();
    if (!H) return set_error(GBR_EINVAL, "NULL handle");
    if (path != GBR_HV_AUTO && path != GBR_HV_FUSED && path != GBR_HV_FACTORED)
        return set_error(GBR_EINVAL, "unknown path %d", path);
    H->path = path;
    return GBR_OK;
}

extern "C" int gbr_ham_get_path(const gbr_ham *H, int *path) {
    clear_error();
    if (!H || !path) return set_error(GBR_EINVAL, "NULL argument");
    *path = H->path;
    return GBR_OK;
}

extern "C" int gbr_hv(const gbr_ham *H, const void *d_x, void *d_y, int fp, void *stream) {
    clear_error();
    if (!H) return set_error(GBR_EINVAL, "NULL handle");
    if (fp != 32 && fp != 64) return set_error(GBR_EINVAL, "fp=%d must be 32 or 64", fp);
    if (!d_x || !d_y) return set_error(GBR_EINVAL, "NULL vector");
    const size_t s = fp == 64 ? 8 : 4;
    const uintptr_t xa = (uintptr_t)d_x, ya = (uintptr_t)d_y;
    if ((xa | ya) % s) return set_error(GBR_EINVAL, "vectors must be aligned to their element size");
    const uintptr_t bytes = (uintptr_t)H->D * s;
    if (xa < ya + bytes && ya < xa + bytes) return set_error(GBR_EINVAL, "x and y overlap");
    return hv_launch(H, d_x, d_y, fp, (cudaStream_t)stream);
}

extern "C" int gbr_hv_stage(const gbr_ham *H, const void *d_x, void *d_y, int fp, int stage, void *stream) {
    clear_error();
    if (!H) return set_error(GBR_EINVAL, "NULL handle");
    if (fp != 32 && fp != 64) return set_error(GBR_EINVAL, "fp=%d must be 32 or 64", fp);
    if (stage < 1 || stage > 4) return set_error(GBR_EINVAL, "stage=%d must be 1..4", stage);
    if (stage == 2 || stage == 4) {
        if (!d_x || !d_y) return set_error(GBR_EINVAL, "NULL vector");
        const size_t s = fp == 64 ? 8 : 4;
        const uintptr_t xa = (uintptr_t)d_x, ya = (uintptr_t)d_y;
        if ((xa | ya) % s) return set_error(GBR_EINVAL, "vectors must be aligned to their element size");
        const uintptr_t bytes = (uintptr_t)H->D * s;
        if (xa < ya + bytes && ya < xa + bytes) return set_error(GBR_EINVAL, "x and y overlap");
    }
    return hv_stage(H, d_x, d_y, fp, stage, (cudaStream_t)stream);
}

extern "C" int gbr_ham_set_shape(gbr_ham *H, int fp, const int *shape) {
    clear_error();
    if (!H || !shape) return set_error(GBR_EINVAL, "NULL argument");
    if (fp != 32 && fp != 64) return set_error(GBR_EINVAL, "fp=%d must be 32 or 64", fp);
    const int fpi = fp == 64 ? 1 : 0;
    if (shape[0] != 0 && shape[0] != 1) return set_error(GBR_EINVAL, "window flag %d must be 0 or 1", shape[0]);
    for (int i = 1; i < 4; ++i) {
        const int v = shape[i];
        const bool okv = v == 0 || (shape[0] ? (v == 32 || v == 64) : (v == 4 || v == 8 || v == 16));
        if (!okv) return set_error(GBR_EINVAL, "rows per CTA %d not allowed for this family", v);
    }
    if (shape[4] != 0 && shape[4] != 4 && shape[4] != 8) return set_error(GBR_EINVAL, "chunk width %d must be 4 or 8", shape[4]);
    if (shape[5] != 0 && shape[5] != 1 && shape[5] != 2 && shape[5] != 4)
        return set_error(GBR_EINVAL, "threads per state %d must be 1, 2 or 4", shape[5]);
    for (int i = 6; i < 9; ++i)
        if (shape[i] != 0 && shape[i] != 64 && shape[i] != 128)
            return set_error(GBR_EINVAL, "threads per CTA %d must be 64 or 128", shape[i]);
    H->rank_R[fpi] = shape[4] ? shape[4] : 8;
    H->fused_tps[fpi] = shape[5] ? shape[5] : 1;
    H->gather_nt[0][fpi] = shape[6] ? shape[6] : 128;
    H->gather_nt[1][fpi] = shape[7] ? shape[7] : 128;
    H->gather_nt[2][fpi] = shape[8] ? shape[8] : 128;
    if (shape[0]) {
        H->win_dn[fpi] = shape[1];
        H->win_up[fpi] = shape[2];
        H->win_lz[fpi] = shape[3];
    } else {
        H->win_dn[fpi] = -1;
        H->tune_dn_rows[fpi] = shape[1];
        H->tune_up_rows[fpi] = shape[2];
        H->tune_lz_rows[fpi] = shape[3];
    }
    return GBR_OK;
}

extern "C" int gbr_ham_get_shape(const gbr_ham *H, int fp, int *shape) {
    clear_error();
    if (!H || !shape) return set_error(GBR_EINVAL, "NULL argument");
    if (fp != 32 && fp != 64) return set_error(GBR_EINVAL, "fp=%d must be 32 or 64", fp);
    const int fpi = fp == 64 ? 1 : 0;
    const bool on = fp == 64 ? gwin_on<double>(H) : gwin_on<float>(H);
    shape[0] = on ? 1 : 0;
    if (on) {
        shape[1] = gwin_rows(H->win_dn[fpi]);
        shape[2] = gwin_rows(H->win_up[fpi]);
        shape[3] = gwin_rows(H->win_lz[fpi]);
    } else {
        auto plain = [](int v, int dflt) { return (v == 4 || v == 8 || v == 16) ? v : dflt; };
        shape[1] = plain(H->tune_dn_rows[fpi], 8);
        shape[2] = plain(H->tune_up_rows[fpi], 8);
        shape[3] = plain(H->tune_lz_rows[fpi], 8);
    }
    shape[4] = H->rank_R[fpi];
    shape[5] = H->fused_tps[fpi];
    for (int i = 0; i < 3; ++i) shape[6 + i] = on ? 256 : H->gather_nt[i][fpi];
    return GBR_OK;
}

extern "C" int gbr_device_status(int clear, int *status) {
    clear_error();
    if (!status) return set_error(GBR_EINVAL, "NULL argument");
    int v = 0;
    GBR_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_gbr_status, sizeof(int)));
    if (clear) {
        const int zero = 0;
        GBR_CUDA_TRY(cudaMemcpyToSymbol(g_gbr_status, &zero, sizeof(int)));
    }
    *status = v;
    return v ? set_error(GBR_ETIMEOUT, "a bounded device-side wait ran out (status 0x%x)", v) : GBR_OK;
}

// Times the candidate launch shapes on scratch vectors and keeps the fastest
// in the handle: the path (fused for sectors up to 2^22 states), the gather
// family (plain row gathers, or windowed gathers with the CTA's own rows in
// shared memory), the rows per CTA of the spin-up and spin-down passes in
// that family, the rows per CTA of the spin-up pass with the fused Lanczos
// update, the chunk width of the per-spin staggered tables, and the threads
// per state of the fused kernel.
extern "C" int gbr_ham_tune(gbr_ham *H, int fp, void *stream) {
    clear_error();
    if (!H) return set_error(GBR_EINVAL, "NULL handle");
    if (fp != 32 && fp != 64) return set_error(GBR_EINVAL, "fp=%d must be 32 or 64", fp);
    const size_t s = fp == 64 ? 8 : 4;
    const int fpi = fp == 64 ? 1 : 0;
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf x, y, lz_part, lz_scal, lz_k;
    int rc;
    if ((rc = x.alloc((size_t)H->D * s))) return rc;
    if ((rc = y.alloc((size_t)H->D * s))) return rc;
    GBR_CUDA_TRY(cudaMemsetAsync(x.p, 0, x.bytes, st));
    cudaEvent_t e0, e1;
    GBR_CUDA_TRY(cudaEventCreate(&e0));
    GBR_CUDA_TRY(cudaEventCreate(&e1));
    auto time_it = [&](float *ms_out) -> int {
        int r = hv_launch(H, x.p, y.p, fp, st);   // warm-up (also sets kernel attributes)
        if (r) return r;
        cudaEventRecord(e0, st);
        for (int i = 0; i < 3; ++i)
            if ((r = hv_launch(H, x.p, y.p, fp, st))) return r;
        cudaEventRecord(e1, st);
        cudaError_t ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) return set_error(GBR_ECUDA, "tune: %s", cudaGetErrorString(ce));
        cudaEventElapsedTime(ms_out, e0, e1);
        return GBR_OK;
    };
    const int keep_path = H->path;
    float best = 1e30f, ms = 0.f;
    int best_path = GBR_HV_FACTORED;
    H->path = GBR_HV_FACTORED;
    const int keep_win = H->win_dn[fpi];
    // rows per CTA of the spin-up (combine) pass, then of the spin-down pass,
    // first with the plain row gathers, then (where the sector allows) with
    // the windowed ones; the faster family stays on
    float best_plain = 1e30f, best_win = 1e30f;
    int win_pick[2] = {0, 0};
    H->win_dn[fpi] = -1;
    for (int pass = 0; pass < 2; ++pass) {
        int *knob = pass == 0 ? &H->tune_up_rows[fpi] : &H->tune_dn_rows[fpi];
        int *nt_knob = &H->gather_nt[pass == 0 ? 1 : 0][fpi];
        int best_tr = 8, best_nt = 128;
        for (int nt : {128, 64})
            for (int tr : {4, 8, 16}) {
                *knob = tr;
                *nt_knob = nt;
                if ((rc = time_it(&ms))) goto done;
                if (ms < best_plain || (tr == 8 && nt == 128 && ms <= best_plain)) {
                    best_plain = ms;
                    best_tr = tr;
                    best_nt = nt;
                }
            }
        *knob = best_tr;
        *nt_knob = best_nt;
    }
    {
        H->win_dn[fpi] = 0;
        if (fp == 64 ? gwin_on<double>(H) : gwin_on<float>(H)) {
            for (int pass = 0; pass < 2; ++pass) {
                int *knob = pass == 0 ? &H->win_up[fpi] : &H->win_dn[fpi];
                int best_tr = 64;
                for (int tr : {32, 64}) {
                    *knob = tr;
                    if ((rc = time_it(&ms))) goto done;
                    if (ms < best_win) { best_win = ms; best_tr = tr; }
                }
                *knob = best_tr;
                win_pick[pass] = best_tr;
            }
        }
    }
    H->win_dn[fpi] = best_win < best_plain ? win_pick[1] : -1;
    best = std::min(best_plain, best_win);
    // rows per CTA of the combine pass as the Lanczos launches it (fused
    // first update, another kernel with its own best tile), timed on that
    // kernel with a stand-in recurrence state (step 1, v_{k-1} = x)
    {
        const int64_t np = hv_lz_parts(H, fp);
        if ((rc = lz_part.alloc(sizeof(double) * (size_t)np))) goto done;
        if ((rc = lz_scal.alloc(sizeof(double) * 8))) goto done;
        if ((rc = lz_k.alloc(sizeof(int)))) goto done;
        const double scal[8] = {1.0, 0.0, 0.0, 0.0, 0.5, 0.5, 0.0, 0.0};
        const int k1 = 1;
        GBR_CUDA_TRY(cudaMemcpyAsync(lz_scal.p, scal, sizeof(scal), cudaMemcpyHostToDevice, st));
        GBR_CUDA_TRY(cudaMemcpyAsync(lz_k.p, &k1, sizeof(int), cudaMemcpyHostToDevice, st));
        const LzHook hook{x.p, lz_scal.as<double>(), lz_k.as<int>(), lz_part.as<double>()};
        auto time_lz = [&](float *ms_out) -> int {
            int np_out = 0;
            int r = hv_launch_lz(H, x.p, y.p, fp, st, nullptr, hook, &np_out);
            if (r) return r;
            cudaEventRecord(e0, st);
            for (int i = 0; i < 3; ++i)
                if ((r = hv_launch_lz(H, x.p, y.p, fp, st, nullptr, hook, &np_out))) return r;
            cudaEventRecord(e1, st);
            cudaError_t ce = cudaEventSynchronize(e1);
            if (ce != cudaSuccess) return set_error(GBR_ECUDA, "tune: %s", cudaGetErrorString(ce));
            cudaEventElapsedTime(ms_out, e0, e1);
            return GBR_OK;
        };
        const bool winmode = H->win_dn[fpi] >= 0;
        float best_lz = 1e30f;
        int best_tr = 0, best_nt = 128;
        for (int nt : {128, 64})
            for (int tr : {4, 8, 16, 32, 64}) {
                if (winmode != (tr >= 32) || (winmode && nt != 128)) continue;
                (winmode ? H->win_lz[fpi] : H->tune_lz_rows[fpi]) = tr;
                H->gather_nt[2][fpi] = nt;
                if ((rc = time_lz(&ms))) goto done;
                if (ms < best_lz) { best_lz = ms; best_tr = tr; best_nt = nt; }
            }
        (winmode ? H->win_lz[fpi] : H->tune_lz_rows[fpi]) = best_tr;
        H->gather_nt[2][fpi] = best_nt;
    }
    // chunk width of the per-spin tables in the factored path (its ranking
    // pass only), then the fused per-element kernel over chunk width and
    // threads per state (Sec. V-B compares R = 4 and 8 inside the H·v)
    {
        H->path = GBR_HV_FACTORED;
        float best_fac = 1e30f;
        int best_R = 8;
        for (int R : {8, 4}) {
            H->rank_R[fpi] = R;
            if ((rc = time_it(&ms))) goto done;
            if (ms < best_fac) { best_fac = ms; best_R = R; }
        }
        H->rank_R[fpi] = best_R;
        best = std::min(best, best_fac);
        if (H->D <= ((int64_t)1 << 22)) {
            H->path = GBR_HV_FUSED;
            float best_fu = 1e30f;
            int bR = 8, bT = 1;
            for (int R : {8, 4})
                for (int tps : {1, 2, 4}) {
                    H->rank_R[fpi] = R;
                    H->fused_tps[fpi] = tps;
                    if ((rc = time_it(&ms))) goto done;
                    if (ms < best_fu) { best_fu = ms; bR = R; bT = tps; }
                }
            H->fused_tps[fpi] = bT;
            if (best_fu < best) {
                best = best_fu;
                best_path = GBR_HV_FUSED;
                H->rank_R[fpi] = bR;
            } else {
                H->rank_R[fpi] = best_R;
            }
        }
    }
    H->path = keep_path == GBR_HV_AUTO ? best_path : keep_path;
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        H->path = keep_path;
        H->win_dn[fpi] = keep_win;
    }
    return rc;
}
