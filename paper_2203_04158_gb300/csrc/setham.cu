// On-the-fly H·v over an arbitrary sorted set of states, ranked by the packed
// trie (Sec. IV of Wallerberger & Held): the case the combinadics cannot
// index -- sectors cut by further quantum numbers, or unions of spin
// sectors such as all S_z at fixed particle number.  No spin factorisation:
// every hop of every member is ranked by a walk of Fig. trielookup over the
// full 2L-bit pattern, and (check mode) verified against the member list.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ham.h"

struct gbr_setham {
    int L = 0, R = 0;
    int bisect = 0;             // 1: rank by bisection in the member list instead of the trie
    int64_t n = 0;
    int64_t elements = 0;
    gbr::HamK k{};
    gbr_trie *trie = nullptr;
    gbr::DevBuf hc64, hc32;     // L x L off-diagonal one-body terms
    gbr::DevBuf hd64, hd32;     // L diagonal one-body terms h_pp
    gbr::DevBuf uv64, uv32;     // U class values
    gbr::LzWork lzw;            // Lanczos work buffers
    ~gbr_setham() { gbr_trie_destroy(trie); }
};

namespace gbr {

struct SetTrieK {
    int H;
    int shift[kMaxChunks];
    int width[kMaxChunks];
    int64_t padded, smem_entries, n;
};

template <typename T, typename E, bool BISECT>
__global__ void __launch_bounds__(256) k_set_hv(const SetTrieK tk, const E *__restrict__ t,
                                                const uint64_t *__restrict__ states, const HamK hk,
                                                const T *__restrict__ hc, const T *__restrict__ hd,
                                                const T *__restrict__ uv, int check, const T *__restrict__ x,
                                                T *__restrict__ y) {
    extern __shared__ __align__(16) unsigned char smr[];
    E *ts = reinterpret_cast<E *>(smr);
    T *hcs = reinterpret_cast<T *>(smr + ((tk.smem_entries * sizeof(E) + 15) & ~(int64_t)15));
    T *hds = hcs + hk.L * hk.L;
    for (int64_t i = threadIdx.x; i < tk.smem_entries; i += blockDim.x) ts[i] = __ldg(t + i);
    for (int i = threadIdx.x; i < hk.L * hk.L; i += blockDim.x) hcs[i] = hc[i];
    for (int i = threadIdx.x; i < hk.L; i += blockDim.x) hds[i] = hd[i];
    T uval[kMaxUClasses];
#pragma unroll
    for (int c = 0; c < kMaxUClasses; ++c) uval[c] = c < hk.nucls ? uv[c] : T(0);
    __syncthreads();
    const E last = (E)(tk.padded - 1), sm_end = (E)tk.smem_entries;
    const int L = hk.L;
    const uint64_t lowmask = L >= 64 ? ~0ull : ((1ull << L) - 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tk.n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t a = states[i];
        const uint32_t ad = (uint32_t)(a & lowmask), au = (uint32_t)(a >> L);
        // diagonal: one-body h_pp n_p for both spins, U on doubly occupied sites
        T dg = 0;
        uint32_t occ = ad | au;
        while (occ) {
            const int p = __ffs(occ) - 1;
            occ &= occ - 1u;
            dg += hds[p] * (T)(((ad >> p) & 1u) + ((au >> p) & 1u));
        }
#pragma unroll
        for (int c = 0; c < kMaxUClasses; ++c) {
            if (c >= hk.nucls) break;
            dg += uval[c] * (T)__popc(ad & au & hk.umask[c]);
        }
        T acc = dg * x[i];
        for (int spin = 0; spin < 2; ++spin) {
            const uint32_t sb = spin ? au : ad;
            const int off = spin ? L : 0;
            uint32_t o = sb;
            while (o) {
                const int p = __ffs(o) - 1;
                o &= o - 1u;
                uint32_t emp = hk.nbr[p] & ~sb;
                while (emp) {
                    const int q = __ffs(emp) - 1;
                    emp &= emp - 1u;
                    const uint64_t b = a ^ ((uint64_t)((1u << p) | (1u << q)) << off);
                    uint64_t k = 0;
                    if (BISECT) {
                        // the established baseline: lower bound in the sorted member list
                        int64_t lo = 0, len = tk.n;
                        while (len > 0) {
                            const int64_t half = len >> 1;
                            if (__ldg(states + lo + half) < b) { lo += half + 1; len -= half + 1; } else { len = half; }
                        }
                        k = (uint64_t)lo;
                    } else {
                        // Fig. trielookup on the full pattern, indices clamped into the table
                        E kk = 0;
                        for (int lvl = 0; lvl < tk.H; ++lvl) {
                            E idx = kk + (E)((uint32_t)(b >> tk.shift[lvl]) & ((1u << tk.width[lvl]) - 1u));
                            idx = idx > last ? last : idx;
                            kk = idx < sm_end ? ts[idx] : __ldg(t + idx);
                        }
                        k = (uint64_t)kk;
                    }
                    if ((check || BISECT) && !(k < (uint64_t)tk.n && __ldg(states + k) == b)) continue;
                    const int lo = min(p, q), hi = max(p, q);
                    const uint32_t between = ((hi >= 32) ? 0xFFFFFFFFu : ((1u << hi) - 1u)) & ~((1u << (lo + 1)) - 1u);
                    const T c = hcs[p * L + q];
                    const T v = x[(int64_t)k];
                    acc += (__popc(sb & between) & 1) ? -c * v : c * v;
                }
            }
        }
        y[i] = acc;
    }
}

template <typename T, typename E>
static int launch_set_hv(const gbr_setham *S, const T *x, T *y, int check, cudaStream_t st) {
    const gbr_trie *tr = S->trie;
    SetTrieK tk;
    memset(&tk, 0, sizeof(tk));
    tk.H = tr->H;
    for (int l = 0; l < tr->H; ++l) { tk.shift[l] = tr->shift[l]; tk.width[l] = tr->width[l]; }
    tk.padded = tr->padded;
    tk.smem_entries = tr->smem_entries;
    tk.n = S->n;
    const int fpi = sizeof(T) == 8;
    const T *hc = fpi ? (const T *)S->hc64.p : (const T *)S->hc32.p;
    const T *hd = fpi ? (const T *)S->hd64.p : (const T *)S->hd32.p;
    const T *uv = fpi ? (const T *)S->uv64.p : (const T *)S->uv32.p;
    const size_t smem = ((tr->smem_entries * sizeof(E) + 15) & ~(size_t)15) + (size_t)(S->L * S->L + S->L) * sizeof(T);
    int64_t blocks = (S->n + 255) / 256;
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sm_count() * 8));
    auto kern = S->bisect ? k_set_hv<T, E, true> : k_set_hv<T, E, false>;
    if (smem > 48 * 1024) GBR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(int)blocks, 256, smem, st>>>(tk, tr->t.as<E>(), tr->members.as<uint64_t>(), S->k, hc, hd, uv, check, x, y);
    GBR_LAUNCH_CHECK();
    count_launches(1);
    return GBR_OK;
}

// y = H x on the set with membership checks (the Lanczos operator; a set
// not closed under H gets the projected operator P H P)
static int set_apply(const void *obj, const void *x, void *y, int fp, cudaStream_t st) {
    const gbr_setham *S = static_cast<const gbr_setham *>(obj);
    if (S->trie->wide) {
        if (fp == 64) return launch_set_hv<double, uint64_t>(S, (const double *)x, (double *)y, 1, st);
        return launch_set_hv<float, uint64_t>(S, (const float *)x, (float *)y, 1, st);
    }
    if (fp == 64) return launch_set_hv<double, uint32_t>(S, (const double *)x, (double *)y, 1, st);
    return launch_set_hv<float, uint32_t>(S, (const float *)x, (float *)y, 1, st);
}

}  // namespace gbr

using namespace gbr;

extern "C" int gbr_setham_lanczos(const gbr_setham *S, const gbr_lanczos_opts *o, const double *d_v0,
                                  gbr_lanczos_result *res, double *h_alpha, double *h_beta, double *h_ritz,
                                  void *stream) {
    clear_error();
    if (!S) return set_error(GBR_EINVAL, "NULL handle");
    const LzOp op{nullptr, S, &set_apply, S->n, &const_cast<gbr_setham *>(S)->lzw};
    return lanczos_solve(op, o, d_v0, res, h_alpha, h_beta, h_ritz, stream);
}

extern "C" int gbr_setham_create_ordered(int L, const double *h, const double *U, const uint64_t *h_states,
                                         int64_t n, int R, int msb_first, gbr_setham **out) {
    clear_error();
    if (!out) return set_error(GBR_EINVAL, "out is NULL");
    *out = nullptr;
    if (L < 1 || L > kMaxL) return set_error(GBR_EINVAL, "L=%d out of range 1..%d", L, kMaxL);
    if (!h || !h_states) return set_error(GBR_EINVAL, "NULL argument");
    if (n < 1) return set_error(GBR_EINVAL, "empty state set");
    for (int p = 0; p < L; ++p)
        for (int q = 0; q < L; ++q) {
            const double a = h[p * L + q];
            if (!std::isfinite(a) || a != h[q * L + p]) return set_error(GBR_EINVAL, "h not finite and symmetric at (%d,%d)", p, q);
        }
    gbr_setham *S = new (std::nothrow) gbr_setham();
    if (!S) return set_error(GBR_ENOMEM, "host allocation failed");
    S->L = L;
    S->R = R;
    S->n = n;
    std::vector<uint16_t> pairs, bidx;
    int rc = build_hamk(L, h, U, GBR_RANK_STAGGERED, &S->k, &pairs, &bidx);
    if (!rc) rc = gbr_trie_create_ordered(h_states, n, 2 * L, R, msb_first, &S->trie);   // validates order, duplicates, width
    if (rc) { delete S; return rc; }
    // elements: the diagonal plus every hop of every member (for a set closed
    // under H, exactly the matrix elements one H·v visits)
    int64_t el = n;
    const uint64_t lowmask = (1ull << L) - 1;
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t sp[2] = {(uint32_t)(h_states[i] & lowmask), (uint32_t)(h_states[i] >> L)};
        for (int s = 0; s < 2; ++s)
            for (int p = 0; p < L; ++p)
                if ((sp[s] >> p) & 1u) el += __builtin_popcount(S->k.nbr[p] & ~sp[s]);
    }
    S->elements = el;
    std::vector<double> hc((size_t)L * L, 0.0), hd((size_t)L), uv(kMaxUClasses, 0.0);
    for (int p = 0; p < L; ++p) {
        hd[(size_t)p] = h[p * L + p];
        for (int q = 0; q < L; ++q)
            if (p != q) hc[(size_t)(p * L + q)] = h[p * L + q];
    }
    for (int c = 0; c < S->k.nucls; ++c) uv[(size_t)c] = S->k.uval[c];
    std::vector<float> hc32(hc.begin(), hc.end()), hd32(hd.begin(), hd.end()), uv32(uv.begin(), uv.end());
    if (!rc) rc = S->hc64.upload(hc.data(), hc.size() * 8);
    if (!rc) rc = S->hd64.upload(hd.data(), hd.size() * 8);
    if (!rc) rc = S->uv64.upload(uv.data(), uv.size() * 8);
    if (!rc) rc = S->hc32.upload(hc32.data(), hc32.size() * 4);
    if (!rc) rc = S->hd32.upload(hd32.data(), hd32.size() * 4);
    if (!rc) rc = S->uv32.upload(uv32.data(), uv32.size() * 4);
    if (rc) { delete S; return rc; }
    *out = S;
    return GBR_OK;
}

extern "C" int gbr_setham_create(int L, const double *h, const double *U, const uint64_t *h_states, int64_t n, int R,
                                 gbr_setham **out) {
    return gbr_setham_create_ordered(L, h, U, h_states, n, R, 1, out);
}

extern "C" void gbr_setham_destroy(gbr_setham *S) { delete S; }

extern "C" int gbr_setham_set_bisect(gbr_setham *S, int bisect) {
    clear_error();
    if (!S) return set_error(GBR_EINVAL, "NULL handle");
    S->bisect = bisect ? 1 : 0;
    return GBR_OK;
}

extern "C" int gbr_setham_info(const gbr_setham *S, int64_t *dim, int64_t *elements, int64_t *trie_elements) {
    clear_error();
    if (!S) return set_error(GBR_EINVAL, "NULL handle");
    if (dim) *dim = S->n;
    if (elements) *elements = S->elements;
    if (trie_elements) *trie_elements = S->trie->size;
    return GBR_OK;
}

extern "C" int gbr_setham_hv(const gbr_setham *S, const void *d_x, void *d_y, int fp, int check, void *stream) {
    clear_error();
    if (!S) return set_error(GBR_EINVAL, "NULL handle");
    if (fp != 32 && fp != 64) return set_error(GBR_EINVAL, "fp=%d must be 32 or 64", fp);
    if (!d_x || !d_y) return set_error(GBR_EINVAL, "NULL vector");
    const size_t s = fp == 64 ? 8 : 4;
    const uintptr_t xa = (uintptr_t)d_x, ya = (uintptr_t)d_y;
    if ((xa | ya) % s) return set_error(GBR_EINVAL, "vectors must be aligned to their element size");
    const uintptr_t bytes = (uintptr_t)S->n * s;
    if (xa < ya + bytes && ya < xa + bytes) return set_error(GBR_EINVAL, "x and y overlap");
    cudaStream_t st = (cudaStream_t)stream;
    if (S->trie->wide) {
        if (fp == 64) return launch_set_hv<double, uint64_t>(S, (const double *)d_x, (double *)d_y, check, st);
        return launch_set_hv<float, uint64_t>(S, (const float *)d_x, (float *)d_y, check, st);
    }
    if (fp == 64) return launch_set_hv<double, uint32_t>(S, (const double *)d_x, (double *)d_y, check, st);
    return launch_set_hv<float, uint32_t>(S, (const float *)d_x, (float *)d_y, check, st);
}
