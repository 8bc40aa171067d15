// General operator-product terms (Appendix: Eqs. Talpha1, Talpha2, ci and the
// product rule of Fig. mul) and an on-the-fly H·v over a trie-ranked state
// set for any list of such terms -- e.g. the O(M^3) two-body terms of the
// momentum-basis Hubbard ring (Sec. V-C, Eq. Hk) in a total-momentum sector.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ham.h"

namespace gbr {

// Building blocks, Eqs. ci: c_i has v = 1, m = r = x = 2^i, l = 0,
// s = 2^i - 1; the creator c^dag_i exchanges l and r.
static gbr_term block(int orbital, bool creator) {
    gbr_term t;
    const uint64_t b = 1ull << orbital;
    t.v = 1.0;
    t.m = b;
    t.x = b;
    t.s = b - 1;
    t.l = creator ? b : 0;
    t.r = creator ? 0 : b;
    return t;
}

// Product T = T_a T_b (Fig. mul): Pauli check on the shared orbitals, union
// of the masks, outer demands r (right) and l (left) with the inner factor
// taking precedence on its own mask, the change mask x = l xor r, the sign
// mask outside m, and the sign of the reordering found by applying both
// factors' sign masks along the way to the state |r>.
static gbr_term mul(const gbr_term &a, const gbr_term &b) {
    gbr_term t;
    t.v = (((a.r ^ b.l) & a.m & b.m) != 0) ? 0.0 : a.v * b.v;
    t.m = a.m | b.m;
    t.r = b.r | (a.r & ~b.m);
    t.l = a.l | (b.l & ~a.m);
    t.x = t.l ^ t.r;
    t.s = (a.s ^ b.s) & ~t.m;
    uint64_t z = t.r;
    uint64_t p = z & b.s;
    z ^= b.x;
    p ^= z & a.s;
    if (__builtin_popcountll(p) & 1) t.v = -t.v;
    return t;
}

struct TermK {
    int nterms;
    int H;
    int shift[kMaxChunks];
    int width[kMaxChunks];
    int64_t padded, smem_entries, n;
};

// One thread per member alpha: every term applied from the left
// (Eq. Talpha2): <alpha| T = v delta(alpha & m, l) (-1)^h(alpha & s) <alpha ^ x|,
// so y_i gathers v (-1)^... x_j at j = rank(alpha ^ x) -- the row of H, for
// any term list, Hermitian or not.  Ranks by the trie walk of Fig.
// trielookup; check = 1 drops targets outside the set.
template <typename T, typename E, bool BISECT>
__global__ void __launch_bounds__(256) k_term_hv(const TermK tk, const E *__restrict__ trie,
                                                 const uint64_t *__restrict__ states, const gbr_term *__restrict__ terms,
                                                 int check, const T *__restrict__ x, T *__restrict__ y) {
    extern __shared__ __align__(16) unsigned char smr[];
    E *ts = reinterpret_cast<E *>(smr);
    for (int64_t i = threadIdx.x; i < tk.smem_entries; i += blockDim.x) ts[i] = __ldg(trie + i);
    __syncthreads();
    const E last = (E)(tk.padded - 1), sm_end = (E)tk.smem_entries;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tk.n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t a = states[i];
        T acc = 0;
        for (int t = 0; t < tk.nterms; ++t) {
            const uint64_t m = __ldg(&terms[t].m), l = __ldg(&terms[t].l);
            if ((a & m) != l) continue;
            const uint64_t xm = __ldg(&terms[t].x);
            const T v = (T)__ldg(&terms[t].v);
            const T sv = (__popcll(a & __ldg(&terms[t].s)) & 1) ? -v : v;
            int64_t j = i;
            if (xm) {
                const uint64_t b = a ^ xm;
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
                    E kk = 0;
                    for (int lvl = 0; lvl < tk.H; ++lvl) {
                        E idx = kk + (E)((uint32_t)(b >> tk.shift[lvl]) & ((1u << tk.width[lvl]) - 1u));
                        idx = idx > last ? last : idx;
                        kk = idx < sm_end ? ts[idx] : __ldg(trie + idx);
                    }
                    k = (uint64_t)kk;
                }
                if ((check || BISECT) && !(k < (uint64_t)tk.n && __ldg(states + k) == b)) continue;
                j = (int64_t)k;
            }
            acc += sv * x[j];
        }
        y[i] = acc;
    }
}

}  // namespace gbr

using namespace gbr;

struct gbr_termham {
    int M = 0;
    int bisect = 0;     // 1: rank by bisection in the member list instead of the trie
    int64_t n = 0;
    int nterms = 0;
    int64_t elements = 0;
    gbr_trie *trie = nullptr;
    gbr::DevBuf terms;
    gbr::LzWork lzw;    // Lanczos work buffers
    ~gbr_termham() { gbr_trie_destroy(trie); }
};

extern "C" int gbr_term_mul(const gbr_term *a, const gbr_term *b, gbr_term *out) {
    clear_error();
    if (!a || !b || !out) return set_error(GBR_EINVAL, "NULL argument");
    *out = mul(*a, *b);
    return GBR_OK;
}

extern "C" int gbr_term_product(const int *ops, int nops, double coef, gbr_term *out) {
    clear_error();
    if (!out || (nops > 0 && !ops) || nops < 0) return set_error(GBR_EINVAL, "bad operator list");
    gbr_term t;
    t.v = coef;
    t.m = t.l = t.r = t.x = t.s = 0;
    for (int o = 0; o < nops; ++o) {
        const int code = ops[o];
        if (code < 0 || (code >> 1) >= 64) return set_error(GBR_EINVAL, "operator code %d out of range", code);
        t = mul(t, block(code >> 1, code & 1));
    }
    *out = t;
    return GBR_OK;
}

extern "C" int gbr_termham_create(int M, const gbr_term *h_terms, int nterms, const uint64_t *h_states, int64_t n,
                                  int R, gbr_termham **out) {
    clear_error();
    if (!out) return set_error(GBR_EINVAL, "out is NULL");
    *out = nullptr;
    if (M < 1 || M > 64) return set_error(GBR_EINVAL, "M=%d out of range 1..64", M);
    if (nterms < 1 || !h_terms) return set_error(GBR_EINVAL, "empty term list");
    const uint64_t all = M == 64 ? ~0ull : ((1ull << M) - 1);
    for (int t = 0; t < nterms; ++t) {
        if ((h_terms[t].m | h_terms[t].l | h_terms[t].r | h_terms[t].x | h_terms[t].s) & ~all)
            return set_error(GBR_EINVAL, "term %d touches orbitals at or above M", t);
        if (!std::isfinite(h_terms[t].v)) return set_error(GBR_EINVAL, "term %d has a non-finite coefficient", t);
    }
    gbr_termham *T = new (std::nothrow) gbr_termham();
    if (!T) return set_error(GBR_ENOMEM, "host allocation failed");
    T->M = M;
    T->n = n;
    T->nterms = nterms;
    // most significant chunk first: neighbouring members share their walks
    int rc = gbr_trie_create_ordered(h_states, n, M, R, 1, &T->trie);
    if (!rc) {
        // matrix elements: every (member, term) pair whose left demand holds
        int64_t el = 0;
        for (int64_t i = 0; i < n; ++i)
            for (int t = 0; t < nterms; ++t)
                if ((h_states[i] & h_terms[t].m) == h_terms[t].l && h_terms[t].v != 0.0) ++el;
        T->elements = el;
        rc = T->terms.upload(h_terms, sizeof(gbr_term) * (size_t)nterms);
    }
    if (rc) { delete T; return rc; }
    *out = T;
    return GBR_OK;
}

extern "C" void gbr_termham_destroy(gbr_termham *T) { delete T; }

extern "C" int gbr_termham_set_bisect(gbr_termham *T, int bisect) {
    clear_error();
    if (!T) return set_error(GBR_EINVAL, "NULL handle");
    T->bisect = bisect ? 1 : 0;
    return GBR_OK;
}

extern "C" int gbr_termham_info(const gbr_termham *T, int64_t *dim, int64_t *elements, int64_t *trie_elements) {
    clear_error();
    if (!T) return set_error(GBR_EINVAL, "NULL handle");
    if (dim) *dim = T->n;
    if (elements) *elements = T->elements;
    if (trie_elements) *trie_elements = T->trie->size;
    return GBR_OK;
}

namespace gbr {
template <typename T, typename E>
static int launch_term_hv(const gbr_termham *Th, const T *x, T *y, int check, cudaStream_t st) {
    const gbr_trie *tr = Th->trie;
    TermK tk;
    memset(&tk, 0, sizeof(tk));
    tk.nterms = Th->nterms;
    tk.H = tr->H;
    for (int l = 0; l < tr->H; ++l) { tk.shift[l] = tr->shift[l]; tk.width[l] = tr->width[l]; }
    tk.padded = tr->padded;
    tk.smem_entries = tr->smem_entries;
    tk.n = Th->n;
    const size_t smem = (size_t)tr->smem_entries * sizeof(E);
    int64_t blocks = (Th->n + 255) / 256;
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sm_count() * 8));
    auto kern = Th->bisect ? k_term_hv<T, E, true> : k_term_hv<T, E, false>;
    if (smem > 48 * 1024) GBR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(int)blocks, 256, smem, st>>>(tk, tr->t.as<E>(), tr->members.as<uint64_t>(), Th->terms.as<gbr_term>(), check, x,
                                         y);
    GBR_LAUNCH_CHECK();
    count_launches(1);
    return GBR_OK;
}
}  // namespace gbr

namespace gbr {
// y = H x over the set with membership checks (the Lanczos operator)
static int term_apply(const void *obj, const void *x, void *y, int fp, cudaStream_t st) {
    const gbr_termham *T = static_cast<const gbr_termham *>(obj);
    if (T->trie->wide) {
        if (fp == 64) return launch_term_hv<double, uint64_t>(T, (const double *)x, (double *)y, 1, st);
        return launch_term_hv<float, uint64_t>(T, (const float *)x, (float *)y, 1, st);
    }
    if (fp == 64) return launch_term_hv<double, uint32_t>(T, (const double *)x, (double *)y, 1, st);
    return launch_term_hv<float, uint32_t>(T, (const float *)x, (float *)y, 1, st);
}
}  // namespace gbr

extern "C" int gbr_termham_lanczos(const gbr_termham *T, const gbr_lanczos_opts *o, const double *d_v0,
                                   gbr_lanczos_result *res, double *h_alpha, double *h_beta, double *h_ritz,
                                   void *stream) {
    clear_error();
    if (!T) return set_error(GBR_EINVAL, "NULL handle");
    const LzOp op{nullptr, T, &term_apply, T->n, &const_cast<gbr_termham *>(T)->lzw};
    return lanczos_solve(op, o, d_v0, res, h_alpha, h_beta, h_ritz, stream);
}

extern "C" int gbr_termham_hv(const gbr_termham *T, const void *d_x, void *d_y, int fp, int check, void *stream) {
    clear_error();
    if (!T) return set_error(GBR_EINVAL, "NULL handle");
    if (fp != 32 && fp != 64) return set_error(GBR_EINVAL, "fp=%d must be 32 or 64", fp);
    if (!d_x || !d_y) return set_error(GBR_EINVAL, "NULL vector");
    const size_t s = fp == 64 ? 8 : 4;
    const uintptr_t xa = (uintptr_t)d_x, ya = (uintptr_t)d_y;
    if ((xa | ya) % s) return set_error(GBR_EINVAL, "vectors must be aligned to their element size");
    const uintptr_t bytes = (uintptr_t)T->n * s;
    if (xa < ya + bytes && ya < xa + bytes) return set_error(GBR_EINVAL, "x and y overlap");
    cudaStream_t st = (cudaStream_t)stream;
    if (T->trie->wide) {
        if (fp == 64) return launch_term_hv<double, uint64_t>(T, (const double *)d_x, (double *)d_y, check, st);
        return launch_term_hv<float, uint64_t>(T, (const float *)d_x, (float *)d_y, check, st);
    }
    if (fp == 64) return launch_term_hv<double, uint32_t>(T, (const double *)d_x, (double *)d_y, check, st);
    return launch_term_hv<float, uint32_t>(T, (const float *)d_x, (float *)d_y, check, st);
}
