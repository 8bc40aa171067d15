/*
 * ORACLE -- test infrastructure only, never part of the product path.
 *
 * Plain, slow, obviously-correct CPU reference for the quantities the GPU
 * library computes (Wallerberger & Held, "Trie-based ranking of quantum
 * many-body states").  Only tests, the smoke check and the benchmark's CPU
 * baseline may call it.  It shares no code with the CUDA library: it keeps
 * its own binomials, its own enumeration, its own operator algebra.
 *
 * Conventions (the ones the GPU library also documents):
 *   * L sites per spin, spin-orbital bit p for (site p, down) and L+p for
 *     (site p, up): least significant bits are spin down (Sec. IV, text
 *     around Eq. rankupdown).
 *   * A sector (N_up, N_dn) is ordered by increasing numeric value of the
 *     2L-bit pattern, i.e. lexicographically (Sec. II, text after Eq. HNcomm;
 *     Sec. III, Eq. comb).  Its index is r_up * D_dn + r_dn (the spin-factored
 *     rank of Eq. rankupdown with the multiplier read as D_dn = C(L, N_dn)).
 *   * H = sum_{sigma} sum_{p,q} h[p][q] c^dag_{p sigma} c_{q sigma}
 *         + sum_p U[p] c^dag_{p up} c^dag_{p dn} c_{p dn} c_{p up}
 *     (Eq. H with t = -h restricted to one-body terms plus on-site U,
 *     Eq. Hring for the U term).
 *
 * Every function names the passage it follows.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- binomials */

/* Binomial coefficient C(n, k) from its product definition, exact for
 * n <= 64 (128-bit intermediate).  C(n, k) = 0 for k > n or k < 0, as in the
 * convention stated after Eq. cns. */
uint64_t ora_binom(int n, int k) {
    if (k < 0 || n < 0 || k > n) return 0;
    unsigned __int128 r = 1;
    for (int i = 1; i <= k; ++i) r = r * (unsigned)(n - k + i) / (unsigned)i;
    return (uint64_t)r;
}

/* number of set bits (Hamming weight h of the paper), clearing the lowest
 * set bit until none is left */
static int ora_popcount(uint64_t x) {
    int c = 0;
    while (x) { x &= x - 1; ++c; }
    return c;
}

/* ------------------------------------------------------------- enumeration */

/* All M-bit patterns with exactly N set bits, in increasing numeric order
 * (the set C^M_N of Eq. comb in lexicographic order).  Brute force over all
 * 2^M patterns, so only for M <= 32.  Returns the count, writing at most cap
 * entries (out may be NULL to count only). */
int64_t ora_enumerate(int M, int N, uint64_t *out, int64_t cap) {
    if (M < 0 || M > 32) return -1;
    int64_t n = 0;
    uint64_t end = (uint64_t)1 << M;
    for (uint64_t a = 0; a < end; ++a) {
        if (ora_popcount(a) != N) continue;
        if (out && n < cap) out[n] = a;
        ++n;
    }
    return n;
}

/* ------------------------------------------------------------------ ranking */

/* Rank by bisection in a sorted list (the established method of Sec. II,
 * last paragraph, and Sec. V-A): the position of alpha in the list, or -1
 * when alpha is not a member. */
int64_t ora_rank_bisect(const uint64_t *list, int64_t n, uint64_t alpha) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (list[mid] < alpha) lo = mid + 1; else hi = mid;
    }
    if (lo < n && list[lo] == alpha) return lo;
    return -1;
}

/* Rank of an N-bit pattern in C^M_N by counting the members below it
 * (Eq. cns and the counting argument after it): scanning alpha from its most
 * significant bit, at a set bit p that is the j-th set bit counted from the
 * bottom, every pattern that agrees with alpha above p, has 0 at p and j set
 * bits below p precedes alpha; there are C(p, j) of them. */
uint64_t ora_rank_count(int M, uint64_t alpha) {
    int j = ora_popcount(alpha);
    uint64_t r = 0;
    for (int p = M - 1; p >= 0; --p) {
        if ((alpha >> p) & 1u) {
            r += ora_binom(p, j);
            --j;
        }
    }
    return r;
}

/* Unrank in C^M_N (Eq. unrank): greedy decomposition of i in the
 * combinatorial number system, from the largest binomial down: the k-th set
 * bit (k = N..1) sits at the largest c with C(c, k) <= remaining rank. */
uint64_t ora_unrank_greedy(int M, int N, uint64_t i) {
    uint64_t a = 0;
    int c = M - 1;
    for (int k = N; k >= 1; --k) {
        while (c >= 0 && ora_binom(c, k) > i) --c;
        if (c < 0) return ~(uint64_t)0;
        a |= (uint64_t)1 << c;
        i -= ora_binom(c, k);
        --c;
    }
    return a;
}

/* -------------------------------------------------------------- packed trie */
/*
 * Linearised, packed trie of Sec. IV (Fig. trie (b), (c), Fig. trielookup):
 *   * chunks of R bits are dispatched from the least significant end; the
 *     first dispatched (root) chunk has width M mod R (or R when R divides
 *     M), every later chunk R bits -- the reading under which the overhead
 *     factors printed in Sec. V-A come out exactly;
 *   * the root is stored in full; every other node stores only the span from
 *     its smallest to its largest present child, and the parent entry holds
 *     (start of span) - (smallest child), so that t[k + r] is the child r;
 *   * nodes are laid out depth first, parent before children, children in
 *     increasing chunk value (the layout of the worked example of Sec. IV:
 *     root at 0..3, node 00 at 4..7, node 0000 at 8, node 0100 at 9..10);
 *   * a leaf entry holds the rank (the position in the numerically sorted
 *     member list).
 */

typedef struct {
    int M, R, H;
    int width[64];
    int shift[64];
} ora_trie_shape;

static void ora_trie_shape_init(ora_trie_shape *s, int M, int R) {
    s->M = M; s->R = R;
    int w0 = M % R ? M % R : R;
    int H = 1 + (M - w0) / R;
    s->H = H;
    int sh = 0;
    for (int d = 0; d < H; ++d) {
        s->width[d] = d == 0 ? w0 : R;
        s->shift[d] = sh;
        sh += s->width[d];
    }
}

static uint64_t ora_chunk(const ora_trie_shape *s, uint64_t a, int d) {
    return (a >> s->shift[d]) & ((((uint64_t)1) << s->width[d]) - 1);
}

/* key whose numeric order groups members by their dispatched prefix: the
 * first dispatched chunk becomes the most significant */
static uint64_t ora_dispatch_key(const ora_trie_shape *s, uint64_t a) {
    uint64_t k = 0;
    for (int d = 0; d < s->H; ++d) k = (k << s->width[d]) | ora_chunk(s, a, d);
    return k;
}

typedef struct { uint64_t key; int64_t rank; } ora_kr;

static int ora_kr_cmp(const void *x, const void *y) {
    const ora_kr *a = (const ora_kr *)x, *b = (const ora_kr *)y;
    return (a->key > b->key) - (a->key < b->key);
}

typedef struct {
    const ora_trie_shape *s;
    const ora_kr *kr;
    int64_t *t;        /* may be NULL: size only */
    int64_t pos;       /* next free element */
} ora_trie_ctx;

/* chunk d of a member, read back from its dispatch key */
static uint64_t ora_key_chunk(const ora_trie_shape *s, uint64_t key, int d) {
    int below = 0;
    for (int e = d + 1; e < s->H; ++e) below += s->width[e];
    return (key >> below) & ((((uint64_t)1) << s->width[d]) - 1);
}

/* lays out the node of depth d holding members [lo, hi) (which share their
 * first d chunks); returns the value to store in the parent's slot */
static int64_t ora_trie_node(ora_trie_ctx *c, int64_t lo, int64_t hi, int d) {
    const ora_trie_shape *s = c->s;
    uint64_t cmin = ora_key_chunk(s, c->kr[lo].key, d);
    uint64_t cmax = ora_key_chunk(s, c->kr[hi - 1].key, d);
    if (d == 0) { cmin = 0; cmax = (((uint64_t)1) << s->width[0]) - 1; }
    int64_t start = c->pos;
    c->pos += (int64_t)(cmax - cmin + 1);
    if (c->t)
        for (int64_t e = start; e < c->pos; ++e) c->t[e] = 0;
    int64_t i = lo;
    while (i < hi) {
        uint64_t ch = ora_key_chunk(s, c->kr[i].key, d);
        int64_t j = i;
        while (j < hi && ora_key_chunk(s, c->kr[j].key, d) == ch) ++j;
        int64_t v;
        if (d == s->H - 1) v = c->kr[i].rank;     /* leaf: the rank */
        else v = ora_trie_node(c, i, j, d + 1);   /* branch: child offset */
        if (c->t) c->t[start + (int64_t)(ch - cmin)] = v;
        i = j;
    }
    return start - (int64_t)cmin;
}

/* Builds the packed trie of the n sorted, distinct M-bit patterns.  Returns
 * the number of elements of t (without trailing padding) and writes them to
 * t when t is non-NULL and cap is large enough; -1 on bad input. */
int64_t ora_trie_build(const uint64_t *sorted, int64_t n, int M, int R, int64_t *t, int64_t cap) {
    if (n <= 0 || M < 1 || M > 64 || R < 1 || R > 24) return -1;
    ora_trie_shape s;
    ora_trie_shape_init(&s, M, R);
    ora_kr *kr = (ora_kr *)malloc(sizeof(ora_kr) * (size_t)n);
    if (!kr) return -1;
    for (int64_t i = 0; i < n; ++i) {
        kr[i].key = ora_dispatch_key(&s, sorted[i]);
        kr[i].rank = i;
    }
    qsort(kr, (size_t)n, sizeof(ora_kr), ora_kr_cmp);
    ora_trie_ctx c = {&s, kr, NULL, 0};
    ora_trie_node(&c, 0, n, 0);        /* first pass: size */
    int64_t size = c.pos;
    if (t && cap >= size) {
        c.t = t; c.pos = 0;
        ora_trie_node(&c, 0, n, 0);
    }
    free(kr);
    return size;
}

/* Fig. trielookup: k = 0; for every chunk but the last, k = t[k + chunk];
 * the rank is t[k + last chunk].  Out-of-range indices (possible only for
 * non-members) return -1. */
int64_t ora_trie_rank(const int64_t *t, int64_t size, int M, int R, uint64_t alpha) {
    ora_trie_shape s;
    ora_trie_shape_init(&s, M, R);
    int64_t k = 0;
    for (int d = 0; d < s.H; ++d) {
        int64_t idx = k + (int64_t)ora_chunk(&s, alpha, d);
        if (idx < 0 || idx >= size) return -1;
        k = t[idx];
    }
    return k;
}

/* ------------------------------------------------- fermionic operators */

/* Annihilator c_j on an occupation-number state (Eq. cee): zero unless bit j
 * is set; otherwise clears it, with sign (-1)^(number of set bits below j).
 * Returns the sign (+1/-1) or 0. */
static int ora_c(uint64_t *a, int j) {
    if (!((*a >> j) & 1u)) return 0;
    int sgn = 1;
    for (int b = 0; b < j; ++b)
        if ((*a >> b) & 1u) sgn = -sgn;
    *a &= ~((uint64_t)1 << j);
    return sgn;
}

/* Creator c^dag_j, the Hermitian conjugate of Eq. cee: zero if bit j is set;
 * otherwise sets it, with the same sign string over the bits below j. */
static int ora_cdag(uint64_t *a, int j) {
    if ((*a >> j) & 1u) return 0;
    int sgn = 1;
    for (int b = 0; b < j; ++b)
        if ((*a >> b) & 1u) sgn = -sgn;
    *a |= (uint64_t)1 << j;
    return sgn;
}

/* ------------------------------------------------------------ the sector */

typedef struct {
    int L, Nup, Ndn;
    int64_t Dup, Ddn;
    uint64_t *Sup, *Sdn;   /* per-spin sorted L-bit patterns */
} ora_sector;

static int ora_sector_init(ora_sector *s, int L, int Nup, int Ndn) {
    if (L < 1 || L > 30 || Nup < 0 || Nup > L || Ndn < 0 || Ndn > L) return -1;
    s->L = L; s->Nup = Nup; s->Ndn = Ndn;
    s->Dup = ora_enumerate(L, Nup, NULL, 0);
    s->Ddn = ora_enumerate(L, Ndn, NULL, 0);
    s->Sup = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)s->Dup);
    s->Sdn = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)s->Ddn);
    if (!s->Sup || !s->Sdn) return -1;
    ora_enumerate(L, Nup, s->Sup, s->Dup);
    ora_enumerate(L, Ndn, s->Sdn, s->Ddn);
    return 0;
}

static void ora_sector_free(ora_sector *s) { free(s->Sup); free(s->Sdn); }

/* full 2L-bit pattern of sector index i (spin-down in the low L bits) */
static uint64_t ora_sector_state(const ora_sector *s, int64_t i) {
    int64_t ru = i / s->Ddn, rd = i % s->Ddn;
    return s->Sdn[rd] | (s->Sup[ru] << s->L);
}

/* sector index of a 2L-bit pattern: r_up * D_dn + r_dn, each per-spin rank by
 * bisection in the per-spin list; -1 if the pattern is not in the sector */
static int64_t ora_sector_rank(const ora_sector *s, uint64_t alpha) {
    uint64_t lo = alpha & ((((uint64_t)1) << s->L) - 1);
    uint64_t hi = alpha >> s->L;
    int64_t rd = ora_rank_bisect(s->Sdn, s->Ddn, lo);
    int64_t ru = ora_rank_bisect(s->Sup, s->Dup, hi);
    if (rd < 0 || ru < 0) return -1;
    return ru * s->Ddn + rd;
}

int64_t ora_sector_dim(int L, int Nup, int Ndn) {
    return (int64_t)ora_binom(L, Nup) * (int64_t)ora_binom(L, Ndn);
}

/* Sector states in index order (for tests of the index convention). */
int ora_sector_states(int L, int Nup, int Ndn, uint64_t *out) {
    ora_sector s;
    if (ora_sector_init(&s, L, Nup, Ndn)) return -1;
    for (int64_t i = 0; i < s.Dup * s.Ddn; ++i) out[i] = ora_sector_state(&s, i);
    ora_sector_free(&s);
    return 0;
}

int64_t ora_sector_rank_of(int L, int Nup, int Ndn, uint64_t alpha) {
    ora_sector s;
    if (ora_sector_init(&s, L, Nup, Ndn)) return -2;
    int64_t r = ora_sector_rank(&s, alpha);
    ora_sector_free(&s);
    return r;
}

/* ------------------------------------------------------------ H applied */
/*
 * Applies every term of H to the basis state alpha (literal operator
 * products, Eq. cee for each factor, rightmost factor first) and calls back
 * with (coefficient * sign, resulting pattern).  Terms:
 *   h[p][q] c^dag_{p s} c_{q s}           for both spins s, all p, q;
 *   U[p] c^dag_{p up} c^dag_{p dn} c_{p dn} c_{p up}   (Eq. Hring).
 */
typedef void (*ora_term_cb)(void *ctx, double coef, uint64_t beta);

static void ora_apply_H(int L, const double *h, const double *U, uint64_t alpha, ora_term_cb cb, void *ctx) {
    for (int spin = 0; spin < 2; ++spin) {
        int off = spin ? L : 0;
        for (int p = 0; p < L; ++p) {
            for (int q = 0; q < L; ++q) {
                double v = h[p * L + q];
                if (v == 0.0) continue;
                uint64_t b = alpha;
                int s1 = ora_c(&b, q + off);
                if (!s1) continue;
                int s2 = ora_cdag(&b, p + off);
                if (!s2) continue;
                cb(ctx, v * s1 * s2, b);
            }
        }
    }
    for (int p = 0; p < L; ++p) {
        double v = U ? U[p] : 0.0;
        if (v == 0.0) continue;
        uint64_t b = alpha;
        int s = ora_c(&b, p + L);
        if (!s) continue;
        int t2 = ora_c(&b, p); if (!t2) continue; s *= t2;
        t2 = ora_cdag(&b, p); if (!t2) continue; s *= t2;
        t2 = ora_cdag(&b, p + L); if (!t2) continue; s *= t2;
        cb(ctx, v * s, b);
    }
}

typedef struct {
    const ora_sector *s;
    const double *x;
    double *y;
    double xj;
    double acc;
    int64_t count;
    int bad;
} ora_hv_ctx;

/* scatter form: column j contributes coef * x_j to row rank(T alpha_j) */
static void ora_cb_scatter(void *vctx, double coef, uint64_t beta) {
    ora_hv_ctx *c = (ora_hv_ctx *)vctx;
    int64_t i = ora_sector_rank(c->s, beta);
    if (i < 0) { c->bad = 1; return; }
    c->y[i] += coef * c->xj;
}

/* Full y = H x over the sector (Eq. mvblock): for every column j, apply every
 * term to alpha_j and scatter.  Returns 0, or -1 if a term left the sector
 * (impossible for a number-conserving H; reported rather than ignored). */
int ora_hv_full(int L, const double *h, const double *U, int Nup, int Ndn, const double *x, double *y) {
    ora_sector s;
    if (ora_sector_init(&s, L, Nup, Ndn)) return -2;
    int64_t D = s.Dup * s.Ddn;
    for (int64_t i = 0; i < D; ++i) y[i] = 0.0;
    ora_hv_ctx c = {&s, x, y, 0.0, 0.0, 0, 0};
    for (int64_t j = 0; j < D; ++j) {
        c.xj = x[j];
        ora_apply_H(L, h, U, ora_sector_state(&s, j), ora_cb_scatter, &c);
    }
    ora_sector_free(&s);
    return c.bad ? -1 : 0;
}

static void ora_cb_gather(void *vctx, double coef, uint64_t beta) {
    ora_hv_ctx *c = (ora_hv_ctx *)vctx;
    int64_t j = ora_sector_rank(c->s, beta);
    if (j < 0) { c->bad = 1; return; }
    c->acc += coef * c->x[j];
    c->count += 1;
}

/* Selected rows of y = H x: y_i = sum_j H_ij x_j = sum_j H_ji x_j, valid
 * because H is real symmetric whenever h is; each term is applied to
 * alpha_i and the coefficient gathers x at the rank of the result.  Used for
 * sampled checks at sizes where the full product is out of reach. */
int ora_hv_rows(int L, const double *h, const double *U, int Nup, int Ndn, const double *x,
                const int64_t *rows, int64_t nrows, double *y_out) {
    ora_sector s;
    if (ora_sector_init(&s, L, Nup, Ndn)) return -2;
    ora_hv_ctx c = {&s, x, NULL, 0.0, 0.0, 0, 0};
    for (int64_t k = 0; k < nrows; ++k) {
        c.acc = 0.0;
        ora_apply_H(L, h, U, ora_sector_state(&s, rows[k]), ora_cb_gather, &c);
        y_out[k] = c.acc;
    }
    ora_sector_free(&s);
    return c.bad ? -1 : 0;
}

/* The seeded input generator, written here from its published definition
 * (splitmix64 of Steele, Lea and Flood, counter mode
 * u(seed, i) = splitmix64(seed XOR i*0x9E3779B97F4A7C15)), so that sampled
 * rows of very large sectors can read x_j = uniform[-1, 1)(seed, j) on demand
 * without materialising x. */
static uint64_t ora_splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double ora_seeded_uniform(uint64_t seed, uint64_t i) {
    uint64_t u = ora_splitmix64(seed ^ (i * 0x9E3779B97F4A7C15ull));
    return 2.0 * ((double)(u >> 11) * 0x1.0p-53) - 1.0;
}

typedef struct {
    const ora_sector *s;
    uint64_t seed;
    double acc;
    int bad;
} ora_seed_ctx;

static void ora_cb_gather_seeded(void *vctx, double coef, uint64_t beta) {
    ora_seed_ctx *c = (ora_seed_ctx *)vctx;
    int64_t j = ora_sector_rank(c->s, beta);
    if (j < 0) { c->bad = 1; return; }
    c->acc += coef * ora_seeded_uniform(c->seed, (uint64_t)j);
}

/* Selected rows of y = H x for x_j = uniform[-1, 1)(seed, j); same gather
 * form as ora_hv_rows. */
int ora_hv_rows_seeded(int L, const double *h, const double *U, int Nup, int Ndn, uint64_t seed,
                       const int64_t *rows, int64_t nrows, double *y_out) {
    ora_sector s;
    if (ora_sector_init(&s, L, Nup, Ndn)) return -2;
    ora_seed_ctx c = {&s, seed, 0.0, 0};
    for (int64_t k = 0; k < nrows; ++k) {
        c.acc = 0.0;
        ora_apply_H(L, h, U, ora_sector_state(&s, rows[k]), ora_cb_gather_seeded, &c);
        y_out[k] = c.acc;
    }
    ora_sector_free(&s);
    return c.bad ? -1 : 0;
}

/* y = P H P x over an arbitrary sorted set of 2L-bit states (Sec. IV: sets
 * defined by further quantum numbers, ranked through a search structure):
 * every term is applied literally to every member; the coefficient is
 * scattered to the rank of the result, found by bisection in the set.
 * Results outside the set are dropped (the set's projection of H; for a
 * set closed under H nothing is dropped) and counted in *dropped. */
int ora_hv_set(int L, const double *h, const double *U, const uint64_t *states, int64_t n, const double *x,
               double *y, int64_t *dropped) {
    typedef struct { const uint64_t *st; int64_t n; double *y; double xj; int64_t drop; } set_ctx;
    for (int64_t i = 0; i < n; ++i) y[i] = 0.0;
    int64_t drop = 0;
    for (int64_t j = 0; j < n; ++j) {
        /* apply every term to member j (same literal operator products as
         * ora_apply_H, written out here for the set's own ranking) */
        uint64_t alpha = states[j];
        for (int spin = 0; spin < 2; ++spin) {
            int off = spin ? L : 0;
            for (int p = 0; p < L; ++p)
                for (int q = 0; q < L; ++q) {
                    double v = h[p * L + q];
                    if (v == 0.0) continue;
                    uint64_t b = alpha;
                    int s1 = ora_c(&b, q + off);
                    if (!s1) continue;
                    int s2 = ora_cdag(&b, p + off);
                    if (!s2) continue;
                    int64_t i = ora_rank_bisect(states, n, b);
                    if (i < 0) { ++drop; continue; }
                    y[i] += v * s1 * s2 * x[j];
                }
        }
        for (int p = 0; p < L; ++p) {
            double v = U ? U[p] : 0.0;
            if (v == 0.0) continue;
            uint64_t b = alpha;
            int s = ora_c(&b, p + L);
            if (!s) continue;
            int t2 = ora_c(&b, p); if (!t2) continue; s *= t2;
            t2 = ora_cdag(&b, p); if (!t2) continue; s *= t2;
            t2 = ora_cdag(&b, p + L); if (!t2) continue; s *= t2;
            int64_t i = ora_rank_bisect(states, n, b);
            if (i < 0) { ++drop; continue; }
            y[i] += v * s * x[j];
        }
    }
    if (dropped) *dropped = drop;
    return 0;
}

/* y = P H P x on a sorted set for H given as a list of operator products
 * (Eq. H in general form).  Term t has coefficient coef[t] and nops[t]
 * operators starting at ops[off[t]], written left to right as in the
 * product; operator code = 2*orbital + (1 for a creator, 0 for an
 * annihilator).  Each product is applied literally to each member, rightmost
 * operator first, by Eq. cee; results outside the set are dropped and
 * counted. */
int ora_hv_ops(const double *coef, const int *nops, const int *off, const int *ops, int nterms,
               const uint64_t *states, int64_t n, const double *x, double *y, int64_t *dropped) {
    for (int64_t i = 0; i < n; ++i) y[i] = 0.0;
    int64_t drop = 0;
    for (int64_t j = 0; j < n; ++j) {
        for (int t = 0; t < nterms; ++t) {
            uint64_t b = states[j];
            int sgn = 1;
            for (int o = nops[t] - 1; o >= 0 && sgn; --o) {
                const int code = ops[off[t] + o];
                const int orb = code >> 1;
                sgn *= (code & 1) ? ora_cdag(&b, orb) : ora_c(&b, orb);
            }
            if (!sgn) continue;
            int64_t i = ora_rank_bisect(states, n, b);
            if (i < 0) { ++drop; continue; }
            y[i] += coef[t] * sgn * x[j];
        }
    }
    if (dropped) *dropped = drop;
    return 0;
}

/* Literal application of one operator product to one state: returns the sign
 * (0 if the product annihilates the state) and the resulting pattern. */
int ora_apply_ops(const int *ops, int nops, uint64_t alpha, uint64_t *beta) {
    uint64_t b = alpha;
    int sgn = 1;
    for (int o = nops - 1; o >= 0 && sgn; --o) {
        const int code = ops[o];
        sgn *= (code & 1) ? ora_cdag(&b, code >> 1) : ora_c(&b, code >> 1);
    }
    *beta = b;
    return sgn;
}

/* Number of matrix elements one H x visits: the D diagonal entries plus every
 * off-diagonal (state, hop) pair that is non-zero.  Counted by applying the
 * off-diagonal hopping terms literally to every state; for rows only in
 * [row0, row1) when row1 > row0 (sampled counts). */
int64_t ora_count_elements(int L, const double *h, int Nup, int Ndn, int64_t row0, int64_t row1) {
    ora_sector s;
    if (ora_sector_init(&s, L, Nup, Ndn)) return -2;
    int64_t D = s.Dup * s.Ddn;
    if (row1 <= row0) { row0 = 0; row1 = D; }
    int64_t n = row1 - row0;
    for (int64_t i = row0; i < row1; ++i) {
        uint64_t a = ora_sector_state(&s, i);
        for (int spin = 0; spin < 2; ++spin) {
            int off = spin ? L : 0;
            for (int p = 0; p < L; ++p)
                for (int q = 0; q < L; ++q) {
                    if (p == q || h[p * L + q] == 0.0) continue;
                    uint64_t b = a;
                    if (!ora_c(&b, q + off)) continue;
                    if (!ora_cdag(&b, p + off)) continue;
                    ++n;
                }
        }
    }
    ora_sector_free(&s);
    return n;
}

/* Dense sector matrix (row-major D x D) by applying H to every basis state
 * (column j of H is H|alpha_j>). */
int ora_dense(int L, const double *h, const double *U, int Nup, int Ndn, double *Hm) {
    ora_sector s;
    if (ora_sector_init(&s, L, Nup, Ndn)) return -2;
    int64_t D = s.Dup * s.Ddn;
    double *col = (double *)malloc(sizeof(double) * (size_t)D);
    double *e = (double *)calloc((size_t)D, sizeof(double));
    int rc = 0;
    for (int64_t j = 0; j < D && !rc; ++j) {
        for (int64_t i = 0; i < D; ++i) col[i] = 0.0;
        ora_hv_ctx c = {&s, e, col, 1.0, 0.0, 0, 0};
        ora_apply_H(L, h, U, ora_sector_state(&s, j), ora_cb_scatter, &c);
        if (c.bad) rc = -1;
        for (int64_t i = 0; i < D; ++i) Hm[i * D + j] = col[i];
    }
    free(col); free(e);
    ora_sector_free(&s);
    return rc;
}

/* ---------------------------------------------------- tridiagonal eigen */

/* Number of eigenvalues of the symmetric tridiagonal T (diagonal a[0..k-1],
 * off-diagonal b[0..k-2]) below x: the count of negative pivots of the
 * LDL^T factorisation of T - x (Sturm sequence). */
static int ora_sturm_count(const double *a, const double *b, int k, double x) {
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < k; ++i) {
        double bb = i ? b[i - 1] * b[i - 1] : 0.0;
        q = (a[i] - x) - (i ? bb / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

/* Lowest eigenvalue of T by bisection on the Sturm count, started from the
 * Gershgorin interval and run until the interval cannot shrink further. */
double ora_tridiag_lowest(const double *a, const double *b, int k) {
    double lo = a[0], hi = a[0];
    for (int i = 0; i < k; ++i) {
        double r = (i ? fabs(b[i - 1]) : 0.0) + (i < k - 1 ? fabs(b[i]) : 0.0);
        if (a[i] - r < lo) lo = a[i] - r;
        if (a[i] + r > hi) hi = a[i] + r;
    }
    for (int it = 0; it < 2000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (ora_sturm_count(a, b, k, mid) >= 1) hi = mid; else lo = mid;
    }
    return hi;
}

/* --------------------------------------------------------------- Lanczos */
/*
 * Plain FP64 Lanczos (the paper cites the method without stating it; this
 * is the textbook three-term recurrence):
 *   v_0 = s/|s|;  for k = 0, 1, ...:
 *     w = H v_k - beta_k v_{k-1};  alpha_k = <w, v_k>;  w -= alpha_k v_k;
 *     optional full re-orthogonalisation: two passes of classical
 *       Gram-Schmidt against v_0..v_k (coefficients not folded into T);
 *     beta_{k+1} = |w|;  stop if beta_{k+1} <= 1e-13 max_j(|alpha_j|, beta_j);
 *     v_{k+1} = w / beta_{k+1}.
 *   E0 = lowest eigenvalue of T (Sturm bisection).
 * Outputs alpha[0..k-1], beta[0..k-2] (beta_1..beta_{k-1}), the number of
 * steps k, E0, and (if eritz != NULL) the lowest Ritz value after every step.
 */
int ora_lanczos(int L, const double *h, const double *U, int Nup, int Ndn, const double *s0, int iters, int reorth,
                double *alpha, double *beta, int *k_out, double *E0, double *eritz) {
    int64_t D = ora_sector_dim(L, Nup, Ndn);
    if (D <= 0 || iters < 1) return -2;
    int nvec = reorth ? iters + 1 : 2;
    double *V = (double *)malloc(sizeof(double) * (size_t)D * (size_t)nvec);
    double *w = (double *)malloc(sizeof(double) * (size_t)D);
    double *c = (double *)malloc(sizeof(double) * (size_t)(iters + 1));
    double *bfull = (double *)calloc((size_t)(iters + 2), sizeof(double));
    if (!V || !w || !c || !bfull) return -3;
    double nrm = 0.0;
    for (int64_t i = 0; i < D; ++i) nrm += s0[i] * s0[i];
    nrm = sqrt(nrm);
    for (int64_t i = 0; i < D; ++i) V[i] = s0[i] / nrm;
    double scale = 0.0;
    int k = 0, rc = 0;
    for (k = 0; k < iters; ++k) {
        double *vk = V + (size_t)D * (size_t)(reorth ? k : (k & 1));
        double *vprev = V + (size_t)D * (size_t)(reorth ? (k ? k - 1 : 0) : ((k + 1) & 1));
        if (ora_hv_full(L, h, U, Nup, Ndn, vk, w)) { rc = -1; break; }
        if (k > 0)
            for (int64_t i = 0; i < D; ++i) w[i] -= bfull[k] * vprev[i];
        double a = 0.0;
        for (int64_t i = 0; i < D; ++i) a += w[i] * vk[i];
        alpha[k] = a;
        for (int64_t i = 0; i < D; ++i) w[i] -= a * vk[i];
        if (reorth) {
            for (int pass = 0; pass < 2; ++pass) {
                for (int j = 0; j <= k; ++j) {
                    double d = 0.0;
                    const double *vj = V + (size_t)D * (size_t)j;
                    for (int64_t i = 0; i < D; ++i) d += w[i] * vj[i];
                    c[j] = d;
                }
                for (int j = 0; j <= k; ++j) {
                    const double *vj = V + (size_t)D * (size_t)j;
                    for (int64_t i = 0; i < D; ++i) w[i] -= c[j] * vj[i];
                }
            }
        }
        double b = 0.0;
        for (int64_t i = 0; i < D; ++i) b += w[i] * w[i];
        b = sqrt(b);
        if (fabs(a) > scale) scale = fabs(a);
        if (eritz) eritz[k] = ora_tridiag_lowest(alpha, bfull + 1, k + 1);
        if (k + 1 == iters) { ++k; break; }
        if (b <= 1e-13 * (b > scale ? b : scale)) { ++k; break; }
        if (b > scale) scale = b;
        bfull[k + 1] = b;
        double *vn = V + (size_t)D * (size_t)(reorth ? k + 1 : ((k + 1) & 1));
        for (int64_t i = 0; i < D; ++i) vn[i] = w[i] / b;
    }
    *k_out = k;
    for (int j = 0; j + 1 < k; ++j) beta[j] = bfull[j + 1];
    *E0 = ora_tridiag_lowest(alpha, bfull + 1, k);
    free(V); free(w); free(c); free(bfull);
    return rc;
}
