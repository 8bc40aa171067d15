/*
 * gbrank -- GB300 (sm_103a) ranking, on-the-fly H·v and Lanczos for
 * quantum many-body states.
 *
 * C ABI of libgbrank.so.  Method: Wallerberger & Held, "Trie-based ranking
 * of quantum many-body states" (arXiv:2203.04158).  Every entry point cites
 * the passage that defines the operation.
 *
 * Conventions shared by all calls
 *   * Status: every call returns an int, GBR_OK (0) on success.  On failure
 *     the thread-local message is available from gbr_last_error().  No C++
 *     exception crosses the ABI.  Argument errors are detected on the host
 *     before anything is launched.
 *   * Handles (gbr_comb, gbr_trie, gbr_ham) are opaque, created and owned by
 *     the library, released with the matching *_destroy (NULL is accepted).
 *     Creation builds tables on the host and copies them to the current
 *     CUDA device synchronously; a handle is used on that device only.
 *   * Buffers named d_* are device pointers owned by the caller (any
 *     cudaMalloc'd or framework-allocated memory).  Buffers named h_* are
 *     host pointers owned by the caller.
 *   * stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that only launch work are asynchronous on that stream:
 *     results are valid after the stream synchronises.  Calls that return
 *     host results (gbr_lanczos, gbr_batch_solve) synchronise the stream.
 *   * Bit patterns: bit i of a uint64_t is spin-orbital i.  A sector of
 *     fixed particle number N in M spin-orbitals is ordered by increasing
 *     numeric value (lexicographic order, Sec. III, Eq. comb).
 *   * Two-spin sectors (Hubbard/impurity Hamiltonians) use L sites per spin,
 *     spin-orbital p = (site p, down) and L+p = (site p, up): least
 *     significant bits are spin down (Sec. IV, around Eq. rankupdown).  The
 *     sector index is r_up * C(L, N_dn) + r_dn (Eq. rankupdown with the
 *     multiplier read as the spin-down dimension, the only reading that is a
 *     bijection when N_up != N_dn).
 */
#ifndef GBRANK_H
#define GBRANK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GBR_OK = 0,
    GBR_EINVAL = 1,      /* bad argument (detected on the host) */
    GBR_ENOMEM = 2,      /* device or host allocation failed */
    GBR_ECUDA = 3,       /* a CUDA runtime call failed */
    GBR_ENOTFOUND = 4,   /* a queried pattern is not a member (check mode) */
    GBR_ETIMEOUT = 5,    /* a bounded device-side wait ran out */
    GBR_EBREAKDOWN = 6,  /* Lanczos stopped early on an invariant subspace */
    GBR_ENONFINITE = 7   /* a non-finite value (NaN or Inf) appeared in a Lanczos scalar */
};

/* Rank value written for a pattern that is not in the set (check mode) and
 * pattern value written for an out-of-range rank. */
#define GBR_NOT_FOUND_U32 0xFFFFFFFFu
#define GBR_NOT_FOUND_U64 0xFFFFFFFFFFFFFFFFull

/* Message of the last failed call on this thread ("" if none). */
const char *gbr_last_error(void);

/* ABI version, currently 1. */
int gbr_version(void);

/* ------------------------------------------------------------------------
 * Fixed-popcount sectors: staggered lookup (Sec. III-B, Fig. fastrank,
 * Eq. partrank) and combinadics unranking (Eq. unrank).
 * --------------------------------------------------------------------- */
typedef struct gbr_comb gbr_comb;

/* Builds the staggered tables rank(r, M', N') of Eq. partrank for the
 * sector C^M_N, chunk width R, restricted to the N' values admissible for N
 * (Sec. III-B, remarks after Eq. stagmem), with entries computed through
 * Eq. reuse from the combinadics ranking of Fig. algr.
 *   M: 1..64 spin-orbitals; N: 0..M particles; R: chunk width 1..12.
 * Entries are 32-bit when C(M, N) <= 2^32, else 64-bit.
 * Errors: GBR_EINVAL for out-of-range arguments, GBR_ENOMEM, GBR_ECUDA. */
int gbr_comb_create(int M, int N, int R, gbr_comb **out);
void gbr_comb_destroy(gbr_comb *c);

/* dim = C(M, N); table_bytes = size of the staggered tables on the device. */
int gbr_comb_info(const gbr_comb *c, uint64_t *dim, int64_t *table_bytes);

/* Ranks n patterns (Fig. fastrank): d_rank[i] = rank of d_pat[i] in C^M_N.
 *   d_pat:  n uint64 patterns (device).  16-byte alignment enables
 *           vectorised loads; any 8-byte aligned pointer is accepted.
 *   d_rank: n ranks (device), uint32 when rank_bits == 32 (requires
 *           C(M, N) <= 2^32) or uint64 when rank_bits == 64.
 *   check:  0 = trust the input (a pattern outside the sector gets an
 *           unspecified rank, but every table access stays in bounds);
 *           1 = patterns with bits at or above M or popcount != N get
 *           GBR_NOT_FOUND_U32 / _U64.
 * n == 0 is a no-op.  Asynchronous on stream. */
int gbr_comb_rank(const gbr_comb *c, const uint64_t *d_pat, void *d_rank, int rank_bits, int64_t n, int check,
                  void *stream);

/* Unranks n ranks (Eq. unrank): d_pat[i] = the d_rank[i]-th member of
 * C^M_N; ranks >= C(M, N) give GBR_NOT_FOUND_U64.  rank_bits 32 or 64. */
int gbr_comb_unrank(const gbr_comb *c, const void *d_rank, int rank_bits, uint64_t *d_pat, int64_t n, void *stream);

/* ------------------------------------------------------------------------
 * Packed tries over arbitrary sorted state sets (Sec. IV, Fig. trie,
 * Fig. trielookup).
 * --------------------------------------------------------------------- */
typedef struct gbr_trie gbr_trie;

/* Builds the linearised, packed trie of radix 2^R over n distinct M-bit
 * patterns given in strictly increasing order (host array, not retained).
 * Chunks are dispatched from the least significant bits; the first
 * dispatched chunk has width M mod R (or R when R divides M); the root is
 * stored in full and every other node as the span between its smallest and
 * largest child, the parent holding (start - smallest child) (Fig. trie (c)).
 * Nodes are stored level by level (breadth first) so that the upper levels
 * form one contiguous prefix.  2^R zero entries pad the end (Sec. IV, remark
 * on trailing elements).  Entries are 32-bit when the table and n fit, else
 * 64-bit.  A device copy of the member list is kept for unranking and for
 * the membership check.
 *   M: 1..64; R: 1..16; n >= 1.
 * Errors: GBR_EINVAL if the input is unsorted, has duplicates or a bit at
 * or above M; GBR_ENOMEM; GBR_ECUDA. */
int gbr_trie_create(const uint64_t *h_sorted, int64_t n, int M, int R, gbr_trie **out);

/* gbr_trie_create with a choice of dispatch order.  msb_first = 0 is the
 * paper's order above (Fig. trielookup).  msb_first = 1 dispatches the most
 * significant chunk first (width M mod R, or R, at the top, then R-bit chunks
 * down to bit 0); the paper has no counterpart: this is an interface of this
 * library.  Ranks are the same either way; with the most significant chunk
 * first, members close in value share their walk down to the last levels,
 * so queries that arrive in increasing order (the hop targets of consecutive
 * members of a sorted set) read neighbouring table entries.  The trie sizes
 * differ for general sets (not for fixed-popcount sectors).
 * Errors: as gbr_trie_create, and GBR_EINVAL for msb_first outside {0, 1}. */
int gbr_trie_create_ordered(const uint64_t *h_sorted, int64_t n, int M, int R, int msb_first, gbr_trie **out);
void gbr_trie_destroy(gbr_trie *t);

/* n_members, n_elements (trie entries without padding; the overhead factor
 * of Sec. IV is n_elements / n_members), entry_bytes (4 or 8), levels
 * (ceil(M / R)). Any output pointer may be NULL. */
int gbr_trie_info(const gbr_trie *t, int64_t *n_members, int64_t *n_elements, int *entry_bytes, int *levels);

/* Host-only construction of the same packed trie into h_t (uint64 entries,
 * capacity cap, padding included); *size_out receives the element count
 * without padding, and the call succeeds with h_t == NULL to query it.
 * Needs no GPU. */
int gbr_trie_build_host(const uint64_t *h_sorted, int64_t n, int M, int R, uint64_t *h_t, int64_t cap,
                        int64_t *size_out);

/* A trie handle from a table kept by the caller (for example one written by
 * gbr_trie_build_host_ordered in an earlier run and stored): the member list
 * is validated as by gbr_trie_create_ordered and fixes the layout, and the
 * table must have exactly that layout's length (cap entries, padding
 * included; GBR_EINVAL otherwise); its contents are uploaded as given, not
 * checked.  gbr_trie_rank with check = 1 verifies every result against the
 * member list, which is what exposes a table that does not belong to it
 * (queries it misroutes get GBR_NOT_FOUND_*).  The paper has no
 * counterpart. */
int gbr_trie_create_from_table(const uint64_t *h_sorted, int64_t n, int M, int R, int msb_first,
                               const uint64_t *h_t, int64_t len, gbr_trie **out);

/* gbr_trie_build_host with the dispatch order of gbr_trie_create_ordered. */
int gbr_trie_build_host_ordered(const uint64_t *h_sorted, int64_t n, int M, int R, int msb_first, uint64_t *h_t,
                                int64_t cap, int64_t *size_out);

/* Ranks n patterns by the trie walk of Fig. trielookup.  Every table index
 * is clamped into the table, so any input is safe.  check = 1 verifies the
 * result against the member list (Sec. IV, validity check) and writes
 * GBR_NOT_FOUND_* for non-members.  rank_bits 32 (requires n_members <=
 * 2^32) or 64.  Asynchronous on stream. */
int gbr_trie_rank(const gbr_trie *t, const uint64_t *d_pat, void *d_rank, int rank_bits, int64_t n, int check,
                  void *stream);

/* Ranks n patterns by bisection in the trie's sorted member list -- the
 * established method the paper replaces with tries (Sec. II, last
 * paragraph; Sec. V-A), kept as a comparison point.  Same arguments and
 * results as gbr_trie_rank (check = 1 marks non-members GBR_NOT_FOUND_*). */
int gbr_trie_rank_bisect(const gbr_trie *t, const uint64_t *d_pat, void *d_rank, int rank_bits, int64_t n, int check,
                         void *stream);

/* Unranks through the stored member list (Sec. II, unranking by a list);
 * out-of-range ranks give GBR_NOT_FOUND_U64. */
int gbr_trie_unrank(const gbr_trie *t, const void *d_rank, int rank_bits, uint64_t *d_pat, int64_t n, void *stream);

/* ------------------------------------------------------------------------
 * Hubbard / impurity Hamiltonians and the on-the-fly H·v (Sec. II,
 * Eqs. Talpha and mvblock; Eq. Hring; Appendix, Eqs. ci and Fig. mul).
 *
 *   H = sum_sigma sum_{p != q} h[p][q] c^dag_{p sigma} c_{q sigma}
 *     + sum_{p, sigma} h[p][p] n_{p sigma} + sum_p U[p] n_{p up} n_{p dn}
 *
 * (Eq. H with t = -h for the one-body part, on-site U as in Eq. Hring.)
 * --------------------------------------------------------------------- */
typedef struct gbr_ham gbr_ham;

enum {
    GBR_RANK_STAGGERED = 0, /* Fig. fastrank with 8-bit chunks */
    GBR_RANK_CNS = 1        /* Fig. algr, one binomial per set bit */
};

enum {
    GBR_HV_AUTO = 0,        /* pick by sector size (and the tuner, if run) */
    GBR_HV_FUSED = 1,       /* one kernel: per element unrank, hop, sign, rank, gather */
    GBR_HV_FACTORED = 2     /* per-spin hop lists ranked once per call, then two gather passes */
};

/* L: 1..32 sites; h: L*L row-major symmetric one-body matrix (host, copied);
 * U: L on-site interactions (host, copied; NULL = all zero);
 * Nup, Ndn: 0..L; rank_method: GBR_RANK_*.
 * Errors: GBR_EINVAL (non-symmetric h, sizes), GBR_ENOMEM, GBR_ECUDA. */
int gbr_ham_create(int L, const double *h, const double *U, int Nup, int Ndn, int rank_method, gbr_ham **out);
void gbr_ham_destroy(gbr_ham *H);

/* dim = C(L,Nup) C(L,Ndn); elements = matrix elements one H·v visits
 * (the diagonal plus every non-zero off-diagonal (state, hop) pair). */
int gbr_ham_info(const gbr_ham *H, int64_t *dim, int64_t *elements);

/* Selects the H·v implementation (GBR_HV_*) used by gbr_hv and gbr_lanczos. */
int gbr_ham_set_path(gbr_ham *H, int path);

/* The H·v implementation the handle currently uses (GBR_HV_*; GBR_HV_AUTO
 * until set or tuned).  Errors: GBR_EINVAL for a NULL argument. */
int gbr_ham_get_path(const gbr_ham *H, int *path);

/* y = H x on the sector (Eq. mvblock with Eq. Talpha applied on the fly).
 *   d_x, d_y: dim elements (device), float when fp == 32, double when
 *   fp == 64; they must not overlap.  Deterministic: each y element has one
 *   owner and a fixed summation order, no atomics.  Asynchronous.  The
 *   factored path uses two scratch vectors owned by the handle (allocated on
 *   first use): calls on one handle must not overlap. */
int gbr_hv(const gbr_ham *H, const void *d_x, void *d_y, int fp, void *stream);

/* gbr_hv for callers that cannot allocate device memory when they multiply
 * (for example code under a fixed memory budget handed out by a host
 * framework, or a loop that must never reach the allocator).  The paper has
 * no counterpart: this is an interface of this library.  It computes exactly what gbr_hv's factored
 * path computes, but its two scratch vectors live in one static device array
 * of 64 MiB that every GPU loading the library reserves until the process
 * exits, so the call itself allocates nothing (no cudaMalloc or cudaFree).
 *   Limit: 2 * dim * (fp / 8) bytes, each vector rounded up to 256 bytes,
 *   must fit in 64 MiB (dim up to about 8.4 million in FP32, 4.2 million in
 *   FP64); larger sectors return GBR_EINVAL before anything is launched.
 *   Set-up: the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current and keeps it; make that
 *   first call before any stream capture, and do not use the call after a
 *   cudaDeviceReset of that device in the same process (the kept address
 *   would be stale).  With lazy module loading the array is reserved when
 *   the module first loads on the device, which may be that first call.
 *   Sharing: every call on a device uses the same array, so calls that can
 *   overlap on the GPU (other streams, other threads) race and must be
 *   ordered by the caller.  Nothing needs clearing between calls: every
 *   scratch element is written before it is read.
 * Arguments and results as for gbr_hv. */
int gbr_hv_static(const gbr_ham *H, const void *d_x, void *d_y, int fp, void *stream);

/* One stage of the factored H·v, for timing and inspection.  With x viewed
 * as the D_up x D_dn matrix X:
 *   stage 1: rank the per-spin hop lists (unrank, hop, sign, staggered or
 *            combinadics rank) into the handle's tables (x, y unused);
 *   stage 2: X^T into the handle's scratch (y unused);
 *   stage 3: Z = X H_dn^T into the handle's scratch, computed as the row
 *            gathers H_dn X^T (x, y unused); stored transposed with the
 *            plain gathers, row-major with the windowed ones;
 *   stage 4: y = H_up X + Dg o X + Z (row gathers, diagonal, combine).
 * Calling 1..4 in order on one stream equals gbr_hv with the factored path.
 * Stages 3 and 4 return GBR_EINVAL until stage 1 has run on the handle and
 * stage 2 (which allocates the handle's scratch, two vectors of dim elements)
 * in this precision.  Arguments as for gbr_hv; one H·v at a time per handle. */
int gbr_hv_stage(const gbr_ham *H, const void *d_x, void *d_y, int fp, int stage, void *stream);

/* A call with a stored basis (store_basis) leaves the basis buffer, its one
 * large allocation, in a process-wide cache rather than in the handle; the
 * next call on the same device reuses it when it is large enough, so
 * repeated solves neither allocate nor free it (the paper has no
 * counterpart: this is an interface of this library).  The cache keeps at
 * most one buffer, the largest, until gbr_release_cache frees it.  Always
 * returns GBR_OK; call it with no solve running. */
int gbr_release_cache(void);

/* Self-check of the FP64 reciprocal the tridiagonal eigensolvers use instead
 * of the division (Newton-Raphson iteration from the single-precision
 * approximate reciprocal; the paper has no counterpart): *h_max_rel_err
 * receives the largest relative difference from the IEEE division over n
 * values from 1e-29 to 1e29 of both signs.  Synchronous; GBR_EINVAL for
 * n < 1 or a NULL output. */
int gbr_check_rcp64(int64_t n, double *h_max_rel_err);

/* Kernels this library has launched in the process so far (eager launches
 * plus, for replayed CUDA graphs, the kernels each replay runs). */
int64_t gbr_launch_count(void);

/* Auto-tunes the H·v launch shape for precision fp on this device by timing
 * the candidates on scratch vectors; the choice is kept in the handle: the
 * path (fused or factored), the gather family of the factored path (plain
 * row gathers, or windowed gathers that stage each CTA's own rows in shared
 * memory), the rows per CTA of each gather pass in that family, and those of
 * the spin-up pass as the Lanczos launches it.  Synchronises the stream. */
int gbr_ham_tune(gbr_ham *H, int fp, void *stream);

/* Launch shape of the H·v for precision fp: the knobs gbr_ham_tune sets,
 * exposed for tests and experiments (the paper has no counterpart).
 * h_shape: 9 ints (host).
 *   [0]: 1 = windowed row gathers in the factored path (each CTA copies its
 *     TR own rows of a 512-byte column slice into shared memory with bulk
 *     copies, serves the hops that stay inside them from there, and the
 *     spin-down pass keeps its product row-major), 0 = plain row gathers;
 *   [1..3]: rows per CTA of the spin-down pass, the spin-up pass and the
 *     spin-up pass with the fused Lanczos update (plain: 4, 8 or 16;
 *     windowed: 32 or 64; 0 = default);
 *   [4]: chunk width R of the per-spin staggered tables (Fig. fastrank):
 *     8 or 4 (0 = 8); the paper compares both inside the H·v (Sec. V-B);
 *   [5]: threads per state of the fused per-element kernel: 1, 2 or 4
 *     (0 = 1); the threads of a state split its occupied sites;
 *   [6..8]: threads per CTA of the plain spin-down, spin-up and fused-update
 *     passes: 128, or 64 for column chunks half as wide (0 = 128); the
 *     windowed kernels always run 256 (reported as such).
 * In the factored path every element sums its hops in the same order under
 * every value of [0..4] and [6..8], so gbr_hv's results do not depend on
 * them; [5] changes the summation order of the fused kernel (a fixed
 * butterfly).
 * The windowed family needs per-spin dimensions whose rows are whole 16-byte
 * packs (gbr_ham_get_shape reports 0 otherwise) and 16-byte aligned vectors
 * (a combine pass on other vectors runs the plain kernel).  Errors:
 * GBR_EINVAL for NULL arguments, fp other than 32 or 64, or values outside
 * the lists above. */
int gbr_ham_set_shape(gbr_ham *H, int fp, const int *h_shape);
/* The shape gbr_hv uses for precision fp (h_shape: 9 ints, as above). */
int gbr_ham_get_shape(const gbr_ham *H, int fp, int *h_shape);

/* Device status word of the library's kernels on the current device (the
 * paper has no counterpart).  Kernels that wait on an mbarrier for their own
 * bulk copies bound the wait (about a second); when it runs out they set bit
 * 0 here and return without computing, instead of trapping or hanging.
 * *status receives the word; clear = 1 resets it.  Returns GBR_ETIMEOUT if
 * the word is non-zero, else GBR_OK (GBR_ECUDA if it cannot be read).
 * Synchronous with respect to the device. */
int gbr_device_status(int clear, int *status);

/* ------------------------------------------------------------------------
 * The same Hamiltonians on an arbitrary sorted set of 2L-bit states, ranked
 * by a packed trie (Sec. IV: sectors cut by further quantum numbers, which
 * combinadics cannot index; here also unions of spin sectors, e.g. every
 * S_z at fixed total particle number).
 * --------------------------------------------------------------------- */
typedef struct gbr_setham gbr_setham;

/* L: 1..32 sites; h, U as for gbr_ham_create; h_states: n distinct 2L-bit
 * patterns in increasing order (spin down in the low L bits; host, copied);
 * R: trie radix bits (1..16, 8 recommended).  Builds the packed trie of the
 * set (gbr_trie_create_ordered's layout, most significant chunk first).
 * Errors: GBR_EINVAL (unsorted set, bits at or above 2L, h not symmetric),
 * GBR_ENOMEM, GBR_ECUDA. */
int gbr_setham_create(int L, const double *h, const double *U, const uint64_t *h_states, int64_t n, int R,
                      gbr_setham **out);

/* gbr_setham_create with the trie's dispatch order (gbr_trie_create_ordered);
 * gbr_setham_create uses msb_first = 1, whose walks for consecutive members
 * stay in one subtree of the table. */
int gbr_setham_create_ordered(int L, const double *h, const double *U, const uint64_t *h_states, int64_t n, int R,
                              int msb_first, gbr_setham **out);
void gbr_setham_destroy(gbr_setham *S);

/* bisect = 1: rank hop targets by bisection in the sorted member list (the
 * established method of Sec. II, the comparison point of Fig. eig-timings;
 * targets are always checked); 0 (default): by the trie.
 * Errors: GBR_EINVAL for a NULL handle. */
int gbr_setham_set_bisect(gbr_setham *S, int bisect);

/* dim = n; elements = n plus every hop of every member (the matrix elements
 * one H·v visits when the set is closed under H); trie_elements = packed
 * trie size without padding. */
int gbr_setham_info(const gbr_setham *S, int64_t *dim, int64_t *elements, int64_t *trie_elements);

/* y = P H P x on the set (Eq. mvblock on the set, Eq. Talpha on the fly):
 * one thread per member applies every term; each hop target is ranked by
 * the trie walk of Fig. trielookup on the full pattern.  check = 1 drops
 * targets outside the set (found by the member-list check of Sec. IV), which
 * makes the result exact for any set; check = 0 trusts the set to be closed
 * under H.  d_x, d_y: n floats (fp 32) or doubles (fp 64), not overlapping.
 * Deterministic; asynchronous on stream. */
int gbr_setham_hv(const gbr_setham *S, const void *d_x, void *d_y, int fp, int check, void *stream);

/* ------------------------------------------------------------------------
 * General operator-product terms (Appendix: Eqs. Talpha1, Talpha2, ci and
 * Fig. mul) and their on-the-fly H·v over a trie-ranked set.
 * --------------------------------------------------------------------- */

/* The tuple of a product T of creators and annihilators with a scalar:
 *   T|a> = v delta(a & m, r) (-1)^h(a & s) |a ^ x>     (Eq. Talpha1)
 *   <a|T = v delta(a & m, l) (-1)^h(a & s) <a ^ x|     (Eq. Talpha2)
 * with h the number of set bits; bit i = spin-orbital i. */
typedef struct {
    double v;
    uint64_t m, l, r, x, s;
} gbr_term;

/* Tuple of coef * O_1 O_2 ... O_nops (O_1 leftmost) built from the blocks of
 * Eqs. ci by the product rule of Fig. mul.  ops[k] = 2 * orbital + 1 for a
 * creator, 2 * orbital for an annihilator (orbital 0..63).  Host only; a
 * product that vanishes by the Pauli principle has v = 0. */
int gbr_term_product(const int *ops, int nops, double coef, gbr_term *out);

/* Tuple of the product a b (Fig. mul).  Host only. */
int gbr_term_mul(const gbr_term *a, const gbr_term *b, gbr_term *out);

typedef struct gbr_termham gbr_termham;

/* H = sum of nterms tuples on M spin-orbitals (M 1..64), acting on the n
 * sorted, distinct M-bit states h_states (host, copied), ranked by a packed
 * trie of radix 2^R (most significant chunk first, as gbr_setham_create).
 * Terms must not touch orbitals at or above M.
 * Errors: GBR_EINVAL, GBR_ENOMEM, GBR_ECUDA. */
int gbr_termham_create(int M, const gbr_term *h_terms, int nterms, const uint64_t *h_states, int64_t n, int R,
                       gbr_termham **out);
void gbr_termham_destroy(gbr_termham *T);

/* bisect = 1: rank hop targets by bisection in the sorted member list (the
 * established method of Sec. II, kept as the comparison point; targets are
 * always checked); 0 (default): by the trie. */
int gbr_termham_set_bisect(gbr_termham *T, int bisect);

/* dim = n; elements = the (member, term) pairs whose left demand holds (the
 * matrix elements one H·v visits); trie_elements = trie size. */
int gbr_termham_info(const gbr_termham *T, int64_t *dim, int64_t *elements, int64_t *trie_elements);

/* y = P H P x on the set: each member applies every term from the left
 * (Eq. Talpha2), so y is the true row action for any term list, Hermitian
 * or not; targets are ranked by the trie walk (Fig. trielookup) and, with
 * check = 1, verified against the member list and dropped when outside.
 * d_x, d_y: n floats (fp 32) or doubles (fp 64).  Asynchronous. */
int gbr_termham_hv(const gbr_termham *T, const void *d_x, void *d_y, int fp, int check, void *stream);

/* ------------------------------------------------------------------------
 * Lanczos ground state (cited in Sec. I and V-B; the recurrence is the
 * textbook three-term one).
 * --------------------------------------------------------------------- */
enum { GBR_PREC_FP64 = 0, GBR_PREC_MIXED = 1 };

typedef struct {
    int iters;        /* H·v steps (>= 1) */
    int reorth;       /* 1 = full re-orthogonalisation (two classical Gram-Schmidt
                         passes in FP64 against every stored vector) */
    int prec;         /* GBR_PREC_FP64: FP64 vectors and H·v;
                         GBR_PREC_MIXED: FP32 vectors and H·v, FP64 scalars */
    int refine;       /* 1 = form the Ritz vector and return the FP64 Rayleigh
                         quotient <x,Hx>/<x,x> and residual |Hx - E x| / |x|.
                         The vector is that of the shortest prefix T_k (k a
                         multiple of 8) whose lowest pair has residual estimate
                         beta_{k+1} |s_k| <= u max_j(|alpha_j|, beta_j), u the unit
                         roundoff of the vectors (2^-24 mixed, 2^-53 FP64), else of
                         the whole T: a run that goes on past that point without
                         re-orthogonalisation grows copies of the converged state,
                         which spoil the Ritz vector of the longer T */
    int store_basis;  /* 1 = keep all vectors (needed by reorth; makes the Ritz
                         vector one pass), 0 = recompute the basis in a second
                         run of the recurrence, -1 = decide from free memory:
                         all vectors if they fit, else the leading ones that fit
                         (at least 8; the second run starts after them),
                         -m (m >= 2) = keep the leading m vectors.  A head is
                         kept only when a vector is a whole number of 16-byte
                         packs (dim * element size divisible by 16) */
    int use_graph;    /* 1 = replay each iteration as a captured CUDA graph */
    int profile;      /* 1 = time every H·v stage with CUDA events (no graphs) */
    double tol;       /* > 0: every 8 steps, stop once the lowest Ritz pair of T
                         has residual estimate beta_{k+1} |s_k| <= tol * max_j(|alpha_j|,
                         beta_j); 0 = run all iters steps */
    double ritz_tail; /* > 0 (refine only): the Ritz vector x = sum_j s_j v_j keeps the
                         leading terms and drops the trailing ones whose coefficients
                         have norm <= ritz_tail |s|; the Rayleigh quotient then moves by
                         about ritz_tail^2 times the spectral spread (it stays an upper
                         bound of the lowest eigenvalue), and the second run of the
                         recurrence (store_basis 0) stops early.  0 = every term */
} gbr_lanczos_opts;

typedef struct {
    double E0;         /* refined energy if refine, else the lowest Ritz value */
    double E_ritz;     /* lowest eigenvalue of the tridiagonal matrix */
    double residual;   /* |H x - E0 x| / |x| (refine only, else -1) */
    int iters_done;    /* H·v steps actually taken */
    int breakdown;     /* 1 if the recurrence stopped on beta ~ 0 */
    int stored_basis;  /* 1 if the basis was kept in device memory */
    double seconds;    /* device time of the whole call (CUDA events) */
    double hv_seconds; /* device time spent inside H·v launches (profile only) */
    double stage_seconds[4]; /* profile: total device time of the H·v stages
                                (hop lists, transpose, spin-down gather,
                                spin-up gather with diagonal; the fused path
                                is counted in the last slot) */
    int stage_launches[4];   /* profile: launches of each stage */
    int converged;           /* 1 if the tol test stopped the recurrence */
    int ritz_terms;          /* Lanczos vectors summed into the Ritz vector (refine):
                                the prefix length, less any ritz_tail terms */
    int basis_head;          /* without a stored basis (refine): leading vectors of
                                the Ritz sum taken from the head of the basis that
                                the first run kept (store_basis -1 keeps as many as
                                fit when the whole basis does not); the second run
                                of the recurrence starts after them.  0 = none */
} gbr_lanczos_result;

/* Runs Lanczos from the start vector d_v0 (dim doubles on the device, not
 * necessarily normalised; the mixed path rounds it to FP32 first).
 * h_alpha, h_beta (host, may be NULL): receive the iters_done diagonal and
 * iters_done-1 off-diagonal entries; h_ritz (host, may be NULL): the lowest
 * Ritz value after every step.  Stops early (breakdown) when
 * beta_{k+1} <= 1e-13 max_j(|alpha_j|, beta_j).  Synchronises the stream.
 * Errors: GBR_EINVAL, GBR_ENOMEM (vectors do not fit), GBR_ECUDA,
 * GBR_ENONFINITE (alpha or beta came out NaN or infinite: a NaN or Inf in the
 * start vector propagates through H·v and the dots and stops the recurrence
 * at the step where it appears; res->iters_done tells which). */
int gbr_lanczos(const gbr_ham *H, const gbr_lanczos_opts *opts, const double *d_v0, gbr_lanczos_result *res,
                double *h_alpha, double *h_beta, double *h_ritz, void *stream);

/* The same Lanczos solve with the trie-ranked H·v of a set Hamiltonian as
 * the operator (Sec. IV: a state set cut by further quantum numbers, ranked
 * by a packed trie; the ground state of, e.g., one S_z sector or one
 * symmetry-cut subset).  The operator is gbr_setham_hv with the membership
 * check on, so a set that H does not map into itself gets the projection
 * P H P.  d_v0: dim doubles (the set's size); arguments, precision paths,
 * refinement and errors as for gbr_lanczos (stage_seconds stay zero). */
int gbr_setham_lanczos(const gbr_setham *S, const gbr_lanczos_opts *opts, const double *d_v0,
                       gbr_lanczos_result *res, double *h_alpha, double *h_beta, double *h_ritz, void *stream);

/* The same Lanczos solve with the term-list H·v (Appendix: Eqs. Talpha2 and
 * Fig. mul; Sec. V-C, Eq. Hk for the momentum-basis ring) as the operator,
 * with the membership check on.  The term list must make a symmetric
 * operator on the set (every term with its adjoint, real coefficients):
 * Lanczos assumes it.  Arguments and errors as for gbr_lanczos. */
int gbr_termham_lanczos(const gbr_termham *T, const gbr_lanczos_opts *opts, const double *d_v0,
                        gbr_lanczos_result *res, double *h_alpha, double *h_beta, double *h_ritz, void *stream);

/* ------------------------------------------------------------------------
 * Batched ground states of many small models, every (N_up, N_dn) sector,
 * in one persistent launch (the impurity-solver use case of Sec. I and VI).
 * --------------------------------------------------------------------- */
typedef struct {
    int L;             /* sites, 1..10 */
    const double *h;   /* L*L symmetric one-body matrix (host) */
    const double *U;   /* L on-site interactions (host, NULL = 0) */
} gbr_model_desc;

/* Number of sectors and total states of the batch: sectors are ordered
 * model by model, then N_up = 0..L, then N_dn = 0..L; sector s starts at
 * state offset sum of the dimensions before it. */
int gbr_batch_layout(int n_models, const gbr_model_desc *models, int64_t *n_sectors, int64_t *n_states);

/* Solves every sector of every model with mixed-precision Lanczos (FP32
 * vectors in shared memory, FP64 scalars, FP64 Rayleigh-quotient
 * refinement of the Ritz vector) in one persistent kernel; each CTA pulls
 * sectors from a device work queue, largest first.
 *   d_start: n_states start-vector entries (device doubles), sector by
 *            sector in the layout above;
 *   iters:   Lanczos steps per sector (capped by the sector dimension);
 *   h_E0:    n_models ground-state energies (host);
 *   h_arg:   2 * n_models (N_up, N_dn) of the minimising sector (host, may
 *            be NULL); ties within 1e-10 |E| go to the lower N_up + N_dn,
 *            then the lower N_up;
 *   h_sector_E (host, may be NULL): n_sectors refined sector energies.
 * The work queue is an atomic counter: no CTA waits on another.
 * Synchronises the stream. Errors: GBR_EINVAL, GBR_ENOMEM, GBR_ECUDA. */
int gbr_batch_solve(int n_models, const gbr_model_desc *models, const double *d_start, int iters, double *h_E0,
                    int *h_arg, double *h_sector_E, void *stream);

/* Launch shape of gbr_batch_solve (process-wide; the paper has no
 * counterpart): threads per CTA (128, 256 or 512) and CTAs per SM
 * (0 = as many as the shared memory and registers allow, else at most that
 * many).  Every shape gives the same sector energies up to FP rounding of
 * the block reductions.  Errors: GBR_EINVAL for other values. */
int gbr_batch_set_shape(int threads, int ctas_per_sm);
int gbr_batch_get_shape(int *threads, int *ctas_per_sm);

/* Auto-tunes the batch solver's launch shape on this batch: solves it with
 * every candidate (threads 128, 256, 512 x CTAs per SM as many as fit, 2, 1),
 * times each whole launch with CUDA events, keeps the fastest as the
 * process-wide shape and returns it in h_shape[2] (threads, CTAs per SM);
 * h_ms (host, may be NULL) receives the 9 times in that order.  Arguments as
 * for gbr_batch_solve.  Synchronises the stream. */
int gbr_batch_tune(int n_models, const gbr_model_desc *models, const double *d_start, int iters, int *h_shape,
                   float *h_ms, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GBRANK_H */
