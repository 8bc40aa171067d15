// Lanczos ground state on the GPU (the paper cites the method in Sec. I and
// V-B without stating it; this is the textbook three-term recurrence):
//   v_0 = s/|s|;  w = H v_k - beta_k v_{k-1};  alpha_k = <w, v_k>;
//   w -= alpha_k v_k;  [two classical Gram-Schmidt passes against v_0..v_k];
//   beta_{k+1} = |w|;  stop if beta_{k+1} <= 1e-13 max_j(|alpha_j|, beta_j);
//   v_{k+1} = w / beta_{k+1};  E = lowest eigenvalue of T_k.
// The vectors are kept unnormalised, u_j = g_j v_j with g_0 = 1 and
// g_j = beta_j: the division by beta_{k+1} is folded into the next step
// (w = H u_k / g_k - (beta_k / g_{k-1}) u_{k-1}, alpha_k = <w, u_k> / g_k,
// w -= (alpha_k / g_k) u_k), which saves a full vector pass per step; the
// scalars alpha, beta are those of the normalised recurrence.
// All scalars stay on the device (no host round trip per step).  Reductions
// use a fixed grid and a fixed summation tree, so every run is bit-identical
// and the basis can be recomputed exactly in a second pass.
//
// Precision.  FP64 path: FP64 vectors, H·v and dots.  Mixed path: FP32
// vectors and H·v; every dot product and norm is accumulated exactly per
// element (the FP32 product split into two floats with an FMA) in a
// two-float running sum, then combined across threads in FP64 -- FP64-grade
// accuracy without the FP64 pipe, which runs at about 1/60 of FP32 rate on
// this GPU.  The tridiagonal eigenproblem, Ritz coefficients and the final
// Rayleigh quotient <x, Hx>/<x, x> with an FP64 H·v are FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "ham.h"
#include "dot.cuh"

namespace gbr {

// State shared by the step kernels (device memory).
struct LzState {
    int k;            // current step
    int stop;         // 1 once the recurrence broke down or finished
    int breakdown;
    int converged;    // 1 once the residual test stopped the recurrence
    double scale;     // max_j(|alpha_j|, beta_j)
    double lam_hint;  // convergence test: previous lowest Ritz value and its last decrease
    double gap_hint;
    int nonfinite;    // 1 once alpha or beta came out NaN or infinite (stops the recurrence)
};

// 16-byte packs of vector elements for the streaming kernels: every vector
// is a cudaMalloc'd buffer (256-byte aligned); elements past the last full
// pack are handled one by one.
template <typename T> struct alignas(16) Pack {
    static constexpr int N = 16 / sizeof(T);
    T e[N];
};

// Per-step scalars of the unnormalised recurrence, 4 doubles per step j,
// written once by the single-thread finalisation (so the vector kernels only
// load them; FP64 division is slow on this GPU) and kept for the second
// pass: [4j] = 1/g_j, [4j+1] = beta_j / g_{j-1} (0 at j = 0),
// [4j+2] = alpha_j / g_j, where g_0 = 1 and g_j = beta_j.
constexpr int kScal = 4;

// w = H u_k / g_k - (beta_k / g_{k-1}) u_{k-1} (k > 0; w = H u_0 at k = 0),
// with H u_k in w on entry; partial <w, u_k>
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_step1(const LzState *st, const double *scal, const T *__restrict__ vprev,
                                                       const T *__restrict__ v, T *__restrict__ w, int64_t n, double *part,
                                                       int want_dot) {
    if (st->stop) return;
    const int k = st->k;
    const T s1 = (T)scal[kScal * k];
    const T b = (T)scal[kScal * k + 1];
    DotAcc<T> acc;
    constexpr int V = Pack<T>::N;
    const int64_t np = n / V;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    const Pack<T> *VP = reinterpret_cast<const Pack<T> *>(vprev), *VV = reinterpret_cast<const Pack<T> *>(v);
    Pack<T> *W = reinterpret_cast<Pack<T> *>(w);
#pragma unroll 2
    for (int64_t p = tid; p < np; p += stride) {
        Pack<T> wp = W[p];
        const Pack<T> vv = VV[p];
        if (k > 0) {
            const Pack<T> pp = VP[p];
#pragma unroll
            for (int j = 0; j < V; ++j) wp.e[j] = lz_rec(s1, wp.e[j], b, pp.e[j]);
            W[p] = wp;
        }
        if (want_dot)
#pragma unroll
            for (int j = 0; j < V; ++j) acc.add(wp.e[j], vv.e[j]);
    }
    for (int64_t i = np * V + tid; i < n; i += stride) {
        T wi = w[i];
        if (k > 0) wi = lz_rec(s1, wi, b, vprev[i]);
        w[i] = wi;
        if (want_dot) acc.add(wi, v[i]);
    }
    if (!want_dot) return;
    const double r = block_sum(acc.value());
    if (threadIdx.x == 0) part[blockIdx.x] = r;
}

// w -= (alpha_k / g_k) u_k, which makes w the next unnormalised vector
// u_{k+1}; partial <w, w>; with a basis of `slots` vectors, u_{k+1} also into
// its slot k + 1 while k + 1 < slots
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_step2(const LzState *st, const double *scal, const T *__restrict__ v,
                                                       T *__restrict__ w, T *__restrict__ basis, int slots, int64_t n,
                                                       double *part, int want_dot) {
    if (st->stop) return;
    const int k = st->k;
    const T a = (T)scal[kScal * k + 2];
    T *vb = (basis && k + 1 < slots) ? basis + (int64_t)(k + 1) * n : nullptr;
    DotAcc<T> acc;
    constexpr int V = Pack<T>::N;
    // the basis slot is aligned to 16 bytes only when n * sizeof(T) is
    const bool vec_ok = !vb || ((uintptr_t)vb & 15u) == 0;
    const int64_t np = vec_ok ? n / V : 0;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    const Pack<T> *VV = reinterpret_cast<const Pack<T> *>(v);
    Pack<T> *W = reinterpret_cast<Pack<T> *>(w), *VB = reinterpret_cast<Pack<T> *>(vb);
#pragma unroll 2
    for (int64_t p = tid; p < np; p += stride) {
        Pack<T> wp = W[p];
        const Pack<T> vv = VV[p];
#pragma unroll
        for (int j = 0; j < V; ++j) wp.e[j] = lz_fnma(a, vv.e[j], wp.e[j]);
        W[p] = wp;
        if (vb) VB[p] = wp;
        if (want_dot)
#pragma unroll
            for (int j = 0; j < V; ++j) acc.add(wp.e[j], wp.e[j]);
    }
    for (int64_t i = np * V + tid; i < n; i += stride) {
        const T wi = lz_fnma(a, v[i], w[i]);
        w[i] = wi;
        if (vb) vb[i] = wi;
        if (want_dot) acc.add(wi, wi);
    }
    if (!want_dot) return;
    const double r = block_sum(acc.value());
    if (threadIdx.x == 0) part[blockIdx.x] = r;
}

// k_step2 for the factored H·v: the same update w -= (alpha_k / g_k) u_k and
// partial <w, w>, over 64 x 64 tiles of the D_up x D_dn matrix, which also
// writes the transpose of the new vector into xt: the spin-down pass of the
// next H·v reads X^T, and this saves it the transpose's read of the vector.
// 16-byte packs; needs rows and cols that are multiples of the pack and
// 16-byte aligned vectors (edge tiles go element by element).
// With a basis of `slots` vectors, u_{k+1} also goes into its slot k + 1
// while k + 1 < slots (rows * cols is a whole number of packs, so every slot
// is 16-byte aligned).
template <typename T>
__global__ void __launch_bounds__(256) k_step2_t(const LzState *st, const double *scal, const T *__restrict__ v,
                                                 T *__restrict__ w, T *__restrict__ xt, T *__restrict__ basis,
                                                 int slots, int64_t rows, int64_t cols, double *part, int want_dot) {
    if (st->stop) return;
    constexpr int TILE = 64, V = Pack<T>::N, RP = TILE / V;
    __shared__ T tile[TILE][TILE + 1];
    const T a = (T)scal[kScal * st->k + 2];
    T *vb = (basis && st->k + 1 < slots) ? basis + (int64_t)(st->k + 1) * rows * cols : nullptr;
    const int64_t c0 = (int64_t)blockIdx.x * TILE, r0 = (int64_t)blockIdx.y * TILE;
    const bool full = r0 + TILE <= rows && c0 + TILE <= cols;
    DotAcc<T> acc;
    for (int idx = threadIdx.x; idx < TILE * RP; idx += blockDim.x) {
        const int i = idx / RP, j = idx % RP;
        const int64_t r = r0 + i, c = c0 + (int64_t)j * V;
        if (full) {
            Pack<T> wp = *reinterpret_cast<const Pack<T> *>(w + r * cols + c);
            const Pack<T> vv = *reinterpret_cast<const Pack<T> *>(v + r * cols + c);
#pragma unroll
            for (int e = 0; e < V; ++e) wp.e[e] = lz_fnma(a, vv.e[e], wp.e[e]);
            *reinterpret_cast<Pack<T> *>(w + r * cols + c) = wp;
            if (vb) *reinterpret_cast<Pack<T> *>(vb + r * cols + c) = wp;
#pragma unroll
            for (int e = 0; e < V; ++e) {
                tile[i][j * V + e] = wp.e[e];
                if (want_dot) acc.add(wp.e[e], wp.e[e]);
            }
        } else {
#pragma unroll
            for (int e = 0; e < V; ++e) {
                T wi = T(0);
                if (r < rows && c + e < cols) {
                    wi = lz_fnma(a, v[r * cols + c + e], w[r * cols + c + e]);
                    w[r * cols + c + e] = wi;
                    if (vb) vb[r * cols + c + e] = wi;
                    if (want_dot) acc.add(wi, wi);
                }
                tile[i][j * V + e] = wi;
            }
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < TILE * RP; idx += blockDim.x) {
        const int c = idx / RP, j = idx % RP;
        const int64_t oc = c0 + c, orow = r0 + (int64_t)j * V;
        Pack<T> o;
#pragma unroll
        for (int e = 0; e < V; ++e) o.e[e] = tile[j * V + e][c];
        if (full) {
            *reinterpret_cast<Pack<T> *>(xt + oc * rows + orow) = o;
        } else if (oc < cols) {
#pragma unroll
            for (int e = 0; e < V; ++e)
                if (orow + e < rows) xt[oc * rows + orow + e] = o.e[e];
        }
    }
    if (!want_dot) return;
    const double r = block_sum(acc.value());
    if (threadIdx.x == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = r;
}

// partial <w, w> only (after re-orthogonalisation)
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_norm2(const LzState *st, const T *__restrict__ w, int64_t n, double *part) {
    if (st->stop) return;
    DotAcc<T> acc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc.add(w[i], w[i]);
    const double r = block_sum(acc.value());
    if (threadIdx.x == 0) part[blockIdx.x] = r;
}

// which: 0 = alpha_k = sum / g_k; 1 = beta_{k+1} = sqrt(sum) with the
// stopping test; each also stores the scalars the vector kernels need
constexpr int kFinThreads = 1024;

__global__ void __launch_bounds__(kFinThreads) k_finalize(LzState *st, double *alpha, double *beta, double *scal,
                                                          const double *part, int nparts, int which, int iters) {
    if (st->stop) return;
    // four independent running sums per thread (fixed order), so the loads
    // of one thread are not one dependency chain
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    const int step = 4 * blockDim.x;
    int i = threadIdx.x;
    for (; i + 3 * (int)blockDim.x < nparts; i += step) {
        v0 += part[i];
        v1 += part[i + blockDim.x];
        v2 += part[i + 2 * blockDim.x];
        v3 += part[i + 3 * blockDim.x];
    }
    for (; i < nparts; i += blockDim.x) v0 += part[i];
    const double s = block_sum<kFinThreads>((v0 + v1) + (v2 + v3));
    if (threadIdx.x != 0) return;
    const int k = st->k;
    if (which == 0) {
        // the partials hold <w, u_k> = g_k alpha_k
        const double a = s * scal[kScal * k];
        alpha[k] = a;
        scal[kScal * k + 2] = a * scal[kScal * k];
        st->scale = fmax(st->scale, fabs(a));
        if (!isfinite(a)) {
            st->stop = 1;
            st->nonfinite = 1;
        }
    } else {
        if (!isfinite(s)) {
            st->stop = 1;
            st->nonfinite = 1;
            return;
        }
        const double b = sqrt(fmax(s, 0.0));
        beta[k + 1] = b;
        scal[kScal * (k + 1)] = 1.0 / b;
        scal[kScal * (k + 1) + 1] = b * scal[kScal * k];
        if (k + 1 >= iters) {
            st->stop = 1;
        } else if (b <= 1e-13 * st->scale) {
            st->stop = 1;
            st->breakdown = 1;
        }
        st->scale = fmax(st->scale, b);
    }
}

// First stage for a long list of partial sums (the spin-up pass of the ring
// writes one per CTA, 2.3 million): block b sums the contiguous segment
// [b * seg, (b + 1) * seg) in a fixed order, so that the single-block
// finalisation reads one value per block instead of the whole list.
constexpr int kReduceAbove = 1 << 16, kReduceBlocks = 512;
__global__ void __launch_bounds__(kRedThreads) k_reduce_parts(const LzState *st, const double *__restrict__ part,
                                                              int nparts, double *__restrict__ out) {
    if (st->stop) return;
    const int seg = (nparts + (int)gridDim.x - 1) / (int)gridDim.x;
    const int lo = (int)blockIdx.x * seg, hi = min(nparts, lo + seg);
    double v = 0.0;
    for (int i = lo + (int)threadIdx.x; i < hi; i += (int)blockDim.x) v += part[i];
    const double r = block_sum(v);
    if (threadIdx.x == 0) out[blockIdx.x] = r;
}

__global__ void k_advance(LzState *st) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && !st->stop) st->k += 1;
}

// Re-orthogonalisation against the stored (unnormalised) basis u_j:
// d_j = <w, u_j> for j = 0..k (grid.y = j), c_j = d_j / g_j^2, then
// w -= sum_j c_j u_j (= sum_j <w, v_j> v_j).
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_multidot(const LzState *st, const T *__restrict__ basis,
                                                          const T *__restrict__ w, int64_t n, double *part) {
    if (st->stop) return;
    const int j = blockIdx.y;
    if (j > st->k) return;
    const T *vj = basis + (int64_t)j * n;
    DotAcc<T> acc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc.add(w[i], vj[i]);
    const double r = block_sum(acc.value());
    if (threadIdx.x == 0) part[(int64_t)j * gridDim.x + blockIdx.x] = r;
}

__global__ void __launch_bounds__(kRedThreads) k_multidot_fin(const LzState *st, const double *scal, const double *part,
                                                              int nparts, double *c) {
    if (st->stop) return;
    const int j = blockIdx.x;
    if (j > st->k) return;
    double v = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += part[(int64_t)j * nparts + i];
    const double s = block_sum(v);
    const double ig = scal[kScal * j];
    if (threadIdx.x == 0) c[j] = s * ig * ig;
}

// w -= sum_j c_j u_j; the last pass also writes the result into slot k + 1
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_multiaxpy(const LzState *st, T *__restrict__ basis, const double *c,
                                                           T *__restrict__ w, int64_t n, int write_slot) {
    if (st->stop) return;
    const int k = st->k;
    T *slot = write_slot ? basis + (int64_t)(k + 1) * n : nullptr;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T wi = w[i];
        for (int j = 0; j <= k; ++j) wi -= (T)c[j] * basis[(int64_t)j * n + i];
        w[i] = wi;
        if (slot) slot[i] = wi;
    }
}

// per-step and final tridiagonal solves share the device routine of tridiag.cuh
#include "tridiag.cuh"

__global__ void __launch_bounds__(kRedThreads) k_tridiag(const LzState *st, const double *alpha, const double *beta,
                                                         int kfixed, double *out, double *s, double *work) {
    const int k = kfixed > 0 ? kfixed : (st->k + 1);
    const double lam = tridiag_lowest_block(alpha, beta, k);
    if (threadIdx.x == 0) {
        out[0] = lam;
        if (s) tridiag_vector_thread(alpha, beta, k, lam, s, work);
    }
}

// Convergence test every 8 steps (after beta_{k+1} is known): residual
// estimate of the lowest Ritz pair, beta_{k+1} |s_k|, against tol * scale.
// One warp does the eigenvalue search (warm-started from the previous test);
// thread 0 the last eigenvector component.
__global__ void __launch_bounds__(32) k_conv_check(LzState *st, const double *alpha, const double *beta, double tol,
                                                   double *work) {
    const int k = st->k + 1;
    if (st->converged || (k % 8) != 0) return;
    const double lam = tridiag_lowest_warm(alpha, beta, k, &st->lam_hint, &st->gap_hint);
    if (threadIdx.x == 0) {
        const double res = beta[k] * tridiag_last_component(alpha, beta, k, lam, work);
        if (res <= tol * st->scale) {
            st->stop = 1;
            st->converged = 1;
        }
    }
}

// The prefix of the recurrence whose Ritz vector the refinement forms: the
// shortest T_k (k = 8, 16, ... below kdone) whose lowest Ritz pair has the
// residual estimate beta_{k+1} |s_k| <= u * max_j(|alpha_j|, beta_j), u the
// unit roundoff of the vectors' precision; kdone if there is none.  A run
// without re-orthogonalisation that goes on past that point grows copies of
// the converged state in T, and the Ritz vector of the longer T loses
// accuracy, while the stored vectors cannot make it more accurate than at
// that prefix.  One warp; *kout receives the prefix length.
__global__ void __launch_bounds__(32) k_ritz_prefix(const LzState *st, const double *alpha, const double *beta,
                                                    int kdone, double u, double *work, int *kout) {
    __shared__ double lam_prev, gap;
    __shared__ int found;
    if (threadIdx.x == 0) {
        lam_prev = 0.0;
        gap = 0.0;
        found = kdone;
    }
    __syncthreads();
    const double thr = u * st->scale;
    for (int k = 8; k < kdone; k += 8) {
        const double lam = tridiag_lowest_warm(alpha, beta, k, &lam_prev, &gap);
        if (threadIdx.x == 0 && beta[k] * tridiag_last_component(alpha, beta, k, lam, work) <= thr) found = k;
        __syncthreads();
        if (found != kdone) break;
    }
    if (threadIdx.x == 0) *kout = found;
}

// per-step Ritz value into ritz[k]
__global__ void k_copy_ritz(const LzState *st, const double *val, double *ritz) {
    if (threadIdx.x == 0) ritz[st->k] = val[0];
}

// x (FP64) = sum_j s_j v_j = sum_j (s_j / g_j) u_j over the stored
// (unnormalised) basis.  FP64 basis: FMA chain.
// FP32 basis: each s_j is split into two floats once (shared memory) and the
// products are accumulated per element in a two-float sum.  Each thread
// takes 16-byte packs of consecutive elements, so one load per basis vector
// serves several elements.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_ritz_from_basis(const T *__restrict__ basis, const double *s,
                                                                 const double *scal, int k, int64_t n,
                                                                 double *__restrict__ x) {
    __shared__ float sh[1024], sl[1024];
    __shared__ double sd[1024];
    constexpr int V = Pack<T>::N;
    const bool vec_ok = (n % V) == 0;       // every basis slot then starts on a 16-byte boundary
    const int64_t np = vec_ok ? n / V : 0;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    for (int j0 = 0; j0 < k; j0 += 1024) {
        const int jn = min(1024, k - j0);
        __syncthreads();
        for (int j = threadIdx.x; j < jn; j += blockDim.x) {
            const double v = s[j0 + j] * scal[kScal * (j0 + j)];
            sd[j] = v;
            sh[j] = (float)v;
            sl[j] = (float)(v - (double)(float)v);
        }
        __syncthreads();
        for (int64_t p = tid; p < np; p += stride) {
            const Pack<T> *B = reinterpret_cast<const Pack<T> *>(basis + (int64_t)j0 * n) + p;
            const int64_t sp = n / V;   // packs per basis vector
            if (sizeof(T) == 8) {
                double acc[V];
#pragma unroll
                for (int e = 0; e < V; ++e) acc[e] = j0 ? x[p * V + e] : 0.0;
#pragma unroll 4
                for (int j = 0; j < jn; ++j) {
                    const Pack<T> b = B[(int64_t)j * sp];
#pragma unroll
                    for (int e = 0; e < V; ++e) acc[e] = fma(sd[j], (double)b.e[e], acc[e]);
                }
#pragma unroll
                for (int e = 0; e < V; ++e) x[p * V + e] = acc[e];
            } else {
                FF acc[V];
#pragma unroll
                for (int e = 0; e < V; ++e) acc[e] = FF{0.f, 0.f};
#pragma unroll 4
                for (int j = 0; j < jn; ++j) {
                    const Pack<T> b = B[(int64_t)j * sp];
#pragma unroll
                    for (int e = 0; e < V; ++e) {
                        const float v = (float)b.e[e];
                        ff_add_prod(acc[e], sh[j], v);
                        acc[e].lo += sl[j] * v;
                    }
                }
#pragma unroll
                for (int e = 0; e < V; ++e) x[p * V + e] = (j0 ? x[p * V + e] : 0.0) + ((double)acc[e].hi + (double)acc[e].lo);
            }
        }
        for (int64_t i = np * V + tid; i < n; i += stride) {
            if (sizeof(T) == 8) {
                double acc = j0 ? x[i] : 0.0;
                for (int j = 0; j < jn; ++j) acc = fma(sd[j], (double)basis[(int64_t)(j0 + j) * n + i], acc);
                x[i] = acc;
            } else {
                FF acc{0.f, 0.f};
                for (int j = 0; j < jn; ++j) {
                    const float v = (float)basis[(int64_t)(j0 + j) * n + i];
                    ff_add_prod(acc, sh[j], v);
                    acc.lo += sl[j] * v;
                }
                x[i] = (j0 ? x[i] : 0.0) + ((double)acc.hi + (double)acc.lo);
            }
        }
    }
}

// x += sum_{t < cnt} (s_{j0+t} / g_{j0+t}) u_t for up to three consecutive
// Lanczos vectors (second pass), x = 0 before the first; FP32 values enter
// exactly
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_ritz_accum3(const T *__restrict__ u0, const T *__restrict__ u1,
                                                             const T *__restrict__ u2, int cnt, const double *s,
                                                             const double *scal, int j0, int64_t n,
                                                             double *__restrict__ x) {
    const double c0 = s[j0] * scal[kScal * j0];
    const double c1 = cnt > 1 ? s[j0 + 1] * scal[kScal * (j0 + 1)] : 0.0;
    const double c2 = cnt > 2 ? s[j0 + 2] * scal[kScal * (j0 + 2)] : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = j0 ? x[i] : 0.0;
        acc = fma(c0, (double)u0[i], acc);
        if (cnt > 1) acc = fma(c1, (double)u1[i], acc);
        if (cnt > 2) acc = fma(c2, (double)u2[i], acc);
        x[i] = acc;
    }
}

// The same sum for FP32 vectors in FP32 arithmetic: x holds an unevaluated
// pair (hi, lo) of floats in each 8-byte slot, every term is added as the
// exact FP32 product of the coefficient's leading part plus the product with
// its trailing part (c = c_hi + c_lo), in two-float sums -- about 2^-48 of
// each term, with FP32 instructions only (the FP64 pipe of this GPU runs the
// FP64 version of this sum at a third of the memory rate).  k_ritz_finish_ff
// turns the pairs into doubles once the sum is complete.
__global__ void __launch_bounds__(kRedThreads) k_ritz_accum3_ff(const float *__restrict__ u0, const float *__restrict__ u1,
                                                                const float *__restrict__ u2, int cnt, const double *s,
                                                                const double *scal, int j0, int64_t n,
                                                                float2 *__restrict__ x2) {
    float ch[3], cl[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const double c = t < cnt ? s[j0 + t] * scal[kScal * (j0 + t)] : 0.0;
        ch[t] = (float)c;
        cl[t] = (float)(c - (double)ch[t]);
    }
    const int64_t np = n / 4;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = tid; p < np; p += stride) {
        float4 a[3];
        a[0] = __ldcs(reinterpret_cast<const float4 *>(u0) + p);
        a[1] = cnt > 1 ? __ldcs(reinterpret_cast<const float4 *>(u1) + p) : make_float4(0.f, 0.f, 0.f, 0.f);
        a[2] = cnt > 2 ? __ldcs(reinterpret_cast<const float4 *>(u2) + p) : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 xa = make_float4(0.f, 0.f, 0.f, 0.f), xb = xa;
        if (j0) {
            xa = reinterpret_cast<const float4 *>(x2)[2 * p];
            xb = reinterpret_cast<const float4 *>(x2)[2 * p + 1];
        }
        FF acc[4] = {{xa.x, xa.y}, {xa.z, xa.w}, {xb.x, xb.y}, {xb.z, xb.w}};
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            if (t >= cnt) break;
            const float v[4] = {a[t].x, a[t].y, a[t].z, a[t].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                ff_add_prod(acc[e], ch[t], v[e]);
                acc[e].lo = fmaf(cl[t], v[e], acc[e].lo);
            }
        }
        reinterpret_cast<float4 *>(x2)[2 * p] = make_float4(acc[0].hi, acc[0].lo, acc[1].hi, acc[1].lo);
        reinterpret_cast<float4 *>(x2)[2 * p + 1] = make_float4(acc[2].hi, acc[2].lo, acc[3].hi, acc[3].lo);
    }
    for (int64_t i = np * 4 + tid; i < n; i += stride) {
        FF acc = j0 ? FF{x2[i].x, x2[i].y} : FF{0.f, 0.f};
        const float v[3] = {u0[i], cnt > 1 ? u1[i] : 0.f, cnt > 2 ? u2[i] : 0.f};
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            if (t >= cnt) break;
            ff_add_prod(acc, ch[t], v[t]);
            acc.lo = fmaf(cl[t], v[t], acc.lo);
        }
        x2[i] = make_float2(acc.hi, acc.lo);
    }
}

// x[i] = hi + lo in FP64, in place (each thread reads and writes its own slots)
__global__ void __launch_bounds__(kRedThreads) k_ritz_finish_ff(double *__restrict__ x, int64_t n) {
    const float2 *x2 = reinterpret_cast<const float2 *>(x);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = x2[i];
        x[i] = (double)v.x + (double)v.y;
    }
}

// FP64 dots <a,b> partials (refinement)
__global__ void __launch_bounds__(kRedThreads) k_dot64(const double *__restrict__ a, const double *__restrict__ b,
                                                       int64_t n, double *part) {
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc = fma(a[i], b[i], acc);
    const double r = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = r;
}

// |Hx - E x|^2 partials
__global__ void __launch_bounds__(kRedThreads) k_resid64(const double *__restrict__ hx, const double *__restrict__ x,
                                                         const double *E, int64_t n, double *part) {
    const double e = E[0];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double r = hx[i] - e * x[i];
        acc = fma(r, r, acc);
    }
    const double r = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = r;
}

__global__ void __launch_bounds__(kRedThreads) k_sum(const double *part, int nparts, double *out) {
    double v = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += part[i];
    const double s = block_sum(v);
    if (threadIdx.x == 0) out[0] = s;
}

// start vector: v0 = s / |s| in the working precision (the mixed path
// rounds s to FP32 first); |s| from the rounded values
template <typename T>
__global__ void k_cast_start(const double *__restrict__ s, T *__restrict__ v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (T)s[i];
}

template <typename T>
__global__ void k_scale_start(T *__restrict__ v, const double *nrm2, int64_t n) {
    const double inv = 1.0 / sqrt(nrm2[0]);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (T)((double)v[i] * inv);
}

// ------------------------------------------------------------------ driver

struct Lz {
    LzOp op;
    int64_t n;
    int fp;            // 32 or 64
    int iters, reorth, store;
    int in_basis = 0;  // the stored basis slots are the working vectors (eager launches only)
    int fuse_t = 0;    // the update writes X^T for the next H·v (k_step2_t)
    int head = 0;      // without a stored basis: leading vectors u_0 .. u_{head-1} kept by the first run
    int64_t part_cap = 0;  // partial sums the part buffer holds before its second-stage block (kReduceBlocks)
    void *xt = nullptr;
    int grid;
    double tol = 0.0;
    cudaStream_t st;
    // work buffers live in the handle (kept between calls)
    DevBuf &state, &alpha, &beta, &scal, &part, &coef, &tri, &svec, &work, &ritz_tmp;
    DevBuf *buf;
    DevBuf &basis, &x, &hx;
    std::vector<cudaEvent_t> evs;   // profile: 5 events per H·v (stage boundaries)
    explicit Lz(const LzOp &o)
        : op(o), state(o.work->state), alpha(o.work->alpha), beta(o.work->beta), scal(o.work->scal),
          part(o.work->part), coef(o.work->coef), tri(o.work->tri), svec(o.work->svec), work(o.work->work),
          ritz_tmp(o.work->ritz), buf(o.work->buf), basis(o.work->basis), x(o.work->x), hx(o.work->hx) {}
    // y = A x in precision fp (the sector Hamiltonian's H·v records the stage events)
    int apply(const void *xin, void *yout, int fp, cudaStream_t s, cudaEvent_t *ev = nullptr) const {
        if (op.ham) return hv_launch(op.ham, xin, yout, fp, s, ev);
        if (ev)
            for (int e = 0; e < 5; ++e) cudaEventRecord(ev[e], s);
        return op.apply(op.obj, xin, yout, fp, s);
    }
    bool factored() const { return op.ham && hv_is_factored(op.ham); }
};

// grows a handle-owned buffer to at least bytes (contents not kept)
static int grow(DevBuf &b, size_t bytes) {
    if (b.p && b.bytes >= bytes) return GBR_OK;
    return b.alloc(bytes);
}

template <typename T>
static int lz_step(Lz &z, int phase, bool pass2, cudaEvent_t *ev4, bool want_ritz, int kh = -1, bool first = false) {
    // three rotating buffers: u_k in B[phase], u_{k-1} in B[phase + 2],
    // w (then u_{k+1}) in B[phase + 1] (indices mod 3), which held u_{k-2};
    // the next step uses phase + 1.  With in_basis (eager launches, host step
    // kh), u_{k-1}, u_k and w are the basis slots k-1, k, k+1 instead, which
    // saves the copy of u_{k+1} into its slot.
    const int64_t n = z.n;
    T *v = z.buf[phase].as<T>(), *vprev = z.buf[(phase + 2) % 3].as<T>(), *w = z.buf[(phase + 1) % 3].as<T>();
    const bool basis_slots = z.in_basis && !pass2 && kh >= 0;
    if (basis_slots) {
        T *bs = z.basis.as<T>();
        v = bs + (int64_t)kh * n;
        vprev = kh > 0 ? bs + (int64_t)(kh - 1) * n : v;
        w = bs + (int64_t)(kh + 1) * n;
    }
    LzState *st = z.state.as<LzState>();
    double *part = z.part.as<double>();
    int64_t nk = 0;
    int nparts = z.grid;
    bool updated = false;
    if (z.factored()) {
        // w = H v - beta_k v_{k-1} and the partials of <w, v> in the H·v
        // epilogue; in the second run (alpha_k stored) the epilogue also
        // finishes the step and writes X^T of u_{k+1} when it can
        LzHook hook{vprev, z.scal.as<double>(), &st->k, pass2 ? nullptr : part};
        if (pass2 && z.fuse_t) hook.xt_next = z.xt;
        // X^T comes from the previous step's update except in each pass's first step
        int rc = hv_launch_lz(z.op.ham, v, w, z.fp, z.st, ev4, hook, &nparts, z.fuse_t && !first, &updated);
        if (rc) return rc;
    } else {
        int rc = z.apply(v, w, z.fp, z.st, ev4);
        if (rc) return rc;
        k_step1<T><<<z.grid, kRedThreads, 0, z.st>>>(st, z.scal.as<double>(), vprev, v, w, n, part, pass2 ? 0 : 1);
        ++nk;
    }
    // alpha (which 0) or beta (which 1) from np partial sums, through the
    // first-stage reduction when there are many
    auto finalize = [&](int np, int which) {
        const double *src = part;
        if (np > kReduceAbove) {
            double *p2 = part + z.part_cap;
            k_reduce_parts<<<kReduceBlocks, kRedThreads, 0, z.st>>>(st, part, np, p2);
            ++nk;
            src = p2;
            np = kReduceBlocks;
        }
        k_finalize<<<1, kFinThreads, 0, z.st>>>(st, z.alpha.as<double>(), z.beta.as<double>(), z.scal.as<double>(), src,
                                                np, which, z.iters);
        ++nk;
    };
    if (!pass2) finalize(nparts, 0);
    // the update also writes u_{k+1} into its basis slot: every slot with a
    // stored basis (with re-orthogonalisation the slot is written after it),
    // the first z.head slots with a kept head of the basis
    T *slot_basis = nullptr;
    int slots = 0;
    if (!pass2 && z.store && !z.reorth && !basis_slots) {
        slot_basis = z.basis.as<T>();
        slots = z.iters + 1;
    } else if (!pass2 && !z.store && z.head > 0) {
        slot_basis = z.basis.as<T>();
        slots = z.head;
    }
    int nparts2 = z.grid;
    if (updated) {
        // u_{k+1} and its transpose came out of the H·v (second run only)
    } else if (z.fuse_t) {
        const int64_t rows = z.op.ham->up.D, cols = z.op.ham->dn.D;
        const dim3 g((unsigned)((cols + 63) / 64), (unsigned)((rows + 63) / 64));
        k_step2_t<T><<<g, 256, 0, z.st>>>(st, z.scal.as<double>(), v, w, (T *)z.xt, slot_basis, slots, rows, cols, part,
                                          pass2 ? 0 : 1);
        nparts2 = (int)(g.x * g.y);
        ++nk;
    } else {
        k_step2<T><<<z.grid, kRedThreads, 0, z.st>>>(st, z.scal.as<double>(), v, w, slot_basis, slots, n, part,
                                                    (pass2 || z.reorth) ? 0 : 1);
        ++nk;
    }
    if (z.reorth && !pass2) {
        T *basis = z.basis.as<T>();
        const int gj = std::max(1, std::min<int>(z.grid, (int)((n + kRedThreads - 1) / kRedThreads)));
        for (int pass = 0; pass < 2; ++pass) {
            dim3 g(gj, z.iters);
            k_multidot<T><<<g, kRedThreads, 0, z.st>>>(st, basis, w, n, part);
            k_multidot_fin<<<z.iters, kRedThreads, 0, z.st>>>(st, z.scal.as<double>(), part, gj, z.coef.as<double>());
            k_multiaxpy<T><<<z.grid, kRedThreads, 0, z.st>>>(st, basis, z.coef.as<double>(), w, n, pass == 1);
            nk += 3;
        }
        k_norm2<T><<<z.grid, kRedThreads, 0, z.st>>>(st, w, n, part);
        ++nk;
    }
    if (!pass2) finalize(nparts2, 1);
    if (z.tol > 0.0 && !pass2) {
        k_conv_check<<<1, 32, 0, z.st>>>(st, z.alpha.as<double>(), z.beta.as<double>(), z.tol, z.work.as<double>());
        ++nk;
    }
    if (want_ritz) {
        k_tridiag<<<1, kRedThreads, 0, z.st>>>(st, z.alpha.as<double>(), z.beta.as<double>(), 0, z.tri.as<double>(),
                                               nullptr, nullptr);
        k_copy_ritz<<<1, 32, 0, z.st>>>(st, z.tri.as<double>(), z.ritz_tmp.as<double>());
        nk += 2;
    }
    k_advance<<<1, 32, 0, z.st>>>(st);
    nk += 1;
    count_launches(nk);
    GBR_LAUNCH_CHECK();
    return GBR_OK;
}

template <typename T>
static int lz_run(Lz &z, const double *d_v0, gbr_lanczos_result *res, const gbr_lanczos_opts *o, double *h_alpha,
                  double *h_beta, double *h_ritz) {
    const int64_t n = z.n;
    cudaStream_t s = z.st;
    LzState zero{};
    GBR_CUDA_TRY(cudaMemcpyAsync(z.state.p, &zero, sizeof(zero), cudaMemcpyHostToDevice, s));
    GBR_CUDA_TRY(cudaMemsetAsync(z.beta.p, 0, sizeof(double) * (size_t)(z.iters + 2), s));
    GBR_CUDA_TRY(cudaMemsetAsync(z.alpha.p, 0, sizeof(double) * (size_t)(z.iters + 2), s));
    GBR_CUDA_TRY(cudaMemsetAsync(z.scal.p, 0, sizeof(double) * kScal * (size_t)(z.iters + 2), s));
    static const double scal0 = 1.0;   // 1/g_0
    GBR_CUDA_TRY(cudaMemcpyAsync(z.scal.p, &scal0, sizeof(double), cudaMemcpyHostToDevice, s));
    T *B0 = z.buf[0].as<T>();
    k_cast_start<T><<<z.grid, kRedThreads, 0, s>>>(d_v0, B0, n);
    k_norm2<T><<<z.grid, kRedThreads, 0, s>>>(z.state.as<LzState>(), B0, n, z.part.as<double>());
    k_sum<<<1, kRedThreads, 0, s>>>(z.part.as<double>(), z.grid, z.tri.as<double>() + 1);
    k_scale_start<T><<<z.grid, kRedThreads, 0, s>>>(B0, z.tri.as<double>() + 1, n);
    if (z.store || z.head > 0) GBR_CUDA_TRY(cudaMemcpyAsync(z.basis.p, B0, (size_t)n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    GBR_LAUNCH_CHECK();
    count_launches(4);

    cudaEvent_t e0, e1;
    cudaEventCreate(&e0); cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    // graph mode: one graph per buffer phase, captured on a private stream
    // after two eager steps (which also set kernel attributes), replayed on s
    const bool graphs = o->use_graph && !o->profile;
    // every basis slot starts on a 16-byte boundary (the step kernels load
    // 16-byte packs) only when a vector is a whole number of packs
    z.in_basis = (z.store && !z.reorth && !graphs && ((size_t)z.n * sizeof(T)) % 16 == 0) ? 1 : 0;
    // the tiled update that also writes X^T (and the basis slot): factored
    // H·v, no re-orthogonalisation (which changes w after the update), and
    // dimensions that are whole 16-byte packs
    {
        const int64_t V = 16 / (int64_t)sizeof(T);
        z.fuse_t = (z.factored() && !z.reorth && z.op.ham->up.D % V == 0 && z.op.ham->dn.D % V == 0 &&
                    (z.op.ham->up.D + 63) / 64 <= 65535) ? 1 : 0;
        z.xt = z.fuse_t ? hv_xt_scratch(z.op.ham, z.fp) : nullptr;
        if (z.fuse_t && !z.xt) return set_error(GBR_ENOMEM, "scratch for X^T");
    }
    cudaGraphExec_t gexec[3] = {nullptr, nullptr, nullptr};
    int64_t gnodes[3] = {0, 0, 0};
    cudaStream_t cap = nullptr;
    if (graphs) GBR_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    int rc = GBR_OK;
    int phase = 0;
    const bool want_ritz = h_ritz != nullptr;
    for (int k = 0; k < z.iters; ++k) {
        if (graphs && k >= 2) {
            if (!gexec[phase]) {
                cudaStream_t keep = z.st;
                z.st = cap;
                const int64_t before = launch_count();
                GBR_CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
                rc = lz_step<T>(z, phase, false, nullptr, want_ritz);
                cudaGraph_t g = nullptr;
                cudaError_t ce = cudaStreamEndCapture(cap, &g);
                z.st = keep;
                gnodes[phase] = launch_count() - before;   // captured, not yet run
                set_launch_count(before);
                if (rc) { if (g) cudaGraphDestroy(g); break; }
                if (ce != cudaSuccess) { rc = set_error(GBR_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce)); break; }
                ce = cudaGraphInstantiate(&gexec[phase], g, 0);
                cudaGraphDestroy(g);
                if (ce != cudaSuccess) { rc = set_error(GBR_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(ce)); break; }
            }
            cudaError_t le = cudaGraphLaunch(gexec[phase], s);
            if (le != cudaSuccess) { rc = set_error(GBR_ECUDA, "graph launch failed: %s", cudaGetErrorString(le)); break; }
            count_launches(gnodes[phase]);
        } else {
            cudaEvent_t *ev4 = nullptr;
            if (o->profile) {
                for (int e = 0; e < 5; ++e) {
                    cudaEvent_t ev;
                    GBR_CUDA_TRY(cudaEventCreate(&ev));
                    z.evs.push_back(ev);
                }
                ev4 = z.evs.data() + z.evs.size() - 5;
            }
            rc = lz_step<T>(z, phase, false, ev4, want_ritz, k, k == 0);
            if (rc) break;
        }
        phase = (phase + 1) % 3;
        if ((k & 31) == 31) {
            LzState hs;
            cudaError_t ce = cudaMemcpyAsync(&hs, z.state.p, sizeof(hs), cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) { rc = set_error(GBR_ECUDA, "sync failed: %s", cudaGetErrorString(ce)); break; }
            if (hs.stop) break;
        }
    }
    for (int p = 0; p < 3; ++p)
        if (gexec[p]) cudaGraphExecDestroy(gexec[p]);
    if (cap) cudaStreamDestroy(cap);
    if (rc) return rc;
    LzState hs;
    GBR_CUDA_TRY(cudaMemcpyAsync(&hs, z.state.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
    GBR_CUDA_TRY(cudaStreamSynchronize(s));
    // steps done: k (advanced once per completed non-final step) + 1 for the step that set stop
    const int kdone = std::min(z.iters, hs.k + 1);
    res->iters_done = kdone;
    if (hs.nonfinite)
        return set_error(GBR_ENONFINITE, "Lanczos step %d produced a non-finite alpha or beta (NaN or Inf in the "
                         "start vector or the operator)", hs.k);
    res->breakdown = hs.breakdown;
    res->converged = hs.converged;
    res->stored_basis = z.store;
    // lowest Ritz value of T_kdone
    double *tri = z.tri.as<double>();
    k_tridiag<<<1, kRedThreads, 0, s>>>(z.state.as<LzState>(), z.alpha.as<double>(), z.beta.as<double>(), kdone, tri,
                                       nullptr, z.work.as<double>());
    GBR_LAUNCH_CHECK();
    count_launches(1);
    double Er = 0.0;
    GBR_CUDA_TRY(cudaMemcpyAsync(&Er, tri, 8, cudaMemcpyDeviceToHost, s));
    GBR_CUDA_TRY(cudaStreamSynchronize(s));
    res->E_ritz = Er;
    res->E0 = Er;
    res->residual = -1.0;
    if (o->refine) {
        DevBuf &x = z.x, &hx = z.hx;
        if ((rc = grow(x, (size_t)n * 8))) return rc;
        if ((rc = grow(hx, (size_t)n * 8))) return rc;
        double *sv = z.svec.as<double>();
        // the Ritz vector of the converged prefix T_kr, then its eigenvector s
        int *kbuf = reinterpret_cast<int *>(tri + 8);
        const double unit = sizeof(T) == 4 ? 5.9604644775390625e-8 : 1.1102230246251565e-16;
        k_ritz_prefix<<<1, 32, 0, s>>>(z.state.as<LzState>(), z.alpha.as<double>(), z.beta.as<double>(), kdone, unit,
                                       z.work.as<double>(), kbuf);
        int kr = kdone;
        GBR_CUDA_TRY(cudaMemcpyAsync(&kr, kbuf, sizeof(int), cudaMemcpyDeviceToHost, s));
        GBR_CUDA_TRY(cudaStreamSynchronize(s));
        if (kr < 1 || kr > kdone) kr = kdone;
        k_tridiag<<<1, kRedThreads, 0, s>>>(z.state.as<LzState>(), z.alpha.as<double>(), z.beta.as<double>(), kr,
                                           tri + 4, sv, z.work.as<double>());
        count_launches(2);
        GBR_LAUNCH_CHECK();
        // terms of the Ritz sum: drop the trailing coefficients whose norm is
        // at most ritz_tail (s is normalised by the tridiagonal solver)
        int nterm = kr;
        if (o->ritz_tail > 0.0 && kr > 1) {
            std::vector<double> hs((size_t)kr);
            GBR_CUDA_TRY(cudaMemcpyAsync(hs.data(), sv, sizeof(double) * (size_t)kr, cudaMemcpyDeviceToHost, s));
            GBR_CUDA_TRY(cudaStreamSynchronize(s));
            double s2 = 0.0;
            for (double v : hs) s2 += v * v;
            const double lim = o->ritz_tail * o->ritz_tail * s2;
            double tail = 0.0;
            while (nterm > 1 && tail + hs[(size_t)(nterm - 1)] * hs[(size_t)(nterm - 1)] <= lim) {
                tail += hs[(size_t)(nterm - 1)] * hs[(size_t)(nterm - 1)];
                --nterm;
            }
        }
        res->ritz_terms = nterm;
        res->basis_head = (!z.store && z.head >= 2) ? std::min(z.head, nterm) : 0;
        if (z.store) {
            k_ritz_from_basis<T><<<z.grid, kRedThreads, 0, s>>>(z.basis.as<T>(), sv, z.scal.as<double>(), nterm, n,
                                                                x.as<double>());
            count_launches(1);
        } else {
            // the Ritz sum takes the vectors three at a time (one pass over x
            // per three): first the head of the basis the first run kept
            // (u_0 .. u_{m-1}), then the rest from a second run of the same
            // recurrence with the stored scalars, restarted from the head's
            // last two vectors (from the start vector without a head)
            const int m = (z.head >= 2) ? std::min(z.head, nterm) : 0;
            auto accum = [&](const T *u0, const T *u1, const T *u2, int cnt, int j0) {
                if (sizeof(T) == 4)
                    k_ritz_accum3_ff<<<z.grid, kRedThreads, 0, s>>>((const float *)u0, (const float *)u1,
                                                                    (const float *)u2, cnt, sv, z.scal.as<double>(), j0,
                                                                    n, x.as<float2>());
                else
                    k_ritz_accum3<T><<<z.grid, kRedThreads, 0, s>>>(u0, u1, u2, cnt, sv, z.scal.as<double>(), j0, n,
                                                                  x.as<double>());
                count_launches(1);
            };
            const T *hb = z.basis.as<T>();
            for (int j0 = 0; j0 < m; j0 += 3) {
                const int cnt = std::min(3, m - j0);
                const T *u0 = hb + (int64_t)j0 * n;
                accum(u0, cnt > 1 ? u0 + n : u0, cnt > 2 ? u0 + 2 * n : u0, cnt, j0);
            }
            if (nterm > m) {
                int jstart = 0;
                if (m >= 2) {
                    LzState rs{};
                    rs.k = m - 1;
                    GBR_CUDA_TRY(cudaMemcpyAsync(z.state.p, &rs, sizeof(rs), cudaMemcpyHostToDevice, s));
                    GBR_CUDA_TRY(cudaMemcpyAsync(z.buf[(m - 2) % 3].p, hb + (int64_t)(m - 2) * n, (size_t)n * sizeof(T),
                                                 cudaMemcpyDeviceToDevice, s));
                    GBR_CUDA_TRY(cudaMemcpyAsync(z.buf[(m - 1) % 3].p, hb + (int64_t)(m - 1) * n, (size_t)n * sizeof(T),
                                                 cudaMemcpyDeviceToDevice, s));
                    jstart = m - 1;
                } else {
                    LzState zero2{};
                    GBR_CUDA_TRY(cudaMemcpyAsync(z.state.p, &zero2, sizeof(zero2), cudaMemcpyHostToDevice, s));
                    k_cast_start<T><<<z.grid, kRedThreads, 0, s>>>(d_v0, B0, n);
                    k_norm2<T><<<z.grid, kRedThreads, 0, s>>>(z.state.as<LzState>(), B0, n, z.part.as<double>());
                    k_sum<<<1, kRedThreads, 0, s>>>(z.part.as<double>(), z.grid, z.tri.as<double>() + 1);
                    k_scale_start<T><<<z.grid, kRedThreads, 0, s>>>(B0, z.tri.as<double>() + 1, n);
                    count_launches(4);
                }
                // u_j sits in buffer j mod 3 until step j + 2 overwrites it
                int ph = jstart % 3, j0 = m;
                for (int j = jstart; j < nterm; ++j) {
                    if (j >= m && ((j - m) % 3 == 2 || j + 1 == nterm)) {
                        const int cnt = j - j0 + 1;
                        const T *u0 = z.buf[j0 % 3].as<T>();
                        accum(u0, cnt > 1 ? z.buf[(j0 + 1) % 3].as<T>() : u0, cnt > 2 ? z.buf[(j0 + 2) % 3].as<T>() : u0,
                              cnt, j0);
                        j0 = j + 1;
                    }
                    if (j + 1 < nterm) {
                        rc = lz_step<T>(z, ph, true, nullptr, false, -1, j == jstart);
                        if (rc) return rc;
                    }
                    ph = (ph + 1) % 3;
                }
            }
            if (sizeof(T) == 4) {
                k_ritz_finish_ff<<<z.grid, kRedThreads, 0, s>>>(x.as<double>(), n);
                count_launches(1);
            }
        }
        GBR_LAUNCH_CHECK();
        if ((rc = z.apply(x.p, hx.p, 64, s))) return rc;
        double *part = z.part.as<double>();
        k_dot64<<<z.grid, kRedThreads, 0, s>>>(x.as<double>(), hx.as<double>(), n, part);
        k_sum<<<1, kRedThreads, 0, s>>>(part, z.grid, tri + 2);
        k_dot64<<<z.grid, kRedThreads, 0, s>>>(x.as<double>(), x.as<double>(), n, part);
        k_sum<<<1, kRedThreads, 0, s>>>(part, z.grid, tri + 3);
        GBR_LAUNCH_CHECK();
        count_launches(4);
        double hd[2];
        GBR_CUDA_TRY(cudaMemcpyAsync(hd, tri + 2, 16, cudaMemcpyDeviceToHost, s));
        GBR_CUDA_TRY(cudaStreamSynchronize(s));
        const double E = hd[0] / hd[1];
        GBR_CUDA_TRY(cudaMemcpyAsync(tri + 4, &E, 8, cudaMemcpyHostToDevice, s));
        k_resid64<<<z.grid, kRedThreads, 0, s>>>(hx.as<double>(), x.as<double>(), tri + 4, n, part);
        k_sum<<<1, kRedThreads, 0, s>>>(part, z.grid, tri + 5);
        count_launches(2);
        double r2 = 0.0;
        GBR_CUDA_TRY(cudaMemcpyAsync(&r2, tri + 5, 8, cudaMemcpyDeviceToHost, s));
        GBR_CUDA_TRY(cudaStreamSynchronize(s));
        res->E0 = E;
        res->residual = sqrt(fmax(r2, 0.0) / hd[1]);
    }
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    res->seconds = ms * 1e-3;
    res->hv_seconds = 0.0;
    for (size_t e = 0; e + 4 < z.evs.size(); e += 5) {
        for (int st3 = 0; st3 < 4; ++st3) {
            float t = 0.f;
            cudaEventElapsedTime(&t, z.evs[e + st3], z.evs[e + st3 + 1]);
            res->stage_seconds[st3] += t * 1e-3;
            res->stage_launches[st3] += 1;
            res->hv_seconds += t * 1e-3;
        }
    }
    for (cudaEvent_t ev : z.evs) cudaEventDestroy(ev);
    z.evs.clear();
    cudaEventDestroy(e0); cudaEventDestroy(e1);
    if (h_alpha) GBR_CUDA_TRY(cudaMemcpy(h_alpha, z.alpha.p, sizeof(double) * (size_t)kdone, cudaMemcpyDeviceToHost));
    if (h_beta && kdone > 1)
        GBR_CUDA_TRY(cudaMemcpy(h_beta, z.beta.as<double>() + 1, sizeof(double) * (size_t)(kdone - 1), cudaMemcpyDeviceToHost));
    if (h_ritz) GBR_CUDA_TRY(cudaMemcpy(h_ritz, z.ritz_tmp.p, sizeof(double) * (size_t)kdone, cudaMemcpyDeviceToHost));
    return GBR_OK;
}

}  // namespace gbr

namespace gbr {

// rcp64 against the IEEE division on n values x_i = +-10^e, e spread over
// [-29, 29] with a splitmix-style integer hash of i for the mantissa and
// sign; each CTA writes its largest relative error.
__global__ void __launch_bounds__(kRedThreads) k_check_rcp64(int64_t n, double *part) {
    double worst = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + 0x2545F4914F6CDD1Dull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const double m = 1.0 + (double)(z >> 12) * 0x1.0p-52;                // [1, 2)
        const double e = -29.0 + 58.0 * (double)((z >> 4) & 0xFFu) / 255.0;  // [-29, 29]
        const double x = ((z & 1u) ? -m : m) * exp10(e);
        const double exact = 1.0 / x;
        const double err = fabs(rcp64(x) - exact) / fabs(exact);
        worst = fmax(worst, err);
    }
    for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_down_sync(0xFFFFFFFFu, worst, o));
    __shared__ double red[kRedThreads / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = worst;
    __syncthreads();
    if (threadIdx.x == 0) {
        double w = 0.0;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) w = fmax(w, red[j]);
        part[blockIdx.x] = w;
    }
}

}  // namespace gbr

using namespace gbr;

// The stored basis (or its kept head) is a solve's one large allocation (105
// GB for 200 FP32 steps on the 4x4 sector).  A finished call leaves it in a
// process-wide cache instead of in the handle; the next call on the same
// device takes it when it is large enough, so repeated solves, also on new
// handles, neither allocate nor free it.  gbr_release_cache frees it, and a
// solve whose working vectors do not fit beside it frees it first.
namespace gbr {
static std::mutex g_cache_mu;
static void *g_cache_p = nullptr;
static size_t g_cache_bytes = 0;
static int g_cache_dev = -1;

static int current_device() {
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess) return -1;
    return d;
}

static void free_on(void *p, int dev) {
    const int cur = current_device();
    if (dev >= 0 && dev != cur) cudaSetDevice(dev);
    cudaFree(p);
    if (dev >= 0 && dev != cur && cur >= 0) cudaSetDevice(cur);
}

// cached bytes usable on the current device
static size_t cache_bytes_here() {
    std::lock_guard<std::mutex> g(g_cache_mu);
    return (g_cache_p && g_cache_dev == current_device()) ? g_cache_bytes : 0;
}

// moves the cached basis into b when b is smaller than need and the cache is
// not; a cached buffer on this device too small for need is freed (the
// free-memory test counted it as available for the new allocation)
static void cache_take(DevBuf &b, size_t need) {
    std::lock_guard<std::mutex> g(g_cache_mu);
    if (!g_cache_p || g_cache_dev != current_device() || (b.p && b.bytes >= need)) return;
    if (g_cache_bytes < need) {
        free_on(g_cache_p, g_cache_dev);
        g_cache_p = nullptr;
        g_cache_bytes = 0;
        g_cache_dev = -1;
        return;
    }
    b.release();
    b.p = g_cache_p;
    b.bytes = g_cache_bytes;
    g_cache_p = nullptr;
    g_cache_bytes = 0;
    g_cache_dev = -1;
}

// moves b into the cache unless the cache holds a larger buffer
static void cache_put(DevBuf &b) {
    if (!b.p) return;
    std::lock_guard<std::mutex> g(g_cache_mu);
    if (g_cache_p && g_cache_bytes >= b.bytes) return;
    if (g_cache_p) free_on(g_cache_p, g_cache_dev);
    g_cache_p = b.p;
    g_cache_bytes = b.bytes;
    g_cache_dev = current_device();
    b.p = nullptr;
    b.bytes = 0;
}

// frees the cached basis when it is on the current device
static void cache_drop_here() {
    std::lock_guard<std::mutex> g(g_cache_mu);
    if (!g_cache_p || g_cache_dev != current_device()) return;
    free_on(g_cache_p, g_cache_dev);
    g_cache_p = nullptr;
    g_cache_bytes = 0;
    g_cache_dev = -1;
}
}  // namespace gbr

extern "C" int gbr_release_cache(void) {
    clear_error();
    std::lock_guard<std::mutex> g(g_cache_mu);
    if (g_cache_p) free_on(g_cache_p, g_cache_dev);
    g_cache_p = nullptr;
    g_cache_bytes = 0;
    g_cache_dev = -1;
    return GBR_OK;
}

extern "C" int gbr_check_rcp64(int64_t n, double *h_max_rel_err) {
    clear_error();
    if (n < 1 || !h_max_rel_err) return set_error(GBR_EINVAL, "bad arguments");
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + kRedThreads - 1) / kRedThreads, 1024));
    DevBuf part;
    int rc = part.alloc(sizeof(double) * (size_t)grid);
    if (rc) return rc;
    k_check_rcp64<<<grid, kRedThreads>>>(n, part.as<double>());
    GBR_LAUNCH_CHECK();
    count_launches(1);
    std::vector<double> h((size_t)grid);
    GBR_CUDA_TRY(cudaMemcpy(h.data(), part.p, sizeof(double) * (size_t)grid, cudaMemcpyDeviceToHost));
    double w = 0.0;
    for (double v : h) w = std::max(w, v);
    *h_max_rel_err = w;
    return GBR_OK;
}

namespace gbr {
int lanczos_solve(const LzOp &op, const gbr_lanczos_opts *o, const double *d_v0, gbr_lanczos_result *res,
                  double *h_alpha, double *h_beta, double *h_ritz, void *stream) {
    if (!o || !res || !d_v0) return set_error(GBR_EINVAL, "NULL argument");
    if (o->iters < 1 || o->iters > 65535) return set_error(GBR_EINVAL, "iters=%d out of range 1..65535", o->iters);
    if (o->prec != GBR_PREC_FP64 && o->prec != GBR_PREC_MIXED) return set_error(GBR_EINVAL, "unknown prec %d", o->prec);
    if (!(o->ritz_tail >= 0.0 && o->ritz_tail < 1.0)) return set_error(GBR_EINVAL, "ritz_tail must be in [0, 1)");
    if ((uintptr_t)d_v0 & 7u) return set_error(GBR_EINVAL, "v0 must be 8-byte aligned");
    memset(res, 0, sizeof(*res));
    Lz z(op);
    z.n = op.n;
    z.fp = o->prec == GBR_PREC_MIXED ? 32 : 64;
    z.iters = (int)std::min<int64_t>(o->iters, op.n);
    z.reorth = o->reorth ? 1 : 0;
    z.tol = o->tol > 0.0 ? o->tol : 0.0;
    z.st = (cudaStream_t)stream;
    const size_t es = z.fp == 64 ? 8 : 4;
    const size_t basis_bytes = (size_t)(z.iters + 1) * (size_t)z.n * es;
    // the working vectors, the FP64 Ritz vector and its product, and the
    // factored H·v's scratch first, so that what remains free is what a
    // basis can have
    // (the scratch in FP64 size with refinement: its FP64 H·v takes the same
    // buffers).  If they do not fit beside a basis kept from an earlier solve
    // (in the process cache or in this handle), that basis is freed first.
    int rc = GBR_OK;
    for (int attempt = 0; attempt < 2; ++attempt) {
        rc = GBR_OK;
        for (int i = 0; i < 3 && !rc; ++i) rc = grow(z.buf[i], (size_t)z.n * es);
        if (!rc && o->refine) rc = grow(z.x, (size_t)z.n * 8);
        if (!rc && o->refine) rc = grow(z.hx, (size_t)z.n * 8);
        if (!rc && z.factored() && !hv_xt_scratch(op.ham, o->refine ? 64 : z.fp))
            rc = set_error(GBR_ENOMEM, "scratch of the factored H·v");
        if (rc != GBR_ENOMEM || attempt == 1) break;
        cache_drop_here();
        z.basis.release();
        clear_error();
    }
    if (rc) return rc;
    // the basis is needed by re-orthogonalisation; with refinement it makes
    // the Ritz vector one pass instead of a second run of the recurrence
    int store = 0, head = 0;
    if (z.reorth) {
        store = 1;
    } else if (o->refine) {
        store = o->store_basis;
        if (store <= -2) {
            // the caller's head: the leading -store_basis vectors
            head = (int)std::min<int64_t>(-(int64_t)store, (int64_t)z.iters + 1);
            store = 0;
        } else if (store < 0) {
            size_t fr = 0, tot = 0;
            GBR_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
            // the handle's and the process cache's bases are reused or released before a larger one is taken
            fr += z.basis.bytes + cache_bytes_here();
            // 2 GB to spare for the smaller buffers
            const size_t fixed = (size_t)2 << 30;
            store = basis_bytes + fixed < fr ? 1 : 0;
            if (!store && fr > fixed) {
                // not the whole basis: keep its leading vectors, as many as fit
                // in nine tenths of what is left (at least 8), so that the
                // second run of the recurrence starts after them
                const size_t per = (size_t)z.n * es;
                const size_t fit = (fr - fixed) / 10 * 9 / per;
                head = (int)std::min<size_t>(fit, (size_t)z.iters + 1);
                if (head < 8) head = 0;
            }
        }
    }
    z.store = store;
    // the head's slots follow one another at the vector's length, and the
    // Ritz sum reads them in 16-byte packs: a head only when a vector is a
    // whole number of packs
    if (((size_t)z.n * es) % 16 != 0) head = 0;
    z.head = store ? 0 : head;
    const int64_t blocks = (z.n + kRedThreads - 1) / kRedThreads;
    z.grid = (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sm_count() * 4));
    if ((rc = grow(z.state, sizeof(LzState)))) return rc;
    if ((rc = grow(z.alpha, sizeof(double) * (size_t)(z.iters + 2)))) return rc;
    if ((rc = grow(z.beta, sizeof(double) * (size_t)(z.iters + 2)))) return rc;
    if ((rc = grow(z.scal, sizeof(double) * kScal * (size_t)(z.iters + 2)))) return rc;
    size_t nparts = (size_t)z.grid * (size_t)(z.reorth ? z.iters + 1 : 1);
    if (op.ham) nparts = std::max(nparts, (size_t)hv_lz_parts(op.ham, z.fp));
    z.part_cap = (int64_t)nparts;
    if ((rc = grow(z.part, sizeof(double) * (nparts + kReduceBlocks)))) return rc;
    if ((rc = grow(z.coef, sizeof(double) * (size_t)(z.iters + 2)))) return rc;
    if ((rc = grow(z.tri, sizeof(double) * 16))) return rc;
    if ((rc = grow(z.svec, sizeof(double) * (size_t)(z.iters + 2)))) return rc;
    if ((rc = grow(z.work, sizeof(double) * 3 * (size_t)(z.iters + 2)))) return rc;
    if ((rc = grow(z.ritz_tmp, sizeof(double) * (size_t)(z.iters + 2)))) return rc;
    if (z.store) {
        cache_take(z.basis, basis_bytes);
        if ((rc = grow(z.basis, basis_bytes))) return rc;
    } else if (z.head > 0) {
        const size_t head_bytes = (size_t)z.head * (size_t)z.n * es;
        cache_take(z.basis, head_bytes);
        if ((rc = grow(z.basis, head_bytes))) return rc;
    }
    rc = z.fp == 64 ? lz_run<double>(z, d_v0, res, o, h_alpha, h_beta, h_ritz)
                    : lz_run<float>(z, d_v0, res, o, h_alpha, h_beta, h_ritz);
    if (z.store || z.head > 0) cache_put(z.basis);
    return rc;
}
}  // namespace gbr

extern "C" int gbr_lanczos(const gbr_ham *H, const gbr_lanczos_opts *o, const double *d_v0, gbr_lanczos_result *res,
                           double *h_alpha, double *h_beta, double *h_ritz, void *stream) {
    clear_error();
    if (!H) return set_error(GBR_EINVAL, "NULL argument");
    const LzOp op{H, nullptr, nullptr, H->D, &const_cast<gbr_ham *>(H)->lzw};
    return lanczos_solve(op, o, d_v0, res, h_alpha, h_beta, h_ritz, stream);
}
