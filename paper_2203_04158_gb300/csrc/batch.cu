// Batched ground states of many small impurity-type models, every
// (N_up, N_dn) sector, in one persistent launch (the impurity-solver use case
// that motivates the paper, Sec. I and VI).
//
// Each CTA takes sectors from a device work queue (largest first) and runs a
// whole mixed-precision Lanczos on one sector inside shared memory: FP32
// vectors, dots in two-float sums finished in FP64, FP64 tridiagonal
// eigenpair, a second pass of the recurrence that forms the Ritz vector in
// FP64, and an FP64 H·v for the Rayleigh quotient.  The H·v is the method of
// the paper on the fly: per element unrank (per-spin lists), diagonal, hops
// with the sign from the popcount of the bits between the two sites, and the
// target's rank by combinadics (Fig. algr) -- the per-spin hop lists are
// ranked once per sector and reused by every step.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "gbr_common.h"
#include "tridiag.cuh"

namespace gbr {

constexpr int kBatchThreads = 256;   // default CTA size of the batch solver
constexpr int kBatchMaxL = 10;

struct SectorDesc {
    int model, L, Nup, Ndn;
    int Dup, Ddn;
    int64_t off;       // start-vector offset
};

struct ModelDev {
    int L;
    double h[kBatchMaxL * kBatchMaxL];
    double U[kBatchMaxL];
};

__device__ __forceinline__ double bsum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
    __syncthreads();
    return r;   // all threads
}

__device__ __forceinline__ void ffp(float &hi, float &lo, float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    const float t = hi + p;
    const float bp = t - hi;
    lo += ((hi - (t - bp)) + (p - bp)) + e;
    hi = t;
}

// k-th (0-based) L-bit pattern with N bits set in increasing order, by
// the greedy combinatorial-number-system unranking (Eq. unrank)
__device__ uint32_t unrank_small(int L, int N, int r, const uint32_t *bin) {
    uint32_t a = 0;
    int c = L - 1;
    for (int k = N; k >= 1; --k) {
        while (c >= 0 && (int)bin[c * (kBatchMaxL + 1) + k] > r) --c;
        a |= 1u << c;
        r -= (int)bin[c * (kBatchMaxL + 1) + k];
        --c;
    }
    return a;
}

// Fig. algr
__device__ __forceinline__ int rank_small(uint32_t a, const uint32_t *bin) {
    int i = 0, k = 1;
    while (a) {
        const int c = __ffs(a) - 1;
        a &= a - 1u;
        i += (int)bin[c * (kBatchMaxL + 1) + k];
        ++k;
    }
    return i;
}

struct SpinLists {
    uint32_t *st;      // states
    uint8_t *cnt;      // hops per state
    uint32_t *ent;     // [state][hmax]: target | bond << 16 | sign << 31
    float *d32;        // one-body diagonal (the FP64 one is summed on the fly)
};

// builds the per-spin state list and hop lists of one spin species
__device__ void build_spin(int L, int N, int D, int hmax, const double *h, const uint8_t *bidx, const uint32_t *bin,
                           SpinLists s) {
    for (int r = threadIdx.x; r < D; r += blockDim.x) {
        const uint32_t a = unrank_small(L, N, r, bin);
        s.st[r] = a;
        double d = 0.0;
        int k = 0;
        for (int p = 0; p < L; ++p) {
            if (!((a >> p) & 1u)) continue;
            d += h[p * L + p];
            for (int q = 0; q < L; ++q) {
                if (q == p || ((a >> q) & 1u) || h[p * L + q] == 0.0) continue;
                const uint32_t b = a ^ ((1u << p) | (1u << q));
                const int lo = min(p, q), hi = max(p, q);
                const uint32_t between = ((1u << hi) - 1u) & ~((1u << (lo + 1)) - 1u);
                const uint32_t sg = (uint32_t)(__popc(a & between) & 1);
                if (k < hmax) s.ent[r * hmax + k] = (uint32_t)rank_small(b, bin) | ((uint32_t)bidx[p * L + q] << 16) | (sg << 31);
                ++k;
            }
        }
        s.cnt[r] = (uint8_t)min(k, hmax);
        s.d32[r] = (float)d;
    }
}

// sum of h_pp over the occupied sites of one spin pattern (ascending p)
__device__ __forceinline__ double diag64(uint32_t a, const double *h, int L) {
    double d = 0.0;
    while (a) {
        const int p = __ffs(a) - 1;
        a &= a - 1u;
        d += h[p * L + p];
    }
    return d;
}

// y = H x on the sector, one element per thread iteration (hs: the L x L
// one-body matrix, for the FP64 diagonal)
template <typename T>
__device__ void hv_small(const SectorDesc &sd, int hmax, const SpinLists &up, const SpinLists &dn, const T *bc,
                         const T *U, const double *hs, const T *x, T *y) {
    const int D = sd.Dup * sd.Ddn;
    for (int i = threadIdx.x; i < D; i += blockDim.x) {
        const int ru = i / sd.Ddn, rd = i - ru * sd.Ddn;
        const uint32_t au = up.st[ru], ad = dn.st[rd];
        T dg = (sizeof(T) == 8) ? (T)(diag64(au, hs, sd.L) + diag64(ad, hs, sd.L)) : (T)(up.d32[ru] + dn.d32[rd]);
        const uint32_t both = au & ad;
        for (int p = 0; p < sd.L; ++p)
            if ((both >> p) & 1u) dg += U[p];
        T acc = dg * x[i];
        for (int k = 0; k < up.cnt[ru]; ++k) {
            const uint32_t e = up.ent[ru * hmax + k];
            const T c = bc[(e >> 16) & 0x7FFFu];
            const T v = x[(int)(e & 0xFFFFu) * sd.Ddn + rd];
            acc += (e >> 31) ? -c * v : c * v;
        }
        for (int k = 0; k < dn.cnt[rd]; ++k) {
            const uint32_t e = dn.ent[rd * hmax + k];
            const T c = bc[(e >> 16) & 0x7FFFu];
            const T v = x[ru * sd.Ddn + (int)(e & 0xFFFFu)];
            acc += (e >> 31) ? -c * v : c * v;
        }
        y[i] = acc;
    }
}

struct BatchSmem {
    int maxD, maxDs, hmax, iters;
    int64_t slot;      // doubles of global scratch per CTA: x, Hx (maxD each), solver work 3 (iters + 2)
};

// xg: per-CTA scratch of lay.slot doubles for the FP64 Ritz vector, its H·v
// and the tridiagonal solver's work (global memory; each CTA reuses its own
// slot, which stays in L2), so that the shared memory holds only the FP32
// recurrence and three CTAs fit on an SM.
//
// NT threads per CTA (128, 256 or 512; the autotuner's choice), at most
// 64 K / (NT x 3 x 256 / NT) registers a thread so that three CTAs fit on an SM
// at 256 and the register budget per SM stays the same at the other sizes.
template <int NT>
__global__ void __launch_bounds__(NT, (NT >= 512 ? 1 : 768 / NT)) k_batch(const SectorDesc *__restrict__ secs, int nsec,
                                                         const ModelDev *__restrict__ models,
                                                         const double *__restrict__ start, int iters, BatchSmem lay,
                                                         int *counter, double *__restrict__ outE, int *__restrict__ outK,
                                                         double *__restrict__ xg) {
    extern __shared__ __align__(16) unsigned char smr[];
    // layout
    unsigned char *p = smr;
    auto take = [&](size_t bytes) { unsigned char *q = p; p += (bytes + 15) & ~(size_t)15; return q; };
    const int maxD = lay.maxD, maxDs = lay.maxDs, hmax = lay.hmax, kmax = lay.iters;
    float *v = (float *)take((size_t)maxD * 4);
    float *vp = (float *)take((size_t)maxD * 4);
    float *w = (float *)take((size_t)maxD * 4);
    double *x = xg + (size_t)blockIdx.x * lay.slot;
    double *hx = x + maxD;
    SpinLists up, dn;
    up.st = (uint32_t *)take((size_t)maxDs * 4); dn.st = (uint32_t *)take((size_t)maxDs * 4);
    up.cnt = (uint8_t *)take((size_t)maxDs); dn.cnt = (uint8_t *)take((size_t)maxDs);
    up.ent = (uint32_t *)take((size_t)maxDs * hmax * 4); dn.ent = (uint32_t *)take((size_t)maxDs * hmax * 4);
    up.d32 = (float *)take((size_t)maxDs * 4); dn.d32 = (float *)take((size_t)maxDs * 4);
    double *alpha = (double *)take((size_t)(kmax + 2) * 8);
    double *beta = (double *)take((size_t)(kmax + 2) * 8);
    double *svec = (double *)take((size_t)(kmax + 2) * 8);
    double *work = xg + (size_t)blockIdx.x * lay.slot + 2 * (size_t)maxD;   // 3 (kmax + 2) doubles
    __shared__ double red[NT / 32];
    __shared__ double hs[kBatchMaxL * kBatchMaxL];
    __shared__ double bc64[kBatchMaxL * kBatchMaxL];
    __shared__ float bc32[kBatchMaxL * kBatchMaxL];
    __shared__ double U64[kBatchMaxL];
    __shared__ float U32[kBatchMaxL];
    __shared__ uint8_t bidx[kBatchMaxL * kBatchMaxL];
    __shared__ uint32_t bin[(kBatchMaxL + 1) * (kBatchMaxL + 1)];
    __shared__ int cur;
    for (int i = threadIdx.x; i < (kBatchMaxL + 1) * (kBatchMaxL + 1); i += blockDim.x) {
        const int n = i / (kBatchMaxL + 1), k = i % (kBatchMaxL + 1);
        // C(n, k) by the multiplicative formula (small n)
        uint32_t c = (k > n) ? 0u : 1u;
        for (int j = 1; j <= k && k <= n; ++j) c = c * (uint32_t)(n - k + j) / (uint32_t)j;
        bin[i] = c;
    }
    __syncthreads();
    while (true) {
        if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
        __syncthreads();
        const int si = cur;
        __syncthreads();
        if (si >= nsec) break;
        const SectorDesc sd = secs[si];
        const ModelDev &m = models[sd.model];
        const int L = sd.L;
        for (int i = threadIdx.x; i < L * L; i += blockDim.x) hs[i] = m.h[i];
        for (int i = threadIdx.x; i < L; i += blockDim.x) { U64[i] = m.U[i]; U32[i] = (float)m.U[i]; }
        __syncthreads();
        if (threadIdx.x == 0) {
            int nb = 0;
            for (int a = 0; a < L; ++a)
                for (int b = 0; b < L; ++b)
                    if (a != b && hs[a * L + b] != 0.0) {
                        bidx[a * L + b] = (uint8_t)nb;
                        bc64[nb] = hs[a * L + b];
                        bc32[nb] = (float)hs[a * L + b];
                        ++nb;
                    }
        }
        __syncthreads();
        build_spin(L, sd.Nup, sd.Dup, hmax, hs, bidx, bin, up);
        build_spin(L, sd.Ndn, sd.Ddn, hmax, hs, bidx, bin, dn);
        const int D = sd.Dup * sd.Ddn;
        const int K = min(iters, D);
        // Restarted Lanczos: each cycle stops as soon as the lowest Ritz pair
        // of T has converged to FP32 level (residual estimate
        // beta_{k+1} |s_k| <= 1e-6 max(|alpha|, beta), tested after 4 steps and
        // then at half the distance the decrease so far predicts (4 to 16
        // steps), with a warm-started eigenvalue search and the last
        // eigenvector component alone, and at the last step of the cycle), which keeps the FP32
        // recurrence from running on after convergence and spoiling the Ritz
        // vector; a cycle that ends unconverged restarts from its Ritz vector
        // (at most three cycles).  Each cycle runs the recurrence twice: once
        // for the scalars, once more (bit identical) to accumulate the Ritz
        // vector x in FP64.
        __shared__ int conv_s;
        __shared__ double lam_hint, gap_hint;   // warm start of the convergence test's eigenvalue search
        __shared__ int next_check, k_last;       // step of the next test; step and residual of the last one
        __shared__ double r_last;
        int kdone = 0;
        for (int cyc = 0; cyc < 3; ++cyc) {
            if (cyc > 0) {
                for (int i = threadIdx.x; i < D; i += blockDim.x) hx[i] = x[i];
                __syncthreads();
            }
            const int Kc = K;
            float fh = 0.f, fl = 0.f;
            for (int i = threadIdx.x; i < D; i += blockDim.x) {
                const float s = (float)(cyc == 0 ? start[sd.off + i] : hx[i]);
                ffp(fh, fl, s, s);
            }
            const double n0 = sqrt(bsum((double)fh + (double)fl, red));
            double scale = 0.0;
            kdone = 0;
            if (threadIdx.x == 0) {
                conv_s = 0;
                lam_hint = 0.0;
                gap_hint = 0.0;
                next_check = 4;
                k_last = 0;
                r_last = 0.0;
            }
            __syncthreads();
            for (int pass = 0; pass < 2; ++pass) {
                for (int i = threadIdx.x; i < D; i += blockDim.x) {
                    const float s = (float)(cyc == 0 ? start[sd.off + i] : hx[i]);
                    v[i] = (float)((double)s / n0);
                    vp[i] = 0.f;
                }
                __syncthreads();
                const int ksteps = pass == 0 ? Kc : kdone;
                for (int k = 0; k < ksteps; ++k) {
                    if (pass == 1) {
                        for (int i = threadIdx.x; i < D; i += blockDim.x) x[i] = fma(svec[k], (double)v[i], k ? x[i] : 0.0);
                        if (k + 1 == ksteps) break;
                    }
                    hv_small<float>(sd, hmax, up, dn, bc32, U32, hs, v, w);
                    __syncthreads();
                    const float bk = k ? (float)beta[k] : 0.f;
                    float ah = 0.f, al = 0.f;
                    for (int i = threadIdx.x; i < D; i += blockDim.x) {
                        float wi = w[i];
                        if (k) wi -= bk * vp[i];
                        w[i] = wi;
                        ffp(ah, al, wi, v[i]);
                    }
                    __syncthreads();
                    if (pass == 0) {
                        const double a = bsum((double)ah + (double)al, red);
                        if (threadIdx.x == 0) alpha[k] = a;
                        scale = fmax(scale, fabs(a));
                    }
                    __syncthreads();
                    const float ak = (float)alpha[k];
                    float bh = 0.f, bl = 0.f;
                    for (int i = threadIdx.x; i < D; i += blockDim.x) {
                        const float wi = w[i] - ak * v[i];
                        w[i] = wi;
                        ffp(bh, bl, wi, wi);
                    }
                    __syncthreads();
                    if (pass == 0) {
                        const double b = sqrt(fmax(bsum((double)bh + (double)bl, red), 0.0));
                        if (threadIdx.x == 0) beta[k + 1] = b;
                        kdone = k + 1;
                        scale = fmax(scale, b);
                        __syncthreads();
                        // lowest Ritz pair of T_{k+1} and its residual estimate,
                        // every 4 steps and at the end of the cycle
                        if (b <= 1e-13 * scale) {
                            if (threadIdx.x == 0) conv_s = 1;
                        }
                        __syncthreads();
                        if (!conv_s && kdone == next_check && k + 1 < Kc) {
                            // residual estimate from the last eigenvector component alone
                            const double lam = tridiag_lowest_warm(alpha, beta, kdone, &lam_hint, &gap_hint);
                            if (threadIdx.x == 0) {
                                const double thr = 1e-6 * scale;
                                const double r = b * tridiag_last_component(alpha, beta, kdone, lam, work);
                                if (r <= thr) {
                                    conv_s = 1;
                                } else {
                                    // next test at half the distance the geometric decrease since
                                    // the last test predicts, 4 to 16 steps ahead
                                    int gap = 4;
                                    if (r_last > 0.0 && r < r_last) {
                                        const double per_step = log(r / r_last) / (double)(kdone - k_last);
                                        const double steps = log(thr / r) / per_step;
                                        gap = 4 * max(1, min(4, (int)(0.5 * steps / 4.0)));
                                    }
                                    next_check = kdone + gap;
                                    r_last = r;
                                    k_last = kdone;
                                }
                            }
                            __syncthreads();
                        }
                        if (conv_s || k + 1 >= Kc) {
                            // the Ritz pair of the final T for the second pass
                            const double lam = tridiag_lowest_warm(alpha, beta, kdone, &lam_hint, &gap_hint);
                            if (threadIdx.x == 0) {
                                tridiag_vector_thread(alpha, beta, kdone, lam, svec, work);
                                if (b * fabs(svec[kdone - 1]) <= 1e-6 * scale) conv_s = 1;
                            }
                            __syncthreads();
                            break;
                        }
                    }
                    __syncthreads();
                    const float inv = 1.0f / (float)beta[k + 1];   // FP32: the FP64 divide is slow here
                    for (int i = threadIdx.x; i < D; i += blockDim.x) {
                        const float vn = w[i] * inv;
                        vp[i] = v[i];
                        v[i] = vn;
                    }
                    __syncthreads();
                }
            }
            __syncthreads();
            if (conv_s) break;
        }
        __syncthreads();
        // FP64 Rayleigh quotient of the Ritz vector
        hv_small<double>(sd, hmax, up, dn, bc64, U64, hs, x, hx);
        __syncthreads();
        double xhx = 0.0, xx = 0.0;
        for (int i = threadIdx.x; i < D; i += blockDim.x) {
            xhx = fma(x[i], hx[i], xhx);
            xx = fma(x[i], x[i], xx);
        }
        const double num = bsum(xhx, red);
        const double den = bsum(xx, red);
        if (threadIdx.x == 0) {
            outE[si] = num / den;
            if (outK) outK[si] = kdone;
        }
        __syncthreads();
    }
}

static int sector_list(int n_models, const gbr_model_desc *models, std::vector<SectorDesc> &secs, int64_t *n_states) {
    secs.clear();
    int64_t off = 0;
    for (int m = 0; m < n_models; ++m) {
        const int L = models[m].L;
        if (L < 1 || L > kBatchMaxL) return set_error(GBR_EINVAL, "model %d: L=%d out of range 1..%d", m, L, kBatchMaxL);
        if (!models[m].h) return set_error(GBR_EINVAL, "model %d: h is NULL", m);
        for (int nu = 0; nu <= L; ++nu)
            for (int nd = 0; nd <= L; ++nd) {
                SectorDesc s;
                s.model = m; s.L = L; s.Nup = nu; s.Ndn = nd;
                s.Dup = (int)binom(L, nu);
                s.Ddn = (int)binom(L, nd);
                s.off = off;
                off += (int64_t)s.Dup * s.Ddn;
                secs.push_back(s);
            }
    }
    if (n_states) *n_states = off;
    return GBR_OK;
}

}  // namespace gbr

using namespace gbr;

extern "C" int gbr_batch_layout(int n_models, const gbr_model_desc *models, int64_t *n_sectors, int64_t *n_states) {
    clear_error();
    if (n_models < 0 || (n_models > 0 && !models)) return set_error(GBR_EINVAL, "bad model list");
    std::vector<SectorDesc> secs;
    int rc = sector_list(n_models, models, secs, n_states);
    if (rc) return rc;
    if (n_sectors) *n_sectors = (int64_t)secs.size();
    return GBR_OK;
}

namespace gbr {
// CTA size and CTAs per SM of the batch solver (process-wide; 0 = as many as
// fit), set by gbr_batch_set_shape or gbr_batch_tune
static int g_batch_threads = kBatchThreads, g_batch_per_sm = 0;

template <int NT>
static int launch_batch(int grid_req_per_sm, size_t smem, int nsec, const SectorDesc *secs, const ModelDev *md,
                        const double *d_start, int K, const BatchSmem &lay, int *ctr, double *E, int *Kout,
                        DevBuf &dx, cudaStream_t st, int *grid_out) {
    auto kern = k_batch<NT>;
    GBR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GBR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
    per_sm = std::max(1, per_sm);
    if (grid_req_per_sm > 0) per_sm = std::min(per_sm, grid_req_per_sm);
    const int grid = std::max(1, std::min<int>(nsec, sm_count() * per_sm));
    int rc;
    if ((rc = dx.alloc((size_t)grid * (size_t)lay.slot * 8))) return rc;
    kern<<<grid, NT, smem, st>>>(secs, nsec, md, d_start, K, lay, ctr, E, Kout, dx.as<double>());
    GBR_LAUNCH_CHECK();
    count_launches(1);
    if (grid_out) *grid_out = grid;
    return GBR_OK;
}

static int batch_run(int n_models, const gbr_model_desc *models, const double *d_start, int iters, double *h_E0,
                     int *h_arg, double *h_sector_E, cudaStream_t st, int threads, int per_sm_req, float *ms_out) {
    if (n_models < 1 || !models) return set_error(GBR_EINVAL, "bad model list");
    if (!d_start || !h_E0) return set_error(GBR_EINVAL, "NULL argument");
    if (iters < 1 || iters > 4096) return set_error(GBR_EINVAL, "iters=%d out of range 1..4096", iters);
    std::vector<SectorDesc> secs;
    int64_t n_states = 0;
    int rc = sector_list(n_models, models, secs, &n_states);
    if (rc) return rc;
    std::vector<ModelDev> md((size_t)n_models);
    int maxD = 1, maxDs = 1, hmax = 1;
    for (int m = 0; m < n_models; ++m) {
        const int L = models[m].L;
        memset(&md[(size_t)m], 0, sizeof(ModelDev));
        md[(size_t)m].L = L;
        for (int p = 0; p < L; ++p) {
            for (int q = 0; q < L; ++q) {
                const double a = models[m].h[p * L + q];
                if (!std::isfinite(a) || a != models[m].h[q * L + p])
                    return set_error(GBR_EINVAL, "model %d: h not finite and symmetric at (%d,%d)", m, p, q);
                md[(size_t)m].h[p * L + q] = a;
            }
            md[(size_t)m].U[p] = models[m].U ? models[m].U[p] : 0.0;
        }
        int nb = 0;
        for (int p = 0; p < L; ++p)
            for (int q = 0; q < L; ++q)
                if (p != q && models[m].h[p * L + q] != 0.0) ++nb;
        if (nb > 0x7FFF) return set_error(GBR_EINVAL, "too many bonds");
        // largest hop count of any per-spin state: N (L - N) bounds it
        for (int N = 0; N <= L; ++N) hmax = std::max(hmax, N * (L - N));
        maxDs = std::max<int>(maxDs, (int)binom(L, L / 2));
    }
    for (const SectorDesc &s : secs) maxD = std::max(maxD, s.Dup * s.Ddn);
    const int K = std::min(iters, maxD);
    BatchSmem lay{maxD, maxDs, hmax, K, 2 * (int64_t)maxD + 3 * (int64_t)(K + 2)};
    auto r16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    size_t smem = 3 * r16((size_t)maxD * 4) + 2 * r16((size_t)maxDs * 4) +
                  2 * r16((size_t)maxDs) + 2 * r16((size_t)maxDs * hmax * 4) + 2 * r16((size_t)maxDs * 4) +
                  3 * r16((size_t)(K + 2) * 8);
    int dev = 0, optin = 0;
    GBR_CUDA_TRY(cudaGetDevice(&dev));
    GBR_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (smem + 8192 > (size_t)optin)
        return set_error(GBR_EINVAL, "largest sector needs %zu bytes of shared memory (limit %d)", smem, optin);
    // largest sectors first
    std::vector<SectorDesc> order(secs);
    std::vector<int> idx(secs.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        return (int64_t)secs[(size_t)a].Dup * secs[(size_t)a].Ddn > (int64_t)secs[(size_t)b].Dup * secs[(size_t)b].Ddn;
    });
    for (size_t i = 0; i < idx.size(); ++i) order[i] = secs[(size_t)idx[i]];
    DevBuf dsec, dmod, dE, dK, dctr, dx;
    if ((rc = dsec.upload(order.data(), order.size() * sizeof(SectorDesc)))) return rc;
    if ((rc = dmod.upload(md.data(), md.size() * sizeof(ModelDev)))) return rc;
    if ((rc = dE.alloc(order.size() * 8))) return rc;
    if ((rc = dK.alloc(order.size() * 4))) return rc;
    if ((rc = dctr.alloc(16))) return rc;
    GBR_CUDA_TRY(cudaMemsetAsync(dctr.p, 0, 16, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms_out) {
        GBR_CUDA_TRY(cudaEventCreate(&e0));
        GBR_CUDA_TRY(cudaEventCreate(&e1));
        cudaEventRecord(e0, st);
    }
    const int nsec = (int)order.size();
    if (threads == 128)
        rc = launch_batch<128>(per_sm_req, smem, nsec, dsec.as<SectorDesc>(), dmod.as<ModelDev>(), d_start, K, lay,
                               dctr.as<int>(), dE.as<double>(), dK.as<int>(), dx, st, nullptr);
    else if (threads == 512)
        rc = launch_batch<512>(per_sm_req, smem, nsec, dsec.as<SectorDesc>(), dmod.as<ModelDev>(), d_start, K, lay,
                               dctr.as<int>(), dE.as<double>(), dK.as<int>(), dx, st, nullptr);
    else
        rc = launch_batch<256>(per_sm_req, smem, nsec, dsec.as<SectorDesc>(), dmod.as<ModelDev>(), d_start, K, lay,
                               dctr.as<int>(), dE.as<double>(), dK.as<int>(), dx, st, nullptr);
    if (rc) return rc;
    if (ms_out) {
        cudaEventRecord(e1, st);
        GBR_CUDA_TRY(cudaEventSynchronize(e1));
        cudaEventElapsedTime(ms_out, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    std::vector<double> E(order.size());
    GBR_CUDA_TRY(cudaMemcpyAsync(E.data(), dE.p, E.size() * 8, cudaMemcpyDeviceToHost, st));
    GBR_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<double> Es(secs.size());
    for (size_t i = 0; i < idx.size(); ++i) Es[(size_t)idx[i]] = E[i];
    if (h_sector_E) memcpy(h_sector_E, Es.data(), Es.size() * 8);
    // per model minimum with the tie rule: within 1e-10 |E| prefer lower N, then lower N_up
    size_t s0 = 0;
    for (int m = 0; m < n_models; ++m) {
        const int L = models[m].L;
        const size_t ns = (size_t)(L + 1) * (L + 1);
        double best = Es[s0];
        for (size_t j = 0; j < ns; ++j) best = std::min(best, Es[s0 + j]);
        const double tol = 1e-10 * std::max(1.0, std::fabs(best));
        int bu = -1, bd = -1;
        for (int N = 0; N <= 2 * L && bu < 0; ++N)
            for (int nu = 0; nu <= L; ++nu) {
                const int nd = N - nu;
                if (nd < 0 || nd > L) continue;
                if (Es[s0 + (size_t)(nu * (L + 1) + nd)] <= best + tol) { bu = nu; bd = nd; break; }
            }
        h_E0[m] = best;
        if (h_arg) { h_arg[2 * m] = bu; h_arg[2 * m + 1] = bd; }
        s0 += ns;
    }
    return GBR_OK;
}
}  // namespace gbr

extern "C" int gbr_batch_solve(int n_models, const gbr_model_desc *models, const double *d_start, int iters,
                               double *h_E0, int *h_arg, double *h_sector_E, void *stream) {
    clear_error();
    return batch_run(n_models, models, d_start, iters, h_E0, h_arg, h_sector_E, (cudaStream_t)stream,
                     g_batch_threads, g_batch_per_sm, nullptr);
}

extern "C" int gbr_batch_set_shape(int threads, int ctas_per_sm) {
    clear_error();
    if (threads != 128 && threads != 256 && threads != 512)
        return set_error(GBR_EINVAL, "threads %d must be 128, 256 or 512", threads);
    if (ctas_per_sm < 0 || ctas_per_sm > 32) return set_error(GBR_EINVAL, "ctas_per_sm %d out of range 0..32", ctas_per_sm);
    g_batch_threads = threads;
    g_batch_per_sm = ctas_per_sm;
    return GBR_OK;
}

extern "C" int gbr_batch_get_shape(int *threads, int *ctas_per_sm) {
    clear_error();
    if (!threads || !ctas_per_sm) return set_error(GBR_EINVAL, "NULL argument");
    *threads = g_batch_threads;
    *ctas_per_sm = g_batch_per_sm;
    return GBR_OK;
}

extern "C" int gbr_batch_tune(int n_models, const gbr_model_desc *models, const double *d_start, int iters,
                              int *h_shape, float *h_ms, void *stream) {
    clear_error();
    if (!h_shape) return set_error(GBR_EINVAL, "NULL argument");
    std::vector<double> E((size_t)std::max(n_models, 1));
    float best = 1e30f;
    int bt = kBatchThreads, bp = 0, i = 0;
    for (int t : {128, 256, 512})
        for (int p : {0, 2, 1}) {
            float ms = 0.f;
            const int rc = batch_run(n_models, models, d_start, iters, E.data(), nullptr, nullptr,
                                     (cudaStream_t)stream, t, p, &ms);
            if (rc) return rc;
            if (h_ms) h_ms[i] = ms;
            ++i;
            if (ms < best) { best = ms; bt = t; bp = p; }
        }
    g_batch_threads = bt;
    g_batch_per_sm = bp;
    h_shape[0] = bt;
    h_shape[1] = bp;
    return GBR_OK;
}
