// Lowest eigenpair of a symmetric tridiagonal matrix T (diagonal a[0..k-1],
// off-diagonal b[1..k-1], indexed like the Lanczos beta_j) in FP64.
#pragma once

// number of eigenvalues of T below x: negative pivots of the LDL^T
// factorisation of T - x (Sturm sequence)
__device__ __forceinline__ int tridiag_sturm_count(const double *a, const double *b, int k, double x) {
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < k; ++i) {
        const double bb = i ? b[i] * b[i] : 0.0;
        q = (a[i] - x) - (i ? bb / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

// Lowest eigenvalue by multisection of the Gershgorin interval: every round
// the first warp evaluates the Sturm count at 32 equally spaced points and
// keeps the cell where the count first reaches 1, until the interval no
// longer shrinks.  (One warp, not the whole block: the FP64 divisions of the
// Sturm recurrence are slow, and 32 points per round already gain 5 bits.)
// Called by every thread of the block; the result is returned to all.
__device__ double tridiag_lowest_block(const double *a, const double *b, int k) {
    __shared__ double lo_s, hi_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double lo = a[0], hi = a[0];
        for (int i = 0; i < k; ++i) {
            const double r = (i ? fabs(b[i]) : 0.0) + (i + 1 < k ? fabs(b[i + 1]) : 0.0);
            lo = fmin(lo, a[i] - r);
            hi = fmax(hi, a[i] + r);
        }
        const double pad = 1e-12 * fmax(fabs(lo), fabs(hi)) + 1e-300;
        lo_s = lo - pad;
        hi_s = hi + pad;
    }
    __syncthreads();
    const int P = 32;
    if (threadIdx.x < 32) {
        for (int round = 0; round < 200; ++round) {
            const double lo = lo_s, hi = hi_s;
            const double x = (threadIdx.x == P - 1) ? hi : lo + (hi - lo) * ((double)(threadIdx.x + 1) / (double)P);
            const int c = tridiag_sturm_count(a, b, k, x);
            const unsigned m = __ballot_sync(0xFFFFFFFFu, c >= 1);
            const int f = m ? __ffs(m) - 1 : P - 1;
            if (threadIdx.x == 0) {
                const double nhi = (f == P - 1) ? hi : lo + (hi - lo) * ((double)(f + 1) / (double)P);
                const double nlo = (f == 0) ? lo : lo + (hi - lo) * ((double)f / (double)P);
                hi_s = fmin(hi, fmax(nhi, lo));
                lo_s = fmax(lo, fmin(nlo, hi_s));
            }
            __syncwarp();
            const double nl = lo_s, nh = hi_s;
            const bool done = !(nl < nh) || nextafter(nl, nh) >= nh || (nh == hi && nl == lo);
            __syncwarp();
            if (done) break;
        }
    }
    __syncthreads();
    const double r = hi_s;
    __syncthreads();
    return r;
}

// Eigenvector for the eigenvalue lam by inverse iteration on (T - lam) z = z
// with Thomas elimination (tiny pivots replaced), three sweeps, normalised.
// One thread; work holds 3k doubles.
__device__ void tridiag_vector_thread(const double *a, const double *b, int k, double lam, double *s, double *work) {
    if (k == 1) {
        s[0] = 1.0;
        return;
    }
    double *dd = work, *zz = work + 2 * k;
    double tn = 0.0;
    for (int i = 0; i < k; ++i) tn = fmax(tn, fabs(a[i]) + (i ? fabs(b[i]) : 0.0));
    const double tiny = fmax(1e-14 * tn, 1e-290);
    for (int i = 0; i < k; ++i) zz[i] = 1.0;
    for (int sweep = 0; sweep < 3; ++sweep) {
        double piv = a[0] - lam;
        if (fabs(piv) < tiny) piv = tiny;
        dd[0] = piv;
        for (int i = 1; i < k; ++i) {
            const double l = b[i] / dd[i - 1];
            piv = (a[i] - lam) - l * b[i];
            if (fabs(piv) < tiny) piv = tiny;
            dd[i] = piv;
            zz[i] -= l * zz[i - 1];
        }
        zz[k - 1] /= dd[k - 1];
        for (int i = k - 2; i >= 0; --i) zz[i] = (zz[i] - b[i + 1] * zz[i + 1]) / dd[i];
        // scale by the largest entry first so that the norm cannot overflow
        double mx = 0.0;
        for (int i = 0; i < k; ++i) mx = fmax(mx, fabs(zz[i]));
        if (!(mx > 0.0) || !isfinite(mx)) {
            for (int i = 0; i < k; ++i) zz[i] = i == 0 ? 1.0 : 0.0;
            continue;
        }
        double nrm = 0.0;
        for (int i = 0; i < k; ++i) {
            zz[i] /= mx;
            nrm += zz[i] * zz[i];
        }
        nrm = sqrt(nrm);
        for (int i = 0; i < k; ++i) zz[i] /= nrm;
    }
    for (int i = 0; i < k; ++i) s[i] = zz[i];
}

// Lowest eigenvalue as tridiag_lowest_block, for a convergence test that runs
// every few steps: by Cauchy interlacing the lowest eigenvalue of T_k is at
// most the previous one (*lam_prev, from a leading block; 0 entries = none),
// so the search starts from the bracket [lam_prev - d, lam_prev] with the
// smallest d = gap * 4^j (j = 0..31, one Sturm count per lane) that has no
// eigenvalue below it, instead of the whole Gershgorin interval.  Updates
// *lam_prev and *gap (the last decrease, floored).  Falls back to the full
// interval when no hint is set or no bracket is found.
__device__ double tridiag_lowest_warm(const double *a, const double *b, int k, double *lam_prev, double *gap) {
    __shared__ double lo_s, hi_s;
    __shared__ int ok_s;
    __syncthreads();
    const double lp = *lam_prev, g0 = *gap;
    if (threadIdx.x == 0) ok_s = 0;
    __syncthreads();
    if (g0 > 0.0 && threadIdx.x < 32) {
        const double x = lp - g0 * exp2(2.0 * (double)threadIdx.x);
        const int c = tridiag_sturm_count(a, b, k, x);
        const unsigned m = __ballot_sync(0xFFFFFFFFu, c == 0);
        const int chi = tridiag_sturm_count(a, b, k, lp + 1e-12 * fabs(lp) + 1e-300);
        if (threadIdx.x == 0 && m && chi >= 1) {
            const int j = __ffs(m) - 1;
            lo_s = lp - g0 * exp2(2.0 * (double)j);
            hi_s = lp + 1e-12 * fabs(lp) + 1e-300;
            ok_s = 1;
        }
    }
    __syncthreads();
    double r;
    if (!ok_s) {
        r = tridiag_lowest_block(a, b, k);
    } else {
        const int P = 32;
        if (threadIdx.x < 32) {
            for (int round = 0; round < 200; ++round) {
                const double lo = lo_s, hi = hi_s;
                const double x = (threadIdx.x == P - 1) ? hi : lo + (hi - lo) * ((double)(threadIdx.x + 1) / (double)P);
                const int c = tridiag_sturm_count(a, b, k, x);
                const unsigned m = __ballot_sync(0xFFFFFFFFu, c >= 1);
                const int f = m ? __ffs(m) - 1 : P - 1;
                if (threadIdx.x == 0) {
                    const double nhi = (f == P - 1) ? hi : lo + (hi - lo) * ((double)(f + 1) / (double)P);
                    const double nlo = (f == 0) ? lo : lo + (hi - lo) * ((double)f / (double)P);
                    hi_s = fmin(hi, fmax(nhi, lo));
                    lo_s = fmax(lo, fmin(nlo, hi_s));
                }
                __syncwarp();
                const double nl = lo_s, nh = hi_s;
                const bool done = !(nl < nh) || nextafter(nl, nh) >= nh || (nh == hi && nl == lo);
                __syncwarp();
                if (done) break;
            }
        }
        __syncthreads();
        r = hi_s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double dec = (g0 > 0.0 || lp != 0.0) ? fabs(lp - r) : 0.0;
        *gap = fmax(dec, 1e-14 * fmax(fabs(r), 1e-300));
        *lam_prev = r;
    }
    __syncthreads();
    return r;
}

// |s_{k-1}|, the last component of the normalised eigenvector of T for the
// eigenvalue lam, from one top-down LDL^T pass of T - lam (pivots d_i) and
// the solution of L^T z = e_{k-1} from the bottom, z_i = -(b_{i+1} / d_i)
// z_{i+1} (the twisted factorisation with the twist at the last index): in
// exact arithmetic z is the eigenvector with z_{k-1} = 1, so the answer is
// 1 / |z|.  k divisions (inverse iteration takes 6k); for the convergence
// test, which needs the size of the residual estimate, not the vector.  One
// thread; work holds k doubles.
__device__ double tridiag_last_component(const double *a, const double *b, int k, double lam, double *work) {
    if (k == 1) return 1.0;
    double tn = 0.0;
    for (int i = 0; i < k; ++i) tn = fmax(tn, fabs(a[i]) + (i ? fabs(b[i]) : 0.0));
    const double tiny = fmax(1e-14 * tn, 1e-290);
    double d = a[0] - lam;
    if (fabs(d) < tiny) d = tiny;
    work[0] = 1.0 / d;
    for (int i = 1; i + 1 < k; ++i) {
        d = (a[i] - lam) - b[i] * b[i] * work[i - 1];
        if (fabs(d) < tiny) d = tiny;
        work[i] = 1.0 / d;
    }
    // z from the bottom, |z|^2 accumulated with rescaling so that it cannot overflow
    double z = 1.0, sum = 1.0, scale = 1.0;   // |z|^2 = sum * scale^2
    for (int i = k - 2; i >= 0; --i) {
        z = -b[i + 1] * z * work[i];
        const double az = fabs(z);
        if (az > 1e100) {
            z /= 1e100;
            sum /= 1e200;
            scale *= 1e100;
        }
        sum += z * z;
    }
    if (!isfinite(sum) || !(sum > 0.0)) return 0.0;
    return 1.0 / (sqrt(sum) * scale);
}
