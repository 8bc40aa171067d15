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
