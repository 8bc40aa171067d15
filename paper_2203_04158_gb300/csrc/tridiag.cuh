// Lowest eigenpair of a symmetric tridiagonal matrix T (diagonal a[0..k-1],
// off-diagonal b[1..k-1], indexed like the Lanczos beta_j) in FP64.
#pragma once

// 1/x by Newton-Raphson iteration on f(r) = 1/r - x, r <- r + r (1 - x r)
// (two FMAs a step), from the single-precision approximate reciprocal: every
// step doubles the correct bits, so two steps from the ~23-bit seed leave an
// error of a few ulp.  These routines divide in long dependent chains, and an
// FP64 division is a much longer chain on this GPU's narrow FP64 pipe.  Values
// outside the single-precision range take the division.
__device__ __forceinline__ double rcp64(double x) {
    const double ax = fabs(x);
    if (!(ax > 1e-30 && ax < 1e30)) return 1.0 / x;
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"((float)x));
    double r = (double)rf;
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    return r;
}

// number of eigenvalues of T below x: negative pivots of the LDL^T
// factorisation of T - x (Sturm sequence)
__device__ __forceinline__ int tridiag_sturm_count(const double *a, const double *b, int k, double x) {
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < k; ++i) {
        const double bb = i ? b[i] * b[i] : 0.0;
        q = (a[i] - x) - (i ? bb * rcp64(q) : 0.0);
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
            const double x = (threadIdx.x == P - 1) ? hi : lo + (hi - lo) * ((double)(threadIdx.x + 1) * (1.0 / P));
            const int c = tridiag_sturm_count(a, b, k, x);
            const unsigned m = __ballot_sync(0xFFFFFFFFu, c >= 1);
            const int f = m ? __ffs(m) - 1 : P - 1;
            if (threadIdx.x == 0) {
                const double nhi = (f == P - 1) ? hi : lo + (hi - lo) * ((double)(f + 1) * (1.0 / P));
                const double nlo = (f == 0) ? lo : lo + (hi - lo) * ((double)f * (1.0 / P));
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
    double *rd = work, *zz = work + 2 * k;   // reciprocal pivots, iterate
    double tn = 0.0;
    for (int i = 0; i < k; ++i) tn = fmax(tn, fabs(a[i]) + (i ? fabs(b[i]) : 0.0));
    const double tiny = fmax(1e-14 * tn, 1e-290);
    for (int i = 0; i < k; ++i) zz[i] = 1.0;
    for (int sweep = 0; sweep < 3; ++sweep) {
        double piv = a[0] - lam;
        if (fabs(piv) < tiny) piv = tiny;
        rd[0] = rcp64(piv);
        for (int i = 1; i < k; ++i) {
            const double l = b[i] * rd[i - 1];
            piv = (a[i] - lam) - l * b[i];
            if (fabs(piv) < tiny) piv = tiny;
            rd[i] = rcp64(piv);
            zz[i] -= l * zz[i - 1];
        }
        zz[k - 1] *= rd[k - 1];
        for (int i = k - 2; i >= 0; --i) zz[i] = (zz[i] - b[i + 1] * zz[i + 1]) * rd[i];
        // scale by the largest entry first so that the norm cannot overflow
        double mx = 0.0;
        for (int i = 0; i < k; ++i) mx = fmax(mx, fabs(zz[i]));
        if (!(mx > 0.0) || !isfinite(mx)) {
            for (int i = 0; i < k; ++i) zz[i] = i == 0 ? 1.0 : 0.0;
            continue;
        }
        const double imx = 1.0 / mx;
        double nrm = 0.0;
        for (int i = 0; i < k; ++i) {
            zz[i] *= imx;
            nrm += zz[i] * zz[i];
        }
        const double inrm = 1.0 / sqrt(nrm);
        for (int i = 0; i < k; ++i) zz[i] *= inrm;
    }
    for (int i = 0; i < k; ++i) s[i] = zz[i];
}

// Rounds of 32-point multisection of the bracket [*lo, *hi] (shared memory)
// by the first warp: each round evaluates the Sturm count at 32 equally
// spaced points and keeps the cell where the count first reaches 1; stops
// after max_rounds or when the bracket no longer shrinks.  Called by every
// thread of the block.
__device__ void tridiag_multisection_rounds(const double *a, const double *b, int k, double *lo_s, double *hi_s,
                                            int max_rounds) {
    const int P = 32;
    if (threadIdx.x < 32) {
        for (int round = 0; round < max_rounds; ++round) {
            const double lo = *lo_s, hi = *hi_s;
            const double x = (threadIdx.x == P - 1) ? hi : lo + (hi - lo) * ((double)(threadIdx.x + 1) * (1.0 / P));
            const int c = tridiag_sturm_count(a, b, k, x);
            const unsigned m = __ballot_sync(0xFFFFFFFFu, c >= 1);
            const int f = m ? __ffs(m) - 1 : P - 1;
            if (threadIdx.x == 0) {
                const double nhi = (f == P - 1) ? hi : lo + (hi - lo) * ((double)(f + 1) * (1.0 / P));
                const double nlo = (f == 0) ? lo : lo + (hi - lo) * ((double)f * (1.0 / P));
                *hi_s = fmin(hi, fmax(nhi, lo));
                *lo_s = fmax(lo, fmin(nlo, *hi_s));
            }
            __syncwarp();
            const double nl = *lo_s, nh = *hi_s;
            const bool done = !(nl < nh) || nextafter(nl, nh) >= nh || (nh == hi && nl == lo);
            __syncwarp();
            if (done) break;
        }
    }
    __syncthreads();
}

// Lowest eigenvalue as tridiag_lowest_block, for tests that run every few
// steps: by Cauchy interlacing the lowest eigenvalue of T_k is at most the
// previous one (*lam_prev, from a leading block; 0 entries = none), so the
// search starts from the bracket [lam_prev - d, lam_prev] with the smallest
// d = gap * 4^j (j = 0..30, one Sturm count per lane) that has no eigenvalue
// below it, instead of the whole Gershgorin interval, and finishes by
// Newton's method from the bracket's lower end (multisection if that fails).
// Updates *lam_prev and *gap (the last decrease, floored).  Falls back to the
// full interval when no hint is set or no bracket is found.
__device__ double tridiag_lowest_warm(const double *a, const double *b, int k, double *lam_prev, double *gap) {
    __shared__ double lo_s, hi_s;
    __shared__ int ok_s;
    __syncthreads();
    const double lp = *lam_prev, g0 = *gap;
    if (threadIdx.x == 0) ok_s = 0;
    __syncthreads();
    if (g0 > 0.0 && threadIdx.x < 32) {
        // lanes 0..30 try lp - gap 4^lane (4^j built from its exponent bits),
        // lane 31 the upper end, which must have an eigenvalue below it
        const double hi = lp + 1e-12 * fabs(lp) + 1e-300;
        const double x = threadIdx.x < 31 ? lp - g0 * __longlong_as_double((long long)(1023 + 2 * threadIdx.x) << 52) : hi;
        const int c = tridiag_sturm_count(a, b, k, x);
        const unsigned m = __ballot_sync(0xFFFFFFFFu, c == 0) & 0x7FFFFFFFu;
        const bool hi_ok = __shfl_sync(0xFFFFFFFFu, c, 31) >= 1;
        if (threadIdx.x == 0 && m && hi_ok) {
            const int j = __ffs(m) - 1;
            lo_s = lp - g0 * __longlong_as_double((long long)(1023 + 2 * j) << 52);
            hi_s = hi;
            ok_s = 1;
        }
    }
    __syncthreads();
    // two multisection rounds shrink the bracket 1024-fold (one Sturm pass
    // each, 32 points in parallel), then Newton's method on det(T - x) from
    // its lower end: the lowest eigenvalue is the smallest zero of a
    // polynomial with only real zeros, so the iterates rise monotonically to
    // it without passing it, and from a bracket that narrow they converge
    // quadratically.  One thread; the step is 1 / sum_i (-d_i' / d_i) over the
    // LDL^T pivots d_i of T - x and their derivatives
    // d_i' = -1 + b_i^2 d_{i-1}' / d_{i-1}^2.  A non-positive pivot means x
    // reached the eigenvalue within rounding.  If Newton fails, multisection
    // finishes the search.
    if (ok_s) tridiag_multisection_rounds(a, b, k, &lo_s, &hi_s, 2);
    __shared__ int newton_ok;
    __shared__ double newton_x;
    if (threadIdx.x == 0) {
        newton_ok = 0;
        if (ok_s) {
            double x = lo_s;
            bool conv = false;
            for (int it = 0; it < 16 && !conv; ++it) {
                double d = a[0] - x, dp = -1.0, acc = 0.0;
                bool pos = d > 0.0;
                double r = pos ? rcp64(d) : 0.0;
                acc += dp * r;
                for (int i = 1; i < k && pos; ++i) {
                    const double bb = b[i] * b[i];
                    dp = -1.0 + bb * dp * r * r;
                    d = (a[i] - x) - bb * r;
                    pos = d > 0.0;
                    r = pos ? rcp64(d) : 0.0;
                    acc += dp * r;
                }
                if (!pos || !(acc < 0.0)) { conv = true; break; }   // at the eigenvalue (within rounding)
                const double xn = x - rcp64(acc);
                if (!(xn > x) || !isfinite(xn)) { conv = true; break; }
                conv = (xn - x) <= 4.0 * 1.1102230246251565e-16 * fabs(xn) + 1e-300;
                x = xn;
            }
            newton_x = x;
            newton_ok = conv && isfinite(x) && x <= hi_s ? 1 : 0;
        }
    }
    __syncthreads();
    double r;
    if (newton_ok) {
        r = newton_x;
    } else if (!ok_s) {
        r = tridiag_lowest_block(a, b, k);
    } else {
        tridiag_multisection_rounds(a, b, k, &lo_s, &hi_s, 200);
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
// 1 / |z|.  k reciprocals (inverse iteration takes 3k); for the convergence
// test, which needs the size of the residual estimate, not the vector.  One
// thread; work holds k doubles.
__device__ double tridiag_last_component(const double *a, const double *b, int k, double lam, double *work) {
    if (k == 1) return 1.0;
    double tn = 0.0;
    for (int i = 0; i < k; ++i) tn = fmax(tn, fabs(a[i]) + (i ? fabs(b[i]) : 0.0));
    const double tiny = fmax(1e-14 * tn, 1e-290);
    double d = a[0] - lam;
    if (fabs(d) < tiny) d = tiny;
    work[0] = rcp64(d);
    for (int i = 1; i + 1 < k; ++i) {
        d = (a[i] - lam) - b[i] * b[i] * work[i - 1];
        if (fabs(d) < tiny) d = tiny;
        work[i] = rcp64(d);
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
