/*
 * Seeded synthetic-input painter (input generation only).
 *
 * Adds truncated Gaussian bumps  A * exp(-c^2 / (2 sigma^2)),  c = chord between
 * the pixel centre and the bump centre, onto a HEALPix RING-ordered map.  The
 * paper measures on ray-traced convergence maps that are not available here; a
 * sum of bumps plus white noise stands in for them with the same map shape.
 *
 * This file holds none of the estimator's arithmetic.  It carries its own copy
 * of the HEALPix RING ring layout (Gorski et al. 2005) because painting needs
 * pixel positions; neither the oracle nor the CUDA library uses it.
 *
 * Determinism: every ring is painted by one thread, bumps are visited in the
 * caller's order, and exp() is a fixed polynomial, so the result does not depend
 * on the thread count.  Build with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int64_t first; /* first pixel index of the ring */
    int64_t npr;   /* pixels in the ring */
    double z, sth; /* cos and sin of the colatitude */
    double phi0;   /* longitude of pixel 0 */
    double dphi;   /* longitude step */
} ring_t;

static void ring_layout(int64_t n, int64_t r, ring_t* R) {
    const double nn = (double)n;
    if (r < n) { /* north polar cap */
        const double t = (double)(r * r) / (3.0 * nn * nn);
        R->npr = 4 * r;
        R->first = 2 * r * (r - 1);
        R->z = 1.0 - t;
        R->sth = sqrt(t * (2.0 - t));
        R->dphi = M_PI / (2.0 * (double)r);
        R->phi0 = 0.5 * R->dphi;
    } else if (r > 3 * n) { /* south polar cap, mirror of ring 4n-r */
        const int64_t rr = 4 * n - r;
        const double t = (double)(rr * rr) / (3.0 * nn * nn);
        R->npr = 4 * rr;
        R->first = 12 * n * n - 2 * rr * (rr + 1);
        R->z = -(1.0 - t);
        R->sth = sqrt(t * (2.0 - t));
        R->dphi = M_PI / (2.0 * (double)rr);
        R->phi0 = 0.5 * R->dphi;
    } else { /* equatorial belt */
        R->npr = 4 * n;
        R->first = 2 * n * (n - 1) + 4 * n * (r - n);
        R->z = 4.0 / 3.0 - 2.0 * (double)r / (3.0 * nn);
        R->sth = sqrt((1.0 - R->z) * (1.0 + R->z));
        R->dphi = M_PI / (2.0 * nn);
        R->phi0 = (((r - n + 1) & 1) != 0) ? 0.5 * R->dphi : 0.0;
    }
}

/* exp(x) for -50 <= x <= 0: Taylor polynomial of degree 9 at x/64, then six
 * squarings (relative error < 1e-10).  Straight-line arithmetic so that the
 * pixel loop vectorises. */
static inline double fixed_exp(double x) {
    x = x < -50.0 ? -50.0 : x; /* clamp (the caller masks these pixels out) */
    const double y = x * (1.0 / 64.0);
    double p = 1.0 / 362880.0;
    p = p * y + 1.0 / 40320.0;
    p = p * y + 1.0 / 5040.0;
    p = p * y + 1.0 / 720.0;
    p = p * y + 1.0 / 120.0;
    p = p * y + 1.0 / 24.0;
    p = p * y + 1.0 / 6.0;
    p = p * y + 0.5;
    p = p * y + 1.0;
    p = p * y + 1.0;
    p = p * p;
    p = p * p;
    p = p * p;
    p = p * p;
    p = p * p;
    p = p * p;
    return p;
}

/* Binary search: first index with key >= v. */
static int64_t lower_bound(const double* a, int64_t n, double v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/*
 * Paint nb bumps onto map[0 .. 12 nside^2) (added to what is there).
 * theta, phi: bump centre colatitude / longitude (rad), sorted by theta.
 * sigma: width (rad); amp: amplitude; trunc: truncation radius in units of sigma
 * (chord).  Returns 0 on success.
 */
int synth_paint_bumps(int64_t nside, int64_t nb, const double* theta, const double* phi,
                      const double* sigma, const double* amp, double trunc, double* map) {
    if (nside < 1 || nb < 0 || trunc <= 0.0) return 1;
    double smax = 0.0;
    for (int64_t b = 0; b < nb; ++b) smax = sigma[b] > smax ? sigma[b] : smax;
    const double cmax = trunc * smax;
    const double dth_max = cmax >= 2.0 ? M_PI : 2.0 * asin(0.5 * cmax);
    const int64_t nrings = 4 * nside - 1;

#pragma omp parallel
    {
        double* cp = NULL;
        double* sp = NULL;
        int64_t cap = 0;
#pragma omp for schedule(dynamic, 4)
        for (int64_t r = 1; r <= nrings; ++r) {
            ring_t R;
            ring_layout(nside, r, &R);
            if (R.npr > cap) {
                free(cp);
                free(sp);
                cap = R.npr;
                cp = (double*)malloc(sizeof(double) * cap);
                sp = (double*)malloc(sizeof(double) * cap);
            }
            for (int64_t p = 0; p < R.npr; ++p) {
                const double ph = R.phi0 + (double)p * R.dphi;
                cp[p] = cos(ph);
                sp[p] = sin(ph);
            }
            const double th_r = atan2(R.sth, R.z);
            const int64_t b0 = lower_bound(theta, nb, th_r - dth_max);
            const int64_t b1 = lower_bound(theta, nb, th_r + dth_max);
            double* out = map + R.first;
            for (int64_t b = b0; b < b1; ++b) {
                const double sg = sigma[b];
                const double cut2 = (trunc * sg) * (trunc * sg);
                const double hd = sin(0.5 * (theta[b] - th_r));
                const double c2_0 = 4.0 * hd * hd; /* chord^2 at equal longitude */
                if (c2_0 >= cut2) continue;
                const double sb = sin(theta[b]);
                const double kk = 2.0 * sb * R.sth; /* chord^2 = c2_0 + kk (1 - cos dphi) */
                const double inv2s2 = 1.0 / (2.0 * sg * sg);
                const double cb = cos(phi[b]), snb = sin(phi[b]);
                int64_t p0, cnt;
                const double q = (kk > 0.0) ? (cut2 - c2_0) / (2.0 * kk) : 2.0; /* sin^2(dphi_max/2) */
                if (q >= 1.0) {
                    p0 = 0;
                    cnt = R.npr;
                } else {
                    const double dmax = 2.0 * asin(sqrt(q));
                    p0 = (int64_t)floor((phi[b] - dmax - R.phi0) / R.dphi);
                    cnt = (int64_t)floor((phi[b] + dmax - R.phi0) / R.dphi) - p0 + 2;
                    if (cnt > R.npr) {
                        p0 = 0;
                        cnt = R.npr;
                    }
                    p0 %= R.npr;
                    if (p0 < 0) p0 += R.npr;
                }
                const double a = amp[b];
                /* at most two wrap-free segments */
                int64_t pa[2] = {p0, 0}, pb[2] = {p0 + cnt, 0};
                if (p0 + cnt > R.npr) {
                    pb[0] = R.npr;
                    pb[1] = p0 + cnt - R.npr;
                }
                for (int seg = 0; seg < 2; ++seg) {
                    const int64_t lo = pa[seg], hi = pb[seg];
#pragma omp simd
                    for (int64_t p = lo; p < hi; ++p) {
                        const double cd = cp[p] * cb + sp[p] * snb; /* cos(phi_p - phi_b) */
                        const double c2 = c2_0 + kk * (1.0 - cd);
                        const double in = (double)(c2 < cut2);
                        out[p] += in * a * fixed_exp(-c2 * inv2s2);
                    }
                }
            }
        }
        free(cp);
        free(sp);
    }
    return 0;
}
