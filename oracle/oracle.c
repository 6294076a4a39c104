/*
 * Plain CPU FP64 oracle for the binned harmonic 3PCF estimator of
 * arXiv:2408.16847 (section 3.1, eqs. Xm.binned, zetamEst, zetamEst2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only the tests, the package's smoke check and the benchmark's CPU
 * baseline use it.  It shares no code, header, table or constant generator with
 * the CUDA library.
 *
 * What it computes, straight from the definitions (no blocking, no recurrences):
 *   - pixel centres of a HEALPix RING map (Gorski et al. 2005), in FP64;
 *   - for every pivot i and every other point j with theta_k <= theta_ij < theta_{k+1}
 *     (bins compared by chord c = |n_j - n_i| against 2 sin(theta/2), FP64):
 *         a_m^k(i) = sum_j w_j d_j exp(-i m phi_ij)          (eq. Xm.binned, unnormalised)
 *         W^k(i)   = sum_j w_j                               (the same sum with d = 1, m = 0)
 *         Q^k(i)   = sum_j (w_j d_j)^2,  QW^k(i) = sum_j w_j^2  (self-pair terms, section 3.4)
 *     where phi_ij is the position angle of n_j about n_i, measured from local north
 *     towards local east, evaluated with atan2 and cos/sin per m;
 *   - the adjoint's neighbour legs  g_p = w_p sum_{i in P, p in nbr(i)} w_i d_i
 *     sum_m Re[exp(-i m phi_ip) h_m^{k(ip)}(i)]  for a given h.
 * The contraction over pivots (eq. zetamEst) and the normalisation are done by the
 * Python wrapper with numpy on the arrays returned here.
 *
 * Neighbour search: a uniform 3-D grid over the cube [-1,1]^3 with cell size >=
 * the largest chord, so every neighbour lies in the 27 cells around the pivot's
 * cell; each candidate is tested exactly.  This is deliberately unrelated to the
 * ring-range search of the CUDA path.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------ HEALPix RING */

/* Ring number (1-based, counted from the nearest pole) of the k-th pixel of a
 * polar cap, where cap ring r holds pixels [2r(r-1), 2r(r+1)). */
static int64_t cap_ring(int64_t k) {
    int64_t r = (int64_t)floor(0.5 * (1.0 + sqrt(1.0 + 2.0 * (double)k)));
    while (2 * r * (r - 1) > k) --r;
    while (2 * (r + 1) * r <= k) ++r;
    return r;
}

/* Unit vector of RING pixel p at resolution nside (Gorski et al. 2005, sec. 4). */
void orc_pix2vec_one(int64_t nside, int64_t p, double* out) {
    const int64_t n = nside;
    const int64_t ncap = 2 * n * (n - 1);
    const int64_t npix = 12 * n * n;
    const double nn = (double)n;
    double z, s, phi;
    if (p < ncap) {
        const int64_t r = cap_ring(p);
        const int64_t j = p - 2 * r * (r - 1);
        const double t = (double)(r * r) / (3.0 * nn * nn); /* 1 - z */
        z = 1.0 - t;
        s = sqrt(t * (2.0 - t));
        phi = ((double)j + 0.5) * M_PI / (2.0 * (double)r);
    } else if (p < npix - ncap) {
        const int64_t q = p - ncap;
        const int64_t r = q / (4 * n) + n; /* ring index from the north pole */
        const int64_t j = q % (4 * n);
        const int64_t shift = (r - n + 1) & 1;
        z = (4.0 / 3.0) - 2.0 * (double)r / (3.0 * nn);
        s = sqrt((1.0 - z) * (1.0 + z));
        phi = ((double)j + 0.5 * (double)shift) * M_PI / (2.0 * nn);
    } else {
        const int64_t q = npix - 1 - p;
        const int64_t r = cap_ring(q); /* counted from the south pole */
        const int64_t j = p - (npix - 2 * r * (r + 1));
        const double t = (double)(r * r) / (3.0 * nn * nn);
        z = -(1.0 - t);
        s = sqrt(t * (2.0 - t));
        phi = ((double)j + 0.5) * M_PI / (2.0 * (double)r);
    }
    out[0] = s * cos(phi);
    out[1] = s * sin(phi);
    out[2] = z;
}

void orc_pix2vec_ring(int64_t nside, int64_t n, const int64_t* pix, double* xyz) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) orc_pix2vec_one(nside, pix[i], xyz + 3 * i);
}

void orc_pix2vec_all(int64_t nside, double* xyz) {
    const int64_t npix = 12 * nside * nside;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < npix; ++p) orc_pix2vec_one(nside, p, xyz + 3 * p);
}

/* -------------------------------------------------------------- 3-D grid */

typedef struct {
    int64_t G;        /* cells per axis */
    double cell;      /* cell size */
    int64_t* start;   /* G^3 + 1 offsets */
    int64_t* order;   /* point indices sorted by cell */
} grid_t;

static int64_t cell_coord(double v, double cell, int64_t G) {
    int64_t c = (int64_t)floor((v + 1.0) / cell);
    if (c < 0) c = 0;
    if (c >= G) c = G - 1;
    return c;
}

static int grid_build(grid_t* g, int64_t n, const double* xyz, double cmax) {
    double cell = cmax > 1e-6 ? cmax : 1e-6;
    int64_t G = (int64_t)ceil(2.0 / cell) + 1;
    if (G > 400) { /* bound the memory; cells stay >= cmax */
        G = 400;
        cell = 2.0 / (double)(G - 1);
        if (cell < cmax) return 1;
    }
    g->G = G;
    g->cell = cell;
    const int64_t nc = G * G * G;
    g->start = (int64_t*)calloc((size_t)(nc + 1), sizeof(int64_t));
    g->order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* cid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!g->start || !g->order || !cid) return 2;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t cx = cell_coord(xyz[3 * i], cell, G);
        const int64_t cy = cell_coord(xyz[3 * i + 1], cell, G);
        const int64_t cz = cell_coord(xyz[3 * i + 2], cell, G);
        cid[i] = (cx * G + cy) * G + cz;
        g->start[cid[i] + 1]++;
    }
    for (int64_t c = 0; c < nc; ++c) g->start[c + 1] += g->start[c];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)nc);
    if (!fill) return 2;
    memcpy(fill, g->start, sizeof(int64_t) * (size_t)nc);
    for (int64_t i = 0; i < n; ++i) g->order[fill[cid[i]]++] = i;
    free(fill);
    free(cid);
    return 0;
}

static void grid_free(grid_t* g) {
    free(g->start);
    free(g->order);
}

/* ------------------------------------------------------ local frame, angle */

/* Local east / north unit vectors at n (east = z x n / |z x n|, north = n x east).
 * At a pole the frame is the limit taken along longitude 0; by the paper's
 * argument (section 3.1, after eq. zetamEst2) any choice gives the same zeta. */
static void local_frame(const double* n, double* east, double* north) {
    const double s = sqrt(n[0] * n[0] + n[1] * n[1]);
    if (s > 1e-12) {
        east[0] = -n[1] / s;
        east[1] = n[0] / s;
        east[2] = 0.0;
        north[0] = -n[2] * n[0] / s;
        north[1] = -n[2] * n[1] / s;
        north[2] = s;
    } else {
        east[0] = 0.0;
        east[1] = 1.0;
        east[2] = 0.0;
        north[0] = n[2] > 0 ? -1.0 : 1.0;
        north[1] = 0.0;
        north[2] = 0.0;
    }
}

/* Bin of chord c: k with ce[k] <= c < ce[k+1], or -1.  Also folds the distance
 * to the nearest edge into *margin (relative). */
static int find_bin(double c, int nb, const double* ce, double* margin) {
    for (int e = 0; e <= nb; ++e) {
        const double m = fabs(c - ce[e]) / ce[e];
        if (m < *margin) *margin = m;
    }
    if (c < ce[0] || c >= ce[nb]) return -1;
    int lo = 0, hi = nb; /* ce[lo] <= c < ce[hi] */
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (c >= ce[mid]) lo = mid; else hi = mid;
    }
    return lo;
}

/* -------------------------------------------------------------- moments */

/*
 * For each pivot piv[t] (t < npiv): the moments a (npiv x nb x (M+1) x 2: re, im),
 * W, Q, QW (npiv x nb).  psi (nullable): per-pivot rotation of the reference
 * direction, phi -> phi - psi[t] (used to test the invariance of section 3.1).
 * stats[0] = number of in-bin ordered pairs (pivots with w != 0), stats[1] = the
 * smallest relative chord-to-edge distance seen among candidate pairs.
 * Returns 0 on success.
 */
int orc_moments(int64_t n, const double* xyz, const double* delta, const double* w,
                int64_t npiv, const int64_t* piv, int nb, const double* chord_edges, int M,
                const double* psi, double* a, double* W, double* Q, double* QW,
                double* stats) {
    grid_t g;
    const double cmax = chord_edges[nb];
    if (grid_build(&g, n, xyz, cmax) != 0) return 2;
    const int64_t G = g.G;
    double pairs = 0.0, margin = 1e300;
    const int64_t stride = (int64_t)nb * (M + 1) * 2;

#pragma omp parallel for schedule(dynamic, 16) reduction(+ : pairs) reduction(min : margin)
    for (int64_t t = 0; t < npiv; ++t) {
        const int64_t i = piv[t];
        const double* ni = xyz + 3 * i;
        double east[3], north[3];
        local_frame(ni, east, north);
        double* at = a + t * stride;
        memset(at, 0, sizeof(double) * (size_t)stride);
        for (int k = 0; k < nb; ++k) {
            W[t * nb + k] = 0.0;
            Q[t * nb + k] = 0.0;
            QW[t * nb + k] = 0.0;
        }
        const int64_t cx = cell_coord(ni[0], g.cell, G);
        const int64_t cy = cell_coord(ni[1], g.cell, G);
        const int64_t cz = cell_coord(ni[2], g.cell, G);
        double lmargin = 1e300;
        for (int64_t ix = cx - 1; ix <= cx + 1; ++ix) {
            if (ix < 0 || ix >= G) continue;
            for (int64_t iy = cy - 1; iy <= cy + 1; ++iy) {
                if (iy < 0 || iy >= G) continue;
                for (int64_t iz = cz - 1; iz <= cz + 1; ++iz) {
                    if (iz < 0 || iz >= G) continue;
                    const int64_t c = (ix * G + iy) * G + iz;
                    for (int64_t s = g.start[c]; s < g.start[c + 1]; ++s) {
                        const int64_t j = g.order[s];
                        if (j == i) continue;
                        const double* nj = xyz + 3 * j;
                        const double d0 = nj[0] - ni[0], d1 = nj[1] - ni[1], d2 = nj[2] - ni[2];
                        const double chord = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                        if (chord > 1.5 * cmax) continue;
                        const int k = find_bin(chord, nb, chord_edges, &lmargin);
                        if (k < 0) continue;
                        const double xe = nj[0] * east[0] + nj[1] * east[1] + nj[2] * east[2];
                        const double xn = nj[0] * north[0] + nj[1] * north[1] + nj[2] * north[2];
                        double phi = atan2(xe, xn);
                        if (psi) phi -= psi[t];
                        const double wd = w[j] * delta[j];
                        double* ak = at + (int64_t)k * (M + 1) * 2;
                        for (int m = 0; m <= M; ++m) {
                            ak[2 * m] += wd * cos((double)m * phi);
                            ak[2 * m + 1] -= wd * sin((double)m * phi);
                        }
                        W[t * nb + k] += w[j];
                        Q[t * nb + k] += wd * wd;
                        QW[t * nb + k] += w[j] * w[j];
                        if (w[i] != 0.0) pairs += 1.0;
                    }
                }
            }
        }
        if (lmargin < margin) margin = lmargin;
    }
    grid_free(&g);
    stats[0] = pairs;
    stats[1] = margin;
    return 0;
}

/*
 * Neighbour legs of the adjoint.  P = piv[0..npiv) is the pivot set whose
 * h (npiv x nb x (M+1) x 2) is given.  For every target tgt[u]:
 *   g[u] = w_p * sum_{i in P, i != p, theta_ip in bin k} w_i d_i sum_m Re[exp(-i m phi_ip) h_m^k(i)]
 * with phi_ip the position angle of p about pivot i.
 */
int orc_neighbor_legs(int64_t n, const double* xyz, const double* delta, const double* w,
                      int64_t npiv, const int64_t* piv, const double* h, int nb,
                      const double* chord_edges, int M, int64_t ntgt, const int64_t* tgt,
                      double* gout) {
    grid_t g;
    const double cmax = chord_edges[nb];
    if (grid_build(&g, n, xyz, cmax) != 0) return 2;
    int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!pos) return 2;
    for (int64_t i = 0; i < n; ++i) pos[i] = -1;
    for (int64_t t = 0; t < npiv; ++t) pos[piv[t]] = t;
    const int64_t G = g.G;
    const int64_t stride = (int64_t)nb * (M + 1) * 2;

#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t u = 0; u < ntgt; ++u) {
        const int64_t p = tgt[u];
        const double* np_ = xyz + 3 * p;
        const int64_t cx = cell_coord(np_[0], g.cell, G);
        const int64_t cy = cell_coord(np_[1], g.cell, G);
        const int64_t cz = cell_coord(np_[2], g.cell, G);
        double acc = 0.0, lmargin = 1e300;
        for (int64_t ix = cx - 1; ix <= cx + 1; ++ix) {
            if (ix < 0 || ix >= G) continue;
            for (int64_t iy = cy - 1; iy <= cy + 1; ++iy) {
                if (iy < 0 || iy >= G) continue;
                for (int64_t iz = cz - 1; iz <= cz + 1; ++iz) {
                    if (iz < 0 || iz >= G) continue;
                    const int64_t c = (ix * G + iy) * G + iz;
                    for (int64_t s = g.start[c]; s < g.start[c + 1]; ++s) {
                        const int64_t i = g.order[s];
                        if (i == p || pos[i] < 0) continue;
                        const double* ni = xyz + 3 * i;
                        const double d0 = np_[0] - ni[0], d1 = np_[1] - ni[1], d2 = np_[2] - ni[2];
                        const double chord = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                        if (chord > 1.5 * cmax) continue;
                        const int k = find_bin(chord, nb, chord_edges, &lmargin);
                        if (k < 0) continue;
                        double east[3], north[3];
                        local_frame(ni, east, north);
                        const double xe = np_[0] * east[0] + np_[1] * east[1] + np_[2] * east[2];
                        const double xn = np_[0] * north[0] + np_[1] * north[1] + np_[2] * north[2];
                        const double phi = atan2(xe, xn);
                        const double* hk = h + pos[i] * stride + (int64_t)k * (M + 1) * 2;
                        double sm = 0.0;
                        for (int m = 0; m <= M; ++m) /* Re[(cos - i sin)(hr + i hi)] */
                            sm += cos((double)m * phi) * hk[2 * m] + sin((double)m * phi) * hk[2 * m + 1];
                        acc += w[i] * delta[i] * sm;
                    }
                }
            }
        }
        gout[u] = w[p] * acc;
    }
    free(pos);
    grid_free(&g);
    return 0;
}

/* Number of in-bin ordered pairs around each pivot (a plain pair count used by
 * the benchmark's CPU baseline bookkeeping and by tests). */
int orc_pair_counts(int64_t n, const double* xyz, int64_t npiv, const int64_t* piv, int nb,
                    const double* chord_edges, int64_t* counts) {
    grid_t g;
    const double cmax = chord_edges[nb];
    if (grid_build(&g, n, xyz, cmax) != 0) return 2;
    const int64_t G = g.G;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < npiv; ++t) {
        const int64_t i = piv[t];
        const double* ni = xyz + 3 * i;
        const int64_t cx = cell_coord(ni[0], g.cell, G);
        const int64_t cy = cell_coord(ni[1], g.cell, G);
        const int64_t cz = cell_coord(ni[2], g.cell, G);
        int64_t cnt = 0;
        double lm = 1e300;
        for (int64_t ix = cx - 1; ix <= cx + 1; ++ix) {
            if (ix < 0 || ix >= G) continue;
            for (int64_t iy = cy - 1; iy <= cy + 1; ++iy) {
                if (iy < 0 || iy >= G) continue;
                for (int64_t iz = cz - 1; iz <= cz + 1; ++iz) {
                    if (iz < 0 || iz >= G) continue;
                    const int64_t c = (ix * G + iy) * G + iz;
                    for (int64_t s = g.start[c]; s < g.start[c + 1]; ++s) {
                        const int64_t j = g.order[s];
                        if (j == i) continue;
                        const double* nj = xyz + 3 * j;
                        const double d0 = nj[0] - ni[0], d1 = nj[1] - ni[1], d2 = nj[2] - ni[2];
                        const double chord = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                        if (chord > 1.5 * cmax) continue;
                        if (find_bin(chord, nb, chord_edges, &lm) >= 0) ++cnt;
                    }
                }
            }
        }
        counts[t] = cnt;
    }
    grid_free(&g);
    return 0;
}
