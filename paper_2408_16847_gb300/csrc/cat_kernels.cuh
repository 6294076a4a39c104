// Catalogue forward kernel: the estimator of Sec. 3.1 (eqs. Xm.binned, zetamEst)
// for points at arbitrary positions, found through the plan's sphere grid.
//
// A tile is 32 consecutive points of the grid order (spatially compact), one pivot
// per lane.  Warp 0 bounds the tile's live pivots by a cap (centre, radius R); every
// point within R + theta_max of the centre lies in the cells the cap overlaps, which
// are a handful of contiguous index ranges per colatitude band.  Every warp walks the
// bands in reach and takes every 8th chunk of 32 candidates (so the warps finish
// together), stages the chunk in shared memory and lets each lane pair its pivot with
// all 32.  Per pair: the chord from fp32 hi/lo positions,
// the bin from a log-scale lookup table (FP64 check within CAT_AMB of an edge), the
// position angle from the pivot's local north/east basis, the harmonics by the
// stable three-term recurrence of map_kernels.cuh (harmonics()).  The per-lane
// register sums follow one bin at a time and are added into the tile's shared-memory moments when the bin changes; the tile
// contraction and the cross-CTA reduction are those of the map path.
#pragma once

#include "map_kernels.cuh"

namespace tpcf {

constexpr float CAT_AMB = 2.0e-6f;  // relative margin of fp32 chord^2 to an edge (error ~3e-7)
constexpr float CAT_MARGIN = 8.0e-6f;  // angular margin of the fp32 cell query (rad)

// Bin of chord^2 in fp64 over the edges (ties to the upper bin) for sorted points j
// (candidate) and si (pivot; si < 0: the placeholder pivot (0, 0, 1) of a padding
// lane): -1 below the first edge, K at or beyond the last.
static __device__ __noinline__ int cat_exact_bin(const double* __restrict__ Ed2, int K, const double* __restrict__ xyz,
                                          int64_t j, int64_t si) {
    const double px = si >= 0 ? xyz[3 * si] : 0.0, py = si >= 0 ? xyz[3 * si + 1] : 0.0,
                 pz = si >= 0 ? xyz[3 * si + 2] : 1.0;
    const double dx = xyz[3 * j] - px, dy = xyz[3 * j + 1] - py, dz = xyz[3 * j + 2] - pz;
    const double c2 = dx * dx + dy * dy + dz * dz;
    int k = -1;
    while (k < K && c2 >= Ed2[k + 1]) ++k;
    return k;
}

// fp32 bin of c2 from the lookup table, corrected against the fp32 edges.
__device__ __forceinline__ int cat_bin(float c2, const float* sE2, const unsigned char* slut, float l0, float linv,
                                       int K) {
    const float x = (__log2f(c2) - l0) * linv;
    int k = x < 0.0f ? -1 : (x >= (float)CAT_LUT ? K : (int)slut[(int)x]);
    while (k < K && c2 >= sE2[k + 1]) ++k;
    while (k >= 0 && c2 < sE2[k]) --k;
    return k;
}

template <int M, bool SELF>
__device__ __forceinline__ void cat_flush(float* sA, float* sW, float* sQ, float* sQW, int k, int lane,
                                          float2 (&acc)[M + 1], float& W, float& Q, float& QW) {
    float* a = sA + (size_t)k * (M + 1) * 2 * TILE;
    atomicAdd(a + lane, acc[0].x);
    acc[0] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int m = 1; m <= M; ++m) {
        atomicAdd(a + (2 * m) * TILE + lane, acc[m].x);
        atomicAdd(a + (2 * m + 1) * TILE + lane, acc[m].y);
        acc[m] = make_float2(0.0f, 0.0f);
    }
    atomicAdd(sW + k * TILE + lane, W);
    W = 0.0f;
    if (SELF) {
        atomicAdd(sQ + k * TILE + lane, Q);
        atomicAdd(sQW + k * TILE + lane, QW);
        Q = 0.0f;
        QW = 0.0f;
    }
}

// Shared memory of the catalogue forward beyond the tile's moments: per-warp
// staging of 32 candidates (hi, lo positions and (w d, w)).
template <int M>
__host__ __device__ inline size_t cat_tile_bytes(int K) {
    return tile_floats<M>(K) * sizeof(float) + (size_t)NWARPS * TILE * (2 * sizeof(float4) + sizeof(float2));
}

// The lane's pivot: fp32 hi/lo position, local north / east basis and its sorted
// index (the FP64 position is read only for the rare exact bin decisions).
struct CatPivot {
    float hx, hy, hz, lx, ly, lz;
    float nx, ny, nz, ex, ey;
    int64_t si;
};

// si < 0: a padding lane, placed at (0, 0, 1).
__device__ __forceinline__ CatPivot cat_pivot(const CatDev& g, int64_t si) {
    CatPivot P;
    P.si = si;
    float4 h = make_float4(0.0f, 0.0f, 1.0f, 0.0f), l = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (si >= 0) {
        h = g.p_hi[si];
        l = g.p_lo[si];
    }
    P.hx = h.x;
    P.hy = h.y;
    P.hz = h.z;
    P.lx = l.x;
    P.ly = l.y;
    P.lz = l.z;
    // the basis in fp32 (its rounding is a fixed rotation of the pivot's frame, which
    // cancels in a conj(a), plus ~1e-7 of non-orthogonality)
    const float s2 = fmaf(P.hx, P.hx, P.hy * P.hy);
    if (s2 > 1e-12f) {
        const float is = rsqrtf(s2);
        P.ex = -P.hy * is;  // east = z x n / |z x n|
        P.ey = P.hx * is;
        P.nx = -P.hz * P.hx * is;  // north = n x east
        P.ny = -P.hz * P.hy * is;
        P.nz = s2 * is;
    } else {  // on the axis: any tangent basis of the same handedness
        P.ex = 0.0f;
        P.ey = 1.0f;
        P.nx = -P.hz;
        P.ny = 0.0f;
        P.nz = 0.0f;
    }
    return P;
}

// Warp 0: a cap holding every live pivot of the tile together with its neighbours
// (radius theta_max), as a range of cell bands and a longitude half-width about the
// cap's centre: s_cap = (phi_c, dphi, first band, last band, full).  All in fp32:
// CAT_MARGIN (rad) exceeds every rounding of the centre, radius, colatitude and band
// division (each below ~1e-6 rad), and the sine ratio is rounded up, so the cells are
// a superset of the exact cap; bins are then decided per candidate.  The caller
// synchronises afterwards.
__device__ __forceinline__ void cat_tile_cap(const CatDev& g, bool live, const CatPivot& P, float* s_cap) {
    const float px = P.hx + P.lx, py = P.hy + P.ly, pz = P.hz + P.lz;
    float sx = live ? px : 0.0f, sy = live ? py : 0.0f, sz = live ? pz : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
    }
    float nrm = sqrtf(fmaf(sx, sx, fmaf(sy, sy, sz * sz)));
    if (!(nrm > 1e-6f)) {  // live pivots cancel out: any centre will do (r is measured from it)
        sx = 0.0f;
        sy = 0.0f;
        sz = 1.0f;
        nrm = 1.0f;
    }
    const float cx = sx / nrm, cy = sy / nrm, cz = sz / nrm;
    float r = 0.0f;
    if (live) {
        const float dx = px - cx, dy = py - cy, dz = pz - cz;
        const float ch = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        r = 2.0f * asinf(fminf(1.0f, 0.5f * ch));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    if ((threadIdx.x & 31) == 0) {
        const float PI_F = 3.14159265f;
        const float Q = r + (float)g.theta_max + CAT_MARGIN;
        const float thc = atan2f(sqrtf(fmaf(cx, cx, cy * cy)), cz);
        float phc = atan2f(cy, cx);
        if (phc < 0.0f) phc += 2.0f * PI_F;
        int b0 = 0, b1 = g.nbands - 1;
        float full = 1.0f, dphi = PI_F;
        const float lo = thc - Q - CAT_MARGIN, hi = thc + Q + CAT_MARGIN;
        if (Q < PI_F) {
            const float hb = (float)g.hband;
            b0 = max(0, (int)floorf(lo / hb));
            b1 = min(g.nbands - 1, (int)floorf(hi / hb));
            if (lo > 0.0f && hi < PI_F) {  // no pole inside: then Q < pi / 2, sin rises with Q
                // sin is concave on [0, pi]: its least value over thc +- margin is at an end
                const float st = fminf(sinf(thc - CAT_MARGIN), sinf(thc + CAT_MARGIN));
                const float x = sinf(Q) / st * (1.0f + 1.0e-6f);
                if (x < 1.0f) {
                    full = 0.0f;
                    dphi = asinf(x) + CAT_MARGIN;
                }
            }
        }
        s_cap[0] = phc;
        s_cap[1] = dphi;
        s_cap[2] = (float)b0;
        s_cap[3] = (float)b1;
        s_cap[4] = full;
    }
}

// Every candidate of the cap for this warp, with its bin k (-1 below the first edge,
// K beyond the last), the chord vector from the lane's pivot, its (w d, w) and its
// sorted index: f(k, dx, dy, dz, v, j).  Calls are warp-uniform (every lane sees the
// same candidate at the same time).  Candidates are staged 32 at a
// time in the warp's shared buffers wh / wl / wv.
template <class F>
__device__ __forceinline__ void cat_walk(const CatDev& g, const float2* __restrict__ wdw, const float* s_cap,
                                         const CatPivot& P, const float* sE2, const unsigned char* slut,
                                         float4* wh, float4* wl, float2* wv, F&& f) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = g.K;
    // sector bounds in fp32: the extra 4e-6 rad covers its rounding (phi < 2 pi), so the
    // cell ranges stay a superset of the cap
    const float phc = s_cap[0], dphi = s_cap[1] + 4.0e-6f;
    const int b0 = (int)s_cap[2], b1 = (int)s_cap[3];
    const bool full = s_cap[4] != 0.0f;
    // every warp walks every band and takes every NWARPS-th chunk of 32 candidates
    int chunk = 0;
    for (int b = b0; b <= b1; ++b) {
        const int64_t ns = g.band_ns[b];
        const int64_t cf = g.band_first[b];
        // at most two cell ranges (the sector range may wrap around phi = 0)
        int64_t ca0 = cf, ca1 = cf + ns, cb0 = 0, cb1 = 0;
        if (!full) {
            const float scale = (float)ns * (float)(0.5 / M_PI);
            const int64_t sa = (int64_t)floorf((phc - dphi) * scale);
            const int64_t sb = (int64_t)floorf((phc + dphi) * scale);
            const int64_t len = sb - sa + 1;
            if (len < ns) {
                int64_t s0 = sa % ns;
                if (s0 < 0) s0 += ns;
                ca0 = cf + s0;
                if (s0 + len <= ns) {
                    ca1 = cf + s0 + len;
                } else {
                    ca1 = cf + ns;
                    cb0 = cf;
                    cb1 = cf + (s0 + len - ns);
                }
            }
        }
#pragma unroll 1
        for (int sg = 0; sg < 2; ++sg) {
            const int64_t cl0 = sg == 0 ? ca0 : cb0, cl1 = sg == 0 ? ca1 : cb1;
            if (cl1 <= cl0) continue;
            const int64_t p0 = g.cell_start[cl0], p1 = g.cell_start[cl1];
            for (int64_t base = p0; base < p1; base += TILE, ++chunk) {
                if ((chunk % NWARPS) != warp) continue;
                const int64_t j = base + lane;
                __syncwarp();
                if (j < p1) {
                    wh[lane] = g.p_hi[j];
                    wl[lane] = g.p_lo[j];
                    wv[lane] = wdw[j];
                }
                __syncwarp();
                const int cnt = (int)min((int64_t)TILE, p1 - base);
                for (int u = 0; u < cnt; ++u) {
                    const float4 qh = wh[u], ql = wl[u];
                    const float dx = (qh.x - P.hx) + (ql.x - P.lx);
                    const float dy = (qh.y - P.hy) + (ql.y - P.ly);
                    const float dz = (qh.z - P.hz) + (ql.z - P.lz);
                    const float c2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    int k = cat_bin(c2, sE2, slut, g.lut_l0, g.lut_inv, K);
                    const int e1 = max(k, 0), e2 = min(k + 1, K);
                    if (fabsf(c2 - sE2[e1]) <= CAT_AMB * sE2[e1] || fabsf(c2 - sE2[e2]) <= CAT_AMB * sE2[e2])
                        k = cat_exact_bin(g.Ed2, K, g.xyz, (int64_t)__float_as_int(ql.w), P.si);
                    f(k, dx, dy, dz, wv[u], __float_as_int(ql.w));
                }
            }
        }
    }
}

// The candidates of the cap grouped by bin, chunk by chunk.  For each staged chunk of
// 32 candidates, pass A bins every candidate for the lane's pivot and records, per
// lane, one bit mask per bin kb + j (j = 0..GROUPS-1, kb = the first in-range bin seen
// in the chunk minus three; a tile's pivots lie close together, so the candidates of a
// chunk cover few bins for every lane) plus a mask of the rare in-range candidates
// beyond that window; out-of-range candidates are dropped there.  With 8 bins in the
// window about 6% of the in-range candidates of the 2e6-point catalogue fall outside
// it (30% with 4), each of which costs a flush of the register sums.  Pass B then runs,
// for each j in lockstep, every lane over the candidates of its own bin kb + j:
//     pair(active, k, dx, dy, dz, v, u)   for each candidate (u its slot in the chunk;
//                                         active false on padding iterations, where k
//                                         may be out of range and must not be used)
//     group_end(k, nonempty)              once per j, warp-uniform
// and the candidates beyond the window one by one: single(k, dx, dy, dz, v, u).
// chunk_end(base, cnt) closes each chunk (uniform).  This replaces per-candidate bin
// changes (a divergent flush whenever one lane's bin changed) by a uniform flush per
// bin and chunk.
constexpr int CAT_GROUPS = 8;

template <class FP, class FE, class FS, class FC>
__device__ __forceinline__ void cat_walk_grouped(const CatDev& g, const float2* __restrict__ wdw,
                                                 const float* s_cap, const CatPivot& P, const float* sE2,
                                                 const unsigned char* slut, float4* wh, float4* wl, float2* wv,
                                                 FP&& pair, FE&& group_end, FS&& single, FC&& chunk_end) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = g.K;
    const float phc = s_cap[0], dphi = s_cap[1] + 4.0e-6f;
    const int b0 = (int)s_cap[2], b1 = (int)s_cap[3];
    const bool full = s_cap[4] != 0.0f;
    int chunk = 0;
    for (int b = b0; b <= b1; ++b) {
        const int64_t ns = g.band_ns[b];
        const int64_t cf = g.band_first[b];
        int64_t ca0 = cf, ca1 = cf + ns, cb0 = 0, cb1 = 0;
        if (!full) {
            const float scale = (float)ns * (float)(0.5 / M_PI);
            const int64_t sa = (int64_t)floorf((phc - dphi) * scale);
            const int64_t sb = (int64_t)floorf((phc + dphi) * scale);
            const int64_t len = sb - sa + 1;
            if (len < ns) {
                int64_t s0 = sa % ns;
                if (s0 < 0) s0 += ns;
                ca0 = cf + s0;
                if (s0 + len <= ns) {
                    ca1 = cf + s0 + len;
                } else {
                    ca1 = cf + ns;
                    cb0 = cf;
                    cb1 = cf + (s0 + len - ns);
                }
            }
        }
#pragma unroll 1
        for (int sg = 0; sg < 2; ++sg) {
            const int64_t cl0 = sg == 0 ? ca0 : cb0, cl1 = sg == 0 ? ca1 : cb1;
            if (cl1 <= cl0) continue;
            const int64_t p0 = g.cell_start[cl0], p1 = g.cell_start[cl1];
            for (int64_t base = p0; base < p1; base += TILE, ++chunk) {
                if ((chunk % NWARPS) != warp) continue;
                const int64_t j = base + lane;
                __syncwarp();
                if (j < p1) {
                    wh[lane] = g.p_hi[j];
                    wl[lane] = g.p_lo[j];
                    wv[lane] = wdw[j];
                }
                __syncwarp();
                const int cnt = (int)min((int64_t)TILE, p1 - base);
                // pass A: bins, per-lane masks
                unsigned mk[CAT_GROUPS];
#pragma unroll
                for (int q = 0; q < CAT_GROUPS; ++q) mk[q] = 0u;
                unsigned mo = 0u;
                int kb = -1000;
                for (int u = 0; u < cnt; ++u) {
                    const float4 qh = wh[u], ql = wl[u];
                    const float dx = (qh.x - P.hx) + (ql.x - P.lx);
                    const float dy = (qh.y - P.hy) + (ql.y - P.ly);
                    const float dz = (qh.z - P.hz) + (ql.z - P.lz);
                    const float c2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    int k = cat_bin(c2, sE2, slut, g.lut_l0, g.lut_inv, K);
                    const int e1 = max(k, 0), e2 = min(k + 1, K);
                    if (fabsf(c2 - sE2[e1]) <= CAT_AMB * sE2[e1] || fabsf(c2 - sE2[e2]) <= CAT_AMB * sE2[e2])
                        k = cat_exact_bin(g.Ed2, K, g.xyz, (int64_t)__float_as_int(ql.w), P.si);
                    if (k < 0 || k >= K) continue;
                    if (kb == -1000) kb = max(k - 3, 0);
                    const int q = k - kb;
                    const unsigned bit = 1u << u;
#pragma unroll
                    for (int r = 0; r < CAT_GROUPS; ++r)
                        if (q == r) mk[r] |= bit;
                    if (q < 0 || q >= CAT_GROUPS) mo |= bit;
                }
                // pass B: per bin of the window, in lockstep
#pragma unroll 1
                for (int r = 0; r < CAT_GROUPS; ++r) {
                    unsigned msk = 0u;
#pragma unroll
                    for (int q = 0; q < CAT_GROUPS; ++q)
                        if (q == r) msk = mk[q];
                    const bool had = msk != 0u;
                    if (!__any_sync(0xffffffffu, had)) continue;
                    while (__any_sync(0xffffffffu, msk != 0u)) {
                        const bool active = msk != 0u;
                        const int u = active ? __ffs(msk) - 1 : 0;
                        msk &= msk - 1u;
                        const float4 qh = wh[u], ql = wl[u];
                        const float dx = (qh.x - P.hx) + (ql.x - P.lx);
                        const float dy = (qh.y - P.hy) + (ql.y - P.ly);
                        const float dz = (qh.z - P.hz) + (ql.z - P.lz);
                        pair(active, kb + r, dx, dy, dz, wv[u], u);
                    }
                    group_end(kb + r, had);
                }
                // the rare in-range candidates outside the window, one by one
                while (__any_sync(0xffffffffu, mo != 0u)) {
                    const bool active = mo != 0u;
                    const int u = active ? __ffs(mo) - 1 : 0;
                    mo &= mo - 1u;
                    if (active) {
                        const float4 qh = wh[u], ql = wl[u];
                        const float dx = (qh.x - P.hx) + (ql.x - P.lx);
                        const float dy = (qh.y - P.hy) + (ql.y - P.ly);
                        const float dz = (qh.z - P.hz) + (ql.z - P.lz);
                        const float c2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        int k = cat_bin(c2, sE2, slut, g.lut_l0, g.lut_inv, K);
                        const int e1 = max(k, 0), e2 = min(k + 1, K);
                        if (fabsf(c2 - sE2[e1]) <= CAT_AMB * sE2[e1] || fabsf(c2 - sE2[e2]) <= CAT_AMB * sE2[e2])
                            k = cat_exact_bin(g.Ed2, K, g.xyz, (int64_t)__float_as_int(ql.w), P.si);
                        single(k, dx, dy, dz, wv[u], u);
                    }
                }
                chunk_end(base, cnt);
            }
        }
    }
}

// The tile's moments over the catalogue walk (the body of the forward): every warp
// walks its share of the cap's candidates for the lane's pivot P with the neighbour
// values `wdw` and adds its register sums into the tile's shared moments once per bin
// and chunk.  The caller zeroes the moments before and synchronises after.
template <int M, bool SELF>
__device__ __forceinline__ void cat_tile_moments(const CatDev& g, const float2* __restrict__ wdw,
                                                 const float* s_cap, const CatPivot& P, const float* sE2,
                                                 const unsigned char* slut, float4* sCh, float4* sCl, float2* sCv,
                                                 float* sA, float* sW, float* sQ, float* sQW) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2 acc[M + 1];
#pragma unroll
    for (int m = 0; m <= M; ++m) acc[m] = make_float2(0.0f, 0.0f);
    float W = 0.0f, Qs = 0.0f, QW = 0.0f;
    cat_walk_grouped(
        g, wdw, s_cap, P, sE2, slut, sCh + warp * TILE, sCl + warp * TILE, sCv + warp * TILE,
        [&](bool active, int, float dx, float dy, float dz, float2 v, int) {
            const float N = fmaf(dx, P.nx, fmaf(dy, P.ny, dz * P.nz));
            const float E = fmaf(dx, P.ex, dy * P.ey);
            const float rinv = rsqrtf(fmaxf(fmaf(N, N, E * E), 1e-30f));
            const float wd = active ? v.x : 0.0f;
            const float ww = active ? v.y : 0.0f;
            harmonics<M>(acc, N * rinv, E * rinv, wd, wd);
            W += ww;
            if (SELF) {
                Qs = fmaf(wd, wd, Qs);
                QW = fmaf(ww, ww, QW);
            }
        },
        [&](int k, bool had) {
            if (had) {
                cat_flush<M, SELF>(sA, sW, sQ, sQW, k, lane, acc, W, Qs, QW);
            }
        },
        [&](int k, float dx, float dy, float dz, float2 v, int) {
            // every group is flushed by now, so the register sums are free
            const float N = fmaf(dx, P.nx, fmaf(dy, P.ny, dz * P.nz));
            const float E = fmaf(dx, P.ex, dy * P.ey);
            const float rinv = rsqrtf(fmaxf(fmaf(N, N, E * E), 1e-30f));
            harmonics<M>(acc, N * rinv, E * rinv, v.x, v.x);
            W = v.y;
            if (SELF) {
                Qs = v.x * v.x;
                QW = v.y * v.y;
            }
            cat_flush<M, SELF>(sA, sW, sQ, sQW, k, lane, acc, W, Qs, QW);
        },
        [&](int64_t, int) {});
}

template <int M, bool SELF>
__global__ void __launch_bounds__(NTHREADS, 3) cat_fwd_kernel(CatDev g, MapCall c) {
    extern __shared__ __align__(16) float smem[];
    __shared__ int s_tile;
    __shared__ float s_cap[5];  // cap query: phi_c, dphi, first band, last band, full
    __shared__ float sE2[TPCF_MAX_BINS + 1];
    __shared__ unsigned char slut[CAT_LUT];
    const int K = g.K;
    float* sA = smem;
    float* sW = sA + (size_t)K * (M + 1) * 2 * TILE;
    float* sQ = sW + K * TILE;
    float* sQW = sQ + K * TILE;
    float* sPiv = sQW + K * TILE;
    float4* sCh = reinterpret_cast<float4*>(smem + tile_floats<M>(K));
    float4* sCl = sCh + NWARPS * TILE;
    float2* sCv = reinterpret_cast<float2*>(sCl + NWARPS * TILE);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t nfl = tile_floats<M>(K) - 2 * TILE;
    for (int e = threadIdx.x; e <= K; e += NTHREADS) sE2[e] = g.E2[e];
    for (int e = threadIdx.x; e < CAT_LUT; e += NTHREADS) slut[e] = g.lut[e];
    double* slot = c.slots + (size_t)blockIdx.x * n_entries(K, M);

    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(c.counter, 1);
        __syncthreads();
        const int tile = s_tile;
        if ((long long)tile >= g.ntiles) break;
        const int64_t si = (int64_t)tile * TILE + lane;
        bool live = false;
        float2 pv = make_float2(0.0f, 0.0f);
        if (si < g.n) {
            const int64_t o = g.orig[si];
            if (o >= c.piv_lo && o < c.piv_hi) {
                pv = c.wdw[si];
                live = pv.y != 0.0f;
                if (!live) pv = make_float2(0.0f, 0.0f);
            }
        }
        if (!__syncthreads_or(live)) continue;
        for (size_t e = threadIdx.x; e < nfl; e += NTHREADS) sA[e] = 0.0f;
        if (threadIdx.x < TILE) {
            sPiv[lane] = pv.x;
            sPiv[TILE + lane] = pv.y;
        }
        const CatPivot P = cat_pivot(g, si < g.n ? si : -1);
        if (warp == 0) cat_tile_cap(g, live, P, s_cap);
        __syncthreads();

        cat_tile_moments<M, SELF>(g, c.wdw, s_cap, P, sE2, slut, sCh, sCl, sCv, sA, sW, sQ, sQW);
        __syncthreads();
        if (c.norm != NORM_NONE) tile_normalize<M>(K, sA, sW, c.norm);
        tile_contract<M>(K, sA, sW, sQ, sQW, sPiv, slot, SELF);
        __syncthreads();
    }
}

// Multi-field forward on a catalogue (tpcf_forward_multi): three fields on the same
// points, each with its own weights.  The tile's cap is walked once per field (the
// moments of the neighbour fields A, B, C), and tile_contract_multi forms the cyclic
// sum over the pivot field.  Shared memory: the three fields' moments, the pivots'
// three (w d, w), and the per-warp candidate staging.
template <int M>
__host__ __device__ inline size_t cat_multi_bytes(int K) {
    return multi_tile_floats(K, M) * sizeof(float) + (size_t)NWARPS * TILE * (2 * sizeof(float4) + sizeof(float2));
}

template <int M>
__global__ void __launch_bounds__(NTHREADS, 1) cat_fwd_multi_kernel(CatDev g, MapCall c,
                                                                    const float2* __restrict__ wdwB,
                                                                    const float2* __restrict__ wdwC) {
    extern __shared__ __align__(16) float smem[];
    __shared__ int s_tile;
    __shared__ float s_cap[5];
    __shared__ float sE2[TPCF_MAX_BINS + 1];
    __shared__ unsigned char slut[CAT_LUT];
    const int K = g.K;
    const size_t fsz = multi_field_floats(K, M);
    float* sF = smem;
    float* sPiv = smem + 3 * fsz;  // [field][w d, w][32]
    float4* sCh = reinterpret_cast<float4*>(smem + multi_tile_floats(K, M));
    float4* sCl = sCh + NWARPS * TILE;
    float2* sCv = reinterpret_cast<float2*>(sCl + NWARPS * TILE);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = threadIdx.x; e <= K; e += NTHREADS) sE2[e] = g.E2[e];
    for (int e = threadIdx.x; e < CAT_LUT; e += NTHREADS) slut[e] = g.lut[e];
    double* slot = c.slots + (size_t)blockIdx.x * n_entries_multi(K, M);
    const float2* arr[3] = {c.wdw, wdwB, wdwC};
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(c.counter, 1);
        __syncthreads();
        const int tile = s_tile;
        if ((long long)tile >= g.ntiles) break;
        const int64_t si = (int64_t)tile * TILE + lane;
        float2 pv[3] = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
        bool live = false;
        if (si < g.n) {
            const int64_t o = g.orig[si];
            if (o >= c.piv_lo && o < c.piv_hi) {
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    pv[f] = arr[f][si];
                    live = live || pv[f].y != 0.0f;
                }
            }
        }
        if (!__syncthreads_or(live)) continue;
        for (size_t e = threadIdx.x; e < 3 * fsz; e += NTHREADS) sF[e] = 0.0f;
        if (threadIdx.x < TILE) {
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                sPiv[f * 2 * TILE + lane] = pv[f].x;
                sPiv[f * 2 * TILE + TILE + lane] = pv[f].y;
            }
        }
        const CatPivot P = cat_pivot(g, si < g.n ? si : -1);
        if (warp == 0) cat_tile_cap(g, live, P, s_cap);
        __syncthreads();
#pragma unroll 1
        for (int f = 0; f < 3; ++f) {
            float* sA = sF + f * fsz;
            cat_tile_moments<M, false>(g, arr[f], s_cap, P, sE2, slut, sCh, sCl, sCv, sA,
                                       sA + (size_t)K * (M + 1) * 2 * TILE, nullptr, nullptr);
        }
        __syncthreads();
        tile_contract_multi<M>(K, sF, sPiv, slot);
        __syncthreads();
    }
}

// Shared memory of the catalogue adjoint: the forward's, plus one m of H and the
// primary-term sums.
template <int M>
__host__ __device__ inline size_t cat_bwd_bytes(int K) {
    return cat_tile_bytes<M>(K) + ((size_t)K * K * 2 + TILE + NWARPS * TILE) * sizeof(float);
}

// Catalogue adjoint, dL/d(delta_p) (the map adjoint's three phases on the catalogue
// walk): phase 1 recomputes the tile's moments, phase 2 forms h = H conj(a) in place
// and the primary term, phase 3 walks the candidates again and adds
// w_j w_i d_i sum_m (cos(m phi) Re h_m^k + sin(m phi) Im h_m^k) for every in-bin pair;
// the 32 pivots' contributions to one candidate are summed across the warp before one
// atomic add to its gradient.
template <int M>
__global__ void __launch_bounds__(NTHREADS, 2) cat_bwd_kernel(CatDev g, MapCall c) {
    extern __shared__ __align__(16) float smem[];
    __shared__ int s_tile;
    __shared__ float s_cap[5];
    __shared__ float sE2[TPCF_MAX_BINS + 1];
    __shared__ unsigned char slut[CAT_LUT];
    const int K = g.K;
    float* sA = smem;
    float* sW = sA + (size_t)K * (M + 1) * 2 * TILE;
    float* sQ = sW + K * TILE;
    float* sQW = sQ + K * TILE;
    float* sPiv = sQW + K * TILE;
    float4* sCh = reinterpret_cast<float4*>(smem + tile_floats<M>(K));
    float4* sCl = sCh + NWARPS * TILE;
    float2* sCv = reinterpret_cast<float2*>(sCl + NWARPS * TILE);
    float* sHm = reinterpret_cast<float*>(sCv + NWARPS * TILE);  // [K][K][2], one m at a time
    float* sPrim = sHm + (size_t)K * K * 2;                       // [TILE], then sG [NWARPS][TILE]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t nfl = tile_floats<M>(K) - 2 * TILE;
    for (int e = threadIdx.x; e <= K; e += NTHREADS) sE2[e] = g.E2[e];
    for (int e = threadIdx.x; e < CAT_LUT; e += NTHREADS) slut[e] = g.lut[e];

    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(c.counter, 1);
        __syncthreads();
        const int tile = s_tile;
        if ((long long)tile >= g.ntiles) break;
        const int64_t si = (int64_t)tile * TILE + lane;
        bool live = false;
        float2 pv = make_float2(0.0f, 0.0f);
        int64_t oi = -1;
        if (si < g.n) {
            oi = g.orig[si];
            if (oi >= c.piv_lo && oi < c.piv_hi) {
                pv = c.wdw[si];
                live = pv.y != 0.0f;
                if (!live) pv = make_float2(0.0f, 0.0f);
            }
        }
        if (!__syncthreads_or(live)) continue;
        for (size_t e = threadIdx.x; e < nfl; e += NTHREADS) sA[e] = 0.0f;
        if (threadIdx.x < TILE) {
            sPiv[lane] = pv.x;
            sPiv[TILE + lane] = pv.y;
            sPrim[lane] = 0.0f;
        }
        const CatPivot P = cat_pivot(g, si < g.n ? si : -1);
        if (warp == 0) cat_tile_cap(g, live, P, s_cap);
        __syncthreads();

        // phase 1: the moments, as in the forward
        {
            float2 acc[M + 1];
#pragma unroll
            for (int m = 0; m <= M; ++m) acc[m] = make_float2(0.0f, 0.0f);
            float W = 0.0f, Qs = 0.0f, QW = 0.0f;
            cat_walk_grouped(
                g, c.wdw, s_cap, P, sE2, slut, sCh + warp * TILE, sCl + warp * TILE, sCv + warp * TILE,
                [&](bool active, int, float dx, float dy, float dz, float2 v, int) {
                    const float N = fmaf(dx, P.nx, fmaf(dy, P.ny, dz * P.nz));
                    const float E = fmaf(dx, P.ex, dy * P.ey);
                    const float rinv = rsqrtf(fmaxf(fmaf(N, N, E * E), 1e-30f));
                    const float wd = active ? v.x : 0.0f;
                    harmonics<M>(acc, N * rinv, E * rinv, wd, wd);
                    W += active ? v.y : 0.0f;
                },
                [&](int k, bool had) {
                    if (had) cat_flush<M, false>(sA, sW, sQ, sQW, k, lane, acc, W, Qs, QW);
                },
                [&](int k, float dx, float dy, float dz, float2 v, int) {
                    const float N = fmaf(dx, P.nx, fmaf(dy, P.ny, dz * P.nz));
                    const float E = fmaf(dx, P.ex, dy * P.ey);
                    const float rinv = rsqrtf(fmaxf(fmaf(N, N, E * E), 1e-30f));
                    harmonics<M>(acc, N * rinv, E * rinv, v.x, v.x);
                    W = v.y;
                    cat_flush<M, false>(sA, sW, sQ, sQW, k, lane, acc, W, Qs, QW);
                },
                [&](int64_t, int) {});
        }
        __syncthreads();
        // phase 2: h = H conj(a) per m, in place; primary term (1/2) sum Re[a h]
        for (int m = 0; m <= M; ++m) {
            for (int e = threadIdx.x; e < K * K * 2; e += NTHREADS) sHm[e] = c.H[(size_t)m * K * K * 2 + e];
            __syncthreads();
            float hrv[(TPCF_MAX_BINS * TILE + NTHREADS - 1) / NTHREADS];
            float hiv[(TPCF_MAX_BINS * TILE + NTHREADS - 1) / NTHREADS];
            int nmine = 0;
            for (int e = threadIdx.x; e < K * TILE; e += NTHREADS, ++nmine) {
                const int k = e / TILE, l = e - k * TILE;
                float hr = 0.0f, hi = 0.0f;
                for (int kp = 0; kp < K; ++kp) {
                    const float Hr = sHm[(k * K + kp) * 2], Hi = sHm[(k * K + kp) * 2 + 1];
                    const float* ap = sA + ((size_t)kp * (M + 1) + m) * 2 * TILE;
                    const float tr = ap[l], ti = ap[TILE + l];
                    hr = fmaf(Hr, tr, fmaf(-Hi, ti, hr));
                    hi = fmaf(Hr, ti, fmaf(Hi, tr, hi));
                }
                const float* ak = sA + ((size_t)k * (M + 1) + m) * 2 * TILE;
                atomicAdd(sPrim + l, fmaf(ak[l], hr, ak[TILE + l] * hi));
                hrv[nmine] = hr;
                hiv[nmine] = hi;
            }
            __syncthreads();
            nmine = 0;
            for (int e = threadIdx.x; e < K * TILE; e += NTHREADS, ++nmine) {
                const int k = e / TILE, l = e - k * TILE;
                float* ak = sA + ((size_t)k * (M + 1) + m) * 2 * TILE;
                ak[l] = hrv[nmine];
                ak[TILE + l] = hiv[nmine];
            }
            __syncthreads();
        }
        if (threadIdx.x < TILE && live) {
            const float gp = 0.5f * pv.y * sPrim[lane];
            if (gp != 0.0f) atomicAdd(c.grad + oi, gp);
        }
        // phase 3: the neighbour legs; each candidate's contributions from the warp's
        // 32 pivots are summed in the warp's shared buffer sG, then added once to its
        // gradient entry at the end of the chunk
        {
            float2 h[M + 1];
            int kh = -1;
            const float wdi = pv.x;
            float* sG = sPrim + TILE + warp * TILE;
            sG[lane] = 0.0f;
            __syncwarp();
            auto load_h = [&](int k) {
                const float* hk = sA + (size_t)k * (M + 1) * 2 * TILE;
#pragma unroll
                for (int m = 0; m <= M; ++m)
                    h[m] = make_float2(hk[(2 * m) * TILE + lane], hk[(2 * m + 1) * TILE + lane]);
                kh = k;
            };
            auto leg = [&](float dx, float dy, float dz, float2 v) {
                const float N = fmaf(dx, P.nx, fmaf(dy, P.ny, dz * P.nz));
                const float E = fmaf(dx, P.ex, dy * P.ey);
                const float rinv = rsqrtf(fmaxf(fmaf(N, N, E * E), 1e-30f));
                float X, Y;
                adj_harmonics<M>(h, N * rinv, E * rinv, X, Y);
                return wdi * v.y * (X + Y);
            };
            cat_walk_grouped(
                g, c.wdw, s_cap, P, sE2, slut, sCh + warp * TILE, sCl + warp * TILE, sCv + warp * TILE,
                [&](bool active, int k, float dx, float dy, float dz, float2 v, int u) {
                    // an inactive lane may have no valid bin in this chunk (k is then
                    // out of range): it neither loads h nor adds anything
                    if (active) {
                        if (k != kh) load_h(k);
                        const float val = leg(dx, dy, dz, v);
                        if (val != 0.0f) atomicAdd(sG + u, val);
                    }
                },
                [&](int, bool) {},
                [&](int k, float dx, float dy, float dz, float2 v, int u) {
                    load_h(k);
                    const float val = leg(dx, dy, dz, v);
                    if (val != 0.0f) atomicAdd(sG + u, val);
                },
                [&](int64_t base, int cnt) {
                    __syncwarp();
                    if (lane < cnt) {
                        const float val = sG[lane];
                        if (val != 0.0f) atomicAdd(c.grad + g.orig[base + lane], val);
                        sG[lane] = 0.0f;
                    }
                    __syncwarp();
                });
        }
        __syncthreads();
    }
}

#if defined(TPCF_M) && TPCF_M == 0  // one definition, in the M = 0 object
// Exact number of in-bin ordered pairs (i, j) with w_i != 0 and caller index of i in
// [lo, hi): counts[0] += total.  Same tiles and candidate walk as the forward.
__global__ void __launch_bounds__(NTHREADS) cat_count_kernel(CatDev g, const float2* __restrict__ wdw, long long lo,
                                                             long long hi, int* counter,
                                                             unsigned long long* counts) {
    __shared__ int s_tile;
    __shared__ float s_cap[5];
    __shared__ float sE2[TPCF_MAX_BINS + 1];
    __shared__ unsigned char slut[CAT_LUT];
    __shared__ __align__(16) float4 sCh[NWARPS * TILE];
    __shared__ __align__(16) float4 sCl[NWARPS * TILE];
    __shared__ __align__(16) float2 sCv[NWARPS * TILE];
    const int K = g.K;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = threadIdx.x; e <= K; e += NTHREADS) sE2[e] = g.E2[e];
    for (int e = threadIdx.x; e < CAT_LUT; e += NTHREADS) slut[e] = g.lut[e];
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
        __syncthreads();
        const int tile = s_tile;
        if ((long long)tile >= g.ntiles) break;
        const int64_t si = (int64_t)tile * TILE + lane;
        bool live = false;
        if (si < g.n) {
            const int64_t o = g.orig[si];
            live = o >= lo && o < hi && wdw[si].y != 0.0f;
        }
        if (!__syncthreads_or(live)) continue;
        const CatPivot P = cat_pivot(g, si < g.n ? si : -1);
        if (warp == 0) cat_tile_cap(g, live, P, s_cap);
        __syncthreads();
        unsigned long long cnt = 0;
        cat_walk(g, wdw, s_cap, P, sE2, slut, sCh + warp * TILE, sCl + warp * TILE, sCv + warp * TILE,
                 [&](int k, float, float, float, float2, int) { cnt += (k >= 0 && k < K) ? 1ull : 0ull; });
        cnt = live ? cnt : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0 && cnt) atomicAdd(counts, cnt);
        __syncthreads();
    }
}
#endif

}  // namespace tpcf
