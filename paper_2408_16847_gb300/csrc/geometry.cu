// Plan-build kernels of the map path (all FP64):
//  * the HEALPix RING ring table (Gorski et al. 2005): first pixel, pixel count,
//    half-pixel shift, cos/sin of the colatitude, colatitude;
//  * for every pivot ring i, the neighbour rings r within the outer bin edge and,
//    per bin k, the rings that can hold bin-k pixels;
//  * for every (i, r) pair, A = sin(theta_i - theta_r) and the edge offsets T_e,
//    e = 0..K: a pixel of ring r at longitude offset o (in ring-r pixels) from a
//    pivot of ring i lies inside edge e (theta < theta_e) iff |o| < T_e, because
//    its quarter squared chord is f(o) = sin^2((theta_r - theta_i)/2)
//    + s_i s_r sin^2(pi o / n_r), increasing in |o|;
//  * the tile list: 32 consecutive pivots of a ring per tile.
#include <math.h>

#include "geometry.cuh"

namespace tpcf {

__global__ void ring_table_kernel(int nside, int nrings, int64_t* first, int* npr, int* shift, double* z,
                                  double* s, double* th, float* zf, float* sf, float* sf_lo, float* step,
                                  float* step_lo, float* invn, float* invn_lo) {
    const int ri = blockIdx.x * blockDim.x + threadIdx.x;
    if (ri >= nrings) return;
    const long long n = nside;
    const long long r = ri + 1;  // 1-based ring number from the north pole
    const double nn = (double)nside;
    double zz, ss;
    if (r < n) {
        const double t = (double)(r * r) / (3.0 * nn * nn);
        npr[ri] = (int)(4 * r);
        first[ri] = 2 * r * (r - 1);
        shift[ri] = 1;
        zz = 1.0 - t;
        ss = sqrt(t * (2.0 - t));
    } else if (r > 3 * n) {
        const long long rr = 4 * n - r;
        const double t = (double)(rr * rr) / (3.0 * nn * nn);
        npr[ri] = (int)(4 * rr);
        first[ri] = 12 * n * n - 2 * rr * (rr + 1);
        shift[ri] = 1;
        zz = -(1.0 - t);
        ss = sqrt(t * (2.0 - t));
    } else {
        npr[ri] = (int)(4 * n);
        first[ri] = 2 * n * (n - 1) + 4 * n * (r - n);
        shift[ri] = (int)((r - n + 1) & 1);
        zz = (double)(4 * n - 2 * r) / (3.0 * nn);
        ss = sqrt((1.0 - zz) * (1.0 + zz));
    }
    z[ri] = zz;
    s[ri] = ss;
    th[ri] = atan2(ss, zz);
    zf[ri] = (float)zz;
    sf[ri] = (float)ss;
    sf_lo[ri] = (float)(ss - (double)(float)ss);
    const double st = M_PI / (double)npr[ri], iv = 1.0 / (double)npr[ri];
    step[ri] = (float)st;
    step_lo[ri] = (float)(st - (double)(float)st);
    invn[ri] = (float)iv;
    invn_lo[ri] = (float)(iv - (double)(float)iv);
}

// Rings r with sin^2((theta_r - theta_i)/2) < E form a contiguous range around i.
__device__ __forceinline__ bool within(const double* th, int i, int r, double E) {
    const double h = sin(0.5 * (th[r] - th[i]));
    return h * h < E;
}

__device__ int2 ring_window(const double* th, int nrings, int i, double E) {
    // lowest r <= i inside, highest r >= i inside (i itself is inside for E > 0)
    int lo = 0, hi = i;
    while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (within(th, i, mid, E)) hi = mid; else lo = mid + 1;
    }
    const int rlo = lo;
    lo = i;
    hi = nrings - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (within(th, i, mid, E)) lo = mid; else hi = mid - 1;
    }
    return make_int2(rlo, lo);
}

__global__ void ring_range_kernel(int nrings, int K, const double* th, const double* E, const int* npr,
                                  int2* ring_range, int2* bin_range, int64_t* npairs, int64_t* ntiles) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrings) return;
    const int2 rr = ring_window(th, nrings, i, E[K]);
    ring_range[i] = rr;
    for (int k = 0; k < K; ++k) bin_range[(size_t)i * K + k] = ring_window(th, nrings, i, E[k + 1]);
    npairs[i] = rr.y - rr.x + 1;
    ntiles[i] = (npr[i] + TILE - 1) / TILE;
}

// Exclusive prefix sum of n int64 values by one block (n is at most 4 * 8192 - 1).
__global__ void exclusive_scan_kernel(const int64_t* in, int64_t* out, int n, int64_t* total) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int chunk = (n + blockDim.x - 1) / blockDim.x;
    const int a = t * chunk, b = min(n, a + chunk);
    int64_t s = 0;
    for (int j = a; j < b; ++j) s += in[j];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        int64_t acc = 0;
        for (int j = 0; j < (int)blockDim.x; ++j) {
            const int64_t v = part[j];
            part[j] = acc;
            acc += v;
        }
        *total = acc;
    }
    __syncthreads();
    int64_t acc = part[t];
    for (int j = a; j < b; ++j) {
        out[j] = acc;
        acc += in[j];
    }
}

__global__ void pair_table_kernel(int nrings, int K, const int64_t* pair_off, int64_t npairs,
                                  const int2* ring_range, const double* th, const double* s, const int* npr,
                                  const double* E, float2* pair_A, int2* pair_T) {
    const int64_t pid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pid >= npairs) return;
    // pivot ring: last i with pair_off[i] <= pid
    int lo = 0, hi = nrings - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (pair_off[mid] <= pid) lo = mid; else hi = mid - 1;
    }
    const int i = lo;
    const int r = ring_range[i].x + (int)(pid - pair_off[i]);
    const double A = sin(th[i] - th[r]);
    const float A_hi = (float)A;
    pair_A[pid] = make_float2(A_hi, (float)(A - (double)A_hi));
    const double h = sin(0.5 * (th[r] - th[i]));
    const double f0 = h * h;
    const double sisr = s[i] * s[r];
    const double nr = (double)npr[r];
    for (int e = 0; e <= K; ++e) {
        const double q = (E[e] - f0) / sisr;
        int2 enc;
        if (q <= 0.0) {
            enc = make_int2(T_ZERO, __float_as_int(0.0f));
        } else if (q > 1.0) {
            enc = make_int2(T_INF, __float_as_int(0.0f));
        } else {
            const double T = nr / M_PI * asin(sqrt(q));
            const double Ti = floor(T);
            float tf = (float)(T - Ti);
            int ti = (int)Ti;
            if (tf >= 1.0f) {  // rounding of the fraction up to 1
                tf = 0.0f;
                ti += 1;
            }
            enc = make_int2(ti, __float_as_int(tf));
        }
        pair_T[pid * (K + 1) + e] = enc;
    }
}

__global__ void tile_list_kernel(int nrings, const int64_t* tile_off, const int64_t* ntiles_ring, int2* tiles) {
    const int i = blockIdx.x;
    if (i >= nrings) return;
    const int64_t o = tile_off[i];
    const int64_t nt = ntiles_ring[i];
    for (int64_t t = threadIdx.x; t < nt; t += blockDim.x) tiles[o + t] = make_int2(i, (int)(t * TILE));
}

__global__ void edges_kernel(int K, const double* theta, double* E) {
    const int e = threadIdx.x;
    if (e > K) return;
    const double h = sin(0.5 * theta[e]);
    E[e] = h * h;
}

}  // namespace tpcf
