// Catalogue plans: the device-built sphere grid (plan creation) and the forward
// call sequence.  The estimator itself runs in cat_fwd_kernel (cat_kernels.cuh) and
// in the reduction / normalisation kernels shared with the map path.
//
// Grid: nb colatitude bands of height h = pi / nb; band b is cut into
// ns_b = floor(2 pi sin(theta*) / h) equal longitude sectors, theta* being the
// band's colatitude nearest the equator, so every cell is at most about h wide.
// h is chosen for about 32 points per cell on average.  Points are counted per
// cell, the counts scanned, and the points scattered into cell order together with
// fp32 hi/lo copies of their coordinates and their caller index.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>

#include "geometry.cuh"
#include "plan.cuh"

namespace tpcf {

// per-M catalogue launchers (map_inst.cu)
#define TPCF_DECL_CAT_M(m)                                                                     \
    cudaError_t cat_fwd_launch_m##m(const CatDev&, const MapCall&, int, cudaStream_t);        \
    int cat_fwd_occupancy_m##m(int, int);                                                     \
    cudaError_t cat_bwd_launch_m##m(const CatDev&, const MapCall&, int, cudaStream_t);        \
    int cat_bwd_occupancy_m##m(int);                                                          \
    cudaError_t cat_fwd_multi_launch_m##m(const CatDev&, const MapCall&, const float2*, const float2*, int, \
                                          cudaStream_t);                                      \
    int cat_fwd_multi_occupancy_m##m(int);
TPCF_DECL_CAT_M(0) TPCF_DECL_CAT_M(1) TPCF_DECL_CAT_M(2) TPCF_DECL_CAT_M(3) TPCF_DECL_CAT_M(4)
TPCF_DECL_CAT_M(5) TPCF_DECL_CAT_M(6) TPCF_DECL_CAT_M(7) TPCF_DECL_CAT_M(8) TPCF_DECL_CAT_M(9)
TPCF_DECL_CAT_M(10) TPCF_DECL_CAT_M(11) TPCF_DECL_CAT_M(12) TPCF_DECL_CAT_M(13) TPCF_DECL_CAT_M(14)
TPCF_DECL_CAT_M(15) TPCF_DECL_CAT_M(16)
#undef TPCF_DECL_CAT_M

struct CLaunch {
    cudaError_t (*fwd)(const CatDev&, const MapCall&, int, cudaStream_t);
    int (*occ)(int, int);
    cudaError_t (*bwd)(const CatDev&, const MapCall&, int, cudaStream_t);
    int (*bwd_occ)(int);
    cudaError_t (*multi)(const CatDev&, const MapCall&, const float2*, const float2*, int, cudaStream_t);
    int (*multi_occ)(int);
};
#define TPCF_CROW(m)                                                                                 \
    {cat_fwd_launch_m##m, cat_fwd_occupancy_m##m, cat_bwd_launch_m##m, cat_bwd_occupancy_m##m,     \
     cat_fwd_multi_launch_m##m, cat_fwd_multi_occupancy_m##m}
static const CLaunch kCat[TPCF_MAX_M + 1] = {
    TPCF_CROW(0),  TPCF_CROW(1),  TPCF_CROW(2),  TPCF_CROW(3),  TPCF_CROW(4),  TPCF_CROW(5),
    TPCF_CROW(6),  TPCF_CROW(7),  TPCF_CROW(8),  TPCF_CROW(9),  TPCF_CROW(10), TPCF_CROW(11),
    TPCF_CROW(12), TPCF_CROW(13), TPCF_CROW(14), TPCF_CROW(15), TPCF_CROW(16)};
#undef TPCF_CROW

constexpr int64_t CAT_MAX_SECTORS = 1 << 22;

__global__ void cat_band_kernel(int nb, double hb, int64_t* ns) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const double lo = b * hb, hi = (b + 1) * hb;
    const double smax = (lo <= 0.5 * M_PI && hi >= 0.5 * M_PI) ? 1.0 : fmax(sin(lo), sin(hi));
    int64_t k = (int64_t)floor(2.0 * M_PI * smax / hb);
    ns[b] = k < 1 ? 1 : (k > CAT_MAX_SECTORS ? CAT_MAX_SECTORS : k);
}

__device__ __forceinline__ int64_t cat_cell_of(double x, double y, double z, int nb, double hb,
                                               const int64_t* band_first, const int64_t* band_ns) {
    const double th = atan2(sqrt(x * x + y * y), z);
    double ph = atan2(y, x);
    if (ph < 0.0) ph += 2.0 * M_PI;
    const int b = min(nb - 1, max(0, (int)floor(th / hb)));
    const int64_t ns = band_ns[b];
    int64_t s = (int64_t)floor(ph * (double)ns / (2.0 * M_PI));
    s = s < 0 ? 0 : (s >= ns ? ns - 1 : s);
    return band_first[b] + s;
}

__global__ void cat_cell_count_kernel(int64_t n, const double* __restrict__ xyz, int nb, double hb,
                                 const int64_t* band_first, const int64_t* band_ns, int64_t* cell,
                                 unsigned long long* count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = cat_cell_of(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], nb, hb, band_first, band_ns);
        cell[i] = c;
        atomicAdd(count + c, 1ull);
    }
}

__global__ void cat_scatter_kernel(int64_t n, const double* __restrict__ xyz, const int64_t* __restrict__ cell,
                                   unsigned long long* cursor, float4* p_hi, float4* p_lo, double* xyz_s,
                                   int64_t* orig) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = (int64_t)atomicAdd(cursor + cell[i], 1ull);
        const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        const float hx = (float)x, hy = (float)y, hz = (float)z;
        p_hi[s] = make_float4(hx, hy, hz, 0.0f);
        p_lo[s] = make_float4((float)(x - (double)hx), (float)(y - (double)hy), (float)(z - (double)hz),
                              __int_as_float((int)s));
        xyz_s[3 * s] = x;
        xyz_s[3 * s + 1] = y;
        xyz_s[3 * s + 2] = z;
        orig[s] = i;
    }
}

// Edge tables: chord^2 = 4 sin^2(theta / 2) in fp64 and fp32, the lookup table over
// log2(chord^2) and its origin / scale (lut_par[0], lut_par[1]).
__global__ void cat_edges_kernel(int K, const double* theta, double* Ed2, float* E2, unsigned char* lut,
                                 float* lut_par) {
    __shared__ float e2[TPCF_MAX_BINS + 1];
    for (int e = threadIdx.x; e <= K; e += blockDim.x) {
        const double h = 2.0 * sin(0.5 * theta[e]);
        Ed2[e] = h * h;
        E2[e] = (float)(h * h);
        e2[e] = (float)(h * h);
    }
    __syncthreads();
    const float l0 = log2f(e2[0]);
    const float span = log2f(e2[K]) - l0;
    const float linv = (float)CAT_LUT / fmaxf(span, 1e-6f);
    for (int t = threadIdx.x; t < CAT_LUT; t += blockDim.x) {
        const float c2 = exp2f(l0 + (float)t / linv);
        int k = 0;
        while (k + 1 < K && c2 >= e2[k + 1]) ++k;
        lut[t] = (unsigned char)k;
    }
    if (threadIdx.x == 0) {
        lut_par[0] = l0;
        lut_par[1] = linv;
    }
}

// (w d, w) of each sorted point, gathered from the caller's order.
__global__ void cat_pack_kernel(int64_t n, const int64_t* __restrict__ orig, const float* __restrict__ delta,
                                const float* __restrict__ w, float2* wdw) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = orig[s];
        const float wi = w[o];
        wdw[s] = make_float2(wi * delta[o], wi);
    }
}

// zeta = sums / (scale * norm), 0 where the denominator is 0 (zeta layout).
__global__ void normalize_kernel(const double* __restrict__ sums, const double* __restrict__ norm, double scale,
                                 int K, int M, double* zeta) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (M + 1) * K * K) return;
    const double d = scale * norm[idx % (K * K)];
    zeta[2 * idx] = d != 0.0 ? sums[2 * idx] / d : 0.0;
    zeta[2 * idx + 1] = d != 0.0 ? sums[2 * idx + 1] / d : 0.0;
}

// m-coupling correction, one CTA per bin pair (k1, k2): the (2M+1) x (2M+1) system
//   sum_{m'=-M..M} scale R_{m-m'} z_{m'} = S_m,   m = -M..M,   X_{-n} = conj(X_n),
// solved by Gaussian elimination with partial pivoting in FP64 shared memory; writes
// z_m, m = 0..M.  R_0 = 0 gives zeta = 0; a zero pivot gives NaN.
constexpr int EC_MAX_N = 2 * TPCF_MAX_M + 1;
constexpr int EC_THREADS = 128;

__device__ __forceinline__ double2 c_ext(const double* X, int K, int k1, int k2, int n) {
    const double* e = X + 2 * (((size_t)(n < 0 ? -n : n) * K + k1) * K + k2);
    return n >= 0 ? make_double2(e[0], e[1]) : make_double2(e[0], -e[1]);
}
__device__ __forceinline__ double2 c_mul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 c_div(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

__global__ void __launch_bounds__(EC_THREADS) edge_correct_kernel(const double* __restrict__ S,
                                                                  const double* __restrict__ R, double scale, int K,
                                                                  int M, double* __restrict__ zeta) {
    __shared__ double2 A[EC_MAX_N][EC_MAX_N + 1];  // augmented: column N holds the right-hand side
    __shared__ int s_piv;
    const int k1 = blockIdx.x / K, k2 = blockIdx.x % K;
    const int N = 2 * M + 1;
    double* out = zeta + 2 * ((size_t)k1 * K + k2);
    const size_t mstride = 2 * (size_t)K * K;
    const double2 r0 = c_ext(R, K, k1, k2, 0);
    if (r0.x == 0.0 && r0.y == 0.0) {
        for (int m = threadIdx.x; m <= M; m += EC_THREADS) out[m * mstride] = out[m * mstride + 1] = 0.0;
        return;
    }
    for (int e = threadIdx.x; e < N * (N + 1); e += EC_THREADS) {
        const int r = e / (N + 1), c = e % (N + 1);
        if (c < N) {
            const double2 v = c_ext(R, K, k1, k2, r - c);
            A[r][c] = make_double2(scale * v.x, scale * v.y);
        } else {
            A[r][c] = c_ext(S, K, k1, k2, r - M);
        }
    }
    __syncthreads();
    for (int j = 0; j < N; ++j) {
        if (threadIdx.x == 0) {
            int best = j;
            double bv = A[j][j].x * A[j][j].x + A[j][j].y * A[j][j].y;
            for (int r = j + 1; r < N; ++r) {
                const double v = A[r][j].x * A[r][j].x + A[r][j].y * A[r][j].y;
                if (v > bv) bv = v, best = r;
            }
            s_piv = best;
        }
        __syncthreads();
        const int p = s_piv;
        if (p != j)
            for (int c = j + threadIdx.x; c <= N; c += EC_THREADS) {
                const double2 t = A[j][c];
                A[j][c] = A[p][c];
                A[p][c] = t;
            }
        __syncthreads();
        const double2 piv = A[j][j];
        const int rows = N - j - 1, cols = N - j;  // rows below j, columns j+1..N
        for (int e = threadIdx.x; e < rows * cols; e += EC_THREADS) {
            const int r = j + 1 + e / cols, c = j + 1 + e % cols;
            const double2 f = c_div(A[r][j], piv);
            const double2 t = c_mul(f, A[j][c]);
            A[r][c] = make_double2(A[r][c].x - t.x, A[r][c].y - t.y);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {  // back substitution into column N
        for (int r = N - 1; r >= 0; --r) {
            double2 acc = A[r][N];
            for (int c = r + 1; c < N; ++c) {
                const double2 t = c_mul(A[r][c], A[c][N]);
                acc = make_double2(acc.x - t.x, acc.y - t.y);
            }
            const double2 d = A[r][r];
            A[r][N] = (d.x == 0.0 && d.y == 0.0) ? make_double2(nan(""), nan("")) : c_div(acc, d);
        }
    }
    __syncthreads();
    for (int m = threadIdx.x; m <= M; m += EC_THREADS) {
        out[m * mstride] = A[M + m][N].x;
        out[m * mstride + 1] = A[M + m][N].y;
    }
}

static int nblk(int64_t n, int bs) { return (int)std::min<int64_t>((n + bs - 1) / bs, 1 << 20); }

tpcf_status build_catalog(tpcf_plan_s* P, const double* d_xyz, int64_t n, cudaStream_t s) {
    CatDev& g = P->cat;
    const int K = P->K;
    g.n = n;
    g.K = K;
    g.M = P->M;
    g.theta_max = P->edges[K];
    double h = sqrt(4.0 * M_PI * 32.0 / (double)n);
    h = std::max(std::min(h, g.theta_max), 2e-4);
    const int nb = (int)std::min<double>(ceil(M_PI / h), 1 << 16);
    g.nbands = nb;
    g.hband = M_PI / nb;
    int64_t *band_ns, *band_first, *cell, *cell_start, *orig;
    double *theta, *Ed2, *xyz_s;
    float *E2, *lut_par;
    unsigned char* lut;
    float4 *p_hi, *p_lo;
    TRY_CUDA(P->alloc(&band_ns, nb));
    TRY_CUDA(P->alloc(&band_first, nb + 1));
    TRY_CUDA(P->alloc(&theta, K + 1));
    TRY_CUDA(P->alloc(&Ed2, K + 1));
    TRY_CUDA(P->alloc(&E2, K + 1));
    TRY_CUDA(P->alloc(&lut, CAT_LUT));
    TRY_CUDA(P->alloc(&lut_par, 2));
    TRY_CUDA(cudaMemcpyAsync(theta, P->edges.data(), sizeof(double) * (K + 1), cudaMemcpyHostToDevice, s));
    cat_edges_kernel<<<1, 256, 0, s>>>(K, theta, Ed2, E2, lut, lut_par);
    cat_band_kernel<<<nblk(nb, 256), 256, 0, s>>>(nb, g.hband, band_ns);
    exclusive_scan_kernel<<<1, 1024, 0, s>>>(band_ns, band_first, nb, band_first + nb);
    TRY_CUDA(cudaGetLastError());
    int64_t ncells = 0;
    float lp[2];
    TRY_CUDA(cudaMemcpyAsync(&ncells, band_first + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaMemcpyAsync(lp, lut_par, sizeof(lp), cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    g.lut_l0 = lp[0];
    g.lut_inv = lp[1];

    // count, scan, scatter (the cell index and cursor arrays are temporary)
    TRY_CUDA(P->alloc(&cell_start, ncells + 1));
    TRY_CUDA(P->alloc(&p_hi, n));
    TRY_CUDA(P->alloc(&p_lo, n));
    TRY_CUDA(P->alloc(&xyz_s, 3 * n));
    TRY_CUDA(P->alloc(&orig, n));
    unsigned long long* cursor = nullptr;
    TRY_CUDA(dev_malloc((void**)&cell, sizeof(int64_t) * n));
    cudaError_t e = dev_malloc((void**)&cursor, sizeof(unsigned long long) * (ncells + 1));
    if (e != cudaSuccess) {
        dev_free(cell);
        return cuda_fail(e, "cudaMalloc(cursor)");
    }
    auto cleanup = [&]() {
        cudaStreamSynchronize(s);
        dev_free(cell);
        dev_free(cursor);
    };
    e = cudaMemsetAsync(cursor, 0, sizeof(unsigned long long) * (ncells + 1), s);
    if (e == cudaSuccess) {
        const int grid = P->num_sms * 8;
        cat_cell_count_kernel<<<grid, 256, 0, s>>>(n, d_xyz, nb, g.hband, band_first, band_ns, cell, cursor);
        exclusive_scan_kernel<<<1, 1024, 0, s>>>((const int64_t*)cursor, cell_start, (int)ncells, cell_start + ncells);
        e = cudaMemcpyAsync(cursor, cell_start, sizeof(int64_t) * (ncells + 1), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            cat_scatter_kernel<<<grid, 256, 0, s>>>(n, d_xyz, cell, cursor, p_hi, p_lo, xyz_s, orig);
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "catalogue grid build");
    g.p_hi = p_hi;
    g.p_lo = p_lo;
    g.xyz = xyz_s;
    g.orig = orig;
    g.cell_start = cell_start;
    g.band_first = band_first;
    g.band_ns = band_ns;
    g.E2 = E2;
    g.Ed2 = Ed2;
    g.lut = lut;
    g.ntiles = (n + TILE - 1) / TILE;

    const int self = (P->flags & TPCF_SELF_PAIRS_SUBTRACT) ? 1 : 0;
    const int occ = kCat[P->M].occ(K, self);
    TRY_CUDA(cudaGetLastError());
    if (occ < 1) {
        set_error("catalogue kernel does not fit on an SM");
        return TPCF_ERR_UNSUPPORTED;
    }
    P->fwd_grid = (int)std::max<int64_t>(1, std::min<int64_t>(g.ntiles, (int64_t)P->num_sms * occ));
    const int occ_b = kCat[P->M].bwd_occ(K);
    TRY_CUDA(cudaGetLastError());
    P->bwd_grid = occ_b < 1 ? 0 : (int)std::max<int64_t>(1, std::min<int64_t>(g.ntiles, (int64_t)P->num_sms * occ_b));
    TRY_CUDA(P->alloc(&P->H, (size_t)(P->M + 1) * K * K * 2 + K));
    P->nent = n_entries(K, P->M);
    TRY_CUDA(P->alloc(&P->wdw, n));
    TRY_CUDA(P->alloc(&P->slots, (size_t)P->fwd_grid * P->nent));
    TRY_CUDA(P->alloc(&P->sums, P->nent));
    TRY_CUDA(P->alloc(&P->counter, 4));
    TRY_CUDA(P->alloc(&P->status, 4));
    TRY_CUDA(cudaMemsetAsync(P->status, 0, sizeof(int) * 4, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    return TPCF_OK;
}

cudaError_t cat_count_launch(const CatDev& g, const float2* wdw, long long lo, long long hi, int* counter,
                             unsigned long long* counts, int grid, cudaStream_t s);

tpcf_status catalog_count(tpcf_plan_s* P, const float* d_w, int64_t lo, int64_t hi, int64_t* d_counts,
                          cudaStream_t s) {
    const CatDev& g = P->cat;
    // only the weights matter: pack them with a zero field
    cat_pack_kernel<<<P->num_sms * 8, 256, 0, s>>>(g.n, g.orig, d_w, d_w, P->wdw);
    P->launches += 2;
    TRY_CUDA(cudaMemsetAsync(d_counts, 0, 3 * sizeof(int64_t), s));
    TRY_CUDA(cudaMemsetAsync(P->counter, 0, sizeof(int), s));
    TRY_CUDA(cat_count_launch(g, P->wdw, lo, hi, P->counter, (unsigned long long*)d_counts, P->num_sms * 4, s));
    // every catalogue pair is visited singly: counts[2] = counts[0]
    TRY_CUDA(cudaMemcpyAsync(d_counts + 2, d_counts, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    return TPCF_OK;
}

tpcf_status catalog_backward(tpcf_plan_s* P, const float* d_delta, const float* d_w, int64_t lo, int64_t hi,
                             const double* d_norm, const double* d_dL, float* d_grad, cudaStream_t s) {
    const CatDev& g = P->cat;
    if (P->flags & TPCF_SELF_PAIRS_SUBTRACT) {
        set_error("catalogue adjoint with self-pair subtraction");
        return TPCF_ERR_UNSUPPORTED;
    }
    if (P->bwd_grid < 1) {
        set_error("catalogue adjoint kernel does not fit on an SM");
        return TPCF_ERR_UNSUPPORTED;
    }
    cat_pack_kernel<<<P->num_sms * 8, 256, 0, s>>>(g.n, g.orig, d_delta, d_w, P->wdw);
    const int nout = (P->M + 1) * P->K * P->K;
    adjoint_prep_kernel<<<(nout + 127) / 128, 128, 0, s>>>(d_dL, d_norm, P->K, P->M, P->H, 0);
    zero_f32_kernel<<<P->num_sms * 8, 256, 0, s>>>(d_grad, g.n);
    P->launches += 4;  // pack, prep, zero, adjoint
    TRY_CUDA(cudaMemsetAsync(P->counter, 0, sizeof(int), s));
    MapCall c{};
    c.wdw = P->wdw;
    c.piv_lo = lo;
    c.piv_hi = hi;
    c.counter = P->counter;
    c.status = P->status;
    c.H = P->H;
    c.grad = d_grad;
    TRY_CUDA(kCat[P->M].bwd(g, c, P->bwd_grid, s));
    return TPCF_OK;
}

// Three fields on the catalogue's points (tpcf_forward_multi on catalogue plans).
tpcf_status catalog_forward_multi(tpcf_plan_s* P, const float* const* d_delta, const float* const* d_w, int64_t lo,
                                  int64_t hi, double* d_zeta, double* d_norm, double* d_sums, cudaStream_t s) {
    const CatDev& g = P->cat;
    const int K = P->K, M = P->M;
    const int nent = n_entries_multi(K, M);
    if (!P->wdw_b) {  // the second and third fields' packed values and the slots, on the first call
        const int occ = kCat[M].multi_occ(K);
        if (occ < 1) {
            char msg[160];
            snprintf(msg, sizeof(msg),
                     "tpcf_forward_multi: three fields' moments (K=%d, m_max=%d) do not fit in shared memory", K, M);
            set_error(msg);
            return TPCF_ERR_UNSUPPORTED;
        }
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(g.ntiles, (int64_t)P->num_sms * occ));
        float2 *b, *c;
        double *sl, *su;
        TRY_CUDA(P->alloc(&b, g.n));
        TRY_CUDA(P->alloc(&c, g.n));
        TRY_CUDA(P->alloc(&sl, (size_t)grid * nent));
        TRY_CUDA(P->alloc(&su, (size_t)nent));
        P->wdw_c = c;
        P->mslots = sl;
        P->msums = su;
        P->multi_grid = grid;
        P->wdw_b = b;
    }
    float2* dst[3] = {P->wdw, P->wdw_b, P->wdw_c};
    for (int f = 0; f < 3; ++f)
        cat_pack_kernel<<<P->num_sms * 8, 256, 0, s>>>(g.n, g.orig, d_delta[f], d_w[f], dst[f]);
    TRY_CUDA(cudaMemsetAsync(P->mslots, 0, sizeof(double) * (size_t)P->multi_grid * nent, s));
    TRY_CUDA(cudaMemsetAsync(P->counter, 0, sizeof(int), s));
    MapCall c{};
    c.wdw = P->wdw;
    c.piv_lo = lo;
    c.piv_hi = hi;
    c.slots = P->mslots;
    c.counter = P->counter;
    c.status = P->status;
    TRY_CUDA(kCat[M].multi(g, c, P->wdw_b, P->wdw_c, P->multi_grid, s));
    reduce_slots_kernel<<<(nent + 127) / 128, 128, 0, s>>>(P->mslots, P->multi_grid, nent, P->msums);
    const int nout = (M + 1) * K * K;
    finalize_full_kernel<<<(nout + 127) / 128, 128, 0, s>>>(P->msums, K, M, d_zeta, d_norm, d_sums);
    P->launches += 6;  // three packs, the pair kernel, reduce, finalize
    TRY_CUDA(cudaGetLastError());
    return TPCF_OK;
}

tpcf_status catalog_forward(tpcf_plan_s* P, const float* d_delta, const float* d_w, int64_t lo, int64_t hi,
                            double* d_zeta, double* d_norm, double* d_sums, cudaStream_t s) {
    const CatDev& g = P->cat;
    cat_pack_kernel<<<P->num_sms * 8, 256, 0, s>>>(g.n, g.orig, d_delta, d_w, P->wdw);
    P->launches += 4;  // pack, forward, reduce, finalize
    TRY_CUDA(cudaMemsetAsync(P->slots, 0, sizeof(double) * (size_t)P->fwd_grid * P->nent, s));
    TRY_CUDA(cudaMemsetAsync(P->counter, 0, sizeof(int), s));
    MapCall c{};
    c.wdw = P->wdw;
    c.piv_lo = lo;
    c.piv_hi = hi;
    c.slots = P->slots;
    c.counter = P->counter;
    c.status = P->status;
    c.self_subtract = (P->flags & TPCF_SELF_PAIRS_SUBTRACT) ? 1 : 0;
    c.norm = norm_of_flags(P->flags);
    TRY_CUDA(kCat[P->M].fwd(g, c, P->fwd_grid, s));
    reduce_slots_kernel<<<(P->nent + 127) / 128, 128, 0, s>>>(P->slots, P->fwd_grid, P->nent, P->sums);
    const int nout = (P->M + 1) * P->K * P->K;
    finalize_kernel<<<(nout + 127) / 128, 128, 0, s>>>(P->sums, P->K, P->M, c.self_subtract, 1.0, d_zeta, d_norm,
                                                       d_sums);
    TRY_CUDA(cudaGetLastError());
    return TPCF_OK;
}

}  // namespace tpcf

extern "C" tpcf_status tpcf_edge_correct(const double* d_sums, const double* d_rsums, double scale, int32_t nbins,
                                         int32_t m_max, double* d_zeta, void* stream) {
    if (!d_sums || !d_rsums || !d_zeta) return TPCF_ERR_INVALID_ARG;
    if (nbins < 1 || nbins > TPCF_MAX_BINS || m_max < 0 || m_max > TPCF_MAX_M) return TPCF_ERR_INVALID_ARG;
    if (!(scale > 0.0) || !isfinite(scale)) return TPCF_ERR_INVALID_ARG;
    tpcf::edge_correct_kernel<<<nbins * nbins, tpcf::EC_THREADS, 0, (cudaStream_t)stream>>>(d_sums, d_rsums, scale,
                                                                                            nbins, m_max, d_zeta);
    TRY_CUDA(cudaGetLastError());
    return TPCF_OK;
}

extern "C" tpcf_status tpcf_normalize(const double* d_sums, const double* d_norm, double scale, int32_t nbins,
                                      int32_t m_max, double* d_zeta, void* stream) {
    if (!d_sums || !d_norm || !d_zeta) return TPCF_ERR_INVALID_ARG;
    if (nbins < 1 || nbins > TPCF_MAX_BINS || m_max < 0 || m_max > TPCF_MAX_M) return TPCF_ERR_INVALID_ARG;
    if (!(scale > 0.0) || !isfinite(scale)) return TPCF_ERR_INVALID_ARG;
    const int nout = (m_max + 1) * nbins * nbins;
    tpcf::normalize_kernel<<<(nout + 127) / 128, 128, 0, (cudaStream_t)stream>>>(d_sums, d_norm, scale, nbins, m_max,
                                                                                  d_zeta);
    TRY_CUDA(cudaGetLastError());
    return TPCF_OK;
}
