// Host side of the C ABI declared in include/tpcf.h: plan objects, validation,
// launch sequencing and error reporting.  Every numerical step runs in the
// kernels of geometry.cu, small_kernels.cu and map_kernels.cuh.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>
#include <vector>

#include "geometry.cuh"
#include "plan.cuh"

using namespace tpcf;

namespace tpcf {
// per-M launchers (map_inst.cu)
#define TPCF_DECL_MULTI(m)                                                                                    \
    cudaError_t map_fwd_multi_launch_m##m(const MapDev&, const MapCall&, const float2*, const float2*, int, \
                                          cudaStream_t);                                                  \
    int map_fwd_multi_occupancy_m##m(int);
TPCF_DECL_MULTI(0) TPCF_DECL_MULTI(1) TPCF_DECL_MULTI(2) TPCF_DECL_MULTI(3) TPCF_DECL_MULTI(4) TPCF_DECL_MULTI(5)
TPCF_DECL_MULTI(6) TPCF_DECL_MULTI(7) TPCF_DECL_MULTI(8) TPCF_DECL_MULTI(9) TPCF_DECL_MULTI(10)
TPCF_DECL_MULTI(11) TPCF_DECL_MULTI(12) TPCF_DECL_MULTI(13) TPCF_DECL_MULTI(14) TPCF_DECL_MULTI(15)
TPCF_DECL_MULTI(16)
#undef TPCF_DECL_MULTI
typedef cudaError_t (*multi_fn)(const MapDev&, const MapCall&, const float2*, const float2*, int, cudaStream_t);
static const multi_fn kMulti[TPCF_MAX_M + 1] = {
    map_fwd_multi_launch_m0,  map_fwd_multi_launch_m1,  map_fwd_multi_launch_m2,  map_fwd_multi_launch_m3,
    map_fwd_multi_launch_m4,  map_fwd_multi_launch_m5,  map_fwd_multi_launch_m6,  map_fwd_multi_launch_m7,
    map_fwd_multi_launch_m8,  map_fwd_multi_launch_m9,  map_fwd_multi_launch_m10, map_fwd_multi_launch_m11,
    map_fwd_multi_launch_m12, map_fwd_multi_launch_m13, map_fwd_multi_launch_m14, map_fwd_multi_launch_m15,
    map_fwd_multi_launch_m16};
static int (*const kMultiOcc[TPCF_MAX_M + 1])(int) = {
    map_fwd_multi_occupancy_m0,  map_fwd_multi_occupancy_m1,  map_fwd_multi_occupancy_m2,
    map_fwd_multi_occupancy_m3,  map_fwd_multi_occupancy_m4,  map_fwd_multi_occupancy_m5,
    map_fwd_multi_occupancy_m6,  map_fwd_multi_occupancy_m7,  map_fwd_multi_occupancy_m8,
    map_fwd_multi_occupancy_m9,  map_fwd_multi_occupancy_m10, map_fwd_multi_occupancy_m11,
    map_fwd_multi_occupancy_m12, map_fwd_multi_occupancy_m13, map_fwd_multi_occupancy_m14,
    map_fwd_multi_occupancy_m15, map_fwd_multi_occupancy_m16};
#define TPCF_DECL_M(m)                                                                         \
    cudaError_t map_fwd_launch_m##m(const MapDev&, const MapCall&, int, int, cudaStream_t);    \
    cudaError_t map_fwd_tc_launch_m##m(const MapDev&, const MapCall&, int, cudaStream_t);      \
    int map_fwd_tc_occupancy_m##m(int, int);                                                  \
    cudaError_t map_bwd_launch_m##m(const MapDev&, const MapCall&, int, int, cudaStream_t);    \
    int map_fwd_occupancy_m##m(int, int, int);                                                \
    int map_bwd_occupancy_m##m(int, int);                                                     \
    size_t map_fwd_smem_m##m(int);                                                            \
    size_t map_bwd_smem_m##m(int);
TPCF_DECL_M(0) TPCF_DECL_M(1) TPCF_DECL_M(2) TPCF_DECL_M(3) TPCF_DECL_M(4) TPCF_DECL_M(5)
TPCF_DECL_M(6) TPCF_DECL_M(7) TPCF_DECL_M(8) TPCF_DECL_M(9) TPCF_DECL_M(10) TPCF_DECL_M(11)
TPCF_DECL_M(12) TPCF_DECL_M(13) TPCF_DECL_M(14) TPCF_DECL_M(15) TPCF_DECL_M(16)
#undef TPCF_DECL_M
cudaError_t map_count_launch(const MapDev& g, const float2* wdw, long long lo, long long hi, long long tlo,
                             long long thi, unsigned long long* counts, int grid, cudaStream_t s);
// catalogue plans (catalog.cu)
tpcf_status build_catalog(tpcf_plan_s* P, const double* d_xyz, int64_t n, cudaStream_t s);
tpcf_status catalog_count(tpcf_plan_s* P, const float* d_w, int64_t lo, int64_t hi, int64_t* d_counts,
                          cudaStream_t s);
tpcf_status catalog_backward(tpcf_plan_s* P, const float* d_delta, const float* d_w, int64_t lo, int64_t hi,
                             const double* d_norm, const double* d_dL, float* d_grad, cudaStream_t s);
tpcf_status catalog_forward(tpcf_plan_s* P, const float* d_delta, const float* d_w, int64_t lo, int64_t hi,
                            double* d_zeta, double* d_norm, double* d_sums, cudaStream_t s);
tpcf_status catalog_forward_multi(tpcf_plan_s* P, const float* const* d_delta, const float* const* d_w, int64_t lo,
                                  int64_t hi, double* d_zeta, double* d_norm, double* d_sums, cudaStream_t s);
// loads the allocation-free forward's scratch array on a device (noalloc.cu)
tpcf_status noalloc_prepare(int dev);

struct MLaunch {
    cudaError_t (*fwd)(const MapDev&, const MapCall&, int, int, cudaStream_t);
    cudaError_t (*fwd_tc)(const MapDev&, const MapCall&, int, cudaStream_t);
    int (*fwd_tc_occ)(int, int);
    cudaError_t (*bwd)(const MapDev&, const MapCall&, int, int, cudaStream_t);
    int (*fwd_occ)(int, int, int);
    int (*bwd_occ)(int, int);
    size_t (*fwd_smem)(int);
    size_t (*bwd_smem)(int);
};
#define TPCF_ROW_M(m) \
    {map_fwd_launch_m##m, map_fwd_tc_launch_m##m, map_fwd_tc_occupancy_m##m, map_bwd_launch_m##m, map_fwd_occupancy_m##m, map_bwd_occupancy_m##m, map_fwd_smem_m##m, map_bwd_smem_m##m}
static const MLaunch kLaunch[TPCF_MAX_M + 1] = {
    TPCF_ROW_M(0),  TPCF_ROW_M(1),  TPCF_ROW_M(2),  TPCF_ROW_M(3),  TPCF_ROW_M(4),  TPCF_ROW_M(5),
    TPCF_ROW_M(6),  TPCF_ROW_M(7),  TPCF_ROW_M(8),  TPCF_ROW_M(9),  TPCF_ROW_M(10), TPCF_ROW_M(11),
    TPCF_ROW_M(12), TPCF_ROW_M(13), TPCF_ROW_M(14), TPCF_ROW_M(15), TPCF_ROW_M(16)};
#undef TPCF_ROW_M

// resident CTAs per SM of each register variant (used by the autotuner, tune.cu)
int map_fwd_occupancy(int M, int K, int self, int variant) { return kLaunch[M].fwd_occ(K, self, variant); }
int map_bwd_occupancy(int M, int K, int variant) { return kLaunch[M].bwd_occ(K, variant); }
// applies a configuration cached by the autotuner (tune.cu)
void tune_from_cache(tpcf_plan_s* P);
}  // namespace tpcf

static thread_local char g_last_error[256] = "";

// Allocation bookkeeping: live device allocations, and the test hook that makes the
// n-th next allocation fail as if the device were out of memory.
static std::atomic<long long> g_live_allocs{0};
static std::atomic<long long> g_fail_countdown{0};

namespace tpcf {
cudaError_t dev_malloc(void** p, size_t bytes) {
    long long c = g_fail_countdown.load();
    while (c > 0) {
        if (g_fail_countdown.compare_exchange_weak(c, c - 1)) {
            if (c == 1) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) ++g_live_allocs;
    return e;
}
void dev_free(void* p) {
    if (!p) return;
    cudaFree(p);
    --g_live_allocs;
}
}  // namespace tpcf

extern "C" void tpcf_test_fail_allocation(int64_t n) { g_fail_countdown.store(n > 0 ? n : 0); }

extern "C" int64_t tpcf_test_live_allocations(void) { return g_live_allocs.load(); }

namespace tpcf {
tpcf_status cuda_fail(cudaError_t e, const char* where) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? TPCF_ERR_OOM : TPCF_ERR_CUDA;
}
void set_error(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }
}  // namespace tpcf

extern "C" const char* tpcf_status_string(tpcf_status s) {
    switch (s) {
        case TPCF_OK: return "TPCF_OK";
        case TPCF_ERR_INVALID_ARG: return "TPCF_ERR_INVALID_ARG";
        case TPCF_ERR_CUDA: return "TPCF_ERR_CUDA";
        case TPCF_ERR_OOM: return "TPCF_ERR_OOM";
        case TPCF_ERR_TIMEOUT: return "TPCF_ERR_TIMEOUT";
        case TPCF_ERR_UNSUPPORTED: return "TPCF_ERR_UNSUPPORTED";
        case TPCF_ERR_DEVICE: return "TPCF_ERR_DEVICE";
    }
    return "TPCF_ERR_UNKNOWN";
}

extern "C" const char* tpcf_last_error(void) { return g_last_error; }

static tpcf_status check_bins(const tpcf_bins* b) {
    if (!b || !b->theta_edges_rad) return TPCF_ERR_INVALID_ARG;
    if (b->nbins < 1 || b->nbins > TPCF_MAX_BINS) return TPCF_ERR_INVALID_ARG;
    if (b->m_max < 0 || b->m_max > TPCF_MAX_M) return TPCF_ERR_INVALID_ARG;
    if (b->flags & ~(uint32_t)(TPCF_SELF_PAIRS_SUBTRACT | TPCF_CONTRACT_TC | NORM_FLAGS)) return TPCF_ERR_INVALID_ARG;
    if ((b->flags & NORM_FLAGS) == NORM_FLAGS) return TPCF_ERR_INVALID_ARG;
    const double* t = b->theta_edges_rad;
    if (!(t[0] > 0.0)) return TPCF_ERR_INVALID_ARG;
    for (int e = 0; e < b->nbins; ++e)
        if (!(t[e + 1] > t[e])) return TPCF_ERR_INVALID_ARG;
    if (!(t[b->nbins] < 0.5 * M_PI)) return TPCF_ERR_INVALID_ARG;
    return TPCF_OK;
}

// Flag combinations the kernels do not implement: a per-pivot normalisation with
// self-pair subtraction or the tensor-core contraction.
static tpcf_status check_norm(const tpcf_bins* b) {
    if ((b->flags & NORM_FLAGS) && (b->flags & (TPCF_SELF_PAIRS_SUBTRACT | TPCF_CONTRACT_TC))) {
        set_error("per-pivot normalisation with self-pair subtraction or the TC contraction");
        return TPCF_ERR_UNSUPPORTED;
    }
    return TPCF_OK;
}

static int n_blocks(int64_t n, int bs) { return (int)((n + bs - 1) / bs); }

static tpcf_status build_map(tpcf_plan_s* P, int64_t nside, cudaStream_t s) {
    MapDev& g = P->map;
    const int nrings = (int)(4 * nside - 1);
    const int K = P->K;
    g.nside = (int)nside;
    g.nrings = nrings;
    g.K = K;
    g.M = P->M;
    g.npix = 12 * nside * nside;
    int64_t *first, *pair_off, *tile_off, *npairs_r, *ntiles_r, *tot;
    int *npr, *shift;
    double *z, *sd, *th, *E, *theta;
    float *zf, *sf, *sf_lo, *rstep, *rstep_lo, *rinvn, *rinvn_lo;
    int2 *ring_range, *bin_range;
    TRY_CUDA(P->alloc(&first, nrings));
    TRY_CUDA(P->alloc(&npr, nrings));
    TRY_CUDA(P->alloc(&shift, nrings));
    TRY_CUDA(P->alloc(&z, nrings));
    TRY_CUDA(P->alloc(&sd, nrings));
    TRY_CUDA(P->alloc(&th, nrings));
    TRY_CUDA(P->alloc(&zf, nrings));
    TRY_CUDA(P->alloc(&sf, nrings));
    TRY_CUDA(P->alloc(&rstep, nrings));
    TRY_CUDA(P->alloc(&rinvn, nrings));
    TRY_CUDA(P->alloc(&sf_lo, nrings));
    TRY_CUDA(P->alloc(&rstep_lo, nrings));
    TRY_CUDA(P->alloc(&rinvn_lo, nrings));
    TRY_CUDA(P->alloc(&ring_range, nrings));
    TRY_CUDA(P->alloc(&bin_range, (size_t)nrings * K));
    TRY_CUDA(P->alloc(&pair_off, nrings));
    TRY_CUDA(P->alloc(&tile_off, nrings));
    TRY_CUDA(P->alloc(&npairs_r, nrings));
    TRY_CUDA(P->alloc(&ntiles_r, nrings));
    TRY_CUDA(P->alloc(&tot, 2));
    TRY_CUDA(P->alloc(&E, K + 1));
    TRY_CUDA(P->alloc(&theta, K + 1));
    TRY_CUDA(cudaMemcpyAsync(theta, P->edges.data(), sizeof(double) * (K + 1), cudaMemcpyHostToDevice, s));
    edges_kernel<<<1, 64, 0, s>>>(K, theta, E);
    ring_table_kernel<<<n_blocks(nrings, 128), 128, 0, s>>>((int)nside, nrings, first, npr, shift, z, sd, th,
                                                            zf, sf, sf_lo, rstep, rstep_lo, rinvn, rinvn_lo);
    ring_range_kernel<<<n_blocks(nrings, 128), 128, 0, s>>>(nrings, K, th, E, npr, ring_range, bin_range,
                                                            npairs_r, ntiles_r);
    exclusive_scan_kernel<<<1, 1024, 0, s>>>(npairs_r, pair_off, nrings, tot);
    exclusive_scan_kernel<<<1, 1024, 0, s>>>(ntiles_r, tile_off, nrings, tot + 1);
    TRY_CUDA(cudaGetLastError());
    int64_t totals[2];
    TRY_CUDA(cudaMemcpyAsync(totals, tot, sizeof(totals), cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    const int64_t npairs = totals[0], ntiles = totals[1];
    P->tile_off_h.resize(nrings);
    TRY_CUDA(cudaMemcpy(P->tile_off_h.data(), tile_off, sizeof(int64_t) * nrings, cudaMemcpyDeviceToHost));
    float2* pair_A;
    int2 *pair_T, *tiles;
    TRY_CUDA(P->alloc(&pair_A, npairs));
    TRY_CUDA(P->alloc(&pair_T, (size_t)npairs * (K + 1)));
    TRY_CUDA(P->alloc(&tiles, ntiles));
    pair_table_kernel<<<n_blocks(npairs, 128), 128, 0, s>>>(nrings, K, pair_off, npairs, ring_range, th, sd,
                                                            npr, E, pair_A, pair_T);
    tile_list_kernel<<<nrings, 128, 0, s>>>(nrings, tile_off, ntiles_r, tiles);
    TRY_CUDA(cudaGetLastError());
    g.ring_first = first;
    g.ring_n = npr;
    g.ring_shift = shift;
    g.ring_zf = zf;
    g.ring_sf = sf;
    g.ring_sf_lo = sf_lo;
    g.ring_step_lo = rstep_lo;
    g.ring_invn_lo = rinvn_lo;
    g.ring_step = rstep;
    g.ring_invn = rinvn;
    g.ring_th = th;
    g.ring_s = sd;
    g.ring_range = ring_range;
    g.bin_range = bin_range;
    g.pair_off = pair_off;
    g.pair_A = pair_A;
    g.pair_T = pair_T;
    g.tiles = tiles;
    g.ntiles = ntiles;
    g.E = E;
    // per-call scratch, sized once so calls allocate nothing
    const MLaunch& L = kLaunch[P->M];
    const int self = (P->flags & TPCF_SELF_PAIRS_SUBTRACT) ? 1 : 0;
    const bool tc = (P->flags & TPCF_CONTRACT_TC) != 0;
    int occ_f = tc ? L.fwd_tc_occ(K, self) : std::max(L.fwd_occ(K, self, 3), L.fwd_occ(K, self, 2));
    int occ_b = std::max(L.bwd_occ(K, 3), L.bwd_occ(K, 2));
    if (occ_f < 1 || occ_b < 1) {
        snprintf(g_last_error, sizeof(g_last_error), "kernel does not fit (K=%d, M=%d)", K, P->M);
        return TPCF_ERR_UNSUPPORTED;
    }
    // slots for the largest grid any configuration launches
    P->fwd_grid = (int)std::min<int64_t>(ntiles, (int64_t)P->num_sms * occ_f);
    P->bwd_grid = (int)std::min<int64_t>(ntiles, (int64_t)P->num_sms * occ_b);
    P->tune_fwd.ctas = tc ? occ_f : L.fwd_occ(K, self, 3);
    P->tune_bwd.ctas = L.bwd_occ(K, 3);
    if (P->tune_fwd.ctas < 1) P->tune_fwd.variant = 2, P->tune_fwd.ctas = L.fwd_occ(K, self, 2);
    if (P->tune_bwd.ctas < 1) P->tune_bwd.variant = 2, P->tune_bwd.ctas = L.bwd_occ(K, 2);
    if (P->fwd_grid < 1) P->fwd_grid = 1;
    if (P->bwd_grid < 1) P->bwd_grid = 1;
    P->nent = n_entries(K, P->M);
    TRY_CUDA(P->alloc(&P->wdw, g.npix));
    TRY_CUDA(P->alloc(&P->slots, (size_t)P->fwd_grid * P->nent));
    TRY_CUDA(P->alloc(&P->sums, P->nent));
    TRY_CUDA(P->alloc(&P->counter, 4));
    TRY_CUDA(P->alloc(&P->status, 4));
    TRY_CUDA(P->alloc(&P->H, (size_t)(P->M + 1) * K * K * 2 + K));  // H, then cdiag (self-pair mode)
    TRY_CUDA(cudaMemsetAsync(P->status, 0, sizeof(int) * 4, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    return TPCF_OK;
}

extern "C" tpcf_status tpcf_plan_create_map(tpcf_plan* out, int64_t nside, const tpcf_bins* bins, void* stream) {
    if (!out) return TPCF_ERR_INVALID_ARG;
    *out = nullptr;
    if (nside < 1 || nside > 8192) return TPCF_ERR_INVALID_ARG;
    tpcf_status st = check_bins(bins);
    if (st == TPCF_OK) st = check_norm(bins);
    if (st != TPCF_OK) return st;
    tpcf_plan_s* P = new (std::nothrow) tpcf_plan_s();
    if (!P) return TPCF_ERR_OOM;
    P->kind = PLAN_MAP;
    P->K = bins->nbins;
    P->M = bins->m_max;
    P->flags = bins->flags;
    P->edges.assign(bins->theta_edges_rad, bins->theta_edges_rad + bins->nbins + 1);
    P->npoints = 12 * nside * nside;
    cudaError_t e = cudaGetDevice(&P->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);
    if (e != cudaSuccess) {
        delete P;
        return cuda_fail(e, "device query");
    }
    cudaStream_t s = (cudaStream_t)stream;
    st = build_map(P, nside, s);
    if (st != TPCF_OK) {
        cudaStreamSynchronize(s);
        delete P;
        return st;
    }
    tune_from_cache(P);
    // place tpcf_forward_noalloc's fixed scratch on this device now, during set-up;
    // on failure that call reports it, so clear the runtime's last-error state here
    if (noalloc_prepare(P->device) != TPCF_OK) cudaGetLastError();
    P->last_stream = s;
    *out = P;
    return TPCF_OK;
}

extern "C" tpcf_status tpcf_plan_create_catalog(tpcf_plan* out, const double* d_xyz, int64_t n,
                                                const tpcf_bins* bins, void* stream) {
    if (!out) return TPCF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!d_xyz || n < 1 || n > 0x7fffffffLL) return TPCF_ERR_INVALID_ARG;
    tpcf_status st = check_bins(bins);
    if (st == TPCF_OK && (bins->flags & TPCF_CONTRACT_TC)) {
        set_error("catalogue plans use the FP32 contraction");
        return TPCF_ERR_UNSUPPORTED;
    }
    if (st == TPCF_OK) st = check_norm(bins);
    if (st != TPCF_OK) return st;
    tpcf_plan_s* P = new (std::nothrow) tpcf_plan_s();
    if (!P) return TPCF_ERR_OOM;
    P->kind = PLAN_CATALOG;
    P->K = bins->nbins;
    P->M = bins->m_max;
    P->flags = bins->flags;
    P->edges.assign(bins->theta_edges_rad, bins->theta_edges_rad + bins->nbins + 1);
    P->npoints = n;
    cudaError_t e = cudaGetDevice(&P->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);
    if (e != cudaSuccess) {
        delete P;
        return cuda_fail(e, "device query");
    }
    cudaStream_t s = (cudaStream_t)stream;
    st = build_catalog(P, d_xyz, n, s);
    if (st != TPCF_OK) {
        cudaStreamSynchronize(s);
        delete P;
        return st;
    }
    P->last_stream = s;
    *out = P;
    return TPCF_OK;
}

extern "C" int64_t tpcf_plan_npoints(tpcf_plan plan) { return plan ? plan->npoints : -1; }

extern "C" int64_t tpcf_plan_kernel_launches(tpcf_plan plan) { return plan ? plan->launches : -1; }

// 0-based ring of RING-order pixel p (HEALPix, Gorski et al. 2005).
static int64_t ring_of_pixel(int64_t nside, int64_t p) {
    const int64_t ncap = 2 * nside * (nside - 1), npix = 12 * nside * nside;
    auto cap_ring = [](int64_t q) {  // 1-based ring r of the north cap holding q: 2r(r-1) <= q
        int64_t r = (int64_t)((1.0 + sqrt(1.0 + 2.0 * (double)q)) * 0.5);
        while (2 * r * (r - 1) > q) --r;
        while (2 * (r + 1) * r <= q) ++r;
        return r;
    };
    if (p < ncap) return cap_ring(p) - 1;
    if (p < npix - ncap) return (p - ncap) / (4 * nside) + nside - 1;
    return 4 * nside - 1 - cap_ring(npix - 1 - p);
}

static int64_t ring_first_pixel(int64_t nside, int64_t ri) {  // 0-based ring
    const int64_t r = ri + 1;
    if (r < nside) return 2 * r * (r - 1);
    if (r <= 3 * nside) return 2 * nside * (nside - 1) + 4 * nside * (r - nside);
    const int64_t rr = 4 * nside - r;
    return 12 * nside * nside - 2 * rr * (rr + 1);
}

// Tiles [*tlo, *thi) that hold the pivots [lo, hi) (tiles are 32 consecutive pixels
// of one ring, rings in order).
// Tiles [tlo, thi) that can hold a pivot of [lo, hi).  Linear layout: the tiles of the
// range's pixels.  Quadrant layout (the forward kernels): a partial ring's pivots are
// spread over all of its tiles, so whole rings at the two ends.
static void tile_range(const tpcf_plan_s* P, int64_t lo, int64_t hi, int64_t* tlo, int64_t* thi, bool quad) {
    if (hi <= lo) {
        *tlo = *thi = 0;
        return;
    }
    const int64_t nside = P->map.nside;
    const int64_t ra = ring_of_pixel(nside, lo), rb = ring_of_pixel(nside, hi - 1);
    if (quad) {
        *tlo = P->tile_off_h[ra];
        *thi = rb + 1 < (int64_t)P->tile_off_h.size() ? P->tile_off_h[rb + 1] : P->map.ntiles;
        return;
    }
    *tlo = P->tile_off_h[ra] + (lo - ring_first_pixel(nside, ra)) / TILE;
    *thi = P->tile_off_h[rb] + (hi - 1 - ring_first_pixel(nside, rb)) / TILE + 1;
}

static int launch_grid(const tpcf_plan_s* P, const tpcf_plan_s::Tune& t, int64_t ntiles, int cap) {
    const int64_t g = std::min<int64_t>(ntiles, (int64_t)P->num_sms * t.ctas);
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

// group > 1: shared neighbour lists over P->gtiles (tpcf_forward_grouped).
static tpcf_status map_forward(tpcf_plan_s* P, const float* d_delta, const float* d_w, int64_t lo, int64_t hi,
                               double* d_zeta, double* d_norm, double* d_sums, cudaStream_t s, int group = 1) {
    const MapDev& g = P->map;
    pack_kernel<<<P->num_sms * 8, 256, 0, s>>>(d_delta, d_w, P->wdw, g.npix);
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
    c.flush = P->tune_fwd.flush;
    if (group > 1) {  // every run tile; those without a pivot in range return at once
        c.group = group;
        c.gtiles = P->gtiles;
        c.tile_lo = 0;
        c.tile_hi = P->ngtiles;
    } else {
        c.quad = P->tune_fwd.quad;
        tile_range(P, lo, hi, &c.tile_lo, &c.tile_hi, c.quad != 0);
    }
    const int grid = launch_grid(P, P->tune_fwd, c.tile_hi - c.tile_lo, P->fwd_grid);
    if (P->flags & TPCF_CONTRACT_TC)
        TRY_CUDA(kLaunch[P->M].fwd_tc(g, c, grid, s));
    else
        TRY_CUDA(kLaunch[P->M].fwd(g, c, grid, P->tune_fwd.variant, s));
    reduce_slots_kernel<<<n_blocks(P->nent, 128), 128, 0, s>>>(P->slots, P->fwd_grid, P->nent, P->sums);
    const int nout = (P->M + 1) * P->K * P->K;
    finalize_kernel<<<n_blocks(nout, 128), 128, 0, s>>>(P->sums, P->K, P->M, c.self_subtract, 1.0, d_zeta,
                                                        d_norm, d_sums);
    TRY_CUDA(cudaGetLastError());
    return TPCF_OK;
}

extern "C" tpcf_status tpcf_forward_grouped(tpcf_plan plan, const float* d_delta, const float* d_w, int32_t group,
                                            int64_t pivot_begin, int64_t pivot_end, double* d_zeta, double* d_norm,
                                            double* d_sums, void* stream) {
    if (!plan || !d_delta || !d_w || !d_zeta || !d_norm) return TPCF_ERR_INVALID_ARG;
    if (pivot_begin < 0 || pivot_end < pivot_begin || pivot_end > plan->npoints) return TPCF_ERR_INVALID_ARG;
    if (group < 1 || group > 4096) return TPCF_ERR_INVALID_ARG;
    if (plan->kind != PLAN_MAP || (plan->flags & (TPCF_CONTRACT_TC | TPCF_SELF_PAIRS_SUBTRACT | NORM_FLAGS))) {
        set_error("tpcf_forward_grouped: map plans with the default flags only");
        return TPCF_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    plan->last_stream = s;
    if (group == 1) return map_forward(plan, d_delta, d_w, pivot_begin, pivot_end, d_zeta, d_norm, d_sums, s);
    tpcf_plan_s* P = plan;
    if (P->ggroup != group) {  // the tile list of this run length: ceil(ceil(n_i / group) / 32) per ring
        const int64_t nside = P->map.nside;
        std::vector<int2> t;
        for (int r = 0; r < P->map.nrings; ++r) {
            const int64_t ri = r + 1;
            const int64_t n = ri < nside ? 4 * ri : (ri <= 3 * nside ? 4 * nside : 4 * (4 * nside - ri));
            const int64_t ng = (n + group - 1) / group;
            for (int64_t f = 0; f < ng; f += TILE) t.push_back(make_int2(r, (int)f));
        }
        if ((int64_t)t.size() > P->gtiles_cap) {
            int2* buf = nullptr;
            TRY_CUDA(P->alloc(&buf, t.size()));
            P->gtiles = buf;
            P->gtiles_cap = (int64_t)t.size();
        }
        TRY_CUDA(cudaMemcpyAsync(P->gtiles, t.data(), sizeof(int2) * t.size(), cudaMemcpyHostToDevice, s));
        TRY_CUDA(cudaStreamSynchronize(s));
        P->ngtiles = (int64_t)t.size();
        P->ggroup = group;
    }
    return map_forward(P, d_delta, d_w, pivot_begin, pivot_end, d_zeta, d_norm, d_sums, s, group);
}

extern "C" tpcf_status tpcf_forward(tpcf_plan plan, const float* d_delta, const float* d_w, int64_t pivot_begin,
                                    int64_t pivot_end, double* d_zeta, double* d_norm, double* d_sums,
                                    void* stream) {
    if (!plan || !d_delta || !d_w || !d_zeta || !d_norm) return TPCF_ERR_INVALID_ARG;
    if (pivot_begin < 0 || pivot_end < pivot_begin || pivot_end > plan->npoints) return TPCF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    plan->last_stream = s;
    if (plan->kind == PLAN_MAP) return map_forward(plan, d_delta, d_w, pivot_begin, pivot_end, d_zeta, d_norm,
                                                   d_sums, s);
    if (plan->kind == PLAN_CATALOG)
        return catalog_forward(plan, d_delta, d_w, pivot_begin, pivot_end, d_zeta, d_norm, d_sums, s);
    return TPCF_ERR_UNSUPPORTED;
}

extern "C" tpcf_status tpcf_forward_multi(tpcf_plan plan, const float* d_delta_a, const float* d_w_a,
                                          const float* d_delta_b, const float* d_w_b, const float* d_delta_c,
                                          const float* d_w_c, int64_t pivot_begin, int64_t pivot_end, double* d_zeta,
                                          double* d_norm, double* d_sums, void* stream) {
    if (!plan || !d_delta_a || !d_w_a || !d_delta_b || !d_w_b || !d_delta_c || !d_w_c || !d_zeta || !d_norm)
        return TPCF_ERR_INVALID_ARG;
    if (pivot_begin < 0 || pivot_end < pivot_begin || pivot_end > plan->npoints) return TPCF_ERR_INVALID_ARG;
    tpcf_plan_s* P = plan;
    if (P->flags & (TPCF_CONTRACT_TC | TPCF_SELF_PAIRS_SUBTRACT | NORM_FLAGS)) {
        set_error("tpcf_forward_multi: plans with the FP32 contraction, self pairs kept, default normalisation");
        return TPCF_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    P->last_stream = s;
    if (P->kind == PLAN_CATALOG) {
        const float* dd[3] = {d_delta_a, d_delta_b, d_delta_c};
        const float* ww[3] = {d_w_a, d_w_b, d_w_c};
        return catalog_forward_multi(P, dd, ww, pivot_begin, pivot_end, d_zeta, d_norm, d_sums, s);
    }
    if (P->kind != PLAN_MAP) return TPCF_ERR_UNSUPPORTED;
    const MapDev& g = P->map;
    const int K = P->K, M = P->M;
    const int nent = n_entries_multi(K, M);
    if (!P->wdw_b) {
        const int occ = kMultiOcc[M](K);
        if (occ < 1) {
            snprintf(g_last_error, sizeof(g_last_error),
                     "tpcf_forward_multi: three fields' moments (K=%d, m_max=%d) do not fit in shared memory", K, M);
            return TPCF_ERR_UNSUPPORTED;
        }
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(g.ntiles, (int64_t)P->num_sms * occ));
        float2 *b, *c;
        double *sl, *su;
        TRY_CUDA(P->alloc(&b, g.npix));
        TRY_CUDA(P->alloc(&c, g.npix));
        TRY_CUDA(P->alloc(&sl, (size_t)grid * nent));
        TRY_CUDA(P->alloc(&su, (size_t)nent));
        P->wdw_c = c;
        P->mslots = sl;
        P->msums = su;
        P->multi_grid = grid;
        P->wdw_b = b;
    }
    pack_kernel<<<P->num_sms * 8, 256, 0, s>>>(d_delta_a, d_w_a, P->wdw, g.npix);
    pack_kernel<<<P->num_sms * 8, 256, 0, s>>>(d_delta_b, d_w_b, P->wdw_b, g.npix);
    pack_kernel<<<P->num_sms * 8, 256, 0, s>>>(d_delta_c, d_w_c, P->wdw_c, g.npix);
    TRY_CUDA(cudaMemsetAsync(P->mslots, 0, sizeof(double) * (size_t)P->multi_grid * nent, s));
    TRY_CUDA(cudaMemsetAsync(P->counter, 0, sizeof(int), s));
    MapCall c{};
    c.wdw = P->wdw;
    c.piv_lo = pivot_begin;
    c.piv_hi = pivot_end;
    c.slots = P->mslots;
    c.counter = P->counter;
    c.status = P->status;
    c.flush = P->tune_fwd.flush;
    tile_range(P, pivot_begin, pivot_end, &c.tile_lo, &c.tile_hi, true);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(c.tile_hi - c.tile_lo, P->multi_grid));
    TRY_CUDA(kMulti[M](g, c, P->wdw_b, P->wdw_c, grid, s));
    reduce_slots_kernel<<<n_blocks(nent, 128), 128, 0, s>>>(P->mslots, P->multi_grid, nent, P->msums);
    const int nout = (M + 1) * K * K;
    finalize_full_kernel<<<n_blocks(nout, 128), 128, 0, s>>>(P->msums, K, M, d_zeta, d_norm, d_sums);
    P->launches += 6;  // three packs, the pair kernel, reduce, finalize
    TRY_CUDA(cudaGetLastError());
    return TPCF_OK;
}

extern "C" tpcf_status tpcf_count_pairs(tpcf_plan plan, const float* d_w, int64_t pivot_begin,
                                        int64_t pivot_end, int64_t* d_counts, void* stream) {
    if (!plan || !d_w || !d_counts) return TPCF_ERR_INVALID_ARG;
    if (pivot_begin < 0 || pivot_end < pivot_begin || pivot_end > plan->npoints) return TPCF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    plan->last_stream = s;
    if (plan->kind == PLAN_CATALOG) return catalog_count(plan, d_w, pivot_begin, pivot_end, d_counts, s);
    if (plan->kind != PLAN_MAP) return TPCF_ERR_UNSUPPORTED;
    const MapDev& g = plan->map;
    // only the weights matter: pack them with a zero field
    pack_kernel<<<plan->num_sms * 8, 256, 0, s>>>(d_w, d_w, plan->wdw, g.npix);
    plan->launches += 2;
    TRY_CUDA(cudaMemsetAsync(d_counts, 0, 3 * sizeof(int64_t), s));
    int64_t tlo, thi;
    tile_range(plan, pivot_begin, pivot_end, &tlo, &thi, false);
    TRY_CUDA(map_count_launch(g, plan->wdw, pivot_begin, pivot_end, tlo, thi, (unsigned long long*)d_counts,
                              plan->num_sms * 4, s));
    return TPCF_OK;
}

static tpcf_status map_backward(tpcf_plan_s* P, const float* d_delta, const float* d_w, int64_t lo, int64_t hi,
                                const double* d_norm, const double* d_dL, float* d_grad, cudaStream_t s) {
    const MapDev& g = P->map;
    pack_kernel<<<P->num_sms * 8, 256, 0, s>>>(d_delta, d_w, P->wdw, g.npix);
    const int nout = (P->M + 1) * P->K * P->K;
    const int self = (P->flags & TPCF_SELF_PAIRS_SUBTRACT) ? 1 : 0;
    adjoint_prep_kernel<<<n_blocks(nout, 128), 128, 0, s>>>(d_dL, d_norm, P->K, P->M, P->H, self);
    zero_f32_kernel<<<P->num_sms * 8, 256, 0, s>>>(d_grad, g.npix);
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
    c.self_subtract = self;
    c.flush = P->tune_bwd.flush;
    tile_range(P, lo, hi, &c.tile_lo, &c.tile_hi, false);
    const int grid = launch_grid(P, P->tune_bwd, c.tile_hi - c.tile_lo, P->bwd_grid);
    TRY_CUDA(kLaunch[P->M].bwd(g, c, grid, P->tune_bwd.variant, s));
    return TPCF_OK;
}

extern "C" tpcf_status tpcf_backward(tpcf_plan plan, const float* d_delta, const float* d_w, int64_t pivot_begin,
                                     int64_t pivot_end, const double* d_norm, const double* d_dL_dzeta,
                                     float* d_grad, void* stream) {
    if (!plan || !d_delta || !d_w || !d_norm || !d_dL_dzeta || !d_grad) return TPCF_ERR_INVALID_ARG;
    if (pivot_begin < 0 || pivot_end < pivot_begin || pivot_end > plan->npoints) return TPCF_ERR_INVALID_ARG;
    if (plan->flags & NORM_FLAGS) {
        set_error("tpcf_backward: plans with a per-pivot normalisation have no adjoint");
        return TPCF_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    plan->last_stream = s;
    if (plan->kind == PLAN_MAP)
        return map_backward(plan, d_delta, d_w, pivot_begin, pivot_end, d_norm, d_dL_dzeta, d_grad, s);
    if (plan->kind == PLAN_CATALOG)
        return catalog_backward(plan, d_delta, d_w, pivot_begin, pivot_end, d_norm, d_dL_dzeta, d_grad, s);
    return TPCF_ERR_UNSUPPORTED;
}

extern "C" tpcf_status tpcf_plan_halo(tpcf_plan plan, int64_t begin, int64_t end, int64_t* halo_begin,
                                      int64_t* halo_end) {
    if (!plan || !halo_begin || !halo_end) return TPCF_ERR_INVALID_ARG;
    if (begin < 0 || end < begin || end > plan->npoints) return TPCF_ERR_INVALID_ARG;
    if (plan->kind != PLAN_MAP) {
        set_error("tpcf_plan_halo: map plans only");
        return TPCF_ERR_UNSUPPORTED;
    }
    if (begin == end) {
        *halo_begin = *halo_end = begin;
        return TPCF_OK;
    }
    const int64_t nside = plan->map.nside;
    const int64_t ra = ring_of_pixel(nside, begin), rb = ring_of_pixel(nside, end - 1);
    int2 wa, wb;
    // ring windows are symmetric (ring r is in reach of ring i iff i is in reach of r)
    // and monotone in the ring index, so the halo rings are those of the end rings
    TRY_CUDA(cudaMemcpy(&wa, plan->map.ring_range + ra, sizeof(int2), cudaMemcpyDeviceToHost));
    TRY_CUDA(cudaMemcpy(&wb, plan->map.ring_range + rb, sizeof(int2), cudaMemcpyDeviceToHost));
    *halo_begin = ring_first_pixel(nside, wa.x);
    *halo_end = ring_first_pixel(nside, (int64_t)wb.y + 1);
    return TPCF_OK;
}

extern "C" tpcf_status tpcf_run_host(tpcf_plan plan, const float* h_delta, const float* h_w,
                                     const double* h_dL_dzeta, double* h_zeta, double* h_norm, float* h_grad,
                                     void* stream) {
    if (!plan || !h_delta || !h_w || !h_zeta || !h_norm) return TPCF_ERR_INVALID_ARG;
    if (h_dL_dzeta && !h_grad) return TPCF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    tpcf_plan_s* P = plan;
    const int64_t n = P->npoints;
    const size_t nz = (size_t)(P->M + 1) * P->K * P->K * 2;
    if (!P->st_delta) {
        // staging buffers, kept by the plan; published together so that a failed
        // allocation leaves the plan as it was (what was allocated is freed with it)
        float *sd, *sw, *sg;
        double *sdl, *sz, *sn;
        TRY_CUDA(P->alloc(&sd, n));
        TRY_CUDA(P->alloc(&sw, n));
        TRY_CUDA(P->alloc(&sdl, nz));
        TRY_CUDA(P->alloc(&sz, nz));
        TRY_CUDA(P->alloc(&sn, (size_t)P->K * P->K));
        TRY_CUDA(P->alloc(&sg, n));
        P->st_w = sw;
        P->st_dL = sdl;
        P->st_zeta = sz;
        P->st_norm = sn;
        P->st_grad = sg;
        P->st_delta = sd;
    }
    TRY_CUDA(cudaMemcpyAsync(P->st_delta, h_delta, sizeof(float) * n, cudaMemcpyHostToDevice, s));
    TRY_CUDA(cudaMemcpyAsync(P->st_w, h_w, sizeof(float) * n, cudaMemcpyHostToDevice, s));
    tpcf_status st = tpcf_forward(P, P->st_delta, P->st_w, 0, n, P->st_zeta, P->st_norm, nullptr, stream);
    if (st != TPCF_OK) return st;
    if (h_dL_dzeta) {
        TRY_CUDA(cudaMemcpyAsync(P->st_dL, h_dL_dzeta, sizeof(double) * nz, cudaMemcpyHostToDevice, s));
        st = tpcf_backward(P, P->st_delta, P->st_w, 0, n, P->st_norm, P->st_dL, P->st_grad, stream);
        if (st != TPCF_OK) return st;
        TRY_CUDA(cudaMemcpyAsync(h_grad, P->st_grad, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    }
    TRY_CUDA(cudaMemcpyAsync(h_zeta, P->st_zeta, sizeof(double) * nz, cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaMemcpyAsync(h_norm, P->st_norm, sizeof(double) * P->K * P->K, cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    return tpcf_plan_sync(P);
}

extern "C" tpcf_status tpcf_plan_sync(tpcf_plan plan) {
    if (!plan) return TPCF_ERR_INVALID_ARG;
    TRY_CUDA(cudaStreamSynchronize(plan->last_stream));
    int st = 0;
    TRY_CUDA(cudaMemcpy(&st, plan->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & ST_TC_TIMEOUT_BIT) {
        snprintf(g_last_error, sizeof(g_last_error), "device status 0x%x (tensor-core wait timed out)", st);
        return TPCF_ERR_TIMEOUT;
    }
    if (st & ST_BAD_TILE) {
        snprintf(g_last_error, sizeof(g_last_error), "device status 0x%x (bad tile table)", st);
        return TPCF_ERR_DEVICE;
    }
    return TPCF_OK;
}

extern "C" void tpcf_plan_destroy(tpcf_plan plan) {
    if (!plan) return;
    cudaStreamSynchronize(plan->last_stream);
    delete plan;
}
