// Per-M instantiation of the map kernels.  The build compiles this file once for
// every multipole limit TPCF_M = 0..TPCF_MAX_M and links the objects together.
#include "cat_kernels.cuh"

#ifndef TPCF_M
#error "compile with -DTPCF_M=<m_max>"
#endif

#define TPCF_CAT2(a, b) a##b
#define TPCF_CAT(a, b) TPCF_CAT2(a, b)

namespace tpcf {

// Every pair kernel asks for the largest shared-memory carveout: they are sized to fit
// 2-3 CTAs per SM only with it (the occupancy queries below assume it as well).
template <class Kern>
static cudaError_t prefer_shared(Kern* k, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
}

// Launch the pair kernel `k` with `smem` bytes of dynamic shared memory.
template <class Kern>
static cudaError_t launch(Kern* k, size_t smem, int grid, const MapDev& g, const MapCall& c, cudaStream_t s) {
    cudaError_t e = prefer_shared(k, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NTHREADS, smem, s>>>(g, c);
    return cudaGetLastError();
}

template <class Kern>
static int occupancy(Kern* k, size_t smem) {
    int nb = 0;
    if (prefer_shared(k, smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NTHREADS, smem) != cudaSuccess) return 0;
    return nb;
}

// The forward pair kernel; variant 3 or 2 = CTAs per SM its registers are sized for.
cudaError_t TPCF_CAT(map_fwd_launch_m, TPCF_M)(const MapDev& g, const MapCall& c, int grid, int variant,
                                               cudaStream_t s) {
    const size_t smem = tile_floats<TPCF_M>(g.K) * sizeof(float);
    if (c.group > 1)  // shared neighbour lists (self pairs kept)
        return launch(map_fwd_kernel<TPCF_M, false, false, 3, true>, smem, grid, g, c, s);
    if (c.self_subtract)
        return variant == 2 ? launch(map_fwd_kernel<TPCF_M, true, false, 2>, smem, grid, g, c, s)
                            : launch(map_fwd_kernel<TPCF_M, true, false, 3>, smem, grid, g, c, s);
    return variant == 2 ? launch(map_fwd_kernel<TPCF_M, false, false, 2>, smem, grid, g, c, s)
                        : launch(map_fwd_kernel<TPCF_M, false, false, 3>, smem, grid, g, c, s);
}

cudaError_t TPCF_CAT(map_bwd_launch_m, TPCF_M)(const MapDev& g, const MapCall& c, int grid, int variant,
                                               cudaStream_t s) {
    const size_t smem = bwd_tile_floats<TPCF_M>(g.K) * sizeof(float);
    if (c.self_subtract)
        return variant == 2 ? launch(map_bwd_kernel<TPCF_M, true, 2>, smem, grid, g, c, s)
                            : launch(map_bwd_kernel<TPCF_M, true, 3>, smem, grid, g, c, s);
    return variant == 2 ? launch(map_bwd_kernel<TPCF_M, false, 2>, smem, grid, g, c, s)
                        : launch(map_bwd_kernel<TPCF_M, false, 3>, smem, grid, g, c, s);
}

// Resident CTAs per SM of the forward variant (shared memory and registers).
int TPCF_CAT(map_fwd_occupancy_m, TPCF_M)(int K, int self_subtract, int variant) {
    const size_t smem = tile_floats<TPCF_M>(K) * sizeof(float);
    if (self_subtract)
        return variant == 2 ? occupancy(map_fwd_kernel<TPCF_M, true, false, 2>, smem)
                            : occupancy(map_fwd_kernel<TPCF_M, true, false, 3>, smem);
    return variant == 2 ? occupancy(map_fwd_kernel<TPCF_M, false, false, 2>, smem)
                        : occupancy(map_fwd_kernel<TPCF_M, false, false, 3>, smem);
}

// Resident CTAs per SM of the adjoint variant (either self-pair mode).
int TPCF_CAT(map_bwd_occupancy_m, TPCF_M)(int K, int variant) {
    const size_t smem = bwd_tile_floats<TPCF_M>(K) * sizeof(float);
    int a, b;
    if (variant == 2) {
        a = occupancy(map_bwd_kernel<TPCF_M, false, 2>, smem);
        b = occupancy(map_bwd_kernel<TPCF_M, true, 2>, smem);
    } else {
        a = occupancy(map_bwd_kernel<TPCF_M, false, 3>, smem);
        b = occupancy(map_bwd_kernel<TPCF_M, true, 3>, smem);
    }
    return a < b ? a : b;
}

// Forward with the split-precision tensor-core contraction.
cudaError_t TPCF_CAT(map_fwd_tc_launch_m, TPCF_M)(const MapDev& g, const MapCall& c, int grid, cudaStream_t s) {
    const size_t smem = tc_smem_bytes(g.K, TPCF_M, c.self_subtract != 0);
    if (c.self_subtract) {
        auto* k = map_fwd_tc_kernel<TPCF_M, true>;
        cudaError_t e = prefer_shared(k, smem);
        if (e != cudaSuccess) return e;
        k<<<grid, NTHREADS, smem, s>>>(g, c);
    } else {
        auto* k = map_fwd_tc_kernel<TPCF_M, false>;
        cudaError_t e = prefer_shared(k, smem);
        if (e != cudaSuccess) return e;
        k<<<grid, NTHREADS, smem, s>>>(g, c);
    }
    return cudaGetLastError();
}

// Resident CTAs per SM from the SM's register file and shared memory.  Used for the
// tensor-core kernel, for which cudaOccupancyMaxActiveBlocksPerMultiprocessor answers 1
// although 3 CTAs fit by registers and shared memory (and the profiler's occupancy
// limits agree); the CTAs are persistent and never wait on each other, so a grid
// larger than what is resident is still correct.
template <class Kern>
static int occupancy_by_resources(Kern* k, size_t smem) {
    if (prefer_shared(k, smem) != cudaSuccess) return 0;
    cudaFuncAttributes a;
    int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0;
    if (cudaFuncGetAttributes(&a, k) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess)
        return 0;
    const size_t per_cta_smem = smem + a.sharedSizeBytes + (size_t)reserved;
    const int warps = NTHREADS / 32;
    const int regs_warp = (a.numRegs * 32 + 255) / 256 * 256;  // allocated per warp in units of 256
    const int by_smem = (int)((size_t)smem_sm / per_cta_smem);
    const int by_regs = regs_warp > 0 ? regs_sm / (regs_warp * warps) : 0;
    return by_smem < by_regs ? by_smem : by_regs;
}

int TPCF_CAT(map_fwd_tc_occupancy_m, TPCF_M)(int K, int self_subtract) {
    const size_t smem = tc_smem_bytes(K, TPCF_M, self_subtract != 0);
    const int nb = self_subtract ? occupancy_by_resources(map_fwd_tc_kernel<TPCF_M, true>, smem)
                                 : occupancy_by_resources(map_fwd_tc_kernel<TPCF_M, false>, smem);
    // at most 512 / TC_TMEM_COLS accumulators per SM; more resident CTAs would wait in tcgen05.alloc
    return nb < 512 / TC_TMEM_COLS ? nb : 512 / TC_TMEM_COLS;
}

// Multi-field forward (three fields on the same pixels).
cudaError_t TPCF_CAT(map_fwd_multi_launch_m, TPCF_M)(const MapDev& g, const MapCall& c, const float2* wdwB,
                                                     const float2* wdwC, int grid, cudaStream_t s) {
    const size_t smem = multi_tile_floats(g.K, TPCF_M) * sizeof(float);
    auto* k = map_fwd_multi_kernel<TPCF_M>;
    cudaError_t e = prefer_shared(k, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NTHREADS, smem, s>>>(g, c, wdwB, wdwC);
    return cudaGetLastError();
}

int TPCF_CAT(map_fwd_multi_occupancy_m, TPCF_M)(int K) {
    return occupancy(map_fwd_multi_kernel<TPCF_M>, multi_tile_floats(K, TPCF_M) * sizeof(float));
}

// Multi-field forward on a catalogue.
cudaError_t TPCF_CAT(cat_fwd_multi_launch_m, TPCF_M)(const CatDev& g, const MapCall& c, const float2* wdwB,
                                                     const float2* wdwC, int grid, cudaStream_t s) {
    const size_t smem = cat_multi_bytes<TPCF_M>(g.K);
    auto* k = cat_fwd_multi_kernel<TPCF_M>;
    cudaError_t e = prefer_shared(k, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NTHREADS, smem, s>>>(g, c, wdwB, wdwC);
    return cudaGetLastError();
}

int TPCF_CAT(cat_fwd_multi_occupancy_m, TPCF_M)(int K) {
    return occupancy(cat_fwd_multi_kernel<TPCF_M>, cat_multi_bytes<TPCF_M>(K));
}

// Forward that reads the caller's delta and w directly (no packed copy).
cudaError_t TPCF_CAT(map_fwd_direct_launch_m, TPCF_M)(const MapDev& g, const MapCall& c, int grid,
                                                      cudaStream_t s) {
    const size_t smem = tile_floats<TPCF_M>(g.K) * sizeof(float);
    auto* k = map_fwd_kernel<TPCF_M, false, true>;
    cudaError_t e = prefer_shared(k, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NTHREADS, smem, s>>>(g, c);
    return cudaGetLastError();
}

size_t TPCF_CAT(map_fwd_smem_m, TPCF_M)(int K) { return tile_floats<TPCF_M>(K) * sizeof(float); }
size_t TPCF_CAT(map_bwd_smem_m, TPCF_M)(int K) { return bwd_tile_floats<TPCF_M>(K) * sizeof(float); }

// Batched forward / adjoint over all the plans of a batch whose largest m_max is this
// M (the dynamic shared memory is the largest any of them needs).
cudaError_t TPCF_CAT(batch_fwd_launch_m, TPCF_M)(const BatchItem* items, int n, long long total,
                                                 unsigned long long* counter, size_t smem, int grid, cudaStream_t s) {
    auto* k = batch_fwd_kernel<TPCF_M>;
    cudaError_t e = prefer_shared(k, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NTHREADS, smem, s>>>(items, n, total, counter);
    return cudaGetLastError();
}

cudaError_t TPCF_CAT(batch_bwd_launch_m, TPCF_M)(const BatchItem* items, int n, long long total,
                                                 unsigned long long* counter, size_t smem, int grid,
                                                 cudaStream_t s) {
    auto* k = batch_bwd_kernel<TPCF_M>;
    cudaError_t e = prefer_shared(k, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NTHREADS, smem, s>>>(items, n, total, counter);
    return cudaGetLastError();
}

int TPCF_CAT(batch_fwd_occupancy_m, TPCF_M)(size_t smem) { return occupancy(batch_fwd_kernel<TPCF_M>, smem); }

int TPCF_CAT(batch_bwd_occupancy_m, TPCF_M)(size_t smem) { return occupancy(batch_bwd_kernel<TPCF_M>, smem); }

// Catalogue forward.
cudaError_t TPCF_CAT(cat_fwd_launch_m, TPCF_M)(const CatDev& g, const MapCall& c, int grid, cudaStream_t s) {
    const size_t smem = cat_tile_bytes<TPCF_M>(g.K);
    if (c.self_subtract) {
        auto* k = cat_fwd_kernel<TPCF_M, true>;
        cudaError_t e = prefer_shared(k, smem);
        if (e != cudaSuccess) return e;
        k<<<grid, NTHREADS, smem, s>>>(g, c);
    } else {
        auto* k = cat_fwd_kernel<TPCF_M, false>;
        cudaError_t e = prefer_shared(k, smem);
        if (e != cudaSuccess) return e;
        k<<<grid, NTHREADS, smem, s>>>(g, c);
    }
    return cudaGetLastError();
}

int TPCF_CAT(cat_fwd_occupancy_m, TPCF_M)(int K, int self_subtract) {
    const size_t smem = cat_tile_bytes<TPCF_M>(K);
    return self_subtract ? occupancy(cat_fwd_kernel<TPCF_M, true>, smem) : occupancy(cat_fwd_kernel<TPCF_M, false>, smem);
}

// Catalogue adjoint.
cudaError_t TPCF_CAT(cat_bwd_launch_m, TPCF_M)(const CatDev& g, const MapCall& c, int grid, cudaStream_t s) {
    const size_t smem = cat_bwd_bytes<TPCF_M>(g.K);
    auto* k = cat_bwd_kernel<TPCF_M>;
    cudaError_t e = prefer_shared(k, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NTHREADS, smem, s>>>(g, c);
    return cudaGetLastError();
}

int TPCF_CAT(cat_bwd_occupancy_m, TPCF_M)(int K) {
    const size_t smem = cat_bwd_bytes<TPCF_M>(K);
    int nb = 0;
    prefer_shared(cat_bwd_kernel<TPCF_M>, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cat_bwd_kernel<TPCF_M>, NTHREADS, smem);
    return nb;
}

#if TPCF_M == 0
cudaError_t cat_count_launch(const CatDev& g, const float2* wdw, long long lo, long long hi, int* counter,
                             unsigned long long* counts, int grid, cudaStream_t s) {
    cat_count_kernel<<<grid, NTHREADS, 0, s>>>(g, wdw, lo, hi, counter, counts);
    return cudaGetLastError();
}

cudaError_t map_count_launch(const MapDev& g, const float2* wdw, long long lo, long long hi, long long tlo,
                             long long thi, unsigned long long* counts, int grid, cudaStream_t s) {
    map_count_kernel<<<grid, NTHREADS, 0, s>>>(g, wdw, lo, hi, tlo, thi, counts);
    return cudaGetLastError();
}
#endif

}  // namespace tpcf
