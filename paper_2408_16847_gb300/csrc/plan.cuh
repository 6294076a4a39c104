// The plan object and the error helpers shared by the host translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdio.h>

#include <vector>

#include "tpcf_internal.cuh"

namespace tpcf {
// Records a message for tpcf_last_error() and maps a CUDA error to a status.
tpcf_status cuda_fail(cudaError_t e, const char* where);
// Records a message for tpcf_last_error().
void set_error(const char* msg);
// Every device allocation of the library goes through these two (api.cu): they keep
// the count of live allocations and honour tpcf_test_fail_allocation().
cudaError_t dev_malloc(void** p, size_t bytes);
void dev_free(void* p);
}  // namespace tpcf

#define TRY_CUDA(call)                                                   \
    do {                                                                 \
        cudaError_t _e = (call);                                         \
        if (_e != cudaSuccess) return tpcf::cuda_fail(_e, #call);        \
    } while (0)

enum PlanKind { PLAN_MAP = 1, PLAN_CATALOG = 2 };

struct tpcf_plan_s {
    using MapDev = tpcf::MapDev;
    int kind = 0;
    int device = 0;
    int num_sms = 0;
    int64_t npoints = 0;
    int K = 0, M = 0;
    uint32_t flags = 0;
    std::vector<double> edges;
    std::vector<void*> allocs;  // everything freed by destroy
    MapDev map{};
    tpcf::CatDev cat{};
    std::vector<int64_t> tile_off_h;  // map plans: first tile of each ring (host copy)
    // launch configuration of the map pair kernels (defaults, or picked by the autotuner):
    // register variant (CTAs per SM the registers are sized for), CTAs per SM launched,
    // rings summed in registers per shared-memory flush
    // and, for the forward, the tile layout (1: quarter-turn runs, 0: consecutive pivots)
    struct Tune {
        int variant = 3, ctas = 0, flush = 8, quad = 0;
    } tune_fwd, tune_bwd;
    bool tuned = false;
    // per-call scratch
    float2* wdw = nullptr;
    double* slots = nullptr;
    int fwd_grid = 0, bwd_grid = 0;
    int nent = 0;
    double* sums = nullptr;
    int* counter = nullptr;
    int* status = nullptr;
    float* H = nullptr;
    // multi-field forward (allocated on its first call): packed fields B and C, slots
    float2* wdw_b = nullptr;
    float2* wdw_c = nullptr;
    double* mslots = nullptr;
    double* msums = nullptr;
    int multi_grid = 0;
    // shared-neighbour-list forward: tile list of the last group size used
    int2* gtiles = nullptr;
    int64_t ngtiles = 0, gtiles_cap = 0;
    int ggroup = 0;
    // staging for tpcf_run_host
    float* st_delta = nullptr;
    float* st_w = nullptr;
    double* st_dL = nullptr;
    double* st_zeta = nullptr;
    double* st_norm = nullptr;
    float* st_grad = nullptr;
    cudaStream_t last_stream = nullptr;
    long long launches = 0;  // kernels this plan has launched (bookkeeping for benchmarks)

    template <typename T>
    cudaError_t alloc(T** p, size_t count) {
        void* q = nullptr;
        cudaError_t e = tpcf::dev_malloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
        if (e != cudaSuccess) return e;
        allocs.push_back(q);
        *p = (T*)q;
        return cudaSuccess;
    }
    ~tpcf_plan_s() {
        for (void* p : allocs) tpcf::dev_free(p);
    }
};
