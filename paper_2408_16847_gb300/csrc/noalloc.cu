// tpcf_forward_noalloc: the map forward without any device allocation.
//
// Who needs it: programs that give all device memory to their own pool allocator
// at start-up (a cudaMalloc made later inside a library call fails, or fragments
// the pool), programs whose hot loop must not enter the CUDA allocator because
// cudaMalloc/cudaFree can synchronise the device, and embedders that account for
// every byte of device memory.  They create the plan once, during set-up, and then
// call this entry point, which uses only the caller's buffers, the plan's
// read-only tables and the fixed scratch array below.
//
// The scratch lives in a file-scope __device__ array.  This file is its own CUDA
// module, and CUDA loads modules lazily, so the array is placed on a device when its
// address is first looked up: tpcf_plan_create_map does that (noalloc_prepare), so
// the 16 MiB are taken while the caller sets up, before its pool allocator claims
// the device, and stay until the process exits.  All calls share it: calls
// whose GPU work overlaps (two streams, two host threads, two plans at once) race
// on it and must be serialised by the caller.  A call clears what must start at
// zero (the work counter and the partial-sum slots) before its kernels run.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "geometry.cuh"
#include "plan.cuh"

namespace tpcf {

#define TPCF_DECL_DIRECT(m) \
    cudaError_t map_fwd_direct_launch_m##m(const MapDev&, const MapCall&, int, cudaStream_t);
TPCF_DECL_DIRECT(0) TPCF_DECL_DIRECT(1) TPCF_DECL_DIRECT(2) TPCF_DECL_DIRECT(3) TPCF_DECL_DIRECT(4)
TPCF_DECL_DIRECT(5) TPCF_DECL_DIRECT(6) TPCF_DECL_DIRECT(7) TPCF_DECL_DIRECT(8) TPCF_DECL_DIRECT(9)
TPCF_DECL_DIRECT(10) TPCF_DECL_DIRECT(11) TPCF_DECL_DIRECT(12) TPCF_DECL_DIRECT(13) TPCF_DECL_DIRECT(14)
TPCF_DECL_DIRECT(15) TPCF_DECL_DIRECT(16)
#undef TPCF_DECL_DIRECT

typedef cudaError_t (*direct_fn)(const MapDev&, const MapCall&, int, cudaStream_t);
static const direct_fn kDirect[TPCF_MAX_M + 1] = {
    map_fwd_direct_launch_m0,  map_fwd_direct_launch_m1,  map_fwd_direct_launch_m2,  map_fwd_direct_launch_m3,
    map_fwd_direct_launch_m4,  map_fwd_direct_launch_m5,  map_fwd_direct_launch_m6,  map_fwd_direct_launch_m7,
    map_fwd_direct_launch_m8,  map_fwd_direct_launch_m9,  map_fwd_direct_launch_m10, map_fwd_direct_launch_m11,
    map_fwd_direct_launch_m12, map_fwd_direct_launch_m13, map_fwd_direct_launch_m14, map_fwd_direct_launch_m15,
    map_fwd_direct_launch_m16};

// Scratch layout: [0, 256) work counter; [256, 256 + 8 nent) reduced sums;
// then one slot of nent doubles per CTA.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(16) << 20;
constexpr size_t NOALLOC_HEADER = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
static std::mutex g_scratch_mu;
static void* g_scratch_addr[MAX_DEVICES];

// Device address of the scratch array on the current device; looked up once per
// device (the host-side name of a __device__ array is not a device address).
static tpcf_status scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= MAX_DEVICES) {
        set_error("tpcf_forward_noalloc: device ordinal out of range");
        return TPCF_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = (unsigned char*)g_scratch_addr[dev];
    return TPCF_OK;
}

// Called by tpcf_plan_create_map with the plan's device current: loads this module
// (and with it the scratch array) on that device and caches the array's address.
// A failure is not fatal for the plan; it is reported again by the first
// tpcf_forward_noalloc on that device.
tpcf_status noalloc_prepare(int dev) {
    unsigned char* p = nullptr;
    return scratch_address(dev, &p);
}

}  // namespace tpcf

using namespace tpcf;

extern "C" tpcf_status tpcf_forward_noalloc(tpcf_plan plan, const float* d_delta, const float* d_w,
                                            int64_t pivot_begin, int64_t pivot_end, double* d_zeta,
                                            double* d_norm, void* stream) {
    if (!plan || !d_delta || !d_w || !d_zeta || !d_norm) return TPCF_ERR_INVALID_ARG;
    if (pivot_begin < 0 || pivot_end < pivot_begin || pivot_end > plan->npoints) return TPCF_ERR_INVALID_ARG;
    if (plan->kind != PLAN_MAP) {
        set_error("tpcf_forward_noalloc: map plans only");
        return TPCF_ERR_UNSUPPORTED;
    }
    if (plan->flags & TPCF_CONTRACT_TC) {
        set_error("tpcf_forward_noalloc: FP32 contraction only");
        return TPCF_ERR_UNSUPPORTED;
    }
    if (plan->flags & TPCF_SELF_PAIRS_SUBTRACT) {
        set_error("tpcf_forward_noalloc: self-pair subtraction is not available here");
        return TPCF_ERR_UNSUPPORTED;
    }
    const size_t nent = (size_t)plan->nent;
    const size_t slot_bytes = nent * sizeof(double);
    const size_t sums_bytes = (slot_bytes + 255) / 256 * 256;
    if (NOALLOC_HEADER + sums_bytes + slot_bytes > NOALLOC_SCRATCH_BYTES) {
        char msg[200];
        snprintf(msg, sizeof(msg),
                 "tpcf_forward_noalloc: K=%d, m_max=%d needs %zu bytes of scratch per CTA; the fixed "
                 "scratch holds %zu bytes",
                 plan->K, plan->M, slot_bytes, NOALLOC_SCRATCH_BYTES - NOALLOC_HEADER - sums_bytes);
        set_error(msg);
        return TPCF_ERR_INVALID_ARG;
    }
    int dev = 0;
    TRY_CUDA(cudaGetDevice(&dev));
    unsigned char* base = nullptr;
    tpcf_status st = scratch_address(dev, &base);
    if (st != TPCF_OK) return st;
    int* counter = (int*)base;
    double* sums = (double*)(base + NOALLOC_HEADER);
    double* slots = (double*)(base + NOALLOC_HEADER + sums_bytes);
    const size_t room = (NOALLOC_SCRATCH_BYTES - NOALLOC_HEADER - sums_bytes) / slot_bytes;
    const int grid = (int)std::min<size_t>((size_t)plan->fwd_grid, room);
    cudaStream_t s = (cudaStream_t)stream;
    plan->last_stream = s;
    TRY_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), s));
    TRY_CUDA(cudaMemsetAsync(slots, 0, slot_bytes * (size_t)grid, s));
    MapCall c{};
    c.delta = d_delta;
    c.w = d_w;
    c.piv_lo = pivot_begin;
    c.piv_hi = pivot_end;
    c.slots = slots;
    c.counter = counter;
    c.status = plan->status;
    c.self_subtract = 0;
    c.norm = norm_of_flags(plan->flags);
    c.quad = plan->tune_fwd.quad;
    c.flush = plan->tune_fwd.flush;
    c.tile_lo = 0;  // every tile; those without a pivot in range return at once
    c.tile_hi = plan->map.ntiles;
    TRY_CUDA(kDirect[plan->M](plan->map, c, grid, s));
    reduce_slots_kernel<<<(plan->nent + 127) / 128, 128, 0, s>>>(slots, grid, plan->nent, sums);
    const int nout = (plan->M + 1) * plan->K * plan->K;
    finalize_kernel<<<(nout + 127) / 128, 128, 0, s>>>(sums, plan->K, plan->M, 0, 1.0, d_zeta, d_norm, nullptr);
    TRY_CUDA(cudaGetLastError());
    plan->launches += 3;
    return TPCF_OK;
}
