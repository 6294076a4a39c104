// Batched execution of several map plans, recorded once into a CUDA graph.
//
// A batch runs the estimator of Sec. 3 for n independent maps (any mix of nside,
// bins, m_max and self-pair mode) with a fixed, short launch sequence whose length
// does not grow with n: the small per-entry kernels take the plan as blockIdx.y, and
// one persistent forward and one persistent adjoint launch, compiled for the batch's
// largest m_max, pull the tiles of every plan from one concatenated work queue (each
// plan's tiles run with its own m_max, bins and self-pair mode).  The sequence is
// captured into a graph at creation; every launch replays it.
#include <cuda_runtime.h>
#include <stdio.h>

#include <algorithm>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "geometry.cuh"
#include "plan.cuh"

using namespace tpcf;

namespace tpcf {
#define TPCF_DECL_BATCH_M(m)                                                                                  \
    cudaError_t batch_fwd_launch_m##m(const BatchItem*, int, long long, unsigned long long*, size_t, int,      \
                                      cudaStream_t);                                                          \
    cudaError_t batch_bwd_launch_m##m(const BatchItem*, int, long long, unsigned long long*, size_t, int,      \
                                      cudaStream_t);                                                          \
    int batch_fwd_occupancy_m##m(size_t);                                                                     \
    int batch_bwd_occupancy_m##m(size_t);
TPCF_DECL_BATCH_M(0) TPCF_DECL_BATCH_M(1) TPCF_DECL_BATCH_M(2) TPCF_DECL_BATCH_M(3) TPCF_DECL_BATCH_M(4)
TPCF_DECL_BATCH_M(5) TPCF_DECL_BATCH_M(6) TPCF_DECL_BATCH_M(7) TPCF_DECL_BATCH_M(8) TPCF_DECL_BATCH_M(9)
TPCF_DECL_BATCH_M(10) TPCF_DECL_BATCH_M(11) TPCF_DECL_BATCH_M(12) TPCF_DECL_BATCH_M(13) TPCF_DECL_BATCH_M(14)
TPCF_DECL_BATCH_M(15) TPCF_DECL_BATCH_M(16)
#undef TPCF_DECL_BATCH_M

struct BLaunch {
    cudaError_t (*fwd)(const BatchItem*, int, long long, unsigned long long*, size_t, int, cudaStream_t);
    cudaError_t (*bwd)(const BatchItem*, int, long long, unsigned long long*, size_t, int, cudaStream_t);
    int (*fwd_occ)(size_t);
    int (*bwd_occ)(size_t);
};
#define TPCF_BROW(m) {batch_fwd_launch_m##m, batch_bwd_launch_m##m, batch_fwd_occupancy_m##m, batch_bwd_occupancy_m##m}
static const BLaunch kBatch[TPCF_MAX_M + 1] = {
    TPCF_BROW(0),  TPCF_BROW(1),  TPCF_BROW(2),  TPCF_BROW(3),  TPCF_BROW(4),  TPCF_BROW(5),
    TPCF_BROW(6),  TPCF_BROW(7),  TPCF_BROW(8),  TPCF_BROW(9),  TPCF_BROW(10), TPCF_BROW(11),
    TPCF_BROW(12), TPCF_BROW(13), TPCF_BROW(14), TPCF_BROW(15), TPCF_BROW(16)};
#undef TPCF_BROW
}  // namespace tpcf

namespace {
// The plans of a batch: one pair-kernel launch each way, compiled for their largest
// m_max.
struct Group {
    int M = 0;
    std::vector<int> members;  // indices into the batch's plan list
    BatchItem* d_items = nullptr;
    long long total_tiles = 0;
    size_t fwd_smem = 0, bwd_smem = 0;
    int fwd_grid = 0, bwd_grid = 0;
};
}  // namespace

struct tpcf_batch_s {
    int n = 0;
    int with_bwd = 0;
    std::vector<tpcf_plan> plans;
    std::vector<Group> groups;
    std::vector<void*> allocs;
    BatchIO* d_io = nullptr;
    unsigned long long* d_counters = nullptr;  // 2 per group (forward, adjoint)
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t last = nullptr;
    int64_t kernels = 0;  // kernel nodes per replay

    template <typename T>
    cudaError_t alloc(T** p, size_t count) {
        void* q = nullptr;
        cudaError_t e = tpcf::dev_malloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
        if (e != cudaSuccess) return e;
        allocs.push_back(q);
        *p = (T*)q;
        return cudaSuccess;
    }
    ~tpcf_batch_s() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
        for (void* p : allocs) tpcf::dev_free(p);
    }
};

static int n_blocks(int64_t n, int bs) { return (int)((n + bs - 1) / bs); }

// Records the whole batch on stream s (which is being captured).
static tpcf_status record(tpcf_batch_s* B, int num_sms, int max_nent, int max_nout, cudaStream_t s) {
    const int n = B->n;
    const dim3 gbig(num_sms * 2, n);
    batch_pack_kernel<<<gbig, 256, 0, s>>>(B->d_io);
    batch_zero_kernel<<<gbig, 256, 0, s>>>(B->d_io, B->with_bwd);
    B->kernels += 2;
    TRY_CUDA(cudaMemsetAsync(B->d_counters, 0, sizeof(unsigned long long) * 2 * B->groups.size(), s));
    for (size_t gi = 0; gi < B->groups.size(); ++gi) {
        const Group& G = B->groups[gi];
        TRY_CUDA(kBatch[G.M].fwd(G.d_items, (int)G.members.size(), G.total_tiles, B->d_counters + 2 * gi,
                                 G.fwd_smem, G.fwd_grid, s));
        B->kernels += 1;
    }
    batch_reduce_kernel<<<dim3(n_blocks(max_nent, 128), n), 128, 0, s>>>(B->d_io);
    batch_finalize_kernel<<<dim3(n_blocks(max_nout, 128), n), 128, 0, s>>>(B->d_io);
    B->kernels += 2;
    if (B->with_bwd) {
        batch_adjoint_prep_kernel<<<dim3(n_blocks(max_nout, 128), n), 128, 0, s>>>(B->d_io);
        B->kernels += 1;
        for (size_t gi = 0; gi < B->groups.size(); ++gi) {
            const Group& G = B->groups[gi];
            TRY_CUDA(kBatch[G.M].bwd(G.d_items, (int)G.members.size(), G.total_tiles, B->d_counters + 2 * gi + 1,
                                     G.bwd_smem, G.bwd_grid, s));
            B->kernels += 1;
        }
    }
    TRY_CUDA(cudaGetLastError());
    return TPCF_OK;
}

static tpcf_status batch_build(tpcf_batch_s* B, const tpcf_plan* plans, const float* const* d_delta,
                               const float* const* d_w, double* const* d_zeta, double* const* d_norm,
                               const double* const* d_dL, float* const* d_grad) {
    const int n = B->n;
    int dev = 0, num_sms = 0;
    TRY_CUDA(cudaGetDevice(&dev));
    TRY_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));

    // one group: every plan, compiled for the largest m_max
    B->groups.emplace_back();
    for (int i = 0; i < n; ++i) {
        B->groups[0].members.push_back(i);
        B->groups[0].M = std::max(B->groups[0].M, plans[i]->M);
    }

    // per-plan slots sized for its group's forward grid
    std::vector<BatchIO> io(n);
    std::vector<int> grid_of(n, 0);
    for (Group& G : B->groups) {
        for (int i : G.members) {
            const tpcf_plan P = plans[i];
            G.fwd_smem = std::max(G.fwd_smem, tile_floats_rt(P->K, P->M) * sizeof(float));
            G.bwd_smem = std::max(G.bwd_smem, bwd_tile_floats_rt(P->K, P->M) * sizeof(float));
        }
        const int of = kBatch[G.M].fwd_occ(G.fwd_smem);
        TRY_CUDA(cudaGetLastError());
        if (of < 1) {
            set_error("batch forward kernel does not fit on an SM");
            return TPCF_ERR_UNSUPPORTED;
        }
        G.fwd_grid = of * num_sms;
        if (B->with_bwd) {
            const int ob = kBatch[G.M].bwd_occ(G.bwd_smem);
            TRY_CUDA(cudaGetLastError());
            if (ob < 1) {
                set_error("batch adjoint kernel does not fit on an SM");
                return TPCF_ERR_UNSUPPORTED;
            }
            G.bwd_grid = ob * num_sms;
        }
        for (int i : G.members) grid_of[i] = G.fwd_grid;
    }
    int max_nent = 0, max_nout = 0;
    for (int i = 0; i < n; ++i) {
        const tpcf_plan P = plans[i];
        BatchIO& b = io[i];
        b.delta = d_delta[i];
        b.w = d_w[i];
        b.wdw = P->wdw;
        b.npix = P->npoints;
        b.nslots = grid_of[i];
        b.nent = P->nent;
        TRY_CUDA(B->alloc(&b.slots, (size_t)b.nslots * b.nent));
        b.sums = P->sums;
        b.K = P->K;
        b.M = P->M;
        b.self_subtract = (P->flags & TPCF_SELF_PAIRS_SUBTRACT) ? 1 : 0;
        b.zeta = d_zeta[i];
        b.norm = d_norm[i];
        b.dL = B->with_bwd ? d_dL[i] : nullptr;
        b.H = P->H;
        b.grad = B->with_bwd ? d_grad[i] : nullptr;
        max_nent = std::max(max_nent, b.nent);
        max_nout = std::max(max_nout, (P->M + 1) * P->K * P->K);
    }
    TRY_CUDA(B->alloc(&B->d_io, (size_t)n));
    TRY_CUDA(cudaMemcpy(B->d_io, io.data(), sizeof(BatchIO) * n, cudaMemcpyHostToDevice));
    TRY_CUDA(B->alloc(&B->d_counters, 2 * B->groups.size()));

    for (Group& G : B->groups) {
        std::vector<BatchItem> items;
        long long t0 = 0;
        for (int i : G.members) {
            const tpcf_plan P = plans[i];
            BatchItem it{};
            it.g = P->map;
            it.c.wdw = P->wdw;
            it.c.delta = d_delta[i];
            it.c.w = d_w[i];
            it.c.piv_lo = 0;
            it.c.piv_hi = P->npoints;
            it.c.slots = io[i].slots;
            it.c.counter = nullptr;
            it.c.status = P->status;
            it.c.H = P->H;
            it.c.grad = io[i].grad;
            it.c.self_subtract = io[i].self_subtract;
            it.c.flush = P->tune_fwd.flush;
            it.c.quad = P->tune_fwd.quad;
            it.c.tile_lo = 0;
            it.c.tile_hi = P->map.ntiles;
            it.tile0 = t0;
            t0 += P->map.ntiles;
            items.push_back(it);
        }
        G.total_tiles = t0;
        TRY_CUDA(B->alloc(&G.d_items, items.size()));
        TRY_CUDA(cudaMemcpy(G.d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice));
    }

    TRY_CUDA(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
    TRY_CUDA(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeRelaxed));
    tpcf_status st = record(B, num_sms, max_nent, max_nout, B->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(B->cap, &g);
    if (st != TPCF_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    B->graph = g;
    TRY_CUDA(cudaGraphInstantiate(&B->exec, B->graph, 0));
    return TPCF_OK;
}

extern "C" tpcf_status tpcf_batch_create(tpcf_batch* out, const tpcf_plan* plans, int32_t n,
                                         const float* const* d_delta, const float* const* d_w,
                                         double* const* d_zeta, double* const* d_norm,
                                         const double* const* d_dL_dzeta, float* const* d_grad, void* stream) {
    if (!out) return TPCF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!plans || n < 1 || n > TPCF_MAX_BATCH || !d_delta || !d_w || !d_zeta || !d_norm)
        return TPCF_ERR_INVALID_ARG;
    int with_bwd = 0;
    if (d_dL_dzeta) {
        if (!d_grad) return TPCF_ERR_INVALID_ARG;
        with_bwd = 1;
    }
    for (int i = 0; i < n; ++i) {
        const tpcf_plan P = plans[i];
        if (!P || P->kind != PLAN_MAP) {
            set_error("batch members must be map plans");
            return P ? TPCF_ERR_UNSUPPORTED : TPCF_ERR_INVALID_ARG;
        }
        if (!d_delta[i] || !d_w[i] || !d_zeta[i] || !d_norm[i]) return TPCF_ERR_INVALID_ARG;
        if (with_bwd && (!d_dL_dzeta[i] || !d_grad[i])) return TPCF_ERR_INVALID_ARG;
        if (P->flags & TPCF_CONTRACT_TC) {
            set_error("batch members use the FP32 contraction (plan has TPCF_CONTRACT_TC)");
            return TPCF_ERR_UNSUPPORTED;
        }
        if (P->flags & NORM_FLAGS) {
            set_error("batch members use the default normalisation");
            return TPCF_ERR_UNSUPPORTED;
        }
        if (with_bwd && (P->flags & TPCF_SELF_PAIRS_SUBTRACT)) {
            set_error("adjoint with self-pair subtraction");
            return TPCF_ERR_UNSUPPORTED;
        }
        for (int j = 0; j < i; ++j)
            if (plans[j] == P) {
                set_error("a plan appears twice in one batch (its scratch would be shared)");
                return TPCF_ERR_INVALID_ARG;
            }
    }
    // the plans' own scratch (packed inputs, sums, adjoint coefficients) must be idle
    for (int i = 0; i < n; ++i) TRY_CUDA(cudaStreamSynchronize(plans[i]->last_stream));
    (void)stream;
    tpcf_batch_s* B = new (std::nothrow) tpcf_batch_s();
    if (!B) return TPCF_ERR_OOM;
    B->n = n;
    B->with_bwd = with_bwd;
    B->plans.assign(plans, plans + n);
    tpcf_status st = batch_build(B, plans, d_delta, d_w, d_zeta, d_norm, d_dL_dzeta, d_grad);
    if (st != TPCF_OK) {
        cudaDeviceSynchronize();
        delete B;
        return st;
    }
    *out = B;
    return TPCF_OK;
}

extern "C" tpcf_status tpcf_batch_launch(tpcf_batch batch, void* stream) {
    if (!batch || !batch->exec) return TPCF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    TRY_CUDA(cudaGraphLaunch(batch->exec, s));
    batch->last = s;
    for (tpcf_plan P : batch->plans) {
        P->last_stream = s;
        P->launches += batch->kernels;  // every plan reports the batch's kernels
    }
    return TPCF_OK;
}

extern "C" int64_t tpcf_batch_kernel_launches(tpcf_batch batch) { return batch ? batch->kernels : -1; }

extern "C" void tpcf_batch_destroy(tpcf_batch batch) {
    if (!batch) return;
    cudaStreamSynchronize(batch->last);
    delete batch;
}

extern "C" tpcf_status tpcf_forward_batched(const tpcf_plan* plans, int32_t n, const float* const* d_delta,
                                            const float* const* d_w, double* const* d_zeta,
                                            double* const* d_norm, const double* const* d_dL_dzeta,
                                            float* const* d_grad, void* stream) {
    tpcf_batch b = nullptr;
    tpcf_status st = tpcf_batch_create(&b, plans, n, d_delta, d_w, d_zeta, d_norm, d_dL_dzeta, d_grad, stream);
    if (st != TPCF_OK) return st;
    st = tpcf_batch_launch(b, stream);
    tpcf_batch_destroy(b);
    return st;
}
