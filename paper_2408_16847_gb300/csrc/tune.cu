// Launch-configuration autotuner of the map pair kernels.
//
// The search space, per pass (forward, adjoint):
//   * register variant: the kernel compiled for 3 resident CTAs per SM (80 registers
//     per thread, a few spills at large m_max) or for 2 (128 registers, none);
//   * CTAs per SM actually launched: the variant's occupancy or one fewer;
//   * rings summed in registers before a shared-memory flush: 4, 8 or 16.
// Each candidate runs the pass on a sample of pivots (slices at three latitudes, about
// 0.5% of a large map, the whole map when it is small), once to warm up and then twice
// timed with CUDA events; the fastest is kept in the plan.  Results are cached in the
// text file named by TPCF_AUTOTUNE_CACHE, keyed by the device, the map resolution, the
// bins and the flags, and plans read that file when they are created.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "plan.cuh"

using namespace tpcf;

namespace tpcf {
int map_fwd_occupancy(int M, int K, int self, int variant);
int map_bwd_occupancy(int M, int K, int variant);

static std::string tune_key(const tpcf_plan_s* P) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, P->device) != cudaSuccess) prop.name[0] = 0;
    unsigned long long h = 1469598103934665603ull;  // FNV-1a over the edge bits
    for (double e : P->edges) {
        unsigned long long b;
        memcpy(&b, &e, sizeof(b));
        for (int i = 0; i < 8; ++i) {
            h ^= (b >> (8 * i)) & 0xff;
            h *= 1099511628211ull;
        }
    }
    char buf[320];
    std::string name(prop.name);
    for (char& c : name)
        if (c == ' ') c = '_';
    snprintf(buf, sizeof(buf), "v2 dev=%s sms=%d map nside=%d K=%d M=%d flags=%u edges=%016llx", name.c_str(),
             P->num_sms, P->map.nside, P->K, P->M, P->flags, h);
    return buf;
}

// Reads the cache; returns true and fills the configuration if the key is present.
static bool cache_lookup(const std::string& key, tpcf_plan_s::Tune* f, tpcf_plan_s::Tune* b) {
    const char* path = getenv("TPCF_AUTOTUNE_CACHE");
    if (!path || !*path) return false;
    FILE* fp = fopen(path, "r");
    if (!fp) return false;
    char line[512];
    bool found = false;
    while (fgets(line, sizeof(line), fp)) {
        const size_t n = key.size();
        if (strncmp(line, key.c_str(), n) != 0 || line[n] != '|') continue;
        tpcf_plan_s::Tune tf, tb;
        if (sscanf(line + n + 1, " fwd %d %d %d %d bwd %d %d %d", &tf.variant, &tf.ctas, &tf.flush, &tf.quad,
                   &tb.variant, &tb.ctas, &tb.flush) == 7) {
            *f = tf;
            *b = tb;
            found = true;  // the last matching line wins
        }
    }
    fclose(fp);
    return found;
}

static void cache_store(const std::string& key, const tpcf_plan_s::Tune& f, const tpcf_plan_s::Tune& b) {
    const char* path = getenv("TPCF_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE* fp = fopen(path, "a");
    if (!fp) return;
    fprintf(fp, "%s| fwd %d %d %d %d bwd %d %d %d\n", key.c_str(), f.variant, f.ctas, f.flush, f.quad, b.variant,
            b.ctas, b.flush);
    fclose(fp);
}

static bool valid(const tpcf_plan_s* P, const tpcf_plan_s::Tune& t, bool bwd) {
    if (t.variant != 2 && t.variant != 3) return false;
    if (t.flush < 1 || t.flush > 64 || t.ctas < 1 || t.quad < 0 || t.quad > 1) return false;
    const int self = (P->flags & TPCF_SELF_PAIRS_SUBTRACT) ? 1 : 0;
    const int occ = bwd ? map_bwd_occupancy(P->M, P->K, t.variant) : map_fwd_occupancy(P->M, P->K, self, t.variant);
    return t.ctas <= occ;
}

// Applies a cached configuration to a new map plan (called at plan creation).
void tune_from_cache(tpcf_plan_s* P) {
    if (P->kind != PLAN_MAP || (P->flags & TPCF_CONTRACT_TC)) return;
    tpcf_plan_s::Tune f, b;
    if (!cache_lookup(tune_key(P), &f, &b)) return;
    if (!valid(P, f, false) || !valid(P, b, true)) return;
    P->tune_fwd = f;
    P->tune_bwd = b;
    P->tuned = true;
}
}  // namespace tpcf

// 1-based ring of a given z in the north half, for the sample slices.
static int64_t first_pixel_of_ring(int64_t nside, int64_t r) {
    if (r < nside) return 2 * r * (r - 1);
    return 2 * nside * (nside - 1) + 4 * nside * (r - nside);
}

extern "C" tpcf_status tpcf_plan_autotune(tpcf_plan plan, const float* d_delta, const float* d_w, int32_t passes,
                                          void* stream) {
    if (!plan || !d_delta || !d_w || passes < 1 || passes > 3) return TPCF_ERR_INVALID_ARG;
    tpcf_plan_s* P = plan;
    if (P->kind != PLAN_MAP || (P->flags & TPCF_CONTRACT_TC)) {
        set_error("tpcf_plan_autotune: map plans with the FP32 contraction only");
        return TPCF_ERR_UNSUPPORTED;
    }
    if (P->flags & NORM_FLAGS) passes &= 1;  // no adjoint for these plans
    const std::string key = tune_key(P);
    {
        tpcf_plan_s::Tune f, b;
        if (cache_lookup(key, &f, &b) && valid(P, f, false) && valid(P, b, true)) {
            P->tune_fwd = f;
            P->tune_bwd = b;
            P->tuned = true;
            return TPCF_OK;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nside = P->map.nside, npix = P->npoints;
    // sample: the whole map when small, else three slices at z ~ 0.85, 0.45, 0.05 of
    // together at least ~1/200 of the map and 3 x 64 tiles per SM, so that every
    // candidate keeps the GPU busy for several waves of tiles
    std::vector<std::pair<int64_t, int64_t>> sample;
    const int64_t min_slice = (int64_t)P->num_sms * 64 * TILE;
    if (npix <= 3 * min_slice) {
        sample.push_back({0, npix});
    } else {
        const int64_t len = std::max<int64_t>(min_slice, npix / 600);
        const double zs[3] = {0.85, 0.45, 0.05};
        for (double z : zs) {
            // ring index of colatitude acos(z): cap rings r < nside have z = 1 - r^2/(3 nside^2)
            int64_t r = z > 2.0 / 3.0 ? (int64_t)(nside * sqrt(3.0 * (1.0 - z))) : (int64_t)(nside * (2.0 - 1.5 * z));
            r = std::max<int64_t>(1, std::min<int64_t>(r, 2 * nside));
            const int64_t a = first_pixel_of_ring(nside, r);
            sample.push_back({a, std::min<int64_t>(npix, a + len)});
        }
    }
    const int K = P->K, M = P->M;
    const size_t nz = (size_t)(M + 1) * K * K * 2;
    double *zeta = nullptr, *norm = nullptr, *dL = nullptr;
    float* grad = nullptr;
    tpcf_status st = TPCF_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto fail = [&](cudaError_t e, const char* where) {
        st = cuda_fail(e, where);
        return st;
    };
    cudaError_t ce;
    if ((ce = dev_malloc((void**)&zeta, nz * sizeof(double))) != cudaSuccess ||
        (ce = dev_malloc((void**)&norm, (size_t)K * K * sizeof(double))) != cudaSuccess ||
        (ce = dev_malloc((void**)&dL, nz * sizeof(double))) != cudaSuccess ||
        ((passes & 2) && (ce = dev_malloc((void**)&grad, (size_t)npix * sizeof(float))) != cudaSuccess) ||
        (ce = cudaEventCreate(&e0)) != cudaSuccess || (ce = cudaEventCreate(&e1)) != cudaSuccess) {
        fail(ce, "tpcf_plan_autotune scratch");
    }
    if (st == TPCF_OK) {
        std::vector<double> ones(nz, 1.0);
        if ((ce = cudaMemcpy(dL, ones.data(), nz * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
            fail(ce, "tpcf_plan_autotune dL");
    }
    // the adjoint candidates take the normalisation D of the first sample slice
    if (st == TPCF_OK && (passes & 2))
        st = tpcf_forward(P, d_delta, d_w, sample[0].first, sample[0].second, zeta, norm, nullptr, s);
    const int self = (P->flags & TPCF_SELF_PAIRS_SUBTRACT) ? 1 : 0;
    for (int pass = 0; pass < 2 && st == TPCF_OK; ++pass) {
        if (!(passes & (1 << pass))) continue;
        const bool bwd = pass == 1;
        tpcf_plan_s::Tune& T = bwd ? P->tune_bwd : P->tune_fwd;
        const tpcf_plan_s::Tune keep = T;
        tpcf_plan_s::Tune best = keep;
        float best_ms = 1e30f;
        // times the configuration in T (the first of three runs warms up) and keeps the best
        auto try_config = [&]() {
            float ms = 1e30f;
            for (int rep = 0; rep < 3 && st == TPCF_OK; ++rep) {
                cudaEventRecord(e0, s);
                for (auto& sl : sample) {
                    st = bwd ? tpcf_backward(P, d_delta, d_w, sl.first, sl.second, norm, dL, grad, s)
                             : tpcf_forward(P, d_delta, d_w, sl.first, sl.second, zeta, norm, nullptr, s);
                    if (st != TPCF_OK) break;
                }
                cudaEventRecord(e1, s);
                if ((ce = cudaEventSynchronize(e1)) != cudaSuccess) {
                    fail(ce, "tpcf_plan_autotune timing");
                    break;
                }
                float t = 0.0f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0) ms = std::min(ms, t);
            }
            if (st == TPCF_OK && ms < best_ms) {
                best_ms = ms;
                best = T;
            }
        };
        for (int variant = 3; variant >= 2 && st == TPCF_OK; --variant) {
            const int occ = bwd ? map_bwd_occupancy(M, K, variant) : map_fwd_occupancy(M, K, self, variant);
            for (int ctas = occ; ctas >= std::max(1, occ - 1) && st == TPCF_OK; --ctas) {
                const int flushes[4] = {4, 8, 16, 32};
                for (int fi = 0; fi < 4 && st == TPCF_OK; ++fi) {
                    T.variant = variant;
                    T.ctas = ctas;
                    T.flush = flushes[fi];
                    try_config();
                }
            }
        }
        if (!bwd && st == TPCF_OK) {  // the forward's tile layout, at the best shape
            T = best;
            T.quad = 1 - best.quad;
            try_config();
        }
        T = st == TPCF_OK ? best : keep;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    dev_free(zeta);
    dev_free(norm);
    dev_free(dL);
    dev_free(grad);
    if (st != TPCF_OK) return st;
    if ((passes & 3) == 3) {
        P->tuned = true;
        cache_store(key, P->tune_fwd, P->tune_bwd);
    }
    return tpcf_plan_sync(P);
}

extern "C" tpcf_status tpcf_plan_launch_config(tpcf_plan plan, int32_t* out7) {
    if (!plan || !out7) return TPCF_ERR_INVALID_ARG;
    const tpcf_plan_s* P = plan;
    out7[0] = P->tune_fwd.variant;
    out7[1] = P->tune_fwd.ctas;
    out7[2] = P->tune_fwd.flush;
    out7[3] = P->tune_fwd.quad;
    out7[4] = P->tune_bwd.variant;
    out7[5] = P->tune_bwd.ctas;
    out7[6] = P->tune_bwd.flush;
    return TPCF_OK;
}

extern "C" tpcf_status tpcf_plan_set_launch_config(tpcf_plan plan, const int32_t* in7) {
    if (!plan || !in7) return TPCF_ERR_INVALID_ARG;
    tpcf_plan_s* P = plan;
    if (P->kind != PLAN_MAP || (P->flags & TPCF_CONTRACT_TC)) return TPCF_ERR_UNSUPPORTED;
    tpcf_plan_s::Tune f{in7[0], in7[1], in7[2], in7[3]}, b{in7[4], in7[5], in7[6], 0};
    if (!valid(P, f, false) || !valid(P, b, true)) return TPCF_ERR_INVALID_ARG;
    P->tune_fwd = f;
    P->tune_bwd = b;
    return TPCF_OK;
}
