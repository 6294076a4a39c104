// Declarations of the plan-build and small per-call kernels.
#pragma once

#include "tpcf_internal.cuh"

namespace tpcf {

__global__ void ring_table_kernel(int nside, int nrings, int64_t* first, int* npr, int* shift, double* z,
                                  double* s, double* th, float* zf, float* sf, float* sf_lo, float* step,
                                  float* step_lo, float* invn, float* invn_lo);
__global__ void ring_range_kernel(int nrings, int K, const double* th, const double* E, const int* npr,
                                  int2* ring_range, int2* bin_range, int64_t* npairs, int64_t* ntiles);
__global__ void exclusive_scan_kernel(const int64_t* in, int64_t* out, int n, int64_t* total);
__global__ void pair_table_kernel(int nrings, int K, const int64_t* pair_off, int64_t npairs,
                                  const int2* ring_range, const double* th, const double* s, const int* npr,
                                  const double* E, float2* pair_A, int2* pair_T);
__global__ void tile_list_kernel(int nrings, const int64_t* tile_off, const int64_t* ntiles_ring, int2* tiles);
__global__ void edges_kernel(int K, const double* theta, double* E);

// small per-call kernels (small_kernels.cu)
__global__ void pack_kernel(const float* delta, const float* w, float2* wdw, int64_t n);
__global__ void reduce_slots_kernel(const double* slots, int nslots, int nent, double* sums);
__global__ void finalize_kernel(const double* sums, int K, int M, int self_subtract, double scale,
                                double* zeta, double* norm, double* raw);
__global__ void finalize_full_kernel(const double* sums, int K, int M, double* zeta, double* norm, double* raw);
__global__ void adjoint_prep_kernel(const double* dL_dzeta, const double* norm, int K, int M, float* H,
                                    int with_diag);
__global__ void zero_f32_kernel(float* p, int64_t n);

// Per-plan arguments of the batched small kernels (device-resident array, one entry
// per plan of a batch).
struct BatchIO {
    const float* delta;
    const float* w;
    float2* wdw;
    int64_t npix;
    double* slots;  // nslots x nent
    int nslots, nent;
    double* sums;   // nent
    int K, M, self_subtract;
    double* zeta;
    double* norm;
    const double* dL;  // NULL without adjoint
    float* H;
    float* grad;       // NULL without adjoint
};
__global__ void batch_pack_kernel(const BatchIO* io);
__global__ void batch_zero_kernel(const BatchIO* io, int with_grad);
__global__ void batch_reduce_kernel(const BatchIO* io);
__global__ void batch_finalize_kernel(const BatchIO* io);
__global__ void batch_adjoint_prep_kernel(const BatchIO* io);

}  // namespace tpcf
