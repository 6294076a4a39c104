// Small per-call kernels: input packing, the cross-CTA FP64 reduction of the
// partial sums, normalisation (zeta = S / D) and the adjoint's coefficient prep.
#include "geometry.cuh"

namespace tpcf {

// (w d, w) per point, so the pair loops read one 8-byte word per neighbour.
__global__ void pack_kernel(const float* __restrict__ delta, const float* __restrict__ w, float2* wdw,
                            int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float wi = w[i];
        wdw[i] = make_float2(wi * delta[i], wi);
    }
}

__global__ void zero_f32_kernel(float* p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 0.0f;
}

// sums[e] = sum over CTA slots of slots[s * nent + e], in FP64.
__global__ void reduce_slots_kernel(const double* __restrict__ slots, int nslots, int nent, double* sums) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nent) return;
    double acc = 0.0;
    for (int s = 0; s < nslots; ++s) acc += slots[(size_t)s * nent + e];
    sums[e] = acc;
}

// zeta_m(k1,k2) = S_m(k1,k2) / (scale * D(k1,k2)), Hermitian fill of the lower triangle,
// zeta = 0 where D = 0.  With self-pair subtraction the diagonal loses
// sum_i w_i d_i Q^k(i) (every m) and D loses sum_i w_i QW^k(i).  One output entry
// idx = (m, k1, k2) per call.
__device__ __forceinline__ void finalize_one(const double* __restrict__ sums, int K, int M, int self_subtract,
                                             double scale, double* zeta, double* norm, double* raw, int idx) {
    const int P = K * (K + 1) / 2;
    const int nS = (M + 1) * P;
    const int m = idx / (K * K);
    const int rem = idx - m * K * K;
    const int k1 = rem / K, k2 = rem - k1 * K;
    const int a = min(k1, k2), b = max(k1, k2);
    const int pidx = b * (b + 1) / 2 + a;
    double sr = sums[2 * (m * P + pidx)];
    double si = sums[2 * (m * P + pidx) + 1];
    double d = sums[2 * nS + pidx];
    if (self_subtract && k1 == k2) {
        sr -= sums[2 * nS + P + k1];
        d -= sums[2 * nS + P + K + k1];
    }
    if (k1 > k2) si = -si;  // S(k2,k1) = conj(S(k1,k2))
    d *= scale;
    double zr = 0.0, zi = 0.0;
    if (d != 0.0) {
        zr = sr / d;
        zi = si / d;
    }
    zeta[2 * idx] = zr;
    zeta[2 * idx + 1] = zi;
    if (raw) {
        raw[2 * idx] = sr;
        raw[2 * idx + 1] = si;
    }
    if (m == 0) norm[rem] = d;
}

// Multi-field estimate: zeta_m(k1,k2) = S_m(k1,k2) / D(k1,k2) over full K x K sums
// (no Hermitian fill: the cyclic three-field sums are not Hermitian); zeta = 0 where
// D = 0.  One output entry idx = (m, k1, k2) per thread.
__global__ void finalize_full_kernel(const double* __restrict__ sums, int K, int M, double* zeta, double* norm,
                                     double* raw) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int KK = K * K, nS = (M + 1) * KK;
    if (idx >= nS) return;
    const int r = idx % KK;
    const double D = sums[2 * nS + r];
    const double sr = sums[2 * idx], si = sums[2 * idx + 1];
    zeta[2 * idx] = D != 0.0 ? sr / D : 0.0;
    zeta[2 * idx + 1] = D != 0.0 ? si / D : 0.0;
    if (raw) {
        raw[2 * idx] = sr;
        raw[2 * idx + 1] = si;
    }
    if (idx < KK) norm[idx] = D;
}

__global__ void finalize_kernel(const double* __restrict__ sums, int K, int M, int self_subtract,
                                double scale, double* zeta, double* norm, double* raw) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (M + 1) * K * K) return;
    finalize_one(sums, K, M, self_subtract, scale, zeta, norm, raw, idx);
}

// H_m(k,k') = conj(C_m(k,k')) + C_m(k',k),  C = (dL/dRe zeta + i dL/dIm zeta) / D.
__device__ __forceinline__ void adjoint_prep_one(const double* __restrict__ dL, const double* __restrict__ norm,
                                                 int K, float* H, int idx) {
    const int m = idx / (K * K);
    const int rem = idx - m * K * K;
    const int k = rem / K, kp = rem - k * K;
    const int t = m * K * K + kp * K + k;  // (k', k)
    const double d1 = norm[k * K + kp], d2 = norm[kp * K + k];
    double c1r = 0.0, c1i = 0.0, c2r = 0.0, c2i = 0.0;
    if (d1 != 0.0) {
        c1r = dL[2 * idx] / d1;
        c1i = dL[2 * idx + 1] / d1;
    }
    if (d2 != 0.0) {
        c2r = dL[2 * t] / d2;
        c2i = dL[2 * t + 1] / d2;
    }
    H[2 * idx] = (float)(c1r + c2r);
    H[2 * idx + 1] = (float)(-c1i + c2i);
}

// With self-pair subtraction H is followed by cdiag_k = sum_m Re dL_m(k,k) / D(k,k)
// (the subtracted diagonal enters every m with the same real weight).
__global__ void adjoint_prep_kernel(const double* __restrict__ dL, const double* __restrict__ norm, int K,
                                    int M, float* H, int with_diag) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (M + 1) * K * K) return;
    adjoint_prep_one(dL, norm, K, H, idx);
    if (with_diag && idx < K) {
        const double d = norm[idx * K + idx];
        double t = 0.0;
        if (d != 0.0)
            for (int m = 0; m <= M; ++m) t += dL[2 * ((size_t)m * K * K + (size_t)idx * K + idx)] / d;
        H[(size_t)(M + 1) * K * K * 2 + idx] = (float)t;
    }
}

// ------------------------------------------------------------------ batches
// The batched forms run the same per-entry work for every plan of a batch at once:
// blockIdx.y selects the plan, blockIdx.x strides over its entries.

__global__ void batch_pack_kernel(const BatchIO* __restrict__ io) {
    const BatchIO& b = io[blockIdx.y];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b.npix;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float wi = b.w[i];
        b.wdw[i] = make_float2(wi * b.delta[i], wi);
    }
}

// Zeroes each plan's CTA slots and, when `with_grad`, its gradient.
__global__ void batch_zero_kernel(const BatchIO* __restrict__ io, int with_grad) {
    const BatchIO& b = io[blockIdx.y];
    const int64_t ns = (int64_t)b.nslots * b.nent;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns;
         i += (int64_t)gridDim.x * blockDim.x)
        b.slots[i] = 0.0;
    if (with_grad)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b.npix;
             i += (int64_t)gridDim.x * blockDim.x)
            b.grad[i] = 0.0f;
}

__global__ void batch_reduce_kernel(const BatchIO* __restrict__ io) {
    const BatchIO& b = io[blockIdx.y];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < b.nent; e += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int s = 0; s < b.nslots; ++s) acc += b.slots[(size_t)s * b.nent + e];
        b.sums[e] = acc;
    }
}

__global__ void batch_finalize_kernel(const BatchIO* __restrict__ io) {
    const BatchIO& b = io[blockIdx.y];
    const int nout = (b.M + 1) * b.K * b.K;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nout; idx += gridDim.x * blockDim.x)
        finalize_one(b.sums, b.K, b.M, b.self_subtract, 1.0, b.zeta, b.norm, nullptr, idx);
}

__global__ void batch_adjoint_prep_kernel(const BatchIO* __restrict__ io) {
    const BatchIO& b = io[blockIdx.y];
    const int nout = (b.M + 1) * b.K * b.K;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nout; idx += gridDim.x * blockDim.x)
        adjoint_prep_one(b.dL, b.norm, b.K, b.H, idx);
}

}  // namespace tpcf
