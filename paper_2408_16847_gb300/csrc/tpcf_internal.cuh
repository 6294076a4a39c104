// Internal declarations shared by the translation units of libtpcf.
// Device views of plans, launch argument blocks and the per-M launcher table.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tpcf.h"

namespace tpcf {

constexpr int TILE = 32;     // pivots per tile: one pivot per lane
constexpr int NWARPS = 8;    // warps per CTA; they split the neighbour rings of a tile
constexpr int NTHREADS = TILE * NWARPS;

// Threshold encoding of pair_T entries (see geometry.cu).
constexpr int T_ZERO = -1;          // every pixel of ring r is at or beyond the edge
constexpr int T_INF = 0x7fffffff;   // every pixel of ring r is inside the edge

// Read-only device view of a map plan (kernels take it by value).
struct MapDev {
    int nside, nrings, K, M;
    int64_t npix;
    const int64_t* ring_first;  // [nrings] first pixel of ring
    const int* ring_n;          // [nrings] pixels in ring (always even)
    const int* ring_shift;      // [nrings] pixel p of the ring sits at phi = pi (2p + shift) / n
    const float* ring_zf;       // [nrings] cos(colatitude), fp32
    const float* ring_sf;       // [nrings] sin(colatitude), fp32 (rounded)
    const float* ring_sf_lo;    // [nrings] sin(colatitude) - ring_sf
    const float* ring_step;     // [nrings] pi / n (half longitude step), fp32
    const float* ring_step_lo;  // [nrings] pi / n - ring_step
    const float* ring_invn;     // [nrings] 1 / n, fp32
    const float* ring_invn_lo;  // [nrings] 1 / n - ring_invn
    const double* ring_th;      // [nrings] colatitude, fp64
    const double* ring_s;       // [nrings] sin(colatitude), fp64
    const int2* ring_range;     // [nrings] neighbour rings (rlo, rhi) of pivot ring i
    const int2* bin_range;      // [nrings * K] rings of pivot ring i that may hold bin-k pixels
    const int64_t* pair_off;    // [nrings] first (i, r) pair index of pivot ring i
    const float2* pair_A;       // [npairs] sin(theta_i - theta_r) as fp32 (hi, lo) from fp64
    const int2* pair_T;         // [npairs * (K+1)] edge offsets T_e in ring-r pixels
    const int2* tiles;          // [ntiles] (ring, first pivot index in ring)
    int64_t ntiles;
    const double* E;            // [K+1] sin^2(theta_e / 2)
};

// Read-only device view of a catalogue plan: the points sorted into a sphere grid
// of colatitude bands, each cut into equal longitude sectors (cells).  Points of a
// cell are contiguous, cells are ordered band by band, sectors by longitude.
constexpr int CAT_LUT = 512;  // entries of the bin lookup table (uniform in log2 chord^2)
struct CatDev {
    int64_t n;
    int K, M;
    const float4* p_hi;          // [n] sorted unit vectors, fp32 part (x, y, z, 0)
    const float4* p_lo;          // [n] fp64 - fp32 remainders (x, y, z), w = sorted index bits
    const double* xyz;           // [3n] sorted unit vectors, fp64
    const int64_t* orig;         // [n] caller's index of each sorted point
    const int64_t* cell_start;   // [ncells + 1] first sorted point of each cell
    const int64_t* band_first;   // [nbands + 1] first cell of each band
    const int64_t* band_ns;      // [nbands] sectors in each band
    int nbands;
    double hband;                // band height (rad)
    double theta_max;            // outer bin edge (rad)
    const float* E2;             // [K+1] chord^2 of the edges, fp32
    const double* Ed2;           // [K+1] chord^2 of the edges, fp64
    const unsigned char* lut;    // [CAT_LUT] bin at the lower end of each table cell
    float lut_l0, lut_inv;       // table origin log2(E2[0]) and entries per unit of log2
    int64_t ntiles;              // ceil(n / TILE)
};

// Per-call arguments of the map kernels.
struct MapCall {
    const float2* wdw;      // [npix] (w * delta, w)
    const float* delta;     // [npix] caller's delta (kernels that read it directly)
    const float* w;         // [npix] caller's weights (idem)
    int64_t piv_lo, piv_hi; // pivot pixel range
    double* slots;          // [grid * nentries] per-CTA fp64 partial sums
    int* counter;           // work counter (zeroed before launch)
    int* status;            // latched device error flags
    const float* H;         // backward: [(M+1) * K * K * 2] fp32, conj(C(k,k')) + C(k',k)
    float* grad;            // backward: [npix]
    int self_subtract;      // subtract the j = k self term
    int flush;              // rings summed in registers before a shared-memory flush (tuned)
    int64_t tile_lo, tile_hi;  // tiles that can hold a pivot of [piv_lo, piv_hi)
    int norm;               // NORM_*: per-pivot normalisation of the moments before the contraction
    int quad;               // forward tiles in the quarter-turn layout (tile_pivot)
    int group;              // > 1: shared neighbour lists, one lane per run of `group` ring pixels
    const int2* gtiles;     // group > 1: tiles (ring, first run of the tile)
};

// One plan of a batch (device-resident): its geometry, its per-call arguments and
// the index of its first tile in the batch's concatenated work queue.
// Per-pivot normalisation of the moments (MapCall::norm): none (zeta = S / D), each
// bin by its own weight W^k(i), or every bin by the pivot's total sum_k W^k(i).
constexpr int NORM_NONE = 0;
constexpr int NORM_BIN_MEAN = 1;
constexpr int NORM_PIVOT_TOTAL = 2;
constexpr uint32_t NORM_FLAGS = TPCF_NORM_BIN_MEAN | TPCF_NORM_PIVOT_TOTAL;
inline int norm_of_flags(uint32_t flags) {
    return (flags & TPCF_NORM_BIN_MEAN) ? NORM_BIN_MEAN : ((flags & TPCF_NORM_PIVOT_TOTAL) ? NORM_PIVOT_TOTAL : NORM_NONE);
}

constexpr int TPCF_MAX_BATCH = 256;
struct BatchItem {
    MapDev g;
    MapCall c;
    long long tile0;
};

// Entries of the per-tile partial sums: S for k1 <= k2 (complex), then D (k1 <= k2),
// then, with self-pair subtraction, the two diagonals sum w d Q and sum w QW.
inline __host__ __device__ int n_pairs_tri(int K) { return K * (K + 1) / 2; }
inline __host__ __device__ int n_entries(int K, int M) {
    return 2 * (M + 1) * n_pairs_tri(K) + n_pairs_tri(K) + 2 * K;
}
// Entries of the multi-field partial sums: full K x K matrices, S (complex) per m, then D.
inline __host__ __device__ int n_entries_multi(int K, int M) { return 2 * (M + 1) * K * K + K * K; }

constexpr int ROW = 512;  // floats per warp row buffer of the adjoint (wider rows: whole-ring or global adds)

// Shared memory (floats) of a map forward tile with runtime m_max mr: moments
// A[k][m][re/im][32], W, Q, QW [k][32], the pivots' (w d, w).
__host__ __device__ inline size_t tile_floats_rt(int K, int mr) {
    return (size_t)K * (mr + 1) * 2 * TILE + 3 * (size_t)K * TILE + 2 * TILE;
}

// Shared memory (floats) of a map adjoint tile: phases 1-2 use the moments, W, Q, QW,
// the pivots, the primary-term sums and one m of H; phase 3 keeps the moments (then
// h) and the warps' row buffers.
__host__ __device__ inline size_t bwd_tile_floats_rt(int K, int mr) {
    const size_t a = (size_t)K * (mr + 1) * 2 * TILE;
    const size_t p12 = a + 3 * (size_t)K * TILE + 2 * TILE + TILE + (size_t)K * K * 2;
    const size_t p3 = a + (size_t)NWARPS * ROW;
    return p12 > p3 ? p12 : p3;
}

// Device status bits.
constexpr int ST_BAD_TILE = 1;
constexpr int ST_ROW_OVERFLOW = 2;   // informational: a row wider than the warp buffer used direct global adds
constexpr int ST_TC_TIMEOUT_BIT = 4;  // a tensor-core completion wait gave up

}  // namespace tpcf
