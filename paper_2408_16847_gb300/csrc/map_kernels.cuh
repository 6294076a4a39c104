// Map-path kernels of the binned harmonic 3PCF estimator (arXiv:2408.16847,
// section 3.1), templated on the largest multipole M.  Included by map_inst.cu,
// which is compiled once per M.
//
// Work decomposition (forward):
//   * a tile is 32 consecutive pivots of one HEALPix ring, one pivot per lane;
//   * a CTA of 8 warps owns one tile at a time (persistent CTAs, 3 per SM, pull
//     tiles from an atomic counter); for every radial bin k the warps split the
//     neighbour rings that can hold bin-k pixels;
//   * on a neighbour ring the bin-k pixels of a pivot form at most two contiguous
//     runs, found from the per-ring-pair edge offsets T_e built by the plan (an
//     exact ring-range disc query); each lane walks its own runs, so the bin is
//     known without a per-pixel test and the (M+1) complex accumulators of the bin
//     stay in registers across rings;
//   * within a run e^{-i m phi} comes from a trig-free recurrence in m (the harmonic
//     step the paper describes in Sec. 3.1 and 3.2, a few operations per m): Reinsch's
//     stable form of the three-term relation on the angle folded into |psi| <= pi/2,
//     with the neighbour weight folded into the start values and the cos and sin
//     chains packed into f32x2 FMAs (see harmonics());
//   * in the equatorial belt a neighbour ring has as many pixels as the pivot ring,
//     so its pixels sit symmetrically about the pivot's meridian: the pixel at +phi
//     and its mirror at -phi share one cos/sin evaluation and one recurrence;
//   * after all bins, the tile's a_m^k(i) sit in shared memory and the CTA forms
//     sum_i w_i d_i a^{k1} conj(a^{k2}) (eq. zetamEst2) and sum_i w_i W^{k1} W^{k2},
//     adding them in FP64 into a slot owned by the CTA (FP32 pipe, or the tensor
//     cores in map_fwd_tc_kernel).
#pragma once

#include <math.h>

#include "tpcf_internal.cuh"

namespace tpcf {

constexpr float AMBIGUITY = 1.0e-6f;  // > worst fp32 error of the edge position (~1.5e-7 px)
constexpr float FAST_XMAX = 0.25f;    // |half longitude offset| covered by the polynomial
constexpr int FLUSH_RINGS = 8;        // default rings summed in registers before a shared-memory flush

// Fire-and-forget FP64 reduction of an fp32 partial sum into a CTA slot.  The float
// is widened by moving its IEEE 754 fields (exponent re-biased by 1023 - 127 = 896,
// mantissa shifted up by 52 - 23 = 29 bits), an exact conversion on the integer pipe:
// the FP64 pipe of this part runs at a few percent of the FP32 rate, and one
// conversion per slot entry and tile kept it half busy on small tiles.  Zeros add
// nothing and are skipped; subnormal, infinite and NaN values take the ordinary
// conversion.
__device__ __forceinline__ void red_add_f32(double* p, float x) {
    const unsigned u = __float_as_uint(x);
    if ((u & 0x7fffffffu) == 0u) return;
    const unsigned e = (u >> 23) & 0xffu;
    double d;
    if (e == 0u || e == 0xffu) {
        d = (double)x;
    } else {
        d = __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) |
                                             ((unsigned long long)(e + 896u) << 52) |
                                             ((unsigned long long)(u & 0x7fffffu) << 29)));
    }
    atomicAdd(p, d);  // result unused: a reduction, no wait
}

__device__ __forceinline__ long long floordiv_ll(long long a, long long b) {
    long long q = a / b;
    if ((a % b) != 0 && a < 0) --q;
    return q;
}

// Position of the lane's pivot in units of ring-r pixels: c = cint + crem / den,
// so that pixel p of ring r is at longitude offset o = p - c pixels from the pivot.
struct LaneC {
    int cint, crem, den;
    float cfrac;
};

// floor(num / den) from an fp32 estimate corrected in exact integer arithmetic (the
// estimate is within one of the true quotient for the sizes used here).
__device__ __forceinline__ LaneC lane_c(int q, int s_i, int n_i, int s_r, int n_r) {
    if (n_r == n_i) {  // same pixel count: c = q + (s_i - s_r) / 2, no division
        LaneC c;
        const int d = s_i - s_r;  // -1, 0 or 1
        c.cint = q + (d < 0 ? -1 : 0);
        c.crem = d != 0 ? n_i : 0;
        c.den = 2 * n_i;
        c.cfrac = d != 0 ? 0.5f : 0.0f;
        return c;
    }
    const long long num = (long long)n_r * (2LL * q + s_i) - (long long)s_r * n_i;
    const int den = 2 * n_i;
    int ci = (int)floorf(__fdividef((float)num, (float)den));
    long long rem = num - (long long)ci * den;
    if (rem < 0) {
        --ci;
        rem += den;
    } else if (rem >= den) {
        ++ci;
        rem -= den;
    }
    LaneC c;
    c.cint = ci;
    c.crem = (int)rem;
    c.den = den;
    c.cfrac = __fdiv_rn((float)c.crem, (float)den);
    return c;
}

// Exact (FP64) quarter squared chord of pixel p of ring r about the pivot:
// f = sin^2((theta_r - theta_i)/2) + s_i s_r sin^2(pi o / n_r).  Only evaluated for
// the rare edge pixels whose fp32 position is ambiguous, so the context holds the
// raw ring values and the FP64 trigonometry runs inside the rare branch.
struct ExactCtx {
    double th_i, th_r, s_i, s_r;
    int n_r;
};

static __device__ __noinline__ double exact_f(double th_i, double th_r, double s_i, double s_r, int n_r,
                                              int cint, int crem, int den, int p) {
    const double h = sin(0.5 * (th_r - th_i));
    const double o = (double)(p - cint) - (double)crem / (double)den;
    const double sp = sinpi(o / (double)n_r);
    return h * h + (s_i * s_r) * sp * sp;
}

// First pixel p (unwrapped index) with p - c >= T (T finite, positive).
__device__ __forceinline__ int pos_edge(const LaneC& c, int2 T, double Ee, const ExactCtx& x) {
    const float y = c.cfrac + __int_as_float(T.y);
    const float ry = rintf(y);
    const int base = c.cint + T.x;
    if (fabsf(y - ry) > AMBIGUITY) return base + (int)ceilf(y);
    const int ps = base + (int)ry;
    return (exact_f(x.th_i, x.th_r, x.s_i, x.s_r, x.n_r, c.cint, c.crem, c.den, ps) >= Ee) ? ps : ps + 1;
}

// Last pixel p with p - c <= -T.
__device__ __forceinline__ int neg_edge(const LaneC& c, int2 T, double Ee, const ExactCtx& x) {
    const float y = c.cfrac - __int_as_float(T.y);
    const float ry = rintf(y);
    const int base = c.cint - T.x;
    if (fabsf(y - ry) > AMBIGUITY) return base + (int)floorf(y);
    const int ps = base + (int)ry;
    return (exact_f(x.th_i, x.th_r, x.s_i, x.s_r, x.n_r, c.cint, c.crem, c.den, ps) >= Ee) ? ps : ps - 1;
}

// Warp-uniform description of neighbour ring r for pivot ring i.
struct RingCtx {
    long long first;
    int n, shift;
    float s_r, s_lo;      // sin(colatitude of r) as an unevaluated fp32 sum s_r + s_lo
    float A, A_lo;        // sin(theta_i - theta_r), likewise
    float B;              // 2 cos(theta_i) sin(theta_r)
    float step, step_lo;  // pi / n (half longitude step) as fp32 hi + lo
    float inv_n, invn_lo; // 1 / n likewise
};

// sin x and cos x for |x| <= FAST_XMAX from their Taylor series (truncation error
// below 2e-11 relative at the end of the range).
__device__ __forceinline__ void sin_cos_series(float x, float& s, float& c) {
    const float x2 = x * x;
    s = x * fmaf(x2, fmaf(x2, fmaf(x2, -1.98412698e-4f, 8.33333333e-3f), -1.66666667e-1f), 1.0f);
    c = fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, 2.48015873e-5f, -1.38888889e-3f), 4.16666667e-2f), -0.5f),
             1.0f);
}

// Direction (cos phi, sin phi) of a neighbour at longitude offset o (ring-r pixels):
// with x = pi o / n (half the longitude difference),
//   east  component  E = s_r sin(2x)
//   north component  N = sin(theta_i - theta_r) + 2 cos(theta_i) s_r sin^2 x,
// the cancellation-free form of n_j . e_N(i); phi is measured from north to east.
// The per-ring constants carry a second fp32 word: their single-fp32 rounding is the
// same for every pixel of a ring and would shift phi coherently ring by ring.  The
// offset o = fi - cfrac is passed as its integer part fi (exact in fp32) and the run
// constants xneg = -cfrac pi/n, uneg = -cfrac/n, so x = pi o / n has one rounding.
template <bool FAST>
__device__ __forceinline__ void pixel_dir(float fi, float xneg, float uneg, const RingCtx& R, float& cph,
                                          float& sph) {
    float sx, cx;
    if (FAST) {
        sin_cos_series(fmaf(fi, R.step, fmaf(fi, R.step_lo, xneg)), sx, cx);
    } else {
        sincospif(fmaf(fi, R.inv_n, fmaf(fi, R.invn_lo, uneg)), &sx, &cx);
    }
    const float s2x = 2.0f * sx * cx;
    const float E = fmaf(R.s_r, s2x, R.s_lo * s2x);
    const float N = fmaf(R.B, sx * sx, R.A_lo) + R.A;
    // the floor only matters for the masked-out iterations of a run (zero weight),
    // which may sit on the pivot itself; real neighbours have N^2 + E^2 = sin^2 theta.
    const float rinv = rsqrtf(fmaxf(fmaf(N, N, E * E), 1e-30f));
    cph = N * rinv;
    sph = E * rinv;
}

// e^{-i m phi} for m = 0..M by Reinsch's modification of the three-term recurrence
// (as in Stoer & Bulirsch, Introduction to Numerical Analysis, chapter 1).  The plain
// Chebyshev recurrence cos((m+1)p) = 2 cos(p) cos(mp) - cos((m-1)p) only sees cos(p),
// which in fp32 loses the angle near p = 0 and pi (an error of roughly m eps/|sin p|)
// and amplifies its rounding like m^2 there.  Here the angle is first folded to
// psi = phi (cos phi >= 0) or phi - pi (cos phi < 0), so that cos psi = |cos phi|,
// sin psi = sigma sin phi with sigma = sign(cos phi), and e^{i m phi} = sigma^m e^{i m psi}.
// With lambda = 2 (cos psi - 1) = -2 sin^2 psi / (1 + cos psi) (no cancellation) and
// the differences D_m = X_m - X_{m-1}, the recurrence
//     D_{m+1} = D_m + lambda X_m,     X_{m+1} = X_m + D_{m+1}
// is the same three-term relation, but its rounding errors grow only about linearly
// in m for every |psi| <= pi/2.  The cosine and sine chains share lambda, so each step
// is one packed f32x2 FMA and one packed add on (cos part, sin part); the neighbour
// weights are folded into the start values, and the sigma^m sign is applied when the
// odd multipoles are accumulated (a packed FMA in place of the packed add).
struct Fold {
    float ac;   // |cos phi| = cos psi
    float ss;   // sigma sin phi = sin psi
    float sg;   // sigma
    float lam;  // 2 (cos psi - 1)
};

__device__ __forceinline__ Fold fold_angle(float cph, float sph) {
    Fold f;
    f.ac = fabsf(cph);
    f.sg = cph < 0.0f ? -1.0f : 1.0f;
    f.ss = f.sg * sph;
    f.lam = -2.0f * __fdividef(sph * sph, 1.0f + f.ac);
    return f;
}

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// acc[m] += (wc cos(m phi), ws sin(m phi)), m = 0..M, from the folded angle.
// mr <= M: the multipoles computed (a runtime m_max below the compiled one).
template <int M>
__device__ __forceinline__ void harmonicsf(float2 (&acc)[M + 1], const Fold& f, float wc, float ws, int mr = M) {
    acc[0].x += wc;
    if constexpr (M >= 1) {
        if (mr < 1) return;
        float2 X = make_float2(wc * f.ac, ws * f.ss);           // X_1 (psi frame)
        float2 D = make_float2(0.5f * f.lam * wc, ws * f.ss);   // X_1 - X_0
        const float2 S2 = make_float2(f.sg, f.sg);
        const float2 L2 = make_float2(f.lam, f.lam);
        acc[1] = __ffma2_rn(S2, X, acc[1]);
#pragma unroll
        for (int m = 2; m <= M; ++m) {
            if (m > mr) break;
            D = __ffma2_rn(L2, X, D);
            X = __fadd2_rn(X, D);
            acc[m] = (m & 1) ? __ffma2_rn(S2, X, acc[m]) : __fadd2_rn(acc[m], X);
        }
    }
}

template <int M>
__device__ __forceinline__ void harmonics(float2 (&acc)[M + 1], float cph, float sph, float wc, float ws,
                                          int mr = M) {
    harmonicsf<M>(acc, fold_angle(cph, sph), wc, ws, mr);
}

// The same for two pixels a and b at once (two independent chains for
// instruction-level parallelism), from their folded angles.
template <int M>
__device__ __forceinline__ void harmonics2f(float2 (&acc)[M + 1], const Fold& fa, float wca, float wsa,
                                            const Fold& fb, float wcb, float wsb, int mr = M) {
    acc[0].x += wca + wcb;
    if constexpr (M >= 1) {
        if (mr < 1) return;
        float2 Xa = make_float2(wca * fa.ac, wsa * fa.ss), Da = make_float2(0.5f * fa.lam * wca, wsa * fa.ss);
        float2 Xb = make_float2(wcb * fb.ac, wsb * fb.ss), Db = make_float2(0.5f * fb.lam * wcb, wsb * fb.ss);
        const float2 Sa = make_float2(fa.sg, fa.sg), Sb = make_float2(fb.sg, fb.sg);
        const float2 La = make_float2(fa.lam, fa.lam), Lb = make_float2(fb.lam, fb.lam);
        acc[1] = __ffma2_rn(Sb, Xb, __ffma2_rn(Sa, Xa, acc[1]));
#pragma unroll
        for (int m = 2; m <= M; ++m) {
            if (m > mr) break;
            Da = __ffma2_rn(La, Xa, Da);
            Db = __ffma2_rn(Lb, Xb, Db);
            Xa = __fadd2_rn(Xa, Da);
            Xb = __fadd2_rn(Xb, Db);
            if (m & 1)
                acc[m] = __ffma2_rn(Sb, Xb, __ffma2_rn(Sa, Xa, acc[m]));
            else
                acc[m] = __fadd2_rn(acc[m], __fadd2_rn(Xa, Xb));
        }
    }
}

template <int M>
__device__ __forceinline__ void harmonics2(float2 (&acc)[M + 1], float ca, float sa, float wca, float wsa, float cb,
                                           float sb, float wcb, float wsb, int mr = M) {
    harmonics2f<M>(acc, fold_angle(ca, sa), wca, wsa, fold_angle(cb, sb), wcb, wsb, mr);
}

// A folded angle held by lane `src`, broadcast to the warp.
__device__ __forceinline__ Fold shfl_fold(const Fold& f, int src) {
    Fold g;
    g.ac = __shfl_sync(0xffffffffu, f.ac, src);
    g.ss = __shfl_sync(0xffffffffu, f.ss, src);
    g.sg = __shfl_sync(0xffffffffu, f.sg, src);
    g.lam = __shfl_sync(0xffffffffu, f.lam, src);
    return g;
}

// p mod n for -n <= p < 2n (every unwrapped index of a run lies in that range).
__device__ __forceinline__ int wrap_idx(int p, int n) {
    return p < 0 ? p + n : (p >= n ? p - n : p);
}

// Neighbour data access: the packed (w d, w) array the library prepares, or the
// caller's delta and w read directly (used where no packing buffer may be allocated).
struct PackedLoad {
    const float2* __restrict__ p;
    __device__ __forceinline__ float2 operator()(long long i) const { return __ldg(p + i); }
    // accessor of one ring's pixels (index relative to the ring's first pixel)
    struct Row {
        const float2* __restrict__ p;
        __device__ __forceinline__ float2 operator()(int i) const { return __ldg(p + i); }
    };
    __device__ __forceinline__ Row row(long long first) const { return Row{p + first}; }
};
struct DirectLoad {
    const float* __restrict__ d;
    const float* __restrict__ w;
    __device__ __forceinline__ float2 operator()(long long i) const {
        const float wi = __ldg(w + i);
        return make_float2(wi * __ldg(d + i), wi);
    }
    struct Row {
        const float* __restrict__ d;
        const float* __restrict__ w;
        __device__ __forceinline__ float2 operator()(int i) const {
            const float wi = __ldg(w + i);
            return make_float2(wi * __ldg(d + i), wi);
        }
    };
    __device__ __forceinline__ Row row(long long first) const { return Row{d + first, w + first}; }
};

// Walk pixels [a, a + len) of ring R (lane-private run), accumulating into the bin.
// Two pixels per iteration.  When no lane's run wraps around the ring, the first
// min-length iterations run without predicates or index wrapping; the rest (and
// wrapping runs) take the general loop.
template <int M, bool FAST, bool SELF, class L>
__device__ __forceinline__ void walk_run(const RingCtx& R, const L& ld, const LaneC& c, int a, int len,
                                         float2 (&acc)[M + 1], float& W, float& Q, float& QW, int mr = M) {
    const int maxlen = __reduce_max_sync(0xffffffffu, len);
    if (maxlen <= 0) return;
    const float i0 = (float)(a - c.cint);
    const float xneg = -c.cfrac * R.step, uneg = -c.cfrac * R.inv_n;
    int idx = wrap_idx(a, R.n);
    const auto row = ld.row(R.first);
    int t = 0;
    const int minlen = __reduce_min_sync(0xffffffffu, len);
    if (minlen >= 2 && __all_sync(0xffffffffu, idx + len <= R.n)) {
        float ft = i0;
        for (; t + 1 < minlen; t += 2, ft += 2.0f) {
            const float2 v0 = row(idx + t), v1 = row(idx + t + 1);
            float ca, sa, cb, sb;
            pixel_dir<FAST>(ft, xneg, uneg, R, ca, sa);
            pixel_dir<FAST>(ft + 1.0f, xneg, uneg, R, cb, sb);
            harmonics2<M>(acc, ca, sa, v0.x, v0.x, cb, sb, v1.x, v1.x, mr);
            W += v0.y + v1.y;
            if (SELF) {
                Q = fmaf(v0.x, v0.x, fmaf(v1.x, v1.x, Q));
                QW = fmaf(v0.y, v0.y, fmaf(v1.y, v1.y, QW));
            }
        }
        idx += t;
        if (idx >= R.n) idx -= R.n;
    }
    for (; t < maxlen; t += 2) {
        const bool on0 = t < len, on1 = t + 1 < len;
        const int idx1 = idx + 1 >= R.n ? idx + 1 - R.n : idx + 1;
        const float2 v0 = on0 ? row(idx) : make_float2(0.0f, 0.0f);
        const float2 v1 = on1 ? row(idx1) : make_float2(0.0f, 0.0f);
        const float oa = on0 ? i0 + (float)t : i0;
        const float ob = on1 ? i0 + (float)(t + 1) : i0;
        float ca, sa, cb, sb;
        pixel_dir<FAST>(oa, xneg, uneg, R, ca, sa);
        pixel_dir<FAST>(ob, xneg, uneg, R, cb, sb);
        harmonics2<M>(acc, ca, sa, v0.x, v0.x, cb, sb, v1.x, v1.x, mr);
        W += v0.y + v1.y;
        if (SELF) {
            Q = fmaf(v0.x, v0.x, fmaf(v1.x, v1.x, Q));
            QW = fmaf(v0.y, v0.y, fmaf(v1.y, v1.y, QW));
        }
        idx = idx1 + 1 >= R.n ? idx1 + 1 - R.n : idx1 + 1;
    }
}

// walk_run for a tile in the quadrant layout (tile_pivot): the four lanes l, l + 8,
// l + 16, l + 24 hold pivots a quarter turn apart, and since every ring has a multiple
// of four pixels they see ring r at the same fractional offset, with runs of the same
// length at the same offset from their own pivot, hence the same position angle at
// every step.  Each lane of a group computes the (folded) angle of one of every four
// steps and the group shares them by shuffles; every lane still sums its own pixels.
// The caller has checked runs_quad().
template <int M, bool FAST, bool SELF, class L>
__device__ __forceinline__ void walk_run_quad(const RingCtx& R, const L& ld, const LaneC& c, int a, int len,
                                              float2 (&acc)[M + 1], float& W, float& Q, float& QW, int mr = M) {
    const int maxlen = __reduce_max_sync(0xffffffffu, len);
    if (maxlen <= 0) return;
    const int lane = threadIdx.x & 31, j = lane >> 3, gb = lane & 7;
    const float i0 = (float)(a - c.cint);
    const float xneg = -c.cfrac * R.step, uneg = -c.cfrac * R.inv_n;
    const int last = max(len - 1, 0);
    int idx = wrap_idx(a, R.n);
    const auto row = ld.row(R.first);
    for (int t0 = 0; t0 < maxlen; t0 += 4) {
        Fold mine;
        {
            // steps past the run take its last offset, a valid direction (zero weight)
            const int tj = min(t0 + j, last);
            float cph, sph;
            pixel_dir<FAST>(i0 + (float)tj, xneg, uneg, R, cph, sph);
            mine = fold_angle(cph, sph);
        }
        // two steps at a time, so that only two shared angles are live
#pragma unroll
        for (int h = 0; h < 4; h += 2) {
            const Fold fa = shfl_fold(mine, gb + 8 * h), fb = shfl_fold(mine, gb + 8 * h + 8);
            const int i1 = idx + 1 >= R.n ? idx + 1 - R.n : idx + 1;
            // (the index test is a guard: a run's indices always lie within the ring)
            const bool ia = t0 + h < len && (unsigned)idx < (unsigned)R.n;
            const bool ib = t0 + h + 1 < len && (unsigned)i1 < (unsigned)R.n;
            const float2 va = ia ? row(idx) : make_float2(0.0f, 0.0f);
            const float2 vb = ib ? row(i1) : make_float2(0.0f, 0.0f);
            harmonics2f<M>(acc, fa, va.x, va.x, fb, vb.x, vb.x, mr);
            W += va.y + vb.y;
            if (SELF) {
                Q = fmaf(va.x, va.x, fmaf(vb.x, vb.x, Q));
                QW = fmaf(va.y, va.y, fmaf(vb.y, vb.y, QW));
            }
            idx = i1 + 1 >= R.n ? i1 + 1 - R.n : i1 + 1;
        }
    }
}

// True when each lane's run has the same offset from its pivot, the same length and
// the same fractional pivot position as the other three lanes of its quadrant group
// (an empty run matches any other empty run).  Every lane takes part in every shuffle.
__device__ __forceinline__ bool runs_quad(const LaneC& c, int a, int len) {
    const int gb = threadIdx.x & 7;
    const int rel = len > 0 ? a - c.cint : 0;
    const unsigned cf = __float_as_uint(c.cfrac);
    const int rel0 = __shfl_sync(0xffffffffu, rel, gb);
    const int len0 = __shfl_sync(0xffffffffu, len, gb);
    const unsigned cf0 = __shfl_sync(0xffffffffu, cf, gb);
    return __all_sync(0xffffffffu, rel == rel0 && len == len0 && cf == cf0);
}

// Walk the pixel pairs (p, mb - p), p in [a, a + len): mirror images about the
// pivot's meridian (belt rings with as many pixels as the pivot ring).  Two pairs
// (four pixels) per iteration; the same no-wrap fast loop as walk_run.
template <int M, bool FAST, bool SELF, class L>
__device__ __forceinline__ void walk_pairs(const RingCtx& R, const L& ld, const LaneC& c, int a, int len,
                                           int mb, float2 (&acc)[M + 1], float& W, float& Q,
                                           float& QW, int mr = M) {
    const int maxlen = __reduce_max_sync(0xffffffffu, len);
    if (maxlen <= 0) return;
    const float i0 = (float)(a - c.cint);
    const float xneg = -c.cfrac * R.step, uneg = -c.cfrac * R.inv_n;
    int ip = wrap_idx(a, R.n);
    int im_ = wrap_idx(mb - a, R.n);
    const auto row = ld.row(R.first);
    int t = 0;
    const int minlen = __reduce_min_sync(0xffffffffu, len);
    if (minlen >= 2 && __all_sync(0xffffffffu, ip + len <= R.n && im_ - len + 1 >= 0)) {
        float ft = i0;
        for (; t + 1 < minlen; t += 2, ft += 2.0f) {
            const float2 p0 = row(ip + t), m0 = row(im_ - t);
            const float2 p1 = row(ip + t + 1), m1 = row(im_ - t - 1);
            float ca, sa, cb, sb;
            pixel_dir<FAST>(ft, xneg, uneg, R, ca, sa);
            pixel_dir<FAST>(ft + 1.0f, xneg, uneg, R, cb, sb);
            harmonics2<M>(acc, ca, sa, p0.x + m0.x, p0.x - m0.x, cb, sb, p1.x + m1.x, p1.x - m1.x, mr);
            W += (p0.y + m0.y) + (p1.y + m1.y);
            if (SELF) {
                Q = fmaf(p0.x, p0.x, fmaf(m0.x, m0.x, fmaf(p1.x, p1.x, fmaf(m1.x, m1.x, Q))));
                QW = fmaf(p0.y, p0.y, fmaf(m0.y, m0.y, fmaf(p1.y, p1.y, fmaf(m1.y, m1.y, QW))));
            }
        }
        ip += t;
        if (ip >= R.n) ip -= R.n;
        im_ -= t;
        if (im_ < 0) im_ += R.n;
    }
    for (; t < maxlen; t += 2) {
        const bool on0 = t < len, on1 = t + 1 < len;
        const int ip1 = ip + 1 >= R.n ? ip + 1 - R.n : ip + 1;
        const int im1 = im_ - 1 < 0 ? im_ - 1 + R.n : im_ - 1;
        const float2 p0 = on0 ? row(ip) : make_float2(0.0f, 0.0f);
        const float2 m0 = on0 ? row(im_) : make_float2(0.0f, 0.0f);
        const float2 p1 = on1 ? row(ip1) : make_float2(0.0f, 0.0f);
        const float2 m1 = on1 ? row(im1) : make_float2(0.0f, 0.0f);
        const float oa = on0 ? i0 + (float)t : i0;
        const float ob = on1 ? i0 + (float)(t + 1) : i0;
        float ca, sa, cb, sb;
        pixel_dir<FAST>(oa, xneg, uneg, R, ca, sa);
        pixel_dir<FAST>(ob, xneg, uneg, R, cb, sb);
        harmonics2<M>(acc, ca, sa, p0.x + m0.x, p0.x - m0.x, cb, sb, p1.x + m1.x, p1.x - m1.x, mr);
        W += (p0.y + m0.y) + (p1.y + m1.y);
        if (SELF) {
            Q = fmaf(p0.x, p0.x, fmaf(m0.x, m0.x, fmaf(p1.x, p1.x, fmaf(m1.x, m1.x, Q))));
            QW = fmaf(p0.y, p0.y, fmaf(m0.y, m0.y, fmaf(p1.y, p1.y, fmaf(m1.y, m1.y, QW))));
        }
        ip = ip1 + 1 >= R.n ? ip1 + 1 - R.n : ip1 + 1;
        im_ = im1 - 1 < 0 ? im1 - 1 + R.n : im1 - 1;
    }
}

// walk_pairs for the case of a belt ring pair (the neighbour ring has as many pixels
// as the pivot ring): the 32 pivots of the tile then sit at the same fractional
// position relative to ring r, so every lane's run starts at the same offset from its
// own pivot and has the same length, and at step t all lanes see a neighbour at the
// same offset, hence the same position angle.  Each lane computes the (folded) angle of
// one step of a block of 32 and the warp shares them by shuffles, instead of every lane
// computing the same angle.  Lane l's pixels are those of lane 0 shifted by l, so the
// loads of a step stay coalesced.
template <int M, bool SELF, class L>
__device__ __forceinline__ void walk_pairs_shared(const RingCtx& R, const L& ld, const LaneC& c, int a, int len,
                                                  int mb, float2 (&acc)[M + 1], float& W, float& Q, float& QW,
                                                  int mr = M) {
    if (len <= 0) return;
    const int lane = threadIdx.x & 31;
    const float i0 = (float)(a - c.cint);
    const float xneg = -c.cfrac * R.step, uneg = -c.cfrac * R.inv_n;
    const auto row = ld.row(R.first);
    int ip = wrap_idx(a, R.n);
    int im_ = wrap_idx(mb - a, R.n);
    for (int t0 = 0; t0 < len; t0 += 32) {
        // this lane's step: t0 + lane
        Fold mine;
        {
            const float ft = i0 + (float)(t0 + lane);
            float cph, sph;
            if (fabsf(ft - c.cfrac) * R.step <= FAST_XMAX)
                pixel_dir<true>(ft, xneg, uneg, R, cph, sph);
            else
                pixel_dir<false>(ft, xneg, uneg, R, cph, sph);
            mine = fold_angle(cph, sph);
        }
        const int nstep = min(32, len - t0);
        int tt = 0;
        for (; tt + 1 < nstep; tt += 2) {
            const Fold fa = shfl_fold(mine, tt), fb = shfl_fold(mine, tt + 1);
            const int ip1 = ip + 1 >= R.n ? ip + 1 - R.n : ip + 1;
            const int im1 = im_ - 1 < 0 ? im_ - 1 + R.n : im_ - 1;
            const float2 p0 = row(ip), m0 = row(im_), p1 = row(ip1), m1 = row(im1);
            harmonics2f<M>(acc, fa, p0.x + m0.x, p0.x - m0.x, fb, p1.x + m1.x, p1.x - m1.x, mr);
            W += (p0.y + m0.y) + (p1.y + m1.y);
            if (SELF) {
                Q = fmaf(p0.x, p0.x, fmaf(m0.x, m0.x, fmaf(p1.x, p1.x, fmaf(m1.x, m1.x, Q))));
                QW = fmaf(p0.y, p0.y, fmaf(m0.y, m0.y, fmaf(p1.y, p1.y, fmaf(m1.y, m1.y, QW))));
            }
            ip = ip1 + 1 >= R.n ? ip1 + 1 - R.n : ip1 + 1;
            im_ = im1 - 1 < 0 ? im1 - 1 + R.n : im1 - 1;
        }
        if (tt < nstep) {
            const Fold fa = shfl_fold(mine, tt);
            const float2 p0 = row(ip), m0 = row(im_);
            harmonicsf<M>(acc, fa, p0.x + m0.x, p0.x - m0.x, mr);
            W += p0.y + m0.y;
            if (SELF) {
                Q = fmaf(p0.x, p0.x, fmaf(m0.x, m0.x, Q));
                QW = fmaf(p0.y, p0.y, fmaf(m0.y, m0.y, QW));
            }
            ip = ip + 1 >= R.n ? ip + 1 - R.n : ip + 1;
            im_ = im_ - 1 < 0 ? im_ - 1 + R.n : im_ - 1;
        }
    }
}

// True when every lane's run has lane 0's start offset and length (belt ring pairs).
__device__ __forceinline__ bool runs_shared(const LaneC& c, int a, int len) {
    const int rel = a - c.cint;
    const int rel0 = __shfl_sync(0xffffffffu, rel, 0), len0 = __shfl_sync(0xffffffffu, len, 0);
    const unsigned cf = __float_as_uint(c.cfrac), cf0 = __shfl_sync(0xffffffffu, cf, 0);
    return __all_sync(0xffffffffu, rel == rel0 && len == len0 && cf == cf0);
}

// Runs of bin k on ring r for the lane's pivot.  Fills up to two runs (a, len) and,
// in mirror mode, one pair run plus an optional centre pixel.
struct BinRuns {
    int a0, n0, a1, n1;  // plain runs
    bool sym;            // pair mode: pairs (p, mb - p), p in [a0, a0 + n0)
    int mb;              // mirror base
    bool centre;         // pixel cint (offset 0) also belongs to the bin (pair mode)
};

__device__ __forceinline__ BinRuns bin_runs(const LaneC& c, int2 Tk, int2 Tk1, double Ek, double Ek1,
                                            const ExactCtx& x, int n_r, bool sym) {
    BinRuns b;
    b.sym = sym;
    b.centre = false;
    b.mb = 0;
    b.a1 = 0;
    b.n1 = 0;
    // upper end of the + side, lower end of the - side
    int pe, ns;
    if (Tk1.x == T_INF) {
        pe = c.cint + n_r / 2;
        ns = c.cint - n_r / 2 + 1;
    } else {
        pe = pos_edge(c, Tk1, Ek1, x) - 1;
        ns = neg_edge(c, Tk1, Ek1, x) + 1;
    }
    if (sym) {
        int a;
        if (Tk.x == T_ZERO) {
            a = c.cint + 1;
            b.centre = (c.crem == 0);
        } else {
            a = pos_edge(c, Tk, Ek, x);
        }
        b.a0 = a;
        b.n0 = max(0, pe - a + 1);
        b.mb = 2 * c.cint + (c.crem != 0 ? 1 : 0);
        return b;
    }
    if (Tk.x == T_ZERO) {
        b.a0 = ns;
        b.n0 = max(0, pe - ns + 1);
    } else {
        const int pa = pos_edge(c, Tk, Ek, x);
        const int nb = neg_edge(c, Tk, Ek, x);
        b.a0 = pa;
        b.n0 = max(0, pe - pa + 1);
        b.a1 = ns;
        b.n1 = max(0, nb - ns + 1);
    }
    return b;
}

// Largest |o| a run reaches, for the FAST test.
__device__ __forceinline__ float run_omax(const LaneC& c, int a, int len) {
    if (len <= 0) return 0.0f;
    const float o0 = (float)(a - c.cint) - c.cfrac;
    return fmaxf(fabsf(o0), fabsf(o0 + (float)(len - 1)));
}

// Everything a warp needs about pivot ring i.
struct PivotRing {
    int i, n_i, s_i;
    float z_i;
    double th_i, s_i_d;
    int rlo;
    long long pair0;
};

__device__ __forceinline__ RingCtx ring_ctx(const MapDev& g, const PivotRing& P, int r, long long pr) {
    RingCtx R;
    R.first = g.ring_first[r];
    R.n = g.ring_n[r];
    R.shift = g.ring_shift[r];
    R.s_r = g.ring_sf[r];
    R.s_lo = g.ring_sf_lo[r];
    const float2 Ap = g.pair_A[pr];
    R.A = Ap.x;
    R.A_lo = Ap.y;
    R.B = 2.0f * P.z_i * R.s_r;
    R.step = g.ring_step[r];
    R.step_lo = g.ring_step_lo[r];
    R.inv_n = g.ring_invn[r];
    R.invn_lo = g.ring_invn_lo[r];
    return R;
}

__device__ __forceinline__ ExactCtx exact_ctx(const MapDev& g, const PivotRing& P, int r) {
    ExactCtx x;
    x.th_i = P.th_i;
    x.th_r = g.ring_th[r];
    x.s_i = P.s_i_d;
    x.s_r = g.ring_s[r];
    x.n_r = g.ring_n[r];
    return x;
}

// Accumulate the bin-k moments of ring r into the lane's registers.
template <int M, bool SELF, class L>
__device__ __forceinline__ void fwd_ring_bin(const MapDev& g, const PivotRing& P, int r, int k, int q,
                                             const L& ld, float2 (&acc)[M + 1], float& W,
                                             float& Q, float& QW, int mr = M, bool quad = false) {
    const long long pr = P.pair0 + (r - P.rlo);
    const int2 Tk = g.pair_T[pr * (g.K + 1) + k];
    const int2 Tk1 = g.pair_T[pr * (g.K + 1) + k + 1];
    if (Tk.x == T_INF || Tk1.x == T_ZERO) return;  // no bin-k pixel on this ring
    const RingCtx R = ring_ctx(g, P, r, pr);
    const ExactCtx x = exact_ctx(g, P, r);
    const LaneC c = lane_c(q, P.s_i, P.n_i, R.shift, R.n);
    const bool sym = (R.n == P.n_i) && (Tk1.x != T_INF);
    const BinRuns b = bin_runs(c, Tk, Tk1, g.E[k], g.E[k + 1], x, R.n, sym);
    if (sym) {
        if (b.centre) {  // the pixel straight north or south of the pivot
            const float2 v = ld(R.first + wrap_idx(c.cint, R.n));
            float cph, sph;
            pixel_dir<false>(0.0f, 0.0f, -c.cfrac * R.inv_n, R, cph, sph);
            harmonics<M>(acc, cph, sph, v.x, v.x, mr);
            W += v.y;
            if (SELF) {
                Q = fmaf(v.x, v.x, Q);
                QW = fmaf(v.y, v.y, QW);
            }
        }
        if (runs_shared(c, b.a0, b.n0)) {
            walk_pairs_shared<M, SELF>(R, ld, c, b.a0, b.n0, b.mb, acc, W, Q, QW, mr);
            return;
        }
        const bool fast = __all_sync(0xffffffffu, run_omax(c, b.a0, b.n0) * R.step <= FAST_XMAX);
        if (fast)
            walk_pairs<M, true, SELF>(R, ld, c, b.a0, b.n0, b.mb, acc, W, Q, QW, mr);
        else
            walk_pairs<M, false, SELF>(R, ld, c, b.a0, b.n0, b.mb, acc, W, Q, QW, mr);
        return;
    }
    const float om = fmaxf(run_omax(c, b.a0, b.n0), run_omax(c, b.a1, b.n1));
    const bool fast = __all_sync(0xffffffffu, om * R.step <= FAST_XMAX);
    if (quad && runs_quad(c, b.a0, b.n0) && runs_quad(c, b.a1, b.n1)) {
        if (fast) {
            walk_run_quad<M, true, SELF>(R, ld, c, b.a0, b.n0, acc, W, Q, QW, mr);
            walk_run_quad<M, true, SELF>(R, ld, c, b.a1, b.n1, acc, W, Q, QW, mr);
        } else {
            walk_run_quad<M, false, SELF>(R, ld, c, b.a0, b.n0, acc, W, Q, QW, mr);
            walk_run_quad<M, false, SELF>(R, ld, c, b.a1, b.n1, acc, W, Q, QW, mr);
        }
        return;
    }
    if (fast) {
        walk_run<M, true, SELF>(R, ld, c, b.a0, b.n0, acc, W, Q, QW, mr);
        walk_run<M, true, SELF>(R, ld, c, b.a1, b.n1, acc, W, Q, QW, mr);
    } else {
        walk_run<M, false, SELF>(R, ld, c, b.a0, b.n0, acc, W, Q, QW, mr);
        walk_run<M, false, SELF>(R, ld, c, b.a1, b.n1, acc, W, Q, QW, mr);
    }
}

// Shared-memory layout of a tile's moments.
//   A[k][m][2][32] : sum w d cos(m phi), sum w d sin(m phi)   (a = re - i im)
//   W[k][32], Q[k][32], QW[k][32], piv[2][32] (w d, w of the pivots)
template <int M>
__host__ __device__ inline size_t tile_floats(int K) {
    return tile_floats_rt(K, M);
}

// Load the tile's pivot description; returns false if no lane has w != 0.
__device__ __forceinline__ PivotRing pivot_ring(const MapDev& g, int i) {
    PivotRing P;
    P.i = i;
    P.n_i = g.ring_n[i];
    P.s_i = g.ring_shift[i];
    P.z_i = g.ring_zf[i];
    P.th_i = g.ring_th[i];
    P.s_i_d = g.ring_s[i];
    P.rlo = g.ring_range[i].x;
    P.pair0 = g.pair_off[i];
    return P;
}

// Pivot of a lane in tile (ring i, start = 32 j).  Linear layout: q = start + lane.
// Quadrant layout (the forward kernels): q = 8 j + (lane & 7) + (lane >> 3) n_i / 4,
// four groups of eight consecutive pivots a quarter turn apart (walk_run_quad); a ring
// has ceil(n_i / 32) tiles either way.  `valid`: q is a pixel of the ring; lanes past
// the end take the geometry qg of the last pivot (of their quadrant), which keeps every
// unwrapped pixel index within [-n_r, 2 n_r).
struct TilePivot {
    int q, qg;
    bool valid;
};

__device__ __forceinline__ TilePivot tile_pivot(int start, int n_i, bool quad) {
    const int lane = threadIdx.x & 31;
    TilePivot t;
    if (quad) {
        const int quarter = n_i >> 2, qq = (start >> 2) + (lane & 7), off = (lane >> 3) * quarter;
        t.valid = qq < quarter;
        t.q = qq + off;
        t.qg = min(qq, quarter - 1) + off;
    } else {
        t.q = start + lane;
        t.valid = t.q < n_i;
        t.qg = min(t.q, n_i - 1);
    }
    return t;
}

// Where the tile's moments live in shared memory.  LayKM: A[k][m][re/im][32 pivots],
// W[k][32], Q[k][32], QW[k][32] (the FP32 contraction and the adjoint read this).
struct LayKM {
    float *sA, *sW, *sQ, *sQW;
    int M1;  // m_max + 1
    __device__ __forceinline__ float* a(int k, int m, int part, int lane) const {
        return sA + ((size_t)(k * M1 + m) * 2 + part) * TILE + lane;
    }
    __device__ __forceinline__ float* w(int k, int lane) const { return sW + k * TILE + lane; }
    __device__ __forceinline__ float* q(int k, int lane) const { return sQ + k * TILE + lane; }
    __device__ __forceinline__ float* qw(int k, int lane) const { return sQW + k * TILE + lane; }
};

// All warps of the CTA: accumulate the moments of the tile into shared memory.
// Smem must be zeroed beforehand; it is complete after the caller's __syncthreads().
template <int M, bool SELF, class L, class Lay>
__device__ __forceinline__ void tile_moments_l(const MapDev& g, const PivotRing& P, int q, const L& ld,
                                               const Lay& lay, int flush, int mr = M, bool quad = false) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < g.K; ++k) {
        const int2 br = g.bin_range[(long long)P.i * g.K + k];
        if (br.x + warp > br.y) continue;
        float2 acc[M + 1];
#pragma unroll
        for (int m = 0; m <= M; ++m) acc[m] = make_float2(0.0f, 0.0f);
        float W = 0.0f, Q = 0.0f, QW = 0.0f;
        // Blocked summation: the registers sum `flush` rings (FLUSH_RINGS unless
        // tuned), then the block is added into shared memory, which keeps the running
        // sums short.
        int nr = 0;
        for (int r = br.x + warp; r <= br.y; r += NWARPS) {
            fwd_ring_bin<M, SELF>(g, P, r, k, q, ld, acc, W, Q, QW, mr, quad);
            if (++nr == flush || r + NWARPS > br.y) {
                nr = 0;
#pragma unroll
                for (int m = 0; m <= M; ++m) {
                    if (m > mr) break;
                    atomicAdd(lay.a(k, m, 0, lane), acc[m].x);
                    atomicAdd(lay.a(k, m, 1, lane), acc[m].y);
                    acc[m] = make_float2(0.0f, 0.0f);
                }
                atomicAdd(lay.w(k, lane), W);
                W = 0.0f;
                if (SELF) {
                    atomicAdd(lay.q(k, lane), Q);
                    atomicAdd(lay.qw(k, lane), QW);
                    Q = 0.0f;
                    QW = 0.0f;
                }
            }
        }
    }
}

template <int M, bool SELF, class L>
__device__ __forceinline__ void tile_moments(const MapDev& g, const PivotRing& P, int q, const L& ld, float* sA,
                                             float* sW, float* sQ, float* sQW, int flush, int mr = M,
                                             bool quad = false) {
    tile_moments_l<M, SELF>(g, P, q, ld, LayKM{sA, sW, sQ, sQW, mr + 1}, flush, mr, quad);
}

// Per-pivot normalisation of the tile's moments (Sec. 3.1): each lane's a_m^k is
// divided by its bin weight W^k (NORM_BIN_MEAN) or by its total sum_k W^k
// (NORM_PIVOT_TOTAL), 0 where that weight is 0; W^k is then set to 1, so that the
// contraction's D entries become the tile's sum of pivot weights.  Layout of
// tile_moments (m-major within each bin, TILE lanes innermost).  Called by every
// thread of the CTA after the moments are complete (contains barriers).
template <int M>
__device__ __forceinline__ void tile_normalize(int K, float* sA, float* sW, int norm, int mr = M) {
    constexpr int PER = (TPCF_MAX_BINS * TILE + NTHREADS - 1) / NTHREADS;
    float inv[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * NTHREADS;
        float W = 0.0f;
        if (e < K * TILE) {
            if (norm == NORM_BIN_MEAN) {
                W = sW[e];
            } else {
                const int l = e & (TILE - 1);
                for (int k = 0; k < K; ++k) W += sW[k * TILE + l];
            }
        }
        inv[u] = W > 0.0f ? 1.0f / W : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * NTHREADS;
        if (e < K * TILE) {
            const int k = e / TILE, l = e & (TILE - 1);
            float* a = sA + (size_t)k * (mr + 1) * 2 * TILE + l;
            for (int j = 0; j < 2 * (mr + 1); ++j) a[j * TILE] *= inv[u];
            sW[e] = 1.0f;
        }
    }
    __syncthreads();
}

// Per-tile partial sums into the CTA's FP64 slot (eq. zetamEst2 summed over the
// tile's pivots).  Slot layout: for m, for pair (k1 <= k2): (Re S, Im S); then D for
// pairs; then sum_i w_i d_i Q^k(i) and sum_i w_i QW^k(i) for k.
template <int M>
__device__ __forceinline__ void tile_contract(int K, const float* sA, const float* sW, const float* sQ,
                                              const float* sQW, const float* sPiv, double* slot,
                                              bool self, int mr = M) {
    const int P = n_pairs_tri(K);
    const int nS = (mr + 1) * P;
    const float* wd = sPiv;
    const float* wt = sPiv + TILE;
    for (int e = threadIdx.x; e < nS + P + (self ? K : 0); e += NTHREADS) {
        if (e < nS) {
            const int m = e / P;
            const int pidx = e - m * P;
            int k2 = (int)((sqrtf(8.0f * pidx + 1.0f) - 1.0f) * 0.5f);
            while (k2 * (k2 + 1) / 2 > pidx) --k2;
            while ((k2 + 1) * (k2 + 2) / 2 <= pidx) ++k2;
            const int k1 = pidx - k2 * (k2 + 1) / 2;
            const float* r1 = sA + ((size_t)k1 * (mr + 1) + m) * 2 * TILE;
            const float* i1 = r1 + TILE;
            const float* r2 = sA + ((size_t)k2 * (mr + 1) + m) * 2 * TILE;
            const float* i2 = r2 + TILE;
            float sr = 0.0f, si = 0.0f;
            // start each thread at its own lane so a warp's 32 rows hit 32 banks
#pragma unroll 8
            for (int j = 0; j < TILE; ++j) {
                const int l = (j + threadIdx.x) & (TILE - 1);
                const float a = r1[l], b = i1[l], cc = r2[l], d = i2[l];
                sr = fmaf(wd[l], fmaf(a, cc, b * d), sr);
                si = fmaf(wd[l], fmaf(a, d, -b * cc), si);
            }
            red_add_f32(slot + 2 * e, sr);
            red_add_f32(slot + 2 * e + 1, si);
        } else if (e < nS + P) {
            const int pidx = e - nS;
            int k2 = (int)((sqrtf(8.0f * pidx + 1.0f) - 1.0f) * 0.5f);
            while (k2 * (k2 + 1) / 2 > pidx) --k2;
            while ((k2 + 1) * (k2 + 2) / 2 <= pidx) ++k2;
            const int k1 = pidx - k2 * (k2 + 1) / 2;
            float s = 0.0f;
#pragma unroll 8
            for (int j = 0; j < TILE; ++j) {
                const int l = (j + threadIdx.x) & (TILE - 1);
                s = fmaf(wt[l], sW[k1 * TILE + l] * sW[k2 * TILE + l], s);
            }
            red_add_f32(slot + nS + e, s);
        } else {
            const int k = e - nS - P;
            float s1 = 0.0f, s2 = 0.0f;
            for (int j = 0; j < TILE; ++j) {
                const int l = (j + threadIdx.x) & (TILE - 1);
                s1 = fmaf(wd[l], sQ[k * TILE + l], s1);
                s2 = fmaf(wt[l], sQW[k * TILE + l], s2);
            }
            red_add_f32(slot + 2 * nS + P + k, s1);
            red_add_f32(slot + 2 * nS + P + K + k, s2);
        }
    }
}

// ------------------------------------------------- tensor-core contraction (TF32x3)
// The contraction of eq. zetamEst2 over a tile's 32 pivots is, for each m, the Gram
// matrix G = X diag(w d) X^T of X = [Re a ; Im a] (rows r = 2k + part, 32 pivot
// columns): S_m(k1,k2) = G[2k1][2k2] + G[2k1+1][2k2+1] + i (G[2k1][2k2+1] - G[2k1+1][2k2])
// in the convention a = re - i im; D is the Gram matrix of the W^k rows with the
// weights w.  On the 5th-generation tensor cores (kind::tf32, FP32 accumulation in
// tensor memory), per block of rows (each m, then the W block):
//   * the moments are accumulated straight into the layout the MMA reads (K-major,
//     no swizzle: 8-row x 16-byte core matrices, pivot-adjacent ones 128 B apart,
//     8-row groups 1024 B apart, blocks starting on a row group); no operand copy of
//     X exists;
//   * with Y = X diag(sqrt|w d|) and s = sign(w d), G = Y diag(s) Y^T.  Y is split into
//     a tf32 part hi (its low 13 mantissa bits cleared, written back in place) and
//     the fp32 remainder lo, and G = hi s hi^T + C + C^T with C = hi s lo^T (the
//     dropped lo s lo^T term is below 2^-22 relative): two MMAs per 8-pivot step,
//     A = hi in place, B = s hi and s lo in a small staging buffer;
//   * the MMA is 128 x N; rows of A beyond the block come from the following shared
//     memory and only reach accumulator rows that are never read;
//   * one thread issues, an mbarrier tracks completion (bounded wait), warps 0-1 read
//     the two accumulators back, C^T goes through shared memory, and S (or D) is added
//     into the CTA's FP64 slot.
// The operands cost no shared memory beyond the moments but the staging buffer, so
// the kernel keeps the FP32 forward's 3 CTAs per SM at 20 bins and m_max 10.
constexpr int TC_TMEM_COLS = 128;  // two accumulators of up to 64 columns
constexpr int ST_TC_TIMEOUT = ST_TC_TIMEOUT_BIT;

// Shared-memory plan of the tensor-core forward tile (in floats from the dynamic
// shared memory base; blocks start on 8-row groups).
struct TcLayout {
    int Rm, RD, NBm, NBd;  // rows per m block and of the W block; MMA N of each
    int x0, D0;            // first row of the moments; first row of the W block
    int offB, offPiv, offSc, offQ, offQW;
    int total;             // floats
};

__host__ __device__ inline TcLayout tc_layout(int K, int M, bool self) {
    TcLayout L;
    L.Rm = (2 * K + 7) & ~7;
    L.RD = (K + 7) & ~7;
    L.NBm = (2 * K + 15) & ~15;
    L.NBd = (K + 15) & ~15;
    L.x0 = 0;
    L.D0 = (M + 1) * L.Rm;
    int off = (L.D0 + L.RD) * TILE;
    L.offB = off;  // B hi rows, then B lo rows (NBm each); reused for the C^T staging
    off += 2 * L.NBm * TILE;
    L.offPiv = off;  // (w d, w) of the pivots
    off += 2 * TILE;
    L.offSc = off;  // sqrt|w d|, sign(w d), sqrt w
    off += 3 * TILE;
    L.offQ = off;
    L.offQW = off + (self ? K * TILE : 0);
    if (self) off += 2 * K * TILE;
    // the MMA of the last block reads 128 rows from its start
    const int need = (L.D0 + 128) * TILE;
    L.total = off > need ? off : need;
    return L;
}

// bytes of dynamic shared memory
__host__ __device__ inline size_t tc_smem_bytes(int K, int M, bool self) {
    return (size_t)tc_layout(K, M, self).total * sizeof(float);
}

// Position of (row r, pivot p) in the K-major canonical layout without swizzle: core
// matrices of 8 rows x 4 pivots (128 contiguous bytes, rows 16 B apart), the 8
// pivot-adjacent core matrices of a row group 128 B apart, row groups 1024 B apart.
__device__ __forceinline__ int kmaj(int r, int p) { return ((r >> 3) << 8) + ((p >> 2) << 5) + ((r & 7) << 2) + (p & 3); }

struct LayTC {
    float* sX;
    float *sQ, *sQW;
    int Rm, D0;
    __device__ __forceinline__ float* a(int k, int m, int part, int lane) const {
        return sX + kmaj(m * Rm + 2 * k + part, lane);
    }
    __device__ __forceinline__ float* w(int k, int lane) const { return sX + kmaj(D0 + k, lane); }
    __device__ __forceinline__ float* q(int k, int lane) const { return sQ + k * TILE + lane; }
    __device__ __forceinline__ float* qw(int k, int lane) const { return sQW + k * TILE + lane; }
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// UMMA shared-memory descriptor, K-major without swizzle: start address, leading
// (pivot-direction) core-matrix offset 128 B, row-group stride 1024 B, descriptor
// version 1.
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(1024u >> 4) << 32) |
           (1ull << 46);
}

// Instruction descriptor: D f32, A and B tf32, both K-major, N, M = 128.
__device__ __forceinline__ uint32_t tc_idesc(int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

// Waits for the mbarrier phase; false after about one second (error path).
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t phase) {
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 1000000000ull) return false;
    }
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Per-CTA tensor-core state: TMEM accumulator base, mbarrier and its phase.
struct TcState {
    uint32_t tmem;
    uint32_t mbar;    // shared address of the mbarrier
    uint32_t phase;
    int* fail;        // shared flag: a wait gave up
};

// Warp 0 allocates the accumulator columns; thread 0 initialises the mbarrier.
__device__ __forceinline__ void tc_setup(uint32_t* s_tmem, uint64_t* s_mbar) {
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(s_mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_teardown(uint32_t tmem) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// The tile's S and D partial sums on the tensor cores (see above); the self-pair
// diagonals stay on the FP32 pipe.  Called by every thread; the moments in sX are
// consumed (truncated in place).
template <int M, bool SELF>
__device__ void tile_contract_tc(int K, float* base, double* slot, TcState& tc, int* status) {
    const TcLayout L = tc_layout(K, M, SELF);
    const int P = n_pairs_tri(K);
    const int nS = (M + 1) * P;
    float* sX = base;
    float* Bhi = base + L.offB;
    const float* sPiv = base + L.offPiv;
    float* sc = base + L.offSc;  // [0] sqrt|w d|, [1] sign(w d), [2] sqrt w
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < TILE) {
        const float wd = sPiv[lane], w = sPiv[TILE + lane];
        sc[lane] = sqrtf(fabsf(wd));
        sc[TILE + lane] = wd < 0.0f ? -1.0f : 1.0f;
        sc[2 * TILE + lane] = sqrtf(w);
    }
    __syncthreads();
    for (int b = 0; b <= M + 1; ++b) {
        const bool isD = b == M + 1;
        const int rows = isD ? K : 2 * K;
        const int N = isD ? L.NBd : L.NBm;
        const int r0 = isD ? L.D0 : b * L.Rm;
        float* Blo = Bhi + N * TILE;
        // split the block: hi in place, (s hi, s lo) into the staging rows; rows of B
        // beyond the block are zero.  e runs over the layout in memory order (row group,
        // pivot chunk, row in group, pivot in chunk); r0 is a multiple of 8, so the
        // block's element e sits at sX[r0 * 32 + e] and B's at B[e].
        for (int e = threadIdx.x; e < N * TILE; e += NTHREADS) {
            const int i = ((e >> 8) << 3) + ((e >> 2) & 7);
            const int p = (((e >> 5) & 7) << 2) + (e & 3);
            float bh = 0.0f, bl = 0.0f;
            if (i < rows) {
                const float x = sX[r0 * TILE + e] * (isD ? sc[2 * TILE + p] : sc[p]);
                const float hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
                const float sg = isD ? 1.0f : sc[TILE + p];
                sX[r0 * TILE + e] = hi;
                bh = sg * hi;
                bl = sg * (x - hi);
            }
            Bhi[e] = bh;
            Blo[e] = bl;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t idesc = tc_idesc(N);
            const uint32_t a0 = smem_u32(sX + r0 * TILE), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
            for (int k8 = 0; k8 < TILE / 8; ++k8) {
                const uint32_t o = (uint32_t)k8 * 256u;  // 8 tf32 pivots = two core matrices per MMA
                tc_mma(tc.tmem, tc_sdesc(a0 + o), tc_sdesc(bh + o), idesc, k8 > 0);
                tc_mma(tc.tmem + (uint32_t)L.NBm, tc_sdesc(a0 + o), tc_sdesc(bl + o), idesc, k8 > 0);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             tc.mbar)
                         : "memory");
            if (!tc_wait(tc.mbar, tc.phase)) {
                *tc.fail = 1;
                atomicOr(status, ST_TC_TIMEOUT);
            }
        }
        tc.phase ^= 1u;
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (*tc.fail) return;
        // C rows into the staging area (the B rows are no longer read): Cst[r][c]
        float* Cst = Bhi;
        const int r = warp * 32 + lane;
        if (warp * 32 < rows) {
            for (int c0 = 0; c0 < N; c0 += 8) {
                float v[8];
                tc_ld8(tc.tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(L.NBm + c0), v);
                if (r < rows) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) Cst[r * N + c0 + j] = v[j];
                }
            }
        }
        __syncthreads();
        if (warp * 32 < rows) {
            for (int c0 = 0; c0 < N; c0 += 8) {
                float gv[8];
                tc_ld8(tc.tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, gv);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int s2 = c0 + j;
                    if (r < rows && s2 < rows) gv[j] += Cst[r * N + s2] + Cst[s2 * N + r];
                }
                if (isD) {
                    if (r < K) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int k2 = c0 + j;
                            if (k2 >= r && k2 < K) red_add_f32(slot + 2 * nS + k2 * (k2 + 1) / 2 + r, gv[j]);
                        }
                    }
                } else {
                    float u[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) u[j] = __shfl_down_sync(0xffffffffu, gv[j], 1);
                    if ((r & 1) == 0 && r < rows) {
                        const int k1 = r >> 1;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int k2 = (c0 >> 1) + j;
                            if (k2 >= k1 && k2 < K) {
                                const int e = b * P + k2 * (k2 + 1) / 2 + k1;
                                red_add_f32(slot + 2 * e, (gv[2 * j] + u[2 * j + 1]));
                                red_add_f32(slot + 2 * e + 1, (gv[2 * j + 1] - u[2 * j]));
                            }
                        }
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (SELF) {
        const float* wd = sPiv;
        const float* wt = sPiv + TILE;
        const float* sQ = base + L.offQ;
        const float* sQW = base + L.offQW;
        for (int k = threadIdx.x; k < K; k += NTHREADS) {
            float s1 = 0.0f, s2 = 0.0f;
            for (int j = 0; j < TILE; ++j) {
                s1 = fmaf(wd[j], sQ[k * TILE + j], s1);
                s2 = fmaf(wt[j], sQW[k * TILE + j], s2);
            }
            red_add_f32(slot + 2 * nS + P + k, s1);
            red_add_f32(slot + 2 * nS + P + K + k, s2);
        }
    }
}

// One forward tile: the moments of its 32 pivots, then their partial sums added to
// the CTA's slot.  Called by every thread of the CTA (contains barriers).
template <int M, bool SELF, bool DIRECT, bool GROUPED = false>
__device__ __forceinline__ void fwd_tile(const MapDev& g, const MapCall& c, int tile, double* slot, float* smem,
                                         int mr = M) {
    const int K = g.K;
    float* sA = smem;
    float* sW = sA + (size_t)K * (mr + 1) * 2 * TILE;
    float* sQ = sW + K * TILE;
    float* sQW = sQ + K * TILE;
    float* sPiv = sQW + K * TILE;
    const int lane = threadIdx.x & 31;
    const size_t nfl = tile_floats_rt(K, mr) - 2 * TILE;
    constexpr bool grouped = GROUPED;  // shared neighbour lists (c.group > 1): own instantiation
    const int2 tq = grouped ? c.gtiles[tile] : g.tiles[tile];
    if (tq.x < 0 || tq.x >= g.nrings) {
        if (threadIdx.x == 0) atomicOr(c.status, ST_BAD_TILE);
        __syncthreads();
        return;
    }
    const PivotRing P = pivot_ring(g, tq.x);
    float2 pv = make_float2(0.0f, 0.0f);
    int qg;  // the lane's geometry; lanes past the ring's end: zero weight, valid geometry
    if (grouped) {
        // shared neighbour lists: the lane stands for the run of c.group consecutive ring
        // pixels gi, sits at the run's middle pixel and carries the run's summed weights
        const int ng = (P.n_i + c.group - 1) / c.group;
        const int gi = tq.y + lane;
        const int s0 = min(gi, ng - 1) * c.group, ln = min(c.group, P.n_i - s0);
        qg = s0 + (ln - 1) / 2;
        if (gi < ng) {
            const long long f = g.ring_first[P.i] + s0;
            for (int u = 0; u < ln; ++u) {
                const long long pix = f + u;
                if (pix >= c.piv_lo && pix < c.piv_hi) {
                    const float2 v = DIRECT ? DirectLoad{c.delta, c.w}(pix) : c.wdw[pix];
                    pv.x += v.x;
                    pv.y += v.y;
                }
            }
        }
    } else {
        const TilePivot tp = tile_pivot(tq.y, P.n_i, c.quad != 0);
        const long long pix = g.ring_first[P.i] + tp.q;
        if (tp.valid && pix >= c.piv_lo && pix < c.piv_hi)
            pv = DIRECT ? DirectLoad{c.delta, c.w}(pix) : c.wdw[pix];
        qg = tp.qg;
    }
    if (!__syncthreads_or(pv.y != 0.0f)) return;
    for (size_t e = threadIdx.x; e < nfl; e += NTHREADS) sA[e] = 0.0f;
    if (threadIdx.x < TILE) {
        sPiv[lane] = pv.x;
        sPiv[TILE + lane] = pv.y;
    }
    __syncthreads();
    if (DIRECT)
        tile_moments<M, SELF>(g, P, qg, DirectLoad{c.delta, c.w}, sA, sW, sQ, sQW, c.flush, mr,
                              !grouped && c.quad);
    else
        tile_moments<M, SELF>(g, P, qg, PackedLoad{c.wdw}, sA, sW, sQ, sQW, c.flush, mr, !grouped && c.quad);
    __syncthreads();
    if (c.norm != NORM_NONE) tile_normalize<M>(K, sA, sW, c.norm, mr);
    tile_contract<M>(K, sA, sW, sQ, sQW, sPiv, slot, SELF && c.self_subtract, mr);
    __syncthreads();
}

// One forward tile with the tensor-core contraction: the moments accumulate in the
// tensor-core layout of tc_layout(), then tile_contract_tc.
template <int M, bool SELF>
__device__ __forceinline__ void fwd_tile_tc(const MapDev& g, const MapCall& c, int tile, double* slot, float* base,
                                            TcState& tc) {
    const int K = g.K;
    const int lane = threadIdx.x & 31;
    const int2 tq = g.tiles[tile];
    if (tq.x < 0 || tq.x >= g.nrings) {
        if (threadIdx.x == 0) atomicOr(c.status, ST_BAD_TILE);
        __syncthreads();
        return;
    }
    const PivotRing P = pivot_ring(g, tq.x);
    const TilePivot tp = tile_pivot(tq.y, P.n_i, c.quad != 0);
    const long long pix = g.ring_first[P.i] + tp.q;
    const bool in = tp.valid && pix >= c.piv_lo && pix < c.piv_hi;
    float2 pv = make_float2(0.0f, 0.0f);
    if (in) pv = c.wdw[pix];
    const int qg = tp.qg;
    if (!__syncthreads_or(pv.y != 0.0f)) return;
    {
        const TcLayout L = tc_layout(K, M, SELF);
        const int nx = (L.D0 + L.RD) * TILE;
        for (int e = threadIdx.x; e < nx; e += NTHREADS) base[e] = 0.0f;
        if (SELF)
            for (int e = threadIdx.x; e < 2 * K * TILE; e += NTHREADS) base[L.offQ + e] = 0.0f;
        if (threadIdx.x < TILE) {
            base[L.offPiv + lane] = pv.x;
            base[L.offPiv + TILE + lane] = pv.y;
        }
    }
    __syncthreads();
    {
        const int Rm = (2 * K + 7) & ~7, D0 = (M + 1) * Rm;
        const TcLayout L = tc_layout(K, M, SELF);
        tile_moments_l<M, SELF>(g, P, qg, PackedLoad{c.wdw}, LayTC{base, base + L.offQ, base + L.offQW, Rm, D0},
                                c.flush, M, c.quad != 0);
    }
    __syncthreads();
    tile_contract_tc<M, SELF>(K, base, slot, tc, c.status);
    __syncthreads();
}

// OCC: CTAs per SM the register allocation is sized for (3: 80 registers, 2: 128);
// the autotuner picks the variant and the grid.
template <int M, bool SELF, bool DIRECT, int OCC = 3, bool GROUPED = false>
__global__ void __launch_bounds__(NTHREADS, OCC) map_fwd_kernel(MapDev g, MapCall c) {
    extern __shared__ float smem[];
    __shared__ int s_tile;
    double* slot = c.slots + (size_t)blockIdx.x * n_entries(g.K, M);
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(c.counter, 1);
        __syncthreads();
        const long long tile = c.tile_lo + s_tile;
        if (tile >= c.tile_hi) break;
        fwd_tile<M, SELF, DIRECT, GROUPED>(g, c, (int)tile, slot, smem);
    }
}

// The forward with the tensor-core contraction (3 CTAs per SM where the shared
// memory allows it; 128 accumulator columns each, so at most 4 fit an SM's TMEM).
template <int M, bool SELF>
__global__ void __launch_bounds__(NTHREADS, 3) map_fwd_tc_kernel(MapDev g, MapCall c) {
    extern __shared__ __align__(16) float smem_tc[];
    __shared__ int s_tile;
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ int s_fail;
    if (threadIdx.x == 0) s_fail = 0;
    tc_setup(&s_tmem, &s_mbar);
    TcState tc{s_tmem, smem_u32(&s_mbar), 0u, &s_fail};
    // the no-swizzle operand layout needs 16-byte alignment only
    float* base = smem_tc;
    double* slot = c.slots + (size_t)blockIdx.x * n_entries(g.K, M);
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(c.counter, 1);
        __syncthreads();
        const long long tile = c.tile_lo + s_tile;
        if (tile >= c.tile_hi || s_fail) break;
        fwd_tile_tc<M, SELF>(g, c, (int)tile, slot, base, tc);
    }
    tc_teardown(s_tmem);
}

// Batched forward over all the plans of a batch, one launch: one work queue over the
// concatenated tiles of all its plans (plan-major); each CTA adds into that plan's
// slot number blockIdx.x.  Compiled for the largest m_max of the batch (M); each
// plan's tiles run with its own m_max (the multipole loops stop there) and its own
// shared-memory layout, and with its own self-pair mode.
template <int M>
__global__ void __launch_bounds__(NTHREADS, 2) batch_fwd_kernel(const BatchItem* __restrict__ items, int n,
                                                               long long total, unsigned long long* counter) {
    extern __shared__ float smem[];
    __shared__ long long s_t;
    __shared__ long long s_first[TPCF_MAX_BATCH + 1];
    for (int i = threadIdx.x; i <= n; i += NTHREADS) s_first[i] = i < n ? items[i].tile0 : total;
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) s_t = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long t = s_t;
        if (t >= total) break;
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (s_first[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const BatchItem& it = items[lo];
        double* slot = it.c.slots + (size_t)blockIdx.x * n_entries(it.g.K, it.g.M);
        fwd_tile<M, true, false>(it.g, it.c, (int)(t - s_first[lo]), slot, smem, it.g.M);
    }
}

// ------------------------------------------------------------ multi-field
// Three fields A, B, C on the same pixels (end of Sec. 2, after eq. ubEstimator): a
// tile accumulates the moments a^k(i; F), W^k(i; F) of every field F in its own block
// of shared memory (three passes of the single-field walk), then adds, over the
// cyclic permutations (P, X, Y) of (A, B, C),
//     S_m(k1,k2) += sum_i w^P_i P_i a_m^{k1}(i; X) conj(a_m^{k2}(i; Y)),
//     D(k1,k2)   += sum_i w^P_i W^{k1}(i; X) W^{k2}(i; Y),
// into the CTA's FP64 slot.  These sums are not Hermitian: the slot holds the full
// K x K matrices, for m, for (k1, k2): (Re S, Im S); then D for (k1, k2).
__host__ __device__ inline size_t multi_field_floats(int K, int M) { return (size_t)K * (M + 1) * 2 * TILE + (size_t)K * TILE; }
__host__ __device__ inline size_t multi_tile_floats(int K, int M) { return 3 * multi_field_floats(K, M) + 6 * TILE; }

template <int M>
__device__ __forceinline__ void tile_contract_multi(int K, const float* sF, const float* sPiv, double* slot) {
    const size_t fsz = multi_field_floats(K, M);
    const int KK = K * K;
    const int nS = (M + 1) * KK;
    const int cyc[3][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}};
    for (int e = threadIdx.x; e < nS + KK; e += NTHREADS) {
        if (e < nS) {
            const int m = e / KK, r = e - m * KK, k1 = r / K, k2 = r - k1 * K;
            float sr = 0.0f, si = 0.0f;
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const float* wd = sPiv + cyc[t][0] * 2 * TILE;
                const float* r1 = sF + cyc[t][1] * fsz + ((size_t)k1 * (M + 1) + m) * 2 * TILE;
                const float* i1 = r1 + TILE;
                const float* r2 = sF + cyc[t][2] * fsz + ((size_t)k2 * (M + 1) + m) * 2 * TILE;
                const float* i2 = r2 + TILE;
#pragma unroll 8
                for (int j = 0; j < TILE; ++j) {
                    const int l = (j + threadIdx.x) & (TILE - 1);
                    const float a = r1[l], b = i1[l], cc = r2[l], d = i2[l];
                    sr = fmaf(wd[l], fmaf(a, cc, b * d), sr);
                    si = fmaf(wd[l], fmaf(a, d, -b * cc), si);
                }
            }
            red_add_f32(slot + 2 * e, sr);
            red_add_f32(slot + 2 * e + 1, si);
        } else {
            const int idx = e - nS, k1 = idx / K, k2 = idx - k1 * K;
            float sd = 0.0f;
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const float* wt = sPiv + cyc[t][0] * 2 * TILE + TILE;
                const float* W1 = sF + cyc[t][1] * fsz + (size_t)K * (M + 1) * 2 * TILE + k1 * TILE;
                const float* W2 = sF + cyc[t][2] * fsz + (size_t)K * (M + 1) * 2 * TILE + k2 * TILE;
                for (int j = 0; j < TILE; ++j) {
                    const int l = (j + threadIdx.x) & (TILE - 1);
                    sd = fmaf(wt[l], W1[l] * W2[l], sd);
                }
            }
            red_add_f32(slot + 2 * nS + idx, sd);
        }
    }
}

// The multi-field forward: c.wdw holds (w d, w) of field A, wdwB and wdwC those of
// B and C.  One tile at a time, as map_fwd_kernel.
template <int M>
__global__ void __launch_bounds__(NTHREADS, 2) map_fwd_multi_kernel(MapDev g, MapCall c,
                                                                    const float2* __restrict__ wdwB,
                                                                    const float2* __restrict__ wdwC) {
    extern __shared__ float smem[];
    __shared__ int s_tile;
    const int K = g.K;
    const size_t fsz = multi_field_floats(K, M);
    float* sF = smem;
    float* sPiv = smem + 3 * fsz;  // [field][w d, w][32]
    double* slot = c.slots + (size_t)blockIdx.x * n_entries_multi(K, M);
    const int lane = threadIdx.x & 31;
    const float2* arr[3] = {c.wdw, wdwB, wdwC};
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(c.counter, 1);
        __syncthreads();
        const long long tile = c.tile_lo + s_tile;
        if (tile >= c.tile_hi) break;
        const int2 tq = g.tiles[tile];
        if (tq.x < 0 || tq.x >= g.nrings) {
            if (threadIdx.x == 0) atomicOr(c.status, ST_BAD_TILE);
            __syncthreads();
            continue;
        }
        const PivotRing P = pivot_ring(g, tq.x);
        const TilePivot tp = tile_pivot(tq.y, P.n_i, true);
        const long long pix = g.ring_first[P.i] + tp.q;
        const bool in = tp.valid && pix >= c.piv_lo && pix < c.piv_hi;
        float2 pv[3];
        bool live = false;
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            pv[f] = in ? arr[f][pix] : make_float2(0.0f, 0.0f);
            live = live || pv[f].y != 0.0f;
        }
        const int qg = tp.qg;
        if (!__syncthreads_or(live)) continue;
        for (size_t e = threadIdx.x; e < 3 * fsz; e += NTHREADS) sF[e] = 0.0f;
        if (threadIdx.x < TILE) {
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                sPiv[f * 2 * TILE + lane] = pv[f].x;
                sPiv[f * 2 * TILE + TILE + lane] = pv[f].y;
            }
        }
        __syncthreads();
        for (int f = 0; f < 3; ++f) {
            float* sA = sF + f * fsz;
            tile_moments<M, false>(g, P, qg, PackedLoad{arr[f]}, sA, sA + (size_t)K * (M + 1) * 2 * TILE, nullptr,
                                   nullptr, c.flush, M, true);
        }
        __syncthreads();
        tile_contract_multi<M>(K, sF, sPiv, slot);
        __syncthreads();
    }
}

// ------------------------------------------------------------- pair count
#if defined(TPCF_M) && TPCF_M == 0  // one definition, in the M = 0 object
// counts[0] += in-bin ordered pairs (i, j) of the pivots with w_i != 0 (any w_j);
// counts[1] += those visited as mirror pairs, counts[2] += those visited singly.
// Uses the same run construction as the forward, without touching pixel data.
__global__ void __launch_bounds__(NTHREADS) map_count_kernel(MapDev g, const float2* __restrict__ wdw,
                                                             long long piv_lo, long long piv_hi,
                                                             long long tile_lo, long long tile_hi,
                                                             unsigned long long* counts) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long tile = tile_lo + blockIdx.x; tile < tile_hi; tile += gridDim.x) {
        const int2 tq = g.tiles[tile];
        const PivotRing P = pivot_ring(g, tq.x);
        const int q = tq.y + lane;
        const long long pix = g.ring_first[P.i] + q;
        const bool in = (q < P.n_i) && pix >= piv_lo && pix < piv_hi;
        const bool live = in && wdw[pix].y != 0.0f;
        if (!__syncthreads_or(live)) continue;
        const int qg = min(q, P.n_i - 1);
        unsigned long long n_sym = 0, n_plain = 0;
        for (int k = 0; k < g.K; ++k) {
            const int2 br = g.bin_range[(long long)P.i * g.K + k];
            for (int r = br.x + warp; r <= br.y; r += NWARPS) {
                const long long pr = P.pair0 + (r - P.rlo);
                const int2 Tk = g.pair_T[pr * (g.K + 1) + k];
                const int2 Tk1 = g.pair_T[pr * (g.K + 1) + k + 1];
                if (Tk.x == T_INF || Tk1.x == T_ZERO) continue;
                const int n_r = g.ring_n[r];
                const ExactCtx x = exact_ctx(g, P, r);
                const LaneC c = lane_c(qg, P.s_i, P.n_i, g.ring_shift[r], n_r);
                const bool sym = (n_r == P.n_i) && (Tk1.x != T_INF);
                const BinRuns b = bin_runs(c, Tk, Tk1, g.E[k], g.E[k + 1], x, n_r, sym);
                if (sym) {
                    n_sym += 2ull * (unsigned long long)b.n0;
                    n_plain += b.centre ? 1ull : 0ull;
                } else {
                    n_plain += (unsigned long long)(b.n0 + b.n1);
                }
            }
        }
        if (live) {
            atomicAdd(counts, n_sym + n_plain);
            atomicAdd(counts + 1, n_sym);
            atomicAdd(counts + 2, n_plain);
        }
    }
}
#endif

// ------------------------------------------------------------------ adjoint
//
// dL/d d_p for L(zeta), with C_m = (dL/dRe zeta + i dL/dIm zeta) / D and
// H_m(k,k') = conj(C_m(k,k')) + C_m(k',k) (prepared by the host side):
//   primary term      w_p * (1/2) sum_{k,m} Re[a_m^k(p) h_m^k(p)]
//   neighbour legs    w_p * sum_{i: p in nbr(i)} w_i d_i sum_m Re[e^{-i m phi_ip} h_m^{k(ip)}(i)]
//   with h_m^k(i) = sum_{k'} H_m(k,k') conj(a_m^{k'}(i)).
// A tile recomputes its a (as the forward), turns it into h in place, then sweeps its
// neighbour rings again; each warp gathers its ring's contributions in a shared-memory
// row buffer and flushes the row to the gradient with one atomic add per pixel.


// val = sum_m (cos(m phi) hr_m + sin(m phi) hi_m): X the cosine part, Y the sine part.
// h[m] = (hr_m, hi_m); the (cos, sin) chains run packed, in the folded frame psi, by
// the recurrence of harmonics(); even and odd multipoles are summed apart and the odd
// sum takes the sign sigma at the end.
template <int M>
__device__ __forceinline__ void adj_harmonicsf(const float2 (&h)[M + 1], const Fold& f, float& X, float& Y,
                                               int mr = M) {
    float2 ev = make_float2(h[0].x, 0.0f);
    float2 od = make_float2(0.0f, 0.0f);
    float sg = 1.0f;
    if constexpr (M >= 1) {
        if (mr < 1) {
            X = ev.x;
            Y = ev.y;
            return;
        }
        sg = f.sg;
        float2 T = make_float2(f.ac, f.ss);
        float2 D = make_float2(0.5f * f.lam, f.ss);
        const float2 L2 = make_float2(f.lam, f.lam);
        od = __ffma2_rn(T, h[1], od);
#pragma unroll
        for (int m = 2; m <= M; ++m) {
            if (m > mr) break;
            D = __ffma2_rn(L2, T, D);
            T = __fadd2_rn(T, D);
            if (m & 1)
                od = __ffma2_rn(T, h[m], od);
            else
                ev = __ffma2_rn(T, h[m], ev);
        }
    }
    X = fmaf(sg, od.x, ev.x);
    Y = fmaf(sg, od.y, ev.y);
}

template <int M>
__device__ __forceinline__ void adj_harmonics(const float2 (&h)[M + 1], float cph, float sph, float& X, float& Y,
                                              int mr = M) {
    adj_harmonicsf<M>(h, fold_angle(cph, sph), X, Y, mr);
}

// Where the contribution to pixel p (unwrapped index on ring R) goes.
struct RowSink {
    float* buf;     // warp row buffer, or NULL for direct global adds
    int lo;         // buffer index = p - lo (window mode) ...
    bool whole;     // ... or = wrap(p) (whole-ring mode)
    float* grad;    // gradient row base (grad + first of ring)
    int n;
};

__device__ __forceinline__ void sink_add(const RowSink& s, int p_unwrapped, int p_wrapped, float v) {
    if (s.buf) {
        atomicAdd(s.buf + (s.whole ? p_wrapped : p_unwrapped - s.lo), v);
    } else {
        atomicAdd(s.grad + p_wrapped, v);
    }
}

template <int M>
__device__ __forceinline__ void adj_harmonics2f(const float2 (&h)[M + 1], const Fold& fa, const Fold& fb, float& Xa,
                                                float& Ya, float& Xb, float& Yb, int mr = M) {
    float2 eva = make_float2(h[0].x, 0.0f), evb = eva;
    float2 oda = make_float2(0.0f, 0.0f), odb = oda;
    float sga = 1.0f, sgb = 1.0f;
    if constexpr (M >= 1) {
        if (mr < 1) {
            Xa = Xb = eva.x;
            Ya = Yb = eva.y;
            return;
        }
        sga = fa.sg;
        sgb = fb.sg;
        float2 Ta = make_float2(fa.ac, fa.ss), Da = make_float2(0.5f * fa.lam, fa.ss);
        float2 Tb = make_float2(fb.ac, fb.ss), Db = make_float2(0.5f * fb.lam, fb.ss);
        const float2 La = make_float2(fa.lam, fa.lam), Lb = make_float2(fb.lam, fb.lam);
        oda = __ffma2_rn(Ta, h[1], oda);
        odb = __ffma2_rn(Tb, h[1], odb);
#pragma unroll
        for (int m = 2; m <= M; ++m) {
            if (m > mr) break;
            Da = __ffma2_rn(La, Ta, Da);
            Db = __ffma2_rn(Lb, Tb, Db);
            Ta = __fadd2_rn(Ta, Da);
            Tb = __fadd2_rn(Tb, Db);
            if (m & 1) {
                oda = __ffma2_rn(Ta, h[m], oda);
                odb = __ffma2_rn(Tb, h[m], odb);
            } else {
                eva = __ffma2_rn(Ta, h[m], eva);
                evb = __ffma2_rn(Tb, h[m], evb);
            }
        }
    }
    Xa = fmaf(sga, oda.x, eva.x);
    Ya = fmaf(sga, oda.y, eva.y);
    Xb = fmaf(sgb, odb.x, evb.x);
    Yb = fmaf(sgb, odb.y, evb.y);
}

template <int M>
__device__ __forceinline__ void adj_harmonics2(const float2 (&h)[M + 1], float ca, float sa, float cb, float sb,
                                               float& Xa, float& Ya, float& Xb, float& Yb, int mr = M) {
    adj_harmonics2f<M>(h, fold_angle(ca, sa), fold_angle(cb, sb), Xa, Ya, Xb, Yb, mr);
}

template <int M, bool FAST, bool SELF = false>
__device__ __forceinline__ void adj_run(const RingCtx& R, const float2* __restrict__ wdw, const LaneC& c,
                                        int a, int len, const float2 (&h)[M + 1], float wdi, const RowSink& s,
                                        float ck = 0.0f, int mr = M) {
    const int maxlen = __reduce_max_sync(0xffffffffu, len);
    const float i0 = (float)(a - c.cint);
    const float xneg = -c.cfrac * R.step, uneg = -c.cfrac * R.inv_n;
    int idx = wrap_idx(a, R.n);
    const float2* row = wdw + R.first;
    for (int t = 0; t < maxlen; t += 2) {
        const bool on0 = t < len, on1 = t + 1 < len;
        const int idx1 = idx + 1 >= R.n ? idx + 1 - R.n : idx + 1;
        const float2 v0 = on0 ? __ldg(row + idx) : make_float2(0.0f, 0.0f);
        const float2 v1 = on1 ? __ldg(row + idx1) : make_float2(0.0f, 0.0f);
        const float oa = on0 ? i0 + (float)t : i0;
        const float ob = on1 ? i0 + (float)(t + 1) : i0;
        float ca, sa, cb, sb, Xa, Ya, Xb, Yb;
        pixel_dir<FAST>(oa, xneg, uneg, R, ca, sa);
        pixel_dir<FAST>(ob, xneg, uneg, R, cb, sb);
        adj_harmonics2<M>(h, ca, sa, cb, sb, Xa, Ya, Xb, Yb, mr);
        if (SELF) {  // self-pair subtraction: -2 cdiag_k (w_p d_p) per neighbour p
            Xa = fmaf(ck, v0.x, Xa);
            Xb = fmaf(ck, v1.x, Xb);
        }
        if (on0) sink_add(s, a + t, idx, wdi * v0.y * (Xa + Ya));
        if (on1) sink_add(s, a + t + 1, idx1, wdi * v1.y * (Xb + Yb));
        idx = idx1 + 1 >= R.n ? idx1 + 1 - R.n : idx1 + 1;
    }
}

template <int M, bool FAST, bool SELF = false>
__device__ __forceinline__ void adj_pairs(const RingCtx& R, const float2* __restrict__ wdw, const LaneC& c,
                                          int a, int len, int mb, const float2 (&h)[M + 1], float wdi,
                                          const RowSink& s, float ck = 0.0f, int mr = M) {
    const int maxlen = __reduce_max_sync(0xffffffffu, len);
    const float i0 = (float)(a - c.cint);
    const float xneg = -c.cfrac * R.step, uneg = -c.cfrac * R.inv_n;
    int ip = wrap_idx(a, R.n);
    int im_ = wrap_idx(mb - a, R.n);
    const float2* row = wdw + R.first;
    for (int t = 0; t < maxlen; t += 2) {
        const bool on0 = t < len, on1 = t + 1 < len;
        const int ip1 = ip + 1 >= R.n ? ip + 1 - R.n : ip + 1;
        const int im1 = im_ - 1 < 0 ? im_ - 1 + R.n : im_ - 1;
        const float2 p0 = on0 ? __ldg(row + ip) : make_float2(0.0f, 0.0f);
        const float2 m0 = on0 ? __ldg(row + im_) : make_float2(0.0f, 0.0f);
        const float2 p1 = on1 ? __ldg(row + ip1) : make_float2(0.0f, 0.0f);
        const float2 m1 = on1 ? __ldg(row + im1) : make_float2(0.0f, 0.0f);
        const float oa = on0 ? i0 + (float)t : i0;
        const float ob = on1 ? i0 + (float)(t + 1) : i0;
        float ca, sa, cb, sb, Xa, Ya, Xb, Yb;
        pixel_dir<FAST>(oa, xneg, uneg, R, ca, sa);
        pixel_dir<FAST>(ob, xneg, uneg, R, cb, sb);
        adj_harmonics2<M>(h, ca, sa, cb, sb, Xa, Ya, Xb, Yb, mr);
        if (on0) {
            sink_add(s, a + t, ip, wdi * p0.y * (Xa + Ya + (SELF ? ck * p0.x : 0.0f)));
            sink_add(s, mb - a - t, im_, wdi * m0.y * (Xa - Ya + (SELF ? ck * m0.x : 0.0f)));
        }
        if (on1) {
            sink_add(s, a + t + 1, ip1, wdi * p1.y * (Xb + Yb + (SELF ? ck * p1.x : 0.0f)));
            sink_add(s, mb - a - t - 1, im1, wdi * m1.y * (Xb - Yb + (SELF ? ck * m1.x : 0.0f)));
        }
        ip = ip1 + 1 >= R.n ? ip1 + 1 - R.n : ip1 + 1;
        im_ = im1 - 1 < 0 ? im1 - 1 + R.n : im1 - 1;
    }
}

// adj_pairs for a belt ring pair, with the position angles shared across the warp
// (see walk_pairs_shared).
template <int M, bool SELF = false>
__device__ __forceinline__ void adj_pairs_shared(const RingCtx& R, const float2* __restrict__ wdw, const LaneC& c,
                                                 int a, int len, int mb, const float2 (&h)[M + 1], float wdi,
                                                 const RowSink& s, float ck = 0.0f, int mr = M) {
    if (len <= 0) return;
    const int lane = threadIdx.x & 31;
    const float i0 = (float)(a - c.cint);
    const float xneg = -c.cfrac * R.step, uneg = -c.cfrac * R.inv_n;
    int ip = wrap_idx(a, R.n);
    int im_ = wrap_idx(mb - a, R.n);
    const float2* row = wdw + R.first;
    for (int t0 = 0; t0 < len; t0 += 32) {
        Fold mine;
        {
            const float ft = i0 + (float)(t0 + lane);
            float cph, sph;
            if (fabsf(ft - c.cfrac) * R.step <= FAST_XMAX)
                pixel_dir<true>(ft, xneg, uneg, R, cph, sph);
            else
                pixel_dir<false>(ft, xneg, uneg, R, cph, sph);
            mine = fold_angle(cph, sph);
        }
        const int nstep = min(32, len - t0);
        for (int tt = 0; tt < nstep; tt += 2) {
            const int t = t0 + tt;
            const bool two = tt + 1 < nstep;
            const Fold fa = shfl_fold(mine, tt), fb = shfl_fold(mine, two ? tt + 1 : tt);
            const int ip1 = ip + 1 >= R.n ? ip + 1 - R.n : ip + 1;
            const int im1 = im_ - 1 < 0 ? im_ - 1 + R.n : im_ - 1;
            const float2 p0 = __ldg(row + ip), m0 = __ldg(row + im_);
            const float2 p1 = two ? __ldg(row + ip1) : make_float2(0.0f, 0.0f);
            const float2 m1 = two ? __ldg(row + im1) : make_float2(0.0f, 0.0f);
            float Xa, Ya, Xb, Yb;
            adj_harmonics2f<M>(h, fa, fb, Xa, Ya, Xb, Yb, mr);
            sink_add(s, a + t, ip, wdi * p0.y * (Xa + Ya + (SELF ? ck * p0.x : 0.0f)));
            sink_add(s, mb - a - t, im_, wdi * m0.y * (Xa - Ya + (SELF ? ck * m0.x : 0.0f)));
            if (two) {
                sink_add(s, a + t + 1, ip1, wdi * p1.y * (Xb + Yb + (SELF ? ck * p1.x : 0.0f)));
                sink_add(s, mb - a - t - 1, im1, wdi * m1.y * (Xb - Yb + (SELF ? ck * m1.x : 0.0f)));
            }
            ip = ip1 + 1 >= R.n ? ip1 + 1 - R.n : ip1 + 1;
            im_ = im1 - 1 < 0 ? im1 - 1 + R.n : im1 - 1;
        }
    }
}

// Neighbour legs of one ring r for the warp's lanes (all bins of r).
template <int M, bool SELF = false>
__device__ __forceinline__ void adj_ring(const MapDev& g, const PivotRing& P, int r, int q, float wdi,
                                         const float2* __restrict__ wdw, const float* sH, float* rowbuf,
                                         float* grad, int* status,
                                         const float* cdiag = nullptr, int mr = M) {
    const int lane = threadIdx.x & 31;
    const long long pr = P.pair0 + (r - P.rlo);
    const int2 TK = g.pair_T[pr * (g.K + 1) + g.K];
    if (TK.x == T_ZERO) return;
    const RingCtx R = ring_ctx(g, P, r, pr);
    const ExactCtx x = exact_ctx(g, P, r);
    const LaneC c = lane_c(q, P.s_i, P.n_i, R.shift, R.n);
    // row window: every pixel of r within the outer edge of some lane's pivot
    RowSink s;
    s.grad = grad + R.first;
    s.n = R.n;
    s.whole = false;
    s.lo = 0;
    s.buf = rowbuf;
    int width;
    {
        const int clo = __shfl_sync(0xffffffffu, c.cint, 0);
        const int chi = __shfl_sync(0xffffffffu, c.cint, 31);
        if (TK.x != T_INF) {
            s.lo = clo - TK.x - 2;
            width = chi + TK.x + 3 - s.lo + 1;
        } else {
            width = ROW + 1;
        }
        if (width > ROW || width >= R.n) {
            if (R.n <= ROW) {
                s.whole = true;
                width = R.n;
            } else {
                s.buf = nullptr;
                width = 0;
                if (lane == 0) atomicOr(status, ST_ROW_OVERFLOW);
            }
        }
    }
    for (int e = lane; e < width; e += 32) rowbuf[e] = 0.0f;
    __syncwarp();
    for (int k = 0; k < g.K; ++k) {
        const int2 br = g.bin_range[(long long)P.i * g.K + k];
        if (r < br.x || r > br.y) continue;
        const int2 Tk = g.pair_T[pr * (g.K + 1) + k];
        const int2 Tk1 = g.pair_T[pr * (g.K + 1) + k + 1];
        if (Tk.x == T_INF || Tk1.x == T_ZERO) continue;
        float2 h[M + 1];
        const float* hk = sH + (size_t)k * (mr + 1) * 2 * TILE;
#pragma unroll
        for (int m = 0; m <= M; ++m) {
            h[m] = m <= mr ? make_float2(hk[(2 * m) * TILE + lane], hk[(2 * m + 1) * TILE + lane])
                           : make_float2(0.0f, 0.0f);
        }
        const bool sym = (R.n == P.n_i) && (Tk1.x != T_INF);
        const BinRuns b = bin_runs(c, Tk, Tk1, g.E[k], g.E[k + 1], x, R.n, sym);
        const float ck = SELF ? -2.0f * cdiag[k] : 0.0f;
        if (sym) {
            if (b.centre) {
                const int p = c.cint;
                const int pw = wrap_idx(p, R.n);
                const float2 v = __ldg(wdw + R.first + pw);
                float cph, sph, X, Y;
                pixel_dir<false>(0.0f, 0.0f, -c.cfrac * R.inv_n, R, cph, sph);
                adj_harmonics<M>(h, cph, sph, X, Y, mr);
                if (SELF) X = fmaf(ck, v.x, X);
                sink_add(s, p, pw, wdi * v.y * (X + Y));
            }
            if (runs_shared(c, b.a0, b.n0)) {
                adj_pairs_shared<M, SELF>(R, wdw, c, b.a0, b.n0, b.mb, h, wdi, s, ck, mr);
            } else {
                const bool fast = __all_sync(0xffffffffu, run_omax(c, b.a0, b.n0) * R.step <= FAST_XMAX);
                if (fast)
                    adj_pairs<M, true, SELF>(R, wdw, c, b.a0, b.n0, b.mb, h, wdi, s, ck, mr);
                else
                    adj_pairs<M, false, SELF>(R, wdw, c, b.a0, b.n0, b.mb, h, wdi, s, ck, mr);
            }
        } else {
            const float om = fmaxf(run_omax(c, b.a0, b.n0), run_omax(c, b.a1, b.n1));
            const bool fast = __all_sync(0xffffffffu, om * R.step <= FAST_XMAX);
            if (fast) {
                adj_run<M, true, SELF>(R, wdw, c, b.a0, b.n0, h, wdi, s, ck, mr);
                adj_run<M, true, SELF>(R, wdw, c, b.a1, b.n1, h, wdi, s, ck, mr);
            } else {
                adj_run<M, false, SELF>(R, wdw, c, b.a0, b.n0, h, wdi, s, ck, mr);
                adj_run<M, false, SELF>(R, wdw, c, b.a1, b.n1, h, wdi, s, ck, mr);
            }
        }
    }
    __syncwarp();
    if (s.buf) {
        for (int e = lane; e < width; e += 32) {
            const float v = rowbuf[e];
            if (v != 0.0f) {
                const int pw = s.whole ? e : wrap_idx(s.lo + e, R.n);
                atomicAdd(s.grad + pw, v);
            }
        }
        __syncwarp();
    }
}

// Shared memory of an adjoint tile: phases 1-2 use the moments A, W, Q, QW, the
// pivot values, the primary-term sums and one m of H; phase 3 keeps only A (now h)
// and puts the warps' row buffers where W and the rest were.
template <int M>
__host__ __device__ inline size_t bwd_tile_floats(int K) {
    return bwd_tile_floats_rt(K, M);
}

// One adjoint tile (all three phases).  Called by every thread of the CTA.  With
// SELF (self-pair subtraction) the subtracted diagonal adds, per bin k with
// cdiag_k = sum_m Re C_m(k,k), -w_p Q^k(p) cdiag_k to a pivot and
// -2 w_p^2 d_p w_i d_i cdiag_k to each neighbour p of pivot i.
template <int M, bool SELF = false>
__device__ __forceinline__ void bwd_tile(const MapDev& g, const MapCall& c, int tile, float* smem, int mr = M) {
    const int K = g.K;
    float* sA = smem;
    float* sW = sA + (size_t)K * (mr + 1) * 2 * TILE;
    float* sQ = sW + K * TILE;
    float* sQW = sQ + K * TILE;
    float* sPiv = sQW + K * TILE;
    float* sPrim = sPiv + 2 * TILE;
    float* sHm = sPrim + TILE;                  // [K][K][2] one m at a time
    float* sRow = sW;                           // [NWARPS][ROW], phase 3 only
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t nfl = (size_t)K * (mr + 1) * 2 * TILE + 3 * (size_t)K * TILE;

    const int2 tq = g.tiles[tile];
    if (tq.x < 0 || tq.x >= g.nrings) {
        if (threadIdx.x == 0) atomicOr(c.status, ST_BAD_TILE);
        __syncthreads();
        return;
    }
    const PivotRing P = pivot_ring(g, tq.x);
    const int q = tq.y + lane;
    const long long pix = g.ring_first[P.i] + q;
    const bool in = (q < P.n_i) && pix >= c.piv_lo && pix < c.piv_hi;
    const float2 pv = in ? c.wdw[pix] : make_float2(0.0f, 0.0f);
    const int qg = min(q, P.n_i - 1);  // see map_fwd_kernel
    if (!__syncthreads_or(pv.y != 0.0f)) return;  // no pivot with w != 0: no term
    for (size_t e = threadIdx.x; e < nfl; e += NTHREADS) sA[e] = 0.0f;
    if (threadIdx.x < TILE) {
        sPiv[lane] = pv.x;
        sPiv[TILE + lane] = pv.y;
        sPrim[lane] = 0.0f;
    }
    __syncthreads();
    // phase 1: the tile's moments, exactly as in the forward
    tile_moments<M, SELF>(g, P, qg, PackedLoad{c.wdw}, sA, sW, sQ, sQW, c.flush, mr);
    __syncthreads();
    // phase 2: h = H conj(a) per m, in place; primary term (1/2) sum Re[a h]
    for (int m = 0; m <= mr; ++m) {
        for (int e = threadIdx.x; e < K * K * 2; e += NTHREADS)
            sHm[e] = c.H[(size_t)m * K * K * 2 + e];
        __syncthreads();
        float hrv[(TPCF_MAX_BINS * TILE + NTHREADS - 1) / NTHREADS];
        float hiv[(TPCF_MAX_BINS * TILE + NTHREADS - 1) / NTHREADS];
        int nmine = 0;
        for (int e = threadIdx.x; e < K * TILE; e += NTHREADS, ++nmine) {
            const int k = e / TILE, l = e - k * TILE;
            float hr = 0.0f, hi = 0.0f;
            for (int kp = 0; kp < K; ++kp) {
                const float Hr = sHm[(k * K + kp) * 2], Hi = sHm[(k * K + kp) * 2 + 1];
                const float* ap = sA + ((size_t)kp * (mr + 1) + m) * 2 * TILE;
                const float tr = ap[l], ti = ap[TILE + l];
                hr = fmaf(Hr, tr, fmaf(-Hi, ti, hr));
                hi = fmaf(Hr, ti, fmaf(Hi, tr, hi));
            }
            const float* ak = sA + ((size_t)k * (mr + 1) + m) * 2 * TILE;
            atomicAdd(sPrim + l, fmaf(ak[l], hr, ak[TILE + l] * hi));
            hrv[nmine] = hr;
            hiv[nmine] = hi;
        }
        __syncthreads();
        nmine = 0;
        for (int e = threadIdx.x; e < K * TILE; e += NTHREADS, ++nmine) {
            const int k = e / TILE, l = e - k * TILE;
            float* ak = sA + ((size_t)k * (mr + 1) + m) * 2 * TILE;
            ak[l] = hrv[nmine];
            ak[TILE + l] = hiv[nmine];
        }
        __syncthreads();
    }
    const float* cdiag = SELF ? c.H + (size_t)(mr + 1) * K * K * 2 : nullptr;
    if (threadIdx.x < TILE && in) {
        float gp = 0.5f * pv.y * sPrim[lane];
        if (SELF) {
            float t = 0.0f;
            for (int k = 0; k < K; ++k) t = fmaf(cdiag[k], sQ[k * TILE + lane], t);
            gp = fmaf(-pv.y, t, gp);
        }
        if (gp != 0.0f) atomicAdd(c.grad + pix, gp);
    }
    __syncthreads();  // the row buffers of phase 3 overlay sPrim and the rest
    // phase 3: neighbour legs, warps split the neighbour rings
    const int2 rr = g.ring_range[P.i];
    for (int r = rr.x + warp; r <= rr.y; r += NWARPS)
        adj_ring<M, SELF>(g, P, r, qg, pv.x, c.wdw, sA, sRow + (size_t)warp * ROW, c.grad, c.status, cdiag, mr);
    __syncthreads();
}

template <int M, bool SELF, int OCC = 3>
__global__ void __launch_bounds__(NTHREADS, OCC) map_bwd_kernel(MapDev g, MapCall c) {
    extern __shared__ float smem[];
    __shared__ int s_tile;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(c.counter, 1);
        __syncthreads();
        const long long tile = c.tile_lo + s_tile;
        if (tile >= c.tile_hi) break;
        bwd_tile<M, SELF>(g, c, (int)tile, smem);
    }
}

template <int M>
__global__ void __launch_bounds__(NTHREADS, 2) batch_bwd_kernel(const BatchItem* __restrict__ items, int n,
                                                               long long total, unsigned long long* counter) {
    extern __shared__ float smem[];
    __shared__ long long s_t;
    __shared__ long long s_first[TPCF_MAX_BATCH + 1];
    for (int i = threadIdx.x; i <= n; i += NTHREADS) s_first[i] = i < n ? items[i].tile0 : total;
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) s_t = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long t = s_t;
        if (t >= total) break;
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (s_first[mid] <= t) lo = mid; else hi = mid - 1;
        }
        bwd_tile<M>(items[lo].g, items[lo].c, (int)(t - s_first[lo]), smem, items[lo].g.M);
    }
}

}  // namespace tpcf
