// ww_df.cuh -- double-float ("float-float") arithmetic and a shared-memory
// FFT in it, for the spectral kernels of the mixed-precision form.
//
// GB300 executes FP32 at 64x the FP64 rate (2 FP64 FMA per clock per SM).
// A double-float value is an unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2, i.e. a 48-bit significand.  Sums and products are built
// from the classical error-free transformations (Knuth's TwoSum, Dekker's
// FastTwoSum, and the FMA-based TwoProduct), so every operation has a
// relative error of a few 2^-48.  A radix-2 butterfly costs ~94 FP32
// instructions against 8 FP64 ones: ~5x faster on this part.  Inputs and
// outputs of the kernels stay FP64; only the transforms run in double-float.
#pragma once

#include <cuda_runtime.h>

namespace ww {
namespace dfl {

struct df {
    float hi, lo;
};

struct cdf {   // complex double-float, 16 bytes like a double2
    float rh, rl, ih, il;
};

// The error-free transformations need every sum and product rounded on its
// own: the _rn intrinsics are never contracted into FMAs by the compiler
// (a contracted p + e with p = a*b silently breaks TwoProduct/FastTwoSum).
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df sub(df a, df b) { return add(a, df{-b.hi, -b.lo}); }

__device__ __forceinline__ df mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ df mulf(df a, float b) {   // b exact in float
    const float p = __fmul_rn(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ df from_double(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

__device__ __forceinline__ double to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ cdf make(df re, df im) { return {re.hi, re.lo, im.hi, im.lo}; }
__device__ __forceinline__ df re(cdf z) { return {z.rh, z.rl}; }
__device__ __forceinline__ df im(cdf z) { return {z.ih, z.il}; }

__device__ __forceinline__ cdf cadd(cdf a, cdf b) { return make(add(re(a), re(b)), add(im(a), im(b))); }
__device__ __forceinline__ cdf csub(cdf a, cdf b) { return make(sub(re(a), re(b)), sub(im(a), im(b))); }
__device__ __forceinline__ cdf cmul(cdf a, cdf w) {
    return make(sub(mul(re(a), re(w)), mul(im(a), im(w))), add(mul(re(a), im(w)), mul(im(a), re(w))));
}
__device__ __forceinline__ cdf cscale(cdf a, df s) { return make(mul(re(a), s), mul(im(a), s)); }
__device__ __forceinline__ cdf cscalef(cdf a, float s) { return make(mulf(re(a), s), mulf(im(a), s)); }
__device__ __forceinline__ cdf times_ik(cdf z, int k) {   // (ik) z, k exact in float
    return make(mulf(im(z), -(float)k), mulf(re(z), (float)k));
}
__device__ __forceinline__ cdf from_d2(double2 z) { return make(from_double(z.x), from_double(z.y)); }
__device__ __forceinline__ double2 to_d2(cdf z) { return make_double2(to_double(re(z)), to_double(im(z))); }

// In-place complex FFT of length N = 2^logN in shared memory, whole block,
// radix-2 decimation in time after a bit-reversal permutation; twiddles
// twd[k] = exp(-2 pi i k/N) (k < N/2) in double-float.  Unscaled inverse.
__device__ __forceinline__ void block_fft(cdf *s, int N, int logN, const cdf *__restrict__ twd, bool inverse) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        int j = (int)(__brev((unsigned)i) >> (32 - logN));
        if (i < j) {
            cdf t = s[i];
            s[i] = s[j];
            s[j] = t;
        }
    }
    __syncthreads();
    const int halfN = N >> 1;
    for (int lh = 0; lh < logN; ++lh) {
        const int half = 1 << lh;
        const int tshift = logN - 1 - lh;
        for (int b = threadIdx.x; b < halfN; b += blockDim.x) {
            const int k = b & (half - 1);
            const int i0 = ((b >> lh) << (lh + 1)) + k;
            const int i1 = i0 + half;
            cdf w = twd[k << tshift];
            if (inverse) {
                w.ih = -w.ih;
                w.il = -w.il;
            }
            const cdf v = cmul(s[i1], w);
            const cdf u = s[i0];
            s[i0] = cadd(u, v);
            s[i1] = csub(u, v);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Stockham FFT in double-float: radix-8 passes (one radix-4 or radix-2 pass
// last when log2 N is not a multiple of 3), each thread taking R points into
// registers, applying the inter-pass twiddles and an R-point DFT, and writing
// them back; natural order in and out, no bit reversal.  Every pass reads all
// its points before a barrier and writes after it, so it runs in place.  The
// intermediate passes use a padded layout (one 16-byte slot every 8 points:
// the first pass writes each thread's 8 outputs contiguously, which the
// padding spreads over all banks), so s needs room for N + N/8 points.
// Stockham's formulation (Stockham 1966; the GPU form of Govindaraju et al.,
// SC 2008):  pass with sub-transform length L (1, R, R^2, ..): thread j reads
// x[j + r N/R], multiplies by W_{L R}^{(j mod L) r}, takes the R-point DFT and
// writes y[(j / L) L R + (j mod L) + r L].
// ---------------------------------------------------------------------------
constexpr double kRsqrt2 = 0.70710678118654752440084436210484903928;

__device__ __forceinline__ df neg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ cdf cneg(cdf a) { return cdf{-a.rh, -a.rl, -a.ih, -a.il}; }
// (-i) z for the forward transform, (+i) z for the inverse
template <bool INV>
__device__ __forceinline__ cdf mul_mi(cdf z) {
    return INV ? cdf{-z.ih, -z.il, z.rh, z.rl} : cdf{z.ih, z.il, -z.rh, -z.rl};
}
// z * (1 -+ i)/sqrt2  (forward: W8^1 = (1 - i)/sqrt2; inverse: its conjugate)
template <bool INV>
__device__ __forceinline__ cdf mul_w8(cdf z) {
    const df c{(float)kRsqrt2, (float)(kRsqrt2 - (double)(float)kRsqrt2)};
    const df a = re(z), b = im(z);
    // forward: ((a + b) + i (b - a)) / sqrt2 ; inverse: ((a - b) + i (a + b)) / sqrt2
    return INV ? make(mul(sub(a, b), c), mul(add(a, b), c)) : make(mul(add(a, b), c), mul(sub(b, a), c));
}

template <bool INV>
__device__ __forceinline__ void dft4(cdf &x0, cdf &x1, cdf &x2, cdf &x3) {
    const cdf t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), t3 = mul_mi<INV>(csub(x1, x3));
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = cadd(t1, t3);
    x3 = csub(t1, t3);
}

// v[k] <- sum_r v[r] W8^{rk}
template <bool INV>
__device__ __forceinline__ void dft8(cdf *v) {
    cdf e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    cdf o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    o1 = mul_w8<INV>(o1);
    o2 = mul_mi<INV>(o2);
    o3 = mul_mi<INV>(mul_w8<INV>(o3));   // W8^3 = W8^1 W8^2
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

__device__ __forceinline__ int pad8(int i) { return i + (i >> 3); }

// W_N^m for 0 <= m < N from the half table twd[k] = exp(-2 pi i k/N), k < N/2
template <bool INV>
__device__ __forceinline__ cdf twiddle(const cdf *__restrict__ twd, int m, int halfN) {
    cdf w = m < halfN ? twd[m] : cneg(twd[m - halfN]);
    if (INV) {
        w.ih = -w.ih;
        w.il = -w.il;
    }
    return w;
}

// The twiddles of one pass with sub-transform length L, W_{L R}^{k r} for
// r = 1..R-1 and k < L, stored row by row: tp[(r - 1) L + k] (forward sign).
// Threads of a warp read consecutive k, i.e. consecutive addresses, so the
// reads from shared memory are free of bank conflicts.
template <bool INV, int R>
__device__ __forceinline__ void stockham_pass(cdf *s, int N, int L, bool pad_in, bool pad_out,
                                              const cdf *tp) {
    // each thread holds up to MAXC groups of R points (N <= 2048 with 256 threads)
    constexpr int MAXC = (R == 8) ? 1 : 2;
    const int NR = N / R;
    cdf v[MAXC][R];
#pragma unroll
    for (int c = 0; c < MAXC; ++c) {
        const int j = c * blockDim.x + threadIdx.x;
        if (j < NR) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = j + r * NR;
                v[c][r] = s[pad_in ? pad8(i) : i];
            }
            const int k = j % L;
            if (k != 0) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    cdf w = tp[(r - 1) * L + k];
                    if (INV) {
                        w.ih = -w.ih;
                        w.il = -w.il;
                    }
                    v[c][r] = cmul(v[c][r], w);
                }
            }
            if (R == 8)
                dft8<INV>(v[c]);
            else
                dft4<INV>(v[c][0], v[c][1], v[c][2], v[c][3]);
        }
    }
    __syncthreads();   // every point of this pass read before any is overwritten
#pragma unroll
    for (int c = 0; c < MAXC; ++c) {
        const int j = c * blockDim.x + threadIdx.x;
        if (j < NR) {
            const int base = (j / L) * L * R + (j % L);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int o = base + r * L;
                s[pad_out ? pad8(o) : o] = v[c][r];
            }
        }
    }
    __syncthreads();
}

// In-place FFT of s[0..N) (natural order in and out), 16 <= N = 2^logN <= 2048
// and blockDim.x == 256 (FFT_STOCKHAM_MAXN), s with room for N + N/8 points,
// twiddles from the per-pass tables of build_stockham_twiddles; unscaled
// inverse.  Radix-8 passes, and one or two radix-4 passes when
// log2 N is not a multiple of 3.  Callers synchronise before (the data is
// complete); the routine ends with a barrier.
constexpr int FFT_STOCKHAM_MAXN = 2048;

// not inlined: the kernels call it 5-7 times and one copy of each direction's
// code keeps the instruction cache warm; one function per direction keeps the
// register footprint of each to its own passes
// the passes of a Stockham transform of 2^logN points: radix-8 ones, then n4 radix-4
__host__ __device__ __forceinline__ int stockham_n4(int logN) { return (logN % 3 == 0) ? 0 : (logN % 3 == 2 ? 1 : 2); }
__host__ __device__ __forceinline__ int stockham_n8(int logN) { return (logN - 2 * stockham_n4(logN)) / 3; }

// entries of the per-pass twiddle tables of a transform of N = 2^logN points:
// (R - 1) L per pass with sub-transform length L (fewer than N in all)
__host__ __device__ __forceinline__ int stockham_table_size(int logN) {
    const int n4 = stockham_n4(logN), n8 = stockham_n8(logN);
    int L = 1, total = 0;
    for (int pi = 0; pi < n4 + n8; ++pi) {
        const int R = pi < n8 ? 8 : 4;
        total += (R - 1) * L;
        L *= R;
    }
    return total;
}

// the per-pass tables (stockham_pass) built by the whole block from the
// half table twd[m] = exp(-2 pi i m / N), m < N/2 (global memory)
__device__ __forceinline__ void build_stockham_twiddles(const cdf *__restrict__ twd, cdf *dst, int N, int logN) {
    const int n4 = stockham_n4(logN), n8 = stockham_n8(logN), halfN = N >> 1;
    int L = 1;
    for (int pi = 0; pi < n4 + n8; ++pi) {
        const int R = pi < n8 ? 8 : 4;
        const int tstride = N / (L * R);   // W_{L R}^{k r} = W_N^{k r N / (L R)}
        for (int e = threadIdx.x; e < (R - 1) * L; e += blockDim.x) {
            const int r = e / L + 1, k = e % L;
            dst[e] = twiddle<false>(twd, k * r * tstride, halfN);
        }
        dst += (R - 1) * L;
        L *= R;
    }
}

// tp: the per-pass tables of build_stockham_twiddles (shared memory)
template <bool INV>
static __device__ __noinline__ void stockham_fft(cdf *s, int N, int logN, const cdf *tp) {
    const int n4 = stockham_n4(logN), n8 = stockham_n8(logN);
    const int npass = n4 + n8;
    int L = 1;
    for (int pi = 0; pi < npass; ++pi) {
        const bool r8 = pi < n8;
        const bool pin = pi > 0, pout = pi < npass - 1;
        if (r8)
            stockham_pass<INV, 8>(s, N, L, pin, pout, tp);
        else
            stockham_pass<INV, 4>(s, N, L, pin, pout, tp);
        tp += (r8 ? 7 : 3) * L;
        L *= r8 ? 8 : 4;
    }
}

static __device__ __forceinline__ void block_fft_stockham(cdf *s, int N, int logN, const cdf *tp, bool inverse) {
    if (inverse)
        stockham_fft<true>(s, N, logN, tp);
    else
        stockham_fft<false>(s, N, logN, tp);
}

}  // namespace dfl
}  // namespace ww
