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

}  // namespace dfl
}  // namespace ww
