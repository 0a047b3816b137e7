// ww_ar.cuh -- the arithmetic of the one-CTA shared-memory transforms and the
// pointwise algebra around them: ArF64 (IEEE double, the WW_FP64 form) and
// ArDF (double-float, the WW_MIXED form's variational columns), plus the
// derivative multiplier.  Shared by the uniform-grid kernels (ww_spectral.cu)
// and the mesh / general-tableau kernels of time segments (ww_segments.cu).
#pragma once

#include "ww_df.cuh"
#include "ww_internal.cuh"

namespace ww {

namespace {

constexpr int FFT_THREADS = 256;

__device__ __forceinline__ double2 times_ik(double2 z, int k) {   // (ik) z
    return make_double2(-(double)k * z.y, (double)k * z.x);
}

// Arithmetic of the in-shared-memory transforms.  ArF64: IEEE double (the
// WW_FP64 form).  ArDF: double-float (ww_df.cuh) for the WW_MIXED form, where
// the FP64 pipe is the bottleneck; inputs, outputs and all pointwise algebra
// stay FP64 in both.
struct ArF64 {
    using C = double2;
    using R = double;   // real values of the pointwise algebra
    using T = double;   // entries of the per-slot / per-point tables
    static __device__ __forceinline__ C mk(double re, double im) { return make_double2(re, im); }
    static __device__ __forceinline__ double2 get(C z) { return z; }
    static __device__ __forceinline__ void fft(C *s, int N, int logN, const void *tw, bool inv) {
        block_fft(s, N, logN, static_cast<const double2 *>(tw), inv);
    }
    // points of shared memory one transform needs
    static __host__ __device__ __forceinline__ int cap(int N) { return N; }
    // the twiddle table the transforms read, staged into shared memory: the
    // half table exp(-2 pi i m / N), m < N/2, as it is
    static __host__ __device__ __forceinline__ int table_entries(int N, int) { return N >> 1; }
    static __device__ __forceinline__ void stage(const void *tw, C *dst, int N, int) {
        const C *src = static_cast<const C *>(tw);
        for (int j = threadIdx.x; j < (N >> 1); j += blockDim.x) dst[j] = src[j];
    }
    static __device__ __forceinline__ C scalef(C z, float f) { return cscale(z, (double)f); }
    static __device__ __forceinline__ C ikscale(C z, int k, float p2) { return cscale(times_ik(z, k), (double)p2); }
    static __device__ __forceinline__ C add(C a, C b) { return cadd(a, b); }
    static __device__ __forceinline__ C zero() { return make_double2(0.0, 0.0); }
    // tables and real arithmetic
    static __device__ __forceinline__ R tab(const void *t, int j) { return static_cast<const T *>(t)[j]; }
    static __device__ __forceinline__ C scale_tab(C z, const void *t, int j) { return cscale(z, tab(t, j)); }
    static __device__ __forceinline__ C re_only_tab(C z, const void *t, int j) { return make_double2(z.x * tab(t, j), 0.0); }
    static __device__ __forceinline__ R from(double x) { return x; }
    static __device__ __forceinline__ R rmul(R a, R b) { return a * b; }
    static __device__ __forceinline__ R radd(R a, R b) { return a + b; }
    static __device__ __forceinline__ R rsub(R a, R b) { return a - b; }
    static __device__ __forceinline__ R rneg(R a) { return -a; }
    static __device__ __forceinline__ C mkr(R re, R im) { return make_double2(re, im); }
    static __device__ __forceinline__ R re(C z) { return z.x; }
    static __device__ __forceinline__ R im(C z) { return z.y; }
    static __device__ __forceinline__ C addr(C z, R a, R b) { return make_double2(z.x + a, z.y + b); }
};

struct ArDF {
    using C = dfl::cdf;
    using R = dfl::df;
    using T = float2;   // double-float table entry (hi, lo)
    static __device__ __forceinline__ C mk(double re, double im) { return dfl::from_d2(make_double2(re, im)); }
    static __device__ __forceinline__ double2 get(C z) { return dfl::to_d2(z); }
    static __device__ __forceinline__ void fft(C *s, int N, int logN, const void *tw, bool inv) {
        if (N >= 16 && N <= dfl::FFT_STOCKHAM_MAXN)
            dfl::block_fft_stockham(s, N, logN, static_cast<const dfl::cdf *>(tw), inv);
        else
            dfl::block_fft(s, N, logN, static_cast<const dfl::cdf *>(tw), inv);
    }
    // points of shared memory one transform needs (the Stockham passes pad)
    static __host__ __device__ __forceinline__ int cap(int N) {
        return (N >= 16 && N <= dfl::FFT_STOCKHAM_MAXN) ? N + N / 8 : N;
    }
    // the twiddles the transforms read, staged into shared memory: the
    // Stockham passes' per-pass tables (conflict-free reads), else the half
    // table exp(-2 pi i m / N), m < N/2, as it is
    static __host__ __device__ __forceinline__ int table_entries(int N, int logN) {
        return (N >= 16 && N <= dfl::FFT_STOCKHAM_MAXN) ? dfl::stockham_table_size(logN) : (N >> 1);
    }
    static __device__ __forceinline__ void stage(const void *tw, C *dst, int N, int logN) {
        const C *src = static_cast<const C *>(tw);
        if (N >= 16 && N <= dfl::FFT_STOCKHAM_MAXN)
            dfl::build_stockham_twiddles(src, dst, N, logN);
        else
            for (int j = threadIdx.x; j < (N >> 1); j += blockDim.x) dst[j] = src[j];
    }
    static __device__ __forceinline__ C scalef(C z, float f) { return dfl::cscalef(z, f); }
    static __device__ __forceinline__ C ikscale(C z, int k, float p2) { return dfl::cscalef(dfl::times_ik(z, k), p2); }
    static __device__ __forceinline__ C add(C a, C b) { return dfl::cadd(a, b); }
    static __device__ __forceinline__ C zero() { return C{0.f, 0.f, 0.f, 0.f}; }
    static __device__ __forceinline__ R tab(const void *t, int j) {
        const float2 v = static_cast<const T *>(t)[j];
        return R{v.x, v.y};
    }
    static __device__ __forceinline__ C scale_tab(C z, const void *t, int j) { return dfl::cscale(z, tab(t, j)); }
    static __device__ __forceinline__ C re_only_tab(C z, const void *t, int j) {
        return dfl::make(dfl::mul(dfl::re(z), tab(t, j)), dfl::df{0.f, 0.f});
    }
    static __device__ __forceinline__ R from(double x) { return dfl::from_double(x); }
    static __device__ __forceinline__ R rmul(R a, R b) { return dfl::mul(a, b); }
    static __device__ __forceinline__ R radd(R a, R b) { return dfl::add(a, b); }
    static __device__ __forceinline__ R rsub(R a, R b) { return dfl::sub(a, b); }
    static __device__ __forceinline__ R rneg(R a) { return R{-a.hi, -a.lo}; }
    static __device__ __forceinline__ C mkr(R re, R im) { return dfl::make(re, im); }
    static __device__ __forceinline__ R re(C z) { return dfl::re(z); }
    static __device__ __forceinline__ R im(C z) { return dfl::im(z); }
    static __device__ __forceinline__ C addr(C z, R a, R b) { return dfl::make(dfl::add(dfl::re(z), a), dfl::add(dfl::im(z), b)); }
};

// The transforms' twiddles (built from the global half table tw, the same
// element type as the transform's data) staged into shared memory at dst,
// right after the kernel's work arrays: the passes then read them at
// shared-memory latency instead of through L1.  The caller synchronises
// before the first transform; the returned pointer replaces tw in every
// transform of the kernel.
template <class AR>
__device__ __forceinline__ const void *stage_twiddles(const void *tw, typename AR::C *dst, int N, int logN) {
    AR::stage(tw, dst, N, logN);
    return dst;
}

// bytes of shared memory of a kernel with `arrays` transform buffers and the staged twiddles
template <class AR>
__host__ __forceinline__ size_t fft_smem_bytes(int N, int arrays) {
    int logN = 0;
    while ((1 << logN) < N) ++logN;
    return sizeof(typename AR::C) * ((size_t)arrays * AR::cap(N) + (size_t)AR::table_entries(N, logN));
}

// s <- s * (ik) / N (Nyquist zero)
template <class AR>
__device__ __forceinline__ void mul_deriv(typename AR::C *s, int N) {
    const float invN = 1.0f / (float)N;   // exact: N is a power of two
    for (int j = threadIdx.x; j < N; j += blockDim.x)
        s[j] = (j == (N >> 1)) ? AR::zero() : AR::ikscale(s[j], wavenum(j, N), invN);
}

}  // namespace

}  // namespace ww
