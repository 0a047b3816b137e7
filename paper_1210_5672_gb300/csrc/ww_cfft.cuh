// ww_cfft.cuh -- FP64 FFT of one length-N vector split over a thread-block
// cluster of CS = 8 CTAs, for transforms on the critical path of an RK stage
// that act on one column (one CTA would be bound by a single SM's FP64 pipe,
// 2 lanes per clock).
//
// Four-step factorisation N = CS x L, with n = r + CS n2 and k = k2 + L k1:
//   forward:  CTA r transforms its decimated samples x[r + CS n2] (length L),
//             multiplies by W_N^{r k2}; then CTA r takes the CS-point DFT over
//             the cluster ranks for its share of k2 (read through distributed
//             shared memory) and holds X[k2 + L k1], k1 = 0..CS-1;
//   inverse:  the same steps in reverse order, back to x[r + CS n2].
// Point-wise work acts on the decimated samples (physical space) or on the
// spectral slots a CTA holds (slot_of).  Unscaled inverse, as in block_fft.
// Everything here has internal linkage: each kernel file gets its own copy.
#pragma once

#include <cooperative_groups.h>

#include "ww_internal.cuh"

namespace cg = cooperative_groups;

namespace ww {

namespace {

constexpr int CB_CS = 8;

constexpr int CB_THREADS = 256;

// W_N^m, 0 <= m < N, from the half table tw[k] = exp(-2 pi i k/N), k < N/2
__device__ __forceinline__ double2 wn(const double2 *__restrict__ tw, int m, int N, bool inv) {
    double2 w = m < (N >> 1) ? __ldg(&tw[m]) : make_double2(-__ldg(&tw[m - (N >> 1)]).x, -__ldg(&tw[m - (N >> 1)]).y);
    if (inv) w.y = -w.y;
    return w;
}

// in-place radix-2 FFT of length L = N / CS in shared memory (twiddles
// W_L^j = W_N^{CS j}), whole block; callers synchronise before, it ends with a barrier
__device__ void local_fft(double2 *s, int L, int logL, const double2 *__restrict__ tw, int N, int CS, bool inv) {
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const int j = (int)(__brev((unsigned)i) >> (32 - logL));
        if (i < j) {
            const double2 t = s[i];
            s[i] = s[j];
            s[j] = t;
        }
    }
    __syncthreads();
    for (int lh = 0; lh < logL; ++lh) {
        const int half = 1 << lh;
        const int tstride = (L >> (lh + 1)) * CS;   // W_{2 half}^k = W_N^{k N / (2 half)}
        for (int b = threadIdx.x; b < (L >> 1); b += blockDim.x) {
            const int k = b & (half - 1);
            const int i0 = ((b >> lh) << (lh + 1)) + k, i1 = i0 + half;
            const double2 w = wn(tw, k * tstride, N, inv);
            const double2 v = cmul(s[i1], w), u = s[i0];
            s[i0] = cadd(u, v);
            s[i1] = csub(u, v);
        }
        __syncthreads();
    }
}

// 8-point DFT in registers (natural order in and out): two 4-point DFTs of the
// even and odd samples and the W_8 combination, all twiddles constants.
template <bool INV>
__device__ __forceinline__ double2 mul_mi(double2 z) {   // (-i) z forward, (+i) z inverse
    return INV ? make_double2(-z.y, z.x) : make_double2(z.y, -z.x);
}
template <bool INV>
__device__ __forceinline__ double2 mul_w8(double2 z) {   // z W_8 (forward (1 - i)/sqrt2, inverse its conjugate)
    const double c = 0.70710678118654752440084436210484903928;
    return INV ? make_double2((z.x - z.y) * c, (z.x + z.y) * c) : make_double2((z.x + z.y) * c, (z.y - z.x) * c);
}
template <bool INV>
__device__ __forceinline__ void dft4(double2 &x0, double2 &x1, double2 &x2, double2 &x3) {
    const double2 t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), t3 = mul_mi<INV>(csub(x1, x3));
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = cadd(t1, t3);
    x3 = csub(t1, t3);
}
template <bool INV>
__device__ __forceinline__ void dft8(double2 (&v)[8]) {
    double2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    o1 = mul_w8<INV>(o1);
    o2 = mul_mi<INV>(o2);
    o3 = mul_mi<INV>(mul_w8<INV>(o3));   // W8^3 = W8 W8^2
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

// Cluster FFT.  xs: L decimated samples of this CTA (n2 = 0..L-1);
// spec: this CTA's spectral slots [k1][k2l], k = (rank P + k2l) + L k1,
// P = L / CS; zs: exchange buffer of L points.
template <int CS>
__device__ void cfft_forward(cg::cluster_group &cl, double2 *xs, double2 *spec, int N, int logN,
                             const double2 *__restrict__ tw) {
    static_assert(CS == 8, "the cluster-rank DFT is the 8-point one");
    const int L = N / CS, logL = logN - (CS == 8 ? 3 : 2), P = L / CS, r = (int)cl.block_rank();
    __syncthreads();
    local_fft(xs, L, logL, tw, N, CS, false);
    for (int k2 = threadIdx.x; k2 < L; k2 += blockDim.x) xs[k2] = cmul(xs[k2], wn(tw, r * k2, N, false));
    cl.sync();
    for (int k2l = threadIdx.x; k2l < P; k2l += blockDim.x) {
        const int k2 = r * P + k2l;
        double2 v[CS];
#pragma unroll
        for (int q = 0; q < CS; ++q) v[q] = cl.map_shared_rank(xs, q)[k2];
        dft8<false>(v);
#pragma unroll
        for (int k1 = 0; k1 < CS; ++k1) spec[k1 * P + k2l] = v[k1];
    }
    cl.sync();   // every CTA read the others' xs
}

template <int CS>
__device__ void cfft_inverse(cg::cluster_group &cl, const double2 *spec, double2 *zs, double2 *xs, int N, int logN,
                             const double2 *__restrict__ tw) {
    static_assert(CS == 8, "the cluster-rank DFT is the 8-point one");
    const int L = N / CS, logL = logN - (CS == 8 ? 3 : 2), P = L / CS, r = (int)cl.block_rank();
    __syncthreads();
    for (int k2l = threadIdx.x; k2l < P; k2l += blockDim.x) {
        const int k2 = r * P + k2l;
        double2 v[CS];
#pragma unroll
        for (int k1 = 0; k1 < CS; ++k1) v[k1] = spec[k1 * P + k2l];
        dft8<true>(v);
#pragma unroll
        for (int q = 0; q < CS; ++q) zs[q * P + k2l] = cmul(v[q], wn(tw, q * k2, N, true));
    }
    cl.sync();
    for (int k2 = threadIdx.x; k2 < L; k2 += blockDim.x) {
        const int q = k2 / P;
        xs[k2] = cl.map_shared_rank(zs, q)[r * P + (k2 - q * P)];
    }
    cl.sync();   // every CTA read the others' zs
    local_fft(xs, L, logL, tw, N, CS, true);
}

// spectral slot of this CTA: t in [0, L) -> (k1, k2l) -> FFT slot k
__device__ __forceinline__ int slot_of(int t, int N, int CS, int r) {
    const int L = N / CS, P = L / CS;
    const int k1 = t / P, k2l = t - k1 * P;
    return (r * P + k2l) + L * k1;
}


template <typename K, typename... Args>
int launch_cluster(K kernel, int CS, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)CS, 1, 1);
    cfg.blockDim = dim3(CB_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    WW_CUDA_TRY(cudaLaunchKernelEx(&cfg, kernel, args...));
    return WW_OK;
}


}  // namespace

}  // namespace ww
