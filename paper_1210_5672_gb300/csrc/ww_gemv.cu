// ww_gemv.cu -- products of an m x k column-major matrix with a narrow block
// of n <= 8 columns: the base-state DtN of every RK stage (one column: the
// solve mu = A^{-1} phi and G gamma, Sec. 2.2 Eq. G) and narrow dtn_apply
// calls.  One column cannot feed a tensor-core tile, so these run on the CUDA
// cores and are bound by streaming the matrix (FP32 X: 16 MB, FP64 A or G:
// 32 MB at N = 2048) or, in FP64, by the FP64 pipe (m k FMAs per column).
//
// Layout of the work.  A CTA owns 64 rows and a 1/KS slice of k; its 8 warps
// split that slice again, each lane holding two adjacent rows (one 8- or
// 16-byte vector load per column of A, a warp reads 64 contiguous rows), with
// eight column loads in flight per lane, and the CTA's slice of B converted
// once into shared memory.  The KS CTAs of a row tile form a
// thread-block cluster: each sums its warps in shared memory, then CTA r adds
// the KS partials of its share of the rows through distributed shared memory,
// in rank order.  Every sum is taken in a fixed order, so results do not
// depend on scheduling, and no workspace or atomics are needed.
#include <cooperative_groups.h>

#include "ww_internal.cuh"

namespace cg = cooperative_groups;

namespace ww {

namespace {

constexpr int NR_ROWS = 64, NR_WARPS = 8, NR_MAXN = 8, NR_MAXKS = 8;

template <typename TA>
struct Vec2;
template <>
struct Vec2<float> {
    using T = float2;
};
template <>
struct Vec2<double> {
    using T = double2;
};

// MODE 0: C = alpha S + beta C (beta == 0: C = alpha S);  MODE 1: C = Psi - S.
// S = A B with products and per-lane sums in TA (FP32 for the FP32 inverse,
// FP64 otherwise); warp, CTA and cluster partials are added in FP64.  NB >= n
// is the compile-time column count (1, 2, 4 or 8): the loops over the columns
// are unrolled to NB, so no predicated-off FMA of an absent column is issued
// (on GB300 the FP64 pipe retires 2 lanes per clock per SM).  The CTA's slice
// of B is converted to TA once and held in shared memory.
template <typename TA, bool VEC, int MODE, int NB>
__global__ void __launch_bounds__(NR_WARPS * 32) k_gemv_nr(int m, int n, int k, double alpha,
                                                           const TA *__restrict__ A, int lda,
                                                           const double *__restrict__ B, int ldb, double beta,
                                                           double *C, int ldc, const double *__restrict__ Psi,
                                                           int ldp, const int *skip) {
    if (skip && *skip) return;   // the same flag for every CTA of the cluster: all leave together
    __shared__ double part[NR_WARPS][NB][NR_ROWS];
    __shared__ double cta[NB][NR_ROWS];
    extern __shared__ __align__(16) unsigned char bsh_raw[];
    TA *bsh = reinterpret_cast<TA *>(bsh_raw);   // [NB][kcl]
    cg::cluster_group cluster = cg::this_cluster();
    const int KS = gridDim.y, rank = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = blockIdx.x * NR_ROWS;
    // rows of this lane: (row0 + 2 lane, +1) with vector loads, else (row0 + lane, + 32)
    const int ra = VEC ? row0 + 2 * lane : row0 + lane;
    const int rb = VEC ? ra + 1 : ra + 32;
    const bool oka = ra < m, okb = rb < m;
    // k slice of this CTA, then of this warp
    const int kc = (k + KS - 1) / KS, kb0 = rank * kc, ke0 = min(k, kb0 + kc);
    const int kcl = max(0, ke0 - kb0);
    for (int t = threadIdx.x; t < NB * kcl; t += blockDim.x) {
        const int j = t / kcl, kk = t - j * kcl;
        bsh[t] = j < n ? (TA)B[(size_t)j * ldb + kb0 + kk] : (TA)0;
    }
    __syncthreads();
    const int wc = (kcl + NR_WARPS - 1) / NR_WARPS;
    const int kb = kb0 + warp * wc, ke = min(ke0, kb + wc);
    TA acc0[NB], acc1[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) acc0[j] = acc1[j] = (TA)0;
    int kk = kb;
    for (; kk + 8 <= ke; kk += 8) {
        TA a0[8], a1[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const TA *col = A + (size_t)(kk + u) * lda;
            if (VEC) {
                typename Vec2<TA>::T v;
                if (oka) {
                    v = *reinterpret_cast<const typename Vec2<TA>::T *>(col + ra);
                } else {
                    v.x = v.y = (TA)0;
                }
                a0[u] = v.x;
                a1[u] = v.y;
            } else {
                a0[u] = oka ? col[ra] : (TA)0;
                a1[u] = okb ? col[rb] : (TA)0;
            }
        }
        const TA *bk = bsh + (kk - kb0);
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                const TA b = bk[j * kcl + u];
                acc0[j] = fma(a0[u], b, acc0[j]);
                acc1[j] = fma(a1[u], b, acc1[j]);
            }
    }
    for (; kk < ke; ++kk) {
        const TA *col = A + (size_t)kk * lda;
        const TA x0 = oka ? col[ra] : (TA)0, x1 = okb ? col[rb] : (TA)0;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const TA b = bsh[j * kcl + (kk - kb0)];
            acc0[j] = fma(x0, b, acc0[j]);
            acc1[j] = fma(x1, b, acc1[j]);
        }
    }
    const int la = VEC ? 2 * lane : lane, lb = VEC ? la + 1 : la + 32;   // local rows
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        part[warp][j][la] = (double)acc0[j];
        part[warp][j][lb] = (double)acc1[j];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n * NR_ROWS; t += blockDim.x) {
        const int j = t / NR_ROWS, r = t % NR_ROWS;
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NR_WARPS; ++w) s += part[w][j][r];
        cta[j][r] = s;
    }
    cluster.sync();   // every CTA's partial is complete and visible to the cluster
    // CTA `rank` finishes rows [rank * 64 / KS, (rank + 1) * 64 / KS) of the tile
    const int r0 = rank * NR_ROWS / KS, r1 = (rank + 1) * NR_ROWS / KS;
    for (int t = threadIdx.x; t < n * (r1 - r0); t += blockDim.x) {
        const int j = t / (r1 - r0), r = r0 + t % (r1 - r0);
        const int gr = row0 + r;
        double s = 0.0;
        for (int q = 0; q < KS; ++q) s += cluster.map_shared_rank(&cta[0][0], q)[j * NR_ROWS + r];
        if (gr < m) {
            double *p = C + (size_t)j * ldc + gr;
            if (MODE == 1)
                *p = Psi[(size_t)j * ldp + gr] - s;
            else
                *p = (beta == 0.0) ? alpha * s : fma(alpha, s, beta * *p);
        }
    }
    cluster.sync();   // no CTA leaves while another still reads its shared memory
}

template <typename TA, bool VEC, int MODE, int NB>
int launch_nr(cudaStream_t s, int m, int n, int k, double alpha, const TA *A, int lda, const double *B, int ldb,
              double beta, double *C, int ldc, const double *Psi, int ldp, const int *skip) {
    // split k over up to 8 CTAs, at least 128 columns each
    int ks = k / 128;
    ks = ks < 1 ? 1 : (ks > NR_MAXKS ? NR_MAXKS : ks);
    const int kcl = (k + ks - 1) / ks;
    const size_t dyn = sizeof(TA) * (size_t)NB * (size_t)(kcl > 0 ? kcl : 1);
    auto kern = k_gemv_nr<TA, VEC, MODE, NB>;
    WW_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((m + NR_ROWS - 1) / NR_ROWS), (unsigned)ks, 1);
    cfg.blockDim = dim3(NR_WARPS * 32, 1, 1);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = (unsigned)ks;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    WW_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, Psi, ldp, skip));
    return WW_OK;
}

template <typename TA, bool VEC, int MODE>
int launch_nb(cudaStream_t s, int m, int n, int k, double alpha, const TA *A, int lda, const double *B, int ldb,
              double beta, double *C, int ldc, const double *Psi, int ldp, const int *skip) {
    if (n == 1) return launch_nr<TA, VEC, MODE, 1>(s, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, Psi, ldp, skip);
    if (n == 2) return launch_nr<TA, VEC, MODE, 2>(s, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, Psi, ldp, skip);
    if (n <= 4) return launch_nr<TA, VEC, MODE, 4>(s, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, Psi, ldp, skip);
    return launch_nr<TA, VEC, MODE, 8>(s, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, Psi, ldp, skip);
}

template <typename TA, int MODE>
int dispatch_nr(cudaStream_t s, int m, int n, int k, double alpha, const TA *A, int lda, const double *B, int ldb,
                double beta, double *C, int ldc, const double *Psi, int ldp, const int *skip) {
    if (m <= 0 || n <= 0) return WW_OK;
    if (n > NR_MAXN) return fail(WW_ERR_ARG, "gemv_narrow: at most 8 columns");
    // two-row vector loads need an aligned base, an even leading dimension and an even m
    const bool vec = (reinterpret_cast<uintptr_t>(A) % (2 * sizeof(TA)) == 0) && (lda % 2 == 0) && (m % 2 == 0);
    if (vec) return launch_nb<TA, true, MODE>(s, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, Psi, ldp, skip);
    return launch_nb<TA, false, MODE>(s, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, Psi, ldp, skip);
}

}  // namespace

int gemv_narrow(cudaStream_t s, int m, int n, int k, double alpha, const double *A, int lda, const double *B, int ldb,
                double beta, double *C, int ldc, const int *skip) {
    return dispatch_nr<double, 0>(s, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, nullptr, 0, skip);
}

int gemv_narrow_f32(cudaStream_t s, int m, int n, int k, const float *A, int lda, const double *B, int ldb,
                    double beta, double *C, int ldc, const int *skip) {
    return dispatch_nr<float, 0>(s, m, n, k, 1.0, A, lda, B, ldb, beta, C, ldc, nullptr, 0, skip);
}

int resid_narrow(cudaStream_t s, int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                 const double *Psi, int ldp, double *R, int ldr, const int *skip) {
    return dispatch_nr<double, 1>(s, m, n, k, 1.0, A, lda, B, ldb, 0.0, R, ldr, Psi, ldp, skip);
}

}  // namespace ww
