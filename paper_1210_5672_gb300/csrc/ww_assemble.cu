// ww_assemble.cu -- boundary-integral kernel matrices of Sec. 2.2, Eq. (K1K2),
// trapezoid collocation K_ij = K(alpha_i, alpha_j)/N, G_ij = G(alpha_i, alpha_j)/N,
// A = 1/2 I + K.  Image kernels K2, G2 (finite depth) enter with a minus sign:
// App. A, Eqs. (Phi), (plemelj:1), (plemelj:2) subtract the mirror-image layer,
// which gives the flat-surface symbol k tanh(kh).
//
// Uniform grid: x = alpha_i - alpha_j = 2 pi (i - j)/N, so cos x, sin x and
// cot(x/2) come from length-N tables.  exp(+-(eta_i -+ eta_j)) are products of
// E = exp(eta) and 1/E, so no entry evaluates a transcendental function.  The
// complex cotangent uses the branch-stable quotient of Sec. 2.2,
//   cot((x+iy)/2) = (cos x + cosh y)/(sin x + i sinh y),   cos x >= 0,
//                 = (sin x - i sinh y)/(cosh y - cos x),   cos x <  0,
// neither of which cancels.  sinh of the small differences eta_i - eta_j is
// taken from its Taylor series so that it keeps full relative accuracy.
#include "ww_internal.cuh"

namespace ww {

namespace {

constexpr int ASM_TI = 128;   // rows (i) per block, one per thread
constexpr int ASM_TJ = 16;    // columns (j) per block, looped by each thread

// sinh(y) for a difference y = eta_i - eta_j: series when small (no cancellation)
__device__ __forceinline__ double sinh_diff(double y, double ey, double eyi) {
    if (fabs(y) < 0.25) {
        double y2 = y * y;
        // y (1 + y^2/3! + y^4/5! + ... + y^12/13!), truncation < 1e-17 relative for |y| < 1/4
        double p = 1.0 / 6227020800.0;
        p = fma(p, y2, 1.0 / 39916800.0);
        p = fma(p, y2, 1.0 / 362880.0);
        p = fma(p, y2, 1.0 / 5040.0);
        p = fma(p, y2, 1.0 / 120.0);
        p = fma(p, y2, 1.0 / 6.0);
        p = fma(p, y2, 1.0);
        return y * p;
    }
    return 0.5 * (ey - eyi);
}

// 1/d for a positive normal d: Newton-Raphson, x <- x + x (1 - d x) (each step
// squares the relative error; the residual 1 - d x is formed with one FMA),
// started from the FP32 hardware reciprocal of d rounded to FP32 (relative
// error ~2^-23): two steps reach the FP64 rounding level (within 1 ulp of the
// division, tested against it by ww_selftest_recip).  Four FP64 operations
// instead of a full FP64 division.
__device__ __forceinline__ double recip_nr(double d) {
    double x = (double)__frcp_rn((float)d);
    x = fma(x, fma(-d, x, 1.0), x);
    return fma(x, fma(-d, x, 1.0), x);
}

// biased exponent field of x (0 for zero), the scale the digit splits take per row
__device__ __forceinline__ int bexp_of(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// cot((x + i y)/2) with cx = cos x, sx = sin x, ch = cosh y, sh = sinh y
__device__ __forceinline__ double2 cot_half(double cx, double sx, double ch, double sh) {
    if (cx >= 0.0) {
        double num = cx + ch;
        double inv = num / fma(sx, sx, sh * sh);
        return make_double2(sx * inv, -sh * inv);
    } else {
        double inv = 1.0 / (ch - cx);
        return make_double2(sx * inv, -sh * inv);
    }
}

__global__ void __launch_bounds__(ASM_TI) k_assemble(const double *__restrict__ eta, const double *__restrict__ eta_x,
                                                     const double *__restrict__ eta_xx, const double *__restrict__ E,
                                                     const double *__restrict__ Einv, const double *__restrict__ cs,
                                                     const double *__restrict__ cot0, int N, int deep, int trans,
                                                     double *A, double *G) {
    const int i = blockIdx.x * ASM_TI + threadIdx.x;
    const int j0 = blockIdx.y * ASM_TJ;
    if (i >= N) return;
    const double invN = 1.0 / N;
    const double ei = eta[i], exi = eta_x[i], Ei = E[i], Eii = Einv[i];
    for (int jj = 0; jj < ASM_TJ; ++jj) {
        const int j = j0 + jj;
        if (j >= N) break;
        const double ej = eta[j], exj = eta_x[j], Ej = E[j], Eij = Einv[j];
        double k1, g1;
        if (i == j) {
            // diagonal limits: zeta''/(2 zeta') = (eta' eta'' + i eta'') / (2 (1 + eta'^2))
            double d = 0.5 / fma(exi, exi, 1.0);
            k1 = -eta_xx[i] * d;
            g1 = exi * eta_xx[i] * d;
        } else {
            int m = i - j;
            if (m < 0) m += N;
            const double cx = cs[m], sx = cs[N + m];
            // y = eta_i - eta_j: e^y = E_i / E_j
            const double y = ei - ej;
            const double ey = Ei * Eij, eyi = Eii * Ej;
            const double ch = 0.5 * (ey + eyi);
            const double sh = sinh_diff(y, ey, eyi);
            double2 ct = cot_half(cx, sx, ch, sh);
            // K1 = Im{ zeta'(beta)/2 cot }, zeta'(beta) = 1 + i eta'_j
            k1 = 0.5 * fma(exj, ct.x, ct.y);
            // G1 = Re{ zeta'(alpha)/2 cot - 1/2 cot((alpha - beta)/2) }, zeta'(alpha) = 1 + i eta'_i
            g1 = 0.5 * (fma(-exi, ct.y, ct.x) - cot0[m]);
        }
        double k2 = 0.0, g2 = 0.0;
        if (!deep) {
            int m = i - j;
            if (m < 0) m += N;
            const double cx = cs[m], sx = cs[N + m];
            // image: zeta(alpha) - conj(zeta(beta)) = x + i (eta_i + eta_j)
            const double ep = Ei * Ej, epi = Eii * Eij;
            const double ch = 0.5 * (ep + epi), sh = 0.5 * (ep - epi);
            double2 ct = cot_half(cx, sx, ch, sh);
            // K2 = -Im{ conj(zeta'(beta))/2 cot },  conj(zeta'(beta)) = 1 - i eta'_j
            k2 = -0.5 * fma(-exj, ct.x, ct.y);
            // G2 = -Re{ zeta'(alpha)/2 cot }
            g2 = -0.5 * fma(-exi, ct.y, ct.x);
        }
        const size_t idx = trans ? (size_t)i * N + j : (size_t)j * N + i;
        A[idx] = (k1 + k2) * invN + (i == j ? 0.5 : 0.0);
        G[idx] = (g1 + g2) * invN;
    }
}

// trans != 0 writes A^T and G^T instead (the operands of the transposed DtN
// of the adjoint sweep).
//
// Symmetric form: cot is odd, so the (j, i) entry follows from the (i, j) one:
//   cot((-x - iy)/2) = -cot((x + iy)/2),  cot((-x + iy')/2) = -conj(cot((x + iy')/2)),
// and cot((alpha_j - alpha_i)/2) = -cot((alpha_i - alpha_j)/2).  Each block
// takes a pair of 32 x 32 tiles (I, J), I < J, evaluates the two cotangents
// of every unordered pair once and writes both tiles (the transposed one
// through shared memory, so both stores are coalesced); diagonal tiles are
// evaluated entry by entry.
constexpr int ST = 32;

// Off-diagonal pair (i, j): the direct cotangent ct1 = cot((x + i y)/2),
// y = eta_i - eta_j, and (finite depth) the image one ct2 = cot((x + i y')/2),
// y' = eta_i + eta_j, share one reciprocal of the product of their denominators;
// the 1/2 of the kernels and the 1/N of the rule are applied once at the end:
//   K_ij ~ exj (ct1 + ct2).x + (ct1 - ct2).y,    G_ij ~ (ct1 - ct2).x - exi (ct1 - ct2).y - cot0
//   K_ji ~ -[exi (ct1 + ct2).x + (ct1 + ct2).y], G_ji ~ (ct2 - ct1).x + exj (ct1 + ct2).y + cot0
// (cot is odd: the (j, i) pair reuses both cotangents, see below).
template <bool DEEP>
__device__ __forceinline__ void pair_entries(double cx, double sx, double c0, double ei, double exi, double Ei,
                                             double Eii, double ej, double exj, double Ej, double Eij, double &kij,
                                             double &gij, double &kji, double &gji) {
    const double y = ei - ej;
    const double ey = Ei * Eij, eyi = Eii * Ej;
    const double ch1 = 0.5 * (ey + eyi), sh1 = sinh_diff(y, ey, eyi);
    double n1, d1, n2 = 0.0, d2 = 1.0, sh2 = 0.0;
    if (cx >= 0.0) {
        n1 = cx + ch1;
        d1 = fma(sx, sx, sh1 * sh1);
    } else {
        n1 = 1.0;
        d1 = ch1 - cx;
    }
    if (!DEEP) {
        const double ep = Ei * Ej, epi = Eii * Eij;
        const double ch2 = 0.5 * (ep + epi);
        sh2 = 0.5 * (ep - epi);
        if (cx >= 0.0) {
            n2 = cx + ch2;
            d2 = fma(sx, sx, sh2 * sh2);
        } else {
            n2 = 1.0;
            d2 = ch2 - cx;
        }
    }
    const double r = recip_nr(d1 * d2);
    const double inv1 = n1 * d2 * r;
    const double c1x = sx * inv1, c1y = -sh1 * inv1;
    double c2x = 0.0, c2y = 0.0;
    if (!DEEP) {
        const double inv2 = n2 * d1 * r;
        c2x = sx * inv2;
        c2y = -sh2 * inv2;
    }
    const double a = c1x + c2x, b = c1y - c2y, c = c1x - c2x, d = c1y + c2y;
    kij = fma(exj, a, b);
    gij = fma(-exi, b, c) - c0;
    kji = -fma(exi, a, d);
    gji = fma(exj, d, -c) + c0;
}

template <bool DEEP>
__global__ void __launch_bounds__(256) k_assemble_sym(const double *__restrict__ eta, const double *__restrict__ eta_x,
                                                      const double *__restrict__ eta_xx, const double *__restrict__ E,
                                                      const double *__restrict__ Einv,
                                                      const double *__restrict__ cs, const double *__restrict__ cot0,
                                                      int N, int trans, double *A, double *G, int *emaxK,
                                                      int *emaxG) {
    __shared__ double tA[ST][ST + 1], tG[ST][ST + 1];
    __shared__ int redK[8][ST], redG[8][ST];   // row exponent maxima per warp (emaxK != NULL)
    // triangular tile index -> (I, J), I <= J
    const int T = N / ST;
    int b = blockIdx.x, I = 0;
    while (b >= T - I) {
        b -= T - I;
        ++I;
    }
    const int J = I + b;
    const double h = 0.5 / N;   // the kernels' 1/2 and the rule's 1/N
    const int il = threadIdx.x & 31;
    const int i = I * ST + il;
    const double ei = eta[i], exi = eta_x[i], Ei = E[i], Eii = Einv[i];
    int mK = 0, mG = 0;   // this thread's row exponent maxima
    for (int jl = threadIdx.x >> 5; jl < ST; jl += 8) {
        const int j = J * ST + jl;
        const double ej = eta[j], exj = eta_x[j], Ej = E[j], Eij = Einv[j];
        double kij, gij, kji, gji;
        int m = i - j;
        if (m < 0) m += N;
        const double cx = cs[m], sx = cs[N + m];
        if (i == j) {
            // diagonal limits of the direct kernels, zeta''/(2 zeta') (doubled: h carries 1/2)
            const double dd = 1.0 / fma(exi, exi, 1.0);
            kij = -eta_xx[i] * dd;
            gij = exi * eta_xx[i] * dd;
            if (!DEEP) {
                const double ep = Ei * Ej, epi = Eii * Eij;
                const double2 ct = cot_half(cx, sx, 0.5 * (ep + epi), 0.5 * (ep - epi));
                kij -= fma(-exj, ct.x, ct.y);
                gij -= fma(-exi, ct.y, ct.x);
            }
            kji = kij;
            gji = gij;
        } else {
            pair_entries<DEEP>(cx, sx, cot0[m], ei, exi, Ei, Eii, ej, exj, Ej, Eij, kij, gij, kji, gji);
        }
        if (trans) {   // entry (i, j) of A^T is entry (j, i) of A
            const double tk = kij, tg = gij;
            kij = kji;
            gij = gji;
            kji = tk;
            gji = tg;
        }
        const size_t idx = (size_t)j * N + i;
        const double aij = fma(h, kij, i == j ? 0.5 : 0.0), gv = h * gij;
        A[idx] = aij;
        G[idx] = gv;
        tA[jl][il] = fma(h, kji, i == j ? 0.5 : 0.0);
        tG[jl][il] = h * gji;
        if (emaxK) {
            mK = max(mK, bexp_of(i == j ? aij - 0.5 : aij));   // K = A - I/2, as the digit split shifts it
            mG = max(mG, bexp_of(gv));
        }
    }
    const int warp = threadIdx.x >> 5;
    if (emaxK) {   // rows I*ST + il: this tile's columns
        redK[warp][il] = mK;
        redG[warp][il] = mG;
        __syncthreads();
        if (threadIdx.x < ST) {
            int k = redK[0][threadIdx.x], g = redG[0][threadIdx.x];
            for (int w = 1; w < 8; ++w) {
                k = max(k, redK[w][threadIdx.x]);
                g = max(g, redG[w][threadIdx.x]);
            }
            atomicMax(&emaxK[I * ST + threadIdx.x], k);
            atomicMax(&emaxG[I * ST + threadIdx.x], g);
        }
    }
    if (I == J) return;   // the diagonal tile is complete (uniform branch: no barrier skipped unevenly)
    __syncthreads();
    // transposed tile: entry (j, i) at A[i * N + j]; consecutive threads walk j
    const int jl2 = threadIdx.x & 31;
    mK = 0;
    mG = 0;
    for (int il2 = threadIdx.x >> 5; il2 < ST; il2 += 8) {
        const size_t idx = (size_t)(I * ST + il2) * N + J * ST + jl2;
        const double a = tA[jl2][il2], g = tG[jl2][il2];
        A[idx] = a;
        G[idx] = g;
        mK = max(mK, bexp_of(a));   // off the diagonal (I < J): no shift
        mG = max(mG, bexp_of(g));
    }
    if (emaxK) {   // rows J*ST + jl2: the mirrored tile's columns
        redK[warp][jl2] = mK;
        redG[warp][jl2] = mG;
        __syncthreads();
        if (threadIdx.x < ST) {
            int k = redK[0][threadIdx.x], g = redG[0][threadIdx.x];
            for (int w = 1; w < 8; ++w) {
                k = max(k, redK[w][threadIdx.x]);
                g = max(g, redG[w][threadIdx.x]);
            }
            atomicMax(&emaxK[J * ST + threadIdx.x], k);
            atomicMax(&emaxG[J * ST + threadIdx.x], g);
        }
    }
}

}  // namespace

int launch_assemble(Ctx *c) {
    if (c->N % ST == 0) {
        const int T = c->N / ST;
        auto kern = c->deep ? k_assemble_sym<true> : k_assemble_sym<false>;
        // the mixed form's digit splits of K and G need each row's largest
        // exponent: taken here, while the entries are in registers
        const bool emax = c->emax_K != nullptr && !c->one_col;
        if (emax) {
            WW_CUDA_TRY(cudaMemsetAsync(c->emax_K, 0, sizeof(int) * c->N, c->stream));
            WW_CUDA_TRY(cudaMemsetAsync(c->emax_G, 0, sizeof(int) * c->N, c->stream));
        }
        kern<<<T * (T + 1) / 2, 256, 0, c->stream>>>(c->eta, c->eta_x, c->eta_xx, c->E, c->Einv, c->cs,
                                                     c->cs + 2 * c->N, c->N, c->trans, c->A, c->G,
                                                     emax ? c->emax_K : nullptr, emax ? c->emax_G : nullptr);
        c->emax_ready = emax;
        WW_CUDA_TRY(cudaGetLastError());
        return WW_OK;
    }
    c->emax_ready = false;
    dim3 grid((c->N + ASM_TI - 1) / ASM_TI, (c->N + ASM_TJ - 1) / ASM_TJ);
    k_assemble<<<grid, ASM_TI, 0, c->stream>>>(c->eta, c->eta_x, c->eta_xx, c->E, c->Einv, c->cs, c->cs + 2 * c->N,
                                               c->N, c->deep ? 1 : 0, c->trans, c->A, c->G);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

namespace {
__global__ void k_recip_test(const double *d, int n, double *maxrel) {
    __shared__ double red[8];
    double m = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double q = 1.0 / d[k];
        m = fmax(m, fabs(recip_nr(d[k]) - q) / q);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = fmax(m, red[w]);
        *maxrel = fmax(m, red[0]);
    }
}
}  // namespace

}  // namespace ww

// self-test (declared in ww.h): max |recip_nr(d) - 1/d| / (1/d) over the n
// positive device doubles d (the assembly's reciprocal against the division)
extern "C" int ww_selftest_recip(const double *d, int n, double *max_rel) {
    using namespace ww;
    if (!d || n <= 0 || !max_rel) return fail(WW_ERR_ARG, "ww_selftest_recip: bad argument");
    double *m = nullptr;
    if (cudaMalloc(&m, sizeof(double)) != cudaSuccess) return fail(WW_ERR_ALLOC, "selftest alloc");
    k_recip_test<<<1, 256>>>(d, n, m);
    cudaError_t e = cudaMemcpy(max_rel, m, sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(m);
    if (e != cudaSuccess) return fail(WW_ERR_CUDA, std::string("ww_selftest_recip: ") + cudaGetErrorString(e));
    return WW_OK;
}
