// ww_mixed.cu -- mixed-precision DtN linear algebra (WW_MIXED).
//
// A = 1/2 I + K is a second-kind operator with condition number ~2 on the
// workloads here (its flat-surface spectrum is 1/2 (1 + exp(-2|k|h)) and the
// paper's GMRES converges in 4-30 iterations, Sec. 2.2), so an FP32-accurate
// approximate inverse X is an excellent preconditioner for iterative
// refinement (Sec. 3.3 uses the same split: residuals in higher precision,
// corrections in lower precision):
//
//   * X is kept from stage to stage and updated by one Newton-Schulz step
//     X <- X (2I - A X) per stage (from X = 4/3 I with several steps on the
//     first call); both products run on the bf16 tensor cores with 3 + 3
//     slices (FP32-accurate);
//   * M = X Psi; repeat { R = Psi - 1/2 M - K M (FP64-accurate, ww_ozaki.cu);
//     M += X R } max_refine times; the residual after the last correction
//     (estimated from the observed contraction, see mixed_solve) is checked
//     against refine_tol (relative to max|Psi| + max|M| per column) and a
//     miss raises WW_ERR_NO_CONVERGENCE;
//   * G gamma is FP64-accurate (ww_ozaki.cu).
// Single-column solves (the base state) use FP64 residuals and G products on
// the FP64 pipe instead, where a tensor-core tile would be 99% padding.
#include <cuda_bf16.h>

#include "ww_internal.cuh"

namespace ww {

// ww_tcgemm.cu
int tc_slice_f32(cudaStream_t s, const float *src, int ld, int rows, int K, int trans, float shift, int S,
                 __nv_bfloat16 *dst, unsigned *dev_max = nullptr);
int tc_slice_f64(cudaStream_t s, const double *src, int ld, int rows, int K, int trans, float shift, int S,
                 __nv_bfloat16 *dst);
int tc_gemm_f32acc(cudaStream_t s, const __nv_bfloat16 *A3, const __nv_bfloat16 *B3, int M, int Nn, int K,
                   int out_mode, float *Cf, double *Cd, int ldc, double alpha, int *err);
// ww_ozaki.cu
int ozaki_digits(cudaStream_t s, const double *X, int ld, int rows, int K, int side, float diag_shift, int *emax,
                 double *scale, __nv_bfloat16 *dst);
int ozaki_gemm(cudaStream_t s, const __nv_bfloat16 *Ad, const double *sa, const __nv_bfloat16 *Bd, const double *sb,
               int M, int Nn, int K, int mode, double *C, int ldc, const double *Psi, int ldpsi, const double *Mh,
               int ldm, unsigned long long *colmax, int *err);

constexpr int NS_INIT = 6;      // Newton-Schulz steps from X = 4/3 I
constexpr int SMALL_COLS = 8;   // solves / G products this narrow use the FP64 pipe

struct Mixed {
    float *X, *P;                          // approximate inverse, N x N work (column-major)
    __nv_bfloat16 *Aslc, *XslcB, *XslcA, *Wslc;   // 3-slice operands (3 x N x N)
    __nv_bfloat16 *Kd, *Gd;                // 7-digit left operands (7 x N x N)
    double *Ks, *Gs;                       // their row scales
    int *Ke, *Ge;                          // row exponent work
    __nv_bfloat16 *Rd;                     // 7-digit right operand (7 x NC x N)
    double *Rs;                            // column scales
    int *Re;
    __nv_bfloat16 *Bslc;                   // 3-slice right operand (3 x NC x N)
    double *R, *Psi;                       // N x NC
    double *psis;                          // N... column scales of Psi
    int *psie;
    unsigned long long *colmax, *colmax0;  // NC: max|R_j| of the last and the previous residual
    double *ratio;                         // worst final residual ratio (device, bits as u64)
    unsigned *nsres;                       // worst max|I - A X| before an update (fp32 bits)
    int *err;
};

namespace {

__global__ void k_scaled_identity(float *X, int N, float v) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < (size_t)N * N) X[i] = ((i % N) == (i / N)) ? v : 0.f;
}

// per-column residual check: ratio = r_j / (max|Psi_j| + max|M_j|), where
// r_j = max|R_j| of the last residual, or, given the previous one, the
// contraction estimate max|R_j|^2 / max|R_prev,j| of the residual after the
// last correction
__global__ void k_check(const unsigned long long *colmax, const unsigned long long *colmax_prev, const double *psis,
                        const double *ms, int ncols, double tol, unsigned long long *ratio, int *status) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ncols) return;
    double r = __longlong_as_double((long long)colmax[j]);
    if (colmax_prev) {
        const double rp = __longlong_as_double((long long)colmax_prev[j]);
        r = rp > 0 ? r * (r / rp) : r;
    }
    const double den = psis[j] + ms[j];
    const double q = den > 0 ? r / den : (r > 0 ? 1.0 : 0.0);
    atomicMax(ratio, (unsigned long long)__double_as_longlong(q));
    if (!(q <= tol)) atomicOr(status, ST_NO_CONV);
}

// column max |.| of an N x ncols column-major block (bits of a positive double)
__global__ void k_colmax(const double *X, int N, unsigned long long *colmax) {
    __shared__ double red[32];
    const double *col = X + (size_t)blockIdx.x * N;
    double m = 0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) m = fmax(m, fabs(col[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) colmax[blockIdx.x] = (unsigned long long)__double_as_longlong(m);
    }
}

__global__ void k_colscale_from_max(const unsigned long long *colmax, int n, double *scale) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) scale[j] = __longlong_as_double((long long)colmax[j]);
}

template <typename T>
int alloc(Ctx *c, T **p, size_t n) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (n ? n : 1));
    if (e != cudaSuccess) return fail(WW_ERR_ALLOC, std::string("mixed workspace: ") + cudaGetErrorString(e));
    return WW_OK;
}

// one Newton-Schulz step X <- X (2I - A X), all products FP32-accurate;
// record: fold max|I - A X| (the contraction of this stage's refinement
// before the update) into the diagnostics
int ns_step(Ctx *c, bool record) {
    Mixed *m = c->mx;
    const int N = c->N;
    cudaStream_t s = c->stream;
    WW_TRY(tc_slice_f32(s, m->X, N, N, N, 0, 0.f, 3, m->XslcB));                 // columns of X
    WW_TRY(tc_gemm_f32acc(s, m->Aslc, m->XslcB, N, N, N, 0, m->P, nullptr, N, 1.0, m->err));   // P = A X
    WW_TRY(tc_slice_f32(s, m->P, N, N, N, 0, 2.f, 3, m->Wslc, record ? m->nsres : nullptr));   // columns of 2I - P
    WW_TRY(tc_slice_f32(s, m->X, N, N, N, 1, 0.f, 3, m->XslcA));                 // rows of X
    WW_TRY(tc_gemm_f32acc(s, m->XslcA, m->Wslc, N, N, N, 0, m->X, nullptr, N, 1.0, m->err));   // X = X W
    return WW_OK;
}

// R = Psi - A M on the FP64 pipe (narrow blocks); colmax <- max|R_j|
int resid_fp64(Ctx *c, const double *M, int ncols, unsigned long long *colmax) {
    Mixed *m = c->mx;
    const int N = c->N;
    WW_CUDA_TRY(cudaMemcpyAsync(m->R, m->Psi, sizeof(double) * N * ncols, cudaMemcpyDeviceToDevice, c->stream));
    WW_TRY(dgemm(c->stream, N, ncols, N, -1.0, c->A, N, M, N, 1.0, m->R, N));
    k_colmax<<<ncols, 256, 0, c->stream>>>(m->R, N, colmax);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

// R = Psi - A M FP64-accurately on the tensor cores (wide blocks); colmax
// (zeroed by the caller) <- max|R_j|
int resid_ozaki(Ctx *c, const double *M, int ncols, unsigned long long *colmax) {
    Mixed *m = c->mx;
    const int N = c->N;
    WW_TRY(ozaki_digits(c->stream, M, N, ncols, N, 1, 0.f, m->Re, m->Rs, m->Rd));
    WW_TRY(ozaki_gemm(c->stream, m->Kd, m->Ks, m->Rd, m->Rs, N, ncols, N, 1, m->R, N, m->Psi, N, M, N, colmax,
                      m->err));
    return WW_OK;
}

}  // namespace

int mixed_create(Ctx *c) {
    Mixed *m = new Mixed();
    memset(m, 0, sizeof(Mixed));
    c->mx = m;
    const size_t N = c->N, NC = c->NC, NN = N * N;
    int st = WW_OK;
#define MA(p, n) \
    if (st == WW_OK) st = alloc(c, &(p), (n))
    MA(m->X, NN);
    MA(m->P, NN);
    MA(m->Aslc, 3 * NN);
    MA(m->XslcB, 3 * NN);
    MA(m->XslcA, 3 * NN);
    MA(m->Wslc, 3 * NN);
    MA(m->Kd, 7 * NN);
    MA(m->Gd, 7 * NN);
    MA(m->Ks, N);
    MA(m->Gs, N);
    MA(m->Ke, N);
    MA(m->Ge, N);
    MA(m->Rd, (7 * NC + 256) * N);   // + rows so that a TMA box never leaves the buffer
    MA(m->Rs, NC);
    MA(m->Re, NC);
    MA(m->Bslc, (3 * NC + 256) * N);
    MA(m->R, N * NC);
    MA(m->Psi, N * NC);
    MA(m->psis, NC);
    MA(m->psie, NC);
    MA(m->colmax, NC);
    MA(m->colmax0, NC);
    MA(m->ratio, 1);
    MA(m->nsres, 1);
    MA(m->err, 1);
#undef MA
    if (st != WW_OK) return st;
    WW_CUDA_TRY(cudaMemset(m->err, 0, sizeof(int)));
    WW_CUDA_TRY(cudaMemset(m->ratio, 0, sizeof(double)));
    WW_CUDA_TRY(cudaMemset(m->nsres, 0, sizeof(unsigned)));
    return WW_OK;
}

void mixed_destroy(Ctx *c) {
    Mixed *m = c->mx;
    if (!m) return;
    void *ptrs[] = {m->X,  m->P,  m->Aslc, m->XslcB, m->XslcA, m->Wslc, m->Kd,  m->Gd,   m->Ks,     m->Gs,    m->Ke,
                    m->Ge, m->Rd, m->Rs,   m->Re,    m->Bslc,  m->R,    m->Psi, m->psis, m->psie, m->colmax, m->colmax0,
                    m->ratio, m->nsres, m->err};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete m;
    c->mx = nullptr;
}

// after assembly: update X (fresh: from 4/3 I) and build the operands of this stage
int mixed_setup(Ctx *c, int fresh) {
    Mixed *m = c->mx;
    const int N = c->N;
    cudaStream_t s = c->stream;
    WW_TRY(tc_slice_f64(s, c->A, N, N, N, 1, 0.f, 3, m->Aslc));   // rows of A
    if (fresh) {
        const size_t NN = (size_t)N * N;
        k_scaled_identity<<<(unsigned)((NN + 255) / 256), 256, 0, s>>>(m->X, N, 4.f / 3.f);
        WW_CUDA_TRY(cudaGetLastError());
        for (int i = 0; i < NS_INIT; ++i) WW_TRY(ns_step(c, false));
    } else {
        WW_TRY(ns_step(c, true));
    }
    WW_TRY(tc_slice_f32(s, m->X, N, N, N, 1, 0.f, 3, m->XslcA));   // rows of the new X
    WW_TRY(ozaki_digits(s, c->A, N, N, N, 0, 0.5f, m->Ke, m->Ks, m->Kd));   // K = A - I/2
    WW_TRY(ozaki_digits(s, c->G, N, N, N, 0, 0.f, m->Ge, m->Gs, m->Gd));
    return WW_OK;
}

// B (N x ncols) <- A^{-1} B
int mixed_solve(Ctx *c, double *B, int ncols) {
    Mixed *m = c->mx;
    const int N = c->N;
    cudaStream_t s = c->stream;
    const bool narrow = ncols <= SMALL_COLS;
    WW_CUDA_TRY(cudaMemcpyAsync(m->Psi, B, sizeof(double) * N * ncols, cudaMemcpyDeviceToDevice, s));
    // column scales of Psi (for the convergence test)
    k_colmax<<<ncols, 256, 0, s>>>(m->Psi, N, m->colmax);
    k_colscale_from_max<<<(ncols + 255) / 256, 256, 0, s>>>(m->colmax, ncols, m->psis);
    WW_CUDA_TRY(cudaGetLastError());
    // M = X Psi
    WW_TRY(tc_slice_f64(s, m->Psi, N, ncols, N, 0, 0.f, 3, m->Bslc));
    WW_TRY(tc_gemm_f32acc(s, m->XslcA, m->Bslc, N, ncols, N, 1, nullptr, B, N, 1.0, m->err));
    // R_k = Psi - A M_k (FP64-accurate), M_{k+1} = M_k + X R_k.  With two or
    // more corrections the final residual is not recomputed: per column it is
    // estimated as |R_last| rho with the observed contraction rho = |R_last| /
    // |R_prev| (the iteration is linear with a fixed X), which saves one
    // FP64-accurate product per solve.  With one correction it is recomputed.
    unsigned long long *cm_prev = m->colmax0, *cm = m->colmax;
    const int nres = c->max_refine >= 2 ? c->max_refine : c->max_refine + 1;
    for (int it = 0; it < nres; ++it) {
        if (it > 0) {
            unsigned long long *t = cm_prev;
            cm_prev = cm;
            cm = t;
        }
        if (narrow) {
            WW_TRY(resid_fp64(c, B, ncols, cm));
        } else {
            WW_CUDA_TRY(cudaMemsetAsync(cm, 0, sizeof(unsigned long long) * ncols, s));
            WW_TRY(resid_ozaki(c, B, ncols, cm));
        }
        if (it == c->max_refine) break;   // one correction: the last residual is the check
        WW_TRY(tc_slice_f64(s, m->R, N, ncols, N, 0, 0.f, 3, m->Bslc));
        WW_TRY(tc_gemm_f32acc(s, m->XslcA, m->Bslc, N, ncols, N, 2, nullptr, B, N, 1.0, m->err));   // M += X R
    }
    // convergence test (scales of M: column max of the solution)
    k_colmax<<<ncols, 256, 0, s>>>(B, N, reinterpret_cast<unsigned long long *>(m->Rs));
    k_colscale_from_max<<<(ncols + 255) / 256, 256, 0, s>>>(reinterpret_cast<unsigned long long *>(m->Rs), ncols,
                                                            m->Rs);
    k_check<<<(ncols + 127) / 128, 128, 0, s>>>(cm, c->max_refine >= 2 ? cm_prev : nullptr, m->psis, m->Rs, ncols,
                                                c->refine_tol, reinterpret_cast<unsigned long long *>(m->ratio),
                                                c->status);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

// Gout[:, col0 .. col0+ncols) += G Gam[:, col0 ..]
int mixed_apply_G(Ctx *c, int col0, int ncols) {
    Mixed *m = c->mx;
    const int N = c->N;
    const double *Gam = c->Gam + (size_t)col0 * N;
    double *Out = c->Gout + (size_t)col0 * N;
    if (ncols <= SMALL_COLS) return dgemm(c->stream, N, ncols, N, 1.0, c->G, N, Gam, N, 1.0, Out, N);
    WW_TRY(ozaki_digits(c->stream, Gam, N, ncols, N, 1, 0.f, m->Re, m->Rs, m->Rd));
    return ozaki_gemm(c->stream, m->Gd, m->Gs, m->Rd, m->Rs, N, ncols, N, 0, Out, N, nullptr, 0, nullptr, 0, nullptr,
                      m->err);
}

// device diagnostics of the mixed path, read (and reset) after a call
int mixed_read_stats(Ctx *c, double *ratio, double *nsres, int *err) {
    Mixed *m = c->mx;
    unsigned nb = 0;
    WW_CUDA_TRY(cudaMemcpyAsync(ratio, m->ratio, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    WW_CUDA_TRY(cudaMemcpyAsync(&nb, m->nsres, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    WW_CUDA_TRY(cudaMemcpyAsync(err, m->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    WW_CUDA_TRY(cudaStreamSynchronize(c->stream));
    float nf;
    memcpy(&nf, &nb, sizeof(nf));
    *nsres = nf;
    WW_CUDA_TRY(cudaMemsetAsync(m->ratio, 0, sizeof(double), c->stream));
    WW_CUDA_TRY(cudaMemsetAsync(m->nsres, 0, sizeof(unsigned), c->stream));
    WW_CUDA_TRY(cudaMemsetAsync(m->err, 0, sizeof(int), c->stream));
    return WW_OK;
}

}  // namespace ww
