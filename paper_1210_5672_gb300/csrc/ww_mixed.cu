// ww_mixed.cu -- mixed-precision DtN linear algebra (WW_MIXED).
//
// A = 1/2 I + K is a second-kind operator with condition number ~2 on the
// workloads here (its flat-surface spectrum is 1/2 (1 + exp(-2|k|h)) and the
// paper's GMRES converges in 4-30 iterations, Sec. 2.2), so an FP32-accurate
// approximate inverse X is an excellent preconditioner for iterative
// refinement (Sec. 3.3 uses the same split: residuals in higher precision,
// corrections in lower precision):
//
//   * X is kept from stage to stage and moved to the current A by a
//     Newton-Schulz step X <- X (2I - A X) (from X = 4/3 I with several steps
//     on the first call); both products run on the bf16 tensor cores with
//     3 + 3 slices (FP32-accurate).  Every other stage reuses the X of the
//     stage before when the last update found it close (max|I - A X| below
//     NS_SKIP), a decision taken on the device;
//   * M = X Psi; then up to max_refine times { R = Psi - 1/2 M - K M
//     (FP64-accurate, ww_ozaki.cu); M += X R } until the residual after the
//     last correction -- estimated per column as |R_k|^2 / |R_{k-1}| from the
//     observed contraction -- is below refine_tol (relative to max|Psi| +
//     max|M|).  The test runs on the device; the remaining iterations of a
//     converged solve are launched but return at once, so the step program
//     stays one CUDA graph.  A solve that does not converge raises
//     WW_ERR_NO_CONVERGENCE.  The products with X in this loop use 2 + 2
//     slices (~2^-16 relative): their error only adds to the contraction
//     factor of the iteration, the residuals stay FP64-accurate;
//   * G gamma is FP64-accurate (ww_ozaki.cu).
// Single-column solves (the base state) use FP64 residuals and FP32 products
// with X on the CUDA cores instead, where a tensor-core tile would be 99%
// padding.
#include <cuda_bf16.h>

#include "ww_internal.cuh"
#include "ww_tc.cuh"

namespace ww {

// ww_tcgemm.cu
int tc_slice_f32(cudaStream_t s, const float *src, int ld, int rows, int K, int trans, float shift, int S,
                 __nv_bfloat16 *dst, unsigned *dev_max = nullptr, const int *skip = nullptr, int run_if_skipped = 0);
int tc_slice_f64(cudaStream_t s, const double *src, int ld, int rows, int K, int trans, float shift, int S,
                 __nv_bfloat16 *dst, const int *skip = nullptr);
int tc_gemm_f32acc(cudaStream_t s, const __nv_bfloat16 *A3, const __nv_bfloat16 *B3, int M, int Nn, int K,
                   int out_mode, float *Cf, double *Cd, int ldc, double alpha, int *err, const int *skip = nullptr);
int tc_gemm_2x2(cudaStream_t s, const __nv_bfloat16 *A2, const __nv_bfloat16 *B2, int M, int Nn, int K, int out_mode,
                float *Cf, double *Cd, int ldc, double alpha, int *err, const int *skip, int bn);
int tc_gemm_f32acc_sliced(cudaStream_t s, const __nv_bfloat16 *A3, const __nv_bfloat16 *B3, int M, int Nn, int K,
                          const TcOut &o, int *err, const int *skip, int bn, int ctas);
// ww_ozaki.cu
int ozaki_digits(cudaStream_t s, const double *X, int ld, int rows, int K, int side, float diag_shift, int *emax,
                 double *scale, __nv_bfloat16 *dst, const int *skip);
int ozaki_gemm(cudaStream_t s, const __nv_bfloat16 *Ad, const double *sa, const __nv_bfloat16 *Bd, const double *sb,
               int M, int Nn, int K, int mode, double *C, int ldc, const double *Psi, int ldpsi, const double *Mh,
               int ldm, unsigned long long *colmax, int *err, const int *skip, __nv_bfloat16 *rslc = nullptr,
               int nd = 7);
int ozaki_digits_rows_emax(cudaStream_t s, const double *X, int ld, int rows, int K, float diag_shift,
                           const int *emax, double *scale, __nv_bfloat16 *dst, const int *skip);
int ozaki_digits_cols(cudaStream_t s, const double *X, int ld, int ncols, int K, double *scale, __nv_bfloat16 *dst,
                      unsigned long long *zero_cm, const int *skip);

constexpr int NS_INIT = 6;          // Newton-Schulz steps from X = 4/3 I
constexpr int SMALL_COLS = 8;       // solves / G products this narrow use the CUDA cores
constexpr float NS_SKIP = 1e-5f;    // max|I - A X| at the last update that lets the next stage reuse X

// scratch of one refinement loop (the base column's narrow solve and the
// columns' wide solve run on different streams, so each has its own)
struct SolveWs {
    double *R, *Psi;                       // N x width
    double *psis, *mscale;                 // width: column maxima of Psi and of the solution
    unsigned long long *colmax, *colmax0;  // width: max|R_j| of the last and the previous residual
    int *done;                             // device decision: the current solve has converged
};

struct Mixed {
    float *X;                              // approximate inverse (column-major)
    __nv_bfloat16 *Aslc, *XslcB, *XslcA, *Wslc;   // 3-slice operands of the inverse update (3 x N x N)
    __nv_bfloat16 *XnA, *XnB;              // the new X's slices, written by the update's second product
    // per-stage operands of the column solves and G-apply, double-buffered by
    // stage parity: the base chain builds stage s+1's while the columns of
    // stage s still read stage s's
    __nv_bfloat16 *Xrow[2];                // 3 slices of the rows of X
    __nv_bfloat16 *Kd[2], *Gd[2];          // 7-digit left operands (7 x N x N) of K = A - I/2 and G
    double *Ks[2], *Gs[2];                 // their row scales
    int *Ke, *Ge;                          // row exponent work
    __nv_bfloat16 *Rd;                     // 7-digit right operand ((7 NC + 256) x N)
    double *Rs;                            // its column scales
    int *Re;
    __nv_bfloat16 *Bslc;                   // 3-slice right operand ((3 NC + 256) x N)
    SolveWs wide, nar;
    double *ratio;                         // worst final residual ratio (bits of a double)
    unsigned *nsres, *nsres_last;          // max|I - A X| before an update: worst, and the latest (fp32 bits)
    int *ns_skip;                          // device decision: this stage reuses the previous X
    int *maxit;                            // [2] most corrections a wide solve of each stage parity took in this shot
    int *iters;                            // [0] most residuals any solve needed, [1] their sum, [2] solves
    int *err;
    // measured residual of sampled wide solves (ww_set_verify)
    unsigned long long *vcm;               // NC: max|R_j| of the verification product
    int *vcount, *vskip;                   // wide solves seen this call; this one is not sampled
    double *vmax;                          // worst measured relative residual (bits of a double)
    int *vn;                               // sampled solves this call
};

namespace {

// reuse X when the last update left max|I - A X| below thr and (maxit, when
// given) no wide solve of this stage parity has yet needed three corrections
__global__ void k_ns_decide(const unsigned *nsres_last, float thr, const int *maxit, int *skip) {
    *skip = (__uint_as_float(*nsres_last) < thr && (!maxit || *maxit < 3)) ? 1 : 0;
}

__global__ void k_fold_nsres(const unsigned *last, unsigned *worst) { atomicMax(worst, *last); }

__global__ void k_scaled_identity(float *X, int N, float v) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < (size_t)N * N) X[i] = ((i % N) == (i / N)) ? v : 0.f;
}

// block max of v (256-thread blocks), every thread gets it
__device__ __forceinline__ double block_max256(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double m = red[0];
    for (int w = 1; w < 8; ++w) m = fmax(m, red[w]);
    __syncthreads();
    return m;
}

// narrow solves, before the first product: Psi = B (one column per block)
// and its column maxima as scales
__global__ void __launch_bounds__(256) k_narrow_prep(const double *__restrict__ B, int N, double *Psi, double *psis) {
    __shared__ double red[8];
    const double *b = B + (size_t)blockIdx.x * N;
    double *p = Psi + (size_t)blockIdx.x * N;
    double m = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double v = b[i];
        p[i] = v;
        m = fmax(m, fabs(v));
    }
    m = block_max256(m, red);
    if (threadIdx.x == 0) psis[blockIdx.x] = m;
}

// narrow solves, after a residual: max|R_j| (bits, for the convergence test)
// and max|M_j| (the test's scale) in one pass, one column per block
__global__ void __launch_bounds__(256) k_narrow_maxima(const double *__restrict__ R, const double *__restrict__ M,
                                                       int N, unsigned long long *cm, double *ms, const int *skip) {
    if (skip && *skip) return;
    __shared__ double red[8];
    const double *r = R + (size_t)blockIdx.x * N, *mm = M + (size_t)blockIdx.x * N;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        a = fmax(a, fabs(r[i]));
        b = fmax(b, fabs(mm[i]));
    }
    a = block_max256(a, red);
    b = block_max256(b, red);
    if (threadIdx.x == 0) {
        cm[blockIdx.x] = (unsigned long long)__double_as_longlong(a);
        ms[blockIdx.x] = b;
    }
}

// Convergence test after residual `it` (0-based) and its correction: per
// column the residual left after the correction is estimated as
// |R_it| (|R_it| / |R_it-1|) (the refinement is a linear iteration with a
// fixed X), relative to max|Psi| + max|M|.  Sets *done when every column is
// below tol; on the last allowed iteration a miss raises ST_NO_CONV.  maxit
// (wide solves; NULL for narrow ones) keeps the most corrections a solve of
// this stage parity has taken in the shot, which the shot-adaptive inverse
// cadence reads.  One block; returns at once when an earlier call already
// set *done.
__global__ void k_converged(const unsigned long long *cm, const unsigned long long *cm_prev, const double *psis,
                            const double *ms, int ncols, double tol, int it, int last, int *done, int *iters,
                            unsigned long long *ratio, int *status, int *maxit) {
    if (*done) return;
    __shared__ double red[32];
    double worst = 0.0;
    for (int j = threadIdx.x; j < ncols; j += blockDim.x) {
        const double r = __longlong_as_double((long long)cm[j]);
        double est;
        if (cm_prev) {
            const double rp = __longlong_as_double((long long)cm_prev[j]);
            est = rp > 0 ? r * (r / rp) : r;
        } else {
            est = r > 0 ? INFINITY : 0.0;   // one residual: no contraction estimate yet
        }
        const double den = psis[j] + ms[j];
        const double q = den > 0 ? est / den : (est > 0 ? INFINITY : 0.0);
        worst = fmax(worst, q);
    }
    for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = worst;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) worst = fmax(worst, red[w]);
        worst = fmax(worst, red[0]);
        if (maxit && (worst <= tol || last)) atomicMax(maxit, it + 1);
        if (worst <= tol) {
            *done = 1;
            atomicMax(iters, it + 1);
            atomicAdd(iters + 1, it + 1);
            atomicAdd(iters + 2, 1);
            atomicMax(ratio, (unsigned long long)__double_as_longlong(worst));
        } else if (last) {
            atomicOr(status, ST_NO_CONV);
            atomicMax(iters, it + 1);
            atomicAdd(iters + 1, it + 1);
            atomicAdd(iters + 2, 1);
            if (isfinite(worst)) atomicMax(ratio, (unsigned long long)__double_as_longlong(worst));
        }
    }
}

// Sampling of the verified solves: solve number *count is measured when it is
// a multiple of `every`.
__global__ void k_verify_tick(int *count, int every, int *skip) {
    *skip = (*count % every) != 0;
    *count += 1;
}

// worst measured relative residual of one sampled solve:
// max_j max|R_j| / (max|Psi_j| + max|M_j|), the normalisation of k_converged
__global__ void k_verify_fold(const unsigned long long *cm, const double *psis, const double *ms, int ncols,
                              const int *skip, unsigned long long *vmax, int *vn) {
    if (*skip) return;
    __shared__ double red[32];
    double worst = 0.0;
    for (int j = threadIdx.x; j < ncols; j += blockDim.x) {
        const double r = __longlong_as_double((long long)cm[j]);
        const double den = psis[j] + ms[j];
        worst = fmax(worst, den > 0 ? r / den : (r > 0 ? INFINITY : 0.0));
    }
    for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = worst;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) worst = fmax(worst, red[w]);
        worst = fmax(worst, red[0]);
        atomicMax(vmax, (unsigned long long)__double_as_longlong(worst));
        atomicAdd(vn, 1);
    }
}

// Start of a wide solve, one block per column: Psi <- B, max|Psi_j| -> psis,
// and the 2 bf16 slices of Psi as the right operand of X Psi.
__global__ void k_prep_psi(const double *__restrict__ B, int N, int ncols, double *Psi, double *psis,
                           __nv_bfloat16 *slc) {
    __shared__ double red[32];
    const int col = blockIdx.x;
    const double *b = B + (size_t)col * N;
    double m = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double x = b[i];
        Psi[(size_t)col * N + i] = x;
        m = fmax(m, fabs(x));
        float v = (float)x;
        const __nv_bfloat16 b0 = __float2bfloat16_rn(v);
        v -= __bfloat162float(b0);
        slc[(size_t)col * N + i] = b0;
        slc[((size_t)ncols + col) * N + i] = __float2bfloat16_rn(v);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) psis[col] = m;
    }
}

template <typename T>
int alloc(T **p, size_t n) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (n ? n : 1));
    if (e != cudaSuccess) return fail(WW_ERR_ALLOC, std::string("mixed workspace: ") + cudaGetErrorString(e));
    return WW_OK;
}

// one Newton-Schulz step X <- X (2I - A X), all products FP32-accurate;
// record: keep max|I - A X| (before the update) for the skip decision and the
// diagnostics; skip: device flag that turns the whole step into no-ops
int ns_step(Ctx *c, bool record, const int *skip) {
    Mixed *m = c->mx;
    const int N = c->N;
    cudaStream_t s = c->stream;
    if (record) WW_CUDA_TRY(cudaMemsetAsync(m->nsres_last, 0, sizeof(unsigned), s));
    // W = 2I - A X, written straight as the slices of the next product's right operand
    if (record) WW_TRY(phase_mark(c, WW_PHASE_INVERSE, 0));
    TcOut o3{};
    o3.mode = 3;
    o3.shift = 2.f;
    o3.s_col = m->Wslc;
    o3.dev_max = record ? m->nsres_last : nullptr;
    WW_TRY(tc_gemm_f32acc_sliced(s, m->Aslc, m->XslcB, N, N, N, o3, m->err, skip, c->sch.inv_bn, c->sch.inv_ctas));
    // X <- X W: the FP32 X, its slices for the next update, and this stage's rows of X
    TcOut o4{};
    o4.mode = 4;
    o4.Cf = m->X;
    o4.ldc = N;
    o4.s_col = m->XnB;
    o4.s_row = m->XnA;
    o4.s_row2 = m->Xrow[c->par];
    WW_TRY(tc_gemm_f32acc_sliced(s, m->XslcA, m->Wslc, N, N, N, o4, m->err, skip, c->sch.inv_bn, c->sch.inv_ctas));
    if (record) WW_TRY(phase_mark(c, WW_PHASE_INVERSE, 1));
    // the product above still reads XslcA while it writes: its slices land in XnA / XnB
    // and move over afterwards (after a skipped update both already hold the same data)
    const size_t bytes = sizeof(__nv_bfloat16) * 3 * (size_t)N * N;
    WW_CUDA_TRY(cudaMemcpyAsync(m->XslcA, m->XnA, bytes, cudaMemcpyDeviceToDevice, s));
    WW_CUDA_TRY(cudaMemcpyAsync(m->XslcB, m->XnB, bytes, cudaMemcpyDeviceToDevice, s));
    if (record) {
        k_fold_nsres<<<1, 1, 0, s>>>(m->nsres_last, m->nsres);
        WW_CUDA_TRY(cudaGetLastError());
    }
    return WW_OK;
}

}  // namespace

int mixed_create(Ctx *c) {
    WW_TRY(tc_init());
    Mixed *m = new Mixed();
    memset(m, 0, sizeof(Mixed));
    c->mx = m;
    const size_t N = c->N, NC = c->NC, NN = N * N;
    int st = WW_OK;
#define MA(p, n)                                                \
    if (st == WW_OK) {                                          \
        st = alloc(&(p), (n));                                  \
        c->dev_bytes += sizeof(*(p)) * (size_t)((n) ? (n) : 1); \
    }
    MA(m->X, NN);
    MA(m->XnA, 3 * NN);
    MA(m->XnB, 3 * NN);
    MA(m->Aslc, 3 * NN);
    MA(m->XslcB, 3 * NN);
    MA(m->XslcA, 3 * NN);
    MA(m->Wslc, 3 * NN);
    for (int q = 0; q < 2; ++q) {
        MA(m->Xrow[q], 3 * NN);
        MA(m->Kd[q], 7 * NN);
        MA(m->Gd[q], 7 * NN);
        MA(m->Ks[q], N);
        MA(m->Gs[q], N);
    }
    MA(m->Ke, N);
    MA(m->Ge, N);
    c->emax_K = m->Ke;
    c->emax_G = m->Ge;
    MA(m->Rd, (7 * NC + 256) * N);   // + rows so that a TMA box never leaves the buffer
    MA(m->Rs, NC);
    MA(m->Re, NC);
    MA(m->Bslc, (3 * NC + 256) * N);
    SolveWs *ws[2] = {&m->wide, &m->nar};
    const size_t width[2] = {NC, (size_t)SMALL_COLS};
    for (int q = 0; q < 2; ++q) {
        MA(ws[q]->R, N * width[q]);
        MA(ws[q]->Psi, N * width[q]);
        MA(ws[q]->psis, width[q]);
        MA(ws[q]->mscale, width[q]);
        MA(ws[q]->colmax, width[q]);
        MA(ws[q]->colmax0, width[q]);
        MA(ws[q]->done, 1);
    }
    MA(m->ratio, 1);
    MA(m->nsres, 1);
    MA(m->nsres_last, 1);
    MA(m->ns_skip, 1);
    MA(m->maxit, 2);
    MA(m->iters, 3);
    MA(m->err, 1);
    MA(m->vcm, NC);
    MA(m->vcount, 1);
    MA(m->vskip, 1);
    MA(m->vmax, 1);
    MA(m->vn, 1);
#undef MA
    if (st != WW_OK) return st;
    WW_CUDA_TRY(cudaMemset(m->err, 0, sizeof(int)));
    WW_CUDA_TRY(cudaMemset(m->ratio, 0, sizeof(double)));
    WW_CUDA_TRY(cudaMemset(m->nsres, 0, sizeof(unsigned)));
    WW_CUDA_TRY(cudaMemset(m->nsres_last, 0xFF, sizeof(unsigned)));   // NaN bits: never skip before an update
    WW_CUDA_TRY(cudaMemset(m->ns_skip, 0, sizeof(int)));
    WW_CUDA_TRY(cudaMemset(m->maxit, 0, 2 * sizeof(int)));
    WW_CUDA_TRY(cudaMemset(m->iters, 0, 3 * sizeof(int)));
    WW_CUDA_TRY(cudaMemset(m->vcount, 0, sizeof(int)));
    WW_CUDA_TRY(cudaMemset(m->vmax, 0, sizeof(double)));
    WW_CUDA_TRY(cudaMemset(m->vn, 0, sizeof(int)));
    return WW_OK;
}

void mixed_destroy(Ctx *c) {
    Mixed *m = c->mx;
    if (!m) return;
    void *ptrs[] = {m->X,          m->XnA,         m->XnB,        m->Aslc,       m->XslcB,        m->XslcA,       m->Wslc,
                    m->Xrow[0],     m->Xrow[1],     m->Kd[0],      m->Kd[1],        m->Gd[0],       m->Gd[1],
                    m->Ks[0],       m->Ks[1],       m->Gs[0],      m->Gs[1],        m->Ke,          m->Ge,
                    m->Rd,          m->Rs,          m->Re,         m->Bslc,         m->wide.R,      m->wide.Psi,
                    m->wide.psis,   m->wide.mscale, m->wide.colmax, m->wide.colmax0, m->wide.done,  m->nar.R,
                    m->nar.Psi,     m->nar.psis,    m->nar.mscale, m->nar.colmax,   m->nar.colmax0, m->nar.done,
                    m->ratio,       m->nsres,       m->nsres_last, m->ns_skip,      m->iters,       m->err,
                    m->vcm,         m->vcount,      m->vskip,      m->vmax,         m->vn};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete m;
    c->mx = nullptr;
}

// after assembly: build this stage's operands and move X to this stage's A
// (fresh: from 4/3 I).  With update == 0 the move is left out on the device
// when the last update found max|I - A X| < NS_SKIP (A changes by O(dt) per
// stage, so the refinement contraction only grows from ~1e-7 to a few 1e-6;
// the adaptive refinement absorbs the rest).
int mixed_setup(Ctx *c, int fresh, int update, bool adaptive) {
    Mixed *m = c->mx;
    const int N = c->N;
    cudaStream_t s = c->stream;
    const int *skip = nullptr;
    if (!fresh && !update) {
        k_ns_decide<<<1, 1, 0, s>>>(m->nsres_last, NS_SKIP,
                                    adaptive && c->sch.ns_every == 2 ? m->maxit + c->par : nullptr, m->ns_skip);
        WW_CUDA_TRY(cudaGetLastError());
        skip = m->ns_skip;
    }
    WW_TRY(tc_slice_f64(s, c->A, N, N, N, 1, 0.f, 3, m->Aslc, skip));   // rows of A
    const int q = c->par;
    if (fresh) {
        const size_t NN = (size_t)N * N;
        k_scaled_identity<<<(unsigned)((NN + 255) / 256), 256, 0, s>>>(m->X, N, 4.f / 3.f);
        WW_CUDA_TRY(cudaGetLastError());
        WW_TRY(tc_slice_f32(s, m->X, N, N, N, 0, 0.f, 3, m->XslcB));   // columns of X
        WW_TRY(tc_slice_f32(s, m->X, N, N, N, 1, 0.f, 3, m->XslcA));   // rows of X
        for (int i = 0; i < NS_INIT; ++i) WW_TRY(ns_step(c, false, nullptr));
        WW_CUDA_TRY(cudaMemsetAsync(m->nsres_last, 0xFF, sizeof(unsigned), s));
        WW_CUDA_TRY(cudaMemsetAsync(m->maxit, 0, 2 * sizeof(int), s));   // a new shot
    } else {
        WW_TRY(ns_step(c, skip == nullptr, skip));
    }
    // an update left out on the device leaves this stage's rows of X to a slice of X
    if (skip) WW_TRY(tc_slice_f32(s, m->X, N, N, N, 1, 0.f, 2, m->Xrow[q], nullptr, skip, 1));
    const bool emax_ready = c->emax_ready;
    c->emax_ready = false;
    if (c->one_col) return WW_OK;   // the narrow solves and products read A and G directly
    if (emax_ready) {   // the assembly already took the row exponent maxima
        WW_TRY(ozaki_digits_rows_emax(s, c->A, N, N, N, 0.5f, m->Ke, m->Ks[q], m->Kd[q], nullptr));   // K = A - I/2
        WW_TRY(ozaki_digits_rows_emax(s, c->G, N, N, N, 0.f, m->Ge, m->Gs[q], m->Gd[q], nullptr));
        return WW_OK;
    }
    WW_TRY(ozaki_digits(s, c->A, N, N, N, 0, 0.5f, m->Ke, m->Ks[q], m->Kd[q], nullptr));   // K = A - I/2
    WW_TRY(ozaki_digits(s, c->G, N, N, N, 0, 0.f, m->Ge, m->Gs[q], m->Gd[q], nullptr));
    return WW_OK;
}

// B (N x ncols) <- A^{-1} B
int mixed_solve(Ctx *c, double *B, int ncols) {
    Mixed *m = c->mx;
    const int N = c->N, q = c->par;
    cudaStream_t s = c->stream;
    const bool narrow = ncols <= SMALL_COLS;
    SolveWs &w = narrow ? m->nar : m->wide;
    WW_CUDA_TRY(cudaMemsetAsync(w.done, 0, sizeof(int), s));
    // Psi = B, the column maxima of Psi (scale of the convergence test), M = X Psi
    if (narrow) {
        k_narrow_prep<<<ncols, 256, 0, s>>>(B, N, w.Psi, w.psis);
        WW_CUDA_TRY(cudaGetLastError());
        WW_TRY(gemv_narrow_f32(s, N, ncols, N, m->X, N, w.Psi, N, 0.0, B, N));
    } else {
        k_prep_psi<<<ncols, 256, 0, s>>>(B, N, ncols, w.Psi, w.psis, m->Bslc);
        WW_CUDA_TRY(cudaGetLastError());
        WW_TRY(tc_gemm_2x2(s, m->Xrow[q], m->Bslc, N, ncols, N, 1, nullptr, B, N, 1.0, m->err, nullptr,
                           c->sch.corr_bn));
    }
    unsigned long long *cm_prev = w.colmax0, *cm = w.colmax;
    const int *done = w.done;
    const int nit = c->max_refine < 1 ? 1 : c->max_refine;
    for (int it = 0; it < nit; ++it) {
        // R = Psi - A M_it (FP64-accurate) and max|R_j|, then M += X R
        if (narrow) {
            WW_TRY(resid_narrow(s, N, ncols, N, c->A, N, B, N, w.Psi, N, w.R, N, done));
            k_narrow_maxima<<<ncols, 256, 0, s>>>(w.R, B, N, cm, w.mscale, done);
            WW_CUDA_TRY(cudaGetLastError());
            WW_TRY(gemv_narrow_f32(s, N, ncols, N, m->X, N, w.R, N, 1.0, B, N, done));
        } else {
            // digits and scales of M (scales -> Rs), max|R| reset; the residual
            // kernel writes R straight into the slices of the correction's operand
            WW_TRY(ozaki_digits_cols(s, B, N, ncols, N, m->Rs, m->Rd, cm, done));
            // the first residual's error is contracted by the next correction: 5 digits
            // (2^-35 of the operands' maxima) leave the result within the 7-digit floor
            WW_TRY(ozaki_gemm(s, m->Kd[q], m->Ks[q], m->Rd, m->Rs, N, ncols, N, 1, nullptr, N, w.Psi, N, B, N, cm,
                              m->err, done, m->Bslc, it == 0 ? 5 : 7));
            WW_TRY(tc_gemm_2x2(s, m->Xrow[q], m->Bslc, N, ncols, N, 2, nullptr, B, N, 1.0, m->err, done,
                               c->sch.corr_bn));
        }
        // converged after this correction?
        k_converged<<<1, 512, 0, s>>>(cm, it > 0 ? cm_prev : nullptr, w.psis, narrow ? w.mscale : m->Rs, ncols,
                                      c->refine_tol, it, it == nit - 1, w.done, m->iters,
                                      reinterpret_cast<unsigned long long *>(m->ratio), c->status,
                                      narrow ? nullptr : m->maxit + q);
        WW_CUDA_TRY(cudaGetLastError());
        unsigned long long *t = cm_prev;
        cm_prev = cm;
        cm = t;
    }
    // measured residual of a sampled solve: R = Psi - 1/2 M - K M of the final M,
    // 7 digits, after the last correction (the estimate above extrapolates it)
    if (!narrow && c->verify_every > 0) {
        k_verify_tick<<<1, 1, 0, s>>>(m->vcount, c->verify_every, m->vskip);
        WW_CUDA_TRY(cudaGetLastError());
        WW_TRY(ozaki_digits_cols(s, B, N, ncols, N, m->Rs, m->Rd, m->vcm, m->vskip));
        WW_TRY(ozaki_gemm(s, m->Kd[q], m->Ks[q], m->Rd, m->Rs, N, ncols, N, 1, nullptr, N, w.Psi, N, B, N, m->vcm,
                          m->err, m->vskip, nullptr, 7));
        k_verify_fold<<<1, 512, 0, s>>>(m->vcm, w.psis, m->Rs, ncols, m->vskip,
                                        reinterpret_cast<unsigned long long *>(m->vmax), m->vn);
        WW_CUDA_TRY(cudaGetLastError());
    }
    return WW_OK;
}

// Gout[:, col0 .. col0+ncols) += G Gam[:, col0 ..]
// part 0: split Gam into digits; part 1: the product (the two run back to back)
int mixed_apply_G(Ctx *c, int col0, int ncols, int part) {
    Mixed *m = c->mx;
    const int N = c->N;
    const double *Gam = c->Gam + (size_t)col0 * N;
    double *Out = c->Gout + (size_t)col0 * N;
    if (ncols <= SMALL_COLS) return part == 0 ? WW_OK : dgemm(c->stream, N, ncols, N, 1.0, c->G, N, Gam, N, 1.0, Out, N);
    if (part == 0) return ozaki_digits(c->stream, Gam, N, ncols, N, 1, 0.f, m->Re, m->Rs, m->Rd, nullptr);
    return ozaki_gemm(c->stream, m->Gd[c->par], m->Gs[c->par], m->Rd, m->Rs, N, ncols, N, 0, Out, N, nullptr, 0, nullptr, 0, nullptr,
                      m->err, nullptr);
}

// the FP32 approximate inverse the updates write and the one-column solves read:
// point it at X (when not NULL) and return the previous pointer
float *mixed_set_inverse(Ctx *c, float *X) {
    float *old = c->mx->X;
    if (X) c->mx->X = X;
    return old;
}

// device diagnostics of the mixed path, read (and reset) after a call
int mixed_read_stats(Ctx *c, double *ratio, double *nsres, int *iters, int *err, double *vmax, int *vn) {
    Mixed *m = c->mx;
    unsigned nb = 0;
    WW_CUDA_TRY(cudaMemcpyAsync(vmax, m->vmax, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    WW_CUDA_TRY(cudaMemcpyAsync(vn, m->vn, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    WW_CUDA_TRY(cudaMemcpyAsync(ratio, m->ratio, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    WW_CUDA_TRY(cudaMemcpyAsync(&nb, m->nsres, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    WW_CUDA_TRY(cudaMemcpyAsync(iters, m->iters, 3 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    WW_CUDA_TRY(cudaMemcpyAsync(err, m->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    WW_CUDA_TRY(cudaStreamSynchronize(c->stream));
    float nf;
    memcpy(&nf, &nb, sizeof(nf));
    *nsres = nf;
    WW_CUDA_TRY(cudaMemsetAsync(m->ratio, 0, sizeof(double), c->stream));
    WW_CUDA_TRY(cudaMemsetAsync(m->nsres, 0, sizeof(unsigned), c->stream));
    WW_CUDA_TRY(cudaMemsetAsync(m->iters, 0, 3 * sizeof(int), c->stream));
    WW_CUDA_TRY(cudaMemsetAsync(m->err, 0, sizeof(int), c->stream));
    WW_CUDA_TRY(cudaMemsetAsync(m->vcount, 0, sizeof(int), c->stream));
    WW_CUDA_TRY(cudaMemsetAsync(m->vmax, 0, sizeof(double), c->stream));
    WW_CUDA_TRY(cudaMemsetAsync(m->vn, 0, sizeof(int), c->stream));
    return WW_OK;
}

}  // namespace ww
