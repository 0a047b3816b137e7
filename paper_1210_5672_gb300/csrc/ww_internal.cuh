// ww_internal.cuh -- context layout, launch helpers and shared-memory FFT of
// the GB300 standing-wave Jacobian library.  Everything here is FP64 unless a
// name says otherwise.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/ww.h"

namespace ww {

// --------------------------------------------------------------------------
// error plumbing (thread-local message, status codes of ww.h)
// --------------------------------------------------------------------------
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
void fill_tables(int N, double *tw /* N */, double *cs /* 3N */);

// on failure the runtime's last-error state is cleared too, so that a
// non-sticky error does not resurface in the next call's launch checks
#define WW_CUDA_TRY(expr)                                                        \
    do {                                                                         \
        cudaError_t e_ = (expr);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            (void)cudaGetLastError();                                            \
            return ::ww::fail(WW_ERR_CUDA, std::string(#expr " : ") +            \
                                               cudaGetErrorString(e_));          \
        }                                                                        \
    } while (0)

#define WW_TRY(expr)                                                             \
    do {                                                                         \
        int s_ = (expr);                                                         \
        if (s_ != WW_OK) return s_;                                              \
    } while (0)

// device status bits (context status word)
enum : int {
    ST_GEOMETRY = 1,     // surface at/below the bottom or non-finite data
    ST_NONFINITE = 2,    // NaN/Inf appeared in a right-hand side
    ST_NO_CONV = 4,      // refinement did not reach its tolerance
};

constexpr int LU_NB = 64;   // block size of the blocked LU / triangular solves

// --------------------------------------------------------------------------
// the per-problem context: all device buffers are allocated in ww_create
// --------------------------------------------------------------------------
struct Mixed;   // mixed-precision workspace (ww_mixed.cu)
struct Seg;     // time-segment workspace: mesh, tableau, stage buffers (ww_segments.cu)

struct Ctx {
    // problem
    int N, logN, n, nc, NC;   // nc = n + 1 Jacobian columns, NC = nc + 1 incl. base
    double g, tau, h;
    bool deep;
    int steps, precision;
    double refine_tol;
    int max_refine;
    int nb;                   // LU block size actually used (min(LU_NB, N))
    cudaStream_t stream;

    // tables
    double2 *tw;              // tw[k] = exp(-2 pi i k / N), k < N/2
    float4 *twd;              // the same twiddles in double-float (WW_MIXED), or NULL
    double *cs;               // cs[m] = cos(2 pi m / N), cs[N + m] = sin(2 pi m / N)

    // base-surface geometry of the current stage (N each)
    double *eta, *eta_x, *eta_xx, *phi_s;   // eta, eta', eta'', phi'
    double *E, *Einv;                        // exp(eta), exp(-eta)
    double *ux, *vy, *w3;                    // phi_x, phi_y, (1+eta'^2)^{-3/2}
    double *curv;                            // d/dx (eta'/sqrt(1+eta'^2))
    double *Fbase;                           // filtered base RHS (2N)
    // The base-state results that the variational columns of a stage read
    // (ux, vy, w3, Fbase above) are double-buffered by stage parity, so the
    // base chain of stage s+1 can run while the columns of stage s still read
    // stage s's; `par` selects the copy the pointers above refer to.
    int par;
    double *ux_p[2], *vy_p[2], *w3_p[2], *Fbase_p[2];
    // double-float copies of ux, vy, w3 for the columns' double-float kernels
    // (WW_MIXED; NULL otherwise), also per parity
    float2 *uxd, *vyd, *w3d;
    float2 *uxd_p[2], *vyd_p[2], *w3d_p[2];
    // filter multipliers exp(-36 (|k|/(N/2))^36) / N per FFT slot: FP64 and double-float
    double *filt_d;
    float2 *filt_df;

    // dense operators
    double *A;                // N x N: 1/2 I + K, overwritten by its LU factors
    double *G;                // N x N
    double *Dinv;             // inverted diagonal LU blocks: [nblk][2][nb x nb] (L^-1, U^-1)

    // time-stepping state: [NC][2][N]  (column c: eta at c*2N, phi at c*2N + N)
    double *Y, *Ys, *Kacc;

    // multi-RHS workspaces (N x NC each, column-major)
    double *M;                // right-hand sides -> solutions mu
    double *Gam;              // gamma = mu'
    double *Gout;             // 1/2 H gamma + G gamma

    double *basis;            // N x 2 x n : column k = (eta part, phi part)
    int *status;              // device status word
    double *small;            // scratch doubles (reductions)

    bool dtn_ready;
    int trans;                // 1 while the adjoint sweep assembles A^T and G^T in place of A and G
    bool one_col;             // only one-column solves and products follow (base-only shots, the adjoint):
                              // the mixed form skips the digit splits of K and G that wide products read
    int verify_every;         // WW_MIXED: measure the true residual of every verify_every-th wide solve (0: off)
    int cur_stage;            // RK stage (0..3) whose work is being issued (phase timing)
    int ckpt_every;           // adjoint: checkpoint the base state every ckpt_every steps (0: keep every record)
    ww_schedule sch;          // tile shapes and stage schedule (ww_set_schedule / ww_autotune)
    int *emax_K, *emax_G;     // WW_MIXED: row exponent maxima of K = A - I/2 and G (the digit splits' scales)
    bool emax_ready;          // the last assembly issued also filled emax_K and emax_G
    size_t dev_bytes;         // device memory this context allocated
    ww_stats stats;
    Mixed *mx;
    Seg *seg;                 // set by ww_set_segment (NULL: the uniform RK4 shot only)
    void *owner;              // the API-side object holding this context (phase timing)
};

// point the per-stage buffers (base results here, mixed operands in ww_mixed.cu)
// at copy p
inline void select_parity(Ctx *c, int p) {
    c->par = p;
    if (c->ux_p[p]) {
        c->ux = c->ux_p[p];
        c->vy = c->vy_p[p];
        c->w3 = c->w3_p[p];
        c->Fbase = c->Fbase_p[p];
        c->uxd = c->uxd_p[p];
        c->vyd = c->vyd_p[p];
        c->w3d = c->w3d_p[p];
    }
}

// a double as a double-float pair (hi, lo): hi = x rounded to float, lo = the rest
__host__ __device__ inline float2 df_split(double x) {
    const float hi = (float)x;
    return make_float2(hi, (float)(x - (double)hi));
}

// --------------------------------------------------------------------------
// complex helpers
// --------------------------------------------------------------------------
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// --------------------------------------------------------------------------
// In-place complex FFT of length N = 2^logN held in shared memory, computed by
// the whole thread block (radix-2, decimation in time after a bit-reversal
// permutation).  Forward sign exp(-2 pi i jk/N); the inverse is unscaled.
// Callers synchronise before and after.  tw may point to global or shared
// memory (kernels stage the table into shared memory), so it is read with
// plain loads, never the global-only __ldg.
// --------------------------------------------------------------------------
__device__ __forceinline__ void block_fft(double2 *s, int N, int logN, const double2 *__restrict__ tw,
                                          bool inverse) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        int j = (int)(__brev((unsigned)i) >> (32 - logN));
        if (i < j) {
            double2 t = s[i];
            s[i] = s[j];
            s[j] = t;
        }
    }
    __syncthreads();
    const int halfN = N >> 1;
    for (int lh = 0; lh < logN; ++lh) {         // half = 2^lh
        const int half = 1 << lh;
        const int tshift = logN - 1 - lh;      // twiddle stride N / (2 half)
        for (int b = threadIdx.x; b < halfN; b += blockDim.x) {
            int k = b & (half - 1);
            int i0 = ((b >> lh) << (lh + 1)) + k;
            int i1 = i0 + half;
            double2 w = tw[k << tshift];
            if (inverse) w.y = -w.y;
            double2 v = cmul(s[i1], w);
            double2 u = s[i0];
            s[i0] = cadd(u, v);
            s[i1] = csub(u, v);
        }
        __syncthreads();
    }
}

// signed wavenumber of FFT slot j
__device__ __forceinline__ int wavenum(int j, int N) { return j <= (N >> 1) ? j : j - N; }

// 36th-order filter of Eq. (filter): exp(-36 (|k| / (N/2))^36)
__device__ __forceinline__ double filt36(int k, int N) {
    double r = fabs((double)k) / (double)(N >> 1);
    double r2 = r * r, r4 = r2 * r2, r8 = r4 * r4, r16 = r8 * r8, r32 = r16 * r16;
    return exp(-36.0 * r32 * r4);
}

// --------------------------------------------------------------------------
// kernels / host launchers implemented in the .cu files
// --------------------------------------------------------------------------
// spectral (ww_spectral.cu)
int prepare_spectral(Ctx *c);                        // shared-memory limits of the FFT kernels
// raise a kernel's dynamic shared-memory limit on the current device to at
// least `bytes` (never lowers it: contexts of different sizes share kernels)
int raise_smem(const void *kernel, size_t bytes);
int launch_base_geometry(Ctx *c, const double *eta, const double *phi, int with_phi);
int launch_gamma(Ctx *c, int col0, int ncols, bool fp64 = false);   // Gam = D M, Gout = 1/2 H D M (columns col0..);
                                                     // fp64: FP64 transforms also in the mixed form
int launch_psi(Ctx *c);                              // M[:,1..nc] = phidot - phi_y etadot
int launch_phi0(Ctx *c);                             // M[:,0] = phi of the base stage state
int launch_base_rhs(Ctx *c, int stage, const double *cvec);
int launch_col_rhs(Ctx *c, int stage, const double *cvec);
int launch_initial(Ctx *c, const double *cvec, int with_columns);
int launch_fill_filter(Ctx *c);                      // filter tables (once, at ww_create)
// the base state's transforms on an 8-CTA cluster (ww_cbase.cu), N >= 512
bool cbase_ok(const Ctx *c);
int launch_cbase_geometry(Ctx *c, const double *eta, const double *phi, int with_phi);
int launch_cbase_gamma(Ctx *c);                      // gamma, 1/2 H gamma of column 0 of M
int launch_cbase_rhs(Ctx *c, int stage, const double *cvec);
int launch_outputs(Ctx *c, double *r, double *J, double *f, int with_J);
int launch_copy_cols(Ctx *c, const double *src, int ncols, double *dst);

// phase timing (ww_api.cu): begin (b = 0) or end (b = 1) event of `phase` in
// the current stage; a no-op unless a timed shot is being issued
int phase_mark(Ctx *c, int phase, int b);
// ww_api.cu: the context behind a handle; the device status word read back
// (and the mixed form's statistics), as every entry point ends
Ctx *ctx_of(ww_ctx *h);
int read_status(Ctx *c);
// ww_segments.cu: free a context's segment workspace
void segment_destroy(Ctx *c);

// assembly (ww_assemble.cu); c->trans selects A^T, G^T
int launch_assemble(Ctx *c);

// the discrete adjoint (ww_adjoint.cu).  Trajectory record per RK stage:
// [eta | phi_x | phi_y | (1+eta'^2)^{-3/2} | F (2N)], ADJ_REC doubles per point
constexpr int ADJ_REC = 6;
struct AdjWs {
    double *rec;              // 4 K records of ADJ_REC * N (K = the steps of records held)
    int kheld;                // K: steps whose records are held (all steps, or the checkpoint interval)
    double *ckpt;             // checkpointed mode: the base state (2N) at steps 0, K, 2K, ...
    size_t bytes;             // device bytes of this workspace
    double *lam;              // 2N: the adjoint state
    double *kb;               // 4 x 2N: adjoints of the stage right-hand sides
    double *eta;              // N: the stage surface fetched for its geometry
    double *chi, *y, *etal, *psil;   // N each
    double *gT;               // 1: d f / d T
    int *step;                // 1: the RK step the record kernels address
    // second copies of A^T, G^T and the FP32 inverse: with them the DtN setup of
    // the next backward stage runs while the adjoint of this one still reads its own
    double *A2, *G2;
    float *X2;
};
int prepare_adjoint(int Nmax);                            // shared-memory limits of the sweep's FFT kernels
int launch_adj_record_eta(Ctx *c, AdjWs *a, int st);      // forward: the stage surface (before its RK update)
int launch_adj_record_fields(Ctx *c, AdjWs *a, int st);   // forward: phi_x, phi_y, w3, F; st == 3 advances the step
int launch_adj_init(Ctx *c, AdjWs *a);                    // lambda = (0, phi(T/4)/N), dT = 0
int launch_adj_set_step(Ctx *c, AdjWs *a, int v);         // record counter = v
int launch_adj_begin_step(Ctx *c, AdjWs *a, const double *cvec);   // step -= 1; filter lambda; kb = b dt/6 lambda
int launch_adj_fetch(Ctx *c, AdjWs *a, int off);          // surface of record 4 step + off into a->eta (none if < 0)
int launch_adj_local(Ctx *c, AdjWs *a, int st, const double *cvec);   // chi, local terms, dT += kb.F/T
int launch_adj_dtn(Ctx *c, AdjWs *a);                     // M[:,0] = D (1/2 H chi - G^T chi)
int launch_adj_update(Ctx *c, AdjWs *a, int st, const double *cvec);  // lambda, kb of the previous stage
int launch_adj_grad(Ctx *c, AdjWs *a, double *grad);      // grad = (dT, basis^T lambda)

// dense FP64 (ww_dense.cu)
int prepare_dense();                                 // shared-memory limit of the LU block kernel
int dgemm(cudaStream_t s, int m, int n, int k, double alpha, const double *A, int lda, const double *B,
          int ldb, double beta, double *C, int ldc);
// narrow products (n <= 8 columns) on the CUDA cores, deterministic (ww_gemv.cu):
// C = alpha A B + beta C (FP64); C = A B + beta C with the FP32 matrix A;
// R = Psi - A B (FP64).  A non-null skip that reads nonzero leaves the call out.
int gemv_narrow(cudaStream_t s, int m, int n, int k, double alpha, const double *A, int lda, const double *B, int ldb,
                double beta, double *C, int ldc, const int *skip = nullptr);
int gemv_narrow_f32(cudaStream_t s, int m, int n, int k, const float *A, int lda, const double *B, int ldb,
                    double beta, double *C, int ldc, const int *skip = nullptr);
int resid_narrow(cudaStream_t s, int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                 const double *Psi, int ldp, double *R, int ldr, const int *skip = nullptr);
int lu_factor_fp64(Ctx *c);
int lu_solve_fp64(Ctx *c, double *B, int ncols);     // B <- A^{-1} B using the factors in c->A

// mixed precision (ww_mixed.cu)
int mixed_create(Ctx *c);
int tc_init();   // resolves the tensor-map encoder (called before any capture)
void mixed_destroy(Ctx *c);
int mixed_setup(Ctx *c, int fresh, int update,       // after assembly: operands, inverse update
                bool adaptive = true);                // (adaptive: honour the schedule's cadence 2)
int mixed_read_stats(Ctx *c, double *ratio, double *nsres, int *iters /* [3]: max, sum, solves */, int *err,
                     double *vmax, int *vn);   // vmax, vn: measured residual of the sampled solves
int mixed_solve(Ctx *c, double *B, int ncols);       // B <- A^{-1} B (refined)
int mixed_apply_G(Ctx *c, int col0, int ncols, int part);   // Gout += G Gam (part 0 split, 1 product; FP64-accurate)
float *mixed_set_inverse(Ctx *c, float *X);          // the FP32 inverse the updates write (NULL: query)

}  // namespace ww
