/*
 * ww_oracle.c -- plain, slow, obviously-correct CPU FP64 oracle for the
 * Jacobian of the standing-water-wave shooting map (Wilkening & Yu,
 * "Overdetermined shooting methods for computing standing water waves with
 * spectral accuracy").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * Everything is IEEE double.  Complex arithmetic uses C99 <complex.h>, the
 * cotangent is the textbook cos/sin quotient (not the branch formula of
 * Sec. 2.2, which the GPU uses), the linear solve is LU with partial
 * pivoting, and the FFT is a textbook iterative radix-2 transform whose
 * twiddles are evaluated directly with cos/sin.  OpenMP (when compiled with
 * -fopenmp) only distributes independent rows / columns over threads; it
 * does not change any arithmetic.
 *
 * Paper references are by section / equation:
 *   Eq. (ww)            free-surface Euler equations               Sec. 2.1
 *   Eqs. (fred), (G)    DtN in three steps                          Sec. 2.1
 *   Eq. (uv:from:G)     surface velocities from (phi', G phi)       Sec. 2.1
 *   Eq. (K1K2)          regularised kernels, trapezoid collocation  Sec. 2.2
 *   Eq. (filter)        36th-order filter                           Sec. 2.2
 *   Eqs. (Phi), (plemelj:1), (plemelj:2)  image-kernel signs        App. A
 *   Eqs. (l5a), (l6a)   linearised (variational) equations          App. B
 *   Eqs. (f:phi), (Jik), (q:qdot)  objective and Jacobian           Sec. 3.1, 3.3
 *
 * Readings where the paper is garbled or silent:
 *  R1 image terms K2, G2 carry a MINUS sign (the integrals of App. A subtract
 *     the mirror-image double layer; the printed "+" in Eq. (K1K2) gives the
 *     symbol k coth(kh) on a flat surface instead of k tanh(kh)).
 *  R2 the T column of J is the variational column w = dq/dT of the discrete
 *     map, w' = DF(q) w + F(q)/T, w(0) = 0, integrated by the same RK4.
 *  R3 derivatives and the Hilbert transform zero the Nyquist mode; second
 *     derivatives are two first derivatives; P removes the k = 0 mode.
 *  R4 the filter multiplies every RHS evaluation and the state after each
 *     full RK4 step (not after stages), base and variational columns alike.
 *  R5 residual weight w = sqrt(1/N) (uniform grid, E = 1 in Eq. (f:phi)).
 *  R6 the linearisation is the continuum one of App. B with the shared
 *     discrete DtN operator (K and G are not differentiated).
 *  R18 the gradient of f (Sec. 3.2, App. C) is the DISCRETE adjoint: the
 *     transpose of the RK4 scheme above, so grad f = J^T r of the discrete
 *     map up to roundoff.  App. C derives the continuous adjoint from the
 *     self-adjointness of the continuous DtN map; its discretisation is only
 *     nearly symmetric, and the discrete adjoint uses its exact transpose
 *     A^{-T} D (1/2 H - G^T).
 */
/* ORC_PLANT (tests only, default 0) compiles a deliberately wrong variant so
 * that the pin tests can show they catch it: 1 = image kernels with the
 * printed "+" sign, 2 = zeta'(alpha) in K1 instead of zeta'(beta), 3 = gravity
 * term dropped from phi_t, 4 = u psi' term dropped from the variational RHS,
 * 5 = the adjoint takes the forward DtN for its transpose (the continuous
 * self-adjointness of App. C applied to the discrete operator), 6 = the DtN on
 * a mesh without the 1/|xi'| of Eq. (G), 7 = P on a mesh as the mean over
 * alpha instead of x, 8 = the adjoint on a mesh takes P for its transpose. */
#ifndef ORC_PLANT
#define ORC_PLANT 0
#endif

#include <stdlib.h>
#include <string.h>

/* The real type: IEEE double, or with ORC_WIDE the platform's long double
 * (x87 80-bit extended on x86-64, IEEE binary128 on aarch64), used only to
 * measure the double build's own rounding error on the same discrete map.
 * <tgmath.h> then selects each math function's long double form. */
#ifdef ORC_WIDE
#include <float.h>
#include <tgmath.h>
typedef long double real;
typedef long double complex cplx;
#define RL(x) x##L
#define CCOS(z) cos(z)
#define CSIN(z) sin(z)
#define CEXP(z) exp(z)
#define NEWTON_TOL (4 * LDBL_EPSILON)
#else
#include <complex.h>
#include <math.h>
typedef double real;
typedef double complex cplx;
#define RL(x) x
#define CCOS(z) ccos(z)
#define CSIN(z) csin(z)
#define CEXP(z) cexp(z)
#define NEWTON_TOL 4e-16
#endif

#ifdef _OPENMP
#include <omp.h>
#endif


/* ------------------------------------------------------------------ */
/* Problem description (oracle-side copy; the CUDA path has its own). */
/* ------------------------------------------------------------------ */
typedef struct {
    int N;          /* grid points alpha_j = 2 pi j / N (uniform, xi = alpha)   */
    int n;          /* number of mode unknowns c_1..c_n                         */
    real g;       /* gravity                                                  */
    real tau;     /* surface tension sigma/rho                                */
    real h;       /* mean depth; isinf(h) => infinite depth, no image kernels */
    int steps;      /* RK4 steps from 0 to T/4                                  */
    const real *basis; /* 2N x n column-major (eta rows, then phi rows) or NULL
                            for the default column k = (cos kx, 0)             */
} orc_problem;

static const real TWO_PI = RL(6.283185307179586476925286766559);

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ------------------------------------------------------------------ */
/* FFT: textbook iterative radix-2 Cooley-Tukey, N a power of two.     */
/* forward: X_k = sum_j x_j exp(-2 pi i jk/N); inverse divides by N.   */
/* ------------------------------------------------------------------ */
void orc_fft(int N, cplx *x, int inverse)
{
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < N; ++i) {
        int bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = x[i]; x[i] = x[j]; x[j] = t; }
    }
    real sgn = inverse ? 1.0 : -1.0;
    for (int len = 2; len <= N; len <<= 1) {
        int half = len >> 1;
        for (int s = 0; s < N; s += len) {
            for (int k = 0; k < half; ++k) {
                real ang = sgn * TWO_PI * (real)k / (real)len;
                cplx w = cos(ang) + I * sin(ang);
                cplx u = x[s + k];
                cplx v = x[s + k + half] * w;
                x[s + k] = u + v;
                x[s + k + half] = u - v;
            }
        }
    }
    if (inverse)
        for (int i = 0; i < N; ++i) x[i] /= (real)N;
}

/* signed wavenumber of FFT slot j */
static int wavenumber(int N, int j) { return j <= N / 2 ? j : j - N; }

/* Fourier multipliers (Sec. 2.1, 2.2; readings R3, R4) */
enum { MUL_DERIV = 0, MUL_HILBERT = 1, MUL_FILTER = 2, MUL_PROJECT = 3 };

static cplx multiplier(int kind, int N, int k)
{
    int nyq = (k == N / 2 || k == -N / 2);
    switch (kind) {
    case MUL_DERIV:   return nyq ? 0.0 : I * (real)k;               /* d/dx     */
    case MUL_HILBERT: return nyq ? 0.0 : -I * (real)((k > 0) - (k < 0)); /* H   */
    case MUL_FILTER: {                                                 /* Eq. (filter) */
        real r = fabs((real)k) / (real)(N / 2);
        return exp(-36.0 * pow(r, 36.0));
    }
    case MUL_PROJECT: return k == 0 ? 0.0 : 1.0;                       /* P = id - P0 */
    }
    return 0.0;
}

/* out = Re IFFT( m(k) * FFT(in) ); in and out may alias */
void orc_spectral(int N, int kind, const real *in, real *out)
{
    cplx *x = malloc(sizeof(cplx) * N);
    for (int j = 0; j < N; ++j) x[j] = in[j];
    orc_fft(N, x, 0);
    for (int j = 0; j < N; ++j) x[j] *= multiplier(kind, N, wavenumber(N, j));
    orc_fft(N, x, 1);
    for (int j = 0; j < N; ++j) out[j] = creal(x[j]);
    free(x);
}

/* A change of variables x = xi(alpha) of the grid alpha_j = 2 pi j / N
 * (Eq. (zeta), Eq. (xi)): x[j] = xi(alpha_j), e[j] = xi'(alpha_j) = E(alpha_j)
 * > 0, e1[j] = xi''(alpha_j).  Every function on the surface is stored as its
 * values at x = xi(alpha_j); a NULL mesh is the uniform grid xi = alpha. */
typedef struct {
    const real *x, *e, *e1;
} orc_mesh;

/* d/dx of a function stored on the mesh: (d/dalpha f) / xi'. */
static void mesh_dx(const orc_mesh *m, int N, const real *in, real *out)
{
    orc_spectral(N, MUL_DERIV, in, out);
    if (m)
        for (int i = 0; i < N; ++i) out[i] /= m->e[i];
}

/* P = id - P0 with P0 f = (1/2 pi) int f(x) dx (Sec. 2.1).  On the mesh the
 * integral is int f(xi(alpha)) xi'(alpha) dalpha, by the trapezoid rule in
 * alpha (reading R22); on the uniform grid it is the k = 0 mode. */
static void mesh_project(const orc_mesh *m, int N, const real *in, real *out)
{
    if (!m || ORC_PLANT == 7) { orc_spectral(N, MUL_PROJECT, in, out); return; }
    real s = 0.0;
    for (int i = 0; i < N; ++i) s += in[i] * m->e[i];
    s /= N;
    for (int i = 0; i < N; ++i) out[i] = in[i] - s;
}

/* ------------------------------------------------------------------ */
/* Kernel assembly, Eq. (K1K2) with reading R1; trapezoid rule (Sec. 2.2) */
/* ------------------------------------------------------------------ */
static cplx ccot(cplx z) { return CCOS(z) / CSIN(z); }

/* A = 1/2 I + K and G, both row-major N x N: row i = collocation point
 * alpha_i, column j = quadrature point beta = alpha_j; entries divided by N.
 * zeta = xi + i eta (Eq. (zeta)); eta_a, eta_aa are alpha-derivatives of the
 * stored eta.  The subtracted cot((alpha - beta)/2) stays in alpha. */
static void assemble_mesh(int N, real h, const orc_mesh *m, const real *eta, const real *eta_a,
                          const real *eta_aa, real *A, real *G)
{
    int deep = isinf(h);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int i = 0; i < N; ++i) {
        real ai = TWO_PI * i / N;
        cplx zi = (m ? m->x[i] : ai) + I * eta[i];
        cplx dzi = (m ? m->e[i] : 1.0) + I * eta_a[i];
        cplx ddzi = m ? m->e1[i] + I * eta_aa[i] : I * eta_aa[i];
        for (int j = 0; j < N; ++j) {
            real aj = TWO_PI * j / N;
            cplx zj = (m ? m->x[j] : aj) + I * eta[j];
            cplx dzj = (m ? m->e[j] : 1.0) + I * eta_a[j];
            real k1, g1, k2 = 0.0, g2 = 0.0;
            if (i == j) {                       /* diagonal limits, Sec. 2.2 */
                k1 = -cimag(ddzi / (2.0 * dzi));
                g1 = creal(ddzi / (2.0 * dzi));
            } else {
                cplx c = ccot((zi - zj) / 2.0);
                cplx c0 = ccot((cplx)((ai - aj) / 2.0));
                k1 = cimag((ORC_PLANT == 2 ? dzi : dzj) / 2.0 * c - 0.5 * c0);
                g1 = creal(dzi / 2.0 * c - 0.5 * c0);
            }
            if (!deep) {                        /* mirror image, reading R1 */
                cplx cb = ccot((zi - conj(zj)) / 2.0);
                real sgn = ORC_PLANT == 1 ? -1.0 : 1.0;
                k2 = -sgn * cimag(conj(dzj) / 2.0 * cb);
                g2 = -sgn * creal(dzi / 2.0 * cb);
            }
            A[(size_t)i * N + j] = (k1 + k2) / N + (i == j ? 0.5 : 0.0);
            G[(size_t)i * N + j] = (g1 + g2) / N;
        }
    }
}

void orc_assemble(int N, real h, const real *eta, const real *eta_x,
                  const real *eta_xx, real *A, real *G)
{
    assemble_mesh(N, h, NULL, eta, eta_x, eta_xx, A, G);
}

/* ------------------------------------------------------------------ */
/* LU with partial pivoting (row-major, in place) and solve.            */
/* ------------------------------------------------------------------ */
int orc_lu(int N, real *A, int *piv)
{
    for (int k = 0; k < N; ++k) {
        int p = k;
        real best = fabs(A[(size_t)k * N + k]);
        for (int i = k + 1; i < N; ++i)
            if (fabs(A[(size_t)i * N + k]) > best) { best = fabs(A[(size_t)i * N + k]); p = i; }
        piv[k] = p;
        if (best == 0.0) return -1;
        if (p != k)
            for (int j = 0; j < N; ++j) {
                real t = A[(size_t)k * N + j];
                A[(size_t)k * N + j] = A[(size_t)p * N + j];
                A[(size_t)p * N + j] = t;
            }
        real d = A[(size_t)k * N + k];
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (N - k > 256)
#endif
        for (int i = k + 1; i < N; ++i) {
            real l = A[(size_t)i * N + k] / d;
            A[(size_t)i * N + k] = l;
            real *ri = A + (size_t)i * N;
            const real *rk = A + (size_t)k * N;
            for (int j = k + 1; j < N; ++j) ri[j] -= l * rk[j];
        }
    }
    return 0;
}

/* x = A^{-1} b using the factors of orc_lu; b and x may alias */
void orc_lu_solve(int N, const real *LU, const int *piv, const real *b, real *x)
{
    if (x != b) memcpy(x, b, sizeof(real) * N);
    for (int k = 0; k < N; ++k)
        if (piv[k] != k) { real t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
    for (int i = 0; i < N; ++i) {            /* unit lower */
        real s = x[i];
        for (int j = 0; j < i; ++j) s -= LU[(size_t)i * N + j] * x[j];
        x[i] = s;
    }
    for (int i = N - 1; i >= 0; --i) {       /* upper */
        real s = x[i];
        for (int j = i + 1; j < N; ++j) s -= LU[(size_t)i * N + j] * x[j];
        x[i] = s / LU[(size_t)i * N + i];
    }
}

/* x = A^{-T} b using the factors of orc_lu: P A = L U, so A^T = U^T L^T P
 * (solve with U^T, then the unit L^T, then undo the interchanges in reverse
 * order); b and x may alias */
void orc_lu_solve_T(int N, const real *LU, const int *piv, const real *b, real *x)
{
    if (x != b) memcpy(x, b, sizeof(real) * N);
    for (int i = 0; i < N; ++i) {            /* U^T: lower, diagonal U_ii */
        real s = x[i];
        for (int j = 0; j < i; ++j) s -= LU[(size_t)j * N + i] * x[j];
        x[i] = s / LU[(size_t)i * N + i];
    }
    for (int i = N - 1; i >= 0; --i) {       /* L^T: unit upper */
        real s = x[i];
        for (int j = i + 1; j < N; ++j) s -= LU[(size_t)j * N + i] * x[j];
        x[i] = s;
    }
    for (int k = N - 1; k >= 0; --k)
        if (piv[k] != k) { real t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
}

/* ------------------------------------------------------------------ */
/* The per-stage DtN of the base surface (Sec. 2.1, Eqs. (fred), (G))  */
/* ------------------------------------------------------------------ */
typedef struct {
    int N;
    const orc_mesh *m;              /* NULL: uniform grid */
    real *eta, *eta_x, *eta_xx;   /* eta and its alpha-derivatives */
    real *LU, *G;
    int *piv;
} dtn_state;

static void dtn_prepare_mesh(dtn_state *s, const orc_mesh *m, int N, real h, const real *eta)
{
    s->N = N;
    s->m = m;
    s->eta = malloc(sizeof(real) * N);
    s->eta_x = malloc(sizeof(real) * N);
    s->eta_xx = malloc(sizeof(real) * N);
    s->LU = malloc(sizeof(real) * (size_t)N * N);
    s->G = malloc(sizeof(real) * (size_t)N * N);
    s->piv = malloc(sizeof(int) * N);
    memcpy(s->eta, eta, sizeof(real) * N);
    orc_spectral(N, MUL_DERIV, eta, s->eta_x);
    orc_spectral(N, MUL_DERIV, s->eta_x, s->eta_xx);
    assemble_mesh(N, h, m, s->eta, s->eta_x, s->eta_xx, s->LU, s->G);
    orc_lu(N, s->LU, s->piv);
}

static void dtn_prepare(dtn_state *s, int N, real h, const real *eta)
{
    dtn_prepare_mesh(s, NULL, N, h, eta);
}

static void dtn_release(dtn_state *s)
{
    free(s->eta); free(s->eta_x); free(s->eta_xx);
    free(s->LU); free(s->G); free(s->piv);
}

/* G phi on the surface (Eq. (G)): mu = A^{-1} phi; gamma = mu' (in alpha);
 * (1/2 H gamma + G gamma) / |xi'| (xi' = 1 on the uniform grid). */
static void dtn_apply_one(const dtn_state *s, const real *phi, real *out)
{
    int N = s->N;
    real *mu = malloc(sizeof(real) * N);
    real *gam = malloc(sizeof(real) * N);
    real *hg = malloc(sizeof(real) * N);
    orc_lu_solve(N, s->LU, s->piv, phi, mu);
    orc_spectral(N, MUL_DERIV, mu, gam);
    orc_spectral(N, MUL_HILBERT, gam, hg);
    for (int i = 0; i < N; ++i) {
        real acc = 0.0;
        for (int j = 0; j < N; ++j) acc += s->G[(size_t)i * N + j] * gam[j];
        out[i] = 0.5 * hg[i] + acc;
        if (s->m && ORC_PLANT != 6) out[i] /= s->m->e[i];
    }
    free(mu); free(gam); free(hg);
}

/* The transpose of the operator of dtn_apply_one (reading R18).  Forward:
 * G phi = diag(1/xi') (1/2 H + G) D A^{-1} phi.  The Fourier multipliers ik
 * and -i sgn k (Nyquist zeroed) are antisymmetric, D^T = -D and H^T = -H, so
 * G^T x = A^{-T} D (1/2 H - G^T) diag(1/xi') x. */
static void dtn_apply_T(const dtn_state *s, const real *x, real *out)
{
    int N = s->N;
    if (ORC_PLANT == 5) { dtn_apply_one(s, x, out); return; }
    real *hx = malloc(sizeof(real) * N);
    real *t = malloc(sizeof(real) * N);
    real *xs = malloc(sizeof(real) * N);          /* diag(1/xi') x on a mesh */
    for (int i = 0; i < N; ++i) xs[i] = s->m ? x[i] / s->m->e[i] : x[i];
    orc_spectral(N, MUL_HILBERT, xs, hx);
    for (int i = 0; i < N; ++i) {
        real acc = 0.0;
        for (int j = 0; j < N; ++j) acc += s->G[(size_t)j * N + i] * xs[j];
        t[i] = 0.5 * hx[i] - acc;
    }
    orc_spectral(N, MUL_DERIV, t, t);
    orc_lu_solve_T(N, s->LU, s->piv, t, out);
    free(hx); free(t); free(xs);
}

/* Public: the transposed DtN of x on surface eta (tests). */
void orc_dtn_T(int N, real h, const real *eta, const real *x, real *out)
{
    dtn_state s;
    dtn_prepare(&s, N, h, eta);
    dtn_apply_T(&s, x, out);
    dtn_release(&s);
}

/* Public: DtN of phi (nrhs columns, each length N, contiguous) on surface eta. */
void orc_dtn(int N, real h, const real *eta, const real *phi, int nrhs, real *out)
{
    dtn_state s;
    dtn_prepare(&s, N, h, eta);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic)
#endif
    for (int c = 0; c < nrhs; ++c)
        dtn_apply_one(&s, phi + (size_t)c * N, out + (size_t)c * N);
    dtn_release(&s);
}

/* Public: the assembled matrices (for tests). */
void orc_dtn_matrices(int N, real h, const real *eta, real *A, real *G)
{
    real *ex = malloc(sizeof(real) * N), *exx = malloc(sizeof(real) * N);
    orc_spectral(N, MUL_DERIV, eta, ex);
    orc_spectral(N, MUL_DERIV, ex, exx);
    orc_assemble(N, h, eta, ex, exx, A, G);
    free(ex); free(exx);
}

/* ------------------------------------------------------------------ */
/* Right-hand sides: Eq. (ww) for the base state, Eqs. (l5a), (l6a) for  */
/* every variational column; all outputs filtered (Eq. (filter)).        */
/* ------------------------------------------------------------------ */

/* state layout used by the oracle's time stepper: ncol+1 columns, each
 * column = [eta (N) | phi (N)]; column 0 is the base state q, columns
 * 1..ncol are the variational columns. */

/* Evaluate the filtered RHS of the base state and of ncol variational
 * columns.  t_col: index (1-based among the variational columns) of the
 * column that additionally receives F(q)/T (reading R2), or 0 for none. */
static void rhs_impl(const orc_problem *p, const orc_mesh *m, int N, real T, const real *y, int ncol,
                     int t_col, real *out);
void orc_rhs(const orc_problem *p, real T, const real *y, int ncol, int t_col, real *out)
{
    rhs_impl(p, NULL, p->N, T, y, ncol, t_col, out);
}

/* The same on N points of a mesh (NULL: uniform): every x-derivative is
 * d/dalpha over xi', P subtracts the x-mean, the filter acts on the alpha
 * grid's Fourier modes (Sec. 2.2). */
static void rhs_impl(const orc_problem *p, const orc_mesh *m, int N, real T, const real *y, int ncol,
                     int t_col, real *out)
{
    const real *eta = y, *phi = y + N;
    dtn_state s;
    dtn_prepare_mesh(&s, m, N, p->h, eta);

    real *phi_p = malloc(sizeof(real) * N);
    real *Gphi = malloc(sizeof(real) * N);
    real *ux = malloc(sizeof(real) * N);  /* phi_x on the surface */
    real *vy = malloc(sizeof(real) * N);  /* phi_y on the surface */
    real *w3 = malloc(sizeof(real) * N);  /* (1 + eta'^2)^{-3/2} */
    real *tmp = malloc(sizeof(real) * N);
    real *etx = malloc(sizeof(real) * N); /* eta' = d eta / dx */

    mesh_dx(m, N, phi, phi_p);
    for (int i = 0; i < N; ++i) etx[i] = m ? s.eta_x[i] / m->e[i] : s.eta_x[i];
    dtn_apply_one(&s, phi, Gphi);
    for (int i = 0; i < N; ++i) {              /* Eq. (uv:from:G) */
        real ex = etx[i], d = 1.0 + ex * ex;
        ux[i] = (phi_p[i] - ex * Gphi[i]) / d;
        vy[i] = (ex * phi_p[i] + Gphi[i]) / d;
        w3[i] = 1.0 / (d * sqrt(d));
    }

    /* base: eta_t = G phi ; phi_t = P[ v eta_t - u^2/2 - v^2/2 - g eta + tau d/dx(eta'/sqrt(1+eta'^2)) ] */
    real *F = out;                 /* column 0 of out */
    for (int i = 0; i < N; ++i) F[i] = Gphi[i];
    for (int i = 0; i < N; ++i) {
        real ex = etx[i];
        tmp[i] = ex / sqrt(1.0 + ex * ex);
    }
    mesh_dx(m, N, tmp, tmp);
    for (int i = 0; i < N; ++i)
        F[N + i] = vy[i] * Gphi[i] - 0.5 * ux[i] * ux[i] - 0.5 * vy[i] * vy[i]
                   - (ORC_PLANT == 3 ? 0.0 : p->g) * eta[i] + p->tau * tmp[i];
    mesh_project(m, N, F + N, F + N);
    orc_spectral(N, MUL_FILTER, F, F);
    orc_spectral(N, MUL_FILTER, F + N, F + N);

#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic)
#endif
    for (int c = 1; c <= ncol; ++c) {
        const real *ed = y + (size_t)c * 2 * N, *pd = ed + N;
        real *oe = out + (size_t)c * 2 * N, *op = oe + N;
        real *psi = malloc(sizeof(real) * N), *Gpsi = malloc(sizeof(real) * N);
        real *dpsi = malloc(sizeof(real) * N), *a = malloc(sizeof(real) * N);
        real *b = malloc(sizeof(real) * N), *e1 = malloc(sizeof(real) * N);
        /* psi = phidot - phi_y etadot : the perturbation potential on the surface */
        for (int i = 0; i < N; ++i) psi[i] = pd[i] - vy[i] * ed[i];
        dtn_apply_one(&s, psi, Gpsi);
        mesh_dx(m, N, psi, dpsi);
        /* Eq. (l5a): etadot_t = G psi - (etadot u)' */
        for (int i = 0; i < N; ++i) a[i] = ed[i] * ux[i];
        mesh_dx(m, N, a, a);
        for (int i = 0; i < N; ++i) oe[i] = Gpsi[i] - a[i];
        /* Eq. (l6a): phidot_t = P[ -(etadot u v)' - u psi' + v G psi - g etadot
         *                        + tau d/dx( etadot' (1+eta'^2)^{-3/2} ) ] */
        for (int i = 0; i < N; ++i) b[i] = ed[i] * ux[i] * vy[i];
        mesh_dx(m, N, b, b);
        mesh_dx(m, N, ed, e1);
        for (int i = 0; i < N; ++i) e1[i] *= w3[i];
        mesh_dx(m, N, e1, e1);
        for (int i = 0; i < N; ++i)
            op[i] = -b[i] - (ORC_PLANT == 4 ? 0.0 : ux[i]) * dpsi[i] + vy[i] * Gpsi[i] - p->g * ed[i]
                    + p->tau * e1[i];
        mesh_project(m, N, op, op);
        orc_spectral(N, MUL_FILTER, oe, oe);
        orc_spectral(N, MUL_FILTER, op, op);
        if (c == t_col)
            for (int i = 0; i < 2 * N; ++i) oe[i] += F[i] / T;
        free(psi); free(Gpsi); free(dpsi); free(a); free(b); free(e1);
    }
    free(phi_p); free(Gphi); free(ux); free(vy); free(w3); free(tmp); free(etx);
    dtn_release(&s);
}

/* ------------------------------------------------------------------ */
/* Initial data (Sec. 3.1, reading of the basis) and RK4 (classic)       */
/* ------------------------------------------------------------------ */
static real basis_entry(const orc_problem *p, int row, int k /* 1..n */)
{
    int N = p->N;
    if (p->basis) return p->basis[(size_t)(k - 1) * 2 * N + row];
    if (row >= N) return 0.0;
    return cos((real)k * TWO_PI * row / N);
}

/* q0 = (mean + sum c_k B_eta[:,k], sum c_k B_phi[:,k]) */
void orc_initial(const orc_problem *p, const real *c, real *q0)
{
    int N = p->N;
    real mean = isinf(p->h) ? 0.0 : p->h;
    for (int r = 0; r < 2 * N; ++r) {
        real s = r < N ? mean : 0.0;
        for (int k = 1; k <= p->n; ++k) s += c[k] * basis_entry(p, r, k);
        q0[r] = s;
    }
}

/* Integrate base + ncol variational columns from 0 to T/4 with p->steps RK4
 * steps; y holds the initial data on entry and the final data on exit.  rec
 * (NULL or (steps + 1) x len) receives y at every step boundary. */
static void integrate_rec(const orc_problem *p, real T, real *y, int ncol, int t_col, real *rec);
static void integrate(const orc_problem *p, real T, real *y, int ncol, int t_col)
{
    integrate_rec(p, T, y, ncol, t_col, NULL);
}
static void integrate_rec(const orc_problem *p, real T, real *y, int ncol, int t_col, real *rec)
{
    int N = p->N;
    size_t len = (size_t)(ncol + 1) * 2 * N;
    real dt = T / 4.0 / p->steps;
    real *k = malloc(sizeof(real) * len), *acc = malloc(sizeof(real) * len);
    real *ys = malloc(sizeof(real) * len);
    static const real a[4] = {0.0, 0.5, 0.5, 1.0};
    static const real b[4] = {1.0, 2.0, 2.0, 1.0};
    if (rec) memcpy(rec, y, sizeof(real) * len);
    for (int n = 0; n < p->steps; ++n) {
        for (size_t i = 0; i < len; ++i) acc[i] = 0.0;
        for (int st = 0; st < 4; ++st) {
            if (st == 0) memcpy(ys, y, sizeof(real) * len);
            else for (size_t i = 0; i < len; ++i) ys[i] = y[i] + a[st] * dt * k[i];
            orc_rhs(p, T, ys, ncol, t_col, k);
            for (size_t i = 0; i < len; ++i) acc[i] += b[st] * k[i];
        }
        for (size_t i = 0; i < len; ++i) y[i] += dt / 6.0 * acc[i];
        for (int c = 0; c <= ncol; ++c) {             /* filter the solution (R4) */
            orc_spectral(N, MUL_FILTER, y + (size_t)c * 2 * N, y + (size_t)c * 2 * N);
            orc_spectral(N, MUL_FILTER, y + (size_t)c * 2 * N + N, y + (size_t)c * 2 * N + N);
        }
        if (rec) memcpy(rec + (size_t)(n + 1) * len, y, sizeof(real) * len);
    }
    free(k); free(acc); free(ys);
}

/* Base state and ncol variational columns (initial data cols, each 2N; column
 * t_col forced as in orc_rhs) at every step boundary: rec is
 * (steps + 1) x (ncol + 1) x 2N. */
void orc_trajectory_columns(const orc_problem *p, real T, const real *q0, const real *cols, int ncol,
                            int t_col, real *rec)
{
    int N = p->N;
    size_t len = (size_t)(ncol + 1) * 2 * N;
    real *y = malloc(sizeof(real) * len);
    memcpy(y, q0, sizeof(real) * 2 * N);
    memcpy(y + 2 * N, cols, sizeof(real) * (size_t)ncol * 2 * N);
    integrate_rec(p, T, y, ncol, t_col, rec);
    free(y);
}

/* Evolve the base state only (no columns): q_end = q(T/4). */
void orc_evolve(const orc_problem *p, real T, const real *q0, real *q_end)
{
    memcpy(q_end, q0, sizeof(real) * 2 * p->N);
    integrate(p, T, q_end, 0, 0);
}

/* Evolve base + ncol given variational columns (each 2N, contiguous) with
 * an optional T-forcing column (t_col as in orc_rhs). */
void orc_evolve_columns(const orc_problem *p, real T, const real *q0, const real *cols,
                        int ncol, int t_col, real *y_end /* (ncol+1)*2N */)
{
    int N = p->N;
    memcpy(y_end, q0, sizeof(real) * 2 * N);
    memcpy(y_end + 2 * N, cols, sizeof(real) * (size_t)ncol * 2 * N);
    integrate(p, T, y_end, ncol, t_col);
}

/* Objective, Eq. (f:phi) with reading R5: r_i = phi(x_i, T/4)/sqrt(N). */
void orc_shoot(const orc_problem *p, const real *c, real *r, real *f)
{
    int N = p->N;
    real *y = malloc(sizeof(real) * 2 * N);
    orc_initial(p, c, y);
    integrate(p, c[0], y, 0, 0);
    real w = 1.0 / sqrt((real)N), s = 0.0;
    for (int i = 0; i < N; ++i) { r[i] = w * y[N + i]; s += r[i] * r[i]; }
    *f = 0.5 * s;
    free(y);
}

/* Jacobian, Eqs. (Jik), (q:qdot) with reading R2: J is N x (n+1) column-major,
 * column 0 = d r / d T, column k = d r / d c_k. */
void orc_shoot_jacobian(const orc_problem *p, const real *c, real *r, real *J, real *f)
{
    int N = p->N, n = p->n, ncol = n + 1;
    size_t len = (size_t)(ncol + 1) * 2 * N;
    real *y = calloc(len, sizeof(real));
    orc_initial(p, c, y);
    /* column 1 (J column 0) = T column, zero initial data; columns 2.. = basis */
    for (int k = 1; k <= n; ++k)
        for (int rr = 0; rr < 2 * N; ++rr)
            y[(size_t)(k + 1) * 2 * N + rr] = basis_entry(p, rr, k);
    integrate(p, c[0], y, ncol, 1);
    real w = 1.0 / sqrt((real)N), s = 0.0;
    for (int i = 0; i < N; ++i) { r[i] = w * y[N + i]; s += r[i] * r[i]; }
    *f = 0.5 * s;
    for (int k = 0; k <= n; ++k)
        for (int i = 0; i < N; ++i)
            J[(size_t)k * N + i] = w * y[(size_t)(k + 1) * 2 * N + N + i];
    free(y);
}

/* ------------------------------------------------------------------ */
/* Gradient by the discrete adjoint (Sec. 3.2 Eqs. (adj), (nabla:f);   */
/* App. C Eq. (adj2); reading R18)                                       */
/* ------------------------------------------------------------------ */

/* Transpose of the filtered variational RHS of orc_rhs at the base state q,
 * applied to kb = (adjoint of etadot_t, adjoint of phidot_t) (each N); out =
 * (adjoint of etadot, adjoint of phidot).  *Fdot = kb . F(q) with F the
 * filtered base RHS (the T column's forcing is F/T).  Term by term this is
 * Eq. (adj2): with et = Filt(kb_eta), pt = P Filt(kb_phi) and the auxiliary
 * chi = et + phi_y pt,
 *   adjoint of phidot = G^T chi + (phi_x pt)'
 *   adjoint of etadot = -phi_y (G^T chi + (phi_x pt)') + phi_x et'
 *                       + phi_x phi_y pt' - g pt + tau (pt' (1+eta'^2)^{-3/2})'
 * (the two phi_y terms combine to App. C's -phi_y phi_x' P phit). */
/* -D_x^T v with D_x = diag(1/xi') D_alpha: D_alpha (v / xi'), i.e. D v on the
 * uniform grid (D^T = -D). */
static void mesh_dxT_neg(const orc_mesh *m, int N, const real *in, real *out)
{
    if (!m) { orc_spectral(N, MUL_DERIV, in, out); return; }
    for (int i = 0; i < N; ++i) out[i] = in[i] / m->e[i];
    orc_spectral(N, MUL_DERIV, out, out);
}

/* P^T of mesh_project: v - xi' (sum v) / N on a mesh; P itself when uniform. */
static void mesh_project_T(const orc_mesh *m, int N, const real *in, real *out)
{
    if (!m) { orc_spectral(N, MUL_PROJECT, in, out); return; }
    if (ORC_PLANT == 8) { mesh_project(m, N, in, out); return; }
    real s = 0.0;
    for (int i = 0; i < N; ++i) s += in[i];
    s /= N;
    for (int i = 0; i < N; ++i) out[i] = in[i] - m->e[i] * s;
}

static void rhs_T_mesh(const orc_problem *p, const orc_mesh *m, int N, const real *q, const real *kb, real *out,
                       real *Fdot);
static void rhs_T(const orc_problem *p, const real *q, const real *kb, real *out, real *Fdot)
{
    rhs_T_mesh(p, NULL, p->N, q, kb, out, Fdot);
}

/* The same on N points of a mesh (NULL: uniform): every D of the uniform form
 * becomes -D_x^T = D_alpha diag(1/xi'), P becomes P^T, and the DtN transpose
 * carries diag(1/xi'). */
static void rhs_T_mesh(const orc_problem *p, const orc_mesh *m, int N, const real *q, const real *kb, real *out,
                       real *Fdot)
{
    const real *eta = q, *phi = q + N;
    real *F = malloc(sizeof(real) * 2 * N);
    rhs_impl(p, m, N, 1.0, q, 0, 0, F);          /* base RHS (no T forcing in column 0) */
    real fd = 0.0;
    for (int i = 0; i < 2 * N; ++i) fd += kb[i] * F[i];
    *Fdot = fd;

    dtn_state s;
    dtn_prepare_mesh(&s, m, N, p->h, eta);
    real *phi_p = malloc(sizeof(real) * N), *Gphi = malloc(sizeof(real) * N);
    real *ux = malloc(sizeof(real) * N), *vy = malloc(sizeof(real) * N);
    real *w3 = malloc(sizeof(real) * N);
    mesh_dx(m, N, phi, phi_p);
    dtn_apply_one(&s, phi, Gphi);
    for (int i = 0; i < N; ++i) {              /* Eq. (uv:from:G), as in orc_rhs */
        real ex = m ? s.eta_x[i] / m->e[i] : s.eta_x[i], d = 1.0 + ex * ex;
        ux[i] = (phi_p[i] - ex * Gphi[i]) / d;
        vy[i] = (ex * phi_p[i] + Gphi[i]) / d;
        w3[i] = 1.0 / (d * sqrt(d));
    }
    real *et = malloc(sizeof(real) * N), *pt = malloc(sizeof(real) * N);
    real *chi = malloc(sizeof(real) * N), *Gchi = malloc(sizeof(real) * N);
    real *d_et = malloc(sizeof(real) * N), *d_pt = malloc(sizeof(real) * N);
    real *t1 = malloc(sizeof(real) * N), *t2 = malloc(sizeof(real) * N);
    orc_spectral(N, MUL_FILTER, kb, et);
    orc_spectral(N, MUL_FILTER, kb + N, pt);
    mesh_project_T(m, N, pt, pt);
    for (int i = 0; i < N; ++i) chi[i] = et[i] + vy[i] * pt[i];
    dtn_apply_T(&s, chi, Gchi);
    mesh_dxT_neg(m, N, et, d_et);
    mesh_dxT_neg(m, N, pt, d_pt);
    for (int i = 0; i < N; ++i) t1[i] = ux[i] * pt[i];
    mesh_dxT_neg(m, N, t1, t1);                /* (phi_x pt)' */
    for (int i = 0; i < N; ++i) t2[i] = w3[i] * d_pt[i];
    mesh_dxT_neg(m, N, t2, t2);                /* (pt' (1+eta'^2)^{-3/2})' */
    for (int i = 0; i < N; ++i) {
        real pb = Gchi[i] + t1[i];
        out[N + i] = pb;
        out[i] = -vy[i] * pb + ux[i] * d_et[i] + ux[i] * vy[i] * d_pt[i] - p->g * pt[i] + p->tau * t2[i];
    }
    free(F); free(phi_p); free(Gphi); free(ux); free(vy); free(w3);
    free(et); free(pt); free(chi); free(Gchi); free(d_et); free(d_pt); free(t1); free(t2);
    dtn_release(&s);
}

/* f and grad f (n+1 entries, grad[0] = d f / d T) by the discrete adjoint of
 * the RK4 scheme of integrate().  The base trajectory runs forward once with
 * every stage state kept; the adjoint starts from lambda = (0, phi(T/4)/N)
 * (the gradient of f = r.r/2, r = phi/sqrt(N), with respect to the final
 * state) and runs the transposed steps backward: per step the filter, then
 * the stages in reverse order, stage st contributing its transposed RHS to
 * lambda and, scaled by a_st dt, to the adjoint of the previous stage's RHS.
 * grad_k = basis_k . lambda(0); grad_0 = sum over stages of kbar . F / T. */
static void adjoint_sweep(const orc_problem *p, const real *c, real *f, real *grad, real *lam_rec);

void orc_objective_and_grad(const orc_problem *p, const real *c, real *f, real *grad)
{
    adjoint_sweep(p, c, f, grad, NULL);
}

/* The adjoint state at every step boundary: lam_rec[n] (n = 0..steps, 2N each)
 * is the gradient of f with respect to the state at the start of step n
 * (lam_rec[steps] = (0, phi(T/4)/N)).  The discrete counterpart of Sec. 3.2's
 * identity <q~(T/4 - t), qdot(t)> = const: lam_rec[n] . w_n is the same for
 * every n when w is an unforced variational column. */
void orc_adjoint_trajectory(const orc_problem *p, const real *c, real *lam_rec)
{
    real f, *grad = malloc(sizeof(real) * (p->n + 1));
    adjoint_sweep(p, c, &f, grad, lam_rec);
    free(grad);
}

static void adjoint_sweep(const orc_problem *p, const real *c, real *f, real *grad, real *lam_rec)
{
    int N = p->N, S = 4 * p->steps;
    size_t n2 = (size_t)2 * N;
    real T = c[0], dt = T / 4.0 / p->steps;
    static const real a[4] = {0.0, 0.5, 0.5, 1.0};
    static const real b[4] = {1.0, 2.0, 2.0, 1.0};
    real *traj = malloc(sizeof(real) * n2 * (size_t)S);
    real *y = malloc(sizeof(real) * n2), *k = malloc(sizeof(real) * n2);
    real *acc = malloc(sizeof(real) * n2);
    orc_initial(p, c, y);
    for (int n = 0; n < p->steps; ++n) {         /* forward: as integrate() with no columns */
        for (size_t i = 0; i < n2; ++i) acc[i] = 0.0;
        for (int st = 0; st < 4; ++st) {
            real *ys = traj + (size_t)(4 * n + st) * n2;
            if (st == 0) memcpy(ys, y, sizeof(real) * n2);
            else for (size_t i = 0; i < n2; ++i) ys[i] = y[i] + a[st] * dt * k[i];
            orc_rhs(p, T, ys, 0, 0, k);
            for (size_t i = 0; i < n2; ++i) acc[i] += b[st] * k[i];
        }
        for (size_t i = 0; i < n2; ++i) y[i] += dt / 6.0 * acc[i];
        orc_spectral(N, MUL_FILTER, y, y);
        orc_spectral(N, MUL_FILTER, y + N, y + N);
    }
    real s = 0.0;
    for (int i = 0; i < N; ++i) s += y[N + i] * y[N + i] / N;
    *f = 0.5 * s;

    real *lam = malloc(sizeof(real) * n2), *kb = malloc(sizeof(real) * n2 * 4);
    real *wb = malloc(sizeof(real) * n2);
    for (int i = 0; i < N; ++i) { lam[i] = 0.0; lam[N + i] = y[N + i] / N; }
    if (lam_rec) memcpy(lam_rec + (size_t)p->steps * n2, lam, sizeof(real) * n2);
    real gT = 0.0;
    for (int n = p->steps - 1; n >= 0; --n) {
        orc_spectral(N, MUL_FILTER, lam, lam);   /* the end-of-step filter, transposed */
        orc_spectral(N, MUL_FILTER, lam + N, lam + N);
        for (int st = 0; st < 4; ++st)
            for (size_t i = 0; i < n2; ++i) kb[st * n2 + i] = b[st] * dt / 6.0 * lam[i];
        for (int st = 3; st >= 0; --st) {
            real Fd;
            rhs_T(p, traj + (size_t)(4 * n + st) * n2, kb + st * n2, wb, &Fd);
            gT += Fd / T;
            for (size_t i = 0; i < n2; ++i) lam[i] += wb[i];
            if (st > 0)
                for (size_t i = 0; i < n2; ++i) kb[(st - 1) * n2 + i] += a[st] * dt * wb[i];
        }
        if (lam_rec) memcpy(lam_rec + (size_t)n * n2, lam, sizeof(real) * n2);
    }
    grad[0] = gT;
    for (int kk = 1; kk <= p->n; ++kk) {
        real g = 0.0;
        for (size_t r = 0; r < n2; ++r) g += basis_entry(p, (int)r, kk) * lam[r];
        grad[kk] = g;
    }
    free(traj); free(y); free(k); free(acc); free(lam); free(kb); free(wb);
}

/* Energy (Sec. 4, energy monitor): E = 1/2 int (phi G phi + g (eta - hbar)^2) dx
 * + tau int (sqrt(1 + eta'^2) - 1) dx, trapezoid rule. */
real orc_energy(const orc_problem *p, const real *q)
{
    int N = p->N;
    const real *eta = q, *phi = q + N;
    real *Gphi = malloc(sizeof(real) * N), *ex = malloc(sizeof(real) * N);
    orc_dtn(N, p->h, eta, phi, 1, Gphi);
    orc_spectral(N, MUL_DERIV, eta, ex);
    real mean = isinf(p->h) ? 0.0 : p->h, e = 0.0;
    for (int i = 0; i < N; ++i) {
        real d = eta[i] - mean;
        e += 0.5 * (phi[i] * Gphi[i] + p->g * d * d) + p->tau * (sqrt(1.0 + ex[i] * ex[i]) - 1.0);
    }
    free(Gphi); free(ex);
    return e * TWO_PI / N;
}

/* ------------------------------------------------------------------ */
/* Time segments, adaptive meshes and a general explicit Runge-Kutta    */
/* scheme (Sec. 2.2, Eq. (xi), Eq. (rho:def); DOP853 of Hairer et al.)  */
/* ------------------------------------------------------------------ */

/* One time segment: M grid points, a fixed number of uniform steps over the
 * fraction theta of the simulated time T/4, and the mesh of Eq. (xi) with
 * parameter rho (0 < rho <= 1; 1 = uniform) refined near x = pi (centre = 1,
 * the sin^4 form) or near x = 0 (centre = 0, the cos^4 form). */
typedef struct {
    int M;
    int steps;
    real theta;
    real rho;
    int centre;
} orc_segment;

/* An explicit Runge-Kutta tableau: s stages, a (s x s, row-major, strictly
 * lower triangular) and the weights b (s).  The equations are autonomous,
 * so the nodes are not needed. */
typedef struct {
    int s;
    const real *a, *b;
} orc_tableau;

/* Eq. (xi): E = 1 - P[A sin^4(alpha/2)] (or cos^4), A = 8 (1 - rho) / (5 + 3 rho).
 * With sin^4(a/2) = 3/8 - cos(a)/2 + cos(2a)/8 and cos^4(a/2) = 3/8 + cos(a)/2
 * + cos(2a)/8, P drops the 3/8 and xi = int_0^alpha E is a trigonometric
 * polynomial in closed form.  Returns xi, E = xi' and E' = xi'' at alpha. */
static void mesh_point(real rho, int centre, real alpha, real *xi, real *E, real *E1)
{
    real A = 8.0 * (1.0 - rho) / (5.0 + 3.0 * rho);
    real s1 = sin(alpha), c1 = cos(alpha), s2 = sin(2.0 * alpha), c2 = cos(2.0 * alpha);
    real sg = centre ? 1.0 : -1.0;       /* sign of the cos(alpha) term */
    *xi = alpha + A * (sg * 0.5 * s1 - s2 / 16.0);
    *E = 1.0 + A * (sg * 0.5 * c1 - c2 / 8.0);
    *E1 = A * (-sg * 0.5 * s1 + s2 / 4.0);
}

/* Public: the mesh of a segment at alpha_j = 2 pi j / M. */
void orc_mesh_eval(real rho, int centre, int M, real *x, real *e, real *e1)
{
    for (int j = 0; j < M; ++j) mesh_point(rho, centre, TWO_PI * j / M, x + j, e + j, e1 + j);
}

/* xi^{-1}(x) by Newton's method (Sec. 2.2), kept inside the bracket
 * |alpha - x| <= A (|xi - alpha| <= 9A/16) by bisection when a step leaves it. */
static real mesh_inverse_one(real rho, int centre, real x)
{
    real A = 8.0 * (1.0 - rho) / (5.0 + 3.0 * rho);
    real lo = x - A - 1e-12, hi = x + A + 1e-12, a = x;
    for (int it = 0; it < 200; ++it) {
        real xi, E, E1;
        mesh_point(rho, centre, a, &xi, &E, &E1);
        real r = xi - x;
        if (r == 0.0) break;
        if (r > 0.0) hi = a; else lo = a;
        real an = a - r / E;
        if (!(an > lo && an < hi)) an = 0.5 * (lo + hi);
        if (fabs(an - a) <= NEWTON_TOL * (1.0 + fabs(a))) { a = an; break; }
        a = an;
    }
    return a;
}

void orc_mesh_inverse(real rho, int centre, int n, const real *x, real *alpha)
{
    for (int i = 0; i < n; ++i) alpha[i] = mesh_inverse_one(rho, centre, x[i]);
}

/* The trigonometric interpolant of f (values at alpha_j = 2 pi j / M) at the
 * points beta[0..n): sum over |k| < M/2 of fhat_k e^{i k beta} plus the
 * Nyquist mode as fhat_{M/2} cos(M beta / 2) (reading R22); direct sums. */
void orc_interp(int M, const real *f, int n, const real *beta, real *out)
{
    cplx *fh = malloc(sizeof(cplx) * M);
    for (int j = 0; j < M; ++j) fh[j] = f[j];
    orc_fft(M, fh, 0);
    for (int j = 0; j < M; ++j) fh[j] /= M;
    for (int i = 0; i < n; ++i) {
        real acc = creal(fh[0]);
        for (int k = 1; k < M / 2; ++k)
            acc += 2.0 * creal(fh[k] * CEXP(I * (real)k * beta[i]));
        acc += creal(fh[M / 2]) * cos(0.5 * M * beta[i]);
        out[i] = acc;
    }
    free(fh);
}

/* The segment's mesh as an orc_mesh (NULL when rho == 1: the uniform grid,
 * so a uniform segment runs exactly the uniform arithmetic). */
typedef struct {
    orc_mesh m;
    real *x, *e, *e1;
} mesh_buf;

static const orc_mesh *mesh_make(mesh_buf *b, const orc_segment *sg)
{
    b->x = b->e = b->e1 = NULL;
    if (sg->rho == 1.0) return NULL;
    b->x = malloc(sizeof(real) * sg->M);
    b->e = malloc(sizeof(real) * sg->M);
    b->e1 = malloc(sizeof(real) * sg->M);
    orc_mesh_eval(sg->rho, sg->centre, sg->M, b->x, b->e, b->e1);
    b->m.x = b->x; b->m.e = b->e; b->m.e1 = b->e1;
    return &b->m;
}

static void mesh_free(mesh_buf *b) { free(b->x); free(b->e); free(b->e1); }

/* Respacing (Sec. 2.2): the new values at alpha'_j (M' points of segment b)
 * are those of the old interpolant at xi_a^{-1}(xi_b(alpha'_j)).  ncols
 * vectors of length Ma in; ncols of length Mb out. */
static void respace(const orc_segment *sa, const orc_segment *sb, int ncols, const real *in, real *out)
{
    int Ma = sa->M, Mb = sb->M;
    real *beta = malloc(sizeof(real) * Mb);
    for (int j = 0; j < Mb; ++j) {
        real xi, E, E1;
        mesh_point(sb->rho, sb->centre, TWO_PI * j / Mb, &xi, &E, &E1);
        beta[j] = mesh_inverse_one(sa->rho, sa->centre, xi);
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic)
#endif
    for (int c = 0; c < ncols; ++c) orc_interp(Ma, in + (size_t)c * Ma, Mb, beta, out + (size_t)c * Mb);
    free(beta);
}

/* One segment: `steps` steps of the tableau of size dt on the mesh, the RHS
 * filtered at every stage (inside rhs_impl) and the solution after every
 * step (reading R4). */
static void integrate_tableau(const orc_problem *p, const orc_mesh *m, int N, const orc_tableau *tb, real T,
                              real dt, int steps, real *y, int ncol, int t_col)
{
    size_t len = (size_t)(ncol + 1) * 2 * N;
    int s = tb->s;
    real *k = malloc(sizeof(real) * len * s), *ys = malloc(sizeof(real) * len);
    for (int n = 0; n < steps; ++n) {
        for (int st = 0; st < s; ++st) {
            for (size_t i = 0; i < len; ++i) {
                real acc = 0.0;
                for (int j = 0; j < st; ++j) acc += tb->a[st * s + j] * k[(size_t)j * len + i];
                ys[i] = y[i] + dt * acc;
            }
            rhs_impl(p, m, N, T, ys, ncol, t_col, k + (size_t)st * len);
        }
        for (size_t i = 0; i < len; ++i) {
            real acc = 0.0;
            for (int j = 0; j < s; ++j) acc += tb->b[j] * k[(size_t)j * len + i];
            y[i] += dt * acc;
        }
        for (int c = 0; c <= ncol; ++c) {
            orc_spectral(N, MUL_FILTER, y + (size_t)c * 2 * N, y + (size_t)c * 2 * N);
            orc_spectral(N, MUL_FILTER, y + (size_t)c * 2 * N + N, y + (size_t)c * 2 * N + N);
        }
    }
    free(k); free(ys);
}

static int segments_valid(const orc_problem *p, int nseg, const orc_segment *sg, const orc_tableau *tb)
{
    if (nseg < 1 || !tb || tb->s < 1) return 0;
    if (sg[0].M != p->N || sg[0].rho != 1.0) return 0;    /* x = alpha on the first segment */
    real th = 0.0;
    for (int l = 0; l < nseg; ++l) {
        int M = sg[l].M;
        if (M < 4 || (M & (M - 1)) || sg[l].steps < 1 || !(sg[l].theta > 0.0)) return 0;
        if (!(sg[l].rho > 0.0 && sg[l].rho <= 1.0)) return 0;
        th += sg[l].theta;
    }
    return fabs(th - 1.0) <= 1e-12;
}

/* Integrate y (ncol + 1 columns on segment 0's grid) through all segments
 * from 0 to T/4; returns the state on the last segment's grid (malloc'd). */
static real *integrate_segments(const orc_problem *p, int nseg, const orc_segment *sg, const orc_tableau *tb,
                                  real T, const real *y0, int ncol, int t_col)
{
    size_t cols = (size_t)(ncol + 1) * 2;
    real *y = malloc(sizeof(real) * cols * sg[0].M);
    memcpy(y, y0, sizeof(real) * cols * sg[0].M);
    for (int l = 0; l < nseg; ++l) {
        if (l > 0) {
            real *z = malloc(sizeof(real) * cols * sg[l].M);
            respace(&sg[l - 1], &sg[l], (int)cols, y, z);
            free(y);
            y = z;
        }
        mesh_buf b;
        const orc_mesh *m = mesh_make(&b, &sg[l]);
        real dt = sg[l].theta * (T / 4.0) / sg[l].steps;
        integrate_tableau(p, m, sg[l].M, tb, T, dt, sg[l].steps, y, ncol, t_col);
        mesh_free(&b);
    }
    return y;
}

/* Residual weights on the last segment: w_i = sqrt(E(alpha_i) / M)
 * (Eq. (f:phi) with the mesh density E). */
static void segment_weights(const orc_segment *sl, real *w)
{
    for (int i = 0; i < sl->M; ++i) {
        real xi, E, E1;
        mesh_point(sl->rho, sl->centre, TWO_PI * i / sl->M, &xi, &E, &E1);
        w[i] = sqrt(E / sl->M);
    }
}

/* Public: evolve q0 (2N on segment 0) to T/4; q_end holds 2 M_last. */
int orc_evolve_segments(const orc_problem *p, int nseg, const orc_segment *sg, const orc_tableau *tb, real T,
                        const real *q0, real *q_end)
{
    if (!segments_valid(p, nseg, sg, tb)) return -1;
    real *y = integrate_segments(p, nseg, sg, tb, T, q0, 0, 0);
    memcpy(q_end, y, sizeof(real) * 2 * sg[nseg - 1].M);
    free(y);
    return 0;
}

/* Public: r (M_last) and f of the segmented shot. */
int orc_shoot_segments(const orc_problem *p, int nseg, const orc_segment *sg, const orc_tableau *tb,
                       const real *c, real *r, real *f)
{
    if (!segments_valid(p, nseg, sg, tb)) return -1;
    int N = p->N, M = sg[nseg - 1].M;
    real *q0 = malloc(sizeof(real) * 2 * N), *w = malloc(sizeof(real) * M);
    orc_initial(p, c, q0);
    real *y = integrate_segments(p, nseg, sg, tb, c[0], q0, 0, 0);
    segment_weights(&sg[nseg - 1], w);
    real s = 0.0;
    for (int i = 0; i < M; ++i) { r[i] = w[i] * y[M + i]; s += r[i] * r[i]; }
    *f = 0.5 * s;
    free(q0); free(w); free(y);
    return 0;
}

/* Public: r, J (M_last x (n + 1), column-major, column 0 = d r / d T) and f.
 * The variational columns ride through the respacing with the base state:
 * respacing is linear, so they stay the exact derivative of the discrete map. */
int orc_shoot_jacobian_segments(const orc_problem *p, int nseg, const orc_segment *sg, const orc_tableau *tb,
                                const real *c, real *r, real *J, real *f)
{
    if (!segments_valid(p, nseg, sg, tb)) return -1;
    int N = p->N, n = p->n, ncol = n + 1, M = sg[nseg - 1].M;
    real *y0 = calloc((size_t)(ncol + 1) * 2 * N, sizeof(real)), *w = malloc(sizeof(real) * M);
    orc_initial(p, c, y0);
    for (int k = 1; k <= n; ++k)
        for (int rr = 0; rr < 2 * N; ++rr)
            y0[(size_t)(k + 1) * 2 * N + rr] = basis_entry(p, rr, k);
    real *y = integrate_segments(p, nseg, sg, tb, c[0], y0, ncol, 1);
    segment_weights(&sg[nseg - 1], w);
    real s = 0.0;
    for (int i = 0; i < M; ++i) { r[i] = w[i] * y[M + i]; s += r[i] * r[i]; }
    *f = 0.5 * s;
    for (int k = 0; k <= n; ++k)
        for (int i = 0; i < M; ++i)
            J[(size_t)k * M + i] = w[i] * y[(size_t)(k + 1) * 2 * M + M + i];
    free(y0); free(w); free(y);
    return 0;
}

/* Public (tests): the RHS of ncol + 1 columns on the mesh of a segment. */
void orc_rhs_segment(const orc_problem *p, const orc_segment *sg, real T, const real *y, int ncol, int t_col,
                     real *out)
{
    mesh_buf b;
    const orc_mesh *m = mesh_make(&b, sg);
    rhs_impl(p, m, sg->M, T, y, ncol, t_col, out);
    mesh_free(&b);
}

/* Public (tests): the DtN of phi on the surface eta, both stored on the mesh. */
void orc_dtn_segment(const orc_segment *sg, real h, const real *eta, const real *phi, real *out)
{
    mesh_buf b;
    const orc_mesh *m = mesh_make(&b, sg);
    dtn_state s;
    dtn_prepare_mesh(&s, m, sg->M, h, eta);
    dtn_apply_one(&s, phi, out);
    dtn_release(&s);
    mesh_free(&b);
}

/* ------------------------------------------------------------------ */
/* The discrete adjoint of the segmented shot (reading R18 carried to   */
/* segments, meshes and any explicit tableau)                            */
/* ------------------------------------------------------------------ */

/* out_a = R^T in_b for the respacing R of respace() (sa -> sb): column j of R
 * is the interpolant of the unit vector e_j at the new points, so R^T is the
 * transpose of the very map the forward shot applies. */
static void respace_T(const orc_segment *sa, const orc_segment *sb, const real *in_b, real *out_a)
{
    int Ma = sa->M, Mb = sb->M;
    real *beta = malloc(sizeof(real) * Mb);
    for (int j = 0; j < Mb; ++j) {
        real xi, E, E1;
        mesh_point(sb->rho, sb->centre, TWO_PI * j / Mb, &xi, &E, &E1);
        beta[j] = mesh_inverse_one(sa->rho, sa->centre, xi);
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic)
#endif
    for (int j = 0; j < Ma; ++j) {
        real *ej = calloc(Ma, sizeof(real)), *col = malloc(sizeof(real) * Mb);
        ej[j] = 1.0;
        orc_interp(Ma, ej, Mb, beta, col);
        real acc = 0.0;
        for (int i = 0; i < Mb; ++i) acc += col[i] * in_b[i];
        out_a[j] = acc;
        free(ej); free(col);
    }
    free(beta);
}

/* f and grad f (n + 1 entries, grad[0] = d f / d T) of the segmented shot by
 * its discrete adjoint.  Forward: every stage state of every step of every
 * segment is kept.  Backward, per step: mu = Filt lambda (the step filter is
 * symmetric); the stages in reverse order, kbar_i = dt (b_i mu + sum_{j>i}
 * a_ji Ybar_j) and Ybar_i = DF(Y_i)^T kbar_i; lambda = mu + sum_i Ybar_i; and
 * d f / d T gains kbar_i . F(Y_i) / T (dt is proportional to T).  Between
 * segments lambda goes back through R^T.  lambda starts from the gradient of
 * f = sum_i w_i^2 phi_i^2 / 2 on the last mesh. */
int orc_objective_and_grad_segments(const orc_problem *p, int nseg, const orc_segment *sg, const orc_tableau *tb,
                                    const real *c, real *f, real *grad)
{
    if (!segments_valid(p, nseg, sg, tb)) return -1;
    int s = tb->s;
    real T = c[0];
    real **traj = malloc(sizeof(real *) * nseg);
    real *y = malloc(sizeof(real) * 2 * p->N);
    orc_initial(p, c, y);
    for (int l = 0; l < nseg; ++l) {                 /* forward, stage states kept */
        int M = sg[l].M;
        size_t n2 = (size_t)2 * M;
        if (l > 0) {
            real *z = malloc(sizeof(real) * n2);
            respace(&sg[l - 1], &sg[l], 2, y, z);
            free(y);
            y = z;
        }
        mesh_buf b;
        const orc_mesh *m = mesh_make(&b, &sg[l]);
        real dt = sg[l].theta * (T / 4.0) / sg[l].steps;
        traj[l] = malloc(sizeof(real) * n2 * (size_t)s * sg[l].steps);
        real *k = malloc(sizeof(real) * n2 * s);
        for (int n = 0; n < sg[l].steps; ++n) {
            for (int st = 0; st < s; ++st) {
                real *ys = traj[l] + ((size_t)n * s + st) * n2;
                for (size_t i = 0; i < n2; ++i) {
                    real acc = 0.0;
                    for (int j = 0; j < st; ++j) acc += tb->a[st * s + j] * k[(size_t)j * n2 + i];
                    ys[i] = y[i] + dt * acc;
                }
                rhs_impl(p, m, M, T, ys, 0, 0, k + (size_t)st * n2);
            }
            for (size_t i = 0; i < n2; ++i) {
                real acc = 0.0;
                for (int j = 0; j < s; ++j) acc += tb->b[j] * k[(size_t)j * n2 + i];
                y[i] += dt * acc;
            }
            orc_spectral(M, MUL_FILTER, y, y);
            orc_spectral(M, MUL_FILTER, y + M, y + M);
        }
        free(k);
        mesh_free(&b);
    }
    int ML = sg[nseg - 1].M;
    real *w = malloc(sizeof(real) * ML);
    segment_weights(&sg[nseg - 1], w);
    real *lam = malloc(sizeof(real) * 2 * ML);
    real sum = 0.0;
    for (int i = 0; i < ML; ++i) {
        real ri = w[i] * y[ML + i];
        sum += ri * ri;
        lam[i] = 0.0;
        lam[ML + i] = w[i] * ri;
    }
    *f = 0.5 * sum;
    real gT = 0.0;
    for (int l = nseg - 1; l >= 0; --l) {            /* backward */
        int M = sg[l].M;
        size_t n2 = (size_t)2 * M;
        mesh_buf b;
        const orc_mesh *m = mesh_make(&b, &sg[l]);
        real dt = sg[l].theta * (T / 4.0) / sg[l].steps;
        real *mu = malloc(sizeof(real) * n2), *kb = malloc(sizeof(real) * n2 * s);
        real *yb = malloc(sizeof(real) * n2);
        for (int n = sg[l].steps - 1; n >= 0; --n) {
            orc_spectral(M, MUL_FILTER, lam, mu);
            orc_spectral(M, MUL_FILTER, lam + M, mu + M);
            for (int st = 0; st < s; ++st)
                for (size_t i = 0; i < n2; ++i) kb[(size_t)st * n2 + i] = dt * tb->b[st] * mu[i];
            memcpy(lam, mu, sizeof(real) * n2);
            for (int st = s - 1; st >= 0; --st) {
                real Fd;
                rhs_T_mesh(p, m, M, traj[l] + ((size_t)n * s + st) * n2, kb + (size_t)st * n2, yb, &Fd);
                gT += Fd / T;
                for (size_t i = 0; i < n2; ++i) lam[i] += yb[i];
                for (int j = 0; j < st; ++j) {
                    real a = tb->a[st * s + j];
                    if (a != 0.0)
                        for (size_t i = 0; i < n2; ++i) kb[(size_t)j * n2 + i] += dt * a * yb[i];
                }
            }
        }
        free(mu); free(kb); free(yb);
        mesh_free(&b);
        free(traj[l]);
        if (l > 0) {
            int Mp = sg[l - 1].M;
            real *z = malloc(sizeof(real) * 2 * Mp);
            respace_T(&sg[l - 1], &sg[l], lam, z);
            respace_T(&sg[l - 1], &sg[l], lam + M, z + Mp);
            free(lam);
            lam = z;
        }
    }
    grad[0] = gT;
    for (int kk = 1; kk <= p->n; ++kk) {
        real g = 0.0;
        for (int r = 0; r < 2 * p->N; ++r) g += basis_entry(p, r, kk) * lam[r];
        grad[kk] = g;
    }
    free(traj); free(y); free(w); free(lam);
    return 0;
}

/* Public (tests): the transposed variational RHS on a segment's mesh at the
 * base state q, applied to kb (2M); *Fdot = kb . F(q). */
void orc_rhs_T_segment(const orc_problem *p, const orc_segment *sg, const real *q, const real *kb, real *out,
                       real *Fdot)
{
    mesh_buf b;
    const orc_mesh *m = mesh_make(&b, sg);
    rhs_T_mesh(p, m, sg->M, q, kb, out, Fdot);
    mesh_free(&b);
}

/* Public (tests): the energy of Sec. 4's monitor for a state stored on a
 * segment's mesh: 1/2 int (phi G phi + g (eta - hbar)^2) dx + tau int
 * (sqrt(1 + eta'^2) - 1) dx, each integral int f dx = int f(xi(alpha)) xi'
 * dalpha by the trapezoid rule in alpha. */
real orc_energy_segment(const orc_problem *p, const orc_segment *sg, const real *q)
{
    int M = sg->M;
    mesh_buf b;
    const orc_mesh *m = mesh_make(&b, sg);
    const real *eta = q, *phi = q + M;
    real *Gphi = malloc(sizeof(real) * M), *ex = malloc(sizeof(real) * M);
    dtn_state s;
    dtn_prepare_mesh(&s, m, M, p->h, eta);
    dtn_apply_one(&s, phi, Gphi);
    dtn_release(&s);
    mesh_dx(m, M, eta, ex);
    real mean = isinf(p->h) ? 0.0 : p->h, e = 0.0;
    for (int i = 0; i < M; ++i) {
        real d = eta[i] - mean;
        real dens = 0.5 * (phi[i] * Gphi[i] + p->g * d * d) + p->tau * (sqrt(1.0 + ex[i] * ex[i]) - 1.0);
        e += dens * (m ? m->e[i] : 1.0);
    }
    free(Gphi); free(ex);
    mesh_free(&b);
    return e * TWO_PI / M;
}
