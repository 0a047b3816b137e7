// ww_segments.cu -- time segments with adaptive meshes and a general explicit
// Runge-Kutta tableau (Sec. 2.2): the paper's production runs split [0, T/4]
// into segments, each with its own grid of M_l points on the mesh x = xi(alpha)
// of Eq. (xi) (refined where the wave sharpens) and its own number of uniform
// steps of an explicit scheme (DOP853 there).  The state is carried from one
// segment to the next by trigonometric interpolation ("respacing").
//
// On a mesh every x-derivative is d/dalpha divided by xi', the DtN of Eq. (G)
// carries the factor 1/|xi'|, the kernels of Eq. (K1K2) see zeta = xi + i eta
// with zeta' = xi' + i eta_alpha, and P removes the mean over x, i.e. the
// xi'-weighted mean over alpha.  The filter acts on the alpha grid's modes.
// The first segment is uniform (xi = alpha) and starts from the initial data.
//
// One context per segment (its N is the segment's M).  Per RK stage of a
// segment: geometry and assembly on the mesh, the factorisation and the
// multi-right-hand-side solves of the context's form (FP64 LU, or the mixed
// form's inverse and refinement: they see only the assembled matrices), the
// base and variational right-hand sides on the mesh (FP64 transforms in both
// forms), and the stage update of the tableau, which keeps every stage's
// right-hand side ([S][n+2][2][N] doubles).  One stage program is captured per context and replayed `steps`
// times; there is no second graph branch here.
//
// Respacing from segment a (M_a points) to b (M_b): the new values at
// alpha'_j are the old interpolant at beta_j = xi_a^{-1}(xi_b(alpha'_j)), so
// Y_b = R Y_a for all 2 (n + 2) state columns at once, one FP64 product with
//   R_jl = (1/M_a) [D(beta_j - alpha_l) + cos(M_a beta_j / 2) (-1)^l],
// D the Dirichlet kernel of the modes |k| < M_a/2 (the Nyquist mode enters
// as f_{M/2} cos(M beta / 2)).  Respacing is linear, so the variational
// columns stay the exact derivative of the discrete map.
//
// The gradient of f on segments (Sec. 3.2 with the meshes of Sec. 2.2) is
// the discrete adjoint of this map: a forward pass of the base state alone
// that records every stage, then, segment by segment from the last, the
// transposed steps of the tableau (the filter, then the stages in reverse
// order, each with kbar_i = dt (b_i mu + sum_{j>i} a_ji Ybar_j) and Ybar_i =
// DF(Y_i)^T kbar_i) and, between segments, lambda <- R^T lambda.  On a mesh
// the transposed stage reads every D_x = diag(1/xi') D_alpha as -D_x^T =
// D_alpha diag(1/xi'), P (the xi'-weighted mean removed) as P^T v = v - xi'
// (sum v) / M, and the DtN's diag(1/xi') on the right of its transpose:
// G^T x = A^{-T} D (1/2 H - G^T) diag(1/xi') x, with A^T and G^T assembled
// on the mesh and factored in the context's form.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ww_ar.cuh"

namespace ww {

constexpr int SEG_MAX_STAGES = 16;

struct Seg {
    int steps, S, centre;
    double theta, rho;
    std::vector<double> a, b;               // tableau (host copies)
    double *d_a = nullptr, *d_b = nullptr;  // the same on the device
    // mesh tables at alpha_j (N each): xi, xi', xi'', cos xi, sin xi, 1/xi',
    // xi'/N (weights of the x-mean), sqrt(xi'/N) (residual weights)
    double *xi = nullptr, *e = nullptr, *e1 = nullptr, *cxi = nullptr, *sxi = nullptr, *einv = nullptr,
           *pw = nullptr, *wts = nullptr;
    double *K = nullptr;                    // stage right-hand sides [S][NC][2][N]
    // respacing into this segment: the interpolation matrix (N x M_a) and the
    // previous segment it was built for
    double *R = nullptr, *beta = nullptr;
    int R_M = 0, R_centre = -1;
    double R_rho = -1.0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int nkern = 0;
    // objective_and_grad_segments (allocated by its first call): the records of
    // the forward pass [steps][S][6][N] (eta, u, v, w3, F_eta, F_phi of each
    // stage), the step counter that addresses them, the adjoint state lambda
    // (2N), the adjoints of the stage right-hand sides [S][2][N], the stage's
    // scratch and this segment's share of d f / d T; the base-only step
    // program (with the records) and the transposed step program
    double *rec = nullptr, *kb = nullptr, *lam = nullptr, *chi = nullptr, *etal = nullptr, *psil = nullptr,
           *y = nullptr, *aeta = nullptr, *gT = nullptr;
    int *rstep = nullptr;
    cudaGraph_t fgraph = nullptr, bgraph = nullptr;
    cudaGraphExec_t fexec = nullptr, bexec = nullptr;
    int fkern = 0, bkern = 0;
    size_t gbytes = 0;                      // of `bytes`, the gradient's workspace
    std::vector<void *> allocs;
    size_t bytes = 0;
};

namespace {

constexpr int SEG_THREADS = 256;
constexpr double TWO_PI_HI = 6.283185307179586232;     // 2 pi rounded to double
constexpr double TWO_PI_LO = 2.4492935982947064e-16;   // 2 pi - TWO_PI_HI

// Eq. (xi): xi' = E(alpha) = 1 - P[A sin^4(alpha/2)] (refined near x = pi) or
// 1 - P[A cos^4(alpha/2)] (near x = 0), A = 8 (1 - rho) / (5 + 3 rho), P the
// mean-free part, so that xi(alpha) = alpha + (a trigonometric polynomial).
// With sin^4(a/2) = 3/8 - cos a/2 + cos 2a/8 and cos^4(a/2) = 3/8 + cos a/2 +
// cos 2a/8: E = 1 + A (sg cos a / 2 - cos 2a / 8), sg = +1 (near pi) or -1.
void mesh_at(double rho, int centre, double al, double *x, double *E, double *E1) {
    const double A = 8.0 * (1.0 - rho) / (5.0 + 3.0 * rho);
    const double sg = centre ? 1.0 : -1.0;
    *x = al + A * (sg * 0.5 * std::sin(al) - std::sin(2.0 * al) / 16.0);
    *E = 1.0 + A * (sg * 0.5 * std::cos(al) - std::cos(2.0 * al) / 8.0);
    *E1 = A * (-sg * 0.5 * std::sin(al) + std::sin(2.0 * al) / 4.0);
}

// xi^{-1}(x): Newton's method on xi(a) - x, safeguarded by bisection inside
// the bracket |a - x| <= A (xi - alpha is bounded by 9A/16)
double mesh_inv(double rho, int centre, double x) {
    const double A = 8.0 * (1.0 - rho) / (5.0 + 3.0 * rho);
    double lo = x - A - 1e-12, hi = x + A + 1e-12, a = x;
    for (int it = 0; it < 200; ++it) {
        double xi, E, E1;
        mesh_at(rho, centre, a, &xi, &E, &E1);
        const double r = xi - x;
        if (r == 0.0) break;
        if (r > 0.0)
            hi = a;
        else
            lo = a;
        double an = a - r / E;
        if (!(an > lo && an < hi)) an = 0.5 * (lo + hi);
        const bool done = std::fabs(an - a) <= 1e-15 * (1.0 + std::fabs(a));
        a = an;
        if (done) break;
    }
    return a;
}

// ---------------------------------------------------------------- geometry on the mesh
// eta_a, eta_aa: alpha-derivatives (the kernels' zeta' = xi' + i eta_a, zeta'' = xi'' + i eta_aa);
// phi_x = phi_a / xi'; curv = d/dx (eta_x / sqrt(1 + eta_x^2)), eta_x = eta_a / xi'
__global__ void __launch_bounds__(SEG_THREADS) k_geom_mesh(const double *__restrict__ eta_in,
                                                           const double *__restrict__ phi_in, int N, int logN,
                                                           int deep, int with_curv, const double2 *__restrict__ tw,
                                                           const double *__restrict__ einv, double *eta,
                                                           double *eta_a, double *eta_aa, double *phi_x, double *curv,
                                                           double *E, double *Einv, int *status) {
    extern __shared__ __align__(16) unsigned char smraw[];
    double2 *s = reinterpret_cast<double2 *>(smraw), *z = s + N;
    int bad = 0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double e = eta_in[j], p = phi_in[j];
        if (!isfinite(e) || !isfinite(p) || (!deep && e <= 0.0)) bad = 1;
        eta[j] = e;
        const double ee = exp(e);
        E[j] = ee;
        Einv[j] = 1.0 / ee;
        s[j] = make_double2(e, p);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, ST_GEOMETRY);
    block_fft(s, N, logN, tw, false);
    const double invN = 1.0 / N;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const int k = wavenum(j, N);
        const bool nyq = 2 * j == N;
        const double2 v = cscale(make_double2(-(double)k * s[j].y, (double)k * s[j].x), invN);
        s[j] = nyq ? make_double2(0.0, 0.0) : v;
        z[j] = nyq ? make_double2(0.0, 0.0) : make_double2(-(double)k * v.y, (double)k * v.x);
    }
    __syncthreads();
    block_fft(s, N, logN, tw, true);
    block_fft(z, N, logN, tw, true);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double ea = s[j].x, ex = ea * einv[j];
        eta_a[j] = ea;
        phi_x[j] = s[j].y * einv[j];
        eta_aa[j] = z[j].x;
        if (with_curv)
            s[j] = make_double2(ex / sqrt(1.0 + ex * ex), 0.0);
        else
            curv[j] = 0.0;
    }
    if (!with_curv) return;
    __syncthreads();
    block_fft(s, N, logN, tw, false);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const int k = wavenum(j, N);
        s[j] = 2 * j == N ? make_double2(0.0, 0.0)
                          : cscale(make_double2(-(double)k * s[j].y, (double)k * s[j].x), invN);
    }
    __syncthreads();
    block_fft(s, N, logN, tw, true);
    for (int j = threadIdx.x; j < N; j += blockDim.x) curv[j] = s[j].x * einv[j];
}

// ---------------------------------------------------------------- assembly on the mesh
// sinh of a small difference by its series (full relative accuracy), else from exponentials
__device__ __forceinline__ double sinh_small(double y, double ey, double eyi) {
    if (fabs(y) < 0.25) {
        const double y2 = y * y;
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

// cos x and sin x of x = xi_i - xi_j: for |x| (taken into (-pi, pi] with a
// double-double 2 pi) below 1/4 from their series, which keeps the relative
// accuracy of the small sines of neighbouring points; otherwise from the
// per-point tables by the angle-difference formulas
__device__ __forceinline__ void cos_sin_diff(double xi_i, double xi_j, double ci, double si, double cj, double sj,
                                             double *cx, double *sx) {
    double x = xi_i - xi_j;
    if (x > 3.0) x = (x - TWO_PI_HI) - TWO_PI_LO;
    else if (x < -3.0) x = (x + TWO_PI_HI) + TWO_PI_LO;
    if (fabs(x) < 0.25) {
        const double x2 = x * x;
        double ps = -1.0 / 1307674368000.0;   // sin: x (1 - x^2/3! + ... - x^14/15!)
        ps = fma(ps, x2, 1.0 / 6227020800.0);
        ps = fma(ps, x2, -1.0 / 39916800.0);
        ps = fma(ps, x2, 1.0 / 362880.0);
        ps = fma(ps, x2, -1.0 / 5040.0);
        ps = fma(ps, x2, 1.0 / 120.0);
        ps = fma(ps, x2, -1.0 / 6.0);
        ps = fma(ps, x2, 1.0);
        double pc = 1.0 / 20922789888000.0;   // cos: 1 - x^2/2! + ... + x^16/16!
        pc = fma(pc, x2, -1.0 / 87178291200.0);
        pc = fma(pc, x2, 1.0 / 479001600.0);
        pc = fma(pc, x2, -1.0 / 3628800.0);
        pc = fma(pc, x2, 1.0 / 40320.0);
        pc = fma(pc, x2, -1.0 / 720.0);
        pc = fma(pc, x2, 1.0 / 24.0);
        pc = fma(pc, x2, -0.5);
        pc = fma(pc, x2, 1.0);
        *sx = x * ps;
        *cx = pc;
    } else {
        *cx = fma(ci, cj, si * sj);
        *sx = fma(si, cj, -(ci * sj));
    }
}

// cot((x + i y)/2) by the branch-stable quotients (cx = cos x, sx = sin x, ch = cosh y, sh = sinh y)
__device__ __forceinline__ double2 cot_half_q(double cx, double sx, double ch, double sh) {
    if (cx >= 0.0) {
        const double inv = (cx + ch) / fma(sx, sx, sh * sh);
        return make_double2(sx * inv, -sh * inv);
    }
    const double inv = 1.0 / (ch - cx);
    return make_double2(sx * inv, -sh * inv);
}

constexpr int MT = 32;

// A = 1/2 I + K, G on the mesh (Eq. (K1K2), images with the minus sign), one
// 32 x 32 tile pair (I <= J) per block: both cotangents of an unordered pair
// give the (i, j) and the (j, i) entries (cot is odd), with zeta' = e + i eta_a:
//   2 K_ij = ea_j (c1 + c2).x + e_j (c1 - c2).y,   2 G_ij = e_i (c1 - c2).x - ea_i (c1 - c2).y - c0
//   2 K_ji = -[ea_i (c1 + c2).x + e_i (c1 + c2).y], 2 G_ji = -e_j (c1 - c2).x + ea_j (c1 + c2).y + c0
// c1 = cot((zeta_i - zeta_j)/2), c2 = cot((zeta_i - conj zeta_j)/2), c0 = cot((alpha_i - alpha_j)/2);
// diagonal: zeta''/(2 zeta') with zeta'' = e1 + i eta_aa.  TR: A^T and G^T
// (the discrete adjoint's transposed DtN).
template <bool DEEP, bool TR>
__global__ void __launch_bounds__(256) k_assemble_mesh(const double *__restrict__ eta, const double *__restrict__ ea,
                                                       const double *__restrict__ eaa, const double *__restrict__ E,
                                                       const double *__restrict__ Einv, const double *__restrict__ xi,
                                                       const double *__restrict__ e, const double *__restrict__ e1,
                                                       const double *__restrict__ cxi, const double *__restrict__ sxi,
                                                       const double *__restrict__ cot0, int N, double *A, double *G) {
    __shared__ double tA[MT][MT + 1], tG[MT][MT + 1];
    const int T = N / MT;
    int b = blockIdx.x, I = 0;
    while (b >= T - I) {
        b -= T - I;
        ++I;
    }
    const int J = I + b;
    const double h = 0.5 / N;
    const int il = threadIdx.x & 31;
    const int i = I * MT + il;
    const double ei = eta[i], exi = ea[i], Ei = E[i], Eii = Einv[i], mi = e[i], xii = xi[i], ci = cxi[i], si = sxi[i];
    for (int jl = threadIdx.x >> 5; jl < MT; jl += 8) {
        const int j = J * MT + jl;
        const double ej = eta[j], exj = ea[j], Ej = E[j], Eij = Einv[j], mj = e[j];
        double kij, gij, kji, gji;
        if (i == j) {
            const double den = 1.0 / fma(mi, mi, exi * exi);
            kij = -fma(eaa[i], mi, -e1[i] * exi) * den;
            gij = fma(e1[i], mi, eaa[i] * exi) * den;
            if (!DEEP) {
                const double ep = Ei * Ej, epi = Eii * Eij;
                const double2 ct = cot_half_q(1.0, 0.0, 0.5 * (ep + epi), 0.5 * (ep - epi));
                kij -= fma(-exj, ct.x, mj * ct.y);
                gij -= fma(-exi, ct.y, mi * ct.x);
            }
            kji = kij;
            gji = gij;
        } else {
            double cx, sx;
            cos_sin_diff(xii, xi[j], ci, si, cxi[j], sxi[j], &cx, &sx);
            int m = i - j;
            if (m < 0) m += N;
            const double c0 = cot0[m];
            const double y = ei - ej;
            const double ey = Ei * Eij, eyi = Eii * Ej;
            const double2 c1 = cot_half_q(cx, sx, 0.5 * (ey + eyi), sinh_small(y, ey, eyi));
            double2 c2 = make_double2(0.0, 0.0);
            if (!DEEP) {
                const double ep = Ei * Ej, epi = Eii * Eij;
                c2 = cot_half_q(cx, sx, 0.5 * (ep + epi), 0.5 * (ep - epi));
            }
            const double a = c1.x + c2.x, bb = c1.y - c2.y, cc = c1.x - c2.x, d = c1.y + c2.y;
            kij = fma(exj, a, mj * bb);
            gij = fma(-exi, bb, mi * cc) - c0;
            kji = -fma(exi, a, mi * d);
            gji = fma(exj, d, -(mj * cc)) + c0;
        }
        if (TR) {   // A^T and G^T: the (j, i) entries go where the (i, j) ones would
            const double tk = kij, tg = gij;
            kij = kji;
            gij = gji;
            kji = tk;
            gji = tg;
        }
        const size_t idx = (size_t)j * N + i;
        A[idx] = fma(h, kij, i == j ? 0.5 : 0.0);
        G[idx] = h * gij;
        tA[jl][il] = fma(h, kji, i == j ? 0.5 : 0.0);
        tG[jl][il] = h * gji;
    }
    if (I == J) return;
    __syncthreads();
    for (int il2 = threadIdx.x >> 5; il2 < MT; il2 += 8) {
        const int jl2 = threadIdx.x & 31;
        const size_t idx = (size_t)(I * MT + il2) * N + J * MT + jl2;
        A[idx] = tA[jl2][il2];
        G[idx] = tG[jl2][il2];
    }
}

// ---------------------------------------------------------------- the tableau's stage update
// s holds the filtered right-hand side k_st of one column (physical values);
// F (or NULL) an FP64 forcing added as F * fs (the T column's F(q)/T, added
// in FP64 so that the column's small values keep their precision in the
// double-float form).  Before the last stage: K[st] = k_st and
// Ys = Y + dt sum_{q <= st} a[st+1][q] K[q]; at the last:
// Y = Ys = filter(Y + dt sum_q b[q] K[q]).
template <class AR>
__device__ void tab_update(typename AR::C *s, int N, int logN, const void *__restrict__ tw,
                           const void *__restrict__ filt, int st, int S, const double *__restrict__ ta,
                           const double *__restrict__ tb, double dt, double *Yc, double *Ysc, double *Kc, size_t ks,
                           const double *__restrict__ F, double fs) {
    auto kval = [&](int j) {
        double2 k = AR::get(s[j]);
        if (F) {
            k.x += F[j] * fs;
            k.y += F[N + j] * fs;
        }
        return k;
    };
    if (st < S - 1) {
        const double *arow = ta + (size_t)(st + 1) * S;
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            const double2 k = kval(j);
            Kc[(size_t)st * ks + j] = k.x;
            Kc[(size_t)st * ks + N + j] = k.y;
            double ae = 0.0, ap = 0.0;
            for (int q = 0; q < st; ++q) {
                ae += arow[q] * Kc[(size_t)q * ks + j];
                ap += arow[q] * Kc[(size_t)q * ks + N + j];
            }
            ae += arow[st] * k.x;
            ap += arow[st] * k.y;
            Ysc[j] = Yc[j] + dt * ae;
            Ysc[N + j] = Yc[N + j] + dt * ap;
        }
        return;
    }
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double2 k = kval(j);
        double ae = 0.0, ap = 0.0;
        for (int q = 0; q < st; ++q) {
            ae += tb[q] * Kc[(size_t)q * ks + j];
            ap += tb[q] * Kc[(size_t)q * ks + N + j];
        }
        ae += tb[st] * k.x;
        ap += tb[st] * k.y;
        s[j] = AR::mk(Yc[j] + dt * ae, Yc[N + j] + dt * ap);
    }
    __syncthreads();
    AR::fft(s, N, logN, tw, false);
    for (int j = threadIdx.x; j < N; j += blockDim.x) s[j] = AR::scale_tab(s[j], filt, j);
    __syncthreads();
    AR::fft(s, N, logN, tw, true);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double2 v = AR::get(s[j]);
        Yc[j] = Ysc[j] = v.x;
        Yc[N + j] = Ysc[N + j] = v.y;
    }
}

// xi'-weighted mean over alpha (the x-mean of P, trapezoid rule): one block, every thread gets it
__device__ double block_wsum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) red[32] = t;
    }
    __syncthreads();
    const double t = red[32];
    __syncthreads();
    return t;
}

// ---------------------------------------------------------------- base right-hand side on the mesh
// Eq. (ww) with Eq. (uv:from:G): G phi = Gout / xi', eta_x = eta_a / xi';
// phi_t = P[v G phi - u^2/2 - v^2/2 - g eta + tau curv], P removing the x-mean
__global__ void __launch_bounds__(SEG_THREADS) k_base_rhs_mesh(
    const double *__restrict__ Gphi, const double *__restrict__ eta, const double *__restrict__ eta_a,
    const double *__restrict__ phi_x, const double *__restrict__ curv, const double *__restrict__ einv,
    const double *__restrict__ pw, double g, double tau, int N, int logN, const double2 *__restrict__ tw,
    const double *__restrict__ filt, double *ux, double *vy, double *w3, float2 *uxd, float2 *vyd, float2 *w3d,
    double *Fbase, double *Y, double *Ys, double *K, size_t ks, int st, int S, const double *__restrict__ ta,
    const double *__restrict__ tb, const double *__restrict__ cvec, double theta, int steps, int *status) {
    extern __shared__ __align__(16) unsigned char smraw[];
    double2 *s = reinterpret_cast<double2 *>(smraw);
    __shared__ double red[33];
    int bad = 0;
    double part = 0.0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double ex = eta_a[j] * einv[j], d = 1.0 + ex * ex, gp = Gphi[j] * einv[j], pp = phi_x[j];
        const double u = (pp - ex * gp) / d;
        const double v = (ex * pp + gp) / d;
        const double w = 1.0 / (d * sqrt(d));
        ux[j] = u;
        vy[j] = v;
        w3[j] = w;
        if (uxd) {
            uxd[j] = df_split(u);
            vyd[j] = df_split(v);
            w3d[j] = df_split(w);
        }
        const double pt = v * gp - 0.5 * u * u - 0.5 * v * v - g * eta[j] + tau * curv[j];
        if (!isfinite(pt) || !isfinite(gp)) bad = 1;
        s[j] = make_double2(gp, pt);
        part += pt * pw[j];
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, ST_NONFINITE);
    const double mean = block_wsum(part, red);
    for (int j = threadIdx.x; j < N; j += blockDim.x) s[j].y -= mean;
    __syncthreads();
    block_fft(s, N, logN, tw, false);
    for (int j = threadIdx.x; j < N; j += blockDim.x) s[j] = cscale(s[j], filt[j]);
    __syncthreads();
    block_fft(s, N, logN, tw, true);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        Fbase[j] = s[j].x;
        Fbase[N + j] = s[j].y;
    }
    const double dt = theta * (cvec[0] / 4.0) / steps;
    __syncthreads();
    tab_update<ArF64>(s, N, logN, tw, filt, st, S, ta, tb, dt, Y, Ys, K, ks, nullptr, 0.0);
}

// ---------------------------------------------------------------- variational right-hand sides on the mesh
// Eqs. (l5a), (l6a) with every d/dx = (d/dalpha) / xi' and G psi = Gout / xi':
//   etadot_t = G psi - (etadot u)_x
//   phidot_t = P[ -(etadot u v)_x - u psi_x + v G psi - g etadot + tau (etadot_x w3)_x ]
// filtered; the T column adds F(q)/T; one column per block
template <class AR>
__global__ void __launch_bounds__(SEG_THREADS, 2) k_col_rhs_mesh(
    const double *__restrict__ Gout, const void *__restrict__ uT, const void *__restrict__ vT,
    const void *__restrict__ wT, const void *__restrict__ einvT, const double *__restrict__ einv,
    const double *__restrict__ vy, const double *__restrict__ pw, const double *__restrict__ Fbase, double g,
    double tau, int N, int logN, const void *__restrict__ tw_table, const void *__restrict__ filt, double *Y, double *Ys,
    double *K, size_t ks, int st, int S, const double *__restrict__ ta, const double *__restrict__ tb,
    const double *__restrict__ cvec, double theta, int steps, int *status) {
    using R = typename AR::R;
    extern __shared__ __align__(16) unsigned char smraw[];
    typename AR::C *s = reinterpret_cast<typename AR::C *>(smraw), *z = s + AR::cap(N);
    const void *tw = stage_twiddles<AR>(tw_table, z + AR::cap(N), N, logN);   // read after the first barrier
    __shared__ double red[33];
    const int c = blockIdx.x + 1;
    double *Yc = Y + (size_t)c * 2 * N, *Ysc = Ys + (size_t)c * 2 * N, *Kc = K + (size_t)c * 2 * N;
    const double *Gpsi = Gout + (size_t)c * N;
    // psi + i etadot  ->  (psi_x, etadot_x)
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double ed = Ysc[j];
        s[j] = AR::mk(Ysc[N + j] - vy[j] * ed, ed);
    }
    __syncthreads();
    AR::fft(s, N, logN, tw, false);
    mul_deriv<AR>(s, N);
    __syncthreads();
    AR::fft(s, N, logN, tw, true);
    int bad = 0;
    const R gR = AR::from(g), tauR = AR::from(tau);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double gpd = Gpsi[j] * einv[j];
        const R ei = AR::tab(einvT, j);
        const R ed = AR::from(Ysc[j]), gp = AR::from(gpd);
        const R u = AR::tab(uT, j), v = AR::tab(vT, j);
        const R dpsi = AR::rmul(AR::re(s[j]), ei), ded = AR::rmul(AR::im(s[j]), ei);
        // undifferentiated terms: (G psi, v G psi - u psi_x - g etadot)
        z[j] = AR::mkr(gp, AR::rsub(AR::rsub(AR::rmul(v, gp), AR::rmul(u, dpsi)), AR::rmul(gR, ed)));
        // terms under one d/dx: (-etadot u, tau etadot_x w3 - etadot u v)
        const R eu = AR::rmul(ed, u);
        R im = AR::rneg(AR::rmul(eu, v));
        if (tau != 0.0) im = AR::radd(im, AR::rmul(tauR, AR::rmul(ded, AR::tab(wT, j))));
        s[j] = AR::mkr(AR::rneg(eu), im);
        if (!isfinite(gpd)) bad = 1;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, ST_NONFINITE);
    AR::fft(s, N, logN, tw, false);
    mul_deriv<AR>(s, N);
    __syncthreads();
    AR::fft(s, N, logN, tw, true);
    // total = z + (derivative terms) / xi', then P on the phi part (x-mean, in FP64)
    double part = 0.0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const R ei = AR::tab(einvT, j);
        z[j] = AR::addr(z[j], AR::rmul(AR::re(s[j]), ei), AR::rmul(AR::im(s[j]), ei));
        part += AR::get(z[j]).y * pw[j];
    }
    const double mean = block_wsum(part, red);
    for (int j = threadIdx.x; j < N; j += blockDim.x) z[j] = AR::addr(z[j], AR::from(0.0), AR::from(-mean));
    __syncthreads();
    AR::fft(z, N, logN, tw, false);
    for (int j = threadIdx.x; j < N; j += blockDim.x) z[j] = AR::scale_tab(z[j], filt, j);
    __syncthreads();
    AR::fft(z, N, logN, tw, true);
    // d/dT column: + F(q) / T (every step's dt is proportional to T), added in FP64
    const double dt = theta * (cvec[0] / 4.0) / steps;
    __syncthreads();
    tab_update<AR>(z, N, logN, tw, filt, st, S, ta, tb, dt, Yc, Ysc, Kc, ks, c == 1 ? Fbase : nullptr,
                   1.0 / cvec[0]);
}

// ---------------------------------------------------------------- respacing and outputs
// R (Mb x Ma, column-major): the trigonometric interpolant of the Ma-point grid at beta_j
__global__ void k_respace_matrix(const double *__restrict__ beta, int Mb, int Ma, double *R) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = blockIdx.y;
    if (j >= Mb || l >= Ma) return;
    const double two_pi = 6.283185307179586476925286766559;
    double th = beta[j] - two_pi * l / Ma;
    th -= two_pi * rint(th / two_pi);                  // into [-pi, pi]
    const double sh = sin(0.5 * th);
    // Dirichlet kernel 1 + 2 sum_{k=1}^{Ma/2-1} cos(k th) = sin((Ma-1) th/2) / sin(th/2)
    const double D = fabs(sh) < 1e-300 ? (double)(Ma - 1) : sin(0.5 * (Ma - 1) * th) / sh;
    const double nyq = cos(0.5 * Ma * beta[j]) * ((l & 1) ? -1.0 : 1.0);
    R[(size_t)l * Mb + j] = (D + nyq) / Ma;
}

// r_i = sqrt(xi'_i / N) phi_i (Eq. (f:phi) with the mesh density), f = r.r/2,
// J_k = sqrt(xi' / N) phidot_k
__global__ void k_outputs_mesh_r(const double *__restrict__ Y, const double *__restrict__ wts, int N, double *r,
                                 double *f) {
    __shared__ double red[33];
    double acc = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double v = Y[N + i] * wts[i];
        r[i] = v;
        acc = fma(v, v, acc);
    }
    const double t = block_wsum(acc, red);
    if (threadIdx.x == 0) *f = 0.5 * t;
}

__global__ void k_outputs_mesh_J(const double *__restrict__ Y, const double *__restrict__ wts, int N, int nc,
                                 double *J) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= N || c >= nc) return;
    J[(size_t)c * N + i] = Y[(size_t)(c + 1) * 2 * N + N + i] * wts[i];
}

// ---------------------------------------------------------------- the discrete adjoint on a segment
constexpr int SEG_REC = 6;   // doubles per point in a stage record

// the record of stage `off` of the current step (off = -1: the last stage of
// the step before), or NULL outside the records held
__device__ __forceinline__ const double *seg_rec_at(const double *rec, const int *rstep, int off, int S, int steps,
                                                    int N) {
    const long idx = (long)(*rstep) * S + off;
    if (idx < 0 || idx >= (long)steps * S) return nullptr;
    return rec + (size_t)idx * SEG_REC * N;
}

// forward: the stage's surface (its eta before the stage) and fields into the
// record of (step, st); the last stage advances the step counter
__global__ void k_seg_record(const double *__restrict__ eta, const double *__restrict__ ux,
                             const double *__restrict__ vy, const double *__restrict__ w3,
                             const double *__restrict__ F, int N, int st, int S, int steps, double *rec, int *rstep) {
    const int n = *rstep;
    if (n >= 0 && n < steps) {
        double *r = rec + ((size_t)n * S + st) * SEG_REC * N;
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            r[j] = eta[j];
            r[N + j] = ux[j];
            r[2 * N + j] = vy[j];
            r[3 * N + j] = w3[j];
            r[4 * N + j] = F[j];
            r[5 * N + j] = F[N + j];
        }
    }
    __syncthreads();   // every thread has read the counter
    if (st == S - 1 && threadIdx.x == 0) *rstep = n + 1;
}

// lambda = (0, w^2 phi) on the last mesh (the gradient of f = sum (w_i phi_i)^2 / 2
// with respect to the final state), f itself, in the order of k_outputs_mesh_r
__global__ void k_seg_adj_init(const double *__restrict__ Y, const double *__restrict__ wts, int N, double *lam,
                               double *f) {
    __shared__ double red[33];
    double acc = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double w = wts[i], v = Y[N + i] * w;
        lam[i] = 0.0;
        lam[N + i] = w * v;
        acc = fma(v, v, acc);
    }
    const double t = block_wsum(acc, red);
    if (threadIdx.x == 0) *f = 0.5 * t;
}

// start of a transposed step: step -= 1; lambda <- Filt lambda (= mu);
// kbar_st = dt b_st mu for every stage
__global__ void __launch_bounds__(SEG_THREADS) k_seg_adj_begin(double *lam, double *kb, int N, int logN,
                                                               const double2 *__restrict__ tw,
                                                               const double *__restrict__ filt,
                                                               const double *__restrict__ tb, int S,
                                                               const double *__restrict__ cvec, double theta,
                                                               int steps, int *rstep) {
    extern __shared__ __align__(16) unsigned char smraw[];
    double2 *s = reinterpret_cast<double2 *>(smraw);
    for (int j = threadIdx.x; j < N; j += blockDim.x) s[j] = make_double2(lam[j], lam[N + j]);
    __syncthreads();
    block_fft(s, N, logN, tw, false);
    for (int j = threadIdx.x; j < N; j += blockDim.x) s[j] = cscale(s[j], filt[j]);
    __syncthreads();
    block_fft(s, N, logN, tw, true);
    const double dt = theta * (cvec[0] / 4.0) / steps;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double2 v = s[j];
        lam[j] = v.x;
        lam[N + j] = v.y;
        for (int st = 0; st < S; ++st) {
            const double w = dt * tb[st];
            kb[(size_t)st * 2 * N + j] = w * v.x;
            kb[(size_t)st * 2 * N + N + j] = w * v.y;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *rstep = *rstep - 1;
}

// the recorded surface of stage `off` of the current step
__global__ void k_seg_adj_fetch(const double *__restrict__ rec, const int *rstep, int off, int S, int steps, int N,
                                double *eta) {
    const double *r = seg_rec_at(rec, rstep, off, S, steps, N);
    if (!r) return;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) eta[j] = r[j];
}

// i k / N on FFT slot j (Nyquist zeroed): the derivative in alpha, normalised
__device__ __forceinline__ double2 deriv_slot(double2 v, int j, int N) {
    if (2 * j == N) return make_double2(0.0, 0.0);
    const double k = (double)wavenum(j, N) / N;
    return make_double2(-k * v.y, k * v.x);
}

// the stage's local adjoint terms on the mesh (one block):
//   et = Filt kbar_eta, pt = P^T Filt kbar_phi, chis = (et + v pt) / xi',
//   etal = u D_a(et/xi') + u v D_a(pt/xi') - g pt + tau D_a(w3 D_a(pt/xi') / xi'),
//   psil = D_a(u pt / xi'), and d f / d T += kbar . F / T
__global__ void __launch_bounds__(SEG_THREADS) k_seg_adj_local(
    const double *__restrict__ kb, const double *__restrict__ rec, const int *rstep, int st, int S, int steps, int N,
    int logN, const double2 *__restrict__ tw, const double *__restrict__ filt, const double *__restrict__ e,
    const double *__restrict__ einv, double g, double tau, const double *__restrict__ cvec, double *chis,
    double *etal, double *psil, double *gT) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[33];
    double2 *s0 = reinterpret_cast<double2 *>(smraw), *s1 = s0 + N;
    const double *r = seg_rec_at(rec, rstep, st, S, steps, N);
    if (!r) return;
    const double *ux = r + N, *vy = r + 2 * N, *w3 = r + 3 * N, *F = r + 4 * N;
    double fd = 0.0;
    for (int j = threadIdx.x; j < 2 * N; j += blockDim.x) fd = fma(kb[j], F[j], fd);
    fd = block_wsum(fd, red);
    if (threadIdx.x == 0) *gT += fd / cvec[0];
    for (int j = threadIdx.x; j < N; j += blockDim.x) s0[j] = make_double2(kb[j], kb[N + j]);
    __syncthreads();
    block_fft(s0, N, logN, tw, false);
    for (int j = threadIdx.x; j < N; j += blockDim.x) s0[j] = cscale(s0[j], filt[j]);
    __syncthreads();
    block_fft(s0, N, logN, tw, true);
    double part = 0.0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) part += s0[j].y;
    const double mean = block_wsum(part, red) / N;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double et = s0[j].x, pt = s0[j].y - e[j] * mean, ei = einv[j];
        chis[j] = fma(vy[j], pt, et) * ei;
        s0[j] = make_double2(et * ei, pt * ei);
        s1[j] = make_double2(pt, 0.0);
    }
    __syncthreads();
    block_fft(s0, N, logN, tw, false);
    for (int j = threadIdx.x; j < N; j += blockDim.x) s0[j] = deriv_slot(s0[j], j, N);
    __syncthreads();
    block_fft(s0, N, logN, tw, true);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double det = s0[j].x, dpt = s0[j].y, u = ux[j], v = vy[j], pt = s1[j].x, ei = einv[j];
        etal[j] = u * det + u * v * dpt - g * pt;
        s0[j] = make_double2(u * pt * ei, w3[j] * dpt * ei);
    }
    __syncthreads();
    block_fft(s0, N, logN, tw, false);
    for (int j = threadIdx.x; j < N; j += blockDim.x) s0[j] = deriv_slot(s0[j], j, N);
    __syncthreads();
    block_fft(s0, N, logN, tw, true);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        psil[j] = s0[j].x;
        etal[j] += tau * s0[j].y;
    }
}

// M[:, 0] = D (1/2 H chis - y), y = G^T chis, from one transform of chis + i y:
// the real multiplier |k|/2 - k (even part |k|/2, the symbol of D H / 2, on
// chis; odd part -k, i.e. -ik = -D, on y), Nyquist zeroed
__global__ void __launch_bounds__(SEG_THREADS) k_seg_adj_dtn(const double *__restrict__ chis,
                                                             const double *__restrict__ y, int N, int logN,
                                                             const double2 *__restrict__ tw, double *M) {
    extern __shared__ __align__(16) unsigned char smraw[];
    double2 *s = reinterpret_cast<double2 *>(smraw);
    for (int j = threadIdx.x; j < N; j += blockDim.x) s[j] = make_double2(chis[j], y[j]);
    __syncthreads();
    block_fft(s, N, logN, tw, false);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double k = (double)wavenum(j, N);
        s[j] = cscale(s[j], 2 * j == N ? 0.0 : (0.5 * fabs(k) - k) / N);
    }
    __syncthreads();
    block_fft(s, N, logN, tw, true);
    for (int j = threadIdx.x; j < N; j += blockDim.x) M[j] = s[j].x;
}

// pb = A^{-T}(...) + psil, eb = etal - v pb; lambda += (eb, pb);
// kbar_q += dt a[st][q] (eb, pb) for the stages q < st
__global__ void k_seg_adj_update(const double *__restrict__ M, const double *__restrict__ psil,
                                 const double *__restrict__ etal, const double *__restrict__ rec, const int *rstep,
                                 int st, int S, int steps, int N, const double *__restrict__ ta, double theta,
                                 const double *__restrict__ cvec, double *lam, double *kb) {
    const double *r = seg_rec_at(rec, rstep, st, S, steps, N);
    if (!r) return;
    const double *vy = r + 2 * N;
    const double dt = theta * (cvec[0] / 4.0) / steps;
    const double *arow = ta + (size_t)st * S;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        const double pb = M[j] + psil[j];
        const double eb = fma(-vy[j], pb, etal[j]);
        lam[j] += eb;
        lam[N + j] += pb;
        for (int q = 0; q < st; ++q) {
            const double a = arow[q];
            if (a == 0.0) continue;
            const double w = dt * a;
            kb[(size_t)q * 2 * N + j] += w * eb;
            kb[(size_t)q * 2 * N + N + j] += w * pb;
        }
    }
}

// lambda_a = R^T lambda_b for both halves (R: Mb x Ma column-major), one block per row of R^T
__global__ void k_seg_respace_T(const double *__restrict__ R, int Mb, int Ma, const double *__restrict__ lb,
                                double *la) {
    __shared__ double red[33];
    const int l = blockIdx.x;
    const double *col = R + (size_t)l * Mb;
    double ae = 0.0, ap = 0.0;
    for (int j = threadIdx.x; j < Mb; j += blockDim.x) {
        ae = fma(col[j], lb[j], ae);
        ap = fma(col[j], lb[Mb + j], ap);
    }
    ae = block_wsum(ae, red);
    ap = block_wsum(ap, red);
    if (threadIdx.x == 0) {
        la[l] = ae;
        la[Ma + l] = ap;
    }
}

// grad[0] += this segment's d f / d T
__global__ void k_seg_add(double *dst, const double *__restrict__ src) { *dst += *src; }

// grad[k] = basis_k . lambda(0) for k = 1..n, one block per entry
__global__ void k_seg_grad(const double *__restrict__ basis, const double *__restrict__ lam, int N, double *grad) {
    __shared__ double red[33];
    const int k = blockIdx.x + 1;
    const double *b = basis + (size_t)(k - 1) * 2 * N;
    double acc = 0.0;
    for (int j = threadIdx.x; j < 2 * N; j += blockDim.x) acc = fma(b[j], lam[j], acc);
    acc = block_wsum(acc, red);
    if (threadIdx.x == 0) grad[k] = acc;
}

template <typename T>
int seg_alloc(Ctx *c, Seg *g, T **p, size_t n) {
    const size_t bytes = sizeof(T) * (n ? n : 1);
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), bytes);
    if (e != cudaSuccess) return fail(WW_ERR_ALLOC, std::string("segment workspace: ") + cudaGetErrorString(e));
    g->allocs.push_back(*p);
    g->bytes += bytes;
    c->dev_bytes += bytes;
    return WW_OK;
}

void free_seg(Ctx *c, Seg *g) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->fexec) cudaGraphExecDestroy(g->fexec);
    if (g->fgraph) cudaGraphDestroy(g->fgraph);
    if (g->bexec) cudaGraphExecDestroy(g->bexec);
    if (g->bgraph) cudaGraphDestroy(g->bgraph);
    for (void *p : g->allocs) cudaFree(p);
    c->dev_bytes -= g->bytes;
    delete g;
}

// ---------------------------------------------------------------- one stage of a segment
// the form's factorisation of the assembled operator; the mixed form moves its
// approximate inverse to it (fresh: from 4/3 I), on odd stages only when the
// last move left max|I - A X| above its threshold unless the schedule updates
// on every stage.  The shot-adaptive cadence is not used here: with a few
// hundred columns a third correction costs less than moving the inverse.
int seg_factor(Ctx *c, bool fresh, int st = 0) {
    if (c->precision == WW_MIXED)
        return mixed_setup(c, fresh ? 1 : 0, c->sch.ns_every == 1 || st % 2 == 0, false);
    return lu_factor_fp64(c);
}

int seg_solve(Ctx *c, double *B, int ncols) {
    if (c->precision == WW_MIXED) return mixed_solve(c, B, ncols);
    return lu_solve_fp64(c, B, ncols);
}

int seg_apply_G(Ctx *c, int col0, int ncols) {
    if (c->precision == WW_MIXED) {
        WW_TRY(mixed_apply_G(c, col0, ncols, 0));
        return mixed_apply_G(c, col0, ncols, 1);
    }
    return dgemm(c->stream, c->N, ncols, c->N, 1.0, c->G, c->N, c->Gam + (size_t)col0 * c->N, c->N, 1.0,
                 c->Gout + (size_t)col0 * c->N, c->N);
}

// the geometry of the surface eta_in (and phi_x of phi_in); the stage state's by default
int seg_geometry(Ctx *c, Seg *g, const double *eta_in = nullptr, const double *phi_in = nullptr,
                 bool with_curv = true) {
    const size_t sm = 2 * sizeof(double2) * (size_t)c->N;
    if (!eta_in) {
        eta_in = c->Ys;
        phi_in = c->Ys + c->N;
    }
    k_geom_mesh<<<1, SEG_THREADS, sm, c->stream>>>(eta_in, phi_in, c->N, c->logN, c->deep ? 1 : 0,
                                                  with_curv && c->tau != 0.0 ? 1 : 0, c->tw, g->einv, c->eta,
                                                  c->eta_x, c->eta_xx, c->phi_s, c->curv, c->E, c->Einv, c->status);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

// A = 1/2 I + K and G on the mesh, or A^T and G^T while c->trans is set
int seg_assemble(Ctx *c, Seg *g) {
    const int T = c->N / MT;
    auto kern = c->deep ? (c->trans ? k_assemble_mesh<true, true> : k_assemble_mesh<true, false>)
                        : (c->trans ? k_assemble_mesh<false, true> : k_assemble_mesh<false, false>);
    kern<<<T * (T + 1) / 2, 256, 0, c->stream>>>(c->eta, c->eta_x, c->eta_xx, c->E, c->Einv, g->xi, g->e, g->e1,
                                                 g->cxi, g->sxi, c->cs + 2 * c->N, c->N, c->A, c->G);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

// the base state's part of stage st: the DtN at the stage's surface and the
// base right-hand side with the tableau's update of column 0
int seg_base(Ctx *c, Seg *g, int st, const double *cvec) {
    select_parity(c, 0);
    const size_t N = (size_t)c->N, ks = (size_t)c->NC * 2 * N;
    WW_TRY(seg_geometry(c, g));
    WW_TRY(seg_assemble(c, g));
    WW_TRY(seg_factor(c, false, st));
    WW_TRY(launch_phi0(c));
    WW_TRY(seg_solve(c, c->M, 1));
    WW_TRY(launch_gamma(c, 0, 1));
    WW_TRY(seg_apply_G(c, 0, 1));
    k_base_rhs_mesh<<<1, SEG_THREADS, sizeof(double2) * N, c->stream>>>(
        c->Gout, c->eta, c->eta_x, c->phi_s, c->curv, g->einv, g->pw, c->g, c->tau, c->N, c->logN, c->tw,
        c->filt_d, c->ux, c->vy, c->w3, c->uxd, c->vyd, c->w3d, c->Fbase, c->Y, c->Ys, g->K, ks, st, g->S, g->d_a,
        g->d_b, cvec, g->theta, g->steps, c->status);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

int seg_stage(Ctx *c, Seg *g, int st, const double *cvec) {
    const size_t N = (size_t)c->N, ks = (size_t)c->NC * 2 * N;
    WW_TRY(seg_base(c, g, st, cvec));
    if (c->nc <= 0) return WW_OK;
    WW_TRY(launch_psi(c));
    WW_TRY(seg_solve(c, c->M + N, c->nc));
    WW_TRY(launch_gamma(c, 1, c->nc, true));
    WW_TRY(seg_apply_G(c, 1, c->nc));
    // The variational transforms of a segment run in FP64 in both forms: on the
    // mesh the double-float transforms' rounding, amplified in the small T
    // column, reached ten times the oracle's own rounding sensitivity.
    k_col_rhs_mesh<ArF64><<<c->nc, SEG_THREADS, fft_smem_bytes<ArF64>(c->N, 2), c->stream>>>(
        c->Gout, c->ux, c->vy, c->w3, g->einv, g->einv, c->vy, g->pw, c->Fbase, c->g, c->tau, c->N, c->logN, c->tw,
        c->filt_d, c->Y, c->Ys, g->K, ks, st, g->S, g->d_a, g->d_b, cvec, g->theta, g->steps, c->status);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

// forward stage of the gradient: the base part, then its record
int seg_fwd_stage(Ctx *c, Seg *g, int st, const double *cvec) {
    WW_TRY(seg_base(c, g, st, cvec));
    k_seg_record<<<1, SEG_THREADS, 0, c->stream>>>(c->eta, c->ux, c->vy, c->w3, c->Fbase, c->N, st, g->S, g->steps,
                                                   g->rec, g->rstep);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

// the DtN setup of the transposed operator at the recorded surface of stage
// `off` of the current step (off = -1: the last stage of the step before)
int seg_adj_setup(Ctx *c, Seg *g, int off, bool fresh) {
    select_parity(c, 0);
    k_seg_adj_fetch<<<(c->N + 255) / 256, 256, 0, c->stream>>>(g->rec, g->rstep, off, g->S, g->steps, c->N, g->aeta);
    WW_CUDA_TRY(cudaGetLastError());
    WW_TRY(seg_geometry(c, g, g->aeta, g->aeta, false));
    WW_TRY(seg_assemble(c, g));   // A^T, G^T (c->trans is set)
    return seg_factor(c, fresh, off < 0 ? 0 : off);
}

// one transposed step of the tableau: Filt, then stages S-1..0
int seg_adj_step(Ctx *c, Seg *g, const double *cvec) {
    const int N = c->N;
    const size_t one = sizeof(double2) * (size_t)N;
    k_seg_adj_begin<<<1, SEG_THREADS, one, c->stream>>>(g->lam, g->kb, N, c->logN, c->tw, c->filt_d, g->d_b, g->S,
                                                        cvec, g->theta, g->steps, g->rstep);
    WW_CUDA_TRY(cudaGetLastError());
    for (int st = g->S - 1; st >= 0; --st) {
        WW_TRY(seg_adj_setup(c, g, st, false));
        k_seg_adj_local<<<1, SEG_THREADS, 2 * one, c->stream>>>(
            g->kb + (size_t)st * 2 * N, g->rec, g->rstep, st, g->S, g->steps, N, c->logN, c->tw, c->filt_d, g->e,
            g->einv, c->g, c->tau, cvec, g->chi, g->etal, g->psil, g->gT);
        WW_CUDA_TRY(cudaGetLastError());
        WW_TRY(gemv_narrow(c->stream, N, 1, N, 1.0, c->G, N, g->chi, N, 0.0, g->y, N));   // G^T chis
        k_seg_adj_dtn<<<1, SEG_THREADS, one, c->stream>>>(g->chi, g->y, N, c->logN, c->tw, c->M);
        WW_CUDA_TRY(cudaGetLastError());
        WW_TRY(seg_solve(c, c->M, 1));   // A^{-T} D (1/2 H - G^T) diag(1/xi') chi
        k_seg_adj_update<<<(N + 255) / 256, 256, 0, c->stream>>>(c->M, g->psil, g->etal, g->rec, g->rstep, st, g->S,
                                                                 g->steps, N, g->d_a, g->theta, cvec, g->lam, g->kb);
        WW_CUDA_TRY(cudaGetLastError());
    }
    return WW_OK;
}

int seg_prepare(Ctx *c) {
    const size_t N = (size_t)c->N;
    const size_t two = 2 * sizeof(double2) * N;
    WW_TRY(raise_smem(reinterpret_cast<const void *>(k_geom_mesh), two));
    WW_TRY(raise_smem(reinterpret_cast<const void *>(k_base_rhs_mesh), two / 2));
    WW_TRY(raise_smem(reinterpret_cast<const void *>(k_col_rhs_mesh<ArF64>), fft_smem_bytes<ArF64>(c->N, 2)));
    WW_TRY(raise_smem(reinterpret_cast<const void *>(k_seg_adj_begin), two / 2));
    WW_TRY(raise_smem(reinterpret_cast<const void *>(k_seg_adj_local), two));
    WW_TRY(raise_smem(reinterpret_cast<const void *>(k_seg_adj_dtn), two / 2));
    return WW_OK;
}

int count_kernels(cudaGraph_t gr, int *out) {
    size_t nn = 0;
    WW_CUDA_TRY(cudaGraphGetNodes(gr, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    WW_CUDA_TRY(cudaGraphGetNodes(gr, nodes.data(), &nn));
    int k = 0;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        WW_CUDA_TRY(cudaGraphNodeGetType(nd, &t));
        if (t == cudaGraphNodeTypeKernel) ++k;
    }
    *out = k;
    return WW_OK;
}

// capture body() on the context's stream into a graph, once
template <class F>
int seg_capture(Ctx *c, cudaGraph_t *graph, cudaGraphExec_t *exec, int *nkern, F body) {
    if (*exec) return WW_OK;
    WW_CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    const int st = body();
    cudaGraph_t gr = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &gr);
    if (st != WW_OK) {
        if (gr) cudaGraphDestroy(gr);
        return st;
    }
    if (e != cudaSuccess) return fail(WW_ERR_CUDA, std::string("segment capture: ") + cudaGetErrorString(e));
    WW_TRY(count_kernels(gr, nkern));
    const cudaError_t ei = cudaGraphInstantiate(exec, gr, 0);
    *graph = gr;
    if (ei != cudaSuccess) return fail(WW_ERR_CUDA, std::string("segment instantiate: ") + cudaGetErrorString(ei));
    return WW_OK;
}

// the segment's step (all S stages) as a graph, captured on first use
int seg_step_graph(Ctx *c, Seg *g, const double *cvec) {
    return seg_capture(c, &g->graph, &g->exec, &g->nkern, [&] {
        int st = WW_OK;
        for (int k = 0; k < g->S && st == WW_OK; ++k) st = seg_stage(c, g, k, cvec);
        return st;
    });
}

// the gradient's step programs: forward (base only, recorded) and transposed
int seg_fwd_graph(Ctx *c, Seg *g, const double *cvec) {
    return seg_capture(c, &g->fgraph, &g->fexec, &g->fkern, [&] {
        int st = WW_OK;
        for (int k = 0; k < g->S && st == WW_OK; ++k) st = seg_fwd_stage(c, g, k, cvec);
        return st;
    });
}

int seg_bwd_graph(Ctx *c, Seg *g, const double *cvec) {
    return seg_capture(c, &g->bgraph, &g->bexec, &g->bkern, [&] { return seg_adj_step(c, g, cvec); });
}

// the gradient's workspace of a segment (first call)
int seg_grad_alloc(Ctx *c, Seg *g) {
    const size_t N = (size_t)c->N, before = g->bytes;
    int st = WW_OK;
#define GA(p, n) \
    if (st == WW_OK && !(p)) st = seg_alloc(c, g, &(p), (n))
    GA(g->rec, (size_t)g->steps * g->S * SEG_REC * N);
    GA(g->kb, (size_t)g->S * 2 * N);
    GA(g->lam, 2 * N);
    GA(g->chi, N);
    GA(g->etal, N);
    GA(g->psil, N);
    GA(g->y, N);
    GA(g->aeta, N);
    GA(g->gT, 1);
    GA(g->rstep, 1);
#undef GA
    g->gbytes += g->bytes - before;
    return st;
}

// the interpolation matrix from the previous segment's grid into this one's
int seg_respace_matrix(Ctx *cb, Seg *gb, int Ma, double rho_a, int centre_a) {
    if (gb->R && gb->R_M == Ma && gb->R_rho == rho_a && gb->R_centre == centre_a) return WW_OK;
    if (gb->R && gb->R_M != Ma) return fail(WW_ERR_ARG, "shoot_jacobian_segments: a context follows segments of "
                                                        "different sizes in different calls");
    const int Mb = cb->N;
    if (!gb->R) {
        WW_TRY(seg_alloc(cb, gb, &gb->R, (size_t)Mb * Ma));
        WW_TRY(seg_alloc(cb, gb, &gb->beta, (size_t)Mb));
    }
    std::vector<double> beta(Mb);
    const double two_pi = 6.283185307179586476925286766559;
    for (int j = 0; j < Mb; ++j) {
        double x, E, E1;
        mesh_at(gb->rho, gb->centre, two_pi * j / Mb, &x, &E, &E1);
        beta[j] = rho_a == 1.0 ? x : mesh_inv(rho_a, centre_a, x);
    }
    WW_CUDA_TRY(cudaMemcpyAsync(gb->beta, beta.data(), sizeof(double) * Mb, cudaMemcpyHostToDevice, cb->stream));
    dim3 grid((Mb + 255) / 256, Ma);
    k_respace_matrix<<<grid, 256, 0, cb->stream>>>(gb->beta, Mb, Ma, gb->R);
    WW_CUDA_TRY(cudaGetLastError());
    WW_CUDA_TRY(cudaStreamSynchronize(cb->stream));   // beta's host buffer
    gb->R_M = Ma;
    gb->R_rho = rho_a;
    gb->R_centre = centre_a;
    return WW_OK;
}

}  // namespace

void segment_destroy(Ctx *c) {
    if (!c->seg) return;
    free_seg(c, c->seg);
    c->seg = nullptr;
}

}  // namespace ww

using namespace ww;

extern "C" int ww_set_segment(ww_ctx *ctx, const ww_segment *sg) {
    if (!ctx) return fail(WW_ERR_ARG, "ww_set_segment: NULL context");
    Ctx *c = ctx_of(ctx);
    WW_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (!sg) {
        segment_destroy(c);
        return WW_OK;
    }
    if (sg->steps < 1 || !(sg->theta > 0.0 && sg->theta <= 1.0) || !(sg->rho > 0.0 && sg->rho <= 1.0) ||
        (sg->centre != 0 && sg->centre != 1))
        return fail(WW_ERR_ARG, "ww_set_segment: steps >= 1, 0 < theta <= 1, 0 < rho <= 1, centre 0 or 1");
    if (sg->stages < 1 || sg->stages > SEG_MAX_STAGES || !sg->a || !sg->b)
        return fail(WW_ERR_ARG, "ww_set_segment: a tableau of 1.." + std::to_string(SEG_MAX_STAGES) + " stages");
    if (c->N % 32 != 0) return fail(WW_ERR_ARG, "ww_set_segment: N must be a multiple of 32");
    const int S = sg->stages;
    for (int i = 0; i < S; ++i)
        for (int j = i; j < S; ++j)
            if (sg->a[(size_t)i * S + j] != 0.0)
                return fail(WW_ERR_ARG, "ww_set_segment: the tableau must be explicit (a strictly lower triangular)");
    WW_TRY(seg_prepare(c));
    segment_destroy(c);
    Seg *g = new Seg();
    g->steps = sg->steps;
    g->S = S;
    g->centre = sg->centre;
    g->theta = sg->theta;
    g->rho = sg->rho;
    g->a.assign(sg->a, sg->a + (size_t)S * S);
    g->b.assign(sg->b, sg->b + S);
    const size_t N = (size_t)c->N;
    int st = WW_OK;
#define SA(p, n) \
    if (st == WW_OK) st = seg_alloc(c, g, &(p), (n))
    SA(g->d_a, (size_t)S * S);
    SA(g->d_b, (size_t)S);
    SA(g->xi, N);
    SA(g->e, N);
    SA(g->e1, N);
    SA(g->cxi, N);
    SA(g->sxi, N);
    SA(g->einv, N);
    SA(g->pw, N);
    SA(g->wts, N);
    SA(g->K, (size_t)S * c->NC * 2 * N);
#undef SA
    if (st != WW_OK) {
        free_seg(c, g);
        return st;
    }
    // the mesh of Eq. (xi) at alpha_j (xi = alpha when rho = 1)
    std::vector<double> x(N), e(N), e1(N), cx(N), sx(N), ei(N), pw(N), wts(N);
    const double two_pi = 6.283185307179586476925286766559;
    for (size_t j = 0; j < N; ++j) {
        const double al = two_pi * (double)j / (double)N;
        if (g->rho == 1.0) {
            x[j] = al;
            e[j] = 1.0;
            e1[j] = 0.0;
        } else {
            mesh_at(g->rho, g->centre, al, &x[j], &e[j], &e1[j]);
        }
        cx[j] = std::cos(x[j]);
        sx[j] = std::sin(x[j]);
        ei[j] = 1.0 / e[j];
        pw[j] = e[j] / (double)N;
        wts[j] = std::sqrt(e[j] / (double)N);
    }
    cudaError_t ce = cudaMemcpy(g->d_a, g->a.data(), sizeof(double) * S * S, cudaMemcpyHostToDevice);
    const std::pair<double *, const std::vector<double> *> tabs[] = {{g->d_b, &g->b}, {g->xi, &x},  {g->e, &e},
                                                                     {g->e1, &e1},    {g->cxi, &cx}, {g->sxi, &sx},
                                                                     {g->einv, &ei},  {g->pw, &pw}, {g->wts, &wts}};
    for (const auto &t : tabs)
        if (ce == cudaSuccess)
            ce = cudaMemcpy(t.first, t.second->data(), sizeof(double) * t.second->size(), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        free_seg(c, g);
        return fail(WW_ERR_CUDA, std::string("ww_set_segment upload: ") + cudaGetErrorString(ce));
    }
    c->seg = g;
    return WW_OK;
}

namespace {

// the contexts of a segmented call, checked: one per segment, each set up by
// ww_set_segment, sharing n, g, tau, h and the form; the first uniform; the
// thetas summing to 1
int segment_contexts(ww_ctx *const *ctx, int nseg, const char *who, std::vector<Ctx *> &cs) {
    const std::string w(who);
    cs.assign(nseg, nullptr);
    double th = 0.0;
    for (int l = 0; l < nseg; ++l) {
        if (!ctx[l]) return fail(WW_ERR_ARG, w + ": NULL context");
        cs[l] = ctx_of(ctx[l]);
        Ctx *c = cs[l];
        if (!c->seg) return fail(WW_ERR_ARG, w + ": segment " + std::to_string(l) + " has no ww_set_segment");
        if (c->stream == nullptr) return fail(WW_ERR_ARG, w + ": the legacy default stream runs no step graphs");
        const Ctx *c0 = cs[0];
        if (c->n != c0->n || c->g != c0->g || c->tau != c0->tau || c->deep != c0->deep ||
            (!c->deep && c->h != c0->h) || c->precision != c0->precision)
            return fail(WW_ERR_ARG, w + ": the segments' contexts differ in n, g, tau, h or form");
        for (int k = 0; k < l; ++k)
            if (cs[k] == c) return fail(WW_ERR_ARG, w + ": a context may serve one segment");
        th += c->seg->theta;
    }
    if (cs[0]->seg->rho != 1.0) return fail(WW_ERR_ARG, w + ": the first segment is uniform (rho = 1)");
    if (std::fabs(th - 1.0) > 1e-12) return fail(WW_ERR_ARG, w + ": the thetas must sum to 1");
    return WW_OK;
}

// every segment's work runs on the first context's stream; the contexts'
// own streams and flags come back on return
struct SegCall {
    std::vector<Ctx *> &cs;
    std::vector<cudaStream_t> saved;
    explicit SegCall(std::vector<Ctx *> &v) : cs(v), saved(v.size()) {
        for (size_t l = 0; l < cs.size(); ++l) {
            saved[l] = cs[l]->stream;
            cs[l]->stream = cs[0]->stream;
        }
    }
    ~SegCall() {
        for (size_t l = 0; l < cs.size(); ++l) {
            cs[l]->stream = saved[l];
            cs[l]->trans = 0;
            cs[l]->one_col = false;
        }
    }
};

}  // namespace

extern "C" int shoot_jacobian_segments(ww_ctx *const *ctx, int nseg, const double *cvec, double *r, double *J,
                                       double *f) {
    if (nseg < 1 || !ctx || !cvec || !r || !J || !f) return fail(WW_ERR_ARG, "shoot_jacobian_segments: bad argument");
    std::vector<Ctx *> cs;
    WW_TRY(segment_contexts(ctx, nseg, "shoot_jacobian_segments", cs));
    cudaStream_t s0 = cs[0]->stream;
    SegCall call(cs);
    long long launches = 0;
    for (int l = 0; l < nseg; ++l) {
        Ctx *c = cs[l];
        Seg *g = c->seg;
        c->one_col = false;
        WW_CUDA_TRY(cudaMemsetAsync(c->status, 0, sizeof(int), s0));
        // T (= c[0]) where the captured stage program reads it: the context's scratch
        WW_CUDA_TRY(cudaMemcpyAsync(c->small, cvec, sizeof(double), cudaMemcpyDeviceToDevice, s0));
        if (l == 0) {
            WW_TRY(launch_initial(c, cvec, 1));
            launches += 1;
        } else {
            Ctx *ca = cs[l - 1];
            WW_TRY(seg_respace_matrix(c, g, ca->N, ca->seg->rho, ca->seg->centre));
            WW_TRY(dgemm(s0, c->N, 2 * c->NC, ca->N, 1.0, g->R, c->N, ca->Y, ca->N, 0.0, c->Y, c->N));
            WW_CUDA_TRY(cudaMemcpyAsync(c->Ys, c->Y, sizeof(double) * 2 * c->NC * c->N, cudaMemcpyDeviceToDevice, s0));
            launches += 1;
        }
        if (c->precision == WW_MIXED) {   // a fresh approximate inverse at the segment's first surface
            select_parity(c, 0);
            WW_TRY(seg_geometry(c, g));
            WW_TRY(seg_assemble(c, g));
            WW_TRY(seg_factor(c, true));
        }
        WW_TRY(seg_step_graph(c, g, c->small));
        for (int s = 0; s < g->steps; ++s) WW_CUDA_TRY(cudaGraphLaunch(g->exec, s0));
        launches += (long long)g->steps * g->nkern;
        c->dtn_ready = false;
    }
    Ctx *cl = cs[nseg - 1];
    k_outputs_mesh_r<<<1, 1024, 0, s0>>>(cl->Y, cl->seg->wts, cl->N, r, f);
    dim3 grid((cl->N + 255) / 256, cl->nc);
    k_outputs_mesh_J<<<grid, 256, 0, s0>>>(cl->Y, cl->seg->wts, cl->N, cl->nc, J);
    WW_CUDA_TRY(cudaGetLastError());
    launches += 2;
    for (int l = 0; l < nseg; ++l) {
        const int st = read_status(cs[l]);
        if (st != WW_OK) return fail(st, "segment " + std::to_string(l) + ": " + ww_last_error());
        cs[l]->stats.stages = cs[l]->seg->S * cs[l]->seg->steps;
        cs[l]->stats.device_bytes = (long long)cs[l]->dev_bytes;
    }
    cs[0]->stats.launches = launches;
    return WW_OK;
}

extern "C" int objective_and_grad_segments(ww_ctx *const *ctx, int nseg, const double *cvec, double *f,
                                           double *grad) {
    if (nseg < 1 || !ctx || !cvec || !f || !grad)
        return fail(WW_ERR_ARG, "objective_and_grad_segments: bad argument");
    std::vector<Ctx *> cs;
    WW_TRY(segment_contexts(ctx, nseg, "objective_and_grad_segments", cs));
    for (Ctx *c : cs) WW_TRY(seg_grad_alloc(c, c->seg));
    cudaStream_t s0 = cs[0]->stream;
    SegCall call(cs);
    long long launches = 0;
    // forward: the base state through the segments, every stage recorded
    for (int l = 0; l < nseg; ++l) {
        Ctx *c = cs[l];
        Seg *g = c->seg;
        c->one_col = true;
        c->trans = 0;
        WW_CUDA_TRY(cudaMemsetAsync(c->status, 0, sizeof(int), s0));
        WW_CUDA_TRY(cudaMemcpyAsync(c->small, cvec, sizeof(double), cudaMemcpyDeviceToDevice, s0));
        if (l == 0) {
            WW_TRY(launch_initial(c, cvec, 0));
        } else {
            Ctx *ca = cs[l - 1];
            WW_TRY(seg_respace_matrix(c, g, ca->N, ca->seg->rho, ca->seg->centre));
            WW_TRY(dgemm(s0, c->N, 2, ca->N, 1.0, g->R, c->N, ca->Y, ca->N, 0.0, c->Y, c->N));
            WW_CUDA_TRY(cudaMemcpyAsync(c->Ys, c->Y, sizeof(double) * 2 * c->N, cudaMemcpyDeviceToDevice, s0));
        }
        launches += 1;
        if (c->precision == WW_MIXED) {
            select_parity(c, 0);
            WW_TRY(seg_geometry(c, g));
            WW_TRY(seg_assemble(c, g));
            WW_TRY(seg_factor(c, true));
        }
        WW_CUDA_TRY(cudaMemsetAsync(g->rstep, 0, sizeof(int), s0));
        WW_TRY(seg_fwd_graph(c, g, c->small));
        for (int s = 0; s < g->steps; ++s) WW_CUDA_TRY(cudaGraphLaunch(g->fexec, s0));
        launches += (long long)g->steps * g->fkern;
    }
    Ctx *cl = cs[nseg - 1];
    k_seg_adj_init<<<1, 1024, 0, s0>>>(cl->Y, cl->seg->wts, cl->N, cl->seg->lam, f);
    WW_CUDA_TRY(cudaGetLastError());
    WW_CUDA_TRY(cudaMemsetAsync(grad, 0, sizeof(double), s0));
    launches += 1;
    // backward: segment by segment from the last
    for (int l = nseg - 1; l >= 0; --l) {
        Ctx *c = cs[l];
        Seg *g = c->seg;
        c->trans = 1;
        WW_CUDA_TRY(cudaMemsetAsync(g->gT, 0, sizeof(double), s0));
        if (c->precision == WW_MIXED) {   // a fresh inverse of A^T at the segment's last stage
            WW_TRY(seg_adj_setup(c, g, -1, true));
        }
        WW_TRY(seg_bwd_graph(c, g, c->small));
        for (int s = 0; s < g->steps; ++s) WW_CUDA_TRY(cudaGraphLaunch(g->bexec, s0));
        launches += (long long)g->steps * g->bkern;
        c->trans = 0;
        k_seg_add<<<1, 1, 0, s0>>>(grad, g->gT);
        if (l > 0) {
            Ctx *ca = cs[l - 1];
            k_seg_respace_T<<<ca->N, 256, 0, s0>>>(g->R, c->N, ca->N, g->lam, ca->seg->lam);
            launches += 1;
        }
        WW_CUDA_TRY(cudaGetLastError());
        launches += 1;
        c->dtn_ready = false;
    }
    Ctx *c0 = cs[0];
    if (c0->n > 0) {
        k_seg_grad<<<c0->n, 256, 0, s0>>>(c0->basis, c0->seg->lam, c0->N, grad);
        WW_CUDA_TRY(cudaGetLastError());
        launches += 1;
    }
    for (int l = 0; l < nseg; ++l) {
        const int st = read_status(cs[l]);
        if (st != WW_OK) return fail(st, "segment " + std::to_string(l) + ": " + ww_last_error());
        cs[l]->stats.stages = 2 * cs[l]->seg->S * cs[l]->seg->steps;
        cs[l]->stats.device_bytes = (long long)cs[l]->dev_bytes;
        cs[l]->stats.adjoint_bytes = (long long)cs[l]->seg->gbytes;
    }
    cs[0]->stats.launches = launches;
    return WW_OK;
}
