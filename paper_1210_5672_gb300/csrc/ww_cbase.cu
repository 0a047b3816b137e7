// ww_cbase.cu -- the base state's spectral kernels (geometry, gamma of the
// base column, base right-hand side with its RK update) on a thread-block
// cluster of CS CTAs (the four-step FFT of ww_cfft.cuh).  These transforms are
// on the critical path of every RK stage and run on one column, so one CTA
// would leave them bound by a single SM's FP64 pipe (2 lanes per clock):
// ~25 us per N = 2048 transform.
#include "ww_cfft.cuh"

namespace ww {

namespace {

// ---------------------------------------------------------------- geometry
template <int CS>
__global__ void __launch_bounds__(CB_THREADS) k_cgeometry(const double *__restrict__ eta_in,
                                                          const double *__restrict__ phi_in, int with_phi, int N,
                                                          int logN, int deep, int with_curv,
                                                          const double2 *__restrict__ tw, double *eta, double *eta_x,
                                                          double *eta_xx, double *phi_s, double *curv, double *E,
                                                          double *Einv, int *status) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cg::cluster_group cl = cg::this_cluster();
    const int L = N / CS, r = (int)cl.block_rank();
    double2 *xs = reinterpret_cast<double2 *>(smraw), *sp = xs + L, *sp2 = sp + L, *zs = sp2 + L;
    int bad = 0;
    for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) {
        const int n = r + CS * n2;
        const double e = eta_in[n];
        const double p = with_phi ? phi_in[n] : 0.0;
        if (!isfinite(e) || !isfinite(p) || (!deep && e <= 0.0)) bad = 1;
        eta[n] = e;
        const double ee = exp(e);
        E[n] = ee;
        Einv[n] = 1.0 / ee;
        xs[n2] = make_double2(e, p);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, ST_GEOMETRY);
    cfft_forward<CS>(cl, xs, sp, N, logN, tw);
    const double invN = 1.0 / N;
    for (int t = threadIdx.x; t < L; t += blockDim.x) {
        const int j = slot_of(t, N, CS, r), k = wavenum(j, N);
        const bool nyq = j == (N >> 1);
        const double2 z = sp[t];
        const double2 v = make_double2(-(double)k * z.y * invN, (double)k * z.x * invN);   // (ik) z / N
        sp[t] = nyq ? make_double2(0.0, 0.0) : v;
        sp2[t] = nyq ? make_double2(0.0, 0.0) : make_double2(-(double)k * v.y, (double)k * v.x);
    }
    cfft_inverse<CS>(cl, sp, zs, xs, N, logN, tw);   // eta' + i phi'
    for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) {
        const int n = r + CS * n2;
        eta_x[n] = xs[n2].x;
        phi_s[n] = xs[n2].y;
    }
    cfft_inverse<CS>(cl, sp2, zs, xs + 0, N, logN, tw);   // eta'' + i phi''
    for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) eta_xx[r + CS * n2] = xs[n2].x;
    __syncthreads();
    if (!with_curv) {
        for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) curv[r + CS * n2] = 0.0;   // multiplied by tau = 0
        cl.sync();
        return;
    }
    for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) {
        const double ex = eta_x[r + CS * n2];
        xs[n2] = make_double2(ex / sqrt(1.0 + ex * ex), 0.0);
    }
    cfft_forward<CS>(cl, xs, sp, N, logN, tw);
    for (int t = threadIdx.x; t < L; t += blockDim.x) {
        const int j = slot_of(t, N, CS, r), k = wavenum(j, N);
        const double2 z = sp[t];
        sp[t] = j == (N >> 1) ? make_double2(0.0, 0.0) : make_double2(-(double)k * z.y * invN, (double)k * z.x * invN);
    }
    cfft_inverse<CS>(cl, sp, zs, xs, N, logN, tw);
    for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) curv[r + CS * n2] = xs[n2].x;
    cl.sync();
}

// ---------------------------------------------------------------- gamma of the base column
// one real column mu: gamma = mu' and 1/2 H gamma = |k|/2 mu^ come back as the
// real and imaginary parts of one inverse transform of (ik + i|k|/2) mu^
template <int CS>
__global__ void __launch_bounds__(CB_THREADS) k_cgamma(const double *__restrict__ mu, int N, int logN,
                                                       const double2 *__restrict__ tw, double *Gam, double *Gout) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cg::cluster_group cl = cg::this_cluster();
    const int L = N / CS, r = (int)cl.block_rank();
    double2 *xs = reinterpret_cast<double2 *>(smraw), *sp = xs + L, *zs = sp + L;
    for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) xs[n2] = make_double2(mu[r + CS * n2], 0.0);
    cfft_forward<CS>(cl, xs, sp, N, logN, tw);
    const double invN = 1.0 / N;
    for (int t = threadIdx.x; t < L; t += blockDim.x) {
        const int j = slot_of(t, N, CS, r), k = wavenum(j, N);
        const double2 z = sp[t];
        // (ik + i |k|/2) z / N
        const double f = ((double)k + 0.5 * fabs((double)k)) * invN;
        sp[t] = j == (N >> 1) ? make_double2(0.0, 0.0) : make_double2(-f * z.y, f * z.x);
    }
    cfft_inverse<CS>(cl, sp, zs, xs, N, logN, tw);
    for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) {
        const int n = r + CS * n2;
        Gam[n] = xs[n2].x;
        Gout[n] = xs[n2].y;
    }
    cl.sync();
}

// ---------------------------------------------------------------- base RHS + RK update
__device__ __forceinline__ double rk_b2(int st) { return (st == 1 || st == 2) ? 2.0 : 1.0; }
__device__ __forceinline__ double rk_a_next2(int st) { return st == 2 ? 1.0 : 0.5; }

template <int CS>
__global__ void __launch_bounds__(CB_THREADS) k_cbase_rhs(
    const double *__restrict__ Gphi, const double *__restrict__ eta, const double *__restrict__ eta_x,
    const double *__restrict__ phi_s, const double *__restrict__ curv, double g, double tau, int N, int logN,
    const double2 *__restrict__ tw, const double *__restrict__ filt, double *ux, double *vy, double *w3, float2 *uxd,
    float2 *vyd, float2 *w3d, double *Fbase, double *Y, double *Ys, double *Acc, int st,
    const double *__restrict__ cvec, int steps, int update, int *status) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cg::cluster_group cl = cg::this_cluster();
    const int L = N / CS, r = (int)cl.block_rank();
    double2 *xs = reinterpret_cast<double2 *>(smraw), *sp = xs + L, *zs = sp + L;
    int bad = 0;
    for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) {
        const int n = r + CS * n2;
        const double ex = eta_x[n], d = 1.0 + ex * ex, gp = Gphi[n], pp = phi_s[n];
        const double u = (pp - ex * gp) / d;
        const double v = (ex * pp + gp) / d;
        const double w = 1.0 / (d * sqrt(d));
        ux[n] = u;
        vy[n] = v;
        w3[n] = w;
        if (uxd) {
            uxd[n] = df_split(u);
            vyd[n] = df_split(v);
            w3d[n] = df_split(w);
        }
        const double pt = v * gp - 0.5 * u * u - 0.5 * v * v - g * eta[n] + tau * curv[n];
        if (!isfinite(pt) || !isfinite(gp)) bad = 1;
        xs[n2] = make_double2(gp, pt);   // eta_t = G phi ; phi_t before P and the filter
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, ST_NONFINITE);
    cfft_forward<CS>(cl, xs, sp, N, logN, tw);
    for (int t = threadIdx.x; t < L; t += blockDim.x) {
        const int j = slot_of(t, N, CS, r);
        const double f = filt[j];
        // P acts on the phi part only: at k = 0 keep Re (eta mean), drop Im (phi mean)
        sp[t] = j == 0 ? make_double2(sp[t].x * f, 0.0) : cscale(sp[t], f);
    }
    cfft_inverse<CS>(cl, sp, zs, xs, N, logN, tw);
    for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) {
        const int n = r + CS * n2;
        Fbase[n] = xs[n2].x;
        Fbase[N + n] = xs[n2].y;
    }
    if (update) {
        const double dt = cvec[0] / (4.0 * steps);
        if (st < 3) {
            const double b = rk_b2(st), a = rk_a_next2(st);
            for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) {
                const int n = r + CS * n2;
                const double2 k = xs[n2];
                if (st == 0) {
                    Acc[n] = b * k.x;
                    Acc[N + n] = b * k.y;
                } else {
                    Acc[n] += b * k.x;
                    Acc[N + n] += b * k.y;
                }
                Ys[n] = Y[n] + a * dt * k.x;
                Ys[N + n] = Y[N + n] + a * dt * k.y;
            }
        } else {
            // end of the step: Y + dt/6 (Acc + k), filtered
            for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) {
                const int n = r + CS * n2;
                const double2 k = xs[n2];
                xs[n2] = make_double2(Y[n] + dt / 6.0 * (Acc[n] + k.x), Y[N + n] + dt / 6.0 * (Acc[N + n] + k.y));
            }
            cfft_forward<CS>(cl, xs, sp, N, logN, tw);
            for (int t = threadIdx.x; t < L; t += blockDim.x) sp[t] = cscale(sp[t], filt[slot_of(t, N, CS, r)]);
            cfft_inverse<CS>(cl, sp, zs, xs, N, logN, tw);
            for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) {
                const int n = r + CS * n2;
                Y[n] = Ys[n] = xs[n2].x;
                Y[N + n] = Ys[N + n] = xs[n2].y;
            }
        }
    }
    cl.sync();
}

}  // namespace

// The cluster kernels need L = N / CS >= 64 (N >= 512 with CS = 8); smaller
// problems keep the one-CTA kernels.
bool cbase_ok(const Ctx *c) { return c->N >= 8 * 64 && c->N <= 8 * 2048; }

int launch_cbase_geometry(Ctx *c, const double *eta, const double *phi, int with_phi) {
    const size_t sm = 4 * sizeof(double2) * (size_t)(c->N / CB_CS);
    return launch_cluster(k_cgeometry<CB_CS>, CB_CS, sm, c->stream, eta, phi, with_phi, c->N, c->logN,
                          c->deep ? 1 : 0, c->tau != 0.0 ? 1 : 0, (const double2 *)c->tw, c->eta, c->eta_x,
                          c->eta_xx, c->phi_s, c->curv, c->E, c->Einv, c->status);
}

int launch_cbase_gamma(Ctx *c) {
    const size_t sm = 3 * sizeof(double2) * (size_t)(c->N / CB_CS);
    return launch_cluster(k_cgamma<CB_CS>, CB_CS, sm, c->stream, (const double *)c->M, c->N, c->logN,
                          (const double2 *)c->tw, c->Gam, c->Gout);
}

int launch_cbase_rhs(Ctx *c, int stage, const double *cvec) {
    const size_t sm = 3 * sizeof(double2) * (size_t)(c->N / CB_CS);
    return launch_cluster(k_cbase_rhs<CB_CS>, CB_CS, sm, c->stream, (const double *)c->Gout, (const double *)c->eta,
                          (const double *)c->eta_x, (const double *)c->phi_s, (const double *)c->curv, c->g, c->tau,
                          c->N, c->logN, (const double2 *)c->tw, (const double *)c->filt_d, c->ux, c->vy, c->w3,
                          c->uxd, c->vyd, c->w3d, c->Fbase, c->Y, c->Ys, c->Kacc, stage < 0 ? 0 : stage, cvec,
                          c->steps, stage >= 0 ? 1 : 0, c->status);
}

}  // namespace ww
