// ww_adjoint.cu -- the gradient of f (Sec. 3.2, Eqs. (adj), (nabla:f); App. C,
// Eq. (adj2)) by the DISCRETE adjoint: the transpose of the RK4 scheme that
// advances the variational columns, so grad f = J^T r of the discrete map up
// to roundoff, from one backward sweep instead of n + 1 forward columns.
//
// Forward, the base trajectory runs once and each RK stage leaves a record
// [eta | phi_x | phi_y | w3 = (1+eta'^2)^{-3/2} | F] (F the filtered base
// right-hand side): 6N doubles a stage.  Either every stage's record stays
// resident (0.4 GB for 2048 steps at N = 1024), or, as the paper's
// mile-markers do (Sec. 3.2), the base state is checkpointed every K steps
// and each segment's records are recomputed from its checkpoint just before
// its backward sweep, so the records of only K steps are held at a time
// (K = sqrt(steps) gives memory ~ sqrt(steps) for one extra forward pass).
//
// Backward, step by step from lambda = (0, phi(T/4)/N) (the gradient of
// f = r.r/2, r = phi/sqrt(N), with respect to the final state): the
// transposed end-of-step filter, then the stages in reverse order.  With kb
// the adjoint of the stage's right-hand side,
//   et = Filt kb_eta,  pt = P Filt kb_phi,  chi = et + phi_y pt,
//   adjoint of phidot  pb = G^T chi + (phi_x pt)',
//   adjoint of etadot  eb = -phi_y pb + phi_x et' + phi_x phi_y pt' - g pt
//                           + tau (w3 pt')',
// (App. C's Eq. (adj2) term by term; phi_x phi_y pt' - phi_y (phi_x pt)'
// = -phi_y phi_x' pt), and the transposed discrete DtN
//   G^T chi = A^{-T} D (1/2 H chi - G^T chi)
// (D^T = -D, H^T = -H: antisymmetric Fourier multipliers with the Nyquist
// mode zeroed).  The continuous DtN map is self-adjoint (App. C); its
// discretisation is only nearly symmetric, and the exact transpose keeps the
// gradient equal to J^T r.  The stage's A and G are assembled TRANSPOSED and
// go through the same factorisation (LU, or the mixed form's approximate
// inverse and refinement) and the same one-column product as the forward
// operator.  Stage st then adds (eb, pb) to lambda and a_st dt (eb, pb) to
// the previous stage's kb; d f / d T gathers kb . F / T over all stages (the
// T column's forcing).
//
// The kernels address the record of the current stage through a device step
// counter, so a step of the sweep can be captured as a graph.  The spectral
// kernels run on an 8-CTA cluster (ww_cfft.cuh) for N >= 512 (one SM's FP64
// pipe would take ~17 us per N = 1024 transform), on one CTA below.
#include "ww_cfft.cuh"

namespace ww {

namespace {

constexpr int AJ_THREADS = 512;

__device__ __forceinline__ double rk_a(int st) { return st == 0 ? 0.0 : (st == 3 ? 1.0 : 0.5); }
__device__ __forceinline__ double rk_bw(int st) { return (st == 1 || st == 2) ? 2.0 : 1.0; }

__device__ __forceinline__ const double *stage_rec(const double *rec, const int *step, int st, int N) {
    return rec + ((size_t)(4 * *step + st)) * ADJ_REC * N;
}

// deterministic block sum (one value per thread in, the total to every thread out)
__device__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int nw = blockDim.x >> 5;
        double t = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) red[32] = t;
    }
    __syncthreads();
    const double t = red[32];
    __syncthreads();
    return t;
}

// Fourier multiplier at FFT slot j times `scale` (Nyquist zeroed): ik (kind 0)
// or -i sgn k (kind 1)
__device__ __forceinline__ double2 mult(double2 v, int j, int N, int kind, double scale) {
    const int k = wavenum(j, N);
    if (2 * j == N) return make_double2(0.0, 0.0);
    const double s = (kind == 0 ? (double)k : -(double)((k > 0) - (k < 0))) * scale;
    return make_double2(-s * v.y, s * v.x);   // (i s) v
}

__global__ void k_rec_eta(const double *__restrict__ Ys, int N, double *rec, const int *step, int st) {
    double *r = rec + ((size_t)(4 * *step + st)) * ADJ_REC * N;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) r[j] = Ys[j];
}

__global__ void k_rec_fields(const double *__restrict__ ux, const double *__restrict__ vy,
                             const double *__restrict__ w3, const double *__restrict__ F, int N, double *rec,
                             int *step, int st) {
    const int s = *step;
    double *r = rec + ((size_t)(4 * s + st)) * ADJ_REC * N;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        r[N + j] = ux[j];
        r[2 * N + j] = vy[j];
        r[3 * N + j] = w3[j];
        r[4 * N + j] = F[j];
        r[5 * N + j] = F[N + j];
    }
    __syncthreads();   // every thread has read the counter
    if (st == 3 && threadIdx.x == 0) *step = s + 1;
}

// lambda = (0, phi(T/4)/N), dT = 0.  The record counter is left as the forward
// pass left it: the number of steps whose records are held.
__global__ void k_adj_init(const double *__restrict__ Y, int N, double *lam, double *gT) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        lam[j] = 0.0;
        lam[N + j] = Y[N + j] / N;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *gT = 0.0;
}

__global__ void k_set_int(int *p, int v) { *p = v; }

// start of a backward step: step -= 1; lambda <- Filt lambda; kb_st = b_st dt/6 lambda
__global__ void __launch_bounds__(AJ_THREADS) k_adj_begin_step(double *lam, double *kb, int N, int logN,
                                                               const double2 *__restrict__ tw,
                                                               const double *__restrict__ filt,
                                                               const double *__restrict__ cvec, int steps, int *step) {
    extern __shared__ __align__(16) unsigned char smraw[];
    double2 *s = reinterpret_cast<double2 *>(smraw);
    for (int j = threadIdx.x; j < N; j += blockDim.x) s[j] = make_double2(lam[j], lam[N + j]);
    __syncthreads();
    block_fft(s, N, logN, tw, false);
    for (int j = threadIdx.x; j < N; j += blockDim.x) s[j] = cscale(s[j], filt[j]);
    __syncthreads();
    block_fft(s, N, logN, tw, true);
    const double dt = cvec[0] / (4.0 * steps);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double2 v = s[j];
        lam[j] = v.x;
        lam[N + j] = v.y;
        for (int st = 0; st < 4; ++st) {
            const double w = rk_bw(st) * dt / 6.0;
            kb[(size_t)st * 2 * N + j] = w * v.x;
            kb[(size_t)st * 2 * N + N + j] = w * v.y;
        }
    }
    __syncthreads();   // every thread has finished with the counter's old value (none read it)
    if (threadIdx.x == 0) *step = *step - 1;
}

// the surface of record 4 step + off (off = -1: the last stage of the step before);
// past the first record there is nothing to fetch and eta keeps its values
__global__ void k_adj_fetch(const double *__restrict__ rec, const int *step, int off, int N, double *eta) {
    const long idx = 4L * *step + off;
    if (idx < 0) return;
    const double *r = rec + (size_t)idx * ADJ_REC * N;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) eta[j] = r[j];
}

// the stage's local adjoint terms (one block, two complex arrays of N in shared memory):
// chi = et + phi_y pt, psil = (phi_x pt)', etal = phi_x et' + phi_x phi_y pt' - g pt
// + tau (w3 pt')', and dT += kb . F / T
__global__ void __launch_bounds__(AJ_THREADS) k_adj_local(const double *__restrict__ kb, const double *__restrict__ rec,
                                                          const int *step, int st, int N, int logN,
                                                          const double2 *__restrict__ tw,
                                                          const double *__restrict__ filt, double g, double tau,
                                                          const double *__restrict__ cvec, double *chi, double *etal,
                                                          double *psil, double *gT) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[33];
    double2 *s0 = reinterpret_cast<double2 *>(smraw);
    double2 *s1 = s0 + N;
    const double *r = stage_rec(rec, step, st, N);
    const double *ux = r + N, *vy = r + 2 * N, *w3 = r + 3 * N, *F = r + 4 * N;
    // d f / d T: the T column's forcing F/T entered this stage's right-hand side
    double fd = 0.0;
    for (int j = threadIdx.x; j < 2 * N; j += blockDim.x) fd = fma(kb[j], F[j], fd);
    fd = block_sum(fd, red);
    if (threadIdx.x == 0) *gT += fd / cvec[0];
    // (et, pt) = (Filt kb_eta, P Filt kb_phi) and their derivatives
    for (int j = threadIdx.x; j < N; j += blockDim.x) s0[j] = make_double2(kb[j], kb[N + j]);
    __syncthreads();
    block_fft(s0, N, logN, tw, false);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        double2 v = cscale(s0[j], filt[j]);
        if (j == 0) v.y = 0.0;   // P removes the mean of the phi part
        s0[j] = v;
        s1[j] = mult(v, j, N, 0, 1.0);   // v carries the 1/N of the filter table
    }
    __syncthreads();
    block_fft(s0, N, logN, tw, true);
    block_fft(s1, N, logN, tw, true);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double et = s0[j].x, pt = s0[j].y, det = s1[j].x, dpt = s1[j].y;
        const double u = ux[j], v = vy[j];
        chi[j] = fma(v, pt, et);
        etal[j] = u * det + u * v * dpt - g * pt;
        s0[j] = make_double2(u * pt, w3[j] * dpt);
    }
    __syncthreads();
    // ((phi_x pt)', (w3 pt')') in one transform
    block_fft(s0, N, logN, tw, false);
    for (int j = threadIdx.x; j < N; j += blockDim.x) s0[j] = mult(s0[j], j, N, 0, 1.0 / N);
    __syncthreads();
    block_fft(s0, N, logN, tw, true);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        psil[j] = s0[j].x;
        etal[j] += tau * s0[j].y;
    }
}

// M[:, 0] = D (1/2 H chi - y), y = G^T chi: the right-hand side of the transposed
// solve.  chi and y share one transform, Z = FFT(chi + i y).  A real multiplier
// m = e + o (e even, o odd in k) applied to Z gives, in the real part of the
// inverse, e acting on chi plus i o acting on y; with e = |k|/2 (the symbol of
// D H / 2) and o = -k (i o = -ik, the symbol of -D) that is the result.
__device__ __forceinline__ double dtn_t_symbol(int j, int N) {
    const int k = wavenum(j, N);
    return 2 * j == N ? 0.0 : (0.5 * fabs((double)k) - (double)k) / N;
}

__global__ void __launch_bounds__(AJ_THREADS) k_adj_dtn(const double *__restrict__ chi, const double *__restrict__ y,
                                                        int N, int logN, const double2 *__restrict__ tw, double *M) {
    extern __shared__ __align__(16) unsigned char smraw[];
    double2 *s = reinterpret_cast<double2 *>(smraw);
    for (int j = threadIdx.x; j < N; j += blockDim.x) s[j] = make_double2(chi[j], y[j]);
    __syncthreads();
    block_fft(s, N, logN, tw, false);
    for (int j = threadIdx.x; j < N; j += blockDim.x) s[j] = cscale(s[j], dtn_t_symbol(j, N));
    __syncthreads();
    block_fft(s, N, logN, tw, true);
    for (int j = threadIdx.x; j < N; j += blockDim.x) M[j] = s[j].x;
}

// ---------------------------------------------------------------- cluster forms (N >= 512)
template <int CS>
__global__ void __launch_bounds__(CB_THREADS) k_cadj_begin_step(double *lam, double *kb, int N, int logN,
                                                                const double2 *__restrict__ tw,
                                                                const double *__restrict__ filt,
                                                                const double *__restrict__ cvec, int steps,
                                                                int *step) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cg::cluster_group cl = cg::this_cluster();
    const int L = N / CS, r = (int)cl.block_rank();
    double2 *xs = reinterpret_cast<double2 *>(smraw), *sp = xs + L, *zs = sp + L;
    for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) {
        const int n = r + CS * n2;
        xs[n2] = make_double2(lam[n], lam[N + n]);
    }
    cfft_forward<CS>(cl, xs, sp, N, logN, tw);
    for (int t = threadIdx.x; t < L; t += blockDim.x) sp[t] = cscale(sp[t], filt[slot_of(t, N, CS, r)]);
    cfft_inverse<CS>(cl, sp, zs, xs, N, logN, tw);
    const double dt = cvec[0] / (4.0 * steps);
    for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) {
        const int n = r + CS * n2;
        const double2 v = xs[n2];
        lam[n] = v.x;
        lam[N + n] = v.y;
        for (int st = 0; st < 4; ++st) {
            const double w = rk_bw(st) * dt / 6.0;
            kb[(size_t)st * 2 * N + n] = w * v.x;
            kb[(size_t)st * 2 * N + N + n] = w * v.y;
        }
    }
    if (r == 0 && threadIdx.x == 0) *step = *step - 1;   // nothing in this kernel reads the counter
}

template <int CS>
__global__ void __launch_bounds__(CB_THREADS) k_cadj_local(const double *__restrict__ kb,
                                                           const double *__restrict__ rec, const int *step, int st,
                                                           int N, int logN, const double2 *__restrict__ tw,
                                                           const double *__restrict__ filt, double g, double tau,
                                                           const double *__restrict__ cvec, double *chi, double *etal,
                                                           double *psil, double *gT) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[33];
    __shared__ double part;
    cg::cluster_group cl = cg::this_cluster();
    const int L = N / CS, r = (int)cl.block_rank();
    double2 *xs = reinterpret_cast<double2 *>(smraw), *sp = xs + L, *sp2 = sp + L, *zs = sp2 + L, *ep = zs + L;
    const double *rc = stage_rec(rec, step, st, N);
    const double *ux = rc + N, *vy = rc + 2 * N, *w3 = rc + 3 * N, *F = rc + 4 * N;
    // d f / d T: this CTA's share of kb . F, then the cluster's sum in rank order
    double fd = 0.0;
    for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) {
        const int n = r + CS * n2;
        fd = fma(kb[n], F[n], fd);
        fd = fma(kb[N + n], F[N + n], fd);
        xs[n2] = make_double2(kb[n], kb[N + n]);
    }
    fd = block_sum(fd, red);
    if (threadIdx.x == 0) part = fd;
    cl.sync();
    if (r == 0 && threadIdx.x == 0) {
        double tot = 0.0;
        for (int q = 0; q < CS; ++q) tot += *cl.map_shared_rank(&part, q);
        *gT += tot / cvec[0];
    }
    // (et, pt) = (Filt kb_eta, P Filt kb_phi) and their derivatives
    cfft_forward<CS>(cl, xs, sp, N, logN, tw);   // (its cluster barriers keep every `part` alive until read)
    for (int t = threadIdx.x; t < L; t += blockDim.x) {
        const int j = slot_of(t, N, CS, r);
        double2 v = cscale(sp[t], filt[j]);
        if (j == 0) v.y = 0.0;   // P removes the mean of the phi part
        sp[t] = v;
        sp2[t] = mult(v, j, N, 0, 1.0);   // v carries the 1/N of the filter table
    }
    cfft_inverse<CS>(cl, sp, zs, xs, N, logN, tw);
    for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) ep[n2] = xs[n2];
    cfft_inverse<CS>(cl, sp2, zs, xs, N, logN, tw);
    for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) {
        const int n = r + CS * n2;
        const double et = ep[n2].x, pt = ep[n2].y, det = xs[n2].x, dpt = xs[n2].y;
        const double u = ux[n], v = vy[n];
        chi[n] = fma(v, pt, et);
        ep[n2].x = u * det + u * v * dpt - g * pt;
        xs[n2] = make_double2(u * pt, w3[n] * dpt);
    }
    // ((phi_x pt)', (w3 pt')') in one transform
    cfft_forward<CS>(cl, xs, sp, N, logN, tw);
    for (int t = threadIdx.x; t < L; t += blockDim.x) sp[t] = mult(sp[t], slot_of(t, N, CS, r), N, 0, 1.0 / N);
    cfft_inverse<CS>(cl, sp, zs, xs, N, logN, tw);
    for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) {
        const int n = r + CS * n2;
        psil[n] = xs[n2].x;
        etal[n] = fma(tau, xs[n2].y, ep[n2].x);
    }
}

template <int CS>
__global__ void __launch_bounds__(CB_THREADS) k_cadj_dtn(const double *__restrict__ chi, const double *__restrict__ y,
                                                         int N, int logN, const double2 *__restrict__ tw, double *M) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cg::cluster_group cl = cg::this_cluster();
    const int L = N / CS, r = (int)cl.block_rank();
    double2 *xs = reinterpret_cast<double2 *>(smraw), *sp = xs + L, *zs = sp + L;
    for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) {
        const int n = r + CS * n2;
        xs[n2] = make_double2(chi[n], y[n]);
    }
    cfft_forward<CS>(cl, xs, sp, N, logN, tw);
    for (int t = threadIdx.x; t < L; t += blockDim.x) sp[t] = cscale(sp[t], dtn_t_symbol(slot_of(t, N, CS, r), N));
    cfft_inverse<CS>(cl, sp, zs, xs, N, logN, tw);
    for (int n2 = threadIdx.x; n2 < L; n2 += blockDim.x) M[r + CS * n2] = xs[n2].x;
}

// pb = A^{-T} (...) + psil, eb = etal - phi_y pb; lambda += (eb, pb); kb_{st-1} += a_st dt (eb, pb)
__global__ void k_adj_update(const double *__restrict__ M, const double *__restrict__ psil,
                             const double *__restrict__ etal, const double *__restrict__ rec, const int *step, int st,
                             int N, const double *__restrict__ cvec, int steps, double *lam, double *kb) {
    const double *vy = stage_rec(rec, step, st, N) + 2 * N;
    const double adt = rk_a(st) * cvec[0] / (4.0 * steps);
    double *kp = kb + (size_t)(st > 0 ? st - 1 : 0) * 2 * N;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        const double pb = M[j] + psil[j];
        const double eb = fma(-vy[j], pb, etal[j]);
        lam[j] += eb;
        lam[N + j] += pb;
        if (st > 0) {
            kp[j] = fma(adt, eb, kp[j]);
            kp[N + j] = fma(adt, pb, kp[N + j]);
        }
    }
}

// grad[0] = d f / d T; grad[k] = basis_k . lambda(0), one block per entry
__global__ void k_adj_grad(const double *__restrict__ basis, const double *__restrict__ lam,
                           const double *__restrict__ gT, int N, int n, double *grad) {
    __shared__ double red[33];
    const int k = blockIdx.x;   // 0..n
    if (k == 0) {
        if (threadIdx.x == 0) grad[0] = *gT;
        return;
    }
    const double *b = basis + (size_t)(k - 1) * 2 * N;
    double acc = 0.0;
    for (int j = threadIdx.x; j < 2 * N; j += blockDim.x) acc = fma(b[j], lam[j], acc);
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) grad[k] = acc;
}

unsigned grid_for(int N) { return (unsigned)((N + 255) / 256); }

size_t fft_smem(int N, int arrays) { return (size_t)arrays * sizeof(double2) * N; }

}  // namespace

int prepare_adjoint(int Nmax) {
    const size_t one = fft_smem(Nmax, 1), two = fft_smem(Nmax, 2);
    WW_TRY(raise_smem(reinterpret_cast<const void *>(k_adj_begin_step), one));
    WW_TRY(raise_smem(reinterpret_cast<const void *>(k_adj_local), two));
    WW_TRY(raise_smem(reinterpret_cast<const void *>(k_adj_dtn), one));
    return WW_OK;
}

int launch_adj_record_eta(Ctx *c, AdjWs *a, int st) {
    k_rec_eta<<<grid_for(c->N), 256, 0, c->stream>>>(c->Ys, c->N, a->rec, a->step, st);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

int launch_adj_record_fields(Ctx *c, AdjWs *a, int st) {
    k_rec_fields<<<1, 1024, 0, c->stream>>>(c->ux, c->vy, c->w3, c->Fbase, c->N, a->rec, a->step, st);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

int launch_adj_init(Ctx *c, AdjWs *a) {
    k_adj_init<<<grid_for(c->N), 256, 0, c->stream>>>(c->Y, c->N, a->lam, a->gT);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

int launch_adj_set_step(Ctx *c, AdjWs *a, int v) {
    k_set_int<<<1, 1, 0, c->stream>>>(a->step, v);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

int launch_adj_begin_step(Ctx *c, AdjWs *a, const double *cvec) {
    if (cbase_ok(c))
        return launch_cluster(k_cadj_begin_step<CB_CS>, CB_CS, 3 * sizeof(double2) * (size_t)(c->N / CB_CS), c->stream,
                              a->lam, a->kb, c->N, c->logN, (const double2 *)c->tw, (const double *)c->filt_d,
                              cvec, c->steps, a->step);
    k_adj_begin_step<<<1, AJ_THREADS, fft_smem(c->N, 1), c->stream>>>(a->lam, a->kb, c->N, c->logN, c->tw, c->filt_d,
                                                                       cvec, c->steps, a->step);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

int launch_adj_fetch(Ctx *c, AdjWs *a, int off) {
    k_adj_fetch<<<grid_for(c->N), 256, 0, c->stream>>>(a->rec, a->step, off, c->N, a->eta);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

int launch_adj_local(Ctx *c, AdjWs *a, int st, const double *cvec) {
    if (cbase_ok(c))
        return launch_cluster(k_cadj_local<CB_CS>, CB_CS, 5 * sizeof(double2) * (size_t)(c->N / CB_CS), c->stream,
                              (const double *)(a->kb + (size_t)st * 2 * c->N), (const double *)a->rec,
                              (const int *)a->step, st, c->N, c->logN, (const double2 *)c->tw,
                              (const double *)c->filt_d, c->g, c->tau, cvec, a->chi, a->etal, a->psil, a->gT);
    k_adj_local<<<1, AJ_THREADS, fft_smem(c->N, 2), c->stream>>>(a->kb + (size_t)st * 2 * c->N, a->rec, a->step, st,
                                                                  c->N, c->logN, c->tw, c->filt_d, c->g, c->tau, cvec,
                                                                  a->chi, a->etal, a->psil, a->gT);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

int launch_adj_dtn(Ctx *c, AdjWs *a) {
    if (cbase_ok(c))
        return launch_cluster(k_cadj_dtn<CB_CS>, CB_CS, 3 * sizeof(double2) * (size_t)(c->N / CB_CS), c->stream,
                              (const double *)a->chi, (const double *)a->y, c->N, c->logN, (const double2 *)c->tw,
                              c->M);
    k_adj_dtn<<<1, AJ_THREADS, fft_smem(c->N, 1), c->stream>>>(a->chi, a->y, c->N, c->logN, c->tw, c->M);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

int launch_adj_update(Ctx *c, AdjWs *a, int st, const double *cvec) {
    k_adj_update<<<grid_for(c->N), 256, 0, c->stream>>>(c->M, a->psil, a->etal, a->rec, a->step, st, c->N, cvec,
                                                        c->steps, a->lam, a->kb);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

int launch_adj_grad(Ctx *c, AdjWs *a, double *grad) {
    k_adj_grad<<<c->n + 1, 256, 0, c->stream>>>(c->basis, a->lam, a->gT, c->N, c->n, grad);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

}  // namespace ww
