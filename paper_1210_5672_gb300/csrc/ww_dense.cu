// ww_dense.cu -- plain FP64 dense linear algebra of the DtN solve (Sec. 3.3:
// "perform an LU-factorization of K ... a single back-solve stage for each
// right-hand side"): a tiled DGEMM, a blocked right-looking LU without
// pivoting and the blocked multi-right-hand-side triangular solves.
//
// Pivoting is skipped: A = 1/2 I + K is a second-kind operator whose
// flat-surface eigenvalues 1/2 (1 + exp(-2|k|h)) lie in (1/2, 1], and the
// paper's GMRES needs only 4-30 iterations on it (Sec. 2.2).  Each diagonal
// block's inverse triangles are kept so that the triangular solves are
// products with 64 x 64 inverses plus DGEMM updates.
//
// Matrices are column-major.
#include "ww_internal.cuh"

namespace ww {

namespace {

// ---------------------------------------------------------------- DGEMM
constexpr int GB_M = 64, GB_N = 64, GB_K = 16;

__global__ void __launch_bounds__(256) k_dgemm(int m, int n, int k, double alpha, const double *__restrict__ A,
                                               int lda, const double *__restrict__ B, int ldb, double beta,
                                               double *C, int ldc) {
    __shared__ double As[GB_K][GB_M + 1];
    __shared__ double Bs[GB_K][GB_N + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int row0 = blockIdx.x * GB_M, col0 = blockIdx.y * GB_N;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

    for (int k0 = 0; k0 < k; k0 += GB_K) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int idx = tid + r * 256;
            int ar = idx & (GB_M - 1), ak = idx >> 6;         // A tile: 64 rows x 16 k
            int gr = row0 + ar, gk = k0 + ak;
            As[ak][ar] = (gr < m && gk < k) ? A[(size_t)gk * lda + gr] : 0.0;
            int bk = idx & (GB_K - 1), bc = idx >> 4;         // B tile: 16 k x 64 cols
            int gk2 = k0 + bk, gc = col0 + bc;
            Bs[bk][bc] = (gk2 < k && gc < n) ? B[(size_t)gc * ldb + gk2] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][tx + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[kk][ty + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int gc = col0 + ty + 16 * c;
        if (gc >= n) continue;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int gr = row0 + tx + 16 * r;
            if (gr >= m) continue;
            double *p = C + (size_t)gc * ldc + gr;
            *p = (beta == 0.0) ? alpha * acc[r][c] : fma(alpha, acc[r][c], beta * *p);
        }
    }
}

// ---------------------------------------------------------------- LU pieces
// Factor the kb x kb diagonal block at A(k0, k0) in place (no pivoting) and
// write its inverse triangles Linv (unit lower) and Uinv (upper), kb x kb,
// column-major.  Everything happens in shared memory (3 x 64 x 65 doubles,
// dynamic), 512 threads.  One SM's FP64 pipe (2 FMA per clock: a warp-wide
// FP64 instruction occupies it for 16 clocks) bounds the block, so the work is
// laid out to keep warps full and divisions out of the loops:
//  * the factorisation pivot by pivot: the column below the pivot is scaled by
//    the pivot's reciprocal, then the trailing block takes its rank-1 update,
//    its (rem x rem) entries spread contiguously over all threads;
//  * the inverse triangles column by column, all 2 x 64 columns at once, four
//    lanes of a warp per column: Linv(r, c) = -sum_{q=c}^{r-1} L(r,q) Linv(q,c)
//    down the column, Uinv(r, c) = -sum_{q=r+1}^{c} U(r,q) Uinv(q,c) / U(r,r)
//    up the column (the reciprocals of U's diagonal taken once), each sum split
//    over the four lanes and combined by shuffles (no block-wide barrier
//    between the rows of a column).
// About 85k FMA for the factors and 88k for the inverses at kb = 64.
constexpr int LD = LU_NB + 1;
constexpr size_t LU_DIAG_SMEM = 3 * sizeof(double) * LU_NB * LD;
constexpr int LU_DIAG_THREADS = 512;

__global__ void __launch_bounds__(LU_DIAG_THREADS) k_lu_diag(double *A, int lda, int k0, int kb, double *Linv,
                                                             double *Uinv, int *status) {
    extern __shared__ double dsm[];
    double(*a)[LD] = reinterpret_cast<double(*)[LD]>(dsm);                    // a[col][row]
    double(*li)[LD] = reinterpret_cast<double(*)[LD]>(dsm + LU_NB * LD);      // li[row][col]
    double(*ui)[LD] = reinterpret_cast<double(*)[LD]>(dsm + 2 * LU_NB * LD);  // ui[row][col]
    __shared__ double rdiag[LU_NB];                                           // 1 / U(r, r)
    const int tid = threadIdx.x;
    for (int idx = tid; idx < kb * kb; idx += blockDim.x) {
        const int r = idx % kb, c = idx / kb;
        a[c][r] = A[(size_t)(k0 + c) * lda + k0 + r];
    }
    __syncthreads();
    for (int p = 0; p < kb; ++p) {
        const int rem = kb - p - 1;
        if (tid < LU_NB) {   // two warps: one reciprocal each lane (divisions are dear on the FP64 pipe)
            const double inv = 1.0 / a[p][p];
            if (tid < rem) a[p][p + 1 + tid] *= inv;
            if (tid == 0) rdiag[p] = inv;
        }
        __syncthreads();
        for (int idx = tid; idx < rem * rem; idx += blockDim.x) {
            const int r = p + 1 + idx % rem, c = p + 1 + idx / rem;
            a[c][r] = fma(-a[p][r], a[c][p], a[c][r]);   // A(r,c) -= L(r,p) U(p,c)
        }
        __syncthreads();
    }
    int bad = 0;
    for (int idx = tid; idx < kb * kb; idx += blockDim.x) {
        const int r = idx % kb, c = idx / kb;
        const double v = a[c][r];
        if (!isfinite(v)) bad = 1;
        A[(size_t)(k0 + c) * lda + k0 + r] = v;
    }
    if (__syncthreads_or(bad) && tid == 0) atomicOr(status, ST_NONFINITE);
    // inverse triangles: warps 0..7 the columns of Linv, warps 8..15 those of Uinv,
    // four lanes per column (8 columns per warp).  Every lane of a warp walks
    // the same rows (uniform loop and shuffles), inactive lanes adding zeros.
    const int lane4 = tid & 3, c = (tid >> 2) & 63;
    const bool own = c < kb;
    if (tid < 256) {
        if (own && lane4 == 0)
            for (int r = 0; r < kb; ++r) li[r][c] = r == c ? 1.0 : 0.0;
        __syncwarp();
        for (int r = 1; r < kb; ++r) {
            const bool act = own && r > c;
            double part = 0.0;
            if (act)
                for (int q = c + lane4; q < r; q += 4) part = fma(-a[q][r], li[q][c], part);
            part += __shfl_xor_sync(0xffffffffu, part, 1);
            part += __shfl_xor_sync(0xffffffffu, part, 2);
            if (act && lane4 == 0) li[r][c] = part;
            __syncwarp();
        }
    } else {
        if (own && lane4 == 0)
            for (int r = 0; r < kb; ++r) ui[r][c] = r == c ? rdiag[c] : 0.0;
        __syncwarp();
        for (int r = kb - 2; r >= 0; --r) {
            const bool act = own && r < c;
            double part = 0.0;
            if (act)
                for (int q = r + 1 + lane4; q <= c; q += 4) part = fma(-a[q][r], ui[q][c], part);
            part += __shfl_xor_sync(0xffffffffu, part, 1);
            part += __shfl_xor_sync(0xffffffffu, part, 2);
            if (act && lane4 == 0) ui[r][c] = part * rdiag[r];
            __syncwarp();
        }
    }
    __syncthreads();
    for (int idx = tid; idx < kb * kb; idx += blockDim.x) {
        const int r = idx % kb, c = idx / kb;
        Linv[(size_t)c * kb + r] = li[r][c];
        Uinv[(size_t)c * kb + r] = ui[r][c];
    }
}

constexpr int AP_T = 16;   // rows per block (apply_right)
constexpr int AP_L = 4;    // columns per block (apply_left): 129 blocks for 513 columns

// B(kb x ncols, leading dim ldb) <- T * B, T kb x kb (in place).
// One block per AP_L columns (enough blocks to fill the GPU at a few hundred
// columns); each block reads its whole column slab before writing it back.
__global__ void __launch_bounds__(256) k_apply_left(const double *__restrict__ T, int kb, double *B, int ldb,
                                                    int ncols) {
    __shared__ double t[LU_NB][LU_NB + 1];   // t[col][row]
    __shared__ double b[AP_L][LU_NB + 1];    // b[col][row]
    const int tid = threadIdx.x;
    const int c0 = blockIdx.x * AP_L;
    const int nc = min(AP_L, ncols - c0);
    for (int idx = tid; idx < kb * kb; idx += blockDim.x) t[idx / kb][idx % kb] = T[idx];
    for (int idx = tid; idx < kb * nc; idx += blockDim.x) {
        int r = idx % kb, c = idx / kb;
        b[c][r] = B[(size_t)(c0 + c) * ldb + r];
    }
    __syncthreads();
    for (int idx = tid; idx < kb * nc; idx += blockDim.x) {
        int r = idx % kb, c = idx / kb;
        double s = 0.0;
        for (int q = 0; q < kb; ++q) s = fma(t[q][r], b[c][q], s);
        B[(size_t)(c0 + c) * ldb + r] = s;
    }
}

// B(nrows x kb, leading dim ldb) <- B * T, T kb x kb (in place).
// One block per AP_T rows.
__global__ void __launch_bounds__(256) k_apply_right(const double *__restrict__ T, int kb, double *B, int ldb,
                                                     int nrows) {
    __shared__ double t[LU_NB][LU_NB + 1];   // t[col][row]
    __shared__ double b[LU_NB][AP_T + 1];    // b[col][row]
    const int tid = threadIdx.x;
    const int r0 = blockIdx.x * AP_T;
    const int nr = min(AP_T, nrows - r0);
    for (int idx = tid; idx < kb * kb; idx += blockDim.x) t[idx / kb][idx % kb] = T[idx];
    for (int idx = tid; idx < nr * kb; idx += blockDim.x) {
        int r = idx % nr, c = idx / nr;
        b[c][r] = B[(size_t)c * ldb + r0 + r];
    }
    __syncthreads();
    for (int idx = tid; idx < nr * kb; idx += blockDim.x) {
        int r = idx % nr, c = idx / nr;
        double s = 0.0;
        for (int q = 0; q < kb; ++q) s = fma(b[q][r], t[c][q], s);
        B[(size_t)c * ldb + r0 + r] = s;
    }
}

}  // namespace

int prepare_dense() {
    WW_CUDA_TRY(cudaFuncSetAttribute(k_lu_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LU_DIAG_SMEM));
    return WW_OK;
}

int dgemm(cudaStream_t s, int m, int n, int k, double alpha, const double *A, int lda, const double *B, int ldb,
          double beta, double *C, int ldc) {
    if (m <= 0 || n <= 0) return WW_OK;
    if (n <= 8) return gemv_narrow(s, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    dim3 grid((m + GB_M - 1) / GB_M, (n + GB_N - 1) / GB_N);
    k_dgemm<<<grid, 256, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

int lu_factor_fp64(Ctx *c) {
    const int N = c->N, nb = c->nb;
    for (int k0 = 0, blk = 0; k0 < N; k0 += nb, ++blk) {
        const int kb = min(nb, N - k0);
        double *Linv = c->Dinv + (size_t)blk * 2 * nb * nb, *Uinv = Linv + (size_t)nb * nb;
        k_lu_diag<<<1, LU_DIAG_THREADS, LU_DIAG_SMEM, c->stream>>>(c->A, N, k0, kb, Linv, Uinv, c->status);
        WW_CUDA_TRY(cudaGetLastError());
        const int r = N - k0 - kb;
        if (r <= 0) continue;
        double *A21 = c->A + (size_t)k0 * N + k0 + kb;      // r x kb
        double *A12 = c->A + (size_t)(k0 + kb) * N + k0;    // kb x r
        double *A22 = c->A + (size_t)(k0 + kb) * N + k0 + kb;
        k_apply_right<<<(r + AP_T - 1) / AP_T, 256, 0, c->stream>>>(Uinv, kb, A21, N, r);   // L21 = A21 U11^-1
        k_apply_left<<<(r + AP_L - 1) / AP_L, 256, 0, c->stream>>>(Linv, kb, A12, N, r);    // U12 = L11^-1 A12
        WW_CUDA_TRY(cudaGetLastError());
        WW_TRY(dgemm(c->stream, r, r, kb, -1.0, A21, N, A12, N, 1.0, A22, N));
    }
    return WW_OK;
}

int lu_solve_fp64(Ctx *c, double *B, int ncols) {
    const int N = c->N, nb = c->nb;
    const int nblk = (N + nb - 1) / nb;
    const unsigned gcols = (unsigned)((ncols + AP_L - 1) / AP_L);
    // forward: L X = B
    for (int blk = 0; blk < nblk; ++blk) {
        const int k0 = blk * nb, kb = min(nb, N - k0);
        const double *Linv = c->Dinv + (size_t)blk * 2 * nb * nb;
        k_apply_left<<<gcols, 256, 0, c->stream>>>(Linv, kb, B + k0, N, ncols);
        WW_CUDA_TRY(cudaGetLastError());
        const int r = N - k0 - kb;
        if (r > 0)
            WW_TRY(dgemm(c->stream, r, ncols, kb, -1.0, c->A + (size_t)k0 * N + k0 + kb, N, B + k0, N, 1.0,
                         B + k0 + kb, N));
    }
    // backward: U X = Y
    for (int blk = nblk - 1; blk >= 0; --blk) {
        const int k0 = blk * nb, kb = min(nb, N - k0);
        const double *Uinv = c->Dinv + (size_t)blk * 2 * nb * nb + (size_t)nb * nb;
        k_apply_left<<<gcols, 256, 0, c->stream>>>(Uinv, kb, B + k0, N, ncols);
        WW_CUDA_TRY(cudaGetLastError());
        if (k0 > 0)
            WW_TRY(dgemm(c->stream, k0, ncols, kb, -1.0, c->A + (size_t)k0 * N, N, B + k0, N, 1.0, B, N));
    }
    return WW_OK;
}

}  // namespace ww
