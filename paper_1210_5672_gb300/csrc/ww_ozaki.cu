// ww_ozaki.cu -- FP64-accurate products on the bf16 tensor cores by exact
// splitting (the Ozaki scheme: Ozaki, Ogita, Oishi & Rump, Numer. Algorithms
// 2012; its tensor-core form: Ootomo, Ozaki & Yokota, IJHPCA 2024), used for
// the refinement residuals R = Psi - A M and for the G apply of the DtN
// (Sec. 3.3 computes its refinement residuals in quad precision for the same
// reason: the correction solves may be inexact, the residual may not).
//
// Splitting.  Row i of the left operand gets a power-of-two scale 2^ea_i >
// max_k |a_ik|, column j of the right operand 2^fb_j.  Each entry is written as
//   a_ik = 2^ea_i sum_{p=1..7} a_p 2^{-6-7(p-1)},   a_p integers in [-64, 64]
// (round-to-nearest digits computed exactly in 64-bit fixed point; 48 bits
// kept, remainder < 2^-49 of the row maximum).  The digits are exact in bf16.
//
// Products.  a_p b_q has weight 2^{E - 7g}, g = p + q - 2, E = ea_i + fb_j - 12.
// All pairs with g <= 6 (28 of 49) are accumulated per group g in TMEM (fp32);
// |digit products| <= 2^12, so a group over a 1024-long K block stays below
// 2^24 for g <= 2 and the tensor cores sum it exactly; groups g >= 3 carry
// weights <= 2^-21 and their fp32 rounding (if any) is below 2^-45 of the
// result.  After each K block the 7 groups are converted to integers and
// folded exactly into two int64 accumulators per entry,
//   hi = V0 2^14 + V1 2^7 + V2,  lo = V3 2^21 + V4 2^14 + V5 2^7 + V6,
// and the result is 2^ea_i 2^fb_j (2^-26 hi + 2^-54 lo).
//
// Kernel.  One CTA per 128 x 64 output tile.  Warps 0 and 10: TMA producers
// (ring of 7 A-digit tiles of 128 x 64 and ring of 2 B stages holding all 7
// B-digit tiles of 64 x 64); warp 1: TMEM owner and tcgen05.mma issuer (M = 128,
// K = 16, N = 64..256: the B digits of one A digit are issued together, 10
// MMAs per K step instead of 28); warps 2..9: fold and epilogue, each thread
// one row and 32 columns.  All waits are bounded.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <string>
#include <vector>

#include "ww_internal.cuh"
#include "ww_tc.cuh"

namespace ww {

int tc_make_map(CUtensorMap *map, const void *ptr, int K, long rows, int box_rows, int box_k);   // ww_tcgemm.cu

namespace {

constexpr int OZ_S = 7;             // digits per operand
constexpr int OZ_G = 7;             // groups g = 0..6
constexpr int OZ_BM = 128, OZ_BN = 64, OZ_BK = 64;
constexpr int OZ_KBLOCK = 16;       // K chunks (of 64) per exact block = 1024
constexpr int OZ_ASLOTS = 7, OZ_BSLOTS = 2;   // one slot per A digit, two B stages
constexpr int OZ_EPI_WARPS = 8;
// warps: 0 producer (B and the even A digits), 1 MMA, 2..9 epilogue, 10 second
// producer (the odd A digits).  One thread issues a TMA load every ~145 ns
// whatever the box size, so two issuers double the rate of 8-16 KB boxes.
constexpr int OZ_PROD2 = 2 + OZ_EPI_WARPS;
constexpr int OZ_THREADS = 32 * (OZ_PROD2 + 1);
constexpr int OZ_A_TILE = OZ_BM * OZ_BK * 2;           // 16 KB
constexpr int OZ_B_TILE = OZ_BN * OZ_BK * 2;           // 8 KB
constexpr int OZ_B_STAGE = OZ_S * OZ_B_TILE;           // 56 KB
constexpr int OZ_SMEM = OZ_ASLOTS * OZ_A_TILE + OZ_BSLOTS * OZ_B_STAGE + 1024 + 256;

struct OzOut {
    int mode;                 // 0: C += value; 1: C = Psi - 0.5 Mh - value (residual)
    double *C;
    int ldc;
    const double *Psi;
    int ldpsi;
    const double *Mh;
    int ldm;
    unsigned long long *colmax;   // mode 1: per-column max |R| (bits of a positive double), or NULL
    __nv_bfloat16 *rslc;          // mode 1: 2 bf16 slices of R ([2][Nn][M], as the next product's B), or NULL
};

// ND <= OZ_S digits of each operand take part (ND = 7: all pairs with g <= 6;
// ND = 5: g <= 4, 15 pairs, the operands to 2^-35 of their row / column maxima,
// for residuals whose error is contracted by a later correction).
template <int ND>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_ozaki(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int Nn, int K,
            const double *__restrict__ sa, const double *__restrict__ sb, OzOut out, int *err, const int *skip) {
    if (skip && *skip) return;   // the caller's device-side decision to leave this product out
    extern __shared__ uint8_t smem_raw[];
    const uint32_t base = tc::smem_u32(smem_raw);
    uint8_t *smem = smem_raw + ((1024 - (base & 1023)) & 1023);
    uint8_t *aring = smem;
    uint8_t *bring = smem + OZ_ASLOTS * OZ_A_TILE;
    uint64_t *bar = reinterpret_cast<uint64_t *>(bring + OZ_BSLOTS * OZ_B_STAGE);
    uint64_t *a_full = bar, *a_empty = bar + OZ_ASLOTS;
    uint64_t *b_full = a_empty + OZ_ASLOTS, *b_empty = b_full + OZ_BSLOTS;
    uint64_t *acc_full = b_empty + OZ_BSLOTS, *acc_empty = acc_full + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(acc_empty + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * OZ_BM, n0 = blockIdx.y * OZ_BN;
    const int nk = K / OZ_BK;
    const int nblk = (nk + OZ_KBLOCK - 1) / OZ_KBLOCK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < OZ_ASLOTS; ++s) {
            tc::mbar_init(&a_full[s], 1);
            tc::mbar_init(&a_empty[s], 1);
        }
        for (int s = 0; s < OZ_BSLOTS; ++s) {
            tc::mbar_init(&b_full[s], 1);
            tc::mbar_init(&b_empty[s], 1);
        }
        tc::mbar_init(acc_full, 1);
        tc::mbar_init(acc_empty, OZ_EPI_WARPS);
        tc::mbar_fence_init();
        tc::prefetch_tmap(&tmA);
        tc::prefetch_tmap(&tmB);
    }
    if (warp == 1) {
        tc::tmem_alloc(tslot, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0 || warp == OZ_PROD2) {
        // ------------------------------------------------ TMA producers (whole warps, one lane issues)
        const uint32_t leader = tc::elect_one();
        const int p0 = warp == 0 ? 0 : 1;   // A digits p0, p0 + 2, ...
        for (int kc = 0; kc < nk; ++kc) {
            if (warp == 0) {
                const int bs = kc % OZ_BSLOTS;
                tc::mbar_wait(&b_empty[bs], ((kc / OZ_BSLOTS) & 1) ^ 1, err);
                tc::mbar_arrive_expect_tx_if(leader, &b_full[bs], ND * OZ_B_TILE);
#pragma unroll
                for (int q = 0; q < ND; ++q)
                    tc::tma_load_2d_if(leader, &tmB, &b_full[bs], bring + bs * OZ_B_STAGE + q * OZ_B_TILE,
                                       kc * OZ_BK, q * Nn + n0);
            }
            for (int p = p0; p < ND; p += 2) {
                const int ai = kc * ND + p, as = ai % OZ_ASLOTS;
                tc::mbar_wait(&a_empty[as], ((ai / OZ_ASLOTS) & 1) ^ 1, err);
                tc::mbar_arrive_expect_tx_if(leader, &a_full[as], OZ_A_TILE);
                tc::tma_load_2d_if(leader, &tmA, &a_full[as], aring + as * OZ_A_TILE, kc * OZ_BK, p * M + m0);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer (whole warp, one lane issues)
        const uint32_t leader = tc::elect_one();
        for (int kc = 0; kc < nk; ++kc) {
            const int kb = kc / OZ_KBLOCK;
            const bool first = (kc % OZ_KBLOCK) == 0;
            if (first && kb > 0) {
                tc::mbar_wait(acc_empty, (kb - 1) & 1, err);   // epilogue drained the last block
                tc::fence_after();
            }
            const int bs = kc % OZ_BSLOTS;
            tc::mbar_wait(&b_full[bs], (kc / OZ_BSLOTS) & 1, err);
            tc::fence_after();
            const uint32_t bst = tc::smem_u32(bring + bs * OZ_B_STAGE);
#pragma unroll
            for (int p = 0; p < ND; ++p) {
                const int ai = kc * ND + p, as = ai % OZ_ASLOTS;
                tc::mbar_wait(&a_full[as], (ai / OZ_ASLOTS) & 1, err);
                tc::fence_after();
                const uint64_t da = tc::desc_k128(tc::smem_u32(aring + as * OZ_A_TILE));
                // pairs (p, q), q = 0 .. 6-p, land in groups p .. 6: consecutive TMEM
                // column blocks, and the B digits q are consecutive 64-row tiles of
                // the stage, so up to four of them form one N = 256 operand.  One
                // wide MMA reads the A digit once instead of once per q.
#pragma unroll
                for (int q0 = 0; q0 + p < ND; q0 += 4) {
                    const int nq = min(4, ND - p - q0);
                    const uint32_t id = tc::idesc_bf16(OZ_BM, OZ_BN * nq);
                    const uint32_t d = tmem + (uint32_t)((p + q0) * OZ_BN);
                    const uint64_t db = tc::desc_k128(bst + q0 * OZ_B_TILE);
#pragma unroll
                    for (int kk = 0; kk < OZ_BK / 16; ++kk)   // +32 B per K step: +2 in the start-address field
                        tc::mma_bf16_if(leader, d, da + 2 * kk, db + 2 * kk, id, !(first && p == 0 && kk == 0));
                }
                tc::mma_commit_if(leader, &a_empty[as]);
            }
            tc::mma_commit_if(leader, &b_empty[bs]);
            if ((kc % OZ_KBLOCK) == OZ_KBLOCK - 1 || kc == nk - 1) tc::mma_commit_if(leader, acc_full);
        }
    } else if (warp >= 2 && warp < OZ_PROD2) {
        // ------------------------------------------------ fold + epilogue
        const int ew = warp - 2;
        const int quarter = warp & 3;            // TMEM lane quarter this warp may access
        const int chalf = ew >> 2;               // columns 32*chalf .. +31
        const int row = m0 + quarter * 32 + lane;
        long long hi[32], lo[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0;
        for (int kb = 0; kb < nblk; ++kb) {
            tc::mbar_wait(acc_full, kb & 1, err);
            tc::fence_after();
#pragma unroll 1
            for (int g = 0; g < ND; ++g) {
                float v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(g * OZ_BN + chalf * 32), v);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const long long iv = (long long)__float2int_rn(v[j]);
                    if (g < 3)
                        hi[j] += iv * (1LL << (7 * (2 - g)));
                    else
                        lo[j] += iv * (1LL << (7 * (6 - g)));
                }
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(acc_empty);
        }
        // column maxima of the residual: reduced over the warp's 32 rows first (one
        // atomic per warp and column instead of one per element) when all 32 rows exist
        const bool full_warp = __all_sync(0xffffffffu, row < M);
        if (row < M) {
            const double si = sa[row];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int col = n0 + chalf * 32 + j;   // the same for every lane of the warp
                if (col < Nn) {
                    const double val = si * sb[col] * fma((double)hi[j], 0x1p-26, (double)lo[j] * 0x1p-54);
                    const size_t ic = (size_t)col * out.ldc + row;
                    if (out.mode == 0) {
                        out.C[ic] += val;
                    } else {
                        const double r = (out.Psi[(size_t)col * out.ldpsi + row] -
                                          0.5 * out.Mh[(size_t)col * out.ldm + row]) - val;
                        if (out.C) out.C[ic] = r;
                        if (out.rslc) {   // the residual as the right operand of the correction X R
                            float v = (float)r;
                            const __nv_bfloat16 b0 = __float2bfloat16_rn(v);
                            v -= __bfloat162float(b0);
                            out.rslc[(size_t)col * M + row] = b0;
                            out.rslc[((size_t)Nn + col) * M + row] = __float2bfloat16_rn(v);
                        }
                        if (out.colmax) {
                            if (full_warp) {
                                double a = fabs(r);
#pragma unroll
                                for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
                                if (lane == 0)
                                    atomicMax(&out.colmax[col], (unsigned long long)__double_as_longlong(a));
                            } else {
                                atomicMax(&out.colmax[col], (unsigned long long)__double_as_longlong(fabs(r)));
                            }
                        }
                    }
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------- digits
__device__ __forceinline__ int bexp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// biased-exponent maxima of the rows of a column-major matrix (one thread per
// row and 64-column strip; emax zeroed by the caller)
__global__ void k_expmax_rows(const double *__restrict__ X, int ld, int rows, int cols, float diag_shift,
                              int *emax) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int c0 = blockIdx.y * 64;
    if (r >= rows) return;
    int m = 0;
    for (int c = c0; c < min(cols, c0 + 64); ++c) {
        double x = X[(size_t)c * ld + r];
        if (diag_shift != 0.f && r == c) x -= (double)diag_shift;
        m = max(m, bexp(x));
    }
    atomicMax(&emax[r], m);
}

// scale 2^ea from the biased exponent maximum: 2^(emax - 1022) > max |x|
__global__ void k_scales(const int *__restrict__ emax, int n, double *scale, const int *skip) {
    if (skip && *skip) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int e = emax[i];
    scale[i] = e == 0 ? 1.0 : ldexp(1.0, e - 1022);
}

// 7 digits of every entry of the left operand (the rows of a column-major
// M x K matrix, minus diag_shift on its diagonal): dst[p][i][k].  Digits are
// computed in 64-bit fixed point: F = x 2^-ea 2^60, a_p = round(F / 2^{54 - 7(p-1)}).
__global__ void k_digits(const double *__restrict__ X, int ld, int rows, int K, float diag_shift,
                         const int *__restrict__ emax, __nv_bfloat16 *dst, const int *skip) {
    if (skip && *skip) return;
    __shared__ long long tile[32][33];
    const int t0 = blockIdx.y * 32, k0 = blockIdx.x * 32;   // t: row of the operand
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int yy = ty; yy < 32; yy += 8) {
        // read coalesced along the rows of the column-major source
        const int t = t0 + tx, k = k0 + yy;
        double x = (t < rows && k < K) ? X[(size_t)k * ld + t] : 0.0;
        if (diag_shift != 0.f && t == k) x -= (double)diag_shift;
        long long F = 0;
        if (t < rows && k < K) {
            const long long bits = __double_as_longlong(x);
            const int e = (int)((bits >> 52) & 0x7FF);
            if (e != 0) {
                const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
                const int sh = e - emax[t] + 7;
                F = sh >= 0 ? (mant << sh) : (sh > -63 ? (mant >> -sh) : 0);
                if (bits < 0) F = -F;
            }
        }
        tile[yy][tx] = F;   // tile[k][t]
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
        const int t = t0 + yy, k = k0 + tx;
        if (t >= rows || k >= K) continue;
        long long F = tile[tx][yy];
#pragma unroll
        for (int p = 0; p < OZ_S; ++p) {
            const int sh = 54 - 7 * p;
            const long long a = (F + (1LL << (sh - 1))) >> sh;   // arithmetic shift: round to nearest
            F -= a * (1LL << sh);
            dst[((size_t)p * rows + t) * K + k] = __int2bfloat16_rn((int)a);
        }
    }
}

// Right operand (side 1) in one pass per column: max exponent, scale, the 7
// digits, and (optionally) a zeroed column maximum for the product's residual.
__global__ void k_col_digits(const double *__restrict__ X, int ld, int ncols, int K, double *scale,
                             __nv_bfloat16 *dst, unsigned long long *zero_cm, const int *skip) {
    if (skip && *skip) return;
    __shared__ int red[32];
    const int col = blockIdx.x;
    const double *x = X + (size_t)col * ld;
    int m = 0;
    for (int r = threadIdx.x; r < K; r += blockDim.x) m = max(m, bexp(x[r]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) {
            red[0] = m;
            scale[col] = m == 0 ? 1.0 : ldexp(1.0, m - 1022);
            if (zero_cm) zero_cm[col] = 0ull;
        }
    }
    __syncthreads();
    const int em = red[0];
    for (int r = threadIdx.x; r < K; r += blockDim.x) {
        const long long bits = __double_as_longlong(x[r]);
        const int e = (int)((bits >> 52) & 0x7FF);
        long long F = 0;
        if (e != 0) {
            const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
            const int sh = e - em + 7;
            F = sh >= 0 ? (mant << sh) : (sh > -63 ? (mant >> -sh) : 0);
            if (bits < 0) F = -F;
        }
#pragma unroll
        for (int p = 0; p < OZ_S; ++p) {
            const int sh = 54 - 7 * p;
            const long long a = (F + (1LL << (sh - 1))) >> sh;   // arithmetic shift: round to nearest
            F -= a * (1LL << sh);
            dst[((size_t)p * ncols + col) * K + r] = __int2bfloat16_rn((int)a);
        }
    }
}

}  // namespace

// Digits and scales of the columns of the K x ncols column-major X (the right
// operand) in one kernel; zero_cm (optional) is set to 0 for each column.
int ozaki_digits_cols(cudaStream_t s, const double *X, int ld, int ncols, int K, double *scale, __nv_bfloat16 *dst,
                      unsigned long long *zero_cm, const int *skip) {
    k_col_digits<<<ncols, 256, 0, s>>>(X, ld, ncols, K, scale, dst, zero_cm, skip);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

// Digits and scales of an operand.  side 0: left operand = the rows of the
// column-major rows x K matrix X (minus diag_shift on its diagonal);
// side 1: right operand = the columns of the column-major K x rows matrix X.
// emax: int[rows] work (zeroed here); scale: double[rows]; dst: 7 x rows x K bf16.
int ozaki_digits(cudaStream_t s, const double *X, int ld, int rows, int K, int side, float diag_shift, int *emax,
                 double *scale, __nv_bfloat16 *dst, const int *skip) {
    if (side == 1) {
        if (diag_shift != 0.f) return fail(WW_ERR_ARG, "ozaki_digits: no diagonal shift on a right operand");
        return ozaki_digits_cols(s, X, ld, rows, K, scale, dst, nullptr, skip);
    }
    WW_CUDA_TRY(cudaMemsetAsync(emax, 0, sizeof(int) * rows, s));
    dim3 g((rows + 127) / 128, (K + 63) / 64);
    k_expmax_rows<<<g, 128, 0, s>>>(X, ld, rows, K, diag_shift, emax);
    k_scales<<<(rows + 255) / 256, 256, 0, s>>>(emax, rows, scale, skip);
    dim3 gd((K + 31) / 32, (rows + 31) / 32);
    k_digits<<<gd, 256, 0, s>>>(X, ld, rows, K, diag_shift, emax, dst, skip);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

// The same digits of a left operand whose row exponent maxima emax (biased,
// of the shifted entries) were taken elsewhere (by the assembly).
int ozaki_digits_rows_emax(cudaStream_t s, const double *X, int ld, int rows, int K, float diag_shift,
                           const int *emax, double *scale, __nv_bfloat16 *dst, const int *skip) {
    k_scales<<<(rows + 255) / 256, 256, 0, s>>>(emax, rows, scale, skip);
    dim3 gd((K + 31) / 32, (rows + 31) / 32);
    k_digits<<<gd, 256, 0, s>>>(X, ld, rows, K, diag_shift, emax, dst, skip);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

// mode 0: C += A B ; mode 1: C = Psi - 0.5 Mh - A B  (A = left digits, B = right digits)
int ozaki_gemm(cudaStream_t s, const __nv_bfloat16 *Ad, const double *sa, const __nv_bfloat16 *Bd, const double *sb,
               int M, int Nn, int K, int mode, double *C, int ldc, const double *Psi, int ldpsi, const double *Mh,
               int ldm, unsigned long long *colmax, int *err, const int *skip, __nv_bfloat16 *rslc, int nd) {
    if (K % OZ_BK != 0) return fail(WW_ERR_ARG, "ozaki_gemm: K must be a multiple of 64");
    if (nd != 5 && nd != OZ_S) return fail(WW_ERR_ARG, "ozaki_gemm: 5 or 7 digits");
    CUtensorMap ta, tb;
    WW_TRY(tc_make_map(&ta, Ad, K, (long)OZ_S * M, OZ_BM, OZ_BK));
    WW_TRY(tc_make_map(&tb, Bd, K, (long)OZ_S * Nn, OZ_BN, OZ_BK));
    auto kern = nd == 5 ? k_ozaki<5> : k_ozaki<OZ_S>;
    WW_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
    OzOut o{mode, C, ldc, Psi, ldpsi, Mh, ldm, colmax, rslc};
    dim3 grid((M + OZ_BM - 1) / OZ_BM, (Nn + OZ_BN - 1) / OZ_BN);
    kern<<<grid, OZ_THREADS, OZ_SMEM, s>>>(ta, tb, M, Nn, K, sa, sb, o, err, skip);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

}  // namespace ww

// -------------------------------------------------------------------------
// self-test (declared in ww.h): C = A B (A: M x K, B: K x Nn, C: M x Nn,
// column-major FP64 device arrays) through the digit path.
// -------------------------------------------------------------------------
extern "C" int ww_selftest_ozaki(const double *A, const double *B, int M, int Nn, int K, double *C) {
    using namespace ww;
    if (!A || !B || !C || M < 1 || Nn < 1 || K < 64 || K % 64)
        return fail(WW_ERR_ARG, "ww_selftest_ozaki: NULL pointer or bad sizes (K a multiple of 64)");
    cudaStream_t s = nullptr;
    __nv_bfloat16 *Ad = nullptr, *Bd = nullptr;
    double *sa = nullptr, *sb = nullptr;
    int *ea = nullptr, *eb = nullptr, *err = nullptr;
    int st = WW_OK;
    if (cudaMalloc(&Ad, 2 * (7 * (size_t)M + 256) * K) != cudaSuccess ||
        cudaMalloc(&Bd, 2 * (7 * (size_t)Nn + 256) * K) != cudaSuccess ||
        cudaMalloc(&sa, 8 * (size_t)M) != cudaSuccess || cudaMalloc(&sb, 8 * (size_t)Nn) != cudaSuccess ||
        cudaMalloc(&ea, 4 * (size_t)M) != cudaSuccess || cudaMalloc(&eb, 4 * (size_t)Nn) != cudaSuccess ||
        cudaMalloc(&err, 4) != cudaSuccess)
        st = fail(WW_ERR_ALLOC, "selftest alloc");
    if (st == WW_OK && (cudaMemset(err, 0, 4) != cudaSuccess || cudaMemset(C, 0, 8 * (size_t)M * Nn) != cudaSuccess))
        st = fail(WW_ERR_CUDA, "selftest memset");
    if (st == WW_OK) st = ozaki_digits(s, A, M, M, K, 0, 0.f, ea, sa, Ad, nullptr);
    if (st == WW_OK) st = ozaki_digits(s, B, K, Nn, K, 1, 0.f, eb, sb, Bd, nullptr);
    if (st == WW_OK)
        st = ozaki_gemm(s, Ad, sa, Bd, sb, M, Nn, K, 0, C, M, nullptr, 0, nullptr, 0, nullptr, err, nullptr, nullptr, 7);
    if (st == WW_OK && cudaDeviceSynchronize() != cudaSuccess) st = fail(WW_ERR_CUDA, "selftest sync");
    if (st == WW_OK) {
        int e = 0;
        cudaMemcpy(&e, err, 4, cudaMemcpyDeviceToHost);
        if (e) st = fail(WW_ERR_TIMEOUT, "ozaki GEMM wait timed out");
    }
    cudaFree(Ad); cudaFree(Bd); cudaFree(sa); cudaFree(sb);
    cudaFree(ea); cudaFree(eb); cudaFree(err);
    return st;
}
