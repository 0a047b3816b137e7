// ww_tcgemm.cu -- tensor-core GEMM on sliced operands (tcgen05 + TMA + TMEM).
//
//   C (+)= alpha * sum_{(p,q) in pairs} A_p * B_q^T
//
// A_p (M x K) and B_q (Nn x K) are bf16 "slices" stored K-contiguous, stacked
// slice after slice ([S][rows][K]).  Writing an FP32 (or FP64) operand as a
// sum of bf16 slices and keeping the products whose combined significance is
// large gives an FP32-accurate (or better) product on the bf16 tensor cores,
// whose rate on GB300 is ~1.9 PFLOP/s against 70 TFLOP/s for FP32 FMA and
// 1 TFLOP/s for FP64.
//
// One CTA computes a 128 x BN tile.  Warps 0 and 6 issue the TMA loads of the
// A and the B slices of a 64-wide K chunk into a ring of 2-4 stages; warp 1 owns the TMEM accumulator and
// issues tcgen05.mma (M = 128, N = BN, K = 16) for every pair; warps 2..5 read
// the accumulator with tcgen05.ld and write C.  Every mbarrier wait is
// bounded (~1 s); a timeout sets *err and the block still exits.
#include <cudaTypedefs.h>

#include <mutex>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "ww_internal.cuh"
#include "ww_tc.cuh"

namespace ww {

namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;   // K chunk of the 128-byte-swizzled tiles; 32 uses 64-byte swizzle
// warps: 0 producer of the A slices, 1 MMA, 2..5 epilogue, 6 producer of the
// B slices (one thread issues a TMA load only every ~145 ns, so two issuers)
constexpr int TC_THREADS = 224;
constexpr int TC_PROD2 = 6;

struct Pairs {
    int n;
    unsigned char p[16], q[16];
};

}  // namespace

// Where a product goes (ww_tc.cuh declares the struct; modes:
//   0: Cf = alpha C (FP32)      1: Cd = alpha C      2: Cd += alpha C
//   3: the 3 bf16 slices of W = shift I - C, column-major as a right operand
//      (s_col[k][j][i] = slice k of W(i, j)), and max|W - shift/2 I| into dev_max
//   4: Cf = C, plus the 3 slices of C as a right operand (s_col) and as a left
//      operand (s_row[k][i][j]), and 2 more left-operand slices (s_row2)).
namespace {

// ring depth: as many K-chunk stages as fit in 216 KB (MINB = 1 CTA per SM)
// or 104 KB (MINB = 2: two CTAs share an SM, so that one's epilogue overlaps
// the other's main loop), at most 4
template <int BN, int SA, int SB, int BK = TC_BK, int MINB = 1>
struct TcSmem {
    static constexpr int A_TILE = TC_BM * BK * 2;   // bytes
    static constexpr int B_TILE = BN * BK * 2;
    static constexpr int STAGE = SA * A_TILE + SB * B_TILE;
    static constexpr int BUDGET = (MINB == 1 ? 216 : 104) * 1024;
    static constexpr int STAGES = (BUDGET / STAGE) < 4 ? (BUDGET / STAGE) : 4;
    static constexpr int BYTES = STAGES * STAGE + 1024 /* align */ + 256 /* barriers */;
};

template <int BN, int SA, int SB, int BK, int MINB>
__global__ void __launch_bounds__(TC_THREADS, MINB)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int Nn, int K,
              Pairs pairs, TcOut o, int *err, const int *skip) {
    if (skip && *skip) return;   // a step the caller decided on the device to leave out
    using L = TcSmem<BN, SA, SB, BK, MINB>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t base = tc::smem_u32(smem_raw);
    uint8_t *smem = smem_raw + ((1024 - (base & 1023)) & 1023);
    uint8_t *tiles = smem;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L::STAGES * L::STAGE);
    uint64_t *empty = full + L::STAGES;
    uint64_t *done = empty + L::STAGES;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * BN;
    const int nk = K / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < L::STAGES; ++s) {
            tc::mbar_init(&full[s], 2);   // one arrival (with its bytes) from each producer
            tc::mbar_init(&empty[s], 1);  // the MMA commit; both producers wait on the same phase
        }
        tc::mbar_init(done, 1);
        tc::mbar_fence_init();
        tc::prefetch_tmap(&tmA);
        tc::prefetch_tmap(&tmB);
    }
    if (warp == 1) {
        tc::tmem_alloc(tslot, BN);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0 || warp == TC_PROD2) {
        // ---------------- TMA producers: A slices (warp 0), B slices (warp 6)
        const uint32_t leader = tc::elect_one();
        const bool pa = warp == 0;
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % L::STAGES;
            const uint32_t ph = (kc / L::STAGES) & 1;
            tc::mbar_wait(&empty[s], ph ^ 1, err);
            tc::mbar_arrive_expect_tx_if(leader, &full[s], pa ? SA * L::A_TILE : SB * L::B_TILE);
            uint8_t *st = tiles + s * L::STAGE;
            if (pa) {
#pragma unroll
                for (int a = 0; a < SA; ++a)
                    tc::tma_load_2d_if(leader, &tmA, &full[s], st + a * L::A_TILE, kc * BK, a * M + m0);
            } else {
#pragma unroll
                for (int b = 0; b < SB; ++b)
                    tc::tma_load_2d_if(leader, &tmB, &full[s], st + SA * L::A_TILE + b * L::B_TILE, kc * BK,
                                       b * Nn + n0);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (whole warp, one elected lane issues)
        const uint32_t leader = tc::elect_one();
        constexpr uint32_t idesc = tc::idesc_bf16(TC_BM, BN);
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % L::STAGES;
            const uint32_t ph = (kc / L::STAGES) & 1;
            tc::mbar_wait(&full[s], ph, err);
            tc::fence_after();
            const uint32_t st = tc::smem_u32(tiles + s * L::STAGE);
            for (int pi = 0; pi < pairs.n; ++pi) {
                const uint32_t sa_ = st + pairs.p[pi] * L::A_TILE, sb_ = st + SA * L::A_TILE + pairs.q[pi] * L::B_TILE;
                const uint64_t da = BK == 64 ? tc::desc_k128(sa_) : tc::desc_k64(sa_);
                const uint64_t db = BK == 64 ? tc::desc_k128(sb_) : tc::desc_k64(sb_);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)   // +32 B per K step: +2 in the start-address field
                    tc::mma_bf16_if(leader, tmem, da + 2 * kk, db + 2 * kk, idesc, (kc | pi | kk) != 0);
            }
            tc::mma_commit_if(leader, &empty[s]);   // frees this stage once its MMAs have read it
        }
        tc::mma_commit_if(leader, done);
    } else if (warp >= 2 && warp < TC_PROD2) {
        // ---------------- epilogue: TMEM -> registers -> C (column-major)
        const int quarter = warp & 3;   // TMEM lanes 32*quarter .. +31
        const int row = m0 + quarter * 32 + lane;
        tc::mbar_wait(done, 0, err);
        tc::fence_after();
        float dmax = 0.f;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + c0, v);
            if (row < M) {
                if (o.mode <= 2) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int col = n0 + c0 + j;
                        if (col < Nn) {
                            const size_t idx = (size_t)col * o.ldc + row;
                            if (o.mode == 0)
                                o.Cf[idx] = v[j] * (float)o.alpha;   // fp32 result: no FP64 work
                            else if (o.mode == 1)
                                o.Cd[idx] = o.alpha * (double)v[j];
                            else
                                o.Cd[idx] += o.alpha * (double)v[j];
                        }
                    }
                } else if (o.mode == 3) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int col = n0 + c0 + j;
                        if (col < Nn) {
                            const bool dg = col == row;
                            float w = (dg ? o.shift : 0.f) - v[j];
                            dmax = fmaxf(dmax, fabsf(w - (dg ? 0.5f * o.shift : 0.f)));
#pragma unroll
                            for (int k = 0; k < 3; ++k) {
                                const __nv_bfloat16 b = __float2bfloat16_rn(w);
                                o.s_col[((size_t)k * Nn + col) * M + row] = b;
                                w -= __bfloat162float(b);
                            }
                        }
                    }
                } else if (n0 + c0 < Nn) {   // mode 4 (square products, whole 32-column groups)
#pragma unroll
                    for (int g = 0; g < 4; ++g) {   // 8 columns at a time: one 16-byte store per slice
                        uint32_t pk[3][4];
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) {
                            const int j = 8 * g + jj, col = n0 + c0 + j;
                            o.Cf[(size_t)col * o.ldc + row] = v[j];
                            float w = v[j];
#pragma unroll
                            for (int k = 0; k < 3; ++k) {
                                const __nv_bfloat16 b = __float2bfloat16_rn(w);
                                o.s_col[((size_t)k * Nn + col) * M + row] = b;
                                const uint32_t u = (uint32_t)__bfloat16_as_ushort(b);
                                if (jj & 1)
                                    pk[k][jj >> 1] |= u << 16;
                                else
                                    pk[k][jj >> 1] = u;
                                w -= __bfloat162float(b);
                            }
                        }
                        const size_t off = (size_t)row * Nn + n0 + c0 + 8 * g;
#pragma unroll
                        for (int k = 0; k < 3; ++k)
                            *reinterpret_cast<uint4 *>(o.s_row + (size_t)k * M * Nn + off) =
                                make_uint4(pk[k][0], pk[k][1], pk[k][2], pk[k][3]);
#pragma unroll
                        for (int k = 0; k < 2; ++k)
                            *reinterpret_cast<uint4 *>(o.s_row2 + (size_t)k * M * Nn + off) =
                                make_uint4(pk[k][0], pk[k][1], pk[k][2], pk[k][3]);
                    }
                }
            }
        }
        if (o.mode == 3 && o.dev_max) {
            for (int off = 16; off > 0; off >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
            if (lane == 0) atomicMax(o.dev_max, __float_as_uint(dmax));
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, BN);
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

int get_encoder() {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_encode) return fail(WW_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    return WW_OK;
}

}  // namespace

// resolve the CUDA driver's tensor-map encoder outside any stream capture
int tc_init() { return get_encoder(); }

// 2-D bf16 tensor [rows][K] (K contiguous), tile box {64, box_rows}, 128-byte swizzle
int tc_make_map(CUtensorMap *map, const void *ptr, int K, long rows, int box_rows, int box_k) {
    WW_TRY(get_encoder());
    // the caller's buffer holds at least box_rows rows; rows past the logical
    // end only feed output rows / columns that the epilogue discards
    if (rows < box_rows) rows = box_rows;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    if (box_k != 64 && box_k != 32) return fail(WW_ERR_ARG, "tc_make_map: K box must be 64 or 32");
    cuuint32_t box[2] = {(cuuint32_t)box_k, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, box_k == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(WW_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return WW_OK;
}

namespace {

template <int BN, int SA, int SB, int BK = TC_BK, int MINB = 1>
int launch_tc(cudaStream_t s, const void *A, const void *B, int M, int Nn, int K, const Pairs &pairs, const TcOut &o,
              int *err, const int *skip) {
    if (o.mode == 4 && (M != Nn || Nn % 32 != 0))
        return fail(WW_ERR_ARG, "tc_gemm: slice output needs a square product with N a multiple of 32");
    using L = TcSmem<BN, SA, SB, BK, MINB>;
    static_assert(MINB == 1 || L::STAGES >= 2, "two CTAs per SM need two stages each");
    static_assert(L::BYTES <= 227 * 1024, "shared memory");
    if (K % BK != 0) return fail(WW_ERR_ARG, "tc_gemm: K must be a multiple of the K chunk");
    CUtensorMap ta, tb;
    WW_TRY(tc_make_map(&ta, A, K, (long)SA * M, TC_BM, BK));
    WW_TRY(tc_make_map(&tb, B, K, (long)SB * Nn, BN, BK));
    auto kern = k_tc_gemm<BN, SA, SB, BK, MINB>;
    WW_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::BYTES));
    dim3 grid((M + TC_BM - 1) / TC_BM, (Nn + BN - 1) / BN);
    kern<<<grid, TC_THREADS, L::BYTES, s>>>(ta, tb, M, Nn, K, pairs, o, err, skip);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

// ---------------------------------------------------------------- slicing
// dst[s][r][k] (bf16, K contiguous) from a column-major source:
//   trans = 1: value(r, k) = src[r + k*ld]   (A side: rows of the source)
//   trans = 0: value(r, k) = src[k + r*ld]   (B side: columns of the source)
// optionally v -> shift*delta(r,k) - v.  S bf16 slices, v = sum_s slice_s + O(2^-8S |v|).
template <typename T>
__global__ void k_slice(const T *__restrict__ src, int ld, int rows, int K, int trans, float shift, int S,
                        __nv_bfloat16 *dst, unsigned *dev_max, const int *skip, int run_if_skipped) {
    // skip: a device decision; run_if_skipped inverts it (this slice replaces a skipped step's output)
    if (skip && ((*skip != 0) != (run_if_skipped != 0))) return;
    __shared__ float tile[32][33];
    float dmax = 0.f;   // with shift = 2: max |(2 delta - v) - delta| = max |delta - v|
    const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
    for (int yy = ty; yy < 32; yy += 8) {
        float v;
        if (trans) {
            // read coalesced along r (column-major source), tile[k][r]
            const int r = r0 + tx, k = k0 + yy;
            v = (r < rows && k < K) ? (float)src[(size_t)k * ld + r] : 0.f;
            if (shift != 0.f) v = (r == k ? shift : 0.f) - v;
            tile[yy][tx] = v;
        } else {
            const int k = k0 + tx, r = r0 + yy;
            v = (r < rows && k < K) ? (float)src[(size_t)r * ld + k] : 0.f;
            if (shift != 0.f) {
                v = (r == k ? shift : 0.f) - v;
                if (r < rows && k < K) dmax = fmaxf(dmax, fabsf(v - (r == k ? 0.5f * shift : 0.f)));
            }
            tile[tx][yy] = v;
        }
    }
    if (dev_max) {
        for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        if ((threadIdx.x & 31) == 0) atomicMax(dev_max, __float_as_uint(dmax));
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
        const int r = r0 + yy, k = k0 + tx;
        if (r >= rows || k >= K) continue;
        float v = tile[tx][yy];
        for (int s = 0; s < S; ++s) {
            __nv_bfloat16 b = __float2bfloat16_rn(v);
            dst[((size_t)s * rows + r) * K + k] = b;
            v -= __bfloat162float(b);
        }
    }
}

}  // namespace

int tc_slice_f32(cudaStream_t s, const float *src, int ld, int rows, int K, int trans, float shift, int S,
                 __nv_bfloat16 *dst, unsigned *dev_max, const int *skip, int run_if_skipped) {
    dim3 grid((K + 31) / 32, (rows + 31) / 32);
    k_slice<float><<<grid, 256, 0, s>>>(src, ld, rows, K, trans, shift, S, dst, dev_max, skip, run_if_skipped);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

int tc_slice_f64(cudaStream_t s, const double *src, int ld, int rows, int K, int trans, float shift, int S,
                 __nv_bfloat16 *dst, const int *skip) {
    dim3 grid((K + 31) / 32, (rows + 31) / 32);
    k_slice<double><<<grid, 256, 0, s>>>(src, ld, rows, K, trans, shift, S, dst, nullptr, skip, 0);
    WW_CUDA_TRY(cudaGetLastError());
    return WW_OK;
}

// FP32-accurate product from 3 + 3 slices (pairs with p + q <= 2, 0-based):
// out_mode 0: Cf = alpha A B^T (fp32); 1: Cd = alpha A B^T; 2: Cd += alpha A B^T
int tc_gemm_f32acc(cudaStream_t s, const __nv_bfloat16 *A3, const __nv_bfloat16 *B3, int M, int Nn, int K,
                   int out_mode, float *Cf, double *Cd, int ldc, double alpha, int *err, const int *skip) {
    if (K % TC_BK != 0) return fail(WW_ERR_ARG, "tc_gemm: K must be a multiple of 64");
    Pairs P{};
    const int pp[6] = {2, 1, 0, 1, 0, 0}, qq[6] = {0, 1, 2, 0, 1, 0};   // smallest terms first
    P.n = 6;
    for (int i = 0; i < 6; ++i) {
        P.p[i] = (unsigned char)pp[i];
        P.q[i] = (unsigned char)qq[i];
    }
    TcOut o{};
    o.mode = out_mode;
    o.Cf = Cf;
    o.Cd = Cd;
    o.ldc = ldc;
    o.alpha = alpha;
    return launch_tc<128, 3, 3, 32>(s, A3, B3, M, Nn, K, P, o, err, skip);
}

// Product from 2 + 2 slices (pairs with p + q <= 1): relative accuracy ~2^-16,
// for the refinement corrections X R, whose error only adds to the contraction
// of the iteration (the residuals themselves are FP64-accurate).  Reads slices
// 0 and 1 of 2- or 3-slice operands.
int tc_gemm_2x2(cudaStream_t s, const __nv_bfloat16 *A2, const __nv_bfloat16 *B2, int M, int Nn, int K, int out_mode,
                float *Cf, double *Cd, int ldc, double alpha, int *err, const int *skip, int bn) {
    if (K % TC_BK != 0) return fail(WW_ERR_ARG, "tc_gemm: K must be a multiple of 64");
    Pairs P{};
    const int pp[3] = {1, 0, 0}, qq[3] = {0, 1, 0};   // smallest terms first
    P.n = 3;
    for (int i = 0; i < 3; ++i) {
        P.p[i] = (unsigned char)pp[i];
        P.q[i] = (unsigned char)qq[i];
    }
    TcOut o{};
    o.mode = out_mode;
    o.Cf = Cf;
    o.Cd = Cd;
    o.ldc = ldc;
    o.alpha = alpha;
    // column tile from the schedule: 64 (default) gives 2x the CTAs of 128-wide
    // tiles for the narrow (513-column) products, 32 4x for a handful of columns
    if (bn == 32) return launch_tc<32, 2, 2>(s, A2, B2, M, Nn, K, P, o, err, skip);
    if (bn == 128) return launch_tc<128, 2, 2>(s, A2, B2, M, Nn, K, P, o, err, skip);
    return launch_tc<64, 2, 2>(s, A2, B2, M, Nn, K, P, o, err, skip);
}

// FP32-accurate product with a sliced output (modes 3 and 4 of TcOut), 3 + 3 slices
int tc_gemm_f32acc_sliced(cudaStream_t s, const __nv_bfloat16 *A3, const __nv_bfloat16 *B3, int M, int Nn, int K,
                          const TcOut &o, int *err, const int *skip, int bn, int ctas) {
    if (K % TC_BK != 0) return fail(WW_ERR_ARG, "tc_gemm: K must be a multiple of 64");
    Pairs P{};
    const int pp[6] = {2, 1, 0, 1, 0, 0}, qq[6] = {0, 1, 2, 0, 1, 0};   // smallest terms first
    P.n = 6;
    for (int i = 0; i < 6; ++i) {
        P.p[i] = (unsigned char)pp[i];
        P.q[i] = (unsigned char)qq[i];
    }
    // 32-wide K chunks (64-byte swizzle): 4 stages of 48 KB instead of 2 of 96 KB;
    // 64-wide column tiles (schedule) double the CTAs of small products; 256-wide
    // ones (3 stages of 72 KB) load a third fewer operand bytes per flop; two
    // CTAs per SM (2 stages each) overlap one tile's epilogue with another's MMAs
    if (ctas == 2 && bn == 64) return launch_tc<64, 3, 3, 32, 2>(s, A3, B3, M, Nn, K, P, o, err, skip);
    if (ctas == 2) return launch_tc<128, 3, 3, 32, 2>(s, A3, B3, M, Nn, K, P, o, err, skip);
    if (bn == 64) return launch_tc<64, 3, 3, 32>(s, A3, B3, M, Nn, K, P, o, err, skip);
    if (bn == 256) return launch_tc<256, 3, 3, 32>(s, A3, B3, M, Nn, K, P, o, err, skip);
    return launch_tc<128, 3, 3, 32>(s, A3, B3, M, Nn, K, P, o, err, skip);
}

}  // namespace ww

// -------------------------------------------------------------------------
// self-test (declared in ww.h): C = A B with A (M x K), B (K x Nn) column-major
// FP64 device arrays through the 3x3-slice tensor-core path; returns the
// max |C - C_fp64| / max |C_fp64| against the FP64 DGEMM of the library.
// -------------------------------------------------------------------------
extern "C" int ww_selftest_f32gemm(const double *A, const double *B, int M, int Nn, int K, double *C) {
    using namespace ww;
    if (!A || !B || !C || M < 1 || Nn < 1 || K < 64 || K % 64)
        return fail(WW_ERR_ARG, "ww_selftest_f32gemm: NULL pointer or bad sizes (K a multiple of 64)");
    cudaStream_t s = nullptr;
    __nv_bfloat16 *As = nullptr, *Bs = nullptr;
    int *err = nullptr;
    int st = WW_OK;
    if (cudaMalloc(&As, sizeof(__nv_bfloat16) * (3 * (size_t)M + 256) * K) != cudaSuccess ||
        cudaMalloc(&Bs, sizeof(__nv_bfloat16) * (3 * (size_t)Nn + 256) * K) != cudaSuccess ||
        cudaMalloc(&err, sizeof(int)) != cudaSuccess)
        st = fail(WW_ERR_ALLOC, "selftest alloc");
    if (st == WW_OK && cudaMemset(err, 0, sizeof(int)) != cudaSuccess) st = fail(WW_ERR_CUDA, "selftest memset");
    if (st == WW_OK) st = tc_slice_f64(s, A, M, M, K, 1, 0.f, 3, As, nullptr);
    if (st == WW_OK) st = tc_slice_f64(s, B, K, Nn, K, 0, 0.f, 3, Bs, nullptr);
    if (st == WW_OK) st = tc_gemm_f32acc(s, As, Bs, M, Nn, K, 1, nullptr, C, M, 1.0, err, nullptr);
    if (st == WW_OK && cudaDeviceSynchronize() != cudaSuccess) st = fail(WW_ERR_CUDA, "selftest sync");
    if (st == WW_OK) {
        int e = 0;
        cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e) st = fail(WW_ERR_TIMEOUT, "tensor-core GEMM wait timed out");
    }
    cudaFree(As);
    cudaFree(Bs);
    cudaFree(err);
    return st;
}

// C = A B with the FP64 DGEMM of the plain form (the same kernel as its LU
// updates, triangular-solve updates and G apply)
extern "C" int ww_selftest_dgemm(const double *A, const double *B, int M, int Nn, int K, double *C) {
    using namespace ww;
    if (!A || !B || !C || M < 1 || Nn < 1 || K < 1) return fail(WW_ERR_ARG, "ww_selftest_dgemm: bad arguments");
    WW_TRY(dgemm(nullptr, M, Nn, K, 1.0, A, M, B, K, 0.0, C, M));
    WW_CUDA_TRY(cudaDeviceSynchronize());
    return WW_OK;
}
