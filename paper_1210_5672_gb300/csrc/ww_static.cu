// ww_static.cu -- dtn_apply_static: the Dirichlet-to-Neumann operator of one
// surface (assembly, factorisation and multi-right-hand-side apply, the same
// kernels as dtn_setup + dtn_apply) in a single call that allocates nothing.
//
// Some callers cannot allocate device memory at the time they need the
// operator: code under a memory-pool or allocator policy that forbids
// cudaMalloc, plug-ins of a host application that owns every allocation, or
// real-time loops that must not touch the allocator.  They pass only their
// inputs and outputs; the workspace is the file-scope device array below,
// sized for N <= WW_STATIC_MAX_N and nrhs <= WW_STATIC_MAX_RHS (1.7 MB, held
// by every GPU that loads the library until the process exits).
//
// Host code cannot use the array's name as a device address: the first call
// on each device, with that device current, looks the address up with
// cudaGetSymbolAddress (and raises the LU kernel's shared-memory limit there),
// and every call passes that address to the kernels.
//
// The array is shared by every call on a device and keeps the last call's
// contents; only the status word has to start at zero and is cleared here.
// The call uploads its small tables from host memory, reads the status word
// back and synchronises its stream before it returns.  Calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// the array: serialise them.
#include <mutex>

#include "ww_internal.cuh"

namespace ww {

namespace {

constexpr int SN = WW_STATIC_MAX_N;
constexpr int SR = WW_STATIC_MAX_RHS;
constexpr int SNB = LU_NB < SN ? LU_NB : SN;

// workspace layout, in doubles
constexpr size_t OFF_TW = 0;                                   // N/2 double2
constexpr size_t OFF_CS = OFF_TW + SN;                         // 3N
constexpr size_t OFF_GEO = OFF_CS + 3 * SN;                    // 7N: eta, eta', eta'', phi', E, 1/E, curv
constexpr size_t OFF_A = OFF_GEO + 7 * SN;                     // N^2
constexpr size_t OFF_G = OFF_A + (size_t)SN * SN;              // N^2
constexpr size_t OFF_DINV = OFF_G + (size_t)SN * SN;           // (N/nb) 2 nb^2
constexpr size_t OFF_M = OFF_DINV + (size_t)(SN / SNB) * 2 * SNB * SNB;
constexpr size_t OFF_GAM = OFF_M + (size_t)SN * SR;
constexpr size_t OFF_GOUT = OFF_GAM + (size_t)SN * SR;
constexpr size_t OFF_STATUS = OFF_GOUT + (size_t)SN * SR;      // one int (in a double slot)
constexpr size_t STATIC_DOUBLES = OFF_STATUS + 2;

__device__ __align__(256) double g_static_ws[STATIC_DOUBLES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double *g_ws_ptr[MAX_DEVICES] = {};

// device address of the workspace on the current device (looked up once per device)
int workspace(double **out) {
    int dev = 0;
    WW_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) return fail(WW_ERR_ARG, "dtn_apply_static: device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ws_ptr[dev]) {
        // publish the address only once the whole set-up has succeeded, so that a
        // failed first call is repeated (with its own error) by the next one
        WW_TRY(prepare_dense());   // shared-memory limit of the LU block kernel on this device
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_ws);
        if (e != cudaSuccess)
            return fail(WW_ERR_CUDA, std::string("dtn_apply_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_ws_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_ws_ptr[dev];
    return WW_OK;
}

}  // namespace
}  // namespace ww

using namespace ww;

extern "C" int dtn_apply_static(const double *eta, const double *phi, int N, int nrhs, double h, double *Gphi,
                                void *stream) {
    if (!eta || !phi || !Gphi) return fail(WW_ERR_ARG, "dtn_apply_static: NULL argument");
    if (N < 16 || N > WW_STATIC_MAX_N || (N & (N - 1)))
        return fail(WW_ERR_ARG, "dtn_apply_static: N must be a power of two in [16, WW_STATIC_MAX_N]");
    if (nrhs < 1 || nrhs > WW_STATIC_MAX_RHS)
        return fail(WW_ERR_ARG, "dtn_apply_static: nrhs must be in [1, WW_STATIC_MAX_RHS]");
    if (!(h > 0.0)) return fail(WW_ERR_ARG, "dtn_apply_static: h must be > 0 (INFINITY for deep water)");
    double *ws = nullptr;
    WW_TRY(workspace(&ws));

    // a host-side context whose buffers are slices of the static workspace
    Ctx c;
    memset(&c, 0, sizeof(c));
    c.N = N;
    while ((1 << c.logN) < N) ++c.logN;
    c.n = nrhs;
    c.nc = nrhs + 1;
    c.NC = nrhs;
    c.h = h;
    c.deep = isinf(h);
    c.nb = N < LU_NB ? N : LU_NB;
    c.precision = WW_FP64;
    c.stream = static_cast<cudaStream_t>(stream);
    c.tw = reinterpret_cast<double2 *>(ws + OFF_TW);
    c.cs = ws + OFF_CS;
    double *geo = ws + OFF_GEO;
    c.eta = geo;
    c.eta_x = geo + N;
    c.eta_xx = geo + 2 * N;
    c.phi_s = geo + 3 * N;
    c.E = geo + 4 * N;
    c.Einv = geo + 5 * N;
    c.curv = geo + 6 * N;
    c.A = ws + OFF_A;
    c.G = ws + OFF_G;
    c.Dinv = ws + OFF_DINV;
    c.M = ws + OFF_M;
    c.Gam = ws + OFF_GAM;
    c.Gout = ws + OFF_GOUT;
    c.status = reinterpret_cast<int *>(ws + OFF_STATUS);

    // tables on the host stack, copied into the workspace
    double tw[SN], cs[3 * SN];
    fill_tables(N, tw, cs);
    WW_CUDA_TRY(cudaMemcpyAsync(c.tw, tw, sizeof(double) * N, cudaMemcpyHostToDevice, c.stream));
    WW_CUDA_TRY(cudaMemcpyAsync(c.cs, cs, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, c.stream));
    WW_CUDA_TRY(cudaMemsetAsync(c.status, 0, sizeof(int), c.stream));

    WW_TRY(launch_base_geometry(&c, eta, nullptr, 0));
    WW_TRY(launch_assemble(&c));
    WW_TRY(lu_factor_fp64(&c));
    WW_TRY(launch_copy_cols(&c, phi, nrhs, c.M));
    WW_TRY(lu_solve_fp64(&c, c.M, nrhs));
    WW_TRY(launch_gamma(&c, 0, nrhs));
    WW_TRY(dgemm(c.stream, N, nrhs, N, 1.0, c.G, N, c.Gam, N, 1.0, c.Gout, N));
    WW_TRY(launch_copy_cols(&c, c.Gout, nrhs, Gphi));

    int st = 0;
    WW_CUDA_TRY(cudaMemcpyAsync(&st, c.status, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    WW_CUDA_TRY(cudaStreamSynchronize(c.stream));
    if (st & (ST_GEOMETRY | ST_NONFINITE))
        return fail(WW_ERR_GEOMETRY, "dtn_apply_static: surface touches the bottom or data are non-finite");
    return WW_OK;
}
