// tile_chol_precision_map_noalloc: the per-tile precision map computed without any
// allocation, for callers that cannot call cudaMalloc.
//
// Who needs this: code held to a fixed device-memory budget or to a custom allocator that
// owns all device memory and forbids runtime allocations, and real-time loops where an
// allocation's latency or failure is not acceptable.  Such callers own their input and
// output buffers and want the library to touch no other memory it has to obtain.
//
// The tile sums of squares that tile_chol_precision_map keeps in handle-owned scratch live
// here in a file-scope __device__ array of fixed size instead.  Every GPU that loads this
// library holds that array (MAX_TILES doubles, 263 KB) until the process exits.
#include "../../include/tile_chol.h"
#include "tc_internal.h"

#include <cmath>
#include <mutex>

namespace {

constexpr int MAX_NT = 256;                               // tiles per column
constexpr int MAX_TILES = MAX_NT * (MAX_NT + 1) / 2;      // 32896 lower tiles
constexpr int MAX_DEVICES = 64;

// Scratch: per-tile sums of squares of the current call.  Shared by all calls on a device.
static __device__ __align__(256) double g_sumsq[MAX_TILES];

// Device address of g_sumsq per device (host code cannot use the symbol's host-side name as
// a device address), with the context it was looked up in: after a device reset the device
// gets a new primary context, the module is loaded again and the address is looked up anew.
double *g_sumsq_addr[MAX_DEVICES] = {nullptr};
CUcontext g_sumsq_ctx[MAX_DEVICES] = {nullptr};
std::mutex g_setup_mutex;

// The current context through the runtime's driver entry point (the library does not link
// the driver library directly, so that it loads on machines without a GPU driver).
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
CUcontext current_context() {
    static CtxGetCurrentFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        fn = reinterpret_cast<CtxGetCurrentFn>(p);
    }
    CUcontext ctx = nullptr;
    return fn(&ctx) == CUDA_SUCCESS ? ctx : nullptr;
}

// A pointer the kernels may dereference on device `dev`: device (or managed) memory of that
// device.
bool on_this_device(const void *p, int dev) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();             // the query's own error (an unknown pointer), not the caller's
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

// Section IV-C criterion on the device from the tile sums of squares: ||A||_F^2 is summed
// in the same order as the host path (row by row, off-diagonal tiles twice) by one thread,
// then every tile is classified.  Same arithmetic as tile_chol_precision_map, so the maps
// are identical.
__global__ void k_map_from_sumsq(const double *sumsq, int nt, double eps_high, int band, int prec_set,
                                 uint8_t *map_out) {
    __shared__ double normA;
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < nt; ++i)
            for (int j = 0; j <= i; ++j) tot += (i == j ? 1.0 : 2.0) * sumsq[tc::tidx(i, j)];
        normA = sqrt(tot);
    }
    __syncthreads();
    const double u[4] = {ldexp(1.0, -53), ldexp(1.0, -24), ldexp(1.0, -11), ldexp(1.0, -4)};
    for (int e = threadIdx.x; e < nt * nt; e += blockDim.x) {
        const int i = e / nt, j = e % nt;
        uint8_t v = TC_FP64;
        if (j < i && i - j > band) {
            const double ratio = (double)nt * sqrt(sumsq[tc::tidx(i, j)]) / normA;
            for (int p = TC_FP8; p >= TC_FP32; --p) {
                if (p > prec_set - 1) continue;
                if (ratio < eps_high / u[p]) {
                    v = (uint8_t)p;
                    break;
                }
            }
        }
        map_out[e] = v;
    }
}

}  // namespace

extern "C" int tile_chol_precision_map_noalloc(int64_t n, int b, const double *A_tiles, double eps_high, int band,
                                               int prec_set, uint8_t *map_out, void *stream) {
    if (n < 1 || b < 64 || b > 4096 || b % 64 || !A_tiles || !map_out) return TC_ERR_ARG;
    if (!(eps_high > 0) || band < 0 || prec_set < 1 || prec_set > 4) return TC_ERR_ARG;
    const int64_t nt = (n + b - 1) / b;
    if (nt > MAX_NT) return TC_ERR_ARG;          // beyond the fixed scratch: 256 tiles per column
    // an error left pending by earlier, unrelated work stays the caller's: report it, do not
    // consume it, and launch nothing
    if (cudaPeekAtLastError() != cudaSuccess) return TC_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return TC_ERR_CUDA;
    if (!on_this_device(A_tiles, dev) || !on_this_device(map_out, dev)) return TC_ERR_ARG;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        CUcontext ctx = current_context();
        if (!ctx) return TC_ERR_CUDA;
        if (!g_sumsq_addr[dev] || g_sumsq_ctx[dev] != ctx) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_sumsq) != cudaSuccess) {
                cudaGetLastError();
                return TC_ERR_CUDA;
            }
            g_sumsq_addr[dev] = static_cast<double *>(p);
            g_sumsq_ctx[dev] = ctx;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    tc::launch_tile_sumsq(A_tiles, (int)nt, b, n, g_sumsq_addr[dev], s);
    k_map_from_sumsq<<<1, 256, 0, s>>>(g_sumsq_addr[dev], (int)nt, eps_high, band, prec_set, map_out);
    // no error was pending before the launches, so one now is theirs
    if (cudaPeekAtLastError() != cudaSuccess) {
        cudaGetLastError();
        return TC_ERR_CUDA;
    }
    return TC_OK;
}
