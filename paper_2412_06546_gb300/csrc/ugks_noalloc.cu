// ugks_noalloc.cu -- residual reduction that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs under an external memory
// manager which has already reserved the device memory, a serving loop that
// admits work against a fixed device budget and must not take hidden
// allocations, or a monitoring hook that must not synchronise the device (which
// cudaMalloc and cudaFree may do).  ugks_residual_noalloc serves them: it
// computes the same residual as ugks_residual, from two conserved-variable
// arrays the caller already holds on the device, and keeps its block partial
// sums in a fixed file-scope device array instead of allocated scratch.
#include "../../include/ugks.h"

#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 8192;                       // => at most 2,097,152 cells
constexpr int kMaxM = 5;                               // D + 2 for D = 3
constexpr long long kMaxCells = (long long)kMaxBlocks * kThreads;

// Block partial sums: [block][2M] = sum (W_new - W_old)^2, sum W_old^2 per
// component.  655 KB held by every device that loads the library, for the life
// of the process.  Every call shares it.
static __device__ __align__(256) double g_res_scratch[kMaxBlocks * 2 * kMaxM];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
// per device: the context in which the array's address was looked up, and the
// address.  A new context on the device (after cudaDeviceReset, or a primary
// context released and created again) maps the array elsewhere, so the address
// is looked up again whenever the current context differs.
struct ScratchSlot {
    CUcontext ctx;
    double *ptr;
};
ScratchSlot g_scratch[kMaxDevices] = {};

// cuCtxGetCurrent through the runtime's driver entry point (the library links
// only the CUDA runtime)
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
cudaError_t current_context(CUcontext *ctx)
{
    static std::once_flag once;
    static CtxGetCurrentFn fn = nullptr;
    static cudaError_t lookup = cudaSuccess;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSuccess;
        lookup = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q);
        if (lookup == cudaSuccess && q != cudaDriverEntryPointSuccess) lookup = cudaErrorSymbolNotFound;
        fn = reinterpret_cast<CtxGetCurrentFn>(p);
    });
    if (lookup != cudaSuccess) return lookup;
    return fn(ctx) == CUDA_SUCCESS ? cudaSuccess : cudaErrorUnknown;
}


template <int M>
__global__ void k_residual_partials(const double *__restrict__ W_old, const double *__restrict__ W_new,
                                    long long n, double *scratch)
{
    __shared__ double red[2 * M][kThreads / 32];
    const long long c = (long long)blockIdx.x * kThreads + threadIdx.x;
    double dsq[M], wsq[M];
#pragma unroll
    for (int m = 0; m < M; ++m) dsq[m] = wsq[m] = 0.0;
    if (c < n) {
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const double o = W_old[c * M + m], d = W_new[c * M + m] - o;
            dsq[m] = d * d;
            wsq[m] = o * o;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        double a = dsq[m], b = wsq[m];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
            red[m][warp] = a;
            red[M + m][warp] = b;
        }
    }
    __syncthreads();
    // every slot of this block is written, so no slot needs clearing between calls
    if (threadIdx.x < 2 * M) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[threadIdx.x][w];
        scratch[(size_t)blockIdx.x * 2 * M + threadIdx.x] = s;
    }
}

template <int M>
__global__ void k_residual_final(const double *scratch, int nblocks, double *res)
{
    __shared__ double acc[2 * M][32];
    const int t = threadIdx.x;
    for (int i = 0; i < 2 * M; ++i) {
        double s = 0.0;
        for (int b = t; b < nblocks; b += 32) s += scratch[(size_t)b * 2 * M + i];
        acc[i][t] = s;
    }
    __syncwarp();
    if (t < M) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 32; ++w) {
            a += acc[t][w];
            b += acc[M + t][w];
        }
        res[t] = b > 0.0 ? sqrt(a) / sqrt(b) : sqrt(a);
    }
}

}  // namespace

namespace ugks {
void set_last_error(const std::string &msg);   // message returned by ugks_last_error()
}

namespace {
ugks_status fail(ugks_status code, const std::string &msg)
{
    ugks::set_last_error(msg);
    return code;
}
}  // namespace

extern "C" ugks_status ugks_residual_noalloc(const double *W_old, const double *W_new, int64_t n_cells, int32_t dim,
                                             double *res, void *stream)
{
    ugks::set_last_error("");
    if (dim != 2 && dim != 3) return fail(UGKS_EINVAL, "ugks_residual_noalloc: dim must be 2 or 3");
    if (n_cells <= 0) return fail(UGKS_EINVAL, "ugks_residual_noalloc: n_cells must be positive");
    if (n_cells > kMaxCells)
        return fail(UGKS_EINVAL, "ugks_residual_noalloc: n_cells " + std::to_string(n_cells) +
                                     " exceeds the fixed scratch limit of " + std::to_string(kMaxCells) + " cells");
    if (!W_old || !W_new || !res) return fail(UGKS_EINVAL, "ugks_residual_noalloc: NULL pointer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(UGKS_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(UGKS_EINVAL, "ugks_residual_noalloc: device index out of range");
    CUcontext ctx = nullptr;
    e = current_context(&ctx);
    if (e != cudaSuccess) return fail(UGKS_ECUDA, std::string("cuCtxGetCurrent: ") + cudaGetErrorString(e));
    double *scratch = nullptr;
    {
        // once per device and context, with that device current: the device
        // address of the file-scope array (its name in host code is only a
        // host-side stand-in).  The lookup makes the device's primary context
        // current if none was, so the context is read again after it.
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        ScratchSlot &slot = g_scratch[dev];
        if (!slot.ptr || !ctx || slot.ctx != ctx) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_res_scratch);
            if (e != cudaSuccess)
                return fail(UGKS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            e = current_context(&ctx);
            if (e != cudaSuccess) return fail(UGKS_ECUDA, std::string("cuCtxGetCurrent: ") + cudaGetErrorString(e));
            slot.ctx = ctx;
            slot.ptr = static_cast<double *>(p);
        }
        scratch = slot.ptr;
    }
    const int nblocks = (int)((n_cells + kThreads - 1) / kThreads);
    cudaStream_t st = (cudaStream_t)stream;
    if (dim == 2) {
        k_residual_partials<4><<<nblocks, kThreads, 0, st>>>(W_old, W_new, n_cells, scratch);
        k_residual_final<4><<<1, 32, 0, st>>>(scratch, nblocks, res);
    } else {
        k_residual_partials<5><<<nblocks, kThreads, 0, st>>>(W_old, W_new, n_cells, scratch);
        k_residual_final<5><<<1, 32, 0, st>>>(scratch, nblocks, res);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(UGKS_ECUDA, std::string("ugks_residual_noalloc launch: ") + cudaGetErrorString(e));
    return UGKS_OK;
}

