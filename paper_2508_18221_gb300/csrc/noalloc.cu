// Context-free CFL time step that allocates nothing (grmhd_cfl_dt_noalloc).
//
// Same quantity as grmhd_cfl_dt: dt = cfl * hmin / max over nodes of
// lambda = |beta|_gamma + max(alpha, sqrt(2 alpha)).  The reduction runs in two passes
// (per-block maxima, then one block over the maxima) and keeps its per-block maxima in
// the file-scope device array below instead of memory obtained from cudaMalloc.
#include <cuda.h>
#include <cuda_runtime.h>

#include <math.h>
#include <mutex>

#include "grmhd_internal.h"

namespace {

constexpr int kBlock = 256;
// Partial maxima of up to kMaxBlocks blocks: 512 KiB per device, so at most
// kMaxBlocks * kBlock = 16,777,216 nodes per call.
constexpr int kMaxBlocks = 65536;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_cfl_partials[kMaxBlocks];

// Device address of g_cfl_partials per device ordinal, looked up on the first call made
// with that device current.  In host code the symbol itself is only a host-side stand-in.
// The address belongs to the device's context: a cudaDeviceReset destroys that context
// and the next one may load the module elsewhere, so each entry also records the unique
// id of the context it was looked up in and is looked up again when the id differs.
double* g_partials_addr[kMaxDevices];
unsigned long long g_partials_ctx[kMaxDevices];
std::mutex g_setup_lock;

typedef CUresult (*ctx_get_current_fn)(CUcontext*);
typedef CUresult (*ctx_get_id_fn)(CUcontext, unsigned long long*);
ctx_get_current_fn g_ctx_get_current;
ctx_get_id_fn g_ctx_get_id;
bool g_driver_looked_up;

// Unique id of the current context (driver entry points found through the runtime, so
// the library does not link the driver library); 0 when the driver does not provide it.
unsigned long long current_context_id() {
    if (!g_driver_looked_up) {
        g_driver_looked_up = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<ctx_get_current_fn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<ctx_get_id_fn>(f);
    }
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&c) != CUDA_SUCCESS || !c || g_ctx_get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

__global__ void __launch_bounds__(kBlock) k_cfl_partial(long long P, const double* __restrict__ U,
                                                        double* __restrict__ partials) {
    __shared__ double warp_max[kBlock / 32];
    long long p = blockIdx.x * (long long)kBlock + threadIdx.x;
    double lam = 0.0;
    if (p < P) {
        using namespace gk;
        double e4 = exp(4.0 * U[V_PHI * P + p]);
        double b[3] = {U[V_BETA * P + p], U[(V_BETA + 1) * P + p], U[(V_BETA + 2) * P + p]};
        const int sidx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
        double bb = 0.0;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) bb += b[i] * b[j] * U[(V_GT + sidx[i][j]) * P + p];
        double al = U[V_ALPHA * P + p];
        lam = sqrt(e4 * bb) + fmax(al, sqrt(2.0 * al));
        if (!(lam >= 0.0)) lam = INFINITY;
    }
    for (int o = 16; o > 0; o >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
    if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = lam;
    __syncthreads();
    if (threadIdx.x < 32) {
        double m = threadIdx.x < kBlock / 32 ? warp_max[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) partials[blockIdx.x] = m;
    }
}

__global__ void __launch_bounds__(1024) k_cfl_final(int nblocks, const double* __restrict__ partials,
                                                    double hmin, double cfl, double* dt) {
    __shared__ double warp_max[32];
    double m = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) m = fmax(m, partials[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x + 31) / 32 ? warp_max[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) *dt = cfl * hmin / v;
    }
}

}  // namespace

extern "C" int grmhd_cfl_dt_noalloc(const double* state, long long n_points, double hmin, double cfl,
                                    double* dt_out, void* cuda_stream) {
    if (!state || !dt_out || n_points < 1 || !(hmin > 0.0) || !(cfl > 0.0)) return GRMHD_EINVAL;
    long long nblocks = (n_points + kBlock - 1) / kBlock;
    if (nblocks > kMaxBlocks) return GRMHD_EINVAL;  // more than 16,777,216 nodes
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GRMHD_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return GRMHD_EUNSUPPORTED;
    double* partials = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_setup_lock);
        // (before the runtime's first call on this thread no context may be current: the
        // id is then 0 and the lookup below, which makes the primary context current,
        // runs and records the id it finds afterwards)
        unsigned long long ctx_id = current_context_id();
        if (!g_partials_addr[dev] || ctx_id == 0 || g_partials_ctx[dev] != ctx_id) {
            void* addr = nullptr;
            if (cudaGetSymbolAddress(&addr, g_cfl_partials) != cudaSuccess || !addr) return GRMHD_ECUDA;
            g_partials_addr[dev] = static_cast<double*>(addr);
            g_partials_ctx[dev] = current_context_id();
        }
        partials = g_partials_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    k_cfl_partial<<<(unsigned)nblocks, kBlock, 0, s>>>(n_points, state, partials);
    k_cfl_final<<<1, 1024, 0, s>>>((int)nblocks, partials, hmin, cfl, dt_out);
    return cudaGetLastError() == cudaSuccess ? GRMHD_OK : GRMHD_ECUDA;
}
