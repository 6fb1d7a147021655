// paris_divergence_noalloc: the divergence step (b = div(u*)/dt, mean removed)
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a solver embedded in a host
// application whose own allocator owns all device memory, or a time loop with
// a fixed memory budget that must not grow or fragment while it runs.  Such a
// caller cannot create a paris_ctx (whose workspace is allocated in
// paris_create).  This entry point needs no context: it takes the grid
// directly, the caller passes the inputs and outputs, and the block partial
// sums of the mean live in a file-scope device array of fixed size that every
// GPU loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/paris.h"
#include "common.cuh"

namespace {

using paris::Geo;

constexpr int kTX = 32, kTY = 8, kTZ = 8;  // one block covers a 32 x 8 x 8 box of cells
constexpr int kMaxBlocks = 16384;          // 512 x 256 x 256 cells at most (16 x 32 x 32 blocks)
constexpr int kNV = 1;                     // partials per block: the sum of b

// Shared scratch of every call on this device: block partials, then the
// finalized mean.  Each call overwrites all of it before reading it.
static __device__ __align__(256) double g_noalloc_scratch[kNV * kMaxBlocks + 8];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};
int g_sms[kMaxDevices] = {0};

// Address of the scratch array on the current device and that device's SM
// count, looked up once per device with the device current (the array's
// host-side name is not a device address).
cudaError_t scratch_on_current_device(double** out, int* sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_sms[dev] = n > 0 ? n : 1;
        g_scratch_addr[dev] = (double*)p;
    }
    *out = g_scratch_addr[dev];
    *sms = g_sms[dev];
    return cudaSuccess;
}

__device__ inline double div_at(const Geo& g, const double* __restrict__ u,
                                const double* __restrict__ v, const double* __restrict__ w, int i,
                                int j, int k) {
    paris::AxisNb ax = paris::axis_nb(i, g.nx, g.wx);
    paris::AxisNb ay = paris::axis_nb(j, g.ny, g.wy);
    paris::AxisNb az = paris::axis_nb(k, g.nz, g.wz);
    double up = ax.wp ? 0.0 : u[g.fx(ax.fp, j, k)];
    double um = ax.wm ? 0.0 : u[g.fx(i, j, k)];
    double vp = ay.wp ? 0.0 : v[g.fy(i, ay.fp, k)];
    double vm = ay.wm ? 0.0 : v[g.fy(i, j, k)];
    double wp = az.wp ? 0.0 : w[g.fz(i, j, az.fp)];
    double wm = az.wm ? 0.0 : w[g.fz(i, j, k)];
    return ((up - um) + (vp - vm)) + (wp - wm);
}

__global__ void __launch_bounds__(kTX* kTY)
    noalloc_div_kernel(Geo g, const double* __restrict__ u, const double* __restrict__ v,
                       const double* __restrict__ w, double inv_hdt, double* __restrict__ rhs,
                       double* scratch) {
    const int i = blockIdx.x * kTX + threadIdx.x;
    const int j = blockIdx.y * kTY + threadIdx.y;
    double acc[kNV] = {0.0};
    if (i < g.nx && j < g.ny) {
        const int k0 = blockIdx.z * kTZ, k1 = min(k0 + kTZ, g.nz);
        for (int k = k0; k < k1; ++k) {
            double b = div_at(g, u, v, w, i, j, k) * inv_hdt;
            rhs[g.cidx(i, j, k)] = b;
            acc[0] += b;
        }
    }
    const int op[kNV] = {0};
    const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    paris::block_reduce_store<kNV>(acc, op, scratch, blk, threadIdx.y * kTX + threadIdx.x);
}

// One CTA folds the block sums in a fixed order; the mean goes to the slot
// after the partials (and to the caller's output when given).
__global__ void noalloc_mean_kernel(int nblocks, double ncells, double* scratch, double* mean_out) {
    __shared__ double sh[paris::kRedThreads / 32];
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += scratch[kNV * b];
    s = paris::warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < paris::kRedThreads / 32; ++q) t += sh[q];
        const double m = t / ncells;
        scratch[kNV * kMaxBlocks] = m;
        if (mean_out) *mean_out = m;
    }
}

__global__ void noalloc_sub_mean_kernel(int64_t n, double* __restrict__ rhs, const double* scratch) {
    const double m = scratch[kNV * kMaxBlocks];
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x)
        rhs[c] -= m;
}

}  // namespace

extern "C" paris_status paris_divergence_noalloc(const paris_grid* g, const double* u,
                                                 const double* v, const double* w, double dt,
                                                 double* rhs, double* mean_removed, void* stream) {
    if (!g || !u || !v || !w || !rhs) return PARIS_ERR_INVALID_ARG;
    if (g->nx < 2 || g->ny < 2 || g->nz < 2 || !(g->h > 0.0) || !(dt > 0.0)) return PARIS_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (g->bc[a] != PARIS_PERIODIC && g->bc[a] != PARIS_WALL) return PARIS_ERR_INVALID_ARG;
    const dim3 grid((g->nx + kTX - 1) / kTX, (g->ny + kTY - 1) / kTY, (g->nz + kTZ - 1) / kTZ);
    const int64_t nblocks = (int64_t)grid.x * grid.y * grid.z;
    if (nblocks > kMaxBlocks) return PARIS_ERR_INVALID_ARG;  // beyond the fixed scratch
    // an error left pending by an unrelated earlier call is not this call's:
    // consume it; one that persists (a sticky error) means the device context
    // is unusable, and nothing is enqueued
    cudaGetLastError();
    if (cudaPeekAtLastError() != cudaSuccess) return PARIS_ERR_CUDA;
    double* scratch = nullptr;
    int sms = 1;
    if (scratch_on_current_device(&scratch, &sms) != cudaSuccess) return PARIS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const Geo geo{g->nx, g->ny, g->nz, g->bc[0] == PARIS_WALL, g->bc[1] == PARIS_WALL,
                  g->bc[2] == PARIS_WALL};
    noalloc_div_kernel<<<grid, dim3(kTX, kTY), 0, st>>>(geo, u, v, w, 1.0 / (g->h * dt), rhs, scratch);
    noalloc_mean_kernel<<<1, paris::kRedThreads, 0, st>>>((int)nblocks, (double)geo.ncell(), scratch,
                                                          mean_removed);
    const int64_t n = geo.ncell();
    int64_t nb = (n + 255) / 256;
    if (nb > (int64_t)sms * 8) nb = (int64_t)sms * 8;  // 8 resident 256-thread blocks per SM
    noalloc_sub_mean_kernel<<<(int)nb, 256, 0, st>>>(n, rhs, scratch);
    return cudaGetLastError() == cudaSuccess ? PARIS_OK : PARIS_ERR_CUDA;
}
