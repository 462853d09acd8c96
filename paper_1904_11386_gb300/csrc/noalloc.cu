// scbb_population_moments_noalloc: FP64 mass and momentum of a device population array with no device
// allocation at all.  Its block partial sums live in a file-scope __device__ array instead of a workspace,
// for callers that cannot allocate device memory themselves: a host framework that owns the device
// allocator and forbids side allocations, or a loop that must not take cudaMalloc's implicit
// synchronisation and the risk of an out-of-memory failure in the middle of a run.
#include <stdio.h>

#include "scbb_internal.cuh"

namespace scbb {

// Fixed scratch: NOALLOC_BLOCKS partial sums of 5 doubles, plus the 5 final sums.  About 20 KB; every GPU
// that loads the library keeps it until the process exits.
constexpr int NOALLOC_BLOCKS = 512;
constexpr int NOALLOC_THREADS = 256;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_BLOCKS * 5 + 8];

// Same sums as the workspace-based moments reduction, but over populations already streamed, stored as
// f[c][i][N] (no pull), partials written to the static scratch.
__global__ void __launch_bounds__(NOALLOC_THREADS)
k_noalloc_moments(const float* __restrict__ f, unsigned int N, int nxy, int nz, int walls, double* scratch) {
    double acc[5] = {0, 0, 0, 0, 0};
    for (unsigned int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        const int z = (int)(n / (unsigned)nxy);
        if (walls && (z == 0 || z == nz - 1)) continue;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const double a = f[(size_t)i * N + n], b = f[(size_t)(Q + i) * N + n];
            acc[0] += a;
            acc[1] += b;
            acc[2] += dir_x(i) * (a + b);
            acc[3] += dir_y(i) * (a + b);
            acc[4] += dir_z(i) * (a + b);
        }
    }
    __shared__ double sh[5][NOALLOC_THREADS];
    for (int q = 0; q < 5; q++) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int s = NOALLOC_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int q = 0; q < 5; q++) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
        __syncthreads();
    }
    // every block writes its slot, so no slot keeps a previous call's value
    if (threadIdx.x == 0)
        for (int q = 0; q < 5; q++) scratch[8 + blockIdx.x * 5 + q] = sh[q][0];
}

__global__ void __launch_bounds__(NOALLOC_THREADS) k_noalloc_sum(double* scratch) {
    __shared__ double sh[NOALLOC_THREADS];
    for (int q = 0; q < 5; q++) {
        double a = 0;
        for (int b = threadIdx.x; b < NOALLOC_BLOCKS; b += blockDim.x) a += scratch[8 + b * 5 + q];
        sh[threadIdx.x] = a;
        __syncthreads();
        for (int s = NOALLOC_THREADS / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) scratch[q] = sh[0];
        __syncthreads();
    }
}

}  // namespace scbb

using namespace scbb;

extern "C" scbb_status scbb_population_moments_noalloc(const float* dev_f, int nx, int ny, int nz, int walls,
                                                      double* out5, void* cuda_stream) {
    if (!dev_f || !out5 || nx < 1 || ny < 1 || nz < 1 || (walls != 0 && walls != 1)) return SCBB_E_INVAL;
    const double nodes = (double)nx * ny * nz;
    if (nodes > (double)SCBB_NOALLOC_MAX_NODES) {
        fprintf(stderr, "scbb_population_moments_noalloc: %.0f nodes exceed the maximum of %d\n", nodes,
                SCBB_NOALLOC_MAX_NODES);
        return SCBB_E_INVAL;
    }
    // the array's address on the current device, looked up on every call (a cached address would outlive a
    // reset of the device's primary context)
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || !addr) return SCBB_E_CUDA;
    double* scratch = (double*)addr;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const unsigned int N = (unsigned int)nodes;
    k_noalloc_moments<<<NOALLOC_BLOCKS, NOALLOC_THREADS, 0, st>>>(dev_f, N, nx * ny, nz, walls, scratch);
    k_noalloc_sum<<<1, NOALLOC_THREADS, 0, st>>>(scratch);
    if (cudaGetLastError() != cudaSuccess) return SCBB_E_CUDA;
    if (cudaMemcpyAsync(out5, scratch, 5 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SCBB_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SCBB_E_CUDA;
    return SCBB_OK;
}
