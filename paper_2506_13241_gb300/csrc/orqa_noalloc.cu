// orqa_expect_noalloc: <0|O|0> of an operator held in caller-owned device
// arrays, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code embedded in a host framework
// whose allocator owns the device memory pool (a stray cudaMalloc there can
// fail or fragment the pool), and latency-critical paths that cannot accept
// the device-wide synchronisation cudaMalloc may imply.  This entry point
// needs no context and no workspace: its only scratch is a file-scope
// device array of fixed size, which every GPU that loads the library holds
// until the process exits.  The caller passes the inputs (device arrays)
// and the output (one host double).
//
// Every call shares that array and it keeps the last call's contents; each
// launch writes every partial it later reads, so nothing has to start at
// zero.  Calls whose kernels overlap on the GPU (for example on two
// streams) race on the shared array and must be serialised by the caller.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "orqa.h"

namespace {

constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_PER_THREAD = 8;
constexpr long long NOALLOC_TILE = (long long)NOALLOC_THREADS * NOALLOC_PER_THREAD;  // 2048 strings
constexpr int NOALLOC_MAX_TILES = (int)(ORQA_NOALLOC_MAX_STRINGS / NOALLOC_TILE);     // 65536
constexpr int NOALLOC_MAX_DEVICES = 64;

static_assert((long long)NOALLOC_MAX_TILES * NOALLOC_TILE == ORQA_NOALLOC_MAX_STRINGS,
              "the string limit is a whole number of tiles");

// One partial sum per 2048-string tile, then the total in the last slot
// (65537 doubles, 512 KiB + 8 bytes).
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_MAX_TILES + 1];

std::mutex g_setup_mutex;
double* g_scratch_ptr[NOALLOC_MAX_DEVICES] = {};

// Tile t sums c over its strings with an all-zero x plane (no sigma_x or
// sigma_y factor, Eq. magnetization) in a fixed order: each thread walks its
// 8 strings in sequence, then a fixed shuffle and shared-memory tree.
template <int W>
__global__ void __launch_bounds__(NOALLOC_THREADS) k_expect_tiles(const uint64_t* __restrict__ x,
                                                                  const double* __restrict__ c,
                                                                  long long n, double* partials) {
    __shared__ double red[NOALLOC_THREADS / 32];
    const long long base = (long long)blockIdx.x * NOALLOC_TILE;
    double acc = 0.0;
    for (int k = 0; k < NOALLOC_PER_THREAD; ++k) {
        const long long i = base + (long long)k * NOALLOC_THREADS + threadIdx.x;
        if (i < n) {
            uint64_t any = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) any |= x[i * W + w];
            if (any == 0) acc = __dadd_rn(acc, c[i]);
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc = __dadd_rn(acc, __shfl_down_sync(0xffffffffu, acc, d));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int k = 0; k < NOALLOC_THREADS / 32; ++k) b = __dadd_rn(b, red[k]);
        partials[blockIdx.x] = b;
    }
}

// Adds the tile partials in a fixed order into scratch[NOALLOC_MAX_TILES].
__global__ void __launch_bounds__(NOALLOC_THREADS) k_expect_tiles_total(double* scratch, int n_tiles) {
    __shared__ double red[NOALLOC_THREADS / 32];
    double acc = 0.0;
    for (int t = threadIdx.x; t < n_tiles; t += NOALLOC_THREADS) acc = __dadd_rn(acc, scratch[t]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc = __dadd_rn(acc, __shfl_down_sync(0xffffffffu, acc, d));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int k = 0; k < NOALLOC_THREADS / 32; ++k) b = __dadd_rn(b, red[k]);
        scratch[NOALLOC_MAX_TILES] = b;
    }
}

// Device address of the scratch array on the current device.  In host code
// the name g_noalloc_scratch is only a host-side stand-in, so the address is
// looked up once per device, with that device current, and cached.
cudaError_t scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// True iff p is device (or managed) memory that the current device can read
// and is 8-byte aligned: a host pointer or an odd address would otherwise
// reach the kernels and fault the GPU instead of returning ORQA_EINVAL.
bool device_readable(const void* p, int dev) {
    if (reinterpret_cast<uintptr_t>(p) % 8 != 0) return false;
    const cudaError_t prior = cudaPeekAtLastError();
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        if (prior == cudaSuccess) cudaGetLastError();  // clear only the failed query's own error
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" orqa_status orqa_expect_noalloc(int32_t n_qubits, int64_t n, const uint64_t* x, const double* c,
                                           double* out, void* stream) {
    if (n_qubits < 1 || n_qubits > 128 || n < 0 || !out) return ORQA_EINVAL;
    if (n > ORQA_NOALLOC_MAX_STRINGS) return ORQA_ECAPACITY;
    if (n > 0 && (!x || !c)) return ORQA_EINVAL;
    if (n == 0) {
        *out = 0.0;
        return ORQA_OK;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ORQA_ECUDA;
    if (!device_readable(x, dev) || !device_readable(c, dev)) return ORQA_EINVAL;
    double* scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return ORQA_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n_tiles = (int)((n + NOALLOC_TILE - 1) / NOALLOC_TILE);
    if (n_qubits <= 64)
        k_expect_tiles<1><<<n_tiles, NOALLOC_THREADS, 0, s>>>(x, c, n, scratch);
    else
        k_expect_tiles<2><<<n_tiles, NOALLOC_THREADS, 0, s>>>(x, c, n, scratch);
    k_expect_tiles_total<<<1, NOALLOC_THREADS, 0, s>>>(scratch, n_tiles);
    // peek, so that an error is left for its owner to see
    if (cudaPeekAtLastError() != cudaSuccess) return ORQA_ECUDA;
    if (cudaMemcpyAsync(out, scratch + NOALLOC_MAX_TILES, sizeof(double), cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
        return ORQA_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return ORQA_ECUDA;
    return ORQA_OK;
}
