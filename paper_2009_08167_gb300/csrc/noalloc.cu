// Allocation-free variant of the SpMV + inner-product kernel of the Lanczos
// step (y = A x and x^T y), for callers that cannot allocate device memory.
//
// The per-block partial sums that the regular path keeps in context-owned
// scratch live here in a file-scope __device__ array of fixed size.  Every GPU
// that loads this library holds the array until the process exits.  Host code
// never dereferences the array's name: the first call on each device looks up
// the array's device address with cudaGetSymbolAddress (with that device
// current) and caches it; every call passes that address to the kernels.
#include <mutex>

#include "ctx.h"

namespace riga {

constexpr int NOALLOC_ROWS_PER_BLOCK = 16;  // 256 threads, 16 lanes per row
constexpr int NOALLOC_MAX_BLOCKS = 65536;   // 512 KiB of partial sums
constexpr long long NOALLOC_MAX_ROWS = (long long)NOALLOC_MAX_BLOCKS * NOALLOC_ROWS_PER_BLOCK;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_partial[NOALLOC_MAX_BLOCKS];

__global__ void __launch_bounds__(256) noalloc_spmv_dot_kernel(long long N, const long long* __restrict__ rowptr,
                                                               const int* __restrict__ col,
                                                               const double* __restrict__ val,
                                                               const double* __restrict__ x, double* __restrict__ y,
                                                               double* __restrict__ partial) {
    __shared__ double red[NOALLOC_ROWS_PER_BLOCK];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long row = t / 16;
    const int lane = (int)(t % 16);
    double s = 0.0;
    if (row < N)
        for (long long e = rowptr[row] + lane; e < rowptr[row + 1]; e += 16) s += val[e] * x[col[e]];
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, 16);
    double d = 0.0;
    if (row < N && lane == 0) {
        y[row] = s;
        d = s * x[row];
    }
    if (lane == 0) red[threadIdx.x / 16] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < NOALLOC_ROWS_PER_BLOCK; ++i) tot += red[i];
        partial[blockIdx.x] = tot;
    }
}

// single block: out = sum of nb partials, in a fixed order
__global__ void noalloc_reduce_kernel(const double* __restrict__ partial, int nb, double* __restrict__ out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

namespace {
std::mutex g_noalloc_mutex;
double* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
int noalloc_scratch(double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        cudaGetLastError();
        return RIGA_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partial) != cudaSuccess || !p) {
            cudaGetLastError();
            return RIGA_ECUDA;
        }
        g_noalloc_addr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_addr[dev];
    return RIGA_OK;
}

// true when p is device (or managed) memory of the current device
bool on_current_device(const void* p) {
    int dev = -1;
    cudaPointerAttributes a;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}
}  // namespace

}  // namespace riga

extern "C" int riga_spmv_dot_noalloc(const long long* rowptr, const int* col, const double* val, long long N,
                                     const double* x, double* y, double* xy, void* cuda_stream) {
    using namespace riga;
    if (!rowptr || !col || !val || !x || !y || !xy || N < 1) return RIGA_EINVAL;
    if (N > NOALLOC_MAX_ROWS) return RIGA_EINVAL;
    // every array must be device memory of the current device: a host
    // pointer or another GPU's memory is refused before anything is launched
    const void* ptrs[6] = {rowptr, col, val, x, y, xy};
    for (const void* p : ptrs)
        if (!on_current_device(p)) return RIGA_EINVAL;
    double* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const unsigned nb = (unsigned)((N + NOALLOC_ROWS_PER_BLOCK - 1) / NOALLOC_ROWS_PER_BLOCK);
    noalloc_spmv_dot_kernel<<<nb, 256, 0, st>>>(N, rowptr, col, val, x, y, scratch);
    noalloc_reduce_kernel<<<1, 256, 0, st>>>(scratch, (int)nb, xy);
    if (cudaGetLastError() != cudaSuccess) return RIGA_ECUDA;
    return RIGA_OK;
}
