// lbpf_field_sums_static: the measurement sums of lbpf_measure over
// caller-provided phi and u arrays, with its scratch in a fixed file-scope
// device array instead of memory from cudaMalloc.
//
// Who needs it: callers that cannot allocate device memory at the point of
// the call — for example applications that hand all device memory to their
// own pool allocator (a cudaMalloc from this library would fail or fragment
// that pool), or latency-critical host loops where cudaMalloc/cudaFree would
// synchronise the device.  They pass their own inputs and a 3-double output
// buffer; everything else lives in the array below.
//
// The array is a property of the loaded library: every GPU that loads it
// holds kStaticPartials * 3 doubles (96 KiB) until the process exits.  All
// calls share it and it keeps the previous call's contents; every slot a call
// reads is written by that same call first, so nothing needs clearing.  Calls
// whose kernels overlap on the GPU (different streams, or different host
// threads on one device) race on the array and must be serialised by the
// caller.
//
// The device address of the array is looked up once per device (the first
// call on that device) and cached; a cudaDeviceReset destroys the context
// that address belongs to, so calls after a device reset are not supported.
#include <cmath>
#include <mutex>

#include "lbpf_internal.cuh"

namespace {

constexpr int kStaticBlockThreads = 256;
constexpr long long kStaticChunk = 65536;   // sites reduced by one block
constexpr int kStaticPartials = 4096;        // blocks (3 doubles each)
constexpr long long kStaticMaxSites = kStaticChunk * kStaticPartials;  // 268,435,456
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_static_partials[kStaticPartials * 3];

// Device addresses of g_static_partials, found once per device.
std::mutex g_setup_mutex;
double* g_partials_ptr[kMaxDevices] = {};

__device__ __forceinline__ double warp_sum_static(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block b reduces sites [b * kStaticChunk, (b + 1) * kStaticChunk) into
// partial[3 b .. 3 b + 2]: sum (1 + phi)/2, sum (u - phi/2), non-finite count.
template <class R>
__global__ void __launch_bounds__(kStaticBlockThreads)
    static_sums_kernel(const R* __restrict__ phi, const R* __restrict__ u, long long n, double* partial)
{
    const long long begin = (long long)blockIdx.x * kStaticChunk;
    long long end = begin + kStaticChunk;
    if (end > n) end = n;
    double sf = 0.0, cs = 0.0, bad = 0.0;
    for (long long s = begin + threadIdx.x; s < end; s += kStaticBlockThreads) {
        const double p = (double)phi[s], v = (double)u[s];
        if (!isfinite(p) || !isfinite(v)) {
            bad += 1.0;
            continue;
        }
        sf += 0.5 * (1.0 + p);
        cs += v - 0.5 * p;
    }
    __shared__ double red[3][kStaticBlockThreads / 32];
    sf = warp_sum_static(sf);
    cs = warp_sum_static(cs);
    bad = warp_sum_static(bad);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[0][w] = sf;
        red[1][w] = cs;
        red[2][w] = bad;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int k = 0; k < kStaticBlockThreads / 32; ++k) t += red[threadIdx.x][k];
        partial[3 * blockIdx.x + threadIdx.x] = t;
    }
}

// Sums the per-block partials in a fixed order (thread t takes blocks t,
// t + 256, ...; then a fixed tree over the threads), so results are
// deterministic run to run.
__global__ void __launch_bounds__(kStaticBlockThreads)
    static_sums_finish_kernel(const double* partial, int nblocks, double* out)
{
    double t[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += kStaticBlockThreads)
#pragma unroll
        for (int k = 0; k < 3; ++k) t[k] += partial[3 * b + k];
    __shared__ double red[3][kStaticBlockThreads / 32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double v = warp_sum_static(t[k]);
        if (l == 0) red[k][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = 0.0;
        for (int j = 0; j < kStaticBlockThreads / 32; ++j) v += red[threadIdx.x][j];
        out[threadIdx.x] = v;
    }
}

}  // namespace

extern "C" int lbpf_field_sums_static(const void* phi, const void* u, long long n, int precision, double* out,
                                      void* stream)
{
    if (!phi || !u || !out) return LBPF_EINVAL;
    if (precision < LBPF_FP64 || precision > LBPF_FP32_FP16DEV_SR) return LBPF_EINVAL;
    if (n < 1 || n > kStaticMaxSites) return LBPF_ERANGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return LBPF_ECUDA;
    }
    double* partials = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_partials_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_static_partials) != cudaSuccess || !p) {
                cudaGetLastError();
                return LBPF_ECUDA;
            }
            g_partials_ptr[dev] = static_cast<double*>(p);
        }
        partials = g_partials_ptr[dev];
    }
    const int blocks = (int)((n + kStaticChunk - 1) / kStaticChunk);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // An error pending before this call belongs to the caller: it is neither
    // reported as ours nor cleared.  A launch error of our own kernels is
    // cleared and reported as LBPF_ECUDA.
    const cudaError_t before = cudaPeekAtLastError();
    if (precision == LBPF_FP64)
        static_sums_kernel<double><<<blocks, kStaticBlockThreads, 0, s>>>(static_cast<const double*>(phi),
                                                                           static_cast<const double*>(u), n, partials);
    else
        static_sums_kernel<float><<<blocks, kStaticBlockThreads, 0, s>>>(static_cast<const float*>(phi),
                                                                          static_cast<const float*>(u), n, partials);
    cudaError_t e = cudaPeekAtLastError();
    if (e == cudaSuccess || e == before)
        static_sums_finish_kernel<<<1, kStaticBlockThreads, 0, s>>>(partials, blocks, out);
    e = cudaPeekAtLastError();
    if (e != cudaSuccess && e != before) {
        cudaGetLastError();
        return LBPF_ECUDA;
    }
    return LBPF_OK;
}
