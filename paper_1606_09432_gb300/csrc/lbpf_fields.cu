// Precision-generic kernels: seeding (Eq. Initial_Condition, Eq. Intial-Cond_u),
// the measurement reductions and tip rays, and index-field copies.
#include "lbpf_internal.cuh"

namespace lbpf {

__device__ __forceinline__ double periodic_delta(double d, int n)
{
    d = fmod(d, (double)n);
    if (d > 0.5 * n) d -= n;
    if (d < -0.5 * n) d += n;
    return d;
}

// phi(x, 0) = max_k tanh((R_k - d_k) dx / (sqrt(2) W0)); u(x, 0) = u0 (held in
// aux until the populations are built); preliminary index = dominant seed.
template <class R>
__global__ void seed_kernel(const DomainDev* dp, long long n, int cur, int acur, const double* seeds, int ns, int dim,
                            double k, double u0)
{
    const DomainDev& d = *dp;
    R* phi = static_cast<R*>(d.phi[cur]);
    R* aux = static_cast<R*>(d.aux[acur]);
    int8_t* I = d.I[cur];
    const long long nxy = (long long)d.nx * d.ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(s / nxy);
        const long long r = s - (long long)z * nxy;
        const int y = (int)(r / d.nx);
        const int x = (int)(r - (long long)y * d.nx);
        double best = -2.0;
        int bestc = 0;
        for (int j = 0; j < ns; ++j) {
            const double* sd = seeds + 5 * j;
            const double ddx = periodic_delta(x - sd[0], d.nx);
            const double ddy = periodic_delta(y - sd[1], d.ny);
            const double ddz = dim == 3 ? periodic_delta(z - sd[2], d.nz) : 0.0;
            const double v = tanh((sd[3] - sqrt(ddx * ddx + ddy * ddy + ddz * ddz)) * k);
            if (v > best) {
                best = v;
                bestc = (int)sd[4];
            }
        }
        phi[s] = R(best);
        aux[s] = R(u0);
        if (d.use_index) I[s] = (int8_t)(bestc + 1);
    }
}

cudaError_t launch_seed(const DomainDev* d, long long n, int cur, int acur, int precision, const double* seeds,
                        int n_seeds, int dim, double dx_over_sqrt2W0, double u0, cudaStream_t s)
{
    const int blocks = (int)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16);
    if (precision == LBPF_FP64)
        seed_kernel<double><<<blocks, 256, 0, s>>>(d, n, cur, acur, seeds, n_seeds, dim, dx_over_sqrt2W0, u0);
    else
        seed_kernel<float><<<blocks, 256, 0, s>>>(d, n, cur, acur, seeds, n_seeds, dim, dx_over_sqrt2W0, u0);
    return cudaGetLastError();
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Per-block FP64 partial sums of (1 + phi)/2 and (u - phi/2) and a count of
// non-finite values, in a fixed order per block (deterministic).
template <class R>
__global__ void __launch_bounds__(256) reduce_kernel(const R* __restrict__ phi, const R* __restrict__ u, long long n,
                                                     double* partial)
{
    double sf = 0.0, cs = 0.0, bad = 0.0;
    for (long long s = blockIdx.x * 256LL + threadIdx.x; s < n; s += (long long)gridDim.x * 256) {
        const double p = (double)phi[s], v = (double)u[s];
        if (!isfinite(p) || !isfinite(v)) {
            bad += 1.0;
            continue;
        }
        sf += 0.5 * (1.0 + p);
        cs += v - 0.5 * p;
    }
    __shared__ double red[3][8];
    sf = warp_sum(sf);
    cs = warp_sum(cs);
    bad = warp_sum(bad);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[0][w] = sf;
        red[1][w] = cs;
        red[2][w] = bad;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += red[threadIdx.x][k];
        partial[3 * blockIdx.x + threadIdx.x] = t;
    }
}

__global__ void reduce_finish_kernel(const double* partial, int nblocks, double* out)
{
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int b = 0; b < nblocks; ++b) t += partial[3 * b + threadIdx.x];
        out[threadIdx.x] = t;
    }
}

cudaError_t launch_reduce(const void* phi, const void* u, long long n, int precision, double* partial, double* out,
                          cudaStream_t s)
{
    if (precision == LBPF_FP64)
        reduce_kernel<double><<<kReduceBlocks, 256, 0, s>>>(static_cast<const double*>(phi),
                                                           static_cast<const double*>(u), n, partial);
    else
        reduce_kernel<float><<<kReduceBlocks, 256, 0, s>>>(static_cast<const float*>(phi),
                                                          static_cast<const float*>(u), n, partial);
    reduce_finish_kernel<<<1, 32, 0, s>>>(partial, kReduceBlocks, out);
    return cudaGetLastError();
}

// Tip crossings: warp w scans the ray of axis w/2, sign +1 (even w) or -1,
// k = 0 .. len-1 with len = half the domain length along the axis; the
// outermost k with phi_k >= 0 > phi_{k+1} gives k + phi_k / (phi_k - phi_{k+1}).
template <class R>
__global__ void tips_kernel(const R* __restrict__ phi, int nx, int ny, int nz, int cx, int cy, int cz, int dim,
                            double* out)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int axis = w >> 1, sign = (w & 1) ? -1 : 1;
    if (w >= 6) return;
    if (axis == 2 && dim == 2) {
        if (l == 0) out[w] = -1.0;
        return;
    }
    const int nax = axis == 0 ? nx : (axis == 1 ? ny : nz);
    const int len = nax / 2;
    auto at = [&](int k) -> double {
        int c[3] = {cx, cy, cz};
        c[axis] += sign * k;
        const int nn[3] = {nx, ny, nz};
        int v = c[axis] % nn[axis];
        if (v < 0) v += nn[axis];
        c[axis] = v;
        return (double)phi[((long long)c[2] * ny + c[1]) * nx + c[0]];
    };
    int best = -1;
    for (int k = l; k < len; k += 32) {
        if (at(k) >= 0.0 && at(k + 1) < 0.0) best = k;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_down_sync(0xffffffffu, best, o));
    if (l == 0) {
        if (best < 0) {
            out[w] = -1.0;
        } else {
            const double p0 = at(best), p1 = at(best + 1);
            out[w] = best + p0 / (p0 - p1);
        }
    }
}

cudaError_t launch_tips(const void* phi, int nx, int ny, int nz, int cx, int cy, int cz, int dim, int precision,
                        double* out, cudaStream_t s)
{
    if (precision == LBPF_FP64)
        tips_kernel<double><<<1, 192, 0, s>>>(static_cast<const double*>(phi), nx, ny, nz, cx, cy, cz, dim, out);
    else
        tips_kernel<float><<<1, 192, 0, s>>>(static_cast<const float*>(phi), nx, ny, nz, cx, cy, cz, dim, out);
    return cudaGetLastError();
}

__global__ void i8_to_i32_kernel(const int8_t* in, int* out, long long n)
{
    for (long long s = blockIdx.x * 256LL + threadIdx.x; s < n; s += (long long)gridDim.x * 256) out[s] = in[s];
}
// Index values outside 0..n_crystals become 0 (no crystal).
__global__ void i32_to_i8_kernel(const int* in, int8_t* out, long long n, int n_crystals)
{
    for (long long s = blockIdx.x * 256LL + threadIdx.x; s < n; s += (long long)gridDim.x * 256) {
        const int v = in[s];
        out[s] = (int8_t)((v < 0 || v > n_crystals) ? 0 : v);
    }
}
__global__ void fill_i8_kernel(int8_t* out, int8_t v, long long n)
{
    for (long long s = blockIdx.x * 256LL + threadIdx.x; s < n; s += (long long)gridDim.x * 256) out[s] = v;
}

static int blocks_for(long long n)
{
    long long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

cudaError_t launch_index_to_i32(const int8_t* in, int* out, long long n, cudaStream_t s)
{
    i8_to_i32_kernel<<<blocks_for(n), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}
cudaError_t launch_index_from_i32(const int* in, int8_t* out, long long n, int n_crystals, cudaStream_t s)
{
    i32_to_i8_kernel<<<blocks_for(n), 256, 0, s>>>(in, out, n, n_crystals);
    return cudaGetLastError();
}
cudaError_t launch_fill_i8(int8_t* out, int8_t v, long long n, cudaStream_t s)
{
    fill_i8_kernel<<<blocks_for(n), 256, 0, s>>>(out, v, n);
    return cudaGetLastError();
}

}  // namespace lbpf
