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
            // minimum image along periodic axes, plain distance along walled ones
            const double ddx = (d.bc & LBPF_BC_WALL_X) ? x - sd[0] : periodic_delta(x - sd[0], d.nx);
            const double ddy = (d.bc & LBPF_BC_WALL_Y) ? y - sd[1] : periodic_delta(y - sd[1], d.ny);
            const double ddz = dim == 3 ? ((d.bc & LBPF_BC_WALL_Z) ? z - sd[2] : periodic_delta(z - sd[2], d.nz)) : 0.0;
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
// With walls (bc != 0), (u - phi/2) of a site on a wall counts 1/2 per walled
// coordinate at a wall: the site lies on a mirror plane (trapezoid rule).
template <class R>
__global__ void __launch_bounds__(256) reduce_kernel(const R* __restrict__ phi, const R* __restrict__ u, long long n,
                                                     double* partial, int nx, int ny, int nz, int bc, int dim)
{
    double sf = 0.0, cs = 0.0, bad = 0.0;
    const long long nxy = (long long)nx * ny;
    for (long long s = blockIdx.x * 256LL + threadIdx.x; s < n; s += (long long)gridDim.x * 256) {
        const double p = (double)phi[s], v = (double)u[s];
        if (!isfinite(p) || !isfinite(v)) {
            bad += 1.0;
            continue;
        }
        double wgt = 1.0;
        if (bc) {
            const int z = (int)(s / nxy);
            const long long r = s - (long long)z * nxy;
            const int y = (int)(r / nx), x = (int)(r - (long long)y * nx);
            if ((bc & LBPF_BC_WALL_X) && (x == 0 || x == nx - 1)) wgt *= 0.5;
            if ((bc & LBPF_BC_WALL_Y) && (y == 0 || y == ny - 1)) wgt *= 0.5;
            if ((bc & LBPF_BC_WALL_Z) && dim == 3 && (z == 0 || z == nz - 1)) wgt *= 0.5;
        }
        sf += 0.5 * (1.0 + p);
        cs += wgt * (v - 0.5 * p);
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
                          cudaStream_t s, int nx, int ny, int nz, int bc, int dim)
{
    if (bc && (long long)nx * ny * nz != n) return cudaErrorInvalidValue;
    if (precision == LBPF_FP64)
        reduce_kernel<double><<<kReduceBlocks, 256, 0, s>>>(static_cast<const double*>(phi),
                                                           static_cast<const double*>(u), n, partial, nx, ny, nz, bc,
                                                           dim);
    else
        reduce_kernel<float><<<kReduceBlocks, 256, 0, s>>>(static_cast<const float*>(phi),
                                                          static_cast<const float*>(u), n, partial, nx, ny, nz, bc,
                                                          dim);
    reduce_finish_kernel<<<1, 32, 0, s>>>(partial, kReduceBlocks, out);
    return cudaGetLastError();
}

// Tip crossings: warp w scans the ray of axis w/2, sign +1 (even w) or -1,
// k = 0 .. len-1 with len = half the domain length along the axis; the
// outermost k with phi_k >= 0 > phi_{k+1} gives k + phi_k / (phi_k - phi_{k+1}).
// A walled axis: the ray runs from the centre to the wall, without wrap.
template <class R>
__global__ void tips_kernel(const R* __restrict__ phi, int nx, int ny, int nz, int cx, int cy, int cz, int dim,
                            double* out, int bc)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int axis = w >> 1, sign = (w & 1) ? -1 : 1;
    if (w >= 6) return;
    if (axis == 2 && dim == 2) {
        if (l == 0) out[w] = -1.0;
        return;
    }
    const int nax = axis == 0 ? nx : (axis == 1 ? ny : nz);
    const int cax = axis == 0 ? cx : (axis == 1 ? cy : cz);
    const int len = (bc >> axis) & 1 ? (sign > 0 ? nax - 1 - cax : cax) : nax / 2;
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
                        double* out, cudaStream_t s, int bc)
{
    if (precision == LBPF_FP64)
        tips_kernel<double><<<1, 192, 0, s>>>(static_cast<const double*>(phi), nx, ny, nz, cx, cy, cz, dim, out, bc);
    else
        tips_kernel<float><<<1, 192, 0, s>>>(static_cast<const float*>(phi), nx, ny, nz, cx, cy, cz, dim, out, bc);
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
__global__ void fill_i32_kernel(int* out, int v, long long n)
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
cudaError_t launch_fill_i32(int* out, int v, long long n, cudaStream_t s)
{
    fill_i32_kernel<<<blocks_for(n), 256, 0, s>>>(out, v, n);
    return cudaGetLastError();
}

}  // namespace lbpf

namespace lbpf {

// Append (time, tip6) to a domain's measurement history slot.
__global__ void hist_append_kernel(const double* tips6, double t, double* slot)
{
    if (threadIdx.x == 0) slot[0] = t;
    if (threadIdx.x < 6) slot[1 + threadIdx.x] = tips6[threadIdx.x];
}

cudaError_t launch_hist_append(const double* tips6, double t, double* slot, cudaStream_t s)
{
    hist_append_kernel<<<1, 32, 0, s>>>(tips6, t, slot);
    return cudaGetLastError();
}

// Least-squares slope (FP64) of each tip distance over time, over the last
// `window` entries of a ring of `cap` entries ending at `last`; entries with
// no crossing (negative) are skipped.  out[d] = slope * dx (physical speed), or
// NaN when fewer than two valid entries remain.
__global__ void tip_velocity_kernel(const double* hist, int cap, int last, int count, int window, double dx,
                                    double* out)
{
    const int d = threadIdx.x;
    if (d >= 6) return;
    const int m = window < count ? window : count;
    double st = 0, sx = 0;
    int k = 0;
    for (int i = 0; i < m; ++i) {
        const double* e = hist + 7 * (size_t)((last - i + cap) % cap);
        if (e[1 + d] < 0) continue;
        st += e[0];
        sx += e[1 + d];
        ++k;
    }
    if (k < 2) {
        out[d] = nan("");
        return;
    }
    const double tm = st / k, xm = sx / k;
    double num = 0, den = 0;
    for (int i = 0; i < m; ++i) {
        const double* e = hist + 7 * (size_t)((last - i + cap) % cap);
        if (e[1 + d] < 0) continue;
        num += (e[0] - tm) * (e[1 + d] - xm);
        den += (e[0] - tm) * (e[0] - tm);
    }
    out[d] = den > 0 ? num / den * dx : nan("");
}

cudaError_t launch_tip_velocity(const double* hist, int cap, int last, int count, int window, double dx, double* out,
                                cudaStream_t s)
{
    tip_velocity_kernel<<<1, 32, 0, s>>>(hist, cap, last, count, window, dx, out);
    return cudaGetLastError();
}

// Tip radius: warp r scans the ray parallel to the tip axis at transverse
// offset j (ray r = plane * (2J+1) + j + J) for its outermost phi = 0
// crossing; thread 0 then fits x_c(j) = a + b j^2 per transverse plane in FP64
// and returns the mean of -1/(2b) over the planes (-1 when no fit).
template <class R>
// Walled axes: transverse offsets beyond a wall are reflected (the mirror
// image of the crystal) and the ray runs to the wall.
__global__ void tip_radius_kernel(const R* __restrict__ phi, int nx, int ny, int nz, int cx, int cy, int cz, int dir,
                                  int J, int dim, double* out, int bc)
{
    __shared__ double xc[32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int axis = dir >> 1, sign = (dir & 1) ? -1 : 1;
    const int nrow = 2 * J + 1;
    const int nplanes = dim - 1;
    const int nn[3] = {nx, ny, nz};
    if (w < nrow * nplanes) {
        const int plane = w / nrow, j = w % nrow - J;
        int tr = -1, cnt = 0;
        for (int a = 0; a < dim; ++a)
            if (a != axis) {
                if (cnt == plane) tr = a;
                ++cnt;
            }
        int c[3] = {cx, cy, cz};
        if ((bc >> tr) & 1) {  // repeated reflection: |j| may exceed the domain
            int v = c[tr] + j;
            while (v < 0 || v > nn[tr] - 1) v = v < 0 ? -v : 2 * (nn[tr] - 1) - v;
            c[tr] = v;
        } else {
            c[tr] = ((c[tr] + j) % nn[tr] + nn[tr]) % nn[tr];
        }
        const int len = (bc >> axis) & 1 ? (sign > 0 ? nn[axis] - 1 - c[axis] : c[axis]) : nn[axis] / 2;
        auto at = [&](int k) -> double {
            int p[3] = {c[0], c[1], c[2]};
            p[axis] = ((c[axis] + sign * k) % nn[axis] + nn[axis]) % nn[axis];
            return (double)phi[((long long)p[2] * ny + p[1]) * nx + p[0]];
        };
        int best = -1;
        for (int k = l; k < len; k += 32)
            if (at(k) >= 0.0 && at(k + 1) < 0.0) best = k;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_down_sync(0xffffffffu, best, o));
        if (l == 0) {
            if (best < 0) {
                xc[w] = -1.0;
            } else {
                const double p0 = at(best), p1 = at(best + 1);
                xc[w] = best + p0 / (p0 - p1);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0;
        int nfit = 0;
        for (int plane = 0; plane < nplanes; ++plane) {
            double s1 = 0, sj = 0, sx = 0, sjj = 0, sjx = 0;
            for (int j = -J; j <= J; ++j) {
                const double x = xc[plane * nrow + j + J];
                if (x < 0) continue;
                const double q = (double)j * j;
                s1 += 1;
                sj += q;
                sx += x;
                sjj += q * q;
                sjx += q * x;
            }
            const double den = s1 * sjj - sj * sj;
            if (s1 >= 3 && den > 0) {
                const double b = (s1 * sjx - sj * sx) / den;
                sum += -1.0 / (2.0 * b);
                ++nfit;
            }
        }
        out[0] = nfit ? sum / nfit : -1.0;
    }
}

cudaError_t launch_tip_radius(const void* phi, int nx, int ny, int nz, int cx, int cy, int cz, int dir, int J, int dim,
                              int precision, double* out, cudaStream_t s, int bc)
{
    const int threads = 32 * (2 * J + 1) * (dim - 1);
    if (precision == LBPF_FP64)
        tip_radius_kernel<double><<<1, threads, 0, s>>>(static_cast<const double*>(phi), nx, ny, nz, cx, cy, cz, dir,
                                                         J, dim, out, bc);
    else
        tip_radius_kernel<float><<<1, threads, 0, s>>>(static_cast<const float*>(phi), nx, ny, nz, cx, cy, cz, dir, J,
                                                        dim, out, bc);
    return cudaGetLastError();
}

}  // namespace lbpf
