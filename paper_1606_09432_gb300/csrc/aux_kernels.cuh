// Per-lattice kernels around the fused step: equilibrium initial
// populations, the heat update that brings a lagged state up to date, and
// decoding reads.  Each is one thread per site with periodic wrap; none of
// them is on the per-step path.
#pragma once

#include "staged_kernel.cuh"

namespace lbpf {

struct SiteNb {
    long long oxm, oxp, oym, oyp, ozm, ozp;
    __device__ __forceinline__ long long off(int ex, int ey, int ez) const
    {
        return (ex < 0 ? oxm : (ex > 0 ? oxp : 0)) + (ey < 0 ? oym : (ey > 0 ? oyp : 0)) +
               (ez < 0 ? ozm : (ez > 0 ? ozp : 0));
    }
};

__device__ __forceinline__ SiteNb site_nb(const DomainDev& d, long long s, int& x, int& y, int& z)
{
    const long long nxy = (long long)d.nx * d.ny;
    z = (int)(s / nxy);
    const long long r = s - (long long)z * nxy;
    y = (int)(r / d.nx);
    x = (int)(r - (long long)y * d.nx);
    // periodic wrap, or reflection at a wall (the image of the node beyond
    // a wall is the node on the other side of it)
    const bool wx = d.bc & LBPF_BC_WALL_X, wy = d.bc & LBPF_BC_WALL_Y, wz = d.bc & LBPF_BC_WALL_Z;
    SiteNb nb;
    nb.oxm = (x == 0) ? (wx ? 1 : d.nx - 1) : -1;
    nb.oxp = (x == d.nx - 1) ? (wx ? -1 : -(d.nx - 1)) : 1;
    nb.oym = (long long)((y == 0) ? (wy ? 1 : d.ny - 1) : -1) * d.nx;
    nb.oyp = (long long)((y == d.ny - 1) ? (wy ? -1 : -(d.ny - 1)) : 1) * d.nx;
    nb.ozm = (d.nz == 1) ? 0 : (long long)((z == 0) ? (wz ? 1 : d.nz - 1) : -1) * nxy;
    nb.ozp = (d.nz == 1) ? 0 : (long long)((z == d.nz - 1) ? (wz ? -1 : -(d.nz - 1)) : 1) * nxy;
    return nb;
}

// Gradient of phi at site s in lattice units (Sec. 4.2), global-memory stencil.
template <class PL, class R>
__device__ __forceinline__ void site_gradient(const R* phi, long long s, const SiteNb& nb, int grad, R& Gx, R& Gy,
                                              R& Gz)
{
    Gx = Gy = Gz = R(0);
    if (grad == LBPF_GRAD_DD) {
#pragma unroll
        for (int i = 1; i < PL::Q; ++i) {
            const int ex = PL::ex(i), ey = PL::ey(i), ez = PL::ez(i);
            const R wd = R(PL::w(i)) * (phi[s + nb.off(ex, ey, ez)] - phi[s + nb.off(-ex, -ey, -ez)]);
            if (ex) Gx += R(ex) * wd;
            if (ey) Gy += R(ey) * wd;
            if (ez) Gz += R(ez) * wd;
        }
        const R k = R(0.5 / PL::E2);
        Gx *= k;
        Gy *= k;
        Gz *= k;
    } else {
        Gx = R(0.5) * (phi[s + nb.oxp] - phi[s + nb.oxm]);
        Gy = R(0.5) * (phi[s + nb.oyp] - phi[s + nb.oym]);
        if (PL::D == 3) Gz = R(0.5) * (phi[s + nb.ozp] - phi[s + nb.ozm]);
    }
}

// e_j . a of heat direction j for a domain with an advective equilibrium
// (DomainDev::adv), zero otherwise.
template <class UL>
__device__ __forceinline__ double adv_dot(const DomainDev& d, int j)
{
    return d.advect ? UL::ex(j) * d.adv[0] + UL::ey(j) * d.adv[1] + UL::ez(j) * d.adv[2] : 0.0;
}

// Equilibrium populations from phi (phi[cur]) and u (held in aux[acur]):
// g_i = g_i^(0)(phi, N), Eq. (Feq_Phase); f_i = w_i u, Eq. (EqFunction_Tempr),
// or w_i u (1 + e_i . a) with an advective equilibrium.
// finalize_index: the seeded index keeps its value only where phi > 0 or
// |grad phi| > xi.  Leaves a synchronised state; aux becomes C = u - phi/2 in
// deviation storage (full storage does not use aux in that state).
template <class PL, class UL, class S>
__global__ void equilibrate_kernel(const DomainDev* dp, int cur, int fcur, int acur, int grad, int finalize_index)
{
    using R = typename S::Real;
    using T = typename S::T;
    const DomainDev& d = *dp;
    const long long n = d.n;
    const R* phi = static_cast<const R*>(d.phi[cur]);
    R* aux = static_cast<R*>(d.aux[acur]);
    T* g = static_cast<T*>(d.g[cur]);
    T* f = static_cast<T*>(d.f[fcur]);
    int8_t* I = d.I[cur];
    const R De2 = R(d.Dphi / PL::E2);
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        const SiteNb nb = site_nb(d, s, x, y, z);
        R Gx, Gy, Gz;
        site_gradient<PL, R>(phi, s, nb, grad, Gx, Gy, Gz);
        const R ph = phi[s];
        int cryst = 1;
        if (d.use_index) {
            int Iv = I[s];
            const double xi = sizeof(R) == 4 ? fmax(d.xi_lu, 1e-6) : d.xi_lu;
            if (finalize_index && !(ph > R(0) || Gx * Gx + Gy * Gy + Gz * Gz > R(xi * xi))) Iv = 0;
            I[s] = (int8_t)Iv;
            cryst = Iv;
        }
        R a = 1, Nx = 0, Ny = 0, Nz = 0;
        if (cryst > 0 && cryst <= d.n_crystals) anisotropy<R, PL::D>(d.cr[cryst - 1], Gx, Gy, Gz, a, Nx, Ny, Nz);
#pragma unroll
        for (int i = 0; i < PL::Q; ++i) {
            const R eN = R(PL::ex(i)) * Nx + R(PL::ey(i)) * Ny + R(PL::ez(i)) * Nz;
            const R dev = -R(PL::w(i)) * De2 * eN;  // g_i^(0) - w_i phi
            if (!S::dev)
                g[(long long)i * n + s] = from_real<T, R>(R(PL::w(i)) * ph + dev);
            else if (i > 0)
                g[(long long)(i - 1) * n + s] = from_real<T, R>(dev);
        }
        const R u = aux[s];
#pragma unroll
        for (int j = 0; j < UL::Q; ++j) {
            if (!S::dev)
                f[(long long)j * n + s] = from_real<T, R>(R(UL::w(j)) * u * (R(1) + R(adv_dot<UL>(d, j))));
            else if (j > 0)  // deviation from w_j u: w_j u (e_j . a)
                f[(long long)(j - 1) * n + s] = from_real<T, R>(R(UL::w(j)) * u * R(adv_dot<UL>(d, j)));
        }
        if (S::dev) aux[s] = u - R(0.5) * ph;
    }
}

// Heat update of step n-1 alone (Eq. LBE_Eq_Temp), lagged -> synchronised:
// reads f[fcur] (f^{n-1}), aux[acur], phi[cur] (phi^n) and, with an
// advective equilibrium, U[acur]; writes f[fcur^1] (f^n) and, in deviation
// storage, aux[acur^1] = C^n.
template <class PL, class UL, class S>
__global__ void heat_sync_kernel(const DomainDev* dp, int cur, int fcur, int acur)
{
    using R = typename S::Real;
    using T = typename S::T;
    const DomainDev& d = *dp;
    const long long n = d.n;
    const R* phi = static_cast<const R*>(d.phi[cur]);
    const R* auxc = static_cast<const R*>(d.aux[acur]);
    R* auxn = static_cast<R*>(d.aux[acur ^ 1]);
    const T* fc = static_cast<const T*>(d.f[fcur]);
    T* fn = static_cast<T*>(d.f[fcur ^ 1]);
    const R* Uc = static_cast<const R*>(d.U[acur]);
    const R om = R(1) - R(d.inv_eta_u);
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        const SiteNb nb = site_nb(d, s, x, y, z);
        R fv[UL::Q];
        R u = 0;
        R d0 = 0;
        if (S::dev) {
#pragma unroll
            for (int j = 1; j < UL::Q; ++j) d0 -= to_real(fc[(long long)(j - 1) * n + s]);
        }
#pragma unroll
        for (int j = 0; j < UL::Q; ++j) {
            const long long src = s + nb.off(-UL::ex(j), -UL::ey(j), -UL::ez(j));
            const R h = auxc[src] + R(0.5) * phi[src];
            R fj;
            if (!S::dev)
                fj = om * to_real(fc[(long long)j * n + src]) + R(UL::w(j)) * h;
            else
                fj = R(UL::w(j)) * h + om * ((j == 0) ? d0 : to_real(fc[(long long)(j - 1) * n + src]));
            if (d.advect && (UL::ex(j) | UL::ey(j) | UL::ez(j))) fj += R(UL::w(j)) * R(adv_dot<UL>(d, j)) * Uc[src];
            fv[j] = fj;
            u += fj;
        }
        if (d.bc) {  // heat populations from beyond a wall: mirrored partners
            const int lo = ((d.bc & LBPF_BC_WALL_X) && x == 0 ? 1 : 0) | ((d.bc & LBPF_BC_WALL_Y) && y == 0 ? 2 : 0) |
                           ((d.bc & LBPF_BC_WALL_Z) && d.nz > 1 && z == 0 ? 4 : 0);
            const int hi = ((d.bc & LBPF_BC_WALL_X) && x == d.nx - 1 ? 1 : 0) |
                           ((d.bc & LBPF_BC_WALL_Y) && y == d.ny - 1 ? 2 : 0) |
                           ((d.bc & LBPF_BC_WALL_Z) && d.nz > 1 && z == d.nz - 1 ? 4 : 0);
            if (lo | hi) {
                mirror_refill<UL, R>(fv, lo, hi);
                u = 0;
#pragma unroll
                for (int j = 0; j < UL::Q; ++j) u += fv[j];
            }
        }
        if (!S::dev) {
#pragma unroll
            for (int j = 0; j < UL::Q; ++j) fn[(long long)j * n + s] = from_real<T, R>(fv[j]);
        } else {
#pragma unroll
            for (int j = 1; j < UL::Q; ++j) fn[(long long)(j - 1) * n + s] = from_real<T, R>(fv[j] - R(UL::w(j)) * u);
            auxn[s] = u - R(0.5) * phi[s];
        }
    }
}

// u of a synchronised state: Eq. (Temperature_LB).
template <class PL, class UL, class S>
__global__ void read_u_kernel(const DomainDev* dp, int cur, int fcur, int acur, typename S::Real* out)
{
    using R = typename S::Real;
    using T = typename S::T;
    const DomainDev& d = *dp;
    const long long n = d.n;
    const T* f = static_cast<const T*>(d.f[fcur]);
    const R* aux = static_cast<const R*>(d.aux[acur]);
    const R* phi = static_cast<const R*>(d.phi[cur]);
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        if (!S::dev) {
            R u = 0;
#pragma unroll
            for (int j = 0; j < UL::Q; ++j) u += to_real(f[(long long)j * n + s]);
            out[s] = u;
        } else {
            out[s] = aux[s] + R(0.5) * phi[s];
        }
    }
}

// Decoded population i of a synchronised state (which = 0: g_i, 1: f_i).
template <class PL, class UL, class S>
__global__ void read_pop_kernel(const DomainDev* dp, int which, int i, int cur, int fcur, int acur,
                                typename S::Real* out)
{
    using R = typename S::Real;
    using T = typename S::T;
    const DomainDev& d = *dp;
    const long long n = d.n;
    const int Q = which == 0 ? PL::Q : UL::Q;
    const T* p = static_cast<const T*>(which == 0 ? d.g[cur] : d.f[fcur]);
    const R* phi = static_cast<const R*>(d.phi[cur]);
    const R* aux = static_cast<const R*>(d.aux[acur]);
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        if (!S::dev) {
            out[s] = to_real(p[(long long)i * n + s]);
        } else {
            const R m = which == 0 ? phi[s] : aux[s] + R(0.5) * phi[s];
            if (i > 0) {
                const R wi = which == 0 ? R(PL::w(i)) : R(UL::w(i));
                out[s] = wi * m + to_real(p[(long long)(i - 1) * n + s]);
            } else {
                R d0 = 0;
                for (int j = 1; j < Q; ++j) d0 -= to_real(p[(long long)(j - 1) * n + s]);
                out[s] = (which == 0 ? R(PL::w(0)) : R(UL::w(0))) * m + d0;
            }
        }
    }
}

// a_s(n) of the current phase field, n = -grad(phi)/|grad(phi)| (Eq.
// Def_Normal_Vector) with the gradient operator of the context, evaluated by
// the step kernel's anisotropy(); the crystal is the current index (one
// crystal: everywhere), a_s = 1 where the index is 0.
template <class PL, class S>
__global__ void read_as_kernel(const DomainDev* dp, int cur, int grad, typename S::Real* out)
{
    using R = typename S::Real;
    const DomainDev& d = *dp;
    const R* phi = static_cast<const R*>(d.phi[cur]);
    const int8_t* I = d.I[cur];
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < d.n; s += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        const SiteNb nb = site_nb(d, s, x, y, z);
        const int cryst = d.use_index ? (int)I[s] : 1;
        R a = 1, Nx, Ny, Nz;
        if (cryst > 0 && cryst <= d.n_crystals) {
            R Gx, Gy, Gz;
            site_gradient<PL, R>(phi, s, nb, grad, Gx, Gy, Gz);
            anisotropy<R, PL::D>(d.cr[cryst - 1], Gx, Gy, Gz, a, Nx, Ny, Nz);
        }
        out[s] = a;
    }
}

inline int grid_for(long long n)
{
    long long b = (n + 255) / 256;
    if (b > 152 * 64) b = 152 * 64;
    if (b < 1) b = 1;
    return (int)b;
}

template <class PL, class UL, class S>
struct LauncherImpl {
    // the step kernel of tile variant V (2D lattices through their XZ view)
    using KP = KernelLattice<PL>;
    using KU = KernelLattice<UL>;
    template <int V> static constexpr int TXV = tile_x(PL::D, V);
    template <int V> static constexpr int TYV = tile_y(PL::D, V);
    // the advective kernel (tile variant 0, with walls)
    static constexpr bool kAdv = true;
    template <int V, bool W = false, bool A = false>
    static constexpr auto kernel()
    {
        return step_kernel<KP, KU, S, TXV<V>, TYV<V>, W, A>;
    }
    template <int V, bool A = false>
    static constexpr size_t smem_v()
    {
        return step_smem_bytes<KP, KU, S, TXV<V>, TYV<V>, A>();
    }

    template <int V, bool W, bool A = false>
    static cudaError_t step_v(const StepArgs& a, int n_blocks, cudaStream_t s)
    {
        kernel<V, W, A>()<<<n_blocks, TXV<V> * TYV<V>, smem_v<V, A>(), s>>>(a);
        return cudaGetLastError();
    }
    // Tile variant 0 is built periodic, with walls and with an advective
    // equilibrium; the 16-row variant 1 only for periodic domains
    // (the context selects it for nothing else).
    static cudaError_t step(int v, int kind, const StepArgs& a, int n_blocks, cudaStream_t s)
    {
        if (v == 1) return kind ? cudaErrorInvalidValue : step_v<1, false>(a, n_blocks, s);
        if (kind & kStepAdvect) {
            if constexpr (kAdv)
                return step_v<0, true, true>(a, n_blocks, s);
            else
                return cudaErrorNotSupported;
        }
        return kind ? step_v<0, true>(a, n_blocks, s) : step_v<0, false>(a, n_blocks, s);
    }
    static size_t smem(int v) { return v == 0 ? smem_v<0>() : smem_v<1>(); }
    static cudaError_t prepare(int v)
    {
        if constexpr (kStaged) {
            if (v == 0) {
                cudaError_t e = cudaFuncSetAttribute(step_kernel_staged<PL, UL, S>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)staged_smem_bytes<PL, UL, S>());
                if (e != cudaSuccess) return e;
            }
        }
        const int b0 = (int)smem_v<0>();
        if (v == 1) return cudaFuncSetAttribute(kernel<1>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_v<1>());
        cudaError_t e = cudaFuncSetAttribute(kernel<0, false>(), cudaFuncAttributeMaxDynamicSharedMemorySize, b0);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel<0, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize, b0);
        if constexpr (kAdv) {
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(kernel<0, true, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_v<0, true>());
        }
        return e;
    }
    // the staged kernel: 3D, 16-bit deviation storage, lattices whose staging
    // fits two blocks per SM (D3Q15, D3Q19)
    static constexpr bool kStaged = PL::D == 3 && S::dev && (PL::Q == 15 || PL::Q == 19);
    static cudaError_t step_staged(const StepArgs& a, int n_blocks, cudaStream_t s)
    {
        if constexpr (kStaged) {
            step_kernel_staged<PL, UL, S><<<n_blocks, 256, staged_smem_bytes<PL, UL, S>(), s>>>(a);
            return cudaGetLastError();
        } else {
            return cudaErrorNotSupported;
        }
    }
    static int staged_blocks_per_sm()
    {
        int nb = 0;
        if constexpr (kStaged) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, step_kernel_staged<PL, UL, S>, 256,
                                                              staged_smem_bytes<PL, UL, S>()) != cudaSuccess) {
                cudaGetLastError();
                return 1;
            }
        }
        return nb > 0 ? nb : 1;
    }
    static int blocks_per_sm(int v, int kind)
    {
        int nb = 0;
        cudaError_t e = cudaErrorInvalidValue;
        if (v == 1)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel<1>(), TXV<1> * TYV<1>, smem_v<1>());
        else if (kind & kStepAdvect) {
            if constexpr (kAdv)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel<0, true, true>(), TXV<0> * TYV<0>,
                                                                  smem_v<0, true>());
        } else if (kind)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel<0, true>(), TXV<0> * TYV<0>, smem_v<0>());
        else
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel<0>(), TXV<0> * TYV<0>, smem_v<0>());
        if (e != cudaSuccess) {
            cudaGetLastError();
            return 1;
        }
        return nb > 0 ? nb : 1;
    }
    static cudaError_t heat_sync(const DomainDev* d, int cur, int fcur, int acur, cudaStream_t s)
    {
        heat_sync_kernel<PL, UL, S><<<152 * 8, 256, 0, s>>>(d, cur, fcur, acur);
        return cudaGetLastError();
    }
    static cudaError_t equilibrate(const DomainDev* d, int cur, int fcur, int acur, int grad, int finalize,
                                   cudaStream_t s)
    {
        equilibrate_kernel<PL, UL, S><<<152 * 8, 256, 0, s>>>(d, cur, fcur, acur, grad, finalize);
        return cudaGetLastError();
    }
    static cudaError_t read_u(const DomainDev* d, int cur, int fcur, int acur, void* out, cudaStream_t s)
    {
        read_u_kernel<PL, UL, S><<<152 * 8, 256, 0, s>>>(d, cur, fcur, acur, static_cast<typename S::Real*>(out));
        return cudaGetLastError();
    }
    static cudaError_t read_pop(const DomainDev* d, int which, int i, int cur, int fcur, int acur, void* out,
                                cudaStream_t s)
    {
        read_pop_kernel<PL, UL, S><<<152 * 8, 256, 0, s>>>(d, which, i, cur, fcur, acur,
                                                           static_cast<typename S::Real*>(out));
        return cudaGetLastError();
    }
    static cudaError_t read_as(const DomainDev* d, int cur, int grad, void* out, cudaStream_t s)
    {
        read_as_kernel<PL, S><<<152 * 8, 256, 0, s>>>(d, cur, grad, static_cast<typename S::Real*>(out));
        return cudaGetLastError();
    }
    static const Launchers* get()
    {
        static const Launchers L = {&step,     &smem,           &prepare,  &blocks_per_sm,
                                    kStaged ? &step_staged : nullptr,      &staged_blocks_per_sm,
                                    &heat_sync, &equilibrate,   &read_u,   &read_pop,
                                    &read_as,  PL::Q,          UL::Q,     PL::D};
        return &L;
    }
};

}  // namespace lbpf
