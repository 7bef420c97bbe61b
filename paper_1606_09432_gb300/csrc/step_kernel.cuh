// Fused time step of the phase-field and heat lattice Boltzmann schemes
// (Younsi & Cartalade, arXiv:1606.09432, Secs. 3.1-3.2), one launch per step.
//
// State at the start of step n (the "lagged" state):
//   g^n (phase-field populations), phi^n (its zeroth moment, Eq. Def_M0_Phi),
//   f^{n-1} (temperature populations one step behind) and the auxiliary field
//     full storage:      aux = psi^{n-1} = u^{n-1} / eta_u - phi^{n-1} / 2
//     deviation storage: aux = C^{n-1}   = u^{n-1} - phi^{n-1} / 2
// One launch produces g^{n+1}, phi^{n+1}, f^n and aux^n.  The heat update of
// step n-1 (Eq. LBE_Eq_Temp with Q_u = (phi^n - phi^{n-1}) / (2 dt), Sec. 3.1)
// is done inside the launch of step n, because the phase-field update of step
// n needs u^n on the neighbours of each site (Q_phi at x - e_i in pull form),
// and u^n in turn needs phi^n, which the previous launch produced.  The
// collision arithmetic is that of the paper; only the launch boundary moves.
// A "load" launch starts from a synchronised state (f^n, u^n known): it skips
// the heat collision and only reads u^n.
//
// Phase-field update in pull form (Eq. LBE_Eq_Phase), destination y,
// source x = y - e_i:
//   g_i^{n+1}(y) = c1(x) g_i^n(x) - c2(x) g_i^n(y) + w_i (s(x) + e_i . v(x))
//   c1 = (1 - 1/eta_phi) / a_s^2,  c2 = (1 - a_s^2) / a_s^2,
//   s  = (phi / eta_phi + (dt/tau0) Q_phi) / a_s^2,
//   v  = -D_phi N / (e^2 eta_phi a_s^2),   D_phi = (W0^2/tau0)(dt/dx^2),
// which is Eq. (LBE_Eq_Phase) divided by a_s^2(x) with g^(0) of Eq.
// (Feq_Phase), eta_phi of Eq. (LBE_RelaxationTime) and Q_phi of Eq.
// (LBE_SourceTerm), all evaluated at the collision node x.  With deviation
// storage (g_i = w_i phi + d_i) the pulled c1 w_i phi(x) is folded into the
// source coefficient, which is then stored as s + c1 phi = (phi + (dt/tau0)
// Q_phi) / a_s^2.
//
// Tiling: a block owns a TXT x TY column of sites and marches along z over
// [z0, z1), keeping rings of planes in shared memory: phi^n and
// h = aux + phi^n / 2 on the tile plus a 2-site halo, and the collision
// coefficients (c1, c2, s, v) on the tile plus a 1-site halo.  Every value
// is read from HBM once per launch except the halo rims, which neighbouring
// blocks share through L2.  Per plane z: wait for the copies of phi/aux
// plane z+2 and form h there, issue the cp.async copies of plane z+3 (in
// 3D interior rows in 16-byte chunks that bypass L1, halo columns by element),
// barrier, coefficients of plane z+1, barrier, output of plane z.  A 2D
// domain is run through the same march with its y axis as the kernel's z
// axis (lattice XZ<>): the tile is one row of TXT sites, without halo rows,
// and the heat pull sources of the next row are staged by cp.async too.
#pragma once

#include "lbpf_internal.cuh"

namespace lbpf {

// Explicitly rounded arithmetic (no contraction), so that the output phases of
// the step kernel and of the staged kernel round the same operations in the
// same order (their results are compared bit for bit).
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// New phase-field population of direction e = (ex, ey, ez) at y (Eq.
// LBE_Eq_Phase divided by a_s^2, pull form): c1 gp - c2 gl + w (s + e . v),
// rounded as a = ((s +- vx) +- vy) +- vz (zero components skipped), then
// fma(w, a, fma(c1, gp, -(c2 gl))).
template <class R>
__device__ __forceinline__ R pull_new(int ex, int ey, int ez, R w, R c1, R c2, R cs, R vx, R vy, R vz, R gp, R gl)
{
    R a = cs;
    if (ex) a = ex > 0 ? add_rn(a, vx) : sub_rn(a, vx);
    if (ey) a = ey > 0 ? add_rn(a, vy) : sub_rn(a, vy);
    if (ez) a = ez > 0 ? add_rn(a, vz) : sub_rn(a, vz);
    return fma_rn(w, a, fma_rn(c1, gp, -mul_rn(c2, gl)));
}

// Collision coefficients of one site, (c1, c2, s, vx, vy, vz), in one plane
// slot of 6 * CP values.  FP32: an array of float4 (c1, c2, s, vx) followed by
// an array of float2 (vy, vz), so that a direction reads one or two vectors;
// FP64: six scalar arrays.
template <class R> struct CoefIO;
template <> struct CoefIO<float> {
    __device__ static void store(float* pl, int CP, int ci, float c1, float c2, float s, float vx, float vy, float vz)
    {
        reinterpret_cast<float4*>(pl)[ci] = make_float4(c1, c2, s, vx);
        reinterpret_cast<float2*>(pl + 4 * CP)[ci] = make_float2(vy, vz);
    }
    __device__ static void load(const float* pl, int CP, int ci, bool need_yz, float& c1, float& c2, float& s,
                                float& vx, float& vy, float& vz)
    {
        const float4 a = reinterpret_cast<const float4*>(pl)[ci];
        c1 = a.x;
        c2 = a.y;
        s = a.z;
        vx = a.w;
        vy = vz = 0.f;
        if (need_yz) {
            const float2 b = reinterpret_cast<const float2*>(pl + 4 * CP)[ci];
            vy = b.x;
            vz = b.y;
        }
    }
};
template <> struct CoefIO<double> {
    __device__ static void store(double* pl, int CP, int ci, double c1, double c2, double s, double vx, double vy,
                                 double vz)
    {
        pl[ci] = c1;
        pl[CP + ci] = c2;
        pl[2 * CP + ci] = s;
        pl[3 * CP + ci] = vx;
        pl[4 * CP + ci] = vy;
        pl[5 * CP + ci] = vz;
    }
    __device__ static void load(const double* pl, int CP, int ci, bool need_yz, double& c1, double& c2, double& s,
                                double& vx, double& vy, double& vz)
    {
        c1 = pl[ci];
        c2 = pl[CP + ci];
        s = pl[2 * CP + ci];
        vx = pl[3 * CP + ci];
        vy = vz = 0.0;
        if (need_yz) {
            vy = pl[4 * CP + ci];
            vz = pl[5 * CP + ci];
        }
    }
};

// Shared memory of the staged heat populations (2D, FP32 full storage) and
// of the U ring (ADV), each rounded up to 16 bytes.
template <class UL, class S, bool XZV>
constexpr size_t stf_bytes(int RP)
{
    return (XZV && sizeof(typename S::T) == 4 && !S::dev) ? (((size_t)UL::Q * RP * sizeof(typename S::T) + 15) & ~size_t(15))
                                                         : 0;
}

// One work item: the column (x0, y0) of one domain over planes [z0, z1).
// WALLS: the domain may have zero-flux walls (mirror planes through the
// boundary nodes, lbpf.h LBPF_BC_WALL_X): stencil indices beyond a wall are
// reflected, and at a wall node every population whose source lies beyond
// the wall takes the value of its mirrored partner (the bounce-back of Sec.
// 3.3), for the phase-field and the heat populations alike.
// ADV: domains with a uniform velocity v use the advective heat equilibrium
// f_j^(0) = w_j u (1 + e_j . a), a = v dt / (dx e^2), so the heat pull gains
// w_j (e_j . a) U(x - e_j), U = u^{n-1} / eta_u, read from a ring of U planes
// staged like h; the launch stores U^n beside aux^n.  With deviation storage
// (f_j = w_j u + d_j) the same term appears: (1 - 1/eta_u) (w_j u + d_j) +
// w_j u (1 + e_j . a) / eta_u + w_j Q_u dt = w_j h + (1 - 1/eta_u) d_j +
// w_j (e_j . a) U.
template <class PL, class UL, class S, int TXT, int TY, bool WALLS, bool ADV>
__device__ __forceinline__ void step_item(const StepArgs& args, const WorkItem it, unsigned char* smem_raw)
{
    static_assert(PL::D == 3 && UL::D == 3, "the step kernel marches along z (2D lattices through XZ)");
    constexpr int NT = TXT * TY;
    using R = typename S::Real;
    using T = typename S::T;
    constexpr int D = PL::D;
    constexpr bool XZV = IsXZ<PL>::value;                   // 2D domain, y marched as z
    constexpr int HL = XZV ? 0 : 2, HC = XZV ? 0 : 1;       // halo rows (y) of the phi and coefficient planes
    // phi frame: tile + 2-site halo; in 3D the tile starts XO elements (16
    // bytes) into each row so that interior rows can be copied in 16-byte
    // chunks (in 2D the chunked copy measured slower and is not used)
    constexpr int XO = (XZV || sizeof(R) >= 8) ? 2 : 4;
    constexpr bool CHUNKED = !XZV;
    constexpr int RX = TXT + 2 * XO, RY = TY + 2 * HL, RP = RX * RY;
    constexpr int CX = TXT + 2, CY = TY + 2 * HC, CP = CX * CY;  // tile + 1-site halo
    // phi / index ring depth: planes z-1 .. z+3 in use while plane z is output
    // (the output phase reads phi^n only at its own plane)
    constexpr int NPH = 5;
    constexpr int NH = 4;                                   // h ring depth (z .. z+3)
    constexpr int NC = 3;                                   // coefficient ring depth
    constexpr int NCO = 6;                                  // c1, c2, s, vx, vy, vz
    constexpr int COP = NCO * CP;                           // reals of one coefficient plane
    constexpr int QG = PL::Q, QU = UL::Q;
    constexpr bool DEV = S::dev;
    (void)RY;
    (void)CY;

    R* s_phi = reinterpret_cast<R*>(smem_raw);
    R* s_h = s_phi + NPH * RP;
    R* s_co = s_h + NH * RP;
    int8_t* s_I = reinterpret_cast<int8_t*>(s_co + NC * COP);
    // 2D, FP32 full storage: the heat populations f^{n-1}_j(x - e_j) of the
    // next coefficient plane are staged too (copied during the output phase).
    // In 3D the extra shared memory costs more L1 than the copies save.
    constexpr bool STF = XZV && sizeof(T) == 4 && !DEV;
    T* s_f = reinterpret_cast<T*>(s_I + ((NPH * RP + 15) & ~15));
    R* s_U = reinterpret_cast<R*>(reinterpret_cast<unsigned char*>(s_f) + stf_bytes<UL, S, XZV>(RP));
    static_assert(!ADV || (sizeof(R) * (NPH * RP + NH * RP + NC * COP) + ((NPH * RP + 15) & ~15)) % 16 == 0,
                  "the U ring is a cp.async 16-byte destination");

    const DomainDev& dm = args.doms[it.dom];
    const int nx = dm.nx, ny = XZV ? 1 : dm.ny, nz = XZV ? dm.ny : dm.nz;
    const long long n = dm.n;
    const long long nxy = (long long)nx * ny;
    const int x0 = it.x0, y0 = it.y0;
    const int tw = min(TXT, nx - x0), th = min(TY, ny - y0);
    const int tid = threadIdx.x;
    const bool collide = args.collide != 0;
    const bool use_index = dm.use_index != 0;
    const bool need_h = collide || DEV;

    const T* __restrict__ gc = static_cast<const T*>(dm.g[args.cur]);
    T* __restrict__ gn = static_cast<T*>(dm.g[args.cur ^ 1]);
    const R* __restrict__ phic = static_cast<const R*>(dm.phi[args.cur]);
    R* __restrict__ phin = static_cast<R*>(dm.phi[args.cur ^ 1]);
    const T* __restrict__ fc = static_cast<const T*>(dm.f[args.fcur]);
    T* __restrict__ fn = static_cast<T*>(dm.f[args.fcur ^ 1]);
    const R* __restrict__ auxc = static_cast<const R*>(dm.aux[args.acur]);
    R* __restrict__ auxn = static_cast<R*>(dm.aux[args.acur ^ 1]);
    const int8_t* __restrict__ Ic = dm.I[args.cur];
    int8_t* __restrict__ In = dm.I[args.cur ^ 1];
    // advective heat equilibrium: U at the aux time level, a in the kernel's
    // axes (a 2D domain's y axis is the kernel's z)
    const bool advect = ADV && dm.advect != 0;
    const bool need_U = advect && collide;
    const R* __restrict__ Uc = ADV ? static_cast<const R*>(dm.U[args.acur]) : nullptr;
    R* __restrict__ Un = ADV ? static_cast<R*>(dm.U[args.acur ^ 1]) : nullptr;
    const R ax = ADV ? R(dm.adv[0]) : R(0);
    const R ay = (ADV && !XZV) ? R(dm.adv[1]) : R(0);
    const R az = ADV ? R(XZV ? dm.adv[1] : dm.adv[2]) : R(0);
    (void)ay;

    constexpr bool SR = UsesSR<S>::value;
    const uint32_t seed = SR ? (uint32_t)args.counters[2 + args.cur] : 0u;
    (void)seed;
    // 16-bit deviation store: round to nearest, or stochastically
    auto store_dev = [&](T* p, R v, uint32_t h, uint32_t pop) {
        if constexpr (SR)
            *p = from_real_sr<T>(v, sr_bits(h, pop));
        else
            *p = from_real<T, R>(v);
    };
    const R Dphi = R(dm.Dphi);
    const R De2 = R(dm.Dphi / PL::E2);
    const R qphi = R(dm.qphi);
    const R lam = R(dm.lambda);
    const R ieu = R(dm.inv_eta_u);
    const R om_u = R(1) - ieu;
    // index threshold; in FP32 not below the rounding noise of the gradient (1e-6)
    const R xi2 = sizeof(R) == 4 ? R(fmax(dm.xi_lu, 1e-6) * fmax(dm.xi_lu, 1e-6)) : R(dm.xi_lu * dm.xi_lu);
    (void)Dphi;

    // walled axes of the kernel's view (a 2D domain's y axis is the kernel's z)
    const int bcm = WALLS ? dm.bc : 0;
    const bool wX = (bcm & LBPF_BC_WALL_X) != 0;
    const bool wY = !XZV && (bcm & LBPF_BC_WALL_Y) != 0;
    const bool wZ = XZV ? (bcm & LBPF_BC_WALL_Y) != 0 : (bcm & LBPF_BC_WALL_Z) != 0;
    auto wrapx = [&](int v) {
        if (WALLS && wX) return reflect_index(v, nx);
        return v < 0 ? v + nx : (v >= nx ? v - nx : v);
    };
    auto wrapy = [&](int v) {
        if (WALLS && wY) return reflect_index(v, ny);
        return v < 0 ? v + ny : (v >= ny ? v - ny : v);
    };
    auto wrapz = [&](int v) {
        if (WALLS && wZ) return reflect_index(v, nz);
        return v < 0 ? v + nz : (v >= nz ? v - nz : v);
    };
    // a site inside the domain on one of its walls
    auto on_wall = [&](int gx, int gy, int gz) {
        return (wX && (gx == 0 || gx == nx - 1)) || (wY && (gy == 0 || gy == ny - 1)) ||
               (wZ && (gz == 0 || gz == nz - 1));
    };
    // walls the site lies on, low and high end of each axis (bit = axis)
    auto wall_lo = [&](int gx, int gy, int gz) {
        return (wX && gx == 0 ? 1 : 0) | (wY && gy == 0 ? 2 : 0) | (wZ && gz == 0 ? 4 : 0);
    };
    auto wall_hi = [&](int gx, int gy, int gz) {
        return (wX && gx == nx - 1 ? 1 : 0) | (wY && gy == ny - 1 ? 2 : 0) | (wZ && gz == nz - 1 ? 4 : 0);
    };
    auto sphi = [&](int zp) { return (zp + 2 * NPH) % NPH; };
    auto sh = [&](int zp) { return (zp + 2 * NH) % NH; };
    auto sco = [&](int zp) { return (zp + 3) % NC; };

    // -- asynchronous copy (cp.async) of one plane of phi^n and aux on the
    // tile + 2-site halo into the rings, issued one plane ahead of its use so
    // that the loads overlap the coefficient and output phases; finish_plane
    // then waits for the thread's own copies and forms h = aux + phi^n / 2 in
    // place on the items that thread copied (a barrier follows before use).
    auto async_plane = [&](int zp) {
        const long long zo = (long long)wrapz(zp) * nxy;
        R* dphi = s_phi + sphi(zp) * RP;
        R* dh = s_h + sh(zp) * RP;
        R* dU = s_U + sh(zp) * RP;
        int8_t* dI = s_I + sphi(zp) * RP;
        const int rows = th + 2 * HL;
        constexpr int EPC = 16 / (int)sizeof(R), NCH = TXT / EPC;
        auto cp4 = [&](R* d, const R* g) {
            asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((unsigned)__cvta_generic_to_shared(d)), "l"(g),
                         "n"((int)sizeof(R)));
        };
        auto cp16 = [&](R* d, const R* g) {
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(d)), "l"(g));
        };
        if (CHUNKED && tw == TXT && nx % EPC == 0) {
            // full tile: interior rows in 16-byte chunks (L2 only), the four
            // halo columns element by element
            const int nint = rows * NCH, nall = nint + rows * 4;
            for (int t = tid; t < nall; t += NT) {
                if (t < nint) {
                    const int ly = t / NCH, c = t - ly * NCH;
                    const long long s = zo + (long long)wrapy(y0 + ly - HL) * nx + x0 + c * EPC;
                    const int k = ly * RX + XO + c * EPC;
                    cp16(dphi + k, phic + s);
                    if (need_h) cp16(dh + k, auxc + s);
                    if (need_U) cp16(dU + k, Uc + s);
                } else {
                    const int u = t - nint, ly = u >> 2, q = u & 3;
                    const int lx = q < 2 ? XO - 2 + q : XO + TXT + (q - 2);
                    const long long s = zo + (long long)wrapy(y0 + ly - HL) * nx + wrapx(x0 + lx - XO);
                    const int k = ly * RX + lx;
                    cp4(dphi + k, phic + s);
                    if (need_h) cp4(dh + k, auxc + s);
                    if (need_U) cp4(dU + k, Uc + s);
                }
            }
            if (use_index)
                for (int k = tid; k < RX * rows; k += NT) {
                    const int ly = k / RX, lx = k - ly * RX;
                    if (lx < XO - 2 || lx >= XO + tw + 2) continue;
                    dI[k] = Ic[zo + (long long)wrapy(y0 + ly - HL) * nx + wrapx(x0 + lx - XO)];
                }
        } else {
            for (int k = tid; k < RX * rows; k += NT) {
                const int ly = k / RX, lx = k - ly * RX;
                if (lx < XO - 2 || lx >= XO + tw + 2) continue;
                const long long s = zo + (long long)wrapy(y0 + ly - HL) * nx + wrapx(x0 + lx - XO);
                cp4(dphi + k, phic + s);
                if (need_h) cp4(dh + k, auxc + s);
                if (need_U) cp4(dU + k, Uc + s);
                if (use_index) dI[k] = Ic[s];
            }
        }
        asm volatile("cp.async.commit_group;");
    };
    auto finish_plane = [&](int zp) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        if (!need_h) return;
        const R* dphi = s_phi + sphi(zp) * RP;
        R* dh = s_h + sh(zp) * RP;
        const int rows = th + 2 * HL;
        constexpr int EPC = 16 / (int)sizeof(R), NCH = TXT / EPC;
        if (CHUNKED && tw == TXT && nx % EPC == 0) {  // the tasks of async_plane's chunked path
            const int nint = rows * NCH, nall = nint + rows * 4;
            for (int t = tid; t < nall; t += NT) {
                if (t < nint) {
                    const int ly = t / NCH, c = t - ly * NCH;
                    const int k = ly * RX + XO + c * EPC;
#pragma unroll
                    for (int e = 0; e < EPC; ++e) dh[k + e] += R(0.5) * dphi[k + e];
                } else {
                    const int u = t - nint, ly = u >> 2, q = u & 3;
                    const int k = ly * RX + (q < 2 ? XO - 2 + q : XO + TXT + (q - 2));
                    dh[k] += R(0.5) * dphi[k];
                }
            }
            return;
        }
        for (int k = tid; k < RX * rows; k += NT) {
            const int ly = k / RX, lx = k - ly * RX;
            if (lx < XO - 2 || lx >= XO + tw + 2) continue;
            dh[k] += R(0.5) * dphi[k];
        }
    };

    // -- load one plane of phi^n (and h, I) on the tile + 2-site halo (the
    // prologue of a work item) -------------------------------------------------
    auto load_plane = [&](int zp) {
        const long long zo = (long long)wrapz(zp) * nxy;
        R* dphi = s_phi + sphi(zp) * RP;
        R* dh = s_h + sh(zp) * RP;
        R* dU = s_U + sh(zp) * RP;
        int8_t* dI = s_I + sphi(zp) * RP;
        const int rows = th + 2 * HL;
        for (int k = tid; k < RX * rows; k += NT) {
            const int ly = k / RX, lx = k - ly * RX;
            if (lx < XO - 2 || lx >= XO + tw + 2) continue;
            const long long s = zo + (long long)wrapy(y0 + ly - HL) * nx + wrapx(x0 + lx - XO);
            const R ph = phic[s];
            dphi[k] = ph;
            if (need_h) dh[k] = auxc[s] + R(0.5) * ph;
            if (need_U) dU[k] = Uc[s];
            if (use_index) dI[k] = Ic[s];
        }
    };

    // -- heat update, gradient, anisotropy, collision coefficients ----------
    // on one plane of the tile + 1-site halo; heat outputs of the tile
    // interior are stored when `store` is set.
    // f_j on the phi frame of plane zp - ez_j (the pull sources of
    // coef_plane(zp)) by cp.async into s_f
    auto stage_f = [&](int zp) {
        const int rows = th + 2 * HL;
        for (int k = tid; k < RX * rows; k += NT) {
            const int ly = k / RX, lx = k - ly * RX;
            if (lx < XO - 2 || lx >= XO + tw + 2) continue;
            const long long rowx = (long long)wrapy(y0 + ly - HL) * nx + wrapx(x0 + lx - XO);
#pragma unroll
            for (int j = 0; j < QU; ++j) {
                const long long s = (long long)wrapz(zp - UL::ez(j)) * nxy + rowx;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                                 (unsigned)__cvta_generic_to_shared(s_f + j * RP + k)),
                             "l"(fc + (long long)j * n + s));
            }
        }
        asm volatile("cp.async.commit_group;");
    };

    auto coef_plane = [&](int zp, bool store, bool staged) {
        const int zw = wrapz(zp);
        const long long zo = (long long)zw * nxy;
        const int zm = wrapz(zp - 1), zq = wrapz(zp + 1);
        const long long ozm = (long long)(zm - zw) * nxy, ozp = (long long)(zq - zw) * nxy;
        R* dco = s_co + sco(zp) * COP;
        const int rows = th + 2 * HC;
        for (int k = tid; k < CX * rows; k += NT) {
            const int ly = k / CX, lx = k - ly * CX;
            if (lx >= tw + 2) continue;
            const int px = lx + XO - 1, py = ly + HL - HC;  // position in the phi frame
            const int gx = wrapx(x0 + lx - 1), gy = wrapy(y0 + ly - HC);
            const long long s = zo + (long long)gy * nx + gx;
            const bool inner = store && lx >= 1 && lx <= tw && ly >= HC && ly < th + HC;
            const R ph = s_phi[sphi(zp) * RP + py * RX + px];

            // offsets of the periodic neighbours of s
            const int gxm = wrapx(gx - 1), gxp = wrapx(gx + 1);
            const int gym = wrapy(gy - 1), gyp = wrapy(gy + 1);
            const long long oxm = gxm - gx, oxp = gxp - gx;
            const long long oym = (long long)(gym - gy) * nx, oyp = (long long)(gyp - gy) * nx;
            auto off = [&](int ex, int ey, int ez) -> long long {
                return (ex < 0 ? oxm : (ex > 0 ? oxp : 0)) + (ey < 0 ? oym : (ey > 0 ? oyp : 0)) +
                       (D == 3 ? (ez < 0 ? ozm : (ez > 0 ? ozp : 0)) : 0);
            };

            // u^n at this site
            R u = 0;
            if (collide) {
                R fv[QU];
                R d0 = 0;
                if (DEV) {
#pragma unroll
                    for (int j = 1; j < QU; ++j) d0 -= to_real(fc[(long long)(j - 1) * n + s]);
                }
#pragma unroll
                for (int j = 0; j < QU; ++j) {
                    const int ex = UL::ex(j), ey = UL::ey(j), ez = UL::ez(j);
                    const R hs = s_h[sh(zp - ez) * RP + (py - ey) * RX + (px - ex)];
                    const long long src = s + off(-ex, -ey, -ez);
                    R fj;
                    if (!DEV) {
                        const R fr = (STF && staged) ? to_real(s_f[j * RP + (py - ey) * RX + (px - ex)])
                                                     : to_real(fc[(long long)j * n + src]);
                        fj = om_u * fr + R(UL::w(j)) * hs;
                    } else {
                        const R dj = (j == 0) ? d0 : to_real(fc[(long long)(j - 1) * n + src]);
                        fj = R(UL::w(j)) * hs + om_u * dj;
                    }
                    if constexpr (ADV) {
                        if (advect && (ex | ey | ez)) {
                            const R ea = R(ex) * ax + R(ey) * ay + R(ez) * az;
                            fj += R(UL::w(j)) * ea * s_U[sh(zp - ez) * RP + (py - ey) * RX + (px - ex)];
                        }
                    }
                    fv[j] = fj;
                    u += fj;
                }
                if constexpr (WALLS) {
                    // a site inside the domain on a wall: heat populations
                    // from beyond the wall are their mirrored partners
                    // (frame sites beyond a wall are ghosts whose values are
                    // never used; along periodic axes every frame site is real)
                    const int gxu = x0 + lx - 1, gyu = y0 + ly - HC;
                    const bool real = (!wX || (gxu >= 0 && gxu < nx)) && (!wY || (gyu >= 0 && gyu < ny)) &&
                                      (!wZ || (zp >= 0 && zp < nz));
                    if (bcm && real && on_wall(gx, gy, zw)) {
                        mirror_refill<UL, R>(fv, wall_lo(gx, gy, zw), wall_hi(gx, gy, zw));
                        u = 0;
#pragma unroll
                        for (int j = 0; j < QU; ++j) u += fv[j];
                    }
                }
                if (inner) {
                    if (!DEV) {
#pragma unroll
                        for (int j = 0; j < QU; ++j) fn[(long long)j * n + s] = from_real<T, R>(fv[j]);
                    } else {
                        const uint32_t h = SR ? sr_hash((uint32_t)s, seed) : 0u;
#pragma unroll
                        for (int j = 1; j < QU; ++j)
                            store_dev(&fn[(long long)(j - 1) * n + s], fv[j] - R(UL::w(j)) * u, h, 32u + j);
                    }
                }
            } else {
                if (!DEV) {
#pragma unroll
                    for (int j = 0; j < QU; ++j) u += to_real(fc[(long long)j * n + s]);
                } else {
                    u = s_h[sh(zp) * RP + py * RX + px];  // C^n + phi^n / 2
                }
            }
            if (inner) auxn[s] = DEV ? (u - R(0.5) * ph) : (u * ieu - R(0.5) * ph);
            if constexpr (ADV) {
                if (inner && advect) Un[s] = u * ieu;
            }

            // gradient of phi^n (Sec. 4.2)
            R Gx = 0, Gy = 0, Gz = 0;
            if (args.grad == LBPF_GRAD_DD) {
                // Eq. (Def_DeriveeDirectionnelle) and Eq. (Grad_DF-Centree); a
                // direction and its opposite give the same term, so each pair is
                // taken once with twice the weight.
#pragma unroll
                for (int i = 1; i < QG; ++i) {
                    if (i > opposite<PL>(i)) continue;
                    const int ex = PL::ex(i), ey = PL::ey(i), ez = PL::ez(i);
                    const R dd = s_phi[sphi(zp + ez) * RP + (py + ey) * RX + (px + ex)] -
                                 s_phi[sphi(zp - ez) * RP + (py - ey) * RX + (px - ex)];
                    const R wd = R(PL::w(i)) * dd;
                    if (ex) Gx += R(ex) * wd;
                    if (ey) Gy += R(ey) * wd;
                    if (ez) Gz += R(ez) * wd;
                }
                const R k = R(1.0 / PL::E2);
                Gx *= k;
                Gy *= k;
                Gz *= k;
            } else {
                const R* pl = s_phi + sphi(zp) * RP;
                Gx = R(0.5) * (pl[py * RX + px + 1] - pl[py * RX + px - 1]);
                if (!XZV) Gy = R(0.5) * (pl[(py + 1) * RX + px] - pl[(py - 1) * RX + px]);
                Gz = R(0.5) * (s_phi[sphi(zp + 1) * RP + py * RX + px] - s_phi[sphi(zp - 1) * RP + py * RX + px]);
            }

            // crystal index (Sec. 4.3): keep a non-zero index; otherwise take
            // the first non-zero neighbour (axes before diagonals) where
            // |grad phi| > xi.
            int cryst = 1;
            if (use_index) {
                int Iv = s_I[sphi(zp) * RP + py * RX + px];
                if (Iv == 0 && Gx * Gx + Gy * Gy + Gz * Gz > xi2) {
#pragma unroll
                    for (int i = 1; i < QG; ++i) {
                        const int ex = PL::ex(i), ey = PL::ey(i), ez = PL::ez(i);
                        const int v = s_I[sphi(zp + ez) * RP + (py + ey) * RX + (px + ex)];
                        if (Iv == 0 && v != 0) Iv = v;
                    }
                }
                if (inner) In[s] = (int8_t)Iv;
                cryst = Iv;
            }

            R a = 1, Nx = 0, Ny = 0, Nz = 0;
            if (cryst > 0 && cryst <= dm.n_crystals) {
                if (XZV) {  // physical (x, y) = kernel (x, z)
                    R n2 = 0;
                    anisotropy<R, 2>(dm.cr[cryst - 1], Gx, Gz, R(0), a, Nx, Nz, n2);
                } else {
                    anisotropy<R, D>(dm.cr[cryst - 1], Gx, Gy, Gz, a, Nx, Ny, Nz);
                }
            }

            const R A2 = a * a;
            const R iA2 = recip<R>(A2);
            const R ieta = recip<R>(A2 * De2 + R(0.5));
            const R omp = (R(1) - ph) * (R(1) + ph);
            const R Qphi = (ph - lam * u * omp) * omp;
            const R vf = -De2 * ieta * iA2;
            // with deviation storage the source coefficient also carries
            // c1 phi (x): c1 (w_i phi + d_i) + w_i s = c1 d_i + w_i (s + c1 phi),
            // and s + c1 phi = (phi + (dt/tau0) Q_phi) / a_s^2
            const R sc = DEV ? (ph + qphi * Qphi) * iA2 : (ph * ieta + qphi * Qphi) * iA2;
            CoefIO<R>::store(dco, CP, ly * CX + lx, (R(1) - ieta) * iA2, iA2 - R(1), sc, vf * Nx, vf * Ny, vf * Nz);
        }
    };

    // -- phase-field collision + streaming for the tile interior of plane z ----
    auto output_plane = [&](int z) {
        const int ltx = tid % TXT, lty = tid / TXT;
        if (ltx >= tw || lty >= th) return;
        const int gx = x0 + ltx, gy = y0 + lty;
        const long long s = (long long)z * nxy + (long long)gy * nx + gx;
        const int gxm = wrapx(gx - 1), gxp = wrapx(gx + 1);
        const int gym = wrapy(gy - 1), gyp = wrapy(gy + 1);
        const long long oxm = gxm - gx, oxp = gxp - gx;
        const long long oym = (long long)(gym - gy) * nx, oyp = (long long)(gyp - gy) * nx;
        long long ozm = 0, ozp = 0;
        if (D == 3) {
            ozm = (long long)(wrapz(z - 1) - z) * nxy;
            ozp = (long long)(wrapz(z + 1) - z) * nxy;
        }
        auto off = [&](int ex, int ey, int ez) -> long long {
            return (ex < 0 ? oxm : (ex > 0 ? oxp : 0)) + (ey < 0 ? oym : (ey > 0 ? oyp : 0)) +
                   (D == 3 ? (ez < 0 ? ozm : (ez > 0 ? ozp : 0)) : 0);
        };
        const int px = ltx + XO, py = lty + HL;  // phi frame
        const int cx = ltx + 1, cy = lty + HC;  // coefficient frame
        // Deviation storage and D2Q9 read each local population in the
        // direction loop, so that only the new populations stay live, and
        // round explicitly (pull_new), as the staged kernel does; with
        // deviation storage the rest population comes last: its deviation
        // d0 = -sum of the others.  The 3D lattices with full storage read
        // their local populations first (more loads in flight), and D3Q15 /
        // D3Q19 leave contraction to the compiler: measured at 256^3 FP32,
        // D3Q15 21.3 / 20.7, D3Q19 18.9 / 16.7, D3Q27 12.7 (explicit) / 12.3
        // GLUPS against the in-loop explicit form; reading first cost 12 %
        // on D3Q19 FP16.
        constexpr bool LOCAL_FIRST = !DEV && QG >= 15;
        constexpr bool CONTRACT = !DEV && (QG == 15 || QG == 19);
        const R phy = DEV ? s_phi[sphi(z) * RP + py * RX + px] : R(0);
        R loc[LOCAL_FIRST ? QG : 1];
        if constexpr (LOCAL_FIRST) {
#pragma unroll
            for (int i = DEV ? 1 : 0; i < QG; ++i) loc[i] = to_real(gc[(long long)(DEV ? i - 1 : i) * n + s]);
        }
        R gnew[QG];
        R phinew = 0, d0 = 0;
#pragma unroll
        for (int k = 0; k < QG; ++k) {
            const int i = DEV ? (k + 1) % QG : k;
            const int ex = PL::ex(i), ey = PL::ey(i), ez = PL::ez(i);
            R c1, c2, cs, vx, vy, vz;
            CoefIO<R>::load(s_co + sco(z - ez) * COP, CP, (cy - ey) * CX + (cx - ex), ey != 0 || ez != 0, c1, c2,
                            cs, vx, vy, vz);
            // gl: g_i(y) (the non-local term); gp: full storage g_i(x),
            // deviation storage d_i(x) (w_i phi(x) is in cs)
            R gl, gp;
            if (!DEV) {
                gl = LOCAL_FIRST ? loc[LOCAL_FIRST ? i : 0] : to_real(gc[(long long)i * n + s]);
                gp = i == 0 ? gl : to_real(gc[(long long)i * n + s + off(-ex, -ey, -ez)]);
            } else if (i > 0) {
                const R d = LOCAL_FIRST ? loc[LOCAL_FIRST ? i : 0] : to_real(gc[(long long)(i - 1) * n + s]);
                d0 = sub_rn(d0, d);
                gl = fma_rn(R(PL::w(i)), phy, d);
                gp = to_real(gc[(long long)(i - 1) * n + s + off(-ex, -ey, -ez)]);
            } else {
                gl = fma_rn(R(PL::w(0)), phy, d0);
                gp = d0;
            }
            R v;
            if constexpr (CONTRACT) {
                R ev = R(0);
                if (ex) ev += R(ex) * vx;
                if (ey) ev += R(ey) * vy;
                if (ez) ev += R(ez) * vz;
                v = c1 * gp - c2 * gl + R(PL::w(i)) * (cs + ev);
                phinew += v;
            } else {
                v = pull_new<R>(ex, ey, ez, R(PL::w(i)), c1, c2, cs, vx, vy, vz, gp, gl);
                phinew = add_rn(phinew, v);
            }
            gnew[i] = v;
        }
        if constexpr (WALLS) {
            if (bcm && on_wall(gx, gy, z)) {
                // populations whose source lies beyond a wall: mirrored partners
                mirror_refill<PL, R>(gnew, wall_lo(gx, gy, z), wall_hi(gx, gy, z));
                phinew = 0;
#pragma unroll
                for (int i = 0; i < QG; ++i) phinew += gnew[i];
            }
        }
        phin[s] = phinew;
        if (!DEV) {
#pragma unroll
            for (int i = 0; i < QG; ++i) gn[(long long)i * n + s] = from_real<T, R>(gnew[i]);
        } else {
            const uint32_t h = SR ? sr_hash((uint32_t)s, seed) : 0u;
#pragma unroll
            for (int i = 1; i < QG; ++i)
                store_dev(&gn[(long long)(i - 1) * n + s], fma_rn(-R(PL::w(i)), phinew, gnew[i]), h, (uint32_t)i);
        }
    };

    {
        const int z0 = it.z0, z1 = it.z1;
        if constexpr (!DEV) {  // prologue copies asynchronous too (+3 % FP32, -2 % deviations: measured)
            for (int p = z0 - 2; p <= z0 + 1; ++p) async_plane(p);
            for (int p = z0 - 2; p <= z0 + 1; ++p) finish_plane(p);
        } else {
            load_plane(z0 - 2);
            load_plane(z0 - 1);
            load_plane(z0);
            load_plane(z0 + 1);
        }
        __syncthreads();
        coef_plane(z0 - 1, false, false);
        coef_plane(z0, true, false);
        __syncthreads();
        async_plane(z0 + 2);
        const bool stf = STF && collide;
        if (stf) stage_f(z0 + 1);
        for (int z = z0; z < z1; ++z) {
            finish_plane(z + 2);
            if (z + 3 <= z1 + 1) async_plane(z + 3);
            __syncthreads();
            coef_plane(z + 1, z + 1 < z1, stf);
            __syncthreads();
            if (stf && z + 2 <= z1) stage_f(z + 2);
            output_plane(z);
            // no barrier here: the next writes into the rings (finish z+3,
            // copy z+4) touch slots no warp still in output_plane(z) reads,
            // and coef_plane(z+2), which overwrites a coefficient plane that
            // output_plane(z) reads, comes after the next barrier
        }
    }
}

// Persistent launch with dynamic scheduling: as many blocks as fit on the GPU
// take work items in list order from a counter.  The host orders the items
// z-segment by z-segment, so that the blocks running at any moment hold
// neighbouring columns at similar heights and their halo rims are served by L2.
// The launch uses counter[cur] and clears counter[cur ^ 1] for the next step
// (launches on one stream run in order; cur alternates every step).
// Launch bounds ask for 1024 resident threads per SM (64 registers a thread).
template <class PL, class UL, class S, int TXT, int TY, bool WALLS, bool ADV = false>
__global__ void __launch_bounds__(TXT * TY, 1024 / (TXT * TY)) step_kernel(const StepArgs args)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_next;
    int* counter = args.counters + args.cur;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        args.counters[args.cur ^ 1] = 0;
        if constexpr (UsesSR<S>::value)
            args.counters[2 + (args.cur ^ 1)] = args.counters[2 + args.cur] + 1;  // next step's rounding seed
    }
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(counter, 1);
        __syncthreads();
        const int k = s_next;
        if (k >= args.n_items) break;
        step_item<PL, UL, S, TXT, TY, WALLS, ADV>(args, args.items[k], smem_raw);
        __syncthreads();
    }
}

template <class PL, class UL, class S, int TXT, int TY, bool ADV = false>
constexpr size_t step_smem_bytes()
{
    using R = typename S::Real;
    constexpr int HL = IsXZ<PL>::value ? 0 : 2, HC = IsXZ<PL>::value ? 0 : 1;
    constexpr int XO = (IsXZ<PL>::value || sizeof(R) >= 8) ? 2 : 4;
    constexpr int RP = (TXT + 2 * XO) * (TY + 2 * HL), CP = (TXT + 2) * (TY + 2 * HC);
    constexpr int NPH = 5, NH = 4, NC = 3;
    constexpr int COP = 6 * CP;
    return sizeof(R) * (size_t)(NPH * RP + NH * RP + NC * COP) + (((size_t)NPH * RP + 15) & ~size_t(15)) +
           stf_bytes<UL, S, IsXZ<PL>::value>(RP) + (ADV ? sizeof(R) * (size_t)NH * RP : 0);
}

}  // namespace lbpf
