// Internal definitions of the lbpf CUDA library: lattice tables, per-domain
// device parameters, storage policies and the anisotropy/coefficient
// arithmetic shared by the kernels of this library.
//
// Method: Younsi & Cartalade, arXiv:1606.09432 (phase-field LB scheme of
// Sec. 3.2, heat LB scheme of Sec. 3.1, lattices of Sec. 3.3, gradients of
// Sec. 4.2, anisotropy functions of Secs. 2, 4.1, 4.3 and 5.2).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/lbpf.h"

namespace lbpf {

constexpr int kMaxCrystals = LBPF_MAX_CRYSTALS;

// ---------------------------------------------------------------------------
// Lattices (Sec. 3.3, Table 1).  Direction numbering follows the paper for
// D2Q5, D2Q9, D3Q7 and D3Q15; D3Q19/D3Q27 list the axes (as D3Q7), then the
// xy-, xz- and yz-edges, then the cube corners (as D3Q15).
// ---------------------------------------------------------------------------
#define LBPF_HD __host__ __device__ __forceinline__

struct D2Q5 {
    static constexpr int D = 2, Q = 5;
    static constexpr double E2 = 1.0 / 3.0;
    LBPF_HD static constexpr int ex(int i) { constexpr int t[5] = {0, 1, 0, -1, 0}; return t[i]; }
    LBPF_HD static constexpr int ey(int i) { constexpr int t[5] = {0, 0, 1, 0, -1}; return t[i]; }
    LBPF_HD static constexpr int ez(int) { return 0; }
    LBPF_HD static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }
};

struct D2Q9 {
    static constexpr int D = 2, Q = 9;
    static constexpr double E2 = 1.0 / 3.0;
    LBPF_HD static constexpr int ex(int i) { constexpr int t[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}; return t[i]; }
    LBPF_HD static constexpr int ey(int i) { constexpr int t[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1}; return t[i]; }
    LBPF_HD static constexpr int ez(int) { return 0; }
    LBPF_HD static constexpr double w(int i) { return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }
};

struct D3Q7 {
    static constexpr int D = 3, Q = 7;
    static constexpr double E2 = 1.0 / 4.0;
    LBPF_HD static constexpr int ex(int i) { constexpr int t[7] = {0, 1, 0, -1, 0, 0, 0}; return t[i]; }
    LBPF_HD static constexpr int ey(int i) { constexpr int t[7] = {0, 0, 1, 0, -1, 0, 0}; return t[i]; }
    LBPF_HD static constexpr int ez(int i) { constexpr int t[7] = {0, 0, 0, 0, 0, 1, -1}; return t[i]; }
    LBPF_HD static constexpr double w(int i) { return i == 0 ? 1.0 / 4.0 : 1.0 / 8.0; }
};

// 27 velocity components in the order: rest, 6 axes, 12 edges, 8 corners.
LBPF_HD constexpr int q27x(int i)
{
    constexpr int t[27] = {0, 1, 0, -1, 0, 0, 0,
                           1, -1, -1, 1, 1, -1, -1, 1, 0, 0, 0, 0,
                           1, -1, -1, 1, 1, -1, -1, 1};
    return t[i];
}
LBPF_HD constexpr int q27y(int i)
{
    constexpr int t[27] = {0, 0, 1, 0, -1, 0, 0,
                           1, 1, -1, -1, 0, 0, 0, 0, 1, -1, -1, 1,
                           1, 1, -1, -1, 1, 1, -1, -1};
    return t[i];
}
LBPF_HD constexpr int q27z(int i)
{
    constexpr int t[27] = {0, 0, 0, 0, 0, 1, -1,
                           0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1,
                           1, 1, 1, 1, -1, -1, -1, -1};
    return t[i];
}

struct D3Q15 {  // rest, axes, corners
    static constexpr int D = 3, Q = 15;
    static constexpr double E2 = 1.0 / 3.0;
    LBPF_HD static constexpr int m(int i) { return i < 7 ? i : i + 12; }
    LBPF_HD static constexpr int ex(int i) { return q27x(m(i)); }
    LBPF_HD static constexpr int ey(int i) { return q27y(m(i)); }
    LBPF_HD static constexpr int ez(int i) { return q27z(m(i)); }
    LBPF_HD static constexpr double w(int i) { return i == 0 ? 2.0 / 9.0 : (i <= 6 ? 1.0 / 9.0 : 1.0 / 72.0); }
};

struct D3Q19 {  // rest, axes, edges
    static constexpr int D = 3, Q = 19;
    static constexpr double E2 = 1.0 / 3.0;
    LBPF_HD static constexpr int ex(int i) { return q27x(i); }
    LBPF_HD static constexpr int ey(int i) { return q27y(i); }
    LBPF_HD static constexpr int ez(int i) { return q27z(i); }
    LBPF_HD static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
};

struct D3Q27 {  // rest, axes, edges, corners
    static constexpr int D = 3, Q = 27;
    static constexpr double E2 = 1.0 / 3.0;
    LBPF_HD static constexpr int ex(int i) { return q27x(i); }
    LBPF_HD static constexpr int ey(int i) { return q27y(i); }
    LBPF_HD static constexpr int ez(int i) { return q27z(i); }
    LBPF_HD static constexpr double w(int i)
    {
        return i == 0 ? 8.0 / 27.0 : (i <= 6 ? 2.0 / 27.0 : (i <= 18 ? 1.0 / 54.0 : 1.0 / 216.0));
    }
};

template <int L> struct Pair;
template <> struct Pair<LBPF_D2Q9_D2Q5> { using P = D2Q9; using U = D2Q5; };
template <> struct Pair<LBPF_D3Q15_D3Q7> { using P = D3Q15; using U = D3Q7; };
template <> struct Pair<LBPF_D3Q19_D3Q7> { using P = D3Q19; using U = D3Q7; };
template <> struct Pair<LBPF_D3Q27_D3Q7> { using P = D3Q27; using U = D3Q7; };

// ---------------------------------------------------------------------------
// Storage policies.  Full storage keeps all Q populations in the arithmetic
// type; deviation storage keeps d_i = p_i - w_i m (m the zeroth moment) for
// i >= 1 in 16 bits and rebuilds p_0 = w_0 m - sum_{i>=1} d_i.
// ---------------------------------------------------------------------------
struct StoreF64 { using Real = double; using T = double; static constexpr bool dev = false; };
struct StoreF32 { using Real = float; using T = float; static constexpr bool dev = false; };
struct StoreF16 { using Real = float; using T = __half; static constexpr bool dev = true; };
struct StoreB16 { using Real = float; using T = __nv_bfloat16; static constexpr bool dev = true; };
// as above, deviations rounded stochastically
struct StoreF16SR : StoreF16 { static constexpr bool sr = true; };
template <class S, class = void> struct UsesSR { static constexpr bool value = false; };
template <class S> struct UsesSR<S, decltype(void(S::sr))> { static constexpr bool value = S::sr; };

__device__ __forceinline__ float to_real(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_real(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_real(float v) { return v; }
__device__ __forceinline__ double to_real(double v) { return v; }

template <class T, class R> __device__ __forceinline__ T from_real(R v);
template <> __device__ __forceinline__ double from_real<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float from_real<float, float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_real<__half, float>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_real<__nv_bfloat16, float>(float v) { return __float2bfloat16_rn(v); }

// Stochastic rounding of 16-bit deviations: round up or down with
// probabilities proportional to the distances, so that rounding errors of
// slowly varying values do not add up step after step.  Random bits come from
// a hash of (site, population, step seed) (lowbias32 finaliser, Wellons 2018),
// so results are reproducible.
__device__ __forceinline__ uint32_t sr_hash(uint32_t site, uint32_t seed)
{
    uint32_t x = site * 0x9E3779B9u ^ seed * 0xC2B2AE35u;
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
// Bits for population `pop` from the site hash h (one multiply-xorshift).
__device__ __forceinline__ uint32_t sr_bits(uint32_t h, uint32_t pop)
{
    uint32_t x = (h ^ (pop * 0x9E3779B9u)) * 0x85EBCA6Bu;
    return x ^ (x >> 13);
}

template <class T> __device__ __forceinline__ T from_real_sr(float v, uint32_t rnd);
// full-precision storage: nothing to round stochastically
template <> __device__ __forceinline__ float from_real_sr<float>(float v, uint32_t) { return v; }
template <> __device__ __forceinline__ double from_real_sr<double>(float v, uint32_t) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_real_sr<__nv_bfloat16>(float v, uint32_t rnd)
{
    const uint32_t b = __float_as_uint(v);
    if (((b >> 23) & 0xFF) == 0xFF) return __float2bfloat16_rn(v);  // Inf, NaN
    // add 16 random bits below the BF16 mantissa, then truncate
    return __ushort_as_bfloat16((unsigned short)((b + (rnd & 0xFFFFu)) >> 16));
}
template <> __device__ __forceinline__ __half from_real_sr<__half>(float v, uint32_t rnd)
{
    const uint32_t b = __float_as_uint(v);
    int e = (int)((b >> 23) & 0xFF) - 127;
    if (e > 15) return __float2half_rn(v);  // beyond the FP16 range (and Inf, NaN)
    if (e < -14) e = -14;                   // FP16 subnormal spacing 2^-24
    const float ulp = __uint_as_float((uint32_t)(e - 10 + 127) << 23);
    const float r = (float)(rnd >> 8) * (1.0f / 16777216.0f) - 0.5f;  // U[-1/2, 1/2)
    return __float2half_rn(v + r * ulp);
}

// Number of stored arrays per population set.
template <class S, int Q> struct NStored { static constexpr int value = S::dev ? Q - 1 : Q; };

// ---------------------------------------------------------------------------
// Per-domain device parameters and buffers.
// ---------------------------------------------------------------------------
struct CrystalDev {
    int kind;
    int q;
    double eps, gamma, phi0;
};

struct DomainDev {
    int nx, ny, nz;
    int bc;             // LBPF_BC_WALL_* bits (0: periodic)
    long long n;        // sites
    double Dphi;        // (W0^2 / tau0) (dt / dx^2), Eq. (LBE_RelaxationTime)
    double qphi;        // dt / tau0, source factor of Eq. (LBE_Eq_Phase)
    double lambda;      // coupling, Eq. (LBE_SourceTerm)
    double inv_eta_u;   // 1 / eta_u, Eq. (ThermalDiffusivity)
    double xi_lu;       // index threshold on |grad phi| in lattice units (xi dx)
    int n_crystals;
    int use_index;
    CrystalDev cr[kMaxCrystals];
    // Buffers (device pointers), typed by the storage policy in the kernels.
    void* g[2];         // phase-field populations (Q or Q-1 arrays of n)
    void* f[2];         // temperature populations
    void* phi[2];       // phi field, arithmetic type
    void* aux[2];       // heat auxiliary field (see the step kernel)
    int8_t* I[2];       // crystal index field (use_index only)
    // Advective heat equilibrium (advect only):
    //   f_i^(0) = w_i u (1 + e_i . a),  a = v dt / (dx e^2)
    // (physical axes; v the domain's uniform velocity), and U = u / eta_u of
    // the aux time level, which the heat pull reads at the source node.
    int advect;
    double adv[3];
    void* U[2];
};

// One thread block's work: a column of TX x TY sites over planes [z0, z1).
struct WorkItem {
    int dom, x0, y0, z0, z1, pad;
};

// Launch arguments of the fused step kernel.
struct StepArgs {
    const DomainDev* doms;
    const WorkItem* items;
    int n_items;
    int* counters;         // [0..1] work counters, [2..3] rounding seeds, used alternately;
                           // [4] device error word (1: a bounded wait of the staged kernel gave up)
    int cur;    // g / phi / I buffer holding time n (new = cur ^ 1)
    int fcur;   // f buffer read (f^{n-1} when collide, f^n when load)
    int acur;   // aux buffer read (new = acur ^ 1)
    int collide;
    int grad;   // LBPF_GRAD_DD / LBPF_GRAD_FD
};

// Tile of one thread block of the step kernel, one thread per site of a tile
// plane; the context picks variant v (autotuned):
//   3D: TX x kTileRows[v] sites of an xy-plane, marching along z;
//   2D: one row of kStripX[v] sites along x, marching along y (the kernel sees
//       the 2D lattice in its xz-plane, see XZ below).
constexpr int TX = 32;
constexpr int kNumTileVariants = 2;
constexpr int kTileRows[kNumTileVariants] = {8, 16};
constexpr int kStripX[kNumTileVariants] = {128, 256};
constexpr int tile_x(int dim, int v) { return dim == 3 ? TX : kStripX[v]; }
constexpr int tile_y(int dim, int v) { return dim == 3 ? kTileRows[v] : 1; }

// A 2D lattice seen by the step kernel in its xz-plane (e_y -> e_z), so that
// the kernel marches along the physical y axis as it marches along z in 3D and
// needs no halo across the strip (which is one row high).
template <class L> struct XZ {
    static_assert(L::D == 2, "XZ views a 2D lattice");
    static constexpr int D = 3, Q = L::Q;
    static constexpr bool xz = true;
    static constexpr double E2 = L::E2;
    LBPF_HD static constexpr int ex(int i) { return L::ex(i); }
    LBPF_HD static constexpr int ey(int) { return 0; }
    LBPF_HD static constexpr int ez(int i) { return L::ey(i); }
    LBPF_HD static constexpr double w(int i) { return L::w(i); }
};
template <class L, class = void> struct IsXZ { static constexpr bool value = false; };
template <class L> struct IsXZ<L, decltype(void(L::xz))> { static constexpr bool value = L::xz; };
// Lattice the step kernel is instantiated with.
template <class L> using KernelLattice = typename std::conditional<L::D == 2, XZ<L>, L>::type;

// Index of the direction of lattice L whose velocity is e_i with the
// components of the axes in mask (bit 0 x, 1 y, 2 z) reversed: the mirror
// image of e_i in walls normal to those axes.
template <class L>
LBPF_HD constexpr int reflect_dir(int i, int mask)
{
    const int tx = (mask & 1) ? -L::ex(i) : L::ex(i);
    const int ty = (mask & 2) ? -L::ey(i) : L::ey(i);
    const int tz = (mask & 4) ? -L::ez(i) : L::ez(i);
    for (int j = 0; j < L::Q; ++j)
        if (L::ex(j) == tx && L::ey(j) == ty && L::ez(j) == tz) return j;
    return -1;
}

// Values of the populations of a site on walls after the specular refill: a
// population whose source lies beyond the wall of axis a takes the value of
// its mirror image in that wall.  Applied axis by axis (x, then y, then z) as
// a permutation with a predicate per direction; a population beyond two or
// three walls (edges, corners) ends with the value of its image in all of
// them, the composition of the single reflections.  lo / hi: the site lies on
// the low / high wall of axis a (bit a).
template <class L, class R>
__device__ __forceinline__ void mirror_refill(R (&v)[L::Q], int lo, int hi)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!(((lo | hi) >> a) & 1)) continue;
        R t[L::Q];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const int e = a == 0 ? L::ex(i) : (a == 1 ? L::ey(i) : L::ez(i));
            const bool beyond = (((lo >> a) & 1) && e > 0) || (((hi >> a) & 1) && e < 0);
            t[i] = beyond ? v[reflect_dir<L>(i, 1 << a)] : v[i];
        }
#pragma unroll
        for (int i = 0; i < L::Q; ++i) v[i] = t[i];
    }
}

// Walls are mirror planes through the boundary nodes: index -k maps to k and
// n - 1 + k to n - 1 - k (n >= 3 for the offsets of at most 2 used here).
LBPF_HD int reflect_index(int v, int n) { return v < 0 ? -v : (v >= n ? 2 * (n - 1) - v : v); }

// Index of the direction opposite to i on lattice L.
template <class L>
LBPF_HD constexpr int opposite(int i)
{
    for (int j = 0; j < L::Q; ++j)
        if (L::ex(j) == -L::ex(i) && L::ey(j) == -L::ey(i) && L::ez(j) == -L::ez(i)) return j;
    return -1;
}

// 1/x: IEEE division in FP64; the hardware reciprocal (2 ulp) in FP32.
template <class R> __device__ __forceinline__ R recip(R x);
template <> __device__ __forceinline__ double recip<double>(double x) { return 1.0 / x; }
template <> __device__ __forceinline__ float recip<float>(float x) { return __fdividef(1.0f, x); }

// ---------------------------------------------------------------------------
// Anisotropy: a_s and N for a lattice-unit gradient G.  Written with the unit
// vector m = G / |G| = -n.  Every form used here except the angle form is an
// even polynomial of n, so a_s(n) = a_s(m), and
//   N = |G|^2 a_s d a_s / dG = |G| a_s (da/dm - m (m . da/dm)),
// which is Eq. (TermesAnisotropes) in lattice units (N_lu = dx N).
// ---------------------------------------------------------------------------
template <class R> __device__ __forceinline__ R rsqrt_r(R x);
template <> __device__ __forceinline__ float rsqrt_r<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_r<double>(double x) { return 1.0 / sqrt(x); }

// Zero-gradient guard: below |G| = 1e-10 (FP64) or 1e-6 (FP32) lattice units
// the direction of G is undefined or set by rounding noise (e.g. at symmetry
// centres); there a_s = 1 and N = 0.
template <class R> __device__ __forceinline__ R guard2();
template <> __device__ __forceinline__ double guard2<double>() { return 1e-20; }
template <> __device__ __forceinline__ float guard2<float>() { return 1e-12f; }

template <class R, int D>
__device__ __forceinline__ void anisotropy(const CrystalDev& c, R Gx, R Gy, R Gz, R& a, R& Nx, R& Ny, R& Nz)
{
    const R g2 = Gx * Gx + Gy * Gy + (D == 3 ? Gz * Gz : R(0));
    Nx = Ny = Nz = R(0);
    a = R(1);
    if (!(g2 > guard2<R>())) return;
    const R eps = R(c.eps), gam = R(c.gamma);
    if (c.kind == LBPF_AS_ANGLE) {
        // Eq. (As_Theta), varphi = atan2(n_y, n_x) with n = -G/|G|;
        // N = a a'(varphi) (-G_y, G_x).
        const R vphi = atan2(-Gy, -Gx);
        R sn, cs;
        sincos(R(c.q) * (vphi - R(c.phi0)), &sn, &cs);
        a = R(1) + eps * cs;
        const R ap = -eps * R(c.q) * sn;
        Nx = -a * ap * Gy;
        Ny = a * ap * Gx;
        return;
    }
    const R rg = rsqrt_r<R>(g2);
    const R mx = Gx * rg, my = Gy * rg, mz = (D == 3) ? Gz * rg : R(0);
    const R x2 = mx * mx, y2 = my * my, z2 = mz * mz;
    R dx_ = 0, dy_ = 0, dz_ = 0;
    switch (c.kind) {
    case LBPF_AS_CUBIC100: {  // Eq. (As_Function_Classical)
        const R Q4 = x2 * x2 + y2 * y2 + z2 * z2;
        a = R(1) - R(3) * eps + R(4) * eps * Q4;
        const R k = R(16) * eps;
        dx_ = k * x2 * mx; dy_ = k * y2 * my; dz_ = k * z2 * mz;
        break;
    }
    case LBPF_AS_Y66: {  // Eq. (As_Y66)
        a = R(1) + eps * (x2 * x2 * x2 - R(15) * x2 * x2 * y2 + R(15) * x2 * y2 * y2 - y2 * y2 * y2);
        dx_ = eps * mx * (R(6) * x2 * x2 - R(60) * x2 * y2 + R(30) * y2 * y2);
        dy_ = eps * my * (R(-30) * x2 * x2 + R(60) * x2 * y2 - R(6) * y2 * y2);
        break;
    }
    case LBPF_AS_HOYT110: {  // Eq. (As_MatSci)
        const R Q4 = x2 * x2 + y2 * y2 + z2 * z2;
        const R S = x2 * y2 * z2;
        a = R(1) + eps * (Q4 - R(0.6)) + gam * (R(3) * Q4 + R(66) * S - R(17.0 / 7.0));
        const R k3 = R(4) * eps + R(12) * gam, k6 = R(132) * gam;
        dx_ = mx * (k3 * x2 + k6 * y2 * z2);
        dy_ = my * (k3 * y2 + k6 * x2 * z2);
        dz_ = mz * (k3 * z2 + k6 * x2 * y2);
        break;
    }
    case LBPF_AS_S111: {  // Eq. (As_Function_S) with the constant term 1
        a = R(1) + R(66) * gam * (x2 * y2 * z2);
        const R k6 = R(132) * gam;
        dx_ = mx * k6 * y2 * z2;
        dy_ = my * k6 * x2 * z2;
        dz_ = mz * k6 * x2 * y2;
        break;
    }
    default:
        return;
    }
    const R md = mx * dx_ + my * dy_ + mz * dz_;
    const R ga = g2 * rg * a;  // |G| a_s
    Nx = ga * (dx_ - mx * md);
    Ny = ga * (dy_ - my * md);
    Nz = (D == 3) ? ga * (dz_ - mz * md) : R(0);
}

// ---------------------------------------------------------------------------
// Launchers exported by the per-lattice translation units.
// ---------------------------------------------------------------------------
constexpr int kStepWalls = 1, kStepAdvect = 2;

struct Launchers {
    // Fused step over all work items, tile variant v (rows kTileRows[v]).
    // kind: 0 periodic domains only; kStepWalls: some domain has zero-flux
    // walls; kStepAdvect: some domain has an advective heat equilibrium (full
    // storage only; the kernel also handles walls).  Kinds other than 0 are
    // built for variant 0 only.
    cudaError_t (*step)(int v, int kind, const StepArgs& a, int n_blocks, cudaStream_t s);
    // Dynamic shared memory of variant v.
    size_t (*step_smem)(int v);
    // Opt variant v (every kind built for it) into its dynamic shared memory.
    cudaError_t (*prepare)(int v);
    // Resident blocks per SM of variant v and step kind.
    int (*blocks_per_sm)(int v, int kind);
    // Staged step kernel (staged_kernel.cuh; tile 32 x 8 of variant 0), or
    // nullptr where it is not built (2D, full storage, D3Q27).
    cudaError_t (*step_staged)(const StepArgs& a, int n_blocks, cudaStream_t s);
    int (*staged_blocks_per_sm)();
    // Heat step alone, lagged -> synced state of one domain (f^{n-1}, aux^{n-1},
    // phi^n -> f^n [+ aux^n]).
    cudaError_t (*heat_sync)(const DomainDev* d, int cur, int fcur, int acur, cudaStream_t s);
    // Populations at equilibrium from the phi field in phi[cur] and u in
    // aux[acur] (index in I[cur]); writes g[cur], f[fcur] (+ aux in place).
    cudaError_t (*equilibrate)(const DomainDev* d, int cur, int fcur, int acur, int grad, int finalize_index,
                               cudaStream_t s);
    // u of a synced state into out (arithmetic type).
    cudaError_t (*read_u)(const DomainDev* d, int cur, int fcur, int acur, void* out, cudaStream_t s);
    // Decoded population i (which = 0: g_i, 1: f_i) of a synced state into out.
    cudaError_t (*read_pop)(const DomainDev* d, int which, int i, int cur, int fcur, int acur, void* out,
                            cudaStream_t s);
    // a_s(n) at every site from phi[cur] and the index field I[cur] (1 where
    // |grad phi| is below the zero-gradient guard or the index is 0).
    cudaError_t (*read_as)(const DomainDev* d, int cur, int grad, void* out, cudaStream_t s);
    int Qphi, Qu, D;
};

// Launchers of a lattice pair (lbpf_lattice) and precision (lbpf_precision),
// nullptr for an unknown pair or precision (lbpf_launchers.cu).
const Launchers* launchers_for_pair(int lattice, int precision);

// Precision-generic kernels (seeding, measurements, index copies), in lbpf_fields.cu.
// Seeds: n_seeds rows (x, y, z, R, crystal) in device memory.  Writes phi[cur],
// aux[acur] = u0 and the preliminary index (dominant seed) in I[cur].
cudaError_t launch_seed(const DomainDev* d, long long n, int cur, int acur, int precision, const double* seeds,
                        int n_seeds, int dim, double dx_over_W0, double u0, cudaStream_t s);
// Sums for the measurements: out[0] = sum (1+phi)/2, out[1] = sum (u - phi/2),
// out[2] = number of non-finite phi or u values; partial[] holds one pair of
// FP64 partial sums and a count per block (scratch of 3 * kReduceBlocks).
constexpr int kReduceBlocks = 304;
// With walls (bc != 0) the u - phi/2 sum weights nodes on a wall by 1/2 per
// walled coordinate (they lie on the mirror planes).
cudaError_t launch_reduce(const void* phi, const void* u, long long n, int precision, double* partial, double* out,
                          cudaStream_t s, int nx = 0, int ny = 0, int nz = 0, int bc = 0, int dim = 3);
// Tip crossings along +-x, +-y, +-z from (cx, cy, cz); out[6].  Rays cover
// half the domain on periodic axes and run to the wall on walled ones.
cudaError_t launch_tips(const void* phi, int nx, int ny, int nz, int cx, int cy, int cz, int dim, int precision,
                        double* out, cudaStream_t s, int bc = 0);
// Measurement history (time, tip6) per domain and the FP64 tip fits.
cudaError_t launch_hist_append(const double* tips6, double t, double* slot, cudaStream_t s);
cudaError_t launch_tip_velocity(const double* hist, int cap, int last, int count, int window, double dx, double* out,
                                cudaStream_t s);
// Tip radius of the tip along dir (0..5) from rays at transverse offsets
// |j| <= J (J <= 7 in 3D, <= 15 in 2D); out[0].
cudaError_t launch_tip_radius(const void* phi, int nx, int ny, int nz, int cx, int cy, int cz, int dir, int J, int dim,
                              int precision, double* out, cudaStream_t s, int bc = 0);
// int8 <-> int32 index copies.
cudaError_t launch_index_to_i32(const int8_t* in, int* out, long long n, cudaStream_t s);
cudaError_t launch_index_from_i32(const int* in, int8_t* out, long long n, int n_crystals, cudaStream_t s);
cudaError_t launch_fill_i8(int8_t* out, int8_t v, long long n, cudaStream_t s);
cudaError_t launch_fill_i32(int* out, int v, long long n, cudaStream_t s);

}  // namespace lbpf
