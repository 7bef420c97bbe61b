// Fused time step for 3D domains with 16-bit deviation storage, with every
// population, phi and aux value the step reads staged in shared memory by
// bulk asynchronous copies (cp.async.bulk, the untiled TMA path) that
// complete on mbarriers.  Same arithmetic, state and launch protocol as
// step_kernel (step_kernel.cuh): the phase-field scheme of Sec. 3.2 (Eq.
// LBE_Eq_Phase in pull form, divided by a_s^2) and the lagged heat scheme of
// Sec. 3.1, one launch per time step; only the data movement differs.
//
// Why: in step_kernel every population read is a global load whose 64-bit
// address (population array, plane, row, x shift, periodic wrap) is formed
// per load; with 16-bit storage that address arithmetic and the loads
// themselves bound the kernel by instruction issue, not by HBM.  Here rows
// are copied whole, and a population pull is a shared-memory load at a
// compile-time offset from the thread's position in the staged tile.
//
// Measured on GB300 (256^3 D3Q15 FP16 deviations): the staging costs about
// 440 thread-instructions a site of its own, the ~95 KB of shared memory a
// block allows 2 blocks (16 warps) per SM against 4 for step_kernel, and one
// bulk copy per row (~260 copies per block and plane) is limited by the
// SM's copy engine; 1.01 ms a step with 16-byte cp.async chunks, 1.12 ms with
// bulk copies, against 0.76 ms for step_kernel.  It is therefore opt-in
// (LBPF_KERNEL=staged); it gives the same results bit for bit.
//
// Staging, per thread block (tile of 32 x 8 sites of an xy-plane, marching
// along z over [z0, z1)):
//   g_i, i = 1..Q-1 (deviations): rows y0-1 .. y0+8, x0-8 .. x0+39 of plane
//     p, kept in a ring of 2 planes (e_i,z = 0) or 3 planes (e_i,z != 0);
//   f_j, j = 1..Q_u-1: rows y0-2 .. y0+9, same x range, rings of 2 or 3;
//   phi, aux: rows y0-2 .. y0+9, x0-4 .. x0+35 (as in step_kernel), rings
//     of 5 and 4 planes; h = aux + phi/2 is formed in place on arrival.
// Each row copy is 16-byte aligned (x0 a multiple of 32, nx a multiple of
// 8); a row crossing the periodic x edge is split in two copies.  Iteration
// z of the march issues the copies of one "stage" (g planes z+1 or z+2, f
// planes z+2 or z+3, phi/aux plane z+3, each the newest plane its ring
// needs) on one of two mbarriers, then computes the collision coefficients
// of plane z+1 and the output of plane z; iteration z+1 waits for that
// stage.  Every wait is bounded by a 2 s timer: on expiry the block records
// an error in counters[4], waits (bounded again) for its copies in flight
// and leaves the launch; the host reports LBPF_ETIMEOUT.
#pragma once

#include "step_kernel.cuh"

namespace lbpf {

template <class PL, class UL>
struct StagedGeom {
    static constexpr int TX = 32, TY = 8, NT = TX * TY;
    static constexpr int GX = 48;                  // staged 16-bit row: x0-8 .. x0+39
    static constexpr int GRY = TY + 2, FRY = TY + 4;
    static constexpr int GSL = GX * GRY, FSL = GX * FRY;  // elements per slot
    static constexpr int QG = PL::Q - 1, QU = UL::Q - 1;  // stored populations
    static constexpr int RX = TX + 8, RY = TY + 4, RP = RX * RY;  // phi/aux frame (x0-4, y0-2)
    static constexpr int CX = TX + 2, CY = TY + 2, CP = CX * CY;  // coefficient frame
    static constexpr int NPH = 5, NH = 4, NC = 3, NCO = 6;
    static constexpr int ROWS = 12;                 // rows per copy group (g groups use 10)
    // bit i set: population i moves along z (ring of 3 planes), resp. moves to -z
    static constexpr unsigned nz_mask(bool g)
    {
        unsigned m = 0;
        for (int i = 1; i < (g ? PL::Q : UL::Q); ++i)
            if ((g ? PL::ez(i) : UL::ez(i)) != 0) m |= 1u << i;
        return m;
    }
    static constexpr unsigned neg_mask(bool g)
    {
        unsigned m = 0;
        for (int i = 1; i < (g ? PL::Q : UL::Q); ++i)
            if ((g ? PL::ez(i) : UL::ez(i)) < 0) m |= 1u << i;
        return m;
    }
    static constexpr int slots(bool g)
    {
        int s = 0;
        for (int i = 1; i < (g ? PL::Q : UL::Q); ++i) s += ((g ? PL::ez(i) : UL::ez(i)) != 0) ? 3 : 2;
        return s;
    }
    // shared memory layout (bytes)
    static constexpr size_t G_BYTES = (size_t)slots(true) * GSL * 2;
    static constexpr size_t F_BYTES = (size_t)slots(false) * FSL * 2;
    static constexpr size_t OFF_F = G_BYTES;
    static constexpr size_t OFF_PHI = OFF_F + F_BYTES;
    static constexpr size_t OFF_H = OFF_PHI + (size_t)NPH * RP * 4;
    static constexpr size_t OFF_CO = OFF_H + (size_t)NH * RP * 4;
    static constexpr size_t OFF_MBAR = OFF_CO + (size_t)NC * NCO * CP * 4;
    static constexpr size_t BYTES = OFF_MBAR + 16;
    // first slot of population i (1-based) in its array, in elements
    LBPF_HD static constexpr int first_slot(int i, unsigned nzm, int sl)
    {
        int c = 0;
        for (int k = 1; k < i; ++k) c += (nzm >> k) & 1u;
        return (2 * (i - 1) + c) * sl;
    }
};

// How rows reach shared memory: 0 = one bulk copy (cp.async.bulk) per row,
// completing on the stage's mbarrier by transaction bytes; 1 = 16-byte
// cp.async chunks issued by the threads, each thread's copies signalling the
// stage's mbarrier through cp.async.mbarrier.arrive.
#ifndef LBPF_STAGED_COPY
#define LBPF_STAGED_COPY 1
#endif
constexpr int kStagedCopy = LBPF_STAGED_COPY;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

// Copy elements [xs, xs + len) of a periodic row of nx elements (row base
// `row`, element size E) to dst: one bulk copy, or two across the x edge; or
// 16-byte cp.async chunks (nx a multiple of 16 / E, so no chunk straddles
// the edge).
template <int E>
__device__ __forceinline__ void bulk_row(uint32_t dst, const char* row, int xs, int len, int nx, uint32_t mbar)
{
    if constexpr (kStagedCopy == 0) {
        const int x = xs < 0 ? xs + nx : xs;
        const int first = min(len, nx - x);
        bulk_g2s(dst, row + (size_t)x * E, (uint32_t)(first * E), mbar);
        if (first < len) bulk_g2s(dst + first * E, row, (uint32_t)((len - first) * E), mbar);
    } else {
        constexpr int EPC = 16 / E;
#pragma unroll 2
        for (int c = 0; c < len / EPC; ++c) {
            int x = xs + c * EPC;
            x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16 * c), "l"(row + (size_t)x * E)
                         : "memory");
        }
    }
}

// Bounded wait for phase `parity` of the mbarrier: true on completion, false
// after about two seconds.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        // the thread is suspended until the phase completes or about 1 ms
        // passes (no spinning)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity), "r"(1000000u)
            : "memory");
        if (done) return true;
        if ((it & 15u) == 0) {
            uint64_t t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (it == 0)
                t0 = t;
            else if (t - t0 > 2000000000ull)
                return false;
        }
    }
}

template <class PL, class UL, class S>
__device__ __forceinline__ void staged_item(const StepArgs& args, const WorkItem it, unsigned char* smem,
                                            uint32_t& stage, volatile int* s_abort)
{
    using G = StagedGeom<PL, UL>;
    using R = typename S::Real;
    using T = typename S::T;
    static_assert(S::dev && sizeof(T) == 2 && sizeof(R) == 4, "16-bit deviation storage only");
    constexpr int TX = G::TX, TY = G::TY, NT = G::NT, GX = G::GX, RX = G::RX, RP = G::RP, CX = G::CX, CP = G::CP;
    constexpr int QG = PL::Q, QU = UL::Q, NCO = G::NCO, ROWS = G::ROWS;
    constexpr unsigned GNZ = G::nz_mask(true), GNEG = G::neg_mask(true);
    constexpr unsigned FNZ = G::nz_mask(false), FNEG = G::neg_mask(false);
    constexpr bool SR = UsesSR<S>::value;

    T* s_g = reinterpret_cast<T*>(smem);
    T* s_f = reinterpret_cast<T*>(smem + G::OFF_F);
    R* s_phi = reinterpret_cast<R*>(smem + G::OFF_PHI);
    R* s_h = reinterpret_cast<R*>(smem + G::OFF_H);
    R* s_co = reinterpret_cast<R*>(smem + G::OFF_CO);
    const uint32_t mbar0 = smem_u32(smem + G::OFF_MBAR);

    const DomainDev& dm = args.doms[it.dom];
    const int nx = dm.nx, ny = dm.ny, nz = dm.nz;
    const long long n = dm.n;
    const long long nxy = (long long)nx * ny;
    const int x0 = it.x0, y0 = it.y0, z0 = it.z0, z1 = it.z1;
    const int tw = min(TX, nx - x0), th = min(TY, ny - y0);
    const int tid = threadIdx.x;
    const bool collide = args.collide != 0;

    const T* __restrict__ gc = static_cast<const T*>(dm.g[args.cur]);
    T* __restrict__ gn = static_cast<T*>(dm.g[args.cur ^ 1]);
    const R* __restrict__ phic = static_cast<const R*>(dm.phi[args.cur]);
    R* __restrict__ phin = static_cast<R*>(dm.phi[args.cur ^ 1]);
    const T* __restrict__ fc = static_cast<const T*>(dm.f[args.fcur]);
    T* __restrict__ fn = static_cast<T*>(dm.f[args.fcur ^ 1]);
    const R* __restrict__ auxc = static_cast<const R*>(dm.aux[args.acur]);
    R* __restrict__ auxn = static_cast<R*>(dm.aux[args.acur ^ 1]);

    const uint32_t seed = SR ? (uint32_t)args.counters[2 + args.cur] : 0u;
    (void)seed;
    auto store_dev = [&](T* p, R v, uint32_t h, uint32_t pop) {
        if constexpr (SR)
            *p = from_real_sr<T>(v, sr_bits(h, pop));
        else
            *p = from_real<T, R>(v);
    };
    const R De2 = R(dm.Dphi / PL::E2);
    const R qphi = R(dm.qphi);
    const R lam = R(dm.lambda);
    const R om_u = R(1) - R(dm.inv_eta_u);
    const CrystalDev cr = dm.cr[0];

    // periodic wrap of indices at most a few sites outside [0, n)
    auto wrapy = [&](int v) {
        while (v < 0) v += ny;
        while (v >= ny) v -= ny;
        return v;
    };
    auto wrapz = [&](int v) {
        while (v < 0) v += nz;
        while (v >= nz) v -= nz;
        return v;
    };
    auto sphi = [&](int zp) { return (zp + 10) % G::NPH; };
    auto sh = [&](int zp) { return (zp + 8) % G::NH; };
    auto sco = [&](int zp) { return (zp + 3) % G::NC; };
    auto ring = [](int p, int nsl) { return (p + 6) % nsl; };

    // ---- copies of one stage: groups of ROWS rows, one row per thread ----
    // group kinds: 0 = g, 1 = f, 2 = phi, 3 = aux; plane p (unwrapped z)
    // slot of plane p of population pop (runtime pop: popcount, no loop)
    auto slot_of = [&](unsigned nzm, int pop, int p, int sl) {
        const int first = 2 * (pop - 1) + __popc(nzm & ((1u << pop) - 1u));
        const int r = ((nzm >> pop) & 1) ? (p + 6) % 3 : (p & 1);
        return (first + r) * sl;
    };
    auto issue_row = [&](int kind, int pop, int p, int r, uint32_t mbar) {
        const long long zo = (long long)wrapz(p) * nxy;
        if (kind == 0) {
            if (r >= G::GRY) return;
            const int sl = slot_of(GNZ, pop, p, G::GSL);
            const char* row = reinterpret_cast<const char*>(gc + (long long)(pop - 1) * n + zo +
                                                            (long long)wrapy(y0 - 1 + r) * nx);
            bulk_row<2>(smem_u32(s_g + sl + r * GX), row, x0 - 8, GX, nx, mbar);
        } else if (kind == 1) {
            const int sl = slot_of(FNZ, pop, p, G::FSL);
            const char* row = reinterpret_cast<const char*>(fc + (long long)(pop - 1) * n + zo +
                                                            (long long)wrapy(y0 - 2 + r) * nx);
            bulk_row<2>(smem_u32(s_f + sl + r * GX), row, x0 - 8, GX, nx, mbar);
        } else {
            R* dst = (kind == 2 ? s_phi + sphi(p) * RP : s_h + sh(p) * RP) + r * RX;
            const R* src = (kind == 2 ? phic : auxc) + zo + (long long)wrapy(y0 - 2 + r) * nx;
            bulk_row<4>(smem_u32(dst), reinterpret_cast<const char*>(src), x0 - 4, RX, nx, mbar);
        }
    };
    constexpr uint32_t G_ROW = GX * 2, PH_ROW = RX * 4;
    constexpr uint32_t G_PLANE = G::GRY * G_ROW, F_PLANE = G::FRY * G_ROW, PH_PLANE = G::RY * PH_ROW;
    // stage kinds: 0 = first of a work item, 1 = second, 2 = steady (iteration z)
    constexpr int NGZ = G::slots(true) - 2 * (QG - 1), NFZ = G::slots(false) - 2 * (QU - 1);
    auto stage_groups = [&](int kind, int& ng, int& nf, int& nph) {
        ng = kind == 0 ? (QG - 1) + NGZ : (kind == 1 ? 0 : QG - 1);
        nf = !collide ? 0 : (kind == 0 ? 2 * (QU - 1) + NFZ : QU - 1);
        nph = kind == 0 ? 4 : 1;
    };
    // arm the mbarrier of the next stage with its byte count (thread 0; a
    // barrier separates this from the copies)
    auto arm_stage = [&](int kind) {
        if (kStagedCopy != 0 || tid != 0) return;
        int ng, nf, nph;
        stage_groups(kind, ng, nf, nph);
        const uint32_t bytes = ng * G_PLANE + nf * F_PLANE + 2 * nph * PH_PLANE;
        const uint32_t mbar = mbar0 + 8u * (stage & 1u);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
    };
    auto issue_stage = [&](int kind, int z) {
        const uint32_t mbar = mbar0 + 8u * (stage & 1u);
        int ng, nf, nph;
        stage_groups(kind, ng, nf, nph);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier accesses before the copies
        const int groups = ng + nf + 2 * nph;
        for (int t = tid; t < groups * ROWS; t += NT) {
            const int gi = t / ROWS, r = t - gi * ROWS;
            int knd, pop = 0, p;
            if (gi < ng) {
                knd = 0;
                if (kind == 2) {
                    pop = gi + 1;
                    p = ((GNEG >> pop) & 1) ? z + 2 : z + 1;
                } else if (gi < QG - 1) {  // first stage: local plane z0 of every population
                    pop = gi + 1;
                    p = z;
                } else {  // and the pull plane of those that move along z
                    pop = __fns(GNZ, 0, gi - (QG - 1) + 1);
                    p = ((GNEG >> pop) & 1) ? z + 1 : z - 1;
                }
            } else if (gi < ng + nf) {
                knd = 1;
                const int fi = gi - ng;
                if (kind != 0) {
                    pop = fi + 1;
                    const int base = kind == 1 ? z + 1 : z + 2;
                    p = ((FNEG >> pop) & 1) ? base + 1 : base;
                } else if (fi < 2 * (QU - 1)) {  // planes z0-1 and z0 of every population
                    pop = fi % (QU - 1) + 1;
                    p = z - 1 + fi / (QU - 1);
                } else {  // and z0-2 (moving to +z) or z0+1 (moving to -z)
                    pop = __fns(FNZ, 0, fi - 2 * (QU - 1) + 1);
                    p = ((FNEG >> pop) & 1) ? z + 1 : z - 2;
                }
            } else {
                const int pi = gi - ng - nf;
                knd = 2 + (pi & 1);
                p = kind == 0 ? z - 2 + (pi >> 1) : (kind == 1 ? z + 2 : z + 3);
            }
            issue_row(knd, pop, p, r, mbar);
        }
        if constexpr (kStagedCopy != 0)  // arrives when this thread's copies have landed
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(mbar) : "memory");
        stage += 1;
    };
    // bounded wait for stage k; on expiry the block records the error and
    // stops after the next barrier
    auto wait_stage = [&](uint32_t k) {
        const uint32_t mbar = mbar0 + 8u * (k & 1u);
        if (!mbar_wait(mbar, (k >> 1) & 1u)) {
            *s_abort = 1;
            atomicExch(args.counters + 4, 1);
            mbar_wait(mbar, (k >> 1) & 1u);  // bounded: let copies in flight land
        }
    };
    // h = aux + phi/2 in place on plane zp (after its copies have landed)
    auto form_h = [&](int zp) {
        const R* dphi = s_phi + sphi(zp) * RP;
        R* dh = s_h + sh(zp) * RP;
        for (int k = tid; k < RP; k += NT) dh[k] += R(0.5) * dphi[k];
    };

    // ---- coefficients (and the lagged heat update) on plane c -------------
    auto coef_plane = [&](int c, bool store) {
        const int cw = wrapz(c);
        const long long zo = (long long)cw * nxy;
        R* dco = s_co + sco(c) * NCO * CP;
        const int rows = th + 2;
        const T* fl[QU];  // local plane c of each f population; pulls at plane c - e_z
        const T* fp[QU];
#pragma unroll
        for (int j = 1; j < QU; ++j) {
            const int nsl = UL::ez(j) != 0 ? 3 : 2;
            const int f0 = G::first_slot(j, FNZ, G::FSL);
            fl[j] = s_f + f0 + ring(c, nsl) * G::FSL;
            fp[j] = s_f + f0 + ring(c - UL::ez(j), nsl) * G::FSL;
        }
        for (int k = tid; k < CX * rows; k += NT) {
            const int ly = k / CX, lx = k - ly * CX;
            if (lx >= tw + 2) continue;
            const int px = lx + 3, py = ly + 1;                 // phi frame (x0-4, y0-2)
            const int ft = (ly + 1) * GX + lx + 7;              // f frame (x0-8, y0-2)
            const bool inner = store && lx >= 1 && lx <= tw && ly >= 1 && ly <= th;
            const R ph = s_phi[sphi(c) * RP + py * RX + px];
            long long s = 0;
            if (inner) s = zo + (long long)(y0 + ly - 1) * nx + (x0 + lx - 1);

            R u = 0;
            if (collide) {
                R fv[QU];
                R d0 = 0;
#pragma unroll
                for (int j = 1; j < QU; ++j) d0 -= to_real(fl[j][ft]);
#pragma unroll
                for (int j = 0; j < QU; ++j) {
                    const int ex = UL::ex(j), ey = UL::ey(j), ez = UL::ez(j);
                    const R hs = s_h[sh(c - ez) * RP + (py - ey) * RX + (px - ex)];
                    const R dj = (j == 0) ? d0 : to_real(fp[j][ft - ey * GX - ex]);
                    const R fj = R(UL::w(j)) * hs + om_u * dj;
                    fv[j] = fj;
                    u += fj;
                }
                if (inner) {
                    const uint32_t h = SR ? sr_hash((uint32_t)s, seed) : 0u;
#pragma unroll
                    for (int j = 1; j < QU; ++j)
                        store_dev(&fn[(long long)(j - 1) * n + s], fv[j] - R(UL::w(j)) * u, h, 32u + j);
                }
            } else {
                u = s_h[sh(c) * RP + py * RX + px];  // C^n + phi^n / 2
            }
            if (inner) auxn[s] = u - R(0.5) * ph;

            // gradient of phi^n (Sec. 4.2)
            R Gx = 0, Gy = 0, Gz = 0;
            if (args.grad == LBPF_GRAD_DD) {
#pragma unroll
                for (int i = 1; i < QG; ++i) {
                    if (i > opposite<PL>(i)) continue;
                    const int ex = PL::ex(i), ey = PL::ey(i), ez = PL::ez(i);
                    const R dd = s_phi[sphi(c + ez) * RP + (py + ey) * RX + (px + ex)] -
                                 s_phi[sphi(c - ez) * RP + (py - ey) * RX + (px - ex)];
                    const R wd = R(PL::w(i)) * dd;
                    if (ex) Gx += R(ex) * wd;
                    if (ey) Gy += R(ey) * wd;
                    if (ez) Gz += R(ez) * wd;
                }
                const R kk = R(1.0 / PL::E2);
                Gx *= kk;
                Gy *= kk;
                Gz *= kk;
            } else {
                const R* pl = s_phi + sphi(c) * RP;
                Gx = R(0.5) * (pl[py * RX + px + 1] - pl[py * RX + px - 1]);
                Gy = R(0.5) * (pl[(py + 1) * RX + px] - pl[(py - 1) * RX + px]);
                Gz = R(0.5) * (s_phi[sphi(c + 1) * RP + py * RX + px] - s_phi[sphi(c - 1) * RP + py * RX + px]);
            }
            R a, Nx, Ny, Nz;
            anisotropy<R, 3>(cr, Gx, Gy, Gz, a, Nx, Ny, Nz);
            const R A2 = a * a;
            const R iA2 = recip<R>(A2);
            const R ieta = recip<R>(A2 * De2 + R(0.5));
            const R omp = (R(1) - ph) * (R(1) + ph);
            const R Qphi = (ph - lam * u * omp) * omp;
            const R vf = -De2 * ieta * iA2;
            // deviation storage: the source coefficient carries c1 phi(x), see step_kernel
            const R sc = (ph + qphi * Qphi) * iA2;
            CoefIO<R>::store(dco, CP, ly * CX + lx, (R(1) - ieta) * iA2, iA2 - R(1), sc, vf * Nx, vf * Ny, vf * Nz);
        }
    };

    // ---- phase-field collision + streaming of plane z ----------------------
    auto output_plane = [&](int z) {
        const int ltx = tid % TX, lty = tid / TX;
        if (ltx >= tw || lty >= th) return;
        const long long s = (long long)wrapz(z) * nxy + (long long)(y0 + lty) * nx + (x0 + ltx);
        const int gt = (lty + 1) * GX + ltx + 8;  // g frame (x0-8, y0-1)
        const int cx = ltx + 1, cy = lty + 1;
        const R phy = s_phi[sphi(z) * RP + (lty + 2) * RX + ltx + 4];
        // directions 1 .. Q-1, then the rest population (as in step_kernel)
        R gnew[QG];
        R phinew = 0, d0 = 0;
#pragma unroll
        for (int k = 0; k < QG; ++k) {
            const int i = (k + 1) % QG;
            const int ex = PL::ex(i), ey = PL::ey(i), ez = PL::ez(i);
            R c1, c2, cs, vx, vy, vz;
            CoefIO<R>::load(s_co + sco(z - ez) * NCO * CP, CP, (cy - ey) * CX + (cx - ex), ey != 0 || ez != 0, c1, c2,
                            cs, vx, vy, vz);
            R gl, gp;
            if (i > 0) {
                const int nsl = ez != 0 ? 3 : 2;
                const int f0 = G::first_slot(i, GNZ, G::GSL);
                const R d = to_real(s_g[f0 + ring(z, nsl) * G::GSL + gt]);
                d0 = sub_rn(d0, d);
                gl = fma_rn(R(PL::w(i)), phy, d);
                gp = to_real(s_g[f0 + ring(z - ez, nsl) * G::GSL + gt - ey * GX - ex]);
            } else {
                gl = fma_rn(R(PL::w(0)), phy, d0);
                gp = d0;
            }
            const R v = pull_new<R>(ex, ey, ez, R(PL::w(i)), c1, c2, cs, vx, vy, vz, gp, gl);
            gnew[i] = v;
            phinew = add_rn(phinew, v);
        }
        phin[s] = phinew;
        const uint32_t h = SR ? sr_hash((uint32_t)s, seed) : 0u;
#pragma unroll
        for (int i = 1; i < QG; ++i)
            store_dev(&gn[(long long)(i - 1) * n + s], fma_rn(-R(PL::w(i)), phinew, gnew[i]), h, (uint32_t)i);
    };

    // ---- the march ---------------------------------------------------------
    arm_stage(0);
    __syncthreads();
    uint32_t k = stage;
    issue_stage(0, z0);
    wait_stage(k);
    for (int p = z0 - 2; p <= z0 + 1; ++p) form_h(p);
    __syncthreads();
    if (*s_abort) return;
    coef_plane(z0 - 1, false);
    coef_plane(z0, true);
    arm_stage(1);
    __syncthreads();
    k = stage;
    issue_stage(1, z0);
    for (int z = z0; z < z1; ++z) {
        wait_stage(k);
        form_h(z + 2);
        const bool more = z <= z1 - 2;
        if (more) arm_stage(2);
        __syncthreads();
        if (*s_abort) return;
        if (more) {
            k = stage;
            issue_stage(2, z);
        }
        coef_plane(z + 1, z + 1 < z1);
        __syncthreads();
        output_plane(z);
        // no barrier: the next writes (h of plane z+3, formed in a slot no one
        // reads now; copies issued after the next barrier) touch nothing that
        // output_plane(z) reads
    }
}

// Persistent launch with the dynamic work list of step_kernel.
template <class PL, class UL, class S>
__global__ void __launch_bounds__(256, 2) step_kernel_staged(const StepArgs args)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_next;
    __shared__ int s_abort;
    using G = StagedGeom<PL, UL>;
    int* counter = args.counters + args.cur;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        args.counters[args.cur ^ 1] = 0;
        if constexpr (UsesSR<S>::value) args.counters[2 + (args.cur ^ 1)] = args.counters[2 + args.cur] + 1;
    }
    if (threadIdx.x == 0) {
        const uint32_t mb = smem_u32(smem_raw + G::OFF_MBAR);
        // bulk copies: one arrival (thread 0's expect_tx) per phase; cp.async:
        // one arrival per thread
        const uint32_t cnt = kStagedCopy == 0 ? 1u : 256u;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(cnt) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb + 8), "r"(cnt) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    __syncthreads();
    uint32_t stage = 0;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(counter, 1);
        __syncthreads();
        const int k = s_next;
        if (k >= args.n_items || s_abort) break;
        staged_item<PL, UL, S>(args, args.items[k], smem_raw, stage, &s_abort);
        __syncthreads();
    }
}

template <class PL, class UL, class S>
constexpr size_t staged_smem_bytes()
{
    return StagedGeom<PL, UL>::BYTES;
}

}  // namespace lbpf
