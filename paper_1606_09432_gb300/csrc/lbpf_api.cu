// Host side of the lbpf C ABI: context, device buffers, launches and the
// lagged/synchronised state of the heat populations.  See include/lbpf.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include <sys/stat.h>
#include <vector>

#include "lbpf_internal.cuh"

using namespace lbpf;

namespace {

thread_local std::string t_err;

// Planes per z-segment of a work item of the step kernel.
// (0: chosen from the work size and the resident block count.)
#ifndef LBPF_SEGMENT
#define LBPF_SEGMENT 0
#endif

constexpr int kHistCap = 64;

// a2 of the thin-interface relations, Eq. (Kinetic-Coeff); lambda* cancels beta.
constexpr double kA2 = 0.6267;

}  // namespace

struct lbpf_ctx {
    int lattice = 0, grad = 0, precision = 0, dim = 2;
    int Qg = 0, Qu = 0, Sg = 0, Su = 0;
    size_t rsize = 8, ssize = 8;
    int n_domains = 0;
    std::vector<lbpf_domain> in;
    std::vector<DomainDev> dd;
    DomainDev* d_dd = nullptr;
    WorkItem* d_items = nullptr;
    int* d_counters = nullptr;
    int n_items = 0, n_blocks = 0, items_cap = 0;
    int tile_v = 0, seg_len = 0, sms = 1;
    bool staged = false;  // step kernel with bulk-copy staging (staged_kernel.cuh)
    int kind = 0;         // step kernel kind: kStepWalls (some domain has walls) | kStepAdvect
    // graphs of kGraphSteps steady-state launches, keyed by (cur, fcur, acur)
    cudaGraphExec_t graphs[8] = {};
    bool graphs_off = false;
    std::string tuned;  // how the schedule was chosen
    bool tune_pending = false;  // time the schedules at the first step (on the seeded state)
    // measurement history: per domain a ring of kHistCap entries (t, tip6)
    double* d_hist = nullptr;
    std::vector<int> hist_count, hist_last;
    cudaStream_t stream = nullptr;
    int device = 0;
    const Launchers* L = nullptr;
    size_t smem = 0;
    int cur = 0, fcur = 0, acur = 0, lagged = 0;
    long long steps = 0, kernels = 0;
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    double* red = nullptr;
    double* d_seeds = nullptr;
    int seeds_cap = 0;
    size_t dev_bytes = 0;
    std::vector<void*> allocs;
    std::string err;
};

static int fail(lbpf_ctx* c, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        t_err = buf;
    return code;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(c, LBPF_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static int dev_alloc(lbpf_ctx* c, void** p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(c, e == cudaErrorMemoryAllocation ? LBPF_ENOMEM : LBPF_ECUDA, "cudaMalloc(%zu bytes): %s", bytes,
                    cudaGetErrorString(e));
    }
    c->allocs.push_back(*p);
    c->dev_bytes += bytes;
    return LBPF_OK;
}

static const Launchers* pick(int lattice, int precision) { return launchers_for_pair(lattice, precision); }

static bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

static void free_all(lbpf_ctx* c)
{
    for (void* p : c->allocs) cudaFree(p);
    c->allocs.clear();
}


// ---------------------------------------------------------------------------
// Work schedule of the step kernel.  Items are columns of tile_x x tile_y
// sites over segments of the marched axis (z in 3D, y in 2D), listed segment
// by segment; the kernel runs as many blocks as fit on the GPU and takes items
// in order (see step_kernel).
// ---------------------------------------------------------------------------
static long long column_units(const lbpf_ctx* c, int v)
{
    const int tx = tile_x(c->dim, v), ty = tile_y(c->dim, v);
    long long units = 0;
    for (const DomainDev& d : c->dd) {
        const int ny = c->dim == 3 ? d.ny : 1, nz = c->dim == 3 ? d.nz : d.ny;
        units += (long long)((d.nx + tx - 1) / tx) * ((ny + ty - 1) / ty) * nz;
    }
    return units;
}

static int blocks_per_sm(const lbpf_ctx* c, int v)
{
    return c->staged ? c->L->staged_blocks_per_sm() : c->L->blocks_per_sm(v, c->kind);
}

// Segment length balancing the per-item prologue (two extra planes) against
// the tail of the dynamic schedule: L ~ sqrt(5 units / resident blocks).
static int default_segment(const lbpf_ctx* c, int v)
{
    if (LBPF_SEGMENT > 0) return LBPF_SEGMENT;
    const double G = (double)blocks_per_sm(c, v) * c->sms;
    int L = (int)std::lround(std::sqrt(5.0 * (double)column_units(c, v) / G));
    return L < 8 ? 8 : (L > 256 ? 256 : L);
}

static int set_schedule(lbpf_ctx* c, int v, int seg)
{
    const int wx = tile_x(c->dim, v), wy = tile_y(c->dim, v);
    std::vector<WorkItem> items;
    for (int k = 0; k < c->n_domains; ++k) {
        const DomainDev& d = c->dd[k];
        // 2D: the kernel marches the y axis (its z) with one-row tiles
        const int ny = c->dim == 3 ? d.ny : 1, nz = c->dim == 3 ? d.nz : d.ny;
        const int tx = (d.nx + wx - 1) / wx, tyn = (ny + wy - 1) / wy;
        const int nseg = (nz + seg - 1) / seg;
        for (int sg = 0; sg < nseg; ++sg) {
            const int z0 = (int)((long long)sg * nz / nseg), z1 = (int)((long long)(sg + 1) * nz / nseg);
            for (int by = 0; by < tyn; ++by)
                for (int bx = 0; bx < tx; ++bx) {
                    WorkItem w;
                    w.dom = k;
                    w.x0 = bx * wx;
                    w.y0 = by * wy;
                    w.z0 = z0;
                    w.z1 = z1;
                    w.pad = 0;
                    items.push_back(w);
                }
        }
    }
    if ((int)items.size() > c->items_cap) {
        int rc;
        void* p = nullptr;
        if ((rc = dev_alloc(c, &p, sizeof(WorkItem) * items.size()))) return rc;
        c->d_items = static_cast<WorkItem*>(p);  // the old table stays in the context's allocation list
        c->items_cap = (int)items.size();
    }
    CK(cudaMemcpyAsync(c->d_items, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->n_items = (int)items.size();
    long long G = (long long)blocks_per_sm(c, v) * c->sms;
    c->n_blocks = (int)(G < c->n_items ? G : c->n_items);
    c->tile_v = v;
    c->seg_len = seg;
    for (cudaGraphExec_t& g : c->graphs)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    return LBPF_OK;
}

static std::string tune_key(const lbpf_ctx* c)
{
    char buf[160];
    // FNV-1a over the domain sizes and the build time of this library, so
    // that a rebuilt kernel is timed again instead of taking a stale choice
    unsigned long long h = 1469598103934665603ULL;
    for (const DomainDev& d : c->dd)
        for (int v : {d.nx, d.ny, d.nz, d.use_index}) {
            h ^= (unsigned long long)(unsigned)v;
            h *= 1099511628211ULL;
        }
    for (const char* p = __DATE__ " " __TIME__; *p; ++p) {
        h ^= (unsigned char)*p;
        h *= 1099511628211ULL;
    }
    snprintf(buf, sizeof(buf), "s2-lat%d-prec%d-grad%d-dom%d-%016llx-sm%d-k%d", c->lattice, c->precision, c->grad,
             c->n_domains, h, c->sms, (c->staged ? 1 : 0) | (c->kind << 1));
    return buf;
}

static std::string tune_cache_path()
{
    const char* p = getenv("LBPF_TUNE_CACHE");
    if (p) return p;
    const char* home = getenv("HOME");
    return std::string(home ? home : "/tmp") + "/.cache/lbpf_tune.txt";
}

// Time a few launches of the current schedule on the live state.  Every trial
// reads the current buffers (cur, fcur, acur) and writes the other ones,
// which the next real step overwrites, so the state is left as it was.
static double time_schedule(lbpf_ctx* c, int launches)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return 1e30;
    }
    StepArgs a;
    a.doms = c->d_dd;
    a.items = c->d_items;
    a.n_items = c->n_items;
    a.counters = c->d_counters;
    a.cur = c->cur;
    a.fcur = c->fcur;
    a.acur = c->acur;
    a.collide = 1;
    a.grad = c->grad;
    double best = 1e30;
    for (int k = 0; k < launches + 2; ++k) {
        if (cudaMemsetAsync(c->d_counters + c->cur, 0, sizeof(int), c->stream) != cudaSuccess) break;
        cudaEventRecord(e0, c->stream);
        if ((c->staged ? c->L->step_staged(a, c->n_blocks, c->stream)
                       : c->L->step(c->tile_v, c->kind, a, c->n_blocks, c->stream)) != cudaSuccess)
            break;
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (k >= 2 && ms < best) best = ms;
    }
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

// Schedule at context creation: a cached choice for this configuration, else
// the rule (tile variant 0, default segment); large configurations (or
// LBPF_AUTOTUNE=1) are then timed at the first step, on the seeded state.
static int initial_schedule(lbpf_ctx* c)
{
    const std::string key = tune_key(c);
    if (FILE* f = fopen(tune_cache_path().c_str(), "r")) {
        char k[200];
        int v, seg;
        while (fscanf(f, "%199s %d %d", k, &v, &seg) == 3)
            if (key == k && v >= 0 && v < (c->staged || c->kind ? 1 : kNumTileVariants) && seg >= 1) {
                fclose(f);
                c->tuned = "cache";
                return set_schedule(c, v, seg);
            }
        fclose(f);
    }
    double sites = 0;
    for (const DomainDev& d : c->dd) sites += (double)d.n;
    const char* env = getenv("LBPF_AUTOTUNE");
    c->tune_pending = env ? atoi(env) != 0 : sites >= 4e6;
    c->tuned = "rule";
    return set_schedule(c, 0, default_segment(c, 0));
}

// Time tile variants x segments {L, L/2, 2L} and keep (and cache) the
// fastest, but leave the rule's schedule (variant 0, segment L) only for one
// at least 3 % faster: short trials at the first step are noisy, and a
// wrong switch has cost up to 10 % in steady state.
static int autotune(lbpf_ctx* c)
{
    CK(cudaStreamSynchronize(c->stream));
    double best_t = 1e30, rule_t = 1e30;
    int best_v = 0, best_seg = default_segment(c, 0);
    for (int v = 0; v < (c->staged || c->kind ? 1 : kNumTileVariants); ++v) {
        const int L0 = default_segment(c, v);
        const int segs[3] = {L0, L0 / 2 > 8 ? L0 / 2 : 8, L0 * 2};
        for (int j = 0; j < 3; ++j) {
            int rc = set_schedule(c, v, segs[j]);
            if (rc) return rc;
            const double t = time_schedule(c, 6);
            if (v == 0 && j == 0) rule_t = t;
            if (t < best_t) {
                best_t = t;
                best_v = v;
                best_seg = segs[j];
            }
        }
    }
    if (!(best_t < 0.97 * rule_t)) {
        best_v = 0;
        best_seg = default_segment(c, 0);
    }
    CK(cudaMemsetAsync(c->d_counters, 0, sizeof(int) * 2, c->stream));
    c->tuned = "timed";
    const std::string path = tune_cache_path();
    const size_t slash = path.find_last_of('/');
    if (slash != std::string::npos && slash > 0) mkdir(path.substr(0, slash).c_str(), 0755);  // e.g. ~/.cache
    if (FILE* f = fopen(path.c_str(), "a")) {
        fprintf(f, "%s %d %d\n", tune_key(c).c_str(), best_v, best_seg);
        fclose(f);
    }
    return set_schedule(c, best_v, best_seg);
}

extern "C" int lbpf_create(const lbpf_domain* domains, int n_domains, int lattice, int grad, int precision,
                           void* stream, lbpf_ctx** out)
{
    lbpf_ctx* c = nullptr;
    if (!out) return fail(nullptr, LBPF_EINVAL, "lbpf_create: out is NULL");
    *out = nullptr;
    if (!domains || n_domains < 1) return fail(nullptr, LBPF_EINVAL, "lbpf_create: need at least one domain");
    if (grad != LBPF_GRAD_DD && grad != LBPF_GRAD_FD) return fail(nullptr, LBPF_EINVAL, "lbpf_create: bad grad %d", grad);
    const Launchers* L = pick(lattice, precision);
    if (!L) return fail(nullptr, LBPF_EINVAL, "lbpf_create: bad lattice %d or precision %d", lattice, precision);
    const int dim = L->D;
    for (int k = 0; k < n_domains; ++k) {
        const lbpf_domain& d = domains[k];
        if (d.nx < 2 || d.ny < 2 || (dim == 2 && d.nz != 1) || (dim == 3 && d.nz < 2))
            return fail(nullptr, LBPF_EINVAL, "domain %d: sizes %d x %d x %d invalid for a %dD lattice (each >= 2; nz = 1 in 2D)",
                        k, d.nx, d.ny, d.nz, dim);
        if (d.bc < 0 || d.bc > 7 || (dim == 2 && (d.bc & LBPF_BC_WALL_Z)) ||
            ((d.bc & LBPF_BC_WALL_X) && d.nx < 3) || ((d.bc & LBPF_BC_WALL_Y) && d.ny < 3) ||
            ((d.bc & LBPF_BC_WALL_Z) && d.nz < 3))
            return fail(nullptr, LBPF_EINVAL,
                        "domain %d: bc %d invalid (LBPF_BC_WALL_* bits, no z wall in 2D, >= 3 sites on a walled axis)",
                        k, d.bc);
        if ((long long)d.nx * d.ny > (1LL << 31) || (long long)d.nx * d.ny * d.nz > (1LL << 40))
            return fail(nullptr, LBPF_EINVAL, "domain %d: too many sites", k);
        if (!finite_pos(d.dx) || !finite_pos(d.dt) || !finite_pos(d.W0) || !finite_pos(d.tau0) || !finite_pos(d.kappa))
            return fail(nullptr, LBPF_EINVAL, "domain %d: dx, dt, W0, tau0, kappa must be finite and > 0", k);
        if (!std::isfinite(d.lambda) || !std::isfinite(d.delta) || !std::isfinite(d.xi) || d.xi < 0)
            return fail(nullptr, LBPF_EINVAL, "domain %d: lambda, delta, xi must be finite (xi >= 0)", k);
        if (!std::isfinite(d.adv[0]) || !std::isfinite(d.adv[1]) || !std::isfinite(d.adv[2]))
            return fail(nullptr, LBPF_EINVAL, "domain %d: adv must be finite", k);
        if (d.adv[0] != 0.0 || d.adv[1] != 0.0 || d.adv[2] != 0.0) {
            if (dim == 2 && d.adv[2] != 0.0)
                return fail(nullptr, LBPF_EINVAL, "domain %d: adv[2] must be 0 on a 2D lattice", k);
            if (((d.bc & LBPF_BC_WALL_X) && d.adv[0] != 0.0) || ((d.bc & LBPF_BC_WALL_Y) && d.adv[1] != 0.0) ||
                ((d.bc & LBPF_BC_WALL_Z) && d.adv[2] != 0.0))
                return fail(nullptr, LBPF_EINVAL, "domain %d: the velocity must be tangential to the walls", k);
        }
        if (d.n_crystals < 1 || d.n_crystals > LBPF_MAX_CRYSTALS)
            return fail(nullptr, LBPF_EINVAL, "domain %d: n_crystals %d not in 1..%d", k, d.n_crystals, LBPF_MAX_CRYSTALS);
        for (int j = 0; j < d.n_crystals; ++j) {
            const lbpf_crystal& cr = d.crystals[j];
            if (cr.kind < LBPF_AS_CUBIC100 || cr.kind > LBPF_AS_S111)
                return fail(nullptr, LBPF_EINVAL, "domain %d crystal %d: unknown anisotropy kind %d", k, j, cr.kind);
            if (cr.kind == LBPF_AS_ANGLE && (dim != 2 || cr.q < 1))
                return fail(nullptr, LBPF_EINVAL, "domain %d crystal %d: the angle form needs a 2D lattice and q >= 1", k, j);
            if (!std::isfinite(cr.eps) || !std::isfinite(cr.gamma) || !std::isfinite(cr.phi0))
                return fail(nullptr, LBPF_EINVAL, "domain %d crystal %d: non-finite parameter", k, j);
        }
    }

    c = new (std::nothrow) lbpf_ctx();
    if (!c) return fail(nullptr, LBPF_ENOMEM, "lbpf_create: out of host memory");
    c->lattice = lattice;
    c->grad = grad;
    c->precision = precision;
    c->dim = dim;
    c->L = L;
    c->Qg = L->Qphi;
    c->Qu = L->Qu;
    const bool dev = precision >= LBPF_FP32_FP16DEV;
    c->Sg = dev ? c->Qg - 1 : c->Qg;
    c->Su = dev ? c->Qu - 1 : c->Qu;
    c->rsize = precision == LBPF_FP64 ? 8 : 4;
    c->ssize = precision == LBPF_FP64 ? 8 : (precision == LBPF_FP32 ? 4 : 2);
    c->n_domains = n_domains;
    c->in.assign(domains, domains + n_domains);
    c->stream = static_cast<cudaStream_t>(stream);
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return fail(nullptr, LBPF_ECUDA, "lbpf_create: no CUDA device");
    }
    const double e2u = (dim == 2) ? 1.0 / 3.0 : 1.0 / 4.0;

    int rc = LBPF_OK;
    long long max_n = 0;
    c->dd.resize(n_domains);
    for (int k = 0; k < n_domains && rc == LBPF_OK; ++k) {
        const lbpf_domain& d = domains[k];
        DomainDev& h = c->dd[k];
        memset(&h, 0, sizeof(h));
        h.nx = d.nx;
        h.ny = d.ny;
        h.nz = d.nz;
        h.bc = d.bc;
        if (d.bc) c->kind |= kStepWalls;
        h.n = (long long)d.nx * d.ny * d.nz;
        max_n = h.n > max_n ? h.n : max_n;
        // D_phi = (W0^2/tau0)(dt/dx^2), Eq. (LBE_RelaxationTime)
        h.Dphi = (d.W0 * d.W0 / d.tau0) * (d.dt / (d.dx * d.dx));
        h.qphi = d.dt / d.tau0;
        h.lambda = d.lambda > 0.0 ? d.lambda : d.kappa * d.tau0 / (kA2 * d.W0 * d.W0);
        // kappa = e^2 (eta_u - 1/2) dx^2 / dt, Eq. (ThermalDiffusivity)
        h.inv_eta_u = 1.0 / (d.kappa * d.dt / (e2u * d.dx * d.dx) + 0.5);
        h.xi_lu = d.xi * d.dx;
        // advective heat equilibrium: a = v dt / (dx e^2)
        h.advect = d.adv[0] != 0.0 || d.adv[1] != 0.0 || d.adv[2] != 0.0;
        if (h.advect) c->kind |= kStepAdvect;
        for (int a = 0; a < 3; ++a) h.adv[a] = d.adv[a] * d.dt / (d.dx * e2u);
        h.n_crystals = d.n_crystals;
        h.use_index = d.n_crystals > 1;
        for (int j = 0; j < d.n_crystals; ++j) {
            h.cr[j].kind = d.crystals[j].kind;
            h.cr[j].q = d.crystals[j].q;
            h.cr[j].eps = d.crystals[j].eps;
            h.cr[j].gamma = d.crystals[j].gamma;
            h.cr[j].phi0 = d.crystals[j].phi0;
        }
        for (int b = 0; b < 2 && rc == LBPF_OK; ++b) {
            rc = dev_alloc(c, &h.g[b], (size_t)c->Sg * h.n * c->ssize);
            if (rc == LBPF_OK) rc = dev_alloc(c, &h.f[b], (size_t)c->Su * h.n * c->ssize);
            if (rc == LBPF_OK) rc = dev_alloc(c, &h.phi[b], (size_t)h.n * c->rsize);
            if (rc == LBPF_OK) rc = dev_alloc(c, &h.aux[b], (size_t)h.n * c->rsize);
            if (rc == LBPF_OK && h.use_index) rc = dev_alloc(c, reinterpret_cast<void**>(&h.I[b]), (size_t)h.n);
            if (rc == LBPF_OK && h.advect) rc = dev_alloc(c, &h.U[b], (size_t)h.n * c->rsize);
        }
        // zero state so that an unseeded domain holds finite values
        for (int b = 0; b < 2 && rc == LBPF_OK; ++b) {
            if (cudaMemsetAsync(h.g[b], 0, (size_t)c->Sg * h.n * c->ssize, c->stream) != cudaSuccess ||
                cudaMemsetAsync(h.f[b], 0, (size_t)c->Su * h.n * c->ssize, c->stream) != cudaSuccess ||
                cudaMemsetAsync(h.phi[b], 0, (size_t)h.n * c->rsize, c->stream) != cudaSuccess ||
                cudaMemsetAsync(h.aux[b], 0, (size_t)h.n * c->rsize, c->stream) != cudaSuccess ||
                (h.use_index && cudaMemsetAsync(h.I[b], 0, (size_t)h.n, c->stream) != cudaSuccess) ||
                (h.advect && cudaMemsetAsync(h.U[b], 0, (size_t)h.n * c->rsize, c->stream) != cudaSuccess))
                rc = fail(c, LBPF_ECUDA, "lbpf_create: cudaMemsetAsync failed");
        }
    }
    if (rc == LBPF_OK) {
        // the staged kernel (opt-in: it measured slower than the generic one,
        // see staged_kernel.cuh) needs 16-byte aligned row copies (nx a
        // multiple of 8), rows wider than the staged 48-site window, one crystal
        const char* kenv = getenv("LBPF_KERNEL");
        c->staged = L->step_staged != nullptr && kenv && strcmp(kenv, "staged") == 0;
        for (const DomainDev& h : c->dd)
            if (h.nx % 8 != 0 || h.nx < 64 || h.use_index || h.bc || h.advect) c->staged = false;
        if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || c->sms < 1)
            c->sms = 1;
        for (int v = 0; v < kNumTileVariants && rc == LBPF_OK; ++v) {
            cudaError_t e = L->prepare(v);
            if (e != cudaSuccess) rc = fail(c, LBPF_ECUDA, "lbpf_create: kernel attribute: %s", cudaGetErrorString(e));
        }
    }
    if (rc == LBPF_OK) rc = dev_alloc(c, reinterpret_cast<void**>(&c->d_counters), sizeof(int) * 8);
    if (rc == LBPF_OK && cudaMemsetAsync(c->d_counters, 0, sizeof(int) * 8, c->stream) != cudaSuccess)
        rc = fail(c, LBPF_ECUDA, "lbpf_create: cudaMemsetAsync failed");
    if (rc == LBPF_OK) rc = dev_alloc(c, reinterpret_cast<void**>(&c->d_dd), sizeof(DomainDev) * n_domains);
    if (rc == LBPF_OK) {
        c->scratch_bytes = (size_t)max_n * (c->rsize > 4 ? c->rsize : 4);
        rc = dev_alloc(c, &c->scratch, c->scratch_bytes);
    }
    if (rc == LBPF_OK) rc = dev_alloc(c, reinterpret_cast<void**>(&c->red), sizeof(double) * (3 * kReduceBlocks + 16));
    if (rc == LBPF_OK) {
        rc = dev_alloc(c, reinterpret_cast<void**>(&c->d_hist), sizeof(double) * 7 * kHistCap * n_domains);
        c->hist_count.assign(n_domains, 0);
        c->hist_last.assign(n_domains, kHistCap - 1);
    }
    if (rc == LBPF_OK) {
        if (cudaMemcpyAsync(c->d_dd, c->dd.data(), sizeof(DomainDev) * n_domains, cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess)
            rc = fail(c, LBPF_ECUDA, "lbpf_create: copying the domain table failed");
    }
    if (rc == LBPF_OK && cudaStreamSynchronize(c->stream) != cudaSuccess)
        rc = fail(c, LBPF_ECUDA, "lbpf_create: stream synchronisation failed");
    if (rc == LBPF_OK) rc = initial_schedule(c);
    if (rc != LBPF_OK) {
        t_err = c->err;
        free_all(c);
        delete c;
        return rc;
    }
    *out = c;
    return LBPF_OK;
}

static int check_ctx(lbpf_ctx* c, int domain)
{
    if (!c) return fail(nullptr, LBPF_EINVAL, "context is NULL");
    if (domain < 0 || domain >= c->n_domains) return fail(c, LBPF_EINVAL, "domain %d out of range", domain);
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, LBPF_ECUDA, "cudaSetDevice(%d) failed", c->device);
    return LBPF_OK;
}

// The device error word (set by a bounded wait of the staged kernel that
// gave up); read after the stream has been synchronised.
static int device_error(lbpf_ctx* c)
{
    int w = 0;
    CK(cudaMemcpy(&w, c->d_counters + 4, sizeof(int), cudaMemcpyDeviceToHost));
    if (w) return fail(c, LBPF_ETIMEOUT, "a bounded wait in the step kernel gave up (device error word %d)", w);
    return LBPF_OK;
}

// Lagged -> synchronised: the heat update of the last step on every domain.
static int sync_state(lbpf_ctx* c)
{
    if (!c->lagged) return LBPF_OK;
    for (int k = 0; k < c->n_domains; ++k) CK(c->L->heat_sync(c->d_dd + k, c->cur, c->fcur, c->acur, c->stream));
    c->fcur ^= 1;
    if (c->Sg != c->Qg) c->acur ^= 1;
    c->lagged = 0;
    return LBPF_OK;
}

extern "C" int lbpf_seed(lbpf_ctx* c, int domain, const lbpf_seed_t* seeds, int n_seeds)
{
    int rc = check_ctx(c, domain);
    if (rc) return rc;
    if (!seeds || n_seeds < 1 || n_seeds > 4096) return fail(c, LBPF_EINVAL, "lbpf_seed: need 1..4096 seeds");
    const lbpf_domain& d = c->in[domain];
    std::vector<double> h(5 * (size_t)n_seeds);
    for (int j = 0; j < n_seeds; ++j) {
        const lbpf_seed_t& s = seeds[j];
        if (s.crystal < 0 || s.crystal >= d.n_crystals)
            return fail(c, LBPF_EINVAL, "lbpf_seed: seed %d crystal %d out of range", j, s.crystal);
        if (!std::isfinite(s.x) || !std::isfinite(s.y) || !std::isfinite(s.z) || !std::isfinite(s.radius))
            return fail(c, LBPF_EINVAL, "lbpf_seed: seed %d not finite", j);
        h[5 * j + 0] = s.x;
        h[5 * j + 1] = s.y;
        h[5 * j + 2] = s.z;
        h[5 * j + 3] = s.radius;
        h[5 * j + 4] = s.crystal;
    }
    if ((rc = sync_state(c))) return rc;
    if (n_seeds > c->seeds_cap) {
        void* p = nullptr;
        if ((rc = dev_alloc(c, &p, sizeof(double) * 5 * n_seeds))) return rc;
        c->d_seeds = static_cast<double*>(p);
        c->seeds_cap = n_seeds;
    }
    CK(cudaMemcpyAsync(c->d_seeds, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, c->stream));
    CK(launch_seed(c->d_dd + domain, c->dd[domain].n, c->cur, c->acur, c->precision, c->d_seeds, n_seeds, c->dim,
                   d.dx / (std::sqrt(2.0) * d.W0), -d.delta, c->stream));
    CK(c->L->equilibrate(c->d_dd + domain, c->cur, c->fcur, c->acur, c->grad, 1, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->steps = 0;
    c->hist_count[domain] = 0;
    return LBPF_OK;
}

extern "C" int lbpf_write_fields(lbpf_ctx* c, int domain, const void* phi, const void* u, const int* index,
                                 int on_device)
{
    int rc = check_ctx(c, domain);
    if (rc) return rc;
    if (!phi || !u) return fail(c, LBPF_EINVAL, "lbpf_write_fields: phi and u are required");
    if ((rc = sync_state(c))) return rc;
    const DomainDev& h = c->dd[domain];
    const size_t bytes = (size_t)h.n * c->rsize;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(h.phi[c->cur], phi, bytes, kind, c->stream));
    CK(cudaMemcpyAsync(h.aux[c->acur], u, bytes, kind, c->stream));
    if (h.use_index) {
        if (index) {
            CK(cudaMemcpyAsync(c->scratch, index, sizeof(int) * h.n, kind, c->stream));
            CK(launch_index_from_i32(static_cast<const int*>(c->scratch), h.I[c->cur], h.n, h.n_crystals, c->stream));
        } else {
            CK(launch_fill_i8(h.I[c->cur], 0, h.n, c->stream));
        }
    }
    CK(c->L->equilibrate(c->d_dd + domain, c->cur, c->fcur, c->acur, c->grad, 0, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->steps = 0;
    c->hist_count[domain] = 0;
    return LBPF_OK;
}

// One launch of the fused step on the context's stream.
static int launch_step(lbpf_ctx* c)
{
    StepArgs a;
    a.doms = c->d_dd;
    a.items = c->d_items;
    a.n_items = c->n_items;
    a.counters = c->d_counters;
    a.cur = c->cur;
    a.fcur = c->fcur;
    a.acur = c->acur;
    a.collide = c->lagged;
    a.grad = c->grad;
    if (c->staged)
        CK(c->L->step_staged(a, c->n_blocks, c->stream));
    else
        CK(c->L->step(c->tile_v, c->kind, a, c->n_blocks, c->stream));
    c->cur ^= 1;
    c->acur ^= 1;
    if (c->lagged) c->fcur ^= 1;
    c->lagged = 1;
    c->steps += 1;
    c->kernels += 1;
    return LBPF_OK;
}

// Steady-state launches come in batches of kGraphSteps replayed from a CUDA
// graph; the launch arguments of a batch depend only on the buffer parities
// (cur, fcur, acur), which return to their start after an even batch.
constexpr int kGraphSteps = 16;

static int graph_batch(lbpf_ctx* c)
{
    const int key = c->cur | (c->fcur << 1) | (c->acur << 2);
    cudaGraphExec_t& ex = c->graphs[key];
    if (!ex) {
        const int cur = c->cur, fcur = c->fcur, acur = c->acur;
        const long long steps = c->steps, kernels = c->kernels;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            c->graphs_off = true;
            return LBPF_OK;
        }
        int rc = LBPF_OK;
        for (int k = 0; k < kGraphSteps && rc == LBPF_OK; ++k) rc = launch_step(c);
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        c->cur = cur;  // capture recorded the launches without running them
        c->fcur = fcur;
        c->acur = acur;
        c->steps = steps;
        c->kernels = kernels;
        if (rc != LBPF_OK || e != cudaSuccess || cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
            ex = nullptr;
            c->graphs_off = true;
            return LBPF_OK;
        }
        cudaGraphDestroy(g);
    }
    CK(cudaGraphLaunch(ex, c->stream));
    c->steps += kGraphSteps;
    c->kernels += kGraphSteps;  // each batch is kGraphSteps step-kernel launches
    return LBPF_OK;
}

extern "C" int lbpf_step(lbpf_ctx* c, int n_steps)
{
    int rc = check_ctx(c, 0);
    if (rc) return rc;
    if (n_steps < 0) return fail(c, LBPF_EINVAL, "lbpf_step: n_steps < 0");
    if (c->tune_pending && n_steps > 0) {
        c->tune_pending = false;
        if ((rc = autotune(c))) return rc;
    }
    // graphs need a capturable stream (not the legacy default stream)
    const bool graphs = c->stream != nullptr && !c->graphs_off;
    while (n_steps > 0) {
        if (graphs && c->lagged && n_steps >= kGraphSteps && !c->graphs_off) {
            if ((rc = graph_batch(c))) return rc;
            if (!c->graphs_off) {
                n_steps -= kGraphSteps;
                continue;
            }
        }
        if ((rc = launch_step(c))) return rc;
        n_steps -= 1;
    }
    return LBPF_OK;
}

// Element size of a field selected by one LBPF_READ_* bit.
static size_t field_esize(const lbpf_ctx* c, unsigned bit) { return bit == LBPF_READ_INDEX ? sizeof(int) : c->rsize; }

extern "C" int lbpf_read_fields(lbpf_ctx* c, int domain, unsigned mask, void* out, int out_on_device, size_t out_bytes)
{
    int rc = check_ctx(c, domain);
    if (rc) return rc;
    constexpr unsigned kAll = LBPF_READ_PHI | LBPF_READ_U | LBPF_READ_AS | LBPF_READ_INDEX;
    if (!out) return fail(c, LBPF_EINVAL, "lbpf_read_fields: out is NULL");
    if (mask == 0 || (mask & ~kAll)) return fail(c, LBPF_EINVAL, "lbpf_read_fields: bad mask 0x%x", mask);
    const DomainDev& h = c->dd[domain];
    size_t need = 0;
    for (unsigned bit = 1; bit <= LBPF_READ_INDEX; bit <<= 1)
        if (mask & bit) need += (size_t)h.n * field_esize(c, bit);
    if (out_bytes < need) return fail(c, LBPF_ERANGE, "lbpf_read_fields: need %zu bytes, got %zu", need, out_bytes);
    if (mask & LBPF_READ_U)
        if ((rc = sync_state(c))) return rc;
    const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    char* o = static_cast<char*>(out);
    for (unsigned bit = 1; bit <= LBPF_READ_INDEX; bit <<= 1) {
        if (!(mask & bit)) continue;
        const size_t bytes = (size_t)h.n * field_esize(c, bit);
        // fields that need a kernel are written in place (device output) or
        // into the context's scratch and copied from there (host output); the
        // copies run in stream order, so the scratch is free again for the
        // next field without a synchronisation
        void* dst = out_on_device ? static_cast<void*>(o) : c->scratch;
        switch (bit) {
        case LBPF_READ_PHI:
            CK(cudaMemcpyAsync(o, h.phi[c->cur], bytes, kind, c->stream));
            dst = nullptr;
            break;
        case LBPF_READ_U: CK(c->L->read_u(c->d_dd + domain, c->cur, c->fcur, c->acur, dst, c->stream)); break;
        case LBPF_READ_AS: CK(c->L->read_as(c->d_dd + domain, c->cur, c->grad, dst, c->stream)); break;
        case LBPF_READ_INDEX:
            if (h.use_index)
                CK(launch_index_to_i32(h.I[c->cur], static_cast<int*>(dst), h.n, c->stream));
            else
                CK(launch_fill_i32(static_cast<int*>(dst), 1, h.n, c->stream));
            break;
        }
        if (dst && !out_on_device) CK(cudaMemcpyAsync(o, dst, bytes, cudaMemcpyDeviceToHost, c->stream));
        o += bytes;
    }
    CK(cudaStreamSynchronize(c->stream));
    return device_error(c);
}

extern "C" int lbpf_read_field(lbpf_ctx* c, int domain, int field, void* out, int out_on_device, size_t out_bytes)
{
    static const unsigned bits[4] = {LBPF_READ_PHI, LBPF_READ_U, LBPF_READ_INDEX, LBPF_READ_AS};
    if (field < LBPF_FIELD_PHI || field > LBPF_FIELD_AS) {
        int rc = check_ctx(c, domain);
        return rc ? rc : fail(c, LBPF_EINVAL, "lbpf_read_field: bad field %d", field);
    }
    return lbpf_read_fields(c, domain, bits[field], out, out_on_device, out_bytes);
}

extern "C" int lbpf_read_populations(lbpf_ctx* c, int domain, int which, void* out, int out_on_device, size_t out_bytes)
{
    int rc = check_ctx(c, domain);
    if (rc) return rc;
    if (!out || (which != 0 && which != 1)) return fail(c, LBPF_EINVAL, "lbpf_read_populations: bad arguments");
    const DomainDev& h = c->dd[domain];
    const int Q = which == 0 ? c->Qg : c->Qu;
    const size_t bytes = (size_t)Q * h.n * c->rsize, one = (size_t)h.n * c->rsize;
    if (out_bytes < bytes) return fail(c, LBPF_ERANGE, "lbpf_read_populations: need %zu bytes, got %zu", bytes, out_bytes);
    if ((rc = sync_state(c))) return rc;
    // one population at a time, host reads through the context's scratch
    for (int i = 0; i < Q; ++i) {
        char* o = static_cast<char*>(out) + (size_t)i * one;
        void* dst = out_on_device ? static_cast<void*>(o) : c->scratch;
        CK(c->L->read_pop(c->d_dd + domain, which, i, c->cur, c->fcur, c->acur, dst, c->stream));
        if (!out_on_device) CK(cudaMemcpyAsync(o, dst, one, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return LBPF_OK;
}

extern "C" int lbpf_measure(lbpf_ctx* c, int domain, int cx, int cy, int cz, double* tip6, double* solid_fraction,
                            double* conserved)
{
    int rc = check_ctx(c, domain);
    if (rc) return rc;
    const DomainDev& h = c->dd[domain];
    if (cx < 0 || cx >= h.nx || cy < 0 || cy >= h.ny || cz < 0 || cz >= h.nz)
        return fail(c, LBPF_EINVAL, "lbpf_measure: centre (%d, %d, %d) outside the domain", cx, cy, cz);
    if ((rc = sync_state(c))) return rc;
    CK(c->L->read_u(c->d_dd + domain, c->cur, c->fcur, c->acur, c->scratch, c->stream));
    double* outp = c->red + 3 * kReduceBlocks;
    CK(launch_reduce(h.phi[c->cur], c->scratch, h.n, c->precision, c->red, outp, c->stream, h.nx, h.ny, h.nz, h.bc,
                     c->dim));
    CK(launch_tips(h.phi[c->cur], h.nx, h.ny, h.nz, cx, cy, cz, c->dim, c->precision, outp + 3, c->stream, h.bc));
    {
        const int slot = (c->hist_last[domain] + 1) % kHistCap;
        CK(launch_hist_append(outp + 3, (double)c->steps * c->in[domain].dt,
                              c->d_hist + 7 * ((size_t)domain * kHistCap + slot), c->stream));
        c->hist_last[domain] = slot;
        if (c->hist_count[domain] < kHistCap) c->hist_count[domain] += 1;
    }
    double hv[9];
    CK(cudaMemcpyAsync(hv, outp, sizeof(hv), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (tip6)
        for (int k = 0; k < 6; ++k) tip6[k] = hv[3 + k];
    if ((rc = device_error(c))) return rc;
    if (solid_fraction) *solid_fraction = hv[0] / (double)h.n;
    if (conserved) *conserved = hv[1];
    if (hv[2] > 0) return fail(c, LBPF_ENONFINITE, "lbpf_measure: %.0f non-finite values in phi or u", hv[2]);
    return LBPF_OK;
}

extern "C" int lbpf_tip_velocity(lbpf_ctx* c, int domain, int window, double* v6)
{
    int rc = check_ctx(c, domain);
    if (rc) return rc;
    if (!v6 || window < 2) return fail(c, LBPF_EINVAL, "lbpf_tip_velocity: need v6 and window >= 2");
    if (c->hist_count[domain] < 2)
        return fail(c, LBPF_EINVAL, "lbpf_tip_velocity: fewer than two measurements since the last seed");
    double* out = c->red + 3 * kReduceBlocks + 9;
    CK(launch_tip_velocity(c->d_hist + 7 * (size_t)domain * kHistCap, kHistCap, c->hist_last[domain],
                           c->hist_count[domain], window, c->in[domain].dx, out, c->stream));
    CK(cudaMemcpyAsync(v6, out, 6 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LBPF_OK;
}

extern "C" int lbpf_tip_radius(lbpf_ctx* c, int domain, int cx, int cy, int cz, int dir, int J, double* rho)
{
    int rc = check_ctx(c, domain);
    if (rc) return rc;
    const DomainDev& h = c->dd[domain];
    if (!rho || dir < 0 || dir >= 2 * c->dim || J < 1 || (2 * J + 1) * (c->dim - 1) > 32)
        return fail(c, LBPF_EINVAL, "lbpf_tip_radius: bad direction or J (1..15 in 2D, 1..7 in 3D)");
    if (cx < 0 || cx >= h.nx || cy < 0 || cy >= h.ny || cz < 0 || cz >= h.nz)
        return fail(c, LBPF_EINVAL, "lbpf_tip_radius: centre outside the domain");
    double* out = c->red + 3 * kReduceBlocks + 15;
    CK(launch_tip_radius(h.phi[c->cur], h.nx, h.ny, h.nz, cx, cy, cz, dir, J, c->dim, c->precision, out, c->stream,
                         h.bc));
    CK(cudaMemcpyAsync(rho, out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LBPF_OK;
}

extern "C" int lbpf_set_schedule(lbpf_ctx* c, int tile_rows, int segment)
{
    int rc = check_ctx(c, 0);
    if (rc) return rc;
    int v = -1;
    for (int k = 0; k < kNumTileVariants; ++k)
        if (kTileRows[k] == tile_rows) v = k;
    if (v < 0 || segment < 1) return fail(c, LBPF_EINVAL, "lbpf_set_schedule: tile_rows must be 8 or 16, segment >= 1");
    if ((c->staged || c->kind) && v != 0)
        return fail(c, LBPF_EINVAL,
                    "lbpf_set_schedule: 16-row tiles exist only for periodic domains without advection (generic kernel)");
    CK(cudaStreamSynchronize(c->stream));
    c->tune_pending = false;
    c->tuned = "set";
    return set_schedule(c, v, segment);
}

extern "C" int lbpf_query(const lbpf_ctx* c, int what, double* value)
{
    if (!c || !value) return fail(nullptr, LBPF_EINVAL, "lbpf_query: NULL argument");
    double v = 0;
    switch (what) {
    case LBPF_Q_SITES:
        for (const DomainDev& h : c->dd) v += (double)h.n;
        break;
    case LBPF_Q_STEPS: v = (double)c->steps; break;
    case LBPF_Q_BYTES_PER_SITE: {
        // read + write of every stored population, of phi and of aux (and of
        // the index field when it is used)
        double idx_sites = 0, all_sites = 0;
        for (const DomainDev& h : c->dd) {
            all_sites += (double)h.n;
            if (h.use_index) idx_sites += (double)h.n;
        }
        v = 2.0 * (c->Sg + c->Su) * c->ssize + 4.0 * c->rsize + 2.0 * idx_sites / all_sites;
        break;
    }
    case LBPF_Q_DEVICE_BYTES: v = (double)c->dev_bytes; break;
    case LBPF_Q_LAMBDA: v = c->dd[0].lambda; break;
    case LBPF_Q_STEP_KERNELS: v = (double)c->kernels; break;
    case LBPF_Q_TILE_ROWS: v = kTileRows[c->tile_v]; break;
    case LBPF_Q_SEGMENT: v = c->seg_len; break;
    case LBPF_Q_BLOCKS: v = c->n_blocks; break;
    case LBPF_Q_KERNEL: v = c->staged ? 1 : 0; break;
    default: return fail(const_cast<lbpf_ctx*>(c), LBPF_EINVAL, "lbpf_query: unknown property %d", what);
    }
    *value = v;
    return LBPF_OK;
}

extern "C" int lbpf_destroy(lbpf_ctx* c)
{
    if (!c) return LBPF_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (cudaGraphExec_t g : c->graphs)
        if (g) cudaGraphExecDestroy(g);
    free_all(c);
    delete c;
    return LBPF_OK;
}

extern "C" const char* lbpf_last_error(const lbpf_ctx* c) { return c ? c->err.c_str() : t_err.c_str(); }
