/*
 * lbpf — lattice Boltzmann phase-field crystal growth on one NVIDIA GB300.
 *
 * C ABI of the per-time-step update of the phase field phi and the
 * dimensionless temperature u of a pure substance, as defined by
 * Younsi & Cartalade, "On anisotropy function in crystal growth simulations
 * using Lattice Boltzmann equation" (arXiv:1606.09432):
 *   - model:  Eq. (PhaseField_KarmaRappel), Eq. (Temp_Ramirez), Eq. (TermesAnisotropes)
 *   - heat LB scheme (Sec. 3.1):  Eqs. (LBE_Eq_Temp)-(ThermalDiffusivity)
 *   - phase-field LB scheme (Sec. 3.2): Eqs. (LBE_Eq_Phase), (Feq_Phase),
 *     (Def_M0_Phi)-(LBE_RelaxationTime)
 *   - lattices (Sec. 3.3, Table 1), gradients (Sec. 4.2),
 *     anisotropy functions (Secs. 2, 4.1, 4.3, 5.2).
 *
 * Conventions for every function:
 *   - The return value is an lbpf_status; nothing throws or aborts across the
 *     ABI.  On failure lbpf_last_error() describes the cause.
 *   - All sizes, positions and radii are in lattice units (sites); physical
 *     parameters (dx, dt, W0, tau0, kappa) are in any consistent unit system.
 *   - Fields are row-major with x fastest: element (x, y, z) of a domain of
 *     size nx*ny*nz is at index (z*ny + y)*nx + x.  Fields read back are
 *     double for LBPF_FP64 and float for the other precisions; the crystal
 *     index field is int32.
 *   - The caller owns every array it passes; inputs are copied during the
 *     call.  The context owns all device memory it allocates and borrows the
 *     CUDA stream given to lbpf_create (NULL = the legacy default stream).
 *   - Calls on one context must not overlap (one host thread at a time).
 *   - Boundaries are periodic, or zero-flux walls per axis (lbpf_domain.bc):
 *     the bounce-back walls of Sec. 3.3, taken as mirror planes through the
 *     boundary nodes (see LBPF_BC_WALL_X).
 */
#ifndef LBPF_H
#define LBPF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbpf_ctx lbpf_ctx;

typedef enum {
    LBPF_OK = 0,
    LBPF_EINVAL = -1,     /* invalid argument or parameter combination         */
    LBPF_ENOMEM = -2,     /* device or host allocation failed                  */
    LBPF_ECUDA = -3,      /* a CUDA runtime call failed (see lbpf_last_error)  */
    LBPF_ETIMEOUT = -4,   /* a bounded wait inside the step kernel gave up (reported by
                             the next call that synchronises: read, measure)    */
    LBPF_ENONFINITE = -5, /* a measurement found NaN or Inf in phi or u        */
    LBPF_ERANGE = -6      /* output buffer too small                           */
} lbpf_status;

/* Lattice pairs (Sec. 3.3): phase-field lattice / temperature lattice.
 * D2Q9/D2Q5 and D3Q15/D3Q7 are the paper's (Table 1); D3Q19 and D3Q27 are
 * mentioned by the paper (Sec. 3.3) with the standard weights
 * (1/3, 1/18, 1/36) and (8/27, 2/27, 1/54, 1/216), e^2 = 1/3. */
typedef enum {
    LBPF_D2Q9_D2Q5 = 0,
    LBPF_D3Q15_D3Q7 = 1,
    LBPF_D3Q19_D3Q7 = 2,
    LBPF_D3Q27_D3Q7 = 3
} lbpf_lattice;

/* Gradient of phi (Sec. 4.2): directional derivatives, Eqs.
 * (Def_DeriveeDirectionnelle) and (Grad_DF-Centree), or central finite
 * differences along the axes. */
typedef enum { LBPF_GRAD_DD = 0, LBPF_GRAD_FD = 1 } lbpf_grad;

/* Arithmetic and storage.
 *   LBPF_FP64:         FP64 arithmetic, FP64 populations.
 *   LBPF_FP32:         FP32 arithmetic, FP32 populations.
 *   LBPF_FP32_FP16DEV: FP32 arithmetic; populations stored as FP16
 *                      deviations g_i - w_i phi and f_i - w_i u for i >= 1
 *                      (the rest population is rebuilt so that the sums
 *                      phi = sum g_i, u = sum f_i hold exactly).
 *   LBPF_FP32_BF16DEV: as above with BF16 deviations.
 *   LBPF_FP32_FP16DEV_SR: FP16 deviations rounded stochastically (up or
 *                      down with probabilities given by the distances, so the
 *                      rounding errors of slowly varying values do not add up
 *                      step after step); the random bits come from a hash of
 *                      site, population and a step counter kept on the device,
 *                      so runs are reproducible.  About half the FP16 error of
 *                      round-to-nearest on a growing dendrite.  (There is no
 *                      BF16 counterpart: noise of BF16 size at the interface
 *                      is amplified by the growth instability.) */
typedef enum {
    LBPF_FP64 = 0,
    LBPF_FP32 = 1,
    LBPF_FP32_FP16DEV = 2,
    LBPF_FP32_BF16DEV = 3,
    LBPF_FP32_FP16DEV_SR = 4
} lbpf_precision;

/* Anisotropy functions a_s(n), n = -grad(phi)/|grad(phi)|, Eq. (Def_Normal_Vector).
 *   LBPF_AS_CUBIC100: 1 - 3 eps + 4 eps sum_a n_a^4, Eq. (As_Function_Classical)
 *   LBPF_AS_ANGLE:    1 + eps cos(q (varphi - phi0)), varphi = atan2(n_y, n_x),
 *                     Eq. (As_Theta); 2D lattices only
 *   LBPF_AS_Y66:      1 + eps (nx^6 - 15 nx^4 ny^2 + 15 nx^2 ny^4 - ny^6), Eq. (As_Y66)
 *   LBPF_AS_HOYT110:  1 + eps (Q - 3/5) + gamma (3 Q + 66 S - 17/7), Eq. (As_MatSci),
 *                     Q = sum n_a^4, S = nx^2 ny^2 nz^2
 *   LBPF_AS_S111:     1 + 66 gamma S.  Eq. (As_Function_S) prints 66 gamma S,
 *                     which vanishes on the axes; the constant term 1 is
 *                     added so that Eq. (LBE_Eq_Phase) stays defined. */
typedef enum {
    LBPF_AS_CUBIC100 = 0,
    LBPF_AS_ANGLE = 1,
    LBPF_AS_Y66 = 2,
    LBPF_AS_HOYT110 = 3,
    LBPF_AS_S111 = 4
} lbpf_aniso;

typedef struct {
    int kind;     /* lbpf_aniso                                  */
    double eps;   /* anisotropy strength eps_s                   */
    double gamma; /* <110>/<111> strength (HOYT110, S111)        */
    int q;        /* mode of the angle form (ANGLE)              */
    double phi0;  /* reference angle of the angle form, radians  */
} lbpf_crystal;

#define LBPF_MAX_CRYSTALS 16

/* Boundary bits of lbpf_domain.bc.  A set bit makes both ends of that axis
 * zero-flux walls (Sec. 3.3: zero fluxes on all boundaries, imposed by
 * bounce-back, for both equations); a clear bit leaves the axis periodic.
 * A wall is a mirror plane through the boundary nodes: the gradient stencil
 * reads phi of the mirror image beyond it (zero normal derivative), and a
 * population arriving from beyond it is the one streamed to the same node in
 * the mirrored direction.  For the axis populations (all of D2Q5 and D3Q7)
 * this is the printed rule f_i = f_i', i' the opposite direction; for the
 * diagonal populations the mirror keeps the wall a symmetry plane, so that a
 * box with walls on the symmetry planes is exactly one octant (quadrant) of
 * the symmetric crystal, as in the octant runs of Sec. 5.3.  Seeds use plain
 * (not periodic) distances along walled axes; the conserved sum of
 * lbpf_measure then weights nodes on a wall by 1/2 per walled coordinate.  A
 * walled axis needs at least 3 sites. */
#define LBPF_BC_WALL_X 1
#define LBPF_BC_WALL_Y 2
#define LBPF_BC_WALL_Z 4

/* One domain and its model parameters (Sec. 2, Sec. 3). */
typedef struct {
    int nx, ny, nz;  /* sites; nz = 1 for 2D lattices; each >= 2 in 3D, nx, ny >= 2 */
    int bc;          /* LBPF_BC_WALL_* bits; 0 = periodic in every direction   */
    double dx, dt;   /* space and time steps                                       */
    double W0, tau0; /* interface thickness and kinetic time, Eq. (PhaseField_KarmaRappel) */
    double kappa;    /* thermal diffusivity, Eq. (Temp_Ramirez)                    */
    double lambda;   /* coupling constant; <= 0 selects lambda* = kappa tau0/(a2 W0^2),
                        a2 = 0.6267, which cancels the kinetic coefficient of
                        Eq. (Kinetic-Coeff)                                        */
    double delta;    /* undercooling: u(x, 0) = -delta, Eq. (Intial-Cond_u)        */
    double xi;       /* index-field threshold on |grad phi| (physical units), Sec. 4.3 */
    int n_crystals;  /* 1..LBPF_MAX_CRYSTALS.  With one crystal its a_s applies
                        everywhere; with several, the crystal-index field of
                        Sec. 4.3 / Eq. (As_Multi) selects it per site          */
    lbpf_crystal crystals[LBPF_MAX_CRYSTALS];
    double adv[3];   /* uniform velocity v (physical units; all zero: pure
                        diffusion, the paper's runs).  Non-zero selects the
                        advection-diffusion form of the heat equilibrium
                        (Sec. 3.1, the equilibrium of Eq. EqFunction_Tempr with
                        a first-order velocity term):
                            f_i^(0) = w_i u (1 + e_i . v dt / (e^2 dx)),
                        whose first moment is u v dt / dx, so the recovered
                        equation is du/dt + div(u v) = kappa lap(u) + Q_u.
                        Every precision; 0 along a 2D lattice's z and along
                        every walled axis (the
                        velocity is tangential to the walls).  Stable for
                        |v| dt / dx well below 1; the scheme adds a numerical
                        diffusion of order |v|^2 dt.  EINVAL otherwise. */
} lbpf_domain;

/* A diffuse spherical (circular in 2D) nucleus, Eq. (Initial_Condition). */
typedef struct {
    double x, y, z; /* centre, lattice units (z ignored in 2D)   */
    double radius;  /* R_s, lattice units                        */
    int crystal;    /* 0 .. n_crystals - 1                       */
} lbpf_seed_t;

/* Create a context holding n_domains independent periodic domains that all
 * use one lattice pair, gradient operator and precision.  Allocates the
 * device state of every domain (two population sets per lattice, phi, an
 * auxiliary heat field, the index field when n_crystals > 1).
 * domains: n_domains entries (host memory, copied).  stream: a cudaStream_t
 * or NULL.  On success *out receives the context.
 * Errors: LBPF_EINVAL (bad sizes or parameters, e.g. the angle form on a 3D
 * lattice, a non-positive dx/dt/W0/tau0/kappa, relaxation rates <= 1/2),
 * LBPF_ENOMEM, LBPF_ECUDA. */
int lbpf_create(const lbpf_domain* domains, int n_domains, int lattice, int grad, int precision,
                void* stream, lbpf_ctx** out);

/* Initial condition of one domain from seeds, Eqs. (Initial_Condition) and
 * (Intial-Cond_u): phi = max over seeds of tanh((R - d) dx / (sqrt(2) W0)),
 * d the periodic (minimum-image) distance to the seed centre; u = -delta; the
 * index field takes the crystal of the dominant seed where phi > 0 or
 * |grad phi| > xi, else 0; populations start at their equilibria
 * g_i = g_i^(0)(phi, N) of Eq. (Feq_Phase) and f_i = w_i u of Eq.
 * (EqFunction_Tempr).  Resets the step counter.  seeds: host memory.
 * Errors: LBPF_EINVAL (domain index, n_seeds < 1 or > 4096, crystal out of range). */
int lbpf_seed(lbpf_ctx* ctx, int domain, const lbpf_seed_t* seeds, int n_seeds);

/* Initial condition from given fields: phi and u (double for LBPF_FP64,
 * float otherwise; nx*ny*nz elements each) and, when the domain has several
 * crystals, the int32 index field (NULL: all zero).  Populations start at
 * equilibrium as in lbpf_seed.  on_device != 0: the pointers are device
 * memory of the context's GPU, else host memory.  Resets the step counter. */
int lbpf_write_fields(lbpf_ctx* ctx, int domain, const void* phi, const void* u, const int* index,
                      int on_device);

/* Advance every domain by n_steps time steps (n_steps >= 0).  One step is
 * the phase-field scheme of Sec. 3.2 followed by the heat scheme of Sec. 3.1
 * with Q_u = (phi(t + dt) - phi(t)) / (2 dt), one kernel launch for all
 * domains.  On a non-default stream, runs of 16 steps are replayed from CUDA
 * graphs captured on first use (do not call lbpf_step while another capture
 * is active on the context's stream).  Asynchronous on the context's stream
 * (except the first call of a context whose schedule is timed, see
 * lbpf_set_schedule); launch errors are returned, device errors surface at
 * the next synchronising call. */
int lbpf_step(lbpf_ctx* ctx, int n_steps);

typedef enum {
    LBPF_FIELD_PHI = 0,   /* phi, Eq. (Def_M0_Phi)                          */
    LBPF_FIELD_U = 1,     /* u, Eq. (Temperature_LB)                        */
    LBPF_FIELD_INDEX = 2, /* crystal index I (int32), Sec. 4.3; all 1 with one crystal */
    LBPF_FIELD_AS = 3     /* a_s(n) of the current phi (see lbpf_read_fields) */
} lbpf_field;

/* Field selection bits of lbpf_read_fields.  The selected fields are written
 * back to back in increasing bit order, each nx*ny*nz elements: phi, u and
 * a_s in the arithmetic type (double for LBPF_FP64, float otherwise), then
 * the index field as int32 (last, so that every double stays 8-byte
 * aligned when out is). */
#define LBPF_READ_PHI   (1u << 0)
#define LBPF_READ_U     (1u << 1)
#define LBPF_READ_AS    (1u << 2)
#define LBPF_READ_INDEX (1u << 3)

/* Copy the fields selected by mask (LBPF_READ_* bits, at least one) of one
 * domain into out, in the order and types given above:
 *   phi: Eq. (Def_M0_Phi), the zeroth moment of the phase-field populations;
 *   u:   Eq. (Temperature_LB), the zeroth moment of the heat populations (a
 *        lagged heat update is brought up to date first);
 *   a_s: the anisotropy function of the site's crystal, Eqs.
 *        (As_Function_Classical), (As_Theta), (As_Y66), (As_MatSci),
 *        (As_Function_S), at the normal n = -grad phi / |grad phi| of Eq.
 *        (Def_Normal_Vector) of the current phi, with the context's gradient
 *        operator (Sec. 4.2); 1 where the crystal index is 0 or |grad phi|
 *        is below the zero-gradient guard (1e-10 lattice units in FP64, 1e-6
 *        in FP32).  Evaluated on the device by the same code as the step;
 *   index: the crystal index field of Sec. 4.3 (1 everywhere with one crystal).
 * out is device memory of the context's GPU if out_on_device != 0, else host
 * memory (pinned memory makes the copies asynchronous DMA); the caller owns
 * it.  out_bytes must cover every selected field.  The library allocates no
 * memory: host reads are staged through a device buffer the context owns.
 * Synchronises the stream once, at the end.
 * Errors: LBPF_EINVAL (bad domain, NULL out, empty or unknown mask bits),
 * LBPF_ERANGE (buffer too small), LBPF_ECUDA. */
int lbpf_read_fields(lbpf_ctx* ctx, int domain, unsigned mask, void* out, int out_on_device, size_t out_bytes);

/* One field of one domain (field: lbpf_field); the same as lbpf_read_fields
 * with the one matching bit.  out_bytes must be at least nx*ny*nz * element
 * size.  Synchronises the stream.
 * Errors: LBPF_ERANGE (buffer too small), LBPF_EINVAL, LBPF_ECUDA. */
int lbpf_read_field(lbpf_ctx* ctx, int domain, int field, void* out, int out_on_device,
                    size_t out_bytes);

/* Copy the populations of one domain, decoded to the arithmetic type
 * (double for LBPF_FP64, float otherwise): which = 0 for g_i (phase field,
 * Q_phi arrays of nx*ny*nz), which = 1 for f_i (temperature, Q_u arrays).
 * Population i of site k is at [i * nx*ny*nz + k]; direction numbering as in
 * Sec. 3.3 (D3Q19/D3Q27: axes, then the xy-, xz-, yz-edges, then corners).
 * Host reads are staged through a device buffer the context owns (no
 * allocation per call).  Synchronises the stream. */
int lbpf_read_populations(lbpf_ctx* ctx, int domain, int which, void* out, int out_on_device,
                          size_t out_bytes);

/* Measurements of one domain (synchronises the stream):
 *   tip6[6]:  distance from the site (cx, cy, cz) to the outermost phi = 0
 *             crossing along +x, -x, +y, -y, +z, -z (linear interpolation,
 *             rays of half the domain length on periodic axes, up to the
 *             wall on walled ones; -1 when a ray has no crossing; the z
 *             entries are -1 in 2D).  The paper defines the tip velocity
 *             V_p from the tip position (Sec. 3.4) but not the position itself.
 *   solid_fraction: mean of (1 + phi)/2.
 *   conserved: sum over sites of (u - phi/2), accumulated in FP64; constant
 *             in a periodic or walled box (integral of Eq. (Temp_Ramirez)
 *             with zero flux); sites on walls count 1/2 per walled coordinate.
 * Any output pointer may be NULL.  Returns LBPF_ENONFINITE if phi or u holds
 * a NaN or Inf. */
int lbpf_measure(lbpf_ctx* ctx, int domain, int cx, int cy, int cz, double* tip6,
                 double* solid_fraction, double* conserved);

/* Tip velocity of one domain (synchronises the stream): the least-squares
 * slope, in FP64, of each tip distance of lbpf_measure (physical length:
 * lattice units x dx) over physical time (steps x dt), over the last `window`
 * measurements (>= 2) since the last seed; lbpf_measure records at most the
 * last 64.  v6 receives the speeds along +x, -x, +y, -y, +z, -z (NaN where
 * fewer than two measurements had a crossing).  The paper reports the tip
 * velocity V_p and its dimensionless form V_p d0 / kappa, d0 = a1 W0 / lambda
 * (Sec. 3.4); the slope fit is a reading (the paper does not say how V_p is
 * taken).  Errors: LBPF_EINVAL (window < 2, fewer than two measurements). */
int lbpf_tip_velocity(lbpf_ctx* ctx, int domain, int window, double* v6);

/* Tip radius (lattice units) of the tip along direction dir (0..5 = +x, -x,
 * +y, -y, +z, -z) seen from the site (cx, cy, cz): the phi = 0 crossings on
 * the rays parallel to the axis at transverse offsets |j| <= J are fitted by
 * x_c(j) = a + b j^2 (least squares, FP64) and rho = -1/(2b); in 3D the mean
 * over the two transverse planes.  The paper does not define a tip radius;
 * this is a reading.  *rho = -1 when no fit is possible.  J: 1..15 in 2D,
 * 1..7 in 3D.  Synchronises the stream.  Errors: LBPF_EINVAL. */
int lbpf_tip_radius(lbpf_ctx* ctx, int domain, int cx, int cy, int cz, int dir, int J, double* rho);

typedef enum {
    LBPF_Q_SITES = 0,          /* total sites over all domains                       */
    LBPF_Q_STEPS = 1,          /* steps done since the last seed / write_fields      */
    LBPF_Q_BYTES_PER_SITE = 2, /* algorithmic HBM bytes one fused step moves per site */
    LBPF_Q_DEVICE_BYTES = 3,   /* device memory held by the context                  */
    LBPF_Q_LAMBDA = 4,         /* lambda of domain 0 (after the lambda* rule)        */
    LBPF_Q_STEP_KERNELS = 5,   /* step-kernel launches issued by lbpf_step so far     */
    LBPF_Q_TILE_ROWS = 6,      /* tile variant of the step kernel (autotuned): 8, 16 */
    LBPF_Q_SEGMENT = 7,        /* z-planes (3D) or y-rows (2D) per work item          */
    LBPF_Q_BLOCKS = 8,         /* resident blocks of the persistent step launch       */
    LBPF_Q_KERNEL = 9          /* step kernel: 0 generic (global-memory pulls, the
                                  default), 1 staged (rows brought to shared memory by
                                  asynchronous copies; chosen by the environment
                                  variable LBPF_KERNEL=staged at lbpf_create for 3D
                                  D3Q15/D3Q19 domains with 16-bit deviation storage,
                                  nx a multiple of 8 and >= 64, one crystal; same
                                  results bit for bit, slower on GB300)             */
} lbpf_query_t;

/* Override the work schedule of the step kernel.  Normally lbpf_create takes
 * a choice cached for the configuration (file LBPF_TUNE_CACHE, default
 * ~/.cache/lbpf_tune.txt) or a rule; configurations of >= 4e6 sites (or any,
 * with LBPF_AUTOTUNE=1; none with LBPF_AUTOTUNE=0) are then timed at the
 * first lbpf_step, on the live state, which that call leaves unchanged (it
 * synchronises the stream once and caches the choice).  The kernel marches
 * a tile along z (3D) or y (2D).  tile_rows is 8 or 16: in 3D the tile is 32
 * sites along x by tile_rows along y; in 2D it is one row of 16 * tile_rows
 * sites (128 or 256) along x.  segment (>= 1) is the number of z-planes (3D)
 * or y-rows (2D) per work item (tile_rows = 16 exists only for periodic
 * domains and the generic kernel).  Results do not depend on the schedule;
 * only speed does.  A performance knob with no counterpart in the paper.
 * Errors: LBPF_EINVAL. */
int lbpf_set_schedule(lbpf_ctx* ctx, int tile_rows, int segment);

/* Read a property of the context into *value. */
int lbpf_query(const lbpf_ctx* ctx, int what, double* value);

/* The two measurement sums of lbpf_measure (sum of (1 + phi)/2 and sum of
 * u - phi/2, FP64 accumulation) over caller-provided fields, for callers that
 * cannot allocate device memory when they call: applications that hand all
 * device memory to their own pool allocator (an allocation by this library
 * would fail or fragment the pool) and latency-critical loops where
 * cudaMalloc/cudaFree would synchronise the device.  The paper has no
 * counterpart; this is an interface convenience.
 *   phi, u: device arrays of n elements (double for LBPF_FP64, float for the
 *           other precisions), e.g. filled by lbpf_read_field(out_on_device=1).
 *   n:      1 .. 268435456 sites; larger sizes return LBPF_ERANGE.
 *   out:    device array of 3 doubles: sum (1 + phi)/2, sum (u - phi/2), and
 *           the number of non-finite phi or u values.
 *   stream: cudaStream_t or NULL; the call is asynchronous on it.
 * Allocates nothing: its scratch is a fixed 96 KiB device array that every
 * GPU loading the library holds until the process exits.  The first call on
 * each device looks up that array's device address (set-up work); make it
 * before any stream capture.  All calls share the array: calls whose kernels
 * overlap on the GPU race and must be serialised by the caller.
 * Errors: LBPF_EINVAL (NULL pointer, bad precision), LBPF_ERANGE, LBPF_ECUDA. */
int lbpf_field_sums_static(const void* phi, const void* u, long long n, int precision, double* out,
                           void* stream);

/* ---------------------------------------------------------------------------
 * Learned surrogate (not in the paper): a 2D U-Net that predicts the change
 * of phi and u over a jump of K lattice Boltzmann steps, used by a controller
 * that alternates network jumps with plain LB validation and falls back to LB.
 * Architecture: `levels` levels with base * 2^l channels at level l (default
 * 3 levels, base 16: 16, 32, 64 channels), two periodic 3x3 convolutions +
 * ReLU per level on the way down (2x2 average pooling between levels) and on
 * the way up (nearest 2x upsampling concatenated with the level's skip), 1x1
 * head to 2 channels.  Input per site (NHWC, FP32): (phi, u, cos 4 theta,
 * sin 4 theta, eps) zero-padded to 16 channels; output (d phi, d u), the phi
 * channel multiplied by (1 - phi^2) so that the bulk phases stay fixed.  3x3
 * convolutions and their weight gradients run on the tensor cores (tcgen05,
 * BF16 operands, FP32 accumulation); everything else in FP32.
 * Parameters: one flat FP32 vector (per 3x3 layer, encoder level by level
 * then decoder from the deepest level up: weights [tap][cout][cin], then
 * biases; then the head's [2][base] weights and 2 biases).
 * All device pointers below are device memory of the current GPU.
 * ------------------------------------------------------------------------- */
typedef struct lbpf_net lbpf_net;

/* Network for batches of `batch` images of H x W sites, He-uniform weights
 * from `seed`: levels 2..5, base 16, 32 or 64 with base 2^(levels - 1) <=
 * 256; H, W multiples of 8 * 2^(levels - 1).  Errors: LBPF_EINVAL,
 * LBPF_ENOMEM, LBPF_ECUDA. */
int lbpf_net_create_arch(int H, int W, int batch, int levels, int base, unsigned long long seed, void* stream,
                         lbpf_net** out);
/* The default network: lbpf_net_create_arch with 3 levels, base 16. */
int lbpf_net_create(int H, int W, int batch, unsigned long long seed, void* stream, lbpf_net** out);
int lbpf_net_destroy(lbpf_net* net);
const char* lbpf_net_last_error(const lbpf_net* net);
int lbpf_net_num_params(const lbpf_net* net, long long* n);
/* Copy the parameters (which = 0) or the last gradients (which = 1) to host. */
int lbpf_net_get_params(lbpf_net* net, float* host, int which);
int lbpf_net_set_params(lbpf_net* net, const float* host);
/* y (N, H, W, 2) = network(x (N, H, W, 5)); y may be NULL (output kept). */
int lbpf_net_forward(lbpf_net* net, const float* x, float* y);
/* Parameter gradients of sum(out * dy) after a forward pass (read them with
 * lbpf_net_get_params(which = 1)). */
int lbpf_net_backward(lbpf_net* net, const float* dy);
/* One Adam step (beta 0.9, 0.999) on the mean squared error to `target`
 * (N, H, W, 2), weighted per site (see lbpf_net_set_loss_weight); *loss (may
 * be NULL) receives the loss before the step. */
int lbpf_net_train_step(lbpf_net* net, const float* x, const float* target, float lr, double* loss);
/* Weight of the training loss: each squared error counts 1 + alpha *
 * max(0, 1 - phi^2) times, phi the input phase field of its site, so that the
 * interface (where a jump changes the fields) outweighs the bulk.  alpha = 0
 * (the default) is the plain mean squared error.  Not in the paper.
 * Errors: LBPF_EINVAL (NULL net, alpha < 0 or NaN). */
int lbpf_net_set_loss_weight(lbpf_net* net, float alpha);
/* Network input from fields: x[p] = (phi, u, cos 4 theta, sin 4 theta, eps)
 * of the crystal I = index[p] (1 everywhere when index is NULL; zeros for
 * I = 0 or I > n_crystals), crystal_tab[2 (I-1)] = eps, [2 (I-1) + 1] = theta. */
int lbpf_net_assemble(const float* phi, const float* u, const int* index, const float* crystal_tab,
                      int n_crystals, float* x, long long sites, void* stream);
/* phi += y[.][0], u += y[.][1] (a network jump). */
int lbpf_net_apply(const float* y, float* phi, float* u, long long sites, void* stream);
/* y = (phi1 - phi0, u1 - u0) per site: the training target of a jump. */
int lbpf_net_delta(const float* phi0, const float* u0, const float* phi1, const float* u1, float* y,
                   long long sites, void* stream);
/* *count (device unsigned int) = number of sites with phi outside [lo, hi]
 * or not finite (the controller's fall-back test). */
int lbpf_net_range_check(const float* phi, long long sites, float lo, float hi, unsigned int* count,
                         void* stream);

/* One periodic 3x3 convolution layer of the surrogate network, on the
 * tensor cores (tcgen05.mma, BF16 operands, FP32 accumulation in tensor
 * memory):
 *   y[n][h][w][co] = act(b[co] + sum_tap sum_ci wt[tap][co][ci] x[n][h'][w'][ci]),
 *   tap = 3 (dy + 1) + (dx + 1), h' = (h + dy) mod H, w' = (w + dx) mod W,
 * act = ReLU if relu != 0, else the identity.  x: FP32 (n, H, W, cin); y:
 * FP32 (n, H, W, cout); wt: BF16 bit patterns [9][cout][cin]; bias: FP32
 * [cout] or NULL.  x is rounded to BF16 (to nearest even) on the way in.
 * All pointers are device memory owned by the caller; the call is
 * asynchronous on `stream`.  cin a multiple of 16; cout split into equal
 * tiles of at most 256 channels (one MMA), each a multiple of 16 (so cout
 * above 256 a multiple of 32, above 512 of 48); n, H, W >= 1: else
 * LBPF_EINVAL; LBPF_ECUDA if the launch fails. */
int lbpf_nn_conv3x3(const float* x, const void* wt, const float* bias, float* y, int n, int H, int W, int cin,
                    int cout, int relu, void* stream);
/* Weight gradient of that layer, added to dwt:
 *   dwt[tap][co][ci] += sum_n,h,w dy[n][h][w][co] x[n][h'][w'][ci]
 * (h', w' as above), on the tensor cores with x and dy rounded to BF16 (to
 * nearest even) and FP32 accumulation; dwt FP32 [9][cout][cin].  Device
 * pointers, asynchronous on `stream`; the sum's order varies from call to
 * call (FP32 atomics).  cin, cout multiples of 16 (cin above 256 a multiple
 * of 32), n, H, W >= 1: else LBPF_EINVAL; LBPF_ECUDA if the launch fails. */
int lbpf_nn_conv3x3_wgrad(const float* x, const float* dy, float* dwt, int n, int H, int W, int cin, int cout,
                          void* stream);
/* *word = the convolution kernels' device error word: 0, or non-zero when a
 * block's bounded wait for its tensor-core work gave up (the block then
 * stops; its outputs are not written).  Synchronises the device first. */
int lbpf_nn_conv_error(int* word);

/* Release every resource of the context (NULL is accepted).  Synchronises
 * the stream first. */
int lbpf_destroy(lbpf_ctx* ctx);

/* Description of the last error on ctx, or of the last error of the calling
 * thread when ctx is NULL (e.g. after a failed lbpf_create).  Never NULL. */
const char* lbpf_last_error(const lbpf_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBPF_H */
