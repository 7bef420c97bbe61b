/*
 * FP64 CPU oracle for the lattice Boltzmann phase-field step of
 * Younsi & Cartalade, "On anisotropy function in crystal growth simulations
 * using Lattice Boltzmann equation" (arXiv:1606.09432).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA path.
 *
 * It is written to be checked against the paper by eye: plain loops over
 * sites and directions, the paper's physical units (dx, dt, W0, tau0, kappa),
 * the paper's order of operations within a time step (Sec. 3.1 for the heat
 * equation, Sec. 3.2 for the phase field, phase field first and heat second),
 * double precision throughout, and no blocking, fusion or reordering.
 *
 * Readings of the paper that this file takes (where the paper is silent or
 * garbled) are marked "Reading:" next to the code they affect.
 *
 * Parity status: every function here is pinned by a CPU test against a
 * closed form, an invariant, a brute-force case or an exact linear
 * propagator, except the tip-position measurement (orc_measure), whose
 * definition is a reading (the paper defines only the tip velocity); that
 * part is "parity unpinned" by the paper and is pinned only by hand-built
 * profiles with known crossings.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXQ 27
#define ORC_MAXC 16

/* Anisotropy function kinds. */
enum {
    ORC_AS_CUBIC100 = 0, /* Eq. (As_Function_Classical): 1 - 3 eps + 4 eps sum n^4          */
    ORC_AS_ANGLE = 1,    /* Eq. (As_Theta): 1 + eps cos(q (varphi - varphi0)), 2D only       */
    ORC_AS_Y66 = 2,      /* Eq. (As_Y66): 1 + eps (nx^6 - 15 nx^4 ny^2 + 15 nx^2 ny^4 - ny^6) */
    ORC_AS_HOYT110 = 3,  /* Eq. (As_MatSci): 1 + eps (Q - 3/5) + gamma (3Q + 66S - 17/7)      */
    ORC_AS_S111 = 4      /* Eq. (As_Function_S), read as 1 + 66 gamma S (see below)          */
};

/* Lattice pairs (phase-field lattice / temperature lattice), Sec. 3.3. */
enum {
    ORC_D2Q9_D2Q5 = 0,
    ORC_D3Q15_D3Q7 = 1,
    ORC_D3Q19_D3Q7 = 2,
    ORC_D3Q27_D3Q7 = 3,
    /* Test lattice: D2Q9 for phi and the xy-projection of D3Q7 for u
     * (w0 = 1/2, w1..4 = 1/8, e^2 = 1/4); used only to check that a z-uniform
     * 3D run reduces exactly to a 2D run. */
    ORC_D2Q9_D2Q5P = 4
};

typedef struct {
    int kind;
    double eps, gamma;
    int q;
    double phi0;
} orc_crystal;

/* Boundary bits (orc_params.bc): a set bit makes both ends of that axis
 * zero-flux walls; a clear bit leaves the axis periodic. */
enum { ORC_WALL_X = 1, ORC_WALL_Y = 2, ORC_WALL_Z = 4 };

typedef struct {
    int lattice;
    int grad; /* 0: directional derivatives (Sec. 4.2), 1: central finite differences */
    int nx, ny, nz;
    int bc;   /* ORC_WALL_* bits; 0 = periodic box */
    double dx, dt, W0, tau0, kappa, lambda, delta, xi;
    int n_crystals;
    orc_crystal crystals[ORC_MAXC];
    /* Advective velocity v of the heat equation (physical units; 0: the
     * pure diffusion of the paper's runs), see heat_equilibrium. */
    double adv[3];
} orc_params;

typedef struct {
    int D, Q;
    int e[ORC_MAXQ][3];
    double w[ORC_MAXQ];
    double e2;
} orc_lattice_t;

/* ------------------------------------------------------------------------- */
/* Lattices (Table 1 and the vectors listed in Sec. 3.3).                      */
/* ------------------------------------------------------------------------- */

static void set_dir(orc_lattice_t* L, int i, int x, int y, int z, double w)
{
    L->e[i][0] = x;
    L->e[i][1] = y;
    L->e[i][2] = z;
    L->w[i] = w;
}

/* D2Q5: e0 = 0, e1 = (1,0), e2 = (0,1), e3 = (-1,0), e4 = (0,-1);
 * w0 = 1/3, w1..4 = 1/6; e^2 = 1/3. */
static void lat_d2q5(orc_lattice_t* L)
{
    L->D = 2;
    L->Q = 5;
    L->e2 = 1.0 / 3.0;
    set_dir(L, 0, 0, 0, 0, 1.0 / 3.0);
    set_dir(L, 1, 1, 0, 0, 1.0 / 6.0);
    set_dir(L, 2, 0, 1, 0, 1.0 / 6.0);
    set_dir(L, 3, -1, 0, 0, 1.0 / 6.0);
    set_dir(L, 4, 0, -1, 0, 1.0 / 6.0);
}

/* Projection of D3Q7 on the xy-plane (test lattice). */
static void lat_d2q5p(orc_lattice_t* L)
{
    L->D = 2;
    L->Q = 5;
    L->e2 = 1.0 / 4.0;
    set_dir(L, 0, 0, 0, 0, 1.0 / 2.0);
    set_dir(L, 1, 1, 0, 0, 1.0 / 8.0);
    set_dir(L, 2, 0, 1, 0, 1.0 / 8.0);
    set_dir(L, 3, -1, 0, 0, 1.0 / 8.0);
    set_dir(L, 4, 0, -1, 0, 1.0 / 8.0);
}

/* D2Q9: D2Q5 directions plus e5 = (1,1), e6 = (-1,1), e7 = (-1,-1),
 * e8 = (1,-1); w0 = 4/9, w1..4 = 1/9, w5..8 = 1/36; e^2 = 1/3. */
static void lat_d2q9(orc_lattice_t* L)
{
    L->D = 2;
    L->Q = 9;
    L->e2 = 1.0 / 3.0;
    set_dir(L, 0, 0, 0, 0, 4.0 / 9.0);
    set_dir(L, 1, 1, 0, 0, 1.0 / 9.0);
    set_dir(L, 2, 0, 1, 0, 1.0 / 9.0);
    set_dir(L, 3, -1, 0, 0, 1.0 / 9.0);
    set_dir(L, 4, 0, -1, 0, 1.0 / 9.0);
    set_dir(L, 5, 1, 1, 0, 1.0 / 36.0);
    set_dir(L, 6, -1, 1, 0, 1.0 / 36.0);
    set_dir(L, 7, -1, -1, 0, 1.0 / 36.0);
    set_dir(L, 8, 1, -1, 0, 1.0 / 36.0);
}

/* D3Q7: e1 = (1,0,0), e2 = (0,1,0), e3 = (-1,0,0), e4 = (0,-1,0),
 * e5 = (0,0,1), e6 = (0,0,-1); w0 = 1/4, w1..6 = 1/8; e^2 = 1/4. */
static void lat_d3q7(orc_lattice_t* L)
{
    L->D = 3;
    L->Q = 7;
    L->e2 = 1.0 / 4.0;
    set_dir(L, 0, 0, 0, 0, 1.0 / 4.0);
    set_dir(L, 1, 1, 0, 0, 1.0 / 8.0);
    set_dir(L, 2, 0, 1, 0, 1.0 / 8.0);
    set_dir(L, 3, -1, 0, 0, 1.0 / 8.0);
    set_dir(L, 4, 0, -1, 0, 1.0 / 8.0);
    set_dir(L, 5, 0, 0, 1, 1.0 / 8.0);
    set_dir(L, 6, 0, 0, -1, 1.0 / 8.0);
}

/* The eight cube diagonals in the paper's D3Q15 order (e7..e14). */
static const int cube_diag[8][3] = {
    {1, 1, 1}, {-1, 1, 1}, {-1, -1, 1}, {1, -1, 1},
    {1, 1, -1}, {-1, 1, -1}, {-1, -1, -1}, {1, -1, -1}};

/* The twelve edge directions (not tabulated by the paper).
 * Reading: xy-edges, then xz-edges, then yz-edges, each in the sign order
 * (+,+), (-,+), (-,-), (+,-). */
static const int cube_edge[12][3] = {
    {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0},
    {1, 0, 1}, {-1, 0, 1}, {-1, 0, -1}, {1, 0, -1},
    {0, 1, 1}, {0, -1, 1}, {0, -1, -1}, {0, 1, -1}};

/* D3Q15: D3Q7 directions plus the cube diagonals; w0 = 2/9, w1..6 = 1/9,
 * w7..14 = 1/72; e^2 = 1/3. */
static void lat_d3q15(orc_lattice_t* L)
{
    lat_d3q7(L);
    L->Q = 15;
    L->e2 = 1.0 / 3.0;
    L->w[0] = 2.0 / 9.0;
    for (int i = 1; i <= 6; ++i) L->w[i] = 1.0 / 9.0;
    for (int k = 0; k < 8; ++k)
        set_dir(L, 7 + k, cube_diag[k][0], cube_diag[k][1], cube_diag[k][2], 1.0 / 72.0);
}

/* D3Q19 (mentioned, not tabulated, by the paper).  Reading: the standard
 * weights w0 = 1/3, w(axis) = 1/18, w(edge) = 1/36; e^2 = 1/3. */
static void lat_d3q19(orc_lattice_t* L)
{
    lat_d3q7(L);
    L->Q = 19;
    L->e2 = 1.0 / 3.0;
    L->w[0] = 1.0 / 3.0;
    for (int i = 1; i <= 6; ++i) L->w[i] = 1.0 / 18.0;
    for (int k = 0; k < 12; ++k)
        set_dir(L, 7 + k, cube_edge[k][0], cube_edge[k][1], cube_edge[k][2], 1.0 / 36.0);
}

/* D3Q27 (mentioned, not tabulated).  Reading: the standard weights
 * w0 = 8/27, w(axis) = 2/27, w(edge) = 1/54, w(corner) = 1/216; e^2 = 1/3. */
static void lat_d3q27(orc_lattice_t* L)
{
    lat_d3q7(L);
    L->Q = 27;
    L->e2 = 1.0 / 3.0;
    L->w[0] = 8.0 / 27.0;
    for (int i = 1; i <= 6; ++i) L->w[i] = 2.0 / 27.0;
    for (int k = 0; k < 12; ++k)
        set_dir(L, 7 + k, cube_edge[k][0], cube_edge[k][1], cube_edge[k][2], 1.0 / 54.0);
    for (int k = 0; k < 8; ++k)
        set_dir(L, 19 + k, cube_diag[k][0], cube_diag[k][1], cube_diag[k][2], 1.0 / 216.0);
}

static int lattice_pair(int lattice, orc_lattice_t* Lg, orc_lattice_t* Lu)
{
    memset(Lg, 0, sizeof(*Lg));
    memset(Lu, 0, sizeof(*Lu));
    switch (lattice) {
    case ORC_D2Q9_D2Q5: lat_d2q9(Lg); lat_d2q5(Lu); return 0;
    case ORC_D3Q15_D3Q7: lat_d3q15(Lg); lat_d3q7(Lu); return 0;
    case ORC_D3Q19_D3Q7: lat_d3q19(Lg); lat_d3q7(Lu); return 0;
    case ORC_D3Q27_D3Q7: lat_d3q27(Lg); lat_d3q7(Lu); return 0;
    case ORC_D2Q9_D2Q5P: lat_d2q9(Lg); lat_d2q5p(Lu); return 0;
    default: return -1;
    }
}

/* Export a lattice table: which = 0 for the phase-field lattice, 1 for the
 * temperature lattice.  e must hold 27*3 ints, w 27 doubles. */
int orc_lattice(int lattice, int which, int* D, int* Q, int* e, double* w, double* e2)
{
    orc_lattice_t Lg, Lu;
    if (lattice_pair(lattice, &Lg, &Lu)) return -1;
    const orc_lattice_t* L = which ? &Lu : &Lg;
    *D = L->D;
    *Q = L->Q;
    *e2 = L->e2;
    for (int i = 0; i < L->Q; ++i) {
        e[3 * i + 0] = L->e[i][0];
        e[3 * i + 1] = L->e[i][1];
        e[3 * i + 2] = L->e[i][2];
        w[i] = L->w[i];
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Grid helpers: periodic wrap, or reflection at zero-flux walls.             */
/* ------------------------------------------------------------------------- */

static int wrap(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

/* Reading (boundary conditions, Sec. 3.3): the paper imposes zero fluxes on
 * all walls for both equations by bounce-back.  A wall is taken as a mirror
 * plane through the boundary nodes: a node at distance k outside the wall is
 * the image of the node at distance k inside it (index -k -> k, and
 * n - 1 + k -> n - 1 - k), so the gradient stencil reads phi of the image
 * there (zero normal derivative), and a population arriving from beyond a
 * wall is the one streamed to the same node in the mirrored direction
 * (fill_walls).  A population streamed out through a wall is discarded, so
 * the non-local term of Eq. (LBE_Eq_Phase) never needs a value beyond the
 * wall.  With these rules an octant run with walls on the symmetry planes is
 * exactly a part of the mirror-symmetric run (Sec. 5.3).  The paper prints
 * the bounce-back with the opposite direction i' (f_i = f_i'); for the axis
 * populations (all of D2Q5 and D3Q7) the mirror and the opposite direction
 * coincide, for diagonal ones only the mirror keeps the wall a symmetry
 * plane. */
static int reflect(int i, int n)
{
    while (i < 0 || i > n - 1) i = (i < 0) ? -i : 2 * (n - 1) - i;
    return i;
}

static int map_axis(const orc_params* p, int axis, int i)
{
    const int n = axis == 0 ? p->nx : (axis == 1 ? p->ny : p->nz);
    return (p->bc & (1 << axis)) ? reflect(i, n) : wrap(i, n);
}

static long site(const orc_params* p, int x, int y, int z)
{
    return ((long)map_axis(p, 2, z) * p->ny + map_axis(p, 1, y)) * p->nx + map_axis(p, 0, x);
}

/* Bit a of the result is set when coordinate a of (x, y, z) lies outside a
 * wall of axis a. */
static int outside_walls(const orc_params* p, int x, int y, int z)
{
    const int c[3] = {x, y, z}, n[3] = {p->nx, p->ny, p->nz};
    int m = 0;
    for (int a = 0; a < 3; ++a)
        if ((p->bc & (1 << a)) && (c[a] < 0 || c[a] > n[a] - 1)) m |= 1 << a;
    return m;
}

/* The direction of lattice L whose velocity is e_i with the components of
 * the axes in `mask` reversed (the mirror image of e_i in those walls). */
static int reflect_dir(const orc_lattice_t* L, int i, int mask)
{
    int t[3];
    for (int a = 0; a < 3; ++a) t[a] = (mask & (1 << a)) ? -L->e[i][a] : L->e[i][a];
    for (int j = 0; j < L->Q; ++j)
        if (L->e[j][0] == t[0] && L->e[j][1] == t[1] && L->e[j][2] == t[2]) return j;
    return -1;
}

/* ------------------------------------------------------------------------- */
/* Gradient of phi (Sec. 4.2).                                                */
/* ------------------------------------------------------------------------- */

/* Physical gradient of phi at (x,y,z).
 * grad = 0: directional derivatives, Eq. (Def_DeriveeDirectionnelle) for
 *   e_i . grad(phi) and Eq. (Grad_DF-Centree) for the gradient:
 *   grad(phi) = (1/e^2) sum_i w_i e_i (e_i . grad(phi)).
 * grad = 1: central finite differences along the coordinate axes. */
static void gradient_at(const orc_params* p, const orc_lattice_t* Lg, const double* phi,
                        int x, int y, int z, double G[3])
{
    G[0] = G[1] = G[2] = 0.0;
    if (p->grad == 0) {
        for (int i = 0; i < Lg->Q; ++i) {
            const int* e = Lg->e[i];
            double dplus = phi[site(p, x + e[0], y + e[1], z + e[2])];
            double dminus = phi[site(p, x - e[0], y - e[1], z - e[2])];
            double ddir = (dplus - dminus) / (2.0 * p->dx); /* e_i . grad(phi) */
            for (int a = 0; a < 3; ++a) G[a] += Lg->w[i] * e[a] * ddir;
        }
        for (int a = 0; a < 3; ++a) G[a] /= Lg->e2;
    } else {
        G[0] = (phi[site(p, x + 1, y, z)] - phi[site(p, x - 1, y, z)]) / (2.0 * p->dx);
        G[1] = (phi[site(p, x, y + 1, z)] - phi[site(p, x, y - 1, z)]) / (2.0 * p->dx);
        if (Lg->D == 3)
            G[2] = (phi[site(p, x, y, z + 1)] - phi[site(p, x, y, z - 1)]) / (2.0 * p->dx);
    }
}

/* Whole-field gradient (physical units), G has 3 entries per site. */
int orc_gradient(const orc_params* p, const double* phi, double* G)
{
    orc_lattice_t Lg, Lu;
    if (lattice_pair(p->lattice, &Lg, &Lu)) return -1;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x)
                gradient_at(p, &Lg, phi, x, y, z, &G[3 * site(p, x, y, z)]);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Anisotropy functions a_s(n) and the vector N (Sec. 2, Sec. 4.1).          */
/* ------------------------------------------------------------------------- */

/* a_s(n) and its partial derivatives da[alpha] = d a_s / d n_alpha, with the
 * components of n treated as independent variables. */
static int as_value(const orc_crystal* c, int D, const double n[3], double* a, double da[3])
{
    const double nx = n[0], ny = n[1], nz = (D == 3) ? n[2] : 0.0;
    const double eps = c->eps, gam = c->gamma;
    double Q, S, dS[3];
    da[0] = da[1] = da[2] = 0.0;
    switch (c->kind) {
    case ORC_AS_CUBIC100:
        /* Eq. (As_Function_Classical) */
        Q = nx * nx * nx * nx + ny * ny * ny * ny + nz * nz * nz * nz;
        *a = 1.0 - 3.0 * eps + 4.0 * eps * Q;
        da[0] = 16.0 * eps * nx * nx * nx;
        da[1] = 16.0 * eps * ny * ny * ny;
        da[2] = 16.0 * eps * nz * nz * nz;
        return 0;
    case ORC_AS_ANGLE: {
        /* Eq. (As_Theta), varphi is the angle of n with the x axis.
         * Reading: varphi = atan2(n_y, n_x) (the quadrant-aware form of
         * tan(varphi) = n_y / n_x), which matters for odd q. */
        if (D != 2) return -1;
        double varphi = atan2(ny, nx);
        double arg = c->q * (varphi - c->phi0);
        *a = 1.0 + eps * cos(arg);
        double da_dvarphi = -eps * c->q * sin(arg);
        double r2 = nx * nx + ny * ny;
        da[0] = da_dvarphi * (-ny / r2);
        da[1] = da_dvarphi * (nx / r2);
        return 0;
    }
    case ORC_AS_Y66: {
        /* Eq. (As_Y66) */
        double x2 = nx * nx, y2 = ny * ny;
        *a = 1.0 + eps * (x2 * x2 * x2 - 15.0 * x2 * x2 * y2 + 15.0 * x2 * y2 * y2 - y2 * y2 * y2);
        da[0] = eps * (6.0 * x2 * x2 * nx - 60.0 * x2 * nx * y2 + 30.0 * nx * y2 * y2);
        da[1] = eps * (-30.0 * x2 * x2 * ny + 60.0 * x2 * y2 * ny - 6.0 * y2 * y2 * ny);
        return 0;
    }
    case ORC_AS_HOYT110:
    case ORC_AS_S111:
        Q = nx * nx * nx * nx + ny * ny * ny * ny + nz * nz * nz * nz;
        S = nx * nx * ny * ny * nz * nz;
        dS[0] = 2.0 * nx * ny * ny * nz * nz;
        dS[1] = 2.0 * ny * nx * nx * nz * nz;
        dS[2] = 2.0 * nz * nx * nx * ny * ny;
        if (c->kind == ORC_AS_HOYT110) {
            /* Eq. (As_MatSci) */
            *a = 1.0 + eps * (Q - 3.0 / 5.0) + gam * (3.0 * Q + 66.0 * S - 17.0 / 7.0);
            da[0] = eps * 4.0 * nx * nx * nx + gam * (12.0 * nx * nx * nx + 66.0 * dS[0]);
            da[1] = eps * 4.0 * ny * ny * ny + gam * (12.0 * ny * ny * ny + 66.0 * dS[1]);
            da[2] = eps * 4.0 * nz * nz * nz + gam * (12.0 * nz * nz * nz + 66.0 * dS[2]);
        } else {
            /* Eq. (As_Function_S) prints a_s = 66 gamma S, which vanishes on
             * the axes and would divide Eq. (LBE_Eq_Phase) by zero.
             * Reading: a_s = 1 + 66 gamma S (the K_{0,0} term plus the S
             * term), which still favours <111>. */
            *a = 1.0 + 66.0 * gam * S;
            da[0] = 66.0 * gam * dS[0];
            da[1] = 66.0 * gam * dS[1];
            da[2] = 66.0 * gam * dS[2];
        }
        return 0;
    default:
        return -1;
    }
}

/* a_s and N for a physical gradient G of phi, Eq. (TermesAnisotropes):
 *   N = |grad phi|^2 a_s (d a_s / d(d_x phi), d a_s / d(d_y phi), d a_s / d(d_z phi)),
 * with n = -grad(phi) / |grad(phi)|, Eq. (Def_Normal_Vector).  The chain rule
 * through n gives d n_b / d(d_a phi) = -(delta_ab - n_a n_b) / |grad phi|.
 * Reading (zero-gradient guard, the paper is silent): where
 * |grad phi| dx <= 1e-10 the normal is undefined (or set by rounding noise,
 * e.g. at symmetry centres of an unsaturated field); there a_s = 1, N = 0. */
int orc_anisotropy(const orc_crystal* c, int D, double dx, const double G[3], double* a, double N[3])
{
    double g2 = G[0] * G[0] + G[1] * G[1] + (D == 3 ? G[2] * G[2] : 0.0);
    N[0] = N[1] = N[2] = 0.0;
    if (g2 * dx * dx <= 1e-20) {
        *a = 1.0;
        return 0;
    }
    double g = sqrt(g2);
    double n[3] = {-G[0] / g, -G[1] / g, D == 3 ? -G[2] / g : 0.0};
    double da[3];
    if (as_value(c, D, n, a, da)) return -1;
    double ndotda = n[0] * da[0] + n[1] * da[1] + n[2] * da[2];
    for (int al = 0; al < D; ++al) {
        double dadG = -(da[al] - n[al] * ndotda) / g; /* d a_s / d(d_al phi) */
        N[al] = g2 * (*a) * dadG;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Simulation state.                                                          */
/* ------------------------------------------------------------------------- */

typedef struct {
    orc_params p;
    orc_lattice_t Lg, Lu;
    long n;
    double *g, *f, *phi, *u;    /* state at time t                          */
    int* I;                     /* crystal index field, 0 = no crystal      */
    double *gnew, *fnew, *phinew;
    double *G, *a, *N;          /* per-site work arrays                     */
    int* Inew;
    long steps;
} orc_state;

static void free_state(orc_state* s)
{
    if (!s) return;
    free(s->g); free(s->f); free(s->phi); free(s->u); free(s->I);
    free(s->gnew); free(s->fnew); free(s->phinew);
    free(s->G); free(s->a); free(s->N); free(s->Inew);
    free(s);
}

void orc_destroy(orc_state* s) { free_state(s); }

orc_state* orc_create(const orc_params* p)
{
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return NULL;
    if (p->n_crystals < 1 || p->n_crystals > ORC_MAXC) return NULL;
    orc_state* s = (orc_state*)calloc(1, sizeof(orc_state));
    if (!s) return NULL;
    s->p = *p;
    if (lattice_pair(p->lattice, &s->Lg, &s->Lu)) { free(s); return NULL; }
    if (s->Lg.D == 2 && p->nz != 1) { free(s); return NULL; }
    s->n = (long)p->nx * p->ny * p->nz;
    long n = s->n;
    s->g = calloc((size_t)n * s->Lg.Q, sizeof(double));
    s->gnew = calloc((size_t)n * s->Lg.Q, sizeof(double));
    s->f = calloc((size_t)n * s->Lu.Q, sizeof(double));
    s->fnew = calloc((size_t)n * s->Lu.Q, sizeof(double));
    s->phi = calloc(n, sizeof(double));
    s->phinew = calloc(n, sizeof(double));
    s->u = calloc(n, sizeof(double));
    s->G = calloc((size_t)3 * n, sizeof(double));
    s->a = calloc(n, sizeof(double));
    s->N = calloc((size_t)3 * n, sizeof(double));
    s->I = calloc(n, sizeof(int));
    s->Inew = calloc(n, sizeof(int));
    if (!s->g || !s->gnew || !s->f || !s->fnew || !s->phi || !s->phinew || !s->u || !s->G ||
        !s->a || !s->N || !s->I || !s->Inew) {
        free_state(s);
        return NULL;
    }
    return s;
}

/* The crystal whose anisotropy applies at a site: with one crystal it holds
 * everywhere; with several, Eq. (As_Multi) selects crystal I - 1 where the
 * index field I is non-zero, and a_s = 1, N = 0 elsewhere (reading). */
static void site_anisotropy(const orc_state* s, int Ival, const double G[3], double* a, double N[3])
{
    const orc_params* p = &s->p;
    if (p->n_crystals == 1) {
        orc_anisotropy(&p->crystals[0], s->Lg.D, p->dx, G, a, N);
    } else if (Ival > 0) {
        orc_anisotropy(&p->crystals[Ival - 1], s->Lg.D, p->dx, G, a, N);
    } else {
        *a = 1.0;
        N[0] = N[1] = N[2] = 0.0;
    }
}

static double grad_norm(const double G[3]) { return sqrt(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]); }

/* Phase-field e.d.f., Eq. (Feq_Phase):
 * g_i^(0) = w_i (phi - (1/e^2) e_i . N (dt/dx) (W0^2/tau0)). */
static double geq_phase(const orc_state* s, int i, double phi, const double N[3])
{
    const orc_params* p = &s->p;
    const int* e = s->Lg.e[i];
    double eN = e[0] * N[0] + e[1] * N[1] + e[2] * N[2];
    return s->Lg.w[i] * (phi - eN / s->Lg.e2 * (p->dt / p->dx) * (p->W0 * p->W0 / p->tau0));
}

/* Temperature e.d.f., Eq. (EqFunction_Tempr), f_i^(0) = w_i u; with an
 * advective velocity v the advection-diffusion form of Sec. 3.1,
 * f_i^(0) = w_i u [1 + e^{-2} e_i . v dt / dx], whose moments are u,
 * v u dt / dx and e^2 u I. */
static double heat_equilibrium(const orc_state* s, int i, double u)
{
    const orc_params* p = &s->p;
    const int* e = s->Lu.e[i];
    const double ev = e[0] * p->adv[0] + e[1] * p->adv[1] + e[2] * p->adv[2];
    return s->Lu.w[i] * u * (1.0 + ev / s->Lu.e2 * p->dt / p->dx);
}

/* Populations from given phi and u fields: g_i = g_i^(0)(phi, N) with N from
 * the gradient of phi, f_i = f_i^(0) (heat_equilibrium).
 * Reading: the paper does not state how the populations are initialised;
 * equilibrium populations are taken, as in the algorithm of Sec. 3.1. */
static void init_populations(orc_state* s)
{
    const orc_params* p = &s->p;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long k = site(p, x, y, z);
                double G[3], a, N[3];
                gradient_at(p, &s->Lg, s->phi, x, y, z, G);
                site_anisotropy(s, s->I[k], G, &a, N);
                for (int i = 0; i < s->Lg.Q; ++i) s->g[(long)i * s->n + k] = geq_phase(s, i, s->phi[k], N);
                for (int i = 0; i < s->Lu.Q; ++i) s->f[(long)i * s->n + k] = heat_equilibrium(s, i, s->u[k]);
            }
    s->steps = 0;
}

/* Minimum-image distance (lattice units) on the periodic box. */
static double periodic_delta(double d, int n)
{
    d = fmod(d, (double)n);
    if (d > 0.5 * n) d -= n;
    if (d < -0.5 * n) d += n;
    return d;
}

/* Seeds, Eq. (Initial_Condition) and Eq. (Intial-Cond_u).
 * seeds holds n_seeds rows (x, y, z, R, crystal), lattice units.
 * Reading: the printed argument (R_s - d_s)/sqrt(2 W0) is read as
 * (R_s - d_s)/(sqrt(2) W0), the equilibrium width of the model; with R, d in
 * lattice units this is (R - d) dx / (sqrt(2) W0).  Several seeds combine by
 * the maximum of their profiles; distances are minimum-image distances on the
 * periodic box (plain distances along walled axes).  The index field starts
 * at I = 1 + crystal of the seed with
 * the largest profile wherever phi > 0 or |grad phi| > xi, and 0 elsewhere. */
int orc_seed(orc_state* s, const double* seeds, int n_seeds)
{
    const orc_params* p = &s->p;
    if (n_seeds < 1) return -1;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long k = site(p, x, y, z);
                double best = -2.0;
                int bestc = 0;
                for (int j = 0; j < n_seeds; ++j) {
                    const double* sd = &seeds[5 * j];
                    /* minimum image along periodic axes, plain distance along walled ones */
                    double ddx = (p->bc & ORC_WALL_X) ? x - sd[0] : periodic_delta(x - sd[0], p->nx);
                    double ddy = (p->bc & ORC_WALL_Y) ? y - sd[1] : periodic_delta(y - sd[1], p->ny);
                    double ddz = (s->Lg.D == 3) ? ((p->bc & ORC_WALL_Z) ? z - sd[2] : periodic_delta(z - sd[2], p->nz))
                                                : 0.0;
                    double d = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
                    double v = tanh((sd[3] - d) * p->dx / (sqrt(2.0) * p->W0));
                    if (v > best) {
                        best = v;
                        bestc = (int)sd[4];
                    }
                }
                s->phi[k] = best;
                s->u[k] = -p->delta; /* u0 = -Delta */
                s->I[k] = bestc + 1;
            }
    /* Index field: keep the seed's index only inside or near the seeds. */
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long k = site(p, x, y, z);
                double G[3];
                gradient_at(p, &s->Lg, s->phi, x, y, z, G);
                s->Inew[k] = (s->phi[k] > 0.0 || grad_norm(G) > p->xi) ? s->I[k] : 0;
            }
    memcpy(s->I, s->Inew, sizeof(int) * s->n);
    if (p->n_crystals == 1)
        for (long k = 0; k < s->n; ++k) s->I[k] = 1;
    init_populations(s);
    return 0;
}

/* Arbitrary phi, u (and optionally I) fields; populations at equilibrium. */
int orc_set_fields(orc_state* s, const double* phi, const double* u, const int* I)
{
    memcpy(s->phi, phi, sizeof(double) * s->n);
    memcpy(s->u, u, sizeof(double) * s->n);
    for (long k = 0; k < s->n; ++k) s->I[k] = (s->p.n_crystals == 1) ? 1 : (I ? I[k] : 0);
    init_populations(s);
    return 0;
}

/* Raw populations (SoA: population i of site k at [i * n + k]). */
int orc_set_populations(orc_state* s, const double* g, const double* f)
{
    memcpy(s->g, g, sizeof(double) * s->n * s->Lg.Q);
    memcpy(s->f, f, sizeof(double) * s->n * s->Lu.Q);
    for (long k = 0; k < s->n; ++k) {
        double ph = 0.0, uu = 0.0;
        for (int i = 0; i < s->Lg.Q; ++i) ph += s->g[(long)i * s->n + k];
        for (int i = 0; i < s->Lu.Q; ++i) uu += s->f[(long)i * s->n + k];
        s->phi[k] = ph;
        s->u[k] = uu;
    }
    return 0;
}

/* Index-field update (Sec. 4.3).  A site whose index is zero and whose
 * gradient exceeds xi takes the index of the nearest site with a non-zero
 * index.  Reading: "nearest" is searched among the phase-field lattice
 * neighbours, shortest |e_i| first, then the lowest direction number (the
 * lattice tables are ordered axis, edge, corner, so this is the first i);
 * the update reads the old field only (Jacobi). */
static int index_update(const orc_state* s, int x, int y, int z, const double G[3])
{
    const orc_params* p = &s->p;
    long k = site(p, x, y, z);
    if (s->I[k] != 0) return s->I[k];
    if (!(grad_norm(G) > p->xi)) return 0;
    for (int i = 1; i < s->Lg.Q; ++i) {
        const int* e = s->Lg.e[i];
        int v = s->I[site(p, x + e[0], y + e[1], z + e[2])];
        if (v != 0) return v;
    }
    return 0;
}

/* After streaming: at every node, each population whose source node lies
 * beyond a wall takes the value of the population streamed to the same node
 * in the direction reflected in that wall (or walls, at edges and corners). */
static void fill_walls(const orc_state* s, const orc_lattice_t* L, double* pop)
{
    const orc_params* p = &s->p;
    const long n = s->n;
    /* each fill reads a population of the same node that is not filled */
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long k = site(p, x, y, z);
                for (int i = 0; i < L->Q; ++i) {
                    const int* e = L->e[i];
                    int out = outside_walls(p, x - e[0], y - e[1], z - e[2]);
                    if (out) pop[(long)i * n + k] = pop[(long)reflect_dir(L, i, out) * n + k];
                }
            }
}

/* One time step: the phase-field scheme (Sec. 3.2) then the heat scheme
 * (Sec. 3.1), in the order the paper prescribes (heat after phase field). */
static void step_once(orc_state* s)
{
    const orc_params* p = &s->p;
    const orc_lattice_t* Lg = &s->Lg;
    const orc_lattice_t* Lu = &s->Lu;
    const long n = s->n;
    const double Dterm = (p->W0 * p->W0 / p->tau0) * (p->dt / (p->dx * p->dx));

    /* (1) gradient, normal, anisotropy, vector N at every node; the index
     * field is updated first so that a_s uses the updated index. */
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long k = site(p, x, y, z);
                double* G = &s->G[3 * k];
                gradient_at(p, Lg, s->phi, x, y, z, G);
                s->Inew[k] = (p->n_crystals == 1) ? 1 : index_update(s, x, y, z, G);
            }
    memcpy(s->I, s->Inew, sizeof(int) * n);
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; ++k) site_anisotropy(s, s->I[k], &s->G[3 * k], &s->a[k], &s->N[3 * k]);

    /* (2) phase-field collision and streaming, Eq. (LBE_Eq_Phase):
     * a_s^2 g_i(x + e_i dx, t + dt) = g_i(x,t) - (1 - a_s^2) g_i(x + e_i dx, t)
     *     - (g_i(x,t) - g_i^(0)(x,t)) / eta_phi + w_i Q_phi dt / tau0,
     * with eta_phi from Eq. (LBE_RelaxationTime) and Q_phi from
     * Eq. (LBE_SourceTerm).  Reading: a_s, N and eta_phi are those of the
     * node x for every occurrence (the paper takes the non-local term
     * explicit in time), and the non-local g_i(x + e_i dx, t) is the
     * population before streaming. */
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long k = site(p, x, y, z);
                double phi = s->phi[k], u = s->u[k], a = s->a[k];
                double a2 = a * a;
                double eta = a2 * Dterm / Lg->e2 + 0.5;
                double Qphi = (phi - p->lambda * u * (1.0 - phi * phi)) * (1.0 - phi * phi);
                for (int i = 0; i < Lg->Q; ++i) {
                    const int* e = Lg->e[i];
                    /* a population streamed beyond a wall leaves the box; the
                     * walls send back its mirror image (fill_walls) */
                    if (outside_walls(p, x + e[0], y + e[1], z + e[2])) continue;
                    long kn = site(p, x + e[0], y + e[1], z + e[2]);
                    double gi = s->g[(long)i * n + k];
                    double gi_next = s->g[(long)i * n + kn];
                    double geq = geq_phase(s, i, phi, &s->N[3 * k]);
                    double rhs = gi - (1.0 - a2) * gi_next - (gi - geq) / eta +
                                 Lg->w[i] * Qphi * p->dt / p->tau0;
                    s->gnew[(long)i * n + kn] = rhs / a2;
                }
            }
    /* Bounce-back at the walls (Sec. 3.3), read as specular reflection: a
     * population whose source node lies beyond a wall is the one streamed to
     * the same node in the reflected direction. */
    if (p->bc) fill_walls(s, Lg, s->gnew);
    /* phi(t + dt), Eq. (Def_M0_Phi) */
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; ++k) {
        double ph = 0.0;
        for (int i = 0; i < Lg->Q; ++i) ph += s->gnew[(long)i * n + k];
        s->phinew[k] = ph;
    }

    /* (3) heat equation, Eq. (LBE_Eq_Temp) with f^(0) = w_i u,
     * Eq. (EqFunction_Tempr) (or its advective form, heat_equilibrium), and
     * Q_u = (1/2) d(phi)/dt, Eq. (Source_Tempr),
     * the time derivative by the explicit Euler difference
     * (phi(t + dt) - phi(t)) / dt of the phase field just computed.
     * eta_u from Eq. (ThermalDiffusivity): kappa = e^2 (eta_u - 1/2) dx^2/dt. */
    const double eta_u = p->kappa * p->dt / (Lu->e2 * p->dx * p->dx) + 0.5;
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long k = site(p, x, y, z);
                double u = s->u[k];
                double Qu = 0.5 * (s->phinew[k] - s->phi[k]) / p->dt;
                for (int i = 0; i < Lu->Q; ++i) {
                    const int* e = Lu->e[i];
                    long kn = site(p, x + e[0], y + e[1], z + e[2]);
                    double fi = s->f[(long)i * n + k];
                    double feq = heat_equilibrium(s, i, u);
                    if (!outside_walls(p, x + e[0], y + e[1], z + e[2])) /* else it leaves the box */
                        s->fnew[(long)i * n + kn] = fi - (fi - feq) / eta_u + Lu->w[i] * Qu * p->dt;
                }
            }
    if (p->bc) fill_walls(s, Lu, s->fnew);
    /* u(t + dt), Eq. (Temperature_LB) */
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; ++k) {
        double uu = 0.0;
        for (int i = 0; i < Lu->Q; ++i) uu += s->fnew[(long)i * n + k];
        s->u[k] = uu;
    }

    double* t;
    t = s->g; s->g = s->gnew; s->gnew = t;
    t = s->f; s->f = s->fnew; s->fnew = t;
    t = s->phi; s->phi = s->phinew; s->phinew = t;
    s->steps += 1;
}

int orc_step(orc_state* s, int nsteps)
{
    for (int k = 0; k < nsteps; ++k) step_once(s);
    return 0;
}

long orc_steps_done(const orc_state* s) { return s->steps; }

int orc_get_fields(const orc_state* s, double* phi, double* u, int* I)
{
    if (phi) memcpy(phi, s->phi, sizeof(double) * s->n);
    if (u) memcpy(u, s->u, sizeof(double) * s->n);
    if (I) memcpy(I, s->I, sizeof(int) * s->n);
    return 0;
}

int orc_get_populations(const orc_state* s, double* g, double* f)
{
    if (g) memcpy(g, s->g, sizeof(double) * s->n * s->Lg.Q);
    if (f) memcpy(f, s->f, sizeof(double) * s->n * s->Lu.Q);
    return 0;
}

/* a_s at every site as used by the last step (computed from the phase
 * field before that step). */
int orc_get_anisotropy(const orc_state* s, double* a)
{
    memcpy(a, s->a, sizeof(double) * s->n);
    return 0;
}

/* a_s at every site of the current phase field (the anisotropy-field
 * pictures of Sec. 4): the normal of Eq. (Def_Normal_Vector) from the
 * gradient of the current phi (Sec. 4.2) and the a_s of the site's crystal
 * for the current index field; a_s = 1 where the index is 0. */
int orc_anisotropy_field(const orc_state* s, double* a)
{
    const orc_params* p = &s->p;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long k = site(p, x, y, z);
                double G[3], N[3];
                gradient_at(p, &s->Lg, s->phi, x, y, z, G);
                site_anisotropy(s, s->I[k], G, &a[k], N);
            }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Measurements.                                                              */
/* ------------------------------------------------------------------------- */

/* Tip position along one axis direction from the integer site c.
 * The paper defines only the tip velocity V_p (Sec. 3.4).  Reading: the tip
 * is the outermost crossing phi = 0 on the ray c + k d, k = 0 .. n/2 - 1
 * (up to the wall on a walled axis),
 * located by linear interpolation, x_tip = k + phi_k / (phi_k - phi_{k+1});
 * -1 when the ray has no crossing. */
static double tip_along(const orc_state* s, const int c[3], int axis, int sign)
{
    const orc_params* p = &s->p;
    const int na = axis == 0 ? p->nx : axis == 1 ? p->ny : p->nz;
    /* half the box on a periodic axis; up to the wall on a walled one */
    int len = (p->bc & (1 << axis)) ? (sign > 0 ? na - 1 - c[axis] : c[axis]) : na / 2;
    double tip = -1.0;
    for (int k = 0; k + 1 <= len; ++k) {
        int a0[3] = {c[0], c[1], c[2]}, a1[3] = {c[0], c[1], c[2]};
        a0[axis] += sign * k;
        a1[axis] += sign * (k + 1);
        double p0 = s->phi[site(p, a0[0], a0[1], a0[2])];
        double p1 = s->phi[site(p, a1[0], a1[1], a1[2])];
        if (p0 >= 0.0 && p1 < 0.0) tip = k + p0 / (p0 - p1);
    }
    return tip;
}

/* tip6: +x, -x, +y, -y, +z, -z tip distances from the centre site (the z
 * entries are -1 in 2D); solid_fraction = mean of (1 + phi)/2;
 * conserved = sum over sites of (u - phi/2), which the scheme keeps constant
 * in a periodic or closed box (integral of Eq. (Temp_Ramirez) with zero
 * flux); nodes on walls count 1/2 per walled coordinate (they lie on the
 * mirror planes). */
int orc_measure(const orc_state* s, int cx, int cy, int cz, double* tip6, double* solid_fraction,
                double* conserved)
{
    int c[3] = {cx, cy, cz};
    for (int a = 0; a < 3; ++a) {
        if (a == 2 && s->Lg.D == 2) {
            tip6[4] = tip6[5] = -1.0;
            continue;
        }
        tip6[2 * a] = tip_along(s, c, a, +1);
        tip6[2 * a + 1] = tip_along(s, c, a, -1);
    }
    double sf = 0.0, cs = 0.0;
    const orc_params* p = &s->p;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long k = site(p, x, y, z);
                /* a node on a wall is shared with its mirror image: weight
                 * 1/2 per walled coordinate at a wall (the trapezoid rule) */
                double wgt = 1.0;
                if ((p->bc & ORC_WALL_X) && (x == 0 || x == p->nx - 1)) wgt *= 0.5;
                if ((p->bc & ORC_WALL_Y) && (y == 0 || y == p->ny - 1)) wgt *= 0.5;
                if ((p->bc & ORC_WALL_Z) && s->Lg.D == 3 && (z == 0 || z == p->nz - 1)) wgt *= 0.5;
                sf += 0.5 * (1.0 + s->phi[k]);
                cs += wgt * (s->u[k] - 0.5 * s->phi[k]);
            }
    *solid_fraction = sf / (double)s->n;
    *conserved = cs;
    return 0;
}
