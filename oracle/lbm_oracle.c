/*
 * lbm_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Bogner & Ruede, "Liquid-gas-solid flows with lattice Boltzmann: Simulation
 * of floating bodies".  One time step, in the paper's order:
 *
 *   C4  momentum exchange on every body link at time t      (Sec. 2.3 Eqs.
 *       momentumexchange, netforce, torque; Sec. 2.4 Eq. momentuminterface)
 *   C1  stream with obstacle bounce-back (Eq. noslip), atmosphere
 *       reconstruction (Eq. reconstruct) and interface mass exchange (Sec. 2.2)
 *   C2  BGK collision with the gravity force term (Eqs. lbgk, equilibrium,
 *       forceterm, density, momentum)
 *   C3  free-surface cell conversions (Sec. 2.2, last paragraph)
 *   C5  rigid-body update (the rigid-body engine of Sec. 2.3)
 *   C6  obstacle remapping with the obstacle-to-fluid rule (Sec. 2.3 body
 *       discretisation; Sec. 2.4 rule over B(x))
 *   C7  invariants: closed interface layer and the mass ledger
 *
 * Readings where the paper is silent, garbled or ambiguous are fixed once and
 * implemented identically by the GPU library (which shares no code with this
 * file): relaxation sign and the Luo force with a c_i factor (Eq. lbgk and
 * Eq. forceterm are garbled), the cell's own density in the moving-wall term,
 * u_w at the link midpoint, the anti-bounce-back of the cell's own outgoing
 * population in Eq. reconstruct, a central-difference normal with
 * c.n < -deadband (default 1e-2, a dead band against noise; 0 gives the bare
 * sign test), eps = 1e-2, Jacobi-style conversions with equal excess-mass
 * split, and the obstacle-to-fluid priority interface > liquid > gas.  The
 * readings that are options (dead band, the neighbour conversion rule, the
 * virtual-mass coefficient and the two-step force mean of the rigid-body
 * update) are set per simulation with orc_set_readings().
 *
 * Floating-point expression order is written out explicitly (left to right,
 * q in the order C,W,E,N,S,T,B,TW,TE,TN,TS,NW,NE,SW,SE,BW,BE,BN,BS of the
 * paper's D3Q19 figure caption) and the file is compiled with
 * -ffp-contract=off, so every operation is a single IEEE-754 rounding.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q 19
enum { LIQ = 1, IFC = 2, GAS = 4, OBS = 8, WALL = 256 };
enum { M_FIXED = 0, M_FREE = 1, M_ROT_AXIS = 2, M_DAMP = 0x100 };
/* Eq. reconstruct selects the directions with c_q . n <= 0.  A direction
 * tangential to a flat surface has c_q . n = 0 up to noise (rounding, storage
 * precision), and a bare sign test turns that noise into a discontinuous
 * reconstruct / stream decision; by default directions count as pointing out
 * of the gas only when c_q . n < -1e-2, i.e. when the fill level changes by
 * more than 2e-2 across the cell (orc_set_readings changes it; 0 is the
 * strict sign test c_q . n < 0). */
#define DEFAULT_DEADBAND 1e-2

/* D3Q19 velocities in the order of the paper's stencil figure. */
static const int C[Q][3] = {
    {0, 0, 0},                                                      /* C */
    {-1, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}, /* W E N S T B */
    {-1, 0, 1}, {1, 0, 1}, {0, 1, 1}, {0, -1, 1},                   /* TW TE TN TS */
    {-1, 1, 0}, {1, 1, 0}, {-1, -1, 0}, {1, -1, 0},                 /* NW NE SW SE */
    {-1, 0, -1}, {1, 0, -1}, {0, 1, -1}, {0, -1, -1}};              /* BW BE BN BS */
static double W[Q];
static int OPP[Q];
static int g_mutation = 0;

static void init_lattice(void) {
    static int done = 0;
    if (done) return;
    for (int q = 0; q < Q; ++q) {
        int s = abs(C[q][0]) + abs(C[q][1]) + abs(C[q][2]);
        W[q] = s == 0 ? 1.0 / 3.0 : (s == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        for (int p = 0; p < Q; ++p)
            if (C[p][0] == -C[q][0] && C[p][1] == -C[q][1] && C[p][2] == -C[q][2]) OPP[q] = p;
    }
    done = 1;
}

typedef struct {
    double o[3], h[3], q[4], dens, v[3], w[3];
    int mode;
    double axis[3], damp;
    double F[3], T[3], S;
    unsigned __int128 acc[7]; /* fixed-point sums of F, T, S (orc_compute_forces) */
    double dv[3], dw[3]; /* last velocity / angular-velocity increments (virtual mass) */
    double Fp[3], Tp[3]; /* the previous step's force and torque */
    int nF;              /* 1 once Fp, Tp hold a step */
    int shape;           /* 0: box of half extents h; 1: sphere of radius h[0] */
} body_t;

/* default virtual-mass coefficient of the rigid-body update (Schwarz, Kempe
 * and Froehlich, J. Comput. Phys. 281 (2015)) */
#define DEFAULT_VIRTUAL_MASS 1.0

struct orc_sim {
    int nx, ny, nz;
    unsigned periodic;
    long n;
    double tau, grav[3], a[3], rho_g, eps;
    double sigma; /* surface tension (0: none) */
    double wall_vel[6][3]; /* velocity of the faces x-, x+, y-, y+, z-, z+ (non-periodic) */
    uint8_t *flag;
    int *body;
    double *f, *fn;     /* [idx*19 + q] at t and t+1 */
    double *phi, *phin; /* fill level at t and t+1 (interface cells) */
    double *m, *mn;     /* interface mass at t and t+1 */
    int nb, cap;
    body_t *b;
    double covered, uncovered, lost, M0;
    double wall; /* mass added to liquid cells by the moving-wall term of Eq. noslip */
    int have_m0, err;
    long t;
    long counts[6];
    /* readings (orc_set_readings) */
    double deadband;     /* Eq. reconstruct: c.n < -deadband selects a direction */
    double vmass;        /* virtual-mass coefficient C of the rigid-body update */
    int force_mean;      /* 1: the update is driven by (F_n + F_{n-1}) / 2; 0: by F_n */
    int nb_rule;         /* 1: interface cells without liquid (gas) neighbours empty (fill) */
};

/* ---------------------------------------------------------------- helpers */

static long cell_index(const orc_sim *s, int x, int y, int z) {
    return (long)x + (long)s->nx * ((long)y + (long)s->ny * (long)z);
}

/* neighbour of (x,y,z) at offset d; -1 when it lies beyond a wall face */
static long neighbour(const orc_sim *s, int x, int y, int z, int dx, int dy, int dz) {
    int p[3] = {x + dx, y + dy, z + dz};
    int nn[3] = {s->nx, s->ny, s->nz};
    for (int k = 0; k < 3; ++k) {
        if (p[k] < 0 || p[k] >= nn[k]) {
            if (!(s->periodic & (1u << k))) return -1;
            p[k] = (p[k] + nn[k]) % nn[k];
        }
    }
    return cell_index(s, p[0], p[1], p[2]);
}

static int class_of(const orc_sim *s, long idx) { return idx < 0 ? WALL : s->flag[idx]; }

static double min_image(const orc_sim *s, double d, int k) {
    if (s->periodic & (1u << k)) {
        double n = k == 0 ? s->nx : (k == 1 ? s->ny : s->nz);
        d = d - n * floor(d / n + 0.5);
    }
    return d;
}

/* Eq. equilibrium with c_s^2 = 1/3: rho w [1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u] */
static double feq(int q, double rho, const double u[3]) {
    double cu = (C[q][0] * u[0] + C[q][1] * u[1]) + C[q][2] * u[2];
    double usq = (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2];
    double t = ((1.0 + 3.0 * cu) + (4.5 * cu) * cu) - 1.5 * usq;
    return (W[q] * rho) * t;
}

/* Eq. forceterm (Luo): w rho [ (c - u)/c_s^2 + (c.u) c / c_s^4 ] . a */
static double force_term(int q, double rho, const double u[3], const double a[3]) {
    double cu = (C[q][0] * u[0] + C[q][1] * u[1]) + C[q][2] * u[2];
    double tx = (3.0 * (C[q][0] - u[0]) + (9.0 * cu) * C[q][0]) * a[0];
    double ty = (3.0 * (C[q][1] - u[1]) + (9.0 * cu) * C[q][1]) * a[1];
    double tz = (3.0 * (C[q][2] - u[2]) + (9.0 * cu) * C[q][2]) * a[2];
    if (g_mutation == 3) tz = (3.0 * (C[q][2] - u[2])) * a[2];
    return (W[q] * rho) * ((tx + ty) + tz);
}

static double density(const double *fc) {
    double r = 0.0;
    for (int q = 0; q < Q; ++q) r += fc[q];
    return r;
}

static void momentum(const double *fc, double j[3]) {
    j[0] = j[1] = j[2] = 0.0;
    for (int q = 0; q < Q; ++q) {
        j[0] += C[q][0] * fc[q];
        j[1] += C[q][1] * fc[q];
        j[2] += C[q][2] * fc[q];
    }
}

/* velocity recovered from post-collision populations: sum c f / rho - a */
static void velocity_after_collision(const orc_sim *s, const double *fc, double rho, double u[3]) {
    double j[3];
    momentum(fc, j);
    for (int k = 0; k < 3; ++k) u[k] = j[k] / rho - s->a[k];
}

/* rotation matrix of the unit quaternion (w, x, y, z) */
static void rotation(const double q[4], double R[3][3]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1.0 - 2.0 * (y * y + z * z);
    R[0][1] = 2.0 * (x * y - w * z);
    R[0][2] = 2.0 * (x * z + w * y);
    R[1][0] = 2.0 * (x * y + w * z);
    R[1][1] = 1.0 - 2.0 * (x * x + z * z);
    R[1][2] = 2.0 * (y * z - w * x);
    R[2][0] = 2.0 * (x * z - w * y);
    R[2][1] = 2.0 * (y * z + w * x);
    R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

/* Sec. 2.3: a cell is an obstacle iff its centre lies inside the body (a box,
 * or a sphere of radius h[0]). */
static int inside(const orc_sim *s, const body_t *b, int x, int y, int z) {
    double R[3][3];
    rotation(b->q, R);
    double d[3] = {min_image(s, (x + 0.5) - b->o[0], 0), min_image(s, (y + 0.5) - b->o[1], 1),
                   min_image(s, (z + 0.5) - b->o[2], 2)};
    if (b->shape == 1) return ((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]) < b->h[0] * b->h[0];
    for (int k = 0; k < 3; ++k) {
        double bk = (R[0][k] * d[0] + R[1][k] * d[1]) + R[2][k] * d[2];
        if (!(fabs(bk) < b->h[k])) return 0;
    }
    return 1;
}

/* rigid-body velocity v + omega x (p - o) at the point p */
static void body_velocity_at(const orc_sim *s, const body_t *b, const double p[3], double uw[3]) {
    double r[3];
    for (int k = 0; k < 3; ++k) r[k] = min_image(s, p[k] - b->o[k], k);
    double cx = b->w[1] * r[2] - b->w[2] * r[1];
    double cy = b->w[2] * r[0] - b->w[0] * r[2];
    double cz = b->w[0] * r[1] - b->w[1] * r[0];
    uw[0] = b->v[0] + cx;
    uw[1] = b->v[1] + cy;
    uw[2] = b->v[2] + cz;
}

/* wall velocity for the link from cell (x,y,z) in direction c_qbar, taken at
 * the link midpoint x_c + c_qbar / 2 */
static void link_wall_velocity(const orc_sim *s, const body_t *b, int x, int y, int z, int q, double uw[3]) {
    int qb = OPP[q];
    double p[3] = {(x + 0.5) + 0.5 * C[qb][0], (y + 0.5) + 0.5 * C[qb][1], (z + 0.5) + 0.5 * C[qb][2]};
    body_velocity_at(s, b, p, uw);
}

/* Eq. noslip at a domain wall: the velocity of the wall face that the link
 * (x, q) crosses (source x - c_q beyond the grid); a link across an edge takes
 * the face of the lowest such axis. */
static void wall_face_velocity(const orc_sim *s, int x, int y, int z, int q, double uw[3]) {
    int p[3] = {x - C[q][0], y - C[q][1], z - C[q][2]};
    int nn[3] = {s->nx, s->ny, s->nz};
    for (int k = 0; k < 3; ++k) {
        if (s->periodic & (1u << k)) continue;
        int face = p[k] < 0 ? 2 * k : (p[k] >= nn[k] ? 2 * k + 1 : -1);
        if (face < 0) continue;
        for (int j = 0; j < 3; ++j) uw[j] = s->wall_vel[face][j];
        return;
    }
}

/* fill level as seen by the normal estimate of an interface cell */
static double fill_seen(const orc_sim *s, long nidx, double own) {
    int c = class_of(s, nidx);
    if (c == LIQ) return 1.0;
    if (c == IFC) return s->phi[nidx];
    if (c == GAS) return 0.0;
    return own; /* obstacle or outside: zero gradient */
}

/* fill level of a cell as seen by its own normal estimate: 1 / phi / 0 */
static double fill_own(const orc_sim *s, long idx) {
    int c = s->flag[idx];
    return c == LIQ ? 1.0 : (c == IFC ? s->phi[idx] : 0.0);
}

/* unit vector of n (zero when n = 0) */
static void unit_vector(const double n[3], double out[3]) {
    double len = sqrt((n[0] * n[0] + n[1] * n[1]) + n[2] * n[2]);
    for (int k = 0; k < 3; ++k) out[k] = len > 0.0 ? n[k] / len : 0.0;
}

/* Sec. 2.2 Laplace pressure: the mean curvature kappa = div(n^)/2 of the
 * interface at cell (x,y,z), from the unit normals n^ = -grad(phi)/|grad phi|
 * (the normals of R6, with the same fill-level rules) of its six axis
 * neighbours by central differences; a neighbour that is an obstacle or lies
 * beyond a wall takes the cell's own unit normal nc.  A liquid sphere of
 * radius R has kappa = 1/R. */
static double curvature(const orc_sim *s, int x, int y, int z, const double nc[3]) {
    double div = 0.0;
    for (int k = 0; k < 3; ++k) {
        double comp[2];
        for (int sgn = 0; sgn < 2; ++sgn) {
            int e[3] = {0, 0, 0};
            e[k] = sgn ? -1 : 1;
            long yi = neighbour(s, x, y, z, e[0], e[1], e[2]);
            int c = class_of(s, yi);
            if (c == WALL || c == OBS) {
                comp[sgn] = nc[k];
                continue;
            }
            int yx = (int)(yi % s->nx), yy = (int)((yi / s->nx) % s->ny), yz = (int)(yi / ((long)s->nx * s->ny));
            double own = fill_own(s, yi), n[3], nh[3];
            for (int j = 0; j < 3; ++j) {
                int f[3] = {0, 0, 0};
                f[j] = 1;
                double pm = fill_seen(s, neighbour(s, yx, yy, yz, -f[0], -f[1], -f[2]), own);
                double pp = fill_seen(s, neighbour(s, yx, yy, yz, f[0], f[1], f[2]), own);
                n[j] = 0.5 * (pm - pp);
            }
            unit_vector(n, nh);
            comp[sgn] = nh[k];
        }
        div += comp[0] - comp[1];
    }
    return 0.25 * div;
}

static double liquid_mass(const orc_sim *s) {
    double M = 0.0;
    for (long i = 0; i < s->n; ++i) {
        if (s->flag[i] == LIQ) M += density(s->f + i * Q);
        else if (s->flag[i] == IFC) M += s->m[i];
    }
    return M;
}

/* ------------------------------------------------------------- lifecycle */

orc_sim *orc_create(int nx, int ny, int nz, unsigned periodic, double tau, const double gravity[3],
                    const double body_accel[3], double rho_gas, double eps, const uint8_t *flags,
                    const double *fill, const double *rho, const double *vel) {
    init_lattice();
    if (nx <= 0 || ny <= 0 || nz <= 0 || !(tau > 0.5)) return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->nx = nx; s->ny = ny; s->nz = nz;
    s->periodic = periodic;
    s->n = (long)nx * ny * nz;
    s->tau = tau;
    for (int k = 0; k < 3; ++k) {
        s->grav[k] = gravity[k];
        s->a[k] = gravity[k] + body_accel[k];
    }
    s->rho_g = rho_gas;
    s->eps = eps;
    s->deadband = DEFAULT_DEADBAND;
    s->vmass = DEFAULT_VIRTUAL_MASS;
    s->force_mean = 1;
    s->nb_rule = 1;
    s->flag = (uint8_t *)calloc(s->n, 1);
    s->body = (int *)calloc(s->n, sizeof(int));
    s->f = (double *)calloc(s->n * Q, sizeof(double));
    s->fn = (double *)calloc(s->n * Q, sizeof(double));
    s->phi = (double *)calloc(s->n, sizeof(double));
    s->phin = (double *)calloc(s->n, sizeof(double));
    s->m = (double *)calloc(s->n, sizeof(double));
    s->mn = (double *)calloc(s->n, sizeof(double));
    double zero[3] = {0.0, 0.0, 0.0};
    for (long i = 0; i < s->n; ++i) {
        int c = flags[i];
        if (c != LIQ && c != IFC && c != GAS) { s->err |= ORC_ERR_BAD_INPUT; c = GAS; }
        s->flag[i] = (uint8_t)c;
        s->body[i] = -1;
        if (c == GAS) continue;
        /* f = f_eq(rho, u) with u = 0 unless a velocity field is given */
        const double *u0 = vel ? vel + 3 * i : zero;
        for (int q = 0; q < Q; ++q) s->f[i * Q + q] = feq(q, rho[i], u0);
        double r = density(s->f + i * Q);
        if (c == IFC) {
            s->m[i] = fill[i] * r;
            s->phi[i] = s->m[i] / r;
        }
    }
    return s;
}

void orc_destroy(orc_sim *s) {
    if (!s) return;
    free(s->flag); free(s->body); free(s->f); free(s->fn);
    free(s->phi); free(s->phin); free(s->m); free(s->mn); free(s->b);
    free(s);
}

int orc_add_box(orc_sim *s, const double center[3], const double half[3], const double quat[4],
                double density_ratio, const double vel[3], const double omega[3], int mode,
                const double rot_axis[3], double lin_damping, int shape) {
    if (s->nb == s->cap) {
        s->cap = s->cap ? 2 * s->cap : 4;
        s->b = (body_t *)realloc(s->b, s->cap * sizeof(body_t));
    }
    body_t *b = &s->b[s->nb];
    memset(b, 0, sizeof(*b));
    for (int k = 0; k < 3; ++k) {
        b->o[k] = center[k]; b->h[k] = half[k]; b->v[k] = vel[k]; b->w[k] = omega[k];
        b->axis[k] = rot_axis[k];
    }
    for (int k = 0; k < 4; ++k) b->q[k] = quat[k];
    b->dens = density_ratio;
    b->mode = mode;
    b->damp = lin_damping;
    b->shape = shape;
    int id = s->nb++;
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long i = cell_index(s, x, y, z);
                if (s->flag[i] == OBS || !inside(s, b, x, y, z)) continue;
                if (s->have_m0) {
                    if (s->flag[i] == LIQ) s->covered += density(s->f + i * Q);
                    else if (s->flag[i] == IFC) s->covered += s->m[i];
                }
                s->flag[i] = OBS;
                s->body[i] = id;
            }
    return id;
}

/* ------------------------------------------------------------------ C4 */

/* The sums of Eqs. netforce and torque evaluated exactly: every term t
 * (|t| < 2^31) is written as the integer floor(t 2^96) -- its bits below 2^-96
 * dropped -- and the integers are added (two's complement, 128 bits), so the
 * sum does not depend on the order of the terms; the total v = H 2^64 + L
 * (H signed, L unsigned) is returned as H 2^-32 + L 2^-96 in double. */
static unsigned __int128 fixed96(double t) {
    double sc = t * 4294967296.0; /* t 2^32, exact */
    double hf = floor(sc);
    long long hi = (long long)hf;
    unsigned long long lo = (unsigned long long)((sc - hf) * 18446744073709551616.0);
    return ((unsigned __int128)(unsigned long long)hi << 64) | (unsigned __int128)lo;
}

static double fixed96_value(unsigned __int128 v) {
    long long H = (long long)(unsigned long long)(v >> 64);
    unsigned long long L = (unsigned long long)v;
    return (double)H * 2.3283064365386962890625e-10 + (double)L * 1.2621774483536188886587657044524580e-29;
}

/* Momentum exchange (Eqs. momentumexchange, momentuminterface) summed over
 * the links of every non-obstacle cell into a body, and the torque about the
 * body centre with the lever arm from the centre of the cell (Eq. torque).
 * Force on the body = -(momentum gained by the fluid): c_qbar * 2(...).  The
 * sums are exact (fixed96). */
void orc_compute_forces(orc_sim *s) {
    init_lattice();
    for (int bi = 0; bi < s->nb; ++bi) {
        body_t *b = &s->b[bi];
        for (int k = 0; k < 7; ++k) b->acc[k] = 0;
    }
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long i = cell_index(s, x, y, z);
                int cl = s->flag[i];
                if (cl == OBS) continue;
                double phi_x = cl == LIQ ? 1.0 : (cl == IFC ? s->phi[i] : 0.0);
                double rho_x = cl == GAS ? 0.0 : density(s->f + i * Q);
                for (int q = 1; q < Q; ++q) {
                    long si = neighbour(s, x, y, z, -C[q][0], -C[q][1], -C[q][2]);
                    if (si < 0 || s->flag[si] != OBS) continue;
                    body_t *b = &s->b[s->body[si]];
                    double uw[3];
                    link_wall_velocity(s, b, x, y, z, q, uw);
                    double cuw = (C[q][0] * uw[0] + C[q][1] * uw[1]) + C[q][2] * uw[2];
                    int qb = OPP[q];
                    double inner;
                    if (cl == GAS) {
                        inner = W[q] * s->rho_g;
                    } else {
                        double A = phi_x * s->f[i * Q + qb];
                        double B = (1.0 - phi_x) * (W[q] * s->rho_g);
                        double Cc = phi_x * (((3.0 * W[q]) * rho_x) * cuw);
                        if (g_mutation == 4) B = 0.0;
                        inner = (A + B) + Cc;
                    }
                    double g = 2.0 * inner;
                    if (g_mutation == 1) g = -g;
                    double Fl[3] = {C[qb][0] * g, C[qb][1] * g, C[qb][2] * g};
                    double r[3] = {min_image(s, (x + 0.5) - b->o[0], 0), min_image(s, (y + 0.5) - b->o[1], 1),
                                   min_image(s, (z + 0.5) - b->o[2], 2)};
                    b->acc[0] += fixed96(Fl[0]);
                    b->acc[1] += fixed96(Fl[1]);
                    b->acc[2] += fixed96(Fl[2]);
                    b->acc[3] += fixed96(r[1] * Fl[2] - r[2] * Fl[1]);
                    b->acc[4] += fixed96(r[2] * Fl[0] - r[0] * Fl[2]);
                    b->acc[5] += fixed96(r[0] * Fl[1] - r[1] * Fl[0]);
                    b->acc[6] += fixed96(fabs(g));
                }
            }
    for (int bi = 0; bi < s->nb; ++bi) {
        body_t *b = &s->b[bi];
        for (int k = 0; k < 3; ++k) {
            b->F[k] = fixed96_value(b->acc[k]);
            b->T[k] = fixed96_value(b->acc[3 + k]);
        }
        b->S = fixed96_value(b->acc[6]);
    }
}

/* ------------------------------------------------------------- C1 + C2 */

/* Stream (Eq. stream) with boundary handling, then collide (Eq. lbgk); writes
 * fn, mn, phin for every liquid and interface cell. */
static void stream_collide(orc_sim *s) {
    const double omega = 1.0 / s->tau;
    memcpy(s->mn, s->m, s->n * sizeof(double));
    memcpy(s->phin, s->phi, s->n * sizeof(double));
    memset(s->fn, 0, s->n * Q * sizeof(double));
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long i = cell_index(s, x, y, z);
                int cl = s->flag[i];
                if (cl != LIQ && cl != IFC) continue;
                const double *fo = s->f + i * Q; /* own post-collision populations at t */
                double rho_x = density(fo);
                double ux[3] = {0.0, 0.0, 0.0};
                if (cl == IFC) velocity_after_collision(s, fo, rho_x, ux);
                long src[Q];
                int scl[Q];
                double fp[Q];
                fp[0] = fo[0];
                /* interface cells: normal n = -grad(phi) by central differences
                 * (R6) and the gas density of the boundary condition, raised
                 * by the Laplace pressure 2 sigma kappa (p = rho / 3) */
                double n[3] = {0.0, 0.0, 0.0};
                double rg = s->rho_g;
                if (cl == IFC) {
                    double own = s->phi[i];
                    for (int k = 0; k < 3; ++k) {
                        int e[3] = {0, 0, 0};
                        e[k] = 1;
                        double pm = fill_seen(s, neighbour(s, x, y, z, -e[0], -e[1], -e[2]), own);
                        double pp = fill_seen(s, neighbour(s, x, y, z, e[0], e[1], e[2]), own);
                        n[k] = g_mutation == 7 ? 0.5 * (pp - pm) : 0.5 * (pm - pp);
                    }
                    if (s->sigma != 0.0) {
                        double nc[3];
                        unit_vector(n, nc);
                        double kappa = curvature(s, x, y, z, nc);
                        if (g_mutation == 8) kappa = -kappa;
                        rg = s->rho_g + (6.0 * s->sigma) * kappa;
                    }
                }
                /* C1: stream with bounce-back / reconstruction */
                for (int q = 1; q < Q; ++q) {
                    int qb = OPP[q];
                    src[q] = neighbour(s, x, y, z, -C[q][0], -C[q][1], -C[q][2]);
                    scl[q] = class_of(s, src[q]);
                    if (scl[q] == WALL || scl[q] == OBS) {
                        /* Eq. noslip: f'_q = f*_qbar + 2/c_s^2 w_q rho (c_q.u_w) */
                        double uw[3] = {0.0, 0.0, 0.0};
                        if (scl[q] == OBS) link_wall_velocity(s, &s->b[s->body[src[q]]], x, y, z, q, uw);
                        else wall_face_velocity(s, x, y, z, q, uw);
                        double cuw = (C[q][0] * uw[0] + C[q][1] * uw[1]) + C[q][2] * uw[2];
                        double src_term = ((6.0 * W[q]) * rho_x) * cuw;
                        fp[q] = (g_mutation == 6 ? fo[q] : fo[qb]) + src_term;
                        if (cl == LIQ) s->wall += src_term;
                    } else if (scl[q] == GAS) {
                        if (cl == LIQ) {
                            s->err |= ORC_ERR_LIQUID_GAS_ADJ;
                            fp[q] = fo[qb];
                        } else {
                            /* Eq. reconstruct with the cell's own outgoing population */
                            fp[q] = (feq(q, rg, ux) + feq(qb, rg, ux)) - fo[qb];
                        }
                    } else {
                        fp[q] = s->f[src[q] * Q + q];
                    }
                }
                if (cl == IFC) {
                    for (int q = 1; q < Q; ++q) {
                        double cn = (C[q][0] * n[0] + C[q][1] * n[1]) + C[q][2] * n[2];
                        if (cn < -s->deadband && scl[q] != OBS && scl[q] != WALL) {
                            int qb = OPP[q];
                            fp[q] = (feq(q, rg, ux) + feq(qb, rg, ux)) - fo[qb];
                        }
                    }
                    /* Sec. 2.2 mass exchange with the neighbour y = x + c_q */
                    double dm = 0.0;
                    for (int q = 1; q < Q; ++q) {
                        int qb = OPP[q];
                        long yi = neighbour(s, x, y, z, C[q][0], C[q][1], C[q][2]);
                        int ycl = class_of(s, yi);
                        if (ycl == LIQ) {
                            if (g_mutation == 2) dm += fo[q] - s->f[yi * Q + qb];
                            else dm += s->f[yi * Q + qb] - fo[q];
                        } else if (ycl == IFC) {
                            double wgt = 0.5 * (s->phi[i] + s->phi[yi]);
                            dm += wgt * (s->f[yi * Q + qb] - fo[q]);
                        }
                    }
                    s->mn[i] = s->m[i] + dm;
                }
                /* C2: BGK collision with the force term */
                double rho = 0.0, j[3] = {0.0, 0.0, 0.0}, u[3];
                for (int q = 0; q < Q; ++q) rho += fp[q];
                for (int q = 0; q < Q; ++q) {
                    j[0] += C[q][0] * fp[q];
                    j[1] += C[q][1] * fp[q];
                    j[2] += C[q][2] * fp[q];
                }
                for (int k = 0; k < 3; ++k) u[k] = j[k] / rho;
                double *fnew = s->fn + i * Q;
                for (int q = 0; q < Q; ++q) {
                    double fe = feq(q, rho, u);
                    double fq = force_term(q, rho, u, s->a);
                    if (g_mutation == 5) fq = -fq;
                    fnew[q] = (fp[q] - omega * (fp[q] - fe)) + fq;
                }
                if (cl == IFC) s->phin[i] = s->mn[i] / density(fnew);
            }
}

/* ------------------------------------------------------------------ C3 */

enum { CV_FILLED = 1, CV_EMPTIED = 2, CV_NEW_FROM_GAS = 4, CV_NEW_FROM_LIQ = 8 };

/* Sec. 2.2 conversions: interface cells with phi >= 1 + eps fill, with
 * phi <= -eps empty; gas neighbours of filled cells and liquid neighbours of
 * emptied cells become interface; excess mass is split equally among the
 * interface neighbours of each converted cell. All decisions use the classes
 * after the collision (Jacobi style). */
static void conversions(orc_sim *s) {
    long n = s->n;
    uint8_t *mark = (uint8_t *)calloc(n, 1);
    for (int k = 0; k < 6; ++k) s->counts[k] = 0;
    /* (1) marks: the fill-level thresholds; and (R23) an interface cell
     * without a liquid neighbour empties, one without a gas neighbour fills
     * (the classes at t; walls and obstacles count as neither) */
    for (long i = 0; i < n; ++i) {
        if (s->flag[i] != IFC) continue;
        if (s->phin[i] >= 1.0 + s->eps) {
            mark[i] |= CV_FILLED;
        } else if (s->phin[i] <= -s->eps) {
            mark[i] |= CV_EMPTIED;
        } else if (s->nb_rule && g_mutation != 9) {
            int x = (int)(i % s->nx), y = (int)((i / s->nx) % s->ny), z = (int)(i / ((long)s->nx * s->ny));
            int liq = 0, gas = 0;
            for (int q = 1; q < Q; ++q) {
                int c = class_of(s, neighbour(s, x, y, z, C[q][0], C[q][1], C[q][2]));
                liq |= c == LIQ;
                gas |= c == GAS;
            }
            if (!liq && gas) mark[i] |= CV_EMPTIED;
            else if (!gas && liq) mark[i] |= CV_FILLED;
        }
    }
    /* (2) filled cells: gas neighbours become interface; emptied neighbours are kept */
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long i = cell_index(s, x, y, z);
                if (!(mark[i] & CV_FILLED)) continue;
                for (int q = 1; q < Q; ++q) {
                    long yi = neighbour(s, x, y, z, C[q][0], C[q][1], C[q][2]);
                    if (yi < 0) continue;
                    if (mark[yi] & CV_EMPTIED) mark[yi] &= (uint8_t)~CV_EMPTIED;
                    if (s->flag[yi] == GAS) mark[yi] |= CV_NEW_FROM_GAS;
                }
            }
    /* new interface cells from gas: f = f_eq(mean rho, mean u) of their liquid
     * and (old) interface neighbours */
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long i = cell_index(s, x, y, z);
                if (!(mark[i] & CV_NEW_FROM_GAS)) continue;
                double sr = 0.0, su[3] = {0.0, 0.0, 0.0};
                int cnt = 0;
                for (int q = 1; q < Q; ++q) {
                    long zi = neighbour(s, x, y, z, C[q][0], C[q][1], C[q][2]);
                    int zc = class_of(s, zi);
                    if (zc != LIQ && zc != IFC) continue;
                    double r = density(s->fn + zi * Q), u[3];
                    velocity_after_collision(s, s->fn + zi * Q, r, u);
                    sr += r;
                    su[0] += u[0];
                    su[1] += u[1];
                    su[2] += u[2];
                    cnt++;
                }
                double rm = sr / cnt, um[3] = {su[0] / cnt, su[1] / cnt, su[2] / cnt};
                for (int q = 0; q < Q; ++q) s->fn[i * Q + q] = feq(q, rm, um);
                s->mn[i] = 0.0;
                s->counts[2]++;
            }
    /* (3) still-emptied cells: liquid neighbours become interface with phi = 1 */
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long i = cell_index(s, x, y, z);
                if (!(mark[i] & CV_EMPTIED)) continue;
                for (int q = 1; q < Q; ++q) {
                    long yi = neighbour(s, x, y, z, C[q][0], C[q][1], C[q][2]);
                    if (yi >= 0 && s->flag[yi] == LIQ) mark[yi] |= CV_NEW_FROM_LIQ;
                }
            }
    for (long i = 0; i < n; ++i)
        if (mark[i] & CV_NEW_FROM_LIQ) {
            s->mn[i] = density(s->fn + i * Q);
            s->counts[3]++;
        }
    /* (4) classes */
    for (long i = 0; i < n; ++i) {
        if (mark[i] & CV_FILLED) { s->flag[i] = LIQ; s->counts[0]++; }
        else if (mark[i] & CV_EMPTIED) { s->flag[i] = GAS; s->counts[1]++; }
        else if (mark[i] & (CV_NEW_FROM_GAS | CV_NEW_FROM_LIQ)) s->flag[i] = IFC;
    }
    /* (5) excess mass e(x), split over the k(x) interface neighbours */
    double *share = (double *)calloc(n, sizeof(double));
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long i = cell_index(s, x, y, z);
                if (!(mark[i] & (CV_FILLED | CV_EMPTIED))) continue;
                double e = (mark[i] & CV_FILLED) ? s->mn[i] - density(s->fn + i * Q) : s->mn[i];
                int k = 0;
                for (int q = 1; q < Q; ++q) {
                    long yi = neighbour(s, x, y, z, C[q][0], C[q][1], C[q][2]);
                    if (yi >= 0 && s->flag[yi] == IFC) k++;
                }
                if (k == 0) s->lost += e;
                else share[i] = e / k;
            }
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long i = cell_index(s, x, y, z);
                if (s->flag[i] != IFC) continue;
                double acc = 0.0;
                int got = 0;
                for (int q = 1; q < Q; ++q) {
                    long yi = neighbour(s, x, y, z, C[q][0], C[q][1], C[q][2]);
                    if (yi >= 0 && (mark[yi] & (CV_FILLED | CV_EMPTIED))) {
                        acc += share[yi];
                        got = 1;
                    }
                }
                if (got || (mark[i] & (CV_NEW_FROM_GAS | CV_NEW_FROM_LIQ))) {
                    s->mn[i] = s->mn[i] + acc;
                    /* (6) fill level of the changed interface cells */
                    s->phin[i] = s->mn[i] / density(s->fn + i * Q);
                    s->counts[4]++;
                }
            }
    for (long i = 0; i < n; ++i) {
        if (mark[i] & CV_FILLED) s->mn[i] = density(s->fn + i * Q);
        else if (mark[i] & CV_EMPTIED) s->mn[i] = 0.0;
    }
    free(share);
    free(mark);
}

/* ------------------------------------------------------------------ C5 */

/* Rigid-body update replacing the external physics engine (Sec. 2.3 leaves
 * it to pe).  An explicit update of a body that is light compared with the
 * liquid is unstable with the momentum-exchange force (the bounce-back
 * answers a velocity change within one step: the added-mass instability), so
 * the update uses the virtual-mass scheme:
 *     (m + C m_f) dv_{n+1} = Fh_n + m g + C m_f dv_n,
 * m the body's mass, m_f the mass of liquid of its volume (liquid density 1),
 * dv the per-step velocity increment and C the virtual-mass coefficient
 * (C = 0 is the explicit Newton update); the same for the angular velocity in
 * the body frame, with the body's principal moments I, the displaced liquid's
 * I / rho_s and the gyroscopic term omega x (I omega) of Euler's equations.
 * Fh_n (and the torque likewise) is the mean of the momentum-exchange force of
 * this step and the previous one (the force itself on the first step), or the
 * force of this step alone when the two-step mean is switched off: near
 * tau = 1/2 the BGK modes that flip sign every step are barely damped, and a
 * force that flips with them feeds back through the wall velocity into a
 * growing oscillation of the body and the liquid under it; the mean removes
 * that component and leaves slower forcing unchanged.  Box of half extents h:
 * V = 8 h0 h1 h2, I_x = m (h1^2 + h2^2) / 3 (= m (b^2 + c^2) / 12 for the full
 * edges b = 2 h1, c = 2 h2); sphere: V = 4/3 pi r^3, I = 2/5 m r^2.  With
 * rotation about one axis a only, the torque is projected on a and the moment
 * of inertia is a^T I a in the body frame.  Position: semi-implicit Euler
 * (o += v_{n+1}); orientation: first-order update of the quaternion by the
 * world-frame angular velocity, q <- normalise(q + 1/2 (0, omega) q), which
 * turns the body by 2 atan(|omega| / 2) per step. */
static void bodies_step(orc_sim *s) {
    const double C = s->vmass;
    for (int bi = 0; bi < s->nb; ++bi) {
        body_t *b = &s->b[bi];
        int base = b->mode & 0xff;
        if (base == M_FIXED) {
            for (int k = 0; k < 3; ++k) b->v[k] = b->w[k] = b->dv[k] = b->dw[k] = 0.0;
            continue;
        }
        double Fh[3], Th[3];
        for (int k = 0; k < 3; ++k) {
            int mean = s->force_mean && b->nF;
            Fh[k] = mean ? 0.5 * (b->F[k] + b->Fp[k]) : b->F[k];
            Th[k] = mean ? 0.5 * (b->T[k] + b->Tp[k]) : b->T[k];
            b->Fp[k] = b->F[k];
            b->Tp[k] = b->T[k];
        }
        b->nF = 1;
        double vol, mass, I[3];
        if (b->shape == 1) { /* sphere: V = 4/3 pi r^3, I = 2/5 m r^2 */
            vol = 4.1887902047863905 * ((b->h[0] * b->h[0]) * b->h[0]);
            mass = b->dens * vol;
            I[0] = I[1] = I[2] = (0.4 * mass) * (b->h[0] * b->h[0]);
        } else {
            vol = ((8.0 * b->h[0]) * b->h[1]) * b->h[2];
            if (g_mutation == 14) vol = (b->h[0] * b->h[1]) * b->h[2];
            mass = b->dens * vol;
            double f = g_mutation == 10 ? 12.0 : 3.0;
            I[0] = (mass / f) * (b->h[1] * b->h[1] + b->h[2] * b->h[2]);
            I[1] = (mass / f) * (b->h[0] * b->h[0] + b->h[2] * b->h[2]);
            I[2] = (mass / f) * (b->h[0] * b->h[0] + b->h[1] * b->h[1]);
        }
        double If[3] = {I[0] / b->dens, I[1] / b->dens, I[2] / b->dens}; /* inertia of the displaced liquid */
        double den = g_mutation == 11 ? mass : mass + C * vol;
        for (int k = 0; k < 3; ++k) {
            double num = (Fh[k] + mass * s->grav[k]) + C * (vol * b->dv[k]);
            b->dv[k] = num / den;
            b->v[k] = b->v[k] + b->dv[k];
        }
        if (b->mode & M_DAMP)
            for (int k = 0; k < 3; ++k) b->v[k] = b->v[k] * (1.0 - b->damp);
        double R[3][3];
        rotation(b->q, R);
        if (base == M_ROT_AXIS) {
            const double *ax = b->axis;
            double ta = (Th[0] * ax[0] + Th[1] * ax[1]) + Th[2] * ax[2];
            double ab[3];
            for (int k = 0; k < 3; ++k) ab[k] = (R[0][k] * ax[0] + R[1][k] * ax[1]) + R[2][k] * ax[2];
            double Ia = (ab[0] * ab[0] * I[0] + ab[1] * ab[1] * I[1]) + ab[2] * ab[2] * I[2];
            double Ifa = Ia / b->dens;
            double ws = (b->w[0] * ax[0] + b->w[1] * ax[1]) + b->w[2] * ax[2];
            b->dw[0] = (ta + C * (Ifa * b->dw[0])) / (Ia + C * Ifa);
            ws = ws + b->dw[0];
            for (int k = 0; k < 3; ++k) b->w[k] = ws * ax[k];
        } else {
            double wb[3], tb[3], L[3], gy[3];
            for (int k = 0; k < 3; ++k) {
                wb[k] = (R[0][k] * b->w[0] + R[1][k] * b->w[1]) + R[2][k] * b->w[2];
                tb[k] = (R[0][k] * Th[0] + R[1][k] * Th[1]) + R[2][k] * Th[2];
                L[k] = I[k] * wb[k];
            }
            gy[0] = wb[1] * L[2] - wb[2] * L[1];
            gy[1] = wb[2] * L[0] - wb[0] * L[2];
            gy[2] = wb[0] * L[1] - wb[1] * L[0];
            if (g_mutation == 12)
                for (int k = 0; k < 3; ++k) gy[k] = -gy[k];
            for (int k = 0; k < 3; ++k) {
                b->dw[k] = ((tb[k] - gy[k]) + C * (If[k] * b->dw[k])) / (I[k] + C * If[k]);
                wb[k] = wb[k] + b->dw[k];
            }
            for (int k = 0; k < 3; ++k) b->w[k] = (R[k][0] * wb[0] + R[k][1] * wb[1]) + R[k][2] * wb[2];
        }
        double nn[3] = {s->nx, s->ny, s->nz};
        for (int k = 0; k < 3; ++k) {
            b->o[k] = b->o[k] + b->v[k];
            if (s->periodic & (1u << k)) {
                if (b->o[k] >= nn[k]) b->o[k] = b->o[k] - nn[k];
                else if (b->o[k] < 0.0) b->o[k] = b->o[k] + nn[k];
            }
        }
        /* q <- normalize(q + 1/2 (0, omega) (x) q) */
        double qw = b->q[0], qx = b->q[1], qy = b->q[2], qz = b->q[3];
        double *w = b->w;
        double dw = -((w[0] * qx + w[1] * qy) + w[2] * qz);
        double dx = qw * w[0] + (w[1] * qz - w[2] * qy);
        double dy = qw * w[1] + (w[2] * qx - w[0] * qz);
        double dz = qw * w[2] + (w[0] * qy - w[1] * qx);
        if (g_mutation == 13) { /* q (x) (0, omega): the body-frame product */
            dx = qw * w[0] - (w[1] * qz - w[2] * qy);
            dy = qw * w[1] - (w[2] * qx - w[0] * qz);
            dz = qw * w[2] - (w[0] * qy - w[1] * qx);
        }
        double nq[4] = {qw + 0.5 * dw, qx + 0.5 * dx, qy + 0.5 * dy, qz + 0.5 * dz};
        double norm = sqrt(((nq[0] * nq[0] + nq[1] * nq[1]) + nq[2] * nq[2]) + nq[3] * nq[3]);
        for (int k = 0; k < 4; ++k) b->q[k] = nq[k] / norm;
    }
}

/* ------------------------------------------------------------------ C6 */

/* Sec. 2.3 / 2.4: map the bodies at their new pose.  Covered fluid becomes
 * obstacle (its mass booked as covered); uncovered obstacle cells take their
 * class from the non-obstacle neighbourhood B(x): liquid and gas -> interface,
 * no gas -> liquid, no liquid -> gas; Jacobi passes until every uncovered cell
 * is assigned (at most four, then gas), followed by a closure pass. */
static void remap(orc_sim *s) {
    long n = s->n;
    if (s->nb == 0) return;
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long i = cell_index(s, x, y, z);
                if (s->flag[i] == OBS) continue;
                for (int bi = 0; bi < s->nb; ++bi) {
                    if (!inside(s, &s->b[bi], x, y, z)) continue;
                    if (s->flag[i] == LIQ) s->covered += density(s->fn + i * Q);
                    else if (s->flag[i] == IFC) s->covered += s->mn[i];
                    s->flag[i] = OBS;
                    s->body[i] = bi;
                    s->counts[5]++;
                    break;
                }
            }
    uint8_t *pend = (uint8_t *)calloc(n, 1);
    uint8_t *fresh = (uint8_t *)calloc(n, 1);
    int any = 0;
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long i = cell_index(s, x, y, z);
                if (s->flag[i] == OBS && !inside(s, &s->b[s->body[i]], x, y, z)) { pend[i] = 1; any = 1; }
            }
    uint8_t *decision = (uint8_t *)calloc(n, 1);
    double *drho = (double *)calloc(n, sizeof(double));
    double *dphi = (double *)calloc(n, sizeof(double));
    for (int pass = 0; pass < 4 && any; ++pass) {
        for (int z = 0; z < s->nz; ++z)
            for (int y = 0; y < s->ny; ++y)
                for (int x = 0; x < s->nx; ++x) {
                    long i = cell_index(s, x, y, z);
                    decision[i] = 0;
                    if (!pend[i]) continue;
                    int nL = 0, nI = 0, nG = 0;
                    double sr = 0.0, sp = 0.0;
                    for (int q = 1; q < Q; ++q) {
                        long yi = neighbour(s, x, y, z, C[q][0], C[q][1], C[q][2]);
                        if (yi < 0 || pend[yi] || s->flag[yi] == OBS) continue;
                        int c = s->flag[yi];
                        if (c == LIQ) { nL++; sr += density(s->fn + yi * Q); }
                        else if (c == IFC) { nI++; sr += density(s->fn + yi * Q); sp += s->phin[yi]; }
                        else if (c == GAS) nG++;
                    }
                    if (nL > 0 && nG > 0) {
                        decision[i] = IFC;
                        drho[i] = sr / (nL + nI);
                        dphi[i] = nI > 0 ? sp / nI : 0.5;
                    } else if (nG == 0 && nL + nI > 0) {
                        decision[i] = LIQ;
                        drho[i] = sr / (nL + nI);
                    } else if (nL == 0 && nG > 0) {
                        decision[i] = GAS;
                    }
                }
        any = 0;
        for (int z = 0; z < s->nz; ++z)
            for (int y = 0; y < s->ny; ++y)
                for (int x = 0; x < s->nx; ++x) {
                    long i = cell_index(s, x, y, z);
                    if (!pend[i]) continue;
                    int d = decision[i];
                    if (d == 0 && pass == 3) d = GAS;
                    if (d == 0) { any = 1; continue; }
                    body_t *b = &s->b[s->body[i]];
                    pend[i] = 0;
                    fresh[i] = 1;
                    s->flag[i] = (uint8_t)d;
                    s->body[i] = -1;
                    if (d == GAS) continue;
                    double p[3] = {x + 0.5, y + 0.5, z + 0.5}, uw[3];
                    body_velocity_at(s, b, p, uw);
                    for (int q = 0; q < Q; ++q) s->fn[i * Q + q] = feq(q, drho[i], uw);
                    if (d == IFC) {
                        s->mn[i] = dphi[i] * drho[i];
                        s->phin[i] = s->mn[i] / density(s->fn + i * Q);
                    }
                }
    }
    /* closure: a new liquid cell next to gas becomes interface with phi = 1 */
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long i = cell_index(s, x, y, z);
                if (!fresh[i] || s->flag[i] != LIQ) continue;
                int gas = 0;
                for (int q = 1; q < Q; ++q) {
                    long yi = neighbour(s, x, y, z, C[q][0], C[q][1], C[q][2]);
                    if (yi >= 0 && s->flag[yi] == GAS) gas = 1;
                }
                if (gas) {
                    s->flag[i] = IFC;
                    s->mn[i] = density(s->fn + i * Q);
                    s->phin[i] = s->mn[i] / density(s->fn + i * Q);
                }
            }
    for (long i = 0; i < n; ++i) {
        if (!fresh[i]) continue;
        if (s->flag[i] == LIQ) s->uncovered += density(s->fn + i * Q);
        else if (s->flag[i] == IFC) s->uncovered += s->mn[i];
    }
    free(pend); free(fresh); free(decision); free(drho); free(dphi);
}

/* ------------------------------------------------------------------ C7 */

static void check_invariants(orc_sim *s) {
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long i = cell_index(s, x, y, z);
                if (s->flag[i] != LIQ) continue;
                for (int q = 1; q < Q; ++q) {
                    long yi = neighbour(s, x, y, z, C[q][0], C[q][1], C[q][2]);
                    if (yi >= 0 && s->flag[yi] == GAS) s->err |= ORC_ERR_LIQUID_GAS_ADJ;
                }
                for (int q = 0; q < Q; ++q)
                    if (!isfinite(s->f[i * Q + q])) s->err |= ORC_ERR_NONFINITE;
            }
}

int orc_step(orc_sim *s, int nsteps) {
    init_lattice();
    for (int it = 0; it < nsteps; ++it) {
        if (!s->have_m0) {
            s->M0 = liquid_mass(s);
            s->have_m0 = 1;
        }
        orc_compute_forces(s); /* C4 at time t */
        stream_collide(s);     /* C1, C2 */
        conversions(s);        /* C3 */
        bodies_step(s);        /* C5 */
        remap(s);              /* C6 */
        double *t;
        t = s->f; s->f = s->fn; s->fn = t;
        t = s->phi; s->phi = s->phin; s->phin = t;
        t = s->m; s->m = s->mn; s->mn = t;
        check_invariants(s);   /* C7 */
        s->t++;
    }
    return s->err;
}

/* --------------------------------------------------------------- queries */

void orc_get_fields(const orc_sim *s, uint8_t *flags, double *fill, double *mass, double *rho, double *u,
                    double *f) {
    for (long i = 0; i < s->n; ++i) {
        int c = s->flag[i];
        int fluid = c == LIQ || c == IFC;
        double r = fluid ? density(s->f + i * Q) : 0.0;
        if (flags) flags[i] = (uint8_t)c;
        if (fill) fill[i] = c == LIQ ? 1.0 : (c == IFC ? s->phi[i] : 0.0);
        if (mass) mass[i] = c == LIQ ? r : (c == IFC ? s->m[i] : 0.0);
        if (rho) rho[i] = r;
        if (u) {
            double v[3] = {0.0, 0.0, 0.0};
            if (fluid) velocity_after_collision(s, s->f + i * Q, r, v);
            u[3 * i] = v[0]; u[3 * i + 1] = v[1]; u[3 * i + 2] = v[2];
        }
        if (f)
            for (int q = 0; q < Q; ++q) f[(long)q * s->n + i] = fluid ? s->f[i * Q + q] : 0.0;
    }
}

void orc_get_body(const orc_sim *s, int bi, double F[3], double T[3], double *S, double center[3],
                  double quat[4], double vel[3], double omega[3]) {
    const body_t *b = &s->b[bi];
    for (int k = 0; k < 3; ++k) {
        if (F) F[k] = b->F[k];
        if (T) T[k] = b->T[k];
        if (center) center[k] = b->o[k];
        if (vel) vel[k] = b->v[k];
        if (omega) omega[k] = b->w[k];
    }
    if (quat) for (int k = 0; k < 4; ++k) quat[k] = b->q[k];
    if (S) *S = b->S;
}

void orc_get_ledger(const orc_sim *s, double out[6]) {
    out[0] = s->covered;
    out[1] = s->uncovered;
    out[2] = s->lost;
    out[3] = s->have_m0 ? s->M0 : liquid_mass(s);
    out[4] = liquid_mass(s);
    out[5] = s->wall;
}

int orc_error(const orc_sim *s) { return s->err; }
long orc_time(const orc_sim *s) { return s->t; }
void orc_get_counts(const orc_sim *s, long out[6]) {
    for (int k = 0; k < 6; ++k) out[k] = s->counts[k];
}

void orc_lattice(int c[19][3], double w[19], int opp[19]) {
    init_lattice();
    for (int q = 0; q < Q; ++q) {
        for (int k = 0; k < 3; ++k) c[q][k] = C[q][k];
        w[q] = W[q];
        opp[q] = OPP[q];
    }
}

void orc_feq(double rho, const double u[3], double out[19]) {
    init_lattice();
    for (int q = 0; q < Q; ++q) out[q] = feq(q, rho, u);
}

void orc_force_term(double rho, const double u[3], const double a[3], double out[19]) {
    init_lattice();
    for (int q = 0; q < Q; ++q) out[q] = force_term(q, rho, u, a);
}

void orc_set_mutation(int m) { g_mutation = m; }

void orc_set_surface_tension(orc_sim *s, double sigma) { s->sigma = sigma; }

void orc_set_wall_velocity(orc_sim *s, const double v[18]) {
    for (int f = 0; f < 6; ++f)
        for (int j = 0; j < 3; ++j) s->wall_vel[f][j] = v[3 * f + j];
}

void orc_set_readings(orc_sim *s, double deadband, double virtual_mass, int force_mean, int neighbour_rule) {
    s->deadband = deadband;
    s->vmass = virtual_mass;
    s->force_mean = force_mean != 0;
    s->nb_rule = neighbour_rule != 0;
}

void orc_set_body_force(orc_sim *s, int bi, const double F[3], const double T[3]) {
    for (int k = 0; k < 3; ++k) {
        s->b[bi].F[k] = F[k];
        s->b[bi].T[k] = T[k];
    }
}

void orc_bodies_step(orc_sim *s) {
    init_lattice();
    bodies_step(s);
}
