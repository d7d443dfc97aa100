/*
 * lbm_oracle.h -- plain FP64 CPU oracle for the liquid-gas-solid lattice
 * Boltzmann method of Bogner & Ruede, "Liquid-gas-solid flows with lattice
 * Boltzmann: Simulation of floating bodies" (Sec. 2.1 - 2.4).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the GPU library: it is an independent,
 * deliberately slow restatement of the method, one cell and one direction at a
 * time, in the paper's order, used to check the GPU results.
 *
 * Cell classes (input and output encoding): 1 liquid, 2 interface, 4 gas,
 * 8 obstacle.  Arrays are indexed idx = x + nx*(y + ny*z).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_sim orc_sim;

/* error bits reported by orc_error() */
#define ORC_ERR_LIQUID_GAS_ADJ 1 /* a liquid cell touched a gas cell */
#define ORC_ERR_BAD_INPUT      2
#define ORC_ERR_NONFINITE      4

/* flags: 1/2/4 per cell; fill, rho per cell; vel: 3 per cell (xyz) or NULL
 * for fluid at rest.  Every fluid cell starts at f = f_eq(rho, vel). */
orc_sim *orc_create(int nx, int ny, int nz, unsigned periodic, double tau,
                    const double gravity[3], const double body_accel[3],
                    double rho_gas, double eps, const uint8_t *flags,
                    const double *fill, const double *rho, const double *vel);
void orc_destroy(orc_sim *s);
/* Adds a box and maps it (cells whose centre is strictly inside become
 * obstacle).  Before the first step the covered mass is simply excluded;
 * between steps it is booked as covered mass. Returns the body id. */
int orc_add_box(orc_sim *s, const double center[3], const double half[3],
                const double quat[4], double density_ratio, const double vel[3],
                const double omega[3], int mode, const double rot_axis[3],
                double lin_damping, int shape); /* shape 0: box; 1: sphere of radius half[0] */
int orc_step(orc_sim *s, int nsteps);
/* momentum exchange (force, torque) on every body from the current state,
 * without advancing time */
void orc_compute_forces(orc_sim *s);
/* canonical fields: fill (L 1, I phi, else 0), mass (L rho, I m, else 0),
 * rho (L/I sum of f, else 0), u (L/I sum c f / rho - a, else 0; xyz per cell),
 * f (SoA [q][idx], L/I only, else 0).  Any pointer may be NULL. */
void orc_get_fields(const orc_sim *s, uint8_t *flags, double *fill, double *mass,
                    double *rho, double *u, double *f);
/* body state: F, T, S (sum of |link terms|), centre, quat, v, omega */
void orc_get_body(const orc_sim *s, int b, double F[3], double T[3], double *S,
                  double center[3], double quat[4], double vel[3], double omega[3]);
/* ledger: [0] covered, [1] uncovered, [2] lost excess, [3] M at the first step,
 * [4] current liquid mass, [5] mass added to liquid cells by the moving-wall
 * term of Eq. noslip.  M = M0 + uncovered - covered - lost + wall. */
void orc_get_ledger(const orc_sim *s, double out[6]);
int orc_error(const orc_sim *s);
long orc_time(const orc_sim *s);
/* cells that the free-surface conversion handled in the last step */
void orc_get_counts(const orc_sim *s, long out[6]);

/* single formulas, exposed for the pin tests */
void orc_lattice(int c[19][3], double w[19], int opp[19]);
void orc_feq(double rho, const double u[3], double out[19]);
void orc_force_term(double rho, const double u[3], const double a[3], double out[19]);
/* Test-only deliberate defects (0 = none), used to show that the pins catch
 * plausible mistakes. */
void orc_set_mutation(int m);
/* surface tension sigma (lattice units): the gas pressure of the interface
 * boundary condition becomes p_G + 2 sigma kappa (Sec. 2.2); 0 disables */
void orc_set_surface_tension(orc_sim *s, double sigma);
/* velocities of the wall faces x-, x+, y-, y+, z-, z+ (3 each; Eq. noslip
 * with u_w at domain walls); zero by default */
void orc_set_wall_velocity(orc_sim *s, const double v[18]);
/* readings where the paper is silent (defaults 1e-2, 1, 1, 1):
 *   deadband       Eq. reconstruct rebuilds a direction when c_q . n < -deadband
 *                  (0: the strict sign test);
 *   virtual_mass   C of the rigid-body update (0: explicit Newton update);
 *   force_mean     1: the update is driven by (F_n + F_{n-1}) / 2, 0: by F_n;
 *   neighbour_rule 1: an interface cell without liquid neighbours (but with
 *                  gas ones) empties, one without gas neighbours (but with
 *                  liquid ones) fills; 0: the fill thresholds only. */
void orc_set_readings(orc_sim *s, double deadband, double virtual_mass, int force_mean, int neighbour_rule);
/* C5 alone, for its pins: set the force and torque of body b as if the
 * momentum exchange had produced them, then run the rigid-body update of every
 * body (no remapping of cells) */
void orc_set_body_force(orc_sim *s, int b, const double F[3], const double T[3]);
void orc_bodies_step(orc_sim *s);

#ifdef __cplusplus
}
#endif
#endif
