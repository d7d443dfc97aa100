/*
 * lbm_fs.h -- C ABI of the GB300 (sm_103a) free-surface lattice Boltzmann
 * library with floating rigid boxes.
 *
 * Method: Bogner & Ruede, "Liquid-gas-solid flows with lattice Boltzmann:
 * Simulation of floating bodies" (arXiv:1201.0351).  One time step is the
 * D3Q19 BGK stream + collide with gravity (Sec. 2.1, Eqs. lbgk, equilibrium,
 * forceterm), the free-surface boundary with interface mass exchange and
 * atmosphere reconstruction (Sec. 2.2, Eq. reconstruct), moving-wall bounce-back
 * at obstacle links with the momentum-exchange force and torque on each box
 * (Sec. 2.3, Eqs. noslip, momentumexchange, netforce, torque; Sec. 2.4, Eq.
 * momentuminterface), the interface cell conversions (Sec. 2.2), the rigid-body
 * update, and the obstacle remapping with the obstacle-to-fluid rule (Sec. 2.4).
 *
 * Conventions (all quantities in lattice units):
 *  - grid nx x ny x nz; cell (x,y,z) is [x,x+1]x[y,y+1]x[z,z+1] (Sec. 2.1);
 *    linear index idx = x + nx*(y + ny*z);
 *  - cell classes: 1 liquid, 2 interface, 4 gas, 8 obstacle;
 *  - a non-periodic face is a resting no-slip wall half a cell outside the grid;
 *  - populations are numbered C,W,E,N,S,T,B,TW,TE,TN,TS,NW,NE,SW,SE,BW,BE,BN,BS
 *    (the order of the paper's D3Q19 stencil figure).
 *
 * Errors: every call returns an lbm_fs_status; nothing is thrown across the
 * ABI.  Invalid arguments give LBM_FS_EINVAL before any allocation.  Device-side
 * conditions (a liquid cell touching gas, a non-finite density, a moving box
 * reaching a domain wall -- contacts are not modelled --, fluid appearing
 * more than a few cells above the previous step's fluid top, which the bulk
 * sweep tracks to skip all-gas tiles and which fluid cannot outrun, a worklist
 * overflow) are sticky bits in a device status word; they are reported as
 * LBM_FS_EUNSTABLE / LBM_FS_EOVERFLOW by the next call that synchronises
 * (lbm_fs_forces, lbm_fs_body_state, lbm_fs_read_fields, lbm_fs_stats,
 * lbm_fs_sync).  lbm_fs_last_error_string() describes the last failure of the
 * calling thread.  A handle may be used by one host thread at a time; distinct
 * handles are independent.
 */
#ifndef LBM_FS_H
#define LBM_FS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_fs lbm_fs; /* opaque; owned by the library */

typedef enum {
    LBM_FS_OK = 0,
    LBM_FS_EINVAL = -1,    /* invalid argument or parameter */
    LBM_FS_ENOMEM = -2,    /* device allocation failed */
    LBM_FS_ECUDA = -3,     /* a CUDA runtime call failed */
    LBM_FS_ESTATE = -4,    /* call not valid in the handle's state */
    LBM_FS_EUNSTABLE = -5, /* non-finite density, or liquid touching gas */
    LBM_FS_ETIMEOUT = -6,  /* a bounded device wait (staged row copies) gave up */
    LBM_FS_EOVERFLOW = -7  /* a device worklist overflowed */
} lbm_fs_status;

/* population storage precision */
enum {
    LBM_FS_F64 = 0,  /* f_q as double; arithmetic in double (the plain path) */
    LBM_FS_F32 = 1,  /* f_q - w_q as float; arithmetic in float */
    LBM_FS_F16S = 2  /* f_q - w_q as half (q >= 1, scaled by 2^10) plus a float
                        rest population that makes the stored cell sum equal the
                        collision density; arithmetic in float */
};
/* With every storage the interface mass and fill levels, the mass ledger and
 * the rigid-body state stay in double.  The float storages sum the momentum
 * exchange per cell in float and across cells exactly: the uniform
 * gas-pressure part as 64-bit integers, the rest in fixed point (2^-32 force,
 * 2^-30 torque), converted to double per body. */

/* cell classes (init_flags input and LBM_FS_FIELD_FLAGS output) */
enum { LBM_FS_LIQUID = 1, LBM_FS_INTERFACE = 2, LBM_FS_GAS = 4, LBM_FS_OBSTACLE = 8 };

/* box motion modes (lbm_fs_box.mode) */
enum {
    LBM_FS_MODE_FIXED = 0,         /* held at its pose, velocity zero */
    LBM_FS_MODE_FREE = 1,          /* 6 degrees of freedom */
    LBM_FS_MODE_ROT_AXIS_ONLY = 2, /* translation + rotation about rot_axis only */
    LBM_FS_MODE_DAMP_TRANSLATION = 0x100 /* flag: v *= (1 - lin_damping) each step */
};

typedef struct {
    int32_t nx, ny, nz;
    uint32_t periodic;     /* bit0 x, bit1 y, bit2 z; other faces are walls */
    double tau;            /* BGK relaxation time, > 1/2 (tau = 3 nu + 1/2) */
    double gravity[3];     /* acceleration on liquid and bodies */
    double body_accel[3];  /* extra acceleration on the liquid only */
    double rho_gas;        /* gas density rho_G = 3 p_G (Eq. pressure) */
    double eps;            /* conversion threshold: fill at phi >= 1+eps, empty at phi <= -eps */
    int32_t storage;       /* LBM_FS_F64 / LBM_FS_F32 / LBM_FS_F16S */
    /* initial state, nx*ny*nz entries each (3 per cell for init_vel, xyz):
     * classes 1/2/4, fill level, density, velocity (NULL = at rest).  Fluid cells
     * start at f = f_eq(rho, u).  The arrays are copied; the caller keeps them.
     * init_flags, init_fill and init_rho are required. */
    const uint8_t *init_flags;
    const double *init_fill;
    const double *init_rho;
    const double *init_vel;
    int32_t init_on_device; /* nonzero: the four init pointers are device pointers */
    /* device memory: dev_alloc / dev_free with alloc_ctx (e.g. a framework's
     * caching allocator); NULL -> cudaMalloc / cudaFree.  dev_alloc must
     * return 16-byte aligned memory (the kernels use vector loads); a
     * misaligned block gives LBM_FS_EINVAL */
    void *(*dev_alloc)(size_t bytes, void *ctx);
    void (*dev_free)(void *ptr, void *ctx);
    void *alloc_ctx;
    void *stream;          /* cudaStream_t for all work; NULL -> legacy default stream */
    int32_t use_graphs;    /* nonzero: steps replay a captured CUDA graph */
    /* surface tension sigma >= 0 (Sec. 2.2): the gas pressure of the interface
     * boundary condition becomes p_G + 2 sigma kappa, kappa the mean curvature
     * div(n^)/2 of the unit normals n^ = -grad(phi)/|grad phi| of the six axis
     * neighbours (central differences; an obstacle or wall neighbour takes the
     * cell's own normal), i.e. the reconstruction uses rho_G + 6 sigma kappa.
     * 0 disables it (no curvature is computed). */
    double sigma;
    /* velocity of each non-periodic face, x-, x+, y-, y+, z-, z+ (Eq. noslip
     * with u_w: a link whose source lies beyond the face takes
     * f*_qbar + 6 w_q rho (c_q . u_w); a link across an edge takes the face of
     * its lowest axis); all zero: resting walls.  The mass a moving wall adds
     * to liquid cells is booked in lbm_fs_stats_t.wall_source. */
    double wall_vel[6][3];
    /* Readings of the paper where it is silent.  A field below is used only
     * when its LBM_FS_READING_* bit is set in `readings`; otherwise its default
     * applies (a zeroed struct gets every default).
     *  normal_deadband (default 1e-2, >= 0): Eq. reconstruct rebuilds the
     *    populations of the directions with c_q . n <= 0 (Sec. 2.2); a
     *    direction counts when c_q . n < -normal_deadband.  0 is the bare
     *    sign test, under which the noise of the estimated normal decides the
     *    tangential directions of a flat surface and the spurious interface
     *    velocities exceed the 1e-5 that Sec. 3.2.1 reports;
     *  virtual_mass (default 1, >= 0): coefficient C of the rigid-body update
     *    (m + C m_f) dv_{n+1} = F + m g + C m_f dv_n (the paper hands the
     *    bodies to an external engine, Sec. 2.3); 0 is the explicit update;
     *  force_mean (default 1): the update is driven by (F_n + F_{n-1}) / 2
     *    (F_n on the first step); 0: by F_n (Eq. netforce / torque);
     *  neighbour_rule (default 1): besides the fill thresholds of Sec. 2.2,
     *    an interface cell with gas but no liquid among its 18 neighbours
     *    empties and one with liquid but no gas fills; 0: thresholds only. */
    uint32_t readings;
    double normal_deadband;
    double virtual_mass;
    int32_t force_mean;
    int32_t neighbour_rule;
} lbm_fs_params;

/* bits of lbm_fs_params.readings */
enum {
    LBM_FS_READING_DEADBAND = 1u << 0,
    LBM_FS_READING_VIRTUAL_MASS = 1u << 1,
    LBM_FS_READING_FORCE_MEAN = 1u << 2,
    LBM_FS_READING_NEIGHBOUR_RULE = 1u << 3
};

typedef struct {
    double center[3];      /* centre of mass (world) */
    double half[3];        /* half extents along the body axes */
    double quat[4];        /* (w, x, y, z), body -> world */
    double density_ratio;  /* body density / liquid density */
    double vel[3];         /* initial velocity */
    double omega[3];       /* initial angular velocity (world) */
    int32_t mode;          /* LBM_FS_MODE_* */
    double rot_axis[3];    /* unit axis (world) for LBM_FS_MODE_ROT_AXIS_ONLY */
    double lin_damping;    /* for LBM_FS_MODE_DAMP_TRANSLATION */
    int32_t shape;         /* 0: box of half extents half; 1: sphere of radius half[0]
                              (volume 4/3 pi r^3, inertia 2/5 m r^2; Sec. 3.2.1) */
} lbm_fs_box;

typedef struct {
    double F[3], T[3];     /* force and torque of the last step (Eqs. netforce, torque) */
    double S;              /* sum of |link terms| (scale of F for tolerances) */
    double center[3], quat[4], vel[3], omega[3];
} lbm_fs_body_state_t;

typedef struct {
    int64_t step;
    double liquid_mass;    /* sum over liquid rho + interface m (computed by this call) */
    double mass0;          /* liquid mass at the first step */
    double covered, uncovered, lost_excess; /* mass ledger */
    int64_t n_interface, n_filled, n_emptied, n_new_from_gas, n_new_from_liquid, n_pending;
    uint32_t status;       /* sticky device status bits */
    int64_t kernel_launches; /* kernels launched by this handle so far */
    double wall_source;    /* mass added to liquid cells by the moving-wall term
                              6 w_q rho (c_q . u_w) of Eq. noslip.  Ledger identity:
                              liquid_mass = mass0 + uncovered - covered
                              - lost_excess + wall_source (to rounding) */
    int64_t n_general;     /* liquid cells of the last step with an obstacle among
                              their neighbours or on a face with moving walls
                              (stepped by the general-gather kernel) */
} lbm_fs_stats_t;

/* field selectors for lbm_fs_read_fields; dst[k] is the buffer for bit k.
 * (The state is set only at creation, from init_flags / init_fill / init_rho /
 * init_vel: there is no write-back call.)  Layouts: FLAGS uint8[N]; FILL, MASS, RHO double[N];
 * VEL double[3N] (xyz per cell); F double[19N] (SoA, [q][idx]).  FILL is 1 for
 * liquid, phi for interface, 0 else; MASS is rho / m / 0; RHO and VEL are the
 * density and the velocity of the last collision (sum c f / rho - a) of liquid
 * and interface cells, 0 else; F is 0 outside liquid and interface cells. */
enum {
    LBM_FS_FIELD_FLAGS = 1u << 0,
    LBM_FS_FIELD_FILL = 1u << 1,
    LBM_FS_FIELD_MASS = 1u << 2,
    LBM_FS_FIELD_RHO = 1u << 3,
    LBM_FS_FIELD_VEL = 1u << 4,
    LBM_FS_FIELD_F = 1u << 5
};

/* Creates a simulation (Sec. 2.1 grid, Sec. 2.2 initial fill).  Validates the
 * parameters (tau > 1/2, sizes, storage, the incompressibility bound of Sec.
 * 2.1: (nx, ny, nz) . |g| < 1/3), allocates the device state and uploads the
 * initial fields.  On success *out owns all device memory until
 * lbm_fs_destroy. */
lbm_fs_status lbm_fs_create(const lbm_fs_params *p, lbm_fs **out);
lbm_fs_status lbm_fs_destroy(lbm_fs *h);

/* Adds a rigid box and maps it to the lattice: a cell is an obstacle iff its
 * centre lies strictly inside the box (Sec. 2.3).  Before the first step the
 * covered mass is excluded from the initial mass; between steps it is booked as
 * covered.  At most 255 boxes. *out_id receives the body id (may be NULL). */
lbm_fs_status lbm_fs_add_box(lbm_fs *h, const lbm_fs_box *b, int32_t *out_id);

/* Enqueues nsteps time steps on the handle's stream and returns without
 * waiting.  One step, in order: the momentum-exchange force and torque on
 * every body from the state at t (Sec. 2.3 Eqs. momentumexchange, netforce,
 * torque; Sec. 2.4 Eq. momentuminterface); stream with no-slip and moving-wall
 * bounce-back (Sec. 2.1 Eq. stream, Sec. 2.3 Eq. noslip), the atmosphere
 * reconstruction and the interface mass exchange (Sec. 2.2 Eq. reconstruct and
 * the mass balance that follows it); BGK collision with the gravity force term
 * (Sec. 2.1 Eqs. lbgk, equilibrium, forceterm, density, momentum) and the new
 * fill levels; the interface conversions with excess-mass redistribution
 * (Sec. 2.2, last paragraph); the rigid-body update (Sec. 2.3); the obstacle
 * remapping, cells covered and uncovered by the moved bodies with the
 * obstacle-to-fluid rule (Sec. 2.3 body discretisation, Sec. 2.4).
 * nsteps < 0 gives LBM_FS_EINVAL; 0 enqueues nothing.  Device-side failures
 * surface at the next synchronising call (header comment). */
lbm_fs_status lbm_fs_step(lbm_fs *h, int32_t nsteps);

/* Synchronises and returns the force F and torque T of the last step on body
 * id (Sec. 2.3 Eqs. netforce and torque: the momentum exchange of Eq.
 * momentumexchange summed over the body's links, with Eq. momentuminterface
 * on interface and gas cells; torque about the body's centre with the lever
 * arm from the fluid cell's centre; FP64) and its current pose (centre,
 * quaternion (w, x, y, z) body -> world).  Caller-owned host arrays; any
 * pointer may be NULL.  An unknown id gives LBM_FS_EINVAL; before the first
 * step F and T are zero. */
lbm_fs_status lbm_fs_forces(lbm_fs *h, int32_t id, double F[3], double T[3],
                            double center[3], double quat[4]);
lbm_fs_status lbm_fs_body_state(lbm_fs *h, int32_t id, lbm_fs_body_state_t *out);
/* Synchronises once and copies the states of bodies first .. first+count-1 into
 * out[0 .. count-1] (one device-to-host copy: the per-step read of a coupled
 * host-side rigid-body engine). */
lbm_fs_status lbm_fs_body_states(lbm_fs *h, int32_t first, int32_t count, lbm_fs_body_state_t *out);

/* Synchronises and copies the selected fields into caller-owned buffers (host
 * or device, per dst_on_device), each sized as documented above: the cell
 * classes, the fill level phi = m / rho of Sec. 2.2, the mass, and the
 * density and velocity of Sec. 2.1 Eqs. density and momentum (of the last
 * collision: rho = sum f*, u = sum c f* / rho - a), and the populations.
 * dst[k] serves bit k of mask; unselected entries may be NULL, a selected
 * NULL gives LBM_FS_EINVAL. */
lbm_fs_status lbm_fs_read_fields(lbm_fs *h, uint32_t mask, void *const *dst,
                                 int32_t dst_on_device);

/* Synchronises and fills *out (computes the current liquid mass on the device). */
lbm_fs_status lbm_fs_stats(lbm_fs *h, lbm_fs_stats_t *out);

/* Synchronises the handle's stream and reports sticky device errors. */
lbm_fs_status lbm_fs_sync(lbm_fs *h);

/* Runs nsteps steps without graphs, timing every kernel with CUDA events on the
 * handle's stream; ms[k] receives the summed milliseconds of kernel k over the
 * steps and names (may be NULL) a static name per kernel.  Returns the number
 * of kernels in *nk (at most cap entries are written). */
lbm_fs_status lbm_fs_kernel_times(lbm_fs *h, int32_t nsteps, double *ms,
                                  const char **names, int32_t cap, int32_t *nk);

/* ---- Batched form: many independent tanks stepped together.
 *
 * The paper steps one domain; stepping many small scenarios (a sweep over heel
 * angles, densities and resolutions) one handle at a time leaves the GPU idle
 * between a small tank's short kernels.  A batch owns `count` tanks, each an
 * ordinary simulation created from params[k] (same storage for all; the
 * batch runs on params[0].stream and uses params[0].use_graphs and its
 * allocator for its own buffers).  Every kernel of a step is launched once
 * for all tanks (at most 64 tanks per launch; larger batches use one launch
 * per group of 64): its blocks walk a packed table of (tank, block) entries,
 * and the bulk stream + collide kernel runs as a persistent grid over that
 * table.  The per-cell arithmetic is that of the single-tank path, so each
 * tank's results equal those of lbm_fs_step on the same tank.
 *
 * lbm_fs_batch_create validates every params[k] like lbm_fs_create (the first
 * failure is returned, with k in the error text) and limits each tank to
 * 65535 cells per axis and nx*ny <= 8388480.  *out owns every tank until
 * lbm_fs_batch_destroy. */
typedef struct lbm_fs_batch lbm_fs_batch; /* opaque; owned by the library */
lbm_fs_status lbm_fs_batch_create(const lbm_fs_params *params, int32_t count, lbm_fs_batch **out);
lbm_fs_status lbm_fs_batch_destroy(lbm_fs_batch *b);

/* Handle of tank k (owned by the batch).  It serves lbm_fs_add_box (between
 * batch steps), lbm_fs_forces, lbm_fs_body_state(s), lbm_fs_read_fields,
 * lbm_fs_stats and lbm_fs_sync; lbm_fs_step, lbm_fs_kernel_times and
 * lbm_fs_destroy on it return LBM_FS_ESTATE. */
lbm_fs_status lbm_fs_batch_tank(lbm_fs_batch *b, int32_t k, lbm_fs **out);

/* Enqueues nsteps steps of every tank and returns without waiting. */
lbm_fs_status lbm_fs_batch_step(lbm_fs_batch *b, int32_t nsteps);

/* Synchronises and reports the first sticky device error of any tank. */
lbm_fs_status lbm_fs_batch_sync(lbm_fs_batch *b);

/* Launch configuration of a batch:
 *   zb          z-planes per bulk tile (1..8);
 *   bulk_blocks persistent grid of the bulk kernel (0: one block per tile);
 *   list_cells  nx*ny cells of a tank per block of the worklist kernels
 *               (a tank gets ceil(nx*ny / list_cells) blocks, at most 304);
 *   lanes       groups of tanks (of about equal cell count) whose step
 *               launches form independent chains that the GPU runs side by
 *               side, one group's short list kernels beside another's bulk
 *               kernel (1..4; 0 keeps the current value; default 1: on the
 *               64-tank sweep 2 to 4 lanes measured no faster, the bulk
 *               kernel filling every SM);
 *   bulk_ms     (autotune output) time of one bulk launch with this setting. */
typedef struct {
    int32_t zb;
    int32_t bulk_blocks;
    int32_t list_cells;
    int32_t lanes;
    double bulk_ms;
} lbm_fs_batch_config_t;

/* Times the batched bulk kernel over a set of candidate tilings (zb in
 * {1, 2, 4, 8}; persistent grids of 1, 2 and 4 times the resident blocks,
 * and one block per tile) on the current state and keeps the fastest;
 * *out (may be NULL) receives it.  The state is not advanced: the timed
 * launches write only the second population grid (rewritten by the next
 * step), and the worklist counters and mass ledger are restored.  Call it
 * between steps; the interface-cell count that lbm_fs_stats reports reads 0
 * until the next step. */
lbm_fs_status lbm_fs_batch_autotune(lbm_fs_batch *b, lbm_fs_batch_config_t *out);
lbm_fs_status lbm_fs_batch_set_config(lbm_fs_batch *b, const lbm_fs_batch_config_t *c);
lbm_fs_status lbm_fs_batch_get_config(lbm_fs_batch *b, lbm_fs_batch_config_t *c);

/* As lbm_fs_kernel_times, for the batched launches (summed over all groups of
 * 64 tanks); *launches (may be NULL) receives the batch's kernel launches
 * since creation. */
lbm_fs_status lbm_fs_batch_kernel_times(lbm_fs_batch *b, int32_t nsteps, double *ms,
                                        const char **names, int32_t cap, int32_t *nk);
lbm_fs_status lbm_fs_batch_launches(lbm_fs_batch *b, int64_t *launches, int64_t *steps);

const char *lbm_fs_last_error_string(void);
int32_t lbm_fs_version(void);

/* Measurement helper (no counterpart in the paper): the rate at which this
 * GPU executes one double-precision operation, op 0 fused multiply-add, 1 add,
 * 2 multiply, in operations (thread instructions) per second, from
 * independent chains on every SM timed with CUDA events on `stream` (NULL =
 * legacy default stream).  The double-storage path is bound by this rate
 * rather than by memory.  iters sets the chain length (2^16 takes about 0.3 s
 * on a GB300, each step of a chain taking ~4.7 us across the full grid).
 * Synchronises; allocates nothing; bad arguments give
 * LBM_FS_EINVAL, a failed launch LBM_FS_ECUDA. */
lbm_fs_status lbm_fs_fp64_rate(int32_t op, int32_t iters, double *ops_per_s, void *stream);

/* Liquid mass without allocating: sum over liquid and interface cells of the
 * per-cell mass, for callers that cannot allocate device memory (a host that
 * owns a fixed memory budget, work recorded inside a CUDA graph capture, or a
 * loop that must not block on an allocator).  The paper has no counterpart:
 * this is a library-level variant of the reduction behind lbm_fs_stats.
 *   flags: device pointer, n class bytes (LBM_FS_FIELD_FLAGS layout);
 *   mass:  device pointer, n doubles (LBM_FS_FIELD_MASS layout);
 *   out:   device pointer, receives one double;
 *   stream: cudaStream_t (NULL = legacy default stream).
 * Block partial sums live in a fixed 512 KiB device array of the library
 * (held by every GPU that loads the library until exit), so n is limited to
 * 268435456 cells; larger n, n < 0 or a null pointer give LBM_FS_EINVAL.  The
 * first call on a device, and the first in any other CUDA context of it (after
 * a cudaDeviceReset, or in a caller's own context), looks up that array's
 * device address in the current context (set-up with the device current);
 * make such a first call before any stream capture.  Every call
 * on a device shares the array and it keeps the last call's contents: calls
 * that overlap on the GPU (different streams, no ordering) race and may return
 * wrong sums.  No cudaMalloc / cudaFree or allocating routine is called.  The
 * call is asynchronous; errors of the launch are returned, the error text is
 * in lbm_fs_noalloc_last_error_string(). */
lbm_fs_status lbm_fs_liquid_mass_noalloc(const uint8_t *flags, const double *mass, int64_t n,
                                         double *out, void *stream);
const char *lbm_fs_noalloc_last_error_string(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_FS_H */
