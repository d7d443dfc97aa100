// Internal declarations shared by the host API and the kernel translation
// units of the free-surface LBM library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmfs {

constexpr int Q = 19;
constexpr int MAX_BODIES = 255;
constexpr int FORCE_BLOCKS = 64;   // blocks per body in the force / remap kernels
constexpr int LIST_BLOCKS = 304;   // 2 x 152 SMs: grid of the worklist kernels
constexpr int LIST_THREADS = 256;
constexpr int REMAP_THREADS = 512;
// bytes before / after each population grid: the staged bulk kernel copies
// whole 128-cell row segments plus a 16-byte halo, which for the last x tile of
// the grid's last row reaches up to (128 + 8) elements past the array end
constexpr int GRID_GUARD = 1024;
#ifndef LBMFS_BULK_THREADS
#define LBMFS_BULK_THREADS 128
#endif
constexpr int BULK_THREADS = LBMFS_BULK_THREADS;  // x extent of a bulk-kernel block
// cells of an xy-plane per bulk-kernel block, by storage: one per thread for
// double, two per thread for the float storages
#ifndef LBMFS_BULK_PAIR
#define LBMFS_BULK_PAIR 0  // tuning knob: float storages on even grids take two cells per bulk-kernel thread
#endif

// cell classes (as in the C ABI) in the low nibble of the flag byte; bit 4
// marks a cell with an obstacle or a wall among its 18 neighbours
enum : uint8_t { CL_L = 1, CL_I = 2, CL_G = 4, CL_O = 8, CL_MASK = 15, NB_OBST = 16 };
// per-cell conversion marks (separate byte array, zero between steps)
enum : uint8_t {
    MK_FILLED = 1, MK_EMPTIED = 2, MK_NEWG = 4, MK_NEWL = 8, MK_RECV = 16, MK_PEND = 32, MK_FRESH = 64
};
// sticky device status bits
enum : uint32_t { ST_LIQUID_GAS = 1, ST_NONFINITE = 2, ST_OVERFLOW = 4, ST_TIMEOUT = 8, ST_CONTACT = 16, ST_TOP = 32 };
// z-planes above the previous step's highest fluid tile that the bulk kernel
// still visits (fluid rises by at most a cell or two per step)
constexpr int ZTOP_MARGIN = 4;

// worklists
enum { WL_IFACE = 0, WL_FILLED, WL_EMPTIED, WL_NEWG, WL_NEWL, WL_RECV, WL_PEND, WL_COVER, WL_GEN, WL_COUNT };
// ledger slots (double)
enum { LG_COVERED = 0, LG_UNCOVERED, LG_LOST, LG_MASS0, LG_MASS, LG_WALL, LG_COUNT };

struct Body {
    double o[3], h[3], q[4], dens, v[3], w[3], axis[3], damp;
    double dv[3], dw[3];
    double F[3], T[3], S;
    double Fp[3], Tp[3];  // the previous step's force and torque (rigid-body update)
    int nF, pad2;         // 1 once Fp, Tp hold a step
    double R[9];        // rotation of q (row-major), recomputed with the pose
    int mode, shape;  // shape 0: box of half extents h; 1: sphere of radius h[0]
    int lo[3], hi[3];   // cells that may be inside at the current pose, [lo, hi)
    int plo[3], phi[3]; // the same at the previous pose
    // the pose in float for the inside pre-test: centre split into its
    // integer part oi and fraction of, R and the half extents rounded to float
    int oi[3];
    float of[3], Rf[9], hf[3];
};

// Everything a kernel needs, passed by value.
struct Dev {
    int nx, ny, nz;
    unsigned periodic;
    long long N;
    double omega, a[3], grav[3], rho_g, eps;
    uint8_t *flags, *bid, *cmark;
    void *fsrc, *fdst;
    double *phisrc, *phidst, *m;
    uint32_t *list[WL_COUNT];
    uint32_t *cnt;  // WL_COUNT counters
    uint32_t cap;
    Body *bodies;
    int nb;
    double *part;   // force partials: MAX_BODIES * FORCE_BLOCKS * 7 slots of 16 bytes
    int part128;    // partials are exact 128-bit fixed-point sums (double storage)
    double *ledger; // LG_COUNT
    uint32_t *status;
    uint8_t *rdec;  // remap scratch: decision per pending item
    double *rrho, *rphi;
    double *red;    // reduction scratch
    int bulk;       // bulk-kernel variant for the float storages (BULK_*)
    // float copies for the float storages' arithmetic (rounded once on the
    // host: no per-cell double-to-float conversions on the GPU's FP64 pipe)
    float omega_f, a_f[3], drg_f, rg1_f;  // 1/tau, a, rho_G - 1, 1 - rho_G
    double sigma;  // surface tension (0: none)
    float sigma_f;
    int walls_move;       // nonzero: some non-periodic face moves
    const double *wallv;  // 6 x 3 face velocities (x-, x+, y-, y+, z-, z+)
    // highest z-plane of a bulk tile holding liquid or interface cells: read
    // (previous step) and written (this step) slots, swapped every step
    int *ztop_rd, *ztop_wr;
    // readings where the paper is silent (lbm_fs_params.readings)
    double deadband;   // Eq. reconstruct: c.n < -deadband selects a direction
    float deadband_f;
    double vmass;      // virtual-mass coefficient of the rigid-body update
    int force_mean;    // rigid-body update driven by (F_n + F_{n-1}) / 2
    int nb_rule;       // interface cells without liquid (gas) neighbours empty (fill)
    int pair_ok;       // nx and N even: the float bulk kernel takes two cells per thread
};

// bulk-kernel variants: direct loads, per-thread cp.async pipeline over z,
// TMA-staged rows (needs 16-byte aligned rows)
enum { BULK_PLAIN = 0, BULK_PIPE = 1, BULK_TMA = 2 };

// ---- batched form: many tanks stepped by one launch per kernel
//
// The descriptors of up to BATCH_TANKS tanks travel by value in the kernel
// parameter space (read-only, served by the constant cache); each launch
// walks a packed block table whose entries name a tank and the block of that
// tank's own grid the entry stands for.
constexpr int BATCH_TANKS = 64;
struct TankSet {
    Dev d[BATCH_TANKS];
};
static_assert(sizeof(TankSet) + 64 <= 32764, "tank descriptors must fit the kernel parameter space");

struct Tile {
    uint16_t tank, x, y, z, nx, ny, nz, pad;  // tank; block (x, y, z) of a (nx, ny, nz) grid
};

// block tables by launch shape
enum {
    SH_FORCE = 0,  // (FORCE_BLOCKS, bodies): forces, remap cover / pending
    SH_BULK,       // (ceil(nx / BULK_THREADS), ny, ceil(nz / zb)): bulk stream + collide
    SH_IFACE,      // (2 lb): interface cells
    SH_LIST,       // (lb): conversion worklists, neighbour-bit refresh
    SH_BODY,       // (bodies): rigid-body step
    SH_ONE,        // (1) per tank with bodies: remap resolution
    SH_TANK,       // (1) per tank: counter reset
    SH_COUNT
};
struct Shape {
    const Tile *table;  // device
    unsigned n;         // entries
    unsigned grid;      // blocks of the launch (each walks entries grid apart)
};
struct BatchLaunch {
    const TankSet *ts;  // host copy, passed by value to every launch
    Shape sh[SH_COUNT];
    int zb;             // z-planes per bulk tile
};

struct KernelSet {
    void (*init_cells)(const Dev &, const uint8_t *flags, const double *fill, const double *rho, const double *vel,
                       cudaStream_t);
    void (*body_prepare)(const Dev &, int b, cudaStream_t);
    void (*map_body)(const Dev &, int b, int book_mass, cudaStream_t);
    // one time step, in order; returns the number of kernels launched
    int (*step)(const Dev &, cudaStream_t, float *ev_ms, cudaEvent_t *ev);
    void (*liquid_mass)(const Dev &, cudaStream_t);  // -> ledger[LG_MASS]
    void (*read_fields)(const Dev &, unsigned mask, void *const *dst, cudaStream_t);
    // one time step of every tank of a batch chunk; same event protocol and
    // kernel slots as step
    int (*batch_step)(const BatchLaunch &, cudaStream_t, cudaEvent_t *ev);
    // the bulk kernel alone over a chunk (autotuning), and its occupancy
    void (*batch_bulk)(const BatchLaunch &, cudaStream_t);
    int (*bulk_blocks_per_sm)();
    int nkernels;
    const char *const *names;
};

// cells of an xy-plane per bulk-kernel block: two per thread for the float
// storages on grids with nx and the cell count even, one otherwise
inline int bulk_cells(int storage, const Dev &d) {
    return (storage != 0 && LBMFS_BULK_PAIR && d.pair_ok) ? 2 * BULK_THREADS : BULK_THREADS;
}

// The rigid-body update (double precision, independent of the storage) is
// compiled once, in the unit built without fused multiply-add, and launched
// from there for every storage: its rounding is then the same in every
// kernel set and in single-tank and batched launches.
void launch_bodies(const Dev &d, cudaStream_t st);
void launch_bodies_batch(const BatchLaunch &b, cudaStream_t st);

KernelSet kernels_f64();
KernelSet kernels_f32();
KernelSet kernels_f16s();

}  // namespace lbmfs
