// Host side of the C ABI declared in include/lbm_fs.h: parameter validation,
// device memory, initial upload, step enqueueing (CUDA graphs), read-back.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <cstdlib>
#include <string>
#include <vector>

#include "lbm_fs.h"
#include "lbmfs_handle.h"
#include "lbmfs_internal.h"

using namespace lbmfs;

namespace {
thread_local std::string g_err;
}  // namespace

namespace lbmfs {

lbm_fs_status fail(lbm_fs_status s, const char *fmt, const char *detail) {
    char buf[512];
    snprintf(buf, sizeof buf, fmt, detail ? detail : "");
    g_err = buf;
    return s;
}

lbm_fs_status cuda_fail(cudaError_t e, const char *where) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
    g_err = buf;
    return e == cudaErrorMemoryAllocation ? LBM_FS_ENOMEM : LBM_FS_ECUDA;
}

lbm_fs_status check_handle(lbm_fs *h) {
    if (!h) return fail(LBM_FS_EINVAL, "null handle%s");
    if (h->dead) return fail(LBM_FS_ESTATE, "handle is in a failed state%s");
    return LBM_FS_OK;
}

#define CK LBMFS_CK

lbm_fs_status read_status(lbm_fs *h) {
    uint32_t st = 0;
    CK(cudaMemcpyAsync(&st, h->d[0].status, sizeof st, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return status_bits(st);
}

lbm_fs_status status_bits(uint32_t st) {
    if (st & ST_OVERFLOW) return fail(LBM_FS_EOVERFLOW, "a device worklist overflowed%s");
    if (st & ST_TIMEOUT) return fail(LBM_FS_ETIMEOUT, "a bounded device wait (staged rows) gave up%s");
    if (st & ST_NONFINITE) return fail(LBM_FS_EUNSTABLE, "non-finite or non-positive density in a fluid cell%s");
    if (st & ST_LIQUID_GAS) return fail(LBM_FS_EUNSTABLE, "a liquid cell touched a gas cell (open interface layer)%s");
    if (st & ST_CONTACT) return fail(LBM_FS_EUNSTABLE, "a moving body reached a domain wall (body-wall contact is not modelled)%s");
    if (st & ST_TOP) return fail(LBM_FS_EUNSTABLE, "fluid appeared above the bulk kernel's tracked fluid top%s");
    return LBM_FS_OK;
}

void begin_mass(lbm_fs *h) {
    if (h->started) return;
    h->ks.liquid_mass(h->d[h->cur], h->st);
    cudaMemcpyAsync(h->d[0].ledger + LG_MASS0, h->d[0].ledger + LG_MASS, sizeof(double), cudaMemcpyDeviceToDevice,
                    h->st);
    h->started = true;
}

}  // namespace lbmfs

namespace {

lbm_fs_status capture_graphs(lbm_fs *h) {
    for (int k = 0; k < 2; ++k) {
        if (h->gexec[k]) {
            cudaGraphExecDestroy(h->gexec[k]);
            h->gexec[k] = nullptr;
        }
    }
    for (int k = 0; k < 2; ++k) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal));
        h->per_step = h->ks.step(h->d[k], h->cap_st, nullptr, nullptr);
        cudaError_t e = cudaStreamEndCapture(h->cap_st, &g);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&h->gexec[k], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    }
    h->graph_nb = h->nb;
    return LBM_FS_OK;
}

void set_grids(lbm_fs *h, void *fA, void *fB, double *pA, double *pB) {
    h->d[0].fsrc = fA;
    h->d[0].fdst = fB;
    h->d[0].phisrc = pA;
    h->d[0].phidst = pB;
    h->d[1].fsrc = fB;
    h->d[1].fdst = fA;
    h->d[1].phisrc = pB;
    h->d[1].phidst = pA;
}

size_t storage_bytes(int storage, long long N) {
    switch (storage) {
        case LBM_FS_F64: return (size_t)N * Q * 8;
        case LBM_FS_F32: return (size_t)N * Q * 4;
        default: return (size_t)N * (4 + (Q - 1) * 2);
    }
}

}  // namespace

extern "C" {

int32_t lbm_fs_version(void) { return 1; }

const char *lbm_fs_last_error_string(void) { return g_err.c_str(); }

lbm_fs_status lbm_fs_create(const lbm_fs_params *p, lbm_fs **out) {
    if (!p || !out) return fail(LBM_FS_EINVAL, "null argument%s");
    *out = nullptr;
    if (p->nx <= 0 || p->ny <= 0 || p->nz <= 0) return fail(LBM_FS_EINVAL, "grid sizes must be positive%s");
    long long N = (long long)p->nx * p->ny * p->nz;
    if (N >= 0xFFFFFFFFll) return fail(LBM_FS_EINVAL, "grid has 2^32 cells or more%s");
    // the float storages' bulk kernel indexes a population as q N + cell in 32 bits
    if (p->storage != LBM_FS_F64 && N * Q >= 0xFFFFFFFFll)
        return fail(LBM_FS_EINVAL, "float storages take fewer than 2^32 / 19 cells%s");
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return fail(LBM_FS_EINVAL, "tau must exceed 1/2%s");
    if (p->storage < LBM_FS_F64 || p->storage > LBM_FS_F16S) return fail(LBM_FS_EINVAL, "unknown storage%s");
    if (!p->init_flags || !p->init_fill || !p->init_rho) return fail(LBM_FS_EINVAL, "init_flags, init_fill and init_rho are required%s");
    if (!(p->rho_gas > 0.0) || !(p->eps >= 0.0)) return fail(LBM_FS_EINVAL, "rho_gas must be positive and eps non-negative%s");
    if ((p->dev_alloc == nullptr) != (p->dev_free == nullptr)) return fail(LBM_FS_EINVAL, "dev_alloc and dev_free go together%s");
    if (!(p->sigma >= 0.0) || !std::isfinite(p->sigma)) return fail(LBM_FS_EINVAL, "sigma must be finite and >= 0%s");
    for (int f = 0; f < 6; ++f)
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(p->wall_vel[f][k])) return fail(LBM_FS_EINVAL, "non-finite wall velocity%s");
    const bool rd_db = p->readings & LBM_FS_READING_DEADBAND, rd_vm = p->readings & LBM_FS_READING_VIRTUAL_MASS;
    if (rd_db && !(p->normal_deadband >= 0.0 && std::isfinite(p->normal_deadband)))
        return fail(LBM_FS_EINVAL, "normal_deadband must be finite and >= 0%s");
    if (rd_vm && !(p->virtual_mass >= 0.0 && std::isfinite(p->virtual_mass)))
        return fail(LBM_FS_EINVAL, "virtual_mass must be finite and >= 0%s");
    double proj = 0.0;
    for (int k = 0; k < 3; ++k) {
        double a = fabs(p->gravity[k] + p->body_accel[k]);
        if (!std::isfinite(a)) return fail(LBM_FS_EINVAL, "non-finite acceleration%s");
        proj += a * (k == 0 ? p->nx : (k == 1 ? p->ny : p->nz));
    }
    // Sec. 2.1 incompressibility condition (l_x, l_y, l_z) . a << c_s^2 = 1/3
    if (proj >= 1.0 / 3.0) return fail(LBM_FS_EINVAL, "(nx, ny, nz) . |a| must stay well below c_s^2 = 1/3%s");

    lbm_fs *h = new lbm_fs();
    h->p = *p;
    h->p.init_flags = nullptr;
    h->p.init_fill = nullptr;
    h->p.init_rho = nullptr;
    h->p.init_vel = nullptr;
    h->st = (cudaStream_t)p->stream;
    switch (p->storage) {
        case LBM_FS_F64: h->ks = kernels_f64(); break;
        case LBM_FS_F32: h->ks = kernels_f32(); break;
        default: h->ks = kernels_f16s(); break;
    }
    auto bail = [&](lbm_fs_status s) {
        h->release();
        delete h;
        return s;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate"));

    Dev d{};
    d.nx = p->nx;
    d.ny = p->ny;
    d.nz = p->nz;
    d.periodic = p->periodic & 7u;
    d.N = N;
    d.omega = 1.0 / p->tau;
    for (int k = 0; k < 3; ++k) {
        d.a[k] = p->gravity[k] + p->body_accel[k];
        d.grav[k] = p->gravity[k];
    }
    d.rho_g = p->rho_gas;
    d.eps = p->eps;
    d.omega_f = (float)d.omega;
    for (int k = 0; k < 3; ++k) d.a_f[k] = (float)d.a[k];
    d.drg_f = (float)(d.rho_g - 1.0);
    d.rg1_f = (float)(1.0 - d.rho_g);
    d.sigma = p->sigma;
    d.sigma_f = (float)p->sigma;
    d.cap = (uint32_t)N;
    d.deadband = rd_db ? p->normal_deadband : 1e-2;
    d.deadband_f = (float)d.deadband;
    d.vmass = rd_vm ? p->virtual_mass : 1.0;
    d.force_mean = (p->readings & LBM_FS_READING_FORCE_MEAN) ? (p->force_mean != 0) : 1;
    d.nb_rule = (p->readings & LBM_FS_READING_NEIGHBOUR_RULE) ? (p->neighbour_rule != 0) : 1;
    d.pair_ok = p->storage != LBM_FS_F64 && p->nx % 2 == 0 && N % 2 == 0;
    // row segments are 16-byte aligned when nx is a multiple of 16 / element size
    // bulk-kernel variant (float storages): direct loads by default;
    // LBMFS_BULK=pipe|tma selects the shared-memory staged variants (both
    // measured slower on GB300; the TMA one needs rows of 16-byte multiples)
    d.bulk = BULK_PLAIN;
    if (const char *v = getenv("LBMFS_BULK")) {
        if (!strcmp(v, "pipe")) d.bulk = BULK_PIPE;
        else if (!strcmp(v, "tma")) d.bulk = BULK_TMA;
    }
    if (d.bulk == BULK_TMA &&
        !((p->storage == LBM_FS_F32 && p->nx % 4 == 0) || (p->storage == LBM_FS_F16S && p->nx % 8 == 0)))
        d.bulk = BULK_PLAIN;
    size_t fb = storage_bytes(p->storage, N);
    size_t nb4 = ((size_t)N + 3) & ~(size_t)3;
    d.flags = (uint8_t *)h->alloc(nb4);
    d.bid = (uint8_t *)h->alloc(nb4);
    d.cmark = (uint8_t *)h->alloc(nb4);
    // population grids with guard bands: the staged bulk kernel reads a
    // 16-byte halo around each row segment, which at the grid's first and
    // last rows reaches past the population array
    void *fA = h->alloc(fb + 2 * GRID_GUARD), *fB = h->alloc(fb + 2 * GRID_GUARD);
    if (fA) fA = (char *)fA + GRID_GUARD;
    if (fB) fB = (char *)fB + GRID_GUARD;
    double *pA = (double *)h->alloc(N * 8), *pB = (double *)h->alloc(N * 8);
    d.m = (double *)h->alloc(N * 8);
    for (int k = 0; k < WL_COUNT; ++k) d.list[k] = (uint32_t *)h->alloc(N * 4);
    d.cnt = (uint32_t *)h->alloc(WL_COUNT * 4);
    d.bodies = (Body *)h->alloc(sizeof(Body) * MAX_BODIES);
    d.part = (double *)h->alloc(2 * sizeof(double) * MAX_BODIES * FORCE_BLOCKS * 7);
    d.part128 = p->storage == LBM_FS_F64;
    d.ledger = (double *)h->alloc(sizeof(double) * LG_COUNT);
    d.status = (uint32_t *)h->alloc(4);
    d.rdec = (uint8_t *)h->alloc(nb4);
    d.rrho = (double *)h->alloc(N * 8);
    d.rphi = (double *)h->alloc(N * 8);
    d.red = (double *)h->alloc(sizeof(double) * LIST_BLOCKS);
    double *wallv = (double *)h->alloc(sizeof(double) * 18);
    d.wallv = wallv;
    int *ztop = (int *)h->alloc(sizeof(int) * 2);
    for (void *ptr : h->allocs)
        if (!ptr) return bail(fail(LBM_FS_ENOMEM, "device allocation failed%s"));
    if (h->allocs.size() != 19 + WL_COUNT) return bail(fail(LBM_FS_ENOMEM, "device allocation failed%s"));
    if (h->misaligned) return bail(fail(LBM_FS_EINVAL, "dev_alloc must return 16-byte aligned memory%s"));
    d.walls_move = 0;
    for (int f = 0; f < 6; ++f)
        for (int k = 0; k < 3; ++k)
            if (p->wall_vel[f][k] != 0.0 && !(d.periodic & (1u << (f / 2)))) d.walls_move = 1;
    cudaStream_t st = h->st;
#define CKB(call)                                                   \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return bail(cuda_fail(e_, #call));   \
    } while (0)
    CKB(cudaMemsetAsync(d.cmark, 0, nb4, st));
    CKB(cudaMemsetAsync((char *)fA - GRID_GUARD, 0, fb + 2 * GRID_GUARD, st));
    CKB(cudaMemsetAsync((char *)fB - GRID_GUARD, 0, fb + 2 * GRID_GUARD, st));
    CKB(cudaMemsetAsync(pA, 0, N * 8, st));
    CKB(cudaMemsetAsync(pB, 0, N * 8, st));
    CKB(cudaMemsetAsync(d.m, 0, N * 8, st));
    CKB(cudaMemsetAsync(d.cnt, 0, WL_COUNT * 4, st));
    CKB(cudaMemsetAsync(d.ledger, 0, sizeof(double) * LG_COUNT, st));
    CKB(cudaMemsetAsync(d.status, 0, 4, st));
    CKB(cudaMemsetAsync(d.part, 0, 2 * sizeof(double) * MAX_BODIES * FORCE_BLOCKS * 7, st));
    CKB(cudaMemcpyAsync(wallv, &p->wall_vel[0][0], sizeof(double) * 18, cudaMemcpyHostToDevice, st));
    // the first step visits every tile (its read slot: nz) and records the top
    const int zt0[2] = {p->nz, -1};
    CKB(cudaMemcpyAsync(ztop, zt0, sizeof zt0, cudaMemcpyHostToDevice, st));
    h->d[0] = d;
    h->d[1] = d;
    set_grids(h, fA, fB, pA, pB);
    h->d[0].ztop_rd = ztop;
    h->d[0].ztop_wr = ztop + 1;
    h->d[1].ztop_rd = ztop + 1;
    h->d[1].ztop_wr = ztop;

    // upload the initial state (staged through temporary device buffers)
    const uint8_t *dfl = p->init_flags;
    const double *dfi = p->init_fill, *drh = p->init_rho, *dvl = p->init_vel;
    void *tmp = nullptr;
    if (!p->init_on_device) {
        size_t bytes = (size_t)N * (1 + 8 + 8) + (p->init_vel ? (size_t)N * 24 : 0) + 64;
        CKB(cudaMalloc(&tmp, bytes));
        char *c = (char *)tmp;
        double *tfi = (double *)c;
        double *trh = tfi + N;
        double *tvl = p->init_vel ? trh + N : nullptr;
        uint8_t *tfl = (uint8_t *)(p->init_vel ? tvl + 3 * N : trh + N);
        CKB(cudaMemcpyAsync(tfl, p->init_flags, N, cudaMemcpyHostToDevice, st));
        CKB(cudaMemcpyAsync(tfi, p->init_fill, N * 8, cudaMemcpyHostToDevice, st));
        CKB(cudaMemcpyAsync(trh, p->init_rho, N * 8, cudaMemcpyHostToDevice, st));
        if (tvl) CKB(cudaMemcpyAsync(tvl, p->init_vel, N * 24, cudaMemcpyHostToDevice, st));
        dfl = tfl;
        dfi = tfi;
        drh = trh;
        dvl = tvl;
    }
    h->ks.init_cells(h->d[0], dfl, dfi, drh, dvl, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return bail(cuda_fail(e, "initial upload"));
#undef CKB
    *out = h;
    return LBM_FS_OK;
}

lbm_fs_status lbm_fs_destroy(lbm_fs *h) {
    if (!h) return fail(LBM_FS_EINVAL, "null handle%s");
    if (h->owner) return fail(LBM_FS_ESTATE, "the tank belongs to a batch (lbm_fs_batch_destroy frees it)%s");
    cudaStreamSynchronize(h->st);
    h->release();
    delete h;
    return LBM_FS_OK;
}

lbm_fs_status lbm_fs_add_box(lbm_fs *h, const lbm_fs_box *b, int32_t *out_id) {
    lbm_fs_status s = check_handle(h);
    if (s) return s;
    if (!b) return fail(LBM_FS_EINVAL, "null box%s");
    if (h->nb >= MAX_BODIES) return fail(LBM_FS_EINVAL, "at most 255 boxes%s");
    for (int k = 0; k < 3; ++k)
        if (!(b->half[k] > 0.0) || !std::isfinite(b->center[k])) return fail(LBM_FS_EINVAL, "box half extents must be positive%s");
    double qn = std::sqrt(b->quat[0] * b->quat[0] + b->quat[1] * b->quat[1] + b->quat[2] * b->quat[2] + b->quat[3] * b->quat[3]);
    if (!(qn > 0.5 && qn < 2.0)) return fail(LBM_FS_EINVAL, "quaternion must be (close to) unit%s");
    if (!(b->density_ratio > 0.0)) return fail(LBM_FS_EINVAL, "density_ratio must be positive%s");
    int base = b->mode & 0xff;
    if (base > 2 || (b->mode & ~0x1ff)) return fail(LBM_FS_EINVAL, "unknown mode%s");
    if (b->shape != 0 && b->shape != 1) return fail(LBM_FS_EINVAL, "unknown shape%s");
    Body hb;
    memset(&hb, 0, sizeof hb);
    for (int k = 0; k < 3; ++k) {
        hb.o[k] = b->center[k];
        hb.h[k] = b->half[k];
        hb.v[k] = b->vel[k];
        hb.w[k] = b->omega[k];
        hb.axis[k] = b->rot_axis[k];
    }
    for (int k = 0; k < 4; ++k) hb.q[k] = b->quat[k];
    hb.dens = b->density_ratio;
    hb.damp = b->lin_damping;
    hb.mode = b->mode;
    hb.shape = b->shape;
    int id = h->nb;
    cudaStream_t st = h->st;
    CK(cudaMemcpyAsync(h->d[0].bodies + id, &hb, sizeof hb, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    h->nb++;
    for (int k = 0; k < 2; ++k) h->d[k].nb = h->nb;
    h->ks.body_prepare(h->d[h->cur], id, st);
    h->ks.map_body(h->d[h->cur], id, h->started ? 1 : 0, st);
    CK(cudaGetLastError());
    if (out_id) *out_id = id;
    return LBM_FS_OK;
}

lbm_fs_status lbm_fs_step(lbm_fs *h, int32_t nsteps) {
    lbm_fs_status s = check_handle(h);
    if (s) return s;
    if (h->owner) return fail(LBM_FS_ESTATE, "the tank belongs to a batch (step it with lbm_fs_batch_step)%s");
    if (nsteps < 0) return fail(LBM_FS_EINVAL, "nsteps must be >= 0%s");
    if (nsteps == 0) return LBM_FS_OK;
    cudaStream_t st = h->st;
    begin_mass(h);
    CK(cudaGetLastError());
    if (h->p.use_graphs && h->graph_nb != h->nb) {
        s = capture_graphs(h);
        if (s) return s;
    }
    for (int32_t k = 0; k < nsteps; ++k) {
        if (h->p.use_graphs) {
            CK(cudaGraphLaunch(h->gexec[h->cur], st));
        } else {
            h->per_step = h->ks.step(h->d[h->cur], st, nullptr, nullptr);
            CK(cudaGetLastError());
        }
        h->launches += h->per_step;
        h->cur ^= 1;
        h->step++;
    }
    return LBM_FS_OK;
}

lbm_fs_status lbm_fs_sync(lbm_fs *h) {
    lbm_fs_status s = check_handle(h);
    if (s) return s;
    return read_status(h);
}

lbm_fs_status lbm_fs_body_state(lbm_fs *h, int32_t id, lbm_fs_body_state_t *out) {
    lbm_fs_status s = check_handle(h);
    if (s) return s;
    if (id < 0 || id >= h->nb || !out) return fail(LBM_FS_EINVAL, "bad body id%s");
    CK(cudaStreamSynchronize(h->st));
    Body hb;
    CK(cudaMemcpy(&hb, h->d[0].bodies + id, sizeof hb, cudaMemcpyDeviceToHost));
    for (int k = 0; k < 3; ++k) {
        out->F[k] = hb.F[k];
        out->T[k] = hb.T[k];
        out->center[k] = hb.o[k];
        out->vel[k] = hb.v[k];
        out->omega[k] = hb.w[k];
    }
    for (int k = 0; k < 4; ++k) out->quat[k] = hb.q[k];
    out->S = hb.S;
    return read_status(h);
}

lbm_fs_status lbm_fs_body_states(lbm_fs *h, int32_t first, int32_t count, lbm_fs_body_state_t *out) {
    lbm_fs_status s = check_handle(h);
    if (s) return s;
    if (first < 0 || count < 0 || first + count > h->nb || (count > 0 && !out))
        return fail(LBM_FS_EINVAL, "bad body range%s");
    if (count == 0) return read_status(h);
    std::vector<Body> hb(count);
    uint32_t st = 0;  // the status word comes with the bodies: one synchronisation
    CK(cudaMemcpyAsync(hb.data(), h->d[0].bodies + first, sizeof(Body) * count, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(&st, h->d[0].status, sizeof st, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    for (int32_t b = 0; b < count; ++b) {
        for (int k = 0; k < 3; ++k) {
            out[b].F[k] = hb[b].F[k];
            out[b].T[k] = hb[b].T[k];
            out[b].center[k] = hb[b].o[k];
            out[b].vel[k] = hb[b].v[k];
            out[b].omega[k] = hb[b].w[k];
        }
        for (int k = 0; k < 4; ++k) out[b].quat[k] = hb[b].q[k];
        out[b].S = hb[b].S;
    }
    return status_bits(st);
}

lbm_fs_status lbm_fs_forces(lbm_fs *h, int32_t id, double F[3], double T[3], double center[3], double quat[4]) {
    lbm_fs_body_state_t bs;
    lbm_fs_status s = lbm_fs_body_state(h, id, &bs);
    if (s != LBM_FS_OK && s != LBM_FS_EUNSTABLE && s != LBM_FS_EOVERFLOW) return s;
    for (int k = 0; k < 3; ++k) {
        if (F) F[k] = bs.F[k];
        if (T) T[k] = bs.T[k];
        if (center) center[k] = bs.center[k];
    }
    if (quat)
        for (int k = 0; k < 4; ++k) quat[k] = bs.quat[k];
    return s;
}

lbm_fs_status lbm_fs_read_fields(lbm_fs *h, uint32_t mask, void *const *dst, int32_t dst_on_device) {
    lbm_fs_status s = check_handle(h);
    if (s) return s;
    if (!dst || (mask & ~63u)) return fail(LBM_FS_EINVAL, "bad field mask or destination%s");
    for (int k = 0; k < 6; ++k)
        if ((mask & (1u << k)) && !dst[k]) return fail(LBM_FS_EINVAL, "missing destination buffer%s");
    const long long N = h->d[0].N;
    const size_t sz[6] = {(size_t)N, (size_t)N * 8, (size_t)N * 8, (size_t)N * 8, (size_t)N * 24, (size_t)N * 8 * Q};
    cudaStream_t st = h->st;
    void *ddst[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    std::vector<void *> tmp;
    for (int k = 0; k < 6; ++k) {
        if (!(mask & (1u << k))) continue;
        if (dst_on_device) {
            ddst[k] = dst[k];
        } else {
            void *ptr = nullptr;
            cudaError_t e = cudaMalloc(&ptr, sz[k]);
            if (e != cudaSuccess) {
                for (void *t : tmp) cudaFree(t);
                return cuda_fail(e, "read_fields staging");
            }
            tmp.push_back(ptr);
            ddst[k] = ptr;
        }
    }
    h->ks.read_fields(h->d[h->cur], mask, ddst, st);
    cudaError_t e = cudaGetLastError();
    for (int k = 0; k < 6 && e == cudaSuccess; ++k)
        if (!dst_on_device && (mask & (1u << k))) e = cudaMemcpyAsync(dst[k], ddst[k], sz[k], cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (void *t : tmp) cudaFree(t);
    if (e != cudaSuccess) return cuda_fail(e, "read_fields");
    return read_status(h);
}

lbm_fs_status lbm_fs_stats(lbm_fs *h, lbm_fs_stats_t *out) {
    lbm_fs_status s = check_handle(h);
    if (s) return s;
    if (!out) return fail(LBM_FS_EINVAL, "null output%s");
    cudaStream_t st = h->st;
    h->ks.liquid_mass(h->d[h->cur], st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    double lg[LG_COUNT];
    uint32_t cnt[WL_COUNT], status;
    CK(cudaMemcpy(lg, h->d[0].ledger, sizeof lg, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(cnt, h->d[0].cnt, sizeof cnt, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&status, h->d[0].status, sizeof status, cudaMemcpyDeviceToHost));
    memset(out, 0, sizeof *out);
    out->step = h->step;
    out->liquid_mass = lg[LG_MASS];
    out->mass0 = h->started ? lg[LG_MASS0] : lg[LG_MASS];
    out->covered = lg[LG_COVERED];
    out->uncovered = lg[LG_UNCOVERED];
    out->lost_excess = lg[LG_LOST];
    out->n_interface = cnt[WL_IFACE];
    out->n_filled = cnt[WL_FILLED];
    out->n_emptied = cnt[WL_EMPTIED];
    out->n_new_from_gas = cnt[WL_NEWG];
    out->n_new_from_liquid = cnt[WL_NEWL];
    out->n_pending = cnt[WL_PEND];
    out->status = status;
    out->kernel_launches = h->launches;
    out->wall_source = lg[LG_WALL];
    out->n_general = cnt[WL_GEN];
    return read_status(h);
}

lbm_fs_status lbm_fs_kernel_times(lbm_fs *h, int32_t nsteps, double *ms, const char **names, int32_t cap, int32_t *nk) {
    lbm_fs_status s = check_handle(h);
    if (s) return s;
    if (h->owner) return fail(LBM_FS_ESTATE, "the tank belongs to a batch (use lbm_fs_batch_kernel_times)%s");
    if (nsteps <= 0 || !ms || cap <= 0) return fail(LBM_FS_EINVAL, "bad arguments%s");
    const int K = h->ks.nkernels;
    std::vector<cudaEvent_t> ev(K + 1);
    for (auto &x : ev) CK(cudaEventCreate(&x));
    std::vector<double> acc(K, 0.0);
    cudaStream_t st = h->st;
    begin_mass(h);
    CK(cudaGetLastError());
    for (int32_t it = 0; it < nsteps; ++it) {
        int n = h->ks.step(h->d[h->cur], st, nullptr, ev.data());
        CK(cudaGetLastError());
        CK(cudaEventSynchronize(ev[K]));
        for (int k = 0; k < K; ++k) {
            float t = 0.0f;
            CK(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
            acc[k] += t;
        }
        h->launches += n;
        h->cur ^= 1;
        h->step++;
    }
    for (auto &x : ev) cudaEventDestroy(x);
    int m = K < cap ? K : cap;
    for (int k = 0; k < m; ++k) {
        ms[k] = acc[k];
        if (names) names[k] = h->ks.names[k];
    }
    if (nk) *nk = K;
    return read_status(h);
}

}  // extern "C"
