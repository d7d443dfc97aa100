// Host side of the batched form declared in include/lbm_fs.h: many tanks, each
// an ordinary simulation handle, stepped by one launch per kernel over packed
// (tank, block) tables, with the step captured in CUDA graphs and the bulk
// tiling picked by timing candidates on the GPU.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <string>
#include <vector>

#include "lbm_fs.h"
#include "lbmfs_handle.h"
#include "lbmfs_internal.h"

using namespace lbmfs;

#define CK LBMFS_CK

namespace {

constexpr int ZB_DEFAULT = 4;
constexpr int LIST_CELLS_DEFAULT = 512;
constexpr int LANES_DEFAULT = 1;

constexpr int MAX_LANES = 4;

// a group of at most BATCH_TANKS tanks served by the same launches
struct Chunk {
    std::vector<int> idx;  // the batch's tank indices, in descriptor order
    int lane = 0;          // concurrent chain the chunk's launches belong to
    TankSet ts[2];         // descriptors for even / odd steps
    Shape sh[SH_COUNT];
};

}  // namespace

struct lbm_fs_batch {
    std::vector<lbm_fs *> tanks;
    KernelSet ks;
    cudaStream_t st = nullptr;
    cudaStream_t cap_st = nullptr;
    bool use_graphs = true;
    int zb = ZB_DEFAULT;
    int bulk_blocks = 0;  // 0: one block per bulk tile
    int list_cells = LIST_CELLS_DEFAULT;
    int lanes = 1;  // groups of tanks whose step chains run concurrently
    cudaStream_t lane_st[MAX_LANES] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[MAX_LANES] = {};
    std::vector<std::unique_ptr<Chunk>> chunks;
    std::vector<int> nb_built;  // bodies per tank when the tables were built
    bool built = false;
    void *tables = nullptr;
    size_t table_cap = 0;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int per_step = 0;
    int cur = 0;
    int64_t step = 0, launches = 0;
    int sms = 0;
    void *(*dev_alloc)(size_t, void *) = nullptr;
    void (*dev_free)(void *, void *) = nullptr;
    void *alloc_ctx = nullptr;

    void *alloc(size_t bytes) {
        void *p = nullptr;
        if (dev_alloc) return dev_alloc(bytes, alloc_ctx);
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void free_(void *p) {
        if (!p) return;
        if (dev_free) dev_free(p, alloc_ctx);
        else cudaFree(p);
    }
    void drop_graphs() {
        for (auto &g : gexec) {
            if (g) cudaGraphExecDestroy(g);
            g = nullptr;
        }
    }
};

namespace {

lbm_fs_status check_batch(lbm_fs_batch *b) {
    if (!b) return fail(LBM_FS_EINVAL, "null batch%s");
    return LBM_FS_OK;
}

int list_blocks(const lbm_fs *t, int list_cells) {
    long long area = (long long)t->d[0].nx * t->d[0].ny;
    long long n = (area + list_cells - 1) / list_cells;
    return (int)std::min<long long>(std::max<long long>(n, 1), LIST_BLOCKS);
}

Tile tile(int tank, int x, int y, int z, int nx, int ny, int nz) {
    Tile t;
    t.tank = (uint16_t)tank;
    t.x = (uint16_t)x;
    t.y = (uint16_t)y;
    t.z = (uint16_t)z;
    t.nx = (uint16_t)nx;
    t.ny = (uint16_t)ny;
    t.nz = (uint16_t)nz;
    t.pad = 0;
    return t;
}

// (Re)build the tank descriptors and block tables of every chunk for the
// current bodies and configuration, and upload the tables.
lbm_fs_status build(lbm_fs_batch *b) {
    std::vector<Tile> all;
    std::vector<size_t> offs;  // per chunk and shape: first entry in `all`
    const int nt = (int)b->tanks.size();
    b->nb_built.assign(nt, 0);
    for (auto &cp : b->chunks) {
        Chunk &c = *cp;
        for (int k = 0; k < 2; ++k) {
            memset(&c.ts[k], 0, sizeof(TankSet));
            for (int j = 0; j < (int)c.idx.size(); ++j) c.ts[k].d[j] = b->tanks[c.idx[j]]->d[k];
        }
        std::vector<Tile> tb[SH_COUNT];
        for (int j = 0; j < (int)c.idx.size(); ++j) {
            const lbm_fs *t = b->tanks[c.idx[j]];
            const Dev &d = t->d[0];
            const int nb = t->nb;
            b->nb_built[c.idx[j]] = nb;
            tb[SH_TANK].push_back(tile(j, 0, 0, 0, 1, 1, 1));
            for (int y = 0; y < nb; ++y)
                for (int x = 0; x < FORCE_BLOCKS; ++x) tb[SH_FORCE].push_back(tile(j, x, y, 0, FORCE_BLOCKS, nb, 1));
            const int bc = bulk_cells(t->p.storage, d);
            const int gx = (int)(((long long)d.nx * d.ny + bc - 1) / bc);
            const int gz = (d.nz + b->zb - 1) / b->zb;
            for (int z = 0; z < gz; ++z)
                for (int x = 0; x < gx; ++x) tb[SH_BULK].push_back(tile(j, x, 0, z, gx, 1, gz));
            const int lb = list_blocks(t, b->list_cells);
            for (int x = 0; x < 2 * lb; ++x) tb[SH_IFACE].push_back(tile(j, x, 0, 0, 2 * lb, 1, 1));
            for (int x = 0; x < lb; ++x) tb[SH_LIST].push_back(tile(j, x, 0, 0, lb, 1, 1));
            for (int x = 0; x < nb; ++x) tb[SH_BODY].push_back(tile(j, x, 0, 0, nb, 1, 1));
            if (nb > 0) tb[SH_ONE].push_back(tile(j, 0, 0, 0, 1, 1, 1));
        }
        for (int s = 0; s < SH_COUNT; ++s) {
            offs.push_back(all.size());
            all.insert(all.end(), tb[s].begin(), tb[s].end());
            c.sh[s].n = (unsigned)tb[s].size();
            unsigned grid = c.sh[s].n;
            if (s == SH_BULK && b->bulk_blocks > 0) grid = std::min<unsigned>(grid, (unsigned)b->bulk_blocks);
            c.sh[s].grid = grid;
            c.sh[s].table = nullptr;
        }
    }
    size_t bytes = std::max<size_t>(all.size(), 1) * sizeof(Tile);
    if (bytes > b->table_cap) {
        CK(cudaStreamSynchronize(b->st));
        b->free_(b->tables);
        b->tables = b->alloc(bytes);
        b->table_cap = b->tables ? bytes : 0;
        if (!b->tables) return fail(LBM_FS_ENOMEM, "batch table allocation failed%s");
    }
    CK(cudaMemcpyAsync(b->tables, all.data(), all.size() * sizeof(Tile), cudaMemcpyHostToDevice, b->st));
    CK(cudaStreamSynchronize(b->st));
    size_t q = 0;
    for (auto &cp : b->chunks)
        for (int s = 0; s < SH_COUNT; ++s) cp->sh[s].table = (const Tile *)b->tables + offs[q++];
    b->built = true;
    b->drop_graphs();
    return LBM_FS_OK;
}

bool stale(lbm_fs_batch *b) {
    if (!b->built) return true;
    for (size_t k = 0; k < b->tanks.size(); ++k)
        if (b->tanks[k]->nb != b->nb_built[k]) return true;
    return false;
}

BatchLaunch launch_of(lbm_fs_batch *b, Chunk &c, int parity) {
    BatchLaunch L;
    L.ts = &c.ts[parity];
    for (int s = 0; s < SH_COUNT; ++s) L.sh[s] = c.sh[s];
    L.zb = b->zb;
    return L;
}

// Split the tanks into b->lanes groups of about equal cell count (largest
// first, each to the lightest group) and the groups into chunks of at most
// BATCH_TANKS tanks.
void make_chunks(lbm_fs_batch *b) {
    const int nt = (int)b->tanks.size();
    std::vector<int> order(nt);
    for (int k = 0; k < nt; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->tanks[a]->d[0].N > b->tanks[c]->d[0].N; });
    std::vector<std::vector<int>> lane(b->lanes);
    std::vector<long long> load(b->lanes, 0);
    for (int k : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lane[l].push_back(k);
        load[l] += b->tanks[k]->d[0].N;
    }
    b->chunks.clear();
    for (int l = 0; l < b->lanes; ++l) {
        std::sort(lane[l].begin(), lane[l].end());
        for (size_t first = 0; first < lane[l].size(); first += BATCH_TANKS) {
            auto c = std::make_unique<Chunk>();
            c->lane = l;
            c->idx.assign(lane[l].begin() + first, lane[l].begin() + std::min(lane[l].size(), first + BATCH_TANKS));
            b->chunks.push_back(std::move(c));
        }
    }
    b->built = false;
}

// One step of every tank.  With several lanes the lanes' launch chains fork
// from st and join back into it, so their kernels may run at the same time
// (one lane's short list kernels beside another's bulk kernel).
int enqueue_step(lbm_fs_batch *b, int parity, cudaStream_t st) {
    int n = 0;
    if (b->lanes == 1) {
        for (auto &cp : b->chunks) n += b->ks.batch_step(launch_of(b, *cp, parity), st, nullptr);
        return n;
    }
    cudaEventRecord(b->fork_ev, st);
    for (int l = 0; l < b->lanes; ++l) {
        cudaStreamWaitEvent(b->lane_st[l], b->fork_ev, 0);
        for (auto &cp : b->chunks)
            if (cp->lane == l) n += b->ks.batch_step(launch_of(b, *cp, parity), b->lane_st[l], nullptr);
        cudaEventRecord(b->join_ev[l], b->lane_st[l]);
        cudaStreamWaitEvent(st, b->join_ev[l], 0);
    }
    return n;
}

lbm_fs_status capture(lbm_fs_batch *b) {
    b->drop_graphs();
    for (int k = 0; k < 2; ++k) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(b->cap_st, cudaStreamCaptureModeThreadLocal));
        b->per_step = enqueue_step(b, k, b->cap_st);
        cudaError_t e = cudaStreamEndCapture(b->cap_st, &g);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture (batch)");
        e = cudaGraphInstantiate(&b->gexec[k], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate (batch)");
    }
    return LBM_FS_OK;
}

lbm_fs_status prepare(lbm_fs_batch *b) {
    for (lbm_fs *t : b->tanks) {
        begin_mass(t);
        CK(cudaGetLastError());
    }
    if (stale(b)) {
        lbm_fs_status s = build(b);
        if (s) return s;
    }
    return LBM_FS_OK;
}

void advance(lbm_fs_batch *b, int per_step) {
    b->launches += per_step;
    b->cur ^= 1;
    b->step++;
    for (lbm_fs *t : b->tanks) {
        t->cur = b->cur;
        t->step++;
    }
}

void destroy_all(lbm_fs_batch *b) {
    if (b->st) cudaStreamSynchronize(b->st);
    b->drop_graphs();
    b->free_(b->tables);
    for (lbm_fs *t : b->tanks) {
        t->owner = nullptr;
        lbm_fs_destroy(t);
    }
    if (b->cap_st) cudaStreamDestroy(b->cap_st);
    for (int l = 0; l < MAX_LANES; ++l) {
        if (b->lane_st[l]) cudaStreamDestroy(b->lane_st[l]);
        if (b->join_ev[l]) cudaEventDestroy(b->join_ev[l]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    delete b;
}

}  // namespace

extern "C" {

lbm_fs_status lbm_fs_batch_create(const lbm_fs_params *params, int32_t count, lbm_fs_batch **out) {
    if (!params || !out || count <= 0) return fail(LBM_FS_EINVAL, "batch needs params, out and count > 0%s");
    *out = nullptr;
    for (int32_t k = 0; k < count; ++k) {
        const lbm_fs_params &p = params[k];
        if (p.storage != params[0].storage) return fail(LBM_FS_EINVAL, "all tanks of a batch share one storage%s");
        if (p.nx <= 0 || p.ny <= 0 || p.nz <= 0 || p.nx > 65535 || p.ny > 65535 || p.nz > 65535 ||
            (long long)p.nx * p.ny > 65535ll * BULK_THREADS)
            return fail(LBM_FS_EINVAL, "batch tanks need 1..65535 cells per axis and nx*ny <= 8388480%s");
    }
    lbm_fs_batch *b = new lbm_fs_batch();
    b->st = (cudaStream_t)params[0].stream;
    b->use_graphs = params[0].use_graphs != 0;
    b->dev_alloc = params[0].dev_alloc;
    b->dev_free = params[0].dev_free;
    b->alloc_ctx = params[0].alloc_ctx;
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap_st, cudaStreamNonBlocking);
    for (int l = 0; l < MAX_LANES && e == cudaSuccess; ++l) {
        e = cudaStreamCreateWithFlags(&b->lane_st[l], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev[l], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        destroy_all(b);
        return cuda_fail(e, "cudaStreamCreate (batch)");
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    for (int32_t k = 0; k < count; ++k) {
        lbm_fs_params p = params[k];
        p.stream = params[0].stream;
        p.use_graphs = 0;
        lbm_fs *t = nullptr;
        lbm_fs_status s = lbm_fs_create(&p, &t);
        if (s) {
            char buf[64];
            snprintf(buf, sizeof buf, " (tank %d)", (int)k);
            std::string msg = std::string(lbm_fs_last_error_string()) + buf;
            destroy_all(b);
            return fail(s, "%s", msg.c_str());
        }
        t->owner = b;
        b->tanks.push_back(t);
    }
    b->ks = b->tanks[0]->ks;
    b->lanes = std::max(1, std::min(LANES_DEFAULT, count));
    make_chunks(b);
    *out = b;
    return LBM_FS_OK;
}

lbm_fs_status lbm_fs_batch_destroy(lbm_fs_batch *b) {
    lbm_fs_status s = check_batch(b);
    if (s) return s;
    destroy_all(b);
    return LBM_FS_OK;
}

lbm_fs_status lbm_fs_batch_tank(lbm_fs_batch *b, int32_t k, lbm_fs **out) {
    lbm_fs_status s = check_batch(b);
    if (s) return s;
    if (!out || k < 0 || k >= (int32_t)b->tanks.size()) return fail(LBM_FS_EINVAL, "bad tank index%s");
    *out = b->tanks[k];
    return LBM_FS_OK;
}

lbm_fs_status lbm_fs_batch_step(lbm_fs_batch *b, int32_t nsteps) {
    lbm_fs_status s = check_batch(b);
    if (s) return s;
    if (nsteps < 0) return fail(LBM_FS_EINVAL, "nsteps must be >= 0%s");
    if (nsteps == 0) return LBM_FS_OK;
    s = prepare(b);
    if (s) return s;
    if (b->use_graphs && !b->gexec[0]) {
        s = capture(b);
        if (s) return s;
    }
    for (int32_t k = 0; k < nsteps; ++k) {
        int n = b->per_step;
        if (b->use_graphs) {
            CK(cudaGraphLaunch(b->gexec[b->cur], b->st));
        } else {
            n = enqueue_step(b, b->cur, b->st);
            CK(cudaGetLastError());
        }
        advance(b, n);
    }
    return LBM_FS_OK;
}

lbm_fs_status lbm_fs_batch_sync(lbm_fs_batch *b) {
    lbm_fs_status s = check_batch(b);
    if (s) return s;
    CK(cudaStreamSynchronize(b->st));
    for (size_t k = 0; k < b->tanks.size(); ++k) {
        s = read_status(b->tanks[k]);
        if (s) {
            char buf[64];
            snprintf(buf, sizeof buf, " (tank %d)", (int)k);
            std::string msg = std::string(lbm_fs_last_error_string()) + buf;
            return fail(s, "%s", msg.c_str());
        }
    }
    return LBM_FS_OK;
}

lbm_fs_status lbm_fs_batch_get_config(lbm_fs_batch *b, lbm_fs_batch_config_t *c) {
    lbm_fs_status s = check_batch(b);
    if (s) return s;
    if (!c) return fail(LBM_FS_EINVAL, "null config%s");
    memset(c, 0, sizeof *c);
    c->zb = b->zb;
    c->bulk_blocks = b->bulk_blocks;
    c->list_cells = b->list_cells;
    c->lanes = b->lanes;
    return LBM_FS_OK;
}

lbm_fs_status lbm_fs_batch_set_config(lbm_fs_batch *b, const lbm_fs_batch_config_t *c) {
    lbm_fs_status s = check_batch(b);
    if (s) return s;
    if (!c || c->zb < 1 || c->zb > 8 || c->bulk_blocks < 0 || c->list_cells < 1 || c->lanes < 0 ||
        c->lanes > MAX_LANES)
        return fail(LBM_FS_EINVAL, "config needs zb in 1..8, bulk_blocks >= 0, list_cells >= 1, lanes in 0..4%s");
    for (lbm_fs *t : b->tanks)
        if ((t->d[0].nz + c->zb - 1) / c->zb > 65535) return fail(LBM_FS_EINVAL, "zb too small for a tank%s");
    CK(cudaStreamSynchronize(b->st));
    b->zb = c->zb;
    b->bulk_blocks = c->bulk_blocks;
    b->list_cells = c->list_cells;
    const int lanes = std::min<int>(c->lanes ? c->lanes : b->lanes, (int)b->tanks.size());
    if (lanes != b->lanes) {
        b->lanes = lanes;
        make_chunks(b);
    }
    b->built = false;
    b->drop_graphs();
    return LBM_FS_OK;
}

lbm_fs_status lbm_fs_batch_autotune(lbm_fs_batch *b, lbm_fs_batch_config_t *out) {
    lbm_fs_status s = check_batch(b);
    if (s) return s;
    s = prepare(b);
    if (s) return s;
    const int nt = (int)b->tanks.size();
    // the timed launches append interface cells and may book moving-wall
    // mass: keep the counters and ledgers and put them back afterwards
    std::vector<double> ledgers((size_t)nt * LG_COUNT);
    std::vector<uint32_t> counters((size_t)nt * WL_COUNT);
    CK(cudaStreamSynchronize(b->st));
    for (int k = 0; k < nt; ++k) {
        CK(cudaMemcpy(&ledgers[(size_t)k * LG_COUNT], b->tanks[k]->d[0].ledger, sizeof(double) * LG_COUNT,
                      cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(&counters[(size_t)k * WL_COUNT], b->tanks[k]->d[0].cnt, sizeof(uint32_t) * WL_COUNT,
                      cudaMemcpyDeviceToHost));
    }
    const int keep_zb = b->zb, keep_blocks = b->bulk_blocks;
    const int per_sm = b->ks.bulk_blocks_per_sm();
    const int zbs[] = {1, 2, 4, 8};
    const int mults[] = {1, 2, 4, 0};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = 1e30;
    int best_zb = keep_zb, best_blocks = keep_blocks;
    lbm_fs_status err = LBM_FS_OK;
    for (int zb : zbs) {
        bool fits = true;
        for (lbm_fs *t : b->tanks) fits = fits && (t->d[0].nz + zb - 1) / zb <= 65535;
        if (!fits) continue;
        for (int m : mults) {
            b->zb = zb;
            b->bulk_blocks = m ? m * per_sm * b->sms : 0;
            err = build(b);
            if (err) break;
            // one warm-up and five timed launches append at most six times a
            // tank's interface cells to its list (capacity: one entry per cell)
            for (lbm_fs *t : b->tanks) cudaMemsetAsync(t->d[0].cnt, 0, sizeof(uint32_t) * WL_COUNT, b->st);
            const int reps = 5;
            for (auto &cp : b->chunks) b->ks.batch_bulk(launch_of(b, *cp, b->cur), b->st);
            cudaEventRecord(e0, b->st);
            for (int r = 0; r < reps; ++r)
                for (auto &cp : b->chunks) b->ks.batch_bulk(launch_of(b, *cp, b->cur), b->st);
            cudaEventRecord(e1, b->st);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                err = cuda_fail(e, "batch autotune");
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            double per = ms / reps;
            if (per < best) {
                best = per;
                best_zb = zb;
                best_blocks = b->bulk_blocks;
            }
        }
        if (err) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int k = 0; k < nt; ++k) {
        CK(cudaMemcpyAsync(b->tanks[k]->d[0].ledger, &ledgers[(size_t)k * LG_COUNT], sizeof(double) * LG_COUNT,
                           cudaMemcpyHostToDevice, b->st));
        CK(cudaMemcpyAsync(b->tanks[k]->d[0].cnt, &counters[(size_t)k * WL_COUNT], sizeof(uint32_t) * WL_COUNT,
                           cudaMemcpyHostToDevice, b->st));
    }
    CK(cudaStreamSynchronize(b->st));
    if (err) return err;
    b->zb = best_zb;
    b->bulk_blocks = best_blocks;
    s = build(b);
    if (s) return s;
    if (out) {
        memset(out, 0, sizeof *out);
        out->zb = b->zb;
        out->bulk_blocks = b->bulk_blocks;
        out->list_cells = b->list_cells;
        out->lanes = b->lanes;
        out->bulk_ms = best;
    }
    return LBM_FS_OK;
}

lbm_fs_status lbm_fs_batch_kernel_times(lbm_fs_batch *b, int32_t nsteps, double *ms, const char **names, int32_t cap,
                                        int32_t *nk) {
    lbm_fs_status s = check_batch(b);
    if (s) return s;
    if (nsteps <= 0 || !ms || cap <= 0) return fail(LBM_FS_EINVAL, "bad arguments%s");
    s = prepare(b);
    if (s) return s;
    const int K = b->ks.nkernels;
    std::vector<cudaEvent_t> ev(K + 1);
    for (auto &x : ev) CK(cudaEventCreate(&x));
    std::vector<double> acc(K, 0.0);
    for (int32_t it = 0; it < nsteps; ++it) {
        int n = 0;
        for (auto &cp : b->chunks) {
            n += b->ks.batch_step(launch_of(b, *cp, b->cur), b->st, ev.data());
            CK(cudaGetLastError());
            CK(cudaEventSynchronize(ev[K]));
            for (int k = 0; k < K; ++k) {
                float t = 0.0f;
                CK(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
                acc[k] += t;
            }
        }
        advance(b, n);
    }
    for (auto &x : ev) cudaEventDestroy(x);
    int m = K < cap ? K : cap;
    for (int k = 0; k < m; ++k) {
        ms[k] = acc[k];
        if (names) names[k] = b->ks.names[k];
    }
    if (nk) *nk = K;
    return lbm_fs_batch_sync(b);
}

lbm_fs_status lbm_fs_batch_launches(lbm_fs_batch *b, int64_t *launches, int64_t *steps) {
    lbm_fs_status s = check_batch(b);
    if (s) return s;
    if (launches) *launches = b->launches;
    if (steps) *steps = b->step;
    return LBM_FS_OK;
}

}  // extern "C"
