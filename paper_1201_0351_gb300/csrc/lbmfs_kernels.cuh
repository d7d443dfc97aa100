// Device code of the free-surface LBM step (Bogner & Ruede, Sec. 2), templated
// on the population storage.  Included by one translation unit per storage:
//   S = 0  f_q as double, double arithmetic.  Every operation is written in the
//          same order as the plain CPU restatement of the method and the unit is
//          compiled with -fmad=false, so this path reproduces it bit for bit
//          (except for the order of the parallel force / ledger sums);
//   S = 1  f_q - w_q as float, float arithmetic on deviations;
//   S = 2  f_q - w_q as half (q >= 1, times 2^10) with a float rest population
//          chosen so that the stored cell sum equals the collision density.
// Interface mass, fill level, forces, torques and the ledger are double in all
// three.
#pragma once
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#include "lbmfs_internal.h"

namespace lbmfs {
namespace {  // internal linkage: one copy per storage translation unit

// ----------------------------------------------------------------- lattice
// D3Q19 in the order C,W,E,N,S,T,B,TW,TE,TN,TS,NW,NE,SW,SE,BW,BE,BN,BS (the
// order of the paper's stencil figure, Eq. links).
__host__ __device__ __forceinline__ constexpr int cx(int q) {
    return q == 1 || q == 7 || q == 11 || q == 13 || q == 15 ? -1
           : (q == 2 || q == 8 || q == 12 || q == 14 || q == 16 ? 1 : 0);
}
__host__ __device__ __forceinline__ constexpr int cy(int q) {
    return q == 3 || q == 9 || q == 11 || q == 12 || q == 17 ? 1
           : (q == 4 || q == 10 || q == 13 || q == 14 || q == 18 ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int cz(int q) {
    return q == 5 || (q >= 7 && q <= 10) ? 1 : (q == 6 || q >= 15 ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int opp(int q) {
    // C-C, W-E, N-S, T-B, TW-BE, TE-BW, TN-BS, TS-BN, NW-SE, NE-SW
    return q == 0 ? 0
                  : (q <= 6 ? (q & 1 ? q + 1 : q - 1)
                            : (q == 7 || q == 8 || q == 15 || q == 16 ? 23 - q
                                                                      : (q <= 14 && q >= 11 ? 25 - q : 27 - q)));
}
// the table is checked at compile time: c_opp(q) = -c_q, weights symmetric
__host__ __device__ constexpr bool lattice_ok() {
    for (int q = 0; q < 19; ++q) {
        int p = opp(q);
        if (cx(p) != -cx(q) || cy(p) != -cy(q) || cz(p) != -cz(q)) return false;
        int s = (cx(q) != 0) + (cy(q) != 0) + (cz(q) != 0);
        if ((q == 0) != (s == 0) || (q >= 1 && q <= 6) != (s == 1) || (q >= 7) != (s == 2)) return false;
    }
    return true;
}
static_assert(lattice_ok(), "D3Q19 table");
// weights of the stencil figure caption: 1/3, 1/18, 1/36
__host__ __device__ __forceinline__ constexpr double wd(int q) {
    return q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}
__host__ __device__ __forceinline__ constexpr float wf(int q) {
    return q == 0 ? 1.0f / 3.0f : (q <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}

#ifndef LBMFS_BULK_MINB
#define LBMFS_BULK_MINB 8  // resident blocks per SM asked of ptxas for the bulk kernel (64 registers)
#endif
#ifndef LBMFS_BULK_PAIR
#define LBMFS_BULK_PAIR 0  // tuning knob: float storages on even grids take two cells per bulk-kernel thread
#endif
#ifndef LBMFS_PAIR_MINB
#define LBMFS_PAIR_MINB 5  // resident blocks per SM of the two-cell bulk kernel (float storages, 96 registers)
#endif
#ifndef LBMFS_BULK_ZB
#define LBMFS_BULK_ZB 8    // z-planes per bulk-kernel block (measured: 8 beat 4 by 2 % for FP32, 2 was far slower)
#endif
#ifndef LBMFS_BULK_PIPE_ZB
#define LBMFS_BULK_PIPE_ZB 16  // z-planes per block of the software-pipelined bulk kernel
#endif
#ifndef LBMFS_FORCE_MINB
#define LBMFS_FORCE_MINB 3  // resident 256-thread blocks per SM of the float-storage force kernel
#endif
#ifndef LBMFS_FORCE_ROWS
#define LBMFS_FORCE_ROWS 1  // 32-cell tasks of a body's range per warp in the float-storage force kernel
#endif
#ifndef LBMFS_IFACE_MINB
#define LBMFS_IFACE_MINB 6  // resident blocks per SM asked of ptxas for the interface kernel (80 registers)
#endif
#ifndef LBMFS_IFACE_GRID
#define LBMFS_IFACE_GRID (16 * 152)  // blocks of the single-tank interface kernel (16 per SM)
#endif
#ifndef LBMFS_ST_CS
#define LBMFS_ST_CS 0      // population stores with the evict-first (streaming) hint
#endif
constexpr float F16_SCALE = 1024.0f;
constexpr float F16_INV_SCALE = 1.0f / 1024.0f;
constexpr int CL_WALL = 256;

// ----------------------------------------------------------------- storage
// population loads / stores (tuning knob: evict-first stores)
template <class T> __device__ __forceinline__ T pop_ld(const T *p) { return *p; }
// through the read-only data path: only for a grid that no thread of the
// launch writes (the bulk kernel's source populations)
template <class T> __device__ __forceinline__ T pop_ldg(const T *p) { return __ldg(p); }
template <class T> __device__ __forceinline__ void pop_st(T *p, T v) {
#if LBMFS_ST_CS
    __stcs(p, v);
#else
    *p = v;
#endif
}
template <int S> struct Sto;

template <> struct Sto<0> {
    using R = double;
    static constexpr bool shifted = false;
    static __device__ __forceinline__ double ld(const void *g, int q, long long i, long long N) {
        return pop_ld(reinterpret_cast<const double *>(g) + ((long long)q * N + i));
    }
    static __device__ __forceinline__ double ldg(const void *g, int q, long long i, long long N) {
        return pop_ldg(reinterpret_cast<const double *>(g) + ((long long)q * N + i));
    }
    static __device__ __forceinline__ void st(void *g, int q, long long i, long long N, double v) {
        pop_st(reinterpret_cast<double *>(g) + ((long long)q * N + i), v);
    }
    // value of f_q as double
    static __device__ __forceinline__ double ldf(const void *g, int q, long long i, long long N) {
        return ld(g, q, i, N);
    }
    // store a full cell given as 19 doubles f_q
    static __device__ __forceinline__ void st_cell(void *g, long long i, long long N, const double *f) {
#pragma unroll
        for (int q = 0; q < Q; ++q) st(g, q, i, N, f[q]);
    }
    static size_t bytes(long long N) { return (size_t)N * Q * sizeof(double); }
    static constexpr int SCALE = 1;
    static __device__ __forceinline__ double ld_raw(const void *g, int q, long long i, long long N) { return ld(g, q, i, N); }
    static __device__ __forceinline__ double ldg_raw(const void *g, int q, long long i, long long N) {
        return ldg(g, q, i, N);
    }
};

template <> struct Sto<1> {
    using R = float;
    static constexpr bool shifted = true;
    static __device__ __forceinline__ float ld(const void *g, int q, long long i, long long N) {
        return pop_ld(reinterpret_cast<const float *>(g) + ((long long)q * N + i));
    }
    static __device__ __forceinline__ float ldg(const void *g, int q, long long i, long long N) {
        return pop_ldg(reinterpret_cast<const float *>(g) + ((long long)q * N + i));
    }
    static __device__ __forceinline__ void st(void *g, int q, long long i, long long N, float v) {
        pop_st(reinterpret_cast<float *>(g) + ((long long)q * N + i), v);
    }
    static __device__ __forceinline__ double ldf(const void *g, int q, long long i, long long N) {
        return wd(q) + (double)ld(g, q, i, N);
    }
    static __device__ __forceinline__ void st_cell(void *g, long long i, long long N, const double *f) {
#pragma unroll
        for (int q = 0; q < Q; ++q) st(g, q, i, N, (float)(f[q] - wd(q)));
    }
    // store the collided deviations dv; the rest population is replaced by
    // dp_0 + sum_{q>=1} (dp_q - dv_q) (equal to dv_0 in exact arithmetic) so
    // that the stored cell sum equals the streamed-in sum of dp up to one
    // rounding of a small number: no mass drift from float rounding
    static __device__ __forceinline__ void st_dev(void *g, long long i, long long N, const float *dv, const float *dp) {
        float rest = 0.0f;
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            st(g, q, i, N, dv[q]);
            rest += dp[q] - dv[q];
        }
        st(g, 0, i, N, dp[0] + rest);
    }
    static size_t bytes(long long N) { return (size_t)N * Q * sizeof(float); }
    // store one deviation, return the value as stored
    static __device__ __forceinline__ float st_one(void *g, int q, long long i, long long N, float v) {
        st(g, q, i, N, v);
        return v;
    }
    // values as stored (no scale)
    static constexpr int SCALE = 1;
    static __device__ __forceinline__ float ld_raw(const void *g, int q, long long i, long long N) { return ld(g, q, i, N); }
    static __device__ __forceinline__ float ldg_raw(const void *g, int q, long long i, long long N) { return ldg(g, q, i, N); }
    static __device__ __forceinline__ float st_raw(void *g, int q, long long i, long long N, float v) {
        return st_one(g, q, i, N, v);
    }
    // the populations q of the cells j, j + 1 (one 8-byte load when the pair
    // starts on an even element, two loads otherwise), through the read-only path
    static __device__ __forceinline__ float2 ldg_pair_raw(const void *g, int q, long long j, long long N) {
        const long long k = (long long)q * N + j;
        const float *b = reinterpret_cast<const float *>(g) + k;
        if (k & 1) return make_float2(pop_ldg(b), pop_ldg(b + 1));
        return pop_ldg(reinterpret_cast<const float2 *>(b));
    }
    // store population q of the cells i, i + 1; returns the values as stored
    static __device__ __forceinline__ float2 st_pair_raw(void *g, int q, long long i, long long N, float2 v) {
        const long long k = (long long)q * N + i;
        float *b = reinterpret_cast<float *>(g) + k;
        if (k & 1) {
            pop_st(b, v.x);
            pop_st(b + 1, v.y);
        } else {
            pop_st(reinterpret_cast<float2 *>(b), v);
        }
        return v;
    }
};

template <> struct Sto<2> {
    using R = float;
    static constexpr bool shifted = true;
    // plane 0: float (N); planes 1..18: half (N each), after it
    static __device__ __forceinline__ const __half *hp(const void *g, long long N) {
        return reinterpret_cast<const __half *>(reinterpret_cast<const float *>(g) + N);
    }
    static __device__ __forceinline__ float ld(const void *g, int q, long long i, long long N) {
        if (q == 0) return pop_ld(reinterpret_cast<const float *>(g) + i);
        return __half2float(pop_ld(hp(g, N) + ((long long)(q - 1) * N + i))) * F16_INV_SCALE;
    }
    static __device__ __forceinline__ float ldg(const void *g, int q, long long i, long long N) {
        if (q == 0) return pop_ldg(reinterpret_cast<const float *>(g) + i);
        return __half2float(pop_ldg(hp(g, N) + ((long long)(q - 1) * N + i))) * F16_INV_SCALE;
    }
    static __device__ __forceinline__ double ldf(const void *g, int q, long long i, long long N) {
        return wd(q) + (double)ld(g, q, i, N);
    }
    // d*_q for q >= 1 rounded to half; the rest population takes
    // dp_0 + sum_{q>=1} (dp_q - dequant(h_q)) so that the stored cell sum
    // equals the streamed-in sum of dp (the collision density) up to one
    // rounding of a small number
    static __device__ __forceinline__ void st_dev(void *g, long long i, long long N, const float *dv, const float *dp) {
        __half *h = const_cast<__half *>(hp(g, N));
        float rest = 0.0f;
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            __half hq = __float2half_rn(dv[q] * F16_SCALE);
            pop_st(h + ((long long)(q - 1) * N + i), hq);
            rest += dp[q] - __half2float(hq) * F16_INV_SCALE;
        }
        pop_st(reinterpret_cast<float *>(g) + i, dp[0] + rest);
    }
    static __device__ __forceinline__ void st_cell(void *g, long long i, long long N, const double *f) {
        float dv[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) dv[q] = (float)(f[q] - wd(q));
        st_dev(g, i, N, dv, dv);
    }
    static size_t bytes(long long N) { return (size_t)N * (sizeof(float) + (Q - 1) * sizeof(__half)); }
    static __device__ __forceinline__ float st_one(void *g, int q, long long i, long long N, float v) {
        if (q == 0) {
            pop_st(reinterpret_cast<float *>(g) + i, v);
            return v;
        }
        __half hq = __float2half_rn(v * F16_SCALE);
        pop_st(const_cast<__half *>(hp(g, N)) + ((long long)(q - 1) * N + i), hq);
        return __half2float(hq) * F16_INV_SCALE;
    }
    // values as stored: q >= 1 times F16_SCALE, the rest population unscaled
    static constexpr int SCALE = (int)F16_SCALE;
    static __device__ __forceinline__ float ld_raw(const void *g, int q, long long i, long long N) {
        if (q == 0) return pop_ld(reinterpret_cast<const float *>(g) + i);
        return __half2float(pop_ld(hp(g, N) + ((long long)(q - 1) * N + i)));
    }
    static __device__ __forceinline__ float ldg_raw(const void *g, int q, long long i, long long N) {
        if (q == 0) return pop_ldg(reinterpret_cast<const float *>(g) + i);
        return __half2float(pop_ldg(hp(g, N) + ((long long)(q - 1) * N + i)));
    }
    static __device__ __forceinline__ float st_raw(void *g, int q, long long i, long long N, float v) {
        if (q == 0) {
            pop_st(reinterpret_cast<float *>(g) + i, v);
            return v;
        }
        __half hq = __float2half_rn(v);
        pop_st(const_cast<__half *>(hp(g, N)) + ((long long)(q - 1) * N + i), hq);
        return __half2float(hq);
    }
    // the populations q of the cells j, j + 1 in raw units: one 4-byte load
    // (8 bytes for the rest population) when the pair starts on an even
    // element, otherwise the two aligned words around it
    static __device__ __forceinline__ float2 ldg_pair_raw(const void *g, int q, long long j, long long N) {
        if (q == 0) {
            const float *b = reinterpret_cast<const float *>(g) + j;
            if (j & 1) return make_float2(pop_ldg(b), pop_ldg(b + 1));
            return pop_ldg(reinterpret_cast<const float2 *>(b));
        }
        const long long k = (long long)(q - 1) * N + j;
        const __half *h = hp(g, N) + k;
        if (k & 1) {
            const __half2 a = pop_ldg(reinterpret_cast<const __half2 *>(h - 1));
            const __half2 b = pop_ldg(reinterpret_cast<const __half2 *>(h + 1));
            return make_float2(__high2float(a), __low2float(b));
        }
        return __half22float2(pop_ldg(reinterpret_cast<const __half2 *>(h)));
    }
    // store population q of the cells i, i + 1 (raw units); returns the
    // values as stored
    static __device__ __forceinline__ float2 st_pair_raw(void *g, int q, long long i, long long N, float2 v) {
        if (q == 0) {
            float *b = reinterpret_cast<float *>(g) + i;
            if (i & 1) {
                pop_st(b, v.x);
                pop_st(b + 1, v.y);
            } else {
                pop_st(reinterpret_cast<float2 *>(b), v);
            }
            return v;
        }
        const long long k = (long long)(q - 1) * N + i;
        __half *h = const_cast<__half *>(hp(g, N)) + k;
        const __half2 hv = __floats2half2_rn(v.x, v.y);
        if (k & 1) {
            pop_st(h, __low2half(hv));
            pop_st(h + 1, __high2half(hv));
        } else {
            pop_st(reinterpret_cast<__half2 *>(h), hv);
        }
        return __half22float2(hv);
    }
};

// The bulk kernel's view of one population grid: 32-bit element indices
// (q N + j < 2^32 for the float storages, checked at create) from one base
// pointer per kind of plane, so an access costs one index multiply-add and
// one widening address computation instead of 64-bit index arithmetic.
template <int S> struct Planes;
template <> struct Planes<1> {
    const float *r;
    float *w;
    uint32_t N;
    __device__ __forceinline__ Planes(const void *src, void *dst, long long n)
        : r(reinterpret_cast<const float *>(src)), w(reinterpret_cast<float *>(dst)), N((uint32_t)n) {}
    __device__ __forceinline__ float ld(int q, uint32_t j) const { return pop_ldg(r + ((uint32_t)q * N + j)); }
    __device__ __forceinline__ float st(int q, uint32_t j, float v) const {
        pop_st(w + ((uint32_t)q * N + j), v);
        return v;
    }
    // the pair j, j + 1 when j + q N is even (one 8-byte load / store)
    __device__ __forceinline__ float2 ld2(int q, uint32_t j) const {
        return pop_ldg(reinterpret_cast<const float2 *>(r + ((uint32_t)q * N + j)));
    }
    // the pair j, j + 1 when j + q N is odd (two loads)
    __device__ __forceinline__ float2 ld2_odd(int q, uint32_t j) const {
        const float *b = r + ((uint32_t)q * N + j);
        return make_float2(pop_ldg(b), pop_ldg(b + 1));
    }
    __device__ __forceinline__ float2 st2(int q, uint32_t j, float2 v) const {
        pop_st(reinterpret_cast<float2 *>(w + ((uint32_t)q * N + j)), v);
        return v;
    }
};
template <> struct Planes<2> {
    const float *r0;
    const __half *rh;
    float *w0;
    __half *wh;
    uint32_t N;
    __device__ __forceinline__ Planes(const void *src, void *dst, long long n)
        : r0(reinterpret_cast<const float *>(src)), rh(reinterpret_cast<const __half *>(r0 + n)),
          w0(reinterpret_cast<float *>(dst)), wh(reinterpret_cast<__half *>(w0 + n)), N((uint32_t)n) {}
    // raw units: q >= 1 times the storage's scale, the rest population unscaled
    __device__ __forceinline__ float ld(int q, uint32_t j) const {
        if (q == 0) return pop_ldg(r0 + j);
        return __half2float(pop_ldg(rh + ((uint32_t)(q - 1) * N + j)));
    }
    __device__ __forceinline__ float st(int q, uint32_t j, float v) const {
        if (q == 0) {
            pop_st(w0 + j, v);
            return v;
        }
        const __half h = __float2half_rn(v);
        pop_st(wh + ((uint32_t)(q - 1) * N + j), h);
        return __half2float(h);
    }
    __device__ __forceinline__ float2 ld2(int q, uint32_t j) const {
        if (q == 0) return pop_ldg(reinterpret_cast<const float2 *>(r0 + j));
        return __half22float2(pop_ldg(reinterpret_cast<const __half2 *>(rh + ((uint32_t)(q - 1) * N + j))));
    }
    __device__ __forceinline__ float2 ld2_odd(int q, uint32_t j) const {
        if (q == 0) return make_float2(pop_ldg(r0 + j), pop_ldg(r0 + j + 1));
        const __half *h = rh + ((uint32_t)(q - 1) * N + j);
        const __half2 a = pop_ldg(reinterpret_cast<const __half2 *>(h - 1));
        const __half2 b = pop_ldg(reinterpret_cast<const __half2 *>(h + 1));
        return make_float2(__high2float(a), __low2float(b));
    }
    __device__ __forceinline__ float2 st2(int q, uint32_t j, float2 v) const {
        if (q == 0) {
            pop_st(reinterpret_cast<float2 *>(w0 + j), v);
            return v;
        }
        const __half2 h = __floats2half2_rn(v.x, v.y);
        pop_st(reinterpret_cast<__half2 *>(wh + ((uint32_t)(q - 1) * N + j)), h);
        return __half22float2(h);
    }
};

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
// order earlier generic-proxy accesses to shared memory before the async-proxy
// (bulk copy) writes that follow
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ long long nbr(const Dev &d, int x, int y, int z, int dx, int dy, int dz) {
    int px = x + dx, py = y + dy, pz = z + dz;
    if (px < 0 || px >= d.nx) {
        if (!(d.periodic & 1u)) return -1;
        px = px < 0 ? px + d.nx : px - d.nx;
    }
    if (py < 0 || py >= d.ny) {
        if (!(d.periodic & 2u)) return -1;
        py = py < 0 ? py + d.ny : py - d.ny;
    }
    if (pz < 0 || pz >= d.nz) {
        if (!(d.periodic & 4u)) return -1;
        pz = pz < 0 ? pz + d.nz : pz - d.nz;
    }
    return px + (long long)d.nx * (py + (long long)d.ny * pz);
}

__device__ __forceinline__ void coords(const Dev &d, long long idx, int &x, int &y, int &z) {
    x = (int)(idx % d.nx);
    long long r = idx / d.nx;
    y = (int)(r % d.ny);
    z = (int)(r / d.ny);
}

// class of cell i (the flag byte without the neighbour-obstacle bit); walls
// (i < 0) report CL_WALL
__device__ __forceinline__ int clsv(const Dev &d, long long i) { return (int)(d.flags[i] & CL_MASK); }
__device__ __forceinline__ int cls(const Dev &d, long long i) { return i < 0 ? CL_WALL : clsv(d, i); }
__device__ __forceinline__ void set_cls(const Dev &d, long long i, int c) {
    d.flags[i] = (uint8_t)((d.flags[i] & NB_OBST) | c);
}

// warp-aggregated append of val to a worklist
__device__ __forceinline__ void wl_append(const Dev &d, bool pred, int list, uint32_t val) {
    unsigned act = __activemask();
    unsigned mask = __ballot_sync(act, pred);
    if (!pred) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&d.cnt[list], (uint32_t)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    uint32_t pos = base + (uint32_t)__popc(mask & ((1u << lane) - 1u));
    if (pos < d.cap) d.list[list][pos] = val;
    else atomicOr(d.status, ST_OVERFLOW);
}

__device__ __forceinline__ uint32_t wl_count(const Dev &d, int list) {
    uint32_t c = *reinterpret_cast<volatile uint32_t *>(&d.cnt[list]);
    return c < d.cap ? c : d.cap;
}

// atomic OR / AND on one byte of the mark array; returns the old byte
__device__ __forceinline__ uint8_t mark_or(const Dev &d, long long i, uint8_t bits) {
    uintptr_t a = reinterpret_cast<uintptr_t>(d.cmark + i);
    unsigned int *w = reinterpret_cast<unsigned int *>(a & ~(uintptr_t)3);
    unsigned sh = (unsigned)(a & 3) * 8u;
    unsigned old = atomicOr(w, (unsigned)bits << sh);
    return (uint8_t)(old >> sh);
}
__device__ __forceinline__ void mark_and(const Dev &d, long long i, uint8_t bits) {
    uintptr_t a = reinterpret_cast<uintptr_t>(d.cmark + i);
    unsigned int *w = reinterpret_cast<unsigned int *>(a & ~(uintptr_t)3);
    unsigned sh = (unsigned)(a & 3) * 8u;
    atomicAnd(w, ~((unsigned)bits << sh));
}

__device__ __forceinline__ double min_image(const Dev &d, double v, int k) {
    if (d.periodic & (1u << k)) {
        double n = k == 0 ? (double)d.nx : (k == 1 ? (double)d.ny : (double)d.nz);
        v = v - n * floor(v / n + 0.5);
    }
    return v;
}

// rotation matrix of the unit quaternion (w, x, y, z), row-major
__device__ __forceinline__ void rotation(const double *q, double *R) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

// Sec. 2.3: cell centre strictly inside the body (box, or sphere of radius
// h[0]); products and sums rounded one by one (no fused multiply-add) so that
// every storage classifies a centre on the surface the same way
// Float pre-test of the cell-centre-inside rule: 1 inside, 0 outside, -1
// undecided.  The cell centre relative to the body comes from the integer part
// and the fraction of the centre (exact integer, fraction rounded once), the
// rotation and the extents in float; every decision keeps a margin of
// 1e-5 (1 + |d|_1 + h) to the surface, well above the float evaluation's error
// bound (a few times 2^-24 (1 + |d|_1 + h)), so where it decides the double
// test below gives the same answer.  GB300's double rate is 1/64 of its float
// rate, and most cells of a body's range lie far from its surface.
__device__ __forceinline__ int inside_float(const Body &b, int x, int y, int z) {
    const float df[3] = {(float)(x - b.oi[0]) + (0.5f - b.of[0]), (float)(y - b.oi[1]) + (0.5f - b.of[1]),
                         (float)(z - b.oi[2]) + (0.5f - b.of[2])};
    const float s = fabsf(df[0]) + fabsf(df[1]) + fabsf(df[2]);
    if (b.shape == 1) {
        const float r2 = df[0] * df[0] + df[1] * df[1] + df[2] * df[2];
        const float m = 1e-5f * (1.0f + s + r2 + b.hf[0]);  // hf[0] holds the squared radius
        return r2 < b.hf[0] - m ? 1 : (r2 > b.hf[0] + m ? 0 : -1);
    }
    int res = 1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float a = fabsf(b.Rf[0 * 3 + k] * df[0] + b.Rf[1 * 3 + k] * df[1] + b.Rf[2 * 3 + k] * df[2]);
        const float m = 1e-5f * (1.0f + s + b.hf[k]);
        if (a > b.hf[k] + m) return 0;
        if (!(a < b.hf[k] - m)) res = -1;
    }
    return res;
}
__device__ __forceinline__ bool inside(const Dev &d, const Body &b, int x, int y, int z) {
    if (!d.periodic) {
        const int r = inside_float(b, x, y, z);
        if (r >= 0) return r != 0;
    }
    double dd[3] = {min_image(d, (x + 0.5) - b.o[0], 0), min_image(d, (y + 0.5) - b.o[1], 1),
                    min_image(d, (z + 0.5) - b.o[2], 2)};
    if (b.shape == 1)
        return __dadd_rn(__dadd_rn(__dmul_rn(dd[0], dd[0]), __dmul_rn(dd[1], dd[1])), __dmul_rn(dd[2], dd[2])) <
               __dmul_rn(b.h[0], b.h[0]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double bk = __dadd_rn(__dadd_rn(__dmul_rn(b.R[0 * 3 + k], dd[0]), __dmul_rn(b.R[1 * 3 + k], dd[1])),
                              __dmul_rn(b.R[2 * 3 + k], dd[2]));
        if (!(fabs(bk) < b.h[k])) return false;
    }
    return true;
}

// Eq. noslip at a domain wall: c_q . u_w with u_w the velocity of the face
// that the link (x, q) crosses (source beyond the grid); a link across an edge
// takes the face of its lowest axis
__device__ __forceinline__ int wall_face(const Dev &d, int x, int y, int z, int q) {
    const int p[3] = {x - cx(q), y - cy(q), z - cz(q)}, nn[3] = {d.nx, d.ny, d.nz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (d.periodic & (1u << k)) continue;
        if (p[k] < 0) return 2 * k;
        if (p[k] >= nn[k]) return 2 * k + 1;
    }
    return -1;
}
__device__ __forceinline__ double wall_cuw(const Dev &d, int x, int y, int z, int q) {
    const int f = wall_face(d, x, y, z, q);
    if (f < 0) return 0.0;
    const double *u = d.wallv + 3 * f;
    return (cx(q) * u[0] + cy(q) * u[1]) + cz(q) * u[2];
}

__device__ __forceinline__ void body_velocity_at(const Dev &d, const Body &b, const double *p, double *uw) {
    double r[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) r[k] = min_image(d, p[k] - b.o[k], k);
    double c0 = b.w[1] * r[2] - b.w[2] * r[1];
    double c1 = b.w[2] * r[0] - b.w[0] * r[2];
    double c2 = b.w[0] * r[1] - b.w[1] * r[0];
    uw[0] = b.v[0] + c0;
    uw[1] = b.v[1] + c1;
    uw[2] = b.v[2] + c2;
}

// c_q . u_w with u_w at the midpoint x_c + c_qbar / 2 of the link (x, q)
__device__ __forceinline__ double link_cuw(const Dev &d, const Body &b, int x, int y, int z, int q) {
    int qb = opp(q);
    double p[3] = {(x + 0.5) + 0.5 * cx(qb), (y + 0.5) + 0.5 * cy(qb), (z + 0.5) + 0.5 * cz(qb)};
    double uw[3];
    body_velocity_at(d, b, p, uw);
    return (cx(q) * uw[0] + cy(q) * uw[1]) + cz(q) * uw[2];
}

// the same in float for the float storages: the body state is rounded once
// (positions relative to the body centre stay well inside float precision).
// BodyF holds what a cell's links share: the cell's offset from the body
// centre, rounded from double, and the body's velocities.
struct BodyF {
    float r0[3], v[3], w[3];
};
__device__ __forceinline__ BodyF body_f(const Body &b, int x, int y, int z) {
    return BodyF{{(float)(x - b.o[0]), (float)(y - b.o[1]), (float)(z - b.o[2])},
                 {(float)b.v[0], (float)b.v[1], (float)b.v[2]},
                 {(float)b.w[0], (float)b.w[1], (float)b.w[2]}};
}
__device__ __forceinline__ float link_cuw_f(const Dev &d, const BodyF &b, int q) {
    const int qb = opp(q);
    float r[3] = {b.r0[0] + (0.5f + 0.5f * cx(qb)), b.r0[1] + (0.5f + 0.5f * cy(qb)), b.r0[2] + (0.5f + 0.5f * cz(qb))};
    const int nn[3] = {d.nx, d.ny, d.nz};
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (d.periodic & (1u << k)) r[k] -= (float)nn[k] * floorf(r[k] / (float)nn[k] + 0.5f);
    const float u0 = b.v[0] + (b.w[1] * r[2] - b.w[2] * r[1]);
    const float u1 = b.v[1] + (b.w[2] * r[0] - b.w[0] * r[2]);
    const float u2 = b.v[2] + (b.w[0] * r[1] - b.w[1] * r[0]);
    return (cx(q) * u0 + cy(q) * u1) + cz(q) * u2;
}
__device__ __forceinline__ float link_cuw_f(const Dev &d, const Body &b, int x, int y, int z, int q) {
    return link_cuw_f(d, body_f(b, x, y, z), q);
}

// ------------------------------------------------- double arithmetic (Sec. 2.1)

// Eq. equilibrium, c_s^2 = 1/3
__device__ __forceinline__ double feq_d(int q, double rho, const double *u) {
    double cu = (cx(q) * u[0] + cy(q) * u[1]) + cz(q) * u[2];
    double usq = (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2];
    double t = ((1.0 + 3.0 * cu) + (4.5 * cu) * cu) - 1.5 * usq;
    return (wd(q) * rho) * t;
}

// Eq. forceterm (Luo): w rho [3 (c - u) + 9 (c.u) c] . a
__device__ __forceinline__ double force_d(int q, double rho, const double *u, const double *a) {
    double cu = (cx(q) * u[0] + cy(q) * u[1]) + cz(q) * u[2];
    double tx = (3.0 * (cx(q) - u[0]) + (9.0 * cu) * cx(q)) * a[0];
    double ty = (3.0 * (cy(q) - u[1]) + (9.0 * cu) * cy(q)) * a[1];
    double tz = (3.0 * (cz(q) - u[2]) + (9.0 * cu) * cz(q)) * a[2];
    return (wd(q) * rho) * ((tx + ty) + tz);
}

template <int S>
__device__ __forceinline__ double cell_density(const Dev &d, const void *g, long long i) {
    if constexpr (S != 0) {
        // deviations summed in float, as the collision does
        float dr = 0.0f;
#pragma unroll
        for (int q = 0; q < Q; ++q) dr += Sto<S>::ld(g, q, i, d.N);
        return 1.0 + (double)dr;
    }
    double r = 0.0;
#pragma unroll
    for (int q = 0; q < Q; ++q) r += Sto<S>::ldf(g, q, i, d.N);
    return r;
}

// density and the velocity of the last collision, sum c f / rho - a
template <int S>
__device__ __forceinline__ double cell_rho_u(const Dev &d, const void *g, long long i, double *u) {
    if constexpr (S != 0) {
        float dr = 0.0f, j0 = 0.0f, j1 = 0.0f, j2 = 0.0f;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            float v = Sto<S>::ld(g, q, i, d.N);
            dr += v;
            if (cx(q)) j0 += cx(q) * v;
            if (cy(q)) j1 += cy(q) * v;
            if (cz(q)) j2 += cz(q) * v;
        }
        float r = 1.0f + dr;
        u[0] = (double)(j0 / r - d.a_f[0]);
        u[1] = (double)(j1 / r - d.a_f[1]);
        u[2] = (double)(j2 / r - d.a_f[2]);
        return 1.0 + (double)dr;
    }
    double f[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) f[q] = Sto<S>::ldf(g, q, i, d.N);
    double r = 0.0;
#pragma unroll
    for (int q = 0; q < Q; ++q) r += f[q];
    double j0 = 0.0, j1 = 0.0, j2 = 0.0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        j0 += cx(q) * f[q];
        j1 += cy(q) * f[q];
        j2 += cz(q) * f[q];
    }
    u[0] = j0 / r - d.a[0];
    u[1] = j1 / r - d.a[1];
    u[2] = j2 / r - d.a[2];
    return r;
}

// double BGK collision of the post-stream cell fp -> fnew (Eq. lbgk, R1 order)
__device__ __forceinline__ void collide_d(const Dev &d, const double *fp, double *fnew) {
    double rho = 0.0, j0 = 0.0, j1 = 0.0, j2 = 0.0;
#pragma unroll
    for (int q = 0; q < Q; ++q) rho += fp[q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        j0 += cx(q) * fp[q];
        j1 += cy(q) * fp[q];
        j2 += cz(q) * fp[q];
    }
    double u[3] = {j0 / rho, j1 / rho, j2 / rho};
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        double fe = feq_d(q, rho, u);
        double fq = force_d(q, rho, u, d.a);
        fnew[q] = (fp[q] - d.omega * (fp[q] - fe)) + fq;
    }
}

// ----------------------------------------- float arithmetic on deviations

// ---- the same collision for one cell (V = float) or two cells at once
// (V = float2, GB300's packed FP32 instructions): every operation is written
// out as one correctly rounded add, multiply or fused multiply-add, so both
// forms round each cell identically and a cell's result does not depend on
// whether it was collided alone or in a pair.
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vrcp(float a) { return __frcp_rn(a); }
#ifndef LBMFS_NO_F32X2
#define LBMFS_NO_F32X2 0  // tuning knob: the pair's arithmetic as two scalar operations
#endif
#if LBMFS_NO_F32X2
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) {
    return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
#else
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
#endif
__device__ __forceinline__ float2 vrcp(float2 a) { return make_float2(__frcp_rn(a.x), __frcp_rn(a.y)); }
template <class V> __device__ __forceinline__ V vbc(float s);
template <> __device__ __forceinline__ float vbc<float>(float s) { return s; }
template <> __device__ __forceinline__ float2 vbc<float2>(float s) { return make_float2(s, s); }
// a - b as one rounding (b * -1 is exact)
template <class V> __device__ __forceinline__ V vsub(V a, V b) { return vfma(b, vbc<V>(-1.0f), a); }
__device__ __forceinline__ bool vpos_finite(float r) { return r > 0.0f && r < 1e30f; }
__device__ __forceinline__ bool vpos_finite(float2 r) { return vpos_finite(r.x) && vpos_finite(r.y); }

// BGK collision with the Luo force term on deviations dp_q = f'_q - w_q (q >= 1
// times SC, a power of two: the FP16 storage's own scale; dp_0 unscaled),
// fused with the store: store(q, dn) writes the collided deviation and returns
// the value as stored.  The rest population is stored as
// dp_0 + sum_{q>=1} (dp_q - stored_q) / SC: equal to the collided rest
// population in exact arithmetic, it makes the stored cell sum equal the
// streamed-in sum up to one rounding (no mass drift from storage rounding).
// For each pair q, qbar the equilibrium and force terms split as
//   f_eq - w = A +- B,  F = C +- D  with
//   A = w dr + w rho (4.5 (c.u)^2 - 1.5 u.u),  B = 3 w rho c.u,
//   C = w rho (9 (c.u)(c.a) - 3 u.a),          D = 3 w rho c.a,
// (c of the pair's member with the positive leading component) so that
//   dn = (1 - omega) dp + (E +- G),  E = omega A + C,  G = omega B + D.
// Returns the collision density.
template <int SC, class V, class Store>
__device__ __forceinline__ V collide_store_v(const Dev &d, const V *dp, Store store) {
    constexpr float sc = (float)SC, isc = 1.0f / (float)SC;
    V dr = dp[0];
#pragma unroll
    for (int q = 1; q < Q; ++q) dr = vfma(dp[q], vbc<V>(isc), dr);
    V j0 = vbc<V>(0.0f), j1 = vbc<V>(0.0f), j2 = vbc<V>(0.0f);
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        if (cx(q) > 0) j0 = vadd(j0, dp[q]);
        if (cx(q) < 0) j0 = vsub(j0, dp[q]);
        if (cy(q) > 0) j1 = vadd(j1, dp[q]);
        if (cy(q) < 0) j1 = vsub(j1, dp[q]);
        if (cz(q) > 0) j2 = vadd(j2, dp[q]);
        if (cz(q) < 0) j2 = vsub(j2, dp[q]);
    }
    const V rho = vadd(vbc<V>(1.0f), dr);
    const V inv = vmul(vrcp(rho), vbc<V>(isc));
    const V ux = vmul(j0, inv), uy = vmul(j1, inv), uz = vmul(j2, inv);
    const V nusq15 = vmul(vfma(uz, uz, vfma(uy, uy, vmul(ux, ux))), vbc<V>(-1.5f));  // -1.5 u.u
    const float om = d.omega_f, om1 = 1.0f - om;
    const float ax = d.a_f[0], ay = d.a_f[1], az = d.a_f[2];
    const V nua3 = vmul(vfma(uz, vbc<V>(az), vfma(uy, vbc<V>(ay), vmul(ux, vbc<V>(ax)))), vbc<V>(-3.0f));
    // per weight class: w dr, w rho, 3 w rho (times SC)
    const V wdr1 = vmul(dr, vbc<V>(wf(1) * sc)), wr1 = vmul(rho, vbc<V>(wf(1) * sc));
    const V wdr2 = vmul(dr, vbc<V>(wf(7) * sc)), wr2 = vmul(rho, vbc<V>(wf(7) * sc));
    const V wr13 = vmul(wr1, vbc<V>(3.0f)), wr23 = vmul(wr2, vbc<V>(3.0f));
    V rest = vbc<V>(0.0f);
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const int qb = opp(q);
        if (qb < q) continue;  // each pair once
        // p: the member whose leading nonzero velocity component is positive
        const int p = (cx(q) > 0 || (cx(q) == 0 && (cy(q) > 0 || (cy(q) == 0 && cz(q) > 0)))) ? q : qb;
        const bool axis = q <= 6;
        const V wdr = axis ? wdr1 : wdr2, wr = axis ? wr1 : wr2, wr3 = axis ? wr13 : wr23;
        V cu = cx(p) ? ux : (cy(p) ? uy : uz);  // the leading component is +1
        if (cx(p) && cy(p) > 0) cu = vadd(cu, uy);
        if (cx(p) && cy(p) < 0) cu = vsub(cu, uy);
        if ((cx(p) || cy(p)) && cz(p) > 0) cu = vadd(cu, uz);
        if ((cx(p) || cy(p)) && cz(p) < 0) cu = vsub(cu, uz);
        const float ca = (float)cx(p) * ax + (float)cy(p) * ay + (float)cz(p) * az;
        const V A = vfma(wr, vfma(vmul(cu, cu), vbc<V>(4.5f), nusq15), wdr);
        const V C = vmul(wr, vfma(cu, vbc<V>(9.0f * ca), nua3));
        const V E = vfma(A, vbc<V>(om), C);
        const V G = vfma(vmul(wr3, cu), vbc<V>(om), vmul(wr3, vbc<V>(ca)));
        const V dnp = vfma(dp[p], vbc<V>(om1), vadd(E, G));
        const int m = p == q ? qb : q;
        const V dnm = vfma(dp[m], vbc<V>(om1), vsub(E, G));
        rest = vadd(rest, vsub(dp[p], store(p, dnp)));
        rest = vadd(rest, vsub(dp[m], store(m, dnm)));
    }
    store(0, vfma(rest, vbc<V>(isc), dp[0]));
    return rho;
}

// f_eq(rho_g, u) - w as float deviation
__device__ __forceinline__ float feq_dev_f(int q, float drg, float ux, float uy, float uz) {
    float cu = (float)cx(q) * ux + (float)cy(q) * uy + (float)cz(q) * uz;
    float usq = ux * ux + uy * uy + uz * uz;
    float s = 3.0f * cu + 4.5f * cu * cu - 1.5f * usq;
    return wf(q) * (drg + s + drg * s);
}

// ------------------------------------------------------------- kernels

// K0: initial populations f = f_eq(rho, u) (u = 0 unless given), interface
// mass m = fill * sum f, fill = m / sum f
template <int S>
__global__ void k_init(Dev d, const uint8_t *flags, const double *fill, const double *rho, const double *vel) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    int c = flags[i];
    d.flags[i] = (uint8_t)c;
    d.bid[i] = 0;
    d.cmark[i] = 0;
    if (c != CL_L && c != CL_I) return;
    double u[3] = {0.0, 0.0, 0.0};
    if (vel) {
        u[0] = vel[3 * i];
        u[1] = vel[3 * i + 1];
        u[2] = vel[3 * i + 2];
    }
    double f[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) f[q] = feq_d(q, rho[i], u);
    Sto<S>::st_cell(d.fsrc, i, d.N, f);
    if (c == CL_I) {
        double r = cell_density<S>(d, d.fsrc, i);
        double m = fill[i] * r;
        d.m[i] = m;
        d.phisrc[i] = m / r;
    }
}

// rotation matrix and the cell range that may lie inside the body
__device__ void body_bounds(const Dev &d, Body &b) {
    rotation(b.q, b.R);
    for (int k = 0; k < 3; ++k) {
        const double fl = floor(b.o[k]);
        b.oi[k] = (int)fl;
        b.of[k] = (float)(b.o[k] - fl);  // o - floor(o) is exact in double
        b.hf[k] = (float)(b.shape == 1 && k == 0 ? b.h[0] * b.h[0] : b.h[k]);
    }
    for (int k = 0; k < 9; ++k) b.Rf[k] = (float)b.R[k];
    int n[3] = {d.nx, d.ny, d.nz};
    for (int k = 0; k < 3; ++k) {
        double e = b.shape == 1 ? b.h[0]
                                : (fabs(b.R[k * 3 + 0]) * b.h[0] + fabs(b.R[k * 3 + 1]) * b.h[1]) + fabs(b.R[k * 3 + 2]) * b.h[2];
        int lo = (int)floor(b.o[k] - e) - 1;
        int hi = (int)floor(b.o[k] + e) + 2;
        if (!(d.periodic & (1u << k))) {
            lo = lo < 0 ? 0 : lo;
            hi = hi > n[k] ? n[k] : hi;
        } else if (hi - lo > n[k]) {
            hi = lo + n[k];
        }
        if (hi < lo) hi = lo;
        b.lo[k] = lo;
        b.hi[k] = hi;
    }
}

__global__ void k_body_prepare(Dev d, int bi) {
    if (threadIdx.x != 0) return;
    Body &b = d.bodies[bi];
    body_bounds(d, b);
    for (int k = 0; k < 3; ++k) {
        b.plo[k] = b.lo[k];
        b.phi[k] = b.hi[k];
    }
}

// iterate the cells of a box range [lo, hi) (wrapped on periodic axes)
__device__ __forceinline__ long long range_count(const int *lo, const int *hi) {
    return (long long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
}
__device__ __forceinline__ void range_cell(const Dev &d, const int *lo, const int *hi, long long k, int &x, int &y,
                                           int &z) {
    int lx = hi[0] - lo[0], ly = hi[1] - lo[1];
    x = lo[0] + (int)(k % lx);
    long long r = k / lx;
    y = lo[1] + (int)(r % ly);
    z = lo[2] + (int)(r / ly);
    x = ((x % d.nx) + d.nx) % d.nx;  // only periodic axes can leave [0, n)
    y = ((y % d.ny) + d.ny) % d.ny;
    z = ((z % d.nz) + d.nz) % d.nz;
}

// mapping of a newly added body (Sec. 2.3); book_mass: charge the covered mass
template <int S>
__global__ void k_map_body(Dev d, int bi, int book_mass) {
    const Body &b = d.bodies[bi];
    long long n = range_count(b.lo, b.hi);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        range_cell(d, b.lo, b.hi, k, x, y, z);
        long long i = x + (long long)d.nx * (y + (long long)d.ny * z);
        int c = clsv(d, i);
        if (c == CL_O || !inside(d, b, x, y, z)) continue;
        if (book_mass) {
            double mass = c == CL_L ? cell_density<S>(d, d.fsrc, i) : (c == CL_I ? d.m[i] : 0.0);
            if (mass != 0.0) atomicAdd(&d.ledger[LG_COVERED], mass);
        }
        set_cls(d, i, CL_O);
        d.bid[i] = (uint8_t)bi;
    }
}

// Coordinates a kernel body runs at: its launch's own block, or one entry of
// a packed block table when a single launch serves many tanks
struct VB {
    unsigned x, y, z, nx, ny, nz;
};
__device__ __forceinline__ VB vb_own() { return VB{blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y, gridDim.z}; }

#define LIST_LOOP(L, var)                                                                                     \
    uint32_t n_##var = wl_count(d, L);                                                                         \
    for (uint32_t it_##var = vb.x * blockDim.x + threadIdx.x; it_##var < n_##var;                              \
         it_##var += vb.nx * blockDim.x)

// neighbour-obstacle bit: set when any of the 18 neighbours is an obstacle
// (the bulk kernel then lists the cell for k_general; walls and periodic
// seams are recognised from the cell's coordinates)
__device__ __forceinline__ void nb_refresh(const Dev &d, long long i) {
    int x, y, z;
    coords(d, i, x, y, z);
    bool nb = false;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        int c = cls(d, nbr(d, x, y, z, cx(q), cy(q), cz(q)));
        nb = nb || c == CL_O;
    }
    d.flags[i] = (uint8_t)((d.flags[i] & CL_MASK) | (nb ? NB_OBST : 0));
}

// neighbour-obstacle bits of the cells x0 <= x < x1 (grid (x-tiles, ny, nz))
__global__ void k_nb_all(Dev d) {
    int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= d.nx) return;
    long long i = x + (long long)d.nx * (y + (long long)d.ny * z);
    bool nb = false;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        int c = cls(d, nbr(d, x, y, z, cx(q), cy(q), cz(q)));
        nb = nb || c == CL_O;
    }
    d.flags[i] = (uint8_t)((d.flags[i] & CL_MASK) | (nb ? NB_OBST : 0));
}

// the same over the cells around body bi (its range widened by one cell)
__global__ void k_nb_body(Dev d, int bi) {
    const Body &b = d.bodies[bi];
    int lo[3] = {b.lo[0] - 1, b.lo[1] - 1, b.lo[2] - 1}, hi[3] = {b.hi[0] + 1, b.hi[1] + 1, b.hi[2] + 1};
    int n3[3] = {d.nx, d.ny, d.nz};
    for (int k = 0; k < 3; ++k) {
        if (!(d.periodic & (1u << k))) {
            lo[k] = lo[k] < 0 ? 0 : lo[k];
            hi[k] = hi[k] > n3[k] ? n3[k] : hi[k];
        } else if (hi[k] - lo[k] > n3[k]) {
            hi[k] = lo[k] + n3[k];
        }
    }
    for (int zz = lo[2] + (int)blockIdx.x; zz < hi[2]; zz += gridDim.x) {
        int z = zz < 0 ? zz + d.nz : (zz >= d.nz ? zz - d.nz : zz);
        for (int yy = lo[1] + (int)threadIdx.y; yy < hi[1]; yy += blockDim.y) {
            int y = yy < 0 ? yy + d.ny : (yy >= d.ny ? yy - d.ny : yy);
            for (int xx = lo[0] + (int)threadIdx.x; xx < hi[0]; xx += blockDim.x) {
                int x = xx < 0 ? xx + d.nx : (xx >= d.nx ? xx - d.nx : xx);
                nb_refresh(d, x + (long long)d.nx * (y + (long long)d.ny * z));
            }
        }
    }
}

// cells whose obstacle status changed this step (covered, uncovered): refresh
// the bit of each and of its 18 neighbours
__device__ __forceinline__ void nb_refresh_around(const Dev &d, long long i) {
    int x, y, z;
    coords(d, i, x, y, z);
    nb_refresh(d, i);
#pragma unroll 1
    for (int q = 1; q < Q; ++q) {
        long long yi = nbr(d, x, y, z, cx(q), cy(q), cz(q));
        if (yi >= 0) nb_refresh(d, yi);
    }
}

// one thread per (listed cell, direction): the cell itself (q = 0) or its
// neighbour in direction q; cells refreshed twice get the same value (the
// classes do not change in this kernel)
__device__ __forceinline__ void nb_update_body(const Dev &d, const VB &vb) {
    const uint32_t nc = wl_count(d, WL_COVER), np = wl_count(d, WL_PEND);
    const unsigned long long n = (unsigned long long)(nc + np) * Q;
    for (unsigned long long it = (unsigned long long)vb.x * blockDim.x + threadIdx.x; it < n;
         it += (unsigned long long)vb.nx * blockDim.x) {
        const uint32_t e = (uint32_t)(it / Q);
        const int q = (int)(it % Q);
        const long long c = e < nc ? (long long)d.list[WL_COVER][e] : (long long)d.list[WL_PEND][e - nc];
        long long t = c;
        if (q > 0) {
            int x, y, z;
            coords(d, c, x, y, z);
            t = nbr(d, x, y, z, cx(q), cy(q), cz(q));
        }
        if (t >= 0) nb_refresh(d, t);
    }
}
__global__ void k_nb_update(const __grid_constant__ Dev d) { nb_update_body(d, vb_own()); }

// ---- C4: momentum exchange at the links into body vb.y (state at t):
// Sec. 2.3 Eqs. momentumexchange, netforce, torque; Sec. 2.4 Eq.
// momentuminterface for interface cells
// Fixed-point sums of the float storages' per-cell force remainders: v * 2^s
// rounded to nearest (ties away from zero), built from the float's bits with
// integer operations (no double arithmetic; integer sums are exact, so the
// block and body totals do not depend on the order of the cells).
// |v| >= 2^(62 - s) (and a non-finite v) saturates at 2^62 in magnitude.
constexpr int FX_FORCE = 32, FX_TORQUE = 30;
__device__ __forceinline__ long long fixed_point(float v, int s) {
    const unsigned b = __float_as_uint(v);
    const int e = (int)((b >> 23) & 0xffu);
    const long long m = (long long)((b & 0x7fffffu) | 0x800000u);
    const int sh = e - 150 + s;  // |v| 2^s = m 2^sh for normal numbers
    long long r;
    if (e == 0 || sh < -25) r = 0;
    else if (sh < 0) r = (m + (1ll << (-sh - 1))) >> -sh;
    else r = sh > 38 ? (1ll << 62) : (m << sh);
    return (b >> 31) ? -r : r;
}

// Double-precision sums of Eqs. netforce and torque, exact and independent of
// the order of the terms: a term t (|t| < 2^31) becomes the integer
// floor(t 2^96) (its bits below 2^-96 dropped) and the integers are added in
// 128-bit two's complement; the total v = H 2^64 + L (H signed, L unsigned)
// becomes the double H 2^-32 + L 2^-96.  The plain CPU restatement sums the
// same way, so both give the same bits whatever the thread order.
__device__ __forceinline__ unsigned __int128 fixed96(double t) {
    const double sc = t * 4294967296.0;  // t 2^32, exact
    const double hf = floor(sc);
    const long long hi = (long long)hf;
    const unsigned long long lo = (unsigned long long)((sc - hf) * 18446744073709551616.0);
    return ((unsigned __int128)(unsigned long long)hi << 64) | (unsigned __int128)lo;
}
__device__ __forceinline__ double fixed96_value(unsigned __int128 v) {
    const long long H = (long long)(unsigned long long)(v >> 64);
    const unsigned long long L = (unsigned long long)v;
    return (double)H * 2.3283064365386962890625e-10 + (double)L * 1.2621774483536188886587657044524580e-29;
}
__device__ __forceinline__ unsigned __int128 shfl_down_128(unsigned __int128 v, int off) {
    const unsigned long long lo = __shfl_down_sync(0xffffffffu, (unsigned long long)v, off);
    const unsigned long long hi = __shfl_down_sync(0xffffffffu, (unsigned long long)(v >> 64), off);
    return ((unsigned __int128)hi << 64) | (unsigned __int128)lo;
}

template <int S>
__device__ __forceinline__ void forces_f64_body(const Dev &d, const VB &vb) {
    int bi = vb.y;
    const Body &b = d.bodies[bi];
    int lo[3] = {b.lo[0] - 1, b.lo[1] - 1, b.lo[2] - 1};
    int hi[3] = {b.hi[0] + 1, b.hi[1] + 1, b.hi[2] + 1};
    int n3[3] = {d.nx, d.ny, d.nz};
    for (int k = 0; k < 3; ++k) {
        if (!(d.periodic & (1u << k))) {
            lo[k] = lo[k] < 0 ? 0 : lo[k];
            hi[k] = hi[k] > n3[k] ? n3[k] : hi[k];
        } else if (hi[k] - lo[k] > n3[k]) {
            hi[k] = lo[k] + n3[k];
        }
    }
    unsigned __int128 acc[7] = {0, 0, 0, 0, 0, 0, 0};
    // the cells of the box around the body spread over all the body's blocks;
    // only cells next to an obstacle (neighbour-obstacle bit) can hold links
    const long long ncell = range_count(lo, hi);
    const int tidf = threadIdx.x + blockDim.x * threadIdx.y, nthr = blockDim.x * blockDim.y;
    for (long long kk = (long long)vb.x * nthr + tidf; kk < ncell; kk += (long long)vb.nx * nthr) {
        int x, y, z;
        range_cell(d, lo, hi, kk, x, y, z);
        long long i = x + (long long)d.nx * (y + (long long)d.ny * z);
        int fb = d.flags[i];
        int cl = fb & CL_MASK;
        if (!(fb & NB_OBST) || cl == CL_O) continue;
        {
            // double, in the order of the plain restatement
            const double phi_x = cl == CL_L ? 1.0 : (cl == CL_I ? d.phisrc[i] : 0.0);
            const double r[3] = {min_image(d, (x + 0.5) - b.o[0], 0), min_image(d, (y + 0.5) - b.o[1], 1),
                                 min_image(d, (z + 0.5) - b.o[2], 2)};
            bool have_rho = false;
            double rho_x = 0.0;
#pragma unroll 1
            for (int q = 1; q < Q; ++q) {
                long long si = nbr(d, x, y, z, -cx(q), -cy(q), -cz(q));
                if (si < 0 || clsv(d, si) != CL_O || d.bid[si] != bi) continue;
                double cuw = link_cuw(d, b, x, y, z, q);
                int qb = opp(q);
                double inner;
                if (cl == CL_G) {
                    inner = wd(q) * d.rho_g;
                } else {
                    double A = phi_x * Sto<S>::ldf(d.fsrc, qb, i, d.N);
                    double B = (1.0 - phi_x) * (wd(q) * d.rho_g);
                    double C;
                    if (cuw == 0.0) {
                        C = phi_x * 0.0;
                    } else {
                        if (!have_rho) {
                            rho_x = cell_density<S>(d, d.fsrc, i);
                            have_rho = true;
                        }
                        C = phi_x * (((3.0 * wd(q)) * rho_x) * cuw);
                    }
                    inner = (A + B) + C;
                }
                double g = 2.0 * inner;
                double F0 = cx(qb) * g, F1 = cy(qb) * g, F2 = cz(qb) * g;
                acc[0] += fixed96(F0);
                acc[1] += fixed96(F1);
                acc[2] += fixed96(F2);
                acc[3] += fixed96(r[1] * F2 - r[2] * F1);
                acc[4] += fixed96(r[2] * F0 - r[0] * F2);
                acc[5] += fixed96(r[0] * F1 - r[1] * F0);
                acc[6] += fixed96(fabs(g));
            }
        }
    }
    // block reduction of the exact integer sums (any order gives the same
    // bits); a warp without any link skips the tree (its sums are zeros).
    // The block's partials go out as 128-bit integers (low, high word).
    __shared__ unsigned __int128 sh[8][7];
    int tid = threadIdx.x + blockDim.x * threadIdx.y;
    int lane = tid & 31, wid = tid >> 5;
    const bool any = __any_sync(0xffffffffu, (acc[6] | acc[0] | acc[1] | acc[2]) != 0);
#pragma unroll
    for (int c = 0; c < 7; ++c) {
        unsigned __int128 v = acc[c];
        if (any)
            for (int off = 16; off > 0; off >>= 1) v += shfl_down_128(v, off);
        if (lane == 0) sh[wid][c] = v;
    }
    __syncthreads();
    if (tid < 7) {
        unsigned __int128 v = 0;
        for (int w = 0; w < 8; ++w) v += sh[w][tid];
        unsigned long long *p = reinterpret_cast<unsigned long long *>(d.part) +
                                2 * (((long long)bi * FORCE_BLOCKS + vb.x) * 7 + tid);
        p[0] = (unsigned long long)v;
        p[1] = (unsigned long long)(v >> 64);
    }
}

// Sum of a 64-bit integer over the 32 lanes of a warp: three limbs (bits
// 0-20, 21-41 and the signed rest) summed by warp reductions, whose 32-lane
// sums stay within 32 bits for |v| < 2^62.
__device__ __forceinline__ long long warp_sum64(long long v) {
    const unsigned c = (unsigned)(v & 0x1fffffll), b = (unsigned)((v >> 21) & 0x1fffffll);
    const int a = (int)(v >> 42);
    const unsigned sc = __reduce_add_sync(0xffffffffu, c), sb = __reduce_add_sync(0xffffffffu, b);
    const int sa = __reduce_add_sync(0xffffffffu, a);
    return (long long)sa * (1ll << 42) + (long long)sb * (1ll << 21) + (long long)sc;
}

// Float storages.  The rows (y, z) of the cell range around the body are
// spread over the body's warps, lanes along x (coalesced flag loads, no
// per-cell division); every sum is an integer, so the totals do not depend
// on that mapping.  The link term is split into the uniform gas-pressure part
// 2 w_q rho_G (exact integer sums of 36 (2 w_q) c_qbar and of the lever arm
// twice the cell centre) and the small remainder 2 (phi (f_qbar - w_q rho_G)
// + moving-wall part), computed in float from the stored deviations f - w and
// summed in fixed point.  The lever arm r is the cell's, so each part is
// summed over the cell's links first and its torque is r x that sum.
template <int S>
__device__ __forceinline__ void forces_float_body(const Dev &d, const VB &vb) {
    const int bi = vb.y;
    const Body &b = d.bodies[bi];
    int lo[3] = {b.lo[0] - 1, b.lo[1] - 1, b.lo[2] - 1};
    int hi[3] = {b.hi[0] + 1, b.hi[1] + 1, b.hi[2] + 1};
    const int n3[3] = {d.nx, d.ny, d.nz};
    for (int k = 0; k < 3; ++k) {
        if (!(d.periodic & (1u << k))) {
            lo[k] = lo[k] < 0 ? 0 : lo[k];
            hi[k] = hi[k] > n3[k] ? n3[k] : hi[k];
        } else if (hi[k] - lo[k] > n3[k]) {
            hi[k] = lo[k] + n3[k];
        }
    }
    long long ia[7] = {0, 0, 0, 0, 0, 0, 0};         // fixed-point remainder sums
    long long ik[3] = {0, 0, 0}, it[3] = {0, 0, 0};  // exact gas-pressure sums
    bool hit = false;
    // body state in float, rounded once per thread
    const float of[3] = {(float)b.o[0], (float)b.o[1], (float)b.o[2]};
    const float vf[3] = {(float)b.v[0], (float)b.v[1], (float)b.v[2]};
    const float wfv[3] = {(float)b.w[0], (float)b.w[1], (float)b.w[2]};
    const float rg = (float)d.rho_g, wrg1 = d.rg1_f;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, wid = tid >> 5, nwarp = (blockDim.x * blockDim.y) >> 5;
    const int lx = hi[0] - lo[0];
    const unsigned ly = (unsigned)(hi[1] - lo[1]), nrows = ly * (unsigned)(hi[2] - lo[2]);
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    // the range's cells in x-fastest order, 32 consecutive cells per warp
    // task (a row shorter or longer than 32 cells leaves no lanes idle); as
    // many of the body's blocks as give each warp LBMFS_FORCE_ROWS tasks, the
    // others contribute zeros
    const unsigned ncell = (unsigned)lx * nrows, ntask = (ncell + 31u) / 32u;
    const unsigned per_block = (unsigned)nwarp * LBMFS_FORCE_ROWS;
    const unsigned used = min((unsigned)vb.nx, (ntask + per_block - 1) / per_block);
    if ((unsigned)vb.x >= used) {
        if (tid < 7) d.part[((long long)bi * FORCE_BLOCKS + vb.x) * 7 + tid] = 0.0;
        return;
    }
    for (unsigned task = (unsigned)vb.x * nwarp + wid; task < ntask; task += used * nwarp) {
        {
            const unsigned kc = task * 32u + (unsigned)lane;
            if (kc >= ncell) continue;
            const unsigned row = kc / (unsigned)lx;
            const int xo = (int)(kc - row * (unsigned)lx);
            int y = lo[1] + (int)(row % ly), z = lo[2] + (int)(row / ly);
            if (y < 0 || y >= d.ny) y = ((y % d.ny) + d.ny) % d.ny;  // only periodic axes leave [0, n)
            if (z < 0 || z >= d.nz) z = ((z % d.nz) + d.nz) % d.nz;
            int x = lo[0] + xo;
            if (x < 0 || x >= d.nx) x = ((x % d.nx) + d.nx) % d.nx;
            const long long i = x + sy * (y + (long long)d.ny * z);
            const int fb = d.flags[i];
            const int cl = fb & CL_MASK;
            if (!(fb & NB_OBST) || cl == CL_O) continue;
            // directions into body bi: all neighbour classes requested at
            // once (linear offsets away from the grid faces), then the body
            // ids of the obstacle directions
            const bool inner = x > 0 && x < d.nx - 1 && y > 0 && y < d.ny - 1 && z > 0 && z < d.nz - 1;
            // a liquid or interface cell's link terms read its populations:
            // requested together with the neighbour classes
            float fc[Q];
            if (cl != CL_G) {
#pragma unroll
                for (int q = 0; q < Q; ++q) fc[q] = Sto<S>::ld(d.fsrc, q, i, d.N);
            }
            unsigned om = 0;
#pragma unroll
            for (int q = 1; q < Q; ++q) {
                const long long si = inner ? i - (cx(q) + cy(q) * sy + cz(q) * sz)
                                           : nbr(d, x, y, z, -cx(q), -cy(q), -cz(q));
                if (si >= 0 && clsv(d, si) == CL_O) om |= 1u << q;
            }
            unsigned lm = om;  // with one body every obstacle cell is its
            if (d.nb > 1) {
                lm = 0;
#pragma unroll
                for (int q = 1; q < Q; ++q)
                    if (om & (1u << q)) {
                        const long long si = inner ? i - (cx(q) + cy(q) * sy + cz(q) * sz)
                                                   : nbr(d, x, y, z, -cx(q), -cy(q), -cz(q));
                        if (d.bid[si] == bi) lm |= 1u << q;
                    }
            }
            if (!lm) continue;
            hit = true;
            const float phf = cl == CL_L ? 1.0f : (cl == CL_I ? (float)d.phisrc[i] : 0.0f);
            // lever arm from the cell centre (minimum image on periodic
            // axes): float for the small remainder, and twice the cell
            // centre as an integer for the exact gas-pressure part
            const int xyz[3] = {x, y, z};
            float rf[3];
            long long c2[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                int xk = xyz[k];
                rf[k] = ((float)xk + 0.5f) - of[k];
                if (d.periodic & (1u << k)) {
                    const int shn = (int)floorf(rf[k] / (float)n3[k] + 0.5f);
                    xk -= shn * n3[k];
                    rf[k] -= (float)(shn * n3[k]);
                }
                c2[k] = 2ll * xk + 1;
            }
            float rho_x = -1.0f;
            int kx = 0, ky = 0, kz = 0;  // sum of 36 (2 w_q) c_qbar over the links
            float gx = 0.0f, gy = 0.0f, gz = 0.0f, fabs_sum = 0.0f;
#pragma unroll
            for (int q = 1; q < Q; ++q) {
                if (!(lm & (1u << q))) continue;
                const int qb = opp(q);
                const int m36 = q <= 6 ? 4 : 2;  // 36 x 2 w_q
                float gdev = 0.0f;
                if (cl != CL_G) {
                    // u_w at the link midpoint, r + c_qbar / 2 from the body centre
                    const float px = rf[0] + 0.5f * cx(qb), py = rf[1] + 0.5f * cy(qb), pz = rf[2] + 0.5f * cz(qb);
                    const float ux = vf[0] + (wfv[1] * pz - wfv[2] * py);
                    const float uy = vf[1] + (wfv[2] * px - wfv[0] * pz);
                    const float uz = vf[2] + (wfv[0] * py - wfv[1] * px);
                    const float cuw = cx(q) * ux + cy(q) * uy + cz(q) * uz;
                    float C = 0.0f;
                    if (cuw != 0.0f) {
                        if (rho_x < 0.0f) {
                            float dr = 0.0f;
#pragma unroll
                            for (int k = 0; k < Q; ++k) dr += fc[k];
                            rho_x = 1.0f + dr;
                        }
                        C = phf * (3.0f * wf(q) * rho_x * cuw);
                    }
                    const float dev = fc[qb] + wf(q) * wrg1;
                    gdev = 2.0f * (phf * dev + C);
                }
                if (cx(qb)) {
                    kx += cx(qb) * m36;
                    gx += cx(qb) * gdev;
                }
                if (cy(qb)) {
                    ky += cy(qb) * m36;
                    gy += cy(qb) * gdev;
                }
                if (cz(qb)) {
                    kz += cz(qb) * m36;
                    gz += cz(qb) * gdev;
                }
                fabs_sum += fabsf((float)m36 * (rg * (1.0f / 36.0f)) + gdev);
            }
            ia[0] += fixed_point(gx, FX_FORCE);
            ia[1] += fixed_point(gy, FX_FORCE);
            ia[2] += fixed_point(gz, FX_FORCE);
            ia[3] += fixed_point(rf[1] * gz - rf[2] * gy, FX_TORQUE);
            ia[4] += fixed_point(rf[2] * gx - rf[0] * gz, FX_TORQUE);
            ia[5] += fixed_point(rf[0] * gy - rf[1] * gx, FX_TORQUE);
            ia[6] += fixed_point(fabs_sum, FX_FORCE);
            // gas-pressure part (rho_G / 36) K: its torque is
            // (rho_G / 36) (sum c2 x K / 2 - o x sum K)
            ik[0] += kx;
            ik[1] += ky;
            ik[2] += kz;
            it[0] += c2[1] * kz - c2[2] * ky;
            it[1] += c2[2] * kx - c2[0] * kz;
            it[2] += c2[0] * ky - c2[1] * kx;
        }
    }
    // warp sums, then the warps' sums in the block (integers: exact); a warp
    // without any link skips the reductions (its sums are zeros)
    __shared__ long long shi[8][13];
    const bool any = __any_sync(0xffffffffu, hit);
#pragma unroll
    for (int c = 0; c < 13; ++c) {
        long long v = c < 7 ? ia[c] : (c < 10 ? ik[c - 7] : it[c - 10]);
        if (any) v = warp_sum64(v);
        if (lane == 0) shi[wid][c] = any ? v : 0ll;
    }
    __syncthreads();
    if (tid < 7) {
        long long I = 0;
        for (int w = 0; w < nwarp; ++w) I += shi[w][tid];
        double v = (double)I * (tid >= 3 && tid < 6 ? 1.0 / (double)(1ll << FX_TORQUE) : 1.0 / (double)(1ll << FX_FORCE));
        if (tid < 6) {
            long long K[3] = {0, 0, 0}, T2[3] = {0, 0, 0};
            for (int w = 0; w < nwarp; ++w)
                for (int k = 0; k < 3; ++k) {
                    K[k] += shi[w][7 + k];
                    T2[k] += shi[w][10 + k];
                }
            const double g36 = d.rho_g / 36.0;
            if (tid < 3) {
                v += g36 * (double)K[tid];
            } else {
                const int k = tid - 3, k1 = (k + 1) % 3, k2 = (k + 2) % 3;
                // (sum c2 x K) / 2 - o x sum K, component k
                const double ox = b.o[k1] * (double)K[k2] - b.o[k2] * (double)K[k1];
                v += g36 * (0.5 * (double)T2[k] - ox);
            }
        }
        d.part[((long long)bi * FORCE_BLOCKS + vb.x) * 7 + tid] = v;
    }
}

template <int S>
__device__ __forceinline__ void forces_body(const Dev &d, const VB &vb) {
    if constexpr (S == 0) forces_f64_body<S>(d, vb);
    else forces_float_body<S>(d, vb);
}

template <int S>
__global__ void __launch_bounds__(256, S == 0 ? 2 : LBMFS_FORCE_MINB) k_forces(const __grid_constant__ Dev d) {
    forces_body<S>(d, vb_own());
}

// ---- C1 + C2 for liquid cells (Sec. 2.1 Eqs. stream, lbgk, forceterm;
// Sec. 2.3 Eq. noslip); interface cells are listed for k_interface
template <int S, int ZBMAX>
__device__ __forceinline__ void liquid_column(const Dev &d, bool in, int x, int y, int z0, int z1);
template <int S, int ZBMAX>
__device__ __forceinline__ void liquid_body_pair(const Dev &d, const VB &vb, int zb);

// A block covers BULK_THREADS consecutive cells of an xy-plane (row ends
// wrap to the next row, so narrow grids keep every lane busy) for zb
// consecutive z: grid (ceil(nx ny / BULK_THREADS), 1, ceil(nz / zb)).
template <int S, int ZBMAX>
__device__ __forceinline__ void liquid_body(const Dev &d, const VB &vb, int zb) {
    // a tile above the previous step's fluid (plus a margin) holds only gas
    if ((int)(vb.z * zb) > __ldg(d.ztop_rd) + ZTOP_MARGIN) return;
    const unsigned p = vb.x * BULK_THREADS + threadIdx.x;
    const bool in = p < (unsigned)d.nx * (unsigned)d.ny;
    const int y = in ? (int)(p / (unsigned)d.nx) : 0;
    const int x = in ? (int)p - y * d.nx : 0;
    const int z0 = vb.z * zb;
    const int z1 = min(z0 + zb, d.nz);
    liquid_column<S, ZBMAX>(d, in, x, y, z0, z1);
}
// the bulk body of a storage: one cell per thread (double), two (float)
template <int S, int ZBMAX>
__device__ __forceinline__ void bulk_body(const Dev &d, const VB &vb, int zb) {
    if constexpr (S == 0 || !LBMFS_BULK_PAIR) liquid_body<S, ZBMAX>(d, vb, zb);
    else if (d.pair_ok) liquid_body_pair<S, ZBMAX>(d, vb, zb);
    else liquid_body<S, ZBMAX>(d, vb, zb);
}
template <int S>
__global__ void __launch_bounds__(BULK_THREADS, S == 0 ? 1 : (LBMFS_BULK_PAIR ? LBMFS_PAIR_MINB : LBMFS_BULK_MINB))
    k_liquid(const __grid_constant__ Dev d) {
    bulk_body<S, LBMFS_BULK_ZB>(d, vb_own(), LBMFS_BULK_ZB);
}

template <int S>
__device__ __forceinline__ void collide_store(const Dev &d, typename Sto<S>::R *fp, long long i) {
    using P = Sto<S>;
    if constexpr (!P::shifted) {
        double fn[Q];
        collide_d(d, fp, fn);
        double r = 0.0;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            P::st(d.fdst, q, i, d.N, fn[q]);
            r += fn[q];
        }
        if (!(r == r) || r <= 0.0) atomicOr(d.status, ST_NONFINITE);
    } else {
        // fp in the storage's raw units (to_raw)
        void *g = d.fdst;
        const long long N = d.N;
        float rho = collide_store_v<P::SCALE, float>(d, fp, [&](int q, float v) { return P::st_raw(g, q, i, N, v); });
        if (!vpos_finite(rho)) atomicOr(d.status, ST_NONFINITE);
    }
}

// populations gathered as values into the storage's raw units (q >= 1 times
// the FP16 storage's scale; exact)
template <int S> __device__ __forceinline__ void to_raw(typename Sto<S>::R *fp) {
    if constexpr (S == 2) {
#pragma unroll
        for (int q = 1; q < Q; ++q) fp[q] *= F16_SCALE;
    }
}

// populations arriving at a liquid cell with an obstacle or wall neighbour, or
// on a periodic seam: per-direction source classes, bounce-back where the
// source is solid (Eq. noslip), 6 w_q rho_x c_q.u_w added where the solid
// moves.  Three rounds of independent loads: the 18 source classes with the
// cell's own 19 populations; the pulled populations with the body ids of the
// obstacle sources; the state of the body (one body for all links when they
// share it, the common case; per link otherwise).  rho_x, in double for the
// FP64 storage and in float for the float storages, sums the own populations
// in q order.  Returns the mass the moving links add to the cell (for the
// ledger).
template <int S>
__device__ __forceinline__ double gather_general(const Dev &d, int x, int y, int z, long long i,
                                                 typename Sto<S>::R *fp) {
    using P = Sto<S>;
    using R = typename P::R;
    const long long N = d.N;
    long long src[Q];
    int ns[Q];
    R own[Q];
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        src[q] = nbr(d, x, y, z, -cx(q), -cy(q), -cz(q));
        ns[q] = src[q] < 0 ? CL_WALL : clsv(d, src[q]);
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) own[q] = P::ld(d.fsrc, q, i, N);
    unsigned moving = 0, obst = 0;  // directions with a moving solid source / an obstacle source
    int bq[Q];
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const bool pull = ns[q] == CL_L || ns[q] == CL_I;
        fp[q] = pull ? P::ld(d.fsrc, q, src[q], N) : own[opp(q)];
        bq[q] = ns[q] == CL_O ? d.bid[src[q]] : -1;
        if (ns[q] == CL_O) obst |= 1u << q;
        if (ns[q] == CL_O || (ns[q] == CL_WALL && d.walls_move)) moving |= 1u << q;
        if (ns[q] == CL_G) atomicOr(d.status, ST_LIQUID_GAS);
    }
    fp[0] = own[0];
    if (!moving) return 0.0;
    int b0 = -1;
    bool one = true;  // every obstacle link belongs to body b0
#pragma unroll
    for (int q = 1; q < Q; ++q)
        if (obst & (1u << q)) {
            if (b0 < 0) b0 = bq[q];
            one = one && bq[q] == b0;
        }
    R wall = 0;
    if constexpr (S == 0) {
        double rho_x = 0.0;
#pragma unroll
        for (int q = 0; q < Q; ++q) rho_x += own[q];
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            if (!(moving & (1u << q))) continue;
            const double cuw = (obst & (1u << q)) ? link_cuw(d, d.bodies[one ? b0 : bq[q]], x, y, z, q)
                                                  : wall_cuw(d, x, y, z, q);
            if (cuw == 0.0) continue;
            const double srcm = ((6.0 * wd(q)) * rho_x) * cuw;
            fp[q] = fp[q] + srcm;
            wall += srcm;
        }
    } else {
        float dr = 0.0f;
#pragma unroll
        for (int k = 0; k < Q; ++k) dr += own[k];
        const float rho_x = 1.0f + dr;
        BodyF bf0;
        if (b0 >= 0) bf0 = body_f(d.bodies[b0], x, y, z);
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            if (!(moving & (1u << q))) continue;
            const float cuw = (obst & (1u << q))
                                  ? (one ? link_cuw_f(d, bf0, q) : link_cuw_f(d, d.bodies[bq[q]], x, y, z, q))
                                  : (float)wall_cuw(d, x, y, z, q);
            if (cuw == 0.0f) continue;
            const float srcm = ((6.0f * wf(q)) * rho_x) * cuw;
            fp[q] = fp[q] + srcm;
            wall += srcm;
        }
    }
    return (double)wall;
}

template <int S>
__device__ __forceinline__ double liquid_cell_general(const Dev &d, int x, int y, int z, long long i) {
    typename Sto<S>::R fp[Q];
    const double wall = gather_general<S>(d, x, y, z, i, fp);
    to_raw<S>(fp);
    collide_store<S>(d, fp, i);
    return wall;
}

// C1 + C2 for the liquid cells the bulk kernel listed (an obstacle among the
// neighbours, or a grid face with moving walls): the general gather, then the
// collision.  They read the source grid and write their own cell of the
// destination grid only, as the bulk kernel would have.
// The mass the moving links add is summed per warp and goes to the ledger
// with one atomic per warp (thousands of cells adding to one address would
// queue on it).  Blocks of GEN_THREADS spread the few listed cells over many
// SMs.
constexpr int GEN_THREADS = 128;
template <int S> __device__ __forceinline__ void general_body(const Dev &d, const VB &vb) {
    double wacc = 0.0;
    LIST_LOOP(WL_GEN, g) {
        const long long i = d.list[WL_GEN][it_g];
        int x, y, z;
        if constexpr (S != 0) {
            // the float storages hold N * 19 < 2^32 elements
            const uint32_t i32 = (uint32_t)i, yz = i32 / (uint32_t)d.nx;
            x = (int)(i32 - yz * (uint32_t)d.nx);
            y = (int)(yz % (uint32_t)d.ny);
            z = (int)(yz / (uint32_t)d.ny);
        } else {
            coords(d, i, x, y, z);
        }
        wacc += liquid_cell_general<S>(d, x, y, z, i);
    }
    if (__any_sync(0xffffffffu, wacc != 0.0)) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) wacc += __shfl_xor_sync(0xffffffffu, wacc, off);
        if ((threadIdx.x & 31) == 0 && wacc != 0.0) atomicAdd(&d.ledger[LG_WALL], wacc);
    }
}
template <int S>
__global__ void __launch_bounds__(GEN_THREADS, 1) k_general(const __grid_constant__ Dev d) {
    general_body<S>(d, vb_own());
}

// One liquid cell (class byte c, coordinates x, y, z, index i; not a
// general_cell): gather its 18 arriving populations by the cheapest rule that
// holds for it, collide and store.
template <int S>
__device__ __forceinline__ void liquid_one(const Dev &d, int c, int x, int y, int z, long long i) {
    using P = Sto<S>;
    using R = typename P::R;
    const long long N = d.N;
    R fp[Q];
    if (c == CL_L && x > 0 && x < d.nx - 1 && y > 0 && y < d.ny - 1 && z > 0 && z < d.nz - 1) {
        // no obstacle or wall in the neighbourhood and a liquid cell never
        // touches gas: plain pull from the 18 neighbours
        const long long sy = d.nx, sz = (long long)d.nx * d.ny;
#pragma unroll
        for (int q = 1; q < Q; ++q) fp[q] = P::ldg_raw(d.fsrc, q, i - (cx(q) + cy(q) * sy + cz(q) * sz), N);
        fp[0] = P::ldg_raw(d.fsrc, 0, i, N);
    } else if (c == CL_L && !d.periodic && !d.walls_move) {
        // on a face of a grid without periodic axes, no obstacle
        // neighbour: a source beyond a face is a resting wall, which
        // returns the cell's own opposite population (Eq. noslip, u_w = 0)
        const long long sy = d.nx, sz = (long long)d.nx * d.ny;
        const bool xl = x == 0, xh = x == d.nx - 1, yl = y == 0, yh = y == d.ny - 1, zl = z == 0, zh = z == d.nz - 1;
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            const bool out = (cx(q) > 0 && xl) || (cx(q) < 0 && xh) || (cy(q) > 0 && yl) || (cy(q) < 0 && yh) ||
                             (cz(q) > 0 && zl) || (cz(q) < 0 && zh);
            fp[q] = out ? P::ldg_raw(d.fsrc, opp(q), i, N)
                        : P::ldg_raw(d.fsrc, q, i - (cx(q) + cy(q) * sy + cz(q) * sz), N);
        }
        fp[0] = P::ldg_raw(d.fsrc, 0, i, N);
    } else {
        // on a face with periodic axes: pull across the seams, walls as above
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            const long long si = nbr(d, x, y, z, -cx(q), -cy(q), -cz(q));
            fp[q] = si >= 0 ? P::ldg_raw(d.fsrc, q, si, N) : P::ldg_raw(d.fsrc, opp(q), i, N);
        }
        fp[0] = P::ldg_raw(d.fsrc, 0, i, N);
    }
    collide_store<S>(d, fp, i);  // one copy of the collision in the kernel
}
// A liquid cell the bulk kernel leaves to k_general (class byte c): an
// obstacle among its neighbours (the neighbour-obstacle bit), or a grid face
// when the walls move.  Its class, body-id and body-state loads depend on one
// another; in k_general they hold none of the bulk kernel's warps.
__device__ __forceinline__ bool general_cell(const Dev &d, int c, int x, int y, int z) {
    return (c & CL_MASK) == CL_L &&
           (c != CL_L || (d.walls_move && !(x > 0 && x < d.nx - 1 && y > 0 && y < d.ny - 1 && z > 0 && z < d.nz - 1)));
}

// The cells (x, y, z0 .. z1-1) of one thread.  The flags of the whole column
// come in one round of loads, so a thread whose column holds no fluid leaves
// after one memory latency, and a fluid cell waits on its populations only.
template <int S, int ZBMAX>
__device__ __forceinline__ void liquid_column(const Dev &d, bool in, int x, int y, int z0, int z1) {
    static_assert(ZBMAX <= 8, "flags of a column (z1 - z0 <= ZBMAX) are packed into 64 bits");
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    long long i = (long long)x + sy * (y + (long long)d.ny * z0);
    uint64_t fl = 0;
#pragma unroll
    for (int k = 0; k < ZBMAX; ++k)
        if (in && z0 + k < z1) fl |= (uint64_t)d.flags[i + k * sz] << (8 * k);
    // record the highest tile holding liquid or interface cells (one atomic per warp)
    if (__any_sync(0xffffffffu, (fl & 0x0303030303030303ull) != 0) && (threadIdx.x & 31) == 0)
        atomicMax(d.ztop_wr, z1 - 1);
    if (fl == 0) return;
#pragma unroll 1
    for (int z = z0; z < z1; ++z, i += sz) {
        const int c = (int)(fl & 0xff);
        fl >>= 8;
        wl_append(d, (c & CL_MASK) == CL_I, WL_IFACE, (uint32_t)i);
        const bool gen = general_cell(d, c, x, y, z);
        wl_append(d, gen, WL_GEN, (uint32_t)i);
        if ((c & CL_MASK) != CL_L || gen) continue;
        liquid_one<S>(d, c, x, y, z, i);  // one copy of the collision in the kernel
    }
}

// Float storages on grids with nx and the cell count even (Dev::pair_ok):
// two cells per thread, the cells p = 2t and 2t + 1 of the xy-plane (a block
// covers 2 BULK_THREADS of them), zb z-planes.  Every pair then starts on an
// even element of each plane, so where both cells are interior liquid cells
// -- almost every liquid cell -- each direction's two arriving populations come
// in one load (two for the +-x directions, whose sources start one element
// off), the two cells collide together in packed FP32 arithmetic (float2
// operations with the same roundings per cell as the single-cell path), and
// each direction's pair is stored at once.  Every other cell takes the
// single-cell path.
template <int S, int ZBMAX>
__device__ __forceinline__ void liquid_body_pair(const Dev &d, const VB &vb, int zb) {
    using P = Sto<S>;
    static_assert(S != 0, "pairs serve the float storages");
    if ((int)(vb.z * zb) > __ldg(d.ztop_rd) + ZTOP_MARGIN) return;
    const unsigned nxy = (unsigned)d.nx * (unsigned)d.ny;
    const unsigned p0 = 2u * (vb.x * BULK_THREADS + threadIdx.x);
    const bool in = p0 < nxy;  // nx even: the pair lies in one row
    const int y0 = in ? (int)(p0 / (unsigned)d.nx) : 0;
    const int x0 = in ? (int)p0 - y0 * d.nx : 0;
    const int z0 = vb.z * zb, z1 = min(z0 + zb, d.nz);
    const uint32_t sy = (uint32_t)d.nx, sz = (uint32_t)nxy;
    uint32_t j = p0 + sz * (uint32_t)z0;  // cell 0 at z (even); cell 1 is j + 1
    // classes of both columns in one round of loads: cell 0 in the low byte
    unsigned fl[ZBMAX];
    unsigned any = 0;
#pragma unroll
    for (int k = 0; k < ZBMAX; ++k) {
        fl[k] = (in && z0 + k < z1) ? (unsigned)*reinterpret_cast<const uint16_t *>(d.flags + j + k * sz) : 0u;
        any |= fl[k];
    }
    if (__any_sync(0xffffffffu, (any & 0x0303u) != 0) && (threadIdx.x & 31) == 0) atomicMax(d.ztop_wr, z1 - 1);
    if (any == 0) return;
    const bool pair_xy = x0 > 0 && x0 + 1 < d.nx - 1 && y0 > 0 && y0 < d.ny - 1;
    const Planes<S> pl(d.fsrc, d.fdst, d.N);
#pragma unroll 1
    for (int k = 0; k < ZBMAX; ++k, j += sz) {
        const int z = z0 + k;
        if (z >= z1) break;
        const int c0 = (int)(fl[k] & 0xffu), c1 = (int)(fl[k] >> 8);
        wl_append(d, (c0 & CL_MASK) == CL_I, WL_IFACE, j);
        wl_append(d, (c1 & CL_MASK) == CL_I, WL_IFACE, j + 1);
        const bool g0 = general_cell(d, c0, x0, y0, z), g1 = general_cell(d, c1, x0 + 1, y0, z);
        wl_append(d, g0, WL_GEN, j);
        wl_append(d, g1, WL_GEN, j + 1);
        if (pair_xy && c0 == CL_L && c1 == CL_L && z > 0 && z < d.nz - 1) {
            float2 fp[Q];
#pragma unroll
            for (int q = 1; q < Q; ++q) {
                const uint32_t src = j - (uint32_t)cx(q) - (uint32_t)cy(q) * sy - (uint32_t)cz(q) * sz;
                fp[q] = cx(q) == 0 ? pl.ld2(q, src) : pl.ld2_odd(q, src);
            }
            fp[0] = pl.ld2(0, j);
            const float2 rho = collide_store_v<P::SCALE, float2>(d, fp, [&](int q, float2 v) { return pl.st2(q, j, v); });
            if (!vpos_finite(rho)) atomicOr(d.status, ST_NONFINITE);
        } else {
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                const int c = h ? c1 : c0;
                if ((c & CL_MASK) != CL_L || (h ? g1 : g0)) continue;
                liquid_one<S>(d, c, x0 + h, y0, z, (long long)(j + h));
            }
        }
    }
}

// ---------------------------------------- software-pipelined bulk kernel
//
// Each thread copies the 19 populations its cell will pull at the next z into
// private shared-memory slots with cp.async (4-byte copies, no register held
// while in flight) before it collides the cell at the current z: two planes of
// loads in flight per thread.  A thread reads only its own slots, so no block
// barrier is needed; cp.async.wait_group orders the copies with the reads.
// FP16 storage copies the aligned 4-byte word holding the wanted half.

__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int S> struct Pipe;
template <> struct Pipe<1> {
    static __device__ __forceinline__ const void *src(const Dev &d, int q, long long e) {
        return reinterpret_cast<const float *>(d.fsrc) + (long long)q * d.N + e;
    }
    static __device__ __forceinline__ float get(const uint32_t *slot, int q, long long, long long) {
        return __uint_as_float(slot[q * BULK_THREADS]);
    }
};
template <> struct Pipe<2> {
    static __device__ __forceinline__ const void *src(const Dev &d, int q, long long e) {
        if (q == 0) return reinterpret_cast<const float *>(d.fsrc) + e;
        const __half *h = reinterpret_cast<const __half *>(reinterpret_cast<const float *>(d.fsrc) + d.N) +
                          (long long)(q - 1) * d.N + e;
        return reinterpret_cast<const void *>(reinterpret_cast<uintptr_t>(h) & ~(uintptr_t)3);
    }
    static __device__ __forceinline__ float get(const uint32_t *slot, int q, long long e, long long N) {
        uint32_t w = slot[q * BULK_THREADS];
        if (q == 0) return __uint_as_float(w);
        // the half planes start 4-byte aligned; the parity of the half's index
        // counted from there picks the half within the copied word
        long long h = (long long)(q - 1) * N + e;
        unsigned short hb = (unsigned short)((h & 1) ? (w >> 16) : (w & 0xffffu));
        return __half2float(__ushort_as_half(hb)) * F16_INV_SCALE;
    }
};

template <int S>
__global__ void __launch_bounds__(BULK_THREADS, LBMFS_BULK_MINB) k_liquid_pipe(Dev d) {
    // this variant visits every tile: record the grid's top so the next step skips none
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) atomicMax(d.ztop_wr, d.nz - 1);
    using P = Sto<S>;
    __shared__ uint32_t slots[2][Q][BULK_THREADS];
    const int tid = threadIdx.x;
    const int x = blockIdx.x * BULK_THREADS + tid, y = blockIdx.y;
    const int z0 = blockIdx.z * LBMFS_BULK_PIPE_ZB, z1 = min(z0 + LBMFS_BULK_PIPE_ZB, d.nz);
    const bool in = x < d.nx;
    const bool xyin = x > 0 && x < d.nx - 1 && y > 0 && y < d.ny - 1;
    const long long sx = 1, sy = d.nx, sz = (long long)d.nx * d.ny;
    const long long irow = (long long)(in ? x : 0) + (long long)d.nx * y;
    auto flag_at = [&](int z) -> int { return (in && z < z1) ? (int)d.flags[irow + sz * z] : 0; };
    auto fast = [&](int fl, int z) -> bool { return fl == CL_L && xyin && z > 0 && z < d.nz - 1; };
    auto issue = [&](int z, int b) {
        const long long i = irow + sz * z;
#pragma unroll
        for (int q = 0; q < Q; ++q)
            cp_async4(&slots[b][q][tid], Pipe<S>::src(d, q, i - (cx(q) * sx + cy(q) * sy + cz(q) * sz)));
    };
    int fl_cur = flag_at(z0);
    bool fast_cur = fast(fl_cur, z0);
    if (fast_cur) issue(z0, 0);
    cp_async_commit();
    int fl_next = flag_at(z0 + 1);
#pragma unroll 1
    for (int z = z0; z < z1; ++z) {
        const int b = (z - z0) & 1;
        const bool fast_next = z + 1 < z1 && fast(fl_next, z + 1);
        if (fast_next) issue(z + 1, b ^ 1);
        cp_async_commit();
        const int fl_after = flag_at(z + 2);
        const long long i = irow + sz * z;
        wl_append(d, (fl_cur & CL_MASK) == CL_I, WL_IFACE, (uint32_t)i);
        if (fast_cur) {
            cp_async_wait<1>();
            float fp[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q)
                fp[q] = Pipe<S>::get(&slots[b][0][tid], q, i - (cx(q) * sx + cy(q) * sy + cz(q) * sz), d.N);
            to_raw<S>(fp);
            collide_store<S>(d, fp, i);
        } else if ((fl_cur & CL_MASK) == CL_L) {
            const double w = liquid_cell_general<S>(d, x, y, z, i);
            if (w != 0.0) atomicAdd(&d.ledger[LG_WALL], w);
        }
        fl_cur = fl_next;
        fl_next = fl_after;
        fast_cur = fast_next;
    }
    cp_async_wait<0>();
}

// ------------------------------------------------ staged bulk kernel (TMA)
//
// One block owns a row segment of BULK_THREADS cells at (y, z) for
// LBMFS_BULK_ZB consecutive z.  For every z it needs, per direction q, the
// source row (y - c_qy, z - c_qz) of plane q shifted by -c_qx: thread 0 stages
// those 19 rows (each widened by a 16-byte halo on both sides so that every
// copy starts 16-byte aligned) into shared memory with 1-D bulk copies that
// complete on an mbarrier, one z ahead of the rows being computed (double
// buffer).  Rows whose segment holds no interior liquid cell (gas, or the
// grid's boundary layers) are not staged.  Cells that need more than a plain
// pull (obstacle or wall neighbours) use the global-memory path.

template <int S> struct Stage;
template <> struct Stage<1> {  // float planes, halo 4 elements
    static constexpr int H = 4;
    static constexpr int ROW = BULK_THREADS + 2 * H;  // elements per staged row
    static constexpr int BYTES = Q * ROW * 4;
    static __device__ __forceinline__ const char *src(const Dev &d, int q, long long e) {
        return reinterpret_cast<const char *>(reinterpret_cast<const float *>(d.fsrc) + (long long)q * d.N + e);
    }
    static __device__ __forceinline__ int row_bytes(int) { return ROW * 4; }
    static __device__ __forceinline__ int row_off(int q) { return q * ROW * 4; }
    static __device__ __forceinline__ float get(const char *stage, int q, int k) {
        return reinterpret_cast<const float *>(stage + row_off(q))[k];
    }
};
template <> struct Stage<2> {  // q = 0 float (halo 4), q >= 1 half (halo 8)
    static constexpr int H0 = 4, H = 8;
    static constexpr int ROW0 = BULK_THREADS + 2 * H0, ROW = BULK_THREADS + 2 * H;
    static constexpr int BYTES = ROW0 * 4 + (Q - 1) * ROW * 2;
    static __device__ __forceinline__ const char *src(const Dev &d, int q, long long e) {
        if (q == 0) return reinterpret_cast<const char *>(reinterpret_cast<const float *>(d.fsrc) + e);
        const __half *hb = reinterpret_cast<const __half *>(reinterpret_cast<const float *>(d.fsrc) + d.N);
        return reinterpret_cast<const char *>(hb + (long long)(q - 1) * d.N + e);
    }
    static __device__ __forceinline__ int row_bytes(int q) { return q == 0 ? ROW0 * 4 : ROW * 2; }
    static __device__ __forceinline__ int row_off(int q) { return q == 0 ? 0 : ROW0 * 4 + (q - 1) * ROW * 2; }
    static __device__ __forceinline__ float get(const char *stage, int q, int k) {
        if (q == 0) return reinterpret_cast<const float *>(stage)[k];
        return __half2float(reinterpret_cast<const __half *>(stage + row_off(q))[k]) * F16_INV_SCALE;
    }
};


__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: gives up after ~2^22 polls (each try_wait also suspends for a
// hardware-chosen interval), far beyond any copy latency
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

template <int S>
__device__ __forceinline__ void stage_row(const Dev &d, char *stage, uint64_t *bar, int x0, int y, int z) {
    using G = Stage<S>;
    fence_async_shared();
    mbar_expect_tx(bar, G::BYTES);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        // the copy starts 16-byte aligned at x0 - h for every direction; the
        // x shift -c_qx is applied when the row is read
        int h = (S == 2 && q > 0) ? Stage<2>::H : 4;
        long long e = (long long)d.nx * ((y - cy(q)) + (long long)d.ny * (z - cz(q))) + x0 - h;
        bulk_g2s(stage + G::row_off(q), G::src(d, q, e), G::row_bytes(q), bar);
    }
}

template <int S>
__global__ void __launch_bounds__(BULK_THREADS, LBMFS_BULK_MINB) k_liquid_tma(Dev d) {
    // this variant visits every tile: record the grid's top so the next step skips none
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) atomicMax(d.ztop_wr, d.nz - 1);
    using P = Sto<S>;
    using G = Stage<S>;
    extern __shared__ __align__(128) char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);  // two mbarriers
    char *buf0 = smem + 128;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * BULK_THREADS, x = x0 + tid, y = blockIdx.y;
    const int z0 = blockIdx.z * LBMFS_BULK_ZB, z1 = min(z0 + LBMFS_BULK_ZB, d.nz);
    const bool in = x < d.nx;
    const bool xin = x > 0 && x < d.nx - 1;
    const bool yin = y > 0 && y < d.ny - 1;
    bool failed = false;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    unsigned phase[2] = {0u, 0u};
    auto flag_at = [&](int z) -> int {
        return (in && z < z1) ? (int)d.flags[x + (long long)d.nx * (y + (long long)d.ny * z)] : 0;
    };
    auto fast = [&](int fl, int z) -> bool { return fl == CL_L && xin && yin && z > 0 && z < d.nz - 1; };
    int fl_cur = flag_at(z0);
    bool staged_cur = __syncthreads_or(fast(fl_cur, z0)) != 0;
    if (staged_cur && tid == 0) stage_row<S>(d, buf0, &bar[0], x0, y, z0);
    int fl_next = flag_at(z0 + 1);
    for (int z = z0; z < z1; ++z) {
        const int b = (z - z0) & 1;
        char *stage = buf0 + b * G::BYTES;
        // every thread is done with the other buffer (previous row) here
        bool staged_next = __syncthreads_or(z + 1 < z1 && fast(fl_next, z + 1)) != 0;
        if (staged_next && tid == 0) stage_row<S>(d, buf0 + (b ^ 1) * G::BYTES, &bar[b ^ 1], x0, y, z + 1);
        int fl_after = flag_at(z + 2);
        const long long i = (long long)(in ? x : 0) + (long long)d.nx * (y + (long long)d.ny * z);
        const int c = fl_cur;
        wl_append(d, (c & CL_MASK) == CL_I, WL_IFACE, (uint32_t)i);
        if (staged_cur) {
            // every thread keeps stepping through the block barriers even if
            // its wait gives up; the outcome is settled after the loop
            if (!mbar_wait(&bar[b], phase[b])) failed = true;
            phase[b] ^= 1u;
        }
        if (fast(c, z)) {
            float fp[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) fp[q] = G::get(stage, q, tid + ((S == 2 && q > 0) ? Stage<2>::H : 4) - cx(q));
            to_raw<S>(fp);
            collide_store<S>(d, fp, i);
        } else if ((c & CL_MASK) == CL_L) {
            const double w = liquid_cell_general<S>(d, x, y, z, i);
            if (w != 0.0) atomicAdd(&d.ledger[LG_WALL], w);
        }
        fl_cur = fl_next;
        fl_next = fl_after;
        staged_cur = staged_next;
    }
    if (__syncthreads_or(failed)) {
        // a staged copy did not complete in time: report it; every staged row
        // has had its (bounded) wait above, so no copy is left unawaited
        if (tid == 0) atomicOr(d.status, ST_TIMEOUT);
    }
}

// fill level of a neighbour as seen by the normal estimate
__device__ __forceinline__ double fill_seen(const Dev &d, long long ni, double own) {
    int c = cls(d, ni);
    if (c == CL_L) return 1.0;
    if (c == CL_I) return d.phisrc[ni];
    if (c == CL_G) return 0.0;
    return own;
}

// ---- Sec. 2.2 Laplace pressure: mean curvature kappa = div(n^)/2 at an
// interface cell from the unit normals of its six axis neighbours (central
// differences; the normals are those of the reconstruction, -grad(phi) with
// the same fill-level rules); an obstacle or wall neighbour takes the cell's
// own unit normal nc.  A liquid sphere of radius R has kappa = 1/R.
__device__ __forceinline__ void unit_vec_d(const double *n, double *out) {
    double len = sqrt((n[0] * n[0] + n[1] * n[1]) + n[2] * n[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) out[k] = len > 0.0 ? n[k] / len : 0.0;
}
__device__ __noinline__ double curvature_d(const Dev &d, int x, int y, int z, double nc0, double nc1, double nc2) {
    const double nc[3] = {nc0, nc1, nc2};
    double div = 0.0;
    for (int k = 0; k < 3; ++k) {
        double comp[2];
        for (int sgn = 0; sgn < 2; ++sgn) {
            const int s = sgn ? -1 : 1;
            const long long yi = nbr(d, x, y, z, k == 0 ? s : 0, k == 1 ? s : 0, k == 2 ? s : 0);
            const int c = cls(d, yi);
            if (c == CL_WALL || c == CL_O) {
                comp[sgn] = nc[k];
                continue;
            }
            int yx, yy, yz;
            coords(d, yi, yx, yy, yz);
            const double own = c == CL_L ? 1.0 : (c == CL_I ? d.phisrc[yi] : 0.0);
            double n[3], nh[3];
            for (int j = 0; j < 3; ++j) {
                const double pm = fill_seen(d, nbr(d, yx, yy, yz, j == 0 ? -1 : 0, j == 1 ? -1 : 0, j == 2 ? -1 : 0), own);
                const double pp = fill_seen(d, nbr(d, yx, yy, yz, j == 0 ? 1 : 0, j == 1 ? 1 : 0, j == 2 ? 1 : 0), own);
                n[j] = 0.5 * (pm - pp);
            }
            unit_vec_d(n, nh);
            comp[sgn] = nh[k];
        }
        div += comp[0] - comp[1];
    }
    return 0.25 * div;
}
// the same in float for the float storages
__device__ __noinline__ float curvature_f(const Dev &d, int x, int y, int z, float nc0, float nc1, float nc2) {
    const float nc[3] = {nc0, nc1, nc2};
    float div = 0.0f;
    for (int k = 0; k < 3; ++k) {
        float comp[2];
        for (int sgn = 0; sgn < 2; ++sgn) {
            const int s = sgn ? -1 : 1;
            const long long yi = nbr(d, x, y, z, k == 0 ? s : 0, k == 1 ? s : 0, k == 2 ? s : 0);
            const int c = cls(d, yi);
            if (c == CL_WALL || c == CL_O) {
                comp[sgn] = nc[k];
                continue;
            }
            int yx, yy, yz;
            coords(d, yi, yx, yy, yz);
            const double own = c == CL_L ? 1.0 : (c == CL_I ? d.phisrc[yi] : 0.0);
            float n[3];
            for (int j = 0; j < 3; ++j) {
                const float pm = (float)fill_seen(d, nbr(d, yx, yy, yz, j == 0 ? -1 : 0, j == 1 ? -1 : 0, j == 2 ? -1 : 0), own);
                const float pp = (float)fill_seen(d, nbr(d, yx, yy, yz, j == 0 ? 1 : 0, j == 1 ? 1 : 0, j == 2 ? 1 : 0), own);
                n[j] = 0.5f * (pm - pp);
            }
            const float len = sqrtf((n[0] * n[0] + n[1] * n[1]) + n[2] * n[2]);
            comp[sgn] = len > 0.0f ? n[k] / len : 0.0f;
        }
        div += comp[0] - comp[1];
    }
    return 0.25f * div;
}

// ---- C1 + C2 for interface cells of the float storages: three threads per
// cell.  Member r of a cell's trio owns three pairs of opposite directions
// (r = 0: W/E, TW/BE, TE/BW; r = 1: N/S, TN/BS, TS/BN; r = 2: T/B, NW/SE,
// NE/SW), so the bounce-back, reconstruction and mass exchange of a link,
// which pair q with qbar, stay inside one thread, and the first pair of
// member r is the axis pair of component r of the normal.  Sums over all
// directions (density, momentum, exchanged mass, the stored cell sum) are
// formed per member and added as member 0 + member 1 + member 2 on all three
// threads, so a trio agrees bit for bit.  Ten trios per warp; lanes 30 and 31
// shadow the last trio and write nothing.

// neighbour (x + dx, y + dy, z + dz) as a 32-bit cell index without
// branches (periodic axes wrap); -1 beyond a wall
__device__ __forceinline__ int nbr32(const Dev &d, int x, int y, int z, int dx, int dy, int dz) {
    int px = x + dx, py = y + dy, pz = z + dz;
    const bool ox = px < 0 || px >= d.nx, oy = py < 0 || py >= d.ny, oz = pz < 0 || pz >= d.nz;
    px = px < 0 ? px + d.nx : (px >= d.nx ? px - d.nx : px);
    py = py < 0 ? py + d.ny : (py >= d.ny ? py - d.ny : py);
    pz = pz < 0 ? pz + d.nz : (pz >= d.nz ? pz - d.nz : pz);
    const bool wall = (ox && !(d.periodic & 1u)) || (oy && !(d.periodic & 2u)) || (oz && !(d.periodic & 4u));
    return wall ? -1 : px + d.nx * (py + d.ny * pz);
}
// moving population q >= 1 of cell j as a float deviation (no branch on q)
template <int S> __device__ __forceinline__ float trio_ld(const void *g, int q, uint32_t j, long long N) {
    if constexpr (S == 1) return __ldg(reinterpret_cast<const float *>(g) + ((long long)q * N + j));
    else return __half2float(__ldg(Sto<2>::hp(g, N) + ((long long)(q - 1) * N + j))) * F16_INV_SCALE;
}
// store moving population q >= 1 of cell j; returns the value as stored
template <int S> __device__ __forceinline__ float trio_st(void *g, int q, uint32_t j, long long N, float v) {
    if constexpr (S == 1) {
        pop_st(reinterpret_cast<float *>(g) + ((long long)q * N + j), v);
        return v;
    } else {
        const __half h = __float2half_rn(v * F16_SCALE);
        pop_st(const_cast<__half *>(Sto<2>::hp(g, N)) + ((long long)(q - 1) * N + j), h);
        return __half2float(h) * F16_INV_SCALE;
    }
}
__host__ __device__ constexpr int trio_q(int r, int k) {
    return r == 0 ? (k == 0 ? 1 : (k == 1 ? 7 : 8)) : (r == 1 ? (k == 0 ? 3 : (k == 1 ? 9 : 10)) : (k == 0 ? 5 : (k == 1 ? 11 : 12)));
}
__host__ __device__ constexpr bool trio_ok() {
    int seen = 0;
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) {
            const int q = trio_q(r, k), b = opp(q);
            if ((seen >> q) & 1 || (seen >> b) & 1) return false;
            seen |= (1 << q) | (1 << b);
            if ((k == 0) != (q <= 6)) return false;  // the first pair is the axis pair
        }
    return seen == (1 << Q) - 2 && trio_q(0, 0) == 1 && trio_q(1, 0) == 3 && trio_q(2, 0) == 5;
}
static_assert(trio_ok(), "trio pairs: each moving direction once, axis pair first");
// the value f(q) for the first direction q of pair k of member r (three
// compile-time constants, selected by r)
template <int K, class F> __device__ __forceinline__ int trio_sel(int r, F f) {
    return r == 0 ? f(trio_q(0, K)) : (r == 1 ? f(trio_q(1, K)) : f(trio_q(2, K)));
}
__device__ __forceinline__ float trio_sum(float v, int b3) {
    const float a = __shfl_sync(0xffffffffu, v, b3), b = __shfl_sync(0xffffffffu, v, b3 + 1),
                c = __shfl_sync(0xffffffffu, v, b3 + 2);
    return (a + b) + c;
}
// f_eq(rho_g, u) - w for a direction of weight w with c.u = cu
__device__ __forceinline__ float feq_dev_cu(float w, float cu, float usq, float drg) {
    const float s = 3.0f * cu + 4.5f * cu * cu - 1.5f * usq;
    return w * (drg + s + drg * s);
}

template <int S>
__device__ __forceinline__ void interface_trio(const Dev &d, const VB &vb) {
    using P = Sto<S>;
    const long long N = d.N;
    const unsigned FULL = 0xffffffffu;
    if (vb.x == 0 && threadIdx.x == 0) *d.ztop_rd = -1;
    const int lane = threadIdx.x & 31;
    const bool lane_ok = lane < 30;
    const int g = lane_ok ? lane / 3 : 9;             // trio of the warp
    const int r = lane_ok ? lane - 3 * g : lane - 30;  // member
    const int b3 = 3 * g;
    // pair k: first direction a = trio_q(r, k) with velocity e, second b = opp(a)
    // with -e; sg = +1 when a is the pair member whose leading nonzero
    // component is positive (the collision's split, see collide_store_v).
    // Packed in one word per pair (a, b: 5 bits each; e + 1: 2 bits per
    // component; sg > 0: 1 bit) to keep the loop's registers for the cells.
    uint32_t pk[3];
    const auto pack = [](int q) {
        const bool pos = cx(q) > 0 || (cx(q) == 0 && (cy(q) > 0 || (cy(q) == 0 && cz(q) > 0)));
        return q | (opp(q) << 5) | ((cx(q) + 1) << 10) | ((cy(q) + 1) << 12) | ((cz(q) + 1) << 14) | ((pos ? 1 : 0) << 16);
    };
    pk[0] = (uint32_t)trio_sel<0>(r, pack);
    pk[1] = (uint32_t)trio_sel<1>(r, pack);
    pk[2] = (uint32_t)trio_sel<2>(r, pack);
#define TRIO_QA(k) ((int)(pk[k] & 31u))
#define TRIO_QB(k) ((int)((pk[k] >> 5) & 31u))
#define TRIO_EX(k) ((int)((pk[k] >> 10) & 3u) - 1)
#define TRIO_EY(k) ((int)((pk[k] >> 12) & 3u) - 1)
#define TRIO_EZ(k) ((int)((pk[k] >> 14) & 3u) - 1)
#define TRIO_POS(k) ((pk[k] >> 16) & 1u)
    const float ax = d.a_f[0], ay = d.a_f[1], az = d.a_f[2];
    const uint32_t n = wl_count(d, WL_IFACE);
    const uint32_t wpb = blockDim.x >> 5;
    for (uint32_t w0 = (vb.x * wpb + (threadIdx.x >> 5)) * 10u; w0 < n; w0 += vb.nx * wpb * 10u) {
        const uint32_t it = w0 + (uint32_t)g;
        const bool valid = lane_ok && it < n;
        const long long i = d.list[WL_IFACE][valid ? it : w0];
        const uint32_t i32 = (uint32_t)i;  // the float storages hold N * 19 < 2^32 elements
        const int x = (int)(i32 % (uint32_t)d.nx);
        const uint32_t yz = i32 / (uint32_t)d.nx;
        const int y = (int)(yz % (uint32_t)d.ny), z = (int)(yz / (uint32_t)d.ny);
        // every load of the cell in one round, independent of the neighbour
        // classes: a source beyond a wall reads the cell itself (unused), so
        // no load waits on another and none sits behind a branch
        const float phx = (float)__ldg(d.phisrc + i);
        float foa[3], fob[3], pa[3], pb[3];
        double ha[3], hb[3];
        int sa[3], sb[3], ca[3], cb[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            foa[k] = trio_ld<S>(d.fsrc, TRIO_QA(k), i32, N);
            fob[k] = trio_ld<S>(d.fsrc, TRIO_QB(k), i32, N);
            sa[k] = nbr32(d, x, y, z, -TRIO_EX(k), -TRIO_EY(k), -TRIO_EZ(k));
            sb[k] = nbr32(d, x, y, z, TRIO_EX(k), TRIO_EY(k), TRIO_EZ(k));
            const uint32_t la = sa[k] < 0 ? i32 : (uint32_t)sa[k], lb = sb[k] < 0 ? i32 : (uint32_t)sb[k];
            ca[k] = __ldg(d.flags + la) & CL_MASK;
            cb[k] = __ldg(d.flags + lb) & CL_MASK;
            pa[k] = trio_ld<S>(d.fsrc, TRIO_QA(k), la, N);
            pb[k] = trio_ld<S>(d.fsrc, TRIO_QB(k), lb, N);
            ha[k] = __ldg(d.phisrc + la);
            hb[k] = __ldg(d.phisrc + lb);
        }
        const float fo0 = r == 0 ? P::ld(d.fsrc, 0, i, N) : 0.0f;
        const double m_old = r == 0 ? d.m[i] : 0.0;  // requested with the populations
        // density and the velocity of the last collision (own populations)
        float drx = fo0, j0 = 0.0f, j1 = 0.0f, j2 = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            drx += foa[k] + fob[k];
            const float df = foa[k] - fob[k];
            j0 += (float)TRIO_EX(k) * df;
            j1 += (float)TRIO_EY(k) * df;
            j2 += (float)TRIO_EZ(k) * df;
        }
        drx = trio_sum(drx, b3);
        j0 = trio_sum(j0, b3);
        j1 = trio_sum(j1, b3);
        j2 = trio_sum(j2, b3);
        const float rx = 1.0f + drx;
        const float irx = __frcp_rn(rx);
        const float ux = j0 * irx - ax, uy = j1 * irx - ay, uz = j2 * irx - az;
        // the arriving populations: pull, Eq. noslip from an obstacle or a
        // wall, gas sources reconstructed below; the mass exchange of the link
        // back to a liquid or interface source; the fill level seen there
        float fpa[3], fpb[3], dm = 0.0f, fsa = phx, fsb = phx;
        unsigned solid = 0, gas = 0, seen_lg = 0;  // per direction slot 2k (a), 2k + 1 (b)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int q = s ? TRIO_QB(k) : TRIO_QA(k);
                const int si = s ? sb[k] : sa[k];
                const int ns = si < 0 ? CL_WALL : (s ? cb[k] : ca[k]);
                const float pq = s ? pb[k] : pa[k];
                const float phy = (float)(s ? hb[k] : ha[k]);
                const float fbar = s ? foa[k] : fob[k];  // own population of the opposite direction
                const unsigned bit = 1u << (2 * k + s);
                const bool sol = ns == CL_WALL || ns == CL_O, gs = ns == CL_G, lq = ns == CL_L;
                // selects rather than branches: the lanes of a warp meet every
                // class, and branches would run one after another; only the
                // moving-solid term (rare) is behind a branch
                float cuw = 0.0f;
                if (ns == CL_O || (sol && d.walls_move))
                    cuw = ns == CL_O ? link_cuw_f(d, d.bodies[d.bid[si]], x, y, z, q) : (float)wall_cuw(d, x, y, z, q);
                seen_lg |= lq ? 1u : (gs ? 2u : 0u);
                solid |= sol ? bit : 0u;
                gas |= gs ? bit : 0u;
                const float fv = sol ? fbar + 6.0f * (k == 0 ? wf(1) : wf(7)) * cuw * rx : (gs ? 0.0f : pq);
                const float wgt = lq ? 1.0f : 0.5f * (phx + phy);
                dm += (sol || gs) ? 0.0f : wgt * (pq - fbar);
                const float seen = sol ? phx : (gs ? 0.0f : (lq ? 1.0f : phy));
                if (s) fpb[k] = fv;
                else fpa[k] = fv;
                if (k == 0) {
                    if (s) fsb = seen;
                    else fsa = seen;
                }
            }
        }
        // normal n = -grad(phi): component r from the member's axis pair
        // (W/E pull from x + e_x / x - e_x, N/S from x - e_y / x + e_y, T/B
        // from x - e_z / x + e_z)
        const float nvr = r == 0 ? 0.5f * (fsb - fsa) : 0.5f * (fsa - fsb);
        const float nv0 = __shfl_sync(FULL, nvr, b3), nv1 = __shfl_sync(FULL, nvr, b3 + 1),
                    nv2 = __shfl_sync(FULL, nvr, b3 + 2);
        float drg = d.drg_f;
        if (d.sigma != 0.0) {
            // gas density raised by the Laplace pressure (curvature by member 0)
            const float len = sqrtf((nv0 * nv0 + nv1 * nv1) + nv2 * nv2);
            const float nu0 = len > 0.0f ? nv0 / len : 0.0f, nu1 = len > 0.0f ? nv1 / len : 0.0f,
                        nu2 = len > 0.0f ? nv2 / len : 0.0f;
            float kap = 0.0f;
            if (r == 0) kap = curvature_f(d, x, y, z, nu0, nu1, nu2);
            kap = __shfl_sync(FULL, kap, b3);
            drg = d.drg_f + (6.0f * d.sigma_f) * kap;
        }
        // Eq. reconstruct for gas-sourced directions and every non-solid
        // direction with c.n below the dead band
        const float usq = ux * ux + uy * uy + uz * uz;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float cn = (float)TRIO_EX(k) * nv0 + (float)TRIO_EY(k) * nv1 + (float)TRIO_EZ(k) * nv2;  // c_a . n
            const float cu = (float)TRIO_EX(k) * ux + (float)TRIO_EY(k) * uy + (float)TRIO_EZ(k) * uz;
            const float w = k == 0 ? wf(1) : wf(7);
            const float fe = feq_dev_cu(w, cu, usq, drg) + feq_dev_cu(w, -cu, usq, drg);
            const unsigned ba = 1u << (2 * k), bb = 2u << (2 * k);
            if ((gas & ba) || (cn < -d.deadband_f && !(solid & ba))) fpa[k] = fe - fob[k];
            if ((gas & bb) || (-cn < -d.deadband_f && !(solid & bb))) fpb[k] = fe - foa[k];
        }
        dm = trio_sum(dm, b3);
        // BGK + Luo force on the deviations (the pair split of collide_store_v)
        const float fp0 = r == 0 ? fo0 : 0.0f;
        float dr = fp0, k0 = 0.0f, k1 = 0.0f, k2 = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            dr += fpa[k] + fpb[k];
            const float df = fpa[k] - fpb[k];
            k0 += (float)TRIO_EX(k) * df;
            k1 += (float)TRIO_EY(k) * df;
            k2 += (float)TRIO_EZ(k) * df;
        }
        dr = trio_sum(dr, b3);
        k0 = trio_sum(k0, b3);
        k1 = trio_sum(k1, b3);
        k2 = trio_sum(k2, b3);
        const float rho = 1.0f + dr;
        const float inv = __frcp_rn(rho);
        const float vx = k0 * inv, vy = k1 * inv, vz = k2 * inv;
        const float nusq15 = (vx * vx + vy * vy + vz * vz) * -1.5f;
        const float nua3 = (vx * ax + vy * ay + vz * az) * -3.0f;
        const float om = d.omega_f, om1 = 1.0f - om;
        void *gdst = d.fdst;
        float rest = 0.0f, drs = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float w = k == 0 ? wf(1) : wf(7);
            const float wdr = dr * w, wr = rho * w, wr3 = wr * 3.0f;
            // p = the member with the positive leading component, m the other
            const float sgk = TRIO_POS(k) ? 1.0f : -1.0f;
            const float cpx = sgk * (float)TRIO_EX(k), cpy = sgk * (float)TRIO_EY(k), cpz = sgk * (float)TRIO_EZ(k);
            const float cu = cpx * vx + cpy * vy + cpz * vz;
            const float ca = cpx * ax + cpy * ay + cpz * az;
            const float A = fmaf(wr, fmaf(cu * cu, 4.5f, nusq15), wdr);
            const float C = wr * fmaf(cu, 9.0f * ca, nua3);
            const float E = fmaf(A, om, C);
            const float G = fmaf(wr3 * cu, om, wr3 * ca);
            const bool a_is_p = TRIO_POS(k) != 0;
            const float fp_p = a_is_p ? fpa[k] : fpb[k], fp_m = a_is_p ? fpb[k] : fpa[k];
            const float dnp = fmaf(fp_p, om1, E + G), dnm = fmaf(fp_m, om1, E - G);
            const int qp = a_is_p ? TRIO_QA(k) : TRIO_QB(k), qm = a_is_p ? TRIO_QB(k) : TRIO_QA(k);
            float stp = dnp, stm = dnm;
            if (valid) {
                stp = trio_st<S>(gdst, qp, i32, N, dnp);
                stm = trio_st<S>(gdst, qm, i32, N, dnm);
            }
            rest += (fp_p - stp) + (fp_m - stm);
            drs += stp + stm;
        }
        rest = trio_sum(rest, b3);
        if (r == 0) {
            const float st0 = fp0 + rest;
            if (valid) P::st_one(gdst, 0, i, N, st0);
            drs += st0;
        }
        drs = trio_sum(drs, b3);
        const unsigned lg = __shfl_sync(FULL, seen_lg, b3) | __shfl_sync(FULL, seen_lg, b3 + 1) |
                            __shfl_sync(FULL, seen_lg, b3 + 2);
        const bool has_l = lg & 1u, has_g = lg & 2u;
        uint8_t mk = 0;
        if (valid && r == 0) {
            const double m_new = m_old + (double)dm;
            const double phin = m_new / (1.0 + (double)drs);
            d.m[i] = m_new;
            d.phidst[i] = phin;
            if (!(rho > 0.0f) || !(rho < 1e30f)) atomicOr(d.status, ST_NONFINITE);
            mk = phin >= 1.0 + d.eps ? MK_FILLED : (phin <= -d.eps ? MK_EMPTIED : 0);
            // an interface cell without a liquid neighbour empties, one without
            // a gas neighbour fills
            if (!mk && d.nb_rule) mk = (!has_l && has_g) ? MK_EMPTIED : ((!has_g && has_l) ? MK_FILLED : 0);
            if (mk) d.cmark[i] = mk;
        }
        wl_append(d, mk == MK_FILLED, WL_FILLED, (uint32_t)i);
        wl_append(d, mk == MK_EMPTIED, WL_EMPTIED, (uint32_t)i);
    }
}
#undef TRIO_QA
#undef TRIO_QB
#undef TRIO_EX
#undef TRIO_EY
#undef TRIO_EZ
#undef TRIO_POS

// ---- C1 + C2 for interface cells (Sec. 2.2): reconstruction, mass exchange.
// Double storage: one thread per cell, every sum in the order of the oracle.
__device__ __forceinline__ void interface_d(const Dev &d, const VB &vb) {
    using P = Sto<0>;
    const long long N = d.N;
    // the bulk kernel has read this step's fluid top: clear the slot for the
    // next step to record into
    if (vb.x == 0 && threadIdx.x == 0) *d.ztop_rd = -1;
    uint32_t n = wl_count(d, WL_IFACE);
    for (uint32_t it = vb.x * blockDim.x + threadIdx.x; it < n; it += vb.nx * blockDim.x) {
        long long i = d.list[WL_IFACE][it];
        int x, y, z;
        coords(d, i, x, y, z);
        double own_phi = d.phisrc[i];
        long long src[Q];
        int scl[Q];
        bool has_l = false, has_g = false;  // any liquid / gas among the 18 neighbours
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            src[q] = nbr(d, x, y, z, -cx(q), -cy(q), -cz(q));
            scl[q] = cls(d, src[q]);
            has_l = has_l || scl[q] == CL_L;
            has_g = has_g || scl[q] == CL_G;
        }
        // normal n = -grad(phi), central differences
        double nv[3];
        {
            double pm = fill_seen(d, nbr(d, x, y, z, -1, 0, 0), own_phi);
            double pp = fill_seen(d, nbr(d, x, y, z, 1, 0, 0), own_phi);
            nv[0] = 0.5 * (pm - pp);
            pm = fill_seen(d, nbr(d, x, y, z, 0, -1, 0), own_phi);
            pp = fill_seen(d, nbr(d, x, y, z, 0, 1, 0), own_phi);
            nv[1] = 0.5 * (pm - pp);
            pm = fill_seen(d, nbr(d, x, y, z, 0, 0, -1), own_phi);
            pp = fill_seen(d, nbr(d, x, y, z, 0, 0, 1), own_phi);
            nv[2] = 0.5 * (pm - pp);
        }
        double fo[Q], fp[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) fo[q] = P::ld(d.fsrc, q, i, N);
        double rho_x = 0.0;
#pragma unroll
        for (int q = 0; q < Q; ++q) rho_x += fo[q];
        double j0 = 0.0, j1 = 0.0, j2 = 0.0;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            j0 += cx(q) * fo[q];
            j1 += cy(q) * fo[q];
            j2 += cz(q) * fo[q];
        }
        double ux[3] = {j0 / rho_x - d.a[0], j1 / rho_x - d.a[1], j2 / rho_x - d.a[2]};
        // gas density of the boundary condition, raised by the Laplace pressure
        double rg = d.rho_g;
        if (d.sigma != 0.0) {
            double nc[3];
            unit_vec_d(nv, nc);
            rg = d.rho_g + (6.0 * d.sigma) * curvature_d(d, x, y, z, nc[0], nc[1], nc[2]);
        }
        fp[0] = fo[0];
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            int qb = opp(q);
            if (scl[q] == CL_WALL || scl[q] == CL_O) {
                double cuw = scl[q] == CL_O ? link_cuw(d, d.bodies[d.bid[src[q]]], x, y, z, q)
                                            : (d.walls_move ? wall_cuw(d, x, y, z, q) : 0.0);
                fp[q] = fo[qb] + ((6.0 * wd(q)) * rho_x) * cuw;
            } else if (scl[q] == CL_G) {
                fp[q] = (feq_d(q, rg, ux) + feq_d(qb, rg, ux)) - fo[qb];
            } else {
                fp[q] = P::ld(d.fsrc, q, src[q], N);
            }
        }
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            double cn = (cx(q) * nv[0] + cy(q) * nv[1]) + cz(q) * nv[2];
            if (cn < -d.deadband && scl[q] != CL_O && scl[q] != CL_WALL) {
                int qb = opp(q);
                fp[q] = (feq_d(q, rg, ux) + feq_d(qb, rg, ux)) - fo[qb];
            }
        }
        double dm = 0.0;
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            int qb = opp(q);
            long long yi = nbr(d, x, y, z, cx(q), cy(q), cz(q));
            int yc = cls(d, yi);
            if (yc == CL_L) {
                dm += P::ld(d.fsrc, qb, yi, N) - fo[q];
            } else if (yc == CL_I) {
                double wgt = 0.5 * (own_phi + d.phisrc[yi]);
                dm += wgt * (P::ld(d.fsrc, qb, yi, N) - fo[q]);
            }
        }
        const double m_new = d.m[i] + dm;
        double fn[Q];
        collide_d(d, fp, fn);
        double r = 0.0;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            P::st(d.fdst, q, i, N, fn[q]);
            r += fn[q];
        }
        double phin = m_new / r;
        d.m[i] = m_new;
        d.phidst[i] = phin;
        if (!(r == r) || r <= 0.0) atomicOr(d.status, ST_NONFINITE);
        uint8_t mk = phin >= 1.0 + d.eps ? MK_FILLED : (phin <= -d.eps ? MK_EMPTIED : 0);
        // an interface cell without a liquid neighbour empties, one without
        // a gas neighbour fills
        if (!mk && d.nb_rule) mk = (!has_l && has_g) ? MK_EMPTIED : ((!has_g && has_l) ? MK_FILLED : 0);
        if (mk) d.cmark[i] = mk;
        wl_append(d, mk == MK_FILLED, WL_FILLED, (uint32_t)i);
        wl_append(d, mk == MK_EMPTIED, WL_EMPTIED, (uint32_t)i);
    }
}
template <int S> __device__ __forceinline__ void interface_body(const Dev &d, const VB &vb) {
    if constexpr (S == 0) interface_d(d, vb);
    else interface_trio<S>(d, vb);
}
template <int S>
__global__ void __launch_bounds__(128, LBMFS_IFACE_MINB) k_interface(const __grid_constant__ Dev d) {
    interface_body<S>(d, vb_own());
}

// ------------------------------------------------- C3: conversions (Sec. 2.2)

// filled cells: emptied neighbours are kept; gas neighbours become interface
// set mark `bit` on the neighbours of (x, y, z) in the direction mask m (the
// atomics issued together) and append the cells whose bit was newly set to
// worklist `list` (one reservation for all of them)
__device__ __forceinline__ void mark_append(const Dev &d, int x, int y, int z, unsigned m, uint8_t bit, int list) {
    if (!m) return;
    unsigned nw = 0;
#pragma unroll
    for (int q = 1; q < Q; ++q)
        if (m & (1u << q)) {
            const uint8_t old = mark_or(d, nbr(d, x, y, z, cx(q), cy(q), cz(q)), bit);
            if (!(old & bit)) nw |= 1u << q;
        }
    if (!nw) return;
    uint32_t pos = atomicAdd(&d.cnt[list], (uint32_t)__popc(nw));
#pragma unroll
    for (int q = 1; q < Q; ++q)
        if (nw & (1u << q)) {
            if (pos < d.cap) d.list[list][pos] = (uint32_t)nbr(d, x, y, z, cx(q), cy(q), cz(q));
            else atomicOr(d.status, ST_OVERFLOW);
            ++pos;
        }
}

__device__ __forceinline__ void conv_filled_body(const Dev &d, const VB &vb) {
    LIST_LOOP(WL_FILLED, a) {
        long long i = d.list[WL_FILLED][it_a];
        int x, y, z;
        coords(d, i, x, y, z);
        // classes and emptied marks requested at once (this kernel sets no
        // emptied mark and changes no class)
        unsigned em = 0, gm = 0;
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            long long yi = nbr(d, x, y, z, cx(q), cy(q), cz(q));
            if (yi < 0) continue;
            if (d.cmark[yi] & MK_EMPTIED) em |= 1u << q;
            if (clsv(d, yi) == CL_G) gm |= 1u << q;
        }
#pragma unroll
        for (int q = 1; q < Q; ++q)
            if (em & (1u << q)) mark_and(d, nbr(d, x, y, z, cx(q), cy(q), cz(q)), MK_EMPTIED);
        mark_append(d, x, y, z, gm, MK_NEWG, WL_NEWG);
    }
}
__global__ void k_conv_filled(const __grid_constant__ Dev d) { conv_filled_body(d, vb_own()); }

// still-emptied cells: liquid neighbours become interface
__device__ __forceinline__ void conv_emptied_body(const Dev &d, const VB &vb) {
    LIST_LOOP(WL_EMPTIED, a) {
        long long i = d.list[WL_EMPTIED][it_a];
        if (!(d.cmark[i] & MK_EMPTIED)) continue;
        int x, y, z;
        coords(d, i, x, y, z);
        // classes requested at once (this kernel changes marks only)
        unsigned lm = 0;
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            long long yi = nbr(d, x, y, z, cx(q), cy(q), cz(q));
            if (yi >= 0 && clsv(d, yi) == CL_L) lm |= 1u << q;
        }
        mark_append(d, x, y, z, lm, MK_NEWL, WL_NEWL);
    }
}
__global__ void k_conv_emptied(const __grid_constant__ Dev d) { conv_emptied_body(d, vb_own()); }

// new interface cells: from gas f = f_eq(mean rho, mean u) of the liquid and
// interface neighbours, m = 0; from liquid m = rho
template <int S>
__device__ __forceinline__ void conv_init_body(const Dev &d, const VB &vb) {
    {
        // one warp per new cell: lane q reads neighbour q (all neighbours'
        // populations in flight together), the sums are taken in q order
        // from the gathered values, lane q evaluates f_eq,q
        const int lane = threadIdx.x & 31;
        const unsigned wpb = blockDim.x >> 5;
        const uint32_t n = wl_count(d, WL_NEWG);
        for (uint32_t w = vb.x * wpb + (threadIdx.x >> 5); w < n; w += vb.nx * wpb) {
            const long long i = d.list[WL_NEWG][w];
            int x, y, z;
            coords(d, i, x, y, z);
            if (lane == 0 && z > *d.ztop_wr + ZTOP_MARGIN) atomicOr(d.status, ST_TOP);
            double r = 0.0, u[3] = {0.0, 0.0, 0.0};
            int fluid = 0;
            if (lane >= 1 && lane < Q) {
                const long long zi = nbr(d, x, y, z, cx(lane), cy(lane), cz(lane));
                const int zc = cls(d, zi);
                if (zc == CL_L || zc == CL_I) {
                    fluid = 1;
                    r = cell_rho_u<S>(d, d.fdst, zi, u);
                }
            }
            double sr = 0.0, su[3] = {0.0, 0.0, 0.0};
            int cnt = 0;
#pragma unroll
            for (int q = 1; q < Q; ++q) {
                const int fq = __shfl_sync(0xffffffffu, fluid, q);
                const double rq = __shfl_sync(0xffffffffu, r, q), u0 = __shfl_sync(0xffffffffu, u[0], q),
                             u1 = __shfl_sync(0xffffffffu, u[1], q), u2 = __shfl_sync(0xffffffffu, u[2], q);
                if (!fq) continue;
                sr += rq;
                su[0] += u0;
                su[1] += u1;
                su[2] += u2;
                cnt++;
            }
            const double rm = sr / cnt;
            const double um[3] = {su[0] / cnt, su[1] / cnt, su[2] / cnt};
            const double fl = feq_d(lane < Q ? lane : 0, rm, um);
            double f[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) f[q] = __shfl_sync(0xffffffffu, fl, q);
            if (lane == 0) {
                Sto<S>::st_cell(d.fdst, i, d.N, f);
                d.m[i] = 0.0;
            }
        }
    }
    {
        LIST_LOOP(WL_NEWL, b) {
            long long i = d.list[WL_NEWL][it_b];
            d.m[i] = cell_density<S>(d, d.fdst, i);
        }
    }
}
template <int S>
__global__ void k_conv_init(const __grid_constant__ Dev d) { conv_init_body<S>(d, vb_own()); }

__device__ __forceinline__ void conv_flags_body(const Dev &d, const VB &vb) {
    {
        LIST_LOOP(WL_FILLED, a) set_cls(d, d.list[WL_FILLED][it_a], CL_L);
    }
    {
        LIST_LOOP(WL_EMPTIED, b) {
            long long i = d.list[WL_EMPTIED][it_b];
            if (d.cmark[i] & MK_EMPTIED) set_cls(d, i, CL_G);
        }
    }
    {
        LIST_LOOP(WL_NEWG, c) set_cls(d, d.list[WL_NEWG][it_c], CL_I);
    }
    {
        LIST_LOOP(WL_NEWL, e) set_cls(d, d.list[WL_NEWL][it_e], CL_I);
    }
}
__global__ void k_conv_flags(const __grid_constant__ Dev d) { conv_flags_body(d, vb_own()); }

template <int S>
__device__ __forceinline__ double excess(const Dev &d, long long i, uint8_t mk);

// interface neighbours of converted cells receive excess mass.  The
// converted cell's share e(x) / k(x) is computed here, once, and kept in its
// mass entry (a converted cell is liquid or gas now, so the entry is not read
// as a mass again before the cell next becomes interface, which sets it); a
// cell without interface neighbours keeps its mass for the lost-mass ledger
template <int S>
__device__ __forceinline__ void claim_receivers(const Dev &d, long long i, uint8_t mk) {
    int x, y, z;
    coords(d, i, x, y, z);
    // classes requested at once (this kernel changes marks and the converted
    // cell's own mass entry only)
    unsigned im = 0;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        long long yi = nbr(d, x, y, z, cx(q), cy(q), cz(q));
        if (yi >= 0 && clsv(d, yi) == CL_I) im |= 1u << q;
    }
    const int k = __popc(im);
    if (k > 0) d.m[i] = excess<S>(d, i, mk) / k;
    mark_append(d, x, y, z, im, MK_RECV, WL_RECV);
}

template <int S>
__device__ __forceinline__ void conv_claim_body(const Dev &d, const VB &vb) {
    {
        LIST_LOOP(WL_FILLED, a) claim_receivers<S>(d, d.list[WL_FILLED][it_a], MK_FILLED);
    }
    {
        LIST_LOOP(WL_EMPTIED, b) {
            long long i = d.list[WL_EMPTIED][it_b];
            const uint8_t mk = d.cmark[i];
            if (mk & MK_EMPTIED) claim_receivers<S>(d, i, mk);
        }
    }
}
template <int S>
__global__ void k_conv_claim(const __grid_constant__ Dev d) { conv_claim_body<S>(d, vb_own()); }

// k(x): interface neighbours of a converted cell (classes after conversion)
__device__ __forceinline__ int iface_neighbours(const Dev &d, long long i) {
    int x, y, z;
    coords(d, i, x, y, z);
    int k = 0;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        long long yi = nbr(d, x, y, z, cx(q), cy(q), cz(q));
        if (yi >= 0 && clsv(d, yi) == CL_I) k++;
    }
    return k;
}

template <int S>
__device__ __forceinline__ double excess(const Dev &d, long long i, uint8_t mk) {
    return (mk & MK_FILLED) ? d.m[i] - cell_density<S>(d, d.fdst, i) : d.m[i];
}

// receivers gather e(x) / k(x) over their converted neighbours in q order
template <int S>
__device__ __forceinline__ void conv_excess_body(const Dev &d, const VB &vb) {
    LIST_LOOP(WL_RECV, a) {
        long long i = d.list[WL_RECV][it_a];
        int x, y, z;
        coords(d, i, x, y, z);
        // the neighbours' marks, then the converted ones' shares e(y) / k(y)
        // (computed when the receivers were claimed), summed in q order
        unsigned cm = 0;
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            long long yi = nbr(d, x, y, z, cx(q), cy(q), cz(q));
            if (yi >= 0 && (d.cmark[yi] & (MK_FILLED | MK_EMPTIED))) cm |= 1u << q;
        }
        double sh[Q];
#pragma unroll
        for (int q = 1; q < Q; ++q) sh[q] = (cm & (1u << q)) ? d.m[nbr(d, x, y, z, cx(q), cy(q), cz(q))] : 0.0;
        double acc = 0.0;
#pragma unroll
        for (int q = 1; q < Q; ++q)
            if (cm & (1u << q)) acc += sh[q];
        double m = d.m[i] + acc;
        d.m[i] = m;
        d.phidst[i] = m / cell_density<S>(d, d.fdst, i);
    }
}
template <int S>
__global__ void k_conv_excess(const __grid_constant__ Dev d) { conv_excess_body<S>(d, vb_own()); }

// mass that found no interface neighbour goes to the ledger; marks are cleared
template <int S>
__device__ __forceinline__ void conv_finish_body(const Dev &d, const VB &vb) {
    {
        LIST_LOOP(WL_FILLED, a) {
            long long i = d.list[WL_FILLED][it_a];
            if (iface_neighbours(d, i) == 0) atomicAdd(&d.ledger[LG_LOST], excess<S>(d, i, MK_FILLED));
            d.cmark[i] = 0;
        }
    }
    {
        LIST_LOOP(WL_EMPTIED, b) {
            long long i = d.list[WL_EMPTIED][it_b];
            uint8_t mk = d.cmark[i];
            if ((mk & MK_EMPTIED) && iface_neighbours(d, i) == 0) atomicAdd(&d.ledger[LG_LOST], excess<S>(d, i, mk));
            d.cmark[i] = 0;
        }
    }
    {
        LIST_LOOP(WL_NEWG, c) d.cmark[d.list[WL_NEWG][it_c]] = 0;
    }
    {
        LIST_LOOP(WL_NEWL, e) d.cmark[d.list[WL_NEWL][it_e]] = 0;
    }
    {
        LIST_LOOP(WL_RECV, g) d.cmark[d.list[WL_RECV][it_g]] = 0;
    }
}
template <int S>
__global__ void k_conv_finish(const __grid_constant__ Dev d) { conv_finish_body<S>(d, vb_own()); }

// ----------------------------------------------- C5: rigid-body update
// (the role the paper gives the pe engine, Sec. 2.3: the body moves under the
// hydrodynamic force and torque and gravity; the paper does not give the
// integrator, this one is a virtual-mass explicit update)

// one warp per body: fixed-order sum of the force partials, then the update
__device__ __forceinline__ void body_step(const Dev &d, Body &b, const double *acc);
__device__ __forceinline__ void bodies_body(const Dev &d, const VB &vb) {
    int bi = vb.x;
    int lane = threadIdx.x;
    double acc[7];
    if (d.part128) {
        // double storage: exact 128-bit partials (fixed96), summed exactly
        const unsigned long long *pp = reinterpret_cast<const unsigned long long *>(d.part);
#pragma unroll 1
        for (int c = 0; c < 7; ++c) {
            unsigned __int128 v = 0;
            for (int k = lane; k < FORCE_BLOCKS; k += 32) {
                const long long j = 2 * (((long long)bi * FORCE_BLOCKS + k) * 7 + c);
                v += ((unsigned __int128)pp[j + 1] << 64) | (unsigned __int128)pp[j];
            }
            for (int off = 16; off > 0; off >>= 1) v += shfl_down_128(v, off);
            acc[c] = fixed96_value(v);
        }
    } else {
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            double v = 0.0;
            for (int k = lane; k < FORCE_BLOCKS; k += 32) v += d.part[((long long)bi * FORCE_BLOCKS + k) * 7 + c];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            acc[c] = v;
        }
    }
    if (lane != 0) return;
    // the body record is read once into registers, updated, and written back
    // (instead of a chain of dependent global-memory reads and writes)
    Body b = d.bodies[bi];
    body_step(d, b, acc);
    d.bodies[bi] = b;
}

__device__ __forceinline__ void body_step(const Dev &d, Body &b, const double *acc) {
    for (int k = 0; k < 3; ++k) {
        b.F[k] = acc[k];
        b.T[k] = acc[3 + k];
    }
    b.S = acc[6];
    for (int k = 0; k < 3; ++k) {
        b.plo[k] = b.lo[k];
        b.phi[k] = b.hi[k];
    }
    int base = b.mode & 0xff;
    if (base == 0) {
        for (int k = 0; k < 3; ++k) b.v[k] = b.w[k] = b.dv[k] = b.dw[k] = 0.0;
        return;
    }
    // the update is driven by the mean of this step's and the previous step's
    // force and torque (the force alone on the first step; the force alone
    // throughout when the two-step mean is switched off): near tau = 1/2 a
    // force that flips sign every step would feed the barely damped BGK modes
    // of that period through the wall velocity
    double Fh[3], Th[3];
    const bool mean = d.force_mean && b.nF;
    for (int k = 0; k < 3; ++k) {
        Fh[k] = mean ? 0.5 * (b.F[k] + b.Fp[k]) : b.F[k];
        Th[k] = mean ? 0.5 * (b.T[k] + b.Tp[k]) : b.T[k];
        b.Fp[k] = b.F[k];
        b.Tp[k] = b.T[k];
    }
    b.nF = 1;
    double vol, mass, I[3];
    if (b.shape == 1) {  // sphere: V = 4/3 pi r^3, I = 2/5 m r^2
        vol = 4.1887902047863905 * ((b.h[0] * b.h[0]) * b.h[0]);
        mass = b.dens * vol;
        I[0] = I[1] = I[2] = (0.4 * mass) * (b.h[0] * b.h[0]);
    } else {
        vol = ((8.0 * b.h[0]) * b.h[1]) * b.h[2];
        mass = b.dens * vol;
        I[0] = (mass / 3.0) * (b.h[1] * b.h[1] + b.h[2] * b.h[2]);
        I[1] = (mass / 3.0) * (b.h[0] * b.h[0] + b.h[2] * b.h[2]);
        I[2] = (mass / 3.0) * (b.h[0] * b.h[0] + b.h[1] * b.h[1]);
    }
    double If[3] = {I[0] / b.dens, I[1] / b.dens, I[2] / b.dens};
    const double C = d.vmass;  // virtual-mass coefficient (Schwarz, Kempe and Froehlich 2015)
    double den = mass + C * vol;
    for (int k = 0; k < 3; ++k) {
        double num = (Fh[k] + mass * d.grav[k]) + C * (vol * b.dv[k]);
        b.dv[k] = num / den;
        b.v[k] = b.v[k] + b.dv[k];
    }
    if (b.mode & 0x100)
        for (int k = 0; k < 3; ++k) b.v[k] = b.v[k] * (1.0 - b.damp);
    double R[9];
    rotation(b.q, R);
    if (base == 2) {
        const double *ax = b.axis;
        double ta = (Th[0] * ax[0] + Th[1] * ax[1]) + Th[2] * ax[2];
        double ab[3];
        for (int k = 0; k < 3; ++k) ab[k] = (R[0 * 3 + k] * ax[0] + R[1 * 3 + k] * ax[1]) + R[2 * 3 + k] * ax[2];
        double Ia = (ab[0] * ab[0] * I[0] + ab[1] * ab[1] * I[1]) + ab[2] * ab[2] * I[2];
        double Ifa = Ia / b.dens;
        double ws = (b.w[0] * ax[0] + b.w[1] * ax[1]) + b.w[2] * ax[2];
        b.dw[0] = (ta + C * (Ifa * b.dw[0])) / (Ia + C * Ifa);
        ws = ws + b.dw[0];
        for (int k = 0; k < 3; ++k) b.w[k] = ws * ax[k];
    } else {
        double wb[3], tb[3], L[3], gy[3];
        for (int k = 0; k < 3; ++k) {
            wb[k] = (R[0 * 3 + k] * b.w[0] + R[1 * 3 + k] * b.w[1]) + R[2 * 3 + k] * b.w[2];
            tb[k] = (R[0 * 3 + k] * Th[0] + R[1 * 3 + k] * Th[1]) + R[2 * 3 + k] * Th[2];
            L[k] = I[k] * wb[k];
        }
        gy[0] = wb[1] * L[2] - wb[2] * L[1];
        gy[1] = wb[2] * L[0] - wb[0] * L[2];
        gy[2] = wb[0] * L[1] - wb[1] * L[0];
        for (int k = 0; k < 3; ++k) {
            b.dw[k] = ((tb[k] - gy[k]) + C * (If[k] * b.dw[k])) / (I[k] + C * If[k]);
            wb[k] = wb[k] + b.dw[k];
        }
        for (int k = 0; k < 3; ++k) b.w[k] = (R[k * 3 + 0] * wb[0] + R[k * 3 + 1] * wb[1]) + R[k * 3 + 2] * wb[2];
    }
    double nn[3] = {(double)d.nx, (double)d.ny, (double)d.nz};
    for (int k = 0; k < 3; ++k) {
        b.o[k] = b.o[k] + b.v[k];
        if (d.periodic & (1u << k)) {
            if (b.o[k] >= nn[k]) b.o[k] = b.o[k] - nn[k];
            else if (b.o[k] < 0.0) b.o[k] = b.o[k] + nn[k];
        }
    }
    double qw = b.q[0], qx = b.q[1], qy = b.q[2], qz = b.q[3];
    const double *w = b.w;
    double dw = -((w[0] * qx + w[1] * qy) + w[2] * qz);
    double dx = qw * w[0] + (w[1] * qz - w[2] * qy);
    double dy = qw * w[1] + (w[2] * qx - w[0] * qz);
    double dz = qw * w[2] + (w[0] * qy - w[1] * qx);
    double nq[4] = {qw + 0.5 * dw, qx + 0.5 * dx, qy + 0.5 * dy, qz + 0.5 * dz};
    double norm = sqrt(((nq[0] * nq[0] + nq[1] * nq[1]) + nq[2] * nq[2]) + nq[3] * nq[3]);
    for (int k = 0; k < 4; ++k) b.q[k] = nq[k] / norm;
    body_bounds(d, b);
    // a moving box that reaches a wall plane would need a contact model
    // (the paper's rigid-body engine); report it instead of running on
    for (int k = 0; k < 3; ++k) {
        if (d.periodic & (1u << k)) continue;
        const double e = b.shape == 1 ? b.h[0]
                                      : (fabs(b.R[k * 3 + 0]) * b.h[0] + fabs(b.R[k * 3 + 1]) * b.h[1]) +
                                            fabs(b.R[k * 3 + 2]) * b.h[2];
        const double n = k == 0 ? d.nx : (k == 1 ? d.ny : d.nz);
        if (b.o[k] - e < 0.0 || b.o[k] + e > n) atomicOr(d.status, ST_CONTACT);
    }
}
__global__ void k_bodies(const __grid_constant__ Dev d) { bodies_body(d, vb_own()); }

// ----------------------------------------------- C6: remap (Sec. 2.3, 2.4)

// cells inside body vb.y at its new pose become obstacle
template <int S>
__device__ __forceinline__ void remap_cover_body(const Dev &d, const VB &vb) {
    int bi = vb.y;
    const Body &b = d.bodies[bi];
    long long n = range_count(b.lo, b.hi);
    for (long long k = vb.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)vb.nx * blockDim.x) {
        int x, y, z;
        range_cell(d, b.lo, b.hi, k, x, y, z);
        long long i = x + (long long)d.nx * (y + (long long)d.ny * z);
        int c = clsv(d, i);
        bool cover = c != CL_O && inside(d, b, x, y, z);
        wl_append(d, cover, WL_COVER, (uint32_t)i);
        if (!cover) continue;
        double mass = c == CL_L ? cell_density<S>(d, d.fdst, i) : (c == CL_I ? d.m[i] : 0.0);
        if (mass != 0.0) atomicAdd(&d.ledger[LG_COVERED], mass);
        set_cls(d, i, CL_O);
        d.bid[i] = (uint8_t)bi;
    }
}
template <int S>
__global__ void k_remap_cover(const __grid_constant__ Dev d) { remap_cover_body<S>(d, vb_own()); }

// obstacle cells of body vb.y outside its new pose are pending
__device__ __forceinline__ void remap_pending_body(const Dev &d, const VB &vb) {
    int bi = vb.y;
    const Body &b = d.bodies[bi];
    long long n = range_count(b.plo, b.phi);
    for (long long k = vb.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)vb.nx * blockDim.x) {
        int x, y, z;
        range_cell(d, b.plo, b.phi, k, x, y, z);
        long long i = x + (long long)d.nx * (y + (long long)d.ny * z);
        bool pend = clsv(d, i) == CL_O && d.bid[i] == bi && !inside(d, b, x, y, z);
        if (pend) d.cmark[i] = MK_PEND;
        wl_append(d, pend, WL_PEND, (uint32_t)i);
    }
}
__global__ void k_remap_pending(const __grid_constant__ Dev d) { remap_pending_body(d, vb_own()); }

// Jacobi passes of the obstacle-to-fluid rule over the pending cells, closure,
// uncovered-mass ledger (one block)
template <int S>
__device__ __forceinline__ void remap_resolve_body(const Dev &d, const VB &vb) {
    uint32_t n = wl_count(d, WL_PEND);
    if (n == 0) return;
    __shared__ int s_any;
    for (int pass = 0; pass < 4; ++pass) {
        for (uint32_t it = threadIdx.x; it < n; it += blockDim.x) {
            long long i = d.list[WL_PEND][it];
            d.rdec[it] = 0;
            if (!(d.cmark[i] & MK_PEND)) continue;
            int x, y, z;
            coords(d, i, x, y, z);
            int nL = 0, nI = 0, nG = 0;
            double sr = 0.0, sp = 0.0;
            // marks and classes requested at once, then the neighbours in q order
            uint8_t cs[Q];
#pragma unroll
            for (int q = 1; q < Q; ++q) {
                long long yi = nbr(d, x, y, z, cx(q), cy(q), cz(q));
                cs[q] = (yi < 0 || (d.cmark[yi] & MK_PEND)) ? (uint8_t)0 : (uint8_t)clsv(d, yi);
            }
#pragma unroll 1
            for (int q = 1; q < Q; ++q) {
                const int c = cs[q];
                if (c == 0 || c == CL_O) continue;
                long long yi = nbr(d, x, y, z, cx(q), cy(q), cz(q));
                if (c == CL_L) {
                    nL++;
                    sr += cell_density<S>(d, d.fdst, yi);
                } else if (c == CL_I) {
                    nI++;
                    sr += cell_density<S>(d, d.fdst, yi);
                    sp += d.phidst[yi];
                } else if (c == CL_G) {
                    nG++;
                }
            }
            uint8_t dec = 0;
            if (nL > 0 && nG > 0) {
                dec = CL_I;
                d.rrho[it] = sr / (nL + nI);
                d.rphi[it] = nI > 0 ? sp / nI : 0.5;
            } else if (nG == 0 && nL + nI > 0) {
                dec = CL_L;
                d.rrho[it] = sr / (nL + nI);
            } else if (nL == 0 && nG > 0) {
                dec = CL_G;
            }
            d.rdec[it] = dec;
        }
        if (threadIdx.x == 0) s_any = 0;
        __syncthreads();
        for (uint32_t it = threadIdx.x; it < n; it += blockDim.x) {
            long long i = d.list[WL_PEND][it];
            if (!(d.cmark[i] & MK_PEND)) continue;
            int dec = d.rdec[it];
            if (dec == 0 && pass == 3) dec = CL_G;
            if (dec == 0) {
                s_any = 1;
                continue;
            }
            const Body &b = d.bodies[d.bid[i]];
            d.cmark[i] = MK_FRESH;
            set_cls(d, i, dec);
            if (dec == CL_G) continue;
            int x, y, z;
            coords(d, i, x, y, z);
            if (z > *d.ztop_wr + ZTOP_MARGIN) atomicOr(d.status, ST_TOP);
            double p[3] = {x + 0.5, y + 0.5, z + 0.5}, uw[3];
            body_velocity_at(d, b, p, uw);
            double f[Q];
            double rho = d.rrho[it];
#pragma unroll
            for (int q = 0; q < Q; ++q) f[q] = feq_d(q, rho, uw);
            Sto<S>::st_cell(d.fdst, i, d.N, f);
            if (dec == CL_I) {
                double m = d.rphi[it] * rho;
                d.m[i] = m;
                d.phidst[i] = m / cell_density<S>(d, d.fdst, i);
            }
        }
        __syncthreads();
        if (!s_any) break;
        __syncthreads();
    }
    // closure: a new liquid cell next to gas becomes interface with phi = 1
    for (uint32_t it = threadIdx.x; it < n; it += blockDim.x) {
        long long i = d.list[WL_PEND][it];
        if (!(d.cmark[i] & MK_FRESH) || clsv(d, i) != CL_L) continue;
        int x, y, z;
        coords(d, i, x, y, z);
        bool gas = false;
        for (int q = 1; q < Q; ++q) {
            long long yi = nbr(d, x, y, z, cx(q), cy(q), cz(q));
            if (yi >= 0 && clsv(d, yi) == CL_G) gas = true;
        }
        d.rdec[it] = gas ? 1 : 0;
    }
    __syncthreads();
    double acc = 0.0;
    for (uint32_t it = threadIdx.x; it < n; it += blockDim.x) {
        long long i = d.list[WL_PEND][it];
        if (!(d.cmark[i] & MK_FRESH)) continue;
        if (clsv(d, i) == CL_L && d.rdec[it]) {
            set_cls(d, i, CL_I);
            double r = cell_density<S>(d, d.fdst, i);
            d.m[i] = r;
            d.phidst[i] = d.m[i] / cell_density<S>(d, d.fdst, i);
        }
        if (clsv(d, i) == CL_L) acc += cell_density<S>(d, d.fdst, i);
        else if (clsv(d, i) == CL_I) acc += d.m[i];
        d.cmark[i] = 0;
    }
    __shared__ double sh[REMAP_THREADS / 32];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        d.ledger[LG_UNCOVERED] += t;
    }
}
template <int S>
__global__ void __launch_bounds__(REMAP_THREADS) k_remap_resolve(const __grid_constant__ Dev d) { remap_resolve_body<S>(d, vb_own()); }

// ------------------------------------------------------ reductions, output

// sum over liquid rho + interface m -> red[block]
template <int S>
__global__ void __launch_bounds__(256) k_mass_partial(Dev d) {
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < d.N; i += (long long)gridDim.x * blockDim.x) {
        int c = clsv(d, i);
        if (c == CL_L) {
            acc += cell_density<S>(d, d.fsrc, i);
            // closed interface layer (Sec. 2.2): no liquid cell touches gas
            int x, y, z;
            coords(d, i, x, y, z);
            for (int q = 1; q < Q; ++q)
                if (cls(d, nbr(d, x, y, z, cx(q), cy(q), cz(q))) == CL_G) atomicOr(d.status, ST_LIQUID_GAS);
        } else if (c == CL_I) {
            acc += d.m[i];
        }
    }
    __shared__ double sh[8];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        d.red[blockIdx.x] = t;
    }
}

__global__ void k_mass_final(Dev d, int nblk) {
    if (threadIdx.x != 0) return;
    double t = 0.0;
    for (int k = 0; k < nblk; ++k) t += d.red[k];
    d.ledger[LG_MASS] = t;
}

template <int S>
__global__ void k_read_fields(Dev d, unsigned mask, uint8_t *flags, double *fill, double *mass, double *rho, double *vel,
                              double *f) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    int c = clsv(d, i);
    bool fluid = c == CL_L || c == CL_I;
    double u[3] = {0.0, 0.0, 0.0};
    double r = fluid ? cell_rho_u<S>(d, d.fsrc, i, u) : 0.0;
    if (flags) flags[i] = (uint8_t)c;
    if (fill) fill[i] = c == CL_L ? 1.0 : (c == CL_I ? d.phisrc[i] : 0.0);
    if (mass) mass[i] = c == CL_L ? r : (c == CL_I ? d.m[i] : 0.0);
    if (rho) rho[i] = r;
    if (vel) {
        vel[3 * i] = u[0];
        vel[3 * i + 1] = u[1];
        vel[3 * i + 2] = u[2];
    }
    if (f)
        for (int q = 0; q < Q; ++q) f[(long long)q * d.N + i] = fluid ? Sto<S>::ldf(d.fsrc, q, i, d.N) : 0.0;
}

// ------------------------------------------------------------ launchers

// ------------------------------------------------------ batched launches
//
// One launch serves all tanks of a TankSet: block b runs the table entries
// b, b + gridDim.x, ... (a persistent walk when the grid is smaller than the
// table), each as the block of its tank's own grid that the entry names, with
// the block size of the single-tank launch.  The per-cell work is the
// single-tank kernels' own code.
template <class K>
__global__ void __launch_bounds__(K::THREADS, K::MINB)
    k_batch(const __grid_constant__ TankSet ts, const Tile *__restrict__ table, unsigned n, int zb) {
    for (unsigned t = blockIdx.x; t < n; t += gridDim.x) {
        const Tile e = table[t];
        const VB vb{e.x, e.y, e.z, e.nx, e.ny, e.nz};
        K::run(ts.d[e.tank], vb, zb);
        // the next entry's body reuses this one's shared memory; bodies
        // without shared memory let a block's warps move on independently
        if constexpr (K::SMEM) __syncthreads();
    }
}

#define LBMFS_BATCH_BODY_SM(NAME, THR, MB, SM, CALL)                                          \
    struct NAME {                                                                              \
        static constexpr int THREADS = THR, MINB = MB;                                         \
        static constexpr bool SMEM = SM;                                                       \
        static __device__ __forceinline__ void run(const Dev &d, const VB &vb, int zb) { CALL; } \
    };
#define LBMFS_BATCH_BODY(NAME, THR, MB, CALL) LBMFS_BATCH_BODY_SM(NAME, THR, MB, false, CALL)
struct BkReset {
    static constexpr int THREADS = 32, MINB = 1;
    static constexpr bool SMEM = false;
    static __device__ __forceinline__ void run(const Dev &d, const VB &, int) {
        if (threadIdx.x < WL_COUNT) d.cnt[threadIdx.x] = 0;
    }
};
template <int S> LBMFS_BATCH_BODY_SM(BkForces, 256, S == 0 ? 2 : LBMFS_FORCE_MINB, true, forces_body<S>(d, vb))
// one instantiation per z-planes-per-tile choice (the column loop unrolled to it)
template <int S, int ZB>
LBMFS_BATCH_BODY(BkLiquid, BULK_THREADS, S == 0 ? 1 : (LBMFS_BULK_PAIR ? LBMFS_PAIR_MINB : LBMFS_BULK_MINB),
                 (bulk_body<S, ZB>(d, vb, zb)))
// the batch's listed cells are spread over many more blocks: 4 resident per SM
// (128 registers) beat 1 there, not on the single tank
template <int S> LBMFS_BATCH_BODY(BkGeneral, GEN_THREADS, 4, general_body<S>(d, vb))
template <int S> LBMFS_BATCH_BODY(BkInterface, 128, LBMFS_IFACE_MINB, interface_body<S>(d, vb))
LBMFS_BATCH_BODY(BkConvFilled, LIST_THREADS, 1, conv_filled_body(d, vb))
LBMFS_BATCH_BODY(BkConvEmptied, LIST_THREADS, 1, conv_emptied_body(d, vb))
template <int S> LBMFS_BATCH_BODY(BkConvInit, LIST_THREADS, 1, conv_init_body<S>(d, vb))
LBMFS_BATCH_BODY(BkConvFlags, LIST_THREADS, 1, conv_flags_body(d, vb))
template <int S> LBMFS_BATCH_BODY(BkConvClaim, LIST_THREADS, 1, conv_claim_body<S>(d, vb))
template <int S> LBMFS_BATCH_BODY(BkConvExcess, LIST_THREADS, 1, conv_excess_body<S>(d, vb))
template <int S> LBMFS_BATCH_BODY(BkConvFinish, LIST_THREADS, 1, conv_finish_body<S>(d, vb))
LBMFS_BATCH_BODY(BkBodies, 32, 1, bodies_body(d, vb))
template <int S> LBMFS_BATCH_BODY(BkRemapCover, 256, 1, remap_cover_body<S>(d, vb))
LBMFS_BATCH_BODY(BkRemapPending, 256, 1, remap_pending_body(d, vb))
template <int S> LBMFS_BATCH_BODY_SM(BkRemapResolve, REMAP_THREADS, 1, true, remap_resolve_body<S>(d, vb))
LBMFS_BATCH_BODY(BkNbUpdate, LIST_THREADS, 1, nb_update_body(d, vb))
#undef LBMFS_BATCH_BODY
#undef LBMFS_BATCH_BODY_SM

template <class K> void batch_launch(const BatchLaunch &b, int sh, dim3 block, cudaStream_t st) {
    const Shape &x = b.sh[sh];
    if (x.n) k_batch<K><<<x.grid, block, 0, st>>>(*b.ts, x.table, x.n, b.zb);
}
template <int S> void batch_bulk_launch(const BatchLaunch &b, cudaStream_t st) {
    switch (b.zb) {
    case 1: batch_launch<BkLiquid<S, 1>>(b, SH_BULK, BULK_THREADS, st); break;
    case 2: batch_launch<BkLiquid<S, 2>>(b, SH_BULK, BULK_THREADS, st); break;
    case 4: batch_launch<BkLiquid<S, 4>>(b, SH_BULK, BULK_THREADS, st); break;
    default: batch_launch<BkLiquid<S, 8>>(b, SH_BULK, BULK_THREADS, st); break;
    }
}

template <int S> struct Launch {
    static void init_cells(const Dev &d, const uint8_t *flags, const double *fill, const double *rho, const double *vel,
                           cudaStream_t st) {
        unsigned blocks = (unsigned)((d.N + 255) / 256);
        k_init<S><<<blocks, 256, 0, st>>>(d, flags, fill, rho, vel);
        k_nb_all<<<dim3((d.nx + 127) / 128, d.ny, d.nz), 128, 0, st>>>(d);
    }
    static void body_prepare(const Dev &d, int b, cudaStream_t st) { k_body_prepare<<<1, 32, 0, st>>>(d, b); }
    static void map_body(const Dev &d, int b, int book, cudaStream_t st) {
        k_map_body<S><<<FORCE_BLOCKS, 256, 0, st>>>(d, b, book);
        k_nb_body<<<FORCE_BLOCKS, dim3(32, 8), 0, st>>>(d, b);
    }
    static void liquid_mass(const Dev &d, cudaStream_t st) {
        k_mass_partial<S><<<LIST_BLOCKS, 256, 0, st>>>(d);
        k_mass_final<<<1, 32, 0, st>>>(d, LIST_BLOCKS);
    }
    static void read_fields(const Dev &d, unsigned mask, void *const *dst, cudaStream_t st) {
        unsigned blocks = (unsigned)((d.N + 255) / 256);
        k_read_fields<S><<<blocks, 256, 0, st>>>(
            d, mask, (mask & 1u) ? (uint8_t *)dst[0] : nullptr, (mask & 2u) ? (double *)dst[1] : nullptr,
            (mask & 4u) ? (double *)dst[2] : nullptr, (mask & 8u) ? (double *)dst[3] : nullptr,
            (mask & 16u) ? (double *)dst[4] : nullptr, (mask & 32u) ? (double *)dst[5] : nullptr);
    }
    // one time step; with ev != nullptr, event k is recorded before kernel k
    // and ev[count] after the last one
    static int step(const Dev &d, cudaStream_t st, float *, cudaEvent_t *ev) {
        int k = 0;
        auto mark = [&]() {
            if (ev) cudaEventRecord(ev[k], st);
            ++k;
        };
        mark();
        cudaMemsetAsync(d.cnt, 0, WL_COUNT * sizeof(uint32_t), st);
        mark();
        if (d.nb > 0) k_forces<S><<<dim3(FORCE_BLOCKS, d.nb), dim3(32, 8), 0, st>>>(d);
        mark();
        {
            const long long nxy = (long long)d.nx * d.ny;
            const int bc = bulk_cells(S, d);
            dim3 grid((unsigned)((nxy + bc - 1) / bc), 1, (d.nz + LBMFS_BULK_ZB - 1) / LBMFS_BULK_ZB);
            if constexpr (S != 0) {
                // the staged variants tile rows: (ceil(nx / BULK_THREADS), ny, z-blocks)
                dim3 rgrid((d.nx + BULK_THREADS - 1) / BULK_THREADS, d.ny, (d.nz + LBMFS_BULK_ZB - 1) / LBMFS_BULK_ZB);
                dim3 pgrid(rgrid.x, rgrid.y, (d.nz + LBMFS_BULK_PIPE_ZB - 1) / LBMFS_BULK_PIPE_ZB);
                if (d.bulk == BULK_TMA) k_liquid_tma<S><<<rgrid, BULK_THREADS, 128 + 2 * Stage<S>::BYTES, st>>>(d);
                else if (d.bulk == BULK_PIPE) k_liquid_pipe<S><<<pgrid, BULK_THREADS, 0, st>>>(d);
                else k_liquid<S><<<grid, BULK_THREADS, 0, st>>>(d);
            } else {
                k_liquid<S><<<grid, BULK_THREADS, 0, st>>>(d);
            }
        }
        mark();
        k_general<S><<<LIST_BLOCKS, GEN_THREADS, 0, st>>>(d);
        mark();
        k_interface<S><<<LBMFS_IFACE_GRID, 128, 0, st>>>(d);
        mark();
        k_conv_filled<<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(d);
        mark();
        k_conv_emptied<<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(d);
        mark();
        k_conv_init<S><<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(d);
        mark();
        k_conv_flags<<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(d);
        mark();
        k_conv_claim<S><<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(d);
        mark();
        k_conv_excess<S><<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(d);
        mark();
        k_conv_finish<S><<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(d);
        mark();
        if (d.nb > 0) launch_bodies(d, st);
        mark();
        if (d.nb > 0) k_remap_cover<S><<<dim3(FORCE_BLOCKS, d.nb), 256, 0, st>>>(d);
        mark();
        if (d.nb > 0) k_remap_pending<<<dim3(FORCE_BLOCKS, d.nb), 256, 0, st>>>(d);
        mark();
        if (d.nb > 0) k_remap_resolve<S><<<1, REMAP_THREADS, 0, st>>>(d);
        mark();
        if (d.nb > 0) k_nb_update<<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(d);
        mark();
        return d.nb > 0 ? 16 : 10;  // kernels (the counter reset is a memset node)
    }
};

// The batched counterpart of Launch<S>::step (same kernel slots).
template <int S> struct BatchStep {
    static int step(const BatchLaunch &b, cudaStream_t st, cudaEvent_t *ev) {
        int k = 0;
        auto mark = [&]() {
            if (ev) cudaEventRecord(ev[k], st);
            ++k;
        };
        mark();
        batch_launch<BkReset>(b, SH_TANK, 32, st);
        mark();
        batch_launch<BkForces<S>>(b, SH_FORCE, dim3(32, 8), st);
        mark();
        batch_bulk_launch<S>(b, st);
        mark();
        batch_launch<BkGeneral<S>>(b, SH_IFACE, GEN_THREADS, st);
        mark();
        batch_launch<BkInterface<S>>(b, SH_IFACE, 128, st);
        mark();
        batch_launch<BkConvFilled>(b, SH_LIST, LIST_THREADS, st);
        mark();
        batch_launch<BkConvEmptied>(b, SH_LIST, LIST_THREADS, st);
        mark();
        batch_launch<BkConvInit<S>>(b, SH_LIST, LIST_THREADS, st);
        mark();
        batch_launch<BkConvFlags>(b, SH_LIST, LIST_THREADS, st);
        mark();
        batch_launch<BkConvClaim<S>>(b, SH_LIST, LIST_THREADS, st);
        mark();
        batch_launch<BkConvExcess<S>>(b, SH_LIST, LIST_THREADS, st);
        mark();
        batch_launch<BkConvFinish<S>>(b, SH_LIST, LIST_THREADS, st);
        mark();
        launch_bodies_batch(b, st);
        mark();
        batch_launch<BkRemapCover<S>>(b, SH_FORCE, 256, st);
        mark();
        batch_launch<BkRemapPending>(b, SH_FORCE, 256, st);
        mark();
        batch_launch<BkRemapResolve<S>>(b, SH_ONE, REMAP_THREADS, st);
        mark();
        batch_launch<BkNbUpdate>(b, SH_LIST, LIST_THREADS, st);
        mark();
        int n = 0;
        const int shapes[] = {SH_TANK, SH_FORCE, SH_BULK, SH_IFACE, SH_IFACE, SH_LIST, SH_LIST, SH_LIST, SH_LIST,
                              SH_LIST, SH_LIST, SH_LIST, SH_BODY, SH_FORCE, SH_FORCE, SH_ONE, SH_LIST};
        for (int sh : shapes) n += b.sh[sh].n ? 1 : 0;
        return n;
    }
    static void bulk(const BatchLaunch &b, cudaStream_t st) { batch_bulk_launch<S>(b, st); }
    static int bulk_blocks_per_sm() {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<BkLiquid<S, 4>>, BULK_THREADS, 0) != cudaSuccess)
            return 1;
        return nb > 0 ? nb : 1;
    }
};

inline const char *const *kernel_names() {
    static const char *const n[] = {"reset_counters", "forces", "liquid", "general", "interface", "conv_filled",
                                    "conv_emptied",    "conv_init", "conv_flags", "conv_claim", "conv_excess",
                                    "conv_finish",     "bodies",  "remap_cover", "remap_pending", "remap_resolve", "nb_update"};
    return n;
}

template <int S> KernelSet make_kernel_set() {
    KernelSet k;
    k.init_cells = &Launch<S>::init_cells;
    k.body_prepare = &Launch<S>::body_prepare;
    k.map_body = &Launch<S>::map_body;
    k.step = &Launch<S>::step;
    k.liquid_mass = &Launch<S>::liquid_mass;
    k.read_fields = &Launch<S>::read_fields;
    k.batch_step = &BatchStep<S>::step;
    k.batch_bulk = &BatchStep<S>::bulk;
    k.bulk_blocks_per_sm = &BatchStep<S>::bulk_blocks_per_sm;
    k.nkernels = 17;
    k.names = kernel_names();
    return k;
}

}  // namespace
}  // namespace lbmfs
