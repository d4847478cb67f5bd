// A ragged batch in ONE persistent launch, reading the set descriptors
// (sph_batch_set) from device memory.
//
// Every block first turns the descriptor array into its own work table in
// shared memory: a stable counting sort of the sets by decreasing l_max and
// the prefix sums of the sets' tile counts in that order. Every block
// computes the same table from the same descriptors, so no block waits for
// another. The blocks (one per SM) then run the l_max classes present one
// after the other: for each class a compile-time l_max body, that class's
// tile size (the single-set POINT tile), its own tile counter, and as many
// active warps as that tile's staging buffer allows in the block's shared
// memory -- so every class runs with the occupancy of a launch of its own,
// inside one launch. A block moves to the next class as soon as the current
// class's counter is exhausted and its warps' bulk stores have read their
// buffers (a block barrier); other blocks move on independently.
//
// The tile counters reset themselves: the last block to finish returns them
// to zero, so a launch needs no memset and no allocation. Counters come from
// a ring of static device slots (or from the caller, for plans).
#pragma once

#include <cuda_runtime.h>

#include "sph_batch.cuh"

namespace sph {

constexpr int kOneMaxSets = 2048;          // sets per launch; the host splits longer arrays
constexpr int kOneRingSlots = 256;         // self-resetting counters per device and flag class
constexpr uint32_t kStatusBatchDesc = 2u;  // a descriptor was rejected and its set skipped
constexpr int kOneMaxTile = 32;            // points per tile (one row per lane)
constexpr int kOneMaxWarps = 16;           // warps per block (register file: 128 registers a thread)
constexpr int kOneKeys = SPH_MAX_L_POINT + 2;  // l_max classes (key 16 - l_max), then rejected sets

struct OneCounter {
    unsigned long long tickets[kOneKeys];  // one tile counter per class
    unsigned int done;
    unsigned int pad;
};

// Per l_max: tile points, staged bytes per warp (128-byte aligned parts) and
// the warps of a block that run that class.
struct OneClass {
    int32_t P;
    int32_t bytes;
    int32_t W;
    int32_t pad;
};

struct OneParams {
    PointTabs<16, float, false> tabs;  // Eq. iter-q / iter-deri for every l <= 16
    OneClass cls[SPH_MAX_L_POINT + 1];
};

// Shared memory after the warps' staging buffers: the sorted set order
// (uint16) and the tile prefix sums (int64, nsets + 1 entries).
__host__ __device__ constexpr size_t one_table_bytes(int nsets) {
    return align16(size_t(nsets) * 2) + align16(size_t(nsets + 1) * 8);
}
// Scratch of the table build, inside the staging area: sort keys (uint8)
// and tile counts (int64) per set.
__host__ __device__ constexpr size_t one_scratch_bytes(int nsets) {
    return align16(size_t(nsets)) + size_t(nsets) * 8;
}

__host__ __device__ constexpr size_t align128(size_t b) { return (b + 127) & ~size_t(127); }

struct OneSet {
    const float* xyz;
    float* sph;
    float* dsph;
    int64_t n;
    int64_t base;  // first tile of the set in the launch's tile order
    int L;
    int P;
    int bulk;
};

// Classes with gradients from l_max kPoint4MinL run 4 lanes per point (one
// per output plane, tiles of <= 8 points); the others one lane per point.
template <int L, int GN>
__host__ __device__ constexpr bool one_four() {
    return (GN & 1) != 0 && L >= kPoint4MinL;
}

template <int L, int GN>
__device__ __forceinline__ void one_tile(const OneSet& s, int64_t t, unsigned char* buf,
                                         const PointTabs<16, float, false>& tb, int lane, float px, float py,
                                         float pz) {
    constexpr int K = (L + 1) * (L + 1);
    constexpr bool GRAD = (GN & 1) != 0;
    constexpr bool NORM = (GN & 2) != 0;
    using RS = RowStride<L>;
    const int P = s.P;
    const int64_t p0 = t * P;
    const int cnt = int(min(int64_t(P), s.n - p0));
    if constexpr (one_four<L, GN>()) {
        point4_tile<L, NORM>(s.sph, s.dsph, p0, cnt, P, s.bulk, buf, tb, lane, px, py, pz);
        return;
    }
    float* s_v = reinterpret_cast<float*>(buf);
    float* s_d = reinterpret_cast<float*>(buf + align128(size_t(P) * RS::V * 4));
    // Rows lane, lane + 32, ...: the next row's coordinates are loaded while
    // the current row is computed (the first row was prefetched by the caller).
    float x = px, y = py, z = pz;
    for (int row = lane; row < cnt; row += 32) {
        float nx = 0.f, ny = 0.f, nz = 0.f;
        if (row + 32 < cnt) {
            const float* q = s.xyz + 3 * (p0 + row + 32);
            nx = q[0];
            ny = q[1];
            nz = q[2];
        }
        float r2, ir = 1.f;
        if (NORM) {
            unit_point(x, y, z, r2, ir);
        } else {
            r2 = x * x + y * y + z * z;
        }
        BatchVis<K, GN> vis{s_v + size_t(row) * RS::V, GRAD ? s_d + size_t(row) * RS::D : nullptr, x, y, z, ir,
                            NORM ? 1 : 0};
        point_core<L, GRAD, false>(x, y, z, r2, tb, vis);
        x = nx;
        y = ny;
        z = nz;
    }
    if constexpr (RS::PAD) {  // even K: odd-stride rows, coalesced plain copy-out
        __syncwarp();
        warp_rows_out<K>(s.sph + p0 * K, s_v, cnt, RS::V, lane);
        if (GRAD) warp_rows_out<3 * K>(s.dsph + p0 * 3 * K, s_d, cnt, RS::D, lane);
        __syncwarp();
        return;
    }
    fence_proxy_async_smem();
    __syncwarp();
    const int64_t ev = int64_t(cnt) * K;
    int64_t ev_bulk = 0, ed_bulk = 0;
    if (s.bulk) {
        ev_bulk = (ev * 4) / 16 * 4;
        ed_bulk = GRAD ? (3 * ev * 4) / 16 * 4 : 0;
        if (lane == 0) {
            if (ev_bulk) bulk_store(s.sph + p0 * K, s_v, uint32_t(ev_bulk * 4));
            if (ed_bulk) bulk_store(s.dsph + p0 * 3 * K, s_d, uint32_t(ed_bulk * 4));
            bulk_commit();
        }
    }
    for (int64_t i = ev_bulk + lane; i < ev; i += 32) s.sph[p0 * K + i] = s_v[i];
    if (GRAD)
        for (int64_t i = ed_bulk + lane; i < 3 * ev; i += 32) s.dsph[p0 * 3 * K + i] = s_d[i];
    if (s.bulk && lane == 0) bulk_wait_read_all();
    __syncwarp();
}

#ifdef SPH_BATCH_ONE_KERNELS
// The ring of self-resetting counters of this translation unit (one per
// flag class); zero when the module loads.
static __device__ OneCounter g_one_ring[kOneRingSlots];

// The tiles of one l_max class: runs of kBatchRun tiles from the class's
// counter, sets at sorted positions [s0, s1), class tiles [T0, T1) of the
// launch's tile order.
template <int L, int GN>
__device__ __forceinline__ void one_class(const sph_batch_set* __restrict__ desc, const uint16_t* ord,
                                          const int64_t* pre, int s0, int s1, int64_t T0, int64_t T1,
                                          unsigned long long* tickets, unsigned char* buf, const OneParams& prm,
                                          int lane) {
    constexpr bool GRAD = (GN & 1) != 0;
    const int P = prm.cls[L].P;
    const int64_t Tc = T1 - T0;
    unsigned long long run = 0, nrun = 0;
    if (lane == 0) run = atomicAdd(tickets, 1ull);
    run = __shfl_sync(0xffffffffu, run, 0);
    if (lane == 0) nrun = atomicAdd(tickets, 1ull);
    int p = -1;
    OneSet s{};
    auto locate = [&](int64_t t) {  // forward scan: t never decreases for a warp
        int q = p < 0 ? s0 : p;
        while (q + 1 < s1 && t >= pre[q + 1]) ++q;
        if (q != p) {
            p = q;
            const sph_batch_set d = desc[ord[q]];
            s.xyz = d.xyz;
            s.sph = d.sph;
            s.dsph = d.dsph;
            s.n = d.n;
            s.L = L;
            s.P = P;
            s.base = pre[q];
            s.bulk = (reinterpret_cast<uintptr_t>(d.sph) % 16 == 0 &&
                      (!GRAD || reinterpret_cast<uintptr_t>(d.dsph) % 16 == 0))
                         ? 1
                         : 0;
        }
    };
    const int me = one_four<L, GN>() ? lane >> 2 : lane;  // this lane's point of a tile
    auto prefetch = [&](int64_t t, float& x, float& y, float& z) {
        const int64_t q = (t - s.base) * P + me;
        if (me < P && q < s.n) {
            x = s.xyz[3 * q];
            y = s.xyz[3 * q + 1];
            z = s.xyz[3 * q + 2];
        }
    };
    int64_t tl = int64_t(run) * kBatchRun;  // class-local tile
    float px = 0.f, py = 0.f, pz = 0.f;
    if (tl < Tc) {
        locate(T0 + tl);
        prefetch(T0 + tl, px, py, pz);
    }
    while (tl < Tc) {
        int64_t tn = tl + 1;
        if (tn % kBatchRun == 0) {
            const unsigned long long r = __shfl_sync(0xffffffffu, nrun, 0);
            tn = int64_t(r) * kBatchRun;
            if (lane == 0) nrun = atomicAdd(tickets, 1ull);
        }
        const OneSet cur = s;
        const float cx = px, cy = py, cz = pz;
        if (tn < Tc) {
            locate(T0 + tn);
            prefetch(T0 + tn, px, py, pz);
        }
        one_tile<L, GN>(cur, T0 + tl - cur.base, buf, prm.tabs, lane, cx, cy, cz);
        tl = tn;
    }
}

// GN = gradients + 2 * normalized, the same for every set of the launch; a
// non-empty set whose descriptor disagrees (dsph NULL with gradients, or the
// reverse; another normalized flag), or a set whose l_max, n or pointers are
// invalid, is skipped and kStatusBatchDesc is OR-ed into *status.
template <int GN>
__global__ void __launch_bounds__(32 * kOneMaxWarps, 1)
    batch_one_kernel(const sph_batch_set* __restrict__ desc, int nsets, OneCounter* __restrict__ ctr_arg, int slot,
                     int staging_bytes, uint32_t* __restrict__ status, const __grid_constant__ OneParams prm) {
    OneCounter* ctr = ctr_arg != nullptr ? ctr_arg : &g_one_ring[slot];
    constexpr bool GRAD = (GN & 1) != 0;
    constexpr bool NORM = (GN & 2) != 0;
    constexpr int kKeys = kOneKeys;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_cnt[kKeys], s_base[kKeys], s_run[kKeys];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char* table = smem + size_t(staging_bytes);
    uint16_t* ord = reinterpret_cast<uint16_t*>(table);
    int64_t* pre = reinterpret_cast<int64_t*>(table + align16(size_t(nsets) * 2));
    uint8_t* key = smem;  // build scratch in the staging area
    int64_t* ntl = reinterpret_cast<int64_t*>(smem + align16(size_t(nsets)));

    // ---- the work table: sets by decreasing l_max (stable), tile prefix sums
    if (threadIdx.x < kKeys) {
        s_cnt[threadIdx.x] = 0;
        s_run[threadIdx.x] = 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nsets; i += blockDim.x) {
        const sph_batch_set d = desc[i];
        const uintptr_t al = reinterpret_cast<uintptr_t>(d.xyz) | reinterpret_cast<uintptr_t>(d.sph) |
                             reinterpret_cast<uintptr_t>(d.dsph);
        // an empty set needs no buffers and no matching flags
        const bool ok = d.l_max >= 0 && d.l_max <= SPH_MAX_L_POINT && d.n >= 0 &&
                        (d.n == 0 || ((al & 3u) == 0 && d.xyz != nullptr && d.sph != nullptr &&
                                      (d.dsph != nullptr) == GRAD && (d.normalized != 0) == NORM));
        int k = kKeys - 1;
        int64_t tiles = 0;
        if (ok) {
            k = SPH_MAX_L_POINT - d.l_max;
            const int P = prm.cls[d.l_max].P;
            tiles = (d.n + P - 1) / P;
        } else if (blockIdx.x == 0 && status != nullptr) {
            atomicOr(status, kStatusBatchDesc);
        }
        key[i] = uint8_t(k);
        ntl[i] = tiles;
        atomicAdd(&s_cnt[k], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int k = 0; k < kKeys; ++k) {
            s_base[k] = acc;
            acc += s_cnt[k];
        }
    }
    __syncthreads();
    if (warp == 0) {
        // stable placement: rank among earlier sets of the same key
        for (int c = 0; c < nsets; c += 32) {
            const int i = c + lane;
            const int k = i < nsets ? int(key[i]) : 255;
            const unsigned m = __match_any_sync(0xffffffffu, k);
            const int rank = __popc(m & ((1u << lane) - 1u));
            if (i < nsets) ord[s_base[k] + s_run[k] + rank] = uint16_t(i);
            __syncwarp();
            if (i < nsets && lane == __ffs(m) - 1) s_run[k] += __popc(m);
            __syncwarp();
        }
        int64_t carry = 0;
        for (int c = 0; c < nsets; c += 32) {
            const int p = c + lane;
            const int64_t v = p < nsets ? ntl[ord[p]] : 0;
            int64_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            if (p < nsets) pre[p] = carry + incl - v;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) pre[nsets] = carry;
    }
    __syncthreads();

    // ---- the classes present, by decreasing l_max
    for (int k = 0; k <= SPH_MAX_L_POINT; ++k) {
        const int cnt = s_cnt[k];
        if (cnt == 0) continue;
        const int s0 = s_base[k], s1 = s0 + cnt;
        const int64_t T0 = pre[s0], T1 = pre[s1];
        if (T1 == T0) continue;
        const int L = SPH_MAX_L_POINT - k;
        if (warp < prm.cls[L].W) {
            unsigned char* buf = smem + size_t(warp) * size_t(prm.cls[L].bytes);
            switch (L) {
#define SPH_CASE(LL)                                                                             \
    case LL:                                                                                     \
        one_class<LL, GN>(desc, ord, pre, s0, s1, T0, T1, &ctr->tickets[k], buf, prm, lane);     \
        break;
                SPH_CASE(0) SPH_CASE(1) SPH_CASE(2) SPH_CASE(3) SPH_CASE(4) SPH_CASE(5) SPH_CASE(6) SPH_CASE(7)
                SPH_CASE(8) SPH_CASE(9) SPH_CASE(10) SPH_CASE(11) SPH_CASE(12) SPH_CASE(13) SPH_CASE(14)
                SPH_CASE(15) SPH_CASE(16)
#undef SPH_CASE
                default:
                    break;
            }
            // the next class lays its buffers out differently: every bulk
            // store of this warp must have read its buffer (4-lane tiles of
            // some l_max send one row per lane)
            bulk_wait_read_all();
        }
        __syncthreads();
    }
    bulk_wait_all();

    // ---- the last block to finish returns the counters to zero
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&ctr->done, 1u);
        if (prev == gridDim.x - 1) {
            for (int k = 0; k < kKeys; ++k) atomicExch(&ctr->tickets[k], 0ull);
            atomicExch(&ctr->done, 0u);
            __threadfence();
        }
    }
}
#endif  // SPH_BATCH_ONE_KERNELS

// One launch over at most kOneMaxSets descriptors.
struct OneArgs {
    const sph_batch_set* desc;  // device
    int nsets;
    OneCounter* ctr;            // nullptr: a slot of the static ring
    int staging_bytes;          // shared memory of the warps' staging buffers
    int W;                      // warps per block
    int blocks;                 // grid (<= blocks resident at once)
    size_t smem;
    const OneClass* cls;        // [SPH_MAX_L_POINT + 1], host
    uint32_t* status;           // device status word or nullptr
    void* stream;
    int* occ_out;               // non-null: set the shared-memory attribute, return the occupancy, no launch
};

}  // namespace sph
