// Ragged-batch tile body and persistent kernels, shared by the batch plans
// (csrc/sph_batch.cu) and the per-l_max instantiations (csrc/sph_point_inst.cu).
//
// A tile holds P consecutive points of one set; its outputs are staged in
// shared memory and written with bulk (TMA) copies (see sph_point.cuh).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "sph_point.cuh"

namespace sph {

constexpr int kBatchMaxTile = 256;  // points per batch tile (8 per lane)

struct BatchSet {
    const float* xyz;
    float* sph;
    float* dsph;
    int64_t n;
    int64_t tile_begin;  // prefix sum of tiles over the (sorted) sets
    int32_t L;
    int32_t P;           // points per tile for this set
    int32_t norm;
    int32_t bulk;        // outputs 16-byte aligned: bulk copies allowed
};

// Gradients / normalization of a tile: GN < 0 reads them from the set at run
// time (one launch for every kind of set); GN = grad + 2 * norm fixes them at
// compile time (one launch per class of equal l_max, gradients and norm).
template <int K, int GN>
struct BatchVis {
    float* rv;
    float* rd;  // nullptr: values only
    float ux, uy, uz, ir;
    int norm;
    __device__ __forceinline__ void emit(int l, int k, Deriv<float> d) {
        rv[k] = d.v;
        const bool grad = GN < 0 ? rd != nullptr : (GN & 1) != 0;
        const bool nrm = GN < 0 ? norm != 0 : (GN & 2) != 0;
        if (grad) {
            if (nrm) normalize_deriv<false>(d, l, ux, uy, uz, ir);
            rd[k] = d.gx;
            rd[K + k] = d.gy;
            rd[2 * K + k] = d.gz;
        }
    }
};

// Per-class launches (flags fixed at compile time) with gradients from
// l_max kPoint4MinL run 4 lanes per point (one per output plane, tiles of
// <= 8 points); every other tile one lane per point.
template <int L, int GN>
__host__ __device__ constexpr bool batch_four() {
    return GN >= 0 && (GN & 1) != 0 && L >= kPoint4MinL;
}

template <int L, int GN>
__device__ __forceinline__ void batch_tile(const BatchSet& s, int64_t t, unsigned char* buf,
                                           const PointTabs<16, float, false>& tb, int lane, float px, float py,
                                           float pz) {
    constexpr int K = (L + 1) * (L + 1);
    using RS = RowStride<L>;
    const int P = s.P;
    const int64_t p0 = t * P;
    const int cnt = int(min(int64_t(P), s.n - p0));
    if constexpr (batch_four<L, GN>()) {
        point4_tile<L, (GN & 2) != 0>(s.sph, s.dsph, p0, cnt, P, s.bulk, buf, tb, lane, px, py, pz);
        return;
    }
    float* s_v = reinterpret_cast<float*>(buf);
    float* s_d = reinterpret_cast<float*>(buf + align16(size_t(P) * RS::V * 4));
    const bool grad = GN < 0 ? s.dsph != nullptr : (GN & 1) != 0;
    const bool norm = GN < 0 ? s.norm != 0 : (GN & 2) != 0;
    // A tile may hold more than 32 points (small l_max): lane j computes the
    // rows j, j+32, ... so that every set's tile fills the per-warp budget.
    for (int row = lane; row < cnt; row += 32) {
        const int64_t p = p0 + row;
        // the first row's coordinates were prefetched by the caller
        float x = px, y = py, z = pz;
        if (row != lane) {
            x = s.xyz[3 * p];
            y = s.xyz[3 * p + 1];
            z = s.xyz[3 * p + 2];
        }
        float r2, ir = 1.f;
        if (norm) {
            unit_point(x, y, z, r2, ir);
        } else {
            r2 = x * x + y * y + z * z;
        }
        BatchVis<K, GN> vis{s_v + size_t(row) * RS::V, grad ? s_d + size_t(row) * RS::D : nullptr, x, y, z, ir,
                            norm ? 1 : 0};
        // The l_max = 16 table holds every l <= 16 with the same layout
        // prefix (entry (l, m) at l(l+1)/2 + m), so it serves every L.
        point_core<L, true, false>(x, y, z, r2, tb, vis);
    }
    if constexpr (RS::PAD) {  // even K: odd-stride rows, coalesced plain copy-out
        __syncwarp();
        warp_rows_out<K>(s.sph + p0 * K, s_v, cnt, RS::V, lane);
        if (grad) warp_rows_out<3 * K>(s.dsph + p0 * 3 * K, s_d, cnt, RS::D, lane);
        __syncwarp();
        return;
    }
    fence_proxy_async_smem();
    __syncwarp();
    const int64_t ev = int64_t(cnt) * K;
    int64_t ev_bulk = 0, ed_bulk = 0;
    if (s.bulk) {
        ev_bulk = (ev * 4) / 16 * 4;
        ed_bulk = grad ? (3 * ev * 4) / 16 * 4 : 0;
        if (lane == 0) {
            if (ev_bulk) bulk_store(s.sph + p0 * K, s_v, uint32_t(ev_bulk * 4));
            if (ed_bulk) bulk_store(s.dsph + p0 * 3 * K, s_d, uint32_t(ed_bulk * 4));
            bulk_commit();
        }
    }
    for (int64_t i = ev_bulk + lane; i < ev; i += 32) s.sph[p0 * K + i] = s_v[i];
    if (grad)
        for (int64_t i = ed_bulk + lane; i < 3 * ev; i += 32) s.dsph[p0 * 3 * K + i] = s_d[i];
    if (s.bulk && lane == 0) bulk_wait_read_all();
    __syncwarp();
}

// Tables of Eq. iter-q / iter-deri for l <= 16, shared by every set.
struct BatchTabs {
    PointTabs<16, float, false> t;
};

constexpr int kBatchRun = 4;  // consecutive tiles a warp takes per counter increment

// The persistent kernel over the tiles [tile_begin, tile_end) of the sets
// [set_begin, set_end) (sets sorted by decreasing l_max, tile prefix sums in
// BatchSet::tile_begin). FIXL < 0: one launch for every l_max, a switch over
// the compile-time bodies; FIXL >= 0: every set of the range has that l_max
// (and, for GN >= 0, those gradient / norm flags) and only its body is
// compiled (one launch per class).
template <int FIXL, int GN>
__global__ void __launch_bounds__(256) batch_kernel_t(const BatchSet* __restrict__ sets, int set_begin, int set_end,
                                                      int64_t tile_begin, int64_t tile_end,
                                                      unsigned long long* __restrict__ counter, int per_warp_bytes,
                                                      const __grid_constant__ BatchTabs tabs) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char* buf = smem + size_t(warp) * per_warp_bytes;
    // Warps take runs of kBatchRun consecutive tiles from the counter (the
    // next run is requested one run ahead). Runs are handed out in increasing
    // order, so each warp finds a tile's set by scanning forward from the set
    // of its previous tile, and prefetches the next tile's coordinates while
    // the current tile is computed.
    unsigned long long run = 0, nrun = 0;
    if (lane == 0) run = atomicAdd(counter, 1ull);
    run = __shfl_sync(0xffffffffu, run, 0);
    if (lane == 0) nrun = atomicAdd(counter, 1ull);
    int si = set_begin;
    BatchSet s = sets[si];
    int64_t s_end = (si + 1 < set_end) ? sets[si + 1].tile_begin : tile_end;
    auto locate = [&](int64_t t) {  // forward scan: t never decreases for a warp
        while (t >= s_end && si + 1 < set_end) {
            ++si;
            s = sets[si];
            s_end = (si + 1 < set_end) ? sets[si + 1].tile_begin : tile_end;
        }
    };
    const int me = (FIXL >= 0 && batch_four<(FIXL >= 0 ? FIXL : 0), GN>()) ? lane >> 2 : lane;  // lane's point
    auto prefetch = [&](int64_t t, float& x, float& y, float& z) {
        const int64_t p = (t - s.tile_begin) * s.P + me;
        if (me < s.P && p < s.n) {
            x = s.xyz[3 * p];
            y = s.xyz[3 * p + 1];
            z = s.xyz[3 * p + 2];
        }
    };
    int64_t t = tile_begin + int64_t(run) * kBatchRun;
    float px = 0.f, py = 0.f, pz = 0.f;
    if (t < tile_end) {
        locate(t);
        prefetch(t, px, py, pz);
    }
    while (t < tile_end) {
        // next tile: the following one in this run, else the first of the next run
        int64_t tn = t + 1;
        if ((tn - tile_begin) % kBatchRun == 0) {
            const unsigned long long r = __shfl_sync(0xffffffffu, nrun, 0);
            tn = tile_begin + int64_t(r) * kBatchRun;
            if (lane == 0) nrun = atomicAdd(counter, 1ull);
        }
        const BatchSet cur = s;
        const int64_t lt = t - cur.tile_begin;
        const float cx = px, cy = py, cz = pz;
        if (tn < tile_end) {
            locate(tn);
            prefetch(tn, px, py, pz);
        }
        if constexpr (FIXL >= 0) {
            batch_tile<FIXL, GN>(cur, lt, buf, tabs.t, lane, cx, cy, cz);
        } else {
            switch (cur.L) {
#define SPH_CASE(LL) \
    case LL:         \
        batch_tile<LL, -1>(cur, lt, buf, tabs.t, lane, cx, cy, cz); \
        break;
                SPH_CASE(0) SPH_CASE(1) SPH_CASE(2) SPH_CASE(3) SPH_CASE(4) SPH_CASE(5) SPH_CASE(6) SPH_CASE(7)
                SPH_CASE(8) SPH_CASE(9) SPH_CASE(10) SPH_CASE(11) SPH_CASE(12) SPH_CASE(13) SPH_CASE(14)
                SPH_CASE(15) SPH_CASE(16)
#undef SPH_CASE
                default:
                    break;
            }
        }
        t = tn;
    }
    bulk_wait_all();  // every lane: 4-lane tiles of some l_max send one row per lane
}

// Host tables of Eq. iter-q / iter-deri for l <= 16 as a kernel parameter.
const BatchTabs& batch_tabs();

// One launch of a batch kernel over a range of sets / tiles.
struct BatchClassArgs {
    const BatchSet* sets;
    int set_begin, set_end;
    int64_t tile_begin, tile_end;
    unsigned long long* counter;
    int per_warp_bytes;
    int W;       // warps per block
    int blocks;  // persistent grid
    size_t smem;
    void* stream;
    int* occ_out;  // non-null: set the shared-memory attribute, return the occupancy, no launch
    int gn;        // class flags grad + 2 * norm (per-class launches), -1: from each set
};

// Shared-memory attribute / occupancy query (occ_out != nullptr) or launch of
// the FIXL kernel; returns a cudaError_t value.
template <int FIXL, int GN>
int batch_kernel_run(const BatchClassArgs& a) {
    auto kern = batch_kernel_t<FIXL, GN>;
    if (a.occ_out) {
        cudaError_t e = ensure_smem(kern, a.smem);
        if (e != cudaSuccess) return int(e);
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, reinterpret_cast<const void*>(kern), 32 * a.W,
                                                          a.smem) != cudaSuccess) {
            cudaGetLastError();
            occ = 1;
        }
        *a.occ_out = std::max(occ, 1);
        return 0;
    }
    kern<<<a.blocks, 32 * a.W, a.smem, static_cast<cudaStream_t>(a.stream)>>>(
        a.sets, a.set_begin, a.set_end, a.tile_begin, a.tile_end, a.counter, a.per_warp_bytes, batch_tabs());
    return int(cudaGetLastError());
}

}  // namespace sph
