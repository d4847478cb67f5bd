// Ragged batches in ONE persistent launch.
//
// Many point sets (e.g. the neighbour lists of many structures), each with its
// own l_max <= SPH_MAX_L_POINT, are evaluated by a single kernel: every warp
// pulls work tiles from a device counter, finds the tile's set by binary
// search over the per-set tile prefix sums, and runs the POINT recursion for
// that set's l_max (a switch over compile-time l_max). Tiles are sized per set
// so that one tile's outputs fill a fixed shared-memory budget per warp: small
// l_max sets get up to 256-point tiles (each lane computes several points),
// large ones fewer than 32 points (idle lanes cost arithmetic, which is cheap
// here, not bandwidth). Sets are ordered by decreasing l_max so the expensive
// tiles start first and warps mostly run the same l_max body together.
//
// The work list lives in device memory owned by the plan; executing the plan
// is a counter reset plus one launch on the caller's stream, which can be
// captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <numeric>
#include <vector>

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

template <int K>
struct BatchVis {
    float* rv;
    float* rd;  // nullptr: values only
    float ux, uy, uz, ir;
    int norm;
    __device__ __forceinline__ void emit(int l, int k, Deriv<float> d) {
        rv[k] = d.v;
        if (rd) {
            if (norm) normalize_deriv<false>(d, l, ux, uy, uz, ir);
            rd[k] = d.gx;
            rd[K + k] = d.gy;
            rd[2 * K + k] = d.gz;
        }
    }
};

template <int L>
__device__ __forceinline__ void batch_tile(const BatchSet& s, int64_t t, unsigned char* buf,
                                           const PointTabs<16, float, false>& tb, int lane, float px, float py,
                                           float pz) {
    constexpr int K = (L + 1) * (L + 1);
    using RS = RowStride<L>;
    const int P = s.P;
    const int64_t p0 = t * P;
    const int cnt = int(min(int64_t(P), s.n - p0));
    float* s_v = reinterpret_cast<float*>(buf);
    float* s_d = reinterpret_cast<float*>(buf + align16(size_t(P) * RS::V * 4));
    const bool grad = s.dsph != nullptr;
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
        if (s.norm) {
            unit_point(x, y, z, r2, ir);
        } else {
            r2 = x * x + y * y + z * z;
        }
        BatchVis<K> vis{s_v + size_t(row) * RS::V, grad ? s_d + size_t(row) * RS::D : nullptr, x, y, z, ir, s.norm};
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

__global__ void __launch_bounds__(256) batch_kernel(const BatchSet* __restrict__ sets, int nsets,
                                                    int64_t total_tiles, unsigned long long* __restrict__ counter,
                                                    int per_warp_bytes, const __grid_constant__ BatchTabs tabs) {
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
    int si = 0;
    BatchSet s = sets[0];
    int64_t s_end = (nsets > 1) ? sets[1].tile_begin : total_tiles;
    auto locate = [&](int64_t t) {  // forward scan: t never decreases for a warp
        while (t >= s_end && si + 1 < nsets) {
            ++si;
            s = sets[si];
            s_end = (si + 1 < nsets) ? sets[si + 1].tile_begin : total_tiles;
        }
    };
    auto prefetch = [&](int64_t t, float& x, float& y, float& z) {
        const int64_t p = (t - s.tile_begin) * s.P + lane;
        if (lane < s.P && p < s.n) {
            x = s.xyz[3 * p];
            y = s.xyz[3 * p + 1];
            z = s.xyz[3 * p + 2];
        }
    };
    int64_t t = int64_t(run) * kBatchRun;
    float px = 0.f, py = 0.f, pz = 0.f;
    if (t < total_tiles) {
        locate(t);
        prefetch(t, px, py, pz);
    }
    while (t < total_tiles) {
        // next tile: the following one in this run, else the first of the next run
        int64_t tn = t + 1;
        if (tn % kBatchRun == 0) {
            const unsigned long long r = __shfl_sync(0xffffffffu, nrun, 0);
            tn = int64_t(r) * kBatchRun;
            if (lane == 0) nrun = atomicAdd(counter, 1ull);
        }
        const BatchSet cur = s;
        const int64_t lt = t - cur.tile_begin;
        const float cx = px, cy = py, cz = pz;
        if (tn < total_tiles) {
            locate(tn);
            prefetch(tn, px, py, pz);
        }
        switch (cur.L) {
#define SPH_CASE(LL) \
    case LL:         \
        batch_tile<LL>(cur, lt, buf, tabs.t, lane, cx, cy, cz); \
        break;
            SPH_CASE(0) SPH_CASE(1) SPH_CASE(2) SPH_CASE(3) SPH_CASE(4) SPH_CASE(5) SPH_CASE(6) SPH_CASE(7)
            SPH_CASE(8) SPH_CASE(9) SPH_CASE(10) SPH_CASE(11) SPH_CASE(12) SPH_CASE(13) SPH_CASE(14)
            SPH_CASE(15) SPH_CASE(16)
#undef SPH_CASE
            default:
                break;
        }
        t = tn;
    }
    if (lane == 0) bulk_wait_all();
}

}  // namespace sph

using namespace sph;

struct sph_batch_plan {
    int device = -1;
    int nsets = 0;
    int64_t total_points = 0;
    int64_t total_tiles = 0;
    BatchSet* d_sets = nullptr;
    unsigned long long* d_counter = nullptr;
    int warps_per_block = 1;
    int blocks = 1;
    int per_warp_bytes = 0;
    size_t smem = 0;
};

namespace {

const BatchTabs& batch_tabs() {
    static const BatchTabs t{make_point_tabs<16, float, false>()};
    return t;
}

int tile_mult4(int L) {
    const int K = (L + 1) * (L + 1);
    const int r = (K * 4) % 16;
    return r == 0 ? 1 : 16 / (r == 8 ? 8 : 4);
}

}  // namespace

extern "C" {

int sphericart_batch_plan_create(const sph_batch_set* sets, int nsets, const sph_launch* launch,
                                 sph_batch_plan** plan_out) {
    if (!plan_out || !sets || nsets <= 0) {
        set_error("batch_plan_create: sets, nsets > 0 and plan are required");
        return SPH_EINVAL;
    }
    *plan_out = nullptr;
    for (int i = 0; i < nsets; ++i) {
        const sph_batch_set& s = sets[i];
        if (s.n < 0 || s.l_max < 0 || s.l_max > SPH_MAX_L_POINT) {
            set_error("batch set %d: n=%lld must be >= 0 and l_max=%d in [0,%d]", i, static_cast<long long>(s.n),
                      s.l_max, SPH_MAX_L_POINT);
            return SPH_EINVAL;
        }
        if (s.n > 0 && (!s.xyz || !s.sph)) {
            set_error("batch set %d: xyz and sph must be non-NULL", i);
            return SPH_EINVAL;
        }
        if ((reinterpret_cast<uintptr_t>(s.xyz) | reinterpret_cast<uintptr_t>(s.sph) |
             reinterpret_cast<uintptr_t>(s.dsph)) % 4 != 0) {
            set_error("batch set %d: buffers must be 4-byte aligned", i);
            return SPH_EINVAL;
        }
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        set_error("batch_plan_create: no usable CUDA device");
        return SPH_ECUDA;
    }
    sph_launch lau = launch ? *launch : sph_launch{0, 0, 0, 0};
    const int W = lau.warps_per_block > 0 ? lau.warps_per_block : 1;
    if (W > 8 || lau.points_per_tile < 0 || lau.points_per_tile > 160) {
        set_error("warps_per_block=%d must be in [1,8], points_per_tile (budget rows) in [0,160]", W);
        return SPH_EINVAL;
    }
    // Per-warp shared-memory budget: one 32-point l_max = 8 value+gradient tile.
    const int budget = lau.points_per_tile > 0 ? lau.points_per_tile * 1296 : 32 * 1296;

    std::vector<int> order(nsets);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sets[a].l_max > sets[b].l_max; });
    std::vector<BatchSet> hs;
    hs.reserve(nsets);
    int64_t tiles = 0, points = 0;
    int max_bytes = 0;
    for (int oi : order) {
        const sph_batch_set& s = sets[oi];
        const int L = s.l_max;
        const int K = (L + 1) * (L + 1);
        const int grad = s.dsph ? 1 : 0;
        const int V = (K % 2 == 0) ? K + 1 : K, D = (K % 2 == 0) ? 3 * K + 1 : 3 * K;  // smem row strides
        const int row = 4 * (V + (grad ? D : 0));
        const int mult = tile_mult4(L);
        int P = std::min(kBatchMaxTile, std::max(1, budget / row));
        P = std::max(mult, P / mult * mult);
        const int bytes = int(align16(size_t(P) * V * 4) + (grad ? align16(size_t(P) * D * 4) : 0));
        max_bytes = std::max(max_bytes, bytes);
        BatchSet b{};
        b.xyz = s.xyz;
        b.sph = s.sph;
        b.dsph = s.dsph;
        b.n = s.n;
        b.tile_begin = tiles;
        b.L = L;
        b.P = P;
        b.norm = s.normalized ? 1 : 0;
        b.bulk = (reinterpret_cast<uintptr_t>(s.sph) % 16 == 0 && reinterpret_cast<uintptr_t>(s.dsph) % 16 == 0) ? 1 : 0;
        tiles += (s.n + P - 1) / P;
        points += s.n;
        hs.push_back(b);
    }
    const size_t smem = size_t(W) * size_t(max_bytes);
    if (smem > size_t(max_smem_optin())) {
        set_error("batch plan needs %zu bytes of shared memory per block", smem);
        return SPH_EINVAL;
    }
    auto* plan = new sph_batch_plan();
    plan->device = dev;
    plan->nsets = nsets;
    plan->total_points = points;
    plan->total_tiles = tiles;
    plan->warps_per_block = W;
    plan->per_warp_bytes = max_bytes;
    plan->smem = smem;
    if (cudaMalloc(&plan->d_sets, sizeof(BatchSet) * hs.size()) != cudaSuccess ||
        cudaMalloc(&plan->d_counter, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(plan->d_sets);
        delete plan;
        set_error("batch plan: device allocation failed");
        return SPH_ENOMEM;
    }
    cudaError_t e = cudaMemcpy(plan->d_sets, hs.data(), sizeof(BatchSet) * hs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = ensure_smem(batch_kernel, smem);
    if (e != cudaSuccess) {
        cudaFree(plan->d_sets);
        cudaFree(plan->d_counter);
        delete plan;
        set_error("batch plan: %s", cudaGetErrorString(e));
        return SPH_ECUDA;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, reinterpret_cast<const void*>(batch_kernel), 32 * W,
                                                      smem) != cudaSuccess)
        occ = 1;
    const int bps = lau.blocks_per_sm > 0 ? std::min(lau.blocks_per_sm, std::max(occ, 1)) : std::max(occ, 1);
    const int64_t want = (tiles + W - 1) / W;
    plan->blocks = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(bps) * sm_count())));
    *plan_out = plan;
    return SPH_OK;
}

int sphericart_batch_execute(const sph_batch_plan* plan, void* stream) {
    if (!plan) {
        set_error("batch_execute: plan is NULL");
        return SPH_EINVAL;
    }
    if (plan->total_tiles == 0) return SPH_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(plan->d_counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) {
        set_error("batch_execute: %s", cudaGetErrorString(e));
        return SPH_ECUDA;
    }
    batch_kernel<<<plan->blocks, 32 * plan->warps_per_block, plan->smem, st>>>(
        plan->d_sets, plan->nsets, plan->total_tiles, plan->d_counter, plan->per_warp_bytes, batch_tabs());
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("batch_execute launch: %s", cudaGetErrorString(e));
        return SPH_ECUDA;
    }
    return SPH_OK;
}

int sphericart_batch_plan_destroy(sph_batch_plan* plan) {
    if (!plan) return SPH_OK;
    int cur = -1;
    cudaGetDevice(&cur);
    if (plan->device >= 0) cudaSetDevice(plan->device);
    cudaDeviceSynchronize();
    cudaFree(plan->d_sets);
    cudaFree(plan->d_counter);
    if (cur >= 0) cudaSetDevice(cur);
    delete plan;
    return SPH_OK;
}

int sphericart_batch_plan_info(const sph_batch_plan* plan, int64_t* total_points, int64_t* total_tiles) {
    if (!plan) {
        set_error("batch_plan_info: plan is NULL");
        return SPH_EINVAL;
    }
    if (total_points) *total_points = plan->total_points;
    if (total_tiles) *total_tiles = plan->total_tiles;
    return SPH_OK;
}

}  // extern "C"

// ----------------------------------------------------------- no-allocation
// A second way to run a ragged batch, for callers that cannot allocate
// device memory: code running under a memory manager that owns every device
// byte (a serving runtime with a fixed arena, a framework's caching
// allocator that must not be bypassed), or code on a latency-critical path
// where cudaMalloc's implicit device synchronisation is not acceptable.
//
// The work list and the tile counter live in the file-scope array below
// instead of a plan's cudaMalloc'd buffers. Every GPU that loads this
// library holds kNoAllocScratchBytes (about 225 KB) of it until the process
// exits. All calls on a device share it and it keeps the last call's
// contents; the counter is cleared on every call.
namespace sph {
namespace {

constexpr int kNoAllocMaxSets = 4096;
constexpr size_t kNoAllocCounterBytes = 256;  // counter, padded to keep the sets 256-byte aligned
constexpr size_t kNoAllocScratchBytes = kNoAllocCounterBytes + sizeof(BatchSet) * kNoAllocMaxSets;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;                            // guards the two arrays below
void* g_noalloc_dev_ptr[kNoAllocMaxDevices] = {};   // device address of g_noalloc_scratch, per device
BatchSet g_noalloc_host[kNoAllocMaxSets];           // host staging of the work list

}  // namespace
}  // namespace sph

extern "C" int sphericart_batch_compute_noalloc(const sph_batch_set* sets, int nsets, const sph_launch* launch,
                                                void* stream) {
    using namespace sph;
    if (!sets || nsets <= 0) {
        set_error("batch_compute_noalloc: sets and nsets > 0 are required");
        return SPH_EINVAL;
    }
    if (nsets > kNoAllocMaxSets) {
        set_error("batch_compute_noalloc: nsets=%d exceeds the static work-list capacity of %d sets", nsets,
                  kNoAllocMaxSets);
        return SPH_EINVAL;
    }
    for (int i = 0; i < nsets; ++i) {
        const sph_batch_set& s = sets[i];
        if (s.n < 0 || s.l_max < 0 || s.l_max > SPH_MAX_L_POINT) {
            set_error("batch set %d: n=%lld must be >= 0 and l_max=%d in [0,%d]", i, static_cast<long long>(s.n),
                      s.l_max, SPH_MAX_L_POINT);
            return SPH_EINVAL;
        }
        if (s.n > 0 && (!s.xyz || !s.sph)) {
            set_error("batch set %d: xyz and sph must be non-NULL", i);
            return SPH_EINVAL;
        }
        if ((reinterpret_cast<uintptr_t>(s.xyz) | reinterpret_cast<uintptr_t>(s.sph) |
             reinterpret_cast<uintptr_t>(s.dsph)) % 4 != 0) {
            set_error("batch set %d: buffers must be 4-byte aligned", i);
            return SPH_EINVAL;
        }
    }
    const sph_launch lau = launch ? *launch : sph_launch{0, 0, 0, 0};
    const int W = lau.warps_per_block > 0 ? lau.warps_per_block : 1;
    if (W > 8 || lau.points_per_tile < 0 || lau.points_per_tile > 160 || lau.blocks_per_sm < 0) {
        set_error("batch_compute_noalloc: bad launch shape");
        return SPH_EINVAL;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        cudaGetLastError();
        set_error("batch_compute_noalloc: no usable CUDA device");
        return SPH_ECUDA;
    }
    const int budget = lau.points_per_tile > 0 ? lau.points_per_tile * 1296 : 32 * 1296;

    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    // Set-up, once per device, with that device current: the device address
    // of the static array (host code must not use the symbol itself).
    if (!g_noalloc_dev_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            set_error("batch_compute_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return SPH_ECUDA;
        }
        g_noalloc_dev_ptr[dev] = p;
    }
    unsigned char* base = static_cast<unsigned char*>(g_noalloc_dev_ptr[dev]);
    unsigned long long* d_counter = reinterpret_cast<unsigned long long*>(base);
    BatchSet* d_sets = reinterpret_cast<BatchSet*>(base + kNoAllocCounterBytes);

    // Work list in host staging: sets grouped by decreasing l_max (a
    // counting sort, no allocation), tile prefix sums as in the plans.
    int count[SPH_MAX_L_POINT + 2] = {0};
    for (int i = 0; i < nsets; ++i) ++count[SPH_MAX_L_POINT - sets[i].l_max + 1];
    for (int b = 1; b <= SPH_MAX_L_POINT + 1; ++b) count[b] += count[b - 1];
    int64_t tiles = 0;
    int max_bytes = 0;
    for (int i = 0; i < nsets; ++i) {
        const sph_batch_set& s = sets[i];
        const int L = s.l_max;
        const int K = (L + 1) * (L + 1);
        const int grad = s.dsph ? 1 : 0;
        const int V = (K % 2 == 0) ? K + 1 : K, D = (K % 2 == 0) ? 3 * K + 1 : 3 * K;  // smem row strides
        const int row = 4 * (V + (grad ? D : 0));
        const int mult = tile_mult4(L);
        int P = std::min(kBatchMaxTile, std::max(1, budget / row));
        P = std::max(mult, P / mult * mult);
        const int bytes = int(align16(size_t(P) * V * 4) + (grad ? align16(size_t(P) * D * 4) : 0));
        max_bytes = std::max(max_bytes, bytes);
        BatchSet& b = g_noalloc_host[count[SPH_MAX_L_POINT - L]++];
        b = BatchSet{};
        b.xyz = s.xyz;
        b.sph = s.sph;
        b.dsph = s.dsph;
        b.n = s.n;
        b.L = L;
        b.P = P;
        b.norm = s.normalized ? 1 : 0;
        b.bulk = (reinterpret_cast<uintptr_t>(s.sph) % 16 == 0 && reinterpret_cast<uintptr_t>(s.dsph) % 16 == 0) ? 1 : 0;
    }
    for (int i = 0; i < nsets; ++i) {
        g_noalloc_host[i].tile_begin = tiles;
        tiles += (g_noalloc_host[i].n + g_noalloc_host[i].P - 1) / g_noalloc_host[i].P;
    }
    if (tiles == 0) return SPH_OK;
    const size_t smem = size_t(W) * size_t(max_bytes);
    if (smem > size_t(max_smem_optin())) {
        set_error("batch_compute_noalloc: needs %zu bytes of shared memory per block", smem);
        return SPH_EINVAL;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // From pageable host memory the copy has consumed g_noalloc_host when it
    // returns, so the staging may be reused by the next call.
    cudaError_t e = cudaMemcpyAsync(d_sets, g_noalloc_host, sizeof(BatchSet) * size_t(nsets), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = ensure_smem(batch_kernel, smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("batch_compute_noalloc: %s", cudaGetErrorString(e));
        return SPH_ECUDA;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, reinterpret_cast<const void*>(batch_kernel), 32 * W,
                                                      smem) != cudaSuccess) {
        cudaGetLastError();
        occ = 1;
    }
    const int bps = lau.blocks_per_sm > 0 ? std::min(lau.blocks_per_sm, std::max(occ, 1)) : std::max(occ, 1);
    const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((tiles + W - 1) / W, int64_t(bps) * sm_count())));
    batch_kernel<<<blocks, 32 * W, smem, st>>>(d_sets, nsets, tiles, d_counter, max_bytes, batch_tabs());
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("batch_compute_noalloc launch: %s", cudaGetErrorString(e));
        return SPH_ECUDA;
    }
    return SPH_OK;
}
