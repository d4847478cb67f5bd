// Ragged batches in persistent launches.
//
// Many point sets (e.g. the neighbour lists of many structures), each with its
// own l_max <= SPH_MAX_L_POINT, are evaluated by persistent kernels: every
// warp pulls work tiles from a device counter, finds the tile's set by a
// forward scan over the per-set tile prefix sums, and runs the POINT recursion
// for that set's l_max. Tiles are sized per set so that one tile's outputs fill
// a shared-memory budget per warp: small l_max sets get up to 256-point tiles
// (each lane computes several points), large ones fewer than 32 points (idle
// lanes cost arithmetic, which is cheap here, not bandwidth). Sets are ordered
// by decreasing l_max.
//
// Two plan modes:
//  * one launch per l_max class (SPH_BATCH_PER_LMAX, the default): the sets of
//    one l_max form a contiguous tile range run by a kernel compiled for that
//    l_max only, with its own tile counter and a shared-memory size fitted to
//    that class's tile -- no branch over l_max in the hot loop, one body in the
//    instruction cache, occupancy set per class;
//  * one launch for the whole batch (SPH_BATCH_ONE_LAUNCH): a switch over the
//    compile-time l_max bodies, shared memory sized for the largest tile.
// The work list and counters live in device memory owned by the plan;
// executing the plan is one counter reset plus the launches on the caller's
// stream, which can be captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <numeric>
#include <vector>

#include "sph_batch.cuh"

namespace sph {

const BatchTabs& batch_tabs() {
    static const BatchTabs t{make_point_tabs<16, float, false>()};
    return t;
}

// One launch of a plan: the sets [set_begin, set_end) and their tiles.
struct BatchLaunch {
    int L = -1;   // l_max of every set in the range, or -1 (all l_max, one launch)
    int gn = -1;  // gradients + 2 * normalized of every set in the range, or -1
    int set_begin = 0, set_end = 0;
    int64_t tile_begin = 0, tile_end = 0;
    int per_warp_bytes = 0;
    int W = 1;  // warps per block
    int blocks = 1;
    size_t smem = 0;
};

int batch_run(const BatchLaunch& b, const BatchSet* sets, unsigned long long* counter, void* stream, int* occ_out) {
    BatchClassArgs a{sets, b.set_begin, b.set_end, b.tile_begin, b.tile_end, counter, b.per_warp_bytes, b.W,
                     b.blocks, b.smem, stream, occ_out, b.gn};
    return b.L >= 0 ? batch_class_fn(b.L)(a) : batch_kernel_run<-1, -1>(a);
}

}  // namespace sph

using namespace sph;

struct sph_batch_plan {
    int device = -1;
    int nsets = 0;
    int mode = SPH_BATCH_PER_LMAX;
    int64_t total_points = 0;
    int64_t total_tiles = 0;
    BatchSet* d_sets = nullptr;
    unsigned long long* d_counter = nullptr;  // one counter per launch
    std::vector<BatchLaunch> launches;
};

namespace {

int tile_mult4(int L) {
    const int K = (L + 1) * (L + 1);
    const int r = (K * 4) % 16;
    return r == 0 ? 1 : 16 / (r == 8 ? 8 : 4);
}

}  // namespace

extern "C" {

int sphericart_batch_plan_create_ex(const sph_batch_set* sets, int nsets, const sph_launch* launch, int mode,
                                    sph_batch_plan** plan_out) {
    if (mode != SPH_BATCH_PER_LMAX && mode != SPH_BATCH_ONE_LAUNCH) {
        set_error("batch_plan_create: mode=%d is not an sph_batch_mode", mode);
        return SPH_EINVAL;
    }
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

    // PER_LMAX without an explicit launch shape: every l_max class takes the
    // tile size and warps per block of the single-set POINT kernel for that
    // l_max (tuned if installed, else its default); otherwise one per-warp
    // budget for all sets.
    const bool class_shapes = mode == SPH_BATCH_PER_LMAX && lau.points_per_tile == 0 && lau.warps_per_block == 0;
    std::vector<int> order(nsets);
    std::iota(order.begin(), order.end(), 0);
    // sets ordered by decreasing l_max, then by (gradients, normalized): every
    // class of equal (l_max, gradients, normalized) is a contiguous range
    auto gn_of = [&](int i) { return (sets[i].dsph ? 1 : 0) + (sets[i].normalized ? 2 : 0); };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (sets[a].l_max != sets[b].l_max) return sets[a].l_max > sets[b].l_max;
        return gn_of(a) < gn_of(b);
    });
    std::vector<BatchSet> hs;
    hs.reserve(nsets);
    std::vector<int> bytes_of(nsets);
    int64_t tiles = 0, points = 0;
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
        if (class_shapes) P = point_fwd_shape(L, grad).points_per_tile;  // a multiple of mult, <= 32
        bytes_of[hs.size()] = int(align16(size_t(P) * V * 4) + (grad ? align16(size_t(P) * D * 4) : 0));
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
    // The launches: one per run of equal (l_max, gradients, normalized) (sets
    // are sorted), or one for all.
    auto gn_hs = [&](int i) { return (hs[i].dsph ? 1 : 0) + (hs[i].norm ? 2 : 0); };
    std::vector<BatchLaunch> launches;
    for (int i = 0; i < nsets;) {
        int j = i;
        int bytes = 0;
        while (j < nsets && (mode == SPH_BATCH_ONE_LAUNCH || (hs[j].L == hs[i].L && gn_hs(j) == gn_hs(i))))
            bytes = std::max(bytes, bytes_of[j++]);
        BatchLaunch bl;
        bl.L = mode == SPH_BATCH_ONE_LAUNCH ? -1 : hs[i].L;
        bl.gn = mode == SPH_BATCH_ONE_LAUNCH ? -1 : gn_hs(i);
        bl.set_begin = i;
        bl.set_end = j;
        bl.tile_begin = hs[i].tile_begin;
        bl.tile_end = (j < nsets) ? hs[j].tile_begin : tiles;
        bl.per_warp_bytes = bytes;
        bl.W = class_shapes ? point_fwd_shape(hs[i].L, hs[i].dsph ? 1 : 0).warps_per_block : W;
        bl.smem = size_t(bl.W) * size_t(bytes);
        if (bl.smem > size_t(max_smem_optin())) {
            set_error("batch plan needs %zu bytes of shared memory per block", bl.smem);
            return SPH_EINVAL;
        }
        if (bl.tile_end > bl.tile_begin) launches.push_back(bl);
        i = j;
    }
    auto* plan = new sph_batch_plan();
    plan->device = dev;
    plan->nsets = nsets;
    plan->mode = mode;
    plan->total_points = points;
    plan->total_tiles = tiles;
    const size_t ncount = std::max<size_t>(1, launches.size());
    if (cudaMalloc(&plan->d_sets, sizeof(BatchSet) * hs.size()) != cudaSuccess ||
        cudaMalloc(&plan->d_counter, sizeof(unsigned long long) * ncount) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(plan->d_sets);
        delete plan;
        set_error("batch plan: device allocation failed");
        return SPH_ENOMEM;
    }
    cudaError_t e = cudaMemcpy(plan->d_sets, hs.data(), sizeof(BatchSet) * hs.size(), cudaMemcpyHostToDevice);
    for (BatchLaunch& bl : launches) {  // shared-memory attribute and persistent grid of every launch
        if (e != cudaSuccess) break;
        int occ = 1;
        e = static_cast<cudaError_t>(batch_run(bl, plan->d_sets, plan->d_counter, nullptr, &occ));
        const int bps = lau.blocks_per_sm > 0 ? std::min(lau.blocks_per_sm, occ) : occ;
        const int64_t want = (bl.tile_end - bl.tile_begin + bl.W - 1) / bl.W;
        bl.blocks = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(bps) * sm_count())));
    }
    if (e != cudaSuccess) {
        cudaFree(plan->d_sets);
        cudaFree(plan->d_counter);
        delete plan;
        set_error("batch plan: %s", cudaGetErrorString(e));
        return SPH_ECUDA;
    }
    plan->launches = std::move(launches);
    *plan_out = plan;
    return SPH_OK;
}

int sphericart_batch_plan_create(const sph_batch_set* sets, int nsets, const sph_launch* launch,
                                 sph_batch_plan** plan_out) {
    return sphericart_batch_plan_create_ex(sets, nsets, launch, SPH_BATCH_PER_LMAX, plan_out);
}

int sphericart_batch_execute(const sph_batch_plan* plan, void* stream) {
    if (!plan) {
        set_error("batch_execute: plan is NULL");
        return SPH_EINVAL;
    }
    if (plan->launches.empty()) return SPH_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e =
        cudaMemsetAsync(plan->d_counter, 0, sizeof(unsigned long long) * plan->launches.size(), st);
    for (size_t i = 0; i < plan->launches.size() && e == cudaSuccess; ++i)
        e = static_cast<cudaError_t>(
            batch_run(plan->launches[i], plan->d_sets, plan->d_counter + i, stream, nullptr));
    if (e != cudaSuccess) {
        set_error("batch_execute: %s", cudaGetErrorString(e));
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
    BatchLaunch bl;  // one launch for every l_max, as SPH_BATCH_ONE_LAUNCH
    bl.W = W;
    bl.set_begin = 0;
    bl.set_end = nsets;
    bl.tile_begin = 0;
    bl.tile_end = tiles;
    bl.per_warp_bytes = max_bytes;
    bl.smem = smem;
    int occ = 1;
    if (e == cudaSuccess) e = static_cast<cudaError_t>(batch_run(bl, d_sets, d_counter, stream, &occ));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("batch_compute_noalloc: %s", cudaGetErrorString(e));
        return SPH_ECUDA;
    }
    const int bps = lau.blocks_per_sm > 0 ? std::min(lau.blocks_per_sm, occ) : occ;
    bl.blocks = int(std::max<int64_t>(1, std::min<int64_t>((tiles + W - 1) / W, int64_t(bps) * sm_count())));
    e = static_cast<cudaError_t>(batch_run(bl, d_sets, d_counter, stream, nullptr));
    if (e != cudaSuccess) {
        set_error("batch_compute_noalloc launch: %s", cudaGetErrorString(e));
        return SPH_ECUDA;
    }
    return SPH_OK;
}
