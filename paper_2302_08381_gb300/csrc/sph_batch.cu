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
#include <map>
#include <mutex>
#include <tuple>
#include <numeric>
#include <vector>

#include "sph_batch.cuh"
#include "sph_batch_one.cuh"

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

namespace {

int tile_mult4(int L) {
    const int K = (L + 1) * (L + 1);
    const int r = (K * 4) % 16;
    return r == 0 ? 1 : 16 / (r == 8 ? 8 : 4);
}

}  // namespace

// ------------------------------------------------------------ one launch
// Shapes of the one-launch kernel for one flag class and one chunk of
// descriptors: per l_max the single-set POINT tile (tuned if installed) or,
// with `budget_rows` > 0, the tile that fits that many l_max = 8
// value+gradient rows (1,296 bytes each); the warps of a block that run that
// class (as many staging buffers as the block's shared memory holds, at most
// `max_warps`); the block's warps and staging bytes (the largest class).
struct OneShapes {
    OneClass cls[SPH_MAX_L_POINT + 1];
    int staging_bytes = 0;
    int W = 1;
};

int one_shapes(int grad, const sph_launch& lau, int nsets, OneShapes* out) {
    OneShapes o;
    const int max_warps = lau.warps_per_block > 0 ? std::min(lau.warps_per_block, kOneMaxWarps) : kOneMaxWarps;
    const size_t optin = size_t(max_smem_optin());
    const size_t reserve = one_table_bytes(nsets) + 1024;  // the work table, static shared memory
    if (optin <= reserve) {
        set_error("batch one-launch: no shared memory left for staging");
        return SPH_EINVAL;
    }
    const size_t S = (optin - reserve) / 128 * 128;
    for (int L = 0; L <= SPH_MAX_L_POINT; ++L) {
        const int K = (L + 1) * (L + 1);
        const int V = (K % 2 == 0) ? K + 1 : K;
        const int D = (K % 2 == 0) ? 3 * K + 1 : 3 * K;
        const int mult = tile_mult4(L);
        int P;
        if (lau.points_per_tile > 0) {
            const int row = 4 * (V + (grad ? D : 0));
            P = std::min(kOneMaxTile, lau.points_per_tile * 1296 / row) / mult * mult;
        } else {
            P = point_fwd_shape(L, grad).points_per_tile;
        }
        P = std::max(P, mult);
        size_t bytes = align128(size_t(P) * V * 4) + (grad ? align128(size_t(P) * D * 4) : 0);
        if (grad && L >= kPoint4MinL) {  // 4 lanes per point (one_four): 8-point tiles
            P = 8;
            bytes = point4_tile_bytes(L, 4, P, 128);
        }
        const int W = int(std::min<size_t>(size_t(max_warps), S / bytes));
        if (W < 1) {
            set_error("batch one-launch: a %d-point tile at l_max %d needs %zu bytes of shared memory", P, L, bytes);
            return SPH_EINVAL;
        }
        o.cls[L] = OneClass{P, int(bytes), W, 0};
        o.W = std::max(o.W, W);
        o.staging_bytes = std::max(o.staging_bytes, int(size_t(W) * bytes));
    }
    o.staging_bytes = std::max(o.staging_bytes, int(align128(one_scratch_bytes(nsets))));
    *out = o;
    return SPH_OK;
}

// Resolved launch of one chunk of <= kOneMaxSets descriptors.
struct OneRec {
    int gn = 0;
    int off = 0;  // first descriptor of the chunk
    int cnt = 0;
    int blocks = 1;
    size_t smem = 0;
    OneShapes sh;
};

// Shapes, shared memory and grid of a chunk; returns SPH_OK or an error code
// with the message set.
int one_resolve(OneRec& r, const sph_launch& lau) {
    int st = one_shapes(r.gn & 1, lau, r.cnt, &r.sh);
    if (st != SPH_OK) return st;
    r.smem = size_t(r.sh.staging_bytes) + one_table_bytes(r.cnt);
    // Shared-memory attribute and occupancy, once per (device, flags, warps,
    // bytes): later calls (e.g. under stream capture) make no such query.
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, size_t>, int> cache;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        set_error("batch one-launch: no usable CUDA device");
        return SPH_ECUDA;
    }
    int occ = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        const auto key = std::make_tuple(dev, r.gn, r.sh.W, r.smem);
        auto it = cache.find(key);
        if (it != cache.end()) {
            occ = it->second;
        } else {
            OneArgs q{};
            q.W = r.sh.W;
            q.smem = r.smem;
            q.occ_out = &occ;
            const int e = batch_one_fn(r.gn)(q);
            if (e != 0) {
                set_error("batch one-launch: %s", cudaGetErrorString(static_cast<cudaError_t>(e)));
                return SPH_ECUDA;
            }
            cache[key] = occ;
        }
    }
    if (occ <= 0) {
        set_error("batch one-launch: a block of %d warps with %zu bytes of shared memory does not fit an SM",
                  r.sh.W, r.smem);
        return SPH_EINVAL;
    }
    const int bps = lau.blocks_per_sm > 0 ? std::min(lau.blocks_per_sm, occ) : occ;
    r.blocks = std::max(1, bps * sm_count());
    return SPH_OK;
}

int one_launch(const OneRec& r, const sph_batch_set* desc, OneCounter* ctr, uint32_t* status, void* stream) {
    OneArgs a{};
    a.desc = desc + r.off;
    a.nsets = r.cnt;
    a.ctr = ctr;
    a.staging_bytes = r.sh.staging_bytes;
    a.W = r.sh.W;
    a.blocks = r.blocks;
    a.smem = r.smem;
    a.cls = r.sh.cls;
    a.status = status;
    a.stream = stream;
    return batch_one_fn(r.gn)(a);
}

bool one_launch_shape_ok(const sph_launch& lau) {
    if (lau.warps_per_block < 0 || lau.warps_per_block > kOneMaxWarps || lau.points_per_tile < 0 ||
        lau.points_per_tile > 160 || lau.blocks_per_sm < 0 || lau.blocks_per_sm > 32) {
        set_error("batch launch: warps_per_block in [0,%d], points_per_tile (budget rows) in [0,160], "
                  "blocks_per_sm in [0,32]", kOneMaxWarps);
        return false;
    }
    return true;
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
    // SPH_BATCH_ONE_LAUNCH: descriptors grouped by flag class, one launch per
    // chunk of <= kOneMaxSets sets of one class (usually a single launch)
    sph_batch_set* d_desc = nullptr;
    OneCounter* d_one_ctr = nullptr;
    std::vector<OneRec> one;
};

namespace {

int gn_of_set(const sph_batch_set& s) { return (s.dsph ? 1 : 0) + (s.normalized ? 2 : 0); }

// SPH_BATCH_ONE_LAUNCH plans: the descriptors (validated by the caller)
// grouped by flag class in a device array, one launch per chunk of one class.
int plan_create_one(const sph_batch_set* sets, int nsets, const sph_launch& lau, int dev, sph_batch_plan** out) {
    if (!one_launch_shape_ok(lau)) return SPH_EINVAL;
    auto* plan = new sph_batch_plan();
    plan->device = dev;
    plan->nsets = nsets;
    plan->mode = SPH_BATCH_ONE_LAUNCH;
    bool need[4] = {false, false, false, false};
    for (int i = 0; i < nsets; ++i) need[gn_of_set(sets[i])] = true;
    std::vector<sph_batch_set> hs;
    hs.reserve(nsets);
    for (int g = 0; g < 4; ++g) {
        if (!need[g]) continue;
        const int off0 = int(hs.size());
        for (int i = 0; i < nsets; ++i)
            if (gn_of_set(sets[i]) == g) hs.push_back(sets[i]);
        for (int c = off0; c < int(hs.size()); c += kOneMaxSets) {
            OneRec r;
            r.gn = g;
            r.off = c;
            r.cnt = std::min(kOneMaxSets, int(hs.size()) - c);
            const int st = one_resolve(r, lau);
            if (st != SPH_OK) {
                delete plan;
                return st;
            }
            for (int i = r.off; i < r.off + r.cnt; ++i) {
                plan->total_points += hs[i].n;
                const int P = r.sh.cls[hs[i].l_max].P;
                plan->total_tiles += (hs[i].n + P - 1) / P;
            }
            plan->one.push_back(r);
        }
    }
    if (cudaMalloc(&plan->d_desc, sizeof(sph_batch_set) * hs.size()) != cudaSuccess ||
        cudaMalloc(&plan->d_one_ctr, sizeof(OneCounter) * plan->one.size()) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(plan->d_desc);
        delete plan;
        set_error("batch plan: device allocation failed");
        return SPH_ENOMEM;
    }
    cudaError_t e = cudaMemcpy(plan->d_desc, hs.data(), sizeof(sph_batch_set) * hs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(plan->d_one_ctr, 0, sizeof(OneCounter) * plan->one.size());
    if (e != cudaSuccess) {
        cudaFree(plan->d_desc);
        cudaFree(plan->d_one_ctr);
        delete plan;
        set_error("batch plan: %s", cudaGetErrorString(e));
        return SPH_ECUDA;
    }
    *out = plan;
    return SPH_OK;
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
    if (mode == SPH_BATCH_ONE_LAUNCH) return plan_create_one(sets, nsets, lau, dev, plan_out);
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
        if (mode == SPH_BATCH_PER_LMAX && grad && L >= kPoint4MinL) {  // 4 lanes per point (batch_four)
            P = 8;
            bytes_of[hs.size()] = int(point4_tile_bytes(L, 4, P, 16));
        }
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
        if (class_shapes && mode == SPH_BATCH_PER_LMAX && hs[i].dsph && hs[i].L >= kPoint4MinL)
            bl.W = point4_default_warps(hs[i].L);
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
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!plan->one.empty()) {
        // The kernels return their counters to zero themselves; the reset
        // here only guards against a previous run that did not finish.
        cudaError_t e = cudaMemsetAsync(plan->d_one_ctr, 0, sizeof(OneCounter) * plan->one.size(), st);
        uint32_t* status = device_status_word();
        for (size_t i = 0; i < plan->one.size() && e == cudaSuccess; ++i) {
            const OneRec& r = plan->one[i];
            e = static_cast<cudaError_t>(
                one_launch(r, plan->d_desc, plan->d_one_ctr + i, status, stream));
        }
        if (e != cudaSuccess) {
            set_error("batch_execute: %s", cudaGetErrorString(e));
            return SPH_ECUDA;
        }
        return SPH_OK;
    }
    if (plan->launches.empty()) return SPH_OK;
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
    cudaFree(plan->d_desc);
    cudaFree(plan->d_one_ctr);
    if (cur >= 0) cudaSetDevice(cur);
    delete plan;
    return SPH_OK;
}

// ------------------------------------------------- device descriptor array
int sphericart_compute_batched_ex(const sph_batch_set* desc, int nsets, int flags, const sph_launch* launch,
                                  void* stream) {
    if (nsets < 0 || (flags & ~(SPH_BATCHED_GRADIENTS | SPH_BATCHED_NORMALIZED)) != 0) {
        set_error("compute_batched: nsets=%d must be >= 0 and flags=%d a combination of SPH_BATCHED_*", nsets, flags);
        return SPH_EINVAL;
    }
    if (nsets == 0) return SPH_OK;
    if (!desc || reinterpret_cast<uintptr_t>(desc) % alignof(sph_batch_set) != 0) {
        set_error("compute_batched: desc must be a non-NULL, %zu-byte aligned device array",
                  alignof(sph_batch_set));
        return SPH_EINVAL;
    }
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, desc) != cudaSuccess || attr.type == cudaMemoryTypeUnregistered) {
        cudaGetLastError();
        set_error("compute_batched: desc must be device, managed or page-locked host memory");
        return SPH_EINVAL;
    }
    const sph_launch lau = launch ? *launch : sph_launch{0, 0, 0, 0};
    if (!one_launch_shape_ok(lau)) return SPH_EINVAL;
    const int gn = flags & 3;
    uint32_t* status = device_status_word();
    for (int c = 0; c < nsets; c += kOneMaxSets) {
        OneRec r;
        r.gn = gn;
        r.off = c;
        r.cnt = std::min(kOneMaxSets, nsets - c);
        const int st = one_resolve(r, lau);
        if (st != SPH_OK) return st;
        const int e = one_launch(r, desc, nullptr, status, stream);
        if (e != 0) {
            set_error("compute_batched launch: %s", cudaGetErrorString(static_cast<cudaError_t>(e)));
            return SPH_ECUDA;
        }
    }
    return SPH_OK;
}

int sphericart_compute_batched(const sph_batch_set* desc, int nsets, int flags, void* stream) {
    return sphericart_compute_batched_ex(desc, nsets, flags, nullptr, stream);
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
// The descriptors are copied into the file-scope array below instead of a
// plan's cudaMalloc'd buffer, and the one-launch kernel runs on them with a
// self-resetting tile counter from its static ring. Every GPU that loads
// this library holds kNoAllocScratchBytes (160 KB) of it until the process
// exits. All calls on a device share it and it keeps the last call's
// descriptors.
namespace sph {
namespace {

constexpr int kNoAllocMaxSets = 4096;
constexpr size_t kNoAllocScratchBytes = sizeof(sph_batch_set) * kNoAllocMaxSets;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;                        // guards the staging array below
sph_batch_set g_noalloc_host[kNoAllocMaxSets];  // host staging of the descriptors

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
    if (!one_launch_shape_ok(lau)) return SPH_EINVAL;
    // The descriptors are copied from host staging that the next call
    // overwrites; a captured copy would read it again at every replay.
    // So a stream that is being captured is refused before anything is
    // enqueued or set up.
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        const cudaError_t qe = cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cs);
        if (qe != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
            if (qe != cudaSuccess) cudaGetLastError();
            set_error("batch_compute_noalloc: the stream is being captured (or its capture state is unknown: %s); "
                      "this entry point stages its work list in host memory that later calls overwrite, so it "
                      "runs eagerly only",
                      qe != cudaSuccess ? cudaGetErrorString(qe) : "capturing");
            return SPH_EINVAL;
        }
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        cudaGetLastError();
        set_error("batch_compute_noalloc: no usable CUDA device");
        return SPH_ECUDA;
    }

    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    // The current device's address of the static array, looked up on every
    // call (host code must not use the symbol itself; a cached address would
    // not survive a device reset or a new primary context).
    void* p = nullptr;
    const cudaError_t es = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (es != cudaSuccess || !p) {
        cudaGetLastError();
        set_error("batch_compute_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(es));
        return SPH_ECUDA;
    }
    sph_batch_set* d_sets = static_cast<sph_batch_set*>(p);

    // Descriptors grouped by flag class (gradients, normalized), stable.
    int count[5] = {0, 0, 0, 0, 0};
    for (int i = 0; i < nsets; ++i) ++count[gn_of_set(sets[i]) + 1];
    for (int g = 1; g <= 4; ++g) count[g] += count[g - 1];
    int start[4] = {count[0], count[1], count[2], count[3]};
    for (int i = 0; i < nsets; ++i) g_noalloc_host[count[gn_of_set(sets[i])]++] = sets[i];
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // From pageable host memory the copy has consumed g_noalloc_host when it
    // returns, so the staging may be reused by the next call.
    cudaError_t e =
        cudaMemcpyAsync(d_sets, g_noalloc_host, sizeof(sph_batch_set) * size_t(nsets), cudaMemcpyHostToDevice, st);
    for (int g = 0; g < 4 && e == cudaSuccess; ++g) {
        const int end = g < 3 ? start[g + 1] : nsets;
        if (end == start[g]) continue;
        for (int c = start[g]; c < end && e == cudaSuccess; c += kOneMaxSets) {
            OneRec r;
            r.gn = g;
            r.off = c;
            r.cnt = std::min(kOneMaxSets, end - c);
            const int rs = one_resolve(r, lau);
            if (rs != SPH_OK) return rs;
            e = static_cast<cudaError_t>(one_launch(r, d_sets, nullptr, nullptr, stream));
        }
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("batch_compute_noalloc: %s", cudaGetErrorString(e));
        return SPH_ECUDA;
    }
    return SPH_OK;
}
