// Instantiates the one-launch batch kernel for one class of flags: the build
// compiles this file four times, with -DSPH_BATCH_GN=<gradients + 2 * normalized>.
#include <atomic>

#define SPH_BATCH_ONE_KERNELS 1
#include "sph_batch_one.cuh"

#ifndef SPH_BATCH_GN
#error "compile with -DSPH_BATCH_GN=<0..3>"
#endif

#define SPH_CAT2(a, b) a##b
#define SPH_CAT(a, b) SPH_CAT2(a, b)

namespace sph {

namespace {
std::atomic<unsigned> g_one_next_slot{0};
}

int SPH_CAT(batch_one_gn, SPH_BATCH_GN)(const OneArgs& a) {
    auto kern = batch_one_kernel<SPH_BATCH_GN>;
    cudaError_t e = ensure_smem(kern, a.smem);
    if (e != cudaSuccess) return int(e);
    if (a.occ_out) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, reinterpret_cast<const void*>(kern), 32 * a.W,
                                                          a.smem) != cudaSuccess) {
            cudaGetLastError();
            occ = 1;
        }
        *a.occ_out = occ;
        return 0;
    }
    static const PointTabs<16, float, false> tabs = make_point_tabs<16, float, false>();
    OneParams prm;
    prm.tabs = tabs;
    for (int L = 0; L <= SPH_MAX_L_POINT; ++L) prm.cls[L] = a.cls[L];
    const int slot = a.ctr ? 0 : int(g_one_next_slot.fetch_add(1u) % unsigned(kOneRingSlots));
    kern<<<a.blocks, 32 * a.W, a.smem, static_cast<cudaStream_t>(a.stream)>>>(a.desc, a.nsets, a.ctr, slot,
                                                                           a.staging_bytes, a.status, prm);
    return int(cudaGetLastError());
}

}  // namespace sph
