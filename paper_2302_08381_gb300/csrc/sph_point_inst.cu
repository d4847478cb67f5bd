// Instantiates the POINT kernels for one compile-time l_max. The build
// compiles this file once per l_max in [0, SPH_MAX_L_POINT] with
// -DSPH_INST_L=<l_max>, in parallel.
#include "sph_batch.cuh"

#ifndef SPH_INST_L
#error "compile with -DSPH_INST_L=<l_max>"
#endif

#define SPH_CAT2(a, b) a##b
#define SPH_CAT(a, b) SPH_CAT2(a, b)

namespace sph {

int SPH_CAT(point_fwd_L, SPH_INST_L)(const FwdArgs& a) {
    constexpr int L = SPH_INST_L;
    const bool grad = a.dsph != nullptr;
    const bool norm = a.normalized != 0;
#define SPH_FWD(T, TO)                                                          \
    return grad ? (norm ? launch_point_fwd<L, true, false, true, T, TO>(a)      \
                        : launch_point_fwd<L, true, false, false, T, TO>(a))    \
                : (norm ? launch_point_fwd<L, false, false, true, T, TO>(a)     \
                        : launch_point_fwd<L, false, false, false, T, TO>(a));
    if (a.launch.lanes_per_point == 10) {  // one lane per distinct plane, Hessians (FP32 arithmetic and storage)
        if (a.ddsph == nullptr || a.dtype != SPH_F32 || a.out != SPH_OUT_SAME) return int(cudaErrorInvalidValue);
        return norm ? launch_point10_fwd<L, true>(a) : launch_point10_fwd<L, false>(a);
    }
    if (a.launch.lanes_per_point == 16) {  // one lane per output plane, Hessians (FP32 arithmetic and storage)
        if (a.ddsph == nullptr || a.dtype != SPH_F32 || a.out != SPH_OUT_SAME) return int(cudaErrorInvalidValue);
        return norm ? launch_point16_fwd<L, true>(a) : launch_point16_fwd<L, false>(a);
    }
    if (a.launch.lanes_per_point == 4) {  // one lane per output plane (FP32 arithmetic, gradients)
        if (!grad || a.ddsph != nullptr || a.dtype != SPH_F32) return int(cudaErrorInvalidValue);
        if (a.out == SPH_OUT_BF16)
            return norm ? launch_point4_fwd<L, true, float, __nv_bfloat16>(a)
                        : launch_point4_fwd<L, false, float, __nv_bfloat16>(a);
        return norm ? launch_point4_fwd<L, true, float, float>(a) : launch_point4_fwd<L, false, float, float>(a);
    }
    if (a.ddsph != nullptr) {  // Hessians (FP32 or FP64 storage; validated by the caller)
        if (a.dtype == SPH_F64)
            return norm ? launch_point_fwd<L, true, true, true, double, double>(a)
                        : launch_point_fwd<L, true, true, false, double, double>(a);
        return norm ? launch_point_fwd<L, true, true, true, float, float>(a)
                    : launch_point_fwd<L, true, true, false, float, float>(a);
    }
    if (a.hc) {  // hybrid: hard-coded l <= 3, the recursion above (values and gradients)
        if constexpr (L <= kHcMaxL) {
#define SPH_FWD_HC(T, TO)                                                            \
    return grad ? (norm ? launch_point_fwd<L, true, false, true, T, TO, true>(a)      \
                        : launch_point_fwd<L, true, false, false, T, TO, true>(a))    \
                : (norm ? launch_point_fwd<L, false, false, true, T, TO, true>(a)     \
                        : launch_point_fwd<L, false, false, false, T, TO, true>(a));
            if (a.dtype == SPH_F64) {
                SPH_FWD_HC(double, double)
            }
            SPH_FWD_HC(float, float)
#undef SPH_FWD_HC
        }
        return int(cudaErrorInvalidValue);
    }
    if (a.dtype == SPH_F64) {
        SPH_FWD(double, double)
    }
    if (a.out == SPH_OUT_BF16) {
        SPH_FWD(float, __nv_bfloat16)
    }
    SPH_FWD(float, float)
#undef SPH_FWD
}

int SPH_CAT(point_bwd_L, SPH_INST_L)(const BwdArgs& a) {
    constexpr int L = SPH_INST_L;
    if (a.dtype == SPH_F64)
        return a.normalized ? launch_point_bwd<L, true, false, double>(a) : launch_point_bwd<L, false, false, double>(a);
    return a.normalized ? launch_point_bwd<L, true, false, float>(a) : launch_point_bwd<L, false, false, float>(a);
}

int SPH_CAT(point_dbwd_L, SPH_INST_L)(const BwdArgs& a) {
    constexpr int L = SPH_INST_L;
    if (a.dtype == SPH_F64)
        return a.normalized ? launch_point_bwd<L, true, true, double>(a) : launch_point_bwd<L, false, true, double>(a);
    return a.normalized ? launch_point_bwd<L, true, true, float>(a) : launch_point_bwd<L, false, true, float>(a);
}

// The ragged-batch kernel restricted to this l_max (one launch per l_max
// class of a batch plan).
int SPH_CAT(batch_class_L, SPH_INST_L)(const BatchClassArgs& a) {
    switch (a.gn) {
        case 0:
            return batch_kernel_run<SPH_INST_L, 0>(a);
        case 1:
            return batch_kernel_run<SPH_INST_L, 1>(a);
        case 2:
            return batch_kernel_run<SPH_INST_L, 2>(a);
        case 3:
            return batch_kernel_run<SPH_INST_L, 3>(a);
        default:
            return batch_kernel_run<SPH_INST_L, -1>(a);
    }
}

}  // namespace sph
