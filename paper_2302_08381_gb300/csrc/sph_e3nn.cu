// The e3nn convention (arXiv 2302.08381, Section 3.2: the library provides
// wrappers with e3nn's conventions).
//
// e3nn's real spherical harmonics take y as the polar axis: its l = 1
// components are proportional to (x, y, z) in that order and its m = 0
// components to P_l(y / r). They equal this library's harmonics evaluated at
// the permuted point (x', y', z') = (z, x, y), for which Y_1 = c (y', z', x')
// = c (x, y, z), times a per-l factor for e3nn's normalizations:
//   integral  (each component squared integrates to 1 over the sphere): 1
//   component (sum over m of Y_l^m(u)^2 = 2l + 1 on the unit sphere): sqrt(4 pi)
//   norm      (sum over m of Y_l^m(u)^2 = 1 on the unit sphere):       sqrt(4 pi / (2l + 1))
// The gradients of the permuted evaluation are with respect to (x', y', z') =
// (z, x, y); e3nn's (d/dx, d/dy, d/dz) are its planes (1, 2, 0).
//
// Path: a permutation kernel writes (z, x, y) into a caller-provided
// workspace, the forward runs on it, and an in-place kernel reorders the
// gradient planes and applies the per-l factor.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "sph_internal.h"

namespace sph {
namespace {

template <typename T>
__global__ void e3nn_permute_kernel(const T* __restrict__ xyz, T* __restrict__ out, int64_t n) {
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < n; p += int64_t(gridDim.x) * blockDim.x) {
        const T x = xyz[3 * p], y = xyz[3 * p + 1], z = xyz[3 * p + 2];
        out[3 * p] = z;
        out[3 * p + 1] = x;
        out[3 * p + 2] = y;
    }
}

template <typename T>
struct E3nnScales {
    T v[SPH_MAX_L + 1];
};

// One thread per (point, column): scale the value and, with gradients,
// rotate the three planes of that column to (d/dx, d/dy, d/dz).
template <typename T>
__global__ void e3nn_finish_kernel(T* __restrict__ sph, T* __restrict__ dsph, int64_t n, int K,
                                   const __grid_constant__ E3nnScales<T> sc) {
    const int64_t total = n * int64_t(K);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t p = i / K;
        const int k = int(i - p * K);
        int l = int(sqrtf(float(k)));  // l with l^2 <= k < (l+1)^2
        while (l * l > k) --l;
        while ((l + 1) * (l + 1) <= k) ++l;
        const T f = sc.v[l];
        sph[i] *= f;
        if (dsph) {
            T* d = dsph + p * 3 * K + k;
            const T dz = d[0], dx = d[K], dy = d[2 * K];  // d/dx' = d/dz, d/dy' = d/dx, d/dz' = d/dy
            d[0] = f * dx;
            d[K] = f * dy;
            d[2 * K] = f * dz;
        }
    }
}

template <typename T>
int e3nn_run(const void* xyz, int64_t n, int l_max, int normalize, int normalization, void* workspace, void* sph,
             void* dsph, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int threads = 256;
    const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads,
                                                                    int64_t(sm_count()) * 8)));
    e3nn_permute_kernel<T><<<blocks, threads, 0, st>>>(static_cast<const T*>(xyz), static_cast<T*>(workspace), n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("compute_e3nn: %s", cudaGetErrorString(e));
        return SPH_ECUDA;
    }
    const int dtype = sizeof(T) == 8 ? SPH_F64 : SPH_F32;
    const int stt = sphericart_compute_ex(workspace, n, l_max, normalize, dtype, SPH_OUT_SAME, SPH_Q_NATIVE,
                                          SPH_KERNEL_AUTO, nullptr, sph, dsph, nullptr, stream);
    if (stt != SPH_OK) return stt;
    if (normalization == SPH_E3NN_INTEGRAL && !dsph) return SPH_OK;  // nothing to scale or reorder
    E3nnScales<T> sc{};
    const double four_pi = 4.0 * 3.14159265358979323846;
    for (int l = 0; l <= l_max; ++l)
        sc.v[l] = T(normalization == SPH_E3NN_INTEGRAL    ? 1.0
                    : normalization == SPH_E3NN_COMPONENT ? std::sqrt(four_pi)
                                                          : std::sqrt(four_pi / double(2 * l + 1)));
    const int K = (l_max + 1) * (l_max + 1);
    const int64_t total = n * int64_t(K);
    const int blocks2 = int(std::max<int64_t>(1, std::min<int64_t>((total + threads - 1) / threads,
                                                                     int64_t(sm_count()) * 16)));
    e3nn_finish_kernel<T><<<blocks2, threads, 0, st>>>(static_cast<T*>(sph), static_cast<T*>(dsph), n, K, sc);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("compute_e3nn: %s", cudaGetErrorString(e));
        return SPH_ECUDA;
    }
    return SPH_OK;
}

}  // namespace
}  // namespace sph

using namespace sph;

extern "C" int sphericart_compute_e3nn(const void* xyz, int64_t n, int l_max, int normalize, int normalization,
                                       int dtype, void* workspace, void* sph, void* dsph, void* stream) {
    if (n < 0 || l_max < 0 || l_max > SPH_MAX_L || (dtype != SPH_F32 && dtype != SPH_F64) ||
        (normalization != SPH_E3NN_INTEGRAL && normalization != SPH_E3NN_COMPONENT &&
         normalization != SPH_E3NN_NORM)) {
        set_error("compute_e3nn: n >= 0, 0 <= l_max <= %d, dtype SPH_F32/SPH_F64 and an sph_e3nn_norm required",
                  SPH_MAX_L);
        return SPH_EINVAL;
    }
    if (n == 0) return SPH_OK;
    const size_t elem = dtype == SPH_F64 ? 8 : 4;
    if (!xyz || !workspace || !sph || reinterpret_cast<uintptr_t>(xyz) % elem ||
        reinterpret_cast<uintptr_t>(workspace) % elem) {
        set_error("compute_e3nn: xyz, workspace ([n,3], the dtype) and sph must be non-NULL and aligned");
        return SPH_EINVAL;
    }
    return dtype == SPH_F64 ? e3nn_run<double>(xyz, n, l_max, normalize, normalization, workspace, sph, dsph, stream)
                            : e3nn_run<float>(xyz, n, l_max, normalize, normalization, workspace, sph, dsph, stream);
}
