// Radial expansion fused with the harmonics (arXiv 2302.08381, Eq. expansion):
//
//   c[i, n, (l,m)] = sum_{k in centre i} R[k, n, l] * Y_l^m(x_k)
//
// for points (edge vectors) grouped by centre in CSR order. The harmonics are
// never written to memory: one warp owns a centre, evaluates Y for 32 of its
// points at a time (one lane per point, the unrolled recursion of the POINT
// kernels, values only) into shared memory, stages the matching rows of R,
// and then each lane accumulates the output columns it owns. Only the
// coordinates, R and the [n_rad, K] result per centre touch HBM.
#include <cuda_runtime.h>

#include <algorithm>

#include "sph_point.cuh"

namespace sph {

constexpr uint32_t kStatusBadOffsets = 2u;
constexpr int kExpansionMaxRad = 64;
constexpr int kExpansionAcc = 8;  // radial channels accumulated per register pass

template <typename T, int K>
struct ValVis {
    T* row;
    __device__ __forceinline__ void emit(int, int k, const Deriv<T>& d) { row[k] = d.v; }
};

__device__ __forceinline__ int l_of_column(int k) {
    int l = int(sqrtf(float(k)));
    if ((l + 1) * (l + 1) <= k) ++l;
    if (l * l > k) --l;
    return l;
}

// Radial channels per point are staged as [l][n] with n padded to a multiple
// of 4 (zeros), so the kExpansionAcc factors a column needs are contiguous
// and 16-byte aligned.
__host__ __device__ constexpr int padded_rad(int nr) { return (nr + 3) / 4 * 4; }

template <int L, typename T>
__host__ __device__ constexpr size_t expansion_warp_bytes(int nr) {
    constexpr int K = (L + 1) * (L + 1);
    constexpr int SY = (K % 2 == 0) ? K + 1 : K;
    const int SR = (L + 1) * padded_rad(nr) + 4;  // row stride, a multiple of 4 (16-byte rows)
    return align16(size_t(32) * SY * sizeof(T)) + align16(size_t(32) * SR * sizeof(T)) +
           align16(size_t(nr) * K * sizeof(T));
}

template <int L, bool NORM, typename T>
__global__ void __launch_bounds__(256) expansion_kernel(const T* __restrict__ xyz, const T* __restrict__ R,
                                                        const int64_t* __restrict__ offsets, int64_t ncent,
                                                        int64_t npts, int nr,
                                                        const __grid_constant__ PointTabs<L, T, false> tb,
                                                        T* __restrict__ c, uint32_t* __restrict__ status) {
    constexpr int K = (L + 1) * (L + 1);
    constexpr int SY = (K % 2 == 0) ? K + 1 : K;
    constexpr int RL = L + 1;
    const int NP = padded_rad(nr);
    const int RW = nr * RL;            // R row width in global memory ([n][l])
    const int SR = RL * NP + 4;        // staged row stride ([l][n_padded])
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    unsigned char* base = smem + size_t(warp) * expansion_warp_bytes<L, T>(nr);
    T* Ys = reinterpret_cast<T*>(base);
    T* Rs = reinterpret_cast<T*>(base + align16(size_t(32) * SY * sizeof(T)));
    T* Cs = reinterpret_cast<T*>(base + align16(size_t(32) * SY * sizeof(T)) + align16(size_t(32) * SR * sizeof(T)));
    const int nout = nr * K;
    // zero the padding channels once (never overwritten)
    for (int t = lane; t < 32 * SR; t += 32) Rs[t] = T(0);
    __syncwarp();

    for (int64_t i = int64_t(blockIdx.x) * W + warp; i < ncent; i += int64_t(gridDim.x) * W) {
        const int64_t e0 = offsets[i], e1 = offsets[i + 1];
        T* ci = c + i * nout;
        if (e0 < 0 || e1 < e0 || e1 > npts) {  // malformed CSR: flag it, write zeros
            if (lane == 0) atomicOr(status, kStatusBadOffsets);
            for (int o = lane; o < nout; o += 32) ci[o] = T(0);
            continue;
        }
        for (int o = lane; o < nout; o += 32) Cs[o] = T(0);
        for (int64_t ch = e0; ch < e1; ch += 32) {
            const int cnt = int(min(int64_t(32), e1 - ch));
            if (lane < cnt) {
                const int64_t p = ch + lane;
                T x = xyz[3 * p], y = xyz[3 * p + 1], z = xyz[3 * p + 2];
                T r2, ir = T(1);
                if (NORM) {
                    unit_point(x, y, z, r2, ir);
                } else {
                    r2 = x * x + y * y + z * z;
                }
                ValVis<T, K> vis{Ys + size_t(lane) * SY};
                point_core<L, false, false>(x, y, z, r2, tb, vis);
            }
            {  // this chunk's radial rows: coalesced reads, [n][l] -> [l][n] in shared memory
                const T* src = R + ch * RW;
                for (int r = 0; r < cnt; ++r) {
                    for (int q = lane; q < RW; q += 32) {
                        const int n = q / RL;  // RL is a compile-time constant
                        Rs[r * SR + (q - n * RL) * NP + n] = src[r * RW + q];
                    }
                }
            }
            __syncwarp();
            for (int k = lane; k < K; k += 32) {
                const int l = l_of_column(k);
                for (int n0 = 0; n0 < nr; n0 += kExpansionAcc) {
                    T acc[kExpansionAcc];
#pragma unroll
                    for (int b = 0; b < kExpansionAcc; ++b) acc[b] = (n0 + b < nr) ? Cs[(n0 + b) * K + k] : T(0);
                    const T* rcol = Rs + l * NP + n0;
#pragma unroll 4
                    for (int e = 0; e < cnt; ++e) {
                        const T yv = Ys[e * SY + k];
                        const T* re = rcol + e * SR;
                        if (n0 + kExpansionAcc <= NP) {
#pragma unroll
                            for (int b = 0; b < kExpansionAcc; ++b) acc[b] += re[b] * yv;
                        } else {
#pragma unroll
                            for (int b = 0; b < kExpansionAcc; ++b)
                                if (n0 + b < NP) acc[b] += re[b] * yv;
                        }
                    }
#pragma unroll
                    for (int b = 0; b < kExpansionAcc; ++b)
                        if (n0 + b < nr) Cs[(n0 + b) * K + k] = acc[b];
                }
            }
            __syncwarp();
        }
        for (int o = lane; o < nout; o += 32) ci[o] = Cs[o];
        __syncwarp();
    }
}

struct ExpArgs {
    const void* xyz;
    const void* radial;
    const int64_t* offsets;
    int64_t ncent;
    int64_t npts;
    int nr;
    int l_max;
    int normalized;
    int dtype;
    void* c;
    void* stream;
    int warps;
    uint32_t* status;
};

template <int L, bool NORM, typename T>
int launch_expansion(const ExpArgs& a) {
    static const PointTabs<L, T, false> tb = make_point_tabs<L, T, false>();
    const int W = a.warps;
    const size_t smem = size_t(W) * expansion_warp_bytes<L, T>(a.nr);
    auto kern = expansion_kernel<L, NORM, T>;
    cudaError_t err = ensure_smem(kern, smem);
    if (err != cudaSuccess) return int(err);
    const int grid = grid_for(kern, 32 * W, smem, a.ncent, 0);
    kern<<<grid, 32 * W, smem, static_cast<cudaStream_t>(a.stream)>>>(
        static_cast<const T*>(a.xyz), static_cast<const T*>(a.radial), a.offsets, a.ncent, a.npts, a.nr, tb,
        static_cast<T*>(a.c), a.status);
    return int(cudaGetLastError());
}

template <int L>
int launch_expansion_l(const ExpArgs& a) {
    if (a.dtype == SPH_F64)
        return a.normalized ? launch_expansion<L, true, double>(a) : launch_expansion<L, false, double>(a);
    return a.normalized ? launch_expansion<L, true, float>(a) : launch_expansion<L, false, float>(a);
}

int launch_expansion_any(const ExpArgs& a) {
    switch (a.l_max) {
#define SPH_CASE(LL) \
    case LL:         \
        return launch_expansion_l<LL>(a);
        SPH_CASE(0) SPH_CASE(1) SPH_CASE(2) SPH_CASE(3) SPH_CASE(4) SPH_CASE(5) SPH_CASE(6) SPH_CASE(7) SPH_CASE(8)
        SPH_CASE(9) SPH_CASE(10) SPH_CASE(11) SPH_CASE(12) SPH_CASE(13) SPH_CASE(14) SPH_CASE(15) SPH_CASE(16)
#undef SPH_CASE
        default:
            return int(cudaErrorInvalidValue);
    }
}

}  // namespace sph

using namespace sph;

extern "C" int sphericart_expansion(const void* xyz, const void* radial, const int64_t* offsets, int64_t n_centres,
                                    int64_t n_points, int n_rad, int l_max, int normalized, int dtype, void* c,
                                    void* stream) {
    if (n_centres < 0 || n_points < 0) {
        set_error("expansion: n_centres and n_points must be >= 0");
        return SPH_EINVAL;
    }
    if (l_max < 0 || l_max > SPH_MAX_L_POINT) {
        set_error("expansion: l_max=%d must be in [0,%d]", l_max, SPH_MAX_L_POINT);
        return SPH_EINVAL;
    }
    if (n_rad < 1 || n_rad > kExpansionMaxRad) {
        set_error("expansion: n_rad=%d must be in [1,%d]", n_rad, kExpansionMaxRad);
        return SPH_EINVAL;
    }
    if (dtype != SPH_F32 && dtype != SPH_F64) {
        set_error("expansion: dtype=%d is not an sph_dtype", dtype);
        return SPH_EINVAL;
    }
    if (n_centres == 0) return SPH_OK;
    if (!offsets || !c || (n_points > 0 && (!xyz || !radial))) {
        set_error("expansion: xyz, radial, offsets and c must be non-NULL");
        return SPH_EINVAL;
    }
    const size_t e = dtype == SPH_F64 ? 8 : 4;
    if (reinterpret_cast<uintptr_t>(xyz) % e || reinterpret_cast<uintptr_t>(radial) % e ||
        reinterpret_cast<uintptr_t>(c) % e || reinterpret_cast<uintptr_t>(offsets) % 8) {
        set_error("expansion: buffers must be aligned to their element size");
        return SPH_EINVAL;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        set_error("expansion: no usable CUDA device");
        return SPH_ECUDA;
    }
    uint32_t* status = device_status_word();
    if (!status) {
        set_error("expansion: could not allocate the device status word");
        return SPH_ENOMEM;
    }
    ExpArgs a{xyz, radial, offsets, n_centres, n_points, n_rad, l_max, normalized ? 1 : 0, dtype, c, stream, 4,
              status};
    // Fit the per-warp staging (Y rows, R rows, accumulators) in the opt-in limit.
    const size_t K = size_t(l_max + 1) * (l_max + 1);
    const size_t per_warp =
        e * (32 * (K + 1) + 32 * (size_t((n_rad + 3) / 4 * 4) * (l_max + 1) + 4) + size_t(n_rad) * K) + 48;
    while (a.warps > 1 && size_t(a.warps) * per_warp > size_t(max_smem_optin())) --a.warps;
    if (per_warp > size_t(max_smem_optin())) {
        set_error("expansion: n_rad=%d with l_max=%d needs %zu bytes of shared memory per warp", n_rad, l_max,
                  per_warp);
        return SPH_EUNSUPPORTED;
    }
    const int err = launch_expansion_any(a);
    if (err) {
        set_error("expansion launch: %s", cudaGetErrorString(static_cast<cudaError_t>(err)));
        return SPH_ECUDA;
    }
    return SPH_OK;
}
