// SLICE kernel family: any l_max <= SPH_MAX_L, chosen at run time.
//
// A group of G lanes (8, 16 or 32) owns one point; lane j of the group owns the
// m channels m = j, j+G, j+2G, ... . The Q_l^m recursion of Eq. iter-q
// (arXiv 2302.08381) only couples equal m, so each lane runs its channels
// independently; the derivative identities of Eq. iter-deri need the
// neighbouring channels m+1 (gradients) and m+2 (Hessians), which the lane
// runs alongside. The loop over l is uniform across the group, so at each l
// the group writes the contiguous columns l*l+l +/- m with coalesced stores and
// needs no shared-memory staging. Tables are read from global memory (cached),
// indexed by (l, m).
//
// This family covers large l_max, Hessians, and the mixed precision mode in
// which all arithmetic runs in FP64 (TQ = double) on FP32 inputs and outputs.
#include <cuda_runtime.h>

#include <algorithm>

#include "sph_core.cuh"
#include "sph_internal.h"

namespace sph {

namespace {

template <typename TQ>
struct V4T;
template <>
struct V4T<float> {
    using type = float4;
};
template <>
struct V4T<double> {
    using type = double4_32a;  // entries are 64-byte strided, so 32-byte aligned
};

// Qtilde_l^c of channel c at degree l from its two previous values, with one
// vector load and no branch: the packed entry folds the diagonal seed and the
// first off-diagonal step into the same formula; l < c gives 0.
template <typename TQ>
__device__ __forceinline__ TQ advance(const TQ* __restrict__ tb, int l, int c, TQ z, TQ r2, TQ q1, TQ q2) {
    using V4 = typename V4T<TQ>::type;
    const bool on = l >= c;
    const V4 t = reinterpret_cast<const V4*>(tb)[2 * tri(l, on ? c : l)];
    const TQ q = (t.x * z) * q1 - (t.y * r2) * q2 + t.z;
    return on ? q : TQ(0);
}

// Visits every column of the lane's channels at one point. For each (l, m)
// with m owned by this lane, calls f(l, k, Deriv) with normalized
// derivatives when NORM.
//
// With TQ wider than T (the mixed mode) the unit-vector scaling and both
// recursions (Eq. iter-sc, Eq. iter-q) run in TQ and only the assembled
// outputs are rounded to T: in FP32 the dominant error is the rounding of
// u = xyz/r and of the c_m/s_m powers (~l eps |Y|), not the Q recursion.
// Rounds every field of a Deriv to T (identity when TQ == T).
template <typename T, typename TQ>
__device__ __forceinline__ Deriv<T> to_type(const Deriv<TQ>& d) {
    Deriv<T> o;
    o.v = T(d.v);
    o.gx = T(d.gx);
    o.gy = T(d.gy);
    o.gz = T(d.gz);
    o.hxx = T(d.hxx);
    o.hxy = T(d.hxy);
    o.hxz = T(d.hxz);
    o.hyy = T(d.hyy);
    o.hyz = T(d.hyz);
    o.hzz = T(d.hzz);
    return o;
}

template <typename TQ, typename T, bool GRAD, bool HESS, bool NORM, int G, typename F>
__device__ __forceinline__ void slice_point(T xin, T yin, T zin, int L, int j, const TQ* __restrict__ tb, int tn,
                                            TQ inv_sqrt2, bool active, F&& f) {
    using V4 = typename V4T<TQ>::type;
    (void)tn;
    TQ xq = TQ(xin), yq = TQ(yin), zq = TQ(zin);
    TQ r2q, irq = TQ(1);
    if (NORM) {
        unit_point(xq, yq, zq, r2q, irq);
    } else {
        r2q = xq * xq + yq * yq + zq * zq;
    }
    for (int m0 = 0; m0 <= L; m0 += G) {
        const int m = m0 + j;
        // c_m, s_m and the two previous pairs by Eq. iter-sc.
        TQ cq = TQ(1), sq = TQ(0), cq1 = TQ(0), sq1 = TQ(0), cq2 = TQ(0), sq2 = TQ(0);
        const int mt = min(m, L);
        for (int t = 1; t <= mt; ++t) {
            const TQ nc = xq * cq - yq * sq;
            const TQ ns = xq * sq + yq * cq;
            cq2 = cq1;
            sq2 = sq1;
            cq1 = cq;
            sq1 = sq;
            cq = nc;
            sq = ns;
        }
        TQ a1 = TQ(0), a2 = TQ(0), b1 = TQ(0), b2 = TQ(0), c1 = TQ(0), c2 = TQ(0);
        for (int l = m0; l <= L; ++l) {
            const TQ qa = advance(tb, l, m, zq, r2q, a1, a2);
            const TQ qb = (GRAD || HESS) ? advance(tb, l, m + 1, zq, r2q, b1, b2) : TQ(0);
            const TQ qc = HESS ? advance(tb, l, m + 2, zq, r2q, c1, c2) : TQ(0);
            if (active && m <= l) {
                const int i = tri(l, m);
                QParts<TQ> qp;
                qp.Q = qa;
                if (GRAD || HESS) {
                    const V4 t0 = reinterpret_cast<const V4*>(tb)[2 * i];
                    const V4 t1 = reinterpret_cast<const V4*>(tb)[2 * i + 1];
                    qp.E1 = t0.w * b1;
                    qp.Qz = t1.x * a1;
                    if (HESS) {
                        qp.G2 = t1.y * c2;
                        qp.G3 = t1.z * b2;
                        qp.G4 = t1.w * a2;
                    } else {
                        qp.G2 = qp.G3 = qp.G4 = TQ(0);
                    }
                } else {
                    qp.E1 = qp.Qz = qp.G2 = qp.G3 = qp.G4 = TQ(0);
                }
                if (m == 0) {
                    Deriv<TQ> d = assemble_m0<GRAD, HESS>(qp, xq, yq, inv_sqrt2);
                    if (NORM && (GRAD || HESS)) normalize_deriv<HESS>(d, l, xq, yq, zq, irq);
                    f(l, l * l + l, to_type<T>(d));
                } else {
                    Deriv<TQ> dc, ds;
                    assemble_m<GRAD, HESS>(qp, xq, yq, TQ(m), TQ(m - 1), cq, sq, cq1, sq1, cq2, sq2, dc, ds);
                    if (NORM && (GRAD || HESS)) {
                        normalize_deriv<HESS>(dc, l, xq, yq, zq, irq);
                        normalize_deriv<HESS>(ds, l, xq, yq, zq, irq);
                    }
                    f(l, l * l + l + m, to_type<T>(dc));
                    f(l, l * l + l - m, to_type<T>(ds));
                }
            }
            a2 = a1;
            a1 = qa;
            b2 = b1;
            b1 = qb;
            c2 = c1;
            c1 = qc;
        }
    }
}

template <typename TI, typename TQ, typename T, typename TO, bool GRAD, bool HESS, bool NORM, int G>
__global__ void __launch_bounds__(256) slice_fwd_kernel(const TI* __restrict__ xyz, int64_t n, int L,
                                                        const TQ* __restrict__ tb, int tn, TQ inv_sqrt2,
                                                        TO* __restrict__ sph, TO* __restrict__ dsph,
                                                        TO* __restrict__ ddsph) {
    constexpr int PPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const int j = lane % G;
    const int grp = lane / G;
    const int64_t K = int64_t(L + 1) * (L + 1);
    const int64_t wid = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t base = wid * PPW; base < n; base += nw * PPW) {
        const int64_t p = base + grp;
        const bool active = p < n;
        T x = T(0), y = T(0), z = T(0);
        if (active) {
            x = T(xyz[3 * p]);
            y = T(xyz[3 * p + 1]);
            z = T(xyz[3 * p + 2]);
        }
        TO* rv = sph + p * K;
        TO* rd = dsph + p * 3 * K;
        TO* rh = ddsph + p * 9 * K;
        slice_point<TQ, T, GRAD, HESS, NORM, G>(x, y, z, L, j, tb, tn, inv_sqrt2, active,
                                                [&](int, int k, const Deriv<T>& d) {
                                                    rv[k] = OutConv<TO>::cv(d.v);
                                                    if (GRAD) {
                                                        rd[k] = OutConv<TO>::cv(d.gx);
                                                        rd[K + k] = OutConv<TO>::cv(d.gy);
                                                        rd[2 * K + k] = OutConv<TO>::cv(d.gz);
                                                    }
                                                    if (HESS) {
                                                        rh[0 * K + k] = OutConv<TO>::cv(d.hxx);
                                                        rh[1 * K + k] = OutConv<TO>::cv(d.hxy);
                                                        rh[2 * K + k] = OutConv<TO>::cv(d.hxz);
                                                        rh[3 * K + k] = OutConv<TO>::cv(d.hxy);
                                                        rh[4 * K + k] = OutConv<TO>::cv(d.hyy);
                                                        rh[5 * K + k] = OutConv<TO>::cv(d.hyz);
                                                        rh[6 * K + k] = OutConv<TO>::cv(d.hxz);
                                                        rh[7 * K + k] = OutConv<TO>::cv(d.hyz);
                                                        rh[8 * K + k] = OutConv<TO>::cv(d.hzz);
                                                    }
                                                });
    }
}

template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off, G);
    return v;
}

// DBW = false: dxyz = sum_k g_k dY_k. DBW = true: grad_g and grad_xyz.
template <typename T, bool NORM, bool DBW, int G>
__global__ void __launch_bounds__(256) slice_bwd_kernel(const T* __restrict__ xyz, const T* __restrict__ g,
                                                        const T* __restrict__ v, int64_t n, int L,
                                                        const T* __restrict__ tb, int tn, T inv_sqrt2,
                                                        T* __restrict__ dxyz, T* __restrict__ grad_g,
                                                        T* __restrict__ grad_xyz) {
    constexpr int PPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const int j = lane % G;
    const int grp = lane / G;
    const int64_t K = int64_t(L + 1) * (L + 1);
    const int64_t wid = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t base = wid * PPW; base < n; base += nw * PPW) {
        const int64_t p = base + grp;
        const bool active = p < n;
        T x = T(0), y = T(0), z = T(0), vx = T(0), vy = T(0), vz = T(0);
        if (active) {
            x = xyz[3 * p];
            y = xyz[3 * p + 1];
            z = xyz[3 * p + 2];
            if (DBW) {
                vx = v[3 * p];
                vy = v[3 * p + 1];
                vz = v[3 * p + 2];
            }
        }
        const T* gr = g + p * K;
        T* go = grad_g ? grad_g + p * K : nullptr;
        T ax = T(0), ay = T(0), az = T(0);
        slice_point<T, T, true, DBW, NORM, G>(x, y, z, L, j, tb, tn, inv_sqrt2, active,
                                              [&](int, int k, const Deriv<T>& d) {
                                                  const T gk = gr[k];
                                                  if (!DBW) {
                                                      ax += gk * d.gx;
                                                      ay += gk * d.gy;
                                                      az += gk * d.gz;
                                                  } else {
                                                      if (go) go[k] = vx * d.gx + vy * d.gy + vz * d.gz;
                                                      ax += gk * (d.hxx * vx + d.hxy * vy + d.hxz * vz);
                                                      ay += gk * (d.hxy * vx + d.hyy * vy + d.hyz * vz);
                                                      az += gk * (d.hxz * vx + d.hyz * vy + d.hzz * vz);
                                                  }
                                              });
        ax = group_sum<G>(ax);
        ay = group_sum<G>(ay);
        az = group_sum<G>(az);
        if (active && j == 0) {
            T* o = DBW ? grad_xyz : dxyz;
            if (o) {
                o[3 * p] = ax;
                o[3 * p + 1] = ay;
                o[3 * p + 2] = az;
            }
        }
    }
}

int pick_group(int L, int requested) {
    if (requested == 8 || requested == 16 || requested == 32) return requested;
    if (L + 1 <= 8) return 8;
    if (L + 1 <= 16) return 16;
    return 32;
}

template <typename Kern>
int slice_grid(Kern kern, int64_t n, int G, int blocks_per_sm) {
    const int threads = 256;
    const int64_t groups_per_block = (threads / 32) * (32 / G);
    int bps = blocks_per_sm;
    if (bps <= 0) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, reinterpret_cast<const void*>(kern), threads, 0) !=
            cudaSuccess)
            occ = 1;
        bps = std::max(occ, 1);
    }
    const int64_t want = (n + groups_per_block - 1) / groups_per_block;
    const int64_t cap = int64_t(bps) * sm_count();
    return int(std::max<int64_t>(1, std::min(want, cap)));
}

template <typename TI, typename TQ, typename T, typename TO, bool GRAD, bool HESS, bool NORM, int G>
int launch_fwd_g(const FwdArgs& a, const TQ* tb) {
    auto kern = slice_fwd_kernel<TI, TQ, T, TO, GRAD, HESS, NORM, G>;
    const int grid = slice_grid(kern, a.n, G, a.launch.blocks_per_sm);
    kern<<<grid, 256, 0, static_cast<cudaStream_t>(a.stream)>>>(
        static_cast<const TI*>(a.xyz), a.n, a.l_max, tb, tri_size(SPH_MAX_L), TQ(host_tables().inv_sqrt2),
        static_cast<TO*>(a.sph), static_cast<TO*>(a.dsph), static_cast<TO*>(a.ddsph));
    return int(cudaGetLastError());
}

template <typename TI, typename TQ, typename T, typename TO, bool GRAD, bool HESS, bool NORM>
int launch_fwd(const FwdArgs& a, const TQ* tb) {
    switch (pick_group(a.l_max, a.launch.lanes_per_point)) {
        case 8:
            return launch_fwd_g<TI, TQ, T, TO, GRAD, HESS, NORM, 8>(a, tb);
        case 16:
            return launch_fwd_g<TI, TQ, T, TO, GRAD, HESS, NORM, 16>(a, tb);
        default:
            return launch_fwd_g<TI, TQ, T, TO, GRAD, HESS, NORM, 32>(a, tb);
    }
}

template <typename TI, typename TQ, typename T, typename TO>
int launch_fwd_flags(const FwdArgs& a, const TQ* tb) {
    const bool grad = a.dsph != nullptr, hess = a.ddsph != nullptr, norm = a.normalized != 0;
    if (hess)
        return norm ? launch_fwd<TI, TQ, T, TO, true, true, true>(a, tb)
                    : launch_fwd<TI, TQ, T, TO, true, true, false>(a, tb);
    if (grad)
        return norm ? launch_fwd<TI, TQ, T, TO, true, false, true>(a, tb)
                    : launch_fwd<TI, TQ, T, TO, true, false, false>(a, tb);
    return norm ? launch_fwd<TI, TQ, T, TO, false, false, true>(a, tb)
                : launch_fwd<TI, TQ, T, TO, false, false, false>(a, tb);
}

template <typename T, bool NORM, bool DBW, int G>
int launch_bwd_g(const BwdArgs& a, const T* tb) {
    auto kern = slice_bwd_kernel<T, NORM, DBW, G>;
    const int grid = slice_grid(kern, a.n, G, a.launch.blocks_per_sm);
    kern<<<grid, 256, 0, static_cast<cudaStream_t>(a.stream)>>>(
        static_cast<const T*>(a.xyz), static_cast<const T*>(a.g), static_cast<const T*>(a.v), a.n, a.l_max, tb,
        tri_size(SPH_MAX_L), T(host_tables().inv_sqrt2), static_cast<T*>(a.dxyz), static_cast<T*>(a.grad_g),
        static_cast<T*>(a.grad_xyz));
    return int(cudaGetLastError());
}

template <typename T, bool DBW>
int launch_bwd(const BwdArgs& a, const T* tb) {
    const int G = pick_group(a.l_max, a.launch.lanes_per_point);
    if (a.normalized) {
        if (G == 8) return launch_bwd_g<T, true, DBW, 8>(a, tb);
        if (G == 16) return launch_bwd_g<T, true, DBW, 16>(a, tb);
        return launch_bwd_g<T, true, DBW, 32>(a, tb);
    }
    if (G == 8) return launch_bwd_g<T, false, DBW, 8>(a, tb);
    if (G == 16) return launch_bwd_g<T, false, DBW, 16>(a, tb);
    return launch_bwd_g<T, false, DBW, 32>(a, tb);
}

}  // namespace

int slice_fwd(const FwdArgs& a) {
    if (a.dtype == SPH_F64) {
        const double* tb = static_cast<const double*>(device_tables(SPH_F64));
        if (!tb) return int(cudaErrorMemoryAllocation);
        return launch_fwd_flags<double, double, double, double>(a, tb);
    }
    if (a.qprec == SPH_Q_F64) {
        const double* tb = static_cast<const double*>(device_tables(SPH_F64));
        if (!tb) return int(cudaErrorMemoryAllocation);
        if (a.out == SPH_OUT_BF16) return launch_fwd_flags<float, double, float, __nv_bfloat16>(a, tb);
        return launch_fwd_flags<float, double, float, float>(a, tb);
    }
    const float* tb = static_cast<const float*>(device_tables(SPH_F32));
    if (!tb) return int(cudaErrorMemoryAllocation);
    if (a.out == SPH_OUT_BF16) return launch_fwd_flags<float, float, float, __nv_bfloat16>(a, tb);
    return launch_fwd_flags<float, float, float, float>(a, tb);
}

int slice_bwd(const BwdArgs& a) {
    if (a.dtype == SPH_F64) {
        const double* tb = static_cast<const double*>(device_tables(SPH_F64));
        if (!tb) return int(cudaErrorMemoryAllocation);
        return launch_bwd<double, false>(a, tb);
    }
    const float* tb = static_cast<const float*>(device_tables(SPH_F32));
    if (!tb) return int(cudaErrorMemoryAllocation);
    return launch_bwd<float, false>(a, tb);
}

int slice_dbwd(const BwdArgs& a) {
    if (a.dtype == SPH_F64) {
        const double* tb = static_cast<const double*>(device_tables(SPH_F64));
        if (!tb) return int(cudaErrorMemoryAllocation);
        return launch_bwd<double, true>(a, tb);
    }
    const float* tb = static_cast<const float*>(device_tables(SPH_F32));
    if (!tb) return int(cudaErrorMemoryAllocation);
    return launch_bwd<float, true>(a, tb);
}

}  // namespace sph
