// ROW Hessians: FP32 values, gradients and Hessians for 0 <= l_max <= 63 on
// the ROW decomposition (see sph_row.cu): 8 lanes per point, lane j owning
// the m channels m = j (mod 8), the degree l outermost and uniform across the
// warp, recursion state in registers, and each point's 13 output rows (value,
// 3 gradient planes, 9 Hessian planes [3][3] row-major) staged in shared
// memory in windows of whole degrees and sent with TMA bulk copies of
// 32-byte-aligned runs.
//
// Per degree d and channel slot k (m = j + 8k) a lane runs one step of
// Eq. iter-q (prefactors folded in, Appendix C) and assembles the +m and -m
// columns of all 13 planes from Eq. iter-deri applied once and twice: the
// terms need Qtilde_{d-1}^{m+1}, Qtilde_{d-2}^{m+1} and Qtilde_{d-2}^{m+2},
// which the lanes holding channels m+1 and m+2 pass with shuffles, and
// c_{m-1}, s_{m-1}, c_{m-2}, s_{m-2} (Eq. iter-sc), kept per slot. The m = 0
// column runs the general assembly with c_0 = 1/sqrt2 and multipliers
// divided by 1/sqrt2 (the table's "unfolded" m = 0 entries); its -m stores
// land on the same column first and are overwritten.
#include <cuda_runtime.h>

#include <algorithm>

#include "sph_core.cuh"
#include "sph_internal.h"

namespace sph {

namespace {

constexpr int kHG = 8;          // lanes per point
constexpr int kHPW = 32 / kHG;  // points per warp
constexpr int kHPlanes = 13;    // value, gradient (3), Hessian (9)
constexpr int kHSE = 8;         // floats per 32-byte sector
constexpr int kHMaxWarps = 2;   // warps per block (the launch bound frees registers)

// Window geometry for a window capacity of CAP columns: a plane buffer holds
// kHSE pre-slots for the row head, then CAP columns; a point's 13 buffers are
// padded so that consecutive points start 8 banks apart.
template <int CAP>
struct HessGeom {
    static constexpr int BUF = kHSE + CAP;  // floats, a multiple of 4
    __host__ __device__ static constexpr int point_stride() {
        constexpr int words = kHPlanes * BUF;
        constexpr int pad = ((8 - words % 32) + 32) % 32;
        return words + pad;
    }
};

template <int CAP>
__host__ __device__ constexpr size_t row_hess_warp_bytes() {
    return size_t(kHPW) * HessGeom<CAP>::point_stride() * sizeof(float);
}

struct CSh {
    float c, s;
    __device__ __forceinline__ CSh times(const CSh& w) const {
        return CSh{fmaf(c, w.c, -(s * w.s)), fmaf(c, w.s, s * w.c)};
    }
};

// The global row of plane i of point p (planes: sph, dsph x/y/z, ddsph [3][3]).
__device__ __forceinline__ float* hess_row(float* sph, float* dsph, float* ddsph, int64_t p, int64_t K, int i) {
    return i == 0 ? sph + p * K : (i < 4 ? dsph + (p * 3 + (i - 1)) * K : ddsph + (p * 9 + (i - 4)) * K);
}

// Staged store of one column's 13 outputs into the plane buffers at column
// index col of the current window (plane i at pst[off[i] + col]).
__device__ __forceinline__ void hess_put(float* __restrict__ pst, const int (&off)[kHPlanes], int col,
                                         const Deriv<float>& d) {
    pst[off[0] + col] = d.v;
    pst[off[1] + col] = d.gx;
    pst[off[2] + col] = d.gy;
    pst[off[3] + col] = d.gz;
    pst[off[4] + col] = d.hxx;
    pst[off[5] + col] = d.hxy;
    pst[off[6] + col] = d.hxz;
    pst[off[7] + col] = d.hxy;
    pst[off[8] + col] = d.hyy;
    pst[off[9] + col] = d.hyz;
    pst[off[10] + col] = d.hxz;
    pst[off[11] + col] = d.hyz;
    pst[off[12] + col] = d.hzz;
}

template <int NCH, bool NORM, int CAP>
__global__ void __launch_bounds__(32 * kHMaxWarps) row_hess_kernel(const float* __restrict__ xyz, int64_t n, int L,
                                                                   const float4* __restrict__ rowA,
                                                                   const float* __restrict__ rowF,
                                                                   const float4* __restrict__ rowG, float inv_sqrt2,
                                                                   float* __restrict__ sph, float* __restrict__ dsph,
                                                                   float* __restrict__ ddsph) {
    // the first degree of a window always fits: 2 l_max + 1 <= 16 NCH - 1 columns
    // plus a carried partial sector
    static_assert(CAP - (kHSE - 1) >= 16 * NCH - 1, "window capacity below one degree");
    constexpr int BUF = HessGeom<CAP>::BUF;
    constexpr int PSTR = HessGeom<CAP>::point_stride();
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const int g = lane / kHG;  // point of the warp tile
    const int j = lane % kHG;  // channel class m = j (mod 8)
    float* const pst = reinterpret_cast<float*>(smem) + (size_t(warp) * kHPW + g) * PSTR;
    const int64_t K = int64_t(L + 1) * (L + 1);
    const int64_t ntiles = (n + kHPW - 1) / kHPW;
    const int nb1 = (lane & ~(kHG - 1)) | ((j + 1) & (kHG - 1));  // holds channel m+1's class
    const int nb2 = (lane & ~(kHG - 1)) | ((j + 2) & (kHG - 1));  // holds channel m+2's class
    const float4* const laneA = rowA + j;
    const float* const laneF = rowF + j;
    const float4* const laneG = rowG + j;

    for (int64_t tile = int64_t(blockIdx.x) * W + warp; tile < ntiles; tile += int64_t(gridDim.x) * W) {
        const int64_t p = tile * kHPW + g;
        const bool live = p < n;
        float x = 0.f, y = 0.f, z = 0.f, ir = 1.f;
        if (live) {
            x = xyz[3 * p];
            y = xyz[3 * p + 1];
            z = xyz[3 * p + 2];
        }
        float r2;
        if (NORM) {
            unit_point(x, y, z, r2, ir);
        } else {
            r2 = fmaf(z, z, fmaf(x, x, y * y));
        }

        // c_m + i s_m, c_{m-1} + i s_{m-1}, c_{m-2} + i s_{m-2} of the lane's
        // channels m = j + 8k (Eq. iter-sc); c_0 of the m = 0 column carries
        // the 1/sqrt2 (its table multipliers are divided by it), the c_0 that
        // channels 1 and 2 reach as c_{m-1}, c_{m-2} is 1.
        float cm[NCH], sm[NCH], cm1[NCH], sm1[NCH], cm2[NCH], sm2[NCH];
        {
            const CSh xy{x, y};
            CSh a{1.f, 0.f}, b{1.f, 0.f}, c{1.f, 0.f}, p6{1.f, 0.f}, p7{1.f, 0.f}, w8{1.f, 0.f};
#pragma unroll
            for (int t = 0; t < kHG; ++t) {
                if (t < j) a = a.times(xy);
                if (t < j - 1) b = b.times(xy);
                if (t < j - 2) c = c.times(xy);
                if (t < 6) p6 = p6.times(xy);
                if (t < 7) p7 = p7.times(xy);
                w8 = w8.times(xy);
            }
            if (j == 0) {  // channels 8k, k >= 1: (x + i y)^(8k-1) and ^(8k-2)
                b = p7;
                c = p6;
            } else if (j == 1) {  // channels 8k + 1, k >= 1: (x + i y)^(8k-1)
                c = p7;
            }
#pragma unroll
            for (int k = 0; k < NCH; ++k) {
                const int m = j + kHG * k;
                cm[k] = m == 0 ? inv_sqrt2 : a.c;
                sm[k] = m == 0 ? 0.f : a.s;
                cm1[k] = m >= 1 ? b.c : 0.f;
                sm1[k] = m >= 1 ? b.s : 0.f;
                cm2[k] = m >= 2 ? c.c : 0.f;
                sm2[k] = m >= 2 ? c.s : 0.f;
                a = a.times(w8);
                if (m >= 1) b = b.times(w8);
                if (m >= 2) c = c.times(w8);
            }
        }
        float q1[NCH], q2[NCH];  // Qtilde_{l-1}^m, Qtilde_{l-2}^m
#pragma unroll
        for (int k = 0; k < NCH; ++k) q1[k] = q2[k] = 0.f;

        // s[i]: first column of plane i held in its buffer (at slot kHSE),
        // 32-byte aligned in global memory.
        int s[kHPlanes];
#pragma unroll
        for (int i = 0; i < kHPlanes; ++i) {
            const float* gr = hess_row(sph, dsph, ddsph, p, K, i);
            const int phase = int((reinterpret_cast<uintptr_t>(gr) / sizeof(float)) % kHSE);
            s[i] = (kHSE - phase) % kHSE;
        }

        // Coefficients of degree 0; with PF, later degrees are loaded one
        // degree ahead (more registers, the loads off the critical path).
        constexpr bool PF = NCH <= 5;
        float4 ta[NCH], tg[NCH];
        float tf[NCH];
        if constexpr (PF) {
#pragma unroll
            for (int k = 0; k < NCH; ++k) {
                ta[k] = laneA[k * kRowLanes];
                tf[k] = laneF[k * kRowLanes];
                tg[k] = laneG[k * kRowLanes];
            }
        }

        int l = 0;
        bool first = true;
        while (l <= L) {
            // A window of whole degrees [l, lw) (the same for the whole warp:
            // the lanes shuffle across point groups); column c of plane i is
            // staged at pst[off[i] + c].
            int off[kHPlanes];
#pragma unroll
            for (int i = 0; i < kHPlanes; ++i) off[i] = i * BUF + kHSE - s[i];
            int d = l;
            while (true) {
                const int ctr = d * d + d;
                const int kend = d / kHG;  // channels m = j + 8k <= d need k <= d/8 (uniform)
                float4 na[PF ? NCH : 1], ng[PF ? NCH : 1];
                float nf[PF ? NCH : 1];
                if constexpr (PF) {
                    const int dn = d < L ? d + 1 : d;
#pragma unroll
                    for (int k = 0; k < NCH; ++k) {
                        const int entn = (dn * kRowSlots + k) * kRowLanes;
                        na[k] = laneA[entn];
                        nf[k] = laneF[entn];
                        ng[k] = laneG[entn];
                    }
                }
#pragma unroll
                for (int k = 0; k < NCH; ++k) {
                    if (k > kend) break;
                    const int ent = (d * kRowSlots + k) * kRowLanes;
                    const float4 t0 = PF ? ta[k] : laneA[ent];  // {A, B, S, e}
                    const float tfk = PF ? tf[k] : laneF[ent];  // f
                    const float4 tgk = PF ? tg[k] : laneG[ent];  // {g2, g3, g4, 0}
                    // what this lane sends for the receivers of channel m+1 (lane j-1, or
                    // lane 7 from lane 0's next slot) and m+2 (lane j-2, or lanes 6, 7
                    // from lanes 0, 1's next slot)
                    const int kn = k + 1 < NCH ? k + 1 : k;
                    const float nx1 = k + 1 < NCH ? q1[kn] : 0.f, nx2 = k + 1 < NCH ? q2[kn] : 0.f;
                    const float q1n = __shfl_sync(0xffffffffu, j == 0 ? nx1 : q1[k], nb1);  // Qtilde_{d-1}^{m+1}
                    const float q2n = __shfl_sync(0xffffffffu, j == 0 ? nx2 : q2[k], nb1);  // Qtilde_{d-2}^{m+1}
                    const float q2nn = __shfl_sync(0xffffffffu, j <= 1 ? nx2 : q2[k], nb2);  // Qtilde_{d-2}^{m+2}
                    // Eq. iter-q (zero for m > d: the table holds zeros there)
                    const float q = fmaf(t0.x * z, q1[k], fmaf(-(t0.y * r2), q2[k], t0.z));
                    const int m = j + kHG * k;
                    if (m <= d) {
                        QParts<float> qp;
                        qp.Q = q;
                        qp.E1 = t0.w * q1n;
                        qp.Qz = tfk * q1[k];
                        qp.G2 = tgk.x * q2nn;
                        qp.G3 = tgk.y * q2n;
                        qp.G4 = tgk.z * q2[k];
                        Deriv<float> dc, ds;
                        assemble_m<true, true>(qp, x, y, float(m), float(m - 1), cm[k], sm[k], cm1[k], sm1[k],
                                               cm2[k], sm2[k], dc, ds);
                        if (NORM) {
                            normalize_deriv<true>(dc, d, x, y, z, ir);
                            normalize_deriv<true>(ds, d, x, y, z, ir);
                        }
                        hess_put(pst, off, ctr - m, ds);  // m = 0: overwritten by the next line
                        hess_put(pst, off, ctr + m, dc);
                    }
                    q2[k] = q1[k];
                    q1[k] = q;
                }
                if constexpr (PF) {
#pragma unroll
                    for (int k = 0; k < NCH; ++k) {
                        ta[k] = na[k];
                        tf[k] = nf[k];
                        tg[k] = ng[k];
                    }
                }
                ++d;
                if (d > L) break;
                if ((d + 1) * (d + 1) - l * l > CAP - (kHSE - 1)) break;
            }
            const int lw = d;

            // Send the window: per plane, the sector-aligned run [s, e) by one
            // bulk copy; the row head (first window) and the row tail (last
            // window) with plain stores; the rest (< one sector) is carried.
            const int c_hi = lw * lw;
            const bool last = lw > L;
            fence_proxy_async_smem();
            __syncwarp();
            int e[kHPlanes];
#pragma unroll
            for (int i = 0; i < kHPlanes; ++i) {
                const int run = last ? (c_hi - s[i]) / 4 * 4 : (c_hi - s[i]) / kHSE * kHSE;
                e[i] = s[i] + max(run, 0);
            }
            if (live) {
                if (j == 0) {
#pragma unroll
                    for (int i = 0; i < kHPlanes; ++i)
                        if (e[i] > s[i])
                            bulk_store(hess_row(sph, dsph, ddsph, p, K, i) + s[i], pst + i * BUF + kHSE,
                                       uint32_t((e[i] - s[i]) * sizeof(float)));
                    bulk_commit();
                }
#pragma unroll
                for (int i = 0; i < kHPlanes; ++i) {
                    float* gr = hess_row(sph, dsph, ddsph, p, K, i);
                    if (first)  // the head, within the row (K < 8 at l_max <= 1)
                        for (int c = j; c < min(s[i], c_hi); c += kHG) gr[c] = pst[i * BUF + c - s[i] + kHSE];
                    if (last)
                        for (int c = e[i] + j; c < c_hi; c += kHG) gr[c] = pst[i * BUF + c - s[i] + kHSE];
                }
                if (j == 0) bulk_wait_read_all();  // the buffers are reused below
            }
            __syncwarp();
            if (!last) {
#pragma unroll
                for (int i = 0; i < kHPlanes; ++i) {
                    for (int c = e[i] + j; c < c_hi; c += kHG) pst[i * BUF + c - e[i] + kHSE] = pst[i * BUF + c - s[i] + kHSE];
                    s[i] = e[i];
                }
                __syncwarp();
            }
            first = false;
            l = lw;
        }
    }
    if (j == 0) bulk_wait_all();
}

template <int NCH, bool NORM, int CAP>
int launch_row_hess(const FwdArgs& a) {
    const float* rt = static_cast<const float*>(device_row_tables());
    if (!rt) return int(cudaErrorMemoryAllocation);
    auto kern = row_hess_kernel<NCH, NORM, CAP>;
    const size_t per_warp = row_hess_warp_bytes<CAP>();
    // default (measured on GB300): 1-warp blocks with the coefficient
    // prefetch (l_max <= 39), 2-warp blocks without it
    const int W = a.launch.warps_per_block > 0 ? a.launch.warps_per_block : (NCH <= 5 ? 1 : kHMaxWarps);
    if (W > kHMaxWarps) return int(cudaErrorInvalidConfiguration);
    const size_t smem = size_t(W) * per_warp;
    if (smem > size_t(max_smem_optin())) return int(cudaErrorInvalidConfiguration);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(kern),
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return int(e);
    }
    int bps = a.launch.blocks_per_sm;
    if (bps <= 0) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, reinterpret_cast<const void*>(kern), 32 * W, smem) !=
            cudaSuccess) {
            cudaGetLastError();
            occ = 1;
        }
        bps = std::max(occ, 1);
    }
    const int64_t ntiles = (a.n + kHPW - 1) / kHPW;
    const int64_t want = (ntiles + W - 1) / W;
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(bps) * sm_count())));
    constexpr int kEntries = kRowLanes * kRowDegrees * kRowSlots;
    kern<<<grid, 32 * W, smem, static_cast<cudaStream_t>(a.stream)>>>(
        static_cast<const float*>(a.xyz), a.n, a.l_max, reinterpret_cast<const float4*>(rt), rt + 4 * kEntries,
        reinterpret_cast<const float4*>(rt + 5 * kEntries), float(host_tables().inv_sqrt2),
        static_cast<float*>(a.sph), static_cast<float*>(a.dsph), static_cast<float*>(a.ddsph));
    return int(cudaGetLastError());
}

// Window capacity (lanes_per_point): 0 or 2 = 136 columns, 1 = the least
// that holds one degree of l_max (16 NCH + 8 columns: the most resident
// warps), 3 = 256 columns (runs of ~1 KB, 4 warps per SM). Measured on GB300
// (FP32, 40k-100k points, l_max 17..63): 136 columns is fastest or equal
// everywhere (2.0-2.9 TB/s; SLICE 1.5-1.9).
template <int NCH, bool NORM>
int launch_row_hess_cap(const FwdArgs& a) {
    const int pol = a.launch.lanes_per_point;
    if (pol == 3) return launch_row_hess<NCH, NORM, 256>(a);
    if (pol == 1) return launch_row_hess<NCH, NORM, 16 * NCH + 8>(a);
    return launch_row_hess<NCH, NORM, 136>(a);
}

template <int NCH>
int launch_row_hess_norm(const FwdArgs& a) {
    return a.normalized ? launch_row_hess_cap<NCH, true>(a) : launch_row_hess_cap<NCH, false>(a);
}

}  // namespace

int row_hess_fwd(const FwdArgs& a) {
    switch ((a.l_max + 1 + kHG - 1) / kHG) {
        case 1:
            return launch_row_hess_norm<1>(a);
        case 2:
            return launch_row_hess_norm<2>(a);
        case 3:
            return launch_row_hess_norm<3>(a);
        case 4:
            return launch_row_hess_norm<4>(a);
        case 5:
            return launch_row_hess_norm<5>(a);
        case 6:
            return launch_row_hess_norm<6>(a);
        case 7:
            return launch_row_hess_norm<7>(a);
        default:
            return launch_row_hess_norm<8>(a);
    }
}

}  // namespace sph
