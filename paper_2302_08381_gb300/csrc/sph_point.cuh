// POINT kernel family: one thread owns one point and runs the whole recursion
// for a compile-time l_max in registers (arXiv 2302.08381, Section 2:
// Eq. iter-sc for c_m/s_m, Eq. iter-q for Q_l^m with the prefactor folded in
// as in Appendix C, Eq. iter-deri for derivatives).
//
// Work decomposition: every warp is independent. It takes tiles of P points
// (P <= 32, lanes >= P idle) from a persistent grid-stride loop. Outputs of a
// tile are contiguous in global memory ([P, K] for sph, [P, 3, K] for dsph), so
// lanes write their rows into a shared-memory image of that range and one lane
// sends it with a bulk (TMA) copy. With K odd (even l_max) the row stride is
// odd and the per-lane stores are bank-conflict free. With K even (odd l_max)
// an image with stride K would put lanes on 4 to 32 times the same bank, so
// rows are padded to an odd stride (K+1, 3K+1) and the warp copies the tile
// out with coalesced plain stores instead. Backward kernels read their [P, K]
// upstream-gradient tile the same way: bulk loads tracked by mbarriers,
// double buffered (odd K), or coalesced plain loads into padded rows (even K).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "sph_core.cuh"
#include "sph_hardcoded.cuh"
#include "sph_internal.h"

namespace sph {

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Tables passed by value as kernel parameters (constant bank), so every
// coefficient is an immediate constant-bank operand of the FMA that uses it.
template <int L, typename T, bool HESS>
struct PointTabs {
    static constexpr int TRI = (L + 1) * (L + 2) / 2;
    static constexpr int TRIH = HESS ? TRI : 1;
    T qll[L + 1];
    T d[L + 1];
    T a[TRI];
    T b[TRI];
    T e[TRI];
    T fz[TRI];
    T g2[TRIH];
    T g3[TRIH];
    T g4[TRIH];
    T inv_sqrt2;
};

template <int L, typename T, bool HESS>
PointTabs<L, T, HESS> make_point_tabs() {
    const HostTables& h = host_tables();
    PointTabs<L, T, HESS> t;
    std::memset(&t, 0, sizeof(t));
    for (int l = 0; l <= L; ++l) {
        t.qll[l] = static_cast<T>(h.qll[tri(l, l)]);
        t.d[l] = (l >= 1) ? static_cast<T>(h.d[tri(l, l - 1)]) : T(0);
        for (int m = 0; m <= l; ++m) {
            const int i = tri(l, m);
            t.a[i] = static_cast<T>(h.a[i]);
            t.b[i] = static_cast<T>(h.b[i]);
            t.e[i] = static_cast<T>(h.e[i]);
            t.fz[i] = static_cast<T>(h.fz[i]);
            if (HESS) {
                t.g2[i] = static_cast<T>(h.g2[i]);
                t.g3[i] = static_cast<T>(h.g3[i]);
                t.g4[i] = static_cast<T>(h.g4[i]);
            }
        }
    }
    t.inv_sqrt2 = static_cast<T>(h.inv_sqrt2);
    return t;
}

// The unrolled recursion for one point from degree L0 on. (x, y, z, r2) are
// the coordinates the polynomials are evaluated at (already divided by r for
// the normalized form); c, s hold c_m, s_m for m <= L; q1, q2 hold
// Qtilde_{L0-1}^m and Qtilde_{L0-2}^m (zero for m beyond the degree).
// Calls vis.emit(l, k, Deriv) once per output column k = l*l + l + m, l >= L0.
template <int L, int L0, bool GRAD, bool HESS, typename T, typename Tabs, typename Vis>
__device__ __forceinline__ void point_core_from(T x, T y, T z, T r2, const Tabs& tb, Vis& vis, const T (&c)[L + 1],
                                                const T (&s)[L + 1], T (&q1)[L + 1], T (&q2)[L + 1]) {
#pragma unroll
    for (int l = L0; l <= L; ++l) {
        T q[L + 1];
        q[l] = tb.qll[l];
        if (l >= 1) q[l - 1] = tb.d[l] * z * q1[l - 1];
#pragma unroll
        for (int m = 0; m + 2 <= l; ++m) {  // Eq. iter-q, folded
            const int i = tri(l, m);
            q[m] = (tb.a[i] * z) * q1[m] - (tb.b[i] * r2) * q2[m];
        }
#pragma unroll
        for (int m = 0; m <= l; ++m) {
            const int i = tri(l, m);
            QParts<T> qp;
            qp.Q = q[m];
            qp.E1 = (m + 1 <= l - 1) ? tb.e[i] * q1[m + 1] : T(0);
            qp.Qz = (m <= l - 1) ? tb.fz[i] * q1[m] : T(0);
            if constexpr (HESS) {
                qp.G2 = (m + 2 <= l - 2) ? tb.g2[i] * q2[m + 2] : T(0);
                qp.G3 = (m + 1 <= l - 2) ? tb.g3[i] * q2[m + 1] : T(0);
                qp.G4 = (m <= l - 2) ? tb.g4[i] * q2[m] : T(0);
            } else {
                qp.G2 = qp.G3 = qp.G4 = T(0);
            }
            if (m == 0) {
                Deriv<T> d = assemble_m0<GRAD, HESS>(qp, x, y, tb.inv_sqrt2);
                vis.emit(l, l * l + l, d);
            } else {
                Deriv<T> dc, ds;
                const T cm2 = (m >= 2) ? c[m >= 2 ? m - 2 : 0] : T(0);
                const T sm2 = (m >= 2) ? s[m >= 2 ? m - 2 : 0] : T(0);
                assemble_m<GRAD, HESS>(qp, x, y, T(m), T(m - 1), c[m], s[m], c[m - 1], s[m - 1], cm2, sm2, dc,
                                       ds);
                vis.emit(l, l * l + l + m, dc);
                vis.emit(l, l * l + l - m, ds);
            }
        }
#pragma unroll
        for (int m = 0; m <= l; ++m) {
            q2[m] = q1[m];
            q1[m] = q[m];
        }
    }
}

template <int L, typename T>
__device__ __forceinline__ void point_cs(T x, T y, T (&c)[L + 1], T (&s)[L + 1]) {
    c[0] = T(1);
    s[0] = T(0);
#pragma unroll
    for (int m = 1; m <= L; ++m) {  // Eq. iter-sc
        c[m] = x * c[m - 1] - y * s[m - 1];
        s[m] = x * s[m - 1] + y * c[m - 1];
    }
}

// The whole recursion for one point (every degree from 0).
template <int L, bool GRAD, bool HESS, typename T, typename Tabs, typename Vis>
__device__ __forceinline__ void point_core(T x, T y, T z, T r2, const Tabs& tb, Vis& vis) {
    T c[L + 1], s[L + 1];
    point_cs<L>(x, y, c, s);
    T q1[L + 1], q2[L + 1];  // Qtilde_{l-1}^m, Qtilde_{l-2}^m
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        q1[m] = T(0);
        q2[m] = T(0);
    }
    point_core_from<L, 0, GRAD, HESS>(x, y, z, r2, tb, vis, c, s, q1, q2);
}

// Hybrid (Section 3.2: hard-coded low degrees, the general recursion above):
// degrees l <= min(L, 3) from the generated straight-line expressions of
// sph_hardcoded.cuh, which also give Qtilde_LH^m and Qtilde_{LH-1}^m, and
// Eq. iter-q from degree LH + 1. Values and gradients (no Hessians).
template <int L, bool GRAD, typename T, typename Tabs, typename Vis>
__device__ __forceinline__ void point_core_hc(T x, T y, T z, T r2, const Tabs& tb, Vis& vis) {
    constexpr int LH = L < 3 ? L : 3;
    T qa[4] = {T(0), T(0), T(0), T(0)}, qb[4] = {T(0), T(0), T(0), T(0)};
    if constexpr (LH == 0) {
        if constexpr (GRAD) hardcoded_l0_grad(x, y, z, r2, vis, qa, qb); else hardcoded_l0_val(x, y, z, r2, vis, qa, qb);
    } else if constexpr (LH == 1) {
        if constexpr (GRAD) hardcoded_l1_grad(x, y, z, r2, vis, qa, qb); else hardcoded_l1_val(x, y, z, r2, vis, qa, qb);
    } else if constexpr (LH == 2) {
        if constexpr (GRAD) hardcoded_l2_grad(x, y, z, r2, vis, qa, qb); else hardcoded_l2_val(x, y, z, r2, vis, qa, qb);
    } else {
        if constexpr (GRAD) hardcoded_l3_grad(x, y, z, r2, vis, qa, qb); else hardcoded_l3_val(x, y, z, r2, vis, qa, qb);
    }
    if constexpr (L > LH) {
        T c[L + 1], s[L + 1];
        point_cs<L>(x, y, c, s);
        T q1[L + 1], q2[L + 1];
#pragma unroll
        for (int m = 0; m <= L; ++m) {
            q1[m] = m <= LH ? qa[m <= LH ? m : 0] : T(0);
            q2[m] = m <= LH - 1 ? qb[m <= LH - 1 ? m : 0] : T(0);
        }
        point_core_from<L, LH + 1, GRAD, false>(x, y, z, r2, tb, vis, c, s, q1, q2);
    }
}

// ------------------------------------------------------------------ forward
template <typename T, typename TO, bool GRAD, bool HESS, bool NORM, int K>
struct FwdVis {
    TO* rv;  // this lane's sph row in shared memory
    TO* rd;  // this lane's dsph row (3 planes of K)
    TO* rh;  // this lane's ddsph row (9 planes of K, i-major)
    T ux, uy, uz, ir;
    __device__ __forceinline__ void emit(int l, int k, Deriv<T> d) {
        if (GRAD || HESS) {
            if (NORM) normalize_deriv<HESS>(d, l, ux, uy, uz, ir);
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
        rv[k] = OutConv<TO>::cv(d.v);
    }
};

// Shared-memory row strides (elements) of a tile: the contiguous image for
// odd K, odd-padded rows for even K.
template <int L>
struct RowStride {
    static constexpr int K = (L + 1) * (L + 1);
    static constexpr bool PAD = (K % 2 == 0);
    static constexpr int V = PAD ? K + 1 : K;          // sph / g rows
    static constexpr int D = PAD ? 3 * K + 1 : 3 * K;  // dsph rows
    static constexpr int H = PAD ? 9 * K + 1 : 9 * K;  // ddsph rows
};

template <int L, bool GRAD, bool HESS, typename TO>
__host__ __device__ constexpr size_t point_fwd_warp_bytes(int P) {
    return align16(size_t(P) * RowStride<L>::V * sizeof(TO)) +
           (GRAD ? align16(size_t(P) * RowStride<L>::D * sizeof(TO)) : 0) +
           (HESS ? align16(size_t(P) * RowStride<L>::H * sizeof(TO)) : 0);
}

// Copies `rows` rows of `cols` elements from a padded shared-memory image
// (row stride `stride`) to a contiguous global range, 32 consecutive
// elements per warp store.
template <int cols, typename TO>
__device__ __forceinline__ void warp_rows_out(TO* __restrict__ gdst, const TO* __restrict__ ssrc, int rows, int stride,
                                              int lane) {
    const int total = rows * cols;
    for (int i = lane; i < total; i += 32) {
        const int r = i / cols;
        gdst[i] = ssrc[r * stride + (i - r * cols)];
    }
}

template <int cols, typename T>
__device__ __forceinline__ void warp_rows_in(T* __restrict__ sdst, const T* __restrict__ gsrc, int rows, int stride,
                                             int lane) {
    const int total = rows * cols;
    for (int i = lane; i < total; i += 32) {
        const int r = i / cols;
        sdst[r * stride + (i - r * cols)] = gsrc[i];
    }
}

template <int L, bool GRAD, bool HESS, bool NORM, typename T, typename TO, bool HC = false>
__global__ void __launch_bounds__(256) point_fwd_kernel(const T* __restrict__ xyz, int64_t n,
                                                        const __grid_constant__ PointTabs<L, T, HESS> tb,
                                                        TO* __restrict__ sph, TO* __restrict__ dsph,
                                                        TO* __restrict__ ddsph, int P, int bulk) {
    constexpr int K = (L + 1) * (L + 1);
    using RS = RowStride<L>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const size_t vbytes = align16(size_t(P) * RS::V * sizeof(TO));
    TO* s_v = reinterpret_cast<TO*>(smem + size_t(warp) * point_fwd_warp_bytes<L, GRAD, HESS, TO>(P));
    TO* s_d = reinterpret_cast<TO*>(reinterpret_cast<unsigned char*>(s_v) + vbytes);
    TO* s_h = reinterpret_cast<TO*>(reinterpret_cast<unsigned char*>(s_d) +
                                    (GRAD ? align16(size_t(P) * RS::D * sizeof(TO)) : 0));

    const int64_t ntiles = (n + P - 1) / P;
    const int64_t stride = int64_t(gridDim.x) * W;
    int64_t tile = int64_t(blockIdx.x) * W + warp;

    // Software-pipelined coordinate loads: the next tile's point is fetched
    // while the current one is computed.
    T nx = T(0), ny = T(0), nz = T(0);
    if (tile < ntiles && lane < P) {
        const int64_t p = tile * P + lane;
        if (p < n) {
            nx = xyz[3 * p];
            ny = xyz[3 * p + 1];
            nz = xyz[3 * p + 2];
        }
    }
    for (; tile < ntiles; tile += stride) {
        T x = nx, y = ny, z = nz;
        const int64_t nt = tile + stride;
        if (nt < ntiles && lane < P) {
            const int64_t p = nt * P + lane;
            if (p < n) {
                nx = xyz[3 * p];
                ny = xyz[3 * p + 1];
                nz = xyz[3 * p + 2];
            }
        }
        const int64_t p0 = tile * P;
        const int cnt = int(min(int64_t(P), n - p0));
        if (lane < cnt) {
            T r2, ir = T(1);
            if (NORM) {
                unit_point(x, y, z, r2, ir);
            } else {
                r2 = x * x + y * y + z * z;
            }
            FwdVis<T, TO, GRAD, HESS, NORM, K> vis{s_v + size_t(lane) * RS::V, s_d + size_t(lane) * RS::D,
                                                   s_h + size_t(lane) * RS::H, x, y, z, ir};
            if constexpr (HC && !HESS)
                point_core_hc<L, GRAD>(x, y, z, r2, tb, vis);
            else
                point_core<L, GRAD, HESS>(x, y, z, r2, tb, vis);
        }
        if constexpr (RS::PAD) {
            __syncwarp();
            warp_rows_out<K>(sph + p0 * K, s_v, cnt, RS::V, lane);
            if (GRAD) warp_rows_out<3 * K>(dsph + p0 * 3 * K, s_d, cnt, RS::D, lane);
            if (HESS) warp_rows_out<9 * K>(ddsph + p0 * 9 * K, s_h, cnt, RS::H, lane);
            __syncwarp();
            continue;
        }
        fence_proxy_async_smem();
        __syncwarp();
        const int64_t ev = int64_t(cnt) * K;  // elements of the sph tile
        int64_t ev_bulk = 0, ed_bulk = 0, eh_bulk = 0;
        if (bulk) {
            ev_bulk = (ev * int64_t(sizeof(TO))) / 16 * 16 / int64_t(sizeof(TO));
            ed_bulk = GRAD ? (3 * ev * int64_t(sizeof(TO))) / 16 * 16 / int64_t(sizeof(TO)) : 0;
            eh_bulk = HESS ? (9 * ev * int64_t(sizeof(TO))) / 16 * 16 / int64_t(sizeof(TO)) : 0;
            if (lane == 0) {
                if (ev_bulk) bulk_store(sph + p0 * K, s_v, uint32_t(ev_bulk * sizeof(TO)));
                if (GRAD && ed_bulk) bulk_store(dsph + p0 * 3 * K, s_d, uint32_t(ed_bulk * sizeof(TO)));
                if (HESS && eh_bulk) bulk_store(ddsph + p0 * 9 * K, s_h, uint32_t(eh_bulk * sizeof(TO)));
                bulk_commit();
            }
        }
        // Ragged remainder (and everything, without bulk copies): plain stores.
        for (int64_t i = ev_bulk + lane; i < ev; i += 32) sph[p0 * K + i] = s_v[i];
        if (GRAD)
            for (int64_t i = ed_bulk + lane; i < 3 * ev; i += 32) dsph[p0 * 3 * K + i] = s_d[i];
        if (HESS)
            for (int64_t i = eh_bulk + lane; i < 9 * ev; i += 32) ddsph[p0 * 9 * K + i] = s_h[i];
        if (bulk && lane == 0) bulk_wait_read_all();
        __syncwarp();
    }
    if (bulk && lane == 0) bulk_wait_all();
}

// -------------------------------------- forward, 4 lanes per point (planes)
// POINT with lanes_per_point = 4 (values and gradients): lane 4j + r of a
// warp owns output plane r (0 the value, 1..3 d/dx, d/dy, d/dz) of the tile's
// point j, so a tile of 8 points keeps all 32 lanes busy where the
// one-lane-per-point tile that fits shared memory at large l_max holds only
// 8 to 16 points. Every lane runs the Q recursion (Eq. iter-q) and Eq.
// iter-sc in full (cheap next to the assembly) and assembles only its plane
// with role weights, the same instruction stream in every lane:
//   plane = A c_m + m Qtilde_l^m C'_m,   A = a0 Qtilde + ax e Qtilde_{l-1}^{m+1} + a3 f Qtilde_{l-1}^m
// (a0, ax, a3) = (1, 0, 0), (0, x, 0), (0, y, 0), (0, 0, 1) by role, and
// C'_m = c_{m-1} (d/dx), -s_{m-1} (d/dy), 0 (value, d/dz); the sin-type column
// takes s_m and S'_m = s_{m-1}, c_{m-1}, 0. These are the terms of Eq.
// iter-deri that assemble_m combines for all four planes at once.
template <int L, bool NORM, typename T, typename TO, typename Tabs>
__device__ __forceinline__ void point4_core(T x, T y, T z, T r2, const Tabs& tb, int r, T ir,
                                            TO* __restrict__ rowp) {
    const T a0 = r == 0 ? T(1) : T(0);
    const T ax = r == 1 ? x : (r == 2 ? y : T(0));
    const T a3 = r == 3 ? T(1) : T(0);
    const T a00 = a0 * tb.inv_sqrt2;  // m = 0 value: Qtilde_l^0 / sqrt2
    T c[L + 1], s[L + 1];
    point_cs<L>(x, y, c, s);
    T c1[L + 1], s1[L + 1];  // (C'_m, S'_m) of this lane's role
    {
        const T k1 = r == 1 ? T(1) : T(0), k2 = r == 2 ? T(-1) : T(0);
        const T k3 = r == 2 ? T(1) : T(0), k4 = r == 1 ? T(1) : T(0);
        c1[0] = T(0);
        s1[0] = T(0);
#pragma unroll
        for (int m = 1; m <= L; ++m) {
            c1[m] = k1 * c[m - 1] + k2 * s[m - 1];
            s1[m] = k3 * c[m - 1] + k4 * s[m - 1];
        }
    }
    // Normalized form (x, y, z = u): plane' = irr (plane - l u_r value), with
    // u_r = 0 and irr = 1 for the value plane.
    const T nu = NORM ? -(r == 1 ? x : (r == 2 ? y : (r == 3 ? z : T(0)))) : T(0);
    const T irr = (NORM && r != 0) ? ir : T(1);
    T q1[L + 1], q2[L + 1];
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        q1[m] = T(0);
        q2[m] = T(0);
    }
#pragma unroll
    for (int l = 0; l <= L; ++l) {
        T q[L + 1];
        q[l] = tb.qll[l];
        if (l >= 1) q[l - 1] = tb.d[l] * z * q1[l - 1];
#pragma unroll
        for (int m = 0; m + 2 <= l; ++m) {  // Eq. iter-q, folded
            const int i = tri(l, m);
            q[m] = (tb.a[i] * z) * q1[m] - (tb.b[i] * r2) * q2[m];
        }
        const T nl = nu * T(l);
#pragma unroll
        for (int m = 0; m <= l; ++m) {
            const int i = tri(l, m);
            const T E1 = (m + 1 <= l - 1) ? tb.e[i] * q1[m + 1] : T(0);
            const T Qz = (m <= l - 1) ? tb.fz[i] * q1[m] : T(0);
            if (m == 0) {
                T out = a00 * q[0] + ax * E1 + a3 * Qz;
                if (NORM) out = irr * fma(nl, q[0] * tb.inv_sqrt2, out);
                rowp[l * l + l] = OutConv<TO>::cv(out);
            } else {
                const T A = a0 * q[m] + ax * E1 + a3 * Qz;
                const T mQ = T(m) * q[m];
                T oc = A * c[m] + mQ * c1[m];
                T os = A * s[m] + mQ * s1[m];
                if (NORM) {
                    oc = irr * fma(nl, q[m] * c[m], oc);
                    os = irr * fma(nl, q[m] * s[m], os);
                }
                rowp[l * l + l + m] = OutConv<TO>::cv(oc);
                rowp[l * l + l - m] = OutConv<TO>::cv(os);
            }
        }
#pragma unroll
        for (int m = 0; m <= l; ++m) {
            q2[m] = q1[m];
            q1[m] = q[m];
        }
    }
}

// Shared-memory image of a 4-lane tile: P value rows and 3P gradient plane
// rows of stride S (point4_stride): MODE 0 the image of the global ranges
// (one bulk copy per array), 1 rows at 16-byte-aligned strides (one bulk copy
// per row, issued by the lane that wrote it), 2 padded rows copied out by the
// warp with coalesced stores.
template <int L, typename TO>
struct Row4 {
    static constexpr int K = (L + 1) * (L + 1);
    static constexpr int S = point4_stride(L, int(sizeof(TO)));
    static constexpr int MODE = point4_out_mode(L, int(sizeof(TO)));
};

template <int L, typename TO>
__host__ __device__ constexpr size_t point4_warp_bytes(int P) {
    return align16(size_t(P) * Row4<L, TO>::S * sizeof(TO)) + align16(size_t(3 * P) * Row4<L, TO>::S * sizeof(TO));
}

// One tile of a set: points [p0, p0 + cnt), cnt <= P <= 8, lane 4j + r
// computing plane r of point j at (x, y, z); outputs staged at buf
// (point4_warp_bytes<L, TO>(P) bytes) and sent to the set's sph / dsph.
// Warp-collective; returns with the staging buffer free for the next tile.
template <int L, bool NORM, typename T, typename TO, typename Tabs>
__device__ __forceinline__ void point4_tile(TO* __restrict__ sph, TO* __restrict__ dsph, int64_t p0, int cnt, int P,
                                            int bulk, unsigned char* buf, const Tabs& tb, int lane, T x, T y, T z) {
    constexpr int K = (L + 1) * (L + 1);
    constexpr int S = Row4<L, TO>::S;
    constexpr int MODE = Row4<L, TO>::MODE;
    const int pt = lane >> 2, r = lane & 3;
    TO* s_v = reinterpret_cast<TO*>(buf);
    TO* s_d = reinterpret_cast<TO*>(buf + align16(size_t(P) * S * sizeof(TO)));
    TO* rowp = r == 0 ? s_v + size_t(pt) * S : s_d + size_t(3 * pt + r - 1) * S;
    if (pt < cnt) {
        T r2, ir = T(1);
        if (NORM) {
            unit_point(x, y, z, r2, ir);
        } else {
            r2 = x * x + y * y + z * z;
        }
        point4_core<L, NORM>(x, y, z, r2, tb, r, ir, rowp);
    }
    if constexpr (MODE == 1) {
        if (bulk) {  // each lane sends the row it wrote (16-byte aligned at both ends)
            if (pt < cnt) {
                fence_proxy_async_smem();
                TO* g = r == 0 ? sph + (p0 + pt) * K : dsph + ((p0 + pt) * 3 + (r - 1)) * K;
                bulk_store(g, rowp, uint32_t(K * sizeof(TO)));
                bulk_commit();
                bulk_wait_read_all();
            }
            __syncwarp();
            return;
        }
    }
    if constexpr (MODE != 0) {
        __syncwarp();
        warp_rows_out<K>(sph + p0 * K, s_v, cnt, S, lane);
        warp_rows_out<K>(dsph + p0 * 3 * K, s_d, 3 * cnt, S, lane);
        __syncwarp();
        return;
    }
    fence_proxy_async_smem();
    __syncwarp();
    const int64_t ev = int64_t(cnt) * K;
    int64_t ev_bulk = 0, ed_bulk = 0;
    if (bulk) {
        ev_bulk = (ev * int64_t(sizeof(TO))) / 16 * 16 / int64_t(sizeof(TO));
        ed_bulk = (3 * ev * int64_t(sizeof(TO))) / 16 * 16 / int64_t(sizeof(TO));
        if (lane == 0) {
            if (ev_bulk) bulk_store(sph + p0 * K, s_v, uint32_t(ev_bulk * sizeof(TO)));
            if (ed_bulk) bulk_store(dsph + p0 * 3 * K, s_d, uint32_t(ed_bulk * sizeof(TO)));
            bulk_commit();
        }
    }
    for (int64_t i = ev_bulk + lane; i < ev; i += 32) sph[p0 * K + i] = s_v[i];
    for (int64_t i = ed_bulk + lane; i < 3 * ev; i += 32) dsph[p0 * 3 * K + i] = s_d[i];
    if (bulk && lane == 0) bulk_wait_read_all();
    __syncwarp();
}

template <int L, bool NORM, typename T, typename TO>
__global__ void __launch_bounds__(256) point4_fwd_kernel(const T* __restrict__ xyz, int64_t n,
                                                         const __grid_constant__ PointTabs<L, T, false> tb,
                                                         TO* __restrict__ sph, TO* __restrict__ dsph, int P,
                                                         int bulk) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const int pt = lane >> 2;
    unsigned char* buf = smem + size_t(warp) * point4_warp_bytes<L, TO>(P);

    const int64_t ntiles = (n + P - 1) / P;
    const int64_t stride = int64_t(gridDim.x) * W;
    int64_t tile = int64_t(blockIdx.x) * W + warp;
    T nx = T(0), ny = T(0), nz = T(0);
    if (tile < ntiles && pt < P) {
        const int64_t p = tile * P + pt;
        if (p < n) {
            nx = xyz[3 * p];
            ny = xyz[3 * p + 1];
            nz = xyz[3 * p + 2];
        }
    }
    for (; tile < ntiles; tile += stride) {
        const T x = nx, y = ny, z = nz;
        const int64_t nt = tile + stride;
        if (nt < ntiles && pt < P) {
            const int64_t p = nt * P + pt;
            if (p < n) {
                nx = xyz[3 * p];
                ny = xyz[3 * p + 1];
                nz = xyz[3 * p + 2];
            }
        }
        const int64_t p0 = tile * P;
        const int cnt = int(min(int64_t(P), n - p0));
        point4_tile<L, NORM>(sph, dsph, p0, cnt, P, bulk, buf, tb, lane, x, y, z);
    }
    if (bulk) bulk_wait_all();  // every lane: row copies are issued per lane
}

// ------------------------- forward with Hessians, 16 lanes per point (planes)
// POINT with lanes_per_point = 16 (FP32 values, gradients and Hessians):
// lane 16j + r owns output plane r of point j of the current pair of points
// (0 the value, 1..3 the gradient, 4..12 the Hessian entries (i, k) row-major;
// lanes 13..15 compute plane 12 again and store nothing). Every lane runs the
// recursions in full and assembles its plane from one instance of the terms
// of Eq. iter-deri applied once and twice:
//   plane = A C + m B T1 + m (m - 1) Qtilde_l^m T2
//   A = aQ Qtilde + aE e Qtilde_{l-1}^{m+1} + az f Qtilde_{l-1}^m
//       + a2 g2 Qtilde_{l-2}^{m+2} + a3 g3 Qtilde_{l-2}^{m+1} + a4 g4 Qtilde_{l-2}^m
//   B = bQ Qtilde + bE e Qtilde_{l-1}^{m+1} + bz f Qtilde_{l-1}^m
// with C = c_m (or s_m for the sin-type column), T1 a role combination of
// c_{m-1}, s_{m-1} and T2 of c_{m-2}, s_{m-2} (the derivatives of c_m, s_m),
// role weights from the point's coordinates. The normalized form needs the
// value and two gradient components of the same column: taken from the
// point's lanes 0 and 1 + i by warp shuffles.
template <int L, bool NORM, bool TWO = false, typename Tabs>
__device__ __forceinline__ void point16_core(float x, float y, float z, float r2, const Tabs& tb, int rr, int base,
                                             float ir, float* __restrict__ rowp, float* __restrict__ rowp2,
                                             bool store) {
    const int hi = rr >= 4 ? (rr - 4) / 3 : 0, hk = rr >= 4 ? (rr - 4) % 3 : 0;
    // the symmetric entry (i, k) with i <= k selects the formula
    const int i0 = hi < hk ? hi : hk, k0 = hi < hk ? hk : hi;
    const bool isv = rr == 0, isgx = rr == 1, isgy = rr == 2, isgz = rr == 3, ish = rr >= 4;
    const bool hxx = ish && i0 == 0 && k0 == 0, hxy = ish && i0 == 0 && k0 == 1, hxz = ish && i0 == 0 && k0 == 2;
    const bool hyy = ish && i0 == 1 && k0 == 1, hyz = ish && i0 == 1 && k0 == 2, hzz = ish && i0 == 2 && k0 == 2;
    const float X = x, Y = y;
    const float aQ = isv ? 1.f : 0.f;
    const float aE = isgx ? X : (isgy ? Y : ((hxx || hyy) ? 1.f : 0.f));
    const float az = isgz ? 1.f : 0.f;
    const float a2 = hxx ? X * X : (hyy ? Y * Y : (hxy ? X * Y : 0.f));
    const float a3 = hxz ? X : (hyz ? Y : 0.f);
    const float a4 = hzz ? 1.f : 0.f;
    const float bQ = (isgx || isgy) ? 1.f : 0.f;
    const float bE = (hxx || hyy || hxy) ? 1.f : 0.f;
    const float bz = (hxz || hyz) ? 1.f : 0.f;
    // T1c = k1c c1 + k1s s1, T1s = k2c c1 + k2s s1, T2c = k3c c2 + k3s s2, T2s = k4c c2 + k4s s2
    float k1c = 0.f, k1s = 0.f, k2c = 0.f, k2s = 0.f, k3c = 0.f, k3s = 0.f, k4c = 0.f, k4s = 0.f;
    if (isgx || hxz) {
        k1c = 1.f;
        k2s = 1.f;
    } else if (isgy || hyz) {
        k1s = -1.f;
        k2c = 1.f;
    } else if (hxx) {
        k1c = 2.f * X;
        k2s = 2.f * X;
        k3c = 1.f;
        k4s = 1.f;
    } else if (hyy) {
        k1s = -2.f * Y;
        k2c = 2.f * Y;
        k3c = -1.f;
        k4s = -1.f;
    } else if (hxy) {
        k1c = Y;
        k1s = -X;
        k2c = X;
        k2s = Y;
        k3s = -1.f;
        k4c = 1.f;
    }
    float c[L + 1], s[L + 1];
    point_cs<L>(x, y, c, s);
    // Normalized form: plane' = sc (plane + wv v + wi g_i + wk g_k), v and g from
    // the point's lanes 0 and 1 + i / 1 + k (raw values at the unit point).
    // (i0, k0) for both (i, k) and (k, i): the two planes of a symmetric pair
    // run the same operations and come out bit-identical; `base` is the lane
    // of the point's value plane, base + 1 + i that of gradient component i
    const int src_i = base + 1 + i0, src_k = base + 1 + k0;
    const float ui = i0 == 0 ? x : (i0 == 1 ? y : z), uk = k0 == 0 ? x : (k0 == 1 ? y : z);
    const float ug = isgx ? x : (isgy ? y : z);  // gradient planes: u of their component
    const float sc = !NORM || isv ? 1.f : (ish ? ir * ir : ir);
    float q1[L + 1], q2[L + 1];
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        q1[m] = 0.f;
        q2[m] = 0.f;
    }
#pragma unroll
    for (int l = 0; l <= L; ++l) {
        float q[L + 1];
        q[l] = tb.qll[l];
        if (l >= 1) q[l - 1] = tb.d[l] * z * q1[l - 1];
#pragma unroll
        for (int m = 0; m + 2 <= l; ++m) {  // Eq. iter-q, folded
            const int i = tri(l, m);
            q[m] = (tb.a[i] * z) * q1[m] - (tb.b[i] * r2) * q2[m];
        }
        const float lf = float(l);
        // normalization weights of this degree
        float wv = 0.f, wi = 0.f, wk = 0.f;
        if (NORM) {
            if (ish) {
                wv = lf * (lf + 2.f) * ui * uk - (i0 == k0 ? lf : 0.f);
                wi = -lf * uk;
                wk = -lf * ui;
            } else if (!isv) {
                wv = -lf * ug;
            }
        }
#pragma unroll
        for (int m = 0; m <= l; ++m) {
            const int i = tri(l, m);
            const float E1 = (m + 1 <= l - 1) ? tb.e[i] * q1[m + 1] : 0.f;
            const float Qz = (m <= l - 1) ? tb.fz[i] * q1[m] : 0.f;
            const float G2 = (m + 2 <= l - 2) ? tb.g2[i] * q2[m + 2] : 0.f;
            const float G3 = (m + 1 <= l - 2) ? tb.g3[i] * q2[m + 1] : 0.f;
            const float G4 = (m <= l - 2) ? tb.g4[i] * q2[m] : 0.f;
            const float A = aE * E1 + az * Qz + a2 * G2 + a3 * G3 + a4 * G4;
            if (m == 0) {
                float out = aQ * tb.inv_sqrt2 * q[0] + A;
                if (NORM) {
                    const float v = __shfl_sync(0xffffffffu, out, base);
                    const float gi = __shfl_sync(0xffffffffu, out, src_i);
                    const float gk = __shfl_sync(0xffffffffu, out, src_k);
                    out = sc * (out + wv * v + wi * gi + wk * gk);
                }
                if (store) {
                    rowp[l * l + l] = out;
                    if (TWO) rowp2[l * l + l] = out;
                }
            } else {
                const float Am = aQ * q[m] + A;
                const float mB = float(m) * (bQ * q[m] + bE * E1 + bz * Qz);
                const float MQ = float(m * (m - 1)) * q[m];
                const float c1 = c[m - 1], s1 = s[m - 1];
                const float c2 = m >= 2 ? c[m >= 2 ? m - 2 : 0] : 0.f, s2 = m >= 2 ? s[m >= 2 ? m - 2 : 0] : 0.f;
                float oc = Am * c[m] + mB * (k1c * c1 + k1s * s1);
                float os = Am * s[m] + mB * (k2c * c1 + k2s * s1);
                if (m >= 2) {
                    oc += MQ * (k3c * c2 + k3s * s2);
                    os += MQ * (k4c * c2 + k4s * s2);
                }
                if (NORM) {
                    const float vc = __shfl_sync(0xffffffffu, oc, base);
                    const float gic = __shfl_sync(0xffffffffu, oc, src_i);
                    const float gkc = __shfl_sync(0xffffffffu, oc, src_k);
                    const float vs = __shfl_sync(0xffffffffu, os, base);
                    const float gis = __shfl_sync(0xffffffffu, os, src_i);
                    const float gks = __shfl_sync(0xffffffffu, os, src_k);
                    oc = sc * (oc + wv * vc + wi * gic + wk * gkc);
                    os = sc * (os + wv * vs + wi * gis + wk * gks);
                }
                if (store) {
                    rowp[l * l + l + m] = oc;
                    rowp[l * l + l - m] = os;
                    if (TWO) {
                        rowp2[l * l + l + m] = oc;
                        rowp2[l * l + l - m] = os;
                    }
                }
            }
        }
#pragma unroll
        for (int m = 0; m <= l; ++m) {
            q2[m] = q1[m];
            q1[m] = q[m];
        }
    }
}

// Shared-memory bytes of a 16-lane Hessian tile of P points: value rows,
// gradient rows and Hessian rows, each part 16-byte aligned, stride
// point4_stride (the same rules as the 4-lane tile).
template <int L>
__host__ __device__ constexpr size_t point16_warp_bytes(int P) {
    constexpr size_t S = size_t(point4_stride(L, 4)) * 4;
    return align16(size_t(P) * S) + align16(size_t(3 * P) * S) + align16(size_t(9 * P) * S);
}

constexpr int kPoint16MaxTile = 8;  // points per tile (pairs of points per pass)

// One tile of P <= 8 points (P even): the warp computes two points per pass,
// 16 lanes each, into the staged image; warp-collective.
template <int L, bool NORM, typename Tabs>
__device__ __forceinline__ void point16_tile(const float* __restrict__ xyz, float* __restrict__ sph,
                                             float* __restrict__ dsph, float* __restrict__ ddsph, int64_t p0,
                                             int cnt, int P, int bulk, unsigned char* buf, const Tabs& tb,
                                             int lane) {
    constexpr int K = (L + 1) * (L + 1);
    constexpr int S = point4_stride(L, 4);
    constexpr int MODE = point4_out_mode(L, 4);
    float* s_v = reinterpret_cast<float*>(buf);
    float* s_d = reinterpret_cast<float*>(buf + align16(size_t(P) * S * 4));
    float* s_h = reinterpret_cast<float*>(buf + align16(size_t(P) * S * 4) + align16(size_t(3 * P) * S * 4));
    const int r = lane & 15, half = lane >> 4;
    // coordinates of every pass of the tile, loaded up front
    float cx[kPoint16MaxTile / 2], cy[kPoint16MaxTile / 2], cz[kPoint16MaxTile / 2];
#pragma unroll
    for (int t = 0; t < kPoint16MaxTile / 2; ++t) {
        const int j = 2 * t + half;
        cx[t] = 0.f;
        cy[t] = 0.f;
        cz[t] = 1.f;  // points past the end run on a unit vector and are not sent
        if (2 * t < P && j < cnt) {
            cx[t] = xyz[3 * (p0 + j)];
            cy[t] = xyz[3 * (p0 + j) + 1];
            cz[t] = xyz[3 * (p0 + j) + 2];
        }
    }
#pragma unroll
    for (int t = 0; t < kPoint16MaxTile / 2; ++t) {
        if (2 * t >= P) break;
        const int j = 2 * t + half;
        float x = cx[t], y = cy[t], z = cz[t], r2, ir = 1.f;
        if (NORM) {
            unit_point(x, y, z, r2, ir);
        } else {
            r2 = x * x + y * y + z * z;
        }
        const int rr = r < 13 ? r : 12;
        float* rowp = rr == 0 ? s_v + size_t(j) * S
                              : (rr < 4 ? s_d + size_t(3 * j + rr - 1) * S : s_h + size_t(9 * j + rr - 4) * S);
        point16_core<L, NORM>(x, y, z, r2, tb, rr, lane & 16, ir, rowp, rowp, r < 13);
        if constexpr (MODE == 1) {
            if (bulk && r < 13 && j < cnt) {  // each lane sends the row it wrote
                fence_proxy_async_smem();
                float* g = rr == 0 ? sph + (p0 + j) * K
                                   : (rr < 4 ? dsph + ((p0 + j) * 3 + rr - 1) * K : ddsph + ((p0 + j) * 9 + rr - 4) * K);
                bulk_store(g, rowp, uint32_t(K * 4));
                bulk_commit();
            }
        }
    }
    if constexpr (MODE == 1) {
        if (bulk) {
            bulk_wait_read_all();
            __syncwarp();
            return;
        }
    }
    if (MODE != 0 || !bulk) {
        __syncwarp();
        warp_rows_out<K>(sph + p0 * K, s_v, cnt, S, lane);
        warp_rows_out<K>(dsph + p0 * 3 * K, s_d, 3 * cnt, S, lane);
        warp_rows_out<K>(ddsph + p0 * 9 * K, s_h, 9 * cnt, S, lane);
        __syncwarp();
        return;
    }
    // MODE 0 with bulk copies: the image of the three global ranges; the tile
    // start is 16-byte aligned (P is a multiple of the tile multiple)
    fence_proxy_async_smem();
    __syncwarp();
    const int64_t ev = int64_t(cnt) * K;
    const int64_t ev_b = (ev * 4) / 16 * 4, ed_b = (3 * ev * 4) / 16 * 4, eh_b = (9 * ev * 4) / 16 * 4;
    if (lane == 0) {
        if (ev_b) bulk_store(sph + p0 * K, s_v, uint32_t(ev_b * 4));
        if (ed_b) bulk_store(dsph + p0 * 3 * K, s_d, uint32_t(ed_b * 4));
        if (eh_b) bulk_store(ddsph + p0 * 9 * K, s_h, uint32_t(eh_b * 4));
        bulk_commit();
    }
    for (int64_t i = ev_b + lane; i < ev; i += 32) sph[p0 * K + i] = s_v[i];
    for (int64_t i = ed_b + lane; i < 3 * ev; i += 32) dsph[p0 * 3 * K + i] = s_d[i];
    for (int64_t i = eh_b + lane; i < 9 * ev; i += 32) ddsph[p0 * 9 * K + i] = s_h[i];
    if (lane == 0) bulk_wait_read_all();
    __syncwarp();
}

template <int L, bool NORM>
__global__ void __launch_bounds__(128, 3) point16_fwd_kernel(const float* __restrict__ xyz, int64_t n,
                                                          const __grid_constant__ PointTabs<L, float, true> tb,
                                                          float* __restrict__ sph, float* __restrict__ dsph,
                                                          float* __restrict__ ddsph, int P, int bulk) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    unsigned char* buf = smem + size_t(warp) * point16_warp_bytes<L>(P);
    const int64_t ntiles = (n + P - 1) / P;
    const int64_t stride = int64_t(gridDim.x) * W;
    for (int64_t tile = int64_t(blockIdx.x) * W + warp; tile < ntiles; tile += stride) {
        const int64_t p0 = tile * P;
        const int cnt = int(min(int64_t(P), n - p0));
        point16_tile<L, NORM>(xyz, sph, dsph, ddsph, p0, cnt, P, bulk, buf, tb, lane);
    }
    if (bulk) bulk_wait_all();  // every lane: rows may leave by per-lane copies
}

// ------------------- forward with Hessians, 10 lanes per point (distinct planes)
// POINT with lanes_per_point = 10 (FP32 values, gradients and Hessians): the
// 30 first lanes of a warp compute 3 points per pass, lane 10j + r owning the
// r-th distinct plane of point j (value, 3 gradient components, the Hessian
// entries xx, xy, xz, yy, yz, zz; lanes 30, 31 idle). The lane of an
// off-diagonal entry also writes its mirror, so no lane repeats another's
// work: 1.6x the points per warp instruction of the 16-lane map. The planes
// come from point16_core (the same role weights).
//
// Shared memory, odd K: the image of the tile's three global ranges, each
// placed at its 16-byte phase so that the interior leaves by one bulk copy
// per array (head and tail by plain stores). Even K (K % 4 == 0 in FP32):
// every row is 16-byte aligned at both ends, so each lane keeps only its
// distinct row (10 row slots per point at stride point4_stride) and sends it
// by one bulk copy per global row, the mirror from the same slot.
template <int L>
__host__ __device__ constexpr size_t point10_warp_bytes(int P) {
    constexpr int K = (L + 1) * (L + 1);
    if constexpr (K % 2) {
        const size_t v = (size_t(P) * K + 4 + 3) / 4 * 4, d = (size_t(3 * P) * K + 4 + 3) / 4 * 4,
                     h = (size_t(9 * P) * K + 4 + 3) / 4 * 4;
        return 4 * (v + d + h);
    } else {
        return size_t(4) * 10 * size_t(P) * size_t(point4_stride(L, 4));
    }
}

__host__ __device__ constexpr int point10_plane(int r) {  // distinct plane r -> index among the 13
    return r < 4 ? r : (r == 4 ? 4 : r == 5 ? 5 : r == 6 ? 6 : r == 7 ? 8 : r == 8 ? 9 : 12);
}
__host__ __device__ constexpr int point10_mirror(int q) {  // Hessian plane 4 + 3i + k -> 4 + 3k + i
    return q < 4 ? q : 4 + 3 * ((q - 4) % 3) + (q - 4) / 3;
}
__host__ __device__ constexpr int point10_slot(int q) {  // plane among the 13 -> its distinct row
    return q < 4 ? q : (q == 4 ? 4 : (q == 5 || q == 7) ? 5 : (q == 6 || q == 10) ? 6 : q == 8 ? 7 : (q == 9 || q == 11) ? 8 : 9);
}

// Sends elements [0, E) of a staged range (image element e at img[e], the
// range's global start g; img and g share their 16-byte phase): the
// 16-byte-aligned interior by one bulk copy from lane 0, the rest by plain
// stores of the warp. Returns whether a bulk copy was issued.
__device__ __forceinline__ bool point10_send(float* __restrict__ g, const float* __restrict__ img, int64_t E, int lane) {
    const int64_t h = (4 - int64_t((reinterpret_cast<uintptr_t>(g) / 4) % 4)) % 4;
    const int64_t nb = E > h ? (E - h) / 4 * 4 : 0;
    if (nb > 0 && lane == 0) bulk_store(g + h, img + h, uint32_t(nb * 4));
    for (int64_t i = lane; i < min(h, E); i += 32) g[i] = img[i];
    for (int64_t i = h + nb + lane; i < E; i += 32) g[i] = img[i];
    return nb > 0;
}

// One tile of P points (P a multiple of 3, <= 12): passes of 3 points.
template <int L, bool NORM, typename Tabs>
__device__ __forceinline__ void point10_tile(const float* __restrict__ xyz, float* __restrict__ sph,
                                             float* __restrict__ dsph, float* __restrict__ ddsph, int64_t p0,
                                             int cnt, int P, int bulk, unsigned char* buf, const Tabs& tb,
                                             int lane) {
    constexpr int K = (L + 1) * (L + 1);
    constexpr bool IMG = (K % 2) != 0;
    constexpr int S = IMG ? K : point4_stride(L, 4);
    const int j = min(lane / 10, 2);
    const int r = min(lane - 10 * j, 9);
    const bool on = lane < 30;
    const int rr = point10_plane(r), rm = point10_mirror(rr);
    float *iv = nullptr, *id = nullptr, *ih = nullptr;
    if constexpr (IMG) {
        float* const sv = reinterpret_cast<float*>(buf);
        float* const sd = sv + (size_t(P) * K + 4 + 3) / 4 * 4;
        float* const sh = sd + (size_t(3 * P) * K + 4 + 3) / 4 * 4;
        // each image shares the 16-byte phase of its global range
        iv = sv + (bulk ? (reinterpret_cast<uintptr_t>(sph + p0 * K) / 4) % 4 : 0);
        id = sd + (bulk ? (reinterpret_cast<uintptr_t>(dsph + p0 * 3 * K) / 4) % 4 : 0);
        ih = sh + (bulk ? (reinterpret_cast<uintptr_t>(ddsph + p0 * 9 * K) / 4) % 4 : 0);
    }
    float* const slots = reinterpret_cast<float*>(buf);  // even K: 10 row slots per point
    for (int t = 0; t < P; t += 3) {
        const int pj = t + j;
        const bool live = on && pj < cnt;
        float x = 0.f, y = 0.f, z = 1.f;  // idle lanes run on a unit vector and store nothing
        if (live) {
            x = xyz[3 * (p0 + pj)];
            y = xyz[3 * (p0 + pj) + 1];
            z = xyz[3 * (p0 + pj) + 2];
        }
        float r2, ir = 1.f;
        if (NORM) {
            unit_point(x, y, z, r2, ir);
        } else {
            r2 = x * x + y * y + z * z;
        }
        if constexpr (IMG) {
            float* rowp = rr == 0 ? iv + size_t(pj) * S
                                  : (rr < 4 ? id + size_t(3 * pj + rr - 1) * S : ih + size_t(9 * pj + rr - 4) * S);
            float* rowp2 = rr < 4 ? rowp : ih + size_t(9 * pj + rm - 4) * S;
            point16_core<L, NORM, true>(x, y, z, r2, tb, rr, 10 * j, ir, rowp, rowp2, live);
        } else {
            float* rowp = slots + size_t(10 * pj + r) * S;
            point16_core<L, NORM, false>(x, y, z, r2, tb, rr, 10 * j, ir, rowp, rowp, live);
            if (bulk && live) {  // rows 16-byte aligned at both ends: one copy per global row
                fence_proxy_async_smem();
                const int64_t gp = p0 + pj;
                float* g1 = rr == 0 ? sph + gp * K : (rr < 4 ? dsph + (gp * 3 + rr - 1) * K : ddsph + (gp * 9 + rr - 4) * K);
                bulk_store(g1, rowp, uint32_t(K * 4));
                if (rm != rr) bulk_store(ddsph + (gp * 9 + rm - 4) * K, rowp, uint32_t(K * 4));
                bulk_commit();
            }
        }
    }
    if constexpr (!IMG) {
        if (bulk) {
            bulk_wait_read_all();
            __syncwarp();
            return;
        }
        // outputs not 16-byte aligned: the warp copies the 13 global rows of
        // each point from their slots
        __syncwarp();
        for (int q = 0; q < 13 * cnt; ++q) {
            const int pj = q / 13, pl = q - 13 * pj;
            const int64_t gp = p0 + pj;
            float* g = pl == 0 ? sph + gp * K : (pl < 4 ? dsph + (gp * 3 + pl - 1) * K : ddsph + (gp * 9 + pl - 4) * K);
            const float* src = slots + size_t(10 * pj + point10_slot(pl)) * S;
            for (int c = lane; c < K; c += 32) g[c] = src[c];
        }
        __syncwarp();
        return;
    } else {
        fence_proxy_async_smem();
        __syncwarp();
        if (bulk) {
            bool any = point10_send(sph + p0 * K, iv, int64_t(cnt) * K, lane);
            any = point10_send(dsph + p0 * 3 * K, id, int64_t(3 * cnt) * K, lane) || any;
            any = point10_send(ddsph + p0 * 9 * K, ih, int64_t(9 * cnt) * K, lane) || any;
            if (lane == 0 && any) {
                bulk_commit();
                bulk_wait_read_all();
            }
        } else {
            for (int64_t i = lane; i < int64_t(cnt) * K; i += 32) sph[p0 * K + i] = iv[i];
            for (int64_t i = lane; i < int64_t(3 * cnt) * K; i += 32) dsph[p0 * 3 * K + i] = id[i];
            for (int64_t i = lane; i < int64_t(9 * cnt) * K; i += 32) ddsph[p0 * 9 * K + i] = ih[i];
        }
        __syncwarp();
    }
}

template <int L, bool NORM>
__global__ void __launch_bounds__(128, 3) point10_fwd_kernel(const float* __restrict__ xyz, int64_t n,
                                                             const __grid_constant__ PointTabs<L, float, true> tb,
                                                             float* __restrict__ sph, float* __restrict__ dsph,
                                                             float* __restrict__ ddsph, int P, int bulk) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    unsigned char* buf = smem + size_t(warp) * point10_warp_bytes<L>(P);
    const int64_t ntiles = (n + P - 1) / P;
    const int64_t stride = int64_t(gridDim.x) * W;
    for (int64_t tile = int64_t(blockIdx.x) * W + warp; tile < ntiles; tile += stride) {
        const int64_t p0 = tile * P;
        const int cnt = int(min(int64_t(P), n - p0));
        point10_tile<L, NORM>(xyz, sph, dsph, ddsph, p0, cnt, P, bulk, buf, tb, lane);
    }
    if (bulk) bulk_wait_all();  // every lane: rows may leave by per-lane copies
}

// ----------------------------------------------------------------- backward
// Loads the [cnt, K] tile of `src` at element offset `off` into `dst`: the
// 16-byte-multiple prefix by a bulk copy on `bar` (if `bulk`), the rest with
// plain loads at consumption time. Returns the number of bulk elements.
template <typename T>
__device__ __forceinline__ int64_t issue_tile_load(T* dst, const T* src, int64_t elems, int bulk, uint64_t* bar,
                                                   int lane) {
    int64_t eb = bulk ? (elems * int64_t(sizeof(T))) / 16 * 16 / int64_t(sizeof(T)) : 0;
    if (eb > 0 && lane == 0) {
        mbar_arrive_expect_tx(bar, uint32_t(eb * sizeof(T)));
        bulk_load(dst, src, uint32_t(eb * sizeof(T)), bar);
    }
    return eb;
}

constexpr uint32_t kWaitPolls = 1u << 22;  // bounded mbarrier wait (>> any real load latency)

template <typename T, bool NORM, int K>
struct BwdVis {
    const T* gr;  // this lane's upstream-gradient row in shared memory
    T ax, ay, az, S;
    __device__ __forceinline__ void emit(int l, int k, const Deriv<T>& d) {
        const T gk = gr[k];
        ax += gk * d.gx;
        ay += gk * d.gy;
        az += gk * d.gz;
        if (NORM) S += gk * (T(l) * d.v);
    }
};

template <typename T, bool NORM, int K>
struct DbwdVis {
    const T* gr;  // upstream gradient row (shared)
    T* orow;      // grad_g row (shared)
    T vx, vy, vz;
    T ux, uy, uz, ir;
    T ax, ay, az;
    __device__ __forceinline__ void emit(int l, int k, Deriv<T> d) {
        if (NORM) normalize_deriv<true>(d, l, ux, uy, uz, ir);
        const T gk = gr[k];
        orow[k] = vx * d.gx + vy * d.gy + vz * d.gz;
        ax += gk * (d.hxx * vx + d.hxy * vy + d.hxz * vz);
        ay += gk * (d.hxy * vx + d.hyy * vy + d.hyz * vz);
        az += gk * (d.hxz * vx + d.hyz * vy + d.hzz * vz);
    }
};

template <int L, typename T>
__host__ __device__ constexpr size_t point_bwd_buf_bytes(int P) {
    return align16(size_t(P) * RowStride<L>::V * sizeof(T));
}

// DBW = false: backward (dxyz). DBW = true: double backward (grad_g, grad_xyz).
// Shared memory per warp: two upstream-gradient buffers, (DBW) one grad_g
// buffer, and two mbarriers.
template <int L, bool NORM, bool DBW, typename T>
__global__ void __launch_bounds__(256) point_bwd_kernel(const T* __restrict__ xyz, const T* __restrict__ g,
                                                        const T* __restrict__ v, int64_t n,
                                                        const __grid_constant__ PointTabs<L, T, DBW> tb,
                                                        T* __restrict__ dxyz, T* __restrict__ grad_g,
                                                        T* __restrict__ grad_xyz, int P, int bulk_in,
                                                        int bulk_out, uint32_t* __restrict__ status) {
    constexpr int K = (L + 1) * (L + 1);
    using RS = RowStride<L>;
    if constexpr (RS::PAD) bulk_in = bulk_out = 0;  // padded rows: plain loads / stores
    (void)bulk_out;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const size_t buf = point_bwd_buf_bytes<L, T>(P);
    const size_t per_warp = (DBW ? 3 : 2) * buf + 16;
    unsigned char* base = smem + size_t(warp) * per_warp;
    T* const sg0 = reinterpret_cast<T*>(base);
    T* const sg1 = reinterpret_cast<T*>(base + buf);
    T* so = reinterpret_cast<T*>(base + 2 * buf);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + (DBW ? 3 : 2) * buf);

    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    fence_proxy_async_smem();
    __syncwarp();

    const int64_t ntiles = (n + P - 1) / P;
    const int64_t stride = int64_t(gridDim.x) * W;
    int64_t tile = int64_t(blockIdx.x) * W + warp;
    uint32_t phase = 0;    // bit b: parity of buffer b's next completion
    uint32_t pending = 0;  // bit b: a bulk load into buffer b is in flight
    int64_t eb0 = 0, eb1 = 0;
    bool failed = false;

    if (tile < ntiles) {
        const int64_t p0 = tile * P;
        const int64_t cnt = min(int64_t(P), n - p0);
        eb0 = issue_tile_load(sg0, g + p0 * K, cnt * K, bulk_in, &bar[0], lane);
        if (eb0 > 0) pending |= 1u;
    }
    int cur = 0;
    for (; tile < ntiles; tile += stride) {
        const int64_t p0 = tile * P;
        const int cnt = int(min(int64_t(P), n - p0));
        // Prefetch the next tile into the other buffer; its previous contents
        // were consumed in the last iteration, which ended with a proxy fence
        // and __syncwarp.
        const int64_t nt = tile + stride;
        const int nxt = cur ^ 1;
        if (nt < ntiles) {
            const int64_t q0 = nt * P;
            const int64_t qc = min(int64_t(P), n - q0);
            const int64_t e = issue_tile_load(nxt ? sg1 : sg0, g + q0 * K, qc * K, bulk_in, &bar[nxt], lane);
            if (nxt) eb1 = e; else eb0 = e;
            if (e > 0) pending |= (1u << nxt);
        }
        // Wait for this tile's bulk part, then load the remainder directly.
        if (pending & (1u << cur)) {
            bool ok = true;
            if (lane == 0) ok = mbar_wait_bounded(&bar[cur], (phase >> cur) & 1u, kWaitPolls);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (ok) {
                phase ^= (1u << cur);
                pending &= ~(1u << cur);
            } else {
                if (lane == 0) atomicOr(status, kStatusLoadTimeout);
                failed = true;
            }
        }
        if (failed) break;
        const int64_t eb_cur = cur ? eb1 : eb0;
        T* const gt = cur ? sg1 : sg0;
        if constexpr (RS::PAD) {
            warp_rows_in<K>(gt, g + p0 * K, cnt, RS::V, lane);
        } else {
            for (int64_t i = eb_cur + lane; i < int64_t(cnt) * K; i += 32) gt[i] = g[p0 * K + i];
        }
        __syncwarp();
        if (lane < cnt) {
            const int64_t p = p0 + lane;
            T x = xyz[3 * p], y = xyz[3 * p + 1], z = xyz[3 * p + 2];
            T r2, ir = T(1);
            if (NORM) {
                unit_point(x, y, z, r2, ir);
            } else {
                r2 = x * x + y * y + z * z;
            }
            if constexpr (!DBW) {
                BwdVis<T, NORM, K> vis{gt + size_t(lane) * RS::V, T(0), T(0), T(0), T(0)};
                point_core<L, true, false>(x, y, z, r2, tb, vis);
                T ax = vis.ax, ay = vis.ay, az = vis.az;
                if (NORM) {
                    ax = ir * (ax - x * vis.S);
                    ay = ir * (ay - y * vis.S);
                    az = ir * (az - z * vis.S);
                }
                dxyz[3 * p] = ax;
                dxyz[3 * p + 1] = ay;
                dxyz[3 * p + 2] = az;
            } else {
                DbwdVis<T, NORM, K> vis{gt + size_t(lane) * RS::V,
                                        so + size_t(lane) * RS::V,
                                        v[3 * p],
                                        v[3 * p + 1],
                                        v[3 * p + 2],
                                        x,
                                        y,
                                        z,
                                        ir,
                                        T(0),
                                        T(0),
                                        T(0)};
                point_core<L, true, true>(x, y, z, r2, tb, vis);
                if (grad_xyz) {
                    grad_xyz[3 * p] = vis.ax;
                    grad_xyz[3 * p + 1] = vis.ay;
                    grad_xyz[3 * p + 2] = vis.az;
                }
            }
        }
        if constexpr (DBW) {
            if (grad_g && RS::PAD) {
                __syncwarp();
                warp_rows_out<K>(grad_g + p0 * K, so, cnt, RS::V, lane);
            } else if (grad_g) {
                fence_proxy_async_smem();
                __syncwarp();
                const int64_t ev = int64_t(cnt) * K;
                int64_t eo = 0;
                if (bulk_out) {
                    eo = (ev * int64_t(sizeof(T))) / 16 * 16 / int64_t(sizeof(T));
                    if (lane == 0 && eo > 0) {
                        bulk_store(grad_g + p0 * K, so, uint32_t(eo * sizeof(T)));
                        bulk_commit();
                    }
                }
                for (int64_t i = eo + lane; i < ev; i += 32) grad_g[p0 * K + i] = so[i];
                if (bulk_out && lane == 0) bulk_wait_read_all();
            }
        }
        fence_proxy_async_smem();
        __syncwarp();
        cur = nxt;
    }
    if (pending && lane == 0) {
        // Loads issued but never observed (after a timeout) may still be in
        // flight: wait for them, bounded, before the shared memory goes away.
        for (int b = 0; b < 2; ++b)
            if (pending & (1u << b)) (void)mbar_wait_bounded(&bar[b], (phase >> b) & 1u, kWaitPolls);
    }
    if (DBW && lane == 0) bulk_wait_all();
    __syncwarp();
}

// ---------------------------------------------------------------- launchers
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Host-side launch cache, keyed by (kernel address, device): the largest
// dynamic shared-memory size already set on the kernel and the occupancy of
// the last (threads, smem) pair queried, so repeated launches skip the
// attribute call and the occupancy query.
struct LaunchEntry {
    int smem_set = 48 * 1024;
    long long occ_key = -1;  // (threads << 32) | smem of `occ`
    int occ = 0;
};

inline std::mutex& launch_cache_mutex() {
    static std::mutex m;
    return m;
}

inline LaunchEntry& launch_entry(const void* kern, int dev) {  // caller holds the mutex
    static std::map<std::pair<const void*, int>, LaunchEntry> cache;
    return cache[std::make_pair(kern, dev)];
}

inline int cache_device() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return d;
}

// Raise the dynamic shared-memory limit of `kern` once per device and size.
template <typename K>
inline cudaError_t ensure_smem(K kern, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    const void* f = reinterpret_cast<const void*>(kern);
    const int d = cache_device();
    std::lock_guard<std::mutex> lk(launch_cache_mutex());
    if (d >= 0 && launch_entry(f, d).smem_set >= int(bytes)) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e == cudaSuccess && d >= 0) launch_entry(f, d).smem_set = int(bytes);
    return e;
}

template <typename K>
inline int grid_for(K kern, int threads, size_t smem, int64_t work_warps, int blocks_per_sm) {
    int bps = blocks_per_sm;
    if (bps <= 0) {
        const void* f = reinterpret_cast<const void*>(kern);
        const int d = cache_device();
        const long long key = (static_cast<long long>(threads) << 32) | static_cast<long long>(smem);
        int occ = 0;
        std::lock_guard<std::mutex> lk(launch_cache_mutex());
        LaunchEntry* c = d >= 0 ? &launch_entry(f, d) : nullptr;
        if (c && c->occ_key == key) {
            occ = c->occ;
        } else {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, threads, smem) != cudaSuccess) {
                cudaGetLastError();
                occ = 1;
            }
            if (c) {
                c->occ = occ;
                c->occ_key = key;
            }
        }
        bps = std::max(occ, 1);
    }
    const int W = threads / 32;
    int64_t want = ceil_div(work_warps, W);
    int64_t cap = int64_t(bps) * sm_count();
    return int(std::max<int64_t>(1, std::min(want, cap)));
}

template <int L, bool GRAD, bool HESS, bool NORM, typename T, typename TO, bool HC = false>
int launch_point_fwd(const FwdArgs& a) {
    static const PointTabs<L, T, HESS> tb = make_point_tabs<L, T, HESS>();
    const int P = a.launch.points_per_tile, W = a.launch.warps_per_block;
    const size_t smem = size_t(W) * point_fwd_warp_bytes<L, GRAD, HESS, TO>(P);
    auto kern = point_fwd_kernel<L, GRAD, HESS, NORM, T, TO, HC>;
    cudaError_t err = ensure_smem(kern, smem);
    if (err != cudaSuccess) return int(err);
    const int64_t ntiles = ceil_div(a.n, P);
    const int grid = grid_for(kern, 32 * W, smem, ntiles, a.launch.blocks_per_sm);
    const bool bulk = (reinterpret_cast<uintptr_t>(a.sph) % 16 == 0) &&
                      (!GRAD || reinterpret_cast<uintptr_t>(a.dsph) % 16 == 0) &&
                      (!HESS || reinterpret_cast<uintptr_t>(a.ddsph) % 16 == 0);
    kern<<<grid, 32 * W, smem, static_cast<cudaStream_t>(a.stream)>>>(
        static_cast<const T*>(a.xyz), a.n, tb, static_cast<TO*>(a.sph), static_cast<TO*>(a.dsph),
        static_cast<TO*>(a.ddsph), P, bulk ? 1 : 0);
    return int(cudaGetLastError());
}

// POINT forward with 4 lanes per point (values and gradients); P <= 8 and W
// resolved by the caller.
template <int L, bool NORM, typename T, typename TO>
int launch_point4_fwd(const FwdArgs& a) {
    static const PointTabs<L, T, false> tb = make_point_tabs<L, T, false>();
    const int P = a.launch.points_per_tile, W = a.launch.warps_per_block;
    const size_t smem = size_t(W) * point4_warp_bytes<L, TO>(P);
    auto kern = point4_fwd_kernel<L, NORM, T, TO>;
    cudaError_t err = ensure_smem(kern, smem);
    if (err != cudaSuccess) return int(err);
    const int64_t ntiles = ceil_div(a.n, P);
    const int grid = grid_for(kern, 32 * W, smem, ntiles, a.launch.blocks_per_sm);
    const bool bulk = (reinterpret_cast<uintptr_t>(a.sph) % 16 == 0) && (reinterpret_cast<uintptr_t>(a.dsph) % 16 == 0);
    kern<<<grid, 32 * W, smem, static_cast<cudaStream_t>(a.stream)>>>(
        static_cast<const T*>(a.xyz), a.n, tb, static_cast<TO*>(a.sph), static_cast<TO*>(a.dsph), P, bulk ? 1 : 0);
    return int(cudaGetLastError());
}

// POINT forward with Hessians, 16 lanes per point (FP32); P (even, <= 8) and
// W resolved by the caller.
template <int L, bool NORM>
int launch_point16_fwd(const FwdArgs& a) {
    static const PointTabs<L, float, true> tb = make_point_tabs<L, float, true>();
    const int P = a.launch.points_per_tile, W = a.launch.warps_per_block;
    const size_t smem = size_t(W) * point16_warp_bytes<L>(P);
    auto kern = point16_fwd_kernel<L, NORM>;
    cudaError_t err = ensure_smem(kern, smem);
    if (err != cudaSuccess) return int(err);
    const int64_t ntiles = ceil_div(a.n, P);
    const int grid = grid_for(kern, 32 * W, smem, ntiles, a.launch.blocks_per_sm);
    const bool bulk = reinterpret_cast<uintptr_t>(a.sph) % 16 == 0 && reinterpret_cast<uintptr_t>(a.dsph) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(a.ddsph) % 16 == 0;
    kern<<<grid, 32 * W, smem, static_cast<cudaStream_t>(a.stream)>>>(
        static_cast<const float*>(a.xyz), a.n, tb, static_cast<float*>(a.sph), static_cast<float*>(a.dsph),
        static_cast<float*>(a.ddsph), P, bulk ? 1 : 0);
    return int(cudaGetLastError());
}

// POINT forward with Hessians, 10 lanes per point (FP32); P (a multiple of 3,
// <= 12) and W resolved by the caller.
template <int L, bool NORM>
int launch_point10_fwd(const FwdArgs& a) {
    static const PointTabs<L, float, true> tb = make_point_tabs<L, float, true>();
    const int P = a.launch.points_per_tile, W = a.launch.warps_per_block;
    const size_t smem = size_t(W) * point10_warp_bytes<L>(P);
    auto kern = point10_fwd_kernel<L, NORM>;
    cudaError_t err = ensure_smem(kern, smem);
    if (err != cudaSuccess) return int(err);
    const int64_t ntiles = ceil_div(a.n, P);
    const int grid = grid_for(kern, 32 * W, smem, ntiles, a.launch.blocks_per_sm);
    const bool bulk = reinterpret_cast<uintptr_t>(a.sph) % 16 == 0 && reinterpret_cast<uintptr_t>(a.dsph) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(a.ddsph) % 16 == 0;
    kern<<<grid, 32 * W, smem, static_cast<cudaStream_t>(a.stream)>>>(
        static_cast<const float*>(a.xyz), a.n, tb, static_cast<float*>(a.sph), static_cast<float*>(a.dsph),
        static_cast<float*>(a.ddsph), P, bulk ? 1 : 0);
    return int(cudaGetLastError());
}

template <int L, bool NORM, bool DBW, typename T>
int launch_point_bwd(const BwdArgs& a) {
    static const PointTabs<L, T, DBW> tb = make_point_tabs<L, T, DBW>();
    const int P = a.launch.points_per_tile, W = a.launch.warps_per_block;
    const size_t smem = size_t(W) * ((DBW ? 3 : 2) * point_bwd_buf_bytes<L, T>(P) + 16);
    auto kern = point_bwd_kernel<L, NORM, DBW, T>;
    cudaError_t err = ensure_smem(kern, smem);
    if (err != cudaSuccess) return int(err);
    const int64_t ntiles = ceil_div(a.n, P);
    const int grid = grid_for(kern, 32 * W, smem, ntiles, a.launch.blocks_per_sm);
    const bool bulk_in = reinterpret_cast<uintptr_t>(a.g) % 16 == 0;
    const bool bulk_out = reinterpret_cast<uintptr_t>(a.grad_g) % 16 == 0;
    kern<<<grid, 32 * W, smem, static_cast<cudaStream_t>(a.stream)>>>(
        static_cast<const T*>(a.xyz), static_cast<const T*>(a.g), static_cast<const T*>(a.v), a.n, tb,
        static_cast<T*>(a.dxyz), static_cast<T*>(a.grad_g), static_cast<T*>(a.grad_xyz), P, bulk_in ? 1 : 0,
        bulk_out ? 1 : 0, a.status);
    return int(cudaGetLastError());
}

}  // namespace sph
