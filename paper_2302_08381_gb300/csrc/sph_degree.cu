// DEGREE kernel family: one thread per point, degree l outermost, any
// l_max <= SPH_MAX_L chosen at run time.
//
// A warp owns a tile of 32 consecutive points, one per lane, and walks the
// degrees l = 0..l_max in order. The recursion state a degree needs from the
// earlier ones is a few columns over m, kept in shared memory as lane-private
// arrays [m][lane] (bank-conflict free, no synchronisation between lanes):
//
//  * upward in l (arXiv 2302.08381, Eq. iter-q, prefactors folded in as in
//    Appendix C): Qtilde_l^m from Qtilde_{l-1}^m and Qtilde_{l-2}^m -- two
//    columns, m ascending; c_m, s_m (Eq. iter-sc) are regenerated in registers
//    alongside m, so they need no storage;
//  * downward in m (Eq. iter-q-alt with its sign corrected): Qtilde_l^m from
//    Qtilde_l^{m+1} and Qtilde_l^{m+2}, started at the tabulated Qtilde_l^l, so
//    the values of a degree need no state from earlier degrees at all; c_m, s_m
//    are read from a per-lane table (m descends) and the gradients of Eq.
//    iter-deri read the previous degree's column, updated in place.
//
// With the upward recursion a point may also be split over LPP = 2 or 4
// lanes (a warp then owns 32/LPP points): lane h of a point runs the channels
// m = h (mod LPP) and steps c_m, s_m by (x + i y)^LPP. The per-warp shared
// memory shrinks by LPP, so more warps are resident to hide the latency of
// the shared-memory traffic.
//
// Outputs: the columns of one degree are contiguous in every output row
// (l*l .. l*l+2l). A degree is produced in chunks of up to 16 m values (at
// most 32 columns: the +m and -m sides of the chunk, or several whole small
// degrees), written by the lanes into a shared-memory stage [plane][point][33]
// (odd stride: conflict free) and then stored by the warp with one lane per
// column and one coalesced store per point, so every warp store writes one or
// two contiguous row segments.
//
// The translation unit is compiled once per variant: SPH_DEGREE_DOWN=1 defines
// the downward-in-m entry point; SPH_DEGREE_DOWN=0 with SPH_DEGREE_LPP = 1, 2
// or 4 the upward-in-l entry point for that many lanes per point.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "sph_core.cuh"
#include "sph_internal.h"

#ifndef SPH_DEGREE_DOWN
#define SPH_DEGREE_DOWN 0
#endif
#ifndef SPH_DEGREE_LPP
#define SPH_DEGREE_LPP 1
#endif

namespace sph {

namespace {

constexpr int kMC = 16;           // m values per chunk
constexpr int kSlots = 2 * kMC;   // staged columns per store pass (<= 32 lanes)
constexpr int kSt = kSlots + 1;   // stage row stride (odd)

template <typename TQ>
struct DegV4;
template <>
struct DegV4<float> {
    using type = float4;
};
template <>
struct DegV4<double> {
    using type = double4_32a;  // 64-byte entries: 32-byte aligned halves
};

__host__ __device__ constexpr size_t deg_align(size_t b) { return (b + 15) & ~size_t(15); }

// FP32 coefficients for l_max <= kConstL live in constant memory: every lane
// of a warp reads the same (l, m) entry, which the constant cache broadcasts
// with a short latency. Entry (l, m): c_tab4 = {A, B, S, e} of this
// translation unit's recursion (upward: a|d_l, b; downward: al, be), S =
// Qtilde_l^l on the diagonal, e the d/dx multiplier; c_tabf = f (d/dz).
constexpr int kConstL = 64;
constexpr int kConstTri = (kConstL + 1) * (kConstL + 2) / 2;
__constant__ float4 c_tab4[kConstTri];
__constant__ float c_tabf[kConstTri];

// Table access: constant memory (CT) or the packed global tables (two
// 4-vectors per entry, see sph_internal.h).
template <typename TQ, bool CT>
struct DegTab {
    using V4 = typename DegV4<TQ>::type;
    const TQ* __restrict__ tb;
    __device__ __forceinline__ V4 t0(int i) const { return reinterpret_cast<const V4*>(tb)[2 * i]; }
    __device__ __forceinline__ TQ f(int i) const { return tb[8 * i + 4]; }
};
template <>
struct DegTab<float, true> {
    const float* __restrict__ tb;  // unused
    __device__ __forceinline__ float4 t0(int i) const { return c_tab4[i]; }
    __device__ __forceinline__ float f(int i) const { return c_tabf[i]; }
};

template <int LPP, typename TO, bool GRAD>
__host__ __device__ constexpr size_t degree_stage_bytes() {
    return deg_align(size_t(GRAD ? 4 : 1) * (32 / LPP) * kSt * sizeof(TO));
}

// Number of state columns (each one entry per point of the warp) a warp keeps.
template <bool GRAD, bool DOWN>
__host__ __device__ constexpr int degree_state_cols(int L) {
    return DOWN ? 2 * (L + 1) + (GRAD ? L + 2 : 0) : 2 * (L + 2);
}

template <int LPP, typename TQ, typename TO, bool GRAD, bool DOWN>
__host__ __device__ constexpr size_t degree_warp_bytes(int L) {
    return degree_stage_bytes<LPP, TO, GRAD>() +
           deg_align(size_t(degree_state_cols<GRAD, DOWN>(L)) * (32 / LPP) * sizeof(TQ));
}

// Writes one column's value (and gradient planes) into this lane's stage row.
// PL: elements of one stage plane.
template <int PL, bool GRAD, typename TO, typename TQ>
__device__ __forceinline__ void stage_put(TO* __restrict__ st, int slot, const Deriv<TQ>& d) {
    st[slot] = OutConv<TO>::cv(d.v);
    if (GRAD) {
        st[PL + slot] = OutConv<TO>::cv(d.gx);
        st[2 * PL + slot] = OutConv<TO>::cv(d.gy);
        st[3 * PL + slot] = OutConv<TO>::cv(d.gz);
    }
}

// Assembles and stages the +m / -m (or m = 0) columns of degree l.
template <int PL, bool GRAD, bool NORM, typename TO, typename TQ>
__device__ __forceinline__ void emit_pair(TO* __restrict__ st, int l, int m, bool zero, int slot_p, int slot_m,
                                          const QParts<TQ>& qp, TQ x, TQ y, TQ z, TQ ir, TQ inv_sqrt2, TQ cm,
                                          TQ sm, TQ cm1, TQ sm1) {
    if (zero) {
        Deriv<TQ> d = assemble_m0<GRAD, false>(qp, x, y, inv_sqrt2);
        if (NORM && GRAD) normalize_deriv<false>(d, l, x, y, z, ir);
        stage_put<PL, GRAD>(st, slot_p, d);
    } else {
        Deriv<TQ> dc, ds;
        assemble_m<GRAD, false>(qp, x, y, TQ(m), TQ(m - 1), cm, sm, cm1, sm1, TQ(0), TQ(0), dc, ds);
        if (NORM && GRAD) {
            normalize_deriv<false>(dc, l, x, y, z, ir);
            normalize_deriv<false>(ds, l, x, y, z, ir);
        }
        stage_put<PL, GRAD>(st, slot_p, dc);
        stage_put<PL, GRAD>(st, slot_m, ds);
    }
}

// Point coordinates and per-point constants of one lane.
template <typename TQ>
struct DegPoint {
    TQ x, y, z;  // the point (divided by r when normalized)
    TQ r2;       // x^2 + y^2 + z^2 of the coordinates above
    TQ rxy2;     // x^2 + y^2
    TQ ir;       // 1/r (normalized), else 1
};

// c_m + i s_m = (x + i y)^m as a pair, advanced by a complex factor.
template <typename TQ>
struct CS {
    TQ c, s;
    __device__ __forceinline__ CS times(const CS& w) const {
        return CS{fma(c, w.c, -(s * w.s)), fma(c, w.s, s * w.c)};
    }
};

// Upward in l: the channels m_lo..m_hi of degree l that this lane owns
// (m = h mod LPP), ascending. q1/q2 are the point's columns
// Qtilde_{l-1}^m / Qtilde_{l-2}^m (element m at [PPW m]); the result
// Qtilde_l^m replaces Qtilde_{l-2}^m in q2. `a` = c_m + i s_m and
// `b` = c_{m-1} + i s_{m-1} of the lane's next channel, carried from chunk to
// chunk; `w` = (x + i y)^LPP.
template <int LPP, bool GRAD, bool NORM, typename TQ, typename TO, typename Tab>
__device__ __forceinline__ void up_chunk(int l, int m_lo, int m_hi, int h, int sp0, int sm0, const Tab& tab,
                                         const DegPoint<TQ>& P, TQ inv_sqrt2, const TQ* __restrict__ q1,
                                         TQ* __restrict__ q2, TO* __restrict__ st, CS<TQ>& a, CS<TQ>& b,
                                         const CS<TQ>& w) {
    constexpr int PPW = 32 / LPP;
    constexpr int PL = PPW * kSt;
    TQ q1n = q1[PPW * m_lo];
#pragma unroll
    for (int k = 0; k < kMC / LPP; ++k) {
        const int m = m_lo + h + LPP * k;
        if (m > m_hi) break;
        const int i = tri(l, m);
        const auto t0 = tab.t0(i);  // {A, B, S, e}
        TQ q1m;
        if (LPP == 1) {  // channel m+1 is this lane's next channel: carry it
            q1m = q1n;
            q1n = q1[PPW * (m + 1)];
        } else {
            q1m = q1[PPW * m];
            q1n = q1[PPW * (m + 1)];
        }
        const TQ q2m = q2[PPW * m];
        // explicit fma: the same rounding in every variant (values-only or not)
        const TQ q = fma(t0.x * P.z, q1m, fma(-(t0.y * P.r2), q2m, t0.z));
        q2[PPW * m] = q;
        QParts<TQ> qp;
        qp.Q = q;
        qp.G2 = qp.G3 = qp.G4 = TQ(0);
        if (GRAD) {
            qp.E1 = t0.w * q1n;
            qp.Qz = tab.f(i) * q1m;
        } else {
            qp.E1 = qp.Qz = TQ(0);
        }
        // m = 0 is only ever the first channel of lane 0 in the chunk at m_lo = 0
        const bool zero = (LPP == 1 ? (k == 0 && m_lo == 0) : (m == 0));
        emit_pair<PL, GRAD, NORM>(st, l, m, zero, sp0 + m, sm0 - m, qp, P.x, P.y, P.z, P.ir, inv_sqrt2, a.c, a.s,
                                  b.c, b.s);
        if (LPP == 1) {  // Eq. iter-sc
            b = a;
            a = a.times(w);
        } else {
            if (!zero) b = b.times(w);  // at m = 0, b already holds (x + i y)^(LPP-1)
            a = a.times(w);
        }
    }
}

// Downward in m: channels m_hi..m_lo (descending) of degree l. (qa1, qa2)
// carry Qtilde_l^{m+1}, Qtilde_l^{m+2}; (cc, ss) carry c_m, s_m, read from
// the lane's tables ct/stb; with gradients, prev holds Qtilde_{l-1}^m (slot m
// is overwritten by Qtilde_l^m once read) and pn carries Qtilde_{l-1}^{m+1}.
template <bool GRAD, bool NORM, typename TQ, typename TO, typename Tab>
__device__ __forceinline__ void down_chunk(int l, int m_lo, int m_hi, int sp0, int sm0, const Tab& tab,
                                           const DegPoint<TQ>& P, TQ inv_sqrt2, const TQ* __restrict__ ct,
                                           const TQ* __restrict__ stb, TQ* __restrict__ prev, TO* __restrict__ st,
                                           TQ& qa1, TQ& qa2, TQ& pn, TQ& cc, TQ& ss) {
#pragma unroll
    for (int j = 0; j < kMC; ++j) {
        const int m = m_hi - j;
        if (m < m_lo) break;
        const int i = tri(l, m);
        const auto t0 = tab.t0(i);  // {al, be, S, e}
        const TQ q = fma(t0.x * P.z, qa1, fma(-(t0.y * P.rxy2), qa2, t0.z));
        qa2 = qa1;
        qa1 = q;
        QParts<TQ> qp;
        qp.Q = q;
        qp.G2 = qp.G3 = qp.G4 = TQ(0);
        if (GRAD) {
            const TQ pm = prev[32 * m];
            prev[32 * m] = q;
            qp.E1 = t0.w * pn;
            qp.Qz = tab.f(i) * pm;
            pn = pm;
        } else {
            qp.E1 = qp.Qz = TQ(0);
        }
        const TQ cm1 = m >= 1 ? ct[32 * (m - 1)] : TQ(0);
        const TQ sm1 = m >= 1 ? stb[32 * (m - 1)] : TQ(0);
        emit_pair<32 * kSt, GRAD, NORM>(st, l, m, m == 0, sp0 + m, sm0 - m, qp, P.x, P.y, P.z, P.ir, inv_sqrt2, cc,
                                        ss, cm1, sm1);
        cc = cm1;
        ss = sm1;
    }
}

// Stores `np` rows of the staged columns: lane t < ncols owns global column
// colA0 + t (t < nA) or offB + t (t >= nA) of every point in the tile.
template <int PPW, typename TO>
__device__ __forceinline__ void store_rows(TO* __restrict__ g, int64_t rstride, const TO* __restrict__ s, int np) {
    if (np == PPW) {
#pragma unroll 8
        for (int p = 0; p < PPW; ++p) g[p * rstride] = s[p * kSt];
    } else {
        for (int p = 0; p < np; ++p) g[p * rstride] = s[p * kSt];
    }
}

template <int PPW, bool GRAD, typename TO>
__device__ __forceinline__ void flush_stage(const TO* __restrict__ stw, TO* __restrict__ sph_t,
                                            TO* __restrict__ dsph_t, int64_t K, int np, int ncols, int nA,
                                            int64_t colA0, int64_t offB, int lane) {
    constexpr int PL = PPW * kSt;
    __syncwarp();
    if (lane < ncols) {
        const int64_t col = lane < nA ? colA0 + lane : offB + lane;
        const TO* s = stw + lane;
        store_rows<PPW>(sph_t + col, K, s, np);
        if (GRAD) {
            store_rows<PPW>(dsph_t + col, 3 * K, s + PL, np);
            store_rows<PPW>(dsph_t + K + col, 3 * K, s + 2 * PL, np);
            store_rows<PPW>(dsph_t + 2 * K + col, 3 * K, s + 3 * PL, np);
        }
    }
    __syncwarp();
}

template <typename TI, typename TQ, typename TO, bool GRAD, bool NORM, bool DOWN, bool CT, int LPP>
__global__ void __launch_bounds__(256) degree_fwd_kernel(const TI* __restrict__ xyz, int64_t n, int L,
                                                         const TQ* __restrict__ tb, TQ inv_sqrt2,
                                                         TO* __restrict__ sph, TO* __restrict__ dsph) {
    static_assert(!DOWN || LPP == 1, "the downward recursion is sequential in m: one lane per point");
    constexpr int PPW = 32 / LPP;  // points per warp tile
    const DegTab<TQ, CT> tab{tb};
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const int pt = lane / LPP;  // this lane's point in the tile
    const int h = lane % LPP;   // its channel class m = h (mod LPP)
    unsigned char* wbase = smem + size_t(warp) * degree_warp_bytes<LPP, TQ, TO, GRAD, DOWN>(L);
    TO* const stw = reinterpret_cast<TO*>(wbase);  // warp stage [plane][point][kSt]
    TO* const stl = stw + pt * kSt;                // this point's stage row
    TQ* const sbase = reinterpret_cast<TQ*>(wbase + degree_stage_bytes<LPP, TO, GRAD>());
    TQ* const state = sbase + pt;                  // column entry m at [PPW m]
    const int nstate = degree_state_cols<GRAD, DOWN>(L) * PPW;
    const int64_t K = int64_t(L + 1) * (L + 1);
    const int64_t ntiles = (n + PPW - 1) / PPW;

    for (int64_t tile = int64_t(blockIdx.x) * W + warp; tile < ntiles; tile += int64_t(gridDim.x) * W) {
        const int64_t p0 = tile * PPW;
        const int np = int(min(int64_t(PPW), n - p0));
        DegPoint<TQ> P;
        P.x = P.y = P.z = TQ(0);
        P.ir = TQ(1);
        if (pt < np) {
            P.x = TQ(xyz[3 * (p0 + pt)]);
            P.y = TQ(xyz[3 * (p0 + pt) + 1]);
            P.z = TQ(xyz[3 * (p0 + pt) + 2]);
        }
        // Sums of squares with explicit fma, so that every variant of the
        // kernel rounds them alike; for the normalized form u = xyz / r and
        // r2 = |u|^2 of the rounded u (0 at r = 0), as in unit_point.
        if (NORM) {
            const TQ rr = fma(P.x, P.x, fma(P.y, P.y, P.z * P.z));
            P.ir = rr > TQ(0) ? TQ(1) / sqrt(rr) : TQ(0);
            P.x *= P.ir;
            P.y *= P.ir;
            P.z *= P.ir;
        }
        P.rxy2 = fma(P.x, P.x, P.y * P.y);
        P.r2 = fma(P.z, P.z, P.rxy2);
        TO* const sph_t = sph + p0 * K;
        TO* const dsph_t = GRAD ? dsph + p0 * 3 * K : nullptr;

        // Starting c/s pairs of this lane's channel class: a0 = (x+iy)^h,
        // b0 = (x+iy)^(h-1) (for h = 0: (x+iy)^(LPP-1), the value b takes
        // after the m = 0 step), w = (x+iy)^LPP.
        const CS<TQ> xy{P.x, P.y};
        CS<TQ> a0{TQ(1), TQ(0)}, b0{TQ(1), TQ(0)}, w{TQ(1), TQ(0)};
#pragma unroll
        for (int t = 0; t < LPP; ++t) {
            if (t < h) a0 = a0.times(xy);
            if (t < (h > 0 ? h - 1 : LPP - 1)) b0 = b0.times(xy);
            w = w.times(xy);
        }

        // State columns of this tile's points.
        TQ* q1 = state;                        // UP: Qtilde_{l-1}   DOWN: c_m table
        TQ* q2 = state + PPW * (L + 2);        // UP: Qtilde_{l-2}   DOWN: s_m table (L+1 entries)
        TQ* prev = state + PPW * (2 * L + 2);  // DOWN + GRAD: Qtilde_{l-1}
        if (!DOWN) {
            for (int e = lane; e < nstate; e += 32) sbase[e] = TQ(0);
            __syncwarp();
        } else {
            TQ* ct = state;
            TQ* stb = state + PPW * (L + 1);
            CS<TQ> c{TQ(1), TQ(0)};
            for (int m = 0; m <= L; ++m) {  // Eq. iter-sc
                ct[PPW * m] = c.c;
                stb[PPW * m] = c.s;
                c = c.times(xy);
            }
            if (GRAD)
                for (int m = 0; m <= L + 1; ++m) prev[PPW * m] = TQ(0);
        }

        int l = 0;
        while (l <= L) {
            if (2 * l + 1 <= kSlots) {
                // Whole small degrees la..lb, contiguous columns la^2 .. (lb+1)^2-1.
                const int la = l;
                int lb = l;
                while (lb < L && (lb + 2) * (lb + 2) - la * la <= kSlots) ++lb;
                const int colA0 = la * la;
                for (int d = la; d <= lb; ++d) {
                    const int c0 = d * d + d - colA0;
                    if (!DOWN) {
                        CS<TQ> a = a0, b = b0;
                        up_chunk<LPP, GRAD, NORM>(d, 0, d, h, c0, c0, tab, P, inv_sqrt2, q1, q2, stl, a, b, w);
                        TQ* t = q1;
                        q1 = q2;
                        q2 = t;
                        if (LPP > 1) __syncwarp();  // degree d+1 reads other lanes' channels
                    } else {
                        TQ qa1 = TQ(0), qa2 = TQ(0), pn = TQ(0);
                        TQ cc = state[PPW * d], ss = state[PPW * (L + 1 + d)];
                        down_chunk<GRAD, NORM>(d, 0, d, c0, c0, tab, P, inv_sqrt2, state, state + PPW * (L + 1),
                                               prev, stl, qa1, qa2, pn, cc, ss);
                    }
                }
                const int nc = (lb + 1) * (lb + 1) - colA0;
                flush_stage<PPW, GRAD>(stw, sph_t, dsph_t, K, np, nc, nc, colA0, colA0, lane);
                l = lb + 1;
            } else {
                const int ctr = l * l + l;
                if (!DOWN) {
                    CS<TQ> a = a0, b = b0;
                    for (int m_lo = 0; m_lo <= l; m_lo += kMC) {
                        const int m_hi = min(l, m_lo + kMC - 1);
                        const int colA0 = ctr - m_hi;
                        const int nA = m_lo == 0 ? 2 * m_hi + 1 : m_hi - m_lo + 1;
                        const int nc = m_lo == 0 ? nA : 2 * nA;
                        const int offB = m_lo == 0 ? colA0 : ctr + m_lo - nA;
                        up_chunk<LPP, GRAD, NORM>(l, m_lo, m_hi, h, ctr - offB, ctr - colA0, tab, P, inv_sqrt2, q1,
                                                  q2, stl, a, b, w);
                        flush_stage<PPW, GRAD>(stw, sph_t, dsph_t, K, np, nc, nA, colA0, offB, lane);
                    }
                    TQ* t = q1;
                    q1 = q2;
                    q2 = t;
                } else {
                    TQ qa1 = TQ(0), qa2 = TQ(0), pn = TQ(0);
                    TQ cc = state[PPW * l], ss = state[PPW * (L + 1 + l)];
                    for (int m_hi = l; m_hi >= 0; m_hi -= kMC) {
                        const int m_lo = max(0, m_hi - kMC + 1);
                        const int colA0 = ctr - m_hi;
                        const int nA = m_lo == 0 ? 2 * m_hi + 1 : m_hi - m_lo + 1;
                        const int nc = m_lo == 0 ? nA : 2 * nA;
                        const int offB = m_lo == 0 ? colA0 : ctr + m_lo - nA;
                        down_chunk<GRAD, NORM>(l, m_lo, m_hi, ctr - offB, ctr - colA0, tab, P, inv_sqrt2, state,
                                               state + PPW * (L + 1), prev, stl, qa1, qa2, pn, cc, ss);
                        flush_stage<PPW, GRAD>(stw, sph_t, dsph_t, K, np, nc, nA, colA0, offB, lane);
                    }
                }
                ++l;
            }
        }
        __syncwarp();  // the next tile re-initialises the state
    }
}

// Warps per block: enough to fill the SM in few blocks without one block
// holding most of its shared memory.
int default_warps(size_t per_warp) {
    const size_t cap = 56 * 1024;
    return int(std::max<size_t>(1, std::min<size_t>(4, cap / std::max<size_t>(per_warp, 1))));
}

constexpr int kLPP = SPH_DEGREE_DOWN ? 1 : SPH_DEGREE_LPP;
static_assert(kLPP == 1 || kLPP == 2 || kLPP == 4, "lanes per point: 1, 2 or 4");

template <typename TI, typename TQ, typename TO, bool GRAD, bool NORM, bool DOWN, bool CT>
int launch_degree(const FwdArgs& a, const TQ* tb) {
    constexpr int PPW = 32 / kLPP;
    auto kern = degree_fwd_kernel<TI, TQ, TO, GRAD, NORM, DOWN, CT, kLPP>;
    const size_t per_warp = degree_warp_bytes<kLPP, TQ, TO, GRAD, DOWN>(a.l_max);
    const int W = a.launch.warps_per_block > 0 ? a.launch.warps_per_block : default_warps(per_warp);
    const size_t smem = size_t(W) * per_warp;
    if (smem > size_t(max_smem_optin())) return int(cudaErrorInvalidConfiguration);
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(reinterpret_cast<const void*>(kern), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(smem));
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
    const int64_t ntiles = (a.n + PPW - 1) / PPW;
    const int64_t want = (ntiles + W - 1) / W;
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(bps) * sm_count())));
    kern<<<grid, 32 * W, smem, static_cast<cudaStream_t>(a.stream)>>>(
        static_cast<const TI*>(a.xyz), a.n, a.l_max, tb, TQ(host_tables().inv_sqrt2), static_cast<TO*>(a.sph),
        static_cast<TO*>(a.dsph));
    return int(cudaGetLastError());
}

template <typename TI, typename TQ, typename TO, bool DOWN, bool CT>
int launch_degree_flags(const FwdArgs& a, const TQ* tb) {
    const bool grad = a.dsph != nullptr, norm = a.normalized != 0;
    if (grad)
        return norm ? launch_degree<TI, TQ, TO, true, true, DOWN, CT>(a, tb)
                    : launch_degree<TI, TQ, TO, true, false, DOWN, CT>(a, tb);
    return norm ? launch_degree<TI, TQ, TO, false, true, DOWN, CT>(a, tb)
                : launch_degree<TI, TQ, TO, false, false, DOWN, CT>(a, tb);
}

// Uploads this translation unit's FP32 constant tables once per device.
template <bool DOWN>
bool ensure_const_tables() {
    static std::mutex mu;
    static bool ready[64] = {false};
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) {
        cudaGetLastError();
        return false;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (ready[d]) return true;
    const HostTables& h = host_tables();
    std::vector<float4> t4(kConstTri);
    std::vector<float> tf(kConstTri);
    for (int l = 0; l <= kConstL; ++l)
        for (int m = 0; m <= l; ++m) {
            const int i = tri(l, m);
            const double S = m == l ? h.qll[i] : 0.0;
            double A, B;
            if (DOWN) {
                A = h.al[i];
                B = h.be[i];
            } else {
                A = m <= l - 2 ? h.a[i] : (m == l - 1 ? h.d[i] : 0.0);
                B = m <= l - 2 ? h.b[i] : 0.0;
            }
            t4[i] = make_float4(float(A), float(B), float(S), float(h.e[i]));
            tf[i] = float(h.fz[i]);
        }
    if (cudaMemcpyToSymbol(c_tab4, t4.data(), sizeof(float4) * kConstTri) != cudaSuccess ||
        cudaMemcpyToSymbol(c_tabf, tf.data(), sizeof(float) * kConstTri) != cudaSuccess) {
        set_error("upload of the DEGREE constant tables failed");
        return false;
    }
    ready[d] = true;
    return true;
}

template <bool DOWN>
int degree_fwd_dir(const FwdArgs& a) {
    const int tdt = (a.dtype == SPH_F64 || a.qprec == SPH_Q_F64) ? SPH_F64 : SPH_F32;
    const void* tb = DOWN ? device_tables_down(tdt) : device_tables(tdt);
    if (!tb) return int(cudaErrorMemoryAllocation);
    if (a.dtype == SPH_F64)
        return launch_degree_flags<double, double, double, DOWN, false>(a, static_cast<const double*>(tb));
    if (a.qprec == SPH_Q_F64) {
        if (a.out == SPH_OUT_BF16)
            return launch_degree_flags<float, double, __nv_bfloat16, DOWN, false>(a, static_cast<const double*>(tb));
        return launch_degree_flags<float, double, float, DOWN, false>(a, static_cast<const double*>(tb));
    }
    const float* tf = static_cast<const float*>(tb);
    if (a.l_max <= kConstL) {
        if (!ensure_const_tables<DOWN>()) return int(cudaErrorMemoryAllocation);
        if (a.out == SPH_OUT_BF16) return launch_degree_flags<float, float, __nv_bfloat16, DOWN, true>(a, tf);
        return launch_degree_flags<float, float, float, DOWN, true>(a, tf);
    }
    if (a.out == SPH_OUT_BF16) return launch_degree_flags<float, float, __nv_bfloat16, DOWN, false>(a, tf);
    return launch_degree_flags<float, float, float, DOWN, false>(a, tf);
}

}  // namespace

#if SPH_DEGREE_DOWN
int degree_fwd_down(const FwdArgs& a) { return degree_fwd_dir<true>(a); }
#elif SPH_DEGREE_LPP == 1
int degree_fwd_up1(const FwdArgs& a) { return degree_fwd_dir<false>(a); }
#elif SPH_DEGREE_LPP == 2
int degree_fwd_up2(const FwdArgs& a) { return degree_fwd_dir<false>(a); }
#else
int degree_fwd_up4(const FwdArgs& a) { return degree_fwd_dir<false>(a); }
#endif

}  // namespace sph
