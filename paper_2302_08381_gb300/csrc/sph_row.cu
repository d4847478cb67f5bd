// ROW kernel family: FP32 forward (values, gradients) for 16 <= l_max <= 63
// whose global writes are long contiguous runs.
//
// On GB300 the write stream reaches the HBM roofline only in contiguous runs
// of about 1 KB or more (measured: scattered 128-byte runs reach ~0.8 TB/s,
// 512-byte runs ~3.2 TB/s, >= 1 KB runs ~6.2 TB/s). A kernel that writes one
// degree (2l+1 columns) of many output rows at a time cannot get there, so
// this family keeps each point's output rows in shared memory in windows of
// whole degrees (about 130..250 columns per plane) and sends every window
// with TMA bulk copies of 32-byte-aligned runs.
//
// Work decomposition (arXiv 2302.08381, Section 2): a group of 8 lanes owns a
// point, a warp owns 4 consecutive points. The degree l is the outer loop and
// is the same for the whole group; lane j owns the m channels m = j (mod 8),
// whose Qtilde_{l-1}^m, Qtilde_{l-2}^m (Eq. iter-q with the prefactors folded
// in, Appendix C) and c_m, s_m, c_{m-1}, s_{m-1} (Eq. iter-sc) stay in
// registers; the derivative identities of Eq. iter-deri need
// Qtilde_{l-1}^{m+1}, which the neighbouring lane holds and passes with a
// shuffle. At every degree the lanes of a group write 8 consecutive columns
// per side, so the shared-memory stores are conflict-free within a group.
//
// The translation unit is compiled twice: SPH_ROW_PART 0 instantiates the
// kernels for 3..5 channels per lane (l_max 16..47), 1 for 6..8 (48..63).
#include <cuda_runtime.h>

#include <algorithm>

#include "sph_core.cuh"
#include "sph_internal.h"

#ifndef SPH_ROW_PART
#define SPH_ROW_PART 0
#endif

namespace sph {

namespace {

constexpr int kG = 8;         // lanes per point
constexpr int kPW = 32 / kG;  // points per warp
constexpr int kCap = 256;     // columns buffered before a window is sent (the backward's window size)

// Per output type, channel slots and window policy: elements per 32-byte
// sector, the plane buffer length (SE pre-slots for the row head, then kCap
// columns, or with MINRUN kCap - 1 columns plus one whole degree of at most
// 16 NCH - 1 columns plus a carried partial sector; a multiple of 16 bytes),
// and the distance between the buffers of consecutive points, which is 8
// four-byte words past a multiple of 32 so that the four point groups of a
// warp, each writing 8 consecutive columns, start 8 banks apart.
template <typename TO, int NCH, bool MINRUN>
struct RowGeom {
    static constexpr int SE = 32 / int(sizeof(TO));
    static constexpr int EL16 = 16 / int(sizeof(TO));
    static constexpr int BUF = MINRUN ? (SE + kCap + 16 * NCH + 8 + EL16 - 1) / EL16 * EL16 : SE + kCap;
    template <int NPL>
    __host__ __device__ static constexpr int point_stride() {
        constexpr int words = NPL * BUF * int(sizeof(TO)) / 4;
        constexpr int pad = ((8 - words % 32) + 32) % 32;  // words of padding
        return NPL * BUF + pad * 4 / int(sizeof(TO));
    }
};

template <typename TO, bool GRAD, int NCH, bool MINRUN>
__host__ __device__ constexpr size_t row_warp_bytes() {
    return size_t(kPW) * RowGeom<TO, NCH, MINRUN>::template point_stride<GRAD ? 4 : 1>() * sizeof(TO);
}

struct CSf {
    float c, s;
    __device__ __forceinline__ CSf times(const CSf& w) const {
        return CSf{fmaf(c, w.c, -(s * w.s)), fmaf(c, w.s, s * w.c)};
    }
};

// Forward kernel. Per degree d and channel slot k (m = j + 8k) a lane runs
// one step of Eq. iter-q (coefficients from the lane-interleaved table, one
// degree ahead, so no index arithmetic), then Eq. real-sh-cartesian and
// Eq. iter-deri for the columns d^2+d+m and d^2+d-m of every plane, stored
// through per-window plane pointers at compile-time offsets. The m = 0
// column takes the same path with c_0 = 1/sqrt2 and s_0 = 0 (its -m stores
// land on the same column first and are overwritten).
constexpr int kRowMaxWarps = 2;  // warps per block (measured: 1 >= 2 > 4 > 8); the bound frees registers

template <typename TO, bool GRAD, bool NORM, int NCH, bool MINRUN>
__global__ void __launch_bounds__(32 * kRowMaxWarps) row_fwd_kernel(const float* __restrict__ xyz, int64_t n, int L,
                                                      const float4* __restrict__ rowA,
                                                      const float* __restrict__ rowF, float inv_sqrt2,
                                                      TO* __restrict__ sph, TO* __restrict__ dsph) {
    constexpr int NPL = GRAD ? 4 : 1;
    constexpr int SE = RowGeom<TO, NCH, MINRUN>::SE;
    constexpr int BUF = RowGeom<TO, NCH, MINRUN>::BUF;
    constexpr int PSTR = RowGeom<TO, NCH, MINRUN>::template point_stride<NPL>();
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const int g = lane / kG;  // point of the warp tile
    const int j = lane % kG;  // channel class m = j (mod 8)
    TO* const pst = reinterpret_cast<TO*>(smem) + (size_t(warp) * kPW + g) * PSTR;  // this point's planes
    const int64_t K = int64_t(L + 1) * (L + 1);
    const int64_t ntiles = (n + kPW - 1) / kPW;
    const int nb_lane = (lane & ~(kG - 1)) | ((j + 1) & (kG - 1));  // the lane holding channel m+1's class
    // this lane's stream: entry (d, k) at laneA[(d * kRowSlots + k) * kRowLanes]
    const float4* const laneA = rowA + j;
    const float* const laneF = rowF + j;

    for (int64_t tile = int64_t(blockIdx.x) * W + warp; tile < ntiles; tile += int64_t(gridDim.x) * W) {
        const int64_t p = tile * kPW + g;
        const bool live = p < n;
        float x = 0.f, y = 0.f, z = 0.f, ir = 1.f;
        if (live) {
            x = xyz[3 * p];
            y = xyz[3 * p + 1];
            z = xyz[3 * p + 2];
        }
        if (NORM) {
            const float rr = fmaf(x, x, fmaf(y, y, z * z));
            ir = rr > 0.f ? 1.f / sqrtf(rr) : 0.f;
            x *= ir;
            y *= ir;
            z *= ir;
        }
        const float r2 = fmaf(z, z, fmaf(x, x, y * y));

        // c_m + i s_m and c_{m-1} + i s_{m-1} of the lane's channels m = j + 8k
        // (Eq. iter-sc); c_0 carries the 1/sqrt2 of the m = 0 column.
        float cm[NCH], sm[NCH], cm1[NCH], sm1[NCH];
        {
            const CSf xy{x, y};
            CSf a{1.f, 0.f}, b{1.f, 0.f}, w8{1.f, 0.f}, p7{1.f, 0.f};
#pragma unroll
            for (int t = 0; t < kG; ++t) {
                if (t < j) a = a.times(xy);
                if (t < j - 1) b = b.times(xy);
                if (t < kG - 1) p7 = p7.times(xy);
                w8 = w8.times(xy);
            }
            if (j == 0) b = p7;  // channel 8k (k >= 1) needs (x + i y)^(8k-1)
#pragma unroll
            for (int k = 0; k < NCH; ++k) {
                const bool none = (j == 0 && k == 0);  // m = 0: no c_{m-1}
                cm[k] = none ? inv_sqrt2 : a.c;
                sm[k] = none ? 0.f : a.s;
                cm1[k] = none ? 0.f : b.c;
                sm1[k] = none ? 0.f : b.s;
                a = a.times(w8);
                if (!none) b = b.times(w8);
            }
        }
        float q1[NCH], q2[NCH];  // Qtilde_{l-1}^m, Qtilde_{l-2}^m
#pragma unroll
        for (int k = 0; k < NCH; ++k) q1[k] = q2[k] = 0.f;

        // Output rows of this point: plane 0 = sph row, planes 1..3 = dsph rows.
        // s[i] = first column held in the plane buffer (at slot SE); it is
        // 32-byte aligned in global memory, so every bulk copy starts and
        // (except at the row end) ends on a sector boundary.
        TO* grow[NPL];
        int s[NPL];
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            grow[i] = (i == 0) ? sph + p * K : dsph + p * 3 * K + (i - 1) * K;
            const int phase = int((reinterpret_cast<uintptr_t>(grow[i]) / sizeof(TO)) % SE);
            s[i] = (SE - phase) % SE;
        }

        // Degree-0 coefficients; later degrees are loaded one degree ahead.
        float4 ta[NCH];
        float tf[NCH];
#pragma unroll
        for (int k = 0; k < NCH; ++k) {
            ta[k] = laneA[k * kRowLanes];
            tf[k] = laneF[k * kRowLanes];
        }
        const float xi = NORM ? x * ir : x, yi = NORM ? y * ir : y;
        const float jf = float(j);

        int l = 0;
        bool first = true;
        while (l <= L) {
            // A window of whole degrees [l, lw), the same for every point of
            // the warp (the lanes shuffle across point groups): degrees are
            // added while the window fits kCap - SE + 1 new columns, or, with
            // MINRUN, until it holds at least that many (runs of >= kCap - SE
            // columns whatever the degree's width, in larger buffers).
            // Column c of plane i is staged at pst[i * BUF + SE - s[i] + c].
            TO* pp[NPL];  // + j: the +m columns
            TO* pn[NPL];  // - j: the -m columns
#pragma unroll
            for (int i = 0; i < NPL; ++i) {
                pp[i] = pst + (i * BUF + SE - s[i] + j);
                pn[i] = pst + (i * BUF + SE - s[i] - j);
            }
            int d = l;
            while (true) {
                const int ctr = d * d + d;
                const int kend = d / kG;  // channels m = j + 8k <= d need k <= d/8 (same for the whole warp)
                const int dn = d < L ? d + 1 : d;
                // all slots every degree (zeros where m > d): a degree-dependent
                // bound here keeps more registers live and ran slower
                float4 na[NCH];
                float nf[NCH];
#pragma unroll
                for (int k = 0; k < NCH; ++k) {  // coefficients of the next degree
                    na[k] = laneA[(dn * kRowSlots + k) * kRowLanes];
                    if (GRAD) nf[k] = laneF[(dn * kRowSlots + k) * kRowLanes];
                }
                float ax = 0.f, ay = 0.f, az = 0.f;
                if (NORM && GRAD) {
                    const float lir = float(d) * ir;
                    ax = lir * x;
                    ay = lir * y;
                    az = lir * z;
                }
                TO* qp[NPL];
                TO* qn_[NPL];
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    qp[i] = pp[i] + ctr;
                    qn_[i] = pn[i] + ctr;
                }
#pragma unroll
                for (int k = 0; k < NCH; ++k) {
                    if (k > kend) break;
                    const float4 t0 = ta[k];  // {A, B, S, e}
                    const float src = (j == 0) ? (k + 1 < NCH ? q1[k + 1 < NCH ? k + 1 : k] : 0.f) : q1[k];
                    const float qnb = __shfl_sync(0xffffffffu, src, nb_lane);  // Qtilde_{l-1}^{m+1}
                    // zero for m > d: the table holds zeros there
                    const float q = fmaf(t0.x * z, q1[k], fmaf(-(t0.y * r2), q2[k], t0.z));
                    if (j + kG * k <= d) {
                        const float c = cm[k], sn = sm[k];
                        const float vc = q * c, vs = q * sn;  // +m (cos) and -m (sin) columns
                        qn_[0][-kG * k] = OutConv<TO>::cv(vs);
                        qp[0][kG * k] = OutConv<TO>::cv(vc);
                        if (GRAD) {
                            // Eq. iter-deri (prefactors folded)
                            const float E1 = t0.w * qnb;  // e Qtilde_{l-1}^{m+1}
                            const float Qz = NORM ? (tf[k] * q1[k]) * ir : tf[k] * q1[k];
                            const float Qx = xi * E1, Qy = yi * E1;
                            const float mQ = (NORM ? (jf + float(kG * k)) * ir : jf + float(kG * k)) * q;
                            const float mc1 = mQ * cm1[k], ms1 = mQ * sm1[k];
                            const float tx_c = NORM ? fmaf(-ax, vc, mc1) : mc1;
                            const float tx_s = NORM ? fmaf(-ax, vs, ms1) : ms1;
                            const float ty_c = NORM ? fmaf(-ay, vc, -ms1) : -ms1;
                            const float ty_s = NORM ? fmaf(-ay, vs, mc1) : mc1;
                            qn_[1 % NPL][-kG * k] = OutConv<TO>::cv(fmaf(Qx, sn, tx_s));
                            qn_[2 % NPL][-kG * k] = OutConv<TO>::cv(fmaf(Qy, sn, ty_s));
                            qn_[3 % NPL][-kG * k] = OutConv<TO>::cv(NORM ? fmaf(Qz, sn, -az * vs) : Qz * sn);
                            qp[1 % NPL][kG * k] = OutConv<TO>::cv(fmaf(Qx, c, tx_c));
                            qp[2 % NPL][kG * k] = OutConv<TO>::cv(fmaf(Qy, c, ty_c));
                            qp[3 % NPL][kG * k] = OutConv<TO>::cv(NORM ? fmaf(Qz, c, -az * vc) : Qz * c);
                        }
                    }
                    q2[k] = q1[k];
                    q1[k] = q;
                }
#pragma unroll
                for (int k = 0; k < NCH; ++k) {
                    ta[k] = na[k];
                    if (GRAD) tf[k] = nf[k];
                }
                ++d;
                if (d > L) break;
                if (MINRUN ? (d * d - l * l >= kCap - (SE - 1)) : ((d + 1) * (d + 1) - l * l > kCap - (SE - 1)))
                    break;
            }
            const int lw = d;

            // Send the window: per plane, the sector-aligned run [s, e) by one
            // bulk copy; the row head (first window) and the row tail (last
            // window) with plain stores; the rest (< one sector) is carried.
            const int c_hi = lw * lw;
            const bool last = lw > L;
            fence_proxy_async_smem();
            __syncwarp();
            int e[NPL];
#pragma unroll
            for (int i = 0; i < NPL; ++i) {
                const int run = last ? (c_hi - s[i]) * int(sizeof(TO)) / 16 * 16 / int(sizeof(TO))
                                     : (c_hi - s[i]) / SE * SE;
                e[i] = s[i] + max(run, 0);
            }
            if (live) {
                if (j == 0) {
#pragma unroll
                    for (int i = 0; i < NPL; ++i)
                        if (e[i] > s[i])
                            bulk_store(grow[i] + s[i], pst + i * BUF + SE, uint32_t((e[i] - s[i]) * sizeof(TO)));
                    bulk_commit();
                }
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    if (first)
                        for (int c = j; c < s[i]; c += kG) grow[i][c] = pst[i * BUF + c - s[i] + SE];
                    if (last)
                        for (int c = e[i] + j; c < c_hi; c += kG) grow[i][c] = pst[i * BUF + c - s[i] + SE];
                }
                if (j == 0) bulk_wait_read_all();  // the buffers are reused below
            }
            __syncwarp();
            if (!last) {
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    for (int c = e[i] + j; c < c_hi; c += kG) pst[i * BUF + c - e[i] + SE] = pst[i * BUF + c - s[i] + SE];
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

// ------------------------------------------------------------- backward
// Fused recompute-backward with the same decomposition: dxyz_i = sum_k g_k
// dY_k/dx_i (Eq. iter-deri), the recursion recomputed in registers, the
// upstream-gradient row of each point read in the same windows of whole
// degrees by TMA bulk loads (double buffered: the next window is in flight
// while the current one is used), the unaligned window edges by plain loads.
// Lane j accumulates its channels' terms; the 8 lanes of a point reduce with
// shuffles at the end. Every mbarrier wait is bounded; a timeout sets the
// device status word and skips the rest of the launch.
constexpr int kBPad = 4;                  // slots before a window's first 16-byte-aligned column
constexpr int kBBuf = kBPad + kCap + 8;   // floats per window buffer
constexpr uint32_t kRowWaitPolls = 1u << 22;

__host__ __device__ constexpr size_t row_bwd_warp_bytes() {
    return size_t(kPW) * 2 * kBBuf * sizeof(float) + size_t(kPW) * 2 * sizeof(uint64_t);
}

// Window of whole degrees starting at degree l: [l, lw).
__device__ __forceinline__ int row_window_end(int l, int L) {
    int lw = l + 1;
    while (lw <= L && (lw + 1) * (lw + 1) - l * l <= kCap - 7) ++lw;
    return lw;
}

// Starts loading the columns [c0, c1) of the upstream-gradient row `grow` into
// `buf` (column c at buf[c - s + kBPad], s = first 16-byte-aligned column >= c0):
// the aligned middle by one bulk copy completing on `bar` (issued by lane j = 0),
// the edges by plain loads of the group's lanes. Returns whether a bulk copy was issued.
__device__ __forceinline__ bool row_window_load(const float* __restrict__ grow, int c0, int c1, float* buf,
                                                uint64_t* bar, int j) {
    const int phase = int((reinterpret_cast<uintptr_t>(grow + c0) / sizeof(float)) % 4);
    const int s = c0 + (4 - phase) % 4;
    const int e = s + max(0, (c1 - s) / 4 * 4);
    const bool bulk = e > s;
    if (bulk && j == 0) {
        mbar_arrive_expect_tx(bar, uint32_t((e - s) * sizeof(float)));
        bulk_load(buf + kBPad, grow + s, uint32_t((e - s) * sizeof(float)), bar);
    }
    for (int c = c0 + j; c < min(s, c1); c += kG) buf[c - s + kBPad] = grow[c];
    for (int c = max(e, c0) + j; c < c1; c += kG) buf[c - s + kBPad] = grow[c];
    return bulk;
}

template <bool NORM, int NCH>
__global__ void __launch_bounds__(256) row_bwd_kernel(const float* __restrict__ xyz, const float* __restrict__ g,
                                                      int64_t n, int L, const float* __restrict__ tb,
                                                      float inv_sqrt2, float* __restrict__ dxyz,
                                                      uint32_t* __restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const int gi = lane / kG;  // point of the warp tile
    const int j = lane % kG;   // channel class m = j (mod 8)
    unsigned char* wbase = smem + size_t(warp) * row_bwd_warp_bytes();
    float* const bufs = reinterpret_cast<float*>(wbase) + size_t(gi) * 2 * kBBuf;  // this point's two windows
    uint64_t* const bars =
        reinterpret_cast<uint64_t*>(wbase + size_t(kPW) * 2 * kBBuf * sizeof(float)) + 2 * gi;
    const int64_t K = int64_t(L + 1) * (L + 1);
    const int64_t ntiles = (n + kPW - 1) / kPW;
    const float4* __restrict__ t4 = reinterpret_cast<const float4*>(tb);
    const int nb_lane = (lane & ~(kG - 1)) | ((j + 1) & (kG - 1));
    const float jf = float(j);

    if (j == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
    }
    fence_proxy_async_smem();
    __syncwarp();
    uint32_t parity = 0;   // bit b: phase of buffer b's next completion (same in the 8 lanes of a point)
    uint32_t pending = 0;  // bit b: a bulk load into buffer b is in flight
    bool failed = false;

    for (int64_t tile = int64_t(blockIdx.x) * W + warp; tile < ntiles && !failed; tile += int64_t(gridDim.x) * W) {
        const int64_t p = tile * kPW + gi;
        const bool live = p < n;
        float x = 0.f, y = 0.f, z = 0.f, ir = 1.f;
        if (live) {
            x = xyz[3 * p];
            y = xyz[3 * p + 1];
            z = xyz[3 * p + 2];
        }
        if (NORM) {
            const float rr = fmaf(x, x, fmaf(y, y, z * z));
            ir = rr > 0.f ? 1.f / sqrtf(rr) : 0.f;
            x *= ir;
            y *= ir;
            z *= ir;
        }
        const float r2 = fmaf(z, z, fmaf(x, x, y * y));
        const float* grow = g + (live ? p : 0) * K;

        float cm[NCH], sm[NCH], cm1[NCH], sm1[NCH];
        {
            const CSf xy{x, y};
            CSf a{1.f, 0.f}, b{1.f, 0.f}, w8{1.f, 0.f}, p7{1.f, 0.f};
#pragma unroll
            for (int t = 0; t < kG; ++t) {
                if (t < j) a = a.times(xy);
                if (t < j - 1) b = b.times(xy);
                if (t < kG - 1) p7 = p7.times(xy);
                w8 = w8.times(xy);
            }
            if (j == 0) b = p7;
#pragma unroll
            for (int k = 0; k < NCH; ++k) {
                cm[k] = a.c;
                sm[k] = a.s;
                const bool none = (j == 0 && k == 0);
                cm1[k] = none ? 0.f : b.c;
                sm1[k] = none ? 0.f : b.s;
                a = a.times(w8);
                if (!none) b = b.times(w8);
            }
        }
        float q1[NCH], q2[NCH];
#pragma unroll
        for (int k = 0; k < NCH; ++k) q1[k] = q2[k] = 0.f;
        float4 ta[NCH];
        float tf[NCH];
#pragma unroll
        for (int k = 0; k < NCH; ++k) {
            ta[k] = t4[0];
            tf[k] = tb[4];
        }
        float ax = 0.f, ay = 0.f, az = 0.f, S = 0.f;

        // window 0 into buffer 0
        int l = 0, lw = row_window_end(0, L), buf = 0;
        if (live && row_window_load(grow, 0, lw * lw, bufs, &bars[0], j)) pending |= 1u;
        while (l <= L) {
            // next window into the other buffer (free: consumed before the last fence + sync)
            const int ln = lw, lwn = ln <= L ? row_window_end(ln, L) : ln;
            if (live && ln <= L && row_window_load(grow, ln * ln, lwn * lwn, bufs + (buf ^ 1) * kBBuf, &bars[buf ^ 1], j))
                pending |= 1u << (buf ^ 1);
            // this window's bulk part
            if (live && (pending & (1u << buf))) {
                if (mbar_wait_bounded(&bars[buf], (parity >> buf) & 1u, kRowWaitPolls)) {
                    parity ^= 1u << buf;
                    pending &= ~(1u << buf);
                } else {
                    if (j == 0) atomicOr(status, kStatusLoadTimeout);
                    failed = true;
                }
            }
            if (__any_sync(0xffffffffu, failed)) {
                failed = true;
                break;
            }
            __syncwarp();  // edge elements loaded by the other lanes
            const float* gb = bufs + buf * kBBuf;
            const int phase = int((reinterpret_cast<uintptr_t>(grow + l * l) / sizeof(float)) % 4);
            const int s0 = l * l + (4 - phase) % 4;  // column at gb[kBPad]
            for (int d = l; d < lw; ++d) {
                const int ctr = d * d + d;
                const int kend = d / kG;
                const int dn = d < L ? d + 1 : L;
                float4 na[NCH];
                float nf[NCH];
#pragma unroll
                for (int k = 0; k < NCH; ++k) {
                    const int mk = j + kG * k;
                    const int i = tri(dn, mk <= dn ? mk : dn);
                    na[k] = t4[2 * i];
                    nf[k] = tb[8 * i + 4];
                }
                const float lf = float(d);
#pragma unroll
                for (int k = 0; k < NCH; ++k) {
                    if (k > kend) break;
                    const int m = j + kG * k;
                    const bool on = m <= d;
                    const float4 t0 = ta[k];
                    const float src = (j == 0) ? (k + 1 < NCH ? q1[k + 1 < NCH ? k + 1 : k] : 0.f) : q1[k];
                    const float qn = __shfl_sync(0xffffffffu, src, nb_lane);
                    float q = fmaf(t0.x * z, q1[k], fmaf(-(t0.y * r2), q2[k], t0.z));
                    q = on ? q : 0.f;
                    if (on) {
                        const float E1 = t0.w * qn;
                        const float Qz = tf[k] * q1[k];
                        const float Qx = x * E1, Qy = y * E1;
                        const float gp = gb[ctr + m - s0 + kBPad];
                        if (k == 0 && j == 0) {  // m = 0: Ytilde_l^0 = Q / sqrt2
                            ax = fmaf(Qx, gp, ax);
                            ay = fmaf(Qy, gp, ay);
                            az = fmaf(Qz, gp, az);
                            if (NORM) S = fmaf(lf * (q * inv_sqrt2), gp, S);
                        } else {
                            const float gn = gb[ctr - m - s0 + kBPad];
                            const float c = cm[k], sn = sm[k], c1 = cm1[k], s1 = sm1[k];
                            const float A = fmaf(gp, c, gn * sn);     // g+ c_m + g- s_m
                            const float B = fmaf(gp, c1, gn * s1);    // g+ c_{m-1} + g- s_{m-1}
                            const float Cc = fmaf(gn, c1, -(gp * s1));  // g- c_{m-1} - g+ s_{m-1}
                            const float mQ = (jf + float(kG * k)) * q;
                            ax = fmaf(Qx, A, fmaf(mQ, B, ax));
                            ay = fmaf(Qy, A, fmaf(mQ, Cc, ay));
                            az = fmaf(Qz, A, az);
                            if (NORM) S = fmaf(lf * q, A, S);
                        }
                    }
                    q2[k] = q1[k];
                    q1[k] = q;
                }
#pragma unroll
                for (int k = 0; k < NCH; ++k) {
                    ta[k] = na[k];
                    tf[k] = nf[k];
                }
            }
            fence_proxy_async_smem();  // this buffer is rewritten by the async proxy two windows on
            __syncwarp();
            l = lw;
            lw = lwn;
            buf ^= 1;
        }
        if (failed) break;
        // reduce over the 8 lanes of the point
#pragma unroll
        for (int off = kG / 2; off > 0; off >>= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, off, kG);
            ay += __shfl_xor_sync(0xffffffffu, ay, off, kG);
            az += __shfl_xor_sync(0xffffffffu, az, off, kG);
            if (NORM) S += __shfl_xor_sync(0xffffffffu, S, off, kG);
        }
        if (live && j == 0) {
            if (NORM) {
                ax = ir * fmaf(-x, S, ax);
                ay = ir * fmaf(-y, S, ay);
                az = ir * fmaf(-z, S, az);
            }
            dxyz[3 * p] = ax;
            dxyz[3 * p + 1] = ay;
            dxyz[3 * p + 2] = az;
        }
    }
    if (pending && j == 0) {
        // loads issued but not observed (after a timeout) may still be in
        // flight: wait for them, bounded, before the shared memory goes away
        for (int b = 0; b < 2; ++b)
            if (pending & (1u << b)) (void)mbar_wait_bounded(&bars[b], (parity >> b) & 1u, kRowWaitPolls);
    }
    __syncwarp();
}

template <typename TO, bool GRAD, bool NORM, int NCH, bool MINRUN>
int launch_row(const FwdArgs& a) {
    const float* rt = static_cast<const float*>(device_row_tables());
    if (!rt) return int(cudaErrorMemoryAllocation);
    auto kern = row_fwd_kernel<TO, GRAD, NORM, NCH, MINRUN>;
    const size_t per_warp = row_warp_bytes<TO, GRAD, NCH, MINRUN>();
    const int W = a.launch.warps_per_block > 0 ? a.launch.warps_per_block : 1;
    if (W > kRowMaxWarps) return int(cudaErrorInvalidConfiguration);
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
    const int64_t ntiles = (a.n + kPW - 1) / kPW;
    const int64_t want = (ntiles + W - 1) / W;
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(bps) * sm_count())));
    constexpr int kEntries = kRowLanes * kRowDegrees * kRowSlots;
    kern<<<grid, 32 * W, smem, static_cast<cudaStream_t>(a.stream)>>>(
        static_cast<const float*>(a.xyz), a.n, a.l_max, reinterpret_cast<const float4*>(rt), rt + 4 * kEntries,
        float(host_tables().inv_sqrt2), static_cast<TO*>(a.sph), static_cast<TO*>(a.dsph));
    return int(cudaGetLastError());
}

template <bool NORM, int NCH>
int launch_row_bwd(const BwdArgs& a, const float* tb) {
    auto kern = row_bwd_kernel<NORM, NCH>;
    const size_t per_warp = row_bwd_warp_bytes();
    const int W = a.launch.warps_per_block > 0 ? a.launch.warps_per_block : 2;
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
    const int64_t ntiles = (a.n + kPW - 1) / kPW;
    const int64_t want = (ntiles + W - 1) / W;
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(bps) * sm_count())));
    kern<<<grid, 32 * W, smem, static_cast<cudaStream_t>(a.stream)>>>(
        static_cast<const float*>(a.xyz), static_cast<const float*>(a.g), a.n, a.l_max, tb,
        float(host_tables().inv_sqrt2), static_cast<float*>(a.dxyz), a.status);
    return int(cudaGetLastError());
}

template <int NCH>
int launch_row_bwd_flags(const BwdArgs& a, const float* tb) {
    return a.normalized ? launch_row_bwd<true, NCH>(a, tb) : launch_row_bwd<false, NCH>(a, tb);
}

// Window policy: launch.lanes_per_point 1 = windows that fit the buffer,
// 2 = windows of at least kCap - SE columns (MINRUN, larger buffers), 0 = by
// measurement on GB300 (200,000 points, l_max 16..63): FP32 rows keep the
// smaller buffers (more warps per SM) except at l_max 28..31, where windows
// that fit fall to ~160 columns (3.26 -> 3.55 TB/s at l_max 30); bf16 rows,
// half the shared memory, take the longer runs (up to +13 % at l_max 63).
inline bool row_minrun_default(int L, bool bf16) { return bf16 || (L >= 28 && L <= 31); }

template <typename TO, int NCH, bool MINRUN>
int launch_row_policy(const FwdArgs& a) {
    const bool grad = a.dsph != nullptr, norm = a.normalized != 0;
    if (grad)
        return norm ? launch_row<TO, true, true, NCH, MINRUN>(a) : launch_row<TO, true, false, NCH, MINRUN>(a);
    return norm ? launch_row<TO, false, true, NCH, MINRUN>(a) : launch_row<TO, false, false, NCH, MINRUN>(a);
}

template <typename TO, int NCH>
int launch_row_flags(const FwdArgs& a) {
    const int pol = a.launch.lanes_per_point;
    const bool minrun = pol == 2 || (pol == 0 && row_minrun_default(a.l_max, sizeof(TO) == 2));
    return minrun ? launch_row_policy<TO, NCH, true>(a) : launch_row_policy<TO, NCH, false>(a);
}

template <int NCH>
int launch_row_out(const FwdArgs& a) {
    if (a.out == SPH_OUT_BF16) return launch_row_flags<__nv_bfloat16, NCH>(a);
    return launch_row_flags<float, NCH>(a);
}

}  // namespace

#if SPH_ROW_PART == 0
int row_bwd_part0(const BwdArgs& a) {
    const float* tb = static_cast<const float*>(device_tables(SPH_F32));
    if (!tb) return int(cudaErrorMemoryAllocation);
    switch ((a.l_max + 1 + kG - 1) / kG) {
        case 3:
            return launch_row_bwd_flags<3>(a, tb);
        case 4:
            return launch_row_bwd_flags<4>(a, tb);
        default:
            return launch_row_bwd_flags<5>(a, tb);
    }
}

int row_fwd_part0(const FwdArgs& a) {
    switch ((a.l_max + 1 + kG - 1) / kG) {
        case 3:
            return launch_row_out<3>(a);
        case 4:
            return launch_row_out<4>(a);
        default:
            return launch_row_out<5>(a);
    }
}
#else
int row_bwd_part1(const BwdArgs& a) {
    const float* tb = static_cast<const float*>(device_tables(SPH_F32));
    if (!tb) return int(cudaErrorMemoryAllocation);
    switch ((a.l_max + 1 + kG - 1) / kG) {
        case 6:
            return launch_row_bwd_flags<6>(a, tb);
        case 7:
            return launch_row_bwd_flags<7>(a, tb);
        default:
            return launch_row_bwd_flags<8>(a, tb);
    }
}

int row_fwd_part1(const FwdArgs& a) {
    switch ((a.l_max + 1 + kG - 1) / kG) {
        case 6:
            return launch_row_out<6>(a);
        case 7:
            return launch_row_out<7>(a);
        default:
            return launch_row_out<8>(a);
    }
}
#endif

}  // namespace sph
