// Radial expansion fused with the harmonics (arXiv 2302.08381, Eq. expansion):
//
//   c[i, n, (l,m)] = sum_{k in centre i} R[k, n, l] * Y_l^m(x_k)
//
// for points (edge vectors) grouped by centre in CSR order. The harmonics are
// never written to memory: each warp owns a contiguous range of centres and
// streams their points in 32-point chunks that cross centre boundaries; it
// evaluates Y for a chunk (one lane per point, the unrolled recursion of the
// POINT kernels, values only) into shared memory, stages the matching rows of
// R, and then each lane accumulates the output columns it owns. Only the
// coordinates, R, the offsets and the [n_rad, K] result per centre touch HBM.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "sph_point.cuh"

namespace sph {

constexpr uint32_t kStatusBadOffsets = 2u;
constexpr int kExpansionMaxRad = 64;

// Row layout of the staged harmonics: the 2l+1 columns of degree l in groups
// of 4 slots (the last group of a degree padded with zeros), group g at word
// 4g + floor(g / 8). The lanes of one contraction round read up to 32
// consecutive groups at the same slot; without the skew of one word per block
// of 8 groups, groups 8 apart would share a bank. With it, 4d + (1 or 2 or 3)
// for groups d < 32 apart is never a multiple of 32 words, so the reads are
// free of bank conflicts, and each lane reads its 4 slots at immediate offsets.
__host__ __device__ constexpr int exp_gstart(int l) { return l == 0 ? 0 : l + (l - 1) * (l - 1) / 4; }
__host__ __device__ constexpr int exp_gbase(int g) { return 4 * g + g / 8; }
__host__ __device__ constexpr int exp_ypos(int l, int k) {
    return exp_gbase(exp_gstart(l) + (k - l * l) / 4) + (k - l * l) % 4;
}
// Row stride in words: odd, so that the lanes' stores (one row each) are
// conflict-free too.
template <int L>
__host__ __device__ constexpr int exp_row_words() {
    return (exp_gbase(exp_gstart(L + 1) - 1) + 4) | 1;
}

// Every column gets its own word inside the row, for every supported l_max.
constexpr bool exp_layout_ok() {
    for (int L = 0; L <= 16; ++L) {
        const int SY = (exp_gbase(exp_gstart(L + 1) - 1) + 4) | 1;
        int prev = -1;
        for (int l = 0; l <= L; ++l)
            for (int k = l * l; k < (l + 1) * (l + 1); ++k) {
                if (exp_ypos(l, k) <= prev) return false;
                prev = exp_ypos(l, k);
            }
        if (prev + 1 >= SY || exp_gbase(exp_gstart(L + 1) - 1) + 3 >= SY) return false;
    }
    return true;
}
static_assert(exp_layout_ok(), "grouped Y layout must be injective and inside the row");

template <typename T>
struct ValVis {
    T* row;
    __device__ __forceinline__ void emit(int l, int k, const Deriv<T>& d) { row[exp_ypos(l, k)] = d.v; }
};

constexpr int kExpBatch = 32;  // centres whose CSR offsets a warp holds in registers
// Radial-row buffers per warp. One buffer, refilled after each chunk's
// contraction while the next chunk's rows were prefetched into L2, leaves
// room for 12 resident warps per SM where two buffers (the next chunk's rows
// loaded into shared memory during the current one) leave 8: measured on
// GB300, 0.267 against 0.369 ms (l_max 6, 8 radial, 100k centres x ~40
// points).
constexpr int kExpRBuf = 1;

// Per-warp shared memory: Y rows of a 32-point chunk (grouped layout),
// kExpRBuf buffers of the chunk's radial rows in their global layout
// [e][n][l] (filled by bulk copies), the [n_rad, K] partial sums of a
// centre that continues into the next chunk, the chunk's segment table (end
// of each centre's points within the chunk, and the centre) and two mbarriers.
template <int L, typename T>
__host__ __device__ constexpr size_t expansion_warp_bytes(int nr) {
    constexpr int K = (L + 1) * (L + 1);
    const int RW = nr * (L + 1);
    // radial buffers: 32 rows plus 3 rows' worth of channels that the masked
    // channels of the last row's items read past its end
    return align16(size_t(32) * exp_row_words<L>() * sizeof(T)) +
           kExpRBuf * align16((size_t(32) * RW + 3 * (L + 1)) * sizeof(T)) + align16(size_t(nr) * K * sizeof(T)) +
           align16(size_t(kExpBatch) * (sizeof(int64_t) + sizeof(int))) + 16;
}

// CSR offsets of kExpBatch consecutive centres [base, base + 32) of a warp's
// range, one centre per lane.
struct ExpBatch {
    int64_t base;
    int64_t lo, hi;  // this lane's centre owns the points [lo, hi)
    bool real;       // base + lane lies in the warp's centre range
    bool ok;         // real and 0 <= lo <= hi <= n_points
};

__device__ __forceinline__ ExpBatch load_batch(const int64_t* __restrict__ offsets, int64_t base, int64_t ce,
                                               int64_t npts, int lane) {
    ExpBatch bt{base, 0, 0, false, false};
    const int64_t ci = base + lane;
    if (ci < ce) {
        bt.real = true;
        bt.lo = offsets[ci];
        bt.hi = offsets[ci + 1];
        bt.ok = bt.lo >= 0 && bt.lo <= bt.hi && bt.hi <= npts;
    }
    return bt;
}

// Position in a batch: the first centre not yet written out, whether its sums
// so far are carried in shared memory, and the next point.
struct ExpCursor {
    int jc;
    bool carry;
    int64_t p;
};

// One chunk: up to 32 consecutive points [p, p + cnt) of a run of consecutive
// well-formed centres (their point ranges abut), and the centres [j, jm) of
// the batch that own them or end in them (empty centres included).
struct ExpChunk {
    int64_t p;
    int cnt;
    int j, jm;
    bool carry_in;  // centre j was started by an earlier chunk
    bool last_fin;  // centre jm - 1 ends in this chunk (else it continues)
    bool valid;     // false: no unfinished well-formed centre left in the batch
};

// Warp-uniform: the chunk that starts at cursor `cu` of batch `bt`.
__device__ __forceinline__ ExpChunk plan_chunk(const ExpBatch& bt, const ExpCursor& cu, int lane) {
    ExpChunk ch{0, 0, 0, 0, false, false, false};
    const unsigned vmask = __ballot_sync(0xffffffffu, bt.ok);
    const unsigned avail = cu.jc < 32 ? vmask & (0xffffffffu << cu.jc) : 0u;
    if (!avail) return ch;
    ch.valid = true;
    const int j = __ffs(avail) - 1;  // == cu.jc when carrying
    ch.j = j;
    ch.carry_in = cu.carry;
    const int64_t loj = __shfl_sync(0xffffffffu, bt.lo, j);
    ch.p = cu.carry ? cu.p : loj;
    // the run ends before the first malformed (or absent) centre after j
    const unsigned inv = ~vmask & (j < 31 ? (0xffffffffu << (j + 1)) : 0u);
    const int k = inv ? __ffs(inv) - 1 : 32;
    const int64_t run_hi = __shfl_sync(0xffffffffu, bt.hi, k - 1);
    ch.cnt = int(min(int64_t(32), run_hi - ch.p));
    const int64_t e = ch.p + ch.cnt;
    // members: the centres of the run up to the first one with points past e
    const unsigned nonmem = __ballot_sync(0xffffffffu, lane > j && lane < k && (bt.lo > e || (bt.lo == e && bt.hi > e)));
    ch.jm = nonmem ? __ffs(nonmem) - 1 : k;
    ch.last_fin = __shfl_sync(0xffffffffu, bt.hi, ch.jm - 1) <= e;
    return ch;
}

__device__ __forceinline__ ExpCursor after_chunk(const ExpChunk& ch) {
    return ch.last_fin ? ExpCursor{ch.jm, false, ch.p + ch.cnt} : ExpCursor{ch.jm - 1, true, ch.p + ch.cnt};
}

// Malformed centres of a batch: flag them and write zeros.
template <typename T>
__device__ __forceinline__ void zero_malformed(const ExpBatch& bt, T* __restrict__ c, int nout,
                                               uint32_t* __restrict__ status, int lane) {
    unsigned bad = __ballot_sync(0xffffffffu, bt.real && !bt.ok);
    if (bad && lane == 0) atomicOr(status, kStatusBadOffsets);
    while (bad) {
        const int m = __ffs(bad) - 1;
        bad &= bad - 1;
        T* ci = c + (bt.base + m) * nout;
        for (int o = lane; o < nout; o += 32) ci[o] = T(0);
    }
}

// Each warp owns a contiguous range of centres and streams their points in
// chunks of 32 that cross centre boundaries: a chunk's harmonics are computed
// one point per lane, and each lane accumulates its (column, channel) items
// over the chunk's segments, writing a centre's sums to global memory from
// registers when the centre ends. The coordinates of the next chunk and the
// offsets of the next 32 centres are loaded one step ahead; the next chunk's
// radial rows are prefetched into L2 during the current chunk and copied into
// the (single) shared-memory buffer once its contraction is done.
template <int L, bool NORM, typename T>
__global__ void __launch_bounds__(256) expansion_kernel(const T* __restrict__ xyz, const T* __restrict__ R,
                                                        const int64_t* __restrict__ offsets, int64_t ncent,
                                                        int64_t npts, int nr,
                                                        const __grid_constant__ PointTabs<L, T, false> tb,
                                                        T* __restrict__ c, uint32_t* __restrict__ status, int bulk) {
    constexpr int K = (L + 1) * (L + 1);
    constexpr int SY = exp_row_words<L>();
    constexpr int RL = L + 1;
    const int RW = nr * RL;  // radial row width ([n][l])
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    unsigned char* base = smem + size_t(warp) * expansion_warp_bytes<L, T>(nr);
    const size_t ybytes = align16(size_t(32) * SY * sizeof(T));
    const size_t rbytes = align16((size_t(32) * RW + 3 * RL) * sizeof(T));
    const size_t cbytes = align16(size_t(nr) * K * sizeof(T));
    T* Ys = reinterpret_cast<T*>(base);
    T* Rb0 = reinterpret_cast<T*>(base + ybytes);
    T* Rb1 = reinterpret_cast<T*>(base + ybytes + (kExpRBuf - 1) * rbytes);
    T* Cs = reinterpret_cast<T*>(base + ybytes + kExpRBuf * rbytes);
    int64_t* seg_cid = reinterpret_cast<int64_t*>(base + ybytes + kExpRBuf * rbytes + cbytes);
    int* seg_end = reinterpret_cast<int*>(seg_cid + kExpBatch);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + ybytes + kExpRBuf * rbytes + cbytes +
                                                align16(size_t(kExpBatch) * (sizeof(int64_t) + sizeof(int))));
    const int nout = nr * K;
    const int NG = (nr + 3) / 4;  // radial channel groups of 4
    int col_groups = 0;           // sum over l of ceil((2l+1)/4)
#pragma unroll
    for (int ll = 0; ll <= L; ++ll) col_groups += (2 * ll + 1 + 3) / 4;
    const int n_items = col_groups * NG;

    // the warp's centres [cb, ce)
    const int64_t G = int64_t(gridDim.x) * W;
    const int64_t g = int64_t(blockIdx.x) * W + warp;
    const int64_t cb = ncent * g / G, ce = ncent * (g + 1) / G;

    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    for (int t = lane; t < 32 * SY; t += 32) Ys[t] = T(0);  // padding slots stay zero
    fence_proxy_async_smem();
    __syncwarp();
    uint32_t phase = 0, pending = 0;
    bool failed = false;

    // Bulk copy of a chunk's radial rows into buffer b (when allowed).
    auto issue = [&](int b, const ExpChunk& ch) {
        if (!bulk || ch.cnt <= 0) return;
        const uint32_t bytes = uint32_t(size_t(ch.cnt) * RW * sizeof(T));
        if (lane == 0) {
            mbar_arrive_expect_tx(&bar[b], bytes);
            bulk_load(b ? Rb1 : Rb0, R + ch.p * RW, bytes, &bar[b]);
        }
        pending |= (1u << b);
    };
    auto coords = [&](const ExpChunk& ch, T& x, T& y, T& z) {
        if (lane < ch.cnt) {
            const int64_t p = ch.p + lane;
            x = xyz[3 * p];
            y = xyz[3 * p + 1];
            z = xyz[3 * p + 2];
        }
    };

    ExpBatch cur = load_batch(offsets, cb, ce, npts, lane);
    ExpBatch nxt = load_batch(offsets, cb + kExpBatch, ce, npts, lane);
    zero_malformed(cur, c, nout, status, lane);
    // the first chunk of the batch sequence from cursor cu (moving to later batches as needed)
    auto next_chunk = [&](ExpCursor cu) -> ExpChunk {
        ExpChunk ch = plan_chunk(cur, cu, lane);
        while (!ch.valid && cur.base + kExpBatch < ce) {
            cur = nxt;
            nxt = load_batch(offsets, cur.base + kExpBatch, ce, npts, lane);
            zero_malformed(cur, c, nout, status, lane);
            ch = plan_chunk(cur, ExpCursor{0, false, 0}, lane);
        }
        return ch;
    };

    ExpChunk ch = next_chunk(ExpCursor{0, false, 0});
    int b = 0;
    T px = T(0), py = T(0), pz = T(0);  // this lane's coordinates for the current chunk
    if (ch.valid) {
        issue(0, ch);
        coords(ch, px, py, pz);
    }
    while (ch.valid) {
        // segment table of this chunk (before `cur` may move to the next batch)
        if (lane >= ch.j && lane < ch.jm) {
            seg_end[lane - ch.j] = int(min(cur.hi, ch.p + ch.cnt) - ch.p);
            seg_cid[lane - ch.j] = cur.base + lane;
        }
        const int nseg = ch.jm - ch.j;
        const int cnt = ch.cnt;
        const bool carry_in = ch.carry_in, last_fin = ch.last_fin;
        const int64_t p0 = ch.p;
        // the next chunk: its radial rows and coordinates are loaded during this one
        const ExpChunk nch = next_chunk(after_chunk(ch));
        const int nb = kExpRBuf == 2 ? (b ^ 1) : 0;
        T nxx = T(0), nxy = T(0), nxz = T(0);
        if (nch.valid && !failed) {
            if constexpr (kExpRBuf == 2) {
                issue(nb, nch);
            } else if (bulk && lane == 0 && nch.cnt > 0) {
                bulk_prefetch_l2(R + nch.p * RW, uint32_t(size_t(nch.cnt) * RW * sizeof(T)));
            }
            coords(nch, nxx, nxy, nxz);
        }
        // harmonics of this chunk, one point per lane
        if (lane < cnt) {
            T x = px, y = py, z = pz, r2, ir = T(1);
            if (NORM) {
                unit_point(x, y, z, r2, ir);
            } else {
                r2 = x * x + y * y + z * z;
            }
            ValVis<T> vis{Ys + size_t(lane) * SY};
            point_core<L, false, false>(x, y, z, r2, tb, vis);
        }
        T* const Rs = b ? Rb1 : Rb0;
        if (pending & (1u << b)) {
            bool ok = true;
            if (lane == 0) ok = mbar_wait_bounded(&bar[b], (phase >> b) & 1u, kWaitPolls);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (ok) {
                phase ^= (1u << b);
                pending &= ~(1u << b);
            } else {
                if (lane == 0) atomicOr(status, kStatusLoadTimeout);
                failed = true;
                break;
            }
        } else if (!bulk) {
            const T* src = R + p0 * RW;
            for (int t = lane; t < cnt * RW; t += 32) Rs[t] = src[t];
        }
        __syncwarp();
        // Contraction, register-blocked: a work item is one group of 4 columns
        // of an l block x 4 radial channels (16 accumulators); items are
        // ordered by (l, column group, channel group) and dealt to lanes
        // round-robin, so a lane owns the same items in every chunk. A lane
        // reads its 4 columns and 4 channels at immediate offsets from one
        // pointer each: padding slots (zero) and channels past n_rad (the next
        // row, or the buffer's tail) feed accumulators masked at the writes.
        // With 2 or 4 channel groups, group g holds the channels g + NG q: the
        // words a round reads for one q are then NG (l_max+1) consecutive
        // ones, not NG runs 4 (l_max+1) apart that wrap around the banks.
        for (int it = lane; it < n_items; it += 32) {
            int l = 0, acc_items = 0;
            for (int ll = 0; ll <= L; ++ll) {  // decode the item
                const int cnt_l = ((2 * ll + 1 + 3) / 4) * NG;
                if (it < acc_items + cnt_l) {
                    l = ll;
                    break;
                }
                acc_items += cnt_l;
            }
            const int r = it - acc_items;
            const int cg = r / NG;
            const int ng = r - cg * NG;
            const bool strided = NG == 2 || NG == 4;
            const int nbase = strided ? ng : 4 * ng;  // channel of slot q: nbase + nstep q
            const int nstep = strided ? NG : 1;
            const int c0 = l * l + cg * 4;
            const int nc = min(4, 2 * l + 1 - cg * 4);
            bool qok[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) qok[q] = nbase + nstep * q < nr;
            const T* yp = Ys + exp_gbase(exp_gstart(l) + cg);
            const T* rp = Rs + nbase * RL + l;
            const int cbase = nbase * K + c0;  // [n][K] offset of the item's first output
            const int cstep = nstep * K;
            T acc[4][4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    acc[j][q] = (carry_in && j < nc && qok[q]) ? Cs[cbase + q * cstep + j] : T(0);
            // the segments of the chunk; S = channel stride of the item's slots
            auto segments = [&](auto s_tag) {
                constexpr int S = decltype(s_tag)::value;
                int s = 0;
                for (int si = 0; si < nseg; ++si) {
                    const int se = seg_end[si];
#pragma unroll 4
                    for (int e = s; e < se; ++e) {
                        const T* ye = yp + e * SY;
                        const T* re = rp + e * RW;
                        T yv[4], rv[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) yv[j] = ye[j];
#pragma unroll
                        for (int q = 0; q < 4; ++q) rv[q] = re[q * S * RL];
#pragma unroll
                        for (int j = 0; j < 4; ++j)
#pragma unroll
                            for (int q = 0; q < 4; ++q) acc[j][q] = fma(yv[j], rv[q], acc[j][q]);
                    }
                    s = se;
                    if (si + 1 < nseg || last_fin) {  // the centre ends here: write it out
                        T* ci = c + seg_cid[si] * nout + cbase;
#pragma unroll
                        for (int j = 0; j < 4; ++j)
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                if (j < nc && qok[q]) ci[q * cstep + j] = acc[j][q];
                                acc[j][q] = T(0);
                            }
                    }
                }
            };
            if (NG == 2) {
                segments(std::integral_constant<int, 2>{});
            } else if (NG == 4) {
                segments(std::integral_constant<int, 4>{});
            } else {
                segments(std::integral_constant<int, 1>{});
            }
            if (!last_fin) {  // carried into the next chunk
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (j < nc && qok[q]) Cs[cbase + q * cstep + j] = acc[j][q];
            }
        }
        fence_proxy_async_smem();  // generic reads of Rs done before the buffer is refilled
        __syncwarp();
        if (kExpRBuf == 1 && nch.valid && !failed) issue(0, nch);  // refill the one buffer
        ch = nch;
        b = nb;
        px = nxx;
        py = nxy;
        pz = nxz;
    }
    if (pending && lane == 0) {  // after a timeout: bounded wait for copies still in flight
        for (int q = 0; q < 2; ++q)
            if (pending & (1u << q)) (void)mbar_wait_bounded(&bar[q], (phase >> q) & 1u, kWaitPolls);
    }
    __syncwarp();
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

// Launches with up to a.warps warps per block, fewer when the per-warp staging
// does not fit the opt-in shared-memory limit; kExpTooBig when one warp's does not.
constexpr int kExpTooBig = -1;

template <int L, bool NORM, typename T>
int launch_expansion(const ExpArgs& a) {
    static const PointTabs<L, T, false> tb = make_point_tabs<L, T, false>();
    const size_t per_warp = expansion_warp_bytes<L, T>(a.nr);
    const size_t limit = size_t(max_smem_optin());
    if (per_warp > limit) return kExpTooBig;
    int W = a.warps;
    while (W > 1 && size_t(W) * per_warp > limit) --W;
    const size_t smem = size_t(W) * per_warp;
    auto kern = expansion_kernel<L, NORM, T>;
    cudaError_t err = ensure_smem(kern, smem);
    if (err != cudaSuccess) return int(err);
    const int grid = grid_for(kern, 32 * W, smem, a.ncent, 0);
    // Bulk copies of whole chunks need 16-byte aligned rows of the radial array.
    const bool bulk = (reinterpret_cast<uintptr_t>(a.radial) % 16 == 0) &&
                      ((size_t(a.nr) * (L + 1) * sizeof(T)) % 16 == 0);
    kern<<<grid, 32 * W, smem, static_cast<cudaStream_t>(a.stream)>>>(
        static_cast<const T*>(a.xyz), static_cast<const T*>(a.radial), a.offsets, a.ncent, a.npts, a.nr, tb,
        static_cast<T*>(a.c), a.status, bulk ? 1 : 0);
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
    const int err = launch_expansion_any(a);
    if (err == kExpTooBig) {
        set_error("expansion: n_rad=%d with l_max=%d needs more shared memory per warp than the device has", n_rad,
                  l_max);
        return SPH_EUNSUPPORTED;
    }
    if (err) {
        set_error("expansion launch: %s", cudaGetErrorString(static_cast<cudaError_t>(err)));
        return SPH_ECUDA;
    }
    return SPH_OK;
}
