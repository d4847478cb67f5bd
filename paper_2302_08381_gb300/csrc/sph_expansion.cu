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

template <typename T, int K>
struct ValVis {
    T* row;
    __device__ __forceinline__ void emit(int, int k, const Deriv<T>& d) { row[k] = d.v; }
};

// Per-warp shared memory: Y rows of a 32-point chunk (odd stride), two
// buffers of the chunk's radial rows in their global layout [e][n][l]
// (filled by bulk copies one chunk ahead), the [n_rad, K] accumulator of the
// current centre, and two mbarriers.
template <int L, typename T>
__host__ __device__ constexpr size_t expansion_warp_bytes(int nr) {
    constexpr int K = (L + 1) * (L + 1);
    constexpr int SY = (K % 2 == 0) ? K + 1 : K;
    const int RW = nr * (L + 1);
    return align16(size_t(32) * SY * sizeof(T)) + 2 * align16(size_t(32) * RW * sizeof(T)) +
           align16(size_t(nr) * K * sizeof(T)) + 16;
}

// The work of one warp is the sequence of (centre, 32-point chunk) items of
// the centres i = first, first + stride, ...; `next_item` advances along it.
struct ExpItem {
    int64_t i;   // centre (>= ncent: done)
    int64_t ch;  // first point of the chunk
    int64_t e1;  // end of the centre's points
    bool valid_centre;
};

__device__ __forceinline__ void first_chunk(ExpItem& it, const int64_t* __restrict__ offsets, int64_t ncent,
                                            int64_t npts, int64_t stride) {
    while (it.i < ncent) {
        const int64_t e0 = offsets[it.i], e1 = offsets[it.i + 1];
        it.valid_centre = !(e0 < 0 || e1 < e0 || e1 > npts);
        it.ch = e0;
        it.e1 = e1;
        return;  // empty and malformed centres are items too (they write their output)
    }
    (void)stride;
}

template <int L, bool NORM, typename T>
__global__ void __launch_bounds__(256) expansion_kernel(const T* __restrict__ xyz, const T* __restrict__ R,
                                                        const int64_t* __restrict__ offsets, int64_t ncent,
                                                        int64_t npts, int nr,
                                                        const __grid_constant__ PointTabs<L, T, false> tb,
                                                        T* __restrict__ c, uint32_t* __restrict__ status, int bulk) {
    constexpr int K = (L + 1) * (L + 1);
    constexpr int SY = (K % 2 == 0) ? K + 1 : K;
    constexpr int RL = L + 1;
    const int RW = nr * RL;  // radial row width ([n][l])
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    unsigned char* base = smem + size_t(warp) * expansion_warp_bytes<L, T>(nr);
    const size_t ybytes = align16(size_t(32) * SY * sizeof(T));
    const size_t rbytes = align16(size_t(32) * RW * sizeof(T));
    T* Ys = reinterpret_cast<T*>(base);
    T* Rb0 = reinterpret_cast<T*>(base + ybytes);
    T* Rb1 = reinterpret_cast<T*>(base + ybytes + rbytes);
    T* Cs = reinterpret_cast<T*>(base + ybytes + 2 * rbytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + ybytes + 2 * rbytes + align16(size_t(nr) * K * sizeof(T)));
    const int nout = nr * K;
    const int64_t stride = int64_t(gridDim.x) * W;
    const int NG = (nr + 3) / 4;  // radial channel groups of 4
    int col_groups = 0;           // sum over l of ceil((2l+1)/4)
#pragma unroll
    for (int ll = 0; ll <= L; ++ll) col_groups += (2 * ll + 1 + 3) / 4;
    const int n_items = col_groups * NG;

    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    fence_proxy_async_smem();
    __syncwarp();
    uint32_t phase = 0, pending = 0;
    bool failed = false;

    // Issues the radial rows of chunk (ch, cnt) into buffer b: bulk copy of
    // the whole rows when allowed, else nothing (loaded at use time).
    auto issue = [&](int b, int64_t ch, int cnt) -> int64_t {
        if (!bulk || cnt <= 0) return 0;
        const uint32_t bytes = uint32_t(size_t(cnt) * RW * sizeof(T));
        if (lane == 0) {
            mbar_arrive_expect_tx(&bar[b], bytes);
            bulk_load(b ? Rb1 : Rb0, R + ch * RW, bytes, &bar[b]);
        }
        pending |= (1u << b);
        return cnt;
    };

    ExpItem cur{int64_t(blockIdx.x) * W + warp, 0, 0, true};
    first_chunk(cur, offsets, ncent, npts, stride);
    int b = 0;
    if (cur.i < ncent && cur.valid_centre) issue(0, cur.ch, int(min(int64_t(32), cur.e1 - cur.ch)));
    T px = T(0), py = T(0), pz = T(0);  // this lane's coordinates for the current chunk
    if (cur.i < ncent && cur.valid_centre && cur.ch + lane < cur.e1) {
        const int64_t p = cur.ch + lane;
        px = xyz[3 * p];
        py = xyz[3 * p + 1];
        pz = xyz[3 * p + 2];
    }
    bool new_centre = true;
    while (cur.i < ncent) {
        T* ci = c + cur.i * nout;
        if (!cur.valid_centre) {  // malformed CSR: flag it, write zeros, move on
            if (lane == 0) atomicOr(status, kStatusBadOffsets);
            for (int o = lane; o < nout; o += 32) ci[o] = T(0);
            cur.i += stride;
            first_chunk(cur, offsets, ncent, npts, stride);
            if (cur.i < ncent && cur.valid_centre) {
                issue(b, cur.ch, int(min(int64_t(32), cur.e1 - cur.ch)));
                if (cur.ch + lane < cur.e1) {
                    const int64_t p = cur.ch + lane;
                    px = xyz[3 * p];
                    py = xyz[3 * p + 1];
                    pz = xyz[3 * p + 2];
                }
            }
            new_centre = true;
            continue;
        }
        if (new_centre) {
            for (int o = lane; o < nout; o += 32) Cs[o] = T(0);
            new_centre = false;
        }
        const int cnt = int(min(int64_t(32), cur.e1 - cur.ch));
        // the next item: the centre's next chunk, else the next centre's first
        ExpItem nx = cur;
        nx.ch = cur.ch + 32;
        bool nx_new_centre = false;
        if (nx.ch >= cur.e1) {
            nx.i = cur.i + stride;
            first_chunk(nx, offsets, ncent, npts, stride);
            nx_new_centre = true;
        }
        const int nb = b ^ 1;
        T nxx = T(0), nxy = T(0), nxz = T(0);
        if (nx.i < ncent && nx.valid_centre && !failed) {
            issue(nb, nx.ch, int(min(int64_t(32), nx.e1 - nx.ch)));
            if (nx.ch + lane < nx.e1) {
                const int64_t p = nx.ch + lane;
                nxx = xyz[3 * p];
                nxy = xyz[3 * p + 1];
                nxz = xyz[3 * p + 2];
            }
        }
        // harmonics of this chunk, one point per lane
        if (lane < cnt) {
            T x = px, y = py, z = pz, r2, ir = T(1);
            if (NORM) {
                unit_point(x, y, z, r2, ir);
            } else {
                r2 = x * x + y * y + z * z;
            }
            ValVis<T, K> vis{Ys + size_t(lane) * SY};
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
        } else {
            const T* src = R + cur.ch * RW;
            for (int t = lane; t < cnt * RW; t += 32) Rs[t] = src[t];
        }
        __syncwarp();
        // Contraction, register-blocked: a work item is up to 4 columns of one
        // l block x 4 radial channels (16 accumulators); items are ordered by
        // (l, column group, channel group) and dealt to lanes round-robin.
        // Out-of-range columns/channels of an item read a valid entry and are
        // masked at the write-back, so the inner loop has no predicates.
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
            const int n0 = (r - cg * NG) * 4;
            const int c0 = l * l + cg * 4;
            const int nc = min(4, 2 * l + 1 - cg * 4);
            int col[4], rof[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) col[j] = c0 + min(j, nc - 1);
#pragma unroll
            for (int q = 0; q < 4; ++q) rof[q] = min(n0 + q, nr - 1) * RL + l;
            T acc[4][4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[j][q] = Cs[min(n0 + q, nr - 1) * K + col[j]];
#pragma unroll 2
            for (int e = 0; e < cnt; ++e) {
                const T* ye = Ys + e * SY;
                const T* re = Rs + e * RW;
                T yv[4], rv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) yv[j] = ye[col[j]];
#pragma unroll
                for (int q = 0; q < 4; ++q) rv[q] = re[rof[q]];
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[j][q] += yv[j] * rv[q];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (j < nc && n0 + q < nr) Cs[(n0 + q) * K + col[j]] = acc[j][q];
        }
        fence_proxy_async_smem();  // generic reads of Rs done before the buffer is refilled
        __syncwarp();
        if (nx_new_centre) {  // centre finished: write it out
            for (int o = lane; o < nout; o += 32) ci[o] = Cs[o];
            __syncwarp();
            new_centre = true;
        }
        cur = nx;
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

template <int L, bool NORM, typename T>
int launch_expansion(const ExpArgs& a) {
    static const PointTabs<L, T, false> tb = make_point_tabs<L, T, false>();
    const int W = a.warps;
    const size_t smem = size_t(W) * expansion_warp_bytes<L, T>(a.nr);
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
    // Fit the per-warp staging (Y rows, R rows, accumulators) in the opt-in limit.
    const size_t K = size_t(l_max + 1) * (l_max + 1);
    const size_t per_warp = e * (32 * (K + 1) + 2 * 32 * size_t(n_rad) * (l_max + 1) + size_t(n_rad) * K) + 80;
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
