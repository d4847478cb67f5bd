// C-ABI entry points of libsphericart_gb300 (declared in
// include/sphericart_gb300.h): argument validation, kernel-family dispatch,
// launch-shape resolution, and the library-owned caches (device tables,
// device status word, tuned launch shapes).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "sph_internal.h"

namespace sph {

// ------------------------------------------------------------------ errors
namespace {
thread_local char g_err[512] = "";
}

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
const char* last_error_message() { return g_err; }

// --------------------------------------------------------- device caches
namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
int g_sms[kMaxDevices] = {0};
int g_smem[kMaxDevices] = {0};
void* g_tab32[kMaxDevices] = {nullptr};
void* g_tab64[kMaxDevices] = {nullptr};
uint32_t* g_status[kMaxDevices] = {nullptr};

int current_device() {
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess) return -1;
    return (d >= 0 && d < kMaxDevices) ? d : -1;
}
}  // namespace

int sm_count() {
    const int d = current_device();
    if (d < 0) return 1;
    if (g_sms[d] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
        g_sms[d] = std::max(v, 1);
    }
    return g_sms[d];
}

int max_smem_optin() {
    const int d = current_device();
    if (d < 0) return 48 * 1024;
    if (g_smem[d] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, d);
        g_smem[d] = std::max(v, 48 * 1024);
    }
    return g_smem[d];
}

namespace {

// Uploads kSliceTables values per (l, m) entry, produced by `pack`, as FP32 or
// FP64 into `slot` (once per device).
template <typename Pack>
const void* upload_packed(void*& slot, int dtype, Pack pack) {
    if (slot) return slot;
    const int tn = tri_size(SPH_MAX_L);
    const size_t elem = (dtype == SPH_F64) ? 8 : 4;
    std::vector<unsigned char> host(size_t(kSliceTables) * tn * elem);
    for (int l = 0; l <= SPH_MAX_L; ++l)
        for (int m = 0; m <= l; ++m) {
            const int i = tri(l, m);
            double v[kSliceTables];
            pack(l, m, i, v);
            for (int t = 0; t < kSliceTables; ++t) {
                const size_t o = size_t(i) * kSliceTables + t;
                if (dtype == SPH_F64)
                    reinterpret_cast<double*>(host.data())[o] = v[t];
                else
                    reinterpret_cast<float*>(host.data())[o] = static_cast<float>(v[t]);
            }
        }
    void* p = nullptr;
    if (cudaMalloc(&p, host.size()) != cudaSuccess) {
        set_error("cudaMalloc of %zu bytes for device tables failed", host.size());
        return nullptr;
    }
    if (cudaMemcpy(p, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(p);
        set_error("upload of device tables failed");
        return nullptr;
    }
    slot = p;
    return slot;
}

void* g_down32[kMaxDevices] = {nullptr};
void* g_down64[kMaxDevices] = {nullptr};

}  // namespace

const void* device_tables(int dtype) {
    const int d = current_device();
    if (d < 0) {
        set_error("no current CUDA device");
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    void*& slot = (dtype == SPH_F64) ? g_tab64[d] : g_tab32[d];
    const HostTables& h = host_tables();
    // Packed per-(l, m) entries of kSliceTables values, see sph_internal.h:
    //   [0] a (m <= l-2), d_l (m = l-1), 0 (m = l)   [1] b (m <= l-2), else 0
    //   [2] Qtilde_l^l on the diagonal, else 0        [3] e
    //   [4] f   [5] g2   [6] g3   [7] g4
    return upload_packed(slot, dtype, [&](int l, int m, int i, double* v) {
        v[0] = m <= l - 2 ? h.a[i] : (m == l - 1 ? h.d[i] : 0.0);
        v[1] = m <= l - 2 ? h.b[i] : 0.0;
        v[2] = m == l ? h.qll[i] : 0.0;
        v[3] = h.e[i];
        v[4] = h.fz[i];
        v[5] = h.g2[i];
        v[6] = h.g3[i];
        v[7] = h.g4[i];
    });
}

const void* device_tables_down(int dtype) {
    const int d = current_device();
    if (d < 0) {
        set_error("no current CUDA device");
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    void*& slot = (dtype == SPH_F64) ? g_down64[d] : g_down32[d];
    const HostTables& h = host_tables();
    //   [0] al  [1] be  [2] Qtilde_l^l on the diagonal, else 0  [3] e  [4] f  [5..7] 0
    return upload_packed(slot, dtype, [&](int l, int m, int i, double* v) {
        v[0] = h.al[i];
        v[1] = h.be[i];
        v[2] = m == l ? h.qll[i] : 0.0;
        v[3] = h.e[i];
        v[4] = h.fz[i];
        v[5] = v[6] = v[7] = 0.0;
    });
}

// Coefficient streams of the ROW kernels (FP32): entry (d * 8 + k) * 8 + j
// holds, for degree d and channel m = j + 8k (lane j, slot k), the float4
// {A, B, S, e} of the packed tables and, in a second array after the first,
// f; zero where m > d. At m = 0, e and f are given WITHOUT the 1/sqrt2 of the
// m = 0 column (the kernel applies it through c_0).
const void* device_row_tables() {
    const int d = current_device();
    if (d < 0) {
        set_error("no current CUDA device");
        return nullptr;
    }
    static void* slots[kMaxDevices] = {nullptr};
    std::lock_guard<std::mutex> lk(g_mu);
    if (slots[d]) return slots[d];
    const HostTables& h = host_tables();
    constexpr int kEntries = kRowLanes * kRowDegrees * kRowSlots;
    std::vector<float> host(size_t(kEntries) * 9, 0.f);
    float* a4 = host.data();
    float* f1 = host.data() + size_t(kEntries) * 4;
    float* g4 = host.data() + size_t(kEntries) * 5;  // {g2, g3, g4, 0} (the ROW Hessian kernel)
    for (int j = 0; j < kRowLanes; ++j)
        for (int l = 0; l < kRowDegrees; ++l)
            for (int k = 0; k < kRowSlots; ++k) {
                const int m = j + kRowLanes * k;
                if (m > l) continue;
                const int i = tri(l, m);
                const size_t o = (size_t(l) * kRowSlots + k) * kRowLanes + j;
                const double unfold = (m == 0) ? 1.0 / h.inv_sqrt2 : 1.0;
                a4[4 * o + 0] = float(m <= l - 2 ? h.a[i] : (m == l - 1 ? h.d[i] : 0.0));
                a4[4 * o + 1] = float(m <= l - 2 ? h.b[i] : 0.0);
                a4[4 * o + 2] = float(m == l ? h.qll[i] : 0.0);
                a4[4 * o + 3] = float(h.e[i] * unfold);
                f1[o] = float(h.fz[i] * unfold);
                g4[4 * o + 0] = float(h.g2[i] * unfold);
                g4[4 * o + 1] = float(h.g3[i] * unfold);
                g4[4 * o + 2] = float(h.g4[i] * unfold);
            }
    void* p = nullptr;
    if (cudaMalloc(&p, host.size() * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of the ROW tables failed");
        return nullptr;
    }
    if (cudaMemcpy(p, host.data(), host.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p);
        set_error("upload of the ROW tables failed");
        return nullptr;
    }
    slots[d] = p;
    return p;
}

uint32_t* device_status_word() {
    const int d = current_device();
    if (d < 0) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_status[d]) {
        void* p = nullptr;
        if (cudaMalloc(&p, sizeof(uint32_t)) != cudaSuccess) return nullptr;
        cudaMemset(p, 0, sizeof(uint32_t));
        cudaDeviceSynchronize();
        g_status[d] = static_cast<uint32_t*>(p);
    }
    return g_status[d];
}

// ------------------------------------------------------------ launch shape
namespace {

using TuneKey = std::tuple<int, int, int, int, int>;  // device, L, dtype, out, grad
std::map<TuneKey, sph_launch> g_tuned;

int elem_size(int dtype, int out) {
    if (dtype == SPH_F64) return 8;
    return out == SPH_OUT_BF16 ? 2 : 4;
}

int gcd_int(int a, int b) {
    while (b) {
        const int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Points per tile must keep every tile's first byte 16-byte aligned.
int tile_multiple(int L, int elem) {
    const int K = (L + 1) * (L + 1);
    return 16 / gcd_int((K * elem) % 16 == 0 ? 16 : (K * elem) % 16, 16);
}

sph_launch default_point_fwd(int L, int grad, int elem, int hess = 0) {
    const size_t row = point_row_bytes(L, grad, elem, hess);
    const int mult = tile_multiple(L, elem);
    if (elem == 8 && !hess) {
        // FP64 arithmetic is the bound (GB300's FP64 FMA rate is 1/73 of
        // FP32): fill as many lanes of each warp as a tile of <= 74 KB allows
        // (three one-warp blocks per SM), one warp per block, a grid of 16
        // blocks per SM in waves. Measured (autotuner, l_max 2..11, 10k and
        // 1M points): within 5 % of the tuned shapes; the earlier 48 KB tile
        // budget left 14 of 32 lanes idle at l_max 8 with gradients (-15 %).
        int P = 32;
        while (P > mult && size_t(P) * row > 74 * 1024) P -= mult;
        P = std::max(mult, P / mult * mult);
        return sph_launch{P, 1, 16, 0};
    }
    const size_t budget = 48 * 1024;
    int P = 32;
    while (P > mult && size_t(P) * row > budget) P -= mult;
    P = std::max(mult, P / mult * mult);
    const size_t tile = size_t(P) * row;
    // Measured on GB300 (l_max 3..8): ~4 tiles per CTA and a grid of 16 CTAs
    // per SM, scheduled in waves, beat a persistent one-wave grid by 10-15%;
    // heavier rows (l_max >= 12) prefer one persistent wave.
    if (tile <= budget && row * 32 <= 48 * 1024) {
        const int W = int(std::max<size_t>(1, std::min<size_t>(8, (166 * 1024) / std::max<size_t>(tile, 1))));
        return sph_launch{P, W, 16, 0};
    }
    int W = int(std::max<size_t>(1, std::min<size_t>(4, budget / std::max<size_t>(tile, 1))));
    return sph_launch{P, W, 0, 0};
}

// Shared-memory bytes per point of the 4-lanes-per-point POINT tile: a value
// row and 3 gradient rows of stride point4_stride.
size_t point4_row_bytes(int L, int elem) { return size_t(elem) * 4 * size_t(point4_stride(L, elem)); }

// Default shape of the 4-lanes-per-point tile: 8 points per warp (all 32
// lanes), point4_default_warps warps per block, a grid of 16 blocks per SM
// scheduled in waves (measured on GB300, 1M points, FP32 gradients).
sph_launch default_point4_fwd(int L, int elem) {
    (void)elem;
    return sph_launch{8, point4_default_warps(L), 16, 4};
}

// Shared-memory bytes per point of the 16-lanes-per-point Hessian tile (FP32):
// 13 rows of stride point4_stride.
size_t point16_row_bytes(int L) { return size_t(4) * 13 * size_t(point4_stride(L, 4)); }

// Default shape of the 16-lanes-per-point Hessian tile: 4 points per warp (two
// passes of two points), as many blocks as fit; 4-warp blocks while three of
// them fit on an SM (l_max <= 8), else one-warp blocks (measured on GB300:
// with larger tiles a 4-warp block leaves the SM at 4 resident warps).
sph_launch default_point16_fwd(int L) {
    const size_t tile = 4 * point16_row_bytes(L) + 64;
    const int W = 3 * 4 * tile <= size_t(max_smem_optin()) ? 4 : 1;
    return sph_launch{4, W, 0, 16};
}

// Shared-memory bytes per warp of the 10-lanes-per-point Hessian tile of P
// points (FP32): for odd K the three images with 4 floats of phase slack each,
// for even K 10 row slots of stride point4_stride per point.
size_t point10_tile_bytes(int L, int P) {
    const size_t K = size_t(L + 1) * (L + 1);
    if (K % 2 == 0) return 10 * size_t(P) * 4 * size_t(point4_stride(L, 4));
    auto part = [](size_t e) { return (e + 4 + 3) / 4 * 4 * 4; };
    return part(size_t(P) * K) + part(3 * size_t(P) * K) + part(9 * size_t(P) * K);
}

// Default shape of the 10-lanes-per-point Hessian tile (measured on GB300,
// 1M / 400k / 200k points): to l_max 8, 6 points per tile (two passes) in
// 2-warp blocks; above, 3 (one pass keeps more warps resident once the tile
// outgrows the register-bound 12 warps per SM), in one-warp blocks for even K
// (per-row copies) and for odd K (whole-image copies) in the largest block of
// 4 or 2 warps that keeps as many warps resident as one-warp blocks would
// (1.1x at l_max 10 and 12), else one warp.
sph_launch default_point10_fwd(int L) {
    if (L <= 8) return sph_launch{6, 2, 0, 10};
    int W = 1;
    if (((L + 1) * (L + 1)) % 2) {
        const size_t tile = point10_tile_bytes(L, 3), smem = size_t(max_smem_optin());
        const size_t best = std::min<size_t>(12, smem / tile);
        for (int w : {4, 2}) {
            if (w * (smem / (w * tile)) >= best) {
                W = w;
                break;
            }
        }
    }
    return sph_launch{3, W, 0, 10};
}

// Whether the POINT default runs FP32 Hessians on 10 lanes per point.
// Measured on GB300 (1M points to l_max 8, 400k / 200k above): faster than
// the one-lane tile and the 16-lane map for the scaled form from l_max 7
// (1.1x the 16-lane map at l_max 8, 2.3x at 11, 3.6x at 16) and for the
// normalized form from l_max 6 (1.2-1.6x); the one-lane tile is faster below;
// AUTO runs ROW from row_hess_min_auto.
bool point10_default(int L, int hess, int normalized, int dtype, int out) {
    if (!hess || dtype != SPH_F32 || out != SPH_OUT_SAME || L >= row_hess_min_auto(normalized)) return false;
    return L >= (normalized ? 6 : 7);
}

// Whether the POINT default (no shape given, none tuned) runs 4 lanes per
// point: FP32 arithmetic with gradients, no Hessians, l_max >= 10 (where the
// one-lane tile that fits shared memory leaves most lanes idle).
bool point4_default(int L, int grad, int elem, int hess, int hc) {
    return grad && !hess && !hc && elem != 8 && L >= kPoint4MinL;
}

sph_launch default_point_bwd(int L, int elem, int dbw) {
    const size_t K = size_t(L + 1) * (L + 1);
    const size_t V = (K % 2 == 0) ? K + 1 : K;
    const int mult = tile_multiple(L, elem);
    const size_t per_pt = V * elem * (dbw ? 3 : 2);
    const size_t budget = 48 * 1024;
    int P = 32;
    while (P > mult && size_t(P) * per_pt > budget) P -= mult;
    P = std::max(mult, P / mult * mult);
    const size_t tile = size_t(P) * per_pt;
    // Measured on GB300 (fused backward, l_max 6, 4.19M points): 2-warp CTAs
    // on a grid of 32 CTAs per SM scheduled in waves beat the persistent
    // one-wave grid by 11 % for small rows; the double backward is
    // insensitive to the shape.
    if (!dbw && tile <= 24 * 1024) return sph_launch{P, 2, 32, 0};
    int W = int(std::max<size_t>(1, std::min<size_t>(4, budget / std::max<size_t>(tile, 1))));
    return sph_launch{P, W, 0, 0};
}

// Validates / completes a POINT launch shape; returns false with a message.
bool resolve_point(sph_launch& s, const sph_launch& dflt, int L, int elem, size_t per_point_bytes) {
    // no shape at all: the whole default, including its grid size
    if (s.points_per_tile == 0 && s.warps_per_block == 0 && s.blocks_per_sm == 0) s.blocks_per_sm = dflt.blocks_per_sm;
    if (s.points_per_tile == 0) s.points_per_tile = dflt.points_per_tile;
    if (s.warps_per_block == 0) s.warps_per_block = dflt.warps_per_block;
    const int mult = tile_multiple(L, elem);
    if (s.points_per_tile < 1 || s.points_per_tile > 32 || s.points_per_tile % mult != 0) {
        set_error("points_per_tile=%d must be in [1,32] and a multiple of %d for l_max=%d", s.points_per_tile,
                  mult, L);
        return false;
    }
    if (s.warps_per_block < 1 || s.warps_per_block > 8) {
        set_error("warps_per_block=%d must be in [1,8]", s.warps_per_block);
        return false;
    }
    if (s.blocks_per_sm < 0 || s.blocks_per_sm > 32) {
        set_error("blocks_per_sm=%d must be in [0,32]", s.blocks_per_sm);
        return false;
    }
    const size_t smem = size_t(s.warps_per_block) * (size_t(s.points_per_tile) * per_point_bytes + 64);
    if (smem > size_t(max_smem_optin())) {
        set_error("launch shape needs %zu bytes of shared memory per block (limit %d)", smem, max_smem_optin());
        return false;
    }
    return true;
}

// Resolves the zero fields of a 10-lanes-per-point shape from the default and
// validates it (message set on failure).
bool resolve_point10(sph_launch& s, int L) {
    const sph_launch d = default_point10_fwd(L);
    if (s.points_per_tile == 0 && s.warps_per_block == 0 && s.blocks_per_sm == 0) s.blocks_per_sm = d.blocks_per_sm;
    if (s.points_per_tile == 0) s.points_per_tile = d.points_per_tile;
    if (s.warps_per_block == 0) s.warps_per_block = d.warps_per_block;
    if (s.points_per_tile < 3 || s.points_per_tile > 12 || s.points_per_tile % 3 || s.warps_per_block < 1 ||
        s.warps_per_block > 4 || s.blocks_per_sm < 0 || s.blocks_per_sm > 32) {
        set_error("POINT with 10 lanes per point: points_per_tile 3, 6, 9 or 12, warps_per_block <= 4");
        return false;
    }
    if (size_t(s.warps_per_block) * point10_tile_bytes(L, s.points_per_tile) > size_t(max_smem_optin())) {
        set_error("POINT with 10 lanes per point: the tile does not fit shared memory");
        return false;
    }
    return true;
}

// Resolves and validates a 16-lanes-per-point shape (message set on failure).
bool resolve_point16(sph_launch& s, int L) {
    if (!resolve_point(s, default_point16_fwd(L), L, 4, point16_row_bytes(L))) return false;
    if (s.points_per_tile > 8 || s.points_per_tile % 2 || s.warps_per_block > 4) {
        set_error("POINT with 16 lanes per point: points_per_tile even and <= 8, warps_per_block <= 4");
        return false;
    }
    return true;
}

}  // namespace

sph_launch point_fwd_shape(int L, int grad) {
    sph_launch s{0, 0, 0, 0};
    if (!tuned_launch(L, SPH_F32, SPH_OUT_SAME, grad, &s)) s = sph_launch{0, 0, 0, 0};
    const sph_launch d = default_point_fwd(L, grad, 4, 0);
    if (s.points_per_tile == 0) s.points_per_tile = d.points_per_tile;
    if (s.warps_per_block == 0) s.warps_per_block = d.warps_per_block;
    return s;
}

bool tuned_launch(int L, int dtype, int out, int grad, sph_launch* s) {
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_tuned.find(TuneKey{d, L, dtype, out, grad >= 2 ? 2 : (grad ? 1 : 0)});
    if (it == g_tuned.end()) return false;
    *s = it->second;
    return true;
}

namespace {

bool valid_lanes(const sph_launch& s) {
    if (s.lanes_per_point != 0 && s.lanes_per_point != 8 && s.lanes_per_point != 16 && s.lanes_per_point != 32) {
        set_error("lanes_per_point=%d must be 0, 8, 16 or 32", s.lanes_per_point);
        return false;
    }
    if (s.blocks_per_sm < 0 || s.blocks_per_sm > 32) {
        set_error("blocks_per_sm=%d must be in [0,32]", s.blocks_per_sm);
        return false;
    }
    return true;
}

bool aligned(const void* p, size_t a) { return reinterpret_cast<uintptr_t>(p) % a == 0; }

// Lanes per point of the upward DEGREE kernel when the caller leaves it 0
// (measured on GB300: FP64 prefers 1 lane per point below l_max 10, 2 up to
// l_max ~ 24 and 4 above, FP32 arithmetic with FP64 Q ("mixed") 2, FP32 /
// bf16 storage 4).
int degree_default_lpp(int l_max, int dtype, int qprec) {
    if (dtype == SPH_F64) return l_max >= 24 ? 4 : (l_max >= 10 ? 2 : 1);
    if (qprec == SPH_Q_F64) return 2;
    return 4;
}

}  // namespace

// FP64 (FP64-pipe bound): the hybrid with hard-coded l <= 3 runs fewer FP64
// instructions; measured 1.07-2.3x faster with gradients up to l_max 8 and
// 1.2-1.5x for values up to l_max 3, equal or slower beyond. In FP32 (bound
// by HBM writes) it makes no difference.
bool point_hybrid_wins(int l_max, int dtype, bool grad) {
    return dtype == SPH_F64 && (grad ? l_max <= kHcMaxL : l_max <= 3);
}

namespace {

// AUTO kernel family of a forward request (measured on GB300). POINT
// (compile-time l_max, TMA bulk stores) wins whenever it applies in FP32, and
// in FP64 up to l_max ~ 10; beyond that FP64 arithmetic (FP64 inputs or the
// mixed mode) is bound by GB300's FP64 pipe, where the DEGREE family (no idle
// lanes) is fastest; beyond POINT's range FP32 arithmetic runs on ROW up to
// its l_max 63 (1.8-2.2x SLICE; FP32 Hessians 1.2-1.7x), then on SLICE
// (DEGREE for bf16 storage).
int auto_family(int l_max, int dtype, int out, int qprec, bool hess, bool grad, int normalized) {
    const bool mixed = dtype == SPH_F32 && qprec == SPH_Q_F64;
    // FP64: DEGREE with gradients from l_max 9 (measured at 1M-4M points:
    // l_max 10 / 11 at 1.65x / 2.0x POINT), values from l_max 14 (POINT 8 %
    // faster at l_max 12, equal at 13; at 10k points POINT up to 16)
    if (!hess && (mixed || (dtype == SPH_F64 && (l_max >= 14 || (grad && l_max >= 9))))) return SPH_KERNEL_DEGREE;
    if (!hess && point_hybrid_wins(l_max, dtype, grad)) return SPH_KERNEL_POINT_HC;
    // FP32 Hessians: ROW from l_max 13 (normalized) or beyond POINT's range
    if (hess && dtype == SPH_F32 && out == SPH_OUT_SAME && l_max >= row_hess_min_auto(normalized) &&
        l_max <= kRowMaxL)
        return SPH_KERNEL_ROW;
    if (l_max <= SPH_MAX_L_POINT && !(hess && out == SPH_OUT_BF16)) return SPH_KERNEL_POINT;
    if (!hess && dtype == SPH_F32 && l_max <= kRowMaxL) return SPH_KERNEL_ROW;
    if (!hess && out == SPH_OUT_BF16) return SPH_KERNEL_DEGREE;
    return SPH_KERNEL_SLICE;
}

int cuda_status(int err, const char* what) {
    if (err == 0) return SPH_OK;
    set_error("%s: %s", what, cudaGetErrorString(static_cast<cudaError_t>(err)));
    return SPH_ECUDA;
}

// Common checks; returns SPH_OK or an error (message set).
int check_common(int64_t n, int l_max, int dtype, int kernel) {
    if (n < 0) {
        set_error("n=%lld must be >= 0", static_cast<long long>(n));
        return SPH_EINVAL;
    }
    if (l_max < 0 || l_max > SPH_MAX_L) {
        set_error("l_max=%d must be in [0,%d]", l_max, SPH_MAX_L);
        return SPH_EINVAL;
    }
    if (dtype != SPH_F32 && dtype != SPH_F64) {
        set_error("dtype=%d is not an sph_dtype", dtype);
        return SPH_EINVAL;
    }
    if (kernel != SPH_KERNEL_AUTO && kernel != SPH_KERNEL_POINT && kernel != SPH_KERNEL_SLICE &&
        kernel != SPH_KERNEL_DEGREE && kernel != SPH_KERNEL_DEGREE_DOWN && kernel != SPH_KERNEL_ROW &&
        kernel != SPH_KERNEL_POINT_HC) {
        set_error("kernel=%d is not an sph_kernel", kernel);
        return SPH_EINVAL;
    }
    return SPH_OK;
}

int ensure_device(const char* what) {
    int d = -1;
    const cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) {
        set_error("%s: no usable CUDA device (%s)", what, cudaGetErrorString(e));
        cudaGetLastError();
        return SPH_ECUDA;
    }
    return SPH_OK;
}

}  // namespace

}  // namespace sph

using namespace sph;

extern "C" {

int sphericart_version(void) { return 10000; }

const char* sphericart_last_error(void) { return last_error_message(); }

int sphericart_max_l(int dtype, int qprec, int kernel) {
    if (kernel == SPH_KERNEL_POINT) return (qprec == SPH_Q_F64 && dtype == SPH_F32) ? -1 : SPH_MAX_L_POINT;
    if (kernel == SPH_KERNEL_POINT_HC) return (qprec == SPH_Q_F64 && dtype == SPH_F32) ? -1 : kHcMaxL;
    if (kernel == SPH_KERNEL_ROW) return (dtype == SPH_F32 && qprec == SPH_Q_NATIVE) ? kRowMaxL : -1;
    (void)dtype;
    return SPH_MAX_L;
}

int sphericart_host_table(int l_max, int which, double* out) {
    if (!out || l_max < 0 || l_max > SPH_MAX_L || which < 0 || which > 8) {
        set_error("host_table: bad arguments (l_max=%d which=%d)", l_max, which);
        return SPH_EINVAL;
    }
    const HostTables& h = host_tables();
    const std::vector<double>* src[] = {&h.F, &h.qll, &h.a, &h.b, &h.e, &h.fz, &h.d, &h.al, &h.be};
    std::memcpy(out, src[which]->data(), sizeof(double) * size_t(tri_size(l_max)));
    return SPH_OK;
}

int sphericart_compute_ex(const void* xyz, int64_t n, int l_max, int normalized, int dtype, int out, int qprec,
                          int kernel, const sph_launch* launch, void* sph, void* dsph, void* ddsph,
                          void* stream) {
    int st = check_common(n, l_max, dtype, kernel);
    if (st) return st;
    if (out != SPH_OUT_SAME && out != SPH_OUT_BF16) {
        set_error("out=%d is not an sph_out", out);
        return SPH_EINVAL;
    }
    if (qprec != SPH_Q_NATIVE && qprec != SPH_Q_F64) {
        set_error("qprec=%d is not an sph_qprec", qprec);
        return SPH_EINVAL;
    }
    if (ddsph && !dsph) {
        set_error("ddsph requires dsph");
        return SPH_EINVAL;
    }
    if (dtype == SPH_F64 && out == SPH_OUT_BF16) {
        set_error("bfloat16 output is only available with FP32 arithmetic");
        return SPH_EUNSUPPORTED;
    }
    const bool mixed = (dtype == SPH_F32 && qprec == SPH_Q_F64);
    const int grad = dsph ? 1 : 0;
    int fam = kernel;
    const bool hess_bf16 = ddsph && out == SPH_OUT_BF16;
    if (fam == SPH_KERNEL_AUTO)
        fam = auto_family(l_max, dtype, out, qprec, ddsph != nullptr, dsph != nullptr, normalized);
    int hc = 0;
    if (fam == SPH_KERNEL_POINT_HC) {
        if (l_max > kHcMaxL || ddsph || mixed || out != SPH_OUT_SAME) {
            set_error("POINT_HC takes l_max <= %d, values and gradients, native Q precision and same-type storage",
                      kHcMaxL);
            return SPH_EUNSUPPORTED;
        }
        hc = 1;
        fam = SPH_KERNEL_POINT;
    }
    if (fam == SPH_KERNEL_POINT && (l_max > SPH_MAX_L_POINT || hess_bf16 || mixed)) {
        set_error("POINT kernels take l_max <= %d, native Q precision, and no bf16 Hessians", SPH_MAX_L_POINT);
        return SPH_EUNSUPPORTED;
    }
    if (fam == SPH_KERNEL_ROW && (mixed || dtype != SPH_F32 || l_max < (ddsph ? 0 : kRowMinL) ||
                                  l_max > kRowMaxL || (ddsph && out != SPH_OUT_SAME))) {
        set_error("ROW kernels take FP32 arithmetic, %d <= l_max <= %d (with Hessians 0 <= l_max <= %d, FP32 "
                  "storage)", kRowMinL, kRowMaxL, kRowMaxL);
        return SPH_EUNSUPPORTED;
    }
    const bool degree = fam == SPH_KERNEL_DEGREE || fam == SPH_KERNEL_DEGREE_DOWN;
    if (degree && ddsph) {
        set_error("DEGREE kernels compute values and gradients only (Hessians: POINT or SLICE)");
        return SPH_EUNSUPPORTED;
    }
    if (n == 0) return SPH_OK;
    if (!xyz || !sph) {
        set_error("xyz and sph must be non-NULL");
        return SPH_EINVAL;
    }
    const int ein = dtype == SPH_F64 ? 8 : 4;
    const int eo = elem_size(dtype, out);
    if (!aligned(xyz, ein) || !aligned(sph, eo) || (dsph && !aligned(dsph, eo)) || (ddsph && !aligned(ddsph, eo))) {
        set_error("buffers must be aligned to their element size");
        return SPH_EINVAL;
    }
    st = ensure_device("compute");
    if (st) return st;

    FwdArgs a{xyz, n, l_max, normalized ? 1 : 0, dtype, out, qprec, sph, dsph, ddsph, stream, sph_launch{0, 0, 0, 0},
              nullptr};
    if (launch) a.launch = *launch;
    a.hc = hc;
    if (fam == SPH_KERNEL_POINT) {
        bool from_default = !launch;
        if (!launch) {
            int d = -1;
            cudaGetDevice(&d);
            std::lock_guard<std::mutex> lk(g_mu);
            auto it = g_tuned.find(TuneKey{d, l_max, dtype, out, ddsph ? 2 : grad});
            if (it != g_tuned.end() && !(hc && it->second.lanes_per_point == 4)) {
                a.launch = it->second;
                from_default = false;
            }
        }
        const int hess = ddsph ? 1 : 0;
        if (from_default && a.launch.points_per_tile == 0 && a.launch.warps_per_block == 0 &&
            a.launch.blocks_per_sm == 0 && a.launch.lanes_per_point == 0) {
            if (point4_default(l_max, grad, eo, hess, hc))
                a.launch.lanes_per_point = 4;
            else if (point10_default(l_max, hess, normalized, dtype, out))
                a.launch.lanes_per_point = 10;
        }
        const int lpp = a.launch.lanes_per_point;
        if (lpp != 0 && lpp != 1 && lpp != 4 && lpp != 10 && lpp != 16) {
            set_error("POINT launch: lanes_per_point must be 0, 1, 4, 10 or 16");
            return SPH_EINVAL;
        }
        if (lpp == 10) {  // tiles of whole passes of three points, any start (no 16-byte tile multiple)
            if (!hess || dtype != SPH_F32 || out != SPH_OUT_SAME || hc) {
                set_error("POINT with 10 lanes per point takes FP32 arithmetic and storage with Hessians");
                return SPH_EUNSUPPORTED;
            }
            sph_launch& s = a.launch;
            if (!resolve_point10(s, l_max)) return SPH_EINVAL;
            if (from_default) {
                const int64_t tiles = (n + s.points_per_tile - 1) / s.points_per_tile;
                const int64_t per_w = std::max<int64_t>(1, tiles / (2 * int64_t(sm_count())));
                s.warps_per_block = int(std::min<int64_t>(s.warps_per_block, per_w));
            }
            return cuda_status(point_fwd_fn(l_max)(a), "POINT forward launch");
        }
        if (lpp == 4 && (!grad || hess || dtype != SPH_F32 || hc)) {
            set_error("POINT with 4 lanes per point takes FP32 arithmetic, values and gradients (no Hessians)");
            return SPH_EUNSUPPORTED;
        }
        if (lpp == 16 && (!hess || dtype != SPH_F32 || out != SPH_OUT_SAME || hc)) {
            set_error("POINT with 16 lanes per point takes FP32 arithmetic and storage with Hessians");
            return SPH_EUNSUPPORTED;
        }
        if (lpp == 16) {
            if (!resolve_point16(a.launch, l_max)) return SPH_EINVAL;
        } else {
            const sph_launch dflt = lpp == 4 ? default_point4_fwd(l_max, eo) : default_point_fwd(l_max, grad, eo, hess);
            const size_t row = lpp == 4 ? point4_row_bytes(l_max, eo) : point_row_bytes(l_max, grad, eo, hess);
            if (!resolve_point(a.launch, dflt, l_max, eo, row)) return SPH_EINVAL;
            if (lpp == 4 && a.launch.points_per_tile > 8) {
                set_error("POINT with 4 lanes per point: points_per_tile must be <= 8 (32 lanes per warp)");
                return SPH_EINVAL;
            }
        }
        if (from_default) {
            // Few tiles (small n): fewer warps per block, so that the blocks
            // spread over every SM instead of filling a few (measured at 10k
            // points: the tuned shapes use one warp per block, 1.3-1.6x faster
            // than eight).
            const int64_t tiles = (n + a.launch.points_per_tile - 1) / a.launch.points_per_tile;
            const int64_t per_w = std::max<int64_t>(1, tiles / (2 * int64_t(sm_count())));
            a.launch.warps_per_block = int(std::min<int64_t>(a.launch.warps_per_block, per_w));
        }
        return cuda_status(point_fwd_fn(l_max)(a), "POINT forward launch");
    }
    if (degree) {
        if (a.launch.warps_per_block < 0 || a.launch.warps_per_block > 8 || a.launch.blocks_per_sm < 0 ||
            a.launch.blocks_per_sm > 32) {
            set_error("DEGREE launch: warps_per_block must be in [0,8] and blocks_per_sm in [0,32]");
            return SPH_EINVAL;
        }
        const int lpp = a.launch.lanes_per_point;
        if (lpp != 0 && lpp != 1 && lpp != 2 && lpp != 4) {
            set_error("DEGREE launch: lanes_per_point must be 0, 1, 2 or 4");
            return SPH_EINVAL;
        }
        if (fam == SPH_KERNEL_DEGREE_DOWN && lpp > 1) {
            set_error("DEGREE_DOWN runs one lane per point (the downward recursion is sequential in m)");
            return SPH_EINVAL;
        }
        int e;
        if (fam == SPH_KERNEL_DEGREE_DOWN)
            e = degree_fwd_down(a);
        else if (lpp == 1)
            e = degree_fwd_up1(a);
        else if (lpp == 4)
            e = degree_fwd_up4(a);
        else if (lpp == 2)
            e = degree_fwd_up2(a);
        else
            e = degree_default_lpp(l_max, dtype, qprec) == 1 ? degree_fwd_up1(a)
                : degree_default_lpp(l_max, dtype, qprec) == 4 ? degree_fwd_up4(a) : degree_fwd_up2(a);
        if (e == int(cudaErrorInvalidConfiguration)) {
            set_error("DEGREE launch shape needs more shared memory per block than the device allows");
            return SPH_EINVAL;
        }
        return cuda_status(e, "DEGREE forward launch");
    }
    if (fam == SPH_KERNEL_ROW) {
        if (a.launch.warps_per_block < 0 || a.launch.warps_per_block > 8 || a.launch.blocks_per_sm < 0 ||
            a.launch.blocks_per_sm > 32) {
            set_error("ROW launch: warps_per_block must be in [0,8] and blocks_per_sm in [0,32]");
            return SPH_EINVAL;
        }
        if (a.launch.lanes_per_point < 0 || a.launch.lanes_per_point > (ddsph ? 3 : 2)) {
            set_error("ROW launch: lanes_per_point selects the window policy: 0 (by l_max), 1 or 2 (Hessians: 0..3)");
            return SPH_EINVAL;
        }
        const int e = ddsph ? row_hess_fwd(a) : ((l_max + 1 + 7) / 8 <= 5 ? row_fwd_part0(a) : row_fwd_part1(a));
        if (e == int(cudaErrorInvalidConfiguration)) {
            set_error("ROW forward launch shape: at most 2 warps per block, within the device's shared memory");
            return SPH_EINVAL;
        }
        return cuda_status(e, ddsph ? "ROW Hessian forward launch" : "ROW forward launch");
    }
    if (!valid_lanes(a.launch)) return SPH_EINVAL;
    return cuda_status(slice_fwd(a), "SLICE forward launch");
}

int sphericart_compute(const float* xyz, int64_t n, int l_max, int normalized, float* sph, float* dsph,
                       float* ddsph, void* stream) {
    return sphericart_compute_ex(xyz, n, l_max, normalized, SPH_F32, SPH_OUT_SAME, SPH_Q_NATIVE, SPH_KERNEL_AUTO,
                                 nullptr, sph, dsph, ddsph, stream);
}

static int backward_common(const void* xyz, const void* g, const void* v, int64_t n, int l_max, int normalized,
                           int dtype, int kernel, const sph_launch* launch, void* dxyz, void* grad_g,
                           void* grad_xyz, void* stream, bool dbw) {
    int st = check_common(n, l_max, dtype, kernel);
    if (st) return st;
    // AUTO: POINT within its l_max range; beyond it the fused backward in FP32
    // runs on ROW (up to its l_max), everything else on SLICE.
    int fam = kernel;
    if (fam == SPH_KERNEL_AUTO) {
        if (l_max <= SPH_MAX_L_POINT)
            fam = SPH_KERNEL_POINT;
        else if (!dbw && dtype == SPH_F32 && l_max <= kRowMaxL)
            fam = SPH_KERNEL_ROW;
        else
            fam = SPH_KERNEL_SLICE;
    }
    if (fam == SPH_KERNEL_POINT && l_max > SPH_MAX_L_POINT) {
        set_error("POINT kernels take l_max <= %d", SPH_MAX_L_POINT);
        return SPH_EUNSUPPORTED;
    }
    if (fam == SPH_KERNEL_DEGREE || fam == SPH_KERNEL_DEGREE_DOWN || fam == SPH_KERNEL_POINT_HC) {
        set_error("backward passes run on the POINT, ROW (backward) or SLICE kernels");
        return SPH_EUNSUPPORTED;
    }
    if (fam == SPH_KERNEL_ROW && (dbw || dtype != SPH_F32 || l_max < kRowMinL || l_max > kRowMaxL)) {
        set_error("the ROW backward takes FP32, %d <= l_max <= %d (double backward: POINT or SLICE)", kRowMinL,
                  kRowMaxL);
        return SPH_EUNSUPPORTED;
    }
    if (n == 0) return SPH_OK;
    if (!xyz || !g || (dbw && !v) || (!dbw && !dxyz)) {
        set_error("xyz, g%s must be non-NULL", dbw ? ", v" : ", dxyz");
        return SPH_EINVAL;
    }
    if (dbw && !grad_g && !grad_xyz) return SPH_OK;
    const int e = dtype == SPH_F64 ? 8 : 4;
    if (!aligned(xyz, e) || !aligned(g, e) || (v && !aligned(v, e)) || (dxyz && !aligned(dxyz, e)) ||
        (grad_g && !aligned(grad_g, e)) || (grad_xyz && !aligned(grad_xyz, e))) {
        set_error("buffers must be aligned to their element size");
        return SPH_EINVAL;
    }
    st = ensure_device(dbw ? "double_backward" : "backward");
    if (st) return st;
    BwdArgs a{xyz, g, v, n, l_max, normalized ? 1 : 0, dtype, dxyz, grad_g, grad_xyz, stream,
              sph_launch{0, 0, 0, 0}, nullptr};
    if (launch) a.launch = *launch;
    if (fam == SPH_KERNEL_POINT) {
        a.status = device_status_word();
        if (!a.status) {
            set_error("could not allocate the device status word");
            return SPH_ENOMEM;
        }
        const size_t K = size_t(l_max + 1) * (l_max + 1);
        const size_t V = (K % 2 == 0) ? K + 1 : K;  // padded smem rows for even K
        if (!resolve_point(a.launch, default_point_bwd(l_max, e, dbw), l_max, e, V * e * (dbw ? 3 : 2)))
            return SPH_EINVAL;
        PointBwdFn fn = dbw ? point_dbwd_fn(l_max) : point_bwd_fn(l_max);
        return cuda_status(fn(a), dbw ? "POINT double-backward launch" : "POINT backward launch");
    }
    if (fam == SPH_KERNEL_ROW) {
        if (a.launch.warps_per_block < 0 || a.launch.warps_per_block > 8 || a.launch.blocks_per_sm < 0 ||
            a.launch.blocks_per_sm > 32) {
            set_error("ROW launch: warps_per_block must be in [0,8] and blocks_per_sm in [0,32]");
            return SPH_EINVAL;
        }
        a.status = device_status_word();
        if (!a.status) {
            set_error("could not allocate the device status word");
            return SPH_ENOMEM;
        }
        const int e2 = (l_max + 1 + 7) / 8 <= 5 ? row_bwd_part0(a) : row_bwd_part1(a);
        if (e2 == int(cudaErrorInvalidConfiguration)) {
            set_error("ROW launch shape needs more shared memory per block than the device allows");
            return SPH_EINVAL;
        }
        return cuda_status(e2, "ROW backward launch");
    }
    if (!valid_lanes(a.launch)) return SPH_EINVAL;
    return cuda_status(dbw ? slice_dbwd(a) : slice_bwd(a), dbw ? "SLICE double-backward launch" : "SLICE backward launch");
}

int sphericart_backward(const void* xyz, const void* g, int64_t n, int l_max, int normalized, int dtype, int kernel,
                        const sph_launch* launch, void* dxyz, void* stream) {
    return backward_common(xyz, g, nullptr, n, l_max, normalized, dtype, kernel, launch, dxyz, nullptr, nullptr,
                           stream, false);
}

int sphericart_double_backward(const void* xyz, const void* g, const void* v, int64_t n, int l_max, int normalized,
                               int dtype, int kernel, const sph_launch* launch, void* grad_g, void* grad_xyz,
                               void* stream) {
    return backward_common(xyz, g, v, n, l_max, normalized, dtype, kernel, launch, nullptr, grad_g, grad_xyz, stream,
                           true);
}

int sphericart_device_status(uint32_t* status) {
    if (!status) {
        set_error("status must be non-NULL");
        return SPH_EINVAL;
    }
    int st = ensure_device("device_status");
    if (st) return st;
    uint32_t* w = device_status_word();
    if (!w) {
        set_error("could not allocate the device status word");
        return SPH_ENOMEM;
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(status, w, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(w, 0, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return cuda_status(int(e), "device_status");
}

int sphericart_launch_info(int l_max, int dtype, int out, int grad, int hess, int* kernel_out,
                           sph_launch* launch_out) {
    if (!kernel_out || !launch_out || l_max < 0 || l_max > SPH_MAX_L || (dtype != SPH_F32 && dtype != SPH_F64) ||
        (out != SPH_OUT_SAME && out != SPH_OUT_BF16)) {
        set_error("launch_info: bad arguments");
        return SPH_EINVAL;
    }
    const int eo = elem_size(dtype, out);
    int fam = auto_family(l_max, dtype, out, SPH_Q_NATIVE, hess != 0, grad != 0, 0);  // (the scaled form's choice)
    const bool hc = fam == SPH_KERNEL_POINT_HC;
    if (hc) fam = SPH_KERNEL_POINT;  // same launch shapes
    if (fam == SPH_KERNEL_DEGREE) {
        *kernel_out = SPH_KERNEL_DEGREE;
        *launch_out = sph_launch{0, 0, 0, degree_default_lpp(l_max, dtype, SPH_Q_NATIVE)};
    } else if (fam == SPH_KERNEL_ROW) {
        *kernel_out = SPH_KERNEL_ROW;
        *launch_out = sph_launch{0, 1, 0, 8};
    } else if (fam == SPH_KERNEL_POINT) {
        *kernel_out = hc ? SPH_KERNEL_POINT_HC : SPH_KERNEL_POINT;
        sph_launch s{0, 0, 0, 0};
        int d = -1;
        if (cudaGetDevice(&d) != cudaSuccess) {
            cudaGetLastError();
            d = -1;
        }
        {
            std::lock_guard<std::mutex> lk(g_mu);
            auto it = g_tuned.find(TuneKey{d, l_max, dtype, out, hess ? 2 : (grad ? 1 : 0)});
            if (it != g_tuned.end()) s = it->second;
        }
        const bool none = s.points_per_tile == 0 && s.warps_per_block == 0 && s.blocks_per_sm == 0 &&
                          s.lanes_per_point == 0;
        const bool four = s.lanes_per_point == 4 || (none && point4_default(l_max, grad, eo, hess, hc ? 1 : 0));
        // (the scaled form's choice: launch_info takes no normalized flag)
        const bool ten = s.lanes_per_point == 10 || (none && !four && point10_default(l_max, hess, 0, dtype, out));
        const bool sixteen = s.lanes_per_point == 16;
        const sph_launch dflt = four      ? default_point4_fwd(l_max, eo)
                                : ten     ? default_point10_fwd(l_max)
                                : sixteen ? default_point16_fwd(l_max)
                                          : default_point_fwd(l_max, grad ? 1 : 0, eo, hess ? 1 : 0);
        if (four) s.lanes_per_point = 4;
        if (ten) s.lanes_per_point = 10;
        // as resolve_point: no tuned shape at all takes the whole default
        if (s.points_per_tile == 0 && s.warps_per_block == 0 && s.blocks_per_sm == 0) s.blocks_per_sm = dflt.blocks_per_sm;
        if (s.points_per_tile == 0) s.points_per_tile = dflt.points_per_tile;
        if (s.warps_per_block == 0) s.warps_per_block = dflt.warps_per_block;
        *launch_out = s;
    } else {
        *kernel_out = SPH_KERNEL_SLICE;
        *launch_out = sph_launch{0, 0, 0, l_max + 1 <= 8 ? 8 : (l_max + 1 <= 16 ? 16 : 32)};
    }
    return SPH_OK;
}

int sphericart_set_launch(int l_max, int dtype, int out, int grad, const sph_launch* launch) {
    if (!launch || l_max < 0 || l_max > SPH_MAX_L_POINT || (dtype != SPH_F32 && dtype != SPH_F64) ||
        (out != SPH_OUT_SAME && out != SPH_OUT_BF16)) {
        set_error("set_launch: bad arguments");
        return SPH_EINVAL;
    }
    int st = ensure_device("set_launch");
    if (st) return st;
    const int eo = elem_size(dtype, out);
    const int g = grad >= 2 ? 2 : (grad ? 1 : 0);  // 2: values + gradients + Hessians
    sph_launch s = *launch;
    if (s.lanes_per_point != 0 && s.lanes_per_point != 1 && s.lanes_per_point != 4 && s.lanes_per_point != 10 &&
        s.lanes_per_point != 16) {
        set_error("set_launch: POINT lanes_per_point must be 0, 1, 4, 10 or 16");
        return SPH_EINVAL;
    }
    if (s.lanes_per_point == 10 || s.lanes_per_point == 16) {
        if (g != 2 || dtype != SPH_F32 || out != SPH_OUT_SAME) {
            set_error("set_launch: 10 or 16 lanes per point take FP32 arithmetic and storage with Hessians");
            return SPH_EINVAL;
        }
        if (!(s.lanes_per_point == 10 ? resolve_point10(s, l_max) : resolve_point16(s, l_max))) return SPH_EINVAL;
    } else if (s.lanes_per_point == 4) {
        if (g != 1 || dtype != SPH_F32) {
            set_error("set_launch: 4 lanes per point take FP32 arithmetic, values and gradients");
            return SPH_EINVAL;
        }
        if (!resolve_point(s, default_point4_fwd(l_max, eo), l_max, eo, point4_row_bytes(l_max, eo)))
            return SPH_EINVAL;
        if (s.points_per_tile > 8) {
            set_error("set_launch: 4 lanes per point take points_per_tile <= 8");
            return SPH_EINVAL;
        }
    } else if (!resolve_point(s, default_point_fwd(l_max, g ? 1 : 0, eo, g == 2), l_max, eo,
                              point_row_bytes(l_max, g ? 1 : 0, eo, g == 2))) {
        return SPH_EINVAL;
    }
    int d = -1;
    cudaGetDevice(&d);
    std::lock_guard<std::mutex> lk(g_mu);
    g_tuned[TuneKey{d, l_max, dtype, out, g}] = s;
    return SPH_OK;
}

int sphericart_tune_clear(void) {
    int st = ensure_device("tune_clear");
    if (st) return st;
    int d = -1;
    cudaGetDevice(&d);
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_tuned.begin(); it != g_tuned.end();) {
        if (std::get<0>(it->first) == d)
            it = g_tuned.erase(it);
        else
            ++it;
    }
    return SPH_OK;
}

}  // extern "C"
