// Internal host-side declarations shared by the translation units of the
// library. Not part of the public C-ABI (see include/sphericart_gb300.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "sphericart_gb300.h"

#ifdef __CUDACC__
#define SPH_HD __host__ __device__
#else
#define SPH_HD
#endif

namespace sph {

// Triangular index of (l, m), 0 <= m <= l.
SPH_HD inline constexpr int tri(int l, int m) { return l * (l + 1) / 2 + m; }
SPH_HD inline constexpr int tri_size(int L) { return (L + 1) * (L + 2) / 2; }

// Host FP64 tables for 0 <= l <= SPH_MAX_L (arXiv 2302.08381, Eq. Flm via the
// Appendix C iteration; the folded recursion coefficients of Appendix C; the
// derivative multipliers of Eq. iter-deri). All in triangular layout.
struct HostTables {
    int lmax = 0;
    std::vector<double> F;    // F_l^m
    std::vector<double> qll;  // Qtilde_l^l on (l,l), zero elsewhere
    std::vector<double> d;    // (2l-1) F_l^{l-1}/F_{l-1}^{l-1} on (l,l-1)
    std::vector<double> a;    // (2l-1)/(l-m) F_l^m/F_{l-1}^m       m <= l-2
    std::vector<double> b;    // (l+m-1)/(l-m) F_l^m/F_{l-2}^m      m <= l-2
    std::vector<double> e;    // F_l^m/F_{l-1}^{m+1}                m <= l-2  (x 1/sqrt2 at m=0)
    std::vector<double> fz;   // (l+m) F_l^m/F_{l-1}^m              m <= l-1  (x 1/sqrt2 at m=0)
    std::vector<double> g2;   // F_l^m/F_{l-2}^{m+2}                m <= l-4  (x 1/sqrt2 at m=0)
    std::vector<double> g3;   // (l+m) F_l^m/F_{l-2}^{m+1}          m <= l-3  (x 1/sqrt2 at m=0)
    std::vector<double> g4;   // (l+m)(l+m-1) F_l^m/F_{l-2}^m       m <= l-2  (x 1/sqrt2 at m=0)
    // Downward-in-m recursion (Eq. iter-q-alt with its sign corrected, folded):
    //   Qtilde_l^m = al z Qtilde_l^{m+1} - be (x^2+y^2) Qtilde_l^{m+2}
    std::vector<double> al;   // -2(m+1)/((l+m+1)(l-m)) F_l^m/F_l^{m+1}   m <= l-1
    std::vector<double> be;   // F_l^m/F_l^{m+2} / ((l+m+1)(l-m))        m <= l-2
    double inv_sqrt2 = 0.0;   // the 1/sqrt2 of the m = 0 column (Eq. real-sh-cartesian)
};

const HostTables& host_tables();

// Values per (l, m) entry of the packed SLICE tables (entry-major, two
// 4-vectors per entry): {A, B, S, e} and {f, g2, g3, g4}, where the Q
// recursion of channel m reads Qtilde_l^m = A z Qtilde_{l-1}^m
// - B r^2 Qtilde_{l-2}^m + S with A = a, B = b for m <= l-2, A = d_l, B = 0
// for m = l-1, and S = Qtilde_l^l, A = B = 0 on the diagonal.
constexpr int kSliceTables = 8;

// Device copy of the packed tables for the current device, FP32 or FP64.
// Returns nullptr and sets the error message on failure.
const void* device_tables(int dtype);

// Packed tables of the downward-in-m recursion for the DEGREE kernels
// (entry-major, two 4-vectors per (l, m)): {al, be, S, e} and {f, 0, 0, 0},
// S = Qtilde_l^l on the diagonal.
const void* device_tables_down(int dtype);

// Coefficient streams of the ROW kernels, FP32 (see sph_capi.cu): entry
// (degree, slot, lane), lane fastest, kRowDegrees x kRowSlots x kRowLanes
// float4 entries {A, B, S, e}, then as many floats f, then as many float4
// {g2, g3, g4, 0} (the second-derivative multipliers of the Hessian kernel).
constexpr int kRowLanes = 8;
constexpr int kRowDegrees = 64;
constexpr int kRowSlots = 8;
const void* device_row_tables();

// Per-device status word written by kernels whose bounded waits time out.
uint32_t* device_status_word();

// Thread-local error message.
void set_error(const char* fmt, ...);
const char* last_error_message();

int sm_count();            // of the current device
int max_smem_optin();      // bytes of opt-in dynamic shared memory per block

// ----------------------------------------------------------------- launches
struct FwdArgs {
    const void* xyz;
    int64_t n;
    int l_max;
    int normalized;
    int dtype;
    int out;
    int qprec;
    void* sph;
    void* dsph;
    void* ddsph;
    void* stream;
    sph_launch launch;   // resolved launch shape
    uint32_t* status;
    int hc = 0;          // POINT: hard-coded degrees l <= 3, then the recursion (l_max <= kHcMaxL)
};

// Smallest l_max at which FP32 gradient tiles run 4 lanes per point (one per
// output plane) by default, in single-set launches and in ragged batches.
constexpr int kPoint4MinL = 10;

// Shared-memory row stride (elements) of the 4-lanes-per-point POINT tile
// and how the tile leaves shared memory:
//   odd K: stride K, the image of the global range, one bulk copy per array;
//   even K with 16-byte rows (K * elem % 16 == 0): a stride of an odd number
//     of 16-byte units (K itself when K * elem / 16 is odd: again the image
//     of the global range), so that 32 lanes writing one column hit 8 banks
//     and every row can leave by its own bulk copy;
//   otherwise: stride K + 1 (conflict-free), copied out by the warp.
SPH_HD constexpr int point4_stride(int L, int elem) {
    const int K = (L + 1) * (L + 1);
    if (K % 2) return K;
    if ((K * elem) % 16) return K + 1;
    return ((K * elem / 16) % 2) ? K : K + 16 / elem;
}
// Staged bytes of a 4-lanes-per-point tile of P points (value rows, then
// gradient rows, each part rounded up to `align` bytes).
inline size_t point4_tile_bytes(int L, int elem, int P, size_t align) {
    const size_t S = size_t(point4_stride(L, elem)) * size_t(elem);
    const size_t v = (size_t(P) * S + align - 1) / align * align;
    const size_t d = (size_t(3 * P) * S + align - 1) / align * align;
    return v + d;
}

// 0: whole-tile bulk copies, 1: one bulk copy per row, 2: warp copy-out.
SPH_HD constexpr int point4_out_mode(int L, int elem) {
    const int K = (L + 1) * (L + 1);
    return point4_stride(L, elem) == K ? 0 : ((K * elem) % 16 ? 2 : 1);
}
// Warps per block of the default 4-lanes-per-point shape (measured on GB300,
// 1M points, FP32, l_max 10..16, grid of 16 blocks per SM in waves): 4, and
// 2 where every row leaves by its own bulk copy.
inline int point4_default_warps(int L) { return point4_out_mode(L, 4) == 1 ? 2 : 4; }

// Largest l_max with the hybrid POINT forward (hard-coded l <= 3) compiled.
constexpr int kHcMaxL = 8;

// Whether AUTO runs the hybrid instead of the all-recursion POINT forward
// (values, or values and gradients; no Hessians).
bool point_hybrid_wins(int l_max, int dtype, bool grad);

struct BwdArgs {
    const void* xyz;
    const void* g;
    const void* v;
    int64_t n;
    int l_max;
    int normalized;
    int dtype;
    void* dxyz;      // backward output
    void* grad_g;    // double backward outputs
    void* grad_xyz;
    void* stream;
    sph_launch launch;
    uint32_t* status;
};

// POINT kernels, one translation unit per compile-time l_max.
// Each returns a cudaError_t value as int (0 = success).
using PointFwdFn = int (*)(const FwdArgs&);
using PointBwdFn = int (*)(const BwdArgs&);
PointFwdFn point_fwd_fn(int L);
PointBwdFn point_bwd_fn(int L);
PointBwdFn point_dbwd_fn(int L);

// Ragged-batch kernel of one compile-time l_max (one object file per l_max).
struct BatchClassArgs;
using BatchClassFn = int (*)(const BatchClassArgs&);
BatchClassFn batch_class_fn(int L);

// One-launch ragged-batch kernel from device descriptors, one object file
// per flag class gn = gradients + 2 * normalized.
struct OneArgs;
using BatchOneFn = int (*)(const OneArgs&);
BatchOneFn batch_one_fn(int gn);

// Tuned POINT forward shape installed for (l_max, dtype, out, grad) on the
// current device; false if none.
bool tuned_launch(int L, int dtype, int out, int grad, sph_launch* s);

// The POINT forward launch shape for FP32 values (+ gradients when grad) at
// this l_max on the current device: the tuned one if installed, else the
// default (points_per_tile and warps_per_block resolved).
sph_launch point_fwd_shape(int L, int grad);

// Bytes of one output row of the POINT forward for this request.
size_t point_row_bytes(int L, int grad, int elem, int hess = 0);

// DEGREE kernels (runtime l_max, degree outermost): Eq. iter-q upward in l
// with 1, 2 or 4 lanes per point, or Eq. iter-q-alt downward in m (one lane
// per point).
int degree_fwd_up1(const FwdArgs& a);
int degree_fwd_up2(const FwdArgs& a);
int degree_fwd_up4(const FwdArgs& a);
int degree_fwd_down(const FwdArgs& a);

// ROW kernels (FP32 arithmetic, 16 <= l_max <= 63, values and gradients):
// part 0 covers 3..5 channels per lane (l_max <= 47), part 1 6..8.
int row_fwd_part0(const FwdArgs& a);
// FP32 forward with Hessians on the ROW decomposition (0 <= l_max <= 63).
int row_hess_fwd(const FwdArgs& a);
// Smallest l_max at which AUTO runs FP32 Hessians on ROW (measured on GB300,
// 400k / 200k points, against POINT with 10 lanes per point): normalized
// from l_max 14 (ROW 1.2x at 14, equal at 15, 2.1x at 16; POINT 1.3-1.5x at
// 12 and 13); the scaled form stays on POINT to its l_max 16 (1.1-2.2x ROW
// at 12..16).
constexpr int kRowHessMinAutoNormalized = 14;
constexpr int kRowHessMinAutoScaled = SPH_MAX_L_POINT + 1;
SPH_HD constexpr int row_hess_min_auto(int normalized) {
    return normalized ? kRowHessMinAutoNormalized : kRowHessMinAutoScaled;
}
int row_fwd_part1(const FwdArgs& a);
int row_bwd_part0(const BwdArgs& a);  // fused recompute-backward (dxyz), FP32
int row_bwd_part1(const BwdArgs& a);
constexpr int kRowMinL = 16;
constexpr int kRowMaxL = 63;

// SLICE kernels (runtime l_max).
int slice_fwd(const FwdArgs& a);
int slice_bwd(const BwdArgs& a);
int slice_dbwd(const BwdArgs& a);

}  // namespace sph
