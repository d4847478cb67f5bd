/*
 * sphericart_gb300.h -- C-ABI of the GB300 (sm_103a) spherical-harmonics library.
 *
 * The library evaluates the real spherical harmonics of arXiv 2302.08381
 * ("Fast evaluation of spherical harmonics with sphericart"), Section 2: for
 * every 0 <= l <= l_max and -l <= m <= l, at n independent Cartesian points,
 *
 *   scaled (solid) form   Ytilde_l^m(x,y,z) = r^l Y_l^m
 *                         = F_l^|m| Q_l^|m|(z, r) * { s_|m|, 1/sqrt2, c_m }     (Eq. real-sh-cartesian)
 *   normalized form       Y_l^m = Ytilde_l^m(x/r, y/r, z/r)                     (Section 3)
 *
 * with c_m, s_m from the complex-multiplication recursion (Eq. iter-sc), Q_l^m
 * from the recursion in z and r^2 (Eq. iter-q), prefactors F_l^m tabulated on
 * the host in FP64 (Eq. Flm, iterative form of Appendix C), and Cartesian
 * derivatives from Eq. iter-deri (Hessians by applying Eq. iter-deri twice).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Layout.   xyz     [n, 3]            row-major (x, y, z per point)
 *           sph     [n, K]            K = (l_max+1)^2, column l*l + l + m
 *           dsph    [n, 3, K]         d/dx, d/dy, d/dz planes per point
 *           ddsph   [n, 3, 3, K]      d^2/(dx_i dx_j), i-major
 *           g       [n, K]            upstream gradient of sph (backward)
 *           dxyz    [n, 3]
 * Memory.   Every data pointer is DEVICE memory owned by the caller, unless the
 *           entry point says "host". The library owns only its cached tables
 *           (host FP64 tables and per-device copies), created on first use and
 *           kept until the process exits.
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *           stream). Work is enqueued asynchronously; nothing synchronises
 *           unless stated.
 * Errors.   Every call returns an sph_status. Argument errors are detected on
 *           the host before any launch and return SPH_EINVAL / SPH_EUNSUPPORTED
 *           without touching device memory. A failed launch returns SPH_ECUDA.
 *           sphericart_last_error() gives a message for the calling thread.
 *           The library never aborts, traps or prints.
 * Edge.     n == 0 is a no-op returning SPH_OK. A NULL derivative output skips
 *           that output; ddsph requires dsph.
 * Alignment Buffers aligned to 16 bytes take the bulk-copy (TMA) path; any other
 *           alignment of the element type takes a plain-store path. Never an error.
 * r = 0.    Scaled outputs are the polynomials' values and derivatives at 0.
 *           Normalized outputs at r = 0: Y_0^0 = 1/sqrt(4 pi), everything else 0.
 */
#ifndef SPHERICART_GB300_H
#define SPHERICART_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes returned by every entry point. */
typedef enum {
    SPH_OK = 0,
    SPH_EINVAL = 1,        /* bad argument (n < 0, l_max out of range, NULL required pointer) */
    SPH_EUNSUPPORTED = 2,  /* valid request the library does not implement      */
    SPH_ECUDA = 3,         /* a CUDA runtime call or launch failed               */
    SPH_ENOMEM = 4,        /* a library-owned table could not be allocated       */
    SPH_ETIMEOUT = 5       /* a device-side bounded wait gave up (see device_status) */
} sph_status;

/* Input / compute precision. SPH_F32: xyz, outputs and arithmetic in FP32.
 * SPH_F64: all in FP64. */
typedef enum { SPH_F32 = 0, SPH_F64 = 1 } sph_dtype;

/* Storage type of sph/dsph/ddsph. SPH_OUT_BF16 (only with SPH_F32): values are
 * computed in FP32 and stored as bfloat16, round-to-nearest-even (uint16 bits). */
typedef enum { SPH_OUT_SAME = 0, SPH_OUT_BF16 = 1 } sph_out;

/* Internal precision. SPH_Q_F64 with SPH_F32 ("mixed") keeps FP32 inputs and
 * outputs but runs the unit-vector scaling, the c_m/s_m (Eq. iter-sc) and
 * Q_l^m (Eq. iter-q) recursions and the assembly in FP64, rounding once on
 * store. Measured: FP32 error at high l_max comes from rounding u = xyz/r and
 * the c_m/s_m powers, not from the Q recursion alone. SLICE and DEGREE
 * kernels. */
typedef enum { SPH_Q_NATIVE = 0, SPH_Q_F64 = 1 } sph_qprec;

/* Kernel family. AUTO picks, by measurement on GB300: DEGREE for FP64
 * arithmetic without Hessians (the mixed mode; SPH_F64 from l_max 14, with
 * gradients from l_max 9); else
 * ROW for FP32 Hessians with FP32 storage up to l_max 63, from l_max 14 in
 * the normalized form and beyond SPH_MAX_L_POINT in the scaled one
 * (launch_info reports the scaled form's choice); else POINT when
 * l_max <= SPH_MAX_L_POINT (except bfloat16 Hessians); else ROW for FP32
 * arithmetic up to l_max 63; else DEGREE for bfloat16 storage without
 * Hessians; else SLICE.
 *   POINT:  one thread per point, the whole (l, m) recursion unrolled in
 *           registers for a compile-time l_max, outputs staged in shared memory
 *           and written with bulk (TMA) copies.
 *   SLICE:  a group of lanes per point, each lane owning the m channels
 *           m = j, j+G, ...; any l_max <= SPH_MAX_L; direct coalesced stores.
 *   DEGREE: one thread per point with the degree l outermost at run time (any
 *           l_max <= SPH_MAX_L): the Q columns of the previous two degrees
 *           (Eq. iter-q) sit in shared memory, each degree's columns are staged
 *           and stored by the warp with coalesced row-segment stores. Values
 *           and gradients (no Hessians, no backward).
 *   DEGREE_DOWN: as DEGREE, with Q_l^m of each degree by the downward-in-m
 *           recursion of Eq. iter-q-alt (its printed overall sign corrected:
 *           Q_l^m = -[2(m+1) z Q_l^{m+1} + (x^2+y^2) Q_l^{m+2}]/((l+m+1)(l-m)))
 *           from the tabulated Q_l^l; the paper's one-degree-at-a-time form.
 *   ROW:    FP32 arithmetic, 16 <= l_max <= 63, values and gradients, or
 *           0 <= l_max <= 63 with Hessians (FP32 storage): 8 lanes per point (lane j owns the
 *           channels m = j mod 8, recursion state in registers, degree l
 *           uniform across the lanes); each point's output rows are staged in
 *           shared memory in windows of whole degrees and written with TMA
 *           bulk copies of 32-byte-aligned runs (~1 KB and longer, which
 *           GB300's HBM needs for full write bandwidth; 136-column windows with
 *           Hessians). Also a fused backward (sphericart_backward).
 *   POINT_HC: POINT with the degrees l <= min(l_max, 3) from generated
 *           straight-line ("hard-coded") expressions and Eq. iter-q above
 *           them, as the paper's GPU kernel does (Section 3.2; the hybrid of
 *           Section 3.1, Table 1). l_max <= 8, values and gradients, FP32 or
 *           FP64, same-type storage. */
typedef enum {
    SPH_KERNEL_AUTO = 0,
    SPH_KERNEL_POINT = 1,
    SPH_KERNEL_SLICE = 2,
    SPH_KERNEL_DEGREE = 3,
    SPH_KERNEL_DEGREE_DOWN = 4,
    SPH_KERNEL_ROW = 5,
    SPH_KERNEL_POINT_HC = 6
} sph_kernel;

#define SPH_MAX_L 128
#define SPH_MAX_L_POINT 16

/* Launch shape of the POINT kernels (all zero = library default / tuned).
 *   points_per_tile  points a warp computes per tile, 4..32, multiple of 4
 *   warps_per_block  independent warps per CTA, 1..8
 *   blocks_per_sm    resident CTAs per SM to size the persistent grid (0 = max)
 *   lanes_per_point  POINT: 0 (default), 1, 4 = one lane per output plane
 *                    (value, d/dx, d/dy, d/dz) of each point, points_per_tile
 *                    <= 8: every lane busy where one-lane tiles that fit
 *                    shared memory are short (FP32 arithmetic, gradients, no
 *                    Hessians), 10 = one lane per distinct plane of the
 *                    value, gradient and symmetric Hessian, three points
 *                    per warp pass, off-diagonal lanes writing both mirrors
 *                    (FP32 Hessians, FP32 storage; points_per_tile 3, 6, 9
 *                    or 12, warps_per_block <= 4; any output alignment), or
 *                    16 = one lane per plane of the value, gradient and 3x3
 *                    Hessian (same limits; points_per_tile even and <= 8);
 *                    SLICE: 8, 16 or 32 (0 = by l_max)
 * DEGREE kernels read warps_per_block (0..8, 0 = by shared memory),
 * blocks_per_sm and lanes_per_point (1, 2 or 4 lanes per point for DEGREE, 0 =
 * by measurement; DEGREE_DOWN takes 1). ROW kernels read warps_per_block
 * (forward 0..2, backward 0..8; 0 = 1 forward, 2 with Hessians and backward),
 * blocks_per_sm, and lanes_per_point as the forward window policy (0 = by
 * l_max, 1, 2; with Hessians 0/2 = 136 columns, 1 = one degree of l_max,
 * 3 = 256 columns).
 * The POINT default (no shape given and none tuned) fills ~48 KB tiles (FP32,
 * bf16) or up to 32 points in <= 74 KB with one warp per block (FP64, bound by
 * the FP64 pipe), and with FP32 gradients from l_max 10 runs 4 lanes per
 * point on 8-point tiles, with FP32 Hessians 10 lanes per point where that
 * measured faster (scaled l_max 7..16, normalized 6..13; ROW above); when a call
 * has fewer than 2 x SMs x
 * warps_per_block tiles, it runs fewer warps per block so that the blocks
 * reach every SM.                                                           */
typedef struct {
    int32_t points_per_tile;
    int32_t warps_per_block;
    int32_t blocks_per_sm;
    int32_t lanes_per_point;
} sph_launch;

/* ------------------------------------------------------------------ forward
 * sphericart_compute: FP32 forward, the paper's problem statement (Section 3:
 * all (l, m) up to l_max for many points, optionally derivatives).
 *   xyz    [n,3] f32 (device)          sph   [n,K] f32 (device, required)
 *   dsph   [n,3,K] f32 or NULL         ddsph [n,3,3,K] f32 or NULL (needs dsph)
 *   normalized  0 = scaled r^l Y_l^m, 1 = Y_l^m on the unit sphere
 * Returns SPH_OK, or SPH_EINVAL for n < 0, l_max outside [0, SPH_MAX_L],
 * NULL xyz/sph, or ddsph without dsph. */
int sphericart_compute(const float* xyz, int64_t n, int l_max, int normalized,
                       float* sph, float* dsph, float* ddsph, void* stream);

/* sphericart_compute_ex: forward with every option (same layout as above).
 *   dtype  sph_dtype of xyz and of the arithmetic
 *   out    sph_out storage of sph/dsph/ddsph (element size 4, 8 or 2 bytes)
 *   qprec  sph_qprec of the Q recursion (SPH_Q_F64 with SPH_F32 only)
 *   kernel sph_kernel family; POINT with l_max > SPH_MAX_L_POINT, with the
 *          mixed mode or with bfloat16 Hessians returns SPH_EUNSUPPORTED, and
 *          so do the DEGREE families with ddsph and ROW outside its range
 *   launch NULL or a launch shape (zeros = default)
 * SPH_EUNSUPPORTED also for BF16 output with FP64 arithmetic. */
int sphericart_compute_ex(const void* xyz, int64_t n, int l_max, int normalized,
                          int dtype, int out, int qprec, int kernel,
                          const sph_launch* launch,
                          void* sph, void* dsph, void* ddsph, void* stream);

/* sphericart_compute_host: forward from HOST memory, end to end. Points are
 * taken in chunks of `chunk_points` (0 = 1,048,576; rounded to a multiple of
 * 32 and shrunk to fit) through a caller-provided DEVICE `workspace` of
 * `workspace_bytes` (256-byte aligned; at least two chunk stages of
 * xyz + sph (+ dsph)), and the host->device copy of chunk i+1, the kernel on
 * chunk i and the device->host copy of chunk i-1 overlap on three streams the
 * library owns (one set per device, created on first use). The work is
 * ordered after everything already enqueued on `stream` and `stream` waits
 * for its end; the call itself returns without synchronising. Host buffers
 * should be pinned (cudaHostAlloc / cudaHostRegister) for the copies to be
 * asynchronous. Layouts, dtype and out as in sphericart_compute_ex (FP32 or
 * FP64, optional bf16 store); no Hessians. Errors: SPH_EINVAL for bad sizes,
 * NULL pointers or a workspace too small for two 32-point stages. */
int sphericart_compute_host(const void* xyz_host, int64_t n, int l_max, int normalized,
                            int dtype, int out, void* sph_host, void* dsph_host,
                            void* workspace, size_t workspace_bytes,
                            int64_t chunk_points, void* stream);

/* ----------------------------------------------------------------- backward
 * sphericart_backward: fused recompute-backward (adjoint of the forward values).
 *   dxyz[n, i] = sum_k g[n, k] * d sph[n, k] / d x_i
 * recomputing the recursions of Eqs. iter-sc, iter-q and iter-deri in
 * registers; no [n,3,K] tensor is written. The paper's PyTorch layer instead
 * contracts the dsph materialised by the forward pass (Section 3); that path
 * is sphericart_compute + a contraction.
 *   xyz [n,3], g [n,K], dxyz [n,3], all of `dtype` (device).
 * kernel: AUTO (POINT up to SPH_MAX_L_POINT, then ROW for FP32 up to l_max 63,
 * else SLICE), POINT, SLICE, or ROW (FP32, 16 <= l_max <= 63: 8 lanes per
 * point, the g rows read by TMA bulk loads of whole-degree windows); the
 * DEGREE families return SPH_EUNSUPPORTED. Errors as sphericart_compute_ex. */
int sphericart_backward(const void* xyz, const void* g, int64_t n, int l_max,
                        int normalized, int dtype, int kernel,
                        const sph_launch* launch, void* dxyz, void* stream);

/* sphericart_double_backward: adjoint of sphericart_backward for a cotangent
 * v [n,3] of dxyz (forces training):
 *   grad_g[n, k]   = sum_j v[n, j] d sph[n, k] / d x_j
 *   grad_xyz[n, i] = sum_k g[n, k] sum_j v[n, j] d^2 sph[n, k] / d x_i d x_j
 * Hessians come from Eq. iter-deri applied twice, in registers.
 * Either output may be NULL (skipped). All device, all of `dtype`. */
int sphericart_double_backward(const void* xyz, const void* g, const void* v,
                               int64_t n, int l_max, int normalized, int dtype,
                               int kernel, const sph_launch* launch,
                               void* grad_g, void* grad_xyz, void* stream);

/* ---------------------------------------------------------------- expansion
 * sphericart_expansion: the radial expansion of the paper's Eq. expansion,
 * fused with the harmonics so that Y is never written to memory:
 *   c[i, n, l*l+l+m] = sum_{k = offsets[i]}^{offsets[i+1]-1} R[k, n, l] * Y_l^m(x_k)
 *   xyz      [n_points, 3]            points grouped by centre (device)
 *   radial   [n_points, n_rad, l_max+1] R_nl at each point (device)
 *   offsets  [n_centres + 1] int64    CSR offsets into the points (device)
 *   c        [n_centres, n_rad, (l_max+1)^2] output (device)
 *   normalized 0: Y is the scaled r^l Y_l^m (the paper folds r^-l into R),
 *              1: Y_l^m on the unit sphere.  dtype: SPH_F32 or SPH_F64 for all.
 * l_max <= SPH_MAX_L_POINT, 1 <= n_rad <= 64. A centre whose offsets are not
 * non-decreasing within [0, n_points] gets zeros and ORs the value 2 into the
 * device status word (sphericart_device_status); nothing outside the buffers
 * is read. Returns SPH_EUNSUPPORTED when one warp's staging (32 harmonic
 * rows, two buffers of 32 radial rows and a centre's sums) exceeds the
 * device's shared memory (e.g. FP64 with l_max 16 and 64 radial channels).
 * Each warp streams a contiguous range of centres in 32-point chunks. */
int sphericart_expansion(const void* xyz, const void* radial, const int64_t* offsets,
                         int64_t n_centres, int64_t n_points, int n_rad, int l_max,
                         int normalized, int dtype, void* c, void* stream);

/* ------------------------------------------------------------------ batched
 * One set of a ragged batch: points xyz[n,3] f32 with their own l_max, outputs
 * sph[n,(l_max+1)^2] and dsph[n,3,(l_max+1)^2] (dsph may be NULL). Device
 * pointers; the descriptor array itself lives in HOST memory. */
typedef struct {
    const float* xyz;
    float* sph;
    float* dsph;
    int64_t n;
    int32_t l_max;
    int32_t normalized;
} sph_batch_set;

/* Opaque plan for a ragged batch (FP32, POINT kernels, l_max <= SPH_MAX_L_POINT). */
typedef struct sph_batch_plan sph_batch_plan;

/* sphericart_batch_plan_create: builds the device work list for `nsets` sets
 * (copied from host memory) for persistent launches in which every warp pulls
 * tiles from a device counter: one launch per distinct l_max (mode
 * SPH_BATCH_PER_LMAX, see sphericart_batch_plan_create_ex). The plan owns
 * its device work list (allocated here, freed by _destroy). Buffers of the sets
 * must stay valid while the plan is executed. `launch` may be NULL (default
 * shape); points_per_tile is chosen per l_max to fit a fixed shared-memory
 * budget per warp. Errors: SPH_EINVAL for a NULL pointer, nsets <= 0, a set
 * with n < 0 or l_max outside [0, SPH_MAX_L_POINT]; SPH_ENOMEM / SPH_ECUDA. */
int sphericart_batch_plan_create(const sph_batch_set* sets, int nsets,
                                 const sph_launch* launch, sph_batch_plan** plan);

/* How a plan runs its sets:
 *   SPH_BATCH_PER_LMAX   one persistent launch per distinct l_max, each compiled
 *                        for that l_max alone, with its own tile counter and a
 *                        shared-memory size fitted to that l_max's tile (the
 *                        default of sphericart_batch_plan_create; measured faster
 *                        on GB300)
 *   SPH_BATCH_ONE_LAUNCH one persistent launch for every set (one per
 *                        combination of gradients / normalized present),
 *                        the kernel of sphericart_compute_batched: the sets
 *                        sorted by l_max in shared memory, a switch over the
 *                        compile-time l_max bodies, per-l_max tiles filling
 *                        one shared-memory budget per warp */
typedef enum { SPH_BATCH_PER_LMAX = 0, SPH_BATCH_ONE_LAUNCH = 1 } sph_batch_mode;

/* sphericart_batch_plan_create_ex: sphericart_batch_plan_create with a mode
 * (sph_batch_mode; SPH_EINVAL for any other value). */
int sphericart_batch_plan_create_ex(const sph_batch_set* sets, int nsets,
                                    const sph_launch* launch, int mode,
                                    sph_batch_plan** plan);

/* sphericart_batch_execute: enqueues the plan's launches (one counter reset,
 * then one persistent kernel per launch) on `stream`. Capturable in a CUDA
 * graph. */
int sphericart_batch_execute(const sph_batch_plan* plan, void* stream);

/* sphericart_batch_plan_destroy: frees the plan (synchronises its device). */
int sphericart_batch_plan_destroy(sph_batch_plan* plan);

/* sphericart_batch_plan_info: total points and work tiles of a plan (host). */
int sphericart_batch_plan_info(const sph_batch_plan* plan, int64_t* total_points,
                               int64_t* total_tiles);

/* Flags of sphericart_compute_batched: every set of one call has the same. */
typedef enum { SPH_BATCHED_GRADIENTS = 1, SPH_BATCHED_NORMALIZED = 2 } sph_batched_flags;

/* sphericart_compute_batched: a ragged batch in ONE persistent launch, from a
 * descriptor array in DEVICE memory (the paper's problem, "all (l,m) up to
 * l_max, possibly for many points", Section 3, for many point sets at once;
 * the batched form addresses the under-filled GPU at small point counts noted
 * with Table 3).
 *   desc   DEVICE (or managed / page-locked host) array of nsets sph_batch_set,
 *          read by the kernel: the caller may fill it on the GPU and replay a
 *          captured call with new sizes. Per set: xyz [n,3] f32, sph
 *          [n,(l_max+1)^2] f32, dsph [n,3,(l_max+1)^2] f32 (non-NULL exactly
 *          when flags has SPH_BATCHED_GRADIENTS), n >= 0, 0 <= l_max <= 16,
 *          normalized equal to (flags & SPH_BATCHED_NORMALIZED) != 0, buffers
 *          4-byte aligned (16 for the bulk-store path). A set with n = 0 is
 *          skipped whatever its pointers and flags.
 *   nsets  >= 0 (0: no-op). Arrays longer than 2048 sets run as one launch
 *          per 2048 sets.
 *   flags  SPH_BATCHED_GRADIENTS | SPH_BATCHED_NORMALIZED.
 * Each block (one per SM) sorts the sets by l_max in shared memory, then
 * runs the l_max classes present one after the other, each with its
 * compile-time body, the single-set POINT tile of that l_max and as many
 * warps as its staging buffers fit in the block's shared memory; warps take
 * tiles from per-class counters that the kernel returns to zero itself (a
 * ring of 256 static counter sets per device and flag combination: at most
 * 256 calls may be in flight at once on one device). Sets whose descriptor is invalid are
 * skipped and the value 2 is OR-ed into the device status word (see
 * sphericart_device_status); the host cannot read device descriptors, so
 * these checks happen on the GPU. Capturable in a CUDA graph once a first
 * call on the device has run eagerly (it sets the kernel's shared-memory
 * attribute and allocates the status word). Errors: SPH_EINVAL for nsets <
 * 0, unknown flags, a NULL or pageable desc; SPH_ECUDA on a launch failure. */
int sphericart_compute_batched(const sph_batch_set* desc, int nsets, int flags, void* stream);

/* sphericart_compute_batched_ex: with a launch shape (NULL = default):
 * points_per_tile = tiles that fit this many l_max = 8 value+gradient rows
 * (1,296 bytes each; 0 = the single-set POINT tile of each l_max),
 * warps_per_block in [0,16] caps the warps of a block (0 = 16), blocks_per_sm
 * (0 = occupancy). */
int sphericart_compute_batched_ex(const sph_batch_set* desc, int nsets, int flags,
                                  const sph_launch* launch, void* stream);

/* sphericart_batch_compute_noalloc: evaluates a ragged batch like a plan does,
 * with the one-launch kernel of sphericart_compute_batched (one launch per
 * combination of gradients / normalized present) on `stream`, without
 * allocating any device memory.
 * It exists for callers that cannot call cudaMalloc -- code whose device
 * memory is owned by a fixed arena or a framework allocator, or code that
 * cannot afford the device synchronisation cudaMalloc implies. (The paper has
 * no counterpart: its library allocates nothing of this kind.)
 *   sets / nsets  as for sphericart_batch_plan_create (HOST array, read during
 *                 the call only); at most 4096 sets, more returns SPH_EINVAL.
 *   launch        NULL or a shape, as for sphericart_batch_plan_create.
 * The descriptors are copied into a static device array of the library
 * (160 KB on every GPU that loads it, held until exit); the tile counters
 * are the self-resetting static ring of sphericart_compute_batched. The
 * first call on a device looks up that array's address (set-up); make that
 * first call before any stream capture. The address is kept for the life of
 * the process: after cudaDeviceReset (or anything else that replaces the
 * device's primary context) this entry point must not be called again.
 * Every call reuses the same array, and calls whose work overlaps on the GPU
 * (different streams, or host threads racing) race on it -- serialise them. The work list is staged in host
 * memory that the next call overwrites, so the call refuses a stream that is
 * being captured (SPH_EINVAL, nothing enqueued). Output buffers are the
 * caller's, as everywhere. */
int sphericart_batch_compute_noalloc(const sph_batch_set* sets, int nsets,
                                     const sph_launch* launch, void* stream);

/* ------------------------------------------------------------ e3nn convention
 * Normalizations of sphericart_compute_e3nn (e3nn's names). */
typedef enum {
    SPH_E3NN_INTEGRAL = 0,   /* each component squared integrates to 1 over the sphere */
    SPH_E3NN_COMPONENT = 1,  /* sum_m Y_l^m(u)^2 = 2l + 1 on the unit sphere */
    SPH_E3NN_NORM = 2        /* sum_m Y_l^m(u)^2 = 1 on the unit sphere */
} sph_e3nn_norm;

/* sphericart_compute_e3nn: the harmonics in e3nn's convention (Section 3.2:
 * the paper's library provides wrappers with e3nn's conventions), so that
 * models written against e3nn can switch. e3nn's polar axis is y: its output
 * equals this library's at the permuted point (z, x, y), times sqrt(4 pi)
 * (component) or sqrt(4 pi / (2l+1)) (norm) per l block, with the gradient
 * planes in (d/dx, d/dy, d/dz) order.
 *   xyz        [n,3] device, dtype (SPH_F32 or SPH_F64)
 *   normalize  1 = inputs normalized to the unit sphere (e3nn's normalize=True),
 *              0 = polynomial (scaled) form
 *   workspace  device [n,3] of the dtype (the permuted points), caller-owned
 *   sph        [n,(l_max+1)^2]; dsph [n,3,(l_max+1)^2] or NULL
 * Two small kernels surround the forward: the permutation, and (unless the
 * normalization is "integral" without gradients) an in-place rescale and
 * plane reorder, which reads and writes the outputs once more. Errors as
 * sphericart_compute_ex, SPH_EINVAL for a bad normalization or NULL workspace. */
int sphericart_compute_e3nn(const void* xyz, int64_t n, int l_max, int normalize, int normalization,
                            int dtype, void* workspace, void* sph, void* dsph, void* stream);

/* ----------------------------------------------------------------- services
 * sphericart_last_error: message of the last failed call on this thread
 * (static storage owned by the library; valid until the next call). */
const char* sphericart_last_error(void);

/* sphericart_max_l: largest l_max a (dtype, qprec, kernel) combination takes. */
int sphericart_max_l(int dtype, int qprec, int kernel);

/* sphericart_host_table: copies the host FP64 table `which` for 0..l_max into
 * `out` (HOST memory, (l_max+1)(l_max+2)/2 doubles, entry (l,m) at
 * l(l+1)/2 + m). Host-only; needs no GPU.
 *   which 0: F_l^m, Eq. Flm by the Appendix C iteration
 *         1: Qtilde_l^l = F_l^l Q_l^l on the diagonal (0 elsewhere), Eq. iter-q
 *         2: a_l^m, 3: b_l^m  coefficients of the folded recursion
 *            Qtilde_l^m = a z Qtilde_{l-1}^m - b r^2 Qtilde_{l-2}^m (Eq. iter-q, App. C)
 *         4: e_l^m = F_l^m / F_{l-1}^{m+1}       (d/dx, d/dy of Eq. iter-deri)
 *         5: f_l^m = (l+m) F_l^m / F_{l-1}^m     (d/dz of Eq. iter-deri)
 *         6: d_l   = (2l-1) F_l^{l-1}/F_{l-1}^{l-1} on entry (l, l-1)
 *         7: al_l^m, 8: be_l^m  coefficients of the folded downward recursion
 *            Qtilde_l^m = al z Qtilde_l^{m+1} - be (x^2+y^2) Qtilde_l^{m+2}
 *            (Eq. iter-q-alt with its overall sign corrected)
 * Tables 4 and 5 carry the 1/sqrt2 of the m = 0 column folded in.
 * Returns SPH_EINVAL for a bad `which`, l_max or NULL out. */
int sphericart_host_table(int l_max, int which, double* out);

/* sphericart_device_status: reads and clears the device-side status word of
 * the current device, an OR of: 1 = a bounded wait timed out inside a kernel,
 * 2 = sphericart_compute_batched skipped a set with an invalid descriptor.
 * Synchronises the device. Returns SPH_OK and writes the word to *status. */
int sphericart_device_status(uint32_t* status);

/* sphericart_launch_info: the launch shape the library would use for a
 * forward call (after tuning), for inspection. kernel_out receives the
 * family (POINT or SLICE). Host-only except for a device-properties query. */
int sphericart_launch_info(int l_max, int dtype, int out, int grad, int hess,
                           int* kernel_out, sph_launch* launch_out);

/* sphericart_set_launch: installs a tuned launch shape for forward calls with
 * this (l_max, dtype, out, grad) on the current device; used by AUTO/POINT
 * calls that pass launch == NULL (grad: 0 values, 1 + gradients, 2 + gradients
 * and Hessians). points_per_tile etc. are validated; lanes_per_point 0, 1, 4
 * (FP32 gradients), 10 or 16 (FP32 Hessians, FP32 storage). */
int sphericart_set_launch(int l_max, int dtype, int out, int grad,
                          const sph_launch* launch);

/* sphericart_tune_clear: removes every tuned or installed POINT shape of the
 * current device, so that later calls take the library defaults again. */
int sphericart_tune_clear(void);

/* ---------------------------------------------------------------- autotuner
 * sphericart_autotune: times every valid POINT forward launch shape (points
 * per tile, warps per block, blocks per SM) for this request on the caller's
 * buffers (sph/dsph are overwritten), `reps` timed runs each (median, CUDA
 * events on `stream`; synchronises), installs the fastest for later calls
 * with launch == NULL (as sphericart_set_launch) and returns it in *best
 * (and its time in *best_ms if non-NULL). l_max <= SPH_MAX_L_POINT, n > 0.
 * The autotuner and the batch autotuner are the project's own: the paper
 * grows its shared-memory allocation on first call instead (Section 3). */
int sphericart_autotune(const void* xyz, int64_t n, int l_max, int normalized,
                        int dtype, int out, void* sph, void* dsph, void* stream,
                        int reps, sph_launch* best, float* best_ms);

/* sphericart_batch_autotune: times batch plans for these sets over a grid of
 * per-warp shared-memory budgets, warps per block and blocks per SM, and
 * returns the fastest shape for sphericart_batch_plan_create (for batch plans
 * points_per_tile, 0..160, sets the per-warp budget as that many l_max = 8
 * FP32 value+gradient rows of 1296 bytes; 0 = 32 rows; with points_per_tile
 * and warps_per_block both 0 a SPH_BATCH_PER_LMAX plan gives every l_max class
 * the single-set POINT kernel's tile and warps per block for that l_max).
 * Overwrites the sets' outputs; synchronises. */
int sphericart_batch_autotune(const sph_batch_set* sets, int nsets, void* stream,
                              int reps, sph_launch* best, float* best_ms);

/* sphericart_tune_export: writes the tuned POINT shapes of the current device
 * as text lines "gpu_name l_max dtype out grad P W B lanes" into buf (NUL-terminated,
 * truncated to len); *needed receives the full size. Host memory. */
int sphericart_tune_export(char* buf, size_t len, size_t* needed);

/* sphericart_tune_import: installs the lines of `text` whose gpu_name matches
 * the current device (others are skipped; a missing lanes field reads as 0);
 * *imported receives the count. */
int sphericart_tune_import(const char* text, int* imported);

/* sphericart_fma_peak: measures this device's fused multiply-add throughput
 * in `dtype` (SPH_F32 or SPH_F64): eight independent FMA chains per thread, 64
 * warps per SM, ~5 ms per run, the best of `reps` runs timed with CUDA events
 * on `stream` (synchronises). Writes TFLOP/s (2 flops per FMA) to *tflops
 * (host memory): the arithmetic ceiling of kernels bound by that pipe.
 * Returns SPH_EINVAL for another dtype, reps < 1 or NULL tflops, SPH_ECUDA
 * without a usable device. */
int sphericart_fma_peak(int dtype, void* stream, int reps, double* tflops);

/* sphericart_version: library version as 10000*major + 100*minor + patch. */
int sphericart_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPHERICART_GB300_H */
