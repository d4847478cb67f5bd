// Autotuner for the POINT forward launch shape (points per tile, warps per
// block, resident blocks per SM) and for ragged batch plans, timed on the
// caller's own buffers with CUDA events; a text export/import of the tuned
// table keyed by GPU name; and a measurement of the FP32 / FP64 FMA
// throughput (the arithmetic ceiling of the kernels bound by those pipes).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <sstream>
#include <string>
#include <vector>

#include "sph_internal.h"

using namespace sph;

namespace {

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    EventPair() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~EventPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

int tile_mult(int L, int elem) {
    const int K = (L + 1) * (L + 1);
    int r = (K * elem) % 16;
    if (r == 0) return 1;
    int g = 16;
    while (r) {
        const int t = g % r;
        g = r;
        r = t;
    }
    return 16 / g;
}

std::string device_name() {
    int d = -1;
    cudaDeviceProp p;
    if (cudaGetDevice(&d) != cudaSuccess || cudaGetDeviceProperties(&p, d) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::string s = p.name;
    for (char& c : s)
        if (c == ' ') c = '_';
    return s;
}

__device__ float g_fma_sink_f;
__device__ double g_fma_sink_d;

// Eight independent FMA chains per thread (a <- a b + c converges to
// c / (1 - b), no denormals); the result is stored only under a condition that
// never holds, which keeps every chain live.
template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(int iters) {
    constexpr int kChains = 8;
    T a[kChains];
    const T b = T(0.9999), c = T(1e-4);
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = T(threadIdx.x + i) * T(1e-3);
#pragma unroll 16
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
    T s = T(0);
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == T(-1)) {
        if constexpr (sizeof(T) == 4) {
            g_fma_sink_f = s;
        } else {
            g_fma_sink_d = s;
        }
    }
}

template <typename T>
int fma_peak(cudaStream_t st, int reps, double* tflops) {
    const int threads = 256;
    const int blocks = 8 * sm_count();  // 64 warps per SM
    EventPair ev;
    auto run = [&](int iters, float* ms) -> bool {
        cudaEventRecord(ev.a, st);
        fma_peak_kernel<T><<<blocks, threads, 0, st>>>(iters);
        cudaEventRecord(ev.b, st);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(ev.b) != cudaSuccess) return false;
        return cudaEventElapsedTime(ms, ev.a, ev.b) == cudaSuccess;
    };
    // calibrate the length to ~5 ms per run
    int iters = 256;
    float ms = 0.f;
    if (!run(iters, &ms)) return SPH_ECUDA;
    iters = int(std::min(double(1 << 24), std::max(256.0, iters * 5.0 / std::max(ms, 1e-3f))));
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        if (!run(iters, &ms)) return SPH_ECUDA;
        best = std::min(best, ms);
    }
    const double flops = 2.0 * 8.0 * double(iters) * double(blocks) * threads;
    *tflops = flops / (double(best) * 1e-3) / 1e12;
    return SPH_OK;
}

}  // namespace

extern "C" {

int sphericart_fma_peak(int dtype, void* stream, int reps, double* tflops) {
    if ((dtype != SPH_F32 && dtype != SPH_F64) || reps < 1 || !tflops) {
        set_error("fma_peak: dtype must be SPH_F32 or SPH_F64, reps >= 1, tflops non-NULL");
        return SPH_EINVAL;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        set_error("fma_peak: no usable CUDA device");
        return SPH_ECUDA;
    }
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int rc = dtype == SPH_F64 ? fma_peak<double>(st, reps, tflops) : fma_peak<float>(st, reps, tflops);
    if (rc != SPH_OK) {
        set_error("fma_peak: %s", cudaGetErrorString(cudaGetLastError()));
    }
    return rc;
}

int sphericart_autotune(const void* xyz, int64_t n, int l_max, int normalized, int dtype, int out, void* sph,
                        void* dsph, void* stream, int reps, sph_launch* best, float* best_ms) {
    if (!best || l_max < 0 || l_max > SPH_MAX_L_POINT || n <= 0 || !xyz || !sph) {
        set_error("autotune: need n > 0, 0 <= l_max <= %d, xyz, sph and best", SPH_MAX_L_POINT);
        return SPH_EINVAL;
    }
    if (reps <= 0) reps = 3;
    const int elem = dtype == SPH_F64 ? 8 : (out == SPH_OUT_BF16 ? 2 : 4);
    const int grad = dsph ? 1 : 0;
    const int mult = tile_mult(l_max, elem);
    const size_t row = point_row_bytes(l_max, grad, elem);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    EventPair ev;
    float best_t = 1e30f;
    sph_launch best_s{0, 0, 0, 0};
    const int Ps[] = {32, 28, 24, 20, 16, 12, 8, 4, 2, 1};
    const int Ws[] = {1, 2, 4, 8};
    const int Bs[] = {0, 1, 2, 3, 4, 6, 8, 12, 16, 24, 32};  // > occupancy: blocks scheduled in waves
    // the POINT variant AUTO runs for this request (both take the same shapes)
    const int fam = point_hybrid_wins(l_max, dtype, grad != 0) ? SPH_KERNEL_POINT_HC : SPH_KERNEL_POINT;
    // one lane per point (lanes_per_point 1), then, for FP32 arithmetic with
    // gradients, one lane per output plane (lanes_per_point 4, <= 8 points)
    const bool four = grad && dtype == SPH_F32 && fam == SPH_KERNEL_POINT;
    for (int pass = 0; pass < (four ? 2 : 1); ++pass)
    for (int P : Ps) {
        if (P % mult != 0 || (pass == 1 && P > 8)) continue;
        for (int W : Ws) {
            const size_t smem = size_t(W) * (size_t(P) * row + 64);
            if (smem > size_t(max_smem_optin())) continue;
            for (int B : Bs) {
                sph_launch s{P, W, B, pass == 1 ? 4 : 0};
                int stt = sphericart_compute_ex(xyz, n, l_max, normalized, dtype, out, SPH_Q_NATIVE, fam, &s, sph,
                                                dsph, nullptr, stream);
                if (stt != SPH_OK) {
                    cudaGetLastError();
                    continue;  // shape not launchable here (occupancy, limits)
                }
                std::vector<float> ts;
                for (int r = 0; r < reps; ++r) {
                    cudaEventRecord(ev.a, st);
                    sphericart_compute_ex(xyz, n, l_max, normalized, dtype, out, SPH_Q_NATIVE, fam, &s, sph, dsph,
                                          nullptr, stream);
                    cudaEventRecord(ev.b, st);
                    if (cudaEventSynchronize(ev.b) != cudaSuccess) {
                        set_error("autotune: %s", cudaGetErrorString(cudaGetLastError()));
                        return SPH_ECUDA;
                    }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, ev.a, ev.b);
                    ts.push_back(ms);
                }
                std::sort(ts.begin(), ts.end());
                const float t = ts[ts.size() / 2];
                if (t < best_t) {
                    best_t = t;
                    best_s = s;
                }
            }
        }
    }
    if (best_s.points_per_tile == 0) {
        set_error("autotune: no launchable shape");
        return SPH_EUNSUPPORTED;
    }
    *best = best_s;
    if (best_ms) *best_ms = best_t;
    return sphericart_set_launch(l_max, dtype, out, grad, &best_s);
}

int sphericart_batch_autotune(const sph_batch_set* sets, int nsets, void* stream, int reps, sph_launch* best,
                              float* best_ms) {
    if (!best || !sets || nsets <= 0) {
        set_error("batch_autotune: sets, nsets > 0 and best are required");
        return SPH_EINVAL;
    }
    if (reps <= 0) reps = 3;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    EventPair ev;
    float best_t = 1e30f;
    sph_launch best_s{0, 0, 0, 0};
    // points_per_tile here scales the per-warp budget (in l_max = 8 gradient
    // rows); budget 0 with 0 warps per block is the plan's per-l_max shape
    // (every l_max class on its single-set POINT shape).
    const int budgets[] = {0, 64, 48, 32, 24, 16, 12, 8};
    const int Ws[] = {1, 2, 4};
    const int Bs[] = {0, 2, 3, 4, 8, 16};
    bool found = false;
    for (int bud : budgets)
        for (int W : Ws)
            for (int B : Bs) {
                if (bud == 0 && W != 1) continue;
                sph_launch s{bud, bud == 0 ? 0 : W, B, 0};
                sph_batch_plan* plan = nullptr;
                if (sphericart_batch_plan_create(sets, nsets, &s, &plan) != SPH_OK) {
                    cudaGetLastError();
                    continue;
                }
                std::vector<float> ts;
                bool ok = sphericart_batch_execute(plan, stream) == SPH_OK;
                for (int r = 0; ok && r < reps; ++r) {
                    cudaEventRecord(ev.a, st);
                    ok = sphericart_batch_execute(plan, stream) == SPH_OK;
                    cudaEventRecord(ev.b, st);
                    ok = ok && cudaEventSynchronize(ev.b) == cudaSuccess;
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, ev.a, ev.b);
                    ts.push_back(ms);
                }
                sphericart_batch_plan_destroy(plan);
                if (!ok || ts.empty()) continue;
                std::sort(ts.begin(), ts.end());
                const float t = ts[ts.size() / 2];
                if (t < best_t) {
                    best_t = t;
                    best_s = s;
                    found = true;
                }
            }
    if (!found) {
        set_error("batch_autotune: no launchable shape");
        return SPH_EUNSUPPORTED;
    }
    *best = best_s;
    if (best_ms) *best_ms = best_t;
    return SPH_OK;
}

int sphericart_tune_export(char* buf, size_t len, size_t* needed) {
    std::ostringstream os;
    const std::string name = device_name();
    for (int L = 0; L <= SPH_MAX_L_POINT; ++L)
        for (int dt = 0; dt <= 1; ++dt)
            for (int out = 0; out <= 1; ++out)
                for (int grad = 0; grad <= 2; ++grad) {
                    if (dt == SPH_F64 && out == SPH_OUT_BF16) continue;
                    int fam = 0;
                    sph_launch s{0, 0, 0, 0};
                    if (!tuned_launch(L, dt, out, grad, &s)) continue;
                    (void)fam;
                    os << name << ' ' << L << ' ' << dt << ' ' << out << ' ' << grad << ' ' << s.points_per_tile
                       << ' ' << s.warps_per_block << ' ' << s.blocks_per_sm << ' ' << s.lanes_per_point << '\n';
                }
    const std::string text = os.str();
    if (needed) *needed = text.size() + 1;
    if (buf && len > 0) {
        const size_t k = std::min(len - 1, text.size());
        std::memcpy(buf, text.data(), k);
        buf[k] = '\0';
    }
    return SPH_OK;
}

int sphericart_tune_import(const char* text, int* imported) {
    if (!text) {
        set_error("tune_import: text is NULL");
        return SPH_EINVAL;
    }
    std::istringstream is(text);
    const std::string name = device_name();
    std::string line;
    int count = 0;
    while (std::getline(is, line)) {
        std::istringstream ls(line);
        std::string gpu;
        int L, dt, out, grad, P, W, B;
        if (!(ls >> gpu >> L >> dt >> out >> grad >> P >> W >> B)) continue;
        if (gpu != name) continue;
        int lanes = 0;  // optional 9th field: lanes_per_point
        if (!(ls >> lanes)) lanes = 0;
        sph_launch s{P, W, B, lanes};
        if (sphericart_set_launch(L, dt, out, grad, &s) == SPH_OK) ++count;
    }
    if (imported) *imported = count;
    return SPH_OK;
}

}  // extern "C"
