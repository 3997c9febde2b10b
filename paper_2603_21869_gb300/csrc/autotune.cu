// Autotuner of the multigrid parameters, written on the public C-ABI: each
// candidate runs on a temporary copy of the case (graph mode, after two
// untimed steps that capture both pointer parities), timed with CUDA events
// on the case's stream over `steps` steps to the case's tolerance.
//
// Pass 1 tries the smoother sweep counts V(nu, nu), nu = 2, 3, 4, the
// V-cycles per FP64 outer residual (1..4 with reduced-precision corrections,
// 1 in FP64), the flexible-CG acceleration off / on and the constant or the
// Chebyshev sweep weights (both off with mg_variant 1); pass 2 tries the z
// planes per block of the four-cell level kernels (the built-in rule,
// 1 .. 32) with the best pass-1 choice; pass 3 tries 1 and 2 sweeps on the
// levels below the finest.  A candidate whose solves stop at max_vcycles
// above the tolerance is not eligible.
#include <cstring>
#include <string>
#include <vector>

#include "fvm_internal.cuh"

namespace {

struct Trial {
    int pre, post, inner, planes, krylov, coarse, smoother;
    double ms;
};

// ms per step of one candidate (< 0: failed or not converged)
double time_candidate(const fvm_case_desc& base, const Trial& t, int steps, cudaStream_t s) {
    fvm_case_desc d = base;
    d.pre_sweeps = t.pre;
    d.post_sweeps = t.post;
    d.inner_cycles = t.inner;
    d.sweep_planes = t.planes;
    d.krylov = t.krylov;
    d.coarse_sweeps = t.coarse;
    d.smoother = t.smoother;
    d.stream = s;
    fvm_case* c = nullptr;
    if (fvm_create_case(&d, &c) != FVM_OK) return -1.0;
    double ms = -1.0;
    cudaEvent_t a = nullptr, b = nullptr;
    if (fvm_step(c, 2, nullptr) == FVM_OK && cudaEventCreate(&a) == cudaSuccess &&
        cudaEventCreate(&b) == cudaSuccess && cudaEventRecord(a, s) == cudaSuccess) {
        const fvm_status st = fvm_step(c, steps, nullptr);
        float t_ms = 0.f;
        if (st == FVM_OK && cudaEventRecord(b, s) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
            cudaEventElapsedTime(&t_ms, a, b) == cudaSuccess)
            ms = (double)t_ms / steps;
    }
    cudaGetLastError();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    fvm_destroy_case(c);
    return ms;
}

}  // namespace

extern "C" fvm_status fvm_autotune(const fvm_case_desc* desc, int32_t steps, fvm_tuning* out) {
    if (!desc || !out) {
        set_last_error("null descriptor or output");
        return FVM_ERR_INVALID;
    }
    if (steps < 1) {
        set_last_error("steps < 1");
        return FVM_ERR_INVALID;
    }
    if (fvm_case_bytes(desc) == 0) return FVM_ERR_INVALID;   // fvm_case_bytes left the reason
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        set_last_error("cudaStreamCreate");
        return FVM_ERR_CUDA;
    }
    std::vector<int> inners;
    if (desc->precision == FVM_FP64) inners = {1};
    else inners = {1, 2, 3, 4};
    Trial best{0, 0, 0, 0, 0, 0, 0, -1.0};
    int tried = 0;
    const int kmax = desc->mg_variant == 1 ? 0 : 1;
    for (int sm = 0; sm <= kmax; ++sm)
        for (int kry = 0; kry <= kmax; ++kry)
            for (int nu : {2, 3, 4})
                for (int inner : inners) {
                    Trial t{nu, nu, inner, 0, kry, 0, sm, 0.0};
                    t.ms = time_candidate(*desc, t, steps, s);
                    ++tried;
                    if (t.ms > 0.0 && (best.ms < 0.0 || t.ms < best.ms)) best = t;
                }
    if (best.ms > 0.0)
        for (int planes : {1, 2, 4, 8, 16, 32}) {
            Trial t = best;
            t.planes = planes;
            t.ms = time_candidate(*desc, t, steps, s);
            ++tried;
            if (t.ms > 0.0 && t.ms < best.ms) best = t;
        }
    if (best.ms > 0.0 && desc->mg_variant == 0)
        for (int k : {1, 2}) {
            if (k >= best.pre) continue;
            Trial t = best;
            t.coarse = k;
            t.ms = time_candidate(*desc, t, steps, s);
            ++tried;
            if (t.ms > 0.0 && t.ms < best.ms) best = t;
        }
    cudaStreamDestroy(s);
    if (best.ms < 0.0) {
        set_last_error("no candidate reached the tolerance within max_vcycles");
        return FVM_ERR_NOT_CONVERGED;
    }
    fvm_tuning o;
    memset(&o, 0, sizeof(o));
    o.pre_sweeps = best.pre;
    o.post_sweeps = best.post;
    o.inner_cycles = best.inner;
    o.sweep_planes = best.planes;
    o.krylov = best.krylov;
    o.coarse_sweeps = best.coarse;
    o.smoother = best.smoother;
    o.ms_per_step = best.ms;
    o.candidates = tried;
    *out = o;
    set_last_error("");
    return FVM_OK;
}
