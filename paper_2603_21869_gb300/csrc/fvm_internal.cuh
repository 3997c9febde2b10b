// Internal declarations of the k-omega finite-volume library: device-side
// case and level descriptions, the ghost-cell rules of the paper's
// boundary treatment (Section 2.5) and the launchers shared between
// translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/fvm.h"

#define FVM_MAX_PATCHES 16
#define FVM_MAX_BOXES 32
#define FVM_MAX_LEVELS 12
#define FVM_MAX_COARSE 1024

// Face kinds seen from a cell, one per side.
enum { FK_INTERIOR = 0, FK_WALL = 1, FK_INLET = 2, FK_OUTLET = 3, FK_EMPTY = 4 };

struct PatchDev {
    int32_t kind;
    int32_t thermal;
    double T_value;      // fixed wall temperature
    double q_coef;       // heat flux q / (rho cp alpha); ghost = T_P + q_coef * h_normal
    double vel[3];       // inlet velocity vector (inward normal * u_normal)
    double T_in, k_in, om_in;
};

struct BoxDev {
    int32_t thermal;
    int32_t pad;
    double T_value;
    double q_coef;
};

// Everything the step kernels need about a case; passed by value.
struct CaseDev {
    int32_t n[3];
    int32_t active[3];       // n > 1
    int64_t N;
    double h[3], inv_h[3], inv_h2[3];
    double nu, alpha;        // molecular viscosity and diffusivity nu / Pr
    double inv_Prt, inv_sigk, inv_sigw;
    double gb[3];            // -g_i beta_T when buoyancy is on, else 0
    double T_ref;
    double om_wall[3];       // 6 nu / (beta_i (h_a / 2)^2)
    double cfl, dt0;
    int32_t dt_adapt;
    int32_t n_patches, n_boxes, pad;
    const uint8_t* tag;      // 0 fluid, b + 1 solid cell of box b
    const uint8_t* face_patch[6];
    PatchDev patch[FVM_MAX_PATCHES];
    BoxDev box[FVM_MAX_BOXES];
};

// One multigrid level (pressure-like fields).
struct LevelDev {
    int32_t n[3];
    int32_t active[3];
    int64_t N;
    double inv_h2[3];
    double inv_D;            // 1 / sum_active 2 / h_a^2
    double wJ;               // Jacobi weight
    const uint8_t* solid;    // nonzero = solid
    const uint8_t* dir[6];   // per boundary-face cell: 1 = Dirichlet (p = 0 on the face)
};

// ---------------------------------------------------------------- helpers
__host__ __device__ __forceinline__ int64_t cell_index(int i, int j, int k, int nx, int ny) {
    return ((int64_t)k * ny + j) * nx + i;
}

// index of boundary cell (i,j,k) on the face map of a face along `axis`
__host__ __device__ __forceinline__ int face_index(int axis, int i, int j, int k, const int32_t* n) {
    if (axis == 0) return j + n[1] * k;
    if (axis == 1) return i + n[0] * k;
    return i + n[0] * j;
}

template <class T> __device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }
template <> __device__ __forceinline__ __nv_bfloat16 ldg(const __nv_bfloat16* p) { return *p; }

template <class C, class S> __device__ __forceinline__ C to_c(S x) { return (C)x; }
template <> __device__ __forceinline__ float to_c<float, __nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <> __device__ __forceinline__ double to_c<double, __nv_bfloat16>(__nv_bfloat16 x) { return (double)__bfloat162float(x); }
template <class S, class C> __device__ __forceinline__ S from_c(C x) { return (S)x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_c<__nv_bfloat16, float>(float x) { return __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 from_c<__nv_bfloat16, double>(double x) { return __float2bfloat16_rn((float)x); }

// ---------------------------------------------------------------- launchers
struct StatePtrs {
    void* f[6];   // u, v, w, T, k, omega
};

// step kernels (step_kernels.cu); prec = FVM_FP64 or FVM_FP32
cudaError_t launch_init_state(int prec, const CaseDev& cd, StatePtrs st, const double* base,
                              uint64_t seed, double eps, cudaStream_t s);
cudaError_t launch_dt(int prec, const CaseDev& cd, StatePtrs st, double* dt_state, cudaStream_t s);
cudaError_t launch_destruction(int prec, const CaseDev& cd, StatePtrs in, void* k_out, void* om_out,
                               const double* dt_state, cudaStream_t s);
cudaError_t launch_explicit(int prec, const CaseDev& cd, StatePtrs in, StatePtrs out,
                            const double* dt_state, cudaStream_t s);
cudaError_t launch_rhs(int prec, const CaseDev& cd, StatePtrs in, void* b, const double* dt_state,
                       cudaStream_t s);
cudaError_t launch_project(int prec, const CaseDev& cd, const LevelDev& L0, StatePtrs in, StatePtrs out,
                           const double* p, const double* dt_state, cudaStream_t s);
cudaError_t launch_pack(int prec, const void* src, double* dst, int64_t N, cudaStream_t s);
cudaError_t launch_unpack(int prec, const double* src, void* dst, int64_t N, cudaStream_t s);

// multigrid kernels (mg_kernels.cu); inner = FVM_FP64 / FVM_FP32 (type of r, e on all levels),
// bprec = storage type of b
cudaError_t launch_resid0(int inner, int bprec, const LevelDev& L, const double* p, const void* b,
                          void* r, double* partials, int want_b2, cudaStream_t s, int* nblocks_out);
cudaError_t launch_norm_finalize(const double* partials, int nblocks, int want_b2, double* out,
                                 cudaStream_t s);
cudaError_t launch_smooth_first(int inner, const LevelDev& L, const void* r, void* e, cudaStream_t s);
cudaError_t launch_smooth(int inner, const LevelDev& L, const void* e_in, const void* r, void* e_out,
                          cudaStream_t s);
cudaError_t launch_smooth_to_p(int inner, const LevelDev& L, const void* e_in, const void* r, double* p,
                               cudaStream_t s);
cudaError_t launch_resid_restrict(int inner, const LevelDev& Lf, const LevelDev& Lc, const void* e,
                                  const void* r, void* rc, cudaStream_t s);
cudaError_t launch_prolong_add(int inner, const LevelDev& Lf, const LevelDev& Lc, const void* ec, void* e,
                               cudaStream_t s);
cudaError_t launch_coarse_solve(int inner, const LevelDev& Lc, const double* Ainv, const void* rc, void* ec,
                                cudaStream_t s);
cudaError_t launch_convert(int src_prec, int dst_prec, const void* src, void* dst, int64_t N, cudaStream_t s);
int resid0_blocks(int64_t N);
