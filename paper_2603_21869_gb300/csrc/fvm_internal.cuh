// Internal declarations of the k-omega finite-volume library: device-side
// case and level descriptions, the ghost-cell rules of the paper's
// boundary treatment (Section 2.7) and the launchers shared between
// translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <type_traits>
#include <utility>
#include <vector>

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
    // FP32 copies of the ghost constants: 2 x the face value, q_coef * h_a
    float vel2f[3], T_in2f, k_in2f, om_in2f, T_value2f, qhf[3];
};

struct BoxDev {
    int32_t thermal;
    int32_t pad;
    double T_value;
    double q_coef;
    float T_value2f, qhf[3];
};

// FP32 copies of the case constants used by the FP32 kernels
struct CaseF {
    float h[3], inv_h[3], inv_h2[3];
    float nu, alpha, inv_Prt, inv_sigk, inv_sigw;
    float gb[3], T_ref, om_wall[3];
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
    const uint16_t* nbf0;    // the level-0 neighbour codes (LevelDev::nbf): a fluid cell whose codes on the
    uint32_t regular_mask;   // active axes (these bits) are all 0 has six fluid in-grid neighbours
    int32_t pad2;
    CaseF f;
    PatchDev patch[FVM_MAX_PATCHES];
    BoxDev box[FVM_MAX_BOXES];
};

// a constant in the compute type: the double for FP64 kernels, its FP32 copy otherwise
template <class C> __device__ __forceinline__ C prm(double d, float f);
template <> __device__ __forceinline__ double prm<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float prm<float>(double, float f) { return f; }

// Double-float values: FP64-accurate quantities handled without the FP64 pipe
// (1/64 of the FP32 rate on this part): ff_add / ff_mul are Dekker's
// error-free sum and the FMA-based product, renormalised.
struct FF {
    float h, l;
};

__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ FF ff_norm(float h, float l) {
    const float s = h + l;
    return {s, l - (s - h)};
}

__device__ __forceinline__ FF ff_add(FF x, FF y) {
    const FF s = ff_two_sum(x.h, y.h);
    return ff_norm(s.h, s.l + (x.l + y.l));
}

__device__ __forceinline__ FF ff_neg(FF x) { return {-x.h, -x.l}; }

__device__ __forceinline__ FF ff_mul(FF x, FF c) {
    const float p = x.h * c.h;
    float e = fmaf(x.h, c.h, -p);
    e = fmaf(x.h, c.l, e);
    e = fmaf(x.l, c.h, e);
    return ff_norm(p, e);
}

// x - y rounded to FP32
__device__ __forceinline__ float ff_diff(FF x, FF y) {
    const FF s = ff_two_sum(x.h, -y.h);
    return s.h + (s.l + (x.l - y.l));
}

// The pressure p.  FP64 cases store it in FP64.  The reduced-precision cases
// store, in the same 8 bytes per cell, a double-float pair: hi and lo, two FP32
// values (interleaved) with p = hi + lo and |lo| <= ulp(hi) / 2, about 48
// significant bits, which their kernels read and update with FP32 arithmetic
// only.  A kernel's compute type says which: FP64 kernels see doubles, FP32 and
// BF16 kernels see pairs (pp_*).
__device__ __forceinline__ FF pp_load(const double* p, int64_t c) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p) + c);
    return {v.x, v.y};
}
// hi + lo + v, renormalised (Knuth's two-sum of hi and v, then the low parts folded in)
__device__ __forceinline__ float2 pp_plus(float2 x, float v) {
    const float s = x.x + v;
    const float bb = s - x.x;
    const float e = (x.x - (s - bb)) + (v - bb) + x.y;
    const float hi = s + e;
    return make_float2(hi, e - (hi - s));
}
__device__ __forceinline__ void pp_add(double* p, int64_t c, float v) {
    float2* q = reinterpret_cast<float2*>(p) + c;
    *q = pp_plus(*q, v);
}
// conversions (FP64 arithmetic: only for reads, writes and the small scalar paths)
__device__ __forceinline__ double pp_get(const double* p, int64_t c) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p) + c);
    return (double)v.x + (double)v.y;
}
__device__ __forceinline__ float2 pp_from_double(double x) {
    const float hi = __double2float_rn(x);
    return make_float2(hi, __double2float_rn(x - (double)hi));
}

// One multigrid level (pressure-like fields).
struct LevelDev {
    int32_t n[3];
    int32_t active[3];
    int64_t N;
    double inv_h2[3];
    double inv_D;            // 1 / sum_active 2 / h_a^2
    double wJ;               // Jacobi weight
    double diag;             // sum_active 2 / h_a^2 (A's diagonal away from boundaries)
    float inv_h2f[3], inv_Df, wJf, diagf;   // FP32 copies (no FP64-pipe conversions in FP32 kernels)
    double ih2a[3];          // inv_h2 on active axes, 0 on a collapsed axis
    float ih2af[3];
    float ih2alo[3];         // ih2a - ih2af (float-float coefficients)
    int32_t zc_fixed;        // z planes per block of the four-cell kernels (0: the rule)
    const uint8_t* solid;    // nonzero = solid
    const uint8_t* dir[6];   // per boundary-face cell: 1 = Dirichlet (p = 0 on the face)
    const uint16_t* nbf;     // per cell: 2 bits per face (x-,x+,y-,y+,z-,z+): 0 fluid neighbour,
                             // 1 zero-gradient ghost, 2 zero-value ghost; bit 12: the cell is solid;
                             // bit 13: a face whose ghost is not the clamped in-grid load (a zero-value
                             // face, or a zero-gradient face towards a solid neighbour)
};

// Device-side state of one pressure solve: the last residual norms and the
// stopping rule, applied by the level-0 residual kernel.
struct SolveState {
    double r2, b2, rel;
    double tol;
    int32_t cycles;          // V-cycles started in this solve
    int32_t active;          // 1 while another cycle runs
    uint32_t counter;        // blocks finished (last-block reduction)
    int32_t nonfinite;       // sticky flag: a non-finite norm was seen
    int32_t total_cycles;    // summed over the current fvm_step call
    int32_t max_cycles;
    int32_t fixed;           // > 0: exactly this many cycles
    int32_t notconv;         // sticky flag: a solve stopped at max_cycles above tol
    int32_t inner;           // V-cycles per outer (FP64) residual
    // flexible CG with one kept direction (krylov = 1)
    uint32_t g_counter;      // blocks finished in the inner-product pass
    int32_t g_valid;         // a previous direction is kept
    double g_alpha, g_beta;  // step along the new direction, its component along the previous one
    double g_dq;             // (d, A d) of the kept direction
};

// Levels lc..L-1, cycled by one CTA in shared memory.
// per-sweep Jacobi weights of the Chebyshev smoother (smoother 1: at most this many sweeps a side)
constexpr int kMaxChebSweeps = 16;

struct CoarseLevels {
    int32_t nl;              // number of levels handled
    int32_t pre, post;
    int32_t cheb;            // 1: sweep i of a side takes w[side][i] (0 pre, 1 post); 0: the level's wJ
    LevelDev lv[FVM_MAX_LEVELS];
    double w[2][kMaxChebSweeps];
    float wf[2][kMaxChebSweeps];
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

// level parameters in the compute type (FP32 kernels read the FP32 copies)
template <class C> struct LP;
template <> struct LP<double> {
    static __device__ __forceinline__ double ih2(const LevelDev& L, int a) { return L.inv_h2[a]; }
    static __device__ __forceinline__ double iD(const LevelDev& L) { return L.inv_D; }
    static __device__ __forceinline__ double wJ(const LevelDev& L) { return L.wJ; }
    static __device__ __forceinline__ double diag(const LevelDev& L) { return L.diag; }
    static __device__ __forceinline__ double ih2a(const LevelDev& L, int a) { return L.ih2a[a]; }
};
template <> struct LP<float> {
    static __device__ __forceinline__ float ih2(const LevelDev& L, int a) { return L.inv_h2f[a]; }
    static __device__ __forceinline__ float iD(const LevelDev& L) { return L.inv_Df; }
    static __device__ __forceinline__ float wJ(const LevelDev& L) { return L.wJf; }
    static __device__ __forceinline__ float diag(const LevelDev& L) { return L.diagf; }
    static __device__ __forceinline__ float ih2a(const LevelDev& L, int a) { return L.ih2af[a]; }
};

// ---------------------------------------------------------------- launchers
struct StatePtrs {
    void* f[6];   // u, v, w, T, k, omega
};

// step kernels (step_kernels.cu); prec = FVM_FP64 or FVM_FP32
cudaError_t launch_init_state(int prec, const CaseDev& cd, StatePtrs st, const double* base,
                              uint64_t seed, double eps, cudaStream_t s);
cudaError_t launch_dt(int prec, const CaseDev& cd, StatePtrs st, double* dt_state, cudaStream_t s);
// b_out not null: also the pressure right-hand side b = -div(u)/dt of the (unchanged) velocity
cudaError_t launch_destruction(int prec, const CaseDev& cd, StatePtrs in, void* k_out, void* om_out,
                               const double* dt_state, void* nut_out, void* b_out, cudaStream_t s);
cudaError_t launch_explicit(int prec, const CaseDev& cd, StatePtrs in, StatePtrs out,
                            const double* dt_state, const void* nut, StatePtrs base, double wb, double ws,
                            cudaStream_t s);
cudaError_t launch_rhs(int prec, const CaseDev& cd, StatePtrs in, void* b, const double* dt_state,
                       cudaStream_t s);
cudaError_t launch_project(int prec, const CaseDev& cd, const LevelDev& L0, StatePtrs in, StatePtrs out,
                           const double* p, const double* dt_state, cudaStream_t s);
cudaError_t launch_lambda2(int prec, const CaseDev& cd, StatePtrs in, double* out, cudaStream_t s);
cudaError_t launch_adj_grad(const CaseDev& cd, const LevelDev& L0, const double* ybar, double* q, double dt,
                            cudaStream_t s);
cudaError_t launch_adj_rhs(const CaseDev& cd, const LevelDev& L0, const double* ybar, const double* lambda,
                           double* xbar, double dt, cudaStream_t s);
// adjoints of the destruction half step (ybar, out: u, v, w, k, omega, 5 N; scratch 17 N) and of the
// forward-Euler explicit stage (ybar, xbar: u, v, w, T, k, omega, 6 N; y the stage's output at x;
// scratch 16 N), FP64 cases
cudaError_t launch_destruction_vjp(const CaseDev& cd, StatePtrs x, double dt, const double* ybar, double* out,
                                   double* scratch, cudaStream_t s);
cudaError_t launch_explicit_vjp(const CaseDev& cd, StatePtrs x, StatePtrs y, double dt, const double* ybar,
                                double* xbar, double* scratch, cudaStream_t s);
cudaError_t launch_pack(int prec, const void* src, double* dst, int64_t N, cudaStream_t s);
// the pressure of a reduced-precision case (double-float pairs) to / from FP64
cudaError_t launch_p_to_double(const double* pp, double* dst, int64_t N, cudaStream_t s);
cudaError_t launch_p_from_double(const double* src, double* pp, int64_t N, cudaStream_t s);
cudaError_t launch_p_to_float(const double* pp, float* dst, int64_t N, cudaStream_t s);
cudaError_t launch_p_from_float(const float* src, double* pp, int64_t N, cudaStream_t s);
cudaError_t launch_unpack(int prec, const double* src, void* dst, int64_t N, cudaStream_t s);

// multigrid kernels (mg_kernels.cu); inner = FVM_FP64 / FVM_FP32 / FVM_BF16_MIXED (type of r, e on all
// levels), bprec = storage type of b
cudaError_t launch_solve_begin(SolveState* st, cudaStream_t s);
cudaError_t launch_resid0(int inner, int bprec, const LevelDev& L, const double* p, const void* b, void* r, void* e,
                          double* partials, SolveState* st, cudaGraphConditionalHandle cond,
                          cudaGraphConditionalHandle cond2, int use_cond, cudaStream_t s);
cudaError_t launch_sweep_first(int inner, const LevelDev& L, const void* r, void* e, const SolveState* st,
                               cudaStream_t s);
cudaError_t launch_sweep(int inner, const LevelDev& L, const void* e_in, const void* r, void* e_out,
                         const SolveState* st, cudaStream_t s);
cudaError_t launch_sweep_to_p(int inner, const LevelDev& L, const void* e_in, const void* r, double* p,
                              const SolveState* st, cudaStream_t s);
// the last level-0 sweep of a BF16 level with its result in FP32 (the flexible-CG direction)
cudaError_t launch_sweep_to_f32(int inner, const LevelDev& L, const void* e_in, const void* r, float* z,
                                const SolveState* st, cudaStream_t s);
// (ec0 not null: also the coarse level's first Jacobi sweep from e = 0)
cudaError_t launch_resid_restrict(int inner, const LevelDev& Lf, const LevelDev& Lc, const void* e, const void* r,
                                  void* rc, void* ec0, const SolveState* st, cudaStream_t s);
cudaError_t launch_prolong_add(int inner, const LevelDev& Lf, const LevelDev& Lc, const void* ec, void* e,
                               const SolveState* st, cudaStream_t s);
cudaError_t prepare_coarse_cta(int inner, size_t smem);
// flexible CG with one kept direction around the V-cycles: the inner products
// of z (the V-cycles' correction) with A z, r and the kept direction d_prev
// (last block: beta, alpha), then d = z - beta d_prev, p += alpha d, d kept.
// z and dp are in the inner type, FP32 for BF16 inner (r stays BF16).
// partials: 4 doubles per block, level0_blocks_max(n) blocks at most.
cudaError_t launch_fcg(int inner, const LevelDev& L, const void* z, const void* r, void* dp, double* p,
                       double* partials, SolveState* st, cudaStream_t s);
// the paper's scheme (Algorithm 1)
cudaError_t launch_restrict(int inner, const LevelDev& Lf, const LevelDev& Lc, const void* r, void* rc,
                            const SolveState* st, cudaStream_t s);
cudaError_t launch_prolong_nearest(int inner, const LevelDev& Lf, const LevelDev& Lc, const void* ec, void* e,
                                   const SolveState* st, cudaStream_t s);
cudaError_t launch_prolong_nearest_to_p(int inner, const LevelDev& Lf, const LevelDev& Lc, const void* ec, double* p,
                                        const SolveState* st, cudaStream_t s);
cudaError_t launch_jacobi_p(int bprec, const LevelDev& L, double* p, const void* b, double* q, const SolveState* st,
                            cudaStream_t s);
cudaError_t launch_coarse_cta(int inner, const CoarseLevels& cl, const void* r_in, void* e_out, const double* Ainv,
                              const SolveState* st, cudaStream_t s);
cudaError_t launch_convert(int src_prec, int dst_prec, const void* src, void* dst, int64_t N, cudaStream_t s);
int resid0_blocks(int nx, int ny, int nz);
int level0_blocks_max(int nx, int ny, int nz);   // blocks of any level-0 reduction pass, at most
size_t coarse_cta_smem(const CoarseLevels& cl, int inner);
// ---------------------------------------------------------------- one case or many per launch
// Every step and multigrid kernel is a functor K with `static constexpr int
// kThreads` and `__device__ void run(const BlockAt&) const` (the level-0
// residual returns an int, see below).  k_one runs it over one case's grid.
// k_many runs a table of functors, one per case, whose grids are laid end to
// end: case c owns blocks [start[c], start[c + 1]) of the batch and sees its
// own block position and grid shape, so the same body serves both.  A
// functor's live() says whether its case still takes part (a converged case
// skips the rest of the V-cycle loop); k_one runs only live cases.
struct BlockAt {
    uint3 b;   // block position in the case's grid
    uint3 g;   // the case's grid
};

struct BatchMap {
    const int* start;    // n + 1 block offsets (device)
    const uint3* grid;   // each case's grid (device)
    int n;
    int total;           // start[n]: the cases' blocks together
};

__device__ __forceinline__ int batch_case(const BatchMap& m, int blk) {
    int lo = 0, hi = m.n - 1;   // last case whose first block is <= blk
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(m.start + mid) <= blk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// blocks per SM a functor asks the register allocator to keep resident (K::kMinBlocks, default 1)
template <class K, class = void>
struct MinBlocks {
    static constexpr int value = 1;
};
template <class K>
struct MinBlocks<K, std::void_t<decltype(K::kMinBlocks)>> {
    static constexpr int value = K::kMinBlocks;
};

// Programmatic dependent launch: a kernel may be scheduled while the one
// before it on the stream drains.  Every kernel first waits for the
// previous grid to complete and flush its memory (griddepcontrol.wait; a
// no-op when launched without the attribute), then lets its own dependents
// be scheduled.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <class K>
__global__ void __launch_bounds__(K::kThreads, MinBlocks<K>::value) k_one(const __grid_constant__ K k) {
    pdl_enter();
    k.run(BlockAt{blockIdx, gridDim});
}

// Batched launches are persistent: block i takes the contiguous range
// [i*per, (i+1)*per) of the cases' blocks, walks it with an incremental block
// position, and copies a case's functor into shared memory when it enters
// that case (skipping the case's blocks if it is no longer live).
template <class K>
__device__ __forceinline__ void batch_enter(const K* __restrict__ ks, const BatchMap& m, int c, unsigned char* buf,
                                            int* s_live) {
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    __syncthreads();   // the previous functor is no longer read
    const uint32_t* src = (const uint32_t*)(ks + c);
    for (int q = tid; q < (int)(sizeof(K) / 4); q += nt) ((uint32_t*)buf)[q] = __ldg(src + q);
    __syncthreads();
    if (tid == 0) *s_live = reinterpret_cast<const K*>(buf)->live() ? 1 : 0;
    __syncthreads();
}

// K::kNoShared: run() uses no shared memory, so a batched block needs no barrier before
// the next block of the same case starts (the functor swap between cases has its own)
template <class K, class = void>
struct NoSharedRun {
    static constexpr bool value = false;
};
template <class K>
struct NoSharedRun<K, std::void_t<decltype(K::kNoShared)>> {
    static constexpr bool value = K::kNoShared;
};

// the body of one block, kept out of line: inlined into the walk below it would keep the
// walk's state live across the whole body and raise the register count
template <class K>
__device__ __noinline__ void batch_block_body(const K& k, BlockAt at) {
    k.run(at);
}

template <class K>
__device__ __forceinline__ void batch_run(const K* __restrict__ ks, const BatchMap& m) {
    static_assert(sizeof(K) % 4 == 0, "functor size");
    __shared__ __align__(16) unsigned char buf[sizeof(K)];
    __shared__ int s_live;
    const int per = (m.total + (int)gridDim.x - 1) / (int)gridDim.x;
    const int lo = (int)blockIdx.x * per, hi = min(m.total, lo + per);
    if (lo >= hi) return;
    int c = batch_case(m, lo);
    uint3 g = m.grid[c];
    unsigned l = (unsigned)(lo - __ldg(m.start + c));
    uint3 b = make_uint3(l % g.x, (l / g.x) % g.y, l / (g.x * g.y));
    int cend = __ldg(m.start + c + 1);
    batch_enter(ks, m, c, buf, &s_live);
    for (int v = lo; v < hi; ++v) {
        if (v == cend) {   // the next case with blocks begins at its own first block
            do {           // (the host rejects empty cases; skipping them keeps the walk in bounds anyway)
                ++c;
                cend = __ldg(m.start + c + 1);
            } while (v == cend);
            g = m.grid[c];
            b = make_uint3(0, 0, 0);
            batch_enter(ks, m, c, buf, &s_live);
        }
        if (s_live) {
            batch_block_body(*reinterpret_cast<const K*>(buf), BlockAt{b, g});
            if constexpr (!NoSharedRun<K>::value) __syncthreads();   // run()'s shared memory is reused next
        }
        if (++b.x == g.x) {
            b.x = 0;
            if (++b.y == g.y) {
                b.y = 0;
                ++b.z;
            }
        }
    }
}

// blocks per SM for the batched (persistent) form: K::kMinBlocksMany, default as k_one
template <class K, class = void>
struct MinBlocksMany {
    static constexpr int value = MinBlocks<K>::value;
};
template <class K>
struct MinBlocksMany<K, std::void_t<decltype(K::kMinBlocksMany)>> {
    static constexpr int value = K::kMinBlocksMany;
};

template <class K>
__global__ void __launch_bounds__(K::kThreads, MinBlocksMany<K>::value) k_many(const K* __restrict__ ks, BatchMap m) {
    pdl_enter();
    batch_run(ks, m);
}

// The level-0 residual decides whether another V-cycle runs.  Over a batch,
// each case's last block applies that case's stopping rule; the last block of
// the whole launch then sets the loop condition to "any case still active".
struct BatchCtl {
    unsigned* counter;        // blocks finished in this launch (reset by the last one)
    SolveState* const* st;    // every case's solve state (device array)
    int n;
    cudaGraphConditionalHandle cond, cond2;
    int use_cond;             // 0: none, 1: cond, 2: cond and cond2
};

template <class K>
__global__ void __launch_bounds__(K::kThreads, MinBlocks<K>::value) k_one_r0(const __grid_constant__ K k, cudaGraphConditionalHandle cond,
                                                        cudaGraphConditionalHandle cond2, int use_cond) {
    pdl_enter();
    const int go = k.run(BlockAt{blockIdx, gridDim});   // >= 0 only in the deciding thread
    if (go >= 0 && use_cond) {
        cudaGraphSetConditional(cond, go ? 1u : 0u);
        if (use_cond > 1) cudaGraphSetConditional(cond2, go ? 1u : 0u);
    }
}

template <class K>
__global__ void __launch_bounds__(K::kThreads, MinBlocksMany<K>::value) k_many_r0(const K* __restrict__ ks, BatchMap m, BatchCtl ctl) {
    pdl_enter();
    batch_run(ks, m);
    if (threadIdx.x + threadIdx.y + threadIdx.z != 0) return;
    __threadfence();   // the decisions this block made, before the count
    if (atomicAdd(ctl.counter, 1u) != gridDim.x - 1u) return;
    __threadfence();
    int any = 0;
    for (int i = 0; i < ctl.n; ++i) any |= ((volatile SolveState*)ctl.st[i])->active;
    *ctl.counter = 0u;
    if (ctl.use_cond) {
        cudaGraphSetConditional(ctl.cond, any ? 1u : 0u);
        if (ctl.use_cond > 1) cudaGraphSetConditional(ctl.cond2, any ? 1u : 0u);
    }
}

// Launch with the programmatic-serialization attribute (off when FVM_NO_PDL is set).
bool pdl_enabled();

template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Host side.  While a Recorder is installed on the calling thread, launches
// are recorded instead of issued: the batch runtime replays one case's
// sequence of launches per case, then issues one k_many launch per site.
using ManyFn = cudaError_t (*)(const void* tab, const BatchMap& m, unsigned nblk, dim3 block, size_t smem,
                               const BatchCtl* ctl, cudaStream_t s);

struct RecLaunch {
    std::string site;                  // launch site (the profiling class name)
    double bytes;                      // algorithmic bytes of this launch
    ManyFn many;                       // issues a table of this functor type
    std::vector<unsigned char> arg;    // the functor
    dim3 grid, block;
    size_t smem;
};

struct Recorder {
    std::vector<RecLaunch> out;
    std::string site;                  // set by the caller before each launch site
    double bytes = 0.0;                // algorithmic bytes of the site (given to its first launch)
};

extern thread_local Recorder* g_rec;

// Raise a kernel's dynamic shared-memory limit to at least `bytes`.  The
// limit belongs to the function, which every case shares, so it only grows
// (a later, smaller case must not lower it below what an earlier one needs).
cudaError_t raise_smem_limit(const void* fn, size_t bytes);
// Has the limit been raised to cover `bytes`?  Launches check this first: a
// launch the runtime would reject is not issued (inside a stream capture such
// a launch brought the process down).
bool smem_limit_covers(const void* fn, size_t bytes);

// Blocks of a persistent batched launch: the SMs times the blocks of this
// kernel that fit on one SM (queried once per kernel and shared-memory size,
// outside any capture, when `query` is set).
int persistent_blocks(const void* fn, int threads, size_t smem, bool query);

// nblk == 0: set the kernel's shared-memory limit and size its persistent
// grid only (done before any capture)
template <class K>
cudaError_t many_launch(const void* tab, const BatchMap& m, unsigned nblk, dim3 block, size_t smem,
                        const BatchCtl*, cudaStream_t s) {
    const void* fn = (const void*)k_many<K>;
    const int threads = (int)(block.x * block.y * block.z);
    if (nblk == 0) {
        const cudaError_t e = smem ? raise_smem_limit(fn, smem) : cudaSuccess;
        if (e != cudaSuccess) return e;
        return persistent_blocks(fn, threads, smem, true) > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
    }
    if (!smem_limit_covers(fn, smem)) return cudaErrorInvalidConfiguration;
    const int pb = persistent_blocks(fn, threads, smem, false);
    if (pb <= 0) return cudaErrorInvalidConfiguration;
    return launch_pdl(k_many<K>, dim3(nblk < (unsigned)pb ? nblk : (unsigned)pb), block, smem, s, (const K*)tab, m);
}

template <class K>
cudaError_t many_launch_r0(const void* tab, const BatchMap& m, unsigned nblk, dim3 block, size_t smem,
                           const BatchCtl* ctl, cudaStream_t s) {
    const void* fn = (const void*)k_many_r0<K>;
    const int threads = (int)(block.x * block.y * block.z);
    if (nblk == 0) return persistent_blocks(fn, threads, smem, true) > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
    const int pb = persistent_blocks(fn, threads, smem, false);
    if (pb <= 0) return cudaErrorInvalidConfiguration;
    return launch_pdl(k_many_r0<K>, dim3(nblk < (unsigned)pb ? nblk : (unsigned)pb), block, smem, s, (const K*)tab, m,
                      *ctl);
}

template <class K>
bool record_launch(const K& k, dim3 grid, dim3 block, size_t smem, ManyFn many) {
    if (!g_rec) return false;
    RecLaunch r;
    r.site = g_rec->site;
    r.bytes = g_rec->bytes;
    g_rec->bytes = 0.0;
    r.many = many;
    r.arg.assign((const unsigned char*)&k, (const unsigned char*)&k + sizeof(K));
    r.grid = grid;
    r.block = block;
    r.smem = smem;
    g_rec->out.push_back(std::move(r));
    return true;
}

template <class K>
cudaError_t launch_k(const K& k, dim3 grid, dim3 block, size_t smem, cudaStream_t s) {
    if (record_launch(k, grid, block, smem, &many_launch<K>)) return cudaSuccess;
    if (!smem_limit_covers((const void*)k_one<K>, smem)) return cudaErrorInvalidConfiguration;
    return launch_pdl(k_one<K>, grid, block, smem, s, k);
}

// a launch that is never batched (no recorder, no table form)
template <class K>
cudaError_t launch_k_one(const K& k, dim3 grid, dim3 block, size_t smem, cudaStream_t s) {
    if (!smem_limit_covers((const void*)k_one<K>, smem)) return cudaErrorInvalidConfiguration;
    return launch_pdl(k_one<K>, grid, block, smem, s, k);
}

template <class K>
cudaError_t launch_r0(const K& k, dim3 grid, dim3 block, cudaGraphConditionalHandle cond,
                      cudaGraphConditionalHandle cond2, int use_cond, cudaStream_t s) {
    if (record_launch(k, grid, block, 0, &many_launch_r0<K>)) return cudaSuccess;
    return launch_pdl(k_one_r0<K>, grid, block, 0, s, k, cond, cond2, use_cond);
}

// message returned by fvm_last_error() on this thread
void set_last_error(const std::string& msg);
