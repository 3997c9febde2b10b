// Multigrid kernels for the pressure Poisson equation A p = b, A = -Laplacian
// with one ghost layer (Section 2.4: Eq. neg_lap_discretize, the printed
// 3x3x3 kernel, Eq. jacobi_pc, Eqs. restriction / prolongation, Algorithm 1).
//
// The solve runs in correction form: the level-0 residual r = b - A p is
// formed from the FP64 pressure with an FP64 norm, a V-cycle computes the
// correction e from A e = r in the inner precision (FP64, or FP32 for the
// reduced-precision modes), and the last post-smoothing sweep adds e to p.
// In exact arithmetic this is the V-cycle on p itself; in finite precision it
// is defect correction with an FP64 outer residual.
//
//   smoother   e <- e + w_J (r - A e) / D, D = sum_active 2 / h_a^2
//   RES        coarse r = mean of the children's residuals r - A e
//   PROL       e += trilinear interpolation of the coarse correction:
//              3/4 parent + 1/4 neighbour per axis, neighbour index clamped
//   coarsest   e = A^{-1} r with the dense inverse built on the host
#include "fvm_internal.cuh"

namespace {

constexpr int kThreads = 256;

inline unsigned nblocks(int64_t N) { return (unsigned)((N + kThreads - 1) / kThreads); }

template <class T> struct Acc { using type = T; };
template <> struct Acc<__nv_bfloat16> { using type = float; };

__device__ __forceinline__ void decode(const LevelDev& L, int64_t c, int& i, int& j, int& k) {
    i = (int)(c % L.n[0]);
    j = (int)((c / L.n[0]) % L.n[1]);
    k = (int)(c / ((int64_t)L.n[0] * L.n[1]));
}

// value across the face on `side` of cell (i,j,k) along `a`: neighbour,
// Neumann ghost (= eP) at walls, inlets and solid cells, -eP on Dirichlet faces
template <class T, class C>
__device__ __forceinline__ C across(const LevelDev& L, const T* e, int i, int j, int k, int a, int side, C eP) {
    int q[3] = {i, j, k};
    q[a] += side;
    if (q[a] < 0 || q[a] >= L.n[a]) {
        const int face = 2 * a + (side > 0 ? 1 : 0);
        return L.dir[face][face_index(a, i, j, k, L.n)] ? -eP : eP;
    }
    const int64_t c = cell_index(q[0], q[1], q[2], L.n[0], L.n[1]);
    return L.solid[c] ? eP : to_c<C>(ldg(e + c));
}

// (A e)(i,j,k) = sum_active (2 eP - eW - eE) / h_a^2
template <class T, class C>
__device__ __forceinline__ C apply_A(const LevelDev& L, const T* e, int i, int j, int k, C eP) {
    C acc = (C)0;
    for (int a = 0; a < 3; ++a) {
        if (!L.active[a]) continue;
        const C w = across<T, C>(L, e, i, j, k, a, -1, eP);
        const C E = across<T, C>(L, e, i, j, k, a, +1, eP);
        acc += ((eP - w) + (eP - E)) * (C)L.inv_h2[a];
    }
    return acc;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

// level 0: r = b - A p (FP64 arithmetic), per-block sums of r^2 (and b^2)
template <class TB, class TI>
__global__ void k_resid0(LevelDev L, const double* __restrict__ p, const TB* __restrict__ b, TI* __restrict__ r,
                         double* __restrict__ partials, int want_b2) {
    __shared__ double red[kThreads / 32];
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double r2 = 0.0, b2 = 0.0;
    if (c < L.N) {
        double rv = 0.0;
        if (!L.solid[c]) {
            int i, j, k;
            decode(L, c, i, j, k);
            const double bv = to_c<double>(ldg(b + c));
            rv = bv - apply_A<double, double>(L, p, i, j, k, __ldg(p + c));
            b2 = bv * bv;
        }
        r[c] = from_c<TI, double>(rv);
        r2 = rv * rv;
    }
    const double s = block_sum(r2, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
    if (want_b2) {
        const double t = block_sum(b2, red);
        if (threadIdx.x == 0) partials[gridDim.x + blockIdx.x] = t;
    }
}

// fixed-order sum of the per-block partials (deterministic norms)
__global__ void k_norm_finalize(const double* __restrict__ partials, int nb, int want_b2, double* out) {
    __shared__ double red[kThreads / 32];
    double a = 0.0, b = 0.0;
    for (int x = threadIdx.x; x < nb; x += blockDim.x) {
        a += partials[x];
        if (want_b2) b += partials[nb + x];
    }
    const double sa = block_sum(a, red);
    const double sb = block_sum(b, red);
    if (threadIdx.x == 0) {
        out[0] = sa;
        if (want_b2) out[1] = sb;
    }
}

// first sweep from e = 0: e = w_J r / D
template <class TI>
__global__ void k_smooth_first(LevelDev L, const TI* __restrict__ r, TI* __restrict__ e) {
    using C = typename Acc<TI>::type;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.N) return;
    C v = (C)0;
    if (!L.solid[c]) v = (C)L.wJ * to_c<C>(ldg(r + c)) * (C)L.inv_D;
    e[c] = from_c<TI, C>(v);
}

template <class TI>
__global__ void k_smooth(LevelDev L, const TI* __restrict__ ein, const TI* __restrict__ r, TI* __restrict__ eout) {
    using C = typename Acc<TI>::type;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.N) return;
    C v = (C)0;
    if (!L.solid[c]) {
        int i, j, k;
        decode(L, c, i, j, k);
        const C eP = to_c<C>(ldg(ein + c));
        v = eP + (C)L.wJ * (to_c<C>(ldg(r + c)) - apply_A<TI, C>(L, ein, i, j, k, eP)) * (C)L.inv_D;
    }
    eout[c] = from_c<TI, C>(v);
}

// last level-0 sweep: p += e + w_J (r - A e) / D
template <class TI>
__global__ void k_smooth_to_p(LevelDev L, const TI* __restrict__ ein, const TI* __restrict__ r,
                              double* __restrict__ p) {
    using C = typename Acc<TI>::type;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.N) return;
    if (L.solid[c]) return;
    int i, j, k;
    decode(L, c, i, j, k);
    const C eP = to_c<C>(ldg(ein + c));
    const C v = eP + (C)L.wJ * (to_c<C>(ldg(r + c)) - apply_A<TI, C>(L, ein, i, j, k, eP)) * (C)L.inv_D;
    p[c] += (double)v;
}

// coarse r = mean over the children of (r - A e); one thread per coarse cell
template <class TI>
__global__ void k_resid_restrict(LevelDev Lf, LevelDev Lc, const TI* __restrict__ e, const TI* __restrict__ r,
                                 TI* __restrict__ rc) {
    using C = typename Acc<TI>::type;
    const int64_t cc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cc >= Lc.N) return;
    int I, J, K;
    decode(Lc, cc, I, J, K);
    const int fx = Lf.active[0] ? 2 : 1, fy = Lf.active[1] ? 2 : 1, fz = Lf.active[2] ? 2 : 1;
    C sum = (C)0;
    for (int dz = 0; dz < fz; ++dz)
        for (int dy = 0; dy < fy; ++dy)
            for (int dx = 0; dx < fx; ++dx) {
                const int i = I * fx + dx, j = J * fy + dy, k = K * fz + dz;
                const int64_t c = cell_index(i, j, k, Lf.n[0], Lf.n[1]);
                if (Lf.solid[c]) continue;
                const C eP = to_c<C>(ldg(e + c));
                sum += to_c<C>(ldg(r + c)) - apply_A<TI, C>(Lf, e, i, j, k, eP);
            }
    rc[cc] = from_c<TI, C>(sum / (C)(fx * fy * fz));
}

// e += PROL(ec) on fluid fine cells
template <class TI>
__global__ void k_prolong_add(LevelDev Lf, LevelDev Lc, const TI* __restrict__ ec, TI* __restrict__ e) {
    using C = typename Acc<TI>::type;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= Lf.N) return;
    if (Lf.solid[c]) return;
    int i, j, k;
    decode(Lf, c, i, j, k);
    const int f[3] = {i, j, k};
    int P[3], Nb[3];
    for (int a = 0; a < 3; ++a) {
        if (Lf.active[a]) {
            P[a] = f[a] >> 1;
            const int s = (f[a] & 1) ? 1 : -1;
            int q = P[a] + s;
            q = q < 0 ? 0 : (q >= Lc.n[a] ? Lc.n[a] - 1 : q);
            Nb[a] = q;
        } else {
            P[a] = f[a];
            Nb[a] = f[a];
        }
    }
    C acc = (C)0;
    for (int sz = 0; sz < 2; ++sz) {
        if (sz && !Lf.active[2]) break;
        const int kk = sz ? Nb[2] : P[2];
        const C wz = Lf.active[2] ? (sz ? (C)0.25 : (C)0.75) : (C)1;
        for (int sy = 0; sy < 2; ++sy) {
            if (sy && !Lf.active[1]) break;
            const int jj = sy ? Nb[1] : P[1];
            const C wy = Lf.active[1] ? (sy ? (C)0.25 : (C)0.75) : (C)1;
            for (int sx = 0; sx < 2; ++sx) {
                if (sx && !Lf.active[0]) break;
                const int ii = sx ? Nb[0] : P[0];
                const C wx = Lf.active[0] ? (sx ? (C)0.25 : (C)0.75) : (C)1;
                acc += wx * wy * wz * to_c<C>(ldg(ec + cell_index(ii, jj, kk, Lc.n[0], Lc.n[1])));
            }
        }
    }
    e[c] = from_c<TI, C>(to_c<C>(e[c]) + acc);
}

// coarsest level: e = A^{-1} r (row-major dense inverse, FP64), one block
template <class TI>
__global__ void k_coarse_solve(int n, const double* __restrict__ Ainv, const TI* __restrict__ rc,
                               TI* __restrict__ ec) {
    __shared__ double rs[FVM_MAX_COARSE];
    for (int x = threadIdx.x; x < n; x += blockDim.x) rs[x] = to_c<double>(rc[x]);
    __syncthreads();
    for (int row = threadIdx.x; row < n; row += blockDim.x) {
        double acc = 0.0;
        const double* a = Ainv + (int64_t)row * n;
        for (int col = 0; col < n; ++col) acc += a[col] * rs[col];
        ec[row] = from_c<TI, double>(acc);
    }
}

template <class A, class B>
__global__ void k_convert(const A* __restrict__ src, B* __restrict__ dst, int64_t N) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) dst[c] = from_c<B, double>(to_c<double>(src[c]));
}

}  // namespace

int resid0_blocks(int64_t N) { return (int)nblocks(N); }

#define DISPATCH_I(inner, ...)                                        \
    do {                                                              \
        if ((inner) == FVM_FP64) { using TI = double; __VA_ARGS__; }  \
        else if ((inner) == FVM_FP32) { using TI = float; __VA_ARGS__; } \
        else { using TI = __nv_bfloat16; __VA_ARGS__; }               \
    } while (0)

cudaError_t launch_resid0(int inner, int bprec, const LevelDev& L, const double* p, const void* b, void* r,
                          double* partials, int want_b2, cudaStream_t s, int* nblocks_out) {
    const unsigned nb = nblocks(L.N);
    if (nblocks_out) *nblocks_out = (int)nb;
    DISPATCH_I(inner, {
        if (bprec == FVM_FP64)
            k_resid0<double, TI><<<nb, kThreads, 0, s>>>(L, p, (const double*)b, (TI*)r, partials, want_b2);
        else if (bprec == FVM_FP32)
            k_resid0<float, TI><<<nb, kThreads, 0, s>>>(L, p, (const float*)b, (TI*)r, partials, want_b2);
        else
            k_resid0<__nv_bfloat16, TI><<<nb, kThreads, 0, s>>>(L, p, (const __nv_bfloat16*)b, (TI*)r, partials,
                                                                 want_b2);
    });
    return cudaGetLastError();
}

cudaError_t launch_norm_finalize(const double* partials, int nb, int want_b2, double* out, cudaStream_t s) {
    k_norm_finalize<<<1, kThreads, 0, s>>>(partials, nb, want_b2, out);
    return cudaGetLastError();
}

cudaError_t launch_smooth_first(int inner, const LevelDev& L, const void* r, void* e, cudaStream_t s) {
    DISPATCH_I(inner, k_smooth_first<TI><<<nblocks(L.N), kThreads, 0, s>>>(L, (const TI*)r, (TI*)e));
    return cudaGetLastError();
}

cudaError_t launch_smooth(int inner, const LevelDev& L, const void* e_in, const void* r, void* e_out,
                          cudaStream_t s) {
    DISPATCH_I(inner, k_smooth<TI><<<nblocks(L.N), kThreads, 0, s>>>(L, (const TI*)e_in, (const TI*)r,
                                                                      (TI*)e_out));
    return cudaGetLastError();
}

cudaError_t launch_smooth_to_p(int inner, const LevelDev& L, const void* e_in, const void* r, double* p,
                               cudaStream_t s) {
    DISPATCH_I(inner, k_smooth_to_p<TI><<<nblocks(L.N), kThreads, 0, s>>>(L, (const TI*)e_in, (const TI*)r, p));
    return cudaGetLastError();
}

cudaError_t launch_resid_restrict(int inner, const LevelDev& Lf, const LevelDev& Lc, const void* e, const void* r,
                                  void* rc, cudaStream_t s) {
    DISPATCH_I(inner, k_resid_restrict<TI><<<nblocks(Lc.N), kThreads, 0, s>>>(Lf, Lc, (const TI*)e,
                                                                               (const TI*)r, (TI*)rc));
    return cudaGetLastError();
}

cudaError_t launch_prolong_add(int inner, const LevelDev& Lf, const LevelDev& Lc, const void* ec, void* e,
                               cudaStream_t s) {
    DISPATCH_I(inner, k_prolong_add<TI><<<nblocks(Lf.N), kThreads, 0, s>>>(Lf, Lc, (const TI*)ec, (TI*)e));
    return cudaGetLastError();
}

cudaError_t launch_coarse_solve(int inner, const LevelDev& Lc, const double* Ainv, const void* rc, void* ec,
                                cudaStream_t s) {
    DISPATCH_I(inner, k_coarse_solve<TI><<<1, kThreads, 0, s>>>((int)Lc.N, Ainv, (const TI*)rc, (TI*)ec));
    return cudaGetLastError();
}

cudaError_t launch_convert(int sp, int dp, const void* src, void* dst, int64_t N, cudaStream_t s) {
    const unsigned nb = nblocks(N);
    if (sp == FVM_FP64 && dp == FVM_FP32) k_convert<double, float><<<nb, kThreads, 0, s>>>((const double*)src, (float*)dst, N);
    else if (sp == FVM_FP32 && dp == FVM_FP64) k_convert<float, double><<<nb, kThreads, 0, s>>>((const float*)src, (double*)dst, N);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}
