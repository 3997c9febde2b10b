// Step kernels of the k-omega finite-volume time step: the seeded initial
// state, the per-step time-step cap, the semi-implicit destruction half
// step (Section 2.5, Eqs. k_des_step / o_des_step, Algorithm 4), the
// explicit stage (Sections 2.3, A.2-A.4, Algorithms 2 and 3), the
// pressure right-hand side (Eq. pc_residual) and the projection.
//
// One thread per cell, x fastest.  Neighbour states come from global
// memory; boundary and obstacle neighbours are replaced by ghost values
// (Section 2.7) computed in registers, so no ghost layer is stored.
#include <cstdio>

#include "fvm_internal.cuh"

namespace {

// Closure constants (Section 2.1; R_beta = 8 is the standard value the paper leaves unstated)
constexpr double kAlphaStarInf = 1.0;
constexpr double kBetaI = 0.072;
constexpr double kAlphaStar0 = kBetaI / 3.0;
constexpr double kRk = 6.0;
constexpr double kAlphaInf = 0.52;
constexpr double kAlpha0 = 1.0 / 9.0;
constexpr double kRw = 2.95;
constexpr double kBetaStarInf = 0.09;
constexpr double kBeta = kBetaI;
constexpr double kRbeta = 8.0;
constexpr double kEpsOmega = 1e-12;
constexpr double kKMin = 1e-14;
constexpr double kOmegaMin = 1e-8;

constexpr int kThreads = 256;
constexpr int BX = 32, BY = 4, BZ = 2;

__device__ __forceinline__ bool cell3(const CaseDev& cd, const BlockAt& at, int& i, int& j, int& k) {
    i = at.b.x * BX + threadIdx.x;
    j = at.b.y * BY + threadIdx.y;
    k = at.b.z * BZ + threadIdx.z;
    return i < cd.n[0] && j < cd.n[1] && k < cd.n[2];
}

template <class C>
struct St {
    C u, v, w, T, k, om;
};

template <class C>
__device__ __forceinline__ C vcomp(const St<C>& s, int a) {
    return a == 0 ? s.u : (a == 1 ? s.v : s.w);
}

template <class C>
__device__ __forceinline__ C thermal_ghost(int thermal, double Tval, float T2f, double qcoef, double h, float qhf,
                                          C TP) {
    if (thermal == FVM_FIXED_T) return prm<C>(2.0 * Tval, T2f) - TP;
    if (thermal == FVM_HEAT_FLUX) return TP + prm<C>(qcoef * h, qhf);
    return TP;
}

// dt (slot 0) or dt/2 (slot 1) in the compute type
template <class C>
__device__ __forceinline__ C dt_of(const double* dt_state, int slot) {
    return prm<C>(dt_state[slot], ((const float*)(dt_state + 4))[slot]);
}

template <class S, class C>
__device__ __forceinline__ St<C> load_state(const StatePtrs& st, int64_t c) {
    St<C> s;
    s.u = to_c<C>(ldg((const S*)st.f[0] + c));
    s.v = to_c<C>(ldg((const S*)st.f[1] + c));
    s.w = to_c<C>(ldg((const S*)st.f[2] + c));
    s.T = to_c<C>(ldg((const S*)st.f[3] + c));
    s.k = to_c<C>(ldg((const S*)st.f[4] + c));
    s.om = to_c<C>(ldg((const S*)st.f[5] + c));
    return s;
}

// State across the face on `side` (-1 / +1) of cell (i,j,k) along `axis`:
// the neighbour's values, or the ghost values of Section 2.7 at a domain
// face or a solid neighbour.  Returns the face kind.
template <class S, class C>
__device__ __forceinline__ int neighbour(const CaseDev& cd, const StatePtrs& st, int i, int j, int k,
                                         int axis, int side, const St<C>& P, St<C>& g) {
    int q[3] = {i, j, k};
    q[axis] += side;
    if (q[axis] < 0 || q[axis] >= cd.n[axis]) {
        const int face = 2 * axis + (side > 0 ? 1 : 0);
        const PatchDev& pt = cd.patch[cd.face_patch[face][face_index(axis, i, j, k, cd.n)]];
        if (pt.kind == FVM_WALL) {
            g.u = -P.u; g.v = -P.v; g.w = -P.w;
            g.k = P.k; g.om = P.om;
            g.T = thermal_ghost<C>(pt.thermal, pt.T_value, pt.T_value2f, pt.q_coef, cd.h[axis], pt.qhf[axis], P.T);
            return FK_WALL;
        }
        if (pt.kind == FVM_INLET) {
            g.u = prm<C>(2.0 * pt.vel[0], pt.vel2f[0]) - P.u;
            g.v = prm<C>(2.0 * pt.vel[1], pt.vel2f[1]) - P.v;
            g.w = prm<C>(2.0 * pt.vel[2], pt.vel2f[2]) - P.w;
            g.T = prm<C>(2.0 * pt.T_in, pt.T_in2f) - P.T;
            g.k = prm<C>(2.0 * pt.k_in, pt.k_in2f) - P.k;
            g.om = prm<C>(2.0 * pt.om_in, pt.om_in2f) - P.om;
            return FK_INLET;
        }
        g = P;
        return pt.kind == FVM_OUTLET ? FK_OUTLET : FK_EMPTY;
    }
    const int c = q[0] + cd.n[0] * (q[1] + cd.n[1] * q[2]);
    const int t = cd.tag[c];
    if (t) {
        const BoxDev& b = cd.box[t - 1];
        g.u = -P.u; g.v = -P.v; g.w = -P.w;
        g.k = P.k; g.om = P.om;
        g.T = thermal_ghost<C>(b.thermal, b.T_value, b.T_value2f, b.q_coef, cd.h[axis], b.qhf[axis], P.T);
        return FK_WALL;
    }
    g = load_state<S, C>(st, c);
    return FK_INTERIOR;
}

// A regular cell: fluid, with a fluid in-grid neighbour across every face of an active axis (all
// level-0 face codes of those axes 0), so its neighbours need no ghost.  Its neighbours are read
// by plain loads at coordinates clamped into the grid: for a regular cell the clamp never acts,
// and whatever a code says, no load leaves the arrays.
__device__ __forceinline__ bool regular_cell(const CaseDev& cd, int c) {
    return (__ldg(cd.nbf0 + c) & cd.regular_mask) == 0u;
}

template <class S, class C>
__device__ __forceinline__ St<C> regular_neighbour(const CaseDev& cd, const StatePtrs& st, int i, int j, int k, int axis,
                                                   int side) {
    int q[3] = {i, j, k};
    q[axis] = min(max(q[axis] + side, 0), cd.n[axis] - 1);
    return load_state<S, C>(st, q[0] + cd.n[0] * (q[1] + cd.n[1] * q[2]));
}

// a / b: the IEEE quotient in FP64 (the parity path); in FP32 the fast quotient
// (__fdividef: within 2 ulp for |b| in [2^-126, 2^126], which every use below
// keeps), its error far inside the FP32 fields' 1e-4 bound
template <class C> __device__ __forceinline__ C qdiv(C a, C b) { return a / b; }
template <> __device__ __forceinline__ float qdiv<float>(float a, float b) { return __fdividef(a, b); }

template <class C>
__device__ __forceinline__ C omega_safe(C om) { return om > (C)kEpsOmega ? om : (C)kEpsOmega; }

// Re_t (Eq. Re_t) and alpha* (Eq. a_star); nu_t = alpha* k / omega (Eq. ko_turb_diff)
template <class C>
__device__ __forceinline__ C re_t(C k, C om, C nu) { return qdiv(k, nu * omega_safe(om)); }

template <class C>
__device__ __forceinline__ C alpha_star_of(C ret) {
    const C r = qdiv(ret, (C)kRk);
    return (C)kAlphaStarInf * qdiv((C)kAlphaStar0 + r, (C)1 + r);
}

template <class C>
__device__ __forceinline__ C nut_of(C k, C om, C nu) {
    return qdiv(alpha_star_of(re_t(k, om, nu)) * k, omega_safe(om));
}

// ------------------------------------------------------------------ init
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t n) {
    // output n (0-based) of SplitMix64 seeded with `seed` (Steele, Lea, Flood 2014)
    uint64_t z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <class S>
__global__ void k_init(CaseDev cd, StatePtrs st, double b0, double b1, double b2, double b3, double b4,
                       double b5, uint64_t seed, double eps) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cd.N) return;
    const double base[6] = {b0, b1, b2, b3, b4, b5};
    const int fid[6] = {FVM_U, FVM_V, FVM_W, FVM_T, FVM_K, FVM_OMEGA};
    const bool solid = cd.tag[c] != 0;
    for (int f = 0; f < 6; ++f) {
        double x = base[f];
        if (eps != 0.0) {
            const uint64_t bits = splitmix64_at(seed, (uint64_t)fid[f] * (uint64_t)cd.N + (uint64_t)c);
            const double xi = (double)(bits >> 11) * 0x1.0p-53 * 2.0 - 1.0;
            x = x * (1.0 + eps * xi);
        }
        ((S*)st.f[f])[c] = from_c<S, double>(solid ? 0.0 : x);
    }
}

// ------------------------------------------------------------------ dt
// rate = sum_active (|u_a| / h_a + 2 Gamma / h_a^2), Gamma = max(nu + nu_t, alpha + nu_t / Pr_t);
// the block maxima go to dt_state[3] (as ordered bits of a non-negative double)
template <class S, class C>
struct RateMaxK {
    static constexpr int kThreads = 256;
    __device__ bool live() const { return true; }
    CaseDev cd;
    StatePtrs st;
    unsigned long long* rate_bits;
    __device__ void run(const BlockAt& at) const;
};

template <class S, class C>
__device__ void RateMaxK<S, C>::run(const BlockAt& at) const {
    const int64_t c = (int64_t)at.b.x * blockDim.x + threadIdx.x;
    C lam = (C)0;   // the warp maximum in the compute type, the block's in FP64
    if (c < cd.N && cd.tag[c] == 0) {
        const C u[3] = {to_c<C>(ldg((const S*)st.f[0] + c)), to_c<C>(ldg((const S*)st.f[1] + c)),
                        to_c<C>(ldg((const S*)st.f[2] + c))};
        const C k = to_c<C>(ldg((const S*)st.f[4] + c));
        const C om = to_c<C>(ldg((const S*)st.f[5] + c));
        const C nut = nut_of<C>(k, om, prm<C>(cd.nu, cd.f.nu));
        const C g1 = prm<C>(cd.nu, cd.f.nu) + nut, g2 = prm<C>(cd.alpha, cd.f.alpha) + nut * prm<C>(cd.inv_Prt, cd.f.inv_Prt);
        const C gam = g1 > g2 ? g1 : g2;
        C l = (C)0;
        for (int a = 0; a < 3; ++a)
            if (cd.active[a]) l += fabs(u[a]) * prm<C>(cd.inv_h[a], cd.f.inv_h[a]) + (C)2 * gam * prm<C>(cd.inv_h2[a], cd.f.inv_h2[a]);
        lam = l == l ? l : (C)INFINITY;   // NaN -> +inf
    }
    __shared__ double red[kThreads / 32];
    for (int off = 16; off > 0; off >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)lam;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        atomicMax(rate_bits, (unsigned long long)__double_as_longlong(m));
    }
}

// dt_state: [0] dt, [1] dt/2, [2] simulated time, [3] rate bits (reset here)
struct DtFinalizeK {
    static constexpr int kThreads = 1;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    __device__ bool live() const { return true; }
    double dt0, cfl;
    int adapt;
    double* dt_state;
    __device__ void run(const BlockAt&) const {
        unsigned long long* bits = (unsigned long long*)(dt_state + 3);
        const double lam = __longlong_as_double((long long)*bits);
        double dt = dt0;
        if (adapt && lam > 0.0) {
            const double cap = cfl / lam;
            dt = cap < dt0 ? cap : dt0;
        }
        dt_state[0] = dt;
        dt_state[1] = 0.5 * dt;
        dt_state[2] += dt;
        ((float*)(dt_state + 4))[0] = (float)dt;
        ((float*)(dt_state + 4))[1] = (float)(0.5 * dt);
        *bits = 0ull;
    }
};

// ------------------------------------------------------------------ destruction
template <class S, class C>
struct DestructionK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    static constexpr int kMinBlocks = sizeof(C) == 4 ? 3 : 1;   // FP32: at most 85 registers
    static constexpr int kMinBlocksMany = sizeof(C) == 4 ? 4 : 1;   // batched FP32: at most 64
    __device__ bool live() const { return true; }
    CaseDev cd;
    StatePtrs in;
    S* k_out;
    S* om_out;
    const double* dt_state;
    S* nut_out;   // nu_t of the updated k, omega (read by the explicit stage), or null
    S* b_out;     // the pressure right-hand side b = -div(u)/dt of the same velocity (Eq. pc_residual), or null
    __device__ void run(const BlockAt& at) const;
    __device__ void cell(int i, int j, int k) const;
};

// k and omega after the semi-implicit destruction half step dt (Eqs. k_des_step, o_des_step) of
// one cell, from its velocity gradient gu[i][a] = d u_i / d x_a and gkw = grad k . grad omega
template <class C>
__device__ __forceinline__ void des_update(const C gu[3][3], C gkw, C k, C om, C nu, C dt, C& knew, C& omnew) {
    const C oms = omega_safe(om);
    // k: chi_k, f_beta*, beta* (Eqs. k_des, beta_star)
    const C chik = gkw / (oms * oms * oms);
    C fbs = (C)1;
    if (chik > (C)0) {
        if (chik > (C)1e8) fbs = (C)(680.0 / 400.0);
        else {
            const C c2 = chik * chik;
            fbs = qdiv((C)1 + (C)680 * c2, (C)1 + (C)400 * c2);
        }
    }
    const C x = qdiv(re_t(k, om, nu), (C)kRbeta);
    C bstar;
    if (x > (C)1e4) bstar = (C)kBetaStarInf;
    else {
        const C x2 = x * x;
        const C x4 = x2 * x2;
        bstar = (C)kBetaStarInf * qdiv((C)(4.0 / 15.0) + x4, (C)1 + x4);
    }
    knew = qdiv(k, (C)1 + dt * bstar * fbs * om);
    // omega: chi_omega = |Omega_ij Omega_jk S_ki| / (beta*_inf omega)^3, f_beta (Eq. o_des).  With
    // the rotation vector w (Omega v = w x v), Omega Omega = w w^T - |w|^2 I, so the trace is
    // w^T S w - |w|^2 tr(S)
    const C w1 = (C)0.5 * (gu[2][1] - gu[1][2]), w2 = (C)0.5 * (gu[0][2] - gu[2][0]);
    const C w3 = (C)0.5 * (gu[1][0] - gu[0][1]);
    const C s01 = (C)0.5 * (gu[0][1] + gu[1][0]), s02 = (C)0.5 * (gu[0][2] + gu[2][0]);
    const C s12 = (C)0.5 * (gu[1][2] + gu[2][1]);
    const C wsw = w1 * w1 * gu[0][0] + w2 * w2 * gu[1][1] + w3 * w3 * gu[2][2] +
                  (C)2 * (w1 * w2 * s01 + w1 * w3 * s02 + w2 * w3 * s12);
    const C tr = wsw - (w1 * w1 + w2 * w2 + w3 * w3) * (gu[0][0] + gu[1][1] + gu[2][2]);
    const C bo = (C)kBetaStarInf * oms;
    const C chiw = fabs(tr / (bo * bo * bo));
    const C fb = chiw > (C)1e30 ? (C)(70.0 / 80.0) : qdiv((C)1 + (C)70 * chiw, (C)1 + (C)80 * chiw);
    omnew = qdiv(om, (C)1 + dt * (C)kBeta * fb * om);
}

template <class S, class C>
__device__ void DestructionK<S, C>::run(const BlockAt& at) const {
    int i, j, k;
    if (cell3(cd, at, i, j, k)) cell(i, j, k);
}

template <class S, class C>
__device__ void DestructionK<S, C>::cell(int i, int j, int k) const {
    const int c = i + cd.n[0] * (j + cd.n[1] * k);
    const St<C> P = load_state<S, C>(in, c);
    if (cd.tag[c]) {
        k_out[c] = from_c<S, C>(P.k);
        om_out[c] = from_c<S, C>(P.om);
        if (nut_out) nut_out[c] = from_c<S, C>((C)0);
        if (b_out) b_out[c] = from_c<S, C>((C)0);
        return;
    }
    const bool reg = regular_cell(cd, c);
    // cell gradients L_j * D_j * BC_j(phi) of u, v, w, k, omega, and the face-velocity divergence
    C gu[3][3], gk[3], gw[3];
    C div = (C)0;
    for (int a = 0; a < 3; ++a) {
        if (!cd.active[a]) {
            gu[0][a] = gu[1][a] = gu[2][a] = (C)0;
            gk[a] = gw[a] = (C)0;
            continue;
        }
        St<C> L, R;
        if (reg) {
            L = regular_neighbour<S, C>(cd, in, i, j, k, a, -1);
            R = regular_neighbour<S, C>(cd, in, i, j, k, a, +1);
        } else {
            neighbour<S, C>(cd, in, i, j, k, a, -1, P, L);
            neighbour<S, C>(cd, in, i, j, k, a, +1, P, R);
        }
        const C ih = prm<C>(cd.inv_h[a], cd.f.inv_h[a]);
        gu[0][a] = (C)0.5 * ((R.u - P.u) * ih + (P.u - L.u) * ih);
        gu[1][a] = (C)0.5 * ((R.v - P.v) * ih + (P.v - L.v) * ih);
        gu[2][a] = (C)0.5 * ((R.w - P.w) * ih + (P.w - L.w) * ih);
        gk[a] = (C)0.5 * ((R.k - P.k) * ih + (P.k - L.k) * ih);
        gw[a] = (C)0.5 * ((R.om - P.om) * ih + (P.om - L.om) * ih);
        if (b_out) {
            const C ue = (C)0.5 * (vcomp(P, a) + vcomp(R, a));
            const C uw = (C)0.5 * (vcomp(L, a) + vcomp(P, a));
            div += (ue - uw) * ih;
        }
    }
    if (b_out) b_out[c] = from_c<S, C>(-div / dt_of<C>(dt_state, 0));
    const C nu = prm<C>(cd.nu, cd.f.nu);
    C knew, omnew;
    des_update<C>(gu, gk[0] * gw[0] + gk[1] * gw[1] + gk[2] * gw[2], P.k, P.om, nu, dt_of<C>(dt_state, 1), knew,
                  omnew);
    k_out[c] = from_c<S, C>(knew);
    om_out[c] = from_c<S, C>(omnew);
    if (nut_out) nut_out[c] = from_c<S, C>(nut_of(knew, omnew, nu));
}

// ------------------------------------------------------------------ four-cell form (FP32 fields)
// The projection with four consecutive x cells per thread, in the multigrid vector kernels'
// layout: a block of 32 x 8 threads, each warp covering row segments of 4 * LR cells (LR = 2^lrl
// lanes, the widest segment of 128, 64, 32 or 16 cells that divides nx), x neighbours passed
// between the lanes of a segment by shuffles and loaded by its two end lanes, rows j +- 1 and
// planes k +- 1 read as 128-bit loads.  Every load takes coordinates clamped into the grid.
// Every thread computes all four cells from the values in registers (so the shuffles see all
// lanes); a regular cell (fluid, every level-0 face code of an active axis 0) keeps that result,
// since its neighbours are the in-grid cells the registers hold, and any other cell of the group
// runs the one-cell code instead.  A collapsed axis (n = 1) clamps both neighbours to the cell
// itself, so its differences vanish as in the one-cell code.  Needs nx % 4 = 0.  (The same form
// of the destruction and explicit kernels measured slower than their one-cell forms on the
// 512 x 256 x 128 room: their cost is the closure arithmetic, which four cells per thread do not
// reduce, while a warp holding a row's end cell waits for that cell's one-cell code.)
constexpr int VX = 32, VY = 8;

struct Idx4 {
    int c, ym, yp, zm, zp, xl, xr;   // the group's first cell, the rows j -+ 1 and planes k -+ 1, the x end cells
    int LR;
    bool lo, hi;                     // the segment's first / last lane
};

struct Grp4 {
    int i, j, k;   // the group's first cell (coordinates clamped into the grid)
    bool in;       // the thread's group lies in the grid
    Idx4 x;
};

__device__ __forceinline__ Grp4 group4(const int n[3], const BlockAt& at, int lrl) {
    Grp4 g;
    const int nx = n[0], ny = n[1], nz = n[2];
    const int LR = 1 << lrl, lane = threadIdx.x & (LR - 1), sub = threadIdx.x >> lrl;
    const int i4 = (int)at.b.x * (4 * LR) + lane * 4;
    const int j = (((int)at.b.y * VY + (int)threadIdx.y) << (5 - lrl)) + sub;
    const int k = min((int)at.b.z, nz - 1);
    g.in = i4 < nx && j < ny && (int)at.b.z < nz;
    g.i = min(i4, nx - 4);
    g.j = min(j, ny - 1);
    g.k = k;
    const int sy = nx, sz = nx * ny;
    const int row = sy * g.j + sz * k;
    g.x.c = g.i + row;
    g.x.ym = g.i + sy * max(g.j - 1, 0) + sz * k;
    g.x.yp = g.i + sy * min(g.j + 1, ny - 1) + sz * k;
    g.x.zm = g.i + sy * g.j + sz * max(k - 1, 0);
    g.x.zp = g.i + sy * g.j + sz * min(k + 1, nz - 1);
    g.x.xl = max(g.i - 1, 0) + row;
    g.x.xr = min(g.i + 4, nx - 1) + row;
    g.x.LR = LR;
    g.x.lo = lane == 0;
    g.x.hi = lane == LR - 1;
    return g;
}

__device__ __forceinline__ float4 ld4(const float* p, int c) { return __ldg(reinterpret_cast<const float4*>(p + c)); }
__device__ __forceinline__ void st4(float* p, int c, const float v[4]) {
    *reinterpret_cast<float4*>(p + c) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void un4(const float4& v, float o[4]) {
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}

// which of the group's four cells are regular (bit t: cell t); 15 when all are
__device__ __forceinline__ uint32_t regular4(const CaseDev& cd, int c) {
    const uint2 w = __ldg(reinterpret_cast<const uint2*>(cd.nbf0 + c));
    const uint32_t m = cd.regular_mask;
    return ((w.x & m) == 0u ? 1u : 0u) | (((w.x >> 16) & m) == 0u ? 2u : 0u) | ((w.y & m) == 0u ? 4u : 0u) |
           (((w.y >> 16) & m) == 0u ? 8u : 0u);
}

// ------------------------------------------------------------------ explicit stage
// Flux of (u, v, w, T, k, omega) through one face with states L (lower) and R (upper):
// -phi_upwind u_face + Gamma (phi_R - phi_L) / h, and -(2/3) k_face on the
// momentum component along the face normal.
template <class C>
__device__ __forceinline__ void face_flux(const CaseDev& cd, int a, const St<C>& L, const St<C>& R, C nut_f,
                                          C fl[6]) {
    const C uf = (C)0.5 * (vcomp(L, a) + vcomp(R, a));
    const bool pos = uf >= (C)0;
    const C ih = prm<C>(cd.inv_h[a], cd.f.inv_h[a]);
    const C nu = prm<C>(cd.nu, cd.f.nu);
    const C gm = nu + nut_f;
    const C gT = prm<C>(cd.alpha, cd.f.alpha) + nut_f * prm<C>(cd.inv_Prt, cd.f.inv_Prt);
    const C gk = nu + nut_f * prm<C>(cd.inv_sigk, cd.f.inv_sigk);
    const C gw = nu + nut_f * prm<C>(cd.inv_sigw, cd.f.inv_sigw);
    fl[0] = -((pos ? L.u : R.u) * uf) + gm * (R.u - L.u) * ih;
    fl[1] = -((pos ? L.v : R.v) * uf) + gm * (R.v - L.v) * ih;
    fl[2] = -((pos ? L.w : R.w) * uf) + gm * (R.w - L.w) * ih;
    fl[3] = -((pos ? L.T : R.T) * uf) + gT * (R.T - L.T) * ih;
    fl[4] = -((pos ? L.k : R.k) * uf) + gk * (R.k - L.k) * ih;
    fl[5] = -((pos ? L.om : R.om) * uf) + gw * (R.om - L.om) * ih;
    fl[a] -= (C)(2.0 / 3.0) * ((C)0.5 * (L.k + R.k));
}

// face nu_t: 0 on walls, the mean of the two cells inside, the cell's own on other faces
template <class C, class N>
__device__ __forceinline__ C face_nut(int kind, C nutP, N nut_nb) {
    if (kind == FK_WALL) return (C)0;
    if (kind == FK_INTERIOR) return (C)0.5 * (nutP + nut_nb());
    return nutP;
}

template <class S, class C, bool kBlend>
struct ExplicitK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    static constexpr int kMinBlocks = sizeof(C) == 4 ? 4 : 1;   // FP32: at most 64 registers
    __device__ bool live() const { return true; }
    CaseDev cd;
    StatePtrs in, out;
    const double* dt_state;
    const S* nut;   // nu_t of the input state (written by the destruction half step), or null: computed here
    // kBlend: a later stage of the Shu-Osher Runge-Kutta schemes, out = wb base + ws E(in), where E
    // is the forward-Euler update (clamps included) and base the stage-0 state (may alias out: each
    // thread reads its own base cell before writing it); wall omega is set after the combination.
    // Otherwise plain forward Euler (base and the weights unused).
    StatePtrs base;
    double wb, ws;
    float wbf, wsf;
    __device__ void run(const BlockAt& at) const;
    __device__ void cell(int i, int j, int k) const;
};

// The cell update of the explicit stage from the summed face fluxes rhs (Algorithm 2): the
// production of k and omega (Eqs. k_gen, o_gen, a) with S2 = 2 S_ij S_ij, Boussinesq buoyancy
// -g beta_T (T - T_ref), the forward-Euler step dt and the lower bounds of k and omega
template <class C>
__device__ __forceinline__ void exp_update(const CaseDev& cd, const St<C>& P, C nutP, C S2, C rhs[6], C dt, C o[6]) {
    const C nu = prm<C>(cd.nu, cd.f.nu);
    const C Gk = nutP * S2;
    const C ret = re_t(P.k, P.om, nu);
    const C rw = qdiv(ret, (C)kRw);
    const C alpha = qdiv((C)kAlphaInf, alpha_star_of(ret)) * qdiv((C)kAlpha0 + rw, (C)1 + rw);
    rhs[4] += Gk;
    rhs[5] += qdiv(alpha * P.om, P.k) * Gk;
    const C dT = P.T - prm<C>(cd.T_ref, cd.f.T_ref);
    rhs[0] += prm<C>(cd.gb[0], cd.f.gb[0]) * dT;
    rhs[1] += prm<C>(cd.gb[1], cd.f.gb[1]) * dT;
    rhs[2] += prm<C>(cd.gb[2], cd.f.gb[2]) * dT;
    o[0] = P.u + dt * rhs[0];
    o[1] = P.v + dt * rhs[1];
    o[2] = P.w + dt * rhs[2];
    o[3] = P.T + dt * rhs[3];
    const C kn = P.k + dt * rhs[4];
    const C on = P.om + dt * rhs[5];
    o[4] = kn > (C)kKMin ? kn : (C)kKMin;
    o[5] = on > (C)kOmegaMin ? on : (C)kOmegaMin;
}

template <class S, class C, bool kBlend>
__device__ void ExplicitK<S, C, kBlend>::run(const BlockAt& at) const {
    int i, j, k;
    if (cell3(cd, at, i, j, k)) cell(i, j, k);
}

template <class S, class C, bool kBlend>
__device__ void ExplicitK<S, C, kBlend>::cell(int i, int j, int k) const {
    const int c = i + cd.n[0] * (j + cd.n[1] * k);
    const St<C> P = load_state<S, C>(in, c);
    S* o[6];
    for (int f = 0; f < 6; ++f) o[f] = (S*)out.f[f];
    if (cd.tag[c]) {
        o[0][c] = from_c<S, C>(P.u); o[1][c] = from_c<S, C>(P.v); o[2][c] = from_c<S, C>(P.w);
        o[3][c] = from_c<S, C>(P.T); o[4][c] = from_c<S, C>(P.k); o[5][c] = from_c<S, C>(P.om);
        return;
    }
    const C nu = prm<C>(cd.nu, cd.f.nu);
    const S* const nutf = nut;
    const C nutP = nutf ? to_c<C>(ldg(nutf + c)) : nut_of(P.k, P.om, nu);
    const int stride[3] = {1, cd.n[0], cd.n[0] * cd.n[1]};
    const bool reg = regular_cell(cd, c);
    C rhs[6] = {(C)0, (C)0, (C)0, (C)0, (C)0, (C)0};
    C gu[3][3];
    C omw = (C)0;
    for (int a = 0; a < 3; ++a) {
        if (!cd.active[a]) {
            gu[0][a] = gu[1][a] = gu[2][a] = (C)0;
            continue;
        }
        St<C> L, R;
        int kl = FK_INTERIOR, kr = FK_INTERIOR;
        if (reg) {
            L = regular_neighbour<S, C>(cd, in, i, j, k, a, -1);
            R = regular_neighbour<S, C>(cd, in, i, j, k, a, +1);
        } else {
            kl = neighbour<S, C>(cd, in, i, j, k, a, -1, P, L);
            kr = neighbour<S, C>(cd, in, i, j, k, a, +1, P, R);
        }
        C fw[6], fe[6];
        // (an interior face's neighbour index, its coordinate clamped into the grid like every load)
        const int q = a == 0 ? i : (a == 1 ? j : k);
        const int cm = c - (q > 0 ? stride[a] : 0), cp = c + (q < cd.n[a] - 1 ? stride[a] : 0);
        auto nb_nut = [&](int side, const St<C>& g) {
            return [&, side]() { return nutf ? to_c<C>(ldg(nutf + (side < 0 ? cm : cp))) : nut_of(g.k, g.om, nu); };
        };
        face_flux(cd, a, L, P, face_nut<C>(kl, nutP, nb_nut(-1, L)), fw);
        face_flux(cd, a, P, R, face_nut<C>(kr, nutP, nb_nut(+1, R)), fe);
        const C ih = prm<C>(cd.inv_h[a], cd.f.inv_h[a]);
        for (int f = 0; f < 6; ++f) rhs[f] += (fe[f] - fw[f]) * ih;
        gu[0][a] = (C)0.5 * ((R.u - P.u) * ih + (P.u - L.u) * ih);
        gu[1][a] = (C)0.5 * ((R.v - P.v) * ih + (P.v - L.v) * ih);
        gu[2][a] = (C)0.5 * ((R.w - P.w) * ih + (P.w - L.w) * ih);
        if (kl == FK_WALL || kr == FK_WALL) {
            const C ow = prm<C>(cd.om_wall[a], cd.f.om_wall[a]);
            omw = ow > omw ? ow : omw;
        }
    }
    // S^2 = 2 S_ij S_ij
    C S2 = (C)0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const C s = (C)0.5 * (gu[a][b] + gu[b][a]);
            S2 += s * s;
        }
    S2 = (C)2 * S2;
    C nw[6];
    exp_update<C>(cd, P, nutP, S2, rhs, dt_of<C>(dt_state, 0), nw);
    if constexpr (kBlend) {
        const C a = prm<C>(wb, wbf), b = prm<C>(ws, wsf);
        for (int f = 0; f < 6; ++f) nw[f] = a * to_c<C>(((const S*)base.f[f])[c]) + b * nw[f];
    }
    if (omw > (C)0) nw[5] = omw;
    for (int f = 0; f < 6; ++f) o[f][c] = from_c<S, C>(nw[f]);
}

// ------------------------------------------------------------------ pressure RHS
template <class S, class C>
struct RhsK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    __device__ bool live() const { return true; }
    CaseDev cd;
    StatePtrs in;
    S* b;
    const double* dt_state;
    __device__ void run(const BlockAt& at) const;
};

template <class S, class C>
__device__ void RhsK<S, C>::run(const BlockAt& at) const {
    int i, j, k;
    if (!cell3(cd, at, i, j, k)) return;
    const int c = i + cd.n[0] * (j + cd.n[1] * k);
    if (cd.tag[c]) {
        b[c] = from_c<S, C>((C)0);
        return;
    }
    const St<C> P = load_state<S, C>(in, c);
    C div = (C)0;
    for (int a = 0; a < 3; ++a) {
        if (!cd.active[a]) continue;
        St<C> L, R;
        neighbour<S, C>(cd, in, i, j, k, a, -1, P, L);
        neighbour<S, C>(cd, in, i, j, k, a, +1, P, R);
        const C ue = (C)0.5 * (vcomp(P, a) + vcomp(R, a));
        const C uw = (C)0.5 * (vcomp(L, a) + vcomp(P, a));
        div += (ue - uw) * prm<C>(cd.inv_h[a], cd.f.inv_h[a]);
    }
    b[c] = from_c<S, C>(-div / dt_of<C>(dt_state, 0));
}

// ------------------------------------------------------------------ projection
// pressure across a face: neighbour, Neumann ghost (walls, inlets, solids) or -p (outlets)
__device__ __forceinline__ double p_across(const LevelDev& L, const double* p, uint32_t f, int c, int a,
                                           int side, double pP) {
    const uint32_t code = (f >> (2 * (2 * a + (side > 0 ? 1 : 0)))) & 3u;
    if (code == 1u) return pP;
    if (code == 2u) return -pP;
    const int stride = a == 0 ? 1 : (a == 1 ? L.n[0] : L.n[0] * L.n[1]);
    return __ldg(p + c + side * stride);
}

// the same in float-float, p held as double-float pairs (P: the cell's own value)
__device__ __forceinline__ FF p_across_ff(const LevelDev& L, const double* p, uint32_t f, int c, int a, int side,
                                          FF P) {
    const uint32_t code = (f >> (2 * (2 * a + (side > 0 ? 1 : 0)))) & 3u;
    if (code == 1u) return P;
    if (code == 2u) return FF{-P.h, -P.l};
    const int stride = a == 0 ? 1 : (a == 1 ? L.n[0] : L.n[0] * L.n[1]);
    return pp_load(p, c + side * stride);
}

template <class S, class C>
struct ProjectK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    __device__ bool live() const { return true; }
    CaseDev cd;
    LevelDev L0;
    StatePtrs in, out;
    const double* p;
    const double* dt_state;
    __device__ void run(const BlockAt& at) const;
    __device__ void cell(int i, int j, int k) const;
};

template <class S, class C>
__device__ void ProjectK<S, C>::run(const BlockAt& at) const {
    int i, j, k;
    if (cell3(cd, at, i, j, k)) cell(i, j, k);
}

template <class S, class C>
__device__ void ProjectK<S, C>::cell(int i, int j, int k) const {
    const int c = i + cd.n[0] * (j + cd.n[1] * k);
    S* o[3] = {(S*)out.f[0], (S*)out.f[1], (S*)out.f[2]};
    const S* q[3] = {(const S*)in.f[0], (const S*)in.f[1], (const S*)in.f[2]};
    if (cd.tag[c]) {
        for (int a = 0; a < 3; ++a) o[a][c] = q[a][c];
        return;
    }
    const uint32_t f = L0.nbf[c];
    const C dt = dt_of<C>(dt_state, 0);
    if constexpr (sizeof(C) == 8) {
        const double pP = __ldg(p + c);
        for (int a = 0; a < 3; ++a) {
            C g = (C)0;
            if (cd.active[a]) {
                // differences of the FP64 pressure are taken in FP64, then rounded
                const double pl = p_across(L0, p, f, c, a, -1, pP);
                const double pr = p_across(L0, p, f, c, a, +1, pP);
                const double ih = cd.inv_h[a];
                g = (C)(0.5 * ((pr - pP) * ih + (pP - pl) * ih));
            }
            o[a][c] = from_c<S, C>(to_c<C>(ldg(q[a] + c)) - dt * g);
        }
    } else {
        // FP32 fields: the pressure differences in float-float (p as double-float pairs), rounded once
        const FF P = pp_load(p, c);
        for (int a = 0; a < 3; ++a) {
            C g = (C)0;
            if (cd.active[a]) {
                const FF pl = p_across_ff(L0, p, f, c, a, -1, P);
                const FF pr = p_across_ff(L0, p, f, c, a, +1, P);
                const float ih = cd.f.inv_h[a];
                g = 0.5f * (ff_diff(pr, P) * ih + ff_diff(P, pl) * ih);
            }
            o[a][c] = from_c<S, C>(to_c<C>(ldg(q[a] + c)) - dt * g);
        }
    }
}

// The projection, four cells per thread (FP32 fields, p as double-float pairs): the layout of
// the other four-cell forms, the pairs of the x neighbours passed between lanes
struct ProjectVK {
    static constexpr int kThreads = VX * VY;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    static constexpr int kMinBlocks = 4;
    __device__ bool live() const { return true; }
    ProjectK<float, float> s;   // the arguments; its one-cell code serves the irregular groups
    int lrl;
    __device__ void run(const BlockAt& at) const;
};

// the pairs of four consecutive cells from c (16-byte aligned: c % 4 = 0)
__device__ __forceinline__ void pp4(const double* p, int c, FF o[4]) {
    const float4* q = reinterpret_cast<const float4*>(p + c);
    const float4 a = __ldg(q), b = __ldg(q + 1);
    o[0] = {a.x, a.y};
    o[1] = {a.z, a.w};
    o[2] = {b.x, b.y};
    o[3] = {b.z, b.w};
}

__device__ void ProjectVK::run(const BlockAt& at) const {
    const CaseDev& cd = s.cd;
    const Grp4 g = group4(cd.n, at, lrl);
    const Idx4& x = g.x;
    FF P[4];
    pp4(s.p, x.c, P);
    float grad[3][4];
    {
        FF left, right;
        left.h = __shfl_up_sync(0xffffffffu, P[3].h, 1, x.LR);
        left.l = __shfl_up_sync(0xffffffffu, P[3].l, 1, x.LR);
        right.h = __shfl_down_sync(0xffffffffu, P[0].h, 1, x.LR);
        right.l = __shfl_down_sync(0xffffffffu, P[0].l, 1, x.LR);
        if (x.lo) left = pp_load(s.p, x.xl);
        if (x.hi) right = pp_load(s.p, x.xr);
        const float ih = cd.f.inv_h[0];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const FF L = t == 0 ? left : P[t - 1], R = t == 3 ? right : P[t + 1];
            grad[0][t] = 0.5f * (ff_diff(R, P[t]) * ih + ff_diff(P[t], L) * ih);
        }
    }
#pragma unroll
    for (int a = 1; a < 3; ++a) {
        FF L[4], R[4];
        pp4(s.p, a == 1 ? x.ym : x.zm, L);
        pp4(s.p, a == 1 ? x.yp : x.zp, R);
        const float ih = cd.f.inv_h[a];
#pragma unroll
        for (int t = 0; t < 4; ++t) grad[a][t] = 0.5f * (ff_diff(R[t], P[t]) * ih + ff_diff(P[t], L[t]) * ih);
    }
    if (!g.in) return;
    const uint32_t reg = regular4(cd, x.c);
    const float dt = dt_of<float>(s.dt_state, 0);
    float v[3][4];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        un4(ld4((const float*)s.in.f[a], x.c), v[a]);
#pragma unroll
        for (int t = 0; t < 4; ++t) v[a][t] = v[a][t] - dt * (cd.active[a] ? grad[a][t] : 0.f);
    }
    if (reg == 15u) {
#pragma unroll
        for (int a = 0; a < 3; ++a) st4((float*)s.out.f[a], x.c, v[a]);
        return;
    }
#pragma unroll 1
    for (int t = 0; t < 4; ++t) {
        if (reg & (1u << t)) {
#pragma unroll
            for (int a = 0; a < 3; ++a) ((float*)s.out.f[a])[x.c + t] = v[a][t];
        } else {
            s.cell(g.i + t, g.j, g.k);
        }
    }
}

// ------------------------------------------------------------------ projection adjoint
// Transposes of the two local maps of the projection, for the vector-Jacobian
// product of u* -> (u^{n+1}, p) (FP64 cases).  With the pressure face codes of
// level 0 (0 fluid neighbour, 1 zero-gradient ghost, 2 zero-value ghost at an
// outlet):
//   projection  out_a(c) = -dt/(2h) (p_{c+} - p_{c-}) on fluid cells, a ghost
//               p_{c+-} = s p_c with s = +1 (code 1) or -1 (code 2);
//   rhs         b(c) = -1/(dt h) sum_a (uf_a(c+1/2) - uf_a(c-1/2)), uf the mean of
//               the two cells across a fluid face, the cell's own value across an
//               outlet face (mirror ghost), 0 across walls, inlets and obstacles
//               (odd ghosts; the inlet's constant drops out of the Jacobian).
// AdjGradK forms q = pbar + (d out / d p)^T ybar; AdjRhsK forms
// xbar = ybar + (d b / d u*)^T lambda.  Solid cells: q = 0 (their p is fixed at
// 0), xbar = ybar (the projection copies their velocities).
__device__ __forceinline__ uint32_t face_code(uint32_t f, int a, int side) {
    return (f >> (2 * (2 * a + (side > 0 ? 1 : 0)))) & 3u;
}

struct AdjGradK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    __device__ bool live() const { return true; }
    CaseDev cd;
    LevelDev L0;
    const double* ybar;   // ubar, vbar, wbar, pbar (4 N)
    double* q;
    double dt;
    __device__ void run(const BlockAt& at) const;
};

__device__ void AdjGradK::run(const BlockAt& at) const {
    int i, j, k;
    if (!cell3(cd, at, i, j, k)) return;
    const int c = i + cd.n[0] * (j + cd.n[1] * k);
    if (cd.tag[c]) {
        q[c] = 0.0;
        return;
    }
    const int64_t N = cd.N;
    const uint32_t f = L0.nbf[c];
    double acc = ybar[3 * N + c];
    for (int a = 0; a < 3; ++a) {
        if (!cd.active[a]) continue;
        const double* ya = ybar + a * N;
        const int stride = a == 0 ? 1 : (a == 1 ? cd.n[0] : cd.n[0] * cd.n[1]);
        const double coef = dt * 0.5 * cd.inv_h[a];
        const uint32_t cm = face_code(f, a, -1), cp = face_code(f, a, +1);
        const double sm = cm == 1u ? 1.0 : (cm == 2u ? -1.0 : 0.0);
        const double sp = cp == 1u ? 1.0 : (cp == 2u ? -1.0 : 0.0);
        acc += coef * (sm - sp) * ya[c];
        if (cm == 0u) acc -= coef * ya[c - stride];
        if (cp == 0u) acc += coef * ya[c + stride];
    }
    q[c] = acc;
}

struct AdjRhsK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    __device__ bool live() const { return true; }
    CaseDev cd;
    LevelDev L0;
    const double* ybar;     // ubar, vbar, wbar (first 3 N used)
    const double* lambda;   // A^{-T} q
    double* xbar;           // 3 N
    double ihdt[3];         // 1 / (h_a dt), formed on the host (no FP64 division per cell)
    __device__ void run(const BlockAt& at) const;
};

__device__ void AdjRhsK::run(const BlockAt& at) const {
    int i, j, k;
    if (!cell3(cd, at, i, j, k)) return;
    const int c = i + cd.n[0] * (j + cd.n[1] * k);
    const int64_t N = cd.N;
    if (cd.tag[c]) {
        for (int a = 0; a < 3; ++a) xbar[a * N + c] = ybar[a * N + c];
        return;
    }
    const uint32_t f = L0.nbf[c];
    const double lc = lambda[c];
    for (int a = 0; a < 3; ++a) {
        double x = ybar[a * N + c];
        if (cd.active[a]) {
            const int stride = a == 0 ? 1 : (a == 1 ? cd.n[0] : cd.n[0] * cd.n[1]);
            const uint32_t cm = face_code(f, a, -1), cp = face_code(f, a, +1);
            double t = 0.0;
            if (cp == 0u) t += 0.5 * (lc - lambda[c + stride]);
            if (cp == 2u) t += lc;
            if (cm == 0u) t -= 0.5 * (lc - lambda[c - stride]);
            if (cm == 2u) t -= lc;
            x -= t * ihdt[a];
        }
        xbar[a * N + c] = x;
    }
}

// ------------------------------------------------------------------ step adjoints (FP64)
// Vector-Jacobian products of the destruction half step and of the forward-Euler
// explicit stage, linearised at a given state (the differentiable step of Section 1,
// with the partial derivatives of Eqs. k_des_step, o_des_step, ko_turb_diff, a_star,
// k_gen, o_gen, beta_star and the fluxes of Algorithms 2 and 3 written out).
// Each runs as two passes: a pointwise pass per cell (partial derivatives, the
// cotangents of the cell gradients) into a scratch array, then a gather per cell of
// everything that reaches it through the stencils.  A ghost of Section 2.7 is
// s * (the cell's own value) + a constant, with s per field and face kind (ghost_sign),
// so a cotangent on a ghost returns to its cell times s.  Solid cells pass their
// cotangents through unchanged.

// the face across side `side` (-1 / +1) of cell (i,j,k) along `axis`: its kind, the
// thermal condition of a wall (domain wall or obstacle) and the neighbour's index
__device__ __forceinline__ int face_kind_of(const CaseDev& cd, int i, int j, int k, int axis, int side, int& thermal,
                                            int& nb) {
    int q[3] = {i, j, k};
    q[axis] += side;
    thermal = FVM_ADIABATIC;
    nb = -1;
    if (q[axis] < 0 || q[axis] >= cd.n[axis]) {
        const int face = 2 * axis + (side > 0 ? 1 : 0);
        const PatchDev& pt = cd.patch[cd.face_patch[face][face_index(axis, i, j, k, cd.n)]];
        thermal = pt.thermal;
        if (pt.kind == FVM_WALL) return FK_WALL;
        if (pt.kind == FVM_INLET) return FK_INLET;
        return pt.kind == FVM_OUTLET ? FK_OUTLET : FK_EMPTY;
    }
    nb = q[0] + cd.n[0] * (q[1] + cd.n[1] * q[2]);
    const int t = cd.tag[nb];
    if (t) {
        thermal = cd.box[t - 1].thermal;
        return FK_WALL;
    }
    return FK_INTERIOR;
}

// s of the ghost s * phi_P + const of field f (0..5 = u, v, w, T, k, omega) across a face
__device__ __forceinline__ double ghost_sign(int f, int kind, int thermal) {
    if (kind == FK_WALL) {
        if (f < 3) return -1.0;                                  // no slip
        if (f == 3) return thermal == FVM_FIXED_T ? -1.0 : 1.0;  // fixed T mirrors; adiabatic, heat flux shift
        return 1.0;                                              // zero gradient of k, omega
    }
    return kind == FK_INLET ? -1.0 : 1.0;                        // inlet mirrors; outlet, empty copy
}

// the cell gradients of (u, v, w, k, omega) at a fluid cell, ghosts included
__device__ __forceinline__ void cell_gradients(const CaseDev& cd, const StatePtrs& in, int i, int j, int k,
                                               const St<double>& P, double (&gu)[3][3], double (&gk)[3],
                                               double (&gw)[3]) {
    for (int a = 0; a < 3; ++a) {
        if (!cd.active[a]) {
            gu[0][a] = gu[1][a] = gu[2][a] = gk[a] = gw[a] = 0.0;
            continue;
        }
        St<double> L, R;
        neighbour<double, double>(cd, in, i, j, k, a, -1, P, L);
        neighbour<double, double>(cd, in, i, j, k, a, +1, P, R);
        const double ih = cd.inv_h[a];
        gu[0][a] = 0.5 * ((R.u - P.u) * ih + (P.u - L.u) * ih);
        gu[1][a] = 0.5 * ((R.v - P.v) * ih + (P.v - L.v) * ih);
        gu[2][a] = 0.5 * ((R.w - P.w) * ih + (P.w - L.w) * ih);
        gk[a] = 0.5 * ((R.k - P.k) * ih + (P.k - L.k) * ih);
        gw[a] = 0.5 * ((R.om - P.om) * ih + (P.om - L.om) * ih);
    }
}

// Transpose of the cell gradient of field f at cell q: gb(m, c) holds the cotangent of
// d phi / d x_m at cell c (component m of the field's gradient); the gradient at a fluid
// cell c along m is (R - L) / (2 h) with R, L the neighbours or their ghosts.
template <class G>
__device__ __forceinline__ double gradient_transpose(const CaseDev& cd, int f, int i, int j, int k, int q, G gb) {
    double acc = 0.0;
    for (int m = 0; m < 3; ++m) {
        if (!cd.active[m]) continue;
        const double c2 = 0.5 * cd.inv_h[m];
        for (int side = -1; side <= 1; side += 2) {
            int thermal, nb;
            const int kind = face_kind_of(cd, i, j, k, m, side, thermal, nb);
            if (kind == FK_INTERIOR) acc += -side * c2 * gb(m, nb);   // q is the neighbour's L (side +) or R (side -)
            else acc += side * ghost_sign(f, kind, thermal) * c2 * gb(m, q);   // q's own ghost
        }
    }
    return acc;
}

// pass 1 of the destruction adjoint: per cell the partial derivatives of (k', omega') and
// the cotangents of the 15 gradient components, gbar = [G (3 x 3, row = velocity
// component), grad k, grad omega] (15 N doubles, component-major)
struct DesAdjAK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;
    __device__ bool live() const { return true; }
    CaseDev cd;
    StatePtrs x;            // the state the step is linearised at
    double dt;              // the half step
    const double* kbar;     // cotangents of k', omega'
    const double* obar;
    double* kout;           // d/dk, d/domega parts of the cotangents of k, omega
    double* oout;
    double* gbar;           // 15 N
    __device__ void run(const BlockAt& at) const;
};

__device__ void DesAdjAK::run(const BlockAt& at) const {
    int i, j, k;
    if (!cell3(cd, at, i, j, k)) return;
    const int c = i + cd.n[0] * (j + cd.n[1] * k);
    const int64_t N = cd.N;
    const double kb = kbar[c], wb = obar[c];
    if (cd.tag[c]) {
        kout[c] = kb;
        oout[c] = wb;
        for (int m = 0; m < 15; ++m) gbar[m * N + c] = 0.0;
        return;
    }
    const St<double> P = load_state<double, double>(x, c);
    double G[3][3], gk[3], gw[3];
    cell_gradients(cd, x, i, j, k, P, G, gk, gw);
    const double nu = cd.nu, kk = P.k, om = P.om;
    const double oms = om > kEpsOmega ? om : kEpsOmega;
    const double doms = om > kEpsOmega ? 1.0 : 0.0;
    // k' = k / Dk, Dk = 1 + dt beta* f_beta* omega
    const double re = kk / (nu * oms), dre_dk = 1.0 / (nu * oms), dre_dom = -re / oms * doms;
    const double x_ = re / kRbeta, x3 = x_ * x_ * x_, x4 = x3 * x_;
    double bs, dbs;
    if (x_ > 1e4) {
        bs = kBetaStarInf;
        dbs = 0.0;
    } else {
        bs = kBetaStarInf * (4.0 / 15.0 + x4) / (1.0 + x4);
        dbs = kBetaStarInf * (11.0 / 15.0) * 4.0 * x3 / (kRbeta * (1.0 + x4) * (1.0 + x4));   // d beta* / d Re_t
    }
    const double dot = gk[0] * gw[0] + gk[1] * gw[1] + gk[2] * gw[2];
    const double o3 = oms * oms * oms;
    const double chik = dot / o3;
    double fbs = 1.0, dfbs = 0.0;
    if (chik > 0.0 && chik <= 1e8) {
        const double c2 = chik * chik, d = 1.0 + 400.0 * c2;
        fbs = (1.0 + 680.0 * c2) / d;
        dfbs = 560.0 * chik / (d * d);
    } else if (chik > 1e8) {
        fbs = 680.0 / 400.0;
    }
    const double Dk = 1.0 + dt * bs * fbs * om;
    const double ck = -kk / (Dk * Dk) * dt;                    // d k' / d (beta* f_beta* omega)
    const double dk_dk = 1.0 / Dk + ck * fbs * om * dbs * dre_dk;
    const double dk_dom = ck * (fbs * om * dbs * dre_dom + bs * om * dfbs * (-3.0 * chik / oms * doms) + bs * fbs);
    const double dk_dg = ck * bs * om * dfbs / o3;             // times grad omega (for grad k) and grad k
    // omega' = omega / Dw, Dw = 1 + dt beta f_beta omega, f_beta of chi_w = |T| / (beta*_inf omega_s)^3
    double S[3][3], O[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            S[a][b] = 0.5 * (G[a][b] + G[b][a]);
            O[a][b] = 0.5 * (G[a][b] - G[b][a]);
        }
    double OO[3][3], SO[3][3], OS[3][3];
    double T = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s1 = 0.0, s2 = 0.0, s3 = 0.0;
            for (int e = 0; e < 3; ++e) {
                s1 += O[a][e] * O[e][b];
                s2 += S[a][e] * O[e][b];
                s3 += O[a][e] * S[e][b];
            }
            OO[a][b] = s1;
            SO[a][b] = s2;
            OS[a][b] = s3;
        }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) T += OO[a][b] * S[b][a];
    const double den = (kBetaStarInf * oms) * (kBetaStarInf * oms) * (kBetaStarInf * oms);
    const double chiw = fabs(T) / den;
    double fb, dfb;
    if (chiw > 1e30) {
        fb = 70.0 / 80.0;
        dfb = 0.0;
    } else {
        const double d = 1.0 + 80.0 * chiw;
        fb = (1.0 + 70.0 * chiw) / d;
        dfb = -10.0 / (d * d);
    }
    const double sgn = T > 0.0 ? 1.0 : (T < 0.0 ? -1.0 : 0.0);
    const double Dw = 1.0 + dt * kBeta * fb * om;
    const double cw = -om / (Dw * Dw) * dt * kBeta;            // d omega' / d (f_beta omega)
    const double dw_dom = 1.0 / Dw + cw * (fb + om * dfb * (-3.0 * chiw / oms * doms));
    const double dwg = cw * om * dfb * sgn / den;              // times d T / d G
    kout[c] = kb * dk_dk;
    oout[c] = kb * dk_dom + wb * dw_dom;
    // d T / d S_ab = (O O)_ba, d T / d O_ab = -(O S + S O)_ab; S, O are the symmetric and
    // antisymmetric parts of G
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const double dS_ab = OO[b][a], dS_ba = OO[a][b];
            const double dO_ab = -(OS[a][b] + SO[a][b]), dO_ba = -(OS[b][a] + SO[b][a]);
            const double dT = 0.5 * (dS_ab + dS_ba) + 0.5 * (dO_ab - dO_ba);
            gbar[(3 * a + b) * N + c] = wb * dwg * dT;
        }
    for (int m = 0; m < 3; ++m) {
        gbar[(9 + m) * N + c] = kb * dk_dg * gw[m];
        gbar[(12 + m) * N + c] = kb * dk_dg * gk[m];
    }
}

// pass 2: the cotangents of (u, v, w, k, omega) before the step: incoming cotangents
// of u, v, w pass through, k and omega take pass 1's parts, and every field gathers
// the transposed gradient stencil of its gbar
struct DesAdjBK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;
    __device__ bool live() const { return true; }
    CaseDev cd;
    const double* ubar_in;   // 3 N: cotangents of u, v, w after the step (unchanged by it)
    const double* kout;
    const double* oout;
    const double* gbar;
    double* out;             // 5 N: u, v, w, k, omega (may alias ubar_in for the first 3 N)
    __device__ void run(const BlockAt& at) const;
};

__device__ void DesAdjBK::run(const BlockAt& at) const {
    int i, j, k;
    if (!cell3(cd, at, i, j, k)) return;
    const int c = i + cd.n[0] * (j + cd.n[1] * k);
    const int64_t N = cd.N;
    const bool fluid = cd.tag[c] == 0;
    double acc[5] = {ubar_in[c], ubar_in[N + c], ubar_in[2 * N + c], kout[c], oout[c]};
    if (fluid) {
        const int field_of[5] = {0, 1, 2, 4, 5};
        for (int v = 0; v < 5; ++v) {
            const double* g = gbar + (size_t)(v < 3 ? 3 * v : (v == 3 ? 9 : 12)) * N;
            acc[v] += gradient_transpose(cd, field_of[v], i, j, k, c,
                                         [&](int m, int q) { return g[(size_t)m * N + q]; });
        }
    }
    for (int v = 0; v < 5; ++v) out[v * N + c] = acc[v];
}

// pass 1 of the explicit-stage adjoint (forward Euler): per fluid cell the cotangents of
// the update's right-hand side, rbar_f = dt ybar_f where the update passes a derivative
// (not for clamped k, omega or the wall omega), the squared strain S^2 and the
// cotangent of the velocity gradient from the production term, Gbar_ab = 4 S_ab S2bar
// (scratch: rbar 6 N, Gbar 9 N, S^2 N)
struct ExpAdjAK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;
    __device__ bool live() const { return true; }
    CaseDev cd;
    StatePtrs x;            // the state the stage is linearised at
    StatePtrs y;            // the stage's output (its clamps decide which cells pass a derivative)
    double dt;
    const double* ybar;     // 6 N: cotangents of the output
    double* rbar;           // 6 N
    double* Gbar;           // 9 N
    double* s2;             // N
    __device__ void run(const BlockAt& at) const;
};

// omega of a fluid cell is set to its wall value after the update when a face of an
// active axis is a wall (domain wall or obstacle)
__device__ __forceinline__ bool wall_cell(const CaseDev& cd, int i, int j, int k) {
    for (int a = 0; a < 3; ++a) {
        if (!cd.active[a]) continue;
        for (int side = -1; side <= 1; side += 2) {
            int thermal, nb;
            if (face_kind_of(cd, i, j, k, a, side, thermal, nb) == FK_WALL) return true;
        }
    }
    return false;
}

__device__ void ExpAdjAK::run(const BlockAt& at) const {
    int i, j, k;
    if (!cell3(cd, at, i, j, k)) return;
    const int c = i + cd.n[0] * (j + cd.n[1] * k);
    const int64_t N = cd.N;
    if (cd.tag[c]) {
        for (int f = 0; f < 6; ++f) rbar[f * N + c] = 0.0;
        for (int m = 0; m < 9; ++m) Gbar[m * N + c] = 0.0;
        s2[c] = 0.0;
        return;
    }
    const double kn = ((const double*)y.f[4])[c], on = ((const double*)y.f[5])[c];
    const bool live_k = kn > kKMin;
    const bool live_o = on > kOmegaMin && !wall_cell(cd, i, j, k);
    for (int f = 0; f < 6; ++f) {
        const bool lv = f < 4 || (f == 4 ? live_k : live_o);
        rbar[f * N + c] = lv ? dt * ybar[f * N + c] : 0.0;
    }
    const St<double> P = load_state<double, double>(x, c);
    double G[3][3], gk[3], gw[3];
    cell_gradients(cd, x, i, j, k, P, G, gk, gw);
    double S[3][3], S2 = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            S[a][b] = 0.5 * (G[a][b] + G[b][a]);
            S2 += S[a][b] * S[a][b];
        }
    S2 *= 2.0;
    s2[c] = S2;
    const double nu = cd.nu;
    const double nut = nut_of<double>(P.k, P.om, nu);
    const double ret = re_t<double>(P.k, P.om, nu), rw = ret / kRw;
    const double alpha = (kAlphaInf / alpha_star_of<double>(ret)) * ((kAlpha0 + rw) / (1.0 + rw));
    const double q = alpha * P.om / P.k;                       // G_omega = q G_k
    const double rk = live_k ? dt * ybar[4 * N + c] : 0.0, ro = live_o ? dt * ybar[5 * N + c] : 0.0;
    const double S2bar = (rk + ro * q) * nut;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Gbar[(3 * a + b) * N + c] = 4.0 * S[a][b] * S2bar;
}

// pass 2: per cell, the identity part of the update, the fluxes of its six faces
// (upwind convection, central diffusion with the face eddy viscosity, the -(2/3) k
// face term of the normal momentum) transposed onto the cell, the production and
// buoyancy sources, the eddy viscosity's dependence on k and omega, and the transposed
// velocity gradient of the production term
struct ExpAdjBK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;
    __device__ bool live() const { return true; }
    CaseDev cd;
    StatePtrs x;
    const double* ybar;     // 6 N
    const double* rbar;     // 6 N (pass 1)
    const double* Gbar;     // 9 N
    const double* s2;       // N
    double* xbar;           // 6 N
    __device__ void run(const BlockAt& at) const;
};

__device__ void ExpAdjBK::run(const BlockAt& at) const {
    int i, j, k;
    if (!cell3(cd, at, i, j, k)) return;
    const int c = i + cd.n[0] * (j + cd.n[1] * k);
    const int64_t N = cd.N;
    if (cd.tag[c]) {
        for (int f = 0; f < 6; ++f) xbar[f * N + c] = ybar[f * N + c];
        return;
    }
    const double nu = cd.nu;
    const double gam[6] = {nu, nu, nu, cd.alpha, nu, nu};
    const double isig[6] = {1.0, 1.0, 1.0, cd.inv_Prt, cd.inv_sigk, cd.inv_sigw};
    const St<double> P = load_state<double, double>(x, c);
    double rb[6], acc[6];
    // the identity part of phi + dt rhs where the update passes a derivative: there rbar =
    // dt ybar, so rbar = 0 with ybar != 0 marks a clamped k or omega or a wall omega
    for (int f = 0; f < 6; ++f) {
        rb[f] = rbar[f * N + c];
        acc[f] = f < 4 || rb[f] != 0.0 ? ybar[f * N + c] : 0.0;
    }
    const double nutP = nut_of<double>(P.k, P.om, nu);
    double nutbar = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (!cd.active[a]) continue;
        const double ih = cd.inv_h[a];
        for (int side = -1; side <= 1; side += 2) {
            int thermal, nb;
            const int kind = face_kind_of(cd, i, j, k, a, side, thermal, nb);
            St<double> Q;   // the state across the face (neighbour or ghost)
            neighbour<double, double>(cd, x, i, j, k, a, side, P, Q);
            const bool interior = kind == FK_INTERIOR;
            // face cotangents F_bar_f = (rbar(L cell) - rbar(R cell)) / h
            double Fb[6];
            for (int f = 0; f < 6; ++f) {
                const double rq = interior ? rbar[f * N + nb] : 0.0;
                Fb[f] = side > 0 ? (rb[f] - rq) * ih : (rq - rb[f]) * ih;
            }
            const St<double>& L = side > 0 ? P : Q;
            const St<double>& R = side > 0 ? Q : P;
            const double uf = 0.5 * (vcomp(L, a) + vcomp(R, a));
            const bool upL = uf >= 0.0;
            const double nutf = kind == FK_WALL ? 0.0
                                : (interior ? 0.5 * (nutP + nut_of<double>(Q.k, Q.om, nu)) : nutP);
            const double phL[6] = {L.u, L.v, L.w, L.T, L.k, L.om}, phR[6] = {R.u, R.v, R.w, R.T, R.k, R.om};
            double ufb = 0.0, nfb = 0.0;
            for (int f = 0; f < 6; ++f) {
                const double G_ = gam[f] + nutf * isig[f];
                const double dL = Fb[f] * ((upL ? -uf : 0.0) - G_ * ih);
                const double dR = Fb[f] * ((upL ? 0.0 : -uf) + G_ * ih);
                // this cell's own side, and (across a ghost face) the ghost built from it
                double d = side > 0 ? dL : dR;
                if (!interior) d += ghost_sign(f, kind, thermal) * (side > 0 ? dR : dL);
                acc[f] += d;
                ufb += -(upL ? phL[f] : phR[f]) * Fb[f];
                nfb += (phR[f] - phL[f]) * ih * isig[f] * Fb[f];
            }
            // face velocity (U_L + U_R) / 2 and the -(k_L + k_R) / 3 of the normal momentum
            const double sa = interior ? 0.0 : ghost_sign(a, kind, thermal);
            acc[a] += 0.5 * ufb * (1.0 + sa);
            const double sk = interior ? 0.0 : ghost_sign(4, kind, thermal);
            acc[4] += -Fb[a] / 3.0 * (1.0 + sk);
            // face eddy viscosity: the mean of the two cells inside, this cell's own on
            // inlet, outlet and empty faces, none on walls
            if (interior) nutbar += 0.5 * nfb;
            else if (kind != FK_WALL) nutbar += nfb;
        }
    }
    // sources: G_k = nu_t S^2, G_omega = q G_k, buoyancy -g_i beta_T (T - T_ref)
    const double S2 = s2[c];
    const double kk = P.k, om = P.om;
    const double oms = om > kEpsOmega ? om : kEpsOmega, doms = om > kEpsOmega ? 1.0 : 0.0;
    const double re = kk / (nu * oms), dre_dk = 1.0 / (nu * oms), dre_dom = -re / oms * doms;
    const double r = re / kRk;
    const double ast = kAlphaStarInf * (kAlphaStar0 + r) / (1.0 + r);
    const double dast = kAlphaStarInf * (1.0 - kAlphaStar0) / (kRk * (1.0 + r) * (1.0 + r));
    const double nut = ast * kk / oms;
    const double dnut_dk = ast / oms + kk / oms * dast * dre_dk;
    const double dnut_dom = -ast * kk / (oms * oms) * doms + kk / oms * dast * dre_dom;
    const double rw = re / kRw;
    const double A = (kAlpha0 + rw) / (1.0 + rw), dA = (1.0 - kAlpha0) / (kRw * (1.0 + rw) * (1.0 + rw));
    const double ac = kAlphaInf * A / ast, dac = kAlphaInf * (dA / ast - A * dast / (ast * ast));
    const double Gk = nut * S2;
    const double q = ac * om / kk;
    const double dq_dk = dac * dre_dk * om / kk - ac * om / (kk * kk);
    const double dq_dom = dac * dre_dom * om / kk + ac / kk;
    const double rk = rb[4], ro = rb[5];
    acc[4] += ro * Gk * dq_dk;
    acc[5] += ro * Gk * dq_dom;
    nutbar += (rk + ro * q) * S2;
    acc[4] += nutbar * dnut_dk;
    acc[5] += nutbar * dnut_dom;
    acc[3] += cd.gb[0] * rb[0] + cd.gb[1] * rb[1] + cd.gb[2] * rb[2];
    // the production's velocity gradient, transposed
    for (int v = 0; v < 3; ++v)
        acc[v] += gradient_transpose(cd, v, i, j, k, c,
                                     [&](int m, int qq) { return Gbar[(size_t)(3 * v + m) * N + qq]; });
    for (int f = 0; f < 6; ++f) xbar[f * N + c] = acc[f];
}

// ------------------------------------------------------------------ lambda_2 diagnostic
// The vortex criterion of the transient results (Section 3.2.3; Jeong and
// Hussain 1995): lambda_2, the middle eigenvalue of the symmetric matrix
// M = S^2 + Omega^2 of the cell velocity gradient.  The gradient is the cell
// gradient L_j * D_j * BC_j(u_i) of Algorithm 4 (the destruction kernel's),
// so wall, inlet, outlet and obstacle neighbours take their Section 2.7
// ghosts.  Solid cells get 0.  The result is written as FP64.
//
// Middle eigenvalue of a symmetric 3x3 matrix by cyclic Jacobi rotations
// (Golub and Van Loan, "Matrix Computations", the symmetric Schur
// decomposition and the cyclic Jacobi method).  The rotation in the (p, q)
// plane with tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| +
// sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c zeroes a_pq and gives
// a_pp - t a_pq, a_qq + t a_pq, and (c a_rp - s a_rq, s a_rp + c a_rq) for
// the third index r.  Sweeps stop once the off-diagonal part is below
// eps |M|_F (the diagonal is then within that of the eigenvalues, by Weyl's
// inequality); three to four sweeps suffice, eight bound the loop.  Unlike
// the trigonometric closed form, whose acos loses half the digits of a
// nearly repeated eigenvalue, this keeps every eigenvalue to a few eps |M|.
template <class C> struct Eps;
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };
template <> struct Eps<float> { static constexpr float v = 1.1920929e-7f; };

template <class C>
__device__ __forceinline__ void jacobi_rotate(C& app, C& aqq, C& apq, C& arp, C& arq) {
    if (apq == (C)0) return;
    const C tau = (aqq - app) / ((C)2 * apq);
    const C t = (tau >= (C)0 ? (C)1 : (C)-1) / (fabs(tau) + sqrt((C)1 + tau * tau));
    const C c = (C)1 / sqrt((C)1 + t * t);
    const C s = t * c;
    app -= t * apq;
    aqq += t * apq;
    apq = (C)0;
    const C rp = c * arp - s * arq;
    arq = s * arp + c * arq;
    arp = rp;
}

template <class C>
__device__ __forceinline__ C sym3_middle_eigenvalue(C a00, C a11, C a22, C a01, C a02, C a12) {
    const C e = Eps<C>::v;
    const C fro2 = a00 * a00 + a11 * a11 + a22 * a22 + (C)2 * (a01 * a01 + a02 * a02 + a12 * a12);
    for (int sweep = 0; sweep < 8; ++sweep) {
        if (a01 * a01 + a02 * a02 + a12 * a12 <= fro2 * e * e) break;
        jacobi_rotate(a00, a11, a01, a02, a12);   // (0,1); r = 2
        jacobi_rotate(a00, a22, a02, a01, a12);   // (0,2); r = 1
        jacobi_rotate(a11, a22, a12, a01, a02);   // (1,2); r = 0
    }
    const C lo = a00 < a11 ? a00 : a11;
    const C hi = a00 < a11 ? a11 : a00;
    return a22 < lo ? lo : (a22 > hi ? hi : a22);
}

template <class S, class C>
struct Lambda2K {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    __device__ bool live() const { return true; }
    CaseDev cd;
    StatePtrs in;
    double* out;
    __device__ void run(const BlockAt& at) const;
};

template <class S, class C>
__device__ void Lambda2K<S, C>::run(const BlockAt& at) const {
    int i, j, k;
    if (!cell3(cd, at, i, j, k)) return;
    const int c = i + cd.n[0] * (j + cd.n[1] * k);
    if (cd.tag[c]) {
        out[c] = 0.0;
        return;
    }
    // only u, v, w of the loaded states are used; the other loads are dead code
    const St<C> P = load_state<S, C>(in, c);
    C g[3][3];   // g[a][b] = d u_a / d x_b
    for (int b = 0; b < 3; ++b) {
        if (!cd.active[b]) {
            g[0][b] = g[1][b] = g[2][b] = (C)0;
            continue;
        }
        St<C> L, R;
        neighbour<S, C>(cd, in, i, j, k, b, -1, P, L);
        neighbour<S, C>(cd, in, i, j, k, b, +1, P, R);
        const C ih = prm<C>(cd.inv_h[b], cd.f.inv_h[b]);
        g[0][b] = (C)0.5 * ((R.u - P.u) * ih + (P.u - L.u) * ih);
        g[1][b] = (C)0.5 * ((R.v - P.v) * ih + (P.v - L.v) * ih);
        g[2][b] = (C)0.5 * ((R.w - P.w) * ih + (P.w - L.w) * ih);
    }
    C Sm[3][3], Om[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            Sm[a][b] = (C)0.5 * (g[a][b] + g[b][a]);
            Om[a][b] = (C)0.5 * (g[a][b] - g[b][a]);
        }
    C M[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b) {
            C acc = (C)0;
            for (int e = 0; e < 3; ++e) acc += Sm[a][e] * Sm[e][b] + Om[a][e] * Om[e][b];
            M[a][b] = acc;
        }
    out[c] = (double)sym3_middle_eigenvalue<C>(M[0][0], M[1][1], M[2][2], M[0][1], M[0][2], M[1][2]);
}

// ------------------------------------------------------------------ pack / unpack
template <class S>
__global__ void k_pack(const S* __restrict__ src, double* __restrict__ dst, int64_t N) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) dst[c] = to_c<double>(src[c]);
}

template <class S>
__global__ void k_unpack(const double* __restrict__ src, S* __restrict__ dst, int64_t N) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) dst[c] = from_c<S, double>(src[c]);
}

inline unsigned nblocks(int64_t N) { return (unsigned)((N + kThreads - 1) / kThreads); }
inline dim3 grid3(const CaseDev& cd) {
    return dim3((unsigned)((cd.n[0] + BX - 1) / BX), (unsigned)((cd.n[1] + BY - 1) / BY),
                (unsigned)((cd.n[2] + BZ - 1) / BZ));
}
const dim3 kBlock3(BX, BY, BZ);

// the four-cell forms: FP32 fields and nx % 4 = 0
inline bool four_cells(int prec, const CaseDev& cd) { return prec != FVM_FP64 && cd.n[0] % 4 == 0; }
// log2 of the lanes of a row segment: the widest of 128, 64, 32 and 16 cells that divides nx
inline int seg_lrl(int nx) {
    for (int l = 5; l >= 2; --l)
        if (nx % (4 << l) == 0) return l;
    return 5;
}
inline dim3 grid4(const CaseDev& cd, int lrl) {
    const int wx = 4 << lrl, wy = VY << (5 - lrl);
    return dim3((unsigned)((cd.n[0] + wx - 1) / wx), (unsigned)((cd.n[1] + wy - 1) / wy), (unsigned)cd.n[2]);
}

}  // namespace

// ---------------------------------------------------------------- launchers
#define DISPATCH(prec, ...)                                    \
    do {                                                       \
        if ((prec) == FVM_FP64) {                              \
            using S = double; using C = double; __VA_ARGS__;   \
        } else {                                               \
            using S = float; using C = float; __VA_ARGS__;     \
        }                                                      \
    } while (0)

cudaError_t launch_init_state(int prec, const CaseDev& cd, StatePtrs st, const double* base, uint64_t seed,
                              double eps, cudaStream_t s) {
    DISPATCH(prec, (void)sizeof(C); k_init<S><<<nblocks(cd.N), kThreads, 0, s>>>(
                       cd, st, base[0], base[1], base[2], base[3], base[4], base[5], seed, eps));
    return cudaGetLastError();
}

cudaError_t launch_dt(int prec, const CaseDev& cd, StatePtrs st, double* dt_state, cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    DISPATCH(prec, err = launch_k(RateMaxK<S, C>{cd, st, (unsigned long long*)(dt_state + 3)}, dim3(nblocks(cd.N)),
                                  dim3(kThreads), 0, s));
    if (err != cudaSuccess) return err;
    return launch_k(DtFinalizeK{cd.dt0, cd.cfl, cd.dt_adapt, dt_state}, dim3(1), dim3(1), 0, s);
}

cudaError_t launch_destruction(int prec, const CaseDev& cd, StatePtrs in, void* k_out, void* om_out,
                               const double* dt_state, void* nut_out, void* b_out, cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    DISPATCH(prec, err = launch_k(DestructionK<S, C>{cd, in, (S*)k_out, (S*)om_out, dt_state, (S*)nut_out, (S*)b_out},
                                  grid3(cd), kBlock3, 0, s));
    return err;
}

cudaError_t launch_explicit(int prec, const CaseDev& cd, StatePtrs in, StatePtrs out, const double* dt_state,
                            const void* nut, StatePtrs base, double wb, double ws, cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    if (base.f[0])
        DISPATCH(prec, err = launch_k(ExplicitK<S, C, true>{cd, in, out, dt_state, (const S*)nut, base, wb, ws,
                                                            (float)wb, (float)ws},
                                      grid3(cd), kBlock3, 0, s));
    else
        DISPATCH(prec, err = launch_k(ExplicitK<S, C, false>{cd, in, out, dt_state, (const S*)nut, base, wb, ws,
                                                             (float)wb, (float)ws},
                                      grid3(cd), kBlock3, 0, s));
    return err;
}

cudaError_t launch_rhs(int prec, const CaseDev& cd, StatePtrs in, void* b, const double* dt_state,
                       cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    DISPATCH(prec, err = launch_k(RhsK<S, C>{cd, in, (S*)b, dt_state}, grid3(cd), kBlock3, 0, s));
    return err;
}

cudaError_t launch_project(int prec, const CaseDev& cd, const LevelDev& L0, StatePtrs in, StatePtrs out,
                           const double* p, const double* dt_state, cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    if (four_cells(prec, cd)) {
        const int lrl = seg_lrl(cd.n[0]);
        return launch_k(ProjectVK{ProjectK<float, float>{cd, L0, in, out, p, dt_state}, lrl}, grid4(cd, lrl),
                        dim3(VX, VY), 0, s);
    }
    DISPATCH(prec, err = launch_k(ProjectK<S, C>{cd, L0, in, out, p, dt_state}, grid3(cd), kBlock3, 0, s));
    return err;
}

cudaError_t launch_adj_grad(const CaseDev& cd, const LevelDev& L0, const double* ybar, double* q, double dt,
                            cudaStream_t s) {
    return launch_k(AdjGradK{cd, L0, ybar, q, dt}, grid3(cd), kBlock3, 0, s);
}

cudaError_t launch_adj_rhs(const CaseDev& cd, const LevelDev& L0, const double* ybar, const double* lambda,
                           double* xbar, double dt, cudaStream_t s) {
    return launch_k(AdjRhsK{cd, L0, ybar, lambda, xbar, {cd.inv_h[0] / dt, cd.inv_h[1] / dt, cd.inv_h[2] / dt}},
                    grid3(cd), kBlock3, 0, s);
}

cudaError_t launch_lambda2(int prec, const CaseDev& cd, StatePtrs in, double* out, cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    DISPATCH(prec, err = launch_k(Lambda2K<S, C>{cd, in, out}, grid3(cd), kBlock3, 0, s));
    return err;
}

cudaError_t launch_pack(int prec, const void* src, double* dst, int64_t N, cudaStream_t s) {
    if (prec == FVM_FP64) k_pack<double><<<nblocks(N), kThreads, 0, s>>>((const double*)src, dst, N);
    else if (prec == FVM_FP32) k_pack<float><<<nblocks(N), kThreads, 0, s>>>((const float*)src, dst, N);
    else k_pack<__nv_bfloat16><<<nblocks(N), kThreads, 0, s>>>((const __nv_bfloat16*)src, dst, N);
    return cudaGetLastError();
}

cudaError_t launch_unpack(int prec, const double* src, void* dst, int64_t N, cudaStream_t s) {
    if (prec == FVM_FP64) k_unpack<double><<<nblocks(N), kThreads, 0, s>>>(src, (double*)dst, N);
    else if (prec == FVM_FP32) k_unpack<float><<<nblocks(N), kThreads, 0, s>>>(src, (float*)dst, N);
    else k_unpack<__nv_bfloat16><<<nblocks(N), kThreads, 0, s>>>(src, (__nv_bfloat16*)dst, N);
    return cudaGetLastError();
}

cudaError_t launch_destruction_vjp(const CaseDev& cd, StatePtrs x, double dt, const double* ybar, double* out,
                                   double* scratch, cudaStream_t s) {
    // ybar: u, v, w, k, omega cotangents (5 N); scratch: kout, oout, gbar (17 N)
    const int64_t N = cd.N;
    double* kout = scratch;
    double* oout = scratch + N;
    double* gbar = scratch + 2 * N;
    cudaError_t e = launch_k(DesAdjAK{cd, x, dt, ybar + 3 * N, ybar + 4 * N, kout, oout, gbar}, grid3(cd), kBlock3, 0, s);
    if (e != cudaSuccess) return e;
    return launch_k(DesAdjBK{cd, ybar, kout, oout, gbar, out}, grid3(cd), kBlock3, 0, s);
}

cudaError_t launch_explicit_vjp(const CaseDev& cd, StatePtrs x, StatePtrs y, double dt, const double* ybar,
                                double* xbar, double* scratch, cudaStream_t s) {
    // scratch: rbar (6 N), Gbar (9 N), S^2 (N)
    const int64_t N = cd.N;
    double* rbar = scratch;
    double* Gbar = scratch + 6 * N;
    double* s2 = scratch + 15 * N;
    cudaError_t e = launch_k(ExpAdjAK{cd, x, y, dt, ybar, rbar, Gbar, s2}, grid3(cd), kBlock3, 0, s);
    if (e != cudaSuccess) return e;
    return launch_k(ExpAdjBK{cd, x, ybar, rbar, Gbar, s2, xbar}, grid3(cd), kBlock3, 0, s);
}
