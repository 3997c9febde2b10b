// Multigrid kernels for the pressure Poisson equation A p = b, A = -Laplacian
// with one ghost layer (Section 2.4: Eq. neg_lap_discretize, the printed
// 3x3x3 kernel, Eq. jacobi_pc, Eqs. restriction / prolongation, Algorithm 1).
//
// The solve runs in correction form: the level-0 residual r = b - A p is
// formed from the FP64 pressure with an FP64 norm, a V-cycle computes the
// correction e from A e = r in the inner precision (FP64, FP32 or BF16
// storage), and the last post-smoothing sweep adds e to p.  In exact
// arithmetic this is the V-cycle on p itself; in finite precision it is
// defect correction with an FP64 outer residual.
//
//   smoother   e <- e + w_J (r - A e) / D, D = sum_active 2 / h_a^2
//   RES        coarse r = mean of the children's residuals r - A e
//   PROL       e += trilinear interpolation of the coarse correction:
//              3/4 parent + 1/4 neighbour per axis, neighbour index clamped
//   coarsest   e = A^{-1} r with the dense inverse built on the host
//
// Every cell carries a 16-bit neighbour code (two bits per face: 0 = fluid
// neighbour, 1 = zero-gradient ghost, 2 = zero-value ghost; bit 12 = solid),
// so the stencil needs one small load instead of mask and face-table lookups.
// Grid kernels use 3D blocks (no integer division).  All levels that fit in
// one CTA's shared memory are cycled by a single CTA.  The level-0 residual
// kernel finishes the norm in its last block and decides on the device
// whether another cycle runs, so the whole solve can live in a CUDA graph.
#include "fvm_internal.cuh"

namespace {

template <class T> struct Acc { using type = T; };
template <> struct Acc<__nv_bfloat16> { using type = float; };

constexpr int BX = 32, BY = 4, BZ = 2;
constexpr int kCtaThreads = 1024;

__device__ __forceinline__ bool cell3(const LevelDev& L, const BlockAt& at, int& i, int& j, int& k) {
    i = at.b.x * BX + threadIdx.x;
    j = at.b.y * BY + threadIdx.y;
    k = at.b.z * BZ + threadIdx.z;
    return i < L.n[0] && j < L.n[1] && k < L.n[2];
}

// value across one face: the neighbour (read through `get`, only for code 0),
// the zero-gradient ghost eP or the zero-value ghost -eP
template <class C, class G>
__device__ __forceinline__ C nb_val(uint32_t code, int idx, C eP, G get) {
    return code == 0 ? get(idx) : (code == 1 ? eP : -eP);
}

// (A e)_P = sum_active (2 eP - e_lo - e_hi) / h_a^2; get(q) reads e at cell q
template <class C, class G>
__device__ __forceinline__ C apply_A_with(const LevelDev& L, uint32_t f, int c, C eP, G get) {
    const int sx = 1, sy = L.n[0], sz = L.n[0] * L.n[1];
    C acc = (C)0;
    if (L.active[0]) {
        const C lo = nb_val<C>(f & 3u, c - sx, eP, get), hi = nb_val<C>((f >> 2) & 3u, c + sx, eP, get);
        acc += ((eP - lo) + (eP - hi)) * LP<C>::ih2(L, 0);
    }
    if (L.active[1]) {
        const C lo = nb_val<C>((f >> 4) & 3u, c - sy, eP, get), hi = nb_val<C>((f >> 6) & 3u, c + sy, eP, get);
        acc += ((eP - lo) + (eP - hi)) * LP<C>::ih2(L, 1);
    }
    if (L.active[2]) {
        const C lo = nb_val<C>((f >> 8) & 3u, c - sz, eP, get), hi = nb_val<C>((f >> 10) & 3u, c + sz, eP, get);
        acc += ((eP - lo) + (eP - hi)) * LP<C>::ih2(L, 2);
    }
    return acc;
}

// A e for e in global memory (read-only path)
template <class C, class T>
__device__ __forceinline__ C apply_A(const LevelDev& L, uint32_t f, const T* e, int c, C eP) {
    return apply_A_with<C>(L, f, c, eP, [&](int q) { return to_c<C>(ldg(e + q)); });
}

__device__ __forceinline__ bool is_solid(uint32_t f) { return (f >> 12) & 1u; }

template <class C>
__device__ __forceinline__ C sel(uint32_t code, C nb, C eP) {
    return code == 0 ? nb : (code == 1 ? eP : -eP);
}

// A e at one cell from its gathered neighbours: the general form, with each
// face's ghost chosen by its code.  Kept out of line so that it cannot be
// predicated into the common path below.
template <class C>
__device__ __noinline__ C A7_general(const LevelDev& L, uint32_t f, C eP, C xm, C xp, C ym, C yp, C zm, C zp) {
    C acc = (C)0;
    if (L.active[0]) acc += ((eP - sel(f & 3u, xm, eP)) + (eP - sel((f >> 2) & 3u, xp, eP))) * LP<C>::ih2(L, 0);
    if (L.active[1]) acc += ((eP - sel((f >> 4) & 3u, ym, eP)) + (eP - sel((f >> 6) & 3u, yp, eP))) * LP<C>::ih2(L, 1);
    if (L.active[2]) acc += ((eP - sel((f >> 8) & 3u, zm, eP)) + (eP - sel((f >> 10) & 3u, zp, eP))) * LP<C>::ih2(L, 2);
    return acc;
}

// A e at one cell.  The neighbour values are loaded with indices clamped into
// the grid, so at a zero-gradient domain face the load already returns eP,
// the ghost value.  Every cell without a zero-value face or a solid neighbour
// (code bit 13 clear) therefore takes diag eP - sum_a ih2_a (lo + hi), with
// ih2_a = 0 on a collapsed axis; the rest take the general form.
template <class C>
__device__ __forceinline__ C A7(const LevelDev& L, uint32_t f, C eP, C xm, C xp, C ym, C yp, C zm, C zp) {
    if (!((f >> 13) & 1u)) {
        C s = (xm + xp) * LP<C>::ih2a(L, 0);
        s = fma(ym + yp, LP<C>::ih2a(L, 1), s);
        s = fma(zm + zp, LP<C>::ih2a(L, 2), s);
        return fma(LP<C>::diag(L), eP, -s);
    }
    return A7_general<C>(L, f, eP, xm, xp, ym, yp, zm, zp);
}

// ------------------------------------------------------------------ level 0 residual
// The last block of a level-0 residual pass: a fixed-order reduction over
// all blocks' partials (r^2, b^2): thread t sums blocks t, t + NT, ... in
// order (L2 loads, independent), then a fixed shuffle tree and a fixed sum
// over warps, so the result is deterministic; then the stopping rule.
// Returns the decision in thread 0, -1 elsewhere.  Out of line: it runs once
// per launch and would otherwise hold registers in every block.
template <int NT>
__device__ __noinline__ int resid0_finish(const double* partials, int nblk, SolveState* st,
                                          double (*red)[NT / 32]) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    double a0 = 0.0, a1 = 0.0;
    for (int x = tid; x < nblk; x += NT) {
        const double2 v = __ldcg((const double2*)partials + x);
        a0 += v.x;
        a1 += v.y;
    }
    for (int off = 16; off > 0; off >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, off);
        a1 += __shfl_xor_sync(0xffffffffu, a1, off);
    }
    __syncthreads();
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = a0;
        red[1][tid >> 5] = a1;
    }
    __syncthreads();
    if (tid != 0) return -1;
    a0 = 0.0;
    a1 = 0.0;
    for (int w = 0; w < NT / 32; ++w) {
        a0 += red[0][w];
        a1 += red[1][w];
    }
    st->counter = 0u;
    st->r2 = a0;
    st->b2 = a1;
    const bool finite = isfinite(a0) && isfinite(a1);
    const double rel = a1 > 0.0 ? sqrt(a0 / a1) : 0.0;
    st->rel = finite ? rel : __longlong_as_double(0x7ff8000000000000ll);
    if (!finite) st->nonfinite = 1;
    int go;
    if (st->fixed > 0) go = st->cycles < st->fixed;
    else go = finite && rel > st->tol && st->cycles < st->max_cycles;
    st->active = go;
    if (!go && st->fixed == 0 && finite && rel > st->tol) st->notconv = 1;
    if (go) {
        st->cycles += st->inner;
        st->total_cycles += st->inner;
    }
    return go;
}

// r = b - A p (FP64), first pre-sweep e = w_J r / D, r^2 and b^2 per block;
// the last block sums the partials in a fixed order and applies the stopping rule.
// run() returns the decision (0 / 1) in the thread that made it, else -1.
template <class TB, class TI>
struct Resid0K {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr int kMinBlocks = 4;   // at most 64 registers (the batched form needs them)
    LevelDev L;
    const double* p;
    const TB* b;
    TI* r;
    TI* e;
    double* partials;
    SolveState* st;
    __device__ bool live() const { return st->active != 0; }   // batched: skip a converged case
    __device__ int run(const BlockAt& at) const;
};

template <class TB, class TI>
__device__ int Resid0K<TB, TI>::run(const BlockAt& at) const {
    using C = typename Acc<TI>::type;
    __shared__ double red[2][BX * BY * BZ / 32];
    __shared__ bool last;
    int i, j, k;
    C r2 = (C)0, b2 = (C)0;     // squares and warp sums in the inner precision, block sums in FP64
    if (cell3(L, at, i, j, k)) {
        const int c = i + L.n[0] * (j + L.n[1] * k);
        const uint32_t f = L.nbf[c];
        // neighbour loads first (clamped indices), then the FP64 stencil
        const int sy = L.n[0], sz = L.n[0] * L.n[1];
        // (reduced-precision cases: p as double-float pairs, summed in FP64 on this small-grid path)
        auto P = [&](int q) { return sizeof(TB) == 8 ? __ldg(p + q) : pp_get(p, q); };
        const double pP = P(c);
        const double xm = P(c - (i > 0 ? 1 : 0)), xp = P(c + (i < L.n[0] - 1 ? 1 : 0));
        const double ym = P(c - (j > 0 ? sy : 0)), yp = P(c + (j < L.n[1] - 1 ? sy : 0));
        const double zm = P(c - (k > 0 ? sz : 0)), zp = P(c + (k < L.n[2] - 1 ? sz : 0));
        const TB braw = ldg(b + c);
        C rc = (C)0, bc = (C)0;
        if (!is_solid(f)) {
            const double bv = to_c<double>(braw);
            const double Ap = A7<double>(L, f, pP, xm, xp, ym, yp, zm, zp);
            const TI rs = from_c<TI, double>(bv - Ap);
            r[c] = rs;
            rc = to_c<C>(rs);
            bc = to_c<C>(braw);
            e[c] = from_c<TI, C>(LP<C>::wJ(L) * rc * LP<C>::iD(L));
        } else {
            r[c] = from_c<TI, C>((C)0);
            e[c] = from_c<TI, C>((C)0);
        }
        r2 = rc * rc;
        b2 = bc * bc;
    }
    const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);
    for (int off = 16; off > 0; off >>= 1) {
        r2 += __shfl_xor_sync(0xffffffffu, r2, off);
        b2 += __shfl_xor_sync(0xffffffffu, b2, off);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = (double)r2;
        red[1][tid >> 5] = (double)b2;
    }
    __syncthreads();
    const int nblk = at.g.x * at.g.y * at.g.z;
    const int bid = at.b.x + at.g.x * (at.b.y + at.g.y * at.b.z);
    if (tid == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int w = 0; w < BX * BY * BZ / 32; ++w) {
            s0 += red[0][w];
            s1 += red[1][w];
        }
        partials[2 * bid] = s0;
        partials[2 * bid + 1] = s1;
        __threadfence();
        const unsigned done = atomicAdd(&st->counter, 1u);
        last = done == (unsigned)nblk - 1u;
    }
    __syncthreads();
    if (!last) return -1;
    __threadfence();
    return resid0_finish<BX * BY * BZ>(partials, nblk, st, red);
}

struct SolveBeginK {
    static constexpr int kThreads = 1;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    SolveState* st;
    __device__ bool live() const { return true; }
    __device__ void run(const BlockAt&) const {
        st->cycles = 0;
        st->counter = 0u;
        st->g_counter = 0u;
        st->g_valid = 0;
        st->active = 1;
    }
};

// ------------------------------------------------------------------ grid kernels (one level)
template <class TI>
struct SweepFirstK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    LevelDev L;
    const TI* r;
    TI* e;
    const SolveState* st;
    __device__ bool live() const { return st->active != 0; }   // batched: skip a converged case
    __device__ void run(const BlockAt& at) const {
        using C = typename Acc<TI>::type;
        int i, j, k;
        if (!cell3(L, at, i, j, k)) return;
        const int c = i + L.n[0] * (j + L.n[1] * k);
        const uint32_t f = L.nbf[c];
        e[c] = from_c<TI, C>(is_solid(f) ? (C)0 : LP<C>::wJ(L) * to_c<C>(ldg(r + c)) * LP<C>::iD(L));
    }
};

// store a restricted residual and, where asked (ec0 not null), the coarse
// level's first Jacobi sweep from e = 0 computed from the stored value, as
// SweepFirstK would: one launch fewer per level and V-cycle
template <class TI, class C>
__device__ __forceinline__ void store_restricted(const LevelDev& Lc, TI* rc, TI* ec0, int idx, C val) {
    const TI rs = from_c<TI, C>(val);
    rc[idx] = rs;
    if (ec0)
        ec0[idx] = from_c<TI, C>(is_solid(Lc.nbf[idx]) ? (C)0 : LP<C>::wJ(Lc) * to_c<C>(rs) * LP<C>::iD(Lc));
}

// coarse r = mean over the children of (r - A e); one thread per coarse cell
template <class TI>
struct ResidRestrictK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    LevelDev Lf, Lc;
    const TI* e;
    const TI* r;
    TI* rc;
    TI* ec0;   // the coarse level's first sweep, or null
    const SolveState* st;
    __device__ bool live() const { return st->active != 0; }   // batched: skip a converged case
    __device__ void run(const BlockAt& at) const;
};

template <class TI>
__device__ void ResidRestrictK<TI>::run(const BlockAt& at) const {
    using C = typename Acc<TI>::type;
    int I, J, K;
    if (!cell3(Lc, at, I, J, K)) return;
    const int fx = Lf.active[0] ? 2 : 1, fy = Lf.active[1] ? 2 : 1, fz = Lf.active[2] ? 2 : 1;
    C sum = (C)0;
    for (int dz = 0; dz < fz; ++dz)
        for (int dy = 0; dy < fy; ++dy)
            for (int dx = 0; dx < fx; ++dx) {
                const int c = (I * fx + dx) + Lf.n[0] * ((J * fy + dy) + Lf.n[1] * (K * fz + dz));
                const uint32_t f = Lf.nbf[c];
                if (is_solid(f)) continue;
                const C eP = to_c<C>(ldg(e + c));
                sum += to_c<C>(ldg(r + c)) - apply_A<C>(Lf, f, e, c, eP);
            }
    store_restricted<TI, C>(Lc, rc, ec0, I + Lc.n[0] * (J + Lc.n[1] * K), sum / (C)(fx * fy * fz));
}

// Trilinear prolongation of a coarse field at fine cell (i,j,k) (Eq.
// prolongation): per active axis 3/4 of the parent and 1/4 of the parent's
// neighbour on the fine cell's side.  A neighbour beyond a domain face is the
// coarse level's ghost of the clamped cell (the boundary rules of Section 2.7
// on every level): the cell's own value across a zero-gradient face, its
// negative across a zero-value (outlet) face; at an edge or corner the signs
// of both faces apply.  get(q) reads the coarse value, code(q) the coarse
// cell's 16-bit neighbour code (two bits per face, 2 = zero-value).
template <class C, class G, class F>
__device__ __forceinline__ C prolong_at(const int* fa, const int* cn, int i, int j, int k, G get, F code) {
    const int f[3] = {i, j, k};
    int P[3], Q[3], side[3];
    bool out[3];
    C w[3][2];
    for (int a = 0; a < 3; ++a) {
        out[a] = false;
        side[a] = 0;
        if (fa[a]) {
            P[a] = f[a] >> 1;
            const int q = P[a] + ((f[a] & 1) ? 1 : -1);
            out[a] = q < 0 || q >= cn[a];
            side[a] = q < 0 ? 0 : 1;
            Q[a] = out[a] ? P[a] : q;
            w[a][0] = (C)0.75;
            w[a][1] = (C)0.25;
        } else {
            P[a] = Q[a] = f[a];
            w[a][0] = (C)1;
            w[a][1] = (C)0;
        }
    }
    C acc = (C)0;
    for (int sz = 0; sz < (fa[2] ? 2 : 1); ++sz)
        for (int sy = 0; sy < (fa[1] ? 2 : 1); ++sy)
            for (int sx = 0; sx < (fa[0] ? 2 : 1); ++sx) {
                const int ii = sx ? Q[0] : P[0], jj = sy ? Q[1] : P[1], kk = sz ? Q[2] : P[2];
                const int q = ii + cn[0] * (jj + cn[1] * kk);
                C v = get(q);
                const bool gx = sx && out[0], gy = sy && out[1], gz = sz && out[2];
                if (gx || gy || gz) {
                    const uint32_t fc = code(q);
                    bool neg = false;
                    if (gx) neg ^= ((fc >> (2 * (0 + side[0]))) & 3u) == 2u;
                    if (gy) neg ^= ((fc >> (2 * (2 + side[1]))) & 3u) == 2u;
                    if (gz) neg ^= ((fc >> (2 * (4 + side[2]))) & 3u) == 2u;
                    if (neg) v = -v;
                }
                acc += w[0][sx] * w[1][sy] * w[2][sz] * v;
            }
    return acc;
}

template <class TI>
struct ProlongK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    LevelDev Lf, Lc;
    const TI* ec;
    TI* e;
    const SolveState* st;
    __device__ bool live() const { return st->active != 0; }   // batched: skip a converged case
    __device__ void run(const BlockAt& at) const {
        using C = typename Acc<TI>::type;
        int i, j, k;
        if (!cell3(Lf, at, i, j, k)) return;
        const int c = i + Lf.n[0] * (j + Lf.n[1] * k);
        if (is_solid(Lf.nbf[c])) return;
        const C add = prolong_at<C>(Lf.active, Lc.n, i, j, k, [&](int q) { return to_c<C>(ldg(ec + q)); },
                                    [&](int q) { return (uint32_t)__ldg(Lc.nbf + q); });
        e[c] = from_c<TI, C>(to_c<C>(e[c]) + add);
    }
};

// ------------------------------------------------------------------ marching kernels (levels >= 0)
// Blocks of TX x TY threads over x-y tiles, marching along z.  Neighbour
// loads use indices clamped into the grid (a face outside the domain reads
// the cell itself), so only cells with code bit 13 need the ghost selects.
constexpr int TX = 32, TY = 8;

struct Walk {
    int i, j, k0, sy, sz, im, ip, jm, jp;
};

__device__ __forceinline__ bool walk_setup(const LevelDev& L, const BlockAt& at, int kz, Walk& w) {
    w.i = at.b.x * TX + threadIdx.x;
    w.j = at.b.y * TY + threadIdx.y;
    w.k0 = at.b.z * kz;
    if (w.i >= L.n[0] || w.j >= L.n[1]) return false;
    w.sy = L.n[0];
    w.sz = L.n[0] * L.n[1];
    w.im = w.i > 0 ? -1 : 0;
    w.ip = w.i < L.n[0] - 1 ? 1 : 0;
    w.jm = w.j > 0 ? -w.sy : 0;
    w.jp = w.j < L.n[1] - 1 ? w.sy : 0;
    return true;
}

// Scalar sweep (FP64 levels, and levels whose x extent is not a multiple of
// 4): each thread walks KZ cells along z, keeping the z neighbours in
// registers; all loads of its cells are issued before any arithmetic.
// MODE 0: eout = sweep(ein); MODE 1: p += sweep(ein) (last level-0 sweep); MODE 2: the
// result in FP32 (the last level-0 sweep under the flexible-CG acceleration of BF16 levels).
template <class TI, int MODE, int KZ>
struct SweepK {
    static constexpr int kThreads = TX * TY;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    LevelDev L;
    const TI* ein;
    const TI* r;
    TI* eout;
    double* p;
    const SolveState* st;
    float* z32;   // MODE 2: the result in FP32
    __device__ bool live() const { return st->active != 0; }   // batched: skip a converged case
    __device__ void run(const BlockAt& at) const;
};

template <class TI, int MODE, int KZ>
__device__ void SweepK<TI, MODE, KZ>::run(const BlockAt& at) const {
    using C = typename Acc<TI>::type;
    Walk w;
    if (!walk_setup(L, at, KZ, w)) return;
    const int nz = L.n[2];
    const int c0 = w.i + w.sy * w.j + w.sz * w.k0;
    const int kn = nz - w.k0 < KZ ? nz - w.k0 : KZ;   // cells of this thread
    C col[KZ + 2], xm[KZ], xp[KZ], ym[KZ], yp[KZ], rr[KZ];
    uint32_t f[KZ];
    col[0] = to_c<C>(ldg(ein + c0 - (w.k0 > 0 ? w.sz : 0)));
#pragma unroll
    for (int kk = 0; kk < KZ; ++kk) {
        if (kk < kn) {
            const int c = c0 + kk * w.sz;
            col[kk + 1] = to_c<C>(ldg(ein + c));
            xm[kk] = to_c<C>(ldg(ein + c + w.im));
            xp[kk] = to_c<C>(ldg(ein + c + w.ip));
            ym[kk] = to_c<C>(ldg(ein + c + w.jm));
            yp[kk] = to_c<C>(ldg(ein + c + w.jp));
            rr[kk] = to_c<C>(ldg(r + c));
            f[kk] = L.nbf[c];
            if (kk == kn - 1)   // the plane above the thread's last cell (itself at the top face)
                col[kk + 2] = w.k0 + kk < nz - 1 ? to_c<C>(ldg(ein + c + w.sz)) : col[kk + 1];
        }
    }
    const C wJ = LP<C>::wJ(L), iD = LP<C>::iD(L);
#pragma unroll
    for (int kk = 0; kk < KZ; ++kk) {
        if (kk < kn) {
            const int c = c0 + kk * w.sz;
            const C eP = col[kk + 1];
            const bool solid = is_solid(f[kk]);
            const C v = solid ? (C)0
                              : eP + wJ * (rr[kk] - A7<C>(L, f[kk], eP, xm[kk], xp[kk], ym[kk], yp[kk], col[kk],
                                                          col[kk + 2])) * iD;
            if (MODE == 0) eout[c] = from_c<TI, C>(v);
            else if (MODE == 2) z32[c] = (float)v;
            else if (!solid) {
                if constexpr (sizeof(TI) == 8) p[c] += (double)v;
                else pp_add(p, c, (float)v);
            }
        }
    }
}

// W consecutive x cells per thread (the vector kernels): W = 4 with 128-bit
// loads for FP32 levels, W = 8 with 128-bit loads for BF16 levels (W = 4,
// 64-bit loads, where nx is not a multiple of 8).  A warp covers W * 32
// cells of a row (or 2, 4, 8 rows of W * 16, W * 8, W * 4 cells: the widest
// segment that divides nx) and marches zc planes in z: rows j +- 1 and the
// plane after next are loaded whole (indices clamped into the grid, so a
// zero-gradient domain face reads the cell itself), the x neighbours come
// from the adjacent lanes by shuffles (the segment's two end cells from
// single loads), and the z neighbours rotate in registers.
__device__ __forceinline__ void bf2_unpack(uint32_t w, float& a, float& b) {
    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
    a = f.x;
    b = f.y;
}
__device__ __forceinline__ uint32_t bf2_pack(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&v);
}

template <class TI, int W> struct VecW;
template <> struct VecW<float, 4> {
    static __device__ __forceinline__ void load(const float* p, int c, float (&o)[4]) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p + c));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    static __device__ __forceinline__ void load_rw(const float* p, int c, float (&o)[4]) {
        const float4 v = *reinterpret_cast<const float4*>(p + c);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    static __device__ __forceinline__ void store(float* p, int c, const float (&v)[4]) {
        *reinterpret_cast<float4*>(p + c) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct VecW<float, 8> {
    static __device__ __forceinline__ void store(float* p, int c, const float (&v)[8]) {
        *reinterpret_cast<float4*>(p + c) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4*>(p + c + 4) = make_float4(v[4], v[5], v[6], v[7]);
    }
};
template <> struct VecW<__nv_bfloat16, 4> {
    static __device__ __forceinline__ void load(const __nv_bfloat16* p, int c, float (&o)[4]) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(p + c));
        bf2_unpack(v.x, o[0], o[1]);
        bf2_unpack(v.y, o[2], o[3]);
    }
    static __device__ __forceinline__ void load_rw(const __nv_bfloat16* p, int c, float (&o)[4]) {
        const uint2 v = *reinterpret_cast<const uint2*>(p + c);
        bf2_unpack(v.x, o[0], o[1]);
        bf2_unpack(v.y, o[2], o[3]);
    }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, int c, const float (&v)[4]) {
        *reinterpret_cast<uint2*>(p + c) = make_uint2(bf2_pack(v[0], v[1]), bf2_pack(v[2], v[3]));
    }
};
template <> struct VecW<__nv_bfloat16, 8> {
    static __device__ __forceinline__ void load(const __nv_bfloat16* p, int c, float (&o)[8]) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(p + c));
        bf2_unpack(v.x, o[0], o[1]);
        bf2_unpack(v.y, o[2], o[3]);
        bf2_unpack(v.z, o[4], o[5]);
        bf2_unpack(v.w, o[6], o[7]);
    }
    static __device__ __forceinline__ void load_rw(const __nv_bfloat16* p, int c, float (&o)[8]) {
        const uint4 v = *reinterpret_cast<const uint4*>(p + c);
        bf2_unpack(v.x, o[0], o[1]);
        bf2_unpack(v.y, o[2], o[3]);
        bf2_unpack(v.z, o[4], o[5]);
        bf2_unpack(v.w, o[6], o[7]);
    }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, int c, const float (&v)[8]) {
        *reinterpret_cast<uint4*>(p + c) =
            make_uint4(bf2_pack(v[0], v[1]), bf2_pack(v[2], v[3]), bf2_pack(v[4], v[5]), bf2_pack(v[6], v[7]));
    }
};
// the four-cell loads of the other kernels
template <class TI> using Vec4 = VecW<TI, 4>;

// the W cells' 16-bit neighbour codes
template <int W> __device__ __forceinline__ void codes_w(const uint16_t* f, int c, uint32_t (&o)[W]);
template <> __device__ __forceinline__ void codes_w<4>(const uint16_t* f, int c, uint32_t (&o)[4]) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(f + c));
    o[0] = v.x & 0xffffu; o[1] = v.x >> 16; o[2] = v.y & 0xffffu; o[3] = v.y >> 16;
}
template <> __device__ __forceinline__ void codes_w<8>(const uint16_t* f, int c, uint32_t (&o)[8]) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(f + c));
    o[0] = v.x & 0xffffu; o[1] = v.x >> 16; o[2] = v.y & 0xffffu; o[3] = v.y >> 16;
    o[4] = v.z & 0xffffu; o[5] = v.z >> 16; o[6] = v.w & 0xffffu; o[7] = v.w >> 16;
}

template <> __device__ __forceinline__ void codes_w<2>(const uint16_t* f, int c, uint32_t (&o)[2]) {
    const uint32_t v = __ldg(reinterpret_cast<const unsigned int*>(f + c));
    o[0] = v & 0xffffu; o[1] = v >> 16;
}

// cells per thread of the vector kernels on a level of this storage type
template <class TI> __device__ __host__ constexpr int vec_w() { return sizeof(TI) == 2 ? 8 : 4; }

// The register image of W cells as loaded (16 bytes for W = 4 FP32 and W = 8
// BF16), converted to FP32 one value at a time where used: keeps the vector
// kernels' rotating planes at 4 registers each.  A BF16 value is the high half
// of its FP32 pattern, so the conversion is one shift or mask.
template <class TI, int W> struct RawW;
template <> struct RawW<float, 4> {
    using T = float4;
    static __device__ __forceinline__ T load(const float* p, int c) { return __ldg(reinterpret_cast<const float4*>(p + c)); }
    static __device__ __forceinline__ float get(const T& v, int t) {
        return t == 0 ? v.x : (t == 1 ? v.y : (t == 2 ? v.z : v.w));
    }
};
template <> struct RawW<float, 2> {
    using T = float2;
    static __device__ __forceinline__ T load(const float* p, int c) { return __ldg(reinterpret_cast<const float2*>(p + c)); }
    static __device__ __forceinline__ float get(const T& v, int t) { return t == 0 ? v.x : v.y; }
};
template <> struct RawW<__nv_bfloat16, 2> {
    using T = uint32_t;
    static __device__ __forceinline__ T load(const __nv_bfloat16* p, int c) {
        return __ldg(reinterpret_cast<const unsigned int*>(p + c));
    }
    static __device__ __forceinline__ float get(const T& v, int t) {
        return __uint_as_float((t & 1) ? (v & 0xffff0000u) : (v << 16));
    }
};
template <> struct RawW<__nv_bfloat16, 4> {
    using T = uint2;
    static __device__ __forceinline__ T load(const __nv_bfloat16* p, int c) {
        return __ldg(reinterpret_cast<const uint2*>(p + c));
    }
    static __device__ __forceinline__ float get(const T& v, int t) {
        const uint32_t w = (t >> 1) == 0 ? v.x : v.y;
        return __uint_as_float((t & 1) ? (w & 0xffff0000u) : (w << 16));
    }
};
template <> struct RawW<__nv_bfloat16, 8> {
    using T = uint4;
    static __device__ __forceinline__ T load(const __nv_bfloat16* p, int c) {
        return __ldg(reinterpret_cast<const uint4*>(p + c));
    }
    static __device__ __forceinline__ float get(const T& v, int t) {
        const uint32_t w = (t >> 1) == 0 ? v.x : ((t >> 1) == 1 ? v.y : ((t >> 1) == 2 ? v.z : v.w));
        return __uint_as_float((t & 1) ? (w & 0xffff0000u) : (w << 16));
    }
};

// Ask L2 for the line holding p (no register is tied up while it lands): the z-march kernels
// name their rows of the plane three ahead, so that those loads later hit L2 instead of
// waiting out a DRAM round trip.
__device__ __forceinline__ void l2_prefetch(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
__device__ __forceinline__ void l1_prefetch(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

template <class TI, int MODE, int W>
struct SweepVK {
    static constexpr int kThreads = TX * TY;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    // at most 64 registers, four blocks per SM (batched too: the few spilled bytes cost less than a
    // block per SM); the eight-cell update of p (MODE 1) at most 80, three blocks.  (Issuing the
    // next plane's loads before the current plane's arithmetic, at 80 / 128 registers, measured
    // slower on the room.)
    static constexpr int kMinBlocks = (W == 8 && MODE == 1) ? 3 : 4;
    LevelDev L;
    const TI* ein;
    const TI* r;
    TI* eout;
    double* p;
    const SolveState* st;
    int zc;    // planes per block
    float* z32;   // MODE 2: the sweep's result in FP32 (the flexible-CG direction of BF16 levels)
    int lrl;   // log2 of the lanes per row segment (5: a warp per W * 32-cell segment; 4, 3, 2: a warp
               // covers 2, 4 or 8 rows, so narrow rows leave no lane idle)
    __device__ bool live() const { return st->active != 0; }   // batched: skip a converged case
    __device__ void run(const BlockAt& at) const;
};

template <class TI, int MODE, int W>
__device__ void SweepVK<TI, MODE, W>::run(const BlockAt& at) const {
    using C = float;
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int LR = 1 << lrl, lane = threadIdx.x & (LR - 1), sub = threadIdx.x >> lrl;
    const int i4 = at.b.x * (W * LR) + lane * W, j = ((at.b.y * TY + threadIdx.y) << (5 - lrl)) + sub;
    const int k0 = at.b.z * zc, k1 = min(nz, k0 + zc);
    const bool in = i4 < nx && j < ny;
    const int sy = nx, sz = nx * ny;
    const int ic = min(i4, nx - W), jc = min(j, ny - 1);
    const int own = ic + sy * jc, om = ic + sy * max(jc - 1, 0), op = ic + sy * min(jc + 1, ny - 1);
    const int xl = max(ic - 1, 0) + sy * jc, xr = min(ic + W, nx - 1) + sy * jc;
    const bool last = i4 + W >= nx;   // the row's last cell is this thread's: its x+ ghost is itself
    const C ihx = LP<C>::ih2a(L, 0), ihy = LP<C>::ih2a(L, 1), ihz = LP<C>::ih2a(L, 2);
    const C dg = LP<C>::diag(L), wiD = LP<C>::wJ(L) * LP<C>::iD(L);
    // the functor's pointers in registers for the whole march
    const TI* const ein = this->ein;
    const TI* const r = this->r;
    TI* const eout = this->eout;
    double* const p = this->p;
    const uint16_t* const nbf = L.nbf;
    using R = RawW<TI, W>;
    typename R::T em = R::load(ein, max(k0 - 1, 0) * sz + own);
    typename R::T ec = R::load(ein, k0 * sz + own);
    typename R::T ep = R::load(ein, min(k0 + 1, nz - 1) * sz + own);
    for (int k = k0; k < k1; ++k) {
        const int base = k * sz;
        uint32_t fs[W];
        const typename R::T ym = R::load(ein, base + om);
        const typename R::T yp = R::load(ein, base + op);
        const typename R::T rr = R::load(r, base + own);
        codes_w<W>(nbf, base + own, fs);
        const C xls = lane == 0 ? to_c<C>(ldg(ein + base + xl)) : (C)0;
        const C xrs = lane == LR - 1 ? to_c<C>(ldg(ein + base + xr)) : (C)0;
        const typename R::T en = R::load(ein, min(k + 2, nz - 1) * sz + own);   // plane after next
        if (k + 3 < k1 + 2 && k + 3 < nz) {   // this row of the plane three ahead
            const int fb = (k + 3) * sz + own;
            l2_prefetch(ein + fb);
            l2_prefetch(r + fb);
            l2_prefetch(nbf + fb);
        }
        // (no L1 prefetch of the next plane here, unlike the residual and inner-product kernels:
        // with two planes a block the sweep measured 2 % faster without it)
        C left = __shfl_up_sync(0xffffffffu, R::get(ec, W - 1), 1, LR);
        C right = __shfl_down_sync(0xffffffffu, R::get(ec, 0), 1, LR);
        if (lane == 0) left = xls;
        if (lane == LR - 1) right = xrs;
        if (last) right = R::get(ec, W - 1);
        C v[W];
        uint32_t any = 0u;   // solid (bit 12) or irregular (bit 13) anywhere among the W cells
#pragma unroll
        for (int t = 0; t < W; ++t) any |= fs[t];
        if (!(any & 0x3000u)) {
            // every cell fluid, each ghost the clamped in-grid load: the plain stencil
#pragma unroll
            for (int t = 0; t < W; ++t) {
                const C eP = R::get(ec, t);
                const C xm = t == 0 ? left : R::get(ec, t - 1), xp = t == W - 1 ? right : R::get(ec, t + 1);
                C s = (xm + xp) * ihx;
                s = fma(R::get(ym, t) + R::get(yp, t), ihy, s);
                s = fma(R::get(em, t) + R::get(ep, t), ihz, s);
                v[t] = fma(wiD, R::get(rr, t) - fma(dg, eP, -s), eP);
            }
        } else {
#pragma unroll
            for (int t = 0; t < W; ++t) {
                const C eP = R::get(ec, t);
                const C xm = t == 0 ? left : R::get(ec, t - 1), xp = t == W - 1 ? right : R::get(ec, t + 1);
                const C zm = R::get(em, t), zp = R::get(ep, t), ya = R::get(ym, t), yb = R::get(yp, t);
                C A;
                if (!((fs[t] >> 13) & 1u)) {
                    C s = (xm + xp) * ihx;
                    s = fma(ya + yb, ihy, s);
                    s = fma(zm + zp, ihz, s);
                    A = fma(dg, eP, -s);
                } else {
                    A = A7_general<C>(L, fs[t], eP, xm, xp, ya, yb, zm, zp);
                }
                v[t] = is_solid(fs[t]) ? (C)0 : fma(wiD, R::get(rr, t) - A, eP);
            }
        }
        if (in) {
            if (MODE == 0) {
                VecW<TI, W>::store(eout, base + own, v);
            } else if (MODE == 2) {
                VecW<float, W>::store(z32, base + own, v);
            } else {   // p (double-float pairs) += the correction, two cells per 16 bytes
                float4* pp = reinterpret_cast<float4*>(p + base + own);
#pragma unroll
                for (int h = 0; h < W / 2; ++h) {
                    float4 a = pp[h];
                    if (!is_solid(fs[2 * h])) {
                        const float2 x = pp_plus(make_float2(a.x, a.y), v[2 * h]);
                        a.x = x.x;
                        a.y = x.y;
                    }
                    if (!is_solid(fs[2 * h + 1])) {
                        const float2 x = pp_plus(make_float2(a.z, a.w), v[2 * h + 1]);
                        a.z = x.x;
                        a.w = x.y;
                    }
                    pp[h] = a;
                }
            }
        }
        em = ec;
        ec = ep;
        ep = en;
    }
}

// The last block of a flexible-CG inner-product pass: sums all blocks'
// partials in a fixed order (thread t: blocks t, t + NT, ...; then a fixed
// shuffle tree and a fixed sum over warps) and sets beta, alpha and the kept
// (d, A d).  Out of line: it runs once per launch and would otherwise hold
// registers in every block.
template <int NT>
__device__ __noinline__ void fcg_finish(const double* partials, int nblk, SolveState* st, bool have,
                                        double (*red)[NT / 32]) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int x = tid; x < nblk; x += NT) {
        const double2 u = __ldcg(reinterpret_cast<const double2*>(partials + 4 * x));
        const double2 v = __ldcg(reinterpret_cast<const double2*>(partials + 4 * x + 2));
        a[0] += u.x;
        a[1] += u.y;
        a[2] += v.x;
        a[3] += v.y;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m)
        for (int off = 16; off > 0; off >>= 1) a[m] += __shfl_xor_sync(0xffffffffu, a[m], off);
    __syncthreads();
    if ((tid & 31) == 0)
        for (int m = 0; m < 4; ++m) red[m][tid >> 5] = a[m];
    __syncthreads();
    if (tid == 0) {
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        for (int m = 0; m < 4; ++m)
            for (int w = 0; w < NT / 32; ++w) t[m] += red[m][w];
        double beta = (have && st->g_dq > 0.0) ? t[1] / st->g_dq : 0.0;
        double dq = t[0] - beta * t[1];
        if (!(dq > 0.0)) {   // restart along z alone
            beta = 0.0;
            dq = t[0];
        }
        st->g_beta = beta;
        st->g_alpha = dq > 0.0 ? (t[2] - beta * t[3]) / dq : 0.0;
        st->g_dq = dq;
        st->g_valid = 1;
        st->g_counter = 0u;
    }
}

// the four sums of one block (each thread's in s) into partials; the last
// block to finish completes the pass (fcg_finish)
template <int NT, class T>
__device__ __forceinline__ void fcg_reduce(T (&s)[4], double* partials, SolveState* st, bool have,
                                           const BlockAt& at) {
    __shared__ double red[4][NT / 32];
    __shared__ bool last;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
#pragma unroll
    for (int m = 0; m < 4; ++m)
        for (int off = 16; off > 0; off >>= 1) s[m] += __shfl_xor_sync(0xffffffffu, s[m], off);
    if ((tid & 31) == 0)
        for (int m = 0; m < 4; ++m) red[m][tid >> 5] = (double)s[m];
    __syncthreads();
    const int nblk = at.g.x * at.g.y * at.g.z;
    if (tid == 0) {
        const int bid = at.b.x + at.g.x * (at.b.y + at.g.y * at.b.z);
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < NT / 32; ++w)
            for (int m = 0; m < 4; ++m) t[m] += red[m][w];
        reinterpret_cast<double2*>(partials + 4 * bid)[0] = make_double2(t[0], t[1]);
        reinterpret_cast<double2*>(partials + 4 * bid)[1] = make_double2(t[2], t[3]);
        __threadfence();
        last = atomicAdd(&st->g_counter, 1u) == (unsigned)nblk - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    fcg_finish<NT>(partials, nblk, st, have, red);
}

// ------------------------------------------------------------------ level 0 residual in float-float
// The reduced-precision cases hold p as double-float pairs (pp_load); this
// path evaluates r = b - A p without the FP64 pipe (1/64 of the FP32 rate
// here): the stencil runs in double-float arithmetic (Dekker's error-free sum
// and FMA-based product), about 2^-48 relative accuracy.  As a difference
// form, A p = sum_a ih2_a ((P - g_lo) + (P - g_hi)) with g the neighbour
// (code 0), P (zero-gradient: no term) or -P (zero-value: 2P), which equals
// both branches of A7.
__device__ __forceinline__ void ff_load4(const double* p, int c, FF (&o)[4]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p + c));
    const float4 b = __ldg(reinterpret_cast<const float4*>(p + c) + 1);
    o[0] = {a.x, a.y};
    o[1] = {a.z, a.w};
    o[2] = {b.x, b.y};
    o[3] = {b.z, b.w};
}

// P - ghost across one face: the neighbour (code 0), none (1) or 2P (2)
__device__ __forceinline__ FF ff_face(uint32_t code, FF P, FF nb) {
    const FF d = ff_add(P, ff_neg(nb));
    if (code == 0u) return d;
    if (code == 1u) return {0.0f, 0.0f};
    return {2.0f * P.h, 2.0f * P.l};
}

// one axis of A p at a regular cell: ih (2P - a - b), the neighbours' sum and
// the difference by error-free sums, the products' low parts by FMA; the
// result is left unnormalised (its low part is small against the high part's
// inputs, which is all the sums below need)
__device__ __forceinline__ FF ff_axis(FF P, FF a, FF b, FF ih) {
    const FF s = ff_two_sum(a.h, b.h);
    const float sl = s.l + (a.l + b.l);
    const FF d = ff_two_sum(2.0f * P.h, -s.h);
    const float dl = d.l + (2.0f * P.l - sl);
    const float p = d.h * ih.h;
    float e = fmaf(d.h, ih.h, -p);
    e = fmaf(d.h, ih.l, e);
    e = fmaf(dl, ih.h, e);
    return {p, e};
}

// b - A p rounded to FP32 at a regular cell (code bit 13 clear: the clamped
// loads are the ghosts), ih2 = 0 on a collapsed axis
__device__ __forceinline__ float ff_resid_regular(float b, FF P, FF xm, FF xp, FF ym, FF yp, FF zm, FF zp, FF ihx,
                                                  FF ihy, FF ihz) {
    const FF ax = ff_axis(P, xm, xp, ihx), ay = ff_axis(P, ym, yp, ihy), az = ff_axis(P, zm, zp, ihz);
    const FF t = ff_two_sum(ax.h, ay.h);
    const FF t2 = ff_two_sum(t.h, az.h);
    const float al = (t.l + t2.l) + (ax.l + ay.l + az.l);
    const FF u = ff_two_sum(b, -t2.h);
    return u.h + (u.l - al);
}

// Two cells' double-float values side by side (cells 2q and 2q + 1 of a thread's four) and
// the arithmetic of ff_axis / ff_resid_regular on both at once with the packed FP32
// instructions (add / mul / fma .f32x2: one instruction for the pair, each lane rounded as the
// scalar instruction rounds it).  A difference a - b is fma(b, -1, a), rounded once like the
// scalar subtraction; a negation is a product by -1 (exact).
struct FF2 {
    float2 h, l;
};
__device__ __forceinline__ float2 p2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 p2neg(float2 a) { return __fmul2_rn(a, make_float2(-1.0f, -1.0f)); }
__device__ __forceinline__ FF2 ff2_two_sum(float2 a, float2 b) {
    const float2 s = p2add(a, b);
    const float2 bb = p2sub(s, a);
    return {s, p2add(p2sub(a, p2sub(s, bb)), p2sub(b, bb))};
}
__device__ __forceinline__ FF2 ff2_axis(FF2 P, FF2 a, FF2 b, float2 ihh, float2 ihl) {
    const FF2 s = ff2_two_sum(a.h, b.h);
    const float2 sl = p2add(s.l, p2add(a.l, b.l));
    const FF2 d = ff2_two_sum(p2add(P.h, P.h), p2neg(s.h));
    const float2 dl = p2add(d.l, p2sub(p2add(P.l, P.l), sl));
    const float2 p = __fmul2_rn(d.h, ihh);
    float2 e = __ffma2_rn(d.h, ihh, p2neg(p));
    e = __ffma2_rn(d.h, ihl, e);
    e = __ffma2_rn(dl, ihh, e);
    return {p, e};
}
__device__ __forceinline__ float2 ff2_resid_regular(float2 b, FF2 P, FF2 xm, FF2 xp, FF2 ym, FF2 yp, FF2 zm, FF2 zp,
                                                    const float2 ih[6]) {
    const FF2 ax = ff2_axis(P, xm, xp, ih[0], ih[1]), ay = ff2_axis(P, ym, yp, ih[2], ih[3]);
    const FF2 az = ff2_axis(P, zm, zp, ih[4], ih[5]);
    const FF2 t = ff2_two_sum(ax.h, ay.h);
    const FF2 t2 = ff2_two_sum(t.h, az.h);
    const float2 al = p2add(p2add(t.l, t2.l), p2add(p2add(ax.l, ay.l), az.l));
    const FF2 u = ff2_two_sum(b, p2neg(t2.h));
    return p2add(u.h, p2sub(u.l, al));
}
__device__ __forceinline__ FF2 ff2_of(const FF& a, const FF& b) { return {make_float2(a.h, b.h), make_float2(a.l, b.l)}; }

// the same for any cell, each face's ghost chosen by its code (out of line: rare)
__device__ __noinline__ float ff_resid_general(uint32_t f, float b, FF P, FF xm, FF xp, FF ym, FF yp, FF zm, FF zp,
                                               FF ihx, FF ihy, FF ihz) {
    const FF ax = ff_mul(ff_add(ff_face(f & 3u, P, xm), ff_face((f >> 2) & 3u, P, xp)), ihx);
    const FF ay = ff_mul(ff_add(ff_face((f >> 4) & 3u, P, ym), ff_face((f >> 6) & 3u, P, yp)), ihy);
    const FF az = ff_mul(ff_add(ff_face((f >> 8) & 3u, P, zm), ff_face((f >> 10) & 3u, P, zp)), ihz);
    const FF A = ff_add(ff_add(ax, ay), az);
    const FF rr = ff_add(FF{b, 0.0f}, ff_neg(A));
    return rr.h + rr.l;
}

template <class TI> __device__ __forceinline__ float round_inner(float v) { return v; }
template <> __device__ __forceinline__ float round_inner<__nv_bfloat16>(float v) {
    return __bfloat162float(__float2bfloat16_rn(v));
}

// r = b - A p (float-float), r^2 and b^2, the first pre-sweep e = w_J r / D;
// four x cells per thread and a z march (the sweep's layout).  FP32 b, nx % 4 = 0.
template <class TI>
struct Resid0V4K {
    static constexpr int kThreads = TX * TY;
    static constexpr int kMinBlocks = 3;       // at most 80 registers
    // the batched form needs more (BF16 spills at 80; with FP32 corrections 80 registers, three
    // blocks per SM, measured slower on 64 channels than 128 and two)
    static constexpr int kMinBlocksMany = 2;
    LevelDev L;
    const double* p;
    const float* b;
    TI* r;
    TI* e;
    double* partials;
    SolveState* st;
    int zc;    // planes per block
    int lrl;   // log2 of the lanes per row segment (as in SweepVK)
    __device__ bool live() const { return st->active != 0; }
    __device__ int run(const BlockAt& at) const;
};

template <class TI>
__device__ int Resid0V4K<TI>::run(const BlockAt& at) const {
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int LR = 1 << lrl, lane = threadIdx.x & (LR - 1), sub = threadIdx.x >> lrl;
    const int i4 = at.b.x * (4 * LR) + lane * 4, j = ((at.b.y * TY + threadIdx.y) << (5 - lrl)) + sub;
    const int k0 = at.b.z * zc, k1 = min(nz, k0 + zc);
    const bool in = i4 < nx && j < ny;
    const int sy = nx, sz = nx * ny;
    const int ic = min(i4, nx - 4), jc = min(j, ny - 1);
    const int own = ic + sy * jc, om = ic + sy * max(jc - 1, 0), op = ic + sy * min(jc + 1, ny - 1);
    const int xl = max(ic - 1, 0) + sy * jc, xr = min(ic + 4, nx - 1) + sy * jc;
    const bool lastc = i4 + 4 >= nx;
    const FF ihx = {L.ih2af[0], L.ih2alo[0]}, ihy = {L.ih2af[1], L.ih2alo[1]}, ihz = {L.ih2af[2], L.ih2alo[2]};
    const float2 ih2[6] = {make_float2(ihx.h, ihx.h), make_float2(ihx.l, ihx.l), make_float2(ihy.h, ihy.h),
                           make_float2(ihy.l, ihy.l), make_float2(ihz.h, ihz.h), make_float2(ihz.l, ihz.l)};
    const float wJ = LP<float>::wJ(L), iD = LP<float>::iD(L);
    const double* const pp = this->p;
    const uint16_t* const nbf = L.nbf;
    FF em[4], ec[4], ep[4];
    ff_load4(pp, max(k0 - 1, 0) * sz + own, em);
    ff_load4(pp, k0 * sz + own, ec);
    ff_load4(pp, min(k0 + 1, nz - 1) * sz + own, ep);
    float r2 = 0.0f, b2 = 0.0f;
    for (int k = k0; k < k1; ++k) {
        const int base = k * sz;
        FF ym[4], yp[4], en[4];
        ff_load4(pp, base + om, ym);
        ff_load4(pp, base + op, yp);
        const float4 bq = __ldg(reinterpret_cast<const float4*>(b + base + own));
        const uint2 fw = __ldg(reinterpret_cast<const uint2*>(nbf + base + own));
        const FF xls = lane == 0 ? pp_load(pp, base + xl) : FF{0.0f, 0.0f};
        const FF xrs = lane == LR - 1 ? pp_load(pp, base + xr) : FF{0.0f, 0.0f};
        ff_load4(pp, min(k + 2, nz - 1) * sz + own, en);
        if (k + 3 < k1 + 2 && k + 3 < nz) {   // this row of the plane three ahead
            const int fb = (k + 3) * sz + own;
            l2_prefetch(pp + fb);
            l2_prefetch(pp + fb + 2);
            l2_prefetch(b + fb);
            l2_prefetch(nbf + fb);
        }
        if (k + 1 < k1) {   // the next plane's rows into L1 (their loads open the next iteration)
            const int nb = (k + 1) * sz;
            l1_prefetch(pp + nb + om);
            l1_prefetch(pp + nb + op);
            l1_prefetch(b + nb + own);
            l1_prefetch(nbf + nb + own);
        }
        FF left = {__shfl_up_sync(0xffffffffu, ec[3].h, 1, LR), __shfl_up_sync(0xffffffffu, ec[3].l, 1, LR)};
        FF right = {__shfl_down_sync(0xffffffffu, ec[0].h, 1, LR), __shfl_down_sync(0xffffffffu, ec[0].l, 1, LR)};
        if (lane == 0) left = xls;
        if (lane == LR - 1) right = xrs;
        if (lastc) right = ec[3];
        const FF xs[6] = {left, ec[0], ec[1], ec[2], ec[3], right};
        const uint32_t fs[4] = {fw.x & 0xffffu, fw.x >> 16, fw.y & 0xffffu, fw.y >> 16};
        const float bb[4] = {bq.x, bq.y, bq.z, bq.w};
        // b - A p: a pair of regular cells (code bit 13 clear) in the packed form, any other cell alone
        float rfs[4];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int t0 = 2 * q, t1 = t0 + 1;
            if (!(((fs[t0] | fs[t1]) >> 13) & 1u)) {
                const float2 rr = ff2_resid_regular(
                    make_float2(bb[t0], bb[t1]), ff2_of(xs[t0 + 1], xs[t1 + 1]), ff2_of(xs[t0], xs[t1]),
                    ff2_of(xs[t0 + 2], xs[t1 + 2]), ff2_of(ym[t0], ym[t1]), ff2_of(yp[t0], yp[t1]),
                    ff2_of(em[t0], em[t1]), ff2_of(ep[t0], ep[t1]), ih2);
                rfs[t0] = rr.x;
                rfs[t1] = rr.y;
            } else {
#pragma unroll
                for (int t = t0; t <= t1; ++t)
                    rfs[t] = !((fs[t] >> 13) & 1u)
                                 ? ff_resid_regular(bb[t], xs[t + 1], xs[t], xs[t + 2], ym[t], yp[t], em[t], ep[t], ihx,
                                                    ihy, ihz)
                                 : ff_resid_general(fs[t], bb[t], xs[t + 1], xs[t], xs[t + 2], ym[t], yp[t], em[t],
                                                    ep[t], ihx, ihy, ihz);
            }
        }
        float rv[4], ev[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const uint32_t f = fs[t];
            const float rf = rfs[t];
            const bool fluid = !is_solid(f);
            const float rc = fluid ? round_inner<TI>(rf) : 0.0f;
            rv[t] = rc;
            ev[t] = wJ * rc * iD;
            if (in) {
                r2 = fmaf(rc, rc, r2);
                if (fluid) b2 = fmaf(bb[t], bb[t], b2);
            }
        }
        if (in) {
            Vec4<TI>::store(r, base + own, rv);
            Vec4<TI>::store(e, base + own, ev);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            em[t] = ec[t];
            ec[t] = ep[t];
            ep[t] = en[t];
        }
    }
    // block sums in FP64, then the last block's fixed-order reduction and the stopping rule
    __shared__ double red[2][kThreads / 32];
    __shared__ bool last;
    const int tid = threadIdx.x + TX * threadIdx.y;
    double s0 = (double)r2, s1 = (double)b2;
    for (int off = 16; off > 0; off >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, off);
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = s0;
        red[1][tid >> 5] = s1;
    }
    __syncthreads();
    const int nblk = at.g.x * at.g.y * at.g.z;
    if (tid == 0) {
        const int bid = at.b.x + at.g.x * (at.b.y + at.g.y * at.b.z);
        double a0 = 0.0, a1 = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            a0 += red[0][w];
            a1 += red[1][w];
        }
        reinterpret_cast<double2*>(partials)[bid] = make_double2(a0, a1);
        __threadfence();
        last = atomicAdd(&st->counter, 1u) == (unsigned)nblk - 1u;
    }
    __syncthreads();
    if (!last) return -1;
    __threadfence();
    return resid0_finish<kThreads>(partials, nblk, st, red);
}

// The flexible-CG inner products with W x cells per thread and a z march
// (the sweep's layout and neighbour scheme): products, the thread's and the
// warp's sums in FP32, block and grid sums in FP64.  Needs nx % W = 0.
// (TR: storage of r; TZ: storage of z and the kept direction, FP32 on BF16 levels)
template <class TR, class TZ, int W>
struct FcgDotVK {
    static constexpr int kThreads = TX * TY;
    static constexpr int kMinBlocks = 4;       // at most 64 registers
    static constexpr int kMinBlocksMany = 3;   // the batched form: at most 80 registers
    LevelDev L;
    const TZ* z;
    const TR* r;
    const TZ* dp;
    double* partials;
    SolveState* st;
    int zc;    // planes per block
    int lrl;   // log2 of the lanes per row segment (as in SweepVK)
    __device__ bool live() const { return st->active != 0; }
    __device__ void run(const BlockAt& at) const;
};

template <class TR, class TZ, int W>
__device__ void FcgDotVK<TR, TZ, W>::run(const BlockAt& at) const {
    using C = float;
    using R = RawW<TZ, W>;
    using RR = RawW<TR, W>;
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int LR = 1 << lrl, lane = threadIdx.x & (LR - 1), sub = threadIdx.x >> lrl;
    const int i4 = at.b.x * (W * LR) + lane * W, j = ((at.b.y * TY + threadIdx.y) << (5 - lrl)) + sub;
    const int k0 = at.b.z * zc, k1 = min(nz, k0 + zc);
    const bool in = i4 < nx && j < ny;
    const int sy = nx, sz = nx * ny;
    const int ic = min(i4, nx - W), jc = min(j, ny - 1);
    const int own = ic + sy * jc, om = ic + sy * max(jc - 1, 0), op = ic + sy * min(jc + 1, ny - 1);
    const int xl = max(ic - 1, 0) + sy * jc, xr = min(ic + W, nx - 1) + sy * jc;
    const bool lastc = i4 + W >= nx;
    const C ihx = LP<C>::ih2a(L, 0), ihy = LP<C>::ih2a(L, 1), ihz = LP<C>::ih2a(L, 2);
    const C dg = LP<C>::diag(L);
    const bool have = st->g_valid != 0;
    const TZ* const zz = this->z;
    const uint16_t* const nbf = L.nbf;
    typename R::T em = R::load(zz, max(k0 - 1, 0) * sz + own);
    typename R::T ec = R::load(zz, k0 * sz + own);
    typename R::T ep = R::load(zz, min(k0 + 1, nz - 1) * sz + own);
    C a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int k = k0; k < k1; ++k) {
        const int base = k * sz;
        const typename R::T ym = R::load(zz, base + om);
        const typename R::T yp = R::load(zz, base + op);
        const typename RR::T rr = RR::load(r, base + own);
        typename R::T dd = {};
        if (have) dd = R::load(dp, base + own);
        uint32_t fs[W];
        codes_w<W>(nbf, base + own, fs);
        const C xls = lane == 0 ? to_c<C>(ldg(zz + base + xl)) : (C)0;
        const C xrs = lane == LR - 1 ? to_c<C>(ldg(zz + base + xr)) : (C)0;
        const typename R::T en = R::load(zz, min(k + 2, nz - 1) * sz + own);
        if (k + 3 < k1 + 2 && k + 3 < nz) {   // this row of the plane three ahead
            const int fb = (k + 3) * sz + own;
            l2_prefetch(zz + fb);
            l2_prefetch(r + fb);
            l2_prefetch(nbf + fb);
            if (have) l2_prefetch(dp + fb);
        }
        if (k + 1 < k1) {   // the next plane's rows into L1 (their loads open the next iteration)
            const int nb = (k + 1) * sz;
            l1_prefetch(zz + nb + om);
            l1_prefetch(zz + nb + op);
            l1_prefetch(r + nb + own);
            l1_prefetch(nbf + nb + own);
            if (have) l1_prefetch(dp + nb + own);
        }
        C left = __shfl_up_sync(0xffffffffu, R::get(ec, W - 1), 1, LR);
        C right = __shfl_down_sync(0xffffffffu, R::get(ec, 0), 1, LR);
        if (lane == 0) left = xls;
        if (lane == LR - 1) right = xrs;
        if (lastc) right = R::get(ec, W - 1);
        uint32_t any = 0u;   // solid (bit 12) or irregular (bit 13) anywhere among the W cells
#pragma unroll
        for (int t = 0; t < W; ++t) any |= fs[t];
        if (in) {
#pragma unroll
            for (int t = 0; t < W; ++t) {
                const bool plain = !(any & 0x3000u);   // every cell fluid with in-grid ghosts
                if (!plain && is_solid(fs[t])) continue;
                const C eP = R::get(ec, t);
                const C xm = t == 0 ? left : R::get(ec, t - 1), xp = t == W - 1 ? right : R::get(ec, t + 1);
                const C ya = R::get(ym, t), yb = R::get(yp, t), za = R::get(em, t), zb = R::get(ep, t);
                C A;
                if (plain || !((fs[t] >> 13) & 1u)) {
                    C q = (xm + xp) * ihx;
                    q = fma(ya + yb, ihy, q);
                    q = fma(za + zb, ihz, q);
                    A = fma(dg, eP, -q);
                } else {
                    A = A7_general<C>(L, fs[t], eP, xm, xp, ya, yb, za, zb);
                }
                const C d = R::get(dd, t), rv = RR::get(rr, t);
                a0 = fma(eP, A, a0);
                a1 = fma(A, d, a1);
                a2 = fma(rv, eP, a2);
                a3 = fma(rv, d, a3);
            }
        }
        em = ec;
        ec = ep;
        ep = en;
    }
    float s[4] = {a0, a1, a2, a3};   // FP32 within a warp, FP64 from the warp sums on
    fcg_reduce<kThreads>(s, partials, st, have, at);
}

// d = z - beta d_prev, p += alpha d (fluid cells), d kept: W consecutive
// cells per thread, one-dimensional grid.  Needs N % W = 0.
template <class TZ, int W>
struct FcgUpdVK {
    static constexpr int kThreads = 256;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    LevelDev L;
    const TZ* z;
    TZ* dp;
    double* p;
    const SolveState* st;
    __device__ bool live() const { return st->active != 0; }
    __device__ void run(const BlockAt& at) const {
        const int c = W * (at.b.x * kThreads + threadIdx.x);
        if (c >= L.N) return;
        const float alpha = (float)st->g_alpha, beta = (float)st->g_beta;
        float zv[W], dv[W];
#pragma unroll
        for (int t = 0; t < W; ++t) dv[t] = 0.f;
        VecW<TZ, W>::load(z, c, zv);
        if (beta != 0.f) VecW<TZ, W>::load_rw(dp, c, dv);
        uint32_t fs[W];
        codes_w<W>(L.nbf, c, fs);
        float d[W];
#pragma unroll
        for (int t = 0; t < W; ++t) d[t] = fma(-beta, dv[t], zv[t]);
        VecW<TZ, W>::store(dp, c, d);
        float4* pp = reinterpret_cast<float4*>(p + c);   // p as double-float pairs, two cells per 16 bytes
#pragma unroll
        for (int h = 0; h < W / 2; ++h) {
            float4 u = pp[h];
            if (!is_solid(fs[2 * h])) {
                const float2 x = pp_plus(make_float2(u.x, u.y), alpha * d[2 * h]);
                u.x = x.x;
                u.y = x.y;
            }
            if (!is_solid(fs[2 * h + 1])) {
                const float2 x = pp_plus(make_float2(u.z, u.w), alpha * d[2 * h + 1]);
                u.z = x.x;
                u.w = x.y;
            }
            pp[h] = u;
        }
    }
};
// Trilinear prolongation and correction, W consecutive x cells per thread (4 or
// 8): a lane's fine cells have the H = W/2 coarse parents I0 = i/2 .. I0 + H - 1
// (one load per coarse row).  The four coarse rows around the fine row (parent
// and neighbour along y and z, ghosts signed) are combined with their y-z
// weights first, then interpolated along x, the x neighbours I0 - 1 and I0 + H
// coming from the adjacent lanes.  Per fine cell and axis the weights are 3/4
// for the parent and 1/4 for the neighbour on the cell's side (Eq.
// prolongation); a neighbour beyond a domain face is the coarse cell's ghost,
// as in prolong_at.  Needs the x and y axes active and nx % W = 0.
template <class TI, int W>
struct ProlongVK {
    static constexpr int kThreads = TX * TY;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    static constexpr int kMinBlocks = 4;
    LevelDev Lf, Lc;
    const TI* ec;
    TI* e;
    const SolveState* st;
    int zc;    // planes per block
    int lrl;   // log2 of the lanes per row segment (as in SweepVK)
    __device__ bool live() const { return st->active != 0; }   // batched: skip a converged case
    __device__ void run(const BlockAt& at) const;
};

// a coarse value across a ghost row or plane: negated for each zero-value face among them
__device__ __forceinline__ float ghost_signed(uint32_t code, bool gy, int sy, bool gz, int sz, float v) {
    bool neg = gy && ((code >> (2 * (2 + sy))) & 3u) == 2u;
    neg ^= gz && ((code >> (2 * (4 + sz))) & 3u) == 2u;
    return neg ? -v : v;
}

template <class TI, int W>
__device__ void ProlongVK<TI, W>::run(const BlockAt& at) const {
    using C = float;
    constexpr int H = W / 2;   // coarse cells under a thread's W fine cells
    using RC = RawW<TI, H>;
    const int nx = Lf.n[0], ny = Lf.n[1], nz = Lf.n[2];
    const int NX = Lc.n[0], NY = Lc.n[1], NZ = Lc.n[2];
    const int LR = 1 << lrl, lane = threadIdx.x & (LR - 1), sub = threadIdx.x >> lrl;
    const int i4 = at.b.x * (W * LR) + lane * W, j = ((at.b.y * TY + threadIdx.y) << (5 - lrl)) + sub;
    const int k0 = at.b.z * zc, k1 = min(nz, k0 + zc);
    const bool in = i4 < nx && j < ny;
    const bool last = i4 + W >= nx;   // the row's last coarse cell is this thread's: its x+ neighbour is a ghost
    const int ic = min(i4, nx - W), jc = min(j, ny - 1);
    const bool first = ic == 0;       // and its first: the x- neighbour is a ghost
    const int I0 = ic >> 1;
    // the y neighbour of the parent row; beyond a domain face it is the ghost row (the parent
    // row's cells, each signed by its own face code)
    const int Pj = jc >> 1, qj = Pj + ((jc & 1) ? 1 : -1);
    const bool outJ = qj < 0 || qj >= NY;
    const int Qj = outJ ? Pj : qj, sJ = qj < 0 ? 0 : 1;
    const bool zact = Lf.active[2] != 0;
    const TI* const ecp = ec;
    TI* const ep = e;
    const uint16_t* const nbf = Lf.nbf;
    const uint16_t* const cnbf = Lc.nbf;
    for (int k = k0; k < k1; ++k) {
        const int Pk = zact ? (k >> 1) : k;
        const int qk = zact ? Pk + ((k & 1) ? 1 : -1) : k;
        const bool outK = qk < 0 || qk >= NZ;
        const int Qk = outK ? Pk : qk, sK = qk < 0 ? 0 : 1;
        const C wz0 = zact ? (C)0.75 : (C)1, wz1 = zact ? (C)0.25 : (C)0;
        // the four coarse rows (parent and neighbour along y and z, ghosts signed) combined with
        // their y-z weights into one row first, then the x interpolation and the shuffles once
        C cvc[H], lc = (C)0, rc = (C)0, lg = (C)0, rg = (C)0;
#pragma unroll
        for (int h = 0; h < H; ++h) cvc[h] = (C)0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int jj = (q & 1) ? Qj : Pj, kk = (q & 2) ? Qk : Pk;
            const bool gy = (q & 1) && outJ, gz = (q & 2) && outK;
            const C w = ((q & 1) ? (C)0.25 : (C)0.75) * ((q & 2) ? wz1 : wz0);
            const int row = NX * (jj + NY * kk);
            const typename RC::T raw = RC::load(ecp, row + I0);
            C cv[H];
#pragma unroll
            for (int h = 0; h < H; ++h) cv[h] = RC::get(raw, h);
            C lft = lane == 0 ? to_c<C>(ldg(ecp + row + max(I0 - 1, 0))) : (C)0;
            C rgt = lane == LR - 1 ? to_c<C>(ldg(ecp + row + min(I0 + H, NX - 1))) : (C)0;
            uint32_t cw[H];   // the codes of the coarse cells (only where a ghost is formed)
#pragma unroll
            for (int h = 0; h < H; ++h) cw[h] = 0u;
            if (gy || gz || first || last) codes_w<H>(cnbf, row + I0, cw);
            if (gy || gz) {
#pragma unroll
                for (int h = 0; h < H; ++h) cv[h] = ghost_signed(cw[h], gy, sJ, gz, sK, cv[h]);
                if (lane == 0 && !first) lft = ghost_signed(__ldg(cnbf + row + I0 - 1), gy, sJ, gz, sK, lft);
                if (lane == LR - 1 && !last) rgt = ghost_signed(__ldg(cnbf + row + I0 + H), gy, sJ, gz, sK, rgt);
            }
#pragma unroll
            for (int h = 0; h < H; ++h) cvc[h] = fma(w, cv[h], cvc[h]);
            lc = fma(w, lft, lc);
            rc = fma(w, rgt, rc);
            if (first) lg = fma(w, (cw[0] & 3u) == 2u ? -cv[0] : cv[0], lg);                       // x- ghost of I0
            if (last) rg = fma(w, ((cw[H - 1] >> 2) & 3u) == 2u ? -cv[H - 1] : cv[H - 1], rg);   // x+ of the last
        }
        C left = __shfl_up_sync(0xffffffffu, cvc[H - 1], 1, LR);
        C right = __shfl_down_sync(0xffffffffu, cvc[0], 1, LR);
        if (lane == 0) left = lc;
        if (lane == LR - 1) right = rc;
        if (first) left = lg;
        if (last) right = rg;
        C add[W];
#pragma unroll
        for (int t = 0; t < W; ++t) {
            const int h = t >> 1;
            const C nb = (t & 1) ? (h == H - 1 ? right : cvc[h + 1]) : (h == 0 ? left : cvc[h - 1]);
            add[t] = (C)0.75 * cvc[h] + (C)0.25 * nb;
        }
        if (in) {
            const int c = ic + nx * (jc + ny * k);
            C v[W];
            uint32_t fs[W];
            VecW<TI, W>::load_rw(ep, c, v);
            codes_w<W>(nbf, c, fs);
#pragma unroll
            for (int t = 0; t < W; ++t)
                if (!is_solid(fs[t])) v[t] += add[t];
            VecW<TI, W>::store(ep, c, v);
        }
    }
}

// Residual and restriction, W x cells per thread: a thread owns the fine
// cells i4..i4+W-1 of rows 2J, 2J+1 and planes 2K, 2K+1 (2D: plane K) and
// writes the W/2 coarse cells I0 = i4/2 .. (mean of their children's r - A e,
// Eq. restriction).  Rows j +- 1 and planes k +- 1 are loaded whole, x
// neighbours by shuffles.  Needs x and y active, nx % W = 0, ny even.
template <class TI, int W>
struct RRVK {
    static constexpr int kThreads = TX * TY;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    static constexpr int kMinBlocks = 4;
    LevelDev Lf, Lc;
    const TI* e;
    const TI* r;
    TI* rc;
    TI* ec0;   // the coarse level's first sweep, or null
    int lrl;   // log2 of the lanes per row segment (as in SweepVK)
    const SolveState* st;
    __device__ bool live() const { return st->active != 0; }   // batched: skip a converged case
    __device__ void run(const BlockAt& at) const;
};

template <class TI, int W>
__device__ void RRVK<TI, W>::run(const BlockAt& at) const {
    using C = float;
    using R = RawW<TI, W>;
    constexpr int H = W / 2;
    const int nx = Lf.n[0], ny = Lf.n[1], nz = Lf.n[2];
    const int NX = Lc.n[0], NY = Lc.n[1];
    const int LR = 1 << lrl, lane = threadIdx.x & (LR - 1), sub = threadIdx.x >> lrl;
    const int i4 = at.b.x * (W * LR) + lane * W, J = ((at.b.y * TY + threadIdx.y) << (5 - lrl)) + sub, K = at.b.z;
    const bool in = i4 < nx && J < NY;
    const bool last = i4 + W >= nx;
    const int fz = Lf.active[2] ? 2 : 1;
    const int ic = min(i4, nx - W), Jc = min(J, NY - 1);
    const int ja = 2 * Jc, jb = ja + 1, jm = max(ja - 1, 0), jp = min(jb + 1, ny - 1);
    const int sy = nx, sz = nx * ny;
    const C ihx = LP<C>::ih2a(Lf, 0), ihy = LP<C>::ih2a(Lf, 1), ihz = LP<C>::ih2a(Lf, 2);
    const C dg = LP<C>::diag(Lf);
    const TI* const ep = e;
    const TI* const rp = r;
    const uint16_t* const nbf = Lf.nbf;
    auto at_ = [&](int jj, int kk) { return ic + sy * jj + sz * kk; };
    C s[H];   // sums of the coarse cells I0 .. I0 + H - 1
#pragma unroll
    for (int h = 0; h < H; ++h) s[h] = (C)0;
    for (int dz = 0; dz < fz; ++dz) {
        const int k = fz * K + dz;
        const int km = max(k - 1, 0), kp = min(k + 1, nz - 1);
#pragma unroll
        for (int row = 0; row < 2; ++row) {
            const int jr = row ? jb : ja;
            const typename R::T ec = R::load(ep, at_(jr, k));
            const typename R::T yl = R::load(ep, at_(row ? ja : jm, k));   // row below
            const typename R::T yh = R::load(ep, at_(row ? jp : jb, k));   // row above
            const typename R::T zl = R::load(ep, at_(jr, km));
            const typename R::T zh = R::load(ep, at_(jr, kp));
            const typename R::T rr = R::load(rp, at_(jr, k));
            uint32_t fs[W];
            codes_w<W>(nbf, at_(jr, k), fs);
            const C lx = lane == 0 ? to_c<C>(ldg(ep + max(ic - 1, 0) + sy * jr + sz * k)) : (C)0;
            const C rx = lane == LR - 1 ? to_c<C>(ldg(ep + min(ic + W, nx - 1) + sy * jr + sz * k)) : (C)0;
            C left = __shfl_up_sync(0xffffffffu, R::get(ec, W - 1), 1, LR);
            C right = __shfl_down_sync(0xffffffffu, R::get(ec, 0), 1, LR);
            if (lane == 0) left = lx;
            if (lane == LR - 1) right = rx;
            if (last) right = R::get(ec, W - 1);
#pragma unroll
            for (int t = 0; t < W; ++t) {
                if (is_solid(fs[t])) continue;
                const C eP = R::get(ec, t);
                const C xm = t == 0 ? left : R::get(ec, t - 1), xp = t == W - 1 ? right : R::get(ec, t + 1);
                const C ya = R::get(yl, t), yb = R::get(yh, t), za = R::get(zl, t), zb = R::get(zh, t);
                C A;
                if (!((fs[t] >> 13) & 1u)) {
                    C sa = (xm + xp) * ihx;
                    sa = fma(ya + yb, ihy, sa);
                    sa = fma(za + zb, ihz, sa);
                    A = fma(dg, eP, -sa);
                } else {
                    A = A7_general<C>(Lf, fs[t], eP, xm, xp, ya, yb, za, zb);
                }
                s[t >> 1] += R::get(rr, t) - A;
            }
        }
    }
    if (in) {
        const C inv = (C)1 / (C)(4 * fz);
        const int o = (ic >> 1) + NX * (Jc + NY * K);
#pragma unroll
        for (int h = 0; h < H; ++h) store_restricted<TI, C>(Lc, rc, ec0, o + h, s[h] * inv);
    }
}

// coarse r = mean of the children's (r - A e): one thread per fine cell (the
// z pair of children in the thread), x / y pairs summed through shared memory.
// Needs x and y active (2 x 2 children in the plane).
template <class TI>
struct RRWalkK {
    static constexpr int kThreads = TX * TY;
    LevelDev Lf, Lc;
    const TI* e;
    const TI* r;
    TI* rc;
    TI* ec0;   // the coarse level's first sweep, or null
    const SolveState* st;
    __device__ bool live() const { return st->active != 0; }   // batched: skip a converged case
    __device__ void run(const BlockAt& at) const;
};

template <class TI>
__device__ void RRWalkK<TI>::run(const BlockAt& at) const {
    using C = typename Acc<TI>::type;
    __shared__ C part[TY][TX + 1];
    const int fz = Lf.active[2] ? 2 : 1;
    Walk w;
    const bool in = walk_setup(Lf, at, fz, w);
    C sum = (C)0;
    if (in) {
        const int nz = Lf.n[2];
        int c = w.i + w.sy * w.j + w.sz * w.k0;
        for (int kk = 0; kk < fz; ++kk) {
            const int k = w.k0 + kk;
            const uint32_t f = Lf.nbf[c];
            const C eP = to_c<C>(ldg(e + c));
            const C zm = k > 0 ? to_c<C>(ldg(e + c - w.sz)) : eP;
            const C zp = k < nz - 1 ? to_c<C>(ldg(e + c + w.sz)) : eP;
            const C xm = to_c<C>(ldg(e + c + w.im)), xp = to_c<C>(ldg(e + c + w.ip));
            const C ym = to_c<C>(ldg(e + c + w.jm)), yp = to_c<C>(ldg(e + c + w.jp));
            const C rr = to_c<C>(ldg(r + c));
            if (!is_solid(f)) sum += rr - A7<C>(Lf, f, eP, xm, xp, ym, yp, zm, zp);
            c += w.sz;
        }
    }
    part[threadIdx.y][threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x < TX / 2 && threadIdx.y < TY / 2) {
        const int I = at.b.x * (TX / 2) + threadIdx.x, J = at.b.y * (TY / 2) + threadIdx.y;
        if (I < Lc.n[0] && J < Lc.n[1]) {
            const int x = 2 * threadIdx.x, y = 2 * threadIdx.y;
            const C s4 = (part[y][x] + part[y][x + 1]) + (part[y + 1][x] + part[y + 1][x + 1]);
            store_restricted<TI, C>(Lc, rc, ec0, I + Lc.n[0] * (J + Lc.n[1] * (int)at.b.z), s4 / (C)(4 * fz));
        }
    }
}

// ------------------------------------------------------------------ coarse levels in one CTA
// V-cycle over levels lc..L-1 in shared memory: reads r on level lc from
// global memory, writes the correction e on level lc.
// A level's stencil constants in registers for the coarse CTA's cell loops (the level
// descriptions live in shared memory, which the loops also write, so the compiler would reload
// them for every cell), and A e with them: a cell whose face codes are all 0 on three active
// axes takes the six neighbours without the per-face code selects, in the same arithmetic order
// as apply_A_with, so both forms give the same value
template <class C>
struct CtaStencil {
    int sy, sz;
    C ih[3];
    bool act[3];
    bool all3;
};

template <class C>
__device__ __forceinline__ CtaStencil<C> cta_stencil(const LevelDev& L) {
    CtaStencil<C> S;
    S.sy = L.n[0];
    S.sz = L.n[0] * L.n[1];
    for (int a = 0; a < 3; ++a) {
        S.ih[a] = LP<C>::ih2(L, a);
        S.act[a] = L.active[a] != 0;
    }
    S.all3 = S.act[0] && S.act[1] && S.act[2];
    return S;
}

template <class C>
__device__ __forceinline__ C cta_A(const CtaStencil<C>& S, uint32_t f, const C* e, int c, C eP) {
    if (S.all3 && (f & 0xfffu) == 0u) {
        C acc = ((eP - e[c - 1]) + (eP - e[c + 1])) * S.ih[0];
        acc += ((eP - e[c - S.sy]) + (eP - e[c + S.sy])) * S.ih[1];
        acc += ((eP - e[c - S.sz]) + (eP - e[c + S.sz])) * S.ih[2];
        return acc;
    }
    const int st[3] = {1, S.sy, S.sz};
    C acc = (C)0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!S.act[a]) continue;
        const C lo = nb_val<C>((f >> (4 * a)) & 3u, c - st[a], eP, [&](int q) { return e[q]; });
        const C hi = nb_val<C>((f >> (4 * a + 2)) & 3u, c + st[a], eP, [&](int q) { return e[q]; });
        acc += ((eP - lo) + (eP - hi)) * S.ih[a];
    }
    return acc;
}

// the weight of sweep i on one side (0 pre, 1 post) of a coarse-CTA level
template <class C> __device__ __forceinline__ C coarse_weight(const CoarseLevels& cl, const LevelDev& L, int side, int i);
template <> __device__ __forceinline__ double coarse_weight<double>(const CoarseLevels& cl, const LevelDev& L, int side,
                                                                   int i) {
    return cl.cheb ? cl.w[side][i] : L.wJ;
}
template <> __device__ __forceinline__ float coarse_weight<float>(const CoarseLevels& cl, const LevelDev& L, int side,
                                                                 int i) {
    return cl.cheb ? cl.wf[side][i] : L.wJf;
}

template <class TI>
struct CoarseK {
    static constexpr int kThreads = kCtaThreads;
    CoarseLevels cl;
    const TI* r_in;
    TI* e_out;
    const double* Ainv;
    const SolveState* st;
    __device__ bool live() const { return st->active != 0; }   // batched: skip a converged case
    __device__ void run(const BlockAt& at) const;
};

template <class TI>
__device__ void coarse_cta_body(const CoarseLevels& cl, const TI* __restrict__ r_in, TI* __restrict__ e_out,
                                const double* __restrict__ Ainv);

template <class TI>
__device__ void CoarseK<TI>::run(const BlockAt&) const {
    coarse_cta_body<TI>(cl, r_in, e_out, Ainv);
}

// c / n for the small levels of the coarse kernel (0 <= c < 2^22, inv_n = 1/n in FP32):
// (c + 1/2)/n is at least 1/(2n) from an integer, more than the FP32 rounding of the product
__device__ __forceinline__ int small_div(int c, float inv_n) { return (int)(((float)c + 0.5f) * inv_n); }

template <class TI>
__device__ void coarse_cta_body(const CoarseLevels& cl, const TI* __restrict__ r_in, TI* __restrict__ e_out,
                                const double* __restrict__ Ainv) {
    using C = typename Acc<TI>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // level descriptions and array bases live in shared memory (one copy per CTA)
    __shared__ LevelDev lvs[FVM_MAX_LEVELS];
    // the arrays' offsets into the dynamic shared memory (elements of C, codes in 16-bit units):
    // pointers formed from smem_raw here let the compiler address them as shared memory (pointers
    // kept in a shared array would be generic, each access a generic load)
    __shared__ int E0o[FVM_MAX_LEVELS];
    __shared__ int E1o[FVM_MAX_LEVELS];
    __shared__ int Ro[FVM_MAX_LEVELS];
    __shared__ int Fo[FVM_MAX_LEVELS];
    C* const Cs = reinterpret_cast<C*>(smem_raw);
    uint16_t* const Us = reinterpret_cast<uint16_t*>(smem_raw);
    auto E0 = [&](int l) { return Cs + E0o[l]; };
    auto E1 = [&](int l) { return Cs + E1o[l]; };
    auto R = [&](int l) { return Cs + Ro[l]; };
    auto F = [&](int l) { return Us + Fo[l]; };
    const int T = blockDim.x, tid = threadIdx.x;
    // the level descriptions, copied word by word by all threads
    {
        const int words = cl.nl * (int)(sizeof(LevelDev) / 4);
        const uint32_t* src = reinterpret_cast<const uint32_t*>(cl.lv);
        for (int w = tid; w < words; w += T) reinterpret_cast<uint32_t*>(lvs)[w] = src[w];
    }
    if (tid == 0) {
        int q = 0;
        for (int l = 0; l < cl.nl; ++l) {
            const int N = (int)cl.lv[l].N;
            E0o[l] = q; q += N;
            E1o[l] = q; q += N;
            Ro[l] = q; q += N;
        }
        int u = q * (int)(sizeof(C) / sizeof(uint16_t));
        for (int l = 0; l < cl.nl; ++l) {
            Fo[l] = u;
            u += (int)cl.lv[l].N;
        }
    }
    __syncthreads();
    for (int l = 0; l < cl.nl; ++l) {
        const int N = (int)lvs[l].N;
        const uint16_t* src = lvs[l].nbf;   // the level's codes in global memory
        for (int c = tid; c < N; c += T) F(l)[c] = src[c];
    }
    {
        const int N0 = (int)lvs[0].N;
        for (int c = tid; c < N0; c += T) R(0)[c] = to_c<C>(r_in[c]);
    }
    __syncthreads();
    __shared__ int cur[FVM_MAX_LEVELS];
    // down: pre-smooth, restrict
    for (int l = 0; l + 1 < cl.nl; ++l) {
        const LevelDev& L = lvs[l];
        const CtaStencil<C> S = cta_stencil<C>(L);
        const uint16_t* const fl = F(l);
        C* const rl = R(l);
        const int N = (int)L.N;
        const C iD = LP<C>::iD(L);
        const C w0 = coarse_weight<C>(cl, L, 0, 0);
        for (int c = tid; c < N; c += T) E0(l)[c] = is_solid(fl[c]) ? (C)0 : w0 * rl[c] * iD;
        __syncthreads();
        int s = 0;
        for (int it = 1; it < cl.pre; ++it) {
            const C w = coarse_weight<C>(cl, L, 0, it);
            C* ein = s ? E1(l) : E0(l);
            C* eo = s ? E0(l) : E1(l);
            for (int c = tid; c < N; c += T) {
                const uint32_t f = fl[c];
                C v = (C)0;
                if (!is_solid(f)) {
                    const C eP = ein[c];
                    v = eP + w * (rl[c] - cta_A<C>(S, f, ein, c, eP)) * iD;
                }
                eo[c] = v;
            }
            s ^= 1;
            __syncthreads();
        }
        if (tid == 0) cur[l] = s;
        const LevelDev& Lc = lvs[l + 1];
        const C* e = s ? E1(l) : E0(l);
        const int fx = L.active[0] ? 2 : 1, fy = L.active[1] ? 2 : 1, fz = L.active[2] ? 2 : 1;
        const int Nc = (int)Lc.N, cn0 = Lc.n[0], cn1 = Lc.n[1], n0 = L.n[0], n1 = L.n[1];
        const float icn0 = 1.0f / (float)cn0, icn01 = 1.0f / (float)(cn0 * cn1);
        C* const rc = R(l + 1);
        // one child per thread: eight consecutive lanes hold one coarse cell's children
        // (missing children of a collapsed axis add 0) and sum them by a fixed shuffle tree
        const int items = 8 * Nc, bound = (items + 31) & ~31;
        for (int w = tid; w < bound; w += T) {
            const int cc = w >> 3, ch = w & 7;
            const int dx = ch & 1, dy = (ch >> 1) & 1, dz = ch >> 2;
            C v = (C)0;
            if (w < items && dx < fx && dy < fy && dz < fz) {
                const int K = small_div(cc, icn01);
                const int rem = cc - K * cn0 * cn1;
                const int J = small_div(rem, icn0);
                const int I = rem - J * cn0;
                const int c = (I * fx + dx) + n0 * ((J * fy + dy) + n1 * (K * fz + dz));
                const uint32_t f = fl[c];
                if (!is_solid(f)) v = rl[c] - cta_A<C>(S, f, e, c, e[c]);
            }
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            if (ch == 0 && w < items) rc[cc] = v / (C)(fx * fy * fz);
        }
        __syncthreads();
    }
    // coarsest: dense solve, one warp per row (coalesced reads of the inverse); in the
    // reduced-precision modes from the FP32 copy of the inverse stored after the FP64 one
    {
        const int l = cl.nl - 1;
        const int N = (int)lvs[l].N;
        const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
        for (int row = warp; row < N; row += nw) {
            if constexpr (sizeof(C) == 8) {
                double acc = 0.0;
                const double* a = Ainv + (size_t)row * N;
                for (int col = lane; col < N; col += 32) acc += __ldg(a + col) * (double)R(l)[col];
                for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
                if (lane == 0) E0(l)[row] = (C)acc;
            } else {
                float acc = 0.0f;
                const float* a = reinterpret_cast<const float*>(Ainv + (size_t)N * N) + (size_t)row * N;
                for (int col = lane; col < N; col += 32) acc = fmaf(__ldg(a + col), R(l)[col], acc);
                for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
                if (lane == 0) E0(l)[row] = acc;
            }
        }
        if (tid == 0) cur[l] = 0;
        __syncthreads();
    }
    // up: prolong, post-smooth
    for (int l = cl.nl - 2; l >= 0; --l) {
        const LevelDev& L = lvs[l];
        const LevelDev& Lc = lvs[l + 1];
        const CtaStencil<C> S = cta_stencil<C>(L);
        C* const Rl = R(l);
        const uint16_t* const fl = F(l);
        const uint16_t* const fc = F(l + 1);
        // the prolongation's axes and coarse extents in registers (see CtaStencil)
        const int fa[3] = {L.active[0], L.active[1], L.active[2]};
        const int cn[3] = {Lc.n[0], Lc.n[1], Lc.n[2]};
        const int N = (int)L.N, n0 = L.n[0], n1 = L.n[1];
        const float in0 = 1.0f / (float)n0, in01 = 1.0f / (float)(n0 * n1);
        const C* ec = cur[l + 1] ? E1(l + 1) : E0(l + 1);
        C* e = cur[l] ? E1(l) : E0(l);
        for (int c = tid; c < N; c += T) {
            if (is_solid(fl[c])) continue;
            const int k = small_div(c, in01);
            const int rem = c - k * n0 * n1;
            const int j = small_div(rem, in0);
            const int i = rem - j * n0;
            e[c] += prolong_at<C>(fa, cn, i, j, k, [&](int q) { return ec[q]; },
                                  [&](int q) { return (uint32_t)fc[q]; });
        }
        __syncthreads();
        int s = cur[l];
        const C iD = LP<C>::iD(L);
        for (int it = 0; it < cl.post; ++it) {
            const C w = coarse_weight<C>(cl, L, 1, it);
            C* ein = s ? E1(l) : E0(l);
            C* eo = s ? E0(l) : E1(l);
            for (int c = tid; c < N; c += T) {
                const uint32_t f = fl[c];
                C v = (C)0;
                if (!is_solid(f)) {
                    const C eP = ein[c];
                    v = eP + w * (Rl[c] - cta_A<C>(S, f, ein, c, eP)) * iD;
                }
                eo[c] = v;
            }
            s ^= 1;
            __syncthreads();
        }
        if (tid == 0) cur[l] = s;
        __syncthreads();
    }
    {
        const C* e = cur[0] ? E1(0) : E0(0);
        const int N0 = (int)lvs[0].N;
        for (int c = tid; c < N0; c += T) e_out[c] = from_c<TI, C>(e[c]);
    }
}

// ------------------------------------------------------------------ flexible CG acceleration (krylov = 1)
// One pass over level 0 with z (the V-cycles' correction for the outer
// residual r) and the kept direction d_prev: A z at each cell from the
// stencil (not stored) and the block sums of (z, A z), (A z, d_prev),
// (r, z), (r, d_prev).  The last block sums them in a fixed order and sets,
// for d = z - beta d_prev,
//   beta   = (A z, d_prev) / (d_prev, A d_prev)   [= (z, A d_prev): A is symmetric]
//   (d, A d) = (z, A z) - beta (A z, d_prev)
//   alpha  = ((r, z) - beta (r, d_prev)) / (d, A d),
// keeping (d, A d) for the next iteration.  Should rounding make (d, A d)
// non-positive (never in exact arithmetic) the direction restarts: beta = 0.
template <class TR, class TZ>
struct FcgDotK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr int kMinBlocks = 4;
    LevelDev L;
    const TZ* z;
    const TR* r;
    const TZ* dp;
    double* partials;
    SolveState* st;
    __device__ bool live() const { return st->active != 0; }
    __device__ void run(const BlockAt& at) const;
};

template <class TR, class TZ>
__device__ void FcgDotK<TR, TZ>::run(const BlockAt& at) const {
    using C = typename Acc<TZ>::type;
    const bool have = st->g_valid != 0;
    double s[4] = {0.0, 0.0, 0.0, 0.0};   // (z,Az), (Az,dp), (r,z), (r,dp)
    int i, j, k;
    if (cell3(L, at, i, j, k)) {
        const int c = i + L.n[0] * (j + L.n[1] * k);
        const uint32_t f = L.nbf[c];
        const int sy = L.n[0], sz = L.n[0] * L.n[1];
        const C eP = to_c<C>(ldg(z + c));
        const C xm = to_c<C>(ldg(z + c - (i > 0 ? 1 : 0))), xp = to_c<C>(ldg(z + c + (i < L.n[0] - 1 ? 1 : 0)));
        const C ym = to_c<C>(ldg(z + c - (j > 0 ? sy : 0))), yp = to_c<C>(ldg(z + c + (j < L.n[1] - 1 ? sy : 0)));
        const C zm = to_c<C>(ldg(z + c - (k > 0 ? sz : 0))), zp = to_c<C>(ldg(z + c + (k < L.n[2] - 1 ? sz : 0)));
        const double rd = to_c<double>(ldg(r + c));
        const double dd = have ? to_c<double>(ldg(dp + c)) : 0.0;
        if (!is_solid(f)) {
            const double zd = (double)eP;
            const double qd = (double)A7<C>(L, f, eP, xm, xp, ym, yp, zm, zp);
            s[0] = zd * qd;
            s[1] = qd * dd;
            s[2] = rd * zd;
            s[3] = rd * dd;
        }
    }
    fcg_reduce<kThreads>(s, partials, st, have, at);
}

// d = z - beta d_prev; p += alpha d on fluid cells; d kept as d_prev
template <class TZ>
struct FcgUpdK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    LevelDev L;
    const TZ* z;
    TZ* dp;
    double* p;
    const SolveState* st;
    __device__ bool live() const { return st->active != 0; }
    __device__ void run(const BlockAt& at) const {
        int i, j, k;
        if (!cell3(L, at, i, j, k)) return;
        const int c = i + L.n[0] * (j + L.n[1] * k);
        const double alpha = st->g_alpha, beta = st->g_beta;
        const double d = to_c<double>(ldg(z + c)) - (beta != 0.0 ? beta * to_c<double>(dp[c]) : 0.0);
        if (!is_solid(L.nbf[c])) {
            if constexpr (sizeof(TZ) == 8) p[c] += alpha * d;
            else pp_add(p, c, (float)(alpha * d));
        }
        dp[c] = from_c<TZ, double>(d);
    }
};

// ------------------------------------------------------------------ the paper's scheme (Algorithm 1)
// coarse r = mean of the children's r (the residual restricted straight down)
template <class TI>
struct RestrictK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    LevelDev Lf, Lc;
    const TI* r;
    TI* rc;
    const SolveState* st;
    __device__ bool live() const { return st->active != 0; }
    __device__ void run(const BlockAt& at) const {
        using C = typename Acc<TI>::type;
        int I, J, K;
        if (!cell3(Lc, at, I, J, K)) return;
        const int fx = Lf.active[0] ? 2 : 1, fy = Lf.active[1] ? 2 : 1, fz = Lf.active[2] ? 2 : 1;
        C sum = (C)0;
        for (int dz = 0; dz < fz; ++dz)
            for (int dy = 0; dy < fy; ++dy)
                for (int dx = 0; dx < fx; ++dx)
                    sum += to_c<C>(ldg(r + (I * fx + dx) + Lf.n[0] * ((J * fy + dy) + Lf.n[1] * (K * fz + dz))));
        rc[I + Lc.n[0] * (J + Lc.n[1] * K)] = from_c<TI, C>(sum / (C)(fx * fy * fz));
    }
};

__device__ __forceinline__ int parent_of(const LevelDev& Lf, const LevelDev& Lc, int i, int j, int k) {
    const int I = Lf.active[0] ? i >> 1 : i, J = Lf.active[1] ? j >> 1 : j, K = Lf.active[2] ? k >> 1 : k;
    return I + Lc.n[0] * (J + Lc.n[1] * K);
}

// e = the parent's correction (nearest upsampling), zero in solid cells
template <class TI>
struct ProlongNearestK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    LevelDev Lf, Lc;
    const TI* ec;
    TI* e;
    const SolveState* st;
    __device__ bool live() const { return st->active != 0; }
    __device__ void run(const BlockAt& at) const {
        int i, j, k;
        if (!cell3(Lf, at, i, j, k)) return;
        const int c = i + Lf.n[0] * (j + Lf.n[1] * k);
        e[c] = is_solid(Lf.nbf[c]) ? from_c<TI, float>(0.f) : ec[parent_of(Lf, Lc, i, j, k)];
    }
};

// p += the parent's level-1 correction (nearest upsampling) in fluid cells
template <class TI>
struct ProlongNearestToPK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    LevelDev Lf, Lc;
    const TI* ec;
    double* p;
    const SolveState* st;
    __device__ bool live() const { return st->active != 0; }
    __device__ void run(const BlockAt& at) const {
        int i, j, k;
        if (!cell3(Lf, at, i, j, k)) return;
        const int c = i + Lf.n[0] * (j + Lf.n[1] * k);
        if (is_solid(Lf.nbf[c])) return;
        if constexpr (sizeof(TI) == 8) p[c] += to_c<double>(ldg(ec + parent_of(Lf, Lc, i, j, k)));
        else pp_add(p, c, to_c<float>(ldg(ec + parent_of(Lf, Lc, i, j, k))));
    }
};

// unweighted Jacobi sweep on the pressure, out of place: q = p + (b - A p) / D (copied back by CopyPK,
// eight bytes per cell in either storage)
template <class TB>
struct JacobiPK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    LevelDev L;
    const double* p;
    const TB* b;
    double* q;
    const SolveState* st;
    __device__ bool live() const { return st->active != 0; }
    __device__ void run(const BlockAt& at) const {
        int i, j, k;
        if (!cell3(L, at, i, j, k)) return;
        const int c = i + L.n[0] * (j + L.n[1] * k);
        const uint32_t f = L.nbf[c];
        if (is_solid(f)) {
            q[c] = 0.0;
            return;
        }
        // (reduced-precision cases: p and q as double-float pairs, the sweep in FP64)
        auto P = [&](int x) { return sizeof(TB) == 8 ? __ldg(p + x) : pp_get(p, x); };
        const int sy = L.n[0], sz = L.n[0] * L.n[1];
        const double pP = P(c);
        const double xm = P(c - (i > 0 ? 1 : 0)), xp = P(c + (i < L.n[0] - 1 ? 1 : 0));
        const double ym = P(c - (j > 0 ? sy : 0)), yp = P(c + (j < L.n[1] - 1 ? sy : 0));
        const double zm = P(c - (k > 0 ? sz : 0)), zp = P(c + (k < L.n[2] - 1 ? sz : 0));
        const double v = pP + (to_c<double>(ldg(b + c)) - A7<double>(L, f, pP, xm, xp, ym, yp, zm, zp)) * L.inv_D;
        if constexpr (sizeof(TB) == 8) q[c] = v;
        else reinterpret_cast<float2*>(q)[c] = pp_from_double(v);
    }
};

struct CopyPK {
    static constexpr int kThreads = BX * BY * BZ;
    static constexpr bool kNoShared = true;   // run() uses no shared memory
    LevelDev L;
    const double* q;
    double* p;
    const SolveState* st;
    __device__ bool live() const { return st->active != 0; }
    __device__ void run(const BlockAt& at) const {
        int i, j, k;
        if (!cell3(L, at, i, j, k)) return;
        const int c = i + L.n[0] * (j + L.n[1] * k);
        p[c] = q[c];
    }
};

__global__ void k_p_to_double(const double* __restrict__ pp, double* __restrict__ dst, int64_t N) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) dst[c] = pp_get(pp, c);
}

__global__ void k_p_from_double(const double* __restrict__ src, double* __restrict__ pp, int64_t N) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) reinterpret_cast<float2*>(pp)[c] = pp_from_double(src[c]);
}

// p to and from FP32 host values: the pair rounded once to FP32 (hi + lo evaluated in FP64,
// exact), and an FP32 value as the pair (value, 0)
__global__ void k_p_to_float(const double* __restrict__ pp, float* __restrict__ dst, int64_t N) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) dst[c] = __double2float_rn(pp_get(pp, c));
}

__global__ void k_p_from_float(const float* __restrict__ src, double* __restrict__ pp, int64_t N) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) reinterpret_cast<float2*>(pp)[c] = make_float2(src[c], 0.0f);
}

template <class A, class B>
__global__ void k_convert(const A* __restrict__ src, B* __restrict__ dst, int64_t N) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) dst[c] = from_c<B, double>(to_c<double>(src[c]));
}

dim3 grid3(const LevelDev& L) {
    return dim3((unsigned)((L.n[0] + BX - 1) / BX), (unsigned)((L.n[1] + BY - 1) / BY),
                (unsigned)((L.n[2] + BZ - 1) / BZ));
}
const dim3 kBlock3(BX, BY, BZ);

}  // namespace

int resid0_blocks(int nx, int ny, int nz) {
    return ((nx + BX - 1) / BX) * ((ny + BY - 1) / BY) * ((nz + BZ - 1) / BZ);
}

// vector kernels with W cells per thread: log2 of the lanes per row segment, the widest
// segment of W * 32, W * 16, W * 8 or W * 4 cells that divides nx (a warp then covers 1, 2, 4
// or 8 rows)
static int vw_lrl(int nx, int W) {
    for (int l = 5; l >= 2; --l)
        if (nx % (W << l) == 0) return l;
    return 5;
}
static int v4_lrl(int nx) { return vw_lrl(nx, 4); }

int level0_blocks_max(int nx, int ny, int nz) {
    // a vector pass (four or eight cells per thread) with this nx's row segments, one plane a block
    int most = resid0_blocks(nx, ny, nz);
    for (int W : {4, 8}) {
        const int lrl = vw_lrl(nx, W), wx = W << lrl, wy = TY << (5 - lrl);
        const int n = ((nx + wx - 1) / wx) * ((ny + wy - 1) / wy) * nz;
        most = n > most ? n : most;
    }
    return most;
}

size_t coarse_cta_smem(const CoarseLevels& cl, int inner) {
    const size_t cs = inner == FVM_FP64 ? 8 : 4;
    size_t n = 0, m = 0;
    for (int l = 0; l < cl.nl; ++l) {
        n += 3 * (size_t)cl.lv[l].N;
        m += (size_t)cl.lv[l].N;
    }
    return n * cs + m * 2 + 16;
}

#define DISPATCH_I(inner, ...)                                            \
    do {                                                                  \
        if ((inner) == FVM_FP64) { using TI = double; __VA_ARGS__; }      \
        else if ((inner) == FVM_FP32) { using TI = float; __VA_ARGS__; } \
        else { using TI = __nv_bfloat16; __VA_ARGS__; }                   \
    } while (0)

cudaError_t launch_solve_begin(SolveState* st, cudaStream_t s) {
    return launch_k(SolveBeginK{st}, dim3(1), dim3(1), 0, s);
}

static int sweep_planes(int tiles, int nz, int fixed, int per_sm);

// vector kernels: the block's x-y extent for W cells per thread and the row segments of lrl;
// per_sm: the blocks per SM the plane rule aims for
static dim3 vw_grid(const LevelDev& L, int W, int lrl, int& zc, int per_sm = 8) {
    const int wx = W << lrl, wy = TY << (5 - lrl);
    const int tiles = ((L.n[0] + wx - 1) / wx) * ((L.n[1] + wy - 1) / wy);
    zc = sweep_planes(tiles, L.n[2], L.zc_fixed, per_sm);
    return dim3((unsigned)((L.n[0] + wx - 1) / wx), (unsigned)((L.n[1] + wy - 1) / wy), (unsigned)((L.n[2] + zc - 1) / zc));
}
static dim3 v4_grid(const LevelDev& L, int lrl, int& zc) { return vw_grid(L, 4, lrl, zc); }

cudaError_t launch_resid0(int inner, int bprec, const LevelDev& L, const double* p, const void* b, void* r, void* e,
                          double* partials, SolveState* st, cudaGraphConditionalHandle cond,
                          cudaGraphConditionalHandle cond2, int use_cond, cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    DISPATCH_I(inner, {
        if constexpr (sizeof(TI) < 8) {
            // four cells per thread in float-float on large levels and in batches
            if (bprec == FVM_FP32 && L.n[0] % 4 == 0 && (L.N >= (1 << 20) || g_rec)) {
                const int lrl = v4_lrl(L.n[0]);
                int zc = 0;
                const dim3 grid = v4_grid(L, lrl, zc);
                // (at most level0_blocks_max(n) blocks: partials has room)
                return launch_r0(Resid0V4K<TI>{L, p, (const float*)b, (TI*)r, (TI*)e, partials, st, zc, lrl}, grid,
                                 dim3(TX, TY), cond, cond2, use_cond, s);
            }
        }
        if (bprec == FVM_FP64)
            err = launch_r0(Resid0K<double, TI>{L, p, (const double*)b, (TI*)r, (TI*)e, partials, st}, grid3(L),
                            kBlock3, cond, cond2, use_cond, s);
        else
            err = launch_r0(Resid0K<float, TI>{L, p, (const float*)b, (TI*)r, (TI*)e, partials, st}, grid3(L),
                            kBlock3, cond, cond2, use_cond, s);
    });
    return err;
}

cudaError_t launch_sweep_first(int inner, const LevelDev& L, const void* r, void* e, const SolveState* st,
                               cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    DISPATCH_I(inner, err = launch_k(SweepFirstK<TI>{L, (const TI*)r, (TI*)e, st}, grid3(L), kBlock3, 0, s));
    return err;
}

static dim3 walk_grid(const LevelDev& L, int kz) {
    return dim3((unsigned)((L.n[0] + TX - 1) / TX), (unsigned)((L.n[1] + TY - 1) / TY),
                (unsigned)((L.n[2] + kz - 1) / kz));
}

// planes per block: the most that still give about per_sm blocks per SM (one plane per
// block on grids too small for that).  The sweep aims for 16: it has no block reduction, and
// shorter columns in more blocks balance better (the room's level-0 sweep: 42.3 us at four
// planes a block, 37.3 at two, 40.0 at one); the kernels that end in a block reduction (the
// residual, the inner products) aim for 8 (at two planes a block both measured about a third
// slower, at eight or more planes a few per cent slower).
static int sweep_planes(int tiles, int nz, int fixed, int per_sm) {
    if (fixed > 0) return fixed < nz ? fixed : nz;
    // in a batch the cases' blocks add up: eight-plane columns (measured on 64 channels against
    // 4, 16 and 32: fewer re-read planes than 4, better balance than 16 or 32)
    if (g_rec) return nz < 8 ? nz : 8;
    for (int zc : {32, 16, 8, 4, 2})
        if (tiles * ((nz + zc - 1) / zc) >= per_sm * 152) return zc;
    return 1;
}

// eight cells per thread on BF16 levels: in batches, and on single-case levels of 2^22 cells or
// more; a smaller level (the room's level 1, 2 M cells) takes four, for twice the threads (at
// eight its residual-restriction launch had 256 blocks for 152 SMs)
static bool wide8(const LevelDev& L) { return L.n[0] % 8 == 0 && (g_rec || L.N >= (1 << 22)); }

template <class TI, int MODE>
static cudaError_t sweep_walk(const LevelDev& L, const TI* ein, const TI* r, TI* eout, double* p,
                              const SolveState* st, cudaStream_t s, float* z32 = nullptr) {
    if constexpr (sizeof(TI) < 8) {
        // four cells per thread on large levels and in batches (their blocks add up over the cases)
        if (L.n[0] % 4 == 0 && (L.N >= (1 << 20) || g_rec)) {
            constexpr int W = vec_w<TI>();
            int zc = 0;
            if (W == 8 && wide8(L)) {
                const int lrl = vw_lrl(L.n[0], 8);
                const dim3 grid = vw_grid(L, 8, lrl, zc, 16);
                return launch_k(SweepVK<TI, MODE, vec_w<TI>()>{L, ein, r, eout, p, st, zc, z32, lrl}, grid,
                                dim3(TX, TY), 0, s);
            }
            const int lrl = vw_lrl(L.n[0], 4);
            const dim3 grid = vw_grid(L, 4, lrl, zc, 16);
            return launch_k(SweepVK<TI, MODE, 4>{L, ein, r, eout, p, st, zc, z32, lrl}, grid, dim3(TX, TY), 0, s);
        }
    }
    // four cells per thread on large grids and in batches (one launch for all cases of a level)
    if (L.N >= (1 << 20) || g_rec)
        return launch_k(SweepK<TI, MODE, 4>{L, ein, r, eout, p, st, z32}, walk_grid(L, 4), dim3(TX, TY), 0, s);
    return launch_k(SweepK<TI, MODE, 1>{L, ein, r, eout, p, st, z32}, walk_grid(L, 1), dim3(TX, TY), 0, s);
}

cudaError_t launch_sweep(int inner, const LevelDev& L, const void* e_in, const void* r, void* e_out,
                         const SolveState* st, cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    DISPATCH_I(inner, err = sweep_walk<TI, 0>(L, (const TI*)e_in, (const TI*)r, (TI*)e_out, nullptr, st, s));
    return err;
}

cudaError_t launch_sweep_to_p(int inner, const LevelDev& L, const void* e_in, const void* r, double* p,
                              const SolveState* st, cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    DISPATCH_I(inner, err = sweep_walk<TI, 1>(L, (const TI*)e_in, (const TI*)r, nullptr, p, st, s));
    return err;
}

cudaError_t launch_sweep_to_f32(int inner, const LevelDev& L, const void* e_in, const void* r, float* z,
                                const SolveState* st, cudaStream_t s) {
    if (inner != FVM_BF16_MIXED) return cudaErrorInvalidValue;
    using TI = __nv_bfloat16;
    return sweep_walk<TI, 2>(L, (const TI*)e_in, (const TI*)r, nullptr, nullptr, st, s, z);
}

template <class TI>
static bool v4_transfer_ok(const LevelDev& Lf) {
    return sizeof(TI) < 8 && Lf.active[0] && Lf.active[1] && Lf.n[0] % 4 == 0 && Lf.n[1] % 2 == 0 &&
           (Lf.N >= (1 << 20) || g_rec);
}

cudaError_t launch_resid_restrict(int inner, const LevelDev& Lf, const LevelDev& Lc, const void* e, const void* r,
                                  void* rc, void* ec0, const SolveState* st, cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    if (inner != FVM_FP64 && v4_transfer_ok<float>(Lf)) {
        const int W = inner == FVM_BF16_MIXED && wide8(Lf) ? 8 : 4;
        const int lrl = vw_lrl(Lf.n[0], W), wx = W << lrl, wy = TY << (5 - lrl);
        const dim3 grid((unsigned)((Lf.n[0] + wx - 1) / wx), (unsigned)((Lc.n[1] + wy - 1) / wy), (unsigned)Lc.n[2]);
        if (inner == FVM_FP32)
            return launch_k(RRVK<float, 4>{Lf, Lc, (const float*)e, (const float*)r, (float*)rc, (float*)ec0, lrl, st},
                            grid, dim3(TX, TY), 0, s);
        using B = __nv_bfloat16;
        if (W == 8)
            return launch_k(RRVK<B, 8>{Lf, Lc, (const B*)e, (const B*)r, (B*)rc, (B*)ec0, lrl, st}, grid, dim3(TX, TY),
                            0, s);
        return launch_k(RRVK<B, 4>{Lf, Lc, (const B*)e, (const B*)r, (B*)rc, (B*)ec0, lrl, st}, grid, dim3(TX, TY), 0,
                        s);
    }
    if (Lf.active[0] && Lf.active[1]) {
        const int fz = Lf.active[2] ? 2 : 1;
        DISPATCH_I(inner, err = launch_k(RRWalkK<TI>{Lf, Lc, (const TI*)e, (const TI*)r, (TI*)rc, (TI*)ec0, st},
                                         walk_grid(Lf, fz), dim3(TX, TY), 0, s));
    } else {
        DISPATCH_I(inner, err = launch_k(ResidRestrictK<TI>{Lf, Lc, (const TI*)e, (const TI*)r, (TI*)rc, (TI*)ec0,
                                                            st},
                                         grid3(Lc), kBlock3, 0, s));
    }
    return err;
}

cudaError_t launch_prolong_add(int inner, const LevelDev& Lf, const LevelDev& Lc, const void* ec, void* e,
                               const SolveState* st, cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    if (inner != FVM_FP64 && v4_transfer_ok<float>(Lf)) {
        int zc = 0;
        if (inner == FVM_FP32) {
            const int lrl = vw_lrl(Lf.n[0], 4);
            const dim3 grid = vw_grid(Lf, 4, lrl, zc);
            return launch_k(ProlongVK<float, 4>{Lf, Lc, (const float*)ec, (float*)e, st, zc, lrl}, grid, dim3(TX, TY),
                            0, s);
        }
        if (wide8(Lf)) {
            const int lrl = vw_lrl(Lf.n[0], 8);
            const dim3 grid = vw_grid(Lf, 8, lrl, zc);
            return launch_k(ProlongVK<__nv_bfloat16, 8>{Lf, Lc, (const __nv_bfloat16*)ec, (__nv_bfloat16*)e, st, zc,
                                                        lrl},
                            grid, dim3(TX, TY), 0, s);
        }
        const int lrl = vw_lrl(Lf.n[0], 4);
        const dim3 grid = vw_grid(Lf, 4, lrl, zc);
        return launch_k(ProlongVK<__nv_bfloat16, 4>{Lf, Lc, (const __nv_bfloat16*)ec, (__nv_bfloat16*)e, st, zc, lrl},
                        grid, dim3(TX, TY), 0, s);
    }
    DISPATCH_I(inner, err = launch_k(ProlongK<TI>{Lf, Lc, (const TI*)ec, (TI*)e, st}, grid3(Lf), kBlock3, 0, s));
    return err;
}

cudaError_t prepare_coarse_cta(int inner, size_t smem) {
    DISPATCH_I(inner, {
        cudaError_t err = raise_smem_limit((const void*)k_one<CoarseK<TI>>, smem);
        if (err != cudaSuccess) return err;
    });
    return cudaSuccess;
}

cudaError_t launch_coarse_cta(int inner, const CoarseLevels& cl, const void* r_in, void* e_out, const double* Ainv,
                              const SolveState* st, cudaStream_t s) {
    const size_t smem = coarse_cta_smem(cl, inner);
    cudaError_t err = cudaSuccess;
    DISPATCH_I(inner, err = launch_k(CoarseK<TI>{cl, (const TI*)r_in, (TI*)e_out, Ainv, st}, dim3(1),
                                     dim3(kCtaThreads), smem, s));
    return err;
}

// z and the kept direction dp in TZ (the inner type, or FP32 on BF16 levels), r in TR
template <class TR, class TZ>
static cudaError_t fcg_launch(const LevelDev& L, const TZ* z, const TR* r, TZ* dp, double* p, double* partials,
                              SolveState* st, cudaStream_t s) {
    if constexpr (sizeof(TR) < 8) {
        if (L.n[0] % 4 == 0 && (L.N >= (1 << 20) || g_rec)) {
            // (at most level0_blocks_max(n) blocks: partials has room)
            int zc = 0;
            constexpr int W = std::is_same<TR, TZ>::value ? vec_w<TR>() : 4;
            if (W == 8 && L.n[0] % 8 == 0) {
                const int lrl = vw_lrl(L.n[0], W);
                const dim3 grid = vw_grid(L, W, lrl, zc);
                cudaError_t err =
                    launch_k(FcgDotVK<TR, TZ, W>{L, z, r, dp, partials, st, zc, lrl}, grid, dim3(TX, TY), 0, s);
                if (err != cudaSuccess) return err;
                const unsigned nb = (unsigned)((L.N / W + FcgUpdVK<TZ, W>::kThreads - 1) / FcgUpdVK<TZ, W>::kThreads);
                return launch_k(FcgUpdVK<TZ, W>{L, z, dp, p, st}, dim3(nb), dim3(FcgUpdVK<TZ, W>::kThreads), 0, s);
            }
            const int lrl = vw_lrl(L.n[0], 4);
            const dim3 grid = vw_grid(L, 4, lrl, zc);
            cudaError_t err =
                launch_k(FcgDotVK<TR, TZ, 4>{L, z, r, dp, partials, st, zc, lrl}, grid, dim3(TX, TY), 0, s);
            if (err != cudaSuccess) return err;
            const unsigned nb = (unsigned)((L.N / 4 + FcgUpdVK<TZ, 4>::kThreads - 1) / FcgUpdVK<TZ, 4>::kThreads);
            return launch_k(FcgUpdVK<TZ, 4>{L, z, dp, p, st}, dim3(nb), dim3(FcgUpdVK<TZ, 4>::kThreads), 0, s);
        }
    }
    cudaError_t err = launch_k(FcgDotK<TR, TZ>{L, z, r, dp, partials, st}, grid3(L), kBlock3, 0, s);
    if (err != cudaSuccess) return err;
    return launch_k(FcgUpdK<TZ>{L, z, dp, p, st}, grid3(L), kBlock3, 0, s);
}

cudaError_t launch_fcg(int inner, const LevelDev& L, const void* z, const void* r, void* dp, double* p,
                       double* partials, SolveState* st, cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    if (inner == FVM_BF16_MIXED)   // z and the kept direction in FP32 (rounding them to BF16 costs V-cycles)
        return fcg_launch<__nv_bfloat16, float>(L, (const float*)z, (const __nv_bfloat16*)r, (float*)dp, p, partials,
                                                st, s);
    DISPATCH_I(inner, err = fcg_launch<TI, TI>(L, (const TI*)z, (const TI*)r, (TI*)dp, p, partials, st, s));
    return err;
}

cudaError_t launch_restrict(int inner, const LevelDev& Lf, const LevelDev& Lc, const void* r, void* rc,
                            const SolveState* st, cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    DISPATCH_I(inner, err = launch_k(RestrictK<TI>{Lf, Lc, (const TI*)r, (TI*)rc, st}, grid3(Lc), kBlock3, 0, s));
    return err;
}

cudaError_t launch_prolong_nearest(int inner, const LevelDev& Lf, const LevelDev& Lc, const void* ec, void* e,
                                   const SolveState* st, cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    DISPATCH_I(inner, err = launch_k(ProlongNearestK<TI>{Lf, Lc, (const TI*)ec, (TI*)e, st}, grid3(Lf), kBlock3, 0, s));
    return err;
}

cudaError_t launch_prolong_nearest_to_p(int inner, const LevelDev& Lf, const LevelDev& Lc, const void* ec, double* p,
                                        const SolveState* st, cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    DISPATCH_I(inner,
               err = launch_k(ProlongNearestToPK<TI>{Lf, Lc, (const TI*)ec, p, st}, grid3(Lf), kBlock3, 0, s));
    return err;
}

cudaError_t launch_jacobi_p(int bprec, const LevelDev& L, double* p, const void* b, double* q, const SolveState* st,
                            cudaStream_t s) {
    cudaError_t err;
    if (bprec == FVM_FP64) err = launch_k(JacobiPK<double>{L, p, (const double*)b, q, st}, grid3(L), kBlock3, 0, s);
    else err = launch_k(JacobiPK<float>{L, p, (const float*)b, q, st}, grid3(L), kBlock3, 0, s);
    if (err != cudaSuccess) return err;
    return launch_k(CopyPK{L, q, p, st}, grid3(L), kBlock3, 0, s);
}

cudaError_t launch_convert(int sp, int dp, const void* src, void* dst, int64_t N, cudaStream_t s) {
    const unsigned nb = (unsigned)((N + 255) / 256);
    if (sp == FVM_FP64 && dp == FVM_FP32) k_convert<double, float><<<nb, 256, 0, s>>>((const double*)src, (float*)dst, N);
    else if (sp == FVM_FP32 && dp == FVM_FP64) k_convert<float, double><<<nb, 256, 0, s>>>((const float*)src, (double*)dst, N);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_p_to_double(const double* pp, double* dst, int64_t N, cudaStream_t s) {
    k_p_to_double<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(pp, dst, N);
    return cudaGetLastError();
}

cudaError_t launch_p_to_float(const double* pp, float* dst, int64_t N, cudaStream_t s) {
    k_p_to_float<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(pp, dst, N);
    return cudaGetLastError();
}

cudaError_t launch_p_from_float(const float* src, double* pp, int64_t N, cudaStream_t s) {
    k_p_from_float<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(src, pp, N);
    return cudaGetLastError();
}

cudaError_t launch_p_from_double(const double* src, double* pp, int64_t N, cudaStream_t s) {
    k_p_from_double<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(src, pp, N);
    return cudaGetLastError();
}
