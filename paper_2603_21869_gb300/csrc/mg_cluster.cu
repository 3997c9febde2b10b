// Coarse multigrid levels in one thread-block cluster.
//
// The levels lc..L-1 of the V-cycle (Algorithm 1 structure; smoother Eq.
// jacobi_pc, transfers Eqs. restriction / prolongation) live in the shared
// memory of one cluster of CS CTAs (up to 16 SMs).  Every level is cut into
// slabs of whole planes along the slowest active axis (z, or y for a 2D
// case); CTA q owns planes [q ppc, (q + 1) ppc) of each level.  Neighbours in
// the next or previous plane may belong to another CTA and are read through
// distributed shared memory; phases are separated by cluster barriers.  The
// last levels (cl.lm and coarser, a few thousand cells) are held whole by
// CTA 0 and cycled with block barriers while the other CTAs wait.  One launch
// replaces the per-level kernels of all coarse levels.
#include <cooperative_groups.h>

#include "fvm_internal.cuh"

namespace cg = cooperative_groups;

namespace {

template <class T> struct Acc { using type = T; };
template <> struct Acc<__nv_bfloat16> { using type = float; };

__device__ __forceinline__ bool solid_code(uint32_t f) { return (f >> 12) & 1u; }

template <class C>
__device__ __forceinline__ C pick(uint32_t code, C nb, C eP) {
    return code == 0 ? nb : (code == 1 ? eP : -eP);
}

template <class TI>
__global__ void __launch_bounds__(1024, 1) k_coarse_cluster(ClusterLevels cl, const TI* __restrict__ r_in,
                                                             TI* __restrict__ e_out, const double* __restrict__ Ainv,
                                                             const SolveState* st) {
    using C = typename Acc<TI>::type;
    if (!st->active) return;   // uniform over the cluster
    cg::cluster_group cluster = cg::this_cluster();
    const int me = (int)cluster.block_rank();
    extern __shared__ __align__(16) unsigned char smem[];
    C* cbase = (C*)smem;
    uint16_t* fbase = (uint16_t*)(smem + cl.fbyte0);
    const int T = blockDim.x, tid = threadIdx.x;
    const int D = cl.D;

    // array a (0: e, 1: e', 2: r) of level l, local slab base
    auto arr = [&](int l, int a) -> C* { return cbase + cl.off[l] + a * cl.ppc[l] * cl.plane[l]; };
    auto codes = [&](int l) -> uint16_t* { return fbase + cl.foff[l]; };
    // pointer to plane z (global index) of a level-l slab array, local or in another CTA
    // levels >= cl.lm are held whole by CTA 0 (ppc = nD there)
    auto owner_of = [&](int l, int z) { return l >= cl.lm ? 0 : fdiv(z, cl.mC[l]); };
    auto plane_ptr = [&](C* base, int l, int z) -> C* {
        const int owner = owner_of(l, z);
        C* p = base + (z - owner * cl.ppc[l]) * cl.plane[l];
        return owner == me ? p : cluster.map_shared_rank(p, owner);
    };
    auto my_z0 = [&](int l) { return l >= cl.lm ? 0 : me * cl.ppc[l]; };
    auto my_n = [&](int l) {
        if (l >= cl.lm) return me == 0 ? (int)cl.lv[l].N : 0;
        const int z0 = me * cl.ppc[l];
        const int z1 = min(cl.nD[l], z0 + cl.ppc[l]);
        return z1 > z0 ? (z1 - z0) * cl.plane[l] : 0;
    };
    // barrier over the CTAs that share level l's data
    auto level_sync = [&](int l) {
        if (l >= cl.lm) __syncthreads();
        else cluster.sync();
    };

    // A e at my local cell t of level l (e = slab array base of that level)
    auto apply_A = [&](int l, C* e, int t, uint32_t f, C eP) -> C {
        const LevelDev& L = cl.lv[l];
        const int P = cl.plane[l];
        const int zl = fdiv(t, cl.mP[l]);
        const int z = my_z0(l) + zl, q = t - zl * P;
        const int nx = L.n[0];
        const int jq = fdiv(q, cl.mX[l]);
        const int i = q - jq * nx;
        C* row = e + (t - q);                     // local plane start
        const C xm = i > 0 ? row[q - 1] : eP, xp = i < nx - 1 ? row[q + 1] : eP;
        C acc = (C)0;
        if (L.active[0]) acc += ((eP - pick(f & 3u, xm, eP)) + (eP - pick((f >> 2) & 3u, xp, eP))) * LP<C>::ih2(L, 0);
        const C zlo = z > 0 ? plane_ptr(e, l, z - 1)[q] : eP;
        const C zhi = z < cl.nD[l] - 1 ? plane_ptr(e, l, z + 1)[q] : eP;
        if (D == 2) {
            const int j = jq;
            const C ym = j > 0 ? row[q - nx] : eP, yp = j < L.n[1] - 1 ? row[q + nx] : eP;
            if (L.active[1])
                acc += ((eP - pick((f >> 4) & 3u, ym, eP)) + (eP - pick((f >> 6) & 3u, yp, eP))) * LP<C>::ih2(L, 1);
            acc += ((eP - pick((f >> 8) & 3u, zlo, eP)) + (eP - pick((f >> 10) & 3u, zhi, eP))) * LP<C>::ih2(L, 2);
        } else {
            acc += ((eP - pick((f >> 4) & 3u, zlo, eP)) + (eP - pick((f >> 6) & 3u, zhi, eP))) * LP<C>::ih2(L, 1);
        }
        return acc;
    };

    // load my slabs: neighbour codes of every level, r of the first level
    for (int l = 0; l < cl.nl; ++l) {
        const int n = my_n(l), off = my_z0(l) * cl.plane[l];
        uint16_t* F = codes(l);
        for (int t = tid; t < n; t += T) F[t] = cl.lv[l].nbf[off + t];
    }
    {
        const int n = my_n(0), off = my_z0(0) * cl.plane[0];
        C* R = arr(0, 2);
        for (int t = tid; t < n; t += T) R[t] = to_c<C>(r_in[off + t]);
    }
    cluster.sync();

    const int down = (cl.pre - 1) & 1;   // buffer holding e after pre-smoothing (same on every level)
    // ---------------------------------------------------------------- down
    for (int l = 0; l + 1 < cl.nl; ++l) {
        const LevelDev& L = cl.lv[l];
        const int n = my_n(l);
        const C w = LP<C>::wJ(L), iD = LP<C>::iD(L);
        C* R = arr(l, 2);
        uint16_t* F = codes(l);
        const bool local = l >= cl.lm;
        if (!local || me == 0) {
            {
                C* E0 = arr(l, 0);
                for (int t = tid; t < n; t += T) E0[t] = solid_code(F[t]) ? (C)0 : w * R[t] * iD;
            }
            level_sync(l);
            int s = 0;
            for (int it = 1; it < cl.pre; ++it) {
                C* ein = arr(l, s);
                C* eo = arr(l, s ^ 1);
#pragma unroll 4
                for (int t = tid; t < n; t += T) {
                    const uint32_t f = F[t];
                    C v = (C)0;
                    if (!solid_code(f)) {
                        const C eP = ein[t];
                        v = eP + w * (R[t] - apply_A(l, ein, t, f, eP)) * iD;
                    }
                    eo[t] = v;
                }
                s ^= 1;
                level_sync(l);
            }
            // residual of my cells into the free buffer
            {
                C* e = arr(l, s);
                C* res = arr(l, s ^ 1);
#pragma unroll 4
                for (int t = tid; t < n; t += T) {
                    const uint32_t f = F[t];
                    res[t] = solid_code(f) ? (C)0 : R[t] - apply_A(l, e, t, f, e[t]);
                }
            }
        }
        // the coarse level's owners read children that other CTAs wrote
        if (l + 1 >= cl.lm && l < cl.lm) cluster.sync();
        else level_sync(l);
        // restriction: my coarse cells average their children (children planes may be remote)
        if (l + 1 < cl.lm || me == 0) {
            const LevelDev& Lc = cl.lv[l + 1];
            C* res = arr(l, down ^ 1);
            C* Rc = arr(l + 1, 2);
            const int nc = my_n(l + 1), Pc = cl.plane[l + 1], zc0 = my_z0(l + 1);
            const int fx = L.active[0] ? 2 : 1, fy = (D == 2 && L.active[1]) ? 2 : 1;
            const int nxf = L.n[0], nxc = Lc.n[0];
            for (int t = tid; t < nc; t += T) {
                const int Zl = fdiv(t, cl.mP[l + 1]);
                const int Z = zc0 + Zl, q = t - Zl * Pc;
                const int J = fdiv(q, cl.mX[l + 1]), I = q - J * nxc;   // J = 0 when D == 1
                C sum = (C)0;
                for (int dz = 0; dz < 2; ++dz) {
                    const C* pl = plane_ptr(res, l, 2 * Z + dz);
                    for (int dy = 0; dy < fy; ++dy)
                        for (int dx = 0; dx < fx; ++dx) sum += pl[(I * fx + dx) + nxf * (J * fy + dy)];
                }
                Rc[t] = sum / (C)(2 * fx * fy);
            }
        }
        level_sync(l + 1);
    }
    // ---------------------------------------------------------------- coarsest: dense solve
    {
        const int l = cl.nl - 1;
        const int n = my_n(l), Pn = cl.plane[l], z0 = my_z0(l);
        const int Nt = (int)cl.lv[l].N;
        C* R = arr(l, 2);
        C* E0 = arr(l, 0);
        const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
        for (int t = warp; t < n; t += nw) {
            const int row = z0 * Pn + t;   // global cell index
            double acc = 0.0;
            const double* a = Ainv + (size_t)row * Nt;
            for (int col = lane; col < Nt; col += 32) {
                const int zc = fdiv(col, cl.mP[l]);
                acc += __ldg(a + col) * (double)plane_ptr(R, l, zc)[col - zc * Pn];
            }
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) E0[t] = (C)acc;
        }
    }
    level_sync(cl.nl - 1);
    // ---------------------------------------------------------------- up
    int fin = 0;
    for (int l = cl.nl - 2; l >= 0; --l) {
        const LevelDev& L = cl.lv[l];
        const LevelDev& Lc = cl.lv[l + 1];
        const int n = my_n(l), P = cl.plane[l], z0 = my_z0(l);
        const int cur_c = (l + 1 == cl.nl - 1) ? 0 : (down ^ (cl.post & 1));
        C* ec = arr(l + 1, cur_c);
        C* e = arr(l, down);
        uint16_t* F = codes(l);
        const bool local = l >= cl.lm;
        // leaving the CTA-0 levels: the other CTAs read the coarse correction from CTA 0
        if (l + 1 == cl.lm) cluster.sync();
        if (!local || me == 0) {
            // prolongation: 3/4 parent + 1/4 neighbour per active axis, neighbour clamped
            {
                const int nxf = L.n[0], nxc = Lc.n[0];
                const int fa_x = L.active[0], fa_y = D == 2 ? L.active[1] : 0;
                const int nyc = D == 2 ? Lc.n[1] : 1;
                const int nzc = cl.nD[l + 1];
                for (int t = tid; t < n; t += T) {
                    if (solid_code(F[t])) continue;
                    const int zl = fdiv(t, cl.mP[l]);
                    const int z = z0 + zl, q = t - zl * P;
                    const int j = fdiv(q, cl.mX[l]), i = q - j * nxf;
                    int Pi, Qi, Pj, Qj;
                    C wx0, wx1, wy0, wy1;
                    if (fa_x) {
                        Pi = i >> 1;
                        Qi = min(max(Pi + ((i & 1) ? 1 : -1), 0), nxc - 1);
                        wx0 = (C)0.75; wx1 = (C)0.25;
                    } else { Pi = Qi = i; wx0 = (C)1; wx1 = (C)0; }
                    if (fa_y) {
                        Pj = j >> 1;
                        Qj = min(max(Pj + ((j & 1) ? 1 : -1), 0), nyc - 1);
                        wy0 = (C)0.75; wy1 = (C)0.25;
                    } else { Pj = Qj = j; wy0 = (C)1; wy1 = (C)0; }
                    const int Pz = z >> 1;
                    const int Qz = min(max(Pz + ((z & 1) ? 1 : -1), 0), nzc - 1);
                    const C* pz0 = plane_ptr(ec, l + 1, Pz);
                    const C* pz1 = plane_ptr(ec, l + 1, Qz);
                    auto plane_val = [&](const C* pl) {
                        C v = wy0 * (wx0 * pl[Pi + nxc * Pj] + wx1 * pl[Qi + nxc * Pj]);
                        if (fa_y) v += wy1 * (wx0 * pl[Pi + nxc * Qj] + wx1 * pl[Qi + nxc * Qj]);
                        return v;
                    };
                    e[t] += (C)0.75 * plane_val(pz0) + (C)0.25 * plane_val(pz1);
                }
            }
            level_sync(l);
            int s = down;
            const C w = LP<C>::wJ(L), iD = LP<C>::iD(L);
            C* R = arr(l, 2);
            for (int it = 0; it < cl.post; ++it) {
                C* ein = arr(l, s);
                C* eo = arr(l, s ^ 1);
#pragma unroll 4
                for (int t = tid; t < n; t += T) {
                    const uint32_t f = F[t];
                    C v = (C)0;
                    if (!solid_code(f)) {
                        const C eP = ein[t];
                        v = eP + w * (R[t] - apply_A(l, ein, t, f, eP)) * iD;
                    }
                    eo[t] = v;
                }
                s ^= 1;
                level_sync(l);
            }
            fin = s;
        }
    }
    {
        const int n = my_n(0), off = my_z0(0) * cl.plane[0];
        const C* e = arr(0, cl.nl > 1 ? fin : 0);
        for (int t = tid; t < n; t += T) e_out[off + t] = from_c<TI, C>(e[t]);
    }
    // no CTA may exit while another still reads its shared memory
    cluster.sync();
}

}  // namespace

size_t cluster_smem_bytes(const ClusterLevels& cl, int inner) {
    (void)inner;
    return (size_t)cl.fbyte0 + (size_t)cl.fcount * 2 + 16;
}

#define DISPATCH_I(inner, ...)                                            \
    do {                                                                  \
        if ((inner) == FVM_FP64) { using TI = double; __VA_ARGS__; }      \
        else if ((inner) == FVM_FP32) { using TI = float; __VA_ARGS__; } \
        else { using TI = __nv_bfloat16; __VA_ARGS__; }                   \
    } while (0)

// Set the kernel attributes for a cluster of cs CTAs with smem bytes each and
// report how many such clusters the GPU can hold (0: not schedulable).
cudaError_t prepare_coarse_cluster(int inner, int cs, size_t smem, int* max_clusters) {
    *max_clusters = 0;
    cudaError_t err = cudaSuccess;
    DISPATCH_I(inner, {
        auto k = k_coarse_cluster<TI>;
        err = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (err == cudaSuccess) err = raise_smem_limit((const void*)k, smem);
        if (err == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(cs);
            cfg.blockDim = dim3(1024);
            cfg.dynamicSmemBytes = smem;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = cs;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            err = cudaOccupancyMaxActiveClusters(max_clusters, (const void*)k, &cfg);
        }
    });
    if (err != cudaSuccess) cudaGetLastError();
    return err;
}

cudaError_t launch_coarse_cluster(int inner, const ClusterLevels& cl, const void* r_in, void* e_out,
                                  const double* Ainv, const SolveState* st, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl.cs);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = cluster_smem_bytes(cl, inner);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    DISPATCH_I(inner, return cudaLaunchKernelEx(&cfg, k_coarse_cluster<TI>, cl, (const TI*)r_in, (TI*)e_out, Ainv, st));
    return cudaErrorInvalidValue;
}
