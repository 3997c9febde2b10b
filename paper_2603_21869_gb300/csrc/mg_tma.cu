// Fused level kernels of the V-cycle fed by the Tensor Memory Accelerator.
//
// Smoother (Eq. jacobi_pc, weighted), residual, restriction (Eq. restriction,
// mean of the 2x2x2 children) and trilinear prolongation (Eq. prolongation)
// for one grid level, with several sweeps in one pass over the data
// (temporal blocking).  A block owns a TX x TY tile of the x-y plane and
// marches through a chunk of z planes.  For each plane, one elected thread
// issues cp.async.bulk.tensor copies of the input planes (with a halo) into a
// ring of shared-memory slots, each guarded by an mbarrier; the sweeps form a
// software pipeline in which stage s computes plane tau - s on a region whose
// halo shrinks by one cell per stage.  Each stage keeps its last three planes
// (the z neighbours of the next stage) in shared memory.
//
//   down<N>: e_in -> N Jacobi sweeps -> e_out, and r_c = RES(r - A e_out)
//   up<N>:   e_in + PROL(e_c) -> N Jacobi sweeps -> e_out (or p += e)
//
// FP32 data; x extent a multiple of TX, y of TY, z of the chunk; 3D grids.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "fvm_internal.cuh"

namespace {

constexpr int TX = 32, TY = 16, NT = TX * TY;   // output tile, threads per block
constexpr int WX = TX + 8;                       // FP32 rows: x halo of 4 on each side (x start 16-byte aligned)
constexpr int WXF = TX + 16;                     // 16-bit code rows: x halo of 8 (x start a multiple of 8 elements)
constexpr int PF = 2;                            // planes loaded ahead
constexpr long long kWaitLimit = 1ll << 22;      // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cta.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// bounded wait on the slot barrier; on time-out record it and report false
__device__ __forceinline__ bool wait_slot(uint64_t* bar, uint32_t parity, SolveState* st) {
    long long it = 0;
    while (!mbar_try_wait(bar, parity)) {
        if (++it > kWaitLimit) {
            st->tma_timeout = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ float pick(uint32_t code, float nb, float eP) {
    return code == 0 ? nb : (code == 1 ? eP : -eP);
}

// one plane of a stage: value at tile-relative (xr, yr); rows of pitch WX start at y = -H
template <int H>
struct PlaneRef {
    float* p;
    __device__ __forceinline__ float& at(int xr, int yr) const { return p[(yr + H) * WX + (xr + 4)]; }
};
template <int H>
struct CodeRef {
    const uint16_t* p;
    __device__ __forceinline__ uint32_t at(int xr, int yr) const { return p[(yr + H) * WXF + (xr + 8)]; }
};

// Jacobi sweep value at (xr, yr) of a plane from the three input planes of the previous stage
template <int H>
__device__ __forceinline__ float sweep_at(const LevelDev& L, int xr, int yr, uint32_t f, PlaneRef<H> em,
                                          PlaneRef<H> ec, PlaneRef<H> ep, float rr) {
    if ((f >> 12) & 1u) return 0.f;
    const float eP = ec.at(xr, yr);
    float acc = ((eP - pick(f & 3u, ec.at(xr - 1, yr), eP)) + (eP - pick((f >> 2) & 3u, ec.at(xr + 1, yr), eP))) *
                L.inv_h2f[0];
    acc += ((eP - pick((f >> 4) & 3u, ec.at(xr, yr - 1), eP)) + (eP - pick((f >> 6) & 3u, ec.at(xr, yr + 1), eP))) *
           L.inv_h2f[1];
    acc += ((eP - pick((f >> 8) & 3u, em.at(xr, yr), eP)) + (eP - pick((f >> 10) & 3u, ep.at(xr, yr), eP))) *
           L.inv_h2f[2];
    return eP + L.wJf * (rr - acc) * L.inv_Df;
}

__device__ __forceinline__ float resid_at(const LevelDev& L, int xr, int yr, uint32_t f, PlaneRef<1> em,
                                          PlaneRef<1> ec, PlaneRef<1> ep, float rr) {
    if ((f >> 12) & 1u) return 0.f;
    const float eP = ec.at(xr, yr);
    float acc = ((eP - pick(f & 3u, ec.at(xr - 1, yr), eP)) + (eP - pick((f >> 2) & 3u, ec.at(xr + 1, yr), eP))) *
                L.inv_h2f[0];
    acc += ((eP - pick((f >> 4) & 3u, ec.at(xr, yr - 1), eP)) + (eP - pick((f >> 6) & 3u, ec.at(xr, yr + 1), eP))) *
           L.inv_h2f[1];
    acc += ((eP - pick((f >> 8) & 3u, em.at(xr, yr), eP)) + (eP - pick((f >> 10) & 3u, ep.at(xr, yr), eP))) *
           L.inv_h2f[2];
    return rr - acc;
}

// shared layout of one input slot: e plane, r plane, codes plane, all WX x (TY + 2H)
constexpr int round128(int b) { return (b + 127) / 128 * 128; }

template <int H>
struct Slot {
    static constexpr int ROWS = TY + 2 * H;
    static constexpr int EB = WX * ROWS * 4, RB = WX * ROWS * 4, FB = WXF * ROWS * 2;   // copied bytes
    static constexpr int EO = 0, RO = round128(EB), FO = RO + round128(RB);              // 128-byte aligned
    static constexpr int BYTES = FO + round128(FB);
};

// ------------------------------------------------------------------ down
// N sweeps on e_in (input halo HALO >= N + 1), then residual + restriction.
constexpr int HALO = 4;   // rows and columns of halo loaded around the tile (covers N <= 3 down, N <= 4 up)

template <int N>
__global__ void __launch_bounds__(NT) k_down_tma(const __grid_constant__ CUtensorMap tm_e,
                                                 const __grid_constant__ CUtensorMap tm_r,
                                                 const __grid_constant__ CUtensorMap tm_f, LevelDev L, LevelDev Lc,
                                                 float* __restrict__ e_out, float* __restrict__ rc, int zc,
                                                 SolveState* st) {
    constexpr int H = HALO;
    static_assert(N + 1 <= HALO, "down: N + 1 halo rows needed");
    constexpr int R = PF + N + 3;   // slots: a plane stays live for N + 2 steps after it lands
    using S = Slot<H>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if (!st->active) return;
    __shared__ uint64_t bars[R];
    // copies land on 128-byte boundaries: align the dynamic region explicitly
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint8_t* slots = smem;
    float* stage_base = (float*)(smem + R * S::BYTES);   // N stages x 3 planes
    float* resp = stage_base + 3 * N * WX * S::ROWS;     // residual tile TY x TX
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * zc;
    const int nz = L.n[2];
    auto slot_e = [&](int pl) { return PlaneRef<H>{(float*)(slots + ((pl % R + R) % R) * S::BYTES)}; };
    auto slot_r = [&](int pl) { return PlaneRef<H>{(float*)(slots + ((pl % R + R) % R) * S::BYTES + S::RO)}; };
    auto slot_f = [&](int pl) {
        return CodeRef<H>{(const uint16_t*)(slots + ((pl % R + R) % R) * S::BYTES + S::FO)};
    };
    auto stage = [&](int s, int pl) { return PlaneRef<H>{stage_base + (s * 3 + ((pl % 3) + 3) % 3) * WX * S::ROWS}; };

    if (tid == 0) {
        for (int i = 0; i < R; ++i) mbar_init(&bars[i], 1);
        fence_barrier_init();
    }
    __syncthreads();
    const int t0 = z0 - N - 1, t1 = z0 + zc + N;   // input planes streamed: [t0, t1]
    auto issue = [&](int pl) {
        if (pl < 0 || pl >= nz || pl > t1) return;
        // order earlier generic-proxy reads of this slot before the copy overwrites it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        uint64_t* b = &bars[((pl % R) + R) % R];
        mbar_expect_tx(b, (uint32_t)(S::EB + S::RB + S::FB));
        tma_load_3d(slot_e(pl).p, &tm_e, b, x0 - 4, y0 - H, pl);
        tma_load_3d(slot_r(pl).p, &tm_r, b, x0 - 4, y0 - H, pl);
        tma_load_3d((void*)slot_f(pl).p, &tm_f, b, x0 - 8, y0 - H, pl);
    };
    if (tid == 0)
        for (int k = 0; k < PF; ++k) issue(t0 + k);
    uint32_t phase = 0;   // bit per slot
    float racc = 0.f;     // restriction accumulator of this thread's coarse cell
    bool ok = true;
    for (int tau = t0; tau <= t1 && ok; ++tau) {
        if (tid == 0) issue(tau + PF);
        if (tau >= 0 && tau < nz) {
            const int sl = ((tau % R) + R) % R;
            const bool mine = wait_slot(&bars[sl], (phase >> sl) & 1u, st);
            phase ^= 1u << sl;
            ok = __syncthreads_and(mine) != 0;   // the whole block agrees before anyone leaves
            if (!ok) break;
        }
        // sweeps: stage s (1..N) computes plane tau - s on halo H - s
#pragma unroll
        for (int s = 1; s <= N; ++s) {
            const int pl = tau - s;
            if (pl >= 0 && pl < nz) {
                const int h = N + 1 - s;   // the residual needs the last sweep on a halo of 1
                const int w = TX + 2 * h, hh = TY + 2 * h;
                const PlaneRef<H> im = s == 1 ? slot_e(pl - 1) : stage(s - 2, pl - 1);
                const PlaneRef<H> ic = s == 1 ? slot_e(pl) : stage(s - 2, pl);
                const PlaneRef<H> ip = s == 1 ? slot_e(pl + 1) : stage(s - 2, pl + 1);
                const PlaneRef<H> rr = slot_r(pl);
                const CodeRef<H> ff = slot_f(pl);
                const PlaneRef<H> out = stage(s - 1, pl);
                for (int q = tid; q < w * hh; q += NT) {
                    const int xr = q % w - h, yr = q / w - h;
                    out.at(xr, yr) = sweep_at<H>(L, xr, yr, ff.at(xr, yr), im, ic, ip, rr.at(xr, yr));
                }
            }
            __syncthreads();
        }
        // residual on plane tau - N - 1 (the tile), e_out, restriction
        const int pl = tau - N - 1;
        if (pl >= z0 && pl < z0 + zc) {
            const int xr = tid % TX, yr = tid / TX;
            float ev, res;
            if (N > 0) {
                const PlaneRef<H> em = stage(N - 1, pl - 1), ec = stage(N - 1, pl), ep = stage(N - 1, pl + 1);
                ev = ec.at(xr, yr);
                res = resid_at(L, xr, yr, slot_f(pl).at(xr, yr), PlaneRef<1>{em.p + (H - 1) * WX},
                               PlaneRef<1>{ec.p + (H - 1) * WX}, PlaneRef<1>{ep.p + (H - 1) * WX},
                               slot_r(pl).at(xr, yr));
            } else {
                const PlaneRef<H> em = slot_e(pl - 1), ec = slot_e(pl), ep = slot_e(pl + 1);
                ev = ec.at(xr, yr);
                res = resid_at(L, xr, yr, slot_f(pl).at(xr, yr), PlaneRef<1>{em.p + (H - 1) * WX},
                               PlaneRef<1>{ec.p + (H - 1) * WX}, PlaneRef<1>{ep.p + (H - 1) * WX},
                               slot_r(pl).at(xr, yr));
            }
            const int c = (x0 + xr) + L.n[0] * ((y0 + yr) + L.n[1] * pl);
            e_out[c] = ev;
            resp[yr * TX + xr] = res;
        }
        __syncthreads();
        if (pl >= z0 && pl < z0 + zc && tid < (TX / 2) * (TY / 2)) {
            const int cx = tid % (TX / 2), cy = tid / (TX / 2);
            const float s4 = (resp[(2 * cy) * TX + 2 * cx] + resp[(2 * cy) * TX + 2 * cx + 1]) +
                             (resp[(2 * cy + 1) * TX + 2 * cx] + resp[(2 * cy + 1) * TX + 2 * cx + 1]);
            if ((pl & 1) == 0) racc = s4;
            else {
                const int C = (x0 / 2 + cx) + Lc.n[0] * ((y0 / 2 + cy) + Lc.n[1] * (pl >> 1));
                rc[C] = (racc + s4) * 0.125f;
            }
        }
        __syncthreads();
    }
    if (!ok) {
        // drain the copies this block issued (bounded), then leave
        for (int i = 0; i < R; ++i) {
            long long it = 0;
            while (!mbar_try_wait(&bars[i], (phase >> i) & 1u) && ++it < kWaitLimit) {
            }
        }
    }
}

// ------------------------------------------------------------------ up
// e' = e_in + PROL(e_c) on halo N, then N sweeps; the last writes e_out, or
// adds into the FP64 pressure (TOP).  Coarse planes stream through a 4-slot ring.
constexpr int CW = 24;                 // coarse tile width: X0 - 4 .. X0 + 19 (16-byte aligned start)
constexpr int CR = TY / 2 + 6;         // coarse tile rows: Y0 - 3 .. Y0 + TY/2 + 2
constexpr int CBYTES = round128(CW * CR * 4);

template <int N, bool TOP>
__global__ void __launch_bounds__(NT) k_up_tma(const __grid_constant__ CUtensorMap tm_e,
                                               const __grid_constant__ CUtensorMap tm_r,
                                               const __grid_constant__ CUtensorMap tm_f,
                                               const __grid_constant__ CUtensorMap tm_c, LevelDev L, LevelDev Lc,
                                               float* __restrict__ e_out, double* __restrict__ p, int zc,
                                               SolveState* st) {
    constexpr int H = HALO;
    static_assert(N <= HALO, "up: N halo rows needed");
    constexpr int R = PF + N + 3;
    using S = Slot<H>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if (!st->active) return;
    __shared__ uint64_t bars[R];
    __shared__ uint64_t cbars[4];
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint8_t* slots = smem;
    float* cslots = (float*)(smem + R * S::BYTES);
    float* stage_base = (float*)(smem + R * S::BYTES + 4 * CBYTES);   // N + 1 stages x 3 planes
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * zc;
    const int nz = L.n[2], ncz = Lc.n[2];
    const int CX0 = x0 / 2 - 4, CY0 = y0 / 2 - 3;
    auto slot_e = [&](int pl) { return PlaneRef<H>{(float*)(slots + ((pl % R + R) % R) * S::BYTES)}; };
    auto slot_r = [&](int pl) { return PlaneRef<H>{(float*)(slots + ((pl % R + R) % R) * S::BYTES + S::RO)}; };
    auto slot_f = [&](int pl) {
        return CodeRef<H>{(const uint16_t*)(slots + ((pl % R + R) % R) * S::BYTES + S::FO)};
    };
    auto cslot = [&](int cp) { return cslots + (cp & 3) * (CBYTES / 4); };
    auto stage = [&](int s, int pl) { return PlaneRef<H>{stage_base + (s * 3 + ((pl % 3) + 3) % 3) * WX * S::ROWS}; };

    if (tid == 0) {
        for (int i = 0; i < R; ++i) mbar_init(&bars[i], 1);
        for (int i = 0; i < 4; ++i) mbar_init(&cbars[i], 1);
        fence_barrier_init();
    }
    __syncthreads();
    const int t0 = z0 - N, t1 = z0 + zc + N - 1;
    auto issue = [&](int pl) {
        if (pl < 0 || pl >= nz || pl > t1) return;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        uint64_t* b = &bars[((pl % R) + R) % R];
        mbar_expect_tx(b, (uint32_t)(S::EB + S::RB + S::FB));
        tma_load_3d(slot_e(pl).p, &tm_e, b, x0 - 4, y0 - H, pl);
        tma_load_3d(slot_r(pl).p, &tm_r, b, x0 - 4, y0 - H, pl);
        tma_load_3d((void*)slot_f(pl).p, &tm_f, b, x0 - 8, y0 - H, pl);
    };
    // fine plane 2m needs coarse planes m - 1, m; plane 2m + 1 needs m, m + 1 (clamped)
    const int cfirst = max(0, (t0 - 1) >> 1), clast = min(ncz - 1, (t1 >> 1) + 1);
    int c_issued = cfirst - 1, c_waited = cfirst - 1;
    uint32_t cphase = 0;
    auto issue_coarse_upto = [&](int cp) {
        cp = min(cp, clast);
        while (c_issued < cp) {
            ++c_issued;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            uint64_t* b = &cbars[c_issued & 3];
            mbar_expect_tx(b, (uint32_t)(CW * CR * 4));
            tma_load_3d(cslot(c_issued), &tm_c, b, CX0, CY0, c_issued);
        }
    };
    if (tid == 0) {
        for (int k = 0; k < PF; ++k) issue(t0 + k);
        issue_coarse_upto(((t0 + 1) >> 1) + 1);
    }
    uint32_t phase = 0;
    bool ok = true;
    for (int tau = t0; tau <= t1 && ok; ++tau) {
        if (tid == 0) {
            issue(tau + PF);
            issue_coarse_upto(((tau + 3) >> 1) + 1);
        }
        bool mine = true;
        if (tau >= 0 && tau < nz) {
            const int sl = ((tau % R) + R) % R;
            mine = wait_slot(&bars[sl], (phase >> sl) & 1u, st);
            phase ^= 1u << sl;
            // coarse planes of this fine plane: parent and clamped neighbour
            const int need = min(ncz - 1, (tau >> 1) + 1);
            while (mine && c_waited < need) {
                ++c_waited;
                mine = wait_slot(&cbars[c_waited & 3], (cphase >> (c_waited & 3)) & 1u, st);
                cphase ^= 1u << (c_waited & 3);
            }
        }
        ok = __syncthreads_and(mine) != 0;
        if (!ok) break;
        // stage 0: prolongation on plane tau, halo N
        if (tau >= 0 && tau < nz) {
            const int w = TX + 2 * N, hh = TY + 2 * N;
            const PlaneRef<H> ein = slot_e(tau);
            const PlaneRef<H> out = stage(0, tau);
            const int Pz = tau >> 1;
            const int Qz = min(max(Pz + ((tau & 1) ? 1 : -1), 0), ncz - 1);
            const float* c0 = cslot(Pz);
            const float* c1 = cslot(Qz);
            for (int q = tid; q < w * hh; q += NT) {
                const int xr = q % w - N, yr = q / w - N;
                const int i = x0 + xr, j = y0 + yr;
                const int Pi = i >> 1, Pj = j >> 1;
                const int Qi = min(max(Pi + ((i & 1) ? 1 : -1), 0), Lc.n[0] - 1);
                const int Qj = min(max(Pj + ((j & 1) ? 1 : -1), 0), Lc.n[1] - 1);
                const int a0 = (Pj - CY0) * CW + (Pi - CX0), a1 = (Pj - CY0) * CW + (Qi - CX0);
                const int b0 = (Qj - CY0) * CW + (Pi - CX0), b1 = (Qj - CY0) * CW + (Qi - CX0);
                const float v0 = 0.75f * (0.75f * c0[a0] + 0.25f * c0[a1]) + 0.25f * (0.75f * c0[b0] + 0.25f * c0[b1]);
                const float v1 = 0.75f * (0.75f * c1[a0] + 0.25f * c1[a1]) + 0.25f * (0.75f * c1[b0] + 0.25f * c1[b1]);
                const uint32_t f = slot_f(tau).at(xr, yr);
                out.at(xr, yr) = ((f >> 12) & 1u) ? 0.f : ein.at(xr, yr) + (0.75f * v0 + 0.25f * v1);
            }
        }
        __syncthreads();
        // sweeps: stage s computes plane tau - s on halo N - s
#pragma unroll
        for (int s = 1; s <= N; ++s) {
            const int pl = tau - s;
            if (pl >= 0 && pl < nz) {
                const int h = N - s;
                const PlaneRef<H> im = stage(s - 1, pl - 1), ic = stage(s - 1, pl), ip = stage(s - 1, pl + 1);
                const PlaneRef<H> rr = slot_r(pl);
                const CodeRef<H> ff = slot_f(pl);
                if (s < N) {
                    const int w = TX + 2 * h, hh = TY + 2 * h;
                    const PlaneRef<H> out = stage(s, pl);
                    for (int q = tid; q < w * hh; q += NT) {
                        const int xr = q % w - h, yr = q / w - h;
                        out.at(xr, yr) = sweep_at<H>(L, xr, yr, ff.at(xr, yr), im, ic, ip, rr.at(xr, yr));
                    }
                } else if (pl >= z0 && pl < z0 + zc) {
                    const int xr = tid % TX, yr = tid / TX;
                    const uint32_t f = ff.at(xr, yr);
                    const float v = sweep_at<H>(L, xr, yr, f, im, ic, ip, rr.at(xr, yr));
                    const int c = (x0 + xr) + L.n[0] * ((y0 + yr) + L.n[1] * pl);
                    if (TOP) {
                        if (!((f >> 12) & 1u)) p[c] += (double)v;
                    } else {
                        e_out[c] = v;
                    }
                }
            }
            __syncthreads();
        }
    }
    if (!ok) {
        for (int i = 0; i < R; ++i) {
            long long it = 0;
            while (!mbar_try_wait(&bars[i], (phase >> i) & 1u) && ++it < kWaitLimit) {
            }
        }
        for (int i = 0; i < 4; ++i) {
            long long it = 0;
            while (!mbar_try_wait(&cbars[i], (cphase >> i) & 1u) && ++it < kWaitLimit) {
            }
        }
    }
}

template <int N>
constexpr size_t down_smem() {
    return 128 + (size_t)(PF + N + 3) * Slot<HALO>::BYTES + (size_t)3 * N * WX * Slot<HALO>::ROWS * 4 + TX * TY * 4;
}
template <int N>
constexpr size_t up_smem() {
    return 128 + (size_t)(PF + N + 3) * Slot<HALO>::BYTES + 4 * CBYTES +
           (size_t)3 * (N + 1) * WX * Slot<HALO>::ROWS * 4;
}

}  // namespace

// ---------------------------------------------------------------- host side
namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool load_encoder() {
    if (g_encode) return true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return false;
    }
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return true;
}

// 3D tiled map of an [nz][ny][nx] array with box {bx, by, 1}
bool encode3d(CUtensorMap* m, const void* base, int elem_bytes, const int* n, int bx, int by) {
    if (!load_encoder()) return false;
    cuuint64_t dims[3] = {(cuuint64_t)n[0], (cuuint64_t)n[1], (cuuint64_t)n[2]};
    cuuint64_t strides[2] = {(cuuint64_t)n[0] * elem_bytes, (cuuint64_t)n[0] * n[1] * elem_bytes};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t es[3] = {1, 1, 1};
    const CUtensorMapDataType t = elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    CUresult r = g_encode(m, t, 3, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

// Does level L qualify for the fused TMA kernels (FP32, 3D, tile-divisible)?
bool tma_level_ok(const LevelDev& L, const LevelDev& Lc) {
    return L.active[0] && L.active[1] && L.active[2] && L.n[0] % TX == 0 && L.n[1] % TY == 0 && L.n[2] % 2 == 0 &&
           (L.n[0] * 4) % 16 == 0 && (L.n[0] * 2) % 16 == 0 && (Lc.n[0] * 4) % 16 == 0 && L.n[0] >= TX &&
           Lc.n[0] * 2 == L.n[0] && Lc.n[1] * 2 == L.n[1] && Lc.n[2] * 2 == L.n[2];
}

// Tensor maps of one level: e[0], e[1], r, codes with the fine box, coarse e[0], e[1] with the coarse box.
bool tma_make_maps(TmaMaps& mp, const LevelDev& L, const LevelDev& Lc, void* const* e, const void* r,
                   void* const* ec) {
    const int* n = L.n;
    bool ok = true;
    for (int b = 0; b < 2; ++b) {
        ok = ok && encode3d(&mp.e[b], e[b], 4, n, WX, TY + 2 * HALO);
        ok = ok && encode3d(&mp.ec[b], ec[b], 4, Lc.n, CW, CR);
    }
    ok = ok && encode3d(&mp.r, r, 4, n, WX, TY + 2 * HALO);
    ok = ok && encode3d(&mp.f, L.nbf, 2, n, WXF, TY + 2 * HALO);
    return ok;
}

// z planes per block: the largest of 16, 8, 4, 2 dividing nz that still gives >= 2 blocks per SM
static int chunk_of(const LevelDev& L) {
    const int tiles = (L.n[0] / TX) * (L.n[1] / TY);
    for (int zc : {16, 8, 4})
        if (L.n[2] % zc == 0 && tiles * (L.n[2] / zc) >= 304) return zc;
    for (int zc : {4, 2})
        if (L.n[2] % zc == 0) return zc;
    return 2;
}

template <int N>
static cudaError_t down_n(const TmaMaps& mp, int ein, const LevelDev& L, const LevelDev& Lc, float* e_out, float* rc,
                          SolveState* st, cudaStream_t s) {
    const size_t smem = down_smem<N>();
    const int zc = chunk_of(L);
    k_down_tma<N><<<dim3(L.n[0] / TX, L.n[1] / TY, L.n[2] / zc), NT, smem, s>>>(mp.e[ein], mp.r, mp.f, L, Lc, e_out,
                                                                             rc, zc, st);
    return cudaGetLastError();
}

template <int N, bool TOP>
static cudaError_t up_n(const TmaMaps& mp, int ein, int ecb, const LevelDev& L, const LevelDev& Lc, float* e_out,
                        double* p, SolveState* st, cudaStream_t s) {
    const size_t smem = up_smem<N>();
    const int zc = chunk_of(L);
    k_up_tma<N, TOP><<<dim3(L.n[0] / TX, L.n[1] / TY, L.n[2] / zc), NT, smem, s>>>(mp.e[ein], mp.r, mp.f, mp.ec[ecb],
                                                                                 L, Lc, e_out, p, zc, st);
    return cudaGetLastError();
}

cudaError_t launch_down_tma(int nsweeps, const TmaMaps& mp, int ein, const LevelDev& L, const LevelDev& Lc,
                            void* e_out, void* rc, SolveState* st, cudaStream_t s) {
    switch (nsweeps) {
        case 0: return down_n<0>(mp, ein, L, Lc, (float*)e_out, (float*)rc, st, s);
        case 1: return down_n<1>(mp, ein, L, Lc, (float*)e_out, (float*)rc, st, s);
        case 2: return down_n<2>(mp, ein, L, Lc, (float*)e_out, (float*)rc, st, s);
        case 3: return down_n<3>(mp, ein, L, Lc, (float*)e_out, (float*)rc, st, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_up_tma(int nsweeps, bool top, const TmaMaps& mp, int ein, int ecb, const LevelDev& L,
                          const LevelDev& Lc, void* e_out, double* p, SolveState* st, cudaStream_t s) {
    if (top) {
        switch (nsweeps) {
            case 1: return up_n<1, true>(mp, ein, ecb, L, Lc, (float*)e_out, p, st, s);
            case 2: return up_n<2, true>(mp, ein, ecb, L, Lc, (float*)e_out, p, st, s);
            case 3: return up_n<3, true>(mp, ein, ecb, L, Lc, (float*)e_out, p, st, s);
            case 4: return up_n<4, true>(mp, ein, ecb, L, Lc, (float*)e_out, p, st, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (nsweeps) {
        case 1: return up_n<1, false>(mp, ein, ecb, L, Lc, (float*)e_out, p, st, s);
        case 2: return up_n<2, false>(mp, ein, ecb, L, Lc, (float*)e_out, p, st, s);
        case 3: return up_n<3, false>(mp, ein, ecb, L, Lc, (float*)e_out, p, st, s);
        case 4: return up_n<4, false>(mp, ein, ecb, L, Lc, (float*)e_out, p, st, s);
        default: return cudaErrorInvalidValue;
    }
}

// shared-memory limits of every fused kernel instance (once per process)
cudaError_t tma_prepare() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* k, size_t b) {
        if (e == cudaSuccess) e = raise_smem_limit(k, b);
    };
    set((const void*)k_down_tma<0>, down_smem<0>());
    set((const void*)k_down_tma<1>, down_smem<1>());
    set((const void*)k_down_tma<2>, down_smem<2>());
    set((const void*)k_down_tma<3>, down_smem<3>());
    set((const void*)k_up_tma<1, false>, up_smem<1>());
    set((const void*)k_up_tma<2, false>, up_smem<2>());
    set((const void*)k_up_tma<3, false>, up_smem<3>());
    set((const void*)k_up_tma<4, false>, up_smem<4>());
    set((const void*)k_up_tma<1, true>, up_smem<1>());
    set((const void*)k_up_tma<2, true>, up_smem<2>());
    set((const void*)k_up_tma<3, true>, up_smem<3>());
    set((const void*)k_up_tma<4, true>, up_smem<4>());
    if (e == cudaSuccess) done = true;
    return e;
}
