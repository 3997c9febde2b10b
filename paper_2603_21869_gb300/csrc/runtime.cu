// Host runtime of the k-omega finite-volume library: descriptor validation,
// boundary and obstacle tables, the multigrid level hierarchy, the dense
// coarsest-level inverse, device memory, and the order of kernels in one
// time step (Section 2.6: dt/2 destruction, explicit stage, dt/2
// destruction, pressure solve, projection).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <tuple>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "fvm_internal.cuh"

namespace {

thread_local std::string g_err;

fvm_status fail(fvm_status st, const std::string& msg) {
    g_err = msg;
    return st;
}

#define CUDA_TRY(expr)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(FVM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));    \
    } while (0)

constexpr double kCmu = 0.09;
constexpr double kBetaI = 0.072;

size_t elem_size(int prec) { return prec == FVM_FP64 ? 8 : (prec == FVM_FP32 ? 4 : 2); }

// The stages of a step before the pressure solve (Section 2.6): the time step, the first
// destruction half step, the explicit stage, and the second half step fused with the pressure
// right-hand side (an internal stage: fvm_run_stage runs the two separately)
constexpr int kStageDestructionRhs = 100;
constexpr int kStepStages[4] = {FVM_STAGE_DT, FVM_STAGE_DESTRUCTION, FVM_STAGE_EXPLICIT, kStageDestructionRhs};

struct HostLevel {
    int n[3];
    int active[3];
    double h[3];
    std::vector<uint8_t> solid;
    std::vector<uint8_t> dir[6];
    std::vector<uint16_t> nbf;
    int64_t N() const { return (int64_t)n[0] * n[1] * n[2]; }
};

// Neighbour codes of every cell (see LevelDev::nbf).
void build_nbf(HostLevel& L) {
    L.nbf.assign(L.N(), 0);
    for (int k = 0; k < L.n[2]; ++k)
        for (int j = 0; j < L.n[1]; ++j)
            for (int i = 0; i < L.n[0]; ++i) {
                const int64_t c = cell_index(i, j, k, L.n[0], L.n[1]);
                if (L.solid[c]) {
                    L.nbf[c] = (uint16_t)(1u << 12);
                    continue;
                }
                uint32_t code = 0;
                bool irregular = false;   // a ghost that a neighbour load clamped into the grid does not give
                const int f[3] = {i, j, k};
                for (int d = 0; d < 6; ++d) {
                    const int a = d / 2, side = (d & 1) ? 1 : -1;
                    int q[3] = {f[0], f[1], f[2]};
                    q[a] += side;
                    uint32_t v;
                    if (q[a] < 0 || q[a] >= L.n[a]) {
                        v = L.dir[d][face_index(a, i, j, k, L.n)] ? 2u : 1u;
                        irregular = irregular || v == 2u;
                    } else {
                        v = L.solid[cell_index(q[0], q[1], q[2], L.n[0], L.n[1])] ? 1u : 0u;
                        irregular = irregular || v == 1u;
                    }
                    code |= v << (2 * d);
                }
                if (irregular) code |= 1u << 13;
                L.nbf[c] = (uint16_t)code;
            }
}

int face_cells(const int* n, int face) {
    const int a = face / 2;
    int m = 1;
    for (int b = 0; b < 3; ++b)
        if (b != a) m *= n[b];
    return m;
}

void face_dims(const int* n, int face, int& na, int& nb) {
    const int a = face / 2;
    const int t0 = a == 0 ? 1 : 0;
    const int t1 = a == 2 ? 1 : 2;
    na = n[t0];
    nb = n[t1];
}

void inlet_kw(const fvm_patch& p, double& k0, double& om0) {
    k0 = 0.0;
    om0 = 0.0;
    if (p.intensity > 0.0 && p.length_scale > 0.0) {
        // Section 3.2.4: k0 = 1.5 (I0 u0)^2, eps0 = k0^1.5 / l0, omega0 = eps0 / (C_mu k0)
        k0 = 1.5 * (p.intensity * p.u_normal) * (p.intensity * p.u_normal);
        const double eps0 = std::pow(k0, 1.5) / p.length_scale;
        om0 = k0 > 0.0 ? eps0 / (kCmu * k0) : 0.0;
    }
    if (p.k_value > 0.0) k0 = p.k_value;
    if (p.omega_value > 0.0) om0 = p.omega_value;
}

HostLevel coarsen(const HostLevel& f) {
    HostLevel c;
    int fac[3];
    for (int a = 0; a < 3; ++a) {
        fac[a] = f.active[a] ? 2 : 1;
        c.n[a] = f.n[a] / fac[a];
        c.h[a] = f.h[a] * fac[a];
        c.active[a] = f.active[a];
    }
    c.solid.assign(c.N(), 1);
    for (int K = 0; K < c.n[2]; ++K)
        for (int J = 0; J < c.n[1]; ++J)
            for (int I = 0; I < c.n[0]; ++I) {
                uint8_t all = 1;
                for (int dz = 0; dz < fac[2]; ++dz)
                    for (int dy = 0; dy < fac[1]; ++dy)
                        for (int dx = 0; dx < fac[0]; ++dx)
                            all &= f.solid[cell_index(I * fac[0] + dx, J * fac[1] + dy, K * fac[2] + dz, f.n[0],
                                                      f.n[1])] ? 1 : 0;
                c.solid[cell_index(I, J, K, c.n[0], c.n[1])] = all;
            }
    for (int face = 0; face < 6; ++face) {
        const int a = face / 2;
        const int t0 = a == 0 ? 1 : 0, t1 = a == 2 ? 1 : 2;
        int cna, cnb, fna, fnb;
        face_dims(c.n, face, cna, cnb);
        face_dims(f.n, face, fna, fnb);
        c.dir[face].assign((size_t)cna * cnb, 0);
        for (int B = 0; B < cnb; ++B)
            for (int A = 0; A < cna; ++A) {
                uint8_t any = 0;
                for (int db = 0; db < fac[t1]; ++db)
                    for (int da = 0; da < fac[t0]; ++da)
                        any |= f.dir[face][(size_t)(A * fac[t0] + da) + (size_t)fna * (B * fac[t1] + db)];
                c.dir[face][(size_t)A + (size_t)cna * B] = any;
            }
    }
    return c;
}

// Dense A of the coarsest level (rows/cols of solid cells are the identity),
// inverted by Gauss-Jordan elimination with partial pivoting.
bool coarse_inverse(const HostLevel& L, std::vector<double>& inv) {
    const int64_t n = L.N();
    std::vector<double> M((size_t)(n * n), 0.0);
    for (int k = 0; k < L.n[2]; ++k)
        for (int j = 0; j < L.n[1]; ++j)
            for (int i = 0; i < L.n[0]; ++i) {
                const int64_t P = cell_index(i, j, k, L.n[0], L.n[1]);
                if (L.solid[P]) {
                    M[P * n + P] = 1.0;
                    continue;
                }
                const int f[3] = {i, j, k};
                for (int a = 0; a < 3; ++a) {
                    if (!L.active[a]) continue;
                    const double ih2 = 1.0 / (L.h[a] * L.h[a]);
                    for (int side = -1; side <= 1; side += 2) {
                        int q[3] = {f[0], f[1], f[2]};
                        q[a] += side;
                        if (q[a] < 0 || q[a] >= L.n[a]) {
                            const int face = 2 * a + (side > 0 ? 1 : 0);
                            if (L.dir[face][face_index(a, i, j, k, L.n)]) M[P * n + P] += 2.0 * ih2;
                            continue;
                        }
                        const int64_t Q = cell_index(q[0], q[1], q[2], L.n[0], L.n[1]);
                        if (L.solid[Q]) continue;
                        M[P * n + P] += ih2;
                        M[P * n + Q] -= ih2;
                    }
                }
            }
    // M is symmetric positive definite when every fluid region reaches a zero-value face
    // (solid rows are identity rows): banded Cholesky M = L L^T, the band being the
    // stride of the outermost active axis, then A^-1 column by column from L y = e_j,
    // L^T x = y, the columns shared out among host threads
    int64_t b = 1;
    for (int a = 0; a < 3; ++a)
        if (L.active[a]) b = a == 0 ? 1 : (a == 1 ? L.n[0] : (int64_t)L.n[0] * L.n[1]);
    double scale = 0.0;
    for (double x : M) scale = std::max(scale, std::fabs(x));
    std::vector<double> C((size_t)(n * (b + 1)), 0.0);   // C[i*(b+1) + (i-j)] = L[i][j], 0 <= i-j <= b
    auto Lij = [&](int64_t i, int64_t j) -> double& { return C[(size_t)(i * (b + 1) + (i - j))]; };
    for (int64_t j = 0; j < n; ++j) {
        double d = M[j * n + j];
        for (int64_t k = std::max<int64_t>(0, j - b); k < j; ++k) d -= Lij(j, k) * Lij(j, k);
        if (!(d > 1e-12 * scale)) return false;   // singular (no zero-value face reached)
        const double ljj = std::sqrt(d);
        Lij(j, j) = ljj;
        for (int64_t i = j + 1; i <= std::min(n - 1, j + b); ++i) {
            double v = M[i * n + j];
            for (int64_t k = std::max<int64_t>(0, i - b); k < j; ++k) v -= Lij(i, k) * Lij(j, k);
            Lij(i, j) = v / ljj;
        }
    }
    inv.assign((size_t)(n * n), 0.0);
    auto columns = [&](int64_t c0, int64_t c1) {
        std::vector<double> y((size_t)n);
        for (int64_t col = c0; col < c1; ++col) {
            std::fill(y.begin(), y.end(), 0.0);
            for (int64_t i = col; i < n; ++i) {   // L y = e_col (y is 0 above col)
                double v = i == col ? 1.0 : 0.0;
                for (int64_t k = std::max<int64_t>(col, i - b); k < i; ++k) v -= Lij(i, k) * y[(size_t)k];
                y[(size_t)i] = v / Lij(i, i);
            }
            for (int64_t i = n - 1; i >= 0; --i) {   // L^T x = y, x over y
                double v = y[(size_t)i];
                for (int64_t k = i + 1; k <= std::min(n - 1, i + b); ++k) v -= Lij(k, i) * y[(size_t)k];
                y[(size_t)i] = v / Lij(i, i);
            }
            for (int64_t r = 0; r < n; ++r) inv[(size_t)(r * n + col)] = y[(size_t)r];
        }
    };
    const int64_t nt = std::max<int64_t>(1, std::min<int64_t>((int64_t)std::thread::hardware_concurrency(), n / 64));
    std::vector<std::thread> pool;
    for (int64_t t = 0; t < nt; ++t) pool.emplace_back(columns, n * t / nt, n * (t + 1) / nt);
    for (auto& th : pool) th.join();
    return true;
}

}  // namespace

void set_last_error(const std::string& msg) { g_err = msg; }

thread_local Recorder* g_rec = nullptr;

bool pdl_enabled() {
    static const bool on = getenv("FVM_NO_PDL") == nullptr || getenv("FVM_NO_PDL")[0] == '0';
    return on;
}

namespace {
std::mutex g_smem_mu;
std::map<const void*, size_t> g_smem_limit;   // dynamic shared-memory limit set per kernel
}  // namespace

cudaError_t raise_smem_limit(const void* fn, size_t bytes) {
    // (set even below 48 KB: static shared memory counts against the default limit too)
    std::lock_guard<std::mutex> lock(g_smem_mu);
    auto& limit = g_smem_limit;
    size_t& have = limit[fn];
    if (bytes <= have) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    else cudaGetLastError();
    return e;
}

int persistent_blocks(const void* fn, int threads, size_t smem, bool query) {
    // keyed by everything the answer depends on: the kernel, its block size and shared memory, the device
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, size_t, int>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(fn, threads, smem, dev);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    if (!query) return 0;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (per_sm < 1) return 0;   // the kernel cannot run with this block: no launch
    const int n = sms * per_sm;
    cache[key] = n;
    return n;
}

bool smem_limit_covers(const void* fn, size_t bytes) {
    if (bytes == 0) return true;
    std::lock_guard<std::mutex> lock(g_smem_mu);
    auto it = g_smem_limit.find(fn);
    return it != g_smem_limit.end() && it->second >= bytes;
}

struct DevLevel {
    LevelDev dev;
    void* e[2] = {nullptr, nullptr};
    void* r = nullptr;
};

struct fvm_case {
    fvm_case_desc desc;
    std::vector<fvm_vent> vents;
    std::vector<fvm_box> boxes;
    int prec = FVM_FP64;    // storage of u, v, w, T, k, omega and b
    int inner = FVM_FP64;   // r, e on every multigrid level
    CaseDev cd;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* cur[6] = {};
    void* nxt[6] = {};
    void* rk3[6] = {};               // rk_stages = 3: the second stage's state
    double* p = nullptr;
    void* b = nullptr;
    double* dt_state = nullptr;
    double* partials = nullptr;
    double* norms = nullptr;
    double* h_norms = nullptr;
    double* h_dt = nullptr;
    double* staging = nullptr;
    double* Ainv = nullptr;
    double* p_tmp = nullptr;         // the paper's scheme: Jacobi on p out of place
    void* kdir = nullptr;            // flexible CG (krylov = 1): the kept direction (level 0, inner
    double* kpart = nullptr;         //   precision, FP32 for BF16) and four partial sums per level-0 block
    float* kz = nullptr;             //   BF16 inner: the V-cycles' level-0 correction z in FP32
    void* nut = nullptr;             // nu_t of the state after a destruction half step
    bool nut_valid = false;          // nut matches the current k, omega
    std::vector<DevLevel> levels;
    SolveState* sst = nullptr;       // device
    SolveState* h_sst = nullptr;     // pinned host copy
    size_t lc = 0;                   // first level cycled by the single-CTA coarse kernel
    int inner_cycles = 1;            // V-cycles per outer residual (adaptive solves)
    int rule_inner = 1;              // the same for the rule in force (1 for fixed-count solves)
    CoarseLevels coarse;
    // CUDA graphs of whole time steps, keyed by the field pointers they were captured with
    bool use_graph = true;
    struct StepGraph {
        void* before[12];
        void* after[12];
        cudaGraph_t g;
        cudaGraphExec_t exec;
    };
    std::vector<StepGraph> graphs;
    cudaStream_t side = nullptr;
    int64_t kpc = 0;                 // kernels in one V-cycle (after the level-0 residual)
    std::vector<void*> allocs;
    int64_t bytes = 0;
    int64_t steps = 0;
    double dt0 = 0.0;
    int nblocks0 = 0;
    // launch accounting and the profiling hook
    int64_t launches = 0;
    bool prof = false;
    struct ProfRec {
        int cls;
        cudaEvent_t a, b;
        double bytes;
    };
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    std::vector<std::string> cls_names;
};

namespace {

struct Plan {
    fvm_case_desc d;
    int prec, inner;
    double dt0;
    double base[6];
    std::vector<HostLevel> levels;
    std::vector<uint8_t> tag;
    std::vector<uint8_t> face_patch[6];
    std::vector<fvm_patch> patches;
    int64_t bytes;
};

fvm_status plan_case(const fvm_case_desc* d, Plan& pl) {
    if (!d) return fail(FVM_ERR_INVALID, "null descriptor");
    pl.d = *d;
    const int n[3] = {d->nx, d->ny, d->nz};
    const double Ls[3] = {d->Lx, d->Ly, d->Lz};
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1) return fail(FVM_ERR_INVALID, "grid dimensions must be >= 1");
        if (!(Ls[a] > 0.0)) return fail(FVM_ERR_INVALID, "domain lengths must be > 0");
        const bool e0 = d->faces[2 * a].kind == FVM_EMPTY, e1 = d->faces[2 * a + 1].kind == FVM_EMPTY;
        if ((n[a] == 1) != e0 || (n[a] == 1) != e1)
            return fail(FVM_ERR_INVALID, "an axis with one cell needs FVM_EMPTY on both faces, and only it");
    }
    const int64_t N = (int64_t)n[0] * n[1] * n[2];
    if (N > (int64_t)1 << 31) return fail(FVM_ERR_INVALID, "more than 2^31 cells");
    if (d->precision < FVM_FP64 || d->precision > FVM_BF16_MIXED) return fail(FVM_ERR_INVALID, "bad precision");
    if (!(d->nu > 0.0) || !(d->Pr > 0.0) || !(d->Prt > 0.0) || !(d->sigma_k > 0.0) || !(d->sigma_w > 0.0))
        return fail(FVM_ERR_INVALID, "nu, Pr, Prt, sigma_k, sigma_w must be > 0");
    if (d->mg_levels < 2 || d->mg_levels > FVM_MAX_LEVELS) return fail(FVM_ERR_INVALID, "mg_levels must be 2..12");
    if (d->pre_sweeps < 1 || d->post_sweeps < 1 || d->pre_sweeps > 64 || d->post_sweeps > 64)
        return fail(FVM_ERR_INVALID, "pre_sweeps and post_sweeps must be 1..64");
    if (d->inner_cycles < 0 || d->inner_cycles > 16) return fail(FVM_ERR_INVALID, "inner_cycles must be 0..16");
    if (d->sweep_planes < 0 || d->sweep_planes > 64) return fail(FVM_ERR_INVALID, "sweep_planes must be 0..64");
    if (d->mg_variant < 0 || d->mg_variant > 1) return fail(FVM_ERR_INVALID, "mg_variant must be 0 or 1");
    if (d->krylov < 0 || d->krylov > 1) return fail(FVM_ERR_INVALID, "krylov must be 0 or 1");
    if (d->krylov == 1 && d->mg_variant == 1) return fail(FVM_ERR_INVALID, "krylov 1 needs mg_variant 0");
    if (d->coarse_sweeps < 0 || d->coarse_sweeps > 64) return fail(FVM_ERR_INVALID, "coarse_sweeps must be 0..64");
    if (d->coarse_sweeps > 0 && d->mg_variant == 1) return fail(FVM_ERR_INVALID, "coarse_sweeps needs mg_variant 0");
    if (d->rk_stages < 0 || d->rk_stages > 3) return fail(FVM_ERR_INVALID, "rk_stages must be 0..3");
    if (d->smoother < 0 || d->smoother > 1) return fail(FVM_ERR_INVALID, "smoother must be 0 or 1");
    if (d->smoother == 1 && d->mg_variant == 1) return fail(FVM_ERR_INVALID, "smoother 1 needs mg_variant 0");
    if (d->smoother == 1 && (d->pre_sweeps > kMaxChebSweeps || d->post_sweeps > kMaxChebSweeps ||
                             d->coarse_sweeps > kMaxChebSweeps))
        return fail(FVM_ERR_INVALID, "smoother 1 takes at most 16 sweeps a side");
    if (d->fixed_vcycles < 0 || (d->fixed_vcycles == 0 && d->max_vcycles < 1))
        return fail(FVM_ERR_INVALID, "need fixed_vcycles > 0 or max_vcycles >= 1");
    if (d->fixed_vcycles == 0 && !(d->mg_rel_tol > 0.0)) return fail(FVM_ERR_INVALID, "mg_rel_tol must be > 0");
    if (d->n_vents < 0 || d->n_vents > FVM_MAX_PATCHES - 6) return fail(FVM_ERR_INVALID, "at most 10 vents");
    if (d->n_boxes < 0 || d->n_boxes > FVM_MAX_BOXES) return fail(FVM_ERR_INVALID, "at most 32 boxes");
    if ((d->n_vents > 0 && !d->vents) || (d->n_boxes > 0 && !d->boxes))
        return fail(FVM_ERR_INVALID, "null vent or box array");
    const int div = 1 << (d->mg_levels - 1);
    int64_t Nc = 1;
    for (int a = 0; a < 3; ++a) {
        if (n[a] == 1) continue;
        if (n[a] % div || n[a] / div < 2)
            return fail(FVM_ERR_INVALID,
                        "active grid dimensions must be divisible by 2^(mg_levels-1) with at least 2 coarsest cells");
        Nc *= n[a] / div;
    }
    if (Nc > FVM_MAX_COARSE) return fail(FVM_ERR_INVALID, "coarsest level above 1024 cells: add multigrid levels");

    pl.patches.assign(d->faces, d->faces + 6);
    for (int v = 0; v < d->n_vents; ++v) {
        const fvm_vent& ve = d->vents[v];
        if (ve.face < 0 || ve.face > 5) return fail(FVM_ERR_INVALID, "vent face must be 0..5");
        int na, nb;
        face_dims(n, ve.face, na, nb);
        if (ve.a0 < 0 || ve.a1 > na || ve.a0 >= ve.a1 || ve.b0 < 0 || ve.b1 > nb || ve.b0 >= ve.b1)
            return fail(FVM_ERR_INVALID, "vent rectangle outside its face");
        if (ve.bc.kind == FVM_EMPTY || d->faces[ve.face].kind == FVM_EMPTY)
            return fail(FVM_ERR_INVALID, "vents cannot be or sit on FVM_EMPTY faces");
        pl.patches.push_back(ve.bc);
    }
    for (const fvm_patch& p : pl.patches) {
        if (p.kind < FVM_WALL || p.kind > FVM_EMPTY) return fail(FVM_ERR_INVALID, "bad patch kind");
        if (p.kind == FVM_WALL && p.thermal == FVM_HEAT_FLUX && !(d->rho > 0.0 && d->cp > 0.0))
            return fail(FVM_ERR_INVALID, "heat-flux walls need rho, cp > 0");
    }
    for (int bi = 0; bi < d->n_boxes; ++bi) {
        const fvm_box& bx = d->boxes[bi];
        if (bx.i0 < 0 || bx.i1 > n[0] || bx.i0 >= bx.i1 || bx.j0 < 0 || bx.j1 > n[1] || bx.j0 >= bx.j1 ||
            bx.k0 < 0 || bx.k1 > n[2] || bx.k0 >= bx.k1)
            return fail(FVM_ERR_INVALID, "box outside the grid");
        if (bx.thermal == FVM_HEAT_FLUX && !(d->rho > 0.0 && d->cp > 0.0))
            return fail(FVM_ERR_INVALID, "heat-flux boxes need rho, cp > 0");
    }
    // tables
    pl.tag.assign(N, 0);
    for (int bi = 0; bi < d->n_boxes; ++bi) {
        const fvm_box& bx = d->boxes[bi];
        for (int k = bx.k0; k < bx.k1; ++k)
            for (int j = bx.j0; j < bx.j1; ++j)
                for (int i = bx.i0; i < bx.i1; ++i) pl.tag[cell_index(i, j, k, n[0], n[1])] = (uint8_t)(bi + 1);
    }
    if (d->n_boxes > 0 && std::find(pl.tag.begin(), pl.tag.end(), (uint8_t)0) == pl.tag.end())
        return fail(FVM_ERR_INVALID, "the boxes leave no fluid cell");
    for (int f = 0; f < 6; ++f) pl.face_patch[f].assign(face_cells(n, f), (uint8_t)f);
    for (int v = 0; v < d->n_vents; ++v) {
        const fvm_vent& ve = d->vents[v];
        int na, nb;
        face_dims(n, ve.face, na, nb);
        for (int bb = ve.b0; bb < ve.b1; ++bb)
            for (int aa = ve.a0; aa < ve.a1; ++aa) pl.face_patch[ve.face][(size_t)aa + (size_t)na * bb] = (uint8_t)(6 + v);
    }
    // level 0 and coarser levels
    HostLevel L0;
    bool any_dir = false;
    for (int a = 0; a < 3; ++a) {
        L0.n[a] = n[a];
        L0.active[a] = n[a] > 1;
        L0.h[a] = Ls[a] / n[a];
    }
    L0.solid.resize(N);
    for (int64_t c = 0; c < N; ++c) L0.solid[c] = pl.tag[c] ? 1 : 0;
    for (int f = 0; f < 6; ++f) {
        L0.dir[f].resize(pl.face_patch[f].size());
        for (size_t x = 0; x < L0.dir[f].size(); ++x) {
            L0.dir[f][x] = pl.patches[pl.face_patch[f][x]].kind == FVM_OUTLET ? 1 : 0;
            any_dir |= L0.dir[f][x] != 0;
        }
    }
    if (!any_dir) return fail(FVM_ERR_INVALID, "no outlet: the pressure problem would be singular");
    pl.levels.clear();
    pl.levels.push_back(L0);
    for (int l = 1; l < d->mg_levels; ++l) pl.levels.push_back(coarsen(pl.levels.back()));
    for (HostLevel& H : pl.levels) build_nbf(H);
    // time step
    double hmin = 1e300;
    for (int a = 0; a < 3; ++a)
        if (n[a] > 1) hmin = std::min(hmin, L0.h[a]);
    if (d->dt > 0.0) pl.dt0 = d->dt;
    else {
        if (!(d->cfl > 0.0)) return fail(FVM_ERR_INVALID, "need dt > 0 or cfl > 0");
        double U = 0.0;
        bool have = false;
        for (const fvm_patch& p : pl.patches)
            if (p.kind == FVM_INLET) {
                U = have ? std::max(U, p.u_normal) : p.u_normal;
                have = true;
            }
        if (!have)
            for (int a = 0; a < 3; ++a) U = std::max(U, std::fabs(d->init_vel[a]));
        if (U <= 0.0) U = 1.0;
        pl.dt0 = d->cfl * hmin / U;
    }
    // initial state base values
    double k0 = d->init_k, om0 = d->init_omega;
    if (k0 <= 0.0 || om0 <= 0.0) {
        bool found = false;
        for (const fvm_patch& p : pl.patches)
            if (p.kind == FVM_INLET) {
                double ik, iw;
                inlet_kw(p, ik, iw);
                if (k0 <= 0.0) k0 = ik;
                if (om0 <= 0.0) om0 = iw;
                found = true;
                break;
            }
        if (!found) return fail(FVM_ERR_INVALID, "init_k / init_omega <= 0 and no inlet to take them from");
    }
    pl.base[0] = d->init_vel[0];
    pl.base[1] = d->init_vel[1];
    pl.base[2] = d->init_vel[2];
    pl.base[3] = d->init_T;
    pl.base[4] = k0;
    pl.base[5] = om0;
    pl.prec = d->precision == FVM_FP64 ? FVM_FP64 : FVM_FP32;
    pl.inner = d->precision == FVM_FP64 ? FVM_FP64 : (d->precision == FVM_FP32 ? FVM_FP32 : FVM_BF16_MIXED);
    // bytes
    const size_t s = elem_size(pl.prec);
    const size_t si = elem_size(pl.inner);
    int64_t bytes = 0;
    bytes += (int64_t)12 * N * s;             // state, two copies of six fields
    bytes += N * 8 + N * s + N;               // p (FP64), b, tag
    bytes += N * 8;                           // staging
    bytes += N * s;                           // nu_t after a destruction half step
    if (d->rk_stages == 3) bytes += (int64_t)6 * N * s;   // the third-order scheme's stage state
    for (int f = 0; f < 6; ++f) bytes += face_cells(n, f);
    for (size_t l = 0; l < pl.levels.size(); ++l) {
        const int64_t NL = pl.levels[l].N();
        bytes += 3 * NL * si + (l ? NL : 0) + 2 * NL;
        for (int f = 0; f < 6; ++f) bytes += l ? (int64_t)pl.levels[l].dir[f].size() : 0;
    }
    const int64_t nc = pl.levels.back().N();
    bytes += nc * nc * 12;   // coarsest inverse, FP64 and FP32
    if (d->mg_variant == 1) bytes += N * 8;
    if (d->krylov == 1) bytes += N * si + (int64_t)4 * level0_blocks_max(n[0], n[1], n[2]) * 8;
    bytes += (int64_t)(2 * level0_blocks_max(n[0], n[1], n[2]) + 16) * 8 + 256;
    pl.bytes = bytes;
    return FVM_OK;
}

void prof_clear(fvm_case* c);
void drop_graphs(fvm_case* c);

void free_case(fvm_case* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    prof_clear(c);
    drop_graphs(c);
    if (c->side) cudaStreamDestroy(c->side);
    for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
    for (void* p : c->allocs) cudaFree(p);
    if (c->h_norms) cudaFreeHost(c->h_norms);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

fvm_status dalloc(fvm_case* c, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(FVM_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->allocs.push_back(*p);
    c->bytes += (int64_t)bytes;
    return FVM_OK;
}

#define ST_TRY(expr)                     \
    do {                                 \
        fvm_status s_ = (expr);          \
        if (s_ != FVM_OK) return s_;     \
    } while (0)

StatePtrs ptrs(void* const* f) {
    StatePtrs s;
    for (int i = 0; i < 6; ++i) s.f[i] = f[i];
    return s;
}

// ------------------------------------------------------------------ profiling
cudaEvent_t take_event(fvm_case* c) {
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

int prof_begin(fvm_case* c, const std::string& name, double bytes) {
    if (!c->prof) return -1;
    int cls = -1;
    for (size_t i = 0; i < c->cls_names.size(); ++i)
        if (c->cls_names[i] == name) cls = (int)i;
    if (cls < 0) {
        cls = (int)c->cls_names.size();
        c->cls_names.push_back(name);
    }
    fvm_case::ProfRec r{cls, take_event(c), take_event(c), bytes};
    if (!r.a || !r.b) return -1;
    cudaEventRecord(r.a, c->stream);
    c->recs.push_back(r);
    return (int)c->recs.size() - 1;
}

void prof_end(fvm_case* c, int idx) {
    if (idx >= 0) cudaEventRecord(c->recs[idx].b, c->stream);
}

void prof_clear(fvm_case* c) {
    for (auto& r : c->recs) {
        c->pool.push_back(r.a);
        c->pool.push_back(r.b);
    }
    c->recs.clear();
    c->cls_names.clear();
}

// Launch `expr` (which issues nk kernels), counting it and bracketing it with
// profiling events when the hook is on.  `bytes` = algorithmic bytes.
#define KLAUNCH(name, bytes_, nk, expr)                  \
    do {                                                \
        if (g_rec) {                                    \
            g_rec->site = (name);                       \
            g_rec->bytes = (bytes_);                     \
        }                                               \
        const int pi_ = prof_begin(c, (name), (bytes_)); \
        CUDA_TRY(expr);                                 \
        prof_end(c, pi_);                               \
        c->launches += (nk);                            \
    } while (0)

std::string lvl_name(const char* base, size_t l) { return std::string(base) + "_L" + std::to_string(l); }

// ------------------------------------------------------------------ solve
// One iteration of the paper's scheme (Algorithm 1) after the level-0 residual:
// restrict r straight down, one unweighted Jacobi step per coarse level on the
// way up from the nearest-upsampled coarser correction (zero on the coarsest),
// p += the upsampled level-1 correction, one unweighted Jacobi sweep on p.
fvm_status paper_cycle(fvm_case* c) {
    cudaStream_t s = c->stream;
    const int nl = (int)c->levels.size();
    const double si = (double)elem_size(c->inner);
    for (int l = 0; l + 1 < nl; ++l) {
        DevLevel& L = c->levels[l];
        DevLevel& Lc = c->levels[l + 1];
        KLAUNCH(lvl_name("restrict", l), (double)L.dev.N * si + (double)Lc.dev.N * si, 1,
                launch_restrict(c->inner, L.dev, Lc.dev, L.r, Lc.r, c->sst, s));
    }
    DevLevel& Lt = c->levels[nl - 1];
    KLAUNCH(lvl_name("sweep_first", nl - 1), 2.0 * Lt.dev.N * si + 2.0 * Lt.dev.N, 1,
            launch_sweep_first(c->inner, Lt.dev, Lt.r, Lt.e[0], c->sst, s));
    int cur = 0;   // buffer holding the correction of the level below the one being built
    for (int l = nl - 2; l >= 1; --l) {
        DevLevel& L = c->levels[l];
        DevLevel& Lc = c->levels[l + 1];
        const double N = (double)L.dev.N;
        KLAUNCH(lvl_name("prolong_nearest", l), N * si + (double)Lc.dev.N * si + 2 * N, 1,
                launch_prolong_nearest(c->inner, L.dev, Lc.dev, Lc.e[cur], L.e[0], c->sst, s));
        KLAUNCH(lvl_name("sweep", l), 3 * N * si + 2 * N, 1,
                launch_sweep(c->inner, L.dev, L.e[0], L.r, L.e[1], c->sst, s));
        cur = 1;
    }
    DevLevel& L0 = c->levels[0];
    DevLevel& L1 = c->levels[1];
    const double N0 = (double)L0.dev.N;
    KLAUNCH("prolong_nearest_to_p_L0", 16 * N0 + (double)L1.dev.N * si + 2 * N0, 1,
            launch_prolong_nearest_to_p(c->inner, L0.dev, L1.dev, L1.e[cur], c->p, c->sst, s));
    KLAUNCH("jacobi_p_L0", N0 * (8 + elem_size(c->prec) + 8 + 2) + 16 * N0, 2,
            launch_jacobi_p(c->prec, L0.dev, c->p, c->b, c->p_tmp, c->sst, s));
    return FVM_OK;
}

// Flexible CG with one kept direction: z = the level-0 correction in e[zi]
// (the V-cycles' result for the residual r), made A-orthogonal to the kept
// direction, then the step minimising the error's A-norm along it.
fvm_status krylov_step(fvm_case* c, int zi) {
    DevLevel& L = c->levels[0];
    const double N = (double)L.dev.N;
    const double si = (double)elem_size(c->inner);
    // BF16 levels: z and the kept direction in FP32 (z from the last sweep), r in BF16
    const bool f32 = c->inner == FVM_BF16_MIXED;
    const double sz = f32 ? 4.0 : si;
    KLAUNCH("fcg_L0", N * (4 * sz + si + sz + 20), 2,
            launch_fcg(c->inner, L.dev, f32 ? (void*)c->kz : L.e[zi], L.r, c->kdir, c->p, c->kpart, c->sst,
                       c->stream));
    return FVM_OK;
}

// pre- and post-sweeps on level l (coarse_sweeps on the levels below the finest, when set)
int pre_at(const fvm_case* c, size_t l) {
    return l > 0 && c->desc.coarse_sweeps > 0 ? c->desc.coarse_sweeps : c->desc.pre_sweeps;
}
int post_at(const fvm_case* c, size_t l) {
    return l > 0 && c->desc.coarse_sweeps > 0 ? c->desc.coarse_sweeps : c->desc.post_sweeps;
}

// The weight of sweep i of the n on one side of a level: the level's constant weight, or
// (smoother 1) the reciprocal of a root of the degree-n Chebyshev polynomial of [1/4, 2],
// (2 + 1/4)/2 + (2 - 1/4)/2 cos((2q + 1) pi / (2n)) for q = i before the coarse correction (largest
// root first) and q = n - 1 - i after it.
double sweep_weight(const fvm_case* c, const LevelDev& L, int n, int i, bool post) {
    if (c->desc.smoother != 1) return L.wJ;
    const int q = post ? n - 1 - i : i;
    return 1.0 / (1.125 + 0.875 * std::cos((2.0 * q + 1.0) * 3.14159265358979323846 / (2.0 * n)));
}

// a level's description with the weight of one sweep (the kernels read wJ / wJf)
LevelDev weighted(LevelDev v, double w) {
    v.wJ = w;
    v.wJf = (float)w;
    return v;
}

// Level l (> 0) gets its first Jacobi sweep from the restriction that forms its r
// (not the levels the single-CTA coarse kernel cycles).
bool first_sweep_fused(const fvm_case* c, size_t l) {
    return l > 0 && l < c->lc;
}

// One V-cycle of the correction equation on levels l.. with r on level l;
// returns the index of the e buffer holding the level's correction.  On
// level 0 the final post-smoothing sweep adds the correction to p instead.
fvm_status cycle(fvm_case* c, size_t l, int& out_idx) {
    if (c->desc.mg_variant == 1) {
        out_idx = 0;
        return paper_cycle(c);
    }
    DevLevel& L = c->levels[l];
    cudaStream_t s = c->stream;
    const double N = (double)L.dev.N;
    const double si = (double)elem_size(c->inner);
    if (l == c->lc) {
        const double nco = (double)c->levels.back().dev.N;
        double cells = 0.0;
        for (size_t q = l; q < c->levels.size(); ++q) cells += (double)c->levels[q].dev.N;
        KLAUNCH("coarse_cta", 2 * N * si + nco * nco * 8 + 2 * cells, 1,
                launch_coarse_cta(c->inner, c->coarse, L.r, L.e[0], c->Ainv, c->sst, s));
        out_idx = 0;
        return FVM_OK;
    }
    DevLevel& Lc = c->levels[l + 1];
    const double Nc = (double)Lc.dev.N;
    // level 0: the residual kernel already did the first sweep from e = 0, and
    // runs inner_cycles V-cycles on the same r; the last sweep of the last one adds e to p
    const int reps = l == 0 ? c->rule_inner : 1;
    int cur = 0;
    const int npre = pre_at(c, l), npost = post_at(c, l);
    for (int rep = 0; rep < reps; ++rep) {
        int pre = npre, first = 0;   // first: the index of the next pre-sweep's weight
        if (rep == 0) {
            if (l > 0 && !first_sweep_fused(c, l))
                KLAUNCH(lvl_name("sweep_first", l), 2 * N * si + 2 * N, 1,
                        launch_sweep_first(c->inner, weighted(L.dev, sweep_weight(c, L.dev, npre, 0, false)), L.r,
                                           L.e[0], c->sst, s));
            pre -= 1;
            first = 1;
        }
        for (int k = 0; k < pre; ++k) {
            KLAUNCH(lvl_name("sweep", l), 3 * N * si + 2 * N, 1,
                    launch_sweep(c->inner, weighted(L.dev, sweep_weight(c, L.dev, npre, first + k, false)),
                                 L.e[cur], L.r, L.e[cur ^ 1], c->sst, s));
            cur ^= 1;
        }
        const bool fuse = first_sweep_fused(c, l + 1);
        const LevelDev Lcw = weighted(Lc.dev, sweep_weight(c, Lc.dev, pre_at(c, l + 1), 0, false));
        KLAUNCH(lvl_name("resid_restrict", l), 2 * N * si + Nc * si + 2 * N + (fuse ? Nc * (si + 2) : 0.0), 1,
                launch_resid_restrict(c->inner, L.dev, Lcw, L.e[cur], L.r, Lc.r, fuse ? Lc.e[0] : nullptr,
                                      c->sst, s));
        int ci = 0;
        ST_TRY(cycle(c, l + 1, ci));
        KLAUNCH(lvl_name("prolong_add", l), 2 * N * si + Nc * si + 2 * N, 1,
                launch_prolong_add(c->inner, L.dev, Lc.dev, Lc.e[ci], L.e[cur], c->sst, s));
        const int post = npost;
        for (int k = 0; k < post; ++k) {
            const LevelDev Lw = weighted(L.dev, sweep_weight(c, L.dev, npost, k, true));
            if (l == 0 && rep == reps - 1 && k == post - 1 && !c->desc.krylov) {
                KLAUNCH("sweep_to_p_L0", 2 * N * si + 16 * N + 2 * N, 1,
                        launch_sweep_to_p(c->inner, Lw, L.e[cur], L.r, c->p, c->sst, s));
            } else if (l == 0 && rep == reps - 1 && k == post - 1 && c->kz) {
                // BF16 levels under the flexible-CG step: the correction z in FP32
                KLAUNCH("sweep_L0", 2 * N * si + 4 * N + 2 * N, 1,
                        launch_sweep_to_f32(c->inner, Lw, L.e[cur], L.r, c->kz, c->sst, s));
            } else {
                KLAUNCH(lvl_name("sweep", l), 3 * N * si + 2 * N, 1,
                        launch_sweep(c->inner, Lw, L.e[cur], L.r, L.e[cur ^ 1], c->sst, s));
                cur ^= 1;
            }
        }
    }
    if (l == 0 && c->desc.krylov) ST_TRY(krylov_step(c, cur));
    out_idx = cur;
    return FVM_OK;
}

// level-0 residual with the norm, the stopping rule and the first pre-sweep
fvm_status residual0(fvm_case* c, cudaGraphConditionalHandle cond, cudaGraphConditionalHandle cond2,
                     int use_cond) {
    const double N = (double)c->cd.N;
    KLAUNCH("resid0", N * (8 + elem_size(c->prec) + 2 * elem_size(c->inner) + 2), 1,
            launch_resid0(c->inner, c->prec,
                          weighted(c->levels[0].dev, sweep_weight(c, c->levels[0].dev, pre_at(c, 0), 0, false)), c->p,
                          c->b, c->levels[0].r, c->levels[0].e[0],
                          c->partials, c->sst, cond, cond2, use_cond, c->stream));
    return FVM_OK;
}

fvm_status read_state(fvm_case* c) {
    CUDA_TRY(cudaMemcpyAsync(c->h_sst, c->sst, sizeof(SolveState), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return FVM_OK;
}

// set the stopping rule of the next solves (fixed > 0: exactly that many cycles)
fvm_status set_rule(fvm_case* c, int fixed) {
    SolveState h;
    memset(&h, 0, sizeof(h));
    h.tol = c->desc.mg_rel_tol;
    h.max_cycles = c->desc.max_vcycles;
    h.fixed = fixed;
    h.inner = fixed > 0 ? 1 : c->inner_cycles;
    h.active = 1;
    c->rule_inner = h.inner;
    CUDA_TRY(cudaMemcpyAsync(c->sst, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return FVM_OK;
}

// V-cycles until the device-side rule stops (one host synchronisation per cycle)
fvm_status solve(fvm_case* c, int& cycles, double& rel) {
    KLAUNCH("solve_begin", 0.0, 1, launch_solve_begin(c->sst, c->stream));
    for (;;) {
        ST_TRY(residual0(c, 0, 0, 0));
        ST_TRY(read_state(c));
        if (!c->h_sst->active) break;
        int idx;
        ST_TRY(cycle(c, 0, idx));
    }
    cycles = c->h_sst->cycles;
    rel = c->h_sst->rel;
    return FVM_OK;
}

// ------------------------------------------------------------------ stages
fvm_status stage(fvm_case* c, int st, int* cycles, double* rel) {
    cudaStream_t s = c->stream;
    const double N = (double)c->cd.N;
    const double sz = (double)elem_size(c->prec);
    switch (st) {
        case FVM_STAGE_DT:
            KLAUNCH("dt", N * (5 * sz + 1), 2, launch_dt(c->prec, c->cd, ptrs(c->cur), c->dt_state, s));
            return FVM_OK;
        case FVM_STAGE_DESTRUCTION:
            KLAUNCH("destruction", N * (8 * sz + 3), 1,
                    launch_destruction(c->prec, c->cd, ptrs(c->cur), c->nxt[4], c->nxt[5], c->dt_state, c->nut,
                                       nullptr, s));
            std::swap(c->cur[4], c->nxt[4]);
            std::swap(c->cur[5], c->nxt[5]);
            c->nut_valid = true;
            return FVM_OK;
        case kStageDestructionRhs:
            // the second half step and the pressure right-hand side in one pass: both read the same
            // velocity, which the destruction step leaves unchanged (no nu_t: the next stage is the solve)
            KLAUNCH("destruction_rhs", N * (8 * sz + 3), 1,
                    launch_destruction(c->prec, c->cd, ptrs(c->cur), c->nxt[4], c->nxt[5], c->dt_state, nullptr,
                                       c->b, s));
            std::swap(c->cur[4], c->nxt[4]);
            std::swap(c->cur[5], c->nxt[5]);
            c->nut_valid = false;
            return FVM_OK;
        case FVM_STAGE_EXPLICIT: {
            // forward Euler, or the first stage of the Shu-Osher schemes: cur -> nxt
            KLAUNCH("explicit", N * (13 * sz + 3), 1,
                    launch_explicit(c->prec, c->cd, ptrs(c->cur), ptrs(c->nxt), c->dt_state,
                                    c->nut_valid ? c->nut : nullptr, StatePtrs{}, 0.0, 0.0, s));
            c->nut_valid = false;
            const int rk = c->desc.rk_stages;
            if (rk <= 1) {
                for (int f = 0; f < 6; ++f) std::swap(c->cur[f], c->nxt[f]);
                return FVM_OK;
            }
            // later stages: a u0 + b E(u_stage), u0 = cur; the last one overwrites cur in place
            // (each cell reads its own u0 value before writing it; the stencil reads u_stage)
            const double rk_bytes = N * (19 * sz + 1);
            if (rk == 2) {
                KLAUNCH("explicit_rk", rk_bytes, 1,
                        launch_explicit(c->prec, c->cd, ptrs(c->nxt), ptrs(c->cur), c->dt_state, nullptr,
                                        ptrs(c->cur), 0.5, 0.5, s));
            } else {
                KLAUNCH("explicit_rk", rk_bytes, 1,
                        launch_explicit(c->prec, c->cd, ptrs(c->nxt), ptrs(c->rk3), c->dt_state, nullptr,
                                        ptrs(c->cur), 0.75, 0.25, s));
                KLAUNCH("explicit_rk", rk_bytes, 1,
                        launch_explicit(c->prec, c->cd, ptrs(c->rk3), ptrs(c->cur), c->dt_state, nullptr,
                                        ptrs(c->cur), 1.0 / 3.0, 2.0 / 3.0, s));
            }
            return FVM_OK;
        }
        case FVM_STAGE_RHS:
            KLAUNCH("rhs", N * (4 * sz + 1), 1, launch_rhs(c->prec, c->cd, ptrs(c->cur), c->b, c->dt_state, s));
            return FVM_OK;
        case FVM_STAGE_SOLVE: {
            int cy = 0;
            double r = 0.0;
            ST_TRY(solve(c, cy, r));
            if (cycles) *cycles = cy;
            if (rel) *rel = r;
            return FVM_OK;
        }
        case FVM_STAGE_PROJECT:
            KLAUNCH("project", N * (6 * sz + 9), 1,
                    launch_project(c->prec, c->cd, c->levels[0].dev, ptrs(c->cur), ptrs(c->nxt), c->p,
                                   c->dt_state, s));
            for (int f = 0; f < 3; ++f) std::swap(c->cur[f], c->nxt[f]);
            return FVM_OK;
        default:
            return fail(FVM_ERR_INVALID, "unknown stage");
    }
}

// ------------------------------------------------------------------ graphs
void save_ptrs(const fvm_case* c, void** out) {
    for (int f = 0; f < 6; ++f) {
        out[f] = c->cur[f];
        out[6 + f] = c->nxt[f];
    }
}

void load_ptrs(fvm_case* c, void* const* in) {
    for (int f = 0; f < 6; ++f) {
        c->cur[f] = in[f];
        c->nxt[f] = in[6 + f];
    }
}

fvm_status stage(fvm_case* c, int st, int* cycles, double* rel);

// Capture one time step into a graph: the step kernels, then a while node
// whose body is the level-0 residual followed by an if node holding the
// V-cycle, both conditions set by the residual kernel.
fvm_status capture_step(fvm_case* c, fvm_case::StepGraph& G) {
    save_ptrs(c, G.before);
    const int64_t launches0 = c->launches;   // captured kernels are counted when they run
    cudaStream_t s = c->stream;
    if (!c->side) CUDA_TRY(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    auto abort_capture = [&](fvm_status st) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
        c->stream = s;
        c->launches = launches0;
        load_ptrs(c, G.before);
        cudaGetLastError();
        return st;
    };
    fvm_status st = FVM_OK;
    for (int k : kStepStages)
        if ((st = stage(c, k, nullptr, nullptr)) != FVM_OK) return abort_capture(st);
    if (launch_solve_begin(c->sst, s) != cudaSuccess) return abort_capture(fail(FVM_ERR_CUDA, "capture solve_begin"));
    c->launches += 1;
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &graph, &deps, nullptr, &ndeps) != cudaSuccess)
        return abort_capture(fail(FVM_ERR_CUDA, "cudaStreamGetCaptureInfo"));
    cudaGraphConditionalHandle hw, hi;
    if (cudaGraphConditionalHandleCreate(&hw, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess)
        return abort_capture(fail(FVM_ERR_CUDA, "cudaGraphConditionalHandleCreate"));
    cudaGraphNodeParams wp = {cudaGraphNodeTypeConditional};
    wp.conditional.handle = hw;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if (cudaGraphAddNode(&wnode, graph, deps, nullptr, ndeps, &wp) != cudaSuccess)
        return abort_capture(fail(FVM_ERR_CUDA, "adding the while node"));
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    // body: residual, then if (go) V-cycle
    if (cudaGraphConditionalHandleCreate(&hi, body, 0, cudaGraphCondAssignDefault) != cudaSuccess)
        return abort_capture(fail(FVM_ERR_CUDA, "cudaGraphConditionalHandleCreate (if)"));
    c->stream = c->side;
    if (cudaStreamBeginCaptureToGraph(c->side, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
        return abort_capture(fail(FVM_ERR_CUDA, "capturing the while body"));
    st = residual0(c, hw, hi, 2);
    cudaStreamCaptureStatus bcs;
    cudaGraph_t bg = nullptr;
    const cudaGraphNode_t* bdeps = nullptr;
    size_t nbdeps = 0;
    cudaGraphNode_t inode;
    cudaGraphNodeParams ip = {cudaGraphNodeTypeConditional};
    bool ok = st == FVM_OK &&
              cudaStreamGetCaptureInfo(c->side, &bcs, nullptr, &bg, &bdeps, nullptr, &nbdeps) == cudaSuccess;
    if (ok) {
        ip.conditional.handle = hi;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        ok = cudaGraphAddNode(&inode, bg, bdeps, nullptr, nbdeps, &ip) == cudaSuccess;
    }
    cudaGraph_t done_body = nullptr;
    cudaStreamEndCapture(c->side, &done_body);
    if (!ok) {
        c->stream = s;
        return abort_capture(st != FVM_OK ? st : fail(FVM_ERR_CUDA, "adding the if node"));
    }
    cudaGraph_t ibody = ip.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(c->side, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess) {
        c->stream = s;
        return abort_capture(fail(FVM_ERR_CUDA, "capturing the V-cycle body"));
    }
    int idx = 0;
    const int64_t before_cycle = c->launches;
    st = cycle(c, 0, idx);
    c->kpc = c->launches - before_cycle;
    cudaGraph_t done_if = nullptr;
    cudaStreamEndCapture(c->side, &done_if);
    c->stream = s;
    if (st != FVM_OK) return abort_capture(st);
    if (cudaStreamUpdateCaptureDependencies(s, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
        return abort_capture(fail(FVM_ERR_CUDA, "cudaStreamUpdateCaptureDependencies"));
    if ((st = stage(c, FVM_STAGE_PROJECT, nullptr, nullptr)) != FVM_OK) return abort_capture(st);
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamEndCapture(s, &g));
    save_ptrs(c, G.after);
    load_ptrs(c, G.before);
    c->launches = launches0;
    G.g = g;
    cudaError_t e = cudaGraphInstantiate(&G.exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(FVM_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    return FVM_OK;
}

int find_graph(fvm_case* c) {
    void* now[12];
    save_ptrs(c, now);
    for (size_t g = 0; g < c->graphs.size(); ++g)
        if (!memcmp(now, c->graphs[g].before, sizeof(now))) return (int)g;
    return -1;
}

void drop_graphs(fvm_case* c) {
    for (auto& G : c->graphs) {
        cudaGraphExecDestroy(G.exec);
        cudaGraphDestroy(G.g);
    }
    c->graphs.clear();
}

int field_slot(int fid) {
    // state slots: u v w T k omega; p is separate
    static const int slot[7] = {0, 1, 2, -1, 3, 4, 5};
    return slot[fid];
}

fvm_status build_case(const Plan& pl, fvm_case* c) {
    const fvm_case_desc& d = pl.d;
    c->desc = d;
    c->vents.assign(d.vents, d.vents + d.n_vents);
    c->boxes.assign(d.boxes, d.boxes + d.n_boxes);
    c->desc.vents = c->vents.data();
    c->desc.boxes = c->boxes.data();
    c->prec = pl.prec;
    c->inner = pl.inner;
    c->inner_cycles = d.mg_variant == 1 ? 1 : (d.inner_cycles > 0 ? d.inner_cycles : (pl.inner == FVM_FP64 ? 1 : 2));
    c->dt0 = pl.dt0;
    if (d.stream) c->stream = (cudaStream_t)d.stream;
    else {
        CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    const HostLevel& L0 = pl.levels[0];
    const int64_t N = L0.N();
    const size_t s = elem_size(pl.prec), si = elem_size(pl.inner);
    // case description for the kernels
    CaseDev& cd = c->cd;
    memset(&cd, 0, sizeof(cd));
    for (int a = 0; a < 3; ++a) {
        cd.n[a] = L0.n[a];
        cd.active[a] = L0.active[a];
        cd.h[a] = L0.h[a];
        cd.inv_h[a] = 1.0 / L0.h[a];
        cd.inv_h2[a] = 1.0 / (L0.h[a] * L0.h[a]);
        const double dw = 0.5 * L0.h[a];
        cd.om_wall[a] = 6.0 * d.nu / (kBetaI * dw * dw);
        cd.gb[a] = d.buoyancy ? -d.gravity[a] * d.beta_T : 0.0;
    }
    cd.N = N;
    cd.nu = d.nu;
    cd.alpha = d.nu / d.Pr;
    cd.inv_Prt = 1.0 / d.Prt;
    cd.inv_sigk = 1.0 / d.sigma_k;
    cd.inv_sigw = 1.0 / d.sigma_w;
    cd.T_ref = d.T_ref;
    cd.cfl = d.cfl;
    cd.dt0 = pl.dt0;
    cd.dt_adapt = d.dt_adapt;
    for (int a = 0; a < 3; ++a) {
        cd.f.h[a] = (float)cd.h[a];
        cd.f.inv_h[a] = (float)cd.inv_h[a];
        cd.f.inv_h2[a] = (float)cd.inv_h2[a];
        cd.f.gb[a] = (float)cd.gb[a];
        cd.f.om_wall[a] = (float)cd.om_wall[a];
    }
    cd.f.nu = (float)cd.nu;
    cd.f.alpha = (float)cd.alpha;
    cd.f.inv_Prt = (float)cd.inv_Prt;
    cd.f.inv_sigk = (float)cd.inv_sigk;
    cd.f.inv_sigw = (float)cd.inv_sigw;
    cd.f.T_ref = (float)cd.T_ref;
    const double rcp_alpha = (d.rho > 0.0 && d.cp > 0.0) ? 1.0 / (d.rho * d.cp * cd.alpha) : 0.0;
    cd.n_patches = (int)pl.patches.size();
    for (size_t pi = 0; pi < pl.patches.size(); ++pi) {
        const fvm_patch& p = pl.patches[pi];
        PatchDev& q = cd.patch[pi];
        q.kind = p.kind;
        q.thermal = p.thermal;
        q.T_value = p.T_value;
        q.q_coef = p.T_value * rcp_alpha;
        q.vel[0] = q.vel[1] = q.vel[2] = 0.0;
        q.T_in = p.T_in;
        inlet_kw(p, q.k_in, q.om_in);
        // the face this patch sits on decides the inward normal
        const int face = pi < 6 ? (int)pi : c->vents[pi - 6].face;
        const double inward = (face % 2 == 0) ? 1.0 : -1.0;
        if (p.kind == FVM_INLET) q.vel[face / 2] = inward * p.u_normal;
        for (int a = 0; a < 3; ++a) {
            q.vel2f[a] = (float)(2.0 * q.vel[a]);
            q.qhf[a] = (float)(q.q_coef * cd.h[a]);
        }
        q.T_in2f = (float)(2.0 * q.T_in);
        q.k_in2f = (float)(2.0 * q.k_in);
        q.om_in2f = (float)(2.0 * q.om_in);
        q.T_value2f = (float)(2.0 * q.T_value);
    }
    cd.n_boxes = d.n_boxes;
    for (int bi = 0; bi < d.n_boxes; ++bi) {
        cd.box[bi].thermal = c->boxes[bi].thermal;
        cd.box[bi].T_value = c->boxes[bi].T_value;
        cd.box[bi].q_coef = c->boxes[bi].T_value * rcp_alpha;
        cd.box[bi].T_value2f = (float)(2.0 * cd.box[bi].T_value);
        for (int a = 0; a < 3; ++a) cd.box[bi].qhf[a] = (float)(cd.box[bi].q_coef * cd.h[a]);
    }
    // device memory
    for (int f = 0; f < 6; ++f) {
        ST_TRY(dalloc(c, &c->cur[f], N * s));
        ST_TRY(dalloc(c, &c->nxt[f], N * s));
        if (c->desc.rk_stages == 3) ST_TRY(dalloc(c, &c->rk3[f], N * s));
    }
    ST_TRY(dalloc(c, (void**)&c->p, N * 8));
    ST_TRY(dalloc(c, &c->b, N * s));
    ST_TRY(dalloc(c, (void**)&c->staging, N * 8));
    ST_TRY(dalloc(c, &c->nut, N * s));
    uint8_t* tag_d;
    ST_TRY(dalloc(c, (void**)&tag_d, N));
    CUDA_TRY(cudaMemcpyAsync(tag_d, pl.tag.data(), N, cudaMemcpyHostToDevice, c->stream));
    cd.tag = tag_d;
    for (int f = 0; f < 6; ++f) {
        uint8_t* fp;
        ST_TRY(dalloc(c, (void**)&fp, pl.face_patch[f].size()));
        CUDA_TRY(cudaMemcpyAsync(fp, pl.face_patch[f].data(), pl.face_patch[f].size(), cudaMemcpyHostToDevice,
                                 c->stream));
        cd.face_patch[f] = fp;
    }
    c->levels.resize(pl.levels.size());
    for (size_t l = 0; l < pl.levels.size(); ++l) {
        const HostLevel& H = pl.levels[l];
        DevLevel& D = c->levels[l];
        LevelDev& v = D.dev;
        memset(&v, 0, sizeof(v));
        double diag = 0.0;
        int nact = 0;
        for (int a = 0; a < 3; ++a) {
            v.n[a] = H.n[a];
            v.active[a] = H.active[a];
            v.inv_h2[a] = 1.0 / (H.h[a] * H.h[a]);
            if (H.active[a]) {
                diag += 2.0 * v.inv_h2[a];
                ++nact;
            }
        }
        v.N = H.N();
        v.inv_D = 1.0 / diag;
        v.diag = diag;
        v.wJ = d.mg_variant == 1 ? 1.0   // the paper's scheme: unweighted Jacobi
                                 : (d.jacobi_weight > 0.0 ? d.jacobi_weight : (nact == 3 ? 6.0 / 7.0 : 4.0 / 5.0));
        for (int a = 0; a < 3; ++a) {
            v.inv_h2f[a] = (float)v.inv_h2[a];
            v.ih2a[a] = H.active[a] ? v.inv_h2[a] : 0.0;
            v.ih2af[a] = (float)v.ih2a[a];
            v.ih2alo[a] = (float)(v.ih2a[a] - (double)v.ih2af[a]);
        }
        v.inv_Df = (float)v.inv_D;
        v.wJf = (float)v.wJ;
        v.diagf = (float)v.diag;
        v.zc_fixed = d.sweep_planes;
        if (l == 0) v.solid = tag_d;
        else {
            uint8_t* sd;
            ST_TRY(dalloc(c, (void**)&sd, v.N));
            CUDA_TRY(cudaMemcpyAsync(sd, H.solid.data(), v.N, cudaMemcpyHostToDevice, c->stream));
            v.solid = sd;
        }
        for (int f = 0; f < 6; ++f) {
            uint8_t* dd;
            ST_TRY(dalloc(c, (void**)&dd, H.dir[f].size()));
            CUDA_TRY(cudaMemcpyAsync(dd, H.dir[f].data(), H.dir[f].size(), cudaMemcpyHostToDevice, c->stream));
            v.dir[f] = dd;
        }
        uint16_t* nb;
        ST_TRY(dalloc(c, (void**)&nb, v.N * 2));
        CUDA_TRY(cudaMemcpyAsync(nb, H.nbf.data(), v.N * 2, cudaMemcpyHostToDevice, c->stream));
        v.nbf = nb;
        if (l == 0) {
            cd.nbf0 = nb;
            cd.regular_mask = (H.active[0] ? 0x00fu : 0u) | (H.active[1] ? 0x0f0u : 0u) | (H.active[2] ? 0xf00u : 0u) |
                              (1u << 12);
        }
        ST_TRY(dalloc(c, &D.e[0], v.N * si));
        ST_TRY(dalloc(c, &D.e[1], v.N * si));
        ST_TRY(dalloc(c, &D.r, v.N * si));
    }
    // the coarsest levels whose e, e', r fit in one CTA's shared memory (level 0 never does)
    {
        // per cell: e, e', r in the compute type plus the 2-byte neighbour code.  FP64 runs
        // at a small fraction of the FP32 rate on this part, so one SM only takes the
        // last few hundred cells of an FP64 hierarchy
        const size_t cs = (pl.inner == FVM_FP64 ? 8 : 4) * 3 + 2;
        const size_t budget = pl.inner == FVM_FP64 ? 16 * 1024 : 200 * 1024;
        size_t lc = c->levels.size() - 1;
        size_t used = (size_t)c->levels[lc].dev.N * cs;
        while (lc > 1 && used + (size_t)c->levels[lc - 1].dev.N * cs <= budget) {
            --lc;
            used += (size_t)c->levels[lc].dev.N * cs;
        }
        c->lc = lc;
        memset(&c->coarse, 0, sizeof(c->coarse));
        c->coarse.nl = (int)(c->levels.size() - lc);
        c->coarse.pre = d.coarse_sweeps > 0 ? d.coarse_sweeps : d.pre_sweeps;   // (levels below the finest)
        c->coarse.post = d.coarse_sweeps > 0 ? d.coarse_sweeps : d.post_sweeps;
        for (int q = 0; q < c->coarse.nl; ++q) c->coarse.lv[q] = c->levels[lc + q].dev;
        c->coarse.cheb = d.smoother == 1 ? 1 : 0;
        if (c->coarse.cheb)
            for (int side = 0; side < 2; ++side) {
                const int n = side ? c->coarse.post : c->coarse.pre;
                for (int i = 0; i < n; ++i) {
                    c->coarse.w[side][i] = sweep_weight(c, c->coarse.lv[0], n, i, side == 1);
                    c->coarse.wf[side][i] = (float)c->coarse.w[side][i];
                }
            }
        CUDA_TRY(prepare_coarse_cta(pl.inner, coarse_cta_smem(c->coarse, pl.inner)));
    }
    // the paper's scheme applies the fine grid's stencil and diagonal on every level
    if (d.mg_variant == 1)
        for (size_t l = 1; l < c->levels.size(); ++l) {
            LevelDev& v = c->levels[l].dev;
            const LevelDev& f0 = c->levels[0].dev;
            for (int a = 0; a < 3; ++a) {
                v.inv_h2[a] = f0.inv_h2[a];
                v.inv_h2f[a] = f0.inv_h2f[a];
                v.ih2a[a] = v.active[a] ? f0.inv_h2[a] : 0.0;
                v.ih2af[a] = (float)v.ih2a[a];
                v.ih2alo[a] = (float)(v.ih2a[a] - (double)v.ih2af[a]);
            }
            v.diag = f0.diag;
            v.diagf = f0.diagf;
            v.inv_D = f0.inv_D;
            v.inv_Df = f0.inv_Df;
        }
    std::vector<double> inv;
    if (!coarse_inverse(pl.levels.back(), inv))
        return fail(FVM_ERR_INVALID, "coarsest-level operator is singular (does an outlet reach every fluid region?)");
    // the coarsest inverse in FP64, followed by its FP32 copy (read by the coarse kernel in
    // the reduced-precision modes)
    std::vector<float> invf(inv.begin(), inv.end());
    ST_TRY(dalloc(c, (void**)&c->Ainv, inv.size() * 12));
    if (d.mg_variant == 1) ST_TRY(dalloc(c, (void**)&c->p_tmp, (size_t)N * 8));
    CUDA_TRY(cudaMemcpyAsync(c->Ainv, inv.data(), inv.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->Ainv + inv.size(), invf.data(), inv.size() * 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->nblocks0 = level0_blocks_max(L0.n[0], L0.n[1], L0.n[2]);
    ST_TRY(dalloc(c, (void**)&c->partials, (size_t)(2 * c->nblocks0) * 8));
    if (d.krylov == 1) {
        const size_t si0 = elem_size(pl.inner == FVM_BF16_MIXED ? FVM_FP32 : pl.inner);
        ST_TRY(dalloc(c, &c->kdir, (size_t)N * si0));
        if (pl.inner == FVM_BF16_MIXED) ST_TRY(dalloc(c, (void**)&c->kz, (size_t)N * 4));
        ST_TRY(dalloc(c, (void**)&c->kpart, (size_t)4 * level0_blocks_max(L0.n[0], L0.n[1], L0.n[2]) * 8));
    }
    ST_TRY(dalloc(c, (void**)&c->norms, 4 * 8));
    ST_TRY(dalloc(c, (void**)&c->dt_state, 6 * 8));
    ST_TRY(dalloc(c, (void**)&c->sst, sizeof(SolveState)));
    CUDA_TRY(cudaMallocHost((void**)&c->h_norms, 8 * sizeof(double) + sizeof(SolveState)));
    c->h_dt = c->h_norms + 4;
    c->h_sst = (SolveState*)(c->h_norms + 8);
    double dts[6] = {pl.dt0, 0.5 * pl.dt0, 0.0, 0.0, 0.0, 0.0};
    ((float*)(dts + 4))[0] = (float)pl.dt0;
    ((float*)(dts + 4))[1] = (float)(0.5 * pl.dt0);
    CUDA_TRY(cudaMemcpyAsync(c->dt_state, dts, sizeof(dts), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemsetAsync(c->p, 0, N * 8, c->stream));
    CUDA_TRY(cudaMemsetAsync(c->b, 0, N * s, c->stream));
    CUDA_TRY(cudaMemsetAsync(c->norms, 0, 4 * 8, c->stream));
    CUDA_TRY(launch_init_state(c->prec, cd, ptrs(c->cur), pl.base, d.seed, d.init_perturb, c->stream));
    ST_TRY(set_rule(c, d.fixed_vcycles));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return FVM_OK;
}


// ------------------------------------------------------------------ batches
// Several cases stepped together: each step kernel and multigrid kernel runs
// once per launch site for all cases (k_many over a table of per-case
// functors), inside one CUDA graph per pointer parity.  The sequence of
// launches is obtained by replaying each case's own step with a Recorder
// installed, so a batched step issues exactly the kernels the cases would
// issue alone, merged site by site.

struct BatchGather {
    int32_t cycles, total_cycles, nonfinite, notconv, inner, active;
    double rel, dt, sim_time;
};

// Copy each case's solve state and time step into one array, and add this
// step's outer V-cycle iterations (the maximum over the cases) to a counter.
__global__ void k_batch_gather(SolveState* const* sts, double* const* dts, BatchGather* out, int n,
                               unsigned long long* outer_sum) {
    int mx = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const SolveState* s = sts[i];
        BatchGather g;
        g.cycles = s->cycles;
        g.total_cycles = s->total_cycles;
        g.nonfinite = s->nonfinite;
        g.notconv = s->notconv;
        g.inner = s->inner;
        g.active = s->active;
        g.rel = s->rel;
        g.dt = dts[i][0];
        g.sim_time = dts[i][2];
        out[i] = g;
        const int outer = s->cycles / (s->inner > 0 ? s->inner : 1);
        mx = outer > mx ? outer : mx;
    }
    for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    __shared__ int wm[32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = max(mx, wm[w]);
        mx = max(mx, wm[0]);
        *outer_sum += (unsigned long long)mx;
    }
}

// One launch of the batched step: a functor type, the cases that take part
// and their recorded functors.
struct Merged {
    ManyFn many;
    std::string site;
    dim3 block;
    size_t smem = 0;
    std::vector<int> cases;
    std::vector<const RecLaunch*> recs;   // valid while the tables are built
    double bytes = 0.0;                   // algorithmic bytes of the launch (all its cases)
    // device table (filled when the arena is built)
    const void* tab = nullptr;
    BatchMap map{};
    unsigned nblk = 0;
    BatchCtl ctl{};
};

// Merge the cases' launch sequences site by site, keeping each case's order.
// A launch is identified by (site, functor type, occurrence of that pair in
// the case's sequence); a key is issued for all cases at once unless a case
// still has it further ahead, in which case another key goes first.
std::vector<Merged> merge_sequences(const std::vector<std::vector<RecLaunch>>& seqs) {
    struct Key {
        std::string site;
        ManyFn many;
        int occ;
        bool operator==(const Key& o) const { return many == o.many && occ == o.occ && site == o.site; }
    };
    const int n = (int)seqs.size();
    std::vector<std::vector<Key>> keys(n);
    for (int i = 0; i < n; ++i) {
        std::vector<std::pair<std::string, ManyFn>> seen;
        std::vector<int> count;
        for (const RecLaunch& r : seqs[i]) {
            int occ = 0;
            size_t q = 0;
            for (; q < seen.size(); ++q)
                if (seen[q].first == r.site && seen[q].second == r.many) break;
            if (q == seen.size()) {
                seen.push_back({r.site, r.many});
                count.push_back(0);
            }
            occ = count[q]++;
            keys[i].push_back(Key{r.site, r.many, occ});
        }
    }
    auto pending_later = [&](int j, size_t from, const Key& k) {
        for (size_t q = from + 1; q < keys[j].size(); ++q)
            if (keys[j][q] == k) return true;
        return false;
    };
    std::vector<size_t> cur(n, 0);
    std::vector<Merged> out;
    for (;;) {
        int pick = -1, first = -1;
        for (int i = 0; i < n && pick < 0; ++i) {
            if (cur[i] >= keys[i].size()) continue;
            if (first < 0) first = i;
            const Key& k = keys[i][cur[i]];
            bool ok = true;
            for (int j = 0; j < n && ok; ++j)
                if (cur[j] < keys[j].size() && !(keys[j][cur[j]] == k) && pending_later(j, cur[j], k)) ok = false;
            if (ok) pick = i;
        }
        if (first < 0) break;
        if (pick < 0) pick = first;
        const Key k = keys[pick][cur[pick]];
        Merged m;
        m.many = k.many;
        m.site = k.site;
        m.block = seqs[pick][cur[pick]].block;
        for (int j = 0; j < n; ++j) {
            if (cur[j] >= keys[j].size() || !(keys[j][cur[j]] == k)) continue;
            const RecLaunch& r = seqs[j][cur[j]];
            m.cases.push_back(j);
            m.recs.push_back(&r);
            m.bytes += r.bytes;
            m.smem = std::max(m.smem, r.smem);
            ++cur[j];
        }
        out.push_back(std::move(m));
    }
    return out;
}

}  // namespace

struct fvm_batch {
    std::vector<fvm_case*> cases;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t side = nullptr;
    struct Graph {
        std::vector<void*> before, after;   // 12 state pointers per case
        cudaGraph_t g = nullptr;
        cudaGraphExec_t exec = nullptr;
        void* arena = nullptr;              // functor tables, block maps, state lists
        int64_t per_step = 0;               // launches outside the V-cycle loop
        int64_t per_outer = 0;              // launches per outer iteration (V-cycle body)
        std::vector<Merged> seg[4];         // step, residual, V-cycle, projection (tables in the arena)
    };
    std::vector<Graph> graphs;
    SolveState** d_sts = nullptr;
    double** d_dts = nullptr;
    BatchGather* d_gather = nullptr;
    BatchGather* h_gather = nullptr;
    unsigned long long* d_outer = nullptr;
    unsigned long long* h_outer = nullptr;
    unsigned long long* d_scratch = nullptr;   // outer-iteration sum of profiled steps (unused)
    int64_t launches = 0;
    int64_t steps = 0;
    // a launch in flight (fvm_batch_launch): its step count and launch tallies
    bool pending = false;
    int32_t pend_steps = 0;
    int64_t pend_fixed = 0, pend_per_outer = 0;
};

namespace {

void free_batch(fvm_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto& G : b->graphs) {
        if (G.exec) cudaGraphExecDestroy(G.exec);
        if (G.g) cudaGraphDestroy(G.g);
        if (G.arena) cudaFree(G.arena);
    }
    if (b->d_sts) cudaFree(b->d_sts);
    if (b->d_dts) cudaFree(b->d_dts);
    if (b->d_gather) cudaFree(b->d_gather);
    if (b->d_outer) cudaFree(b->d_outer);
    if (b->d_scratch) cudaFree(b->d_scratch);
    if (b->h_gather) cudaFreeHost(b->h_gather);
    if (b->h_outer) cudaFreeHost(b->h_outer);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// Lay the merged launches' tables into one device buffer: per launch the
// functor table, the block offsets, the per-case grids, and (resid0) the
// block counter and the list of its cases' solve states.
fvm_status build_arena(std::vector<Merged>* segs, int nseg, const std::vector<fvm_case*>& cases, void** arena_out) {
    auto up = [](size_t x, size_t a) { return (x + a - 1) / a * a; };
    size_t bytes = 0;
    for (int s = 0; s < nseg; ++s)
        for (Merged& m : segs[s]) {
            const size_t n = m.cases.size();
            bytes = up(bytes, 256) + n * m.recs[0]->arg.size();
            bytes = up(bytes, 16) + (n + 1) * sizeof(int);
            bytes = up(bytes, 16) + n * sizeof(uint3);
            bytes = up(bytes, 16) + n * sizeof(SolveState*);
            bytes = up(bytes, 16) + 16;
        }
    bytes = up(bytes, 256);
    std::vector<unsigned char> host(bytes, 0);
    void* dev = nullptr;
    cudaError_t e = cudaMalloc(&dev, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(FVM_ERR_OOM, std::string("batch tables: ") + cudaGetErrorString(e));
    }
    unsigned char* d = (unsigned char*)dev;
    size_t off = 0;
    for (int s = 0; s < nseg; ++s)
        for (Merged& m : segs[s]) {
            const size_t n = m.cases.size();
            const size_t ksz = m.recs[0]->arg.size();
            off = up(off, 256);
            m.tab = d + off;
            for (size_t i = 0; i < n; ++i) memcpy(&host[off + i * ksz], m.recs[i]->arg.data(), ksz);
            off += n * ksz;
            off = up(off, 16);
            int* start = (int*)&host[off];
            m.map.start = (const int*)(d + off);
            int64_t tot = 0;
            for (size_t i = 0; i < n; ++i) {
                start[i] = (int)tot;
                const dim3 g = m.recs[i]->grid;
                const int64_t nb = (int64_t)g.x * g.y * g.z;
                if (nb < 1) {   // every case of a launch owns at least one block (the device walk relies on it)
                    cudaFree(dev);
                    return fail(FVM_ERR_INVALID, "batched launch " + m.site + ": a case with an empty grid");
                }
                tot += nb;
            }
            start[n] = (int)tot;
            off += (n + 1) * sizeof(int);
            off = up(off, 16);
            uint3* grid = (uint3*)&host[off];
            m.map.grid = (const uint3*)(d + off);
            for (size_t i = 0; i < n; ++i)
                grid[i] = make_uint3(m.recs[i]->grid.x, m.recs[i]->grid.y, m.recs[i]->grid.z);
            off += n * sizeof(uint3);
            off = up(off, 16);
            SolveState** lst = (SolveState**)&host[off];
            m.ctl.st = (SolveState* const*)(d + off);
            for (size_t i = 0; i < n; ++i) lst[i] = cases[m.cases[i]]->sst;
            off += n * sizeof(SolveState*);
            off = up(off, 16);
            m.ctl.counter = (unsigned*)(d + off);   // zero
            off += 16;
            m.map.n = (int)n;
            m.ctl.n = (int)n;
            if (tot >= ((int64_t)1 << 31)) {
                cudaFree(dev);
                return fail(FVM_ERR_INVALID, "batch too large for one launch");
            }
            m.nblk = (unsigned)tot;
            m.map.total = (int)tot;
        }
    e = cudaMemcpy(dev, host.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dev);
        return fail(FVM_ERR_CUDA, std::string("batch tables upload: ") + cudaGetErrorString(e));
    }
    *arena_out = dev;
    return FVM_OK;
}

fvm_status issue(std::vector<Merged>& seg, cudaStream_t s) {
    for (Merged& m : seg) {
        cudaError_t e = m.many(m.tab, m.map, m.nblk, m.block, m.smem, &m.ctl, s);
        if (e != cudaSuccess) return fail(FVM_ERR_CUDA, "batched launch " + m.site + ": " + cudaGetErrorString(e));
    }
    return FVM_OK;
}

// Record every case's step (four segments: step kernels up to the solve,
// the level-0 residual, one V-cycle, the projection), merge, build the
// tables and capture the graph.
fvm_status batch_capture(fvm_batch* B, fvm_batch::Graph& G) {
    const int n = (int)B->cases.size();
    std::vector<std::vector<RecLaunch>> rec[4];
    for (int s = 0; s < 4; ++s) rec[s].resize(n);
    G.before.assign(12 * (size_t)n, nullptr);
    G.after.assign(12 * (size_t)n, nullptr);
    fvm_status st = FVM_OK;
    for (int i = 0; i < n && st == FVM_OK; ++i) {
        fvm_case* c = B->cases[i];
        save_ptrs(c, &G.before[12 * (size_t)i]);
        const int64_t launches0 = c->launches;
        Recorder R;
        g_rec = &R;
        for (int k : kStepStages)
            if (st == FVM_OK) st = stage(c, k, nullptr, nullptr);
        if (st == FVM_OK) {
            R.site = "solve_begin";
            if (launch_solve_begin(c->sst, c->stream) != cudaSuccess) st = fail(FVM_ERR_CUDA, "solve_begin");
        }
        rec[0][i].swap(R.out);
        if (st == FVM_OK) st = residual0(c, 0, 0, 0);
        rec[1][i].swap(R.out);
        int idx = 0;
        if (st == FVM_OK) st = cycle(c, 0, idx);
        rec[2][i].swap(R.out);
        if (st == FVM_OK) st = stage(c, FVM_STAGE_PROJECT, nullptr, nullptr);
        rec[3][i].swap(R.out);
        g_rec = nullptr;
        save_ptrs(c, &G.after[12 * (size_t)i]);
        load_ptrs(c, &G.before[12 * (size_t)i]);
        c->launches = launches0;
    }
    g_rec = nullptr;
    if (st != FVM_OK) return st;
    std::vector<Merged>* seg = G.seg;
    for (int s = 0; s < 4; ++s) seg[s] = merge_sequences(rec[s]);
    if (seg[1].size() != 1)
        return fail(FVM_ERR_INVALID, "batched cases need the same precisions (one level-0 residual launch)");
    ST_TRY(build_arena(seg, 4, B->cases, &G.arena));
    for (int s = 0; s < 4; ++s)
        for (Merged& m : seg[s]) m.recs.clear();   // the recorded functors now live in the arena
    // dynamic shared-memory limits of the batched kernels (outside the capture)
    for (int s = 0; s < 4; ++s)
        for (Merged& m : seg[s]) CUDA_TRY(m.many(m.tab, m.map, 0, m.block, m.smem, &m.ctl, B->stream));
    G.per_step = (int64_t)(seg[0].size() + seg[3].size()) + 1 /* gather */ + 1 /* last residual */;
    G.per_outer = 1 + (int64_t)seg[2].size();
    cudaStream_t s = B->stream;
    if (!B->side) CUDA_TRY(cudaStreamCreateWithFlags(&B->side, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    auto abort_capture = [&](fvm_status e) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return e;
    };
    if ((st = issue(seg[0], s)) != FVM_OK) return abort_capture(st);
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &graph, &deps, nullptr, &ndeps) != cudaSuccess)
        return abort_capture(fail(FVM_ERR_CUDA, "cudaStreamGetCaptureInfo"));
    cudaGraphConditionalHandle hw, hi;
    if (cudaGraphConditionalHandleCreate(&hw, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess)
        return abort_capture(fail(FVM_ERR_CUDA, "cudaGraphConditionalHandleCreate"));
    cudaGraphNodeParams wp = {cudaGraphNodeTypeConditional};
    wp.conditional.handle = hw;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if (cudaGraphAddNode(&wnode, graph, deps, nullptr, ndeps, &wp) != cudaSuccess)
        return abort_capture(fail(FVM_ERR_CUDA, "adding the while node"));
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    if (cudaGraphConditionalHandleCreate(&hi, body, 0, cudaGraphCondAssignDefault) != cudaSuccess)
        return abort_capture(fail(FVM_ERR_CUDA, "cudaGraphConditionalHandleCreate (if)"));
    if (cudaStreamBeginCaptureToGraph(B->side, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
        return abort_capture(fail(FVM_ERR_CUDA, "capturing the while body"));
    Merged& r0 = seg[1][0];
    r0.ctl.cond = hw;
    r0.ctl.cond2 = hi;
    r0.ctl.use_cond = 2;
    st = issue(seg[1], B->side);
    cudaStreamCaptureStatus bcs;
    cudaGraph_t bg = nullptr;
    const cudaGraphNode_t* bdeps = nullptr;
    size_t nbdeps = 0;
    cudaGraphNode_t inode;
    cudaGraphNodeParams ip = {cudaGraphNodeTypeConditional};
    bool ok = st == FVM_OK &&
              cudaStreamGetCaptureInfo(B->side, &bcs, nullptr, &bg, &bdeps, nullptr, &nbdeps) == cudaSuccess;
    if (ok) {
        ip.conditional.handle = hi;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        ok = cudaGraphAddNode(&inode, bg, bdeps, nullptr, nbdeps, &ip) == cudaSuccess;
    }
    cudaGraph_t done_body = nullptr;
    cudaStreamEndCapture(B->side, &done_body);
    if (!ok) return abort_capture(st != FVM_OK ? st : fail(FVM_ERR_CUDA, "adding the if node"));
    cudaGraph_t ibody = ip.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(B->side, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
        return abort_capture(fail(FVM_ERR_CUDA, "capturing the V-cycle body"));
    st = issue(seg[2], B->side);
    cudaGraph_t done_if = nullptr;
    cudaStreamEndCapture(B->side, &done_if);
    if (st != FVM_OK) return abort_capture(st);
    if (cudaStreamUpdateCaptureDependencies(s, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
        return abort_capture(fail(FVM_ERR_CUDA, "cudaStreamUpdateCaptureDependencies"));
    if ((st = issue(seg[3], s)) != FVM_OK) return abort_capture(st);
    k_batch_gather<<<1, 256, 0, s>>>(B->d_sts, B->d_dts, B->d_gather, n, B->d_outer);
    if (cudaGetLastError() != cudaSuccess) return abort_capture(fail(FVM_ERR_CUDA, "gather launch"));
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamEndCapture(s, &g));
    G.g = g;
    cudaError_t e = cudaGraphInstantiate(&G.exec, g, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(FVM_ERR_CUDA, std::string("cudaGraphInstantiate (batch): ") + cudaGetErrorString(e));
    }
    return FVM_OK;
}

int find_batch_graph(fvm_batch* B);

// the graph (and launch tables) for the cases' current pointers, captured if new
fvm_status batch_graph(fvm_batch* B, int& g) {
    g = find_batch_graph(B);
    if (g >= 0) return FVM_OK;
    fvm_batch::Graph G;
    fvm_status st = batch_capture(B, G);
    if (st != FVM_OK) {
        if (G.exec) cudaGraphExecDestroy(G.exec);
        if (G.g) cudaGraphDestroy(G.g);
        if (G.arena) cudaFree(G.arena);
        return st;
    }
    B->graphs.push_back(std::move(G));
    g = (int)B->graphs.size() - 1;
    return FVM_OK;
}

int find_batch_graph(fvm_batch* B) {
    const size_t n = B->cases.size();
    std::vector<void*> now(12 * n);
    for (size_t i = 0; i < n; ++i) save_ptrs(B->cases[i], &now[12 * i]);
    for (size_t g = 0; g < B->graphs.size(); ++g)
        if (B->graphs[g].before == now) return (int)g;
    return -1;
}

// Can these cases be stepped as one batch?
fvm_status batch_check(fvm_case* const* cases, int n) {
    if (!cases || n < 1) return fail(FVM_ERR_INVALID, "need at least one case");
    for (int i = 0; i < n; ++i) {
        const fvm_case* c = cases[i];
        if (!c) return fail(FVM_ERR_INVALID, "null case in the batch");
        for (int j = 0; j < i; ++j)
            if (cases[j] == c) return fail(FVM_ERR_INVALID, "a case appears twice in the batch");
        if (c->prec != cases[0]->prec || c->inner != cases[0]->inner)
            return fail(FVM_ERR_INVALID, "batched cases need the same precision");
        if (c->prof) return fail(FVM_ERR_INVALID, "profiling is on for a batched case");
    }
    return FVM_OK;
}

}  // namespace

// ====================================================================== C-ABI
extern "C" {

size_t fvm_case_bytes(const fvm_case_desc* desc) {
    Plan pl;
    if (plan_case(desc, pl) != FVM_OK) return 0;
    return (size_t)pl.bytes;
}

fvm_status fvm_create_case(const fvm_case_desc* desc, fvm_case** out) {
    if (!out) return fail(FVM_ERR_INVALID, "null output pointer");
    Plan pl;
    ST_TRY(plan_case(desc, pl));
    fvm_case* c = new fvm_case();
    fvm_status st = build_case(pl, c);
    if (st != FVM_OK) {
        std::string msg = g_err;
        free_case(c);
        g_err = msg;
        return st;
    }
    g_err.clear();
    *out = c;
    return FVM_OK;
}

void fvm_destroy_case(fvm_case* c) { free_case(c); }

fvm_status fvm_run_stage(fvm_case* c, int st) {
    if (!c) return fail(FVM_ERR_INVALID, "null case");
    ST_TRY(stage(c, st, nullptr, nullptr));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return FVM_OK;
}

fvm_status fvm_step(fvm_case* c, int nsteps, fvm_step_stats* out) {
    if (!c) return fail(FVM_ERR_INVALID, "null case");
    if (nsteps < 0) return fail(FVM_ERR_INVALID, "nsteps < 0");
    fvm_step_stats stats;
    memset(&stats, 0, sizeof(stats));
    fvm_status result = FVM_OK;
    // clear the per-call counters of the solve state
    CUDA_TRY(cudaMemsetAsync(&c->sst->total_cycles, 0, sizeof(int32_t), c->stream));
    CUDA_TRY(cudaMemsetAsync(&c->sst->nonfinite, 0, sizeof(int32_t), c->stream));
    CUDA_TRY(cudaMemsetAsync(&c->sst->notconv, 0, sizeof(int32_t), c->stream));
    const bool graph = c->use_graph && !c->prof;
    int graph_steps = 0;
    for (int n = 0; n < nsteps; ++n) {
        if (graph) {
            int g = find_graph(c);
            if (g < 0) {
                fvm_case::StepGraph G;
                ST_TRY(capture_step(c, G));
                c->graphs.push_back(G);
                g = (int)c->graphs.size() - 1;
            }
            CUDA_TRY(cudaGraphLaunch(c->graphs[g].exec, c->stream));
            load_ptrs(c, c->graphs[g].after);
            ++c->steps;
            ++graph_steps;
            stats.steps++;
            continue;
        }
        int cycles = 0;
        double rel = 0.0;
        for (int k : kStepStages) ST_TRY(stage(c, k, nullptr, nullptr));
        ST_TRY(stage(c, FVM_STAGE_SOLVE, &cycles, &rel));
        ST_TRY(stage(c, FVM_STAGE_PROJECT, nullptr, nullptr));
        ++c->steps;
        stats.steps++;
        if (!std::isfinite(rel)) break;
    }
    ST_TRY(read_state(c));
    CUDA_TRY(cudaMemcpyAsync(c->h_dt, c->dt_state, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    stats.vcycles_total = c->h_sst->total_cycles;
    // kernels run by the graphs: 7 step kernels per step (one more per later Runge-Kutta stage),
    // one residual per outer iteration plus the last one of each step, and kpc kernels per outer
    // iteration (inner V-cycles of the if node)
    if (graph_steps) {
        const int64_t outer = (int64_t)stats.vcycles_total / std::max(1, c->rule_inner);
        const int64_t step_kernels = 7 + (c->desc.rk_stages > 1 ? c->desc.rk_stages - 1 : 0);
        c->launches += step_kernels * (int64_t)graph_steps + (int64_t)graph_steps + outer * (1 + c->kpc);
    }
    stats.vcycles_last = c->h_sst->cycles;
    stats.rel_residual = c->h_sst->rel;
    stats.dt_last = c->h_dt[0];
    stats.sim_time = c->h_dt[2];
    if (c->h_sst->nonfinite) result = fail(FVM_ERR_DIVERGED, "non-finite pressure residual");
    else if (c->h_sst->notconv) {
        result = FVM_ERR_NOT_CONVERGED;
        g_err = "V-cycle cap reached above the tolerance";
    }
    if (out) *out = stats;
    return result;
}

fvm_status fvm_vcycle(fvm_case* c, int ncycles, double* rel_residual) {
    if (!c) return fail(FVM_ERR_INVALID, "null case");
    if (ncycles < 0) return fail(FVM_ERR_INVALID, "ncycles < 0");
    int cycles = 0;
    double rel = 0.0;
    fvm_status st = FVM_OK;
    if (ncycles > 0) {
        ST_TRY(set_rule(c, ncycles));
        st = solve(c, cycles, rel);
    } else {
        // residual only: whatever the rule decides, no cycle is launched (the rule is reset
        // first: the residual kernel skips a solve that is no longer active)
        ST_TRY(set_rule(c, c->desc.fixed_vcycles));
        ST_TRY(residual0(c, 0, 0, 0));
        ST_TRY(read_state(c));
        rel = c->h_sst->rel;
    }
    fvm_status st2 = set_rule(c, c->desc.fixed_vcycles);
    if (st != FVM_OK) return st;
    if (st2 != FVM_OK) return st2;
    if (rel_residual) *rel_residual = rel;
    return FVM_OK;
}

fvm_status fvm_read_fields(fvm_case* c, unsigned mask, double* host_out, size_t n) {
    if (!c || (!host_out && mask)) return fail(FVM_ERR_INVALID, "null case or buffer");
    if (mask >= (1u << 7)) return fail(FVM_ERR_INVALID, "field mask has bits above 6");
    const int64_t N = c->cd.N;
    size_t need = 0;
    for (int f = 0; f < 7; ++f)
        if (mask & (1u << f)) need += (size_t)N;
    if (n < need) return fail(FVM_ERR_INVALID, "host buffer too small");
    size_t off = 0;
    for (int f = 0; f < 7; ++f) {
        if (!(mask & (1u << f))) continue;
        if (f == FVM_P && c->prec == FVM_FP64) {
            CUDA_TRY(cudaMemcpyAsync(host_out + off, c->p, N * 8, cudaMemcpyDeviceToHost, c->stream));
        } else if (f == FVM_P) {   // double-float pairs to FP64
            CUDA_TRY(launch_p_to_double(c->p, c->staging, N, c->stream));
            CUDA_TRY(cudaMemcpyAsync(host_out + off, c->staging, N * 8, cudaMemcpyDeviceToHost, c->stream));
        } else {
            // (stream order: the next field's pack waits for this copy out of the staging buffer)
            CUDA_TRY(launch_pack(c->prec, c->cur[field_slot(f)], c->staging, N, c->stream));
            CUDA_TRY(cudaMemcpyAsync(host_out + off, c->staging, N * 8, cudaMemcpyDeviceToHost, c->stream));
        }
        off += (size_t)N;
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return FVM_OK;
}

fvm_status fvm_write_fields(fvm_case* c, unsigned mask, const double* host_in, size_t n) {
    if (!c || (!host_in && mask)) return fail(FVM_ERR_INVALID, "null case or buffer");
    if (mask >= (1u << 7)) return fail(FVM_ERR_INVALID, "field mask has bits above 6");
    const int64_t N = c->cd.N;
    size_t need = 0;
    for (int f = 0; f < 7; ++f)
        if (mask & (1u << f)) need += (size_t)N;
    if (n < need) return fail(FVM_ERR_INVALID, "host buffer too small");
    size_t off = 0;
    for (int f = 0; f < 7; ++f) {
        if (!(mask & (1u << f))) continue;
        if (f == FVM_P && c->prec == FVM_FP64) {
            CUDA_TRY(cudaMemcpyAsync(c->p, host_in + off, N * 8, cudaMemcpyHostToDevice, c->stream));
        } else if (f == FVM_P) {   // FP64 to double-float pairs
            CUDA_TRY(cudaMemcpyAsync(c->staging, host_in + off, N * 8, cudaMemcpyHostToDevice, c->stream));
            CUDA_TRY(launch_p_from_double(c->staging, c->p, N, c->stream));
        } else {
            // (stream order: the next field's copy into the staging buffer waits for this unpack)
            CUDA_TRY(cudaMemcpyAsync(c->staging, host_in + off, N * 8, cudaMemcpyHostToDevice, c->stream));
            CUDA_TRY(launch_unpack(c->prec, c->staging, c->cur[field_slot(f)], N, c->stream));
            c->nut_valid = false;
        }
        off += (size_t)N;
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return FVM_OK;
}

// FP32 host values: a reduced-precision case's state fields move as stored (one copy each, no
// staging), p through the staging buffer as FP32; an FP64 case's fields through the staging
// buffer, converted there.
fvm_status fvm_read_fields_f32(fvm_case* c, unsigned mask, float* host_out, size_t n) {
    if (!c || (!host_out && mask)) return fail(FVM_ERR_INVALID, "null case or buffer");
    if (mask >= (1u << 7)) return fail(FVM_ERR_INVALID, "field mask has bits above 6");
    const int64_t N = c->cd.N;
    size_t need = 0;
    for (int f = 0; f < 7; ++f)
        if (mask & (1u << f)) need += (size_t)N;
    if (n < need) return fail(FVM_ERR_INVALID, "host buffer too small");
    float* const stage = (float*)c->staging;
    size_t off = 0;
    for (int f = 0; f < 7; ++f) {
        if (!(mask & (1u << f))) continue;
        const void* src = nullptr;
        if (f == FVM_P) {
            if (c->prec == FVM_FP64) CUDA_TRY(launch_convert(FVM_FP64, FVM_FP32, c->p, stage, N, c->stream));
            else CUDA_TRY(launch_p_to_float(c->p, stage, N, c->stream));
            src = stage;
        } else if (c->prec == FVM_FP64) {
            CUDA_TRY(launch_convert(FVM_FP64, FVM_FP32, c->cur[field_slot(f)], stage, N, c->stream));
            src = stage;
        } else {
            src = c->cur[field_slot(f)];
        }
        // (stream order: a later conversion into the staging buffer waits for this copy)
        CUDA_TRY(cudaMemcpyAsync(host_out + off, src, N * 4, cudaMemcpyDeviceToHost, c->stream));
        off += (size_t)N;
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return FVM_OK;
}

fvm_status fvm_write_fields_f32(fvm_case* c, unsigned mask, const float* host_in, size_t n) {
    if (!c || (!host_in && mask)) return fail(FVM_ERR_INVALID, "null case or buffer");
    if (mask >= (1u << 7)) return fail(FVM_ERR_INVALID, "field mask has bits above 6");
    const int64_t N = c->cd.N;
    size_t need = 0;
    for (int f = 0; f < 7; ++f)
        if (mask & (1u << f)) need += (size_t)N;
    if (n < need) return fail(FVM_ERR_INVALID, "host buffer too small");
    float* const stage = (float*)c->staging;
    size_t off = 0;
    for (int f = 0; f < 7; ++f) {
        if (!(mask & (1u << f))) continue;
        if (f != FVM_P && c->prec != FVM_FP64) {
            CUDA_TRY(cudaMemcpyAsync(c->cur[field_slot(f)], host_in + off, N * 4, cudaMemcpyHostToDevice, c->stream));
        } else {
            // (stream order: the next copy into the staging buffer waits for this conversion)
            CUDA_TRY(cudaMemcpyAsync(stage, host_in + off, N * 4, cudaMemcpyHostToDevice, c->stream));
            if (f == FVM_P && c->prec != FVM_FP64) CUDA_TRY(launch_p_from_float(stage, c->p, N, c->stream));
            else CUDA_TRY(launch_convert(FVM_FP32, FVM_FP64, stage, f == FVM_P ? (void*)c->p : c->cur[field_slot(f)], N,
                                         c->stream));
        }
        if (f != FVM_P) c->nut_valid = false;
        off += (size_t)N;
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return FVM_OK;
}

fvm_status fvm_set_poisson_rhs(fvm_case* c, const double* host_b, size_t n) {
    if (!c || !host_b) return fail(FVM_ERR_INVALID, "null case or buffer");
    const int64_t N = c->cd.N;
    if (n < (size_t)N) return fail(FVM_ERR_INVALID, "host buffer too small");
    CUDA_TRY(cudaMemcpyAsync(c->staging, host_b, N * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(launch_unpack(c->prec, c->staging, c->b, N, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return FVM_OK;
}

fvm_status fvm_read_poisson_rhs(fvm_case* c, double* host_b, size_t n) {
    if (!c || !host_b) return fail(FVM_ERR_INVALID, "null case or buffer");
    const int64_t N = c->cd.N;
    if (n < (size_t)N) return fail(FVM_ERR_INVALID, "host buffer too small");
    CUDA_TRY(launch_pack(c->prec, c->b, c->staging, N, c->stream));
    CUDA_TRY(cudaMemcpyAsync(host_b, c->staging, N * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return FVM_OK;
}

fvm_status fvm_lambda2(fvm_case* c, double* host_out, size_t n) {
    if (!c || !host_out) return fail(FVM_ERR_INVALID, "null case or buffer");
    const int64_t N = c->cd.N;
    if (n < (size_t)N) return fail(FVM_ERR_INVALID, "host buffer too small");
    const double sz = (double)elem_size(c->prec);
    // algorithmic bytes: u, v, w, the cell tag, the FP64 result
    KLAUNCH("lambda2", (double)N * (3 * sz + 1 + 8), 1,
            launch_lambda2(c->prec, c->cd, ptrs(c->cur), c->staging, c->stream));
    CUDA_TRY(cudaMemcpyAsync(host_out, c->staging, N * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return FVM_OK;
}

namespace {

// The projection's vector-Jacobian product on device buffers: ybar (u, v, w, p: 4 N) -> xbar
// (u, v, w: 3 N).  A lambda = q by the case's own V-cycles from zero (A is symmetric on the fluid
// cells); the case's p and b are saved into save (2 N) and put back, whatever happens.
fvm_status projection_vjp_dev(fvm_case* c, double dt, const double* ybar, double* xbar, double rel_tol,
                              int32_t max_vcycles, double* save, double* rel_out) {
    const int64_t N = c->cd.N;
    cudaStream_t s = c->stream;
    double* p_save = save;
    double* b_save = save + N;
    double* b = (double*)c->b;
    double rel = 0.0;
    bool saved = false;
    auto run = [&]() -> fvm_status {
        CUDA_TRY(cudaMemcpyAsync(p_save, c->p, N * 8, cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(b_save, b, N * 8, cudaMemcpyDeviceToDevice, s));
        saved = true;
        KLAUNCH("adj_grad", (double)N * (5 * 8 + 2 + 1), 1, launch_adj_grad(c->cd, c->levels[0].dev, ybar, b, dt, s));
        CUDA_TRY(cudaMemsetAsync(c->p, 0, N * 8, s));
        int done = 0;
        const int chunk = 4;
        for (;;) {
            ST_TRY(fvm_vcycle(c, chunk, &rel));
            done += chunk;
            if (!std::isfinite(rel)) return fail(FVM_ERR_DIVERGED, "non-finite residual in the adjoint solve");
            if (rel <= rel_tol || done >= max_vcycles) break;
        }
        KLAUNCH("adj_rhs", (double)N * (3 * 8 + 8 + 3 * 8 + 2 + 1), 1,
                launch_adj_rhs(c->cd, c->levels[0].dev, ybar, c->p, xbar, dt, s));
        return rel <= rel_tol ? FVM_OK : FVM_ERR_NOT_CONVERGED;
    };
    fvm_status st = run();
    if (saved) {   // the case's p and b back, whatever happened after they were saved
        const std::string msg = g_err;
        cudaError_t e1 = cudaMemcpyAsync(c->p, p_save, N * 8, cudaMemcpyDeviceToDevice, s);
        cudaError_t e2 = cudaMemcpyAsync(b, b_save, N * 8, cudaMemcpyDeviceToDevice, s);
        cudaError_t e3 = cudaStreamSynchronize(s);
        g_err = msg;
        const bool restored = e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess;
        if (!restored && (st == FVM_OK || st == FVM_ERR_NOT_CONVERGED))
            st = fail(FVM_ERR_CUDA, "restoring p and b after the adjoint solve");
    }
    if (rel_out) *rel_out = rel;
    return st;
}

// device scratch of the vector-Jacobian products, freed when it goes out of scope
struct DevScratch {
    double* d = nullptr;
    ~DevScratch() {
        if (d) cudaFree(d);
    }
};

fvm_status vjp_checks(fvm_case* c, double dt, const void* a, const void* b) {
    if (!c || !a || !b) return fail(FVM_ERR_INVALID, "null case or buffer");
    if (c->prec != FVM_FP64 || c->inner != FVM_FP64) return fail(FVM_ERR_INVALID, "FP64 cases only");
    if (!(dt > 0.0)) return fail(FVM_ERR_INVALID, "dt must be > 0");
    return FVM_OK;
}

}  // namespace

fvm_status fvm_projection_vjp(fvm_case* c, double dt, const double* host_ybar, double* host_xbar, size_t n,
                              double rel_tol, int32_t max_vcycles, double* rel_out) {
    ST_TRY(vjp_checks(c, dt, host_ybar, host_xbar));
    if (!(rel_tol > 0.0) || max_vcycles < 1) return fail(FVM_ERR_INVALID, "need rel_tol > 0 and max_vcycles >= 1");
    const int64_t N = c->cd.N;
    if (n < (size_t)(4 * N)) return fail(FVM_ERR_INVALID, "buffers too small (4 N in, 3 N out)");
    cudaStream_t s = c->stream;
    DevScratch sc;   // ybar (4 N), xbar (3 N), the case's p and b (2 N)
    CUDA_TRY(cudaMalloc((void**)&sc.d, (size_t)9 * N * 8));
    double* ybar = sc.d;
    double* xbar = sc.d + 4 * N;
    CUDA_TRY(cudaMemcpyAsync(ybar, host_ybar, (size_t)4 * N * 8, cudaMemcpyHostToDevice, s));
    double rel = 0.0;
    const fvm_status st = projection_vjp_dev(c, dt, ybar, xbar, rel_tol, max_vcycles, sc.d + 7 * N, &rel);
    if (st == FVM_OK || st == FVM_ERR_NOT_CONVERGED) {
        CUDA_TRY(cudaMemcpyAsync(host_xbar, xbar, (size_t)3 * N * 8, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (st == FVM_ERR_NOT_CONVERGED) fail(st, "adjoint solve stopped at max_vcycles above rel_tol");
    if (rel_out) *rel_out = rel;
    return st;
}

fvm_status fvm_destruction_vjp(fvm_case* c, double dt, const double* host_ybar, double* host_xbar, size_t n) {
    ST_TRY(vjp_checks(c, dt, host_ybar, host_xbar));
    const int64_t N = c->cd.N;
    if (n < (size_t)(5 * N)) return fail(FVM_ERR_INVALID, "buffers too small (5 N in and out)");
    cudaStream_t s = c->stream;
    DevScratch sc;   // ybar (5 N), xbar (5 N), kernel scratch (17 N)
    CUDA_TRY(cudaMalloc((void**)&sc.d, (size_t)27 * N * 8));
    double* ybar = sc.d;
    double* xbar = sc.d + 5 * N;
    CUDA_TRY(cudaMemcpyAsync(ybar, host_ybar, (size_t)5 * N * 8, cudaMemcpyHostToDevice, s));
    KLAUNCH("adj_destruction", (double)N * (5 * 8 * 2 + 5 * 8 + 17 * 8 * 2), 2,
            launch_destruction_vjp(c->cd, ptrs(c->cur), dt, ybar, xbar, sc.d + 10 * N, s));
    CUDA_TRY(cudaMemcpyAsync(host_xbar, xbar, (size_t)5 * N * 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return FVM_OK;
}

namespace {

// The explicit stage of the current state into y (6 fields, forward Euler) with a fixed time step:
// the destruction-free explicit kernel with a time-step record holding dt.
fvm_status explicit_forward(fvm_case* c, double dt, StatePtrs x, StatePtrs y, double* dt_dev) {
    double h[4] = {dt, 0.5 * dt, 0.0, 0.0};
    float hf[2] = {(float)dt, (float)(0.5 * dt)};
    CUDA_TRY(cudaMemcpyAsync(dt_dev, h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(dt_dev + 4, hf, sizeof(hf), cudaMemcpyHostToDevice, c->stream));
    KLAUNCH("explicit", (double)c->cd.N * (13 * 8 + 3), 1,
            launch_explicit(c->prec, c->cd, x, y, dt_dev, nullptr, StatePtrs{}, 0.0, 0.0, c->stream));
    return FVM_OK;
}

}  // namespace

fvm_status fvm_explicit_vjp(fvm_case* c, double dt, const double* host_ybar, double* host_xbar, size_t n) {
    ST_TRY(vjp_checks(c, dt, host_ybar, host_xbar));
    if (c->desc.rk_stages > 1) return fail(FVM_ERR_INVALID, "forward-Euler cases only (rk_stages 0 or 1)");
    const int64_t N = c->cd.N;
    if (n < (size_t)(6 * N)) return fail(FVM_ERR_INVALID, "buffers too small (6 N in and out)");
    cudaStream_t s = c->stream;
    DevScratch sc;   // ybar (6 N), xbar (6 N), the stage's output (6 N), kernel scratch (16 N), time step
    CUDA_TRY(cudaMalloc((void**)&sc.d, (size_t)34 * N * 8 + 64));
    double* ybar = sc.d;
    double* xbar = sc.d + 6 * N;
    StatePtrs y;
    for (int f = 0; f < 6; ++f) y.f[f] = sc.d + (12 + f) * N;
    double* dt_dev = sc.d + 34 * N;
    CUDA_TRY(cudaMemcpyAsync(ybar, host_ybar, (size_t)6 * N * 8, cudaMemcpyHostToDevice, s));
    ST_TRY(explicit_forward(c, dt, ptrs(c->cur), y, dt_dev));
    KLAUNCH("adj_explicit", (double)N * (6 * 8 * 4 + 6 * 8 * 2 + 16 * 8 * 2), 2,
            launch_explicit_vjp(c->cd, ptrs(c->cur), y, dt, ybar, xbar, sc.d + 18 * N, s));
    CUDA_TRY(cudaMemcpyAsync(host_xbar, xbar, (size_t)6 * N * 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return FVM_OK;
}

fvm_status fvm_step_vjp(fvm_case* c, double dt, const double* host_ybar, double* host_xbar, size_t n,
                        double rel_tol, int32_t max_vcycles, double* rel_out) {
    ST_TRY(vjp_checks(c, dt, host_ybar, host_xbar));
    if (!(rel_tol > 0.0) || max_vcycles < 1) return fail(FVM_ERR_INVALID, "need rel_tol > 0 and max_vcycles >= 1");
    if (c->desc.rk_stages > 1) return fail(FVM_ERR_INVALID, "forward-Euler cases only (rk_stages 0 or 1)");
    const int64_t N = c->cd.N;
    if (n < (size_t)(7 * N)) return fail(FVM_ERR_INVALID, "buffers too small (7 N in, 6 N out)");
    cudaStream_t s = c->stream;
    // scratch (doubles): ybar 7 N | s1 k, omega 2 N | s2 6 N | bar 6 N | tmp 6 N | kernel 17 N |
    // projection save 2 N | time step
    DevScratch sc;
    CUDA_TRY(cudaMalloc((void**)&sc.d, (size_t)46 * N * 8 + 64));
    double* d = sc.d;
    double* ybar = d;
    double* s1k = d + 7 * N;
    double* s1o = d + 8 * N;
    StatePtrs s2;
    for (int f = 0; f < 6; ++f) s2.f[f] = d + (9 + f) * N;
    double* bar = d + 15 * N;      // u, v, w, T, k, omega
    double* tmp = d + 21 * N;
    double* kern = d + 27 * N;
    double* psave = d + 44 * N;
    double* dt_dev = d + 46 * N;
    CUDA_TRY(cudaMemcpyAsync(ybar, host_ybar, (size_t)7 * N * 8, cudaMemcpyHostToDevice, s));
    // forward: s1 = D(x0) over dt/2 (k, omega only), s2 = E(s1) over dt
    const StatePtrs x0 = ptrs(c->cur);
    double h[4] = {dt, 0.5 * dt, 0.0, 0.0};
    float hf[2] = {(float)dt, (float)(0.5 * dt)};
    CUDA_TRY(cudaMemcpyAsync(dt_dev, h, sizeof(h), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(dt_dev + 4, hf, sizeof(hf), cudaMemcpyHostToDevice, s));
    KLAUNCH("destruction", (double)N * (8 * 8 + 3), 1,
            launch_destruction(c->prec, c->cd, x0, s1k, s1o, dt_dev, nullptr, nullptr, s));
    StatePtrs s1 = x0;
    s1.f[4] = s1k;
    s1.f[5] = s1o;
    ST_TRY(explicit_forward(c, dt, s1, s2, dt_dev));
    // backward: the projection (u, v, w, p cotangents; ybar holds u, v, w, p in id order)
    double rel = 0.0;
    const fvm_status pst = projection_vjp_dev(c, dt, ybar, bar, rel_tol, max_vcycles, psave, &rel);
    if (pst != FVM_OK && pst != FVM_ERR_NOT_CONVERGED) return pst;
    // bar: u, v, w (from the projection), T, k, omega (of the output)
    CUDA_TRY(cudaMemcpyAsync(bar + 3 * N, ybar + 4 * N, (size_t)3 * N * 8, cudaMemcpyDeviceToDevice, s));
    // through the second half step at s2: (u, v, w, k, omega) cotangents, T passes
    auto through_destruction = [&](StatePtrs x) -> fvm_status {
        // tmp: u, v, w, k, omega of bar (contiguous for the kernel)
        CUDA_TRY(cudaMemcpyAsync(tmp, bar, (size_t)3 * N * 8, cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(tmp + 3 * N, bar + 4 * N, (size_t)2 * N * 8, cudaMemcpyDeviceToDevice, s));
        KLAUNCH("adj_destruction", (double)N * (5 * 8 * 2 + 5 * 8 + 17 * 8 * 2), 2,
                launch_destruction_vjp(c->cd, x, 0.5 * dt, tmp, tmp, kern, s));
        CUDA_TRY(cudaMemcpyAsync(bar, tmp, (size_t)3 * N * 8, cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(bar + 4 * N, tmp + 3 * N, (size_t)2 * N * 8, cudaMemcpyDeviceToDevice, s));
        return FVM_OK;
    };
    ST_TRY(through_destruction(s2));
    // through the explicit stage at s1 (its output s2 decides the clamps)
    KLAUNCH("adj_explicit", (double)N * (6 * 8 * 4 + 6 * 8 * 2 + 16 * 8 * 2), 2,
            launch_explicit_vjp(c->cd, s1, s2, dt, bar, tmp, kern, s));
    CUDA_TRY(cudaMemcpyAsync(bar, tmp, (size_t)6 * N * 8, cudaMemcpyDeviceToDevice, s));
    // through the first half step at x0
    ST_TRY(through_destruction(x0));
    CUDA_TRY(cudaMemcpyAsync(host_xbar, bar, (size_t)6 * N * 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (rel_out) *rel_out = rel;
    if (pst == FVM_ERR_NOT_CONVERGED) return fail(pst, "adjoint solve stopped at max_vcycles above rel_tol");
    return FVM_OK;
}

fvm_status fvm_batch_create(fvm_case* const* cases, int32_t n, void* stream, fvm_batch** out) {
    if (!out) return fail(FVM_ERR_INVALID, "null output");
    ST_TRY(batch_check(cases, n));
    fvm_batch* B = new fvm_batch;
    B->cases.assign(cases, cases + n);
    auto bail = [&](fvm_status st) {
        free_batch(B);
        return st;
    };
    if (stream) B->stream = (cudaStream_t)stream;
    else {
        if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(FVM_ERR_CUDA, "cudaStreamCreate"));
        B->own_stream = true;
    }
    std::vector<SolveState*> sts(n);
    std::vector<double*> dts(n);
    for (int i = 0; i < n; ++i) {
        sts[i] = cases[i]->sst;
        dts[i] = cases[i]->dt_state;
    }
    if (cudaMalloc((void**)&B->d_sts, n * sizeof(SolveState*)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_dts, n * sizeof(double*)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_gather, n * sizeof(BatchGather)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_outer, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_scratch, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost((void**)&B->h_gather, n * sizeof(BatchGather)) != cudaSuccess ||
        cudaMallocHost((void**)&B->h_outer, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(FVM_ERR_OOM, "batch buffers"));
    }
    if (cudaMemcpy(B->d_sts, sts.data(), n * sizeof(SolveState*), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B->d_dts, dts.data(), n * sizeof(double*), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(fail(FVM_ERR_CUDA, "batch pointer tables"));
    g_err.clear();
    *out = B;
    return FVM_OK;
}

void fvm_batch_destroy(fvm_batch* b) { free_batch(b); }

fvm_status fvm_batch_launch(fvm_batch* B, int32_t nsteps) {
    if (!B) return fail(FVM_ERR_INVALID, "null batch");
    if (nsteps < 0) return fail(FVM_ERR_INVALID, "nsteps < 0");
    if (B->pending) return fail(FVM_ERR_INVALID, "the batch already has steps in flight");
    ST_TRY(batch_check(B->cases.data(), (int)B->cases.size()));
    const int n = (int)B->cases.size();
    cudaStream_t s = B->stream;
    // earlier work on the cases' own streams comes first
    for (fvm_case* c : B->cases)
        if (c->stream != s) CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (fvm_case* c : B->cases) {
        CUDA_TRY(cudaMemsetAsync(&c->sst->total_cycles, 0, sizeof(int32_t), s));
        CUDA_TRY(cudaMemsetAsync(&c->sst->nonfinite, 0, sizeof(int32_t), s));
        CUDA_TRY(cudaMemsetAsync(&c->sst->notconv, 0, sizeof(int32_t), s));
    }
    CUDA_TRY(cudaMemsetAsync(B->d_outer, 0, sizeof(unsigned long long), s));
    int64_t fixed = 0, per_outer = 0;
    for (int k = 0; k < nsteps; ++k) {
        int g = -1;
        ST_TRY(batch_graph(B, g));
        const fvm_batch::Graph& G = B->graphs[g];
        CUDA_TRY(cudaGraphLaunch(G.exec, s));
        for (int i = 0; i < n; ++i) {
            load_ptrs(B->cases[i], &G.after[12 * (size_t)i]);
            ++B->cases[i]->steps;
        }
        fixed += G.per_step;
        per_outer = G.per_outer;
        ++B->steps;
    }
    CUDA_TRY(cudaMemcpyAsync(B->h_gather, B->d_gather, n * sizeof(BatchGather), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(B->h_outer, B->d_outer, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    B->pending = true;
    B->pend_steps = nsteps;
    B->pend_fixed = fixed;
    B->pend_per_outer = per_outer;
    return FVM_OK;
}

fvm_status fvm_batch_wait(fvm_batch* B, fvm_step_stats* stats) {
    if (!B) return fail(FVM_ERR_INVALID, "null batch");
    if (!B->pending) return fail(FVM_ERR_INVALID, "no steps in flight");
    B->pending = false;
    const int n = (int)B->cases.size();
    const int32_t nsteps = B->pend_steps;
    CUDA_TRY(cudaStreamSynchronize(B->stream));
    if (nsteps > 0) B->launches += B->pend_fixed + (int64_t)*B->h_outer * B->pend_per_outer;
    fvm_status result = FVM_OK;
    for (int i = 0; i < n; ++i) {
        const BatchGather& q = B->h_gather[i];
        if (stats) {
            fvm_step_stats& o = stats[i];
            memset(&o, 0, sizeof(o));
            o.steps = nsteps;
            if (nsteps > 0) {
                o.vcycles_total = q.total_cycles;
                o.vcycles_last = q.cycles;
                o.rel_residual = q.rel;
                o.dt_last = q.dt;
                o.sim_time = q.sim_time;
            }
        }
        if (nsteps > 0 && q.nonfinite && result != FVM_ERR_DIVERGED)
            result = fail(FVM_ERR_DIVERGED, "non-finite pressure residual in case " + std::to_string(i));
        else if (nsteps > 0 && q.notconv && result == FVM_OK) {
            result = FVM_ERR_NOT_CONVERGED;
            g_err = "V-cycle cap reached above the tolerance in case " + std::to_string(i);
        }
    }
    return result;
}

fvm_status fvm_batch_step(fvm_batch* B, int32_t nsteps, fvm_step_stats* stats) {
    ST_TRY(fvm_batch_launch(B, nsteps));
    return fvm_batch_wait(B, stats);
}

fvm_status fvm_batch_get_info(const fvm_batch* B, fvm_batch_info* out) {
    if (!B || !out) return fail(FVM_ERR_INVALID, "null batch or output");
    fvm_batch_info info;
    memset(&info, 0, sizeof(info));
    info.n_cases = (int32_t)B->cases.size();
    info.graphs = (int32_t)B->graphs.size();
    info.steps = B->steps;
    info.kernel_launches = B->launches;
    int64_t cells = 0;
    for (const fvm_case* c : B->cases) cells += c->cd.N;
    info.cells = cells;
    if (!B->graphs.empty()) {
        info.launches_per_step = B->graphs[0].per_step;
        info.launches_per_outer = B->graphs[0].per_outer;
    }
    *out = info;
    return FVM_OK;
}

fvm_status fvm_batch_profile(fvm_batch* B, int32_t nsteps, fvm_kernel_stat* out, int32_t cap, int32_t* n_out) {
    if (!B || (!out && cap > 0)) return fail(FVM_ERR_INVALID, "null batch or output");
    if (nsteps < 0) return fail(FVM_ERR_INVALID, "nsteps < 0");
    if (B->pending) return fail(FVM_ERR_INVALID, "the batch has steps in flight");
    ST_TRY(batch_check(B->cases.data(), (int)B->cases.size()));
    const int n = (int)B->cases.size();
    cudaStream_t s = B->stream;
    for (fvm_case* c : B->cases) CUDA_TRY(cudaStreamSynchronize(c->stream));
    struct Ev {
        int site;
        cudaEvent_t a, b;
    };
    std::vector<Ev> evs;
    std::vector<std::string> names;
    std::vector<double> bytes;
    std::vector<int64_t> count;
    auto release = [&]() {
        for (Ev& e : evs) {
            cudaEventDestroy(e.a);
            cudaEventDestroy(e.b);
        }
        evs.clear();
    };
    auto run = [&](const Merged& m) -> fvm_status {
        int site = -1;
        for (size_t q = 0; q < names.size(); ++q)
            if (names[q] == m.site) site = (int)q;
        if (site < 0) {
            site = (int)names.size();
            names.push_back(m.site);
            bytes.push_back(0.0);
            count.push_back(0);
        }
        Ev e{site, nullptr, nullptr};
        if (cudaEventCreate(&e.a) != cudaSuccess || cudaEventCreate(&e.b) != cudaSuccess)
            return fail(FVM_ERR_CUDA, "cudaEventCreate");
        evs.push_back(e);
        BatchCtl ctl = m.ctl;
        ctl.use_cond = 0;   // the host drives the loop
        CUDA_TRY(cudaEventRecord(e.a, s));
        cudaError_t err = m.many(m.tab, m.map, m.nblk, m.block, m.smem, &ctl, s);
        if (err != cudaSuccess) return fail(FVM_ERR_CUDA, "batched launch " + m.site + ": " + cudaGetErrorString(err));
        CUDA_TRY(cudaEventRecord(e.b, s));
        bytes[site] += m.bytes;
        count[site] += 1;
        B->launches += 1;
        return FVM_OK;
    };
    fvm_status st = FVM_OK;
    for (int k = 0; k < nsteps && st == FVM_OK; ++k) {
        int g = -1;
        if ((st = batch_graph(B, g)) != FVM_OK) break;
        fvm_batch::Graph& G = B->graphs[g];
        for (const Merged& m : G.seg[0])
            if (st == FVM_OK) st = run(m);
        for (int it = 0; st == FVM_OK; ++it) {
            st = run(G.seg[1][0]);
            if (st != FVM_OK) break;
            k_batch_gather<<<1, 256, 0, s>>>(B->d_sts, B->d_dts, B->d_gather, n, B->d_scratch);
            if (cudaMemcpyAsync(B->h_gather, B->d_gather, n * sizeof(BatchGather), cudaMemcpyDeviceToHost, s) !=
                    cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                st = fail(FVM_ERR_CUDA, "reading the batch's solve states");
                break;
            }
            bool any = false;
            for (int i = 0; i < n; ++i) any = any || B->h_gather[i].active;
            if (!any) break;
            for (const Merged& m : G.seg[2])
                if (st == FVM_OK) st = run(m);
        }
        for (const Merged& m : G.seg[3])
            if (st == FVM_OK) st = run(m);
        if (st != FVM_OK) break;
        for (int i = 0; i < n; ++i) {
            load_ptrs(B->cases[i], &G.after[12 * (size_t)i]);
            ++B->cases[i]->steps;
        }
        ++B->steps;
    }
    if (st == FVM_OK && cudaStreamSynchronize(s) != cudaSuccess) st = fail(FVM_ERR_CUDA, "profiled batch steps");
    std::vector<double> ms(names.size(), 0.0);
    if (st == FVM_OK)
        for (Ev& e : evs) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, e.a, e.b) == cudaSuccess) ms[e.site] += t;
        }
    release();
    if (st != FVM_OK) return st;
    const int m = (int)names.size();
    for (int i = 0; i < m && i < cap; ++i) {
        memset(&out[i], 0, sizeof(out[i]));
        strncpy(out[i].name, names[i].c_str(), sizeof(out[i].name) - 1);
        out[i].launches = count[i];
        out[i].ms = ms[i];
        out[i].bytes = bytes[i];
    }
    if (n_out) *n_out = m;
    return FVM_OK;
}

fvm_status fvm_step_batch(fvm_case* const* cases, int n, int nsteps, fvm_step_stats* stats) {
    if (!cases || n < 0) return fail(FVM_ERR_INVALID, "bad case array");
    if (n == 0) return FVM_OK;
    fvm_batch* B = nullptr;
    ST_TRY(fvm_batch_create(cases, n, nullptr, &B));
    fvm_status st = fvm_batch_step(B, nsteps, stats);
    const std::string msg = g_err;
    free_batch(B);
    g_err = msg;
    return st;
}

fvm_status fvm_case_get_info(const fvm_case* c, fvm_case_info* out) {
    if (!c || !out) return fail(FVM_ERR_INVALID, "null case or output");
    fvm_case_info info;
    memset(&info, 0, sizeof(info));
    info.cells = c->cd.N;
    info.levels = (int32_t)c->levels.size();
    info.precision = c->desc.precision;
    info.dt0 = c->dt0;
    double dts[3] = {0, 0, 0};
    if (cudaMemcpy(dts, c->dt_state, sizeof(dts), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(FVM_ERR_CUDA, "reading dt");
    info.dt = dts[0];
    info.sim_time = dts[2];
    info.device_bytes = c->bytes;
    info.steps = c->steps;
    info.kernel_launches = c->launches;
    *out = info;
    return FVM_OK;
}

fvm_status fvm_set_option(fvm_case* c, int option, int64_t value) {
    if (!c) return fail(FVM_ERR_INVALID, "null case");
    if (option == FVM_OPT_GRAPH) {
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        c->use_graph = value != 0;
        if (!c->use_graph) drop_graphs(c);
        return FVM_OK;
    }
    return fail(FVM_ERR_INVALID, "unknown option");
}

fvm_status fvm_profile_enable(fvm_case* c, int enable) {
    if (!c) return fail(FVM_ERR_INVALID, "null case");
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    prof_clear(c);
    c->prof = enable != 0;
    return FVM_OK;
}

fvm_status fvm_profile_read(fvm_case* c, fvm_kernel_stat* out, int cap, int* n_out) {
    if (!c || (cap > 0 && !out)) return fail(FVM_ERR_INVALID, "null case or output");
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    std::vector<fvm_kernel_stat> acc(c->cls_names.size());
    for (size_t i = 0; i < acc.size(); ++i) {
        memset(&acc[i], 0, sizeof(fvm_kernel_stat));
        snprintf(acc[i].name, sizeof(acc[i].name), "%s", c->cls_names[i].c_str());
    }
    for (auto& r : c->recs) {
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
        acc[r.cls].launches += 1;
        acc[r.cls].ms += ms;
        acc[r.cls].bytes += r.bytes;
    }
    for (int i = 0; i < (int)acc.size() && i < cap; ++i) out[i] = acc[i];
    if (n_out) *n_out = (int)acc.size();
    prof_clear(c);
    return FVM_OK;
}

void fvm_struct_sizes(size_t out[11]) {
    out[0] = sizeof(fvm_patch);
    out[1] = sizeof(fvm_vent);
    out[2] = sizeof(fvm_box);
    out[3] = sizeof(fvm_case_desc);
    out[4] = sizeof(fvm_step_stats);
    out[5] = sizeof(fvm_case_info);
    out[6] = sizeof(fvm_kernel_stat);
    out[7] = sizeof(fvm_batch_info);
    out[8] = sizeof(fvm_request_result);
    out[9] = sizeof(fvm_server_info);
    out[10] = sizeof(fvm_tuning);
}

const char* fvm_last_error(void) { return g_err.c_str(); }

}  // extern "C"
