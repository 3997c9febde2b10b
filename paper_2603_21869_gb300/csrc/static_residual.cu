// Pressure residual and norms without any device allocation.
//
// Some callers cannot allocate device memory: a host program whose memory is
// owned by a pooling allocator that forbids raw cudaMalloc, a control loop
// that must not pay the latency (and implicit synchronisation) of an
// allocation, or a plug-in that has to keep the process's device footprint
// fixed.  This file gives them r = b - A p and the squared norms ||r||^2,
// ||b||^2 on their own device buffers.  The only scratch the kernel needs
// (one pair of partial sums per block and a block counter) lives in the
// file-scope array below, which every GPU that loads the library holds until
// the process exits.
#include <mutex>
#include <string>

#include "fvm_internal.cuh"

namespace {

constexpr int SX = 32, SY = 4, SZ = 2;                  // block shape: 256 cells
constexpr int kMaxBlocks = 1 << 16;                     // 65,536 blocks = 16,777,216 cells at most
constexpr int kScratchDoubles = 2 * kMaxBlocks + 32;    // partial sums, then the block counter

static __device__ __align__(256) double g_residual_scratch[kScratchDoubles];

// r = b - A p on a box without obstacles: a face of the domain is
// zero-gradient (dirichlet[face] = 0) or zero-value (1) for p.
__global__ void __launch_bounds__(SX * SY * SZ) k_residual_static(const double* __restrict__ p,
                                                                  const double* __restrict__ b,
                                                                  double* __restrict__ r, double* __restrict__ norms,
                                                                  double* scratch, int nx, int ny, int nz,
                                                                  double ih2x, double ih2y, double ih2z,
                                                                  unsigned dir_mask) {
    __shared__ double red[2][SX * SY * SZ / 32];
    __shared__ bool last;
    const int i = blockIdx.x * SX + threadIdx.x, j = blockIdx.y * SY + threadIdx.y, k = blockIdx.z * SZ + threadIdx.z;
    const int tid = threadIdx.x + SX * (threadIdx.y + SY * threadIdx.z);
    double r2 = 0.0, b2 = 0.0;
    if (i < nx && j < ny && k < nz) {
        const int sy = nx, sz = nx * ny;
        const int c = i + sy * j + sz * k;
        const double pP = p[c];
        // across a face: the neighbour, or the ghost pP (zero gradient) / -pP (zero value)
        auto across = [&](bool inside, int q, int face) {
            if (inside) return p[q];
            return ((dir_mask >> face) & 1u) ? -pP : pP;
        };
        double Ap = 0.0;
        if (nx > 1) Ap += ((pP - across(i > 0, c - 1, 0)) + (pP - across(i < nx - 1, c + 1, 1))) * ih2x;
        if (ny > 1) Ap += ((pP - across(j > 0, c - sy, 2)) + (pP - across(j < ny - 1, c + sy, 3))) * ih2y;
        if (nz > 1) Ap += ((pP - across(k > 0, c - sz, 4)) + (pP - across(k < nz - 1, c + sz, 5))) * ih2z;
        const double bv = b[c];
        const double rv = bv - Ap;
        r[c] = rv;
        r2 = rv * rv;
        b2 = bv * bv;
    }
    for (int off = 16; off > 0; off >>= 1) {
        r2 += __shfl_xor_sync(0xffffffffu, r2, off);
        b2 += __shfl_xor_sync(0xffffffffu, b2, off);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = r2;
        red[1][tid >> 5] = b2;
    }
    __syncthreads();
    const int nblk = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    unsigned* counter = (unsigned*)(scratch + 2 * kMaxBlocks);
    if (tid == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int w = 0; w < SX * SY * SZ / 32; ++w) {
            s0 += red[0][w];
            s1 += red[1][w];
        }
        scratch[2 * bid] = s0;
        scratch[2 * bid + 1] = s1;
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned)nblk - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the last block sums the partials in a fixed order
    double a0 = 0.0, a1 = 0.0;
    for (int x = tid; x < nblk; x += SX * SY * SZ) {
        a0 += __ldcg(scratch + 2 * x);
        a1 += __ldcg(scratch + 2 * x + 1);
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
    if (tid == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int w = 0; w < SX * SY * SZ / 32; ++w) {
            s0 += red[0][w];
            s1 += red[1][w];
        }
        norms[0] = s0;
        norms[1] = s1;
        *counter = 0u;
    }
}

// Device address of the scratch array, looked up once per device.
std::mutex g_mu;
double* g_scratch_ptr[256] = {};

fvm_status scratch_for_current_device(double** out, std::string& err) {
    // first use on a device: look up the array's device address with that device current
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) {
        err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return FVM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_residual_scratch);
        if (e != cudaSuccess || !ptr) {
            err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return FVM_ERR_CUDA;
        }
        g_scratch_ptr[dev] = (double*)ptr;
    }
    *out = g_scratch_ptr[dev];
    return FVM_OK;
}

}  // namespace

extern "C" fvm_status fvm_poisson_residual_static(const double* p, const double* b, int32_t nx, int32_t ny,
                                                  int32_t nz, const double h[3], const int32_t dirichlet[6],
                                                  double* r, double* norms, void* stream) {
    if (!p || !b || !r || !norms || !h || !dirichlet) {
        set_last_error("null argument");
        return FVM_ERR_INVALID;
    }
    if (nx < 1 || ny < 1 || nz < 1 || !(h[0] > 0.0) || !(h[1] > 0.0) || !(h[2] > 0.0)) {
        set_last_error("grid dimensions must be >= 1 and spacings > 0");
        return FVM_ERR_INVALID;
    }
    // block counts in 64-bit arithmetic (nx near INT32_MAX must not wrap), each factor checked
    // before the product: y and z are also bounded by the launch limit of 65,535 blocks
    const int64_t gx = ((int64_t)nx + SX - 1) / SX, gy = ((int64_t)ny + SY - 1) / SY, gz = ((int64_t)nz + SZ - 1) / SZ;
    if (gx > kMaxBlocks || gy > 65535 || gz > 65535 || gx * gy > kMaxBlocks || gx * gy * gz > kMaxBlocks) {
        set_last_error("grid larger than the static scratch holds (65,536 blocks of 32 x 4 x 2 cells, at most "
                       "65,535 along y and z)");
        return FVM_ERR_INVALID;
    }
    const dim3 block(SX, SY, SZ);
    const dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)gz);
    double* scratch = nullptr;
    std::string err;
    fvm_status st = scratch_for_current_device(&scratch, err);
    if (st != FVM_OK) {
        set_last_error(err);
        return st;
    }
    unsigned mask = 0;
    for (int f = 0; f < 6; ++f)
        if (dirichlet[f]) mask |= 1u << f;
    cudaStream_t s = (cudaStream_t)stream;
    // the block counter must start at zero (a memset, not an allocation)
    cudaError_t e = cudaMemsetAsync(scratch + 2 * kMaxBlocks, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) {
        k_residual_static<<<grid, block, 0, s>>>(p, b, r, norms, scratch, nx, ny, nz, 1.0 / (h[0] * h[0]),
                                                 1.0 / (h[1] * h[1]), 1.0 / (h[2] * h[2]), mask);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_last_error(std::string("launch: ") + cudaGetErrorString(e));
        return FVM_ERR_CUDA;
    }
    set_last_error("");
    return FVM_OK;
}
