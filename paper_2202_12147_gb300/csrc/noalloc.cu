// Deterministic force spreading that allocates nothing: the fixed-point
// accumulation grid lives in a library-owned static device array instead of
// caller memory.  See ib_spread_fixed_noalloc in include/lbib.h.
//
// The arithmetic is the same as the deterministic spreading of a context
// (k_ib_gather_spread with 64-bit fixed-point atomics): the same stencil
// set-up, the same per-contribution rounding to 2^-48 units and an exact
// integer sum, so both give bitwise the same force field for the same node
// positions and forces.
#include <mutex>
#include <string>

#include "lbib_internal.cuh"

using namespace lbib;

namespace {

// Largest box the scratch grid holds: 64^3 cells, three int64 planes (6 MiB).
constexpr long long NOALLOC_MAX_CELLS = 262144;
constexpr int MAX_DEVICES = 64;

// The scratch grid.  In host code this name is only a stand-in for the
// device array; kernels are given the device address obtained below.
static __device__ __align__(256) unsigned long long g_spread_acc[3 * NOALLOC_MAX_CELLS];

std::mutex g_mu;
unsigned long long *g_acc_addr[MAX_DEVICES] = {};

void noalloc_msg(const std::string &m) { lbib::set_last_error(m.c_str()); }

// Device address of the scratch grid on the current device, looked up once
// per device (with that device current) and cached.
cudaError_t scratch_address(unsigned long long **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_acc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_spread_acc);
        if (e != cudaSuccess) return e;
        g_acc_addr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = g_acc_addr[dev];
    return cudaSuccess;
}

__global__ void k_acc_clear(unsigned long long *acc, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        acc[k] = 0ull;
}

// KW^2 threads per node, one per (y, z) stencil row, as in the context path.
template <int KW>
__global__ void k_spread_fixed(const double *r, const float *f, int n_nodes, int nx, int ny, int nz,
                               unsigned long long *acc, long long N) {
    constexpr int ROWS = KW * KW;
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long j = gt / ROWS;
    const int row = (int)(gt % ROWS);
    if (j >= n_nodes) return;
    float fr;
    float wx[KW], wy[KW], wz[KW];
    const int ox = stencil_axis(r[3 * j + 0], nx, KW, fr);
    weights1d<KW>(fr, wx);
    const int oy = stencil_axis(r[3 * j + 1], ny, KW, fr);
    weights1d<KW>(fr, wy);
    const int oz = stencil_axis(r[3 * j + 2], nz, KW, fr);
    weights1d<KW>(fr, wz);
    const float fx = f[3 * j + 0], fy = f[3 * j + 1], fz = f[3 * j + 2];
    const int dy = row % KW, dz = row / KW;
    const int yy = (oy + dy) % ny, zz = (oz + dz) % nz;
    const float wyz = wy[dy] * wz[dz];
    const unsigned rowbase = (unsigned)nx * ((unsigned)yy + (unsigned)ny * (unsigned)zz);
#pragma unroll
    for (int k = 0; k < KW; ++k) {
        const unsigned cell = rowbase + (unsigned)((ox + k) % nx);
        const float w = wx[k] * wyz;
        // scaling by 2^48 is exact in FP32, so this is the nearest integer to
        // the FP32 contribution in 2^-48 units, with no FP64 arithmetic
        atomicAdd(&acc[cell], (unsigned long long)__float2ll_rn((w * fx) * FIX_SCALE_F));
        atomicAdd(&acc[N + cell], (unsigned long long)__float2ll_rn((w * fy) * FIX_SCALE_F));
        atomicAdd(&acc[2 * N + cell], (unsigned long long)__float2ll_rn((w * fz) * FIX_SCALE_F));
    }
}

__global__ void k_acc_to_float(const unsigned long long *acc, long long N, float *out) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N; k += (long long)gridDim.x * blockDim.x)
        // one rounding (integer to FP32), then an exact scaling by 2^-48
        for (int a = 0; a < 3; ++a) out[3 * k + a] = __ll2float_rn((long long)acc[a * N + k]) * FIX_INV_F;
}

}  // namespace

extern "C" int ib_spread_fixed_noalloc(const double *nodes, const float *node_forces, int n_nodes, int nx, int ny,
                                       int nz, int kernel, float *F_out, void *stream) {
    if (nx < 1 || ny < 1 || nz < 1 || n_nodes < 0) {
        noalloc_msg("box dimensions must be >= 1 and n_nodes >= 0");
        return LBIB_EINVAL;
    }
    if (kernel != LBIB_PESKIN4 && kernel != LBIB_LINEAR2) {
        noalloc_msg("unknown delta kernel");
        return LBIB_EINVAL;
    }
    const long long N = (long long)nx * ny * nz;
    if (N > NOALLOC_MAX_CELLS) {
        noalloc_msg("box of " + std::to_string(N) + " cells exceeds the " + std::to_string(NOALLOC_MAX_CELLS) +
                    "-cell maximum of the library-owned scratch grid");
        return LBIB_ESIZE;
    }
    if (!F_out || (n_nodes > 0 && (!nodes || !node_forces))) {
        noalloc_msg("NULL pointer argument");
        return LBIB_EINVAL;
    }
    unsigned long long *acc = nullptr;
    cudaError_t e = scratch_address(&acc);
    if (e != cudaSuccess) {
        noalloc_msg(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return LBIB_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int tpb = 256;
    const int clear_blocks = (int)((3 * N + tpb - 1) / tpb);
    k_acc_clear<<<clear_blocks, tpb, 0, s>>>(acc, 3 * N);
    if (n_nodes > 0) {
        const int rows = kernel == LBIB_LINEAR2 ? 4 : 16;
        const int blocks = (int)(((long long)n_nodes * rows + tpb - 1) / tpb);
        if (kernel == LBIB_LINEAR2) k_spread_fixed<2><<<blocks, tpb, 0, s>>>(nodes, node_forces, n_nodes, nx, ny, nz, acc, N);
        else k_spread_fixed<4><<<blocks, tpb, 0, s>>>(nodes, node_forces, n_nodes, nx, ny, nz, acc, N);
    }
    k_acc_to_float<<<(int)((N + tpb - 1) / tpb), tpb, 0, s>>>(acc, N, F_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        noalloc_msg(std::string("kernel launch: ") + cudaGetErrorString(e));
        return LBIB_ECUDA;
    }
    return LBIB_OK;
}
