// D3Q19 BGK fused collide-and-stream with body forcing, in place (AA pattern).
//
// Physics (Sec. 2.1): f_i(x + c_i, t + 1) = f_i - (f_i - f_i^eq)/tau
// (Eq. lbe) with the second-order equilibrium (Eq. lbm:equilibrium), density
// rho = sum f_i and physical velocity rho u = sum f_i c_i + F/2.  Force
// inclusion: Guo's source term (default) or the paper's Shan-Chen shift
// rho u^eq = sum f_i c_i + tau F (Eq. sc).
//
// Storage: populations are kept as shifted deviations d_i = f_i - w_i rho0,
// one plane per direction ([i][z][y][x], plane stride Npad), in FP32, or in
// FP16/BF16 as d_i / w_i * S.  The collision is written in deviation form,
// rho = rho0 + sum d_i and sum f_i c_i = sum d_i c_i, so FP32 keeps ~7
// significant digits of the small velocities a low-Reynolds swimmer makes.
//
// In-place streaming, AA pattern: an even step reads d_i from its own cell
// and writes the post-collision value of direction i into slot opp(i) of the
// same cell; an odd step reads direction i from slot opp(i) of cell x - c_i
// and writes it into slot i of cell x + c_i.  Each step touches every
// population once for reading and once for writing (2 x 19 values per cell),
// and a location is only ever read and written by the thread of one cell, so
// one array suffices and any partition of the cells can be updated
// concurrently.
//
// Immersed-boundary coupling: the cells are grouped in tiles (runs of up to
// tile_x cells along x of one (y, z) row).  Before a step, the tiles that the
// nodes' delta-kernel stencils touch are marked and listed (one mark array and
// one list per step parity).  k_lb_main updates every unmarked tile and never
// touches the force and velocity fields; k_lb_marked walks the list, reads F
// there, writes the physical velocity u for the interpolation and clears F.
// The two kernels cover disjoint cells, so k_lb_main can run while the
// immersed-boundary kernels of the same step run on another stream.
#include "lbib_internal.cuh"

namespace lbib {

template <int S>
struct Store;
template <>
struct Store<LBIB_F32> {
    using T = float;
    static __device__ __forceinline__ float ld(const T *p, float) { return *p; }
    static __device__ __forceinline__ void st(T *p, float v, float) { *p = v; }
    static constexpr bool scaled = false;
};
template <>
struct Store<LBIB_F16> {
    using T = __half;
    static __device__ __forceinline__ float ld(const T *p, float m) { return __half2float(*p) * m; }
    static __device__ __forceinline__ void st(T *p, float v, float m) { *p = __float2half_rn(v * m); }
    static constexpr bool scaled = true;
};
template <>
struct Store<LBIB_BF16> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float ld(const T *p, float m) { return __bfloat162float(*p) * m; }
    static __device__ __forceinline__ void st(T *p, float v, float m) { *p = __float2bfloat16_rn(v * m); }
    static constexpr bool scaled = true;
};

// BGK collision with body force on one cell, in deviation form (Sec. 2.1,
// Eqs. lbe and lbm:equilibrium; physical velocity with F/2).  Opposite
// directions i, i+1 (odd i) share c_{i+1} = -c_i, so each pair needs one c.u:
// the equilibrium splits into an even part w (drho + rho (4.5 (c.u)^2 - 1.5 u.u))
// and an odd part 3 w rho (c.u), and Guo's source term likewise into
// w gu (9 (c.u)(c.F) - 3 u.F) and 3 w gu (c.F).  d[] holds the pre-collision
// deviations on entry and the post-collision deviations on exit.
template <int FORCING>
__device__ __forceinline__ void collide_cell(float (&d)[Q], const DevCtx &c, bool forced, float Fx, float Fy, float Fz,
                                             float &ux, float &uy, float &uz, float &rho) {
    float drho = d[0], jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int k = 1; k < Q; k += 2) {
        const float sm = d[k] + d[k + 1], df = d[k] - d[k + 1];
        drho += sm;
        if (cx(k)) jx += cx(k) > 0 ? df : -df;
        if (cy(k)) jy += cy(k) > 0 ? df : -df;
        if (cz(k)) jz += cz(k) > 0 ? df : -df;
    }
    rho = c.rho0 + drho;
    const float irho = 1.0f / rho;
    ux = (jx + 0.5f * Fx) * irho;
    uy = (jy + 0.5f * Fy) * irho;
    uz = (jz + 0.5f * Fz) * irho;
    float ex = ux, ey = uy, ez = uz;
    if (FORCING == LBIB_SHAN_CHEN) {
        ex = (jx + c.tau * Fx) * irho;
        ey = (jy + c.tau * Fy) * irho;
        ez = (jz + c.tau * Fz) * irho;
    }
    const float om = c.omega;
    const float base = drho - rho * 1.5f * (ex * ex + ey * ey + ez * ez);
    const bool guo = FORCING == LBIB_GUO && forced;
    const float gu = guo ? 1.0f - 0.5f * om : 0.f;
    const float uF3 = guo ? 3.0f * (ux * Fx + uy * Fy + uz * Fz) : 0.f;
    {
        float post = d[0] + om * (wgt(0) * base - d[0]);
        if (guo) post -= gu * wgt(0) * uF3;
        d[0] = post;
    }
#pragma unroll
    for (int k = 1; k < Q; k += 2) {
        const float w = wgt(k);
        const float cu = cx(k) * ex + cy(k) * ey + cz(k) * ez;
        const float ev = w * fmaf(4.5f * rho * cu, cu, base);
        const float od = 3.0f * w * rho * cu;
        float p0 = d[k] + om * ((ev + od) - d[k]);
        float p1 = d[k + 1] + om * ((ev - od) - d[k + 1]);
        if (guo) {
            const float cF = cx(k) * Fx + cy(k) * Fy + cz(k) * Fz;
            const float sev = gu * w * (9.0f * cu * cF - uF3);
            const float sod = 3.0f * gu * w * cF;
            p0 += sev + sod;
            p1 += sev - sod;
        }
        d[k] = p0;
        d[k + 1] = p1;
    }
}

// Read the 3 fixed-point force components of a cell and clear them.
__device__ __forceinline__ float3 take_fdet(unsigned long long *Fd, long long Npad, unsigned cell) {
    long long a = (long long)Fd[cell], b = (long long)Fd[Npad + cell], c = (long long)Fd[2 * Npad + cell];
    Fd[cell] = 0ull;
    Fd[Npad + cell] = 0ull;
    Fd[2 * Npad + cell] = 0ull;
    return make_float3((float)((double)a * FIX_INV), (float)((double)b * FIX_INV), (float)((double)c * FIX_INV));
}

// Full update of cell (x, y, z): load (streaming pull of the AA pattern),
// collide, store.  MARKED cells also consume F and publish u.  Returns false
// if the density or velocity is not finite.
template <int ST, bool ODD, int FORCING, bool DET, bool MARKED>
__device__ __forceinline__ bool lb_cell(const DevCtx &c, unsigned x, unsigned y, unsigned z) {
    using S = Store<ST>;
    using T = typename S::T;
    T *__restrict__ P = reinterpret_cast<T *>(c.pops);
    const unsigned nx = c.nx, ny = c.ny, nz = c.nz, nxy = nx * ny;
    const unsigned xm = x ? x - 1 : nx - 1, xp = (x + 1 == nx) ? 0 : x + 1;
    const unsigned rm = (y ? y - 1 : ny - 1) * nx, r0 = y * nx, rp = ((y + 1 == ny) ? 0 : y + 1) * nx;
    const unsigned sm = (z ? z - 1 : nz - 1) * nxy, s0 = z * nxy, sp = ((z + 1 == nz) ? 0 : z + 1) * nxy;
    const unsigned cell = x + r0 + s0;
    const size_t Np = (size_t)c.Npad;
    float d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float m = S::scaled ? wgt(i) * c.st_inv_scale : 1.0f;
        if (ODD) {
            // direction i of this cell sits in slot opp(i) of cell x - c_i
            const int dx = -cx(i), dy = -cy(i), dz = -cz(i);
            const unsigned nb = (dx < 0 ? xm : dx > 0 ? xp : x) + (dy < 0 ? rm : dy > 0 ? rp : r0) +
                                (dz < 0 ? sm : dz > 0 ? sp : s0);
            d[i] = S::ld(P + opp(i) * Np + nb, m);
        } else {
            d[i] = S::ld(P + i * Np + cell, m);
        }
    }
    const bool forced = MARKED || c.has_g;
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    if (MARKED) {
        if (DET) {
            const float3 f = take_fdet(c.Fdet, c.Npad, cell);
            Fx = f.x; Fy = f.y; Fz = f.z;
        } else {
            const float4 f = c.F[cell];
            c.F[cell] = make_float4(0.f, 0.f, 0.f, 0.f);
            Fx = f.x; Fy = f.y; Fz = f.z;
        }
    }
    if (forced) {
        Fx += c.g[0];
        Fy += c.g[1];
        Fz += c.g[2];
    }
    float ux, uy, uz, rho;
    collide_cell<FORCING>(d, c, forced, Fx, Fy, Fz, ux, uy, uz, rho);
    if (MARKED) c.U[cell] = make_float4(ux, uy, uz, rho);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float m = S::scaled ? c.st_scale / wgt(i) : 1.0f;
        if (ODD) {
            const int dx = cx(i), dy = cy(i), dz = cz(i);
            const unsigned nb = (dx < 0 ? xm : dx > 0 ? xp : x) + (dy < 0 ? rm : dy > 0 ? rp : r0) +
                                (dz < 0 ? sm : dz > 0 ? sp : s0);
            S::st(P + i * Np + nb, d[i], m);
        } else {
            S::st(P + opp(i) * Np + cell, d[i], m);
        }
    }
    return isfinite(rho) && isfinite(ux + uy + uz);
}

__device__ __forceinline__ void report_bad(const DevCtx &c, bool bad) {
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&c.ctl->err, ERR_NONFINITE);
}

// Every unmarked tile: one block per tile, grid (tiles_x, ny, nz).
#ifndef LBIB_LB_GENERIC_MINB
#define LBIB_LB_GENERIC_MINB 3
#endif
template <int ST, bool ODD, int FORCING>
__global__ void __launch_bounds__(LB_TPB, LBIB_LB_GENERIC_MINB) k_lb_main(const DevCtx c) {
    const unsigned tile = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (c.marks[(ODD ? c.n_tiles : 0) + tile]) return;  // updated by k_lb_marked
    const unsigned x = blockIdx.x * c.tile_x + threadIdx.x;
    bool ok = true;
    if (threadIdx.x < (unsigned)c.tile_x && x < (unsigned)c.nx)
        ok = lb_cell<ST, ODD, FORCING, false, false>(c, x, blockIdx.y, blockIdx.z);
    report_bad(c, !ok);
    if (c.n_nodes == 0 && tile == 0 && threadIdx.x == 0) c.ctl->step += 1;  // no IB chain to advance it
}

// The marked tiles of this parity's list: a persistent grid walks the list.
template <int ST, bool ODD, int FORCING, bool DET>
__global__ void __launch_bounds__(LB_TPB, LBIB_LB_GENERIC_MINB) k_lb_marked(const DevCtx c) {
    const int p = ODD ? 1 : 0;
    const int n = c.tile_count[p];
    const int *list = c.tile_list + (size_t)p * c.n_tiles;
    bool ok = true;
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int tile = list[k];
        const unsigned tx = tile % c.tiles_x, yz = tile / c.tiles_x;
        const unsigned y = yz % c.ny, z = yz / c.ny;
        const unsigned x = tx * c.tile_x + threadIdx.x;
        if (threadIdx.x < (unsigned)c.tile_x && x < (unsigned)c.nx)
            ok &= lb_cell<ST, ODD, FORCING, DET, true>(c, x, y, z);
    }
    report_bad(c, !ok);
}

template <int ST, bool ODD>
__global__ void __launch_bounds__(LB_TPB) k_lb_macros(const DevCtx c, float *rho_out, float *u_out) {
    using S = Store<ST>;
    using T = typename S::T;
    const T *__restrict__ P = reinterpret_cast<const T *>(c.pops);
    const unsigned cell = blockIdx.x * LB_TPB + threadIdx.x;
    if (cell >= (unsigned)c.N) return;
    const unsigned nx = c.nx, ny = c.ny, nz = c.nz, nxy = nx * ny;
    const unsigned yz = cell / nx, x = cell - yz * nx;
    const unsigned z = yz / ny, y = yz - z * ny;
    const size_t Np = (size_t)c.Npad;
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float m = S::scaled ? wgt(i) * c.st_inv_scale : 1.0f;
        float v;
        if (ODD) {
            const unsigned xs = (x + nx - cx(i)) % nx, ys = (y + ny - cy(i)) % ny, zs = (z + nz - cz(i)) % nz;
            v = S::ld(P + opp(i) * Np + xs + nx * ys + nxy * zs, m);
        } else {
            v = S::ld(P + i * Np + cell, m);
        }
        drho += v;
        jx += cx(i) * v;
        jy += cy(i) * v;
        jz += cz(i) * v;
    }
    const float rho = c.rho0 + drho;
    rho_out[cell] = rho;
    u_out[3 * cell + 0] = jx / rho;
    u_out[3 * cell + 1] = jy / rho;
    u_out[3 * cell + 2] = jz / rho;
}

// ---------------------------------------------------------------- launchers

static unsigned tile_threads(const DevCtx &c) { return (unsigned)((c.tile_x + 31) / 32 * 32); }

template <int ST, int FORCING>
static void main_dispatch(const DevCtx &c, bool odd, cudaStream_t s) {
    const dim3 blocks((unsigned)c.tiles_x, (unsigned)c.ny, (unsigned)c.nz);
    if (odd) k_lb_main<ST, true, FORCING><<<blocks, tile_threads(c), 0, s>>>(c);
    else k_lb_main<ST, false, FORCING><<<blocks, tile_threads(c), 0, s>>>(c);
}

template <int ST, int FORCING>
static void marked_dispatch(const DevCtx &c, bool odd, cudaStream_t s) {
    const unsigned blocks = (unsigned)(c.n_tiles < c.marked_grid ? c.n_tiles : c.marked_grid);
    if (c.deterministic) {
        if (odd) k_lb_marked<ST, true, FORCING, true><<<blocks, tile_threads(c), 0, s>>>(c);
        else k_lb_marked<ST, false, FORCING, true><<<blocks, tile_threads(c), 0, s>>>(c);
    } else {
        if (odd) k_lb_marked<ST, true, FORCING, false><<<blocks, tile_threads(c), 0, s>>>(c);
        else k_lb_marked<ST, false, FORCING, false><<<blocks, tile_threads(c), 0, s>>>(c);
    }
}

#define LBIB_DISPATCH(fn, storage, forcing, ...)                                        \
    do {                                                                                \
        if (forcing == LBIB_SHAN_CHEN) {                                                \
            if (storage == LBIB_F16) fn<LBIB_F16, LBIB_SHAN_CHEN>(__VA_ARGS__);          \
            else if (storage == LBIB_BF16) fn<LBIB_BF16, LBIB_SHAN_CHEN>(__VA_ARGS__);   \
            else fn<LBIB_F32, LBIB_SHAN_CHEN>(__VA_ARGS__);                             \
        } else {                                                                        \
            if (storage == LBIB_F16) fn<LBIB_F16, LBIB_GUO>(__VA_ARGS__);                \
            else if (storage == LBIB_BF16) fn<LBIB_BF16, LBIB_GUO>(__VA_ARGS__);         \
            else fn<LBIB_F32, LBIB_GUO>(__VA_ARGS__);                                   \
        }                                                                               \
    } while (0)

cudaError_t launch_lb_main(const DevCtx &c, int storage, int forcing, bool odd, cudaStream_t s) {
    LBIB_DISPATCH(main_dispatch, storage, forcing, c, odd, s);
    return cudaGetLastError();
}

cudaError_t launch_lb_marked(const DevCtx &c, int storage, int forcing, bool odd, cudaStream_t s) {
    LBIB_DISPATCH(marked_dispatch, storage, forcing, c, odd, s);
    return cudaGetLastError();
}

template <int ST>
static cudaError_t macros_dispatch(const DevCtx &c, bool odd, float *rho, float *u, cudaStream_t s) {
    const unsigned blocks = (unsigned)((c.N + LB_TPB - 1) / LB_TPB);
    if (odd) k_lb_macros<ST, true><<<blocks, LB_TPB, 0, s>>>(c, rho, u);
    else k_lb_macros<ST, false><<<blocks, LB_TPB, 0, s>>>(c, rho, u);
    return cudaGetLastError();
}

cudaError_t launch_lb_macros(const DevCtx &c, int storage, bool odd, float *rho, float *u, cudaStream_t s) {
    if (storage == LBIB_F16) return macros_dispatch<LBIB_F16>(c, odd, rho, u, s);
    if (storage == LBIB_BF16) return macros_dispatch<LBIB_BF16>(c, odd, rho, u, s);
    return macros_dispatch<LBIB_F32>(c, odd, rho, u, s);
}

}  // namespace lbib
