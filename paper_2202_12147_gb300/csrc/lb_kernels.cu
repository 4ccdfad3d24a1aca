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
// one array suffices.
//
// Immersed-boundary coupling: spreading marks the tiles (runs of up to
// tile_x cells along x) its stencils touch.  A block whose tile is marked reads F there, writes the
// physical velocity u (for the interpolation that follows), clears F and the
// mark; every other block skips both fields.
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

// Read the 3 fixed-point force components of a cell and clear them.
__device__ __forceinline__ float3 take_fdet(unsigned long long *Fd, long long Npad, unsigned cell) {
    long long a = (long long)Fd[cell], b = (long long)Fd[Npad + cell], c = (long long)Fd[2 * Npad + cell];
    Fd[cell] = 0ull;
    Fd[Npad + cell] = 0ull;
    Fd[2 * Npad + cell] = 0ull;
    return make_float3((float)((double)a * FIX_INV), (float)((double)b * FIX_INV), (float)((double)c * FIX_INV));
}

// One block per run of up to tile_x consecutive cells of one (y, z) row: the
// y/z neighbour rows are uniform across the block, so every population
// address is a block-uniform plane/row base plus a per-thread x offset.
template <int ST, bool ODD, int FORCING, bool DET>
__global__ void __launch_bounds__(LB_TPB, 3) k_lb_step(const DevCtx c) {
    using S = Store<ST>;
    using T = typename S::T;
    T *__restrict__ P = reinterpret_cast<T *>(c.pops);
    const unsigned tile = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    __shared__ int s_flag;
    if (threadIdx.x == 0) {
        int f = c.flags[tile];
        s_flag = f;
        if (f) c.flags[tile] = 0;
    }
    __syncthreads();
    const bool flagged = s_flag != 0;
    const bool forced = flagged || c.has_g;
    const unsigned nx = c.nx, ny = c.ny, nz = c.nz, nxy = nx * ny;
    const unsigned x = blockIdx.x * c.tile_x + threadIdx.x;
    const unsigned y = blockIdx.y, z = blockIdx.z;
    bool bad = false;
    if (threadIdx.x < (unsigned)c.tile_x && x < nx) {
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
        // moments of the deviations
        float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            drho += d[i];
            if (cx(i)) jx += cx(i) > 0 ? d[i] : -d[i];
            if (cy(i)) jy += cy(i) > 0 ? d[i] : -d[i];
            if (cz(i)) jz += cz(i) > 0 ? d[i] : -d[i];
        }
        float Fx = 0.f, Fy = 0.f, Fz = 0.f;
        if (forced) {
            if (flagged) {
                if (DET) {
                    float3 f = take_fdet(c.Fdet, c.Npad, cell);
                    Fx = f.x; Fy = f.y; Fz = f.z;
                } else {
                    float4 f = c.F[cell];
                    c.F[cell] = make_float4(0.f, 0.f, 0.f, 0.f);
                    Fx = f.x; Fy = f.y; Fz = f.z;
                }
            }
            Fx += c.g[0]; Fy += c.g[1]; Fz += c.g[2];
        }
        const float rho = c.rho0 + drho;
        const float irho = 1.0f / rho;
        const float ux = (jx + 0.5f * Fx) * irho, uy = (jy + 0.5f * Fy) * irho, uz = (jz + 0.5f * Fz) * irho;
        if (flagged) c.U[cell] = make_float4(ux, uy, uz, rho);
        bad = !isfinite(rho) || !isfinite(ux + uy + uz);
        float ex = ux, ey = uy, ez = uz;
        if (FORCING == LBIB_SHAN_CHEN) {
            ex = (jx + c.tau * Fx) * irho;
            ey = (jy + c.tau * Fy) * irho;
            ez = (jz + c.tau * Fz) * irho;
        }
        const float usq15 = 1.5f * (ex * ex + ey * ey + ez * ez);
        const float om = c.omega;
        const float gu = (FORCING == LBIB_GUO && forced) ? 1.0f - 0.5f * om : 0.f;
        const float uF = ux * Fx + uy * Fy + uz * Fz;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float cu = cx(i) * ex + cy(i) * ey + cz(i) * ez;
            const float deq = wgt(i) * (drho + rho * (3.0f * cu + 4.5f * cu * cu - usq15));
            float post = d[i] + om * (deq - d[i]);
            if (FORCING == LBIB_GUO && forced) {
                const float cF = cx(i) * Fx + cy(i) * Fy + cz(i) * Fz;
                post += gu * wgt(i) * (3.0f * (cF - uF) + 9.0f * cu * cF);
            }
            d[i] = post;
        }
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
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&c.ctl->err, ERR_NONFINITE);
    if (tile == 0 && threadIdx.x == 0) c.ctl->step += 1;
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

template <int ST, int FORCING>
static cudaError_t lb_step_dispatch(const DevCtx &c, bool odd, cudaStream_t s) {
    const dim3 blocks((unsigned)c.tiles_x, (unsigned)c.ny, (unsigned)c.nz);
    const unsigned threads = (unsigned)((c.tile_x + 31) / 32 * 32);
    if (c.deterministic) {
        if (odd) k_lb_step<ST, true, FORCING, true><<<blocks, threads, 0, s>>>(c);
        else k_lb_step<ST, false, FORCING, true><<<blocks, threads, 0, s>>>(c);
    } else {
        if (odd) k_lb_step<ST, true, FORCING, false><<<blocks, threads, 0, s>>>(c);
        else k_lb_step<ST, false, FORCING, false><<<blocks, threads, 0, s>>>(c);
    }
    return cudaGetLastError();
}

cudaError_t launch_lb_step(const DevCtx &c, int storage, int forcing, bool odd, cudaStream_t s) {
    if (forcing == LBIB_SHAN_CHEN) {
        if (storage == LBIB_F16) return lb_step_dispatch<LBIB_F16, LBIB_SHAN_CHEN>(c, odd, s);
        if (storage == LBIB_BF16) return lb_step_dispatch<LBIB_BF16, LBIB_SHAN_CHEN>(c, odd, s);
        return lb_step_dispatch<LBIB_F32, LBIB_SHAN_CHEN>(c, odd, s);
    }
    if (storage == LBIB_F16) return lb_step_dispatch<LBIB_F16, LBIB_GUO>(c, odd, s);
    if (storage == LBIB_BF16) return lb_step_dispatch<LBIB_BF16, LBIB_GUO>(c, odd, s);
    return lb_step_dispatch<LBIB_F32, LBIB_GUO>(c, odd, s);
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
