// Reverse-mode derivative of the coupled lattice-Boltzmann / immersed-
// boundary step (Sec. 2.1-2.3) for gradients of swimmer displacements with
// respect to the per-bead drive parameters (Sec. 2.2, driving-force equation).
//
// The engine keeps its own forward step on a plain layout so that every
// intermediate the reverse sweep needs is a stored array: per step k of a
// segment, slot k holds the populations f^k (shifted deviations, 19 planes),
// the force field F^k, the velocity u^k (3 planes each), node positions r^k,
// nodal forces f_j^k, bead centres R^k and the external bead forces.  Forward
// step k reads slot k and writes the populations, positions and a cleared
// force field of slot k + 1 (push streaming into a second array).  A
// checkpoint (populations + positions) is kept every K steps; the reverse
// sweep recomputes each segment from its checkpoint, then walks it backward.
//
// Forward step (the order the oracle and lb_step use):
//   R_b = mean_j r_j;  e_b = f^d_b(t) x + f^s_b(R)                (Sec. 2.2)
//   f_j = sum_triangles -dW/dr_j + e_b / N_b                        (Sec. 2.2)
//   F(x) = sum_j f_j Delta(x - r_j)                                 (Sec. 2.3)
//   rho, u = (sum f c + F/2)/rho; f* = f - (f - f^eq)/tau + Guo source; push (Sec. 2.1)
//   r_j += sum_x u(x) Delta(x - r_j)                                (Sec. 2.3)
// Reverse step, with adjoints lam_f (populations), lam_r (positions):
//   lam_U = lam_r;  lam_u(x) += Delta lam_U;  lam_r += grad_r <u, lam_U> Delta
//   per cell: lam*_i(x) = lam_f_i(x + c_i); the collision's Jacobian is
//     (1 - omega) I plus a rank-4 term through rho and rho u, so
//     lam_f_i = (1 - omega) lam*_i + lam_rho + c_i . lam_m, and lam_F
//   lam_fj = sum_x lam_F(x) Delta;  lam_r += grad_r <lam_F, f_j> Delta
//   lam_r += (d f_mem / d r) lam_f  (symmetric: minus the membrane Hessian)
//   lam_e_b = mean over the bead of lam_fj -> drive gradient, spring Jacobian
//     -> lam_R_b -> lam_r += lam_R_b / N_b
// Fluid arrays are FP32 or FP64 (template T); everything node-level is FP64.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <cooperative_groups.h>

#include "lbib_internal.cuh"

using namespace lbib;

namespace {

constexpr size_t AL = 256;
size_t up(size_t v) { return (v + AL - 1) / AL * AL; }

struct Dims {
    int nx, ny, nz;
    long long N, Npad;
};

// Structure tables (device pointers)
struct Mesh {
    int M, T, B, S;
    const int *tris;        // T x 3 node ids
    const double *G;        // T x 3 rest metric G00, G01, G11
    const double *A0Gs;     // T: rest area x shear modulus
    const double *iG;       // T: 1 / det G
    const int *csr_ptr;     // M + 1
    const int *csr_ent;     // 3T entries 3 t + q
    const int *node_bead;   // M
    const int *bead_start;  // B
    const int *bead_count;  // B
    const double *bead_inv; // B: 1 / node count
    const int *bead_swim;   // B
};

struct Swim {
    int bead[3];
    int balance;
    double k, L, period;
};

__device__ __forceinline__ int wrapi(long long a, int n) {
    long long r = a % n;
    return (int)(r < 0 ? r + n : r);
}

// Peskin's 4-point weight of stencil cell q (of floor(p) - 1 .. floor(p) + 2)
// at fractional offset f, and its derivative with respect to p: with
// s = sqrt(1 + 4f - 4f^2) the weights are (3 - 2f - s)/8, (3 - 2f + s)/8,
// (1 + 2f + s)/8, (1 + 2f - s)/8, and ds/df = (2 - 4f)/s.  W is the
// precision of the weights (that of the fluid state).
template <typename W>
__device__ __forceinline__ void peskin_q(W f, W s, W ds, int q, W &w, W &dw) {
    const W A = q < 2 ? (W)3 - (W)2 * f : (W)1 + (W)2 * f, dA = q < 2 ? (W)-2 : (W)2;
    const W sg = (q == 1 || q == 2) ? (W)1 : (W)-1;
    w = (A + sg * s) * (W)0.125;
    dw = (dA + sg * ds) * (W)0.125;
}

// The two stencil cells of a lane (numbers lane and lane + 32 of the 64,
// x fastest: they differ in z only), their weights Delta(x - r) and
// gradients d Delta / d r.  The fractional offsets are taken in FP64 from
// the FP64 positions.
template <typename W>
__device__ __forceinline__ void lane_cells(const Dims &d, const double *r, int lane, int cell[2], W w[2],
                                           W g[2][3]) {
    const int qx = lane & 3, qy = (lane >> 2) & 3, qz = lane >> 4;
    const double fx = floor(r[0]), fy = floor(r[1]), fz = floor(r[2]);
    const W ax = (W)(r[0] - fx), ay = (W)(r[1] - fy), az = (W)(r[2] - fz);
    const W sx = sqrt((W)1 + (W)4 * ax - (W)4 * ax * ax), sy = sqrt((W)1 + (W)4 * ay - (W)4 * ay * ay),
            sz = sqrt((W)1 + (W)4 * az - (W)4 * az * az);
    W wx, dx, wy, dy;
    peskin_q<W>(ax, sx, ((W)2 - (W)4 * ax) / sx, qx, wx, dx);
    peskin_q<W>(ay, sy, ((W)2 - (W)4 * ay) / sy, qy, wy, dy);
    const int X = wrapi((long long)fx - 1 + qx, d.nx), Y = wrapi((long long)fy - 1 + qy, d.ny);
    const W dsz = ((W)2 - (W)4 * az) / sz;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        W wz, dz;
        peskin_q<W>(az, sz, dsz, qz + 2 * h, wz, dz);
        const int Z = wrapi((long long)fz - 1 + qz + 2 * h, d.nz);
        cell[h] = X + d.nx * (Y + d.ny * Z);
        w[h] = wx * wy * wz;
        g[h][0] = dx * wy * wz;
        g[h][1] = wx * dy * wz;
        g[h][2] = wx * wy * dz;
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of three doubles over each 256-thread group of a 768-thread block (one
// group per bead of a swimmer); the group's sum is written to out[group].
__device__ __forceinline__ void group_sum3(double v[3], double (*sh)[3], double (*out)[3]) {
    for (int a = 0; a < 3; ++a) v[a] = warp_sum(v[a]);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
        for (int a = 0; a < 3; ++a) sh[w][a] = v[a];
    __syncthreads();
    if (threadIdx.x < 3 * 32) {  // warp q adds the 8 warp sums of group q
        const int q = threadIdx.x >> 5;
        for (int a = 0; a < 3; ++a) {
            double x = l < 8 ? sh[8 * q + l][a] : 0.0;
            x = warp_sum(x);
            if (l == 0) out[q][a] = x;
        }
    }
    __syncthreads();
}

constexpr int SWIM_THREADS = 768;  // three groups of 256: one per bead
constexpr int BEAD_THREADS = 256;  // one block of a swimmer's three-block cluster: one bead
constexpr int TRI_THREADS = 32;    // per-triangle FP64 kernels: one warp per block

// The same fixed-order sum as one 256-thread group of group_sum3: warp sums,
// then warp 0 adds the 8 warp sums in order.  Result in out[3].
__device__ __forceinline__ void bead_sum3(double v[3], double (*sh)[3], double *out) {
    for (int a = 0; a < 3; ++a) v[a] = warp_sum(v[a]);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
        for (int a = 0; a < 3; ++a) sh[w][a] = v[a];
    __syncthreads();
    if (threadIdx.x < 32) {
        for (int a = 0; a < 3; ++a) {
            double x = l < 8 ? sh[l][a] : 0.0;
            x = warp_sum(x);
            if (l == 0) out[a] = x;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- membrane
// Neo-Hookean linear FEM triangle (Sec. 2.2): with edge vectors d = [d1 d2],
// rest metric G, E = (d^T d - G)/2 (FP64, small near rest),
// I2 = 2 tr(G^-1 E) + 4 det E / det G, J^4 = (1 + I2)^2:
//   dW/dd = s d M,  s = A0 Gs / (det G J^4),
//   M = (J^4 - 1) adj G - 2 adj E,  adj [[a, b], [b, c]] = [[c, -b], [-b, a]],
// and the corner forces are f1 = -P[:,0], f2 = -P[:,1], f0 = P[:,0] + P[:,1].
// FP64 runs at 1/64 of the FP32 rate here and one warp per SM carries these
// kernels, so every FP64 divide is a long serial sequence: 1 / det G comes
// precomputed per triangle and 1 / J^4 is formed once.
struct TriState {
    double d1[3], d2[3];
    double E00, E01, E11, iG, I2, J2, iJ4, s, M00, M01, M11;
};

__device__ __forceinline__ void tri_state(const double *G, double iG, double A0Gs, const double *x0, const double *x1,
                                          const double *x2, TriState &S) {
    for (int a = 0; a < 3; ++a) {
        S.d1[a] = x1[a] - x0[a];
        S.d2[a] = x2[a] - x0[a];
    }
    const double g00 = S.d1[0] * S.d1[0] + S.d1[1] * S.d1[1] + S.d1[2] * S.d1[2];
    const double g01 = S.d1[0] * S.d2[0] + S.d1[1] * S.d2[1] + S.d1[2] * S.d2[2];
    const double g11 = S.d2[0] * S.d2[0] + S.d2[1] * S.d2[1] + S.d2[2] * S.d2[2];
    S.E00 = 0.5 * (g00 - G[0]);
    S.E01 = 0.5 * (g01 - G[1]);
    S.E11 = 0.5 * (g11 - G[2]);
    S.iG = iG;
    const double trGiE = (G[2] * S.E00 - 2.0 * G[1] * S.E01 + G[0] * S.E11) * iG;
    const double detE = S.E00 * S.E11 - S.E01 * S.E01;
    S.I2 = 2.0 * trGiE + 4.0 * detE * iG;
    S.J2 = 1.0 + S.I2;
    S.iJ4 = 1.0 / (S.J2 * S.J2);
    S.s = A0Gs * iG * S.iJ4;
    const double c = S.I2 * (S.I2 + 2.0);  // J^4 - 1
    S.M00 = c * G[2] - 2.0 * S.E11;
    S.M01 = -c * G[1] + 2.0 * S.E01;
    S.M11 = c * G[0] - 2.0 * S.E00;
}

// directional derivative of the corner forces along node displacements
// v0, v1, v2 (the force Jacobian is minus the energy Hessian: symmetric, so
// this is also the transposed product the reverse sweep needs)
__device__ __forceinline__ void tri_force_jvp(const double *G, const TriState &S, const double *v0, const double *v1,
                                              const double *v2, double df[3][3]) {
    double e1[3], e2[3];
    for (int a = 0; a < 3; ++a) {
        e1[a] = v1[a] - v0[a];
        e2[a] = v2[a] - v0[a];
    }
    const double dE00 = S.d1[0] * e1[0] + S.d1[1] * e1[1] + S.d1[2] * e1[2];
    const double dE11 = S.d2[0] * e2[0] + S.d2[1] * e2[1] + S.d2[2] * e2[2];
    const double dE01 = 0.5 * (S.d1[0] * e2[0] + S.d1[1] * e2[1] + S.d1[2] * e2[2] + e1[0] * S.d2[0] +
                               e1[1] * S.d2[1] + e1[2] * S.d2[2]);
    const double dtr = (G[2] * dE00 - 2.0 * G[1] * dE01 + G[0] * dE11) * S.iG;
    const double ddetE = dE00 * S.E11 + S.E00 * dE11 - 2.0 * S.E01 * dE01;
    const double dI2 = 2.0 * dtr + 4.0 * ddetE * S.iG;
    const double dJ4 = 2.0 * S.J2 * dI2;
    const double ds = -S.s * dJ4 * S.iJ4;
    const double dM00 = dJ4 * G[2] - 2.0 * dE11;
    const double dM01 = -dJ4 * G[1] + 2.0 * dE01;
    const double dM11 = dJ4 * G[0] - 2.0 * dE00;
    for (int a = 0; a < 3; ++a) {
        const double P0 = S.d1[a] * S.M00 + S.d2[a] * S.M01;
        const double P1 = S.d1[a] * S.M01 + S.d2[a] * S.M11;
        const double dP0 = ds * P0 + S.s * (e1[a] * S.M00 + e2[a] * S.M01 + S.d1[a] * dM00 + S.d2[a] * dM01);
        const double dP1 = ds * P1 + S.s * (e1[a] * S.M01 + e2[a] * S.M11 + S.d1[a] * dM01 + S.d2[a] * dM11);
        df[0][a] = dP0 + dP1;
        df[1][a] = -dP0;
        df[2][a] = -dP1;
    }
}

// ---------------------------------------------------------------- forward kernels

// sin and cos of the drive phases omega t + phi_q (Sec. 2.2, driving-force
// equation) for every step t of the run, swimmer and bead: one thread each,
// once per forward sweep, so the per-step swimmer kernels only look them up
__global__ void k_drive_table(const Swim *sw, const double *theta, long long n_steps, int S, double *tbl) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n_steps * S * 3) return;
    const int q = (int)(i % 3), s = (int)((i / 3) % S);
    const long long n = i / (3 * S);
    const double om = 2.0 * 3.14159265358979323846 / sw[s].period;
    const double arg = om * (double)n + theta[6 * s + 3 + q];
    double *o = tbl + (n * S + s) * 6;
    o[q] = sin(arg);
    o[3 + q] = cos(arg);
}

// one cluster of three blocks per swimmer, block q summing the positions of
// bead q (FP64, fixed order); block 0 reads the three centres from the
// blocks' shared memory (distributed shared memory) and evaluates the drive
// and spring forces (thread 0)
__global__ void __cluster_dims__(3, 1, 1) __launch_bounds__(BEAD_THREADS)
    k_fwd_swimmer(Mesh m, const Swim *sw, const double *theta, const double *drv, const double *r,
                  const long long *t_base, int k, double *R, double *ext) {
    namespace cg = cooperative_groups;
    __shared__ double sh[BEAD_THREADS / 32][3];
    __shared__ double Rq[3];
    cg::cluster_group cl = cg::this_cluster();
    const int s = blockIdx.x / 3, q = (int)cl.block_rank();
    const Swim w = sw[s];
    {
        const int b = w.bead[q], n0 = m.bead_start[b], nn = m.bead_count[b];
        double acc[3] = {0.0, 0.0, 0.0};
        for (int j = n0 + threadIdx.x; j < n0 + nn; j += BEAD_THREADS)
            for (int a = 0; a < 3; ++a) acc[a] += r[3 * j + a];
        bead_sum3(acc, sh, Rq);
        if (threadIdx.x < 3) {
            Rq[threadIdx.x] *= m.bead_inv[b];
            R[3 * b + threadIdx.x] = Rq[threadIdx.x];
        }
    }
    cl.sync();
    if (q == 0 && threadIdx.x < 32) {
        // warp 0 of block 0: the two springs on lanes 0 and 1 (side q = 0, 2)
        const int l = threadIdx.x;
        double Rs[3][3];
        for (int qq = 0; qq < 3; ++qq) {
            const double *p = cl.map_shared_rank(Rq, qq);
            for (int a = 0; a < 3; ++a) Rs[qq][a] = p[a];
        }
        const double *th = theta + 6 * s;
        const double *dv = drv + ((*t_base + k) * (long long)(gridDim.x / 3) + s) * 6;
        double fd[3];
        fd[0] = th[0] * dv[0];
        fd[2] = th[2] * dv[2];
        fd[1] = w.balance ? -fd[0] - fd[2] : th[1] * dv[1];
        const int qs = l ? 2 : 0;
        double dd[3], n2 = 0.0, fq[3];
        for (int a = 0; a < 3; ++a) {
            dd[a] = Rs[qs][a] - Rs[1][a];
            n2 += dd[a] * dd[a];
        }
        const double n = sqrt(n2), h = -w.k * (n - w.L) / n;
        for (int a = 0; a < 3; ++a) fq[a] = h * dd[a];
        double fs[3][3];
        for (int a = 0; a < 3; ++a) {
            fs[0][a] = __shfl_sync(0xffffffffu, fq[a], 0);
            fs[2][a] = __shfl_sync(0xffffffffu, fq[a], 1);
            fs[1][a] = -fs[0][a] - fs[2][a];
        }
        if (l < 9) {
            const int qq = l / 3, a = l % 3;
            ext[3 * w.bead[qq] + a] = fs[qq][a] + (a == 0 ? fd[qq] : 0.0);
        }
    }
    cl.sync();  // the blocks' shared memory outlives block 0's reads
}

// one thread per triangle: corner forces -dW/dr
__global__ void k_fwd_tri(Mesh m, const double *r, double *tri_f) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.T) return;
    const int *v = m.tris + 3 * t;
    TriState S;
    tri_state(m.G + 3 * t, m.iG[t], m.A0Gs[t], r + 3 * v[0], r + 3 * v[1], r + 3 * v[2], S);
    for (int a = 0; a < 3; ++a) {
        const double P0 = S.s * (S.d1[a] * S.M00 + S.d2[a] * S.M01);
        const double P1 = S.s * (S.d1[a] * S.M01 + S.d2[a] * S.M11);
        tri_f[9 * t + a] = P0 + P1;
        tri_f[9 * t + 3 + a] = -P0;
        tri_f[9 * t + 6 + a] = -P1;
    }
}

// one warp per node: f_j = sum of its corner forces + e_b / N_b (lanes gather
// the corners, fixed order), recorded, then F(x) += f_j Delta(x - r_j)
template <typename T>
__global__ void k_fwd_spread(Dims d, Mesh m, const double *r, const double *tri_f, const double *ext, double *fn,
                             T *F, int *rowtag, int *rlist, int *rcnt, const long long *tb, int k) {
    const int j = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (j >= m.M) return;
    const int e0 = m.csr_ptr[j], e1 = m.csr_ptr[j + 1];
    double f[3] = {0.0, 0.0, 0.0};
    for (int e = e0 + lane; e < e1; e += 32) {
        const int k = m.csr_ent[e];
        for (int a = 0; a < 3; ++a) f[a] += tri_f[3 * k + a];
    }
    const int b = m.node_bead[j];
    const double inv = m.bead_inv[b];
    for (int a = 0; a < 3; ++a) f[a] = warp_sum(f[a]) + ext[3 * b + a] * inv;
    if (lane == 0)
        for (int a = 0; a < 3; ++a) fn[3 * j + a] = f[a];
    int cell[2];
    T w[2], g[2][3];
    lane_cells<T>(d, r + 3 * j, lane, cell, w, g);
    // tag the rows (y, z) of the stencil cells with the step (absolute index
    // + 1) and list each row once (the lane that changes its tag): both fluid
    // updates of this step treat them apart from the rest of the box.  The
    // tags of a slot set are cleared before it is recorded again.
    const int tag = (int)(*tb + k + 1);
    for (int h = 0; h < 2; ++h) {
        atomicAdd(F + cell[h], (T)f[0] * w[h]);
        atomicAdd(F + d.Npad + cell[h], (T)f[1] * w[h]);
        atomicAdd(F + 2 * d.Npad + cell[h], (T)f[2] * w[h]);
        if ((lane & 3) == 0) {  // one lane per stencil row
            const int row = cell[h] / d.nx;
            if (rowtag[row] != tag && atomicExch(rowtag + row, tag) != tag) rlist[atomicAdd(rcnt, 1)] = row;
        }
    }
}

// zero the row tags and row counts of the n_slots slots of a slot set
__global__ void k_clear_rows(char *slot0, size_t slot_bytes, size_t off_tags, size_t off_count, int nrow,
                             int n_slots) {
    const long long n = (long long)n_slots * nrow;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int sl = (int)(i / nrow), r = (int)(i - (long long)sl * nrow);
        char *base = slot0 + (size_t)sl * slot_bytes;
        reinterpret_cast<int *>(base + off_tags)[r] = 0;
        if (r == 0) *reinterpret_cast<int *>(base + off_count) = 0;
    }
}

// per-cell moments of the shifted deviations: drho = sum d, m = sum d c
template <typename T>
__device__ __forceinline__ void moments(const T *dv, T &drho, T m[3]) {
    drho = 0;
    m[0] = m[1] = m[2] = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += dv[i];
        if (cx(i)) m[0] += cx(i) > 0 ? dv[i] : -dv[i];
        if (cy(i)) m[1] += cy(i) > 0 ? dv[i] : -dv[i];
        if (cz(i)) m[2] += cz(i) > 0 ? dv[i] : -dv[i];
    }
}

// cell = x + nx (y + ny z) < 2^31
__device__ __forceinline__ void cell_xyz(const Dims &d, int cell, int &x, int &y, int &z) {
    const int yz = cell / d.nx;
    x = cell - yz * d.nx;
    z = yz / d.ny;
    y = yz - z * d.ny;
}

// Offsets from a cell to its periodic neighbours along +-x, +-y, +-z.
struct Nbr {
    int xp, xm, yp, ym, zp, zm;
    __device__ __forceinline__ Nbr(const Dims &d, int x, int y, int z) {
        const int sy = d.nx, sz = d.nx * d.ny;
        xp = x == d.nx - 1 ? 1 - d.nx : 1;
        xm = x == 0 ? d.nx - 1 : -1;
        yp = y == d.ny - 1 ? (1 - d.ny) * sy : sy;
        ym = y == 0 ? (d.ny - 1) * sy : -sy;
        zp = z == d.nz - 1 ? (1 - d.nz) * sz : sz;
        zm = z == 0 ? (d.nz - 1) * sz : -sz;
    }
    // offset of the neighbour at x + c_i
    __device__ __forceinline__ int off(int i) const {
        return (cx(i) > 0 ? xp : cx(i) < 0 ? xm : 0) + (cy(i) > 0 ? yp : cy(i) < 0 ? ym : 0) +
               (cz(i) > 0 ? zp : cz(i) < 0 ? zm : 0);
    }
};

// BGK collision with Guo forcing (Sec. 2.1, Eq. lbe) of one cell's shifted
// deviations dv: post-collision values (before streaming) and the physical
// velocity u.  Opposite directions i, i+1 (c_{i+1} = -c_i) share the even and
// odd parts of the equilibrium and of the source term.
template <typename T>
__device__ __forceinline__ void fwd_cell(const T (&dv)[Q], T Fx, T Fy, T Fz, T omega, T rho0, T (&post)[Q], T (&u)[3]) {
    T drho, m[3];
    moments(dv, drho, m);
    const T rho = rho0 + drho;
    const T ux = (m[0] + (T)0.5 * Fx) / rho, uy = (m[1] + (T)0.5 * Fy) / rho, uz = (m[2] + (T)0.5 * Fz) / rho;
    const T uu = ux * ux + uy * uy + uz * uz, uF = ux * Fx + uy * Fy + uz * Fz;
    const T src = (T)1 - (T)0.5 * omega, keep = (T)1 - omega;
    {
        const T w = (T)wgt_d(0);
        post[0] = keep * dv[0] + omega * w * (drho - rho * (T)1.5 * uu) + src * w * ((T)-3 * uF);
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const T cu = (T)cx(i) * ux + (T)cy(i) * uy + (T)cz(i) * uz;
        const T cF = (T)cx(i) * Fx + (T)cy(i) * Fy + (T)cz(i) * Fz;
        const T w = (T)wgt_d(i);
        const T eq_e = w * (drho + rho * ((T)4.5 * cu * cu - (T)1.5 * uu)), eq_o = w * rho * (T)3 * cu;
        const T S_e = w * ((T)9 * cu * cF - (T)3 * uF), S_o = w * (T)3 * cF;
        const T e = omega * eq_e + src * S_e, o = omega * eq_o + src * S_o;
        post[i] = keep * dv[i] + e + o;
        post[i + 1] = keep * dv[i + 1] + e - o;
    }
    u[0] = ux;
    u[1] = uy;
    u[2] = uz;
}

// one thread per cell: collide, push into the next slot, the velocity u^k, and
// a cleared force field of the next slot
template <typename T>
__global__ void __launch_bounds__(256, 2) k_fwd_lb(Dims d, T omega, T rho0, double gx, double gy,
                                                                       double gz, const T *pops, const T *F, T *out,
                                                                       T *u_out, T *F_next) {
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= d.N) return;
    int x, y, z;
    cell_xyz(d, cell, x, y, z);
    const Nbr nb(d, x, y, z);
    T dv[Q], post[Q], u[3];
#pragma unroll
    for (int i = 0; i < Q; ++i) dv[i] = pops[i * d.Npad + cell];
    fwd_cell(dv, F[cell] + (T)gx, F[d.Npad + cell] + (T)gy, F[2 * d.Npad + cell] + (T)gz, omega, rho0, post, u);
#pragma unroll
    for (int i = 0; i < Q; ++i) out[i * d.Npad + cell + nb.off(i)] = post[i];
    for (int a = 0; a < 3; ++a) {
        u_out[a * d.Npad + cell] = u[a];
        F_next[a * d.Npad + cell] = 0;
    }
}

// FP32, rows of even length: two adjacent cells per thread, with 8-byte
// vector loads and stores wherever both cells' values stay adjacent (every
// load, and the stores of directions with c_x = 0)
__global__ void __launch_bounds__(128, 4) k_fwd_lb2(Dims d, float omega, float rho0, double gx, double gy, double gz,
                                                    const float *pops, const float *F, float *out, float *u_out,
                                                    float *F_next) {
    const int cell = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (cell >= d.N) return;
    int x, y, z;
    cell_xyz(d, cell, x, y, z);
    const Nbr n0(d, x, y, z), n1(d, x + 1, y, z);
    float dv0[Q], dv1[Q], p0[Q], p1[Q], u0[3], u1[3];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float2 v = *reinterpret_cast<const float2 *>(pops + i * d.Npad + cell);
        dv0[i] = v.x;
        dv1[i] = v.y;
    }
    float2 Fv[3];
    for (int a = 0; a < 3; ++a) Fv[a] = *reinterpret_cast<const float2 *>(F + a * d.Npad + cell);
    fwd_cell(dv0, Fv[0].x + (float)gx, Fv[1].x + (float)gy, Fv[2].x + (float)gz, omega, rho0, p0, u0);
    fwd_cell(dv1, Fv[0].y + (float)gx, Fv[1].y + (float)gy, Fv[2].y + (float)gz, omega, rho0, p1, u1);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float *pl = out + i * d.Npad;
        if (cx(i) == 0) {
            *reinterpret_cast<float2 *>(pl + cell + n0.off(i)) = make_float2(p0[i], p1[i]);
        } else {
            pl[cell + n0.off(i)] = p0[i];
            pl[cell + 1 + n1.off(i)] = p1[i];
        }
    }
    for (int a = 0; a < 3; ++a) {
        *reinterpret_cast<float2 *>(u_out + a * d.Npad + cell) = make_float2(u0[a], u1[a]);
        *reinterpret_cast<float2 *>(F_next + a * d.Npad + cell) = make_float2(0.f, 0.f);
    }
}

// one warp per node: r_j^{k+1} = r_j^k + sum_x u(x) Delta(x - r_j)
// The forward record update by rows (y, z), as the reverse one: NEAR launches
// update the rows under the step's node stencils (tagged by the spreading of
// this step), reading F and writing the velocity the interpolation needs; the
// others update the rest of the box, where F is the uniform body force and
// the velocity is not needed.  Both push into the next slot and clear its
// force field.
template <typename T, bool NEAR, bool PAIR>
__global__ void __launch_bounds__(128) k_fwd_lb_rows(Dims d, T omega, T rho0, double gx, double gy, double gz,
                                                     const T *pops, const T *F, T *out, T *u_out, T *F_next,
                                                     const int *rowtag, const int *rlist, const int *rcnt,
                                                     const long long *tb, int k) {
    // NEAR: the rows the spreading listed, grid-stride; otherwise one block
    // per row, skipping the tagged ones
    const int tag = (int)(*tb + k + 1);
    const int n_it = NEAR ? *rcnt : 1;
    constexpr int CPT = PAIR ? 2 : 1;
    const T G[3] = {(T)gx, (T)gy, (T)gz};  // converted once, not per cell (FP64 converts issue slowly here)
    for (int it = NEAR ? (int)blockIdx.x : 0; it < n_it; it += NEAR ? (int)gridDim.x : 1) {
        const int row = NEAR ? rlist[it] : (int)blockIdx.x;
        if (!NEAR && rowtag[row] == tag) return;
        const int y = row % d.ny, z = row / d.ny;
        for (int x = CPT * threadIdx.x; x < d.nx; x += CPT * blockDim.x) {
            const int cell = x + d.nx * row;
            T dv[CPT][Q], p[CPT][Q], u[CPT][3];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if constexpr (PAIR) {
                    const float2 v = *reinterpret_cast<const float2 *>(pops + i * d.Npad + cell);
                    dv[0][i] = v.x;
                    dv[1][i] = v.y;
                } else {
                    dv[0][i] = pops[i * d.Npad + cell];
                }
            }
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                T Fv[3] = {G[0], G[1], G[2]};
                if constexpr (NEAR)
                    for (int a = 0; a < 3; ++a) Fv[a] += F[a * d.Npad + cell + c];
                fwd_cell(dv[c], Fv[0], Fv[1], Fv[2], omega, rho0, p[c], u[c]);
            }
            const Nbr n0(d, x, y, z);
            if constexpr (PAIR) {
                const Nbr n1(d, x + 1, y, z);
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    float *pl = out + i * d.Npad;
                    if (cx(i) == 0) {
                        *reinterpret_cast<float2 *>(pl + cell + n0.off(i)) = make_float2(p[0][i], p[1][i]);
                    } else {
                        pl[cell + n0.off(i)] = p[0][i];
                        pl[cell + 1 + n1.off(i)] = p[1][i];
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < Q; ++i) out[i * d.Npad + cell + n0.off(i)] = p[0][i];
            }
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < CPT; ++c) {
                    if constexpr (NEAR) u_out[a * d.Npad + cell + c] = u[c][a];
                    F_next[a * d.Npad + cell + c] = (T)0;
                }
        }
    }
}

template <typename T>
__global__ void k_fwd_interp(Dims d, int M, const double *r, const T *u, double *r_next, int *err) {
    const int j = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (j >= M) return;
    int cell[2];
    T w[2], g[2][3];
    lane_cells<T>(d, r + 3 * j, lane, cell, w, g);
    double U[3] = {0.0, 0.0, 0.0};
    for (int h = 0; h < 2; ++h)
        for (int a = 0; a < 3; ++a) U[a] += (double)(w[h] * u[a * d.Npad + cell[h]]);
    for (int a = 0; a < 3; ++a) U[a] = warp_sum(U[a]);
    if (lane == 0) {
        bool bad = false, fast = false;
        for (int a = 0; a < 3; ++a) {
            r_next[3 * j + a] = r[3 * j + a] + U[a];
            bad |= !isfinite(U[a]);
            fast |= fabs(U[a]) > 0.1;
        }
        if (bad) atomicOr(err, ERR_NONFINITE);
        else if (fast) atomicOr(err, ERR_UNSTABLE);
    }
}

// one block per swimmer (a group per bead): disp_s = x_cm(final) - x_cm(initial)
__global__ void __launch_bounds__(SWIM_THREADS) k_disp(Mesh m, const Swim *sw, const double *rf, const double *ri,
                                                       double *disp) {
    __shared__ double sh[SWIM_THREADS / 32][3];
    __shared__ double tot[3][3];
    const int s = blockIdx.x, q = threadIdx.x >> 8, tq = threadIdx.x & 255;
    const int b = sw[s].bead[q], n0 = m.bead_start[b], nn = m.bead_count[b];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int j = n0 + tq; j < n0 + nn; j += 256)
        for (int a = 0; a < 3; ++a) acc[a] += rf[3 * j + a] - ri[3 * j + a];
    group_sum3(acc, sh, tot);
    if (threadIdx.x < 3) {
        const int a = threadIdx.x;
        double x = 0.0;
        for (int qq = 0; qq < 3; ++qq) x += tot[qq][a] / m.bead_count[sw[s].bead[qq]];
        disp[3 * s + a] = x / 3.0;
    }
}

// ---------------------------------------------------------------- reverse kernels

// lam_r_j (+)= sign * seed_s / (3 N_b): the derivative of x_cm of swimmer s
// (mean of its three bead centres, each the mean of N_b nodes)
__global__ void k_adj_seed(Mesh m, const double *seed_disp, double sign, int add, double *lam_r) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m.M) return;
    const int b = m.node_bead[j], s = m.bead_swim[b];
    const double f = sign / (3.0 * m.bead_count[b]);
    for (int a = 0; a < 3; ++a) {
        const double v = f * seed_disp[3 * s + a];
        lam_r[3 * j + a] = add ? lam_r[3 * j + a] + v : v;
    }
}

// one warp per node: transpose of r^{k+1} = r^k + interp(u^k, r^k)
template <typename T>
__global__ void k_adj_interp(Dims d, int M, const double *r, const T *u, double *lam_r, T *lam_u) {
    const int j = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (j >= M) return;
    int cell[2];
    T w[2], g[2][3];
    lane_cells<T>(d, r + 3 * j, lane, cell, w, g);
    const double L0 = lam_r[3 * j], L1 = lam_r[3 * j + 1], L2 = lam_r[3 * j + 2];
    double G[3] = {0.0, 0.0, 0.0};
    for (int h = 0; h < 2; ++h) {
        const double u0 = (double)u[cell[h]], u1 = (double)u[d.Npad + cell[h]], u2 = (double)u[2 * d.Npad + cell[h]];
        atomicAdd(lam_u + cell[h], w[h] * (T)L0);
        atomicAdd(lam_u + d.Npad + cell[h], w[h] * (T)L1);
        atomicAdd(lam_u + 2 * d.Npad + cell[h], w[h] * (T)L2);
        const double dot = L0 * u0 + L1 * u1 + L2 * u2;
        for (int a = 0; a < 3; ++a) G[a] += dot * (double)g[h][a];
    }
    for (int a = 0; a < 3; ++a) G[a] = warp_sum(G[a]);
    if (lane == 0)
        for (int a = 0; a < 3; ++a) lam_r[3 * j + a] += G[a];
}

// Transpose of one cell's collision (+ the velocity output).  With the pulled
// adjoints lam*_i and s0 = sum w l, s1 = sum w l c, s2 = sum w l c c (over
// opposite pairs: even parts l_i + l_{i+1} feed s0 and s2, odd parts
// l_i - l_{i+1} feed s1):
//   P = s0 (1 - 3/2 u.u) + 3 s1.u + 9/2 u.s2.u,  Q = 3 s1 - 3 s0 u + 9 s2 u,
//   a_u = omega rho Q + (1 - omega/2)(9 s2 F - 3 s0 F) + lam_u,
//   lam_F = (1 - omega/2) Q + a_u / (2 rho),  lam_m = a_u / rho,
//   lam_rho = omega P - a_u.u / rho,
//   lam_i = (1 - omega) lam*_i + lam_rho + c_i . lam_m.
template <typename T>
__device__ __forceinline__ void adj_cell(const T (&ls)[Q], const T (&dv)[Q], const T (&Fv)[3], const T (&lu)[3], T omega,
                                         T rho0, T (&lam)[Q], T (&lF)[3]) {
    T drho, m[3];
    moments(dv, drho, m);
    const T rho = rho0 + drho, ir = (T)1 / rho;
    const T u[3] = {(m[0] + (T)0.5 * Fv[0]) * ir, (m[1] + (T)0.5 * Fv[1]) * ir, (m[2] + (T)0.5 * Fv[2]) * ir};
    T s0 = (T)wgt_d(0) * ls[0], s1[3] = {0, 0, 0}, s2[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const T w = (T)wgt_d(i);
        const T ev = w * (ls[i] + ls[i + 1]), od = w * (ls[i] - ls[i + 1]);
        const int c[3] = {cx(i), cy(i), cz(i)};
        s0 += ev;
        for (int a = 0; a < 3; ++a) {
            if (c[a]) s1[a] += c[a] > 0 ? od : -od;
            for (int b = a; b < 3; ++b)
                if (c[a] && c[b]) s2[a][b] += c[a] * c[b] > 0 ? ev : -ev;
        }
    }
    s2[1][0] = s2[0][1];
    s2[2][0] = s2[0][2];
    s2[2][1] = s2[1][2];
    const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    T s2u[3], s2F[3], Pq = s0 * ((T)1 - (T)1.5 * uu);
    for (int a = 0; a < 3; ++a) {
        s2u[a] = s2[a][0] * u[0] + s2[a][1] * u[1] + s2[a][2] * u[2];
        s2F[a] = s2[a][0] * Fv[0] + s2[a][1] * Fv[1] + s2[a][2] * Fv[2];
        Pq += (T)3 * s1[a] * u[a] + (T)4.5 * u[a] * s2u[a];
    }
    const T src = (T)1 - (T)0.5 * omega, keep = (T)1 - omega;
    T lm[3], au_u = 0;
    for (int a = 0; a < 3; ++a) {
        const T Qa = (T)3 * s1[a] - (T)3 * s0 * u[a] + (T)9 * s2u[a];
        const T au = omega * rho * Qa + src * ((T)9 * s2F[a] - (T)3 * s0 * Fv[a]) + lu[a];
        lF[a] = src * Qa + (T)0.5 * au * ir;
        lm[a] = au * ir;
        au_u += au * u[a];
    }
    const T lrho = omega * Pq - au_u * ir;
    lam[0] = keep * ls[0] + lrho;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const T cm = (T)cx(i) * lm[0] + (T)cy(i) * lm[1] + (T)cz(i) * lm[2];
        lam[i] = keep * ls[i] + lrho + cm;
        lam[i + 1] = keep * ls[i + 1] + lrho - cm;
    }
}

// one thread per cell: pull lam*_i(x) = lam_i^{n+1}(x + c_i) (the transpose
// of the push), transpose the collision, clear lam_u
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_adj_lb(Dims d, T omega, T rho0, double gx, double gy,
                                                                       double gz, const T *pops, const T *F,
                                                                       const T *lam_next, T *lam_u, T *lam_cur,
                                                                       T *lam_F) {
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= d.N) return;
    int x, y, z;
    cell_xyz(d, cell, x, y, z);
    const Nbr nb(d, x, y, z);
    T ls[Q], dv[Q], lam[Q], lF[3];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        ls[i] = lam_next[i * d.Npad + cell + nb.off(i)];
        dv[i] = pops[i * d.Npad + cell];
    }
    const T Fv[3] = {F[cell] + (T)gx, F[d.Npad + cell] + (T)gy, F[2 * d.Npad + cell] + (T)gz};
    const T lu[3] = {lam_u[cell], lam_u[d.Npad + cell], lam_u[2 * d.Npad + cell]};
    adj_cell(ls, dv, Fv, lu, omega, rho0, lam, lF);
#pragma unroll
    for (int i = 0; i < Q; ++i) lam_cur[i * d.Npad + cell] = lam[i];
    for (int a = 0; a < 3; ++a) {
        lam_F[a * d.Npad + cell] = lF[a];
        lam_u[a * d.Npad + cell] = 0;
    }
}

// FP32, rows of even length: two adjacent cells per thread with 8-byte
// vector loads and stores wherever both cells' values stay adjacent (every
// access except the pulled adjoints of directions with c_x != 0)
__global__ void __launch_bounds__(128, 4) k_adj_lb2(Dims d, float omega, float rho0, double gx, double gy, double gz,
                                                    const float *pops, const float *F, const float *lam_next,
                                                    float *lam_u, float *lam_cur, float *lam_F) {
    const int cell = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (cell >= d.N) return;
    int x, y, z;
    cell_xyz(d, cell, x, y, z);
    const Nbr n0(d, x, y, z), n1(d, x + 1, y, z);
    float ls0[Q], ls1[Q], dv0[Q], dv1[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float *pl = lam_next + i * d.Npad;
        if (cx(i) == 0) {
            const float2 v = *reinterpret_cast<const float2 *>(pl + cell + n0.off(i));
            ls0[i] = v.x;
            ls1[i] = v.y;
        } else {
            ls0[i] = pl[cell + n0.off(i)];
            ls1[i] = pl[cell + 1 + n1.off(i)];
        }
        const float2 v = *reinterpret_cast<const float2 *>(pops + i * d.Npad + cell);
        dv0[i] = v.x;
        dv1[i] = v.y;
    }
    float2 Fv[3], lu[3];
    for (int a = 0; a < 3; ++a) {
        Fv[a] = *reinterpret_cast<const float2 *>(F + a * d.Npad + cell);
        lu[a] = *reinterpret_cast<const float2 *>(lam_u + a * d.Npad + cell);
    }
    float lam0[Q], lam1[Q], lF0[3], lF1[3];
    {
        const float F0[3] = {Fv[0].x + (float)gx, Fv[1].x + (float)gy, Fv[2].x + (float)gz};
        const float l0[3] = {lu[0].x, lu[1].x, lu[2].x};
        adj_cell(ls0, dv0, F0, l0, omega, rho0, lam0, lF0);
    }
    {
        const float F1[3] = {Fv[0].y + (float)gx, Fv[1].y + (float)gy, Fv[2].y + (float)gz};
        const float l1[3] = {lu[0].y, lu[1].y, lu[2].y};
        adj_cell(ls1, dv1, F1, l1, omega, rho0, lam1, lF1);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) *reinterpret_cast<float2 *>(lam_cur + i * d.Npad + cell) = make_float2(lam0[i], lam1[i]);
    for (int a = 0; a < 3; ++a) {
        *reinterpret_cast<float2 *>(lam_F + a * d.Npad + cell) = make_float2(lF0[a], lF1[a]);
        *reinterpret_cast<float2 *>(lam_u + a * d.Npad + cell) = make_float2(0.f, 0.f);
    }
}

// The reverse fluid update by rows (y, z): NEAR launches update the rows under
// the step's node stencils (tagged by the forward spreading), the others the
// rest of the box.  Away from the stencils F = 0 (apart from a uniform body
// force), lam_u = 0 and lam_F is never read, so those rows skip them.  One
// block per row, two adjacent cells per thread (FP32, even rows) or one.
template <typename T, bool NEAR, bool PAIR>
__global__ void __launch_bounds__(128) k_adj_lb_rows(Dims d, T omega, T rho0, double gx, double gy, double gz,
                                                     const T *pops, const T *F, const T *lam_next, T *lam_u, T *lam_cur,
                                                     T *lam_F, const int *rowtag, const int *rlist, const int *rcnt,
                                                     const long long *tb, int k) {
    // NEAR: the rows the spreading listed, grid-stride; otherwise one block
    // per row, skipping the tagged ones
    const int tag = (int)(*tb + k + 1);
    const int n_it = NEAR ? *rcnt : 1;
    constexpr int CPT = PAIR ? 2 : 1;
    const T G[3] = {(T)gx, (T)gy, (T)gz};  // converted once, not per cell (FP64 converts issue slowly here)
    for (int it = NEAR ? (int)blockIdx.x : 0; it < n_it; it += NEAR ? (int)gridDim.x : 1) {
        const int row = NEAR ? rlist[it] : (int)blockIdx.x;
        if (!NEAR && rowtag[row] == tag) return;
        const int y = row % d.ny, z = row / d.ny;
        for (int x = CPT * threadIdx.x; x < d.nx; x += CPT * blockDim.x) {
            const int cell = x + d.nx * row;
            T ls[CPT][Q], dv[CPT][Q];
            const Nbr n0(d, x, y, z);
            if constexpr (PAIR) {
                // 8-byte vector accesses wherever both cells' values stay adjacent
                const Nbr n1(d, x + 1, y, z);
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const float *pl = lam_next + i * d.Npad;
                    if (cx(i) == 0) {
                        const float2 v = *reinterpret_cast<const float2 *>(pl + cell + n0.off(i));
                        ls[0][i] = v.x;
                        ls[1][i] = v.y;
                    } else {
                        ls[0][i] = pl[cell + n0.off(i)];
                        ls[1][i] = pl[cell + 1 + n1.off(i)];
                    }
                    const float2 v = *reinterpret_cast<const float2 *>(pops + i * d.Npad + cell);
                    dv[0][i] = v.x;
                    dv[1][i] = v.y;
                }
            } else {
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    ls[0][i] = lam_next[i * d.Npad + cell + n0.off(i)];
                    dv[0][i] = pops[i * d.Npad + cell];
                }
            }
            T lam[CPT][Q], lF[CPT][3];
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                T Fv[3] = {G[0], G[1], G[2]}, lu[3] = {0, 0, 0};
                if constexpr (NEAR) {
                    for (int a = 0; a < 3; ++a) {
                        Fv[a] += F[a * d.Npad + cell + c];
                        lu[a] = lam_u[a * d.Npad + cell + c];
                    }
                }
                adj_cell(ls[c], dv[c], Fv, lu, omega, rho0, lam[c], lF[c]);
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if constexpr (PAIR) *reinterpret_cast<float2 *>(lam_cur + i * d.Npad + cell) = make_float2(lam[0][i], lam[1][i]);
                else lam_cur[i * d.Npad + cell] = lam[0][i];
            }
            if constexpr (NEAR) {
                for (int a = 0; a < 3; ++a)
                    for (int c = 0; c < CPT; ++c) {
                        lam_F[a * d.Npad + cell + c] = lF[c][a];
                        lam_u[a * d.Npad + cell + c] = 0;
                    }
            }
        }
    }
}

// one warp per node: transpose of spreading
template <typename T>
__global__ void k_adj_spread(Dims d, int M, const double *r, const double *fn, const T *lam_F, double *lam_r,
                             double *lam_fn) {
    const int j = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (j >= M) return;
    int cell[2];
    T w[2], g[2][3];
    lane_cells<T>(d, r + 3 * j, lane, cell, w, g);
    const double f0 = fn[3 * j], f1 = fn[3 * j + 1], f2 = fn[3 * j + 2];
    double lf[3] = {0.0, 0.0, 0.0}, G[3] = {0.0, 0.0, 0.0};
    for (int h = 0; h < 2; ++h) {
        const double l0 = (double)lam_F[cell[h]], l1 = (double)lam_F[d.Npad + cell[h]],
                     l2 = (double)lam_F[2 * d.Npad + cell[h]];
        lf[0] += (double)w[h] * l0;
        lf[1] += (double)w[h] * l1;
        lf[2] += (double)w[h] * l2;
        const double dot = l0 * f0 + l1 * f1 + l2 * f2;
        for (int a = 0; a < 3; ++a) G[a] += dot * (double)g[h][a];
    }
    for (int a = 0; a < 3; ++a) {
        lf[a] = warp_sum(lf[a]);
        G[a] = warp_sum(G[a]);
    }
    if (lane == 0)
        for (int a = 0; a < 3; ++a) {
            lam_fn[3 * j + a] = lf[a];
            lam_r[3 * j + a] += G[a];
        }
}

// one thread per triangle: membrane force Jacobian times lam_f at its corners
__global__ void k_adj_tri(Mesh m, const double *r, const double *lam_fn, double *tri_adj) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.T) return;
    const int *v = m.tris + 3 * t;
    TriState S;
    tri_state(m.G + 3 * t, m.iG[t], m.A0Gs[t], r + 3 * v[0], r + 3 * v[1], r + 3 * v[2], S);
    double df[3][3];
    tri_force_jvp(m.G + 3 * t, S, lam_fn + 3 * v[0], lam_fn + 3 * v[1], lam_fn + 3 * v[2], df);
    for (int q = 0; q < 3; ++q)
        for (int a = 0; a < 3; ++a) tri_adj[9 * t + 3 * q + a] = df[q][a];
}

// one cluster of three blocks per swimmer, block q summing lam_fj over bead
// q; block 0 reads the three sums from the blocks' shared memory and
// (thread 0) forms lam_e_b = the mean over bead b, the drive-parameter
// gradient and the transpose of the spring forces -> lam_R
__global__ void __cluster_dims__(3, 1, 1) __launch_bounds__(BEAD_THREADS)
    k_adj_swimmer(Mesh m, const Swim *sw, const double *theta, const double *drv, const double *R,
                  const double *lam_fn, const long long *t_base, int k, double *lam_R, double *grad) {
    namespace cg = cooperative_groups;
    __shared__ double sh[BEAD_THREADS / 32][3];
    __shared__ double lq[3];
    cg::cluster_group cl = cg::this_cluster();
    const int s = blockIdx.x / 3, q = (int)cl.block_rank();
    const Swim w = sw[s];
    {
        const int b = w.bead[q], n0 = m.bead_start[b], nn = m.bead_count[b];
        double acc[3] = {0.0, 0.0, 0.0};
        for (int j = n0 + threadIdx.x; j < n0 + nn; j += BEAD_THREADS)
            for (int a = 0; a < 3; ++a) acc[a] += lam_fn[3 * j + a];
        bead_sum3(acc, sh, lq);
    }
    cl.sync();
    if (q == 0 && threadIdx.x < 32) {
        // warp 0 of block 0: lane q < 3 the drive gradient of bead q, lanes 0
        // and 1 the spring transposes of sides 0 and 2
        const int l = threadIdx.x;
        double le[3][3];
        for (int qq = 0; qq < 3; ++qq) {
            const double *p = cl.map_shared_rank(lq, qq);
            for (int a = 0; a < 3; ++a) le[qq][a] = p[a];
        }
        for (int qq = 0; qq < 3; ++qq)
            for (int a = 0; a < 3; ++a) le[qq][a] *= m.bead_inv[w.bead[qq]];
        // drive: f_q = A_q sin(om t + phi_q) along x (balance: f_1 = -f_0 - f_2)
        const double *th = theta + 6 * s;
        const double *dv = drv + ((*t_base + k) * (long long)(gridDim.x / 3) + s) * 6;
        double sens[3];
        if (w.balance) {
            sens[0] = le[0][0] - le[1][0];
            sens[1] = 0.0;
            sens[2] = le[2][0] - le[1][0];
        } else {
            for (int qq = 0; qq < 3; ++qq) sens[qq] = le[qq][0];
        }
        if (l < 3 && !(w.balance && l == 1)) {
            grad[6 * s + l] += dv[l] * sens[l];
            grad[6 * s + 3 + l] += th[l] * dv[3 + l] * sens[l];
        }
        // springs: f_0 = h(R_0 - R_1), f_2 = h(R_2 - R_1), f_1 = -f_0 - f_2 with
        // h(d) = -k (|d| - L) d/|d|, dh/dd = -k [(1 - L/|d|) I + (L/|d|) dhat dhat^T]
        const int qs = l ? 2 : 0;
        double dd[3], n2 = 0.0, lv[3], ld[3];
        for (int a = 0; a < 3; ++a) {
            dd[a] = R[3 * w.bead[qs] + a] - R[3 * w.bead[1] + a];
            n2 += dd[a] * dd[a];
            lv[a] = le[qs][a] - le[1][a];
        }
        const double n = sqrt(n2), in = 1.0 / n, c1 = 1.0 - w.L * in, c2 = w.L * in * in * in;
        const double dl = dd[0] * lv[0] + dd[1] * lv[1] + dd[2] * lv[2];
        for (int a = 0; a < 3; ++a) ld[a] = -w.k * (c1 * lv[a] + c2 * dd[a] * dl);
        for (int a = 0; a < 3; ++a) {
            const double l0 = __shfl_sync(0xffffffffu, ld[a], 0), l2 = __shfl_sync(0xffffffffu, ld[a], 1);
            if (l == 0) {
                lam_R[3 * w.bead[0] + a] = l0;
                lam_R[3 * w.bead[1] + a] = -l0 - l2;
                lam_R[3 * w.bead[2] + a] = l2;
            }
        }
    }
    cl.sync();  // the blocks' shared memory outlives block 0's reads
}

// one thread per node: lam_r_j += sum of its corners' membrane terms + lam_R_b / N_b
__global__ void k_adj_node(Mesh m, const double *tri_adj, const double *lam_R, double *lam_r) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m.M) return;
    double f[3] = {0.0, 0.0, 0.0};
    for (int e = m.csr_ptr[j]; e < m.csr_ptr[j + 1]; ++e) {
        const int k = m.csr_ent[e];
        for (int a = 0; a < 3; ++a) f[a] += tri_adj[3 * k + a];
    }
    const int b = m.node_bead[j];
    const double inv = m.bead_inv[b];
    for (int a = 0; a < 3; ++a) lam_r[3 * j + a] += f[a] + lam_R[3 * b + a] * inv;
}

// ---------------------------------------------------------------- host side

int fail(int code, const std::string &msg) {
    set_last_error(msg.c_str());
    return code;
}

#define CU(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(LBIB_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
    } while (0)

struct Plan {
    Dims d;
    size_t esize;
    int M, T, B, S;
    long long n_steps;
    int K, n_seg;
    // per-slot offsets
    size_t s_pops, s_F, s_u, s_r, s_fn, s_R, s_ext, s_rows, s_rlist, s_rcnt, slot_bytes;
    // per-checkpoint offsets
    size_t c_pops, c_r, ck_bytes;
    // workspace offsets
    size_t o_drv = 0;  // drive table: per step and swimmer sin and cos of (omega t + phi_q), q = 0..2
    size_t o_tris, o_G, o_A0, o_iG, o_bi, o_cptr, o_cent, o_nb, o_bs, o_bc, o_bw, o_swim, o_theta, o_grad, o_disp, o_err,
        o_seed, o_lf0, o_lf1, o_lu, o_lF, o_lr, o_lfn, o_trif, o_tria, o_lR, o_tb, o_tbt, o_ck, o_slots[2], total;
};

Plan make_plan(const lb_params *p, const lbib_structure *s, long long n_steps, int K) {
    Plan P;
    P.d.nx = p->nx;
    P.d.ny = p->ny;
    P.d.nz = p->nz;
    P.d.N = (long long)p->nx * p->ny * p->nz;
    P.d.Npad = (P.d.N + 63) / 64 * 64;
    P.esize = p->storage == LBIB_F64 ? 8 : 4;
    P.M = s ? s->n_nodes : 0;
    P.T = s ? s->n_tris : 0;
    P.B = s ? s->n_beads : 0;
    P.S = s ? s->n_swimmers : 0;
    P.n_steps = n_steps;
    P.K = K;
    P.n_seg = (int)((n_steps + K - 1) / K);
    const size_t fp = (size_t)P.d.Npad * P.esize, nd = 3 * (size_t)std::max(P.M, 1) * 8,
                 bd = 3 * (size_t)std::max(P.B, 1) * 8;
    size_t o = 0;
    P.s_pops = o; o += up(Q * fp);
    P.s_F = o; o += up(3 * fp);
    P.s_u = o; o += up(3 * fp);
    P.s_r = o; o += up(nd);
    P.s_fn = o; o += up(nd);
    P.s_R = o; o += up(bd);
    P.s_ext = o; o += up(bd);
    P.s_rows = o; o += up((size_t)p->ny * p->nz * 4);   // tags of the rows (y, z) under the step's stencils
    P.s_rlist = o; o += up((size_t)p->ny * p->nz * 4);  // those rows, listed once each
    P.s_rcnt = o; o += up(16);                          // how many
    P.slot_bytes = o;
    o = 0;
    P.c_pops = o; o += up(Q * fp);
    P.c_r = o; o += up(nd);
    P.ck_bytes = o;
    const size_t Tn = std::max(P.T, 1), Mn = std::max(P.M, 1), Bn = std::max(P.B, 1), Sn = std::max(P.S, 1);
    o = 0;
    P.o_tris = o; o += up(3 * Tn * 4);
    P.o_G = o; o += up(3 * Tn * 8);
    P.o_A0 = o; o += up(Tn * 8);
    P.o_iG = o; o += up(Tn * 8);
    P.o_bi = o; o += up(Bn * 8);
    P.o_cptr = o; o += up((Mn + 1) * 4);
    P.o_cent = o; o += up(3 * Tn * 4);
    P.o_nb = o; o += up(Mn * 4);
    P.o_bs = o; o += up(Bn * 4);
    P.o_bc = o; o += up(Bn * 4);
    P.o_bw = o; o += up(Bn * 4);
    P.o_swim = o; o += up(Sn * sizeof(Swim));
    P.o_theta = o; o += up(6 * Sn * 8);
    P.o_grad = o; o += up(6 * Sn * 8);
    P.o_disp = o; o += up(3 * Sn * 8);
    P.o_err = o; o += up(4);
    P.o_seed = o; o += up(3 * Sn * 8);
    P.o_drv = o; o += up((size_t)P.n_steps * Sn * 6 * 8);
    P.o_lf0 = o; o += up(Q * fp);
    P.o_lf1 = o; o += up(Q * fp);
    P.o_lu = o; o += up(3 * fp);
    P.o_lF = o; o += up(3 * fp);
    P.o_lr = o; o += up(nd);
    P.o_lfn = o; o += up(nd);
    P.o_trif = o; o += up(9 * Tn * 8);
    P.o_tria = o; o += up(9 * Tn * 8);
    P.o_lR = o; o += up(bd);
    P.o_tb = o; o += up(16);                         // first step of the segment in each slot set
    P.o_tbt = o; o += up((size_t)P.n_seg * 8);       // g K for every segment g
    P.o_ck = o; o += (size_t)(P.n_seg + 1) * P.ck_bytes;  // + the final state
    // two sets of K + 1 step records: the reverse sweep of one segment runs
    // beside the recompute of the segment before it
    P.o_slots[0] = o; o += (size_t)(K + 1) * P.slot_bytes;
    P.o_slots[1] = o; o += (size_t)(K + 1) * P.slot_bytes;
    P.total = o;
    return P;
}

bool check(const lb_params *p, const lbib_structure *s, long long n_steps, int K, std::string &why) {
    if (!p) { why = "params is NULL"; return false; }
    if (p->storage != LBIB_F32 && p->storage != LBIB_F64) {
        why = "the adjoint engine stores populations as LBIB_F32 or LBIB_F64";
        return false;
    }
    lb_params q = *p;
    q.storage = LBIB_F32;
    if (!check_params(&q, why) || !check_structure(&q, s, why)) return false;
    if (p->forcing != LBIB_GUO) { why = "the adjoint engine supports Guo forcing only"; return false; }
    if (p->kernel != LBIB_PESKIN4) {
        why = "the adjoint engine needs the differentiable 4-point kernel";
        return false;
    }
    if (n_steps < 1 || K < 1) { why = "n_steps and K must be >= 1"; return false; }
    if (n_steps > (1ll << 40)) { why = "n_steps too large"; return false; }
    for (int b = 0; s && b < s->n_beads; ++b)
        if (s->beads[b].law != LBIB_NEOHOOKE || s->beads[b].kb != 0.0 || s->beads[b].kv != 0.0) {
            why = "the adjoint engine supports the neo-Hookean membrane without bending or volume terms";
            return false;
        }
    return true;
}

}  // namespace

struct lbib_adjoint {
    lb_params p;
    Plan P;
    cudaStream_t s;
    char *ws;
    Mesh m;
    std::vector<double> rest;  // rest node positions (host)
    int slots_seg[2] = {-1, -1};  // segment whose steps each slot set currently holds
    bool have_fwd = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // the reverse sweep recomputes segment g - 1 on stream s2 while the caller
    // stream runs the reverse steps of segment g: e_ready[set] marks a
    // recompute done, e_free[set] the reverse steps that read the set done
    cudaStream_t s2 = nullptr;
    cudaEvent_t e_ready[2] = {nullptr, nullptr}, e_free[2] = {nullptr, nullptr};
    // the reverse steps run on a high-priority stream forked from the caller's,
    // so the recompute beside them takes the SM slots they leave
    cudaStream_t s_rev = nullptr;
    cudaEvent_t e_fork = nullptr, e_join = nullptr;
    // the reverse fluid update of the rows away from the stencils, beside the
    // node chain: its stream, its capture stream and the step-to-step events
    cudaStream_t s_bulk = nullptr, cap_b = nullptr;
    cudaEvent_t e_near = nullptr, e_bulk = nullptr;
    // the same split of the recorded forward steps: the rows away from the
    // stencils of the forward sweep (beside a->s) and of the recompute (beside s2)
    cudaStream_t s_fb = nullptr, s2b = nullptr;
    cudaEvent_t e_nearf = nullptr, e_bulkf = nullptr;
    // a third stream beside each chain stream (the forward sweep's, the
    // recompute's, the reverse's, the capture's): the triangle kernel of a
    // step runs on it beside the swimmer kernel, which it does not depend on
    cudaStream_t s_t = nullptr, s2t = nullptr, s_revt = nullptr, cap_t = nullptr;
    cudaEvent_t e_tf_fork = nullptr, e_tf_join = nullptr, e_tr_fork = nullptr, e_tr_join = nullptr;
    float fwd_ms = 0.f, bwd_ms = 0.f;
    long long fwd_launches = 0, bwd_launches = 0, launches = 0;
    // CUDA graphs of one full K-step segment: the forward steps, and the
    // reverse steps for either parity of the adjoint population buffers
    cudaStream_t cap = nullptr;
    cudaGraphExec_t g_fwd[2] = {nullptr, nullptr}, g_rev[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    bool graphs = true;  // replay segment graphs (LBIB_GRAPHS=0: launch directly)
    long long n_fwd = 0, n_rev[2] = {0, 0};

    ~lbib_adjoint() {
        for (cudaGraphExec_t g : g_fwd)
            if (g) cudaGraphExecDestroy(g);
        for (auto &gp : g_rev)
            for (cudaGraphExec_t g : gp)
                if (g) cudaGraphExecDestroy(g);
        if (cap) cudaStreamDestroy(cap);
        if (s2) cudaStreamDestroy(s2);
        if (s_rev) cudaStreamDestroy(s_rev);
        if (s_bulk) cudaStreamDestroy(s_bulk);
        if (cap_b) cudaStreamDestroy(cap_b);
        if (e_near) cudaEventDestroy(e_near);
        if (e_bulk) cudaEventDestroy(e_bulk);
        if (s_fb) cudaStreamDestroy(s_fb);
        if (s2b) cudaStreamDestroy(s2b);
        if (e_nearf) cudaEventDestroy(e_nearf);
        if (e_bulkf) cudaEventDestroy(e_bulkf);
        for (cudaStream_t x : {s_t, s2t, s_revt, cap_t})
            if (x) cudaStreamDestroy(x);
        for (cudaEvent_t x : {e_tf_fork, e_tf_join, e_tr_fork, e_tr_join})
            if (x) cudaEventDestroy(x);
        if (e_fork) cudaEventDestroy(e_fork);
        if (e_join) cudaEventDestroy(e_join);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        for (int k = 0; k < 2; ++k) {
            if (e_ready[k]) cudaEventDestroy(e_ready[k]);
            if (e_free[k]) cudaEventDestroy(e_free[k]);
        }
    }
    template <typename X> X *at(size_t off) const { return (X *)(ws + off); }
    char *slot(int k, int set) const { return ws + P.o_slots[set] + (size_t)k * P.slot_bytes; }
    long long *tbase(int set) const { return (long long *)(ws + P.o_tb) + set; }
    char *ck(int c) const { return ws + P.o_ck + (size_t)c * P.ck_bytes; }
    int seg_len(int g) const { return (int)std::min<long long>(P.K, P.n_steps - (long long)g * P.K); }
};

namespace {

// Row-kernel launches.  The stencil rows (NEAR) run on a fixed grid that
// walks the step's row list; every other row is one block.  Two cells per
// thread (FP32, even rows) or one.
constexpr unsigned NEAR_BLOCKS = 512;

template <bool NEAR>
unsigned rows_grid(unsigned nrow) { return NEAR ? std::min(nrow, NEAR_BLOCKS) : nrow; }

template <typename T, bool NEAR>
void fwd_rows(const Plan &P, bool pair, unsigned nrow, unsigned tpb, cudaStream_t s, T om, T r0, double g0, double g1,
              double g2, const char *sl, const T *F, T *out, T *u, T *F_next, const long long *tb, int k) {
    const int *tags = (const int *)(sl + P.s_rows), *list = (const int *)(sl + P.s_rlist),
              *cnt = (const int *)(sl + P.s_rcnt);
    const T *pops = (const T *)(sl + P.s_pops);
    if constexpr (sizeof(T) == 4) {
        if (pair) {
            k_fwd_lb_rows<T, NEAR, true><<<rows_grid<NEAR>(nrow), tpb, 0, s>>>(P.d, om, r0, g0, g1, g2, pops, F, out, u,
                                                                             F_next, tags, list, cnt, tb, k);
            return;
        }
    }
    k_fwd_lb_rows<T, NEAR, false><<<rows_grid<NEAR>(nrow), tpb, 0, s>>>(P.d, om, r0, g0, g1, g2, pops, F, out, u,
                                                                      F_next, tags, list, cnt, tb, k);
}

template <typename T, bool NEAR>
void adj_rows(const Plan &P, bool pair, unsigned nrow, unsigned tpb, cudaStream_t s, T om, T r0, double g0, double g1,
              double g2, const char *sl, const T *F, const T *lam_next, T *lam_u, T *lam_cur, T *lam_F,
              const long long *tb, int k) {
    const int *tags = (const int *)(sl + P.s_rows), *list = (const int *)(sl + P.s_rlist),
              *cnt = (const int *)(sl + P.s_rcnt);
    const T *pops = (const T *)(sl + P.s_pops);
    if constexpr (sizeof(T) == 4) {
        if (pair) {
            k_adj_lb_rows<T, NEAR, true><<<rows_grid<NEAR>(nrow), tpb, 0, s>>>(P.d, om, r0, g0, g1, g2, pops, F,
                                                                             lam_next, lam_u, lam_cur, lam_F, tags,
                                                                             list, cnt, tb, k);
            return;
        }
    }
    k_adj_lb_rows<T, NEAR, false><<<rows_grid<NEAR>(nrow), tpb, 0, s>>>(P.d, om, r0, g0, g1, g2, pops, F, lam_next,
                                                                      lam_u, lam_cur, lam_F, tags, list, cnt, tb, k);
}

// One recorded forward step on two streams: st carries the node-level chain
// and the fluid update of the rows under the stencils (which the
// interpolation reads), sb the fluid update of every other row, beside the
// chain.  The spreading of step k waits for the other rows of step k - 1
// (they clear the force field it adds into, and push populations step k
// reads), and the other rows of step k wait for the spreading of step k
// (their row tags; the stencil rows of step k - 1 come before it on st).
template <typename T>
cudaError_t fwd_step(lbib_adjoint *a, int k, cudaStream_t st, cudaStream_t sb, cudaStream_t sx, int set) {
    const Plan &P = a->P;
    char *sl = a->slot(k, set), *sn = a->slot(k + 1, set);
    const double *r = (const double *)(sl + P.s_r);
    double *fn = (double *)(sl + P.s_fn), *R = (double *)(sl + P.s_R), *ext = (double *)(sl + P.s_ext);
    T *F = (T *)(sl + P.s_F), *u = (T *)(sl + P.s_u);
    const int M = P.M;
    const T om = (T)(1.0 / a->p.tau), r0 = (T)a->p.rho0;
    const double g0 = a->p.g[0], g1 = a->p.g[1], g2 = a->p.g[2];
    const bool pair = sizeof(T) == 4 && P.d.nx % 2 == 0;
    cudaError_t e;
    if (M > 0) {
        const unsigned nrow = (unsigned)(P.d.ny * P.d.nz);
        const unsigned tpb = (unsigned)std::min(128, std::max(32, (P.d.nx / (pair ? 2 : 1) + 31) / 32 * 32));
        // the triangles' corner forces (sx) beside the bead centres and
        // swimmer forces (st): both read only this step's positions
        if ((e = cudaEventRecord(a->e_tf_fork, st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(sx, a->e_tf_fork, 0)) != cudaSuccess) return e;
        // FP64-latency-bound: small blocks spread the triangles over every SM
        k_fwd_tri<<<(P.T + TRI_THREADS - 1) / TRI_THREADS, TRI_THREADS, 0, sx>>>(a->m, r, a->at<double>(P.o_trif));
        if ((e = cudaEventRecord(a->e_tf_join, sx)) != cudaSuccess) return e;
        k_fwd_swimmer<<<3 * P.S, BEAD_THREADS, 0, st>>>(a->m, a->at<Swim>(P.o_swim), a->at<double>(P.o_theta),
                                                         a->at<double>(P.o_drv), r, a->tbase(set), k, R, ext);
        if ((e = cudaStreamWaitEvent(st, a->e_tf_join, 0)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(st, a->e_bulkf, 0)) != cudaSuccess) return e;
        k_fwd_spread<T><<<(M + 3) / 4, 128, 0, st>>>(P.d, a->m, r, a->at<double>(P.o_trif), ext, fn, F,
                                                      (int *)(sl + P.s_rows), (int *)(sl + P.s_rlist),
                                                      (int *)(sl + P.s_rcnt), a->tbase(set), k);
        a->launches += 3;
        if ((e = cudaEventRecord(a->e_nearf, st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(sb, a->e_nearf, 0)) != cudaSuccess) return e;
        fwd_rows<T, false>(P, pair, nrow, tpb, sb, om, r0, g0, g1, g2, sl, F, (T *)(sn + P.s_pops), u,
                           (T *)(sn + P.s_F), a->tbase(set), k);
        if ((e = cudaEventRecord(a->e_bulkf, sb)) != cudaSuccess) return e;
        fwd_rows<T, true>(P, pair, nrow, tpb, st, om, r0, g0, g1, g2, sl, F, (T *)(sn + P.s_pops), u,
                          (T *)(sn + P.s_F), a->tbase(set), k);
        k_fwd_interp<T><<<(M + 3) / 4, 128, 0, st>>>(P.d, M, r, u, (double *)(sn + P.s_r), a->at<int>(P.o_err));
        a->launches += 3;
        return cudaGetLastError();
    }
    if (pair) {
        const unsigned nb = (unsigned)((P.d.N / 2 + 127) / 128);
        k_fwd_lb2<<<nb, 128, 0, st>>>(P.d, (float)om, (float)r0, g0, g1, g2, (const float *)(sl + P.s_pops),
                                      (const float *)F, (float *)(sn + P.s_pops), (float *)u, (float *)(sn + P.s_F));
    } else {
        const unsigned nb = (unsigned)((P.d.N + 255) / 256);
        k_fwd_lb<T><<<nb, 256, 0, st>>>(P.d, om, r0, g0, g1, g2, (const T *)(sl + P.s_pops), F, (T *)(sn + P.s_pops),
                                         u, (T *)(sn + P.s_F));
    }
    a->launches += 1;
    return cudaGetLastError();
}

// One reverse step on two streams: st carries the node-level chain and the
// fluid update of the rows under the step's stencils, sb the fluid update of
// every other row, which needs no immersed-boundary quantity and runs beside
// the chain.  The rows' update of step k waits for the other rows of step
// k + 1 (e_bulk), and the other rows of step k for the stencil rows of step k
// (e_near: then every value they pull of step k + 1 is final, and the buffer
// they write was last read by step k + 1).
template <typename T>
cudaError_t adj_step(lbib_adjoint *a, int k, T *lam_next, T *lam_cur, cudaStream_t st, cudaStream_t sb,
                     cudaStream_t sx, int set) {
    const Plan &P = a->P;
    char *sl = a->slot(k, set);
    const double *r = (const double *)(sl + P.s_r), *fn = (const double *)(sl + P.s_fn),
                 *R = (const double *)(sl + P.s_R);
    const T *F = (const T *)(sl + P.s_F), *u = (const T *)(sl + P.s_u);
    T *lam_u = a->at<T>(P.o_lu), *lam_F = a->at<T>(P.o_lF);
    double *lam_r = a->at<double>(P.o_lr), *lam_fn = a->at<double>(P.o_lfn);
    const int M = P.M;
    const unsigned nrow = (unsigned)(P.d.ny * P.d.nz);
    const bool pair = sizeof(T) == 4 && P.d.nx % 2 == 0;
    const unsigned tpb = (unsigned)std::min(128, std::max(32, (P.d.nx / (pair ? 2 : 1) + 31) / 32 * 32));
    const T om = (T)(1.0 / a->p.tau), r0 = (T)a->p.rho0;
    const double g0 = a->p.g[0], g1 = a->p.g[1], g2 = a->p.g[2];
    cudaError_t e;
    if (M > 0) {
        k_adj_interp<T><<<(M + 3) / 4, 128, 0, st>>>(P.d, M, r, u, lam_r, lam_u);
        a->launches += 1;
        if ((e = cudaStreamWaitEvent(st, a->e_bulk, 0)) != cudaSuccess) return e;
        adj_rows<T, true>(P, pair, nrow, tpb, st, om, r0, g0, g1, g2, sl, F, lam_next, lam_u, lam_cur, lam_F,
                          a->tbase(set), k);
        a->launches += 1;
        if ((e = cudaEventRecord(a->e_near, st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(sb, a->e_near, 0)) != cudaSuccess) return e;
        adj_rows<T, false>(P, pair, nrow, tpb, sb, om, r0, g0, g1, g2, sl, F, lam_next, lam_u, lam_cur, lam_F,
                           a->tbase(set), k);
        a->launches += 1;
        if ((e = cudaEventRecord(a->e_bulk, sb)) != cudaSuccess) return e;
        k_adj_spread<T><<<(M + 3) / 4, 128, 0, st>>>(P.d, M, r, fn, lam_F, lam_r, lam_fn);
        // the triangles' transposes (sx) beside the swimmer's (st): both read
        // lam_fn only, and the node kernel sums what both wrote
        if ((e = cudaEventRecord(a->e_tr_fork, st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(sx, a->e_tr_fork, 0)) != cudaSuccess) return e;
        k_adj_tri<<<(P.T + TRI_THREADS - 1) / TRI_THREADS, TRI_THREADS, 0, sx>>>(a->m, r, lam_fn,
                                                                                a->at<double>(P.o_tria));
        if ((e = cudaEventRecord(a->e_tr_join, sx)) != cudaSuccess) return e;
        k_adj_swimmer<<<3 * P.S, BEAD_THREADS, 0, st>>>(a->m, a->at<Swim>(P.o_swim), a->at<double>(P.o_theta),
                                                         a->at<double>(P.o_drv), R, lam_fn, a->tbase(set), k,
                                                         a->at<double>(P.o_lR), a->at<double>(P.o_grad));
        if ((e = cudaStreamWaitEvent(st, a->e_tr_join, 0)) != cudaSuccess) return e;
        k_adj_node<<<(M + TRI_THREADS - 1) / TRI_THREADS, TRI_THREADS, 0, st>>>(a->m, a->at<double>(P.o_tria),
                                                                               a->at<double>(P.o_lR), lam_r);
        a->launches += 4;
        return cudaGetLastError();
    }
    // no nodes: the whole box in one launch
    if (pair) {
        const unsigned nb = (unsigned)((P.d.N / 2 + 127) / 128);
        k_adj_lb2<<<nb, 128, 0, st>>>(P.d, (float)om, (float)r0, g0, g1, g2, (const float *)(sl + P.s_pops),
                                      (const float *)F, (const float *)lam_next, (float *)lam_u, (float *)lam_cur,
                                      (float *)lam_F);
    } else {
        const unsigned nb = (unsigned)((P.d.N + 255) / 256);
        k_adj_lb<T><<<nb, 256, 0, st>>>(P.d, om, r0, g0, g1, g2, (const T *)(sl + P.s_pops), F, lam_next, lam_u,
                                         lam_cur, lam_F);
    }
    a->launches += 1;
    return cudaGetLastError();
}

// Start a run of recorded forward steps on stream st with the second stream
// sb: sb follows st through each step's spreading, and the first step's
// spreading need not wait for sb.
cudaError_t fwd_fork(lbib_adjoint *a, cudaStream_t st, cudaStream_t sb) {
    cudaError_t e;
    if ((e = cudaEventRecord(a->e_nearf, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(sb, a->e_nearf, 0)) != cudaSuccess) return e;
    return cudaEventRecord(a->e_bulkf, st);
}

// Start a run of reverse steps on stream st with the second stream sb: sb
// follows st, and the first step's stencil rows need not wait for sb.
cudaError_t rev_fork(lbib_adjoint *a, cudaStream_t st, cudaStream_t sb) {
    cudaError_t e;
    if ((e = cudaEventRecord(a->e_near, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(sb, a->e_near, 0)) != cudaSuccess) return e;
    return cudaEventRecord(a->e_bulk, st);
}

// capture the K forward steps of a full segment (slots 0 -> K of a slot set),
// or its K reverse steps starting on adjoint buffer `par`, into a graph
template <typename T>
cudaError_t capture(lbib_adjoint *a, bool reverse, int par, int set) {
    const Plan &P = a->P;
    const long long n0 = a->launches;
    cudaError_t e = cudaStreamBeginCapture(a->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    T *lam[2] = {a->at<T>(P.o_lf0), a->at<T>(P.o_lf1)};
    int nxt = par;
    e = reverse ? rev_fork(a, a->cap, a->cap_b) : fwd_fork(a, a->cap, a->cap_b);
    for (int k = 0; k < P.K && e == cudaSuccess; ++k) {
        if (reverse) {
            const int kk = P.K - 1 - k;
            e = adj_step<T>(a, kk, lam[nxt], lam[1 - nxt], a->cap, a->cap_b, a->cap_t, set);
            nxt = 1 - nxt;
        } else {
            e = fwd_step<T>(a, k, a->cap, a->cap_b, a->cap_t, set);
        }
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(a->cap, reverse ? a->e_bulk : a->e_bulkf, 0);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(a->cap, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(reverse ? &a->g_rev[par][set] : &a->g_fwd[set], g, 0);
    if (g) cudaGraphDestroy(g);
    (reverse ? a->n_rev[par] : a->n_fwd) = a->launches - n0;
    a->launches = n0;
    return e;
}

// set the step counter of a slot set to the first step of segment g
cudaError_t set_tbase(lbib_adjoint *a, int g, int set, cudaStream_t st) {
    return cudaMemcpyAsync(a->tbase(set), a->at<long long>(a->P.o_tbt) + g, 8, cudaMemcpyDeviceToDevice, st);
}

// run segment g forward from its checkpoint, filling slots 0..len of a set
template <typename T>
cudaError_t run_segment(lbib_adjoint *a, int g, int set, cudaStream_t st, cudaStream_t sb, cudaStream_t sx) {
    const Plan &P = a->P;
    char *s0 = a->slot(0, set), *c = a->ck(g);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(s0 + P.s_pops, c + P.c_pops, Q * (size_t)P.d.Npad * P.esize, cudaMemcpyDeviceToDevice,
                             st)) != cudaSuccess)
        return e;
    if (P.M > 0 &&
        (e = cudaMemcpyAsync(s0 + P.s_r, c + P.c_r, 3 * (size_t)P.M * 8, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(s0 + P.s_F, 0, 3 * (size_t)P.d.Npad * P.esize, st)) != cudaSuccess) return e;
    if ((e = set_tbase(a, g, set, st)) != cudaSuccess) return e;
    if (P.M > 0) {
        // fresh row tags and lists: a row is listed by the lane that changes its tag
        const int nrow = P.d.ny * P.d.nz;
        k_clear_rows<<<(unsigned)std::min<long long>(1024, ((long long)(P.K + 1) * nrow + 255) / 256), 256, 0, st>>>(
            s0, P.slot_bytes, P.s_rows, P.s_rcnt, nrow, P.K + 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        a->launches += 1;
    }
    const int len = a->seg_len(g);
    if (len == P.K && a->graphs) {
        if (!a->g_fwd[set] && (e = capture<T>(a, false, 0, set)) != cudaSuccess) return e;
        if ((e = cudaGraphLaunch(a->g_fwd[set], st)) != cudaSuccess) return e;
        a->launches += a->n_fwd;
    } else {
        if ((e = fwd_fork(a, st, sb)) != cudaSuccess) return e;
        for (int k = 0; k < len; ++k)
            if ((e = fwd_step<T>(a, k, st, sb, sx, set)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(st, a->e_bulkf, 0)) != cudaSuccess) return e;
    }
    a->slots_seg[set] = g;
    return cudaSuccess;
}

// copy the populations and positions of slot k into checkpoint c
cudaError_t save_ck(lbib_adjoint *a, int k, int c) {
    const Plan &P = a->P;
    cudaError_t e = cudaMemcpyAsync(a->ck(c) + P.c_pops, a->slot(k, 0) + P.s_pops, Q * (size_t)P.d.Npad * P.esize,
                                    cudaMemcpyDeviceToDevice, a->s);
    if (e == cudaSuccess && P.M > 0)
        e = cudaMemcpyAsync(a->ck(c) + P.c_r, a->slot(k, 0) + P.s_r, 3 * (size_t)P.M * 8, cudaMemcpyDeviceToDevice,
                            a->s);
    return e;
}

template <typename T>
int forward_impl(lbib_adjoint *a, double *disp) {
    const Plan &P = a->P;
    CU(cudaMemsetAsync(a->at<int>(P.o_err), 0, 4, a->s));
    CU(cudaEventRecord(a->ev[0], a->s));
    a->launches = 0;
    if (P.S > 0) {  // the drive phases of every step, from the current theta
        const long long n = P.n_steps * P.S * 3;
        k_drive_table<<<(unsigned)((n + 255) / 256), 256, 0, a->s>>>(a->at<Swim>(P.o_swim), a->at<double>(P.o_theta),
                                                                   P.n_steps, P.S, a->at<double>(P.o_drv));
        a->launches += 1;
        CU(cudaGetLastError());
    }
    a->slots_seg[1] = -1;
    for (int g = 0; g < P.n_seg; ++g) {
        CU(run_segment<T>(a, g, 0, a->s, a->s_fb, a->s_t));
        CU(save_ck(a, a->seg_len(g), g + 1));  // the next checkpoint (the last one: the final state)
    }
    if (P.S > 0) {
        k_disp<<<P.S, SWIM_THREADS, 0, a->s>>>(a->m, a->at<Swim>(P.o_swim), (const double *)(a->ck(P.n_seg) + P.c_r),
                                      (const double *)(a->ck(0) + P.c_r), a->at<double>(P.o_disp));
        a->launches += 1;
        CU(cudaGetLastError());
    }
    CU(cudaEventRecord(a->ev[1], a->s));
    int err = 0;
    CU(cudaMemcpyAsync(&err, a->at<int>(P.o_err), 4, cudaMemcpyDeviceToHost, a->s));
    CU(cudaStreamSynchronize(a->s));
    CU(cudaEventElapsedTime(&a->fwd_ms, a->ev[0], a->ev[1]));
    a->fwd_launches = a->launches;
    if (err & ERR_NONFINITE) return fail(LBIB_ENONFINITE, "a node velocity became non-finite");
    if (err & ERR_UNSTABLE) return fail(LBIB_EUNSTABLE, "a node moved faster than 0.1 lattice units per step");
    if (disp && P.S > 0) {
        CU(cudaMemcpy(disp, a->at<double>(P.o_disp), 3 * (size_t)P.S * 8, cudaMemcpyDeviceToHost));
    }
    a->have_fwd = true;
    return LBIB_OK;
}

// host [19][N] raw populations <-> device deviations (lattice order of this
// library, planes Npad apart)
template <typename T>
void to_dev_layout(const lbib_adjoint *a, const double *hf, bool shift, std::vector<T> &out) {
    const Plan &P = a->P;
    out.assign(Q * (size_t)P.d.Npad, (T)0);
    for (int i = 0; i < Q; ++i) {
        const double base = shift ? wgt_d(i) * a->p.rho0 : 0.0;
        for (long long c = 0; c < P.d.N; ++c) out[i * P.d.Npad + c] = (T)(hf[i * P.d.N + c] - base);
    }
}

template <typename T>
int from_dev(const lbib_adjoint *a, const void *dev, bool shift, double *hf) {
    const Plan &P = a->P;
    std::vector<T> h(Q * (size_t)P.d.Npad);
    CU(cudaMemcpyAsync(h.data(), dev, h.size() * sizeof(T), cudaMemcpyDeviceToHost, a->s));
    CU(cudaStreamSynchronize(a->s));
    for (int i = 0; i < Q; ++i) {
        const double base = shift ? wgt_d(i) * a->p.rho0 : 0.0;
        for (long long c = 0; c < P.d.N; ++c) hf[i * P.d.N + c] = base + (double)h[i * P.d.Npad + c];
    }
    return LBIB_OK;
}

template <typename T>
int upload_pops(lbib_adjoint *a, const double *hf, bool shift, void *dev) {
    std::vector<T> h;
    to_dev_layout<T>(a, hf, shift, h);
    CU(cudaMemcpyAsync(dev, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, a->s));
    CU(cudaStreamSynchronize(a->s));
    return LBIB_OK;
}

template <typename T>
int backward_impl(lbib_adjoint *a, const double *seed_disp, const double *seed_f, const double *seed_r,
                  double *grad_theta, double *grad_f0, double *grad_r0) {
    const Plan &P = a->P;
    const size_t fp = (size_t)P.d.Npad * sizeof(T);
    T *lam[2] = {a->at<T>(P.o_lf0), a->at<T>(P.o_lf1)};
    int nxt = 0;
    // seeds
    if (seed_f) {
        int st = upload_pops<T>(a, seed_f, false, lam[nxt]);
        if (st) return st;
    } else {
        CU(cudaMemsetAsync(lam[nxt], 0, Q * fp, a->s));
    }
    double *lam_r = a->at<double>(P.o_lr);
    if (P.M > 0) {
        if (seed_r) CU(cudaMemcpyAsync(lam_r, seed_r, 3 * (size_t)P.M * 8, cudaMemcpyHostToDevice, a->s));
        CU(cudaMemcpyAsync(a->at<double>(P.o_seed), seed_disp, 3 * (size_t)P.S * 8, cudaMemcpyHostToDevice, a->s));
    }
    CU(cudaMemsetAsync(a->at<T>(P.o_lu), 0, 3 * fp, a->s));
    CU(cudaMemsetAsync(a->at<double>(P.o_grad), 0, 6 * (size_t)std::max(P.S, 1) * 8, a->s));
    CU(cudaEventRecord(a->ev[2], a->s));
    a->launches = 0;
    if (P.M > 0) {
        k_adj_seed<<<(P.M + 127) / 128, 128, 0, a->s>>>(a->m, a->at<double>(P.o_seed), 1.0, seed_r ? 1 : 0, lam_r);
        a->launches += 1;
        CU(cudaGetLastError());
    }
    // segment g's records in slot set `cur`; the recompute of segment g - 1
    // into the other set runs on s2 beside the reverse steps of segment g
    int cur = a->slots_seg[0] == P.n_seg - 1 ? 0 : (a->slots_seg[1] == P.n_seg - 1 ? 1 : -1);
    if (cur < 0) {
        cur = 0;
        CU(run_segment<T>(a, P.n_seg - 1, 0, a->s, a->s_fb, a->s_t));
    }
    cudaStream_t rs = a->s_rev;
    CU(cudaEventRecord(a->e_fork, a->s));
    CU(cudaStreamWaitEvent(rs, a->e_fork, 0));
    CU(cudaEventRecord(a->e_free[0], rs));
    CU(cudaEventRecord(a->e_free[1], rs));
    bool ready_on_s2[2] = {false, false};
    for (int g = P.n_seg - 1; g >= 0; --g) {
        const int oth = 1 - cur;
        if (g > 0) {
            CU(cudaStreamWaitEvent(a->s2, a->e_free[oth], 0));
            CU(run_segment<T>(a, g - 1, oth, a->s2, a->s2b, a->s2t));
            CU(cudaEventRecord(a->e_ready[oth], a->s2));
            ready_on_s2[oth] = true;
        }
        if (ready_on_s2[cur]) {
            CU(cudaStreamWaitEvent(rs, a->e_ready[cur], 0));
            ready_on_s2[cur] = false;
        }
        CU(set_tbase(a, g, cur, rs));
        const int len = a->seg_len(g);
        if (len == P.K && a->graphs) {
            if (!a->g_rev[nxt][cur]) CU(capture<T>(a, true, nxt, cur));
            CU(cudaGraphLaunch(a->g_rev[nxt][cur], rs));
            a->launches += a->n_rev[nxt];
            if (P.K & 1) nxt = 1 - nxt;
        } else {
            CU(rev_fork(a, rs, a->s_bulk));
            for (int k = len - 1; k >= 0; --k) {
                CU(adj_step<T>(a, k, lam[nxt], lam[1 - nxt], rs, a->s_bulk, a->s_revt, cur));
                nxt = 1 - nxt;
            }
            CU(cudaStreamWaitEvent(rs, a->e_bulk, 0));
        }
        CU(cudaEventRecord(a->e_free[cur], rs));
        cur = oth;
    }
    CU(cudaEventRecord(a->e_join, rs));
    CU(cudaStreamWaitEvent(a->s, a->e_join, 0));
    if (P.M > 0) {  // x_cm(0) enters the displacement with a minus sign
        k_adj_seed<<<(P.M + 127) / 128, 128, 0, a->s>>>(a->m, a->at<double>(P.o_seed), -1.0, 1, lam_r);
        a->launches += 1;
        CU(cudaGetLastError());
    }
    CU(cudaEventRecord(a->ev[3], a->s));
    CU(cudaStreamSynchronize(a->s));
    CU(cudaEventElapsedTime(&a->bwd_ms, a->ev[2], a->ev[3]));
    a->bwd_launches = a->launches;
    if (P.S > 0) CU(cudaMemcpy(grad_theta, a->at<double>(P.o_grad), 6 * (size_t)P.S * 8, cudaMemcpyDeviceToHost));
    if (grad_f0) {
        int st = from_dev<T>(a, lam[nxt], false, grad_f0);
        if (st) return st;
    }
    if (grad_r0 && P.M > 0) CU(cudaMemcpy(grad_r0, lam_r, 3 * (size_t)P.M * 8, cudaMemcpyDeviceToHost));
    return LBIB_OK;
}

}  // namespace

extern "C" {

int lb_adjoint_required_bytes(const lb_params *p, const lbib_structure *s, long long n_steps, int K, size_t *bytes) {
    std::string why;
    if (!bytes) return fail(LBIB_EINVAL, "bytes is NULL");
    if (!check(p, s, n_steps, K, why)) return fail(LBIB_EINVAL, why);
    *bytes = make_plan(p, s, n_steps, K).total;
    return LBIB_OK;
}

int lb_adjoint_create(const lb_params *p, const lbib_structure *s, long long n_steps, int K, void *workspace,
                      size_t workspace_bytes, void *stream, lbib_adjoint **out) {
    std::string why;
    if (!out) return fail(LBIB_EINVAL, "out is NULL");
    *out = nullptr;
    if (!check(p, s, n_steps, K, why)) return fail(LBIB_EINVAL, why);
    const Plan P = make_plan(p, s, n_steps, K);
    if (!workspace) return fail(LBIB_EINVAL, "workspace is NULL");
    if ((uintptr_t)workspace % AL) return fail(LBIB_EINVAL, "workspace must be 256-byte aligned");
    if (workspace_bytes < P.total) return fail(LBIB_ESIZE, "workspace smaller than lb_adjoint_required_bytes");
    const int M = P.M, T = P.T, B = P.B, S = P.S;
    // host tables
    std::vector<int> tris(3 * (size_t)T), cptr(M + 1, 0), cent(3 * (size_t)T), nb(M), bs(B), bc(B), bw(B, 0);
    std::vector<double> G(3 * (size_t)T), A0(T), iG(T), bi(B), theta(6 * (size_t)S);
    std::vector<Swim> sw(S);
    for (int b = 0; b < B; ++b) {
        const lbib_bead &bd = s->beads[b];
        bs[b] = bd.node_start;
        bc[b] = bd.node_count;
        bi[b] = 1.0 / bd.node_count;
        for (int j = bd.node_start; j < bd.node_start + bd.node_count; ++j) nb[j] = b;
        for (int t = bd.tri_start; t < bd.tri_start + bd.tri_count; ++t) {
            const int *v = s->tris + 3 * t;
            const double *X = s->rest_nodes;
            double e1[3], e2[3];
            for (int a = 0; a < 3; ++a) {
                e1[a] = X[3 * v[1] + a] - X[3 * v[0] + a];
                e2[a] = X[3 * v[2] + a] - X[3 * v[0] + a];
                tris[3 * t + a] = v[a];
            }
            G[3 * t] = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
            G[3 * t + 1] = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
            G[3 * t + 2] = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
            const double det = G[3 * t] * G[3 * t + 2] - G[3 * t + 1] * G[3 * t + 1];
            if (!(det > 0.0)) return fail(LBIB_EINVAL, "degenerate rest triangle");
            A0[t] = 0.5 * std::sqrt(det) * bd.Gs;
            iG[t] = 1.0 / det;
        }
    }
    for (int t = 0; t < T; ++t)
        for (int q = 0; q < 3; ++q) cptr[s->tris[3 * t + q] + 1]++;
    for (int j = 0; j < M; ++j) cptr[j + 1] += cptr[j];
    {
        std::vector<int> fill(cptr.begin(), cptr.end() - 1);
        for (int t = 0; t < T; ++t)
            for (int q = 0; q < 3; ++q) cent[fill[s->tris[3 * t + q]]++] = 3 * t + q;
    }
    for (int k = 0; k < S; ++k) {
        const lbib_swimmer &w = s->swimmers[k];
        for (int q = 0; q < 3; ++q) {
            sw[k].bead[q] = w.bead[q];
            bw[w.bead[q]] = k;
            theta[6 * k + q] = w.amp[q];
            theta[6 * k + 3 + q] = w.phase[q];
        }
        sw[k].balance = w.balance;
        sw[k].k = w.k_spring;
        sw[k].L = w.L_spring;
        sw[k].period = w.period;
    }

    lbib_adjoint *a = new lbib_adjoint();
    a->p = *p;
    a->P = P;
    a->s = (cudaStream_t)stream;
    a->ws = (char *)workspace;
    {
        const char *g = getenv("LBIB_GRAPHS");
        a->graphs = !(g && g[0] == '0');
    }
    a->rest.assign(s && M ? s->rest_nodes : nullptr, s && M ? s->rest_nodes + 3 * (size_t)M : nullptr);
    Mesh &m = a->m;
    m.M = M;
    m.T = T;
    m.B = B;
    m.S = S;
    m.tris = a->at<int>(P.o_tris);
    m.G = a->at<double>(P.o_G);
    m.A0Gs = a->at<double>(P.o_A0);
    m.iG = a->at<double>(P.o_iG);
    m.bead_inv = a->at<double>(P.o_bi);
    m.csr_ptr = a->at<int>(P.o_cptr);
    m.csr_ent = a->at<int>(P.o_cent);
    m.node_bead = a->at<int>(P.o_nb);
    m.bead_start = a->at<int>(P.o_bs);
    m.bead_count = a->at<int>(P.o_bc);
    m.bead_swim = a->at<int>(P.o_bw);
    auto cleanup = [&](int code) {
        delete a;
        return code;
    };
#define CUA(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return cleanup(fail(LBIB_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_))); \
    } while (0)
    for (int k = 0; k < 4; ++k) CUA(cudaEventCreate(&a->ev[k]));
    for (int k = 0; k < 2; ++k) {
        CUA(cudaEventCreateWithFlags(&a->e_ready[k], cudaEventDisableTiming));
        CUA(cudaEventCreateWithFlags(&a->e_free[k], cudaEventDisableTiming));
    }
    CUA(cudaStreamCreateWithFlags(&a->cap, cudaStreamNonBlocking));
    CUA(cudaStreamCreateWithFlags(&a->s2, cudaStreamNonBlocking));
    {
        int lo = 0, hi = 0;
        CUA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        CUA(cudaStreamCreateWithPriority(&a->s_rev, cudaStreamNonBlocking, hi));
        CUA(cudaStreamCreateWithPriority(&a->s_revt, cudaStreamNonBlocking, hi));
    }
    CUA(cudaEventCreateWithFlags(&a->e_fork, cudaEventDisableTiming));
    CUA(cudaStreamCreateWithFlags(&a->s_bulk, cudaStreamNonBlocking));
    CUA(cudaStreamCreateWithFlags(&a->cap_b, cudaStreamNonBlocking));
    CUA(cudaEventCreateWithFlags(&a->e_near, cudaEventDisableTiming));
    CUA(cudaEventCreateWithFlags(&a->e_bulk, cudaEventDisableTiming));
    CUA(cudaStreamCreateWithFlags(&a->s_fb, cudaStreamNonBlocking));
    CUA(cudaStreamCreateWithFlags(&a->s2b, cudaStreamNonBlocking));
    CUA(cudaEventCreateWithFlags(&a->e_nearf, cudaEventDisableTiming));
    CUA(cudaEventCreateWithFlags(&a->e_bulkf, cudaEventDisableTiming));
    CUA(cudaStreamCreateWithFlags(&a->s_t, cudaStreamNonBlocking));
    CUA(cudaStreamCreateWithFlags(&a->s2t, cudaStreamNonBlocking));
    CUA(cudaStreamCreateWithFlags(&a->cap_t, cudaStreamNonBlocking));
    for (cudaEvent_t *x : {&a->e_tf_fork, &a->e_tf_join, &a->e_tr_fork, &a->e_tr_join})
        CUA(cudaEventCreateWithFlags(x, cudaEventDisableTiming));
    CUA(cudaEventCreateWithFlags(&a->e_join, cudaEventDisableTiming));
    std::vector<long long> tb(P.n_seg);
    for (int g = 0; g < P.n_seg; ++g) tb[g] = (long long)g * K;
    auto put = [&](size_t off, const void *src, size_t n) {
        return n ? cudaMemcpyAsync(a->ws + off, src, n, cudaMemcpyHostToDevice, a->s) : cudaSuccess;
    };
    CUA(put(P.o_tris, tris.data(), tris.size() * 4));
    CUA(put(P.o_G, G.data(), G.size() * 8));
    CUA(put(P.o_A0, A0.data(), A0.size() * 8));
    CUA(put(P.o_iG, iG.data(), iG.size() * 8));
    CUA(put(P.o_bi, bi.data(), bi.size() * 8));
    CUA(put(P.o_cptr, cptr.data(), cptr.size() * 4));
    CUA(put(P.o_cent, cent.data(), cent.size() * 4));
    CUA(put(P.o_nb, nb.data(), nb.size() * 4));
    CUA(put(P.o_bs, bs.data(), bs.size() * 4));
    CUA(put(P.o_bc, bc.data(), bc.size() * 4));
    CUA(put(P.o_bw, bw.data(), bw.size() * 4));
    CUA(put(P.o_swim, sw.data(), sw.size() * sizeof(Swim)));
    CUA(put(P.o_theta, theta.data(), theta.size() * 8));
    CUA(put(P.o_tbt, tb.data(), tb.size() * 8));
    // rest initial state: zero deviations, nodes at the rest shape
    CUA(cudaMemsetAsync(a->ck(0) + P.c_pops, 0, Q * (size_t)P.d.Npad * P.esize, a->s));
    CUA(put(P.o_ck + P.c_r, a->rest.data(), a->rest.size() * 8));
    CUA(cudaStreamSynchronize(a->s));
#undef CUA
    *out = a;
    return LBIB_OK;
}

int lb_adjoint_set_drive(lbib_adjoint *a, const double *theta) {
    if (!a || (!theta && a->P.S)) return fail(LBIB_EINVAL, "NULL argument");
    for (long long k = 0; k < 6ll * a->P.S; ++k)
        if (!std::isfinite(theta[k])) return fail(LBIB_EINVAL, "non-finite drive parameter");
    if (a->P.S) {
        CU(cudaMemcpyAsync(a->at<double>(a->P.o_theta), theta, 6 * (size_t)a->P.S * 8, cudaMemcpyHostToDevice, a->s));
        CU(cudaStreamSynchronize(a->s));
    }
    a->have_fwd = false;
    a->slots_seg[0] = a->slots_seg[1] = -1;
    return LBIB_OK;
}

int lb_adjoint_set_initial(lbib_adjoint *a, const double *f, const double *r) {
    if (!a) return fail(LBIB_EINVAL, "NULL argument");
    const Plan &P = a->P;
    if (f) {
        for (long long k = 0; k < Q * P.d.N; ++k)
            if (!std::isfinite(f[k])) return fail(LBIB_EINVAL, "non-finite population");
        const int st = P.esize == 8 ? upload_pops<double>(a, f, true, a->ck(0) + P.c_pops)
                                    : upload_pops<float>(a, f, true, a->ck(0) + P.c_pops);
        if (st) return st;
    }
    if (r && P.M) {
        for (long long k = 0; k < 3ll * P.M; ++k)
            if (!std::isfinite(r[k])) return fail(LBIB_EINVAL, "non-finite node position");
        CU(cudaMemcpyAsync(a->ck(0) + P.c_r, r, 3 * (size_t)P.M * 8, cudaMemcpyHostToDevice, a->s));
        CU(cudaStreamSynchronize(a->s));
    }
    a->have_fwd = false;
    a->slots_seg[0] = a->slots_seg[1] = -1;
    return LBIB_OK;
}

int lb_adjoint_forward(lbib_adjoint *a, double *disp) {
    if (!a) return fail(LBIB_EINVAL, "NULL argument");
    a->have_fwd = false;
    return a->P.esize == 8 ? forward_impl<double>(a, disp) : forward_impl<float>(a, disp);
}

int lb_adjoint_backward(lbib_adjoint *a, const double *seed_disp, const double *seed_f, const double *seed_r,
                        double *grad_theta, double *grad_f0, double *grad_r0) {
    if (!a || (a->P.S && (!seed_disp || !grad_theta))) return fail(LBIB_EINVAL, "NULL argument");
    if (!a->have_fwd) return fail(LBIB_EINVAL, "no forward sweep with the current drive and initial state");
    return a->P.esize == 8 ? backward_impl<double>(a, seed_disp, seed_f, seed_r, grad_theta, grad_f0, grad_r0)
                           : backward_impl<float>(a, seed_disp, seed_f, seed_r, grad_theta, grad_f0, grad_r0);
}

int lb_adjoint_get_final(lbib_adjoint *a, double *f, double *r) {
    if (!a) return fail(LBIB_EINVAL, "NULL argument");
    if (!a->have_fwd) return fail(LBIB_EINVAL, "no forward sweep");
    const Plan &P = a->P;
    const char *c = a->ck(P.n_seg);
    if (f) {
        const int st = P.esize == 8 ? from_dev<double>(a, c + P.c_pops, true, f) : from_dev<float>(a, c + P.c_pops, true, f);
        if (st) return st;
    }
    if (r && P.M) CU(cudaMemcpy(r, c + P.c_r, 3 * (size_t)P.M * 8, cudaMemcpyDeviceToHost));
    return LBIB_OK;
}

int lb_adjoint_timing(lbib_adjoint *a, double *forward_ms, double *backward_ms, long long *forward_launches,
                      long long *backward_launches) {
    if (!a) return fail(LBIB_EINVAL, "NULL argument");
    if (forward_ms) *forward_ms = a->fwd_ms;
    if (backward_ms) *backward_ms = a->bwd_ms;
    if (forward_launches) *forward_launches = a->fwd_launches;
    if (backward_launches) *backward_launches = a->bwd_launches;
    return LBIB_OK;
}

int lb_adjoint_destroy(lbib_adjoint *a) {
    if (!a) return fail(LBIB_EINVAL, "NULL argument");
    cudaError_t e = cudaStreamSynchronize(a->s);
    delete a;
    if (e != cudaSuccess) return fail(LBIB_ECUDA, cudaGetErrorString(e));
    return LBIB_OK;
}

}  // extern "C"
