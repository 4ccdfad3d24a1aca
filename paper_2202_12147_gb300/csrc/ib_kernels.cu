// Immersed-boundary side of the coupled step: bead reductions, drive and
// springs, the linear-FEM membrane, spreading and interpolation.
//
//   k_ib_prepare       blocks [0, n_swimmers): bead centres, drive f^d(t)
//                      and springs f^s(R) (Sec. 2.2), stored as the per-node
//                      share (f^d + f^s)/N_v;
//                      remaining blocks: one thread per triangle computes the
//                      three corner forces -dW/dr of the neo-Hookean linear
//                      FEM element (Sec. 2.2, virtual work).
//   k_ib_gather_spread one thread per node sums its incident corner forces in
//                      a fixed order plus the bead share (total nodal force,
//                      Sec. 2.2) and sets up its stencil; then KW^2 threads
//                      per node spread it over the KW^3 stencil (Sec. 2.3,
//                      Eq. spreading) with vector float atomics, or 64-bit
//                      fixed-point atomics (bitwise reproducible).
//   k_ib_mark          stamps (and lists) the fluid tiles the node stencils
//                      touch with the step number (the advecting interpolation
//                      does the same for the next step).
//   k_ib_interp        KW threads per node gather u over the stencil
//                      (Sec. 2.3, Eq. interpolation), reduce with shuffles in
//                      a fixed order, move the node r += rdot in FP64 (front
//                      tracking, Sec. 2.3) and stamp the next step's tiles.
//
// FP64 on this GPU issues at a small fraction of the FP32 rate, so it is kept
// to what needs it: node positions and their update, the bead centres, the
// metric difference of the membrane element, and the argument of the drive.
// The bead centre R_b = mean of the bead's nodes (Fig. 1 caption) is kept up
// to date incrementally: after an advection by node velocities v_j,
// R_b += mean_j v_j (the mean is linear), folded in by the last block of the
// interpolation; k_bead_init recomputes it from the positions whenever they
// are set from outside.
//
// Membrane element.  With rest edge metric G = D^T D, current metric
// g = d^T d = G + 2E and J^2 = det g / det G, the neo-Hookean energy
// A0 Gs/2 (I1 - 1 + 1/J^2) has gradient
//   dW/dd = A0 Gs / (det G J^4) * d * [ I2 (I2 + 2) adj(G) - 2 adj(E) ],
// with I1 = 2 tr(G^{-1}E) and I2 = J^2 - 1 = 2 tr(G^{-1}E) + 4 det(E)/det(G).
// Only E = (g - G)/2 is formed in FP64 (it is a small difference of O(1)
// numbers); everything after it runs in FP32 without cancellation.
#include "lbib_internal.cuh"

namespace lbib {

constexpr int PREP_TPB = 128;
constexpr int GS_TPB = 128;
constexpr int GS_NODES = 32;  // nodes per gather/spread block
// deterministic spreading: per-block hash table of stencil cells
constexpr int GS_HT_BITS = 10;
constexpr int GS_HT = 1 << GS_HT_BITS;
constexpr int GS_HT_PROBES = 16;
constexpr unsigned GS_HT_EMPTY = 0xffffffffu;
constexpr int INT_TPB = 128;

// deterministic block reductions (fixed shuffle tree, then warps in order)
template <typename T>
__device__ __forceinline__ void block_sum3(T &a, T &b, T &c, T *sm /* 3*32 */) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) {
        sm[w] = a;
        sm[32 + w] = b;
        sm[64 + w] = c;
    }
    __syncthreads();
    a = b = c = T(0);
    for (int k = 0; k < nw; ++k) {
        a += sm[k];
        b += sm[32 + k];
        c += sm[64 + k];
    }
    __syncthreads();
}

// Swimmer block: drive (Sec. 2.2, driving-force equation) and springs
// (Sec. 2.2) from the bead centres, stored as the per-node share.
__device__ void swimmer_forces(const DevCtx &c, int s) {
    if (threadIdx.x != 0) return;
    const SwimDev sw = c.swims[s];
    double R[3][3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double *r = c.bead_R + 4 * sw.bead[q];
        R[q][0] = r[0];
        R[q][1] = r[1];
        R[q][2] = r[2];
    }
    // drive: sin(2 pi (t / T + phase / 2 pi)), argument reduced in FP64
    const double tt = (double)c.ctl->step * sw.inv_period;
    float fd[3];
    for (int q = 0; q < 3; q += 2) {
        const double x = tt + sw.phase_turns[q];
        fd[q] = sw.amp[q] * sinpif(2.0f * (float)(x - floor(x)));
    }
    if (sw.balance) {
        fd[1] = -fd[0] - fd[2];
    } else {
        const double x = tt + sw.phase_turns[1];
        fd[1] = sw.amp[1] * sinpif(2.0f * (float)(x - floor(x)));
    }
    // springs: |d| - L = (|d|^2 - L^2) / (|d| + L), the difference in FP64
    float fs[3][3];
    for (int q = 0; q < 3; q += 2) {
        const double dx = R[q][0] - R[1][0], dy = R[q][1] - R[1][1], dz = R[q][2] - R[1][2];
        const double n2 = fma(dx, dx, fma(dy, dy, dz * dz));
        const float nf = sqrtf((float)n2);
        const float stretch = (float)(n2 - sw.L2) / (nf + (float)sw.L);
        const float m = -(float)sw.k * stretch / nf;
        fs[q][0] = m * (float)dx;
        fs[q][1] = m * (float)dy;
        fs[q][2] = m * (float)dz;
    }
    for (int a = 0; a < 3; ++a) fs[1][a] = -fs[0][a] - fs[2][a];
    for (int q = 0; q < 3; ++q) {
        const float inv = c.beads[sw.bead[q]].inv_count;
        c.bead_ext[sw.bead[q]] = make_float4((fd[q] + fs[q][0]) * inv, fs[q][1] * inv, fs[q][2] * inv, 0.f);
    }
}

// Enclosed volume of a bead by the divergence theorem, V = sum over its
// triangles of (1/6) p0 . (p1 x p2) with p = r - R_b: each triangle adds its
// term in FP64, rounded to VOL_FIX units, to the bead's sum (integer adds:
// the same result in any order); the corners keep dV/dr = (1/6) p_next x
// p_prev for the nodal forces.  Called by every lane of a warp (active: this
// lane has a triangle).
__device__ __forceinline__ void triangle_volume(const DevCtx &c, int t, bool active) {
    long long q = 0;
    int b = -1;
    if (active) {
        const TriDev T = c.tris[t];
        b = c.node_bead[T.v[0]];
        if (c.beads[b].kv > 0.f) {
            const double *R = c.bead_R + 4 * b;
            double p[3][3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                p[k][0] = c.rx[T.v[k]] - R[0];
                p[k][1] = c.ry[T.v[k]] - R[1];
                p[k][2] = c.rz[T.v[k]] - R[2];
            }
            const double v = p[0][0] * (p[1][1] * p[2][2] - p[1][2] * p[2][1]) +
                             p[0][1] * (p[1][2] * p[2][0] - p[1][0] * p[2][2]) +
                             p[0][2] * (p[1][0] * p[2][1] - p[1][1] * p[2][0]);
            q = __double2ll_rn(v * (VOL_FIX / 6.0));
            float4 *g = c.tri_vgrad + 3 * (size_t)t;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
                const float ux = (float)p[k1][0], uy = (float)p[k1][1], uz = (float)p[k1][2];
                const float wx = (float)p[k2][0], wy = (float)p[k2][1], wz = (float)p[k2][2];
                g[k] = make_float4((uy * wz - uz * wy) * (1.0f / 6.0f), (uz * wx - ux * wz) * (1.0f / 6.0f),
                                   (ux * wy - uy * wx) * (1.0f / 6.0f), 0.f);
            }
        } else {
            b = -1;
        }
    }
    // one atomic per warp when its lanes hold triangles of one bead (the usual case)
    const int b0 = __shfl_sync(0xffffffffu, b, 0);
    long long *acc = c.bead_Vfix;
    if (__all_sync(0xffffffffu, b == b0)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        if ((threadIdx.x & 31) == 0 && b0 >= 0)
            atomicAdd(reinterpret_cast<unsigned long long *>(acc + b0), (unsigned long long)q);
    } else if (b >= 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(acc + b), (unsigned long long)q);
    }
}

__device__ void triangle_forces(const DevCtx &c, int t) {
    const TriDev T = c.tris[t];
    const int n0 = T.v[0], n1 = T.v[1], n2 = T.v[2];
    const double x0 = c.rx[n0], y0 = c.ry[n0], z0 = c.rz[n0];
    const double ax = c.rx[n1] - x0, ay = c.ry[n1] - y0, az = c.rz[n1] - z0;
    const double bx = c.rx[n2] - x0, by = c.ry[n2] - y0, bz = c.rz[n2] - z0;
    const float E00 = (float)(0.5 * (fma(ax, ax, fma(ay, ay, az * az)) - T.G[0]));
    const float E01 = (float)(0.5 * (fma(ax, bx, fma(ay, by, az * bz)) - T.G[1]));
    const float E11 = (float)(0.5 * (fma(bx, bx, fma(by, by, bz * bz)) - T.G[2]));
    const float trM = T.Gi[0] * E00 + 2.0f * T.Gi[1] * E01 + T.Gi[2] * E11;
    const float detM = (E00 * E11 - E01 * E01) * T.inv_detG;
    const float I2 = 2.0f * trM + 4.0f * detM;
    // dW/dd = d S with S = K [cG adj(G) + cE adj(E)], K = A0 modulus / det G:
    //   neo-Hookean: cG = I2 (I2 + 2) / J^4, cE = -2 / J^4 (J^2 = 1 + I2);
    //   Skalak:      cG = I1 + C I2,       cE = 2 (C I2 - 1)  (I1 = 2 tr M)
    float cG, cE;
    if (T.law == LBIB_SKALAK) {
        const float I1 = 2.0f * trM;
        cG = I1 + T.skC * I2;
        cE = 2.0f * (T.skC * I2 - 1.0f);
    } else {
        const float J2 = 1.0f + I2;
        const float iJ4 = 1.0f / (J2 * J2);
        cG = I2 * (I2 + 2.0f) * iJ4;
        cE = -2.0f * iJ4;
    }
    const float S00 = T.K * (cG * (float)T.G[2] + cE * E11);
    const float S01 = T.K * (-cG * (float)T.G[1] - cE * E01);
    const float S11 = T.K * (cG * (float)T.G[0] + cE * E00);
    const float d1x = (float)ax, d1y = (float)ay, d1z = (float)az;
    const float d2x = (float)bx, d2y = (float)by, d2z = (float)bz;
    // dW/dd1 = d1 S00 + d2 S01, dW/dd2 = d1 S01 + d2 S11
    const float w1x = d1x * S00 + d2x * S01, w1y = d1y * S00 + d2y * S01, w1z = d1z * S00 + d2z * S01;
    const float w2x = d1x * S01 + d2x * S11, w2y = d1y * S01 + d2y * S11, w2z = d1z * S01 + d2z * S11;
    float4 *o = c.tri_force + 3 * (size_t)t;
    o[0] = make_float4(w1x + w2x, w1y + w2y, w1z + w2z, 0.f);
    o[1] = make_float4(-w1x, -w1y, -w1z, 0.f);
    o[2] = make_float4(-w2x, -w2y, -w2z, 0.f);
}

// Bending of one edge (Sec. 2.2, Kantor-Nelson discretisation of the
// Helfrich energy): W = kb (1 - cos(theta - theta0)), theta the angle from the
// normal n1 of triangle (a, b, c) to the normal n2 of triangle (b, a, d) about
// the edge direction, so f_k = -kb sin(theta - theta0) dtheta/dr_k with the
// angle's gradient for the two wings and the edge nodes
//   dtheta/dc = -|e| n1 / |N1|,  dtheta/dd = -|e| n2 / |N2|,
//   dtheta/da = -(1 - s) dtheta/dc - (1 - s') dtheta/dd,
//   dtheta/db = -s dtheta/dc - s' dtheta/dd,
// e = b - a and s, s' the positions of c and d projected onto the edge in
// units of |e|.  Positions are taken relative to a in FP64, the rest in FP32.
__device__ void edge_forces(const DevCtx &c, int k) {
    const EdgeDev Ed = c.edges[k];
    const int a = Ed.v[0];
    const double ox = c.rx[a], oy = c.ry[a], oz = c.rz[a];
    float P[3][3];  // b, c, d relative to a
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int n = Ed.v[q + 1];
        P[q][0] = (float)(c.rx[n] - ox);
        P[q][1] = (float)(c.ry[n] - oy);
        P[q][2] = (float)(c.rz[n] - oz);
    }
    const float ex = P[0][0], ey = P[0][1], ez = P[0][2];
    const float ux = P[1][0], uy = P[1][1], uz = P[1][2];                          // c - a
    const float wx = P[2][0] - ex, wy = P[2][1] - ey, wz = P[2][2] - ez;          // d - b
    // N1 = e x (c - a), N2 = (d - b) x e
    const float N1x = ey * uz - ez * uy, N1y = ez * ux - ex * uz, N1z = ex * uy - ey * ux;
    const float N2x = wy * ez - wz * ey, N2y = wz * ex - wx * ez, N2z = wx * ey - wy * ex;
    const float le2 = ex * ex + ey * ey + ez * ez;
    const float il1 = rsqrtf(N1x * N1x + N1y * N1y + N1z * N1z);
    const float il2 = rsqrtf(N2x * N2x + N2y * N2y + N2z * N2z);
    const float ile = rsqrtf(le2);
    const float m1x = N1x * il1, m1y = N1y * il1, m1z = N1z * il1;
    const float m2x = N2x * il2, m2y = N2y * il2, m2z = N2z * il2;
    const float cth = m1x * m2x + m1y * m2y + m1z * m2z;
    const float sth = ((m1y * m2z - m1z * m2y) * ex + (m1z * m2x - m1x * m2z) * ey + (m1x * m2y - m1y * m2x) * ez) * ile;
    // -dW/dtheta
    const float g = -Ed.kb * (sth * Ed.c0 - cth * Ed.s0);
    const float le = le2 * ile;
    const float hc = -le * il1, hd = -le * il2;  // dtheta/dc = hc n1, dtheta/dd = hd n2
    const float s1 = (ux * ex + uy * ey + uz * ez) / le2;
    const float s2 = (P[2][0] * ex + P[2][1] * ey + P[2][2] * ez) / le2;
    const float gcx = hc * m1x, gcy = hc * m1y, gcz = hc * m1z;
    const float gdx = hd * m2x, gdy = hd * m2y, gdz = hd * m2z;
    float4 *o = c.tri_force + 3 * (size_t)c.n_tris + 4 * (size_t)k;
    o[0] = make_float4(g * (-(1.f - s1) * gcx - (1.f - s2) * gdx), g * (-(1.f - s1) * gcy - (1.f - s2) * gdy),
                       g * (-(1.f - s1) * gcz - (1.f - s2) * gdz), 0.f);
    o[1] = make_float4(g * (-s1 * gcx - s2 * gdx), g * (-s1 * gcy - s2 * gdy), g * (-s1 * gcz - s2 * gdz), 0.f);
    o[2] = make_float4(g * gcx, g * gcy, g * gcz, 0.f);
    o[3] = make_float4(g * gdx, g * gdy, g * gdz, 0.f);
}

// blocks of k_ib_prepare: swimmers, then triangles, then bending edges
__device__ __forceinline__ void prepare_body(const DevCtx &c, int bid) {
    // the other parity's tile list (the previous step's) is consumed: empty it
    // for the marks of the next step
    if (bid == 0 && threadIdx.x == 0) c.tile_count[(c.ctl->step + 1) & 1] = 0;
    const int tri_blocks = (c.n_tris + PREP_TPB - 1) / PREP_TPB;
    if (bid < c.n_swimmers) {
        swimmer_forces(c, bid);
    } else if (bid < c.n_swimmers + tri_blocks) {
        const int t = (bid - c.n_swimmers) * PREP_TPB + threadIdx.x;
        if (t < c.n_tris) triangle_forces(c, t);
        if (c.has_volume) triangle_volume(c, t, t < c.n_tris);
    } else {
        const int k = (bid - c.n_swimmers - tri_blocks) * PREP_TPB + threadIdx.x;
        if (k < c.n_edges) edge_forces(c, k);
    }
}

__global__ void __launch_bounds__(PREP_TPB) k_ib_prepare(const DevCtx c) { prepare_body(c, blockIdx.x); }

// Bead centres from the positions (FP64 mean, fixed order); clears the
// pending advection marks.
__global__ void __launch_bounds__(PREP_TPB) k_bead_init(const DevCtx c) {
    __shared__ double sm[96];
    const int b = blockIdx.x;
    const BeadDev bd = c.beads[b];
    double a = 0.0, bb = 0.0, cc = 0.0;
    for (int j = bd.node_start + threadIdx.x; j < bd.node_start + bd.node_count; j += blockDim.x) {
        a += c.rx[j];
        bb += c.ry[j];
        cc += c.rz[j];
    }
    block_sum3(a, bb, cc, sm);
    if (threadIdx.x == 0) {
        double *R = c.bead_R + 4 * b;
        R[0] = a / bd.node_count;
        R[1] = bb / bd.node_count;
        R[2] = cc / bd.node_count;
    }
}

template <int KW, bool DET>
__device__ __forceinline__ void gather_spread_body(const DevCtx &c, int bid) {
    __shared__ float4 sf[GS_NODES];
    __shared__ int so[GS_NODES][3];
    __shared__ float sw[GS_NODES][3][KW];
    const int j0 = bid * GS_NODES;
    const int nloc = min(GS_NODES, c.n_nodes - j0);
    if ((int)threadIdx.x < nloc) {
        const int j = j0 + threadIdx.x;
        float fx = 0.f, fy = 0.f, fz = 0.f;
        const int e0 = c.csr_ptr[j], e1 = c.csr_ptr[j + 1];
        // up to 8 incident corners with independent loads, in list order
        int ent[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) ent[k] = e0 + k < e1 ? c.csr_ent[e0 + k] : -1;
        float4 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = ent[k] >= 0 ? c.tri_force[ent[k]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            fx += v[k].x;
            fy += v[k].y;
            fz += v[k].z;
        }
        for (int e = e0 + 8; e < e1; ++e) {
            const float4 w = c.tri_force[c.csr_ent[e]];
            fx += w.x;
            fy += w.y;
            fz += w.z;
        }
        const int bj = c.node_bead[j];
        if (c.has_volume && c.beads[bj].kv > 0.f) {
            // volume penalty (Sec. 2.2, Eq. vol_cons): f_j = -kv (V - V0) / V0 dV/dr_j,
            // dV/dr_j summed over the node's triangle corners in list order
            const BeadDev bd = c.beads[bj];
            const double V = (double)c.bead_Vfix[bj] * (1.0 / VOL_FIX);
            const float fac = (float)(-(double)bd.kv * (V - bd.V0) / bd.V0);
            float gx = 0.f, gy = 0.f, gz = 0.f;
            for (int e = e0; e < e1; ++e) {
                const int en = c.csr_ent[e];
                if (en >= 3 * c.n_tris) break;  // the node's bending-edge entries follow its triangle corners
                const float4 w = c.tri_vgrad[en];
                gx += w.x;
                gy += w.y;
                gz += w.z;
            }
            fx += fac * gx;
            fy += fac * gy;
            fz += fac * gz;
        }
        const float4 ext = c.bead_ext[bj];
        const float4 f = make_float4(fx + ext.x, fy + ext.y, fz + ext.z, 0.f);
        sf[threadIdx.x] = f;
        c.node_force[j] = f;
        float fr;
        so[threadIdx.x][0] = stencil_axis(c.rx[j], c.nx, KW, fr);
        weights1d<KW>(fr, sw[threadIdx.x][0]);
        so[threadIdx.x][1] = stencil_axis(c.ry[j], c.ny, KW, fr);
        weights1d<KW>(fr, sw[threadIdx.x][1]);
        so[threadIdx.x][2] = stencil_axis(c.rz[j], c.nz, KW, fr);
        weights1d<KW>(fr, sw[threadIdx.x][2]);
    }
    // deterministic mode: the block's fixed-point contributions are summed
    // per cell in a shared hash table first (integer sums: the same result in
    // any order), then added to the field once per distinct cell; neighbouring
    // nodes share most of their stencil cells
    unsigned *hk = nullptr;
    unsigned long long (*hv)[3] = nullptr;
    if constexpr (DET) {
        __shared__ unsigned s_hk[GS_HT];
        __shared__ unsigned long long s_hv[GS_HT][3];
        hk = s_hk;
        hv = s_hv;
        for (int i = threadIdx.x; i < GS_HT; i += blockDim.x) {
            s_hk[i] = GS_HT_EMPTY;
            s_hv[i][0] = s_hv[i][1] = s_hv[i][2] = 0ull;
        }
    }
    __syncthreads();
    constexpr int ROWS = KW * KW;
    const int nx = c.nx, ny = c.ny, nz = c.nz;
    const int stamp = (int)c.ctl->step;
    const int *marks = c.marks + (size_t)(stamp & 1) * c.n_tiles;
    bool unmarked = false;
    for (int task = threadIdx.x; task < nloc * ROWS; task += GS_TPB) {
        const int ln = task / ROWS, row = task % ROWS;
        const int dy = row % KW, dz = row / KW;
        const int ox = so[ln][0];
        const int yy = (so[ln][1] + dy) % ny, zz = (so[ln][2] + dz) % nz;  // boxes may be narrower than the stencil
        const float wyz = sw[ln][1][dy] * sw[ln][2][dz];
        const float4 f = sf[ln];
        const unsigned rowbase = (unsigned)nx * ((unsigned)yy + (unsigned)ny * (unsigned)zz);
        // the marked region of this step must cover every cell the stencil touches
        const int trow = c.tiles_x * (yy + ny * zz);
        unmarked |= (marks[ox / c.tile_x + trow] != stamp) | (marks[((ox + KW - 1) % nx) / c.tile_x + trow] != stamp);
#pragma unroll
        for (int k = 0; k < KW; ++k) {
            const int xx = (ox + k) % nx;
            const unsigned cell = rowbase + (unsigned)xx;
            const float w = sw[ln][0][k] * wyz;
            if (DET) {
                // the FP32 contribution scaled by 2^48 (exact) and rounded to the
                // nearest integer: no FP64 arithmetic, which is slow on this GPU
                const unsigned long long q[3] = {(unsigned long long)__float2ll_rn((w * f.x) * FIX_SCALE_F),
                                                 (unsigned long long)__float2ll_rn((w * f.y) * FIX_SCALE_F),
                                                 (unsigned long long)__float2ll_rn((w * f.z) * FIX_SCALE_F)};
                // linear probing, bounded: a full neighbourhood goes straight to the field
                unsigned h = (cell * 2654435761u) >> (32 - GS_HT_BITS);
                bool held = false;
                for (int pr = 0; pr < GS_HT_PROBES; ++pr) {
                    const unsigned old = atomicCAS(&hk[h], GS_HT_EMPTY, cell);
                    if (old == GS_HT_EMPTY || old == cell) {
                        held = true;
                        break;
                    }
                    h = (h + 1) & (GS_HT - 1);
                }
                for (int a = 0; a < 3; ++a) {
                    if (held) atomicAdd(&hv[h][a], q[a]);
                    else atomicAdd(&c.Fdet[(size_t)a * c.Npad + cell], q[a]);
                }
            } else {
                atomicAdd(&c.F[cell], make_float4(w * f.x, w * f.y, w * f.z, 0.f));
            }
        }
    }
    if constexpr (DET) {
        __syncthreads();
        for (int i = threadIdx.x; i < GS_HT; i += blockDim.x) {
            const unsigned cell = hk[i];
            if (cell == GS_HT_EMPTY) continue;
            for (int a = 0; a < 3; ++a)
                if (hv[i][a] != 0ull) atomicAdd(&c.Fdet[(size_t)a * c.Npad + cell], hv[i][a]);
        }
    }
    if (__any_sync(0xffffffffu, unmarked) && (threadIdx.x & 31) == 0) atomicOr(&c.ctl->err, ERR_MARK);
    if (c.has_volume) {
        // the last block to finish clears the bead volumes for the next
        // k_ib_prepare (a completion count, no waiting)
        __shared__ int s_vlast;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0)
            s_vlast = atomicAdd(&c.ctl->vol_done, 1) == (c.n_nodes + GS_NODES - 1) / GS_NODES - 1;
        __syncthreads();
        if (s_vlast) {
            for (int i = threadIdx.x; i < c.n_beads; i += blockDim.x) c.bead_Vfix[i] = 0;
            if (threadIdx.x == 0) c.ctl->vol_done = 0;
        }
    }
}

template <int KW, bool DET>
__global__ void __launch_bounds__(GS_TPB) k_ib_gather_spread(const DevCtx c) { gather_spread_body<KW, DET>(c, blockIdx.x); }

// Fold an advection into the bead centres: R_b += mean_j v_j (the mean is
// linear, so this keeps R_b the centre of mass of its nodes, Fig. 1 caption).
// The blocks of the interpolation have summed their nodes' velocities into
// bead_acc in fixed point (2^-48 units, exact integer sums); one thread per
// bead takes and clears its sums.  Run by one block.
__device__ void fold_bead_velocities(const DevCtx &c) {
    for (int b = threadIdx.x; b < c.n_beads; b += blockDim.x) {
        const double inv = 1.0 / c.beads[b].node_count;
        double *R = c.bead_R + 4 * b;
        double v[3];
        for (int a = 0; a < 3; ++a) {
            const long long q = (long long)atomicExch(&c.bead_acc[3 * b + a], 0ull);
            v[a] = (double)q * FIX_INV * inv;
            R[a] += v[a];
        }
        c.bead_V[b] = make_float4((float)v[0], (float)v[1], (float)v[2], 0.f);
    }
}

// Stamp, with step number `stamp`, the tiles of the KW x KW stencil rows of
// plane z = oz + l of a node whose stencil origin is (ox, oy, oz); a tile is
// appended to its parity's list by the thread that changes its stamp.
template <int KW>
__device__ __forceinline__ void mark_stencil_plane(const DevCtx &c, int ox, int oy, int oz, int l, int stamp) {
    const int p = stamp & 1;
    int *marks = c.marks + (size_t)p * c.n_tiles;
    const int zz = (oz + l) % c.nz;
    const int t0 = ox / c.tile_x, t1 = ((ox + KW - 1) % c.nx) / c.tile_x;
    int tile[2 * KW];
    int old[2 * KW];
#pragma unroll
    for (int dy = 0; dy < KW; ++dy) {
        const int trow = c.tiles_x * ((oy + dy) % c.ny + c.ny * zz);
        tile[2 * dy] = t0 + trow;
        tile[2 * dy + 1] = t1 + trow;
    }
#pragma unroll
    for (int k = 0; k < 2 * KW; ++k) old[k] = marks[tile[k]];
    // neighbouring nodes share most of their tiles: of the lanes of this warp
    // that would stamp the same tile, only the lowest does the atomic
    const unsigned act = __activemask();
#pragma unroll
    for (int k = 0; k < 2 * KW; ++k) {
        const bool want = !((k & 1) && tile[k] == tile[k - 1])  // both ends of the row in one tile
                          && old[k] != stamp;
        const unsigned wm = __ballot_sync(act, want);
        if (want) {
            const unsigned peers = __match_any_sync(wm, tile[k]);
            if ((int)(threadIdx.x & 31) == __ffs(peers) - 1 && atomicExch(&marks[tile[k]], stamp) != stamp)
                c.tile_list[(size_t)p * c.n_tiles + atomicAdd(&c.tile_count[p], 1)] = tile[k];
        }
    }
}

// Stamp the tiles of every node's stencil for the current step (KW lanes per node).
template <int KW>
__global__ void __launch_bounds__(INT_TPB) k_ib_mark(const DevCtx c) {
    const int gt = blockIdx.x * INT_TPB + threadIdx.x;
    const int j = gt / KW, l = gt % KW;
    if (j >= c.n_nodes) return;
    float fr;
    const int ox = stencil_axis(c.rx[j], c.nx, KW, fr), oy = stencil_axis(c.ry[j], c.ny, KW, fr),
              oz = stencil_axis(c.rz[j], c.nz, KW, fr);
    mark_stencil_plane<KW>(c, ox, oy, oz, l, (int)c.ctl->step);
    if (gt == 0) c.ctl->gen[c.ctl->step & 1] = (int)c.ctl->step;
}

// KW lanes per node, lane l gathering the KW x KW cells of stencil plane
// z = oz + l; the lanes' partial sums are reduced with shuffles in a fixed
// order.  With ADVECT, lane 0 moves the node (FP64) and, if mark_parity >= 0,
// the lanes mark the tiles of the moved node's stencil for the next step.
template <int KW, bool ADVECT>
__device__ __forceinline__ void interp_body(const DevCtx &c, int bid, int nblk, float *vel_out, int mark_parity) {
    const int gt = bid * INT_TPB + threadIdx.x;
    const int j = gt / KW, l = gt % KW;
    const bool active = j < c.n_nodes;
    const int nx = c.nx, ny = c.ny, nz = c.nz;
    double px = 0.0, py = 0.0, pz = 0.0;
    float vx = 0.f, vy = 0.f, vz = 0.f;
    // fixed-point sums of this block's node velocities per bead (bead index
    // minus that of the block's first node), flushed once per block: the
    // bead-velocity means need no serial pass over the nodes afterwards
    constexpr int SLOTS = INT_TPB / KW;
    __shared__ unsigned long long s_acc[SLOTS][3];
    __shared__ int s_b0;
    const bool fold = ADVECT && mark_parity >= 0;
    if (fold) {
        for (int i = threadIdx.x; i < 3 * SLOTS; i += blockDim.x) s_acc[i / 3][i % 3] = 0ull;
        if (threadIdx.x == 0) s_b0 = bid * SLOTS < c.n_nodes ? c.node_bead[bid * SLOTS] : 0;
        __syncthreads();
    }
    if (active) {
        px = c.rx[j];
        py = c.ry[j];
        pz = c.rz[j];
        float fx, fy, fz;
        const int ox = stencil_axis(px, nx, KW, fx), oy = stencil_axis(py, ny, KW, fy), oz = stencil_axis(pz, nz, KW, fz);
        float wx[KW], wy[KW], wz[KW];
        weights1d<KW>(fx, wx);
        weights1d<KW>(fy, wy);
        weights1d<KW>(fz, wz);
        float wzl = wz[0];
#pragma unroll
        for (int k = 1; k < KW; ++k)
            if (l == k) wzl = wz[k];
        const unsigned zoff = (unsigned)nx * (unsigned)ny * (unsigned)((oz + l) % nz);
#pragma unroll
        for (int dy = 0; dy < KW; ++dy) {
            const unsigned rowbase = zoff + (unsigned)nx * (unsigned)((oy + dy) % ny);
            const float wyz = wy[dy] * wzl;
#pragma unroll
            for (int k = 0; k < KW; ++k) {
                const float4 u = c.U[rowbase + (unsigned)((ox + k) % nx)];
                const float w = wx[k] * wyz;
                vx += w * u.x;
                vy += w * u.y;
                vz += w * u.z;
            }
        }
    }
    // fixed-order reduction over the KW lanes of this node (aligned groups within a warp)
#pragma unroll
    for (int s = KW / 2; s > 0; s >>= 1) {
        vx += __shfl_xor_sync(0xffffffffu, vx, s);
        vy += __shfl_xor_sync(0xffffffffu, vy, s);
        vz += __shfl_xor_sync(0xffffffffu, vz, s);
    }
    if (active && l == 0) {
        if (vel_out) {
            vel_out[3 * j + 0] = vx;
            vel_out[3 * j + 1] = vy;
            vel_out[3 * j + 2] = vz;
        }
        if (ADVECT) {
            // front tracking (Sec. 2.3): r <- r + rdot (dt = 1) in FP64
            px += (double)vx;
            py += (double)vy;
            pz += (double)vz;
            c.rx[j] = px;
            c.ry[j] = py;
            c.rz[j] = pz;
            c.node_vel[j] = make_float4(vx, vy, vz, 0.f);
            const float sp2 = vx * vx + vy * vy + vz * vz;
            if (!isfinite(sp2) || !isfinite(px + py + pz)) atomicOr(&c.ctl->err, ERR_NONFINITE);
            else if (sp2 > 0.01f) atomicOr(&c.ctl->err, ERR_UNSTABLE);
            if (fold) {
                const int b = c.node_bead[j], sl = b - s_b0;
                const unsigned long long q[3] = {(unsigned long long)__float2ll_rn(vx * FIX_SCALE_F),
                                                 (unsigned long long)__float2ll_rn(vy * FIX_SCALE_F),
                                                 (unsigned long long)__float2ll_rn(vz * FIX_SCALE_F)};
                for (int a = 0; a < 3; ++a) {
                    if (sl >= 0 && sl < SLOTS) atomicAdd(&s_acc[sl][a], q[a]);
                    else atomicAdd(&c.bead_acc[3 * b + a], q[a]);
                }
            }
        }
    }
    if (ADVECT && mark_parity >= 0) {
        // stamp the tiles of the moved node's stencil for the next step
        const int next = (int)c.ctl->step + 1;
        const int gbase = (threadIdx.x & 31) & ~(KW - 1);
        px = __shfl_sync(0xffffffffu, px, gbase);
        py = __shfl_sync(0xffffffffu, py, gbase);
        pz = __shfl_sync(0xffffffffu, pz, gbase);
        if (active) {
            float fr;
            const int ox = stencil_axis(px, nx, KW, fr), oy = stencil_axis(py, ny, KW, fr), oz = stencil_axis(pz, nz, KW, fr);
            mark_stencil_plane<KW>(c, ox, oy, oz, l, next);
        }
        // the block's bead sums into the global accumulators (integer sums:
        // the same result in any order)
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * SLOTS; i += blockDim.x) {
            const unsigned long long v = s_acc[i / 3][i % 3];
            if (v != 0ull) atomicAdd(&c.bead_acc[3 * (s_b0 + i / 3) + i % 3], v);
        }
        // the last block to finish folds the step's velocities into the bead
        // centres and closes the step (a completion count, no waiting)
        __shared__ int s_last;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = atomicAdd(&c.ctl->done, 1) == nblk - 1;
        __syncthreads();
        if (s_last) {
            __threadfence();
            fold_bead_velocities(c);
            __syncthreads();
            // a drive period ends with this step: record x_cm (mean of the
            // three bead centres) for the period-averaged velocity (Sec. 3)
            // this step's trajectory points, slot (next - 1) mod LBIB_TRACK_STEPS:
            // one thread per (swimmer, field) of the 22 fields of a point
            {
                lbib_track_point *tp = c.track + (size_t)((next - 1) % LBIB_TRACK_STEPS) * c.n_swimmers;
                for (int i = threadIdx.x; i < 22 * c.n_swimmers; i += blockDim.x) {
                    const int sw = i / 22, f = i % 22;
                    const SwimDev d = c.swims[sw];
                    if (f == 0) {
                        tp[sw].step = next;
                    } else if (f < 4) {
                        const int a = f - 1;
                        tp[sw].x_cm[a] = (c.bead_R[4 * d.bead[0] + a] + c.bead_R[4 * d.bead[1] + a] +
                                          c.bead_R[4 * d.bead[2] + a]) / 3.0;
                    } else if (f < 13) {
                        const int q = (f - 4) / 3, a = (f - 4) % 3;
                        tp[sw].R[q][a] = c.bead_R[4 * d.bead[q] + a];
                    } else {
                        const int q = (f - 13) / 3, a = (f - 13) % 3;
                        const float4 V = c.bead_V[d.bead[q]];
                        tp[sw].V[q][a] = a == 0 ? V.x : (a == 1 ? V.y : V.z);
                    }
                }
            }
            for (int sw = threadIdx.x; sw < c.n_swimmers; sw += blockDim.x) {
                const SwimDev d = c.swims[sw];
                if (floor((double)next / d.period) > floor((double)(next - 1) / d.period)) {
                    double *rec = c.sw_period + 8 * sw;
                    for (int a = 0; a < 3; ++a) {
                        const double x = (c.bead_R[4 * d.bead[0] + a] + c.bead_R[4 * d.bead[1] + a] +
                                          c.bead_R[4 * d.bead[2] + a]) / 3.0;
                        rec[3 + a] = rec[a];
                        rec[a] = x;
                    }
                    rec[6] += 1.0;
                }
            }
            if (threadIdx.x == 0) {
                c.ctl->done = 0;
                c.ctl->gen[next & 1] = next;
                c.ctl->step = next;
            }
        }
    }
}

template <int KW, bool ADVECT>
__global__ void __launch_bounds__(INT_TPB) k_ib_interp(const DevCtx c, float *vel_out, int mark_parity) {
    interp_body<KW, ADVECT>(c, blockIdx.x, gridDim.x, vel_out, mark_parity);
}

// Observables, part 1: one block per (swimmer, bead), sums in a fixed order.
// The centre is the FP64 mean of the node positions.  The bead force
// F_b = sum_j f_j and torque T_b = sum_j (r_j - R_b) x f_j are summed in FP64:
// the membrane forces cancel over a bead (translation and rotation invariance
// of the strain energy, Sec. 2.2), so F_b (the drive plus the springs) is a
// small remainder of much larger node forces and T_b a remainder near zero;
// an FP32 sum would lose the digits that are left.  The mean bead velocity
// stays an FP32 sum like the FP32 node velocities it comes from.
__global__ void __launch_bounds__(PREP_TPB) k_swimmer_beads(const DevCtx c) {
    __shared__ double smd[96];
    __shared__ float smf[96];
    const int s = blockIdx.x / 3, q = blockIdx.x % 3;
    const SwimDev sw = c.swims[s];
    lbib_swimmer_state *st = c.sw_state + s;
    const BeadDev bd = c.beads[sw.bead[q]];
    const int j0 = bd.node_start, j1 = bd.node_start + bd.node_count;
    const double inv = 1.0 / bd.node_count;
    double a = 0.0, b = 0.0, cc = 0.0;
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        a += c.rx[j];
        b += c.ry[j];
        cc += c.rz[j];
    }
    block_sum3(a, b, cc, smd);
    const double R0 = a * inv, R1 = b * inv, R2 = cc * inv;
    float va = 0.f, vb = 0.f, vc = 0.f;
    double fa = 0.0, fb = 0.0, fc = 0.0, ta = 0.0, tb = 0.0, tc = 0.0;
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const float4 v = c.node_vel[j];
        const float4 f = c.node_force[j];
        const double dx = c.rx[j] - R0, dy = c.ry[j] - R1, dz = c.rz[j] - R2;
        const double gx = f.x, gy = f.y, gz = f.z;
        va += v.x;
        vb += v.y;
        vc += v.z;
        fa += gx;
        fb += gy;
        fc += gz;
        ta += dy * gz - dz * gy;
        tb += dz * gx - dx * gz;
        tc += dx * gy - dy * gx;
    }
    block_sum3(va, vb, vc, smf);
    block_sum3(fa, fb, fc, smd);
    block_sum3(ta, tb, tc, smd);
    if (threadIdx.x == 0) {
        st->R[q][0] = R0;
        st->R[q][1] = R1;
        st->R[q][2] = R2;
        st->V[q][0] = va * inv;
        st->V[q][1] = vb * inv;
        st->V[q][2] = vc * inv;
        st->F[q][0] = fa;
        st->F[q][1] = fb;
        st->F[q][2] = fc;
        st->T[q][0] = ta;
        st->T[q][1] = tb;
        st->T[q][2] = tc;
    }
}

// Observables, part 2: one thread per swimmer, from its three bead records.
__global__ void k_swimmer_finish(const DevCtx c, int init) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= c.n_swimmers) return;
    const SwimDev sw = c.swims[s];
    lbib_swimmer_state *st = c.sw_state + s;
    st->step = c.ctl->step;
    double *rec = c.sw_period + 8 * s;
    for (int a = 0; a < 3; ++a) {
        const double x = (st->R[0][a] + st->R[1][a] + st->R[2][a]) / 3.0;
        st->x_cm[a] = x;
        if (init) {
            c.xcm0[3 * s + a] = x;
            rec[a] = rec[3 + a] = x;  // t = 0 is the first period boundary
        }
        st->disp[a] = x - c.xcm0[3 * s + a];
    }
    if (init) rec[6] = 0.0;
    // period-averaged swimming velocity (Sec. 3, Eq. vel_swim) and the
    // Reynolds numbers with nu = (tau - 1/2)/3 and a the rest radius
    st->periods = (long long)rec[6];
    const double nu = ((double)c.tau - 0.5) / 3.0;
    double vv = 0.0;
    for (int a = 0; a < 3; ++a) {
        st->v_period[a] = rec[6] >= 1.0 ? (rec[a] - rec[3 + a]) / sw.period : 0.0;
        vv += st->v_period[a] * st->v_period[a];
    }
    const double rad = (double)c.beads[sw.bead[0]].reach - 1.0;
    double ls2 = 0.0, vb = 0.0;
    for (int a = 0; a < 3; ++a) ls2 += (st->R[2][a] - st->R[0][a]) * (st->R[2][a] - st->R[0][a]);
    for (int q = 0; q < 3; ++q)
        vb = fmax(vb, sqrt(st->V[q][0] * st->V[q][0] + st->V[q][1] * st->V[q][1] + st->V[q][2] * st->V[q][2]));
    st->re_swim = sqrt(vv) * (sqrt(ls2) + 2.0 * rad) / nu;
    st->re_bead = vb * rad / nu;
}

// ---------------------------------------------------------------- batches
// One launch serves every box of a batch: block b of the launch belongs to the
// box whose prefix range [off[box], off[box + 1]) holds b, and runs that box's
// code with its local block index.
__device__ __forceinline__ int batch_box(const int *off, int n, int b) {
    int lo = 0, hi = n;  // off[lo] <= b < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= b) lo = mid;
        else hi = mid;
    }
    return lo;
}

// The batched immersed-boundary kernels walk their virtual blocks (the
// blocks each box would launch alone) with a grid of at most a few blocks per
// SM, so that the chain of many boxes, which runs at high priority beside the
// main fluid launches, holds a bounded share of every SM.
__global__ void __launch_bounds__(PREP_TPB) k_ib_prepare_batch(const BatchDev bt) {
    for (int vb = blockIdx.x; vb < bt.blocks_prep; vb += gridDim.x) {
        const int b = batch_box(bt.off_prep, bt.n_boxes, vb);
        prepare_body(bt.boxes[b], vb - bt.off_prep[b]);
    }
}

template <int KW, bool DET>
__global__ void __launch_bounds__(GS_TPB) k_ib_gather_spread_batch(const BatchDev bt) {
    for (int vb = blockIdx.x; vb < bt.blocks_gs; vb += gridDim.x) {
        const int b = batch_box(bt.off_gs, bt.n_boxes, vb);
        gather_spread_body<KW, DET>(bt.boxes[b], vb - bt.off_gs[b]);
        __syncthreads();  // the shared node tables are refilled by the next virtual block
    }
}

template <int KW>
__global__ void __launch_bounds__(INT_TPB) k_ib_interp_batch(const BatchDev bt) {
    for (int vb = blockIdx.x; vb < bt.blocks_int; vb += gridDim.x) {
        const int b = batch_box(bt.off_int, bt.n_boxes, vb);
        const DevCtx &c = bt.boxes[b];
        interp_body<KW, true>(c, vb - bt.off_int[b], bt.off_int[b + 1] - bt.off_int[b], nullptr,
                              (int)((c.ctl->step + 1) & 1));
        __syncthreads();  // shared accumulators and the last-block flag are reused
    }
}

static int batch_ib_grid(const BatchDev &bt, int blocks) {
    return bt.ib_grid_cap > 0 && blocks > bt.ib_grid_cap ? bt.ib_grid_cap : blocks;
}

cudaError_t launch_ib_batch(const BatchDev &bt, int kernel, int deterministic, int phase, cudaStream_t s) {
    if (phase == 0) {
        if (bt.blocks_prep) launch_prio(k_ib_prepare_batch, batch_ib_grid(bt, bt.blocks_prep), PREP_TPB, 0, s, bt);
    } else if (phase == 1) {
        if (!bt.blocks_gs) return cudaSuccess;
        const int g = batch_ib_grid(bt, bt.blocks_gs);
        if (kernel == LBIB_LINEAR2) {
            if (deterministic) launch_prio(k_ib_gather_spread_batch<2, true>, g, GS_TPB, 0, s, bt);
            else launch_prio(k_ib_gather_spread_batch<2, false>, g, GS_TPB, 0, s, bt);
        } else {
            if (deterministic) launch_prio(k_ib_gather_spread_batch<4, true>, g, GS_TPB, 0, s, bt);
            else launch_prio(k_ib_gather_spread_batch<4, false>, g, GS_TPB, 0, s, bt);
        }
    } else {
        if (!bt.blocks_int) return cudaSuccess;
        const int g = batch_ib_grid(bt, bt.blocks_int);
        if (kernel == LBIB_LINEAR2) launch_prio(k_ib_interp_batch<2>, g, INT_TPB, 0, s, bt);
        else launch_prio(k_ib_interp_batch<4>, g, INT_TPB, 0, s, bt);
    }
    return cudaGetLastError();
}

int ib_blocks_prepare(const DevCtx &c) {
    return c.n_swimmers + (c.n_tris + PREP_TPB - 1) / PREP_TPB + (c.n_edges + PREP_TPB - 1) / PREP_TPB;
}
int ib_blocks_spread(const DevCtx &c) { return (c.n_nodes + GS_NODES - 1) / GS_NODES; }
int ib_blocks_interp(const DevCtx &c, int kernel) {
    const int lanes = kernel == LBIB_LINEAR2 ? 2 : 4;
    return (int)(((long long)c.n_nodes * lanes + INT_TPB - 1) / INT_TPB);
}

cudaError_t launch_ib_prepare(const DevCtx &c, cudaStream_t s) {
    const int blocks = ib_blocks_prepare(c);
    if (blocks == 0) return cudaSuccess;
    launch_prio(k_ib_prepare, blocks, PREP_TPB, 0, s, c);
    return cudaGetLastError();
}

cudaError_t launch_bead_init(const DevCtx &c, cudaStream_t s) {
    if (c.n_beads == 0) return cudaSuccess;
    k_bead_init<<<c.n_beads, PREP_TPB, 0, s>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_ib_gather_spread(const DevCtx &c, int kernel, cudaStream_t s) {
    if (c.n_nodes == 0) return cudaSuccess;
    const int blocks = (c.n_nodes + GS_NODES - 1) / GS_NODES;
    if (kernel == LBIB_LINEAR2) {
        if (c.deterministic) launch_prio(k_ib_gather_spread<2, true>, blocks, GS_TPB, 0, s, c);
        else launch_prio(k_ib_gather_spread<2, false>, blocks, GS_TPB, 0, s, c);
    } else {
        if (c.deterministic) launch_prio(k_ib_gather_spread<4, true>, blocks, GS_TPB, 0, s, c);
        else launch_prio(k_ib_gather_spread<4, false>, blocks, GS_TPB, 0, s, c);
    }
    return cudaGetLastError();
}

cudaError_t launch_ib_interp(const DevCtx &c, int kernel, bool advect, float *vel_out, int mark_parity, cudaStream_t s) {
    if (c.n_nodes == 0) return cudaSuccess;
    const int lanes = kernel == LBIB_LINEAR2 ? 2 : 4;
    const long long threads = (long long)c.n_nodes * lanes;
    const int blocks = (int)((threads + INT_TPB - 1) / INT_TPB);
    if (kernel == LBIB_LINEAR2) {
        if (advect) launch_prio(k_ib_interp<2, true>, blocks, INT_TPB, 0, s, c, vel_out, mark_parity);
        else launch_prio(k_ib_interp<2, false>, blocks, INT_TPB, 0, s, c, vel_out, -1);
    } else {
        if (advect) launch_prio(k_ib_interp<4, true>, blocks, INT_TPB, 0, s, c, vel_out, mark_parity);
        else launch_prio(k_ib_interp<4, false>, blocks, INT_TPB, 0, s, c, vel_out, -1);
    }
    return cudaGetLastError();
}

cudaError_t launch_ib_mark(const DevCtx &c, int kernel, cudaStream_t s) {
    if (c.n_nodes == 0) return cudaSuccess;
    const int lanes = kernel == LBIB_LINEAR2 ? 2 : 4;
    const int blocks = (int)(((long long)c.n_nodes * lanes + INT_TPB - 1) / INT_TPB);
    if (kernel == LBIB_LINEAR2) k_ib_mark<2><<<blocks, INT_TPB, 0, s>>>(c);
    else k_ib_mark<4><<<blocks, INT_TPB, 0, s>>>(c);
    return cudaGetLastError();
}


cudaError_t launch_swimmer_state(const DevCtx &c, bool init, cudaStream_t s) {
    if (c.n_swimmers == 0) return cudaSuccess;
    k_swimmer_beads<<<3 * c.n_swimmers, PREP_TPB, 0, s>>>(c);
    k_swimmer_finish<<<(c.n_swimmers + 127) / 128, 128, 0, s>>>(c, init ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace lbib
