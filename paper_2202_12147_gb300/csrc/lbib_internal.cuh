// Internal declarations shared by the CUDA translation units of liblbib.
// Device data layouts, the D3Q19 lattice of the CUDA path, launchers.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>

#include "lbib.h"

namespace lbib {

// ---------------------------------------------------------------- lattice
// D3Q19 (Sec. 2.1).  Opposite directions are adjacent: (1,2), (3,4), ...
// 0 rest; 1,2 +-x; 3,4 +-y; 5,6 +-z; 7,8 (1,1,0)/(-1,-1,0); 9,10 (1,-1,0)/(-1,1,0);
// 11,12 (1,0,1)/(-1,0,-1); 13,14 (1,0,-1)/(-1,0,1); 15,16 (0,1,1)/(0,-1,-1);
// 17,18 (0,1,-1)/(0,-1,1).
constexpr int Q = 19;
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
           : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
           : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
           : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
// weights 1/3, 1/18, 1/36 (Sec. 2.1)
__host__ __device__ constexpr float wgt(int i) { return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f); }
__host__ __device__ constexpr double wgt_d(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

// maximum cells per LB thread block (a run along x of one row); one tile
// flag per block
constexpr int LB_TPB = 256;
// threads per node in spreading / interpolation (one per (y, z) stencil row)
constexpr int ROWS4 = 16;

// device error bits, latched in Control::err
constexpr int ERR_NONFINITE = 1;
constexpr int ERR_UNSTABLE = 2;
constexpr int ERR_TIMEOUT = 4;
constexpr int ERR_MARK = 8;  // a node stencil reached a tile its bead's marked region does not cover

struct Control {
    long long step;  // time steps completed by the immersed-boundary chain; t of its next step
    int err;
    int done;        // blocks of the current interpolation launch that have finished
    int gen[2];      // per step parity: the step whose stamps mark the tiles (see k_lb_main)
    int vol_done;    // blocks of the current gather/spread launch that have read the bead volumes
};

// Per-triangle reference data of the linear FEM membrane.
struct TriDev {
    double G[3];     // rest metric G = D^T D: G00, G01, G11
    float Gi[3];     // G^{-1}: Gi00, Gi01, Gi11
    float K;         // A0 * Gs / det G
    float inv_detG;  // 1 / det G
    int v[3];        // node ids
    float skC;       // Skalak: C (kappa_a / kappa_s = 1 + 2 C)
    int law;         // LBIB_NEOHOOKE (K = A0 Gs / det G) or LBIB_SKALAK (K = A0 kappa_s / det G)
};
static_assert(sizeof(TriDev) == 64, "TriDev layout");

// One bending edge: node ids a, b (the edge), c, d (the opposite corners of
// the triangles a, b, c and b, a, d, both outward); cos and sin of the rest
// angle between the two triangles' normals; the discrete modulus.
struct EdgeDev {
    int v[4];
    float c0, s0;
    float kb;        // 2 sqrt(3) times the bending modulus
    int pad;
};
static_assert(sizeof(EdgeDev) == 32, "EdgeDev layout");

struct BeadDev {
    int node_start, node_count;
    int swimmer, slot;  // owning swimmer and position 0..2 along its axis
    float inv_count;    // 1 / node_count
    float reach;        // bound on |r_j - R| over the bead's nodes (rest radius + margin)
    float kv;           // volume-penalty modulus (0: off)
    int pad;
    double V0;          // enclosed volume of the rest shape
    double pad2;
};
static_assert(sizeof(BeadDev) == 48, "BeadDev layout");

// fixed-point scale of the bead volume sums: 2^40 units per cubic lattice unit
constexpr double VOL_FIX = 1099511627776.0;

struct SwimDev {
    int bead[3];
    int balance;
    double k, L, L2;        // spring stiffness, rest length, its square
    double inv_period;      // 1 / drive period
    double phase_turns[3];  // phase / (2 pi)
    float amp[3];
    int pad;
    double period;          // drive period (steps)
};

// Everything a kernel needs, by value.
struct DevCtx {
    int nx, ny, nz;
    long long N;      // cells
    long long Npad;   // population plane stride
    int n_tiles;
    int tile_x, tiles_x;  // cells per tile along x, tiles per row
    int marked_grid;      // persistent grid of the marked-tile fluid kernel
    int cells_per_thread; // adjacent cells per fluid thread: 1, 2 (even rows) or 4 (16-bit storage, rows of 4k)
    float tau, omega, rho0;
    float g[3];
    int has_g;
    float st_scale, st_inv_scale;  // F16/BF16 scaling
    int n_nodes, n_tris, n_beads, n_swimmers;
    int deterministic;
    // buffers
    void *pops;
    float4 *F;                 // force density per cell (float atomics)
    unsigned long long *Fdet;  // 3 x Npad fixed-point force (deterministic mode)
    float4 *U;                 // velocity (x, y, z, rho) per cell
    int *marks;                // [2][n_tiles]: step number whose node stencils touch the tile, per step parity
                               // (tile = x / tile_x + tiles_x * (y + ny * z))
    int *tile_list;            // [2][n_tiles]: the marked tiles of each parity, in marking order
    int *tile_count;           // [2]: entries in each list
    double *rx, *ry, *rz;      // node positions (SoA)
    float4 *node_force;        // f^tot per node
    float4 *node_vel;          // interpolated velocity per node
    float4 *tri_force;         // 3 corner forces per triangle, then 4 per bending edge
    const TriDev *tris;
    int n_edges;               // bending edges (beads with a bending modulus)
    int has_volume;            // some bead has a volume penalty
    const EdgeDev *edges;
    float4 *tri_vgrad;         // per triangle corner: (1/6) (r_next - R) x (r_prev - R), R the bead centre
    long long *bead_Vfix;      // [n_beads] enclosed volume of each bead at this step's positions, fixed point
                               // (VOL_FIX); summed by k_ib_prepare, read and cleared by k_ib_gather_spread
    const int *csr_ptr;        // node -> incident corner entries: triangle*3 + corner, then
    const int *csr_ent;        //         3*n_tris + edge*4 + slot for bending edges
    const int *node_bead;
    const BeadDev *beads;
    const SwimDev *swims;
    double *bead_R;            // bead centres, 4 doubles per bead
    float4 *bead_ext;          // (f^d + f^s) / N_v per bead
    float4 *bead_V;            // mean node velocity of each bead in the last step
    unsigned long long *bead_acc;  // [n_beads][3] fixed-point sums of the step's node velocities (zero between steps)
    lbib_track_point *track;   // [LBIB_TRACK_STEPS][n_swimmers] ring of trajectory points

    Control *ctl;
    lbib_swimmer_state *sw_state;
    double *xcm0;              // x_cm at init, 3 per swimmer
    double *sw_period;         // per swimmer: x_cm at the last two period boundaries, completed periods (8 doubles)
};

// most boxes one batch holds
constexpr int LBIB_MAX_BATCH = 1024;

// A batch of boxes advanced by shared launches: the per-box descriptors in
// device memory and, per kernel, prefix sums of each box's block count.
struct BatchDev {
    int n_boxes;
    const DevCtx *boxes;
    const int *off_main, *off_prep, *off_gs, *off_int;  // [n_boxes + 1]
    int blocks_main, blocks_prep, blocks_gs, blocks_int, blocks_marked;
    int max_tile_threads;  // widest tile of any box, in threads
    int cells_per_thread;  // common to every box of the batch
    int ib_grid_cap;       // most blocks of a batched immersed-boundary launch (BATCH_IB_BLOCKS_PER_SM per SM)
};

// blocks per SM of the batched immersed-boundary launches, which walk their
// virtual blocks in a grid-stride loop (measured: 1 too few, 2 best, 4 and
// uncapped slower on the 64-box ensemble)
constexpr int BATCH_IB_BLOCKS_PER_SM = 2;

// Boxes of one size passed by value to one launch of the main fluid kernel
// (grid (tiles_x, ny, nz * n)); the descriptors sit in the parameter bank.
constexpr int LBIB_CLASS_BOXES = 64;
struct ClassArgs {
    int n;
    DevCtx box[LBIB_CLASS_BOXES];
};

// fixed-point scale of deterministic spreading: 2^48 units per force unit
// (resolution 3.6e-15, range +-32768 per cell)
constexpr double FIX_SCALE = 281474976710656.0;
constexpr double FIX_INV = 1.0 / 281474976710656.0;
// the same powers of two in FP32 (exact), for conversions without FP64
// arithmetic: the fixed-point values are the same integers as with the FP64
// scaling, and the read-back equals it for |F| < 32 per cell (integers below
// 2^53, exact in FP64)
constexpr float FIX_SCALE_F = 281474976710656.0f;
constexpr float FIX_INV_F = 3.5527136788005009e-15f;

// ---------------------------------------------------------------- delta-kernel stencil
// 1-D kernel weights on the KW stencil cells floor(p) - KW/2 + 1 ... floor(p) + KW/2.
// Peskin's 4-point kernel evaluated at the four distances 1+f, f, 1-f, 2-f
// (f = p - floor p) needs one square root: with q = sqrt(1 + 4f - 4f^2)
// the weights are (3 - 2f - q)/8, (3 - 2f + q)/8, (1 + 2f + q)/8, (1 + 2f - q)/8.
template <int KW>
__device__ __forceinline__ void weights1d(float f, float *w) {
    if (KW == 4) {
        const float q = sqrtf(1.0f + 4.0f * f - 4.0f * f * f);
        w[0] = (3.0f - 2.0f * f - q) * 0.125f;
        w[1] = (3.0f - 2.0f * f + q) * 0.125f;
        w[2] = (1.0f + 2.0f * f + q) * 0.125f;
        w[3] = (1.0f + 2.0f * f - q) * 0.125f;
    } else {
        w[0] = 1.0f - f;
        w[1] = f;
    }
}

// stencil origin (wrapped into [0, n)) and fractional offset along one axis
__device__ __forceinline__ int stencil_axis(double p, int n, int kw, float &frac) {
    const double fl = floor(p);
    frac = (float)(p - fl);
    long long o = (long long)fl - (kw / 2 - 1);
    o %= n;
    if (o < 0) o += n;
    return (int)o;
}

// Launch on stream s with s's priority as a launch attribute: a CUDA graph
// captured from s keeps it on the kernel node (the immersed-boundary chain
// runs on a high-priority stream beside the main fluid update).
template <typename... Exp, typename... Act>
inline cudaError_t launch_prio(void (*k)(Exp...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Act &&...args) {
    int prio = 0;
    cudaError_t e = cudaStreamGetPriority(s, &prio);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributePriority;
    attr.val.priority = prio;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, static_cast<Act &&>(args)...);
}

// message returned by lbib_last_error() on this thread
void set_last_error(const char *msg);
// argument checks of lb_init (api.cu), shared with the adjoint engine
bool check_params(const lb_params *p, std::string &why);
bool check_structure(const lb_params *p, const lbib_structure *s, std::string &why);

// ---------------------------------------------------------------- launchers
// LB (lb_kernels.cu)
cudaError_t launch_lb_main(const DevCtx &c, int storage, int forcing, bool odd, cudaStream_t s);
cudaError_t launch_lb_marked(const DevCtx &c, int storage, int forcing, bool odd, cudaStream_t s);
cudaError_t launch_lb_macros(const DevCtx &c, int storage, bool odd, float *rho, float *u, cudaStream_t s);
cudaError_t launch_lb_batch(const BatchDev &bt, int storage, int forcing, int det, bool marked, bool odd, cudaStream_t s);
cudaError_t launch_lb_class(const ClassArgs &ca, int storage, int forcing, int cpt, bool odd, cudaStream_t s);
// IB (ib_kernels.cu)
cudaError_t launch_ib_prepare(const DevCtx &c, cudaStream_t s);
cudaError_t launch_ib_gather_spread(const DevCtx &c, int kernel, cudaStream_t s);
cudaError_t launch_ib_interp(const DevCtx &c, int kernel, bool advect, float *vel_out, int mark_parity, cudaStream_t s);
cudaError_t launch_swimmer_state(const DevCtx &c, bool init, cudaStream_t s);
cudaError_t launch_bead_init(const DevCtx &c, cudaStream_t s);
cudaError_t launch_ib_mark(const DevCtx &c, int kernel, cudaStream_t s);
// phase 0: prepare, 1: gather/spread, 2: advecting interpolation, for every box
cudaError_t launch_ib_batch(const BatchDev &bt, int kernel, int deterministic, int phase, cudaStream_t s);
int ib_blocks_prepare(const DevCtx &c);
int ib_blocks_spread(const DevCtx &c);
int ib_blocks_interp(const DevCtx &c, int kernel);

}  // namespace lbib
