/*
 * FP64 CPU oracle for the coupled lattice-Boltzmann / immersed-boundary step
 * of "Lattice Boltzmann Simulations of Two Linear Microswimmers Using the
 * Immersed Boundary Method" (Geyer et al., arXiv 2202.12147).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the
 * CUDA path.  Only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it; the product library never does.  It shares
 * no code, header, table or constant with the CUDA sources.
 *
 * Deliberately plain: raw (unshifted) populations f[cell][i] in array-of-
 * structures order, a separate post-collision array and a push stream that
 * is the lattice Boltzmann equation written out, scalar loops, no atomics,
 * spreading as one sequential loop over nodes.  Every function names the
 * passage of the paper it follows.
 *
 * Readings where the paper is silent or differs from the workload statement
 * (each one is also listed in the design notes):
 *   - body force: Guo's forcing scheme by default; the paper's Shan-Chen
 *     velocity shift (Sec. 2.1, Eq. sc) with forcing = ORC_SHAN_CHEN;
 *   - delta kernel: Peskin's 4-point kernel by default; the paper's 2-point
 *     linear kernel (Sec. 2.3) with kernel = ORC_LINEAR2;
 *   - membrane: neo-Hookean w = Gs/2 (I1 - 1 + 1/(I2+1)) per reference area;
 *     the paper's Skalak law (Sec. 2.2) with law = ORC_SKALAK;
 *   - lattice nodes at integer coordinates of a periodic box; Lagrangian
 *     node coordinates are unwrapped and reduced modulo the box per stencil
 *     cell.
 *
 * The time-step functions live in lbib_oracle_step.inc, compiled here twice:
 * over double (the oracle) and over double complex (suffix _cs), the latter
 * giving exact derivatives of the discrete step by the complex-step method.
 */
#include <complex.h>
#include <omp.h>
#include <stddef.h>
#include <string.h>
#include <tgmath.h>

#define ORC_Q 19
#define ORC_GUO 0
#define ORC_SHAN_CHEN 1
#define ORC_PESKIN4 0
#define ORC_LINEAR2 1
#define ORC_NEOHOOKE 0
#define ORC_SKALAK 1

/* D3Q19 velocity set in the paper's numbering i = 1..19 (stored 0..18):
 * rest, the six axis directions, the twelve face diagonals (Sec. 2.1). */
static const int OC[ORC_Q][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {1, -1, 0}, {-1, 1, 0}, {-1, -1, 0},
    {1, 0, 1}, {1, 0, -1}, {-1, 0, 1}, {-1, 0, -1},
    {0, 1, 1}, {0, 1, -1}, {0, -1, 1}, {0, -1, -1},
};

/* Lattice weights 1/3, 1/18, 1/36 for i = 1, 2..7, 8..19 (Sec. 2.1). */
static double ow(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

static const double CS2 = 1.0 / 3.0; /* c_s^2 in lattice units (Sec. 2.1) */

void orc_lattice(int *c, double *w)
{
    for (int i = 0; i < ORC_Q; ++i) {
        c[3 * i + 0] = OC[i][0];
        c[3 * i + 1] = OC[i][1];
        c[3 * i + 2] = OC[i][2];
        w[i] = ow(i);
    }
}

static long wrap(long a, long n)
{
    long r = a % n;
    return r < 0 ? r + n : r;
}

/* Integer cells whose kernel weight can be non-zero for coordinate p:
 * floor(p) - h + 1 .. floor(p) + h, with h = 2 (4-point) or 1 (2-point). */
static int support_half(int kernel) { return kernel == ORC_LINEAR2 ? 1 : 2; }

/* The time-step functions, in FP64 ... */
#define REAL double
#define FN(name) name
#define RE(x) (x)
#include "lbib_oracle_step.inc"
#undef REAL
#undef FN
#undef RE

/* ... and the same functions over double complex, for complex-step
 * derivatives of the discrete step (names suffixed _cs). */
#define REAL double complex
#define FN(name) name##_cs
#define RE(x) creal(x)
#include "lbib_oracle_step.inc"
#undef REAL
#undef FN
#undef RE

/* Density and momentum-only velocity (sum f c / rho) of a population field;
 * no force term.  Used to compare states between steps. */
void orc_macros(long n_cells, const double *f, double *rho, double *u)
{
#pragma omp parallel for schedule(static)
    for (long cell = 0; cell < n_cells; ++cell) {
        const double *fc = f + cell * ORC_Q;
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < ORC_Q; ++i) {
            r += fc[i];
            for (int a = 0; a < 3; ++a) j[a] += fc[i] * OC[i][a];
        }
        rho[cell] = r;
        for (int a = 0; a < 3; ++a) u[3 * cell + a] = j[a] / r;
    }
}

/* Threads of the OpenMP loops (for single-core timings); returns the count
 * now in effect. */
int orc_set_threads(int n)
{
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
}

/* The 1-D delta kernel at one point (real and complex argument). */
double orc_phi(int kernel, double r) { return phi_k(kernel, r); }

void orc_phi_cs(int kernel, const double complex *r, double complex *out) { *out = phi_k_cs(kernel, *r); }

double orc_membrane_energy(int law, double p1, double p2, int nt, const int *tris, const double *X, const double *x)
{
    double W;
    orc_membrane_energy_v(law, p1, p2, nt, tris, X, x, &W);
    return W;
}
