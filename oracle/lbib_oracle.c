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
 */
#include <math.h>
#include <stddef.h>
#include <string.h>

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

/* Second-order equilibrium, Sec. 2.1 Eq. (lbm:equilibrium):
 * f_i^eq = w_i rho [1 + c.u/cs^2 - u.u/(2 cs^2) + (c.u)^2/(2 cs^4)]. */
void orc_equilibrium(double rho, const double *u, double *feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < ORC_Q; ++i) {
        double cu = OC[i][0] * u[0] + OC[i][1] * u[1] + OC[i][2] * u[2];
        feq[i] = ow(i) * rho * (1.0 + cu / CS2 - uu / (2.0 * CS2) + cu * cu / (2.0 * CS2 * CS2));
    }
}

static long wrap(long a, long n)
{
    long r = a % n;
    return r < 0 ? r + n : r;
}

/* One lattice Boltzmann time step on the whole periodic box.
 *
 * Collision, Sec. 2.1 Eq. (lbe):  f*_i = f_i - (f_i - f_i^eq) / tau.
 * Moments, Sec. 2.1: rho = sum f_i; physical velocity
 *   rho u = sum f_i c_i + F/2          (the unnumbered equation after Eq. sc).
 * Force inclusion:
 *   ORC_GUO:       f^eq taken at the physical u, plus the source term
 *                  (1 - 1/(2 tau)) w_i [(c_i - u)/cs^2 + (c_i.u) c_i/cs^4] . F;
 *   ORC_SHAN_CHEN: f^eq taken at u^eq, rho u^eq = sum f_i c_i + tau F (Eq. sc).
 * Streaming (the left side of Eq. lbe): f_i(x + c_i, t + 1) = f*_i(x, t),
 * written here as a push into the separate array fnew.
 *
 * f, fnew: n_cells x 19 (cell = x + nx (y + ny z)); F: n_cells x 3 force
 * density or NULL; g: uniform force density added everywhere.
 * rho_out, u_out (n_cells, n_cells x 3, may be NULL): density and physical
 * velocity at time t, the field the IB interpolation reads (Sec. 2.3). */
void orc_lb_step(int nx, int ny, int nz, double tau, int forcing, const double *F, const double *g,
                 const double *f, double *fnew, double *rho_out, double *u_out)
{
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z) {
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                long cell = x + (long)nx * (y + (long)ny * z);
                const double *fc = f + cell * ORC_Q;
                double Ft[3] = {g[0], g[1], g[2]};
                if (F) {
                    Ft[0] += F[3 * cell + 0];
                    Ft[1] += F[3 * cell + 1];
                    Ft[2] += F[3 * cell + 2];
                }
                double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < ORC_Q; ++i) {
                    rho += fc[i];
                    j[0] += fc[i] * OC[i][0];
                    j[1] += fc[i] * OC[i][1];
                    j[2] += fc[i] * OC[i][2];
                }
                double u[3], ueq[3], feq[ORC_Q], fpost[ORC_Q];
                for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * Ft[a]) / rho;
                if (forcing == ORC_SHAN_CHEN) {
                    for (int a = 0; a < 3; ++a) ueq[a] = (j[a] + tau * Ft[a]) / rho;
                } else {
                    for (int a = 0; a < 3; ++a) ueq[a] = u[a];
                }
                orc_equilibrium(rho, ueq, feq);
                for (int i = 0; i < ORC_Q; ++i) {
                    fpost[i] = fc[i] - (fc[i] - feq[i]) / tau;
                    if (forcing == ORC_GUO) {
                        double cu = OC[i][0] * u[0] + OC[i][1] * u[1] + OC[i][2] * u[2];
                        double s = 0.0;
                        for (int a = 0; a < 3; ++a)
                            s += ((OC[i][a] - u[a]) / CS2 + cu * OC[i][a] / (CS2 * CS2)) * Ft[a];
                        fpost[i] += (1.0 - 1.0 / (2.0 * tau)) * ow(i) * s;
                    }
                }
                for (int i = 0; i < ORC_Q; ++i) {
                    long xd = wrap(x + OC[i][0], nx), yd = wrap(y + OC[i][1], ny), zd = wrap(z + OC[i][2], nz);
                    long dst = xd + (long)nx * (yd + (long)ny * zd);
                    fnew[dst * ORC_Q + i] = fpost[i];
                }
                if (rho_out) rho_out[cell] = rho;
                if (u_out) {
                    u_out[3 * cell + 0] = u[0];
                    u_out[3 * cell + 1] = u[1];
                    u_out[3 * cell + 2] = u[2];
                }
            }
        }
    }
}

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

/* One-dimensional kernels of the smoothed delta function, Sec. 2.3.
 * PESKIN4: Peskin's 4-point kernel (Peskin 2002, cited in Sec. 2):
 *   |r| <= 1:      (3 - 2|r| + sqrt(1 + 4|r| - 4 r^2)) / 8
 *   1 <= |r| <= 2: (5 - 2|r| - sqrt(-7 + 12|r| - 4 r^2)) / 8
 * LINEAR2: the two-point linear interpolation the paper uses, 1 - |r|. */
double orc_phi(int kernel, double r)
{
    double a = fabs(r);
    if (kernel == ORC_LINEAR2) return a < 1.0 ? 1.0 - a : 0.0;
    if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    if (a <= 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
    return 0.0;
}

/* Integer cells whose kernel weight can be non-zero for coordinate p:
 * floor(p) - h + 1 .. floor(p) + h, with h = 2 (4-point) or 1 (2-point). */
static int support_half(int kernel) { return kernel == ORC_LINEAR2 ? 1 : 2; }

/* Force spreading, Sec. 2.3 Eq. (spreading):
 * F(x) += sum_j f_j Delta(x - r_j), Delta(x) = phi(x1) phi(x2) phi(x3).
 * One sequential loop over the nodes (accumulates into F). */
void orc_spread(int kernel, int nx, int ny, int nz, int M, const double *r, const double *fn, double *F)
{
    int h = support_half(kernel);
    for (int j = 0; j < M; ++j) {
        long b0 = (long)floor(r[3 * j + 0]), b1 = (long)floor(r[3 * j + 1]), b2 = (long)floor(r[3 * j + 2]);
        for (long cz = b2 - h + 1; cz <= b2 + h; ++cz)
            for (long cy = b1 - h + 1; cy <= b1 + h; ++cy)
                for (long cx = b0 - h + 1; cx <= b0 + h; ++cx) {
                    double d = orc_phi(kernel, cx - r[3 * j + 0]) * orc_phi(kernel, cy - r[3 * j + 1]) *
                               orc_phi(kernel, cz - r[3 * j + 2]);
                    long cell = wrap(cx, nx) + (long)nx * (wrap(cy, ny) + (long)ny * wrap(cz, nz));
                    for (int a = 0; a < 3; ++a) F[3 * cell + a] += fn[3 * j + a] * d;
                }
    }
}

/* Velocity interpolation, Sec. 2.3 Eq. (interpolation):
 * rdot_j = sum_x u(x) Delta(x - r_j). */
void orc_interpolate(int kernel, int nx, int ny, int nz, int M, const double *r, const double *u, double *v)
{
    int h = support_half(kernel);
    for (int j = 0; j < M; ++j) {
        double acc[3] = {0.0, 0.0, 0.0};
        long b0 = (long)floor(r[3 * j + 0]), b1 = (long)floor(r[3 * j + 1]), b2 = (long)floor(r[3 * j + 2]);
        for (long cz = b2 - h + 1; cz <= b2 + h; ++cz)
            for (long cy = b1 - h + 1; cy <= b1 + h; ++cy)
                for (long cx = b0 - h + 1; cx <= b0 + h; ++cx) {
                    double d = orc_phi(kernel, cx - r[3 * j + 0]) * orc_phi(kernel, cy - r[3 * j + 1]) *
                               orc_phi(kernel, cz - r[3 * j + 2]);
                    long cell = wrap(cx, nx) + (long)nx * (wrap(cy, ny) + (long)ny * wrap(cz, nz));
                    for (int a = 0; a < 3; ++a) acc[a] += u[3 * cell + a] * d;
                }
        for (int a = 0; a < 3; ++a) v[3 * j + a] = acc[a];
    }
}

/* Bead position = centre of mass of its mesh nodes (Fig. 1 caption),
 * equal node masses. */
void orc_bead_centres(int n_beads, const int *beads /* n x 4: node_start, count, tri_start, tri_count */,
                      const double *r, double *R)
{
    for (int b = 0; b < n_beads; ++b) {
        double s[3] = {0.0, 0.0, 0.0};
        int n0 = beads[4 * b + 0], n = beads[4 * b + 1];
        for (int j = n0; j < n0 + n; ++j)
            for (int a = 0; a < 3; ++a) s[a] += r[3 * j + a];
        for (int a = 0; a < 3; ++a) R[3 * b + a] = s[a] / n;
    }
}

/* Driving forces, Sec. 2.2 Eq. (ext forces), along x, omega = 2 pi / T:
 * balance = 1: f1 = A1 sin(wt + p1), f3 = A3 sin(wt + p3), f2 = -f1 - f3
 *              (the paper: p1 = 0, A3 = B, p3 = alpha);
 * balance = 0: every bead carries its own A_b sin(wt + p_b). */
void orc_drive(const double *amp, const double *phase, int balance, double period, double t, double *fd)
{
    double w = 2.0 * M_PI / period;
    double f1 = amp[0] * sin(w * t + phase[0]);
    double f3 = amp[2] * sin(w * t + phase[2]);
    double f2 = balance ? -f1 - f3 : amp[1] * sin(w * t + phase[1]);
    memset(fd, 0, 9 * sizeof(double));
    fd[0] = f1;
    fd[3] = f2;
    fd[6] = f3;
}

/* Harmonic springs, Sec. 2.2:
 * f1 = -k (|R1 - R2| - L) (R1 - R2)/|R1 - R2|, f3 likewise with R3 - R2,
 * f2 = -f1 - f3. */
void orc_springs(double k, double L, const double *R, double *fs)
{
    for (int side = 0; side < 2; ++side) {
        int b = side == 0 ? 0 : 2;
        double d[3], n = 0.0;
        for (int a = 0; a < 3; ++a) {
            d[a] = R[3 * b + a] - R[3 + a];
            n += d[a] * d[a];
        }
        n = sqrt(n);
        for (int a = 0; a < 3; ++a) fs[3 * b + a] = -k * (n - L) * d[a] / n;
    }
    for (int a = 0; a < 3; ++a) fs[3 + a] = -fs[a] - fs[6 + a];
}

/* Linear finite-element membrane (Sec. 2.2).  Per triangle the in-plane
 * deformation maps the rest edge vectors D = [X1-X0, X2-X0] to the current
 * d = [x1-x0, x2-x0].  With the metrics G = D^T D and g = d^T d the right
 * Cauchy-Green tensor in the rest basis is C = G^{-1} g, whose eigenvalues are
 * lambda_1^2, lambda_2^2, giving the invariants of Sec. 2.2
 *   I1 = lambda_1^2 + lambda_2^2 - 2,   I2 = lambda_1^2 lambda_2^2 - 1.
 * Strain energy per triangle: A0 w(I1, I2), A0 the rest area, with
 *   ORC_NEOHOOKE: w = Gs/2 (I1 - 1 + 1/(I2 + 1));
 *   ORC_SKALAK:   w = ks/4 (I1^2 + 2 I1 - 2 I2 + C I2^2)   (Sec. 2.2, W_sk). */
static void tri_metrics(const double *P, const int *t, double m[3])
{
    double d1[3], d2[3];
    for (int a = 0; a < 3; ++a) {
        d1[a] = P[3 * t[1] + a] - P[3 * t[0] + a];
        d2[a] = P[3 * t[2] + a] - P[3 * t[0] + a];
    }
    m[0] = d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2];
    m[1] = d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2];
    m[2] = d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2];
}

static void invariants(const double G[3], const double g[3], double *I1, double *I2)
{
    double detG = G[0] * G[2] - G[1] * G[1];
    /* C = G^{-1} g as a 2x2 matrix */
    double Gi00 = G[2] / detG, Gi01 = -G[1] / detG, Gi11 = G[0] / detG;
    double C00 = Gi00 * g[0] + Gi01 * g[1], C01 = Gi00 * g[1] + Gi01 * g[2];
    double C10 = Gi01 * g[0] + Gi11 * g[1], C11 = Gi01 * g[1] + Gi11 * g[2];
    /* eigenvalues lambda^2 of C by the quadratic formula */
    double tr = C00 + C11, det = C00 * C11 - C01 * C10;
    double disc = tr * tr / 4.0 - det;
    if (disc < 0.0) disc = 0.0;
    double l1 = tr / 2.0 + sqrt(disc), l2 = tr / 2.0 - sqrt(disc);
    *I1 = l1 + l2 - 2.0;
    *I2 = l1 * l2 - 1.0;
}

static double law_w(int law, double p1, double p2, double I1, double I2)
{
    if (law == ORC_SKALAK) return p1 / 4.0 * (I1 * I1 + 2.0 * I1 - 2.0 * I2 + p2 * I2 * I2);
    return p1 / 2.0 * (I1 - 1.0 + 1.0 / (I2 + 1.0));
}

/* dw/dI1, dw/dI2 of the law above. */
static void law_dw(int law, double p1, double p2, double I1, double I2, double *w1, double *w2)
{
    if (law == ORC_SKALAK) {
        *w1 = p1 / 4.0 * (2.0 * I1 + 2.0);
        *w2 = p1 / 4.0 * (-2.0 + 2.0 * p2 * I2);
    } else {
        *w1 = p1 / 2.0;
        *w2 = -p1 / 2.0 / ((I2 + 1.0) * (I2 + 1.0));
    }
}

/* Total membrane strain energy of triangles [t0, t0 + nt). p1 = Gs (neo-Hookean)
 * or ks (Skalak); p2 = C (Skalak only). */
double orc_membrane_energy(int law, double p1, double p2, int nt, const int *tris, const double *X, const double *x)
{
    double W = 0.0;
    for (int t = 0; t < nt; ++t) {
        double G[3], g[3], I1, I2;
        tri_metrics(X, tris + 3 * t, G);
        tri_metrics(x, tris + 3 * t, g);
        double A0 = 0.5 * sqrt(G[0] * G[2] - G[1] * G[1]);
        invariants(G, g, &I1, &I2);
        W += A0 * law_w(law, p1, p2, I1, I2);
    }
    return W;
}

/* Membrane nodal forces by virtual work, Sec. 2.2: f_j = -dW/dr_j, added
 * into fout.  With tr C and det C = det g / det G,
 *   d(tr C)/dd  = 2 d G^{-1},   d(det C)/dd = 2 det C d g^{-1},
 * so dW/dd = A0 [w1 2 d G^{-1} + w2 2 det C d g^{-1}], column a of which is
 * dW/dd_a; node 1 gets -dW/dd_1, node 2 -dW/dd_2, node 0 the sum of both. */
void orc_membrane_forces(int law, double p1, double p2, int nt, const int *tris, const double *X, const double *x,
                         double *fout)
{
    for (int t = 0; t < nt; ++t) {
        const int *tv = tris + 3 * t;
        double G[3], g[3], I1, I2, w1, w2;
        tri_metrics(X, tv, G);
        tri_metrics(x, tv, g);
        double detG = G[0] * G[2] - G[1] * G[1], detg = g[0] * g[2] - g[1] * g[1];
        double A0 = 0.5 * sqrt(detG);
        invariants(G, g, &I1, &I2);
        law_dw(law, p1, p2, I1, I2, &w1, &w2);
        double detC = detg / detG;
        double Gi[2][2] = {{G[2] / detG, -G[1] / detG}, {-G[1] / detG, G[0] / detG}};
        double gi[2][2] = {{g[2] / detg, -g[1] / detg}, {-g[1] / detg, g[0] / detg}};
        double d[3][2];
        for (int a = 0; a < 3; ++a) {
            d[a][0] = x[3 * tv[1] + a] - x[3 * tv[0] + a];
            d[a][1] = x[3 * tv[2] + a] - x[3 * tv[0] + a];
        }
        for (int a = 0; a < 3; ++a) {
            double dW[2];
            for (int c = 0; c < 2; ++c) {
                double dGi = d[a][0] * Gi[0][c] + d[a][1] * Gi[1][c];
                double dgi = d[a][0] * gi[0][c] + d[a][1] * gi[1][c];
                dW[c] = A0 * (2.0 * w1 * dGi + 2.0 * w2 * detC * dgi);
            }
            fout[3 * tv[1] + a] -= dW[0];
            fout[3 * tv[2] + a] -= dW[1];
            fout[3 * tv[0] + a] += dW[0] + dW[1];
        }
    }
}
