/*
 * lbm_oracle.c -- TEST INFRASTRUCTURE, not part of the product path.
 *
 * Plain FP64, single-threaded restatement of the fractional-step MRT lattice
 * Boltzmann method of Zhang, Guo & Li (arXiv:1812.02459).  Every quantity is
 * computed into its own array, in the order the paper's sections give the
 * pieces, with no fusion.  Only tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file.  Build: gcc -O2 -ffp-contract=off.
 *
 * Readings of points the paper leaves open (each is also a test case):
 *  - J_d = lambda*J_phi + q (lambda weights the profile term, Sec. IV.B).
 *  - The CH collision relaxes the zeroth moment to the corrected phi with
 *    s_0 = 1, so the LBE inherits the finite-difference correction exactly.
 *  - G_i uses u(F/rho - grad p) in its second-order term (Eq. Gi and App. A).
 *  - Gradients of the LBE/force part use the isotropic stencils of
 *    Eq. (dicretized); everything inside L(psi) of the finite-difference step
 *    uses fourth-order central differences (Eq. fourOrder_FDM), with the
 *    5-point fourth-order second derivative for the Laplacian of mu_psi.
 *  - n = grad phi / sqrt(|grad phi|^2 + eps^2), and |grad phi| in J_phi is
 *    the same regularised norm.
 *  - phi is clamped to [-1,1] only inside the rho(phi), mu(phi) interpolation.
 *  - After the filter, the next collision uses the filtered (p,u) for the
 *    equilibrium part and keeps g's own non-equilibrium part:
 *        m* = m_eq(p_f,u_f) + (I-S)(m - m_eq(p_hat,u_hat)) + (I-S/2) G~ .
 *  - Walls: halfway bounce-back for f and g; for stencils, fields are
 *    mirrored about the halfway wall (phi, mu, p even; u odd).
 *  - Implicit velocity: Picard sweeps, sweep 0 evaluates the velocity
 *    gradients with u^n.  d_t u in the CH source is u^n - u^{n-1}.
 *
 * What pins it (tests/test_oracle_pins.py): lattice isotropy, M M^-1 = I and
 * the row structure of M; equilibrium and source moments, including App. A's
 * printed moment form of G; closed forms of the collision (s=1, s=0, BGK);
 * streaming as a permutation and bounce-back; plane-wave closed forms of every
 * stencil, with and without walls; the App. B filter table, its identities and
 * transfer function; the RK3 growth factor; conservation of sum(phi); a flat
 * interface staying put; the Laplace law; viscous decay of a shear wave;
 * hydrostatic balance; Galilean translation of a drop; a layered channel
 * against its 1-D steady solution; removal of normal diffusion by q; the
 * azimuthal acceleration Omega J_r that F_m = J.grad u alone gives a
 * non-equilibrium drop in rigid rotation.
 * The dynamic pressure p' = rho p is pinned by the Laplace law, which takes
 * its jump across a static drop.
 * The choice of u_hat inside the filtered-equilibrium reading above is a
 * reading, not a law, and has no pin beyond GPU-oracle parity.
 * A uniform phi in a steady rotation staying uniform pins the acceleration
 * of the CH source.
 * Parity unpinned by a law: the odd mirror of u at walls in the velocity
 * gradients and in the filter.  Slips planted there survive the pins
 * (oracle/planted_mistakes.py); the comparison with the independent
 * restatement in oracle/torch_ref.py catches them.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q 9
static const double CS2 = 1.0 / 3.0; /* c_s^2 with c_s = 1/sqrt(3), Sec. III.A */

/* ------------------------------------------------------------------------ */
/* Lattice, Sec. III.A Eq. (D2Q9) and the weights below it.                  */
/* ------------------------------------------------------------------------ */
void orc_lattice(int c[18], double w[9])
{
    const double pi = acos(-1.0);
    c[0] = 0; c[1] = 0;
    for (int i = 1; i <= 4; ++i) {
        c[2 * i] = (int)lround(cos((i - 1) * pi / 2));
        c[2 * i + 1] = (int)lround(sin((i - 1) * pi / 2));
    }
    for (int i = 5; i <= 8; ++i) {
        c[2 * i] = (int)lround(sqrt(2.0) * cos((i - 5) * pi / 2 + pi / 4));
        c[2 * i + 1] = (int)lround(sqrt(2.0) * sin((i - 5) * pi / 2 + pi / 4));
    }
    /* omega_0 = 4/9, omega_{1..4} = 1/9, omega_{5..8} = 1/36 (the text's
       second "1..8" index is a typo for 5..8). */
    w[0] = 4.0 / 9.0;
    for (int i = 1; i <= 4; ++i) w[i] = 1.0 / 9.0;
    for (int i = 5; i <= 8; ++i) w[i] = 1.0 / 36.0;
}

static int g_c[18];
static double g_w[9];
static double g_M[81], g_Minv[81];
static int g_init = 0;

/* Transformation matrix, Sec. III.A Eq. (D2Q9MRT), typed row by row. */
void orc_mrt_matrix(double M[81])
{
    static const double rows[81] = {
         1,  1,  1,  1,  1,  1,  1,  1,  1,
        -4, -1, -1, -1, -1,  2,  2,  2,  2,
         4, -2, -2, -2, -2,  1,  1,  1,  1,
         0,  1,  0, -1,  0,  1, -1, -1,  1,
         0, -2,  0,  2,  0,  1, -1, -1,  1,
         0,  0,  1,  0, -1,  1,  1, -1, -1,
         0,  0, -2,  0,  2,  1,  1, -1, -1,
         0,  1, -1,  1, -1,  0,  0,  0,  0,
         0,  0,  0,  0,  0,  1, -1,  1, -1};
    memcpy(M, rows, sizeof rows);
}

/* M^{-1} by Gauss-Jordan elimination with partial pivoting. */
void orc_mrt_inverse(double Minv[81])
{
    double a[9][18];
    double M[81];
    orc_mrt_matrix(M);
    for (int r = 0; r < 9; ++r)
        for (int k = 0; k < 18; ++k)
            a[r][k] = k < 9 ? M[r * 9 + k] : (k - 9 == r ? 1.0 : 0.0);
    for (int col = 0; col < 9; ++col) {
        int piv = col;
        for (int r = col + 1; r < 9; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (piv != col)
            for (int k = 0; k < 18; ++k) { double t = a[col][k]; a[col][k] = a[piv][k]; a[piv][k] = t; }
        double d = a[col][col];
        for (int k = 0; k < 18; ++k) a[col][k] /= d;
        for (int r = 0; r < 9; ++r) {
            if (r == col) continue;
            double m = a[r][col];
            if (m != 0.0)
                for (int k = 0; k < 18; ++k) a[r][k] -= m * a[col][k];
        }
    }
    for (int r = 0; r < 9; ++r)
        for (int k = 0; k < 9; ++k) Minv[r * 9 + k] = a[r][k + 9];
}

static void orc_init_tables(void)
{
    if (g_init) return;
    orc_lattice(g_c, g_w);
    orc_mrt_matrix(g_M);
    orc_mrt_inverse(g_Minv);
    g_init = 1;
}

/* Explicit centred selective filters, App. B table (d_0..d_5). */
void orc_filter_coeffs(int order, double d[6])
{
    for (int k = 0; k < 6; ++k) d[k] = 0.0;
    switch (order) {
    case 5:
        d[0] = 6.0 / 16; d[1] = -4.0 / 16; d[2] = 1.0 / 16; break;
    case 7:
        d[0] = 5.0 / 16; d[1] = -15.0 / 64; d[2] = 3.0 / 32; d[3] = -1.0 / 64; break;
    case 9:
        d[0] = 0.243527493120; d[1] = -0.204788880640; d[2] = 0.120007591680;
        d[3] = -0.045211119360; d[4] = 0.008228661760; break;
    case 11:
        d[0] = 0.215044884112; d[1] = -0.187772883589; d[2] = 0.123755948787;
        d[3] = -0.059227575576; d[4] = 0.018721609157; d[5] = -0.002999540835; break;
    default: break;
    }
}

/* ------------------------------------------------------------------------ */
/* Equilibria and sources.                                                   */
/* ------------------------------------------------------------------------ */

/* CH equilibrium, Sec. III.A Eq. (feq_CH). */
void orc_feq(double phi, double mu, double ux, double uy, double eta, double out[9])
{
    orc_init_tables();
    double u2 = ux * ux + uy * uy;
    for (int i = 0; i < Q; ++i) {
        double cu = g_c[2 * i] * ux + g_c[2 * i + 1] * uy;
        if (i == 0)
            out[i] = phi + (g_w[0] - 1.0) * eta * mu - g_w[0] * phi * u2 / (2 * CS2);
        else
            out[i] = g_w[i] * eta * mu
                   + g_w[i] * phi * (cu / CS2 + cu * cu / (2 * CS2 * CS2) - u2 / (2 * CS2));
    }
}

/* Velocity-based NS equilibrium, Sec. III.B Eq. (geq). */
void orc_geq(double p, double ux, double uy, double out[9])
{
    orc_init_tables();
    double u2 = ux * ux + uy * uy;
    for (int i = 0; i < Q; ++i) {
        double cu = g_c[2 * i] * ux + g_c[2 * i + 1] * uy;
        out[i] = g_w[i] * (p / CS2 + cu / CS2 + cu * cu / (2 * CS2 * CS2) - u2 / (2 * CS2));
    }
}

/* CH source, Sec. III.A Eq. (Fi): omega_i phi c_i.(d_t u + u.grad u)/c_s^2,
   with a = d_t u + u.grad u passed in. */
void orc_src_ch(double phi, double ax, double ay, double out[9])
{
    orc_init_tables();
    for (int i = 0; i < Q; ++i)
        out[i] = g_w[i] * phi * (g_c[2 * i] * ax + g_c[2 * i + 1] * ay) / CS2;
}

/* NS source, Sec. III.B Eq. (Gi), second-order term read as u(F/rho - grad p):
   G_i = w_i [ c.F/(rho cs2) + u_a b_b (c_a c_b - cs2 delta_ab)/cs2^2 ],
   b = F/rho - grad p. */
void orc_src_ns(double rho, double Fx, double Fy, double ux, double uy,
                double dpx, double dpy, double out[9])
{
    orc_init_tables();
    double bx = Fx / rho - dpx, by = Fy / rho - dpy;
    double u[2] = {ux, uy}, b[2] = {bx, by};
    for (int i = 0; i < Q; ++i) {
        double c[2] = {(double)g_c[2 * i], (double)g_c[2 * i + 1]};
        double first = (c[0] * Fx + c[1] * Fy) / (rho * CS2);
        double second = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int bb = 0; bb < 2; ++bb)
                second += u[a] * b[bb] * (c[a] * c[bb] - (a == bb ? CS2 : 0.0));
        out[i] = g_w[i] * (first + second / (CS2 * CS2));
    }
}

static void matvec(const double *A, const double *x, double *y)
{
    for (int r = 0; r < Q; ++r) {
        double s = 0.0;
        for (int k = 0; k < Q; ++k) s += A[r * Q + k] * x[k];
        y[r] = s;
    }
}

/* MRT collision with forcing, Sec. III.A Eqs. (distribution_CH), (collison):
   f* = f - M^-1 S M (f - feq) + M^-1 (I - S/2) M F, carried out in moment space. */
void orc_collide_f(const double f[9], const double feq[9], const double F[9],
                   const double s[9], double out[9])
{
    orc_init_tables();
    double m[9], meq[9], mF[9], ms[9];
    matvec(g_M, f, m);
    matvec(g_M, feq, meq);
    matvec(g_M, F, mF);
    for (int k = 0; k < Q; ++k)
        ms[k] = m[k] - s[k] * (m[k] - meq[k]) + (1.0 - 0.5 * s[k]) * mF[k];
    matvec(g_Minv, ms, out);
}

/* NS collision, Sec. III.B Eq. (distribution_NS), with the filtered (p,u)
   carried in as the equilibrium part:
   m* = M geq_f + (I - S)(M g - M geq_hat) + (I - S/2) M G. */
void orc_collide_g(const double g[9], const double geq_f[9], const double geq_hat[9],
                   const double G[9], const double s[9], double out[9])
{
    orc_init_tables();
    double m[9], mf[9], mh[9], mG[9], ms[9];
    matvec(g_M, g, m);
    matvec(g_M, geq_f, mf);
    matvec(g_M, geq_hat, mh);
    matvec(g_M, G, mG);
    for (int k = 0; k < Q; ++k)
        ms[k] = mf[k] + (1.0 - s[k]) * (m[k] - mh[k]) + (1.0 - 0.5 * s[k]) * mG[k];
    matvec(g_Minv, ms, out);
}

/* Strain rate grad u + grad u^T from the non-equilibrium part of the NS
   populations, Sec. III.B Eq. (Fmu) (whose sum is printed over f; the
   populations of the NS equation are g):
     grad u + grad u^T = [(s_7 - s_1)(F.u) I - s_7 (F u + u F)] / (2 rho cs^2)
                         - sum_i c_i c_i [M^-1 S M (g - g_eq)]_i / cs^2 .
   out = (S_xx, S_xy, S_yy); s are the NS rates with s_7 = 1/tau_g. */
void orc_strain_moments(const double g[9], const double geq[9], const double s[9], double rho,
                        double Fx, double Fy, double ux, double uy, double out[3])
{
    orc_init_tables();
    double d[9], m[9], h[9];
    for (int k = 0; k < Q; ++k) d[k] = g[k] - geq[k];
    matvec(g_M, d, m);
    for (int k = 0; k < Q; ++k) m[k] *= s[k];
    matvec(g_Minv, m, h);
    double pxx = 0.0, pxy = 0.0, pyy = 0.0;
    for (int i = 0; i < Q; ++i) {
        double cx = g_c[2 * i], cy = g_c[2 * i + 1];
        pxx += cx * cx * h[i];
        pxy += cx * cy * h[i];
        pyy += cy * cy * h[i];
    }
    double Fu = Fx * ux + Fy * uy, a = 1.0 / (2.0 * rho * CS2);
    out[0] = ((s[7] - s[1]) * Fu - s[7] * 2.0 * Fx * ux) * a - pxx / CS2;
    out[1] = -s[7] * (Fx * uy + ux * Fy) * a - pxy / CS2;
    out[2] = ((s[7] - s[1]) * Fu - s[7] * 2.0 * Fy * uy) * a - pyy / CS2;
}

/* ------------------------------------------------------------------------ */
/* Padded fields: a field with G ghost layers on every side.  Ghosts wrap on */
/* periodic axes and mirror about the halfway wall otherwise, multiplied by  */
/* the field's parity (+1 even, -1 odd).                                     */
/* ------------------------------------------------------------------------ */
typedef struct { int nx, ny, G; double *a; } pf;

static pf pf_new(int nx, int ny, int G)
{
    pf r = {nx, ny, G, (double *)calloc((size_t)(nx + 2 * G) * (ny + 2 * G), sizeof(double))};
    return r;
}
static void pf_free(pf *f) { free(f->a); f->a = NULL; }
static inline double *PA(const pf *f, int i, int j)
{
    return &f->a[(size_t)(j + f->G) * (f->nx + 2 * f->G) + (i + f->G)];
}

/* Map a coordinate k of an axis of length n onto the domain. */
static int map_axis(int k, int n, int periodic, int *flip)
{
    if (periodic) { int r = k % n; if (r < 0) r += n; return r; }
    int m = k;
    while (m < 0 || m >= n) {            /* repeated reflection about -1/2 and n-1/2 */
        if (m < 0) { m = -m - 1; *flip = !*flip; }
        if (m >= n) { m = 2 * n - 1 - m; *flip = !*flip; }
    }
    return m;
}

static pf pad(const double *src, int nx, int ny, int G, int parity, int px, int py)
{
    pf r = pf_new(nx, ny, G);
    for (int j = -G; j < ny + G; ++j)
        for (int i = -G; i < nx + G; ++i) {
            int fx = 0, fy = 0;
            int ii = map_axis(i, nx, px, &fx);
            int jj = map_axis(j, ny, py, &fy);
            double v = src[(size_t)jj * nx + ii];
            if (parity < 0 && (fx ^ fy)) v = -v;
            *PA(&r, i, j) = v;
        }
    return r;
}

/* Isotropic gradient, Sec. III.B Eq. (dicretized), output has G-1 ghosts. */
static void iso_grad(const pf *in, pf *gx, pf *gy)
{
    orc_init_tables();
    int G = in->G - 1;
    *gx = pf_new(in->nx, in->ny, G);
    *gy = pf_new(in->nx, in->ny, G);
    for (int j = -G; j < in->ny + G; ++j)
        for (int i = -G; i < in->nx + G; ++i) {
            double sx = 0.0, sy = 0.0;
            for (int q = 1; q < Q; ++q) {
                double v = *PA(in, i + g_c[2 * q], j + g_c[2 * q + 1]);
                sx += g_w[q] * g_c[2 * q] * v / CS2;
                sy += g_w[q] * g_c[2 * q + 1] * v / CS2;
            }
            *PA(gx, i, j) = sx;
            *PA(gy, i, j) = sy;
        }
}

/* Isotropic Laplacian, Sec. III.B Eq. (dicretized). */
static pf iso_lap(const pf *in)
{
    orc_init_tables();
    int G = in->G - 1;
    pf r = pf_new(in->nx, in->ny, G);
    for (int j = -G; j < in->ny + G; ++j)
        for (int i = -G; i < in->nx + G; ++i) {
            double c0 = *PA(in, i, j), s = 0.0;
            for (int q = 1; q < Q; ++q)
                s += 2.0 * g_w[q] * (*PA(in, i + g_c[2 * q], j + g_c[2 * q + 1]) - c0) / CS2;
            *PA(&r, i, j) = s;
        }
    return r;
}

/* Fourth-order central first derivatives, Sec. III.A Eq. (fourOrder_FDM). */
static void fd4_grad(const pf *in, pf *gx, pf *gy)
{
    int G = in->G - 2;
    *gx = pf_new(in->nx, in->ny, G);
    *gy = pf_new(in->nx, in->ny, G);
    for (int j = -G; j < in->ny + G; ++j)
        for (int i = -G; i < in->nx + G; ++i) {
            *PA(gx, i, j) = (*PA(in, i - 2, j) - 8.0 * *PA(in, i - 1, j)
                             + 8.0 * *PA(in, i + 1, j) - *PA(in, i + 2, j)) / 12.0;
            *PA(gy, i, j) = (*PA(in, i, j - 2) - 8.0 * *PA(in, i, j - 1)
                             + 8.0 * *PA(in, i, j + 1) - *PA(in, i, j + 2)) / 12.0;
        }
}

/* Fourth-order central second derivatives summed over both axes. */
static pf fd4_lap(const pf *in)
{
    int G = in->G - 2;
    pf r = pf_new(in->nx, in->ny, G);
    for (int j = -G; j < in->ny + G; ++j)
        for (int i = -G; i < in->nx + G; ++i) {
            double c = *PA(in, i, j);
            double dxx = (-*PA(in, i - 2, j) + 16.0 * *PA(in, i - 1, j) - 30.0 * c
                          + 16.0 * *PA(in, i + 1, j) - *PA(in, i + 2, j)) / 12.0;
            double dyy = (-*PA(in, i, j - 2) + 16.0 * *PA(in, i, j - 1) - 30.0 * c
                          + 16.0 * *PA(in, i, j + 1) - *PA(in, i, j + 2)) / 12.0;
            *PA(&r, i, j) = dxx + dyy;
        }
    return r;
}

static void unpad(const pf *in, double *dst)
{
    for (int j = 0; j < in->ny; ++j)
        for (int i = 0; i < in->nx; ++i) dst[(size_t)j * in->nx + i] = *PA(in, i, j);
}

void orc_grad_iso(int nx, int ny, int px, int py, int parity, const double *in,
                  double *gx, double *gy)
{
    pf a = pad(in, nx, ny, 1, parity, px, py), x, y;
    iso_grad(&a, &x, &y);
    unpad(&x, gx); unpad(&y, gy);
    pf_free(&a); pf_free(&x); pf_free(&y);
}

void orc_lap_iso(int nx, int ny, int px, int py, int parity, const double *in, double *out)
{
    pf a = pad(in, nx, ny, 1, parity, px, py);
    pf r = iso_lap(&a);
    unpad(&r, out);
    pf_free(&a); pf_free(&r);
}

void orc_grad_fd4(int nx, int ny, int px, int py, int parity, const double *in,
                  double *gx, double *gy)
{
    pf a = pad(in, nx, ny, 2, parity, px, py), x, y;
    fd4_grad(&a, &x, &y);
    unpad(&x, gx); unpad(&y, gy);
    pf_free(&a); pf_free(&x); pf_free(&y);
}

void orc_lap_fd4(int nx, int ny, int px, int py, int parity, const double *in, double *out)
{
    pf a = pad(in, nx, ny, 2, parity, px, py);
    pf r = fd4_lap(&a);
    unpad(&r, out);
    pf_free(&a); pf_free(&r);
}

/* Selective filter, Sec. III.B Eq. (filter) with the App. B coefficients:
   chi(x) <- chi(x) - a sum_{alpha} sum_{j=-P..P} d_|j| chi(x + j e_alpha),
   every node from the unfiltered field. */
void orc_filter(int nx, int ny, int px, int py, int parity, int order, double a,
                const double *in, double *out)
{
    double d[6];
    orc_filter_coeffs(order, d);
    int P = order / 2;
    if (order == 0) { memcpy(out, in, sizeof(double) * (size_t)nx * ny); return; }
    pf c = pad(in, nx, ny, P, parity, px, py);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double s = 0.0;
            for (int k = -P; k <= P; ++k) s += d[abs(k)] * *PA(&c, i + k, j);
            for (int k = -P; k <= P; ++k) s += d[abs(k)] * *PA(&c, i, j + k);
            out[(size_t)j * nx + i] = *PA(&c, i, j) - a * s;
        }
    pf_free(&c);
}

/* Pull streaming f_i(x) = f*_i(x - c_i) (Eqs. distribution_CH/NS); a source
   outside a wall returns the node's own opposite population (halfway
   bounce-back). */
void orc_stream(int nx, int ny, int px, int py, const double *fstar, double *fout)
{
    orc_init_tables();
    size_t N = (size_t)nx * ny;
    for (int q = 0; q < Q; ++q) {
        int opp = 0;
        for (int r = 0; r < Q; ++r)
            if (g_c[2 * r] == -g_c[2 * q] && g_c[2 * r + 1] == -g_c[2 * q + 1]) opp = r;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int si = i - g_c[2 * q], sj = j - g_c[2 * q + 1];
                int out_x = !px && (si < 0 || si >= nx);
                int out_y = !py && (sj < 0 || sj >= ny);
                double v;
                if (out_x || out_y) v = fstar[opp * N + (size_t)j * nx + i];
                else {
                    si = ((si % nx) + nx) % nx;
                    sj = ((sj % ny) + ny) % ny;
                    v = fstar[q * N + (size_t)sj * nx + si];
                }
                fout[q * N + (size_t)j * nx + i] = v;
            }
    }
}

/* ------------------------------------------------------------------------ */
/* Step 2 of the fractional step: d_t phi = div J_d, Sec. II.A Eq. (step2),  */
/* discretised with Eq. (fourOrder_FDM) and advanced by Eq. (TVD-3order).    */
/* ------------------------------------------------------------------------ */
void orc_fd_rhs(const orc_params *prm, const double *psi, double *out)
{
    int nx = prm->nx, ny = prm->ny;
    double kappa = 3.0 * prm->sigma * prm->W / 8.0, beta = 3.0 * prm->sigma / (4.0 * prm->W);
    double e2 = prm->grad_eps * prm->grad_eps;
    pf P = pad(psi, nx, ny, 6, +1, prm->periodic_x, prm->periodic_y);
    pf gx, gy;
    fd4_grad(&P, &gx, &gy);                       /* 4 ghosts */
    pf lap = fd4_lap(&P);                         /* 4 ghosts */
    pf mu = pf_new(nx, ny, 4);
    for (int j = -4; j < ny + 4; ++j)
        for (int i = -4; i < nx + 4; ++i) {
            double v = *PA(&P, i, j);
            *PA(&mu, i, j) = 4.0 * beta * (v * v * v - v) - kappa * *PA(&lap, i, j);
        }
    pf mx, my;
    fd4_grad(&mu, &mx, &my);                      /* 2 ghosts */
    pf Jx = pf_new(nx, ny, 2), Jy = pf_new(nx, ny, 2);
    for (int j = -2; j < ny + 2; ++j)
        for (int i = -2; i < nx + 2; ++i) {
            double ax = *PA(&gx, i, j), ay = *PA(&gy, i, j), v = *PA(&P, i, j);
            double mag = sqrt(ax * ax + ay * ay + e2);
            double nxv = ax / mag, nyv = ay / mag;
            double jphi = mag - 2.0 * (1.0 - v * v) / prm->W;      /* J_phi = (.) n */
            double jx = prm->lambda * jphi * nxv, jy = prm->lambda * jphi * nyv;
            if (prm->flux_correction) {
                double dmn = *PA(&mx, i, j) * nxv + *PA(&my, i, j) * nyv;  /* q = -M (grad mu . n) n */
                jx += -prm->M * dmn * nxv;
                jy += -prm->M * dmn * nyv;
            }
            *PA(&Jx, i, j) = jx;
            *PA(&Jy, i, j) = jy;
        }
    pf dJx, dummy1, dummy2, dJy;
    fd4_grad(&Jx, &dJx, &dummy1);
    fd4_grad(&Jy, &dummy2, &dJy);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            out[(size_t)j * nx + i] = *PA(&dJx, i, j) + *PA(&dJy, i, j);
    pf_free(&P); pf_free(&gx); pf_free(&gy); pf_free(&lap); pf_free(&mu);
    pf_free(&mx); pf_free(&my); pf_free(&Jx); pf_free(&Jy);
    pf_free(&dJx); pf_free(&dJy); pf_free(&dummy1); pf_free(&dummy2);
}

/* Third-order TVD Runge-Kutta (Shu-Osher form), Sec. III.A Eq. (TVD-3order). */
void orc_rk3(int n, const double *phibar, double *out, orc_rhs_fn L, void *ctx)
{
    double *p1 = malloc(sizeof(double) * n), *p2 = malloc(sizeof(double) * n);
    double *Lv = malloc(sizeof(double) * n);
    L(phibar, Lv, n, ctx);
    for (int k = 0; k < n; ++k) p1[k] = phibar[k] + Lv[k];
    L(p1, Lv, n, ctx);
    for (int k = 0; k < n; ++k) p2[k] = 0.75 * phibar[k] + 0.25 * (p1[k] + Lv[k]);
    L(p2, Lv, n, ctx);
    for (int k = 0; k < n; ++k) out[k] = phibar[k] / 3.0 + 2.0 / 3.0 * (p2[k] + Lv[k]);
    free(p1); free(p2); free(Lv);
}

static void fd_rhs_cb(const double *psi, double *out, int n, void *ctx)
{
    (void)n;
    orc_fd_rhs((const orc_params *)ctx, psi, out);
}

/* ------------------------------------------------------------------------ */
/* Whole-method simulation.                                                  */
/* ------------------------------------------------------------------------ */
struct orc_sim {
    orc_params p;
    double kappa, beta, tau_f;
    double *f, *g;                  /* post-stream populations [9][N] */
    double *phi;                    /* corrected order parameter */
    double *pf_, *uxf, *uyf;        /* filtered kinematic pressure and velocity */
    double *uhx, *uhy;              /* unfiltered velocity from the implicit update */
    double *upx, *upy;              /* filtered velocity of the previous step */
    int last_sweeps;
};

static double clamp1(double v) { return v < -1.0 ? -1.0 : (v > 1.0 ? 1.0 : v); }

/* Density and dynamic viscosity interpolation, Sec. II.B Eq. (rho) and
   Sec. III.B Eq. (dynamic_vis); mu_H = rho_H nu_H, mu_L = rho_L nu_L. */
static double rho_of(const orc_params *p, double phi)
{
    double c = clamp1(phi);
    return p->rho_H * (1.0 + c) / 2.0 + p->rho_L * (1.0 - c) / 2.0;
}
static double visc_of(const orc_params *p, double phi)
{
    double c = clamp1(phi);
    return p->rho_H * p->nu_H * (1.0 + c) / 2.0 + p->rho_L * p->nu_L * (1.0 - c) / 2.0;
}

/* u-independent field quantities at one time level, on the interior. */
typedef struct {
    double *rho, *nu, *mu, *gphx, *gphy, *grx, *gry, *Jx, *Jy, *Fsx, *Fsy, *gpx, *gpy;
} fields_t;

static void fields_alloc(fields_t *F, size_t N)
{
    double **v[] = {&F->rho, &F->nu, &F->mu, &F->gphx, &F->gphy, &F->grx, &F->gry,
                    &F->Jx, &F->Jy, &F->Fsx, &F->Fsy, &F->gpx, &F->gpy};
    for (size_t k = 0; k < sizeof v / sizeof v[0]; ++k) *v[k] = calloc(N, sizeof(double));
}
static void fields_free(fields_t *F)
{
    double *v[] = {F->rho, F->nu, F->mu, F->gphx, F->gphy, F->grx, F->gry,
                   F->Jx, F->Jy, F->Fsx, F->Fsy, F->gpx, F->gpy};
    for (size_t k = 0; k < sizeof v / sizeof v[0]; ++k) free(v[k]);
}

/* Chemical potential (Sec. II.A Eq. chemical), density gradient, diffusion
   flux J = (d rho/d phi) M grad mu (Sec. II.B), surface force
   F_s = kappa div(|grad phi|^2 I - grad phi grad phi) (Eq. surfaceforce),
   pressure gradient; all with the isotropic stencils of Eq. (dicretized). */
static void compute_fields(const orc_sim *s, const double *phi, const double *p, fields_t *F)
{
    const orc_params *q = &s->p;
    int nx = q->nx, ny = q->ny, px = q->periodic_x, py = q->periodic_y;
    pf PH = pad(phi, nx, ny, 2, +1, px, py);
    pf lap = iso_lap(&PH);                               /* 1 ghost */
    pf MU = pf_new(nx, ny, 1);
    for (int j = -1; j < ny + 1; ++j)
        for (int i = -1; i < nx + 1; ++i) {
            double v = *PA(&PH, i, j);
            *PA(&MU, i, j) = 4.0 * s->beta * (v * v * v - v) - s->kappa * *PA(&lap, i, j);
        }
    pf gx, gy;
    iso_grad(&PH, &gx, &gy);                             /* 1 ghost */
    pf Txx = pf_new(nx, ny, 1), Txy = pf_new(nx, ny, 1), Tyy = pf_new(nx, ny, 1);
    for (int j = -1; j < ny + 1; ++j)
        for (int i = -1; i < nx + 1; ++i) {
            double a = *PA(&gx, i, j), b = *PA(&gy, i, j), m2 = a * a + b * b;
            *PA(&Txx, i, j) = m2 - a * a;
            *PA(&Txy, i, j) = -a * b;
            *PA(&Tyy, i, j) = m2 - b * b;
        }
    pf dTxx_x, dTxx_y, dTxy_x, dTxy_y, dTyy_x, dTyy_y, gmx, gmy;
    iso_grad(&Txx, &dTxx_x, &dTxx_y);
    iso_grad(&Txy, &dTxy_x, &dTxy_y);
    iso_grad(&Tyy, &dTyy_x, &dTyy_y);
    iso_grad(&MU, &gmx, &gmy);
    pf PP = pad(p, nx, ny, 1, +1, px, py), gpx, gpy;
    iso_grad(&PP, &gpx, &gpy);
    double drho = (q->rho_H - q->rho_L) / 2.0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = (size_t)j * nx + i;
            F->rho[k] = rho_of(q, phi[k]);
            F->nu[k] = visc_of(q, phi[k]) / F->rho[k];
            F->mu[k] = *PA(&MU, i, j);
            F->gphx[k] = *PA(&gx, i, j);
            F->gphy[k] = *PA(&gy, i, j);
            F->grx[k] = drho * F->gphx[k];
            F->gry[k] = drho * F->gphy[k];
            F->Jx[k] = drho * q->M * *PA(&gmx, i, j);
            F->Jy[k] = drho * q->M * *PA(&gmy, i, j);
            F->Fsx[k] = s->kappa * (*PA(&dTxx_x, i, j) + *PA(&dTxy_y, i, j));
            F->Fsy[k] = s->kappa * (*PA(&dTxy_x, i, j) + *PA(&dTyy_y, i, j));
            F->gpx[k] = *PA(&gpx, i, j);
            F->gpy[k] = *PA(&gpy, i, j);
        }
    pf_free(&PH); pf_free(&lap); pf_free(&MU); pf_free(&gx); pf_free(&gy);
    pf_free(&Txx); pf_free(&Txy); pf_free(&Tyy);
    pf_free(&dTxx_x); pf_free(&dTxx_y); pf_free(&dTxy_x); pf_free(&dTxy_y);
    pf_free(&dTyy_x); pf_free(&dTyy_y); pf_free(&gmx); pf_free(&gmy);
    pf_free(&PP); pf_free(&gpx); pf_free(&gpy);
}

/* Velocity gradients (isotropic) of a velocity field; u is odd at walls. */
static void vel_grads(const orc_sim *s, const double *ux, const double *uy,
                      double *dxux, double *dyux, double *dxuy, double *dyuy)
{
    const orc_params *q = &s->p;
    orc_grad_iso(q->nx, q->ny, q->periodic_x, q->periodic_y, -1, ux, dxux, dyux);
    orc_grad_iso(q->nx, q->ny, q->periodic_x, q->periodic_y, -1, uy, dxuy, dyuy);
}

/* Total force F = F_p + F_s + F_nu + F_m + F_g of Sec. II.B Eq. (reformNS):
   F_p = -p grad rho, F_nu = nu (grad u + grad u^T).grad rho, F_m = J.grad u,
   F_g = (rho - rho_ref) g (rho_ref = 0: rho g as printed; otherwise gravity is
   measured against the hydrostatic pressure of a fluid of density rho_ref). */
static void force_with_strain(const orc_sim *s, const fields_t *F, const double *p,
                              const double *dxux, const double *dyux, const double *dxuy,
                              const double *dyuy, double Sxx, double Sxy, double Syy, size_t k,
                              double *Fx, double *Fy)
{
    const orc_params *q = &s->p;
    double Fpx = -p[k] * F->grx[k], Fpy = -p[k] * F->gry[k];
    double Fnx = F->nu[k] * (Sxx * F->grx[k] + Sxy * F->gry[k]);
    double Fny = F->nu[k] * (Sxy * F->grx[k] + Syy * F->gry[k]);
    double Fmx = F->Jx[k] * dxux[k] + F->Jy[k] * dyux[k];
    double Fmy = F->Jx[k] * dxuy[k] + F->Jy[k] * dyuy[k];
    double Fgx = (F->rho[k] - q->g_rho_ref) * q->gx, Fgy = (F->rho[k] - q->g_rho_ref) * q->gy;
    *Fx = Fpx + F->Fsx[k] + Fnx + Fmx + Fgx;
    *Fy = Fpy + F->Fsy[k] + Fny + Fmy + Fgy;
}

/* The total force with the strain rate grad u + grad u^T of F_nu taken from
   the velocity gradients (isotropic stencils). */
static void total_force(const orc_sim *s, const fields_t *F, const double *p,
                        const double *dxux, const double *dyux, const double *dxuy,
                        const double *dyuy, size_t k, double *Fx, double *Fy)
{
    force_with_strain(s, F, p, dxux, dyux, dxuy, dyuy, 2.0 * dxux[k], dyux[k] + dxuy[k], 2.0 * dyuy[k], k, Fx,
                      Fy);
}

int orc_create(const orc_params *prm, const double *phi0, const double *p0,
               const double *ux0, const double *uy0, orc_sim **out)
{
    orc_init_tables();
    if (prm->nx < 1 || prm->ny < 1) return 1;
    orc_sim *s = calloc(1, sizeof *s);
    s->p = *prm;
    s->kappa = 3.0 * prm->sigma * prm->W / 8.0;          /* Sec. II.A, below Eq. (free_energy) */
    s->beta = 3.0 * prm->sigma / (4.0 * prm->W);
    s->tau_f = 0.5 + prm->M / (prm->eta * CS2);          /* Sec. III.A Eq. (mobility) */
    size_t N = (size_t)prm->nx * prm->ny;
    s->f = calloc(Q * N, sizeof(double));
    s->g = calloc(Q * N, sizeof(double));
    double **v[] = {&s->phi, &s->pf_, &s->uxf, &s->uyf, &s->uhx, &s->uhy, &s->upx, &s->upy};
    for (size_t k = 0; k < sizeof v / sizeof v[0]; ++k) *v[k] = calloc(N, sizeof(double));
    memcpy(s->phi, phi0, N * sizeof(double));
    memcpy(s->pf_, p0, N * sizeof(double));
    memcpy(s->uxf, ux0, N * sizeof(double));
    memcpy(s->uyf, uy0, N * sizeof(double));
    memcpy(s->uhx, ux0, N * sizeof(double));
    memcpy(s->uhy, uy0, N * sizeof(double));
    memcpy(s->upx, ux0, N * sizeof(double));
    memcpy(s->upy, uy0, N * sizeof(double));
    /* f = f_eq(phi0, mu(phi0), u0), g = g_eq(p0, u0). */
    double *lap = malloc(N * sizeof(double));
    orc_lap_iso(prm->nx, prm->ny, prm->periodic_x, prm->periodic_y, +1, phi0, lap);
    for (size_t k = 0; k < N; ++k) {
        double ph = phi0[k];
        double mu = 4.0 * s->beta * (ph * ph * ph - ph) - s->kappa * lap[k];
        double fe[9], ge[9];
        orc_feq(ph, mu, ux0[k], uy0[k], prm->eta, fe);
        orc_geq(p0[k], ux0[k], uy0[k], ge);
        for (int q = 0; q < Q; ++q) { s->f[q * N + k] = fe[q]; s->g[q * N + k] = ge[q]; }
    }
    free(lap);
    *out = s;
    return 0;
}

static int step_once(orc_sim *s)
{
    const orc_params *q = &s->p;
    int nx = q->nx, ny = q->ny;
    size_t N = (size_t)nx * ny;
    double *fs = malloc(Q * N * sizeof(double)), *gs = malloc(Q * N * sizeof(double));
    double *dxux = malloc(N * sizeof(double)), *dyux = malloc(N * sizeof(double));
    double *dxuy = malloc(N * sizeof(double)), *dyuy = malloc(N * sizeof(double));
    fields_t F;
    fields_alloc(&F, N);

    /* (1) Field quantities and forces at t^n from phi^n and the filtered p^n, u^n. */
    compute_fields(s, s->phi, s->pf_, &F);
    vel_grads(s, s->uxf, s->uyf, dxux, dyux, dxuy, dyuy);

    double sf[9], sg[9];
    memcpy(sf, q->s_f, sizeof sf);
    sf[3] = sf[5] = 1.0 / s->tau_f;                        /* Sec. III.A below Eq. (CH_Sf) */
    memcpy(sg, q->s_g, sizeof sg);

    /* (2) Collision of both population sets at every node. */
    for (size_t k = 0; k < N; ++k) {
        double fl[9], gl[9], fe[9], Fi[9], out[9];
        for (int c = 0; c < Q; ++c) { fl[c] = s->f[c * N + k]; gl[c] = s->g[c * N + k]; }
        double ux = s->uxf[k], uy = s->uyf[k];
        double ax = (ux - s->upx[k]) + ux * dxux[k] + uy * dyux[k];   /* d_t u + u.grad u */
        double ay = (uy - s->upy[k]) + ux * dxuy[k] + uy * dyuy[k];
        orc_feq(s->phi[k], F.mu[k], ux, uy, q->eta, fe);
        orc_src_ch(s->phi[k], ax, ay, Fi);
        orc_collide_f(fl, fe, Fi, sf, out);
        for (int c = 0; c < Q; ++c) fs[c * N + k] = out[c];

        double Fx, Fy;
        total_force(s, &F, s->pf_, dxux, dyux, dxuy, dyuy, k, &Fx, &Fy);
        double ge_f[9], ge_h[9], Gi[9], phat = 0.0;
        for (int c = 0; c < Q; ++c) phat += gl[c];
        phat *= CS2;                                                /* Sec. III.B Eq. (p) */
        orc_geq(s->pf_[k], ux, uy, ge_f);
        orc_geq(phat, s->uhx[k], s->uhy[k], ge_h);
        orc_src_ns(F.rho[k], Fx, Fy, ux, uy, F.gpx[k], F.gpy[k], Gi);
        double tau_g = F.nu[k] / CS2 + 0.5;                        /* Sec. III.B, below Eq. (dynamic_vis) */
        sg[7] = sg[8] = 1.0 / tau_g;
        orc_collide_g(gl, ge_f, ge_h, Gi, sg, out);
        for (int c = 0; c < Q; ++c) gs[c * N + k] = out[c];
    }

    /* (3) Streaming. */
    orc_stream(nx, ny, q->periodic_x, q->periodic_y, fs, s->f);
    orc_stream(nx, ny, q->periodic_x, q->periodic_y, gs, s->g);

    /* (4) LBE predictor phi_bar = sum f (Eq. compute_phi); p = cs2 sum g (Eq. p);
       j = sum c g (first part of Eq. u). */
    double *phibar = calloc(N, sizeof(double)), *phat = calloc(N, sizeof(double));
    double *jx = calloc(N, sizeof(double)), *jy = calloc(N, sizeof(double));
    for (size_t k = 0; k < N; ++k) {
        double sp = 0.0, sgv = 0.0, sx = 0.0, sy = 0.0;
        for (int c = 0; c < Q; ++c) {
            sp += s->f[c * N + k];
            double gv = s->g[c * N + k];
            sgv += gv;
            sx += g_c[2 * c] * gv;
            sy += g_c[2 * c + 1] * gv;
        }
        phibar[k] = sp; phat[k] = CS2 * sgv; jx[k] = sx; jy[k] = sy;
    }

    /* (5) Finite-difference correction step by TVD-RK3. */
    double *phin = malloc(N * sizeof(double));
    orc_rk3((int)N, phibar, phin, fd_rhs_cb, (void *)q);

    /* (6) Implicit velocity u = j + F(u)/(2 rho), Eq. (u), by Picard sweeps. */
    compute_fields(s, phin, phat, &F);
    double *ukx = malloc(N * sizeof(double)), *uky = malloc(N * sizeof(double));
    double *unx = malloc(N * sizeof(double)), *uny = malloc(N * sizeof(double));
    memcpy(ukx, s->uxf, N * sizeof(double));
    memcpy(uky, s->uyf, N * sizeof(double));
    int sweeps = 0;
    for (int it = 0; it < (q->picard_iters > 0 ? q->picard_iters : 1); ++it) {
        vel_grads(s, ukx, uky, dxux, dyux, dxuy, dyuy);
        double num = 0.0, den = 0.0;
        for (size_t k = 0; k < N; ++k) {
            double Fx, Fy;
            if (q->flags & 1u) {
                /* F_nu's strain rate from the post-stream g (Eq. Fmu), with
                   g_eq(p_hat, u^k) and, in its forcing term, the force of this
                   sweep without F_nu (the part Eq. Fmu does not need itself) */
                double gl[9], ge[9], S[3], F0x, F0y;
                for (int c = 0; c < Q; ++c) gl[c] = s->g[c * N + k];
                orc_geq(phat[k], ukx[k], uky[k], ge);
                force_with_strain(s, &F, phat, dxux, dyux, dxuy, dyuy, 0.0, 0.0, 0.0, k, &F0x, &F0y);
                sg[7] = sg[8] = 1.0 / (F.nu[k] / CS2 + 0.5);
                orc_strain_moments(gl, ge, sg, F.rho[k], F0x, F0y, ukx[k], uky[k], S);
                force_with_strain(s, &F, phat, dxux, dyux, dxuy, dyuy, S[0], S[1], S[2], k, &Fx, &Fy);
            } else {
                total_force(s, &F, phat, dxux, dyux, dxuy, dyuy, k, &Fx, &Fy);
            }
            unx[k] = jx[k] + Fx / (2.0 * F.rho[k]);
            uny[k] = jy[k] + Fy / (2.0 * F.rho[k]);
            num += hypot(unx[k] - ukx[k], uny[k] - uky[k]);
            den += hypot(unx[k], uny[k]);
        }
        memcpy(ukx, unx, N * sizeof(double));
        memcpy(uky, uny, N * sizeof(double));
        ++sweeps;
        if (q->picard_zeta > 0.0 && num <= q->picard_zeta * den) break;
    }
    s->last_sweeps = sweeps;

    /* (7) Selective filter on chi = (p, u), Eq. (filter). */
    memcpy(s->upx, s->uxf, N * sizeof(double));          /* (8) u^{n-1} <- u^n */
    memcpy(s->upy, s->uyf, N * sizeof(double));
    orc_filter(nx, ny, q->periodic_x, q->periodic_y, +1, q->filter_order, q->filter_a, phat, s->pf_);
    orc_filter(nx, ny, q->periodic_x, q->periodic_y, -1, q->filter_order, q->filter_a, ukx, s->uxf);
    orc_filter(nx, ny, q->periodic_x, q->periodic_y, -1, q->filter_order, q->filter_a, uky, s->uyf);
    memcpy(s->uhx, ukx, N * sizeof(double));
    memcpy(s->uhy, uky, N * sizeof(double));
    memcpy(s->phi, phin, N * sizeof(double));

    free(fs); free(gs); free(dxux); free(dyux); free(dxuy); free(dyuy);
    free(phibar); free(phat); free(jx); free(jy); free(phin);
    free(ukx); free(uky); free(unx); free(uny);
    fields_free(&F);
    for (size_t k = 0; k < N; ++k)
        if (!isfinite(s->phi[k]) || !isfinite(s->pf_[k]) || !isfinite(s->uxf[k]) || !isfinite(s->uyf[k]))
            return 2;
    return 0;
}

/* One step of the Cahn-Hilliard part alone with a prescribed velocity u
   (the paper's interface-capturing tests, Sec. IV.A, where the flow is
   given): mu from phi^n, the CH collision with f_eq(phi, mu, u) and the
   source built from d_t u + u.grad u of the given field, streaming,
   phi_bar = sum f and the TVD-RK3 correction.  The NS populations, p and
   the implicit velocity are not touched; u becomes the state's velocity
   (and u^{n-1} of the next step). */
static int step_ch_once(orc_sim *s, const double *ux, const double *uy)
{
    const orc_params *q = &s->p;
    int nx = q->nx, ny = q->ny;
    size_t N = (size_t)nx * ny;
    double *fs = malloc(Q * N * sizeof(double));
    double *dxux = malloc(N * sizeof(double)), *dyux = malloc(N * sizeof(double));
    double *dxuy = malloc(N * sizeof(double)), *dyuy = malloc(N * sizeof(double));
    fields_t F;
    fields_alloc(&F, N);
    compute_fields(s, s->phi, s->pf_, &F);                    /* mu, Eq. (chemical) */
    vel_grads(s, ux, uy, dxux, dyux, dxuy, dyuy);
    double sf[9];
    memcpy(sf, q->s_f, sizeof sf);
    sf[3] = sf[5] = 1.0 / s->tau_f;
    for (size_t k = 0; k < N; ++k) {
        double fl[9], fe[9], Fi[9], out[9];
        for (int c = 0; c < Q; ++c) fl[c] = s->f[c * N + k];
        double ax = (ux[k] - s->upx[k]) + ux[k] * dxux[k] + uy[k] * dyux[k];
        double ay = (uy[k] - s->upy[k]) + ux[k] * dxuy[k] + uy[k] * dyuy[k];
        orc_feq(s->phi[k], F.mu[k], ux[k], uy[k], q->eta, fe);
        orc_src_ch(s->phi[k], ax, ay, Fi);
        orc_collide_f(fl, fe, Fi, sf, out);
        for (int c = 0; c < Q; ++c) fs[c * N + k] = out[c];
    }
    orc_stream(nx, ny, q->periodic_x, q->periodic_y, fs, s->f);
    double *phibar = calloc(N, sizeof(double)), *phin = malloc(N * sizeof(double));
    for (size_t k = 0; k < N; ++k)
        for (int c = 0; c < Q; ++c) phibar[k] += s->f[c * N + k];
    orc_rk3((int)N, phibar, phin, fd_rhs_cb, (void *)q);
    memcpy(s->phi, phin, N * sizeof(double));
    memcpy(s->upx, ux, N * sizeof(double));
    memcpy(s->upy, uy, N * sizeof(double));
    memcpy(s->uxf, ux, N * sizeof(double));
    memcpy(s->uyf, uy, N * sizeof(double));
    free(fs); free(dxux); free(dyux); free(dxuy); free(dyuy); free(phibar); free(phin);
    fields_free(&F);
    for (size_t k = 0; k < N; ++k)
        if (!isfinite(s->phi[k])) return 2;
    return 0;
}

int orc_step_ch(orc_sim *s, int n, const double *ux, const double *uy)
{
    for (int t = 0; t < n; ++t) {
        int rc = step_ch_once(s, ux, uy);
        if (rc) return rc;
    }
    return 0;
}

int orc_step(orc_sim *s, int n)
{
    for (int t = 0; t < n; ++t) {
        int rc = step_once(s);
        if (rc) return rc;
    }
    return 0;
}

void orc_fields(const orc_sim *s, double *phi, double *p, double *ux, double *uy)
{
    size_t N = (size_t)s->p.nx * s->p.ny;
    if (phi) memcpy(phi, s->phi, N * sizeof(double));
    if (p) memcpy(p, s->pf_, N * sizeof(double));
    if (ux) memcpy(ux, s->uxf, N * sizeof(double));
    if (uy) memcpy(uy, s->uyf, N * sizeof(double));
}

/* Dynamic pressure p' = rho(phi) p at every node: the kinematic pressure of
   the state is p = p'/rho (Sec. II.B, below Eq. reformNS), with rho(phi) of
   Eq. (rho) as the step uses it (phi clamped to [-1,1]). */
void orc_dynamic_pressure(const orc_sim *s, double *out)
{
    size_t N = (size_t)s->p.nx * s->p.ny;
    for (size_t k = 0; k < N; ++k) out[k] = rho_of(&s->p, s->phi[k]) * s->pf_[k];
}

void orc_state(const orc_sim *s, double *f, double *g, double *uhx, double *uhy,
               double *upx, double *upy)
{
    size_t N = (size_t)s->p.nx * s->p.ny;
    if (f) memcpy(f, s->f, Q * N * sizeof(double));
    if (g) memcpy(g, s->g, Q * N * sizeof(double));
    if (uhx) memcpy(uhx, s->uhx, N * sizeof(double));
    if (uhy) memcpy(uhy, s->uhy, N * sizeof(double));
    if (upx) memcpy(upx, s->upx, N * sizeof(double));
    if (upy) memcpy(upy, s->upy, N * sizeof(double));
}

void orc_set_state(orc_sim *s, const double *f, const double *g, const double *phi,
                   const double *p, const double *ux, const double *uy,
                   const double *uhx, const double *uhy, const double *upx, const double *upy)
{
    size_t N = (size_t)s->p.nx * s->p.ny;
    memcpy(s->f, f, Q * N * sizeof(double));
    memcpy(s->g, g, Q * N * sizeof(double));
    memcpy(s->phi, phi, N * sizeof(double));
    memcpy(s->pf_, p, N * sizeof(double));
    memcpy(s->uxf, ux, N * sizeof(double));
    memcpy(s->uyf, uy, N * sizeof(double));
    memcpy(s->uhx, uhx, N * sizeof(double));
    memcpy(s->uhy, uhy, N * sizeof(double));
    memcpy(s->upx, upx, N * sizeof(double));
    memcpy(s->upy, upy, N * sizeof(double));
}

/* Volume and bubble diagnostics, Sec. IV.C (volume error) and Sec. IV.E
   Eqs. (quantify-yc), (quantify-uc), as node sums:
   [0] sum phi  [1] #(phi>0)  [2] #(phi<0)  [3] sum_{phi<0} y  [4] sum_{phi<0} u_y
   [5] sum w  [6] sum w y  [7] sum w u_y   (w = (1-phi)/2)  [8] max phi  [9] min phi */
void orc_diagnostics(const orc_sim *s, double out[ORC_NDIAG])
{
    int nx = s->p.nx, ny = s->p.ny;
    for (int k = 0; k < ORC_NDIAG; ++k) out[k] = 0.0;
    out[8] = -INFINITY; out[9] = INFINITY;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = (size_t)j * nx + i;
            double ph = s->phi[k], v = s->uyf[k], w = (1.0 - ph) / 2.0;
            out[0] += ph;
            if (ph > 0) out[1] += 1.0;
            if (ph < 0) { out[2] += 1.0; out[3] += j; out[4] += v; }
            out[5] += w; out[6] += w * j; out[7] += w * v;
            if (ph > out[8]) out[8] = ph;
            if (ph < out[9]) out[9] = ph;
        }
}

int orc_last_picard_sweeps(const orc_sim *s) { return s->last_sweeps; }

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    free(s->f); free(s->g); free(s->phi); free(s->pf_); free(s->uxf); free(s->uyf);
    free(s->uhx); free(s->uhy); free(s->upx); free(s->upy);
    free(s);
}
