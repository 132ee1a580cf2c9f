/*
 * lbm_oracle.h -- TEST INFRASTRUCTURE, not part of the product path.
 *
 * A plain, slow, single-threaded FP64 restatement of the fractional-step
 * MRT lattice Boltzmann method of Zhang, Guo & Li, "A fractional step lattice
 * Boltzmann model for two phase flows with large density differences"
 * (arXiv:1812.02459).  It exists so that the CUDA path can be checked against
 * something written directly from the paper.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Layout: every scalar field is a row-major double array [ny][nx]
 * (index j*nx + i, x = i, y = j); population sets are [9][ny][nx].
 * Lattice directions follow Sec. III.A, Eq. (D2Q9):
 *   c0=(0,0) c1=(1,0) c2=(0,1) c3=(-1,0) c4=(0,-1)
 *   c5=(1,1) c6=(-1,1) c7=(-1,-1) c8=(1,-1).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_NDIAG 10

typedef struct {
    int nx, ny;
    int periodic_x, periodic_y;   /* 0 on an axis => halfway bounce-back walls there */
    double M;        /* mobility of the Cahn-Hilliard equation, Sec. II.A Eq. (final_mCHE) */
    double eta;      /* adjustable CH equilibrium parameter, Sec. III.A Eqs. (feq_CH), (mobility) */
    double W;        /* interface width, Sec. II.A Eq. (equilibrium_profile) */
    double sigma;    /* surface tension; kappa=3 sigma W/8, beta=3 sigma/(4W), Sec. II.A */
    double lambda;   /* weight of the profile-correction flux J_phi (Sec. IV.B) */
    int flux_correction;  /* 1: include q (Sec. II.A); 0: drop it */
    double rho_H, rho_L;  /* densities of phi=+1 and phi=-1, Sec. II.B Eq. (rho) */
    double nu_H, nu_L;    /* kinematic viscosities of the two fluids */
    double s_f[9], s_g[9];/* MRT rates; s_f[3]=s_f[5]=1/tau_f and s_g[7]=s_g[8]=1/tau_g are overridden */
    double gx, gy;        /* gravitational acceleration */
    double g_rho_ref;     /* F_g = (rho - g_rho_ref) g; 0 gives rho g as printed */
    int filter_order;     /* 0 (off), 5, 7, 9 or 11: selective filter SF-n, App. B */
    double filter_a;      /* filter intensity a, Sec. III.B Eq. (filter) */
    int picard_iters;     /* sweeps of the implicit velocity update (maximum when zeta>0) */
    double picard_zeta;   /* 0: fixed number of sweeps; >0: stop when the residual < zeta */
    double grad_eps;      /* regularisation of |grad phi| inside n = grad phi / |grad phi| */
    unsigned flags;       /* bit 0: F_nu of the Picard sweeps takes its strain rate from Eq. (Fmu) */
} orc_params;

typedef struct orc_sim orc_sim;

/* ---- lattice and operator building blocks (exported for the pins) ---- */
void orc_lattice(int c[18], double w[9]);
void orc_mrt_matrix(double M[81]);
void orc_mrt_inverse(double Minv[81]);
void orc_filter_coeffs(int order, double d[6]);
void orc_feq(double phi, double mu, double ux, double uy, double eta, double out[9]);
void orc_geq(double p, double ux, double uy, double out[9]);
void orc_src_ch(double phi, double ax, double ay, double out[9]);
void orc_src_ns(double rho, double Fx, double Fy, double ux, double uy,
                double dpx, double dpy, double out[9]);
void orc_collide_f(const double f[9], const double feq[9], const double F[9],
                   const double s[9], double out[9]);
void orc_collide_g(const double g[9], const double geq_f[9], const double geq_hat[9],
                   const double G[9], const double s[9], double out[9]);
void orc_strain_moments(const double g[9], const double geq[9], const double s[9], double rho,
                        double Fx, double Fy, double ux, double uy, double out[3]);

/* Stencils on full periodic/walled fields; parity +1 even, -1 odd about a wall. */
void orc_grad_iso(int nx, int ny, int px, int py, int parity, const double *in,
                  double *gx, double *gy);
void orc_lap_iso(int nx, int ny, int px, int py, int parity, const double *in, double *out);
void orc_grad_fd4(int nx, int ny, int px, int py, int parity, const double *in,
                  double *gx, double *gy);
void orc_lap_fd4(int nx, int ny, int px, int py, int parity, const double *in, double *out);
void orc_filter(int nx, int ny, int px, int py, int parity, int order, double a,
                const double *in, double *out);
void orc_stream(int nx, int ny, int px, int py, const double *fstar, double *fout);
void orc_fd_rhs(const orc_params *prm, const double *psi, double *out);
typedef void (*orc_rhs_fn)(const double *psi, double *out, int n, void *ctx);
void orc_rk3(int n, const double *phibar, double *out, orc_rhs_fn L, void *ctx);

/* ---- whole-method simulation ---- */
int  orc_create(const orc_params *prm, const double *phi0, const double *p0,
                const double *ux0, const double *uy0, orc_sim **out);
int  orc_step(orc_sim *s, int n);
/* n steps of the Cahn-Hilliard part alone under the prescribed velocity
   (ux, uy) [ny][nx] (held for the n steps): collide and stream f, phi_bar,
   TVD-RK3.  Returns 2 on a non-finite phi. */
int  orc_step_ch(orc_sim *s, int n, const double *ux, const double *uy);
void orc_fields(const orc_sim *s, double *phi, double *p, double *ux, double *uy);
/* p' = rho(phi) p (the dynamic pressure) into out[ny][nx]. */
void orc_dynamic_pressure(const orc_sim *s, double *out);
void orc_state(const orc_sim *s, double *f, double *g, double *uhx, double *uhy,
               double *upx, double *upy);
void orc_set_state(orc_sim *s, const double *f, const double *g, const double *phi,
                   const double *p, const double *ux, const double *uy,
                   const double *uhx, const double *uhy, const double *upx, const double *upy);
void orc_diagnostics(const orc_sim *s, double out[ORC_NDIAG]);
int  orc_last_picard_sweeps(const orc_sim *s);
void orc_destroy(orc_sim *s);

#ifdef __cplusplus
}
#endif
#endif
