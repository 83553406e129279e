/*
 * oracle.h -- plain, slow FP64 reference of one explicit four-stage
 * low-storage Runge-Kutta step of the All-Mach THINC-TDU scheme
 * (Jiao, Schmidt & Adams, arXiv 2304.00140).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * Every step follows the paper in its own order (Algorithm 1, Sec. 3.1):
 * boundary update, primitive/thermodynamic update (App. A, App. B),
 * sensor (App. D, Eq. D.4), reconstruction (Sec. 3.3, Eq. 3-3/3-4,
 * Table 4.2; App. D Eq. D.1-D.3), thermodynamic-dependent update
 * (Eq. 3-5/3-6), all-Mach Riemann flux (Eq. 3-1/3-2; D.5/D.6), viscous
 * stress and heat conduction fluxes (Eq. 2-2, mixture viscosity Eq. 2-8),
 * CSF and gravity sources (Sec. 2.3, Sec. 3.5, Eq. 3-9/3-10, the
 * height-function option; Eq. 2-2 Q), flux divergence and the low-storage
 * Runge-Kutta update (Sec. 3.1).  Closures: stiffened / ideal gas
 * (App. A.1), Peng-Robinson (App. A.2.1), the barotropic model of Sec. 2.2
 * with the liquid-vapour density THINC of Sec. 3.4.
 *
 * Layouts: conserved state q and primitive state W are SoA float64 arrays
 * [nv][nz][ny][nx], x fastest, interior cells only.
 *   q = (rho, rho u_0..rho u_{d-1}, rho E, rho Y_0..rho Y_{N-2})   (Eq. 2-1)
 *   W = (u_0..u_{d-1}, p, T, Y_0..Y_{N-2})
 * With the barotropic closure (Sec. 2.2) p does not depend on the energy:
 * the slot of T holds the specific internal energy e.
 * The mass fraction of the last component is 1 - sum of the others.
 */
#ifndef THINC_ORACLE_H
#define THINC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAXC 4
#define OR_MAXV 10

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_NONPHYS = 2, OR_ERR_NONCONV = 3 };
enum { OR_BC_PERIODIC = 0, OR_BC_REFLECT = 1, OR_BC_OUTFLOW = 2, OR_BC_INFLOW = 3 };
enum { OR_SG = 0, OR_PR = 1, OR_BARO = 2 };
enum { OR_MINMOD = 0, OR_KOREN = 1, OR_VANLEER = 2, OR_VANALBADA = 3,
       OR_CHAKRAVARTHY = 4, OR_MC = 5, OR_SUPERBEE = 6 };

typedef struct {
    int kind;                         /* OR_SG (ideal gas when pinf = 0) or OR_PR */
    double gamma, pinf, cv, q;        /* Eq. A.1.1 */
    double Tc, pc, omega, M;          /* Eq. A.2.1 (M in kg/mol) */
    double mu, kc;                    /* viscosity (Pa s), conductivity (W/(m K)); Eq. 2-2, 2-8 */
    /* OR_BARO (Sec. 2.2): the liquid (rho_sl > 0) has saturation pressure
     * psat, saturated liquid / vapour densities rho_sl, rho_sv and liquid
     * sound speed cl (Eq. 2-3, 2-4, 2-7); a gas has rt = R T_ref (Eq. 2-5) */
    double psat, rho_sl, rho_sv, cl, rt;
} or_comp;

typedef struct {
    int ndim;                         /* 1, 2 or 3 */
    int n[3];                         /* interior cells; unused dims = 1 */
    double dx[3];
    int bc[3][2];                     /* OR_BC_* per dim, low/high side */
    int ncomp;                        /* N >= 2 */
    int liquid;                       /* component whose volume fraction feeds CSF */
    or_comp comp[OR_MAXC];
    int iles;                         /* 0: plain (f = 1 everywhere), 1: App. D switch */
    int thinc;                        /* THINC for mass fractions on eligible cells */
    double beta, thinc_eps, thinc_gamma;
    int lim_vel, lim_scalar;          /* limiter ids for velocity and p, T, Y */
    double thr_ducros, thr_gas, eps_ducros, d3p_coef;
    double sigma;                     /* surface tension coefficient; 0 = off */
    double grad_eps;                  /* |grad alpha~| * dx below this: n = 0 */
    /* inflow disc on the x-low face (OR_BC_INFLOW) */
    double in_yc, in_zc, in_radius, in_T;
    double in_Y[OR_MAXC];             /* tracked mass fractions of the inflow */
    const double* in_u;               /* [3][nz][ny] inflow velocity, or NULL */
    double in_u0[3];                  /* uniform inflow velocity used when in_u is NULL */
    double grav[3];                   /* body force per unit mass g (m/s^2), Eq. 2-2 Q */
    double thr_vap;                   /* App. D vapour-fraction threshold (barotropic closure) */
    int curv;                         /* CSF curvature: 0 Gaussian-smoothed vertex normals,
                                         1 height function (Sec. 3.5) */
    int st_model;                     /* surface tension: 0 CSF volume force (Sec. 2.3, 3.5),
                                         1 capillary pressure jump in the Riemann solver
                                         (the Sec. 3.5 alternative) */
} or_params;

/* threads of the cell loops (OpenMP; results do not depend on the count);
 * n < 1 keeps the setting; returns the count in use */
int or_set_threads(int n);

/* closure, pointwise (Yt = the N-1 tracked mass fractions) */
int or_closure_forward(const or_params* P, double p, double T, const double* Yt,
                       double* rho, double* e, double* c, double* alpha /* N */);
int or_closure_inverse(const or_params* P, double rho, double e, const double* Yt,
                       double* p, double* T);

/* Peng-Robinson pieces at (T, molar volume v): out = p, e, c, cv, a, b, M, da/dT */
int or_pr_state(const or_params* P, double T, double v, const double* Yt, double* out);

/* reconstruction pieces */
double or_limiter(int id, double r);
void or_muscl(int id, double x1, double x2, double x3, double x4, double* L, double* R);
void or_thinc(double beta, double gam, double x1, double x2, double x3, double x4,
              double* L, double* R);

/* one face: four cells' primitives along direction d (W[c*OR_MAXV + v]) and,
 * for the App. D switch, the face sensor value f and cell rho, c */
int or_face_flux(const or_params* P, int d, const double* W4, const double* rho4,
                 const double* c4, int f, double* F);

/* whole-field operations */
int or_prim_to_cons(const or_params* P, const double* W, double* q);
int or_cons_to_prim(const or_params* P, const double* q, double* W);
int or_stage(const or_params* P, int k, double dt, const double* q0, const double* qprev,
             double* qout, const int* wlo, const int* whi);
int or_dt(const or_params* P, const double* q, double cfl, double* dt);
int or_step(const or_params* P, double* q, int nsteps, double cfl, double* t);
void or_totals(const or_params* P, const double* q, double* out /* nv */);
/* CSF source on the interior (S[d+1][cells]: momentum then energy) */
/* curvature used by the CSF source on the interior (kappa[cells]) */
int or_curvature(const or_params* P, const double* q, double* kappa);
int or_csf_source(const or_params* P, const double* q, double* S);
/* App. D cell sensor f (0/1) on the interior */
/* Gaussian-smoothed liquid fraction of every interior cell (Eq. 3-9) */
int or_smoothed_fraction(const or_params* P, const double* q, double* out);
/* sound speed of a barotropic face state (p, rho, xi) (Sec. 3.4 Remark 2) */
int or_baro_sound_rho(const or_params* P, double p, double rho, const double* Yt, double* c);
int or_sensor(const or_params* P, const double* q, double* f);
/* App. D switch arguments on the interior: out[5][cells] = theta^D,
 * theta^Gas, theta^alpha, |div u|, |curl u| (Eq. D.4) */
int or_sensor_args(const or_params* P, const double* q, double* out);
/* height-function column axis (0..ndim-1) of each interior cell and the
 * relative gap between the largest and second-largest central difference
 * of the liquid fraction (Sec. 3.5 option) */
int or_hf_axis(const or_params* P, const double* q, double* axis, double* gap);
/* cell mixture viscosity and conductivity on the interior (out[2][cells]) */
int or_transport(const or_params* P, const double* q, double* out);
/* barotropic closure (Sec. 2.2): vapour volume fraction (Eq. 2-7) at p with
 * the phase fractions alpha of or_closure_forward */
double or_baro_vapour(const or_params* P, double p, const double* alpha);
/* one face with the cells' vapour fractions av4 for the liquid-vapour
 * density THINC (Sec. 3.4 Remarks 1-2; av4 NULL: none) */
int or_face_flux_av(const or_params* P, int d, const double* W4, const double* rho4, const double* c4,
                    const double* av4, int f, double* F);

/* capillary-jump surface tension (st_model = 1, the Sec. 3.5 alternative):
 * the momentum source of the face pressure jumps on each interior cell
 * (S[ndim][cells]), and one face with the curvatures and liquid fractions
 * al2 of its two cells (G: J/2 and u* J/2, the jump halves the two sides
 * take) */
int or_capillary_force(const or_params* P, const double* q, double* S);
int or_face_flux_kappa(const or_params* P, int d, const double* W4, const double* rho4, const double* c4, int f,
                       double kapL, double kapR, const double* al2, double* F, double* G);

#ifdef __cplusplus
}
#endif
#endif
