/*
 * ppm_oracle.h -- plain FP64 CPU oracle for the per-step bond loop of
 * updated Lagrangian unsaturated periporomechanics (Menon & Song,
 * arXiv:2203.05562).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may include,
 * link or call this code; only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no header, helper or
 * kernel with the CUDA path.
 *
 * Units are SI throughout (m, s, kg, Pa).  Sign convention: tension
 * positive for the solid skeleton, pore water pressure compression positive
 * (Sec. 1), so suction s > 0 means p_w = -s.
 *
 * Array layout: every per-point vector field is component-major,
 * f[c*n + i] for component c of point i; the symmetric stress uses the
 * order xx, yy, zz, yz, xz, xy.  The family is CSR: row_ptr[n+1],
 * col[B] (ascending within a row), rev[B] = index of bond (j,i) in row j.
 */
#ifndef PPM_ORACLE_H
#define PPM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t nx, ny, nz;          /* lattice of one soil column                */
    int32_t model;               /* 0 = bond-associated sub-horizon (Sec 2.2) */
                                 /* 1 = standard correspondence (Sec 2.1)     */
                                 /* 2 = sub-horizon, power-conjugate force    */
    double dx, horizon_factor;   /* lattice spacing, delta = factor * dx      */
    double rho, K, mu;           /* mixture density, bulk and shear modulus   */
    double M, lambda_t, kappa_t; /* critical-state slope, compression indices */
    double pc0, eta;             /* initial preconsolidation (>0), viscosity  */
    double suction;              /* constant matric suction s >= 0           */
    double vg_alpha, vg_n;       /* van Genuchten retention parameters        */
    double b1, b2;               /* Eq. 45 exponents; only b1=0, b2=1 allowed */
    double gravity[3];
    double dt;                   /* <= 0: 0.3 * dx / p-wave speed             */
    int32_t rebuild_every;       /* family rebuilt when (n+1) % R == 0; 0=never */
    int32_t init_stress;         /* 0 = K0 geostatic, 1 = zero                */
    int32_t visc_form;           /* 0 = eta scaled by pc_n^2, 1 = literal     */
    int32_t newton_max_iter;
    double newton_tol;
    int32_t lock_lateral;        /* 1: x,y motion suppressed (uniaxial strain) */
    int32_t bc;                  /* 0: base layer iz = 0 fixed (R18)          */
                                 /* 1: uniaxial compression along x (Sec. 4.1):
                                    the load_layers planes at ix = 0 held in x,
                                    those at ix = nx-1 moved at v_x =
                                    -load_rate; no fixed base                 */
    double load_rate;            /* m/s, bc = 1                               */
    int32_t elastic;             /* 1: linear (hypo-)elastic skeleton of Sec. 4.1,
                                    the yield test switched off               */
    int32_t load_layers;         /* bc = 1: lattice planes held / driven at each
                                    x end; 0 = floor(horizon_factor), the
                                    horizon's thickness                        */
    int32_t halt_on_unstable;    /* 1: once a step fails the Eq. 69 check, later
                                    steps change nothing                      */
    int32_t contact;             /* 1: a rigid flat substrate at z = -delta_c
                                    (Sec. 4.2, Eq. 91-93, readings R31-R33)
                                    instead of the fixed base layer           */
    double contact_modulus;      /* C_s (Pa)                                   */
    double friction;             /* mu_f                                       */
    double contact_cutoff;       /* delta_c / dx                               */
    double energy_tol;           /* tolerance of the Eq. 69 check; 0 = 1e-2    */
    int32_t plane_strain;        /* 1: plane strain in x-z (reading R35): y is
                                    periodic with period ny dx (ny dx > 4 delta)
                                    and v_y is held at zero                   */
    int32_t coupled;             /* 1: deformation-dependent porosity, degree of
                                    saturation, volume and mass (Eq. 15-16, 48-49;
                                    reading R37); rho and vg_* are then unused */
    double porosity;             /* phi_0, initial porosity                    */
    double rho_s, rho_w;         /* solid and water densities (kg/m^3)         */
    double wr_a1, wr_a2, wr_n;   /* Eq. 15: a1 (1/Pa), a2, n                   */
} ppmo_params;

typedef struct {
    int64_t n;                   /* points                                    */
    int64_t cap;                 /* bond capacity of col / rev / tforce       */
    int64_t nbonds;              /* bonds of the current family               */
    double *u, *v, *a;           /* 3n each                                   */
    double *sig;                 /* 6n effective stress                       */
    double *pc;                  /* n   preconsolidation pressure (negative)  */
    double *eps_s;               /* n   accumulated equivalent shear strain   */
    double *fint;                /* 3n  internal force of the last bond pass  */
    double *tforce;              /* 3*cap force state per bond (component-major, stride cap) */
    int32_t *row_ptr;            /* n+1 */
    int32_t *col, *rev;          /* cap */
    int64_t step;
    double W_int, W_ext, W_kin, W_kin0;
    int64_t n_plastic, n_nonconv, n_singular, n_overflow;
    int64_t unstable;            /* 1 once a step failed the Eq. 69 check         */
    int64_t halted_step;         /* halt_on_unstable: that step (from 1), else 0  */
    int64_t unstable_step;       /* the first step that failed it (from 1), else 0 */
    double *J;                   /* n: volume ratio (coupled = 1; else unused)   */
} ppmo_state;

/* Eq. (15) replaced by the van Genuchten curve (see DESIGN readings). */
double ppmo_saturation(double suction, double alpha, double n);
/* Coupled mode (reading R37): S_r of Eq. 15 at volume ratio J and suction s,
 * the porosity of Eq. 16 and the mixture density of Eq. 48 per current
 * volume. */
double ppmo_coupled_saturation(const ppmo_params* p, double J, double suction);
double ppmo_coupled_porosity(const ppmo_params* p, double J);
double ppmo_coupled_density(const ppmo_params* p, double J, double suction);
/* Time step used when p->dt <= 0: 0.3 dx / sqrt((K + 4 mu / 3) / rho), rho
 * the initial mixture density in the coupled mode. */
double ppmo_time_step(const ppmo_params* p);

/* Eq. (1): brute-force family search.  x is 3n component-major.  group may
 * be NULL (one body) or give a body id per point; points of different
 * bodies never bond.  Returns the bond count, or -1 if it exceeds cap
 * (row_ptr is still filled then). */
int64_t ppmo_family(int64_t n, const double* x, const int32_t* group, double delta,
                    int64_t cap, int32_t* row_ptr, int32_t* col, int32_t* rev);

/* Reference positions X0 = (ix, iy, iz) * dx of point ix + nx*(iy + ny*iz). */
void ppmo_reference_positions(const ppmo_params* p, double* X0);

/* Eq. (5)/(23), (25): per-bond shape tensor K_b (6 per bond, xx yy zz yz xz
 * xy), velocity gradient L_b (9 per bond, row-major L[r*3+c]), sub-horizon
 * size, and an active flag.  Positions x and velocities vel are 3n. */
int ppmo_bond_kinematics(const ppmo_params* p, int64_t n, const double* x, const double* vel,
                         const int32_t* row_ptr, const int32_t* col,
                         double* Kb, double* Lb, int32_t* count, int32_t* active);

/* Eq. (5), (8): full-horizon velocity gradient per point (9n, row-major). */
int ppmo_full_horizon_L(const ppmo_params* p, int64_t n, const double* x, const double* vel,
                        const int32_t* row_ptr, const int32_t* col, double* L);

/* Sec. 2.3 / 3.2.1: one constitutive update from the point state with the
 * velocity gradient L (row-major) over dt.  flags: bit0 plastic,
 * bit1 Newton did not converge.  deps_s = equivalent shear strain of dt*D. */
int ppmo_material_update(const ppmo_params* p, const double sig_n[6], double pc_n,
                         const double L[9], double dt, double sig_out[6], double* pc_out,
                         double* deps_s, int32_t* flags);

/* Eq. (73)-(75) residual and its exact Jacobian (row-major) at x = (p, q, pc). */
void ppmo_return_residual(const ppmo_params* p, double c, double p_tr, double q_tr,
                          double pc_n, const double x[3], double r[3], double J[9]);

/* Eq. (49), (51): internal force when every bond carries its point's stress
 * (no constitutive change).  f is 3n; T (3*B, may be NULL) gets the force states. */
int ppmo_internal_force(const ppmo_params* p, int64_t n, const double* x, const double* sig,
                        const int32_t* row_ptr, const int32_t* col, const int32_t* rev,
                        double* f);

/* Alg. 2, its initial state.  v0 is 3n (base layer is zeroed). */
int ppmo_init(const ppmo_params* p, const double* v0, ppmo_state* s);
/* The same with a given initial effective stress sig0 (6n; NULL: the
 * geostatic state of ppmo_initial_stress). */
int ppmo_init_with_stress(const ppmo_params* p, const double* v0, const double* sig0,
                          ppmo_state* s);
/* The same from an initial displacement u0 (3n; NULL: zero). */
int ppmo_init_state(const ppmo_params* p, const double* u0, const double* v0, const double* sig0,
                    ppmo_state* s);
/* Initial effective stress of the column (6n), O(n). */
void ppmo_initial_stress(const ppmo_params* p, double* sig);
/* Alg. 2, its time loop: n_steps explicit central-difference steps. */
int ppmo_step(const ppmo_params* p, ppmo_state* s, int n_steps);

/* J = sum over the top layer of (u_x^2 + u_y^2) after n_steps (Alg. 2 from
 * the initial state with velocities v0) and dJ/d(M, eta, suction, pc0) by
 * the reverse of every step, with the families, sub-horizons and
 * elastic/plastic branches of the forward run held fixed.  Models 0 and 1. */
int ppmo_objective_gradient(const ppmo_params* p, const double* v0, int n_steps, int64_t cap,
                            double* J, double grad[4]);

/* Threads used by the OpenMP loops (results do not depend on it). */
/* Critical time step of Eq. 65 (reading R30) over the current family and
 * positions of s; the minimum over points with bonds. */
double ppmo_critical_time_step(const ppmo_params* p, const ppmo_state* s);

int ppmo_num_threads(void);
void ppmo_set_num_threads(int t);

#ifdef __cplusplus
}
#endif
#endif
