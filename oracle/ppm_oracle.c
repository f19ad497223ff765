/*
 * ppm_oracle.c -- plain, slow FP64 CPU oracle of the per-step bond loop of
 * updated Lagrangian unsaturated periporomechanics (Menon & Song,
 * arXiv:2203.05562).
 *
 * TEST INFRASTRUCTURE ONLY: it exists so the GPU library can be checked
 * against something written straight from the paper.  The product library
 * never includes, links or calls it; only the tests, the package smoke
 * check and the benchmark's CPU-baseline leg do.
 *
 * Every loop follows the paper's statement in the paper's order; nothing is
 * blocked, fused or reordered for speed.  Compiled with -ffp-contract=off so
 * that no multiply-add is fused behind our back.  The only parallelism is an
 * OpenMP loop over points in which every point writes only its own outputs,
 * so results do not depend on the thread count.
 *
 * Readings of passages that are silent, garbled or inconsistent (each is
 * listed with its reason in the design notes):
 *   - a point is not a member of its own family; the bond partner j is a
 *     member of its own sub-horizon (Eq. 1, Eq. 22 and the sub-horizon test of Alg. 1);
 *   - membership is inclusive, tested on ((dx*dx + dy*dy) + dz*dz) <= delta^2;
 *   - influence function omega = 1; all point volumes V = dx^3, mass rho V;
 *   - D = sym(L) (Eq. 26), not the mixed form printed in Eq. 58;
 *   - objective stress rate: Hughes-Winget incremental rotation with the
 *     bond spin W = skew(L) (the paper is silent on the spin);
 *   - every bond starts from its point's state; the point state of step n+1
 *     is the varpi-weighted mean over its active bonds (internal variables on
 *     Lagrangian points, Sec. 1);
 *   - hardening follows Eq. 46 (compaction hardens), not the sign of Eq. 72;
 *     the viscosity is scaled by pc_n^2 unless visc_form = 1;
 *   - S_r from van Genuchten at constant suction (Eq. 15 is garbled);
 *   - Eq. 60 is read with the missing dt: v~ = v + (1-beta1) dt a;
 *   - the substrate of Eq. 91-93 is the plane z = -delta_c, its normal force
 *     C_s dx^2 (delta_c - d) / delta_c, its friction Coulomb's on the trial
 *     tangential velocity and never reversing it; the same repulsion acts
 *     between soil points closer than delta_c;
 *   - the tolerance of the Eq. 69 check is a parameter (1e-2 by default);
 *   - plane strain is a slab periodic in y with v_y held at zero;
 *   - the coupled mode reads Eq. 15 with the exponent -(n-1)/n, the void
 *     ratio J / (1 - phi_0) - 1 and a1 per Pa, and updates J from the bonds'
 *     volumetric rate.
 *
 * Parity unpinned (nothing in the paper or the mathematics fixes the
 * result independently of the reading): the configuration of the bond loop,
 * omega = 1, the constant point volumes, the point-state mean, the
 * viscosity scaling, b1 = 0 and b2 = 1 of Eq. 45, the geostatic initial
 * state, the van Genuchten curve, the ensemble sampler, and which force
 * state is used.  Everything else is pinned by the CPU tests against closed
 * forms, brute force, invariants or special cases.
 */
#include "ppm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* small dense 3x3 helpers, written out plainly                        */
/* ------------------------------------------------------------------ */

static void sym_to_mat(const double s[6], double m[3][3]) {
    m[0][0] = s[0]; m[1][1] = s[1]; m[2][2] = s[2];
    m[1][2] = s[3]; m[2][1] = s[3];
    m[0][2] = s[4]; m[2][0] = s[4];
    m[0][1] = s[5]; m[1][0] = s[5];
}

static void mat_to_sym(double m[3][3], double s[6]) {
    s[0] = m[0][0]; s[1] = m[1][1]; s[2] = m[2][2];
    s[3] = 0.5 * (m[1][2] + m[2][1]);
    s[4] = 0.5 * (m[0][2] + m[2][0]);
    s[5] = 0.5 * (m[0][1] + m[1][0]);
}

static double det3(double m[3][3]) {
    return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
         - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
         + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
}

/* inverse through the adjugate; returns 0 if det == 0 */
static int inv3(double m[3][3], double out[3][3]) {
    double d = det3(m);
    if (d == 0.0) return 0;
    out[0][0] = (m[1][1] * m[2][2] - m[1][2] * m[2][1]) / d;
    out[0][1] = (m[0][2] * m[2][1] - m[0][1] * m[2][2]) / d;
    out[0][2] = (m[0][1] * m[1][2] - m[0][2] * m[1][1]) / d;
    out[1][0] = (m[1][2] * m[2][0] - m[1][0] * m[2][2]) / d;
    out[1][1] = (m[0][0] * m[2][2] - m[0][2] * m[2][0]) / d;
    out[1][2] = (m[0][2] * m[1][0] - m[0][0] * m[1][2]) / d;
    out[2][0] = (m[1][0] * m[2][1] - m[1][1] * m[2][0]) / d;
    out[2][1] = (m[0][1] * m[2][0] - m[0][0] * m[2][1]) / d;
    out[2][2] = (m[0][0] * m[1][1] - m[0][1] * m[1][0]) / d;
    return 1;
}

static void matmul3(double A[3][3], double B[3][3], double C[3][3]) {
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            double s = 0.0;
            for (int m = 0; m < 3; m++) s += A[r][m] * B[m][c];
            C[r][c] = s;
        }
}

/* Gaussian elimination with partial pivoting: solves J x = r. */
static int solve3(double J[9], const double r[3], double x[3]) {
    double a[3][4];
    for (int i = 0; i < 3; i++) {
        for (int j = 0; j < 3; j++) a[i][j] = J[i * 3 + j];
        a[i][3] = r[i];
    }
    for (int c = 0; c < 3; c++) {
        int piv = c;
        for (int i = c + 1; i < 3; i++)
            if (fabs(a[i][c]) > fabs(a[piv][c])) piv = i;
        if (a[piv][c] == 0.0) return 0;
        if (piv != c)
            for (int j = 0; j < 4; j++) { double t = a[c][j]; a[c][j] = a[piv][j]; a[piv][j] = t; }
        for (int i = c + 1; i < 3; i++) {
            double m = a[i][c] / a[c][c];
            for (int j = c; j < 4; j++) a[i][j] -= m * a[c][j];
        }
    }
    for (int i = 2; i >= 0; i--) {
        double s = a[i][3];
        for (int j = i + 1; j < 3; j++) s -= a[i][j] * x[j];
        x[i] = s / a[i][i];
    }
    return 1;
}

/* ------------------------------------------------------------------ */
/* material data                                                       */
/* ------------------------------------------------------------------ */

/* van Genuchten retention curve at constant suction (stands in for the
 * garbled Eq. 15): S_r = [1 + (alpha s)^n]^-(1 - 1/n). */
double ppmo_saturation(double suction, double alpha, double n) {
    if (suction <= 0.0) return 1.0;
    return pow(1.0 + pow(alpha * suction, n), -(1.0 - 1.0 / n));
}

/* Eq. 15 with the exponent -(n - 1)/n (as printed, S_r >= 1) and the
 * porosity in it the initial one, so that J / (1 - phi_0) - 1 is the void
 * ratio e; p_w = -s.  A point with no voids left is saturated. */
double ppmo_coupled_saturation(const ppmo_params* p, double J, double suction) {
    const double e = J / (1.0 - p->porosity) - 1.0;
    if (!(suction > 0.0) || !(e > 0.0)) return 1.0;
    const double alpha = p->wr_a1 * pow(e, p->wr_a2) * J;
    return pow(1.0 + pow(alpha * suction, p->wr_n), -(p->wr_n - 1.0) / p->wr_n);
}

/* Eq. 16: phi = 1 - (1 - phi_0) / J */
double ppmo_coupled_porosity(const ppmo_params* p, double J) {
    return 1.0 - (1.0 - p->porosity) / J;
}

/* Eq. 48 per current volume: rho_s (1 - phi) + rho_w S_r phi */
double ppmo_coupled_density(const ppmo_params* p, double J, double suction) {
    const double phi = ppmo_coupled_porosity(p, J);
    return p->rho_s * (1.0 - phi) + p->rho_w * ppmo_coupled_saturation(p, J, suction) * phi;
}

/* the mixture density and S_r s at the start (J = 1) */
static double rho_start(const ppmo_params* p) {
    return p->coupled ? ppmo_coupled_density(p, 1.0, p->suction) : p->rho;
}
static double srs_at(const ppmo_params* p, double J) {
    if (p->coupled) return ppmo_coupled_saturation(p, J, p->suction) * p->suction;
    return ppmo_saturation(p->suction, p->vg_alpha, p->vg_n) * p->suction;
}

double ppmo_time_step(const ppmo_params* p) {
    if (p->dt > 0.0) return p->dt;
    double cp = sqrt((p->K + 4.0 * p->mu / 3.0) / rho_start(p));
    return 0.3 * p->dx / cp;
}

static int params_ok(const ppmo_params* p) {
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return 0;
    if (!(p->dx > 0) || !(p->horizon_factor > 0) || !(p->rho > 0)) return 0;
    if (!(p->K > 0) || !(p->mu > 0) || !(p->M > 0)) return 0;
    if (!(p->lambda_t > p->kappa_t) || !(p->eta > 0) || !(p->pc0 > 0)) return 0;
    if (p->b1 != 0.0 || p->b2 != 1.0) return 0;
    if (p->model < 0 || p->model > 2) return 0;
    if (p->newton_max_iter < 1 || !(p->newton_tol > 0)) return 0;
    if (!(p->energy_tol >= 0) || !isfinite(p->energy_tol)) return 0;
    if (p->plane_strain != 0 && p->plane_strain != 1) return 0;
    if (p->plane_strain && !((double)p->ny > 4.0 * p->horizon_factor)) return 0;
    if (p->coupled != 0 && p->coupled != 1) return 0;
    if (p->coupled && (!(p->porosity > 0.0 && p->porosity < 1.0) || !(p->rho_s > 0) ||
                       !(p->rho_w >= 0) || !(p->wr_a1 > 0) || !(p->wr_a2 >= 0) || !(p->wr_n > 1)))
        return 0;
    return 1;
}

/* ------------------------------------------------------------------ */
/* positions and family (Eq. 1; the family of Alg. 1)                   */
/* ------------------------------------------------------------------ */

void ppmo_reference_positions(const ppmo_params* p, double* X0) {
    int64_t n = (int64_t)p->nx * p->ny * p->nz;
    for (int64_t id = 0; id < n; id++) {
        int64_t ix = id % p->nx;
        int64_t iy = (id / p->nx) % p->ny;
        int64_t iz = id / ((int64_t)p->nx * p->ny);
        X0[0 * n + id] = (double)ix * p->dx;
        X0[1 * n + id] = (double)iy * p->dx;
        X0[2 * n + id] = (double)iz * p->dx;
    }
}

/* x_b - x_a, component c.  Under plane strain (reading R35) y is periodic
 * with period L = ny dx and the image of b is chosen by the lattice offset
 * so that |iy_b - iy_a| <= ny / 2: the image's y is x_b + s L, s = -1, 0, 1. */
static double rel(const ppmo_params* p, int64_t n, const double* x, int64_t a, int64_t b, int c) {
    if (c != 1 || !p || !p->plane_strain) return x[c * n + b] - x[c * n + a];
    const int64_t dl = (b / p->nx) % p->ny - (a / p->nx) % p->ny;
    const double L = (double)p->ny * p->dx;
    double xb = x[n + b];
    if (2 * dl > p->ny) xb = xb + -L;
    else if (2 * dl < -p->ny) xb = xb + L;
    return xb - x[n + a];
}

/* squared distance from a to b with the images of rel() */
static double dist2p(const ppmo_params* p, const double* x, int64_t n, int64_t a, int64_t b) {
    const double d0 = rel(p, n, x, a, b, 0), d1 = rel(p, n, x, a, b, 1), d2 = rel(p, n, x, a, b, 2);
    return (d0 * d0 + d1 * d1) + d2 * d2;
}

static int64_t family_impl(const ppmo_params* p, int64_t n, const double* x, const int32_t* group,
                           double delta, int64_t cap, int32_t* row_ptr, int32_t* col, int32_t* rev);

int64_t ppmo_family(int64_t n, const double* x, const int32_t* group, double delta,
                    int64_t cap, int32_t* row_ptr, int32_t* col, int32_t* rev) {
    return family_impl(NULL, n, x, group, delta, cap, row_ptr, col, rev);
}

/* Eq. 1 by brute force: H_i = {j != i : |x_j - x_i| <= delta}, ascending j */
static int64_t family_impl(const ppmo_params* p, int64_t n, const double* x, const int32_t* group,
                           double delta, int64_t cap, int32_t* row_ptr, int32_t* col, int32_t* rev) {
    const double d2max = delta * delta;
    int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -2;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        int64_t c = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            if (group && group[j] != group[i]) continue;
            if (dist2p(p, x, n, i, j) <= d2max) c++;
        }
        cnt[i + 1] = c;
    }
    for (int64_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    int64_t total = cnt[n];
    for (int64_t i = 0; i <= n; i++) row_ptr[i] = (int32_t)cnt[i];
    free(cnt);
    if (total > cap) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        int64_t pos = row_ptr[i];
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            if (group && group[j] != group[i]) continue;
            if (dist2p(p, x, n, i, j) <= d2max) col[pos++] = (int32_t)j;
        }
    }
    /* rev[b]: position of bond (j, i) in row j, found by bisection */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; b++) {
            int64_t j = col[b];
            int64_t lo = row_ptr[j], hi = row_ptr[j + 1];
            int32_t found = -1;
            while (lo < hi) {
                int64_t mid = (lo + hi) / 2;
                if (col[mid] < i) lo = mid + 1;
                else hi = mid;
            }
            if (lo < row_ptr[j + 1] && col[lo] == i) found = (int32_t)lo;
            rev[b] = found;
        }
    }
    return total;
}

/* ------------------------------------------------------------------ */
/* constitutive update (Sec. 2.3, Eq. 40-46; Sec. 3.2.1, Eq. 70-76)     */
/* ------------------------------------------------------------------ */

/* Residual of Eq. 73-75 with the hardening sign of Eq. 46, and its exact
 * Jacobian.  c = dt / eta_eff; x = (pbar, q, pbar_c).  Eq. 75 is taken in
 * logarithmic form, ln(pc / pc_n) + c f f_p / (lambda - kappa) = 0: the
 * same root, without overflow of the exponential far outside the yield
 * surface.  r[2] is +inf when pc / pc_n <= 0. */
void ppmo_return_residual(const ppmo_params* p, double c, double p_tr, double q_tr,
                          double pc_n, const double x[3], double r[3], double J[9]) {
    const double M2 = p->M * p->M;
    const double lk = p->lambda_t - p->kappa_t;
    double pb = x[0], q = x[1], pc = x[2];
    double f = q * q / M2 + pb * (pb - pc);          /* Eq. 40 */
    double fp = 2.0 * pb - pc;                       /* df/dp  */
    double fq = 2.0 * q / M2;                        /* df/dq  */
    double fc = -pb;                                 /* df/dpc, Eq. 87 */
    r[0] = pb - p_tr + p->K * c * f * fp;            /* Eq. 73 */
    r[1] = q - q_tr + 3.0 * p->mu * c * f * fq;      /* Eq. 74 */
    double ratio = pc / pc_n;
    r[2] = (ratio > 0.0) ? log(ratio) + c * f * fp / lk : INFINITY;   /* Eq. 75, 46 */
    if (J) {
        J[0] = 1.0 + p->K * c * (fp * fp + 2.0 * f);
        J[1] = p->K * c * fq * fp;
        J[2] = p->K * c * (fc * fp - f);
        J[3] = 3.0 * p->mu * c * fp * fq;
        J[4] = 1.0 + 3.0 * p->mu * c * (fq * fq + 2.0 * f / M2);
        J[5] = 3.0 * p->mu * c * fc * fq;
        J[6] = c / lk * (fp * fp + 2.0 * f);
        J[7] = c / lk * (fq * fp);
        J[8] = 1.0 / pc + c / lk * (fc * fp - f);
    }
}

/* residual with the two stress rows divided by the stress scale, so that
 * all three rows are dimensionless */
static void scaled_residual(const ppmo_params* p, double c, double p_tr, double q_tr,
                            double pc_n, double inv_scale, const double x[3], double r[3],
                            double* J) {
    ppmo_return_residual(p, c, p_tr, q_tr, pc_n, x, r, J);
    r[0] *= inv_scale;
    r[1] *= inv_scale;
    if (J)
        for (int k = 0; k < 6; k++) J[k] *= inv_scale;
}

static int finite3(const double r[3]) {
    return isfinite(r[0]) && isfinite(r[1]) && isfinite(r[2]);
}

static double norm_inf3(const double r[3]) {
    double m = fabs(r[0]);
    if (fabs(r[1]) > m) m = fabs(r[1]);
    if (fabs(r[2]) > m) m = fabs(r[2]);
    return m;
}

static double norm2_3(const double r[3]) {
    return sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
}

/* Backward-Euler visco-plastic return (Eq. 70-76) by Newton from the trial
 * state, with backtracking: a step is halved (at most 20 times) until the
 * scaled residual is finite and its 2-norm decreases.  Converged when the
 * scaled residual's max-norm is <= newton_tol, or when the Newton step is
 * below 1e-14 of the state.  Returns 1 if converged;
 * otherwise x keeps the last accepted iterate. */
static int return_map(const ppmo_params* p, double c, double p_tr, double q_tr, double pc_n,
                      double x[3]) {
    double scale = fabs(pc_n);
    if (fabs(p_tr) > scale) scale = fabs(p_tr);
    if (q_tr > scale) scale = q_tr;
    if (scale < 1.0) scale = 1.0;
    const double inv_scale = 1.0 / scale;
    x[0] = p_tr; x[1] = q_tr; x[2] = pc_n;
    double r[3], J[9];
    for (int it = 0; ; it++) {
        scaled_residual(p, c, p_tr, q_tr, pc_n, inv_scale, x, r, J);
        if (norm_inf3(r) <= p->newton_tol) return 1;
        if (it >= p->newton_max_iter) return 0;
        double dx[3];
        if (!solve3(J, r, dx)) return 0;
        /* a Newton step below 1e-14 of the state is the rounding floor of
         * the residual (f cancels near the yield surface): converged */
        if (fabs(dx[0]) <= 1e-14 * scale && fabs(dx[1]) <= 1e-14 * scale &&
            fabs(dx[2]) <= 1e-14 * fabs(x[2]))
            return 1;
        double rn = norm2_3(r);
        double lam = 1.0, xt[3], rt[3];
        int accepted = 0;
        for (int ls = 0; ls < 20; ls++) {
            for (int k = 0; k < 3; k++) xt[k] = x[k] - lam * dx[k];
            scaled_residual(p, c, p_tr, q_tr, pc_n, inv_scale, xt, rt, NULL);
            if (finite3(rt) && norm2_3(rt) < rn) { accepted = 1; break; }
            lam *= 0.5;
        }
        if (!accepted) return 0;
        for (int k = 0; k < 3; k++) x[k] = xt[k];
    }
}

/* Everything one constitutive update computes, kept for its reverse. */
typedef struct {
    double dt, pc_n;
    double W[3][3], Bm[3][3], Cm[3][3], Bi[3][3], Q[3][3], S[3][3], R[3][3];
    double de[3][3], Str[3][3], s_tr[3][3];
    double p_tr, q_tr, f_tr, c, eta_eff;
    double x[3];
    int plastic, converged, floored;
    double sig_out[6], pc_out, deps_s;
} mu_trace;

/* Sec. 2.3 / 3.2.1: rotation, trial stress, yield test and return */
static int mu_forward(const ppmo_params* p, const double sig_n[6], double pc_n, const double L[9],
                      double dt, mu_trace* t) {
    double D[3][3];
    t->dt = dt;
    t->pc_n = pc_n;
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            D[r][c] = 0.5 * (L[r * 3 + c] + L[c * 3 + r]);   /* Eq. 26 */
            t->W[r][c] = 0.5 * (L[r * 3 + c] - L[c * 3 + r]);
        }
    /* Hughes-Winget: Q = (I - dt/2 W)^-1 (I + dt/2 W), sigma_rot = Q sigma Q^T */
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            double I = (r == c) ? 1.0 : 0.0;
            t->Bm[r][c] = I - 0.5 * dt * t->W[r][c];
            t->Cm[r][c] = I + 0.5 * dt * t->W[r][c];
        }
    if (!inv3(t->Bm, t->Bi)) return -1;
    matmul3(t->Bi, t->Cm, t->Q);
    double QS[3][3], QT[3][3];
    sym_to_mat(sig_n, t->S);
    matmul3(t->Q, t->S, QS);
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) QT[r][c] = t->Q[c][r];
    matmul3(QS, QT, t->R);
    /* strain increment (Eq. 59) and linear hypo-elastic trial (Eq. 41) */
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) t->de[r][c] = dt * D[r][c];
    double trv = t->de[0][0] + t->de[1][1] + t->de[2][2];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            double I = (r == c) ? 1.0 : 0.0;
            t->Str[r][c] = t->R[r][c] + p->K * trv * I + 2.0 * p->mu * (t->de[r][c] - trv / 3.0 * I);
        }
    /* equivalent shear strain of the increment */
    double ss = 0.0;
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            double I = (r == c) ? 1.0 : 0.0;
            double e = t->de[r][c] - trv / 3.0 * I;
            ss += e * e;
        }
    t->deps_s = sqrt(2.0 / 3.0 * ss);
    /* invariants and yield function, Eq. 40 */
    t->p_tr = (t->Str[0][0] + t->Str[1][1] + t->Str[2][2]) / 3.0;
    double sn = 0.0;
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            double I = (r == c) ? 1.0 : 0.0;
            t->s_tr[r][c] = t->Str[r][c] - t->p_tr * I;
            sn += t->s_tr[r][c] * t->s_tr[r][c];
        }
    t->q_tr = sqrt(1.5 * sn);
    t->f_tr = t->q_tr * t->q_tr / (p->M * p->M) + t->p_tr * (t->p_tr - pc_n);
    t->plastic = 0;
    t->converged = 1;
    t->floored = 0;
    if (!(t->f_tr > 0.0) || dt == 0.0 || p->elastic) {   /* elastic, Eq. 44 */
        mat_to_sym(t->Str, t->sig_out);
        t->pc_out = pc_n;
        return 0;
    }
    t->plastic = 1;
    t->eta_eff = (p->visc_form == 0) ? p->eta * pc_n * pc_n : p->eta;
    t->c = dt / t->eta_eff;
    t->converged = return_map(p, t->c, t->p_tr, t->q_tr, pc_n, t->x);
    double ratio = (t->q_tr > 0.0) ? t->x[1] / t->q_tr : 0.0;
    double out[3][3];
    for (int r = 0; r < 3; r++)
        for (int cc = 0; cc < 3; cc++) {
            double I = (r == cc) ? 1.0 : 0.0;
            out[r][cc] = t->x[0] * I + ratio * t->s_tr[r][cc];
        }
    mat_to_sym(out, t->sig_out);
    double pc_new = t->x[2];
    if (pc_new > -1.0) { pc_new = -1.0; t->floored = 1; }   /* floor at the apex */
    t->pc_out = pc_new;
    return 0;
}

int ppmo_material_update(const ppmo_params* p, const double sig_n[6], double pc_n,
                         const double L[9], double dt, double sig_out[6], double* pc_out,
                         double* deps_s, int32_t* flags) {
    mu_trace t;
    if (mu_forward(p, sig_n, pc_n, L, dt, &t) != 0) return -1;
    for (int c = 0; c < 6; c++) sig_out[c] = t.sig_out[c];
    *pc_out = t.pc_out;
    *deps_s = t.deps_s;
    *flags = t.plastic ? (1 | (t.converged ? 0 : 2)) : 0;
    return 0;
}

/* ------------------------------------------------------------------ */
/* bond-associated sub-horizon kinematics (Eq. 22-26, 55, 57)          */
/* ------------------------------------------------------------------ */

typedef struct {
    double K[3][3], A[3][3];
    int32_t count;
} subhorizon_sums;

/* Sums over the sub-horizon of bond (i, j): S = {k in H_i : |x_k - x_j| <= delta}
 * (the sub-horizon test of Alg. 1); the standard model takes S = H_i. */
static void subhorizon(const ppmo_params* p, int64_t n, const double* x, const double* vel,
                       const int32_t* row_ptr, const int32_t* col, int64_t i, int64_t j,
                       subhorizon_sums* s) {
    const double delta = p->horizon_factor * p->dx;
    const double d2max = delta * delta;
    const double V = p->dx * p->dx * p->dx;
    const double omega = 1.0;
    memset(s, 0, sizeof(*s));
    for (int64_t b2 = row_ptr[i]; b2 < row_ptr[i + 1]; b2++) {
        int64_t k = col[b2];
            int member = (p->model == 1) || (dist2p(p, x, n, j, k) <= d2max);
        if (!member) continue;
        double zeta[3], ydot[3];
        for (int c = 0; c < 3; c++) {
            zeta[c] = rel(p, n, x, i, k, c);
            ydot[c] = vel[c * n + k] - vel[c * n + i];
        }
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) {
                s->K[r][c] += omega * zeta[r] * zeta[c] * V;   /* Eq. 23 */
                s->A[r][c] += omega * ydot[r] * zeta[c] * V;   /* Eq. 25 / 57 */
            }
        s->count++;
    }
}

/* Inactive-bond rule: fewer than three sub-horizon members or a shape
 * tensor whose determinant is below 1e-12 (tr K / 3)^3. */
static int shape_ok(int32_t count, double K[3][3]) {
    if (count < 3) return 0;
    double t = (K[0][0] + K[1][1] + K[2][2]) / 3.0;
    return det3(K) > 1e-12 * t * t * t;
}

int ppmo_bond_kinematics(const ppmo_params* p, int64_t n, const double* x, const double* vel,
                         const int32_t* row_ptr, const int32_t* col,
                         double* Kb, double* Lb, int32_t* count, int32_t* active) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; b++) {
            subhorizon_sums s;
            subhorizon(p, n, x, vel, row_ptr, col, i, col[b], &s);
            double ks[6];
            mat_to_sym(s.K, ks);
            for (int c = 0; c < 6; c++) Kb[b * 6 + c] = ks[c];
            count[b] = s.count;
            double Ki[3][3], L[3][3];
            int ok = shape_ok(s.count, s.K) && inv3(s.K, Ki);
            active[b] = ok;
            if (ok) matmul3(s.A, Ki, L);
            for (int r = 0; r < 3; r++)
                for (int c = 0; c < 3; c++) Lb[b * 9 + r * 3 + c] = ok ? L[r][c] : 0.0;
        }
    }
    return 0;
}

int ppmo_full_horizon_L(const ppmo_params* p, int64_t n, const double* x, const double* vel,
                        const int32_t* row_ptr, const int32_t* col, double* Lout) {
    const double V = p->dx * p->dx * p->dx;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double K[3][3] = {{0}}, A[3][3] = {{0}};
        for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; b++) {
            int64_t k = col[b];
            double zeta[3], ydot[3];
            for (int c = 0; c < 3; c++) {
                zeta[c] = rel(p, n, x, i, k, c);
                ydot[c] = vel[c * n + k] - vel[c * n + i];
            }
            for (int r = 0; r < 3; r++)
                for (int c = 0; c < 3; c++) {
                    K[r][c] += zeta[r] * zeta[c] * V;          /* Eq. 5 */
                    A[r][c] += ydot[r] * zeta[c] * V;          /* Eq. 8 */
                }
        }
        double Ki[3][3], L[3][3];
        int ok = inv3(K, Ki);
        if (ok) matmul3(A, Ki, L);
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) Lout[i * 9 + r * 3 + c] = ok ? L[r][c] : 0.0;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* the bond pass: Alg. 1 (force states, Eq. 31-32, 51-56)               */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t plastic, nonconv, singular;
} pass_counts;

/* One pass over every bond of every point at positions x and velocities
 * vel.  T (3 x cap, component-major) receives the total force state of
 * each bond; fint the internal force per point (Eq. 49-50).  With dt == 0
 * every bond carries its point's stress unchanged; otherwise the point
 * state (sig, pc, eps_s) is replaced by the varpi-weighted bond mean. */
static void bond_pass(const ppmo_params* p, int64_t n, const double* x, const double* vel,
                      double dt, const int32_t* row_ptr, const int32_t* col,
                      const int32_t* rev, int64_t cap, double* sig, double* pc,
                      double* eps_s, int update, double* T, double* fint,
                      pass_counts* cnt_out, const double* J, double* Jnew) {
    const double V = p->dx * p->dx * p->dx;
    const double omega = 1.0;
    const double Srs = srs_at(p, 1.0);
    const double delta = p->horizon_factor * p->dx;
    const double d2max = delta * delta;
    int64_t plastic = 0, nonconv = 0, singular = 0;
#pragma omp parallel for schedule(static) reduction(+ : plastic, nonconv, singular)
    for (int64_t i = 0; i < n; i++) {
        int64_t nb = row_ptr[i + 1] - row_ptr[i];
        double sig_i[6];
        for (int c = 0; c < 6; c++) sig_i[c] = sig[c * n + i];
        double pc_i = pc[i];
        double w = 0.0, acc_sig[6] = {0}, acc_pc = 0.0, acc_es = 0.0, acc_ev = 0.0;
        /* coupled mode: S_r of the point's volume at the start of the step */
        const double Srs_i = (p->coupled && J) ? srs_at(p, J[i]) : Srs;
        for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; b++)
            for (int c = 0; c < 3; c++) T[c * cap + b] = 0.0;
        for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; b++) {
            int64_t j = col[b];
            subhorizon_sums s;
            subhorizon(p, n, x, vel, row_ptr, col, i, j, &s);
            double Ki[3][3];
            if (!shape_ok(s.count, s.K) || !inv3(s.K, Ki)) {
                singular++;
                continue;
            }
            double varpi = (double)s.count / (double)nb;          /* Eq. 55 */
            double sig_b[6], pc_b = pc_i, des = 0.0;
            if (dt == 0.0) {
                for (int c = 0; c < 6; c++) sig_b[c] = sig_i[c];
            } else {
                double L[3][3], Lf[9];
                matmul3(s.A, Ki, L);                                  /* Eq. 57 */
                for (int r = 0; r < 3; r++)
                    for (int c = 0; c < 3; c++) Lf[r * 3 + c] = L[r][c];
                int32_t fl = 0;
                ppmo_material_update(p, sig_i, pc_i, Lf, dt, sig_b, &pc_b, &des, &fl);
                if (fl & 1) plastic++;
                if (fl & 2) nonconv++;
                /* the bond's volumetric strain increment (reading R37) */
                acc_ev += varpi * dt * (L[0][0] + L[1][1] + L[2][2]);
            }
            /* total stress sigma_bar - S_r p_w 1 with p_w = -s (Eq. 32) */
            double St[3][3], SK[3][3];
            sym_to_mat(sig_b, St);
            for (int c = 0; c < 3; c++) St[c][c] += Srs_i;
            matmul3(St, Ki, SK);
            if (p->model == 2) {
                /* power-conjugate form: the force state of this sub-horizon
                 * acts on every member k of it (Eq. 27, 30-31 read as a state
                 * over H_s); the row is normalised by sum(varpi) below */
                for (int64_t b2 = row_ptr[i]; b2 < row_ptr[i + 1]; b2++) {
                    int64_t k = col[b2];
                    if (!(dist2p(p, x, n, j, k) <= d2max)) continue;
                    double zk[3];
                    for (int c = 0; c < 3; c++) zk[c] = rel(p, n, x, i, k, c);
                    for (int r = 0; r < 3; r++) {
                        double t = 0.0;
                        for (int c = 0; c < 3; c++) t += SK[r][c] * zk[c];
                        T[r * cap + b2] += varpi * omega * t;
                    }
                }
            } else {
                /* Eq. 31-32, 51: the force state on the bond itself */
                double zj[3];
                for (int c = 0; c < 3; c++) zj[c] = rel(p, n, x, i, j, c);
                for (int r = 0; r < 3; r++) {
                    double t = 0.0;
                    for (int c = 0; c < 3; c++) t += SK[r][c] * zj[c];
                    T[r * cap + b] = varpi * omega * t;
                }
            }
            w += varpi;
            for (int c = 0; c < 6; c++) acc_sig[c] += varpi * sig_b[c];
            acc_pc += varpi * pc_b;
            acc_es += varpi * des;
        }
        if (p->model == 2 && w > 0.0)
            for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; b++)
                for (int c = 0; c < 3; c++) T[c * cap + b] /= w;
        if (update && w > 0.0) {
            for (int c = 0; c < 6; c++) sig[c * n + i] = acc_sig[c] / w;
            pc[i] = acc_pc / w;
            eps_s[i] += acc_es / w;
        }
        /* J_{n+1} = J_n exp(varpi-mean of dt tr L_b) (reading R37) */
        if (Jnew) Jnew[i] = (update && w > 0.0) ? J[i] * exp(acc_ev / w) : J[i];
    }
    /* pairwise nodal force, Eq. 49-50: f_i = V_i sum_j (T_(ij) - T_(ji)) V_j,
     * with V = J dx^3 in the coupled mode (J at the start of the step) */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        for (int c = 0; c < 3; c++) {
            double s = 0.0;
            for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; b++) {
                const double Vj = (p->coupled && J) ? J[col[b]] : 1.0;
                s += (T[c * cap + b] - T[c * cap + rev[b]]) * Vj;
            }
            fint[c * n + i] = V * V * s * ((p->coupled && J) ? J[i] : 1.0);
        }
    }
    /* Eq. 91 between material points of the soil (reading R36): a pair
     * closer than delta_c (always family members, delta_c < delta) pushes
     * each of its points from the other by C_s dx^2 (delta_c - r) / delta_c
     * along the line joining them; coincident points get nothing */
    if (p->contact) {
        const double dc = p->contact_cutoff * p->dx;
        const double kc = p->contact_modulus * p->dx * p->dx / dc;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++)
            for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; b++) {
                double d[3];
                for (int c = 0; c < 3; c++) d[c] = rel(p, n, x, i, col[b], c);
                const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                if (r > 0.0 && r < dc)
                    for (int c = 0; c < 3; c++) fint[c * n + i] -= kc * (dc - r) * d[c] / r;
            }
    }
    if (cnt_out) {
        cnt_out->plastic = plastic;
        cnt_out->nonconv = nonconv;
        cnt_out->singular = singular;
    }
}

int ppmo_internal_force(const ppmo_params* p, int64_t n, const double* x, const double* sig,
                        const int32_t* row_ptr, const int32_t* col, const int32_t* rev,
                        double* f) {
    int64_t B = row_ptr[n];
    double* T = (double*)malloc(sizeof(double) * 3 * (size_t)(B > 0 ? B : 1));
    double* sg = (double*)malloc(sizeof(double) * 6 * (size_t)n);
    double* pcs = (double*)calloc((size_t)n, sizeof(double));
    double* es = (double*)calloc((size_t)n, sizeof(double));
    if (!T || !sg || !pcs || !es) { free(T); free(sg); free(pcs); free(es); return -2; }
    memcpy(sg, sig, sizeof(double) * 6 * (size_t)n);
    double* vel = (double*)calloc(3 * (size_t)n, sizeof(double));
    bond_pass(p, n, x, vel, 0.0, row_ptr, col, rev, B, sg, pcs, es, 0, T, f, NULL, NULL, NULL);
    free(vel); free(T); free(sg); free(pcs); free(es);
    return 0;
}

/* ------------------------------------------------------------------ */
/* explicit Newmark / central difference (Eq. 60-64, Alg. 2)           */
/* ------------------------------------------------------------------ */

static int is_base(const ppmo_params* p, int64_t id) {
    return (id / ((int64_t)p->nx * p->ny)) == 0;
}

/* Boundary conditions (R18; the loading of Sec. 4.1): returns 1 when
 * velocity component c of point id is prescribed, with the value in *vbar.
 * bc = 0: the base layer and, with lock_lateral, the x and y components
 * are held at zero.  bc = 1: the load_layers lattice planes at the x = 0
 * end are held in x and those at the other end move at v_x = -load_rate
 * (lock_lateral still holds x, y); by default the loaded regions are a
 * horizon thick (reading R28). */
static int constrained(const ppmo_params* p, int64_t id, int c, double* vbar) {
    *vbar = 0.0;
    if (p->lock_lateral && c < 2) return 1;
    if (p->plane_strain && c == 1) return 1;
    if (p->bc == 0) return !p->contact && is_base(p, id);
    if (c != 0) return 0;
    const int64_t ix = id % p->nx;
    int64_t nl = p->load_layers > 0 ? p->load_layers : (int64_t)p->horizon_factor;
    if (nl < 1) nl = 1;
    if (ix < nl) return 1;
    if (ix >= p->nx - nl) {
        *vbar = -p->load_rate;
        return 1;
    }
    return 0;
}

/* Contact with a rigid flat substrate (Sec. 4.2, Eq. 91-93; readings
 * R31-R33): the substrate is the plane z = -delta_c below the bottom layer;
 * each point's virtual bond goes to its projection on the plane.  At a
 * distance d < delta_c the normal force is C_s dx^2 (delta_c - d) / delta_c
 * (the contact modulus on the point's tributary area), and Coulomb friction
 * opposes the tangential velocity the point would have at the end of the
 * half step without it, |F_t| <= mu_f F_n, limited so that it never
 * reverses that velocity.  The forces are added to f (x: positions, w: the
 * velocity the step starts the half step from, hdt: half the step). */
/* point masses (Eq. 48): rho dx^3, or in the coupled mode the mixture
 * density of the volume ratio J times J dx^3 */
static void point_masses(const ppmo_params* p, int64_t n, const double* J, double* mass) {
    const double V = p->dx * p->dx * p->dx;
    for (int64_t i = 0; i < n; i++)
        mass[i] = p->coupled ? ppmo_coupled_density(p, J[i], p->suction) * J[i] * V : p->rho * V;
}

static void add_contact(const ppmo_params* p, int64_t n, const double* x, const double* w,
                        double hdt, const double* mass, double* f) {
    const double dc = p->contact_cutoff * p->dx;
    const double zs = -dc;
    for (int64_t i = 0; i < n; i++) {
        const double d = x[2 * n + i] - zs;
        if (!(d < dc)) continue;
        const double Fn = p->contact_modulus * p->dx * p->dx * (dc - d) / dc;
        f[2 * n + i] += Fn;
        if (p->friction > 0.0 && hdt > 0.0) {
            double vt[2], nrm = 0.0;
            for (int c = 0; c < 2; c++) {
                vt[c] = w[c * n + i] + hdt * (f[c * n + i] / mass[i] + p->gravity[c]);
                nrm += vt[c] * vt[c];
            }
            nrm = sqrt(nrm);
            if (nrm > 0.0) {
                const double Ft = fmin(p->friction * Fn, mass[i] * nrm / hdt);
                for (int c = 0; c < 2; c++) f[c * n + i] -= Ft * vt[c] / nrm;
            }
        }
    }
}

static void current_positions(const ppmo_params* p, int64_t n, const double* u, double* x) {
    ppmo_reference_positions(p, x);
    for (int64_t k = 0; k < 3 * n; k++) x[k] += u[k];
}

static int rebuild(const ppmo_params* p, ppmo_state* s, const double* x) {
    int32_t* rp = (int32_t*)malloc(sizeof(int32_t) * ((size_t)s->n + 1));
    int32_t* cl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s->cap > 0 ? s->cap : 1));
    int32_t* rv = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s->cap > 0 ? s->cap : 1));
    if (!rp || !cl || !rv) { free(rp); free(cl); free(rv); return -2; }
    int64_t B = family_impl(p, s->n, x, NULL, p->horizon_factor * p->dx, s->cap, rp, cl, rv);
    if (B < 0) {                      /* keep the previous family */
        s->n_overflow++;
        free(rp); free(cl); free(rv);
        return (int)B;
    }
    memcpy(s->row_ptr, rp, sizeof(int32_t) * ((size_t)s->n + 1));
    memcpy(s->col, cl, sizeof(int32_t) * (size_t)B);
    memcpy(s->rev, rv, sizeof(int32_t) * (size_t)B);
    s->nbonds = B;
    free(rp); free(cl); free(rv);
    return 0;
}

/* R13: geostatic effective stress with a traction-free top -- total stress
 * sigma_zz = -rho g d, sigma_xx = sigma_yy = K0 sigma_zz with K0 = nu/(1 - nu),
 * d the depth below the top layer; effective = total - S_r s 1.  Zero when
 * init_stress = 1.  sig is 6n. */
void ppmo_initial_stress(const ppmo_params* p, double* sig) {
    int64_t n = (int64_t)p->nx * p->ny * p->nz;
    const double Srs = srs_at(p, 1.0);
    const double nu = (3.0 * p->K - 2.0 * p->mu) / (2.0 * (3.0 * p->K + p->mu));
    const double K0 = nu / (1.0 - nu);
    const double gmag = -p->gravity[2];
    for (int64_t i = 0; i < n; i++) {
        int64_t iz = i / ((int64_t)p->nx * p->ny);
        for (int c = 0; c < 6; c++) sig[c * n + i] = 0.0;
        if (p->init_stress == 0) {
            double d = (double)(p->nz - 1 - iz) * p->dx;
            double szz = -rho_start(p) * gmag * d;
            sig[0 * n + i] = K0 * szz - Srs;
            sig[1 * n + i] = K0 * szz - Srs;
            sig[2 * n + i] = szz - Srs;
        }
    }
}

int ppmo_init_with_stress(const ppmo_params* p, const double* v0, const double* sig0,
                          ppmo_state* s) {
    return ppmo_init_state(p, NULL, v0, sig0, s);
}

int ppmo_init_state(const ppmo_params* p, const double* u0, const double* v0, const double* sig0,
                    ppmo_state* s) {
    if (!params_ok(p)) return -1;
    int64_t n = (int64_t)p->nx * p->ny * p->nz;
    if (s->n != n) return -1;
    for (int64_t i = 0; i < n; i++) {
        for (int c = 0; c < 3; c++) {
            s->u[c * n + i] = u0 ? u0[c * n + i] : 0.0;
            double vv = v0 ? v0[c * n + i] : 0.0, vbar;
            if (constrained(p, i, c, &vbar)) vv = vbar;
            s->v[c * n + i] = vv;
        }
        s->pc[i] = -p->pc0;        /* b1 = 0, b2 = 1: pbar_c = p_c (Eq. 45) */
        s->eps_s[i] = 0.0;
    }
    if (sig0) memcpy(s->sig, sig0, sizeof(double) * 6 * (size_t)n);
    else ppmo_initial_stress(p, s->sig);
    double* x = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    if (!x) return -2;
    current_positions(p, n, s->u, x);
    s->n_overflow = 0;
    int rc = rebuild(p, s, x);
    if (rc < 0) { free(x); return rc; }
    for (int64_t i = 0; i < n; i++) s->J[i] = 1.0;
    double* mass = (double*)malloc(sizeof(double) * (size_t)n);
    if (!mass) { free(x); return -2; }
    point_masses(p, n, s->J, mass);
    bond_pass(p, n, x, s->v, 0.0, s->row_ptr, s->col, s->rev, s->cap, s->sig, s->pc,
              s->eps_s, 0, s->tforce, s->fint, NULL, s->J, NULL);
    if (p->contact) add_contact(p, n, x, s->v, 0.5 * ppmo_time_step(p), mass, s->fint);
    double wk = 0.0;
    for (int64_t i = 0; i < n; i++)
        for (int c = 0; c < 3; c++) {
            double a = s->fint[c * n + i] / mass[i] + p->gravity[c], vbar;      /* Eq. 62 */
            if (constrained(p, i, c, &vbar)) a = 0.0;
            s->a[c * n + i] = a;
            wk += 0.5 * mass[i] * s->v[c * n + i] * s->v[c * n + i];
        }
    free(x); free(mass);
    s->step = 0;
    s->W_int = 0.0; s->W_ext = 0.0; s->W_kin = wk; s->W_kin0 = wk;
    s->n_plastic = s->n_nonconv = s->n_singular = 0;
    s->unstable = 0;
    s->halted_step = 0;
    s->unstable_step = 0;
    return 0;
}

int ppmo_init(const ppmo_params* p, const double* v0, ppmo_state* s) {
    return ppmo_init_with_stress(p, v0, NULL, s);
}

int ppmo_step(const ppmo_params* p, ppmo_state* s, int n_steps) {
    if (!params_ok(p)) return -1;
    const int64_t n = s->n;
    const double dt = ppmo_time_step(p);
    double* x = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* vh = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* f_old = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* mass = (double*)malloc(sizeof(double) * (size_t)n);
    double* Jnew = (double*)malloc(sizeof(double) * (size_t)n);
    if (!x || !vh || !f_old || !mass || !Jnew) {
        free(x); free(vh); free(f_old); free(mass); free(Jnew);
        return -2;
    }
    for (int st = 0; st < n_steps; st++) {
        if (p->halt_on_unstable && s->halted_step) {     /* the run has stopped */
            s->step++;
            continue;
        }
        memcpy(f_old, s->fint, sizeof(double) * 3 * (size_t)n);
        /* masses of the volumes at the start of the step (Eq. 48) */
        point_masses(p, n, s->J, mass);
        /* predictor, Eq. 60-61 with beta1 = 1/2, beta2 = 0; boundary
         * conditions; displacement, Eq. 64 (the predictor of Alg. 2) */
        for (int64_t i = 0; i < n; i++)
            for (int c = 0; c < 3; c++) {
                double v = s->v[c * n + i] + 0.5 * dt * s->a[c * n + i], vbar;
                if (constrained(p, i, c, &vbar)) v = vbar;
                vh[c * n + i] = v;
                s->u[c * n + i] += dt * v;
            }
        current_positions(p, n, s->u, x);
        if (p->rebuild_every > 0 && (s->step + 1) % p->rebuild_every == 0) rebuild(p, s, x);
        /* internal force, Alg. 1 (called from the time loop of Alg. 2) */
        pass_counts pcnt;
        bond_pass(p, n, x, vh, dt, s->row_ptr, s->col, s->rev, s->cap, s->sig, s->pc,
                  s->eps_s, 1, s->tforce, s->fint, &pcnt, s->J, Jnew);
        s->n_plastic += pcnt.plastic;
        s->n_nonconv += pcnt.nonconv;
        s->n_singular += pcnt.singular;
        if (p->contact) add_contact(p, n, x, vh, 0.5 * dt, mass, s->fint);
        /* acceleration and velocity corrector, Eq. 62-63 */
        double dWi = 0.0, dWe = 0.0, wk = 0.0;
        for (int64_t i = 0; i < n; i++)
            for (int c = 0; c < 3; c++) {
                const double m = mass[i];
                double a = s->fint[c * n + i] / m + p->gravity[c], vbar;
                const int fixed = constrained(p, i, c, &vbar);
                if (fixed) a = 0.0;
                s->a[c * n + i] = a;
                double v = vh[c * n + i] + 0.5 * dt * a;
                s->v[c * n + i] = v;
                /* energies, Eq. 66-68: stored energy = minus the work of the
                 * internal force; external work of gravity */
                dWi += -0.5 * dt * vh[c * n + i] * (f_old[c * n + i] + s->fint[c * n + i]);
                dWe += 0.5 * dt * vh[c * n + i] * (2.0 * m * p->gravity[c]);
                /* a prescribed component moves under the reaction R = -(f + m g)
                 * that cancels its acceleration; its work is external (zero
                 * where the component is held) */
                if (fixed)
                    dWe += -0.5 * dt * vh[c * n + i] *
                           (f_old[c * n + i] + s->fint[c * n + i] + 2.0 * m * p->gravity[c]);
                wk += 0.5 * m * v * v;
            }
        s->W_int += dWi;
        s->W_ext += dWe;
        s->W_kin = wk;
        s->step++;
        if (p->coupled) memcpy(s->J, Jnew, sizeof(double) * (size_t)n);
        /* the energy check of Eq. 69 (R20): diagnostic, or a hard stop */
        const double bal = fabs(s->W_int + s->W_kin - s->W_ext - s->W_kin0);
        const double mx = fmax(fmax(s->W_kin, fabs(s->W_int)), fmax(fabs(s->W_ext), s->W_kin0));
        if (bal > (p->energy_tol > 0 ? p->energy_tol : 1e-2) * mx) {
            if (!s->unstable) s->unstable_step = s->step;
            s->unstable = 1;
            if (p->halt_on_unstable && !s->halted_step) s->halted_step = s->step;
        }
    }
    free(x); free(vh); free(f_old); free(mass); free(Jnew);
    return 0;
}

/* ------------------------------------------------------------------ */
/* reverse (adjoint) of the step, for the gradient of an objective     */
/* ------------------------------------------------------------------ */

static void transpose3(double A[3][3], double T[3][3]) {
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) T[r][c] = A[c][r];
}

/* full symmetric adjoint (off-diagonals shared) -> 6 stored components */
static void sym_adj_to6(double M[3][3], double a6[6]) {
    a6[0] = M[0][0]; a6[1] = M[1][1]; a6[2] = M[2][2];
    a6[3] = M[1][2] + M[2][1]; a6[4] = M[0][2] + M[2][0]; a6[5] = M[0][1] + M[1][0];
}

/* 6 stored components -> full symmetric adjoint */
static void six_to_sym_adj(const double a6[6], double M[3][3]) {
    M[0][0] = a6[0]; M[1][1] = a6[1]; M[2][2] = a6[2];
    M[1][2] = M[2][1] = 0.5 * a6[3];
    M[0][2] = M[2][0] = 0.5 * a6[4];
    M[0][1] = M[1][0] = 0.5 * a6[5];
}

/* Reverse of mu_forward.  In: Sbo (adjoint of the output stress, full
 * symmetric), pcbo (of the output pc).  Out (accumulated): Sbi (of the input
 * stress, full), *pcbi, Lb (of L), *Mb, *etab. */
static void mu_reverse(const ppmo_params* p, const mu_trace* t, double Sbo[3][3], double pcbo,
                       double Sbi[3][3], double* pcbi, double Lb[3][3], double* Mb,
                       double* etab) {
    double Strb[3][3];
    const double dt = t->dt;
    if (!t->plastic) {
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) Strb[r][c] = Sbo[r][c];
        *pcbi += pcbo;
    } else {
        const double q_tr = t->q_tr;
        const double ratio = (q_tr > 0.0) ? t->x[1] / q_tr : 0.0;
        double xb[3], sb[3][3];
        xb[0] = Sbo[0][0] + Sbo[1][1] + Sbo[2][2];
        double ratiob = 0.0;
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) {
                ratiob += Sbo[r][c] * t->s_tr[r][c];
                sb[r][c] = ratio * Sbo[r][c];
            }
        double q_trb = 0.0;
        xb[1] = 0.0;
        if (q_tr > 0.0) {
            xb[1] = ratiob / q_tr;
            q_trb = -ratiob * t->x[1] / (q_tr * q_tr);
        }
        xb[2] = t->floored ? 0.0 : pcbo;
        /* implicit function: J_x^T lambda = xb, ybar = -J_y^T lambda */
        double r[3], J[9], JT[9], lam[3] = {0, 0, 0};
        ppmo_return_residual(p, t->c, t->p_tr, q_tr, t->pc_n, t->x, r, J);
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) JT[a * 3 + b] = J[b * 3 + a];
        if (!solve3(JT, xb, lam)) { lam[0] = lam[1] = lam[2] = 0.0; }
        const double M2 = p->M * p->M, lk = p->lambda_t - p->kappa_t, c = t->c;
        const double pb = t->x[0], q = t->x[1], pc = t->x[2];
        const double f = q * q / M2 + pb * (pb - pc);
        const double fp = 2.0 * pb - pc, fq = 2.0 * q / M2;
        double p_trb = lam[0];
        q_trb += lam[1];
        double pc_nb = lam[2] / t->pc_n;
        double cb = -(lam[0] * p->K * f * fp + lam[1] * 3.0 * p->mu * f * fq + lam[2] * f * fp / lk);
        const double dfdM = -2.0 * q * q / (M2 * p->M), dfqdM = -4.0 * q / (M2 * p->M);
        *Mb -= lam[0] * p->K * c * fp * dfdM + lam[1] * 3.0 * p->mu * c * (dfdM * fq + f * dfqdM) +
               lam[2] * c * fp * dfdM / lk;
        /* c = dt / eta_eff */
        *etab += cb * (-c / p->eta);
        if (p->visc_form == 0) pc_nb += cb * (-2.0 * c / t->pc_n);
        *pcbi += pc_nb;
        /* p_tr = tr(Str)/3, s_tr = Str - p_tr 1, q_tr = sqrt(1.5 s:s) */
        if (q_tr > 0.0)
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) sb[a][b] += q_trb * 1.5 * t->s_tr[a][b] / q_tr;
        double trs = sb[0][0] + sb[1][1] + sb[2][2];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++)
                Strb[a][b] = sb[a][b] + ((a == b) ? (p_trb - trs) / 3.0 : 0.0);
    }
    /* Str = R + K tr(de) 1 + 2 mu dev(de) */
    double trS = Strb[0][0] + Strb[1][1] + Strb[2][2], deb[3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            deb[a][b] = 2.0 * p->mu * (Strb[a][b] - ((a == b) ? trS / 3.0 : 0.0)) +
                        ((a == b) ? p->K * trS : 0.0);
    /* R = Q S Q^T */
    double QT[3][3], tmp[3][3], Sb[3][3], Qb[3][3], RRT[3][3];
    transpose3((double(*)[3])t->Q, QT);
    matmul3(QT, Strb, tmp);
    matmul3(tmp, (double(*)[3])t->Q, Sb);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            Sbi[a][b] += Sb[a][b];
            RRT[a][b] = Strb[a][b] + Strb[b][a];
        }
    matmul3(RRT, (double(*)[3])t->Q, tmp);
    matmul3(tmp, (double(*)[3])t->S, Qb);
    /* Q = Bi Cm, Bi = Bm^-1 */
    double BiT[3][3], CmT[3][3], Cmb[3][3], Bib[3][3], Bmb[3][3];
    transpose3((double(*)[3])t->Bi, BiT);
    transpose3((double(*)[3])t->Cm, CmT);
    matmul3(BiT, Qb, Cmb);
    matmul3(Qb, CmT, Bib);
    matmul3(BiT, Bib, tmp);
    matmul3(tmp, BiT, Bmb);
    double Wb[3][3], Db[3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            Wb[a][b] = 0.5 * dt * (Cmb[a][b] + Bmb[a][b]);   /* adjoint of Bm is -Bmb; Bm = I - dt/2 W */
            Db[a][b] = dt * deb[a][b];
        }
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            Lb[a][b] += 0.5 * (Db[a][b] + Db[b][a]) + 0.5 * (Wb[a][b] - Wb[b][a]);
}

typedef struct {
    int32_t *row_ptr, *col, *rev;
} family_copy;

/* Reverse of one step n -> n+1 from its start state, with the family the
 * forward step used.  ub, vb, ab (3n), sb (6n), pcb (n) hold the adjoint of
 * the state after the step on entry and of the state before it on exit;
 * thb accumulates (M, eta, S_r s). */
static void reverse_step(const ppmo_params* p, int64_t n, const double* u, const double* v,
                         const double* a, const double* sig, const double* pc,
                         const family_copy* F, double* ub, double* vb, double* ab, double* sb,
                         double* pcb, double thb[3]) {
    const double dt = ppmo_time_step(p), h = 0.5 * dt;
    const double V = p->dx * p->dx * p->dx, m = p->rho * V;
    const double Srs = ppmo_saturation(p->suction, p->vg_alpha, p->vg_n) * p->suction;
    const double delta = p->horizon_factor * p->dx, d2max = delta * delta;
    double* x = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* vh = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* fb = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* u1b = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* vhb = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* sbn = (double*)calloc(6 * (size_t)n, sizeof(double));
    double* pcbn = (double*)calloc((size_t)n, sizeof(double));
    ppmo_reference_positions(p, x);
    for (int64_t i = 0; i < n; i++)
        for (int c = 0; c < 3; c++) {
            size_t t = (size_t)c * n + i;
            double w = v[t] + h * a[t];
            double vbar;
            int fixed = constrained(p, i, c, &vbar);
            if (fixed) w = vbar;
            vh[t] = w;
            x[t] += u[t] + dt * w;
            /* v' = vh + h a' ; a' = f/m + g (fixed components: a' = 0) */
            double abt = ab[t] + h * vb[t];
            fb[t] = fixed ? 0.0 : abt / m;
            vhb[t] = vb[t];
            u1b[t] = ub[t];
        }
    for (int64_t i = 0; i < n; i++) {
        const int64_t r0 = F->row_ptr[i], r1 = F->row_ptr[i + 1], nb = r1 - r0;
        double sig_i[6];
        for (int c = 0; c < 6; c++) sig_i[c] = sig[c * n + i];
        /* forward recompute: active bonds and their weights */
        double w = 0.0;
        for (int64_t b = r0; b < r1; b++) {
            subhorizon_sums ss;
            subhorizon(p, n, x, vh, F->row_ptr, F->col, i, F->col[b], &ss);
            double Ki[3][3];
            if (shape_ok(ss.count, ss.K) && inv3(ss.K, Ki)) w += (double)ss.count / (double)nb;
        }
        double Spt[3][3];
        double a6[6];
        for (int c = 0; c < 6; c++) a6[c] = sb[c * n + i];
        six_to_sym_adj(a6, Spt);
        const double pcpt = pcb[i];
        double Sbi[3][3] = {{0}};
        double pcbi = 0.0;
        if (!(w > 0.0)) {
            for (int c = 0; c < 6; c++) sbn[c * n + i] += a6[c];
            pcbn[i] += pcpt;
        }
        for (int64_t b = r0; b < r1; b++) {
            const int64_t j = F->col[b];
            subhorizon_sums ss;
            subhorizon(p, n, x, vh, F->row_ptr, F->col, i, j, &ss);
            double Ki[3][3];
            if (!(shape_ok(ss.count, ss.K) && inv3(ss.K, Ki))) continue;
            const double varpi = (double)ss.count / (double)nb;
            double L[3][3], Lf[9];
            matmul3(ss.A, Ki, L);
            for (int r = 0; r < 3; r++)
                for (int c = 0; c < 3; c++) Lf[r * 3 + c] = L[r][c];
            mu_trace t;
            mu_forward(p, sig_i, pc[i], Lf, dt, &t);
            double Sh[3][3], zj[3], g[3], Tb[3];
            sym_to_mat(t.sig_out, Sh);
            for (int c = 0; c < 3; c++) Sh[c][c] += Srs;
            for (int c = 0; c < 3; c++) {
                zj[c] = rel(p, n, x, i, j, c);
                Tb[c] = V * V * (fb[c * n + i] - fb[c * n + j]);   /* Eq. 49 reversed */
            }
            for (int r = 0; r < 3; r++) {
                g[r] = 0.0;
                for (int c = 0; c < 3; c++) g[r] += Ki[r][c] * zj[c];
            }
            /* T = varpi Sh Ki zj */
            double Sob[3][3], STb[3], Kib[3][3], zjb[3];
            for (int r = 0; r < 3; r++)
                for (int c = 0; c < 3; c++) Sob[r][c] = varpi * 0.5 * (Tb[r] * g[c] + g[r] * Tb[c]);
            thb[2] += Sob[0][0] + Sob[1][1] + Sob[2][2];
            for (int r = 0; r < 3; r++) {
                STb[r] = 0.0;
                for (int c = 0; c < 3; c++) STb[r] += Sh[c][r] * Tb[c];
            }
            for (int r = 0; r < 3; r++)
                for (int c = 0; c < 3; c++) Kib[r][c] = varpi * STb[r] * zj[c];
            for (int r = 0; r < 3; r++) {
                zjb[r] = 0.0;
                for (int c = 0; c < 3; c++) zjb[r] += varpi * Ki[r][c] * STb[c];
            }
            /* point state: sig' = sum varpi sig_b / w */
            for (int r = 0; r < 3; r++)
                for (int c = 0; c < 3; c++) Sob[r][c] += varpi / w * Spt[r][c];
            const double pcbo = varpi / w * pcpt;
            double Lb[3][3] = {{0}};
            mu_reverse(p, &t, Sob, pcbo, Sbi, &pcbi, Lb, &thb[0], &thb[1]);
            /* L = A Ki */
            double KiT[3][3], AT[3][3], Ab[3][3], tmp[3][3], Kb[3][3];
            transpose3(Ki, KiT);
            transpose3(ss.A, AT);
            matmul3(Lb, KiT, Ab);
            matmul3(AT, Lb, tmp);
            for (int r = 0; r < 3; r++)
                for (int c = 0; c < 3; c++) Kib[r][c] += tmp[r][c];
            /* Ki = K^-1 */
            matmul3(KiT, Kib, tmp);
            matmul3(tmp, KiT, Kb);
            for (int r = 0; r < 3; r++)
                for (int c = 0; c < 3; c++) Kb[r][c] = -Kb[r][c];
            /* K = V sum zeta zeta^T, A = V sum Ydot zeta^T over the sub-horizon */
            for (int64_t b2 = r0; b2 < r1; b2++) {
                const int64_t k = F->col[b2];
                if (!((p->model == 1) || (dist2p(p, x, n, j, k) <= d2max))) continue;
                double zk[3], yk[3], zb[3], yb[3];
                for (int c = 0; c < 3; c++) {
                    zk[c] = rel(p, n, x, i, k, c);
                    yk[c] = vh[c * n + k] - vh[c * n + i];
                }
                for (int r = 0; r < 3; r++) {
                    zb[r] = 0.0;
                    yb[r] = 0.0;
                    for (int c = 0; c < 3; c++) {
                        zb[r] += V * (Kb[r][c] + Kb[c][r]) * zk[c] + V * Ab[c][r] * yk[c];
                        yb[r] += V * Ab[r][c] * zk[c];
                    }
                }
                for (int c = 0; c < 3; c++) {
                    u1b[c * n + k] += zb[c];
                    u1b[c * n + i] -= zb[c];
                    vhb[c * n + k] += yb[c];
                    vhb[c * n + i] -= yb[c];
                }
            }
            for (int c = 0; c < 3; c++) {
                u1b[c * n + j] += zjb[c];
                u1b[c * n + i] -= zjb[c];
            }
        }
        double s6[6];
        sym_adj_to6(Sbi, s6);
        for (int c = 0; c < 6; c++) sbn[c * n + i] += s6[c];
        pcbn[i] += pcbi;
    }
    /* predictor: u' = u + dt vh, vh = v + h a (fixed components: 0) */
    for (int64_t i = 0; i < n; i++)
        for (int c = 0; c < 3; c++) {
            size_t t = (size_t)c * n + i;
            double vht = vhb[t] + dt * u1b[t], vbar;
            int fixed = constrained(p, i, c, &vbar);
            ub[t] = u1b[t];
            vb[t] = fixed ? 0.0 : vht;
            ab[t] = fixed ? 0.0 : h * vht;
        }
    memcpy(sb, sbn, sizeof(double) * 6 * (size_t)n);
    memcpy(pcb, pcbn, sizeof(double) * (size_t)n);
    free(x); free(vh); free(fb); free(u1b); free(vhb); free(sbn); free(pcbn);
}

/* Reverse of the initial pass a0 = f0/m + g (every bond carries sigma0). */
static void reverse_initial(const ppmo_params* p, int64_t n, const double* sig0,
                            const family_copy* F, const double* ab, double* sb, double* Srsb) {
    const double V = p->dx * p->dx * p->dx, m = p->rho * V;
    double* x = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* fb = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* zero = (double*)calloc(3 * (size_t)n, sizeof(double));
    ppmo_reference_positions(p, x);
    for (int64_t i = 0; i < n; i++)
        for (int c = 0; c < 3; c++) {
            size_t t = (size_t)c * n + i;
            double vbar;
            int fixed = constrained(p, i, c, &vbar);
            fb[t] = fixed ? 0.0 : ab[t] / m;
        }
    for (int64_t i = 0; i < n; i++) {
        const int64_t r0 = F->row_ptr[i], r1 = F->row_ptr[i + 1], nb = r1 - r0;
        double Sacc[3][3] = {{0}};
        for (int64_t b = r0; b < r1; b++) {
            const int64_t j = F->col[b];
            subhorizon_sums ss;
            subhorizon(p, n, x, zero, F->row_ptr, F->col, i, j, &ss);
            double Ki[3][3];
            if (!(shape_ok(ss.count, ss.K) && inv3(ss.K, Ki))) continue;
            const double varpi = (double)ss.count / (double)nb;
            double zj[3], g[3], Tb[3];
            for (int c = 0; c < 3; c++) {
                zj[c] = rel(p, n, x, i, j, c);
                Tb[c] = V * V * (fb[c * n + i] - fb[c * n + j]);
            }
            for (int r = 0; r < 3; r++) {
                g[r] = 0.0;
                for (int c = 0; c < 3; c++) g[r] += Ki[r][c] * zj[c];
            }
            for (int r = 0; r < 3; r++)
                for (int c = 0; c < 3; c++) Sacc[r][c] += varpi * 0.5 * (Tb[r] * g[c] + g[r] * Tb[c]);
        }
        *Srsb += Sacc[0][0] + Sacc[1][1] + Sacc[2][2];
        double s6[6];
        sym_adj_to6(Sacc, s6);
        for (int c = 0; c < 6; c++) sb[c * n + i] += s6[c];
    }
    free(x); free(fb); free(zero);
}

static double dSrs_ds(const ppmo_params* p) {
    const double s = p->suction, al = p->vg_alpha, nn = p->vg_n, mm = 1.0 - 1.0 / nn;
    if (s <= 0.0) return 1.0;
    const double base = 1.0 + pow(al * s, nn);
    const double Sr = pow(base, -mm);
    const double dSr = -mm * pow(base, -mm - 1.0) * nn * pow(al * s, nn - 1.0) * al;
    return Sr + s * dSr;
}

static int is_top(const ppmo_params* p, int64_t id) {
    return (id / ((int64_t)p->nx * p->ny)) == p->nz - 1;
}

int ppmo_objective_gradient(const ppmo_params* p, const double* v0, int n_steps, int64_t cap,
                            double* J, double grad[4]) {
    if (!params_ok(p) || p->model == 2 || n_steps < 0 || p->contact || p->halt_on_unstable ||
        p->plane_strain || p->coupled)
        return -1;
    const int64_t n = (int64_t)p->nx * p->ny * p->nz;
    ppmo_state s;
    memset(&s, 0, sizeof(s));
    s.n = n;
    s.cap = cap;
    s.u = (double*)calloc(3 * (size_t)n, sizeof(double));
    s.v = (double*)calloc(3 * (size_t)n, sizeof(double));
    s.a = (double*)calloc(3 * (size_t)n, sizeof(double));
    s.sig = (double*)calloc(6 * (size_t)n, sizeof(double));
    s.pc = (double*)calloc((size_t)n, sizeof(double));
    s.eps_s = (double*)calloc((size_t)n, sizeof(double));
    s.fint = (double*)calloc(3 * (size_t)n, sizeof(double));
    s.tforce = (double*)calloc(3 * (size_t)cap, sizeof(double));
    s.row_ptr = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
    s.col = (int32_t*)calloc((size_t)cap, sizeof(int32_t));
    s.rev = (int32_t*)calloc((size_t)cap, sizeof(int32_t));
    s.J = (double*)calloc((size_t)n, sizeof(double));
    /* states before every step and the family each step used */
    const size_t N3 = 3 * (size_t)n, N6 = 6 * (size_t)n;
    double* hist = (double*)malloc(sizeof(double) * (N3 * 3 + N6 + (size_t)n) * ((size_t)n_steps + 1));
    family_copy* fam = (family_copy*)calloc((size_t)n_steps + 1, sizeof(family_copy));
    int rc = ppmo_init(p, v0, &s);
    if (rc != 0) return rc;
    const size_t per = N3 * 3 + N6 + (size_t)n;
    double* sig0 = (double*)malloc(sizeof(double) * N6);
    memcpy(sig0, s.sig, sizeof(double) * N6);
    family_copy fam0;
    fam0.row_ptr = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
    fam0.col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s.nbonds > 0 ? s.nbonds : 1));
    fam0.rev = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s.nbonds > 0 ? s.nbonds : 1));
    memcpy(fam0.row_ptr, s.row_ptr, sizeof(int32_t) * ((size_t)n + 1));
    memcpy(fam0.col, s.col, sizeof(int32_t) * (size_t)s.nbonds);
    memcpy(fam0.rev, s.rev, sizeof(int32_t) * (size_t)s.nbonds);
    for (int st = 0; st < n_steps; st++) {
        double* hp = hist + per * (size_t)st;
        memcpy(hp, s.u, sizeof(double) * N3);
        memcpy(hp + N3, s.v, sizeof(double) * N3);
        memcpy(hp + 2 * N3, s.a, sizeof(double) * N3);
        memcpy(hp + 3 * N3, s.sig, sizeof(double) * N6);
        memcpy(hp + 3 * N3 + N6, s.pc, sizeof(double) * (size_t)n);
        ppmo_step(p, &s, 1);
        fam[st].row_ptr = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
        fam[st].col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s.nbonds > 0 ? s.nbonds : 1));
        fam[st].rev = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s.nbonds > 0 ? s.nbonds : 1));
        memcpy(fam[st].row_ptr, s.row_ptr, sizeof(int32_t) * ((size_t)n + 1));
        memcpy(fam[st].col, s.col, sizeof(int32_t) * (size_t)s.nbonds);
        memcpy(fam[st].rev, s.rev, sizeof(int32_t) * (size_t)s.nbonds);
    }
    /* objective: sum over the top layer of u_x^2 + u_y^2 */
    double* ub = (double*)calloc(N3, sizeof(double));
    double* vb = (double*)calloc(N3, sizeof(double));
    double* ab = (double*)calloc(N3, sizeof(double));
    double* sb = (double*)calloc(N6, sizeof(double));
    double* pcb = (double*)calloc((size_t)n, sizeof(double));
    double Jv = 0.0;
    for (int64_t i = 0; i < n; i++)
        if (is_top(p, i))
            for (int c = 0; c < 2; c++) {
                Jv += s.u[c * n + i] * s.u[c * n + i];
                ub[c * n + i] = 2.0 * s.u[c * n + i];
            }
    double thb[3] = {0.0, 0.0, 0.0};
    for (int st = n_steps - 1; st >= 0; st--) {
        double* hp = hist + per * (size_t)st;
        reverse_step(p, n, hp, hp + N3, hp + 2 * N3, hp + 3 * N3, hp + 3 * N3 + N6, &fam[st], ub,
                     vb, ab, sb, pcb, thb);
    }
    reverse_initial(p, n, sig0, &fam0, ab, sb, &thb[2]);
    /* initial state: sigma0 = geostatic - S_r s 1 (init_stress 0), pc = -pc0 */
    double pc0b = 0.0;
    for (int64_t i = 0; i < n; i++) {
        if (p->init_stress == 0) thb[2] -= sb[0 * n + i] + sb[1 * n + i] + sb[2 * n + i];
        pc0b -= pcb[i];
    }
    *J = Jv;
    grad[0] = thb[0];
    grad[1] = thb[1];
    grad[2] = thb[2] * dSrs_ds(p);
    grad[3] = pc0b;
    for (int st = 0; st < n_steps; st++) { free(fam[st].row_ptr); free(fam[st].col); free(fam[st].rev); }
    free(fam); free(hist); free(sig0);
    free(fam0.row_ptr); free(fam0.col); free(fam0.rev);
    free(ub); free(vb); free(ab); free(sb); free(pcb);
    free(s.u); free(s.v); free(s.a); free(s.sig); free(s.pc); free(s.eps_s); free(s.fint);
    free(s.tforce); free(s.row_ptr); free(s.col); free(s.rev); free(s.J);
    return 0;
}

/* Critical time step of Eq. 65 in the current configuration.  Eq. 65 as
 * printed divides by sum V C |zeta|, which is not a time squared; the
 * estimate it cites divides the micro-modulus by the bond length (reading
 * R30): dt_i = sqrt(2 rho / sum_j V C / |x_j - x_i|) over the family of i,
 * with the bond-based micro-modulus C = 18 K / (pi delta^4) and the mixture
 * density for (1 - phi) rho_s (R5).  Returns the minimum over the points
 * that have bonds (INFINITY if none). */
double ppmo_critical_time_step(const ppmo_params* p, const ppmo_state* s) {
    const int64_t n = s->n;
    double* x = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    if (!x) return NAN;
    current_positions(p, n, s->u, x);
    const double delta = p->horizon_factor * p->dx;
    const double pi = 3.14159265358979323846;
    const double C = 18.0 * p->K / (pi * delta * delta * delta * delta);
    const double V = p->dx * p->dx * p->dx;
    double best = INFINITY;
    for (int64_t i = 0; i < n; i++) {
        double sum = 0.0;
        for (int64_t b = s->row_ptr[i]; b < s->row_ptr[i + 1]; b++) {
            const int64_t j = s->col[b];
            const double d0 = rel(p, n, x, i, j, 0), d1 = rel(p, n, x, i, j, 1),
                         d2 = rel(p, n, x, i, j, 2);
            sum += 1.0 / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        }
        if (sum > 0.0) {
            const double dt = sqrt(2.0 * rho_start(p) / (V * C * sum));
            if (dt < best) best = dt;
        }
    }
    free(x);
    return best;
}

int ppmo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ppmo_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
