// The per-step kernels of the explicit bond loop:
//   k_predictor  -- Newmark predictor, boundary conditions, displacement
//                   (Eq. 60-61, 64; Alg. 2 lines 6-8)
//   k_bond       -- fused per-point kernel: sub-horizon membership and sums
//                   (Eq. 22-25, 55, 57), FP64 shape-tensor inverse, velocity
//                   gradient, rate of deformation and spin (Eq. 26),
//                   Hughes-Winget rotation, linear trial stress (Eq. 41),
//                   critical-state Perzyna return in FP64 (Eq. 40-46,
//                   70-76), force state (Eq. 31-32, 51) and the point-state
//                   reduction; Alg. 1 lines 2-27
//   k_gather     -- deterministic pairwise nodal force (Eq. 49-50), the
//                   acceleration and velocity corrector (Eq. 62-63) and the
//                   energy increments (Eq. 66-68); Alg. 1 lines 29-31
//
// Scaled variables: bond vectors are carried in lattice units
// zeta~ = zeta / dx, the shape tensor as K~ = sum zeta~ zeta~^T (the paper's
// K = V dx^2 K~), and the stored force state as T^ = varpi sigma K~^-1
// zeta~ (the paper's T = T^ / (V dx)), so that FP32 stays far from its
// range limits at every lattice spacing.  Then L = (sum Ydot zeta~^T)
// K~^-1 / dx and the nodal force is f = dx^2 (sum T^ - sum T^').
#include <cuda_runtime.h>
#include <math.h>

#include "ppm_internal.cuh"

namespace ppm {
namespace {

template <typename Real>
struct alignas(4 * sizeof(Real)) R4 {
    Real x, y, z, w;
};

// ---------------------------------------------------------------------------
// predictor (Eq. 60-61, 64 with beta1 = 1/2, beta2 = 0)
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void k_predictor(DevState<Real> s, StepConst k) {
    const size_t n = (size_t)k.npoints;
    const Real dt = (Real)k.dt, hdt = (Real)(0.5 * k.dt);
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < 3 * n;
         t += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / n);
        const size_t i = t - (size_t)c * n;
        Real v = s.v[t] + hdt * s.a[t];
        if (lat_z(s.lat[i]) == 0 || (k.lock_lateral && c < 2)) v = (Real)0;
        s.vh[t] = v;
        if constexpr (sizeof(Real) == 8) {
            s.u[t] = s.u[t] + dt * v;
        } else {
            // compensated (Kahan) accumulation of the displacement
            float y = (float)(dt * v) - s.ulo[t];
            float u0 = (float)s.u[t];
            float u1 = u0 + y;
            s.ulo[t] = (u1 - u0) - y;
            s.u[t] = (Real)u1;
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 pieces: symmetric 3x3 inverse and the visco-plastic return
// ---------------------------------------------------------------------------

// K in order xx yy zz yz xz xy; returns false for a degenerate tensor
// (the same rule as the oracle: det <= 1e-12 (tr K / 3)^3 or det == 0)
__device__ __forceinline__ bool inverse_sym_fp64(const double k[6], double inv[6]) {
    const double k00 = k[0], k11 = k[1], k22 = k[2], k12 = k[3], k02 = k[4], k01 = k[5];
    const double c00 = k11 * k22 - k12 * k12;
    const double c11 = k00 * k22 - k02 * k02;
    const double c22 = k00 * k11 - k01 * k01;
    const double c12 = k01 * k02 - k00 * k12;
    const double c02 = k01 * k12 - k02 * k11;
    const double c01 = k02 * k12 - k01 * k22;
    const double det = k00 * c00 + k01 * c01 + k02 * c02;
    const double t = (k00 + k11 + k22) * (1.0 / 3.0);
    if (!(det > 1e-12 * t * t * t) || det == 0.0) return false;
    const double r = 1.0 / det;
    inv[0] = c00 * r; inv[1] = c11 * r; inv[2] = c22 * r;
    inv[3] = c12 * r; inv[4] = c02 * r; inv[5] = c01 * r;
    return true;
}

// Mixed path: the cancellation-prone steps -- cofactors and determinant --
// in FP64 from the FP32 sums; the degeneracy test, the reciprocal of the
// determinant and the final scaling in FP32 (the result is FP32 either
// way, so a full FP64 division would change it by at most an ulp).
__device__ __forceinline__ bool inverse_sym_mixed(float K00, float K11, float K22, float K12,
                                                  float K02, float K01, float inv[6]) {
    const double k00 = K00, k11 = K11, k22 = K22, k12 = K12, k02 = K02, k01 = K01;
    const double c00 = k11 * k22 - k12 * k12;
    const double c11 = k00 * k22 - k02 * k02;
    const double c22 = k00 * k11 - k01 * k01;
    const double c12 = k01 * k02 - k00 * k12;
    const double c02 = k01 * k12 - k02 * k11;
    const double c01 = k02 * k12 - k01 * k22;
    const float det = (float)(k00 * c00 + k01 * c01 + k02 * c02);
    const float t = (K00 + K11 + K22) * (1.0f / 3.0f);
    if (!(det > 1e-12f * t * t * t) || det == 0.0f) return false;
    const float r = 1.0f / det;
    inv[0] = (float)c00 * r; inv[1] = (float)c11 * r; inv[2] = (float)c22 * r;
    inv[3] = (float)c12 * r; inv[4] = (float)c02 * r; inv[5] = (float)c01 * r;
    return true;
}

struct ReturnConst {
    double K, mu, M2, lk, c, inv_scale;
    double p_tr, q_tr, pc_n;
};

// Eq. 73-75 (Eq. 75 in log form, hardening sign of Eq. 46), stress rows
// divided by the stress scale; J is the exact Jacobian of the scaled rows.
template <bool WANT_J>
__device__ __forceinline__ void return_residual(const ReturnConst& R, const double x[3],
                                                double r[3], double J[9]) {
    const double pb = x[0], q = x[1], pc = x[2];
    const double f = q * q / R.M2 + pb * (pb - pc);
    const double fp = 2.0 * pb - pc;
    const double fq = 2.0 * q / R.M2;
    const double fc = -pb;
    r[0] = (pb - R.p_tr + R.K * R.c * f * fp) * R.inv_scale;
    r[1] = (q - R.q_tr + 3.0 * R.mu * R.c * f * fq) * R.inv_scale;
    const double ratio = pc / R.pc_n;
    r[2] = (ratio > 0.0) ? log(ratio) + R.c * f * fp / R.lk : (double)INFINITY;
    if (WANT_J) {
        const double a = R.K * R.c * R.inv_scale, b = 3.0 * R.mu * R.c * R.inv_scale;
        const double g = R.c / R.lk;
        J[0] = R.inv_scale + a * (fp * fp + 2.0 * f);
        J[1] = a * fq * fp;
        J[2] = a * (fc * fp - f);
        J[3] = b * fp * fq;
        J[4] = R.inv_scale + b * (fq * fq + 2.0 * f / R.M2);
        J[5] = b * fc * fq;
        J[6] = g * (fp * fp + 2.0 * f);
        J[7] = g * (fq * fp);
        J[8] = 1.0 / pc + g * (fc * fp - f);
    }
}

// Newton with backtracking from the trial state; the same stopping rules as
// the oracle (scaled residual max-norm <= tol, or a step below 1e-14 of the
// state; at most max_iter steps; a step is halved up to 20 times until the
// residual is finite and its 2-norm decreases).  3x3 solve by Cramer's rule.
__device__ __noinline__ int return_map(const ReturnConst& R, double tol, int max_iter,
                                       double x[3]) {
    const double scale = 1.0 / R.inv_scale;
    x[0] = R.p_tr; x[1] = R.q_tr; x[2] = R.pc_n;
    double r[3], J[9];
    for (int it = 0;; it++) {
        return_residual<true>(R, x, r, J);
        if (fmax(fabs(r[0]), fmax(fabs(r[1]), fabs(r[2]))) <= tol) return 1;
        if (it >= max_iter) return 0;
        const double m0 = J[4] * J[8] - J[5] * J[7];
        const double m1 = J[3] * J[8] - J[5] * J[6];
        const double m2 = J[3] * J[7] - J[4] * J[6];
        const double det = J[0] * m0 - J[1] * m1 + J[2] * m2;
        if (det == 0.0 || !isfinite(det)) return 0;
        const double id = 1.0 / det;
        double dx[3];
        dx[0] = (r[0] * m0 - J[1] * (r[1] * J[8] - J[5] * r[2]) + J[2] * (r[1] * J[7] - J[4] * r[2])) * id;
        dx[1] = (J[0] * (r[1] * J[8] - J[5] * r[2]) - r[0] * m1 + J[2] * (J[3] * r[2] - r[1] * J[6])) * id;
        dx[2] = (J[0] * (J[4] * r[2] - r[1] * J[7]) - J[1] * (J[3] * r[2] - r[1] * J[6]) + r[0] * m2) * id;
        if (fabs(dx[0]) <= 1e-14 * scale && fabs(dx[1]) <= 1e-14 * scale &&
            fabs(dx[2]) <= 1e-14 * fabs(x[2]))
            return 1;
        const double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        double lam = 1.0, xt[3], rt[3];
        bool accepted = false;
        for (int ls = 0; ls < 20; ls++) {
            for (int q = 0; q < 3; q++) xt[q] = x[q] - lam * dx[q];
            return_residual<false>(R, xt, rt, nullptr);
            if (isfinite(rt[0]) && isfinite(rt[1]) && isfinite(rt[2]) &&
                sqrt(rt[0] * rt[0] + rt[1] * rt[1] + rt[2] * rt[2]) < rn) {
                accepted = true;
                break;
            }
            lam *= 0.5;
        }
        if (!accepted) return 0;
        x[0] = xt[0]; x[1] = xt[1]; x[2] = xt[2];
    }
}

// Mixed path: the same return solved in FP32, in increments from the trial
// state, x = (dp, dq, dpc) with p = p_tr + dp, q = q_tr + dq, pc = pc_n + dpc,
// so that the small corrections keep their precision; Eq. 75 in the form
// log1p(dpc / pc_n) + c f f_p / (lambda - kappa) = 0.  Stopping rules as in
// the FP64 solve with an FP32 tolerance.  Returns 1 if converged.
struct ReturnConstF {
    float K, mu, M2, lk, c, inv_scale, scale;
    float p_tr, q_tr, pc_n, tol;
    int max_iter;
};

template <bool WANT_J>
__device__ __forceinline__ void return_residual_f(const ReturnConstF& R, const float x[3],
                                                  float r[3], float J[9]) {
    const float pb = R.p_tr + x[0], q = R.q_tr + x[1], pc = R.pc_n + x[2];
    const float f = q * q / R.M2 + pb * (pb - pc);
    const float fp = 2.0f * pb - pc;
    const float fq = 2.0f * q / R.M2;
    const float fc = -pb;
    r[0] = (x[0] + R.K * R.c * f * fp) * R.inv_scale;
    r[1] = (x[1] + 3.0f * R.mu * R.c * f * fq) * R.inv_scale;
    const float rel = x[2] / R.pc_n;
    r[2] = (rel > -1.0f) ? log1pf(rel) + R.c * f * fp / R.lk : INFINITY;
    if (WANT_J) {
        const float a = R.K * R.c * R.inv_scale, b = 3.0f * R.mu * R.c * R.inv_scale;
        const float g = R.c / R.lk;
        J[0] = R.inv_scale + a * (fp * fp + 2.0f * f);
        J[1] = a * fq * fp;
        J[2] = a * (fc * fp - f);
        J[3] = b * fp * fq;
        J[4] = R.inv_scale + b * (fq * fq + 2.0f * f / R.M2);
        J[5] = b * fc * fq;
        J[6] = g * (fp * fp + 2.0f * f);
        J[7] = g * (fq * fp);
        J[8] = 1.0f / pc + g * (fc * fp - f);
    }
}

__device__ __noinline__ int return_map_f32(const ReturnConstF& R, float x[3]) {
    x[0] = 0.0f; x[1] = 0.0f; x[2] = 0.0f;
    float r[3], J[9];
    for (int it = 0;; it++) {
        return_residual_f<true>(R, x, r, J);
        if (fmaxf(fabsf(r[0]), fmaxf(fabsf(r[1]), fabsf(r[2]))) <= R.tol) return 1;
        if (it >= R.max_iter) return 0;
        const float m0 = J[4] * J[8] - J[5] * J[7];
        const float m1 = J[3] * J[8] - J[5] * J[6];
        const float m2 = J[3] * J[7] - J[4] * J[6];
        const float det = J[0] * m0 - J[1] * m1 + J[2] * m2;
        if (det == 0.0f || !isfinite(det)) return 0;
        const float id = 1.0f / det;
        float dx[3];
        dx[0] = (r[0] * m0 - J[1] * (r[1] * J[8] - J[5] * r[2]) + J[2] * (r[1] * J[7] - J[4] * r[2])) * id;
        dx[1] = (J[0] * (r[1] * J[8] - J[5] * r[2]) - r[0] * m1 + J[2] * (J[3] * r[2] - r[1] * J[6])) * id;
        dx[2] = (J[0] * (J[4] * r[2] - r[1] * J[7]) - J[1] * (J[3] * r[2] - r[1] * J[6]) + r[0] * m2) * id;
        const float small = 2e-7f * R.scale;
        if (fabsf(dx[0]) <= small && fabsf(dx[1]) <= small && fabsf(dx[2]) <= small) return 1;
        const float rn = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        float lam = 1.0f, xt[3], rt[3];
        bool accepted = false;
        for (int ls = 0; ls < 20; ls++) {
            for (int q = 0; q < 3; q++) xt[q] = x[q] - lam * dx[q];
            return_residual_f<false>(R, xt, rt, nullptr);
            if (isfinite(rt[0]) && isfinite(rt[1]) && isfinite(rt[2]) &&
                sqrtf(rt[0] * rt[0] + rt[1] * rt[1] + rt[2] * rt[2]) < rn) {
                accepted = true;
                break;
            }
            lam *= 0.5f;
        }
        if (!accepted) return 0;
        x[0] = xt[0]; x[1] = xt[1]; x[2] = xt[2];
    }
}

// ---------------------------------------------------------------------------
// constitutive update of one bond (Sec. 2.3; Sec. 3.2.1)
// ---------------------------------------------------------------------------
template <typename Real>
struct BondStress {
    Real sig[6];
    Real pc, des;
    int plastic, nonconv, ret64;
};

template <typename Real>
__device__ __forceinline__ void material_update(const Real L[9], const Real sn[6], Real pc_n,
                                                const StepConst& k, double M, float Mf,
                                                BondStress<Real>& o) {
    constexpr bool F64 = sizeof(Real) == 8;
    const Real dt = F64 ? (Real)k.dt : (Real)k.dtf;
    const Real Kb = F64 ? (Real)k.K : (Real)k.Kf;
    const Real mu = F64 ? (Real)k.mu : (Real)k.muf;
    // rate of deformation and spin (Eq. 26)
    const Real D00 = L[0], D11 = L[4], D22 = L[8];
    const Real D12 = (Real)0.5 * (L[5] + L[7]);
    const Real D02 = (Real)0.5 * (L[2] + L[6]);
    const Real D01 = (Real)0.5 * (L[1] + L[3]);
    // Hughes-Winget: Q = (I - A)^-1 (I + A) with A = dt/2 W, in closed
    // (Cayley) form Q = I + 2/(1 + a.a) (A + a a^T - (a.a) I), a = axial(A)
    const Real h = (Real)0.5 * dt;
    const Real a1 = h * (Real)0.5 * (L[7] - L[5]);
    const Real a2 = h * (Real)0.5 * (L[2] - L[6]);
    const Real a3 = h * (Real)0.5 * (L[3] - L[1]);
    const Real aa = a1 * a1 + a2 * a2 + a3 * a3;
    const Real kap = (Real)2 / ((Real)1 + aa);
    Real Q[9];
    Q[0] = (Real)1 + kap * (a1 * a1 - aa); Q[1] = kap * (-a3 + a1 * a2); Q[2] = kap * (a2 + a1 * a3);
    Q[3] = kap * (a3 + a2 * a1); Q[4] = (Real)1 + kap * (a2 * a2 - aa); Q[5] = kap * (-a1 + a2 * a3);
    Q[6] = kap * (-a2 + a3 * a1); Q[7] = kap * (a1 + a3 * a2); Q[8] = (Real)1 + kap * (a3 * a3 - aa);
    const Real S[9] = {sn[0], sn[5], sn[4], sn[5], sn[1], sn[3], sn[4], sn[3], sn[2]};
    Real P[9];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++)
            P[r * 3 + c] = Q[r * 3 + 0] * S[0 * 3 + c] + Q[r * 3 + 1] * S[1 * 3 + c] + Q[r * 3 + 2] * S[2 * 3 + c];
    auto rot = [&](int r, int c) {
        return P[r * 3 + 0] * Q[c * 3 + 0] + P[r * 3 + 1] * Q[c * 3 + 1] + P[r * 3 + 2] * Q[c * 3 + 2];
    };
    // strain increment (Eq. 59) and linear trial stress (Eq. 41)
    const Real e00 = dt * D00, e11 = dt * D11, e22 = dt * D22;
    const Real e12 = dt * D12, e02 = dt * D02, e01 = dt * D01;
    const Real tr = e00 + e11 + e22, tr3 = tr * (Real)(1.0 / 3.0);
    const Real lam = Kb * tr;
    Real st[6];
    st[0] = rot(0, 0) + lam + (Real)2 * mu * (e00 - tr3);
    st[1] = rot(1, 1) + lam + (Real)2 * mu * (e11 - tr3);
    st[2] = rot(2, 2) + lam + (Real)2 * mu * (e22 - tr3);
    st[3] = (Real)0.5 * (rot(1, 2) + rot(2, 1)) + (Real)2 * mu * e12;
    st[4] = (Real)0.5 * (rot(0, 2) + rot(2, 0)) + (Real)2 * mu * e02;
    st[5] = (Real)0.5 * (rot(0, 1) + rot(1, 0)) + (Real)2 * mu * e01;
    const Real d0 = e00 - tr3, d1 = e11 - tr3, d2 = e22 - tr3;
    o.des = sqrt((Real)(2.0 / 3.0) *
                 (d0 * d0 + d1 * d1 + d2 * d2 + (Real)2 * (e12 * e12 + e02 * e02 + e01 * e01)));
    // invariants and yield function (Eq. 40)
    const Real p_tr = (st[0] + st[1] + st[2]) * (Real)(1.0 / 3.0);
    const Real s0 = st[0] - p_tr, s1 = st[1] - p_tr, s2 = st[2] - p_tr;
    const Real q_tr = sqrt((Real)1.5 * (s0 * s0 + s1 * s1 + s2 * s2 +
                                        (Real)2 * (st[3] * st[3] + st[4] * st[4] + st[5] * st[5])));
    const Real Mr = F64 ? (Real)M : (Real)Mf;
    const Real f_tr = q_tr * q_tr / (Mr * Mr) + p_tr * (p_tr - pc_n);
    o.plastic = 0;
    o.nonconv = 0;
    o.ret64 = 0;
    if (!(f_tr > (Real)0)) {
#pragma unroll
        for (int c = 0; c < 6; c++) o.sig[c] = st[c];
        o.pc = pc_n;
        return;
    }
    o.plastic = 1;
    o.ret64 = 0;
    Real p_new = p_tr, q_new = q_tr, pc_new = pc_n;
    bool need64 = F64;
    if constexpr (!F64) {
        // FP32 return unless the state is near the critical-state apex
        // (mean stress within 5% of the preconsolidation pressure from
        // zero, or tensile) or the preconsolidation pressure has nearly
        // vanished; any FP32 solve that fails is redone in FP64
        need64 = (p_tr > 0.05f * pc_n) || (pc_n > -100.0f);
        if (!need64) {
            ReturnConstF R;
            R.K = k.Kf; R.mu = k.muf; R.M2 = Mf * Mf; R.lk = (float)k.lk;
            R.p_tr = p_tr; R.q_tr = q_tr; R.pc_n = pc_n;
            const float eta_eff = (k.visc_form == 0) ? k.etaf * pc_n * pc_n : k.etaf;
            R.c = k.dtf / eta_eff;
            float scale = fmaxf(fmaxf(fabsf(pc_n), fabsf(p_tr)), fmaxf(q_tr, 1.0f));
            R.scale = scale;
            R.inv_scale = 1.0f / scale;
            R.tol = fmaxf((float)k.tol, 2e-6f);
            R.max_iter = k.max_iter;
            float x[3];
            if (return_map_f32(R, x)) {
                p_new = p_tr + x[0];
                q_new = q_tr + x[1];
                pc_new = pc_n + x[2];
                o.nonconv = 0;
            } else {
                need64 = true;
            }
        }
    }
    if (need64) {
        // visco-plastic return in FP64
        ReturnConst R;
        R.K = k.K; R.mu = k.mu; R.M2 = M * M; R.lk = k.lk;
        R.p_tr = (double)p_tr; R.q_tr = (double)q_tr; R.pc_n = (double)pc_n;
        const double eta_eff = (k.visc_form == 0) ? k.eta * R.pc_n * R.pc_n : k.eta;
        R.c = k.dt / eta_eff;
        double scale = fabs(R.pc_n);
        if (fabs(R.p_tr) > scale) scale = fabs(R.p_tr);
        if (R.q_tr > scale) scale = R.q_tr;
        if (scale < 1.0) scale = 1.0;
        R.inv_scale = 1.0 / scale;
        double x[3];
        const int ok = return_map(R, k.tol, k.max_iter, x);
        o.nonconv = !ok;
        o.ret64 = 1;
        p_new = (Real)x[0];
        q_new = (Real)x[1];
        pc_new = (Real)(x[2] > -1.0 ? -1.0 : x[2]);
    }
    const Real ratio = (q_tr > (Real)0) ? q_new / q_tr : (Real)0;
    const Real pn = p_new;
    o.sig[0] = pn + ratio * s0;
    o.sig[1] = pn + ratio * s1;
    o.sig[2] = pn + ratio * s2;
    o.sig[3] = ratio * st[3];
    o.sig[4] = ratio * st[4];
    o.sig[5] = ratio * st[5];
    if (pc_new > (Real)-1) pc_new = (Real)-1;   // floor at the apex
    o.pc = pc_new;
}

// Predicated sub-horizon accumulation: when tst <= 0 (member), add the
// outer products zeta~ zeta~^T (6), Ydot zeta~^T (9) and 1 to the count; the
// predicate guards each FMA, so non-members cost no extra multiplies and the
// warp never branches.
__device__ __forceinline__ void masked_accumulate(float tst, float zx, float zy, float zz,
                                                  float yx, float yy, float yz, float (&K)[6],
                                                  float (&A)[9], float& cnt) {
    asm("{\n\t.reg .pred p;\n\t"
        "setp.le.f32 p, %16, 0f00000000;\n\t"
        "@p fma.rn.f32 %0, %17, %17, %0;\n\t"
        "@p fma.rn.f32 %1, %18, %18, %1;\n\t"
        "@p fma.rn.f32 %2, %19, %19, %2;\n\t"
        "@p fma.rn.f32 %3, %18, %19, %3;\n\t"
        "@p fma.rn.f32 %4, %17, %19, %4;\n\t"
        "@p fma.rn.f32 %5, %17, %18, %5;\n\t"
        "@p fma.rn.f32 %6, %20, %17, %6;\n\t"
        "@p fma.rn.f32 %7, %20, %18, %7;\n\t"
        "@p fma.rn.f32 %8, %20, %19, %8;\n\t"
        "@p fma.rn.f32 %9, %21, %17, %9;\n\t"
        "@p fma.rn.f32 %10, %21, %18, %10;\n\t"
        "@p fma.rn.f32 %11, %21, %19, %11;\n\t"
        "@p fma.rn.f32 %12, %22, %17, %12;\n\t"
        "@p fma.rn.f32 %13, %22, %18, %13;\n\t"
        "@p fma.rn.f32 %14, %22, %19, %14;\n\t"
        "@p add.f32 %15, %15, 0f3F800000;\n\t"
        "}"
        : "+f"(K[0]), "+f"(K[1]), "+f"(K[2]), "+f"(K[3]), "+f"(K[4]), "+f"(K[5]),
          "+f"(A[0]), "+f"(A[1]), "+f"(A[2]), "+f"(A[3]), "+f"(A[4]), "+f"(A[5]),
          "+f"(A[6]), "+f"(A[7]), "+f"(A[8]), "+f"(cnt)
        : "f"(tst), "f"(zx), "f"(zy), "f"(zz), "f"(yx), "f"(yy), "f"(yz));
}

// Predicated sum of a sender's 3x3 matrix (M) into N when tst <= 0.
__device__ __forceinline__ void masked_add9(float tst, const float4& m0, const float4& m1,
                                            float m8, float (&N)[9]) {
    asm("{\n\t.reg .pred p;\n\t"
        "setp.le.f32 p, %9, 0f00000000;\n\t"
        "@p add.f32 %0, %0, %10;\n\t"
        "@p add.f32 %1, %1, %11;\n\t"
        "@p add.f32 %2, %2, %12;\n\t"
        "@p add.f32 %3, %3, %13;\n\t"
        "@p add.f32 %4, %4, %14;\n\t"
        "@p add.f32 %5, %5, %15;\n\t"
        "@p add.f32 %6, %6, %16;\n\t"
        "@p add.f32 %7, %7, %17;\n\t"
        "@p add.f32 %8, %8, %18;\n\t"
        "}"
        : "+f"(N[0]), "+f"(N[1]), "+f"(N[2]), "+f"(N[3]), "+f"(N[4]), "+f"(N[5]), "+f"(N[6]),
          "+f"(N[7]), "+f"(N[8])
        : "f"(tst), "f"(m0.x), "f"(m0.y), "f"(m0.z), "f"(m0.w), "f"(m1.x), "f"(m1.y), "f"(m1.z),
          "f"(m1.w), "f"(m8));
}

// deterministic block sum: butterfly within warps, then warps in order
template <int NV, typename T>
__device__ __forceinline__ void block_sum(T (&v)[NV], T (*sm)[NV]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < NV; e++)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[e] += __shfl_xor_sync(0xffffffffu, v[e], off);
    if (lane == 0)
#pragma unroll
        for (int e = 0; e < NV; e++) sm[w][e] = v[e];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < NV; e++) {
        T t = sm[0][e];
        for (int q = 1; q < (int)(blockDim.x >> 5); q++) t += sm[q][e];
        v[e] = t;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// fused bond kernel: one CTA per point, one thread per bond
// ---------------------------------------------------------------------------
// TPP threads per point (a tile the autotuner picks among 64, 128, 256); the
// register budget targets 640 resident threads per SM for FP32
template <typename Real, int MODEL, int TPP>
__global__ void __launch_bounds__(TPP, sizeof(Real) == 4 ? (640 / TPP) : (256 / TPP > 0 ? 256 / TPP : 1))
k_bond(DevState<Real> s, StepConst k, int with_dt, int update) {
    constexpr bool F64 = sizeof(Real) == 8;
    constexpr int NW = TPP / 32;
    __shared__ R4<Real> s_z[kMaxRow];                         // zeta~_k, lattice units
    __shared__ R4<Real> s_y[kMaxRow];                         // Ydot_k, m/s
    __shared__ double s_p[F64 ? 3 : 1][F64 ? kMaxRow : 1];    // FP64: absolute x_k
    // model 2: per sender bond, its matrix M = varpi sigma K^-1 (9), and (FP32) the
    // terms of its membership test, -2 zeta~ (3) and |zeta~|^2 - hf^2 (1)
    __shared__ alignas(16) Real s_M[MODEL == 2 ? kMaxRow : 1][F64 ? 9 : 16];
    __shared__ Real s_red[NW][12];
    __shared__ unsigned s_cnt[NW][5];

    const int i = blockIdx.x;
    const size_t n = (size_t)k.npoints;
    const int r0 = s.row_ptr[i];
    int nb = s.row_ptr[i + 1] - r0;
    if (nb > kMaxRow) nb = 0;
    const int li = s.lat[i];
    const int ix = lat_x(li), iy = lat_y(li), iz = lat_z(li);
    const Real inv_dx = F64 ? (Real)k.inv_dx : (Real)k.inv_dxf;

    // stage the family of i: bond vectors and relative velocities
    double pxi = 0, pyi = 0, pzi = 0;
    if constexpr (F64) {
        pxi = __dadd_rn(__dmul_rn((double)ix, k.dx), (double)s.u[i]);
        pyi = __dadd_rn(__dmul_rn((double)iy, k.dx), (double)s.u[n + i]);
        pzi = __dadd_rn(__dmul_rn((double)iz, k.dx), (double)s.u[2 * n + i]);
    }
    const Real uxi = s.u[i], uyi = s.u[n + i], uzi = s.u[2 * n + i];
    const Real vxi = s.vh[i], vyi = s.vh[n + i], vzi = s.vh[2 * n + i];
    for (int t = threadIdx.x; t < nb; t += TPP) {
        const int j = s.col[r0 + t];
        const int lj = s.lat[j];
        R4<Real> z, y;
        if constexpr (F64) {
            const double px = __dadd_rn(__dmul_rn((double)lat_x(lj), k.dx), (double)s.u[j]);
            const double py = __dadd_rn(__dmul_rn((double)lat_y(lj), k.dx), (double)s.u[n + j]);
            const double pz = __dadd_rn(__dmul_rn((double)lat_z(lj), k.dx), (double)s.u[2 * n + j]);
            s_p[0][t] = px; s_p[F64 ? 1 : 0][t] = py; s_p[F64 ? 2 : 0][t] = pz;
            z.x = (Real)((px - pxi) * k.inv_dx);
            z.y = (Real)((py - pyi) * k.inv_dx);
            z.z = (Real)((pz - pzi) * k.inv_dx);
        } else {
            z.x = (Real)(lat_x(lj) - ix) + (s.u[j] - uxi) * inv_dx;
            z.y = (Real)(lat_y(lj) - iy) + (s.u[n + j] - uyi) * inv_dx;
            z.z = (Real)(lat_z(lj) - iz) + (s.u[2 * n + j] - uzi) * inv_dx;
        }
        z.w = z.x * z.x + z.y * z.y + z.z * z.z;
        y.x = s.vh[j] - vxi;
        y.y = s.vh[n + j] - vyi;
        y.z = s.vh[2 * n + j] - vzi;
        y.w = (Real)0;
        s_z[t] = z;
        s_y[t] = y;
    }
    __syncthreads();

    Real sig_i[6];
#pragma unroll
    for (int c = 0; c < 6; c++) sig_i[c] = s.sig[c * n + i];
    const Real pc_i = s.pc[i];
    const ColumnConst cc = s.cols[s.colid[i]];
    const Real Srs = F64 ? (Real)cc.Srs : (Real)cc.Srsf;
    const Real hf2 = (Real)k.hf2f;
    const Real inv_nb = nb > 0 ? (Real)1 / (Real)nb : (Real)0;

    // per-thread partial sums over its bonds (fixed order)
    Real red[12];
#pragma unroll
    for (int e = 0; e < 12; e++) red[e] = (Real)0;
    unsigned n_plastic = 0, n_nonconv = 0, n_singular = 0, n_pairs = 0, n_ret64 = 0;

    for (int t = threadIdx.x; t < nb; t += TPP) {
        const R4<Real> zj = s_z[t];
        // mixed-path test |z_k - z_j|^2 - hf^2 = |z_k|^2 + (|z_j|^2 - hf^2) - 2 z_k.z_j
        const Real mjx = (Real)-2 * zj.x, mjy = (Real)-2 * zj.y, mjz = (Real)-2 * zj.z;
        const Real cj = zj.w - hf2;
        double pjx = 0, pjy = 0, pjz = 0;
        if constexpr (F64) { pjx = s_p[0][t]; pjy = s_p[F64 ? 1 : 0][t]; pjz = s_p[F64 ? 2 : 0][t]; }
        Real K00 = 0, K11 = 0, K22 = 0, K12 = 0, K02 = 0, K01 = 0;
        Real A00 = 0, A01 = 0, A02 = 0, A10 = 0, A11 = 0, A12 = 0, A20 = 0, A21 = 0, A22 = 0;
        int cnt = 0;
        // sub-horizon of bond (i, j): k in H_i with |x_k - x_j| <= delta
        // (Alg. 1 line 4); the standard model takes all of H_i
        if constexpr (F64 || MODEL == 1) {
#pragma unroll 2
            for (int q = 0; q < nb; q++) {
                const R4<Real> zk = s_z[q];
                bool member = true;
                if constexpr (MODEL != 1) {
                    const double d0 = __dsub_rn(s_p[0][q], pjx);
                    const double d1 = __dsub_rn(s_p[F64 ? 1 : 0][q], pjy);
                    const double d2 = __dsub_rn(s_p[F64 ? 2 : 0][q], pjz);
                    member = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)),
                                       __dmul_rn(d2, d2)) <= k.delta2;
                }
                if (member) {
                    const R4<Real> yk = s_y[q];
                    K00 += zk.x * zk.x; K11 += zk.y * zk.y; K22 += zk.z * zk.z;
                    K12 += zk.y * zk.z; K02 += zk.x * zk.z; K01 += zk.x * zk.y;
                    A00 += yk.x * zk.x; A01 += yk.x * zk.y; A02 += yk.x * zk.z;
                    A10 += yk.y * zk.x; A11 += yk.y * zk.y; A12 += yk.y * zk.z;
                    A20 += yk.z * zk.x; A21 += yk.z * zk.y; A22 += yk.z * zk.z;
                    cnt++;
                }
            }
        } else {
            // FP32 sub-horizon sums, predicated (no branches, no mask multiplies)
            float Kf[6] = {0, 0, 0, 0, 0, 0}, Af[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            float cntf = 0.0f;
#pragma unroll 4
            for (int q = 0; q < nb; q++) {
                const R4<Real> zk = s_z[q];
                const R4<Real> yk = s_y[q];
                const float tst = zk.x * mjx + (zk.y * mjy + (zk.z * mjz + (zk.w + cj)));
                masked_accumulate(tst, zk.x, zk.y, zk.z, yk.x, yk.y, yk.z, Kf, Af, cntf);
            }
            K00 = Kf[0]; K11 = Kf[1]; K22 = Kf[2]; K12 = Kf[3]; K02 = Kf[4]; K01 = Kf[5];
            A00 = Af[0]; A01 = Af[1]; A02 = Af[2]; A10 = Af[3]; A11 = Af[4]; A12 = Af[5];
            A20 = Af[6]; A21 = Af[7]; A22 = Af[8];
            cnt = (int)cntf;
        }
        n_pairs += cnt;
        // shape-tensor inverse with FP64 cofactors and determinant (Eq. 23, 25)
        Real Kid[6];
        bool active = cnt >= 3;
        if constexpr (F64) {
            const double Kd[6] = {K00, K11, K22, K12, K02, K01};
            active = active && inverse_sym_fp64(Kd, Kid);
        } else {
            active = active && inverse_sym_mixed(K00, K11, K22, K12, K02, K01, Kid);
        }
        if (!active) {
            n_singular++;
            if constexpr (MODEL != 2) {
                s.T[r0 + t] = (Real)0;
                s.T[k.cap + r0 + t] = (Real)0;
                s.T[2 * k.cap + r0 + t] = (Real)0;
                const int rb = s.rev[r0 + t];
                if (rb >= 0) {
                    s.Trev[rb] = (Real)0;
                    s.Trev[k.cap + rb] = (Real)0;
                    s.Trev[2 * k.cap + rb] = (Real)0;
                }
            } else {
#pragma unroll
                for (int e = 0; e < 9; e++) s_M[t][e] = (Real)0;
                if constexpr (!F64) {
                    s_M[t][9] = mjx; s_M[t][10] = mjy; s_M[t][11] = mjz; s_M[t][12] = cj;
                }
            }
            continue;
        }
        const Real Ki[9] = {(Real)Kid[0], (Real)Kid[5], (Real)Kid[4],
                            (Real)Kid[5], (Real)Kid[1], (Real)Kid[3],
                            (Real)Kid[4], (Real)Kid[3], (Real)Kid[2]};
        const Real varpi = (Real)cnt * inv_nb;              // Eq. 55
        BondStress<Real> bs;
        if (with_dt) {
            // velocity gradient L = A~ K~^-1 / dx (Eq. 25, 57)
            const Real A[9] = {A00, A01, A02, A10, A11, A12, A20, A21, A22};
            Real L[9];
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int c = 0; c < 3; c++)
                    L[r * 3 + c] = (A[r * 3 + 0] * Ki[0 * 3 + c] + A[r * 3 + 1] * Ki[1 * 3 + c] +
                                    A[r * 3 + 2] * Ki[2 * 3 + c]) * inv_dx;
            material_update<Real>(L, sig_i, pc_i, k, cc.M, cc.Mf, bs);
            n_plastic += bs.plastic;
            n_nonconv += bs.nonconv;
            n_ret64 += bs.ret64;
        } else {
#pragma unroll
            for (int c = 0; c < 6; c++) bs.sig[c] = sig_i[c];
            bs.pc = pc_i;
            bs.des = (Real)0;
        }
        // total stress sigma_bar - S_r p_w 1 = sigma_bar + S_r s 1 (Eq. 32)
        const Real S[9] = {bs.sig[0] + Srs, bs.sig[5], bs.sig[4],
                           bs.sig[5], bs.sig[1] + Srs, bs.sig[3],
                           bs.sig[4], bs.sig[3], bs.sig[2] + Srs};
        Real SK[9];
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int c = 0; c < 3; c++)
                SK[r * 3 + c] = varpi * (S[r * 3 + 0] * Ki[0 * 3 + c] + S[r * 3 + 1] * Ki[1 * 3 + c] +
                                         S[r * 3 + 2] * Ki[2 * 3 + c]);
        if constexpr (MODEL != 2) {
            // force state on the bond itself (Eq. 31-32, 51)
            const Real T0 = SK[0] * zj.x + SK[1] * zj.y + SK[2] * zj.z;
            const Real T1 = SK[3] * zj.x + SK[4] * zj.y + SK[5] * zj.z;
            const Real T2 = SK[6] * zj.x + SK[7] * zj.y + SK[8] * zj.z;
            s.T[r0 + t] = T0;
            s.T[k.cap + r0 + t] = T1;
            s.T[2 * k.cap + r0 + t] = T2;
            const int rb = s.rev[r0 + t];
            if (rb >= 0) {
                s.Trev[rb] = T0;
                s.Trev[k.cap + rb] = T1;
                s.Trev[2 * k.cap + rb] = T2;
            }
            red[9] += T0; red[10] += T1; red[11] += T2;
        } else {
#pragma unroll
            for (int e = 0; e < 9; e++) s_M[t][e] = SK[e];
            if constexpr (!F64) {
                s_M[t][9] = mjx; s_M[t][10] = mjy; s_M[t][11] = mjz; s_M[t][12] = cj;
            }
        }
        red[0] += varpi;
#pragma unroll
        for (int c = 0; c < 6; c++) red[1 + c] += varpi * bs.sig[c];
        red[7] += varpi * bs.pc;
        red[8] += varpi * bs.des;
    }
    block_sum<12, Real>(red, s_red);
    const Real w = red[0];

    if constexpr (MODEL == 2) {
        // power-conjugate form: every sub-horizon's force acts on each of its
        // members; the row is normalised by sum(varpi)
        Real ts[3] = {(Real)0, (Real)0, (Real)0};
        const Real inv_w = w > (Real)0 ? (Real)1 / w : (Real)0;
        for (int t = threadIdx.x; t < nb; t += TPP) {
            const R4<Real> zt = s_z[t];
            double ptx = 0, pty = 0, ptz = 0;
            if constexpr (F64) { ptx = s_p[0][t]; pty = s_p[F64 ? 1 : 0][t]; ptz = s_p[F64 ? 2 : 0][t]; }
            Real N[9];
#pragma unroll
            for (int e = 0; e < 9; e++) N[e] = (Real)0;
            if constexpr (F64) {
                for (int q = 0; q < nb; q++) {
                    const double d0 = __dsub_rn(s_p[0][q], ptx);
                    const double d1 = __dsub_rn(s_p[F64 ? 1 : 0][q], pty);
                    const double d2 = __dsub_rn(s_p[F64 ? 2 : 0][q], ptz);
                    const bool member = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)),
                                                  __dmul_rn(d2, d2)) <= k.delta2;
                    if (member)
#pragma unroll
                        for (int e = 0; e < 9; e++) N[e] += s_M[q][e];
                }
            } else {
                // receiver t is a member of sender q's sub-horizon: the same
                // expression (and rounding) as the sender's own test
                float Nf[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll 2
                for (int q = 0; q < nb; q++) {
                    const float4 m0 = *reinterpret_cast<const float4*>(&s_M[q][0]);
                    const float4 m1 = *reinterpret_cast<const float4*>(&s_M[q][4]);
                    const float4 m2 = *reinterpret_cast<const float4*>(&s_M[q][8]);
                    const float4 m3 = *reinterpret_cast<const float4*>(&s_M[q][12]);
                    const float tst = zt.x * m2.y + (zt.y * m2.z + (zt.z * m2.w + (zt.w + m3.x)));
                    masked_add9(tst, m0, m1, m2.x, Nf);
                }
#pragma unroll
                for (int e = 0; e < 9; e++) N[e] = Nf[e];
            }
            const Real T0 = (N[0] * zt.x + N[1] * zt.y + N[2] * zt.z) * inv_w;
            const Real T1 = (N[3] * zt.x + N[4] * zt.y + N[5] * zt.z) * inv_w;
            const Real T2 = (N[6] * zt.x + N[7] * zt.y + N[8] * zt.z) * inv_w;
            s.T[r0 + t] = T0;
            s.T[k.cap + r0 + t] = T1;
            s.T[2 * k.cap + r0 + t] = T2;
            const int rb = s.rev[r0 + t];
            if (rb >= 0) {
                s.Trev[rb] = T0;
                s.Trev[k.cap + rb] = T1;
                s.Trev[2 * k.cap + rb] = T2;
            }
            ts[0] += T0; ts[1] += T1; ts[2] += T2;
        }
        block_sum<3, Real>(ts, reinterpret_cast<Real(*)[3]>(&s_red[0][0]));
        red[9] = ts[0]; red[10] = ts[1]; red[11] = ts[2];
    }

    unsigned cnts[5] = {n_plastic, n_nonconv, n_singular, n_pairs, n_ret64};
    block_sum<5, unsigned>(cnts, s_cnt);
    if (threadIdx.x == 0) {
        if (update && w > (Real)0) {
            const Real iw = (Real)1 / w;
#pragma unroll
            for (int c = 0; c < 6; c++) s.sig[c * n + i] = red[1 + c] * iw;
            s.pc[i] = red[7] * iw;
            s.eps[i] = s.eps[i] + red[8] * iw;
        }
        s.tsum[i] = red[9];
        s.tsum[n + i] = red[10];
        s.tsum[2 * n + i] = red[11];
        if (with_dt && cnts[3]) atomicAdd(&s.ctr->pairs, (unsigned long long)cnts[3]);
        if (cnts[0]) atomicAdd(&s.ctr->plastic, (unsigned long long)cnts[0]);
        if (cnts[4]) atomicAdd(&s.ctr->ret64, (unsigned long long)cnts[4]);
        if (cnts[1]) {
            atomicAdd(&s.ctr->nonconv, (unsigned long long)cnts[1]);
            atomicOr(&s.ctr->status, PPM_STATUS_NONCONV);
        }
        if (with_dt && cnts[2]) {
            atomicAdd(&s.ctr->singular, (unsigned long long)cnts[2]);
            atomicOr(&s.ctr->status, PPM_STATUS_SINGULAR);
        }
    }
}

// ---------------------------------------------------------------------------
// gather: f_i = dx^2 (sum_own T^ - sum T^[rev]); acceleration, corrector
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

template <typename Real>
__global__ void __launch_bounds__(kWarpPointsPerBlock * 32)
k_gather(DevState<Real> s, StepConst k, double dt, int initial) {
    constexpr bool F64 = sizeof(Real) == 8;
    constexpr int kIt = kMaxRow / 32;
    __shared__ Real s_e[kWarpPointsPerBlock][3];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int i = blockIdx.x * kWarpPointsPerBlock + wib;       // one warp per point
    const size_t n = (size_t)k.npoints;
    const Real m = F64 ? (Real)(k.rho * k.dx * k.dx * k.dx) : (Real)k.massf;
    const Real dx2 = F64 ? (Real)(k.dx * k.dx) : (Real)k.dx2f;
    const Real inv_rho_dx = F64 ? (Real)(1.0 / (k.rho * k.dx)) : (Real)k.inv_rho_dxf;
    const Real dtr = F64 ? (Real)dt : (Real)(float)dt;
    const Real hdt = (Real)0.5 * dtr;
    Real dwi = 0, dwe = 0, wk = 0;
    if (i < k.npoints) {
        const int r0 = s.row_ptr[i], r1 = s.row_ptr[i + 1];
        // lanes 0..2 fetch the per-point data of component c = lane early
        const int c = lane < 3 ? lane : 0;
        const size_t t = (size_t)c * n + i;
        const Real ts = s.tsum[t], fo = s.fint[t], vh = s.vh[t], v0 = s.v[t];
        const bool base = lat_z(s.lat[i]) == 0;
        // every load of the row T_(ji) (stored contiguously in Trev) first
        Real x[3][kIt];
#pragma unroll
        for (int it = 0; it < kIt; it++) {
            const int b = r0 + lane + 32 * it;
#pragma unroll
            for (int q = 0; q < 3; q++) x[q][it] = b < r1 ? s.Trev[(size_t)q * k.cap + b] : (Real)0;
        }
        Real sum[3], cmp[3];
#pragma unroll
        for (int q = 0; q < 3; q++) {
            sum[q] = (Real)0;
            cmp[q] = (Real)0;
#pragma unroll
            for (int it = 0; it < kIt; it++) {
                if constexpr (F64) {
                    sum[q] += x[q][it];
                } else {
                    float ss, ee;          // compensated running sum
                    two_sum(sum[q], x[q][it], ss, ee);
                    sum[q] = ss;
                    cmp[q] += ee;
                }
            }
        }
        // fixed-order butterfly over lanes (every lane ends with the total)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
            for (int q = 0; q < 3; q++) {
                const Real so = __shfl_xor_sync(0xffffffffu, sum[q], off);
                const Real co = __shfl_xor_sync(0xffffffffu, cmp[q], off);
                if constexpr (F64) {
                    sum[q] += so;
                } else {
                    float ss, ee;
                    two_sum(sum[q], so, ss, ee);
                    sum[q] = ss;
                    cmp[q] = cmp[q] + co + ee;
                }
            }
        }
        if (lane < 3) {
            const Real g = F64 ? (Real)k.g[c] : (Real)k.gf[c];
            const Real gathered = c == 0 ? sum[0] + cmp[0] : (c == 1 ? sum[1] + cmp[1] : sum[2] + cmp[2]);
            const Real fhat = ts - gathered;
            const Real f = fhat * dx2;                               // Eq. 49-50
            Real a = fhat * inv_rho_dx + g;                          // Eq. 62
            if (base || (k.lock_lateral && c < 2)) a = (Real)0;
            if (!isfinite(a)) atomicOr(&s.ctr->status, PPM_STATUS_NONFINITE);
            s.fint[t] = f;
            s.a[t] = a;
            if (initial) {
                wk = (Real)0.5 * m * v0 * v0;
            } else {
                const Real v = vh + hdt * a;                         // Eq. 63
                s.v[t] = v;
                dwi = -hdt * vh * (fo + f);                          // Eq. 66
                dwe = dtr * m * vh * g;                              // Eq. 67
                wk = (Real)0.5 * m * v * v;                          // Eq. 68
            }
        }
    }
    // energies of the point: lanes 0..2 hold the three components
    dwi += __shfl_down_sync(0xffffffffu, dwi, 1) + __shfl_down_sync(0xffffffffu, dwi, 2);
    dwe += __shfl_down_sync(0xffffffffu, dwe, 1) + __shfl_down_sync(0xffffffffu, dwe, 2);
    wk += __shfl_down_sync(0xffffffffu, wk, 1) + __shfl_down_sync(0xffffffffu, wk, 2);
    if (lane == 0) {
        s_e[wib][0] = dwi;
        s_e[wib][1] = dwe;
        s_e[wib][2] = wk;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double tot = 0.0;
        for (int q = 0; q < kWarpPointsPerBlock; q++) tot += (double)s_e[q][threadIdx.x];
        s.epart[(size_t)blockIdx.x * 3 + threadIdx.x] = tot;
    }
}

__global__ void k_energy_reduce(const double* epart, int nblocks, DevCounters* ctr, int initial,
                                const int32_t* row_ptr, int npoints) {
    __shared__ double sm[3][256];
    double t[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int e = 0; e < 3; e++) t[e] += epart[(size_t)b * 3 + e];
    for (int e = 0; e < 3; e++) sm[e][threadIdx.x] = t[e];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int e = 0; e < 3; e++) sm[e][threadIdx.x] += sm[e][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (initial) {
            ctr->W_int = 0.0;
            ctr->W_ext = 0.0;
            ctr->W_kin = sm[2][0];
            ctr->W_kin0 = sm[2][0];
        } else {
            ctr->bond_steps += (unsigned long long)row_ptr[npoints];
            ctr->W_int += sm[0][0];
            ctr->W_ext += sm[1][0];
            ctr->W_kin = sm[2][0];
            const double bal = fabs(ctr->W_int + ctr->W_kin - ctr->W_ext - ctr->W_kin0);
            const double mx = fmax(fmax(ctr->W_kin, fabs(ctr->W_int)), fmax(fabs(ctr->W_ext), ctr->W_kin0));
            if (bal > 1e-2 * mx) atomicOr(&ctr->status, PPM_STATUS_UNSTABLE);   // Eq. 69
        }
    }
}

// ---------------------------------------------------------------------------
// initial state (Alg. 2 line 1) and velocity boundary conditions
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void k_init_state(DevState<Real> s, StepConst k, int init_stress, double pc0) {
    const size_t n = (size_t)k.npoints;
    const double nu = (3.0 * k.K - 2.0 * k.mu) / (2.0 * (3.0 * k.K + k.mu));
    const double K0 = nu / (1.0 - nu);
    const double gmag = -k.g[2];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const ColumnConst cc = s.cols[s.colid[i]];
        const int iz = lat_z(s.lat[i]);
        for (int c = 0; c < 3; c++) {
            const size_t t = (size_t)c * n + i;
            s.u[t] = (Real)0; s.v[t] = (Real)0; s.vh[t] = (Real)0; s.a[t] = (Real)0;
            s.fint[t] = (Real)0; s.tsum[t] = (Real)0;
            if (s.ulo) s.ulo[t] = 0.0f;
        }
        double sg[6] = {0, 0, 0, 0, 0, 0};
        if (init_stress == 0) {
            // geostatic with a traction-free top: total sigma_zz = -rho g d,
            // sigma_xx = sigma_yy = K0 sigma_zz; effective = total - S_r s 1
            const double d = (double)(cc.nz - 1 - iz) * k.dx;
            const double szz = -k.rho * gmag * d;
            sg[0] = K0 * szz - cc.Srs;
            sg[1] = K0 * szz - cc.Srs;
            sg[2] = szz - cc.Srs;
        }
        for (int c = 0; c < 6; c++) s.sig[(size_t)c * n + i] = (Real)sg[c];
        s.pc[i] = (Real)(-pc0);
        s.eps[i] = (Real)0;
    }
}

template <typename Real>
__global__ void k_velocity_bc(DevState<Real> s, StepConst k) {
    const size_t n = (size_t)k.npoints;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < 3 * n;
         t += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / n);
        const size_t i = t - (size_t)c * n;
        if (lat_z(s.lat[i]) == 0 || (k.lock_lateral && c < 2)) s.v[t] = (Real)0;
    }
}

inline int blocks_for(size_t work, int tpb) {
    size_t b = (work + tpb - 1) / tpb;
    return (int)(b < 65536 ? (b > 0 ? b : 1) : 65536);
}

}  // namespace

template <typename Real>
cudaError_t launch_init_state(const DevState<Real>& s, const StepConst& k, int init_stress,
                              double pc0, cudaStream_t st) {
    k_init_state<Real><<<blocks_for(k.npoints, 256), 256, 0, st>>>(s, k, init_stress, pc0);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_apply_velocity_bc(const DevState<Real>& s, const StepConst& k, cudaStream_t st) {
    k_velocity_bc<Real><<<blocks_for(3 * (size_t)k.npoints, 256), 256, 0, st>>>(s, k);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_predictor(const DevState<Real>& s, const StepConst& k, cudaStream_t st) {
    k_predictor<Real><<<blocks_for(3 * (size_t)k.npoints, 256), 256, 0, st>>>(s, k);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_bond(const DevState<Real>& s, const StepConst& k, double dt, int update,
                        cudaStream_t st) {
    if (k.npoints <= 0) return cudaSuccess;
    const int with_dt = dt != 0.0;
    const int tpp = (k.tile == 64 || k.tile == 256) ? k.tile : 128;
#define PPM_BOND(M, T) k_bond<Real, M, T><<<k.npoints, T, 0, st>>>(s, k, with_dt, update)
#define PPM_BOND_TILES(M)                           \
    if (tpp == 64) PPM_BOND(M, 64);                 \
    else if (tpp == 256) PPM_BOND(M, 256);          \
    else PPM_BOND(M, 128);
    switch (k.model) {
        case 0: PPM_BOND_TILES(0); break;
        case 1: PPM_BOND_TILES(1); break;
        default: PPM_BOND_TILES(2); break;
    }
#undef PPM_BOND_TILES
#undef PPM_BOND
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_gather(const DevState<Real>& s, const StepConst& k, double dt, int initial,
                          int gather_blocks, cudaStream_t st) {
    k_gather<Real><<<gather_blocks, kWarpPointsPerBlock * 32, 0, st>>>(s, k, dt, initial);
    return cudaGetLastError();
}

cudaError_t launch_energy_reduce(double* epart, int nblocks, DevCounters* ctr, int initial,
                                 const int32_t* row_ptr, int npoints, cudaStream_t st) {
    k_energy_reduce<<<1, 256, 0, st>>>(epart, nblocks, ctr, initial, row_ptr, npoints);
    return cudaGetLastError();
}

#define PPM_INSTANTIATE(R)                                                                         \
    template cudaError_t launch_init_state<R>(const DevState<R>&, const StepConst&, int, double,   \
                                              cudaStream_t);                                       \
    template cudaError_t launch_apply_velocity_bc<R>(const DevState<R>&, const StepConst&,         \
                                                     cudaStream_t);                                \
    template cudaError_t launch_predictor<R>(const DevState<R>&, const StepConst&, cudaStream_t);  \
    template cudaError_t launch_bond<R>(const DevState<R>&, const StepConst&, double, int,         \
                                        cudaStream_t);                                             \
    template cudaError_t launch_gather<R>(const DevState<R>&, const StepConst&, double, int, int,  \
                                          cudaStream_t);
PPM_INSTANTIATE(double)
PPM_INSTANTIATE(float)
#undef PPM_INSTANTIATE

}  // namespace ppm
