// Device routines shared by the forward bond kernel (bond.cu) and its
// reverse (adjoint.cu): shape-tensor inverses, the visco-plastic return in
// FP64 and FP32, the constitutive update of one bond, predicated
// sub-horizon accumulation and deterministic block sums.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>

#include "ppm_internal.cuh"

namespace ppm {
namespace {

template <typename Real>
struct alignas(4 * sizeof(Real)) R4 {
    Real x, y, z, w;
};

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

// Mixed path: the determinant -- the step where cancellation decides the
// degeneracy test and the scale of every entry -- in FP64 from the FP32
// sums (its three first-row cofactors too); the six cofactors of the
// inverse's entries in FP32, each a 2 x 2 minor a b - c d by Kahan's FMA
// algorithm (minor2_f32: relative error at most 2u, so each entry is within
// a few ulp of the one full FP64 cofactors give); the degeneracy test, the
// reciprocal of the determinant and the final scaling in FP32 (the result is
// FP32 either way, so a full FP64 division would change it by at most an
// ulp).
//
// On GB300 the hardware conversions between binary32 and binary64 issue on
// the FP64 pipe at the FP64 rate (about 1/64 of FP32), so the tensor is first
// brought to a range where both conversions are short integer re-encodings:
// it is multiplied by the power of two that puts its largest |entry| in
// [1, 2), and entries below 2^-40 of that are taken as zero (far below the
// rounding of the FP32 sums they come from).  Every entry is then zero or a
// normal binary32 number of at least 2^-40, exact in binary64; the product
// of two entries is exact in binary64 with an ulp of at least 2^-126, so
// every nonzero cofactor lies in [2^-126, 8], the normal binary32 range, and
// a determinant below that range fails the degeneracy test (whose bound is
// at least 1e-12 / 27 on the scaled tensor).  The re-encodings give the
// hardware's bits (binary32 -> binary64 exact, binary64 -> binary32 round to
// nearest even) and every scaling is by a power of two without overflow, so
// the inverse is the one the unscaled steps give.  Tensors whose largest
// |entry| lies outside [2^-30, 2^31) (or is not finite) take the unscaled
// steps with the hardware conversions, out of line.

// binary32 -> binary64 for |f| >= 2^-40 (a normal number: the exponent is
// re-biased by 1023 - 127 = 896 and the 23-bit fraction moves to the top of
// the 52-bit one), and a zero of the same sign for smaller |f|
__device__ __forceinline__ double f32_to_f64_flushed(float f) {
    const unsigned u = __float_as_uint(f);
    const bool keep = (u & 0x7fffffffu) >= 0x2B800000u;          // |f| >= 2^-40
    const unsigned hi = (u & 0x80000000u) | (keep ? ((u & 0x7fffffffu) >> 3) + 0x38000000u : 0u);
    return __hiloint2double((int)hi, keep ? (int)(u << 29) : 0);
}

// binary64 -> binary32, round to nearest even, for zero and for |d| in the
// normal binary32 range: a funnel shift keeps the top 23 fraction bits below
// the exponent's low 9 bits, adding 2^30 re-biases that exponent (896 = 1024
// - 128, modulo 2^9), the 29 dropped bits decide the rounding (above half:
// up; exactly half: up when the kept lsb is odd), and a carry out of the
// fraction moves into the exponent, as the rounding rule requires
__device__ __forceinline__ float f64_to_f32_regular(double d) {
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    unsigned f = __funnelshift_l(lo, hi, 3) + 0x40000000u;
    const unsigned rem = lo & 0x1fffffffu;
    f += (rem + (f & 1u)) > 0x10000000u ? 1u : 0u;
    f = (hi & 0x7fffffffu) ? f : 0u;
    return __uint_as_float(f | (hi & 0x80000000u));
}

// a b - c d of binary32 numbers by Kahan's algorithm: w = RN(c d), its
// rounding error w - c d recovered exactly by an FMA, and RN(a b - w) plus
// that error; relative error at most 2u (Jeannerod, Louvet and Muller, Math.
// Comp. 82, 2013), barring underflow of the error term
__device__ __forceinline__ float minor2_f32(float a, float b, float c, float d) {
    const float w = __fmul_rn(c, d);
    const float e = __fmaf_rn(-c, d, w);
    const float f = __fmaf_rn(a, b, -w);
    return __fadd_rn(f, e);
}

// the unscaled steps with the hardware conversions (tensors outside the
// range of the re-encodings: zero, non-finite, tiny or huge entries)
__device__ __noinline__ bool inverse_sym_mixed_slow(float K00, float K11, float K22, float K12,
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
    const float r = __frcp_rn(det);                     // = 1 / det, correctly rounded
    inv[0] = (float)c00 * r; inv[1] = (float)c11 * r; inv[2] = (float)c22 * r;
    inv[3] = (float)c12 * r; inv[4] = (float)c02 * r; inv[5] = (float)c01 * r;
    return true;
}

__device__ __forceinline__ bool inverse_sym_mixed(float K00, float K11, float K22, float K12,
                                                  float K02, float K01, float inv[6]) {
    // the largest |entry| by its bit pattern (NaN and infinity order above
    // every finite value); the scaled path needs it in [2^-30, 2^31)
    const unsigned m = max(max(max(__float_as_uint(K00) & 0x7fffffffu, __float_as_uint(K11) & 0x7fffffffu),
                               max(__float_as_uint(K22) & 0x7fffffffu, __float_as_uint(K12) & 0x7fffffffu)),
                           max(__float_as_uint(K02) & 0x7fffffffu, __float_as_uint(K01) & 0x7fffffffu));
    if (m - 0x30800000u >= 0x1E800000u) return inverse_sym_mixed_slow(K00, K11, K22, K12, K02, K01, inv);
    // 2^(127 - e) for 2^e <= max |entry| < 2^(e+1): the scaled maximum is in [1, 2)
    const float sc = __uint_as_float((254u - (m >> 23)) << 23);
    const float s00 = K00 * sc, s11 = K11 * sc, s22 = K22 * sc;
    const float s12 = K12 * sc, s02 = K02 * sc, s01 = K01 * sc;
    const double k00 = f32_to_f64_flushed(s00), k11 = f32_to_f64_flushed(s11);
    const double k22 = f32_to_f64_flushed(s22), k12 = f32_to_f64_flushed(s12);
    const double k02 = f32_to_f64_flushed(s02), k01 = f32_to_f64_flushed(s01);
    const double c00 = k11 * k22 - k12 * k12;
    const double c02 = k01 * k12 - k02 * k11;
    const double c01 = k02 * k12 - k01 * k22;
    const double det64 = k00 * c00 + k01 * c01 + k02 * c02;
    // below the normal binary32 range, zero or negative: degenerate
    if ((int)__double2hiint(det64) <= 0x38100000) return false;
    const float det = f64_to_f32_regular(det64);
    const float t = (s00 + s11 + s22) * (1.0f / 3.0f);
    if (!(det > 1e-12f * t * t * t)) return false;
    const float r = __frcp_rn(det) * sc;                // sc / det of the scaled tensor = 1 / det
    inv[0] = minor2_f32(s11, s22, s12, s12) * r;        // c00
    inv[1] = minor2_f32(s00, s22, s02, s02) * r;        // c11
    inv[2] = minor2_f32(s00, s11, s01, s01) * r;        // c22
    inv[3] = minor2_f32(s01, s02, s00, s12) * r;        // c12
    inv[4] = minor2_f32(s01, s12, s02, s11) * r;        // c02
    inv[5] = minor2_f32(s02, s12, s01, s22) * r;        // c01
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

// Mixed path, near the apex: iterative refinement of the FP32 root in FP64.
// Each step evaluates the residual of Eq. 73-75 in FP64 (as above, with the
// divisions by M^2, pc_n and lambda - kappa taken as products with
// reciprocals) and corrects x by the FP32 Jacobian's solve, which the FP32
// Newton formed at its root; the iteration contracts by about the FP32
// rounding of that Jacobian per step, so a start within the FP32 tolerance
// reaches the FP64 tolerance in one or two steps.  A step is accepted only
// if the residual is finite and its 2-norm decreases; returns 0 (the caller
// then solves from the trial state in FP64) otherwise, or after max_iter.
__device__ __forceinline__ void refine_residual(const ReturnConst& R, double inv_M2, double inv_pcn,
                                                double g, const double x[3], double r[3]) {
    const double pb = x[0], q = x[1], pc = x[2];
    const double f = q * q * inv_M2 + pb * (pb - pc);
    const double fp = 2.0 * pb - pc;
    r[0] = (pb - R.p_tr + R.K * R.c * f * fp) * R.inv_scale;
    r[1] = (q - R.q_tr + 6.0 * R.mu * R.c * f * q * inv_M2) * R.inv_scale;
    const double ratio = pc * inv_pcn;
    r[2] = (ratio > 0.0) ? log(ratio) + g * f * fp : (double)INFINITY;
}

__device__ __noinline__ int return_refine64(const ReturnConst& R, double tol, int max_iter,
                                            double x[3], const float Jf[9]) {
    // inverse of the FP32 Jacobian by its adjugate
    const float m0 = Jf[4] * Jf[8] - Jf[5] * Jf[7];
    const float m1 = Jf[5] * Jf[6] - Jf[3] * Jf[8];
    const float m2 = Jf[3] * Jf[7] - Jf[4] * Jf[6];
    const float det = Jf[0] * m0 + Jf[1] * m1 + Jf[2] * m2;
    if (det == 0.0f || !isfinite(det)) return 0;
    const float id = __frcp_rn(det);
    const float Ji[9] = {m0 * id, (Jf[2] * Jf[7] - Jf[1] * Jf[8]) * id, (Jf[1] * Jf[5] - Jf[2] * Jf[4]) * id,
                         m1 * id, (Jf[0] * Jf[8] - Jf[2] * Jf[6]) * id, (Jf[2] * Jf[3] - Jf[0] * Jf[5]) * id,
                         m2 * id, (Jf[1] * Jf[6] - Jf[0] * Jf[7]) * id, (Jf[0] * Jf[4] - Jf[1] * Jf[3]) * id};
    const double inv_M2 = 1.0 / R.M2, inv_pcn = 1.0 / R.pc_n, g = R.c / R.lk;
    double r[3];
    refine_residual(R, inv_M2, inv_pcn, g, x, r);
    if (!(isfinite(r[0]) && isfinite(r[1]) && isfinite(r[2]))) return 0;
    for (int it = 0; it < max_iter; it++) {
        if (fmax(fabs(r[0]), fmax(fabs(r[1]), fabs(r[2]))) <= tol) return 1;
        const float rf[3] = {(float)r[0], (float)r[1], (float)r[2]};
        double xt[3], rt[3];
#pragma unroll
        for (int q = 0; q < 3; q++)
            xt[q] = x[q] - (double)(Ji[q * 3 + 0] * rf[0] + Ji[q * 3 + 1] * rf[1] + Ji[q * 3 + 2] * rf[2]);
        refine_residual(R, inv_M2, inv_pcn, g, xt, rt);
        if (!(isfinite(rt[0]) && isfinite(rt[1]) && isfinite(rt[2])) ||
            !(rt[0] * rt[0] + rt[1] * rt[1] + rt[2] * rt[2] < r[0] * r[0] + r[1] * r[1] + r[2] * r[2]))
            return 0;
        x[0] = xt[0]; x[1] = xt[1]; x[2] = xt[2];
        r[0] = rt[0]; r[1] = rt[1]; r[2] = rt[2];
    }
    return fmax(fabs(r[0]), fmax(fabs(r[1]), fabs(r[2]))) <= tol;
}

// Mixed path: the same return solved in FP32, in increments from the trial
// state, x = (dp, dq, dpc) with p = p_tr + dp, q = q_tr + dq, pc = pc_n + dpc,
// so that the small corrections keep their precision; Eq. 75 in the form
// log1p(dpc / pc_n) + c f f_p / (lambda - kappa) = 0, divisions by constants
// taken as products with their reciprocals.  Stopping rules as in
// the FP64 solve with an FP32 tolerance.  Returns 1 if converged.
struct ReturnConstF {
    float K, mu, M2, lk, c, inv_scale, scale;
    float p_tr, q_tr, pc_n, tol;
    float inv_M2, inv_pcn, g;   // 1 / M^2, 1 / pc_n, c / (lambda - kappa)
    int max_iter;
};

template <bool WANT_J>
__device__ __forceinline__ void return_residual_f(const ReturnConstF& R, const float x[3],
                                                  float r[3], float J[9]) {
    const float pb = R.p_tr + x[0], q = R.q_tr + x[1], pc = R.pc_n + x[2];
    const float f = q * q * R.inv_M2 + pb * (pb - pc);
    const float fp = 2.0f * pb - pc;
    const float fq = 2.0f * q * R.inv_M2;
    const float fc = -pb;
    r[0] = (x[0] + R.K * R.c * f * fp) * R.inv_scale;
    r[1] = (x[1] + 3.0f * R.mu * R.c * f * fq) * R.inv_scale;
    const float rel = x[2] * R.inv_pcn;
    r[2] = (rel > -1.0f) ? log1pf(rel) + R.g * f * fp : INFINITY;
    if (WANT_J) {
        const float a = R.K * R.c * R.inv_scale, b = 3.0f * R.mu * R.c * R.inv_scale;
        const float g = R.g;
        J[0] = R.inv_scale + a * (fp * fp + 2.0f * f);
        J[1] = a * fq * fp;
        J[2] = a * (fc * fp - f);
        J[3] = b * fp * fq;
        J[4] = R.inv_scale + b * (fq * fq + 2.0f * f * R.inv_M2);
        J[5] = b * fc * fq;
        J[6] = g * (fp * fp + 2.0f * f);
        J[7] = g * (fq * fp);
        J[8] = 1.0f / pc + g * (fc * fp - f);
    }
}

__device__ __noinline__ int return_map_f32(const ReturnConstF& R, float x[3], float Jo[9]) {
    x[0] = 0.0f; x[1] = 0.0f; x[2] = 0.0f;
    float r[3], J[9];
    for (int it = 0;; it++) {
        return_residual_f<true>(R, x, r, J);
        if (fmaxf(fabsf(r[0]), fmaxf(fabsf(r[1]), fabsf(r[2]))) <= R.tol) {
            for (int e = 0; e < 9; e++) Jo[e] = J[e];
            return 1;
        }
        if (it >= R.max_iter) return 0;
        const float m0 = J[4] * J[8] - J[5] * J[7];
        const float m1 = J[3] * J[8] - J[5] * J[6];
        const float m2 = J[3] * J[7] - J[4] * J[6];
        const float det = J[0] * m0 - J[1] * m1 + J[2] * m2;
        if (det == 0.0f || !isfinite(det)) return 0;
        const float id = __frcp_rn(det);
        float dx[3];
        dx[0] = (r[0] * m0 - J[1] * (r[1] * J[8] - J[5] * r[2]) + J[2] * (r[1] * J[7] - J[4] * r[2])) * id;
        dx[1] = (J[0] * (r[1] * J[8] - J[5] * r[2]) - r[0] * m1 + J[2] * (J[3] * r[2] - r[1] * J[6])) * id;
        dx[2] = (J[0] * (J[4] * r[2] - r[1] * J[7]) - J[1] * (J[3] * r[2] - r[1] * J[6]) + r[0] * m2) * id;
        const float small = 2e-7f * R.scale;
        if (fabsf(dx[0]) <= small && fabsf(dx[1]) <= small && fabsf(dx[2]) <= small) {
            for (int e = 0; e < 9; e++) Jo[e] = J[e];
            return 1;
        }
        // backtracking on the squared 2-norm of the residual
        const float rn2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        float lam = 1.0f, xt[3], rt[3];
        bool accepted = false;
        for (int ls = 0; ls < 20; ls++) {
            for (int q = 0; q < 3; q++) xt[q] = x[q] - lam * dx[q];
            return_residual_f<false>(R, xt, rt, nullptr);
            if (isfinite(rt[0]) && isfinite(rt[1]) && isfinite(rt[2]) &&
                rt[0] * rt[0] + rt[1] * rt[1] + rt[2] * rt[2] < rn2) {
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

// what the reverse of one update needs from its forward
template <typename Real>
struct MatTrace {
    Real Q[9];          // rotation
    Real a[3], kap;     // axial vector of dt/2 W and 2 / (1 + a.a)
    Real st[6];         // trial stress
    Real p_tr, q_tr;
    int plastic, floored;
    double x[3];        // return solution (p, q, pc) before the floor
    double c;           // dt / eta_eff
};

// Elastic part of the update of one bond: rate of deformation and spin
// (Eq. 26), Hughes-Winget rotation of the stress, linear trial stress
// (Eq. 41), its invariants and the yield test (Eq. 40).  Returns true when
// the trial state lies outside the yield surface (plastic).
template <typename Real>
__device__ __forceinline__ bool material_trial(const Real L[9], const Real sn[6], Real pc_n,
                                               const StepConst& k, double M, float Mf,
                                               Real st[6], Real& des,
                                               MatTrace<Real>* trace = nullptr) {
    constexpr bool F64 = sizeof(Real) == 8;
    const Real dt = F64 ? (Real)k.dt : (Real)k.dtf;
    const Real Kb = F64 ? (Real)k.K : (Real)k.Kf;
    const Real mu = F64 ? (Real)k.mu : (Real)k.muf;
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
    // 2 / (1 + a.a); twice the correctly rounded reciprocal is the same number
    Real kap;
    if constexpr (F64) kap = (Real)2 / ((Real)1 + aa);
    else kap = 2.0f * __frcp_rn(1.0f + aa);
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
    st[0] = rot(0, 0) + lam + (Real)2 * mu * (e00 - tr3);
    st[1] = rot(1, 1) + lam + (Real)2 * mu * (e11 - tr3);
    st[2] = rot(2, 2) + lam + (Real)2 * mu * (e22 - tr3);
    st[3] = (Real)0.5 * (rot(1, 2) + rot(2, 1)) + (Real)2 * mu * e12;
    st[4] = (Real)0.5 * (rot(0, 2) + rot(2, 0)) + (Real)2 * mu * e02;
    st[5] = (Real)0.5 * (rot(0, 1) + rot(1, 0)) + (Real)2 * mu * e01;
    const Real d0 = e00 - tr3, d1 = e11 - tr3, d2 = e22 - tr3;
    des = sqrt((Real)(2.0 / 3.0) *
               (d0 * d0 + d1 * d1 + d2 * d2 + (Real)2 * (e12 * e12 + e02 * e02 + e01 * e01)));
    // invariants and yield function (Eq. 40)
    const Real p_tr = (st[0] + st[1] + st[2]) * (Real)(1.0 / 3.0);
    const Real s0 = st[0] - p_tr, s1 = st[1] - p_tr, s2 = st[2] - p_tr;
    const Real q_tr = sqrt((Real)1.5 * (s0 * s0 + s1 * s1 + s2 * s2 +
                                        (Real)2 * (st[3] * st[3] + st[4] * st[4] + st[5] * st[5])));
    const Real Mr = F64 ? (Real)M : (Real)Mf;
    const Real f_tr = q_tr * q_tr / (Mr * Mr) + p_tr * (p_tr - pc_n);
    if (trace) {
#pragma unroll
        for (int e = 0; e < 9; e++) trace->Q[e] = Q[e];
        trace->a[0] = a1; trace->a[1] = a2; trace->a[2] = a3; trace->kap = kap;
#pragma unroll
        for (int e = 0; e < 6; e++) trace->st[e] = st[e];
        trace->p_tr = p_tr; trace->q_tr = q_tr;
        trace->plastic = 0; trace->floored = 0;
    }
    return f_tr > (Real)0 && !k.elastic;
}

// Plastic part: the visco-plastic return from the trial stress st (Eq. 42-46,
// 70-76) and the radial scaling of its deviator; o.des is left to the caller.
// Kept out of line: it runs for a minority of bonds, and as a call its
// register needs do not constrain the bond pass around it.
template <typename Real>
__device__ __noinline__ void material_return(const Real st[6], Real pc_n, const StepConst& k,
                                                double M, float Mf, BondStress<Real>& o,
                                                MatTrace<Real>* trace = nullptr) {
    constexpr bool F64 = sizeof(Real) == 8;
    const Real p_tr = (st[0] + st[1] + st[2]) * (Real)(1.0 / 3.0);
    const Real s0 = st[0] - p_tr, s1 = st[1] - p_tr, s2 = st[2] - p_tr;
    const Real q_tr = sqrt((Real)1.5 * (s0 * s0 + s1 * s1 + s2 * s2 +
                                        (Real)2 * (st[3] * st[3] + st[4] * st[4] + st[5] * st[5])));
    o.plastic = 1;
    o.nonconv = 0;
    o.ret64 = 0;
    Real p_new = p_tr, q_new = q_tr, pc_new = pc_n;
    bool need64 = F64;
    bool warm = false;
    double x64[3] = {0.0, 0.0, 0.0};
    float Jf64[9];   // the FP32 Jacobian at the FP32 root, for the refinement
    if constexpr (!F64) {
        // FP32 return first.  Near the critical-state apex (mean stress within
        // 5% of the preconsolidation pressure from zero, or tensile) or where
        // the preconsolidation pressure has nearly vanished, the FP32 root
        // only starts the FP64 Newton solve, which then takes one or two
        // steps to the FP64 tolerance (mixed-precision refinement); an FP32
        // solve that fails is redone in FP64 from the trial state
        const bool near_apex = (p_tr > 0.05f * pc_n) || (pc_n > -100.0f);
        {
            ReturnConstF R;
            R.K = k.Kf; R.mu = k.muf; R.M2 = Mf * Mf; R.lk = (float)k.lk;
            R.p_tr = p_tr; R.q_tr = q_tr; R.pc_n = pc_n;
            const float eta_eff = (k.visc_form == 0) ? k.etaf * pc_n * pc_n : k.etaf;
            R.c = k.dtf / eta_eff;
            R.inv_M2 = 1.0f / R.M2;
            R.inv_pcn = 1.0f / pc_n;
            R.g = R.c / R.lk;
            float scale = fmaxf(fmaxf(fabsf(pc_n), fabsf(p_tr)), fmaxf(q_tr, 1.0f));
            R.scale = scale;
            R.inv_scale = 1.0f / scale;
            R.tol = fmaxf((float)k.tol, 2e-6f);
            R.max_iter = k.max_iter;
            float x[3], Jf[9];
            if (return_map_f32(R, x, Jf)) {
                p_new = p_tr + x[0];
                q_new = q_tr + x[1];
                pc_new = pc_n + x[2];
                o.nonconv = 0;
                if (near_apex) {
                    need64 = warm = true;
#pragma unroll
                    for (int e = 0; e < 9; e++) Jf64[e] = Jf[e];
                    x64[0] = (double)p_tr + (double)x[0];
                    x64[1] = (double)q_tr + (double)x[1];
                    x64[2] = (double)pc_n + (double)x[2];
                }
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
        double x[3] = {x64[0], x64[1], x64[2]};
        int ok = warm ? return_refine64(R, k.tol, k.max_iter, x, Jf64) : 0;
        if (!ok) ok = return_map(R, k.tol, k.max_iter, x);
        o.nonconv = !ok;
        o.ret64 = 1;
        p_new = (Real)x[0];
        q_new = (Real)x[1];
        pc_new = (Real)x[2];
    }
    const Real ratio = (q_tr > (Real)0) ? q_new / q_tr : (Real)0;
    const Real pn = p_new;
    o.sig[0] = pn + ratio * s0;
    o.sig[1] = pn + ratio * s1;
    o.sig[2] = pn + ratio * s2;
    o.sig[3] = ratio * st[3];
    o.sig[4] = ratio * st[4];
    o.sig[5] = ratio * st[5];
    if (trace) {
        trace->plastic = 1;
        trace->x[0] = (double)p_new; trace->x[1] = (double)q_new; trace->x[2] = (double)pc_new;
        trace->floored = pc_new > (Real)-1;
        const double pcn = (double)pc_n;
        trace->c = k.dt / ((k.visc_form == 0) ? k.eta * pcn * pcn : k.eta);
    }
    if (pc_new > (Real)-1) pc_new = (Real)-1;   // floor at the apex
    o.pc = pc_new;
}


// The whole update of one bond (elastic trial, then the return if plastic).
template <typename Real>
__device__ __forceinline__ void material_update(const Real L[9], const Real sn[6], Real pc_n,
                                                const StepConst& k, double M, float Mf,
                                                BondStress<Real>& o,
                                                MatTrace<Real>* trace = nullptr) {
    Real st[6], des;
    const bool plastic = material_trial<Real>(L, sn, pc_n, k, M, Mf, st, des, trace);
    if (plastic) {
        material_return<Real>(st, pc_n, k, M, Mf, o, trace);
    } else {
#pragma unroll
        for (int c = 0; c < 6; c++) o.sig[c] = st[c];
        o.pc = pc_n;
        o.plastic = 0;
        o.nonconv = 0;
        o.ret64 = 0;
    }
    o.des = des;
}

// Predicated sub-horizon accumulation: when tst <= thr (member), add the
// outer products zeta~ zeta~^T (6), Ydot zeta~^T (9) and 1 to the count; the
// predicate guards each FMA, so non-members cost no extra multiplies and the
// warp never branches.
__device__ __forceinline__ void masked_accumulate(float tst, float thr, float zx, float zy,
                                                  float zz, float yx, float yy, float yz,
                                                  float (&K)[6], float (&A)[9], float& cnt) {
    asm("{\n\t.reg .pred p;\n\t"
        "setp.le.f32 p, %16, %23;\n\t"
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
        : "f"(tst), "f"(zx), "f"(zy), "f"(zz), "f"(yx), "f"(yy), "f"(yz), "f"(thr));
}

// Predicated sum of a sender's 3x3 matrix (M) into N when tst <= thr.
__device__ __forceinline__ void masked_add9(float tst, float thr, const float4& m0,
                                            const float4& m1, float m8, float (&N)[9]) {
    asm("{\n\t.reg .pred p;\n\t"
        "setp.le.f32 p, %9, %19;\n\t"
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
          "f"(m1.w), "f"(m8), "f"(thr));
}

// Predicated sum of a sender's 6 + 9 adjoint terms (G in g0, g1.xy; Ab in
// g1.zw, g2, g3.xyz) into G, A when tst <= thr.
__device__ __forceinline__ void masked_add15(float tst, float thr, const float4& g0,
                                             const float4& g1, const float4& g2,
                                             const float4& g3, float (&G)[6], float (&A)[9]) {
    asm("{\n\t.reg .pred p;\n\t"
        "setp.le.f32 p, %15, %16;\n\t"
        "@p add.f32 %0, %0, %17;\n\t"
        "@p add.f32 %1, %1, %18;\n\t"
        "@p add.f32 %2, %2, %19;\n\t"
        "@p add.f32 %3, %3, %20;\n\t"
        "@p add.f32 %4, %4, %21;\n\t"
        "@p add.f32 %5, %5, %22;\n\t"
        "@p add.f32 %6, %6, %23;\n\t"
        "@p add.f32 %7, %7, %24;\n\t"
        "@p add.f32 %8, %8, %25;\n\t"
        "@p add.f32 %9, %9, %26;\n\t"
        "@p add.f32 %10, %10, %27;\n\t"
        "@p add.f32 %11, %11, %28;\n\t"
        "@p add.f32 %12, %12, %29;\n\t"
        "@p add.f32 %13, %13, %30;\n\t"
        "@p add.f32 %14, %14, %31;\n\t"
        "}"
        : "+f"(G[0]), "+f"(G[1]), "+f"(G[2]), "+f"(G[3]), "+f"(G[4]), "+f"(G[5]),
          "+f"(A[0]), "+f"(A[1]), "+f"(A[2]), "+f"(A[3]), "+f"(A[4]), "+f"(A[5]), "+f"(A[6]),
          "+f"(A[7]), "+f"(A[8])
        : "f"(tst), "f"(thr), "f"(g0.x), "f"(g0.y), "f"(g0.z), "f"(g0.w), "f"(g1.x), "f"(g1.y),
          "f"(g1.z), "f"(g1.w), "f"(g2.x), "f"(g2.y), "f"(g2.z), "f"(g2.w), "f"(g3.x), "f"(g3.y),
          "f"(g3.z));
}

// butterfly sum within one warp: every lane ends with the same bits
template <int NV, typename T>
__device__ __forceinline__ void warp_sum(T (&v)[NV]) {
#pragma unroll
    for (int e = 0; e < NV; e++)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[e] += __shfl_xor_sync(0xffffffffu, v[e], off);
}

// deterministic block sum: butterfly within warps, then warps in order.  The
// butterfly leaves every lane with the same bits (each stage adds the same two
// operands on both partners), so a one-warp block needs nothing more.
template <int NV, typename T>
__device__ __forceinline__ void block_sum(T (&v)[NV], T (*sm)[NV]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < NV; e++)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[e] += __shfl_xor_sync(0xffffffffu, v[e], off);
    if (blockDim.x == 32) return;
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

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// A non-negative integer held exactly in a float (below 2^22) as an int,
// by adding 1.5 * 2^23 so that the value lands in the low mantissa bits:
// the same result as the conversion instruction, which on GB300 issues on
// the FP64 pipe.
__device__ __forceinline__ int small_count(float c) {
    return __float_as_int(c + 12582912.0f) - 0x4B400000;
}

// A small integer (|x| < 2^22) as a float, exactly, by the inverse of
// small_count: the conversion instruction issues on the FP64 pipe on GB300.
__device__ __forceinline__ float small_float(int x) {
    return __int_as_float(0x4B400000 + x) - 12582912.0f;
}

// FP32 sub-horizon membership test of member k (z_k = (zeta~_k, |zeta~_k|^2))
// for bond j, with m_j = (-2 zeta~_j, hf^2 - |zeta~_j|^2):
// |z_k|^2 - 2 z_k.z_j <= hf^2 - |z_j|^2, i.e. |zeta~_k - zeta~_j|^2 <= hf^2
// (the sub-horizon test of Alg. 1), always with this rounding sequence, so
// that every scalar kernel that tests a pair takes the same decision (the
// tensor-core kernel below has its own test, shared by its two passes).
__device__ __forceinline__ float member_test_lhs(float zx, float zy, float zz, float zw, float mx,
                                                 float my, float mz) {
    return __fmaf_rn(zx, mx, __fmaf_rn(zy, my, __fmaf_rn(zz, mz, zw)));
}

// ---------------------------------------------------------------------------
// Sub-horizon sums on the tensor cores (mixed path)
// ---------------------------------------------------------------------------
// For one point with nb <= kTcRows bonds, the sums of every bond t over its
// sub-horizon (Eq. 23-25, 55) form a product: F = Mask * Phi, where
// Mask[t][k] = 1 if family member k lies in the sub-horizon of bond t and
// Phi[k] holds the member's features zeta~ zeta~^T (6), Ydot zeta~^T (9) and
// 1 (count).  Mask is exact in fp16.  Each feature is scaled by a power of
// two into [-1, 1] and split (Veltkamp, in FP32) into a part of 11
// significant bits and the remainder; both are fp16 terms, together within
// 2^-24 of the largest scaled feature.  The products are exact and
// accumulate in FP32 (mma.sync m16n8k16), so the sums have the accuracy of
// the FP32 sums they replace, with another rounding order.  One warp does a
// point: the features once, then 32 bonds (two 16-row tiles) per pass, just
// before their updates.
//
// The membership test itself is a tensor-core product too.  With zeta~
// scaled by sT (a power of two that brings the point's largest |component|
// into [1/2, 1)), d(t, k) = sT^2 (|zeta~_k - zeta~_t|^2 - hf^2)
//   = sum_c (-2 c_t)(c_k) + w_k + e_t,  w = sT^2 |zeta~|^2, e_t = w_t - sT^2 hf^2,
// and member k lies in the sub-horizon of bond t when d(t, k) < 0.  Each
// scaled component is split c = c^h + c^l (c^h exact in fp16, c^l rounded
// to fp16) and so is w; a bond row carries (-2c^h, -2c^h, -2c^l, -2c^l) per
// component and (1, 1) against the member column's (c^h, c^l, c^h, c^l)
// and (w^h, w^l): 14 of the 16 terms of one m16n8k16 product, whose
// accumulator starts at e_t (FP32).  The split keeps each component to
// 2^-24 and w to 2^-22 of the scaled range, so the decision carries about
// the rounding of the FP32 test (member_test_lhs), from another sequence;
// pairs within ~1e-6 of the sub-horizon radius may be decided differently
// from the FP64 oracle, as with the FP32 test.  The signs of a 16 x 16 tile
// of d become the mask fragment directly (the accumulator layout of the
// product is the operand layout of the next one).  Both passes of the
// power-conjugate force state take the same products (same operands, same
// instruction), so every decision is taken once, bit for bit.
constexpr int kTcRows = 128;        // bonds (and members) of a point summed this way
constexpr int kTcPhiWords = 32 * 64;   // feature rows x member pairs (fp16 pairs)
constexpr int kTcF = 17;            // floats per bond row of a pass's sums (odd: conflict-free)
constexpr int kTcYF = (kTcRows * 16 > 32 * kTcF * 4) ? kTcRows * 16 : 32 * kTcF * 4;
constexpr unsigned kTcOnes = 0x3C003C00u;   // the fp16 pair (1, 1)
constexpr unsigned kTcFarWord = 0x7753u;    // the fp16 pair (30000, 0): a member in no sub-horizon
constexpr float kTcFar = 30000.0f;          // and the accumulator start of a bond with no members

// Word index of member pair kp (fp16 pair) in feature row f of phi.  Rows
// are 256 bytes apart; the 16-byte chunk c of row f is stored at c ^ (f & 7),
// so that the eight rows of one ldmatrix fall in eight different bank groups.
__device__ __forceinline__ int tc_phi_word(int f, int kp) {
    return f * 64 + ((((kp >> 2) ^ (f & 7)) << 2) | (kp & 3));
}

// 2^-(e+1) for 2^e <= m < 2^(e+1): m times it lies in [1/2, 1)
__device__ __forceinline__ float tc_scale(float m) {
    const int e = (int)((__float_as_uint(m) >> 23) & 0xffu);
    if (e == 0 || e >= 253) return 1.0f;
    return __uint_as_float((unsigned)(253 - e) << 23);
}

// two FP32 values as an fp16 pair (lo in the low half), one packed conversion
__device__ __forceinline__ unsigned tc_pack(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const unsigned*>(&h);
}

// Veltkamp split with the factor 2^13 + 1: hi keeps 11 significant bits of
// f, lo = f - hi exactly (no contraction into fused operations)
__device__ __forceinline__ void tc_split(float f, float& hi, float& lo) {
    const float c = __fmul_rn(f, 8193.0f);
    hi = __fsub_rn(c, __fsub_rn(c, f));
    lo = __fsub_rn(f, hi);
}

__device__ __forceinline__ unsigned tc_split_pack(float f) {
    float h, l;
    tc_split(f, h, l);
    return tc_pack(h, l);
}

__device__ __forceinline__ void tc_mma(float (&c)[4], unsigned a0, unsigned a1, unsigned a2,
                                       unsigned a3, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void tc_ldmatrix_x4(unsigned addr, unsigned& r0, unsigned& r1,
                                               unsigned& r2, unsigned& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

// the 8 x 8 matrix of fp16 pairs held as one mma fragment, transposed
__device__ __forceinline__ unsigned tc_transpose8(unsigned a) {
    unsigned d;
    asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(d) : "r"(a));
    return d;
}

// The mask pair of two test values: fp16 1.0 in the low half when lo < 0
// (its sign bit set), in the high half when hi < 0.  The permute replicates
// each sign bit over two bytes; the mask keeps the bits of 1.0.
__device__ __forceinline__ unsigned tc_sign_pair(float lo, float hi) {
    unsigned r;
    asm("prmt.b32 %0, %1, %2, 0xFFBB;" : "=r"(r) : "r"(__float_as_uint(lo)), "r"(__float_as_uint(hi)));
    return r & kTcOnes;
}

// The bond-side terms of row r of the test for this lane's column group tq
// (rows of the product: tq < 3 component tq, tq == 3 the |zeta~|^2 terms):
// first = the terms against the member's (c^h, c^l) in k-columns 2tq, 2tq + 1,
// second = those in k-columns 2tq + 8, 2tq + 9, and the accumulator start e.
// tw holds the member words (tc_build_features); a row without a finite,
// representable bond vector (or a padding row) gets e = kTcFar: no members.
__device__ __forceinline__ void tc_bond_terms(const unsigned* tw, const R4<float>* s_z, int r, int tq,
                                              float sT2, float hf2s, unsigned& first,
                                              unsigned& second, float& e) {
    const unsigned wq = tw[4 * r + tq], ww = tw[4 * r + 3];
    unsigned dh, dl;
    asm("prmt.b32 %0, %1, %1, 0x1010;" : "=r"(dh) : "r"(wq));   // (c^h, c^h)
    asm("prmt.b32 %0, %1, %1, 0x3232;" : "=r"(dl) : "r"(wq));   // (c^l, c^l)
    const __half2 m2 = __float2half2_rn(-2.0f);                  // exact products
    const __half2 ph = __hmul2(*reinterpret_cast<const __half2*>(&dh), m2);
    const __half2 pl = __hmul2(*reinterpret_cast<const __half2*>(&dl), m2);
    first = tq < 3 ? *reinterpret_cast<const unsigned*>(&ph) : kTcOnes;
    second = tq < 3 ? *reinterpret_cast<const unsigned*>(&pl) : 0u;
    e = ww == kTcFarWord ? kTcFar : __fmaf_rn(s_z[r].w, sT2, -hf2s);
}

// The 15 scaled features and the count of member k (all zero for a padding
// member or one without a finite position: it is in no sub-horizon; a
// non-finite velocity stays in its features and makes the point's velocity
// gradients NaN, as in the scalar sums)
// (the same from the member's values and its validity ok)
__device__ __forceinline__ void tc_member_features_of(R4<float> z, R4<float> y, bool ok, float sK,
                                                      float sA, float (&f)[16]) {
    if (!ok) {
        z.x = z.y = z.z = 0.0f;
        y.x = y.y = y.z = 0.0f;
    }
    f[0] = z.x * z.x * sK; f[1] = z.y * z.y * sK; f[2] = z.z * z.z * sK;
    f[3] = z.y * z.z * sK; f[4] = z.x * z.z * sK; f[5] = z.x * z.y * sK;
    f[6] = y.x * z.x * sA; f[7] = y.x * z.y * sA; f[8] = y.x * z.z * sA;
    f[9] = y.y * z.x * sA; f[10] = y.y * z.y * sA; f[11] = y.y * z.z * sA;
    f[12] = y.z * z.x * sA; f[13] = y.z * z.y * sA; f[14] = y.z * z.z * sA;
    f[15] = ok ? 1.0f : 0.0f;
}

__device__ __forceinline__ void tc_member_features(const R4<float>* s_z, const R4<float>* s_y, int k,
                                                   int nb, float sK, float sA, float (&f)[16]) {
    R4<float> z, y;
    z.x = z.y = z.z = z.w = 0.0f;
    y = z;
    if (k < nb) {
        z = s_z[k];
        y = s_y[k];
    }
    const bool ok = k < nb && fmaxf(fabsf(z.x), fmaxf(fabsf(z.y), fabsf(z.z))) <= FLT_MAX;
    tc_member_features_of(z, y, ok, sK, sA, f);
}

// The member features of a point into phi (row 2f: the high part
// of feature f, row 2f + 1: the low part, 32 rows of fp16 pairs along the
// members), the factors uK, uA that undo the scaling of the K~ and A~ sums,
// the member words of the test into tw (4 per member: (c^h, c^l) of the
// three scaled components and of w; kTcFarWord in the last for a member in
// no sub-horizon, zeros before it) and the test's scale sT.  Members
// [nb, 16 ceil(nb/16)) are padding: zero features, far words, and zeroed
// in s_z.
// NTH threads build them together: one warp (NTH = 32), or a whole block of
// NTH threads, which then needs 2 NTH / 32 floats of shared scratch for the
// maxima and synchronises the block.
template <int NTH>
__device__ __forceinline__ void tc_sync() {
    if constexpr (NTH == 32) __syncwarp();
    else __syncthreads();
}

// the largest of v over the NTH threads (non-negative floats order as
// their bit patterns)
template <int NTH>
__device__ __forceinline__ float tc_group_max(float v, float* scratch) {
    v = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(v)));
    if constexpr (NTH > 32) {
        if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = v;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NTH / 32; q++) v = fmaxf(v, scratch[q]);
        __syncthreads();
    }
    return v;
}

template <int NTH>
__device__ __forceinline__ void tc_build_features(R4<float>* s_z, const R4<float>* s_y, int nb,
                                                  unsigned* phi, unsigned* tw, float& uK,
                                                  float& uA, float& sT, float* scratch = nullptr) {
    const int lane = NTH == 32 ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
    const int KT = (nb + 15) >> 4;
    // largest |component| of zeta~ and of Ydot over the members with finite values
    float mz = 0.0f, my = 0.0f;
    for (int k = lane; k < nb; k += NTH) {
        const R4<float> z = s_z[k], y = s_y[k];
        const float az = fmaxf(fabsf(z.x), fmaxf(fabsf(z.y), fabsf(z.z)));
        const float ay = fmaxf(fabsf(y.x), fmaxf(fabsf(y.y), fabsf(y.z)));
        if (az <= FLT_MAX) mz = fmaxf(mz, az);
        if (az <= FLT_MAX && ay <= FLT_MAX) my = fmaxf(my, ay);
    }
    mz = tc_group_max<NTH>(mz, scratch);
    my = tc_group_max<NTH>(my, scratch);
    const float sK = tc_scale(mz * mz), sA = tc_scale(mz * my);
    uK = 1.0f / sK;                                      // powers of two: exact
    uA = 1.0f / sA;
    sT = tc_scale(mz);
    const float sT2 = sT * sT;
    for (int kp = lane; kp < KT * 8; kp += NTH) {
        float f0[16], f1[16];
        tc_member_features(s_z, s_y, 2 * kp, nb, sK, sA, f0);
        tc_member_features(s_z, s_y, 2 * kp + 1, nb, sK, sA, f1);
#pragma unroll
        for (int e = 0; e < 15; e++) {
            float h0, l0, h1, l1;
            tc_split(f0[e], h0, l0);
            tc_split(f1[e], h1, l1);
            phi[tc_phi_word(2 * e, kp)] = tc_pack(h0, h1);      // exact: 11 significant bits
            phi[tc_phi_word(2 * e + 1, kp)] = tc_pack(l0, l1);
        }
        phi[tc_phi_word(30, kp)] = tc_pack(f0[15], f1[15]);
        phi[tc_phi_word(31, kp)] = 0u;
    }
    for (int k = lane; k < KT * 16; k += NTH) {
        uint4 W = make_uint4(0u, 0u, 0u, kTcFarWord);
        if (k < nb) {
            const R4<float> z = s_z[k];
            const float cx = z.x * sT, cy = z.y * sT, cz = z.z * sT, cw = z.w * sT2;
            // comparisons with NaN are false: such a member stays far
            if (fabsf(cx) < 2.0f && fabsf(cy) < 2.0f && fabsf(cz) < 2.0f && cw < 16.0f)
                W = make_uint4(tc_split_pack(cx), tc_split_pack(cy), tc_split_pack(cz), tc_split_pack(cw));
        }
        reinterpret_cast<uint4*>(tw)[k] = W;
    }
    tc_sync<NTH>();
    for (int k = nb + lane; k < KT * 16; k += NTH) {
        R4<float> zero;
        zero.x = zero.y = zero.z = zero.w = 0.0f;
        s_z[k] = zero;
    }
    tc_sync<NTH>();
}

// One warp, pass p: the sums of bonds 32p .. 32p + 31 (row tiles 2p, 2p + 1)
// into rows of FS floats, F[r FS + 0..15]: 0..5 = K~ (xx yy zz yz xz xy),
// 6..14 = A~ (row-major, A_rc = sum Ydot_r zeta~_c), 15 = |S| of bond 32p + r.
// hf2s = sT^2 hf^2.
template <int FS>
__device__ __forceinline__ void tc_pass_sums(const R4<float>* s_z, const unsigned* tw, int nb, int p,
                                             float sT2, float hf2s, const unsigned* phi, float* F,
                                             float uK, float uA) {
    const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    const int KT = (nb + 15) >> 4;
    const int nm = KT - 2 * p >= 2 ? 2 : 1;              // row tiles with bonds in this pass
    // the test's bond-side terms of this lane's rows 32p + 16m + g (+ 8):
    // ta[m] = (a0, a1, a2, a3) of the product, te[m] = accumulator starts
    unsigned ta[2][4];
    float te[2][2];
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int h = 0; h < 2; h++) {
            ta[m][h] = ta[m][2 + h] = 0u;
            te[m][h] = kTcFar;
            if (m < nm)
                tc_bond_terms(tw, s_z, 32 * p + 16 * m + g + 8 * h, tq, sT2, hf2s, ta[m][h],
                              ta[m][2 + h], te[m][h]);
        }
    float acc[2][4][4];
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int nt = 0; nt < 4; nt++)
#pragma unroll
            for (int e = 0; e < 4; e++) acc[m][nt][e] = 0.0f;
    // ldmatrix rows: lanes 8q .. 8q + 7 address matrix q = (n-tile q/2, k half q%2)
    const int lm = lane >> 3, lr = lane & 7;
    const unsigned phi_base = (unsigned)__cvta_generic_to_shared(phi);
    for (int kt = 0; kt < KT; kt++) {
        // the test's member-side terms of members 16kt + g and 16kt + 8 + g
        const unsigned w0 = tw[4 * (16 * kt + g) + tq], w1 = tw[4 * (16 * kt + 8 + g) + tq];
        const unsigned v0 = tq < 3 ? w0 : 0u, v1 = tq < 3 ? w1 : 0u;
        unsigned b[4][2];
#pragma unroll
        for (int np = 0; np < 2; np++) {
            const int row = 8 * (2 * np + (lm >> 1)) + lr;
            const unsigned addr = phi_base + 4u * (unsigned)tc_phi_word(row, 8 * kt + 4 * (lm & 1));
            tc_ldmatrix_x4(addr, b[2 * np][0], b[2 * np][1], b[2 * np + 1][0], b[2 * np + 1][1]);
        }
#pragma unroll
        for (int m = 0; m < 2; m++) {
            if (m >= nm) continue;                       // warp-uniform
            float d0[4] = {te[m][0], te[m][0], te[m][1], te[m][1]};
            float d1[4] = {te[m][0], te[m][0], te[m][1], te[m][1]};
            tc_mma(d0, ta[m][0], ta[m][1], ta[m][2], ta[m][3], w0, v0);   // members 16kt + 0..7
            tc_mma(d1, ta[m][0], ta[m][1], ta[m][2], ta[m][3], w1, v1);   // members 16kt + 8..15
            const unsigned a0 = tc_sign_pair(d0[0], d0[1]);   // row g, columns 2tq, 2tq + 1
            const unsigned a1 = tc_sign_pair(d0[2], d0[3]);   // row g + 8
            const unsigned a2 = tc_sign_pair(d1[0], d1[1]);   // row g, columns 2tq + 8, 2tq + 9
            const unsigned a3 = tc_sign_pair(d1[2], d1[3]);   // row g + 8
#pragma unroll
            for (int nt = 0; nt < 4; nt++) tc_mma(acc[m][nt], a0, a1, a2, a3, b[nt][0], b[nt][1]);
        }
    }
#pragma unroll
    for (int m = 0; m < 2; m++) {
        if (m >= nm) continue;
#pragma unroll
        for (int nt = 0; nt < 4; nt++) {
            const int f = 4 * nt + tq;                   // columns 2f (high part) and 2f + 1 (low)
            const float u = f < 6 ? uK : (f < 15 ? uA : 1.0f);
            F[(16 * m + g) * FS + f] = (acc[m][nt][0] + acc[m][nt][1]) * u;
            F[(16 * m + g + 8) * FS + f] = (acc[m][nt][2] + acc[m][nt][3]) * u;
        }
    }
    __syncwarp();
}

// One warp, pass p of receiver sums: for receivers t = 32p .. 32p + 31,
// N_t = sum over senders q of [t in S_q] V_q, where V_q holds nf < 16 values
// of sender bond q (the power-conjugate force state: M_q = varpi sigma K^-1,
// 9 values; the adjoint: its 6 + 9 sender terms).  The mask element (t, q)
// is the sender pass's own decision: the test tile is taken with the
// senders as rows and the receivers as columns, exactly as tc_pass_sums took
// it (same operands, same product), and its mask fragments are transposed
// (movmatrix).  phi holds V split into fp16 pairs (row 2f: high, 2f + 1: low
// part of value f; the other rows zero) scaled by powers of two: u_lo undoes
// the scaling of values f < f_split, u_hi that of the others.  Writes
// F[r FS + f], f < nf, for receiver 32p + r; NT n-tiles of 8 rows of phi
// (3 for 9 values, 4 for 15).
template <int NT, int FS>
__device__ __forceinline__ void tc_pass_receiver(const R4<float>* s_z, const unsigned* tw, int nb,
                                                 int p, float sT2, float hf2s, const unsigned* phi,
                                                 float* F, float u_lo, float u_hi, int f_split,
                                                 int nf) {
    const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    const int KT = (nb + 15) >> 4;
    const int nm = KT - 2 * p >= 2 ? 2 : 1;
    // the test's member-side terms of this lane's receivers 32p + 16m + 8n + g
    unsigned rw[2][2], rv[2][2];
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int n = 0; n < 2; n++) {
            rw[m][n] = m < nm ? tw[4 * (32 * p + 16 * m + 8 * n + g) + tq] : 0u;
            rv[m][n] = tq < 3 ? rw[m][n] : 0u;
        }
    static_assert(NT == 3 || NT == 4, "three or four n-tiles of values");
    float acc[2][NT][4];
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int nt = 0; nt < NT; nt++)
#pragma unroll
            for (int e = 0; e < 4; e++) acc[m][nt][e] = 0.0f;
    const int lm = lane >> 3, lr = lane & 7;
    const unsigned phi_base = (unsigned)__cvta_generic_to_shared(phi);
    for (int kt = 0; kt < KT; kt++) {
        // the test's bond-side terms of senders 16kt + g and 16kt + 8 + g
        unsigned sa[4];
        float se[2];
        tc_bond_terms(tw, s_z, 16 * kt + g, tq, sT2, hf2s, sa[0], sa[2], se[0]);
        tc_bond_terms(tw, s_z, 16 * kt + 8 + g, tq, sT2, hf2s, sa[1], sa[3], se[1]);
        unsigned b[4][2];
        {
            const int row = 8 * (lm >> 1) + lr;
            const unsigned addr = phi_base + 4u * (unsigned)tc_phi_word(row, 8 * kt + 4 * (lm & 1));
            tc_ldmatrix_x4(addr, b[0][0], b[0][1], b[1][0], b[1][1]);
            const unsigned addr2 = phi_base + 4u * (unsigned)tc_phi_word(16 + row, 8 * kt + 4 * (lm & 1));
            tc_ldmatrix_x4(addr2, b[2][0], b[2][1], b[3][0], b[3][1]);   // rows 24..31: used with NT = 4
        }
#pragma unroll
        for (int m = 0; m < 2; m++) {
            if (m >= nm) continue;
            float d0[4] = {se[0], se[0], se[1], se[1]};
            float d1[4] = {se[0], se[0], se[1], se[1]};
            tc_mma(d0, sa[0], sa[1], sa[2], sa[3], rw[m][0], rv[m][0]);   // receivers 0..7 of the tile
            tc_mma(d1, sa[0], sa[1], sa[2], sa[3], rw[m][1], rv[m][1]);   // receivers 8..15
            // the senders' mask (rows q, columns t) in four 8 x 8 blocks, transposed
            const unsigned f0 = tc_sign_pair(d0[0], d0[1]), f1 = tc_sign_pair(d0[2], d0[3]);
            const unsigned f2 = tc_sign_pair(d1[0], d1[1]), f3 = tc_sign_pair(d1[2], d1[3]);
            const unsigned a0 = tc_transpose8(f0), a1 = tc_transpose8(f2);
            const unsigned a2 = tc_transpose8(f1), a3 = tc_transpose8(f3);
#pragma unroll
            for (int nt = 0; nt < NT; nt++) tc_mma(acc[m][nt], a0, a1, a2, a3, b[nt][0], b[nt][1]);
        }
    }
#pragma unroll
    for (int m = 0; m < 2; m++) {
        if (m >= nm) continue;
#pragma unroll
        for (int nt = 0; nt < NT; nt++) {
            const int f = 4 * nt + tq;
            if (f < nf) {
                const float u = f < f_split ? u_lo : u_hi;
                F[(16 * m + g) * FS + f] = (acc[m][nt][0] + acc[m][nt][1]) * u;
                F[(16 * m + g + 8) * FS + f] = (acc[m][nt][2] + acc[m][nt][3]) * u;
            }
        }
    }
    __syncwarp();
}

// One warp: the senders' matrices sM[q][0..8] (q < nb) into phi for
// tc_pass_receiver, scaled by a power of two below the largest |entry|;
// returns the factor that undoes the scaling.  Rows 18..31 are zero, and so
// are members [nb, 16 ceil(nb/16)).
template <int W>
__device__ __forceinline__ float tc_build_sender_features(const float (*sM)[W], int nb,
                                                          unsigned* phi) {
    const int lane = threadIdx.x & 31;
    const int KT = (nb + 15) >> 4;
    float mx = 0.0f;
    for (int q = lane; q < nb; q += 32)
#pragma unroll
        for (int e = 0; e < 9; e++) {
            const float a = fabsf(sM[q][e]);
            if (a <= FLT_MAX) mx = fmaxf(mx, a);
        }
    mx = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(mx)));
    const float sc = tc_scale(mx);
    for (int kp = lane; kp < KT * 8; kp += 32) {
        const int q0 = 2 * kp, q1 = 2 * kp + 1;
#pragma unroll
        for (int e = 0; e < 9; e++) {
            const float v0 = q0 < nb ? sM[q0][e] * sc : 0.0f;
            const float v1 = q1 < nb ? sM[q1][e] * sc : 0.0f;
            float h0, l0, h1, l1;
            tc_split(v0, h0, l0);
            tc_split(v1, h1, l1);
            phi[tc_phi_word(2 * e, kp)] = tc_pack(h0, h1);
            phi[tc_phi_word(2 * e + 1, kp)] = tc_pack(l0, l1);
        }
#pragma unroll
        for (int r = 18; r < 32; r++) phi[tc_phi_word(r, kp)] = 0u;
    }
    __syncwarp();
    return 1.0f / sc;
}

// NTH threads (tc_build_features): the adjoint's sender terms of bonds q < nb (rows of stride
// floats: G at row[0..5], Ab at row[6..14]) into phi for tc_pass_receiver
// (row 2f: high, 2f + 1: low part of value f; rows 30, 31 and members
// [nb, 16 ceil(nb/16)) zero), G and Ab each scaled by a power of two below
// its largest |entry|; uG, uAb undo the scalings.
template <int NTH>
__device__ __forceinline__ void tc_build_adj_sender_features(const float* rows, int stride, int nb,
                                                             unsigned* phi, float& uG, float& uAb,
                                                             float* scratch) {
    const int lane = NTH == 32 ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
    const int KT = (nb + 15) >> 4;
    // maxima: consecutive threads take consecutive values of a row (few bank conflicts)
    float mg = 0.0f, ma = 0.0f;
    for (int idx = lane; idx < 15 * nb; idx += NTH) {
        const int q = idx / 15, e = idx - 15 * q;
        const float a = fabsf(rows[q * stride + e]);
        if (a <= FLT_MAX) {
            if (e < 6) mg = fmaxf(mg, a);
            else ma = fmaxf(ma, a);
        }
    }
    mg = tc_group_max<NTH>(mg, scratch);
    ma = tc_group_max<NTH>(ma, scratch);
    const float sg = tc_scale(mg), sa = tc_scale(ma);
    // value e (e < 15; 15: the zero rows 30, 31) of member pair kp
    for (int idx = lane; idx < 16 * KT * 8; idx += NTH) {
        const int kp = idx >> 4, e = idx & 15;
        const int q0 = 2 * kp, q1 = 2 * kp + 1;
        unsigned hi = 0u, lo = 0u;
        if (e < 15) {
            const float sc = e < 6 ? sg : sa;
            const float v0 = q0 < nb ? rows[q0 * stride + e] * sc : 0.0f;
            const float v1 = q1 < nb ? rows[q1 * stride + e] * sc : 0.0f;
            float h0, l0, h1, l1;
            tc_split(v0, h0, l0);
            tc_split(v1, h1, l1);
            hi = tc_pack(h0, h1);
            lo = tc_pack(l0, l1);
        }
        phi[tc_phi_word(2 * e, kp)] = hi;
        phi[tc_phi_word(2 * e + 1, kp)] = lo;
    }
    tc_sync<NTH>();
    uG = 1.0f / sg;
    uAb = 1.0f / sa;
}

// ---------------------------------------------------------------------------
// Sub-horizon tests and sums in tensor memory (tcgen05, mixed path, Eq. 51)
// ---------------------------------------------------------------------------
// One CTA of 128 threads does a point, thread t its bond t and its member t.
// Operands sit in shared memory in the no-swizzle K-major core-matrix layout
// (8 rows x 16 bytes per core matrix; 128 bytes between core matrices along
// K, 128 * K / 8 bytes between groups of 8 rows), accumulators in 128 columns
// of tensor memory (row t = lane t).  Per point two products, each issued by
// one thread and awaited on an mbarrier:
//   d (128 x 128, f32) = bond terms (128 x 16) * member terms (128 x 16)^T:
//       the squared distances of the sub-horizon test, as in the warp kernel
//       (slots per component c: bond (-2c^h, -2c^h, -2c^l, -2c^l) against
//       member (c^h, c^l, c^h, c^l); then (1, 1) against (w^h, w^l) and
//       (e^h, e^l) against (1, 1), e = sT^2 (|zeta~_t|^2 - hf^2));
//   F (128 x 32, f32) = Mask (128 x 128) * Phi (32 x 128)^T in eight steps of
//       K = 16, Mask[t][k] = [d(t, k) < 0] written by thread t from its row.
constexpr int kT5Threads = 128;
constexpr unsigned kT5Cols = 128;                 // tensor-memory columns per CTA
constexpr int kT5Mask = 0;                        // Mask: 128 x 128 fp16 (32 KB); later the park rows
constexpr int kT5Phi = 32768;                     // Phi: 32 x 128 fp16 (8 KB)
constexpr int kT5Bond = 40960;                    // bond terms: 128 x 16 fp16 (4 KB)
constexpr int kT5Memb = 45056;                    // member terms: 128 x 16 fp16 (4 KB)
constexpr int kT5Smem = 49152;                    // dynamic shared memory per CTA
// instruction descriptors (kind::f16): f32 accumulator (bits 4-5 = 1), f16 A
// and B (0), both K-major (0), N >> 3 in bits 17-22, M >> 4 in bits 24-28
constexpr uint32_t kT5IdescDist = (1u << 4) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t kT5IdescSums = (1u << 4) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
// a wait is given up after about a second (global timer), or after 2^24
// polls should the timer not advance
constexpr unsigned long long kT5WaitNs = 1000000000ull;
constexpr int kT5WaitPolls = 1 << 24;

// byte offset of element (r, k) in a K-major matrix with K columns
__device__ __forceinline__ uint32_t t5_off(int r, int k, int K) {
    return (uint32_t)(r >> 3) * (uint32_t)(16 * K) + (uint32_t)(k >> 3) * 128u + (uint32_t)(r & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

// shared-memory matrix descriptor: start, leading (K-direction) and stride
// (8-row) byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t t5_desc(uint32_t saddr, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void t5_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void t5_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(mbar) : "memory");
}

__device__ __forceinline__ unsigned long long t5_now() {
    unsigned long long ns;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(ns));
    return ns;
}

// bounded wait for the completion of phase `parity` of the mbarrier: true
// once it completes, false when the time or poll bound runs out first
__device__ __forceinline__ bool t5_wait(uint32_t mbar, uint32_t parity) {
    unsigned long long t0 = 0;
    for (int it = 0; it < kT5WaitPolls; it++) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n" : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
        if (ok) return true;
        const unsigned long long now = t5_now();
        if (it == 0) t0 = now;
        else if (now - t0 > kT5WaitNs) return false;
    }
    return false;
}

__device__ __forceinline__ void t5_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void t5_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// shared-memory writes of the threads become visible to the tensor cores
__device__ __forceinline__ void t5_fence_proxy() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 consecutive columns of this thread's lane (32x32b shape, 32 repetitions)
__device__ __forceinline__ void t5_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                 "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                   "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                   "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; j++) v[j] = __uint_as_float(r[j]);
}

}  // namespace
}  // namespace ppm
