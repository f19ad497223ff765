// Reverse (adjoint) of the explicit step, for gradients of an objective of
// the final displacement with respect to the critical-state slope M, the
// viscosity eta, the suction (through S_r s) and the initial
// preconsolidation pressure.  Each reverse step restores the step's start
// state, recomputes its forward bond pass -- families, sub-horizons and
// elastic/plastic branches as the forward took them -- and applies the
// transposed chain rule of: the velocity corrector and acceleration
// (Eq. 62-63), the pairwise force gather (Eq. 49-50), the force state
// (Eq. 31-32, 51), the point-state mean, the constitutive update
// (Hughes-Winget rotation, trial stress Eq. 41, and the implicit function of
// the return solve Eq. 73-75), the velocity gradient and shape-tensor
// inverse (Eq. 25, 57), the sub-horizon sums (Eq. 23, 25) and the Newmark
// predictor (Eq. 60-61, 64).
//
// Scaled variables as in the forward kernel: zeta~ = zeta / dx,
// K~ = sum zeta~ zeta~^T, A~ = sum Ydot zeta~^T, L = A~ K~^-1 / dx,
// T^ = varpi S K~^-1 zeta~_j, f = dx^2 (sum T^ - sum T^').
#include <cuda_runtime.h>
#include <math.h>

#include "bond_device.cuh"
#include "ppm_internal.cuh"

namespace ppm {
namespace {

// full symmetric 3x3 adjoint (off-diagonals shared) <-> 6 stored components
template <typename Real>
__device__ __forceinline__ void six_to_full(const Real a6[6], Real M[9]) {
    M[0] = a6[0]; M[4] = a6[1]; M[8] = a6[2];
    M[5] = M[7] = (Real)0.5 * a6[3];
    M[2] = M[6] = (Real)0.5 * a6[4];
    M[1] = M[3] = (Real)0.5 * a6[5];
}

template <typename Real>
__device__ __forceinline__ void full_to_six(const Real M[9], Real a6[6]) {
    a6[0] = M[0]; a6[1] = M[4]; a6[2] = M[8];
    a6[3] = M[5] + M[7]; a6[4] = M[2] + M[6]; a6[5] = M[1] + M[3];
}

// Reverse of material_update.  Sbo: adjoint of the output stress (full,
// symmetric); pcbo of the output pc.  Accumulates the adjoint of the input
// stress (Sbi, full), of pc_n, of L (Lb), and of M and eta (FP64).
template <typename Real>
__device__ void material_reverse(const MatTrace<Real>& t, const Real sn[6], Real pc_n,
                                 const StepConst& k, double M, const Real Sbo[9], Real pcbo,
                                 Real Sbi[9], Real& pcbi, Real Lb[9], double& Mb, double& etab) {
    constexpr bool F64 = sizeof(Real) == 8;
    const Real dt = F64 ? (Real)k.dt : (Real)k.dtf;
    const Real Kb = F64 ? (Real)k.K : (Real)k.Kf;
    const Real mu = F64 ? (Real)k.mu : (Real)k.muf;
    Real Strb[9];
    if (!t.plastic) {
#pragma unroll
        for (int e = 0; e < 9; e++) Strb[e] = Sbo[e];
        pcbi += pcbo;
    } else {
        const Real q_tr = t.q_tr;
        const Real s_tr[9] = {t.st[0] - t.p_tr, t.st[5], t.st[4],
                              t.st[5], t.st[1] - t.p_tr, t.st[3],
                              t.st[4], t.st[3], t.st[2] - t.p_tr};
        const Real ratio = q_tr > (Real)0 ? (Real)(t.x[1] / (double)q_tr) : (Real)0;
        double xb[3];
        xb[0] = (double)(Sbo[0] + Sbo[4] + Sbo[8]);
        Real ratiob = 0, sb[9];
#pragma unroll
        for (int e = 0; e < 9; e++) {
            ratiob += Sbo[e] * s_tr[e];
            sb[e] = ratio * Sbo[e];
        }
        double q_trb = 0.0;
        xb[1] = 0.0;
        if (q_tr > (Real)0) {
            xb[1] = (double)ratiob / (double)q_tr;
            q_trb = -(double)ratiob * t.x[1] / ((double)q_tr * (double)q_tr);
        }
        xb[2] = t.floored ? 0.0 : (double)pcbo;
        // implicit function of the return: J^T lambda = xb; ybar = -J_y^T lambda
        const double M2 = M * M, lk = k.lk, c = t.c, pcn = (double)pc_n;
        const double pb = t.x[0], q = t.x[1], pc = t.x[2];
        const double f = q * q / M2 + pb * (pb - pc);
        const double fp = 2.0 * pb - pc, fq = 2.0 * q / M2, fc = -pb;
        const double a = k.K * c, b = 3.0 * k.mu * c, g = c / lk;
        const double J0 = 1.0 + a * (fp * fp + 2.0 * f), J1 = a * fq * fp, J2 = a * (fc * fp - f);
        const double J3 = b * fp * fq, J4 = 1.0 + b * (fq * fq + 2.0 * f / M2), J5 = b * fc * fq;
        const double J6 = g * (fp * fp + 2.0 * f), J7 = g * (fq * fp), J8 = 1.0 / pc + g * (fc * fp - f);
        // transpose: T = [[J0, J3, J6], [J1, J4, J7], [J2, J5, J8]]
        const double m0 = J4 * J8 - J7 * J5, m1 = J1 * J8 - J7 * J2, m2 = J1 * J5 - J4 * J2;
        const double det = J0 * m0 - J3 * m1 + J6 * m2;
        double lam[3] = {0.0, 0.0, 0.0};
        if (det != 0.0 && isfinite(det)) {
            const double id = 1.0 / det;
            lam[0] = (xb[0] * m0 - J3 * (xb[1] * J8 - J7 * xb[2]) + J6 * (xb[1] * J5 - J4 * xb[2])) * id;
            lam[1] = (J0 * (xb[1] * J8 - J7 * xb[2]) - xb[0] * m1 + J6 * (J1 * xb[2] - xb[1] * J2)) * id;
            lam[2] = (J0 * (J4 * xb[2] - xb[1] * J5) - J3 * (J1 * xb[2] - xb[1] * J2) + xb[0] * m2) * id;
        }
        const double p_trb = lam[0];
        q_trb += lam[1];
        double pc_nb = lam[2] / pcn;
        const double cb = -(lam[0] * k.K * f * fp + lam[1] * 3.0 * k.mu * f * fq + lam[2] * f * fp / lk);
        const double dfdM = -2.0 * q * q / (M2 * M), dfqdM = -4.0 * q / (M2 * M);
        Mb -= lam[0] * k.K * c * fp * dfdM + lam[1] * 3.0 * k.mu * c * (dfdM * fq + f * dfqdM) +
              lam[2] * c * fp * dfdM / lk;
        etab += cb * (-c / k.eta);
        if (k.visc_form == 0) pc_nb += cb * (-2.0 * c / pcn);
        pcbi += (Real)pc_nb;
        if (q_tr > (Real)0) {
            const Real qs = (Real)(q_trb * 1.5 / (double)q_tr);
#pragma unroll
            for (int e = 0; e < 9; e++) sb[e] += qs * s_tr[e];
        }
        const Real trs = sb[0] + sb[4] + sb[8];
        const Real shift = ((Real)p_trb - trs) * (Real)(1.0 / 3.0);
#pragma unroll
        for (int e = 0; e < 9; e++) Strb[e] = sb[e] + ((e == 0 || e == 4 || e == 8) ? shift : (Real)0);
    }
    // trial: Str = R + K tr(de) 1 + 2 mu dev(de)
    const Real trS = Strb[0] + Strb[4] + Strb[8];
    Real deb[9];
#pragma unroll
    for (int e = 0; e < 9; e++) {
        const bool dg = (e == 0 || e == 4 || e == 8);
        deb[e] = (Real)2 * mu * (Strb[e] - (dg ? trS * (Real)(1.0 / 3.0) : (Real)0)) + (dg ? Kb * trS : (Real)0);
    }
    // R = Q S Q^T: S-bar = Q^T R-bar Q, Q-bar = 2 R-bar Q S (R-bar, S symmetric)
    const Real* Q = t.Q;
    const Real S[9] = {sn[0], sn[5], sn[4], sn[5], sn[1], sn[3], sn[4], sn[3], sn[2]};
    Real RQ[9], QS[9];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            RQ[r * 3 + c] = Strb[r * 3 + 0] * Q[0 * 3 + c] + Strb[r * 3 + 1] * Q[1 * 3 + c] + Strb[r * 3 + 2] * Q[2 * 3 + c];
            QS[r * 3 + c] = Q[r * 3 + 0] * S[0 * 3 + c] + Q[r * 3 + 1] * S[1 * 3 + c] + Q[r * 3 + 2] * S[2 * 3 + c];
        }
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++)
            Sbi[r * 3 + c] += Q[0 * 3 + r] * RQ[0 * 3 + c] + Q[1 * 3 + r] * RQ[1 * 3 + c] + Q[2 * 3 + r] * RQ[2 * 3 + c];
    Real Qb[9];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++)
            Qb[r * 3 + c] = (Real)2 * (Strb[r * 3 + 0] * QS[0 * 3 + c] + Strb[r * 3 + 1] * QS[1 * 3 + c] + Strb[r * 3 + 2] * QS[2 * 3 + c]);
    // Q = 1 + kap B, B = A + a a^T - (a.a) 1, kap = 2 / (1 + a.a)
    const Real a1 = t.a[0], a2 = t.a[1], a3 = t.a[2], kap = t.kap;
    const Real aa = a1 * a1 + a2 * a2 + a3 * a3;
    const Real B[9] = {a1 * a1 - aa, -a3 + a1 * a2, a2 + a1 * a3,
                       a3 + a2 * a1, a2 * a2 - aa, -a1 + a2 * a3,
                       -a2 + a3 * a1, a1 + a3 * a2, a3 * a3 - aa};
    Real kapb = 0;
#pragma unroll
    for (int e = 0; e < 9; e++) kapb += Qb[e] * B[e];
    Real Bb[9];
#pragma unroll
    for (int e = 0; e < 9; e++) Bb[e] = kap * Qb[e];
    const Real av[3] = {a1, a2, a3};
    const Real trB = Bb[0] + Bb[4] + Bb[8];
    Real ab[3] = {Bb[7] - Bb[5], Bb[2] - Bb[6], Bb[3] - Bb[1]};
#pragma unroll
    for (int r = 0; r < 3; r++) {
        Real s = 0;
#pragma unroll
        for (int c = 0; c < 3; c++) s += (Bb[r * 3 + c] + Bb[c * 3 + r]) * av[c];
        ab[r] += s - (Real)2 * trB * av[r] - kapb * kap * kap * av[r];
    }
    // a = (dt/4) (L21 - L12, L02 - L20, L10 - L01); D = sym(L), de = dt D
    const Real q4 = (Real)0.25 * dt;
    Lb[7] += q4 * ab[0]; Lb[5] -= q4 * ab[0];
    Lb[2] += q4 * ab[1]; Lb[6] -= q4 * ab[1];
    Lb[3] += q4 * ab[2]; Lb[1] -= q4 * ab[2];
#pragma unroll
    for (int e = 0; e < 9; e++) Lb[e] += dt * deb[e];
}


// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// v' = vh + dt/2 a', a' = f/m + g (fixed components: 0):
// fb = (ab + dt/2 vb) / m, vhb = vb, u1b = ub; for the initial pass fb = ab / m
template <typename Real>
__global__ void k_adj_pre(DevState<Real> s, AdjState<Real> a, StepConst k, int initial) {
    const size_t n = (size_t)k.npoints;
    const Real h = sizeof(Real) == 8 ? (Real)(0.5 * k.dt) : (Real)k.hdtf;
    const Real inv_m = (Real)(1.0 / (k.rho * k.dx * k.dx * k.dx));
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < 3 * n;
         t += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / n);
        const size_t i = t - (size_t)c * n;
        Real vbar;
        const bool fixed = prescribed(s, k, (size_t)i, c, vbar);
        const Real abt = initial ? a.ab[t] : a.ab[t] + h * a.vb[t];
        a.fb[t] = fixed ? (Real)0 : abt * inv_m;
        if (!initial) {
            a.vhb[t] = a.vb[t];
            a.u1b[t] = a.ub[t];
        }
    }
}

constexpr int kAdjThreads = 128;
constexpr int kAdjSlots = 25;   // per-bond shared slots (an odd row stride: each thread walks its
                                //   own row without bank conflicts):
constexpr int kSlTest = 0;      //   -2 zeta~_j (3) and hf^2 - |zeta~_j|^2: the membership test
constexpr int kSlG = 4;         //   K~ sums (pass 1), then G = K~-bar + K~-bar^T (pass 2): 6
constexpr int kSlAb = 10;       //   A~ sums (pass 1), then A~-bar (pass 2): 9
constexpr int kSlCnt = 19, kSlAct = 20, kSlZown = 21;   // |S|, active, own zeta~-bar (3)

template <typename Real>
size_t adj_smem_bytes() {
    return 2 * kMaxRow * sizeof(R4<Real>) + (sizeof(Real) == 8 ? 3 * kMaxRow * sizeof(double) : 0) +
           (size_t)kMaxRow * kAdjSlots * sizeof(Real);
}

// One CTA per point: recompute the forward bond pass of the point, then
// reverse it.  INITIAL: the state-preserving initial pass (no constitutive
// update, positions fixed).
template <typename Real, int MODEL, bool INITIAL>
__global__ void __launch_bounds__(kAdjThreads, sizeof(Real) == 4 ? 4 : 2)
k_adj_bond(DevState<Real> s, AdjState<Real> a, StepConst k) {
    constexpr bool F64 = sizeof(Real) == 8;
    constexpr int NW = kAdjThreads / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R4<Real>* s_z = reinterpret_cast<R4<Real>*>(smem_raw);
    R4<Real>* s_y = s_z + kMaxRow;
    double* s_p = reinterpret_cast<double*>(s_y + kMaxRow);               // FP64 only
    Real* s_b = reinterpret_cast<Real*>(s_p + (F64 ? 3 * kMaxRow : 0));   // [kMaxRow][kAdjSlots]
    __shared__ Real s_red[NW][16];
    __shared__ double s_redd[NW][4];
    __shared__ float s_tcs[kAdjThreads / 32];                     // block maxima
    // the tensor-core sums (mixed path, Eq. 51, at most kTcRows bonds) keep
    // their feature rows and test words in the upper half of the bond slots,
    // which only points with more bonds use
    static_assert((kMaxRow - kTcRows) * kAdjSlots >= kTcPhiWords + 4 * kTcRows, "tensor-core scratch");
    unsigned* tc_phi = reinterpret_cast<unsigned*>(s_b + (size_t)kTcRows * kAdjSlots);
    unsigned* tc_tw = tc_phi + kTcPhiWords;
    const int wid = threadIdx.x >> 5;

    const int i = blockIdx.x;
    const size_t n = (size_t)k.npoints;
    const int r0 = s.row_ptr[i];
    int nb = s.row_ptr[i + 1] - r0;
    if (nb > kMaxRow) nb = 0;
    const int li = s.lat[i];
    const int ix = lat_x(li), iy = lat_y(li), iz = lat_z(li);
    const Real inv_dx = F64 ? (Real)k.inv_dx : (Real)k.inv_dxf;
    const Real dx2 = F64 ? (Real)(k.dx * k.dx) : (Real)k.dx2f;

    // stage the family exactly as the forward kernel does
    double pxi = 0, pyi = 0, pzi = 0;
    if constexpr (F64) {
        pxi = __dadd_rn(__dmul_rn((double)ix, k.dx), (double)s.u[i]);
        pyi = __dadd_rn(__dmul_rn((double)iy, k.dx), (double)s.u[n + i]);
        pzi = __dadd_rn(__dmul_rn((double)iz, k.dx), (double)s.u[2 * n + i]);
    }
    const Real uxi = s.u[i], uyi = s.u[n + i], uzi = s.u[2 * n + i];
    const Real vxi = INITIAL ? (Real)0 : s.vh[i], vyi = INITIAL ? (Real)0 : s.vh[n + i],
               vzi = INITIAL ? (Real)0 : s.vh[2 * n + i];
    for (int t = threadIdx.x; t < nb; t += kAdjThreads) {
        const int j = s.col[r0 + t];
        const int lj = s.lat[j];
        R4<Real> z, y;
        if constexpr (F64) {
            const double px = __dadd_rn(__dmul_rn((double)lat_x(lj), k.dx), (double)s.u[j]);
            const double py = __dadd_rn(__dmul_rn((double)lat_y(lj), k.dx), (double)s.u[n + j]);
            const double pz = __dadd_rn(__dmul_rn((double)lat_z(lj), k.dx), (double)s.u[2 * n + j]);
            s_p[t] = px; s_p[kMaxRow + t] = py; s_p[2 * kMaxRow + t] = pz;
            z.x = (Real)((px - pxi) * k.inv_dx);
            z.y = (Real)((py - pyi) * k.inv_dx);
            z.z = (Real)((pz - pzi) * k.inv_dx);
        } else {
            z.x = small_float(lat_x(lj) - ix) + (s.u[j] - uxi) * inv_dx;
            z.y = small_float(lat_y(lj) - iy) + (s.u[n + j] - uyi) * inv_dx;
            z.z = small_float(lat_z(lj) - iz) + (s.u[2 * n + j] - uzi) * inv_dx;
        }
        z.w = z.x * z.x + z.y * z.y + z.z * z.z;
        if (INITIAL) {
            y.x = y.y = y.z = (Real)0;
        } else {
            y.x = s.vh[j] - vxi;
            y.y = s.vh[n + j] - vyi;
            y.z = s.vh[2 * n + j] - vzi;
        }
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
    const Real fbi[3] = {a.fb[i], a.fb[n + i], a.fb[2 * n + i]};

    // the forward's tensor-core tests and sums (the same operands and
    // products as k_bond_tcw, so the same bits): warp w sums bonds 32w ..
    // 32w + 31 straight into their slots (K~ at kSlG, A~ at kSlAb, |S| at kSlCnt)
    bool use_tc = false;
    float tc_sT2 = 0.0f, tc_hf2s = 0.0f;
    if constexpr (!F64 && MODEL == 0) {
        use_tc = nb <= kTcRows;                                     // block-uniform
        if (use_tc) {
            float uK, uA, sT;
            tc_build_features<kAdjThreads>(s_z, s_y, nb, tc_phi, tc_tw, uK, uA, sT, s_tcs);
            tc_sT2 = sT * sT;
            tc_hf2s = k.hf2f * tc_sT2;
            if (32 * wid < nb)
                tc_pass_sums<kAdjSlots>(s_z, tc_tw, nb, wid, tc_sT2, tc_hf2s, tc_phi,
                                        s_b + (size_t)32 * wid * kAdjSlots + kSlG, uK, uA);
        }
    }

    // pass 1: sub-horizon sums, kept per bond
    Real wpart[1] = {(Real)0};
    Real kid1[6] = {0, 0, 0, 0, 0, 0};     // the thread's bond inverse, kept for pass 2 (use_tc)
    for (int t = threadIdx.x; t < nb; t += kAdjThreads) {
        const R4<Real> zj = s_z[t];
        const Real mjx = (Real)-2 * zj.x, mjy = (Real)-2 * zj.y, mjz = (Real)-2 * zj.z;
        const Real thj = hf2 - zj.w;   // the forward's test, the same rounding
        Real K00 = 0, K11 = 0, K22 = 0, K12 = 0, K02 = 0, K01 = 0;
        Real A00 = 0, A01 = 0, A02 = 0, A10 = 0, A11 = 0, A12 = 0, A20 = 0, A21 = 0, A22 = 0;
        int cnt = 0;
        if constexpr (F64 || MODEL == 1) {
            double pjx = 0, pjy = 0, pjz = 0;
            if constexpr (F64) { pjx = s_p[t]; pjy = s_p[kMaxRow + t]; pjz = s_p[2 * kMaxRow + t]; }
            for (int q = 0; q < nb; q++) {
                const R4<Real> zk = s_z[q];
                bool member = true;
                if constexpr (MODEL != 1) {
                    const double d0 = __dsub_rn(s_p[q], pjx);
                    const double d1 = __dsub_rn(s_p[kMaxRow + q], pjy);
                    const double d2 = __dsub_rn(s_p[2 * kMaxRow + q], pjz);
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
        } else if (use_tc) {
            const Real* sbt = s_b + (size_t)t * kAdjSlots;          // this warp's rows
            K00 = sbt[kSlG + 0]; K11 = sbt[kSlG + 1]; K22 = sbt[kSlG + 2];
            K12 = sbt[kSlG + 3]; K02 = sbt[kSlG + 4]; K01 = sbt[kSlG + 5];
            A00 = sbt[kSlAb + 0]; A01 = sbt[kSlAb + 1]; A02 = sbt[kSlAb + 2];
            A10 = sbt[kSlAb + 3]; A11 = sbt[kSlAb + 4]; A12 = sbt[kSlAb + 5];
            A20 = sbt[kSlAb + 6]; A21 = sbt[kSlAb + 7]; A22 = sbt[kSlAb + 8];
            cnt = small_count(sbt[kSlCnt]);
        } else {
            float Kf[6] = {0, 0, 0, 0, 0, 0}, Af[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            float cntf = 0.0f;
#pragma unroll 4
            for (int q = 0; q < nb; q++) {
                const R4<Real> zk = s_z[q];
                const R4<Real> yk = s_y[q];
                const float tst = member_test_lhs(zk.x, zk.y, zk.z, zk.w, mjx, mjy, mjz);
                masked_accumulate(tst, thj, zk.x, zk.y, zk.z, yk.x, yk.y, yk.z, Kf, Af, cntf);
            }
            K00 = Kf[0]; K11 = Kf[1]; K22 = Kf[2]; K12 = Kf[3]; K02 = Kf[4]; K01 = Kf[5];
            A00 = Af[0]; A01 = Af[1]; A02 = Af[2]; A10 = Af[3]; A11 = Af[4]; A12 = Af[5];
            A20 = Af[6]; A21 = Af[7]; A22 = Af[8];
            cnt = (int)cntf;
        }
        Real* sb = s_b + (size_t)t * kAdjSlots;
        sb[kSlG + 0] = K00; sb[kSlG + 1] = K11; sb[kSlG + 2] = K22;
        sb[kSlG + 3] = K12; sb[kSlG + 4] = K02; sb[kSlG + 5] = K01;
        sb[kSlAb + 0] = A00; sb[kSlAb + 1] = A01; sb[kSlAb + 2] = A02;
        sb[kSlAb + 3] = A10; sb[kSlAb + 4] = A11; sb[kSlAb + 5] = A12;
        sb[kSlAb + 6] = A20; sb[kSlAb + 7] = A21; sb[kSlAb + 8] = A22;
        Real Kid[6];
        bool active = cnt >= 3;
        if constexpr (F64) {
            const double Kd[6] = {K00, K11, K22, K12, K02, K01};
            active = active && inverse_sym_fp64(Kd, Kid);
        } else {
            active = active && inverse_sym_mixed(K00, K11, K22, K12, K02, K01, Kid);
        }
        sb[kSlCnt] = (Real)cnt;
        sb[kSlAct] = active ? (Real)1 : (Real)0;
        sb[kSlTest + 0] = mjx; sb[kSlTest + 1] = mjy; sb[kSlTest + 2] = mjz; sb[kSlTest + 3] = thj;
        if (active) wpart[0] += (Real)cnt * inv_nb;
        if (use_tc) {                       // at most one bond per thread
#pragma unroll
            for (int c = 0; c < 6; c++) kid1[c] = Kid[c];
        }
    }
    block_sum<1, Real>(wpart, reinterpret_cast<Real(*)[1]>(&s_red[0][0]));
    const Real w = wpart[0];

    // point adjoints of the state after the step
    Real Spt[9], sbi6[6];
#pragma unroll
    for (int c = 0; c < 6; c++) sbi6[c] = INITIAL ? (Real)0 : a.sb[c * n + i];
    six_to_full(sbi6, Spt);
    const Real pcpt = INITIAL ? (Real)0 : a.pcb[i];

    // pass 2: reverse of every active bond
    Real Sacc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    Real pcacc = 0;
    double Mb = 0.0, etab = 0.0, Srsb = 0.0;
    for (int t = threadIdx.x; t < nb; t += kAdjThreads) {
        Real* sb = s_b + (size_t)t * kAdjSlots;
        const bool active = sb[kSlAct] != (Real)0;
        const R4<Real> zj = s_z[t];
        Real Kid[6];
        if (active) {
            if (use_tc) {
#pragma unroll
                for (int c = 0; c < 6; c++) Kid[c] = kid1[c];
            } else if constexpr (F64) {
                const double Kd[6] = {sb[kSlG + 0], sb[kSlG + 1], sb[kSlG + 2],
                                      sb[kSlG + 3], sb[kSlG + 4], sb[kSlG + 5]};
                inverse_sym_fp64(Kd, Kid);
            } else {
                inverse_sym_mixed(sb[kSlG + 0], sb[kSlG + 1], sb[kSlG + 2], sb[kSlG + 3],
                                  sb[kSlG + 4], sb[kSlG + 5], Kid);
            }
        }
        Real G[6] = {0, 0, 0, 0, 0, 0}, Ab[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, zown[3] = {0, 0, 0};
        if (active) {
            const Real Ki[9] = {Kid[0], Kid[5], Kid[4], Kid[5], Kid[1], Kid[3], Kid[4], Kid[3], Kid[2]};
            const Real varpi = sb[kSlCnt] * inv_nb;
            const Real A[9] = {sb[kSlAb + 0], sb[kSlAb + 1], sb[kSlAb + 2], sb[kSlAb + 3], sb[kSlAb + 4],
                               sb[kSlAb + 5], sb[kSlAb + 6], sb[kSlAb + 7], sb[kSlAb + 8]};
            Real L[9];
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int c = 0; c < 3; c++)
                    L[r * 3 + c] = (A[r * 3 + 0] * Ki[0 * 3 + c] + A[r * 3 + 1] * Ki[1 * 3 + c] +
                                    A[r * 3 + 2] * Ki[2 * 3 + c]) * inv_dx;
            BondStress<Real> bs;
            MatTrace<Real> tr;
            if constexpr (INITIAL) {
#pragma unroll
                for (int c = 0; c < 6; c++) bs.sig[c] = sig_i[c];
            } else {
                material_update<Real>(L, sig_i, pc_i, k, cc.M, cc.Mf, bs, &tr);
            }
            const Real Sh[9] = {bs.sig[0] + Srs, bs.sig[5], bs.sig[4],
                                bs.sig[5], bs.sig[1] + Srs, bs.sig[3],
                                bs.sig[4], bs.sig[3], bs.sig[2] + Srs};
            // T^ = varpi Sh Ki zeta~_j; its adjoint from the gather
            const int j = s.col[r0 + t];
            Real Tb[3];
#pragma unroll
            for (int c = 0; c < 3; c++) Tb[c] = dx2 * (fbi[c] - a.fb[(size_t)c * n + j]);
            const Real zjv[3] = {zj.x, zj.y, zj.z};
            Real g[3], STb[3];
#pragma unroll
            for (int r = 0; r < 3; r++) {
                g[r] = Ki[r * 3 + 0] * zjv[0] + Ki[r * 3 + 1] * zjv[1] + Ki[r * 3 + 2] * zjv[2];
                STb[r] = Sh[0 * 3 + r] * Tb[0] + Sh[1 * 3 + r] * Tb[1] + Sh[2 * 3 + r] * Tb[2];
            }
            Real Sob[9], Kib[9];
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    Sob[r * 3 + c] = varpi * (Real)0.5 * (Tb[r] * g[c] + g[r] * Tb[c]);
                    Kib[r * 3 + c] = varpi * STb[r] * zjv[c];
                }
            Srsb += (double)(Sob[0] + Sob[4] + Sob[8]);
#pragma unroll
            for (int r = 0; r < 3; r++)
                zown[r] = varpi * (Ki[r * 3 + 0] * STb[0] + Ki[r * 3 + 1] * STb[1] + Ki[r * 3 + 2] * STb[2]);
            if constexpr (INITIAL) {
#pragma unroll
                for (int e = 0; e < 9; e++) Sacc[e] += Sob[e];
            } else {
                // point-state mean: sig' = sum varpi sig_b / w
                const Real vw = varpi / w;
#pragma unroll
                for (int e = 0; e < 9; e++) Sob[e] += vw * Spt[e];
                Real Lb[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
                material_reverse<Real>(tr, sig_i, pc_i, k, cc.M, Sob, vw * pcpt, Sacc, pcacc, Lb,
                                       Mb, etab);
                // L = A~ Ki / dx
#pragma unroll
                for (int r = 0; r < 3; r++)
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        Ab[r * 3 + c] = (Lb[r * 3 + 0] * Ki[c * 3 + 0] + Lb[r * 3 + 1] * Ki[c * 3 + 1] +
                                         Lb[r * 3 + 2] * Ki[c * 3 + 2]) * inv_dx;
                        Kib[r * 3 + c] += (A[0 * 3 + r] * Lb[0 * 3 + c] + A[1 * 3 + r] * Lb[1 * 3 + c] +
                                           A[2 * 3 + r] * Lb[2 * 3 + c]) * inv_dx;
                    }
                // Ki = K~^-1: K~-bar = -Ki Ki-bar Ki; G = K~-bar + K~-bar^T
                Real T1[9], Kb[9];
#pragma unroll
                for (int r = 0; r < 3; r++)
#pragma unroll
                    for (int c = 0; c < 3; c++)
                        T1[r * 3 + c] = Ki[r * 3 + 0] * Kib[0 * 3 + c] + Ki[r * 3 + 1] * Kib[1 * 3 + c] +
                                        Ki[r * 3 + 2] * Kib[2 * 3 + c];
#pragma unroll
                for (int r = 0; r < 3; r++)
#pragma unroll
                    for (int c = 0; c < 3; c++)
                        Kb[r * 3 + c] = -(T1[r * 3 + 0] * Ki[0 * 3 + c] + T1[r * 3 + 1] * Ki[1 * 3 + c] +
                                          T1[r * 3 + 2] * Ki[2 * 3 + c]);
                G[0] = (Real)2 * Kb[0]; G[1] = (Real)2 * Kb[4]; G[2] = (Real)2 * Kb[8];
                G[3] = Kb[5] + Kb[7]; G[4] = Kb[2] + Kb[6]; G[5] = Kb[1] + Kb[3];
            }
        }
        if constexpr (!INITIAL) {
            // sender data for the receiver pass (reuses the slots of the sums)
#pragma unroll
            for (int e = 0; e < 6; e++) sb[kSlG + e] = G[e];
#pragma unroll
            for (int e = 0; e < 9; e++) sb[kSlAb + e] = Ab[e];
        }
        sb[kSlZown + 0] = zown[0];
        sb[kSlZown + 1] = zown[1];
        sb[kSlZown + 2] = zown[2];
    }
    __syncthreads();

    Real zs[6] = {0, 0, 0, 0, 0, 0};   // sums over the row of the position / velocity adjoints
    if constexpr (!INITIAL) {
        // the tensor-core receiver sums: the senders' terms G, Ab (in their
        // slots after pass 2) as features, the forward's mask tiles transposed;
        // warp w writes the sums of receivers 32w .. 32w + 31 into their slots
        if constexpr (!F64 && MODEL == 0) {
            if (use_tc) {
                float uG, uAb;
                tc_build_adj_sender_features<kAdjThreads>(s_b + kSlG, kAdjSlots, nb, tc_phi, uG, uAb, s_tcs);
                if (32 * wid < nb)
                    tc_pass_receiver<4, kAdjSlots>(s_z, tc_tw, nb, wid, tc_sT2, tc_hf2s, tc_phi,
                                                   s_b + (size_t)32 * wid * kAdjSlots + kSlG, uG, uAb, 6, 15);
            }
        }
        // pass 3: receiver t gathers from every sender q whose sub-horizon holds
        // it: zeta~-bar += G zeta~_t + Ab^T Ydot_t and Ydot-bar += Ab zeta~_t,
        // with G and Ab first summed over those senders
        for (int t = threadIdx.x; t < nb; t += kAdjThreads) {
            const R4<Real> zt = s_z[t];
            const R4<Real> yt = s_y[t];
            const Real* sbt = s_b + (size_t)t * kAdjSlots;
            Real Gs[6] = {0, 0, 0, 0, 0, 0}, As[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            if (use_tc) {
#pragma unroll
                for (int e = 0; e < 6; e++) Gs[e] = sbt[kSlG + e];
#pragma unroll
                for (int e = 0; e < 9; e++) As[e] = sbt[kSlAb + e];
            } else if constexpr (!F64 && MODEL != 1) {
                // the sender's own membership test, same operands and rounding
                float Gf[6] = {0, 0, 0, 0, 0, 0}, Af[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll 2
                for (int q = 0; q < nb; q++) {
                    const float* sq = s_b + (size_t)q * kAdjSlots;
                    // rows are 25 floats apart: scalar loads (every thread reads the same row)
                    const float4 m = make_float4(sq[kSlTest], sq[kSlTest + 1], sq[kSlTest + 2], sq[kSlTest + 3]);
                    const float4 g0 = make_float4(sq[4], sq[5], sq[6], sq[7]);
                    const float4 g1 = make_float4(sq[8], sq[9], sq[10], sq[11]);
                    const float4 g2 = make_float4(sq[12], sq[13], sq[14], sq[15]);
                    const float4 g3 = make_float4(sq[16], sq[17], sq[18], sq[19]);
                    const float tst = member_test_lhs(zt.x, zt.y, zt.z, zt.w, m.x, m.y, m.z);
                    masked_add15(tst, m.w, g0, g1, g2, g3, Gf, Af);
                }
#pragma unroll
                for (int e = 0; e < 6; e++) Gs[e] = Gf[e];
#pragma unroll
                for (int e = 0; e < 9; e++) As[e] = Af[e];
            } else {
                for (int q = 0; q < nb; q++) {
                    const Real* sq = s_b + (size_t)q * kAdjSlots;
                    bool member = true;
                    if constexpr (MODEL != 1) {
                        const double d0 = __dsub_rn(s_p[t], s_p[q]);
                        const double d1 = __dsub_rn(s_p[kMaxRow + t], s_p[kMaxRow + q]);
                        const double d2 = __dsub_rn(s_p[2 * kMaxRow + t], s_p[2 * kMaxRow + q]);
                        member = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)),
                                           __dmul_rn(d2, d2)) <= k.delta2;
                    }
                    if (member) {
#pragma unroll
                        for (int e = 0; e < 6; e++) Gs[e] += sq[kSlG + e];
#pragma unroll
                        for (int e = 0; e < 9; e++) As[e] += sq[kSlAb + e];
                    }
                }
            }
            // G holds (00, 11, 22, 12, 02, 01); Ab is row-major
            Real Zb[3] = {sbt[kSlZown + 0], sbt[kSlZown + 1], sbt[kSlZown + 2]};
            Zb[0] += Gs[0] * zt.x + Gs[5] * zt.y + Gs[4] * zt.z + As[0] * yt.x + As[3] * yt.y + As[6] * yt.z;
            Zb[1] += Gs[5] * zt.x + Gs[1] * zt.y + Gs[3] * zt.z + As[1] * yt.x + As[4] * yt.y + As[7] * yt.z;
            Zb[2] += Gs[4] * zt.x + Gs[3] * zt.y + Gs[2] * zt.z + As[2] * yt.x + As[5] * yt.y + As[8] * yt.z;
            Real Yb[3];
            Yb[0] = As[0] * zt.x + As[1] * zt.y + As[2] * zt.z;
            Yb[1] = As[3] * zt.x + As[4] * zt.y + As[5] * zt.z;
            Yb[2] = As[6] * zt.x + As[7] * zt.y + As[8] * zt.z;
            // zeta~ = (x_k - x_i) / dx: position adjoint of the neighbour
#pragma unroll
            for (int c = 0; c < 3; c++) Zb[c] *= inv_dx;
            const int rb = s.rev[r0 + t];
            if (rb >= 0) {
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    a.Zrev[(size_t)c * k.cap + rb] = Zb[c];
                    a.Yrev[(size_t)c * k.cap + rb] = Yb[c];
                }
            }
#pragma unroll
            for (int c = 0; c < 3; c++) {
                zs[c] += Zb[c];
                zs[3 + c] += Yb[c];
            }
        }
    }
    // block sums: stress adjoint (9), pc adjoint, row sums (6)
    Real red[16];
#pragma unroll
    for (int e = 0; e < 9; e++) red[e] = Sacc[e];
    red[9] = pcacc;
#pragma unroll
    for (int e = 0; e < 6; e++) red[10 + e] = zs[e];
    block_sum<16, Real>(red, s_red);
    double dred[3] = {Mb, etab, Srsb};
    block_sum<3, double>(dred, reinterpret_cast<double(*)[3]>(&s_redd[0][0]));
    if (threadIdx.x == 0) {
        Real o6[6];
        full_to_six(red, o6);
        if constexpr (INITIAL) {
#pragma unroll
            for (int c = 0; c < 6; c++) a.sbn[c * n + i] = a.sb[c * n + i] + o6[c];
            a.pcbn[i] = a.pcb[i];
        } else {
            const bool pass = !(w > (Real)0);     // no active bond: the state is unchanged
#pragma unroll
            for (int c = 0; c < 6; c++) a.sbn[c * n + i] = o6[c] + (pass ? sbi6[c] : (Real)0);
            a.pcbn[i] = red[9] + (pass ? pcpt : (Real)0);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                a.zsum[c * n + i] = red[10 + c];
                a.ysum[c * n + i] = red[13 + c];
            }
        }
        a.thpart[(size_t)i * 3 + 0] = dred[0];
        a.thpart[(size_t)i * 3 + 1] = dred[1];
        a.thpart[(size_t)i * 3 + 2] = dred[2];
    }
}

// neighbours' position and velocity adjoints gathered over the row (rev
// slots), then the reverse of the predictor u' = u + dt vh, vh = v + dt/2 a
template <typename Real>
__global__ void __launch_bounds__(kWarpPointsPerBlock * 32)
k_adj_post(DevState<Real> s, AdjState<Real> a, StepConst k) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int i = blockIdx.x * kWarpPointsPerBlock + wib;
    if (i >= k.npoints) return;
    const size_t n = (size_t)k.npoints;
    const Real dt = sizeof(Real) == 8 ? (Real)k.dt : (Real)k.dtf;
    const Real h = (Real)0.5 * dt;
    const int r0 = s.row_ptr[i], r1 = s.row_ptr[i + 1];
    Real z[6] = {0, 0, 0, 0, 0, 0};
    for (int b = r0 + lane; b < r1; b += 32)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            z[c] += a.Zrev[(size_t)c * k.cap + b];
            z[3 + c] += a.Yrev[(size_t)c * k.cap + b];
        }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int e = 0; e < 6; e++) z[e] += __shfl_xor_sync(0xffffffffu, z[e], off);
    if (lane < 3) {
        const int c = lane;
        const size_t t = (size_t)c * n + i;
        const Real gz = c == 0 ? z[0] : (c == 1 ? z[1] : z[2]);
        const Real gy = c == 0 ? z[3] : (c == 1 ? z[4] : z[5]);
        const Real u1b = a.u1b[t] + gz - a.zsum[t];
        const Real vhb = a.vhb[t] + gy - a.ysum[t] + dt * u1b;
        Real vbar;
        const bool fixed = prescribed(s, k, (size_t)i, c, vbar);
        a.ub[t] = u1b;
        a.vb[t] = fixed ? (Real)0 : vhb;
        a.ab[t] = fixed ? (Real)0 : h * vhb;
    }
    if (lane < 6) {
        a.sb[(size_t)lane * n + i] = a.sbn[(size_t)lane * n + i];
        if (lane == 0) a.pcb[i] = a.pcbn[i];
    }
}

// deterministic sums: acc[0..2] += sum over points of thpart; when
// with_state (after the initial pass), acc[3] = sum tr(sigma0-bar) and
// acc[4] = sum pc0-bar
// per-step sums of the parameter partials (and, for the initial pass, of
// the state adjoints): a fixed chunk of points per block, then the blocks'
// partials in order, so the result does not depend on scheduling
template <typename Real>
__global__ void __launch_bounds__(256)
k_adj_reduce_part(AdjState<Real> a, int npoints, double* part, int with_state) {
    __shared__ double sm[5][256];
    double t[5] = {0, 0, 0, 0, 0};
    const size_t n = (size_t)npoints;
    const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const size_t p0 = (size_t)blockIdx.x * chunk;
    const size_t p1 = p0 + chunk < n ? p0 + chunk : n;
    for (size_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        for (int e = 0; e < 3; e++) t[e] += a.thpart[p * 3 + e];
        if (with_state) {
            t[3] += (double)a.sbn[p] + (double)a.sbn[n + p] + (double)a.sbn[2 * n + p];
            t[4] += (double)a.pcbn[p];
        }
    }
    for (int e = 0; e < 5; e++) sm[e][threadIdx.x] = t[e];
    __syncthreads();
    for (int wdt = blockDim.x / 2; wdt > 0; wdt >>= 1) {
        if ((int)threadIdx.x < wdt)
            for (int e = 0; e < 5; e++) sm[e][threadIdx.x] += sm[e][threadIdx.x + wdt];
        __syncthreads();
    }
    if (threadIdx.x < 5) part[(size_t)blockIdx.x * 5 + threadIdx.x] = sm[threadIdx.x][0];
}

__global__ void k_adj_reduce_final(const double* part, int nparts, double* acc, int with_state) {
    const int e = threadIdx.x;
    if (e >= 5) return;
    double t = 0.0;
    for (int b = 0; b < nparts; b++) t += part[(size_t)b * 5 + e];
    if (e < 3) acc[e] += t;
    else if (with_state) acc[e] = t;
}

template <typename Real>
__global__ void k_convert_adjoint(const double* src, Real* dst, size_t count) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count;
         t += (size_t)gridDim.x * blockDim.x)
        dst[t] = (Real)src[t];
}

}  // namespace

template <typename Real>
cudaError_t launch_adjoint_step(const DevState<Real>& s, const AdjState<Real>& a, const StepConst& k,
                                double* acc, int initial, cudaStream_t st) {
    const int n = k.npoints;
    const size_t work = 3 * (size_t)n;
    const int pblocks = (int)((work + 255) / 256 < 65536 ? (work + 255) / 256 : 65536);
    k_adj_pre<Real><<<pblocks > 0 ? pblocks : 1, 256, 0, st>>>(s, a, k, initial);
    const size_t smem = adj_smem_bytes<Real>();
    cudaError_t e;
#define PPM_ADJ(M, I)                                                                      \
    e = cudaFuncSetAttribute(k_adj_bond<Real, M, I>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)smem);                                                   \
    if (e != cudaSuccess) return e;                                                        \
    k_adj_bond<Real, M, I><<<n, kAdjThreads, smem, st>>>(s, a, k)
    if (initial) {
        if (k.model == 1) { PPM_ADJ(1, true); } else { PPM_ADJ(0, true); }
    } else {
        if (k.model == 1) { PPM_ADJ(1, false); } else { PPM_ADJ(0, false); }
        k_adj_post<Real><<<(n + kWarpPointsPerBlock - 1) / kWarpPointsPerBlock,
                           kWarpPointsPerBlock * 32, 0, st>>>(s, a, k);
    }
#undef PPM_ADJ
    double* part = acc + kAdjAccDoubles;
    k_adj_reduce_part<Real><<<kAdjRedBlocks, 256, 0, st>>>(a, n, part, initial);
    k_adj_reduce_final<<<1, 32, 0, st>>>(part, kAdjRedBlocks, acc, initial);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_convert_adjoint(const double* src, Real* dst, size_t count, cudaStream_t st) {
    const int blocks = (int)((count + 255) / 256 < 65536 ? (count + 255) / 256 : 65536);
    k_convert_adjoint<Real><<<blocks > 0 ? blocks : 1, 256, 0, st>>>(src, dst, count);
    return cudaGetLastError();
}

template cudaError_t launch_adjoint_step<double>(const DevState<double>&, const AdjState<double>&,
                                                 const StepConst&, double*, int, cudaStream_t);
template cudaError_t launch_adjoint_step<float>(const DevState<float>&, const AdjState<float>&,
                                                const StepConst&, double*, int, cudaStream_t);
template cudaError_t launch_convert_adjoint<double>(const double*, double*, size_t, cudaStream_t);
template cudaError_t launch_convert_adjoint<float>(const double*, float*, size_t, cudaStream_t);

}  // namespace ppm
