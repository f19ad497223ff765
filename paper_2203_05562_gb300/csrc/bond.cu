// The per-step kernels of the explicit bond loop:
//   k_predictor  -- Newmark predictor, boundary conditions, displacement
//                   (Eq. 60-61, 64; the predictor of Alg. 2)
//   k_bond       -- fused per-point kernel: sub-horizon membership and sums
//                   (Eq. 22-25, 55, 57), FP64 shape-tensor inverse, velocity
//                   gradient, rate of deformation and spin (Eq. 26),
//                   Hughes-Winget rotation, linear trial stress (Eq. 41),
//                   critical-state Perzyna return in FP64 (Eq. 40-46,
//                   70-76), force state (Eq. 31-32, 51; or the standard and
//                   power-conjugate forms) with the repulsion between points
//                   closer than delta_c (Eq. 91), and the point-state
//                   reduction; Alg. 1 up to the force state.  A separate
//                   instantiation carries the coupled mode (Eq. 15-16,
//                   48-49: per-point volume ratio, saturation and volumes).
//                   Under plane strain the bond vectors take the nearest
//                   periodic image in y at staging
//   k_gather     -- deterministic pairwise nodal force (Eq. 49-50), the
//                   substrate's normal force and friction (Eq. 91-93), the
//                   acceleration and velocity corrector (Eq. 62-63) and the
//                   energy increments (Eq. 66-68); the force assembly of Alg. 1
//   k_energy_reduce -- the Eq. 69 check as a status bit or a hard stop
//
// Scaled variables: bond vectors are carried in lattice units
// zeta~ = zeta / dx, the shape tensor as K~ = sum zeta~ zeta~^T (the paper's
// K = V dx^2 K~), and the stored force state as T^ = varpi sigma K~^-1
// zeta~ (the paper's T = T^ / (V dx)), so that FP32 stays far from its
// range limits at every lattice spacing.  Then L = (sum Ydot zeta~^T)
// K~^-1 / dx and the nodal force is f = dx^2 (sum T^ - sum T^').
#include <cuda_runtime.h>
#include <math.h>

#include "bond_device.cuh"
#include "ppm_internal.cuh"

namespace ppm {
namespace {


// ---------------------------------------------------------------------------
// predictor (Eq. 60-61, 64 with beta1 = 1/2, beta2 = 0)
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void k_predictor(DevState<Real> s, StepConst k) {
    if (k.halt && (s.ctr->status & PPM_STATUS_HALTED)) return;   // the run has stopped
    const size_t n = (size_t)k.npoints;
    const Real dt = (Real)k.dt, hdt = (Real)(0.5 * k.dt);
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < 3 * n;
         t += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / n);
        const size_t i = t - (size_t)c * n;
        Real v = s.v[t] + hdt * s.a[t], vbar;
        if (prescribed(s, k, i, c, vbar)) v = vbar;
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
// The update of one bond (i, j) after its sub-horizon sums (the part of
// Alg. 1 after the sub-horizon loop): FP64 inverse of the shape tensor
// (Eq. 23, 25), velocity gradient (Eq. 25, 57), constitutive update (Sec.
// 2.3), force state (Eq. 31-32, 51; model 2: the sender matrix in sM) and
// the bond's share of the point-state reduction (red).  b: the bond's row
// slot, rb: its reverse slot, zj: its vector (lattice units, |.|^2), Jj:
// the member's volume ratio (coupled mode), K (xx yy zz yz xz xy), A (row-
// major) and cntr = |S_b| its sums, (mjx, mjy, mjz, thj): the terms of its
// membership test, park: a 16-entry row the thread owns (FP32 path).
template <typename Real, int MODEL, bool CPL, int NRED, int SMW = 16>
__device__ __forceinline__ void bond_epilogue(
    const DevState<Real>& s, const StepConst& k, int i, int r0, int t, int rb, const R4<Real>& zj,
    Real Jj, Real K00, Real K11, Real K22, Real K12, Real K02, Real K01, Real A00, Real A01,
    Real A02, Real A10, Real A11, Real A12, Real A20, Real A21, Real A22, Real cntr, int cnt,
    Real mjx, Real mjy, Real mjz, Real thj, const Real (&sig_i)[6], Real pc_i,
    const ColumnConst& cc, Real Srs, Real inv_nb, Real inv_dx, int with_dt, Real* park, Real* sM,
    Real (&red)[NRED], unsigned& n_pairs, unsigned& n_plastic, unsigned& n_nonconv,
    unsigned& n_singular, unsigned& n_ret64) {
    constexpr bool F64 = sizeof(Real) == 8;
    n_pairs += (unsigned)cnt;
    // shape-tensor inverse (Eq. 23, 25): FP64 on the FP64 path; the mixed
    // path keeps FP64 for the determinant (inverse_sym_mixed)
    Real Kid[6];
    bool active = cntr >= (Real)3;
    if constexpr (F64) {
        const double Kd[6] = {K00, K11, K22, K12, K02, K01};
        active = active && inverse_sym_fp64(Kd, Kid);
    } else {
        active = active && inverse_sym_mixed(K00, K11, K22, K12, K02, K01, Kid);
    }
    if (!active) {
        n_singular++;
        if constexpr (MODEL != 2) {
            Real o[3];
            store_force_state<CPL>(s, k, (size_t)r0 + t, rb, (Real)0, (Real)0, (Real)0, zj,
                              Jj, CPL ? s.J[i] : (Real)1, o);
            red[9] += o[0]; red[10] += o[1]; red[11] += o[2];
        } else {
#pragma unroll
            for (int e = 0; e < 9; e++) sM[e] = (Real)0;
            if constexpr (!F64 && SMW >= 13) {
                sM[9] = mjx; sM[10] = mjy; sM[11] = mjz; sM[12] = thj;
            }
        }
        return;
    }
    Real Ki[9] = {(Real)Kid[0], (Real)Kid[5], (Real)Kid[4],
                  (Real)Kid[5], (Real)Kid[1], (Real)Kid[3],
                  (Real)Kid[4], (Real)Kid[3], (Real)Kid[2]};
    Real varpi = cntr * inv_nb;                         // Eq. 55
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
        if constexpr (CPL) red[NRED - 1] += varpi * (L[0] + L[4] + L[8]) * (F64 ? (Real)k.dt : (Real)k.dtf);
        Real st[6], des;
        if (material_trial<Real>(L, sig_i, pc_i, k, cc.M, cc.Mf, st, des)) {
            if constexpr (!F64) {
                // the bond waits in shared memory while the return runs, so
                // that none of it is held in registers across the return's
                // calls (the compiler barriers keep it from being forwarded)
                Real* pk = (MODEL == 2 && SMW >= 14) ? sM : park;
#pragma unroll
                for (int c = 0; c < 6; c++) pk[c] = st[c];
#pragma unroll
                for (int c = 0; c < 6; c++) pk[6 + c] = Kid[c];
                pk[12] = varpi;
                pk[13] = des;
                asm volatile("" ::: "memory");
                Real stp[6];
#pragma unroll
                for (int c = 0; c < 6; c++) stp[c] = pk[c];
                material_return<Real>(stp, pc_i, k, cc.M, cc.Mf, bs);
                asm volatile("" ::: "memory");
                const Real* q = (MODEL == 2 && SMW >= 14) ? sM : park;
                Ki[0] = q[6]; Ki[1] = q[11]; Ki[2] = q[10];
                Ki[3] = q[11]; Ki[4] = q[7]; Ki[5] = q[9];
                Ki[6] = q[10]; Ki[7] = q[9]; Ki[8] = q[8];
                varpi = q[12];
                bs.des = q[13];
            } else {
                material_return<Real>(st, pc_i, k, cc.M, cc.Mf, bs);
                bs.des = des;
            }
            n_plastic++;
            n_nonconv += bs.nonconv;
            n_ret64 += bs.ret64;
        } else {
#pragma unroll
            for (int c = 0; c < 6; c++) bs.sig[c] = st[c];
            bs.pc = pc_i;
            bs.des = des;
        }
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
    Real SK[9];          // varpi S K^-1 (the FP64 path's force state; model 2's sender matrix)
    if constexpr (MODEL == 2 || sizeof(Real) == 8) {
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int c = 0; c < 3; c++)
                SK[r * 3 + c] = varpi * (S[r * 3 + 0] * Ki[0 * 3 + c] + S[r * 3 + 1] * Ki[1 * 3 + c] +
                                         S[r * 3 + 2] * Ki[2 * 3 + c]);
    }
    if constexpr (MODEL != 2) {
        // force state on the bond itself (Eq. 31-32, 51)
        Real T0, T1, T2;
        if constexpr (sizeof(Real) == 8) {
            T0 = SK[0] * zj.x + SK[1] * zj.y + SK[2] * zj.z;
            T1 = SK[3] * zj.x + SK[4] * zj.y + SK[5] * zj.z;
            T2 = SK[6] * zj.x + SK[7] * zj.y + SK[8] * zj.z;
        } else {
            // mixed path: T = varpi S (K^-1 zeta~), 18 products instead of 36
            const Real y0 = Ki[0] * zj.x + Ki[1] * zj.y + Ki[2] * zj.z;
            const Real y1 = Ki[3] * zj.x + Ki[4] * zj.y + Ki[5] * zj.z;
            const Real y2 = Ki[6] * zj.x + Ki[7] * zj.y + Ki[8] * zj.z;
            T0 = varpi * (S[0] * y0 + S[1] * y1 + S[2] * y2);
            T1 = varpi * (S[3] * y0 + S[4] * y1 + S[5] * y2);
            T2 = varpi * (S[6] * y0 + S[7] * y1 + S[8] * y2);
        }
        Real o[3];
        store_force_state<CPL>(s, k, (size_t)r0 + t, rb, T0, T1, T2, zj, Jj, CPL ? s.J[i] : (Real)1, o);
        red[9] += o[0]; red[10] += o[1]; red[11] += o[2];
    } else {
#pragma unroll
        for (int e = 0; e < 9; e++) sM[e] = SK[e];
        if constexpr (!F64 && SMW >= 13) {
            sM[9] = mjx; sM[10] = mjy; sM[11] = mjz; sM[12] = thj;
        }
    }
    red[0] += varpi;
#pragma unroll
    for (int c = 0; c < 6; c++) red[1 + c] += varpi * bs.sig[c];
    red[7] += varpi * bs.pc;
    red[8] += varpi * bs.des;
}

// The point's new state (the varpi-weighted means of its bonds, reading R8),
// its row sum of force states and the step's counters, written by one
// thread (red and cnts are sums over the point's bonds).
template <typename Real, bool CPL, int NRED>
__device__ __forceinline__ void point_commit(const DevState<Real>& s, int i, size_t n,
                                             const Real (&red)[NRED], Real w, Real eps_i,
                                             const unsigned (&cnts)[5], int update) {
    {
        if (update && w > (Real)0) {
            const Real iw = (Real)1 / w;
#pragma unroll
            for (int c = 0; c < 6; c++) s.sig[c * n + i] = red[1 + c] * iw;
            s.pc[i] = red[7] * iw;
            s.eps[i] = eps_i + red[8] * iw;
        }
        // coupled mode: J_{n+1} = J_n exp(varpi-mean of dt tr L_b)
        if constexpr (CPL)
            if (update) s.Jn[i] = w > (Real)0 ? s.J[i] * exp(red[NRED - 1] / w) : s.J[i];
        s.tsum[i] = red[9];
        s.tsum[n + i] = red[10];
        s.tsum[2 * n + i] = red[11];
        // only committed passes count (not the initial pass or the autotuner's)
        if (update && cnts[3]) atomicAdd(&s.ctr->pairs, (unsigned long long)cnts[3]);
        if (update && cnts[0]) atomicAdd(&s.ctr->plastic, (unsigned long long)cnts[0]);
        if (update && cnts[4]) atomicAdd(&s.ctr->ret64, (unsigned long long)cnts[4]);
        if (update && cnts[1]) {
            atomicAdd(&s.ctr->nonconv, (unsigned long long)cnts[1]);
            atomicOr(&s.ctr->status, PPM_STATUS_NONCONV);
        }
        if (update && cnts[2]) {
            atomicAdd(&s.ctr->singular, (unsigned long long)cnts[2]);
            atomicOr(&s.ctr->status, PPM_STATUS_SINGULAR);
        }
    }
}

// ---------------------------------------------------------------------------
// fused bond kernel: one CTA per point, one thread per bond
// ---------------------------------------------------------------------------
// TPP threads per point (a tile the autotuner picks among 32, 64, 128, 256); the
// register budget targets 640 resident threads per SM for FP32.  CPL: the
// coupled mode (per-point volume ratio, saturation and volumes), a separate
// instantiation so that the other modes carry none of it
template <typename Real, int MODEL, int TPP, bool CPL>
__device__ __forceinline__ void bond_point(const DevState<Real>& s, const StepConst& k, const int i,
                                           int with_dt, int update) {
    constexpr bool F64 = sizeof(Real) == 8;
    constexpr int NW = TPP / 32;
    // a block that takes several points in turn: the previous one is done
    // with the shared arrays
    __syncthreads();
    __shared__ R4<Real> s_z[kMaxRow];                         // zeta~_k, lattice units
    __shared__ R4<Real> s_y[kMaxRow];                         // Ydot_k, m/s
    __shared__ double s_p[F64 ? 3 : 1][F64 ? kMaxRow : 1];    // FP64: absolute x_k
    // model 2: per sender bond, its matrix M = varpi sigma K^-1 (9), and (FP32) the
    // terms of its membership test, -2 zeta~ (3) and |zeta~|^2 - hf^2 (1)
    __shared__ alignas(16) Real s_M[MODEL == 2 ? kMaxRow : 1][F64 ? 9 : 16];
    // per-point sums (see red below): 12, and the volumetric increment in the coupled mode
    constexpr int NRED = CPL ? 13 : 12;
    __shared__ Real s_red[NW][NRED];
    __shared__ unsigned s_cnt[NW][5];
    // FP32 path: a plastic bond's trial stress, K~^-1, varpi and strain
    // measure, parked by its thread while the return runs (model 2 parks in
    // the bond's own row of s_M, which is written only after the return)
    __shared__ alignas(16) Real s_park[(F64 || MODEL == 2) ? 1 : TPP][16];

    const size_t n = (size_t)k.npoints;
    const int r0 = s.row_ptr[i];
    int nb = s.row_ptr[i + 1] - r0;
    if (nb > kMaxRow) nb = 0;
    const int li = s.lat[i];
    const int ix = lat_x(li), iy = lat_y(li), iz = lat_z(li);
    const Real inv_dx = F64 ? (Real)k.inv_dx : (Real)k.inv_dxf;
    // the point's state and column constants, issued before the family
    // gathers so that their latencies overlap
    Real sig_i[6];
#pragma unroll
    for (int c = 0; c < 6; c++) sig_i[c] = s.sig[c * n + i];
    const Real pc_i = s.pc[i];
    const Real eps_i = s.eps[i];
    const ColumnConst cc = s.cols[s.colid[i]];
    Real Srs = F64 ? (Real)cc.Srs : (Real)cc.Srsf;
    // coupled mode: S_r of the point's volume ratio at the start of the step
    if constexpr (CPL) {
        Real mass_unused;
        coupled_point<Real>(k, s.J[i], Srs, mass_unused);
    }

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
            double py = __dadd_rn(__dmul_rn((double)lat_y(lj), k.dx), (double)s.u[n + j]);
            const int sh = image_shift(k, lj, li);     // plane strain: nearest image
            if (sh) py = __dadd_rn(py, (double)sh * k.pbc_L);
            const double pz = __dadd_rn(__dmul_rn((double)lat_z(lj), k.dx), (double)s.u[2 * n + j]);
            s_p[0][t] = px; s_p[F64 ? 1 : 0][t] = py; s_p[F64 ? 2 : 0][t] = pz;
            z.x = (Real)((px - pxi) * k.inv_dx);
            z.y = (Real)((py - pyi) * k.inv_dx);
            z.z = (Real)((pz - pzi) * k.inv_dx);
        } else {
            z.x = small_float(lat_x(lj) - ix) + (s.u[j] - uxi) * inv_dx;
            z.y = small_float(lat_y(lj) - iy + image_shift(k, lj, li) * k.pbc_ny) + (s.u[n + j] - uyi) * inv_dx;
            z.z = small_float(lat_z(lj) - iz) + (s.u[2 * n + j] - uzi) * inv_dx;
        }
        z.w = z.x * z.x + z.y * z.y + z.z * z.z;
        y.x = s.vh[j] - vxi;
        y.y = s.vh[n + j] - vyi;
        y.z = s.vh[2 * n + j] - vzi;
        y.w = CPL ? s.J[j] : (Real)0;                // the member's volume ratio
        s_z[t] = z;
        s_y[t] = y;
    }
    __syncthreads();

    const Real hf2 = (Real)k.hf2f;
    const Real inv_nb = nb > 0 ? (Real)1 / (Real)nb : (Real)0;

    // per-thread partial sums over its bonds (fixed order)
    // red: sum varpi, varpi sigma (6), varpi pc, varpi deps_s, row sum of T
    // (3), and in the coupled mode varpi dt tr L
    Real red[NRED];
#pragma unroll
    for (int e = 0; e < NRED; e++) red[e] = (Real)0;
    unsigned n_plastic = 0, n_nonconv = 0, n_singular = 0, n_pairs = 0, n_ret64 = 0;

    if constexpr (MODEL == 1) {
        // standard correspondence (Sec. 2.1): every bond's sub-horizon is the
        // whole family, so K~, A~, L, the updated stress and the force-state
        // matrix belong to the point.  Each warp sums the family with its 32
        // lanes (lane l takes members l, l + 32, ...) and a butterfly, which
        // leaves the same bits in every lane of every warp whatever the tile;
        // every thread then applies the point's result to its bonds.
        Real Ks[15] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int q = (int)(threadIdx.x & 31); q < nb; q += 32) {
            const R4<Real> zk = s_z[q];
            const R4<Real> yk = s_y[q];
            Ks[0] += zk.x * zk.x; Ks[1] += zk.y * zk.y; Ks[2] += zk.z * zk.z;
            Ks[3] += zk.y * zk.z; Ks[4] += zk.x * zk.z; Ks[5] += zk.x * zk.y;
            Ks[6] += yk.x * zk.x; Ks[7] += yk.x * zk.y; Ks[8] += yk.x * zk.z;
            Ks[9] += yk.y * zk.x; Ks[10] += yk.y * zk.y; Ks[11] += yk.y * zk.z;
            Ks[12] += yk.z * zk.x; Ks[13] += yk.z * zk.y; Ks[14] += yk.z * zk.z;
        }
#pragma unroll
        for (int e = 0; e < 15; e++)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) Ks[e] += __shfl_xor_sync(0xffffffffu, Ks[e], off);
        const Real K00 = Ks[0], K11 = Ks[1], K22 = Ks[2], K12 = Ks[3], K02 = Ks[4], K01 = Ks[5];
        const Real A00 = Ks[6], A01 = Ks[7], A02 = Ks[8], A10 = Ks[9], A11 = Ks[10], A12 = Ks[11];
        const Real A20 = Ks[12], A21 = Ks[13], A22 = Ks[14];
        const int cnt = nb;
        Real Kid[6];
        bool active = cnt >= 3;
        if constexpr (F64) {
            const double Kd[6] = {K00, K11, K22, K12, K02, K01};
            active = active && inverse_sym_fp64(Kd, Kid);
        } else {
            active = active && inverse_sym_mixed(K00, K11, K22, K12, K02, K01, Kid);
        }
        const Real varpi = (Real)cnt * inv_nb;              // Eq. 55 (= 1)
        BondStress<Real> bs;
        bs.plastic = 0; bs.nonconv = 0; bs.ret64 = 0;
        Real SK[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        Real ev = (Real)0;                                  // dt tr L of the point (CPL)
        if (active) {
            const Real Ki[9] = {(Real)Kid[0], (Real)Kid[5], (Real)Kid[4],
                                (Real)Kid[5], (Real)Kid[1], (Real)Kid[3],
                                (Real)Kid[4], (Real)Kid[3], (Real)Kid[2]};
            if (with_dt) {
                const Real A[9] = {A00, A01, A02, A10, A11, A12, A20, A21, A22};
                Real L[9];
#pragma unroll
                for (int r = 0; r < 3; r++)
#pragma unroll
                    for (int c = 0; c < 3; c++)
                        L[r * 3 + c] = (A[r * 3 + 0] * Ki[0 * 3 + c] + A[r * 3 + 1] * Ki[1 * 3 + c] +
                                        A[r * 3 + 2] * Ki[2 * 3 + c]) * inv_dx;
                if constexpr (CPL) ev = (L[0] + L[4] + L[8]) * (F64 ? (Real)k.dt : (Real)k.dtf);
                Real st[6], des;
                if (material_trial<Real>(L, sig_i, pc_i, k, cc.M, cc.Mf, st, des)) {
                    material_return<Real>(st, pc_i, k, cc.M, cc.Mf, bs);
                    bs.des = des;
                } else {
#pragma unroll
                    for (int c = 0; c < 6; c++) bs.sig[c] = st[c];
                    bs.pc = pc_i;
                    bs.des = des;
                }
            } else {
#pragma unroll
                for (int c = 0; c < 6; c++) bs.sig[c] = sig_i[c];
                bs.pc = pc_i;
                bs.des = (Real)0;
            }
            const Real S[9] = {bs.sig[0] + Srs, bs.sig[5], bs.sig[4],
                               bs.sig[5], bs.sig[1] + Srs, bs.sig[3],
                               bs.sig[4], bs.sig[3], bs.sig[2] + Srs};
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int c = 0; c < 3; c++)
                    SK[r * 3 + c] = varpi * (S[r * 3 + 0] * Ki[0 * 3 + c] + S[r * 3 + 1] * Ki[1 * 3 + c] +
                                             S[r * 3 + 2] * Ki[2 * 3 + c]);
        }
        for (int t = threadIdx.x; t < nb; t += TPP) {
            const int rb = s.rev[r0 + t];
            n_pairs += cnt;
            if (!active) {
                n_singular++;
                Real o[3];
                store_force_state<CPL>(s, k, (size_t)r0 + t, rb, (Real)0, (Real)0, (Real)0, s_z[t],
                                  s_y[t].w, CPL ? s.J[i] : (Real)1, o);
                red[9] += o[0]; red[10] += o[1]; red[11] += o[2];
                continue;
            }
            n_plastic += bs.plastic;
            n_nonconv += bs.nonconv;
            n_ret64 += bs.ret64;
            const R4<Real> zj = s_z[t];
            const Real T0 = SK[0] * zj.x + SK[1] * zj.y + SK[2] * zj.z;
            const Real T1 = SK[3] * zj.x + SK[4] * zj.y + SK[5] * zj.z;
            const Real T2 = SK[6] * zj.x + SK[7] * zj.y + SK[8] * zj.z;
            Real o[3];
            store_force_state<CPL>(s, k, (size_t)r0 + t, rb, T0, T1, T2, zj, s_y[t].w, CPL ? s.J[i] : (Real)1, o);
            red[9] += o[0]; red[10] += o[1]; red[11] += o[2];
            if constexpr (CPL) red[NRED - 1] += varpi * ev;
            red[0] += varpi;
#pragma unroll
            for (int c = 0; c < 6; c++) red[1 + c] += varpi * bs.sig[c];
            red[7] += varpi * bs.pc;
            red[8] += varpi * bs.des;
        }
    } else {
    for (int t = threadIdx.x; t < nb; t += TPP) {
        const R4<Real> zj = s_z[t];
        // the bond's reverse slot, loaded now so that its latency is hidden by the sums
        int rb = -1;
        if constexpr (MODEL != 2) rb = s.rev[r0 + t];
        // mixed-path test |z_k - z_j|^2 <= hf^2 as
        // |z_k|^2 - 2 z_k.z_j <= hf^2 - |z_j|^2 (threshold thj per bond)
        const Real mjx = (Real)-2 * zj.x, mjy = (Real)-2 * zj.y, mjz = (Real)-2 * zj.z;
        const Real thj = hf2 - zj.w;
        double pjx = 0, pjy = 0, pjz = 0;
        if constexpr (F64) { pjx = s_p[0][t]; pjy = s_p[F64 ? 1 : 0][t]; pjz = s_p[F64 ? 2 : 0][t]; }
        Real K00 = 0, K11 = 0, K22 = 0, K12 = 0, K02 = 0, K01 = 0;
        Real A00 = 0, A01 = 0, A02 = 0, A10 = 0, A11 = 0, A12 = 0, A20 = 0, A21 = 0, A22 = 0;
        int cnt = 0;
        Real cntr = (Real)0;
        // sub-horizon of bond (i, j): k in H_i with |x_k - x_j| <= delta
        // (the sub-horizon test of Alg. 1)
        if constexpr (F64) {
#pragma unroll 2
            for (int q = 0; q < nb; q++) {
                const R4<Real> zk = s_z[q];
                const double d0 = __dsub_rn(s_p[0][q], pjx);
                const double d1 = __dsub_rn(s_p[F64 ? 1 : 0][q], pjy);
                const double d2 = __dsub_rn(s_p[F64 ? 2 : 0][q], pjz);
                const bool member = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)),
                                              __dmul_rn(d2, d2)) <= k.delta2;
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
            cntr = (Real)cnt;
        } else {
            // FP32 sub-horizon sums, predicated (no branches, no mask multiplies)
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
            cntr = cntf;
            cnt = small_count(cntf);
        }
        bond_epilogue<Real, MODEL, CPL, NRED>(
            s, k, i, r0, t, rb, zj, s_y[t].w, K00, K11, K22, K12, K02, K01, A00, A01, A02, A10, A11,
            A12, A20, A21, A22, cntr, cnt, mjx, mjy, mjz, thj, sig_i, pc_i, cc, Srs, inv_nb, inv_dx,
            with_dt, s_park[(F64 || MODEL == 2) ? 0 : threadIdx.x], s_M[MODEL == 2 ? t : 0], red,
            n_pairs, n_plastic, n_nonconv, n_singular, n_ret64);
    }
    }
    block_sum<NRED, Real>(red, s_red);
    const Real w = red[0];

    if constexpr (MODEL == 2) {
        // power-conjugate form: every sub-horizon's force acts on each of its
        // members; the row is normalised by sum(varpi)
        Real ts[3] = {(Real)0, (Real)0, (Real)0};
        const Real inv_w = w > (Real)0 ? (Real)1 / w : (Real)0;
        for (int t = threadIdx.x; t < nb; t += TPP) {
            const R4<Real> zt = s_z[t];
            const int rb = s.rev[r0 + t];     // loaded before the member loop hides its latency
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
                    const float tst = member_test_lhs(zt.x, zt.y, zt.z, zt.w, m2.y, m2.z, m2.w);
                    masked_add9(tst, m3.x, m0, m1, m2.x, Nf);
                }
#pragma unroll
                for (int e = 0; e < 9; e++) N[e] = Nf[e];
            }
            const Real T0 = (N[0] * zt.x + N[1] * zt.y + N[2] * zt.z) * inv_w;
            const Real T1 = (N[3] * zt.x + N[4] * zt.y + N[5] * zt.z) * inv_w;
            const Real T2 = (N[6] * zt.x + N[7] * zt.y + N[8] * zt.z) * inv_w;
            Real o[3];
            store_force_state<CPL>(s, k, (size_t)r0 + t, rb, T0, T1, T2, zt, s_y[t].w, CPL ? s.J[i] : (Real)1, o);
            ts[0] += o[0]; ts[1] += o[1]; ts[2] += o[2];
        }
        block_sum<3, Real>(ts, reinterpret_cast<Real(*)[3]>(&s_red[0][0]));
        red[9] = ts[0]; red[10] = ts[1]; red[11] = ts[2];
    }

    unsigned cnts[5] = {n_plastic, n_nonconv, n_singular, n_pairs, n_ret64};
    block_sum<5, unsigned>(cnts, s_cnt);
    if (threadIdx.x == 0) point_commit<Real, CPL, NRED>(s, i, n, red, w, eps_i, cnts, update);
}

template <typename Real, int MODEL, int TPP, bool CPL>
__global__ void __launch_bounds__(TPP, sizeof(Real) == 4 ? (640 / TPP) : (256 / TPP > 0 ? 256 / TPP : 1))
k_bond(DevState<Real> s, StepConst k, int with_dt, int update) {
    // the run has stopped (set by the energy check between steps, so every
    // thread of the block reads the same value)
    if (k.halt && (s.ctr->status & PPM_STATUS_HALTED)) return;
    bond_point<Real, MODEL, TPP, CPL>(s, k, blockIdx.x, with_dt, update);
}

// The points with more than kTcRows bonds, for the tensor-core kernel below
// (which leaves them): one warp per block scans 32 points at a time and
// runs the scalar sums on each that has more.  Only the mixed path with the
// force state of Eq. 51 or the power-conjugate one runs this pair of kernels.
template <int MODEL, bool CPL>
__global__ void __launch_bounds__(32, 16)
k_bond_big(DevState<float> s, StepConst k, int with_dt, int update) {
    if (k.halt && (s.ctr->status & PPM_STATUS_HALTED)) return;
    for (int base = blockIdx.x * 32; base < k.npoints; base += gridDim.x * 32) {
        const int i = base + (int)threadIdx.x;
        const bool big = i < k.npoints && s.row_ptr[i + 1] - s.row_ptr[i] > kTcRows;
        unsigned m = __ballot_sync(0xffffffffu, big);
        while (m) {
            const int l = __ffs(m) - 1;
            m &= m - 1;
            bond_point<float, MODEL, 32, CPL>(s, k, base + l, with_dt, update);
        }
    }
}

// Fused bond kernel with the sub-horizon sums on the tensor cores
// (tc_pass_sums): one warp per point with at most kTcRows bonds, the mixed
// path, the force state of Eq. 51 (MODEL 0) or the power-conjugate one
// (MODEL 2), and the coupled mode.  The member features are built once;
// then, 32 bonds at a time, their sums and their updates (bond_epilogue), as
// in bond_point.  Model 2 then sums each receiver's senders the same way
// (tc_pass_receiver).  PPB warps per block, each on its own points: warp w
// of block b takes points (b PPB + w) + m gridDim.x PPB, m = 0, 1, ..., so
// the grid may cover every point once or be a persistent wave of resident
// blocks that loop over them (the launch shape the autotuner picks).
template <int MODEL, bool CPL, int PPB>
__global__ void __launch_bounds__(32 * PPB, 16 / PPB)
k_bond_tcw(DevState<float> s, StepConst k, int with_dt, int update) {
    using Real = float;
    constexpr int NRED = CPL ? 13 : 12;
    static_assert(MODEL == 0 || MODEL == 2, "the sub-horizon force states");
    if (k.halt && (s.ctr->status & PPM_STATUS_HALTED)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const size_t n = (size_t)k.npoints;
    __shared__ R4<float> s_zs[PPB][kTcRows];          // zeta~_k, lattice units, |zeta~_k|^2
    // Ydot_k while the features are built, then the sums of a pass (and the
    // rows where plastic bonds park during their returns)
    __shared__ alignas(16) unsigned char s_yFs[PPB][kTcYF];
    __shared__ float s_Jms[PPB][CPL ? kTcRows : 1];   // coupled mode: the members' volume ratios
    __shared__ alignas(16) unsigned s_phis[PPB][kTcPhiWords];
    __shared__ alignas(16) unsigned s_tws[PPB][4 * kTcRows];   // the test's member words
    // model 2: each sender's matrix M = varpi sigma K^-1
    __shared__ float s_Ms[PPB][MODEL == 2 ? kTcRows : 1][9];
    R4<float>* s_z = s_zs[w];
    float(*s_M)[9] = s_Ms[w];
    R4<float>* s_y = reinterpret_cast<R4<float>*>(s_yFs[w]);
    float(*F)[kTcF] = reinterpret_cast<float(*)[kTcF]>(s_yFs[w]);
    float* s_Jm = s_Jms[w];
    unsigned* s_phi = s_phis[w];
    unsigned* s_tw = s_tws[w];

    for (int i = blockIdx.x * PPB + w; i < k.npoints; i += gridDim.x * PPB) {
        const int r0 = s.row_ptr[i];
        const int nb = s.row_ptr[i + 1] - r0;
        if (nb > kTcRows) continue;                   // k_bond_big takes this point (warp-uniform)
        __syncwarp();                                 // the previous point is done with the arrays
        const int li = s.lat[i];
        const int ix = lat_x(li), iy = lat_y(li), iz = lat_z(li);
        const Real inv_dx = k.inv_dxf;
        Real sig_i[6];
#pragma unroll
        for (int c = 0; c < 6; c++) sig_i[c] = s.sig[c * n + i];
        const Real pc_i = s.pc[i];
        const Real eps_i = s.eps[i];
        const ColumnConst cc = s.cols[s.colid[i]];
        Real Srs = cc.Srsf;
        if constexpr (CPL) {
            Real mass_unused;
            coupled_point<Real>(k, s.J[i], Srs, mass_unused);
        }
        // stage the family of i (the FP32 staging of bond_point)
        const Real uxi = s.u[i], uyi = s.u[n + i], uzi = s.u[2 * n + i];
        const Real vxi = s.vh[i], vyi = s.vh[n + i], vzi = s.vh[2 * n + i];
        for (int t = lane; t < nb; t += 32) {
            const int j = s.col[r0 + t];
            const int lj = s.lat[j];
            R4<Real> z, y;
            z.x = small_float(lat_x(lj) - ix) + (s.u[j] - uxi) * inv_dx;
            z.y = small_float(lat_y(lj) - iy + image_shift(k, lj, li) * k.pbc_ny) + (s.u[n + j] - uyi) * inv_dx;
            z.z = small_float(lat_z(lj) - iz) + (s.u[2 * n + j] - uzi) * inv_dx;
            z.w = z.x * z.x + z.y * z.y + z.z * z.z;
            y.x = s.vh[j] - vxi;
            y.y = s.vh[n + j] - vyi;
            y.z = s.vh[2 * n + j] - vzi;
            y.w = (Real)0;
            s_z[t] = z;
            s_y[t] = y;
            if constexpr (CPL) s_Jm[t] = s.J[j];
        }
        __syncwarp();
        float uK, uA, sT;
        tc_build_features<32>(s_z, s_y, nb, s_phi, s_tw, uK, uA, sT);   // s_y is free afterwards
        const float sT2 = sT * sT, hf2s = k.hf2f * sT2;        // the test's scaled radius
        const Real inv_nb = nb > 0 ? (Real)1 / (Real)nb : (Real)0;
        Real red[NRED];
#pragma unroll
        for (int e = 0; e < NRED; e++) red[e] = (Real)0;
        unsigned n_plastic = 0, n_nonconv = 0, n_singular = 0, n_pairs = 0, n_ret64 = 0;
        // one copy of the pass in the code (its body is large: the loop is not unrolled)
#pragma unroll 1
        for (int p = 0; 32 * p < nb; p++) {
            const int t = 32 * p + lane;
            // the bond's reverse slot, issued before the sums so that its latency hides
            const int rb = (MODEL == 0 && t < nb) ? s.rev[r0 + t] : -1;
            __syncwarp();                             // the previous pass's rows are free
            tc_pass_sums<kTcF>(s_z, s_tw, nb, p, sT2, hf2s, s_phi, &F[0][0], uK, uA);
            if (t < nb) {
                const float* Fr = F[lane];
                const Real K00 = Fr[0], K11 = Fr[1], K22 = Fr[2], K12 = Fr[3], K02 = Fr[4], K01 = Fr[5];
                const Real A00 = Fr[6], A01 = Fr[7], A02 = Fr[8], A10 = Fr[9], A11 = Fr[10], A12 = Fr[11];
                const Real A20 = Fr[12], A21 = Fr[13], A22 = Fr[14];
                const Real cntr = Fr[15];
                const R4<Real> zj = s_z[t];
                // the row is this lane's until the next pass: it parks there
                bond_epilogue<Real, MODEL, CPL, NRED, 9>(
                    s, k, i, r0, t, rb, zj, CPL ? s_Jm[t] : (Real)1, K00, K11, K22, K12, K02, K01,
                    A00, A01, A02, A10, A11, A12, A20, A21, A22, cntr, small_count(cntr), (Real)0,
                    (Real)0, (Real)0, (Real)0, sig_i, pc_i, cc, Srs, inv_nb, inv_dx, with_dt, F[lane],
                    s_M[MODEL == 2 ? t : 0], red, n_pairs, n_plastic, n_nonconv, n_singular, n_ret64);
            }
        }
        warp_sum<NRED, Real>(red);
        if constexpr (MODEL == 2) {
            // power-conjugate form: every sub-horizon's force acts on each of
            // its members; the row is normalised by sum(varpi)
            const Real w_sum = red[0];
            const Real inv_w = w_sum > (Real)0 ? (Real)1 / w_sum : (Real)0;
            __syncwarp();                             // every sender's row of s_M is written
            const float uM = tc_build_sender_features(s_M, nb, s_phi);
            Real ts[3] = {(Real)0, (Real)0, (Real)0};
#pragma unroll 1
            for (int p = 0; 32 * p < nb; p++) {
                const int t = 32 * p + lane;
                const int rb = t < nb ? s.rev[r0 + t] : -1;
                __syncwarp();
                tc_pass_receiver<3, kTcF>(s_z, s_tw, nb, p, sT2, hf2s, s_phi, &F[0][0], uM, uM, 9, 9);
                if (t < nb) {
                    const float* Nr = F[lane];
                    const R4<Real> zt = s_z[t];
                    const Real T0 = (Nr[0] * zt.x + Nr[1] * zt.y + Nr[2] * zt.z) * inv_w;
                    const Real T1 = (Nr[3] * zt.x + Nr[4] * zt.y + Nr[5] * zt.z) * inv_w;
                    const Real T2 = (Nr[6] * zt.x + Nr[7] * zt.y + Nr[8] * zt.z) * inv_w;
                    Real o[3];
                    store_force_state<CPL>(s, k, (size_t)r0 + t, rb, T0, T1, T2, zt,
                                           CPL ? s_Jm[t] : (Real)1, CPL ? s.J[i] : (Real)1, o);
                    ts[0] += o[0]; ts[1] += o[1]; ts[2] += o[2];
                }
            }
            warp_sum<3, Real>(ts);
            red[9] = ts[0]; red[10] = ts[1]; red[11] = ts[2];
        }
        unsigned cnts[5] = {n_plastic, n_nonconv, n_singular, n_pairs, n_ret64};
        warp_sum<5, unsigned>(cnts);
        if (lane == 0) point_commit<Real, CPL, NRED>(s, i, n, red, red[0], eps_i, cnts, update);
    }
}

// Fused bond kernel with the sub-horizon tests and sums in tensor memory
// (tcgen05): the mixed path, the force state of Eq. 51, not the coupled
// mode, points with at most kTcRows bonds (k_bond_big takes the others).
// One CTA of kT5Threads threads per point, thread t its bond t and its
// member t; a persistent wave of CTAs loops over the points, each holding
// kT5Cols columns of tensor memory for its whole life.  Per point: the
// staging, the member features (Phi) and the test terms of thread t's bond
// and member in shared memory; the distance product and, from its signs,
// the mask; the sums product; then each thread updates its bond
// (bond_epilogue) and the CTA commits the point.  The next point's
// neighbour data is fetched by cp.async while the current point's bonds
// are updated, so that its staging finds it in shared memory.  A wait that
// runs out (about a second) sets PPM_STATUS_TC_TIMEOUT and stops the CTA
// (its remaining points keep their state); the CTA still waits for its
// product in flight (bounded) and frees its tensor memory.

// words of the prefetched staging data: per bond (lat, u xyz, vh xyz, rev
// of the neighbour) and per point (lat, u xyz, vh xyz, sigma, pc, eps, column)
constexpr int kT5StageWords = 8;
constexpr int kT5PointWords = 16;

__device__ __forceinline__ void t5_cp4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;"
                 :: "r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}

// Issue the copies of point i's staging data (thread t: its bond's
// neighbour; threads below kT5PointWords: one word of the point's own
// data).  r0, nb: the point's row; j: its t-th neighbour (t < nb).
__device__ __forceinline__ void t5_prefetch(const DevState<float>& s, size_t n, int i, int r0, int nb,
                                            int j, int t, unsigned* stage, unsigned* pt) {
    if (nb <= kTcRows && t < nb) {
        unsigned* d = stage + kT5StageWords * t;
        t5_cp4(d + 0, s.lat + j);
        t5_cp4(d + 1, s.u + j);
        t5_cp4(d + 2, s.u + n + j);
        t5_cp4(d + 3, s.u + 2 * n + j);
        t5_cp4(d + 4, s.vh + j);
        t5_cp4(d + 5, s.vh + n + j);
        t5_cp4(d + 6, s.vh + 2 * n + j);
        t5_cp4(d + 7, s.rev + r0 + t);
    }
    if (t < kT5PointWords) {
        const void* src = t == 0 ? (const void*)(s.lat + i)
                        : t < 4 ? (const void*)(s.u + (size_t)(t - 1) * n + i)
                        : t < 7 ? (const void*)(s.vh + (size_t)(t - 4) * n + i)
                        : t < 13 ? (const void*)(s.sig + (size_t)(t - 7) * n + i)
                        : t == 13 ? (const void*)(s.pc + i)
                        : t == 14 ? (const void*)(s.eps + i) : (const void*)(s.colid + i);
        t5_cp4(pt + t, src);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__global__ void __launch_bounds__(kT5Threads, 4)
k_bond_t5(DevState<float> s, StepConst k, int with_dt, int update) {
    using Real = float;
    constexpr int NRED = 12;
    if (k.halt && (s.ctr->status & PPM_STATUS_HALTED)) return;   // the whole CTA, before any allocation
    extern __shared__ __align__(128) unsigned char t5s[];
    __shared__ alignas(8) uint64_t s_mbar;
    __shared__ alignas(8) uint64_t s_spare;                        // fault injection (t5_withhold)
    __shared__ uint32_t s_tmem;
    __shared__ float s_max[2][kT5Threads / 32];
    __shared__ float s_red[2][kT5Threads / 32][NRED];             // by point parity
    __shared__ unsigned s_cnt[2][kT5Threads / 32][5];
    __shared__ unsigned s_pt[kT5PointWords];
    // the staging buffer shares the test-term region, free between the
    // distance product of one point and the term writes of the next
    unsigned* stage = reinterpret_cast<unsigned*>(t5s + kT5Bond);
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const size_t n = (size_t)k.npoints;
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"((uint32_t)__cvta_generic_to_shared(&s_tmem)), "r"(kT5Cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::);
    }
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&s_mbar);
    const uint32_t mb_spare = (uint32_t)__cvta_generic_to_shared(&s_spare);
    // with t5_withhold the CTA's first product signals the spare barrier, so
    // that the wait on mb runs out; the drain below then waits on the spare
    const bool withhold = k.t5_withhold != 0;
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb_spare) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the first point's staging data
    int i = blockIdx.x;
    int r0 = 0, nb = 0;
    if (i < k.npoints) {
        r0 = s.row_ptr[i];
        nb = s.row_ptr[i + 1] - r0;
        t5_prefetch(s, n, i, r0, nb, (nb <= kTcRows && t < nb) ? s.col[r0 + t] : 0, t, stage, s_pt);
    }
    t5_fence_before();
    __syncthreads();
    t5_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t tl = tmem + ((uint32_t)(32 * w) << 16);        // this warp's 32 lanes
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(t5s);
    uint32_t phase = 0;
    int parity = 0;
    bool ok = true;
    for (; i < k.npoints; i += gridDim.x) {
        const int in = i + gridDim.x;                               // this CTA's next point
        // this point's staging data has landed (every thread's copies)
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        if (nb > kTcRows) {                                         // CTA-uniform: k_bond_big's point
            if (in < k.npoints) {
                const int r0n = s.row_ptr[in], nbn = s.row_ptr[in + 1] - r0n;
                t5_prefetch(s, n, in, r0n, nbn, (nbn <= kTcRows && t < nbn) ? s.col[r0n + t] : 0, t, stage, s_pt);
                r0 = r0n;
                nb = nbn;
            }
            continue;
        }
        const bool in_row = t < nb;
        const int li = (int)s_pt[0];
        const int ix = lat_x(li), iy = lat_y(li), iz = lat_z(li);
        const Real inv_dx = k.inv_dxf;
        Real sig_i[6];
#pragma unroll
        for (int c = 0; c < 6; c++) sig_i[c] = __uint_as_float(s_pt[7 + c]);
        const Real pc_i = __uint_as_float(s_pt[13]);
        const Real eps_i = __uint_as_float(s_pt[14]);
        const ColumnConst cc = s.cols[(int)s_pt[15]];
        const Real Srs = cc.Srsf;
        // staging of bond / member t (the FP32 staging of bond_point)
        R4<Real> z, y;
        z.x = z.y = z.z = z.w = (Real)0;
        y = z;
        int rb = -1;
        if (in_row) {
            const unsigned* sg = stage + kT5StageWords * t;
            const int lj = (int)sg[0];
            rb = (int)sg[7];
            z.x = small_float(lat_x(lj) - ix) + (__uint_as_float(sg[1]) - __uint_as_float(s_pt[1])) * inv_dx;
            z.y = small_float(lat_y(lj) - iy + image_shift(k, lj, li) * k.pbc_ny) +
                  (__uint_as_float(sg[2]) - __uint_as_float(s_pt[2])) * inv_dx;
            z.z = small_float(lat_z(lj) - iz) + (__uint_as_float(sg[3]) - __uint_as_float(s_pt[3])) * inv_dx;
            z.w = z.x * z.x + z.y * z.y + z.z * z.z;
            y.x = __uint_as_float(sg[4]) - __uint_as_float(s_pt[4]);
            y.y = __uint_as_float(sg[5]) - __uint_as_float(s_pt[5]);
            y.z = __uint_as_float(sg[6]) - __uint_as_float(s_pt[6]);
        }
        // largest |component| of zeta~ and of Ydot over the members with finite values
        const float az = fmaxf(fabsf(z.x), fmaxf(fabsf(z.y), fabsf(z.z)));
        const float ay = fmaxf(fabsf(y.x), fmaxf(fabsf(y.y), fabsf(y.z)));
        const bool zfin = in_row && az <= FLT_MAX;
        float mz = zfin ? az : 0.0f, my = (zfin && ay <= FLT_MAX) ? ay : 0.0f;
        mz = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(mz)));
        my = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(my)));
        if (lane == 0) { s_max[0][w] = mz; s_max[1][w] = my; }
        __syncthreads();                                            // the staging buffer is read
#pragma unroll
        for (int q = 0; q < kT5Threads / 32; q++) { mz = fmaxf(mz, s_max[0][q]); my = fmaxf(my, s_max[1][q]); }
        const float sK = tc_scale(mz * mz), sA = tc_scale(mz * my), sT = tc_scale(mz);
        const float uK = 1.0f / sK, uA = 1.0f / sA, sT2 = sT * sT, hf2s = k.hf2f * sT2;
        // member features of member t into Phi (rows 2f / 2f + 1: high / low part of
        // feature f, row 30 the count, row 31 zero): neighbouring threads pair up so
        // that each writes one fp16 pair
        {
            float f[16];
            tc_member_features_of(z, y, zfin, sK, sA, f);
            const bool odd = t & 1;
#pragma unroll
            for (int e = 0; e < 16; e++) {
                float h, l;
                if (e < 15) tc_split(f[e], h, l);
                else { h = f[15]; l = 0.0f; }
                const float x = __shfl_xor_sync(0xffffffffu, odd ? h : l, 1);
                const int row = 2 * e + (odd ? 1 : 0);
                const unsigned word = odd ? tc_pack(x, l) : tc_pack(h, x);
                *reinterpret_cast<unsigned*>(t5s + kT5Phi + t5_off(row, t & ~1, 128)) = word;
            }
        }
        // test terms of bond t (a row of the distance product) and of member t (a column)
        {
            const float cx = z.x * sT, cy = z.y * sT, cz = z.z * sT, cw = z.w * sT2;
            const bool tok = in_row && fabsf(cx) < 2.0f && fabsf(cy) < 2.0f && fabsf(cz) < 2.0f && cw < 16.0f;
            uint4 a0 = make_uint4(0u, 0u, 0u, 0u), a1 = make_uint4(0u, 0u, kTcOnes, kTcFarWord);
            uint4 b0 = make_uint4(0u, 0u, 0u, 0u), b1 = make_uint4(0u, 0u, kTcFarWord, kTcOnes);
            if (tok) {
                float xh, xl, yh, yl, zh, zl;
                tc_split(cx, xh, xl);
                tc_split(cy, yh, yl);
                tc_split(cz, zh, zl);
                a0 = make_uint4(tc_pack(-2.0f * xh, -2.0f * xh), tc_pack(-2.0f * xl, -2.0f * xl),
                                tc_pack(-2.0f * yh, -2.0f * yh), tc_pack(-2.0f * yl, -2.0f * yl));
                a1 = make_uint4(tc_pack(-2.0f * zh, -2.0f * zh), tc_pack(-2.0f * zl, -2.0f * zl), kTcOnes,
                                tc_split_pack(__fmaf_rn(z.w, sT2, -hf2s)));
                b0 = make_uint4(tc_pack(xh, xl), tc_pack(xh, xl), tc_pack(yh, yl), tc_pack(yh, yl));
                b1 = make_uint4(tc_pack(zh, zl), tc_pack(zh, zl), tc_split_pack(cw), kTcOnes);
            }
            *reinterpret_cast<uint4*>(t5s + kT5Bond + t5_off(t, 0, 16)) = a0;
            *reinterpret_cast<uint4*>(t5s + kT5Bond + t5_off(t, 8, 16)) = a1;
            *reinterpret_cast<uint4*>(t5s + kT5Memb + t5_off(t, 0, 16)) = b0;
            *reinterpret_cast<uint4*>(t5s + kT5Memb + t5_off(t, 8, 16)) = b1;
        }
        t5_fence_proxy();
        t5_fence_before();
        __syncthreads();
        t5_fence_after();
        if (t == 0) {
            t5_mma(tmem, t5_desc(sbase + kT5Bond, 256), t5_desc(sbase + kT5Memb, 256), kT5IdescDist, 0);
            t5_commit(withhold ? mb_spare : mb);
        }
        // the next point's row, while the product runs
        int r0n = 0, nbn = 0;
        if (in < k.npoints) {
            r0n = s.row_ptr[in];
            nbn = s.row_ptr[in + 1] - r0n;
        }
        ok = __syncthreads_and(t5_wait(mb, phase));
        phase ^= 1u;
        if (!ok) break;
        t5_fence_after();
        // the next point's t-th neighbour, for its copies
        const int jn = (in < k.npoints && nbn <= kTcRows && t < nbn) ? s.col[r0n + t] : 0;
        // the mask row of bond t from the signs of its distances
#pragma unroll 1
        for (int c = 0; c < 4; c++) {
            float v[32];
            t5_ld32(tl + 32u * c, v);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint4 m = make_uint4(tc_sign_pair(v[8 * q], v[8 * q + 1]), tc_sign_pair(v[8 * q + 2], v[8 * q + 3]),
                                           tc_sign_pair(v[8 * q + 4], v[8 * q + 5]), tc_sign_pair(v[8 * q + 6], v[8 * q + 7]));
                *reinterpret_cast<uint4*>(t5s + kT5Mask + t5_off(t, 32 * c + 8 * q, 128)) = m;
            }
        }
        t5_fence_proxy();
        t5_fence_before();
        __syncthreads();
        t5_fence_after();
        if (t == 0) {
#pragma unroll 1
            for (int kk = 0; kk < 8; kk++)
                t5_mma(tmem, t5_desc(sbase + kT5Mask + 256u * kk, 2048), t5_desc(sbase + kT5Phi + 256u * kk, 2048),
                       kT5IdescSums, kk > 0);
            t5_commit(mb);
        }
        ok = __syncthreads_and(t5_wait(mb, phase));
        phase ^= 1u;
        if (!ok) break;
        t5_fence_after();
        Real F[16];
        {
            float v[32];
            t5_ld32(tl, v);
#pragma unroll
            for (int f = 0; f < 16; f++) F[f] = (v[2 * f] + v[2 * f + 1]) * (f < 6 ? uK : (f < 15 ? uA : 1.0f));
        }
        // the test terms are consumed: the next point's copies land there during the updates
        if (in < k.npoints) t5_prefetch(s, n, in, r0n, nbn, jn, t, stage, s_pt);
        Real red[NRED];
#pragma unroll
        for (int e = 0; e < NRED; e++) red[e] = (Real)0;
        unsigned n_plastic = 0, n_nonconv = 0, n_singular = 0, n_pairs = 0, n_ret64 = 0;
        if (in_row) {
            // the mask has been read: its rows park the plastic bonds
            float* park = reinterpret_cast<float*>(t5s + kT5Mask) + 16 * t;
            bond_epilogue<Real, 0, false, NRED>(
                s, k, i, r0, t, rb, z, (Real)1, F[0], F[1], F[2], F[3], F[4], F[5], F[6], F[7], F[8],
                F[9], F[10], F[11], F[12], F[13], F[14], F[15], small_count(F[15]), (Real)0, (Real)0,
                (Real)0, (Real)0, sig_i, pc_i, cc, Srs, nb > 0 ? (Real)1 / (Real)nb : (Real)0, inv_dx,
                with_dt, park, park, red, n_pairs, n_plastic, n_nonconv, n_singular, n_ret64);
        }
        unsigned cnts[5] = {n_plastic, n_nonconv, n_singular, n_pairs, n_ret64};
        warp_sum<NRED, Real>(red);
#pragma unroll
        for (int e = 0; e < 5; e++) cnts[e] = __reduce_add_sync(0xffffffffu, cnts[e]);
        if (lane == 0) {
#pragma unroll
            for (int e = 0; e < NRED; e++) s_red[parity][w][e] = red[e];
#pragma unroll
            for (int e = 0; e < 5; e++) s_cnt[parity][w][e] = cnts[e];
        }
        __syncthreads();
        if (t == 0) {
#pragma unroll
            for (int q = 1; q < kT5Threads / 32; q++) {
#pragma unroll
                for (int e = 0; e < NRED; e++) red[e] += s_red[parity][q][e];
#pragma unroll
                for (int e = 0; e < 5; e++) cnts[e] += s_cnt[parity][q][e];
            }
            point_commit<Real, false, NRED>(s, i, n, red, red[0], eps_i, cnts, update);
        }
        // the next point's sums go to the other half of s_red / s_cnt, so the
        // CTA moves on without waiting for the commit
        parity ^= 1;
        r0 = r0n;
        nb = nbn;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!ok) {
        if (t == 0) atomicOr(&s.ctr->status, PPM_STATUS_TC_TIMEOUT);
        // the product in flight completes the phase the failed wait was on
        // (with t5_withhold: the spare barrier's first phase)
        (void)__syncthreads_and(withhold ? t5_wait(mb_spare, 0u) : t5_wait(mb, phase ^ 1u));
    }
    t5_fence_before();
    __syncthreads();
    if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kT5Cols));
}

// ---------------------------------------------------------------------------
// gather: f_i = dx^2 (sum_own T^ - sum T^[rev]); acceleration, corrector
// ---------------------------------------------------------------------------

// G lanes per point (4: eight points per warp, or 8: four; the autotuner
// times both): each lane sums every G-th entry of the point's row with a
// compensated running sum,
// then the group combines its lanes in a fixed butterfly; lanes 0..2 of the
// group finish the point's three components
template <typename Real, int G>
__global__ void __launch_bounds__(kGatherPointsPerBlock * G)
k_gather(DevState<Real> s, StepConst k, double dt, int initial) {
    constexpr bool F64 = sizeof(Real) == 8;
    static_assert(G == 4 || G == 8, "four or eight lanes per point");
    if (k.halt && (s.ctr->status & PPM_STATUS_HALTED)) return;   // the run has stopped
    __shared__ Real s_e[kGatherPointsPerBlock][3];
    const int lane = threadIdx.x & 31, sub = threadIdx.x & (G - 1), grp = threadIdx.x / G;
    const int lead = lane & ~(G - 1);                            // the group's first lane
    const int i = blockIdx.x * kGatherPointsPerBlock + grp;
    const bool valid = i < k.npoints;
    const size_t n = (size_t)k.npoints;
    Real m = F64 ? (Real)(k.rho * k.dx * k.dx * k.dx) : (Real)k.massf;
    Real dx2 = F64 ? (Real)(k.dx * k.dx) : (Real)k.dx2f;
    // coupled mode: the point's mass and its volume factor J (start of the step)
    if (k.coupled && valid) {
        const Real Jp = s.J[i];
        Real srs_unused;
        coupled_point<Real>(k, Jp, srs_unused, m);
        dx2 = dx2 * Jp;
    }
    const Real inv_rho_dx = F64 ? (Real)(1.0 / (k.rho * k.dx)) : (Real)k.inv_rho_dxf;
    const Real dtr = F64 ? (Real)dt : (Real)(float)dt;
    const Real hdt = (Real)0.5 * dtr;
    Real dwi = 0, dwe = 0, wk = 0;
    // lanes 0..2 of the group fetch the per-point data of component c = sub early
    const int c = sub < 3 ? sub : 0;
    const size_t t = (size_t)c * n + (valid ? i : 0);
    Real ts = 0, fo = 0, vh = 0, v0 = 0, vbar = 0;
    bool fixed = false;
    int r0 = 0, r1 = 0;
    if (valid) {
        r0 = s.row_ptr[i];
        r1 = s.row_ptr[i + 1];
        ts = s.tsum[t]; fo = s.fint[t]; vh = s.vh[t]; v0 = s.v[t];
        fixed = prescribed(s, k, (size_t)i, c, vbar);
    }
    // the row T_(ji) (stored contiguously in Trev), four strides of loads at a time
    Real sum[3], cmp[3];
#pragma unroll
    for (int q = 0; q < 3; q++) { sum[q] = (Real)0; cmp[q] = (Real)0; }
    for (int b0 = r0 + sub; b0 < r1; b0 += 4 * G) {
        Real x[3][4];
#pragma unroll
        for (int it = 0; it < 4; it++) {
            const int b = b0 + G * it;
#pragma unroll
            for (int q = 0; q < 3; q++) x[q][it] = b < r1 ? s.Trev[(size_t)q * k.cap + b] : (Real)0;
        }
#pragma unroll
        for (int q = 0; q < 3; q++)
#pragma unroll
            for (int it = 0; it < 4; it++) {
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
    // fixed-order butterfly over the group's lanes (each ends with the total)
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
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
    // contact with the rigid substrate (Sec. 4.2, Eq. 91-93; readings
    // R31-R33): the plane z = -delta_c below the bottom layer; normal
    // force C_s dx^2 (delta_c - d) / delta_c at a distance d < delta_c,
    // Coulomb friction on the tangential velocity the point would have
    // after the half step without it, never reversing that velocity
    Real fcon = (Real)0;
    if (k.contact) {
        const Real tsx = __shfl_sync(0xffffffffu, ts, lead), tsy = __shfl_sync(0xffffffffu, ts, lead + 1);
        if (valid && sub < 3) {
            const int li = s.lat[i];
            Real z;
            if constexpr (F64) z = __dadd_rn(__dmul_rn((double)lat_z(li), k.dx), (double)s.u[2 * n + i]);
            else z = (float)lat_z(li) * k.dxf + s.u[2 * n + i];
            const Real dc = F64 ? (Real)k.contact_dc : (Real)k.contact_dcf;
            const Real d = z + dc;
            if (d < dc) {
                const Real Fn = F64 ? (Real)(k.contact_modulus * k.dx * k.dx) * (dc - d) / dc
                                    : (Real)k.contact_kf * (dc - d) / dc;
                if (c == 2) {
                    fcon = Fn;
                } else if (k.friction > 0.0) {
                    const Real hdc = F64 ? (Real)(0.5 * k.dt) : (Real)k.hdtf;
                    const Real* w = initial ? s.v : s.vh;
                    const Real gx = F64 ? (Real)k.g[0] : (Real)k.gf[0];
                    const Real gy = F64 ? (Real)k.g[1] : (Real)k.gf[1];
                    const Real vtx = w[i] + hdc * ((tsx - (sum[0] + cmp[0])) * dx2 / m + gx);
                    const Real vty = w[n + i] + hdc * ((tsy - (sum[1] + cmp[1])) * dx2 / m + gy);
                    const Real nrm = sqrt(vtx * vtx + vty * vty);
                    if (nrm > (Real)0) {
                        const Real mu = F64 ? (Real)k.friction : (Real)k.frictionf;
                        const Real Ft = fmin(mu * Fn, m * nrm / hdc);
                        fcon = -Ft * (c == 0 ? vtx : vty) / nrm;
                    }
                }
            }
        }
    }
    if (valid && sub < 3) {
        const Real g = F64 ? (Real)k.g[c] : (Real)k.gf[c];
        const Real gathered = c == 0 ? sum[0] + cmp[0] : (c == 1 ? sum[1] + cmp[1] : sum[2] + cmp[2]);
        const Real fhat = ts - gathered;
        Real f = fhat * dx2;                                     // Eq. 49-50
        Real a = fhat * inv_rho_dx + g;                          // Eq. 62
        if (k.coupled) a = f / m + g;
        if (k.contact) {
            f += fcon;                                           // Eq. 93
            a = f / m + g;
        }
        if (fixed) a = (Real)0;
        bool bad = !isfinite(a);
        s.fint[t] = f;
        s.a[t] = a;
        if (initial) {
            bad = bad || !isfinite(v0);
            wk = (Real)0.5 * m * v0 * v0;
        } else {
            const Real v = vh + hdt * a;                         // Eq. 63
            // a point whose position stopped being finite leaves every
            // family and keeps a finite acceleration: its velocity tells
            bad = bad || !isfinite(v);
            s.v[t] = v;
            dwi = -hdt * vh * (fo + f);                          // Eq. 66
            dwe = dtr * m * vh * g;                              // Eq. 67
            // a prescribed component moves under the reaction -(f + m g);
            // its work is external (zero where the component is held)
            if (fixed) dwe += -hdt * vh * (fo + f + (Real)2 * m * g);
            wk = (Real)0.5 * m * v * v;                          // Eq. 68
        }
        if (bad) atomicOr(&s.ctr->status, PPM_STATUS_NONFINITE);
    }
    // coupled mode: the volume ratio the bond pass computed is the next
    // step's (every reader of J in this step has run)
    if (k.coupled && !initial && valid && sub == 0) s.J[i] = s.Jn[i];
    // energies of the point: lanes 0..2 of the group hold the three components
    dwi += __shfl_down_sync(0xffffffffu, dwi, 1) + __shfl_down_sync(0xffffffffu, dwi, 2);
    dwe += __shfl_down_sync(0xffffffffu, dwe, 1) + __shfl_down_sync(0xffffffffu, dwe, 2);
    wk += __shfl_down_sync(0xffffffffu, wk, 1) + __shfl_down_sync(0xffffffffu, wk, 2);
    if (sub == 0) {
        s_e[grp][0] = valid ? dwi : (Real)0;
        s_e[grp][1] = valid ? dwe : (Real)0;
        s_e[grp][2] = valid ? wk : (Real)0;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double tot = 0.0;
        for (int q = 0; q < kGatherPointsPerBlock; q++) tot += (double)s_e[q][threadIdx.x];
        s.epart[(size_t)blockIdx.x * 3 + threadIdx.x] = tot;
    }
}

__global__ void __launch_bounds__(1024)
k_energy_reduce(const double* epart, int nblocks, DevCounters* ctr, int initial,
                const int32_t* row_ptr, int npoints, int halt, double tol) {
    if (halt && (ctr->status & PPM_STATUS_HALTED)) return;     // the run has stopped
    __shared__ double sm[3][1024];
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
            ctr->steps_done += 1;
            const double bal = fabs(ctr->W_int + ctr->W_kin - ctr->W_ext - ctr->W_kin0);
            const double mx = fmax(fmax(ctr->W_kin, fabs(ctr->W_int)), fmax(fabs(ctr->W_ext), ctr->W_kin0));
            if (bal > tol * mx) {                                          // Eq. 69
                if (!(ctr->status & PPM_STATUS_UNSTABLE)) ctr->unstable_step = (long long)ctr->steps_done;
                atomicOr(&ctr->status, PPM_STATUS_UNSTABLE);
                if (halt && !(ctr->status & PPM_STATUS_HALTED)) {
                    // hard stop: the following steps' kernels find this bit and return
                    atomicOr(&ctr->status, PPM_STATUS_HALTED);
                    ctr->halted_step = (long long)ctr->steps_done;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// initial state (Alg. 2) and velocity boundary conditions
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
        s.J[i] = (Real)1;
        s.Jn[i] = (Real)1;
    }
}

template <typename Real>
__global__ void k_velocity_bc(DevState<Real> s, StepConst k) {
    const size_t n = (size_t)k.npoints;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < 3 * n;
         t += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / n);
        const size_t i = t - (size_t)c * n;
        Real vbar;
        if (prescribed(s, k, i, c, vbar)) s.v[t] = vbar;
    }
}

template <typename Real>
__global__ void k_tforce_from_rev(DevState<Real> s, long long cap, long long nbonds) {
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nbonds;
         b += (long long)gridDim.x * blockDim.x) {
        const long long rb = s.rev[b];
#pragma unroll
        for (int q = 0; q < 3; q++) s.T[q * cap + b] = s.Trev[q * cap + rb];
    }
}

// blocks of k_bond_big: each scans 32 points at a time
inline int big_blocks(int npoints) {
    const int b = (npoints + 31) / 32;
    return b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16;
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
    const int tpp = (k.tile == 32 || k.tile == 64 || k.tile == 256) ? k.tile : 128;
    // the coupled mode runs its own instantiations
#define PPM_BOND(M, T) do {                                                                        \
        if (k.coupled) k_bond<Real, M, T, true><<<k.npoints, T, 0, st>>>(s, k, with_dt, update);  \
        else k_bond<Real, M, T, false><<<k.npoints, T, 0, st>>>(s, k, with_dt, update);           \
    } while (0)
#define PPM_BOND_TILES(M)                           \
    if (tpp == 32) PPM_BOND(M, 32);                 \
    else if (tpp == 64) PPM_BOND(M, 64);            \
    else if (tpp == 256) PPM_BOND(M, 256);          \
    else PPM_BOND(M, 128);
    if constexpr (sizeof(Real) == 4) {
        if (k.model == 0 && !k.coupled && tpp == 128 && k.t5_blocks > 0) {
            // tensor-memory tests and sums, one CTA per point; then the points
            // with more than kTcRows bonds with the scalar sums
            const int grid = k.t5_blocks < k.npoints ? k.t5_blocks : k.npoints;
            k_bond_t5<<<grid, kT5Threads, kT5Smem, st>>>(s, k, with_dt, update);
            k_bond_big<0, false><<<big_blocks(k.npoints), 32, 0, st>>>(s, k, with_dt, update);
            return cudaGetLastError();
        }
        if ((k.model == 0 || k.model == 2) && tpp == 32) {
            // tensor-core sums, one warp per point; then the points with more
            // than kTcRows bonds (normally none) with the scalar sums
            const int ppb = k.tc_ppb == 2 ? 2 : 1;
            const int full = (k.npoints + ppb - 1) / ppb;
            const int grid = (k.tc_blocks > 0 && k.tc_blocks < full) ? k.tc_blocks : full;
#define PPM_TCW(M, C)                                                                               \
    do {                                                                                            \
        if (ppb == 1) k_bond_tcw<M, C, 1><<<grid, 32, 0, st>>>(s, k, with_dt, update);              \
        else k_bond_tcw<M, C, 2><<<grid, 64, 0, st>>>(s, k, with_dt, update);                       \
        k_bond_big<M, C><<<big_blocks(k.npoints), 32, 0, st>>>(s, k, with_dt, update);              \
    } while (0)
            if (k.model == 0) {
                if (k.coupled) PPM_TCW(0, true); else PPM_TCW(0, false);
            } else {
                if (k.coupled) PPM_TCW(2, true); else PPM_TCW(2, false);
            }
#undef PPM_TCW
            return cudaGetLastError();
        }
    }
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
    if (k.gather_lanes == 8) k_gather<Real, 8><<<gather_blocks, kGatherPointsPerBlock * 8, 0, st>>>(s, k, dt, initial);
    else k_gather<Real, 4><<<gather_blocks, kGatherPointsPerBlock * 4, 0, st>>>(s, k, dt, initial);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_tforce_from_rev(const DevState<Real>& s, const StepConst& k, long long nbonds,
                                   cudaStream_t st) {
    if (nbonds <= 0) return cudaSuccess;
    k_tforce_from_rev<Real><<<blocks_for((size_t)nbonds, 256), 256, 0, st>>>(s, k.cap, nbonds);
    return cudaGetLastError();
}

cudaError_t bond_tc_resident_blocks(int model, int ppb, int coupled, int* blocks) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
#define PPM_OCC(M, C, P) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bond_tcw<M, C, P>, 32 * P, 0)
    if (model == 2) {
        if (ppb == 2) e = coupled ? PPM_OCC(2, true, 2) : PPM_OCC(2, false, 2);
        else e = coupled ? PPM_OCC(2, true, 1) : PPM_OCC(2, false, 1);
    } else {
        if (ppb == 2) e = coupled ? PPM_OCC(0, true, 2) : PPM_OCC(0, false, 2);
        else e = coupled ? PPM_OCC(0, true, 1) : PPM_OCC(0, false, 1);
    }
#undef PPM_OCC
    *blocks = sms * (per_sm > 0 ? per_sm : 1);
    return e;
}

cudaError_t bond_t5_prepare(int* blocks) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bond_t5, cudaFuncAttributeMaxDynamicSharedMemorySize, kT5Smem);
    // the whole unified L1 / shared array as shared memory, so that four CTAs fit
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_bond_t5, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    // resident CTAs per SM from the kernel's registers and shared memory (the
    // occupancy query answers one for this kernel, while four run side by
    // side), and at most four: each holds kT5Cols of the SM's 512 columns
    cudaFuncAttributes fa;
    int smem_sm = 0, regs_sm = 0, reserved = 0;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_bond_t5);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e != cudaSuccess) return e;
    const int by_smem = smem_sm / (kT5Smem + (int)fa.sharedSizeBytes + reserved);
    const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;     // allocated per warp in 256s
    const int by_regs = regs_sm / (regs_warp * (kT5Threads / 32));
    per_sm = 512 / (int)kT5Cols;
    if (by_smem < per_sm) per_sm = by_smem;
    if (by_regs < per_sm) per_sm = by_regs;
    *blocks = sms * (per_sm > 0 ? per_sm : 1);
    return cudaSuccess;
}

cudaError_t launch_energy_reduce(double* epart, int nblocks, DevCounters* ctr, int initial,
                                 const int32_t* row_ptr, int npoints, int halt, double tol,
                                 cudaStream_t st) {
    k_energy_reduce<<<1, 1024, 0, st>>>(epart, nblocks, ctr, initial, row_ptr, npoints, halt, tol);
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
                                          cudaStream_t);                                           \
    template cudaError_t launch_tforce_from_rev<R>(const DevState<R>&, const StepConst&, long long, \
                                                   cudaStream_t);
PPM_INSTANTIATE(double)
PPM_INSTANTIATE(float)
#undef PPM_INSTANTIATE

}  // namespace ppm
