// Internal declarations of the sm_103a library (kernels + host runtime).
// Not part of the public ABI; see include/ppm.h for that.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ppm.h"

namespace ppm {

constexpr int kMaxRow = 256;          // hard cap of bonds per point (smem staging)
constexpr int kDefaultMaxFamily = 192;
constexpr int kWarpPointsPerBlock = 8;  // family kernels: one warp per point
constexpr int kGatherPointsPerBlock = 32;   // force gather: points per block (4 or 8 lanes each)
constexpr int kAdjAccDoubles = 32;     // adjoint accumulators (gradient, state sums) ...
constexpr int kAdjRedBlocks = 152;     // ... followed by 5 partial sums per reduction block
constexpr int kLatBits = 10;          // packed lattice index: ix | iy << 10 | iz << 20
constexpr int kLatMask = (1 << kLatBits) - 1;

__host__ __device__ __forceinline__ int lat_x(int l) { return l & kLatMask; }
__host__ __device__ __forceinline__ int lat_y(int l) { return (l >> kLatBits) & kLatMask; }
__host__ __device__ __forceinline__ int lat_z(int l) { return l >> (2 * kLatBits); }

// per-column constants (ensembles have one entry per column)
struct ColumnConst {
    double M;       // critical-state slope
    double Srs;     // S_r * suction: total stress = effective + Srs * 1
    float Mf, Srsf; // the same in FP32
    int32_t nx, ny, nz, pad;
    int64_t offset; // first point id of the column
};

// device-resident counters and status word
struct DevCounters {
    unsigned long long plastic, nonconv, singular, rebuilds, bond_steps, pairs, ret64;
    unsigned int status, pad;
    int family_ok, pad2;
    double W_int, W_ext, W_kin, W_kin0;
    unsigned long long steps_done;   // completed (not halted) steps
    long long halted_step;           // the step whose energy check halted the run
    long long unstable_step;         // the first step that failed the energy check
};

// uniform cell grid of the family search (device-computed)
struct CellGrid {
    double lo[3];
    double h, inv_h;
    int dims[3];
    int ncell;      // cells per column
};

// constants of the time step shared by all kernels
struct StepConst {
    double dx, inv_dx, delta2;   // delta2 = delta * delta in m^2 (FP64 tests)
    float hf2f;                   // (delta / dx)^2 for FP32 lattice-unit tests
    double dt, rho, K, mu, lk, eta, tol;
    double g[3];
    int visc_form, max_iter, model, lock_lateral;
    int bc;                      // 0: fixed base layer; 1: uniaxial compression along x
    double load_rate;            // m/s, bc = 1
    float load_ratef;
    int elastic;                 // 1: linear elastic skeleton, the yield test off
    int load_layers;             // bc = 1: planes held / driven at each x end
    int halt;                    // 1: the Eq. 69 check stops the run (kernels skip)
    double energy_tol;           // the Eq. 69 tolerance (resolved: > 0)
    int pbc_ny;                  // plane strain: the y period in lattice planes, else 0
    double pbc_L;                // plane strain: the y period ny * dx (m)
    int contact;                 // 1: rigid flat substrate at z = -delta_c (no fixed base)
    double contact_modulus, friction, contact_dc;   // C_s (Pa), mu_f, delta_c (m)
    float contact_kf, frictionf, contact_dcf;        // C_s dx^2, mu_f, delta_c in FP32
    int coupled;                 // 1: J-dependent porosity, S_r, volume and mass
    double phi0, rho_s, rho_w, wr_a1, wr_a2, wr_n, wr_s;     // and the column's suction
    float phi0f, rho_sf, rho_wf, wr_a1f, wr_a2f, wr_nf, wr_sf;
    double pair_dc, pair_kappa;  // between points: delta_c / dx and C_s / (2 delta_c / dx)
    float pair_dcf, pair_kappaf; // the same in FP32
    int npoints, ncols, max_family, tile;   // tile: bond-kernel threads per point
    int tc_ppb, tc_blocks;       // tensor-core bond kernel: points per block; grid (0: one
                                 // point per warp, else a persistent grid of that many blocks)
    int t5_blocks;               // tensor-memory bond kernel: its persistent grid
    int gather_lanes;            // force gather: lanes per point, 4 or 8
    int t5_withhold;             // fault injection: tensor-memory products signal a spare barrier
    long long cap;               // bond capacity
    // FP32 copies used by the mixed path (no FP64 conversions in its loops)
    float dxf, inv_dxf, dtf, hdtf, Kf, muf, rhof, inv_rho_dxf, dx2f, massf, etaf;
    float gf[3];
};

// Short-range repulsion between two material points closer than delta_c
// (Eq. 91 between points of the soil; reading R36), added to the force
// state of bond (i, j) in lattice units, z = (zeta / dx, |zeta / dx|^2): the
// opposite term sits in bond (j, i), so each point of the pair is pushed
// from the other by C_s dx^2 (delta_c - r) / delta_c.  Coincident points
// (no direction) get nothing.
template <typename Real, typename V4>
__device__ __forceinline__ void pair_contact(const StepConst& k, const V4& z, Real& T0, Real& T1, Real& T2) {
    constexpr bool F64 = sizeof(Real) == 8;
    const Real dc = F64 ? (Real)k.pair_dc : (Real)k.pair_dcf;
    if (k.contact && z.w < dc * dc && z.w > (Real)0) {
        const Real kap = F64 ? (Real)k.pair_kappa : (Real)k.pair_kappaf;
        const Real a = kap * (dc / sqrt(z.w) - (Real)1);
        T0 -= a * z.x;
        T1 -= a * z.y;
        T2 -= a * z.z;
    }
}

// Coupled mode at volume ratio J: S_r s of Eq. 15 (exponent -(n - 1)/n,
// void ratio e = J / (1 - phi_0) - 1, p_w = -s; saturated when no voids or
// no suction) and the point mass [rho_s (1 - phi) + rho_w S_r phi] J dx^3
// with phi = 1 - (1 - phi_0) / J (Eq. 16, 48).
template <typename Real>
__device__ __forceinline__ void coupled_point(const StepConst& k, Real J, Real& Srs, Real& mass) {
    constexpr bool F64 = sizeof(Real) == 8;
    const Real phi0 = F64 ? (Real)k.phi0 : (Real)k.phi0f;
    const Real s = F64 ? (Real)k.wr_s : (Real)k.wr_sf;
    const Real e = J / ((Real)1 - phi0) - (Real)1;
    Real Sr = (Real)1;
    if (s > (Real)0 && e > (Real)0) {
        const Real a1 = F64 ? (Real)k.wr_a1 : (Real)k.wr_a1f;
        const Real a2 = F64 ? (Real)k.wr_a2 : (Real)k.wr_a2f;
        const Real nn = F64 ? (Real)k.wr_n : (Real)k.wr_nf;
        const Real alpha = a1 * pow(e, a2) * J;
        Sr = pow((Real)1 + pow(alpha * s, nn), -(nn - (Real)1) / nn);
    }
    const Real phi = (Real)1 - ((Real)1 - phi0) / J;
    const Real rs = F64 ? (Real)k.rho_s : (Real)k.rho_sf;
    const Real rw = F64 ? (Real)k.rho_w : (Real)k.rho_wf;
    const Real dx3 = F64 ? (Real)(k.dx * k.dx * k.dx) : (Real)k.dxf * (Real)k.dxf * (Real)k.dxf;
    Srs = Sr * s;
    mass = (rs * ((Real)1 - phi) + rw * Sr * phi) * J * dx3;
}

// plane strain: the periodic image of point j (lattice index lj) nearest to
// point i (li) in y, as a multiple of the period: -1, 0 or 1
__host__ __device__ __forceinline__ int image_shift(const StepConst& k, int lj, int li) {
    if (!k.pbc_ny) return 0;
    const int dl = lat_y(lj) - lat_y(li);
    return 2 * dl > k.pbc_ny ? -1 : (2 * dl < -k.pbc_ny ? 1 : 0);
}

// device pointers of one context (Real = double for FP64, float for mixed)
template <typename Real>
struct DevState {
    const double* xabs;  // family search only: explicit FP64 positions (3N), else null
    int32_t* lat;        // packed lattice index, N (may be null when xabs is set)
    int32_t* colid;      // column of each point, N (null: one column)
    const ColumnConst* cols;
    Real* u;             // 3N
    float* ulo;          // 3N compensation of u (mixed only; else null)
    Real* v;             // 3N
    Real* vh;            // 3N half-step velocity
    Real* a;             // 3N
    Real* sig;           // 6N
    Real* pc;            // N
    Real* eps;           // N
    Real* fint;          // 3N
    Real* tsum;          // 3N sum of own force states (scaled)
    Real* J;             // N volume ratio at the start of the step (coupled mode)
    Real* Jn;            // N its update by the bond pass, copied to J by the gather
    int32_t* row_ptr;    // N+1
    int32_t* col;        // cap
    int32_t* rev;        // cap
    Real* T;             // 3 x cap scaled force state, bond order (written by the step in the
                         // coupled mode only; otherwise rebuilt from Trev when read)
    Real* Trev;          // 3 x cap: Trev[rev[b]] = T[b], so row j holds T_(ij)
    double* epart;       // energy partials, 3 x gather blocks
    DevCounters* ctr;
    // family scratch
    CellGrid* grid;
    long long* bbox;     // 6 ordered-int encodings (min xyz, max xyz)
    int32_t* cellkey;    // N
    int32_t* cellcnt;    // ncell_cap + 1
    int32_t* cellstart;  // ncell_cap + 1
    int32_t* cellfill;   // ncell_cap
    int32_t* sorted;     // N
    int32_t* rowlen;     // N + 1
    int32_t* scanbuf;    // block sums of the scans
    int ncell_cap;
};

// Stores the force state T of bond (i, j) (row slot b, reverse slot rb) with
// the pair repulsion of the bond (z: the bond in lattice units) and, in the
// coupled mode, the point volumes: the own row carries J_j T + C / J_i and
// the reverse slot J_i T + C / J_j, so that the gather's factor J dx^2 gives
// V_i V_j (T_ij - T_ji) (Eq. 49) and the unscaled pair force.  Returns the
// own-row value for the row sum.  Only the reverse slot is written: the
// gather reads that copy, and outside the coupled mode the bond-order value
// is Trev[rev[b]] (rebuilt on demand when a caller reads the force states);
// in the coupled mode the two differ and the bond-order copy is kept.
template <bool CPL, typename Real, typename V4>
__device__ __forceinline__ void store_force_state(const DevState<Real>& s, const StepConst& k,
                                                  size_t b, int rb, Real T0, Real T1, Real T2,
                                                  const V4& z, Real Jj, Real Ji, Real out[3]) {
    Real C0 = (Real)0, C1 = (Real)0, C2 = (Real)0;
    pair_contact(k, z, C0, C1, C2);
    Real o[3], r[3];
    if constexpr (CPL) {
        o[0] = Jj * T0 + C0 / Ji; o[1] = Jj * T1 + C1 / Ji; o[2] = Jj * T2 + C2 / Ji;
        r[0] = Ji * T0 + C0 / Jj; r[1] = Ji * T1 + C1 / Jj; r[2] = Ji * T2 + C2 / Jj;
    } else {
        o[0] = r[0] = T0 + C0; o[1] = r[1] = T1 + C1; o[2] = r[2] = T2 + C2;
    }
    if constexpr (CPL) {
        s.T[b] = o[0];
        s.T[k.cap + b] = o[1];
        s.T[2 * k.cap + b] = o[2];
    }
    if (rb >= 0) {
        s.Trev[rb] = r[0];
        s.Trev[k.cap + rb] = r[1];
        s.Trev[2 * k.cap + rb] = r[2];
    }
    out[0] = o[0]; out[1] = o[1]; out[2] = o[2];
}

// Boundary conditions (the fixed base; the loading of Sec. 4.1): true when
// velocity component c of point i is prescribed, with the value in vbar.
// bc = 0: the base layer (unless the substrate carries the column) and, with
// lock_lateral, the x and y components are held at zero; under plane strain
// the y component is held at zero.  bc = 1: the load_layers planes at the x = 0 end of the
// point's column are held in x and those at the other end move at
// v_x = -load_rate.
template <typename Real>
__device__ __forceinline__ bool prescribed(const DevState<Real>& s, const StepConst& k, size_t i,
                                           int c, Real& vbar) {
    vbar = (Real)0;
    if (k.lock_lateral && c < 2) return true;
    if (k.pbc_ny && c == 1) return true;          // plane strain
    const int li = s.lat[i];
    if (k.bc == 0) return !k.contact && lat_z(li) == 0;
    if (c != 0) return false;
    const int ix = lat_x(li);
    if (ix < k.load_layers) return true;
    if (ix >= s.cols[s.colid[i]].nx - k.load_layers) {
        vbar = sizeof(Real) == 8 ? (Real)-k.load_rate : (Real)-k.load_ratef;
        return true;
    }
    return false;
}

// adjoint arrays (adjoint.cu); Real as the forward path
template <typename Real>
struct AdjState {
    Real *ub, *vb, *ab;        // 3N: adjoint of u, v, a (after the step on entry, before on exit)
    Real *sb, *pcb;            // 6N, N: adjoint of the point stress and pc
    Real *sbn, *pcbn;          // 6N, N: their new values (before the step)
    Real *fb, *u1b, *vhb;      // 3N: force, positions after the predictor, half-step velocity
    Real *zsum, *ysum;         // 3N: row sums of the position / velocity adjoints
    Real *Zrev, *Yrev;         // 3 x cap: neighbour adjoints at their reverse slots
    double* thpart;            // 3N: per-point partial adjoints of (M, eta, S_r s)
};

// ---- launchers (family.cu) ----
// *nlaunch (if not null) is incremented by the number of kernels launched
template <typename Real>
cudaError_t launch_critical_dt(const DevState<Real>& s, const StepConst& k, long long* out,
                               cudaStream_t st);
template <typename Real>
cudaError_t launch_family_build(const DevState<Real>& s, const StepConst& k, cudaStream_t st,
                                long long* nlaunch);
// exclusive scan of n int32 values in place (n <= 16M); scanbuf >= 8192 ints
cudaError_t launch_exclusive_scan(int32_t* data, int n, int32_t* scanbuf, cudaStream_t st,
                                  long long* nlaunch);

// ---- launchers (bond.cu) ----
template <typename Real>
cudaError_t launch_init_state(const DevState<Real>& s, const StepConst& k, int init_stress,
                              double pc0, cudaStream_t st);
template <typename Real>
cudaError_t launch_apply_velocity_bc(const DevState<Real>& s, const StepConst& k, cudaStream_t st);
template <typename Real>
cudaError_t launch_predictor(const DevState<Real>& s, const StepConst& k, cudaStream_t st);
template <typename Real>
cudaError_t launch_bond(const DevState<Real>& s, const StepConst& k, double dt, int update,
                        cudaStream_t st);
template <typename Real>
cudaError_t launch_gather(const DevState<Real>& s, const StepConst& k, double dt, int initial,
                          int gather_blocks, cudaStream_t st);
// bond-order force states from the reverse slots: T[b] = Trev[rev[b]]
template <typename Real>
cudaError_t launch_tforce_from_rev(const DevState<Real>& s, const StepConst& k, long long nbonds,
                                   cudaStream_t st);
cudaError_t launch_energy_reduce(double* epart, int nblocks, DevCounters* ctr, int initial,
                                 const int32_t* row_ptr, int npoints, int halt, double tol,
                                 cudaStream_t st);
// blocks of one resident wave of the tensor-core bond kernel (force state
// model 0 or 2, points per block ppb = 1 or 2) on the current device
cudaError_t bond_tc_resident_blocks(int model, int ppb, int coupled, int* blocks);
// the tensor-memory bond kernel on the current device: sets its dynamic
// shared memory limit and returns the blocks of one resident wave
cudaError_t bond_t5_prepare(int* blocks);

// ---- launchers (adjoint.cu) ----
// one reverse step from the restored start state (predictor already
// recomputed): acc[0..2] += adjoints of (M, eta, S_r s); with initial, the
// reverse of the initial pass and acc[3] = sum tr(sigma-bar), acc[4] = sum pc-bar
template <typename Real>
cudaError_t launch_adjoint_step(const DevState<Real>& s, const AdjState<Real>& a, const StepConst& k,
                                double* acc, int initial, cudaStream_t st);
template <typename Real>
cudaError_t launch_convert_adjoint(const double* src, Real* dst, size_t count, cudaStream_t st);

}  // namespace ppm
