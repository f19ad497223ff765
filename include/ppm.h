/*
 * ppm.h -- C ABI of the GB300 (sm_103a) library for the per-time-step bond
 * loop of updated Lagrangian unsaturated periporomechanics (Menon & Song,
 * arXiv:2203.05562).
 *
 * One explicit step (Alg. 2) is: Newmark predictor and boundary conditions
 * (Eq. 60-61, 64) -> family search in the current configuration when due
 * (Eq. 1, the family of Alg. 1) -> for every bond the sub-horizon shape tensor and
 * velocity gradient (Eq. 22-26, 55, 57), the critical-state visco-plastic
 * update at constant suction (Sec. 2.3, Eq. 40-46, 70-76) and the force
 * state (Eq. 31-32, 51) -> pairwise nodal forces (Eq. 49-50) -> acceleration
 * and velocity corrector (Eq. 62-63) and the energy terms (Eq. 66-68).
 *
 * Conventions: SI units; tension positive; suction s > 0 (p_w = -s).
 * Per-point vector fields are component-major (f[c*N + i]); the symmetric
 * stress has 6 components in the order xx, yy, zz, yz, xz, xy.  Point id
 * of lattice site (ix, iy, iz) of column c is offset[c] + ix + nx*(iy +
 * ny*iz); columns are stored one after another.  The base layer (iz = 0)
 * of every column is fixed.
 *
 * Ownership: the caller allocates one device workspace of the size
 * ppm_workspace_size() reports and keeps it alive until ppm_destroy();
 * the library never calls cudaMalloc.  Host buffers passed to read/write
 * calls belong to the caller.  All device work is issued on the stream
 * given to ppm_init() and is asynchronous unless stated otherwise.
 *
 * Errors: every function returns PPM_OK (0) or a negative PPM_E* code
 * synchronously; nothing aborts or traps.  Conditions found on the device
 * (Newton non-convergence, degenerate shape tensors, non-finite values,
 * family capacity exceeded) set bits of a status word that ppm_status()
 * returns.
 */
#ifndef PPM_H
#define PPM_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define PPM_OK        0
#define PPM_EINVAL   -1   /* invalid argument or parameter                  */
#define PPM_ENOSPACE -2   /* workspace smaller than ppm_workspace_size()    */
#define PPM_ECUDA    -3   /* a CUDA runtime call failed                     */
#define PPM_ESTATE   -4   /* call not valid in the context's current state  */

/* device status bits (ppm_counters.status) */
#define PPM_STATUS_NONCONV        1u  /* a return-map Newton solve did not converge */
#define PPM_STATUS_SINGULAR       2u  /* a bond had a degenerate shape tensor       */
#define PPM_STATUS_NONFINITE      4u  /* a non-finite acceleration or velocity      */
#define PPM_STATUS_FAMILY_FULL    8u  /* bonds exceeded the workspace capacity      */
#define PPM_STATUS_ROW_FULL      16u  /* a point had more than max_family bonds     */
#define PPM_STATUS_UNSTABLE      32u  /* energy balance of Eq. 69 above 1e-2        */
#define PPM_STATUS_HALTED        64u  /* halt_on_unstable: the steps after the one
                                         whose Eq. 69 check failed did nothing   */
#define PPM_STATUS_TC_TIMEOUT   128u  /* a tensor-memory bond pass stopped waiting
                                         for its products: points it had not
                                         reached kept their state                */

/* precision of the path */
#define PPM_FP64  0   /* everything in FP64                                     */
#define PPM_MIXED 1   /* FP32 kinematics, stress and forces; FP64 shape-tensor
                         inverse and visco-plastic return solve               */

/* force-state model */
#define PPM_SUBHORIZON           0  /* Eq. 51: force state on the bond itself      */
#define PPM_STANDARD             1  /* Sec. 2.1: full-horizon correspondence       */
#define PPM_SUBHORIZON_CONJUGATE 2  /* Eq. 27-31 as a state over each sub-horizon  */

/* state fields for ppm_read_state / ppm_write_state; element type is
 * double for PPM_FP64 and float for PPM_MIXED unless noted */
#define PPM_FIELD_U        0   /* displacement, 3N                           */
#define PPM_FIELD_V        1   /* velocity, 3N                               */
#define PPM_FIELD_A        2   /* acceleration, 3N                           */
#define PPM_FIELD_SIGMA    3   /* effective stress, 6N                       */
#define PPM_FIELD_PC       4   /* preconsolidation pressure (negative), N   */
#define PPM_FIELD_EPS_S    5   /* accumulated equivalent shear strain, N     */
#define PPM_FIELD_FINT     6   /* internal force of the last pass, 3N        */
#define PPM_FIELD_ROW_PTR  7   /* int32, N+1                                 */
#define PPM_FIELD_COL      8   /* int32, bonds (ascending within a row)      */
#define PPM_FIELD_REV      9   /* int32, bonds: index of bond (j,i), -1 none */
#define PPM_FIELD_TFORCE  10   /* force state per bond, 3 x bonds            */
#define PPM_FIELD_J       11   /* volume ratio J (coupled = 1), N            */

typedef struct {
    int32_t nx, ny, nz;          /* lattice of the column (single-column runs)  */
    int32_t model;               /* PPM_SUBHORIZON / _STANDARD / _CONJUGATE     */
    double dx, horizon_factor;   /* spacing; horizon delta = factor * dx        */
    double rho, K, mu;           /* mixture density, bulk and shear modulus     */
    double M, lambda_t, kappa_t; /* critical-state slope; compression indices   */
    double pc0, eta;             /* initial preconsolidation (> 0); viscosity   */
    double suction;              /* constant matric suction (>= 0)              */
    double vg_alpha, vg_n;       /* van Genuchten S_r(s) parameters             */
    double b1, b2;               /* Eq. 45; only b1 = 0, b2 = 1 are accepted    */
    double gravity[3];
    double dt;                   /* <= 0: 0.3 dx / sqrt((K + 4mu/3) / rho)      */
    int32_t rebuild_every;       /* family rebuilt before step n+1 when
                                    (n+1) % R == 0; 0 = never                   */
    int32_t init_stress;         /* 0: K0 geostatic, 1: zero                    */
    int32_t visc_form;           /* 0: eta scaled by pc_n^2 (Pa s), 1: literal  */
    int32_t newton_max_iter;
    double newton_tol;
    int32_t lock_lateral;        /* 1: x and y motion suppressed               */
    int32_t precision;           /* PPM_FP64 or PPM_MIXED                       */
    int32_t max_family;          /* bond capacity per point (0: 192; max 256)  */
    int32_t use_graph;           /* 1: replay steps through CUDA graphs; a whole
                                    rebuild period (R <= 64) is one graph      */
    int32_t bond_tile;           /* bond-kernel threads per point: 32, 64, 128,
                                    256, or 0 to time each on the first call's
                                    bond pass and keep the fastest (results
                                    are bitwise reproducible for a fixed tile).
                                    PPM_MIXED with model 0 outside the coupled
                                    mode: 32 is the warp tensor-core kernel
                                    and 128 the tensor-memory (tcgen05) one,
                                    one thread per bond                       */
    int32_t bc;                  /* boundary conditions: 0 = base layer iz = 0
                                    fixed (the column collapse); 1 = uniaxial
                                    compression along x (Sec. 4.1): the
                                    load_layers planes at ix = 0 are held in x
                                    and those at ix = nx-1 move at v_x =
                                    -load_rate; no fixed base.  lock_lateral
                                    holds x and y in both                     */
    double load_rate;            /* m/s, bc = 1 (>= 0)                          */
    int32_t elastic;             /* 1: linear (hypo-)elastic skeleton, as in the
                                    compression test of Sec. 4.1: the yield test
                                    is switched off (0: critical-state model) */
    int32_t load_layers;         /* bc = 1: lattice planes held / driven at each
                                    x end; 0 = floor(horizon_factor), the
                                    horizon's thickness                        */
    int32_t halt_on_unstable;    /* 1: the Eq. 69 check is a hard stop -- once a
                                    step fails it, later steps change nothing
                                    (PPM_STATUS_HALTED, halted_step); decided
                                    on the device, so it also holds inside CUDA
                                    graphs.  Not with the adjoint calls.      */
    int32_t contact;             /* 1: the column rests on a rigid flat substrate
                                    (Sec. 4.2, Eq. 91-93) instead of a fixed base
                                    layer: the plane z = -contact_cutoff * dx;
                                    a point at distance d < delta_c is pushed
                                    up by C_s dx^2 (delta_c - d) / delta_c and
                                    held by Coulomb friction mu_f on its
                                    tangential velocity.  Not with the adjoint
                                    calls.                                      */
    double contact_modulus;      /* C_s (Pa), contact = 1                      */
    double friction;             /* mu_f, contact = 1                          */
    double contact_cutoff;       /* delta_c / dx, contact = 1                  */
    double energy_tol;           /* the tolerance of the Eq. 69 check (> 0), or
                                    0 for 1e-2; the paper gives its order only */
    int32_t plane_strain;        /* 1: plane strain in the x-z plane, the setting
                                    of the paper's experiments (Sec. 4): y is
                                    periodic with period ny * dx, which must
                                    exceed 4 delta, bond vectors take the
                                    nearest periodic image, and v_y is held at
                                    zero, so a y-invariant start stays
                                    y-invariant.  Single columns only; not
                                    with the adjoint calls                     */
    int32_t coupled;             /* 1: deformation-dependent porosity, degree of
                                    saturation, volume and mass (Eq. 15-16,
                                    48-49): each point carries its volume ratio
                                    J, updated from its bonds' volumetric rate;
                                    phi = 1 - (1 - phi_0) / J; S_r from Eq. 15
                                    (exponent -(n-1)/n, void ratio J / (1 -
                                    phi_0) - 1); V = J dx^3 in the pairwise
                                    force and the mass [rho_s (1 - phi) + rho_w
                                    S_r phi] V, all at J of the start of the
                                    step.  rho and vg_* are then unused.
                                    Single columns only; not with the adjoint */
    double porosity;             /* phi_0 in (0, 1), coupled = 1               */
    double rho_s, rho_w;         /* solid and water densities, coupled = 1     */
    double wr_a1, wr_a2, wr_n;   /* Eq. 15: a1 (1/Pa, > 0), a2 (>= 0), n (> 1) */
    int32_t points_per_block;    /* tensor-core bond kernel (PPM_MIXED, model 0,
                                    bond_tile 32): points (one warp each) per
                                    block, 1 or 2 (0: 1); with bond_tile = 0
                                    the autotuner chooses                      */
    int32_t bond_grid;           /* that kernel's grid: 1 (or 0) one warp per
                                    point; 2 a persistent resident wave of
                                    blocks looping over the points; with
                                    bond_tile = 0 the autotuner chooses        */
    int32_t gather_lanes;        /* force gather: lanes per point, 4 or 8, or 0
                                    for 4 (with bond_tile = 0 the first call
                                    times both and keeps the faster)           */
    int32_t withhold_tc_product; /* fault injection for tests, normally 0.  1:
                                    in every pass of the tensor-memory bond
                                    kernel (bond_tile 128) each CTA's first
                                    product signals a spare mbarrier instead
                                    of the one awaited, so that the wait runs
                                    out after about a second: the pass sets
                                    PPM_STATUS_TC_TIMEOUT and the points it
                                    had not reached keep their state.  The
                                    product still completes (on the spare
                                    barrier), and the context stays usable  */
} ppm_params;

/* one column of a batched ensemble; other parameters come from ppm_params */
typedef struct {
    int32_t nx, ny, nz, pad_;
    double suction, M;
} ppm_column;

typedef struct {
    int64_t steps;               /* steps taken                                 */
    int64_t nbonds;              /* bonds of the current family                 */
    int64_t bond_steps;          /* sum over steps of the bond count            */
    int64_t plastic;             /* bond updates that took the plastic branch   */
    int64_t nonconv;             /* Newton solves that did not converge         */
    int64_t singular;            /* bond updates with a degenerate shape tensor */
    int64_t rebuilds;            /* family searches done                        */
    int64_t pairs;               /* sum over updated bonds of the sub-horizon
                                    size |S_b| (member pairs visited)          */
    int64_t launches;            /* CUDA kernels this context has issued        */
    int64_t returns_fp64;        /* plastic returns solved in FP64 (all of them
                                    in PPM_FP64; in PPM_MIXED those near the
                                    apex or whose FP32 solve failed)           */
    int32_t bond_tile;           /* tile in use                                 */
    int32_t halted_step;         /* PPM_STATUS_HALTED: the step whose energy
                                    check failed (counted from 1), else 0     */
    uint32_t status;             /* PPM_STATUS_* bits                           */
    int32_t unstable_step;       /* PPM_STATUS_UNSTABLE: the first step that
                                    failed the Eq. 69 check (from 1), else 0  */
    double W_int, W_ext, W_kin, W_kin0;   /* Eq. 66-68 (summed over points)   */
    int32_t points_per_block;    /* tensor-core bond kernel: points per block   */
    int32_t bond_blocks;         /* its grid: 0 one warp per point, else the
                                    blocks of the persistent wave (the
                                    tensor-memory kernel, bond_tile 128, always
                                    runs one: its CTAs in flight)              */
    int32_t gather_lanes;        /* force gather: lanes per point in use        */
} ppm_counters;

typedef struct ppm_ctx ppm_ctx;

/* Bytes of device workspace needed for these parameters.  n_columns = 0
 * (cols = NULL) means one column described by p->nx, ny, nz, suction, M.
 * Plumbing of the library (the caller owns the device memory); the paper
 * has no counterpart. */
int ppm_workspace_size(const ppm_params* p, int n_columns, const ppm_column* cols,
                       size_t* bytes);

/* Creates a context on the current CUDA device.  d_workspace: device
 * pointer to at least ppm_workspace_size() bytes, 256-byte aligned.
 * cuda_stream: the cudaStream_t to issue all work on (NULL: default
 * stream).  Initial state (Alg. 2): u = v = a = 0, effective stress
 * per init_stress, pc = -pc0.  The family is not built yet. */
int ppm_init(const ppm_params* p, int n_columns, const ppm_column* cols, void* d_workspace,
             size_t bytes, void* cuda_stream, ppm_ctx** out);

/* Family search in the current configuration (Eq. 1): uniform-grid cell
 * list, then the bond-major CSR family with rows ascending and the reverse
 * index.  Asynchronous. */
int ppm_build_families(ppm_ctx* c);

/* Advances n_steps explicit steps (the time loop of Alg. 2).  The first call
 * applies the boundary conditions to the velocities, builds the family if
 * needed and computes the initial acceleration (Alg. 2).
 * Asynchronous; no host synchronisation. */
int ppm_step(ppm_ctx* c, int n_steps);

/* Like ppm_step but without graph replay, recording CUDA events on the
 * context's stream around each phase and adding the elapsed milliseconds
 * to ms[0] (predictor and, when due, the family search), ms[1] (the fused
 * bond kernel) and ms[2] (gather, corrector and energy terms).
 * Synchronises the stream after every step.  Measurement plumbing: the
 * step it times is ppm_step's; the timing has no counterpart in the paper. */
int ppm_step_timed(ppm_ctx* c, int n_steps, double ms[3]);

/* Adjoint (reverse-mode gradient) of n_steps explicit steps.  The paper has
 * no sensitivity analysis; this exposes the discrete adjoint of the step
 * it defines (Eq. 23-26, 31-32, 40-46, 49-51, 60-64, 73-75), with the
 * families, sub-horizons and elastic/plastic branches of the forward run
 * held fixed.  Single-column contexts, force-state models 0 and 1.
 *
 * ppm_adjoint_workspace_size: device bytes for checkpoints every ckpt_every
 * steps, one segment of step states and the adjoint arrays.
 * ppm_adjoint_forward: from a fresh context (after ppm_init and
 * ppm_write_state of the velocities, before any ppm_step), runs the initial
 * pass and n_steps steps, saving checkpoints in d_ws (caller-allocated,
 * 256-byte aligned, kept until the reverse call).  The context then holds
 * the final state.
 * ppm_adjoint_reverse: given dJ/du of the final displacement (3N doubles,
 * component-major, device or host), recomputes every segment from its
 * checkpoint and sweeps backwards; grad receives dJ/dM, dJ/deta, dJ/ds
 * (suction, through S_r s and the initial stress) and dJ/dpc0.  The context
 * is left at the final state again.  Synchronises the stream. */
int ppm_adjoint_workspace_size(const ppm_ctx* c, int n_steps, int ckpt_every, size_t* bytes);
int ppm_adjoint_forward(ppm_ctx* c, int n_steps, int ckpt_every, void* d_ws, size_t bytes);
int ppm_adjoint_reverse(ppm_ctx* c, const double* dJ_du, int src_is_device, double grad[4]);

/* Copies a state field (PPM_FIELD_*) to dst (device pointer if
 * dst_is_device, else host).  bytes must be at least the field's size.
 * Synchronises the stream when dst is a host pointer.  PPM_FIELD_TFORCE:
 * the step keeps the force states at their reverse slots only (outside the
 * coupled mode), so this call first rebuilds the bond-order copy (one
 * kernel).  Plumbing (state transfer for checkpoints, tests and output);
 * the paper has no counterpart. */
int ppm_read_state(ppm_ctx* c, int field, void* dst, size_t bytes, int dst_is_device);

/* Overwrites a state field from src (same layout and type as read).
 * Writing PPM_FIELD_U marks the family as stale (rebuilt before the next
 * step).  Writing PPM_FIELD_J sets the volume ratio the next step starts
 * from (coupled = 1; it is 1 after ppm_init).  Family fields are
 * read-only.  Plumbing (resume from a checkpoint, set an initial state);
 * the paper has no counterpart. */
int ppm_write_state(ppm_ctx* c, int field, const void* src, size_t bytes, int src_is_device);

/* Critical time step of Eq. 65 over the current family and positions (the
 * family is built first if there is none): the minimum over points with
 * bonds of sqrt(2 rho / sum_j V C / |x_j - x_i|), V = dx^3 (rho: the initial
 * mixture density in the coupled mode), with the
 * bond-based micro-modulus C = 18 K / (pi delta^4).  Eq. 65 as printed
 * multiplies C by |zeta|, which does not give a time; the micro-modulus is
 * divided by the bond length, as in the estimate the paper cites.  *dt is
 * +inf when no point has a bond.  Synchronises the stream. */
int ppm_critical_time_step(ppm_ctx* c, double* dt);

/* Number of bonds of the current family (synchronises the stream).
 * Plumbing; the paper has no counterpart. */
int ppm_num_bonds(ppm_ctx* c, int64_t* nbonds);

/* Synchronises the stream and returns the counters and status word.
 * Plumbing; the paper has no counterpart, except the energy terms of
 * Eq. 66-68 and the check of Eq. 69 that they carry. */
int ppm_status(ppm_ctx* c, ppm_counters* out);

/* Time step in use and total number of points.  Plumbing; the paper
 * has no counterpart. */
int ppm_info(const ppm_ctx* c, double* dt, int64_t* npoints);

/* Family search (as ppm_build_families) of n points with explicit FP64
 * positions, allocating nothing.  The paper has no counterpart of this
 * call; it exists for callers that cannot allocate device memory --
 * real-time loops that must not enter the allocator (cudaMalloc can block
 * and synchronise the device), hosts whose device memory belongs to
 * another allocator or pool.  The caller passes the inputs and outputs;
 * the scratch lives in the library itself.
 *
 *   d_x        device, 3n doubles, component-major (x[c*n + i])
 *   delta      horizon; j is in the family of i iff j != i and
 *              ((dx*dx + dy*dy) + dz*dz) <= delta*delta
 *   max_family most bonds one point may have (1..256); a point with more
 *              gets an empty row and the call returns PPM_ENOSPACE
 *   d_row_ptr  device, n+1 int32 (written); d_col, d_rev: device, cap int32
 *              each (written: rows ascending, rev[b] = index of (j,i))
 *   cuda_stream a stream of the current device (NULL: the default stream)
 *   nbonds     host, may be NULL: bonds found
 * Returns PPM_EINVAL for n < 1 or n > 262,144 points (the size of the
 * built-in scratch), a stream of another device, or bad arguments;
 * PPM_ENOSPACE if the bonds exceed cap (row_ptr is then all zero, *nbonds
 * 0).  The scratch is one fixed array of about 9.5 MB in the library's
 * device image, which every GPU that loads the library holds until exit.
 * Its device address is looked up on the first call on each device, with
 * that device current, and kept (the lookup is guarded for concurrent host
 * threads).  All calls share the array and the array keeps the last call's
 * contents (the call clears what must start at zero): calls that overlap
 * on the GPU race.  The call synchronises the stream to return its status. */
int ppm_family_noalloc(int64_t n, const double* d_x, double delta, int max_family,
                       int32_t* d_row_ptr, int32_t* d_col, int32_t* d_rev, int64_t cap,
                       void* cuda_stream, int64_t* nbonds);

/* Measured FP32 fused multiply-add rate of the current device in TFLOP/s
 * (*tflops): independent FMA chains on every SM, the best of three timed
 * launches on cuda_stream (which it synchronises).  Measurement plumbing
 * with no counterpart in the paper: the benchmark divides the bond
 * kernel's algorithmic FLOP rate by it.  Allocates nothing. */
int ppm_measure_fp32_peak(void* cuda_stream, double* tflops);

/* Text of a return code.  Plumbing; the paper has no counterpart. */
const char* ppm_error_string(int code);

/* sizeof of the ABI structs as compiled into the library, so that a
 * binding can check its own layout: which = 0 ppm_params, 1 ppm_column,
 * 2 ppm_counters; 0 for anything else.  Needs no GPU.  Plumbing; the
 * paper has no counterpart. */
size_t ppm_struct_size(int which);

/* Frees host-side resources (graphs, events).  The workspace stays the
 * caller's.  Plumbing; the paper has no counterpart. */
void ppm_destroy(ppm_ctx* c);

#ifdef __cplusplus
}
#endif
#endif
