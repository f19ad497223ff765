// Host runtime behind the C ABI of include/ppm.h: parameter checks,
// workspace carving (the library never allocates device memory), the step
// sequence of Alg. 2, CUDA-graph replay of whole steps, state transfer and
// the status word.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <cmath>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ppm_internal.cuh"

using namespace ppm;

struct ppm_ctx {
    ppm_params p;
    int ncols;
    std::vector<ColumnConst> cols;
    int64_t N;
    long long cap;
    int ncell_cap;
    int gather_blocks;
    cudaStream_t stream;
    cudaStream_t cap_stream;
    StepConst k;
    DevState<double> sd;
    DevState<float> sf;
    ColumnConst* d_cols;
    bool started;
    bool family_built;
    int64_t step;
    cudaGraphExec_t g_plain, g_rebuild, g_segment;   // one step; one rebuild period
    cudaEvent_t ev[8];
    bool events_ok;
    long long launches;          // kernels issued (graph replays count their kernels)
    long long launches_plain, launches_rebuild, launches_segment;   // kernels per graph
    int segment_len;             // steps in g_segment (the rebuild period)
    // adjoint bookkeeping (ppm_adjoint_forward / ppm_adjoint_reverse)
    bool adj_ready;
    int adj_steps, adj_every, adj_nck, adj_nver;
    char* adj_ws;
    size_t adj_bytes;
};

namespace {

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// NVTX range over a host-side scope (phases of a step, graph launches, the
// family, adjoint and Eq. 65 calls), for timeline profilers; header-only
// NVTX costs a few nanoseconds when no tool is attached
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

// Offsets of every buffer in the caller's workspace.
struct Layout {
    size_t total = 0;
    template <typename T>
    T* take(char* base, size_t count) {
        size_t off = total;
        total = align_up(total + sizeof(T) * (count > 0 ? count : 1), 256);
        return base ? reinterpret_cast<T*>(base + off) : nullptr;
    }
};

double saturation(double s, double alpha, double n) {
    if (s <= 0.0) return 1.0;
    return pow(1.0 + pow(alpha * s, n), -(1.0 - 1.0 / n));
}

// coupled mode (Eq. 15-16, 48) at volume ratio J, on the host: S_r with the
// void ratio J / (1 - phi_0) - 1 and the mixture density per current volume
double coupled_saturation(const ppm_params* p, double J, double s) {
    const double e = J / (1.0 - p->porosity) - 1.0;
    if (!(s > 0.0) || !(e > 0.0)) return 1.0;
    const double alpha = p->wr_a1 * pow(e, p->wr_a2) * J;
    return pow(1.0 + pow(alpha * s, p->wr_n), -(p->wr_n - 1.0) / p->wr_n);
}

double coupled_density(const ppm_params* p, double J, double s) {
    const double phi = 1.0 - (1.0 - p->porosity) / J;
    return p->rho_s * (1.0 - phi) + p->rho_w * coupled_saturation(p, J, s) * phi;
}

int check_params(const ppm_params* p) {
    if (!p) return PPM_EINVAL;
    if (!(p->dx > 0) || !(p->horizon_factor > 0) || !(p->rho > 0)) return PPM_EINVAL;
    if (!(p->K > 0) || !(p->mu > 0) || !(p->M > 0)) return PPM_EINVAL;
    if (!(p->lambda_t > p->kappa_t) || !(p->eta > 0) || !(p->pc0 > 0)) return PPM_EINVAL;
    if (p->b1 != 0.0 || p->b2 != 1.0) return PPM_EINVAL;
    if (p->model < 0 || p->model > 2) return PPM_EINVAL;
    if (p->precision != PPM_FP64 && p->precision != PPM_MIXED) return PPM_EINVAL;
    if (p->newton_max_iter < 1 || !(p->newton_tol > 0)) return PPM_EINVAL;
    if (p->max_family < 0 || p->max_family > kMaxRow) return PPM_EINVAL;
    if (p->bond_tile != 0 && p->bond_tile != 32 && p->bond_tile != 64 && p->bond_tile != 128 &&
        p->bond_tile != 256)
        return PPM_EINVAL;
    if (p->points_per_block < 0 || p->points_per_block > 2 || p->bond_grid < 0 || p->bond_grid > 2)
        return PPM_EINVAL;
    if (p->gather_lanes != 0 && p->gather_lanes != 4 && p->gather_lanes != 8) return PPM_EINVAL;
    if (p->withhold_tc_product != 0 && p->withhold_tc_product != 1) return PPM_EINVAL;
    if (p->rebuild_every < 0 || p->suction < 0 || !(p->vg_n > 1.0) || !(p->vg_alpha >= 0))
        return PPM_EINVAL;
    if ((p->bc != 0 && p->bc != 1) || !(p->load_rate >= 0) || !std::isfinite(p->load_rate))
        return PPM_EINVAL;
    if (p->elastic != 0 && p->elastic != 1) return PPM_EINVAL;
    if (p->load_layers < 0) return PPM_EINVAL;
    if (p->halt_on_unstable != 0 && p->halt_on_unstable != 1) return PPM_EINVAL;
    if (p->contact != 0 && p->contact != 1) return PPM_EINVAL;
    if (!(p->energy_tol >= 0) || !std::isfinite(p->energy_tol)) return PPM_EINVAL;
    if (p->plane_strain != 0 && p->plane_strain != 1) return PPM_EINVAL;
    if (p->coupled != 0 && p->coupled != 1) return PPM_EINVAL;
    if (p->coupled && (!(p->porosity > 0.0 && p->porosity < 1.0) || !(p->rho_s > 0) ||
                       !(p->rho_w >= 0) || !(p->wr_a1 > 0) || !(p->wr_a2 >= 0) || !(p->wr_n > 1) ||
                       !std::isfinite(p->rho_s) || !std::isfinite(p->rho_w) ||
                       !std::isfinite(p->wr_a1) || !std::isfinite(p->wr_a2) || !std::isfinite(p->wr_n)))
        return PPM_EINVAL;
    if (p->contact && (!(p->contact_modulus >= 0) || !(p->friction >= 0) || !(p->contact_cutoff > 0) ||
                       !std::isfinite(p->contact_modulus) || !std::isfinite(p->friction)))
        return PPM_EINVAL;
    return PPM_OK;
}

int collect_columns(const ppm_params* p, int n_columns, const ppm_column* cols,
                    std::vector<ColumnConst>& out, int64_t* N) {
    out.clear();
    int64_t off = 0;
    const int nc = n_columns > 0 ? n_columns : 1;
    if (n_columns > 0 && !cols) return PPM_EINVAL;
    if (p->plane_strain && n_columns > 1) return PPM_EINVAL;      // one periodic slab
    if (p->coupled && n_columns > 1) return PPM_EINVAL;           // one column
    for (int c = 0; c < nc; c++) {
        int nx = n_columns > 0 ? cols[c].nx : p->nx;
        int ny = n_columns > 0 ? cols[c].ny : p->ny;
        int nz = n_columns > 0 ? cols[c].nz : p->nz;
        double s = n_columns > 0 ? cols[c].suction : p->suction;
        double M = n_columns > 0 ? cols[c].M : p->M;
        if (nx < 1 || ny < 1 || nz < 1 || nx > kLatMask + 1 || ny > kLatMask + 1 ||
            nz > kLatMask + 1 || s < 0 || !(M > 0))
            return PPM_EINVAL;
        // plane strain: the y period must exceed 4 delta, so that the nearest
        // images of two members of one family are each other's nearest
        if (p->plane_strain && !((double)ny > 4.0 * p->horizon_factor)) return PPM_EINVAL;
        ColumnConst cc;
        cc.M = M;
        cc.Srs = (p->coupled ? coupled_saturation(p, 1.0, s) : saturation(s, p->vg_alpha, p->vg_n)) * s;
        cc.Mf = (float)cc.M;
        cc.Srsf = (float)cc.Srs;
        cc.nx = nx; cc.ny = ny; cc.nz = nz; cc.pad = 0;
        cc.offset = off;
        out.push_back(cc);
        off += (int64_t)nx * ny * nz;
    }
    *N = off;
    if (off < 1 || off > (1LL << 27)) return PPM_EINVAL;
    return PPM_OK;
}

// shared by ppm_workspace_size and ppm_init
template <typename Real>
void carve(Layout& L, char* base, int64_t N, long long cap, int ncell_cap, int gather_blocks,
           int ncols, bool mixed, DevState<Real>& s, ColumnConst** d_cols) {
    const size_t n = (size_t)N;
    s.xabs = nullptr;
    s.lat = L.take<int32_t>(base, n);
    s.colid = L.take<int32_t>(base, n);
    *d_cols = L.take<ColumnConst>(base, (size_t)ncols);
    s.cols = *d_cols;
    s.u = L.take<Real>(base, 3 * n);
    s.ulo = mixed ? L.take<float>(base, 3 * n) : nullptr;
    s.v = L.take<Real>(base, 3 * n);
    s.vh = L.take<Real>(base, 3 * n);
    s.a = L.take<Real>(base, 3 * n);
    s.sig = L.take<Real>(base, 6 * n);
    s.pc = L.take<Real>(base, n);
    s.eps = L.take<Real>(base, n);
    s.fint = L.take<Real>(base, 3 * n);
    s.tsum = L.take<Real>(base, 3 * n);
    s.J = L.take<Real>(base, n);
    s.Jn = L.take<Real>(base, n);
    s.row_ptr = L.take<int32_t>(base, n + 1);
    s.col = L.take<int32_t>(base, (size_t)cap);
    s.rev = L.take<int32_t>(base, (size_t)cap);
    s.T = L.take<Real>(base, 3 * (size_t)cap);
    s.Trev = L.take<Real>(base, 3 * (size_t)cap);
    s.epart = L.take<double>(base, 3 * (size_t)gather_blocks);
    s.ctr = L.take<DevCounters>(base, 1);
    s.grid = L.take<CellGrid>(base, 1);
    s.bbox = L.take<long long>(base, 6);
    s.cellkey = L.take<int32_t>(base, n);
    s.cellcnt = L.take<int32_t>(base, (size_t)ncell_cap + 1);
    s.cellstart = L.take<int32_t>(base, (size_t)ncell_cap + 1);
    s.cellfill = L.take<int32_t>(base, (size_t)ncell_cap);
    s.sorted = L.take<int32_t>(base, n);
    s.rowlen = L.take<int32_t>(base, n + 1);
    s.scanbuf = L.take<int32_t>(base, 8192);
    s.ncell_cap = ncell_cap;
}

struct Sizes {
    int64_t N;
    long long cap;
    int ncell_cap, gather_blocks, max_family;
};

Sizes sizes_for(const ppm_params* p, int64_t N) {
    Sizes z;
    z.N = N;
    z.max_family = p->max_family > 0 ? p->max_family : kDefaultMaxFamily;
    z.cap = (long long)N * z.max_family;
    if (z.cap > 0x7fffffffLL) z.cap = 0x7fffffffLL;
    z.ncell_cap = (int)((2 * N > 4096) ? 2 * N : 4096);
    // the gather runs kGatherPointsPerBlock points per block
    z.gather_blocks = (int)((N + kGatherPointsPerBlock - 1) / kGatherPointsPerBlock);
    return z;
}

size_t workspace_bytes(const ppm_params* p, int ncols, const Sizes& z) {
    Layout L;
    ColumnConst* dc;
    if (p->precision == PPM_FP64) {
        DevState<double> s;
        carve<double>(L, nullptr, z.N, z.cap, z.ncell_cap, z.gather_blocks, ncols, false, s, &dc);
    } else {
        DevState<float> s;
        carve<float>(L, nullptr, z.N, z.cap, z.ncell_cap, z.gather_blocks, ncols, true, s, &dc);
    }
    return L.total;
}

#define CU(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return PPM_ECUDA; \
    } while (0)

template <typename Real>
int run_family(ppm_ctx* c, const DevState<Real>& s) {
    Range r("ppm family search");
    CU(launch_family_build<Real>(s, c->k, c->stream, &c->launches));
    c->family_built = true;
    return PPM_OK;
}

template <typename Real>
int autotune_tile(ppm_ctx* c, const DevState<Real>& s);

// Eq. 65 over the current family (built first if there is none); the result
// comes back through the first slot of the family search's bounding-box
// scratch, unused between family builds
template <typename Real>
int critical_dt(ppm_ctx* c, const DevState<Real>& s, double* out) {
    if (!c->family_built) {
        int rc = run_family<Real>(c, s);
        if (rc) return rc;
    }
    CU(launch_critical_dt<Real>(s, c->k, s.bbox, c->stream));
    c->launches += 2;
    long long h = 0;
    CU(cudaMemcpyAsync(&h, s.bbox, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (h == 0x7fffffffffffffffLL) {
        *out = INFINITY;
    } else {
        h ^= (h >> 63) & 0x7fffffffffffffffLL;     // back from the ordered encoding
        memcpy(out, &h, sizeof(h));
    }
    return PPM_OK;
}

template <typename Real>
int issue_initial(ppm_ctx* c, const DevState<Real>& s) {
    Range r("ppm initial pass");
    CU(launch_apply_velocity_bc<Real>(s, c->k, c->stream));
    if (!c->family_built) {
        int rc = run_family<Real>(c, s);
        if (rc) return rc;
    }
    if (c->p.bond_tile == 0) {
        int rc = autotune_tile<Real>(c, s);
        if (rc) return rc;
    }
    CU(launch_bond<Real>(s, c->k, 0.0, 0, c->stream));
    if (c->p.bond_tile == 0 && c->p.gather_lanes == 0) {
        // the gather's lanes per point, timed on the initial gather (which
        // only recomputes the initial forces and accelerations: repeating it
        // leaves the same state)
        float best = 1e30f;
        int pick = 4;
        for (int lanes : {4, 8}) {
            c->k.gather_lanes = lanes;
            CU(launch_gather<Real>(s, c->k, 0.0, 1, c->gather_blocks, c->stream));      // warm
            CU(cudaEventRecord(c->ev[4], c->stream));
            for (int r = 0; r < 3; r++) CU(launch_gather<Real>(s, c->k, 0.0, 1, c->gather_blocks, c->stream));
            CU(cudaEventRecord(c->ev[5], c->stream));
            CU(cudaEventSynchronize(c->ev[5]));
            float ms = 0.f;
            CU(cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]));
            c->launches += 4;
            if (ms < best) { best = ms; pick = lanes; }
        }
        c->k.gather_lanes = pick;
    }
    CU(launch_gather<Real>(s, c->k, 0.0, 1, c->gather_blocks, c->stream));
    CU(launch_energy_reduce(s.epart, c->gather_blocks, s.ctr, 1, s.row_ptr, c->k.npoints, c->k.halt,
                            c->k.energy_tol, c->stream));
    c->launches += 4;
    return PPM_OK;
}

// one explicit step (the time loop of Alg. 2) issued on stream st; ev (optional)
// records phase boundaries: 0 start, 1 after predictor+family, 2 after
// bond, 3 after gather
template <typename Real>
int issue_step(ppm_ctx* c, const DevState<Real>& s, bool rebuild, cudaStream_t st,
               cudaEvent_t* ev, long long* nlaunch) {
    if (ev) CU(cudaEventRecord(ev[0], st));
    {
        Range r("ppm predictor");
        CU(launch_predictor<Real>(s, c->k, st));
    }
    if (rebuild) {
        Range r("ppm family search");
        CU(launch_family_build<Real>(s, c->k, st, nlaunch));
    }
    *nlaunch += 4;   // predictor, bond, gather, energy reduction
    if (ev) CU(cudaEventRecord(ev[1], st));
    {
        Range r("ppm bond pass");
        CU(launch_bond<Real>(s, c->k, c->k.dt, 1, st));
    }
    if (ev) CU(cudaEventRecord(ev[2], st));
    {
        Range r("ppm gather and energy");
        CU(launch_gather<Real>(s, c->k, c->k.dt, 0, c->gather_blocks, st));
        CU(launch_energy_reduce(s.epart, c->gather_blocks, s.ctr, 0, s.row_ptr, c->k.npoints,
                                c->k.halt, c->k.energy_tol, st));
    }
    if (ev) CU(cudaEventRecord(ev[3], st));
    return PPM_OK;
}

template <typename Real>
int capture_step(ppm_ctx* c, const DevState<Real>& s, bool rebuild, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    long long nl = 0;
    int rc = issue_step<Real>(c, s, rebuild, c->cap_stream, nullptr, &nl);
    (rebuild ? c->launches_rebuild : c->launches_plain) = nl;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (rc != PPM_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return PPM_ECUDA;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e == cudaSuccess ? PPM_OK : PPM_ECUDA;
}

// a whole rebuild period (a family search, then R - 1 plain steps) as one graph
template <typename Real>
int capture_segment(ppm_ctx* c, const DevState<Real>& s, int len, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    long long nl = 0;
    int rc = PPM_OK;
    for (int q = 0; q < len && rc == PPM_OK; q++)
        rc = issue_step<Real>(c, s, q == 0, c->cap_stream, nullptr, &nl);
    c->launches_segment = nl;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (rc != PPM_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return PPM_ECUDA;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e == cudaSuccess ? PPM_OK : PPM_ECUDA;
}

// Launch shape of the bond pass: time a full bond pass (with the time step,
// so the constitutive update runs, but without committing the point state)
// for each candidate and keep the fastest.  Candidates: 32, 64, 128 and 256
// threads per point; for the mixed path with a sub-horizon force state
// (Eq. 51 or the power-conjugate one), 32 means the tensor-core kernel,
// tried with one and two points per block, each with a grid that covers
// every point once and with a persistent resident wave that loops over
// the points; for the mixed path with Eq. 51 outside the coupled mode, 128
// means the tensor-memory (tcgen05) kernel, one CTA per point.
struct LaunchShape {
    int tile, ppb, blocks;
};

template <typename Real>
int autotune_tile(ppm_ctx* c, const DevState<Real>& s) {
    LaunchShape cand[8];
    int nc = 0;
    const bool tc = sizeof(Real) == 4 && (c->k.model == 0 || c->k.model == 2);
    if (tc) {
        for (int ppb = 1; ppb <= 2; ppb++) {
            int resident = 0;
            CU(bond_tc_resident_blocks(c->k.model, ppb, c->k.coupled, &resident));
            cand[nc++] = {32, ppb, 0};
            cand[nc++] = {32, ppb, resident};
        }
    } else {
        cand[nc++] = {32, 1, 0};
    }
    cand[nc++] = {64, 1, 0};
    cand[nc++] = {128, 1, 0};
    cand[nc++] = {256, 1, 0};
    float best = 1e30f;
    LaunchShape pick = {128, 1, 0};
    for (int q = 0; q < nc; q++) {
        c->k.tile = cand[q].tile;
        c->k.tc_ppb = cand[q].ppb;
        c->k.tc_blocks = cand[q].blocks;
        CU(launch_bond<Real>(s, c->k, c->k.dt, 0, c->stream));      // warm
        CU(cudaEventRecord(c->ev[4], c->stream));
        for (int r = 0; r < 2; r++) CU(launch_bond<Real>(s, c->k, c->k.dt, 0, c->stream));
        CU(cudaEventRecord(c->ev[5], c->stream));
        CU(cudaEventSynchronize(c->ev[5]));
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]));
        c->launches += 3;
        if (ms < best) { best = ms; pick = cand[q]; }
    }
    c->k.tile = pick.tile;
    c->k.tc_ppb = pick.ppb;
    c->k.tc_blocks = pick.blocks;
    return PPM_OK;
}

bool rebuild_due(const ppm_ctx* c) {
    return c->p.rebuild_every > 0 && (c->step + 1) % c->p.rebuild_every == 0;
}

template <typename Real>
int do_steps(ppm_ctx* c, const DevState<Real>& s, int n_steps, double* phase_ms) {
    if (!c->started) {
        int rc = issue_initial<Real>(c, s);
        if (rc) return rc;
        c->started = true;
    }
    const int R = c->p.rebuild_every;
    for (int t = 0; t < n_steps; t++) {
        const bool rebuild = rebuild_due(c);
        if (!phase_ms && c->p.use_graph && rebuild && R > 1 && R <= 64 && n_steps - t >= R) {
            if (!c->g_segment) {
                int rc = capture_segment<Real>(c, s, R, &c->g_segment);
                if (rc) return rc;
                c->segment_len = R;
            }
            {
                Range r("ppm rebuild period (graph)");
                CU(cudaGraphLaunch(c->g_segment, c->stream));
            }
            c->launches += c->launches_segment;
            c->step += R;
            t += R - 1;
            continue;
        }
        if (phase_ms) {
            int rc = issue_step<Real>(c, s, rebuild, c->stream, c->ev, &c->launches);
            if (rc) return rc;
            CU(cudaEventSynchronize(c->ev[3]));
            float ms;
            CU(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1])); phase_ms[0] += ms;
            CU(cudaEventElapsedTime(&ms, c->ev[1], c->ev[2])); phase_ms[1] += ms;
            CU(cudaEventElapsedTime(&ms, c->ev[2], c->ev[3])); phase_ms[2] += ms;
        } else if (c->p.use_graph) {
            cudaGraphExec_t* g = rebuild ? &c->g_rebuild : &c->g_plain;
            if (!*g) {
                int rc = capture_step<Real>(c, s, rebuild, g);
                if (rc) return rc;
            }
            {
                Range r(rebuild ? "ppm step with family search (graph)" : "ppm step (graph)");
                CU(cudaGraphLaunch(*g, c->stream));
            }
            c->launches += rebuild ? c->launches_rebuild : c->launches_plain;
        } else {
            int rc = issue_step<Real>(c, s, rebuild, c->stream, nullptr, &c->launches);
            if (rc) return rc;
        }
        c->step++;
    }
    CU(cudaGetLastError());
    return PPM_OK;
}

struct FieldView {
    void* ptr;
    size_t bytes;
    size_t stride_bytes;   // for TFORCE: bytes between components on device
    int ncomp;
};

int field_view(ppm_ctx* c, int field, int64_t nbonds, FieldView* v) {
    const size_t n = (size_t)c->N;
    const bool f64 = c->p.precision == PPM_FP64;
    const size_t rs = f64 ? sizeof(double) : sizeof(float);
    void* base = nullptr;
    size_t count = 0;
    v->ncomp = 1;
    v->stride_bytes = 0;
#define PICK(member) (f64 ? (void*)c->sd.member : (void*)c->sf.member)
    switch (field) {
        case PPM_FIELD_U: base = PICK(u); count = 3 * n; break;
        case PPM_FIELD_V: base = PICK(v); count = 3 * n; break;
        case PPM_FIELD_A: base = PICK(a); count = 3 * n; break;
        case PPM_FIELD_SIGMA: base = PICK(sig); count = 6 * n; break;
        case PPM_FIELD_PC: base = PICK(pc); count = n; break;
        case PPM_FIELD_EPS_S: base = PICK(eps); count = n; break;
        case PPM_FIELD_FINT: base = PICK(fint); count = 3 * n; break;
        case PPM_FIELD_J: base = PICK(J); count = n; break;
        case PPM_FIELD_ROW_PTR:
            v->ptr = f64 ? (void*)c->sd.row_ptr : (void*)c->sf.row_ptr;
            v->bytes = sizeof(int32_t) * (n + 1);
            return PPM_OK;
        case PPM_FIELD_COL:
            v->ptr = f64 ? (void*)c->sd.col : (void*)c->sf.col;
            v->bytes = sizeof(int32_t) * (size_t)nbonds;
            return PPM_OK;
        case PPM_FIELD_REV:
            v->ptr = f64 ? (void*)c->sd.rev : (void*)c->sf.rev;
            v->bytes = sizeof(int32_t) * (size_t)nbonds;
            return PPM_OK;
        case PPM_FIELD_TFORCE:
            v->ptr = PICK(T);
            v->bytes = rs * (size_t)nbonds;
            v->stride_bytes = rs * (size_t)c->cap;
            v->ncomp = 3;
            return PPM_OK;
        default: return PPM_EINVAL;
    }
#undef PICK
    v->ptr = base;
    v->bytes = rs * count;
    return PPM_OK;
}

int read_nbonds(ppm_ctx* c, int64_t* nb) {
    int32_t* rp = c->p.precision == PPM_FP64 ? c->sd.row_ptr : c->sf.row_ptr;
    int32_t h = 0;
    CU(cudaMemcpyAsync(&h, rp + c->N, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    *nb = h;
    return PPM_OK;
}

}  // namespace

namespace {

// ---- adjoint workspace: checkpoints, one segment of step states, family
// versions, the final forward state and the adjoint arrays ----
struct AdjLayout {
    size_t state_bytes, fam_bytes, total;
    size_t off_ck, off_seg, off_ver, off_final, off_ctr, off_adj, off_acc;
    int nck, nver, every;
};

template <typename Real>
size_t state_bytes_of(int64_t N, bool mixed) {
    const size_t n = (size_t)N;
    return align_up(sizeof(Real) * (3 * 3 * n + 6 * n + n) + (mixed ? sizeof(float) * 3 * n : 0), 256);
}

size_t adj_region_bytes(bool f64, size_t n, size_t cap);

AdjLayout adj_layout(const ppm_ctx* c, int n_steps, int every) {
    AdjLayout L;
    const bool f64 = c->p.precision == PPM_FP64;
    const bool mixed = !f64;
    const size_t n = (size_t)c->N, cap = (size_t)c->cap;
    L.every = every;
    L.state_bytes = f64 ? state_bytes_of<double>(c->N, false) : state_bytes_of<float>(c->N, true);
    L.fam_bytes = align_up(sizeof(int32_t) * (n + 1 + 2 * cap), 256);
    L.nck = (n_steps + every - 1) / every + 1;
    const int rb = c->p.rebuild_every;
    L.nver = rb > 0 ? (every < (every + rb - 1) / rb + 1 ? every : (every + rb - 1) / rb + 1) + 1 : 1;
    size_t off = 0;
    L.off_ck = off; off += (size_t)L.nck * (L.state_bytes + L.fam_bytes);
    L.off_seg = off; off += (size_t)every * L.state_bytes;
    L.off_ver = off; off += (size_t)L.nver * L.fam_bytes;
    L.off_final = off; off += L.state_bytes + L.fam_bytes;
    L.off_ctr = off; off += align_up(sizeof(DevCounters), 256);
    L.off_adj = off;
    off += adj_region_bytes(f64, n, cap);
    L.off_acc = off; off += align_up(sizeof(double) * (kAdjAccDoubles + 5 * kAdjRedBlocks), 256);
    L.total = off;
    (void)mixed;
    return L;
}

template <typename Real>
int copy_state(ppm_ctx* c, const DevState<Real>& s, char* buf, bool save, cudaStream_t st) {
    const size_t n = (size_t)c->N;
    const size_t R = sizeof(Real);
    struct Part { void* p; size_t bytes; } parts[7] = {
        {s.u, R * 3 * n}, {s.v, R * 3 * n}, {s.a, R * 3 * n}, {s.sig, R * 6 * n}, {s.pc, R * n},
        {s.ulo, s.ulo ? sizeof(float) * 3 * n : 0}, {nullptr, 0}};
    size_t off = 0;
    for (int q = 0; parts[q].p; q++) {
        if (!parts[q].bytes) continue;
        if (save) CU(cudaMemcpyAsync(buf + off, parts[q].p, parts[q].bytes, cudaMemcpyDeviceToDevice, st));
        else CU(cudaMemcpyAsync(parts[q].p, buf + off, parts[q].bytes, cudaMemcpyDeviceToDevice, st));
        off += parts[q].bytes;
    }
    return PPM_OK;
}

template <typename Real>
int copy_family(ppm_ctx* c, const DevState<Real>& s, char* buf, bool save, cudaStream_t st) {
    const size_t n = (size_t)c->N, cap = (size_t)c->cap;
    void* parts[3] = {s.row_ptr, s.col, s.rev};
    const size_t bytes[3] = {sizeof(int32_t) * (n + 1), sizeof(int32_t) * cap, sizeof(int32_t) * cap};
    size_t off = 0;
    for (int q = 0; q < 3; q++) {
        if (save) CU(cudaMemcpyAsync(buf + off, parts[q], bytes[q], cudaMemcpyDeviceToDevice, st));
        else CU(cudaMemcpyAsync(parts[q], buf + off, bytes[q], cudaMemcpyDeviceToDevice, st));
        off += bytes[q];
    }
    return PPM_OK;
}

template <typename Real>
void adj_take(Layout& Q, char* base, size_t n, size_t cap, AdjState<Real>& a) {
    a.ub = Q.take<Real>(base, 3 * n); a.vb = Q.take<Real>(base, 3 * n); a.ab = Q.take<Real>(base, 3 * n);
    a.fb = Q.take<Real>(base, 3 * n); a.u1b = Q.take<Real>(base, 3 * n); a.vhb = Q.take<Real>(base, 3 * n);
    a.zsum = Q.take<Real>(base, 3 * n); a.ysum = Q.take<Real>(base, 3 * n);
    a.sb = Q.take<Real>(base, 6 * n); a.sbn = Q.take<Real>(base, 6 * n);
    a.pcb = Q.take<Real>(base, n); a.pcbn = Q.take<Real>(base, n);
    a.Zrev = Q.take<Real>(base, 3 * cap); a.Yrev = Q.take<Real>(base, 3 * cap);
    a.thpart = Q.take<double>(base, 3 * n);
}

size_t adj_region_bytes(bool f64, size_t n, size_t cap) {
    Layout Q;
    if (f64) {
        AdjState<double> a;
        adj_take<double>(Q, nullptr, n, cap, a);
    } else {
        AdjState<float> a;
        adj_take<float>(Q, nullptr, n, cap, a);
    }
    return Q.total;
}

template <typename Real>
AdjState<Real> adj_arrays(ppm_ctx* c, const AdjLayout& L) {
    Layout Q;
    AdjState<Real> a;
    adj_take<Real>(Q, c->adj_ws + L.off_adj, (size_t)c->N, (size_t)c->cap, a);
    return a;
}

template <typename Real>
int adjoint_forward(ppm_ctx* c, const DevState<Real>& s, int n_steps, int every) {
    const AdjLayout L = adj_layout(c, n_steps, every);
    cudaStream_t st = c->stream;
    int rc = issue_initial<Real>(c, s);
    if (rc) return rc;
    c->started = true;
    auto ck = [&](int q) { return c->adj_ws + L.off_ck + (size_t)q * (L.state_bytes + L.fam_bytes); };
    for (int t = 0; t < n_steps; t++) {
        if (t % every == 0) {
            char* b = ck(t / every);
            if ((rc = copy_state<Real>(c, s, b, true, st))) return rc;
            if ((rc = copy_family<Real>(c, s, b + L.state_bytes, true, st))) return rc;
        }
        if ((rc = issue_step<Real>(c, s, rebuild_due(c), st, nullptr, &c->launches))) return rc;
        c->step++;
    }
    char* fin = c->adj_ws + L.off_final;
    if ((rc = copy_state<Real>(c, s, fin, true, st))) return rc;
    if ((rc = copy_family<Real>(c, s, fin + L.state_bytes, true, st))) return rc;
    CU(cudaMemcpyAsync(c->adj_ws + L.off_ctr, s.ctr, sizeof(DevCounters), cudaMemcpyDeviceToDevice, st));
    CU(cudaGetLastError());
    return PPM_OK;
}

double dsrs_ds(const ppm_params* p) {
    const double sct = p->suction, al = p->vg_alpha, nn = p->vg_n, mm = 1.0 - 1.0 / nn;
    if (sct <= 0.0) return 1.0;
    const double base = 1.0 + pow(al * sct, nn);
    const double Sr = pow(base, -mm);
    const double dSr = -mm * pow(base, -mm - 1.0) * nn * pow(al * sct, nn - 1.0) * al;
    return Sr + sct * dSr;
}

template <typename Real>
int adjoint_reverse(ppm_ctx* c, const DevState<Real>& s, const double* d_dJdu, double grad[4]) {
    const int n_steps = c->adj_steps, every = c->adj_every;
    const AdjLayout L = adj_layout(c, n_steps, every);
    cudaStream_t st = c->stream;
    const size_t n = (size_t)c->N;
    AdjState<Real> a = adj_arrays<Real>(c, L);
    double* acc = reinterpret_cast<double*>(c->adj_ws + L.off_acc);
    CU(cudaMemsetAsync(c->adj_ws + L.off_adj, 0, L.off_acc - L.off_adj, st));
    CU(cudaMemsetAsync(acc, 0, 8 * sizeof(double), st));
    CU(launch_convert_adjoint<Real>(d_dJdu, a.ub, 3 * n, st));   // before the segment buffer is reused
    auto ck = [&](int q) { return c->adj_ws + L.off_ck + (size_t)q * (L.state_bytes + L.fam_bytes); };
    std::vector<int> ver_of(every);
    int rc;
    for (int seg = (n_steps - 1) / every; seg >= 0 && n_steps > 0; seg--) {
        const int t0 = seg * every, t1 = (t0 + every < n_steps) ? t0 + every : n_steps;
        char* b = ck(seg);
        if ((rc = copy_state<Real>(c, s, b, false, st))) return rc;
        if ((rc = copy_family<Real>(c, s, b + L.state_bytes, false, st))) return rc;
        if ((rc = copy_family<Real>(c, s, c->adj_ws + L.off_ver, true, st))) return rc;
        int ver = 0;
        c->step = t0;
        for (int t = t0; t < t1; t++) {
            if ((rc = copy_state<Real>(c, s, c->adj_ws + L.off_seg + (size_t)(t - t0) * L.state_bytes, true, st)))
                return rc;
            const bool rb = rebuild_due(c);
            if ((rc = issue_step<Real>(c, s, rb, st, nullptr, &c->launches))) return rc;
            if (rb) {
                ver++;
                if (ver >= L.nver) return PPM_ESTATE;
                if ((rc = copy_family<Real>(c, s, c->adj_ws + L.off_ver + (size_t)ver * L.fam_bytes, true, st)))
                    return rc;
            }
            ver_of[t - t0] = ver;
            c->step++;
        }
        for (int t = t1 - 1; t >= t0; t--) {
            if ((rc = copy_state<Real>(c, s, c->adj_ws + L.off_seg + (size_t)(t - t0) * L.state_bytes, false, st)))
                return rc;
            if ((rc = copy_family<Real>(c, s, c->adj_ws + L.off_ver + (size_t)ver_of[t - t0] * L.fam_bytes, false, st)))
                return rc;
            CU(launch_predictor<Real>(s, c->k, st));
            CU(launch_adjoint_step<Real>(s, a, c->k, acc, 0, st));
            c->launches += 5;
        }
    }
    // reverse of the initial pass, from checkpoint 0 (initial stress and family)
    if ((rc = copy_state<Real>(c, s, ck(0), false, st))) return rc;
    if ((rc = copy_family<Real>(c, s, ck(0) + L.state_bytes, false, st))) return rc;
    CU(launch_adjoint_step<Real>(s, a, c->k, acc, 1, st));
    c->launches += 3;
    double h[5];
    CU(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st));
    // back to the state at the end of the forward run
    char* fin = c->adj_ws + L.off_final;
    if ((rc = copy_state<Real>(c, s, fin, false, st))) return rc;
    if ((rc = copy_family<Real>(c, s, fin + L.state_bytes, false, st))) return rc;
    CU(cudaMemcpyAsync(s.ctr, c->adj_ws + L.off_ctr, sizeof(DevCounters), cudaMemcpyDeviceToDevice, st));
    CU(cudaStreamSynchronize(st));
    c->step = n_steps;
    // initial state: sigma0 = geostatic - S_r s 1 (K0 start), pc = -pc0
    const double srsb = h[2] - (c->p.init_stress == 0 ? h[3] : 0.0);
    grad[0] = h[0];
    grad[1] = h[1];
    grad[2] = srsb * dsrs_ds(&c->p);
    grad[3] = -h[4];
    return PPM_OK;
}

}  // namespace

extern "C" {

int ppm_workspace_size(const ppm_params* p, int n_columns, const ppm_column* cols, size_t* bytes) {
    if (!bytes) return PPM_EINVAL;
    int rc = check_params(p);
    if (rc) return rc;
    std::vector<ColumnConst> cc;
    int64_t N = 0;
    rc = collect_columns(p, n_columns, cols, cc, &N);
    if (rc) return rc;
    Sizes z = sizes_for(p, N);
    *bytes = workspace_bytes(p, (int)cc.size(), z);
    return PPM_OK;
}

int ppm_init(const ppm_params* p, int n_columns, const ppm_column* cols, void* d_workspace,
             size_t bytes, void* cuda_stream, ppm_ctx** out) {
    if (!out) return PPM_EINVAL;
    *out = nullptr;
    int rc = check_params(p);
    if (rc) return rc;
    if (!d_workspace || ((uintptr_t)d_workspace & 255u)) return PPM_EINVAL;
    ppm_ctx* c = new (std::nothrow) ppm_ctx();
    if (!c) return PPM_EINVAL;
    c->p = *p;
    rc = collect_columns(p, n_columns, cols, c->cols, &c->N);
    if (rc) { delete c; return rc; }
    c->ncols = (int)c->cols.size();
    Sizes z = sizes_for(p, c->N);
    if (bytes < workspace_bytes(p, c->ncols, z)) { delete c; return PPM_ENOSPACE; }
    c->cap = z.cap;
    c->ncell_cap = z.ncell_cap;
    c->gather_blocks = z.gather_blocks;
    c->stream = (cudaStream_t)cuda_stream;
    Layout L;
    char* base = (char*)d_workspace;
    const bool mixed = p->precision == PPM_MIXED;
    if (mixed) carve<float>(L, base, c->N, c->cap, c->ncell_cap, c->gather_blocks, c->ncols, true, c->sf, &c->d_cols);
    else carve<double>(L, base, c->N, c->cap, c->ncell_cap, c->gather_blocks, c->ncols, false, c->sd, &c->d_cols);

    // step constants
    StepConst& k = c->k;
    memset(&k, 0, sizeof(k));
    const double delta = p->horizon_factor * p->dx;
    k.dx = p->dx;
    k.inv_dx = 1.0 / p->dx;
    k.delta2 = delta * delta;
    k.hf2f = (float)(p->horizon_factor * p->horizon_factor);
    // the mixture density at the start (coupled mode: of J = 1)
    const double rho0 = p->coupled ? coupled_density(p, 1.0, p->suction) : p->rho;
    k.dt = p->dt > 0 ? p->dt : 0.3 * p->dx / sqrt((p->K + 4.0 * p->mu / 3.0) / rho0);
    k.rho = rho0; k.K = p->K; k.mu = p->mu;
    k.coupled = p->coupled;
    k.phi0 = p->porosity; k.rho_s = p->rho_s; k.rho_w = p->rho_w;
    k.wr_a1 = p->wr_a1; k.wr_a2 = p->wr_a2; k.wr_n = p->wr_n; k.wr_s = p->suction;
    k.phi0f = (float)k.phi0; k.rho_sf = (float)k.rho_s; k.rho_wf = (float)k.rho_w;
    k.wr_a1f = (float)k.wr_a1; k.wr_a2f = (float)k.wr_a2; k.wr_nf = (float)k.wr_n;
    k.wr_sf = (float)k.wr_s;
    k.lk = p->lambda_t - p->kappa_t;
    k.eta = p->eta;
    k.tol = p->newton_tol;
    for (int d = 0; d < 3; d++) k.g[d] = p->gravity[d];
    k.visc_form = p->visc_form;
    k.max_iter = p->newton_max_iter;
    k.model = p->model;
    k.lock_lateral = p->lock_lateral;
    k.bc = p->bc;
    k.load_rate = p->load_rate;
    k.load_ratef = (float)p->load_rate;
    k.elastic = p->elastic;
    k.halt = p->halt_on_unstable;
    k.energy_tol = p->energy_tol > 0 ? p->energy_tol : 1e-2;
    k.pbc_ny = p->plane_strain ? c->cols[0].ny : 0;
    k.pair_dc = p->contact_cutoff;
    k.pair_kappa = p->contact ? p->contact_modulus / (2.0 * p->contact_cutoff) : 0.0;
    k.pair_dcf = (float)k.pair_dc;
    k.pair_kappaf = (float)k.pair_kappa;
    k.pbc_L = (double)k.pbc_ny * p->dx;
    k.contact = p->contact;
    k.contact_modulus = p->contact_modulus;
    k.friction = p->friction;
    k.contact_dc = p->contact_cutoff * p->dx;
    k.contact_kf = (float)(p->contact_modulus * p->dx * p->dx);
    k.frictionf = (float)p->friction;
    k.contact_dcf = (float)(p->contact_cutoff * p->dx);
    k.load_layers = p->load_layers > 0 ? p->load_layers : (int)p->horizon_factor;
    if (k.load_layers < 1) k.load_layers = 1;
    k.npoints = (int)c->N;
    k.ncols = c->ncols;
    k.max_family = z.max_family;
    k.tile = p->bond_tile ? p->bond_tile : 128;
    k.tc_ppb = p->points_per_block == 2 ? 2 : 1;
    k.tc_blocks = 0;
    if (p->bond_grid == 2 && p->precision == PPM_MIXED) {
        int resident = 0;
        if (bond_tc_resident_blocks(p->model, k.tc_ppb, p->coupled, &resident) != cudaSuccess) {
            delete c;
            return PPM_ECUDA;
        }
        k.tc_blocks = resident;
    }
    k.gather_lanes = p->gather_lanes == 8 ? 8 : 4;
    k.t5_withhold = p->withhold_tc_product;
    k.t5_blocks = 0;
    if (p->precision == PPM_MIXED && p->model == 0 && !p->coupled) {
        if (bond_t5_prepare(&k.t5_blocks) != cudaSuccess) {
            delete c;
            return PPM_ECUDA;
        }
    }
    k.cap = c->cap;
    k.dxf = (float)k.dx;
    k.inv_dxf = (float)k.inv_dx;
    k.dtf = (float)k.dt;
    k.hdtf = (float)(0.5 * k.dt);
    k.Kf = (float)k.K;
    k.muf = (float)k.mu;
    k.rhof = (float)k.rho;
    k.inv_rho_dxf = (float)(1.0 / (k.rho * k.dx));
    k.dx2f = (float)(k.dx * k.dx);
    k.massf = (float)(k.rho * k.dx * k.dx * k.dx);
    k.etaf = (float)k.eta;
    for (int d = 0; d < 3; d++) k.gf[d] = (float)k.g[d];

    // lattice indices and column ids (host-built, copied once)
    std::vector<int32_t> lat((size_t)c->N), colid((size_t)c->N);
    for (int ci = 0; ci < c->ncols; ci++) {
        const ColumnConst& cc = c->cols[ci];
        int64_t id = cc.offset;
        for (int iz = 0; iz < cc.nz; iz++)
            for (int iy = 0; iy < cc.ny; iy++)
                for (int ix = 0; ix < cc.nx; ix++, id++) {
                    lat[(size_t)id] = ix | (iy << kLatBits) | (iz << (2 * kLatBits));
                    colid[(size_t)id] = ci;
                }
    }
    int32_t* d_lat = mixed ? c->sf.lat : c->sd.lat;
    int32_t* d_colid = mixed ? c->sf.colid : c->sd.colid;
    DevCounters* d_ctr = mixed ? c->sf.ctr : c->sd.ctr;
    cudaError_t e = cudaSuccess;
    e = cudaMemcpyAsync(d_lat, lat.data(), sizeof(int32_t) * lat.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_colid, colid.data(), sizeof(int32_t) * colid.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_cols, c->cols.data(), sizeof(ColumnConst) * c->cols.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_ctr, 0, sizeof(DevCounters), c->stream);
    int32_t* rp = mixed ? c->sf.row_ptr : c->sd.row_ptr;
    if (e == cudaSuccess) e = cudaMemsetAsync(rp, 0, sizeof(int32_t) * ((size_t)c->N + 1), c->stream);
    if (e == cudaSuccess) {
        e = mixed ? launch_init_state<float>(c->sf, k, p->init_stress, p->pc0, c->stream)
                  : launch_init_state<double>(c->sd, k, p->init_stress, p->pc0, c->stream);
    }
    // host copies of lat/colid must outlive the async copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    c->events_ok = true;
    for (int q = 0; q < 8 && e == cudaSuccess; q++) e = cudaEventCreate(&c->ev[q]);
    if (e != cudaSuccess) {
        delete c;
        return PPM_ECUDA;
    }
    c->started = false;
    c->family_built = false;
    c->step = 0;
    c->g_plain = nullptr;
    c->g_rebuild = nullptr;
    c->g_segment = nullptr;
    c->segment_len = 0;
    c->adj_ready = false;
    c->launches = 1;   // initial-state kernel
    *out = c;
    return PPM_OK;
}

int ppm_build_families(ppm_ctx* c) {
    if (!c) return PPM_EINVAL;
    return c->p.precision == PPM_FP64 ? run_family<double>(c, c->sd) : run_family<float>(c, c->sf);
}

int ppm_step(ppm_ctx* c, int n_steps) {
    if (!c || n_steps < 0) return PPM_EINVAL;
    Range r("ppm_step");
    return c->p.precision == PPM_FP64 ? do_steps<double>(c, c->sd, n_steps, nullptr)
                                      : do_steps<float>(c, c->sf, n_steps, nullptr);
}

/* Like ppm_step, without graphs, timing each phase with CUDA events on the
 * context's stream: ms[0] predictor (+ family search when due), ms[1] the
 * fused bond kernel, ms[2] gather + corrector + energies (accumulated). */
int ppm_step_timed(ppm_ctx* c, int n_steps, double* ms) {
    if (!c || n_steps < 0 || !ms) return PPM_EINVAL;
    return c->p.precision == PPM_FP64 ? do_steps<double>(c, c->sd, n_steps, ms)
                                      : do_steps<float>(c, c->sf, n_steps, ms);
}

int ppm_critical_time_step(ppm_ctx* c, double* dt) {
    if (!c || !dt) return PPM_EINVAL;
    Range r("ppm_critical_time_step");
    return c->p.precision == PPM_FP64 ? critical_dt<double>(c, c->sd, dt)
                                      : critical_dt<float>(c, c->sf, dt);
}

int ppm_num_bonds(ppm_ctx* c, int64_t* nbonds) {
    if (!c || !nbonds) return PPM_EINVAL;
    return read_nbonds(c, nbonds);
}

int ppm_read_state(ppm_ctx* c, int field, void* dst, size_t bytes, int dst_is_device) {
    if (!c || !dst) return PPM_EINVAL;
    int64_t nb = 0;
    if (field == PPM_FIELD_COL || field == PPM_FIELD_REV || field == PPM_FIELD_TFORCE) {
        int rc = read_nbonds(c, &nb);
        if (rc) return rc;
    }
    FieldView v;
    int rc = field_view(c, field, nb, &v);
    if (rc) return rc;
    if (bytes < v.bytes * (size_t)v.ncomp) return PPM_EINVAL;
    // the step keeps only the reverse-slot copy of the force states (outside
    // the coupled mode): the bond-order copy is rebuilt here
    if (field == PPM_FIELD_TFORCE && !c->p.coupled) {
        if (c->p.precision == PPM_FP64) CU(launch_tforce_from_rev<double>(c->sd, c->k, nb, c->stream));
        else CU(launch_tforce_from_rev<float>(c->sf, c->k, nb, c->stream));
        c->launches += 1;
    }
    const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int q = 0; q < v.ncomp; q++)
        CU(cudaMemcpyAsync((char*)dst + q * v.bytes, (char*)v.ptr + q * v.stride_bytes, v.bytes,
                           kind, c->stream));
    if (!dst_is_device) CU(cudaStreamSynchronize(c->stream));
    return PPM_OK;
}

int ppm_write_state(ppm_ctx* c, int field, const void* src, size_t bytes, int src_is_device) {
    if (!c || !src) return PPM_EINVAL;
    if (field == PPM_FIELD_ROW_PTR || field == PPM_FIELD_COL || field == PPM_FIELD_REV ||
        field == PPM_FIELD_TFORCE)
        return PPM_EINVAL;
    FieldView v;
    int rc = field_view(c, field, 0, &v);
    if (rc) return rc;
    if (bytes < v.bytes) return PPM_EINVAL;
    const cudaMemcpyKind kind = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CU(cudaMemcpyAsync(v.ptr, src, v.bytes, kind, c->stream));
    if (field == PPM_FIELD_U && c->p.precision == PPM_MIXED)
        CU(cudaMemsetAsync(c->sf.ulo, 0, sizeof(float) * 3 * (size_t)c->N, c->stream));
    if (!src_is_device) CU(cudaStreamSynchronize(c->stream));
    return PPM_OK;
}

int ppm_status(ppm_ctx* c, ppm_counters* out) {
    if (!c || !out) return PPM_EINVAL;
    DevCounters h;
    DevCounters* d = c->p.precision == PPM_FP64 ? c->sd.ctr : c->sf.ctr;
    CU(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    int64_t nb = 0;
    int rc = read_nbonds(c, &nb);
    if (rc) return rc;
    memset(out, 0, sizeof(*out));
    out->steps = c->step;
    out->nbonds = nb;
    out->bond_steps = (int64_t)h.bond_steps;
    out->plastic = (int64_t)h.plastic;
    out->nonconv = (int64_t)h.nonconv;
    out->singular = (int64_t)h.singular;
    out->rebuilds = (int64_t)h.rebuilds;
    out->pairs = (int64_t)h.pairs;
    out->returns_fp64 = (int64_t)h.ret64;
    out->bond_tile = c->k.tile;
    out->points_per_block = c->k.tc_ppb;
    // the persistent grid in use: the tensor-memory kernel's, or the warp kernel's
    const bool t5 = c->k.tile == 128 && c->k.t5_blocks > 0 && c->k.model == 0 && !c->k.coupled;
    out->bond_blocks = t5 ? c->k.t5_blocks : c->k.tc_blocks;
    out->gather_lanes = c->k.gather_lanes;
    out->halted_step = (int32_t)h.halted_step;
    out->unstable_step = (int32_t)h.unstable_step;
    out->launches = c->launches;
    out->status = h.status;
    out->W_int = h.W_int;
    out->W_ext = h.W_ext;
    out->W_kin = h.W_kin;
    out->W_kin0 = h.W_kin0;
    return PPM_OK;
}

int ppm_info(const ppm_ctx* c, double* dt, int64_t* npoints) {
    if (!c) return PPM_EINVAL;
    if (dt) *dt = c->k.dt;
    if (npoints) *npoints = c->N;
    return PPM_OK;
}

const char* ppm_error_string(int code) {
    switch (code) {
        case PPM_OK: return "ok";
        case PPM_EINVAL: return "invalid argument or parameter";
        case PPM_ENOSPACE: return "workspace smaller than ppm_workspace_size()";
        case PPM_ECUDA: return "a CUDA runtime call failed";
        case PPM_ESTATE: return "call not valid in the context's current state";
        default: return "unknown error";
    }
}

int ppm_adjoint_workspace_size(const ppm_ctx* c, int n_steps, int ckpt_every, size_t* bytes) {
    if (!c || !bytes || n_steps < 0 || ckpt_every < 1) return PPM_EINVAL;
    *bytes = adj_layout(c, n_steps, ckpt_every).total;
    return PPM_OK;
}

int ppm_adjoint_forward(ppm_ctx* c, int n_steps, int ckpt_every, void* d_ws, size_t bytes) {
    if (!c || n_steps < 0 || ckpt_every < 1 || !d_ws || ((uintptr_t)d_ws & 255u)) return PPM_EINVAL;
    if (c->started || c->ncols != 1 || c->p.model == 2 || c->p.halt_on_unstable || c->p.contact ||
        c->p.plane_strain || c->p.coupled)
        return PPM_ESTATE;
    if (bytes < adj_layout(c, n_steps, ckpt_every).total) return PPM_ENOSPACE;
    Range r("ppm_adjoint_forward");
    c->adj_ws = (char*)d_ws;
    c->adj_bytes = bytes;
    c->adj_steps = n_steps;
    c->adj_every = ckpt_every;
    int rc = c->p.precision == PPM_FP64 ? adjoint_forward<double>(c, c->sd, n_steps, ckpt_every)
                                        : adjoint_forward<float>(c, c->sf, n_steps, ckpt_every);
    c->adj_ready = rc == PPM_OK;
    return rc;
}

int ppm_adjoint_reverse(ppm_ctx* c, const double* dJ_du, int src_is_device, double grad[4]) {
    if (!c || !dJ_du || !grad) return PPM_EINVAL;
    if (!c->adj_ready) return PPM_ESTATE;
    Range r("ppm_adjoint_reverse");
    const AdjLayout L = adj_layout(c, c->adj_steps, c->adj_every);
    const double* d_src = dJ_du;
    if (!src_is_device) {
        // stage the host values in the segment buffer (at least 3N doubles)
        double* stage = reinterpret_cast<double*>(c->adj_ws + L.off_seg);
        CU(cudaMemcpyAsync(stage, dJ_du, sizeof(double) * 3 * (size_t)c->N, cudaMemcpyHostToDevice,
                           c->stream));
        CU(cudaStreamSynchronize(c->stream));
        d_src = stage;
    }
    return c->p.precision == PPM_FP64 ? adjoint_reverse<double>(c, c->sd, d_src, grad)
                                      : adjoint_reverse<float>(c, c->sf, d_src, grad);
}

size_t ppm_struct_size(int which) {
    switch (which) {
        case 0: return sizeof(ppm_params);
        case 1: return sizeof(ppm_column);
        case 2: return sizeof(ppm_counters);
        default: return 0;
    }
}

void ppm_destroy(ppm_ctx* c) {
    if (!c) return;
    if (c->g_plain) cudaGraphExecDestroy(c->g_plain);
    if (c->g_rebuild) cudaGraphExecDestroy(c->g_rebuild);
    if (c->g_segment) cudaGraphExecDestroy(c->g_segment);
    for (int q = 0; q < 8; q++)
        if (c->ev[q]) cudaEventDestroy(c->ev[q]);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

}  // extern "C"
