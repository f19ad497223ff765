// Family search in the current configuration (Eq. 1; the family of Alg. 1) on a
// uniform cell grid, producing a bond-major CSR family with ascending rows
// and the reverse index rev[b] = position of bond (j, i) in row j.
//
// Pipeline (all sized by the point count, no host round trip):
//   bounding box -> grid (cell edge >= delta) -> cell histogram -> scan ->
//   scatter -> per-point count over the 27 neighbouring cells -> scan ->
//   per-point fill and in-warp rank sort -> reverse index by bisection.
// Points of different columns never bond: the cell key includes the column.
#include <cuda_runtime.h>
#include <cmath>

#include "ppm_internal.cuh"

namespace ppm {
namespace {

template <typename Real>
__device__ __forceinline__ int lat_of(const DevState<Real>& s, int i) { return s.lat ? s.lat[i] : 0; }
template <typename Real>
__device__ __forceinline__ int col_of(const DevState<Real>& s, int i) { return s.colid ? s.colid[i] : 0; }

template <typename Real>
struct Geometry;

// FP64: absolute positions x = X0 + u with X0 = (double)ix * dx, and the
// membership test |x_j - x_i|^2 <= delta^2 evaluated as ((d0*d0 + d1*d1) +
// d2*d2) with every operation rounded separately, so that a CPU program
// doing the same arithmetic gets the same bit pattern.
template <>
struct Geometry<double> {
    static __device__ __forceinline__ double pos(const DevState<double>& s, const StepConst& k,
                                                 int i, int c, int l) {
        if (s.xabs) return s.xabs[(size_t)c * k.npoints + i];
        int ic = c == 0 ? lat_x(l) : (c == 1 ? lat_y(l) : lat_z(l));
        return __dadd_rn(__dmul_rn((double)ic, k.dx), s.u[(size_t)c * k.npoints + i]);
    }
    static __device__ __forceinline__ bool within(const DevState<double>& s, const StepConst& k,
                                                  int i, int li, int j, int lj) {
        double d0 = __dsub_rn(pos(s, k, j, 0, lj), pos(s, k, i, 0, li));
        double d1 = __dsub_rn(image_y(s, k, j, lj, li), pos(s, k, i, 1, li));
        double d2 = __dsub_rn(pos(s, k, j, 2, lj), pos(s, k, i, 2, li));
        double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
        return r2 <= k.delta2;
    }
    // y of the image of j nearest to i (plane strain), y_j + s L
    static __device__ __forceinline__ double image_y(const DevState<double>& s, const StepConst& k,
                                                     int j, int lj, int li) {
        const double y = pos(s, k, j, 1, lj);
        const int sh = image_shift(k, lj, li);
        return sh ? __dadd_rn(y, (double)sh * k.pbc_L) : y;
    }
};

// Mixed: the bond vector in lattice units, zeta~ = (I_j - I_i) + (u_j -
// u_i) / dx in FP32, tested against (delta / dx)^2 -- the same expression
// the bond kernel uses for its sub-horizon test.
template <>
struct Geometry<float> {
    static __device__ __forceinline__ double pos(const DevState<float>& s, const StepConst& k,
                                                 int i, int c, int l) {
        int ic = c == 0 ? lat_x(l) : (c == 1 ? lat_y(l) : lat_z(l));
        return (double)ic * k.dx + (double)s.u[(size_t)c * k.npoints + i];
    }
    static __device__ __forceinline__ bool within(const DevState<float>& s, const StepConst& k,
                                                  int i, int li, int j, int lj) {
        const float inv = (float)k.inv_dx;
        const size_t n = (size_t)k.npoints;
        float z0 = (float)(lat_x(lj) - lat_x(li)) + (s.u[j] - s.u[i]) * inv;
        float z1 = (float)(lat_y(lj) - lat_y(li) + image_shift(k, lj, li) * k.pbc_ny) +
                   (s.u[n + j] - s.u[n + i]) * inv;
        float z2 = (float)(lat_z(lj) - lat_z(li)) + (s.u[2 * n + j] - s.u[2 * n + i]) * inv;
        return z0 * z0 + z1 * z1 + z2 * z2 <= k.hf2f;
    }
    static __device__ __forceinline__ double image_y(const DevState<float>& s, const StepConst& k,
                                                     int j, int lj, int li) {
        return pos(s, k, j, 1, lj) + (double)image_shift(k, lj, li) * k.pbc_L;
    }
};

__device__ __forceinline__ long long ordered(double x) {
    long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double unordered(long long b) {
    b ^= (b >> 63) & 0x7fffffffffffffffLL;
    return __longlong_as_double(b);
}

__global__ void k_bbox_reset(long long* bbox, unsigned long long* rebuilds) {
    if (threadIdx.x < 3) bbox[threadIdx.x] = 0x7fffffffffffffffLL;
    else if (threadIdx.x < 6) bbox[threadIdx.x] = (long long)0x8000000000000000ULL;
    if (threadIdx.x == 0) *rebuilds += 1;
}

template <typename Real>
__global__ void k_bbox(DevState<Real> s, StepConst k) {
    long long mn[3], mx[3];
    for (int c = 0; c < 3; c++) {
        mn[c] = 0x7fffffffffffffffLL;
        mx[c] = (long long)0x8000000000000000ULL;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k.npoints; i += gridDim.x * blockDim.x) {
        int l = lat_of(s, i);
        for (int c = 0; c < 3; c++) {
            long long o = ordered(Geometry<Real>::pos(s, k, i, c, l));
            mn[c] = min(mn[c], o);
            mx[c] = max(mx[c], o);
        }
    }
    for (int c = 0; c < 3; c++) {
        for (int off = 16; off > 0; off >>= 1) {
            mn[c] = min(mn[c], (long long)__shfl_down_sync(0xffffffffu, mn[c], off));
            mx[c] = max(mx[c], (long long)__shfl_down_sync(0xffffffffu, mx[c], off));
        }
    }
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < 3; c++) {
            atomicMin(&s.bbox[c], mn[c]);
            atomicMax(&s.bbox[3 + c], mx[c]);
        }
}

// cell edge >= delta, grown while the grid would exceed the cell capacity;
// a single cell per column if nothing fits (non-finite positions)
__global__ void k_grid_setup(const long long* bbox, CellGrid* g, double delta, int ncols,
                             int ncell_cap, int periodic_y) {
    double lo[3], ext[3];
    for (int c = 0; c < 3; c++) {
        double a = unordered(bbox[c]), b = unordered(bbox[3 + c]);
        if (!(a <= b) || !(b - a < 1e30)) { a = 0.0; b = 0.0; }
        lo[c] = a;
        ext[c] = b - a;
    }
    double h = delta * (1.0 + 1e-9);
    int d[3] = {1, 1, 1};
    bool fits = false;
    for (int it = 0; it < 400 && !fits; it++) {
        double tot = (double)ncols;
        for (int c = 0; c < 3; c++) {
            // periodic y (plane strain): one cell spans the period and the
            // images are taken per pair
            d[c] = (c == 1 && periodic_y) ? 1 : (int)fmin(ext[c] / h, 1e9) + 3;
            tot *= (double)d[c];
        }
        fits = tot <= (double)ncell_cap;
        if (!fits) h *= 1.25;
    }
    if (!fits) { d[0] = d[1] = d[2] = 1; h = 1e300; }
    for (int c = 0; c < 3; c++) g->lo[c] = lo[c] - h;
    g->h = h;
    g->inv_h = 1.0 / h;
    g->dims[0] = d[0]; g->dims[1] = d[1]; g->dims[2] = d[2];
    g->ncell = d[0] * d[1] * d[2];
}

template <typename Real>
__device__ __forceinline__ void cell_of(const DevState<Real>& s, const StepConst& k,
                                        const CellGrid& g, int i, int l, int cc[3]) {
    for (int c = 0; c < 3; c++) {
        double q = (Geometry<Real>::pos(s, k, i, c, l) - g.lo[c]) * g.inv_h;
        int v = (q >= 0.0 && q < 2e9) ? (int)q : 0;
        cc[c] = min(max(v, 0), g.dims[c] - 1);
    }
}

template <typename Real>
__global__ void k_cell_count(DevState<Real> s, StepConst k) {
    const CellGrid g = *s.grid;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k.npoints; i += gridDim.x * blockDim.x) {
        int cc[3];
        cell_of(s, k, g, i, lat_of(s, i), cc);
        int key = col_of(s, i) * g.ncell + (cc[2] * g.dims[1] + cc[1]) * g.dims[0] + cc[0];
        s.cellkey[i] = key;
        atomicAdd(&s.cellcnt[key], 1);
    }
}

template <typename Real>
__global__ void k_cell_scatter(DevState<Real> s, StepConst k) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k.npoints; i += gridDim.x * blockDim.x) {
        int key = s.cellkey[i];
        int pos = s.cellstart[key] + atomicAdd(&s.cellfill[key], 1);
        s.sorted[pos] = i;
    }
}

// Visit every candidate j of point i in the 27 neighbouring cells; calls
// fn(mask_of_members, j) once per 32-candidate slab (warp-synchronous).
template <typename Real, typename Fn>
__device__ __forceinline__ void for_each_member(const DevState<Real>& s, const StepConst& k,
                                                const CellGrid& g, int i, int li, Fn fn) {
    const int lane = threadIdx.x & 31;
    int cc[3];
    cell_of(s, k, g, i, li, cc);
    const int base = col_of(s, i) * g.ncell;
    for (int dz = -1; dz <= 1; dz++) {
        int z = cc[2] + dz;
        if (z < 0 || z >= g.dims[2]) continue;
        for (int dy = -1; dy <= 1; dy++) {
            int y = cc[1] + dy;
            if (y < 0 || y >= g.dims[1]) continue;
            for (int dxx = -1; dxx <= 1; dxx++) {
                int x = cc[0] + dxx;
                if (x < 0 || x >= g.dims[0]) continue;
                int key = base + (z * g.dims[1] + y) * g.dims[0] + x;
                int a = s.cellstart[key], b = s.cellstart[key + 1];
                for (int t = a; t < b; t += 32) {
                    int idx = t + lane;
                    int j = -1;
                    bool ok = false;
                    if (idx < b) {
                        j = s.sorted[idx];
                        ok = (j != i) && Geometry<Real>::within(s, k, i, li, j, lat_of(s, j));
                    }
                    unsigned m = __ballot_sync(0xffffffffu, ok);
                    fn(m, j, ok);
                }
            }
        }
    }
}

template <typename Real>
__global__ void k_family_count(DevState<Real> s, StepConst k) {
    const CellGrid g = *s.grid;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int i = warp; i < k.npoints; i += nwarps) {
        int cnt = 0;
        for_each_member(s, k, g, i, lat_of(s, i), [&](unsigned m, int, bool) { cnt += __popc(m); });
        if (lane == 0) {
            if (cnt > k.max_family) {
                atomicOr(&s.ctr->status, PPM_STATUS_ROW_FULL);
                cnt = 0;
            }
            s.rowlen[i] = cnt;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) s.rowlen[k.npoints] = 0;
}

__global__ void k_family_guard(const int32_t* row_ptr, int n, long long cap, DevCounters* ctr) {
    long long total = row_ptr[n];
    int ok = total <= cap;
    ctr->family_ok = ok;
    if (!ok) atomicOr(&ctr->status, PPM_STATUS_FAMILY_FULL);
}

__global__ void k_family_zero_if_full(int32_t* row_ptr, int n, const DevCounters* ctr) {
    if (ctr->family_ok) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x)
        row_ptr[i] = 0;
}

template <typename Real>
__global__ void __launch_bounds__(kWarpPointsPerBlock * 32)
k_family_fill(DevState<Real> s, StepConst k) {
    __shared__ int buf[kWarpPointsPerBlock][kMaxRow];
    if (!s.ctr->family_ok) return;
    const CellGrid g = *s.grid;
    const int wib = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    int* mybuf = buf[wib];
    for (int i = warp; i < k.npoints; i += nwarps) {
        const int r0 = s.row_ptr[i];
        const int len = s.row_ptr[i + 1] - r0;
        if (len == 0) continue;
        int found = 0;
        for_each_member(s, k, g, i, lat_of(s, i), [&](unsigned m, int j, bool ok) {
            int pos = found + __popc(m & ((1u << lane) - 1u));
            if (ok && pos < kMaxRow) mybuf[pos] = j;
            found += __popc(m);
        });
        __syncwarp();
        const int nf = min(found, len);
        // rank sort: every member is distinct, so its rank is its position
        for (int t = lane; t < nf; t += 32) {
            int e = mybuf[t];
            int rank = 0;
            for (int u = 0; u < nf; u++) rank += (mybuf[u] < e);
            s.col[r0 + rank] = e;
        }
        __syncwarp();
    }
}

template <typename Real>
__global__ void k_family_rev(DevState<Real> s, StepConst k) {
    if (!s.ctr->family_ok) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int i = warp; i < k.npoints; i += nwarps) {
        const int r0 = s.row_ptr[i], r1 = s.row_ptr[i + 1];
        for (int b = r0 + lane; b < r1; b += 32) {
            int j = s.col[b];
            int lo = s.row_ptr[j], hi = s.row_ptr[j + 1];
            const int end = hi;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (s.col[mid] < i) lo = mid + 1;
                else hi = mid;
            }
            const int rb = (lo < end && s.col[lo] == i) ? lo : -1;
            s.rev[b] = rb;
            // a bond without a reverse partner receives no force state
            if (rb < 0 && s.Trev) {
                s.Trev[b] = (Real)0;
                s.Trev[k.cap + b] = (Real)0;
                s.Trev[2 * k.cap + b] = (Real)0;
            }
        }
    }
}

// ---- exclusive scan (in place) ----
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int v, int* total) {
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : 0;
        for (int off = 1; off < 32; off <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, off);
            if (lane >= off) t += y;
        }
        wsum[lane] = t;
    }
    __syncthreads();
    int prefix = (w > 0 ? wsum[w - 1] : 0) + x - v;
    *total = wsum[(blockDim.x >> 5) - 1];
    __syncthreads();
    return prefix;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(int32_t* data, int n, int32_t* sums) {
    const long long base = (long long)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems], loc = 0;
    for (int t = 0; t < kScanItems; t++) {
        long long idx = base + t;
        v[t] = idx < n ? data[idx] : 0;
        loc += v[t];
    }
    int total;
    int pre = block_exclusive_scan(loc, &total);
    for (int t = 0; t < kScanItems; t++) {
        long long idx = base + t;
        if (idx < n) data[idx] = pre;
        pre += v[t];
    }
    if (threadIdx.x == 0 && sums) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(int32_t* data, int n, const int32_t* sums) {
    const long long base = (long long)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    const int add = sums[blockIdx.x];
    for (int t = 0; t < kScanItems; t++) {
        long long idx = base + t;
        if (idx < n) data[idx] += add;
    }
}

// Critical time step of Eq. 65 (reading R30: micro-modulus over bond
// length): one warp per point sums 1 / |x_j - x_i| over the family in FP64
// (lane-strided, then a butterfly), dt_i = sqrt(2 rho / (V C sum)), and the
// minimum over points goes to *out by an atomic min on the ordered bits,
// exact and independent of the order.
template <typename Real>
__global__ void __launch_bounds__(kWarpPointsPerBlock * 32)
k_critical_dt(DevState<Real> s, StepConst k, double VC, long long* out) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kWarpPointsPerBlock + (threadIdx.x >> 5);
    if (i >= k.npoints) return;                     // the whole warp leaves together
    const int li = s.lat[i];
    const int r0 = s.row_ptr[i], r1 = s.row_ptr[i + 1];
    const double xi = Geometry<Real>::pos(s, k, i, 0, li);
    const double yi = Geometry<Real>::pos(s, k, i, 1, li);
    const double zi = Geometry<Real>::pos(s, k, i, 2, li);
    double acc = 0.0;
    for (int b = r0 + lane; b < r1; b += 32) {
        const int j = s.col[b];
        const int lj = s.lat[j];
        const double d0 = Geometry<Real>::pos(s, k, j, 0, lj) - xi;
        const double d1 = Geometry<Real>::image_y(s, k, j, lj, li) - yi;
        const double d2 = Geometry<Real>::pos(s, k, j, 2, lj) - zi;
        acc += 1.0 / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0 && acc > 0.0) atomicMin(out, ordered(sqrt(2.0 * k.rho / (VC * acc))));
}

__global__ void k_critical_dt_reset(long long* out) { *out = 0x7fffffffffffffffLL; }

}  // namespace

cudaError_t launch_exclusive_scan(int32_t* data, int n, int32_t* scanbuf, cudaStream_t st,
                                  long long* nlaunch) {
    if (n <= 0) return cudaSuccess;
    const int tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        k_scan_tiles<<<1, kScanThreads, 0, st>>>(data, n, nullptr);
        if (nlaunch) *nlaunch += 1;
        return cudaGetLastError();
    }
    if (tiles > kScanTile) return cudaErrorInvalidValue;
    k_scan_tiles<<<tiles, kScanThreads, 0, st>>>(data, n, scanbuf);
    k_scan_tiles<<<1, kScanThreads, 0, st>>>(scanbuf, tiles, nullptr);
    k_scan_add<<<tiles, kScanThreads, 0, st>>>(data, n, scanbuf);
    if (nlaunch) *nlaunch += 3;
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_family_build(const DevState<Real>& s, const StepConst& k, cudaStream_t st,
                                long long* nlaunch) {
    const int n = k.npoints;
    const int tpb = 256;
    const int pblocks = (n + tpb - 1) / tpb;
    const int wblocks = (n + kWarpPointsPerBlock - 1) / kWarpPointsPerBlock;
    const double delta = sqrt(k.delta2);
    k_bbox_reset<<<1, 32, 0, st>>>(s.bbox, &s.ctr->rebuilds);
    k_bbox<Real><<<min(pblocks, 4096), tpb, 0, st>>>(s, k);
    k_grid_setup<<<1, 1, 0, st>>>(s.bbox, s.grid, delta, k.ncols, s.ncell_cap, k.pbc_ny != 0);
    cudaMemsetAsync(s.cellcnt, 0, sizeof(int32_t) * (size_t)(s.ncell_cap + 1), st);
    cudaMemsetAsync(s.cellfill, 0, sizeof(int32_t) * (size_t)s.ncell_cap, st);
    k_cell_count<Real><<<pblocks, tpb, 0, st>>>(s, k);
    cudaMemcpyAsync(s.cellstart, s.cellcnt, sizeof(int32_t) * (size_t)(s.ncell_cap + 1),
                    cudaMemcpyDeviceToDevice, st);
    cudaError_t e = launch_exclusive_scan(s.cellstart, s.ncell_cap + 1, s.scanbuf, st, nlaunch);
    if (e != cudaSuccess) return e;
    k_cell_scatter<Real><<<pblocks, tpb, 0, st>>>(s, k);
    k_family_count<Real><<<wblocks, kWarpPointsPerBlock * 32, 0, st>>>(s, k);
    cudaMemcpyAsync(s.row_ptr, s.rowlen, sizeof(int32_t) * (size_t)(n + 1),
                    cudaMemcpyDeviceToDevice, st);
    e = launch_exclusive_scan(s.row_ptr, n + 1, s.scanbuf, st, nlaunch);
    if (e != cudaSuccess) return e;
    k_family_guard<<<1, 1, 0, st>>>(s.row_ptr, n, k.cap, s.ctr);
    k_family_zero_if_full<<<min(pblocks + 1, 1024), tpb, 0, st>>>(s.row_ptr, n, s.ctr);
    k_family_fill<Real><<<wblocks, kWarpPointsPerBlock * 32, 0, st>>>(s, k);
    k_family_rev<Real><<<wblocks, kWarpPointsPerBlock * 32, 0, st>>>(s, k);
    if (nlaunch) *nlaunch += 10;   // bbox_reset .. rev, scans counted above
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_critical_dt(const DevState<Real>& s, const StepConst& k, long long* out,
                               cudaStream_t st) {
    if (k.npoints <= 0) return cudaSuccess;
    const double delta = std::sqrt(k.delta2);
    const double C = 18.0 * k.K / (3.14159265358979323846 * delta * delta * delta * delta);
    const double VC = k.dx * k.dx * k.dx * C;
    const int wblocks = (k.npoints + kWarpPointsPerBlock - 1) / kWarpPointsPerBlock;
    k_critical_dt_reset<<<1, 1, 0, st>>>(out);
    k_critical_dt<Real><<<wblocks, kWarpPointsPerBlock * 32, 0, st>>>(s, k, VC, out);
    return cudaGetLastError();
}

template cudaError_t launch_critical_dt<double>(const DevState<double>&, const StepConst&,
                                                long long*, cudaStream_t);
template cudaError_t launch_critical_dt<float>(const DevState<float>&, const StepConst&,
                                               long long*, cudaStream_t);

template cudaError_t launch_family_build<double>(const DevState<double>&, const StepConst&,
                                                 cudaStream_t, long long*);
template cudaError_t launch_family_build<float>(const DevState<float>&, const StepConst&,
                                                cudaStream_t, long long*);

}  // namespace ppm
