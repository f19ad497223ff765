// Family search without any device allocation: the same cell-list kernels
// as ppm_build_families, with their scratch in a fixed-size array that is
// part of the library image instead of the caller's workspace.
//
// For callers that cannot allocate device memory: real-time loops that must
// not enter the allocator (cudaMalloc can block and synchronise the
// device), and hosts whose device memory is owned by another allocator or
// memory pool that the library must not touch.
#include <cuda_runtime.h>

#include <mutex>

#include "ppm_internal.cuh"

using namespace ppm;

namespace {

constexpr int kNoAllocMaxPoints = 262144;
constexpr int kNoAllocCellCap = 2 * kNoAllocMaxPoints;
constexpr size_t kAlign = 256;

constexpr size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// scratch layout inside the static array
constexpr size_t kOffCtr = 0;
constexpr size_t kOffGrid = kOffCtr + up(sizeof(DevCounters));
constexpr size_t kOffBbox = kOffGrid + up(sizeof(CellGrid));
constexpr size_t kOffCellKey = kOffBbox + up(6 * sizeof(long long));
constexpr size_t kOffCellCnt = kOffCellKey + up(sizeof(int32_t) * kNoAllocMaxPoints);
constexpr size_t kOffCellStart = kOffCellCnt + up(sizeof(int32_t) * (kNoAllocCellCap + 1));
constexpr size_t kOffCellFill = kOffCellStart + up(sizeof(int32_t) * (kNoAllocCellCap + 1));
constexpr size_t kOffSorted = kOffCellFill + up(sizeof(int32_t) * kNoAllocCellCap);
constexpr size_t kOffRowLen = kOffSorted + up(sizeof(int32_t) * kNoAllocMaxPoints);
constexpr size_t kOffScan = kOffRowLen + up(sizeof(int32_t) * (kNoAllocMaxPoints + 1));
constexpr size_t kScratchBytes = kOffScan + up(sizeof(int32_t) * 8192);

// About 9.5 MB; every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_family_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
char* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;   // guards g_scratch_addr against concurrent host threads

// Device address of the scratch array on device dev, looked up on the first
// call for that device (with dev current) and kept for the life of the
// process.  In host code the array's name is only a host-side stand-in,
// so the kernels get this address, never the name.
int scratch_address(int dev, char** out) {
    if (dev < 0 || dev >= kMaxDevices) return PPM_ECUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_family_scratch) != cudaSuccess || !ptr) return PPM_ECUDA;
        g_scratch_addr[dev] = static_cast<char*>(ptr);
    }
    *out = g_scratch_addr[dev];
    return PPM_OK;
}

}  // namespace

extern "C" int ppm_family_noalloc(int64_t n, const double* d_x, double delta, int max_family,
                                  int32_t* d_row_ptr, int32_t* d_col, int32_t* d_rev,
                                  int64_t cap, void* cuda_stream, int64_t* nbonds) {
    if (n < 1 || n > kNoAllocMaxPoints) return PPM_EINVAL;
    if (!d_x || !d_row_ptr || !d_col || !d_rev || !(delta > 0.0)) return PPM_EINVAL;
    if (max_family < 1 || max_family > kMaxRow || cap < 0 || cap > 0x7fffffffLL) return PPM_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the stream must belong to the current device, whose copy of the
    // array the kernels will use
    int dev = -1, sdev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaStreamGetDevice(st, &sdev) != cudaSuccess)
        return PPM_ECUDA;
    if (sdev != dev) return PPM_EINVAL;
    char* base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc) return rc;

    DevState<double> s = {};
    s.xabs = d_x;
    s.row_ptr = d_row_ptr;
    s.col = d_col;
    s.rev = d_rev;
    s.ctr = reinterpret_cast<DevCounters*>(base + kOffCtr);
    s.grid = reinterpret_cast<CellGrid*>(base + kOffGrid);
    s.bbox = reinterpret_cast<long long*>(base + kOffBbox);
    s.cellkey = reinterpret_cast<int32_t*>(base + kOffCellKey);
    s.cellcnt = reinterpret_cast<int32_t*>(base + kOffCellCnt);
    s.cellstart = reinterpret_cast<int32_t*>(base + kOffCellStart);
    s.cellfill = reinterpret_cast<int32_t*>(base + kOffCellFill);
    s.sorted = reinterpret_cast<int32_t*>(base + kOffSorted);
    s.rowlen = reinterpret_cast<int32_t*>(base + kOffRowLen);
    s.scanbuf = reinterpret_cast<int32_t*>(base + kOffScan);
    s.ncell_cap = kNoAllocCellCap;

    StepConst k = {};
    k.delta2 = delta * delta;
    k.npoints = (int)n;
    k.ncols = 1;
    k.max_family = max_family;
    k.cap = cap;

    // the array keeps the previous call's contents: clear what the kernels
    // expect at zero (the cell histograms are cleared inside the build)
    if (cudaMemsetAsync(s.ctr, 0, sizeof(DevCounters), st) != cudaSuccess) return PPM_ECUDA;
    if (launch_family_build<double>(s, k, st, nullptr) != cudaSuccess) return PPM_ECUDA;

    DevCounters h;
    int32_t total = 0;
    if (cudaMemcpyAsync(&h, s.ctr, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&total, d_row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PPM_ECUDA;
    if (nbonds) *nbonds = h.family_ok ? total : 0;
    if (!h.family_ok || (h.status & PPM_STATUS_ROW_FULL)) return PPM_ENOSPACE;
    return PPM_OK;
}
