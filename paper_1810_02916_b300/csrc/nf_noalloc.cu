// nf_noalloc.cu -- a near-field force pass that allocates no memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory pool it
// does not own, plugins whose host process forbids new device allocations
// after start-up, or real-time loops that must not risk the implicit
// synchronisation and fragmentation of an allocation.  They can call
// nf_forces_noalloc: it works on the caller's own device arrays (cell table,
// positions, output) and keeps its work list and counters in one file-scope
// device array of fixed size, g_scratch below.  Every GPU that loads the
// library holds that array (9,439,488 bytes) until the process exits.
//
// The host code reaches the array only through the device address returned
// by cudaGetSymbolAddress: the symbol's name in host code is a host-side
// stand-in, and a kernel given it would fault or silently touch the wrong
// memory.  The address is looked up once per device, with that device
// current, on the first call made on the device.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/nearfield.h"
#include "nf_internal.cuh"

namespace {

constexpr int kMaxCpd = 64;
constexpr int64_t kMaxCells = static_cast<int64_t>(kMaxCpd) * kMaxCpd * kMaxCpd;   // 262144
constexpr int64_t kMaxParticles = int64_t(1) << 21;                              // 2097152
constexpr int64_t kMaxItems = kMaxCells + kMaxParticles / 16 + 16;   // items per cell <= 1 + n_c / 16
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kCellInts = static_cast<size_t>(kMaxCells) + 2;
constexpr size_t kScanInts = static_cast<size_t>((kMaxCells + 1 + 4095) / 4096) + 2;

// byte offsets of the parts of the scratch array
constexpr size_t kOffDesc = 0;
constexpr size_t kOffItems = align256(kOffDesc + sizeof(nf::BoxDev));
constexpr size_t kOffCounts = align256(kOffItems + sizeof(nf::Item) * static_cast<size_t>(kMaxItems));
constexpr size_t kOffOffsets = align256(kOffCounts + sizeof(int) * kCellInts);
constexpr size_t kOffNbr = align256(kOffOffsets + sizeof(int) * kCellInts);
constexpr size_t kOffScan = align256(kOffNbr + sizeof(int) * kCellInts);
constexpr size_t kOffWords = align256(kOffScan + sizeof(int) * kScanInts);   // item counts, queues, error flag
constexpr size_t kOffPairs = align256(kOffWords + 8 * sizeof(int));          // the pass's pair count
constexpr size_t kScratchBytes = align256(kOffPairs + sizeof(unsigned long long));

static_assert(kScratchBytes == 9439488, "the documented scratch size is out of date");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

__global__ void write_desc(nf::BoxDev *dst, nf::BoxDev v) { *dst = v; }

// cell_start must run from 0 to n without decreasing; any violation sets *bad
__global__ void check_cell_start(const int *__restrict__ cs, int ncell, int n, int *__restrict__ bad)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > ncell) return;
    const int v = cs[c];
    if ((c == 0 && v != 0) || (c == ncell && v != n) || v < 0 || v > n || (c < ncell && cs[c + 1] < v)) atomicOr(bad, 1);
}

int say(char *err, int err_len, int code, const char *msg)
{
    if (err && err_len > 0) std::snprintf(err, static_cast<size_t>(err_len), "%s", msg);
    return code;
}

// device memory of device `dev` (the kernels run there and make no peer access),
// or managed memory
bool on_device(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" int nf_forces_noalloc(int cpd, double eps, double box, const int32_t *cell_start, const float *pos,
                                 int64_t n, float *acc, void *stream, char *err, int err_len)
{
    char msg[256];
    if (cpd < 5 || cpd > kMaxCpd) {
        std::snprintf(msg, sizeof(msg), "nf_forces_noalloc: cpd = %d outside [5, %d] (scratch holds %lld cells)", cpd,
                      kMaxCpd, static_cast<long long>(kMaxCells));
        return say(err, err_len, NF_EINVAL, msg);
    }
    if (n < 0 || n > kMaxParticles) {
        std::snprintf(msg, sizeof(msg), "nf_forces_noalloc: n = %lld outside [0, %lld]", static_cast<long long>(n),
                      static_cast<long long>(kMaxParticles));
        return say(err, err_len, NF_EINVAL, msg);
    }
    if (!(box > 0) || !(eps >= std::ldexp(box / cpd, -20)) || !(eps < box / cpd))
        return say(err, err_len, NF_EINVAL, "nf_forces_noalloc: need box > 0 and 2^-20 box / cpd <= eps < box / cpd");
    if (!cell_start || (n > 0 && (!pos || !acc)))
        return say(err, err_len, NF_EINVAL, "nf_forces_noalloc: NULL array");
    if ((reinterpret_cast<uintptr_t>(pos) | reinterpret_cast<uintptr_t>(acc)) & 15u)
        return say(err, err_len, NF_EINVAL, "nf_forces_noalloc: pos and acc must be 16-byte aligned");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return say(err, err_len, NF_ECUDA, "nf_forces_noalloc: no device");
    if (!on_device(cell_start, dev) || (n > 0 && (!on_device(pos, dev) || !on_device(acc, dev))))
        return say(err, err_len, NF_EINVAL,
                   "nf_forces_noalloc: cell_start, pos and acc must be device memory of the current device");
    char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_addr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_scratch);
            if (e != cudaSuccess || !ptr) {
                std::snprintf(msg, sizeof(msg), "nf_forces_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                cudaGetLastError();
                return say(err, err_len, NF_ECUDA, msg);
            }
            g_scratch_addr[dev] = ptr;
        }
        base = static_cast<char *>(g_scratch_addr[dev]);
    }
    nf::BoxDev *desc = reinterpret_cast<nf::BoxDev *>(base + kOffDesc);
    nf::Item *items = reinterpret_cast<nf::Item *>(base + kOffItems);
    int *counts = reinterpret_cast<int *>(base + kOffCounts);
    int *offsets = reinterpret_cast<int *>(base + kOffOffsets);
    int *nbr = reinterpret_cast<int *>(base + kOffNbr);
    void *scan_tmp = base + kOffScan;
    int *words = reinterpret_cast<int *>(base + kOffWords);
    int *n_items = words, *queue = words + 2, *bad = words + 4;   // n_items[2], queue[2]
    unsigned long long *pairs = reinterpret_cast<unsigned long long *>(base + kOffPairs);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int ncell = cpd * cpd * cpd;

#define NA_CK(call)                                                                                  \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) {                                                                     \
            std::snprintf(msg, sizeof(msg), "nf_forces_noalloc: %s: %s", #call, cudaGetErrorString(e_)); \
            return say(err, err_len, NF_ECUDA, msg);                                                 \
        }                                                                                            \
    } while (0)

    // the cell table bounds every index the planner and the kernel form: check it first
    int hbad = 0;
    NA_CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
    check_cell_start<<<(ncell + 256) / 256, 256, 0, st>>>(cell_start, ncell, static_cast<int>(n), bad);
    NA_CK(cudaGetLastError());
    NA_CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if (hbad) return say(err, err_len, NF_EINVAL, "nf_forces_noalloc: cell_start is not a scan from 0 to n");
    if (n == 0) return NF_OK;

    // work list (items ordered largest cells first), then the descriptor, then the pair kernel
    NA_CK(nf::neighbour_pairs(cell_start, cpd, 0, pairs, counts, offsets, nbr, nullptr, st));
    NA_CK(nf::zero_device_int(n_items, st));
    for (int cls = 0; cls < nf::kClasses; ++cls)
        NA_CK(nf::plan_items_class(cell_start, nbr, ncell, 0, cls, items, n_items, counts, offsets, scan_tmp,
                                   nf::kDefaultTiles, st));
    NA_CK(nf::plan_lane_items(cell_start, nbr, cpd, 0, items, n_items, counts, offsets, scan_tmp, st));
    const double inv_w = static_cast<double>(cpd) / box;
    const double ec = eps * inv_w;
    nf::BoxDev d{};
    d.pos = reinterpret_cast<const float4 *>(pos);
    d.cell_start = cell_start;
    d.acc_out = reinterpret_cast<float4 *>(acc);
    d.acc64 = nullptr;
    d.cot = nullptr;
    d.cpd = cpd;
    d.n = static_cast<int>(n);
    d.a0 = static_cast<float>(10.0 / (ec * ec * ec));
    d.a1 = static_cast<float>(-15.0 / (ec * ec * ec * ec));
    d.a2 = static_cast<float>(6.0 / (ec * ec * ec * ec * ec));
    d.eps2 = static_cast<float>(ec * ec);
    d.acc_scale = inv_w * inv_w;
    d.grad_scale = inv_w * inv_w * inv_w;
    write_desc<<<1, 1, 0, st>>>(desc, d);
    NA_CK(cudaGetLastError());
    NA_CK(cudaMemsetAsync(queue, 0, sizeof(int), st));
    int sms = 0;
    NA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    NA_CK(nf::launch_pair(desc, items, n_items, queue, 1, 0, 0, nf::PairShape{8, 128, 0}, sms, st));
#undef NA_CK
    return NF_OK;
}
