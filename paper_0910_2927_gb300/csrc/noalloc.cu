// sgn_inner_products_noalloc: the inner products of sgn_inner_products for
// callers that cannot allocate device memory -- applications under a framework
// that owns every device allocation (a fixed arena, no outside cudaMalloc), and
// latency-critical loops that must not pay for cudaMalloc/cudaFree, which can
// synchronise the device.  The per-block partial sums live in one file-scope
// device array instead of memory from an allocator.
#include "blas.cuh"

#include <mutex>

namespace sgn {
namespace {

// Scratch shared by every call on a device (held by each device that loads
// the library until the process exits): 8 MiB of partial sums plus flags.
constexpr size_t kStaticScratchBytes = size_t(8) << 20;
constexpr size_t kFlagBytes = 4096;  // per-column zero flags read by the reduction (<= 512 columns)
static __device__ __align__(256) unsigned char g_noalloc_scratch[kStaticScratchBytes + kFlagBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array for the current device.  The host-side
// name of a __device__ array is only a stand-in, never a device address, so the
// address is asked for once per device, with that device current, on the first
// call there, and kept for the life of the process (a cudaDeviceReset reloads the
// module and leaves the kept address stale; the header says so).
int scratch_address(void** out) {
    int dev = 0;
    SGN_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("sgn_inner_products_noalloc: device index out of range");
        return SGN_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("sgn_inner_products_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return SGN_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SGN_OK;
}

}  // namespace
}  // namespace sgn

using namespace sgn;

SGN_API int sgn_inner_products_noalloc(const double* V, int J, const double* w, long long n, int nrhs, double* out,
                                       void* stream) {
    if (!V || !w || !out || J < 1 || J > 64 || nrhs < 1 || n < 2 || (n % 2) != 0) {
        set_error("sgn_inner_products_noalloc: need 1 <= J <= 64, nrhs >= 1, even n >= 2, non-NULL pointers");
        return SGN_ERR_ARG;
    }
    const int nblk = reduce_blocks<double2>((int64_t)n);
    const size_t need = sizeof(double2) * (size_t)nrhs * J * nblk;
    if (need > kStaticScratchBytes || (size_t)nrhs * 2 * sizeof(int) > kFlagBytes) {
        set_error("sgn_inner_products_noalloc: nrhs * J * ceil(n / 1024) * 16 bytes = " + std::to_string(need) +
                  " exceeds the fixed scratch of " + std::to_string(kStaticScratchBytes) +
                  " bytes (or nrhs > 512); use sgn_inner_products");
        return SGN_ERR_ARG;
    }
    void* base = nullptr;
    SGN_CHECK(scratch_address(&base));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* p = reinterpret_cast<char*>(base);
    DevState S{};
    S.red = reinterpret_cast<double2*>(out);  // results go straight to the caller's buffer
    S.rstride = J;
    S.skip = reinterpret_cast<int*>(p + kStaticScratchBytes);
    S.done = S.skip + nrhs;
    // the array keeps the previous call's contents: the flags must start at zero
    SGN_CUDA(cudaMemsetAsync(S.skip, 0, sizeof(int) * 2 * (size_t)nrhs, st));
    const Reduce rd{reinterpret_cast<double2*>(p), nblk, J};
    SGN_CUDA(mdot<double2>(Basis<double2>{reinterpret_cast<const double2*>(V), (int64_t)n, 0}, J,
                           reinterpret_cast<const double2*>(w), (int64_t)n, (int64_t)n, nrhs, rd, 0, nullptr, st));
    SGN_CUDA(reduce(rd, J, nrhs, RM_STORE, 0, S, nullptr, st));
    return SGN_OK;
}
