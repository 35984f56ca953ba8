// Allocation-free K_r table build.
//
// ksc_make_split_real allocates the table's node scratch with cudaMalloc.
// Some callers cannot allocate device memory at the point where they need a
// table: code running under a caching allocator or a fixed memory budget that
// owns every device byte, real-time loops where cudaMalloc's implicit device
// synchronisation is unacceptable, and work issued on a stream that is being
// captured into a CUDA graph.  This entry point builds the same table with
// its scratch in a file-scope __device__ array instead.
//
// Scratch: kNoAllocNodes node values and as many node slopes (FP64), i.e.
// tables of up to kNoAllocMaxIntervals = 8192 intervals (131 kB held on every
// device that loads the library, until the process exits).  Each call
// overwrites every scratch value it reads, so nothing needs clearing between
// calls; but all calls share the one array, so calls that overlap on the GPU
// (different streams, no ordering between them) race and may corrupt each
// other's tables.  A call made outside stream capture looks up the array's
// device address (cudaGetSymbolAddress, which must not run during capture) and
// remembers it for the device, so the address follows a reset of the device's
// context; a call made while its stream is being captured uses the address
// remembered by the last call outside capture on that device, so make one call
// before any capture (and again after a device reset).
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "ksc_internal.h"

namespace {

constexpr int kNoAllocMaxIntervals = 8192;
constexpr int kNoAllocNodes = kNoAllocMaxIntervals + 1;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_table_scratch[2 * kNoAllocNodes];

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

int fail(int code, const std::string &msg) {
    ksc::set_last_error(msg);
    return code;
}

} // namespace

extern "C" {

int ksc_build_table_noalloc(const double *d_c, int lmax, double theta_cut, int n_intervals,
                            float *d_table, void *stream) {
    if (!d_c || !d_table) return fail(KSC_ERR_ARG, "null pointer");
    if ((uintptr_t)d_table & 15u) return fail(KSC_ERR_ARG, "table must be 16-byte aligned");
    if (lmax < 1 || lmax > 16384) return fail(KSC_ERR_ARG, "lmax outside 1..16384");
    if (!(theta_cut > 0.0) || theta_cut > 3.14159265358979323846)
        return fail(KSC_ERR_ARG, "theta_cut outside (0, pi]");
    if (n_intervals < 1 || n_intervals > kNoAllocMaxIntervals)
        return fail(KSC_ERR_ARG,
                    "n_intervals outside 1..8192 (the size of the built-in scratch array)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(KSC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(KSC_ERR_UNSUPPORTED, "device index above 63");
    double *scratch = nullptr;
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        const bool capturing =
            cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess ||
            cs != cudaStreamCaptureStatusNone;
        if (capturing) (void)cudaGetLastError();  // (an illegal query during capture)
        std::lock_guard<std::mutex> lk(g_mu);
        if (!capturing) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_table_scratch);
            if (e != cudaSuccess)
                return fail(KSC_ERR_CUDA,
                            std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_ptr[dev] = static_cast<double *>(p);
        } else if (!g_scratch_ptr[dev]) {
            return fail(KSC_ERR_ARG, "first call on this device made during stream capture");
        }
        scratch = g_scratch_ptr[dev];
    }
    const double chord_cut = 2.0 * std::sin(0.5 * theta_cut);
    ksc::TableBuild tb{d_c, lmax, n_intervals, chord_cut / n_intervals,
                       reinterpret_cast<float4 *>(d_table), scratch};
    e = ksc::launch_table_build(tb, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return fail(KSC_ERR_CUDA, std::string("table build launch: ") + cudaGetErrorString(e));
    return KSC_OK;
}

} // extern "C"
