// ssa_noalloc.cu -- ssa_ensemble_mean_static: the ensemble mean with its scratch in a fixed
// device array instead of a caller-provided workspace.
//
// Who needs it: code that must not allocate device memory at call time -- a caller recording the
// call into a CUDA graph (cudaMalloc is not allowed during stream capture), a real-time loop that
// forbids allocator calls and their synchronisation, or a host library that has no handle to the
// application's allocator and so cannot hand over a workspace.
//
// The scratch is the file-scope array below. Every GPU that loads the library holds it until the
// process exits. Host code cannot use the array's name as a device address (in host code it names
// a host-side stand-in), so the address is obtained once per device with cudaGetSymbolAddress
// while that device is current, and passed to the kernels. The address is cached per device index for
// the life of the process; after cudaDeviceReset the device code may be reloaded elsewhere, so the entry
// point must not be used across a reset of the device.
#include <mutex>

#include "ssa_internal.cuh"

namespace ssa {
cudaError_t launch_ensemble_mean(const void *obs, bool is_int, int64_t n_traj, int64_t row_len, float *partial,
                                 int64_t chunk, float *out, cudaStream_t st);
ssa_status set_error(ssa_status code, const char *text);
}  // namespace ssa

namespace {

// Maximum scratch: ceil(n_traj / 256) * row_len floats (4 MiB).
constexpr int64_t kStaticScratchFloats = int64_t(1) << 20;
constexpr int64_t kChunk = 256;
constexpr int kMaxDevices = 64;

__device__ __align__(256) float g_static_mean_scratch[kStaticScratchFloats];

std::mutex g_setup_mutex;
float *g_scratch_addr[kMaxDevices] = {};

}  // namespace

// Resolve the device address of the scratch array for the current device (once per device). The lookup
// may load the library's device code, which a stream that is being captured into a graph does not allow:
// a first call on a capturing stream is refused with a message instead of failing inside the capture.
static ssa_status static_scratch(float **out, cudaStream_t stream)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ssa::set_error(SSA_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return ssa::set_error(SSA_ERR_UNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(stream, &cap) == cudaSuccess && cap != cudaStreamCaptureStatusNone)
            return ssa::set_error(SSA_ERR_UNSUPPORTED,
                                  "ssa_ensemble_mean_static: the first call on a device looks up its scratch address "
                                  "and cannot run during stream capture; make one call before capturing");
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_mean_scratch);
        if (e != cudaSuccess || !p)
            return ssa::set_error(SSA_ERR_CUDA, e != cudaSuccess ? cudaGetErrorString(e) : "no symbol address");
        g_scratch_addr[dev] = static_cast<float *>(p);
    }
    *out = g_scratch_addr[dev];
    return SSA_OK;
}

extern "C" ssa_status ssa_ensemble_mean_static(const void *obs, int32_t obs_is_int, int64_t n_traj, int64_t row_len,
                                               float *mean_out, void *stream)
{
    if (n_traj < 0 || row_len < 0) return ssa::set_error(SSA_ERR_INVALID_ARG, "negative size");
    if ((n_traj > 0 && row_len > 0 && !obs) || (row_len > 0 && !mean_out))
        return ssa::set_error(SSA_ERR_INVALID_ARG, "NULL pointer");
    const int64_t n_chunks = (n_traj + kChunk - 1) / kChunk;
    if (row_len > 0 && n_chunks > kStaticScratchFloats / row_len)
        return ssa::set_error(SSA_ERR_UNSUPPORTED,
                              "ssa_ensemble_mean_static: ceil(n_traj/256) * row_len exceeds the 1,048,576-float "
                              "static scratch; use ssa_ensemble_mean with a workspace");
    float *scratch = nullptr;
    const ssa_status s = static_scratch(&scratch, static_cast<cudaStream_t>(stream));
    if (s != SSA_OK) return s;
    // every scratch entry the reduction reads is written earlier in the same call, so nothing has to
    // be cleared between calls
    cudaError_t e = ssa::launch_ensemble_mean(obs, obs_is_int != 0, n_traj, row_len, scratch, kChunk, mean_out,
                                              static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SSA_OK : ssa::set_error(SSA_ERR_CUDA, cudaGetErrorString(e));
}
