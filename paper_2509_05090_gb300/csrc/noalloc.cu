// ctm_gemm_noalloc: the contraction engine with its scratch memory in a fixed,
// library-owned device array instead of a caller-supplied workspace.
//
// Some callers cannot allocate device memory: a plugin hosted by a framework
// that owns every device allocation (its allocator neither permits nor tracks
// a direct cudaMalloc), a latency-critical loop that cannot afford an
// allocation or its possible failure in the middle of a run, or a service
// whose device-memory budget is fixed at start-up.  This entry point lets them
// run the engine with only their own inputs and outputs.
//
// The scratch is the file-scope array below, CTM_NOALLOC_SCRATCH_BYTES long.
// Every GPU that loads this library holds it until the process exits.  Host
// code must not use the array's name as a device address: the first call on a
// device looks the address up with cudaGetSymbolAddress (with that device
// current) and caches it per device; that first call should therefore come
// before any stream capture.  Every call shares the array and leaves its
// contents behind; the engine clears what must start at zero (its error flag
// and the split-K integer accumulator) at the start of each call, so calls
// that overlap on the GPU race and must be serialised by the caller.
#include <mutex>

#include "ctm_internal.h"

static __device__ __align__(256) unsigned char g_ctm_noalloc_scratch[CTM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

int noalloc_scratch(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return CTM_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return CTM_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_ctm_noalloc_scratch) != cudaSuccess || !p) return CTM_ECUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return CTM_OK;
}

}  // namespace

extern "C" int ctm_gemm_noalloc(int M, int N, int K, const double *A_dev, const double *B_dev, double *C_dev,
                                int precision, int n_split, void *stream)
{
    if (M <= 0 || N <= 0 || K <= 0 || !A_dev || !B_dev || !C_dev) return CTM_EINVAL;
    const size_t need = ctm_gemm_workspace_bytes(M, N, K, precision, n_split);
    if (need == 0) return CTM_EINVAL;
    if (need > (size_t)CTM_NOALLOC_SCRATCH_BYTES) return CTM_ENOMEM;   // beyond the fixed scratch
    void *scratch = nullptr;
    const int rc = noalloc_scratch(&scratch);
    if (rc != CTM_OK) return rc;
    return ctm_gemm(M, N, K, A_dev, B_dev, C_dev, precision, n_split, scratch, (size_t)CTM_NOALLOC_SCRATCH_BYTES,
                    stream);
}
