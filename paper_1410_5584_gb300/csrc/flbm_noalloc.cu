// flbm_noalloc.cu -- stepping on caller-owned populations with no device
// allocation at all.
//
// Some callers cannot call cudaMalloc: code running inside an arena or pool
// that owns all device memory, or a real-time loop where an allocation could
// stall or fail.  flbm_step_noalloc serves them: the only device memory it
// needs besides the caller's populations -- the density field and the status
// word -- lives in one file-scope __device__ array of fixed size, which every
// GPU that loads this library holds until the process exits.
#include <cstdint>

#include "flbm_internal.h"

namespace {

constexpr int64_t kNoAllocMaxSites = int64_t(1) << 21; // 2,097,152 sites
constexpr size_t kStatusBytes = 256;                    // status word, padded to keep the field aligned
constexpr size_t kScratchBytes = kStatusBytes + (size_t)kNoAllocMaxSites * 2 * sizeof(float);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// The array's name in host code is only a host-side stand-in; its device
// address is looked up on every call, with the calling device current, so a
// device reset between calls (which gives the array a new address) is harmless.
cudaError_t scratch_address(void **addr) { return cudaGetSymbolAddress(addr, g_noalloc_scratch); }

flbm_status cuda_error(cudaError_t e) { return e == cudaSuccess ? FLBM_OK : FLBM_ECUDA; }

} // namespace

extern "C" flbm_status flbm_step_noalloc(const flbm_ctx *ctx, void *pop, int parity, int64_t step, int64_t n,
                                         void *stream, unsigned *status_out)
{
    using namespace flbm;
    CtxView v;
    if (!ctx_view(ctx, &v) || !pop || (parity != 0 && parity != 1) || step < 0 || n < 0) return FLBM_EINVAL;
    if (v.batch) return FLBM_EINVAL;                 // one box per call: a batch steps through flbm_step
    if (reinterpret_cast<uintptr_t>(pop) & 255u) return FLBM_EINVAL; // rejected here, not left to fault on the device
    if (v.N > kNoAllocMaxSites) return FLBM_EINVAL; // the box exceeds the static scratch (2^21 sites)
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return cuda_error(e);
    unsigned *status = static_cast<unsigned *>(base);
    float *rho = reinterpret_cast<float *>(static_cast<unsigned char *>(base) + kStatusBytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the array keeps the previous call's contents: the status must start at zero
    if ((e = cudaMemsetAsync(status, 0, sizeof(unsigned), st)) != cudaSuccess) return cuda_error(e);
    StepParams p = v.params;
    for (int64_t t = 0; t < n; t++) {
        p.step = (uint32_t)(step + t);
        if ((e = launch_density(v.lat, v.storage, parity, p, pop, rho, st)) != cudaSuccess) return cuda_error(e);
        if ((e = launch_collide(v.lat, v.storage, parity, p, pop, pop, rho, status, st)) != cudaSuccess) return cuda_error(e);
        parity ^= 1;
    }
    unsigned h = 0;
    if ((e = cudaMemcpyAsync(&h, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_error(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_error(e);
    if (status_out) *status_out = h;
    return (h & kStatusNonFinite) ? FLBM_ENONFINITE : FLBM_OK;
}
