// flbm_dispatch.cu -- run-time dispatch from (lattice, storage) to the kernel
// instances of flbm_kernels.cuh.
#include "flbm_launch.h"

namespace flbm {

namespace {

template <template <class, class> class F, class... A>
cudaError_t dispatch(int lat, int storage, A &&...args)
{
    if (lat == FLBM_D2Q9) {
        if (storage == FLBM_STORE_F32) return F<D2Q9, StoreF32>::run(args...);
        if (storage == FLBM_STORE_F16) return F<D2Q9, StoreF16>::run(args...);
        return F<D2Q9, StoreBF16>::run(args...);
    }
    if (storage == FLBM_STORE_F32) return F<D3Q19, StoreF32>::run(args...);
    if (storage == FLBM_STORE_F16) return F<D3Q19, StoreF16>::run(args...);
    return F<D3Q19, StoreBF16>::run(args...);
}

template <class L, class S> struct DensityF {
    template <class... A> static cudaError_t run(A... a) { return Launch<L, S>::density(a...); }
};
template <class L, class S> struct CollideF {
    template <class... A> static cudaError_t run(A... a) { return Launch<L, S>::collide(a...); }
};
template <class L, class S> struct FusedF {
    template <class... A> static cudaError_t run(A... a) { return Launch<L, S>::step_fused(a...); }
};
template <class L, class S> struct PipeGeomF {
    template <class... A> static cudaError_t run(A... a) { return Launch<L, S>::pipe_geometry(a...); }
};
template <class L, class S> struct PipeF {
    template <class... A> static cudaError_t run(A... a) { return Launch<L, S>::step_pipe(a...); }
};
template <class L, class S> struct BatchF {
    template <class... A> static cudaError_t run(A... a) { return Launch<L, S>::batch_step(a...); }
};
template <class L, class S> struct TiledF {
    template <class... A> static cudaError_t run(A... a) { return Launch<L, S>::step_tiled(a...); }
};
template <class L, class S> struct BatchTiledF {
    template <class... A> static cudaError_t run(A... a) { return Launch<L, S>::batch_step_tiled(a...); }
};
template <class L, class S> struct InitF {
    template <class... A> static cudaError_t run(A... a) { return Launch<L, S>::init_rest(a...); }
};
template <class L, class S> struct GatherF {
    template <class... A> static cudaError_t run(A... a) { return Launch<L, S>::gather(a...); }
};
template <class L, class S> struct SfkF {
    template <class... A> static cudaError_t run(A... a) { return Launch<L, S>::sfk_fields(a...); }
};
template <class L, class S> struct ObsF {
    template <class... A> static cudaError_t run(A... a) { return Launch<L, S>::observables(a...); }
};

} // namespace

cudaError_t launch_density(int lat, int storage, int parity, const StepParams &p, const void *pop, float *rho,
                           cudaStream_t stream)
{
    return dispatch<DensityF>(lat, storage, parity, p, pop, rho, stream);
}

cudaError_t launch_collide(int lat, int storage, int parity, const StepParams &p, void *pop, void *pop_out,
                           const float *rho, unsigned *status, cudaStream_t stream)
{
    return dispatch<CollideF>(lat, storage, parity, p, pop, pop_out, rho, status, stream);
}

cudaError_t launch_step_fused(int lat, int storage, int parity, const StepParams &p, void *pop, float *rho,
                              unsigned *status, unsigned *counters, double wait_ms, int stall, int lag,
                              cudaStream_t stream)
{
    return dispatch<FusedF>(lat, storage, parity, p, pop, rho, status, counters, wait_ms, stall, lag, stream);
}

cudaError_t pipe_geometry(int lat, int storage, const StepParams &p, bool mom, int lag_opt, int *lag, int *ring_slots,
                          size_t *ring_floats, size_t *counters)
{
    return dispatch<PipeGeomF>(lat, storage, p, mom, lag_opt, lag, ring_slots, ring_floats, counters);
}

cudaError_t launch_step_pipe(int lat, int storage, const StepParams &p, const void *pop, void *pop_out, float *ring,
                             unsigned *counters, int ring_slots, int lag, bool mom, unsigned *status, double wait_ms,
                             int stall, cudaStream_t stream)
{
    return dispatch<PipeF>(lat, storage, p, pop, pop_out, ring, counters, ring_slots, lag, mom, status, wait_ms, stall,
                           stream);
}

cudaError_t launch_batch_step(int lat, int storage, int parity, const RepInfo *reps, const int2 *tiles, int ntiles,
                              void *pop, void *pop_out, float *rho, unsigned *status, const unsigned *step_base,
                              unsigned k, bool full, cudaStream_t stream)
{
    return dispatch<BatchF>(lat, storage, parity, reps, tiles, ntiles, pop, pop_out, rho, status, step_base, k, full,
                            stream);
}

cudaError_t launch_step_tiled(int lat, int storage, const StepParams &p, const void *pop, void *pop_out,
                              unsigned *status, cudaStream_t stream)
{
    return dispatch<TiledF>(lat, storage, p, pop, pop_out, status, stream);
}

cudaError_t launch_batch_step_tiled(int lat, int storage, const RepInfo *reps, const int4 *tiles, int ntiles,
                                    const void *pop, void *pop_out, unsigned *status, const unsigned *step_base,
                                    unsigned k, bool full, cudaStream_t stream)
{
    return dispatch<BatchTiledF>(lat, storage, reps, tiles, ntiles, pop, pop_out, status, step_base, k, full, stream);
}

int tiled_step_rows(int lat) { return lat == FLBM_D2Q9 ? Launch<D2Q9, StoreF32>::tile_rows() : 0; }

cudaError_t launch_init_rest(int lat, int storage, const StepParams &p, const float *rho_in, void *pop,
                             cudaStream_t stream)
{
    return dispatch<InitF>(lat, storage, p, rho_in, pop, stream);
}

cudaError_t launch_gather_sites(int lat, int storage, int parity, const StepParams &p, const void *pop,
                                const int64_t *sites, int64_t nsites, double *out, cudaStream_t stream)
{
    return dispatch<GatherF>(lat, storage, parity, p, pop, sites, nsites, out, stream);
}

cudaError_t launch_sfk_fields(int lat, int storage, int parity, const StepParams &p, const void *pop, float2 *z,
                              double *partials, int *nblocks, cudaStream_t stream)
{
    return dispatch<SfkF>(lat, storage, parity, p, pop, z, partials, nblocks, stream);
}

cudaError_t launch_observables(int lat, int storage, int parity, const StepParams &p, const void *pop,
                               const float *rho, double *rho_a, double *rho_b, double *u, double *partials,
                               int *nblocks, cudaStream_t stream)
{
    return dispatch<ObsF>(lat, storage, parity, p, pop, rho, rho_a, rho_b, u, partials, nblocks, stream);
}

} // namespace flbm
