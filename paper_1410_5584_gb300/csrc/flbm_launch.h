// flbm_launch.h -- per-(lattice, storage) launchers; defined in
// flbm_kernels.cuh and explicitly instantiated in the inst_*.cu files.
#pragma once
#include "flbm_internal.h"
#include "flbm_lattice.cuh"

namespace flbm {

template <class L, class S> struct Launch {
    static cudaError_t density(int parity, const StepParams &p, const void *pop, float *rho, cudaStream_t st);
    // parity 0 / 1: in place in pop; kPush (2): read pop, write pop_out
    static cudaError_t collide(int parity, const StepParams &p, void *pop, void *pop_out, const float *rho,
                               unsigned *status, cudaStream_t st);
    static cudaError_t step_fused(int parity, const StepParams &p, void *pop, float *rho, unsigned *status,
                                  unsigned *counters, double wait_ms, int stall, int lag, cudaStream_t st);
    // pipelined two-array step: lag and ring slots for this box (ring_slots = 0:
    // too few slices), and the ring's size in floats
    static cudaError_t pipe_geometry(const StepParams &p, bool mom, int lag_opt, int *lag, int *ring_slots,
                                     size_t *ring_floats, size_t *counters);
    static cudaError_t step_pipe(const StepParams &p, const void *pop, void *pop_out, float *ring, unsigned *counters,
                                 int ring_slots, int lag, bool mom, unsigned *status, double wait_ms, int stall,
                                 cudaStream_t st);
    // parity 0 / 1: in place in pop; kPush: read pop, write pop_out
    static cudaError_t batch_step(int parity, const RepInfo *reps, const int2 *tiles, int ntiles, void *pop,
                                  void *pop_out, float *rho, unsigned *status, const unsigned *step_base, unsigned k,
                                  bool full, cudaStream_t st);
    // tiled two-array step (2D lattices; cudaErrorNotSupported otherwise)
    static cudaError_t step_tiled(const StepParams &p, const void *pop, void *pop_out, unsigned *status,
                                  cudaStream_t st);
    static cudaError_t batch_step_tiled(const RepInfo *reps, const int4 *tiles, int ntiles, const void *pop,
                                        void *pop_out, unsigned *status, const unsigned *step_base, unsigned k,
                                        bool full, cudaStream_t st);
    static int tile_rows();
    static cudaError_t init_rest(const StepParams &p, const float *rho_in, void *pop, cudaStream_t st);
    static cudaError_t gather(int parity, const StepParams &p, const void *pop, const int64_t *sites, int64_t n,
                              double *out, cudaStream_t st);
    static cudaError_t sfk_fields(int parity, const StepParams &p, const void *pop, float2 *z, double *partials,
                                  int *nblocks, cudaStream_t st);
    static cudaError_t observables(int parity, const StepParams &p, const void *pop, const float *rho, double *ra,
                                   double *rb, double *u, double *partials, int *nblocks, cudaStream_t st);
};

extern template struct Launch<D2Q9, StoreF32>;
extern template struct Launch<D2Q9, StoreF16>;
extern template struct Launch<D2Q9, StoreBF16>;
extern template struct Launch<D3Q19, StoreF32>;
extern template struct Launch<D3Q19, StoreF16>;
extern template struct Launch<D3Q19, StoreBF16>;

} // namespace flbm
