// ttc_launch.h -- host entry points into the kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include "ttc_internal.cuh"

namespace ttc {

enum Phase {
  PH_INIT1 = 0, PH_INIT2 = 1, PH_INIT3 = 2, PH_SCREEN = 3, PH_DECIDE = 4, PH_UPDATE = 5,
  PH_REFINE = 6, PH_DECIDE2 = 7, PH_TABLES = 8, PH_ROOK_SCAN = 9, PH_ROOK_DECIDE = 10,
  PH_FINALIZE = 11
};

size_t phase_smem_bytes();
cudaError_t persistent_occupancy(int *blocks_per_sm);
cudaError_t launch_persistent(const RunArgs &ra, int grid, cudaStream_t s);
cudaError_t launch_phase(int phase, const RunArgs &ra, int grid, cudaStream_t s);
cudaError_t launch_core(const InstDev *d_inst, int m, double *dst, cudaStream_t s);
// core construction from the pivot sets (scratch: nb * RCAP * RCAP doubles)
cudaError_t launch_rebuild_cores(const InstDev *d_inst, int nb, double *scratch, int grid,
                                 cudaStream_t s);
// user generator: count / gather / scatter of the entries entering the
// superblocks (first != 0: the rank-one superblocks), and the error samples
cudaError_t launch_user_count(const InstDev *d_inst, int first, int64_t *counts, cudaStream_t s);
cudaError_t launch_user_gather(const InstDev *d_inst, int first, const int64_t *counts,
                               int32_t *idx, cudaStream_t s);
cudaError_t launch_user_scatter(const InstDev *d_inst, int first, const int64_t *counts,
                                const double *vals, cudaStream_t s);
cudaError_t launch_user_samples(const InstDev *d_inst, int32_t *idx, cudaStream_t s);
cudaError_t launch_maxwellian_tables(const InstDev *d_inst, double *coef, double *nh, double *cosx);

// tile geometry used to size the candidate buffer (host mirror of tile_geo)
int64_t host_tiles(int64_t n_b, int64_t n_b1, int64_t rl, int64_t rr, int32_t pr, int32_t pc);
// host replay of the kernels' tile arithmetic for one bond: violations found
int64_t host_check_bond_tiles(int d, const int64_t *n, const int32_t *r, const int32_t *r_stored,
                              const int32_t *grid, int b, int te, int64_t *ntiles);

}  // namespace ttc
