// mixed.h -- the MIXED32 particle half (int cell + FP32 offset, FP32 gather/push/deposit,
// tile-binned particles with shared-memory field and current windows), for one or many
// simulations sharing each launch.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "pic.h"
#include "pic_internal.cuh"

namespace pic {

struct MixedState;

// Choose tiles and allocate bins for ngrids simulations (fills the tile fields of the
// host descriptors G[0..ngrids), which the caller then copies to dgrids).
int mixed_create(MixedState** out, const pic_params* p, int ngrids, GridDev* G,
                 const GridDev* dgrids, long long ntot, float* F32, long long* Jfix, CgState* cg,
                 DevStatus* st, std::string& err);
void mixed_destroy(MixedState* m);
// Replace one species' particles of simulation g (FP64 physical positions and momenta,
// host or device).
int mixed_load(MixedState* m, int g, int sp, const double* x, const double* y, const double* ux,
               const double* uy, const double* uz, long long n, cudaStream_t s, std::string& err);
// Enqueue one part of the particle half of a step (the fixed-point current already
// zeroed): part 0 = overflow-list push, 1 = tile kernels, 2 = buffer swap.
void mixed_enqueue(MixedState* m, cudaStream_t s, int part);
// Host bookkeeping around a pic_step call (re-bin when bins overflowed).
int mixed_before_steps(MixedState* m, cudaStream_t s, std::string& err);
int mixed_after_steps(MixedState* m, cudaStream_t s, std::string& err);

// Kernels mixed_enqueue launches per step (all three parts together).
int mixed_step_kernels(const MixedState* m);
long long mixed_count(MixedState* m, int g, int sp);
// Add simulation g's node density into rho (device, ncell values; may be null), each
// particle of species s contributing q[s] (0: the species is left out), and w * its
// total momentum into mom (device, 3 values; may be null).
int mixed_rho_momentum(MixedState* m, int g, const double q[2], double* rho, double* mom, cudaStream_t s,
                       std::string& err);
long long mixed_rebins(MixedState* m);
// Bumped whenever device buffers are reallocated: step graphs captured before hold stale
// pointers and must be rebuilt.
long long mixed_generation(MixedState* m);
// Copy out one species of simulation g as FP64 [x, y, ux, uy, uz] (physical units).
int mixed_particles(MixedState* m, int g, int sp, double* out5xn, long long n, cudaStream_t s,
                    std::string& err);

}  // namespace pic
