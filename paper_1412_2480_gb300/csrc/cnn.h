// cnn.h -- the learned warm start of the PCG solve (see cnn.cu), as a handle uses it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "pic.h"
#include "pic_internal.cuh"

namespace pic {

// Taps of the collapsed network: the four 3x3 layers compose into one 9x9 stencil.
constexpr int kGuessTaps = 9;
constexpr int kGuessWeights = 3 * 3 * kGuessTaps * kGuessTaps;  // K[co][ci][dy + 4][dx + 4]
constexpr int kGuessParams = kGuessWeights + 3;                 // then the bias of each output

// One image (simulation grid) of a tensor-core convolution launch: its first pixel and
// size. Pixels are cells, index off + j nx + i; every image holds a multiple of 128.
struct CnnImg {
    long long off;
    int nx, ny;
};

// The learned guess of a handle: the network's exact collapse (FP32 stencil and bias,
// device memory) and the 32 x 8 cell tiles of all its simulations.
struct CnnGuess {
    float* K = nullptr;        // kGuessParams values
    int* tile_grid = nullptr;  // simulation of each tile
    int* tile_local = nullptr; // tile index within its simulation
    int ntiles = 0;
};

// Collapse the network's current parameters and build the tile tables.
int cnn_make_guess(const pic_cnn* net, const GridDev* hgrids, int ngrids, CnnGuess* out, std::string& err);
void cnn_free_guess(CnnGuess* g);

// Enqueue x0 = K * b + bias rms(b) for every simulation (rms over its 3 ncell values of
// b, from cg[g].bb): the network's output for input b / rms(b), scaled back by rms(b).
// b is read from b32 (an FP32 copy) when set, else from b; x0 goes to x (FP64) and/or
// x32 (FP32), whichever is set. With walls the stencil sees the conductor's images of b.
void launch_learned_guess(const CnnGuess& g, const GridDev* grids, const CgState* cg, long long ntot,
                          const double* b, const float* b32, double* x, float* x32, cudaStream_t st);

}  // namespace pic
