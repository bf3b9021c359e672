// cnn.h -- the learned warm start of the PCG solve (see cnn.cu), as used by a handle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "pic.h"
#include "pic_internal.cuh"

namespace pic {

// One image (simulation grid) of a convolution launch: its first pixel and size.
// Pixels are cells, index cell_off + j nx + i; every image holds a multiple of 128.
struct CnnImg {
    long long off;
    int nx, ny;
};

// Forward-pass weights in tensor-core operand layout, owned by whoever copied them.
struct CnnWeights {
    uint16_t* wf[4] = {nullptr, nullptr, nullptr, nullptr};
    float* bias[4] = {nullptr, nullptr, nullptr, nullptr};
};

// Activation buffers and geometry tables for the grids of a handle.
struct CnnWork {
    uint16_t* X0 = nullptr;   // [npix][16] BF16 input
    uint16_t* Xa = nullptr;   // [npix][32] BF16 hidden (ping)
    uint16_t* Xb = nullptr;   // [npix][32] BF16 hidden (pong)
    float* out = nullptr;     // [npix][16] FP32 output
    CnnImg* imgs = nullptr;   // [ngrids]
    int* tile_img = nullptr;  // [npix / 128]
    long long npix = 0;
};

int cnn_copy_weights(const pic_cnn* net, CnnWeights* dst, std::string& err);
void cnn_free_weights(CnnWeights* w);
int cnn_alloc_work(CnnWork* w, const GridDev* hgrids, int ngrids, long long ntot, std::string& err);
void cnn_free_work(CnnWork* w);

// Enqueue the learned initial guess for every simulation: input b / rms(b) (rms over the
// simulation's 3 ncell values of b, from cg[g].bb), the network, x = output * rms(b).
// A simulation with b = 0 gets x = 0. tc_timeout is set if a tensor-core wait ran out.
void launch_learned_guess(const CnnWeights& w, const CnnWork& work, const GridDev* grids,
                          const CgState* cg, long long ntot, const double* b, double* x,
                          unsigned int* tc_timeout, cudaStream_t st);

}  // namespace pic
