// cnn.cu -- learned initial guess for the PCG solve of Eq. (7).
//
// A convolutional network of four 3x3 layers (3 -> 32 -> 32 -> 32 -> 3 channels,
// periodic padding, biases, no activation) maps b / rms(b) to dB_0 / rms(b), the three
// components of b and dB being three channels on the cell grid. The map it has to
// learn, b -> A^{-1} b, is linear (A = I - (theta c dt)^2 Lap), so the network is kept
// linear: a rectifier between layers only costs accuracy here. Scaling by rms(b) outside
// the network makes the guess exact in the scale of b whatever the grid size.
//
// Every convolution is an implicit GEMM on the tcgen05 tensor cores: a CTA of 128
// threads gathers the 3x3 neighbourhoods of 128 pixels (im2col, BF16) and the weights
// into shared memory, one thread issues the K/16 MMAs into an FP32 accumulator in tensor
// memory, and the accumulator is read back for the epilogue. The backward pass runs the
// same kernel with the transposed, flipped weights (input gradients) and a second
// tensor-core kernel for the weight gradients (pixels as the reduction dimension).
// Training keeps FP32 master weights updated by Adam.
//
// Quantisation points (a CPU reference reproduces them exactly): the input, the
// weights and every hidden activation and back-propagated gradient are rounded to BF16
// (round to nearest even); accumulation is FP32; the output and the loss are FP32.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cnn.h"
#include "tc.cuh"

struct pic_cnn {
    std::string err;
    int device = 0;
    cudaStream_t stream = nullptr;
    float* params = nullptr;  // FP32 master weights, PIC_CNN_NPARAMS
    float* grads = nullptr;
    float* m1 = nullptr;      // Adam moments
    float* m2 = nullptr;
    long long adam_t = 0;
    uint16_t* wf[4] = {nullptr, nullptr, nullptr, nullptr};  // forward operands
    uint16_t* wd[4] = {nullptr, nullptr, nullptr, nullptr};  // input-gradient operands (layers 2-4)
    // per-call buffers, grown on demand
    long long cap = 0;
    uint16_t* X[4] = {nullptr, nullptr, nullptr, nullptr};   // X0 [P][16], X1..X3 [P][32]
    uint16_t* dY[4] = {nullptr, nullptr, nullptr, nullptr};  // dY1..dY3 [P][32], dY4 [P][16]
    float* out = nullptr;     // [P][16]
    float* planes = nullptr;  // 2 x [P][3] staging of caller inputs
    pic::CnnImg* imgs = nullptr;
    int* tile_img = nullptr;
    int geo_nimg = 0, geo_nx = 0, geo_ny = 0;
    double* d_loss = nullptr;
    unsigned int* d_err = nullptr;
};

namespace pic {

namespace {

using bf16 = __nv_bfloat16;

struct Layer {
    int cin, cout, cin_pad, cout_pad;
    long long w_off, b_off;  // offsets of W[cout][9][cin] and b[cout] in the parameters
};

// parameters: layer by layer, W[co][tap][ci] (tap = 3 (dy + 1) + (dx + 1)) then b[co]
#define PIC_CNN_LAYERS                                      \
    {                                                       \
        {3, 32, 16, 32, 0, 864},                            \
        {32, 32, 32, 32, 896, 896 + 9216},                  \
        {32, 32, 32, 32, 896 + 9248, 896 + 9248 + 9216},    \
        {32, 3, 32, 16, 896 + 2 * 9248, 896 + 2 * 9248 + 864} \
    }
constexpr Layer kL[4] = PIC_CNN_LAYERS;
__constant__ Layer kLd[4] = PIC_CNN_LAYERS;  // the same table for device code
constexpr long long kNParams = 896 + 2 * 9248 + 867;
static_assert(kNParams == PIC_CNN_NPARAMS, "parameter count");

constexpr int kTile = 128;  // pixels per conv CTA
constexpr int kChunk = 64;  // pixels per weight-gradient MMA round

__device__ __forceinline__ int wrapn(int k, int n) { return k < 0 ? k + n : (k >= n ? k - n : k); }

// ---- convolution (forward, or input gradient with transposed weights) ---------------
struct ConvArgs {
    const CnnImg* imgs;
    const int* tile_img;
    const bf16* X;          // [P][CIN]
    const uint16_t* Wc;     // [NOUT x 9 CIN] BF16 in operand layout
    const float* bias;      // [cout] or nullptr
    int cout;               // channels that get a bias
    void* Y;                // [P][NOUT], BF16 or FP32
    unsigned int* err;
};

template <int CIN, int NOUT, bool OUTF32>
__global__ void __launch_bounds__(kTile) k_conv(const ConvArgs a) {
    constexpr int K = 9 * CIN;
    constexpr uint32_t SBO = (K / 8) * 128;
    constexpr int ABYTES = kTile * K * 2;
    constexpr int BBYTES = NOUT * K * 2;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;
    unsigned char* sB = smem + ABYTES;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) tc::tmem_alloc(&s_tmem, 32);
    if (tid == 0) tc::mbar_init(&bar, 1);
    // im2col: row tid = this thread's pixel, columns (tap, channel)
    const CnnImg im = a.imgs[a.tile_img[blockIdx.x]];
    const long long l = (long long)blockIdx.x * kTile + tid - im.off;
    const int j = (int)(l / im.nx), i = (int)(l - (long long)j * im.nx);
#pragma unroll
    for (int tap = 0; tap < 9; tap++) {
        const int ni = wrapn(i + tap % 3 - 1, im.nx), nj = wrapn(j + tap / 3 - 1, im.ny);
        const uint4* src = reinterpret_cast<const uint4*>(a.X + (im.off + (long long)nj * im.nx + ni) * CIN);
#pragma unroll
        for (int k8 = 0; k8 < CIN / 8; k8++)
            *reinterpret_cast<uint4*>(sA + tc::canon_offset(tid, tap * CIN + k8 * 8, K)) = __ldg(src + k8);
    }
    for (int q = tid; q < BBYTES / 16; q += kTile)
        reinterpret_cast<uint4*>(sB)[q] = __ldg(reinterpret_cast<const uint4*>(a.Wc) + q);
    tc::fence_smem_to_async();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    if (tid == 0) {
        const uint32_t idesc = tc::make_idesc(kTile, NOUT);
        const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
#pragma unroll 1
        for (int s = 0; s < K / 16; s++)
            tc::mma_bf16(tmem, tc::make_desc(a0 + s * 256, tc::kLbo, SBO), tc::make_desc(b0 + s * 256, tc::kLbo, SBO),
                         idesc, s > 0 ? 1u : 0u);
        tc::mma_commit(&bar);
    }
    // err[1]: the wait's poll limit (0: the default bound)
    const bool ok = __syncthreads_and(tc::mbar_wait_lim(&bar, 0, __ldg(a.err + 1)) ? 1 : 0) != 0;
    tc::fence_after_sync();
    if (ok) {
        float acc[NOUT];
#pragma unroll
        for (int c0 = 0; c0 < NOUT; c0 += 16) tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, acc + c0);
        if (a.bias) {
#pragma unroll
            for (int c = 0; c < NOUT; c++)
                if (c < a.cout) acc[c] += __ldg(a.bias + c);
        }
        const long long p = (long long)blockIdx.x * kTile + tid;
        if constexpr (OUTF32) {
            float4* dst = reinterpret_cast<float4*>(static_cast<float*>(a.Y) + p * NOUT);
#pragma unroll
            for (int c = 0; c < NOUT; c += 4) dst[c / 4] = make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
        } else {
            uint4* dst = reinterpret_cast<uint4*>(static_cast<bf16*>(a.Y) + p * NOUT);
#pragma unroll
            for (int c = 0; c < NOUT; c += 8) {
                uint4 v;
                __nv_bfloat162 h0 = __floats2bfloat162_rn(acc[c], acc[c + 1]);
                __nv_bfloat162 h1 = __floats2bfloat162_rn(acc[c + 2], acc[c + 3]);
                __nv_bfloat162 h2 = __floats2bfloat162_rn(acc[c + 4], acc[c + 5]);
                __nv_bfloat162 h3 = __floats2bfloat162_rn(acc[c + 6], acc[c + 7]);
                v.x = *reinterpret_cast<uint32_t*>(&h0);
                v.y = *reinterpret_cast<uint32_t*>(&h1);
                v.z = *reinterpret_cast<uint32_t*>(&h2);
                v.w = *reinterpret_cast<uint32_t*>(&h3);
                dst[c / 8] = v;
            }
        }
    } else if (tid == 0) {
        atomicExch(a.err, 1u);
        tc::mbar_wait(&bar, 0);  // drain: the MMA still reads shared and writes tensor memory
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, 32);
}

template <int CIN, int NOUT, bool OUTF32>
constexpr int conv_smem() {
    return kTile * 9 * CIN * 2 + NOUT * 9 * CIN * 2;
}

// ---- weight gradient: dW[co][tap][ci] += sum_p dY[p][co] X[nbr(p, tap)][ci] ----------
// A = rows (tap, ci) x pixels, B = co x pixels; pixels are the reduction dimension, in
// rounds of 64 pixels; the MT row tiles of 128 accumulate side by side in tensor memory.
struct WgradArgs {
    const CnnImg* imgs;
    const int* tile_img;
    const bf16* X;    // [P][CIN]
    const bf16* dY;   // [P][NOUT]
    float* dW;        // this layer's W[cout][9][cin] gradient
    int cin, cout;    // real channel counts
    long long nchunks;
    int chunks_per_cta;
    unsigned int* err;
};

template <int CIN, int NOUT>
__global__ void __launch_bounds__(128) k_wgrad(const WgradArgs a) {
    constexpr int ROWS = 9 * CIN;
    constexpr int MT = (ROWS + 127) / 128;
    constexpr int ABYTES = MT * 128 * kChunk * 2;
    constexpr uint32_t SBO = (kChunk / 8) * 128;
    constexpr uint32_t NCOLS = MT * NOUT <= 32 ? 32 : (MT * NOUT <= 64 ? 64 : 128);
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;
    unsigned char* sB = smem + ABYTES;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(&s_tmem, NCOLS);
    if (tid == 0) tc::mbar_init(&bar, 1);
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const long long c0 = (long long)blockIdx.x * a.chunks_per_cta;
    const long long c1 = min(a.nchunks, c0 + a.chunks_per_cta);
    const uint32_t lim = __ldg(a.err + 1);  // the waits' poll limit (0: the default bound)
    bool ok = true;
    for (long long c = c0; c < c1; c++) {
        const int q = (int)(c - c0);
        if (q > 0) ok = __syncthreads_and((ok && tc::mbar_wait_lim(&bar, (uint32_t)((q - 1) & 1), lim)) ? 1 : 0) != 0;
        if (!ok) {  // drain the round in flight before the shared and tensor memory go
            if (tid == 0) tc::mbar_wait(&bar, (uint32_t)((q - 1) & 1));
            break;
        }
        const long long pix0 = c * kChunk;
        const CnnImg im = a.imgs[a.tile_img[pix0 / kTile]];
        for (int idx = tid; idx < kChunk * 9; idx += 128) {
            const int px = idx % kChunk, tap = idx / kChunk;
            const long long l = pix0 + px - im.off;
            const int j = (int)(l / im.nx), i = (int)(l - (long long)j * im.nx);
            const int ni = wrapn(i + tap % 3 - 1, im.nx), nj = wrapn(j + tap / 3 - 1, im.ny);
            const uint4* src = reinterpret_cast<const uint4*>(a.X + (im.off + (long long)nj * im.nx + ni) * CIN);
#pragma unroll
            for (int k8 = 0; k8 < CIN / 8; k8++) {
                const uint4 v = __ldg(src + k8);
                const uint16_t* e = reinterpret_cast<const uint16_t*>(&v);
#pragma unroll
                for (int t = 0; t < 8; t++)
                    *reinterpret_cast<uint16_t*>(sA + tc::canon_offset(tap * CIN + k8 * 8 + t, px, kChunk)) = e[t];
            }
        }
        for (int idx = tid; idx < kChunk * (NOUT / 8); idx += 128) {
            const int px = idx / (NOUT / 8), c8 = idx % (NOUT / 8);
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(a.dY + (pix0 + px) * NOUT) + c8);
            const uint16_t* e = reinterpret_cast<const uint16_t*>(&v);
#pragma unroll
            for (int t = 0; t < 8; t++)
                *reinterpret_cast<uint16_t*>(sB + tc::canon_offset(c8 * 8 + t, px, kChunk)) = e[t];
        }
        tc::fence_smem_to_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t idesc = tc::make_idesc(128, NOUT);
            const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
#pragma unroll 1
            for (int m = 0; m < MT; m++)
#pragma unroll 1
                for (int s = 0; s < kChunk / 16; s++)
                    tc::mma_bf16(tmem + (uint32_t)(m * NOUT),
                                 tc::make_desc(a0 + (uint32_t)m * 128u * kChunk * 2u + s * 256, tc::kLbo, SBO),
                                 tc::make_desc(b0 + s * 256, tc::kLbo, SBO), idesc, (q > 0 || s > 0) ? 1u : 0u);
            tc::mma_commit(&bar);
        }
    }
    const int nq = (int)(c1 - c0);
    if (ok && nq > 0) {
        ok = __syncthreads_and(tc::mbar_wait_lim(&bar, (uint32_t)((nq - 1) & 1), lim) ? 1 : 0) != 0;
        if (!ok && tid == 0) tc::mbar_wait(&bar, (uint32_t)((nq - 1) & 1));  // drain
    }
    tc::fence_after_sync();
    if (ok && nq > 0) {
#pragma unroll 1
        for (int m = 0; m < MT; m++) {
            float acc[NOUT];
#pragma unroll
            for (int cc = 0; cc < NOUT; cc += 16)
                tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(m * NOUT + cc), acc + cc);
            const int row = m * 128 + warp * 32 + lane;
            if (row < ROWS) {
                const int tap = row / CIN, ci = row % CIN;
                if (ci < a.cin) {
#pragma unroll
                    for (int co = 0; co < NOUT; co++)
                        if (co < a.cout) atomicAdd(a.dW + ((long long)co * 9 + tap) * a.cin + ci, acc[co]);
                }
            }
        }
    } else if (!ok && tid == 0) {
        atomicExch(a.err, 1u);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, NCOLS);
}

template <int CIN, int NOUT>
constexpr int wgrad_smem() {
    return ((9 * CIN + 127) / 128) * 128 * kChunk * 2 + NOUT * kChunk * 2;
}

// ---- small kernels -------------------------------------------------------------------
// Operand-layout BF16 weights from the FP32 parameters: forward (rows = output
// channels, columns = (tap, input channel)) and input gradient (rows = input channels,
// columns = (tap', output channel) with the tap mirrored).
__global__ void k_pack(const float* __restrict__ prm, uint16_t* wf0, uint16_t* wf1, uint16_t* wf2, uint16_t* wf3,
                       uint16_t* wd1, uint16_t* wd2, uint16_t* wd3) {
    uint16_t* wf[4] = {wf0, wf1, wf2, wf3};
    uint16_t* wd[4] = {nullptr, wd1, wd2, wd3};
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    int base = 0;
    for (int L = 0; L < 4; L++) {
        const Layer y = kLd[L];
        const int Kf = 9 * y.cin_pad, nf = y.cout_pad * Kf;
        if (t >= base && t < base + nf) {
            const int e = t - base, n = e / Kf, k = e % Kf, tap = k / y.cin_pad, ci = k % y.cin_pad;
            const float v = (n < y.cout && ci < y.cin) ? prm[y.w_off + ((long long)n * 9 + tap) * y.cin + ci] : 0.f;
            const bf16 h = __float2bfloat16_rn(v);
            wf[L][tc::canon_offset(n, k, Kf) / 2] = *reinterpret_cast<const uint16_t*>(&h);
        }
        base += nf;
        if (L == 0) continue;
        const int Kd = 9 * y.cout_pad, nd = y.cin * Kd;  // rows: the layer's input channels
        if (t >= base && t < base + nd) {
            const int e = t - base, n = e / Kd, k = e % Kd, tp = k / y.cout_pad, co = k % y.cout_pad;
            const float v = (co < y.cout) ? prm[y.w_off + ((long long)co * 9 + (8 - tp)) * y.cin + n] : 0.f;
            const bf16 h = __float2bfloat16_rn(v);
            wd[L][tc::canon_offset(n, k, Kd) / 2] = *reinterpret_cast<const uint16_t*>(&h);
        }
        base += nd;
    }
}

int pack_total() {
    int n = 0;
    for (int L = 0; L < 4; L++) {
        n += kL[L].cout_pad * 9 * kL[L].cin_pad;
        if (L) n += kL[L].cin * 9 * kL[L].cout_pad;
    }
    return n;
}

// Caller planes [img][3][ny][nx] (FP32) -> BF16 [P][16].
__global__ void k_planes_in(long long P, long long npi, const float* __restrict__ in, bf16* __restrict__ X0) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const long long img = p / npi, l = p - img * npi;
    __align__(16) bf16 v[16];
#pragma unroll
    for (int c = 0; c < 16; c++) v[c] = __float2bfloat16_rn(c < 3 ? in[(img * 3 + c) * npi + l] : 0.f);
    reinterpret_cast<uint4*>(X0 + p * 16)[0] = reinterpret_cast<const uint4*>(v)[0];
    reinterpret_cast<uint4*>(X0 + p * 16)[1] = reinterpret_cast<const uint4*>(v)[1];
}

__global__ void k_planes_out(long long P, long long npi, const float* __restrict__ out, float* __restrict__ planes) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const long long img = p / npi, l = p - img * npi;
#pragma unroll
    for (int c = 0; c < 3; c++) planes[(img * 3 + c) * npi + l] = out[p * 16 + c];
}

// Mean squared error over the 3 output channels and its gradient, rounded to BF16.
__global__ void k_loss(long long P, long long npi, const float* __restrict__ out, const float* __restrict__ tgt,
                       bf16* __restrict__ dY4, double* loss) {
    __shared__ double red[32];
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (p < P) {
        const long long img = p / npi, l = p - img * npi;
        const float sc = 2.0f / (float)(3 * P);
        __align__(16) bf16 v[16];
#pragma unroll
        for (int c = 0; c < 16; c++) {
            float g = 0.f;
            if (c < 3) {
                const float d = out[p * 16 + c] - tgt[(img * 3 + c) * npi + l];
                s += (double)d * d;
                g = sc * d;
            }
            v[c] = __float2bfloat16_rn(g);
        }
        reinterpret_cast<uint4*>(dY4 + p * 16)[0] = reinterpret_cast<const uint4*>(v)[0];
        reinterpret_cast<uint4*>(dY4 + p * 16)[1] = reinterpret_cast<const uint4*>(v)[1];
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) atomicAdd(loss, s / (double)(3 * P));
}

// db[co] += sum_p dY[p][co], co < cout.
template <int NOUT>
__global__ void k_bias_grad(long long P, const bf16* __restrict__ dY, int cout, float* db) {
    __shared__ float red[32];
    for (int co = 0; co < cout; co++) {
        float s = 0.f;
        for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x)
            s += __bfloat162float(dY[p * NOUT + co]);
        s = block_sum(s, red);
        if (threadIdx.x == 0) atomicAdd(db + co, s);
        __syncthreads();
    }
}

__global__ void k_adam(long long n, float* w, const float* g, float* m1, float* m2, float lr, float c1, float c2) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float gi = g[k];
    const float a = b1 * m1[k] + (1.f - b1) * gi;
    const float b = b2 * m2[k] + (1.f - b2) * gi * gi;
    m1[k] = a;
    m2[k] = b;
    w[k] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

// The learned guess of the solver: x0 = K * b + bias rms(b), K the network collapsed
// into one 9x9 stencil (3 -> 3 channels). One CTA of 128 threads per 32 x 32 cell tile;
// b (FP64) of the tile and a 4-cell periodic halo is staged in shared memory as FP32.
// Each thread computes a column strip of kStrip cells for all three outputs: for every
// input channel and tap column it holds the strip's kStrip + 8 inputs in registers and
// reuses each for up to 9 x 3 products (one shared load per 5 FMAs instead of two per FMA).
constexpr int kGX = 32, kGY = 32, kGH = 4, kStrip = 8;
constexpr int kGuessThreads = kGX * (kGY / kStrip);

__global__ void __launch_bounds__(kGuessThreads) k_guess(const GridDev* __restrict__ grids,
                                                         const int* __restrict__ tile_grid,
                                                         const int* __restrict__ tile_local, long long ntot,
                                                         const double* __restrict__ b, const float* __restrict__ b32,
                                                         double* __restrict__ x, float* __restrict__ x32,
                                                         const float* __restrict__ Kg, const CgState* __restrict__ cg) {
    constexpr int WX = kGX + 2 * kGH, WY = kGY + 2 * kGH;
    __shared__ float sK[kGuessParams];
    __shared__ float sb[3][WY][WX];
    const int tid = threadIdx.x;
    const int g = tile_grid[blockIdx.x];
    const GridDev& G = grids[g];
    const int lt = tile_local[blockIdx.x];
    const int ntx = (G.nx + kGX - 1) / kGX;
    const int x0 = (lt % ntx) * kGX, y0 = (lt / ntx) * kGY;
    for (int k = tid; k < kGuessParams; k += blockDim.x) sK[k] = Kg[k];
    for (int k = tid; k < 3 * WY * WX; k += blockDim.x) {
        const int c = k / (WY * WX), r = k - c * (WY * WX), yy = r / WX, xx = r - yy * WX;
        int gx = ((x0 - kGH + xx) % G.nx + G.nx) % G.nx, sgn = 1;
        // with walls the halo holds the conductor's images of b: Bx odd on the integer-x
        // lattice, By and Bz even on the half-integer one (the images of the field solve)
        if (G.walls) gx = wall_col(x0 - kGH + xx, G.nx, c != 0, c == 0, sgn);
        const int gy = ((y0 - kGH + yy) % G.ny + G.ny) % G.ny;
        const long long o = c * ntot + G.cell_off + (long long)gy * G.nx + gx;
        sb[c][yy][xx] = sgn == 0 ? 0.f : (float)sgn * (b32 ? b32[o] : (float)b[o]);
    }
    __syncthreads();
    const int tx = tid % kGX, ys = (tid / kGX) * kStrip;  // this thread's column and first row
    float acc[3][kStrip];
#pragma unroll
    for (int co = 0; co < 3; co++)
#pragma unroll
        for (int r = 0; r < kStrip; r++) acc[co][r] = 0.f;
#pragma unroll 1
    for (int ci = 0; ci < 3; ci++) {
#pragma unroll 1
        for (int dx = 0; dx < kGuessTaps; dx++) {
            float in[kStrip + kGuessTaps - 1];
#pragma unroll
            for (int t = 0; t < kStrip + kGuessTaps - 1; t++) in[t] = sb[ci][ys + t][tx + dx];
#pragma unroll
            for (int dy = 0; dy < kGuessTaps; dy++) {
                const float k0 = sK[((0 * 3 + ci) * kGuessTaps + dy) * kGuessTaps + dx];
                const float k1 = sK[((1 * 3 + ci) * kGuessTaps + dy) * kGuessTaps + dx];
                const float k2 = sK[((2 * 3 + ci) * kGuessTaps + dy) * kGuessTaps + dx];
#pragma unroll
                for (int r = 0; r < kStrip; r++) {
                    acc[0][r] = fmaf(k0, in[r + dy], acc[0][r]);
                    acc[1][r] = fmaf(k1, in[r + dy], acc[1][r]);
                    acc[2][r] = fmaf(k2, in[r + dy], acc[2][r]);
                }
            }
        }
    }
    const int i = x0 + tx;
    if (i >= G.nx) return;
    const double rms = sqrt(cg[g].bb / (3.0 * G.ncell));
#pragma unroll
    for (int co = 0; co < 3; co++) {
        const double bias = (double)sK[kGuessWeights + co] * rms;
        const float biasf = (float)bias;
#pragma unroll
        for (int r = 0; r < kStrip; r++) {
            const int j = y0 + ys + r;
            if (j >= G.ny) continue;
            const long long o = co * ntot + G.cell_off + (long long)j * G.nx + i;
            if (x) x[o] = (double)acc[co][r] + bias;
            if (x32) x32[o] = acc[co][r] + biasf;  // the guess in FP32 for an FP32 residual
        }
    }
}

// ---- the GEMM building block, exposed for testing -----------------------------------
// D[M x N] = A[M x K] B[N x K]^T, one CTA per 128 rows.
__global__ void __launch_bounds__(128) k_tc_gemm(int N, int K, const uint16_t* __restrict__ A,
                                                 const uint16_t* __restrict__ B, float* __restrict__ D,
                                                 unsigned int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;
    unsigned char* sB = smem + 128 * K * 2;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5;
    uint32_t ncols = 32;
    while ((int)ncols < N) ncols <<= 1;
    if (warp == 0) tc::tmem_alloc(&s_tmem, ncols);
    if (tid == 0) tc::mbar_init(&bar, 1);
    const uint16_t* arow = A + ((long long)blockIdx.x * 128 + tid) * K;
    for (int k8 = 0; k8 < K / 8; k8++)
        *reinterpret_cast<uint4*>(sA + tc::canon_offset(tid, k8 * 8, K)) = reinterpret_cast<const uint4*>(arow)[k8];
    for (int idx = tid; idx < N * (K / 8); idx += 128) {
        const int n = idx / (K / 8), k8 = idx % (K / 8);
        *reinterpret_cast<uint4*>(sB + tc::canon_offset(n, k8 * 8, K)) =
            reinterpret_cast<const uint4*>(B + (long long)n * K)[k8];
    }
    tc::fence_smem_to_async();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const uint32_t sbo = (uint32_t)(K / 8) * 128u;
    if (tid == 0) {
        const uint32_t idesc = tc::make_idesc(128, N);
        const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
        for (int s = 0; s < K / 16; s++)
            tc::mma_bf16(tmem, tc::make_desc(a0 + s * 256, tc::kLbo, sbo), tc::make_desc(b0 + s * 256, tc::kLbo, sbo),
                         idesc, s > 0 ? 1u : 0u);
        tc::mma_commit(&bar);
    }
    const bool ok = __syncthreads_and(tc::mbar_wait_lim(&bar, 0, __ldg(err + 1)) ? 1 : 0) != 0;
    tc::fence_after_sync();
    if (ok) {
        float* drow = D + ((long long)blockIdx.x * 128 + tid) * N;
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int c = 0; c < 16; c++) drow[c0 + c] = v[c];
        }
    } else if (tid == 0) {
        atomicExch(err, 1u);
        tc::mbar_wait(&bar, 0);  // drain
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, ncols);
}

// ---- host side -------------------------------------------------------------------------
unsigned blocks(long long n, int b = 256) { return (unsigned)std::max<long long>(1, (n + b - 1) / b); }

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
    *p = nullptr;
    return cudaMalloc((void**)p, (n ? n : 1) * sizeof(T));
}

cudaError_t set_smem_once() {
    static cudaError_t e = [] {
        cudaError_t r = cudaFuncSetAttribute(k_conv<16, 32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             conv_smem<16, 32, false>());
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k_conv<32, 32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     conv_smem<32, 32, false>());
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k_conv<32, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     conv_smem<32, 16, true>());
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k_wgrad<16, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, wgrad_smem<16, 32>());
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k_wgrad<32, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, wgrad_smem<32, 32>());
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k_wgrad<32, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, wgrad_smem<32, 16>());
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        return r;
    }();
    return e;
}

template <int CIN, int NOUT, bool OUTF32>
void conv(long long ntiles, const CnnImg* imgs, const int* tile_img, const uint16_t* X, const uint16_t* W,
          const float* bias, int cout, void* Y, unsigned int* err, cudaStream_t st) {
    ConvArgs a{imgs, tile_img, reinterpret_cast<const bf16*>(X), W, bias, cout, Y, err};
    k_conv<CIN, NOUT, OUTF32><<<(unsigned)ntiles, kTile, conv_smem<CIN, NOUT, OUTF32>(), st>>>(a);
}

template <int CIN, int NOUT>
void wgrad(long long P, const CnnImg* imgs, const int* tile_img, const uint16_t* X, const uint16_t* dY, float* dW,
           int cin, int cout, unsigned int* err, cudaStream_t st) {
    WgradArgs a{};
    a.imgs = imgs;
    a.tile_img = tile_img;
    a.X = reinterpret_cast<const bf16*>(X);
    a.dY = reinterpret_cast<const bf16*>(dY);
    a.dW = dW;
    a.cin = cin;
    a.cout = cout;
    a.nchunks = P / kChunk;
    a.chunks_per_cta = 16;
    a.err = err;
    const long long ncta = (a.nchunks + a.chunks_per_cta - 1) / a.chunks_per_cta;
    k_wgrad<CIN, NOUT><<<(unsigned)ncta, 128, wgrad_smem<CIN, NOUT>(), st>>>(a);
}

// The forward pass X0 -> out through buffers Xa, Xb (X1..X3 kept when keep != null).
void forward(uint16_t* const wf[4], float* const bias[4], const float* prm, long long P, const CnnImg* imgs,
             const int* tile_img, const uint16_t* X0, uint16_t* X1, uint16_t* X2, uint16_t* X3, float* out,
             unsigned int* err, cudaStream_t st) {
    const long long nt = P / kTile;
    auto B = [&](int L) { return bias ? bias[L] : prm + kL[L].b_off; };
    conv<16, 32, false>(nt, imgs, tile_img, X0, wf[0], B(0), 32, X1, err, st);
    conv<32, 32, false>(nt, imgs, tile_img, X1, wf[1], B(1), 32, X2, err, st);
    conv<32, 32, false>(nt, imgs, tile_img, X2, wf[2], B(2), 32, X3, err, st);
    conv<32, 16, true>(nt, imgs, tile_img, X3, wf[3], B(3), 3, out, err, st);
}

}  // namespace

// ---- handle integration ------------------------------------------------------------------

// The four layers composed exactly (FP64, from the FP32 parameters): a chain of 3x3
// convolutions y(p) = sum_t W[t] x(p + off(t)) + b composes into one stencil whose
// offsets are the sums of the layers' offsets, and a bias that carries each earlier
// bias through the later layers' weights.
void collapse(const float* prm, double* K, double* bias) {
    // running composite: C x 3 channels, S x S taps (offset index = offset + (S - 1) / 2)
    int S = 3, C = kL[0].cout;
    std::vector<double> cur((size_t)C * 3 * S * S, 0.0), cb(C, 0.0);
    for (int o = 0; o < C; o++) {
        for (int t = 0; t < 9; t++)
            for (int i = 0; i < 3; i++)
                cur[((size_t)(o * 3 + i) * S + t / 3) * S + t % 3] = prm[kL[0].w_off + (o * 9 + t) * 3 + i];
        cb[o] = prm[kL[0].b_off + o];
    }
    for (int L = 1; L < 4; L++) {
        const Layer& y = kL[L];
        const int S2 = S + 2, C2 = y.cout;
        std::vector<double> nxt((size_t)C2 * 3 * S2 * S2, 0.0), nb(C2, 0.0);
        for (int o = 0; o < C2; o++) {
            nb[o] = prm[y.b_off + o];
            for (int t = 0; t < 9; t++) {
                const int ty = t / 3, tx = t % 3;  // offset + 1
                for (int m = 0; m < y.cin; m++) {
                    const double w = prm[y.w_off + (o * 9 + t) * y.cin + m];
                    nb[o] += w * cb[m];
                    for (int i = 0; i < 3; i++)
                        for (int a = 0; a < S; a++)
                            for (int c = 0; c < S; c++)
                                nxt[((size_t)(o * 3 + i) * S2 + a + ty) * S2 + c + tx] +=
                                    w * cur[((size_t)(m * 3 + i) * S + a) * S + c];
                }
            }
        }
        cur.swap(nxt);
        cb.swap(nb);
        S = S2;
        C = C2;
    }
    for (size_t k = 0; k < (size_t)kGuessWeights; k++) K[k] = cur[k];
    for (int o = 0; o < 3; o++) bias[o] = cb[o];
}

int cnn_make_guess(const pic_cnn* net, const GridDev* hg, int ngrids, CnnGuess* out, std::string& err) {
    cnn_free_guess(out);
    std::vector<float> prm(kNParams);
    std::vector<double> K(kGuessWeights), bias(3);
    cudaError_t e = cudaStreamSynchronize(net->stream);
    if (e == cudaSuccess) e = cudaMemcpy(prm.data(), net->params, kNParams * sizeof(float), cudaMemcpyDeviceToHost);
    std::vector<float> kf(kGuessParams);
    std::vector<int> tg, tl;
    if (e == cudaSuccess) {
        collapse(prm.data(), K.data(), bias.data());
        for (int k = 0; k < kGuessWeights; k++) kf[k] = (float)K[k];
        for (int o = 0; o < 3; o++) kf[kGuessWeights + o] = (float)bias[o];
        for (int g = 0; g < ngrids; g++) {
            const int nt = ((hg[g].nx + kGX - 1) / kGX) * ((hg[g].ny + kGY - 1) / kGY);
            for (int t = 0; t < nt; t++) {
                tg.push_back(g);
                tl.push_back(t);
            }
        }
        e = dalloc(&out->K, (size_t)kGuessParams);
    }
    if (e == cudaSuccess) e = dalloc(&out->tile_grid, tg.size());
    if (e == cudaSuccess) e = dalloc(&out->tile_local, tl.size());
    if (e == cudaSuccess) e = cudaMemcpy(out->K, kf.data(), kf.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(out->tile_grid, tg.data(), tg.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(out->tile_local, tl.data(), tl.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        err = std::string("learned guess set-up failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        cnn_free_guess(out);
        return PIC_ECUDA;
    }
    out->ntiles = (int)tg.size();
    return PIC_OK;
}

void cnn_free_guess(CnnGuess* g) {
    void* ps[] = {g->K, g->tile_grid, g->tile_local};
    for (void* p : ps)
        if (p) cudaFree(p);
    *g = CnnGuess{};
}

void launch_learned_guess(const CnnGuess& g, const GridDev* grids, const CgState* cg, long long ntot,
                          const double* b, const float* b32, double* x, float* x32, cudaStream_t st) {
    k_guess<<<(unsigned)g.ntiles, kGuessThreads, 0, st>>>(grids, g.tile_grid, g.tile_local, ntot, b, b32, x, x32,
                                                          g.K, cg);
}

}  // namespace pic

// =====================================================================================
using namespace pic;

namespace {

std::string g_cnn_err;

int cfail(pic_cnn* c, int code, const std::string& m) {
    if (c) c->err = m;
    else g_cnn_err = m;
    return code;
}

#define CCK(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            cudaGetLastError();                                                                     \
            return cfail(c, PIC_ECUDA, std::string(#call) + " failed: " + cudaGetErrorString(e_));  \
        }                                                                                           \
    } while (0)

void free_call_buffers(pic_cnn* c) {
    for (int L = 0; L < 4; L++) {
        if (c->X[L]) cudaFree(c->X[L]);
        if (c->dY[L]) cudaFree(c->dY[L]);
        c->X[L] = c->dY[L] = nullptr;
    }
    void* ps[] = {c->out, c->planes, c->imgs, c->tile_img};
    for (void* p : ps)
        if (p) cudaFree(p);
    c->out = nullptr;
    c->planes = nullptr;
    c->imgs = nullptr;
    c->tile_img = nullptr;
    c->cap = 0;
    c->geo_nimg = c->geo_nx = c->geo_ny = 0;
}

// Buffers and geometry for nimg images of nx x ny.
int prepare(pic_cnn* c, int nimg, int nx, int ny) {
    if (nimg < 1 || nx < 3 || ny < 3 || nimg > (1 << 20)) return cfail(c, PIC_EINVAL, "need nimg >= 1 and nx, ny >= 3");
    const long long npi = (long long)nx * ny;
    if (npi % kTile) return cfail(c, PIC_EINVAL, "nx*ny must be a multiple of 128");
    const long long P = npi * nimg;
    if (P > (1ll << 31)) return cfail(c, PIC_EINVAL, "too many pixels");
    if (P > c->cap) {
        free_call_buffers(c);
        for (int L = 0; L < 4; L++) {
            CCK(dalloc(&c->X[L], (size_t)P * (L == 0 ? 16 : 32)));
            CCK(dalloc(&c->dY[L], (size_t)P * (L == 3 ? 16 : 32)));
        }
        CCK(dalloc(&c->out, (size_t)P * 16));
        CCK(dalloc(&c->planes, (size_t)P * 6));
        CCK(dalloc(&c->tile_img, (size_t)(P / kTile)));
        c->cap = P;
    }
    if (c->geo_nimg != nimg || c->geo_nx != nx || c->geo_ny != ny) {
        if (c->imgs) cudaFree(c->imgs);
        c->imgs = nullptr;
        std::vector<CnnImg> im(nimg);
        std::vector<int> ti(P / kTile);
        for (int g = 0; g < nimg; g++) {
            im[g] = CnnImg{g * npi, nx, ny};
            for (long long t = g * npi / kTile; t < (g + 1) * npi / kTile; t++) ti[t] = g;
        }
        CCK(dalloc(&c->imgs, (size_t)nimg));
        CCK(cudaMemcpy(c->imgs, im.data(), nimg * sizeof(CnnImg), cudaMemcpyHostToDevice));
        CCK(cudaMemcpy(c->tile_img, ti.data(), ti.size() * sizeof(int), cudaMemcpyHostToDevice));
        c->geo_nimg = nimg;
        c->geo_nx = nx;
        c->geo_ny = ny;
    }
    return PIC_OK;
}

int pack(pic_cnn* c) {
    k_pack<<<blocks(pack_total()), 256, 0, c->stream>>>(c->params, c->wf[0], c->wf[1], c->wf[2], c->wf[3], c->wd[1],
                                                         c->wd[2], c->wd[3]);
    CCK(cudaGetLastError());
    return PIC_OK;
}

int check_err(pic_cnn* c) {
    unsigned int h = 0;
    CCK(cudaMemcpyAsync(&h, c->d_err, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CCK(cudaStreamSynchronize(c->stream));
    if (h) {
        CCK(cudaMemsetAsync(c->d_err, 0, sizeof(unsigned int), c->stream));  // reported once
        CCK(cudaStreamSynchronize(c->stream));
        return cfail(c, PIC_ETIMEOUT, "a tensor-core completion wait timed out");
    }
    return PIC_OK;
}

// forward (kept activations) + loss + backward into c->grads (zeroed first)
int gradient(pic_cnn* c, int nimg, int nx, int ny, const float* in, const float* tgt, double* loss) {
    if (int rc = prepare(c, nimg, nx, ny)) return rc;
    const long long npi = (long long)nx * ny, P = npi * nimg, nt = P / kTile;
    cudaStream_t st = c->stream;
    CCK(cudaMemcpyAsync(c->planes, in, P * 3 * sizeof(float), cudaMemcpyDefault, st));
    CCK(cudaMemcpyAsync(c->planes + P * 3, tgt, P * 3 * sizeof(float), cudaMemcpyDefault, st));
    if (int rc = pack(c)) return rc;
    k_planes_in<<<blocks(P), 256, 0, st>>>(P, npi, c->planes, reinterpret_cast<bf16*>(c->X[0]));
    forward(c->wf, nullptr, c->params, P, c->imgs, c->tile_img, c->X[0], c->X[1], c->X[2], c->X[3], c->out, c->d_err, st);
    CCK(cudaMemsetAsync(c->d_loss, 0, sizeof(double), st));
    k_loss<<<blocks(P), 256, 0, st>>>(P, npi, c->out, c->planes + P * 3, reinterpret_cast<bf16*>(c->dY[3]), c->d_loss);
    // input gradients: dY3 = bf16(dY4 * W4^T), dY2, dY1
    conv<16, 32, false>(nt, c->imgs, c->tile_img, c->dY[3], c->wd[3], nullptr, 0, c->dY[2], c->d_err, st);
    conv<32, 32, false>(nt, c->imgs, c->tile_img, c->dY[2], c->wd[2], nullptr, 0, c->dY[1], c->d_err, st);
    conv<32, 32, false>(nt, c->imgs, c->tile_img, c->dY[1], c->wd[1], nullptr, 0, c->dY[0], c->d_err, st);
    // weight and bias gradients
    CCK(cudaMemsetAsync(c->grads, 0, kNParams * sizeof(float), st));
    wgrad<16, 32>(P, c->imgs, c->tile_img, c->X[0], c->dY[0], c->grads + kL[0].w_off, 3, 32, c->d_err, st);
    wgrad<32, 32>(P, c->imgs, c->tile_img, c->X[1], c->dY[1], c->grads + kL[1].w_off, 32, 32, c->d_err, st);
    wgrad<32, 32>(P, c->imgs, c->tile_img, c->X[2], c->dY[2], c->grads + kL[2].w_off, 32, 32, c->d_err, st);
    wgrad<32, 16>(P, c->imgs, c->tile_img, c->X[3], c->dY[3], c->grads + kL[3].w_off, 32, 3, c->d_err, st);
    const unsigned bb = (unsigned)std::min<long long>(blocks(P), 304);
    k_bias_grad<32><<<bb, 256, 0, st>>>(P, reinterpret_cast<bf16*>(c->dY[0]), 32, c->grads + kL[0].b_off);
    k_bias_grad<32><<<bb, 256, 0, st>>>(P, reinterpret_cast<bf16*>(c->dY[1]), 32, c->grads + kL[1].b_off);
    k_bias_grad<32><<<bb, 256, 0, st>>>(P, reinterpret_cast<bf16*>(c->dY[2]), 32, c->grads + kL[2].b_off);
    k_bias_grad<16><<<bb, 256, 0, st>>>(P, reinterpret_cast<bf16*>(c->dY[3]), 3, c->grads + kL[3].b_off);
    CCK(cudaGetLastError());
    if (loss) CCK(cudaMemcpyAsync(loss, c->d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    return check_err(c);
}

}  // namespace

extern "C" {

int pic_cnn_create(pic_cnn** out) {
    if (!out) return cfail(nullptr, PIC_EINVAL, "out is NULL");
    *out = nullptr;
    pic_cnn* c = new (std::nothrow) pic_cnn();
    if (!c) return cfail(nullptr, PIC_ENOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = dalloc(&c->params, kNParams);
    if (e == cudaSuccess) e = dalloc(&c->grads, kNParams);
    if (e == cudaSuccess) e = dalloc(&c->m1, kNParams);
    if (e == cudaSuccess) e = dalloc(&c->m2, kNParams);
    for (int L = 0; L < 4 && e == cudaSuccess; L++) {
        e = dalloc(&c->wf[L], (size_t)kL[L].cout_pad * 9 * kL[L].cin_pad);
        if (e == cudaSuccess && L) e = dalloc(&c->wd[L], (size_t)kL[L].cin * 9 * kL[L].cout_pad);
    }
    if (e == cudaSuccess) e = dalloc(&c->d_loss, 1);
    if (e == cudaSuccess) e = dalloc(&c->d_err, 2);  // [0] a wait ran out, [1] the waits' poll limit
    if (e == cudaSuccess) e = cudaMemset(c->params, 0, kNParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(c->m1, 0, kNParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(c->m2, 0, kNParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, 2 * sizeof(unsigned int));
    if (e == cudaSuccess) e = set_smem_once();
    if (e == cudaSuccess && pack(c) != PIC_OK) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        g_cnn_err = std::string("pic_cnn_create: ") + cudaGetErrorString(e);
        cudaGetLastError();
        pic_cnn_free(c);
        return PIC_ECUDA;
    }
    *out = c;
    return PIC_OK;
}

void pic_cnn_free(pic_cnn* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_call_buffers(c);
    void* ps[] = {c->params, c->grads, c->m1, c->m2, c->d_loss, c->d_err};
    for (void* p : ps)
        if (p) cudaFree(p);
    for (int L = 0; L < 4; L++) {
        if (c->wf[L]) cudaFree(c->wf[L]);
        if (c->wd[L]) cudaFree(c->wd[L]);
    }
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char* pic_cnn_last_error(const pic_cnn* c) { return c ? c->err.c_str() : g_cnn_err.c_str(); }

int pic_cnn_set_params(pic_cnn* c, const float* p, int64_t n) {
    if (!c) return PIC_EINVAL;
    cudaSetDevice(c->device);
    if (!p || n != kNParams) return cfail(c, PIC_EINVAL, "need PIC_CNN_NPARAMS values");
    CCK(cudaMemcpyAsync(c->params, p, kNParams * sizeof(float), cudaMemcpyDefault, c->stream));
    CCK(cudaMemsetAsync(c->m1, 0, kNParams * sizeof(float), c->stream));
    CCK(cudaMemsetAsync(c->m2, 0, kNParams * sizeof(float), c->stream));
    c->adam_t = 0;
    if (int rc = pack(c)) return rc;
    CCK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

int pic_cnn_get_params(pic_cnn* c, float* p, int64_t n) {
    if (!c) return PIC_EINVAL;
    cudaSetDevice(c->device);
    if (!p || n != kNParams) return cfail(c, PIC_EINVAL, "need PIC_CNN_NPARAMS values");
    CCK(cudaMemcpyAsync(p, c->params, kNParams * sizeof(float), cudaMemcpyDefault, c->stream));
    CCK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

int pic_cnn_forward(pic_cnn* c, int32_t nimg, int32_t nx, int32_t ny, const float* in, float* out) {
    if (!c) return PIC_EINVAL;
    cudaSetDevice(c->device);
    if (!in || !out) return cfail(c, PIC_EINVAL, "NULL array");
    if (int rc = prepare(c, nimg, nx, ny)) return rc;
    const long long npi = (long long)nx * ny, P = npi * nimg;
    cudaStream_t st = c->stream;
    CCK(cudaMemcpyAsync(c->planes, in, P * 3 * sizeof(float), cudaMemcpyDefault, st));
    if (int rc = pack(c)) return rc;
    k_planes_in<<<blocks(P), 256, 0, st>>>(P, npi, c->planes, reinterpret_cast<bf16*>(c->X[0]));
    forward(c->wf, nullptr, c->params, P, c->imgs, c->tile_img, c->X[0], c->X[1], c->X[2], c->X[3], c->out, c->d_err, st);
    k_planes_out<<<blocks(P), 256, 0, st>>>(P, npi, c->out, c->planes + P * 3);
    CCK(cudaGetLastError());
    CCK(cudaMemcpyAsync(out, c->planes + P * 3, P * 3 * sizeof(float), cudaMemcpyDefault, st));
    return check_err(c);
}

int pic_cnn_gradient(pic_cnn* c, int32_t nimg, int32_t nx, int32_t ny, const float* in, const float* target,
                     float* grad, double* loss) {
    if (!c) return PIC_EINVAL;
    cudaSetDevice(c->device);
    if (!in || !target || !grad) return cfail(c, PIC_EINVAL, "NULL array");
    if (int rc = gradient(c, nimg, nx, ny, in, target, loss)) return rc;
    CCK(cudaMemcpyAsync(grad, c->grads, kNParams * sizeof(float), cudaMemcpyDefault, c->stream));
    CCK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

int pic_cnn_train_step(pic_cnn* c, int32_t nimg, int32_t nx, int32_t ny, const float* in, const float* target,
                       float lr, double* loss) {
    if (!c) return PIC_EINVAL;
    cudaSetDevice(c->device);
    if (!in || !target) return cfail(c, PIC_EINVAL, "NULL array");
    if (!(lr > 0.f) || lr > 1.f) return cfail(c, PIC_EINVAL, "lr must lie in (0, 1]");
    if (int rc = gradient(c, nimg, nx, ny, in, target, loss)) return rc;
    c->adam_t++;
    const float c1 = 1.f - std::pow(0.9f, (float)c->adam_t), c2 = 1.f - std::pow(0.999f, (float)c->adam_t);
    k_adam<<<blocks(kNParams), 256, 0, c->stream>>>(kNParams, c->params, c->grads, c->m1, c->m2, lr, c1, c2);
    CCK(cudaGetLastError());
    CCK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

int pic_cnn_stencil(pic_cnn* c, float* out, int64_t n) {
    if (!c) return PIC_EINVAL;
    cudaSetDevice(c->device);
    if (!out || n != kGuessParams) return cfail(c, PIC_EINVAL, "need PIC_CNN_STENCIL values");
    std::vector<float> prm(kNParams);
    std::vector<double> K(kGuessWeights), bias(3);
    CCK(cudaStreamSynchronize(c->stream));
    CCK(cudaMemcpy(prm.data(), c->params, kNParams * sizeof(float), cudaMemcpyDeviceToHost));
    collapse(prm.data(), K.data(), bias.data());
    std::vector<float> kf(kGuessParams);
    for (int k = 0; k < kGuessWeights; k++) kf[k] = (float)K[k];
    for (int o = 0; o < 3; o++) kf[kGuessWeights + o] = (float)bias[o];
    CCK(cudaMemcpy(out, kf.data(), kf.size() * sizeof(float), cudaMemcpyDefault));
    return PIC_OK;
}

int pic_tc_gemm_bf16(int32_t M, int32_t N, int32_t K, const uint16_t* A, const uint16_t* B, float* D) {
    pic_cnn* c = nullptr;
    if (M < 128 || M % 128 || N < 16 || N > 256 || N % 16 || K < 16 || K > 256 || K % 16 || !A || !B || !D)
        return cfail(c, PIC_EINVAL, "need M % 128 == 0, N in [16, 256] and K in [16, 256], multiples of 16");
    CCK(set_smem_once());
    unsigned int* err = nullptr;
    uint16_t *dA = nullptr, *dB = nullptr;
    float* dD = nullptr;
    CCK(dalloc(&err, 2));
    CCK(dalloc(&dA, (size_t)M * K));
    CCK(dalloc(&dB, (size_t)N * K));
    CCK(dalloc(&dD, (size_t)M * N));
    CCK(cudaMemcpy(dA, A, (size_t)M * K * 2, cudaMemcpyDefault));
    CCK(cudaMemcpy(dB, B, (size_t)N * K * 2, cudaMemcpyDefault));
    CCK(cudaMemset(err, 0, 2 * sizeof(unsigned int)));
    k_tc_gemm<<<M / 128, 128, (size_t)(128 + N) * K * 2>>>(N, K, dA, dB, dD, err);
    CCK(cudaGetLastError());
    unsigned int h = 0;
    CCK(cudaMemcpy(D, dD, (size_t)M * N * 4, cudaMemcpyDefault));
    CCK(cudaMemcpy(&h, err, sizeof h, cudaMemcpyDeviceToHost));
    cudaFree(err);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    if (h) return cfail(c, PIC_ETIMEOUT, "a tensor-core completion wait timed out");
    return PIC_OK;
}

int pic_cnn_set_wait_limit(pic_cnn* c, int32_t spins) {
    if (!c) return PIC_EINVAL;
    cudaSetDevice(c->device);
    if (spins < 0) return cfail(c, PIC_EINVAL, "spins must be >= 0");
    const unsigned int v = (unsigned int)spins;
    CCK(cudaMemcpyAsync(c->d_err + 1, &v, sizeof v, cudaMemcpyHostToDevice, c->stream));
    CCK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

}  // extern "C"
