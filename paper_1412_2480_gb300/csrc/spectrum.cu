// spectrum.cu -- Fourier diagnostics of a grid quantity (the k-space maps of B_z in
// Sec. 3.1, Fig. 3): the 2D discrete Fourier transform
//   F^(p, q) = sum_{l, m} F(l, m) exp(-2 pi i (p l / nx + q m / ny)),
// returned as the amplitude |F^(p, q)| / (nx ny) in the fields' (ny, nx) layout, p and q
// in FFT order (index p >= nx/2 is the wave number 2 pi (p - nx) / (nx dx)).
//
// Each 1D transform runs in one CTA on shared memory as a Stockham autosort FFT
// (Stockham 1966; the per-stage indexing of Govindaraju et al., SC 2008): stage s with
// radix R combines R sub-transforms of length Ns into one of length Ns R; thread work
// item j reads x[j + t N/R] (t < R), multiplies by exp(-2 pi i t (j mod Ns) / (Ns R)),
// takes the R-point DFT and writes x'[(j / Ns) Ns R + (j mod Ns) + t Ns]. Lengths of the
// form 2^a 3^b 5^c up to kMaxN use radices 4, 2, 3, 5; other lengths fall back to the
// direct O(N^2) sum. Arithmetic is FP64 throughout, twiddles from sincospi.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "engine.h"
#include "pic.h"

namespace pic {

namespace {

constexpr int kFftThreads = 512;
constexpr int kMaxN = 8192;  // 128 KB of complex FP64 in shared memory
constexpr int kMaxStages = 16;

struct Plan {
    int n;
    int nst;
    int radix[kMaxStages];
    bool direct;  // not of the form 2^a 3^b 5^c (or longer than kMaxN): O(N^2) sum
};

Plan make_plan(int n) {
    Plan p{};
    p.n = n;
    int m = n;
    while (m % 4 == 0 && p.nst < kMaxStages) { p.radix[p.nst++] = 4; m /= 4; }
    while (m % 2 == 0 && p.nst < kMaxStages) { p.radix[p.nst++] = 2; m /= 2; }
    while (m % 3 == 0 && p.nst < kMaxStages) { p.radix[p.nst++] = 3; m /= 3; }
    while (m % 5 == 0 && p.nst < kMaxStages) { p.radix[p.nst++] = 5; m /= 5; }
    p.direct = m != 1 || n > kMaxN;
    return p;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place R-point forward DFT of v (exp(-2 pi i jk / R)), R = 2, 3, 4, 5.
template <int R>
__device__ __forceinline__ void dft_small(double2 v[R]) {
    if (R == 2) {
        const double2 a = v[0], b = v[1];
        v[0] = make_double2(a.x + b.x, a.y + b.y);
        v[1] = make_double2(a.x - b.x, a.y - b.y);
    } else if (R == 4) {
        const double2 a = make_double2(v[0].x + v[2].x, v[0].y + v[2].y);
        const double2 b = make_double2(v[0].x - v[2].x, v[0].y - v[2].y);
        const double2 c = make_double2(v[1].x + v[3].x, v[1].y + v[3].y);
        const double2 d = make_double2(v[1].x - v[3].x, v[1].y - v[3].y);  // times -i below
        v[0] = make_double2(a.x + c.x, a.y + c.y);
        v[2] = make_double2(a.x - c.x, a.y - c.y);
        v[1] = make_double2(b.x + d.y, b.y - d.x);
        v[3] = make_double2(b.x - d.y, b.y + d.x);
    } else {
        // general small R: direct sum with exact-angle twiddles
        double2 out[R];
#pragma unroll
        for (int k = 0; k < R; k++) {
            double2 acc = make_double2(0.0, 0.0);
#pragma unroll
            for (int j = 0; j < R; j++) {
                double s, c;
                sincospi(-2.0 * (double)((j * k) % R) / (double)R, &s, &c);
                acc.x += v[j].x * c - v[j].y * s;
                acc.y += v[j].x * s + v[j].y * c;
            }
            out[k] = acc;
        }
#pragma unroll
        for (int k = 0; k < R; k++) v[k] = out[k];
    }
}

// One Stockham stage of radix R on buf (length n), sub-transform length ns.
template <int R>
__device__ __forceinline__ void stage(double2* buf, int n, int ns) {
    constexpr int kPer = (kMaxN / R + kFftThreads - 1) / kFftThreads;  // work items per thread
    const int items = n / R;
    double2 v[kPer][R];
#pragma unroll
    for (int b = 0; b < kPer; b++) {
        const int j = threadIdx.x + b * kFftThreads;
        if (j < items) {
            const int jm = j % ns;
#pragma unroll
            for (int t = 0; t < R; t++) {
                double2 x = buf[j + t * items];
                if (t > 0 && jm > 0) {
                    double s, c;
                    sincospi(-2.0 * (double)(t * jm) / (double)(ns * R), &s, &c);
                    x = cmul(x, make_double2(c, s));
                }
                v[b][t] = x;
            }
            dft_small<R>(v[b]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < kPer; b++) {
        const int j = threadIdx.x + b * kFftThreads;
        if (j < items) {
            const int jm = j % ns;
            const int base = (j / ns) * ns * R + jm;
#pragma unroll
            for (int t = 0; t < R; t++) buf[base + t * ns] = v[b][t];
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void fft_smem(double2* buf, const Plan& p) {
    int ns = 1;
    for (int s = 0; s < p.nst; s++) {
        switch (p.radix[s]) {
        case 4: stage<4>(buf, p.n, ns); break;
        case 2: stage<2>(buf, p.n, ns); break;
        case 3: stage<3>(buf, p.n, ns); break;
        default: stage<5>(buf, p.n, ns); break;
        }
        ns *= p.radix[s];
    }
}

// Rows: the real field row m (length nx) -> its DFT along x into W (ny x nx complex).
__global__ void __launch_bounds__(kFftThreads) k_fft_rows(const double* __restrict__ F, int nx, int ny,
                                                          const Plan p, double2* __restrict__ W) {
    extern __shared__ double2 sbuf[];
    const int m = blockIdx.x;
    if (m >= ny) return;
    for (int l = threadIdx.x; l < nx; l += blockDim.x) sbuf[l] = make_double2(F[(long long)m * nx + l], 0.0);
    __syncthreads();
    fft_smem(sbuf, p);
    for (int l = threadIdx.x; l < nx; l += blockDim.x) W[(long long)m * nx + l] = sbuf[l];
}

// Columns: column p of W (length ny) -> its DFT along y, written as |.| * scale.
__global__ void __launch_bounds__(kFftThreads) k_fft_cols(const double2* __restrict__ W, int nx, int ny,
                                                          const Plan p, double scale, double* __restrict__ out) {
    extern __shared__ double2 sbuf[];
    const int col = blockIdx.x;
    if (col >= nx) return;
    for (int m = threadIdx.x; m < ny; m += blockDim.x) sbuf[m] = W[(long long)m * nx + col];
    __syncthreads();
    fft_smem(sbuf, p);
    for (int m = threadIdx.x; m < ny; m += blockDim.x) {
        const double2 z = sbuf[m];
        out[(long long)m * nx + col] = hypot(z.x, z.y) * scale;
    }
}

// Direct sums for lengths with other prime factors. Along x (complex out into W) ...
__global__ void k_dft_rows(const double* __restrict__ F, int nx, int ny, double2* __restrict__ W) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nx * ny) return;
    const int m = (int)(t / nx), k = (int)(t - (long long)m * nx);
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < nx; l++) {
        double s, c;
        sincospi(-2.0 * (double)(((long long)l * k) % nx) / (double)nx, &s, &c);
        const double f = F[(long long)m * nx + l];
        acc.x += f * c;
        acc.y += f * s;
    }
    W[t] = acc;
}

// ... and along y (amplitude out).
__global__ void k_dft_cols(const double2* __restrict__ W, int nx, int ny, double scale, double* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nx * ny) return;
    const int q = (int)(t / nx), col = (int)(t - (long long)q * nx);
    double2 acc = make_double2(0.0, 0.0);
    for (int m = 0; m < ny; m++) {
        double s, c;
        sincospi(-2.0 * (double)(((long long)m * q) % ny) / (double)ny, &s, &c);
        const double2 z = W[(long long)m * nx + col];
        acc.x += z.x * c - z.y * s;
        acc.y += z.x * s + z.y * c;
    }
    out[t] = hypot(acc.x, acc.y) * scale;
}

}  // namespace

int spectrum_2d(const double* F, int nx, int ny, double* out, cudaStream_t st, std::string& err) {
    const Plan px = make_plan(nx), py = make_plan(ny);
    const long long n = (long long)nx * ny;
    double2* W = nullptr;
    cudaError_t e = cudaMallocAsync(&W, n * sizeof(double2), st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        err = std::string("spectrum scratch: ") + cudaGetErrorString(e);
        return PIC_ENOMEM;
    }
    cudaFuncSetAttribute(k_fft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxN * (int)sizeof(double2));
    cudaFuncSetAttribute(k_fft_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxN * (int)sizeof(double2));
    const double scale = 1.0 / (double)n;
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (px.direct) k_dft_rows<<<nb, 256, 0, st>>>(F, nx, ny, W);
    else k_fft_rows<<<ny, kFftThreads, nx * sizeof(double2), st>>>(F, nx, ny, px, W);
    if (py.direct) k_dft_cols<<<nb, 256, 0, st>>>(W, nx, ny, scale, out);
    else k_fft_cols<<<nx, kFftThreads, ny * sizeof(double2), st>>>(W, nx, ny, py, scale, out);
    e = cudaGetLastError();
    cudaFreeAsync(W, st);
    if (e != cudaSuccess) {
        err = std::string("spectrum: ") + cudaGetErrorString(e);
        return PIC_ECUDA;
    }
    return PIC_OK;
}

}  // namespace pic
