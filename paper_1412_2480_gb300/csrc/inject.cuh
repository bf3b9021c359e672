// inject.cuh -- the moving injector of the shock configuration (include/pic.h): which
// pairs enter at the end of step n, and where and with which momenta. Used by the FP64
// and the MIXED32 particle halves alike.
#pragma once

#include "pic_internal.cuh"

namespace pic {

// splitmix64 (Steele, Lea & Flood 2014) as a stateless hash of a 64-bit counter.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Uniform in (0, 1) for draw d of pair k of row j at step n, species s.
__device__ __forceinline__ double inj_uniform(unsigned long long seed, long long n, int j, long long k, int s,
                                              int d) {
    const unsigned long long key = seed * 0xD1B54A32D192ED03ull + (unsigned long long)n * 0xABC98388FB8FAC03ull +
                                   (unsigned long long)j * 0x8CB92BA72F3D8DD7ull +
                                   (unsigned long long)k * 0x9E3779B97F4A7C15ull +
                                   (unsigned long long)s * 0xC2B2AE3D27D4EB4Full + (unsigned long long)d;
    return ((double)(splitmix64(key) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

// Slab width (cells) the injector fills per step, and the pairs per row injected in
// the first n steps.
__device__ __forceinline__ double inj_width(const GridDev& G) {
    return (1.0 + sqrt(1.0 - 1.0 / (G.gamma0 * G.gamma0))) * G.cfl;
}
__device__ __forceinline__ long long inj_cumulative(const GridDev& G, long long n) {
    return (long long)floor(((double)G.ppc * inj_width(G)) * (double)n);
}

// Pairs per row entering at the end of step n (0 once the plane has passed x = nx).
__device__ __forceinline__ long long inj_count(const GridDev& G, long long n) {
    if (!G.inject || G.inj_x0 + (double)(n + 1) * G.cfl > (double)G.nx) return 0;
    return inj_cumulative(G, n + 1) - inj_cumulative(G, n);
}

// Position (cells) of pair k of row j entering at the end of step n, and the momenta of
// species s.
__device__ __forceinline__ void inj_position(const GridDev& G, long long n, int j, long long k, double& x,
                                             double& y) {
    const double xf = G.inj_x0 + (double)(n + 1) * G.cfl;
    x = xf - inj_width(G) * inj_uniform(G.inj_seed, n, j, k, 0, 0);
    y = (double)j + inj_uniform(G.inj_seed, n, j, k, 0, 1);
}

__device__ __forceinline__ void inj_momentum(const GridDev& G, long long n, int j, long long k, int s,
                                             double u[3]) {
    const double two_pi = 6.283185307179586476925286766559;
    const double r0 = sqrt(-2.0 * log(inj_uniform(G.inj_seed, n, j, k, s, 2)));
    const double a0 = two_pi * inj_uniform(G.inj_seed, n, j, k, s, 3);
    const double r1 = sqrt(-2.0 * log(inj_uniform(G.inj_seed, n, j, k, s, 4)));
    const double a1 = two_pi * inj_uniform(G.inj_seed, n, j, k, s, 5);
    const double upx = G.u_th * r0 * cos(a0), upy = G.u_th * r0 * sin(a0), upz = G.u_th * r1 * cos(a1);
    const double gp = sqrt(1.0 + upx * upx + upy * upy + upz * upz);
    const double beta0 = sqrt(1.0 - 1.0 / (G.gamma0 * G.gamma0));
    u[0] = -G.gamma0 * (upx + beta0 * gp);
    u[1] = upy;
    u[2] = upz;
}

}  // namespace pic
