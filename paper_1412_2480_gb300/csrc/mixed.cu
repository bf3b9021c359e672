// mixed.cu -- the MIXED32 particle half of the step.
//
// Particles: int32 cell (i | j << 16) + FP32 in-cell offsets (ox, oy) in [0,1) + FP32
// momenta: 24 bytes per particle, structure-of-arrays, binned by (tile, species); a tile
// is tx x ty cells. Each bin has a stayer segment (capacity cap) and eight outboxes
// (capacity capo each), one per neighbouring tile. Bins are double-buffered: a step reads
// buffer `parity` and writes buffer `parity ^ 1`.
//
// A handle may hold many simulations of different sizes and shape orders (the batched
// parameter scan). Their tiles form one global list; each simulation's bins and count
// slots sit at its own offsets.
//
// Per step (inside the captured step graph):
//   0. k_mixed_begin / k_push_overflow: particles parked in the overflow list (no room
//      in a bin; normally none) are pushed straight from global memory;
//   1. k_push_tile<P>, one persistent launch per shape order P present: each CTA takes
//      the next tile of that order from a device work counter (tiles listed largest
//      first, so uneven simulations balance across the SMs), stages the FP32 field window
//      (tile + 2 cells below, 3 above, in x and y) into shared memory and zeroes a
//      fixed-point current window of the same size. Its particles are its own stayer segment plus the eight
//      neighbours' outboxes addressed to it. Warps run independently (no block barrier in
//      the particle loop): each gathers E^n, B^n, pushes (Boris), moves and deposits
//      J^{n+1/2} (Esirkepov) with native integer shared-memory atomics, then writes each
//      particle to the next buffer's stayer segment or to the outbox of the neighbour it
//      moved into, taking slots from warp-aggregated shared-memory counters. The current
//      window is added to the global fixed-point current at the end;
//   2. k_mixed_swap: the buffers swap.
// No global atomics are needed in steady state and no migration kernel runs. A particle
// found outside its tile is pushed with the same arithmetic and the same current
// rounding on global memory, so results never depend on bin capacity; a particle that
// finds no room goes to the overflow list and the host re-sorts with larger bins after
// the pic_step call. Count slots record every particle sent to a segment, parked ones
// included; readers clamp them to the segment's capacity.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "esirkepov.cuh"
#include "inject.cuh"
#include "mixed.h"

namespace pic {

constexpr int kTileThreads = 256;
constexpr int kNbr = 8;          // outboxes per bin, one per neighbouring tile
constexpr int kSegs = 1 + kNbr;  // count slots per bin: [0] stayers, [1 + o] outbox o

struct PartArrays {  // staging: one plain array per attribute
    int* cij;
    float *ox, *oy, *ux, *uy, *uz;
    int* gs;
};

// Bins and overflow lists: AoSoA of 32-particle chunks, each chunk holding its 32 cells,
// then 32 x-offsets, y-offsets, ux, uy, uz (6 x 128 bytes): a warp touches whole lines
// and one base pointer addresses every attribute.
constexpr int kFields = 6;
struct Slots {
    unsigned* p;
    int* gs;  // species of each slot (overflow lists only)
};

__host__ __device__ __forceinline__ size_t aos(long long k, int f) {
    return (size_t)(k >> 5) * (32 * kFields) + (size_t)f * 32 + (size_t)(k & 31);
}

struct MixedArgs {
    const GridDev* grids;
    const int* tile_grid;  // simulation of each global tile
    const int* tlist;      // tiles of this launch's shape order, largest first
    int ntl;               // entries of tlist
    int* work;             // next entry of tlist to take (zeroed every step)
    long long ntot;
    const float* F32;
    long long* Jfix;
    unsigned* buf[2];
    int* cnt[2];     // [nbins * kSegs] per parity: particles sent to each segment
    int* ovf_in[2];  // [ntiles_total] per parity: particles the overflow kernel moved in
    Slots ovf[2];
    long long ovf_cap;
    CgState* cg;
    DevStatus* st;
};

struct MixedState {
    int ngrids = 0;
    GridDev* G = nullptr;  // host descriptors [ngrids], owned by the caller
    const GridDev* dgrids = nullptr;
    long long ntot = 0;
    float* F32 = nullptr;
    long long* Jfix = nullptr;
    CgState* cg = nullptr;
    DevStatus* st = nullptr;
    unsigned* buf[2] = {nullptr, nullptr};
    Slots ovf[2]{};
    int* cnt[2] = {nullptr, nullptr};  // [ntiles_total * 2 * kSegs] per parity, then ovf_in
    int* ovf_in[2] = {nullptr, nullptr};  // [ntiles_total] per parity (inside cnt's block)
    long long nslots = 0, ovf_cap = 0;
    int ntiles_total = 0;
    int* tile_grid = nullptr;     // device [ntiles_total]
    int* tlist = nullptr;         // device: tiles grouped by shape order, largest first
    int* work = nullptr;          // device [4]: work counter of each order's launch
    int order_first[4] = {0, 0, 0, 0}, order_n[4] = {0, 0, 0, 0};
    size_t smem[4] = {0, 0, 0, 0};  // dynamic shared memory of each order's launch
    int pblocks[4] = {0, 0, 0, 0};  // persistent CTAs of each order's launch
    std::vector<long long> n;     // live particles [2 g + species]
    unsigned long long* injected = nullptr;  // device [2 ngrids]: pairs added by the injector
    int inject_grids = 0;         // simulations with an injector
    long long inject_threads = 0; // rows x most pairs per row, over those simulations
    int* inj_grid = nullptr;      // device [inject_grids]: their indices
    long long* inj_first = nullptr;  // device [inject_grids + 1]: first thread of each
    long long rebins = 0;
    long long gen = 0;  // allocation generation of the bin buffers
};

namespace {

__host__ __device__ __forceinline__ long long bin_stride(const GridDev& G) {
    return G.cap + kNbr * G.capo;
}

// Outbox index of a move by (dx, dy) tiles, (dx, dy) != (0, 0).
__host__ __device__ __forceinline__ int outbox_of(int dx, int dy) {
    const int d = (dy + 1) * 3 + (dx + 1);
    return d < 4 ? d : d - 1;
}

__host__ __device__ __forceinline__ void dir_of(int o, int& dx, int& dy) {
    const int d = o < 4 ? o : o + 1;
    dx = d % 3 - 1;
    dy = d / 3 - 1;
}

// The tile (within its simulation) whose bin holds segment k of the particles tile
// (txi, tyi) pushes: its own stayers (k = 0), or the outbox k - 1 of the neighbour on the
// opposite side, which is addressed to it.
__device__ __forceinline__ int segment_source(const GridDev& G, int txi, int tyi, int k) {
    if (k == 0) return tyi * G.ntx + txi;
    int dx, dy;
    dir_of(k - 1, dx, dy);
    const int sx = (txi - dx + G.ntx) % G.ntx, sy = (tyi - dy + G.nty) % G.nty;
    return sy * G.ntx + sx;
}

// Particles of species s sent to segment k of bin `src` in the last step (count slots of
// the current buffer). The count includes those that found no room and were parked in
// the overflow list; the segment itself holds at most its capacity of them.
__device__ __forceinline__ int segment_sent(const GridDev& G, const int* ccur, int src, int s, int k) {
    return ccur[((long long)G.tile_first * 2 + (long long)src * 2 + s) * kSegs + k];
}

// Particles whose cell lies in tile lt at the start of the step, both species, wherever
// they are stored: those sent to its segments (parked ones included) and those the
// overflow kernel moved into it. This count does not depend on which particles found
// room in the bins, so neither does the rounding it sets.
__device__ __forceinline__ int tile_population(const GridDev& G, const int* ccur, const int* oin, int lt) {
    const int tyi = lt / G.ntx, txi = lt - tyi * G.ntx;
    int n = oin[G.tile_first + lt];
    for (int s = 0; s < 2; s++)
        for (int k = 0; k < kSegs; k++) n += segment_sent(G, ccur, segment_source(G, txi, tyi, k), s, k);
    return n;
}

// Tile (within its simulation) of cell (i, j).
__device__ __forceinline__ int tile_of(const GridDev& G, int i, int j) { return (j / G.ty) * G.ntx + i / G.tx; }

// ---------------------------------------------------------------------------------
// Memory views used by the shared push arithmetic.
// ---------------------------------------------------------------------------------
// The tile's current window accumulates fixed point in two 32-bit words per node: 32-bit
// integer shared atomics are single native instructions, while float and 64-bit ones
// loop on compare-and-swap. Every single-particle contribution to a node is bounded by
// u/2 (GridDev::jscale = 2^40/u). A contribution v becomes x = v 2^k/u, split into its
// nearest integer hi and the rest r = x - hi in [-1/2, 1/2], and lo = round(r 2^lb);
// integers come from one FMA with 1.5 * 2^23 (exact below 2^22 in magnitude). Each tile
// picks k, lb <= 30 - log2(n + 1) from its population n, the particles whose cell lies in
// it (no word can wrap, whatever the distribution), with k <= 22 and lb <= 16, i.e. a
// resolution of 2^-(k+lb) u. The flush adds hi 2^(40-k) + lo 2^(40-k-lb) exactly into
// the 64-bit global current.
// A particle pushed on global memory (outside its tile's window, or parked in the
// overflow list) rounds the same way, with the k and lb of the tile its cell lies in, so
// a particle's current does not depend on the path it takes and a run is bit-for-bit
// reproducible whichever particles find room in the bins.
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;

struct FixedScale {
    int k, lb;
    float js;   // window scale 2^k / u
    float jlb;  // 2^lb
};

__device__ __forceinline__ FixedScale fixed_scale(const GridDev& G, int n_tile) {
    const int room = 30 - (32 - __clz(n_tile));  // n_tile < 2^(30 - room)
    FixedScale f;
    f.k = min(22, room);
    f.lb = min(16, room);
    f.js = G.js40 * __int_as_float((127 + f.k) << 23);  // js40 2^k: exact, = jscale 2^(k-40) rounded
    f.jlb = (float)(1 << f.lb);
    return f;
}

// x (window units) -> the two words (hi, lo)
__device__ __forceinline__ void fixed_split(float x, float jlb, int& hi, int& lo) {
    const float xr = xadd(x, kMagic);
    hi = __float_as_int(xr) - kMagicBits;
    const float r = xsub(x, xsub(xr, kMagic));  // exact: |r| <= 1/2
    lo = __float_as_int(xfma(r, jlb, kMagic)) - kMagicBits;
}

// (hi, lo) summed in a window -> global fixed-point units
__device__ __forceinline__ long long fixed_value(long long hi, long long lo, const FixedScale& f) {
    return hi * (1ll << (40 - f.k)) + lo * (1ll << (40 - f.k - f.lb));
}

// The tile's field window pairs the components that share a lattice -- (Ex, By) at
// (i+1/2, j) and (Ey, Bx) at (i, j+1/2) -- as float2, so one 64-bit load serves two
// components; Ez and Bz follow as plain arrays: [(Ex,By) x NW][(Ey,Bx) x NW][Ez][Bz].
struct WinMem {  // tile window in shared memory; indices are window-local
    const float* fw;
    int* jhi;
    int* jlo;
    int wx, nw;
    float js;   // window scale 2^k / u
    float jlb;  // 2^lb
    __device__ __forceinline__ float2 ld_exby(int ix, int iy) const {
        return reinterpret_cast<const float2*>(fw)[iy * wx + ix];
    }
    __device__ __forceinline__ float2 ld_eybx(int ix, int iy) const {
        return reinterpret_cast<const float2*>(fw + 2 * nw)[iy * wx + ix];
    }
    __device__ __forceinline__ float ld_ez(int ix, int iy) const { return fw[4 * nw + iy * wx + ix]; }
    __device__ __forceinline__ float ld_bz(int ix, int iy) const { return fw[5 * nw + iy * wx + ix]; }
    // x: the contribution already in window units (the push folds js into its deposit
    // constants). A lane whose high word is zero leaves it alone for Jy and Jz (c, a
    // constant once the deposit is unrolled): below half a window unit, as the transverse
    // currents of a relativistic beam are, a contribution lives in the low word only, and
    // an atomic with fewer active lanes takes fewer shared-memory wavefronts (its bank
    // conflicts are among the active lanes). Jx, large along the beam, skips the test.
    // Adding zero changes nothing, so the current is the same to the bit.
    __device__ __forceinline__ void add(int c, int ix, int iy, float x) const {
        int hi, lo;
        fixed_split(x, jlb, hi, lo);
        const int k = c * nw + iy * wx + ix;
        if (c == 0 || hi != 0) atomicAdd(&jhi[k], hi);
        atomicAdd(&jlo[k], lo);
    }
};

struct GlobalMem {  // global grid arrays of one simulation; indices are global
    const float* F;
    unsigned long long* J;
    long long ntot;
    int nx, ny;
    FixedScale f;  // the rounding of the tile the particle's cell lies in
    float js;      // = f.js: contributions arrive in that tile's window units
    int walls;
    __device__ __forceinline__ long long at(int ix, int iy) const {
        return (long long)wrapi(iy, ny) * nx + wrapi(ix, nx);
    }
    __device__ __forceinline__ float ld(int c, int ix, int iy) const {
        if (!walls) return __ldg(F + c * ntot + at(ix, iy));
        const bool half = c == 0 || c == 4 || c == 5;  // Ex, By, Bz at half-integer x
        int s;
        const int cx = wall_col(ix, nx, half, !half, s);
        return s == 0 ? 0.f : (float)s * __ldg(F + c * ntot + (long long)wrapi(iy, ny) * nx + cx);
    }
    // x: the contribution in window units (times js), rounded as the window rounds it
    __device__ __forceinline__ void add(int c, int ix, int iy, float x) const {
        int hi, lo;
        fixed_split(x, f.jlb, hi, lo);
        const long long v = fixed_value(hi, lo, f);
        if (!walls) {
            atomicAdd(J + c * ntot + at(ix, iy), (unsigned long long)v);
            return;
        }
        int s;
        const int cx = wall_col(ix, nx, c == 0, c == 0, s);  // mirror image: Jx odd
        if (s != 0) atomicAdd(J + c * ntot + (long long)wrapi(iy, ny) * nx + cx, (unsigned long long)(s * v));
    }
};

template <int P, typename Mem>
__device__ __forceinline__ float gather(const Mem& M, int c, int bx, const float wx[P + 1], int by,
                                        const float wy[P + 1]) {
    float acc = 0.f;
#pragma unroll
    for (int b = 0; b <= P; b++) {
        float ra = 0.f;
#pragma unroll
        for (int a = 0; a <= P; a++) ra = fmaf(wx[a], M.ld(c, bx + a, by + b), ra);
        acc = fmaf(wy[b], ra, acc);
    }
    return acc;
}

// All six components at a particle: E, B. (bxe, wxe, bye, wye): the x and y shape of the
// half-integer-x lattice components (Ex, By, Bz in x; Ey, Bx, Bz in y use (bxh..)); in
// the node-averaged reading every component uses the node shape.
template <int P>
__device__ __forceinline__ void gather_fields(const GlobalMem& M, int bx0, const float wx0[P + 1], int bxh,
                                              const float wxh[P + 1], int by0, const float wy0[P + 1], int byh,
                                              const float wyh[P + 1], float E[3], float B[3]) {
    E[0] = gather<P>(M, 0, bxh, wxh, by0, wy0);
    E[1] = gather<P>(M, 1, bx0, wx0, byh, wyh);
    E[2] = gather<P>(M, 2, bx0, wx0, by0, wy0);
    B[0] = gather<P>(M, 3, bx0, wx0, byh, wyh);
    B[1] = gather<P>(M, 4, bxh, wxh, by0, wy0);
    B[2] = gather<P>(M, 5, bxh, wxh, byh, wyh);
}

template <int P>
__device__ __forceinline__ void gather_fields(const WinMem& M, int bx0, const float wx0[P + 1], int bxh,
                                              const float wxh[P + 1], int by0, const float wy0[P + 1], int byh,
                                              const float wyh[P + 1], float E[3], float B[3]) {
    float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
    float ez = 0.f, bz = 0.f;
#pragma unroll
    for (int r = 0; r <= P; r++) {
        float2 ra = make_float2(0.f, 0.f), rb = make_float2(0.f, 0.f);
        float rz = 0.f, rbz = 0.f;
#pragma unroll
        for (int t = 0; t <= P; t++) {
            const float2 va = M.ld_exby(bxh + t, by0 + r);
            const float2 vb = M.ld_eybx(bx0 + t, byh + r);
            ra.x = fmaf(wxh[t], va.x, ra.x);
            ra.y = fmaf(wxh[t], va.y, ra.y);
            rb.x = fmaf(wx0[t], vb.x, rb.x);
            rb.y = fmaf(wx0[t], vb.y, rb.y);
            rz = fmaf(wx0[t], M.ld_ez(bx0 + t, by0 + r), rz);
            rbz = fmaf(wxh[t], M.ld_bz(bxh + t, byh + r), rbz);
        }
        a.x = fmaf(wy0[r], ra.x, a.x);
        a.y = fmaf(wy0[r], ra.y, a.y);
        b.x = fmaf(wyh[r], rb.x, b.x);
        b.y = fmaf(wyh[r], rb.y, b.y);
        ez = fmaf(wy0[r], rz, ez);
        bz = fmaf(wyh[r], rbz, bz);
    }
    E[0] = a.x;
    B[1] = a.y;
    E[1] = b.x;
    B[0] = b.y;
    E[2] = ez;
    B[2] = bz;
}

struct PushConst {
    float h;        // (q/m) dt / 2
    float dt_idx;   // dt / dx
    float dt_idy;   // dt / dy
    float fx, fy;   // q dx / (dt dx dy), q dy / (dt dx dy)
    float fz;       // q / (dx dy)   (times vz)
    int deposit;
    int nodal;      // the fields hold node averages: every component on the node lattice
};

// Gather, Boris push, move with carry into the neighbouring cell, and deposit, for one
// particle at cell (i, j) of M's index space with offsets (ox, oy). On return ox, oy, u
// hold the new state and di, dj the cell carry (-1, 0, +1). Returns false (and leaves
// the position unchanged) if the move is not below one cell or is not finite.
template <int P, typename Mem>
__device__ __forceinline__ bool push_one(const Mem& M, const PushConst& K, int i, int j, float& ox,
                                         float& oy, float u[3], int& di, int& dj, float& ek) {
    int bx0, by0;
    float wx0[P + 1], wy0[P + 1];
    shape_nodes<P, float>(i, ox, bx0, wx0);
    shape_nodes<P, float>(j, oy, by0, wy0);
    float E[3], B[3];
    if (K.nodal) {  // node-averaged fields: the deposit's weights for every component
        gather_fields<P>(M, bx0, wx0, bx0, wx0, by0, wy0, by0, wy0, E, B);
    } else {
        // Ex (i+1/2, j), Ey (i, j+1/2), Ez (i, j), Bx (i, j+1/2), By (i+1/2, j), Bz (i+1/2, j+1/2)
        int bxh, byh;
        float wxh[P + 1], wyh[P + 1];
        shape_nodes_half<P, float>(i, ox, bxh, wxh);
        shape_nodes_half<P, float>(j, oy, byh, wyh);
        gather_fields<P>(M, bx0, wx0, bxh, wxh, by0, wy0, byh, wyh, E, B);
    }
    // (the rounding of the update is explicit: xmul, xfma, ... in pic_internal.cuh)
    const float g2_old = xfma(u[2], u[2], xfma(u[1], u[1], xfma(u[0], u[0], 1.f)));
    boris<float>(K.h, E, B, u);
    const float ig = rsqrtf(xfma(u[2], u[2], xfma(u[1], u[1], xfma(u[0], u[0], 1.f))));
    const float dX = xmul(xmul(K.dt_idx, u[0]), ig), dY = xmul(xmul(K.dt_idy, u[1]), ig);
    di = 0;
    dj = 0;
    if (!(fabsf(dX) < 1.f && fabsf(dY) < 1.f)) return false;
    ek += xmul(g2_old, rsqrtf(g2_old)) + rcp_push(ig) - 2.f;  // gamma before + gamma after - 2
    float x1 = xadd(ox, dX), y1 = xadd(oy, dY);
    if (x1 >= 1.f) { x1 = xsub(x1, 1.f); di = 1; }
    else if (x1 < 0.f) { x1 = xadd(x1, 1.f); di = -1; if (x1 >= 1.f) { x1 = 0.f; di = 0; } }
    if (y1 >= 1.f) { y1 = xsub(y1, 1.f); dj = 1; }
    else if (y1 < 0.f) { y1 = xadd(y1, 1.f); dj = -1; if (y1 >= 1.f) { y1 = 0.f; dj = 0; } }
    if (K.deposit)
        esirkepov<P, float>(i, ox, j, oy, i + di, x1, j + dj, y1, xmul(K.fx, M.js), xmul(K.fy, M.js),
                            xmul(xmul(K.fz, xmul(u[2], ig)), M.js),
                            [M](int c, int ix, int iy, float v) { M.add(c, ix, iy, v); });
    ox = x1;
    oy = y1;
    return true;
}

__device__ __forceinline__ PushConst push_const(const GridDev& G, int s) {
    PushConst K;
    K.h = G.pk_h[s];
    K.dt_idx = G.pk_dtx;
    K.dt_idy = G.pk_dty;
    K.fx = G.pk_fx[s];
    K.fy = G.pk_fy[s];
    K.fz = G.pk_fz[s];
    K.deposit = G.deposit;
    K.nodal = G.nodal;
    return K;
}

__device__ __forceinline__ void flag_bad(DevStatus* st, const float u[3]) {
    if (isfinite(u[0] + u[1] + u[2])) atomicAdd(&st->cfl_viol, 1ull);
    else atomicAdd(&st->nan_count, 1ull);
    st->stop_next = 1u;
}

__device__ __forceinline__ void put(unsigned* P, long long k, int c, float ox, float oy,
                                    const float u[3]) {
    __stcs(P + aos(k, 0), (unsigned)c);
    __stcs(reinterpret_cast<float*>(P) + aos(k, 1), ox);
    __stcs(reinterpret_cast<float*>(P) + aos(k, 2), oy);
    __stcs(reinterpret_cast<float*>(P) + aos(k, 3), u[0]);
    __stcs(reinterpret_cast<float*>(P) + aos(k, 4), u[1]);
    __stcs(reinterpret_cast<float*>(P) + aos(k, 5), u[2]);
}

__device__ __forceinline__ void get(const unsigned* P, long long k, int& c, float& ox, float& oy,
                                    float u[3]) {
    const float* F = reinterpret_cast<const float*>(P);
    c = (int)__ldcs(P + aos(k, 0));
    ox = __ldcs(F + aos(k, 1));
    oy = __ldcs(F + aos(k, 2));
    u[0] = __ldcs(F + aos(k, 3));
    u[1] = __ldcs(F + aos(k, 4));
    u[2] = __ldcs(F + aos(k, 5));
}

// Append to the overflow list of the next buffer; a full list is a fatal error. An
// entry records its simulation and species as gs = species | (simulation << 1).
__device__ __forceinline__ void to_overflow(unsigned* op, int* ogs, long long ovf_cap, DevStatus* st,
                                         int nxt, int c, float ox, float oy, float u0, float u1,
                                         float u2, int gs) {
    const unsigned long long o = atomicAdd(&st->ovf_count[nxt], 1ull);
    atomicAdd(&st->overflow, 1ull);
    if ((long long)o < ovf_cap) {
        const float u[3] = {u0, u1, u2};
        put(op, (long long)o, c, ox, oy, u);
        ogs[o] = gs;
    } else {
        atomicAdd(&st->lost, 1ull);  // storage exhausted: the step fails with PIC_ENOMEM
        st->stop_next = 1u;
    }
}

// ---------------------------------------------------------------------------------
// 1. Tile kernel
// ---------------------------------------------------------------------------------
// Resident CTAs per SM the order-2 tile kernel is compiled for (register budget).
#ifndef PIC_TILE_MIN_BLOCKS_P2
#define PIC_TILE_MIN_BLOCKS_P2 3
#endif

template <int P>
__global__ void __launch_bounds__(kTileThreads, P == 1 ? 3 : (P == 2 ? PIC_TILE_MIN_BLOCKS_P2 : 2))
k_push_tile(const MixedArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_start[2][kSegs + 1];     // virtual start of each segment, per species
    __shared__ long long s_base[2][kSegs];     // physical first slot of each segment
    __shared__ int s_out[2][kSegs];            // next-buffer counts (stayers, outboxes)
    __shared__ int s_sent[2][kSegs + 1];       // particles sent to each segment; [0][kSegs]: moved
                                               // in by the overflow kernel
    __shared__ double s_red[32];
    __shared__ int s_item, s_pop;
    DevStatus* st = a.st;
    if (st->stop) return;
    const int par = (int)st->parity, nxp = par ^ 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (;;) {
        // every thread reads s_item between these two barriers; thread 0 writes it again
        // only after the barriers inside the tile body
        if (threadIdx.x == 0) s_item = atomicAdd(a.work, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.ntl) break;
        const int t = __ldg(a.tlist + item);  // global tile
        const int g = __ldg(a.tile_grid + t);
        const GridDev& G = a.grids[g];
        const int lt = t - G.tile_first;      // tile within its simulation
        const int tyi = lt / G.ntx, txi = lt - tyi * G.ntx;
        const int X0 = txi * G.tx, Y0 = tyi * G.ty;
        const int X1 = min(X0 + G.tx, G.nx), Y1 = min(Y0 + G.ty, G.ny);
        const int nx = G.nx, ny = G.ny;
        const int WX = G.wx, NW = G.wx * G.wy;
        const long long cap = G.cap, capo = G.capo, stride = bin_stride(G);
        int* jw = reinterpret_cast<int*>(smem_raw);  // [0, 3 NW) hi words, [3 NW, 6 NW) lo words
        float* fw = reinterpret_cast<float*>(smem_raw + (size_t)6 * NW * sizeof(int));
        if (threadIdx.x < 2 * kSegs) {
            const int s = threadIdx.x / kSegs, k = threadIdx.x - (threadIdx.x / kSegs) * kSegs;
            const int src = segment_source(G, txi, tyi, k);
            const long long off = k == 0 ? 0 : cap + (long long)(k - 1) * capo;
            const long long b = (long long)src * 2 + s;
            const int sent = segment_sent(G, par ? a.cnt[1] : a.cnt[0], src, s, k);
            s_sent[s][k] = sent;
            s_start[s][k + 1] = (int)min((long long)sent, k == 0 ? cap : capo);  // prefix-summed below
            s_base[s][k] = G.bin_off + b * stride + off;
            if (threadIdx.x == 0) {
                int* oin = par ? a.ovf_in[1] : a.ovf_in[0];
                s_sent[0][kSegs] = oin[t];
                oin[t] = 0;  // read; the overflow kernel of the next step counts into it again
            }
            s_out[s][k] = 0;
        }
        const float* Fg = a.F32 + G.cell_off;
        for (int idx = threadIdx.x; idx < 6 * NW; idx += blockDim.x) {
            const int c = idx / NW;
            const int w = idx - c * NW;
            const int wy = w / WX;
            const int wx = w - wy * WX;
            int gx = ((X0 - 2 + wx) % nx + nx) % nx, s = 1;
            if (G.walls) {  // conductor images: Ex, By, Bz even, Ey, Ez, Bx odd
                const bool half = c == 0 || c == 4 || c == 5;
                gx = wall_col(X0 - 2 + wx, nx, half, !half, s);
            }
            const int gy = ((Y0 - 2 + wy) % ny + ny) % ny;
            // (Ex, By) pairs, (Ey, Bx) pairs, Ez, Bz
            const int dst = c == 0 ? 2 * w : c == 4 ? 2 * w + 1 : c == 1 ? 2 * NW + 2 * w
                          : c == 3 ? 2 * NW + 2 * w + 1 : c == 2 ? 4 * NW + w : 5 * NW + w;
            fw[dst] = s == 0 ? 0.f : (float)s * Fg[c * a.ntot + (long long)gy * nx + gx];
        }
        for (int idx = threadIdx.x; idx < 6 * NW; idx += blockDim.x) jw[idx] = 0;
        __syncthreads();
        if (threadIdx.x < 2) {
            const int s = threadIdx.x;
            s_start[s][0] = 0;
            for (int k = 1; k <= kSegs; k++) s_start[s][k] += s_start[s][k - 1];
        } else if (threadIdx.x == 2) {  // the sum tile_population() forms
            int n = s_sent[0][kSegs];
            for (int s = 0; s < 2; s++)
                for (int k = 0; k < kSegs; k++) n += s_sent[s][k];
            s_pop = n;
        }
        __syncthreads();
        const FixedScale fs = fixed_scale(G, s_pop);
        const WinMem W{fw, jw, jw + 3 * NW, WX, NW, fs.js, fs.jlb};
        const GlobalMem M{a.F32 + G.cell_off, reinterpret_cast<unsigned long long*>(a.Jfix + G.cell_off),
                          a.ntot, nx, ny, fs, fs.js, G.walls};
        const unsigned* cur = par ? a.buf[1] : a.buf[0];
        unsigned* nxt = par ? a.buf[0] : a.buf[1];
        float ek = 0.f;
        for (int s = 0; s < 2; s++) {
            const PushConst K = push_const(G, s);
            const int total = s_start[s][kSegs];
            const long long own = G.bin_off + ((long long)lt * 2 + s) * stride;
            const int st1 = s_start[s][1];  // end of the stayer segment
            for (int c0 = warp * 32; c0 < total; c0 += nwarp * 32) {
                const int v = c0 + lane;
                const bool valid = v < total;
                int dest = -1, cnew = 0;
                float ox = 0.f, oy = 0.f, u[3] = {0.f, 0.f, 0.f};
                if (valid) {
                    // segment of slot v: the stayers, else one of the outboxes addressed here
                    int seg = 0;
                    if (v >= st1) {
                        seg = 1;
#pragma unroll
                        for (int k = 2; k < kSegs; k++) seg += (v >= s_start[s][k]) ? 1 : 0;
                    }
                    const long long e = s_base[s][seg] + (v - s_start[s][seg]);
                    int c;
                    get(cur, e, c, ox, oy, u);
                    const int ci = c & 0xffff, cj = c >> 16;
                    int di, dj;
                    bool ok;
                    if (ci >= X0 && ci < X1 && cj >= Y0 && cj < Y1)
                        ok = push_one<P>(W, K, ci - X0 + 2, cj - Y0 + 2, ox, oy, u, di, dj, ek);
                    else
                        ok = push_one<P>(M, K, ci, cj, ox, oy, u, di, dj, ek);
                    if (!ok) flag_bad(st, u);
                    const int ni = G.walls ? reflect_x(ci + di, nx, ox, u[0]) : wrapi(ci + di, nx);
                    const int nj = wrapi(cj + dj, ny);
                    cnew = ni | (nj << 16);
                    if (ni >= X0 && ni < X1 && nj >= Y0 && nj < Y1) {
                        dest = 0;
                    } else {
                        int dtx = ni / G.tx - txi, dty = nj / G.ty - tyi;
                        if (dtx > 1) dtx -= G.ntx;
                        if (dtx < -1) dtx += G.ntx;
                        if (dty > 1) dty -= G.nty;
                        if (dty < -1) dty += G.nty;
                        dest = (abs(dtx) <= 1 && abs(dty) <= 1 && (dtx | dty)) ? 1 + outbox_of(dtx, dty) : -1;
                    }
                }
                const unsigned act = __ballot_sync(0xffffffffu, valid);
                const unsigned stay = __ballot_sync(0xffffffffu, valid && dest == 0);
                if (valid) {
                    // lanes bound for the same bin (usually the whole warp stays in its tile)
                    const unsigned grp = stay == act ? act : __match_any_sync(act, dest);
                    const int leader = __ffs(grp) - 1;
                    const int rank = __popc(grp & ((1u << lane) - 1u));
                    int b0 = 0;
                    if (lane == leader && dest >= 0) b0 = atomicAdd(&s_out[s][dest], __popc(grp));
                    b0 = __shfl_sync(grp, b0, leader) + rank;
                    long long slot = -1;
                    if (dest == 0 && b0 < cap) slot = own + b0;
                    else if (dest > 0 && b0 < capo) slot = own + cap + (long long)(dest - 1) * capo + b0;
                    if (slot >= 0) {
                        put(nxt, slot, cnew, ox, oy, u);
                    } else {
                        to_overflow(nxp ? a.ovf[1].p : a.ovf[0].p, nxp ? a.ovf[1].gs : a.ovf[0].gs,
                                    a.ovf_cap, st, nxp, cnew, ox, oy, u[0], u[1], u[2], s | (g << 1));
                        if (dest < 0)  // sent to no bin: count it in its tile's population
                            atomicAdd((nxp ? a.ovf_in[1] : a.ovf_in[0]) + G.tile_first +
                                          tile_of(G, cnew & 0xffff, cnew >> 16), 1);
                    }
                }
            }
        }
        __syncthreads();
        if (threadIdx.x < 2 * kSegs) {
            const int s = threadIdx.x / kSegs, k = threadIdx.x - (threadIdx.x / kSegs) * kSegs;
            int* cnxt = nxp ? a.cnt[1] : a.cnt[0];
            cnxt[((long long)t * 2 + s) * kSegs + k] = s_out[s][k];  // sent, parked ones included
        }
        // add the current window into the global fixed-point current
        unsigned long long* Jg = reinterpret_cast<unsigned long long*>(a.Jfix + G.cell_off);
        for (int idx = threadIdx.x; idx < 3 * NW; idx += blockDim.x) {
            const int hi = jw[idx], lo = jw[3 * NW + idx];
            if ((hi | lo) == 0) continue;
            const unsigned long long v = (unsigned long long)fixed_value(hi, lo, fs);
            const int c = idx / NW;
            const int w = idx - c * NW;
            const int wy = w / WX;
            const int wx = w - wy * WX;
            int gx = ((X0 - 2 + wx) % nx + nx) % nx, s = 1;
            if (G.walls) gx = wall_col(X0 - 2 + wx, nx, c == 0, c == 0, s);  // mirror: Jx odd
            if (s == 0) continue;
            const int gy = ((Y0 - 2 + wy) % ny + ny) % ny;
            atomicAdd(Jg + c * a.ntot + (long long)gy * nx + gx, s > 0 ? v : 0ull - v);
        }
        const double sum = block_sum((double)ek, s_red);  // begins with a block barrier
        if (threadIdx.x == 0 && sum != 0.0) atomicAdd(&a.cg[g].uk, 0.5 * G.w * sum);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------
// 0. Overflow particles: global-memory push; they stay in the overflow list until the
// host re-sorts after the pic_step call.
// ---------------------------------------------------------------------------------
__global__ void k_mixed_begin(DevStatus* st, int* work) {
    if (threadIdx.x < 4) work[threadIdx.x] = 0;
    if (threadIdx.x == 0 && !st->stop) st->ovf_count[st->parity ^ 1u] = 0ull;
}

template <int P>
__device__ __forceinline__ bool push_global(const GridDev& G, const GlobalMem& M, int s, int ci, int cj,
                                            float& ox, float& oy, float u[3], int& di, int& dj,
                                            float& ek) {
    return push_one<P>(M, push_const(G, s), ci, cj, ox, oy, u, di, dj, ek);
}

__global__ void __launch_bounds__(kTileThreads)
k_push_overflow(const MixedArgs a) {
    DevStatus* st = a.st;
    if (st->stop) return;
    const int par = (int)st->parity;
    const long long n = min((long long)st->ovf_count[par], a.ovf_cap);
    const Slots O = par ? a.ovf[1] : a.ovf[0];
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        int c;
        float ox, oy, u[3];
        get(O.p, k, c, ox, oy, u);
        const int gs = O.gs[k];
        const int s = gs & 1, g = gs >> 1;
        const GridDev& G = a.grids[g];
        const int ci = c & 0xffff, cj = c >> 16;
        // round the current as the tile the particle's cell lies in rounds its window
        const FixedScale fs = fixed_scale(G, tile_population(G, par ? a.cnt[1] : a.cnt[0],
                                                             par ? a.ovf_in[1] : a.ovf_in[0], tile_of(G, ci, cj)));
        const GlobalMem M{a.F32 + G.cell_off, reinterpret_cast<unsigned long long*>(a.Jfix + G.cell_off),
                          a.ntot, G.nx, G.ny, fs, fs.js, G.walls};
        int di, dj;
        float ek = 0.f;
        bool ok;
        switch (G.order) {
        case 1: ok = push_global<1>(G, M, s, ci, cj, ox, oy, u, di, dj, ek); break;
        case 2: ok = push_global<2>(G, M, s, ci, cj, ox, oy, u, di, dj, ek); break;
        default: ok = push_global<3>(G, M, s, ci, cj, ox, oy, u, di, dj, ek); break;
        }
        if (!ok) flag_bad(st, u);
        if (ek != 0.f) atomicAdd(&a.cg[g].uk, 0.5 * G.w * (double)ek);
        const int ni = G.walls ? reflect_x(ci + di, G.nx, ox, u[0]) : wrapi(ci + di, G.nx);
        const int nj = wrapi(cj + dj, G.ny);
        const int cnew = ni | (nj << 16);
        to_overflow(par ? a.ovf[0].p : a.ovf[1].p, par ? a.ovf[0].gs : a.ovf[1].gs, a.ovf_cap, st,
                    par ^ 1, cnew, ox, oy, u[0], u[1], u[2], gs);
        atomicAdd((par ? a.ovf_in[0] : a.ovf_in[1]) + G.tile_first + tile_of(G, ni, nj), 1);
    }
}

// The injector's pairs of this step, straight into the next buffer: the stayer segment
// of the tile holding their cell (the tile kernels have finished with it), or the
// overflow list when it is full. One thread per (simulation, row, pair).
__global__ void k_inject_mixed(const MixedArgs a, const int* inj_grid, const long long* inj_first, int ngr,
                               unsigned long long* injected) {
    DevStatus* st = a.st;
    if (st->stop) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int q = 0;
    while (q + 1 < ngr && t >= inj_first[q + 1]) q++;
    if (t >= inj_first[ngr]) return;
    const int g = inj_grid[q];
    const GridDev& G = a.grids[g];
    const long long local = t - inj_first[q];
    const long long kmax = (long long)ceil(G.ppc * inj_width(G)) + 1;
    const int j = (int)(local / kmax);
    const long long k = local - (long long)j * kmax;
    const long long n = (long long)st->steps_done - 1;
    if (j >= G.ny || k >= inj_count(G, n)) return;
    double x, y;
    inj_position(G, n, j, k, x, y);
    int ci = (int)floor(x);
    float ox = (float)(x - ci);
    if (ox >= 1.f) {
        ox = 0.f;
        ci += 1;
    }
    if (ci < 0 || ci >= G.nx) return;  // (the plane starts at least two cells from the wall)
    const int cj = j;
    const float oy = (float)(y - cj);
    const int nxp = (int)st->parity ^ 1;
    unsigned* nxt = nxp ? a.buf[1] : a.buf[0];
    int* cnxt = nxp ? a.cnt[1] : a.cnt[0];
    const int lt = (cj / G.ty) * G.ntx + ci / G.tx;
    const long long stride = bin_stride(G);
    for (int s = 0; s < 2; s++) {
        double u[3];
        inj_momentum(G, n, j, k, s, u);
        const float uf[3] = {(float)u[0], (float)u[1], (float)u[2]};
        const int cell = ci | (cj << 16);
        const int slot = atomicAdd(&cnxt[((long long)(G.tile_first + lt) * 2 + s) * kSegs], 1);
        if (slot < G.cap)
            put(nxt, G.bin_off + ((long long)lt * 2 + s) * stride + slot, cell, ox, oy, uf);
        else
            to_overflow(nxp ? a.ovf[1].p : a.ovf[0].p, nxp ? a.ovf[1].gs : a.ovf[0].gs, a.ovf_cap, st, nxp,
                        cell, ox, oy, uf[0], uf[1], uf[2], s | (g << 1));
        atomicAdd(&injected[2 * g + s], 1ull);
    }
}

__global__ void k_mixed_swap(DevStatus* st) {
    if (threadIdx.x == 0 && !st->stop) st->parity ^= 1u;
}

// ---------------------------------------------------------------------------------
// Loading and re-sorting (one simulation at a time; tile indices are local to it)
// ---------------------------------------------------------------------------------
// FP64 physical particles -> staging (cell + FP32 offsets, FP32 momenta).
__global__ void k_stage_fp64(long long n, const double* x, const double* y, const double* ux,
                             const double* uy, const double* uz, GridDev G, PartArrays S,
                             unsigned long long* nbad) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double X = x[k], Y = y[k];
    const double a = ux[k], b = uy[k], c = uz[k];
    if (!isfinite(X) || !isfinite(Y) || !isfinite(a) || !isfinite(b) || !isfinite(c) ||
        (G.walls && !(X >= 0.0 && X < G.nx * G.dx))) {
        atomicAdd(nbad, 1ull);
        X = 0.0;
        Y = 0.0;
    }
    const double Lx = G.nx * G.dx, Ly = G.ny * G.dy;
    X = (X - floor(X / Lx) * Lx) * G.idx;
    Y = (Y - floor(Y / Ly) * Ly) * G.idy;
    int i = (int)floor(X), j = (int)floor(Y);
    float fx = (float)(X - i), fy = (float)(Y - j);
    if (fx >= 1.f) { fx = 0.f; i += 1; }
    if (fy >= 1.f) { fy = 0.f; j += 1; }
    i = ((i % G.nx) + G.nx) % G.nx;
    j = ((j % G.ny) + G.ny) % G.ny;
    S.cij[k] = i | (j << 16);
    S.ox[k] = fx;
    S.oy[k] = fy;
    S.ux[k] = (float)a;
    S.uy[k] = (float)b;
    S.uz[k] = (float)c;
}

// ---- the load / re-sort into tile bins (a counting sort, no library) ------------------
// A bin lists one particle of every cell of its tile, then a second of every cell, and
// so on, so that the 32 lanes of a warp work on 32 different cells: the particle of rank
// r in its cell (0, 1, ...) at cell cin of the tile goes to the slot that the key
// r * cells_per_tile + cin has among the tile's occupied keys. Keys are unique within a
// tile, so the slot is a prefix count over an occupancy bitmap of the tile's key range:
//   k_rank      rank within the cell (counter per cell), the tile and the key; tile
//               counts; the largest rank;
//   k_setbits   one bit per particle in its tile's bitmap;
//   k_scanbits  per tile, the exclusive prefix of the bitmap words' bit counts;
//   k_scatter   slot = prefix of the key's word + bits below the key within the word.
__global__ void k_rank(long long n, GridDev G, const int* cij, unsigned int* cellcnt, int* bincnt,
                       unsigned int* maxrank, unsigned int* key, int* tile) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = k < n;
    const int c = valid ? cij[k] : 0;
    const int i = c & 0xffff, j = c >> 16;
    const long long cell = (long long)j * G.nx + i;
    // warp-aggregated rank within the cell (neighbouring particles often share a cell)
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    if (!valid) return;
    const unsigned grp = __match_any_sync(act, cell);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(grp) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(&cellcnt[cell], (unsigned)__popc(grp));
    const unsigned rank = __shfl_sync(grp, base, leader) + __popc(grp & ((1u << lane) - 1u));
    const int t = (j / G.ty) * G.ntx + i / G.tx;
    const unsigned grpt = __match_any_sync(act, t);
    if (lane == __ffs(grpt) - 1) atomicAdd(&bincnt[t], __popc(grpt));
    const unsigned rmax = __reduce_max_sync(act, rank);
    if (lane == __ffs(act) - 1) atomicMax(maxrank, rmax);
    const unsigned cin = (unsigned)((j - (j / G.ty) * G.ty) * G.tx + (i - (i / G.tx) * G.tx));
    key[k] = rank * (unsigned)(G.tx * G.ty) + cin;
    tile[k] = t;
}

// words: bitmap words per tile; the bitmap holds tiles t0 .. t0 + ntg - 1
__global__ void k_setbits(long long n, const unsigned int* key, const int* tile, int t0, int ntg, long long words,
                          unsigned int* bits) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int t = tile[k] - t0;
    if (t < 0 || t >= ntg) return;
    const unsigned q = key[k];
    atomicOr(bits + (long long)t * words + (q >> 5), 1u << (q & 31));
}

// One block per tile: pref[w] = bits set in words 0 .. w-1 of the tile's bitmap.
__global__ void __launch_bounds__(256) k_scanbits(long long words, const unsigned int* bits, unsigned int* pref) {
    __shared__ unsigned int s_warp[8];
    __shared__ unsigned int s_carry;
    const unsigned int* b = bits + (long long)blockIdx.x * words;
    unsigned int* o = pref + (long long)blockIdx.x * words;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (long long w0 = 0; w0 < words; w0 += blockDim.x) {
        const long long w = w0 + threadIdx.x;
        const unsigned v = w < words ? (unsigned)__popc(b[w]) : 0u;
        unsigned x = v;  // inclusive scan within the warp
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        unsigned before = s_carry;
        for (int q = 0; q < warp; q++) before += s_warp[q];
        if (w < words) o[w] = before + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = before + x;
        __syncthreads();
    }
}

__global__ void k_scatter(long long n, GridDev G, int s, const unsigned int* key, const int* tile, int t0,
                          int ntg, long long words, const unsigned int* bits, const unsigned int* pref,
                          PartArrays S, unsigned* B) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int t = tile[p];
    if (t < t0 || t >= t0 + ntg) return;
    const unsigned q = key[p];
    const long long wq = (long long)(t - t0) * words + (q >> 5);
    const long long r = (long long)pref[wq] + __popc(bits[wq] & ((1u << (q & 31)) - 1u));
    const long long dst = G.bin_off + ((long long)t * 2 + s) * bin_stride(G) + r;
    const float u[3] = {S.ux[p], S.uy[p], S.uz[p]};
    put(B, dst, S.cij[p], S.ox[p], S.oy[p], u);
}

// cnt points at the simulation's first count slot.
__global__ void k_set_counts(int ntiles, int s, const int* bincnt, int* cnt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    int* c = cnt + ((long long)t * 2 + s) * kSegs;
    c[0] = bincnt[t];
    for (int k = 1; k < kSegs; k++) c[k] = 0;
}

// Copy every segment of species s's bins (offsets from a host prefix sum, one entry per
// (tile, segment)) into staging form.
__device__ __forceinline__ void to_staging(const unsigned* P, long long k, PartArrays S, long long d) {
    int c;
    float ox, oy, u[3];
    get(P, k, c, ox, oy, u);
    S.cij[d] = c;
    S.ox[d] = ox;
    S.oy[d] = oy;
    S.ux[d] = u[0];
    S.uy[d] = u[1];
    S.uz[d] = u[2];
}

__global__ void k_gather_bins(GridDev G, int s, const int* cnt, const long long* off, const unsigned* B,
                              PartArrays S) {
    const int t = blockIdx.x / kSegs, k = blockIdx.x - (blockIdx.x / kSegs) * kSegs;
    const long long b = (long long)t * 2 + s;
    const long long lim = k == 0 ? G.cap : G.capo;
    const int n = (int)min((long long)cnt[b * kSegs + k], lim);
    const long long src0 = G.bin_off + b * bin_stride(G) + (k == 0 ? 0 : G.cap + (long long)(k - 1) * G.capo);
    const long long dst0 = off[blockIdx.x];
    for (int q = threadIdx.x; q < n; q += blockDim.x) to_staging(B, src0 + q, S, dst0 + q);
}

// Overflow-list entries with code gs (species | simulation << 1) appended after `base`.
__global__ void k_gather_overflow(long long n_over, int gs, Slots O, long long base,
                                  unsigned long long* cursor, PartArrays S) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_over || O.gs[k] != gs) return;
    const long long d = base + (long long)atomicAdd(cursor, 1ull);
    to_staging(O.p, k, S, d);
}

template <int P>
__global__ void k_rho_staged(long long n, GridDev G, PartArrays S, double q, double* rho) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int c = S.cij[k];
    deposit_rho<P>(G, c & 0xffff, (double)S.ox[k], c >> 16, (double)S.oy[k], q, rho);
}

__global__ void k_momentum_staged(long long n, PartArrays S, double w, double* out) {
    __shared__ double red[32];
    double s[3] = {0.0, 0.0, 0.0};
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        s[0] += S.ux[k];
        s[1] += S.uy[k];
        s[2] += S.uz[k];
    }
    for (int c = 0; c < 3; c++) {
        const double t = block_sum(s[c], red);
        if (threadIdx.x == 0) atomicAdd(out + c, w * t);
        __syncthreads();
    }
}

__global__ void k_unstage(long long n, GridDev G, PartArrays S, double* out) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int c = S.cij[k];
    out[k] = ((double)(c & 0xffff) + (double)S.ox[k]) * G.dx;
    out[n + k] = ((double)(c >> 16) + (double)S.oy[k]) * G.dy;
    out[2 * n + k] = S.ux[k];
    out[3 * n + k] = S.uy[k];
    out[4 * n + k] = S.uz[k];
}

// ---- host helpers -------------------------------------------------------------------

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
    *p = nullptr;
    return cudaMalloc((void**)p, (n ? n : 1) * sizeof(T));
}

// Temporaries of loads, re-sorts and diagnostics (staging arrays, sort keys, bitmaps)
// come from a library-owned stream-ordered memory pool that keeps its memory for the
// next call (release threshold: never), so that a load or a re-sort does not map and
// unmap gigabytes of device memory each time (cudaMalloc / cudaFree of that size cost
// from tens to hundreds of ms, depending on the device's history).
cudaMemPool_t temp_pool(cudaError_t* e) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    *e = cudaGetDevice(&dev);
    if (*e != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= 64) {
        *e = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
        cudaMemPoolProps pp{};
        pp.allocType = cudaMemAllocationTypePinned;
        pp.location.type = cudaMemLocationTypeDevice;
        pp.location.id = dev;
        *e = cudaMemPoolCreate(&pools[dev], &pp);
        if (*e != cudaSuccess) {
            pools[dev] = nullptr;
            return nullptr;
        }
        unsigned long long keep = ~0ull;  // the attribute is a 64-bit unsigned
        *e = cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        if (*e != cudaSuccess) return nullptr;
    }
    return pools[dev];
}

template <typename T>
cudaError_t talloc(T** p, size_t n, cudaStream_t st) {
    *p = nullptr;
    cudaError_t e = cudaSuccess;
    cudaMemPool_t pool = temp_pool(&e);
    if (!pool) return e == cudaSuccess ? cudaErrorMemoryAllocation : e;
    return cudaMallocFromPoolAsync(reinterpret_cast<void**>(p), (n ? n : 1) * sizeof(T), pool, st);
}

void tfree(void* p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

void free_parts(PartArrays& A, cudaStream_t st) {
    void* ps[] = {A.cij, A.ox, A.oy, A.ux, A.uy, A.uz, A.gs};
    for (void* p : ps) tfree(p, st);
    A = PartArrays{};
}

cudaError_t alloc_parts(PartArrays& A, size_t n, bool with_gs, cudaStream_t st) {
    A = PartArrays{};
    cudaError_t e = talloc(&A.cij, n, st);
    if (e == cudaSuccess) e = talloc(&A.ox, n, st);
    if (e == cudaSuccess) e = talloc(&A.oy, n, st);
    if (e == cudaSuccess) e = talloc(&A.ux, n, st);
    if (e == cudaSuccess) e = talloc(&A.uy, n, st);
    if (e == cudaSuccess) e = talloc(&A.uz, n, st);
    if (e == cudaSuccess && with_gs) e = talloc(&A.gs, n, st);
    if (e != cudaSuccess) free_parts(A, st);
    return e;
}

// Staged particles of every (simulation, species), index 2 g + s.
struct Staged {
    std::vector<PartArrays> S;
    std::vector<long long> n;
    cudaStream_t st;
    Staged(int ngrids, cudaStream_t stream) : S(2 * ngrids), n(2 * ngrids, 0), st(stream) {}
    ~Staged() {
        for (PartArrays& a : S) free_parts(a, st);
    }
};

MixedArgs make_args(MixedState* m, int order) {
    MixedArgs a{};
    a.grids = m->dgrids;
    a.tile_grid = m->tile_grid;
    a.tlist = m->tlist + m->order_first[order];
    a.ntl = m->order_n[order];
    a.work = m->work + order;
    a.ntot = m->ntot;
    a.F32 = m->F32;
    a.Jfix = m->Jfix;
    for (int p = 0; p < 2; p++) {
        a.buf[p] = m->buf[p];
        a.cnt[p] = m->cnt[p];
        a.ovf_in[p] = m->ovf_in[p];
        a.ovf[p] = m->ovf[p];
    }
    a.ovf_cap = m->ovf_cap;
    a.cg = m->cg;
    a.st = m->st;
    return a;
}

unsigned grid1(long long n, int b = 256) { return (unsigned)std::max<long long>(1, (n + b - 1) / b); }

#define MCK(call)                                                                     \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            err = std::string(#call) + " failed: " + cudaGetErrorString(e_);          \
            return PIC_ECUDA;                                                         \
        }                                                                             \
    } while (0)

int read_status(MixedState* m, DevStatus& hs, cudaStream_t st, std::string& err) {
    MCK(cudaMemcpyAsync(&hs, m->st, sizeof hs, cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    return PIC_OK;
}

long long round32(double c) { return ((long long)std::ceil(c) + 31) / 32 * 32; }

int* cnt_of(MixedState* m, int par, int g) {
    return m->cnt[par] + (long long)m->G[g].tile_first * 2 * kSegs;
}

// Sort n staged particles of species s of simulation g into the stayer segments of
// buffer `par`. Returns PIC_ENOMEM (nothing written) when a bin would overflow, with
// the fullest bin's count in *need.
int sort_into_bins(MixedState* m, int g, int par, int s, PartArrays S, long long n, cudaStream_t st,
                   long long* need, std::string& err) {
    const GridDev& G = m->G[g];
    const int ntiles = G.ntiles;
    unsigned int* cellcnt = nullptr;
    int* bincnt = nullptr;
    unsigned int* maxrank = nullptr;
    unsigned int *key = nullptr, *bits = nullptr, *pref = nullptr;
    int* tile = nullptr;
    int rc = PIC_OK;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    A(talloc(&cellcnt, (size_t)G.ncell, st));
    A(talloc(&bincnt, (size_t)ntiles, st));
    A(talloc(&maxrank, 1, st));
    A(talloc(&key, (size_t)n, st));
    A(talloc(&tile, (size_t)n, st));
    if (e == cudaSuccess) {
        A(cudaMemsetAsync(cellcnt, 0, G.ncell * sizeof(unsigned), st));
        A(cudaMemsetAsync(bincnt, 0, ntiles * sizeof(int), st));
        A(cudaMemsetAsync(maxrank, 0, sizeof(unsigned), st));
        if (n) k_rank<<<grid1(n), 256, 0, st>>>(n, G, S.cij, cellcnt, bincnt, maxrank, key, tile);
        A(cudaGetLastError());
    }
    std::vector<int> hcnt(ntiles);
    unsigned int hmax = 0;
    if (e == cudaSuccess) {
        A(cudaMemcpyAsync(hcnt.data(), bincnt, ntiles * sizeof(int), cudaMemcpyDeviceToHost, st));
        A(cudaMemcpyAsync(&hmax, maxrank, sizeof hmax, cudaMemcpyDeviceToHost, st));
        A(cudaStreamSynchronize(st));
    }
    if (e == cudaSuccess) {
        long long mx = 0;
        for (int t = 0; t < ntiles; t++) mx = std::max<long long>(mx, hcnt[t]);
        if (need) *need = mx;
        const long long cpt = (long long)G.tx * G.ty;
        if (mx > G.cap) {
            rc = PIC_ENOMEM;  // caller grows the bins and retries
        } else if ((long long)hmax + 1 > (long long)(0xffffffffu / cpt)) {
            err = "a cell holds too many particles of one species for the bin keys";
            rc = PIC_EINVAL;  // (not PIC_ENOMEM: larger bins would not help)
        } else {
            // a tile's keys are rank * cells + cell: ranks 0 .. hmax. Tiles go in groups
            // whose bitmaps fit a fixed budget (one group unless cells are very uneven).
            const long long words = ((long long)(hmax + 1) * cpt + 31) / 32;
            const long long budget = 64ll << 20;  // bitmap words per group (256 MB)
            const int group = (int)std::max(1ll, std::min<long long>(ntiles, budget / words));
            A(talloc(&bits, (size_t)group * words, st));
            A(talloc(&pref, (size_t)group * words, st));
            for (int t0 = 0; t0 < ntiles && e == cudaSuccess; t0 += group) {
                const int ntg = std::min(group, ntiles - t0);
                A(cudaMemsetAsync(bits, 0, (size_t)ntg * words * sizeof(unsigned), st));
                if (n) k_setbits<<<grid1(n), 256, 0, st>>>(n, key, tile, t0, ntg, words, bits);
                k_scanbits<<<(unsigned)ntg, 256, 0, st>>>(words, bits, pref);
                if (n)
                    k_scatter<<<grid1(n), 256, 0, st>>>(n, G, s, key, tile, t0, ntg, words, bits, pref, S,
                                                        m->buf[par]);
                A(cudaGetLastError());
            }
            if (e == cudaSuccess) {
                k_set_counts<<<grid1(ntiles), 256, 0, st>>>(ntiles, s, bincnt, cnt_of(m, par, g));
                A(cudaGetLastError());
                A(cudaStreamSynchronize(st));
            }
        }
    }
    void* ps[] = {cellcnt, bincnt, maxrank, key, tile, bits, pref};
    for (void* p : ps) tfree(p, st);
    if (e != cudaSuccess) {
        err = std::string("bin sort failed: ") + cudaGetErrorString(e);
        return PIC_ECUDA;
    }
    return rc;
}

// All live particles of species s of simulation g (every bin segment of buffer `par` +
// its overflow-list entries) into a new staging set.
int gather_species(MixedState* m, int g, int par, int s, PartArrays& S, long long& n, cudaStream_t st,
                   std::string& err) {
    const GridDev& G = m->G[g];
    const long long nb_seg = (long long)G.ntiles * kSegs;
    std::vector<int> cnt(2 * nb_seg);
    MCK(cudaMemcpyAsync(cnt.data(), cnt_of(m, par, g), cnt.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
    DevStatus hs{};
    MCK(cudaMemcpyAsync(&hs, m->st, sizeof hs, cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    std::vector<long long> off(nb_seg + 1, 0);
    for (int t = 0; t < G.ntiles; t++)
        for (int k = 0; k < kSegs; k++) {
            const long long lim = k == 0 ? G.cap : G.capo;
            const long long q = (long long)t * kSegs + k;
            off[q + 1] = off[q] + std::min<long long>(cnt[((long long)t * 2 + s) * kSegs + k], lim);
        }
    const long long nb = off[nb_seg];
    const long long no = std::min<long long>((long long)hs.ovf_count[par], m->ovf_cap);
    MCK(alloc_parts(S, (size_t)(nb + no), false, st));
    long long* doff = nullptr;
    unsigned long long* cursor = nullptr;
    MCK(talloc(&doff, off.size(), st));
    MCK(talloc(&cursor, 1, st));
    MCK(cudaMemcpyAsync(doff, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice, st));
    MCK(cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), st));
    k_gather_bins<<<(unsigned)nb_seg, 256, 0, st>>>(G, s, cnt_of(m, par, g), doff, m->buf[par], S);
    if (no) k_gather_overflow<<<grid1(no), 256, 0, st>>>(no, s | (g << 1), m->ovf[par], nb, cursor, S);
    unsigned long long hcur = 0;
    MCK(cudaMemcpyAsync(&hcur, cursor, sizeof hcur, cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    tfree(doff, st);
    tfree(cursor, st);
    n = nb + (long long)hcur;
    return PIC_OK;
}

// (Re)allocate both bin buffers with per-simulation stayer capacity cap[g] and outbox
// capacity capo[g] (contents are not preserved; all counts are zeroed).
int alloc_bins(MixedState* m, const std::vector<long long>& cap, const std::vector<long long>& capo,
               cudaStream_t st, std::string& err) {
    for (int p = 0; p < 2; p++) {
        if (m->buf[p]) cudaFree(m->buf[p]);
        m->buf[p] = nullptr;
    }
    m->gen++;
    long long off = 0;
    for (int g = 0; g < m->ngrids; g++) {
        GridDev& G = m->G[g];
        G.cap = cap[g];
        G.capo = capo[g];
        G.bin_off = off;
        off += (long long)G.ntiles * 2 * bin_stride(G);
    }
    m->nslots = off;
    for (int p = 0; p < 2; p++) {
        cudaError_t e = dalloc(&m->buf[p], (size_t)m->nslots * kFields);
        if (e != cudaSuccess) {
            cudaGetLastError();
            err = "bin allocation failed (" + std::to_string(m->nslots) + " slots per buffer)";
            return PIC_ENOMEM;
        }
        MCK(cudaMemsetAsync(m->cnt[p], 0, (size_t)m->ntiles_total * (2 * kSegs + 1) * sizeof(int), st));
    }
    return PIC_OK;
}

// Gather every simulation's particles of buffer `par` into staging.
int gather_all(MixedState* m, int par, Staged& A, cudaStream_t st, std::string& err) {
    for (int g = 0; g < m->ngrids; g++)
        for (int s = 0; s < 2; s++)
            if (int rc = gather_species(m, g, par, s, A.S[2 * g + s], A.n[2 * g + s], st, err)) return rc;
    return PIC_OK;
}

// Allocate bins of at least the given capacities and sort everything staged in A into
// buffer `par`, growing a simulation's stayer capacity whenever one of its bins would
// overflow. Uploads the descriptors and clears the overflow lists.
int place_all(MixedState* m, int par, Staged& A, std::vector<long long> cap, std::vector<long long> capo,
              cudaStream_t st, std::string& err) {
    int rc = PIC_OK;
    for (int attempt = 0; attempt < 8; attempt++) {
        rc = alloc_bins(m, cap, capo, st, err);
        if (rc) return rc;
        bool grown = false;
        for (int g = 0; g < m->ngrids && rc == PIC_OK; g++)
            for (int s = 0; s < 2 && rc == PIC_OK; s++) {
                long long need = 0;
                rc = sort_into_bins(m, g, par, s, A.S[2 * g + s], A.n[2 * g + s], st, &need, err);
                if (rc == PIC_ENOMEM) {
                    cap[g] = std::max(cap[g] * 3 / 2 + 32, round32(1.25 * (double)need + 32.0));
                    grown = true;
                }
            }
        if (!grown) break;
        rc = PIC_ENOMEM;
    }
    if (rc) return rc;
    MCK(cudaMemcpyAsync((void*)m->dgrids, m->G, m->ngrids * sizeof(GridDev), cudaMemcpyHostToDevice, st));
    MCK(cudaMemsetAsync(&m->st->ovf_count, 0, sizeof(DevStatus::ovf_count), st));
    // the counts now come from the bins themselves, injected pairs included
    MCK(cudaMemsetAsync(m->injected, 0, 2 * m->ngrids * sizeof(unsigned long long), st));
    MCK(cudaStreamSynchronize(st));
    for (int q = 0; q < 2 * m->ngrids; q++) m->n[q] = A.n[q];
    return PIC_OK;
}

// Re-sort every simulation into fresh bins with capacities at least (cap_min, capo_min).
int rebuild(MixedState* m, std::vector<long long> cap_min, std::vector<long long> capo_min,
            cudaStream_t st, std::string& err) {
    DevStatus hs{};
    if (int rc = read_status(m, hs, st, err)) return rc;
    const int par = (int)hs.parity;
    Staged A(m->ngrids, st);
    if (int rc = gather_all(m, par, A, st, err)) return rc;
    for (int g = 0; g < m->ngrids; g++) {
        cap_min[g] = std::max(cap_min[g], m->G[g].cap);
        capo_min[g] = std::max(capo_min[g], m->G[g].capo);
    }
    if (int rc = place_all(m, par, A, cap_min, capo_min, st, err)) return rc;
    m->rebins++;
    return PIC_OK;
}

std::vector<long long> current_caps(MixedState* m, bool outboxes) {
    std::vector<long long> v(m->ngrids);
    for (int g = 0; g < m->ngrids; g++) v[g] = outboxes ? m->G[g].capo : m->G[g].cap;
    return v;
}

}  // namespace

// =====================================================================================

int mixed_create(MixedState** out, const pic_params* p, int ngrids, GridDev* G,
                 const GridDev* dgrids, long long ntot, float* F32, long long* Jfix, CgState* cg,
                 DevStatus* st, std::string& err) {
    *out = nullptr;
    MixedState* m = new MixedState();
    m->ngrids = ngrids;
    m->G = G;
    m->dgrids = dgrids;
    m->ntot = ntot;
    m->F32 = F32;
    m->Jfix = Jfix;
    m->cg = cg;
    m->st = st;
    m->n.assign(2 * ngrids, 0);
    // tiles of every simulation, one global numbering
    int ntiles = 0;
    long long expect = 0;
    std::vector<long long> cap(ngrids), capo(ngrids);
    for (int g = 0; g < ngrids; g++) {
        const pic_params& q = p[g];
        GridDev& D = G[g];
        int tx = q.tile_x, ty = q.tile_y;
        if (tx <= 0) tx = std::min(32, q.nx);
        if (ty <= 0) ty = std::min(16, q.ny);
        D.tx = std::min(tx, q.nx);
        D.ty = std::min(ty, q.ny);
        D.ntx = (q.nx + D.tx - 1) / D.tx;
        D.nty = (q.ny + D.ty - 1) / D.ty;
        D.ntiles = D.ntx * D.nty;
        D.tile_first = ntiles;
        ntiles += D.ntiles;
        D.wx = D.tx + 5;
        D.wy = D.ty + 5;
        const size_t sm = (size_t)6 * D.wx * D.wy * sizeof(int) + (size_t)6 * D.wx * D.wy * sizeof(float);
        m->smem[D.order] = std::max(m->smem[D.order], sm);
        const double slack = q.bin_slack > 0 ? q.bin_slack : 1.25;
        cap[g] = round32((double)q.ppc * D.tx * D.ty * slack + 64.0);
        capo[g] = round32((double)q.ppc * std::max(D.tx, D.ty) * 1.5 + 32.0);
        expect += 2ll * q.ppc * (long long)q.nx * q.ny;
    }
    m->ntiles_total = ntiles;
    // per-order tile lists, largest expected work first
    std::vector<int> tg(ntiles), tl;
    std::vector<std::pair<long long, int>> order_tiles[4];
    for (int g = 0; g < ngrids; g++) {
        const GridDev& D = G[g];
        for (int t = 0; t < D.ntiles; t++) {
            tg[D.tile_first + t] = g;
            const int tyi = t / D.ntx, txi = t - tyi * D.ntx;
            const long long cells = (long long)(std::min(D.tx, D.nx - txi * D.tx)) *
                                    std::min(D.ty, D.ny - tyi * D.ty);
            order_tiles[D.order].push_back({cells * p[g].ppc, D.tile_first + t});
        }
    }
    for (int P = 1; P <= 3; P++) {
        std::stable_sort(order_tiles[P].begin(), order_tiles[P].end(),
                         [](const std::pair<long long, int>& x, const std::pair<long long, int>& y) {
                             return x.first > y.first;
                         });
        m->order_first[P] = (int)tl.size();
        m->order_n[P] = (int)order_tiles[P].size();
        for (auto& e : order_tiles[P]) tl.push_back(e.second);
    }
    m->ovf_cap = std::max<long long>(65536, expect / 8);
    m->ovf_cap = (m->ovf_cap + 31) / 32 * 32;
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < 2 && e == cudaSuccess; q++) {
        e = dalloc(&m->cnt[q], (size_t)ntiles * (2 * kSegs + 1));
        if (e == cudaSuccess) m->ovf_in[q] = m->cnt[q] + (size_t)ntiles * 2 * kSegs;
        if (e == cudaSuccess) e = dalloc(&m->ovf[q].p, (size_t)m->ovf_cap * kFields);
        if (e == cudaSuccess) e = dalloc(&m->ovf[q].gs, (size_t)m->ovf_cap);
    }
    // injector tables
    {
        std::vector<int> ig;
        std::vector<long long> first(1, 0);
        for (int g = 0; g < ngrids; g++) {
            if (!G[g].inject) continue;
            const double w = (1.0 + std::sqrt(1.0 - 1.0 / (G[g].gamma0 * G[g].gamma0))) * G[g].cfl;
            const long long kmax = (long long)std::ceil(G[g].ppc * w) + 1;
            ig.push_back(g);
            first.push_back(first.back() + (long long)G[g].ny * kmax);
        }
        m->inject_grids = (int)ig.size();
        m->inject_threads = first.back();
        if (e == cudaSuccess) e = dalloc(&m->injected, (size_t)2 * ngrids);
        if (e == cudaSuccess) e = cudaMemset(m->injected, 0, 2 * ngrids * sizeof(unsigned long long));
        if (e == cudaSuccess && !ig.empty()) {
            e = dalloc(&m->inj_grid, ig.size());
            if (e == cudaSuccess) e = dalloc(&m->inj_first, first.size());
            if (e == cudaSuccess) e = cudaMemcpy(m->inj_grid, ig.data(), ig.size() * sizeof(int), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(m->inj_first, first.data(), first.size() * sizeof(long long), cudaMemcpyHostToDevice);
        }
    }
    if (e == cudaSuccess) e = dalloc(&m->tile_grid, (size_t)ntiles);
    if (e == cudaSuccess) e = dalloc(&m->tlist, (size_t)ntiles);
    if (e == cudaSuccess) e = dalloc(&m->work, 4);
    if (e == cudaSuccess) e = cudaMemcpy(m->tile_grid, tg.data(), ntiles * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->tlist, tl.data(), ntiles * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->work, 0, 4 * sizeof(int));
    int rc = PIC_OK;
    if (e == cudaSuccess) {
        rc = alloc_bins(m, cap, capo, 0, err);
        if (rc == PIC_OK) e = cudaDeviceSynchronize();
    }
    // Shared-memory opt-in: only ever raised, since the attribute belongs to the kernel
    // and other handles in the process may need more than this one.
    int dev = 0, nsm = 152;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    auto setup = [&](auto kern, int P) {
        if (m->order_n[P] == 0) return cudaSuccess;
        cudaFuncAttributes fa{};
        cudaError_t r = cudaFuncGetAttributes(&fa, kern);
        if (r == cudaSuccess && (size_t)fa.maxDynamicSharedSizeBytes < m->smem[P])
            r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m->smem[P]);
        int nb = 0;
        if (r == cudaSuccess)
            r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kTileThreads, m->smem[P]);
        if (r == cudaSuccess && nb < 1) r = cudaErrorInvalidConfiguration;
        m->pblocks[P] = std::min(m->order_n[P], nb * nsm);
        return r;
    };
    if (rc == PIC_OK && e == cudaSuccess) e = setup(k_push_tile<1>, 1);
    if (rc == PIC_OK && e == cudaSuccess) e = setup(k_push_tile<2>, 2);
    if (rc == PIC_OK && e == cudaSuccess) e = setup(k_push_tile<3>, 3);
    if (rc == PIC_OK && e == cudaSuccess) {
        e = cudaMemcpy((void*)dgrids, G, ngrids * sizeof(GridDev), cudaMemcpyHostToDevice);
    }
    if (rc == PIC_OK && e != cudaSuccess) {
        err = std::string("MIXED32 setup failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        rc = PIC_ENOMEM;
    }
    if (rc != PIC_OK) {
        mixed_destroy(m);
        return rc;
    }
    *out = m;
    return PIC_OK;
}

void mixed_destroy(MixedState* m) {
    if (!m) return;
    for (int p = 0; p < 2; p++) {
        void* ps[] = {m->buf[p], m->ovf[p].p, m->ovf[p].gs, m->cnt[p]};
        for (void* q : ps)
            if (q) cudaFree(q);
    }
    void* ps[] = {m->tile_grid, m->tlist, m->work, m->injected, m->inj_grid, m->inj_first};
    for (void* q : ps)
        if (q) cudaFree(q);
    delete m;
}

int mixed_load(MixedState* m, int g, int s, const double* x, const double* y, const double* ux,
               const double* uy, const double* uz, long long n, cudaStream_t st, std::string& err) {
    DevStatus hs{};
    if (int rc = read_status(m, hs, st, err)) return rc;
    // fold any overflow-list particles back into bins first so the list holds none of s
    if (hs.ovf_count[hs.parity]) {
        int rc = rebuild(m, current_caps(m, false), current_caps(m, true), st, err);
        if (rc) return rc;
    }
    const int par = (int)hs.parity;
    double* in = nullptr;
    PartArrays S{};
    unsigned long long* nbad = nullptr;
    MCK(talloc(&in, 5 * (size_t)std::max<long long>(n, 1), st));
    const double* src[5] = {x, y, ux, uy, uz};
    for (int a = 0; a < 5 && n; a++)
        MCK(cudaMemcpyAsync(in + a * n, src[a], n * sizeof(double), cudaMemcpyDefault, st));
    MCK(alloc_parts(S, (size_t)n, false, st));
    MCK(talloc(&nbad, 1, st));
    MCK(cudaMemsetAsync(nbad, 0, sizeof(unsigned long long), st));
    if (n)
        k_stage_fp64<<<grid1(n), 256, 0, st>>>(n, in, in + n, in + 2 * n, in + 3 * n, in + 4 * n, m->G[g],
                                               S, nbad);
    unsigned long long hbad = 0;
    MCK(cudaMemcpyAsync(&hbad, nbad, sizeof hbad, cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    tfree(in, st);
    tfree(nbad, st);
    if (hbad) {
        free_parts(S, st);
        err = "non-finite particle position or momentum, or a position outside the walls";
        return PIC_EINVAL;
    }
    long long need = 0;
    int rc = sort_into_bins(m, g, par, s, S, n, st, &need, err);  // also zeroes s's outbox counts
    if (rc == PIC_ENOMEM) {
        // a bin would overflow: re-sort everything with larger bins for this simulation
        Staged A(m->ngrids, st);
        rc = gather_all(m, par, A, st, err);
        if (rc == PIC_OK) {
            free_parts(A.S[2 * g + s], st);
            A.S[2 * g + s] = S;
            A.n[2 * g + s] = n;
            S = PartArrays{};
            std::vector<long long> cap = current_caps(m, false);
            cap[g] = std::max(cap[g], round32(1.25 * (double)need + 32.0));
            rc = place_all(m, par, A, cap, current_caps(m, true), st, err);
            m->rebins++;
        }
    } else if (rc == PIC_OK) {
        MCK(cudaMemcpyAsync((void*)(m->dgrids + g), m->G + g, sizeof(GridDev), cudaMemcpyHostToDevice, st));
        MCK(cudaStreamSynchronize(st));
        m->n[2 * g + s] = n;
    }
    free_parts(S, st);
    return rc;
}

void mixed_enqueue(MixedState* m, cudaStream_t st, int part) {
    if (part == 0) {
        k_mixed_begin<<<1, 32, 0, st>>>(m->st, m->work);
        k_push_overflow<<<152, kTileThreads, 0, st>>>(make_args(m, 0));
    } else if (part == 1) {
        for (int P = 1; P <= 3; P++) {
            if (m->order_n[P] == 0) continue;
            const MixedArgs a = make_args(m, P);
            const unsigned nb = (unsigned)m->pblocks[P];
            switch (P) {
            case 1: k_push_tile<1><<<nb, kTileThreads, m->smem[1], st>>>(a); break;
            case 2: k_push_tile<2><<<nb, kTileThreads, m->smem[2], st>>>(a); break;
            default: k_push_tile<3><<<nb, kTileThreads, m->smem[3], st>>>(a); break;
            }
        }
    } else {
        if (m->inject_grids)
            k_inject_mixed<<<(unsigned)((m->inject_threads + 255) / 256), 256, 0, st>>>(
                make_args(m, 0), m->inj_grid, m->inj_first, m->inject_grids, m->injected);
        k_mixed_swap<<<1, 32, 0, st>>>(m->st);
    }
}

int mixed_before_steps(MixedState*, cudaStream_t, std::string&) { return PIC_OK; }

int mixed_step_kernels(const MixedState* m) {
    int k = 3;  // k_mixed_begin, k_push_overflow, k_mixed_swap
    for (int P = 1; P <= 3; P++) k += m->order_n[P] > 0 ? 1 : 0;
    return k + (m->inject_grids ? 1 : 0);
}

int mixed_after_steps(MixedState* m, cudaStream_t st, std::string& err) {
    DevStatus hs{};
    if (int rc = read_status(m, hs, st, err)) return rc;
    if (m->inject_grids) {  // the injector's pairs join the live counts
        std::vector<unsigned long long> add((size_t)2 * m->ngrids);
        MCK(cudaMemcpyAsync(add.data(), m->injected, add.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        MCK(cudaMemsetAsync(m->injected, 0, add.size() * sizeof(unsigned long long), st));
        MCK(cudaStreamSynchronize(st));
        for (size_t q = 0; q < add.size(); q++) m->n[q] += (long long)add[q];
    }
    const int par = (int)hs.parity;
    if (hs.ovf_count[par] == 0) return PIC_OK;
    // particles are parked in the overflow list: re-sort with room to spare. Grow each
    // simulation's stayer capacity to 1.25x its fullest tile and double its outboxes if
    // any is full.
    std::vector<int> cnt((size_t)m->ntiles_total * 2 * kSegs);
    MCK(cudaMemcpyAsync(cnt.data(), m->cnt[par], cnt.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    std::vector<long long> cap(m->ngrids), capo(m->ngrids);
    const long long excess = (long long)hs.ovf_count[par];  // upper bound on any tile's excess
    for (int g = 0; g < m->ngrids; g++) {
        const GridDev& G = m->G[g];
        long long mx = 0;
        bool outbox_full = false;
        for (long long b = (long long)G.tile_first * 2; b < (long long)(G.tile_first + G.ntiles) * 2; b++) {
            long long tot = 0;
            for (int k = 0; k < kSegs; k++) {
                tot += cnt[b * kSegs + k];
                if (k > 0 && cnt[b * kSegs + k] >= G.capo) outbox_full = true;
            }
            mx = std::max(mx, tot);
        }
        cap[g] = std::max(round32(1.25 * (double)std::min(mx + excess, 2 * mx + 64)), G.cap);
        capo[g] = outbox_full ? 2 * G.capo : G.capo;
    }
    return rebuild(m, cap, capo, st, err);
}

long long mixed_count(MixedState* m, int g, int s) { return m->n[2 * g + s]; }

int mixed_rho_momentum(MixedState* m, int g, const double q_s[2], double* rho, double* mom, cudaStream_t st,
                       std::string& err) {
    DevStatus hs{};
    if (int rc = read_status(m, hs, st, err)) return rc;
    const GridDev& G = m->G[g];
    for (int s = 0; s < 2; s++) {
        PartArrays S{};
        long long n = 0;
        if (int rc = gather_species(m, g, (int)hs.parity, s, S, n, st, err)) return rc;
        if (n && rho && q_s[s] != 0.0) {
            const double q = q_s[s];
            switch (G.order) {
            case 1: k_rho_staged<1><<<grid1(n), 256, 0, st>>>(n, G, S, q, rho); break;
            case 2: k_rho_staged<2><<<grid1(n), 256, 0, st>>>(n, G, S, q, rho); break;
            default: k_rho_staged<3><<<grid1(n), 256, 0, st>>>(n, G, S, q, rho); break;
            }
        }
        if (n && mom) k_momentum_staged<<<304, 256, 0, st>>>(n, S, G.w, mom);
        const cudaError_t e = cudaStreamSynchronize(st);
        free_parts(S, st);
        if (e != cudaSuccess) {
            err = std::string("diagnostics: ") + cudaGetErrorString(e);
            return PIC_ECUDA;
        }
    }
    return PIC_OK;
}
long long mixed_rebins(MixedState* m) { return m->rebins; }
long long mixed_generation(MixedState* m) { return m->gen; }

int mixed_particles(MixedState* m, int g, int s, double* out, long long n, cudaStream_t st,
                    std::string& err) {
    DevStatus hs{};
    if (int rc = read_status(m, hs, st, err)) return rc;
    PartArrays S{};
    long long got = 0;
    int rc = gather_species(m, g, (int)hs.parity, s, S, got, st, err);
    if (rc) return rc;
    if (got != n) {
        free_parts(S, st);
        err = "particle count mismatch (" + std::to_string(got) + " live, " + std::to_string(n) + " requested)";
        return PIC_ESTATE;
    }
    double* t = nullptr;
    MCK(talloc(&t, 5 * (size_t)std::max<long long>(n, 1), st));
    if (n) k_unstage<<<grid1(n), 256, 0, st>>>(n, m->G[g], S, t);
    MCK(cudaMemcpyAsync(out, t, 5 * n * sizeof(double), cudaMemcpyDefault, st));
    MCK(cudaStreamSynchronize(st));
    tfree(t, st);
    free_parts(S, st);
    return PIC_OK;
}

}  // namespace pic
