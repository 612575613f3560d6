// common.cuh -- shared device definitions of the GB300 LBM-DEM library.
//
// D3Q19 lattice (Sec. 2.1) with the velocity ordering fixed by rows 2-4 of the
// moment matrix in App. A, storage traits for the shifted PDF formats, the
// layout of the device state and small helpers.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace lbmdem {

constexpr int Q = 19;

// Lattice velocities c_q, q = 0..18, as fixed by rows 2-4 of M (App. A):
// 0 rest, 1 N(0,1,0), 2 S(0,-1,0), 3 W(-1,0,0), 4 E(1,0,0), 5 T(0,0,1),
// 6 B(0,0,-1), 7 NW, 8 NE, 9 SW, 10 SE, 11 TN, 12 TS, 13 TW, 14 TE,
// 15 BN, 16 BS, 17 BW, 18 BE.
__host__ __device__ constexpr int cx(int q) {
    constexpr int t[Q] = {0, 0, 0, -1, 1, 0, 0, -1, 1, -1, 1, 0, 0, -1, 1, 0, 0, -1, 1};
    return t[q];
}
__host__ __device__ constexpr int cy(int q) {
    constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, -1, 0, 0, 1, -1, 0, 0};
    return t[q];
}
__host__ __device__ constexpr int cz(int q) {
    constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, 1, 1, -1, -1, -1, -1};
    return t[q];
}
// opposite direction qbar with c_qbar = -c_q
__host__ __device__ constexpr int opp(int q) {
    constexpr int t[Q] = {0, 2, 1, 4, 3, 6, 5, 10, 9, 8, 7, 16, 15, 18, 17, 12, 11, 14, 13};
    return t[q];
}
// squared length |c_q|^2 (0, 1 or 2); lattice weights 1/3, 1/18, 1/36
__host__ __device__ constexpr int c2(int q) { return cx(q) * cx(q) + cy(q) * cy(q) + cz(q) * cz(q); }
template <typename T>
__host__ __device__ constexpr T wq(int q) {
    return c2(q) == 0 ? T(1) / T(3) : (c2(q) == 1 ? T(1) / T(18) : T(1) / T(36));
}

// lattice direction components as 2-bit fields (c + 1) of one word per axis,
// for directions chosen at run time (one per lane)
__host__ __device__ constexpr unsigned long long pack_dirs(int axis) {
    unsigned long long v = 0;
    for (int q = 0; q < Q; ++q)
        v |= (unsigned long long)((axis == 0 ? cx(q) : axis == 1 ? cy(q) : cz(q)) + 1) << (2 * q);
    return v;
}
__device__ __forceinline__ int dir_c(unsigned long long packed, int q) { return (int)((packed >> (2 * q)) & 3ull) - 1; }

// NaN marker held by every PDF slot of a solid cell: a quiet NaN whose low 22
// bits carry owner + 1 in the 4- and 8-byte formats (the 16-bit formats keep
// no payload). Arithmetic NaNs are canonical (all payload bits set), which
// decodes to an index above every particle count the library accepts.
constexpr unsigned int MARKER_PAYLOAD = 0x3FFFFFu;
__device__ __forceinline__ unsigned int marker_bits32(int owner) { return 0x7FC00000u | (unsigned)(owner + 1); }
__device__ __forceinline__ unsigned long long marker_bits64(int owner) {
    return 0x7FF8000000000000ull | (unsigned long long)(owner + 1);
}
__device__ __forceinline__ int marker_owner(float v) { return (int)(__float_as_uint(v) & MARKER_PAYLOAD) - 1; }
__device__ __forceinline__ int marker_owner(double v) {
    return (int)((unsigned long long)__double_as_longlong(v) & MARKER_PAYLOAD) - 1;
}

// flag bits (mirrors LBM_FLAG_* of the public header)
constexpr uint8_t FL_SOLID = 0x01, FL_SHELL = 0x02, FL_NEAR = 0x04, FL_MISS = 0x08,
                  FL_NEWFLUID = 0x10, FL_MULTI = 0x20;

// device status bits (sticky, reported to the host by lbm_sync)
constexpr int ST_UNSTABLE = 1, ST_TILE_OVERFLOW = 2, ST_NBR_OVERFLOW = 4, ST_BIN_OVERFLOW = 8,
              ST_REFILL_OVERFLOW = 16, ST_HIST_OVERFLOW = 32, ST_FAST_PARTICLE = 64,
              ST_FIXED_OVERFLOW = 128, ST_TIMEOUT = 256;

// capacities of the fixed-size device lists
#ifndef LBM_TILE_Z
#define LBM_TILE_Z 4
#endif
constexpr int TILE_X = 32, TILE_Y = 4, TILE_Z = LBM_TILE_Z;   // mapping tile (512 cells at depth 4)
constexpr int TILE_CAP = 64;                          // candidate particles per tile
constexpr int BIN_CAP = 32;                           // particles per DEM bin
constexpr int NBR_CAP = 32;                           // neighbour candidates per particle
constexpr double NBR_SKIN = 1.0;                      // Verlet skin of the per-step list

// --------------------------------------------------------------------------
// storage traits: every format stores the shifted PDF f_q - w_q
// --------------------------------------------------------------------------
template <typename S> struct Store;
template <> struct Store<double> {
    using T = double;
    __device__ static T load(const double* p) { return __ldg(p); }
    __device__ static void store(double* p, T v) { *p = v; }
};
template <> struct Store<float> {
    using T = float;
    __device__ static T load(const float* p) { return __ldg(p); }
    __device__ static void store(float* p, T v) { *p = v; }
};
template <> struct Store<__half> {
    using T = float;
    __device__ static T load(const __half* p) { return __half2float(__ldg(p)); }
    __device__ static void store(__half* p, T v) { *p = __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
    using T = float;
    __device__ static T load(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
    __device__ static void store(__nv_bfloat16* p, T v) { *p = __float2bfloat16_rn(v); }
};

// --------------------------------------------------------------------------
// device state
// --------------------------------------------------------------------------
struct Geom {
    int n[3];            // nx, ny, nz
    int per[3];          // periodic axis flags
    long long ncells;    // nx ny nz
    double wall_vel[2][3][3];   // [side][axis][component]
};

// float view of a particle for the float32 kernels: position split into an
// integer cell base and a fraction so that cell-relative offsets keep full
// float precision anywhere in the box
struct __align__(16) PartView {
    int base[3];
    float frac[3];
    float R;
    float u[3];
    float om[3];
    float C;               // |g|^2 - R^2 with g = 1/2 - frac (per-axis fractional offsets),
    float C_lo;            // in two parts: C + C_lo holds it to float64 accuracy
};

// C and C_lo of a view whose frac is set, from the float32 g = 1/2 - frac the
// link arithmetic uses (so |n + g|^2 - R^2 = |n|^2 + 2 n.g + C + C_lo is the
// exact value for the sphere centred at base + frac)
__device__ __forceinline__ void set_view_c(PartView& v, double R) {
    double gg = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float gf = 0.5f - v.frac[d];
        gg += (double)gf * (double)gf;
    }
    const double C = gg - R * R;
    v.C = (float)C;
    v.C_lo = (float)(C - (double)v.C);
}

struct Particles {
    int n;                 // particle count
    double* x;             // [3n] centre positions
    double* u;             // [3n] translational velocities
    double* om;            // [3n] angular velocities
    double* R;             // [n]  radii
    double* rho;           // [n]  density ratios rho_p / rho_f
    double* m;             // [n]  masses rho_p pi D^3 / 6
    double* I;             // [n]  moments of inertia 2/5 m R^2
    double* hm;            // [n]  1 / (2 m)
    double* hI;            // [n]  1 / (2 I)
    double* ext;           // [3n] external force V (rho_p - rho_f) g
    double* F_prev;        // [3n] total force of the last subcycle
    double* T_prev;        // [3n]
    double* F_new;         // [3n] total force of the current subcycle
    double* T_new;         // [3n]
    double* acc_d;         // [6n] float64 link-force accumulators (F, T)
    long long* acc_i;      // [6n] fixed-point link-force accumulators (float32 kernels)
    long long* acc_k;      // [3n] exact 36 x (constant link force, its torque about the base cell), two per word
    double* fp;            // [6n] F^fp, T^fp of the last step
    double* fp_old;        // [6n] F^fp, T^fp of the step before
    double* fbar;          // [6n] averaged F^fp, T^fp used by the DEM
    PartView* view;        // [n]
    float* xf;             // [3n] float32 copy of x for neighbour prefilters
    // double-buffered subcycle state: index 0 is x/u/om/xf above, 1 the copy
    double* xs[2];
    double* us[2];
    double* oms[2];
    float* xfs[2];
    float* ufs[2];         // float32 copies of us, oms for the float32 pair laws
    float* omfs[2];
    // DEM neighbour structure and contact history
    int* bin_count;        // [nbins]
    int* bin_list;         // [nbins * BIN_CAP]
    int* nbr_count;        // [n]
    int* nbr;              // [n * NBR_CAP]
    int* hist_id[2];       // [n * NBR_CAP] partner of each neighbour slot in contact (-1: none)
    double* hist_d[2];     // [n * NBR_CAP * 3] tangential springs
    int* hist_n[2];        // [n] number of valid slots
    double* whist[2];      // [n * 6 * 3] wall tangential springs per face
    unsigned char* wact[2];// [n * 6] wall contact active flags
};

// fixed-point scale of the float32 link-force accumulation: 2^32
constexpr double FIX_SCALE = 4294967296.0;

__device__ __forceinline__ int wrap_idx(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

}  // namespace lbmdem
