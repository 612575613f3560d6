// links.cuh -- device helpers shared by the kernels that handle particle
// links: fixed-point and warp-segmented force sums, the particle view used by
// the float32 kernels, the link fraction of Eq. (14) and warp prefix sums.
#pragma once

#include "common.cuh"

namespace lbmdem {

// float -> fixed point with scale 2^32: v 2^32 is exact in float32 and
// rounds to the nearest 64-bit integer. |v| must stay below 2^31.
__device__ __forceinline__ long long to_fixed(float v, int* status) {
    if (!(fabsf(v) < 2147483520.0f)) {
        atomicOr(status, ST_FIXED_OVERFLOW);
        return 0;
    }
    return __float2ll_rn(v * 4294967296.0f);
}

// per-lane partial sums of one particle's link forces and torques
template <typename T>
struct Acc {
    int key = -1;                  // particle index, -1 = nothing accumulated
    T f[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    int k[6] = {0, 0, 0, 0, 0, 0}; // float32 path: 36 x constant force, 36 x (n x c) torque
};

struct Sinks {
    double* acc_d;
    long long* acc_i;
    long long* acc_k;
    int* status;
};

__device__ __forceinline__ void add_float(const Sinks& s, int i, int c, double v) { atomicAdd(s.acc_d + 6 * i + c, v); }
__device__ __forceinline__ void add_float(const Sinks& s, int i, int c, float v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(s.acc_i + 6 * i + c), (unsigned long long)to_fixed(v, s.status));
}
// two exact integer sums (components 2 c2 and 2 c2 + 1) in one 64-bit word,
// lo + hi 2^32: a particle's totals stay inside 32 bits (radius <= 100), so
// the halves separate exactly however the adds wrap
__device__ __forceinline__ void add_int2(const Sinks& s, int i, int c2, int lo, int hi) {
    if (lo | hi)
        atomicAdd(reinterpret_cast<unsigned long long*>(s.acc_k + 3 * i + c2),
                  ((unsigned long long)(long long)hi << 32) + (unsigned long long)(long long)lo);
}

template <typename T>
__device__ __forceinline__ void flush(Acc<T>& a, const Sinks& s) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        add_float(s, a.key, c, a.f[c]);
        if (sizeof(T) == 4 && (c & 1)) add_int2(s, a.key, c >> 1, a.k[c - 1], a.k[c]);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        a.f[c] = T(0);
        a.k[c] = 0;
    }
}

// warp-level commit of the per-lane partial sums: lanes holding the same
// particle (found with match_any) are reduced by a tree over their ranks and
// the lowest lane of each group issues the atomics
template <typename T>
__device__ __forceinline__ void commit(Acc<T>& a, const Sinks& s) {
    const unsigned full = 0xffffffffu;
    if (__ballot_sync(full, a.key >= 0) == 0) return;
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(full, a.key);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    const int size = __popc(peers);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        // partner: the peer whose rank is rank + off (only read when it exists)
        const int pr = rank + off;
        const int src = pr < size ? (int)__fns(peers, 0, pr + 1) : lane;
        const bool take = (rank & (2 * off - 1)) == 0 && pr < size;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const T v = __shfl_sync(full, a.f[c], src);
            if (take) a.f[c] += v;
            if (sizeof(T) == 4) {
                const int iv = __shfl_sync(full, a.k[c], src);
                if (take) a.k[c] += iv;
            }
        }
    }
    if (rank == 0 && a.key >= 0) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            add_float(s, a.key, c, a.f[c]);
            if (sizeof(T) == 4 && (c & 1)) add_int2(s, a.key, c >> 1, a.k[c - 1], a.k[c]);
        }
    }
}

template <typename T>
__device__ __forceinline__ void accumulate(int i, const T (&F)[3], const T (&Tq)[3], const int (&K)[6], Acc<T>& a,
                                           const Sinks& s) {
    if (a.key >= 0 && a.key != i) flush(a, s);   // a second particle in the same lane
    a.key = i;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a.f[c] += F[c];
        a.f[3 + c] += Tq[c];
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) a.k[c] += K[c];
}

__device__ __forceinline__ double min_image_d(double d, int n, int per) {
    if (per) {
        double half = 0.5 * (double)n;
        if (d > half) d -= (double)n;
        if (d < -half) d += (double)n;
    }
    return d;
}

// offset r = (cell centre - particle centre) with minimum image, the integer
// part n of that offset from the particle's base cell (float32 path), and the
// rigid body data of particle i, in the compute precision T
template <typename T> struct PartOps;
template <> struct PartOps<double> {
    template <typename A>
    __device__ static void load(const A& a, int i, int x, int y, int z, double (&r)[3], int (&n)[3], double& R,
                                double (&u)[3], double (&om)[3]) {
        const int c[3] = {x, y, z};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            r[d] = min_image_d(((double)c[d] + 0.5) - a.px[3 * i + d], a.g.n[d], a.g.per[d]);
            n[d] = 0;
            u[d] = a.pu[3 * i + d];
            om[d] = a.pom[3 * i + d];
        }
        R = a.pR[i];
    }
};
template <> struct PartOps<float> {
    template <typename A>
    __device__ static void load(const A& a, int i, int x, int y, int z, float (&r)[3], int (&n)[3], float& R,
                                float (&u)[3], float (&om)[3]) {
        float g[3], C[2];
        load(a, i, x, y, z, r, n, g, C, R, u, om);
    }
    // also the fractional offset g and C = |g|^2 - R^2 of the particle. The
    // image is chosen on the integer offset: a link cell lies within R + 2
    // cells of the centre on every axis and a periodic side is longer than
    // 2 R + 4, so exactly one image has |n_d| <= floor(n / 2)
    template <typename A>
    __device__ static void load(const A& a, int i, int x, int y, int z, float (&r)[3], int (&n)[3], float (&g)[3],
                                float (&C)[2], float& R, float (&u)[3], float (&om)[3]) {
        const PartView v = a.view[i];
        const int c[3] = {x, y, z};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            int nd = c[d] - v.base[d];
            g[d] = 0.5f - v.frac[d];
            if (a.g.per[d]) {
                const int L = a.g.n[d], half = L >> 1;
                if (nd > half) nd -= L;
                else if (nd < -half) nd += L;
            }
            n[d] = nd;
            r[d] = (float)nd + g[d];
            u[d] = v.u[d];
            om[d] = v.om[d];
        }
        R = v.R;
        C[0] = v.C;
        C[1] = v.C_lo;
    }
};

// error-free transformations (Knuth's TwoSum, FMA product error)
template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <> __device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <> __device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return fma(a, b, c); }
template <typename T>
__device__ __forceinline__ T two_sum(T a, T b, T& err) {
    const T s = a + b;
    const T bb = s - a;
    err += (a - (s - bb)) + (b - bb);
    return s;
}

// square root and quotient: hardware approximations (a few ulp) for float32,
// IEEE for float64
__device__ __forceinline__ float fast_sqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
__device__ __forceinline__ double fast_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fast_div(double a, double b) { return a / b; }

// smallest t in [0, 1] with |r + t c| = R (link fraction delta of Eq. (14)).
// |r|^2 - R^2 cancels strongly near the surface, so it is formed from exact
// products and compensated sums; the root uses the cancellation-free form
// t = 2 cc / (-b + sqrt(b^2 - 4 a cc)) of the smaller root.
template <typename T>
__device__ __forceinline__ T link_root(const T (&r)[3], T cc, T c0, T c1, T c2_, T cc2) {
    const T b = T(2) * (r[0] * c0 + r[1] * c1 + r[2] * c2_);
    const T disc = b * b - T(4) * cc2 * cc;
    if (disc < T(0)) return T(0.5);
    const T sq = fast_sqrt(disc);
    const bool neg = b < T(0);
    const T t = fast_div(neg ? T(2) * cc : -b - sq, neg ? sq - b : T(2) * cc2);
    return t < T(0) ? T(0) : (t > T(1) ? T(1) : t);
}

// |r|^2 - R^2 from exact products and compensated sums
template <typename T>
__device__ __forceinline__ T surface_cc(const T (&r)[3], T R) {
    T err = T(0);
    const T p0 = r[0] * r[0], p1 = r[1] * r[1], p2 = r[2] * r[2], pR = R * R;
    const T e = (fma_t<T>(r[0], r[0], -p0) + fma_t<T>(r[1], r[1], -p1)) +
                (fma_t<T>(r[2], r[2], -p2) - fma_t<T>(R, R, -pR));
    T sum = two_sum<T>(p0, p1, err);
    sum = two_sum<T>(sum, p2, err);
    sum = two_sum<T>(sum, -pR, err);
    return sum + (err + e);
}

// the same for r = n + g with integer n and the particle's common fractional
// offset g: (|n|^2 + C) + (2 n.g + C_lo), with C + C_lo = |g|^2 - R^2
// precomputed per particle to float64 accuracy. Near the surface |n|^2 and
// -C agree to within a factor of two, so their sum is exact and only the
// small terms round.
__device__ __forceinline__ float surface_cc_split(const int (&n)[3], const float (&g)[3], const float (&C)[2]) {
    const int nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
    const float ng = fmaf((float)n[2], g[2], fmaf((float)n[1], g[1], (float)n[0] * g[0]));
    return ((float)nn + C[0]) + fmaf(2.0f, ng, C[1]);
}

template <typename T>
__device__ __forceinline__ T link_fraction(const T (&r)[3], T c0, T c1, T c2_, T cc2, T R) {
    return link_root<T>(r, surface_cc<T>(r, R), c0, c1, c2_, cc2);
}

// lattice directions as run-time tables (for link work distributed over lanes)
static __constant__ signed char k_c[Q][3] = {{0, 0, 0},   {0, 1, 0},   {0, -1, 0},  {-1, 0, 0},  {1, 0, 0},
                                      {0, 0, 1},   {0, 0, -1},  {-1, 1, 0},  {1, 1, 0},   {-1, -1, 0},
                                      {1, -1, 0},  {0, 1, 1},   {0, -1, 1},  {-1, 0, 1},  {1, 0, 1},
                                      {0, 1, -1},  {0, -1, -1}, {-1, 0, -1}, {1, 0, -1}};
static __constant__ signed char k_opp[Q] = {0, 2, 1, 4, 3, 6, 5, 10, 9, 8, 7, 16, 15, 18, 17, 12, 11, 14, 13};

// inclusive prefix sum over the warp
__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

}  // namespace lbmdem
