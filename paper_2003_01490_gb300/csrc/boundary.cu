// boundary.cu -- particle links and their forces: the first kernel of one
// lattice Boltzmann step with moving particles (Algorithm 1, line 1, the
// boundary handling before the stream).
//
// One warp per particle i. The warp walks the cells whose centre lies in the
// shell R_i - 0.01 < |x - x_i| <= R_i + sqrt(2) + 0.03 around its sphere,
// column by column (the x range of each (y, z) column follows from the circle
// equation; float32 with margins, so the walk covers every fluid cell that can
// have a link into sphere i), keeps the fluid cells (owner -1) and finds the
// directions q whose upstream cell y = x - c_q is a cell of particle i
// (owner[y] == i). Each such link gets the CLI moving no-slip condition of
// Eq. (14) along p = qbar (link fraction delta_p from the ray-sphere
// intersection; bounce-back, delta = 1/2 in the coefficients, when x + c_q is
// not fluid): the value f_q(x, t+1) is written into the slot f_q(y) of the
// solid cell, the one slot that the pull of x reads, so the dense kernel needs
// no boundary logic. The link force of Eq. (15) and its torque are summed in
// the warp's registers and added to particle i once (Eqs. (16)-(17)): no
// contention between particles, and a summation order that does not depend on
// scheduling. A cell next to two spheres is visited by both warps, each taking
// the links into its own sphere.
//
// Float32 compute: the link force splits into the constant part 2 w_p c_p,
// an integer multiple of c_p / 36, and the small remainder
// c_p (f~_p + f_q) - u_b (f~_p - f_q). The constant part and its torque
// 2 w_p (n + g) x c_p (n the integer offset of the cell from the particle's
// base cell, g the fractional offset common to all links) are summed exactly
// in integers; the remainder is summed per lane in compensated float32
// (TwoSum) and over the warp in 64-bit fixed point (scale 2^32). No float64
// instruction runs per link on the float32 path. Float64 storage sums in
// float64.
//
// Missing links (Sec. 2.2): the blocks after the particle blocks walk the
// missing-link list of the mapping (solid cells next to another body); each
// missing link adds F_q = 2 w_q c_q, reduced per warp and added atomically.
#include "common.cuh"
#include "launch.h"

// minimum resident blocks (of 128 threads) per SM with 4-byte or smaller
// storage: a register cap
#ifndef LBM_BC_MIN_BLOCKS
#define LBM_BC_MIN_BLOCKS 6
#endif

namespace lbmdem {

template <typename S>
struct BcArgs {
    S* src;                          // written only in solid-cell slots
    const uint8_t* __restrict__ flags;
    const int* __restrict__ owner;   // particle of a solid cell, -1 for fluid
    Geom g;
    int np;                          // particles (one warp each)
    int pblocks;                     // blocks of particle warps; the rest walk the missing-link list
    const unsigned int* __restrict__ miss;   // solid cells with possible missing links
    const int* miss_count;
    int miss_cap;
    const double* __restrict__ px;
    const double* __restrict__ pu;
    const double* __restrict__ pom;
    const double* __restrict__ pR;
    const PartView* __restrict__ view;
    double* acc_d;
    long long* acc_i;
    long long* acc_k;
    int missing_links;
    int* status;
    // fluid body force of the step: a_user - ext_total / N_fluid (counter force)
    double a_user[3];
    double ext_total[3];
    int counterforce;
    const unsigned long long* n_solid;
    double* accel_d;
    float* accel_f;
};

// ------------------------------------------------------------------ helpers

// float -> fixed point with scale 2^32 using float32 and int32 operations only;
// exact up to the final rounding at 2^-32. |v| must stay below 2^31.
__device__ __forceinline__ long long to_fixed(float v, int* status) {
    float hi = truncf(v);
    float r1 = (v - hi) * 65536.0f;
    float mid = truncf(r1);
    float r2 = (r1 - mid) * 65536.0f;
    if (!(fabsf(hi) < 2147483520.0f)) {
        atomicOr(status, ST_FIXED_OVERFLOW);
        return 0;
    }
    unsigned long long h = (unsigned long long)(long long)__float2int_rz(hi);
    long long m = (long long)__float2int_rz(mid);
    long long l = (long long)__float2int_rn(r2);
    return (long long)(h << 32) + m * 65536LL + l;
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
__device__ __forceinline__ void add_int(const Sinks& s, int i, int c, int v) {
    if (v) atomicAdd(reinterpret_cast<unsigned long long*>(s.acc_k + 6 * i + c), (unsigned long long)(long long)v);
}

template <typename T>
__device__ __forceinline__ void flush(Acc<T>& a, const Sinks& s) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        add_float(s, a.key, c, a.f[c]);
        if (sizeof(T) == 4) add_int(s, a.key, c, a.k[c]);
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
            if (sizeof(T) == 4) add_int(s, a.key, c, a.k[c]);
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
        const PartView v = a.view[i];
        const int c[3] = {x, y, z};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            int nd = c[d] - v.base[d];
            const float g = 0.5f - v.frac[d];
            if (a.g.per[d]) {
                const float half = 0.5f * (float)a.g.n[d];
                const float rd = (float)nd + g;
                if (rd > half) nd -= a.g.n[d];
                else if (rd < -half) nd += a.g.n[d];
            }
            n[d] = nd;
            r[d] = (float)nd + g;
            u[d] = v.u[d];
            om[d] = v.om[d];
        }
        R = v.R;
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

// smallest t in [0, 1] with |r + t c| = R (link fraction delta of Eq. (14)).
// |r|^2 - R^2 cancels strongly near the surface, so it is formed from exact
// products and compensated sums; the root uses the cancellation-free form
// t = 2 cc / (-b + sqrt(b^2 - 4 a cc)) of the smaller root.
template <typename T>
__device__ __forceinline__ T link_fraction(const T (&r)[3], T c0, T c1, T c2_, T cc2, T R) {
    const T b = T(2) * (r[0] * c0 + r[1] * c1 + r[2] * c2_);
    T err = T(0);
    const T p0 = r[0] * r[0], p1 = r[1] * r[1], p2 = r[2] * r[2], pR = R * R;
    const T e = (fma_t<T>(r[0], r[0], -p0) + fma_t<T>(r[1], r[1], -p1)) +
                (fma_t<T>(r[2], r[2], -p2) - fma_t<T>(R, R, -pR));
    T sum = two_sum<T>(p0, p1, err);
    sum = two_sum<T>(sum, p2, err);
    sum = two_sum<T>(sum, -pR, err);
    const T cc = sum + (err + e);
    const T disc = b * b - T(4) * cc2 * cc;
    if (disc < T(0)) return T(0.5);
    const T sq = sqrt(disc);
    const T t = b < T(0) ? (T(2) * cc) / (sq - b) : (-b - sq) / (T(2) * cc2);
    return t < T(0) ? T(0) : (t > T(1) ? T(1) : t);
}

// lattice directions as run-time tables (for link work distributed over lanes)
__constant__ signed char k_c[Q][3] = {{0, 0, 0},   {0, 1, 0},   {0, -1, 0},  {-1, 0, 0},  {1, 0, 0},
                                      {0, 0, 1},   {0, 0, -1},  {-1, 1, 0},  {1, 1, 0},   {-1, -1, 0},
                                      {1, -1, 0},  {0, 1, 1},   {0, -1, 1},  {-1, 0, 1},  {1, 0, 1},
                                      {0, 1, -1},  {0, -1, -1}, {-1, 0, -1}, {1, 0, -1}};
__constant__ signed char k_opp[Q] = {0, 2, 1, 4, 3, 6, 5, 10, 9, 8, 7, 16, 15, 18, 17, 12, 11, 14, 13};


// missing links of a solid cell s of particle i: links x -> s from cells x of
// another body whose centre is not inside sphere i
template <typename S, typename T>
__device__ __forceinline__ void missing_links(const BcArgs<S>& a, long long idx, Acc<T>& acc, const Sinks& sk) {
    const int nx = a.g.n[0], ny = a.g.n[1];
    const long long plane = (long long)nx * ny;
    const int x = (int)(idx % nx), y = (int)((idx / nx) % ny), z = (int)(idx / plane);
    const int cpos[3] = {x, y, z};
    const int i = a.owner[idx];
    unsigned cand = 0, solidm = 0;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        int v[3];
        bool outside = false;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            v[d] = cpos[d] - (d == 0 ? cx(q) : d == 1 ? cy(q) : cz(q));
            if (!a.g.per[d] && (v[d] < 0 || v[d] >= a.g.n[d])) outside = true;
            v[d] = wrap_idx(v[d], a.g.n[d]);
        }
        if (outside) cand |= 1u << q;
        else if (a.flags[(long long)v[2] * plane + (long long)v[1] * nx + v[0]] & FL_SOLID) solidm |= 1u << q;
    }
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        if (!(solidm & (1u << q))) continue;
        const int v0 = wrap_idx(x - cx(q), nx), v1 = wrap_idx(y - cy(q), ny), v2 = wrap_idx(z - cz(q), a.g.n[2]);
        if (a.owner[(long long)v2 * plane + (long long)v1 * nx + v0] != i) cand |= 1u << q;
    }
    while (cand) {
        const int q = __ffs(cand) - 1;
        cand &= cand - 1;
        const int c[3] = {k_c[q][0], k_c[q][1], k_c[q][2]};
        // exact float64 inside test of the far cell centre against sphere i,
        // in the operation order of the mapping
        double dd[3];
#pragma unroll
        for (int d = 0; d < 3; ++d)
            dd[d] = min_image_d(((double)(cpos[d] - c[d]) + 0.5) - a.px[3 * i + d], a.g.n[d], a.g.per[d]);
        const double Ri = a.pR[i];
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dd[0], dd[0]), __dmul_rn(dd[1], dd[1])), __dmul_rn(dd[2], dd[2]));
        if (!(d2 > __dmul_rn(Ri, Ri))) continue;
        T r[3], R, u[3], om[3];
        int n[3];
        PartOps<T>::load(a, i, x - c[0], y - c[1], z - c[2], r, n, R, u, om);
        const int cc2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        int K[6] = {0, 0, 0, 0, 0, 0};
        T F[3] = {T(0), T(0), T(0)}, Tq[3] = {T(0), T(0), T(0)};
        if (sizeof(T) == 4) {
            // F = 2 w_q c_q and torque 2 w_q (r x c_q), r = n + g: exact integers (x 36)
            const int kw = cc2 == 1 ? 4 : 2;
            K[0] = kw * c[0]; K[1] = kw * c[1]; K[2] = kw * c[2];
            K[3] = kw * (n[1] * c[2] - n[2] * c[1]);
            K[4] = kw * (n[2] * c[0] - n[0] * c[2]);
            K[5] = kw * (n[0] * c[1] - n[1] * c[0]);
        } else {
            const T cf0 = (T)c[0], cf1 = (T)c[1], cf2 = (T)c[2];
            const T t = link_fraction<T>(r, cf0, cf1, cf2, (T)cc2, R);
            const T rb[3] = {r[0] + t * cf0, r[1] + t * cf1, r[2] + t * cf2};
            const T w2 = cc2 == 1 ? T(2) / T(18) : T(2) / T(36);
            F[0] = w2 * cf0; F[1] = w2 * cf1; F[2] = w2 * cf2;
            Tq[0] = rb[1] * F[2] - rb[2] * F[1];
            Tq[1] = rb[2] * F[0] - rb[0] * F[2];
            Tq[2] = rb[0] * F[1] - rb[1] * F[0];
        }
        accumulate<T>(i, F, Tq, K, acc, sk);
    }
}

// ------------------------------------------------------------------ particle links

// CLI condition and momentum exchange of one link of particle i: fluid cell
// cpos (integer offset n from the particle's base cell), pull direction q,
// solid upstream cell cpos - c_q of particle i. Sums into the lane's
// accumulators: fs (and its TwoSum error fe) for the float part, ks for the
// exact integer part of the float32 path.
template <typename S, typename T>
__device__ __forceinline__ void particle_link(const BcArgs<S>& a, const int (&cpos)[3], const int (&n)[3], int q,
                                              const float (&gf)[3], const double (&px)[3], T R, const T (&u)[3],
                                              const T (&om)[3], T (&fs)[6], T (&fe)[6], int (&ks)[6]) {
    const int nx = a.g.n[0], ny = a.g.n[1];
    const int plane = nx * ny;
    const long long N = a.g.ncells;
    const int c[3] = {k_c[q][0], k_c[q][1], k_c[q][2]};
    const int p = k_opp[q];
    int uv[3], dv[3];
    bool cli = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        uv[d] = wrap_idx(cpos[d] - c[d], a.g.n[d]);
        dv[d] = cpos[d] + c[d];
        if (!a.g.per[d] && (dv[d] < 0 || dv[d] >= a.g.n[d])) cli = false;
        dv[d] = wrap_idx(dv[d], a.g.n[d]);
    }
    const int idx = cpos[2] * plane + cpos[1] * nx + cpos[0];
    const int up = uv[2] * plane + uv[1] * nx + uv[0];
    const int down = dv[2] * plane + dv[1] * nx + dv[0];
    const T fout = Store<S>::load(a.src + p * N + idx);
    const T fin = Store<S>::load(a.src + q * N + idx);
    if (cli) cli = !(a.flags[down] & FL_SOLID);
    const T fdown = cli ? Store<S>::load(a.src + p * N + down) : T(0);
    T r[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if constexpr (sizeof(T) == 8) r[d] = min_image_d(((double)cpos[d] + 0.5) - px[d], a.g.n[d], a.g.per[d]);
        else r[d] = (float)n[d] + gf[d];
    }
    const int cp[3] = {-c[0], -c[1], -c[2]};
    const T cp0 = (T)cp[0], cp1 = (T)cp[1], cp2 = (T)cp[2];
    const int cc2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    const T w = cc2 == 1 ? T(1) / T(18) : T(1) / T(36);
    const T delta = link_fraction<T>(r, cp0, cp1, cp2, (T)cc2, R);
    const T dbc = cli ? delta : T(0.5);
    const T kappa = (T(1) - T(2) * dbc) / (T(1) + T(2) * dbc);
    const T rb[3] = {r[0] + delta * cp0, r[1] + delta * cp1, r[2] + delta * cp2};
    const T ub[3] = {u[0] + (om[1] * rb[2] - om[2] * rb[1]), u[1] + (om[2] * rb[0] - om[0] * rb[2]),
                     u[2] + (om[0] * rb[1] - om[1] * rb[0])};
    const T ubc = ub[0] * cp0 + ub[1] * cp1 + ub[2] * cp2;
    const T v = fout + kappa * (fdown - fin) - (T(12) * w / (T(1) + T(2) * dbc)) * ubc;
    // the pull of x in direction q reads exactly this solid-cell slot
    Store<S>::store(a.src + q * N + up, v);
    // Eq. (15) on shifted PDFs: F = c_p (2 w + f~_p + f_q) - u_b (f~_p - f_q)
    const T dif = fout - v;
    T sum;
    if constexpr (sizeof(T) == 4) {
        // 2 w_p c_p and its torque 2 w_p (n x c_p) as exact integers (x 36)
        const int kw = cc2 == 1 ? 4 : 2;
        sum = fout + v;
        ks[0] += kw * cp[0];
        ks[1] += kw * cp[1];
        ks[2] += kw * cp[2];
        ks[3] += kw * (n[1] * cp[2] - n[2] * cp[1]);
        ks[4] += kw * (n[2] * cp[0] - n[0] * cp[2]);
        ks[5] += kw * (n[0] * cp[1] - n[1] * cp[0]);
    } else {
        sum = T(2) * w + fout + v;
    }
    const T F[3] = {cp0 * sum - ub[0] * dif, cp1 * sum - ub[1] * dif, cp2 * sum - ub[2] * dif};
    const T Tq[6] = {F[0], F[1], F[2], rb[1] * F[2] - rb[2] * F[1], rb[2] * F[0] - rb[0] * F[2],
                     rb[0] * F[1] - rb[1] * F[0]};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        if constexpr (sizeof(T) == 4) fs[k] = two_sum<T>(fs[k], Tq[k], fe[k]);
        else fs[k] += Tq[k];
    }
}

// inclusive prefix sum over the warp and the lane holding rank k of it
__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}
__device__ __forceinline__ int owner_lane(int incl, int k) {
    int src = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int t = __shfl_sync(0xffffffffu, incl, src + step - 1);
        if (t <= k) src += step;
    }
    return src > 31 ? 31 : src;
}

// all links of particle i, one warp
template <typename S, typename T>
__device__ __forceinline__ void particle_warp(const BcArgs<S>& a, int i, int lane) {
    const unsigned FULL = 0xffffffffu;
    const int L3[3] = {a.g.n[0], a.g.n[1], a.g.n[2]};
    const int plane = L3[0] * L3[1];
    const PartView v = a.view[i];
    const float gf[3] = {0.5f - v.frac[0], 0.5f - v.frac[1], 0.5f - v.frac[2]};
    T R, u[3], om[3];
    double px[3] = {0.0, 0.0, 0.0};
    if constexpr (sizeof(T) == 8) {
        R = a.pR[i];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            u[d] = a.pu[3 * i + d];
            om[d] = a.pom[3 * i + d];
            px[d] = a.px[3 * i + d];
        }
    } else {
        R = v.R;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            u[d] = v.u[d];
            om[d] = v.om[d];
        }
    }
    // integer offsets n of the walked cells from the base cell, per axis: the
    // outer radius, one image per cell on periodic axes (-L/2 < n + g <= L/2),
    // the box on the others
    const float Rout = v.R + 1.4142135f + 0.03f;
    const float Rin = v.R - 0.01f;
    const float R2tol = v.R * v.R * 1.00001f + 1e-3f;   // superset of the float64 inside test
    int lo[3], hi[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        lo[d] = (int)ceilf(-Rout - gf[d]);
        hi[d] = (int)floorf(Rout - gf[d]);
        if (a.g.per[d]) {
            const float h = 0.5f * (float)L3[d];
            lo[d] = max(lo[d], (int)floorf(-h - gf[d]) + 1);
            hi[d] = min(hi[d], (int)floorf(h - gf[d]));
        } else {
            lo[d] = max(lo[d], -v.base[d]);
            hi[d] = min(hi[d], L3[d] - 1 - v.base[d]);
        }
    }
    const int wy = hi[1] - lo[1] + 1, wz = hi[2] - lo[2] + 1;
    if (wy <= 0 || wz <= 0 || hi[0] < lo[0]) return;   // warp-uniform
    const int ncol = wy * wz;
    T fs[6], fe[6];
    int ks[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        fs[k] = T(0);
        fe[k] = T(0);
        ks[k] = 0;
    }
    for (int c0 = 0; c0 < ncol; c0 += 32) {
        // this lane's column: cells [a0, a0 + na) and [b0, b0 + nb) in x
        const int col = c0 + lane;
        int col_y = 0, col_z = 0, a0 = 0, na = 0, b0 = 0, nb = 0;
        if (col < ncol) {
            const int kz = col / wy;
            col_z = lo[2] + kz;
            col_y = lo[1] + (col - kz * wy);
            const float ry = (float)col_y + gf[1], rz = (float)col_z + gf[2];
            const float s = ry * ry + rz * rz;
            const float o2 = Rout * Rout - s;
            if (o2 >= 0.f) {
                const float wo = sqrtf(o2);
                const int x0 = max(lo[0], (int)ceilf(-wo - gf[0]));
                const int x1 = min(hi[0], (int)floorf(wo - gf[0]));
                // cells with |n + g| < R - 0.01 are inside the sphere (solid)
                const float i2 = Rin * Rin - s;
                int e0 = 1, e1 = 0;
                if (Rin > 0.f && i2 > 0.f) {
                    const float wi = sqrtf(i2);
                    e0 = (int)floorf(-wi - gf[0]) + 1;
                    e1 = (int)ceilf(wi - gf[0]) - 1;
                }
                a0 = x0;
                if (e1 < e0) {
                    na = max(0, x1 - x0 + 1);
                } else {
                    na = max(0, min(x1, e0 - 1) - x0 + 1);
                    b0 = max(x0, e1 + 1);
                    nb = max(0, x1 - b0 + 1);
                }
            }
        }
        const int cnt = na + nb;
        const int incl = warp_incl_scan(cnt, lane);
        const int total = __shfl_sync(FULL, incl, 31);
        for (int k0 = 0; k0 < total; k0 += 32) {
            // cell k0 + lane of this batch of columns
            const int kk = k0 + lane;
            const int src = owner_lane(incl, kk);
            const int s_cy = __shfl_sync(FULL, col_y, src), s_cz = __shfl_sync(FULL, col_z, src);
            const int s_a0 = __shfl_sync(FULL, a0, src), s_na = __shfl_sync(FULL, na, src);
            const int s_b0 = __shfl_sync(FULL, b0, src), s_ex = __shfl_sync(FULL, incl - cnt, src);
            int n3[3] = {0, s_cy, s_cz};
            int cpos[3] = {0, 0, 0};
            unsigned m = 0;   // directions q with a link into particle i
            if (kk < total) {
                const int loc = kk - s_ex;
                n3[0] = loc < s_na ? s_a0 + loc : s_b0 + (loc - s_na);
#pragma unroll
                for (int d = 0; d < 3; ++d) cpos[d] = wrap_idx(v.base[d] + n3[d], L3[d]);
                if (a.owner[cpos[2] * plane + cpos[1] * L3[0] + cpos[0]] < 0) {
                    const float r0 = (float)n3[0] + gf[0], r1 = (float)n3[1] + gf[1], r2 = (float)n3[2] + gf[2];
#pragma unroll
                    for (int q = 1; q < Q; ++q) {
                        const float d0 = r0 - (float)cx(q), d1 = r1 - (float)cy(q), d2 = r2 - (float)cz(q);
                        if (d0 * d0 + d1 * d1 + d2 * d2 > R2tol) continue;
                        const int y3[3] = {cpos[0] - cx(q), cpos[1] - cy(q), cpos[2] - cz(q)};
                        bool out = false;
                        int yw[3];
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            if (!a.g.per[d] && (y3[d] < 0 || y3[d] >= L3[d])) out = true;
                            yw[d] = wrap_idx(y3[d], L3[d]);
                        }
                        if (!out && a.owner[yw[2] * plane + yw[1] * L3[0] + yw[0]] == i) m |= 1u << q;
                    }
                }
            }
            // the links of these 32 cells, spread evenly over the lanes
            const int lc = __popc(m);
            const int lincl = warp_incl_scan(lc, lane);
            const int ltot = __shfl_sync(FULL, lincl, 31);
            for (int r0 = 0; r0 < ltot; r0 += 32) {
                const int k2 = r0 + lane;
                const int s2 = owner_lane(lincl, k2);
                const unsigned sm = __shfl_sync(FULL, m, s2);
                const int sex = __shfl_sync(FULL, lincl - lc, s2);
                const int lp[3] = {__shfl_sync(FULL, cpos[0], s2), __shfl_sync(FULL, cpos[1], s2),
                                   __shfl_sync(FULL, cpos[2], s2)};
                const int ln[3] = {__shfl_sync(FULL, n3[0], s2), __shfl_sync(FULL, n3[1], s2),
                                   __shfl_sync(FULL, n3[2], s2)};
                if (k2 < ltot)
                    particle_link<S, T>(a, lp, ln, (int)__fns(sm, 0, k2 - sex + 1), gf, px, R, u, om, fs, fe, ks);
            }
        }
    }
    // one add per component and particle
    if constexpr (sizeof(T) == 4) {
        long long fx[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) fx[k] = to_fixed(fs[k], a.status) + to_fixed(fe[k], a.status);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                fx[k] += __shfl_xor_sync(FULL, fx[k], o);
                ks[k] += __shfl_xor_sync(FULL, ks[k], o);
            }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                if (fx[k]) atomicAdd(reinterpret_cast<unsigned long long*>(a.acc_i + 6 * i + k), (unsigned long long)fx[k]);
                if (ks[k]) atomicAdd(reinterpret_cast<unsigned long long*>(a.acc_k + 6 * i + k),
                                     (unsigned long long)(long long)ks[k]);
            }
        }
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < 6; ++k) fs[k] += __shfl_xor_sync(FULL, fs[k], o);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) atomicAdd(a.acc_d + 6 * i + k, (double)fs[k]);
        }
    }
}

template <typename S>
__global__ void __launch_bounds__(128, sizeof(S) == 8 ? 4 : LBM_BC_MIN_BLOCKS) boundary_kernel(const BcArgs<S> a) {
    using T = typename Store<S>::T;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double acc3[3] = {a.a_user[0], a.a_user[1], a.a_user[2]};
        if (a.counterforce) {
            const double nf = (double)(a.g.ncells - (long long)(*a.n_solid));
            for (int d = 0; d < 3; ++d) acc3[d] -= a.ext_total[d] / nf;
        }
        for (int d = 0; d < 3; ++d) {
            a.accel_d[d] = acc3[d];
            a.accel_f[d] = (float)acc3[d];
        }
    }
    const int lane = threadIdx.x & 31;
    if ((int)blockIdx.x < a.pblocks) {
        const int i = (int)blockIdx.x * 4 + (threadIdx.x >> 5);
        if (i < a.np) particle_warp<S, T>(a, i, lane);
        return;
    }
    // ------------------------------------------- missing links (Sec. 2.2)
    if (!a.missing_links) return;
    const Sinks sk{a.acc_d, a.acc_i, a.acc_k, a.status};
    const int mcount = min(*a.miss_count, a.miss_cap);
    const int mb = (int)gridDim.x - a.pblocks;
    for (int base = ((int)blockIdx.x - a.pblocks) * blockDim.x; base < mcount; base += mb * blockDim.x) {
        const int k = base + threadIdx.x;
        Acc<T> acc;
        if (k < mcount) missing_links<S, T>(a, (long long)a.miss[k], acc, sk);
        commit<T>(acc, sk);
    }
}

template <typename S>
void launch_boundary_t(const LbmStepParams& p, cudaStream_t st) {
    BcArgs<S> b;
    b.src = static_cast<S*>(const_cast<void*>(p.src));
    b.flags = p.flags;
    b.owner = p.owner;
    b.g = p.g;
    b.np = p.P.n;
    b.pblocks = (p.P.n + 3) / 4;
    b.miss = p.miss_list;
    b.miss_count = p.miss_count;
    b.miss_cap = p.miss_cap;
    b.px = p.P.x;
    b.pu = p.P.u;
    b.pom = p.P.om;
    b.pR = p.P.R;
    b.view = p.P.view;
    b.acc_d = p.P.acc_d;
    b.acc_i = p.P.acc_i;
    b.acc_k = p.P.acc_k;
    b.missing_links = p.missing_links;
    b.status = p.status;
    for (int d = 0; d < 3; ++d) {
        b.a_user[d] = p.a_user[d];
        b.ext_total[d] = p.ext_total[d];
    }
    b.counterforce = p.counterforce;
    b.n_solid = p.n_solid;
    b.accel_d = p.accel_d;
    b.accel_f = p.accel_f;
    const int mblocks = p.missing_links ? (p.num_sms > 0 ? p.num_sms : 1) : 0;
    const int blocks = b.pblocks + mblocks > 0 ? b.pblocks + mblocks : 1;
    boundary_kernel<S><<<blocks, 128, 0, st>>>(b);
}

void launch_boundary(const LbmStepParams& p, cudaStream_t st) {
    switch (p.storage) {
        case 0: launch_boundary_t<double>(p, st); break;
        case 1: launch_boundary_t<float>(p, st); break;
        case 2: launch_boundary_t<__half>(p, st); break;
        default: launch_boundary_t<__nv_bfloat16>(p, st); break;
    }
}

}  // namespace lbmdem
