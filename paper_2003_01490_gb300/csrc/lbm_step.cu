// lbm_step.cu -- the two kernels of one lattice Boltzmann step with moving
// particles (Algorithm 1, lines 1-3).
//
// boundary_kernel: the near-boundary list of the mapping holds fluid cells
//   that may have particle links. For a fluid cell x and a direction q whose
//   upstream cell y = x - c_q is solid (particle i), the CLI moving no-slip
//   condition of Eq. (14) along the link p = qbar (link fraction delta_p from
//   the ray-sphere intersection; bounce-back, delta = 1/2 in the coefficients,
//   when x + c_q is not fluid) gives f_q(x, t+1). The value is written into
//   the slot f_q(y) of the solid cell, the one slot the pull of x reads, so
//   the dense kernel needs no boundary logic. The link force of Eq. (15) and
//   its torque are summed per particle (Eqs. (16)-(17)). The links of a warp's
//   cells are spread evenly over its lanes. The missing-link list holds solid
//   cells next to another body; each missing link adds F_q = 2 w_q c_q
//   (Sec. 2.2).
// stream_collide_kernel: one thread per cell, pull streaming (Eq. (2)) with
//   halfway bounce-back on the walls of the box (Eq. (14), delta = 1/2, wall
//   velocity), then the two-relaxation-time collision (Eq. (10), magic
//   parameter Eq. (11)) with Guo forcing; in TRT+aB shell cells (Sec. 2.3.2)
//   and for Lambda_b,bulk != 1 the two bulk moments m4, m5 relax with s_b
//   (Eq. (12)) through a rank-2 correction in moment space.
//
// PDFs are stored shifted (f_q - w_q) in SoA layout f[q][z][y][x], read from
// one buffer and written to the other.
//
// Per-particle sums. Float64 storage: float64 partial sums per warp, float64
// atomics. Float32 compute: the link force is split into the constant part
// 2 w_p c_p, which is an integer multiple of c_p / 36, and the small
// remainder c_p (f~_p + f_q) - u_b (f~_p - f_q). The constant part and its
// torque 2 w_p (n + g) x c_p (n the integer cell offset from the particle's
// base cell, g its fractional offset, common to all links) are summed exactly
// in integers; the remainder is summed per warp in float32 and per particle
// in 64-bit fixed point (scale 2^32) through integer atomics. No float64
// instruction runs per cell on the float32 path.
#include "common.cuh"
#include "launch.h"

// minimum resident blocks per SM requested for the stream/collide kernel
// (a register cap); tuned on GB300, see the design notes
#ifndef LBM_SC_MIN_BLOCKS
#define LBM_SC_MIN_BLOCKS 4
#endif
// the same for the boundary kernel
#ifndef LBM_BC_MIN_BLOCKS
#define LBM_BC_MIN_BLOCKS 4
#endif
// cache policy of the dense kernel: 0 default loads and stores, 1 streaming
// (evict-first) stores, 2 streaming loads and stores
#ifndef LBM_SC_HINTS
#define LBM_SC_HINTS 0
#endif

namespace lbmdem {

template <typename S>
struct BcArgs {
    S* src;                          // written only in solid-cell slots
    const uint8_t* __restrict__ flags;
    const int* __restrict__ owner;
    Geom g;
    const unsigned int* __restrict__ list;   // fluid cells with possible particle links
    const int* count;
    int cap;
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

template <typename S, typename T>
struct SCArgs {
    const S* __restrict__ src;
    S* __restrict__ dst;
    const uint8_t* __restrict__ flags;
    Geom g;
    T s_plus, s_minus, s_b_shell, s_b_bulk;
    T uw[2][3][3];                   // wall velocities [side][axis][component]
    int bulk_corr;
    const T* __restrict__ accel;     // [3]
    int* status;
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

// ------------------------------------------------------------------ boundary kernel

// CLI condition and momentum exchange of one particle link: fluid cell
// (x, y, z), pull direction q, solid upstream cell x - c_q
template <typename S, typename T>
__device__ __forceinline__ void particle_link(const BcArgs<S>& a, int x, int y, int z, int q, Acc<T>& acc,
                                              const Sinks& sk) {
    const int nx = a.g.n[0], ny = a.g.n[1];
    const int plane = nx * ny;
    const long long N = a.g.ncells;
    const int c[3] = {k_c[q][0], k_c[q][1], k_c[q][2]};
    const int p = k_opp[q];
    const int cpos[3] = {x, y, z};
    int uv[3], dv[3];
    bool cli = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        uv[d] = wrap_idx(cpos[d] - c[d], a.g.n[d]);
        dv[d] = cpos[d] + c[d];
        if (!a.g.per[d] && (dv[d] < 0 || dv[d] >= a.g.n[d])) cli = false;
        dv[d] = wrap_idx(dv[d], a.g.n[d]);
    }
    const int idx = z * plane + y * nx + x;
    const int up = uv[2] * plane + uv[1] * nx + uv[0];
    const int down = dv[2] * plane + dv[1] * nx + dv[0];
    const int i = a.owner[up];
    const T fout = Store<S>::load(a.src + p * N + idx);
    const T fin = Store<S>::load(a.src + q * N + idx);
    if (cli) cli = !(a.flags[down] & FL_SOLID);
    const T fdown = cli ? Store<S>::load(a.src + p * N + down) : T(0);
    T r[3], R, u[3], om[3];
    int n[3];
    PartOps<T>::load(a, i, x, y, z, r, n, R, u, om);
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
    int K[6] = {0, 0, 0, 0, 0, 0};
    T sum;
    if (sizeof(T) == 4) {
        // 2 w_p c_p and its torque 2 w_p (n x c_p) as exact integers (x 36)
        const int kw = cc2 == 1 ? 4 : 2;
        sum = fout + v;
        K[0] = kw * cp[0]; K[1] = kw * cp[1]; K[2] = kw * cp[2];
        K[3] = kw * (n[1] * cp[2] - n[2] * cp[1]);
        K[4] = kw * (n[2] * cp[0] - n[0] * cp[2]);
        K[5] = kw * (n[0] * cp[1] - n[1] * cp[0]);
    } else {
        sum = T(2) * w + fout + v;
    }
    const T F[3] = {cp0 * sum - ub[0] * dif, cp1 * sum - ub[1] * dif, cp2 * sum - ub[2] * dif};
    const T Tq[3] = {rb[1] * F[2] - rb[2] * F[1], rb[2] * F[0] - rb[0] * F[2], rb[0] * F[1] - rb[1] * F[0]};
    accumulate<T>(i, F, Tq, K, acc, sk);
}

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

template <typename S>
__global__ void __launch_bounds__(256, LBM_BC_MIN_BLOCKS) boundary_kernel(const BcArgs<S> a) {
    using T = typename Store<S>::T;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const Sinks sk{a.acc_d, a.acc_i, a.acc_k, a.status};
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
    const int nx = a.g.n[0], ny = a.g.n[1];
    const int plane = nx * ny;
    const int stride = gridDim.x * blockDim.x;

    // ------------------------------------------- particle links of fluid cells
    const int count = min(*a.count, a.cap);
    for (int base = blockIdx.x * blockDim.x; base < count; base += stride) {
        const int k = base + threadIdx.x;
        Acc<T> acc;
        unsigned mask = 0;          // directions with a solid upstream cell
        int x = 0, y = 0, z = 0;
        if (k < count) {
            const int idx = (int)a.list[k];
            z = idx / plane;
            const int rem = idx - z * plane;
            y = rem / nx;
            x = rem - y * nx;
#pragma unroll
            for (int q = 1; q < Q; ++q) {
                int v[3] = {x - cx(q), y - cy(q), z - cz(q)};
                bool outside = false;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (!a.g.per[d] && (v[d] < 0 || v[d] >= a.g.n[d])) outside = true;
                    v[d] = wrap_idx(v[d], a.g.n[d]);
                }
                if (!outside && (a.flags[v[2] * plane + v[1] * nx + v[0]] & FL_SOLID))
                    mask |= 1u << q;
            }
        }
        // the warp's links in direction-major order: for q = 1..18 the cells
        // with a link in direction q, in lane order, packed 32 links to a
        // round, so that the lanes of a round mostly read and write
        // neighbouring cells of the same PDF arrays
        const int total = __reduce_add_sync(FULL, __popc(mask));
        int q = 1, done = 0;
        unsigned bal = __ballot_sync(FULL, (mask >> 1) & 1u);
        int cnt = __popc(bal);
        for (int r0 = 0; r0 < total; r0 += 32) {
            int my_q = 0, my_src = 0, filled = 0;
            while (filled < 32 && q < Q) {   // warp-uniform
                const int take = min(cnt - done, 32 - filled);
                const int j = lane - filled;
                if (j >= 0 && j < take) {
                    my_q = q;
                    my_src = (int)__fns(bal, 0, done + j + 1);
                }
                filled += take;
                done += take;
                if (done == cnt) {
                    ++q;
                    done = 0;
                    bal = __ballot_sync(FULL, q < Q ? (mask >> q) & 1u : 0u);
                    cnt = __popc(bal);
                }
            }
            const int sx = __shfl_sync(FULL, x, my_src);
            const int sy = __shfl_sync(FULL, y, my_src);
            const int sz = __shfl_sync(FULL, z, my_src);
            if (my_q) particle_link<S, T>(a, sx, sy, sz, my_q, acc, sk);
        }
        commit<T>(acc, sk);
    }

    // ------------------------------------------- missing links (Sec. 2.2)
    if (!a.missing_links) return;
    const int mcount = min(*a.miss_count, a.miss_cap);
    for (int base = blockIdx.x * blockDim.x; base < mcount; base += stride) {
        const int k = base + threadIdx.x;
        Acc<T> acc;
        if (k < mcount) missing_links<S, T>(a, (long long)a.miss[k], acc, sk);
        commit<T>(acc, sk);
    }
}

// ------------------------------------------------------------------ stream + collide

// loads and stores of the dense kernel with the cache policy LBM_SC_HINTS
template <typename S>
__device__ __forceinline__ typename Store<S>::T sc_load(const S* p) {
#if LBM_SC_HINTS >= 2
    if constexpr (sizeof(S) == 8) return (typename Store<S>::T)__ldcs(reinterpret_cast<const double*>(p));
    else if constexpr (sizeof(S) == 4) return (typename Store<S>::T)__ldcs(reinterpret_cast<const float*>(p));
    else return Store<S>::load(p);
#else
    return Store<S>::load(p);
#endif
}
template <typename S>
__device__ __forceinline__ void sc_store(S* p, typename Store<S>::T v) {
#if LBM_SC_HINTS >= 1
    if constexpr (sizeof(S) == 8) __stcs(reinterpret_cast<double*>(p), (double)v);
    else if constexpr (sizeof(S) == 4) __stcs(reinterpret_cast<float*>(p), (float)v);
    else Store<S>::store(p, v);
#else
    Store<S>::store(p, v);
#endif
}

// Cell indices are 32-bit (the library limits boxes to fewer than 2^31
// cells); each PDF array q starts at the uniform pointer src + q N.
template <typename S, typename T>
__global__ void __launch_bounds__(256, LBM_SC_MIN_BLOCKS) stream_collide_kernel(const SCArgs<S, T> a) {
    const int nx = a.g.n[0], ny = a.g.n[1], nz = a.g.n[2];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    const bool valid = x < nx && y < ny;
    const int plane = nx * ny;
    const long long N = a.g.ncells;
    const int idx = z * plane + y * nx + x;
    const uint8_t fl = valid ? a.flags[idx] : FL_SOLID;
    const bool fluid = !(fl & FL_SOLID);
    // Solid cells that share a 32-byte sector with fluid cells also write
    // (zeros; solid slots are never read before the boundary kernel rewrites
    // them), so every written sector is complete and L2 needs no fill read.
    constexpr int G = 32 / (int)sizeof(S);
    const unsigned bal = __ballot_sync(0xffffffffu, fluid && valid);
    const int lane = threadIdx.x & 31;
    const unsigned gmask = (G >= 32 ? 0xffffffffu : ((1u << G) - 1u)) << (lane & ~(G - 1));

    if (!fluid) {
        if (valid && (bal & gmask)) {
#pragma unroll
            for (int q = 0; q < Q; ++q) sc_store<S>(a.dst + q * N + idx, T(0));
        }
        return;
    }
    {
        // neighbour offsets with periodic wrap (walls are handled below)
        const int OX[3] = {x == 0 ? nx - 1 : -1, 0, x == nx - 1 ? 1 - nx : 1};
        const int OY[3] = {y == 0 ? plane - nx : -nx, 0, y == ny - 1 ? nx - plane : nx};
        const int OZ[3] = {z == 0 ? (nz - 1) * plane : -plane, 0, z == nz - 1 ? (1 - nz) * plane : plane};
        T f[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q)
            f[q] = sc_load<S>(a.src + q * N + (idx + OX[1 - cx(q)] + OY[1 - cy(q)] + OZ[1 - cz(q)]));
        // halfway bounce-back on the box walls (Eq. (14) with delta = 1/2)
        const bool wx = !a.g.per[0] && (x == 0 || x == nx - 1);
        const bool wy = !a.g.per[1] && (y == 0 || y == ny - 1);
        const bool wz = !a.g.per[2] && (z == 0 || z == nz - 1);
        if (wx || wy || wz) {
#pragma unroll
            for (int q = 1; q < Q; ++q) {
                const int u0 = x - cx(q), u1 = y - cy(q), u2 = z - cz(q);
                int axis = -1, side = 0;
                if (wz && (u2 < 0 || u2 >= nz)) { axis = 2; side = u2 < 0 ? 0 : 1; }
                else if (wy && (u1 < 0 || u1 >= ny)) { axis = 1; side = u1 < 0 ? 0 : 1; }
                else if (wx && (u0 < 0 || u0 >= nx)) { axis = 0; side = u0 < 0 ? 0 : 1; }
                if (axis < 0) continue;
                const int p = opp(q);
                const T ucp = a.uw[side][axis][0] * (T)(-cx(q)) + a.uw[side][axis][1] * (T)(-cy(q)) +
                              a.uw[side][axis][2] * (T)(-cz(q));
                f[q] = Store<S>::load(a.src + p * N + idx) - T(6) * wq<T>(p) * ucp;
            }
        }

        // ------------------------------------------- TRT+aB collision (in place)
        T drho = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            drho += f[q];
            if (cx(q)) jx += cx(q) > 0 ? f[q] : -f[q];
            if (cy(q)) jy += cy(q) > 0 ? f[q] : -f[q];
            if (cz(q)) jz += cz(q) > 0 ? f[q] : -f[q];
        }
        const T ax = a.accel[0], ay = a.accel[1], az = a.accel[2];
        const T ux = jx + T(0.5) * ax, uy = jy + T(0.5) * ay, uz = jz + T(0.5) * az;
        const T usq = ux * ux + uy * uy + uz * uz;
        const T ua = ux * ax + uy * ay + uz * az;
        const T sp = a.s_plus, sm = a.s_minus;
        const T gp = T(1) - T(0.5) * sp, gm = T(1) - T(0.5) * sm;
        // bulk moments m4 = sum (c^2 - 1) f and m5 (row 6 of M) of the streamed
        // PDFs relax with s_b in shell cells (and everywhere when Lambda_b,bulk != 1)
        const bool shell = (fl & FL_SHELL) != 0;
        const bool bulk = shell || a.bulk_corr;
        T k4 = T(0), k5 = T(0);
        if (bulk) {
            const T ds = (shell ? a.s_b_shell : a.s_b_bulk) - sp;
            T saxis = T(0), sdiag = T(0);
#pragma unroll
            for (int q = 1; q < Q; ++q) {
                if (c2(q) == 1) saxis += f[q]; else sdiag += f[q];
            }
            const T m4 = -f[0] + sdiag;
            const T m5 = f[0] - T(2) * saxis + sdiag;
            // M^-1 e_k = w_q M_kq / (sum_q w_q M_kq^2): norms 2/3 (row 4) and 2 (row 5)
            k4 = T(1.5) * (ds * ((usq - m4) - ua));
            k5 = T(0.5) * (ds * (-m5));
        }
        {
            const T w0 = wq<T>(0);
            const T feq0 = w0 * (drho - T(1.5) * usq);
            f[0] = f[0] - sp * (f[0] - feq0) + gp * (w0 * (T(-3) * ua)) + w0 * (k5 - k4);
        }
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            const int qb = opp(q);
            if (qb < q) continue;
            const T w = wq<T>(q);
            const T cu = (T)cx(q) * ux + (T)cy(q) * uy + (T)cz(q) * uz;
            const T ca = (T)cx(q) * ax + (T)cy(q) * ay + (T)cz(q) * az;
            const T ep = w * (drho + T(4.5) * cu * cu - T(1.5) * usq);
            const T em = w * (T(3) * cu);
            const T Fp = w * (T(-3) * ua + T(9) * cu * ca);
            const T Fm = w * (T(3) * ca);
            const T fp = T(0.5) * (f[q] + f[qb]);
            const T fm = T(0.5) * (f[q] - f[qb]);
            const T corr = c2(q) == 1 ? w * (T(-2) * k5) : w * (k4 + k5);
            const T dp = -sp * (fp - ep) + gp * Fp + corr;
            const T dm = -sm * (fm - em) + gm * Fm;
            f[q] = f[q] + dp + dm;
            f[qb] = f[qb] + dp - dm;
        }
        if (!(drho < T(0.5) && drho > T(-0.5))) atomicOr(a.status, ST_UNSTABLE);
#pragma unroll
        for (int q = 0; q < Q; ++q) sc_store<S>(a.dst + q * N + idx, f[q]);
    }
}

template <typename S>
void launch_boundary_t(const LbmStepParams& p, cudaStream_t st) {
    BcArgs<S> b;
    b.src = static_cast<S*>(const_cast<void*>(p.src));
    b.flags = p.flags;
    b.owner = p.owner;
    b.g = p.g;
    b.list = p.near_list;
    b.count = p.near_count;
    b.cap = p.near_cap;
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
    const int bblocks = p.near_blocks > 0 ? p.near_blocks : 1;
    boundary_kernel<S><<<bblocks, 256, 0, st>>>(b);
}

template <typename S>
void launch_stream_collide_t(const LbmStepParams& p, cudaStream_t st) {
    using T = typename Store<S>::T;
    SCArgs<S, T> a;
    a.src = static_cast<const S*>(p.src);
    a.dst = static_cast<S*>(p.dst);
    a.flags = p.flags;
    a.g = p.g;
    a.s_plus = (T)p.s_plus;
    a.s_minus = (T)p.s_minus;
    a.s_b_shell = (T)p.s_b_shell;
    a.s_b_bulk = (T)p.s_b_bulk;
    for (int s = 0; s < 2; ++s)
        for (int ax = 0; ax < 3; ++ax)
            for (int c = 0; c < 3; ++c) a.uw[s][ax][c] = (T)p.g.wall_vel[s][ax][c];
    a.bulk_corr = p.bulk_corr;
    a.accel = reinterpret_cast<const T*>(sizeof(T) == 8 ? (const void*)p.accel_d : (const void*)p.accel_f);
    a.status = p.status;
    const int nx = p.g.n[0];
    int bx = nx >= 128 ? 128 : ((nx + 31) / 32) * 32;
    int by = 256 / bx;
    dim3 block(bx, by, 1);
    dim3 grid((nx + bx - 1) / bx, (p.g.n[1] + by - 1) / by, p.g.n[2]);
    stream_collide_kernel<S, T><<<grid, block, 0, st>>>(a);
}

void launch_boundary(const LbmStepParams& p, cudaStream_t st) {
    switch (p.storage) {
        case 0: launch_boundary_t<double>(p, st); break;
        case 1: launch_boundary_t<float>(p, st); break;
        case 2: launch_boundary_t<__half>(p, st); break;
        default: launch_boundary_t<__nv_bfloat16>(p, st); break;
    }
}

void launch_stream_collide(const LbmStepParams& p, cudaStream_t st) {
    switch (p.storage) {
        case 0: launch_stream_collide_t<double>(p, st); break;
        case 1: launch_stream_collide_t<float>(p, st); break;
        case 2: launch_stream_collide_t<__half>(p, st); break;
        default: launch_stream_collide_t<__nv_bfloat16>(p, st); break;
    }
}

}  // namespace lbmdem
