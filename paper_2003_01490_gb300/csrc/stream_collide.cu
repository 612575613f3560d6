// stream_collide.cu -- the dense kernel of one lattice Boltzmann step
// (Algorithm 1, lines 2-3): one thread per cell, pull streaming (Eq. (2)) with
// halfway bounce-back on the walls of the box (Eq. (14), delta = 1/2, wall
// velocity), then the two-relaxation-time collision (Eq. (10), magic
// parameter Eq. (11)) with Guo forcing; in TRT+aB shell cells (Sec. 2.3.2) and
// for Lambda_b,bulk != 1 the two bulk moments m4, m5 relax with s_b (Eq. (12))
// through a rank-2 correction in moment space.
//
// PDFs are stored shifted (f_q - w_q) in SoA layout f[q][z][y][x], read from
// one buffer and written to the other. Particle links need no logic here: the
// boundary kernel has already written their CLI values into the solid-cell
// slots that the pull of a fluid cell reads.
#include "common.cuh"
#include "launch.h"

// minimum resident blocks per SM requested for the kernel with 4-byte or
// smaller storage (a register cap of 64 at 256 threads); tuned on GB300
#ifndef LBM_SC_MIN_BLOCKS
#define LBM_SC_MIN_BLOCKS 4
#endif
// cache policy: 0 default loads and stores, 1 streaming (evict-first) stores,
// 2 streaming loads and stores
#ifndef LBM_SC_HINTS
#define LBM_SC_HINTS 0
#endif

namespace lbmdem {

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
__global__ void __launch_bounds__(256, sizeof(S) == 8 ? 1 : LBM_SC_MIN_BLOCKS) stream_collide_kernel(const SCArgs<S, T> a) {
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

void launch_stream_collide(const LbmStepParams& p, cudaStream_t st) {
    switch (p.storage) {
        case 0: launch_stream_collide_t<double>(p, st); break;
        case 1: launch_stream_collide_t<float>(p, st); break;
        case 2: launch_stream_collide_t<__half>(p, st); break;
        default: launch_stream_collide_t<__nv_bfloat16>(p, st); break;
    }
}


}  // namespace lbmdem
