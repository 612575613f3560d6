// sc_common.cuh -- arithmetic shared by the dense stream/collide kernels:
// the CLI moving no-slip value of one particle link with its momentum-exchange
// force and torque (Eqs. (14)-(17)), and the TRT(+aB) collision with Guo
// forcing of one fluid cell and the store of its PDFs (Eqs. (5), (10)-(12),
// Sec. 2.3.2). See stream_collide.cu for the data layout.
#pragma once

#include "common.cuh"
#include "launch.h"
#include "links.cuh"

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
    int zchunk;                      // z planes per block
    int bx;                          // x extent of a block's tile (a multiple of 32; 256 / bx rows)
    // particles (for the links)
    int np;
    const int* __restrict__ owner;   // particle of a solid cell, -1 for fluid
    const double* __restrict__ px;
    const double* __restrict__ pu;
    const double* __restrict__ pom;
    const double* __restrict__ pR;
    const PartView* __restrict__ view;
    double* acc_d;
    long long* acc_i;
    long long* acc_k;
};

// kernel arguments from the step parameters
template <typename S, typename T>
void fill_sc_args(const LbmStepParams& p, SCArgs<S, T>& a) {
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
    a.zchunk = 0;
    a.bx = 128;
    a.np = p.P.n;
    a.owner = p.owner;
    a.px = p.P.x;
    a.pu = p.P.u;
    a.pom = p.P.om;
    a.pR = p.P.R;
    a.view = p.P.view;
    a.acc_d = p.P.acc_d;
    a.acc_i = p.P.acc_i;
    a.acc_k = p.P.acc_k;
}

// NaN marker of a solid cell of particle owner, and a plain NaN
template <typename T>
__device__ __forceinline__ T solid_marker(int owner);
template <> __device__ __forceinline__ float solid_marker<float>(int owner) { return __uint_as_float(marker_bits32(owner)); }
template <> __device__ __forceinline__ double solid_marker<double>(int owner) {
    return __longlong_as_double((long long)marker_bits64(owner));
}
template <typename T>
__device__ __forceinline__ T plain_nan() { return solid_marker<T>(MARKER_PAYLOAD - 1); }

// CLI value f_q(x, t+1) of the link of fluid cell (x, y, z) in pull direction
// q into the solid cell x - c_q, and its force and torque into acc (float32
// path: the remainder part in floats, the constant part as exact integers)
// per-direction word of the link code: c_q + 1 in bits 0-1, 2-3, 4-5, the
// opposite direction in bits 6-10 (read from shared memory: a warp's lanes
// hold different directions)
__host__ __device__ constexpr int qinfo(int q) { return (cx(q) + 1) | ((cy(q) + 1) << 2) | ((cz(q) + 1) << 4) | (opp(q) << 6); }

template <typename S, typename T>
__device__ __forceinline__ T link_value(const SCArgs<S, T>& a, int x, int y, int z, int q, int qi, int key1,
                                        unsigned lm_src, T fdown_raw, Acc<T>& acc, const Sinks& sk) {
    const int nx = a.g.n[0], ny = a.g.n[1];
    const int plane = nx * ny;
    const long long N = a.g.ncells;
    const int c[3] = {(qi & 3) - 1, ((qi >> 2) & 3) - 1, ((qi >> 4) & 3) - 1};
    const int p = (qi >> 6) & 31;
    const int idx = z * plane + y * nx + x;
    // the particle from the marker's payload (the owner array for 16-bit storage)
    int i = key1 - 1;
    if (key1 <= 0) {
        const int uv[3] = {wrap_idx(x - c[0], nx), wrap_idx(y - c[1], ny), wrap_idx(z - c[2], a.g.n[2])};
        i = a.owner[uv[2] * plane + uv[1] * nx + uv[0]];
    }
    if (i < 0 || i >= a.np) return plain_nan<T>();   // a NaN from a fluid cell: left for the stability check
    const T fout = Store<S>::load(a.src + p * N + idx);
    const T fin = Store<S>::load(a.src + q * N + idx);
    // CLI needs x + c_q fluid and inside the box; its post-collision f_p is the
    // cell's own pull in direction p (marker there: bounce-back coefficients)
    bool cli = !((lm_src >> p) & 1u);
    if (!a.g.per[0] && (x + c[0] < 0 || x + c[0] >= nx)) cli = false;
    if (!a.g.per[1] && (y + c[1] < 0 || y + c[1] >= ny)) cli = false;
    if (!a.g.per[2] && (z + c[2] < 0 || z + c[2] >= a.g.n[2])) cli = false;
    const T fdown = cli ? fdown_raw : T(0);
    T r[3], R, u[3], om[3];
    int n[3];
    T cc;   // |r|^2 - R^2
    if constexpr (sizeof(T) == 4) {
        float g[3], C[2];
        PartOps<T>::load(a, i, x, y, z, r, n, g, C, R, u, om);
        cc = surface_cc_split(n, g, C);
    } else {
        PartOps<T>::load(a, i, x, y, z, r, n, R, u, om);
        cc = surface_cc<T>(r, R);
    }
    const int cp[3] = {-c[0], -c[1], -c[2]};
    const T cp0 = (T)cp[0], cp1 = (T)cp[1], cp2 = (T)cp[2];
    const int cc2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    const T w = cc2 == 1 ? T(1) / T(18) : T(1) / T(36);
    const T delta = link_root<T>(r, cc, cp0, cp1, cp2, (T)cc2);
    const T dbc = cli ? delta : T(0.5);
    const T inv = fast_div(T(1), T(1) + T(2) * dbc);
    const T kappa = (T(1) - T(2) * dbc) * inv;
    const T rb[3] = {r[0] + delta * cp0, r[1] + delta * cp1, r[2] + delta * cp2};
    const T ub[3] = {u[0] + (om[1] * rb[2] - om[2] * rb[1]), u[1] + (om[2] * rb[0] - om[0] * rb[2]),
                     u[2] + (om[0] * rb[1] - om[1] * rb[0])};
    const T ubc = ub[0] * cp0 + ub[1] * cp1 + ub[2] * cp2;
    const T v = fout + kappa * (fdown - fin) - (T(12) * w * inv) * ubc;
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
    return v;
}

// TRT+aB collision of one fluid cell, in place, with the body force (ax, ay,
// az); returns false when the density deviation of the streamed PDFs leaves
// (-0.5, 0.5) or is NaN. The arithmetic is that of the moment-space update
// with S of Eq. (12) written per pair of opposite directions (q, qbar): with
// s = f_q + f_qbar and d = f_q - f_qbar the even part relaxes with s_nu and
// the odd part with s_nu^- (Eq. (10)),
//   dp = -s_nu (s/2 - w X) + (1 - s_nu/2) w Y + corr,   X = drho - 3/2 u^2 + 9/2 (c.u)^2
//   dm = -s_nu^- (d/2 - 3 w c.u) + (1 - s_nu^-/2) 3 w c.a, Y = -3 u.a + 9 (c.u)(c.a)
//   f_q += dp + dm,  f_qbar += dp - dm,
// the Guo source in Y and 3 w c.a; corr is the rank-2 bulk correction of the
// shell cells. Each pair costs one chain of fused multiply-adds.
template <typename T>
__device__ __forceinline__ bool collide_core(T (&f)[Q], uint8_t fl, T ax, T ay, T az, T sp, T sm, T s_b_shell,
                                             T s_b_bulk, int bulk_corr) {
    T sq[Q], dq[Q];   // pair sums and differences, entries q < opp(q) only
    T drho = f[0], jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const int qb = opp(q);
        if (qb < q) continue;
        sq[q] = f[q] + f[qb];
        dq[q] = f[q] - f[qb];
        drho += sq[q];
        if (cx(q)) jx += cx(q) > 0 ? dq[q] : -dq[q];
        if (cy(q)) jy += cy(q) > 0 ? dq[q] : -dq[q];
        if (cz(q)) jz += cz(q) > 0 ? dq[q] : -dq[q];
    }
    const T ux = jx + T(0.5) * ax, uy = jy + T(0.5) * ay, uz = jz + T(0.5) * az;
    const T usq = ux * ux + uy * uy + uz * uz;
    const T ua = ux * ax + uy * ay + uz * az;
    const T gp = T(1) - T(0.5) * sp, gm = T(1) - T(0.5) * sm;
    // bulk moments m4 = sum (c^2 - 1) f and m5 (row 6 of M) of the streamed
    // PDFs relax with s_b in shell cells (and everywhere when Lambda_b,bulk != 1)
    const bool shell = (fl & FL_SHELL) != 0;
    const bool bulk = shell || bulk_corr;
    T k4 = T(0), k5 = T(0);
    if (bulk) {
        const T ds = (shell ? s_b_shell : s_b_bulk) - sp;
        T saxis = T(0), sdiag = T(0);
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            if (opp(q) < q) continue;
            if (c2(q) == 1) saxis += sq[q]; else sdiag += sq[q];
        }
        const T m4 = -f[0] + sdiag;
        const T m5 = f[0] - T(2) * saxis + sdiag;
        // M^-1 e_k = w_q M_kq / (sum_q w_q M_kq^2): norms 2/3 (row 4) and 2 (row 5)
        k4 = T(1.5) * (ds * ((usq - m4) - ua));
        k5 = T(0.5) * (ds * (-m5));
    }
    const T drp = drho - T(1.5) * usq;
    const T m3ua = T(-3) * ua;
    // Weights of the update: w2 = 2 w (even parts), w6 = 6 w (odd parts) per
    // class (axis, diagonal) and w0. In float32 they are chosen within 1.2e-7
    // of the exact fractions such that w0 + 3 w2_axis + 6 w2_diag = 1 and
    // w6_axis + 4 w6_diag = 1 hold exactly: the relaxation towards the
    // equilibrium then keeps the mass and momentum of every cell, where the
    // plain roundings of 1/18, 1/36 and 1/3 would leave a steady source of
    // relative size 3e-8 per step that builds up over a long run.
    const T w2d = sizeof(T) == 4 ? T(0.0555555522441864) : T(1) / T(18);
    const T w2a = T(2) * w2d;
    const T w0 = T(1) - T(12) * w2d;
    const T w6d = T(1) / T(6);
    const T w6a = T(1) - T(4) * w6d;
    {
        f[0] = f[0] + sp * (w0 * drp - f[0]) + gp * (w0 * m3ua) + w0 * (k5 - k4);
    }
    const T hsp = T(-0.5) * sp, hsm = T(-0.5) * sm;
    // per weight class (axis, diagonal); each part relaxes as rate x (value
    // - its equilibrium)
    const T w2[2] = {w2a, w2d}, w6[2] = {w6a, w6d};
    const T gpw[2] = {T(0.5) * gp * w2a, T(0.5) * gp * w2d}, gmw3[2] = {T(0.5) * gm * w6a, T(0.5) * gm * w6d};
    const T corr[2] = {-w2a * k5, T(0.5) * w2d * (k4 + k5)};
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const int qb = opp(q);
        if (qb < q) continue;
        const int k = c2(q) == 1 ? 0 : 1;
        T cu = T(0), ca = T(0);
        if (cx(q)) { cu += cx(q) > 0 ? ux : -ux; ca += cx(q) > 0 ? ax : -ax; }
        if (cy(q)) { cu += cy(q) > 0 ? uy : -uy; ca += cy(q) > 0 ? ay : -ay; }
        if (cz(q)) { cu += cz(q) > 0 ? uz : -uz; ca += cz(q) > 0 ? az : -az; }
        const T X = fma_t<T>(T(4.5) * cu, cu, drp);
        const T Y = fma_t<T>(T(9) * cu, ca, m3ua);
        const T dp = fma_t<T>(hsp, fma_t<T>(-w2[k], X, sq[q]), fma_t<T>(gpw[k], Y, corr[k]));
        const T dm = fma_t<T>(hsm, fma_t<T>(-w6[k], cu, dq[q]), gmw3[k] * ca);
        f[q] = f[q] + (dp + dm);
        f[qb] = f[qb] + (dp - dm);
    }
    return drho < T(0.5) && drho > T(-0.5);
}

template <typename S, typename T>
__device__ __forceinline__ bool collide_cell_a(const SCArgs<S, T>& a, T (&f)[Q], uint8_t fl, T ax, T ay, T az) {
    return collide_core<T>(f, fl, ax, ay, az, a.s_plus, a.s_minus, a.s_b_shell, a.s_b_bulk, a.bulk_corr);
}

template <typename S, typename T>
__device__ __forceinline__ bool collide_cell(const SCArgs<S, T>& a, T (&f)[Q], uint8_t fl) {
    return collide_cell_a<S, T>(a, f, fl, a.accel[0], a.accel[1], a.accel[2]);
}

// collision of one fluid cell and the store of its PDFs
template <typename S, typename T>
__device__ __forceinline__ void collide_store(const SCArgs<S, T>& a, T (&f)[Q], uint8_t fl, long long N, int idx) {
    if (!collide_cell<S, T>(a, f, fl)) atomicOr(a.status, ST_UNSTABLE);
#pragma unroll
    for (int q = 0; q < Q; ++q) Store<S>::store(a.dst + q * N + idx, f[q]);
}


}  // namespace lbmdem
