// boundary.cu -- the first kernel of one lattice Boltzmann step with moving
// particles: the fluid body force of the step and the missing-link
// correction (Sec. 2.2).
//
// Thread 0 of block 0 forms the fluid body force a_user - ext_total / N_fluid
// (the counter force of a periodic suspension, N_fluid from the last mapping)
// that the dense kernel and the refill use (mode BC_ACCEL). The other work
// (mode BC_LINKS, launched beside the dense kernel on a second stream) walks the
// missing-link list of the mapping (solid cells next to another body): a link
// x -> s into a solid cell s of particle i is missing when x belongs to
// another body (or lies behind a wall) and its centre is not inside sphere i;
// each adds F_q = 2 w_q c_q with its torque, reduced per warp by particle and
// added atomically (64-bit fixed point on the float32 path, float64 atomics
// on the float64 path).
//
// The particle links themselves (CLI condition of Eq. (14), momentum exchange
// of Eq. (15)) are handled inside the dense stream/collide kernel, which finds
// them from the marker that solid cells hold in their PDF slots.
#include <cstring>

#include "common.cuh"
#include "gang.cuh"
#include "launch.h"
#include "links.cuh"

namespace lbmdem {

template <typename S>
struct BcArgs {
    const uint8_t* __restrict__ flags;
    const int* __restrict__ owner;   // particle of a solid cell, -1 for fluid
    Geom g;
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

// mode BC_ACCEL: one thread forms the fluid body force of the step; mode
// BC_LINKS: the missing-link terms 2 w_q c_q of Sec. 2.2 and their torques, one
// thread per listed solid cell, committed per warp
// (block bx of a grid of gx blocks)
template <typename S>
__device__ __forceinline__ void boundary_body(const BcArgs<S>& a, int mode, int bx, int gx) {
    using T = typename Store<S>::T;
    if ((mode & BC_ACCEL) && bx == 0 && threadIdx.x == 0) {
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
    if (!(mode & BC_LINKS) || !a.missing_links) return;
    const Sinks sk{a.acc_d, a.acc_i, a.acc_k, a.status};
    const int mcount = min(*a.miss_count, a.miss_cap);
    const int stride = (int)(gx * blockDim.x);
    for (int base = (int)(bx * blockDim.x); base < mcount; base += stride) {
        const int k = base + threadIdx.x;
        Acc<T> acc;
        if (k < mcount) missing_links<S, T>(a, (long long)a.miss[k], acc, sk);
        commit<T>(acc, sk);
    }
}

template <typename S>
__global__ void __launch_bounds__(128) boundary_kernel(const BcArgs<S> a, int mode) {
    boundary_body<S>(a, mode, (int)blockIdx.x, (int)gridDim.x);
}

template <typename S>
__global__ void __launch_bounds__(128) boundary_gang_kernel(const BcArgs<S>* __restrict__ table,
                                                            const int* __restrict__ off, int n, int mode) {
    __shared__ __align__(16) BcArgs<S> a;
    const int i = gang_instance(off, n, (int)blockIdx.x);
    gang_load(table, i, a);
    boundary_body<S>(a, mode, (int)blockIdx.x - off[i], off[i + 1] - off[i]);
}

template <typename S>
void fill_bc_args_t(const LbmStepParams& p, BcArgs<S>& b) {
    b.flags = p.flags;
    b.owner = p.owner;
    b.g = p.g;
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
}

template <typename S>
void launch_boundary_t(const LbmStepParams& p, cudaStream_t st, int mode) {
    BcArgs<S> b;
    fill_bc_args_t<S>(p, b);
    const int blocks = (mode & BC_LINKS) && p.missing_links ? 8 * (p.num_sms > 0 ? p.num_sms : 1) : 1;
    boundary_kernel<S><<<blocks, 128, 0, st>>>(b, mode);
}

size_t bc_args_bytes() { return sizeof(BcArgs<float>); }

void fill_bc_args(const LbmStepParams& p, void* out) {
    // the argument block does not depend on the storage format
    static_assert(sizeof(BcArgs<float>) == sizeof(BcArgs<double>), "one layout for all formats");
    BcArgs<float> b;
    std::memset(&b, 0, sizeof(b));
    fill_bc_args_t<float>(p, b);
    std::memcpy(out, &b, sizeof(b));
}

void launch_boundary_gang(int storage, const void* table, const int* off, int n, int blocks, int mode,
                          cudaStream_t st) {
    if (n <= 0 || blocks <= 0) return;
    switch (storage) {
        case 0: boundary_gang_kernel<double><<<blocks, 128, 0, st>>>(static_cast<const BcArgs<double>*>(table), off, n, mode); break;
        case 1: boundary_gang_kernel<float><<<blocks, 128, 0, st>>>(static_cast<const BcArgs<float>*>(table), off, n, mode); break;
        case 2: boundary_gang_kernel<__half><<<blocks, 128, 0, st>>>(static_cast<const BcArgs<__half>*>(table), off, n, mode); break;
        default: boundary_gang_kernel<__nv_bfloat16><<<blocks, 128, 0, st>>>(static_cast<const BcArgs<__nv_bfloat16>*>(table), off, n, mode); break;
    }
}

void launch_boundary(const LbmStepParams& p, cudaStream_t st, int mode) {
    switch (p.storage) {
        case 0: launch_boundary_t<double>(p, st, mode); break;
        case 1: launch_boundary_t<float>(p, st, mode); break;
        case 2: launch_boundary_t<__half>(p, st, mode); break;
        default: launch_boundary_t<__nv_bfloat16>(p, st, mode); break;
    }
}

}  // namespace lbmdem
