// dem.cu -- particle side of Algorithm 1 in float64: force finalisation and
// two-step averaging of the momentum-exchange force (Sec. 4.2), neighbour
// search, lubrication correction (Eqs. (25)-(33)), linear spring-dashpot
// contact with Coulomb-limited tangential spring (Eqs. (39)-(52)) and the
// Velocity-Verlet subcycles (Eqs. (37)-(38)).
//
// One thread per particle gathers every interaction of its particle, so no
// force atomics are needed; a pair is evaluated by both partners with exactly
// mirrored operands (n_ji = -n_ij, u_ji = -u_ij, ...), which makes the pair
// forces exactly opposite. Each particle keeps its own copy of the
// tangential spring of every active contact (double buffered per subcycle).
#include "common.cuh"
#include "launch.h"

namespace lbmdem {

struct V3 {
    double x, y, z;
};
__device__ __forceinline__ V3 mk(double x, double y, double z) { return {x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator-(V3 a) { return {-a.x, -a.y, -a.z}; }
__device__ __forceinline__ V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ V3 ld3(const double* p, int i) { return {p[3 * i], p[3 * i + 1], p[3 * i + 2]}; }
__device__ __forceinline__ void st3(double* p, int i, V3 v) {
    p[3 * i] = v.x;
    p[3 * i + 1] = v.y;
    p[3 * i + 2] = v.z;
}
__device__ __forceinline__ float mimgf(float d, int n, int per) {
    if (per) {
        const float half = 0.5f * (float)n;
        if (d > half) d -= (float)n;
        if (d < -half) d += (float)n;
    }
    return d;
}
__device__ __forceinline__ double mimg(double d, int n, int per) {
    if (per) {
        double half = 0.5 * (double)n;
        if (d > half) d -= (double)n;
        if (d < -half) d += (double)n;
    }
    return d;
}

// ------------------------------------------------------------ particle view

__global__ void view_kernel(const Particles P) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    PartView v;
    double gg = 0.0;
    for (int d = 0; d < 3; ++d) {
        const double x = P.x[3 * i + d];
        const double b = floor(x);
        v.base[d] = (int)b;
        v.frac[d] = (float)(x - b);
        const double g = 0.5 - (x - b);
        gg += g * g;
        v.u[d] = (float)P.u[3 * i + d];
        v.om[d] = (float)P.om[3 * i + d];
        P.xf[3 * i + d] = (float)x;
    }
    v.R = (float)P.R[i];
    v.C = (float)(gg - P.R[i] * P.R[i]);
    P.view[i] = v;
}

void launch_view_update(const Particles& P, cudaStream_t st) {
    if (P.n == 0) return;
    view_kernel<<<(P.n + 127) / 128, 128, 0, st>>>(P);
}

// ------------------------------------------------------------ finalisation

__global__ void finalize_kernel(const FinalizeParams p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.P.n) return;
    double exact[6] = {0, 0, 0, 0, 0, 0};
    if (p.use_fixed) {
        // constant link parts summed exactly by the float32 boundary kernel:
        // K = 36 sum 2 w c and 36 sum 2 w (n x c); torque adds g x (K / 36)
        // with g = 1/2 - (x - floor(x)) the common fractional cell offset
        double k[6], g[3];
        for (int c = 0; c < 6; ++c) {
            k[c] = (double)p.P.acc_k[6 * i + c] * (1.0 / 36.0);
            p.P.acc_k[6 * i + c] = 0;
        }
        for (int d = 0; d < 3; ++d) {
            const double x = p.P.x[3 * i + d];
            g[d] = 0.5 - (x - floor(x));
        }
        exact[0] = k[0];
        exact[1] = k[1];
        exact[2] = k[2];
        exact[3] = k[3] + (g[1] * k[2] - g[2] * k[1]);
        exact[4] = k[4] + (g[2] * k[0] - g[0] * k[2]);
        exact[5] = k[5] + (g[0] * k[1] - g[1] * k[0]);
    }
    for (int c = 0; c < 6; ++c) {
        double v;
        if (p.use_fixed) {
            v = (double)p.P.acc_i[6 * i + c] * (1.0 / FIX_SCALE) + exact[c];
            p.P.acc_i[6 * i + c] = 0;
        } else {
            v = p.P.acc_d[6 * i + c];
            p.P.acc_d[6 * i + c] = 0.0;
        }
        const double old = p.first_step ? v : p.P.fp_old[6 * i + c];
        p.P.fp[6 * i + c] = v;
        p.P.fbar[6 * i + c] = p.averaging ? 0.5 * (v + old) : v;
        p.P.fp_old[6 * i + c] = v;
    }
}

void launch_finalize(const FinalizeParams& p, cudaStream_t st) {
    if (p.P.n == 0) return;
    finalize_kernel<<<(p.P.n + 127) / 128, 128, 0, st>>>(p);
}

// ------------------------------------------------------------ neighbour bins

__device__ __forceinline__ int bin_coord(float x, float bs, int nb) {
    int b = (int)(x / bs);
    return b < 0 ? 0 : (b >= nb ? nb - 1 : b);
}

__global__ void bin_fill_kernel(const DemParams p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.P.n) return;
    int b[3];
    for (int d = 0; d < 3; ++d) b[d] = bin_coord(p.P.xf[3 * i + d], (float)p.binsize[d], p.nbins[d]);
    const long long bi = ((long long)b[2] * p.nbins[1] + b[1]) * p.nbins[0] + b[0];
    const int slot = atomicAdd(p.P.bin_count + bi, 1);
    if (slot < BIN_CAP) p.P.bin_list[bi * BIN_CAP + slot] = i;
    else atomicOr(p.status, ST_BIN_OVERFLOW);
}

void launch_bins(const DemParams& p, cudaStream_t st) {
    if (p.P.n == 0) return;
    bin_fill_kernel<<<(p.P.n + 127) / 128, 128, 0, st>>>(p);
}

// one warp per particle: lane k tests entry k of each of the 27 bins around it
// (a bin holds at most BIN_CAP = 32 particles); hits are appended in bin order
__global__ void neighbour_kernel(const DemParams p) {
    static_assert(BIN_CAP == 32, "one lane per bin entry");
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= p.P.n) return;   // warp-uniform
    const unsigned FULL = 0xffffffffu;
    const float xi[3] = {p.P.xf[3 * i], p.P.xf[3 * i + 1], p.P.xf[3 * i + 2]};
    const float Ri = (float)p.P.R[i];
    const float extra = (float)(p.cut_max + NBR_SKIN) + 0.01f;
    int b[3], lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        b[d] = bin_coord(xi[d], (float)p.binsize[d], p.nbins[d]);
        if (p.nbins[d] < 3) { lo[d] = 0; hi[d] = p.nbins[d] - 1; }
        else if (p.g.per[d]) { lo[d] = b[d] - 1; hi[d] = b[d] + 1; }
        else { lo[d] = b[d] > 0 ? b[d] - 1 : 0; hi[d] = b[d] < p.nbins[d] - 1 ? b[d] + 1 : b[d]; }
    }
    int cnt = 0;
    for (int bz = lo[2]; bz <= hi[2]; ++bz)
        for (int by = lo[1]; by <= hi[1]; ++by)
            for (int bx = lo[0]; bx <= hi[0]; ++bx) {
                const int wx = (p.nbins[0] >= 3) ? wrap_idx(bx, p.nbins[0]) : bx;
                const int wy = (p.nbins[1] >= 3) ? wrap_idx(by, p.nbins[1]) : by;
                const int wz = (p.nbins[2] >= 3) ? wrap_idx(bz, p.nbins[2]) : bz;
                const long long bi = ((long long)wz * p.nbins[1] + wy) * p.nbins[0] + wx;
                const int nb = min(p.P.bin_count[bi], BIN_CAP);
                bool hit = false;
                int j = -1;
                if (lane < nb) {
                    j = p.P.bin_list[bi * BIN_CAP + lane];
                    if (j != i) {
                        float d2 = 0.f;
                        for (int d = 0; d < 3; ++d) {
                            const float dd = mimgf(xi[d] - p.P.xf[3 * j + d], p.g.n[d], p.g.per[d]);
                            d2 += dd * dd;
                        }
                        const float reach = Ri + (float)p.P.R[j] + extra;
                        hit = d2 < reach * reach;
                    }
                }
                const unsigned m = __ballot_sync(FULL, hit);
                if (hit) {
                    const int slot = cnt + __popc(m & ((1u << lane) - 1u));
                    if (slot < NBR_CAP) p.P.nbr[i * NBR_CAP + slot] = j;
                }
                cnt += __popc(m);
            }
    if (lane == 0) {
        if (cnt > NBR_CAP) {
            atomicOr(p.status, ST_NBR_OVERFLOW);
            cnt = NBR_CAP;
        }
        p.P.nbr_count[i] = cnt;
    }
}

void launch_neighbours(const DemParams& p, cudaStream_t st) {
    if (p.P.n == 0) return;
    const long long threads = 32LL * p.P.n;
    neighbour_kernel<<<(int)((threads + 127) / 128), 128, 0, st>>>(p);
}

// ------------------------------------------------------------ Velocity Verlet

__device__ __forceinline__ double wrap_pos(double x, int n, int per) {
    if (per) {
        const double L = (double)n;
        if (x >= L) x -= L;
        if (x < 0.0) x += L;
    }
    return x;
}

__device__ __forceinline__ void position_update(const DemParams& p, int i) {
    // Eq. (37): x += dt u + dt^2 / (2 m) F
    const double dt = p.dt;
    const double c = dt * dt * p.P.hm[i];
    for (int d = 0; d < 3; ++d) {
        const double x = wrap_pos(p.P.x[3 * i + d] + dt * p.P.u[3 * i + d] + c * p.P.F_prev[3 * i + d],
                                  p.g.n[d], p.g.per[d]);
        p.P.x[3 * i + d] = x;
        p.P.xf[3 * i + d] = (float)x;
    }
}

__global__ void position_kernel(const DemParams p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.P.n) return;
    position_update(p, i);
}

void launch_dem_position(const DemParams& p, cudaStream_t st) {
    if (p.P.n == 0) return;
    position_kernel<<<(p.P.n + 127) / 128, 128, 0, st>>>(p);
}

// ------------------------------------------------------------ interaction laws

// lubrication force and torque on i due to j (Rj <= 0: plane wall), Eqs. (27)-(33)
__device__ void lubrication_on_i(const DemParams& p, double Ri, double Rj, double delta, V3 n, V3 uij,
                                 V3 omi, V3 omj, double dmin, V3& F, V3& T) {
    const double pi = 3.14159265358979323846;
    const double mu = p.mu_f;
    const double dl = delta > dmin ? delta : dmin;
    const V3 un = dot(uij, n) * n;
    const V3 ut = uij - un;
    double c_n, c_ftt, c_ttt, c_ftr, c_ttr;
    V3 om_ftr, om_ttr;
    if (Rj <= 0.0) {
        c_n = 1.0; c_ftt = 8.0 / 15.0; c_ttt = 1.0 / 10.0; c_ftr = 2.0 / 15.0; c_ttr = 2.0 / 5.0;
        om_ftr = omi;
        om_ttr = omi;
    } else if (Rj == Ri) {
        // k = 1: the coefficients below are exact binary fractions or the
        // correctly rounded quotients the general formulas give
        c_n = 0.25; c_ftt = 1.0 / 6.0; c_ttt = 0.125; c_ftr = 1.0 / 30.0; c_ttr = 0.2;
        const V3 oms = omi + omj;
        om_ftr = oms + 4.0 * omi + 4.0 * omj;
        om_ttr = omi + 0.25 * omj;
    } else {
        const double k = Rj / Ri;
        const double k1 = 1.0 + k;
        const double i1 = 1.0 / k1;
        const double i2 = i1 * i1;
        c_n = k * k * i2;
        c_ftt = 4.0 * k * (2.0 + k + 2.0 * k * k) * (i2 * i1) * (1.0 / 15.0);
        c_ttt = k * (4.0 + k) * i2 * 0.1;
        c_ftr = 2.0 * k * k * i2 * (1.0 / 15.0);
        c_ttr = 2.0 * k * i1 * 0.2;
        const V3 oms = omi + omj;
        om_ftr = oms + (4.0 * Ri / Rj) * omi + (4.0 * k) * omj;
        om_ttr = omi + (k * 0.25) * omj;
    }
    if (delta > 0.0 && delta < p.cut_n)
        F = F + (-6.0 * pi * mu * Ri * Ri * c_n * (1.0 / dl - p.inv_cut_n)) * un;
    const bool tt = p.tangential && delta > 0.0 && delta < p.cut_tt;
    const bool tr = p.tangential && delta > 0.0 && delta < p.cut_tr;
    if (tt || tr) {
        const double lg_tt = log(dl * p.inv_cut_tt);
        const double lg_tr = p.cut_tr == p.cut_tt ? lg_tt : log(dl * p.inv_cut_tr);
        if (tt) {
            F = F + (6.0 * pi * mu * Ri * c_ftt * lg_tt) * ut;
            T = T + (8.0 * pi * mu * Ri * Ri * c_ttt * lg_tt) * cross(uij, n);
        }
        if (tr) {
            F = F + (-6.0 * pi * mu * Ri * Ri * c_ftr * lg_tr) * cross(om_ftr, n);
            T = T + (8.0 * pi * mu * Ri * Ri * Ri * c_ttr * lg_tr) * (om_ttr - dot(om_ttr, n) * n);
        }
    }
}

// normal + Coulomb-limited tangential contact force on i, Eqs. (41)-(50)
__device__ void contact_force(const DemParams& p, V3 n, double delta, V3 ucp, V3 uij, double m_eff,
                              double Tc, V3 dt_old, V3& Fn, V3& Ft, V3& dt_new) {
    const double iT = 1.0 / Tc;
    const double kn = m_eff * p.pi2_log_e2 * (iT * iT);
    const double dn = -2.0 * m_eff * p.log_e * iT;
    const double kt = p.kappa * kn, dtg = p.sqrt_kappa * dn;
    const V3 un = dot(uij, n) * n;
    const V3 ut = ucp - un;
    Fn = (-kn * delta) * n - dn * un;
    const V3 proj = dt_old - dot(dt_old, n) * n;
    const double lp = sqrt(dot(proj, proj));
    const V3 rot = lp > 0.0 ? (sqrt(dot(dt_old, dt_old)) / lp) * proj : mk(0, 0, 0);
    const V3 Fsd = (-kt) * rot - dtg * ut;
    const double fc = p.mu_p * sqrt(dot(Fn, Fn));
    const double lsd = sqrt(dot(Fsd, Fsd));
    if (lsd < fc) {
        Ft = Fsd;
        dt_new = rot + p.dt * ut;
    } else {
        const V3 t = lsd > 0.0 ? (1.0 / lsd) * Fsd : mk(0, 0, 0);
        Ft = fc * t;
        dt_new = (-1.0 / kt) * (fc * t + dtg * ut);
    }
}

__device__ __forceinline__ double collision_time(double diameter, double Tc) {
    return Tc > 0.0 ? Tc : 2.31 * diameter * 1.7320508075688772;
}

// Force and torque on particle i from its neighbour j (lubrication,
// Eqs. (25)-(33), and contact, Eqs. (39)-(50)) at the subcycle's positions;
// contact = the spring of the pair continues, dnew its new value.
__device__ __forceinline__ void pair_force(const DemParams& p, int cur, int i, int j, V3& F, V3& T, bool& contact,
                                           V3& dnew) {
    const Particles& P = p.P;
    const double* X = P.xs[cur];
    const double* Uv = P.us[cur];
    const double* Om = P.oms[cur];
    const V3 xi = ld3(X, i), xj = ld3(X, j);
    const V3 d = mk(mimg(xi.x - xj.x, p.g.n[0], p.g.per[0]), mimg(xi.y - xj.y, p.g.n[1], p.g.per[1]),
                    mimg(xi.z - xj.z, p.g.n[2], p.g.per[2]));
    const double dist = sqrt(dot(d, d));
    const double Ri = P.R[i], Rj = P.R[j];
    const double delta = dist - (Ri + Rj);
    F = mk(0, 0, 0);
    T = mk(0, 0, 0);
    contact = false;
    dnew = mk(0, 0, 0);
    if (delta >= p.cut_max && delta >= 0.0) return;
    const V3 n = (1.0 / dist) * d;
    const V3 ui = ld3(Uv, i), omi = ld3(Om, i), uj = ld3(Uv, j), omj = ld3(Om, j);
    const V3 uij = ui - uj;
    if (p.lubrication) {
        const double Rm = 0.5 * (Ri + Rj);
        const double dmin = (p.min_a + p.min_b * Rm) * Rm;
        lubrication_on_i(p, Ri, Rj, delta, n, uij, omi, omj, dmin, F, T);
    }
    if (delta < 0.0) {
        const V3 ri = (-0.5) * d, rj = 0.5 * d;
        const V3 ucp = (ui + cross(omi, ri)) - (uj + cross(omj, rj));
        const double mi = P.m[i], mj = P.m[j];
        const double m_eff = mi * mj / (mi + mj);
        const double Tc = collision_time(Ri + Rj, p.Tc);
        V3 old = mk(0, 0, 0);
        const int nin = P.hist_n[p.hin][i];
        for (int h = 0; h < nin; ++h)
            if (P.hist_id[p.hin][i * NBR_CAP + h] == j) {
                const double* s = P.hist_d[p.hin] + 3 * (i * NBR_CAP + h);
                old = mk(s[0], s[1], s[2]);
                break;
            }
        V3 Fn, Ft;
        contact_force(p, n, delta, ucp, uij, m_eff, Tc, old, Fn, Ft, dnew);
        F = F + (Fn + Ft);
        T = T + cross(ri, Ft);
        contact = true;
    }
}

// One Velocity-Verlet subcycle (Algorithm 1, inner loop) for 32 particles per
// block of 128 threads. Pass 1, four lanes per particle: a float32 prefilter
// of the neighbour slots (float positions are within 1e-4 of the float64
// ones, so a gap above cut_max + 1e-3 there is above cut_max exactly); the
// surviving (particle, slot) pairs are queued in shared memory in particle
// and slot order. Pass 2: all 128 threads evaluate the queued pairs in
// float64 (lubrication, Eqs. (25)-(33); contact, Eqs. (39)-(50)), so the
// slow float64 units see full warps; each particle then sums its pairs in
// slot order (the result does not depend on scheduling). Pass 3, one thread
// per particle: plane walls, the averaged fluid force and V (rho_p - rho_f) g,
// then the velocities (Eq. (38)) and, unless it is the last subcycle, the
// positions of the next subcycle (Eq. (37)) into buffer 1 - cur.
// init = 1 evaluates the initial force F(t = 0) only (no state or history
// update). Pair terms are evaluated by both partners with mirrored operands.
constexpr int PPB = 32;          // particles per block
constexpr int PAIR_CHUNK = 128;  // queued pairs evaluated per pass of the block

__global__ void __launch_bounds__(128) subcycle_kernel(const DemParams p, int cur, int init, int last) {
    const Particles& P = p.P;
    const int tid = threadIdx.x;
    const int pl = tid >> 2, sub = tid & 3;   // pass 1: particle of the block, lane of its group
    const int i = blockIdx.x * PPB + pl;
    const int hout = p.hout;
    __shared__ unsigned short s_queue[PPB * NBR_CAP];   // pl << 5 | slot
    __shared__ int s_off[PPB + 1];
    __shared__ double s_res[PAIR_CHUNK][6];
    __shared__ double s_sum[PPB][6];
    const float* Xf = P.xfs[cur];
    const unsigned FULL = 0xffffffffu;

    // pass 1: candidate slots of particle pl (bit k = slot k)
    unsigned mask = 0;
    int nn = 0;
    if (i < P.n) {
        nn = P.nbr_count[i];
        const float xif[3] = {Xf[3 * i], Xf[3 * i + 1], Xf[3 * i + 2]};
        const float Rif = (float)P.R[i];
        const float reach_pad = (float)p.cut_max + 1e-3f;
        for (int k = sub; k < nn; k += 4) {
            const int j = P.nbr[i * NBR_CAP + k];
            float d2f = 0.f;
            for (int d = 0; d < 3; ++d) {
                const float dd = mimgf(xif[d] - Xf[3 * j + d], p.g.n[d], p.g.per[d]);
                d2f += dd * dd;
            }
            const float reach = Rif + (float)P.R[j] + reach_pad;
            if (d2f < reach * reach) mask |= 1u << k;
            else if (!init) P.hist_id[hout][i * NBR_CAP + k] = -1;   // no spring on this slot
        }
    }
    mask |= __shfl_xor_sync(FULL, mask, 1);
    mask |= __shfl_xor_sync(FULL, mask, 2);
    if (sub == 0) s_off[pl] = __popc(mask);
    if (tid < 6 * PPB) reinterpret_cast<double*>(s_sum)[tid] = 0.0;
    if (tid + 128 < 6 * PPB) reinterpret_cast<double*>(s_sum)[tid + 128] = 0.0;
    __syncthreads();
    if (tid < 32) {   // exclusive prefix over the 32 particles
        const int c = s_off[tid];
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (tid >= o) incl += v;
        }
        s_off[tid] = incl - c;
        if (tid == 31) s_off[PPB] = incl;
    }
    __syncthreads();
    {
        // the group's lanes write the queue entries of their particle, in slot order
        unsigned m = mask;
        int r = 0;
        const int base = s_off[pl];
        while (m) {
            const int k = __ffs(m) - 1;
            m &= m - 1;
            if ((r & 3) == sub) s_queue[base + r] = (unsigned short)((pl << 5) | k);
            ++r;
        }
    }
    __syncthreads();
    // pass 2: the queued pairs in chunks of 128, one per thread
    const int total = s_off[PPB];
    for (int c0 = 0; c0 < total; c0 += PAIR_CHUNK) {
        const int e = c0 + tid;
        if (e < total) {
            const int q = s_queue[e];
            const int ep = q >> 5, k = q & 31;
            const int ei = blockIdx.x * PPB + ep;
            const int j = P.nbr[ei * NBR_CAP + k];
            V3 F, T, dnew;
            bool contact;
            pair_force(p, cur, ei, j, F, T, contact, dnew);
            s_res[tid][0] = F.x; s_res[tid][1] = F.y; s_res[tid][2] = F.z;
            s_res[tid][3] = T.x; s_res[tid][4] = T.y; s_res[tid][5] = T.z;
            if (!init) {
                // tangential spring of this neighbour slot for the next subcycle
                P.hist_id[hout][ei * NBR_CAP + k] = contact ? j : -1;
                if (contact) {
                    double* sd = P.hist_d[hout] + 3 * (ei * NBR_CAP + k);
                    sd[0] = dnew.x; sd[1] = dnew.y; sd[2] = dnew.z;
                }
            }
        }
        __syncthreads();
        if (tid < PPB) {   // particle tid adds its pairs of this chunk in slot order
            const int lo = max(s_off[tid], c0), hi = min(s_off[tid + 1], c0 + PAIR_CHUNK);
            for (int e2 = lo; e2 < hi; ++e2)
                for (int c = 0; c < 6; ++c) s_sum[tid][c] += s_res[e2 - c0][c];
        }
        __syncthreads();
    }
    // pass 3: one thread per particle
    if (tid >= PPB) return;
    const int ip = blockIdx.x * PPB + tid;
    if (ip >= P.n) return;
    const double* X = P.xs[cur];
    const double* Uv = P.us[cur];
    const double* Om = P.oms[cur];
    V3 F = mk(s_sum[tid][0], s_sum[tid][1], s_sum[tid][2]);
    V3 T = mk(s_sum[tid][3], s_sum[tid][4], s_sum[tid][5]);
    {
        // plane walls on the faces of non-periodic axes
        const V3 xi = ld3(X, ip), ui = ld3(Uv, ip), omi = ld3(Om, ip);
        const double Ri = P.R[ip], mi = P.m[ip];
        const double xa[3] = {xi.x, xi.y, xi.z};
        for (int a = 0; a < 3; ++a) {
            if (p.g.per[a]) continue;
            for (int side = 0; side < 2; ++side) {
                const int face = 2 * a + side;
                V3 nw = mk(0, 0, 0);
                const double sgn = side == 0 ? 1.0 : -1.0;
                if (a == 0) nw.x = sgn; else if (a == 1) nw.y = sgn; else nw.z = sgn;
                const double xw = side == 0 ? 0.0 : (double)p.g.n[a];
                const double delta = (xa[a] - xw) * sgn - Ri;
                const double* uwp = p.g.wall_vel[side][a];
                const V3 uw = mk(uwp[0], uwp[1], uwp[2]);
                const V3 uij = ui - uw;
                if (p.lubrication) {
                    const double dmin = (p.min_a + p.min_b * Ri) * Ri;
                    lubrication_on_i(p, Ri, -1.0, delta, nw, uij, omi, mk(0, 0, 0), dmin, F, T);
                }
                if (!init) P.wact[hout][6 * ip + face] = 0;
                if (delta < 0.0) {
                    const V3 ri = (-(Ri + 0.5 * delta)) * nw;
                    const V3 ucp = (ui + cross(omi, ri)) - uw;
                    const double Tc = collision_time(2.0 * Ri, p.Tc);
                    V3 old = mk(0, 0, 0);
                    if (P.wact[p.hin][6 * ip + face]) {
                        const double* sd = P.whist[p.hin] + 3 * (6 * ip + face);
                        old = mk(sd[0], sd[1], sd[2]);
                    }
                    V3 Fn, Ft, dnew;
                    contact_force(p, nw, delta, ucp, uij, mi, Tc, old, Fn, Ft, dnew);
                    F = F + (Fn + Ft);
                    T = T + cross(ri, Ft);
                    if (!init) {
                        double* sd = P.whist[hout] + 3 * (6 * ip + face);
                        sd[0] = dnew.x; sd[1] = dnew.y; sd[2] = dnew.z;
                        P.wact[hout][6 * ip + face] = 1;
                    }
                }
            }
        }
    }
    const V3 Fs = mk(F.x + P.fbar[6 * ip] + P.ext[3 * ip], F.y + P.fbar[6 * ip + 1] + P.ext[3 * ip + 1],
                     F.z + P.fbar[6 * ip + 2] + P.ext[3 * ip + 2]);
    const V3 Ts = mk(T.x + P.fbar[6 * ip + 3], T.y + P.fbar[6 * ip + 4], T.z + P.fbar[6 * ip + 5]);
    if (init) {
        st3(P.F_prev, ip, Fs);
        st3(P.T_prev, ip, Ts);
        return;
    }
    P.hist_n[hout][ip] = P.nbr_count[ip];
    // Eq. (38) for u and its rotational analogue for omega (hm = 1/(2m), hI = 1/(2I))
    const double cu = p.dt * P.hm[ip], co = p.dt * P.hI[ip];
    const V3 Fp = ld3(P.F_prev, ip), Tp = ld3(P.T_prev, ip);
    const V3 u = ld3(Uv, ip) + cu * (Fp + Fs);
    const V3 om = ld3(Om, ip) + co * (Tp + Ts);
    st3(P.F_prev, ip, Fs);
    st3(P.T_prev, ip, Ts);
    if (!(dot(u, u) < 0.25)) atomicOr(p.status, ST_FAST_PARTICLE);
    const int nxt = 1 - cur;
    st3(P.us[nxt], ip, u);
    st3(P.oms[nxt], ip, om);
    const double ua[3] = {u.x, u.y, u.z};
    const double Fa[3] = {Fs.x, Fs.y, Fs.z};
    const double c = p.dt * cu;
    PartView v;
    double gg = 0.0;
    for (int d = 0; d < 3; ++d) {
        // Eq. (37) for the next subcycle; the last subcycle keeps its positions
        double x = X[3 * ip + d];
        if (!last) x = wrap_pos(x + p.dt * ua[d] + c * Fa[d], p.g.n[d], p.g.per[d]);
        P.xs[nxt][3 * ip + d] = x;
        P.xfs[nxt][3 * ip + d] = (float)x;
        if (last) {
            const double b = floor(x);
            v.base[d] = (int)b;
            v.frac[d] = (float)(x - b);
            const double g = 0.5 - (x - b);
            gg += g * g;
            v.u[d] = (float)ua[d];
            v.om[d] = (float)(d == 0 ? om.x : d == 1 ? om.y : om.z);
        }
    }
    if (last) {
        v.R = (float)P.R[ip];
        v.C = (float)(gg - P.R[ip] * P.R[ip]);
        P.view[ip] = v;
    }
}

void launch_dem_subcycle(const DemParams& p, int cur, int init, int last, cudaStream_t st) {
    if (p.P.n == 0) return;
    subcycle_kernel<<<(p.P.n + PPB - 1) / PPB, 128, 0, st>>>(p, cur, init, last);
}

// copy state buffer 1 into buffer 0 (after an odd number of subcycles)
__global__ void state_copy_kernel(const Particles P) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 3 * P.n) return;
    P.xs[0][k] = P.xs[1][k];
    P.us[0][k] = P.us[1][k];
    P.oms[0][k] = P.oms[1][k];
    P.xfs[0][k] = P.xfs[1][k];
}

void launch_state_copy(const Particles& P, cudaStream_t st) {
    if (P.n == 0) return;
    state_copy_kernel<<<(3 * P.n + 255) / 256, 256, 0, st>>>(P);
}

}  // namespace lbmdem
