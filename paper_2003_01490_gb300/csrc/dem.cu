// dem.cu -- particle side of Algorithm 1: force finalisation and two-step
// averaging of the momentum-exchange force (Sec. 4.2), neighbour search,
// lubrication correction (Eqs. (25)-(33)), linear spring-dashpot contact with
// Coulomb-limited tangential spring (Eqs. (39)-(52)) and the Velocity-Verlet
// subcycles (Eqs. (37)-(38)); the prescribed-motion update. Particle state
// and integration are float64; the pair and wall laws run in float64 for
// float64 PDF storage and in float32 (separations and overlaps from float64
// positions) for the other formats.
//
// Each particle gathers every interaction of its own (its block evaluates
// the queued pairs with all threads, then sums them per particle in slot
// order), so no force atomics are needed; a pair is evaluated by both
// partners with mirrored operands (n_ji = -n_ij, u_ji = -u_ij, ...). Each
// particle keeps its own copy of the tangential spring of every active
// contact (double buffered per subcycle). Up to 32 particles run a whole
// step's subcycles in one block.
#include <cstring>

#include "common.cuh"
#include "gang.cuh"
#include "launch.h"

namespace lbmdem {

template <typename T>
struct Vec3 {
    T x, y, z;
};
using V3 = Vec3<double>;
__device__ __forceinline__ V3 mk(double x, double y, double z) { return {x, y, z}; }
template <typename T>
__device__ __forceinline__ Vec3<T> zero3() { return {T(0), T(0), T(0)}; }
template <typename T>
__device__ __forceinline__ Vec3<T> operator+(Vec3<T> a, Vec3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename T>
__device__ __forceinline__ Vec3<T> operator-(Vec3<T> a, Vec3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename T>
__device__ __forceinline__ Vec3<T> operator-(Vec3<T> a) { return {-a.x, -a.y, -a.z}; }
template <typename T>
__device__ __forceinline__ Vec3<T> operator*(T s, Vec3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <typename T>
__device__ __forceinline__ T dot(Vec3<T> a, Vec3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T>
__device__ __forceinline__ Vec3<T> cross(Vec3<T> a, Vec3<T> b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ V3 ld3(const double* p, int i) { return {p[3 * i], p[3 * i + 1], p[3 * i + 2]}; }
__device__ __forceinline__ Vec3<float> ld3(const float* p, int i) { return {p[3 * i], p[3 * i + 1], p[3 * i + 2]}; }
__device__ __forceinline__ void st3(double* p, int i, V3 v) {
    p[3 * i] = v.x;
    p[3 * i + 1] = v.y;
    p[3 * i + 2] = v.z;
}
template <typename T, typename U>
__device__ __forceinline__ Vec3<T> cvt3(Vec3<U> v) { return {(T)v.x, (T)v.y, (T)v.z}; }
__device__ __forceinline__ float tlog(float x) { return logf(x); }
__device__ __forceinline__ double tlog(double x) { return log(x); }
__device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
// the interaction constants in the pair arithmetic's precision
template <typename T>
__device__ __forceinline__ const DemConsts<T>& consts(const DemParams& p);
template <> __device__ __forceinline__ const DemConsts<double>& consts<double>(const DemParams& p) { return p.kd; }
template <> __device__ __forceinline__ const DemConsts<float>& consts<float>(const DemParams& p) { return p.kf; }
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

__device__ __forceinline__ void write_view(const Particles& P, int i) {
    PartView v;
    for (int d = 0; d < 3; ++d) {
        const double x = P.x[3 * i + d];
        const double b = floor(x);
        v.base[d] = (int)b;
        v.frac[d] = (float)(x - b);
        v.u[d] = (float)P.u[3 * i + d];
        v.om[d] = (float)P.om[3 * i + d];
        P.xf[3 * i + d] = (float)x;
    }
    v.R = (float)P.R[i];
    set_view_c(v, P.R[i]);
    P.view[i] = v;
}

// rebuild the float view of every particle (after insertion or a velocity
// change): the link arithmetic of Eqs. (14)-(17) reads it
__global__ void view_kernel(const Particles P) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    write_view(P, i);
}

void launch_view_update(const Particles& P, cudaStream_t st) {
    if (P.n == 0) return;
    view_kernel<<<(P.n + 127) / 128, 128, 0, st>>>(P);
}

// ------------------------------------------------------------ finalisation

// per particle: the step's hydrodynamic force and torque (Eqs. (16)-(17)) from
// the float64 or fixed-point link sums and the exact integer missing-link
// sums, their two-step average (Sec. 4.2), and the accumulators cleared
__device__ __forceinline__ void finalize_body(const FinalizeParams& p, int bx) {
    const int i = bx * blockDim.x + threadIdx.x;
    if (i >= p.P.n) return;
    double exact[6] = {0, 0, 0, 0, 0, 0};
    if (p.use_fixed) {
        // constant link parts summed exactly by the float32 boundary kernel:
        // K = 36 sum 2 w c and 36 sum 2 w (n x c); torque adds g x (K / 36)
        // with g = 1/2 - (x - floor(x)) the common fractional cell offset
        // (two components per word: lo + hi 2^32)
        double k[6], g[3];
        for (int c2 = 0; c2 < 3; ++c2) {
            const unsigned long long w = (unsigned long long)p.P.acc_k[3 * i + c2];
            const long long lo = (long long)(int)(unsigned)(w & 0xffffffffull);
            const long long hi = (long long)(w - (unsigned long long)lo) >> 32;
            k[2 * c2] = (double)lo * (1.0 / 36.0);
            k[2 * c2 + 1] = (double)hi * (1.0 / 36.0);
            p.P.acc_k[3 * i + c2] = 0;
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

__global__ void finalize_kernel(const FinalizeParams p) { finalize_body(p, (int)blockIdx.x); }

__global__ void finalize_gang_kernel(const FinalizeParams* __restrict__ table, const int* __restrict__ off, int n) {
    __shared__ __align__(16) FinalizeParams sp;
    const int i = gang_instance(off, n, (int)blockIdx.x);
    gang_load(table, i, sp);
    finalize_body(sp, (int)blockIdx.x - off[i]);
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

// particles into uniform bins no smaller than the largest interaction reach,
// for the neighbour search of the lubrication and contact pairs (Secs. 3.1, 4.1)
__device__ __forceinline__ void bin_fill_body(const DemParams& p, int bx) {
    const int i = bx * blockDim.x + threadIdx.x;
    if (i >= p.P.n) return;
    int b[3];
    for (int d = 0; d < 3; ++d) b[d] = bin_coord(p.P.xf[3 * i + d], (float)p.binsize[d], p.nbins[d]);
    const long long bi = ((long long)b[2] * p.nbins[1] + b[1]) * p.nbins[0] + b[0];
    if (p.pair_f32) {   // float32 copies of the subcycle state read by the float32 pair laws
        for (int d = 0; d < 3; ++d) {
            p.P.ufs[0][3 * i + d] = (float)p.P.us[0][3 * i + d];
            p.P.omfs[0][3 * i + d] = (float)p.P.oms[0][3 * i + d];
        }
    }
    const int slot = atomicAdd(p.P.bin_count + bi, 1);
    if (slot < BIN_CAP) p.P.bin_list[bi * BIN_CAP + slot] = i;
    else atomicOr(p.status, ST_BIN_OVERFLOW);
}

__global__ void bin_fill_kernel(const DemParams p) { bin_fill_body(p, (int)blockIdx.x); }

__global__ void bin_fill_gang_kernel(const DemParams* __restrict__ table, const int* __restrict__ off, int n) {
    __shared__ __align__(16) DemParams sp;
    const int i = gang_instance(off, n, (int)blockIdx.x);
    gang_load(table, i, sp);
    bin_fill_body(sp, (int)blockIdx.x - off[i]);
}

void launch_bins(const DemParams& p, cudaStream_t st) {
    if (p.P.n == 0) return;
    bin_fill_kernel<<<(p.P.n + 127) / 128, 128, 0, st>>>(p);
}

// one warp per particle: lane k tests entry k of each of the 27 bins around it
// (a bin holds at most BIN_CAP = 32 particles); hits are appended in bin order
__device__ __forceinline__ void neighbour_body(const DemParams& p, int bx) {
    static_assert(BIN_CAP == 32, "one lane per bin entry");
    const int i = (bx * blockDim.x + threadIdx.x) >> 5;
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
    // ascending partner order (a bitonic sort over the warp), so that the
    // subcycles' pair sums, taken in slot order, do not depend on the order
    // in which atomics filled the bins
    const int m = cnt < NBR_CAP ? cnt : NBR_CAP;
    __syncwarp();
    int v = lane < m ? p.P.nbr[i * NBR_CAP + lane] : 0x7fffffff;
    for (int k = 2; k <= 32; k <<= 1)
        for (int j2 = k >> 1; j2 > 0; j2 >>= 1) {
            const int o = __shfl_xor_sync(FULL, v, j2);
            v = (((lane & j2) == 0) == ((lane & k) == 0)) ? min(v, o) : max(v, o);
        }
    if (lane < m) p.P.nbr[i * NBR_CAP + lane] = v;
    if (lane == 0) {
        if (cnt > NBR_CAP) {
            atomicOr(p.status, ST_NBR_OVERFLOW);
            cnt = NBR_CAP;
        }
        p.P.nbr_count[i] = cnt;
    }
}

__global__ void neighbour_kernel(const DemParams p) { neighbour_body(p, (int)blockIdx.x); }

__global__ void neighbour_gang_kernel(const DemParams* __restrict__ table, const int* __restrict__ off, int n) {
    __shared__ __align__(16) DemParams sp;
    const int i = gang_instance(off, n, (int)blockIdx.x);
    gang_load(table, i, sp);
    neighbour_body(sp, (int)blockIdx.x - off[i]);
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

// the first Velocity-Verlet position update of a step (Eq. (37)); later
// subcycles update positions inside the subcycle kernel
__global__ void position_kernel(const DemParams p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.P.n) return;
    position_update(p, i);
}

void launch_dem_position(const DemParams& p, cudaStream_t st) {
    if (p.P.n == 0) return;
    position_kernel<<<(p.P.n + 127) / 128, 128, 0, st>>>(p);
}

// prescribed motion: every particle moves by its velocity over one time step
// (Eq. (37) with no force and dt = 1), then its view is rebuilt
__global__ void prescribed_move_kernel(const Particles P, const Geom g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    for (int d = 0; d < 3; ++d) P.x[3 * i + d] = wrap_pos(P.x[3 * i + d] + P.u[3 * i + d], g.n[d], g.per[d]);
    write_view(P, i);
}

void launch_prescribed_move(const Particles& P, const Geom& g, cudaStream_t st) {
    if (P.n == 0) return;
    prescribed_move_kernel<<<(P.n + 127) / 128, 128, 0, st>>>(P, g);
}


// ------------------------------------------------------------ interaction laws

// lubrication force and torque on i due to j (Rj <= 0: plane wall), Eqs. (27)-(33)
template <typename T>
__device__ void lubrication_on_i(const DemConsts<T>& k, int tangential, T Ri, T Rj, T delta, Vec3<T> n,
                                 Vec3<T> uij, Vec3<T> omi, Vec3<T> omj, T dmin, Vec3<T>& F, Vec3<T>& Tq) {
    // no term acts outside (0, largest cut-off): a far wall or partner costs nothing
    if (!(delta > T(0) && delta < k.cut_max)) return;
    const T pi = T(3.14159265358979323846);
    const T mu = k.mu_f;
    const T dl = delta > dmin ? delta : dmin;
    const Vec3<T> un = dot(uij, n) * n;
    const Vec3<T> ut = uij - un;
    T c_n, c_ftt, c_ttt, c_ftr, c_ttr;
    Vec3<T> om_ftr, om_ttr;
    if (Rj <= T(0)) {
        c_n = T(1); c_ftt = T(8.0 / 15.0); c_ttt = T(1.0 / 10.0); c_ftr = T(2.0 / 15.0); c_ttr = T(2.0 / 5.0);
        om_ftr = omi;
        om_ttr = omi;
    } else if (Rj == Ri) {
        // k = 1: the coefficients below are exact binary fractions or the
        // correctly rounded quotients the general formulas give
        c_n = T(0.25); c_ftt = T(1.0 / 6.0); c_ttt = T(0.125); c_ftr = T(1.0 / 30.0); c_ttr = T(0.2);
        const Vec3<T> oms = omi + omj;
        om_ftr = oms + T(4) * omi + T(4) * omj;
        om_ttr = omi + T(0.25) * omj;
    } else {
        const T kr = Rj / Ri;
        const T k1 = T(1) + kr;
        const T i1 = T(1) / k1;
        const T i2 = i1 * i1;
        c_n = kr * kr * i2;
        c_ftt = T(4) * kr * (T(2) + kr + T(2) * kr * kr) * (i2 * i1) * T(1.0 / 15.0);
        c_ttt = kr * (T(4) + kr) * i2 * T(0.1);
        c_ftr = T(2) * kr * kr * i2 * T(1.0 / 15.0);
        c_ttr = T(2) * kr * i1 * T(0.2);
        const Vec3<T> oms = omi + omj;
        om_ftr = oms + (T(4) * Ri / Rj) * omi + (T(4) * kr) * omj;
        om_ttr = omi + (kr * T(0.25)) * omj;
    }
    if (delta > T(0) && delta < k.cut_n)
        F = F + (T(-6) * pi * mu * Ri * Ri * c_n * (T(1) / dl - k.inv_cut_n)) * un;
    const bool tt = tangential && delta > T(0) && delta < k.cut_tt;
    const bool tr = tangential && delta > T(0) && delta < k.cut_tr;
    if (tt || tr) {
        const T lg_tt = tlog(dl * k.inv_cut_tt);
        const T lg_tr = k.cut_tr == k.cut_tt ? lg_tt : tlog(dl * k.inv_cut_tr);
        if (tt) {
            F = F + (T(6) * pi * mu * Ri * c_ftt * lg_tt) * ut;
            Tq = Tq + (T(8) * pi * mu * Ri * Ri * c_ttt * lg_tt) * cross(uij, n);
        }
        if (tr) {
            F = F + (T(-6) * pi * mu * Ri * Ri * c_ftr * lg_tr) * cross(om_ftr, n);
            Tq = Tq + (T(8) * pi * mu * Ri * Ri * Ri * c_ttr * lg_tr) * (om_ttr - dot(om_ttr, n) * n);
        }
    }
}

// normal + Coulomb-limited tangential contact force on i, Eqs. (41)-(50)
template <typename T>
__device__ void contact_force(const DemConsts<T>& k, Vec3<T> n, T delta, Vec3<T> ucp, Vec3<T> uij, T m_eff,
                              T Tc, Vec3<T> dt_old, Vec3<T>& Fn, Vec3<T>& Ft, Vec3<T>& dt_new) {
    const T iT = T(1) / Tc;
    const T kn = m_eff * k.pi2_log_e2 * (iT * iT);
    const T dn = T(-2) * m_eff * k.log_e * iT;
    const T kt = k.kappa * kn, dtg = k.sqrt_kappa * dn;
    const Vec3<T> un = dot(uij, n) * n;
    const Vec3<T> ut = ucp - un;
    Fn = (-kn * delta) * n - dn * un;
    const Vec3<T> proj = dt_old - dot(dt_old, n) * n;
    const T lp = tsqrt(dot(proj, proj));
    const Vec3<T> rot = lp > T(0) ? (tsqrt(dot(dt_old, dt_old)) / lp) * proj : zero3<T>();
    const Vec3<T> Fsd = (-kt) * rot - dtg * ut;
    const T fc = k.mu_p * tsqrt(dot(Fn, Fn));
    const T lsd = tsqrt(dot(Fsd, Fsd));
    if (lsd < fc) {
        Ft = Fsd;
        dt_new = rot + k.dt * ut;
    } else {
        const Vec3<T> t = lsd > T(0) ? (T(1) / lsd) * Fsd : zero3<T>();
        Ft = fc * t;
        dt_new = (T(-1) / kt) * (fc * t + dtg * ut);
    }
}

template <typename T>
__device__ __forceinline__ T collision_time(T diameter, T Tc) {
    return Tc > T(0) ? Tc : T(2.31) * diameter * T(1.7320508075688772);
}

// periodic shift (0 or -+n) that takes the separation of a close pair to its
// minimum image, decided on the float32 copy of the separation
__device__ __forceinline__ double image_shift(float d, int n, int per) {
    if (per) {
        const float half = 0.5f * (float)n;
        if (d > half) return -(double)n;
        if (d < -half) return (double)n;
    }
    return 0.0;
}

// Force and torque on particle i from its neighbour j (lubrication,
// Eqs. (25)-(33), and contact, Eqs. (39)-(50)) at the subcycle's positions;
// contact = the spring of the pair continues, dnew its new value. T = double:
// all in float64. T = float: the separation and |d|^2 - (Ri + Rj)^2 in
// float64 (the overlap delta = that / (|d| + Ri + Rj) keeps float32 relative
// accuracy), the interaction laws in float32.
template <typename T>
__device__ __forceinline__ void pair_force(const DemParams& p, int cur, int hin, int i, int j, Vec3<T>& F,
                                           Vec3<T>& Tq, bool& contact, Vec3<T>& dnew) {
    const Particles& P = p.P;
    const DemConsts<T>& k = consts<T>(p);
    const double* X = P.xs[cur];
    const V3 xi = ld3(X, i), xj = ld3(X, j);
    Vec3<T> d;
    T dist, delta, Ri, Rj;
    if constexpr (sizeof(T) == 8) {
        d = mk(mimg(xi.x - xj.x, p.g.n[0], p.g.per[0]), mimg(xi.y - xj.y, p.g.n[1], p.g.per[1]),
               mimg(xi.z - xj.z, p.g.n[2], p.g.per[2]));
        dist = sqrt(dot(d, d));
        Ri = P.R[i];
        Rj = P.R[j];
        delta = dist - (Ri + Rj);
    } else {
        const float* Xf = P.xfs[cur];
        V3 dd = xi - xj;
        dd.x += image_shift(Xf[3 * i] - Xf[3 * j], p.g.n[0], p.g.per[0]);
        dd.y += image_shift(Xf[3 * i + 1] - Xf[3 * j + 1], p.g.n[1], p.g.per[1]);
        dd.z += image_shift(Xf[3 * i + 2] - Xf[3 * j + 2], p.g.n[2], p.g.per[2]);
        const double S = P.R[i] + P.R[j];
        const double e = fma(-S, S, dot(dd, dd));
        d = cvt3<float>(dd);
        dist = sqrtf(dot(d, d));
        Ri = P.view[i].R;
        Rj = P.view[j].R;
        delta = (float)e / (dist + (float)S);
    }
    F = zero3<T>();
    Tq = zero3<T>();
    contact = false;
    dnew = zero3<T>();
    if (delta >= k.cut_max && delta >= T(0)) return;
    const Vec3<T> n = (T(1) / dist) * d;
    Vec3<T> ui, omi, uj, omj;
    if constexpr (sizeof(T) == 8) {
        ui = ld3(P.us[cur], i); omi = ld3(P.oms[cur], i); uj = ld3(P.us[cur], j); omj = ld3(P.oms[cur], j);
    } else {
        ui = ld3(P.ufs[cur], i); omi = ld3(P.omfs[cur], i); uj = ld3(P.ufs[cur], j); omj = ld3(P.omfs[cur], j);
    }
    const Vec3<T> uij = ui - uj;
    if (p.lubrication) {
        const T Rm = T(0.5) * (Ri + Rj);
        const T dmin = (k.min_a + k.min_b * Rm) * Rm;
        lubrication_on_i<T>(k, p.tangential, Ri, Rj, delta, n, uij, omi, omj, dmin, F, Tq);
    }
    if (delta < T(0)) {
        const Vec3<T> ri = T(-0.5) * d, rj = T(0.5) * d;
        const Vec3<T> ucp = (ui + cross(omi, ri)) - (uj + cross(omj, rj));
        const T mi = (T)P.m[i], mj = (T)P.m[j];
        const T m_eff = mi * mj / (mi + mj);
        const T Tc = collision_time<T>(Ri + Rj, k.Tc);
        Vec3<T> old = zero3<T>();
        const int nin = P.hist_n[hin][i];
        for (int h = 0; h < nin; ++h)
            if (P.hist_id[hin][i * NBR_CAP + h] == j) {
                const double* s = P.hist_d[hin] + 3 * (i * NBR_CAP + h);
                old = Vec3<T>{(T)s[0], (T)s[1], (T)s[2]};
                break;
            }
        Vec3<T> Fn, Ft;
        contact_force<T>(k, n, delta, ucp, uij, m_eff, Tc, old, Fn, Ft, dnew);
        F = F + (Fn + Ft);
        Tq = Tq + cross(ri, Ft);
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
constexpr int PPB = DEM_ONE_BLOCK_MAX;   // particles per block
constexpr int PAIR_CHUNK = 128;  // queued pairs evaluated per pass of the block

// pass 3 of a subcycle for particle ip: plane walls, the averaged fluid force
// and V (rho_p - rho_f) g, the velocities (Eq. (38)) and, unless it is the
// last subcycle, the positions of the next subcycle (Eq. (37)) into buffer
// 1 - cur; sum holds the particle's pair forces and torques
template <typename T>
__device__ void integrate_particle(const DemParams& p, int ip, const T (&sum)[6], int cur, int hin, int hout, int init,
                                   int last) {
    const Particles& P = p.P;
    const double* X = P.xs[cur];
    const double* Uv = P.us[cur];
    const double* Om = P.oms[cur];
    Vec3<T> F = {sum[0], sum[1], sum[2]};
    Vec3<T> Tq = {sum[3], sum[4], sum[5]};
    {
        // plane walls on the faces of non-periodic axes
        const DemConsts<T>& k = consts<T>(p);
        const V3 xd = ld3(X, ip);
        Vec3<T> ui, omi;
        if constexpr (sizeof(T) == 8) {
            ui = ld3(Uv, ip);
            omi = ld3(Om, ip);
        } else {
            ui = ld3(P.ufs[cur], ip);
            omi = ld3(P.omfs[cur], ip);
        }
        const double Rid = P.R[ip];
        const T Ri = (T)Rid, mi = (T)P.m[ip];
        const double xa[3] = {xd.x, xd.y, xd.z};
        for (int a = 0; a < 3; ++a) {
            if (p.g.per[a]) continue;
            for (int side = 0; side < 2; ++side) {
                const int face = 2 * a + side;
                Vec3<T> nw = zero3<T>();
                const T sgn = side == 0 ? T(1) : T(-1);
                if (a == 0) nw.x = sgn; else if (a == 1) nw.y = sgn; else nw.z = sgn;
                const double xw = side == 0 ? 0.0 : (double)p.g.n[a];
                const T delta = (T)((xa[a] - xw) * (side == 0 ? 1.0 : -1.0) - Rid);
                const double* uwp = p.g.wall_vel[side][a];
                const Vec3<T> uw = {(T)uwp[0], (T)uwp[1], (T)uwp[2]};
                const Vec3<T> uij = ui - uw;
                if (p.lubrication) {
                    const T dmin = (k.min_a + k.min_b * Ri) * Ri;
                    lubrication_on_i<T>(k, p.tangential, Ri, T(-1), delta, nw, uij, omi, zero3<T>(), dmin, F, Tq);
                }
                if (!init) P.wact[hout][6 * ip + face] = 0;
                if (delta < T(0)) {
                    const Vec3<T> ri = (-(Ri + T(0.5) * delta)) * nw;
                    const Vec3<T> ucp = (ui + cross(omi, ri)) - uw;
                    const T Tc = collision_time<T>(T(2) * Ri, k.Tc);
                    Vec3<T> old = zero3<T>();
                    if (P.wact[hin][6 * ip + face]) {
                        const double* sd = P.whist[hin] + 3 * (6 * ip + face);
                        old = Vec3<T>{(T)sd[0], (T)sd[1], (T)sd[2]};
                    }
                    Vec3<T> Fn, Ft, dnew;
                    contact_force<T>(k, nw, delta, ucp, uij, mi, Tc, old, Fn, Ft, dnew);
                    F = F + (Fn + Ft);
                    Tq = Tq + cross(ri, Ft);
                    if (!init) {
                        double* sd = P.whist[hout] + 3 * (6 * ip + face);
                        sd[0] = (double)dnew.x; sd[1] = (double)dnew.y; sd[2] = (double)dnew.z;
                        P.wact[hout][6 * ip + face] = 1;
                    }
                }
            }
        }
    }
    const V3 Fd = cvt3<double>(F), Td = cvt3<double>(Tq);
    const V3 Fs = mk(Fd.x + P.fbar[6 * ip] + P.ext[3 * ip], Fd.y + P.fbar[6 * ip + 1] + P.ext[3 * ip + 1],
                     Fd.z + P.fbar[6 * ip + 2] + P.ext[3 * ip + 2]);
    const V3 Ts = mk(Td.x + P.fbar[6 * ip + 3], Td.y + P.fbar[6 * ip + 4], Td.z + P.fbar[6 * ip + 5]);
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
    if constexpr (sizeof(T) == 4) {
        for (int d = 0; d < 3; ++d) {
            P.ufs[nxt][3 * ip + d] = (float)(d == 0 ? u.x : d == 1 ? u.y : u.z);
            P.omfs[nxt][3 * ip + d] = (float)(d == 0 ? om.x : d == 1 ? om.y : om.z);
        }
    }
    const double ua[3] = {u.x, u.y, u.z};
    const double Fa[3] = {Fs.x, Fs.y, Fs.z};
    const double c = p.dt * cu;
    PartView v;
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
            v.u[d] = (float)ua[d];
            v.om[d] = (float)(d == 0 ? om.x : d == 1 ? om.y : om.z);
        }
    }
    if (last) {
        v.R = (float)P.R[ip];
        set_view_c(v, P.R[ip]);
        P.view[ip] = v;
    }
}


template <typename T>
__device__ __forceinline__ void subcycle_body(const DemParams& p, int cur, int hin, int hout, int init, int last, int pblock) {
    const Particles& P = p.P;
    const int tid = threadIdx.x;
    const int pl = tid >> 2, sub = tid & 3;   // pass 1: particle of the block, lane of its group
    const int i = pblock * PPB + pl;
    __shared__ unsigned short s_queue[PPB * NBR_CAP];   // pl << 5 | slot
    __shared__ int s_off[PPB + 1];
    __shared__ T s_res[PAIR_CHUNK][6];
    __shared__ T s_sum[PPB][6];
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
    if (tid < 6 * PPB) reinterpret_cast<T*>(s_sum)[tid] = T(0);
    if (tid + 128 < 6 * PPB) reinterpret_cast<T*>(s_sum)[tid + 128] = T(0);
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
            const int ei = pblock * PPB + ep;
            const int j = P.nbr[ei * NBR_CAP + k];
            Vec3<T> F, Tq, dnew;
            bool contact;
            pair_force<T>(p, cur, hin, ei, j, F, Tq, contact, dnew);
            s_res[tid][0] = F.x; s_res[tid][1] = F.y; s_res[tid][2] = F.z;
            s_res[tid][3] = Tq.x; s_res[tid][4] = Tq.y; s_res[tid][5] = Tq.z;
            if (!init) {
                // tangential spring of this neighbour slot for the next subcycle
                P.hist_id[hout][ei * NBR_CAP + k] = contact ? j : -1;
                if (contact) {
                    double* sd = P.hist_d[hout] + 3 * (ei * NBR_CAP + k);
                    sd[0] = (double)dnew.x; sd[1] = (double)dnew.y; sd[2] = (double)dnew.z;
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
    // pass 3: one thread per particle, lanes 0-7 of each warp (the float64
    // work of the block spread over the four schedulers)
    if ((tid & 31) < PPB / 4) {
        const int pl3 = (tid >> 5) * (PPB / 4) + (tid & 31);
        const int ip = pblock * PPB + pl3;
        if (ip < P.n) {
            T sum[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) sum[c] = s_sum[pl3][c];
            integrate_particle<T>(p, ip, sum, cur, hin, hout, init, last);
        }
    }
}

// one DEM subcycle of Algorithm 1: lubrication (Eqs. (25)-(34)) and contact
// (Eqs. (39)-(52)) for every pair and wall, then the Velocity-Verlet velocity
// update (Eq. (38)) and the next position update (Eq. (37))
template <typename T>
__global__ void __launch_bounds__(128) subcycle_kernel(const DemParams p, int cur, int init, int last) {
    subcycle_body<T>(p, cur, p.hin, p.hout, init, last, blockIdx.x);
}

// All subcycles of a step in one block when the particles fit in it (at most
// PPB): the first position update, n_sub subcycles separated by block
// barriers (each reads the positions and velocities the previous one wrote),
// and the copy back into buffer 0 after an odd count. The particles' state
// stays in shared memory for the whole step: the block loads it once, points
// the particle arrays of its (shared) parameter copy at the staged arrays, runs
// the subcycles there -- the code of the multi-block path, reaching shared
// memory through generic pointers -- and writes back what the step changed.
// The neighbour counts are staged too (read every subcycle); the neighbour
// lists, pair springs and the particle views stay in global memory.
// Latency, not arithmetic, sets the time of a few-particle DEM step, so each
// dependent global round trip saved per subcycle counts.
struct DemStage {
    double x[2][3 * PPB], u[2][3 * PPB], om[2][3 * PPB];
    float xf[2][3 * PPB], uf[2][3 * PPB], omf[2][3 * PPB];
    double F_prev[3 * PPB], T_prev[3 * PPB], ext[3 * PPB], fbar[6 * PPB];
    double hm[PPB], hI[PPB], R[PPB], m[PPB];
    double whist[2][18 * PPB];
    unsigned char wact[2][6 * PPB];
    int nbr_count[PPB];
};

// sp: the step's parameters in shared memory (n <= PPB particles); g receives
// the global particle arrays
template <typename T>
__device__ void dem_step_block(DemParams& sp, Particles& g, DemStage& st, int hcur, int n_sub) {
    const int tid = threadIdx.x;
    const int n = sp.P.n;
    if (tid == 0) g = sp.P;
    __syncthreads();
    for (int k = tid; k < 3 * n; k += blockDim.x) {
        st.x[0][k] = g.x[k];
        st.u[0][k] = g.u[k];
        st.om[0][k] = g.om[k];
        st.xf[0][k] = g.xf[k];
        st.uf[0][k] = g.ufs[0][k];
        st.omf[0][k] = g.omfs[0][k];
        st.F_prev[k] = g.F_prev[k];
        st.T_prev[k] = g.T_prev[k];
        st.ext[k] = g.ext[k];
    }
    for (int k = tid; k < 6 * n; k += blockDim.x) {
        st.fbar[k] = g.fbar[k];
        st.wact[0][k] = g.wact[0][k];
        st.wact[1][k] = g.wact[1][k];
    }
    for (int k = tid; k < 18 * n; k += blockDim.x) {
        st.whist[0][k] = g.whist[0][k];
        st.whist[1][k] = g.whist[1][k];
    }
    for (int k = tid; k < n; k += blockDim.x) {
        st.hm[k] = g.hm[k];
        st.hI[k] = g.hI[k];
        st.R[k] = g.R[k];
        st.m[k] = g.m[k];
        st.nbr_count[k] = g.nbr_count[k];
    }
    if (tid == 0) {
        Particles& P = sp.P;
        P.x = P.xs[0] = st.x[0];
        P.xs[1] = st.x[1];
        P.u = P.us[0] = st.u[0];
        P.us[1] = st.u[1];
        P.om = P.oms[0] = st.om[0];
        P.oms[1] = st.om[1];
        P.xf = P.xfs[0] = st.xf[0];
        P.xfs[1] = st.xf[1];
        for (int h = 0; h < 2; ++h) {
            P.ufs[h] = st.uf[h];
            P.omfs[h] = st.omf[h];
            P.whist[h] = st.whist[h];
            P.wact[h] = st.wact[h];
        }
        P.F_prev = st.F_prev;
        P.T_prev = st.T_prev;
        P.ext = st.ext;
        P.fbar = st.fbar;
        P.hm = st.hm;
        P.hI = st.hI;
        P.R = st.R;
        P.m = st.m;
        P.nbr_count = st.nbr_count;
    }
    __syncthreads();
    if (tid < n) position_update(sp, tid);
    __syncthreads();
    int cur = 0;
    for (int s = 0; s < n_sub; ++s) {
        subcycle_body<T>(sp, cur, hcur, 1 - hcur, 0, s == n_sub - 1, 0);
        __syncthreads();
        hcur = 1 - hcur;
        cur = 1 - cur;
    }
    // the state after the last subcycle is in buffer cur; buffer 0 of the
    // global arrays receives it
    for (int k = tid; k < 3 * n; k += blockDim.x) {
        g.x[k] = st.x[cur][k];
        g.u[k] = st.u[cur][k];
        g.om[k] = st.om[cur][k];
        g.xf[k] = st.xf[cur][k];
        g.ufs[0][k] = st.uf[cur][k];
        g.omfs[0][k] = st.omf[cur][k];
        g.F_prev[k] = st.F_prev[k];
        g.T_prev[k] = st.T_prev[k];
    }
    for (int k = tid; k < 6 * n; k += blockDim.x) {
        g.wact[0][k] = st.wact[0][k];
        g.wact[1][k] = st.wact[1][k];
    }
    for (int k = tid; k < 18 * n; k += blockDim.x) {
        g.whist[0][k] = st.whist[0][k];
        g.whist[1][k] = st.whist[1][k];
    }
}

template <typename T>
__global__ void __launch_bounds__(128) dem_step_one_block_kernel(const DemParams p, int hcur, int n_sub) {
    __shared__ __align__(16) DemParams sp;
    __shared__ __align__(16) Particles g;
    __shared__ __align__(16) DemStage st;
    constexpr int WORDS = (int)(sizeof(DemParams) / 4);
    static_assert(sizeof(DemParams) % 4 == 0, "parameters copied in words");
    const int* src = reinterpret_cast<const int*>(&p);
    int* dst = reinterpret_cast<int*>(&sp);
    for (int w = threadIdx.x; w < WORDS; w += blockDim.x) dst[w] = src[w];
    __syncthreads();
    dem_step_block<T>(sp, g, st, hcur, n_sub);
}

// The one-block DEM steps of many instances in one launch: block b runs the
// step of entry b of the table (its parameters, history parity and subcycle
// count), exactly as dem_step_one_block_kernel does for one instance.
struct DemBatchEntry {
    DemParams p;
    int hcur, n_sub;
};

template <typename T>
__global__ void __launch_bounds__(128) dem_step_batch_kernel(const DemBatchEntry* __restrict__ table) {
    __shared__ __align__(16) DemBatchEntry e;
    __shared__ __align__(16) Particles g;
    __shared__ __align__(16) DemStage st;
    constexpr int WORDS = (int)(sizeof(DemBatchEntry) / 4);
    static_assert(sizeof(DemBatchEntry) % 4 == 0, "entry copied in words");
    const int* src = reinterpret_cast<const int*>(table + blockIdx.x);
    int* dst = reinterpret_cast<int*>(&e);
    for (int w = threadIdx.x; w < WORDS; w += blockDim.x) dst[w] = src[w];
    __syncthreads();
    dem_step_block<T>(e.p, g, st, e.hcur, e.n_sub);
}

size_t dem_batch_entry_bytes() { return sizeof(DemBatchEntry); }

void fill_dem_batch_entry(const DemParams& p, int hcur, int n_sub, void* out) {
    DemBatchEntry e;
    std::memset(&e, 0, sizeof(e));
    e.p = p;
    e.hcur = hcur;
    e.n_sub = n_sub;
    std::memcpy(out, &e, sizeof(e));
}

void launch_dem_step_batch(const void* d_table, int count, int pair_f32, cudaStream_t st) {
    if (count <= 0) return;
    const DemBatchEntry* t = static_cast<const DemBatchEntry*>(d_table);
    if (pair_f32) dem_step_batch_kernel<float><<<count, 128, 0, st>>>(t);
    else dem_step_batch_kernel<double><<<count, 128, 0, st>>>(t);
}

void launch_dem_step_one_block(const DemParams& p, int hcur, int n_sub, cudaStream_t st) {
    if (p.P.n == 0) return;
    if (p.pair_f32) dem_step_one_block_kernel<float><<<1, 128, 0, st>>>(p, hcur, n_sub);
    else dem_step_one_block_kernel<double><<<1, 128, 0, st>>>(p, hcur, n_sub);
}

void launch_dem_subcycle(const DemParams& p, int cur, int init, int last, cudaStream_t st) {
    if (p.P.n == 0) return;
    if (p.pair_f32) subcycle_kernel<float><<<(p.P.n + PPB - 1) / PPB, 128, 0, st>>>(p, cur, init, last);
    else subcycle_kernel<double><<<(p.P.n + PPB - 1) / PPB, 128, 0, st>>>(p, cur, init, last);
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

// F^fp and T^fp of each particle ([n][6]) into two blocks [n][3] | [n][3],
// the layout of the host read-out
__global__ void fp_split_kernel(const double* __restrict__ fp, double* __restrict__ out, int n) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= 6LL * n) return;
    const long long i = k / 6;
    const int c = (int)(k - 6 * i);
    out[(c < 3 ? 0 : 3LL * n) + 3 * i + (c < 3 ? c : c - 3)] = fp[k];
}

// The multi-block DEM step and prescribed motion of many instances: one
// launch per phase (first position update, each subcycle, the copy back after
// an odd count, the prescribed move), each block running its block of one
// instance's grid with that instance's entry.
template <typename T>
__global__ void __launch_bounds__(128) dem_gang_kernel(const DemGangEntry* __restrict__ table,
                                                       const int* __restrict__ off, int n, int kind) {
    __shared__ __align__(16) DemGangEntry e;
    const int i = gang_instance(off, n, (int)blockIdx.x);
    gang_load(table, i, e);
    const int bx = (int)blockIdx.x - off[i];
    const Particles& P = e.p.P;
    if (kind == DEM_GANG_SUBCYCLE) {
        subcycle_body<T>(e.p, e.cur, e.p.hin, e.p.hout, 0, e.last, bx);
        return;
    }
    const int k = bx * blockDim.x + threadIdx.x;
    if (kind == DEM_GANG_POSITION) {
        if (k < P.n) position_update(e.p, k);
    } else if (kind == DEM_GANG_COPY) {
        if (k < 3 * P.n) {
            P.xs[0][k] = P.xs[1][k];
            P.us[0][k] = P.us[1][k];
            P.oms[0][k] = P.oms[1][k];
            P.xfs[0][k] = P.xfs[1][k];
        }
    } else if (k < P.n) {   // prescribed motion
        for (int d = 0; d < 3; ++d)
            P.x[3 * k + d] = wrap_pos(P.x[3 * k + d] + P.u[3 * k + d], e.p.g.n[d], e.p.g.per[d]);
        write_view(P, k);
    }
}

void launch_dem_gang(int kind, int pair_f32, const void* table, const int* off, int n, int blocks, cudaStream_t st) {
    if (n <= 0 || blocks <= 0) return;
    const DemGangEntry* t = static_cast<const DemGangEntry*>(table);
    if (pair_f32) dem_gang_kernel<float><<<blocks, 128, 0, st>>>(t, off, n, kind);
    else dem_gang_kernel<double><<<blocks, 128, 0, st>>>(t, off, n, kind);
}

// words set to zero, per instance a span (the counters a step starts from)
__global__ void zero_gang_kernel(const ZeroSpan* __restrict__ table, const int* __restrict__ off, int n) {
    const int i = gang_instance(off, n, (int)blockIdx.x);
    const ZeroSpan z = table[i];
    const int bx = (int)blockIdx.x - off[i], gx = off[i + 1] - off[i];
    for (int k = bx * blockDim.x + threadIdx.x; k < z.words; k += gx * blockDim.x) z.p[k] = 0;
}

void launch_gang(int kind, const void* table, const int* off, int n, int blocks, cudaStream_t st) {
    if (n <= 0 || blocks <= 0) return;
    switch (kind) {
        case GANG_FINALIZE:
            finalize_gang_kernel<<<blocks, 128, 0, st>>>(static_cast<const FinalizeParams*>(table), off, n);
            break;
        case GANG_BINS:
            bin_fill_gang_kernel<<<blocks, 128, 0, st>>>(static_cast<const DemParams*>(table), off, n);
            break;
        case GANG_NEIGHBOURS:
            neighbour_gang_kernel<<<blocks, 128, 0, st>>>(static_cast<const DemParams*>(table), off, n);
            break;
        default:
            zero_gang_kernel<<<blocks, 128, 0, st>>>(static_cast<const ZeroSpan*>(table), off, n);
            break;
    }
}

void launch_fp_split(const double* fp, double* out, int n, cudaStream_t st) {
    if (n <= 0) return;
    fp_split_kernel<<<(int)((6LL * n + 255) / 256), 256, 0, st>>>(fp, out, n);
}

}  // namespace lbmdem
