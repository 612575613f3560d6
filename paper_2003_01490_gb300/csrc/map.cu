// map.cu -- explicit particle mapping (Sec. 2.2), TRT+aB shell (Sec. 2.3.2),
// refill of uncovered cells (Eq. (18)) and the field read-out.
//
// Mapping: every particle registers itself in the candidate list of each
// 32x4x4 tile that its influence sphere (R + max(delta_aB, sqrt 2)) touches;
// then one thread per (x, y) column of the tile tests the tile's candidates
// against its four cells. The solid test |x_c - x_p|^2 <= R^2 and the shell
// test R^2 < |x_c - x_p|^2 <= (R + delta_aB)^2 are decided in float32 when the
// margin is clear and re-evaluated in float64 with round-to-nearest and no
// contraction, ((dx dx + dy dy) + dz dz), when a value lies within 1e-5
// (relative) of a threshold, so the flags are exactly those of a plain float64
// evaluation. The lowest particle index owns a cell inside several spheres;
// fluid cells have owner -1. Cells that were solid and are now fluid go to the
// refill list with their former particle. Fluid cells within R + sqrt(2) of a
// particle get the NEAR flag; solid cells next to another body (candidates for
// missing links) go to the missing-link list that the boundary kernel of the
// next step reads. A cell that turns solid gets the NaN marker in all its PDF
// slots of both buffers.
#include <type_traits>

#include "common.cuh"
#include "gang.cuh"
#include "launch.h"

// minimum resident mapping blocks per SM (a register cap)
#ifndef LBM_MAP_MIN_BLOCKS
#define LBM_MAP_MIN_BLOCKS 16
#endif

namespace lbmdem {

__device__ __forceinline__ double min_image_dd(double d, int n, int per) {
    if (per) {
        double half = 0.5 * (double)n;
        if (d > half) d -= (double)n;
        if (d < -half) d += (double)n;
    }
    return d;
}
// ------------------------------------------------------------ tile scatter

__device__ int axis_pieces(double xc, double r, int n, int per, int (&a)[2], int (&b)[2]) {
    // cells whose centre (i + 1/2) lies in [xc - r, xc + r]
    long long lo = (long long)ceil(xc - r - 0.5);
    long long hi = (long long)floor(xc + r - 0.5);
    if (hi < lo) return 0;
    if (!per) {
        if (lo < 0) lo = 0;
        if (hi > n - 1) hi = n - 1;
        if (hi < lo) return 0;
        a[0] = (int)lo; b[0] = (int)hi;
        return 1;
    }
    if (hi - lo + 1 >= n) { a[0] = 0; b[0] = n - 1; return 1; }
    long long lw = ((lo % n) + n) % n, hw = ((hi % n) + n) % n;
    if (lw <= hw) { a[0] = (int)lw; b[0] = (int)hw; return 1; }
    a[0] = (int)lw; b[0] = n - 1; a[1] = 0; b[1] = (int)hw;
    return 2;
}

// distinct tile indices covering the cell pieces of one axis
__device__ int axis_tiles(int np, const int (&a)[2], const int (&b)[2], int tsize, int (&t0)[2],
                          int (&t1)[2]) {
    if (np == 0) return 0;
    t0[0] = a[0] / tsize; t1[0] = b[0] / tsize;
    if (np == 1) return 1;
    int s = a[1] / tsize, e = b[1] / tsize;
    // trim the part of the second range already covered by the first
    if (e >= t0[0]) e = t0[0] - 1;
    if (s > e) return 1;
    t0[1] = s; t1[1] = e;
    return 2;
}

// one warp per particle; the lanes share out the tiles of its box
__device__ __forceinline__ void tile_scatter_body(const MapParams& p, int bx) {
    const int i = (bx * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= p.P.n) return;   // warp-uniform
    const double r = p.P.R[i] + fmax(p.shell_width, 1.4142135623730951) + 0.02;
    const int ts[3] = {TILE_X, TILE_Y, TILE_Z};
    int na[3], t0[3][2], t1[3][2], cnt[3];
    for (int d = 0; d < 3; ++d) {
        int a[2], b[2];
        int np = axis_pieces(p.P.x[3 * i + d], r, p.g.n[d], p.g.per[d], a, b);
        na[d] = axis_tiles(np, a, b, ts[d], t0[d], t1[d]);
        if (na[d] == 0) return;
        cnt[d] = 0;
        for (int k = 0; k < na[d]; ++k) cnt[d] += t1[d][k] - t0[d][k] + 1;
    }
    const int total = cnt[0] * cnt[1] * cnt[2];
    for (int k = lane; k < total; k += 32) {
        int rest = k;
        int tt[3];
        for (int d = 0; d < 3; ++d) {
            int m = rest % cnt[d];
            rest /= cnt[d];
            // the m-th tile of the axis' pieces
            const int len0 = t1[d][0] - t0[d][0] + 1;
            tt[d] = m < len0 ? t0[d][0] + m : t0[d][1] + (m - len0);
        }
        const long long t = ((long long)tt[2] * p.ntile[1] + tt[1]) * p.ntile[0] + tt[0];
        const int slot = atomicAdd(p.tile_count + t, 1);
        if (slot < TILE_CAP) p.tile_list[t * TILE_CAP + slot] = i;
        else atomicOr(p.status, ST_TILE_OVERFLOW);
    }
}

__global__ void tile_scatter_kernel(const MapParams p) { tile_scatter_body(p, (int)blockIdx.x); }

__global__ void tile_scatter_gang_kernel(const MapParams* __restrict__ table, const int* __restrict__ off, int n) {
    __shared__ __align__(16) MapParams sp;
    const int i = gang_instance(off, n, (int)blockIdx.x);
    gang_load(table, i, sp);
    tile_scatter_body(sp, (int)blockIdx.x - off[i]);
}

void launch_tile_scatter(const MapParams& p, cudaStream_t st) {
    if (p.P.n == 0) return;
    const long long threads = 32LL * p.P.n;
    tile_scatter_kernel<<<(int)((threads + 127) / 128), 128, 0, st>>>(p);
}

// ------------------------------------------------------------ mapping

// The NaN marker of a solid cell (owner + 1 in the payload of the 4- and
// 8-byte formats) into all its PDF slots of both buffers; the dense kernel
// finds particle links and their particle by it.
__device__ __forceinline__ void put_markers(void* const (&pdf)[2], int elem, long long ncells, long long idx,
                                            int owner) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        for (int q = 0; q < Q; ++q) {
            const long long k = (long long)q * ncells + idx;
            if (elem == 8) reinterpret_cast<unsigned long long*>(pdf[b])[k] = marker_bits64(owner);
            else if (elem == 4) reinterpret_cast<unsigned int*>(pdf[b])[k] = marker_bits32(owner);
            else reinterpret_cast<unsigned short*>(pdf[b])[k] = (unsigned short)0x7fff;
        }
    }
}

// Exact float64 decision of the solid and shell tests for a cell centre whose
// float32 distance lies within the tolerance of a threshold (kept out of line:
// it runs for a tiny fraction of the tests). Returns bit 0 inside, bit 1 shell.
__device__ __noinline__ int exact_tests(const MapParams& p, int id, int x, int y, int z) {
    const int cpos[3] = {x, y, z};
    const double R = p.P.R[id];
    double dd[3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
        dd[d] = min_image_dd(((double)cpos[d] + 0.5) - p.P.x[3 * id + d], p.g.n[d], p.g.per[d]);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dd[0], dd[0]), __dmul_rn(dd[1], dd[1])), __dmul_rn(dd[2], dd[2]));
    const double rs = __dadd_rn(R, p.shell_width);
    const bool inside = d2 <= __dmul_rn(R, R);
    const bool in_shell = !inside && d2 <= __dmul_rn(rs, rs);
    return (inside ? 1 : 0) | (in_shell ? 2 : 0);
}

// minimum image on a short periodic axis, decided on 2 (n + g) against L
__device__ __forceinline__ float short_axis_image(float n, float g, int L) {
    const float tw = 2.0f * n + 2.0f * g;
    const float fl = (float)L;
    return tw > fl ? n - fl : (tw < -fl ? n + fl : n);
}

// One block per 32x4x4 tile, 128 threads; warp w takes the 8x4x4 brick of
// x in [8w, 8w + 8) (a compact brick meets fewer spheres than a 32-cell row),
// lane l the column x = 8w + (l & 7), y = l >> 3 of its four z cells. Per
// candidate the shared arrays hold the integer offset n0 of the tile's first
// cell from the particle's base cell (as an exact float; on long periodic
// axes already moved to the image nearest to the tile), the common fractional
// offset g = 1/2 - frac, R^2 and the thresholds of the shell and near tests
// with their float32 tolerances. A cell's offset is (n0 + l) + g with the
// integer part formed first, so no float32 intermediate is larger than the
// offset itself. Each warp first drops the candidates that cannot reach its
// brick.
// (tile bx, by, bz of the box)
__device__ __forceinline__ void map_body(const MapParams& p, int bx, int by, int bz) {
    static_assert(TILE_X == 32 && TILE_Y == 4, "four 8x4 column bricks per tile");
    __shared__ float4 cn[TILE_CAP];
    __shared__ float4 ca[TILE_CAP];
    __shared__ float4 cb[TILE_CAP];
    __shared__ unsigned int s_cnt[4];          // per warp: missing-link cells
    __shared__ unsigned int s_solid[4];
    __shared__ unsigned int s_base;
    const long long t = ((long long)bz * p.ntile[1] + by) * p.ntile[0] + bx;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lx = 8 * warp + (lane & 7), ly = lane >> 3;
    const int org[3] = {bx * TILE_X, by * TILE_Y, bz * TILE_Z};
    const int x = org[0] + lx, y = org[1] + ly;
    const int nx = p.g.n[0], ny = p.g.n[1], nz = p.g.n[2];
    const long long plane = (long long)nx * ny;
    const bool valid_xy = x < nx && y < ny;
    const long long idx0 = (long long)org[2] * plane + (long long)y * nx + x;
    // previous flags of the column, loaded before the candidate tests
    static_assert(TILE_Z <= 8, "previous flags of a column packed in one word");
    using ZWord = typename std::conditional<(TILE_Z > 4), unsigned long long, unsigned>::type;
    ZWord old4 = 0;
#pragma unroll
    for (int j = 0; j < TILE_Z; ++j)
        if (valid_xy && org[2] + j < nz) old4 |= (ZWord)p.flags[idx0 + j * plane] << (8 * j);
    const int c = p.tile_count[t];
    const int ncand = c < TILE_CAP ? c : TILE_CAP;
    if (tid < ncand) {
        const int i = p.tile_list[t * TILE_CAP + tid];
        const PartView v = p.P.view[i];
        const int ts[3] = {TILE_X, TILE_Y, TILE_Z};
        float n0[3], g[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            int n = org[d] - v.base[d];
            g[d] = 0.5f - v.frac[d];
            if (p.g.per[d] && !p.small[d]) {
                // image nearest to the tile centre
                const int L = p.g.n[d];
                const float cc = (float)(2 * n + ts[d] - 1) + 2.0f * g[d];   // twice the centre offset
                if (cc > (float)L) n -= L;
                else if (cc < -(float)L) n += L;
            }
            n0[d] = (float)n;
        }
        const float R = v.R;
        const float Rs = R + (float)p.shell_width;
        const float Rn = R + 1.4142135f + 0.02f;
        const float R2 = R * R, Rs2 = Rs * Rs;
        cn[tid] = make_float4(n0[0], n0[1], n0[2], __int_as_float(i));
        ca[tid] = make_float4(g[0], g[1], g[2], R2);
        cb[tid] = make_float4(Rs2, Rn * Rn, 1e-5f * (R2 + 1.0f), 1e-5f * (Rs2 + 1.0f));
    }
    __syncthreads();
    // the tile's candidate count is consumed: reset it for the next scatter
    if (tid == 0) p.tile_count[t] = 0;

    const bool any_small = p.small[0] | p.small[1] | p.small[2];
    const float flx = (float)lx, fly = (float)ly;
    const float bx0 = (float)(8 * warp);
    // candidates that may reach this warp's brick (conservative float bound)
    unsigned relm[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = lane + 32 * h;
        bool rel = false;
        if (k < ncand) {
            if (any_small) {
                rel = true;
            } else {
                const float4 Nn = cn[k], A = ca[k], B = cb[k];
                const float xlo = (Nn.x + bx0) + A.x, xhi = (Nn.x + (bx0 + 7.0f)) + A.x;
                const float ylo = Nn.y + A.y, yhi = (Nn.y + (float)(TILE_Y - 1)) + A.y;
                const float zlo = Nn.z + A.z, zhi = (Nn.z + (float)(TILE_Z - 1)) + A.z;
                const float dx = xlo > 0.f ? xlo : (xhi < 0.f ? -xhi : 0.f);
                const float dy = ylo > 0.f ? ylo : (yhi < 0.f ? -yhi : 0.f);
                const float dz = zlo > 0.f ? zlo : (zhi < 0.f ? -zhi : 0.f);
                const float reach = fmaxf(B.y, B.x + B.w) * 1.0001f + 0.01f;
                rel = dx * dx + dy * dy + dz * dz <= reach;
            }
        }
        relm[h] = __ballot_sync(0xffffffffu, rel);
    }

    int own[TILE_Z];
    unsigned shell4 = 0;               // per z: shell bit
    unsigned near1 = 0, near2 = 0;     // per z: near one / two particles
    unsigned multi4 = 0;               // per z: inside a second sphere
#pragma unroll
    for (int j = 0; j < TILE_Z; ++j) own[j] = 0x7fffffff;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        unsigned mm = relm[h];
        while (mm) {
            const int k = __ffs(mm) - 1 + 32 * h;
            mm &= mm - 1;
            const float4 Nn = cn[k], A = ca[k], B = cb[k];
            const int id = __float_as_int(Nn.w);
            float fx = Nn.x + flx, fy = Nn.y + fly;
            if (any_small) {
                if (p.small[0]) fx = short_axis_image(fx, A.x, nx);
                if (p.small[1]) fy = short_axis_image(fy, A.y, ny);
            }
            const float dx = fx + A.x, dy = fy + A.y;
            const float sxy = dx * dx + dy * dy;
            const float far2 = B.x + B.w;
#pragma unroll
            for (int j = 0; j < TILE_Z; ++j) {
                float fz = Nn.z + (float)j;
                if (any_small && p.small[2]) fz = short_axis_image(fz, A.z, nz);
                const float dz = fz + A.z;
                const float d2f = sxy + dz * dz;
                if (d2f <= B.y) {
                    near2 |= near1 & (1u << j);
                    near1 |= 1u << j;
                }
                if (d2f > far2) continue;
                const bool exact_needed = fabsf(d2f - A.w) <= B.z || fabsf(d2f - B.x) <= B.w;
                bool inside, in_shell;
                if (!exact_needed) {
                    inside = d2f < A.w;
                    in_shell = !inside && d2f < B.x;
                } else {
                    const int r = exact_tests(p, id, x, y, org[2] + j);
                    inside = r & 1;
                    in_shell = (r & 2) != 0;
                }
                if (inside) {
                    if (own[j] != 0x7fffffff) multi4 |= 1u << j;
                    if (id < own[j]) own[j] = id;
                }
                else if (in_shell) shell4 |= 1u << j;
            }
        }
    }

    bool wall_xy = false;
    if (!p.g.per[0] && (x == 0 || x == nx - 1)) wall_xy = true;
    if (!p.g.per[1] && (y == 0 || y == ny - 1)) wall_xy = true;
    unsigned miss_bits = 0, solid_bits = 0;
#pragma unroll
    for (int j = 0; j < TILE_Z; ++j) {
        const int z = org[2] + j;
        if (!valid_xy || z >= nz) continue;
        const long long idx = idx0 + j * plane;
        const bool wall_adj = wall_xy || (!p.g.per[2] && (z == 0 || z == nz - 1));
        const unsigned nn = ((near1 >> j) & 1u) + ((near2 >> j) & 1u);
        const uint8_t old = (uint8_t)(old4 >> (8 * j));
        uint8_t nf = 0;
        if (own[j] != 0x7fffffff) {
            nf = FL_SOLID;
            solid_bits |= 1u << j;
            if (nn >= 2u || wall_adj) {
                nf |= FL_MISS;
                miss_bits |= 1u << j;
            }
            // new solid cells get markers; the particle of a solid cell can only
            // change where spheres overlap (now or at the last mapping), so
            // those cells get them again
            const bool multi = (multi4 >> j) & 1u;
            if (multi) nf |= FL_MULTI;
            p.owner[idx] = own[j];
            if ((!(old & FL_SOLID) || multi || (old & FL_MULTI)) && p.pdf[0])
                put_markers(p.pdf, p.elem, p.g.ncells, idx, own[j]);
        } else {
            if (shell4 & (1u << j)) nf |= FL_SHELL;
            if (nn >= 1u) nf |= FL_NEAR;
            if (old & FL_SOLID) {
                // uncovered this step: refill with the former particle's velocity
                nf |= FL_NEWFLUID;
                const int prev = p.owner[idx];
                p.owner[idx] = -1;
                const int slot = atomicAdd(p.refill_count, 1);
                if (slot < p.refill_cap) {
                    p.refill_list[slot] = (unsigned int)idx;
                    p.refill_owner[slot] = prev;
                } else {
                    atomicOr(p.status, ST_REFILL_OVERFLOW);
                }
            }
        }
        p.flags[idx] = nf;
    }

    // block-aggregated append to the missing-link list and solid count
    const unsigned FULL = 0xffffffffu;
    const unsigned lt = (1u << lane) - 1u;
    unsigned mb[TILE_Z];
    unsigned wm = 0, ws = 0;
#pragma unroll
    for (int j = 0; j < TILE_Z; ++j) {
        mb[j] = __ballot_sync(FULL, (miss_bits >> j) & 1u);
        wm += __popc(mb[j]);
        ws += __popc(__ballot_sync(FULL, (solid_bits >> j) & 1u));
    }
    if (lane == 0) {
        s_cnt[warp] = wm;
        s_solid[warp] = ws;
    }
    __syncthreads();
    if (tid == 0) {
        unsigned tm = 0;
        unsigned long long tsol = 0;
        for (int w = 0; w < 4; ++w) {
            const unsigned c = s_cnt[w];
            s_cnt[w] = tm;
            tm += c;
            tsol += s_solid[w];
        }
        s_base = tm ? (unsigned)atomicAdd(p.miss_count, (int)tm) : 0u;
        if (tsol) atomicAdd(p.n_solid, tsol);
    }
    __syncthreads();
    if (miss_bits) {
        int sm = (int)(s_base + s_cnt[warp]);
#pragma unroll
        for (int j = 0; j < TILE_Z; ++j) {
            if ((miss_bits >> j) & 1u) {
                const int slot = sm + __popc(mb[j] & lt);
                if (slot < p.miss_cap) p.miss_list[slot] = (unsigned)(idx0 + j * plane);
                else atomicOr(p.status, ST_REFILL_OVERFLOW);
            }
            sm += __popc(mb[j]);
        }
    }
}

__global__ void __launch_bounds__(128, LBM_MAP_MIN_BLOCKS) map_kernel(const __grid_constant__ MapParams p) {
    map_body(p, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z);
}

// instance i's tiles are its blocks off[i] .. off[i + 1] - 1, x fastest
__global__ void __launch_bounds__(128, LBM_MAP_MIN_BLOCKS / 2)
    map_gang_kernel(const MapParams* __restrict__ table, const int* __restrict__ off, int n) {
    __shared__ __align__(16) MapParams sp;
    const int i = gang_instance(off, n, (int)blockIdx.x);
    gang_load(table, i, sp);
    const int b = (int)blockIdx.x - off[i];
    const int t0 = sp.ntile[0], t1 = sp.ntile[1];
    map_body(sp, b % t0, (b / t0) % t1, b / (t0 * t1));
}

void launch_map(const MapParams& p, cudaStream_t st) {
    dim3 grid(p.ntile[0], p.ntile[1], p.ntile[2]);
    map_kernel<<<grid, TILE_X * TILE_Y, 0, st>>>(p);
}

__global__ void solid_markers_kernel(const __grid_constant__ MapParams p) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < p.g.ncells; idx += stride)
        if (p.flags[idx] & FL_SOLID) put_markers(p.pdf, p.elem, p.g.ncells, idx, p.owner[idx]);
}

void launch_solid_markers(const MapParams& p, cudaStream_t st) {
    if (!p.pdf[0]) return;
    solid_markers_kernel<<<152 * 8, 256, 0, st>>>(p);
}

// ------------------------------------------------------------ refill

// One warp per uncovered cell: lane q (1..18) reads the neighbour x + c_q
// (its 19 PDFs, when it was fluid before and after the update), the warp sums
// densities and shares the axis neighbours' velocities, and lane q (0..18)
// writes f_q of Eq. (18).
template <typename S>
__device__ __forceinline__ void refill_body(const RefillParams& p, int bx, int gx) {
    using T = typename Store<S>::T;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int count = min(*p.count, p.cap);
    const S* f = static_cast<const S*>(p.f);
    S* fw = static_cast<S*>(p.f);
    const long long N = p.g.ncells;
    const int nx = p.g.n[0], ny = p.g.n[1];
    const T ax = (T)p.accel[0], ay = (T)p.accel[1], az = (T)p.accel[2];
    constexpr unsigned long long PX = pack_dirs(0), PY = pack_dirs(1), PZ = pack_dirs(2);
    const int warps = gx * (blockDim.x >> 5);
    for (int k = bx * (blockDim.x >> 5) + (threadIdx.x >> 5); k < count; k += warps) {   // warp-uniform
        const long long idx = p.list[k];
        const int x = (int)(idx % nx);
        const int y = (int)((idx / nx) % ny);
        const int z = (int)(idx / ((long long)nx * ny));
        const int cpos[3] = {x, y, z};
        const int i = p.list_owner[k];
        const int q = lane < Q ? lane : 0;
        const int c[3] = {dir_c(PX, q), dir_c(PY, q), dir_c(PZ, q)};
        // lane q: neighbour x + c_q, fluid before and after the update
        bool ok = false;
        T dr = T(0), jx = T(0), jy = T(0), jz = T(0);
        if (q >= 1) {
            int nb[3] = {x + c[0], y + c[1], z + c[2]};
            bool out = false;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (p.g.per[d]) nb[d] = wrap_idx(nb[d], p.g.n[d]);
                else if (nb[d] < 0 || nb[d] >= p.g.n[d]) out = true;
            }
            if (!out) {
                const long long j = ((long long)nb[2] * ny + nb[1]) * nx + nb[0];
                if (!(p.flags[j] & (FL_SOLID | FL_NEWFLUID))) {
                    ok = true;
#pragma unroll
                    for (int r = 0; r < Q; ++r) {
                        const T v = Store<S>::load(f + (long long)r * N + j);
                        dr += v;
                        jx += (T)cx(r) * v;
                        jy += (T)cy(r) * v;
                        jz += (T)cz(r) * v;
                    }
                }
            }
        }
        T drho_sum = dr;   // neighbour densities minus rho0 (shifted, no cancellation)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) drho_sum += __shfl_xor_sync(FULL, drho_sum, o);
        const unsigned okm = __ballot_sync(FULL, ok);
        const int nnb = __popc(okm);
        // velocities of the axis neighbours +x -x +y -y +z -z (lanes 4, 3, 1, 2, 5, 6)
        const T vx = jx - T(0.5) * ax, vy = jy - T(0.5) * ay, vz = jz - T(0.5) * az;
        constexpr int SLOT_Q[6] = {4, 3, 1, 2, 5, 6};
        T uax[6][3];
        bool okax[6];
#pragma unroll
        for (int sl = 0; sl < 6; ++sl) {
            uax[sl][0] = __shfl_sync(FULL, vx, SLOT_Q[sl]);
            uax[sl][1] = __shfl_sync(FULL, vy, SLOT_Q[sl]);
            uax[sl][2] = __shfl_sync(FULL, vz, SLOT_Q[sl]);
            okax[sl] = (okm >> SLOT_Q[sl]) & 1u;
        }
        const T drb = nnb ? drho_sum / (T)nnb : T(0);
        const T rb = T(1) + drb;
        // velocity of the former particle at the cell centre (rigid body)
        T ut[3], rr[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double dd = ((double)cpos[d] + 0.5) - p.P.x[3 * i + d];
            if (p.g.per[d]) {
                double half = 0.5 * p.g.n[d];
                if (dd > half) dd -= p.g.n[d];
                if (dd < -half) dd += p.g.n[d];
            }
            rr[d] = (T)dd;
        }
        const T om0 = (T)p.P.om[3 * i], om1 = (T)p.P.om[3 * i + 1], om2 = (T)p.P.om[3 * i + 2];
        ut[0] = (T)p.P.u[3 * i] + (om1 * rr[2] - om2 * rr[1]);
        ut[1] = (T)p.P.u[3 * i + 1] + (om2 * rr[0] - om0 * rr[2]);
        ut[2] = (T)p.P.u[3 * i + 2] + (om0 * rr[1] - om1 * rr[0]);
        T g[3][3];   // g[a][b] = d u_a / d x_b
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int sp = 2 * b, sm = 2 * b + 1;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (okax[sp] && okax[sm]) g[a][b] = T(0.5) * (uax[sp][a] - uax[sm][a]);
                else if (okax[sp]) g[a][b] = uax[sp][a] - ut[a];
                else if (okax[sm]) g[a][b] = ut[a] - uax[sm][a];
                else g[a][b] = T(0);
            }
        }
        if (lane < Q) {
            const T coef = T(1) / (T(3) * (T)p.s_nu);   // c_s^2 / s_nu
            const T cf[3] = {(T)c[0], (T)c[1], (T)c[2]};
            T second = T(0);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const T pab = rb * ut[a] * ut[b] - rb * coef * (g[a][b] + g[b][a]);
                    second += pab * (cf[a] * cf[b] - (a == b ? T(1) / T(3) : T(0)));
                }
            const T cu = cf[0] * ut[0] + cf[1] * ut[1] + cf[2] * ut[2];
            const int cc = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
            const T w = cc == 0 ? T(1) / T(3) : (cc == 1 ? T(1) / T(18) : T(1) / T(36));
            // f_q - w_q written without forming f_q: w_q (rho_bar - 1) + ...
            const T dfq = w * (drb + T(3) * rb * cu + T(4.5) * second);
            Store<S>::store(fw + (long long)q * N + idx, dfq);
        }
    }
}

template <typename S>
__global__ void __launch_bounds__(128) refill_kernel(const RefillParams p) {
    refill_body<S>(p, (int)blockIdx.x, (int)gridDim.x);
}

template <typename S>
__global__ void __launch_bounds__(128) refill_gang_kernel(const RefillParams* __restrict__ table,
                                                          const int* __restrict__ off, int n) {
    __shared__ __align__(16) RefillParams sp;
    const int i = gang_instance(off, n, (int)blockIdx.x);
    gang_load(table, i, sp);
    refill_body<S>(sp, (int)blockIdx.x - off[i], off[i + 1] - off[i]);
}

void launch_map_gang(int kind, int storage, const void* table, const int* off, int n, int blocks, cudaStream_t st) {
    if (n <= 0 || blocks <= 0) return;
    if (kind == GANG_SCATTER) {
        tile_scatter_gang_kernel<<<blocks, 128, 0, st>>>(static_cast<const MapParams*>(table), off, n);
    } else if (kind == GANG_MAP) {
        map_gang_kernel<<<blocks, TILE_X * TILE_Y, 0, st>>>(static_cast<const MapParams*>(table), off, n);
    } else {
        const RefillParams* t = static_cast<const RefillParams*>(table);
        switch (storage) {
            case 0: refill_gang_kernel<double><<<blocks, 128, 0, st>>>(t, off, n); break;
            case 1: refill_gang_kernel<float><<<blocks, 128, 0, st>>>(t, off, n); break;
            case 2: refill_gang_kernel<__half><<<blocks, 128, 0, st>>>(t, off, n); break;
            default: refill_gang_kernel<__nv_bfloat16><<<blocks, 128, 0, st>>>(t, off, n); break;
        }
    }
}

void launch_refill(const RefillParams& p, cudaStream_t st) {
    const int blocks = 152 * 8, threads = 128;   // 4 warps (cells) per block
    switch (p.storage) {
        case 0: refill_kernel<double><<<blocks, threads, 0, st>>>(p); break;
        case 1: refill_kernel<float><<<blocks, threads, 0, st>>>(p); break;
        case 2: refill_kernel<__half><<<blocks, threads, 0, st>>>(p); break;
        default: refill_kernel<__nv_bfloat16><<<blocks, threads, 0, st>>>(p); break;
    }
}

// ------------------------------------------------------------ fields

template <typename S>
__global__ void fields_kernel(const FieldsParams p) {
    using T = typename Store<S>::T;
    const S* f = static_cast<const S*>(p.f);
    const long long N = p.g.ncells;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < p.count;
         k += (long long)gridDim.x * blockDim.x) {
        const long long idx = p.first_cell + k;
        double rho = 0, u[3] = {0, 0, 0};
        if (!(p.flags[idx] & FL_SOLID)) {
            // moments in the compute precision (float64 sums cost ten times
            // the read-out on GB300 and change u by less than 1e-8 relative)
            T dr = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const T v = Store<S>::load(f + (long long)q * N + idx);
                dr += v;
                jx += (T)cx(q) * v;
                jy += (T)cy(q) * v;
                jz += (T)cz(q) * v;
            }
            rho = 1.0 + (double)dr;
            u[0] = (double)jx - 0.5 * p.accel[0];
            u[1] = (double)jy - 0.5 * p.accel[1];
            u[2] = (double)jz - 0.5 * p.accel[2];
        }
        p.out[k] = rho;
        p.out[p.count + k] = u[0];
        p.out[2 * p.count + k] = u[1];
        p.out[3 * p.count + k] = u[2];
    }
}

void launch_fields(const FieldsParams& p, cudaStream_t st) {
    const int blocks = 152 * 8, threads = 256;
    switch (p.storage) {
        case 0: fields_kernel<double><<<blocks, threads, 0, st>>>(p); break;
        case 1: fields_kernel<float><<<blocks, threads, 0, st>>>(p); break;
        case 2: fields_kernel<__half><<<blocks, threads, 0, st>>>(p); break;
        default: fields_kernel<__nv_bfloat16><<<blocks, threads, 0, st>>>(p); break;
    }
}

// density at sample points: trilinear interpolation of the cell-centred
// density (cell i has its centre at i + 1/2); periodic axes wrap, wall axes
// clamp to the first and last cell; solid cells count with the reference
// density 1
template <typename S>
__global__ void sample_density_kernel(const SampleParams p) {
    using T = typename Store<S>::T;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= p.n) return;
    const S* f = static_cast<const S*>(p.f);
    const long long N = p.g.ncells;
    int i0[3];
    double t[3];
    for (int d = 0; d < 3; ++d) {
        const double g = p.pos[3 * k + d] - 0.5;
        const double b = floor(g);
        i0[d] = (int)b;
        t[d] = g - b;
    }
    double v = 0.0;
    for (int c = 0; c < 8; ++c) {
        int idx3[3];
        double wgt = 1.0;
        for (int d = 0; d < 3; ++d) {
            const int o = (c >> d) & 1;
            int i = i0[d] + o;
            const int n = p.g.n[d];
            if (p.g.per[d]) i = ((i % n) + n) % n;
            else i = i < 0 ? 0 : (i >= n ? n - 1 : i);
            idx3[d] = i;
            wgt *= o ? t[d] : 1.0 - t[d];
        }
        const long long idx = ((long long)idx3[2] * p.g.n[1] + idx3[1]) * p.g.n[0] + idx3[0];
        double rho = 1.0;
        if (!(p.flags[idx] & FL_SOLID)) {
            T dr = T(0);
#pragma unroll
            for (int q = 0; q < Q; ++q) dr += Store<S>::load(f + (long long)q * N + idx);
            rho = 1.0 + (double)dr;
        }
        v += wgt * rho;
    }
    p.out[k] = v;
}

void launch_sample_density(const SampleParams& p, cudaStream_t st) {
    if (p.n <= 0) return;
    const int blocks = (p.n + 127) / 128;
    switch (p.storage) {
        case 0: sample_density_kernel<double><<<blocks, 128, 0, st>>>(p); break;
        case 1: sample_density_kernel<float><<<blocks, 128, 0, st>>>(p); break;
        case 2: sample_density_kernel<__half><<<blocks, 128, 0, st>>>(p); break;
        default: sample_density_kernel<__nv_bfloat16><<<blocks, 128, 0, st>>>(p); break;
    }
}

}  // namespace lbmdem
