// map.cu -- explicit particle mapping (Sec. 2.2), TRT+aB shell (Sec. 2.3.2),
// refill of uncovered cells (Eq. (18)) and the field read-out.
//
// Mapping: every particle registers itself in the candidate list of each
// 32x4x4 tile that its influence sphere (R + max(delta_aB, sqrt 2)) touches;
// then one thread per cell tests the tile's candidates. The solid test
// |x_c - x_p|^2 <= R^2 and the shell test R^2 < |x_c - x_p|^2 <= (R + delta_aB)^2
// are decided in float32 when the margin is clear and re-evaluated in float64
// with round-to-nearest and no contraction, ((dx dx + dy dy) + dz dz), when a
// value lies within 1e-5 (relative) of a threshold, so the flags are exactly
// those of a plain float64 evaluation. The lowest particle index owns a cell
// inside several spheres. Cells that were solid and are now fluid are
// appended to the refill list; the owner field keeps their former particle.
// Fluid cells within R + sqrt(2) of a particle (candidates for particle links)
// and solid cells next to another body (candidates for missing links) go to
// the near-boundary list that the boundary kernel of the next step reads.
#include "common.cuh"
#include "launch.h"

namespace lbmdem {

__device__ __forceinline__ double min_image_dd(double d, int n, int per) {
    if (per) {
        double half = 0.5 * (double)n;
        if (d > half) d -= (double)n;
        if (d < -half) d += (double)n;
    }
    return d;
}
__device__ __forceinline__ float min_image_ff(float d, int n, int per) {
    if (per) {
        float half = 0.5f * (float)n;
        if (d > half) d -= (float)n;
        if (d < -half) d += (float)n;
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

__global__ void tile_scatter_kernel(const MapParams p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.P.n) return;
    const double r = p.P.R[i] + fmax(p.shell_width, 1.4142135623730951) + 0.02;
    const int ts[3] = {TILE_X, TILE_Y, TILE_Z};
    int na[3], t0[3][2], t1[3][2];
    for (int d = 0; d < 3; ++d) {
        int a[2], b[2];
        int np = axis_pieces(p.P.x[3 * i + d], r, p.g.n[d], p.g.per[d], a, b);
        na[d] = axis_tiles(np, a, b, ts[d], t0[d], t1[d]);
        if (na[d] == 0) return;
    }
    for (int pz = 0; pz < na[2]; ++pz)
        for (int tz = t0[2][pz]; tz <= t1[2][pz]; ++tz)
            for (int py = 0; py < na[1]; ++py)
                for (int ty = t0[1][py]; ty <= t1[1][py]; ++ty)
                    for (int px = 0; px < na[0]; ++px)
                        for (int tx = t0[0][px]; tx <= t1[0][px]; ++tx) {
                            long long t = ((long long)tz * p.ntile[1] + ty) * p.ntile[0] + tx;
                            int slot = atomicAdd(p.tile_count + t, 1);
                            if (slot < TILE_CAP) p.tile_list[t * TILE_CAP + slot] = i;
                            else atomicOr(p.status, ST_TILE_OVERFLOW);
                        }
}

void launch_tile_scatter(const MapParams& p, cudaStream_t st) {
    if (p.P.n == 0) return;
    tile_scatter_kernel<<<(p.P.n + 127) / 128, 128, 0, st>>>(p);
}

// ------------------------------------------------------------ mapping

// block-aggregated append: one global atomic per block and list
__device__ __forceinline__ void block_append(bool take, unsigned int entry, unsigned int* list, int* count, int cap,
                                             int* status, int* s_warp, int* s_base) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
    const unsigned am = __ballot_sync(0xffffffffu, take);
    if (lane == 0) s_warp[warp] = __popc(am);
    __syncthreads();
    if (tid == 0) {
        int tot = 0;
        for (int w = 0; w < nwarps; ++w) {
            const int c = s_warp[w];
            s_warp[w] = tot;
            tot += c;
        }
        *s_base = tot ? atomicAdd(count, tot) : 0;
    }
    __syncthreads();
    if (take) {
        const int slot = *s_base + s_warp[warp] + __popc(am & ((1u << lane) - 1u));
        if (slot < cap) list[slot] = entry;
        else atomicOr(status, ST_REFILL_OVERFLOW);
    }
    __syncthreads();
}

// Per candidate: integer offset n0 of the tile's first cell from the
// particle's base cell (for long periodic axes already moved to the image
// nearest to the tile), the common fractional offset g = 1/2 - frac, R^2, and
// the thresholds of the shell and near tests with their float32 tolerances.
// A cell's offset is (float)(n0 + l) + g: integer first, so no float32
// intermediate is larger than the offset itself.
__global__ void __launch_bounds__(512) map_kernel(const MapParams p) {
    __shared__ int4 cn[TILE_CAP];
    __shared__ float4 ca[TILE_CAP];
    __shared__ float4 cb[TILE_CAP];
    __shared__ int ncand;
    __shared__ unsigned int nsolid_blk;
    const long long t = ((long long)blockIdx.z * p.ntile[1] + blockIdx.y) * p.ntile[0] + blockIdx.x;
    const int tid = threadIdx.x + TILE_X * (threadIdx.y + TILE_Y * threadIdx.z);
    const int org[3] = {(int)blockIdx.x * TILE_X, (int)blockIdx.y * TILE_Y, (int)blockIdx.z * TILE_Z};
    if (tid == 0) {
        int c = p.tile_count[t];
        ncand = c < TILE_CAP ? c : TILE_CAP;
        nsolid_blk = 0;
    }
    __syncthreads();
    if (tid < ncand) {
        const int i = p.tile_list[t * TILE_CAP + tid];
        const PartView v = p.P.view[i];
        const int ts[3] = {TILE_X, TILE_Y, TILE_Z};
        int n0[3];
        float g[3];
        for (int d = 0; d < 3; ++d) {
            n0[d] = org[d] - v.base[d];
            g[d] = 0.5f - v.frac[d];
            if (p.g.per[d] && !p.small[d]) {
                // image nearest to the tile centre
                const int L = p.g.n[d];
                const float c = (float)(2 * n0[d] + ts[d] - 1) + 2.0f * g[d];   // twice the centre offset
                if (c > (float)L) n0[d] -= L;
                else if (c < -(float)L) n0[d] += L;
            }
        }
        const float R = v.R;
        const float Rs = R + (float)p.shell_width;
        const float Rn = R + 1.4142135f + 0.02f;
        const float R2 = R * R, Rs2 = Rs * Rs;
        cn[tid] = make_int4(n0[0], n0[1], n0[2], i);
        ca[tid] = make_float4(g[0], g[1], g[2], R2);
        cb[tid] = make_float4(Rs2, Rn * Rn, 1e-5f * (R2 + 1.0f), 1e-5f * (Rs2 + 1.0f));
    }
    __syncthreads();

    const int x = org[0] + threadIdx.x;
    const int y = org[1] + threadIdx.y;
    const int z = org[2] + threadIdx.z;
    const bool valid = x < p.g.n[0] && y < p.g.n[1] && z < p.g.n[2];
    bool solid = false;
    bool near_fluid = false;   // into the particle-link list of the next step
    bool miss_solid = false;   // into the missing-link list of the next step
    unsigned int entry = 0;
    if (valid) {
        const long long idx = ((long long)z * p.g.n[1] + y) * p.g.n[0] + x;
        const int cpos[3] = {x, y, z};
        const int lx = threadIdx.x, ly = threadIdx.y, lz = threadIdx.z;
        const bool any_small = p.small[0] | p.small[1] | p.small[2];
        int own = 0x7fffffff;
        bool shell = false;
        int nnear = 0;
        for (int k = 0; k < ncand; ++k) {
            const int4 Nn = cn[k];
            const float4 A = ca[k];
            int n[3] = {Nn.x + lx, Nn.y + ly, Nn.z + lz};
            if (any_small) {
                const float gg[3] = {A.x, A.y, A.z};
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (!p.small[d]) continue;
                    // minimum image decided on 2 (n + g) against L
                    const int L = p.g.n[d];
                    const float tw = (float)(2 * n[d]) + 2.0f * gg[d];
                    if (tw > (float)L) n[d] -= L;
                    else if (tw < -(float)L) n[d] += L;
                }
            }
            const float dx = (float)n[0] + A.x, dy = (float)n[1] + A.y, dz = (float)n[2] + A.z;
            const float d2f = (dx * dx + dy * dy) + dz * dz;
            const float4 B = cb[k];
            if (d2f <= B.y) ++nnear;
            if (d2f > B.x + B.w) continue;
            const bool exact_needed = fabsf(d2f - A.w) <= B.z || fabsf(d2f - B.x) <= B.w;
            bool inside, in_shell;
            const int id = Nn.w;
            if (!exact_needed) {
                inside = d2f < A.w;
                in_shell = !inside && d2f < B.x;
            } else {
                const double R = p.P.R[id];
                double dd[3];
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    dd[d] = min_image_dd(((double)cpos[d] + 0.5) - p.P.x[3 * id + d], p.g.n[d], p.g.per[d]);
                const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dd[0], dd[0]), __dmul_rn(dd[1], dd[1])),
                                            __dmul_rn(dd[2], dd[2]));
                const double rs = __dadd_rn(R, p.shell_width);
                inside = d2 <= __dmul_rn(R, R);
                in_shell = !inside && d2 <= __dmul_rn(rs, rs);
            }
            if (inside) { if (id < own) own = id; }
            else if (in_shell) shell = true;
        }
        bool wall_adj = false;
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (!p.g.per[d] && (cpos[d] == 0 || cpos[d] == p.g.n[d] - 1)) wall_adj = true;
        const uint8_t old = p.flags[idx];
        uint8_t nf = 0;
        if (own != 0x7fffffff) {
            solid = true;
            nf = FL_SOLID;
            if (nnear >= 2 || wall_adj) {
                nf |= FL_MISS;
                miss_solid = true;
            }
            p.owner[idx] = own;
        } else {
            if (shell) nf |= FL_SHELL;
            if (nnear >= 1) {
                nf |= FL_NEAR;
                near_fluid = true;
            }
            if (old & FL_SOLID) {
                nf |= FL_NEWFLUID;
                int slot = atomicAdd(p.refill_count, 1);
                if (slot < p.refill_cap) p.refill_list[slot] = (unsigned int)idx;
                else atomicOr(p.status, ST_REFILL_OVERFLOW);
            }
        }
        p.flags[idx] = nf;
        entry = (unsigned int)idx;
    }
    // block-aggregated appends to the particle-link and missing-link lists
    __shared__ int s_warp[16];
    __shared__ int s_base;
    block_append(near_fluid, entry, p.near_list, p.near_count, p.near_cap, p.status, s_warp, &s_base);
    block_append(miss_solid, entry, p.miss_list, p.miss_count, p.miss_cap, p.status, s_warp, &s_base);
    unsigned bal = __ballot_sync(0xffffffffu, solid);
    if ((threadIdx.x & 31) == 0 && bal) atomicAdd(&nsolid_blk, (unsigned)__popc(bal));
    __syncthreads();
    if (tid == 0 && nsolid_blk) atomicAdd(p.n_solid, (unsigned long long)nsolid_blk);
}

void launch_map(const MapParams& p, cudaStream_t st) {
    dim3 block(TILE_X, TILE_Y, TILE_Z);
    dim3 grid(p.ntile[0], p.ntile[1], p.ntile[2]);
    map_kernel<<<grid, block, 0, st>>>(p);
}

// ------------------------------------------------------------ refill

template <typename S>
__global__ void refill_kernel(const RefillParams p) {
    using T = typename Store<S>::T;
    const int count = min(*p.count, p.cap);
    const S* f = static_cast<const S*>(p.f);
    S* fw = static_cast<S*>(p.f);
    const long long N = p.g.ncells;
    const int nx = p.g.n[0], ny = p.g.n[1];
    const T ax = (T)p.accel[0], ay = (T)p.accel[1], az = (T)p.accel[2];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        const long long idx = p.list[k];
        const int x = (int)(idx % nx);
        const int y = (int)((idx / nx) % ny);
        const int z = (int)(idx / ((long long)nx * ny));
        const int cpos[3] = {x, y, z};
        const int i = p.owner[idx];
        T drho_sum = T(0);    // neighbour densities minus rho0 (shifted, no cancellation)
        int nnb = 0;
        T uax[6][3];      // velocities of the axis neighbours +x -x +y -y +z -z
        bool okax[6] = {false, false, false, false, false, false};
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            int nb[3] = {x + cx(q), y + cy(q), z + cz(q)};
            bool out = false;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (p.g.per[d]) nb[d] = wrap_idx(nb[d], p.g.n[d]);
                else if (nb[d] < 0 || nb[d] >= p.g.n[d]) out = true;
            }
            if (out) continue;
            const long long j = ((long long)nb[2] * ny + nb[1]) * nx + nb[0];
            const uint8_t fl = p.flags[j];
            if (fl & (FL_SOLID | FL_NEWFLUID)) continue;
            T dr = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
            for (int r = 0; r < Q; ++r) {
                const T v = Store<S>::load(f + (long long)r * N + j);
                dr += v;
                jx += (T)cx(r) * v;
                jy += (T)cy(r) * v;
                jz += (T)cz(r) * v;
            }
            drho_sum += dr;
            ++nnb;
            const int slot = c2(q) != 1 ? -1 : (cx(q) == 1 ? 0 : cx(q) == -1 ? 1 : cy(q) == 1 ? 2 : cy(q) == -1 ? 3 : cz(q) == 1 ? 4 : 5);
            if (slot >= 0) {
                okax[slot] = true;
                uax[slot][0] = jx - T(0.5) * ax;
                uax[slot][1] = jy - T(0.5) * ay;
                uax[slot][2] = jz - T(0.5) * az;
            }
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
        const T coef = T(1) / (T(3) * (T)p.s_nu);   // c_s^2 / s_nu
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const T c[3] = {(T)cx(q), (T)cy(q), (T)cz(q)};
            T second = T(0);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const T pab = rb * ut[a] * ut[b] - rb * coef * (g[a][b] + g[b][a]);
                    second += pab * (c[a] * c[b] - (a == b ? T(1) / T(3) : T(0)));
                }
            const T cu = c[0] * ut[0] + c[1] * ut[1] + c[2] * ut[2];
            // f_q - w_q written without forming f_q: w_q (rho_bar - 1) + ...
            const T dfq = wq<T>(q) * (drb + T(3) * rb * cu + T(4.5) * second);
            Store<S>::store(fw + (long long)q * N + idx, dfq);
        }
    }
}

void launch_refill(const RefillParams& p, cudaStream_t st) {
    const int blocks = 152 * 4, threads = 128;
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

}  // namespace lbmdem
