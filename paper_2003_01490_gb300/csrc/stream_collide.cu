// stream_collide.cu -- the dense kernel of one lattice Boltzmann step with
// moving particles (Algorithm 1, lines 1-3): one thread per cell, pull
// streaming (Eq. (2)), the particle links of the cell (CLI moving no-slip
// condition, Eq. (14), and momentum exchange, Eqs. (15)-(17)), halfway
// bounce-back on the walls of the box (Eq. (14), delta = 1/2, wall velocity),
// then the two-relaxation-time collision (Eq. (10), magic parameter
// Eq. (11)) with Guo forcing; in TRT+aB shell cells (Sec. 2.3.2) and for
// Lambda_b,bulk != 1 the two bulk moments m4, m5 relax with s_b (Eq. (12))
// through a rank-2 correction in moment space.
//
// PDFs are stored shifted (f_q - w_q) in SoA layout f[q][z][y][x], read from
// one buffer and written to the other (fluid cells only). Every PDF slot of a
// solid cell holds a NaN marker written by the mapping (with the owning
// particle in its payload for 4- and 8-byte storage), so the pull of a fluid
// cell x finds its particle links for free: direction q is a link exactly
// when the value pulled from y = x - c_q is a marker. The warp then spreads
// its links evenly over its lanes; each link's CLI value f_q(x, t+1) (link
// fraction delta_p from the ray-sphere intersection; bounce-back, delta = 1/2
// in the coefficients, when x + c_q is not fluid) goes through shared memory
// to the thread of x, and its force and torque are summed per lane while the
// particle stays the same, then per warp by particle (lanes with the same
// particle found with match_any) and added atomically.
//
// Per-particle sums. Float64 storage: float64 partial sums, float64 atomics.
// Float32 compute: the link force splits into the constant part 2 w_p c_p,
// an integer multiple of c_p / 36, and the small remainder
// c_p (f~_p + f_q) - u_b (f~_p - f_q). The constant part and its torque
// 2 w_p (n + g) x c_p (n the integer offset of the cell from the particle's
// base cell, g the fractional offset common to all links) are summed exactly
// in integers; the remainder is summed per warp in float32 and per particle
// in 64-bit fixed point (scale 2^32) through integer atomics. No float64
// arithmetic runs per cell or link on the float32 path.
#include <cstring>

#include "sc_common.cuh"

// minimum resident blocks per SM requested for the kernel with 4-byte or
// smaller storage (a register cap of 64 at 256 threads); tuned on GB300
#ifndef LBM_SC_MIN_BLOCKS
#define LBM_SC_MIN_BLOCKS 4
#endif
// the same for float64 storage
#ifndef LBM_SC_MIN_BLOCKS_F64
#define LBM_SC_MIN_BLOCKS_F64 2
#endif
// longest chunk of consecutive z planes marched by one block (shorter when
// the box is too small to give every SM several blocks); tuned on GB300
#ifndef LBM_SC_ZCHUNK
#define LBM_SC_ZCHUNK 24
#endif
// x extent of a block (a multiple of 32; 256 / LBM_SC_BX rows in y)
#ifndef LBM_SC_BX
#define LBM_SC_BX 128
#endif
namespace lbmdem {

// a lane's open force sums between rows: particle, float sums and the exact
// integer sums (float32 path) as two 16-bit halves per word; sums that could
// leave 16 bits are flushed to the particle first
template <typename T>
__device__ __forceinline__ void load_sums(Acc<T>& acc, const int* s_key, T (*s_sum)[256], int (*s_int)[256], int tid) {
    acc.key = s_key[tid];
#pragma unroll
    for (int c = 0; c < 6; ++c) acc.f[c] = s_sum[c][tid];
    if (sizeof(T) == 4) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int v = s_int[c][tid];
            acc.k[2 * c] = (int)(short)(v & 0xffff);
            acc.k[2 * c + 1] = v >> 16;
        }
    }
}
template <typename T>
__device__ __forceinline__ void store_sums(Acc<T>& acc, int* s_key, T (*s_sum)[256], int (*s_int)[256], int tid,
                                           const Sinks& sk) {
    if (sizeof(T) == 4) {
        bool big = false;
#pragma unroll
        for (int c = 0; c < 6; ++c) big |= acc.k[c] > 30000 || acc.k[c] < -30000;
        if (big && acc.key >= 0) flush<T>(acc, sk);
#pragma unroll
        for (int c = 0; c < 3; ++c) s_int[c][tid] = (acc.k[2 * c] & 0xffff) | (acc.k[2 * c + 1] << 16);
    }
    s_key[tid] = acc.key;
#pragma unroll
    for (int c = 0; c < 6; ++c) s_sum[c][tid] = acc.f[c];
}

// One tile of bx x (256 / bx) cells in (x, y) from (x0, y0), planes z_begin
// .. z_end - 1 marched in order: the links a warp meets in consecutive rows
// mostly belong to the same spheres, so a lane's force sums (kept in shared
// memory between rows) rarely change particle and the warp commits them once
// per tile. Thread tid of the block's 256 handles column x0 + tid % bx, row
// y0 + tid / bx (warps hold 32 consecutive tids). Cell indices are 32-bit
// (the library limits boxes to 2^31 - 2^24 cells); each PDF array q starts at
// src + q N. s_qi holds the link codes qinfo(q).
// A single-box launch has blocks of (bx, 256 / bx) threads and takes its tile
// from the block index (BATCH false: x0, y0 unused); the batched launch has
// blocks of 256 threads and passes the tile.
template <typename S, typename T, bool BATCH>
__device__ __forceinline__ void sc_tile(const SCArgs<S, T>& a, int x0, int y0, int z_begin, int z_end, int bx,
                                        unsigned char* sc_smem, const int* s_qi) {
    const int nx = a.g.n[0], ny = a.g.n[1], nz = a.g.n[2];
    // bx is 32, 64 or 128
    const int tid = BATCH ? (int)threadIdx.x : (int)(threadIdx.x + blockDim.x * threadIdx.y);
    const int x = BATCH ? x0 + (tid & (bx - 1)) : (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int y = BATCH ? y0 + (tid >> (bx == 128 ? 7 : (bx == 64 ? 6 : 5)))
                        : (int)(blockIdx.y * blockDim.y + threadIdx.y);
    const bool valid = x < nx && y < ny;
    const int plane = nx * ny;
    const long long N = a.g.ncells;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    // dynamic shared memory (sc_smem_bytes): PDFs of the cells of warps with
    // links [q][thread]; per lane the particle of its open force sums (-1:
    // none), the open float sums (F, T) and the exact integer sums (float32
    // path, two 16-bit halves per word); per warp the link entries q | lane << 8
    T (*s_f)[256] = reinterpret_cast<T (*)[256]>(sc_smem);
    T (*s_sum)[256] = reinterpret_cast<T (*)[256]>(sc_smem + Q * 256 * sizeof(T));
    int (*s_int)[256] = reinterpret_cast<int (*)[256]>(sc_smem + (Q + 6) * 256 * sizeof(T));
    int* s_key = reinterpret_cast<int*>(sc_smem + (Q + 6) * 256 * sizeof(T) + (sizeof(T) == 4 ? 3 * 256 * 4 : 0));
    unsigned short (*s_queue)[32 * (Q - 1)] =
        reinterpret_cast<unsigned short (*)[32 * (Q - 1)]>(reinterpret_cast<unsigned char*>(s_key) + 256 * 4);
    const Sinks sk{a.acc_d, a.acc_i, a.acc_k, a.status};
    s_key[tid] = -1;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        s_sum[c][tid] = T(0);
        if (sizeof(T) == 4 && c < 3) s_int[c][tid] = 0;
    }
    bool open = false;   // warp-uniform: some lane of the warp holds sums

    // the 19 pulls of cell (x, y, zz) with periodic wrap (walls are handled
    // below), issued only for a fluid cell
    auto pull_row = [&](int zz, bool fluid_zz, T (&g)[Q]) {
        if (!fluid_zz) return;
        const int idz = zz * plane + y * nx + x;
        const int OX[3] = {x == 0 ? nx - 1 : -1, 0, x == nx - 1 ? 1 - nx : 1};
        const int OY[3] = {y == 0 ? plane - nx : -nx, 0, y == ny - 1 ? nx - plane : nx};
        const int OZ[3] = {zz == 0 ? (nz - 1) * plane : -plane, 0, zz == nz - 1 ? (1 - nz) * plane : plane};
#pragma unroll
        for (int q = 0; q < Q; ++q)
            g[q] = Store<S>::load(a.src + q * N + (idz + OX[1 - cx(q)] + OY[1 - cy(q)] + OZ[1 - cz(q)]));
    };
    for (int z = z_begin; z < z_end; ++z) {
        const int idx = z * plane + y * nx + x;
        T f[Q];
        const uint8_t fl = valid ? a.flags[idx] : FL_SOLID;
        pull_row(z, !(fl & FL_SOLID), f);
        const bool fluid = !(fl & FL_SOLID);
        unsigned lmask = 0;   // pull directions of this cell that are particle links
        if (fluid) {
#pragma unroll
            for (int q = 1; q < Q; ++q)
                if (f[q] != f[q]) lmask |= 1u << q;   // marker of a solid upstream cell
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
                    lmask &= ~(1u << q);
                }
            }
        }
        // particle links of the warp, spread evenly over its lanes: each lane
        // with links queues (direction, lane) entries in shared memory at its
        // prefix-sum offset
        if (a.np > 0 && __any_sync(FULL, lmask != 0)) {
            const int cnt = __popc(lmask);
            const int incl = warp_incl_scan(cnt, lane);
            const int total = __shfl_sync(FULL, incl, 31);
            // the cell's PDFs wait in shared memory (freeing their registers for
            // the link work); each link's CLI value lands in its cell's slot
#pragma unroll
            for (int q = 0; q < Q; ++q) s_f[q][tid] = f[q];
            // entries q | lane << 8
            unsigned short* queue = s_queue[tid >> 5];
            {
                unsigned mm = lmask;
                int pos = incl - cnt;
                while (mm) {
                    const int q = __ffs(mm) - 1;
                    mm &= mm - 1;
                    queue[pos++] = (unsigned short)(q | (lane << 8));
                }
            }
            __syncwarp();
            Acc<T> acc;
            load_sums<T>(acc, s_key, s_sum, s_int, tid);
            // lane l takes the m consecutive entries l m .. l m + m - 1
            const int m = (total + 31) >> 5;
            for (int j = 0; j < m; ++j) {
                const int k = lane * m + j;
                const unsigned e = k < total ? queue[k] : 0u;
                const int q = (int)(e & 31u), src = (int)(e >> 8);
                const unsigned lm_src = __shfl_sync(FULL, lmask, src);
                if (k < total) {
                    const int st = tid - lane + src;
                    const int qi = s_qi[q];
                    // the particle from the marker's payload, still in the slot
                    // (0: look it up in the owner array)
                    int key1 = 0;
                    if constexpr (sizeof(S) >= 4) key1 = marker_owner(s_f[q][st]) + 1;
                    // f_p pulled by the same cell: f~_p(x + c_q) (read before any
                    // link of direction p could overwrite it; such a link makes
                    // x + c_q solid and its value unused)
                    const T fdown_raw = s_f[(qi >> 6) & 31][st];
                    s_f[q][st] = link_value<S, T>(a, x - lane + src, y, z, q, qi, key1, lm_src, fdown_raw, acc, sk);
                }
            }
            store_sums<T>(acc, s_key, s_sum, s_int, tid, sk);
            open = true;
            __syncwarp();
#pragma unroll
            for (int q = 0; q < Q; ++q) f[q] = s_f[q][tid];
        }
        // solid cells store nothing: their slots keep the marker of the mapping
        if (fluid) {
            collide_store<S, T>(a, f, fl, N, idx);
        }

    }
    if (open) {   // warp-uniform
        Acc<T> acc;
        load_sums<T>(acc, s_key, s_sum, s_int, tid);
        commit<T>(acc, sk);
    }
}


// link codes of the directions into shared memory (before the first tile)
__device__ __forceinline__ void load_qinfo(int* s_qi) {
    const int t = threadIdx.x + blockDim.x * threadIdx.y;
    if (t < Q) {
        constexpr int QI[Q] = {qinfo(0), qinfo(1), qinfo(2), qinfo(3), qinfo(4), qinfo(5), qinfo(6),
                               qinfo(7), qinfo(8), qinfo(9), qinfo(10), qinfo(11), qinfo(12), qinfo(13),
                               qinfo(14), qinfo(15), qinfo(16), qinfo(17), qinfo(18)};
        s_qi[t] = QI[t];
    }
}

// One box: block (bx, 256 / bx) tiles from blockIdx.x, blockIdx.y, a chunk of
// a.zchunk planes from blockIdx.z.
template <typename S, typename T>
__global__ void __launch_bounds__(256, sizeof(S) == 8 ? LBM_SC_MIN_BLOCKS_F64 : LBM_SC_MIN_BLOCKS)
    stream_collide_kernel(const SCArgs<S, T> a) {
    extern __shared__ __align__(16) unsigned char sc_smem[];
    __shared__ int s_qi[Q];
    load_qinfo(s_qi);
    __syncthreads();
    const int z_begin = blockIdx.z * a.zchunk;
    sc_tile<S, T, false>(a, 0, 0, z_begin, min(a.g.n[2], z_begin + a.zchunk), (int)blockDim.x, sc_smem, s_qi);
}

// Many boxes in one persistent launch: block b takes the work items b,
// b + gridDim.x, ... of the table (instance, x0, y0, z0), copies the
// arguments of the item's instance into shared memory and runs its tile
// (a.bx x 256 / a.bx cells, a.zchunk planes from z0).
template <typename S, typename T>
__global__ void __launch_bounds__(256, sizeof(S) == 8 ? LBM_SC_MIN_BLOCKS_F64 : LBM_SC_MIN_BLOCKS)
    stream_collide_batch_kernel(const SCArgs<S, T>* __restrict__ args, const int4* __restrict__ items, int n_items) {
    extern __shared__ __align__(16) unsigned char sc_smem[];
    __shared__ int s_qi[Q];
    __shared__ __align__(16) SCArgs<S, T> s_a;
    load_qinfo(s_qi);
    constexpr int WORDS = (int)(sizeof(SCArgs<S, T>) / 4);
    static_assert(sizeof(SCArgs<S, T>) % 4 == 0, "argument block copied in words");
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int4 item = items[it];
        __syncthreads();                 // the previous tile is done with s_a
        const int* src = reinterpret_cast<const int*>(args + item.x);
        int* dst = reinterpret_cast<int*>(&s_a);
        for (int w = threadIdx.x; w < WORDS; w += blockDim.x) dst[w] = src[w];
        __syncthreads();
        sc_tile<S, T, true>(s_a, item.y, item.z, item.w, min(s_a.g.n[2], item.w + s_a.zchunk), s_a.bx, sc_smem,
                            s_qi);
    }
}

// bytes of dynamic shared memory of the kernel (256 threads)
template <typename T>
constexpr size_t sc_smem_bytes() {
    return (Q + 6) * 256 * sizeof(T) + (sizeof(T) == 4 ? 3 * 256 * 4 : 0) + 256 * 4 + 8 * 32 * (Q - 1) * 2;
}

template <typename S>
void launch_stream_collide_t(const LbmStepParams& p, cudaStream_t st) {
    using T = typename Store<S>::T;
    SCArgs<S, T> a;
    fill_sc_args<S, T>(p, a);
    const int nx = p.g.n[0];
    int bx = nx >= LBM_SC_BX ? LBM_SC_BX : ((nx + 31) / 32) * 32;
    if (p.tile_bx > 0) bx = p.tile_bx;
    int by = 256 / bx;
    a.bx = bx;
    dim3 block(bx, by, 1);
    const int bxy = ((nx + bx - 1) / bx) * ((p.g.n[1] + by - 1) / by);
    // at least 4 blocks per SM where the box allows, else shorter chunks
    const long long want = 4LL * (p.num_sms > 0 ? p.num_sms : 152);
    int zc = (int)((long long)bxy * p.g.n[2] / want);
    a.zchunk = zc < 1 ? 1 : (zc > LBM_SC_ZCHUNK ? LBM_SC_ZCHUNK : zc);
    if (p.zchunk > 0) a.zchunk = p.zchunk;
    dim3 grid((nx + bx - 1) / bx, (p.g.n[1] + by - 1) / by, (p.g.n[2] + a.zchunk - 1) / a.zchunk);
    constexpr size_t smem = sc_smem_bytes<T>();
    stream_collide_kernel<S, T><<<grid, block, smem, st>>>(a);
}

// ------------------------------------------------------------ batched launch

template <typename S>
static void fill_batch_args_t(const LbmStepParams& p, int tile_bx, int zchunk, void* out) {
    using T = typename Store<S>::T;
    SCArgs<S, T> a;
    fill_sc_args<S, T>(p, a);
    a.bx = tile_bx;
    a.zchunk = zchunk;
    std::memcpy(out, &a, sizeof(a));
}

size_t batch_args_bytes(int storage) {
    switch (storage) {
        case 0: return sizeof(SCArgs<double, double>);
        case 1: return sizeof(SCArgs<float, float>);
        case 2: return sizeof(SCArgs<__half, float>);
        default: return sizeof(SCArgs<__nv_bfloat16, float>);
    }
}

void fill_batch_args(const LbmStepParams& p, int tile_bx, int zchunk, void* out) {
    switch (p.storage) {
        case 0: fill_batch_args_t<double>(p, tile_bx, zchunk, out); break;
        case 1: fill_batch_args_t<float>(p, tile_bx, zchunk, out); break;
        case 2: fill_batch_args_t<__half>(p, tile_bx, zchunk, out); break;
        default: fill_batch_args_t<__nv_bfloat16>(p, tile_bx, zchunk, out); break;
    }
}

int default_tile_bx(int nx) { return nx >= LBM_SC_BX ? LBM_SC_BX : ((nx + 31) / 32) * 32; }

template <typename S>
static void launch_batch_t(const void* d_args, const int4* d_items, int n_items, int grid, cudaStream_t st) {
    using T = typename Store<S>::T;
    constexpr size_t smem = sc_smem_bytes<T>();
    stream_collide_batch_kernel<S, T>
        <<<grid, 256, smem, st>>>(static_cast<const SCArgs<S, T>*>(d_args), d_items, n_items);
}

void launch_stream_collide_batch(int storage, const void* d_args, const int4* d_items, int n_items, int grid,
                                 cudaStream_t st) {
    switch (storage) {
        case 0: launch_batch_t<double>(d_args, d_items, n_items, grid, st); break;
        case 1: launch_batch_t<float>(d_args, d_items, n_items, grid, st); break;
        case 2: launch_batch_t<__half>(d_args, d_items, n_items, grid, st); break;
        default: launch_batch_t<__nv_bfloat16>(d_args, d_items, n_items, grid, st); break;
    }
}

template <typename S>
cudaError_t prepare_t() {
    using T = typename Store<S>::T;
    constexpr size_t smem = sc_smem_bytes<T>();
    if (smem <= 48 * 1024) return cudaSuccess;
    // float64 storage: above the default dynamic shared memory limit
    cudaError_t e =
        cudaFuncSetAttribute(stream_collide_kernel<S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(stream_collide_batch_kernel<S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

cudaError_t prepare_stream_collide(int storage) {
    cudaError_t e;
    switch (storage) {
        case 0: e = prepare_t<double>(); break;
        case 1: e = prepare_t<float>(); break;
        case 2: e = prepare_t<__half>(); break;
        default: e = prepare_t<__nv_bfloat16>(); break;
    }
    return e == cudaSuccess ? prepare_stream_collide_staged(storage) : e;
}

void launch_stream_collide(const LbmStepParams& p, cudaStream_t st) {
    // on request, for 4- and 2-byte formats on boxes whose rows start on
    // 16-byte boundaries: the kernel with bulk-copy staging
    // (stream_collide_staged.cu)
    if (p.use_staged && staged_applicable(p)) {
        launch_stream_collide_staged(p, st);
        return;
    }
    switch (p.storage) {
        case 0: launch_stream_collide_t<double>(p, st); break;
        case 1: launch_stream_collide_t<float>(p, st); break;
        case 2: launch_stream_collide_t<__half>(p, st); break;
        default: launch_stream_collide_t<__nv_bfloat16>(p, st); break;
    }
}


}  // namespace lbmdem
