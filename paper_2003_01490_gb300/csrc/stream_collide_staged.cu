// stream_collide_staged.cu -- the dense kernel of one lattice Boltzmann step
// with moving particles (Algorithm 1, lines 1-3) for the 4- and 2-byte PDF
// formats, with the pulled PDFs staged in shared memory by bulk asynchronous
// copies.
//
// The arithmetic is that of stream_collide.cu (sc_common.cuh: pull
// streaming, Eq. (2); CLI moving no-slip condition and momentum exchange,
// Eqs. (14)-(17); wall bounce-back; TRT(+aB) collision with Guo forcing); what
// differs is how the data moves:
//
//  * A block owns a tile of TX x TY cells in (x, y) and marches chunks of z
//    planes. For every plane and direction q the cells of the tile pull from
//    the tile shifted by -c_q: TY rows of TX cells plus a 16-byte halo on each
//    side in x. One producer warp copies these 19 x TY rows (global -> shared,
//    cp.async.bulk, 16-byte aligned and sized; periodic wraps in x, y and z
//    resolved in the copy addresses) into a ring of SC_STAGES stages, each
//    completed by a transaction-count mbarrier; the consumers release a stage
//    through a second mbarrier. Memory latency is hidden by the copies in
//    flight, not by the number of resident threads.
//  * TX x TY / 32 consumer warps read their 19 pulls from shared memory (one
//    load with a constant offset each), find the particle links from the NaN
//    markers as before, put each link's CLI value into a per-warp buffer
//    (the stages are only read, so the copy engine and the warps never write
//    the same shared memory), collide, and store every cell of the row: fluid cells their new
//    PDFs, solid cells their own marker again (pulled from the rest direction
//    of the stage), so the stores fill whole 32-byte sectors.
//  * Blocks are persistent: block b takes work items b, b + gridDim.x, ...
//    (tile, z chunk); the producer runs ahead across item boundaries, so the
//    ring never drains between items. A lane's particle-force sums stay in
//    registers for a whole item and are committed per warp at its end.
//
// Every wait on an mbarrier has a deadline (globaltimer): when it passes, the
// waiting warp sets ST_TIMEOUT in the device status word and leaves; the
// producer then still waits (again with a deadline) for the copies it has
// issued before the block exits, so no copy outlives its shared memory.
#include <algorithm>

#include "sc_common.cuh"

namespace lbmdem {

constexpr int SC_STAGES = 4;
constexpr unsigned long long SC_WAIT_NS = 1000000000ull;   // 1 s deadline per wait

template <typename S, int TX_, int TY_>
struct StagedShape {
    static constexpr int TX = TX_, TY = TY_;
    static constexpr int H = 16 / (int)sizeof(S);               // halo elements: 16 bytes
    static constexpr int RE = TX + 2 * H;                        // elements per row slot
    static constexpr int ROWB = RE * (int)sizeof(S);             // bytes per row slot (multiple of 16)
    static constexpr int FLB = TY * TX;                          // flag bytes per stage
    static constexpr int SB = (Q * TY * ROWB + FLB + 127) / 128 * 128; // bytes per stage: rows, then flags
    static constexpr int NW = TX * TY / 32;                      // consumer warps
    static constexpr int WX = TX / 32;                           // consumer warps per row
    static constexpr int THREADS = (NW + 1) * 32;                // + the producer warp
    static constexpr int QUEUE_B = NW * 32 * (Q - 1) * 2;        // link queues
    static constexpr int LINK_B = NW * (Q - 1) * 32 * 4;         // link values per warp [q - 1][lane]
    static constexpr int SMEM = SC_STAGES * SB + 2 * SC_STAGES * 8 + LINK_B + QUEUE_B + 2 * Q * 4;
};

struct StagedPlan {
    int flags_bulk;    // 1: flag rows start on 16-byte boundaries (nx % 16 == 0) and travel with the copies
    int ntile[2];      // tiles in x, y
    int zchunk;        // z planes per work item
    int nzc;           // chunks per column
    int n_items;       // ntile[0] ntile[1] nzc
};

// ----------------------------------------------------------------- PTX
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// wait for the phase of the given parity to complete, at most SC_WAIT_NS
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > SC_WAIT_NS) return false;
    }
    return true;
}
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// shared-memory element access in the storage format
template <typename S> __device__ __forceinline__ typename Store<S>::T lds(const S* p);
template <> __device__ __forceinline__ float lds<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float lds<__half>(const __half* p) { return __half2float(*p); }
template <> __device__ __forceinline__ float lds<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// work item -> tile origin and z range
struct Item {
    int x0, y0, z0, z1;
};
__device__ __forceinline__ Item item_of(int it, const StagedPlan& pl, int TX, int TY, int nz) {
    const int ntiles = pl.ntile[0] * pl.ntile[1];
    const int c = it / ntiles, t = it - c * ntiles;
    Item r;
    r.x0 = (t % pl.ntile[0]) * TX;
    r.y0 = (t / pl.ntile[0]) * TY;
    r.z0 = c * pl.zchunk;
    r.z1 = min(nz, r.z0 + pl.zchunk);
    return r;
}

// The copies of one row slot (direction q, tile row ty) of plane z: the
// source row y0 + ty - cy(q) of plane z - cz(q) (wrapped on periodic axes; a
// row beyond a wall is not copied, its cells use the wall condition), x from
// x0 - H to x0 + TX + H clipped to the box, plus the periodic halos at the
// box's x faces. Returns the bytes; issues the copies when bar != 0.
template <typename S, int TX, int TY>
__device__ __forceinline__ uint32_t row_copies(const S* __restrict__ src, const Geom& g, long long N, int q, int ty,
                                               int x0, int y0, int z, uint32_t slot, uint32_t bar) {
    using SH = StagedShape<S, TX, TY>;
    constexpr int H = SH::H;
    constexpr int es = (int)sizeof(S);
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    if (y0 + ty >= ny) return 0;   // tile row beyond the box
    // q is chosen at run time here: its components from the packed 2-bit words
    int ys = y0 + ty - dir_c(pack_dirs(1), q);
    int zs = z - dir_c(pack_dirs(2), q);
    if (ys < 0 || ys >= ny) {
        if (!g.per[1]) return 0;
        ys = ys < 0 ? ys + ny : ys - ny;
    }
    if (zs < 0 || zs >= nz) {
        if (!g.per[2]) return 0;
        zs = zs < 0 ? zs + nz : zs - nz;
    }
    const S* row = src + (long long)q * N + ((long long)zs * ny + ys) * nx;
    const int xa = max(x0 - H, 0), xb = min(x0 + TX + H, nx);
    uint32_t bytes = (uint32_t)(xb - xa) * es;
    if (bar) bulk_copy_g2s(slot + (uint32_t)(xa - (x0 - H)) * es, row + xa, (uint32_t)(xb - xa) * es, bar);
    if (g.per[0] && x0 == 0) {
        // x = -H .. -1 wraps to nx - H .. nx - 1
        bytes += H * es;
        if (bar) bulk_copy_g2s(slot, row + (nx - H), H * es, bar);
    }
    if (g.per[0] && x0 + TX >= nx) {
        // x = nx .. nx + H - 1 wraps to 0 .. H - 1
        bytes += H * es;
        if (bar) bulk_copy_g2s(slot + (uint32_t)(nx - x0 + H) * es, row, H * es, bar);
    }
    return bytes;
}

// The flags of tile row ty of plane z: TX bytes from x0, rounded up to whole
// 16-byte units (the flag array is padded so the last row may be over-read).
template <int TX>
__device__ __forceinline__ uint32_t flag_copy(const uint8_t* __restrict__ flags, const Geom& g, int ty, int x0,
                                              int y0, int z, uint32_t dst, uint32_t bar) {
    const int nx = g.n[0], ny = g.n[1];
    if (y0 + ty >= ny) return 0;
    const int n = (min(TX, nx - x0) + 15) & ~15;
    if (bar) bulk_copy_g2s(dst, flags + ((long long)z * ny + y0 + ty) * nx + x0, (uint32_t)n, bar);
    return (uint32_t)n;
}

template <typename S, typename T, int TX, int TY>
__global__ void __launch_bounds__(StagedShape<S, TX, TY>::THREADS, 2)
    stream_collide_staged_kernel(const SCArgs<S, T> a, const StagedPlan pl) {
    using SH = StagedShape<S, TX, TY>;
    constexpr int H = SH::H, RE = SH::RE, NW = SH::NW, WX = SH::WX;
    const int nx = a.g.n[0], ny = a.g.n[1], nz = a.g.n[2];
    const int plane = nx * ny;
    const long long N = a.g.ncells;
    const unsigned FULL = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // after a timed-out wait in an earlier launch the context is in error:
    // leave at once instead of waiting again
    if (*reinterpret_cast<volatile int*>(a.status) & ST_TIMEOUT) return;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* ring = smem;
    uint64_t* full_bar = reinterpret_cast<uint64_t*>(smem + SC_STAGES * SH::SB);
    uint64_t* empty_bar = full_bar + SC_STAGES;
    T* links = reinterpret_cast<T*>(empty_bar + SC_STAGES);   // [warp][q - 1][lane], float or double
    unsigned short* queues = reinterpret_cast<unsigned short*>(reinterpret_cast<unsigned char*>(empty_bar + SC_STAGES) +
                                                               SH::LINK_B);
    int* s_qi = reinterpret_cast<int*>(queues + NW * 32 * (Q - 1));
    int* s_off = s_qi + Q;   // element offset of the pull of direction q within a stage, cell at (0, 0)
    if (threadIdx.x < Q) {
        // the link code of direction q (layout of qinfo()) from the constant tables
        const int q = threadIdx.x;
        s_qi[q] = (k_c[q][0] + 1) | ((k_c[q][1] + 1) << 2) | ((k_c[q][2] + 1) << 4) | ((int)k_opp[q] << 6);
        s_off[q] = q * TY * RE + H - k_c[q][0];
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < SC_STAGES; ++s) {
            mbar_init(smem_addr(full_bar + s), 1);
            mbar_init(smem_addr(empty_bar + s), NW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == NW) {
        // ------------------------------------------------------------ producer
        const S* src = a.src;
        int i = 0;
        bool ok = true;
        for (int it = blockIdx.x; it < pl.n_items && ok; it += gridDim.x) {
            const Item r = item_of(it, pl, TX, TY, nz);
            for (int z = r.z0; z < r.z1; ++z, ++i) {
                const int s = i % SC_STAGES;
                if (i >= SC_STAGES && !mbar_wait(smem_addr(empty_bar + s), ((i / SC_STAGES) - 1) & 1)) {
                    ok = false;
                    break;
                }
                const uint32_t stage = smem_addr(ring + s * SH::SB);
                const uint32_t bar = smem_addr(full_bar + s);
                // the Q x TY row slots, spread over the lanes
                uint32_t bytes = 0;
                for (int k = lane; k < Q * TY; k += 32) {
                    const int q = k / TY, ty = k - q * TY;
                    bytes += row_copies<S, TX, TY>(src, a.g, N, q, ty, r.x0, r.y0, z, 0u, 0u);
                }
                if (pl.flags_bulk && lane < TY) bytes += flag_copy<TX>(a.flags, a.g, lane, r.x0, r.y0, z, 0u, 0u);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(FULL, bytes, o);
                if (lane == 0) mbar_arrive_expect_tx(bar, bytes);
                __syncwarp();
                for (int k = lane; k < Q * TY; k += 32) {
                    const int q = k / TY, ty = k - q * TY;
                    row_copies<S, TX, TY>(src, a.g, N, q, ty, r.x0, r.y0, z,
                                          stage + (uint32_t)(k * SH::ROWB), bar);
                }
                if (pl.flags_bulk && lane < TY)
                    flag_copy<TX>(a.flags, a.g, lane, r.x0, r.y0, z, stage + (uint32_t)(Q * TY * SH::ROWB + lane * TX), bar);
            }
        }
        if (!ok && lane == 0) atomicOr(a.status, ST_TIMEOUT);
        // no copy may outlive the block's shared memory: wait for the last
        // issued stages (their phases complete when their bytes have landed)
        for (int j = max(0, i - SC_STAGES); j < i; ++j) {
            if (!mbar_wait(smem_addr(full_bar + j % SC_STAGES), (j / SC_STAGES) & 1)) {
                if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
                break;
            }
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    const int tx = lane + 32 * (warp % WX), ty = warp / WX;
    const int tid = threadIdx.x;
    const Sinks sk{a.acc_d, a.acc_i, a.acc_k, a.status};
    unsigned short* queue = queues + warp * 32 * (Q - 1);
    T* wlink = links + warp * (Q - 1) * 32;   // this warp's link values [q - 1][lane]
    int i = 0;
    for (int it = blockIdx.x; it < pl.n_items; it += gridDim.x) {
        const Item r = item_of(it, pl, TX, TY, nz);
        const int x = r.x0 + tx, y = r.y0 + ty;
        const bool valid = x < nx && y < ny;
        Acc<T> acc;
        bool open = false;   // warp-uniform: some lane holds force sums
        const T ax = a.accel[0], ay = a.accel[1], az = a.accel[2];   // body force of the step
        // flags through the copies, or (rows not 16-byte aligned) loaded one
        // plane ahead from global memory
        uint8_t fl_next = (!pl.flags_bulk && valid) ? a.flags[r.z0 * plane + y * nx + x] : FL_SOLID;
        for (int z = r.z0; z < r.z1; ++z, ++i) {
            const int idx = z * plane + y * nx + x;
            const int s = i % SC_STAGES;
            uint8_t fl = fl_next;
            if (!pl.flags_bulk && valid && z + 1 < r.z1) fl_next = a.flags[idx + plane];
            if (!mbar_wait(smem_addr(full_bar + s), (i / SC_STAGES) & 1)) {
                if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
                return;
            }
            S* stage = reinterpret_cast<S*>(ring + s * SH::SB);
            S* mine = stage + ty * RE + tx;   // + s_off[q] -> this cell's pull of direction q
            if (pl.flags_bulk) fl = valid ? ring[s * SH::SB + Q * TY * SH::ROWB + ty * TX + tx] : FL_SOLID;
            const bool fluid = valid && !(fl & FL_SOLID);
            T f[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) f[q] = lds<S>(mine + (q * TY * RE + H - cx(q)));
            unsigned lmask = 0;
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
            // particle links of the warp, spread evenly over its lanes; each
            // link's CLI value goes to the warp's link buffer, slot (q, cell)
            if (a.np > 0 && __any_sync(FULL, lmask != 0)) {
                const int cnt = __popc(lmask);
                const int incl = warp_incl_scan(cnt, lane);
                const int total = __shfl_sync(FULL, incl, 31);
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
                const int m = (total + 31) >> 5;
                for (int j = 0; j < m; ++j) {
                    const int k = lane * m + j;
                    const unsigned e = k < total ? queue[k] : 0u;
                    const int q = (int)(e & 31u), src = (int)(e >> 8);
                    const unsigned lm_src = __shfl_sync(FULL, lmask, src);
                    if (k < total) {
                        const int qi = s_qi[q];
                        const int p = (qi >> 6) & 31;
                        S* cell = stage + ty * RE + (tx - lane + src);
                        int key1 = 0;
                        if constexpr (sizeof(S) >= 4) key1 = marker_owner(lds<S>(cell + s_off[q])) + 1;
                        // f~_p(x + c_q), the cell's own pull in direction p (a link
                        // of direction p would make x + c_q solid and it unused)
                        const T fdown_raw = lds<S>(cell + s_off[p]);
                        wlink[(q - 1) * 32 + src] =
                            link_value<S, T>(a, x - lane + src, y, z, q, qi, key1, lm_src, fdown_raw, acc, sk);
                    }
                }
                open = true;
                __syncwarp();
                if (lmask) {
#pragma unroll
                    for (int q = 1; q < Q; ++q)
                        if ((lmask >> q) & 1u) f[q] = wlink[(q - 1) * 32 + lane];
                }
            }
            // release the stage: this warp only read it
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(empty_bar + s));
            if (valid) {
                if (fluid) {
                    if (!collide_cell_a<S, T>(a, f, fl, ax, ay, az)) atomicOr(a.status, ST_UNSTABLE);
                } else {
                    // a solid cell keeps its marker: its own value, pulled
                    // through the rest direction
#pragma unroll
                    for (int q = 1; q < Q; ++q) f[q] = f[0];
                }
#pragma unroll
                for (int q = 0; q < Q; ++q) Store<S>::store(a.dst + q * N + idx, f[q]);
            }
        }
        if (open) commit<T>(acc, sk);
    }
    (void)tid;
}

// tile of the staged kernel for a box (x extent rounded up to whole warps)
static int staged_tx(int nx) { return nx > 64 ? 128 : (nx > 32 ? 64 : 32); }

template <typename S, int TX, int TY>
static cudaError_t staged_prepare() {
    using T = typename Store<S>::T;
    return cudaFuncSetAttribute(stream_collide_staged_kernel<S, T, TX, TY>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, StagedShape<S, TX, TY>::SMEM);
}

template <typename S>
static cudaError_t staged_prepare_all() {
    cudaError_t e = staged_prepare<S, 128, 2>();
    if (e == cudaSuccess) e = staged_prepare<S, 64, 4>();
    if (e == cudaSuccess) e = staged_prepare<S, 32, 8>();
    return e;
}

cudaError_t prepare_stream_collide_staged(int storage) {
    switch (storage) {
        case 1: return staged_prepare_all<float>();
        case 2: return staged_prepare_all<__half>();
        case 3: return staged_prepare_all<__nv_bfloat16>();
        default: return cudaSuccess;
    }
}

bool staged_applicable(const LbmStepParams& p) {
    if (p.storage < 1 || p.storage > 3) return false;
    const int es = p.storage == 1 ? 4 : 2;
    // rows start on 16-byte boundaries; the box is at least one halo wide
    return (p.g.n[0] * es) % 16 == 0 && p.g.n[0] >= 16 / es && p.g.n[1] >= 1;
}

template <typename S, int TX, int TY>
static void staged_launch(const SCArgs<S, typename Store<S>::T>& a, const LbmStepParams& p, cudaStream_t st) {
    using SH = StagedShape<S, TX, TY>;
    StagedPlan pl;
    pl.flags_bulk = p.g.n[0] % 16 == 0;
    pl.ntile[0] = (p.g.n[0] + TX - 1) / TX;
    pl.ntile[1] = (p.g.n[1] + TY - 1) / TY;
    const int sms = p.num_sms > 0 ? p.num_sms : 152;
    const long long tiles = (long long)pl.ntile[0] * pl.ntile[1];
    // z chunks: about eight work items per resident block where the box
    // allows, at least four planes per item
    int zc = p.staged_zchunk > 0 ? p.staged_zchunk
                                 : (int)((tiles * p.g.n[2]) / (8LL * 2 * sms));
    zc = zc < 4 ? 4 : (zc > p.g.n[2] ? p.g.n[2] : zc);
    pl.zchunk = zc;
    pl.nzc = (p.g.n[2] + zc - 1) / zc;
    pl.n_items = (int)(tiles * pl.nzc);
    const int grid = (int)std::min<long long>(pl.n_items, 2LL * sms);
    stream_collide_staged_kernel<S, typename Store<S>::T, TX, TY><<<grid, SH::THREADS, SH::SMEM, st>>>(a, pl);
}

template <typename S>
static void staged_launch_t(const LbmStepParams& p, cudaStream_t st) {
    using T = typename Store<S>::T;
    SCArgs<S, T> a;
    fill_sc_args<S, T>(p, a);
    switch (staged_tx(p.g.n[0])) {
        case 128: staged_launch<S, 128, 2>(a, p, st); break;
        case 64: staged_launch<S, 64, 4>(a, p, st); break;
        default: staged_launch<S, 32, 8>(a, p, st); break;
    }
}

void launch_stream_collide_staged(const LbmStepParams& p, cudaStream_t st) {
    switch (p.storage) {
        case 1: staged_launch_t<float>(p, st); break;
        case 2: staged_launch_t<__half>(p, st); break;
        default: staged_launch_t<__nv_bfloat16>(p, st); break;
    }
}

}  // namespace lbmdem
