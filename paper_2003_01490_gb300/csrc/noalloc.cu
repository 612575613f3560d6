// noalloc.cu -- sphere-to-cell mapping that allocates no device memory.
//
// For callers that cannot call cudaMalloc (a host program whose device memory
// comes from a fixed pool owned by someone else, code running under a
// strict memory budget, or a plug-in that must not change the process's
// allocation state): the caller passes device buffers for the inputs and the
// outputs, and the temporary tile lists live in a file-scope device array of
// fixed size that every device holds from the time the library is loaded.
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/lbmdem.h"
#include "common.cuh"
#include "launch.h"

namespace lbmdem {

// limits of the static scratch: mapping tiles of 32 x 4 x 4 cells and spheres
constexpr int NOALLOC_MAX_TILES = 98304;      // boxes up to 50,331,648 cells
constexpr int NOALLOC_MAX_SPHERES = 65536;

struct NoallocScratch {
    int tile_count[NOALLOC_MAX_TILES];
    int tile_list[NOALLOC_MAX_TILES * TILE_CAP];
    PartView view[NOALLOC_MAX_SPHERES];
    float xf[3 * NOALLOC_MAX_SPHERES];
    unsigned long long n_solid;
    int counters[4];          // refill and missing-link counts (the lists are disabled)
    int status;
    unsigned int dummy_list[4];
};

// about 29 MB; shared by every call on a device
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// float views (base cell + fraction, radius) of the spheres for the mapping
__global__ void noalloc_view_kernel(int n, const double* __restrict__ pos, const double* __restrict__ radius,
                                    NoallocScratch* s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PartView v;
    for (int d = 0; d < 3; ++d) {
        const double x = pos[3 * i + d];
        const double b = floor(x);
        v.base[d] = (int)b;
        v.frac[d] = (float)(x - b);
        v.u[d] = 0.f;
        v.om[d] = 0.f;
        s->xf[3 * i + d] = (float)x;
    }
    v.R = (float)radius[i];
    v.C = 0.f;   // unused by the mapping
    v.C_lo = 0.f;
    s->view[i] = v;
}

namespace {

std::mutex g_mutex;
NoallocScratch* g_scratch_ptr[64] = {nullptr};
// one lock per device, held for a whole call (which ends with a stream
// synchronise), so calls from several host threads never share the scratch
std::mutex g_call_mutex[64];

lbm_status noalloc_fail(lbm_status s, const std::string& m) {
    set_global_error(m);   // reported by lbm_last_error(NULL)
    return s;
}

}  // namespace
}  // namespace lbmdem

using namespace lbmdem;

extern "C" lbm_status lbm_map_spheres_noalloc(const lbm_grid* grid, double shell_width, int n, const double* d_pos,
                                              const double* d_radius, unsigned char* d_flags, int* d_owner,
                                              void* cuda_stream) {
    if (!grid || n < 0 || (n > 0 && (!d_pos || !d_radius)) || !d_flags || !d_owner)
        return noalloc_fail(LBM_ERR_INVALID, "invalid arguments");
    if (grid->nx < 3 || grid->ny < 3 || grid->nz < 3) return noalloc_fail(LBM_ERR_INVALID, "box too small");
    const long long ncells = (long long)grid->nx * grid->ny * grid->nz;
    const int nt[3] = {(grid->nx + TILE_X - 1) / TILE_X, (grid->ny + TILE_Y - 1) / TILE_Y,
                       (grid->nz + TILE_Z - 1) / TILE_Z};
    const long long ntiles = (long long)nt[0] * nt[1] * nt[2];
    if (ntiles > NOALLOC_MAX_TILES || ncells >= (1LL << 31))
        return noalloc_fail(LBM_ERR_INVALID, "box exceeds the static scratch limit of 98304 tiles of 32x4x4 cells");
    if (n > NOALLOC_MAX_SPHERES) return noalloc_fail(LBM_ERR_INVALID, "more than 65536 spheres");
    if (!(shell_width >= 0.0)) return noalloc_fail(LBM_ERR_INVALID, "shell_width must be >= 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) return noalloc_fail(LBM_ERR_CUDA, "cudaGetDevice failed");
    NoallocScratch* s = nullptr;
    {
        // once per device, with that device current: the device address of the
        // static scratch (the host-side symbol is only a stand-in)
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_ptr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess)
                return noalloc_fail(LBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_ptr[dev] = static_cast<NoallocScratch*>(ptr);
        }
        s = g_scratch_ptr[dev];
    }
    // every buffer must live on the current device, the one whose scratch
    // this call uses
    {
        const void* bufs[4] = {d_flags, d_owner, d_pos, d_radius};
        const char* names[4] = {"d_flags", "d_owner", "d_pos", "d_radius"};
        for (int b = 0; b < (n > 0 ? 4 : 2); ++b) {
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, bufs[b]) != cudaSuccess || at.type != cudaMemoryTypeDevice ||
                at.device != dev) {
                cudaGetLastError();
                return noalloc_fail(LBM_ERR_INVALID,
                                    std::string(names[b]) + " is not device memory of the current device");
            }
        }
    }
    std::lock_guard<std::mutex> call_lock(g_call_mutex[dev]);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // every return after the first queued operation waits for the stream, so
    // the next holder of the lock never overlaps this call's work on the scratch
    struct SyncOnExit {
        cudaStream_t st;
        bool armed = true;
        ~SyncOnExit() {
            if (armed) {
                cudaStreamSynchronize(st);
                cudaGetLastError();
            }
        }
    } sync_on_exit{st};
    // outputs start as a box without particles; shared counters start at zero
    if ((e = cudaMemsetAsync(d_flags, 0, (size_t)ncells, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(d_owner, 0xff, 4 * (size_t)ncells, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(s->tile_count, 0, sizeof(int) * (size_t)ntiles, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(&s->n_solid, 0, sizeof(unsigned long long), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(s->counters, 0, sizeof(s->counters), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(&s->status, 0, sizeof(int), st)) != cudaSuccess)
        return noalloc_fail(LBM_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    Particles P{};
    P.n = n;
    P.x = const_cast<double*>(d_pos);
    P.R = const_cast<double*>(d_radius);
    P.view = s->view;
    P.xf = s->xf;
    if (n > 0) noalloc_view_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, d_pos, d_radius, s);
    MapParams mp{};
    mp.g.n[0] = grid->nx; mp.g.n[1] = grid->ny; mp.g.n[2] = grid->nz;
    for (int a = 0; a < 3; ++a) {
        mp.g.per[a] = grid->periodic[a] ? 1 : 0;
        mp.ntile[a] = nt[a];
        mp.small[a] = mp.g.per[a];   // per-cell minimum image on every periodic axis
    }
    mp.g.ncells = ncells;
    mp.P = P;
    mp.flags = d_flags;
    mp.owner = d_owner;
    mp.tile_count = s->tile_count;
    mp.tile_list = s->tile_list;
    mp.shell_width = shell_width;
    // the refill and missing-link lists of the time stepper are not produced here
    mp.refill_list = s->dummy_list; mp.refill_owner = reinterpret_cast<int*>(s->dummy_list);
    mp.refill_count = &s->counters[0]; mp.refill_cap = 0;
    mp.miss_list = s->dummy_list; mp.miss_count = &s->counters[1]; mp.miss_cap = 0;
    mp.n_solid = &s->n_solid;
    mp.status = &s->status;
    launch_tile_scatter(mp, st);
    launch_map(mp, st);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return noalloc_fail(LBM_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    int status = 0;
    if ((e = cudaMemcpyAsync(&status, &s->status, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return noalloc_fail(LBM_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
    sync_on_exit.armed = false;   // the stream was synchronised just above
    if (status & ST_TILE_OVERFLOW)
        return noalloc_fail(LBM_ERR_CAPACITY, "more than 64 spheres reach one 32x4x4 tile");
    return LBM_OK;
}
