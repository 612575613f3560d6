// api.cu -- C ABI of the library (declared in include/lbmdem.h): context
// management, device memory layout, particle insertion and the per-step
// launch sequence of Algorithm 1 (Sec. 4.2).
#include <algorithm>
#include <chrono>
#include <map>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lbmdem.h"
#include "common.cuh"
#include "launch.h"


using namespace lbmdem;

// phases of lbm_profile(): boundary, stream+collide, force finalisation, DEM,
// mapping, refill
constexpr int LBM_PHASES = 6;

struct lbm_ctx {
    Geom g{};
    lbm_relax relax{};
    lbm_dem dem{};
    double a_user[3] = {0, 0, 0};
    int storage = 1;
    int max_particles = 0;
    cudaStream_t stream = nullptr;
    bool own_memory = false;
    char* base = nullptr;
    size_t bytes = 0;
    size_t elem = 4;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    uint8_t* flags = nullptr;
    int* owner = nullptr;
    int ntile[3] = {1, 1, 1};
    long long ntiles = 1;
    int* tile_count = nullptr;
    int* tile_list = nullptr;
    unsigned int* refill_list = nullptr;
    int* refill_owner = nullptr;
    int* refill_count = nullptr;
    int refill_cap = 0;
    unsigned long long* n_solid = nullptr;
    int* status = nullptr;
    double* accel = nullptr;
    float* accel_f = nullptr;
    unsigned int* miss_list = nullptr;
    int* miss_count = nullptr;
    int miss_cap = 0;
    double* scratch = nullptr;
    long long scratch_cells = 0;
    long long bin_cap = 1;
    Particles P{};
    int hcur = 0;
    bool stepped = false;
    long long launches = 0;
    // captured steady-state steps, one per (PDF buffer, history buffer) parity
    cudaStream_t capture_stream = nullptr;
    // second stream for work beside the dense kernel, with its fork/join events
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // asynchronous particle-state read-out: a device snapshot taken on the
    // context stream, copied to the host on its own stream
    cudaStream_t readout_stream = nullptr;
    cudaEvent_t ev_snap = nullptr, ev_read = nullptr;
    double* snap = nullptr;        // [15 max_particles]: x, u, om, F, T blocks
    bool read_pending = false;
    cudaGraphExec_t step_graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    long long graph_launches[2][2] = {{0, 0}, {0, 0}};   // kernel launches in each graph
    int graph_hcur[2][2] = {{0, 0}, {0, 0}};            // history parity after each graph
    bool graphs_off = false;
    bool dem_restart = false;   // DEM switched on after the first step: initial force pending
    int num_sms = 152;             // multiprocessors of the device (grid sizing)
    double ext_total[3] = {0, 0, 0};
    double r_max = 0.0;
    std::vector<double> hx, hR;    // host copies for insertion checks
    std::string err;
    // phase timing (lbm_profile)
    bool profiling = false;
    std::vector<cudaEvent_t> events;
    size_t ev_used = 0;
    long long prof_steps = 0;
};

// streams, events and graphs a context holds (device memory is separate)
void destroy_handles(lbm_ctx* ctx) {
    for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
    ctx->events.clear();
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            if (ctx->step_graph[a][b]) {
                cudaGraphExecDestroy(ctx->step_graph[a][b]);
                ctx->step_graph[a][b] = nullptr;
            }
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    if (ctx->side_stream) {
        cudaStreamSynchronize(ctx->side_stream);
        cudaStreamDestroy(ctx->side_stream);
    }
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    ctx->capture_stream = ctx->side_stream = nullptr;
    ctx->ev_fork = ctx->ev_join = nullptr;
    if (ctx->readout_stream) {
        cudaStreamSynchronize(ctx->readout_stream);
        cudaStreamDestroy(ctx->readout_stream);
    }
    if (ctx->ev_snap) cudaEventDestroy(ctx->ev_snap);
    if (ctx->ev_read) cudaEventDestroy(ctx->ev_read);
    if (ctx->snap) cudaFree(ctx->snap);
    ctx->readout_stream = nullptr;
    ctx->ev_snap = ctx->ev_read = nullptr;
    ctx->snap = nullptr;
}

namespace {

thread_local std::string g_err;

lbm_status fail(lbm_ctx* c, lbm_status s, const std::string& msg) {
    if (c) c->err = msg;
    g_err = msg;
    return s;
}

lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
    return fail(c, LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
    } while (0)

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

size_t elem_size(lbm_storage s) {
    switch (s) {
        case LBM_STORE_F64: return 8;
        case LBM_STORE_F32: return 4;
        default: return 2;
    }
}

// device memory layout: every piece 256-byte aligned, in a fixed order
struct Layout {
    size_t off[64];
    size_t size[64];
    int n = 0;
    size_t total = 0;
    int add(size_t bytes) {
        off[n] = total;
        size[n] = bytes;
        total += align256(bytes ? bytes : 1);
        return n++;
    }
};

struct Sizes {
    long long ncells;
    int ntile[3];
    long long ntiles;
    int refill_cap;
    long long scratch_cells;
    long long bin_cap;
};

Sizes compute_sizes(const lbm_grid* g, int max_particles) {
    Sizes s;
    s.ncells = (long long)g->nx * g->ny * g->nz;
    s.ntile[0] = (g->nx + TILE_X - 1) / TILE_X;
    s.ntile[1] = (g->ny + TILE_Y - 1) / TILE_Y;
    s.ntile[2] = (g->nz + TILE_Z - 1) / TILE_Z;
    s.ntiles = (long long)s.ntile[0] * s.ntile[1] * s.ntile[2];
    long long rc = 65536 + 1024LL * max_particles;
    if (rc > s.ncells) rc = s.ncells;
    s.refill_cap = (int)rc;
    long long sc = s.ncells < (4LL << 20) ? s.ncells : (4LL << 20);
    s.scratch_cells = sc;
    long long bc = 4LL * max_particles + 64;
    if (bc > s.ncells) bc = s.ncells;
    s.bin_cap = bc;
    return s;
}

void build_layout(const lbm_grid* g, lbm_storage st, int np, Layout& L, const Sizes& s) {
    const size_t es = elem_size(st);
    const size_t N = (size_t)s.ncells;
    const size_t n = (size_t)np;
    L.add(19 * N * es);                 // 0 f[0]
    L.add(19 * N * es);                 // 1 f[1]
    L.add(N + 256);                     // 2 flags (+ padding: the staged dense kernel copies whole 16-byte units)
    L.add(4 * N);                       // 3 owner
    L.add(4 * s.ntiles);                // 4 tile_count
    L.add(4 * s.ntiles * TILE_CAP);     // 5 tile_list
    L.add(4 * (size_t)s.refill_cap);    // 6 refill_list
    L.add(4);                           // 7 (unused)
    L.add(32);                          // 8 counters: n_solid, missing-link and refill counts
    L.add(4);                           // 9 status
    L.add(8 * 3);                       // 10 accel
    L.add(8 * 4 * (size_t)s.scratch_cells);  // 11 scratch
    // particles
    L.add(8 * 3 * n);  // 12 x
    L.add(8 * 3 * n);  // 13 u
    L.add(8 * 3 * n);  // 14 om
    L.add(8 * n);      // 15 R
    L.add(8 * n);      // 16 rho
    L.add(8 * n);      // 17 m
    L.add(8 * n);      // 18 I
    L.add(8 * 3 * n);  // 19 F_prev
    L.add(8 * 3 * n);  // 20 T_prev
    L.add(8 * 3 * n);  // 21 F_new
    L.add(8 * 3 * n);  // 22 T_new
    L.add(8 * 6 * n);  // 23 acc_d
    L.add(8 * 6 * n);  // 24 acc_i
    L.add(8 * 6 * n);  // 25 fp
    L.add(8 * 6 * n);  // 26 fp_old
    L.add(8 * 6 * n);  // 27 fbar
    L.add(sizeof(PartView) * n);                 // 28 view
    L.add(4 * (size_t)s.bin_cap);                // 29 bin_count
    L.add(4 * (size_t)s.bin_cap * BIN_CAP);      // 30 bin_list
    L.add(4 * n);                                // 31 nbr_count
    L.add(4 * n * NBR_CAP);                      // 32 nbr
    for (int h = 0; h < 2; ++h) {
        L.add(4 * n * NBR_CAP);                  // 33/38 hist_id
        L.add(8 * 3 * n * NBR_CAP);              // 34/39 hist_d
        L.add(4 * n);                            // 35/40 hist_n
        L.add(8 * 3 * 6 * n);                    // 36/41 whist
        L.add(6 * n);                            // 37/42 wact
    }
    L.add(4);                                    // 43 (unused)
    L.add(4);                                    // 44 (unused)
    L.add(4 * 3);                                // 45 accel_f
    L.add(4 * 3 * n);                            // 46 xf
    L.add(4 * N);                                // 47 miss_list
    L.add(4);                                    // 48 (unused)
    L.add(8 * 6 * n);                            // 49 acc_k
    L.add(8 * 3 * n);                            // 50 x (second subcycle buffer)
    L.add(8 * 3 * n);                            // 51 u
    L.add(8 * 3 * n);                            // 52 om
    L.add(4 * 3 * n);                            // 53 xf
    L.add(8 * n);                                // 54 hm
    L.add(8 * n);                                // 55 hI
    L.add(8 * 3 * n);                            // 56 ext
    L.add(4 * (size_t)s.refill_cap);             // 57 refill_owner
    for (int h = 0; h < 2; ++h) {
        L.add(4 * 3 * n);                        // 58/60 float32 u
        L.add(4 * 3 * n);                        // 59/61 float32 omega
    }
    (void)g;
}

lbm_status validate(const lbm_grid* g, const lbm_relax* r, const lbm_dem* d, lbm_storage st,
                    int max_particles) {
    if (!g || !r || !d) return fail(nullptr, LBM_ERR_INVALID, "null parameter struct");
    if (g->nx < 3 || g->ny < 3 || g->nz < 3) return fail(nullptr, LBM_ERR_INVALID, "box must be at least 3 cells per axis");
    long long nc = (long long)g->nx * g->ny * g->nz;
    // 32-bit cell indices in the kernels, with room for a grid-stride step
    if (nc > (1LL << 31) - (1LL << 24))
        return fail(nullptr, LBM_ERR_INVALID, "box has more than 2^31 - 2^24 cells");
    if (g->nz > 65535 || g->ny > 65535 * 2) return fail(nullptr, LBM_ERR_INVALID, "ny or nz too large");
    if (!(r->tau > 0.5)) return fail(nullptr, LBM_ERR_INVALID, "tau must be > 1/2");
    if (!(r->magic > 0.0) || !(r->lambda_b_shell > 0.0) || !(r->lambda_b_bulk > 0.0) || !(r->shell_width >= 0.0))
        return fail(nullptr, LBM_ERR_INVALID, "magic, lambda_b must be > 0 and shell_width >= 0");
    if (st < LBM_STORE_F64 || st > LBM_STORE_BF16) return fail(nullptr, LBM_ERR_INVALID, "unknown storage format");
    // the NaN marker of a solid cell carries particle + 1 in 22 bits
    if (max_particles < 0 || max_particles > 4000000)
        return fail(nullptr, LBM_ERR_INVALID, "max_particles must be in [0, 4,000,000]");
    if (d->n_sub < 1) return fail(nullptr, LBM_ERR_INVALID, "n_sub must be >= 1");
    if (!(d->e_dry > 0.0 && d->e_dry <= 1.0)) return fail(nullptr, LBM_ERR_INVALID, "e_dry must be in (0, 1]");
    if (!(d->nu_p >= 0.0 && d->nu_p < 1.0)) return fail(nullptr, LBM_ERR_INVALID, "nu_p must be in [0, 1)");
    if (!(d->mu_p >= 0.0)) return fail(nullptr, LBM_ERR_INVALID, "mu_p must be >= 0");
    if (!(d->lub_cut_n > 0 && d->lub_cut_tt > 0 && d->lub_cut_tr > 0))
        return fail(nullptr, LBM_ERR_INVALID, "lubrication cut-offs must be > 0");
    if (d->fixed_particles < 0 || d->fixed_particles > 2)
        return fail(nullptr, LBM_ERR_INVALID, "fixed_particles must be 0 (DEM), 1 (fixed) or 2 (prescribed motion)");
    return LBM_OK;
}

lbm_status create_impl(const lbm_grid* g, const lbm_relax* r, const double* bf, const lbm_dem* d,
                       lbm_storage st, int max_particles, void* stream, void* arena, size_t arena_bytes,
                       lbm_ctx** out) {
    if (!out) return fail(nullptr, LBM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    lbm_status v = validate(g, r, d, st, max_particles);
    if (v != LBM_OK) return v;
    lbm_ctx* ctx = new lbm_ctx();
    ctx->relax = *r;
    ctx->dem = *d;
    ctx->storage = (int)st;
    ctx->elem = elem_size(st);
    ctx->max_particles = max_particles;
    ctx->stream = static_cast<cudaStream_t>(stream);
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            ctx->num_sms = sms;
        cudaError_t pe = prepare_stream_collide((int)st);
        if (pe == cudaSuccess) pe = cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking);
        if (pe == cudaSuccess) pe = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
        if (pe == cudaSuccess) pe = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
        if (pe != cudaSuccess) {
            destroy_handles(ctx);
            delete ctx;
            return fail(nullptr, LBM_ERR_CUDA, std::string("kernel attributes: ") + cudaGetErrorString(pe));
        }
    }
    ctx->g.n[0] = g->nx; ctx->g.n[1] = g->ny; ctx->g.n[2] = g->nz;
    for (int a = 0; a < 3; ++a) {
        ctx->g.per[a] = g->periodic[a] ? 1 : 0;
        for (int c = 0; c < 3; ++c) {
            ctx->g.wall_vel[0][a][c] = g->wall_vel_lo[a][c];
            ctx->g.wall_vel[1][a][c] = g->wall_vel_hi[a][c];
        }
        ctx->a_user[a] = bf ? bf[a] : 0.0;
    }
    ctx->g.ncells = (long long)g->nx * g->ny * g->nz;
    Sizes s = compute_sizes(g, max_particles);
    Layout L;
    build_layout(g, st, max_particles, L, s);
    ctx->bytes = L.total;
    if (arena) {
        if (reinterpret_cast<uintptr_t>(arena) % 256 != 0) {
            destroy_handles(ctx);
            delete ctx;
            return fail(nullptr, LBM_ERR_INVALID, "arena must be 256-byte aligned");
        }
        if (arena_bytes < L.total) {
            destroy_handles(ctx);
            delete ctx;
            return fail(nullptr, LBM_ERR_OOM, "arena smaller than lbm_required_bytes()");
        }
        ctx->base = static_cast<char*>(arena);
        ctx->own_memory = false;
    } else {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, L.total);
        if (e != cudaSuccess) {
            destroy_handles(ctx);
            delete ctx;
            return fail(nullptr, LBM_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        ctx->base = static_cast<char*>(p);
        ctx->own_memory = true;
    }
    char* b = ctx->base;
    auto at = [&](int k) { return (void*)(b + L.off[k]); };
    ctx->f[0] = at(0);
    ctx->f[1] = at(1);
    ctx->flags = (uint8_t*)at(2);
    ctx->owner = (int*)at(3);
    for (int a = 0; a < 3; ++a) ctx->ntile[a] = s.ntile[a];
    ctx->ntiles = s.ntiles;
    ctx->tile_count = (int*)at(4);
    ctx->tile_list = (int*)at(5);
    ctx->refill_list = (unsigned int*)at(6);
    ctx->refill_owner = (int*)at(57);
    ctx->refill_cap = s.refill_cap;
    // one 32-byte block of counters, cleared by one memset per remap
    ctx->n_solid = (unsigned long long*)at(8);
    ctx->miss_count = (int*)((char*)at(8) + 8);
    ctx->refill_count = (int*)((char*)at(8) + 12);
    ctx->status = (int*)at(9);
    ctx->accel = (double*)at(10);
    ctx->accel_f = (float*)at(45);
    ctx->P.xf = (float*)at(46);
    ctx->miss_list = (unsigned int*)at(47);
    ctx->miss_cap = (int)s.ncells;
    ctx->P.acc_k = (long long*)at(49);
    ctx->P.xs[1] = (double*)at(50);
    ctx->P.us[1] = (double*)at(51);
    ctx->P.oms[1] = (double*)at(52);
    ctx->P.xfs[1] = (float*)at(53);
    ctx->P.hm = (double*)at(54);
    ctx->P.hI = (double*)at(55);
    ctx->P.ext = (double*)at(56);
    for (int h = 0; h < 2; ++h) {
        ctx->P.ufs[h] = (float*)at(58 + 2 * h);
        ctx->P.omfs[h] = (float*)at(59 + 2 * h);
    }
    ctx->scratch = (double*)at(11);
    ctx->scratch_cells = s.scratch_cells;
    ctx->bin_cap = s.bin_cap;
    Particles& P = ctx->P;
    P.n = 0;
    P.x = (double*)at(12); P.u = (double*)at(13); P.om = (double*)at(14); P.R = (double*)at(15);
    P.xs[0] = P.x; P.us[0] = P.u; P.oms[0] = P.om; P.xfs[0] = P.xf;
    P.rho = (double*)at(16); P.m = (double*)at(17); P.I = (double*)at(18);
    P.F_prev = (double*)at(19); P.T_prev = (double*)at(20); P.F_new = (double*)at(21); P.T_new = (double*)at(22);
    P.acc_d = (double*)at(23); P.acc_i = (long long*)at(24);
    P.fp = (double*)at(25); P.fp_old = (double*)at(26); P.fbar = (double*)at(27);
    P.view = (PartView*)at(28);
    P.bin_count = (int*)at(29); P.bin_list = (int*)at(30);
    P.nbr_count = (int*)at(31); P.nbr = (int*)at(32);
    for (int h = 0; h < 2; ++h) {
        P.hist_id[h] = (int*)at(33 + 5 * h);
        P.hist_d[h] = (double*)at(34 + 5 * h);
        P.hist_n[h] = (int*)at(35 + 5 * h);
        P.whist[h] = (double*)at(36 + 5 * h);
        P.wact[h] = (unsigned char*)at(37 + 5 * h);
    }
    // initial state: fluid at rest with rho = 1 (shifted PDFs are zero), no particles
    cudaStream_t sm = ctx->stream;
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMemsetAsync(ctx->f[0], 0, L.size[0], sm);
    e = e ? e : cudaMemsetAsync(ctx->f[1], 0, L.size[1], sm);
    e = e ? e : cudaMemsetAsync(ctx->flags, 0, L.size[2], sm);
    e = e ? e : cudaMemsetAsync(ctx->owner, 0xff, L.size[3], sm);
    for (int k = 4; k < L.n && e == cudaSuccess; ++k)
        if (k != 11) e = cudaMemsetAsync(b + L.off[k], 0, L.size[k] ? L.size[k] : 1, sm);
    double acc0[3] = {ctx->a_user[0], ctx->a_user[1], ctx->a_user[2]};
    float acc0f[3] = {(float)acc0[0], (float)acc0[1], (float)acc0[2]};
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->accel, acc0, sizeof(acc0), cudaMemcpyHostToDevice, sm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->accel_f, acc0f, sizeof(acc0f), cudaMemcpyHostToDevice, sm);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sm);
    if (e != cudaSuccess) {
        if (ctx->own_memory) cudaFree(ctx->base);
        destroy_handles(ctx);
        delete ctx;
        return fail(nullptr, LBM_ERR_CUDA, std::string("initialisation: ") + cudaGetErrorString(e));
    }
    // the wall-adjacent cells need the NEAR flag even without particles
    MapParams mp{};
    mp.g = ctx->g; mp.P = ctx->P; mp.flags = ctx->flags; mp.owner = ctx->owner;
    mp.pdf[0] = ctx->f[0]; mp.pdf[1] = ctx->f[1]; mp.elem = (int)ctx->elem;
    for (int a = 0; a < 3; ++a) mp.ntile[a] = ctx->ntile[a];
    mp.tile_count = ctx->tile_count; mp.tile_list = ctx->tile_list;
    mp.shell_width = ctx->relax.shell_width;
    mp.refill_list = ctx->refill_list; mp.refill_owner = ctx->refill_owner;
    mp.refill_count = ctx->refill_count; mp.refill_cap = ctx->refill_cap;
    mp.n_solid = ctx->n_solid; mp.status = ctx->status;
    mp.miss_list = ctx->miss_list; mp.miss_count = ctx->miss_count; mp.miss_cap = ctx->miss_cap;
    launch_map(mp, sm);
    ctx->launches += 1;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(sm);
    if (e != cudaSuccess) {
        if (ctx->own_memory) cudaFree(ctx->base);
        destroy_handles(ctx);
        delete ctx;
        return fail(nullptr, LBM_ERR_CUDA, std::string("initial mapping: ") + cudaGetErrorString(e));
    }
    *out = ctx;
    return LBM_OK;
}

double s_minus_of(double s_nu, double magic) { return 1.0 / (0.5 + magic / (1.0 / s_nu - 0.5)); }
double s_b_of(double s_nu, double lb) { return 1.0 / (0.5 + lb * (1.0 / s_nu - 0.5)); }

MapParams map_params(lbm_ctx* ctx) {
    MapParams mp{};
    const int ts[3] = {TILE_X, TILE_Y, TILE_Z};
    const double reach = ctx->r_max + std::fmax(ctx->relax.shell_width, 1.4142135623730951) + 0.02;
    for (int a = 0; a < 3; ++a)
        mp.small[a] = ctx->g.per[a] && ctx->g.n[a] <= 2.0 * reach + ts[a] + 2.0;
    mp.g = ctx->g; mp.P = ctx->P; mp.flags = ctx->flags; mp.owner = ctx->owner;
    mp.pdf[0] = ctx->f[0]; mp.pdf[1] = ctx->f[1]; mp.elem = (int)ctx->elem;
    for (int a = 0; a < 3; ++a) mp.ntile[a] = ctx->ntile[a];
    mp.tile_count = ctx->tile_count; mp.tile_list = ctx->tile_list;
    mp.shell_width = ctx->relax.shell_width;
    mp.refill_list = ctx->refill_list; mp.refill_owner = ctx->refill_owner;
    mp.refill_count = ctx->refill_count; mp.refill_cap = ctx->refill_cap;
    mp.n_solid = ctx->n_solid; mp.status = ctx->status;
    mp.miss_list = ctx->miss_list; mp.miss_count = ctx->miss_count; mp.miss_cap = ctx->miss_cap;
    return mp;
}

// remap all particles: clear tile lists and counters, scatter, map
lbm_status remap(lbm_ctx* ctx, cudaStream_t sm) {
    // tile counts are zero here: the mapping kernel resets each one it reads
    CK(cudaMemsetAsync(ctx->n_solid, 0, 16, sm));
    MapParams mp = map_params(ctx);
    launch_tile_scatter(mp, sm);
    launch_map(mp, sm);
    ctx->launches += (ctx->P.n > 0 ? 1 : 0) + 1;
    return LBM_OK;
}

template <typename T>
void fill_consts(const DemParams& dp, DemConsts<T>& k) {
    k.mu_f = (T)dp.mu_f; k.cut_n = (T)dp.cut_n; k.cut_tt = (T)dp.cut_tt; k.cut_tr = (T)dp.cut_tr;
    k.cut_max = (T)dp.cut_max; k.inv_cut_n = (T)dp.inv_cut_n; k.inv_cut_tt = (T)dp.inv_cut_tt;
    k.inv_cut_tr = (T)dp.inv_cut_tr; k.min_a = (T)dp.min_a; k.min_b = (T)dp.min_b; k.log_e = (T)dp.log_e;
    k.pi2_log_e2 = (T)dp.pi2_log_e2; k.kappa = (T)dp.kappa; k.sqrt_kappa = (T)dp.sqrt_kappa;
    k.mu_p = (T)dp.mu_p; k.Tc = (T)dp.Tc; k.dt = (T)dp.dt;
}

DemParams dem_params(lbm_ctx* ctx) {
    DemParams dp{};
    dp.g = ctx->g;
    dp.P = ctx->P;
    const lbm_dem& d = ctx->dem;
    dp.cut_max = std::fmax(d.lub_cut_n, std::fmax(d.lub_cut_tt, d.lub_cut_tr));
    // bins no smaller than the largest interaction reach, at most bin_cap of them
    const double bin_min = 2.0 * ctx->r_max + dp.cut_max + NBR_SKIN;
    long long total = 1;
    for (int a = 0; a < 3; ++a) {
        int nb = (int)std::floor(ctx->g.n[a] / bin_min);
        dp.nbins[a] = nb < 1 ? 1 : nb;
        total *= dp.nbins[a];
    }
    while (total > ctx->bin_cap) {
        int amax = 0;
        for (int a = 1; a < 3; ++a)
            if (dp.nbins[a] > dp.nbins[amax]) amax = a;
        total /= dp.nbins[amax];
        dp.nbins[amax] = dp.nbins[amax] / 2 > 0 ? dp.nbins[amax] / 2 : 1;
        total *= dp.nbins[amax];
    }
    for (int a = 0; a < 3; ++a) dp.binsize[a] = (double)ctx->g.n[a] / dp.nbins[a];
    dp.e_dry = d.e_dry; dp.Tc = d.Tc; dp.nu_p = d.nu_p; dp.mu_p = d.mu_p;
    dp.cut_n = d.lub_cut_n; dp.cut_tt = d.lub_cut_tt; dp.cut_tr = d.lub_cut_tr;
    dp.min_a = d.lub_min_a; dp.min_b = d.lub_min_b;
    dp.inv_cut_n = 1.0 / d.lub_cut_n;
    dp.inv_cut_tt = 1.0 / d.lub_cut_tt;
    dp.inv_cut_tr = 1.0 / d.lub_cut_tr;
    dp.log_e = std::log(d.e_dry);
    dp.pi2_log_e2 = 3.14159265358979323846 * 3.14159265358979323846 + dp.log_e * dp.log_e;
    dp.kappa = 2.0 * (1.0 - d.nu_p) / (2.0 - d.nu_p);
    dp.sqrt_kappa = std::sqrt(dp.kappa);
    for (int a = 0; a < 3; ++a) dp.gravity[a] = d.gravity[a];
    dp.mu_f = (ctx->relax.tau - 0.5) / 3.0;
    dp.lubrication = d.lubrication;
    dp.tangential = d.tangential_lubrication;
    dp.dt = 1.0 / d.n_sub;
    dp.status = ctx->status;
    dp.pair_f32 = ctx->storage != LBM_STORE_F64;
    fill_consts(dp, dp.kd);
    fill_consts(dp, dp.kf);
    return dp;
}

// record the next profiling event on the context stream (no-op when off)
cudaError_t prof_mark(lbm_ctx* ctx) {
    if (!ctx->profiling) return cudaSuccess;
    // an NVTX range per phase on the host side (profilers show it beside the
    // launches); the device times come from the CUDA events
    static const char* const PHASE_NAMES[LBM_PHASES] = {"boundary", "stream_collide", "force_finalize",
                                                        "dem", "mapping", "refill"};
    const size_t k = ctx->ev_used % (LBM_PHASES + 1);
    if (k > 0) nvtxRangePop();
    if (k < LBM_PHASES) nvtxRangePushA(PHASE_NAMES[k]);
    if (ctx->ev_used == ctx->events.size()) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        ctx->events.push_back(e);
    }
    return cudaEventRecord(ctx->events[ctx->ev_used++], ctx->stream);
}

lbm_status check_status(lbm_ctx* ctx) {
    int st = 0;
    CK(cudaMemcpyAsync(&st, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (st & ST_UNSTABLE) return fail(ctx, LBM_ERR_UNSTABLE, "density left (0.5, 1.5) or became NaN");
    if (st & (ST_TILE_OVERFLOW | ST_NBR_OVERFLOW | ST_BIN_OVERFLOW | ST_REFILL_OVERFLOW | ST_HIST_OVERFLOW |
              ST_FIXED_OVERFLOW)) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "device list capacity exceeded (status bits 0x%x)", st);
        return fail(ctx, LBM_ERR_CAPACITY, buf);
    }
    if (st & ST_FAST_PARTICLE) return fail(ctx, LBM_ERR_UNSTABLE, "particle speed above 0.5 cells per step");
    if (st & ST_TIMEOUT)
        return fail(ctx, LBM_ERR_TIMEOUT, "a wait of the staged dense kernel on its copy pipeline ran out");
    return LBM_OK;
}

}  // namespace

void lbmdem::set_global_error(const std::string& msg) { g_err = msg; }

// ====================================================================== ABI

extern "C" {

lbm_status lbm_default_params(lbm_relax* relax, lbm_dem* dem) {
    if (relax) {
        relax->tau = 0.6;
        relax->magic = 3.0 / 16.0;
        relax->lambda_b_shell = 100.0;
        relax->lambda_b_bulk = 1.0;
        relax->shell_width = 2.0;
    }
    if (dem) {
        dem->e_dry = 0.97;
        dem->Tc = 0.0;
        dem->nu_p = 0.23;
        dem->mu_p = 0.15;
        dem->n_sub = 10;
        dem->lub_cut_n = 2.0 / 3.0;
        dem->lub_cut_tt = 0.5;
        dem->lub_cut_tr = 0.5;
        dem->lub_min_a = 0.001;
        dem->lub_min_b = 0.00007;
        dem->gravity[0] = dem->gravity[1] = dem->gravity[2] = 0.0;
        dem->lubrication = 1;
        dem->tangential_lubrication = 1;
        dem->force_averaging = 1;
        dem->fluid_counterforce = 0;
        dem->fixed_particles = 0;
        dem->missing_links = 1;
    }
    return LBM_OK;
}

lbm_status lbm_required_bytes(const lbm_grid* grid, lbm_storage storage, int max_particles, size_t* bytes_out) {
    if (!grid || !bytes_out || max_particles < 0 || grid->nx < 3 || grid->ny < 3 || grid->nz < 3)
        return fail(nullptr, LBM_ERR_INVALID, "invalid arguments");
    if (storage < LBM_STORE_F64 || storage > LBM_STORE_BF16)
        return fail(nullptr, LBM_ERR_INVALID, "unknown storage format");
    Sizes s = compute_sizes(grid, max_particles);
    Layout L;
    build_layout(grid, storage, max_particles, L, s);
    *bytes_out = L.total;
    return LBM_OK;
}

lbm_status lbm_create(const lbm_grid* grid, const lbm_relax* relax, const double* body_force, const lbm_dem* dem,
                      lbm_storage storage, int max_particles, void* cuda_stream, lbm_ctx** out) {
    return create_impl(grid, relax, body_force, dem, storage, max_particles, cuda_stream, nullptr, 0, out);
}

lbm_status lbm_create_in_arena(const lbm_grid* grid, const lbm_relax* relax, const double* body_force,
                               const lbm_dem* dem, lbm_storage storage, int max_particles, void* cuda_stream,
                               void* arena, size_t arena_bytes, lbm_ctx** out) {
    if (!arena) return fail(nullptr, LBM_ERR_INVALID, "arena is NULL");
    return create_impl(grid, relax, body_force, dem, storage, max_particles, cuda_stream, arena, arena_bytes, out);
}

lbm_status lbm_add_spheres(lbm_ctx* ctx, int n, const double* pos, const double* vel, const double* omega,
                           const double* radius, const double* density, int* first_id_out) {
    if (!ctx) return fail(nullptr, LBM_ERR_INVALID, "ctx is NULL");
    if (ctx->stepped) return fail(ctx, LBM_ERR_STATE, "spheres can only be added before the first step");
    if (n < 0 || (n > 0 && (!pos || !radius || !density))) return fail(ctx, LBM_ERR_INVALID, "invalid arrays");
    if (ctx->P.n + n > ctx->max_particles) return fail(ctx, LBM_ERR_CAPACITY, "max_particles exceeded");
    const int n0 = ctx->P.n;
    std::vector<double> hx(ctx->hx), hR(ctx->hR);
    double rmax = ctx->r_max;
    for (int k = 0; k < n; ++k) {
        const double R = radius[k], rho = density[k];
        if (!(R >= 1.0 && R <= 100.0)) return fail(ctx, LBM_ERR_INVALID, "radius must be in [1, 100] cells");
        if (!(rho > 0.0)) return fail(ctx, LBM_ERR_INVALID, "density ratio must be > 0");
        for (int a = 0; a < 3; ++a) {
            const double x = pos[3 * k + a];
            const double L = ctx->g.n[a];
            if (!(x >= 0.0 && x < L)) return fail(ctx, LBM_ERR_INVALID, "sphere centre outside the box");
            if (!ctx->g.per[a] && (x - R < 0.0 || x + R > L))
                return fail(ctx, LBM_ERR_INVALID, "sphere crosses a wall");
            if (ctx->g.per[a] && 2.0 * R + 4.0 >= L)
                return fail(ctx, LBM_ERR_INVALID, "periodic side not longer than 2 R + 4 cells");
        }
        if (R > rmax) rmax = R;
    }
    // overlap test on a uniform grid of buckets no smaller than 2 R_max: an
    // overlapping pair (distance < R_i + R_j) lies in neighbouring buckets
    {
        int dims[3];
        long long total = 1;
        for (int a = 0; a < 3; ++a) {
            dims[a] = (int)std::floor(ctx->g.n[a] / (2.0 * rmax));
            if (dims[a] < 1) dims[a] = 1;
            total *= dims[a];
        }
        while (total > (1LL << 22)) {
            int amax = 0;
            for (int a = 1; a < 3; ++a)
                if (dims[a] > dims[amax]) amax = a;
            total /= dims[amax];
            dims[amax] = (dims[amax] + 1) / 2;
            total *= dims[amax];
        }
        auto bucket_of = [&](const double* x, int (&b)[3]) {
            for (int a = 0; a < 3; ++a) {
                int v = (int)(x[a] / ctx->g.n[a] * dims[a]);
                b[a] = v < 0 ? 0 : (v >= dims[a] ? dims[a] - 1 : v);
            }
        };
        std::vector<std::vector<int>> buckets((size_t)total);
        auto slot = [&](const int (&b)[3]) { return ((size_t)b[2] * dims[1] + b[1]) * dims[0] + b[0]; };
        const int m0 = (int)hR.size();
        for (int j = 0; j < m0; ++j) {
            int b[3];
            bucket_of(&hx[3 * j], b);
            buckets[slot(b)].push_back(j);
        }
        for (int k = 0; k < n; ++k) {
            const double R = radius[k];
            const double* xk = pos + 3 * k;
            int b[3];
            bucket_of(xk, b);
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int nb[3] = {b[0] + dx, b[1] + dy, b[2] + dz};
                        bool skip = false;
                        for (int a = 0; a < 3; ++a) {
                            if (nb[a] < 0 || nb[a] >= dims[a]) {
                                if (!ctx->g.per[a]) skip = true;
                                nb[a] = (nb[a] + dims[a]) % dims[a];
                            }
                        }
                        if (skip) continue;
                        for (int j : buckets[slot(nb)]) {
                            double d2 = 0;
                            for (int a = 0; a < 3; ++a) {
                                double d = xk[a] - hx[3 * j + a];
                                if (ctx->g.per[a]) {
                                    const double L = ctx->g.n[a];
                                    if (d > 0.5 * L) d -= L;
                                    if (d < -0.5 * L) d += L;
                                }
                                d2 += d * d;
                            }
                            const double rr = R + hR[j];
                            if (d2 < rr * rr) return fail(ctx, LBM_ERR_INVALID, "spheres overlap");
                        }
                    }
            const int j = (int)hR.size();
            for (int a = 0; a < 3; ++a) hx.push_back(xk[a]);
            hR.push_back(R);
            buckets[slot(b)].push_back(j);
        }
    }
    if (n == 0) {
        if (first_id_out) *first_id_out = n0;
        return LBM_OK;
    }
    const double pi = 3.14159265358979323846;
    std::vector<double> x(3 * n), u(3 * n, 0.0), om(3 * n, 0.0), R(n), rho(n), m(n), I(n), hm(n), hI(n),
        ext(3 * n);
    for (int k = 0; k < n; ++k) {
        for (int a = 0; a < 3; ++a) {
            x[3 * k + a] = pos[3 * k + a];
            if (vel) u[3 * k + a] = vel[3 * k + a];
            if (omega) om[3 * k + a] = omega[3 * k + a];
        }
        R[k] = radius[k];
        rho[k] = density[k];
        const double D = 2.0 * R[k];
        const double V = pi * D * D * D / 6.0;
        m[k] = rho[k] * V;
        I[k] = 0.4 * m[k] * R[k] * R[k];
        hm[k] = 0.5 / m[k];
        hI[k] = 0.5 / I[k];
        for (int a = 0; a < 3; ++a) {
            ext[3 * k + a] = V * (rho[k] - 1.0) * ctx->dem.gravity[a];
            ctx->ext_total[a] += ext[3 * k + a];
        }
        if (R[k] > ctx->r_max) ctx->r_max = R[k];
    }
    cudaStream_t sm = ctx->stream;
    Particles& P = ctx->P;
    CK(cudaMemcpyAsync(P.x + 3 * n0, x.data(), 8 * 3 * n, cudaMemcpyHostToDevice, sm));
    CK(cudaMemcpyAsync(P.u + 3 * n0, u.data(), 8 * 3 * n, cudaMemcpyHostToDevice, sm));
    CK(cudaMemcpyAsync(P.om + 3 * n0, om.data(), 8 * 3 * n, cudaMemcpyHostToDevice, sm));
    CK(cudaMemcpyAsync(P.R + n0, R.data(), 8 * n, cudaMemcpyHostToDevice, sm));
    CK(cudaMemcpyAsync(P.rho + n0, rho.data(), 8 * n, cudaMemcpyHostToDevice, sm));
    CK(cudaMemcpyAsync(P.m + n0, m.data(), 8 * n, cudaMemcpyHostToDevice, sm));
    CK(cudaMemcpyAsync(P.I + n0, I.data(), 8 * n, cudaMemcpyHostToDevice, sm));
    CK(cudaMemcpyAsync(P.hm + n0, hm.data(), 8 * n, cudaMemcpyHostToDevice, sm));
    CK(cudaMemcpyAsync(P.hI + n0, hI.data(), 8 * n, cudaMemcpyHostToDevice, sm));
    CK(cudaMemcpyAsync(P.ext + 3 * n0, ext.data(), 8 * 3 * n, cudaMemcpyHostToDevice, sm));
    P.n = n0 + n;
    ctx->hx.swap(hx);
    ctx->hR.swap(hR);
    launch_view_update(P, sm);
    ctx->launches += 1;
    lbm_status s = remap(ctx, ctx->stream);
    if (s != LBM_OK) return s;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(sm));
    if (first_id_out) *first_id_out = n0;
    return check_status(ctx);
}

// One time step of Algorithm 1 queued on stream sm, in two parts around the
// dense kernel: enqueue_pre queues everything before it (the fluid body force;
// on the side stream the missing links and the DEM neighbour lists) and fills
// the dense kernel's parameters; enqueue_post queues everything after it (the
// force finalisation, the DEM, the mapping and the refill) and updates the
// host-side state (buffer parities, launch count). A batch does not use
// them: it captures the same kernels as gang launches over its instances
// (batch_capture_gang).
struct StepState {
    LbmStepParams lp{};
    bool side = false;
    bool first = false;
    bool move = false;
    bool dem = false;
};

// parameters of the step's boundary and dense kernels from the context state
void fill_step_params(const lbm_ctx* ctx, LbmStepParams& lp) {
    const lbm_relax& r = ctx->relax;
    const lbm_dem& d = ctx->dem;
    const double s_nu = 1.0 / r.tau;
    lp = LbmStepParams{};
    lp.storage = ctx->storage;
    lp.src = ctx->f[ctx->cur];
    lp.dst = ctx->f[1 - ctx->cur];
    lp.flags = ctx->flags;
    lp.owner = ctx->owner;
    lp.g = ctx->g;
    lp.s_plus = s_nu;
    lp.s_minus = s_minus_of(s_nu, r.magic);
    lp.s_b_shell = s_b_of(s_nu, r.lambda_b_shell);
    lp.s_b_bulk = s_b_of(s_nu, r.lambda_b_bulk);
    lp.bulk_corr = r.lambda_b_bulk != 1.0;
    for (int a = 0; a < 3; ++a) {
        lp.a_user[a] = ctx->a_user[a];
        lp.ext_total[a] = ctx->ext_total[a];
    }
    lp.n_solid = ctx->n_solid;
    lp.counterforce = d.fluid_counterforce && ctx->P.n > 0;
    lp.P = ctx->P;
    lp.missing_links = d.missing_links && ctx->P.n > 0;
    lp.status = ctx->status;
    lp.miss_list = ctx->miss_list;
    lp.miss_count = ctx->miss_count;
    lp.miss_cap = ctx->miss_cap;
    lp.num_sms = ctx->num_sms;
    lp.accel_d = ctx->accel;
    lp.accel_f = ctx->accel_f;
}

lbm_status enqueue_pre(lbm_ctx* ctx, DemParams& dp, cudaStream_t sm, StepState& ss) {
    const lbm_relax& r = ctx->relax;
    const lbm_dem& d = ctx->dem;
    const double s_nu = 1.0 / r.tau;
    // particles move by the DEM (fixed_particles 0) or by their prescribed
    // velocities (2); both remap and refill
    const bool move = ctx->P.n > 0 && d.fixed_particles != 1;
    const bool dem = move && d.fixed_particles == 0;
    const bool first = !ctx->stepped;
    const bool init_dem = dem && (first || ctx->dem_restart);
    ctx->dem_restart = false;
    if (first) ctx->stepped = true;
    ss.first = first;
    ss.move = move;
    ss.dem = dem;
    if (init_dem) {
        // the force of the first Velocity-Verlet position update at the current
        // state (F(t = 0) on the first step, where the averaged fluid force is
        // still zero) needs the neighbour lists of the current positions
        dp.hin = ctx->hcur;
        dp.hout = 1 - ctx->hcur;
        dp.P = ctx->P;
        CK(cudaMemsetAsync(ctx->P.bin_count, 0, sizeof(int) * dp.nbins[0] * dp.nbins[1] * dp.nbins[2], sm));
        launch_bins(dp, sm);
        launch_neighbours(dp, sm);
        launch_dem_subcycle(dp, 0, 1, 0, sm);
        ctx->launches += 3;
    }
    // Algorithm 1, lines 1-3: boundary conditions, interaction force, LBM step
    CK(prof_mark(ctx));
    LbmStepParams& lp = ss.lp;
    fill_step_params(ctx, lp);
    launch_boundary(lp, sm, BC_ACCEL);
    // beside the dense kernel, on the side stream: the missing links (their
    // sums commute with the dense kernel's) and the DEM's neighbour lists,
    // which read only the positions the dense kernel reads too; finalize
    // waits for both streams
    const bool side = lp.missing_links || dem;
    ss.side = side;
    if (side) {
        CK(cudaEventRecord(ctx->ev_fork, sm));
        CK(cudaStreamWaitEvent(ctx->side_stream, ctx->ev_fork, 0));
        if (lp.missing_links) {
            launch_boundary(lp, ctx->side_stream, BC_LINKS);
            ctx->launches += 1;
        }
        if (dem) {
            dp.P = ctx->P;
            CK(cudaMemsetAsync(ctx->P.bin_count, 0, sizeof(int) * dp.nbins[0] * dp.nbins[1] * dp.nbins[2],
                               ctx->side_stream));
            launch_bins(dp, ctx->side_stream);
            launch_neighbours(dp, ctx->side_stream);
            ctx->launches += 2;
        }
        CK(cudaEventRecord(ctx->ev_join, ctx->side_stream));
    }
    CK(prof_mark(ctx));
    return LBM_OK;
}

lbm_status enqueue_post_a(lbm_ctx* ctx, DemParams& dp, cudaStream_t sm, StepState& ss);
lbm_status enqueue_post_b(lbm_ctx* ctx, DemParams& dp, cudaStream_t sm, const StepState& ss);

lbm_status enqueue_post(lbm_ctx* ctx, DemParams& dp, cudaStream_t sm, StepState& ss) {
    lbm_status st = enqueue_post_a(ctx, dp, sm, ss);
    return st != LBM_OK ? st : enqueue_post_b(ctx, dp, sm, ss);
}

// after the dense kernel: force finalisation and the DEM (Algorithm 1,
// lines 4-10)
lbm_status enqueue_post_a(lbm_ctx* ctx, DemParams& dp, cudaStream_t sm, StepState& ss) {
    const lbm_relax& r = ctx->relax;
    const lbm_dem& d = ctx->dem;
    const double s_nu = 1.0 / r.tau;
    const bool first = ss.first, move = ss.move, dem = ss.dem, side = ss.side;
    CK(prof_mark(ctx));
    if (side) CK(cudaStreamWaitEvent(sm, ctx->ev_join, 0));
    FinalizeParams fpp{};
    fpp.P = ctx->P;
    fpp.use_fixed = ctx->storage != LBM_STORE_F64;
    fpp.first_step = first;
    fpp.averaging = d.force_averaging;
    launch_finalize(fpp, sm);
    ctx->launches += 2 + (ctx->P.n > 0 ? 1 : 0);
    CK(prof_mark(ctx));
    if (move) {
        if (dem && ctx->P.n <= DEM_ONE_BLOCK_MAX) {
            // Algorithm 1, lines 4-10, in one block: few particles
            launch_dem_step_one_block(dp, ctx->hcur, d.n_sub, sm);
            ctx->launches += 1;
            if (d.n_sub & 1) ctx->hcur = 1 - ctx->hcur;
        } else if (dem) {
            // Algorithm 1, lines 4-10: DEM subcycles
            launch_dem_position(dp, sm);
            ctx->launches += 1;
            int cur = 0;
            for (int s = 0; s < d.n_sub; ++s) {
                dp.hin = ctx->hcur;
                dp.hout = 1 - ctx->hcur;
                launch_dem_subcycle(dp, cur, 0, s == d.n_sub - 1, sm);
                ctx->hcur = 1 - ctx->hcur;
                cur = 1 - cur;
                ctx->launches += 1;
            }
            if (cur == 1) {
                launch_state_copy(ctx->P, sm);
                ctx->launches += 1;
            }
        } else {
            // prescribed motion: x += u over the step
            launch_prescribed_move(ctx->P, ctx->g, sm);
            ctx->launches += 1;
        }
    }
    return LBM_OK;
}

// the mapping update and refill (Algorithm 1, line 11) and the host-side
// step state
lbm_status enqueue_post_b(lbm_ctx* ctx, DemParams& dp, cudaStream_t sm, const StepState& ss) {
    (void)dp;
    const double s_nu = 1.0 / ctx->relax.tau;
    if (ss.move) {
        CK(prof_mark(ctx));
        // Algorithm 1, line 11: mapping update and refill
        lbm_status st = remap(ctx, sm);
        if (st != LBM_OK) return st;
        CK(prof_mark(ctx));
        RefillParams rp{};
        rp.storage = ctx->storage;
        rp.f = ctx->f[1 - ctx->cur];
        rp.flags = ctx->flags;
        rp.list_owner = ctx->refill_owner;
        rp.g = ctx->g;
        rp.P = ctx->P;
        rp.list = ctx->refill_list;
        rp.count = ctx->refill_count;
        rp.cap = ctx->refill_cap;
        rp.s_nu = s_nu;
        rp.accel = ctx->accel;
        launch_refill(rp, sm);
        ctx->launches += 1;
        CK(prof_mark(ctx));
    } else {
        CK(prof_mark(ctx));
        CK(prof_mark(ctx));
        CK(prof_mark(ctx));
    }
    if (ctx->profiling) ctx->prof_steps += 1;
    ctx->cur = 1 - ctx->cur;
    return LBM_OK;
}

lbm_status enqueue_step(lbm_ctx* ctx, DemParams& dp, cudaStream_t sm) {
    StepState ss;
    lbm_status st = enqueue_pre(ctx, dp, sm, ss);
    if (st != LBM_OK) return st;
    launch_stream_collide(ss.lp, sm);
    return enqueue_post(ctx, dp, sm, ss);
}

// Steady-state steps (after the first, profiling off) run as CUDA graphs: the
// step's ~20 launches are captured once per (PDF buffer, history buffer)
// parity on a private stream and replayed on the context stream, which
// removes the launch overhead that dominates small boxes.
lbm_status graph_step(lbm_ctx* ctx, DemParams& dp, bool& done) {
    done = false;
    if (ctx->graphs_off) return LBM_OK;
    const int pc = ctx->cur, ph = ctx->hcur;
    cudaGraphExec_t& ex = ctx->step_graph[pc][ph];
    if (!ex) {
        if (!ctx->capture_stream &&
            cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            ctx->graphs_off = true;
            return LBM_OK;
        }
        const long long l0 = ctx->launches;
        const int cur0 = ctx->cur, h0 = ctx->hcur;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal);
        lbm_status st = LBM_OK;
        if (e == cudaSuccess) {
            st = enqueue_step(ctx, dp, ctx->capture_stream);
            e = cudaStreamEndCapture(ctx->capture_stream, &g);
        }
        // the capture ran nothing: keep its host-side updates for the replays
        // and undo them here
        ctx->graph_launches[pc][ph] = ctx->launches - l0;
        ctx->graph_hcur[pc][ph] = ctx->hcur;
        ctx->launches = l0;
        ctx->cur = cur0;
        ctx->hcur = h0;
        if (e == cudaSuccess && st == LBM_OK) e = cudaGraphInstantiate(&ex, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess || st != LBM_OK) {
            cudaGetLastError();
            ex = nullptr;
            ctx->graphs_off = true;   // fall back to plain launches for good
            return LBM_OK;
        }
    }
    CK(cudaGraphLaunch(ex, ctx->stream));
    ctx->launches += ctx->graph_launches[pc][ph];
    ctx->hcur = ctx->graph_hcur[pc][ph];
    ctx->cur = 1 - ctx->cur;
    done = true;
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* ctx, int n_steps) {
    if (!ctx) return fail(nullptr, LBM_ERR_INVALID, "ctx is NULL");
    if (n_steps < 0) return fail(ctx, LBM_ERR_INVALID, "n_steps must be >= 0");
    DemParams dp = dem_params(ctx);
    for (int step = 0; step < n_steps; ++step) {
        if (ctx->stepped && !ctx->profiling && !ctx->dem_restart) {
            bool done = false;
            lbm_status st = graph_step(ctx, dp, done);
            if (st != LBM_OK) return st;
            if (done) continue;
        }
        lbm_status st = enqueue_step(ctx, dp, ctx->stream);
        if (st != LBM_OK) return st;
    }
    CK(cudaGetLastError());
    return LBM_OK;
}

lbm_status lbm_set_stream(lbm_ctx* ctx, void* cuda_stream) {
    if (!ctx) return fail(nullptr, LBM_ERR_INVALID, "ctx is NULL");
    if (ctx->profiling) return fail(ctx, LBM_ERR_STATE, "lbm_set_stream: phase timing is on");
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    return check_status(ctx);
}

lbm_status lbm_sync(lbm_ctx* ctx) {
    if (!ctx) return fail(nullptr, LBM_ERR_INVALID, "ctx is NULL");
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->readout_stream) CK(cudaStreamSynchronize(ctx->readout_stream));
    return check_status(ctx);
}

lbm_status lbm_get_particle_state(lbm_ctx* ctx, int n_cap, double* pos, double* vel, double* omega,
                                  double* force_hyd, double* torque_hyd, int* n_out) {
    if (!ctx) return fail(nullptr, LBM_ERR_INVALID, "ctx is NULL");
    const int n = ctx->P.n;
    if (n_out) *n_out = n;
    if (n_cap < n && (pos || vel || omega || force_hyd || torque_hyd))
        return fail(ctx, LBM_ERR_INVALID, "n_cap smaller than the particle count");
    cudaStream_t sm = ctx->stream;
    if (n > 0) {
        if (pos) CK(cudaMemcpyAsync(pos, ctx->P.x, 24 * (size_t)n, cudaMemcpyDeviceToHost, sm));
        if (vel) CK(cudaMemcpyAsync(vel, ctx->P.u, 24 * (size_t)n, cudaMemcpyDeviceToHost, sm));
        if (omega) CK(cudaMemcpyAsync(omega, ctx->P.om, 24 * (size_t)n, cudaMemcpyDeviceToHost, sm));
    }
    std::vector<double> fp;
    if (n > 0 && (force_hyd || torque_hyd)) {
        fp.resize(6 * (size_t)n);
        CK(cudaMemcpyAsync(fp.data(), ctx->P.fp, 48 * (size_t)n, cudaMemcpyDeviceToHost, sm));
    }
    CK(cudaStreamSynchronize(sm));
    for (int i = 0; i < n && !fp.empty(); ++i)
        for (int a = 0; a < 3; ++a) {
            if (force_hyd) force_hyd[3 * i + a] = fp[6 * i + a];
            if (torque_hyd) torque_hyd[3 * i + a] = fp[6 * i + 3 + a];
        }
    return check_status(ctx);
}

// The state is copied on the context stream into a device snapshot (x, u,
// omega, and F, T split out of [n][6]), and from there to the host on the
// read-out stream, so the host copies overlap the steps queued after them.
// The next snapshot waits for the previous host copies.
lbm_status lbm_get_particle_state_async(lbm_ctx* ctx, int n_cap, double* pos, double* vel, double* omega,
                                        double* force_hyd, double* torque_hyd, int* n_out) {
    if (!ctx) return fail(nullptr, LBM_ERR_INVALID, "ctx is NULL");
    const int n = ctx->P.n;
    if (n_out) *n_out = n;
    if (n_cap < n && (pos || vel || omega || force_hyd || torque_hyd))
        return fail(ctx, LBM_ERR_INVALID, "n_cap smaller than the particle count");
    if (n == 0 || !(pos || vel || omega || force_hyd || torque_hyd)) return LBM_OK;
    if (!ctx->readout_stream) {
        CK(cudaMalloc(&ctx->snap, 15 * sizeof(double) * (size_t)std::max(ctx->max_particles, 1)));
        CK(cudaStreamCreateWithFlags(&ctx->readout_stream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ctx->ev_snap, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->ev_read, cudaEventDisableTiming));
    }
    cudaStream_t sm = ctx->stream, rs = ctx->readout_stream;
    const size_t b3 = 24 * (size_t)n;
    double* sx = ctx->snap;
    double* su = sx + 3 * (size_t)n;
    double* so = su + 3 * (size_t)n;
    double* sf = so + 3 * (size_t)n;   // F block, then T block
    if (ctx->read_pending) CK(cudaStreamWaitEvent(sm, ctx->ev_read, 0));
    if (pos) CK(cudaMemcpyAsync(sx, ctx->P.x, b3, cudaMemcpyDeviceToDevice, sm));
    if (vel) CK(cudaMemcpyAsync(su, ctx->P.u, b3, cudaMemcpyDeviceToDevice, sm));
    if (omega) CK(cudaMemcpyAsync(so, ctx->P.om, b3, cudaMemcpyDeviceToDevice, sm));
    if (force_hyd || torque_hyd) {
        launch_fp_split(ctx->P.fp, sf, n, sm);
        CK(cudaGetLastError());
        ctx->launches += 1;
    }
    CK(cudaEventRecord(ctx->ev_snap, sm));
    CK(cudaStreamWaitEvent(rs, ctx->ev_snap, 0));
    if (pos) CK(cudaMemcpyAsync(pos, sx, b3, cudaMemcpyDeviceToHost, rs));
    if (vel) CK(cudaMemcpyAsync(vel, su, b3, cudaMemcpyDeviceToHost, rs));
    if (omega) CK(cudaMemcpyAsync(omega, so, b3, cudaMemcpyDeviceToHost, rs));
    if (force_hyd) CK(cudaMemcpyAsync(force_hyd, sf, b3, cudaMemcpyDeviceToHost, rs));
    if (torque_hyd) CK(cudaMemcpyAsync(torque_hyd, sf + 3 * (size_t)n, b3, cudaMemcpyDeviceToHost, rs));
    CK(cudaEventRecord(ctx->ev_read, rs));
    ctx->read_pending = true;
    return LBM_OK;
}

// ------------------------------------------------------------ checkpoints

// a checkpoint: this header, the host-side insertion copies (fixed size for
// max_particles) and the whole device arena
struct CkptHeader {
    char magic[8];
    int32_t version, storage, max_particles, n[3];
    uint64_t arena_bytes;
    int32_t cur, hcur, stepped, dem_restart, motion, np;
    double ext_total[3], r_max;
};
constexpr char CKPT_MAGIC[8] = {'L', 'B', 'M', 'D', 'E', 'M', 'C', 'K'};

static size_t ckpt_bytes(const lbm_ctx* ctx) {
    return sizeof(CkptHeader) + 4 * sizeof(double) * (size_t)ctx->max_particles + ctx->bytes;
}

static void reset_graphs(lbm_ctx* ctx) {
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            if (ctx->step_graph[a][b]) {
                cudaGraphExecDestroy(ctx->step_graph[a][b]);
                ctx->step_graph[a][b] = nullptr;
                ctx->graph_launches[a][b] = 0;
            }
}

lbm_status lbm_checkpoint_bytes(const lbm_ctx* ctx, size_t* bytes) {
    if (!ctx || !bytes) return fail(nullptr, LBM_ERR_INVALID, "NULL argument");
    *bytes = ckpt_bytes(ctx);
    return LBM_OK;
}

lbm_status lbm_save(lbm_ctx* ctx, void* buf, size_t bytes) {
    if (!ctx || !buf) return fail(ctx, LBM_ERR_INVALID, "NULL argument");
    if (bytes < ckpt_bytes(ctx)) return fail(ctx, LBM_ERR_INVALID, "buffer smaller than lbm_checkpoint_bytes()");
    CK(cudaStreamSynchronize(ctx->stream));
    lbm_status st = check_status(ctx);
    if (st != LBM_OK) return st;
    CkptHeader h{};
    std::memcpy(h.magic, CKPT_MAGIC, 8);
    h.version = 1;
    h.storage = ctx->storage;
    h.max_particles = ctx->max_particles;
    for (int a = 0; a < 3; ++a) {
        h.n[a] = ctx->g.n[a];
        h.ext_total[a] = ctx->ext_total[a];
    }
    h.arena_bytes = ctx->bytes;
    h.cur = ctx->cur;
    h.hcur = ctx->hcur;
    h.stepped = ctx->stepped;
    h.dem_restart = ctx->dem_restart;
    h.motion = ctx->dem.fixed_particles;
    h.np = ctx->P.n;
    h.r_max = ctx->r_max;
    char* out = static_cast<char*>(buf);
    std::memcpy(out, &h, sizeof(h));
    double* hd = reinterpret_cast<double*>(out + sizeof(h));
    const size_t mp = (size_t)ctx->max_particles;
    std::fill(hd, hd + 4 * mp, 0.0);
    std::copy(ctx->hx.begin(), ctx->hx.end(), hd);
    std::copy(ctx->hR.begin(), ctx->hR.end(), hd + 3 * mp);
    CK(cudaMemcpy(out + sizeof(h) + 4 * sizeof(double) * mp, ctx->base, ctx->bytes, cudaMemcpyDeviceToHost));
    return LBM_OK;
}

lbm_status lbm_restore(lbm_ctx* ctx, const void* buf, size_t bytes) {
    if (!ctx || !buf) return fail(ctx, LBM_ERR_INVALID, "NULL argument");
    CkptHeader h;
    if (bytes < sizeof(h)) return fail(ctx, LBM_ERR_INVALID, "buffer too small for a checkpoint");
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, CKPT_MAGIC, 8) != 0 || h.version != 1)
        return fail(ctx, LBM_ERR_INVALID, "not a checkpoint of this library");
    if (h.storage != ctx->storage || h.max_particles != ctx->max_particles || h.n[0] != ctx->g.n[0] ||
        h.n[1] != ctx->g.n[1] || h.n[2] != ctx->g.n[2] || h.arena_bytes != ctx->bytes)
        return fail(ctx, LBM_ERR_INVALID, "checkpoint of a context with another grid, storage or capacity");
    if (bytes < ckpt_bytes(ctx)) return fail(ctx, LBM_ERR_INVALID, "checkpoint truncated");
    // the host-side state it carries must be one this context can hold
    if (h.np < 0 || h.np > ctx->max_particles || (h.cur != 0 && h.cur != 1) || (h.hcur != 0 && h.hcur != 1) ||
        h.motion < 0 || h.motion > 2 || !(h.r_max >= 0.0 && h.r_max <= 100.0))
        return fail(ctx, LBM_ERR_INVALID, "checkpoint header out of range");
    CK(cudaStreamSynchronize(ctx->stream));
    const char* in = static_cast<const char*>(buf);
    const double* hd = reinterpret_cast<const double*>(in + sizeof(h));
    const size_t mp = (size_t)ctx->max_particles;
    CK(cudaMemcpy(ctx->base, in + sizeof(h) + 4 * sizeof(double) * mp, ctx->bytes, cudaMemcpyHostToDevice));
    ctx->cur = h.cur;
    ctx->hcur = h.hcur;
    ctx->stepped = h.stepped != 0;
    ctx->dem_restart = h.dem_restart != 0;
    ctx->dem.fixed_particles = h.motion;
    ctx->P.n = h.np;
    ctx->r_max = h.r_max;
    for (int a = 0; a < 3; ++a) ctx->ext_total[a] = h.ext_total[a];
    ctx->hx.assign(hd, hd + 3 * (size_t)h.np);
    ctx->hR.assign(hd + 3 * mp, hd + 3 * mp + (size_t)h.np);
    reset_graphs(ctx);
    return LBM_OK;
}

lbm_status lbm_set_motion(lbm_ctx* ctx, int mode) {
    if (!ctx) return fail(nullptr, LBM_ERR_INVALID, "ctx is NULL");
    if (mode < 0 || mode > 2) return fail(ctx, LBM_ERR_INVALID, "mode must be 0 (DEM), 1 (fixed) or 2 (prescribed motion)");
    if (mode == ctx->dem.fixed_particles) return LBM_OK;
    CK(cudaStreamSynchronize(ctx->stream));
    // captured steps hold the old step structure
    reset_graphs(ctx);
    // the DEM's first Velocity-Verlet update needs F at the current state
    if (mode == 0 && ctx->stepped) ctx->dem_restart = true;
    ctx->dem.fixed_particles = mode;
    return LBM_OK;
}

lbm_status lbm_set_particle_velocity(lbm_ctx* ctx, int n, const double* vel, const double* omega) {
    if (!ctx) return fail(nullptr, LBM_ERR_INVALID, "ctx is NULL");
    if (n < 0 || n > ctx->P.n) return fail(ctx, LBM_ERR_INVALID, "n outside [0, particle count]");
    if (n == 0) return LBM_OK;
    cudaStream_t sm = ctx->stream;
    if (vel) CK(cudaMemcpyAsync(ctx->P.u, vel, 24 * (size_t)n, cudaMemcpyHostToDevice, sm));
    if (omega) CK(cudaMemcpyAsync(ctx->P.om, omega, 24 * (size_t)n, cudaMemcpyHostToDevice, sm));
    // the float32 view carries the velocities into the link arithmetic
    launch_view_update(ctx->P, sm);
    ctx->launches += 1;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(sm));
    return check_status(ctx);
}

lbm_status lbm_get_fields(lbm_ctx* ctx, double* rho, double* u, unsigned char* flags) {
    if (!ctx) return fail(nullptr, LBM_ERR_INVALID, "ctx is NULL");
    cudaStream_t sm = ctx->stream;
    const long long N = ctx->g.ncells;
    if (flags) CK(cudaMemcpyAsync(flags, ctx->flags, (size_t)N, cudaMemcpyDeviceToHost, sm));
    if (rho || u) {
        std::vector<double> buf(4 * (size_t)ctx->scratch_cells);
        for (long long first = 0; first < N; first += ctx->scratch_cells) {
            const long long cnt = (N - first) < ctx->scratch_cells ? (N - first) : ctx->scratch_cells;
            FieldsParams fp{};
            fp.storage = ctx->storage;
            fp.f = ctx->f[ctx->cur];
            fp.flags = ctx->flags;
            fp.g = ctx->g;
            fp.first_cell = first;
            fp.count = cnt;
            fp.accel = ctx->accel;
            fp.out = ctx->scratch;
            launch_fields(fp, sm);
            ctx->launches += 1;
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(buf.data(), ctx->scratch, 32 * (size_t)cnt, cudaMemcpyDeviceToHost, sm));
            CK(cudaStreamSynchronize(sm));
            if (rho) std::memcpy(rho + first, buf.data(), 8 * (size_t)cnt);
            if (u)
                for (int c = 0; c < 3; ++c)
                    std::memcpy(u + (size_t)c * N + first, buf.data() + (size_t)(c + 1) * cnt, 8 * (size_t)cnt);
        }
    }
    CK(cudaStreamSynchronize(sm));
    return check_status(ctx);
}

lbm_status lbm_sample_density(lbm_ctx* ctx, int n, const double* pos, double* rho) {
    if (!ctx || (n > 0 && (!pos || !rho))) return fail(ctx, LBM_ERR_INVALID, "NULL argument");
    if (n < 0 || (long long)n > ctx->scratch_cells) return fail(ctx, LBM_ERR_INVALID, "n outside [0, scratch size]");
    if (n == 0) return LBM_OK;
    cudaStream_t sm = ctx->stream;
    // points and results in the scratch buffer (4 doubles per scratch cell)
    CK(cudaMemcpyAsync(ctx->scratch, pos, 24 * (size_t)n, cudaMemcpyHostToDevice, sm));
    SampleParams sp{};
    sp.storage = ctx->storage;
    sp.f = ctx->f[ctx->cur];
    sp.flags = ctx->flags;
    sp.g = ctx->g;
    sp.n = n;
    sp.pos = ctx->scratch;
    sp.out = ctx->scratch + 3 * (size_t)n;
    launch_sample_density(sp, sm);
    ctx->launches += 1;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(rho, sp.out, 8 * (size_t)n, cudaMemcpyDeviceToHost, sm));
    CK(cudaStreamSynchronize(sm));
    return check_status(ctx);
}

lbm_status lbm_get_owner(lbm_ctx* ctx, int* owner) {
    if (!ctx || !owner) return fail(ctx, LBM_ERR_INVALID, "NULL argument");
    CK(cudaMemcpyAsync(owner, ctx->owner, 4 * (size_t)ctx->g.ncells, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

static double w_of(int q) { return q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

lbm_status lbm_get_pdfs(lbm_ctx* ctx, double* f) {
    if (!ctx || !f) return fail(ctx, LBM_ERR_INVALID, "NULL argument");
    const size_t N = (size_t)ctx->g.ncells;
    std::vector<char> raw(19 * N * ctx->elem);
    CK(cudaMemcpyAsync(raw.data(), ctx->f[ctx->cur], raw.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int q = 0; q < 19; ++q) {
        const double w = w_of(q);
        for (size_t k = 0; k < N; ++k) {
            const size_t j = q * N + k;
            double v;
            switch (ctx->storage) {
                case LBM_STORE_F64: v = reinterpret_cast<const double*>(raw.data())[j]; break;
                case LBM_STORE_F32: v = reinterpret_cast<const float*>(raw.data())[j]; break;
                case LBM_STORE_F16: v = __half2float(reinterpret_cast<const __half*>(raw.data())[j]); break;
                default: v = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(raw.data())[j]); break;
            }
            f[j] = v + w;
        }
    }
    return LBM_OK;
}

lbm_status lbm_set_pdfs(lbm_ctx* ctx, const double* f) {
    if (!ctx || !f) return fail(ctx, LBM_ERR_INVALID, "NULL argument");
    const size_t N = (size_t)ctx->g.ncells;
    std::vector<char> raw(19 * N * ctx->elem);
    for (int q = 0; q < 19; ++q) {
        const double w = w_of(q);
        for (size_t k = 0; k < N; ++k) {
            const size_t j = q * N + k;
            const double v = f[j] - w;
            switch (ctx->storage) {
                case LBM_STORE_F64: reinterpret_cast<double*>(raw.data())[j] = v; break;
                case LBM_STORE_F32: reinterpret_cast<float*>(raw.data())[j] = (float)v; break;
                case LBM_STORE_F16: reinterpret_cast<__half*>(raw.data())[j] = __float2half_rn((float)v); break;
                default: reinterpret_cast<__nv_bfloat16*>(raw.data())[j] = __float2bfloat16_rn((float)v); break;
            }
        }
    }
    CK(cudaMemcpyAsync(ctx->f[ctx->cur], raw.data(), raw.size(), cudaMemcpyHostToDevice, ctx->stream));
    // solid cells keep their NaN marker whatever was uploaded for them
    launch_solid_markers(map_params(ctx), ctx->stream);
    ctx->launches += 1;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

lbm_status lbm_profile(lbm_ctx* ctx, int enable) {
    if (!ctx) return fail(nullptr, LBM_ERR_INVALID, "ctx is NULL");
    if (enable) {
        CK(cudaStreamSynchronize(ctx->stream));
        ctx->ev_used = 0;
        ctx->prof_steps = 0;
    }
    ctx->profiling = enable != 0;
    return LBM_OK;
}

lbm_status lbm_profile_read(lbm_ctx* ctx, double* phase_ms, long long* steps) {
    if (!ctx || !phase_ms) return fail(ctx, LBM_ERR_INVALID, "NULL argument");
    CK(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < LBM_PHASES; ++k) phase_ms[k] = 0.0;
    for (size_t b = 0; b + LBM_PHASES + 1 <= ctx->ev_used; b += LBM_PHASES + 1)
        for (int k = 0; k < LBM_PHASES; ++k) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ctx->events[b + k], ctx->events[b + k + 1]));
            phase_ms[k] += ms;
        }
    if (steps) *steps = ctx->prof_steps;
    return LBM_OK;
}

long long lbm_launch_count(const lbm_ctx* ctx) { return ctx ? ctx->launches : 0; }

const char* lbm_last_error(const lbm_ctx* ctx) {
    if (ctx) return ctx->err.c_str();
    return g_err.c_str();
}

void lbm_destroy(lbm_ctx* ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    destroy_handles(ctx);
    if (ctx->own_memory && ctx->base) cudaFree(ctx->base);
    delete ctx;
}

// ====================================================================== batches

struct lbm_batch {
    std::vector<lbm_ctx*> ctx;
    std::vector<int> active;
    std::vector<int> tile_bx, zchunk;   // per instance, 0: automatic
    int blocks_per_sm = 0;              // 0: automatic
    int storage = 1;
    int num_sms = 152;
    int config_version = 0;
    cudaStream_t stream = nullptr;      // the stream the batch's steps run on
    std::vector<cudaStream_t> ctx_streams;   // the distinct streams of the contexts
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaStream_t capture = nullptr;     // private stream the steps are captured on
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        void* d_args = nullptr;
        int4* d_items = nullptr;
        void* d_dem = nullptr;             // one-block DEM steps of the instances, one entry each
        int n_items = 0;
        int n_dem = 0;
        void* d_gang = nullptr;            // parameter tables and block offsets of the gang launches
        int gang_launches = 0;             // gang launches in one step (0: per-instance branches)
        std::vector<long long> launches;   // kernel launches per instance in one step
        std::vector<int> hcur_after;       // history parity per instance after the step
    };
    // one captured step per (configuration, per instance: inactive, or buffer and history parities)
    std::map<std::vector<int>, Graph> graphs;
    long long launches = 0;             // launches of the batched dense kernel
    int captures = 0;                   // graphs captured so far
    double capture_ms = 0.0;            // host time spent capturing and instantiating them
    std::string err;
};

namespace {

lbm_status batch_fail(lbm_batch* b, lbm_status s, const std::string& msg) {
    if (b) b->err = msg;
    set_global_error(msg);
    return s;
}

#define BCK(call)                                                                                \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return batch_fail(b, LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void batch_clear_graphs(lbm_batch* b) {
    for (auto& kv : b->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.d_args) cudaFree(kv.second.d_args);
        if (kv.second.d_items) cudaFree(kv.second.d_items);
        if (kv.second.d_dem) cudaFree(kv.second.d_dem);
        if (kv.second.d_gang) cudaFree(kv.second.d_gang);
    }
    b->graphs.clear();
}

int batch_zchunk(const lbm_batch* b, int i) {
    const int z = b->zchunk[i];
    return z > 0 ? z : 16;
}
// the batched kernel's tiles are 32, 64 or 128 cells wide (threads map to
// cells by masks and shifts): the narrowest that covers the box, at most 128
int batch_tile_bx(const lbm_batch* b, int i) {
    const int t = b->tile_bx[i];
    const int nx = b->ctx[i]->g.n[0];
    return t > 0 ? t : (nx > 64 ? 128 : (nx > 32 ? 64 : 32));
}

// work items of the active instances, interleaved across instances so that
// concurrently running blocks spread over them
std::vector<int4> batch_items(const lbm_batch* b) {
    std::vector<std::vector<int4>> per(b->ctx.size());
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        if (!b->active[i]) continue;
        const Geom& g = b->ctx[i]->g;
        const int bx = batch_tile_bx(b, (int)i), by = 256 / bx, zc = batch_zchunk(b, (int)i);
        for (int z0 = 0; z0 < g.n[2]; z0 += zc)
            for (int y0 = 0; y0 < g.n[1]; y0 += by)
                for (int x0 = 0; x0 < g.n[0]; x0 += bx) per[i].push_back(make_int4((int)i, x0, y0, z0));
    }
    std::vector<int4> out;
    for (size_t k = 0;; ++k) {
        bool any = false;
        for (auto& v : per)
            if (k < v.size()) {
                out.push_back(v[k]);
                any = true;
            }
        if (!any) break;
    }
    return out;
}

// The table of one kind of gang launch: a parameter block per instance that
// takes part, and the prefix sums of the instances' launch-block counts.
struct GangTable {
    std::vector<unsigned char> bytes;
    std::vector<int> off{0};
    size_t elem = 0;
    int count() const { return (int)off.size() - 1; }
    int blocks() const { return off.back(); }
    void add(const void* params, int blocks) {
        const size_t at = bytes.size();
        bytes.resize(at + elem);
        std::memcpy(bytes.data() + at, params, elem);
        off.push_back(off.back() + blocks);
    }
};

// Capture one step of every active instance as gang launches (each per-step
// kernel once for all instances; the dense kernels in one persistent launch,
// the one-block DEM steps in one launch, the multi-block DEM steps as a
// position launch and one launch per subcycle, prescribed moves in one), in
// the order of a single instance's step: fluid body force and missing links,
// neighbour bins and lists, dense kernel, force finalisation, DEM, counters,
// tile scatter, mapping, refill.
lbm_status batch_capture_gang(lbm_batch* b, lbm_batch::Graph& G) {
    const size_t n = b->ctx.size();
    const size_t ab = batch_args_bytes(b->storage);
    const size_t db = dem_batch_entry_bytes();
    const std::vector<int4> items = batch_items(b);
    G.n_items = (int)items.size();
    std::vector<unsigned char> host(ab * n, 0), host_dem(db * n, 0);
    GangTable bc, zb, bins, nbr, fin, zc, scat, map, ref, pos, copy, pres;
    std::vector<GangTable> sub;   // one table per subcycle of the multi-block DEM steps
    bc.elem = bc_args_bytes();
    zb.elem = zc.elem = sizeof(ZeroSpan);
    bins.elem = nbr.elem = sizeof(DemParams);
    fin.elem = sizeof(FinalizeParams);
    scat.elem = map.elem = sizeof(MapParams);
    ref.elem = sizeof(RefillParams);
    pos.elem = copy.elem = pres.elem = sizeof(DemGangEntry);
    G.launches.assign(n, 0);
    G.hcur_after.assign(n, 0);
    for (size_t i = 0; i < n; ++i) {
        lbm_ctx* c = b->ctx[i];
        G.hcur_after[i] = c->hcur;
        if (!b->active[i]) continue;
        const lbm_dem& d = c->dem;
        const int np = c->P.n;
        const bool move = np > 0 && d.fixed_particles != 1;
        const bool dem = move && d.fixed_particles == 0;
        LbmStepParams lp;
        fill_step_params(c, lp);
        std::vector<unsigned char> bca(bc.elem, 0);
        fill_bc_args(lp, bca.data());
        // the missing-link and refill lists grow with the particle count
        const int list_blocks = std::min(8 * b->num_sms, 1 + np / 8);
        bc.add(bca.data(), lp.missing_links ? list_blocks : 1);
        fill_batch_args(lp, batch_tile_bx(b, (int)i), batch_zchunk(b, (int)i), &host[ab * i]);
        DemParams dp = dem_params(c);
        if (dem) {
            const ZeroSpan z{c->P.bin_count, dp.nbins[0] * dp.nbins[1] * dp.nbins[2], 0};
            zb.add(&z, (z.words + 127) / 128 < 64 ? (z.words + 127) / 128 : 64);
            bins.add(&dp, (np + 127) / 128);
            nbr.add(&dp, (32 * np + 127) / 128);
        }
        if (np > 0) {
            FinalizeParams fp{};
            fp.P = c->P;
            fp.use_fixed = c->storage != LBM_STORE_F64;
            fp.first_step = 0;
            fp.averaging = d.force_averaging;
            fin.add(&fp, (np + 127) / 128);
        }
        if (dem && np <= DEM_ONE_BLOCK_MAX) {
            fill_dem_batch_entry(dp, c->hcur, d.n_sub, &host_dem[db * G.n_dem]);
            G.n_dem += 1;
            if (d.n_sub & 1) G.hcur_after[i] = 1 - c->hcur;
        } else if (dem) {
            // the multi-block DEM step: first position update, n_sub
            // subcycles (history parity and state buffer alternating), the
            // copy back into buffer 0 after an odd count
            DemGangEntry ge{};
            ge.p = dp;
            pos.add(&ge, (np + 127) / 128);
            int hc = c->hcur, cur = 0;
            for (int k = 0; k < d.n_sub; ++k) {
                if ((int)sub.size() <= k) {
                    sub.emplace_back();
                    sub.back().elem = sizeof(DemGangEntry);
                }
                ge.p.hin = hc;
                ge.p.hout = 1 - hc;
                ge.cur = cur;
                ge.last = k == d.n_sub - 1;
                sub[k].add(&ge, (np + DEM_ONE_BLOCK_MAX - 1) / DEM_ONE_BLOCK_MAX);
                hc = 1 - hc;
                cur = 1 - cur;
            }
            if (cur == 1) copy.add(&ge, (3 * np + 127) / 128);
            G.hcur_after[i] = hc;
        } else if (move) {
            DemGangEntry ge{};
            ge.p = dp;
            pres.add(&ge, (np + 127) / 128);
        }
        if (move) {
            // n_solid and the missing-link and refill counts (16 bytes)
            const ZeroSpan z{reinterpret_cast<int*>(c->n_solid), 4, 0};
            zc.add(&z, 1);
            const MapParams mp = map_params(c);
            scat.add(&mp, (32 * np + 127) / 128);
            map.add(&mp, (int)c->ntiles);
            RefillParams rp{};
            rp.storage = c->storage;
            rp.f = c->f[1 - c->cur];
            rp.flags = c->flags;
            rp.list_owner = c->refill_owner;
            rp.g = c->g;
            rp.P = c->P;
            rp.list = c->refill_list;
            rp.count = c->refill_count;
            rp.cap = c->refill_cap;
            rp.s_nu = 1.0 / c->relax.tau;
            rp.accel = c->accel;
            ref.add(&rp, list_blocks);
        }
    }
    // one device buffer: the tables, then their offsets (16-byte aligned pieces)
    std::vector<GangTable*> tabs = {&bc, &zb, &bins, &nbr, &fin, &zc, &scat, &map, &ref, &pos, &copy, &pres};
    for (auto& t : sub) tabs.push_back(&t);
    const int nt = (int)tabs.size();
    size_t total = 0;
    std::vector<size_t> at_tab(nt), at_off(nt);
    for (int k = 0; k < nt; ++k) {
        at_tab[k] = total;
        total += (tabs[k]->bytes.size() + 15) & ~size_t(15);
        at_off[k] = total;
        total += (sizeof(int) * tabs[k]->off.size() + 15) & ~size_t(15);
    }
    BCK(cudaMalloc(&G.d_args, ab * n));
    BCK(cudaMalloc(&G.d_items, sizeof(int4) * std::max<size_t>(1, items.size())));
    BCK(cudaMalloc(&G.d_dem, db * n));
    BCK(cudaMalloc(&G.d_gang, std::max<size_t>(total, 16)));
    std::vector<unsigned char> gang(std::max<size_t>(total, 16), 0);
    for (int k = 0; k < nt; ++k) {
        if (!tabs[k]->bytes.empty()) std::memcpy(gang.data() + at_tab[k], tabs[k]->bytes.data(), tabs[k]->bytes.size());
        std::memcpy(gang.data() + at_off[k], tabs[k]->off.data(), sizeof(int) * tabs[k]->off.size());
    }
    char* dg = static_cast<char*>(G.d_gang);
    auto T = [&](int k) { return static_cast<const void*>(dg + at_tab[k]); };
    auto O = [&](int k) { return reinterpret_cast<const int*>(dg + at_off[k]); };
    cudaGraph_t g = nullptr;
    const cudaStream_t cs = b->capture;
    int launches = 0;
    auto gl = [&](int k) { return tabs[k]->count() > 0 ? 1 : 0; };
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        launch_boundary_gang(b->storage, T(0), O(0), bc.count(), bc.blocks(), BC_ACCEL | BC_LINKS, cs);
        launch_gang(GANG_ZERO, T(1), O(1), zb.count(), zb.blocks(), cs);
        launch_gang(GANG_BINS, T(2), O(2), bins.count(), bins.blocks(), cs);
        launch_gang(GANG_NEIGHBOURS, T(3), O(3), nbr.count(), nbr.blocks(), cs);
        launches += gl(0) + gl(1) + gl(2) + gl(3);
        if (G.n_items > 0) {
            const int bps = b->blocks_per_sm > 0 ? b->blocks_per_sm : (b->storage == 0 ? 2 : 4);
            const int grid = std::min(G.n_items, bps * b->num_sms);
            launch_stream_collide_batch(b->storage, G.d_args, G.d_items, G.n_items, grid, cs);
            launches += 1;
        }
        launch_gang(GANG_FINALIZE, T(4), O(4), fin.count(), fin.blocks(), cs);
        launches += gl(4);
        const int pf32 = b->storage != LBM_STORE_F64;
        if (G.n_dem > 0) {
            launch_dem_step_batch(G.d_dem, G.n_dem, pf32, cs);
            launches += 1;
        }
        launch_dem_gang(DEM_GANG_POSITION, pf32, T(9), O(9), pos.count(), pos.blocks(), cs);
        launches += gl(9);
        for (int k = 0; k < (int)sub.size(); ++k) {
            launch_dem_gang(DEM_GANG_SUBCYCLE, pf32, T(12 + k), O(12 + k), sub[k].count(), sub[k].blocks(), cs);
            launches += gl(12 + k);
        }
        launch_dem_gang(DEM_GANG_COPY, pf32, T(10), O(10), copy.count(), copy.blocks(), cs);
        launch_dem_gang(DEM_GANG_PRESCRIBED, pf32, T(11), O(11), pres.count(), pres.blocks(), cs);
        launches += gl(10) + gl(11);
        launch_gang(GANG_ZERO, T(5), O(5), zc.count(), zc.blocks(), cs);
        launch_map_gang(GANG_SCATTER, b->storage, T(6), O(6), scat.count(), scat.blocks(), cs);
        launch_map_gang(GANG_MAP, b->storage, T(7), O(7), map.count(), map.blocks(), cs);
        launch_map_gang(GANG_REFILL, b->storage, T(8), O(8), ref.count(), ref.blocks(), cs);
        launches += gl(5) + gl(6) + gl(7) + gl(8);
        e = cudaGetLastError();
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = e2;
    }
    G.gang_launches = launches;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    BCK(e);
    BCK(cudaMemcpy(G.d_args, host.data(), host.size(), cudaMemcpyHostToDevice));
    if (G.n_items > 0)
        BCK(cudaMemcpy(G.d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
    if (G.n_dem > 0) BCK(cudaMemcpy(G.d_dem, host_dem.data(), db * G.n_dem, cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(G.d_gang, gang.data(), gang.size(), cudaMemcpyHostToDevice));
    return LBM_OK;
}

}  // namespace

lbm_status lbm_batch_create(lbm_ctx* const* ctxs, int n, void* cuda_stream, lbm_batch** out) {
    lbm_batch* b = nullptr;
    if (!ctxs || n < 1 || !out) return batch_fail(b, LBM_ERR_INVALID, "lbm_batch_create: ctxs, n >= 1 and out required");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return batch_fail(b, LBM_ERR_INVALID, "lbm_batch_create: NULL context");
        if (ctxs[i]->storage != ctxs[0]->storage)
            return batch_fail(b, LBM_ERR_INVALID, "lbm_batch_create: all instances need one storage format");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return batch_fail(b, LBM_ERR_INVALID, "lbm_batch_create: a context appears twice");
    }
    b = new lbm_batch();
    b->ctx.assign(ctxs, ctxs + n);
    b->active.assign(n, 1);
    b->tile_bx.assign(n, 0);
    b->zchunk.assign(n, 0);
    b->storage = ctxs[0]->storage;
    b->num_sms = ctxs[0]->num_sms;
    b->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctxs[0]->stream;
    for (int i = 0; i < n; ++i)
        if (std::find(b->ctx_streams.begin(), b->ctx_streams.end(), ctxs[i]->stream) == b->ctx_streams.end())
            b->ctx_streams.push_back(ctxs[i]->stream);
    cudaError_t e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        lbm_batch_destroy(b);
        cudaGetLastError();
        return batch_fail(nullptr, LBM_ERR_CUDA, std::string("lbm_batch_create: ") + cudaGetErrorString(e));
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_set_launch(lbm_batch* b, int instance, int tile_bx, int zchunk, int blocks_per_sm) {
    if (!b) return batch_fail(b, LBM_ERR_INVALID, "batch is NULL");
    if (instance < -1 || instance >= (int)b->ctx.size())
        return batch_fail(b, LBM_ERR_INVALID, "instance out of range (-1 = all)");
    if (!(tile_bx == 0 || tile_bx == 32 || tile_bx == 64 || tile_bx == 128))
        return batch_fail(b, LBM_ERR_INVALID, "tile_bx must be 0 (automatic), 32, 64 or 128");
    if (zchunk < 0 || zchunk > 4096) return batch_fail(b, LBM_ERR_INVALID, "zchunk must be in 0 .. 4096");
    if (blocks_per_sm < 0 || blocks_per_sm > 8) return batch_fail(b, LBM_ERR_INVALID, "blocks_per_sm must be in 0 .. 8");
    for (size_t i = 0; i < b->ctx.size(); ++i)
        if (instance < 0 || (int)i == instance) {
            b->tile_bx[i] = tile_bx;
            b->zchunk[i] = zchunk;
        }
    b->blocks_per_sm = blocks_per_sm;
    BCK(cudaStreamSynchronize(b->stream));
    batch_clear_graphs(b);
    b->config_version += 1;
    return LBM_OK;
}

lbm_status lbm_batch_set_active(lbm_batch* b, int instance, int active) {
    if (!b) return batch_fail(b, LBM_ERR_INVALID, "batch is NULL");
    if (instance < 0 || instance >= (int)b->ctx.size()) return batch_fail(b, LBM_ERR_INVALID, "instance out of range");
    b->active[instance] = active ? 1 : 0;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int n_steps) {
    if (!b) return batch_fail(b, LBM_ERR_INVALID, "batch is NULL");
    if (n_steps < 0) return batch_fail(b, LBM_ERR_INVALID, "n_steps must be >= 0");
    bool any = false;
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        if (!b->active[i]) continue;
        const lbm_ctx* c = b->ctx[i];
        if (!c->stepped || c->dem_restart || c->profiling)
            return batch_fail(b, LBM_ERR_STATE,
                              "lbm_batch_step: every active instance must have stepped once on its own, "
                              "without a pending motion switch or phase timing");
        any = true;
    }
    if (!any || n_steps == 0) return LBM_OK;
    // the steps start after the work queued on the contexts' streams and that
    // work resumes after them
    const bool foreign = b->ctx_streams.size() != 1 || b->ctx_streams[0] != b->stream;
    if (foreign)
        for (cudaStream_t cs : b->ctx_streams) {
            BCK(cudaEventRecord(b->ev_in, cs));
            BCK(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
        }
    for (int step = 0; step < n_steps; ++step) {
        std::vector<int> key{b->config_version};
        for (size_t i = 0; i < b->ctx.size(); ++i)
            key.push_back(b->active[i] ? 2 * b->ctx[i]->cur + b->ctx[i]->hcur : -1);
        auto it = b->graphs.find(key);
        if (it == b->graphs.end()) {
            lbm_batch::Graph G;
            const auto t0 = std::chrono::steady_clock::now();
            lbm_status st = batch_capture_gang(b, G);
            b->capture_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            b->captures += 1;
            if (st != LBM_OK) {
                if (G.exec) cudaGraphExecDestroy(G.exec);
                if (G.d_args) cudaFree(G.d_args);
                if (G.d_items) cudaFree(G.d_items);
                if (G.d_dem) cudaFree(G.d_dem);
                if (G.d_gang) cudaFree(G.d_gang);
                return st;
            }
            it = b->graphs.emplace(key, G).first;
        }
        const lbm_batch::Graph& G = it->second;
        BCK(cudaGraphLaunch(G.exec, b->stream));
        b->launches += G.gang_launches > 0 ? G.gang_launches : (G.n_items > 0 ? 1 : 0) + (G.n_dem > 0 ? 1 : 0);
        for (size_t i = 0; i < b->ctx.size(); ++i) {
            if (!b->active[i]) continue;
            lbm_ctx* c = b->ctx[i];
            c->launches += G.launches[i];
            c->hcur = G.hcur_after[i];
            c->cur = 1 - c->cur;
        }
    }
    if (foreign) {
        BCK(cudaEventRecord(b->ev_out, b->stream));
        for (cudaStream_t cs : b->ctx_streams) BCK(cudaStreamWaitEvent(cs, b->ev_out, 0));
    }
    return LBM_OK;
}

lbm_status lbm_batch_sync(lbm_batch* b) {
    if (!b) return batch_fail(b, LBM_ERR_INVALID, "batch is NULL");
    BCK(cudaStreamSynchronize(b->stream));
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        lbm_status st = check_status(b->ctx[i]);
        if (st != LBM_OK) return batch_fail(b, st, "instance " + std::to_string(i) + ": " + b->ctx[i]->err);
    }
    return LBM_OK;
}

long long lbm_batch_launch_count(const lbm_batch* b) { return b ? b->launches : 0; }

lbm_status lbm_batch_capture_stats(const lbm_batch* b, int* captures, double* capture_ms) {
    if (!b) return batch_fail(nullptr, LBM_ERR_INVALID, "batch is NULL");
    if (captures) *captures = b->captures;
    if (capture_ms) *capture_ms = b->capture_ms;
    return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : g_err.c_str(); }

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_clear_graphs(b);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->capture) cudaStreamDestroy(b->capture);
    delete b;
}

}  // extern "C"
