// launch.h -- host-side launchers of the device kernels (internal to the library).
#pragma once

#include <string>

#include "common.cuh"

namespace lbmdem {

struct LbmStepParams {
    int storage;                 // 0 f64, 1 f32, 2 f16, 3 bf16
    const void* src;
    void* dst;
    const uint8_t* flags;
    const int* owner;                // particle of a solid cell, -1 for fluid
    Geom g;
    double s_plus, s_minus, s_b_shell, s_b_bulk;
    int bulk_corr;
    double a_user[3];
    double ext_total[3];
    const unsigned long long* n_solid;
    int counterforce;
    Particles P;
    int missing_links;
    int* status;
    const unsigned int* miss_list;   // solid cells with possible missing links
    const int* miss_count;
    int miss_cap;
    int num_sms;                     // multiprocessors of the device (grid sizing)
    double* accel_d;                 // out: fluid body force of the step [3]
    float* accel_f;
    int use_staged;                  // 1: the dense kernel with bulk-copy staging where it applies
    int tile_bx;                     // x extent of the dense kernel's tile (0: automatic)
    int zchunk;                      // z planes per block of the dense kernel (0: automatic)
    int staged_zchunk;               // z planes per work item of the staged kernel (0: automatic)
};
// BC_ACCEL: the fluid body force of the step; BC_LINKS: the missing links
constexpr int BC_ACCEL = 1, BC_LINKS = 2;
void launch_boundary(const LbmStepParams& p, cudaStream_t st, int mode);
void launch_stream_collide(const LbmStepParams& p, cudaStream_t st);
// kernel attributes on the current device (before any launch or capture)
cudaError_t prepare_stream_collide(int storage);
// the dense kernels of many boxes in one persistent launch: per instance one
// argument block (batch_args_bytes(storage) bytes, filled by fill_batch_args)
// in device memory, and a table of work items (instance, x0, y0, z0)
size_t batch_args_bytes(int storage);
void fill_batch_args(const LbmStepParams& p, int tile_bx, int zchunk, void* out);
int default_tile_bx(int nx);
void launch_stream_collide_batch(int storage, const void* d_args, const int4* d_items, int n_items, int grid,
                                 cudaStream_t st);
// the dense kernel with bulk-copy staging of the pulls (4- and 2-byte formats)
bool staged_applicable(const LbmStepParams& p);
void launch_stream_collide_staged(const LbmStepParams& p, cudaStream_t st);
cudaError_t prepare_stream_collide_staged(int storage);

struct MapParams {
    Geom g;
    Particles P;
    uint8_t* flags;
    int* owner;
    void* pdf[2];           // both PDF buffers (NaN markers into cells that turn solid), or NULL
    int elem;               // bytes per stored PDF value (8, 4 or 2)
    int ntile[3];
    int* tile_count;
    int* tile_list;
    double shell_width;
    unsigned int* refill_list;
    int* refill_owner;      // former particle of each refill-list cell
    int* refill_count;
    int refill_cap;
    unsigned long long* n_solid;
    unsigned int* miss_list;
    int* miss_count;
    int miss_cap;
    int small[3];           // periodic axis too short for one image per tile
    int* status;
};
void launch_tile_scatter(const MapParams& p, cudaStream_t st);
void launch_map(const MapParams& p, cudaStream_t st);
// NaN markers into every PDF slot of every solid cell of both buffers
void launch_solid_markers(const MapParams& p, cudaStream_t st);

struct RefillParams {
    int storage;
    void* f;
    const uint8_t* flags;
    const int* list_owner;  // former particle of each list cell
    Geom g;
    Particles P;
    const unsigned int* list;
    const int* count;
    int cap;
    double s_nu;
    const double* accel;   // fluid body force of the step [3]
};
void launch_refill(const RefillParams& p, cudaStream_t st);

struct FieldsParams {
    int storage;
    const void* f;
    const uint8_t* flags;
    Geom g;
    long long first_cell;   // slab of cells [first_cell, first_cell + count)
    long long count;
    const double* accel;
    double* out;            // [4 * count]: rho, ux, uy, uz blocks
};
void launch_fields(const FieldsParams& p, cudaStream_t st);

struct SampleParams {
    int storage;
    const void* f;
    const uint8_t* flags;
    Geom g;
    int n;
    const double* pos;      // [3n] sample points
    double* out;            // [n] density at each point
};
void launch_sample_density(const SampleParams& p, cudaStream_t st);

struct FinalizeParams {
    Particles P;
    int use_fixed;          // accumulators in fixed point (float32 path)
    int first_step;
    int averaging;
};
void launch_finalize(const FinalizeParams& p, cudaStream_t st);

// interaction constants of the DEM in the precision of its pair arithmetic
template <typename T>
struct DemConsts {
    T mu_f, cut_n, cut_tt, cut_tr, cut_max, inv_cut_n, inv_cut_tt, inv_cut_tr, min_a, min_b;
    T log_e, pi2_log_e2, kappa, sqrt_kappa, mu_p, Tc, dt;
};

struct DemParams {
    Geom g;
    Particles P;
    int nbins[3];
    double binsize[3];
    double cut_max;         // largest lubrication cut-off
    double e_dry, Tc, nu_p, mu_p;
    double cut_n, cut_tt, cut_tr, min_a, min_b;
    // derived on the host: 1 / cut-offs, log e_dry, pi^2 + (log e_dry)^2,
    // kappa = 2 (1 - nu) / (2 - nu) and its square root
    double inv_cut_n, inv_cut_tt, inv_cut_tr, log_e, pi2_log_e2, kappa, sqrt_kappa;
    double gravity[3];
    double mu_f;            // dynamic fluid viscosity rho0 nu
    int lubrication, tangential;
    double dt;              // subcycle time step 1/n_sub
    int hin, hout;          // history buffers to read and write
    // 1: pair and wall laws in float32 (separations and overlaps from the
    // float64 positions), 0: all in float64
    int pair_f32;
    DemConsts<double> kd;
    DemConsts<float> kf;
    int* status;
};
// the one-block DEM steps of many instances in one launch (batches)
size_t dem_batch_entry_bytes();
void fill_dem_batch_entry(const DemParams& p, int hcur, int n_sub, void* out);
void launch_dem_step_batch(const void* d_table, int count, int pair_f32, cudaStream_t st);
void launch_bins(const DemParams& p, cudaStream_t st);
void launch_neighbours(const DemParams& p, cudaStream_t st);
void launch_dem_position(const DemParams& p, cudaStream_t st);
void launch_dem_subcycle(const DemParams& p, int cur, int init, int last, cudaStream_t st);
// at most this many particles: the position update, all subcycles and the
// state copy of a step in one single-block launch
constexpr int DEM_ONE_BLOCK_MAX = 32;
void launch_dem_step_one_block(const DemParams& p, int hcur, int n_sub, cudaStream_t st);
void launch_state_copy(const Particles& P, cudaStream_t st);
void launch_fp_split(const double* fp, double* out, int n, cudaStream_t st);

// Gang launches (gang.cuh): one launch of a per-step kernel for many
// instances; table holds n parameter blocks in device memory, off the n + 1
// prefix sums of their block counts (blocks = off[n]).
enum { GANG_FINALIZE = 1, GANG_BINS, GANG_NEIGHBOURS, GANG_ZERO, GANG_SCATTER, GANG_MAP, GANG_REFILL };
struct ZeroSpan {
    int* p;        // words set to zero
    int words;
    int pad;
};
void launch_gang(int kind, const void* table, const int* off, int n, int blocks, cudaStream_t st);
void launch_map_gang(int kind, int storage, const void* table, const int* off, int n, int blocks, cudaStream_t st);
// an instance's entry of a DEM gang launch: its parameters (hin, hout for a
// subcycle), the subcycle's state buffer and whether it is the last one
enum { DEM_GANG_POSITION = 1, DEM_GANG_SUBCYCLE, DEM_GANG_COPY, DEM_GANG_PRESCRIBED };
struct DemGangEntry {
    DemParams p;
    int cur, last, pad0, pad1;
};
void launch_dem_gang(int kind, int pair_f32, const void* table, const int* off, int n, int blocks, cudaStream_t st);
size_t bc_args_bytes();
void fill_bc_args(const LbmStepParams& p, void* out);
void launch_boundary_gang(int storage, const void* table, const int* off, int n, int blocks, int mode,
                          cudaStream_t st);
void launch_view_update(const Particles& P, cudaStream_t st);
void launch_prescribed_move(const Particles& P, const Geom& g, cudaStream_t st);

// message returned by lbm_last_error(NULL)
void set_global_error(const std::string& msg);

}  // namespace lbmdem
