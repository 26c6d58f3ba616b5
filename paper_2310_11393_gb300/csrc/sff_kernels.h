// Host-side launch interface of the kernels (no CUDA types beyond the runtime's).
#pragma once

#include <cuda_runtime.h>

#include "sff_common.cuh"

namespace sff {

// Field array layout: 18 components of na_z*na_y*na_x elements each:
//   [0..5]  E, B of buffer set 0   [6..11] E, B of buffer set 1
//   [12..14] J of set 0            [15..17] J of set 1
// The push reads set p and deposits J_p; the field solver reads set p and J_p, writes
// set 1-p and clears J_{1-p}.  p = DevState::parity flips at the end of each step.
constexpr int NFCOMP = 18;
// With the incident field on the grid, components 18..23 hold E, B of the total field at t^n
// (scattered + incident), which the push gathers.
constexpr int COMP_TOTAL = 18, NFCOMP_INC = 24;
__host__ __device__ constexpr int comp_eb(int parity) { return 6 * parity; }
__host__ __device__ constexpr int comp_j(int parity) { return 12 + 3 * parity; }

// One launch group: simulations of one dimension and precision advanced together.
// Particles are processed in chunks of at most SimDev::chunk particles of one tile; the
// chunks of all simulations of the group are numbered 0 .. gprefix[nsims)-1 each step.
struct Group {
    const SimDev* sims;    // device array
    int nsims;
    int* gprefix;          // device [nsims + 1]: first global chunk of each simulation
    const Work* ywork;     // field-solver tiles, device
    int nywork;
    int* counters;         // device: [0] push, [1] scatter, [2] field solver
    int dim, prec;
    size_t push_smem, yee_smem;
    int push_grid, yee_grid, scatter_grid;
    int inc_any, inc_segs, inc_rows;   // incident field on the grid: any member, x segments, rows
    int scan_blocks;                   // single simulation: blocks of the multi-block tile scan
    int cellscan_grid;                 // cell sort: blocks per simulation of the per-tile cell scan
    const SimDev* one;                 // single simulation: its host descriptor, passed by value to the
                                       // push (the same contents as sims[0]); nullptr for batches
};

// 3D field solver: columns of Y3_PX x Y3_PY points (x, y) marching along z through a
// segment of planes; a ring of Y3_NS planes of E, B, J per column (TMA), Y3_NT threads.
constexpr int Y3_PX = 32, Y3_PY = 8, Y3_NS = 4, Y3_NT = 384;
constexpr int Y3_BX = Y3_PX + 8, Y3_BY = Y3_PY + 4;
// 2D field solver: tiles of 32 x Y2_PY points, one warp per box row plus the rest
constexpr int Y2_PX = 32, Y2_PY = 16;
constexpr int Y2_NT = 32 * ((Y2_PY + 3) + (3 * Y2_PY + 8 + 31) / 32);
// dynamic shared memory of the 2D field solver: two box buffers, Bh, N, the output tile
__host__ __device__ constexpr size_t yee2_smem(int es)
{
    return 2 * round128(round128(6ull * (Y2_PX + 8) * (Y2_PY + 4) * es) + 3ull * (Y2_PX + 8) * (Y2_PY + 4) * es) +
           2 * round128(3ull * (Y2_PX + 8) * (Y2_PY + 4) * es) + 6ull * Y2_PX * Y2_PY * es;
}
// dynamic shared memory of the 3D field solver for element size es (bytes)
__host__ __device__ constexpr size_t yee3_smem(int es)
{
    return Y3_NS * round128(9ull * Y3_BX * Y3_BY * es) + round128(9ull * Y3_BX * Y3_BY * es) +
           round128(6ull * Y3_BX * Y3_BY * es) + round128(12ull * Y3_PX * Y3_PY * es);
}

// per-step kernels (asynchronous)
void launch_prefix(const Group& g, cudaStream_t s);
// push + deposit; each particle goes straight into its destination tile's slots of the
// other buffer set (`sorting`: members with a cell sort are pushed in place instead and
// placed by launch_cell_sort)
void launch_push(const Group& g, bool sorting, cudaStream_t s);
void launch_scan(const Group& g, cudaStream_t s);
// the placement of a cell-sort step: cell counts, per-tile cell scan, scatter by cell of
// the members that have a cell sort (after launch_push(.., true, ..) and the tile scan)
void launch_cell_sort(const Group& g, cudaStream_t s);
void launch_yee(const Group& g, cudaStream_t s);
void launch_step_end(const Group& g, cudaStream_t s);
void launch_incident_grid(const Group& g, cudaStream_t s);

// set-up: particles written linearly into buffer set 1, then sorted into set 0
void launch_gen_slab(const SimDev* sim, int dim, int prec, long long n, int ppc, const int slab_lo[3],
                     const int slab_n[3], unsigned long long seed, double weight, cudaStream_t s);
void launch_count_linear(const SimDev* sim, int dim, int prec, long long n, cudaStream_t s);
void launch_sort_linear(const SimDev* sim, int dim, int prec, long long n, cudaStream_t s);
void launch_place_slab(const SimDev* sim, int dim, int prec, long long n, int ppc, const int lo[3], const int hi[3],
                       cudaStream_t s);
// set-up: compact slots of set q from the counts, then (after the particles are placed)
// the frame counts of its n particles and the slots of set 1 - q
void launch_scan_one(const SimDev* sim, int q, cudaStream_t s);
void launch_next_slots(const SimDev* sim, int dim, int prec, int q, long long n, cudaStream_t s);

// diagnostics
// adds scale * rho_e of the particles in the n_slots slots of the current set to rho
void launch_charge(const SimDev* sim, int dim, int prec, long long n_slots, double* rho, cudaStream_t s,
                   double scale = 1.0);
void launch_gauss(const SimDev* sim, int dim, int prec, const int n[3], const double* rho, unsigned long long* out_bits,
                  cudaStream_t s);
void launch_energy_fields(const SimDev* sim, int dim, int prec, const int n[3], double* acc2, cudaStream_t s);
void launch_energy_particles(const SimDev* sim, int dim, int prec, long long n_alive, long long n_exits,
                             double* acc2, cudaStream_t s);
void launch_histogram(const SimDev* sim, int dim, int prec, long long n_alive, long long n_exits, int n_e,
                      double e_max, int n_a, double* bins, cudaStream_t s);
void launch_eval_incident(const SimDev* sim, int dim, int prec, long long n, const double* pts, double* out,
                          cudaStream_t s);

// streaming multiprocessors of the current device (queried once per device)
int device_sms();

// Is field-solver tile t a work item?  In 2D and 3D a tile (column) whose first point lies on
// the node line / plane x = n_x (or y = n_y), which holds nothing else, is not: the one before
// it writes that line / plane of E and B and clears its J.
inline bool yee_tile_active(const SimDev& h, int dim, int t)
{
    if (dim == 1) return true;
    const int cx = t % h.nyt[0], cy = (t / h.nyt[0]) % h.nyt[1];
    return cx * h.yt[0] != h.n[0] && cy * h.yt[1] != h.n[1];
}

// kernel attributes (dynamic shared memory opt-in); returns blocks per SM
int prepare_push(int dim, int prec, size_t smem);
int prepare_yee(int dim, int prec, size_t smem);
int scatter_blocks_per_sm(int dim, int prec);

}  // namespace sff
