// Host-side simulation handle shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/pic.h"
#include "sff_common.cuh"
#include "sff_kernels.h"

using sff::Group;
using sff::SimDev;
using sff::Work;

// bump allocator over one device allocation (256-byte aligned pieces)
struct Arena {
    char* base = nullptr;
    size_t size = 0, used = 0;
    void* take(size_t bytes)
    {
        size_t off = (used + 255) & ~size_t(255);
        if (off + bytes > size) return nullptr;
        used = off + bytes;
        return base + off;
    }
};

struct GraphBundle {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

struct pic_sim {
    pic_config cfg;
    pic_params prm;
    int device = 0;
    int es = 4;                  // element size
    SimDev h;                    // host copy of the descriptor
    SimDev* d = nullptr;         // device descriptor
    pic_allocator alloc{};
    bool use_cuda_malloc = true;
    Arena arena;
    // single-simulation launch group
    Group grp{};
    Work* d_ywork = nullptr;
    int nywork = 0;              // field-solver work items (yee_tile_active)
    int* d_gprefix = nullptr;    // chunk numbering of the single-simulation group
    int* d_counters = nullptr;
    double* d_acc = nullptr;     // 8 doubles
    unsigned long long* d_bits = nullptr;
    GraphBundle step_graph;
    // id of the launch group whose chunk numbering and work counters are set for this sim's
    // current particle layout (each step ends by setting them for its own group; any other
    // change of the layout clears it, and the next step of a group starts with k_prefix)
    long long prefix_group = 0;
    long long own_group_id = 0;  // id of the single-simulation group
    GraphBundle sort_graph;      // the step whose re-sort orders the tiles by cell
    int sort_every = 0;          // steps between cell sorts (0: none)
    int since_sort = 0;          // steps through pic_step / pic_profile_step since the last one
    cudaStream_t cap_stream = nullptr;
    cudaStream_t cap_stream2 = nullptr;   // the field-solve branch of the captured step
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::string err;
    long long nalloc_tot = 0;    // na_x*na_y*na_z
    long long pcap = 0;          // particle capacity (the buffer sets hold h.cap slots)
};


// a fresh launch-group id (never 0; never reused in the process)
long long new_group_id();

// drop cached batch graphs that contain `s` (called by pic_destroy)
void batch_forget(pic_sim* s);
