// Batched stepping of independent simulations (pic_batch_step): simulations of the
// same dimension and precision form one launch group; each phase of the step (push +
// deposit + placement, tile scan, field solve, step end; the cell count, cell scan and
// scatter on cell-sort steps) is ONE launch over the
// (simulation, tile) work items of the whole group, pulled from a device counter.  The
// step of all groups is captured once as a CUDA graph (and once more with the cell sort),
// cached per exact list of sims.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "sim_internal.h"

namespace {

struct GroupRes {
    Group g{};
    void* mem = nullptr;
    // the group tables come from the first member's device-memory provider (pic_allocator, or
    // cudaMalloc when it gave none) and go back to it; an entry is dropped (batch_forget) when
    // any member is destroyed, before that member releases anything
    pic_allocator al{};
    bool cuda = true;
};

struct BatchEntry {
    long long id = new_group_id();        // launch-group id of all groups of this list
    std::vector<pic_sim*> sims;
    std::vector<GroupRes> groups;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t sort_graph = nullptr;     // the step whose re-sort orders the tiles by cell
    cudaGraphExec_t sort_exec = nullptr;
    int sort_every = 0;                   // smallest positive sort_every of the members (0: none)
    int since_sort = 0;
    cudaStream_t cs = nullptr;
    cudaStream_t cs2 = nullptr;           // the field-solve branch
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

std::mutex g_mu;
std::map<std::vector<pic_sim*>, BatchEntry*> g_batches;

void free_entry(BatchEntry* e)
{
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    if (e->sort_exec) cudaGraphExecDestroy(e->sort_exec);
    if (e->sort_graph) cudaGraphDestroy(e->sort_graph);
    if (e->cs) cudaStreamDestroy(e->cs);
    if (e->cs2) cudaStreamDestroy(e->cs2);
    if (e->ev_fork) cudaEventDestroy(e->ev_fork);
    if (e->ev_join) cudaEventDestroy(e->ev_join);
    for (auto& gr : e->groups) {
        if (!gr.mem) continue;
        if (gr.cuda) cudaFree(gr.mem);
        else gr.al.free(gr.mem, gr.al.ctx);
    }
    delete e;
}

size_t a256(size_t b) { return (b + 255) & ~size_t(255); }

pic_status build_entry(const std::vector<pic_sim*>& sims, BatchEntry** out, std::string& err)
{
    std::map<std::pair<int, int>, std::vector<int>> by;
    for (int i = 0; i < (int)sims.size(); ++i) by[{sims[i]->cfg.dim, sims[i]->cfg.precision}].push_back(i);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    BatchEntry* e = new BatchEntry();
    e->sims = sims;
    for (auto& kv : by) {
        const std::vector<int>& mem = kv.second;
        const int n = (int)mem.size();
        long long nyw = 0, nch = 0;
        size_t psm = 0, ysm = 0;
        for (int i : mem) {
            nyw += sims[i]->nywork;
            nch += sims[i]->h.max_chunks;
            psm = std::max(psm, sims[i]->grp.push_smem);
            ysm = std::max(ysm, sims[i]->grp.yee_smem);
        }
        const size_t bytes = a256(sizeof(SimDev) * n) + a256(sizeof(Work) * nyw) + a256(sizeof(int) * (n + 1)) + a256(64);
        GroupRes gr;
        const pic_sim* owner = sims[mem[0]];
        gr.cuda = owner->use_cuda_malloc;
        gr.al = owner->alloc;
        if (gr.cuda) {
            if (cudaMalloc(&gr.mem, bytes) != cudaSuccess) gr.mem = nullptr;
        } else {
            gr.mem = gr.al.alloc(bytes, gr.al.ctx);
        }
        if (!gr.mem) {
            err = "batch descriptor allocation failed";
            free_entry(e);
            return PIC_ENOMEM;
        }
        char* p = (char*)gr.mem;
        SimDev* d_sims = (SimDev*)p;
        p += a256(sizeof(SimDev) * n);
        Work* d_yw = (Work*)p;
        p += a256(sizeof(Work) * nyw);
        int* d_gp = (int*)p;
        p += a256(sizeof(int) * (n + 1));
        int* d_cnt = (int*)p;
        std::vector<SimDev> hs(n);
        std::vector<Work> yw;
        yw.reserve(nyw);
        for (int k = 0; k < n; ++k) {
            pic_sim* s = sims[mem[k]];
            hs[k] = s->h;
            for (int t = 0; t < s->h.nytiles; ++t)
                if (yee_tile_active(s->h, s->cfg.dim, t)) yw.push_back({k, t});
        }
        cudaMemcpy(d_sims, hs.data(), sizeof(SimDev) * n, cudaMemcpyHostToDevice);
        cudaMemcpy(d_yw, yw.data(), sizeof(Work) * nyw, cudaMemcpyHostToDevice);
        cudaMemset(d_gp, 0, sizeof(int) * (n + 1));
        cudaMemset(d_cnt, 0, 64);
        Group& g = gr.g;
        g.sims = d_sims;
        g.one = nullptr;
        g.nsims = n;
        g.gprefix = d_gp;
        g.ywork = d_yw;
        g.nywork = (int)nyw;
        g.counters = d_cnt;
        g.dim = kv.first.first;
        g.prec = kv.first.second;
        g.push_smem = psm;
        g.yee_smem = ysm;
        g.inc_any = 0;
        g.scan_blocks = n == 1 ? sims[mem[0]]->h.nscanblk : 0;
        int maxtiles = 1;
        for (int i : mem) {
            maxtiles = std::max(maxtiles, sims[i]->h.nptiles);
            const int k = sims[i]->sort_every;
            if (k > 0 && (e->sort_every == 0 || k < e->sort_every)) e->sort_every = k;
        }
        g.inc_segs = g.inc_rows = 1;
        for (int i : mem) {
            const pic_config& c = sims[i]->cfg;
            g.inc_any |= sims[i]->h.incgrid;
            g.inc_segs = std::max(g.inc_segs, (c.n[0] + 1 + 255) / 256);
            g.inc_rows = std::max(g.inc_rows, (c.dim > 1 ? c.n[1] + 1 : 1) * (c.dim > 2 ? c.n[2] + 1 : 1));
        }
        const int nsm = prop.multiProcessorCount;
        const int bp = std::max(1, sff::prepare_push(g.dim, g.prec, psm));
        const int byy = std::max(1, sff::prepare_yee(g.dim, g.prec, ysm));
        const int bs = std::max(1, sff::scatter_blocks_per_sm(g.dim, g.prec));
        g.push_grid = (int)std::max<long long>(1, std::min<long long>(nch, (long long)bp * nsm));
        g.yee_grid = (int)std::max<long long>(1, std::min<long long>(nyw, (long long)byy * nsm));
        g.scatter_grid = (int)std::max<long long>(1, std::min<long long>(nch, (long long)bs * nsm));
        g.cellscan_grid = std::max(1, std::min(maxtiles, 8 * nsm));
        e->groups.push_back(gr);
    }
    if (cudaStreamCreateWithFlags(&e->cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&e->cs2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        err = "batch capture could not start";
        free_entry(e);
        return PIC_ECUDA;
    }
    // the plain step, and (when a member sorts by cell) the cell-sort step
    for (int v = 0; v < (e->sort_every > 0 ? 2 : 1); ++v) {
        if (cudaStreamBeginCapture(e->cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            err = "batch capture could not start";
            free_entry(e);
            return PIC_ECUDA;
        }
        // per group: push, then the tile scan (and cell sort) and the field solve
        // concurrently, then the step end
        cudaError_t ce = cudaSuccess;
        for (auto& gr : e->groups) {
            sff::launch_incident_grid(gr.g, e->cs);
            sff::launch_push(gr.g, v == 1, e->cs);
            if (ce == cudaSuccess) ce = cudaEventRecord(e->ev_fork, e->cs);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(e->cs2, e->ev_fork, 0);
            if (ce == cudaSuccess) {
                sff::launch_yee(gr.g, e->cs2);
                ce = cudaEventRecord(e->ev_join, e->cs2);
            }
            sff::launch_scan(gr.g, e->cs);
            if (v == 1) sff::launch_cell_sort(gr.g, e->cs);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(e->cs, e->ev_join, 0);
            sff::launch_step_end(gr.g, e->cs);
        }
        cudaGraph_t* gp = v == 1 ? &e->sort_graph : &e->graph;
        cudaGraphExec_t* xp = v == 1 ? &e->sort_exec : &e->exec;
        const cudaError_t ec = cudaStreamEndCapture(e->cs, gp);
        if (ce == cudaSuccess) ce = ec;
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(xp, *gp, 0);
        if (ce != cudaSuccess) {
            err = std::string("batch graph: ") + cudaGetErrorString(ce);
            free_entry(e);
            return PIC_ECUDA;
        }
    }
    *out = e;
    return PIC_OK;
}

}  // namespace

void batch_forget(pic_sim* s)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_batches.begin(); it != g_batches.end();) {
        if (std::find(it->first.begin(), it->first.end(), s) != it->first.end()) {
            free_entry(it->second);
            it = g_batches.erase(it);
        } else {
            ++it;
        }
    }
}

namespace {
// The cached entry of this exact list of simulations (built on first use); PIC_EINVAL for a
// bad list.
pic_status entry_of(pic_sim** sims, int n_sims, std::vector<pic_sim*>& key, BatchEntry** out)
{
    if (!sims || n_sims <= 0) return PIC_EINVAL;
    key.assign(sims, sims + n_sims);
    for (pic_sim* s : key)
        if (!s) return PIC_EINVAL;
    {
        std::vector<pic_sim*> u = key;
        std::sort(u.begin(), u.end());
        if (std::adjacent_find(u.begin(), u.end()) != u.end()) {
            key[0]->err = "a simulation appears twice in the batch";
            return PIC_EINVAL;
        }
    }
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_batches.find(key);
    if (it != g_batches.end()) {
        *out = it->second;
        return PIC_OK;
    }
    std::string err;
    BatchEntry* e = nullptr;
    pic_status r = build_entry(key, &e, err);
    if (r != PIC_OK) {
        key[0]->err = err;
        return r;
    }
    g_batches[key] = e;
    *out = e;
    return PIC_OK;
}

// before the first step of this list after anything else changed a member's layout: number
// the work items of its launch groups
void ensure_prefix(BatchEntry* e, const std::vector<pic_sim*>& key, cudaStream_t st)
{
    bool fresh = true;
    for (pic_sim* s : key) fresh = fresh && s->prefix_group == e->id;
    if (!fresh) {
        for (auto& gr : e->groups) sff::launch_prefix(gr.g, st);
        for (pic_sim* s : key) s->prefix_group = e->id;
    }
}
}  // namespace

extern "C" pic_status pic_batch_profile_step(pic_sim** sims, int n_sims, int n_steps, void* stream, double* seconds)
{
    if (!seconds || n_steps < 0) return PIC_EINVAL;
    std::vector<pic_sim*> key;
    BatchEntry* e = nullptr;
    pic_status r = entry_of(sims, n_sims, key, &e);
    if (r != PIC_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < 5; ++i) seconds[i] = 0.0;
    cudaEvent_t ev[6];
    for (int i = 0; i < 6; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) {
            for (int k = 0; k < i; ++k) cudaEventDestroy(ev[k]);
            key[0]->err = "batch profile: event creation failed";
            return PIC_ECUDA;
        }
    if (n_steps > 0) ensure_prefix(e, key, st);
    for (int k = 0; k < n_steps && r == PIC_OK; ++k) {
        bool sort = false;
        if (e->sort_every > 0 && ++e->since_sort >= e->sort_every) {
            e->since_sort = 0;
            sort = true;
        }
        // the phases of every launch group one after another, the same launches as the graph
        cudaEventRecord(ev[0], st);
        for (auto& gr : e->groups) {
            sff::launch_incident_grid(gr.g, st);
            sff::launch_push(gr.g, sort, st);
        }
        cudaEventRecord(ev[1], st);
        for (auto& gr : e->groups) sff::launch_scan(gr.g, st);
        cudaEventRecord(ev[2], st);
        if (sort)
            for (auto& gr : e->groups) sff::launch_cell_sort(gr.g, st);
        cudaEventRecord(ev[3], st);
        for (auto& gr : e->groups) sff::launch_yee(gr.g, st);
        cudaEventRecord(ev[4], st);
        for (auto& gr : e->groups) sff::launch_step_end(gr.g, st);
        cudaEventRecord(ev[5], st);
        const cudaError_t ce = cudaEventSynchronize(ev[5]);
        if (ce != cudaSuccess) {
            key[0]->err = std::string("batch profiled step: ") + cudaGetErrorString(ce);
            r = PIC_ECUDA;
            break;
        }
        for (int i = 0; i < 5; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
            seconds[i] += 1e-3 * ms;
        }
    }
    for (int i = 0; i < 6; ++i) cudaEventDestroy(ev[i]);
    return r;
}

extern "C" pic_status pic_batch_step(pic_sim** sims, int n_sims, int n_steps, void* stream)
{
    if (!sims || n_sims <= 0 || n_steps < 0) return PIC_EINVAL;
    std::vector<pic_sim*> key;
    BatchEntry* e = nullptr;
    pic_status r = entry_of(sims, n_sims, key, &e);
    if (r != PIC_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    // the graph starts at the push: the chunks are numbered by the previous step's end when
    // that step was this list's, else here
    if (n_steps > 0) ensure_prefix(e, key, st);
    for (int i = 0; i < n_steps; ++i) {
        bool sort = false;
        if (e->sort_every > 0 && ++e->since_sort >= e->sort_every) {
            e->since_sort = 0;
            sort = true;
        }
        cudaError_t ce = cudaGraphLaunch(sort ? e->sort_exec : e->exec, st);
        if (ce != cudaSuccess) {
            key[0]->err = std::string("batch graph launch: ") + cudaGetErrorString(ce);
            return PIC_ECUDA;
        }
    }
    return PIC_OK;
}
