// Autotuner of the particle tile and the push work-item size (pic_autotune).
//
// The push kernel stages one tile's field box in shared memory per work item, so the tile
// sets the box's halo overhead, the shared memory per block (and with it the blocks per SM)
// and the particles that share a box; the work-item size sets the load balance across the
// SMs.  The best pair depends on the dimension, the precision, the particles per cell and
// the beam, so it is measured: every candidate is run for a few steps from the start of
// the run (cold plasma) and again with the pulse on the plasma, and the fastest on the mean
// of the two is kept (cached per shape for the process).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pic.h"
#include "sff_kernels.h"

namespace {

struct Choice {
    int tile[3];
    int chunk;
    double ms;
};

std::mutex g_mu;
std::map<std::string, Choice> g_cache;

std::string key_of(const pic_config* c)
{
    char b[256];
    snprintf(b, sizeof b, "%d|%d|%d,%d,%d|%d|%d|%d,%d,%d|%d,%d,%d|%d,%d,%d|%d|%d", c->dim, c->precision, c->n[0],
             c->n[1], c->n[2], c->ppc, c->beam, c->slab_lo[0], c->slab_lo[1], c->slab_lo[2], c->slab_hi[0],
             c->slab_hi[1], c->slab_hi[2], c->tile[0], c->tile[1], c->tile[2], c->chunk, c->sort_every);
    return b;
}

std::vector<std::vector<int>> tile_candidates(int dim)
{
    if (dim == 1) return {{32, 1, 1}, {64, 1, 1}, {128, 1, 1}, {16, 1, 1}};
    // tiles 32 cells wide put a warp's 32 lanes (consecutive cells) on one row of the box
    if (dim == 2) return {{16, 16, 1}, {32, 16, 1}, {16, 8, 1}, {32, 32, 1}, {8, 8, 1}, {64, 8, 1}, {64, 16, 1}};
    return {{8, 8, 8}, {16, 8, 8}, {8, 8, 4}, {16, 8, 4}, {8, 4, 4}, {32, 4, 4}, {32, 4, 2}, {32, 8, 2}};
}

// time per step of one candidate, or a negative pic_status
double trial(const pic_config& c, int steps, cudaStream_t st, pic_status* err)
{
    pic_sim* s = nullptr;
    pic_status r = pic_init(&c, nullptr, st, &s);
    if (r != PIC_OK) {
        *err = r;
        return -1.0;
    }
    pic_params p;
    pic_derive_params(&c, &p);
    // two stretches: from t = 0 (cold plasma, pulse not yet on it), then with the clock
    // moved to the time the pulse is on the plasma, so that the incident field and the
    // deposit do their full work
    double t_on = -1.0;
    if (c.beam == PIC_BEAM_LP || c.beam == PIC_BEAM_RP || c.beam == PIC_BEAM_GAUSS2D) {
        t_on = c.t_focus;
    } else if (c.beam == PIC_BEAM_PLANE && c.ppc > 0) {
        // envelope centre (Gaussian: xi = t_focus; sin^2: xi = duration) at the slab centre
        const double xc = 0.5 * (c.slab_lo[0] + c.slab_hi[0]) * c.dx;
        t_on = xc - c.focus[0] + (c.envelope == PIC_ENV_GAUSS ? c.t_focus : c.duration);
    }
    // per stretch: untimed steps, then the faster of two timed runs (the GPU is shared: a
    // run can be slowed by something else)
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool ev = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    auto stretch = [&]() {
        double best = -1.0;
        if (!ev || pic_step(s, steps, st) != PIC_OK) return -1.0;
        for (int rep = 0; rep < 2; ++rep) {
            float t = 0.f;
            if (cudaEventRecord(e0, st) == cudaSuccess && pic_step(s, steps, st) == PIC_OK &&
                cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && t > 0.f) {
                const double m = t / steps;
                best = best < 0 ? m : std::min(best, m);
            } else {
                return -1.0;
            }
        }
        return best;
    };
    double ms = stretch();
    if (ms > 0 && t_on > 0 && p.dt > 0) {
        // the second stretch centred on the pulse's arrival: reached by stepping (electrons
        // heated by the pulse: the deposit's windows and the incident field as in the run)
        // when that takes at most 1500 steps, else by moving the clock
        const long long k = std::max<long long>(3 * steps, std::llround(t_on / p.dt) - steps);
        const long long done = 3LL * steps;
        pic_status adv = PIC_OK;
        if (k - done <= 1500) adv = k > done ? pic_step(s, (int)(k - done), st) : PIC_OK;
        else adv = pic_set_step(s, k, st);
        const double ms_on = adv == PIC_OK ? stretch() : -1.0;
        ms = ms_on > 0 ? 0.5 * (ms + ms_on) : -1.0;
    }
    pic_info inf;
    if (ms > 0 && pic_info_get(s, &inf, st) == PIC_OK && (inf.status & PIC_FLAG_TIMEOUT)) ms = -1.0;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    pic_destroy(s);
    *err = ms > 0 ? PIC_OK : PIC_ECUDA;
    return ms;
}

}  // namespace

extern "C" pic_status pic_autotune(pic_config* cfg, int trial_steps, void* stream, double* ms_per_step)
{
    if (!cfg || trial_steps < 1) return PIC_EINVAL;
    pic_params p;
    pic_status r = pic_derive_params(cfg, &p);
    if (r != PIC_OK) return r;
    const bool tune_tile = cfg->tile[0] == 0 && (cfg->dim < 2 || cfg->tile[1] == 0) && (cfg->dim < 3 || cfg->tile[2] == 0);
    const bool tune_chunk = cfg->chunk == 0;
    if (!tune_tile && !tune_chunk) {
        if (ms_per_step) *ms_per_step = 0.0;
        return PIC_OK;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PIC_ENODEV;
    const std::string key = std::to_string(dev) + "#" + key_of(cfg);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            for (int d = 0; d < 3; ++d) cfg->tile[d] = it->second.tile[d];
            cfg->chunk = it->second.chunk;
            if (ms_per_step) *ms_per_step = it->second.ms;
            return PIC_OK;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    pic_config c = *cfg;
    c.autotune_steps = 0;
    // the work-item size the tile search runs at: 4096 for a run with at least 16 such work
    // items per SM (its per-item overhead matters most there; at the focus of the 3D
    // workload 4096 beats 2048 by ~2 %, about the trial's noise, so the larger size is the
    // one a smaller size has to beat), 2048 otherwise
    const int base_chunk = p.n_particles >= 4096LL * 16 * sff::device_sms() ? 4096 : 2048;
    Choice best{{cfg->tile[0], cfg->tile[1], cfg->tile[2]}, cfg->chunk, -1.0};
    pic_status first_err = PIC_OK;
    auto consider = [&](const pic_config& cand) {
        pic_status e = PIC_OK;
        const double ms = trial(cand, trial_steps, st, &e);
        // a later candidate must win by more than 1 %, the trials' noise on a shared GPU, so
        // that the order of the candidate lists (the more robust choices first) breaks ties
        if (ms > 0 && (best.ms < 0 || ms < 0.99 * best.ms)) {
            best.ms = ms;
            for (int d = 0; d < 3; ++d) best.tile[d] = cand.tile[d];
            best.chunk = cand.chunk;
        } else if (ms <= 0 && first_err == PIC_OK) {
            first_err = e;
        }
        cudaGetLastError();      // a candidate that failed leaves no sticky error behind
    };
    // tiles first (work items at the default size), then work-item sizes at the best tile
    if (tune_tile) {
        const auto cands = tile_candidates(cfg->dim);
        for (size_t k = 0; k < cands.size(); ++k) {
            const auto& t = cands[k];
            // besides the default (first) tile, a tile should hold at least one default work
            // item of particles (2048): smaller tiles multiply the field-box loads and the
            // scatter's destinations per particle, a cost a short trial at the focus under-weighs
            long long vol = 1;
            for (int d = 0; d < cfg->dim; ++d) vol *= t[d];
            // (unless the particles are too few to give every SM several work items anyway)
            if (k > 0 && cfg->ppc > 0 && vol * cfg->ppc < 2048 && p.n_particles / 2048 > 4LL * sff::device_sms()) continue;
            pic_config cand = c;
            for (int d = 0; d < 3; ++d) cand.tile[d] = d < cfg->dim ? t[d] : 0;
            if (tune_chunk) cand.chunk = base_chunk;
            consider(cand);
        }
    } else {
        consider(c);
    }
    if (best.ms < 0) return first_err != PIC_OK ? first_err : PIC_ECUDA;
    if (tune_chunk) {
        best.chunk = base_chunk;      // the measurements above ran at this size
        // small work items spread a small run over more SMs; large ones cut the per-item
        // overhead of a large run
        for (int ch : {256, 512, 1024, 2048, 4096}) {
            if (ch == base_chunk) continue;
            pic_config cand = c;
            for (int d = 0; d < 3; ++d) cand.tile[d] = best.tile[d];
            cand.chunk = ch;
            consider(cand);
        }
    }
    for (int d = 0; d < 3; ++d) cfg->tile[d] = best.tile[d];
    cfg->chunk = best.chunk;
    if (ms_per_step) *ms_per_step = best.ms;
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[key] = best;
    return PIC_OK;
}
