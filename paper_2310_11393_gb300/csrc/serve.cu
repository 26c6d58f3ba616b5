// Continuous-batching request server (pic_serve_*): parameter-scan simulations arrive
// at any time; a host scheduling thread admits queued requests whenever a resident
// slot and device memory (estimated with pic_derive_params) are free, and each quantum
// advances a batch of resident simulations together through the batched step, or a batch
// of one through its own step graph (each simulation stops exactly at its requested step
// count).  The batch is chosen shortest
// remaining work first (steps left x electrons) until it holds fill_particles electrons,
// enough to fill the GPU: short requests finish early instead of sharing the device with
// every long one to the end, and the device stays full.  Finished simulations retire
// with their energies; submit / start / finish times are on one clock.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "sim_internal.h"

namespace {

struct Request {
    uint64_t ticket;
    pic_config cfg;
    int64_t n_steps;
    int64_t bytes;
};

struct Resident {
    uint64_t ticket;
    pic_sim* sim;
    int64_t remaining;
    int64_t bytes;
};

}  // namespace

struct pic_server {
    pic_serve_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> queue;
    std::map<uint64_t, pic_result> results;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    std::chrono::steady_clock::time_point t0;
    int64_t budget = 0;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    void run();
};

void pic_server::run()
{
    cudaSetDevice(device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    std::vector<Resident> res;
    int64_t used = 0;
    const int max_res = cfg.max_resident > 0 ? cfg.max_resident : 256;
    const int quantum = cfg.quantum > 0 ? cfg.quantum : 50;
    const int64_t fill = cfg.fill_particles > 0 ? cfg.fill_particles : (cfg.fill_particles < 0 ? -1 : 2000000);
    for (;;) {
        // ---- admission (FIFO while memory and slots allow) ----
        std::vector<Request> admit;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (res.empty() && queue.empty() && !stop)
                cv.wait_for(lk, std::chrono::milliseconds(50), [&] { return stop || !queue.empty(); });
            if (stop && queue.empty() && res.empty()) break;
            int64_t room = budget - used;
            while (!queue.empty() && (int)(res.size() + admit.size()) < max_res && queue.front().bytes <= room) {
                room -= queue.front().bytes;
                admit.push_back(queue.front());
                queue.pop_front();
            }
            // a request larger than the whole budget can never run
            while (!queue.empty() && queue.front().bytes > budget) {
                pic_result& r = results[queue.front().ticket];
                r.state = -1;
                r.error = PIC_ECAPACITY;
                r.finish_time = now();
                queue.pop_front();
            }
        }
        for (const Request& q : admit) {
            pic_sim* s = nullptr;
            const double ts = now();
            pic_status e = pic_init(&q.cfg, nullptr, st, &s);
            std::lock_guard<std::mutex> lk(mu);
            pic_result& r = results[q.ticket];
            if (e != PIC_OK) {
                r.state = -1;
                r.error = e;
                r.finish_time = now();
                continue;
            }
            r.state = 1;
            r.start_time = ts;
            res.push_back({q.ticket, s, q.n_steps, q.bytes});
            used += q.bytes;
        }
        if (res.empty()) continue;
        // ---- the batch of this quantum: least remaining work first, until full ----
        std::vector<int64_t> alive(res.size());
        for (size_t i = 0; i < res.size(); ++i) {
            pic_info inf;
            alive[i] = pic_info_get(res[i].sim, &inf, st) == PIC_OK ? inf.n_alive : 0;
        }
        std::vector<size_t> order(res.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
            return res[a].remaining * std::max<int64_t>(alive[a], 1) < res[b].remaining * std::max<int64_t>(alive[b], 1);
        });
        std::vector<char> chosen(res.size(), 0);
        int64_t in_batch = 0;
        for (size_t k = 0; k < order.size(); ++k) {
            if (fill >= 0 && k > 0 && in_batch >= fill) break;
            chosen[order[k]] = 1;
            in_batch += alive[order[k]];
        }
        int64_t q = quantum;
        std::vector<pic_sim*> list;
        for (size_t i = 0; i < res.size(); ++i)
            if (chosen[i]) {
                q = std::min(q, res[i].remaining);
                list.push_back(res[i].sim);
            }
        // one member: its own step graph (the single-simulation kernels); several: one batched
        // launch per phase over all of them
        pic_status e = PIC_OK;
        if (q > 0) e = list.size() == 1 ? pic_step(list[0], (int)q, st) : pic_batch_step(list.data(), (int)list.size(), (int)q, st);
        cudaStreamSynchronize(st);
        // ---- bookkeeping and retirement ----
        std::vector<Resident> keep;
        for (size_t i = 0; i < res.size(); ++i) {
            Resident r = res[i];
            if (!chosen[i]) {
                keep.push_back(r);
                continue;
            }
            r.remaining -= q;
            {
                std::lock_guard<std::mutex> lk(mu);
                pic_result& out = results[r.ticket];
                out.steps_done += q;
                out.pushes += alive[i] * q;
            }
            if (e != PIC_OK || r.remaining <= 0) {
                double en[8] = {0};
                pic_status de = e != PIC_OK ? e : pic_diag(r.sim, PIC_DIAG_ENERGIES, en, sizeof en, st);
                pic_destroy(r.sim);
                used -= r.bytes;
                std::lock_guard<std::mutex> lk(mu);
                pic_result& out = results[r.ticket];
                out.state = de == PIC_OK ? 2 : -1;
                out.error = de;
                for (int k = 0; k < 8; ++k) out.energies[k] = en[k];
                out.finish_time = now();
            } else {
                keep.push_back(r);
            }
        }
        res.swap(keep);
    }
    cudaStreamDestroy(st);
}

extern "C" {

pic_status pic_serve_open(const pic_serve_config* cfg, pic_server** out)
{
    if (!out) return PIC_EINVAL;
    *out = nullptr;
    pic_server* s = new pic_server();
    if (cfg) s->cfg = *cfg;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return PIC_ENODEV;
    }
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        delete s;
        return PIC_ENODEV;
    }
    s->budget = s->cfg.memory_budget > 0 ? s->cfg.memory_budget : (int64_t)(0.8 * (double)fr);
    s->t0 = std::chrono::steady_clock::now();
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return PIC_OK;
}

pic_status pic_serve_submit(pic_server* s, const pic_config* cfg, int64_t n_steps, uint64_t* ticket)
{
    if (!s || !cfg || !ticket || n_steps < 0) return PIC_EINVAL;
    pic_params p;
    pic_status r = pic_derive_params(cfg, &p);
    if (r != PIC_OK) return r;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return PIC_EINVAL;
    const uint64_t t = s->next_ticket++;
    s->queue.push_back({t, *cfg, n_steps, p.device_bytes});
    pic_result res{};
    res.state = 0;
    res.submit_time = s->now();
    s->results[t] = res;
    *ticket = t;
    s->cv.notify_all();
    return PIC_OK;
}

pic_status pic_serve_poll(pic_server* s, uint64_t ticket, pic_result* out)
{
    if (!s || !out) return PIC_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return PIC_ENOTFOUND;
    *out = it->second;
    if (it->second.state == 0 || it->second.state == 1) return PIC_EBUSY;
    return it->second.state == 2 ? PIC_OK : (pic_status)it->second.error;
}

double pic_serve_clock(const pic_server* s) { return s ? s->now() : 0.0; }

pic_status pic_serve_close(pic_server* s)
{
    if (!s) return PIC_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    delete s;
    return PIC_OK;
}

}  // extern "C"
