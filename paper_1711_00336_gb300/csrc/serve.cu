// serve.cu -- continuous batching of settling-suspension runs on one GPU.
//
// A worker thread owns one batch (include/dps.h batch API) per subcycle class
// (n_int, n_DEM): a batch advances all its boxes with one launch per phase,
// and the boxes of a batch must share the subcycle counts.  Between chunks of
// steps the worker admits queued requests, first come first served, into the
// batch of their class while a slot is free and the device has room
// (cudaMemGetInfo against dps_box_bytes plus a reserve), so a request arriving
// while others run joins the next chunk; the class batches step concurrently
// (each on its own stream); the worker samples each box's mean particle
// velocity once per chunk and retires boxes whose windowed mean velocity
// converged (or hit the step cap), freeing their memory for the queue.  Each
// box sees exactly the same step sequence as it would alone, so its result
// does not depend on the mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "dps.h"

namespace {

struct Req {
    int64_t id = 0;
    dps_request r{};
    std::vector<double> x, d, rho;
    dps_result res{};
    dps_batch b = nullptr;  // the batch of its subcycle class
    int box = -1;
    bool cancel = false;
    double win_sum[3] = {0, 0, 0};
    int win_n = 0;
    double prev[3] = {0, 0, 0};
    bool have_prev = false;
    double ghat[3] = {0, 0, -1};
};

using clk = std::chrono::steady_clock;

}  // namespace

struct dps_server_s {
    dps_serve_desc desc{};
    std::map<std::pair<int, int>, dps_batch> batches;  // (n_int, n_DEM) -> batch
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req *> queue;
    std::map<int64_t, Req *> all;
    std::vector<Req *> running;
    bool stop = false;
    int admitting = 0;  // requests taken from the queue, not yet in `running`
    int64_t next_id = 1;
    clk::time_point t0;
    dps_serve_stats st{};
    double busy_since = -1;

    double now() const { return std::chrono::duration<double>(clk::now() - t0).count(); }

    void finish(Req *q, int state, int status) {
        // final observables of the box, then release it
        if (state == DPS_REQ_DONE) {
            dps_stats s;
            if (dps_batch_stats(q->b, q->box, &s) == DPS_OK)
                for (int a = 0; a < 3; ++a) q->res.u_pS[a] = s.u_pS[a];
        }
        dps_batch_remove_box(q->b, q->box);
        std::lock_guard<std::mutex> lk(mu);
        q->res.state = state;
        q->res.status = status;
        q->res.t_end = now();
        if (state == DPS_REQ_DONE) st.completed++;
        if (state == DPS_REQ_FAILED) st.failed++;
        st.running--;
    }

    // admit queued requests (worker thread, lock held by the caller)
    void admit(std::unique_lock<std::mutex> &lk) {
        while (!queue.empty() && (int)running.size() < desc.max_boxes) {
            Req *q = queue.front();
            if (q->cancel) {
                queue.pop_front();
                q->res.state = DPS_REQ_CANCELLED;
                st.queued--;
                continue;
            }
            size_t need = 0, fre = 0, tot = 0;
            dps_box_bytes(desc.precision, q->r.n, q->r.np, &need);
            cudaMemGetInfo(&fre, &tot);
            if (fre < need + desc.hbm_reserve_bytes) {
                if (running.empty()) {  // would never fit: fail it
                    queue.pop_front();
                    st.queued--;
                    q->res.state = DPS_REQ_FAILED;
                    q->res.status = DPS_ERR_OOM;
                    st.failed++;
                    continue;
                }
                break;  // wait for running boxes to retire
            }
            queue.pop_front();
            st.queued--;
            admitting++;
            lk.unlock();
            int box = -1, rc = DPS_OK;
            // the batch of the request's subcycle class (created on first use)
            const std::pair<int, int> cls(q->r.closure.n_int, q->r.closure.n_dem);
            auto it = batches.find(cls);
            if (it == batches.end()) {
                dps_batch_desc bd{};
                bd.precision = desc.precision;
                dps_batch nb = nullptr;
                rc = dps_batch_create(&bd, &nb);
                if (rc == DPS_OK) it = batches.emplace(cls, nb).first;
            }
            if (rc == DPS_OK) {
                q->b = it->second;
                rc = dps_batch_add_box(q->b, q->r.n, q->r.periodic, q->r.tau, q->r.rho_f, q->r.np, &box);
            }
            if (rc == DPS_OK && q->r.np)
                rc = dps_batch_add_particles(q->b, box, q->r.np, q->x.data(), nullptr, nullptr, q->d.data(),
                                             q->rho.data());
            if (rc == DPS_OK) rc = dps_batch_set_closure(q->b, box, &q->r.closure);
            lk.lock();
            admitting--;
            if (rc != DPS_OK) {
                if (box >= 0) {
                    lk.unlock();
                    dps_batch_remove_box(q->b, box);
                    lk.lock();
                }
                q->res.state = DPS_REQ_FAILED;
                q->res.status = rc;
                st.failed++;
                continue;
            }
            q->box = box;
            q->res.state = DPS_REQ_RUNNING;
            q->res.t_start = now();
            running.push_back(q);
            st.admitted++;
            st.running++;
            if ((int)running.size() > st.peak_boxes) st.peak_boxes = (int)running.size();
        }
    }

    void loop() {
        cudaSetDevice(desc.device);
        const int64_t chunk = desc.chunk_steps;
        while (true) {
            std::unique_lock<std::mutex> lk(mu);
            admit(lk);
            if (running.empty()) {
                if (busy_since >= 0) {
                    st.busy_s += now() - busy_since;
                    busy_since = -1;
                }
                if (stop) return;
                cv.notify_all();  // idle: wake dps_serve_wait_idle
                cv.wait(lk, [&] { return stop || !queue.empty(); });
                continue;
            }
            if (busy_since < 0) busy_since = now();
            // cancelled running requests leave before the next chunk
            std::vector<Req *> cancelled;
            for (Req *q : running)
                if (q->cancel) cancelled.push_back(q);
            lk.unlock();
            for (Req *q : cancelled) {
                finish(q, DPS_REQ_CANCELLED, DPS_OK);
                std::lock_guard<std::mutex> g(mu);
                running.erase(std::find(running.begin(), running.end(), q));
            }
            if (running.empty()) continue;
            // every class batch with running boxes advances one chunk; the
            // batches run on their own streams, so their work overlaps
            std::vector<dps_batch> active;
            for (Req *q : running)
                if (std::find(active.begin(), active.end(), q->b) == active.end()) active.push_back(q->b);
            std::vector<int> brc(active.size(), DPS_OK);
            for (size_t k = 0; k < active.size(); ++k) brc[k] = dps_batch_step_async(active[k], chunk);
            for (size_t k = 0; k < active.size(); ++k)
                if (brc[k] == DPS_OK) brc[k] = dps_batch_check(active[k]);
            std::vector<std::pair<Req *, int>> done;  // request, state
            std::vector<dps_batch> failed_all;        // batches whose every box failed
            double cells = 0;
            for (size_t k = 0; k < active.size(); ++k) {
                if (brc[k] == DPS_OK) {
                    for (Req *q : running)
                        if (q->b == active[k]) cells += (double)q->r.n[0] * q->r.n[1] * q->r.n[2];
                    continue;
                }
                // boxes are independent: retire those whose status word flags
                // the failure; if none does (a CUDA error), all boxes of the batch
                int flagged = 0;
                for (Req *q : running) {
                    dps_stats bs;
                    if (q->b == active[k] && brc[k] == DPS_ERR_UNSTABLE &&
                        dps_batch_stats(q->b, q->box, &bs) == DPS_OK && bs.status) {
                        done.push_back({q, DPS_REQ_FAILED});
                        flagged++;
                    }
                }
                if (!flagged) {
                    failed_all.push_back(active[k]);
                    for (Req *q : running)
                        if (q->b == active[k]) done.push_back({q, DPS_REQ_FAILED});
                }
            }
            {
                std::lock_guard<std::mutex> g(mu);
                st.cell_updates += cells * chunk;
            }
            // the error code of a box's batch (a flagged box of a batch that
            // returned DPS_OK cannot occur)
            auto batch_rc = [&](const Req *q) {
                for (size_t k = 0; k < active.size(); ++k)
                    if (active[k] == q->b) return brc[k];
                return (int)DPS_OK;
            };
            {
                for (Req *q : running) {
                    if (std::find(failed_all.begin(), failed_all.end(), q->b) != failed_all.end()) continue;
                    if (std::find_if(done.begin(), done.end(), [&](const std::pair<Req *, int> &p) {
                            return p.first == q;
                        }) != done.end())
                        continue;
                    q->res.steps += chunk;
                    double u[3];
                    dps_batch_particle_mean(q->b, q->box, u);
                    for (int a = 0; a < 3; ++a) q->win_sum[a] += u[a];
                    q->win_n++;
                    if (q->res.steps % q->r.window == 0) {
                        double wm[3], dotn = 0, dotp = 0;
                        for (int a = 0; a < 3; ++a) {
                            wm[a] = q->win_sum[a] / q->win_n;
                            dotn += wm[a] * q->ghat[a];
                            dotp += q->prev[a] * q->ghat[a];
                            q->win_sum[a] = 0;
                        }
                        q->win_n = 0;
                        bool conv = q->have_prev && std::fabs(dotn - dotp) < q->r.rel_tol * std::fabs(dotp);
                        for (int a = 0; a < 3; ++a) {
                            q->prev[a] = wm[a];
                            q->res.up_mean[a] = wm[a];
                        }
                        q->have_prev = true;
                        if (conv) done.push_back({q, DPS_REQ_DONE});
                        else if (q->res.steps >= q->r.max_steps) {
                            q->res.capped = 1;
                            done.push_back({q, DPS_REQ_DONE});
                        }
                    } else if (q->res.steps >= q->r.max_steps) {
                        q->res.capped = 1;
                        done.push_back({q, DPS_REQ_DONE});
                    }
                }
            }
            for (auto &p : done) {
                const int brq = batch_rc(p.first);
                finish(p.first, p.second, p.second == DPS_REQ_FAILED ? (brq ? brq : DPS_ERR_UNSTABLE) : DPS_OK);
                std::lock_guard<std::mutex> g(mu);
                running.erase(std::find(running.begin(), running.end(), p.first));
            }
            // a class batch left without boxes is released (its streams,
            // graphs and tile lists); the class's next request creates it anew
            for (auto it = batches.begin(); it != batches.end();) {
                bool used = false;
                for (Req *q : running) used = used || q->b == it->second;
                if (!used) {
                    dps_batch_destroy(it->second);
                    it = batches.erase(it);
                } else {
                    ++it;
                }
            }
            cv.notify_all();
        }
    }
};

extern "C" {

int dps_serve_create(const dps_serve_desc *desc, dps_server *out) {
    if (out) *out = nullptr;
    if (!desc || !out || desc->max_boxes < 1 || desc->chunk_steps < 1 || desc->precision < DPS_F64 ||
        desc->precision > DPS_F16S)
        return DPS_ERR_ARG;
    dps_server s = new dps_server_s();
    s->desc = *desc;
    if (cudaSetDevice(desc->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return DPS_ERR_CUDA;
    }
    s->t0 = clk::now();
    s->worker = std::thread([s] { s->loop(); });
    *out = s;
    return DPS_OK;
}

int dps_serve_submit(dps_server s, const dps_request *r, int64_t *id) {
    if (!s || !r || !id || r->np < 0 || (r->np > 0 && (!r->x3 || !r->d || !r->rho_p)) || r->window < 1 ||
        r->window % s->desc.chunk_steps != 0 || r->max_steps < 1 || !(r->rel_tol > 0))
        return DPS_ERR_ARG;
    Req *q = new Req();
    q->r = *r;
    q->x.assign(r->x3, r->x3 + 3 * r->np);
    q->d.assign(r->d, r->d + r->np);
    q->rho.assign(r->rho_p, r->rho_p + r->np);
    double gn = std::sqrt(r->closure.g[0] * r->closure.g[0] + r->closure.g[1] * r->closure.g[1] +
                          r->closure.g[2] * r->closure.g[2]);
    if (gn > 0)
        for (int a = 0; a < 3; ++a) q->ghat[a] = r->closure.g[a] / gn;
    q->r.x3 = q->x.data();
    q->r.d = q->d.data();
    q->r.rho_p = q->rho.data();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        q->id = s->next_id++;
        q->res.state = DPS_REQ_QUEUED;
        q->res.t_submit = s->now();
        s->all[q->id] = q;
        s->queue.push_back(q);
        s->st.submitted++;
        s->st.queued++;
        *id = q->id;
    }
    s->cv.notify_all();
    return DPS_OK;
}

int dps_serve_poll(dps_server s, int64_t id, dps_result *res) {
    if (!s || !res) return DPS_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return DPS_ERR_ARG;
    *res = it->second->res;
    return DPS_OK;
}

int dps_serve_cancel(dps_server s, int64_t id) {
    if (!s) return DPS_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return DPS_ERR_ARG;
    it->second->cancel = true;
    s->cv.notify_all();
    return DPS_OK;
}

int dps_serve_wait_idle(dps_server s, double timeout_s) {
    if (!s) return DPS_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto idle = [&] { return s->queue.empty() && s->running.empty() && s->admitting == 0; };
    if (timeout_s < 0) {
        s->cv.wait(lk, idle);
        return DPS_OK;
    }
    return s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), idle) ? DPS_OK : DPS_ERR_TIMEOUT;
}

int dps_serve_stats_get(dps_server s, dps_serve_stats *st) {
    if (!s || !st) return DPS_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *st = s->st;
    st->wall_s = s->now();
    if (s->busy_since >= 0) st->busy_s += s->now() - s->busy_since;
    return DPS_OK;
}

int dps_serve_destroy(dps_server s) {
    if (!s) return DPS_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Req *q : s->queue) q->cancel = true;
        s->queue.clear();
        for (Req *q : s->running) q->cancel = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &p : s->batches) dps_batch_destroy(p.second);
    for (auto &p : s->all) delete p.second;
    delete s;
    return DPS_OK;
}

}  // extern "C"
