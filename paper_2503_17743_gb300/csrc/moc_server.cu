// Serving engine: independent eigenvalue and fixed-source solves of different
// geometries and group counts, kept resident on the device and advanced
// together (continuous batching).  The paper solves one problem at a time;
// this is a library service around its solver.
//
// * Requests queue in arrival order.  A request is admitted when a slot is
//   free and its device footprint (moc_query_footprint: resident state plus
//   stored templates) fits the memory budget next to the resident solves; a
//   request larger than the whole budget finishes with MOC_ERR_OUT_OF_MEMORY.
// * A solve that fails (generation, an enqueue, a kernel) finishes with its
//   own error status; the other resident solves go on.
// * Every resident solve owns its stream and its captured iteration graphs.
//   One engine step enqueues a quantum of outer iterations on every resident
//   solve that is idle, so the kernels of different solves overlap on the
//   device, then waits for the oldest quantum in flight and retires every
//   solve whose stopping rule held (or that reached max_iter), freeing its
//   slot and memory for the queue.
// * Track generation (host laydown and tracing, device tables, graph capture)
//   runs on a pool of host worker threads, so admitting a request does not
//   stall the quanta of the resident solves.
// * A converged solve's later iterations are no-ops on the device, so the
//   quantum does not change any result: a solve gives the same answer alone
//   and in any mix (up to the order of floating-point atomic adds).
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "moc_serve.h"

namespace {

double now_seconds() {
    using clk = std::chrono::steady_clock;
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

struct Request {
    int64_t ticket = 0;
    std::unique_ptr<moc_geometry> geom;
    moc_track_params tp{};
    moc_solve_params sp{};
    int64_t bytes = 0;
    double t_submit = 0;
};

struct Slot {
    Request req;
    moc_tracks *tr = nullptr;
    cudaEvent_t ev = nullptr;
    int enqueued = 0;
    bool in_flight = false;
    double t_start = 0;
    int gen_status = MOC_OK;  // outcome of the generation on a worker thread
    std::string gen_error;
};

struct Finished {
    int status = MOC_OK;
    std::string error;
    moc_result res{};
    std::vector<double> phi;
    double t_submit = 0, t_start = 0, t_finish = 0;
};

}  // namespace

struct moc_server {
    int device = 0;
    int max_active = 16;
    int64_t budget = 0;
    int quantum = 8;
    int64_t next_ticket = 1;
    int64_t bytes_resident = 0;
    int64_t n_finished = 0, n_admitted = 0, max_resident = 0;
    std::deque<Request> queue;
    std::vector<std::unique_ptr<Slot>> active;
    std::map<int64_t, Finished> done;
    // generation on worker threads: `generating` counts admitted requests not
    // yet resident; `to_gen` / `gen_done` are guarded by `mu`
    int generating = 0;
    std::set<int64_t> gen_tickets;  // main thread only
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::unique_ptr<Slot>> to_gen, gen_done;
    bool stop = false;
    std::vector<std::thread> workers;

    void worker() {
        cudaSetDevice(device);
        for (;;) {
            std::unique_ptr<Slot> s;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] { return stop || !to_gen.empty(); });
                if (stop && to_gen.empty()) return;
                s = std::move(to_gen.front());
                to_gen.pop_front();
            }
            int rc = moc_generate_tracks(s->req.geom.get(), &s->req.tp, &s->tr);
            if (rc == MOC_OK) rc = tracks_start_solve(s->tr, &s->req.sp);
            if (rc == MOC_OK && cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming) != cudaSuccess) {
                moc_set_error("cudaEventCreate failed");
                rc = MOC_ERR_CUDA;
            }
            s->gen_status = rc;
            if (rc != MOC_OK) s->gen_error = moc_last_error();
            {
                std::lock_guard<std::mutex> lk(mu);
                gen_done.push_back(std::move(s));
            }
            cv_done.notify_all();
        }
    }

    void start_workers(int n) {
        for (int i = 0; i < n; ++i) workers.emplace_back([this] { worker(); });
    }

    ~moc_server() {
        {
            std::lock_guard<std::mutex> lk(mu);
            stop = true;
        }
        cv_work.notify_all();
        for (auto &t : workers) t.join();
        auto drop = [](std::unique_ptr<Slot> &s) {
            if (s->tr) moc_destroy_tracks(s->tr);
            if (s->ev) cudaEventDestroy(s->ev);
        };
        for (auto &s : active) drop(s);
        for (auto &s : to_gen) drop(s);
        for (auto &s : gen_done) drop(s);
    }

    void finish(std::unique_ptr<Slot> &s, int status, const std::string &err) {
        Finished f;
        f.status = status;
        f.error = err;
        f.t_submit = s->req.t_submit;
        f.t_start = s->t_start;
        if (s->tr && status == MOC_OK) {
            int conv = 0;
            int rc = tracks_read_state(s->tr, &f.res, &conv);
            if (rc == MOC_OK) {
                f.phi.resize((size_t)s->req.geom->nfsr * s->req.geom->G);
                rc = moc_get_flux(s->tr, f.phi.data(), nullptr);
            }
            if (rc != MOC_OK) {
                f.status = rc;
                f.error = moc_last_error();
            } else if (!conv && s->req.sp.tol_src > 0) {
                f.status = MOC_ERR_NOT_CONVERGED;
                f.error = "not converged within max_iter";
            }
        }
        f.t_finish = now_seconds();
        if (s->tr) moc_destroy_tracks(s->tr);
        s->tr = nullptr;
        if (s->ev) cudaEventDestroy(s->ev);
        s->ev = nullptr;
        bytes_resident -= s->req.bytes;
        done[s->req.ticket] = std::move(f);
        ++n_finished;
    }

    // a queued request that can never be admitted: finished with its error
    void reject(Request &&r, int status, const std::string &err) {
        Finished f;
        f.status = status;
        f.error = err;
        f.t_submit = r.t_submit;
        f.t_start = f.t_finish = now_seconds();
        done[r.ticket] = std::move(f);
        ++n_finished;
    }

    // admit queued requests while a slot and the memory allow; their tracks
    // are generated on the worker threads.  A request whose footprint alone
    // exceeds the budget finishes with MOC_ERR_OUT_OF_MEMORY (its neighbours
    // are not disturbed).  Returns the requests rejected.
    int admit() {
        int added = 0, rejected = 0;
        while (!queue.empty() && queue.front().bytes > budget) {
            Request r = std::move(queue.front());
            queue.pop_front();
            const std::string msg = "request footprint " + std::to_string(r.bytes) +
                                    " bytes exceeds the memory budget of " + std::to_string(budget);
            reject(std::move(r), MOC_ERR_OUT_OF_MEMORY, msg);
            ++rejected;
        }
        while (!queue.empty() && (int)active.size() + generating < max_active &&
               ((active.empty() && generating == 0) || bytes_resident + queue.front().bytes <= budget)) {
            auto s = std::make_unique<Slot>();
            s->req = std::move(queue.front());
            queue.pop_front();
            s->t_start = now_seconds();
            bytes_resident += s->req.bytes;
            ++n_admitted;
            ++generating;
            ++added;
            gen_tickets.insert(s->req.ticket);
            std::lock_guard<std::mutex> lk(mu);
            to_gen.push_back(std::move(s));
            while (!queue.empty() && queue.front().bytes > budget) {
                Request r = std::move(queue.front());
                queue.pop_front();
                reject(std::move(r), MOC_ERR_OUT_OF_MEMORY, "request footprint exceeds the memory budget");
                ++rejected;
            }
        }
        if (added) cv_work.notify_all();
        return rejected;
    }

    // generated requests become resident (or finish with their error); with
    // `wait` and nothing resident, block until one generation completes
    void take_generated(bool wait) {
        std::deque<std::unique_ptr<Slot>> got;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (wait && gen_done.empty() && generating > 0)
                cv_done.wait_for(lk, std::chrono::milliseconds(200), [&] { return !gen_done.empty(); });
            got.swap(gen_done);
        }
        for (auto &s : got) {
            --generating;
            gen_tickets.erase(s->req.ticket);
            if (s->gen_status != MOC_OK) {
                finish(s, s->gen_status, s->gen_error);
                continue;
            }
            active.push_back(std::move(s));
            max_resident = std::max<int64_t>(max_resident, (int64_t)active.size());
        }
    }

    // a quantum of iterations on every idle resident solve; a solve whose
    // enqueue fails finishes with that error and the others go on.  Returns
    // the solves finished here.
    int launch() {
        int nf = 0;
        for (size_t i = 0; i < active.size();) {
            auto &s = active[i];
            if (!s->in_flight) {
                const int n = std::min(quantum, s->req.sp.max_iter - s->enqueued);
                const int rc = tracks_enqueue_iterations(s->tr, n, s->ev);
                if (rc != MOC_OK) {
                    finish(s, rc, moc_last_error());
                    active.erase(active.begin() + i);
                    ++nf;
                    continue;
                }
                s->enqueued += n;
                s->in_flight = true;
            }
            ++i;
        }
        return nf;
    }

    // retire the solves whose quantum has completed and whose stopping rule
    // held (or that used up max_iter)
    int collect(int *finished) {
        int nf = 0;
        for (size_t i = 0; i < active.size();) {
            auto &s = active[i];
            cudaError_t q = cudaEventQuery(s->ev);
            if (q == cudaErrorNotReady) { ++i; continue; }
            if (q != cudaSuccess) {
                finish(s, MOC_ERR_CUDA, std::string("solve: ") + cudaGetErrorString(q));
            } else {
                s->in_flight = false;
                moc_result r{};
                int conv = 0;
                int rc = tracks_read_state(s->tr, &r, &conv);
                if (rc != MOC_OK) finish(s, rc, moc_last_error());
                else if (conv || s->enqueued >= s->req.sp.max_iter) finish(s, MOC_OK, "");
                else { ++i; continue; }
            }
            ++nf;
            active.erase(active.begin() + i);
        }
        *finished += nf;
        return MOC_OK;
    }
};

extern "C" int moc_server_create(const moc_server_params *p, moc_server **out) {
    if (!p || !out) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    if (p->max_active < 0 || p->iterations_per_poll < 0 || p->memory_budget_bytes < 0) {
        moc_set_error("moc_server_create: negative parameter");
        return MOC_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(p->device) != cudaSuccess) { moc_set_error("cudaSetDevice failed"); return MOC_ERR_CUDA; }
    auto s = std::make_unique<moc_server>();
    s->device = p->device;
    s->max_active = p->max_active > 0 ? p->max_active : 16;
    s->quantum = p->iterations_per_poll > 0 ? p->iterations_per_poll : 8;
    if (p->memory_budget_bytes > 0) {
        s->budget = p->memory_budget_bytes;
    } else {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            moc_set_error("cudaMemGetInfo failed");
            return MOC_ERR_CUDA;
        }
        s->budget = (int64_t)(0.8 * (double)free_b);
    }
    s->start_workers(4);
    *out = s.release();
    return MOC_OK;
}

extern "C" void moc_server_destroy(moc_server *s) {
    if (!s) return;
    cudaSetDevice(s->device);
    delete s;
}

extern "C" int moc_server_submit(moc_server *s, const moc_geometry *g, const moc_track_params *tp,
                                 const moc_solve_params *sp, int64_t *ticket) {
    if (!s || !g || !tp || !sp || !ticket) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    if (sp->max_iter < 1) { moc_set_error("moc_server_submit: max_iter < 1"); return MOC_ERR_INVALID_ARG; }
    if (tp->device != s->device) { moc_set_error("moc_server_submit: track parameters name another device"); return MOC_ERR_INVALID_ARG; }
    int64_t resident = 0, preload = 0;
    int rc = moc_query_footprint(g, tp, &resident, &preload);
    if (rc) return rc;
    Request r;
    r.ticket = s->next_ticket++;
    r.geom = std::make_unique<moc_geometry>(*g);
    r.tp = *tp;
    r.sp = *sp;
    r.sp.use_graph = 1;
    r.bytes = resident + (tp->preload_budget_bytes < 0 ? preload : std::min(preload, tp->preload_budget_bytes));
    r.t_submit = now_seconds();
    *ticket = r.ticket;
    s->queue.push_back(std::move(r));
    return MOC_OK;
}

extern "C" int moc_server_step(moc_server *s, int32_t *finished, int32_t *pending) {
    if (finished) *finished = 0;
    if (!s) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    if (pending) *pending = (int32_t)(s->queue.size() + s->active.size() + s->generating);
    if (cudaSetDevice(s->device) != cudaSuccess) { moc_set_error("cudaSetDevice failed"); return MOC_ERR_CUDA; }
    int nf = s->admit();
    s->take_generated(s->active.empty());
    nf += s->launch();
    // wait for the oldest quantum in flight, then retire what is done and
    // keep the rest busy.  A solve that failed on the device is finished with
    // its error by collect(); the step itself fails only when the error is
    // sticky (the device context is lost for every solve).
    bool sticky = false;
    if (!s->active.empty() && cudaEventSynchronize(s->active.front()->ev) != cudaSuccess) {
        (void)cudaGetLastError();
        sticky = cudaGetLastError() != cudaSuccess;
    }
    s->collect(&nf);
    if (!sticky) {
        nf += s->admit();
        s->take_generated(false);
        nf += s->launch();
    }
    if (finished) *finished = nf;
    if (pending) *pending = (int32_t)(s->queue.size() + s->active.size() + s->generating);
    if (sticky) {
        moc_set_error("moc_server_step: the device context reported a sticky error");
        return MOC_ERR_CUDA;
    }
    return MOC_OK;
}

extern "C" int moc_server_result(moc_server *s, int64_t ticket, moc_result *res, double *phi,
                                 int64_t phi_len, double *times, int32_t *ready) {
    if (!s || !ready) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    auto it = s->done.find(ticket);
    if (it == s->done.end()) {
        bool known = false;
        for (auto &r : s->queue) known |= r.ticket == ticket;
        for (auto &a : s->active) known |= a->req.ticket == ticket;
        known |= s->gen_tickets.count(ticket) > 0;
        if (!known) { moc_set_error("moc_server_result: unknown or already fetched ticket"); return MOC_ERR_INVALID_ARG; }
        *ready = 0;
        return MOC_OK;
    }
    Finished &f = it->second;
    *ready = 1;
    if (res) *res = f.res;
    if (phi) {
        if (phi_len < (int64_t)f.phi.size()) { moc_set_error("moc_server_result: phi buffer too small"); return MOC_ERR_INVALID_ARG; }
        std::copy(f.phi.begin(), f.phi.end(), phi);
    }
    if (times) {
        times[0] = f.t_start - f.t_submit;   // queueing
        times[1] = f.t_finish - f.t_submit;  // latency
    }
    const int status = f.status;
    if (status != MOC_OK) moc_set_error(f.error);
    s->done.erase(it);
    return status;
}

extern "C" int moc_server_stats(const moc_server *s, int64_t *out, int32_t n) {
    if (!s || !out) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    const int64_t v[7] = {(int64_t)s->queue.size() + s->generating, (int64_t)s->active.size(), s->n_admitted,
                          s->n_finished, s->bytes_resident, s->budget, s->max_resident};
    for (int i = 0; i < n && i < 7; ++i) out[i] = v[i];
    return MOC_OK;
}
