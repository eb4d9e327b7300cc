// Serving engine of libibrigid: a request loop over constrained rigid-body
// Stokes solves (the problem of Sec. III.B / III.D, solved as in Sec. V) with
// continuous batching on one GPU.
//
//  - `slots` worker threads, each issuing its solves on its own non-blocking
//    CUDA stream: requests that run at the same time overlap on the device.
//  - Admission by an HBM budget: a request is started when a slot is free and
//    the device bytes it needs (the grid-size estimate of
//    ibr_estimate_device_bytes) fit next to what the running requests and the
//    resident grids hold; the oldest waiting request may evict idle resident
//    grids (least recently used first); younger requests may start ahead of
//    an oldest one that does not fit, at most kMaxBypass times in a row.
//  - Residency: a finished request's grid (multigrid hierarchy, Krylov
//    workspace, marker data, factorised mobility, captured preconditioner
//    graph) stays on the device; the next request of the same shape reuses
//    it, and one with the same geometry also skips the set-up (binning, M~
//    build and factorisation).
//  - Optional schedule autotuning: the first request of each shape is solved
//    once per candidate (inner iterations N_s, multigrid sweeps) and the
//    fastest schedule is kept for that shape; requests of a shape under
//    tuning wait for it.
// Results (status, iterations, residual, timestamps, Lambda, body forces and
// optionally the fields) are kept on the host until the caller polls them.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ibr_internal.cuh"

namespace ibr {
long long estimate_grid_bytes(int d, const int* n, int B, const int* Nb, int restart, int ns, int precision,
                              int mob_model);
void grid_clear_bodies(ibr_grid* G);
void grid_set_stream(ibr_grid* G, cudaStream_t s);
}  // namespace ibr

namespace {

using ibr::Error;

constexpr int kMaxBypass = 8;

struct Hash2 {
    unsigned long long a = 1469598103934665603ULL, b = 0x9E3779B97F4A7C15ULL;
    void add(const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) {
            a = (a ^ c[i]) * 1099511628211ULL;
            b = (b ^ c[i]) * 0x100000001B3ULL + 0x632BE59BD9B4E019ULL;
        }
    }
    template <typename T>
    void add(const T& v) {
        add(&v, sizeof(T));
    }
    std::string key() const { return std::to_string(a) + ":" + std::to_string(b); }
};

// a request's data, copied at submission
struct Spec {
    int dim = 3;
    int n[3] = {1, 1, 1};
    double L[3] = {1, 1, 1};
    double eta = 1.0;
    int precision = IBR_MIXED;
    int B = 0;
    std::vector<double> xc, quat;  // [B][3], [B][4]
    std::vector<int> kin, nm;      // [B]
    std::vector<double> rb;        // concatenated body-frame offsets
    std::vector<double> UO;
    ibr_solve_opts opts;
    bool opts_given = false;  // the schedule is fixed by the request (n_s != 0)
    int want_fields = 0;
    int N = 0;
    long long ncell = 1;
    std::string shape, geom;
};

struct Ticket {
    Spec sp;
    ibr_result res;
    std::string err;
    std::vector<double> lam, ft, v, p;
    long long est = 0;
    bool done = false;
};

struct Resident {
    ibr_grid* g = nullptr;
    std::string shape, geom;
    long long bytes = 0;
};

struct Tuned {
    int n_s = 0, pre = 2, post = 2;
    bool busy = false;  // a worker is tuning this shape
    bool ready = false;
};

double since_ms(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

void req(bool c, const char* msg) {
    if (!c) throw Error{IBR_EINVAL, msg};
}

}  // namespace

struct ibr_server {
    int device = 0;
    int nslots = 1;
    long long budget = 0;
    int autotune = 0;
    std::chrono::steady_clock::time_point t0;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<long long> pending;
    std::unordered_map<long long, std::unique_ptr<Ticket>> tickets;
    std::list<Resident> idle;  // front: most recently used
    std::map<std::string, Tuned> tuned;
    long long next_ticket = 1;
    long long reserved = 0, peak = 0;
    int bypassed = 0;
    bool stop = false;
    ibr_server_stats st;

    // picks the next request to start (under mu): the request, the resident
    // grid it reuses (or none) and the idle grids to evict first
    bool pick(Ticket*& tk, long long& id, Resident& res, bool& have_res, std::vector<ibr_grid*>& evict) {
        int idx = 0;
        bool head_wants_memory = false;  // the oldest request waits for device memory
        for (auto it = pending.begin(); it != pending.end(); ++it, ++idx) {
            if (head_wants_memory && bypassed >= kMaxBypass) return false;
            Ticket* t = tickets.at(*it).get();
            if (autotune) {
                auto tu = tuned.find(t->sp.shape);
                if (tu != tuned.end() && tu->second.busy) continue;  // shape under tuning
            }
            // a resident grid of the same geometry, else of the same shape
            auto match = idle.end();
            for (auto r = idle.begin(); r != idle.end(); ++r)
                if (r->shape == t->sp.shape) {
                    if (r->geom == t->sp.geom) {
                        match = r;
                        break;
                    }
                    if (match == idle.end()) match = r;
                }
            long long gb = match != idle.end() ? match->bytes : 0;
            long long delta = std::max(gb, t->est) - gb;
            long long free_bytes = budget - reserved;
            std::vector<std::list<Resident>::iterator> ev;
            if (delta > free_bytes && idx == 0) {
                // the oldest request may evict idle grids, least recently used first
                long long gain = 0;
                for (auto r = idle.end(); r != idle.begin();) {
                    --r;
                    if (r == match) continue;
                    ev.push_back(r);
                    gain += r->bytes;
                    if (delta <= free_bytes + gain) break;
                }
                if (delta > free_bytes + gain) ev.clear();
                else free_bytes += gain;
            }
            if (delta > free_bytes) {
                if (idx == 0) head_wants_memory = true;
                continue;
            }
            for (auto& r : ev) {
                reserved -= r->bytes;
                evict.push_back(r->g);
                idle.erase(r);
                st.evictions++;
            }
            have_res = match != idle.end();
            if (have_res) {
                res = *match;
                idle.erase(match);
                res.bytes = std::max(res.bytes, t->est);
            } else {
                res = Resident();
                res.bytes = t->est;
                res.shape = t->sp.shape;
            }
            reserved += delta;
            peak = std::max(peak, reserved);
            tk = t;
            id = *it;
            pending.erase(it);
            bypassed = head_wants_memory ? bypassed + 1 : 0;
            t->res.status = IBR_RUNNING;
            st.queued--;
            st.running++;
            if (autotune) {
                Tuned& tu = tuned[t->sp.shape];
                if (!tu.ready && !tu.busy && !t->sp.opts_given) tu.busy = true;
            }
            return true;
        }
        return false;
    }

    // one solve on the worker's stream; returns the status and the grid to keep
    // (nullptr when it was destroyed after an error)
    int run(int slot, Ticket* t, Resident& r, bool have_res) {
        const Spec& sp = t->sp;
        cudaStream_t s = streams[slot];
        ibr_grid* g = have_res ? r.g : nullptr;
        auto fail = [&](int rc) {
            t->err = ibr_last_error();
            return rc;
        };
        if (!g) {
            int bc[6] = {IBR_PERIODIC, IBR_PERIODIC, IBR_PERIODIC, IBR_PERIODIC, IBR_PERIODIC, IBR_PERIODIC};
            int rc = ibr_create_grid(&g, sp.dim, sp.n, sp.L, bc, sp.eta, 0.0, 0.0, IBR_KERNEL_PESKIN4, sp.precision, s);
            if (rc != IBR_OK) return fail(rc);
            r.g = g;
            st_add(&ibr_server_stats::grids_created);
        } else {
            ibr::grid_set_stream(g, s);
            st_add(&ibr_server_stats::grids_reused);
        }
        t->res.reused_grid = have_res ? 1 : 0;
        if (!(have_res && r.geom == sp.geom)) {
            ibr::grid_clear_bodies(g);
            r.geom.clear();
            const double* rb = sp.rb.data();
            for (int b = 0; b < sp.B; ++b) {
                int id = 0;
                int rc = ibr_add_body(g, &sp.xc[3 * b], &sp.quat[4 * b], sp.kin[b], &id);
                if (rc == IBR_OK) rc = ibr_set_markers(g, id, rb, sp.nm[b]);
                if (rc != IBR_OK) return fail(rc);
                rb += (size_t)sp.nm[b] * sp.dim;
            }
            r.geom = sp.geom;
        } else {
            t->res.reused_geometry = 1;
            st_add(&ibr_server_stats::geometry_reused);
        }
        ibr_solve_opts o = sp.opts;
        ibr_solve_info info;
        std::memset(&info, 0, sizeof(info));
        int rc = IBR_OK;
        bool tune_now = false;
        if (autotune && !sp.opts_given) {
            std::lock_guard<std::mutex> lk(mu);
            Tuned& tu = tuned[sp.shape];
            if (tu.ready) {
                o.n_s = tu.n_s;
                o.mg_pre = tu.pre;
                o.mg_post = tu.post;
            } else {
                tune_now = tu.busy;
            }
        }
        if (tune_now) {
            // candidates: N_s in {1, 2, 3} x sweeps in {1/1, 2/2}; the first
            // solve also runs the set-up, so it is repeated after the others
            const int cand[6][3] = {{2, 2, 2}, {1, 2, 2}, {3, 2, 2}, {2, 1, 1}, {1, 1, 1}, {3, 1, 1}};
            double best = 1e300;
            int bi = 0;
            for (int c = 0; c <= 6; ++c) {
                const int k = c < 6 ? c : 0;
                ibr_solve_opts oc = o;
                oc.n_s = cand[k][0];
                oc.mg_pre = cand[k][1];
                oc.mg_post = cand[k][2];
                ibr_solve_info ic;
                int rcc = ibr_solve_coupled(g, sp.UO.data(), nullptr, 0, &oc, &ic);
                if (c == 0) continue;
                if ((rcc == IBR_OK) && ic.ms_solve < best) {
                    best = ic.ms_solve;
                    bi = k;
                }
            }
            o.n_s = cand[bi][0];
            o.mg_pre = cand[bi][1];
            o.mg_post = cand[bi][2];
            {
                std::lock_guard<std::mutex> lk(mu);
                Tuned& tu = tuned[sp.shape];
                tu.n_s = o.n_s;
                tu.pre = o.mg_pre;
                tu.post = o.mg_post;
                tu.busy = false;
                tu.ready = true;
                st.tuned_shapes++;
            }
            cv_work.notify_all();
            t->res.tuned = 1;
        }
        t->res.n_s = o.n_s;
        t->res.mg_pre = o.mg_pre;
        t->res.mg_post = o.mg_post;
        rc = ibr_solve_coupled(g, sp.UO.data(), nullptr, 0, &o, &info);
        t->res.iters = info.iters;
        t->res.rel_res_true = info.rel_res_true;
        t->res.ms_setup = info.ms_setup;
        t->res.ms_solve = info.ms_solve;
        if (rc != IBR_OK && rc != IBR_ENOTCONV && rc != IBR_ETIMEOUT) return fail(rc);
        const int rot = sp.dim == 2 ? 1 : 3;
        t->lam.resize((size_t)sp.N * sp.dim);
        t->ft.resize((size_t)sp.B * (sp.dim + rot));
        int rc2 = ibr_get_forces(g, t->lam.data(), t->ft.data());
        if (rc2 == IBR_OK && sp.want_fields) {
            t->v.resize((size_t)sp.dim * sp.ncell);
            t->p.resize((size_t)sp.ncell);
            rc2 = ibr_get_fields(g, t->v.data(), t->p.data(), 0);
        }
        if (rc2 != IBR_OK) return fail(rc2);
        if (rc != IBR_OK) t->err = ibr_last_error();
        return rc;
    }

    void st_add(long long ibr_server_stats::*f) {
        std::lock_guard<std::mutex> lk(mu);
        st.*f += 1;
    }

    void worker(int slot) {
        cudaSetDevice(device);
        while (true) {
            Ticket* t = nullptr;
            long long id = 0;
            Resident r;
            bool have_res = false;
            std::vector<ibr_grid*> evict;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] { return stop || pick(t, id, r, have_res, evict); });
                if (!t) return;  // stop with nothing picked
                t->res.t_start_ms = since_ms(t0);
                t->res.slot = slot;
                t->res.reserved_bytes = r.bytes;
            }
            for (ibr_grid* g : evict) {
                // idle grids were synchronised when their request ended; moved
                // to this worker's stream, their destruction waits for nobody else
                ibr::grid_set_stream(g, streams[slot]);
                ibr_destroy_grid(g);
            }
            int rc = IBR_ECUDA;
            try {
                rc = run(slot, t, r, have_res);
            } catch (...) {
                t->err = "ibr_server: worker failed";
                rc = IBR_ECUDA;
            }
            // a grid whose solve failed for another reason than convergence is not kept
            const bool keep = r.g && (rc == IBR_OK || rc == IBR_ENOTCONV || rc == IBR_ETIMEOUT);
            if (!keep && r.g) {
                ibr_destroy_grid(r.g);
                r.g = nullptr;
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                t->res.status = rc;
                t->res.t_end_ms = since_ms(t0);
                t->done = true;
                st.running--;
                st.completed++;
                if (keep) {
                    idle.push_front(r);
                } else {
                    reserved -= r.bytes;
                }
                if (autotune) {
                    auto tu = tuned.find(t->sp.shape);
                    if (tu != tuned.end() && tu->second.busy && !tu->second.ready) tu->second.busy = false;
                }
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
    }
};

namespace {

int guarded(const char* fn, const std::function<void()>& body) {
    try {
        body();
        ibr::set_error("");
        return IBR_OK;
    } catch (const Error& e) {
        ibr::set_error(std::string(fn) + ": " + e.msg);
        return e.code;
    } catch (const std::bad_alloc&) {
        ibr::set_error(std::string(fn) + ": host allocation failed");
        return IBR_ENOMEM;
    } catch (const std::exception& e) {
        ibr::set_error(std::string(fn) + ": " + e.what());
        return IBR_EINVAL;
    }
}

}  // namespace

extern "C" {

int ibr_server_create(ibr_server** out, int slots, long long hbm_budget_bytes, int flags) {
    return guarded("ibr_server_create", [&] {
        req(out != nullptr, "out is NULL");
        *out = nullptr;
        req(slots >= 1 && slots <= 64, "slots must be in [1, 64]");
        req(hbm_budget_bytes > 0, "hbm_budget_bytes must be positive");
        req((flags & ~IBR_SERVER_AUTOTUNE) == 0, "unknown flags");
        std::unique_ptr<ibr_server> S(new ibr_server());
        IBR_CUDA_TRY(cudaGetDevice(&S->device));
        S->nslots = slots;
        S->budget = hbm_budget_bytes;
        S->autotune = (flags & IBR_SERVER_AUTOTUNE) ? 1 : 0;
        S->t0 = std::chrono::steady_clock::now();
        std::memset(&S->st, 0, sizeof(S->st));
        for (int i = 0; i < slots; ++i) {
            cudaStream_t s;
            cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
                throw Error{IBR_ECUDA, std::string("cudaStreamCreateWithFlags: ") + cudaGetErrorString(e)};
            }
            S->streams.push_back(s);
        }
        ibr_server* raw = S.get();
        for (int i = 0; i < slots; ++i) S->workers.emplace_back([raw, i] { raw->worker(i); });
        *out = S.release();
    });
}

int ibr_server_submit(ibr_server* S, const ibr_request* r, long long* ticket) {
    return guarded("ibr_server_submit", [&] {
        req(S && r && ticket, "server, request and ticket must be non-NULL");
        std::unique_ptr<Ticket> t(new Ticket());
        Spec& sp = t->sp;
        req(r->dim == 2 || r->dim == 3, "dim must be 2 or 3");
        sp.dim = r->dim;
        sp.ncell = 1;
        for (int a = 0; a < sp.dim; ++a) {
            req(r->n[a] >= 4 && r->n[a] % 2 == 0, "each n[a] must be even and >= 4");
            req(r->L[a] > 0, "L[a] must be positive");
            sp.n[a] = r->n[a];
            sp.L[a] = r->L[a];
            sp.ncell *= r->n[a];
        }
        req(r->eta > 0, "eta must be positive");
        req(r->precision == IBR_FP64 || r->precision == IBR_MIXED, "bad precision");
        req(r->n_bodies >= 1, "n_bodies must be >= 1");
        req(r->x_c && r->n_markers && r->r_body && r->body_UO, "x_c, n_markers, r_body, body_UO must be non-NULL");
        sp.eta = r->eta;
        sp.precision = r->precision;
        sp.B = r->n_bodies;
        const int rot = sp.dim == 2 ? 1 : 3;
        sp.xc.assign((size_t)3 * sp.B, 0.0);
        sp.quat.assign((size_t)4 * sp.B, 0.0);
        sp.kin.assign(sp.B, IBR_PRESCRIBED);
        sp.nm.assign(r->n_markers, r->n_markers + sp.B);
        for (int b = 0; b < sp.B; ++b) {
            for (int a = 0; a < sp.dim; ++a) sp.xc[3 * b + a] = r->x_c[(size_t)sp.dim * b + a];
            if (r->quat)
                for (int q = 0; q < 4; ++q) sp.quat[4 * b + q] = r->quat[4 * b + q];
            else
                sp.quat[4 * b] = 1.0;
            if (r->kinematics) sp.kin[b] = r->kinematics[b];
            req(sp.nm[b] >= 1, "every body needs >= 1 marker");
            sp.N += sp.nm[b];
        }
        sp.rb.assign(r->r_body, r->r_body + (size_t)sp.N * sp.dim);
        sp.UO.assign(r->body_UO, r->body_UO + (size_t)sp.B * (sp.dim + rot));
        if (r->opts) {
            sp.opts = *r->opts;
        } else {
            ibr_solve_opts_default(&sp.opts);
        }
        // the autotuner may choose N_s and the multigrid sweeps unless the
        // request fixes N_s (opts with n_s != 0)
        sp.opts_given = sp.opts.n_s != 0;
        sp.want_fields = r->want_fields;
        Hash2 hs;
        hs.add(sp.dim);
        hs.add(sp.n);
        hs.add(sp.L);
        hs.add(sp.eta);
        hs.add(sp.precision);
        sp.shape = hs.key();
        Hash2 hg = hs;
        hg.add(sp.B);
        hg.add(sp.xc.data(), sp.xc.size() * sizeof(double));
        hg.add(sp.quat.data(), sp.quat.size() * sizeof(double));
        hg.add(sp.kin.data(), sp.kin.size() * sizeof(int));
        hg.add(sp.nm.data(), sp.nm.size() * sizeof(int));
        hg.add(sp.rb.data(), sp.rb.size() * sizeof(double));
        hg.add(sp.opts.mob_model);
        hg.add(sp.opts.mob_a_over_h);
        hg.add(sp.opts.mob_coef);
        sp.geom = hg.key();
        // N_s = 0 is 2 on periodic grids; the autotuner may pick up to 3
        const int ns = sp.opts.n_s > 0 ? sp.opts.n_s : (S->autotune && !sp.opts_given ? 3 : 2);
        t->est = ibr::estimate_grid_bytes(sp.dim, sp.n, sp.B, sp.nm.data(), sp.opts.restart, ns, sp.precision,
                                          sp.opts.mob_model);
        std::memset(&t->res, 0, sizeof(t->res));
        t->res.n_markers = sp.N;
        t->res.n_bodies = sp.B;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            t->res.t_submit_ms = since_ms(S->t0);
            long long id = S->next_ticket++;
            S->st.submitted++;
            if (t->est > S->budget) {
                // can never fit: finished at once with IBR_ENOMEM
                t->res.status = IBR_ENOMEM;
                t->res.t_start_ms = t->res.t_end_ms = t->res.t_submit_ms;
                t->res.reserved_bytes = t->est;
                t->err = "ibr_server: the request needs " + std::to_string(t->est) +
                         " device bytes, more than the server's budget";
                t->done = true;
                S->st.rejected++;
                S->st.completed++;
            } else {
                t->res.status = IBR_QUEUED;
                S->pending.push_back(id);
                S->st.queued++;
            }
            S->tickets[id] = std::move(t);
            *ticket = id;
        }
        S->cv_work.notify_all();
    });
}

int ibr_server_poll(ibr_server* S, long long ticket, double timeout_ms, ibr_result* res, double* Lambda,
                    double* body_FT, double* v, double* p) {
    std::unique_ptr<Ticket> t;
    int rc = guarded("ibr_server_poll", [&] {
        req(S != nullptr, "server is NULL");
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->tickets.find(ticket);
        req(it != S->tickets.end(), "unknown ticket (never issued, or already collected)");
        Ticket* tp = it->second.get();
        auto ready = [&] { return tp->done; };
        if (timeout_ms < 0)
            S->cv_done.wait(lk, ready);
        else if (timeout_ms > 0)
            S->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), ready);
        if (!tp->done) {
            if (res) *res = tp->res;
            throw Error{IBR_EPENDING, "ticket not finished"};
        }
        t = std::move(it->second);
        S->tickets.erase(it);
    });
    if (!t) return rc;
    const Spec& sp = t->sp;
    if (res) *res = t->res;
    if (Lambda && !t->lam.empty()) std::memcpy(Lambda, t->lam.data(), t->lam.size() * sizeof(double));
    if (body_FT && !t->ft.empty()) std::memcpy(body_FT, t->ft.data(), t->ft.size() * sizeof(double));
    if (v && !t->v.empty()) std::memcpy(v, t->v.data(), t->v.size() * sizeof(double));
    if (p && !t->p.empty()) std::memcpy(p, t->p.data(), t->p.size() * sizeof(double));
    (void)sp;
    ibr::set_error(t->err);
    return t->res.status;
}

int ibr_server_get_stats(ibr_server* S, ibr_server_stats* out) {
    return guarded("ibr_server_get_stats", [&] {
        req(S && out, "server and out must be non-NULL");
        std::lock_guard<std::mutex> lk(S->mu);
        *out = S->st;
        out->reserved_bytes = S->reserved;
        out->peak_reserved_bytes = S->peak;
        out->budget_bytes = S->budget;
        out->resident_grids = (long long)S->idle.size();
    });
}

int ibr_server_destroy(ibr_server* S) {
    if (!S) return IBR_OK;
    return guarded("ibr_server_destroy", [&] {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop = true;
            // requests not yet started are dropped
            S->pending.clear();
        }
        S->cv_work.notify_all();
        for (auto& w : S->workers) w.join();
        for (auto& r : S->idle) ibr_destroy_grid(r.g);
        S->idle.clear();
        for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
        delete S;
    });
}

}  // extern "C"
