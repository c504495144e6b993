// Request server: continuous batching of forward + adjoint + sensitivity requests on
// one GPU.  Requests wait in a FIFO queue; a slot takes the head request as soon as a
// slot is free and its device-memory footprint fits the budget, so requests that arrive
// while others run are admitted as slots and memory free up and their work overlaps
// on the device (one CUDA stream per slot).  Meshes (hierarchy and Krylov buffers) are
// kept in an idle pool keyed by their description and reused by later requests of the
// same shape; idle meshes are released when the budget needs the room.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/st.h"

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Pool key of a mesh description: its fields one by one (the struct's padding bytes, which
// a C caller may leave uninitialised, take no part).
template <typename V>
void put(std::string& k, const V& v) {
    k.append(reinterpret_cast<const char*>(&v), sizeof(v));
}

std::string desc_key(const st_mesh_desc& d) {
    std::string k;
    put(k, d.ndim_space);
    for (int q = 0; q < 3; ++q) put(k, d.n[q]);
    put(k, d.n_t);
    for (int q = 0; q < 3; ++q) put(k, d.ext[q]);
    put(k, d.tau);
    put(k, d.mat.C_ins);
    put(k, d.mat.C_con);
    put(k, d.mat.k_ins);
    put(k, d.mat.k_con);
    put(k, d.mat.p_c);
    put(k, d.mat.p_k);
    put(k, d.bc);
    put(k, d.bc_width);
    put(k, d.lambda_crit);
    put(k, d.coarse_dof_cap);
    put(k, d.max_levels);
    put(k, d.coarsening);
    put(k, d.device);
    put(k, d.coarse_solver);
    put(k, d.coarse_max_it);
    put(k, d.coarse_rtol);
    put(k, d.march_blocks);
    put(k, d.smoother);
    put(k, d.smoother_omega);
    return k;
}

struct Job {
    uint64_t ticket = 0;
    st_request req{};
    std::vector<double> gamma;
    std::vector<double> grad;
    st_result res{};
    long long footprint = 0;
    double t_submit = 0, t_admit = 0;
    bool done = false;
    st_mesh* mesh = nullptr;  // an idle mesh of the request's shape taken at admission, if any
    long long nodes = 0;      // fine-level node count
};

bool same_options(const st_options& a, const st_options& b) {
    return a.rtol == b.rtol && a.max_it == b.max_it && a.restart == b.restart && a.precision == b.precision &&
           a.warm_start == b.warm_start && a.smooth_steps == b.smooth_steps && a.use_graphs == b.use_graphs;
}

struct Pooled {
    st_mesh* mesh;
    long long bytes;
};

}  // namespace

struct st_server {
    st_server_desc desc{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> queue;
    std::map<uint64_t, std::shared_ptr<Job>> jobs;
    std::multimap<std::string, Pooled> idle;
    std::list<std::string> idle_lru;  // keys, most recent at the back
    long long in_use = 0, idle_bytes = 0;
    uint64_t next_ticket = 1;
    bool stopping = false;
    std::vector<std::thread> workers;

    // Take idle meshes (least recently used first) out of the pool until `need` more bytes
    // fit; the caller destroys them after releasing the lock (st_destroy_mesh frees device
    // memory, which synchronises the device, and must not stall the other slots' admission).
    void evict_for(long long need, std::vector<st_mesh*>& doomed) {
        while (in_use + idle_bytes + need > desc.hbm_budget && !idle_lru.empty()) {
            const std::string key = idle_lru.front();
            idle_lru.pop_front();
            auto it = idle.find(key);
            if (it == idle.end()) continue;
            idle_bytes -= it->second.bytes;
            doomed.push_back(it->second.mesh);
            idle.erase(it);
        }
    }

    int max_batch() const { return desc.max_batch > 0 ? desc.max_batch : 8; }
    long long batch_nodes() const { return desc.batch_nodes > 0 ? desc.batch_nodes : (1LL << 21); }
    bool small(const Job& j) const { return j.nodes <= batch_nodes(); }

    // Admission of job j (server lock held): an idle mesh of its shape, else its footprint
    // within the budget (after taking idle meshes out of the pool when allow_evict).
    bool admit(Job& j, bool allow_evict, std::vector<st_mesh*>& doomed) {
        const std::string key = desc_key(j.req.mesh);
        auto it = idle.find(key);
        if (it != idle.end()) {  // reuse an idle mesh of this shape
            j.mesh = it->second.mesh;
            idle_bytes -= it->second.bytes;
            in_use += j.footprint;
            idle.erase(it);
            for (auto l = idle_lru.begin(); l != idle_lru.end(); ++l)
                if (*l == key) {
                    idle_lru.erase(l);
                    break;
                }
            return true;
        }
        if (allow_evict) evict_for(j.footprint, doomed);
        if (in_use + idle_bytes + j.footprint <= desc.hbm_budget) {
            in_use += j.footprint;
            return true;
        }
        return false;
    }

    void worker(int slot) {
        cudaSetDevice(desc.device);
        cudaStream_t stream = nullptr;
        cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
        (void)slot;
        for (;;) {
            std::vector<std::shared_ptr<Job>> batch;
            std::vector<st_mesh*> doomed;
            {
                std::unique_lock<std::mutex> lk(mu);
                for (;;) {
                    if (stopping && queue.empty()) break;
                    if (!queue.empty()) {
                        std::shared_ptr<Job> head = queue.front();
                        if (admit(*head, true, doomed)) {
                            queue.pop_front();
                            batch.push_back(head);
                            // queued small requests with the same options join the head's batch
                            // as long as they fit without evicting anything
                            if (small(*head))
                                for (auto it = queue.begin(); it != queue.end() && (int)batch.size() < max_batch();) {
                                    if (small(**it) && same_options((*it)->req.options, head->req.options) &&
                                        admit(**it, false, doomed)) {
                                        batch.push_back(*it);
                                        it = queue.erase(it);
                                    } else {
                                        ++it;
                                    }
                                }
                            break;
                        }
                    }
                    if (!doomed.empty()) break;  // free them unlocked, then look again
                    cv_work.wait(lk);
                }
            }
            for (st_mesh* d : doomed) st_destroy_mesh(d);
            if (batch.empty()) {
                if (!doomed.empty()) continue;
                break;
            }
            run_batch(batch, stream);
            {
                std::lock_guard<std::mutex> lk(mu);
                for (auto& j : batch) {
                    in_use -= j->footprint;
                    j->done = true;
                }
            }
            cv_work.notify_all();
            cv_done.notify_all();
        }
        if (stream) cudaStreamDestroy(stream);
    }

    // One batch: set-up of every request's mesh, the forward solves of all of them together
    // (st_solve_forward_batch: shared graph launches, convergence decided on the device), the
    // adjoint solves together, then the sensitivities; a request that fails drops out.
    void run_batch(std::vector<std::shared_ptr<Job>>& batch, cudaStream_t stream) {
        const int n = (int)batch.size();
        const double ta = now_s();
        std::vector<Job*> ok;
        for (auto& jp : batch) {
            Job* job = jp.get();
            job->t_admit = ta;
            st_result& r = job->res;
            memset(&r, 0, sizeof(r));
            r.footprint = job->footprint;
            r.batch = n;
            st_status s = ST_OK;
            if (!job->mesh) s = st_create_mesh(&job->req.mesh, &job->mesh);
            if (s == ST_OK) s = st_set_stream(job->mesh, stream);
            if (s == ST_OK)
                s = st_set_design(job->mesh, job->gamma.data(), job->req.layout, job->gamma.size(), ST_MEM_HOST);
            r.status = s;
            if (s == ST_OK) ok.push_back(job);
        }
        auto hard = [](st_status s) { return !(s == ST_OK || s == ST_ERR_NOT_CONVERGED || s == ST_ERR_NUMERIC); };
        const st_options opt = batch[0]->req.options;
        // forward
        std::vector<st_mesh*> ms;
        std::vector<st_source> src;
        for (Job* j : ok) {
            ms.push_back(j->mesh);
            src.push_back(j->req.source);
        }
        const int k = (int)ok.size();
        std::vector<st_stats> fst(k);
        std::vector<st_status> fs(k, ST_OK);
        if (k > 0) {
            const st_status r = st_solve_forward_batch(ms.data(), k, src.data(), &opt, fst.data(), fs.data());
            if (hard(r)) std::fill(fs.begin(), fs.end(), r);
        }
        // adjoint, for the requests with a state
        std::vector<Job*> ok2;
        std::vector<st_mesh*> ms2;
        std::vector<st_objective> obj;
        for (int q = 0; q < k; ++q) {
            ok[q]->res.forward = fst[q];
            if (fs[q] == ST_OK || fs[q] == ST_ERR_NOT_CONVERGED) {
                ok2.push_back(ok[q]);
                ms2.push_back(ok[q]->mesh);
                obj.push_back(ok[q]->req.objective);
            } else {
                ok[q]->res.status = fs[q];
            }
        }
        const int k2 = (int)ok2.size();
        std::vector<st_stats> ast(k2);
        std::vector<st_status> as(k2, ST_OK);
        std::vector<double> phi(k2, 0.0);
        if (k2 > 0) {
            const st_status r =
                st_solve_adjoint_batch(ms2.data(), k2, obj.data(), &opt, phi.data(), ast.data(), as.data());
            if (hard(r)) std::fill(as.begin(), as.end(), r);
        }
        for (int q = 0; q < k2; ++q) {
            Job* job = ok2[q];
            st_result& r = job->res;
            r.adjoint = ast[q];
            r.phi = phi[q];
            st_status s = (as[q] == ST_OK || as[q] == ST_ERR_NOT_CONVERGED) ? ST_OK : as[q];
            if (s == ST_OK && job->req.want_gradient) {
                job->grad.resize(job->gamma.size());
                s = st_sensitivities(job->mesh, job->grad.data(), job->grad.size(), ST_MEM_HOST);
            }
            if (s == ST_OK && !(r.forward.converged && r.adjoint.converged)) s = ST_ERR_NOT_CONVERGED;
            r.status = s;
        }
        const double t = now_s();
        for (auto& jp : batch) {
            Job* job = jp.get();
            job->res.latency_s = t - job->t_submit;
            job->res.queue_s = job->t_admit - job->t_submit;
            st_mesh* mesh = job->mesh;
            job->mesh = nullptr;
            if (!mesh) continue;
            st_set_stream(mesh, nullptr);
            st_mesh_info info{};
            st_mesh_info_get(mesh, &info);
            bool pooled = false;
            {
                std::lock_guard<std::mutex> lk(mu);
                const std::string key = desc_key(job->req.mesh);
                if (!stopping && info.device_bytes <= desc.hbm_budget) {
                    idle.insert({key, Pooled{mesh, info.device_bytes}});
                    idle_lru.push_back(key);
                    idle_bytes += info.device_bytes;
                    pooled = true;
                }
            }
            if (!pooled) st_destroy_mesh(mesh);
        }
    }
};

extern "C" {

long long st_footprint_bytes(const st_mesh_desc* d, int precision, int restart) {
    if (!d) return -1;
    // Hierarchy sizes by the same halving rule the mesh uses, with the worst-case
    // (space-time) element storage; see st_create_mesh for the rule itself.
    const int sd = d->ndim_space;
    long long n[3] = {d->n[0], d->n[1], sd == 3 ? d->n[2] : 1};
    long long nt = d->n_t;
    const int NS = 1 << sd, NV = 4 * NS * (NS + 1) / 2;
    const double Deff = sqrt(d->mat.k_con * d->mat.k_ins / (d->mat.C_con * d->mat.C_ins));
    double h[3] = {d->ext[0] / d->n[0], d->ext[1] / d->n[1], sd == 3 ? d->ext[2] / d->n[2] : 1.0};
    double dt = d->tau / d->n_t;
    const int tsz = precision == ST_PREC_FP64 ? 8 : 4;
    long long bytes = 0, N0 = 0, ne0 = 0, nc = 0;
    bool space_only = true;  // every coarsening so far halved space only
    for (int l = 0; l < 40; ++l) {
        long long N = nt + 1, ne = nt;
        for (int q = 0; q < sd; ++q) {
            N *= n[q] + 1;
            ne *= n[q];
        }
        if (l == 0) {
            N0 = N;
            ne0 = ne;
        } else {
            bytes += ne * NV * 12;  // FP64 + FP32 element blocks
            if (sd == 2 && space_only) bytes += ne * 128;  // M, K rows of the marching kernels
        }
        // b, x, r, dinv, w and, with the GMRES smoother, its 11 basis vectors
        bytes += N * (long long)tsz * (d->smoother == ST_SMOOTH_JACOBI ? 5 : 16);
        nc = N;
        bool can_s = true;
        for (int q = 0; q < sd; ++q) can_s = can_s && n[q] % 2 == 0 && n[q] >= 4;
        const bool can_t = nt % 2 == 0 && nt >= 2;
        if (N <= d->coarse_dof_cap || (d->max_levels > 0 && l + 1 >= d->max_levels)) break;
        int kind;
        if (d->coarsening == ST_COARSEN_FULL) {
            kind = (can_s && can_t) ? 2 : -1;
        } else {
            double hmin = h[0];
            for (int q = 1; q < sd; ++q) hmin = hmin < h[q] ? hmin : h[q];
            kind = Deff * dt / (hmin * hmin) < d->lambda_crit ? 1 : 0;
            if (kind == 1 && !can_t) kind = can_s ? 0 : -1;
            else if (kind == 0 && !can_s) kind = can_t ? 1 : -1;
        }
        if (kind < 0) break;
        space_only = space_only && kind == 0;
        if (kind != 1)
            for (int q = 0; q < sd; ++q) {
                n[q] /= 2;
                h[q] *= 2;
            }
        if (kind != 0) {
            nt /= 2;
            dt *= 2;
        }
    }
    bytes += N0 * 8LL * (5 + restart + 1) + N0 * (long long)tsz * restart;  // FP64 vectors, V, Z
    bytes += ne0 * 26LL;                                                     // design copies, sensitivities
    const bool iter = d->coarse_solver == ST_COARSE_GMRES || (d->coarse_solver == ST_COARSE_AUTO && nc > 4096);
    bytes += iter ? nc * 8LL * 23 : 2 * nc * nc * 8;  // Jacobi-GMRES(16) vectors or the dense inverse
    bytes += 4 << 20;
    return bytes;
}

st_status st_server_create(const st_server_desc* d, st_server** out) {
    if (!d || !out || d->max_inflight < 1 || d->hbm_budget <= 0) return ST_ERR_ARG;
    st_server* s = new st_server();
    s->desc = *d;
    for (int q = 0; q < d->max_inflight; ++q) s->workers.emplace_back([s, q] { s->worker(q); });
    *out = s;
    return ST_OK;
}

st_status st_server_destroy(st_server* s) {
    if (!s) return ST_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->idle) st_destroy_mesh(kv.second.mesh);
    delete s;
    return ST_OK;
}

st_status st_submit(st_server* s, const st_request* r, uint64_t* ticket) {
    if (!s || !r || !ticket || !r->gamma) return ST_ERR_ARG;
    auto job = std::make_shared<Job>();
    job->req = *r;
    job->gamma.assign(r->gamma, r->gamma + r->count);
    job->req.gamma = nullptr;
    job->footprint = st_footprint_bytes(&r->mesh, r->options.precision, r->options.restart > 0 ? r->options.restart : 30);
    job->nodes = r->mesh.n_t + 1LL;
    for (int q = 0; q < (r->mesh.ndim_space == 3 ? 3 : 2); ++q) job->nodes *= r->mesh.n[q] + 1LL;
    if (job->footprint <= 0 || job->footprint > s->desc.hbm_budget) return ST_ERR_BUSY;
    job->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) return ST_ERR_STATE;
        job->ticket = s->next_ticket++;
        s->jobs[job->ticket] = job;
        s->queue.push_back(job);
        *ticket = job->ticket;
    }
    s->cv_work.notify_all();
    return ST_OK;
}

st_status st_cancel(st_server* s, uint64_t ticket) {
    if (!s) return ST_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(ticket);
        if (it == s->jobs.end()) return ST_ERR_NOT_FOUND;
        std::shared_ptr<Job> job = it->second;
        if (job->done) return ST_ERR_STATE;  // finished: poll it instead
        bool queued = false;
        for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
            if (q->get() == job.get()) {
                s->queue.erase(q);
                queued = true;
                break;
            }
        if (!queued) return ST_ERR_BUSY;  // admitted and running on the device
        memset(&job->res, 0, sizeof(job->res));
        job->res.status = ST_ERR_CANCELLED;
        job->res.latency_s = now_s() - job->t_submit;
        job->res.queue_s = job->res.latency_s;
        job->done = true;
    }
    s->cv_done.notify_all();
    return ST_OK;
}

st_status st_poll(st_server* s, uint64_t ticket, st_result* out, double* grad, size_t count, int* done) {
    if (!s || !done) return ST_ERR_ARG;
    std::shared_ptr<Job> job;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(ticket);
        if (it == s->jobs.end()) return ST_ERR_NOT_FOUND;
        job = it->second;
        *done = job->done ? 1 : 0;
        if (!job->done) return ST_OK;
        if (grad && !job->grad.empty() && count != job->grad.size()) return ST_ERR_ARG;
        s->jobs.erase(it);
    }
    if (out) *out = job->res;
    if (grad && !job->grad.empty()) {
        memcpy(grad, job->grad.data(), count * sizeof(double));
    }
    return ST_OK;
}

}  // extern "C"
