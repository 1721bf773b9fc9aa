// Request loop for steady solves with continuous batching (no counterpart in the paper; the
// solve itself is the FAS V-cycle of Sec. 2.3 iterated to the drop of Sec. 4).
//
// Every admitted request owns a context: its stream, state, Jacobian blocks and Krylov
// arrays stay on the device until it ends.  Requests wait in arrival order; the head is
// admitted when a slot is free and its footprint fits in what the memory budget has left.
// Each active solve keeps one V-cycle in flight.  emg_server_step only polls events and,
// for every solve whose residual check has arrived, decides (converged / limit / failure)
// and enqueues its next cycle, so the cycles of different solves overlap on the device.
// A solve's arithmetic depends on nothing outside its context (fixed-order reductions,
// no atomics), so its result is bitwise the same alone and in the mix.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <memory>
#include <unordered_map>
#include <vector>

#include "common.cuh"

using namespace emg;

namespace {

struct Request {
    int64_t id = 0;
    int dim = 0;
    int64_t n_nodes = 0, n_elems = 0;
    std::vector<double> xyz, wn;
    std::vector<int64_t> en;
    std::vector<int32_t> fbc;
    emg_params prm{};
    std::vector<double> U0;
    int64_t est = 0;
    double t_submit = 0.0, t_admit = -1.0, t_done = -1.0;
    emg_ctx* c = nullptr;
    cudaEvent_t ev = nullptr;
    double r0 = -1.0, res = 0.0, best = 0.0;
    int64_t cycles = 0, best_at = 0;
    int64_t held = 0;  // bytes charged to the budget
    emg_status status = EMG_OK;
    bool cancel = false;  // withdrawn while active: end at the next residual check
};

int64_t modes(int dim, int p) { return dim == 2 ? (p + 1) * (p + 2) / 2 : (p + 1) * (p + 2) * (p + 3) / 6; }

emg_status estimate(const emg_mesh_desc* m, const emg_params* prm, int64_t* bytes) {
    if (!m || !prm || !bytes || (m->dim != 2 && m->dim != 3) || m->n_elems <= 0 || !m->face_bc ||
        prm->p_max < 0 || prm->p_max > MAX_P || prm->krylov_m < 1 || prm->krylov_m > MAX_KRYLOV)
        return EMG_ERR_ARG;
    const int nf = 2 * m->dim;
    int64_t nb = 0;
    for (int64_t k = 0; k < m->n_elems * nf; ++k) nb += m->face_bc[k] >= 0 ? 1 : 0;
    if ((m->n_elems * nf - nb) % 2 != 0) return EMG_ERR_ARG;
    const int64_t F_int = (m->n_elems * nf - nb) / 2;
    const bool rot = prm->omega[0] != 0.0 || prm->omega[1] != 0.0 || prm->omega[2] != 0.0;
    *bytes = estimate_bytes(m->dim, m->n_elems, F_int + nb, F_int, prm->p_max, prm->krylov_m, prm->prec, rot);
    return EMG_OK;
}

}  // namespace

struct emg_server {
    emg_server_params prm{};
    std::string err;
    std::chrono::steady_clock::time_point t0;
    int64_t next_id = 0;
    int64_t mem_used = 0;
    std::deque<std::unique_ptr<Request>> queue;
    std::vector<std::unique_ptr<Request>> active;
    std::deque<emg_request_result> done;
    std::unordered_map<int64_t, std::vector<double>> states;

    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }

    // Residual check of the current cycle: R_pmax(v), the norm and CFL_n on the device,
    // then the scalars to page-locked host memory and an event behind them.
    emg_status enqueue_check(Request* r) {
        emg_ctx* c = r->c;
        emg_status st = vcycle_entry(c);
        if (st != EMG_OK) return st;
        EMG_CUDA_TRY(c, cudaMemcpyAsync(c->sc_host, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
        EMG_CUDA_TRY(c, cudaEventRecord(r->ev, c->stream));
        return EMG_OK;
    }

    void finish(std::unique_ptr<Request>& r, emg_status st, const std::string& msg) {
        r->status = st;
        r->t_done = now();
        if (r->c) {
            if (prm.keep_state && st == EMG_OK) {
                const int64_t n = r->n_elems * 5 * modes(r->dim, r->prm.p_max);
                std::vector<double> U((size_t)n);
                if (emg_get_state(r->c, U.data(), 0) == EMG_OK) states[r->id] = std::move(U);
            }
            emg_destroy(r->c);
            r->c = nullptr;
        }
        if (r->ev) cudaEventDestroy(r->ev);
        r->ev = nullptr;
        mem_used -= r->held;
        r->held = 0;
        emg_request_result out{};
        out.id = r->id;
        out.status = st;
        out.cycles = r->cycles;
        out.res0 = r->r0;
        out.res_final = r->res;
        out.t_submit = r->t_submit;
        out.t_admit = r->t_admit;
        out.t_done = r->t_done;
        out.device_bytes = r->est;
        done.push_back(out);
        if (!msg.empty()) err = "request " + std::to_string(r->id) + ": " + msg;
    }

    // Create the context of the head request and enqueue its first residual check.
    void admit(std::unique_ptr<Request>& r) {
        r->t_admit = now();
        emg_mesh_desc d{};
        d.dim = r->dim;
        d.n_nodes = r->n_nodes;
        d.xyz = r->xyz.data();
        d.n_elems = r->n_elems;
        d.elem_nodes = r->en.data();
        d.face_bc = r->fbc.data();
        d.wall_normal = r->wn.empty() ? nullptr : r->wn.data();
        emg_params p = r->prm;
        p.cuda_stream = nullptr;  // every solve gets a stream of its own
        p.coop_krylov = 0;        // solves share the device: no kernel may wait for co-resident blocks
        emg_status st = emg_create_mesh(&d, &p, &r->c);
        if (st == EMG_OK && !r->U0.empty()) st = emg_set_state(r->c, r->U0.data(), 0);
        if (st == EMG_OK && cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) st = EMG_ERR_CUDA;
        r->held = r->c ? std::max(r->est, r->c->bytes) : 0;
        mem_used += r->held;
        if (st == EMG_OK) st = enqueue_check(r.get());
        if (st != EMG_OK) {
            const std::string msg = r->c ? r->c->err : std::string("context creation failed");
            finish(r, st, msg);
        }
    }

    // The residual check of an active solve has arrived: end it or enqueue the next cycle.
    // Returns true when the solve ended.
    bool advance(std::unique_ptr<Request>& r) {
        emg_ctx* c = r->c;
        if (r->cancel) {
            finish(r, EMG_CANCELLED, "");
            return true;
        }
        emg_status st = check_flags(c);
        if (st != EMG_OK) {
            finish(r, st, c->err);
            return true;
        }
        r->res = c->sc_host->res;
        if (r->r0 < 0.0) r->r0 = r->best = r->res;
        if (r->res < r->best) {
            r->best = r->res;
            r->best_at = r->cycles;
        }
        if (r->res <= prm.drop * r->r0) {
            finish(r, EMG_OK, "");
            return true;
        }
        if (r->cycles >= prm.max_cycles) {
            finish(r, EMG_ERR_NOT_CONVERGED, "max_cycles reached");
            return true;
        }
        if (prm.stall_cycles > 0 && r->cycles - r->best_at >= prm.stall_cycles) {
            finish(r, EMG_ERR_NOT_CONVERGED, "no new residual minimum in stall_cycles cycles");
            return true;
        }
        st = run_body(c);
        if (st == EMG_OK) {
            c->cycle_n += 1;
            r->cycles += 1;
            st = enqueue_check(r.get());
        }
        if (st != EMG_OK) {
            finish(r, st, c->err);
            return true;
        }
        return false;
    }
};

extern "C" {

emg_status emg_estimate_device_bytes(const emg_mesh_desc* mesh, const emg_params* params, int64_t* bytes) {
    return estimate(mesh, params, bytes);
}

emg_status emg_server_create(const emg_server_params* params, emg_server** out) {
    if (!out) return EMG_ERR_ARG;
    *out = nullptr;
    if (!params || params->max_active < 1 || !(params->drop > 0.0) || params->max_cycles < 0 || params->stall_cycles < 0)
        return EMG_ERR_ARG;
    emg_server* s = new (std::nothrow) emg_server();
    if (!s) return EMG_ERR_OOM;
    s->prm = *params;
    if (s->prm.mem_budget <= 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            delete s;
            return EMG_ERR_CUDA;
        }
        s->prm.mem_budget = (int64_t)(0.9 * (double)fr);
    }
    s->t0 = std::chrono::steady_clock::now();
    *out = s;
    return EMG_OK;
}

emg_status emg_server_destroy(emg_server* s) {
    if (!s) return EMG_OK;
    for (auto& r : s->active) {
        if (r->c) emg_destroy(r->c);
        if (r->ev) cudaEventDestroy(r->ev);
    }
    delete s;
    return EMG_OK;
}

const char* emg_server_last_error(const emg_server* s) { return s ? s->err.c_str() : "null server"; }

double emg_server_clock(const emg_server* s) { return s ? s->now() : 0.0; }

emg_status emg_server_submit(emg_server* s, const emg_mesh_desc* m, const emg_params* prm, const double* U0,
                             int64_t* id) {
    if (!s || !m || !prm || !m->xyz || !m->elem_nodes || !m->face_bc || m->n_nodes <= 0) return EMG_ERR_ARG;
    auto r = std::make_unique<Request>();
    emg_status st = estimate(m, prm, &r->est);
    if (st != EMG_OK) {
        s->err = "submit: invalid mesh or parameters";
        return st;
    }
    const int nn = 1 << m->dim, nf = 2 * m->dim;
    r->id = s->next_id++;
    r->dim = m->dim;
    r->n_nodes = m->n_nodes;
    r->n_elems = m->n_elems;
    r->xyz.assign(m->xyz, m->xyz + m->dim * m->n_nodes);
    if (m->wall_normal) r->wn.assign(m->wall_normal, m->wall_normal + m->dim * m->n_nodes);
    r->en.assign(m->elem_nodes, m->elem_nodes + m->n_elems * nn);
    r->fbc.assign(m->face_bc, m->face_bc + m->n_elems * nf);
    r->prm = *prm;
    if (U0) r->U0.assign(U0, U0 + m->n_elems * 5 * modes(m->dim, prm->p_max));
    r->t_submit = s->now();
    if (id) *id = r->id;
    s->queue.push_back(std::move(r));
    return EMG_OK;
}

emg_status emg_server_step(emg_server* s, int32_t* n_active, int32_t* n_queued) {
    if (!s) return EMG_ERR_ARG;
    // 1. poll every active solve; a finished one frees its slot and its memory
    for (size_t k = 0; k < s->active.size();) {
        auto& r = s->active[k];
        const cudaError_t q = cudaEventQuery(r->ev);
        bool ended = false;
        if (q == cudaSuccess) {
            ended = s->advance(r);
        } else if (q != cudaErrorNotReady) {
            s->finish(r, EMG_ERR_CUDA, cudaGetErrorString(q));
            ended = true;
        }
        if (ended) {
            s->active.erase(s->active.begin() + (ptrdiff_t)k);
        } else {
            ++k;
        }
    }
    // 2. admit in arrival order while a slot and the memory budget allow
    while (!s->queue.empty() && (int)s->active.size() < s->prm.max_active) {
        auto& h = s->queue.front();
        if (h->est > s->prm.mem_budget) {
            h->t_admit = s->now();
            s->finish(h, EMG_ERR_OOM, "footprint exceeds the server's memory budget");
            s->queue.pop_front();
            continue;
        }
        if (s->mem_used + h->est > s->prm.mem_budget) break;
        std::unique_ptr<Request> r = std::move(h);
        s->queue.pop_front();
        s->admit(r);
        if (r->status == EMG_OK && r->t_done < 0.0) s->active.push_back(std::move(r));
    }
    if (n_active) *n_active = (int32_t)s->active.size();
    if (n_queued) *n_queued = (int32_t)s->queue.size();
    return EMG_OK;
}

emg_status emg_server_results(emg_server* s, emg_request_result* out, int32_t capacity, int32_t* n_out) {
    if (!s || !n_out || (capacity > 0 && !out)) return EMG_ERR_ARG;
    int32_t n = 0;
    while (n < capacity && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    *n_out = n;
    return EMG_OK;
}

emg_status emg_server_cancel(emg_server* s, int64_t id) {
    if (!s) return EMG_ERR_ARG;
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        if ((*it)->id == id) {
            (*it)->t_admit = s->now();
            s->finish(*it, EMG_CANCELLED, "");
            s->queue.erase(it);
            return EMG_OK;
        }
    }
    for (auto& r : s->active) {
        if (r->id == id) {
            r->cancel = true;   // the request ends at its next residual check (emg_server_step)
            return EMG_OK;
        }
    }
    s->err = "cancel: request " + std::to_string(id) + " is not queued or active";
    return EMG_ERR_ARG;
}

emg_status emg_server_take_state(emg_server* s, int64_t id, double* U, int64_t n) {
    if (!s || !U) return EMG_ERR_ARG;
    auto it = s->states.find(id);
    if (it == s->states.end()) {
        s->err = "no kept state for request " + std::to_string(id);
        return EMG_ERR_ARG;
    }
    if ((int64_t)it->second.size() != n) {
        s->err = "state size mismatch";
        return EMG_ERR_ARG;
    }
    std::memcpy(U, it->second.data(), (size_t)n * sizeof(double));
    s->states.erase(it);
    return EMG_OK;
}

}  // extern "C"
