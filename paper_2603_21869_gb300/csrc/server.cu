// Request loop over resident cases (continuous batching), written on the
// public C-ABI only: cases are created, batched, stepped and destroyed
// through fvm_create_case / fvm_batch_* / fvm_destroy_case.
//
// One scheduling round launches the steps of all resident cases together
// (one batch per precision, rebuilt when the set of cases changes); while
// they run, admits the queued requests that have arrived, first come first
// served, while their device bytes fit the budget (case creation on the host
// overlaps the device work); waits for the steps and retires the finished
// requests.  An admitted request joins the others at the next round, so their
// work overlaps on the device.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "fvm_internal.cuh"

namespace {

enum { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2 };

struct Request {
    int64_t id = 0;
    fvm_case_desc desc;
    std::vector<fvm_vent> vents;
    std::vector<fvm_box> boxes;
    int32_t nsteps = 0;
    int32_t done_steps = 0;
    int32_t vcycles = 0;
    int state = Q_QUEUED;
    fvm_status status = FVM_OK;
    double rel = 0.0;
    double t_arrive = 0.0, t_admit = 0.0, t_done = 0.0;
    int64_t bytes = 0;
    int64_t cells = 0;
    fvm_case* c = nullptr;
};

fvm_status fail(fvm_status st, const std::string& msg) {
    set_last_error(msg);
    return st;
}

}  // namespace

struct fvm_server {
    int64_t budget = 0;
    int32_t max_cases = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool keep = false;
    std::chrono::steady_clock::time_point t0;
    int64_t next_id = 1;
    std::deque<Request*> queue;      // by submission order
    std::vector<Request*> running;   // resident, in admission order
    std::map<int64_t, std::unique_ptr<Request>> all;
    std::map<int32_t, fvm_batch*> batches;   // precision -> batch of its running cases
    std::map<int32_t, std::vector<Request*>> members;
    bool dirty = false;
    int64_t used = 0;
    int64_t rounds = 0, rebuilds = 0, cell_steps = 0, done = 0;
    double t_admit = 0.0, t_rebuild = 0.0, t_step = 0.0;   // host seconds per phase
};

namespace {

double now_of(const fvm_server* s) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

void drop_batches(fvm_server* s) {
    for (auto& kv : s->batches) fvm_batch_destroy(kv.second);
    s->batches.clear();
    s->members.clear();
}

void free_case(fvm_server* s, Request* r) {
    if (r->c) {
        fvm_destroy_case(r->c);
        r->c = nullptr;
        s->used -= r->bytes;
    }
}

// group the running cases by precision and batch each group
fvm_status rebuild(fvm_server* s) {
    drop_batches(s);
    for (Request* r : s->running) s->members[r->desc.precision].push_back(r);
    for (auto& kv : s->members) {
        std::vector<fvm_case*> cs;
        for (Request* r : kv.second) cs.push_back(r->c);
        fvm_batch* b = nullptr;
        fvm_status st = fvm_batch_create(cs.data(), (int32_t)cs.size(), s->stream, &b);
        if (st != FVM_OK) {
            drop_batches(s);
            return st;
        }
        s->batches[kv.first] = b;
    }
    s->dirty = false;
    ++s->rebuilds;
    return FVM_OK;
}

void retire(fvm_server* s, Request* r, fvm_status st, double t) {
    r->state = Q_DONE;
    r->status = st;
    r->t_done = t;
    ++s->done;
    if (!s->keep || st != FVM_OK) free_case(s, r);
    s->dirty = true;
}

fvm_request_result result_of(const Request* r) {
    fvm_request_result o;
    memset(&o, 0, sizeof(o));
    o.id = r->id;
    o.status = r->status;
    o.steps = r->done_steps;
    o.cells = r->cells;
    o.device_bytes = r->bytes;
    o.vcycles_total = r->vcycles;
    o.rel_residual = r->rel;
    o.t_arrive = r->t_arrive;
    o.t_admit = r->t_admit;
    o.t_done = r->t_done;
    return o;
}

}  // namespace

extern "C" {

fvm_status fvm_server_create(int64_t budget_bytes, int32_t max_cases, void* stream, int32_t keep_results,
                             fvm_server** out) {
    if (!out) return fail(FVM_ERR_INVALID, "null output");
    if (budget_bytes <= 0 || max_cases < 0) return fail(FVM_ERR_INVALID, "budget must be > 0, max_cases >= 0");
    fvm_server* s = new fvm_server;
    s->budget = budget_bytes;
    s->max_cases = max_cases;
    s->keep = keep_results != 0;
    s->t0 = std::chrono::steady_clock::now();
    if (stream) s->stream = (cudaStream_t)stream;
    else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return fail(FVM_ERR_CUDA, "cudaStreamCreate");
        }
        s->own_stream = true;
    }
    set_last_error("");
    *out = s;
    return FVM_OK;
}

double fvm_server_now(const fvm_server* s) { return s ? now_of(s) : 0.0; }

fvm_status fvm_server_submit(fvm_server* s, const fvm_case_desc* desc, int32_t nsteps, double t_arrive,
                             int64_t* id_out) {
    if (!s || !desc) return fail(FVM_ERR_INVALID, "null server or descriptor");
    if (nsteps < 0) return fail(FVM_ERR_INVALID, "nsteps < 0");
    const int64_t bytes = (int64_t)fvm_case_bytes(desc);
    if (bytes <= 0) return FVM_ERR_INVALID;   // fvm_case_bytes left the reason
    if (bytes > s->budget) return fail(FVM_ERR_BUDGET, "the case alone needs more than the device budget");
    std::unique_ptr<Request> r(new Request);
    r->id = s->next_id++;
    r->desc = *desc;
    r->vents.assign(desc->vents, desc->vents + desc->n_vents);
    r->boxes.assign(desc->boxes, desc->boxes + desc->n_boxes);
    r->desc.vents = r->vents.data();
    r->desc.boxes = r->boxes.data();
    r->desc.stream = nullptr;   // a stream of the case's own: its creation runs beside the batch in flight
    r->nsteps = nsteps;
    r->t_arrive = t_arrive;
    r->bytes = bytes;
    r->cells = (int64_t)desc->nx * desc->ny * desc->nz;
    if (id_out) *id_out = r->id;
    s->queue.push_back(r.get());
    s->all[r->id] = std::move(r);
    set_last_error("");
    return FVM_OK;
}

fvm_status fvm_server_poll(fvm_server* s, int32_t chunk, fvm_request_result* done, int32_t cap, int32_t* n_done) {
    if (!s) return fail(FVM_ERR_INVALID, "null server");
    if (chunk < 1) return fail(FVM_ERR_INVALID, "chunk < 1");
    if (n_done) *n_done = 0;
    int32_t nd = 0;
    auto report = [&](const Request* r) {
        if (done && nd < cap) done[nd] = result_of(r);
        ++nd;
    };
    // 1. this round's steps for the resident cases are launched first, so that admitting
    //    new requests (host-side case creation) overlaps them on the device
    const double t0 = now_of(s);
    int32_t steps = 0;
    if (!s->running.empty()) {
        if (s->dirty) {
            fvm_status st = rebuild(s);
            if (st != FVM_OK) return st;
        }
        steps = chunk;
        for (Request* r : s->running) steps = std::min(steps, r->nsteps - r->done_steps);
        for (auto& kv : s->batches) {
            fvm_status st = fvm_batch_launch(kv.second, steps);
            if (st != FVM_OK) {
                for (auto& kw : s->batches) fvm_batch_wait(kw.second, nullptr);   // (refuses those not launched)
                return st;
            }
        }
    }
    const double t1 = now_of(s);
    s->t_rebuild += t1 - t0;
    // 2. admission, first come first served; admitted cases join the next round
    std::vector<Request*> joined;
    while (!s->queue.empty()) {
        Request* r = s->queue.front();
        if (r->t_arrive > t1) break;
        if (s->used + r->bytes > s->budget) break;
        if (s->max_cases > 0 && (int32_t)(s->running.size() + joined.size()) >= s->max_cases) break;
        s->queue.pop_front();
        fvm_status st = fvm_create_case(&r->desc, &r->c);
        if (st == FVM_ERR_OOM) {   // the device holds less than the budget says: retry later
            s->queue.push_front(r);
            break;
        }
        r->t_admit = now_of(s);
        if (st != FVM_OK) {
            retire(s, r, st, r->t_admit);
            report(r);
            continue;
        }
        s->used += r->bytes;
        r->state = Q_RUNNING;
        if (r->nsteps == 0) {
            retire(s, r, FVM_OK, r->t_admit);
            report(r);
            continue;
        }
        joined.push_back(r);
    }
    const double t2 = now_of(s);
    s->t_admit += t2 - t1;
    // 3. the round's results
    if (steps > 0) {
        for (auto& kv : s->batches) {
            std::vector<Request*>& mem = s->members[kv.first];
            std::vector<fvm_step_stats> stats(mem.size());
            const fvm_status st = fvm_batch_wait(kv.second, stats.data());
            if (st != FVM_OK && st != FVM_ERR_NOT_CONVERGED && st != FVM_ERR_DIVERGED) return st;
            for (size_t q = 0; q < mem.size(); ++q) {
                Request* r = mem[q];
                r->done_steps += stats[q].steps;
                r->vcycles += stats[q].vcycles_total;
                r->rel = stats[q].rel_residual;
                s->cell_steps += r->cells * (int64_t)stats[q].steps;
                // a case whose own solve diverged ends with that status; a case that hit the
                // V-cycle cap keeps running (its result carries the residual)
                if (st == FVM_ERR_DIVERGED && !(stats[q].rel_residual == stats[q].rel_residual))
                    retire(s, r, FVM_ERR_DIVERGED, now_of(s));
            }
        }
        ++s->rounds;
    }
    // 4. retirement
    const double t_end = now_of(s);
    s->t_step += t_end - t2;
    for (size_t q = 0; q < s->running.size();) {
        Request* r = s->running[q];
        if (r->state != Q_DONE && r->done_steps >= r->nsteps) retire(s, r, FVM_OK, t_end);
        if (r->state == Q_DONE) {
            report(r);
            s->running.erase(s->running.begin() + q);
        } else {
            ++q;
        }
    }
    // 5. the admitted cases become resident
    for (Request* r : joined) s->running.push_back(r);
    if (!joined.empty()) s->dirty = true;
    if (s->running.empty()) drop_batches(s);
    if (n_done) *n_done = nd;
    set_last_error("");
    return FVM_OK;
}

fvm_status fvm_server_get_info(const fvm_server* s, fvm_server_info* out) {
    if (!s || !out) return fail(FVM_ERR_INVALID, "null server or output");
    fvm_server_info o;
    memset(&o, 0, sizeof(o));
    o.queued = (int64_t)s->queue.size();
    o.running = (int64_t)s->running.size();
    o.done = s->done;
    o.bytes_in_use = s->used;
    o.rounds = s->rounds;
    o.batch_rebuilds = s->rebuilds;
    o.cell_steps = s->cell_steps;
    o.t_admit_s = s->t_admit;
    o.t_rebuild_s = s->t_rebuild;
    o.t_step_s = s->t_step;
    *out = o;
    return FVM_OK;
}

fvm_status fvm_server_read_fields(fvm_server* s, int64_t id, unsigned field_mask, double* host_out, size_t n) {
    if (!s) return fail(FVM_ERR_INVALID, "null server");
    auto it = s->all.find(id);
    if (it == s->all.end()) return fail(FVM_ERR_INVALID, "unknown request");
    Request* r = it->second.get();
    if (r->state != Q_DONE || !r->c) return fail(FVM_ERR_INVALID, "the request has no kept result");
    return fvm_read_fields(r->c, field_mask, host_out, n);
}

fvm_status fvm_server_release(fvm_server* s, int64_t id) {
    if (!s) return fail(FVM_ERR_INVALID, "null server");
    auto it = s->all.find(id);
    if (it == s->all.end()) return fail(FVM_ERR_INVALID, "unknown request");
    Request* r = it->second.get();
    if (r->state != Q_DONE) return fail(FVM_ERR_INVALID, "the request has not finished");
    free_case(s, r);
    s->all.erase(it);
    return FVM_OK;
}

void fvm_server_destroy(fvm_server* s) {
    if (!s) return;
    drop_batches(s);
    for (auto& kv : s->all) free_case(s, kv.second.get());
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
