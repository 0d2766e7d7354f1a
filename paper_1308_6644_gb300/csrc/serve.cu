// Request loop with continuous batching (declared in include/nuasm.h).
//
// Host side: one FIFO queue, `slots` worker threads each owning a CUDA
// stream, a budget of device bytes, and a table of resident point sets.  A
// worker admits the queue head when the budget has room (evicting idle
// resident sets least recently used first), then runs the request on its own
// stream: bins the points if the set is not resident, builds the request's
// FP64 transfer-function tables, copies the input in, launches the solve on
// a view of the resident plan that points at the request's tables and
// workspace, copies the output back and waits for its stream.  Slots run
// concurrently, so one request's copies and kernels overlap another's.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "nuasm_internal.h"

using namespace nuasm;
using Clock = std::chrono::steady_clock;

namespace {

constexpr int kMaxSlots = 32;
constexpr int64_t kDefaultBudget = int64_t(150) * 1000 * 1000 * 1000;

nuasm_status status_of(cudaError_t e) {
    if (e == cudaSuccess) return NUASM_OK;
    return e == cudaErrorMemoryAllocation ? NUASM_ENOMEM : NUASM_ECUDA;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Identity of a resident point set: the caller's key plus everything the bins depend on.
struct SetKey {
    uint64_t id;
    int n, n_pad, prec, kernel, tile;
    double pitch, tol;
    bool operator==(const SetKey& o) const {
        return id == o.id && n == o.n && n_pad == o.n_pad && prec == o.prec && kernel == o.kernel &&
               tile == o.tile && pitch == o.pitch && tol == o.tol;
    }
};

SetKey key_of(uint64_t id, const nuasm_params_t& rp) {
    return SetKey{id, rp.n, rp.n_pad, rp.prec, rp.kernel, rp.tile, rp.pitch, rp.tol};
}

struct PointSet {
    SetKey key{};
    bool keep = true;                  // points_id != 0
    nuasm_plan_s* plan = nullptr;      // bins and twiddles, no workspace
    std::vector<double> phihat;        // kernel transform at k/G (geometry only)
    int64_t bytes = 0;                 // budget charge (estimate while building)
    int refs = 0;
    enum State { kBuilding, kReady, kFailed } state = kBuilding;
    nuasm_status fail = NUASM_OK;
    uint64_t last_use = 0;
};

struct Job {
    int64_t ticket = 0;
    nuasm_request_t r{};
    nuasm_params_t rp{};
    Geometry g{};
    int64_t bytes = 0;                 // tables + workspace + input/output copies
    Clock::time_point submit;
};

struct Done {
    bool done = false;
    nuasm_request_result_t res{};
};

int64_t elems_in(const Job& j) { return j.r.type == 1 ? j.r.m : int64_t(j.g.n) * j.g.n; }
int64_t elems_out(const Job& j) { return j.r.type == 1 ? int64_t(j.g.n) * j.g.n : j.r.m; }

int64_t job_bytes(const Job& j, bool in_dev, bool out_dev) {
    const size_t eb = j.rp.prec == NUASM_PREC_F64 ? 16 : 8;
    size_t b = align256(table_bytes(j.g, j.rp.prec == NUASM_PREC_F64, false));
    b += align256(ws_win_elems(j.g) * eb) + align256(ws_bufA_elems(j.g) * eb) + align256(ws_bufB_elems(j.g) * eb);
    if (!in_dev) b += align256(size_t(elems_in(j)) * eb);
    if (!out_dev) b += align256(size_t(elems_out(j)) * eb);
    return int64_t(b);
}

// Rough device bytes of a resident set before it is built (corrected after).
int64_t set_bytes_estimate(const Job& j) {
    const bool f64 = j.rp.prec == NUASM_PREC_F64;
    return int64_t(table_bytes(j.g, f64, true) + record_bytes(f64) * size_t(j.r.m) * 2 +
                   sizeof(int) * (2 * size_t(j.g.ntiles) + 2) + (64 << 10));
}

}  // namespace

struct nuasm_server_s {
    nuasm_server_config_t cfg{};
    cudaMemPool_t pool = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job> queue;
    std::unordered_map<int64_t, Done> done;
    std::vector<std::unique_ptr<PointSet>> sets;
    std::vector<std::thread> workers;
    bool stopping = false;
    int64_t next_ticket = 1;
    int64_t used = 0, peak = 0, resident = 0;
    int inflight = 0;                  // admitted requests not yet completed
    uint64_t tick = 0;
    // statistics
    int64_t submitted = 0, completed = 0, failed = 0, points = 0, built = 0, reused = 0, evictions = 0;
    std::vector<double> lat;
    bool have_first = false;
    Clock::time_point first_submit, last_done;
};

namespace {

using Server = nuasm_server_s;

// Per-slot resources, owned by the worker thread.
struct Slot {
    cudaStream_t st = nullptr;
    int* d_err = nullptr;
    int* h_err = nullptr;
    char* h_tab = nullptr;
    size_t h_tab_bytes = 0;
    ~Slot() {
        xstream_destroy(st);
        xfree(d_err);
        xfree_host(h_err);
        xfree_host(h_tab);
    }
};

PointSet* find_set(Server& S, const SetKey& k) {
    if (k.id == 0) return nullptr;
    for (auto& p : S.sets)
        if (p->keep && p->key == k) return p.get();
    return nullptr;
}

// Remove a set from the table (caller holds the lock); its plan is returned
// for release outside the lock.
nuasm_plan_s* drop_set(Server& S, PointSet* ps) {
    nuasm_plan_s* plan = ps->plan;
    S.used -= ps->bytes;
    if (ps->keep) S.resident -= ps->bytes;
    for (auto it = S.sets.begin(); it != S.sets.end(); ++it)
        if (it->get() == ps) {
            S.sets.erase(it);
            break;
        }
    return plan;
}

// Admit the queue head if the budget allows (lock held).  On success the
// job's bytes (and a new set's estimate) are charged and the set is referenced.
bool try_admit(Server& S, const Job& j, PointSet** out, bool* build, std::vector<nuasm_plan_s*>* victims) {
    const SetKey k = key_of(j.r.points_id, j.rp);
    PointSet* ps = find_set(S, k);
    const int64_t set_need = ps ? 0 : set_bytes_estimate(j);
    const int64_t budget = S.cfg.hbm_budget;
    while (S.used + j.bytes + set_need > budget) {
        PointSet* victim = nullptr;
        for (auto& p : S.sets)
            if (p.get() != ps && p->refs == 0 && p->state != PointSet::kBuilding &&
                (!victim || p->last_use < victim->last_use))
                victim = p.get();
        if (!victim) {
            // with nothing else running nothing will free up: admit over the
            // budget rather than wait forever (the set's estimate was low)
            if (S.inflight == 0) break;
            return false;
        }
        victims->push_back(drop_set(S, victim));
        S.evictions += 1;
    }
    if (!ps) {
        auto fresh = std::make_unique<PointSet>();
        fresh->key = k;
        fresh->keep = j.r.points_id != 0;
        fresh->bytes = set_need;
        ps = fresh.get();
        S.sets.push_back(std::move(fresh));
        S.used += set_need;
        if (ps->keep) S.resident += set_need;
        *build = true;
    } else {
        *build = false;
    }
    ps->refs += 1;
    S.inflight += 1;
    S.used += j.bytes;
    S.peak = std::max(S.peak, S.used);
    *out = ps;
    return true;
}

// Bin the job's points into a plan without workspace and publish the set.
nuasm_status build_set(Server& S, Slot& sl, const Job& j, PointSet* ps) {
    const int64_t m = j.r.m;
    const double* dx = j.r.x;
    const double* dy = j.r.y;
    char* tmp = nullptr;
    cudaError_t e = cudaSuccess;
    if (m > 0 && (!device_accessible(j.r.x) || !device_accessible(j.r.y))) {
        e = xmalloc_pool(reinterpret_cast<void**>(&tmp), sizeof(double) * 2 * size_t(m), S.pool, sl.st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(tmp, j.r.x, sizeof(double) * size_t(m), cudaMemcpyDefault, sl.st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(tmp + sizeof(double) * size_t(m), j.r.y, sizeof(double) * size_t(m),
                                cudaMemcpyDefault, sl.st);
        dx = reinterpret_cast<const double*>(tmp);
        dy = reinterpret_cast<const double*>(tmp) + m;
    }
    nuasm_plan_s* P = nullptr;
    nuasm_status s = e == cudaSuccess ? plan_create(&P, &j.rp, m, dx, dy, nullptr, sl.st, false) : status_of(e);
    if (tmp) {
        xfree_async(tmp, sl.st);
        cudaStreamSynchronize(sl.st);
    }
    std::vector<double> ph;
    if (s == NUASM_OK) {
        ph.resize(j.g.np);
        phihat_table(j.g, ph.data());
    }
    std::lock_guard<std::mutex> lk(S.mu);
    if (s == NUASM_OK) {
        ps->plan = P;
        ps->phihat.swap(ph);
        const int64_t actual = P->device_bytes;
        S.used += actual - ps->bytes;
        if (ps->keep) S.resident += actual - ps->bytes;
        ps->bytes = actual;
        S.peak = std::max(S.peak, S.used);
        ps->state = PointSet::kReady;
        S.built += 1;
    } else {
        ps->state = PointSet::kFailed;
        ps->fail = s;
    }
    S.cv_done.notify_all();
    return s;
}

// Run one admitted job on the slot's stream and wait for it.
nuasm_status run_job(Server& S, Slot& sl, const Job& j, PointSet* ps, bool build, bool* reused) {
    *reused = false;
    if (build) {
        const nuasm_status s = build_set(S, sl, j, ps);
        if (s != NUASM_OK) return s;
    } else {
        std::unique_lock<std::mutex> lk(S.mu);
        S.cv_done.wait(lk, [&] { return ps->state != PointSet::kBuilding; });
        if (ps->state == PointSet::kFailed) return ps->fail;
        *reused = true;
    }
    const nuasm_plan_s* B = ps->plan;
    if (B->m != j.r.m) return NUASM_EINVAL;   // same key, different point count
    const bool f64 = j.rp.prec == NUASM_PREC_F64;
    const size_t eb = f64 ? 16 : 8;
    const Geometry& g = j.g;

    // the request's transfer-function tables (FP64 on the host, packed in the plan precision)
    HostTables ht{};
    build_tables(j.rp, g, &ht, ps->phihat.data(), false);
    const size_t tb = table_bytes(g, f64, false);
    if (sl.h_tab_bytes < tb) {
        xfree_host(sl.h_tab);
        sl.h_tab = nullptr;
        sl.h_tab_bytes = 0;
        if (xmalloc_host(reinterpret_cast<void**>(&sl.h_tab), tb, cudaHostAllocDefault) != cudaSuccess) {
            free_tables(&ht);
            cudaGetLastError();
            return NUASM_ENOMEM;
        }
        sl.h_tab_bytes = tb;
    }
    pack_tables(ht, g, f64, false, sl.h_tab);
    const double rc = ht.rc, rmax = ht.rmax;
    free_tables(&ht);

    // one pool allocation: tables | window | bufA | bufB | input copy | output copy
    const int64_t ni = elems_in(j), no = elems_out(j);
    const bool in_dev = ni == 0 || device_accessible(j.r.in);
    const bool out_dev = no == 0 || device_accessible(j.r.out);
    const size_t sz[6] = {align256(tb), align256(ws_win_elems(g) * eb), align256(ws_bufA_elems(g) * eb),
                          align256(ws_bufB_elems(g) * eb), in_dev ? 0 : align256(size_t(ni) * eb),
                          out_dev ? 0 : align256(size_t(no) * eb)};
    size_t total = 0;
    for (size_t v : sz) total += v;
    char* base = nullptr;
    cudaError_t e = xmalloc_pool(reinterpret_cast<void**>(&base), total, S.pool, sl.st);
    if (e != cudaSuccess) return status_of(e);
    char* part[6];
    size_t off = 0;
    for (int i = 0; i < 6; ++i) {
        part[i] = base + off;
        off += sz[i];
    }
    const int np = g.np;
    nuasm_plan_s view = *B;
    view.p = j.rp;
    view.g = g;
    view.rc = rc;
    view.nonsep_mode = choose_nonsep_mode(j.rp, rmax);
    view.d.tables = part[0];
    view.d.t1x = part[0];
    view.d.t1y = part[0] + np * eb;
    view.d.t2x = part[0] + 2 * np * eb;
    view.d.t2y = part[0] + 3 * np * eb;
    view.d.t3x = part[0] + 4 * np * eb;
    view.d.t3y = part[0] + 5 * np * eb;
    view.d.s = part[0] + 6 * np * eb;
    view.d.tw = B->d.tw;
    view.d.tw_df = B->d.tw_df;
    view.d.etab = nullptr;   // one solve per table: E is evaluated per mode
    view.d.etab2 = nullptr;
    view.d.win = part[1];
    view.d.bufA = part[2];
    view.d.bufB = part[3];
    view.d.stage_in = view.d.stage_out = nullptr;
    view.d.err = sl.d_err;
    view.d.h_err = nullptr;   // the slot's word is device memory, read back below
    view.prof = false;
    view.prof_state = nullptr;
    const void* din = in_dev ? j.r.in : part[4];
    void* dout = out_dev ? j.r.out : part[5];

    e = cudaMemcpyAsync(part[0], sl.h_tab, tb, cudaMemcpyHostToDevice, sl.st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sl.d_err, 0, sizeof(int), sl.st);
    if (e == cudaSuccess && !in_dev)
        e = cudaMemcpyAsync(part[4], j.r.in, size_t(ni) * eb, cudaMemcpyHostToDevice, sl.st);
    if (e == cudaSuccess) e = j.r.type == 1 ? chain_type1(&view, din, dout, sl.st) : chain_type2(&view, din, dout, sl.st);
    if (e == cudaSuccess && !out_dev)
        e = cudaMemcpyAsync(j.r.out, part[5], size_t(no) * eb, cudaMemcpyDeviceToHost, sl.st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_err, sl.d_err, sizeof(int), cudaMemcpyDeviceToHost, sl.st);
    xfree_async(base, sl.st);
    const cudaError_t es = cudaStreamSynchronize(sl.st);
    if (e == cudaSuccess) e = es;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return status_of(e);
    }
    return (*sl.h_err & 2) ? NUASM_ETIMEOUT : NUASM_OK;
}

void worker_main(Server* S) {
    Slot sl;
    // a slot that cannot get its resources fails every request it takes
    cudaError_t se = cudaSetDevice(S->cfg.device);
    if (se == cudaSuccess) se = xstream_create(&sl.st);
    if (se == cudaSuccess) se = xmalloc(reinterpret_cast<void**>(&sl.d_err), sizeof(int));
    if (se == cudaSuccess) se = xmalloc_host(reinterpret_cast<void**>(&sl.h_err), sizeof(int), cudaHostAllocDefault);
    const bool ok = se == cudaSuccess;
    const nuasm_status slot_status = status_of(se);
    if (!ok) cudaGetLastError();
    for (;;) {
        Job j;
        PointSet* ps = nullptr;
        bool build = false;
        std::vector<nuasm_plan_s*> victims;
        Clock::time_point admitted;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                if (S->queue.empty()) {
                    if (S->stopping) return;
                    S->cv_work.wait(lk);
                    continue;
                }
                if (try_admit(*S, S->queue.front(), &ps, &build, &victims)) {
                    j = S->queue.front();
                    S->queue.pop_front();
                    break;
                }
                S->cv_work.wait(lk);   // room appears when a running request completes
            }
            admitted = Clock::now();
        }
        for (nuasm_plan_s* v : victims) plan_release(v);
        bool reused = false;
        const nuasm_status s = ok ? run_job(*S, sl, j, ps, build, &reused) : slot_status;
        const Clock::time_point t_done = Clock::now();
        nuasm_plan_s* drop = nullptr;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->used -= j.bytes;
            S->inflight -= 1;
            ps->refs -= 1;
            ps->last_use = ++S->tick;
            if (ps->refs == 0 && (!ps->keep || ps->state == PointSet::kFailed)) drop = drop_set(*S, ps);
            Done& d = S->done[j.ticket];
            d.done = true;
            d.res.status = s;
            d.res.reused_points = reused ? 1 : 0;
            d.res.latency_ms = std::chrono::duration<double, std::milli>(t_done - j.submit).count();
            d.res.queue_ms = std::chrono::duration<double, std::milli>(admitted - j.submit).count();
            if (s == NUASM_OK) {
                S->completed += 1;
                S->points += j.r.m;
                S->lat.push_back(d.res.latency_ms);
                if (reused) S->reused += 1;
            } else {
                S->failed += 1;
            }
            S->last_done = t_done;
            S->cv_done.notify_all();
            S->cv_work.notify_all();
        }
        if (drop) plan_release(drop);
    }
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    size_t k = size_t(q * double(v.size()));   // nearest rank
    if (k >= v.size()) k = v.size() - 1;
    std::nth_element(v.begin(), v.begin() + k, v.end());
    return v[k];
}

}  // namespace

extern "C" {

nuasm_status nuasm_server_create(nuasm_server_t* out, const nuasm_server_config_t* cfg) {
    if (!out || !cfg) return NUASM_EINVAL;
    *out = nullptr;
    nuasm_server_config_t c = *cfg;
    if (c.slots == 0) c.slots = 4;
    if (c.hbm_budget == 0) c.hbm_budget = kDefaultBudget;
    if (c.slots < 1 || c.slots > kMaxSlots || c.hbm_budget < 0 || c.device < 0) return NUASM_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return NUASM_ECUDA;
    }
    if (c.device >= ndev) return NUASM_EINVAL;
    nuasm_server_s* S = new (std::nothrow) nuasm_server_s();
    if (!S) return NUASM_ENOMEM;
    S->cfg = c;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = c.device;
    cudaError_t e = xpool_create(&S->pool, &props);
    if (e != cudaSuccess) {
        delete S;
        return status_of(e);
    }
    uint64_t keep = UINT64_MAX;   // freed blocks stay reserved for the next request
    cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    int no = 0;                   // never make one slot's allocation wait on another slot's stream
    cudaMemPoolSetAttribute(S->pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    try {
        for (int i = 0; i < c.slots; ++i) S->workers.emplace_back(worker_main, S);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stopping = true;
        }
        S->cv_work.notify_all();
        for (auto& t : S->workers) t.join();
        xpool_destroy(S->pool);
        delete S;
        return NUASM_ENOMEM;
    }
    *out = S;
    return NUASM_OK;
}

nuasm_status nuasm_server_submit(nuasm_server_t S, const nuasm_request_t* req, int64_t* ticket) {
    if (!S || !req || !ticket) return NUASM_EINVAL;
    Job j;
    j.r = *req;
    const nuasm_status s = validate(req->p, req->m, &j.rp);
    if (s != NUASM_OK) return s;
    if (req->type != 1 && req->type != 2) return NUASM_EINVAL;
    j.g = make_geometry(j.rp);
    const int64_t ni = elems_in(j), no = elems_out(j);
    if ((req->m > 0 && (!req->x || !req->y)) || (ni > 0 && !req->in) || (no > 0 && !req->out)) return NUASM_EINVAL;
    const bool in_dev = ni == 0 || device_accessible(req->in);
    const bool out_dev = no == 0 || device_accessible(req->out);
    j.bytes = job_bytes(j, in_dev, out_dev);
    if (j.bytes + set_bytes_estimate(j) > S->cfg.hbm_budget) return NUASM_ENOMEM;
    std::lock_guard<std::mutex> lk(S->mu);
    j.ticket = S->next_ticket++;
    j.submit = Clock::now();
    if (!S->have_first) {
        S->have_first = true;
        S->first_submit = j.submit;
    }
    S->submitted += 1;
    S->done.emplace(j.ticket, Done{});
    *ticket = j.ticket;
    S->queue.push_back(j);
    S->cv_work.notify_all();
    return NUASM_OK;
}

nuasm_status nuasm_server_wait(nuasm_server_t S, int64_t ticket, double timeout_s, nuasm_request_result_t* res) {
    if (!S || !res) return NUASM_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->done.find(ticket);
    if (it == S->done.end()) return NUASM_EINVAL;
    Done* d = &it->second;   // element references survive rehashing
    if (timeout_s < 0) {
        S->cv_done.wait(lk, [&] { return d->done; });
    } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return d->done; })) {
        return NUASM_ETIMEOUT;
    }
    *res = d->res;
    S->done.erase(ticket);
    return NUASM_OK;
}

nuasm_status nuasm_server_stats(nuasm_server_t S, nuasm_server_stats_t* st, int32_t reset) {
    if (!S || !st) return NUASM_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(st, 0, sizeof(*st));
    st->submitted = S->submitted;
    st->completed = S->completed;
    st->failed = S->failed;
    st->points = S->points;
    st->p50_ms = percentile(S->lat, 0.50);
    st->p99_ms = percentile(S->lat, 0.99);
    st->wall_s = S->have_first && S->completed + S->failed > 0
                     ? std::chrono::duration<double>(S->last_done - S->first_submit).count()
                     : 0.0;
    for (auto& p : S->sets)
        if (p->keep && p->state == PointSet::kReady) st->resident_sets += 1;
    st->resident_bytes = S->resident;
    st->bins_built = S->built;
    st->bins_reused = S->reused;
    st->evictions = S->evictions;
    st->peak_bytes = S->peak;
    if (reset) {
        S->submitted = S->completed = S->failed = S->points = S->built = S->reused = S->evictions = 0;
        S->lat.clear();
        S->have_first = false;
        S->peak = S->used;
    }
    return NUASM_OK;
}

nuasm_status nuasm_server_destroy(nuasm_server_t S) {
    if (!S) return NUASM_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    for (auto& p : S->sets)
        if (p->plan) plan_release(p->plan);
    S->sets.clear();
    const cudaError_t e = xpool_destroy(S->pool);
    delete S;
    return status_of(e);
}

}  // extern "C"
