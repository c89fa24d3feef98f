// Native continuous-batching server: the scheduling loop of a serving run in C++, so that
// the host side of a batch (descriptor table, graph launch, completion event) costs a few
// microseconds instead of the tens that a Python loop spends per batch.
//
// Scheduling (the same rules as paper_2206_05506_gb300/serve.py's Server, decision for
// decision -- pnce_sched_simulate runs them on a virtual clock so that the two can be
// compared exactly): requests are admitted in arrival order while the bytes of admitted,
// unfinished work stay under a cap (a request is admitted regardless when nothing is in
// flight); admitted requests wait in buckets keyed by (N, lag class); whenever a stream
// slot is free, the bucket whose oldest request arrived first (ties: the smaller key) is
// launched, packing its requests in order while their antennas fit max_batch_rows (at
// least one request per batch); completions are polled in launch order.
//
// Execution: one CUDA graph per (slot, N, lag class, capacity) captured around one
// pnce_estimate_grouped call, whose descriptor table sits in page-locked host memory and
// is rewritten before each replay; one stream and one completion event per slot.  A table
// is rewritten only after its slot's previous batch completed.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <memory>
#include <tuple>
#include <unordered_map>
#include <utility>
#include <vector>

#include "pnce_internal.h"

namespace {

// lag classes and batch capacities (antennas) of the serving shapes
constexpr int kKlClasses[3] = {64, 256, 1024};
constexpr int kCapacities[4] = {64, 256, 1024, 4096};

int kl_class(int KL, int N) {
    for (int c : kKlClasses)
        if (c >= KL) return std::min(c, N);
    return std::min((KL + 1023) / 1024 * 1024, N);
}

int capacity_for(long long rows) {
    for (int c : kCapacities)
        if (c >= rows) return c;
    return (int)((rows + 4095) / 4096 * 4096);
}

struct ReqState {
    double nbytes = 0.0;
    int klc = 0;
};

// One request in the scheduler: the caller's description, what the run reports for it,
// and its footprint and lag class.
struct Entry {
    pnce_serve_req r;
    pnce_serve_out o;
    double nbytes;
    int klc;
};

// The scheduling rules over an executor E:
//   double E::footprint(const pnce_serve_req&)
//   bool   E::launch(int slot, int N, int klc, const std::vector<const pnce_serve_req*>& rs,
//                    long long rows, int* status)      -- false: the batch failed to start
//   int    E::done(int slot)                           -- 1 done, 0 running, < 0 failed
// Requests enter with submit() (tickets 0, 1, ... in submission order), each step() polls
// completions, admits and launches, and drain() hands over the requests finished since
// the last drain and forgets them.
template <class E>
class Scheduler {
  public:
    Scheduler(E& ex, int slots, double mem_cap, int max_rows)
        : ex_(ex), cap_(mem_cap), max_rows_(max_rows) {
        for (int s = slots - 1; s >= 0; --s) free_.push_back(s);
    }

    long long submit(const pnce_serve_req& r) {
        const long long t = next_ticket_++;
        live_.emplace(t, Entry{r, pnce_serve_out{-1.0, -1.0, -1.0, -1, 0}, ex_.footprint(r),
                               kl_class(r.K * r.L, r.N)});
        pending_.push_back(t);
        return t;
    }

    // one pass: complete, admit and launch
    void step(double now) {
        complete(now);
        admit(now);
        launch(now);
    }

    // f(ticket, entry) for every request finished since the last drain
    template <class F>
    void drain(F&& f) {
        for (long long t : finished_) {
            auto it = live_.find(t);
            f(t, it->second);
            live_.erase(it);
        }
        finished_.clear();
    }

    // nothing waiting, in flight or unreported
    bool idle() const { return live_.empty(); }
    int batches() const { return batches_; }
    size_t open() const { return live_.size(); }

  private:
    struct Busy {
        int slot;
        std::vector<long long> ids;
    };

    void release(const std::vector<long long>& ids, double now, int status) {
        for (long long t : ids) {
            Entry& e = live_.find(t)->second;
            e.o.t_done = now;
            e.o.status = status;
            inflight_ -= e.nbytes;
            finished_.push_back(t);
        }
    }

    void complete(double now) {
        std::vector<Busy> still;
        for (auto& b : busy_) {
            const int d = ex_.done(b.slot);
            if (d == 0) {
                still.push_back(std::move(b));
                continue;
            }
            release(b.ids, now, d > 0 ? (int)PNCE_OK : (int)PNCE_ECUDA);
            free_.push_back(b.slot);
        }
        busy_.swap(still);
    }

    void admit(double now) {
        while (!pending_.empty()) {
            Entry& e = live_.find(pending_.front())->second;
            if (inflight_ + e.nbytes > cap_ && inflight_ > 0) break;   // wait for memory
            inflight_ += e.nbytes;
            e.o.t_admit = now;
            buckets_[{e.r.N, e.klc}].push_back(pending_.front());
            pending_.pop_front();
        }
    }

    void launch(double now) {
        while (!free_.empty()) {
            // the bucket whose head arrived first; ties go to the smaller (N, klc) key
            std::deque<long long>* q = nullptr;
            std::pair<int, int> key{0, 0};
            double best = 0.0;
            for (auto& b : buckets_) {
                if (b.second.empty()) continue;
                const double t = live_.find(b.second.front())->second.r.t_arrival;
                if (!q || t < best) {
                    q = &b.second;
                    key = b.first;
                    best = t;
                }
            }
            if (!q) return;
            std::vector<long long> ids;
            std::vector<const pnce_serve_req*> rs;
            long long rows = 0;
            while (!q->empty()) {
                const Entry& e = live_.find(q->front())->second;
                if (rows + e.r.M > max_rows_ && !ids.empty()) break;
                rows += e.r.M;                 // (a single request above max_rows goes alone)
                ids.push_back(q->front());
                rs.push_back(&e.r);
                q->pop_front();
                if (rows >= max_rows_) break;
            }
            const int slot = free_.back();
            free_.pop_back();
            for (long long t : ids) {
                Entry& e = live_.find(t)->second;
                e.o.t_launch = now;
                e.o.batch = batches_;
            }
            int status = PNCE_OK;
            if (!ex_.launch(slot, key.first, key.second, rs, rows, &status)) {
                release(ids, now, status == PNCE_OK ? (int)PNCE_ECUDA : status);
                free_.push_back(slot);
                continue;
            }
            busy_.push_back(Busy{slot, std::move(ids)});
            ++batches_;
        }
    }

    E& ex_;
    double cap_;
    int max_rows_;
    std::unordered_map<long long, Entry> live_;
    std::vector<long long> finished_;
    long long next_ticket_ = 0;
    std::deque<long long> pending_;
    std::map<std::pair<int, int>, std::deque<long long>> buckets_;
    std::vector<int> free_;
    std::vector<Busy> busy_;
    double inflight_ = 0.0;
    int batches_ = 0;
};

// Virtual time (no GPU): a batch of r rows takes base + per_row * r seconds; a request's
// footprint is M * row_bytes; the clock advances by dt at every pass of the loop.  Faults
// made on the host: every fail_launch-th launch is refused, and every fail_done-th batch
// that started reports a failure when it completes (0: never).
struct SimExec {
    double* t;
    double base, per_row, row_bytes;
    int fail_launch, fail_done;
    std::vector<double> end;
    std::vector<char> running, fault;
    long long calls = 0, started = 0;
    double footprint(const pnce_serve_req& r) const { return (double)r.M * row_bytes; }
    bool launch(int slot, int, int, const std::vector<const pnce_serve_req*>&, long long rows,
                int* status) {
        ++calls;
        if (fail_launch > 0 && calls % fail_launch == 0) {
            *status = PNCE_ECUDA;
            return false;
        }
        ++started;
        end[(size_t)slot] = *t + base + per_row * (double)rows;
        running[(size_t)slot] = 1;
        fault[(size_t)slot] = fail_done > 0 && started % fail_done == 0;
        return true;
    }
    int done(int slot) {
        if (running[(size_t)slot] && *t >= end[(size_t)slot]) {
            running[(size_t)slot] = 0;
            if (fault[(size_t)slot]) return -1;
        }
        return running[(size_t)slot] ? 0 : 1;
    }
};

bool req_ok(const pnce_serve_req& r) {
    return r.M >= 1 && r.N >= 2 && r.K >= 1 && r.L >= 1 && (long long)r.K * r.L <= r.N &&
           std::isfinite(r.t_arrival);
}

bool serve_args_ok(const pnce_serve_req* reqs, int n, const pnce_serve_out* out, int slots,
                   double mem_cap, int max_rows) {
    if (n < 0 || (n > 0 && (!reqs || !out)) || slots < 1 || slots > 64 || max_rows < 1 ||
        !(mem_cap > 0.0))
        return false;
    for (int i = 0; i < n; ++i)
        if (!req_ok(reqs[i]) || (i > 0 && reqs[i].t_arrival < reqs[i - 1].t_arrival))
            return false;
    return true;
}

// Open-loop replay of a trace: at each pass the requests that have arrived by now are
// submitted (ticket i for request i), the scheduler steps, and finished requests are
// copied out.
template <class S, class Clock>
void replay(S& sch, const pnce_serve_req* reqs, int n, pnce_serve_out* out, Clock&& now_fn) {
    for (int i = 0; i < n; ++i) out[i] = pnce_serve_out{-1.0, -1.0, -1.0, -1, -1};   // not run
    int next = 0;
    while (next < n || !sch.idle()) {
        const double now = now_fn();
        while (next < n && reqs[next].t_arrival <= now) sch.submit(reqs[next++]);
        sch.step(now);
        sch.drain([&](long long t, const Entry& e) { out[t] = e.o; });
    }
}

// The entry points allocate through the standard library; nothing may throw across the C
// boundary, so an exception (out of host memory) becomes PNCE_ENOMEM.
template <class F>
pnce_status guarded(F&& f) {
    try {
        return f();
    } catch (...) {
        return PNCE_ENOMEM;
    }
}

}  // namespace

extern "C" pnce_status pnce_sched_simulate(const pnce_serve_req* reqs, int n, int slots,
                                           double mem_cap, int max_batch_rows, double row_bytes,
                                           double base_s, double per_row_s, double clock_dt,
                                           int fail_launch_every, int fail_done_every,
                                           pnce_serve_out* out, int* batches) {
    if (!serve_args_ok(reqs, n, out, slots, mem_cap, max_batch_rows) || !(clock_dt > 0.0) ||
        !(base_s >= 0.0) || !(per_row_s >= 0.0) || !(row_bytes >= 0.0) ||
        fail_launch_every < 0 || fail_done_every < 0)
        return PNCE_EINVAL;
    return guarded([&] {
        double t = 0.0;
        SimExec ex{&t, base_s, per_row_s, row_bytes, fail_launch_every, fail_done_every,
                   std::vector<double>((size_t)slots, 0.0), std::vector<char>((size_t)slots, 0),
                   std::vector<char>((size_t)slots, 0)};
        Scheduler<SimExec> sch(ex, slots, mem_cap, max_batch_rows);
        replay(sch, reqs, n, out, [&] { return t += clock_dt; });
        if (batches) *batches = sch.batches();
        return PNCE_OK;
    });
}

namespace {

// One batch shape on one slot: its workspace, its page-locked descriptor table and the
// graph captured around pnce_estimate_grouped over them.
struct ServeShape {
    int N = 0, klc = 0, cap = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    pnce_req_desc* desc = nullptr;
    int used = 0;                            // descriptors written by the last batch
    cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct pnce_server {
    pnce_handle* h = nullptr;
    int dtype = PNCE_FP16;
    int slots = 0;
    double mem_cap = 0.0;
    int max_rows = 0;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::map<int, const pnce_pilot*> pilots;                 // by N; not owned
    std::map<std::tuple<int, int, int, int>, std::unique_ptr<ServeShape>> shapes;
    void* online = nullptr;                                  // OnlineSession, owned
    void (*online_free)(void*) = nullptr;
};

namespace {

void free_shape(ServeShape* s) {
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->ws) cudaFree(s->ws);
    if (s->desc) cudaFreeHost(s->desc);
    s->exec = nullptr;
    s->ws = nullptr;
    s->desc = nullptr;
}

// Create and capture shape (slot, N, klc, cap), or return the existing one.
pnce_status get_shape(pnce_server* sv, int slot, int N, int klc, int cap, ServeShape** out) {
    const auto key = std::make_tuple(slot, N, klc, cap);
    auto it = sv->shapes.find(key);
    if (it != sv->shapes.end()) {
        *out = it->second.get();
        return PNCE_OK;
    }
    auto pit = sv->pilots.find(N);
    if (pit == sv->pilots.end()) return PNCE_EINVAL;
    const pnce_pilot* pilot = pit->second;
    auto sh = std::make_unique<ServeShape>();
    sh->N = N;
    sh->klc = klc;
    sh->cap = cap;
    sh->ws_bytes = pnce_grouped_workspace_size(cap, N, klc, sv->dtype);
    if (sh->ws_bytes == 0) return PNCE_EINVAL;
    if (cudaMalloc(&sh->ws, sh->ws_bytes) != cudaSuccess) {
        cudaGetLastError();
        return PNCE_ENOMEM;
    }
    if (cudaHostAlloc(reinterpret_cast<void**>(&sh->desc), sizeof(pnce_req_desc) * (size_t)cap,
                      cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        free_shape(sh.get());
        return PNCE_ENOMEM;
    }
    std::fill(sh->desc, sh->desc + cap, pnce_req_desc{nullptr, nullptr, 0, 0, 0, 0});
    cudaStream_t s = sv->streams[(size_t)slot];
    // an eager run first (it sets the kernels' attributes), then the capture
    pnce_status st = pnce_estimate_grouped(sv->h, pilot, sh->desc, cap, cap, klc, sv->dtype,
                                           sh->ws, sh->ws_bytes, s);
    if (st == PNCE_OK && cudaStreamSynchronize(s) != cudaSuccess) st = PNCE_ECUDA;
    if (st != PNCE_OK) {
        free_shape(sh.get());
        return st;
    }
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        free_shape(sh.get());
        return PNCE_ECUDA;
    }
    st = pnce_estimate_grouped(sv->h, pilot, sh->desc, cap, cap, klc, sv->dtype, sh->ws,
                               sh->ws_bytes, s);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (st == PNCE_OK && (ce != cudaSuccess || !g)) st = PNCE_ECUDA;
    if (st == PNCE_OK && cudaGraphInstantiate(&sh->exec, g, 0) != cudaSuccess) st = PNCE_ECUDA;
    if (g) cudaGraphDestroy(g);
    if (st != PNCE_OK) {
        cudaGetLastError();
        free_shape(sh.get());
        return st;
    }
    *out = sh.get();
    sv->shapes.emplace(key, std::move(sh));
    return PNCE_OK;
}

// Executes batches on the GPU for the scheduler: footprint as the Python engine counts it
// (received rows, operand rows, result rows of the batch buffers).
struct CudaExec {
    pnce_server* sv;
    int elt;
    double footprint(const pnce_serve_req& r) const {
        const double pitch = (double)((r.N + 63) / 64 * 64);
        return (double)r.M * (8.0 * r.N + 2.0 * elt * pitch + 8.0 * kl_class(r.K * r.L, r.N));
    }
    bool launch(int slot, int N, int klc, const std::vector<const pnce_serve_req*>& rs,
                long long rows, int* status) {
        ServeShape* sh = nullptr;
        const pnce_status st = get_shape(sv, slot, N, klc, capacity_for(rows), &sh);
        if (st != PNCE_OK) {
            *status = st;
            return false;
        }
        int off = 0;
        const int n = (int)rs.size();
        for (int k = 0; k < n; ++k) {
            const pnce_serve_req& r = *rs[(size_t)k];
            sh->desc[k] = pnce_req_desc{r.Y, r.H, r.M, r.K, r.L, off};
            off += r.M;
        }
        for (int k = n; k < sh->used; ++k) sh->desc[k].M = 0;    // empty slots
        sh->used = n;
        cudaStream_t s = sv->streams[(size_t)slot];
        if (cudaGraphLaunch(sh->exec, s) != cudaSuccess ||
            cudaEventRecord(sv->events[(size_t)slot], s) != cudaSuccess) {
            cudaGetLastError();
            *status = PNCE_ECUDA;
            return false;
        }
        return true;
    }
    int done(int slot) {
        const cudaError_t e = cudaEventQuery(sv->events[(size_t)slot]);
        if (e == cudaSuccess) return 1;
        if (e == cudaErrorNotReady) return 0;
        cudaGetLastError();
        return -1;
    }
};

// An online session: requests submitted one by one and stamped with the session clock,
// each poll one scheduling pass; finished requests wait in `ready` until reported.
struct OnlineSession {
    CudaExec ex;
    Scheduler<CudaExec> sch;
    std::chrono::steady_clock::time_point t0;
    std::deque<std::pair<long long, pnce_serve_out>> ready;
    OnlineSession(pnce_server* sv, int elt)
        : ex{sv, elt}, sch(ex, sv->slots, sv->mem_cap, sv->max_rows),
          t0(std::chrono::steady_clock::now()) {}
    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};
void online_free(void* p) { delete static_cast<OnlineSession*>(p); }
OnlineSession* online_of(pnce_server* sv) { return static_cast<OnlineSession*>(sv->online); }

int operand_elt(int dtype) {
    switch (dtype) {
        case PNCE_FP32_SIMT: return 0;
        case PNCE_TF32: return 4;
        case PNCE_FP8E4M3: return 1;
        default: return 2;                   // fp16, bf16, and PNCE_AUTO's upper bound
    }
}

}  // namespace

extern "C" {

pnce_status pnce_server_create(pnce_handle* h, int dtype, int slots, double mem_cap_bytes,
                               int max_batch_rows, pnce_server** out) {
    if (!h || !out || slots < 1 || slots > 64 || !(mem_cap_bytes > 0.0) || max_batch_rows < 1)
        return PNCE_EINVAL;
    if (!(dtype == PNCE_FP32_SIMT || dtype == PNCE_TF32 || dtype == PNCE_FP16 ||
          dtype == PNCE_BF16 || dtype == PNCE_FP8E4M3 || dtype == PNCE_AUTO))
        return PNCE_EINVAL;
    *out = nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return PNCE_ECUDA;
    if (dev != h->device) return PNCE_ESTATE;
    return guarded([&]() -> pnce_status {
        auto sv = std::make_unique<pnce_server>();
        sv->h = h;
        sv->dtype = dtype;
        sv->slots = slots;
        sv->mem_cap = mem_cap_bytes;
        sv->max_rows = max_batch_rows;
        for (int i = 0; i < slots; ++i) {
            cudaStream_t s = nullptr;
            cudaEvent_t e = nullptr;
            if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
                pnce_server_destroy(sv.release());
                return PNCE_ECUDA;
            }
            sv->streams.push_back(s);
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
                pnce_server_destroy(sv.release());
                return PNCE_ECUDA;
            }
            sv->events.push_back(e);
        }
        *out = sv.release();
        return PNCE_OK;
    });
}

pnce_status pnce_server_destroy(pnce_server* sv) {
    if (!sv) return PNCE_EINVAL;
    for (cudaStream_t s : sv->streams) cudaStreamSynchronize(s);
    if (sv->online) sv->online_free(sv->online);
    for (auto& kv : sv->shapes) free_shape(kv.second.get());
    for (cudaEvent_t e : sv->events) cudaEventDestroy(e);
    for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
    delete sv;
    return PNCE_OK;
}

pnce_status pnce_server_add_pilot(pnce_server* sv, const pnce_pilot* pilot) {
    if (!sv || !pilot) return PNCE_EINVAL;
    if (pilot->device != sv->h->device) return PNCE_ESTATE;
    return guarded([&]() -> pnce_status {
        auto it = sv->pilots.find(pilot->N);
        if (it != sv->pilots.end() && it->second != pilot) {
            // the graphs captured for this N read the old pilot's table: drop them (they are
            // captured again on first use), so the old pilot may be destroyed
            for (cudaStream_t s : sv->streams)
                if (cudaStreamSynchronize(s) != cudaSuccess) return PNCE_ECUDA;
            for (auto sit = sv->shapes.begin(); sit != sv->shapes.end();) {
                if (std::get<1>(sit->first) == pilot->N) {
                    free_shape(sit->second.get());
                    sit = sv->shapes.erase(sit);
                } else {
                    ++sit;
                }
            }
        }
        sv->pilots[pilot->N] = pilot;
        return PNCE_OK;
    });
}

pnce_status pnce_server_prepare(pnce_server* sv, int N, int kl_class_, int capacity) {
    if (!sv || capacity < 1 || kl_class_ < 1 || kl_class_ > N) return PNCE_EINVAL;
    return guarded([&] {
        for (int slot = 0; slot < sv->slots; ++slot) {
            ServeShape* sh = nullptr;
            const pnce_status st = get_shape(sv, slot, N, kl_class_, capacity, &sh);
            if (st != PNCE_OK) return st;
        }
        return PNCE_OK;
    });
}

pnce_status pnce_server_run(pnce_server* sv, const pnce_serve_req* reqs, int n,
                            pnce_serve_out* out, int* batches) {
    if (!sv || !serve_args_ok(reqs, n, out, sv->slots, sv->mem_cap, sv->max_rows))
        return PNCE_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!reqs[i].Y || !reqs[i].H) return PNCE_EINVAL;
    // the online session's batches use the same slots and tables
    const OnlineSession* o = online_of(sv);
    if (o && (!o->sch.idle() || !o->ready.empty())) return PNCE_ESTATE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return PNCE_ECUDA;
    if (dev != sv->h->device) return PNCE_ESTATE;
    int nb = 0;
    const pnce_status st = guarded([&] {
        CudaExec ex{sv, operand_elt(sv->dtype)};
        Scheduler<CudaExec> sch(ex, sv->slots, sv->mem_cap, sv->max_rows);
        using clk = std::chrono::steady_clock;
        const clk::time_point t0 = clk::now();
        replay(sch, reqs, n, out,
               [&] { return std::chrono::duration<double>(clk::now() - t0).count(); });
        nb = sch.batches();
        return PNCE_OK;
    });
    if (batches) *batches = nb;
    if (st != PNCE_OK) {                   // out of host memory part-way: let the GPU finish
        for (cudaStream_t s : sv->streams) cudaStreamSynchronize(s);
        return st;
    }
    // a kernel of these batches may have latched an error (a bounded wait that ran out, an
    // invalid descriptor): then some results may be wrong, and the run says so
    for (cudaStream_t s : sv->streams)
        if (cudaStreamSynchronize(s) != cudaSuccess) return PNCE_ECUDA;
    return pnce_get_status(sv->h, sv->streams[0]);
}

pnce_status pnce_server_start(pnce_server* sv) {
    if (!sv) return PNCE_EINVAL;
    OnlineSession* o = online_of(sv);
    if (o && (!o->sch.idle() || !o->ready.empty())) return PNCE_ESTATE;   // still open
    return guarded([&] {
        auto fresh = std::make_unique<OnlineSession>(sv, operand_elt(sv->dtype));
        if (sv->online) sv->online_free(sv->online);
        sv->online = fresh.release();
        sv->online_free = online_free;
        return PNCE_OK;
    });
}

pnce_status pnce_server_submit(pnce_server* sv, const pnce_serve_req* req, long long* ticket) {
    if (!sv || !req || !ticket) return PNCE_EINVAL;
    OnlineSession* o = online_of(sv);
    if (!o) return PNCE_ESTATE;
    pnce_serve_req r = *req;
    r.t_arrival = o->now();
    if (!r.Y || !r.H || !req_ok(r)) return PNCE_EINVAL;
    return guarded([&] {
        *ticket = o->sch.submit(r);
        return PNCE_OK;
    });
}

pnce_status pnce_server_poll(pnce_server* sv, long long* tickets, pnce_serve_out* outs,
                             int max_out, int* n_out) {
    if (!sv || !n_out || max_out < 0 || (max_out > 0 && (!tickets || !outs))) return PNCE_EINVAL;
    *n_out = 0;
    OnlineSession* o = online_of(sv);
    if (!o) return PNCE_ESTATE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return PNCE_ECUDA;
    if (dev != sv->h->device) return PNCE_ESTATE;
    return guarded([&] {
        o->sch.step(o->now());
        o->sch.drain([&](long long t, const Entry& e) { o->ready.emplace_back(t, e.o); });
        int k = 0;
        while (k < max_out && !o->ready.empty()) {
            tickets[k] = o->ready.front().first;
            outs[k] = o->ready.front().second;
            o->ready.pop_front();
            ++k;
        }
        *n_out = k;
        return PNCE_OK;
    });
}

pnce_status pnce_server_open(pnce_server* sv, int* n) {
    if (!sv || !n) return PNCE_EINVAL;
    OnlineSession* o = online_of(sv);
    *n = o ? (int)(o->sch.open() + o->ready.size()) : 0;
    return PNCE_OK;
}

}  // extern "C"
