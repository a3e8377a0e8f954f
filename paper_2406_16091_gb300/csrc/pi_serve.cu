// pi_serve.cu -- a request loop for interaction jobs over device-resident
// contexts ("slots"): continuous batching on one GPU, host code only.
//
// Every slot is a single-system context with its own stream, completion
// event and pinned scratch block for results.  A job runs on one slot as one
// pi_submit_host_strided call (re-target, copy in, bin, interact, copy out),
// the same kernels a lone pi_bin + pi_interact runs, so its results do not
// depend on the mix.  Slots come in capacity buckets; a job waits in the
// queue of the smallest bucket that fits it and may take a free slot of a
// larger one.  When every slot that fits a job is busy, a new slot is made
// while the bucket's slot limit, the server's HBM budget and the device's
// free memory allow (memory-based admission); otherwise the job waits.
// Completion is polled with cudaEventQuery; nothing on the device waits.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "pi.h"

namespace {

struct Slot {
    pi_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    float* scratch = nullptr;  // pinned: 5 arrays of results for jobs without outputs
    int64_t cap = 0;
    int bucket = 0;
    int64_t job = -1;
};

// Largest FP32 cutoff not above 1/k: a unit box then has exactly k cells
// per axis under the grid rule floor(1 / r_c).
float rc_for_cells(int64_t k)
{
    float rc = (float)(1.0 / (double)k);
    while ((double)rc * (double)k > 1.0) rc = std::nextafterf(rc, 0.0f);
    return rc;
}

int64_t round4(int64_t n) { return (n + 3) & ~(int64_t)3; }

// Cells of a job's grid: the rule of pi_create, in FP64.
int64_t grid_cells(const pi_box& b, float r_c)
{
    int64_t c = 1;
    for (int d = 0; d < 3; ++d) {
        const double n = std::floor(((double)b.hi[d] - (double)b.lo[d]) / (double)r_c);
        c *= n < 1.0 ? 1 : (int64_t)n;
    }
    return c;
}

}  // namespace

struct pi_server {
    int device = 0;
    std::vector<int64_t> caps;  // ascending
    int max_per_bucket = 8;
    int64_t budget = 0, used = 0;
    std::vector<std::vector<Slot*>> slots, free;
};

namespace {

void destroy_slot(Slot* s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->ctx) pi_destroy(s->ctx);
    if (s->done) cudaEventDestroy(s->done);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->scratch) cudaFreeHost(s->scratch);
    delete s;
}

// A new slot of bucket b if the bucket's limit, the HBM budget and the
// device's free memory allow it; *made = false (and PI_OK) when they do not.
pi_status grow(pi_server* srv, int b, bool* made)
{
    *made = false;
    if ((int)srv->slots[b].size() >= srv->max_per_bucket) return PI_OK;
    const int64_t cap = srv->caps[b];
    const int64_t need = pi_server_slot_bytes(cap);
    if (srv->used + need > srv->budget) return PI_OK;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return PI_ERR_CUDA;
    if ((size_t)need > free_b) return PI_OK;
    Slot* s = new (std::nothrow) Slot;
    if (!s) return PI_ERR_NOMEM;
    s->cap = cap;
    s->bucket = b;
    // a unit box with k^3 >= cap cells sizes the grid capacity
    int64_t k = (int64_t)std::ceil(std::cbrt((double)cap) - 1e-9);
    while (k * k * k < cap) ++k;
    const pi_box unit = {{0.f, 0.f, 0.f}, {1.f, 1.f, 1.f}};
    pi_status st = pi_create(&unit, rc_for_cells(k), cap, &s->ctx);
    if (st == PI_OK && cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) st = PI_ERR_CUDA;
    if (st == PI_OK && cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming) != cudaSuccess) st = PI_ERR_CUDA;
    if (st == PI_OK &&
        cudaHostAlloc((void**)&s->scratch, (size_t)5 * (size_t)round4(cap) * sizeof(float), cudaHostAllocDefault) !=
            cudaSuccess)
        st = PI_ERR_NOMEM;
    if (st == PI_OK) {
        // allocate the context's staging buffers now, outside the request loop
        const int64_t d = round4(cap);
        float* o = s->scratch;
        st = pi_submit_host_strided(s->ctx, &unit, rc_for_cells(k), o, o, o, 0, 0, 0.5f, o, o + d, o + 2 * d,
                                    o + 3 * d, (uint32_t*)(o + 4 * d), d, PI_ORDER_ORIGINAL, s->stream);
    }
    if (st == PI_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) st = PI_ERR_CUDA;
    if (st != PI_OK) {
        destroy_slot(s);
        return st;
    }
    srv->slots[b].push_back(s);
    srv->free[b].push_back(s);
    srv->used += need;
    *made = true;
    return PI_OK;
}

// Smallest bucket whose slots fit the job, -1 if none does.
int bucket_of(const pi_server* srv, const pi_job& j)
{
    const int64_t cells = grid_cells(j.box, j.r_c);
    for (size_t b = 0; b < srv->caps.size(); ++b)
        if (srv->caps[b] >= j.n && srv->caps[b] >= cells) return (int)b;
    return -1;
}

pi_status check_job(const pi_server* srv, const pi_job& j)
{
    if (j.n < 0 || !(j.r_c > 0.f) || !(j.h > 0.f) || !std::isfinite(j.arrival)) return PI_ERR_INVALID_ARG;
    if (j.n > 0 && (!j.x || (j.in_stride == 0 && (!j.y || !j.z)))) return PI_ERR_INVALID_ARG;
    const bool any = j.S || j.Vx || j.Vy || j.Vz, all = j.S && j.Vx && j.Vy && j.Vz;
    if (any && !all) return PI_ERR_INVALID_ARG;
    if (bucket_of(srv, j) < 0) return PI_ERR_CAPACITY;
    return PI_OK;
}

// Enqueues job j on slot s (nothing waits).
pi_status start(pi_server* srv, Slot* s, pi_job& j)
{
    (void)srv;
    const float* y = j.in_stride ? j.x + j.in_stride : j.y;
    const float* z = j.in_stride ? j.x + 2 * j.in_stride : j.z;
    pi_status st;
    if (j.S) {
        st = pi_submit_host_strided(s->ctx, &j.box, j.r_c, j.x, y, z, j.in_stride, j.n, j.h, j.S, j.Vx, j.Vy, j.Vz,
                                    j.nbr, j.out_stride, PI_ORDER_ORIGINAL, s->stream);
    } else {
        // results into the slot's scratch block, one copy out
        const int64_t d = round4(j.n);
        float* o = s->scratch;
        st = pi_submit_host_strided(s->ctx, &j.box, j.r_c, j.x, y, z, j.in_stride, j.n, j.h, o, o + d, o + 2 * d,
                                    o + 3 * d, (uint32_t*)(o + 4 * d), d, PI_ORDER_ORIGINAL, s->stream);
    }
    if (st != PI_OK) return st;
    if (cudaEventRecord(s->done, s->stream) != cudaSuccess) return PI_ERR_CUDA;
    return PI_OK;
}

}  // namespace

extern "C" {

int64_t pi_server_slot_bytes(int64_t capacity)
{
    // the context (72 bytes per particle, up to 28 per cell, cells <= particles,
    // rounded up), its host-transfer staging (32 bytes per particle) and 1 MiB
    return capacity * (80 + 32) + capacity * 32 + (1 << 20);
}

pi_status pi_server_create(int32_t num_buckets, const int64_t* capacity, const int32_t* initial_slots,
                           int32_t max_slots_per_bucket, int64_t hbm_budget, pi_server** out)
{
    if (!out || num_buckets < 1 || num_buckets > PI_SERVER_MAX_BUCKETS || !capacity || max_slots_per_bucket < 1)
        return PI_ERR_INVALID_ARG;
    *out = nullptr;
    std::vector<std::pair<int64_t, int32_t>> b;
    for (int i = 0; i < num_buckets; ++i) {
        if (capacity[i] < 1 || capacity[i] > ((int64_t)1 << 30)) return PI_ERR_INVALID_ARG;
        const int32_t k = initial_slots ? initial_slots[i] : 0;
        if (k < 0) return PI_ERR_INVALID_ARG;
        b.push_back({capacity[i], k});
    }
    std::sort(b.begin(), b.end());
    for (size_t i = 1; i < b.size(); ++i)
        if (b[i].first == b[i - 1].first) return PI_ERR_INVALID_ARG;
    pi_server* srv = new (std::nothrow) pi_server;
    if (!srv) return PI_ERR_NOMEM;
    if (cudaGetDevice(&srv->device) != cudaSuccess) {
        delete srv;
        return PI_ERR_CUDA;
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete srv;
        return PI_ERR_CUDA;
    }
    srv->budget = hbm_budget > 0 ? hbm_budget : (int64_t)(free_b / 2);
    srv->max_per_bucket = max_slots_per_bucket;
    for (auto& e : b) srv->caps.push_back(e.first);
    srv->slots.assign(b.size(), {});
    srv->free.assign(b.size(), {});
    for (size_t i = 0; i < b.size(); ++i)
        for (int32_t k = 0; k < b[i].second; ++k) {
            bool made = false;
            const pi_status st = grow(srv, (int)i, &made);
            if (st != PI_OK) {
                pi_server_destroy(srv);
                return st;
            }
            if (!made) break;
        }
    *out = srv;
    return PI_OK;
}

pi_status pi_server_run(pi_server* srv, pi_job* jobs, int64_t num_jobs, double* makespan_s)
{
    if (!srv || num_jobs < 0 || (num_jobs > 0 && !jobs)) return PI_ERR_INVALID_ARG;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(srv->device) != cudaSuccess) return PI_ERR_CUDA;
    struct Restore {
        int d;
        ~Restore() { cudaSetDevice(d); }
    } restore{prev};
    for (int64_t k = 0; k < num_jobs; ++k) {
        const pi_status st = check_job(srv, jobs[k]);
        if (st != PI_OK) return st;
        jobs[k].t_start = jobs[k].t_done = -1.0;
        jobs[k].slot_capacity = 0;
    }
    std::vector<int64_t> order((size_t)num_jobs);
    for (int64_t k = 0; k < num_jobs; ++k) order[(size_t)k] = k;
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t a, int64_t b) { return jobs[a].arrival < jobs[b].arrival; });
    const size_t nb = srv->caps.size();
    std::vector<std::deque<int64_t>> queues(nb);
    std::vector<Slot*> busy;
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    auto now = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
    size_t next = 0;
    int64_t done = 0;
    pi_status err = PI_OK;
    while (done < num_jobs && err == PI_OK) {
        const double t = now();
        bool arrived = false, freed = false;
        while (next < order.size() && jobs[order[next]].arrival <= t) {
            const int64_t k = order[next++];
            queues[(size_t)bucket_of(srv, jobs[k])].push_back(k);
            arrived = true;
        }
        // completions
        for (size_t i = 0; i < busy.size();) {
            Slot* s = busy[i];
            const cudaError_t q = cudaEventQuery(s->done);
            if (q == cudaSuccess) {
                jobs[s->job].t_done = now();
                s->job = -1;
                srv->free[(size_t)s->bucket].push_back(s);
                busy[i] = busy.back();
                busy.pop_back();
                ++done;
                freed = true;
            } else if (q == cudaErrorNotReady) {
                ++i;
            } else {
                err = PI_ERR_CUDA;
                break;
            }
        }
        if (err != PI_OK) break;
        if (arrived || freed) {
            // each bucket from the largest down: its free slots take the
            // oldest job among its own queue and those of smaller buckets
            for (int b = (int)nb - 1; b >= 0 && err == PI_OK; --b) {
                for (;;) {
                    int best = -1;
                    for (int q = 0; q <= b; ++q)
                        if (!queues[q].empty() &&
                            (best < 0 || jobs[queues[q].front()].arrival < jobs[queues[best].front()].arrival))
                            best = q;
                    if (best < 0) break;
                    if (srv->free[(size_t)b].empty()) {
                        bool made = false;
                        if ((err = grow(srv, b, &made)) != PI_OK || !made) break;
                    }
                    Slot* s = srv->free[(size_t)b].back();
                    srv->free[(size_t)b].pop_back();
                    const int64_t k = queues[best].front();
                    queues[best].pop_front();
                    jobs[k].t_start = now();
                    jobs[k].slot_capacity = s->cap;
                    s->job = k;
                    if ((err = start(srv, s, jobs[k])) != PI_OK) {
                        // the slot stays usable for later runs; the run ends
                        s->job = -1;
                        srv->free[(size_t)b].push_back(s);
                        break;
                    }
                    busy.push_back(s);
                }
            }
        }
        if (busy.empty() && next < order.size()) {
            bool queued = false;
            for (auto& q : queues) queued = queued || !q.empty();
            if (!queued) {
                // idle until the next arrival (short sleeps keep the latency low)
                const double wait = jobs[order[next]].arrival - now();
                if (wait > 2e-4) std::this_thread::sleep_for(std::chrono::microseconds(100));
            }
        }
    }
    if (makespan_s) *makespan_s = now();
    // drain and collect device-side errors of every slot
    for (auto& lst : srv->slots)
        for (Slot* s : lst) {
            const pi_status st = pi_sync_status(s->ctx, s->stream, nullptr);
            if (err == PI_OK && st != PI_OK) err = st;
        }
    // after an error, slots still marked busy are drained: free them again
    for (Slot* s : busy) {
        s->job = -1;
        srv->free[(size_t)s->bucket].push_back(s);
    }
    return err;
}

pi_status pi_server_info(const pi_server* srv, int32_t* num_buckets, int64_t* capacity, int32_t* slots,
                         int64_t* hbm_used)
{
    if (!srv) return PI_ERR_INVALID_ARG;
    if (num_buckets) *num_buckets = (int32_t)srv->caps.size();
    for (size_t b = 0; b < srv->caps.size(); ++b) {
        if (capacity) capacity[b] = srv->caps[b];
        if (slots) slots[b] = (int32_t)srv->slots[b].size();
    }
    if (hbm_used) *hbm_used = srv->used;
    return PI_OK;
}

pi_status pi_server_destroy(pi_server* srv)
{
    if (!srv) return PI_OK;
    for (auto& lst : srv->slots)
        for (Slot* s : lst) destroy_slot(s);
    delete srv;
    return PI_OK;
}

}  // extern "C"
