// Request server: asynchronous clustering jobs with continuous batching (host runtime).
//
// Jobs are queued by hca_submit.  Worker threads (each with its own CUDA stream) repeatedly
// take every queued job that fits the device-memory budget (each charged its points, labels
// and the hca_workspace_bytes bound of its workspace), group them by (d, dtype), stage each
// group's points into the worker's resident device buffer, cluster the group with one
// hca_dbscan_batched call, copy each job's labels to its destination, and complete the jobs.  Jobs that arrive
// while a batch is on the GPU join the next batch of a free worker, and the workers keep as many
// batches in flight.  All waits on the host are condition-variable waits with deadlines.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "hca_internal.cuh"

struct hca_server {
    struct Job {
        hca_request req;
        int state;  // 0 queued, 1 running, 2 done, 3 cancelled
        int rc;
        std::chrono::steady_clock::time_point t_submit, t_done;
        int64_t bytes;
    };
    int device;
    int64_t budget;
    int64_t in_flight = 0;
    int64_t next_ticket = 1;
    bool stop = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> queue;
    std::map<int64_t, Job> jobs;
    std::vector<std::thread> workers;
};

namespace {

using Clock = std::chrono::steady_clock;

// Device memory a job is charged for: its points and labels in the worker's staging buffers
// and the bound of hca_workspace_bytes on the clustering workspace, plus 16 bytes per point
// for the power-of-two rounding of the hash table when jobs share a call and 1 KB for the
// per-set tables.
int64_t job_bytes(const hca_request &r) {
    const int64_t esz = r.dtype == HCA_F32 ? 4 : 8;
    int64_t ws = 0;
    if (hca_workspace_bytes(r.n, r.d, r.dtype, 0, &ws) != HCA_OK) ws = r.n * 2048;
    return r.n * (r.d * esz + 4) + ws + 16 * r.n + 1024;
}

// Device buffers a worker keeps from batch to batch: the staged points and the labels of
// its current group, grown (never shrunk) as larger groups arrive.
struct Staging {
    void *dp = nullptr;
    size_t dp_cap = 0;
    void *dl = nullptr;
    size_t dl_cap = 0;
};

bool ensure(void **p, size_t *cap, size_t bytes, cudaStream_t s) {
    if (bytes <= *cap) return true;
    size_t want = *cap + *cap / 2;
    if (want < bytes) want = bytes;
    if (*p) hca::pool_free(*p, s);
    *p = nullptr;
    *cap = 0;
    if (hca::pool_alloc(p, want, s) != cudaSuccess || !*p) return false;
    *cap = want;
    return true;
}

void run_group(hca_server *sv, std::vector<int64_t> &ids, cudaStream_t s, Staging &stg) {
    // ids share d and dtype; copy their jobs' requests (the map is not touched while running)
    std::vector<hca_request> reqs;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (int64_t id : ids) reqs.push_back(sv->jobs[id].req);
    }
    const int32_t d = reqs[0].d, dtype = reqs[0].dtype;
    const size_t esz = dtype == HCA_F32 ? 4 : 8;
    std::vector<int64_t> off(reqs.size() + 1, 0);
    std::vector<double> eps(reqs.size());
    std::vector<int32_t> mp(reqs.size()), dims(reqs.size(), d);
    for (size_t i = 0; i < reqs.size(); ++i) {
        off[i + 1] = off[i] + reqs[i].n;
        eps[i] = reqs[i].eps;
        mp[i] = reqs[i].min_pts;
    }
    const int64_t n = off.back();
    int rc = HCA_OK;
    if (n > 0 && (!ensure(&stg.dp, &stg.dp_cap, (size_t)n * d * esz, s) ||
                  !ensure(&stg.dl, &stg.dl_cap, (size_t)n * 4, s)))
        rc = HCA_ENOMEM;
    void *dp = stg.dp, *dl = stg.dl;
    for (size_t i = 0; i < reqs.size() && rc == HCA_OK; ++i) {
        if (reqs[i].n == 0) continue;
        const cudaMemcpyKind kind = reqs[i].on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (cudaMemcpyAsync((char *)dp + (size_t)off[i] * d * esz, reqs[i].points, (size_t)reqs[i].n * d * esz,
                            kind, s) != cudaSuccess)
            rc = HCA_ECUDA;
    }
    if (rc == HCA_OK && n > 0)
        rc = hca_dbscan_batched(dp, dtype, (int32_t)reqs.size(), off.data(), dims.data(), eps.data(), mp.data(),
                                (int32_t *)dl, nullptr, (void *)s, nullptr, 0);
    for (size_t i = 0; i < reqs.size() && rc == HCA_OK; ++i) {
        if (reqs[i].n == 0) continue;
        const cudaMemcpyKind kind = reqs[i].on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (cudaMemcpyAsync(reqs[i].labels, (int32_t *)dl + off[i], (size_t)reqs[i].n * 4, kind, s) != cudaSuccess)
            rc = HCA_ECUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == HCA_OK) rc = HCA_ECUDA;
    const auto now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (int64_t id : ids) {
            hca_server::Job &j = sv->jobs[id];
            j.state = 2;
            j.rc = rc;
            j.t_done = now;
            sv->in_flight -= j.bytes;
        }
    }
    sv->cv_done.notify_all();
}

void worker_main(hca_server *sv) {
    cudaSetDevice(sv->device);
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return;
    Staging stg;
    for (;;) {
        std::vector<int64_t> batch;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_work.wait(lk, [&] { return sv->stop || !sv->queue.empty(); });
            if (sv->stop && sv->queue.empty()) break;
            // admission: queued jobs in arrival order while they fit the budget (a job larger
            // than the whole budget runs alone once nothing else is in flight)
            while (!sv->queue.empty()) {
                const int64_t id = sv->queue.front();
                hca_server::Job &j = sv->jobs[id];
                if (!batch.empty() || sv->in_flight > 0) {
                    if (sv->in_flight + j.bytes > sv->budget) break;
                }
                sv->queue.pop_front();
                j.state = 1;
                sv->in_flight += j.bytes;
                batch.push_back(id);
            }
            if (batch.empty()) {  // budget full: wait for a batch to finish
                sv->cv_done.wait_for(lk, std::chrono::milliseconds(5));
                continue;
            }
        }
        // one batched call per (d, dtype) group, the groups with the fewest point coordinates
        // first (their jobs complete soonest)
        std::map<std::pair<int32_t, int32_t>, std::vector<int64_t>> groups;
        std::map<std::pair<int32_t, int32_t>, int64_t> work;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (int64_t id : batch) {
                const hca_request &r = sv->jobs[id].req;
                groups[{r.d, r.dtype}].push_back(id);
                work[{r.d, r.dtype}] += r.n * r.d;
            }
        }
        std::vector<std::pair<int64_t, std::pair<int32_t, int32_t>>> order;
        for (auto &kv : work) order.push_back({kv.second, kv.first});
        std::sort(order.begin(), order.end());
        for (auto &o : order) run_group(sv, groups[o.second], s, stg);
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
    if (stg.dp) hca::pool_free(stg.dp, s);
    if (stg.dl) hca::pool_free(stg.dl, s);
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
}

}  // namespace

extern "C" int hca_server_create(hca_server **out, int32_t device, int64_t hbm_budget_bytes, int32_t workers) {
    if (!out || hbm_budget_bytes <= 0 || workers < 1 || workers > 16) return HCA_EINVAL;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return HCA_EINVAL;
    hca_server *sv = new hca_server();
    sv->device = device;
    sv->budget = hbm_budget_bytes;
    for (int i = 0; i < workers; ++i) sv->workers.emplace_back(worker_main, sv);
    *out = sv;
    return HCA_OK;
}

extern "C" int hca_server_destroy(hca_server *sv) {
    if (!sv) return HCA_EINVAL;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        for (int64_t id : sv->queue) {
            sv->jobs[id].state = 3;
            sv->jobs[id].rc = HCA_ECANCELED;
        }
        sv->queue.clear();
    }
    sv->cv_work.notify_all();
    for (std::thread &t : sv->workers) t.join();
    delete sv;
    return HCA_OK;
}

extern "C" int hca_submit(hca_server *sv, const hca_request *r, int64_t *ticket) {
    if (!sv || !r || !ticket) return HCA_EINVAL;
    if (r->n < 0 || r->n >= ((int64_t)1 << 31) || r->d < 1 || r->d > 64) return HCA_EINVAL;
    if (r->dtype != HCA_F32 && r->dtype != HCA_F64) return HCA_EINVAL;
    if (!(r->eps > 0.0) || r->eps != r->eps || r->eps > 1.7e308 || r->min_pts < 1) return HCA_EINVAL;
    if (r->n > 0 && (!r->points || !r->labels)) return HCA_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return HCA_ECANCELED;
    const int64_t id = sv->next_ticket++;
    hca_server::Job j;
    j.req = *r;
    j.state = 0;
    j.rc = HCA_OK;
    j.t_submit = Clock::now();
    j.t_done = j.t_submit;
    j.bytes = job_bytes(*r);
    sv->jobs[id] = j;
    sv->queue.push_back(id);
    *ticket = id;
    sv->cv_work.notify_one();
    return HCA_OK;
}

extern "C" int hca_poll(hca_server *sv, int64_t ticket) {
    if (!sv) return HCA_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) return HCA_EINVAL;
    if (it->second.state == 2) return it->second.rc == HCA_OK ? 1 : it->second.rc;
    if (it->second.state == 3) return HCA_ECANCELED;
    return 0;
}

extern "C" int hca_wait(hca_server *sv, int64_t ticket, int64_t timeout_ms, double *latency_ms) {
    if (!sv) return HCA_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) return HCA_EINVAL;
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (it->second.state < 2) {
        if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && it->second.state < 2)
            return HCA_ETIMEDOUT;
        it = sv->jobs.find(ticket);
        if (it == sv->jobs.end()) return HCA_EINVAL;
    }
    const int rc = it->second.state == 3 ? HCA_ECANCELED : it->second.rc;
    if (latency_ms)
        *latency_ms = std::chrono::duration<double, std::milli>(it->second.t_done - it->second.t_submit).count();
    sv->jobs.erase(it);
    return rc;
}

extern "C" int hca_cancel(hca_server *sv, int64_t ticket) {
    if (!sv) return HCA_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) return HCA_EINVAL;
    if (it->second.state != 0) return HCA_EBUSY;
    sv->queue.erase(std::remove(sv->queue.begin(), sv->queue.end(), ticket), sv->queue.end());
    it->second.state = 3;
    it->second.rc = HCA_ECANCELED;
    it->second.t_done = Clock::now();
    sv->cv_done.notify_all();
    return HCA_OK;
}
