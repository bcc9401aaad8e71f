// Serving: continuous batching of ragged solver jobs behind a non-blocking
// queue (the nefty_serve_* calls of nefty.h).
//
// A Server owns `lanes` worker threads (job slots).  Each lane has its own
// CUDA stream and its own nefty_handle (so its own workspace, budget = total /
// lanes), takes the oldest queued job whenever it is free and runs it through
// the public solver calls on its handle.  The job's checkpoint stride follows
// the lane's memory share (ckpt_every = 0), and submit refuses, with
// NEFTY_ENOMEM, a job whose smallest workspace does not fit a share.
//
// Batched mode: the lanes' handles hand their TMA-staged FP32 sweeps to one
// Batcher instead of launching them.  The Batcher thread repeatedly takes
// every pending sweep (at most kMaxBatch, in arrival order) and launches them
// together as one persistent grid over the whole device
// (tiled::group_tiled): each sweep gets its own range of CTAs, in proportion
// to its work per step, and runs there as in a launch of its own, so the
// sweeps proceed independently.  Each sweep runs time steps until the
// launch's device-time budget has passed and reports the step it reached;
// the sweeps of a launch thus end together whatever their speeds (no CTA
// waits for a slower sweep), and the next launch, composed once this one is
// done, continues each from where it stopped and takes the jobs admitted
// meanwhile.  Ordering: a launch waits for the work each lane issued before
// its sweep (an event per request), and a lane's stream waits for the launch
// that ran its sweep's last step.  Unbatched mode (and the sweeps the
// grouped kernel does not take) runs each lane's own cooperative grid on
// 1 / lanes of the SMs, resident beside the others.  A job's results depend
// on the CTAs it gets (its reduction order), not otherwise on the other
// jobs: alone and in a mix they agree to rounding.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "nefty.h"

namespace nefty {
namespace {

uint64_t steady_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// alpha <- max(alpha - lr * g, floor): one projected gradient step.
template <typename Real>
__global__ void project_step_kernel(Real* alpha, const Real* g, Real lr, Real lo, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const Real a = alpha[i] - lr * g[i];
        alpha[i] = a > lo ? a : lo;
    }
}

bool is_device(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

struct Job {
    uint64_t id = 0;
    nefty_job desc{};
    nefty_job_result res{};
    std::atomic<bool> cancel{false};
};

// One sweep handed to the Batcher: the whole sweep and where it stands.
struct BatchReq {
    tiled::BatchSweep whole{};     // the sweep's full descriptor (all its steps)
    int cursor = 0;                // forward: the next step; adjoint: the next step downwards
    cudaEvent_t ready = nullptr;   // the lane's work before the sweep
    cudaStream_t stream = nullptr; // the lane's stream, ordered after the last launch
    int launches = 0, shared = 0;
    cudaError_t err = cudaSuccess;
    bool finished = false;
    int end() const { return whole.adjoint ? whole.a.n0 : whole.f.n1; }
};

// The part of a sweep that a launch runs: from `cursor` on, at most `cap`
// steps (0: to the end), stopping early once `budget_ns` of device time has
// passed, with the step it reached written to `progress`.  The same
// arithmetic as a launch of its own from that step: increments, the carried
// residual and the per-step choices continue from the workspace.
tiled::BatchSweep resume(const BatchReq& r, int cap, unsigned long long budget_ns, int* progress) {
    tiled::BatchSweep c = r.whole;
    const int m = r.cursor;
    if (!r.whole.adjoint) {
        const tiled::FwdTiled& a = r.whole.f;
        tiled::FwdTiled& f = c.f;
        f.n0 = m;
        f.n1 = cap > 0 ? std::min(a.n1, m + cap) : a.n1;
        f.src = a.src + (m - a.n0);
        f.dst = a.dst + (m - a.n0);
        f.hist0 = std::min(a.hist0 + (m - a.n0), tiled::kRing);
        f.ring_load = m == a.n0 ? a.ring_load : nullptr;
        f.ring_save = a.ring_save ? a.ring_save + (m - a.n0) : nullptr;
        f.carry = m == a.n0 ? a.carry : 1;
        f.c.iters = a.c.iters + (m - a.n0);
        f.c.resid = a.c.resid + (m - a.n0);
        f.loss_add = 1;
        f.budget_ns = budget_ns;
        f.progress = progress;
    } else {
        const tiled::AdjTiled& a = r.whole.a;
        tiled::AdjTiled& b = c.a;
        b.n1 = m;
        b.n0 = cap > 0 ? std::max(a.n0, m - cap) : a.n0;
        b.T = a.T + (b.n0 - a.n0);   // T^n at index n - n0
        b.hist0 = std::min(a.hist0 + (a.n1 - m), tiled::kRing);
        b.carry = m == a.n1 ? a.carry : 1;
        b.c.iters = a.c.iters + (a.n1 - m);
        b.c.resid = a.c.resid + (a.n1 - m);
        b.budget_ns = budget_ns;
        b.progress = progress;
    }
    return c;
}

}  // namespace

class Batcher {
  public:
    Batcher(int device, int chunk_steps, int launch_us)
        : device_(device), chunk_steps_(chunk_steps), launch_us_(launch_us) {}
    ~Batcher() { stop(); }

    nefty_status start(std::string* why) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device_);
        nefty_status st = NEFTY_OK;
        grid_ = std::min(tiled_grid_blocks(device_), tiled::kMaxGrid);
        if (grid_ <= 0) {
            *why = "cannot size the batched solver grid on this device";
            st = NEFTY_ECUDA;
        } else if (cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking) != cudaSuccess ||
                   cudaEventCreateWithFlags(&done_, cudaEventDisableTiming) != cudaSuccess ||
                   cudaMalloc((void**)&progress_dev_, tiled::kMaxBatch * sizeof(int)) != cudaSuccess ||
                   cudaHostAlloc((void**)&progress_host_, tiled::kMaxBatch * sizeof(int), cudaHostAllocDefault) !=
                       cudaSuccess) {
            *why = "cannot create the batcher's stream and progress slots";
            st = NEFTY_ECUDA;
        }
        cudaGetLastError();
        cudaSetDevice(cur);
        if (st != NEFTY_OK) {
            release();
            return st;
        }
        thread_ = std::thread([this] { main(); });
        return NEFTY_OK;
    }

    void stop() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stopping_ = true;
        }
        cv_.notify_all();
        if (thread_.joinable()) thread_.join();
        release();
    }

    int grid() const { return grid_; }
    // Device time of a launch: each of its sweeps runs steps until this much
    // has passed since the launch began (at least one step), so the sweeps of
    // a launch end together whatever their speeds, and a job admitted
    // meanwhile joins within this time.  chunk_steps > 0 also caps the steps
    // of every sweep per launch.
    static constexpr int kDefaultLaunchUs = 20000;
    unsigned long long budget_ns() const {
        return (unsigned long long)(launch_us_ > 0 ? launch_us_ : kDefaultLaunchUs) * 1000ull;
    }

    nefty_status run(const tiled::BatchSweep& whole, int grid, cudaStream_t s, int* launches, int* shared,
                     std::string* why) {
        *launches = *shared = 0;
        if (grid != grid_) {
            *why = "internal error: a batched sweep was sized for another grid";
            return NEFTY_ECUDA;
        }
        BatchReq r;
        r.whole = whole;
        r.cursor = whole.adjoint ? whole.a.n1 : whole.f.n0;
        r.stream = s;
        if (r.cursor == r.end()) return NEFTY_OK;
        if (cudaEventCreateWithFlags(&r.ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(r.ready, s) != cudaSuccess) {
            cudaGetLastError();
            if (r.ready) cudaEventDestroy(r.ready);
            *why = "cannot record the start of a batched sweep";
            return NEFTY_ECUDA;
        }
        {
            std::unique_lock<std::mutex> lk(mu_);
            if (stopping_) {
                cudaEventDestroy(r.ready);
                *why = "the batcher is stopping";
                return NEFTY_EBUSY;
            }
            pending_.push_back(&r);
            cv_.notify_all();
            cv_.wait(lk, [&] { return r.finished; });
        }
        cudaEventDestroy(r.ready);
        *launches = r.launches;
        *shared = r.shared;
        if (r.err != cudaSuccess) {
            *why = std::string("batched solver launch: ") + cudaGetErrorName(r.err);
            return NEFTY_ECUDA;
        }
        return NEFTY_OK;
    }

  private:
    void release() {
        if (done_) cudaEventDestroy(done_);
        done_ = nullptr;
        if (progress_dev_) cudaFree(progress_dev_);
        progress_dev_ = nullptr;
        if (progress_host_) cudaFreeHost(progress_host_);
        progress_host_ = nullptr;
        if (stream_) cudaStreamDestroy(stream_);
        stream_ = nullptr;
    }

    // CTA ranges of the sweeps taken for one launch: shares of the grid in
    // proportion to each sweep's work per step (cells, adjoint sweeps weighted
    // 1.5 for their extra gradient pass and iterations), at least one CTA, at
    // most the CTAs a launch of its own would use (one per two tile-planes).
    // The sweeps that do not fit wait for the next launch; returns how many fit.
    int shares(const std::vector<tiled::BatchSweep>& sw, int* off) const {
        const int n = (int)sw.size();
        std::vector<double> cost(n);
        std::vector<int> cap(n), g(n, 1);
        for (int i = 0; i < n; ++i) {
            const tiled::Common& c = sw[i].adjoint ? sw[i].a.c : sw[i].f.c;
            cost[i] = (double)c.g.S * c.g.nz * (sw[i].adjoint ? 1.5 : 1.0);
            cap[i] = std::max(1, std::min(grid_, (int)(c.g.units / 2)));
        }
        int used = 0, fit = 0;
        for (; fit < n && used + 1 <= grid_; ++fit) used += 1;   // one CTA each first
        if (fit == 0) return 0;
        int left = grid_ - fit;
        double tf = 0.0;
        for (int i = 0; i < fit; ++i) tf += cost[i];
        for (int i = 0; i < fit; ++i) {
            const int add = std::min(cap[i] - 1, (int)((double)(grid_ - fit) * cost[i] / tf));
            g[i] += std::max(0, add);
            left -= std::max(0, add);
        }
        for (bool more = true; left > 0 && more;) {   // the rest, largest first, up to the caps
            more = false;
            int best = -1;
            for (int i = 0; i < fit; ++i)
                if (g[i] < cap[i] && (best < 0 || cost[i] / g[i] > cost[best] / g[best])) best = i;
            if (best >= 0) {
                ++g[best];
                --left;
                more = true;
            }
        }
        off[0] = 0;
        for (int i = 0; i < fit; ++i) off[i + 1] = off[i] + g[i];
        return fit;
    }

    void main() {
        cudaSetDevice(device_);
        tiled::BatchArgs args;
        while (true) {
            std::vector<BatchReq*> take;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return stopping_ || !pending_.empty(); });
                if (pending_.empty()) break;   // stopping, nothing left
                for (BatchReq* r : pending_) {
                    if ((int)take.size() == tiled::kMaxBatch) break;
                    take.push_back(r);
                }
            }
            // one launch with the next part of every request taken (those
            // whose CTA shares fit)
            std::vector<tiled::BatchSweep> sw;
            for (size_t i = 0; i < take.size(); ++i)
                sw.push_back(resume(*take[i], chunk_steps_, budget_ns(), progress_dev_ + i));
            args.n = shares(sw, args.off);
            take.resize(args.n);
            cudaError_t e = cudaSuccess;
            for (int i = 0; i < args.n && e == cudaSuccess; ++i) {
                args.s[i] = sw[i];
                e = cudaStreamWaitEvent(stream_, take[i]->ready, 0);
                // grid-barrier counters: the sweep's launches alternate between its
                // two counters, each launch zeroing the other one at its end (both are
                // zero at the start of every library call)
                tiled::Common& c = args.s[i].adjoint ? args.s[i].a.c : args.s[i].f.c;
                unsigned& par = parity_[c.ctl];
                c.bar_sel = (int)(par & 1u);
                par += 1;
            }
            if (e == cudaSuccess) e = launch_batch_tiled(args, grid_, stream_);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(progress_host_, progress_dev_, (size_t)args.n * sizeof(int),
                                    cudaMemcpyDeviceToHost, stream_);
            if (e == cudaSuccess) e = cudaEventRecord(done_, stream_);
            if (e == cudaSuccess) e = cudaEventSynchronize(done_);   // where each sweep stopped
            if (e != cudaSuccess) cudaGetLastError();
            {
                std::lock_guard<std::mutex> lk(mu_);
                for (int i = 0; i < args.n; ++i) {
                    BatchReq* r = take[i];
                    r->launches += 1;
                    if (args.n > 1) r->shared += 1;
                    if (e != cudaSuccess) r->err = e;
                    else r->cursor = progress_host_[i];
                    if (e != cudaSuccess || r->cursor == r->end()) {
                        // the lane continues after this launch
                        if (e == cudaSuccess) cudaStreamWaitEvent(r->stream, done_, 0);
                        r->finished = true;
                        pending_.erase(std::find(pending_.begin(), pending_.end(), r));
                    }
                }
                ++launches_;
            }
            cv_.notify_all();
        }
    }

    int device_;
    int chunk_steps_;
    int launch_us_;
    int grid_ = 0;
    cudaStream_t stream_ = nullptr;
    cudaEvent_t done_ = nullptr;
    int* progress_dev_ = nullptr;    // [kMaxBatch] where each sweep of the last launch stopped
    int* progress_host_ = nullptr;   // pinned copy
    std::unordered_map<DevCtl*, unsigned> parity_;   // grouped launches per control block
    std::thread thread_;
    std::mutex mu_;
    std::condition_variable cv_;
    std::deque<BatchReq*> pending_;
    bool stopping_ = false;
    long long launches_ = 0;
};

int batcher_grid(Batcher* b) { return b->grid(); }
nefty_status batcher_run(Batcher* b, const tiled::BatchSweep& whole, int grid, cudaStream_t s, int* launches,
                         int* shared, std::string* why) {
    return b->run(whole, grid, s, launches, shared, why);
}

class Server {
  public:
    Server(int device, const nefty_serve_config& cfg) : device_(device), cfg_(cfg) {}

    ~Server() { stop(); }

    nefty_status start(std::string* why) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device_);
        nefty_status st = NEFTY_OK;
        const uint64_t share = cfg_.mem_budget_bytes / (uint64_t)cfg_.lanes;
        if (cfg_.batched >= 0) {
            batcher_ = std::make_unique<Batcher>(device_, cfg_.chunk_steps, cfg_.launch_us);
            st = batcher_->start(why);
            if (st != NEFTY_OK) {
                batcher_.reset();
                cudaSetDevice(cur);
                return st;
            }
        }
        // the probe handle sizes jobs at submit; it never runs work
        st = nefty_create(&probe_, device_, share);
        for (int l = 0; l < cfg_.lanes && st == NEFTY_OK; ++l) {
            nefty_handle* h = nullptr;
            st = nefty_create(&h, device_, share);
            if (st != NEFTY_OK) break;
            set_grid_share(h, cfg_.lanes);
            if (batcher_) set_batcher(h, batcher_.get());
            handles_.push_back(h);
            cudaStream_t s = nullptr;
            if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
                st = NEFTY_ECUDA;
                break;
            }
            streams_.push_back(s);
        }
        if (probe_) {
            set_grid_share(probe_, cfg_.lanes);
            if (batcher_) set_batcher(probe_, batcher_.get());
        }
        cudaSetDevice(cur);
        if (st != NEFTY_OK) {
            *why = std::string("cannot set up the serving lanes: ") + nefty_last_error(nullptr);
            release();
            return st;
        }
        for (int l = 0; l < cfg_.lanes; ++l) threads_.emplace_back([this, l] { lane_main(l); });
        return NEFTY_OK;
    }

    nefty_status submit(const nefty_job& j, uint64_t* id, std::string* why) {
        if (j.kind != NEFTY_JOB_FORWARD && j.kind != NEFTY_JOB_INVERSION) {
            *why = "unknown job kind";
            return NEFTY_EINVAL;
        }
        if (!j.alpha) {
            *why = "job.alpha is NULL";
            return NEFTY_EINVAL;
        }
        if (j.kind == NEFTY_JOB_INVERSION &&
            (j.iters < 1 || !(j.lr > 0) || !(j.alpha_floor > 0) || !j.obs)) {
            *why = "an inversion job needs iters >= 1, lr > 0, alpha_floor > 0 and obs";
            return NEFTY_EINVAL;
        }
        nefty_status st = nefty_problem_check(&j.problem);
        if (st != NEFTY_OK) {
            *why = nefty_last_error(nullptr);
            return st;
        }
        {
            // the job's workspace, planned within one lane's share less what
            // the job holds outside the workspace (inversions: gradient and
            // alpha copy), exactly as its lane will plan it
            std::lock_guard<std::mutex> lk(probe_mu_);
            const uint64_t share = cfg_.mem_budget_bytes / (uint64_t)cfg_.lanes;
            const uint64_t extra = job_extra_bytes(j);
            size_t bytes = 0;
            if (extra < share) {
                const uint64_t old = set_budget(probe_, share - extra);
                st = job_workspace_bytes(probe_, &j.problem, j.kind == NEFTY_JOB_INVERSION, j.alpha, j.T0,
                                         j.q_face, j.q_full, j.obs, &bytes);
                set_budget(probe_, old);
                if (st != NEFTY_OK) {
                    *why = nefty_last_error(probe_);
                    return st;
                }
            }
            if (extra >= share || bytes + extra > share) {
                *why = "the job needs " + std::to_string(bytes + extra) + " bytes, more than a lane's share of " +
                       std::to_string(share);
                return NEFTY_ENOMEM;
            }
        }
        auto job = std::make_shared<Job>();
        job->desc = j;
        job->res.state = NEFTY_JOB_QUEUED;
        job->res.status = NEFTY_OK;
        job->res.lane = -1;
        std::lock_guard<std::mutex> lk(mu_);
        if (stopping_ || (int)queue_.size() >= cfg_.max_queue) {
            *why = stopping_ ? "the server is stopping" : "the serving queue is full";
            return NEFTY_EBUSY;
        }
        job->id = next_id_++;
        job->res.t_submit_ns = steady_ns();
        jobs_[job->id] = job;
        queue_.push_back(job);
        *id = job->id;
        cv_.notify_one();
        return NEFTY_OK;
    }

    nefty_status poll(uint64_t id, nefty_job_result* out) {
        std::lock_guard<std::mutex> lk(mu_);
        auto it = jobs_.find(id);
        if (it == jobs_.end()) return NEFTY_ENOTFOUND;
        *out = it->second->res;
        return NEFTY_OK;
    }

    nefty_status cancel(uint64_t id) {
        std::lock_guard<std::mutex> lk(mu_);
        auto it = jobs_.find(id);
        if (it == jobs_.end()) return NEFTY_ENOTFOUND;
        Job& j = *it->second;
        j.cancel = true;
        if (j.res.state == NEFTY_JOB_QUEUED) {
            queue_.erase(std::remove(queue_.begin(), queue_.end(), it->second), queue_.end());
            j.res.state = NEFTY_JOB_CANCELLED;
            j.res.status = NEFTY_ECANCELLED;
            j.res.t_done_ns = steady_ns();
        }
        return NEFTY_OK;
    }

    void stop() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            if (stopping_ && threads_.empty()) return;
            stopping_ = true;
            for (auto& j : queue_) {
                j->res.state = NEFTY_JOB_CANCELLED;
                j->res.status = NEFTY_ECANCELLED;
                j->res.t_done_ns = steady_ns();
            }
            queue_.clear();
        }
        cv_.notify_all();
        for (auto& t : threads_) t.join();
        threads_.clear();
        release();
    }

  private:
    void release() {
        for (cudaStream_t s : streams_) cudaStreamDestroy(s);
        streams_.clear();
        for (nefty_handle* h : handles_) nefty_destroy(h);
        handles_.clear();
        if (probe_) nefty_destroy(probe_);
        probe_ = nullptr;
        batcher_.reset();   // after the lanes, whose sweeps it runs
    }

    void finish(Job& j, int state, nefty_status st) {
        std::lock_guard<std::mutex> lk(mu_);
        j.res.state = state;
        j.res.status = st;
        j.res.t_done_ns = steady_ns();
    }

    void lane_main(int lane) {
        cudaSetDevice(device_);
        nefty_handle* h = handles_[lane];
        cudaStream_t s = streams_[lane];
        while (true) {
            std::shared_ptr<Job> job;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return stopping_ || !queue_.empty(); });
                if (queue_.empty()) return;   // stopping
                job = queue_.front();
                queue_.pop_front();
                job->res.state = NEFTY_JOB_RUNNING;
                job->res.lane = lane;
                job->res.t_admit_ns = steady_ns();
            }
            run(*job, h, s);
        }
    }

    // Device memory a job holds outside its handle's workspace.
    static uint64_t job_extra_bytes(const nefty_job& j) {
        const uint64_t R = j.problem.prec == NEFTY_FP64 ? 8 : 4;
        const uint64_t N = (uint64_t)j.problem.nx * j.problem.ny * j.problem.nz;
        return j.kind == NEFTY_JOB_INVERSION ? 2 * N * R : 0;   // gradient + alpha copy
    }

    void run(Job& job, nefty_handle* h, cudaStream_t s) {
        // the workspace is planned within the lane's share less the job's other memory
        const uint64_t share = cfg_.mem_budget_bytes / (uint64_t)cfg_.lanes;
        set_budget(h, share - job_extra_bytes(job.desc));
        run_job(job, h, s);
        set_budget(h, share);
    }

    void run_job(Job& job, nefty_handle* h, cudaStream_t s) {
        const nefty_job& j = job.desc;
        nefty_problem p = j.problem;
        p.ckpt_every = p.ckpt_every > 0 ? p.ckpt_every : 0;
        int l0 = 0, s0 = 0;
        batch_counts(h, &l0, &s0);
        if (j.kind == NEFTY_JOB_FORWARD) {
            double loss = 0.0;
            const nefty_status st = nefty_forward(h, &p, j.alpha, j.T0, j.q_face, j.q_steps, j.q_full,
                                                  j.frames_out, nullptr, j.obs, j.obs ? &loss : nullptr, nullptr, s);
            count_launches(job, h, l0, s0);
            {
                std::lock_guard<std::mutex> lk(mu_);
                job.res.loss = loss;
            }
            const bool ok = st == NEFTY_OK || st == NEFTY_ENOTCONV;
            finish(job, ok ? NEFTY_JOB_DONE : NEFTY_JOB_FAILED, st);
            return;
        }
        // inversion: projected gradient steps on a device copy of alpha
        const size_t N = (size_t)p.nx * p.ny * p.nz;
        const bool f64 = p.prec == NEFTY_FP64;
        const size_t R = f64 ? 8 : 4;
        const bool alpha_dev = is_device(j.alpha);
        void* a = alpha_dev ? j.alpha : nullptr;
        void* g = nullptr;
        nefty_status st = NEFTY_OK;
        if (cudaMallocAsync(&g, N * R, s) != cudaSuccess ||
            (!alpha_dev && cudaMallocAsync(&a, N * R, s) != cudaSuccess)) {
            cudaGetLastError();
            st = NEFTY_ENOMEM;
        }
        if (st == NEFTY_OK && !alpha_dev &&
            cudaMemcpyAsync(a, j.alpha, N * R, cudaMemcpyHostToDevice, s) != cudaSuccess)
            st = NEFTY_ECUDA;
        bool cancelled = false;
        for (int it = 0; st == NEFTY_OK && it < j.iters; ++it) {
            if (job.cancel) {
                cancelled = true;
                break;
            }
            double loss = 0.0;
            st = nefty_adjoint_grad(h, &p, a, j.T0, j.q_face, j.q_steps, j.q_full, j.obs, &loss, g, nullptr,
                                    nullptr, s);
            if (st != NEFTY_OK && st != NEFTY_ENOTCONV) break;
            st = NEFTY_OK;
            const unsigned blocks = (unsigned)std::min<size_t>(4096, (N + 255) / 256);
            if (f64)
                project_step_kernel<double><<<blocks, 256, 0, s>>>((double*)a, (const double*)g, j.lr, j.alpha_floor,
                                                                    N);
            else
                project_step_kernel<float><<<blocks, 256, 0, s>>>((float*)a, (const float*)g, (float)j.lr,
                                                                   (float)j.alpha_floor, N);
            if (cudaGetLastError() != cudaSuccess) st = NEFTY_ECUDA;
            count_launches(job, h, l0, s0);
            std::lock_guard<std::mutex> lk(mu_);
            job.res.loss = loss;
            job.res.iters_done = it + 1;
        }
        if (!alpha_dev && a && st == NEFTY_OK &&
            cudaMemcpyAsync(j.alpha, a, N * R, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            st = NEFTY_ECUDA;
        if (g) cudaFreeAsync(g, s);
        if (!alpha_dev && a) cudaFreeAsync(a, s);
        if (cudaStreamSynchronize(s) != cudaSuccess && st == NEFTY_OK) st = NEFTY_ECUDA;
        if (cancelled) finish(job, NEFTY_JOB_CANCELLED, NEFTY_ECANCELLED);
        else finish(job, st == NEFTY_OK ? NEFTY_JOB_DONE : NEFTY_JOB_FAILED, st);
    }

    // launches of the batcher that carried h's sweeps since (l0, s0)
    void count_launches(Job& job, nefty_handle* h, int l0, int s0) {
        int l = 0, sh = 0;
        batch_counts(h, &l, &sh);
        std::lock_guard<std::mutex> lk(mu_);
        job.res.launches = l - l0;
        job.res.shared_launches = sh - s0;
    }

    int device_;
    nefty_serve_config cfg_;
    std::unique_ptr<Batcher> batcher_;
    nefty_handle* probe_ = nullptr;
    std::mutex probe_mu_;
    std::vector<nefty_handle*> handles_;
    std::vector<cudaStream_t> streams_;
    std::vector<std::thread> threads_;
    std::mutex mu_;
    std::condition_variable cv_;
    std::deque<std::shared_ptr<Job>> queue_;
    std::unordered_map<uint64_t, std::shared_ptr<Job>> jobs_;
    uint64_t next_id_ = 1;
    bool stopping_ = false;
};

Server* server_start(int device, const nefty_serve_config* cfg, nefty_status* st, std::string* why) {
    nefty_serve_config c{};
    if (cfg) c = *cfg;
    if (c.lanes == 0) c.lanes = 2;
    if (c.max_queue == 0) c.max_queue = 4096;
    if (c.lanes < 1 || c.lanes > tiled::kMaxBatch || c.max_queue < 1 || c.batched < -1 || c.batched > 1 ||
        c.chunk_steps < 0 || c.launch_us < 0 || c.launch_us > 10000000) {
        *why = "need 1 <= lanes <= 16, max_queue >= 1, batched in {-1, 0, 1}, chunk_steps >= 0 and "
               "0 <= launch_us <= 10000000";
        *st = NEFTY_EINVAL;
        return nullptr;
    }
    if (c.mem_budget_bytes == 0) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        size_t free_b = 0, total_b = 0;
        const cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
        cudaSetDevice(cur);
        if (e != cudaSuccess) {
            *why = std::string("cudaMemGetInfo: ") + cudaGetErrorName(e);
            *st = NEFTY_ECUDA;
            return nullptr;
        }
        c.mem_budget_bytes = (uint64_t)(0.8 * (double)free_b);
    }
    Server* s = new Server(device, c);
    *st = s->start(why);
    if (*st != NEFTY_OK) {
        delete s;
        return nullptr;
    }
    return s;
}
void server_stop(Server* s) { delete s; }
nefty_status server_submit(Server* s, const nefty_job* j, uint64_t* id, std::string* why) {
    return s->submit(*j, id, why);
}
nefty_status server_poll(Server* s, uint64_t id, nefty_job_result* out) { return s->poll(id, out); }
nefty_status server_cancel(Server* s, uint64_t id) { return s->cancel(id); }

}  // namespace nefty
