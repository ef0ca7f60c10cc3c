// The batcher of the serving loop's Chebyshev refinements (batch.h): a
// thread that gathers the jobs handed to it and launches them together.
//
// Protocol.  A scene's solve records `ready` on its stream, hands the job
// over and blocks until the job is launched.  The thread takes every waiting
// job of the same W (warps per group) as the oldest one, up to
// kChebMaxJobs, copies them to the device, makes its stream wait for every
// job's `ready`, launches them in one cooperative kernel, records every
// job's `done` and lets their callers go on: each makes its own stream wait
// for its `done`.  Jobs that arrive while a launch runs form the next one.
#include <cuda_runtime.h>

#include <algorithm>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "batch.h"

namespace tk {

// One launch lane: a stream with its own device job array, barrier state
// and pinned upload buffers.  Lanes take turns, so a batch can start while
// the previous one still runs.
struct BatchLane {
    cudaStream_t st = nullptr;
    ChebJob *d_jobs = nullptr;                   // device copy of one launch's jobs
    ChebJob *h_jobs[2] = {nullptr, nullptr};     // pinned upload buffers, alternating
    cudaEvent_t h_free[2] = {nullptr, nullptr};  // the upload from h_jobs[i] has completed
    BatchBarrier *bar = nullptr;
    int upload = 0;
};

class ChebBatcher {
  public:
    int device = 0;
    BatchLane lane[kBatchLanes];
    int next_lane = 0;
    std::mutex mu;
    std::condition_variable cv, cv_launched;
    struct Pending {
        const ChebJob *job;
        cudaEvent_t ready, done;
        bool launched = false, ok = false;
    };
    std::deque<Pending *> q;
    std::thread th;
    bool stop = false;
    long long batches = 0, jobs = 0;
    int max_jobs = 0;

    void loop();
};

void ChebBatcher::loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        cv.wait(lk, [&] { return stop || !q.empty(); });
        if (q.empty()) return;  // stopping
        // the oldest job's W, and every waiting job of the same W (in order)
        const int W = q.front()->job->W;
        std::vector<Pending *> take;
        for (auto it = q.begin(); it != q.end() && (int)take.size() < kChebMaxJobs;) {
            if ((*it)->job->W == W) {
                take.push_back(*it);
                it = q.erase(it);
            } else {
                ++it;
            }
        }
        lk.unlock();
        BatchLane &L = lane[next_lane];
        next_lane = (next_lane + 1) % kBatchLanes;
        ChebJob *h = L.h_jobs[L.upload];
        bool ok = cudaEventSynchronize(L.h_free[L.upload]) == cudaSuccess;  // the buffer's last upload is done
        int tile0 = 0;
        for (size_t i = 0; i < take.size(); ++i) {
            h[i] = *take[i]->job;
            h[i].tile0 = tile0;
            tile0 += batch_tiles(h[i].g);
        }
        const int n = (int)take.size();
        ok = ok && cudaMemcpyAsync(L.d_jobs, h, sizeof(ChebJob) * n, cudaMemcpyHostToDevice, L.st) == cudaSuccess;
        ok = ok && cudaEventRecord(L.h_free[L.upload], L.st) == cudaSuccess;
        L.upload ^= 1;
        for (Pending *p : take) ok = ok && cudaStreamWaitEvent(L.st, p->ready, 0) == cudaSuccess;
        ok = ok && cudaMemsetAsync(L.bar, 0, sizeof(BatchBarrier), L.st) == cudaSuccess;
        ok = ok && launch_cheb_batch(L.st, L.d_jobs, h, n, W, L.bar, kBatchLanes) == cudaSuccess;
        for (Pending *p : take) ok = ok && cudaEventRecord(p->done, L.st) == cudaSuccess;
        if (!ok) cudaGetLastError();  // a launch error stays with this thread: the callers run their own passes
        lk.lock();
        if (ok) {
            batches++;
            jobs += n;
            max_jobs = std::max(max_jobs, n);
        }
        for (Pending *p : take) {
            p->launched = true;
            p->ok = ok;
        }
        cv_launched.notify_all();
    }
}

ChebBatcher *batcher_create() {
    ChebBatcher *b = new (std::nothrow) ChebBatcher();
    if (!b) return nullptr;
    bool ok = cudaGetDevice(&b->device) == cudaSuccess;
    for (int l = 0; l < kBatchLanes && ok; ++l) {
        BatchLane &L = b->lane[l];
        ok = cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking) == cudaSuccess &&
             cudaMalloc((void **)&L.d_jobs, sizeof(ChebJob) * kChebMaxJobs) == cudaSuccess &&
             cudaMalloc((void **)&L.bar, sizeof(BatchBarrier)) == cudaSuccess;
        for (int i = 0; i < 2 && ok; ++i) {
            ok = cudaMallocHost((void **)&L.h_jobs[i], sizeof(ChebJob) * kChebMaxJobs) == cudaSuccess &&
                 cudaEventCreateWithFlags(&L.h_free[i], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventRecord(L.h_free[i], L.st) == cudaSuccess;
        }
    }
    if (!ok) {
        batcher_destroy(b);
        return nullptr;
    }
    b->th = std::thread([b] { b->loop(); });
    return b;
}

void batcher_destroy(ChebBatcher *b) {
    if (!b) return;
    {
        std::lock_guard<std::mutex> lk(b->mu);
        b->stop = true;
        b->cv.notify_all();
    }
    if (b->th.joinable()) b->th.join();
    for (int l = 0; l < kBatchLanes; ++l) {
        BatchLane &L = b->lane[l];
        if (L.st) cudaStreamSynchronize(L.st);
        for (int i = 0; i < 2; ++i) {
            if (L.h_jobs[i]) cudaFreeHost(L.h_jobs[i]);
            if (L.h_free[i]) cudaEventDestroy(L.h_free[i]);
        }
        if (L.d_jobs) cudaFree(L.d_jobs);
        if (L.bar) cudaFree(L.bar);
        if (L.st) cudaStreamDestroy(L.st);
    }
    delete b;
}

bool batcher_run(ChebBatcher *b, const ChebJob &job, cudaEvent_t ready, cudaEvent_t done) {
    if (!b || !batch_eligible(job.g, job.nsteps) || job.W != job.g.wq) return false;
    ChebBatcher::Pending p;
    p.job = &job;
    p.ready = ready;
    p.done = done;
    std::unique_lock<std::mutex> lk(b->mu);
    if (b->stop) return false;
    b->q.push_back(&p);
    b->cv.notify_all();
    b->cv_launched.wait(lk, [&] { return p.launched; });
    return p.ok;
}

void batcher_stats(ChebBatcher *b, long long *batches, long long *jobs, int *max_jobs) {
    std::lock_guard<std::mutex> lk(b->mu);
    if (batches) *batches = b->batches;
    if (jobs) *jobs = b->jobs;
    if (max_jobs) *max_jobs = b->max_jobs;
}

}  // namespace tk
