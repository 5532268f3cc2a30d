// A process-wide pool of host worker threads for the parallel parts of net
// loading (parsing and placing many nets).  Threads are started once, on
// first use, and wait on a condition variable between jobs, so a batch does
// not pay for creating and joining threads.  One job runs at a time; a
// caller that finds the pool busy (another context loading on another
// thread), or a process forked after the pool started (its workers do not
// exist there), runs the whole job itself.
#pragma once

#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

namespace inet {

class HostPool {
 public:
  using Body = std::function<void(int32_t, int32_t)>;

  // Never destroyed: its threads wait for work until the process ends, and
  // a process forked after they started (which has the objects but not the
  // threads) must not join or detach them when it exits.
  static HostPool& get() {
    static HostPool* pool = new HostPool();
    return *pool;
  }

  // body(lo, hi) over [0, n) in ranges of `grain`, on the workers and the
  // calling thread; returns when every range is done.
  void run(int32_t n, int32_t grain, const Body& body) {
    if (n <= 0) return;
    grain = std::max<int32_t>(1, grain);
    std::unique_lock<std::mutex> job(job_mu_, std::try_to_lock);
    if (n <= grain || !job.owns_lock() || getpid() != pid_) {
      body(0, n);
      return;
    }
    start_workers();
    if (workers_.empty()) {
      body(0, n);
      return;
    }
    {
      std::lock_guard<std::mutex> lk(mu_);
      body_ = &body;
      n_ = n;
      grain_ = grain;
      next_.store(0);
      active_ = (int)workers_.size();
      gen_++;
    }
    cv_.notify_all();
    work(body, n, grain);
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return active_ == 0; });
    body_ = nullptr;
  }

 private:
  HostPool() : pid_(getpid()) {}

  void start_workers() {
    if (started_) return;
    started_ = true;
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const unsigned k = std::min(hw, 16u) - 1;
    for (unsigned i = 0; i < k; i++) workers_.emplace_back([this] { loop(); });
  }

  void work(const Body& body, int32_t n, int32_t grain) {
    for (;;) {
      const int32_t lo = next_.fetch_add(grain);
      if (lo >= n) return;
      body(lo, std::min(n, lo + grain));
    }
  }

  void loop() {
    uint64_t seen = 0;
    for (;;) {
      std::unique_lock<std::mutex> lk(mu_);
      cv_.wait(lk, [&] { return gen_ != seen; });
      seen = gen_;
      const Body* b = body_;
      const int32_t n = n_, grain = grain_;
      lk.unlock();
      work(*b, n, grain);
      lk.lock();
      if (--active_ == 0) done_cv_.notify_all();
    }
  }

  const pid_t pid_;
  bool started_ = false;  // guarded by job_mu_
  std::mutex job_mu_;
  std::mutex mu_;
  std::condition_variable cv_, done_cv_;
  std::vector<std::thread> workers_;
  uint64_t gen_ = 0;
  const Body* body_ = nullptr;
  int32_t n_ = 0, grain_ = 1;
  std::atomic<int32_t> next_{0};
  int active_ = 0;
};

}  // namespace inet
