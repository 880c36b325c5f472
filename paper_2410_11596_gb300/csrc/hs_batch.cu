// Batched CTMRG: one move of many independent instances (different D and chi)
// at once. Each instance has its own context (stream, workspace, solver
// handles); a pool of host threads drives the instances' moves concurrently,
// so that the GPU overlaps their kernels across streams. This is the runtime
// around the per-instance move of hs_api.cu, not a new contraction.
#include <chrono>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "hs_ctx.cuh"

namespace hs {
namespace {

// A fixed pool of worker threads that runs a batch of indexed tasks and
// returns when all of them are done.
class Pool {
 public:
  explicit Pool(int n) {
    for (int i = 0; i < n; ++i) workers_.emplace_back([this] { loop(); });
  }
  ~Pool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : workers_) t.join();
  }
  int size() const { return (int)workers_.size(); }

  void run(int ntask, const std::function<void(int)>& fn) {
    std::unique_lock<std::mutex> lk(mu_);
    fn_ = &fn;
    ntask_ = ntask;
    next_ = 0;
    done_ = 0;
    ++gen_;
    cv_.notify_all();
    done_cv_.wait(lk, [this] { return done_ == ntask_; });
    fn_ = nullptr;
  }

 private:
  void loop() {
    long long seen = 0;
    for (;;) {
      std::unique_lock<std::mutex> lk(mu_);
      cv_.wait(lk, [&] { return stop_ || (gen_ != seen && next_ < ntask_); });
      if (stop_) return;
      seen = gen_;
      while (next_ < ntask_) {
        const int i = next_++;
        const std::function<void(int)>* fn = fn_;
        lk.unlock();
        (*fn)(i);
        lk.lock();
        if (++done_ == ntask_) done_cv_.notify_all();
      }
    }
  }

  std::vector<std::thread> workers_;
  std::mutex mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(int)>* fn_ = nullptr;
  int ntask_ = 0, next_ = 0, done_ = 0;
  long long gen_ = 0;
  bool stop_ = false;
};

std::mutex g_pool_mu;
Pool* g_pool = nullptr;

Pool* pool(int nthreads) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool || g_pool->size() != nthreads) {
    delete g_pool;
    g_pool = new Pool(nthreads);
  }
  return g_pool;
}

}  // namespace
}  // namespace hs

using namespace hs;

extern "C" hs_status hs_ctmrg_move_batched(hs_ctx* ctxs, int n, const hs_z2_tensor* const* a, hs_env* const* env,
                                           const int* chi, hs_move_info* info, double* ms, int nthreads) {
  if (n < 0 || (n > 0 && (!ctxs || !a || !env || !chi)) || nthreads < 1 || nthreads > 256)
    return fail(HS_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return HS_OK;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j)
      if (ctxs[i] == ctxs[j]) return fail(HS_ERR_INVALID_ARG, "instances %d and %d share a context", j, i);
  std::vector<hs_status> st(n, HS_OK);
  std::vector<std::string> msg(n);
  pool(nthreads < n ? nthreads : n)->run(n, [&](int i) {
    const auto t0 = std::chrono::steady_clock::now();
    st[i] = hs_ctmrg_move(ctxs[i], a[i], env[i], chi[i], info ? &info[i] : nullptr);
    if (st[i] != HS_OK) msg[i] = hs_last_error();
    if (ms) ms[i] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  });
  for (int i = 0; i < n; ++i)
    if (st[i] != HS_OK) return fail(st[i], "instance %d: %s", i, msg[i].c_str());
  return HS_OK;
}
