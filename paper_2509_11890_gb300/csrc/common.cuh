// Shared device plumbing for the TT-SDP library: status codes, error
// propagation, stream-ordered device buffers and small host helpers.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <ctime>
#include <cstdio>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/tt_sdp.h"

namespace ttsdp {

// Every failure inside the library is thrown as TTError and converted to a
// status code at the C boundary; nothing crosses the ABI as an exception.
struct TTError : public std::runtime_error {
  tt_status status;
  TTError(tt_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define TT_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      throw ::ttsdp::TTError(TT_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define TT_CHECK(cond, st, msg)                     \
  do {                                              \
    if (!(cond)) throw ::ttsdp::TTError(st, msg);   \
  } while (0)

inline void check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw TTError(TT_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// The library's single ordered stream (set by the context or per call).
struct StreamScope {
  static cudaStream_t& current() {
    static thread_local cudaStream_t s = nullptr;
    return s;
  }
};
inline cudaStream_t cur_stream() { return StreamScope::current(); }

// The caller's device allocator (tt_allocator) while a call on its context
// runs on this thread; null: the device's default stream-ordered pool.
struct AllocScope {
  static const tt_allocator*& current() {
    static thread_local const tt_allocator* a = nullptr;
    return a;
  }
};

// Device buffer allocated stream-ordered from the device's default memory
// pool, or from the caller's allocator when one is in scope (the buffer
// remembers which, and frees through the same one).
template <typename T>
class DBuf {
 public:
  DBuf() = default;
  explicit DBuf(size_t n) { alloc(n); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p_(o.p_), n_(o.n_), al_(o.al_) { o.p_ = nullptr; o.n_ = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p_ = o.p_; n_ = o.n_; al_ = o.al_; o.p_ = nullptr; o.n_ = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(size_t n) {
    release();
    n_ = n;
    al_ = AllocScope::current();
    if (!n) return;
    if (al_) {
      p_ = static_cast<T*>(al_->alloc(n * sizeof(T), (void*)cur_stream(), al_->user));
      if (!p_) {
        n_ = 0;
        throw TTError(TT_E_NOMEM, "the caller's allocator returned NULL");
      }
    } else {
      TT_CUDA(cudaMallocAsync((void**)&p_, n * sizeof(T), cur_stream()));
    }
  }
  void release() {
    if (p_) {
      if (al_) al_->free(p_, (void*)cur_stream(), al_->user);
      else cudaFreeAsync(p_, cur_stream());
    }
    p_ = nullptr;
    n_ = 0;
  }
  T* get() const { return p_; }
  size_t size() const { return n_; }

 private:
  T* p_ = nullptr;
  size_t n_ = 0;
  const tt_allocator* al_ = nullptr;
};

// Counts kernel launches issued by the library (reported by the benchmark).
struct LaunchCounter {
  static std::atomic<unsigned long long>& value() {
    static std::atomic<unsigned long long> v{0};
    return v;
  }
};
inline void count_launch() { LaunchCounter::value().fetch_add(1, std::memory_order_relaxed); }

inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

// Number of solves running concurrently in this process (tt_sdp_solve_batch
// workers). With more than one, host threads that wait for their stream sleep
// on a blocking-sync event instead of spinning: spinning waiters occupy host
// cores that the other solves need to launch their kernels.
inline std::atomic<int>& concurrent_solves() {
  static std::atomic<int> n{0};
  return n;
}

// Waits until all work queued on st has finished (cudaStreamSynchronize
// semantics).
inline cudaError_t sync_stream(cudaStream_t st) {
  if (concurrent_solves().load(std::memory_order_relaxed) <= 1) return cudaStreamSynchronize(st);
  struct Holder {
    cudaEvent_t ev = nullptr;
    ~Holder() {
      if (ev) cudaEventDestroy(ev);
    }
  };
  static thread_local Holder h;
  if (!h.ev) {
    cudaError_t e = cudaEventCreateWithFlags(&h.ev, cudaEventBlockingSync | cudaEventDisableTiming);
    if (e != cudaSuccess) {
      h.ev = nullptr;
      return e;
    }
  }
  cudaError_t e = cudaEventRecord(h.ev, st);
  if (e != cudaSuccess) return e;
  return cudaEventSynchronize(h.ev);
}

// Phase timer for diagnosing where an iteration spends its time. Enabled by
// the environment variable TTSDP_PROFILE=1; then each scope synchronises the
// current stream on entry and exit and accumulates host wall time per name.
struct Profiler {
  static bool enabled() {
    static int e = -1;
    if (e < 0) {
      const char* v = std::getenv("TTSDP_PROFILE");
      e = (v && v[0] == '1') ? 1 : 0;
    }
    return e == 1;
  }
  static std::vector<std::pair<std::string, double>>& table() {
    static std::vector<std::pair<std::string, double>> t;
    return t;
  }
  static void add(const char* name, double s) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    for (auto& p : table())
      if (p.first == name) {
        p.second += s;
        return;
      }
    table().emplace_back(name, s);
  }
};

struct ProfScope {
  const char* name;
  double t0 = 0.0;
  static double now() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return ts.tv_sec + 1e-9 * ts.tv_nsec;
  }
  explicit ProfScope(const char* n) : name(n) {
    if (Profiler::enabled()) {
      sync_stream(cur_stream());
      t0 = now();
    }
  }
  ~ProfScope() {
    if (Profiler::enabled()) {
      sync_stream(cur_stream());
      Profiler::add(name, now() - t0);
    }
  }
};

}  // namespace ttsdp
