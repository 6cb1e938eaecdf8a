// Named CUDA-event timers for the library's launches (sldm_timers_* in sldm.h).
#include <atomic>
#include <cstring>
#include <exception>
#include <string>
#include <map>
#include <mutex>

#include "internal.h"

namespace sldm {

// ---------------------------------------------------------------- device-memory budget
static std::atomic<int64_t> g_bytes{0};
static std::atomic<int64_t> g_budget{0};

void budget_take(size_t bytes) {
  const int64_t b = int64_t(bytes);
  const int64_t now = g_bytes.fetch_add(b) + b;
  const int64_t lim = g_budget.load();
  if (lim > 0 && now > lim) {
    g_bytes.fetch_sub(b);
    throw Error{SLDM_ENOMEM, "device-memory budget exceeded: " + std::to_string(now) + " > " + std::to_string(lim) +
                                 " bytes"};
  }
}
void budget_give(size_t bytes) { g_bytes.fetch_sub(int64_t(bytes)); }

static std::atomic<int> g_lu_stall{0};
bool take_lu_stall() {
  int v = g_lu_stall.load();
  while (v > 0)
    if (g_lu_stall.compare_exchange_weak(v, v - 1)) return true;
  return false;
}

namespace {
struct Pending {
  std::string name;
  cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<cudaEvent_t> g_pool;
std::vector<Pending> g_pending;
thread_local std::vector<std::pair<std::string, cudaEvent_t>> t_open;  // per begin, matched LIFO by end in its thread
std::map<std::string, std::pair<double, int64_t>> g_acc;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void resolve_locked() {
  for (auto& p : g_pending) {
    float ms = 0;
    cudaEventSynchronize(p.b);
    cudaEventElapsedTime(&ms, p.a, p.b);
    auto& acc = g_acc[p.name];
    acc.first += ms;
    acc.second += 1;
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_pending.clear();
}
}  // namespace

thread_local bool t_mute = false;  // this thread's launches are not timed (tuning passes)
bool timers_on() { return g_on && !t_mute; }
void timers_mute(bool m) { t_mute = m; }

void timer_begin(const char* name, cudaStream_t s) {
  std::lock_guard<std::mutex> l(g_mu);
  cudaEvent_t a = get_event();
  cudaEventRecord(a, s);
  t_open.push_back({name, a});
}

void timer_end(cudaStream_t s) {
  std::lock_guard<std::mutex> l(g_mu);
  if (t_open.empty()) return;
  auto o = t_open.back();
  t_open.pop_back();
  cudaEvent_t b = get_event();
  cudaEventRecord(b, s);
  g_pending.push_back({o.first, o.second, b});
  if (g_pending.size() > 4096) resolve_locked();
}

// algorithmic units (bytes, evaluations) of the timed launches, per name
static std::map<std::string, double> g_units;
void timer_units(const char* name, double units) {
  std::lock_guard<std::mutex> l(g_mu);
  if (g_on && !t_mute) g_units[name] += units;
}

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

}  // namespace sldm

namespace {
// host-side failure inside a C entry point (an allocation of the bookkeeping):
// reported as a status, never thrown across the C ABI
int host_failure(const std::exception& e) {
  sldm::set_error(std::string("timers: ") + e.what());
  return SLDM_ENOMEM;
}
}  // namespace

extern "C" {

int sldm_launch_count(int64_t* out) {
  if (!out) return SLDM_EINVAL;
  *out = sldm::g_launches.load(std::memory_order_relaxed);
  return SLDM_OK;
}

int sldm_timers_enable(int32_t on) {
  std::lock_guard<std::mutex> l(sldm::g_mu);
  sldm::g_on = on != 0;
  return SLDM_OK;
}

int sldm_timers_reset(void) {
  try {
    std::lock_guard<std::mutex> l(sldm::g_mu);
    sldm::resolve_locked();
    sldm::g_acc.clear();
    sldm::g_units.clear();
    return SLDM_OK;
  } catch (const std::exception& e) {
    return host_failure(e);
  }
}

int sldm_timer_units(const char* name, double* units) {
  if (!name || !units) return SLDM_EINVAL;
  try {
    std::lock_guard<std::mutex> l(sldm::g_mu);
    auto it = sldm::g_units.find(name);
    *units = it == sldm::g_units.end() ? 0.0 : it->second;
    return SLDM_OK;
  } catch (const std::exception& e) {
    return host_failure(e);
  }
}

int sldm_timer_get(const char* name, double* total_ms, int64_t* count) {
  try {
    std::lock_guard<std::mutex> l(sldm::g_mu);
    sldm::resolve_locked();
    auto it = sldm::g_acc.find(name ? name : "");
    if (total_ms) *total_ms = it == sldm::g_acc.end() ? 0.0 : it->second.first;
    if (count) *count = it == sldm::g_acc.end() ? 0 : it->second.second;
    return SLDM_OK;
  } catch (const std::exception& e) {
    return host_failure(e);
  }
}

int sldm_timer_names(char* buf, size_t len) {
  try {
    std::lock_guard<std::mutex> l(sldm::g_mu);
    sldm::resolve_locked();
    std::string s;
    for (auto& kv : sldm::g_acc) {
      if (!s.empty()) s += ",";
      s += kv.first;
    }
    if (buf && len) {
      size_t n = std::min(len - 1, s.size());
      std::memcpy(buf, s.data(), n);
      buf[n] = 0;
    }
    return SLDM_OK;
  } catch (const std::exception& e) {
    return host_failure(e);
  }
}

}  // extern "C"

extern "C" int sldm_set_device_budget(int64_t bytes) {
  if (bytes < 0) {
    sldm::set_error("set_device_budget: negative budget");
    return SLDM_EINVAL;
  }
  sldm::g_budget.store(bytes);
  return SLDM_OK;
}

extern "C" int sldm_device_bytes(int64_t* in_use) {
  if (!in_use) {
    sldm::set_error("device_bytes: null argument");
    return SLDM_EINVAL;
  }
  *in_use = sldm::g_bytes.load();
  return SLDM_OK;
}

extern "C" int sldm_test_inject(int32_t what, int32_t count) {
  if (what != SLDM_INJECT_LU_STALL || count < 0) {
    sldm::set_error("test_inject: unknown injection or negative count");
    return SLDM_EINVAL;
  }
  sldm::g_lu_stall.store(count);
  return SLDM_OK;
}
