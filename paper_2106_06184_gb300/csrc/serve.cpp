// Serving: a request loop over many configurations sharing one GPU (no
// counterpart in the paper, which solves one configuration at a time).
//
// A request names a registered model (mesh + background + materials), a
// frequency and plane waves.  Assembled operators stay resident in a cache keyed
// by (model, frequency); a new one is admitted within the device-memory budget
// by evicting the least recently used operators that no worker holds.  Each
// worker thread owns a CUDA stream; it takes the oldest queued request whose
// key no other worker is serving, together with the following requests of the
// same key while their right-hand sides fit in max_batch, and solves them in one
// lockstep GMRES.  Workers serving different keys overlap on the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "internal.h"

namespace sldm {

// ---------------------------------------------------------------- policies (host only)
// LRU cache of sized entries under a byte budget; pinned entries are never evicted.
struct LruCache {
  struct Entry {
    int64_t bytes = 0;
    int pins = 0;
    std::list<int64_t>::iterator pos;
  };
  int64_t budget = 0;  // 0 = unbounded
  int64_t used = 0;
  std::list<int64_t> order;  // front = most recently used
  std::unordered_map<int64_t, Entry> map;

  bool contains(int64_t key) const { return map.count(key) != 0; }
  void touch(int64_t key) {
    Entry& e = map.at(key);
    order.erase(e.pos);
    order.push_front(key);
    e.pos = order.begin();
  }
  // Keys to evict (least recently used first, unpinned) so that `bytes` more fit;
  // ok = false when even evicting every unpinned entry would not make room.
  std::vector<int64_t> victims(int64_t bytes, bool* ok) const {
    std::vector<int64_t> out;
    *ok = true;
    if (budget <= 0) return out;
    int64_t need = used + bytes - budget;
    for (auto it = order.rbegin(); it != order.rend() && need > 0; ++it) {
      const Entry& e = map.at(*it);
      if (e.pins > 0) continue;
      out.push_back(*it);
      need -= e.bytes;
    }
    if (need > 0) *ok = false;
    return out;
  }
  void insert(int64_t key, int64_t bytes) {
    order.push_front(key);
    Entry e;
    e.bytes = bytes;
    e.pos = order.begin();
    map[key] = e;
    used += bytes;
  }
  void erase(int64_t key) {
    auto it = map.find(key);
    if (it == map.end()) return;
    used -= it->second.bytes;
    order.erase(it->second.pos);
    map.erase(it);
  }
};

// The batch a worker takes from a FIFO queue: the oldest request whose key is
// not busy, then the following requests of that key while the right-hand sides
// fit in max_batch (a first request larger than max_batch goes alone).
struct QItem {
  int64_t key;
  int32_t nrhs;
};
static std::vector<size_t> take_batch(const std::vector<QItem>& q, int32_t max_batch,
                                      const std::vector<int64_t>& busy) {
  std::vector<size_t> out;
  size_t first = q.size();
  for (size_t i = 0; i < q.size(); ++i)
    if (std::find(busy.begin(), busy.end(), q[i].key) == busy.end()) {
      first = i;
      break;
    }
  if (first == q.size()) return out;
  out.push_back(first);
  int32_t n = q[first].nrhs;
  if (n >= max_batch) return out;
  for (size_t i = first + 1; i < q.size(); ++i)
    if (q[i].key == q[first].key && n + q[i].nrhs <= max_batch) {
      out.push_back(i);
      n += q[i].nrhs;
    }
  return out;
}

// ---------------------------------------------------------------- the server
struct Model {
  const sldm_mesh* mesh;
  const sldm_stack* stack;
  std::vector<sldm_material> mats;
  int64_t N;
  int64_t bytes_seen = 0;  // device bytes of its last assembled operator (admission estimate)
};

struct Req {
  int64_t ticket;
  int32_t model, nrhs;
  double freq, tol;
  std::vector<double> khat, pol;
  void* x;
  int64_t key;
  sldm_result res{};
  std::string msg;  // the failure's message, if any
  bool done = false;
};

struct CacheSlot {
  sldm_op* op = nullptr;
};

}  // namespace sldm

struct sldm_server {
  sldm_server_opts opts{};
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::vector<std::unique_ptr<sldm::Model>> models;
  std::deque<std::shared_ptr<sldm::Req>> queue;
  std::map<int64_t, std::shared_ptr<sldm::Req>> tickets;
  int64_t next_ticket = 1;
  std::vector<int64_t> busy;  // keys being served
  // cache (guarded by mu)
  sldm::LruCache lru;
  std::unordered_map<int64_t, sldm::CacheSlot> ops;
  std::map<std::pair<int32_t, double>, int64_t> keys;  // (model, frequency) -> key
  std::vector<std::pair<int32_t, double>> key_of;
  // stats (guarded by mu)
  int64_t n_req = 0, n_rhs = 0, n_batch = 0, hits = 0, misses = 0, evictions = 0, rejected = 0;
  std::vector<double> lat;
  std::vector<std::thread> workers;

  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
  void worker_loop();
  sldm_op* acquire(int64_t key, bool* hit, cudaStream_t s);
  void release(int64_t key);
};

using namespace sldm;

// An Error carrying a failed library call's status and its message (the
// message is kept per thread, so it is read here, in the worker).
static Error failed(int rc, const char* what) {
  char buf[512];
  sldm_last_error(buf, sizeof(buf));
  return Error{rc, std::string(what) + ": " + buf};
}

// Destroys evicted operators outside the lock.
static void destroy_ops(std::vector<sldm_op*>& v) {
  for (sldm_op* op : v) sldm_op_destroy(op);
  v.clear();
}

// The operator of `key`, pinned; assembled (after evicting least recently used
// unpinned operators to fit the budget) when not resident.  The key is busy
// (this worker alone serves it), so no other worker assembles it meanwhile.
sldm_op* sldm_server::acquire(int64_t key, bool* hit, cudaStream_t s) {
  std::vector<sldm_op*> dead;
  Model* m = nullptr;
  double freq = 0;
  {
    std::lock_guard<std::mutex> l(mu);
    if (lru.contains(key)) {
      lru.touch(key);
      lru.map.at(key).pins++;
      ++hits;
      *hit = true;
      return ops.at(key).op;
    }
    *hit = false;
    ++misses;
    m = models[key_of[key].first].get();
    freq = key_of[key].second;
    // admission: the model's last operator size, else the global blocks' size
    int64_t est = m->bytes_seen;
    if (est == 0) {
      sldm_mesh_info mi{};
      sldm_mesh_info_get(m->mesh, &mi);
      // complex64 (8 bytes), complex128 or complex64 hi + lo (16 bytes) per entry
      const int64_t es = opts.precision == SLDM_PREC_F32 ? 8 : 16;
      est = (mi.ne * mi.ne + mi.nt * mi.nt) * es;
    }
    bool ok = false;
    const std::vector<int64_t> v = lru.victims(est, &ok);
    if (!ok) {
      ++rejected;
      throw Error{SLDM_ENOMEM, "server: the operator does not fit the cache budget"};
    }
    for (int64_t k : v) {
      dead.push_back(ops.at(k).op);
      ops.erase(k);
      lru.erase(k);
      ++evictions;
    }
  }
  destroy_ops(dead);
  sldm_assemble_opts ao{};
  ao.precision = opts.precision;
  ao.stream = s;
  sldm_op* op = nullptr;
  const int rc = sldm_assemble(m->mesh, m->stack, m->mats.data(), freq, &ao, &op);
  if (rc != SLDM_OK) throw failed(rc, "server: assembly");
  sldm_op_info info{};
  sldm_op_info_get(op, &info);
  std::lock_guard<std::mutex> l(mu);
  m->bytes_seen = info.device_bytes;
  lru.insert(key, info.device_bytes);
  lru.map.at(key).pins = 1;
  ops[key].op = op;
  return op;
}

void sldm_server::release(int64_t key) {
  std::lock_guard<std::mutex> l(mu);
  auto it = lru.map.find(key);
  if (it != lru.map.end() && it->second.pins > 0) it->second.pins--;
}

void sldm_server::worker_loop() {
  cudaSetDevice(device);
  cudaStream_t s = nullptr;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  DBuf<double2> db, dx;
  for (;;) {
    std::vector<std::shared_ptr<Req>> batch;
    int64_t key = -1;
    {
      std::unique_lock<std::mutex> l(mu);
      for (;;) {
        std::vector<QItem> q;
        q.reserve(queue.size());
        for (auto& r : queue) q.push_back({r->key, r->nrhs});
        const std::vector<size_t> pick = take_batch(q, opts.max_batch, busy);
        if (!pick.empty()) {
          key = queue[pick[0]]->key;
          for (size_t i : pick) batch.push_back(queue[i]);
          for (size_t k = pick.size(); k-- > 0;) queue.erase(queue.begin() + int64_t(pick[k]));
          busy.push_back(key);
          break;
        }
        if (stop && queue.empty()) {
          l.unlock();
          db.release();
          dx.release();
          cudaStreamDestroy(s);
          return;
        }
        cv_work.wait(l);
      }
    }
    const double t_start = now();
    int code = SLDM_OK;
    std::string msg;
    bool hit = false;
    int total = 0;
    for (auto& r : batch) total += r->nrhs;
    std::vector<int32_t> iters(batch.size(), 0);
    std::vector<double> relres(batch.size(), 0.0);
    try {
      sldm_op* op = acquire(key, &hit, s);
      const Model* m = models[batch[0]->model].get();
      const int64_t N = m->N;
      // the batch's right-hand sides in request order, solved in slices of max_batch
      std::vector<std::pair<int, int>> cols;  // (request, column)
      for (size_t i = 0; i < batch.size(); ++i)
        for (int c = 0; c < batch[i]->nrhs; ++c) cols.push_back({int(i), c});
      const int mb = opts.max_batch;
      try {
        db.alloc(size_t(N) * std::min(mb, total));
        dx.alloc(size_t(N) * std::min(mb, total));
        for (int c0 = 0; c0 < total; c0 += mb) {
          const int n = std::min(mb, total - c0);
          std::vector<double> kh(3 * size_t(n)), po(3 * size_t(n));
          double tol = 0;
          for (int c = 0; c < n; ++c) {
            const Req& r = *batch[cols[c0 + c].first];
            const int j = cols[c0 + c].second;
            for (int d = 0; d < 3; ++d) {
              kh[3 * c + d] = r.khat[3 * j + d];
              po[3 * c + d] = r.pol[3 * j + d];
            }
            tol = tol == 0 ? r.tol : std::min(tol, r.tol);
          }
          int rc = sldm_rhs_planewave(op, kh.data(), po.data(), n, db.p, SLDM_DEVICE, s);
          if (rc != SLDM_OK) throw failed(rc, "server: right-hand sides");
          sldm_solve_opts so{};
          so.tol = tol;
          so.maxit = opts.maxit;
          sldm_solve_info si{};
          rc = sldm_solve(op, db.p, dx.p, n, &so, &si, SLDM_DEVICE, s);
          if (rc != SLDM_OK && rc != SLDM_ENOTCONV) throw failed(rc, "server: solve");
          if (rc == SLDM_ENOTCONV) code = SLDM_ENOTCONV;
          for (int c = 0; c < n; ++c) {
            const int i = cols[c0 + c].first, j = cols[c0 + c].second;
            double2* dst = reinterpret_cast<double2*>(batch[i]->x) + int64_t(j) * N;
            SLDM_CUDA(cudaMemcpyAsync(dst, dx.p + int64_t(c) * N, size_t(N) * sizeof(double2), cudaMemcpyDeviceToHost, s));
            if (c == 0 || cols[c0 + c - 1].first != i) iters[i] += si.iters;  // once per solve that carries request i
            relres[i] = std::max(relres[i], si.relres);
          }
          SLDM_CUDA(cudaStreamSynchronize(s));
        }
      } catch (...) {
        release(key);
        throw;
      }
      release(key);
    } catch (const Error& e) {
      code = e.code;
      msg = e.msg;
    } catch (const std::exception& e) {
      code = SLDM_EINVAL;
      msg = e.what();
    }
    const double t_done = now();
    {
      std::lock_guard<std::mutex> l(mu);
      busy.erase(std::find(busy.begin(), busy.end(), key));
      ++n_batch;
      for (size_t i = 0; i < batch.size(); ++i) {
        Req& r = *batch[i];
        r.res.code = code;
        r.res.iters = iters[i];
        r.res.relres = relres[i];
        r.res.t_start = t_start;
        r.res.t_done = t_done;
        r.res.cache_hit = hit ? 1 : 0;
        r.res.batch_rhs = total;
        r.msg = msg;
        r.done = true;
        ++n_req;
        n_rhs += r.nrhs;
        lat.push_back(t_done - r.res.t_submit);
      }
    }
    cv_done.notify_all();
    cv_work.notify_all();  // the key is free again
  }
}

#define API_BEGIN try {
#define API_END                            \
  }                                        \
  catch (const sldm::Error& e) {           \
    sldm::set_error(e.msg);                \
    return e.code;                         \
  }                                        \
  catch (const std::exception& e) {        \
    sldm::set_error(e.what());             \
    return SLDM_EINVAL;                    \
  }                                        \
  return SLDM_OK;

extern "C" {

int sldm_server_create(const sldm_server_opts* opts, sldm_server** out) {
  API_BEGIN
  SLDM_REQUIRE(opts && out && opts->workers >= 1 && opts->workers <= 16 && opts->max_batch >= 1 && opts->max_batch <= 32 &&
                   opts->budget_bytes >= 0 && opts->maxit >= 0 &&
                   (opts->precision == SLDM_PREC_F64 || opts->precision == SLDM_PREC_F32 ||
                    opts->precision == SLDM_PREC_F32X2),
               SLDM_EINVAL, "server_create: invalid options");
  auto* srv = new sldm_server();
  srv->opts = *opts;
  srv->t0 = std::chrono::steady_clock::now();
  srv->lru.budget = opts->budget_bytes;
  cudaGetDevice(&srv->device);
  for (int w = 0; w < opts->workers; ++w) srv->workers.emplace_back([srv] { srv->worker_loop(); });
  *out = srv;
  API_END
}

int sldm_server_add_model(sldm_server* srv, const sldm_mesh* mesh, const sldm_stack* stack, const sldm_material* per_obj,
                          int32_t* model) {
  API_BEGIN
  SLDM_REQUIRE(srv && mesh && stack && per_obj && model, SLDM_EINVAL, "server_add_model: invalid arguments");
  sldm_mesh_info mi{};
  int rc = sldm_mesh_info_get(mesh, &mi);
  if (rc != SLDM_OK) return rc;
  auto m = std::make_unique<Model>();
  m->mesh = mesh;
  m->stack = stack;
  m->mats.assign(per_obj, per_obj + mi.nobj);
  m->N = mi.n_unknowns;
  std::lock_guard<std::mutex> l(srv->mu);
  srv->models.push_back(std::move(m));
  *model = int32_t(srv->models.size() - 1);
  API_END
}

int sldm_server_submit(sldm_server* srv, const sldm_request* req, int64_t* ticket) {
  API_BEGIN
  SLDM_REQUIRE(srv && req && ticket && req->nrhs >= 1 && req->khat && req->pol && req->x && req->freq_hz > 0 &&
                   req->tol >= 0,
               SLDM_EINVAL, "server_submit: invalid request");
  auto r = std::make_shared<Req>();
  r->model = req->model;
  r->nrhs = req->nrhs;
  r->freq = req->freq_hz;
  r->tol = req->tol > 0 ? req->tol : 1e-8;
  r->khat.assign(req->khat, req->khat + 3 * size_t(req->nrhs));
  r->pol.assign(req->pol, req->pol + 3 * size_t(req->nrhs));
  r->x = req->x;
  {
    std::lock_guard<std::mutex> l(srv->mu);
    SLDM_REQUIRE(req->model >= 0 && req->model < int32_t(srv->models.size()), SLDM_EINVAL, "server_submit: unknown model");
    SLDM_REQUIRE(!srv->stop, SLDM_EINVAL, "server_submit: the server is stopping");
    const auto kk = std::make_pair(req->model, req->freq_hz);
    auto it = srv->keys.find(kk);
    if (it == srv->keys.end()) {
      it = srv->keys.emplace(kk, int64_t(srv->key_of.size())).first;
      srv->key_of.push_back(kk);
    }
    r->key = it->second;
    r->ticket = srv->next_ticket++;
    r->res.t_submit = srv->now();
    srv->queue.push_back(r);
    srv->tickets[r->ticket] = r;
    *ticket = r->ticket;
  }
  srv->cv_work.notify_one();
  API_END
}

int sldm_server_wait(sldm_server* srv, int64_t ticket, double timeout_s, sldm_result* res) {
  API_BEGIN
  SLDM_REQUIRE(srv && res, SLDM_EINVAL, "server_wait: invalid arguments");
  std::unique_lock<std::mutex> l(srv->mu);
  auto it = srv->tickets.find(ticket);
  SLDM_REQUIRE(it != srv->tickets.end(), SLDM_EINVAL, "server_wait: unknown ticket");
  std::shared_ptr<Req> r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_s < 0) {
    srv->cv_done.wait(l, ready);
  } else if (!srv->cv_done.wait_for(l, std::chrono::duration<double>(timeout_s), ready)) {
    throw Error{SLDM_ETIMEOUT, "server_wait: the request is still pending"};
  }
  *res = r->res;
  srv->tickets.erase(ticket);
  // a failed request's message becomes this thread's last error (sldm_last_error)
  if (r->res.code != SLDM_OK && !r->msg.empty()) set_error(r->msg);
  API_END
}

int sldm_server_stats_get(sldm_server* srv, sldm_server_stats* st) {
  API_BEGIN
  SLDM_REQUIRE(srv && st, SLDM_EINVAL, "server_stats: invalid arguments");
  std::lock_guard<std::mutex> l(srv->mu);
  *st = sldm_server_stats{};
  st->requests = srv->n_req;
  st->rhs = srv->n_rhs;
  st->batches = srv->n_batch;
  st->hits = srv->hits;
  st->misses = srv->misses;
  st->evictions = srv->evictions;
  st->rejected = srv->rejected;
  st->cached_ops = int64_t(srv->ops.size());
  st->cached_bytes = srv->lru.used;
  if (!srv->lat.empty()) {
    std::vector<double> v = srv->lat;
    std::sort(v.begin(), v.end());
    auto q = [&](double p) { return v[std::min(v.size() - 1, size_t(p * double(v.size() - 1) + 0.5))]; };
    st->lat_p50 = q(0.50);
    st->lat_p99 = q(0.99);
    st->lat_max = v.back();
  }
  API_END
}

int sldm_server_flush(sldm_server* srv) {
  API_BEGIN
  SLDM_REQUIRE(srv, SLDM_EINVAL, "server_flush: invalid arguments");
  std::vector<sldm_op*> dead;
  {
    std::lock_guard<std::mutex> l(srv->mu);
    std::vector<int64_t> ks;
    for (auto& kv : srv->lru.map)
      if (kv.second.pins == 0) ks.push_back(kv.first);
    for (int64_t k : ks) {
      dead.push_back(srv->ops.at(k).op);
      srv->ops.erase(k);
      srv->lru.erase(k);
    }
  }
  destroy_ops(dead);
  API_END
}

int sldm_server_destroy(sldm_server* srv) {
  API_BEGIN
  if (!srv) return SLDM_OK;
  {
    std::lock_guard<std::mutex> l(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  for (auto& t : srv->workers) t.join();
  for (auto& kv : srv->ops) sldm_op_destroy(kv.second.op);
  delete srv;
  API_END
}

int sldm_cache_plan(int64_t n, const int64_t* keys, const int64_t* bytes, int64_t budget, int32_t* action,
                    int32_t* evicted) {
  API_BEGIN
  SLDM_REQUIRE(n >= 0 && (n == 0 || (keys && bytes && action && evicted)) && budget >= 0, SLDM_EINVAL,
               "cache_plan: invalid arguments");
  LruCache c;
  c.budget = budget;
  for (int64_t i = 0; i < n; ++i) {
    evicted[i] = 0;
    if (c.contains(keys[i])) {
      c.touch(keys[i]);
      action[i] = 0;
      continue;
    }
    bool ok = false;
    const std::vector<int64_t> v = c.victims(bytes[i], &ok);
    if (!ok) {
      action[i] = 2;
      continue;
    }
    for (int64_t k : v) c.erase(k);
    evicted[i] = int32_t(v.size());
    c.insert(keys[i], bytes[i]);
    action[i] = 1;
  }
  API_END
}

int sldm_batch_plan(int64_t n, const int64_t* keys, const int32_t* nrhs, int32_t max_batch, int32_t* batch) {
  API_BEGIN
  SLDM_REQUIRE(n >= 0 && (n == 0 || (keys && nrhs && batch)) && max_batch >= 1, SLDM_EINVAL,
               "batch_plan: invalid arguments");
  std::vector<QItem> q;
  std::vector<int64_t> idx;
  for (int64_t i = 0; i < n; ++i) {
    SLDM_REQUIRE(nrhs[i] >= 1, SLDM_EINVAL, "batch_plan: nrhs < 1");
    q.push_back({keys[i], nrhs[i]});
    idx.push_back(i);
  }
  int32_t b = 0;
  while (!q.empty()) {
    const std::vector<size_t> pick = take_batch(q, max_batch, {});
    for (size_t i : pick) batch[idx[i]] = b;
    for (size_t k = pick.size(); k-- > 0;) {
      q.erase(q.begin() + int64_t(pick[k]));
      idx.erase(idx.begin() + int64_t(pick[k]));
    }
    ++b;
  }
  API_END
}

}  // extern "C"
