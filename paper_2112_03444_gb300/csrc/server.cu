// Continuous-batching server over hc_track_batch (declared in include/hc.h).
//
// Requests are single system instances queued per problem.  A dispatcher
// thread owns n_streams CUDA streams; whenever a stream is free it takes the
// problem whose oldest pending request has waited longest (no problem holding
// more than half the streams while others wait), packs up to
// max_batch_instances of its pending requests into one batch (one persistent
// launch), and enqueues it if the device memory of the in-flight batches
// plus the new one stays within max_device_bytes.  Finished batches are
// harvested with hc_poll(timeout 0); their per-request slices are copied out
// and waiters are woken.  Requests that arrive while batches run are
// admitted into the next free stream, so their work overlaps on the device.
// Pinned staging buffers are kept per stream and only grow.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "hc.h"
#include "kernels.cuh"

namespace {

constexpr uint32_t kServerMagic = 0x48435356u;  // "HCSV"

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  hc_problem* p = nullptr;
  std::vector<double> input;  // [inputs][2]
  int64_t paths = 0;
  int n = 0;
  std::vector<double> x;
  std::vector<uint8_t> status;
  Clock::time_point t_submit, t_dispatch, t_done;
  int state = 0;  // 0 pending, 1 in flight, 2 done
  hc_status err = HC_OK;
  int batch_instances = 0;
};

struct Pinned {
  void* ptr = nullptr;
  size_t bytes = 0;
  bool ensure(size_t want) {
    if (want <= bytes) return true;
    if (ptr) cudaFreeHost(ptr);
    ptr = nullptr;
    bytes = 0;
    if (cudaMallocHost(&ptr, want) != cudaSuccess) return false;
    bytes = want;
    return true;
  }
  ~Pinned() {
    if (ptr) cudaFreeHost(ptr);
  }
};

struct Slot {
  cudaStream_t stream = nullptr;
  bool busy = false;
  hc_batch* batch = nullptr;
  hc_problem* problem = nullptr;
  std::vector<Request*> reqs;
  size_t bytes = 0;
  Pinned in, x, st, steps;
};

}  // namespace

struct hc_server {
  uint32_t magic = kServerMagic;
  hc_server_config cfg{};
  int device = 0;
  std::vector<std::unique_ptr<Slot>> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::map<hc_problem*, std::deque<Request*>> pending;
  std::unordered_map<uint64_t, Request*> all;
  size_t bytes_inflight = 0;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  int64_t stats[5] = {0, 0, 0, 0, 0};
  int inflight = 0;
};

namespace {

void harvest(hc_server* s) {
  for (auto& sp : s->slots) {
    Slot& sl = *sp;
    if (!sl.busy) continue;
    hc_batch_result r;
    const hc_status rc = hc_poll(sl.batch, 0, &r);
    if (rc == HC_PENDING) continue;
    const auto now = Clock::now();
    for (size_t k = 0; k < sl.reqs.size(); ++k) {
      Request* q = sl.reqs[k];
      const size_t nx = (size_t)q->paths * q->n * 2;
      q->x.resize(nx);
      q->status.resize(q->paths);
      if (rc == HC_OK) {
        std::memcpy(q->x.data(), static_cast<double*>(sl.x.ptr) + k * nx, nx * sizeof(double));
        std::memcpy(q->status.data(), static_cast<uint8_t*>(sl.st.ptr) + k * q->paths, q->paths);
      }
      q->err = rc;
      q->t_done = now;
      q->state = 2;
      s->stats[0] += 1;
    }
    hc_destroy(sl.batch);
    sl.batch = nullptr;
    sl.reqs.clear();
    s->bytes_inflight -= sl.bytes;
    sl.bytes = 0;
    sl.busy = false;
    s->inflight -= 1;
    s->cv_done.notify_all();
  }
}

// Dispatch as many batches as free streams and the memory cap allow.
void dispatch(hc_server* s) {
  for (;;) {
    Slot* free_slot = nullptr;
    for (auto& sp : s->slots)
      if (!sp->busy) {
        free_slot = sp.get();
        break;
      }
    if (!free_slot) return;
    // The problem with the oldest waiting request -- but while other
    // problems have requests waiting, none may hold more than half the
    // streams: long batches of a hard problem (seconds of re-tracking tail)
    // would otherwise take every stream and queue the quick ones behind them.
    int waiting_problems = 0;
    for (auto& kv : s->pending) waiting_problems += kv.second.empty() ? 0 : 1;
    const int share = std::max(1, (int)s->slots.size() / 2);
    hc_problem* best = nullptr;
    Clock::time_point oldest;
    for (auto& kv : s->pending) {
      if (kv.second.empty()) continue;
      if (waiting_problems > 1) {
        int held = 0;
        for (auto& sp : s->slots) held += (sp->busy && sp->problem == kv.first) ? 1 : 0;
        if (held >= share) continue;
      }
      const auto t = kv.second.front()->t_submit;
      if (!best || t < oldest) {
        best = kv.first;
        oldest = t;
      }
    }
    if (!best) return;
    hc_problem_info info;
    hc_problem_query(best, &info);
    std::deque<Request*>& q = s->pending[best];
    const int64_t per = info.device_bytes_per_instance;
    int64_t room = s->cfg.max_device_bytes - (int64_t)s->bytes_inflight;
    int64_t k = std::min<int64_t>((int64_t)q.size(), s->cfg.max_batch_instances);
    if (per > 0) k = std::min<int64_t>(k, room / per);
    if (k < 1) {
      if (s->inflight > 0) return;  // wait for memory to free up
      k = 1;                        // a request larger than the cap runs alone
    }
    Slot& sl = *free_slot;
    const size_t nin = (size_t)info.inputs_per_instance * 2;
    const size_t nx = (size_t)info.paths * info.n * 2;
    if (!sl.in.ensure(k * nin * sizeof(double)) || !sl.x.ensure(k * nx * sizeof(double)) ||
        !sl.st.ensure(k * info.paths) || !sl.steps.ensure(k * info.paths * 3 * sizeof(int32_t))) {
      return;  // host memory exhausted: retry after completions
    }
    std::vector<Request*> take;
    for (int64_t i = 0; i < k; ++i) {
      Request* r = q.front();
      q.pop_front();
      std::memcpy(static_cast<double*>(sl.in.ptr) + i * nin, r->input.data(), nin * sizeof(double));
      take.push_back(r);
    }
    hc_batch_desc b;
    std::memset(&b, 0, sizeof(b));
    b.n_instances = (int32_t)k;
    b.flags = 0;
    if (info.kind != HC_TOTAL_DEGREE)
      b.p1 = static_cast<const double*>(sl.in.ptr);
    else
      b.coef = static_cast<const double*>(sl.in.ptr);
    b.stream = sl.stream;
    b.x_out = static_cast<double*>(sl.x.ptr);
    b.status_out = static_cast<uint8_t*>(sl.st.ptr);
    b.steps_out = static_cast<int32_t*>(sl.steps.ptr);
    hc_batch* bt = nullptr;
    const hc_status rc = hc_track_batch(best, &b, &bt);
    const auto now = Clock::now();
    if (rc != HC_OK) {
      for (Request* r : take) {
        r->err = rc;
        r->t_dispatch = r->t_done = now;
        r->state = 2;
        s->stats[0] += 1;
      }
      s->cv_done.notify_all();
      continue;
    }
    for (Request* r : take) {
      r->t_dispatch = now;
      r->state = 1;
      r->batch_instances = (int)k;
    }
    sl.busy = true;
    sl.batch = bt;
    sl.problem = best;
    sl.reqs = std::move(take);
    sl.bytes = (size_t)(per * k);
    s->bytes_inflight += sl.bytes;
    s->inflight += 1;
    s->stats[1] += 1;
    s->stats[2] = std::max<int64_t>(s->stats[2], s->inflight);
    s->stats[3] = std::max<int64_t>(s->stats[3], (int64_t)s->bytes_inflight);
    s->stats[4] = std::max<int64_t>(s->stats[4], k);
  }
}

void worker_loop(hc_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    harvest(s);
    dispatch(s);
    bool any_pending = false;
    for (auto& kv : s->pending) any_pending = any_pending || !kv.second.empty();
    if (s->inflight > 0)
      s->cv_work.wait_for(lk, std::chrono::microseconds(50));
    else if (!any_pending)
      s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
  }
  // drain: wait for in-flight batches so their streams can be destroyed
  while (s->inflight > 0) {
    harvest(s);
    if (s->inflight > 0) s->cv_work.wait_for(lk, std::chrono::microseconds(200));
  }
}

}  // namespace

namespace hc {
bool destroy_server_if(void* handle, uint32_t magic) {
  if (magic != kServerMagic) return false;
  hc_server* s = static_cast<hc_server*>(handle);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->all) delete kv.second;
  for (auto& sp : s->slots)
    if (sp->stream) cudaStreamDestroy(sp->stream);
  s->slots.clear();
  s->magic = 0;
  delete s;
  return true;
}
}  // namespace hc

extern "C" {

hc_server_config hc_server_default_config(void) {
  hc_server_config c;
  c.n_streams = 4;
  c.max_batch_instances = 64;
  c.max_device_bytes = (int64_t)8 << 30;
  return c;
}

hc_status hc_server_create(const hc_server_config* cfg, hc_server** out) {
  if (!out) return HC_ERR_INVALID;
  hc_server_config c = cfg ? *cfg : hc_server_default_config();
  if (c.n_streams < 1 || c.n_streams > 64 || c.max_batch_instances < 1 || c.max_device_bytes < 1) {
    hc::set_last_error("invalid server configuration");
    return HC_ERR_INVALID;
  }
  hc_server* s = new hc_server;
  s->cfg = c;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    hc::set_last_error("no current CUDA device");
    return HC_ERR_CUDA;
  }
  for (int i = 0; i < c.n_streams; ++i) {
    auto sl = std::make_unique<Slot>();
    if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto& sp : s->slots) cudaStreamDestroy(sp->stream);
      delete s;
      hc::set_last_error("cudaStreamCreate failed");
      return HC_ERR_CUDA;
    }
    s->slots.push_back(std::move(sl));
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return HC_OK;
}

hc_status hc_server_submit(hc_server* s, hc_problem* p, const double* input, uint64_t* request_id) {
  if (!s || s->magic != kServerMagic || !p || !input || !request_id) return HC_ERR_INVALID;
  hc_problem_info info;
  if (hc_problem_query(p, &info) != HC_OK) return HC_ERR_INVALID;
  Request* r = new Request;
  r->p = p;
  r->input.assign(input, input + (size_t)info.inputs_per_instance * 2);
  r->paths = info.paths;
  r->n = info.n;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    s->all[r->id] = r;
    s->pending[p].push_back(r);
  }
  s->cv_work.notify_one();
  *request_id = r->id;
  return HC_OK;
}

hc_status hc_server_wait(hc_server* s, uint64_t request_id, int64_t timeout_us, double* x_out,
                         uint8_t* status_out, hc_request_info* info) {
  if (!s || s->magic != kServerMagic) return HC_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(request_id);
  if (it == s->all.end()) return HC_ERR_INVALID;
  Request* r = it->second;
  const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
  while (r->state != 2) {
    if (timeout_us < 0) {
      s->cv_done.wait(lk);
    } else if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->state != 2) {
      return HC_PENDING;
    }
  }
  if (x_out && !r->x.empty()) std::memcpy(x_out, r->x.data(), r->x.size() * sizeof(double));
  if (status_out && !r->status.empty()) std::memcpy(status_out, r->status.data(), r->status.size());
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->paths = r->paths;
    for (uint8_t v : r->status) {
      info->finite += ((v & 0x7f) == HC_PATH_FINITE);
      info->real += ((v & 0x7f) == HC_PATH_FINITE) && (v & HC_PATH_REAL);
    }
    info->queue_us = std::chrono::duration<double, std::micro>(r->t_dispatch - r->t_submit).count();
    info->latency_us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
    info->batch_instances = r->batch_instances;
  }
  const hc_status err = r->err;
  s->all.erase(it);
  delete r;
  return err;
}

hc_status hc_server_stats(hc_server* s, int64_t* out5) {
  if (!s || s->magic != kServerMagic || !out5) return HC_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  for (int i = 0; i < 5; ++i) out5[i] = s->stats[i];
  return HC_OK;
}

}  // extern "C"
