// Serving loop for Z[x] products (zx_server_*): continuous batching on one GPU.
//
// Requests (products of device operands) enter a FIFO. A worker thread admits the longest
// prefix of the FIFO whose ring buffers fit the free part of a device arena reserved at
// creation and whose estimated time fits the wave budget, lays it out as one batch (the merged launches of zx_batch.cu) and enqueues it on a
// free stream slot; a host function enqueued after the batch marks its requests complete and
// returns their arena block. Requests that arrive while batches run are admitted as soon as a
// slot and enough arena are free, so their work overlaps with the batches already on the GPU.
// The transform state of every admitted request stays in the arena until its product is
// written. Latency is measured from submission to the host function that follows the batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/tftgpu.h"
#include "common.h"
#include "host.h"

struct zx_server;

namespace tftgpu {

namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t kArenaAlign = 256;
constexpr int kMaxWaveProducts = 512;
// A batch completes as a whole, so its size bounds the latency of its requests: a wave takes
// requests until their estimated time (a fixed cost model) reaches this budget, or one request
// exceeds it. A wave runs its ring groups one after another on its slot's stream, so larger
// waves lose concurrency: on GB300, a budget scaled up with the backlog served 0.8x and one
// scaled down by the measured time 0.9x the products per second of this fixed one. The server
// keeps the ratio of measured wave time (enqueue to completion) to the model's estimate, a
// running average, and reports it (zx_server_info.time_scale).
constexpr double kWaveBudgetUs = 20000.0;
constexpr double kScaleMin = 0.05, kScaleMax = 20.0, kScaleWeight = 0.25;

// First-fit allocator over the offsets of one device block; adjacent free ranges merge.
class Arena {
 public:
  void init(size_t bytes) {
    free_.clear();
    free_[0] = bytes;
    used_ = peak_ = 0;
  }
  static size_t round(size_t b) { return (b + kArenaAlign - 1) & ~(kArenaAlign - 1); }
  bool alloc(size_t bytes, size_t *off) {
    bytes = round(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes, next = it->first + bytes;
      free_.erase(it);
      if (rest) free_[next] = rest;
      used_ += bytes;
      peak_ = std::max(peak_, used_);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = round(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t largest() const {
    size_t m = 0;
    for (const auto &kv : free_) m = std::max(m, kv.second);
    return m;
  }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0, peak_ = 0;
};

struct Request {
  int64_t id = 0;
  BatchProduct p;
  size_t bytes = 0;       // arena bound: ring buffers plus one cell of alignment
  size_t desc_bytes = 0;  // descriptor bound
  double est_us = 0;      // estimated device time
  Clock::time_point t_submit, t_done;
  int status = ZX_OK;
};

struct Wave {
  zx_server *srv = nullptr;
  int slot = 0;
  std::vector<Request *> reqs;
  size_t off = 0, bytes = 0;
  double est_us = 0;             // cost-model estimate of the wave
  Clock::time_point t_launch;    // when it was enqueued
};

}  // namespace

}  // namespace tftgpu

struct zx_server {
  int dev = 0;
  size_t cap = 0;
  unsigned char *base = nullptr;
  tftgpu::Arena arena;
  int nslots = 0;
  size_t desc_cap = 0;
  std::vector<cudaStream_t> streams;
  std::vector<unsigned char *> d_desc, h_desc;
  std::vector<char> busy;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<tftgpu::Request *> pending;
  std::vector<tftgpu::Wave *> finished;
  std::deque<tftgpu::Request *> completed;
  int64_t next_id = 1;
  int running = 0;
  bool stop = false;
  std::thread worker;
  int64_t n_submitted = 0, n_completed = 0, n_waves = 0, max_wave = 0;
  int max_running = 0;
  double scale = 1.0;  // learned ratio of measured wave time to the cost model's estimate
};

namespace tftgpu {

namespace {

void CUDART_CB on_wave_done(void *arg) {
  Wave *w = static_cast<Wave *>(arg);
  zx_server *S = w->srv;
  const Clock::time_point t = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (Request *r : w->reqs) r->t_done = t;
    S->finished.push_back(w);
  }
  S->cv.notify_all();
}

// Lay out and enqueue one wave (called without the server lock). Returns false on failure,
// with every request of the wave marked failed.
bool launch_wave(zx_server *S, Wave *w) {
  std::vector<BatchProduct> items;
  std::vector<int> idx;
  for (size_t k = 0; k < w->reqs.size(); k++) {
    items.push_back(w->reqs[k]->p);
    idx.push_back(int(k));
  }
  std::vector<unsigned char> desc;
  BatchLayout lay;
  std::string msg;
  int rc = layout_batch(items, idx, &desc, &lay, &msg);
  cudaError_t ce = cudaSuccess;
  if (rc == ZX_OK && (lay.pool_bytes > w->bytes || desc.size() > S->desc_cap)) rc = ZX_ENOMEM;
  const cudaStream_t s = S->streams[w->slot];
  if (rc == ZX_OK) {
    std::memcpy(S->h_desc[w->slot], desc.data(), desc.size());
    ce = cudaMemcpyAsync(S->d_desc[w->slot], S->h_desc[w->slot], desc.size(), cudaMemcpyHostToDevice, s);
    for (size_t g = 0; ce == cudaSuccess && g < lay.groups.size(); g++)
      ce = enqueue_group(lay.groups[g], S->d_desc[w->slot], S->base + w->off, s);
    if (ce != cudaSuccess) rc = ZX_ECUDA;
  }
  if (rc == ZX_OK) {
    ce = cudaLaunchHostFunc(s, on_wave_done, w);
    if (ce == cudaSuccess) return true;
    rc = ZX_ECUDA;
    // work may be in flight on the slot: wait for it before the arena block is reused
    cudaStreamSynchronize(s);
  }
  for (Request *r : w->reqs) {
    r->status = rc;
    r->t_done = Clock::now();
  }
  return false;
}

void worker_main(zx_server *S) {
  cudaSetDevice(S->dev);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    for (Wave *w : S->finished) {
      if (w->est_us > 0 && !w->reqs.empty() && w->reqs.front()->status == ZX_OK) {
        const double took = std::chrono::duration<double, std::micro>(w->reqs.front()->t_done - w->t_launch).count();
        const double ratio = std::min(kScaleMax, std::max(kScaleMin, took / w->est_us));
        S->scale = (1.0 - kScaleWeight) * S->scale + kScaleWeight * ratio;
      }
      S->arena.release(w->off, w->bytes);
      S->busy[w->slot] = 0;
      S->running--;
      for (Request *r : w->reqs) S->completed.push_back(r);
      S->n_completed += int64_t(w->reqs.size());
      delete w;
    }
    if (!S->finished.empty()) {
      S->finished.clear();
      S->cv.notify_all();
    }
    if (S->stop && S->pending.empty() && S->running == 0) break;
    int slot = -1;
    for (int k = 0; k < S->nslots; k++)
      if (!S->busy[k]) {
        slot = k;
        break;
      }
    if (slot >= 0 && !S->pending.empty()) {
      // the longest FIFO prefix whose ring buffers and descriptors fit
      const size_t avail = S->arena.largest();
      size_t need = 0, dneed = 0;
      size_t take = 0;
      double est = 0;
      for (Request *r : S->pending) {
        if (take >= size_t(kMaxWaveProducts) || need + r->bytes > avail || dneed + r->desc_bytes > S->desc_cap)
          break;
        if (take > 0 && est + r->est_us > kWaveBudgetUs) break;
        need += r->bytes;
        dneed += r->desc_bytes;
        est += r->est_us;
        take++;
      }
      size_t off = 0;
      if (take > 0 && S->arena.alloc(need, &off)) {
        Wave *w = new Wave();
        w->srv = S;
        w->slot = slot;
        w->off = off;
        w->bytes = need;
        w->est_us = est;
        w->t_launch = Clock::now();
        for (size_t k = 0; k < take; k++) {
          w->reqs.push_back(S->pending.front());
          S->pending.pop_front();
        }
        S->busy[slot] = 1;
        S->running++;
        S->n_waves++;
        S->max_running = std::max(S->max_running, S->running);
        S->max_wave = std::max<int64_t>(S->max_wave, int64_t(take));
        lk.unlock();
        const bool ok = launch_wave(S, w);
        lk.lock();
        if (!ok) {
          S->arena.release(w->off, w->bytes);
          S->busy[slot] = 0;
          S->running--;
          for (Request *r : w->reqs) S->completed.push_back(r);
          S->n_completed += int64_t(w->reqs.size());
          delete w;
          S->cv.notify_all();
        }
        continue;
      }
    }
    S->cv.wait(lk);
  }
}

// upper bound on the descriptor bytes of one product inside a wave
size_t desc_bound(const BatchProduct &p) {
  int passes = 0, lt = 0, li = 0, onchip = 0, cl = 0;
  int64_t jobs = 0;
  plan_shape(KIND_TFT, p.l, std::max(p.len_f, p.len_g), p.nf, 0, p.N, &passes, &lt, &jobs, &onchip, &cl);
  plan_shape(KIND_ITFT, p.l, p.nf, p.nf, 0, p.N, &passes, &li, &jobs, &onchip, &cl);
  // pack (2), pointwise and lift items, one segment per launch of two TFTs and one ITFT, and
  // 16-byte alignment slack (the job lists themselves stay in the plan cache)
  return 2 * sizeof(PackItem) + sizeof(PointwiseItem) + sizeof(LiftItem) + size_t(2 * lt + li) * sizeof(Segment) +
         16 * 16;
}

}  // namespace

}  // namespace tftgpu

using namespace tftgpu;

extern "C" {

int zx_server_create(int64_t arena_bytes, int slots, zx_server **out) {
  if (!out) {
    set_error("out is NULL");
    return ZX_EINVAL;
  }
  *out = nullptr;
  if (slots < 1 || slots > 8) {
    set_error("slots must be in [1, 8]");
    return ZX_EINVAL;
  }
  zx_server *S = new zx_server();
  cudaGetDevice(&S->dev);
  if (arena_bytes <= 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete S;
      set_error("cudaMemGetInfo failed");
      return ZX_ECUDA;
    }
    arena_bytes = int64_t(fr / 2);
  }
  S->cap = size_t(arena_bytes) & ~(kArenaAlign - 1);
  S->nslots = slots;
  S->desc_cap = size_t(32) << 20;
  bool ok = cudaMalloc(reinterpret_cast<void **>(&S->base), S->cap) == cudaSuccess;
  for (int k = 0; ok && k < slots; k++) {
    cudaStream_t st;
    unsigned char *d = nullptr, *h = nullptr;
    ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) S->streams.push_back(st);
    ok = ok && cudaMalloc(reinterpret_cast<void **>(&d), S->desc_cap) == cudaSuccess;
    if (d) S->d_desc.push_back(d);
    ok = ok && cudaHostAlloc(reinterpret_cast<void **>(&h), S->desc_cap, cudaHostAllocDefault) == cudaSuccess;
    if (h) S->h_desc.push_back(h);
  }
  if (!ok) {
    for (cudaStream_t st : S->streams) cudaStreamDestroy(st);
    for (unsigned char *d : S->d_desc) cudaFree(d);
    for (unsigned char *h : S->h_desc) cudaFreeHost(h);
    if (S->base) cudaFree(S->base);
    delete S;
    set_error("server allocation failed");
    return ZX_ENOMEM;
  }
  S->busy.assign(size_t(slots), 0);
  S->arena.init(S->cap);
  S->worker = std::thread(worker_main, S);
  *out = S;
  return ZX_OK;
}

int zx_server_submit(zx_server *S, const zx_poly *f, const zx_poly *g, zx_poly *h, int64_t *id) {
  if (!S || !id) {
    set_error("server or id is NULL");
    return ZX_EINVAL;
  }
  Request *r = new Request();
  int rc = device_product(f, g, h, &r->p);
  if (rc) {
    delete r;
    return rc;
  }
  r->bytes = Arena::round(product_pool_bytes(r->p) + size_t(r->p.stride) * 8);
  r->desc_bytes = desc_bound(r->p);
  {
    // three transforms of two passes over nf cells (read and write) at about 700 GB/s, and
    // nf pointwise products of (N/32)^2 word multiply-adds at about 5e12 per second
    const double cell = 8.0 * double(r->p.N / 64 + 1), nw = double(r->p.N / 32);
    r->est_us = 12.0 * double(r->p.nf) * cell / 700e3 + double(r->p.nf) * nw * nw / 5e6 + 20.0;
  }
  if (r->bytes > S->cap || r->desc_bytes > S->desc_cap) {
    const size_t need = r->bytes;
    delete r;
    set_error("the product needs " + std::to_string(need) + " bytes of ring buffers; the server arena holds " +
              std::to_string(S->cap));
    return ZX_ENOMEM;
  }
  h->is_signed = r->p.sgn;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
      delete r;
      set_error("server is shutting down");
      return ZX_EINVAL;
    }
    r->id = S->next_id++;
    r->t_submit = Clock::now();
    S->pending.push_back(r);
    S->n_submitted++;
    *id = r->id;
  }
  S->cv.notify_all();
  return ZX_OK;
}

int zx_server_poll(zx_server *S, int64_t *ids, int32_t *status, double *latency_s, int max, int *count) {
  if (!S || !count || max < 0 || (max > 0 && !ids)) {
    set_error("bad poll arguments");
    return ZX_EINVAL;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  int k = 0;
  while (k < max && !S->completed.empty()) {
    Request *r = S->completed.front();
    S->completed.pop_front();
    ids[k] = r->id;
    if (status) status[k] = r->status;
    if (latency_s) latency_s[k] = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    delete r;
    k++;
  }
  *count = k;
  return ZX_OK;
}

int zx_server_drain(zx_server *S, double timeout_s) {
  if (!S) {
    set_error("server is NULL");
    return ZX_EINVAL;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  auto idle = [S] { return S->pending.empty() && S->running == 0; };
  if (timeout_s < 0) {
    S->cv.wait(lk, idle);
    return ZX_OK;
  }
  if (!S->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), idle)) {
    set_error("requests still pending after the drain timeout");
    return ZX_ETIMEOUT;
  }
  return ZX_OK;
}

int zx_server_stats(zx_server *S, zx_server_info *out) {
  if (!S || !out) {
    set_error("server or out is NULL");
    return ZX_EINVAL;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(out, 0, sizeof *out);
  out->submitted = S->n_submitted;
  out->completed = S->n_completed;
  out->pending = int64_t(S->pending.size());
  out->waves = S->n_waves;
  out->max_wave_products = S->max_wave;
  out->slots = S->nslots;
  out->max_waves_in_flight = S->max_running;
  out->arena_bytes = int64_t(S->cap);
  out->arena_peak_bytes = int64_t(S->arena.peak());
  out->time_scale = S->scale;
  return ZX_OK;
}

int zx_server_destroy(zx_server *S) {
  if (!S) return ZX_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (cudaStream_t st : S->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (unsigned char *d : S->d_desc) cudaFree(d);
  for (unsigned char *h : S->h_desc) cudaFreeHost(h);
  cudaFree(S->base);
  for (Request *r : S->completed) delete r;
  delete S;
  return ZX_OK;
}

}  // extern "C"
