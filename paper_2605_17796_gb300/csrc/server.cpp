// Continuous-batching decode server over the library's own entry points.
//
// Requests (one shot's syndromes, both sides, for one of several prepared codes) are submitted
// with an arrival time; a dispatcher thread admits each request once its arrival time has
// passed, groups ready requests of one code into a batch as soon as a stream slot is free, and
// keeps up to `streams` batches in flight on the device at once (their kernels overlap). A slot
// owns its device buffers for `max_batch` shots, and the number of slots is set by the memory
// budget. Completion is detected with cudaEventQuery (no host or device spin on the GPU);
// results carry the request id, per-side status, the correction and the latency from arrival to
// completion. Each shot's decode is independent of the others in its batch, so a request's
// result does not depend on what it was batched with. The per-(code, side) tables of Phases 1-2
// (the local posterior table for the code's p and its class tables) are built once when the
// server is created and shared by every batch, so a batch launches only the min-sum kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "lead_internal.h"

namespace lead {
int launch_table(const lead_code* code, int side, double p, float* table, cudaStream_t stream, int estimator,
                 int32_t* iters);
int launch_classify(const lead_code* code, int side, float alpha, int prec, const float* table, void* extra,
                    cudaStream_t stream);
int launch_bp(const lead_code* code, const lead_decode_opts* o, const uint32_t* syn, int64_t shots,
              uint32_t* corr, uint8_t* status, int32_t* iters, float* llr, const float* table,
              cudaStream_t stream, const float* lam_in, void* classes);
size_t table_bytes_of(const lead_code* code, int side);
}  // namespace lead

namespace {

using Clock = std::chrono::steady_clock;

int64_t now_ns(Clock::time_point t0) {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - t0).count();
}

struct Request {
  uint64_t id;
  int32_t code;
  int64_t arrival_ns;          // relative to the server's start
  std::vector<uint32_t> syn;   // words_m[0] + words_m[1] words
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaStream_t stream1 = nullptr;   // side 1's decode, concurrent with side 0's
  cudaEvent_t done = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  uint32_t* d_syn = nullptr;     // max_batch x (wm0 + wm1)
  uint32_t* d_corr = nullptr;    // 2 x max_batch x words_n
  uint8_t* d_status = nullptr;   // 2 x max_batch
  uint32_t* h_syn = nullptr;     // pinned staging
  uint32_t* h_corr = nullptr;
  uint8_t* h_status = nullptr;
  bool busy = false;
  int32_t code = -1;
  std::vector<Request> batch;
};

}  // namespace

struct lead_server {
  std::vector<lead_code*> codes;
  std::vector<double> p_side;
  int32_t sides_mask = 3, max_batch = 0, max_iter = 32, precision = LEAD_PREC_FP32;
  float alpha = 1.0f;
  int32_t wm[2] = {0, 0}, wn = 0;    // maxima over the codes
  std::vector<void*> tables;          // per code, per side: local posterior table + class tables
  int device = 0;
  std::vector<Slot> slots;
  Clock::time_point t0;

  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request> scheduled;        // sorted by arrival
  std::vector<std::deque<Request>> ready;
  std::deque<lead_server_result> results;
  std::deque<std::vector<uint32_t>> result_corr;
  std::atomic<bool> stop{false};
  int error = LEAD_OK;
  std::thread worker;
  int64_t in_flight = 0;
};

namespace {

int launch_batch(lead_server* s, Slot& sl) {
  const lead_code* code = s->codes[sl.code];
  const int n = (int)sl.batch.size();
  const int wm0 = code->side[0].params.words_m, wm1 = code->side[1].params.words_m, wn = code->words_n;
  for (int i = 0; i < n; ++i)
    std::memcpy(sl.h_syn + (size_t)i * (wm0 + wm1), sl.batch[i].syn.data(), sizeof(uint32_t) * (wm0 + wm1));
  // the request layout interleaves sides per shot; the decoder wants one row array per side
  uint32_t* d_side[2] = {sl.d_syn, sl.d_syn + (size_t)s->max_batch * s->wm[0]};
  for (int side = 0; side < 2; ++side) {
    const int w = side ? wm1 : wm0, off = side ? wm0 : 0;
    if (cudaMemcpy2DAsync(d_side[side], sizeof(uint32_t) * w, sl.h_syn + off, sizeof(uint32_t) * (wm0 + wm1),
                          sizeof(uint32_t) * w, n, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
      return LEAD_ECUDA;
  }
  // the two sides decode independently: side 1 on the slot's second stream, joined before the
  // copies back
  const bool both = (s->sides_mask & 3) == 3;
  if (both && (cudaEventRecord(sl.fork, sl.stream) != cudaSuccess ||
               cudaStreamWaitEvent(sl.stream1, sl.fork, 0) != cudaSuccess))
    return LEAD_ECUDA;
  for (int side = 0; side < 2; ++side) {
    if (!((s->sides_mask >> side) & 1)) continue;
    cudaStream_t st = (both && side == 1) ? sl.stream1 : sl.stream;
    lead_decode_opts o{};
    o.side = side;
    o.use_lead = 1;
    o.max_iter = s->max_iter;
    o.precision = s->precision;
    o.alpha = s->alpha;
    o.p = s->p_side[sl.code];
    char* tab = static_cast<char*>(s->tables[2 * (size_t)sl.code + side]);
    int rc = lead::launch_bp(code, &o, d_side[side], n, sl.d_corr + (size_t)side * s->max_batch * s->wn,
                             sl.d_status + (size_t)side * s->max_batch, nullptr, nullptr,
                             reinterpret_cast<const float*>(tab), st, nullptr,
                             tab + lead::table_bytes_of(code, side));
    if (rc != LEAD_OK) return rc;
  }
  if (both && (cudaEventRecord(sl.join, sl.stream1) != cudaSuccess ||
               cudaStreamWaitEvent(sl.stream, sl.join, 0) != cudaSuccess))
    return LEAD_ECUDA;
  for (int side = 0; side < 2; ++side) {
    // device rows have the code's own pitch (words_n); host rows the server's widest pitch
    if (cudaMemcpy2DAsync(sl.h_corr + (size_t)side * s->max_batch * s->wn, sizeof(uint32_t) * s->wn,
                          sl.d_corr + (size_t)side * s->max_batch * s->wn, sizeof(uint32_t) * wn,
                          sizeof(uint32_t) * wn, n, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
      return LEAD_ECUDA;
  }
  if (cudaMemcpyAsync(sl.h_status, sl.d_status, 2 * (size_t)s->max_batch, cudaMemcpyDeviceToHost, sl.stream) !=
          cudaSuccess ||
      cudaEventRecord(sl.done, sl.stream) != cudaSuccess)
    return LEAD_ECUDA;
  return LEAD_OK;
}

void finish_batch(lead_server* s, Slot& sl, int64_t t_done) {
  const lead_code* code = s->codes[sl.code];
  const int wn = code->words_n;
  std::lock_guard<std::mutex> lock(s->mu);
  for (size_t i = 0; i < sl.batch.size(); ++i) {
    const Request& r = sl.batch[i];
    lead_server_result res{};
    res.id = r.id;
    res.code = r.code;
    res.status[0] = ((s->sides_mask >> 0) & 1) ? sl.h_status[i] : 0;
    res.status[1] = ((s->sides_mask >> 1) & 1) ? sl.h_status[s->max_batch + i] : 0;
    res.arrival_ns = r.arrival_ns;
    res.done_ns = t_done;
    std::vector<uint32_t> corr(2 * (size_t)s->wn, 0u);     // side 0 row, side 1 row at offset W
    std::memcpy(corr.data(), sl.h_corr + i * s->wn, sizeof(uint32_t) * wn);
    std::memcpy(corr.data() + s->wn, sl.h_corr + ((size_t)s->max_batch + i) * s->wn, sizeof(uint32_t) * wn);
    s->results.push_back(res);
    s->result_corr.push_back(std::move(corr));
  }
  s->in_flight -= (int64_t)sl.batch.size();
  sl.batch.clear();
  sl.busy = false;
  sl.code = -1;
}

void run(lead_server* s) {
  cudaSetDevice(s->device);
  while (!s->stop.load()) {
    bool worked = false;
    const int64_t t = now_ns(s->t0);
    // completed batches
    for (Slot& sl : s->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaSuccess) {
        finish_batch(s, sl, now_ns(s->t0));
        worked = true;
      } else if (q != cudaErrorNotReady) {
        std::lock_guard<std::mutex> lock(s->mu);
        s->error = LEAD_ECUDA;
      }
    }
    // admit arrived requests, then fill free slots with the code whose oldest request waits longest
    {
      std::unique_lock<std::mutex> lock(s->mu);
      while (!s->scheduled.empty() && s->scheduled.front().arrival_ns <= t) {
        Request r = std::move(s->scheduled.front());
        s->scheduled.pop_front();
        s->ready[r.code].push_back(std::move(r));
      }
      for (Slot& sl : s->slots) {
        if (sl.busy) continue;
        int best = -1;
        for (size_t c = 0; c < s->ready.size(); ++c)
          if (!s->ready[c].empty() &&
              (best < 0 || s->ready[c].front().arrival_ns < s->ready[best].front().arrival_ns))
            best = (int)c;
        if (best < 0) break;
        auto& q = s->ready[best];
        const size_t n = std::min<size_t>(q.size(), (size_t)s->max_batch);
        sl.batch.assign(std::make_move_iterator(q.begin()), std::make_move_iterator(q.begin() + n));
        q.erase(q.begin(), q.begin() + n);
        sl.code = best;
        sl.busy = true;
        s->in_flight += (int64_t)n;
        lock.unlock();
        const int rc = launch_batch(s, sl);
        lock.lock();
        if (rc != LEAD_OK) s->error = rc;
        worked = true;
      }
    }
    if (!worked) std::this_thread::sleep_for(std::chrono::microseconds(2));
  }
}

void free_slots(lead_server* s) {
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.stream1) cudaStreamSynchronize(sl.stream1);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.fork) cudaEventDestroy(sl.fork);
    if (sl.join) cudaEventDestroy(sl.join);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.stream1) cudaStreamDestroy(sl.stream1);
    cudaFree(sl.d_syn);
    cudaFree(sl.d_corr);
    cudaFree(sl.d_status);
    cudaFreeHost(sl.h_syn);
    cudaFreeHost(sl.h_corr);
    cudaFreeHost(sl.h_status);
  }
  s->slots.clear();
  for (void* t : s->tables) cudaFree(t);
  s->tables.clear();
}

// The Phases 1-2 tables of every (code, side) the server decodes, built once on the device.
int build_tables(lead_server* s) {
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return LEAD_ECUDA;
  int rc = LEAD_OK;
  s->tables.assign(2 * s->codes.size(), nullptr);
  for (size_t c = 0; c < s->codes.size() && rc == LEAD_OK; ++c) {
    const lead_code* code = s->codes[c];
    for (int side = 0; side < 2 && rc == LEAD_OK; ++side) {
      if (!((s->sides_mask >> side) & 1)) continue;
      void*& t = s->tables[2 * c + side];
      if (cudaMalloc(&t, lead::decode_workspace_bytes(code, side)) != cudaSuccess) {
        rc = LEAD_EOOM;
        break;
      }
      rc = lead::launch_table(code, side, s->p_side[c], static_cast<float*>(t), st, LEAD_EST_EXACT, nullptr);
      if (rc == LEAD_OK)
        rc = lead::launch_classify(code, side, s->alpha, LEAD_PREC_FP32, static_cast<float*>(t),
                                   static_cast<char*>(t) + lead::table_bytes_of(code, side), st);
      // the storage mode's kernel, compiled and loaded now rather than in the first batch
      if (rc == LEAD_OK) rc = lead::jit_ensure(code, side, s->precision);
    }
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == LEAD_OK) rc = LEAD_ECUDA;
  cudaStreamDestroy(st);
  return rc;
}

}  // namespace

extern "C" {

int lead_server_create(const lead_server_config* cfg, lead_server** out) {
  if (!cfg || !out || cfg->ncodes < 1 || !cfg->codes || !cfg->p_side || cfg->max_batch < 1 || cfg->streams < 1 ||
      cfg->precision < 0 || cfg->precision >= lead::kPrecModes)
    return LEAD_EINVAL;
  *out = nullptr;
  lead_server* s = new (std::nothrow) lead_server();
  if (!s) return LEAD_EOOM;
  s->sides_mask = cfg->sides_mask & 3;
  s->max_batch = cfg->max_batch;
  s->max_iter = cfg->max_iter;
  s->alpha = cfg->alpha;
  s->precision = cfg->precision;
  s->device = -1;
  for (int c = 0; c < cfg->ncodes; ++c) {
    lead_code* code = cfg->codes[c];
    if (!code || code->device < 0 || (s->device >= 0 && code->device != s->device) ||
        !(cfg->p_side[c] > 0.0 && cfg->p_side[c] < 0.5)) {
      delete s;
      return code && code->device < 0 ? LEAD_ESTATE : LEAD_EINVAL;
    }
    s->device = code->device;
    s->codes.push_back(code);
    s->p_side.push_back(cfg->p_side[c]);
    for (int side = 0; side < 2; ++side) s->wm[side] = std::max(s->wm[side], code->side[side].params.words_m);
    s->wn = std::max(s->wn, code->words_n);
  }
  s->ready.resize(cfg->ncodes);
  // memory admission: as many slots as the budget allows, at most cfg->streams
  const size_t per_slot = sizeof(uint32_t) * (size_t)s->max_batch * (s->wm[0] + s->wm[1]) +
                          sizeof(uint32_t) * 2 * (size_t)s->max_batch * s->wn + 2 * (size_t)s->max_batch + 1024;
  const int nslots = (int)std::min<size_t>((size_t)cfg->streams, cfg->budget_bytes / per_slot);
  if (nslots < 1) {
    delete s;
    return LEAD_EOOM;
  }
  if (cudaSetDevice(s->device) != cudaSuccess) {
    delete s;
    return LEAD_ECUDA;
  }
  s->slots.resize(nslots);
  for (Slot& sl : s->slots) {
    const size_t wsyn = (size_t)s->max_batch * (s->wm[0] + s->wm[1]);
    const size_t wcor = 2 * (size_t)s->max_batch * s->wn;
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&sl.stream1, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.join, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&sl.d_syn, sizeof(uint32_t) * wsyn) != cudaSuccess ||
        cudaMalloc(&sl.d_corr, sizeof(uint32_t) * wcor) != cudaSuccess ||
        cudaMalloc(&sl.d_status, 2 * (size_t)s->max_batch) != cudaSuccess ||
        cudaMallocHost(&sl.h_syn, sizeof(uint32_t) * wsyn) != cudaSuccess ||
        cudaMallocHost(&sl.h_corr, sizeof(uint32_t) * wcor) != cudaSuccess ||
        cudaMallocHost(&sl.h_status, 2 * (size_t)s->max_batch) != cudaSuccess) {
      free_slots(s);
      delete s;
      return LEAD_EOOM;
    }
  }
  const int trc = build_tables(s);
  if (trc != LEAD_OK) {
    free_slots(s);
    delete s;
    return trc;
  }
  s->t0 = Clock::now();
  s->worker = std::thread(run, s);
  *out = s;
  return LEAD_OK;
}

int lead_server_submit(lead_server* s, int32_t code, int64_t n, const uint32_t* syn, const uint64_t* ids,
                       const int64_t* arrival_ns) {
  if (!s || code < 0 || code >= (int32_t)s->codes.size() || n < 0 || (n && (!syn || !ids))) return LEAD_EINVAL;
  const lead_code* c = s->codes[code];
  const int w = c->side[0].params.words_m + c->side[1].params.words_m;
  const int64_t t = now_ns(s->t0);
  std::vector<Request> reqs((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    reqs[i].id = ids[i];
    reqs[i].code = code;
    reqs[i].arrival_ns = arrival_ns ? std::max<int64_t>(arrival_ns[i], 0) : t;
    reqs[i].syn.assign(syn + i * w, syn + (i + 1) * w);
  }
  // keep the schedule sorted by arrival: sort the new requests, then one linear merge
  auto by_arrival = [](const Request& x, const Request& y) { return x.arrival_ns < y.arrival_ns; };
  std::stable_sort(reqs.begin(), reqs.end(), by_arrival);
  std::lock_guard<std::mutex> lock(s->mu);
  std::deque<Request> merged;
  std::merge(std::make_move_iterator(s->scheduled.begin()), std::make_move_iterator(s->scheduled.end()),
             std::make_move_iterator(reqs.begin()), std::make_move_iterator(reqs.end()),
             std::back_inserter(merged), by_arrival);
  s->scheduled.swap(merged);
  return s->error;
}

int lead_server_poll(lead_server* s, lead_server_result* out, uint32_t* corr, int64_t max, int64_t* got) {
  if (!s || !got || max < 0 || (max && !out)) return LEAD_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  int64_t k = 0;
  while (k < max && !s->results.empty()) {
    out[k] = s->results.front();
    if (corr) std::memcpy(corr + k * 2 * (size_t)s->wn, s->result_corr.front().data(),
                          sizeof(uint32_t) * s->result_corr.front().size());
    s->results.pop_front();
    s->result_corr.pop_front();
    ++k;
  }
  *got = k;
  return s->error;
}

int lead_server_pending(lead_server* s, int64_t* pending) {
  if (!s || !pending) return LEAD_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  int64_t p = (int64_t)s->scheduled.size() + s->in_flight;
  for (auto& q : s->ready) p += (int64_t)q.size();
  *pending = p;
  return s->error;
}

int lead_server_clock_ns(lead_server* s, int64_t* t) {
  if (!s || !t) return LEAD_EINVAL;
  *t = now_ns(s->t0);
  return LEAD_OK;
}

void lead_server_destroy(lead_server* s) {
  if (!s) return;
  s->stop.store(true);
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  free_slots(s);
  delete s;
}

}  // extern "C"
