// Serving: continuous batching of independent fused SI+SQ requests.
//
// A worker thread owns `slots` contexts (one CUDA stream each).  Submitted
// requests wait in a FIFO; the head is admitted as soon as a slot is free and
// the HBM budget covers its footprint (factor + sweep temporaries, and the
// tensor-core scratch in QSI_FP64_EMU).  Admitted requests are enqueued on
// their slot's stream, so requests that arrive while others run overlap on the
// device.  Completion is detected with a CUDA event per request, after which
// the slot and the budget are released; a timing event before the request's
// first operation and its completion event give its interval on the device
// (against a reference event recorded when the server starts), so overlap
// between requests can be read from the results.  Every request runs the same kernels
// in the same order whatever else is in flight, so its result does not depend
// on the mix.
#include <chrono>
#include <cstdlib>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "qsi_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Ticket {
  qsi_request req;
  qsi_bta A, B, GR, GL;  // copies of the caller's descriptors
  bool has_b = false;
  size_t bytes = 0;
  int state = 0;  // 0 queued, 1 running, 2 done
  int slot = -1;
  qsi_status status = QSI_OK;
  Clock::time_point t_submit, t_admit, t_done;
  qsi_factor *f = nullptr;
  cudaEvent_t ev = nullptr, ev_start = nullptr;  // completion; start (both with timing)
  double dev_start_ms = 0.0, dev_end_ms = 0.0;
};

struct Slot {
  qsi_ctx *ctx = nullptr;
  cudaStream_t stream = nullptr;
  uint64_t busy = 0;  // ticket id, 0 = free
};

}  // namespace

struct qsi_server {
  int device = 0;
  size_t budget = 0, in_use = 0;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Ticket> tickets;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  cudaEvent_t ev_ref = nullptr;  // reference of the requests' device times
};

namespace {

size_t tc_scratch_bound(qsi_shape s) {
  // largest grouped phase: up to 8 products of at most (b+a) x (b+a) with two
  // terms of depth b+a: 34 bf16 planes per operand and 34 int8 residues per
  // element (17 moduli x re/im), with 36 for margin
  const size_t w = (size_t)s.b + s.a;
  return 8 * (36 * w * w + 2 * 2 * 36 * 2 * (w + 128) * (w + 64)) + (1 << 20);
}

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// Enqueue the whole request on its slot (called without the server lock).
qsi_status launch(qsi_server *srv, Ticket &t, Slot &sl) {
  if (cudaEventRecord(t.ev_start, sl.stream) != cudaSuccess) return QSI_ERR_CUDA;
  qsi_status r = qsi_bta_factor(sl.ctx, t.req.shape, &t.A, t.has_b ? &t.B : nullptr, t.req.precision, &t.f);
  if (r == QSI_OK) r = t.has_b ? qsi_bta_selquad(sl.ctx, t.f, &t.GR, &t.GL) : qsi_bta_selinv(sl.ctx, t.f, &t.GR);
  if (t.f) {
    qsi_factor_destroy(t.f);  // stream-ordered: released after the sweeps
    t.f = nullptr;
  }
  if (r == QSI_OK && cudaEventRecord(t.ev, sl.stream) != cudaSuccess) r = QSI_ERR_CUDA;
  (void)srv;
  return r;
}

void worker_loop(qsi_server *srv) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  while (true) {
    // completions
    for (size_t si = 0; si < srv->slots.size(); ++si) {
      Slot &sl = srv->slots[si];
      if (!sl.busy) continue;
      Ticket &t = srv->tickets[sl.busy];
      const cudaError_t q = cudaEventQuery(t.ev);
      if (q == cudaErrorNotReady) continue;
      qsi_status st = (q == cudaSuccess) ? QSI_OK : QSI_ERR_CUDA;
      if (st == QSI_OK) st = qsi_synchronize(sl.ctx);  // stream is idle: reports device-side errors
      float ms0 = 0.f, ms1 = 0.f;
      if (st == QSI_OK && cudaEventElapsedTime(&ms0, srv->ev_ref, t.ev_start) == cudaSuccess &&
          cudaEventElapsedTime(&ms1, srv->ev_ref, t.ev) == cudaSuccess) {
        t.dev_start_ms = ms0;
        t.dev_end_ms = ms1;
      }
      t.status = st;
      t.state = 2;
      t.t_done = Clock::now();
      srv->in_use -= t.bytes;
      sl.busy = 0;
    }
    // admissions, FIFO
    bool launched = false;
    while (!srv->queue.empty()) {
      const uint64_t id = srv->queue.front();
      Ticket &t = srv->tickets[id];
      if (srv->in_use + t.bytes > srv->budget) break;
      int free_slot = -1;
      for (size_t si = 0; si < srv->slots.size(); ++si)
        if (!srv->slots[si].busy) {
          free_slot = (int)si;
          break;
        }
      if (free_slot < 0) break;
      srv->queue.pop_front();
      Slot &sl = srv->slots[free_slot];
      sl.busy = id;
      t.slot = free_slot;
      t.state = 1;
      t.t_admit = Clock::now();
      srv->in_use += t.bytes;
      lk.unlock();
      const qsi_status r = launch(srv, t, sl);
      lk.lock();
      if (r != QSI_OK) {
        // nothing of this request is left in flight that the event would track
        cudaStreamSynchronize(sl.stream);
        t.status = r;
        t.state = 2;
        t.t_done = Clock::now();
        srv->in_use -= t.bytes;
        sl.busy = 0;
      }
      launched = true;
    }
    bool running = false;
    for (const Slot &sl : srv->slots) running |= sl.busy != 0;
    if (srv->stop && !running && srv->queue.empty()) break;
    if (!launched) srv->cv.wait_for(lk, std::chrono::microseconds(running ? 50 : 2000));
  }
}

}  // namespace

extern "C" {

size_t qsi_request_bytes(qsi_shape shape, int with_b, qsi_precision precision) {
  size_t bytes = qsi_factor_bytes(shape, with_b, precision);
  // the server's contexts split the backward sweep unless QSI_BWD_OVERLAP=0 when they are created
  const size_t fw = qsi_forward_tmp_elems(shape.b, shape.a, 1, 1, precision != QSI_FP64 ? shape.n_blocks : 0),
               bw = qsi_backward_tmp_elems(shape.b, shape.a, 1, 1, qsi_bwd_overlap_default());
  bytes += (fw > bw ? fw : bw) * sizeof(zc);
  if (precision != QSI_FP64) bytes += tc_scratch_bound(shape);
  return bytes;
}

qsi_status qsi_serve_create(qsi_server **out, int device, int slots, size_t hbm_budget) {
  if (!out || slots < 1 || slots > 64) return QSI_ERR_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return QSI_ERR_CUDA;
  qsi_server *srv = new (std::nothrow) qsi_server;
  if (!srv) return QSI_ERR_OOM;
  srv->device = device;
  if (hbm_budget == 0) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      delete srv;
      return QSI_ERR_CUDA;
    }
    hbm_budget = free_b / 10 * 9;
  }
  srv->budget = hbm_budget;
  for (int i = 0; i < slots; ++i) {
    Slot sl;
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        qsi_create(&sl.ctx, device, sl.stream) != QSI_OK) {
      for (Slot &s2 : srv->slots) {
        qsi_destroy(s2.ctx);
        cudaStreamDestroy(s2.stream);
      }
      if (sl.stream) cudaStreamDestroy(sl.stream);
      delete srv;
      return QSI_ERR_CUDA;
    }
    srv->slots.push_back(sl);
  }
  if (cudaEventCreate(&srv->ev_ref) != cudaSuccess || cudaEventRecord(srv->ev_ref, srv->slots[0].stream) != cudaSuccess ||
      cudaEventSynchronize(srv->ev_ref) != cudaSuccess) {
    for (Slot &s2 : srv->slots) {
      qsi_destroy(s2.ctx);
      cudaStreamDestroy(s2.stream);
    }
    if (srv->ev_ref) cudaEventDestroy(srv->ev_ref);
    delete srv;
    return QSI_ERR_CUDA;
  }
  srv->worker = std::thread(worker_loop, srv);
  *out = srv;
  return QSI_OK;
}

qsi_status qsi_serve_submit(qsi_server *srv, const qsi_request *req, uint64_t *ticket) {
  if (!srv || !req || !ticket || !req->A || !req->GR) return QSI_ERR_ARG;
  if (req->B && !req->GL) return QSI_ERR_ARG;
  const qsi_shape s = req->shape;
  if (s.n_blocks < 1 || s.b < 1 || s.a < 0) return QSI_ERR_ARG;
  if (!qsi_precision_valid(req->precision))
    return QSI_ERR_UNSUPPORTED;
  Ticket t;
  t.req = *req;
  t.A = *req->A;
  t.GR = *req->GR;
  t.has_b = req->B != nullptr;
  if (t.has_b) {
    t.B = *req->B;
    t.GL = *req->GL;
  }
  t.bytes = qsi_request_bytes(s, t.has_b, req->precision);
  if (t.bytes > srv->budget) return QSI_ERR_BUSY;  // can never be admitted
  if (cudaSetDevice(srv->device) != cudaSuccess) return QSI_ERR_CUDA;
  if (cudaEventCreate(&t.ev) != cudaSuccess) return QSI_ERR_CUDA;
  if (cudaEventCreate(&t.ev_start) != cudaSuccess) {
    cudaEventDestroy(t.ev);
    return QSI_ERR_CUDA;
  }
  t.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) {
      cudaEventDestroy(t.ev);
      cudaEventDestroy(t.ev_start);
      return QSI_ERR_STATE;
    }
    const uint64_t id = srv->next_id++;
    srv->tickets.emplace(id, t);
    srv->queue.push_back(id);
    *ticket = id;
  }
  srv->cv.notify_one();
  return QSI_OK;
}

qsi_status qsi_serve_poll(qsi_server *srv, uint64_t ticket, int *done, qsi_result *res) {
  if (!srv || !done) return QSI_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->tickets.find(ticket);
  if (it == srv->tickets.end()) return QSI_ERR_ARG;
  Ticket &t = it->second;
  *done = t.state == 2;
  if (t.state != 2) return QSI_OK;
  if (res) {
    res->status = t.status;
    res->slot = t.slot;
    res->queue_ms = ms_between(t.t_submit, t.t_admit);
    res->latency_ms = ms_between(t.t_submit, t.t_done);
    res->device_start_ms = t.dev_start_ms;
    res->device_end_ms = t.dev_end_ms;
  }
  cudaEventDestroy(t.ev);
  cudaEventDestroy(t.ev_start);
  srv->tickets.erase(it);
  return QSI_OK;
}

qsi_status qsi_serve_destroy(qsi_server *srv) {
  if (!srv) return QSI_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv.notify_one();
  if (srv->worker.joinable()) srv->worker.join();
  cudaSetDevice(srv->device);
  for (auto &kv : srv->tickets) {
    if (kv.second.ev) cudaEventDestroy(kv.second.ev);
    if (kv.second.ev_start) cudaEventDestroy(kv.second.ev_start);
  }
  if (srv->ev_ref) cudaEventDestroy(srv->ev_ref);
  for (Slot &sl : srv->slots) {
    qsi_destroy(sl.ctx);
    cudaStreamDestroy(sl.stream);
  }
  delete srv;
  return QSI_OK;
}

}  // extern "C"
