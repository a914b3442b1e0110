// qap_server.cu -- continuous-batching solve server of libqapsa (host runtime).
//
// A worker thread owns the GPU side.  Submitted requests wait in a FIFO; the
// worker admits the head of the queue as soon as enough SMs (one per chain, or
// the cluster size for large N) and enough of the device-memory budget are
// free, sets the chain up on its own stream and enqueues its whole run.  Many
// chains are on the device at once and their kernels overlap; a request that
// arrives while others run is admitted the moment a slot and memory free up.
// Each chain's Delta, B', p and counters stay on the device from set-up to the
// end of its run.  Completion is detected with an event per chain; the result
// is read back and the chain's memory freed.  The paper has no counterpart (it
// runs one chain); a chain's trajectory is the one qap_sa_run gives it alone.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "qap_internal.h"
#include "qap_sa.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  int32_t N = 0;
  std::vector<int32_t> A, B, p0;  // freed once the chain is set up
  qap_schedule sched{};
  uint64_t seed = 0, iters = 0;
  int sms = 1;
  size_t bytes = 0;
  Clock::time_point t_submit, t_start, t_done;
  qap_sa *h = nullptr;
  cudaEvent_t done_ev = nullptr;
  bool done = false;
  int32_t status = QAP_OK;
  int64_t cost = 0;
  uint64_t accepts = 0;
  std::vector<int32_t> p;
};

}  // namespace

struct qap_server {
  qap_server_cfg cfg{};
  int device = 0;
  int max_sms = 0;
  size_t budget = 0;
  std::mutex mu;
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> by_ticket;
  std::vector<std::shared_ptr<Request>> running;  // worker thread only
  int sms_used = 0;
  size_t bytes_used = 0;
  uint64_t next_ticket = 1;
  std::atomic<bool> stopping{false};
  std::atomic<int> max_running{0};
  std::thread worker;
  // admitted requests wait here for a set-up thread (under mu); set-up threads
  // hand started chains to the worker through `started` (under mu)
  std::deque<std::shared_ptr<Request>> setup_q;
  std::vector<std::shared_ptr<Request>> started;
  int in_setup = 0;             // admitted, not yet started or failed (under mu)
  int head_bypassed = 0;        // requests admitted past a head that did not fit
  std::condition_variable setup_cv;
  std::vector<std::thread> setup_threads;
};

namespace {

void finish(qap_server *s, const std::shared_ptr<Request> &r) {
  std::vector<int32_t> p(r->N);
  int64_t cost = 0;
  uint64_t acc = 0;
  int st = qap_sa_sync(r->h);
  if (st == QAP_OK) st = qap_sa_result(r->h, p.data(), &cost, &acc);
  qap_sa_destroy(r->h);
  r->h = nullptr;
  cudaEventDestroy(r->done_ev);
  r->done_ev = nullptr;
  std::lock_guard<std::mutex> lock(s->mu);
  r->p.swap(p);
  r->cost = cost;
  r->accepts = acc;
  r->status = st;
  r->t_done = Clock::now();
  r->done = true;
  s->sms_used -= r->sms;
  s->bytes_used -= r->bytes;
}

// Sets the chain up on its own stream and enqueues its whole run; false if
// the request failed (its status is recorded).
bool launch(qap_server *s, const std::shared_ptr<Request> &r) {
  qap_sa *h = nullptr;
  int st = qap_sa_create(r->A.data(), r->B.data(), r->N, r->p0.data(), &r->sched,
                         r->seed, &h);
  if (st == QAP_OK) qapsa_keep_delta_mode(h);  // one launch per piece: SMs held
  if (st == QAP_OK) st = qap_sa_run_async(h, r->iters);
  cudaEvent_t ev = nullptr;
  if (st == QAP_OK && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
    st = QAP_E_CUDA;
  if (st == QAP_OK && cudaEventRecord(ev, qapsa_handle_stream(h)) != cudaSuccess)
    st = QAP_E_CUDA;
  std::vector<int32_t>().swap(r->A);
  std::vector<int32_t>().swap(r->B);
  if (st != QAP_OK) {
    if (ev) cudaEventDestroy(ev);
    qap_sa_destroy(h);
    std::lock_guard<std::mutex> lock(s->mu);
    r->status = st;
    r->t_done = Clock::now();
    r->done = true;
    s->sms_used -= r->sms;
    s->bytes_used -= r->bytes;
    return false;
  }
  r->h = h;
  r->done_ev = ev;
  return true;
}

// Requests that may be admitted past a head waiting for SMs or memory, before
// the head is waited for: small requests fill the gaps a cluster-sized head
// leaves, and the head is not starved.
constexpr int kMaxBypass = 32;
constexpr int kSetupThreads = 4;

// Set-up threads: create each admitted chain on its own stream and enqueue its
// whole run, off the worker's path (a set-up waits for its kernels).
void setup_main(qap_server *s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->setup_cv.wait(lock, [s] { return !s->setup_q.empty() || s->stopping.load(); });
      if (s->setup_q.empty()) {
        if (s->stopping.load()) return;
        continue;
      }
      r = s->setup_q.front();
      s->setup_q.pop_front();
    }
    const bool ok = launch(s, r);
    std::lock_guard<std::mutex> lock(s->mu);
    --s->in_setup;
    if (ok) s->started.push_back(r);
  }
}

void worker_main(qap_server *s) {
  cudaSetDevice(s->device);
  for (;;) {
    bool progress = false;
    {  // chains the set-up threads have started
      std::lock_guard<std::mutex> lock(s->mu);
      for (auto &r : s->started) s->running.push_back(r);
      if (!s->started.empty()) progress = true;
      s->started.clear();
    }
    if ((int)s->running.size() > s->max_running.load())
      s->max_running.store((int)s->running.size());
    // ---- completions ----
    for (size_t i = 0; i < s->running.size();) {
      const std::shared_ptr<Request> &r = s->running[i];
      if (cudaEventQuery(r->done_ev) == cudaErrorNotReady) {
        ++i;
        continue;
      }
      finish(s, r);
      s->running[i] = s->running.back();
      s->running.pop_back();
      progress = true;
    }
    // ---- admissions: arrival order, as SMs and memory allow; while the head
    //      waits for room, up to kMaxBypass later requests that fit may pass it ----
    {
      std::lock_guard<std::mutex> lock(s->mu);
      auto fits = [s](const Request &q) {
        return s->sms_used + q.sms <= s->max_sms && s->bytes_used + q.bytes <= s->budget;
      };
      auto admit = [s](std::deque<std::shared_ptr<Request>>::iterator it) {
        std::shared_ptr<Request> r = *it;
        s->sms_used += r->sms;
        s->bytes_used += r->bytes;
        r->t_start = Clock::now();
        ++s->in_setup;
        s->setup_q.push_back(r);
        return s->queue.erase(it);
      };
      bool admitted = false;
      while (!s->queue.empty()) {
        Request &head = *s->queue.front();
        const bool nothing_on_gpu = s->running.empty() && s->in_setup == 0;
        if (fits(head) || nothing_on_gpu) {  // an oversize request runs alone
          admit(s->queue.begin());
          s->head_bypassed = 0;
          admitted = true;
          continue;
        }
        for (auto it = s->queue.begin() + 1;
             it != s->queue.end() && s->head_bypassed < kMaxBypass;) {
          if (fits(**it)) {
            it = admit(it);
            ++s->head_bypassed;
            admitted = true;
          } else {
            ++it;
          }
        }
        break;  // the head waits for a slot to free up
      }
      if (admitted) {
        progress = true;
        s->setup_cv.notify_all();
      }
    }
    if (!progress) {
      bool idle;
      {
        std::lock_guard<std::mutex> lock(s->mu);
        idle = s->queue.empty() && s->running.empty() && s->in_setup == 0 &&
               s->started.empty();
      }
      if (idle && s->stopping.load()) return;
      std::this_thread::sleep_for(std::chrono::microseconds(idle ? 200 : 20));
    }
  }
}

}  // namespace

extern "C" {

int qap_server_start(const qap_server_cfg *cfg, qap_server **out) {
  if (!out) return QAP_E_INVAL;
  *out = nullptr;
  qap_server *s = new (std::nothrow) qap_server();
  if (!s) return QAP_E_NOMEM;
  if (cfg) s->cfg = *cfg;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return QAP_E_CUDA;
  }
  int sms = 0;
  size_t free_b = 0, total_b = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess ||
      cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    delete s;
    return QAP_E_CUDA;
  }
  // Chains fill at most all SMs but a few: an SM that holds one (255 registers
  // a thread at 256 threads, or 96 at 640) has no room left for another block,
  // so the set-up kernels of an admission -- which the worker waits for -- and
  // the cluster tier's Delta rebuilds need SMs that no chain occupies.
  constexpr int kFreeSMs = 4;
  s->max_sms = (s->cfg.max_sms > 0 && s->cfg.max_sms < sms) ? s->cfg.max_sms
                                                             : (sms > 2 * kFreeSMs ? sms - kFreeSMs : sms);
  s->budget = s->cfg.mem_budget_bytes ? (size_t)s->cfg.mem_budget_bytes
                                      : (size_t)(0.8 * (double)free_b);
  // Grow the device's default pool once, now, while nothing runs: growing it
  // later, with chains on the device, would synchronise with them.  The
  // library keeps freed pool memory (release threshold raised at set-up).
  {
    qap_sa_max_n();  // device attributes and pool settings initialised
    const size_t reserve = s->budget < ((size_t)4 << 30) ? s->budget : ((size_t)4 << 30);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
      uint64_t keep = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      void *p = nullptr;
      if (cudaMallocAsync(&p, reserve, 0) == cudaSuccess) cudaFreeAsync(p, 0);
      cudaStreamSynchronize(0);
    }
    cudaGetLastError();
  }
  s->worker = std::thread(worker_main, s);
  for (int k = 0; k < kSetupThreads; ++k) s->setup_threads.emplace_back(setup_main, s);
  *out = s;
  return QAP_OK;
}

int qap_server_submit(qap_server *s, const qap_problem *q, uint64_t iters,
                      uint64_t *ticket) {
  if (!s || !q || !ticket || !q->A || !q->B || !q->p0 || q->N < 2) return QAP_E_INVAL;
  if (s->stopping.load()) return QAP_E_STATE;
  if (iters > q->sched.total_iters) return QAP_E_RANGE;
  if (q->N > qap_sa_max_n_tier(2)) return QAP_E_UNSUPPORTED;
  // The server shares the GPU between chains of one SM or one cluster each; a
  // chain that needs the grid tier (general instance, wide entries, random
  // order) is not served.
  if (q->sched.flags & QAP_ORDER_RANDOM) return QAP_E_UNSUPPORTED;
  {
    const int32_t N = q->N;
    for (int32_t i = 0; i < N; ++i)
      for (int32_t j = 0; j < N; ++j) {
        const int32_t a = q->A[(size_t)i * N + j], b = q->B[(size_t)i * N + j];
        if (a != q->A[(size_t)j * N + i] || b != q->B[(size_t)j * N + i] ||
            (i == j && (a != 0 || b != 0)) || a > 127 || a < -127 || b > 127 || b < -127)
          return QAP_E_UNSUPPORTED;
      }
  }
  auto r = std::make_shared<Request>();
  const size_t nn = (size_t)q->N * q->N;
  r->N = q->N;
  r->A.assign(q->A, q->A + nn);
  r->B.assign(q->B, q->B + nn);
  r->p0.assign(q->p0, q->p0 + q->N);
  r->sched = q->sched;
  r->seed = q->seed;
  r->iters = iters;
  r->sms = qapsa_sms_for(q->N);
  r->bytes = qapsa_bytes_for(q->N);
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lock(s->mu);
  r->ticket = s->next_ticket++;
  s->queue.push_back(r);
  s->by_ticket[r->ticket] = r;
  *ticket = r->ticket;
  return QAP_OK;
}

int qap_server_poll(qap_server *s, uint64_t ticket, qap_result *out, int32_t *p_out) {
  if (!s || !out) return QAP_E_INVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->by_ticket.find(ticket);
  if (it == s->by_ticket.end()) return QAP_E_INVAL;
  const Request &r = *it->second;
  out->done = r.done ? 1 : 0;
  out->status = r.status;
  if (!r.done) return QAP_OK;
  out->cost = r.cost;
  out->accepts = r.accepts;
  out->iterations = r.iters;
  out->queue_s = std::chrono::duration<double>(r.t_start - r.t_submit).count();
  out->latency_s = std::chrono::duration<double>(r.t_done - r.t_submit).count();
  if (p_out && !r.p.empty()) std::copy(r.p.begin(), r.p.end(), p_out);
  return QAP_OK;
}

int qap_server_max_running(qap_server *s) { return s ? s->max_running.load() : 0; }

int qap_server_stop(qap_server *s) {
  if (!s) return QAP_E_INVAL;
  s->stopping.store(true);
  if (s->worker.joinable()) s->worker.join();  // returns once everything finished
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->setup_cv.notify_all();
  }
  for (auto &t : s->setup_threads)
    if (t.joinable()) t.join();
  delete s;
  return QAP_OK;
}

}  // extern "C"
