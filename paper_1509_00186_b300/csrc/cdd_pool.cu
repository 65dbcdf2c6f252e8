// cdd_pool.cu -- serving pool: concurrent observation streams on one GPU with
// admission against an HBM budget (immediate, or through a first-come queue
// that is served whenever a release frees memory or a slot), one CUDA stream
// per observation, blocks submitted from device or host buffers, and
// per-block latency from the block's arrival to the completion of its work,
// stamped on the host by a stream callback.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <chrono>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/cdd.h"

namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Ticket {
  double t_arrival = 0;
  std::atomic<double> t_done{0};
  std::atomic<int> done{0};
  cudaEvent_t ev = nullptr;
};

// Runs on a CUDA runtime thread once the stream reaches it; no CUDA calls here.
void CUDART_CB stamp_done(void* arg) {
  Ticket* t = static_cast<Ticket*>(arg);
  t->t_done.store(now_ms());
  t->done.store(1);
}

struct Slot {
  bool used = false;
  cdd_plan plan = nullptr;
  cudaStream_t stream = nullptr;
  int64_t bytes = 0;
  int64_t next_seq = 0;
  int64_t gaps = 0;
  int64_t blocks = 0;
  bool host = false;          // host-buffer staging reserved
};

// A queued admission: the stream's (uncommitted) plan and its device bytes.
struct Request {
  int64_t id = 0;
  cdd_plan plan = nullptr;
  int64_t need = 0;
  bool host = false;
};
enum { kQueued = 0, kAdmitted = 1, kFailed = 2 };
struct RequestState {
  int state = kQueued;
  int stream_id = -1;
  int rc = CDD_OK;
};

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev_);
    cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev_ >= 0) cudaSetDevice(prev_);
  }

 private:
  int prev_ = -1;
};

}  // namespace

struct cdd_pool_s {
  std::mutex mu;
  std::mutex pump_mu;         // one admission pass at a time (keeps the queue's order)
  int64_t budget = 0;
  int64_t used = 0;
  int device = -1;
  std::vector<Slot> slots;
  std::unordered_map<int64_t, Ticket*> tickets;
  int64_t next_ticket = 1;
  std::deque<Request> queue;
  std::unordered_map<int64_t, RequestState> requests;
  int64_t next_request = 1;
};

namespace {

// Create a stream's plan (no device work) and its admission size.
int make_plan(double f_center_mhz, double bandwidth_mhz, int n_chan, double dm, int n_fft, int n_avg,
              int segments_per_block, int taper, int flags, cdd_plan* out, int64_t* need) {
  if (flags & ~CDD_POOL_HOST_INGEST) return CDD_EINVAL;
  cdd_plan plan = nullptr;
  int rc = cdd_plan_create(&plan, f_center_mhz, bandwidth_mhz, n_chan, dm, n_fft, n_avg);
  if (rc) return rc;
  if ((rc = cdd_plan_set(plan, CDD_ATTR_SEGMENTS_PER_BLOCK, segments_per_block)) ||
      (rc = cdd_plan_set(plan, CDD_ATTR_TAPER, taper))) {
    cdd_destroy(plan);
    return rc;
  }
  int64_t b = 0, h = 0;
  cdd_plan_get(plan, CDD_ATTR_BYTES_NEEDED, &b);
  if (flags & CDD_POOL_HOST_INGEST) cdd_plan_get(plan, CDD_ATTR_HOST_STAGING_BYTES, &h);
  *out = plan;
  *need = b + h;
  return CDD_OK;
}

// Reserve a free slot and `need` bytes (under the lock); -1 if either is short.
int reserve(cdd_pool p, int64_t need) {
  if (p->used + need > p->budget) return -1;
  for (size_t i = 0; i < p->slots.size(); ++i)
    if (!p->slots[i].used) {
      p->slots[i].used = true;
      p->slots[i].bytes = need;
      p->used += need;
      return (int)i;
    }
  return -1;
}

// Allocate a reserved stream's device state (outside the lock) and fill its slot.
int activate(cdd_pool p, int id, cdd_plan plan, bool host) {
  cudaStream_t s = nullptr;
  int rc;
  {
    DeviceGuard g(p->device);
    rc = cdd_plan_commit(plan);
    if (rc == CDD_OK && host) rc = cdd_plan_prepare_host(plan);
    if (rc == CDD_OK && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) rc = CDD_ECUDA;
  }
  std::lock_guard<std::mutex> lock(p->mu);
  Slot& sl = p->slots[id];
  if (rc != CDD_OK) {
    if (s) cudaStreamDestroy(s);
    cdd_destroy(plan);
    p->used -= sl.bytes;
    sl = Slot();
    return rc;
  }
  sl.plan = plan;
  sl.stream = s;
  sl.host = host;
  sl.next_seq = sl.gaps = sl.blocks = 0;
  return CDD_OK;
}

// Admit queued requests in arrival order while the head fits.
void pump(cdd_pool p) {
  std::lock_guard<std::mutex> order(p->pump_mu);
  for (;;) {
    Request r;
    int id;
    {
      std::lock_guard<std::mutex> lock(p->mu);
      if (p->queue.empty()) return;
      id = reserve(p, p->queue.front().need);
      if (id < 0) return;                    // the head waits; so does everyone behind it
      r = p->queue.front();
      p->queue.pop_front();
    }
    const int rc = activate(p, id, r.plan, r.host);
    std::lock_guard<std::mutex> lock(p->mu);
    RequestState& st = p->requests[r.id];
    st.state = rc == CDD_OK ? kAdmitted : kFailed;
    st.stream_id = rc == CDD_OK ? id : -1;
    st.rc = rc;
  }
}

bool valid_slot(cdd_pool p, int id) { return id >= 0 && id < (int)p->slots.size() && p->slots[id].used && p->slots[id].plan; }

// Enqueue one block of an admitted stream (device or host buffers); the lock is held.
int submit_locked(cdd_pool p, int id, int64_t seq, const int8_t* in, float* out, double t_arrival,
                  bool host, int64_t* ticket) {
  if (!valid_slot(p, id)) return CDD_EINVAL;
  Slot& sl = p->slots[id];
  if (host && !sl.host) return CDD_ESTATE;          // admitted without host staging
  // A block out of order is refused: an older or repeated number, or a gap
  // (a later number while an earlier one is missing; cdd_pool_stream_resync
  // moves past a loss).
  if (seq != sl.next_seq) return CDD_EINVAL;
  Ticket* t = new (std::nothrow) Ticket();
  if (!t) return CDD_ENOMEM;
  t->t_arrival = t_arrival;
  int rc;
  {
    DeviceGuard g(p->device);
    rc = host ? cdd_execute_host_async(sl.plan, in, out, sl.stream) : cdd_execute(sl.plan, in, out, sl.stream);
    if (rc == CDD_OK && (cudaEventCreateWithFlags(&t->ev, cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventRecord(t->ev, sl.stream) != cudaSuccess ||
                         cudaLaunchHostFunc(sl.stream, stamp_done, t) != cudaSuccess))
      rc = CDD_ECUDA;
  }
  if (rc != CDD_OK) {
    if (t->ev) cudaEventDestroy(t->ev);
    delete t;
    return rc;
  }
  sl.next_seq = seq + 1;
  sl.blocks += 1;
  *ticket = p->next_ticket++;
  p->tickets[*ticket] = t;
  return CDD_OK;
}

}  // namespace

extern "C" {

double cdd_pool_clock_ms(void) { return now_ms(); }

int cdd_pool_create(cdd_pool* out, int64_t hbm_budget_bytes, int max_streams) {
  if (!out || hbm_budget_bytes <= 0 || max_streams <= 0 || max_streams > 4096) return CDD_EINVAL;
  *out = nullptr;
  cdd_pool p = new (std::nothrow) cdd_pool_s();
  if (!p) return CDD_ENOMEM;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return CDD_ECUDA;
  }
  p->budget = hbm_budget_bytes;
  p->slots.resize(max_streams);
  *out = p;
  return CDD_OK;
}

int cdd_pool_admit_ex(cdd_pool p, double f_center_mhz, double bandwidth_mhz, int n_chan, double dm,
                      int n_fft, int n_avg, int segments_per_block, int taper, int flags, int* stream_id) {
  if (!p || !stream_id) return CDD_EINVAL;
  *stream_id = -1;
  cdd_plan plan = nullptr;
  int64_t need = 0;
  int rc = make_plan(f_center_mhz, bandwidth_mhz, n_chan, dm, n_fft, n_avg, segments_per_block, taper,
                     flags, &plan, &need);
  if (rc) return rc;
  int id;
  {
    std::lock_guard<std::mutex> lock(p->mu);
    // queued requests keep their turn: an immediate admission never overtakes them
    id = p->queue.empty() ? reserve(p, need) : -1;
  }
  if (id < 0) {
    cdd_destroy(plan);
    return CDD_EBUSY;
  }
  if ((rc = activate(p, id, plan, (flags & CDD_POOL_HOST_INGEST) != 0))) return rc;
  *stream_id = id;
  return CDD_OK;
}

int cdd_pool_admit(cdd_pool p, double f_center_mhz, double bandwidth_mhz, int n_chan, double dm,
                   int n_fft, int n_avg, int segments_per_block, int taper, int* stream_id) {
  return cdd_pool_admit_ex(p, f_center_mhz, bandwidth_mhz, n_chan, dm, n_fft, n_avg, segments_per_block,
                           taper, 0, stream_id);
}

int cdd_pool_request(cdd_pool p, double f_center_mhz, double bandwidth_mhz, int n_chan, double dm,
                     int n_fft, int n_avg, int segments_per_block, int taper, int flags, int64_t* request) {
  if (!p || !request) return CDD_EINVAL;
  cdd_plan plan = nullptr;
  int64_t need = 0;
  int rc = make_plan(f_center_mhz, bandwidth_mhz, n_chan, dm, n_fft, n_avg, segments_per_block, taper,
                     flags, &plan, &need);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lock(p->mu);
    if (need > p->budget) {                         // could never be admitted
      cdd_destroy(plan);
      return CDD_EBUSY;
    }
    Request r;
    r.id = p->next_request++;
    r.plan = plan;
    r.need = need;
    r.host = (flags & CDD_POOL_HOST_INGEST) != 0;
    p->queue.push_back(r);
    p->requests[r.id] = RequestState();
    *request = r.id;
  }
  pump(p);
  return CDD_OK;
}

int cdd_pool_request_status(cdd_pool p, int64_t request, int* stream_id) {
  if (!p || !stream_id) return CDD_EINVAL;
  *stream_id = -1;
  pump(p);
  std::lock_guard<std::mutex> lock(p->mu);
  auto it = p->requests.find(request);
  if (it == p->requests.end()) return CDD_EINVAL;
  const RequestState st = it->second;
  if (st.state == kQueued) return CDD_EBUSY;
  p->requests.erase(it);                            // reported once
  if (st.state == kFailed) return st.rc;
  *stream_id = st.stream_id;
  return CDD_OK;
}

int cdd_pool_stream_get(cdd_pool p, int id, int attr, int64_t* v) {
  if (!p || !v) return CDD_EINVAL;
  std::lock_guard<std::mutex> lock(p->mu);
  if (!valid_slot(p, id)) return CDD_EINVAL;
  if (attr == CDD_ATTR_SEQ_GAPS) {
    *v = p->slots[id].gaps;
    return CDD_OK;
  }
  return cdd_plan_get(p->slots[id].plan, attr, v);
}

int cdd_pool_submit_at(cdd_pool p, int id, int64_t seq, const int8_t* d_in, float* d_out,
                       double t_arrival_ms, int64_t* ticket) {
  if (!p || !d_in || !d_out || !ticket) return CDD_EINVAL;
  std::lock_guard<std::mutex> lock(p->mu);
  return submit_locked(p, id, seq, d_in, d_out, t_arrival_ms, false, ticket);
}

int cdd_pool_submit(cdd_pool p, int id, int64_t seq, const int8_t* d_in, float* d_out, int64_t* ticket) {
  return cdd_pool_submit_at(p, id, seq, d_in, d_out, now_ms(), ticket);
}

int cdd_pool_submit_host(cdd_pool p, int id, int64_t seq, const int8_t* h_in, float* h_out,
                         double t_arrival_ms, int64_t* ticket) {
  if (!p || !h_in || !h_out || !ticket) return CDD_EINVAL;
  std::lock_guard<std::mutex> lock(p->mu);
  return submit_locked(p, id, seq, h_in, h_out, t_arrival_ms, true, ticket);
}

int cdd_pool_submit_many(cdd_pool p, int n, const int* ids, const int64_t* seqs, const int8_t* const* ins,
                         float* const* outs, const double* t_arrival_ms, int host, int64_t* tickets,
                         int* submitted) {
  if (!p || n < 0 || !ids || !seqs || !ins || !outs || !tickets || !submitted) return CDD_EINVAL;
  *submitted = 0;
  std::lock_guard<std::mutex> lock(p->mu);
  for (int i = 0; i < n; ++i) {
    if (!ins[i] || !outs[i]) return CDD_EINVAL;
    const double ta = t_arrival_ms ? t_arrival_ms[i] : now_ms();
    const int rc = submit_locked(p, ids[i], seqs[i], ins[i], outs[i], ta, host != 0, &tickets[i]);
    if (rc) return rc;
    *submitted = i + 1;
  }
  return CDD_OK;
}

int cdd_pool_wait(cdd_pool p, int64_t ticket, double* latency_ms) {
  if (!p) return CDD_EINVAL;
  Ticket* t = nullptr;
  {
    std::lock_guard<std::mutex> lock(p->mu);
    auto it = p->tickets.find(ticket);
    if (it == p->tickets.end()) return CDD_EINVAL;
    t = it->second;
    p->tickets.erase(it);
  }
  int rc = cudaEventSynchronize(t->ev) == cudaSuccess ? CDD_OK : CDD_ECUDA;
  // the completion callback follows the event on the stream; give it a bounded wait
  for (int i = 0; rc == CDD_OK && !t->done.load() && i < 200000; ++i)
    std::this_thread::sleep_for(std::chrono::microseconds(5));
  if (rc == CDD_OK && !t->done.load()) rc = CDD_ECUDA;
  if (latency_ms) *latency_ms = rc == CDD_OK ? t->t_done.load() - t->t_arrival : -1.0;
  cudaEventDestroy(t->ev);
  if (t->done.load()) delete t;                    // else leak rather than free under the callback
  return rc;
}

int cdd_pool_stream_resync(cdd_pool p, int id, int64_t seq) {
  if (!p) return CDD_EINVAL;
  std::lock_guard<std::mutex> lock(p->mu);
  if (!valid_slot(p, id)) return CDD_EINVAL;
  Slot& sl = p->slots[id];
  if (seq < sl.next_seq) return CDD_EINVAL;
  int rc;
  {
    DeviceGuard g(p->device);
    rc = cudaStreamSynchronize(sl.stream) == cudaSuccess ? cdd_reset(sl.plan) : CDD_ECUDA;
  }
  if (rc) return rc;
  sl.gaps += seq - sl.next_seq;
  sl.next_seq = seq;
  return CDD_OK;
}

int cdd_pool_stream_state_bytes(cdd_pool p, int id, int64_t* bytes) {
  if (!p || !bytes) return CDD_EINVAL;
  std::lock_guard<std::mutex> lock(p->mu);
  if (!valid_slot(p, id)) return CDD_EINVAL;
  return cdd_plan_state_bytes(p->slots[id].plan, bytes);
}

int cdd_pool_stream_export(cdd_pool p, int id, void* state, int64_t bytes, int64_t* next_seq) {
  if (!p || !state || !next_seq) return CDD_EINVAL;
  std::lock_guard<std::mutex> lock(p->mu);
  if (!valid_slot(p, id)) return CDD_EINVAL;
  Slot& sl = p->slots[id];
  int rc;
  {
    DeviceGuard g(p->device);
    rc = cdd_plan_export_state(sl.plan, state, bytes, sl.stream);
  }
  if (rc == CDD_OK) *next_seq = sl.next_seq;
  return rc;
}

int cdd_pool_stream_import(cdd_pool p, int id, const void* state, int64_t bytes, int64_t next_seq) {
  if (!p || !state || next_seq < 0) return CDD_EINVAL;
  std::lock_guard<std::mutex> lock(p->mu);
  if (!valid_slot(p, id)) return CDD_EINVAL;
  Slot& sl = p->slots[id];
  int rc;
  {
    DeviceGuard g(p->device);
    rc = cdd_plan_import_state(sl.plan, state, bytes, sl.stream);
  }
  if (rc == CDD_OK) sl.next_seq = next_seq;
  return rc;
}

int cdd_pool_release(cdd_pool p, int id) {
  if (!p) return CDD_EINVAL;
  Slot sl;
  {
    std::lock_guard<std::mutex> lock(p->mu);
    if (!valid_slot(p, id)) return CDD_EINVAL;
    sl = p->slots[id];
    p->slots[id] = Slot();
    p->slots[id].used = true;                      // keep the slot until freed below
  }
  int rc;
  {
    DeviceGuard g(p->device);
    rc = cudaStreamSynchronize(sl.stream) == cudaSuccess ? CDD_OK : CDD_ECUDA;
    cudaStreamDestroy(sl.stream);
    cdd_destroy(sl.plan);
  }
  {
    std::lock_guard<std::mutex> lock(p->mu);
    p->used -= sl.bytes;
    p->slots[id] = Slot();
  }
  pump(p);                                         // memory and a slot freed: serve the queue
  return rc;
}

int cdd_pool_get(cdd_pool p, int attr, int64_t* v) {
  if (!p || !v) return CDD_EINVAL;
  std::lock_guard<std::mutex> lock(p->mu);
  switch (attr) {
    case CDD_POOL_BUDGET: *v = p->budget; return CDD_OK;
    case CDD_POOL_USED_BYTES: *v = p->used; return CDD_OK;
    case CDD_POOL_STREAMS: {
      int64_t n = 0;
      for (auto& s : p->slots) n += s.used ? 1 : 0;
      *v = n;
      return CDD_OK;
    }
    case CDD_POOL_QUEUED: *v = (int64_t)p->queue.size(); return CDD_OK;
    default: return CDD_EINVAL;
  }
}

int cdd_pool_destroy(cdd_pool p) {
  if (!p) return CDD_OK;
  {
    std::lock_guard<std::mutex> lock(p->mu);
    for (Request& r : p->queue) cdd_destroy(r.plan);
    p->queue.clear();
  }
  for (int i = 0; i < (int)p->slots.size(); ++i)
    if (p->slots[i].used && p->slots[i].plan) cdd_pool_release(p, i);
  std::vector<int64_t> left;
  {
    std::lock_guard<std::mutex> lock(p->mu);
    for (auto& kv : p->tickets) left.push_back(kv.first);
  }
  for (int64_t t : left) cdd_pool_wait(p, t, nullptr);
  delete p;
  return CDD_OK;
}

}  // extern "C"
