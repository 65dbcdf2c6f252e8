// cdd_pool.cu -- serving pool: concurrent observation streams on one GPU with
// admission against an HBM budget, one CUDA stream per observation, and
// per-block latency stamped on the host when the block's kernels complete.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <chrono>
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
  double t_submit = 0;
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
};

}  // namespace

struct cdd_pool_s {
  std::mutex mu;
  int64_t budget = 0;
  int64_t used = 0;
  int device = -1;
  std::vector<Slot> slots;
  std::unordered_map<int64_t, Ticket*> tickets;
  int64_t next_ticket = 1;
};

extern "C" {

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

int cdd_pool_admit(cdd_pool p, double f_center_mhz, double bandwidth_mhz, int n_chan, double dm,
                   int n_fft, int n_avg, int segments_per_block, int taper, int* stream_id) {
  if (!p || !stream_id) return CDD_EINVAL;
  *stream_id = -1;
  cdd_plan plan = nullptr;
  int rc = cdd_plan_create(&plan, f_center_mhz, bandwidth_mhz, n_chan, dm, n_fft, n_avg);
  if (rc) return rc;
  if ((rc = cdd_plan_set(plan, CDD_ATTR_SEGMENTS_PER_BLOCK, segments_per_block)) ||
      (rc = cdd_plan_set(plan, CDD_ATTR_TAPER, taper))) {
    cdd_destroy(plan);
    return rc;
  }
  int64_t need = 0;
  cdd_plan_get(plan, CDD_ATTR_BYTES_NEEDED, &need);
  int id = -1;
  {
    std::lock_guard<std::mutex> lock(p->mu);
    if (p->used + need > p->budget) {
      cdd_destroy(plan);
      return CDD_EBUSY;
    }
    for (size_t i = 0; i < p->slots.size(); ++i)
      if (!p->slots[i].used) {
        id = (int)i;
        break;
      }
    if (id < 0) {
      cdd_destroy(plan);
      return CDD_EBUSY;
    }
    p->slots[id].used = true;             // reserve slot and bytes before allocating
    p->slots[id].bytes = need;
    p->used += need;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(p->device);
  cudaStream_t s = nullptr;
  rc = cdd_plan_commit(plan);
  if (rc == CDD_OK && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) rc = CDD_ECUDA;
  if (prev >= 0) cudaSetDevice(prev);
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
  sl.next_seq = 0;
  sl.gaps = 0;
  sl.blocks = 0;
  *stream_id = id;
  return CDD_OK;
}

int cdd_pool_stream_get(cdd_pool p, int id, int attr, int64_t* v) {
  if (!p || !v) return CDD_EINVAL;
  std::lock_guard<std::mutex> lock(p->mu);
  if (id < 0 || id >= (int)p->slots.size() || !p->slots[id].used) return CDD_EINVAL;
  if (attr == CDD_ATTR_SEQ_GAPS) {
    *v = p->slots[id].gaps;
    return CDD_OK;
  }
  return cdd_plan_get(p->slots[id].plan, attr, v);
}

int cdd_pool_submit(cdd_pool p, int id, int64_t seq, const int8_t* d_in, float* d_out,
                    int64_t* ticket) {
  if (!p || !d_in || !d_out || !ticket) return CDD_EINVAL;
  std::lock_guard<std::mutex> lock(p->mu);
  if (id < 0 || id >= (int)p->slots.size() || !p->slots[id].used) return CDD_EINVAL;
  Slot& sl = p->slots[id];
  if (seq < sl.next_seq) return CDD_EINVAL;        // repeated or late block
  Ticket* t = new (std::nothrow) Ticket();
  if (!t) return CDD_ENOMEM;
  t->t_submit = now_ms();
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(p->device);
  int rc = cdd_execute(sl.plan, d_in, d_out, sl.stream);
  if (rc == CDD_OK && (cudaEventCreateWithFlags(&t->ev, cudaEventDisableTiming) != cudaSuccess ||
                       cudaEventRecord(t->ev, sl.stream) != cudaSuccess ||
                       cudaLaunchHostFunc(sl.stream, stamp_done, t) != cudaSuccess))
    rc = CDD_ECUDA;
  if (prev >= 0) cudaSetDevice(prev);
  if (rc != CDD_OK) {
    if (t->ev) cudaEventDestroy(t->ev);
    delete t;
    return rc;
  }
  sl.gaps += seq - sl.next_seq;
  sl.next_seq = seq + 1;
  sl.blocks += 1;
  *ticket = p->next_ticket++;
  p->tickets[*ticket] = t;
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
  if (latency_ms) *latency_ms = rc == CDD_OK ? t->t_done.load() - t->t_submit : -1.0;
  cudaEventDestroy(t->ev);
  if (t->done.load()) delete t;                    // else leak rather than free under the callback
  return rc;
}

int cdd_pool_stream_state_bytes(cdd_pool p, int id, int64_t* bytes) {
  if (!p || !bytes) return CDD_EINVAL;
  std::lock_guard<std::mutex> lock(p->mu);
  if (id < 0 || id >= (int)p->slots.size() || !p->slots[id].used) return CDD_EINVAL;
  return cdd_plan_state_bytes(p->slots[id].plan, bytes);
}

int cdd_pool_stream_export(cdd_pool p, int id, void* state, int64_t bytes, int64_t* next_seq) {
  if (!p || !state || !next_seq) return CDD_EINVAL;
  std::lock_guard<std::mutex> lock(p->mu);
  if (id < 0 || id >= (int)p->slots.size() || !p->slots[id].used) return CDD_EINVAL;
  Slot& sl = p->slots[id];
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(p->device);
  const int rc = cdd_plan_export_state(sl.plan, state, bytes, sl.stream);
  if (prev >= 0) cudaSetDevice(prev);
  if (rc == CDD_OK) *next_seq = sl.next_seq;
  return rc;
}

int cdd_pool_stream_import(cdd_pool p, int id, const void* state, int64_t bytes, int64_t next_seq) {
  if (!p || !state || next_seq < 0) return CDD_EINVAL;
  std::lock_guard<std::mutex> lock(p->mu);
  if (id < 0 || id >= (int)p->slots.size() || !p->slots[id].used) return CDD_EINVAL;
  Slot& sl = p->slots[id];
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(p->device);
  const int rc = cdd_plan_import_state(sl.plan, state, bytes, sl.stream);
  if (prev >= 0) cudaSetDevice(prev);
  if (rc == CDD_OK) sl.next_seq = next_seq;
  return rc;
}

int cdd_pool_release(cdd_pool p, int id) {
  if (!p) return CDD_EINVAL;
  Slot sl;
  {
    std::lock_guard<std::mutex> lock(p->mu);
    if (id < 0 || id >= (int)p->slots.size() || !p->slots[id].used) return CDD_EINVAL;
    sl = p->slots[id];
    p->slots[id] = Slot();
    p->slots[id].used = true;                      // keep the slot until freed below
  }
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(p->device);
  const int rc = cudaStreamSynchronize(sl.stream) == cudaSuccess ? CDD_OK : CDD_ECUDA;
  cudaStreamDestroy(sl.stream);
  cdd_destroy(sl.plan);
  if (prev >= 0) cudaSetDevice(prev);
  std::lock_guard<std::mutex> lock(p->mu);
  p->used -= sl.bytes;
  p->slots[id] = Slot();
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
    default: return CDD_EINVAL;
  }
}

int cdd_pool_destroy(cdd_pool p) {
  if (!p) return CDD_OK;
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
