// cdd_api.cu -- the C ABI declared in include/cdd.h: plan geometry, device
// state, and the device-buffer and host-buffer execute calls.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/cdd.h"
#include "cdd_internal.h"

namespace {

constexpr double kDispD = 4.148808e3;   // s MHz^2 cm^3 / pc (Sec. 2.1, Eq. 3)
constexpr int kMinLogN = 6;
constexpr int kMaxLogN = 16;

}  // namespace

constexpr int kTimingSlots = 256;   // stage-timing event triples per plan

struct cdd_plan_s {
  // observation and geometry (fixed at create)
  double f_center = 0, bandwidth = 0, dm = 0, chan_bw = 0, f_lo0 = 0, n_disp = 0;
  double f_base = 0;
  int sideband = 1;
  int n_chan = 0, n_fft = 0, logn = 0, n_ov = 0, hop = 0, n_avg = 0;
  std::vector<int64_t> shift;
  int64_t r_max = 0;
  // settable before the first execute
  int q = 1;
  int taper = CDD_TAPER_NONE;
  int precision = CDD_PRECISION_FP32;
  int chunks = 1;
  bool chunks_set = false;
  // device state
  bool committed = false;
  int device = -1;
  int sticky = CDD_OK;
  float2* d_chirp = nullptr;
  float2* d_tw = nullptr;
  char2* d_tail[2] = {nullptr, nullptr};
  float* d_ring = nullptr;
  int* d_shift = nullptr;
  int* d_err = nullptr;      // the kernels' wait-timeout flags (1 tensor-core products, 2 tile copies)
  bool turn_tma = false;     // corner turn by tensor tile copies (CDD_ATTR_TURN_TMA)
  void* d_dft = nullptr;     // tensor-core forms: the DFT matrices
  char2* d_in_cm = nullptr;  // channel-major copy of the block (corner-turn path)
  long long ring_len = 0;
  size_t bytes_device = 0;
  // second polarisation: its own overlap tails, ring and stream position,
  // sharing the tables (CDD_ATTR_POLARISATIONS = 2)
  int pols = 1;
  char2* d_tail_b[2] = {nullptr, nullptr};
  float* d_ring_b = nullptr;
  float* d_pol_tmp = nullptr;
  long long g_next_b = 0;
  int parity_b = 0;
  // stream position
  long long g_next = 0;     // stream index of the next integrated output
  int parity = 0;           // which tail buffer holds the previous block's tail
  int64_t blocks = 0;
  int last_launches = 0;
  // host-buffer path
  int8_t* d_in_stage[2] = {nullptr, nullptr};
  float* d_out_stage[2] = {nullptr, nullptr};
  cudaStream_t st_h2d = nullptr, st_comp = nullptr, st_d2h = nullptr;
  cudaEvent_t ev_start = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr},
              ev_out[2] = {nullptr, nullptr};
  bool host_ready = false;
  // stage timing (CDD_ATTR_STAGE_TIMING): kTimingSlots triples of events
  // {before corner turn, between, after fused kernel}, reused round robin
  bool timing = false;
  std::vector<cudaEvent_t> t_ev;
  std::vector<char> t_pending;
  int64_t t_next = 0, t_blocks = 0, t_ct_ns = 0, t_ols_ns = 0;
};

namespace cdd {

int64_t shift_of(const Geometry& g, int k) {
  const double ref = pow(g.f_ref, -2.0);
  const double f_k = chan_lower_edge(g, k);
  const double delay = kDispD * g.dm * (pow(f_k, -2.0) - ref);   // <= 0: f_k arrives first
  const double r = rint(-delay * g.chan_bw * 1e6 / g.n_avg);
  return (r >= 0 && r < 2e9) ? (int64_t)r : -1;
}

static int next_pow2_above(double x) {
  long long n = 1;
  while ((double)n <= x && n < (1LL << 40)) n *= 2;
  return n > (1LL << 30) ? -1 : (int)n;
}

int geometry(Geometry* g, double f_center, double bandwidth, int n_chan, double dm, int n_fft,
             int n_avg) {
  if (!(f_center > 0) || !(bandwidth != 0) || !isfinite(bandwidth) || n_chan <= 0 ||
      !(dm >= 0) || n_avg <= 0 || n_fft < 0 || !isfinite(dm))
    return CDD_EINVAL;
  g->f_center = f_center;
  g->bandwidth = bandwidth;
  g->dm = dm;
  g->n_chan = n_chan;
  g->n_avg = n_avg;
  g->sideband = bandwidth > 0 ? 1 : -1;
  g->chan_bw = fabs(bandwidth) / n_chan;
  g->f_lo0 = f_center - fabs(bandwidth) / 2.0;
  g->f_base = g->sideband > 0 ? g->f_lo0 : f_center + fabs(bandwidth) / 2.0;
  g->f_ref = chan_lower_edge(*g, g->sideband > 0 ? 0 : n_chan - 1);
  if (!(g->f_ref > 0)) return CDD_EINVAL;
  // dispersion time across the lowest (most smeared) channel, in samples
  const double t_d = kDispD * dm * (pow(g->f_ref, -2.0) - pow(g->f_ref + g->chan_bw, -2.0));
  g->n_disp = t_d * g->chan_bw * 1e6;
  if (!(g->n_disp < 1e9)) return CDD_EINVAL;
  long long n_ov = (long long)ceil(g->n_disp);
  n_ov = (n_ov + n_avg - 1) / n_avg * n_avg;
  if (n_fft == 0) {
    int a = next_pow2_above(2.0 * g->n_disp), b = next_pow2_above((double)n_ov);
    if (a < 0 || b < 0) return CDD_EINVAL;
    n_fft = a > b ? a : b;
    if (n_fft < 64) n_fft = 64;
    while ((long long)n_fft < 2LL * n_avg) n_fft *= 2;
  }
  if (n_fft <= 0 || (n_fft & (n_fft - 1)) || (long long)n_fft <= n_ov) return CDD_EINVAL;
  const int hop = n_fft - (int)n_ov;
  if (hop % n_avg) return CDD_EINVAL;
  int logn = 0;
  while ((1 << logn) < n_fft) ++logn;
  g->n_fft = n_fft;
  g->logn = logn;
  g->n_ov = (int)n_ov;
  g->hop = hop;
  g->r_max = 0;
  for (int k = 0; k < n_chan; ++k) {
    const int64_t r = shift_of(*g, k);
    if (r < 0) return CDD_EINVAL;
    if (r > g->r_max) g->r_max = r;
  }
  if (logn < kMinLogN || logn > kMaxLogN) return CDD_EUNSUPPORTED;
  // N > 16384 runs as a cluster of N/2^kClusterLogS CTAs, each holding every
  // (N/2^kClusterLogS)-th sample run of 2^kClusterLogS/CL; an integration
  // window must not span two of them
  if (logn > 14 && n_avg > (1 << kClusterLogS) / (n_fft >> kClusterLogS)) return CDD_EUNSUPPORTED;
  return CDD_OK;
}

}  // namespace cdd

namespace {

int fail_cuda(cdd_plan p, cudaError_t e) {
  if (e == cudaSuccess) return CDD_OK;
  if (p) p->sticky = CDD_ECUDA;
  return CDD_ECUDA;
}

#define CDD_TRY(p, call)                           \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return fail_cuda(p, e_); \
  } while (0)

int64_t n_out_per_block(const cdd_plan p) { return (int64_t)p->q * p->hop / p->n_avg; }

// Host-buffer pipeline: the most chunks (a divisor of q) of at least 4
// segments each, so the copy-out and compute of the last chunk, which
// nothing overlaps, stay short (19 chunks of 4 for q = 76).
int default_chunks(int q) {
  for (int d = q / 4; d > 1; --d)
    if (q % d == 0) return d;
  return 1;
}

// Device bytes the first execute allocates (tables, tails, ring, shifts and the
// channel-major block copy), exactly as commit_once requests them.
int64_t bytes_needed(const cdd_plan p) {
  const int64_t C = p->n_chan;
  int64_t b = C * p->n_fft * (int64_t)sizeof(float2);
  b += (int64_t)cdd::twiddle_table_len(p->logn) * (int64_t)sizeof(float2);
  if (p->n_ov > 0) b += 2 * C * p->n_ov * (int64_t)sizeof(char2);
  b += C * (p->r_max + n_out_per_block(p)) * (int64_t)sizeof(float);
  b += C * (int64_t)sizeof(int);
  b += C * p->q * p->hop * (int64_t)sizeof(char2);
  b += (int64_t)sizeof(int);
  if (p->precision != CDD_PRECISION_FP32) b += (int64_t)cdd::tc_dft_bytes();
  if (p->pols == 2) {
    if (p->n_ov > 0) b += 2 * C * p->n_ov * (int64_t)sizeof(char2);
    b += C * (p->r_max + n_out_per_block(p)) * (int64_t)sizeof(float);
    b += C * n_out_per_block(p) * (int64_t)sizeof(float);
  }
  return b;
}

// Geometry of Sec. 2.2 / 2.3 and the channel alignment of Sec. 1.2, held by
// the plan (with its per-channel shifts).
int compute_geometry(cdd_plan p, int n_fft) {
  cdd::Geometry g;
  const int rc = cdd::geometry(&g, p->f_center, p->bandwidth, p->n_chan, p->dm, n_fft, p->n_avg);
  if (rc != CDD_OK) return rc;
  p->chan_bw = g.chan_bw;
  p->f_lo0 = g.f_lo0;
  p->f_base = g.f_base;
  p->sideband = g.sideband;
  p->n_disp = g.n_disp;
  p->n_fft = g.n_fft;
  p->logn = g.logn;
  p->n_ov = g.n_ov;
  p->hop = g.hop;
  p->r_max = g.r_max;
  p->shift.assign(p->n_chan, 0);
  for (int k = 0; k < p->n_chan; ++k) p->shift[k] = cdd::shift_of(g, k);
  return CDD_OK;
}

void free_device(cdd_plan p) {
  cudaFree(p->d_chirp);
  cudaFree(p->d_tw);
  cudaFree(p->d_tail[0]);
  cudaFree(p->d_tail[1]);
  cudaFree(p->d_ring);
  cudaFree(p->d_shift);
  cudaFree(p->d_err);
  cudaFree(p->d_dft);
  cudaFree(p->d_in_cm);
  cudaFree(p->d_tail_b[0]);
  cudaFree(p->d_tail_b[1]);
  cudaFree(p->d_ring_b);
  cudaFree(p->d_pol_tmp);
  for (int i = 0; i < 2; ++i) {
    cudaFree(p->d_in_stage[i]);
    cudaFree(p->d_out_stage[i]);
    if (p->ev_in[i]) cudaEventDestroy(p->ev_in[i]);
    if (p->ev_comp[i]) cudaEventDestroy(p->ev_comp[i]);
    if (p->ev_out[i]) cudaEventDestroy(p->ev_out[i]);
  }
  if (p->ev_start) cudaEventDestroy(p->ev_start);
  for (cudaEvent_t e : p->t_ev)
    if (e) cudaEventDestroy(e);
  if (p->st_h2d) cudaStreamDestroy(p->st_h2d);
  if (p->st_comp) cudaStreamDestroy(p->st_comp);
  if (p->st_d2h) cudaStreamDestroy(p->st_d2h);
}

template <class T>
int dalloc(cdd_plan p, T** ptr, size_t bytes) {
  cudaError_t e = cudaMalloc((void**)ptr, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    *ptr = nullptr;
    return CDD_ENOMEM;
  }
  if (e != cudaSuccess) return fail_cuda(p, e);
  p->bytes_device += bytes;
  return CDD_OK;
}

int zero_state(cdd_plan p, cudaStream_t s) {
  const size_t tb = (size_t)p->n_chan * p->n_ov * sizeof(char2);
  const size_t rb = (size_t)p->n_chan * p->ring_len * sizeof(float);
  if (p->n_ov > 0) {
    CDD_TRY(p, cudaMemsetAsync(p->d_tail[0], 0, tb, s));
    CDD_TRY(p, cudaMemsetAsync(p->d_tail[1], 0, tb, s));
  }
  CDD_TRY(p, cudaMemsetAsync(p->d_ring, 0, rb, s));
  if (p->pols == 2) {
    if (p->n_ov > 0) {
      CDD_TRY(p, cudaMemsetAsync(p->d_tail_b[0], 0, tb, s));
      CDD_TRY(p, cudaMemsetAsync(p->d_tail_b[1], 0, tb, s));
    }
    CDD_TRY(p, cudaMemsetAsync(p->d_ring_b, 0, rb, s));
  }
  p->g_next = p->g_next_b = 0;
  p->parity = p->parity_b = 0;
  p->blocks = 0;
  return CDD_OK;
}

// First execute: bind the device, allocate the plan's state and build its
// tables.  Synchronous.
int commit_once(cdd_plan p) {
  CDD_TRY(p, cudaGetDevice(&p->device));
  const int N = p->n_fft;
  int rc;
  p->ring_len = p->r_max + n_out_per_block(p);
  if ((rc = dalloc(p, &p->d_chirp, (size_t)p->n_chan * N * sizeof(float2)))) return rc;
  if ((rc = dalloc(p, &p->d_tw, (size_t)cdd::twiddle_table_len(p->logn) * sizeof(float2)))) return rc;
  if (p->n_ov > 0) {
    for (int i = 0; i < 2; ++i)
      if ((rc = dalloc(p, &p->d_tail[i], (size_t)p->n_chan * p->n_ov * sizeof(char2)))) return rc;
  }
  if ((rc = dalloc(p, &p->d_ring, (size_t)p->n_chan * p->ring_len * sizeof(float)))) return rc;
  if ((rc = dalloc(p, &p->d_shift, (size_t)p->n_chan * sizeof(int)))) return rc;
  // channel-major copy of a block: the fused kernel then reads each segment contiguously
  if ((rc = dalloc(p, &p->d_in_cm, (size_t)p->n_chan * p->q * p->hop * sizeof(char2)))) return rc;
  if ((rc = dalloc(p, &p->d_err, sizeof(int)))) return rc;
  CDD_TRY(p, cudaMemset(p->d_err, 0, sizeof(int)));
  const bool tc = p->precision != CDD_PRECISION_FP32;
  if (tc) {
    if ((rc = dalloc(p, &p->d_dft, cdd::tc_dft_bytes()))) return rc;
  }
  if (p->pols == 2) {
    if (p->n_ov > 0)
      for (int i = 0; i < 2; ++i)
        if ((rc = dalloc(p, &p->d_tail_b[i], (size_t)p->n_chan * p->n_ov * sizeof(char2)))) return rc;
    if ((rc = dalloc(p, &p->d_ring_b, (size_t)p->n_chan * p->ring_len * sizeof(float)))) return rc;
    if ((rc = dalloc(p, &p->d_pol_tmp, (size_t)p->n_chan * n_out_per_block(p) * sizeof(float)))) return rc;
  }
  if (p->timing) {
    p->t_ev.assign(3 * kTimingSlots, nullptr);
    p->t_pending.assign(kTimingSlots, 0);
    for (cudaEvent_t& e : p->t_ev) CDD_TRY(p, cudaEventCreate(&e));
  }
  std::vector<int> sh(p->shift.begin(), p->shift.end());
  CDD_TRY(p, cudaMemcpy(p->d_shift, sh.data(), sh.size() * sizeof(int), cudaMemcpyHostToDevice));
  cudaStream_t s;
  CDD_TRY(p, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaError_t e = cdd::launch_twiddle_table(p->logn, p->d_tw, s);
  if (e == cudaSuccess)
    e = cdd::launch_chirp_table(p->logn, p->d_chirp, p->n_chan, p->f_base, p->chan_bw, p->dm,
                                p->taper, p->sideband, s, tc ? cdd::tc_chirp_scale() : 0.0);
  if (e == cudaSuccess && tc) e = cdd::launch_tc_dft_table(p->precision, p->d_dft, s);
  if (e == cudaSuccess && (rc = zero_state(p, s)) != CDD_OK) {
    cudaStreamDestroy(s);
    return rc;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (e != cudaSuccess) return fail_cuda(p, e);
  p->committed = true;
  return CDD_OK;
}

// A failed commit leaves the plan unusable (sticky) rather than half built.
int commit(cdd_plan p) {
  if (p->committed) return CDD_OK;
  const int rc = commit_once(p);
  if (rc != CDD_OK) p->sticky = rc;
  return rc;
}

int check_device(cdd_plan p) {
  int dev = -1;
  CDD_TRY(p, cudaGetDevice(&dev));
  return dev == p->device ? CDD_OK : CDD_EINVAL;
}

// Fold a finished timing slot into the sums (waits for its last event).
int harvest_slot(cdd_plan p, int slot) {
  cudaEvent_t* e = &p->t_ev[3 * slot];
  CDD_TRY(p, cudaEventSynchronize(e[2]));
  float ct = 0.f, ols = 0.f;
  CDD_TRY(p, cudaEventElapsedTime(&ct, e[0], e[1]));
  CDD_TRY(p, cudaEventElapsedTime(&ols, e[1], e[2]));
  p->t_ct_ns += llround((double)ct * 1e6);
  p->t_ols_ns += llround((double)ols * 1e6);
  p->t_blocks += 1;
  p->t_pending[slot] = 0;
  return CDD_OK;
}

int harvest_all(cdd_plan p) {
  for (int i = 0; i < (int)p->t_pending.size(); ++i)
    if (p->t_pending[i]) {
      const int rc = harvest_slot(p, i);
      if (rc) return rc;
    }
  return CDD_OK;
}

// One block of q segments on `s` for polarisation `pol`; advances its stream position.
int run_block(cdd_plan p, const int8_t* d_in, float* d_out, float* d_volt, int q, cudaStream_t s,
              int pol = 0) {
  char2** tail = pol == 0 ? p->d_tail : p->d_tail_b;
  int& parity = pol == 0 ? p->parity : p->parity_b;
  long long& g_next = pol == 0 ? p->g_next : p->g_next_b;
  cdd::OlsArgs a;
  a.in = reinterpret_cast<const char2*>(d_in);
  a.rows = (long long)q * p->hop;
  a.in_cm = p->d_in_cm;
  a.out = d_out;
  a.chirp = p->d_chirp;
  a.tw = p->d_tw;
  a.tail_rd = tail[parity];
  a.tail_wr = tail[parity ^ 1];
  a.ring = pol == 0 ? p->d_ring : p->d_ring_b;
  a.shift = p->d_shift;
  a.volt = reinterpret_cast<float2*>(d_volt);
  a.dft = p->d_dft;
  a.n_chan = p->n_chan;
  a.n_ov = p->n_ov;
  a.hop = p->hop;
  a.n_avg = p->n_avg;
  a.q = q;
  a.n_out = (int)((int64_t)q * p->hop / p->n_avg);
  a.g0 = g_next;
  a.ring_len = p->ring_len;
  cudaEvent_t* te = nullptr;
  if (p->timing) {
    const int slot = (int)(p->t_next++ % kTimingSlots);
    if (p->t_pending[slot]) {
      const int rc = harvest_slot(p, slot);
      if (rc) return rc;
    }
    te = &p->t_ev[3 * slot];
    p->t_pending[slot] = 1;
    CDD_TRY(p, cudaEventRecord(te[0], s));
  }
  CDD_TRY(p, cdd::launch_corner_turn(a.in, p->d_in_cm, 0, a.rows, a.rows, p->n_chan, s,
                                     p->turn_tma ? p->d_err : nullptr));
  if (te) CDD_TRY(p, cudaEventRecord(te[1], s));
  a.s_begin = 0;
  a.s_count = q;
  if (p->precision == CDD_PRECISION_FP32) CDD_TRY(p, cdd::launch_ols(p->logn, a, s));
  else CDD_TRY(p, cdd::launch_ols_tc(p->logn, p->precision, a, p->d_err, s));
  if (te) CDD_TRY(p, cudaEventRecord(te[2], s));
  const int launches = 2;
  p->last_launches = launches;
  g_next += a.n_out;
  parity ^= 1;
  if (pol == 0) p->blocks += 1;
  return CDD_OK;
}

int prepare(cdd_plan p) {
  if (!p) return CDD_EINVAL;
  if (p->sticky) return p->sticky;
  int rc = commit(p);
  if (rc) return rc;
  return check_device(p);
}

// Device bytes of the host-buffer path's staging: two chunks of input and
// two of output (copy-in, compute and copy-out overlap, Sec. 4.2).
int64_t host_staging_bytes(const cdd_plan p) {
  const int64_t q_c = p->q / p->chunks;
  return 2 * (q_c * p->hop * p->n_chan * 2 + (int64_t)p->n_chan * (q_c * p->hop / p->n_avg) * (int64_t)sizeof(float));
}

int setup_host_path(cdd_plan p) {
  if (p->host_ready) return CDD_OK;
  const int64_t q_c = p->q / p->chunks;
  const size_t in_b = (size_t)q_c * p->hop * p->n_chan * 2;
  const size_t out_b = (size_t)p->n_chan * (q_c * p->hop / p->n_avg) * sizeof(float);
  int rc;
  for (int i = 0; i < 2; ++i) {
    if ((rc = dalloc(p, &p->d_in_stage[i], in_b))) return rc;
    if ((rc = dalloc(p, &p->d_out_stage[i], out_b))) return rc;
    CDD_TRY(p, cudaEventCreateWithFlags(&p->ev_in[i], cudaEventDisableTiming));
    CDD_TRY(p, cudaEventCreateWithFlags(&p->ev_comp[i], cudaEventDisableTiming));
    CDD_TRY(p, cudaEventCreateWithFlags(&p->ev_out[i], cudaEventDisableTiming));
  }
  CDD_TRY(p, cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming));
  CDD_TRY(p, cudaStreamCreateWithFlags(&p->st_h2d, cudaStreamNonBlocking));
  CDD_TRY(p, cudaStreamCreateWithFlags(&p->st_comp, cudaStreamNonBlocking));
  CDD_TRY(p, cudaStreamCreateWithFlags(&p->st_d2h, cudaStreamNonBlocking));
  p->host_ready = true;
  return CDD_OK;
}

}  // namespace

extern "C" {

int cdd_version(void) { return 100; }

const char* cdd_strerror(int code) {
  switch (code) {
    case CDD_OK: return "success";
    case CDD_EINVAL: return "invalid argument or geometry";
    case CDD_ENOMEM: return "out of device or host memory";
    case CDD_ECUDA: return "CUDA error (sticky for this plan)";
    case CDD_EUNSUPPORTED: return "not supported by this library";
    case CDD_ESTATE: return "not allowed in the plan's current state";
    case CDD_ETOOBIG: return "request exceeds the fixed scratch of cdd_execute_static";
    case CDD_EBUSY: return "admission refused: HBM budget or stream slots exhausted";
    default: return "unknown error code";
  }
}

int cdd_plan_create(cdd_plan* plan, double f_center_mhz, double bandwidth_mhz, int n_chan,
                    double dm, int n_fft, int n_avg) {
  if (!plan) return CDD_EINVAL;
  *plan = nullptr;
  cdd_plan p = new (std::nothrow) cdd_plan_s();
  if (!p) return CDD_ENOMEM;
  p->f_center = f_center_mhz;
  p->bandwidth = bandwidth_mhz;
  p->n_chan = n_chan;
  p->dm = dm;
  p->n_avg = n_avg;
  const int rc = compute_geometry(p, n_fft);
  if (rc != CDD_OK) {
    delete p;
    return rc;
  }
  *plan = p;
  return CDD_OK;
}

int cdd_plan_set(cdd_plan p, int attr, int64_t value) {
  if (!p) return CDD_EINVAL;
  if (p->committed) return CDD_ESTATE;
  switch (attr) {
    case CDD_ATTR_SEGMENTS_PER_BLOCK:
      if (value < 1 || value > (1 << 24)) return CDD_EINVAL;
      if ((int64_t)value * p->hop * p->n_chan > (int64_t)1 << 40) return CDD_EINVAL;
      if ((int64_t)value * p->n_chan >= (int64_t)1 << 31) return CDD_EINVAL;
      p->q = (int)value;
      if (!p->chunks_set || p->q % p->chunks) p->chunks = default_chunks(p->q);
      return CDD_OK;
    case CDD_ATTR_TAPER:
      if (value < CDD_TAPER_NONE || value > CDD_TAPER_WELCH) return CDD_EINVAL;
      p->taper = (int)value;
      return CDD_OK;
    case CDD_ATTR_PIPELINE_CHUNKS:
      if (value < 1 || value > p->q || p->q % value) return CDD_EINVAL;
      p->chunks = (int)value;
      p->chunks_set = true;
      return CDD_OK;
    case CDD_ATTR_POLARISATIONS:
      if (value != 1 && value != 2) return CDD_EINVAL;
      p->pols = (int)value;
      return CDD_OK;
    case CDD_ATTR_STAGE_TIMING:
      if (value != 0 && value != 1) return CDD_EINVAL;
      p->timing = value == 1;
      return CDD_OK;
    case CDD_ATTR_TURN_TMA:
      if (value != 0 && value != 1) return CDD_EINVAL;
      p->turn_tma = value == 1;
      return CDD_OK;
    case CDD_ATTR_PRECISION:
      if (value < CDD_PRECISION_FP32 || value > CDD_PRECISION_BF16) return CDD_EINVAL;
      if (value != CDD_PRECISION_FP32 && !cdd::tc_supported(p->logn, (int)value)) return CDD_EUNSUPPORTED;
      p->precision = (int)value;
      return CDD_OK;
    default:
      return CDD_EINVAL;
  }
}

int cdd_plan_get(cdd_plan p, int attr, int64_t* v) {
  if (!p || !v) return CDD_EINVAL;
  switch (attr) {
    case CDD_ATTR_N_FFT: *v = p->n_fft; break;
    case CDD_ATTR_N_OV: *v = p->n_ov; break;
    case CDD_ATTR_HOP: *v = p->hop; break;
    case CDD_ATTR_N_AVG: *v = p->n_avg; break;
    case CDD_ATTR_N_CHAN: *v = p->n_chan; break;
    case CDD_ATTR_SEGMENTS_PER_BLOCK: *v = p->q; break;
    case CDD_ATTR_BLOCK_SAMPLES: *v = (int64_t)p->q * p->hop; break;
    case CDD_ATTR_N_OUT_PER_BLOCK: *v = n_out_per_block(p); break;
    case CDD_ATTR_R_MAX: *v = p->r_max; break;
    case CDD_ATTR_BYTES_DEVICE: *v = (int64_t)p->bytes_device; break;
    case CDD_ATTR_TAPER: *v = p->taper; break;
    case CDD_ATTR_BLOCKS_DONE: *v = p->blocks; break;
    case CDD_ATTR_PIPELINE_CHUNKS: *v = p->chunks; break;
    case CDD_ATTR_KERNEL_LAUNCHES: *v = p->last_launches; break;
    case CDD_ATTR_BYTES_NEEDED: *v = bytes_needed(p); break;
    case CDD_ATTR_HOST_STAGING_BYTES: *v = host_staging_bytes(p); break;
    case CDD_ATTR_POLARISATIONS: *v = p->pols; break;
    case CDD_ATTR_STAGE_TIMING: *v = p->timing ? 1 : 0; break;
    case CDD_ATTR_PRECISION: *v = p->precision; break;
    case CDD_ATTR_TURN_TMA: *v = p->turn_tma ? 1 : 0; break;
    case CDD_ATTR_DEVICE_ERRORS: {
      int e = 0;
      if (p->d_err) {
        if (p->sticky) return p->sticky;
        CDD_TRY(p, cudaMemcpy(&e, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
      }
      *v = e;
      break;
    }
    case CDD_ATTR_TIMED_BLOCKS:
    case CDD_ATTR_CORNER_TURN_NS:
    case CDD_ATTR_OLS_NS: {
      if (p->timing && p->committed) {
        if (p->sticky) return p->sticky;
        const int rc = harvest_all(p);
        if (rc) return rc;
      }
      *v = attr == CDD_ATTR_TIMED_BLOCKS ? p->t_blocks
         : attr == CDD_ATTR_CORNER_TURN_NS ? p->t_ct_ns : p->t_ols_ns;
      break;
    }
    default: return CDD_EINVAL;
  }
  return CDD_OK;
}

int cdd_plan_commit(cdd_plan p) { return prepare(p); }

int cdd_plan_shifts(cdd_plan p, int64_t* shifts) {
  if (!p || !shifts) return CDD_EINVAL;
  memcpy(shifts, p->shift.data(), p->shift.size() * sizeof(int64_t));
  return CDD_OK;
}

int cdd_execute_voltages(cdd_plan p, const int8_t* d_in, float* d_out, float* d_volt,
                         cudaStream_t stream) {
  if (!p || !d_in || !d_out) return CDD_EINVAL;
  int rc = prepare(p);
  if (rc) return rc;
  rc = run_block(p, d_in, d_out, d_volt, p->q, stream);
  if (rc) p->last_launches = 0;
  return rc;
}

int cdd_execute(cdd_plan p, const int8_t* d_in, float* d_out, cudaStream_t stream) {
  return cdd_execute_voltages(p, d_in, d_out, nullptr, stream);
}

int cdd_execute_dual(cdd_plan p, const int8_t* d_in_a, const int8_t* d_in_b, float* d_out,
                     cudaStream_t stream) {
  if (!p || !d_in_a || !d_in_b || !d_out) return CDD_EINVAL;
  if (p->pols != 2) return CDD_ESTATE;
  int rc = prepare(p);
  if (rc) return rc;
  if ((rc = run_block(p, d_in_a, d_out, nullptr, p->q, stream, 0))) return rc;
  if ((rc = run_block(p, d_in_b, p->d_pol_tmp, nullptr, p->q, stream, 1))) return rc;
  const int per_pol = p->last_launches;
  CDD_TRY(p, cdd::launch_accumulate(d_out, p->d_pol_tmp, (long long)p->n_chan * n_out_per_block(p), stream));
  p->last_launches = 2 * per_pol + 1;
  return CDD_OK;
}

int cdd_band_sum(const float* d_out, int64_t n_planes, int n_chan, int64_t n_out, float* d_sum,
                 cudaStream_t stream) {
  if (!d_out || !d_sum || n_planes <= 0 || n_chan <= 0 || n_out <= 0) return CDD_EINVAL;
  return cdd::launch_band_sum(d_out, n_planes, n_chan, n_out, d_sum, stream) == cudaSuccess
             ? CDD_OK : CDD_ECUDA;
}

int cdd_execute_host_async(cdd_plan p, const int8_t* h_in, float* h_out, cudaStream_t stream) {
  if (!p || !h_in || !h_out) return CDD_EINVAL;
  int rc = prepare(p);
  if (rc) return rc;
  if ((rc = setup_host_path(p))) return rc;
  const int nc = p->chunks;
  const int q_c = p->q / nc;
  const size_t rows_c = (size_t)q_c * p->hop;
  const size_t in_b = rows_c * p->n_chan * 2;
  const size_t out_c = rows_c / p->n_avg;                 // outputs per channel per chunk
  const size_t out_total = (size_t)n_out_per_block(p);
  // everything below is ordered after the caller's earlier work on `stream`
  CDD_TRY(p, cudaEventRecord(p->ev_start, stream));
  CDD_TRY(p, cudaStreamWaitEvent(p->st_h2d, p->ev_start, 0));
  CDD_TRY(p, cudaStreamWaitEvent(p->st_comp, p->ev_start, 0));
  CDD_TRY(p, cudaStreamWaitEvent(p->st_d2h, p->ev_start, 0));
  for (int c = 0; c < nc; ++c) {
    const int slot = c & 1;
    if (c >= 2) CDD_TRY(p, cudaStreamWaitEvent(p->st_h2d, p->ev_comp[slot], 0));
    CDD_TRY(p, cudaMemcpyAsync(p->d_in_stage[slot], h_in + (size_t)c * in_b, in_b,
                               cudaMemcpyHostToDevice, p->st_h2d));
    CDD_TRY(p, cudaEventRecord(p->ev_in[slot], p->st_h2d));
    CDD_TRY(p, cudaStreamWaitEvent(p->st_comp, p->ev_in[slot], 0));
    if (c >= 2) CDD_TRY(p, cudaStreamWaitEvent(p->st_comp, p->ev_out[slot], 0));
    if ((rc = run_block(p, p->d_in_stage[slot], p->d_out_stage[slot], nullptr, q_c, p->st_comp)))
      return rc;
    CDD_TRY(p, cudaEventRecord(p->ev_comp[slot], p->st_comp));
    CDD_TRY(p, cudaStreamWaitEvent(p->st_d2h, p->ev_comp[slot], 0));
    CDD_TRY(p, cudaMemcpy2DAsync(h_out + (size_t)c * out_c, out_total * sizeof(float),
                                 p->d_out_stage[slot], out_c * sizeof(float),
                                 out_c * sizeof(float), (size_t)p->n_chan,
                                 cudaMemcpyDeviceToHost, p->st_d2h));
    CDD_TRY(p, cudaEventRecord(p->ev_out[slot], p->st_d2h));
  }
  // the caller's stream continues after the last copy-out, which completes
  // every earlier copy and kernel of this call
  CDD_TRY(p, cudaStreamWaitEvent(stream, p->ev_out[(nc - 1) & 1], 0));
  p->last_launches *= nc;
  return CDD_OK;
}

int cdd_execute_host(cdd_plan p, const int8_t* h_in, float* h_out, cudaStream_t stream) {
  const int rc = cdd_execute_host_async(p, h_in, h_out, stream);
  if (rc) return rc;
  CDD_TRY(p, cudaStreamSynchronize(p->st_d2h));
  return CDD_OK;
}

int cdd_plan_prepare_host(cdd_plan p) {
  const int rc = prepare(p);
  if (rc) return rc;
  return setup_host_path(p);
}

}  // extern "C"

namespace {

struct StateHeader {
  uint32_t magic, version;
  int32_t n_chan, n_fft, n_ov, hop, n_avg, q, pols, taper;
  int64_t ring_len, r_max, g_next, g_next_b, blocks;
  double f_center, bandwidth, dm;
};
constexpr uint32_t kStateMagic = 0x43444453u;     // "SDDC"
constexpr uint32_t kStateVersion = 1;

int64_t state_bytes(const cdd_plan p) {
  const int64_t per_pol = (int64_t)p->n_chan * p->n_ov * (int64_t)sizeof(char2) +
                          (int64_t)p->n_chan * p->r_max * (int64_t)sizeof(float);
  return (int64_t)sizeof(StateHeader) + p->pols * per_pol;
}

StateHeader header_of(const cdd_plan p) {
  StateHeader h = {};
  h.magic = kStateMagic;
  h.version = kStateVersion;
  h.n_chan = p->n_chan;
  h.n_fft = p->n_fft;
  h.n_ov = p->n_ov;
  h.hop = p->hop;
  h.n_avg = p->n_avg;
  h.q = p->q;
  h.pols = p->pols;
  h.taper = p->taper;
  h.ring_len = p->r_max + n_out_per_block(p);
  h.r_max = p->r_max;
  h.f_center = p->f_center;
  h.bandwidth = p->bandwidth;
  h.dm = p->dm;
  return h;
}

bool same_geometry(const StateHeader& a, const StateHeader& b) {
  return a.magic == b.magic && a.version == b.version && a.n_chan == b.n_chan && a.n_fft == b.n_fft &&
         a.n_ov == b.n_ov && a.hop == b.hop && a.n_avg == b.n_avg && a.q == b.q && a.pols == b.pols &&
         a.taper == b.taper && a.ring_len == b.ring_len && a.r_max == b.r_max &&
         a.f_center == b.f_center && a.bandwidth == b.bandwidth && a.dm == b.dm;
}

// The ring entries of stream indices [g_next - r_max, g_next) of every
// channel: at most two column ranges of the [C][ring_len] ring.
template <class F>
int ring_window(cdd_plan p, long long g_next, F copy) {
  const long long L = p->ring_len, rm = p->r_max;
  if (rm == 0) return CDD_OK;
  const long long start = ((g_next - rm) % L + L) % L;
  const long long first = start + rm <= L ? rm : L - start;
  int rc = copy(start, 0LL, first);
  if (rc == CDD_OK && first < rm) rc = copy(0LL, first, rm - first);
  return rc;
}

}  // namespace

extern "C" {

int cdd_plan_state_bytes(cdd_plan p, int64_t* bytes) {
  if (!p || !bytes) return CDD_EINVAL;
  *bytes = state_bytes(p);
  return CDD_OK;
}

int cdd_plan_export_state(cdd_plan p, void* state, int64_t bytes, cudaStream_t s) {
  if (!p || !state || bytes < state_bytes(p)) return CDD_EINVAL;
  if (p->sticky) return p->sticky;
  StateHeader h = header_of(p);
  char* out = static_cast<char*>(state);
  const size_t tb = (size_t)p->n_chan * p->n_ov * sizeof(char2);
  const size_t rb = (size_t)p->n_chan * p->r_max * sizeof(float);
  if (!p->committed) {                       // a fresh stream: zero history
    h.g_next = h.g_next_b = h.blocks = 0;
    memcpy(out, &h, sizeof(h));
    memset(out + sizeof(h), 0, (size_t)(state_bytes(p) - (int64_t)sizeof(h)));
    return CDD_OK;
  }
  int rc = check_device(p);
  if (rc) return rc;
  CDD_TRY(p, cudaStreamSynchronize(s));
  h.g_next = p->g_next;
  h.g_next_b = p->g_next_b;
  h.blocks = p->blocks;
  memcpy(out, &h, sizeof(h));
  char* cur = out + sizeof(h);
  for (int pol = 0; pol < p->pols; ++pol) {
    const char2* tail = pol == 0 ? p->d_tail[p->parity] : p->d_tail_b[p->parity_b];
    const float* ring = pol == 0 ? p->d_ring : p->d_ring_b;
    const long long g = pol == 0 ? p->g_next : p->g_next_b;
    if (tb) CDD_TRY(p, cudaMemcpy(cur, tail, tb, cudaMemcpyDeviceToHost));
    float* rdst = reinterpret_cast<float*>(cur + tb);
    rc = ring_window(p, g, [&](long long col, long long off, long long n) -> int {
      CDD_TRY(p, cudaMemcpy2D(rdst + off, (size_t)p->r_max * sizeof(float), ring + col,
                              (size_t)p->ring_len * sizeof(float), (size_t)n * sizeof(float),
                              (size_t)p->n_chan, cudaMemcpyDeviceToHost));
      return CDD_OK;
    });
    if (rc) return rc;
    cur += tb + rb;
  }
  return CDD_OK;
}

int cdd_plan_import_state(cdd_plan p, const void* state, int64_t bytes, cudaStream_t s) {
  if (!p || !state || bytes < state_bytes(p)) return CDD_EINVAL;
  StateHeader h;
  memcpy(&h, state, sizeof(h));
  if (!same_geometry(h, header_of(p)) || h.g_next < 0 || h.g_next_b < 0 || h.blocks < 0)
    return CDD_EINVAL;
  int rc = prepare(p);
  if (rc) return rc;
  CDD_TRY(p, cudaStreamSynchronize(s));
  const char* cur = static_cast<const char*>(state) + sizeof(h);
  const size_t tb = (size_t)p->n_chan * p->n_ov * sizeof(char2);
  const size_t rb = (size_t)p->n_chan * p->r_max * sizeof(float);
  for (int pol = 0; pol < p->pols; ++pol) {
    char2* tail = pol == 0 ? p->d_tail[0] : p->d_tail_b[0];
    float* ring = pol == 0 ? p->d_ring : p->d_ring_b;
    const long long g = pol == 0 ? h.g_next : h.g_next_b;
    if (tb) CDD_TRY(p, cudaMemcpy(tail, cur, tb, cudaMemcpyHostToDevice));
    const float* rsrc = reinterpret_cast<const float*>(cur + tb);
    rc = ring_window(p, g, [&](long long col, long long off, long long n) -> int {
      CDD_TRY(p, cudaMemcpy2D(ring + col, (size_t)p->ring_len * sizeof(float), rsrc + off,
                              (size_t)p->r_max * sizeof(float), (size_t)n * sizeof(float),
                              (size_t)p->n_chan, cudaMemcpyHostToDevice));
      return CDD_OK;
    });
    if (rc) return rc;
    cur += tb + rb;
  }
  p->g_next = h.g_next;
  p->g_next_b = h.g_next_b;
  p->parity = p->parity_b = 0;
  p->blocks = h.blocks;
  return CDD_OK;
}

int cdd_reset(cdd_plan p) {
  if (!p) return CDD_EINVAL;
  if (p->sticky) return p->sticky;
  if (!p->committed) {
    p->g_next = 0;
    p->parity = 0;
    p->blocks = 0;
    return CDD_OK;
  }
  int rc = check_device(p);
  if (rc) return rc;
  CDD_TRY(p, cudaDeviceSynchronize());
  cudaStream_t s;
  CDD_TRY(p, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  rc = zero_state(p, s);
  cudaError_t e = cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (rc) return rc;
  return fail_cuda(p, e);
}

int cdd_destroy(cdd_plan p) {
  if (!p) return CDD_OK;
  if (p->device >= 0) {
    int prev = -1;
    cudaGetDevice(&prev);
    if (p->device >= 0) cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    free_device(p);
    if (prev >= 0) cudaSetDevice(prev);
  }
  delete p;
  return CDD_OK;
}

}  // extern "C"
