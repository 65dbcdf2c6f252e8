// cdd_static.cu -- cdd_execute_static: one block through the fused kernel
// with every piece of scratch memory carved from a fixed file-scope device
// array, for callers that cannot allocate device memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/cdd.h"
#include "cdd_internal.h"

namespace {

constexpr size_t kScratchBytes = CDD_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The scratch itself.  In host code `g_scratch` names a host-side stand-in,
// not device memory: only the address returned by cudaGetSymbolAddress may be
// handed to a kernel.
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

void* g_scratch_dev[kMaxDevices] = {};
std::mutex g_scratch_mu;

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Device address of g_scratch on the current device (looked up once per device).
cudaError_t scratch_address(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_dev[dev] == nullptr) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = ptr;
  }
  *out = static_cast<unsigned char*>(g_scratch_dev[dev]);
  return cudaSuccess;
}

}  // namespace

extern "C" int cdd_execute_static(double f_center_mhz, double bandwidth_mhz, int n_chan,
                                  double dm, int n_fft, int n_avg, int n_seg, int taper,
                                  const int8_t* d_in, float* d_out, cudaStream_t stream) {
  cdd::Geometry g;
  int rc = cdd::geometry(&g, f_center_mhz, bandwidth_mhz, n_chan, dm, n_fft, n_avg);
  if (rc != CDD_OK) return rc;
  if (cdd::needs_channel_major(g.logn)) return CDD_EUNSUPPORTED;   // cluster form needs a copy
  if (!d_in || !d_out || n_seg < 1 || taper < CDD_TAPER_NONE || taper > CDD_TAPER_WELCH)
    return CDD_EINVAL;
  if ((int64_t)n_seg * n_chan >= ((int64_t)1 << 31)) return CDD_EINVAL;
  const int64_t n_out = (int64_t)n_seg * g.hop / n_avg;
  if (n_out >= ((int64_t)1 << 31)) return CDD_EINVAL;
  const int64_t ring_len = g.r_max > 0 ? g.r_max : 1;    // only spilled outputs land here

  // scratch layout, each piece 256-byte aligned
  const size_t b_tw = align256((size_t)cdd::twiddle_table_len(g.logn) * sizeof(float2));
  const size_t b_chirp = align256((size_t)n_chan * g.n_fft * sizeof(float2));
  const size_t b_shift = align256((size_t)n_chan * sizeof(int));
  const size_t b_tail = align256((size_t)n_chan * (g.n_ov > 0 ? g.n_ov : 1) * sizeof(char2));
  const size_t b_ring = align256((size_t)n_chan * ring_len * sizeof(float));
  const size_t total = b_tw + b_chirp + b_shift + 2 * b_tail + b_ring;
  if (total > kScratchBytes) return CDD_ETOOBIG;

  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return CDD_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return CDD_EUNSUPPORTED;
  unsigned char* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess) return CDD_ECUDA;

  float2* tw = reinterpret_cast<float2*>(base);
  float2* chirp = reinterpret_cast<float2*>(base + b_tw);
  int* shift = reinterpret_cast<int*>(base + b_tw + b_chirp);
  char2* tail_zero = reinterpret_cast<char2*>(base + b_tw + b_chirp + b_shift);
  char2* tail_sink = reinterpret_cast<char2*>(base + b_tw + b_chirp + b_shift + b_tail);
  float* ring = reinterpret_cast<float*>(base + b_tw + b_chirp + b_shift + 2 * b_tail);

  cudaError_t e = cdd::launch_twiddle_table(g.logn, tw, stream);
  if (e == cudaSuccess)
    e = cdd::launch_chirp_table(g.logn, chirp, n_chan, g.f_base, g.chan_bw, dm, taper, g.sideband,
                                stream);
  if (e == cudaSuccess)
    e = cdd::launch_shift_table(shift, n_chan, g.f_base, g.f_ref, g.chan_bw, dm, n_avg, g.sideband,
                                stream);
  if (e == cudaSuccess && g.n_ov > 0)     // the stream starts with zeros; the array keeps old data
    e = cudaMemsetAsync(tail_zero, 0, (size_t)n_chan * g.n_ov * sizeof(char2), stream);
  if (e != cudaSuccess) return CDD_ECUDA;

  cdd::OlsArgs a;
  a.in = reinterpret_cast<const char2*>(d_in);
  a.in_cm = nullptr;
  a.rows = 0;
  a.out = d_out;
  a.chirp = chirp;
  a.tw = tw;
  a.tail_rd = g.n_ov > 0 ? tail_zero : nullptr;
  a.tail_wr = g.n_ov > 0 ? tail_sink : nullptr;
  a.ring = ring;
  a.shift = shift;
  a.volt = nullptr;
  a.dft = nullptr;
  a.n_chan = n_chan;
  a.n_ov = g.n_ov;
  a.hop = g.hop;
  a.n_avg = n_avg;
  a.q = n_seg;
  a.s_begin = 0;
  a.s_count = n_seg;
  a.n_out = (int)n_out;
  a.g0 = 0;
  a.ring_len = ring_len;
  return cdd::launch_ols(g.logn, a, stream) == cudaSuccess ? CDD_OK : CDD_ECUDA;
}
