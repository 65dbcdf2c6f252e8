// cdd_kernels.cu -- the fused per-channel overlap-save coherent-dedispersion
// kernel and the FP64 table builders.
//
// One transform (one channel, one overlap-save segment) per T = N / R_0
// threads; for small N a CTA holds several transforms so that it has at least
// 256 threads.  A segment never leaves the SM between the int8 load and the
// float intensity store:
//
//   pass 0 fwd   int8 (re,im) gathered from [row][C] -> registers -> radix R_0
//                DIF butterfly -> twiddle -> shared memory
//   passes 1..   radix DIF passes in shared memory (in place)
//   middle       last forward radix, multiply by the chirp function
//                (Sec. 2.1 Eq. 3 times the Sec. 2.2 taper, 1/N folded in),
//                first inverse radix -- one register round trip
//   passes ..1   radix DIT passes in shared memory
//   pass 0 inv   twiddle -> radix R_0 DIT -> natural-order voltages
//                -> |v|^2 (Sec. 3.1) -> shared memory -> sums of n_avg
//                -> discard the first n_ov (Sec. 2.2) -> aligned store
//                (Sec. 1.2): output index = stream index + r_k, or the ring
//                when it falls in a later block.
//
// The overlap of segment 0 (the last n_ov samples of the previous block) is
// read from a per-channel tail that the last segment of every block rewrites
// (Sec. 4.3: the samples lost at the end of a block are prefixed to the next).
#include "cdd_fft.cuh"
#include "cdd_internal.h"

namespace cdd {

namespace {

constexpr double kDispD = 4.148808e3;   // s MHz^2 cm^3 / pc (Eq. 3)
constexpr int kMinCtaThreads = 256;

template <int LOGN>
struct Cfg {
  using PL = PassPlan<LOGN>;
  static constexpr int T = PL::T;
  static constexpr int G = T >= kMinCtaThreads ? 1 : kMinCtaThreads / T;   // transforms per CTA
  static constexpr int THREADS = G * T;
#ifdef CDD_OLS_MINB
  static constexpr int MINB = THREADS <= 256 ? CDD_OLS_MINB : 1;          // CTAs per SM to aim for
#else
  static constexpr int MINB = THREADS <= 256 ? 2 : 1;
#endif
  static constexpr int SEG_F2 = padded_len(PL::N);                       // float2 per transform
  static constexpr size_t SMEM = size_t(G) * SEG_F2 * sizeof(float2);
};

// Forward (DIF) radix pass p >= 1, in place.
template <int LOGN, int p>
__device__ __forceinline__ void fwd_pass(float2* buf, const float2* __restrict__ tw, int lt) {
  using PL = PassPlan<LOGN>;
  constexpr int R = PL::R(p), S = PL::S(p), M = PL::M(p);
  constexpr int PER = (PL::N / R) / PL::T;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int b = lt + i * PL::T;
    const int t = b % S;
    const int base = (b / S) * M + t;
    float2 v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = buf[pad(base + S * j)];
    dft<R, -1>(v);
    if constexpr (S > 1) {
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmul(v[k], __ldg(&tw[PL::TwOff(p) + k * S + t]));
    }
#pragma unroll
    for (int k = 0; k < R; ++k) buf[pad(base + S * k)] = v[k];
  }
}

// Inverse (DIT) radix pass p >= 1, in place: conjugate twiddle, then butterfly.
template <int LOGN, int p>
__device__ __forceinline__ void inv_pass(float2* buf, const float2* __restrict__ tw, int lt) {
  using PL = PassPlan<LOGN>;
  constexpr int R = PL::R(p), S = PL::S(p), M = PL::M(p);
  constexpr int PER = (PL::N / R) / PL::T;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int b = lt + i * PL::T;
    const int t = b % S;
    const int base = (b / S) * M + t;
    float2 v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = buf[pad(base + S * k)];
    if constexpr (S > 1) {
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmulc(v[k], __ldg(&tw[PL::TwOff(p) + k * S + t]));
    }
    dft<R, 1>(v);
#pragma unroll
    for (int j = 0; j < R; ++j) buf[pad(base + S * j)] = v[j];
  }
}

// Last forward radix, chirp multiply, first inverse radix (stride-1 groups).
template <int LOGN>
__device__ __forceinline__ void chirp_pass(float2* buf, const float2* __restrict__ chirp_k, int lt) {
  using PL = PassPlan<LOGN>;
  constexpr int R = PL::RL;
  constexpr int NG = PL::N / R;
  constexpr int PER = NG / PL::T;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int q = lt + i * PL::T;
    const int base = q * R;
    float2 v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = buf[pad(base + j)];
    dft<R, -1>(v);
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = cmul(v[k], __ldg(&chirp_k[k * NG + q]));
    dft<R, 1>(v);
#pragma unroll
    for (int j = 0; j < R; ++j) buf[pad(base + j)] = v[j];
  }
}

template <int LOGN>
__global__ void __launch_bounds__(Cfg<LOGN>::THREADS, Cfg<LOGN>::MINB)
ols_kernel(const OlsArgs a) {
  using PL = PassPlan<LOGN>;
  using CF = Cfg<LOGN>;
  constexpr int N = PL::N;
  constexpr int T = PL::T;
  constexpr int R0 = PL::R(0);
  static_assert(PL::S(0) == T, "pass 0 stride must equal the threads per transform");

  extern __shared__ float2 smem[];
  const int g = threadIdx.x / T;
  const int lt = threadIdx.x % T;
  float2* buf = smem + g * CF::SEG_F2;
  const int w = blockIdx.x * CF::G + g;        // n_chan * q < 2^31 (checked by the plan)
  const bool active = w < a.n_chan * a.q;
  const int k = active ? w % a.n_chan : 0;     // channel fastest: neighbouring CTAs
  const int s = active ? w / a.n_chan : 0;     // share the input rows in L2

  // ---- pass 0, forward: unpack and gather x[lt + T*j] of this segment
  float2 v[R0];
  if (active) {
    const long long row0 = (long long)s * a.hop - a.n_ov;
    const bool last = (s == a.q - 1);
    char2 c[R0];
#pragma unroll
    for (int j = 0; j < R0; ++j) {                 // issue every load before using any
      const long long row = row0 + lt + T * j;
      const char2* src = row >= 0 ? a.in + row * a.n_chan + k
                                  : a.tail_rd + (long long)k * a.n_ov + (row + a.n_ov);
      c[j] = __ldg(src);
    }
#pragma unroll
    for (int j = 0; j < R0; ++j) {
      const int n = lt + T * j;
      if (last && n >= N - a.n_ov) a.tail_wr[(long long)k * a.n_ov + (n - (N - a.n_ov))] = c[j];
      v[j] = make_float2((float)c[j].x, (float)c[j].y);
    }
    dft<R0, -1>(v);
#pragma unroll
    for (int kk = 1; kk < R0; ++kk) v[kk] = cmul(v[kk], __ldg(&a.tw[kk * T + lt]));
#pragma unroll
    for (int kk = 0; kk < R0; ++kk) buf[pad(lt + T * kk)] = v[kk];
  }
  __syncthreads();

  static_for<1, PL::P - 1>([&](auto P_) {
    if (active) fwd_pass<LOGN, decltype(P_)::value>(buf, a.tw, lt);
    __syncthreads();
  });

  if (active) chirp_pass<LOGN>(buf, a.chirp + (size_t)k * N, lt);
  __syncthreads();

  static_for<1, PL::P - 1>([&](auto I_) {
    if (active) inv_pass<LOGN, PL::P - 1 - decltype(I_)::value>(buf, a.tw, lt);
    __syncthreads();
  });

  // ---- pass 0, inverse: natural-order voltages v[j] = z[lt + T*j]
  if (active) {
#pragma unroll
    for (int kk = 0; kk < R0; ++kk) v[kk] = buf[pad(lt + T * kk)];
#pragma unroll
    for (int kk = 1; kk < R0; ++kk) v[kk] = cmulc(v[kk], __ldg(&a.tw[kk * T + lt]));
    dft<R0, 1>(v);
    if (a.volt != nullptr) {
      const long long vbase = ((long long)k * a.q + s) * a.hop - a.n_ov;
#pragma unroll
      for (int j = 0; j < R0; ++j) {
        const int n = lt + T * j;
        if (n >= a.n_ov) a.volt[vbase + n] = v[j];
      }
    }
  }
  __syncthreads();                       // every thread has read buf: reuse it
  float* pw = reinterpret_cast<float*>(buf);
  if (active) {
#pragma unroll
    for (int j = 0; j < R0; ++j) {
      const int n = lt + T * j;
      pw[n + (n >> 5)] = fmaf(v[j].x, v[j].x, v[j].y * v[j].y);   // one spare word per 32
    }
  }
  __syncthreads();

  if (active) {
    const int n_int = a.hop / a.n_avg;
    const int r = __ldg(&a.shift[k]);
    const long long gseg = a.g0 + (long long)s * n_int;
    float* outk = a.out + (size_t)k * a.n_out;
    float* ringk = a.ring + (size_t)k * a.ring_len;
    for (int m = lt; m < n_int; m += T) {
      const int n0 = a.n_ov + m * a.n_avg;
      float acc = 0.f;
      for (int i = 0; i < a.n_avg; ++i) acc += pw[(n0 + i) + ((n0 + i) >> 5)];
      const long long gi = gseg + m;              // stream index of this output
      const long long dst = gi + r - a.g0;        // its aligned index in this block
      if (dst < a.n_out) outk[dst] = acc;
      else ringk[gi % a.ring_len] = acc;
    }
    if (s == 0) {                                 // block prefix: earlier blocks' samples
      const int lim = r < a.n_out ? r : a.n_out;
      for (int m = lt; m < lim; m += T) {
        const long long src = a.g0 + m - r;
        outk[m] = src >= 0 ? ringk[src % a.ring_len] : 0.f;
      }
    }
  }
}

template <int LOGN>
__global__ void chirp_table_kernel(float2* chirp, int n_chan, double f_lo0, double chan_bw,
                                   double dm, int taper) {
  using PL = PassPlan<LOGN>;
  constexpr int N = PL::N;
  constexpr int NG = N / PL::RL;
  const long long total = (long long)n_chan * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / N);
    const int idx = (int)(e % N);
    const int pos = (idx % NG) * PL::RL + idx / NG;       // table index kk*NG + q
    const int bin = position_to_bin<LOGN>(pos);
    const int sbin = bin < N / 2 ? bin : bin - N;
    const double f_lo = f_lo0 + chan_bw * k;
    const double f_l = sbin * (chan_bw / N) + 0.5 * chan_bw;
    // Eq. 3 phase in turns, reduced to [-1/2, 1/2] before the sine and cosine
    const double turns = kDispD * 1e6 * dm * f_l * f_l / ((f_l + f_lo) * f_lo * f_lo);
    const double frac = turns - rint(turns);
    double sn, cs;
    sincospi(2.0 * frac, &sn, &cs);
    double wt = 1.0;
    const double x = f_l / chan_bw;
    if (taper == 1) {
      const double sx = sinpi(x);
      wt = sx * sx;
    } else if (taper == 2) {
      const double y = 2.0 * x - 1.0;
      wt = 1.0 - y * y;
    }
    const double sc = wt / N;
    chirp[e] = make_float2((float)(cs * sc), (float)(-sn * sc));   // exp(-i Phi) w / N
  }
}

// Twiddle table in the per-pass thread-major layout of PassPlan::TwOff.
template <int LOGN>
__global__ void twiddle_kernel(float2* tw) {
  using PL = PassPlan<LOGN>;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < PL::TW_LEN; e += gridDim.x * blockDim.x) {
    int p = 0;
    while (p + 1 < PL::P - 1 && e >= PL::TwOff(p + 1)) ++p;
    const int local = e - PL::TwOff(p);
    const int stride = p == 0 ? PL::T : PL::S(p);            // thread index range
    const int modulus = p == 0 ? PL::N : PL::M(p);
    const int t = local % stride, k = local / stride;
    const int m = (t * k) % modulus;
    double sn, cs;
    sincospi(2.0 * m / modulus, &sn, &cs);
    tw[e] = make_float2((float)cs, (float)(-sn));           // exp(-2 pi i m / modulus)
  }
}

// Alignment shifts r_k (Sec. 1.2) computed on the device, for callers that
// keep no host-side copy of them.
__global__ void shift_kernel(int* shift, int n_chan, double f_lo0, double chan_bw, double dm,
                             int n_avg) {
  const double ref = pow(f_lo0, -2.0);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_chan; k += gridDim.x * blockDim.x) {
    const double f_k = f_lo0 + chan_bw * k;
    const double delay = kDispD * dm * (pow(f_k, -2.0) - ref);
    shift[k] = (int)rint(-delay * chan_bw * 1e6 / n_avg);
  }
}

template <int LOGN>
cudaError_t launch_ols_t(const OlsArgs& a, cudaStream_t s) {
  using CF = Cfg<LOGN>;
  static bool attr_set[128] = {};            // per device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  if (!attr_set[dev]) {
    e = cudaFuncSetAttribute(ols_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CF::SMEM);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const long long work = (long long)a.n_chan * a.q;
  const unsigned grid = (unsigned)((work + CF::G - 1) / CF::G);
  ols_kernel<LOGN><<<grid, CF::THREADS, CF::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int LOGN>
cudaError_t launch_chirp_t(float2* chirp, int n_chan, double f_lo0, double chan_bw, double dm,
                           int taper, cudaStream_t s) {
  const long long total = (long long)n_chan << LOGN;
  const unsigned grid = (unsigned)((total + 255) / 256 < 65535 ? (total + 255) / 256 : 65535);
  chirp_table_kernel<LOGN><<<grid, 256, 0, s>>>(chirp, n_chan, f_lo0, chan_bw, dm, taper);
  return cudaGetLastError();
}

}  // namespace

#define CDD_LOGN_CASES(X) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14)

cudaError_t launch_ols(int logn, const OlsArgs& a, cudaStream_t s) {
  switch (logn) {
#define X(L) case L: return launch_ols_t<L>(a, s);
    CDD_LOGN_CASES(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_chirp_table(int logn, float2* chirp, int n_chan, double f_lo0_mhz,
                               double chan_bw_mhz, double dm, int taper, cudaStream_t s) {
  switch (logn) {
#define X(L) case L: return launch_chirp_t<L>(chirp, n_chan, f_lo0_mhz, chan_bw_mhz, dm, taper, s);
    CDD_LOGN_CASES(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

template <int LOGN>
cudaError_t launch_twiddle_t(float2* tw, cudaStream_t s) {
  twiddle_kernel<LOGN><<<(PassPlan<LOGN>::TW_LEN + 255) / 256, 256, 0, s>>>(tw);
  return cudaGetLastError();
}

cudaError_t launch_twiddle_table(int logn, float2* tw, cudaStream_t s) {
  switch (logn) {
#define X(L) case L: return launch_twiddle_t<L>(tw, s);
    CDD_LOGN_CASES(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_shift_table(int* shift, int n_chan, double f_lo0_mhz, double chan_bw_mhz,
                               double dm, int n_avg, cudaStream_t s) {
  const int grid = (n_chan + 255) / 256 < 1024 ? (n_chan + 255) / 256 : 1024;
  shift_kernel<<<grid, 256, 0, s>>>(shift, n_chan, f_lo0_mhz, chan_bw_mhz, dm, n_avg);
  return cudaGetLastError();
}

int twiddle_table_len(int logn) {
  switch (logn) {
#define X(L) case L: return PassPlan<L>::TW_LEN;
    CDD_LOGN_CASES(X)
#undef X
    default: return 0;
  }
}

int ols_threads(int logn) {
  switch (logn) {
#define X(L) case L: return Cfg<L>::THREADS;
    CDD_LOGN_CASES(X)
#undef X
    default: return 0;
  }
}

int ols_segments_per_cta(int logn) {
  switch (logn) {
#define X(L) case L: return Cfg<L>::G;
    CDD_LOGN_CASES(X)
#undef X
    default: return 0;
  }
}

size_t ols_smem_bytes(int logn) {
  switch (logn) {
#define X(L) case L: return Cfg<L>::SMEM;
    CDD_LOGN_CASES(X)
#undef X
    default: return 0;
  }
}

}  // namespace cdd
