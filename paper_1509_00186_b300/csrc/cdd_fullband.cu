// cdd_fullband.cu -- the paper's full-band mode: the voltage beam's frames of
// 2C-point spectra are inverse transformed back to the real series (Sec. 3.1),
// and one long transform over the whole band is chirped and inverted with
// overlap-save (Sec. 2.3, Sec. 4.3), then squared and integrated (Sec. 3.1).
//
// The real series is transformed as a complex one (zero imaginary part) with a
// Hermitian chirp, so the inverse is real up to rounding and its real part is
// kept.  N = L_out * L_mid, L_mid = min(N, 16384) below N = 2^20 and 8192
// from there on:
//   outer DIF passes   through HBM: radix-64 and radix-128 tiles of
//                      neighbouring butterflies, their DFT done in two radix
//                      stages through shared memory, and radix <= 16 register
//                      passes (one thread per butterfly) for the bits left
//   middle kernel      each contiguous L_mid sub-transform in shared memory:
//                      forward passes, chirp, inverse passes
//   outer DIT passes   back through HBM; the last writes Re(y)^2, or sums the
//                      windows of the kept part across lanes and writes them
//   integrate          sums n_avg samples of the kept part of the segment,
//                      where the last pass does not
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/cdd.h"
#include "cdd_fft.cuh"
#include "cdd_internal.h"
#include "cdd_passes.cuh"

namespace cdd {
namespace {

using namespace passes;

constexpr int kMidLog = 14;                 // L_mid for 16384 < N < 2^kTileMinLog
constexpr int kTileMinLog = 20;             // from here on L_mid = 8192 with tile passes around it
constexpr int kTwLoBits = 13;               // two-level twiddle table split

// w_N^e = hi[e >> 13] * lo[e & 8191]
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ hi, const float2* __restrict__ lo,
                                          long long e) {
  return cmul(__ldg(&hi[e >> kTwLoBits]), __ldg(&lo[e & ((1 << kTwLoBits) - 1)]));
}

// w[k] = w_N^{k e1} for 0 < k < R: the powers of two from the tables, the
// rest as products (at most three deep), so a radix-16 butterfly makes 8
// table loads instead of 30.
template <int R>
__device__ __forceinline__ void twiddle_powers(const float2* __restrict__ hi, const float2* __restrict__ lo,
                                               long long e1, float2 (&w)[R]) {
  static_for<1, R>([&](auto K_) {
    constexpr int k = decltype(K_)::value;
    constexpr int top = 1 << ilog2(k);             // highest power of two <= k
    if constexpr (top == k) w[k] = twiddle(hi, lo, e1 * k);
    else w[k] = cmul(w[k - top], w[top]);
  });
}

// ---- inverse channelisation: frame t of C bins -> 2C real samples --------
// x[n] = (1/F) sum_b Y[b] e^{+2 pi i b n / F} over the Hermitian extension Y
// of the frame (bin 0 real part only, bin C zero), F = 2C.  Since x is real,
// x[n] = Re(DFT(conj Y))[n] / F: the forward passes run on conj Y gathered in
// natural bin order straight from the frame (neighbouring lanes read
// neighbouring bytes), and sample n is read back from the position that holds
// bin n, so the stores are coalesced too.
template <int LOGF>
__global__ void __launch_bounds__(Cfg<LOGF>::THREADS)
icf_kernel(const char2* __restrict__ in, float* __restrict__ ts, const float2* __restrict__ twf,
           long long n_frames, int n_chan) {
  using PL = PassPlan<LOGF>;
  using CF = Cfg<LOGF>;
  constexpr int F = PL::N;                  // 2C
  constexpr int C = F / 2;
  constexpr int T = PL::T;
  constexpr int R0 = PL::R(0);
  constexpr int RL = PL::RL;
  static_assert(RL <= 16, "stride-1 groups must not cross a padding word");
  extern __shared__ __align__(16) float2 smem[];
  const int g = threadIdx.x / T;
  const int lt = threadIdx.x % T;
  float2* buf = smem + g * CF::SEG_F2;
  const long long t = (long long)blockIdx.x * CF::G + g;
  const bool active = t < n_frames;
  if (active) {
    const unsigned short* row = reinterpret_cast<const unsigned short*>(in) + t * n_chan;
    float2 v[R0];
#pragma unroll
    for (int j = 0; j < R0; ++j) {
      const int b = lt + T * j;
      if (b < C) {                            // conj X[b]; bin 0 keeps its real part only
        v[j] = unpack_i8x2(__ldg(row + b));
        v[j].y = b == 0 ? 0.f : -v[j].y;
      } else if (b > C) {                     // conj of conj X[F - b]
        v[j] = unpack_i8x2(__ldg(row + (F - b)));
      } else {
        v[j] = make_float2(0.f, 0.f);         // the Nyquist bin is not recorded
      }
    }
    dft<R0, -1>(v);
#pragma unroll
    for (int kk = 1; kk < R0; ++kk) v[kk] = cmul(v[kk], __ldg(&twf[kk * T + lt]));
    float2* pb0 = buf + pad<LOGF>(lt);
#pragma unroll
    for (int kk = 0; kk < R0; ++kk) pb0[poff<LOGF, T>(kk)] = v[kk];
  }
  __syncthreads();
  static_for<1, PL::P - 1>([&](auto P_) {
    if (active) fwd_pass<LOGF, decltype(P_)::value>(buf, twf, lt);
    __syncthreads();
  });
  if constexpr (PL::P >= 2) {                 // the last radix on stride-1 groups
    if (active) {
      for (int q = lt; q < F / RL; q += T) {
        float2* pb = buf + pad<LOGF>(q * RL);
        float2 x[RL];
        load_group<LOGF, RL>(pb, x);
        dft<RL, -1>(x);
        store_group<LOGF, RL>(pb, x);
      }
    }
    __syncthreads();
  }
  if (active) {
    float* out = ts + t * F;
    for (int n = lt; n < F; n += T) out[n] = buf[pad<LOGF>(bin_to_position<LOGF>(n))].x * (1.0f / F);
  }
}

// Frames of C = 2^LOGC bins (F = 2C real samples), the same result through a
// C-point complex transform: with X[C] = 0 and bin 0 real,
//   E[k] = X[k] + conj X[C-k],  O[k] = (X[k] - conj X[C-k]) e^{+2 pi i k/F},
//   z[n] = x[2n] + i x[2n+1] = (1/F) sum_k (E[k] + i O[k]) e^{+2 pi i k n/C}
// (split the F-point sum into even and odd samples; Hermitian symmetry gives
// X[k+C] = conj X[C-k]).  As above, the forward passes run on conj(E + iO)
// in natural order and z[n] = conj(Y[n]) / F is read back from the position
// holding bin n; each z[n] is one float2 store of two neighbouring samples.
template <int LOGC>
__global__ void __launch_bounds__(Cfg<LOGC>::THREADS, Cfg<LOGC>::MINB)
icf_half_kernel(const char2* __restrict__ in, float* __restrict__ ts, const float2* __restrict__ twc,
                const float2* __restrict__ wk, long long n_frames) {
  using PL = PassPlan<LOGC>;
  using CF = Cfg<LOGC>;
  constexpr int C = PL::N;
  constexpr int F = 2 * C;
  constexpr int T = PL::T;
  constexpr int R0 = PL::R(0);
  constexpr int RL = PL::RL;
  static_assert(RL <= 16, "stride-1 groups must not cross a padding word");
  extern __shared__ __align__(16) float2 smem[];
  const int g = threadIdx.x / T;
  const int lt = threadIdx.x % T;
  float2* buf = smem + g * CF::SEG_F2;
  const long long t = (long long)blockIdx.x * CF::G + g;
  const bool active = t < n_frames;
  if (active) {
    const unsigned short* row = reinterpret_cast<const unsigned short*>(in) + t * C;
    float2 v[R0];
#pragma unroll
    for (int j = 0; j < R0; ++j) {
      const int k = lt + T * j;
      float2 xk = unpack_i8x2(__ldg(row + k));
      float2 xp = unpack_i8x2(__ldg(row + (k == 0 ? 0 : C - k)));   // X[C - k]
      if (k == 0) {                          // bin 0 real part only; X[C] is not recorded
        xk.y = 0.f;
        xp = make_float2(0.f, 0.f);
      }
      const float2 e = make_float2(xk.x + xp.x, xk.y - xp.y);
      const float2 o = cmul(make_float2(xk.x - xp.x, xk.y + xp.y), __ldg(&wk[k]));
      v[j] = make_float2(e.x - o.y, -(e.y + o.x));                   // conj(E + i O)
    }
    dft<R0, -1>(v);
#pragma unroll
    for (int kk = 1; kk < R0; ++kk) v[kk] = cmul(v[kk], __ldg(&twc[kk * T + lt]));
    float2* pb0 = buf + pad<LOGC>(lt);
#pragma unroll
    for (int kk = 0; kk < R0; ++kk) pb0[poff<LOGC, T>(kk)] = v[kk];
  }
  __syncthreads();
  static_for<1, PL::P - 1>([&](auto P_) {
    if (active) fwd_pass<LOGC, decltype(P_)::value>(buf, twc, lt);
    __syncthreads();
  });
  if (active) {                              // the last radix on stride-1 groups
    for (int q = lt; q < C / RL; q += T) {
      float2* pb = buf + pad<LOGC>(q * RL);
      float2 x[RL];
      load_group<LOGC, RL>(pb, x);
      dft<RL, -1>(x);
      store_group<LOGC, RL>(pb, x);
    }
  }
  __syncthreads();
  if (active) {
    float2* out2 = reinterpret_cast<float2*>(ts + t * F);
#pragma unroll 4
    for (int n = lt; n < C; n += T) {
      const float2 y = buf[pad<LOGC>(bin_to_position<LOGC>(n))];
      out2[n] = make_float2(y.x * (1.0f / F), -y.y * (1.0f / F));
    }
  }
}

// wk[k] = e^{+2 pi i k / (2C)}, k < C (FP64, rounded once)
__global__ void fb_wk_kernel(float2* wk, int c) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < c; k += gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi((double)k / (double)c, &sn, &cs);
    wk[k] = make_float2((float)cs, (float)sn);
  }
}

// ---- outer passes through HBM --------------------------------------------
// DIF radix-R pass of stride S = 2^ls over N points (sub-problems of M = R*S),
// in place.  FIRST: the input is the real series ts (imaginary part zero).
// Butterfly b: t = b mod S, base = (b div S) * M + t; its twiddles are
// w_M^{t k} = w_N^{t k N/M} with t k < M, so no reduction is needed.
template <int R, bool FIRST>
__global__ void __launch_bounds__(256, 3)
outer_fwd_kernel(float2* __restrict__ w, const float* __restrict__ ts, long long n, int ls,
                 const float2* __restrict__ thi, const float2* __restrict__ tlo) {
  constexpr int LR = ilog2(R);
  const long long s = 1LL << ls;
  const long long nb = n >> LR;
  const long long step = n >> (ls + LR);
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb;
       b += (long long)gridDim.x * blockDim.x) {
    const long long t = b & (s - 1);
    const long long base = ((b >> ls) << (ls + LR)) + t;
    float2 v[R];
#pragma unroll
    for (int j = 0; j < R; ++j)
      v[j] = FIRST ? make_float2(__ldg(&ts[base + s * j]), 0.f) : w[base + s * j];
    dft<R, -1>(v);
    float2 tw[R];
    twiddle_powers<R>(thi, tlo, t * step, tw);
#pragma unroll
    for (int k = 1; k < R; ++k) v[k] = cmul(v[k], tw[k]);
#pragma unroll
    for (int k = 0; k < R; ++k) w[base + s * k] = v[k];
  }
}

// DIT radix-R pass of stride S = 2^ls, in place.  LAST (stride N/R, so a
// thread's butterfly is samples b + S*j): NA = 0 writes Re(y)^2 to pw; NA > 0
// also detects and sums windows of NA samples across neighbouring lanes
// (consecutive b are consecutive samples; NA <= R, a power of two) and writes
// the window sums of the kept part straight to out (window m starts at
// n_ov + m*NA).
template <int R, bool LAST, int NA = 0>
__global__ void __launch_bounds__(256, 3)
outer_inv_kernel(float2* __restrict__ w, float* __restrict__ pw, long long n, int ls,
                 const float2* __restrict__ thi, const float2* __restrict__ tlo,
                 float* __restrict__ out, long long n_ov) {
  constexpr int LR = ilog2(R);
  static_assert(NA == 0 || (LAST && NA <= R && (NA & (NA - 1)) == 0), "lane windows");
  const long long s = 1LL << ls;
  const long long nb = n >> LR;
  const long long step = n >> (ls + LR);
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb;
       b += (long long)gridDim.x * blockDim.x) {
    const long long t = b & (s - 1);
    const long long base = ((b >> ls) << (ls + LR)) + t;
    const long long e1 = t * step;
    float2 v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = w[base + s * k];
    float2 tw[R];
    twiddle_powers<R>(thi, tlo, e1, tw);
#pragma unroll
    for (int k = 1; k < R; ++k) v[k] = cmulc(v[k], tw[k]);
    dft<R, 1>(v);
    if constexpr (NA > 0) {
      float u[R];
#pragma unroll
      for (int j = 0; j < R; ++j) u[j] = v[j].x * v[j].x;
      const int lane = threadIdx.x & 31;
      lane_window_sums<R, NA>(u, lane);
      constexpr int V = R / NA;
      const long long first = base - (lane & (NA - 1));
#pragma unroll
      for (int i = 0; i < V; ++i) {
        const long long n0 = first + s * (V * (lane & (NA - 1)) + i);
        if (n0 >= n_ov) out[(n0 - n_ov) / NA] = u[i];
      }
    } else {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        if (LAST) pw[base + s * j] = v[j].x * v[j].x;
        else w[base + s * j] = v[j];
      }
    }
  }
}

// ---- outer radix-64 passes, as 8 x 8 through shared memory ----------------
// The same DIF (forward) and DIT (inverse) radix-64 butterflies as the
// register passes above, one HBM round trip for six bits of the outer index
// instead of four.  A CTA takes kTileCols neighbouring butterflies of one
// stride-S block: rows base + S*j (j < 64) by columns t0 .. t0 + kTileCols - 1,
// a lane two neighbouring columns, so every warp access is a 512-byte row
// piece of 16-byte words.  With j = 8*j1 + j2 and k = k1 + 8*k2,
//   X[k1 + 8 k2] = sum_j2 w_8^{j2 k2} w_64^{j2 k1} sum_j1 w_8^{j1 k1} v[8 j1 + j2]:
// warp j2 does the inner radix-8 over j1 straight from global memory and
// parks Y_j2[k1] (times w_64^{j2 k1}) in row 8*k1 + j2 of the tile; after the
// barrier warp k1 reads rows 8*k1 .. 8*k1 + 7 and does the radix-8 over j2.
// w_64^m = w_N^{m N/64} is one entry of the high table (N/64 is a multiple
// of its 8192-entry step).
constexpr int kTileCols = 64;
constexpr int kTileThreads = 256;              // 8 warps: j2 (stage 1) or k1 (stage 2)

__device__ __forceinline__ float2 w64(const float2* __restrict__ thi, long long n, int m) {
  return __ldg(&thi[(long long)(m & 63) * (n >> 19)]);
}
__device__ __forceinline__ float4 pack2(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

// The outer twiddles of a lane's two columns t and t + 1 for its rows
// k = k1 + 8*k2 (k2 < 8), w_N^{e1 k} with e1 = t*step: w_N^{e1 k1} times the
// powers of w_N^{8 e1}, and those of column t + 1 the same times w_N^{step k}
// (entries that are the same across the warp).  A lane's column is
// t = t0 + 2*lane (t0 the tile's first column), so w_N^{m t step} is the
// warp's w_N^{m t0 step} times the lane-table entry w_N^{2 m lane step}
// (kLaneRows rows of 32 lanes per pass, m = 1..7, 8, 16, 32; then the 64
// factors w_N^{step k}): every table access is either one entry for the whole
// warp or 32 neighbouring entries.
constexpr int kLaneRows = 10;
__host__ __device__ constexpr int lane_row_m(int r) { return r < 7 ? r + 1 : 8 << (r - 7); }
// The radix-128 passes (one column per lane, t = t0 + lane) use rows
// w_N^{m lane step} for m = 1..15, 16, 32, 64.
constexpr int kLaneRows128 = 18;
__host__ __device__ constexpr int lane_row_m128(int r) { return r < 15 ? r + 1 : 16 << (r - 15); }
constexpr int kLaneTable = kLaneRows * 32 + 64 > kLaneRows128 * 32 ? kLaneRows * 32 + 64 : kLaneRows128 * 32;

struct Tw8x2 {
  float2 u[8], v[8];
  __device__ __forceinline__ Tw8x2(const float2* __restrict__ thi, const float2* __restrict__ tlo,
                                   const float2* __restrict__ lanes, long long t0, long long step, int k1,
                                   int lane) {
    // w_N^{m t step} for the lane's t, from row r of the lane table
    auto wt = [&](int r) {
      return cmul(twiddle(thi, tlo, (long long)lane_row_m(r) * t0 * step), __ldg(&lanes[r * 32 + lane]));
    };
    float2 q[8];                                   // q[k2] = w_N^{8 e1 k2}
    q[1] = wt(7);
    q[2] = wt(8);
    q[4] = wt(9);
    q[3] = cmul(q[2], q[1]);
    q[5] = cmul(q[4], q[1]);
    q[6] = cmul(q[4], q[2]);
    q[7] = cmul(q[4], q[3]);
    const float2 a = k1 == 0 ? make_float2(1.f, 0.f) : wt(k1 - 1);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
      u[k2] = k2 == 0 ? a : cmul(a, q[k2]);
      v[k2] = cmul(u[k2], __ldg(&lanes[kLaneRows * 32 + k1 + 8 * k2]));
    }
  }
};

// Radix 64: lanes[r * 32 + l] = w_N^{2 m_r l step}, lanes[kLaneRows * 32 + k]
// = w_N^{step k}.  Radix 128: lanes[r * 32 + l] = w_N^{m_r l step}.  FP64,
// rounded once.
__global__ void fb_lane_table_kernel(float2* lanes, long long n, long long step, int radix) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  long long m;
  if (radix == 128) {
    if (e >= kLaneRows128 * 32) return;
    m = (long long)lane_row_m128(e / 32) * (e % 32) * step;
  } else {
    if (e >= kLaneRows * 32 + 64) return;
    m = e < kLaneRows * 32 ? (long long)lane_row_m(e / 32) * 2 * (e % 32) * step
                           : (long long)(e - kLaneRows * 32) * step;
  }
  double sn, cs;
  sincospi(2.0 * (double)(m % n) / (double)n, &sn, &cs);
  lanes[e] = make_float2((float)cs, (float)(-sn));
}

template <bool FIRST>
__global__ void __launch_bounds__(kTileThreads, 4)
outer64_fwd_kernel(float2* __restrict__ w, const float* __restrict__ ts, long long n, int ls,
                   const float2* __restrict__ thi, const float2* __restrict__ tlo,
                   const float2* __restrict__ lanes) {
  __shared__ float4 tile[64][kTileCols / 2];
  const long long s = 1LL << ls;
  const int c = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const long long b = (long long)blockIdx.x * kTileCols + 2 * c;    // butterflies b, b + 1
  const long long t = b & (s - 1);
  const long long base = ((b >> ls) << (ls + 6)) + t;
  const int k1 = wp;
  float2 twu[8], twv[8];
  {
    const int j2 = wp;
    float2 u[8], v[8];
#pragma unroll
    for (int j1 = 0; j1 < 8; ++j1) {
      const long long at = base + s * (8 * j1 + j2);
      if constexpr (FIRST) {
        const float2 r = __ldg(reinterpret_cast<const float2*>(ts + at));
        u[j1] = make_float2(r.x, 0.f);
        v[j1] = make_float2(r.y, 0.f);
      } else {
        const float4 r = *reinterpret_cast<const float4*>(w + at);
        u[j1] = make_float2(r.x, r.y);
        v[j1] = make_float2(r.z, r.w);
      }
    }
    {
      // the second stage's outer twiddles while the loads are in flight
      // (w_M^{t k} = w_N^{t k N/M}; the tile's first column t0 = t - 2*lane)
      const Tw8x2 tw(thi, tlo, lanes, t - 2 * c, n >> (ls + 6), k1, c);
#pragma unroll
      for (int k2 = 0; k2 < 8; ++k2) {
        twu[k2] = tw.u[k2];
        twv[k2] = tw.v[k2];
      }
    }
    dft<8, -1>(u);
    dft<8, -1>(v);
    tile[j2][c] = pack2(u[0], v[0]);
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) {
      const float2 wk = w64(thi, n, j2 * k1);
      tile[8 * k1 + j2][c] = pack2(cmul(u[k1], wk), cmul(v[k1], wk));
    }
  }
  __syncthreads();
  float2 u[8], v[8];
#pragma unroll
  for (int j2 = 0; j2 < 8; ++j2) {
    const float4 r = tile[8 * k1 + j2][c];
    u[j2] = make_float2(r.x, r.y);
    v[j2] = make_float2(r.z, r.w);
  }
  dft<8, -1>(u);                               // u[k2] = X[k1 + 8 k2] of butterfly b
  dft<8, -1>(v);                               // ... of butterfly b + 1
#pragma unroll
  for (int k2 = 0; k2 < 8; ++k2) {
    u[k2] = cmul(u[k2], twu[k2]);
    v[k2] = cmul(v[k2], twv[k2]);
  }
#pragma unroll
  for (int k2 = 0; k2 < 8; ++k2) *reinterpret_cast<float4*>(w + base + s * (k1 + 8 * k2)) = pack2(u[k2], v[k2]);
}

// Inverse: y[8 j1 + j2] = sum_k1 w_8^{-j1 k1} w_64^{-j2 k1} sum_k2 w_8^{-j2 k2} V[k1 + 8 k2],
// V[k] = W[k] conj(w_N^{e1 k}).  LAST (stride N/64, consecutive butterflies
// are consecutive samples): NA = 0 writes Re(y)^2 to pw; NA > 0 sums windows
// of NA neighbouring columns of Re(y)^2 across lanes and writes those of the
// kept part (window m starts at n_ov + m*NA) to out.
template <bool LAST, int NA>
__global__ void __launch_bounds__(kTileThreads, 4)
outer64_inv_kernel(float2* __restrict__ w, float* __restrict__ pw, long long n, int ls,
                   const float2* __restrict__ thi, const float2* __restrict__ tlo,
                   const float2* __restrict__ lanes, float* __restrict__ out, long long n_ov) {
  static_assert(NA == 0 || (LAST && NA <= 32 && (NA & (NA - 1)) == 0), "column windows");
  __shared__ float4 tile[64][kTileCols / 2];
  const long long s = 1LL << ls;
  const int c = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const long long b = (long long)blockIdx.x * kTileCols + 2 * c;
  const long long t = b & (s - 1);
  const long long base = ((b >> ls) << (ls + 6)) + t;
  {
    const int k1 = wp;
    float2 u[8], v[8];
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
      const float4 r = *reinterpret_cast<const float4*>(w + base + s * (k1 + 8 * k2));
      u[k2] = make_float2(r.x, r.y);
      v[k2] = make_float2(r.z, r.w);
    }
    {
      const Tw8x2 tw(thi, tlo, lanes, t - 2 * c, n >> (ls + 6), k1, c);
#pragma unroll
      for (int k2 = 0; k2 < 8; ++k2) {
        u[k2] = cmulc(u[k2], tw.u[k2]);
        v[k2] = cmulc(v[k2], tw.v[k2]);
      }
    }
    dft<8, 1>(u);                              // u[j2] = Z_k1[j2]
    dft<8, 1>(v);
    tile[k1][c] = pack2(u[0], v[0]);
#pragma unroll
    for (int j2 = 1; j2 < 8; ++j2) {
      const float2 wk = w64(thi, n, j2 * k1);
      tile[8 * j2 + k1][c] = pack2(cmulc(u[j2], wk), cmulc(v[j2], wk));
    }
  }
  __syncthreads();
  const int j2 = wp;
  float2 u[8], v[8];
#pragma unroll
  for (int k1 = 0; k1 < 8; ++k1) {
    const float4 r = tile[8 * j2 + k1][c];
    u[k1] = make_float2(r.x, r.y);
    v[k1] = make_float2(r.z, r.w);
  }
  dft<8, 1>(u);                                // u[j1] = y[8 j1 + j2] of butterfly b
  dft<8, 1>(v);                                // ... of butterfly b + 1
  if constexpr (!LAST) {
#pragma unroll
    for (int j1 = 0; j1 < 8; ++j1) *reinterpret_cast<float4*>(w + base + s * (8 * j1 + j2)) = pack2(u[j1], v[j1]);
  } else if constexpr (NA == 0) {
#pragma unroll
    for (int j1 = 0; j1 < 8; ++j1)
      *reinterpret_cast<float2*>(pw + base + s * (8 * j1 + j2)) = make_float2(u[j1].x * u[j1].x, v[j1].x * v[j1].x);
  } else if constexpr (NA == 1) {
#pragma unroll
    for (int j1 = 0; j1 < 8; ++j1) {
      const long long n0 = base + s * (8 * j1 + j2);
      if (n0 >= n_ov) out[n0 - n_ov] = u[j1].x * u[j1].x;
      if (n0 + 1 >= n_ov) out[n0 + 1 - n_ov] = v[j1].x * v[j1].x;
    }
  } else {
    // a lane holds samples (2c, 2c + 1) of each row: windows of NA samples
    // are NA/2 neighbouring lanes of pair sums
    constexpr int NH = NA / 2;
    float p[8];
#pragma unroll
    for (int j1 = 0; j1 < 8; ++j1) p[j1] = u[j1].x * u[j1].x + v[j1].x * v[j1].x;
    const long long t0 = (long long)blockIdx.x * kTileCols;    // sample of column 0 in row 0
    if constexpr (NH <= 8) {
      lane_window_sums<8, NH>(p, c);
      constexpr int V = 8 / NH;
      const int lo = c & (NH - 1);
#pragma unroll
      for (int i = 0; i < V; ++i) {
        const long long n0 = t0 + 2 * (c - lo) + s * (8 * (V * lo + i) + j2);
        if (n0 >= n_ov) out[(n0 - n_ov) / NA] = p[i];
      }
    } else {
      lane_window_sums<8, 8>(p, c);            // p[0]: 8 lanes of row 8*(c & 7) + j2
#pragma unroll
      for (int o = 8; o < NH; o <<= 1) p[0] += __shfl_xor_sync(0xffffffffu, p[0], o);
      if ((c & (NH - 1)) < 8) {
        const long long n0 = t0 + 2 * (c & ~(NH - 1)) + s * (8 * (c & 7) + j2);
        if (n0 >= n_ov) out[(n0 - n_ov) / NA] = p[0];
      }
    }
  }
}

// ---- outer radix-128 passes, as 16 x 8 through shared memory --------------
// As the radix-64 tiles, with j = 8*j1 + j2 (j1 < 16) and k = k1 + 16*k2:
//   X[k1 + 16 k2] = sum_j2 w_8^{j2 k2} w_128^{j2 k1} sum_j1 w_16^{j1 k1} v[8 j1 + j2].
// A CTA takes 32 neighbouring butterflies, one column per lane (256-byte row
// pieces): warp j2 does the radix-16 over j1, and each warp then does the
// radix-8 over j2 for k1 = warp and warp + 8.  The tile is 128 rows of 32.
// w_128^m = w_N^{m N/128} is one entry of the high table (N >= 2^20).
constexpr int kTile128Cols = 32;

__device__ __forceinline__ float2 w128(const float2* __restrict__ thi, long long n, int m) {
  return __ldg(&thi[(long long)(m & 127) * (n >> 20)]);
}

// w_N^{e1 k} for a lane's column t = t0 + lane (e1 = t*step) and rows
// k = k1 + 16*k2, k2 < 8: w_N^{e1 k1} times the powers of w_N^{16 e1}, each
// w_N^{m t step} being the warp's w_N^{m t0 step} times the lane-table entry
struct Tw16x8 {
  float2 u[8];
  __device__ __forceinline__ Tw16x8(const float2* __restrict__ thi, const float2* __restrict__ tlo,
                                    const float2* __restrict__ lanes, long long t0, long long step, int k1,
                                    int lane) {
    auto wt = [&](int r) {
      return cmul(twiddle(thi, tlo, (long long)lane_row_m128(r) * t0 * step), __ldg(&lanes[r * 32 + lane]));
    };
    float2 q[8];                                   // q[k2] = w_N^{16 e1 k2}
    q[1] = wt(15);
    q[2] = wt(16);
    q[4] = wt(17);
    q[3] = cmul(q[2], q[1]);
    q[5] = cmul(q[4], q[1]);
    q[6] = cmul(q[4], q[2]);
    q[7] = cmul(q[4], q[3]);
    const float2 a = k1 == 0 ? make_float2(1.f, 0.f) : wt(k1 - 1);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) u[k2] = k2 == 0 ? a : cmul(a, q[k2]);
  }
};

template <bool FIRST>
__global__ void __launch_bounds__(kTileThreads, 4)
outer128_fwd_kernel(float2* __restrict__ w, const float* __restrict__ ts, long long n, int ls,
                    const float2* __restrict__ thi, const float2* __restrict__ tlo,
                    const float2* __restrict__ lanes) {
  __shared__ float2 tile[128][kTile128Cols];
  const long long s = 1LL << ls;
  const int c = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const long long b = (long long)blockIdx.x * kTile128Cols + c;
  const long long t = b & (s - 1);
  const long long base = ((b >> ls) << (ls + 7)) + t;
  {
    const int j2 = wp;
    float2 v[16];
#pragma unroll
    for (int j1 = 0; j1 < 16; ++j1) {
      const long long at = base + s * (8 * j1 + j2);
      v[j1] = FIRST ? make_float2(__ldg(&ts[at]), 0.f) : w[at];
    }
    dft<16, -1>(v);
    tile[j2][c] = v[0];
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) tile[8 * k1 + j2][c] = cmul(v[k1], w128(thi, n, j2 * k1));
  }
  __syncthreads();
  const long long step = n >> (ls + 7);        // w_M^{t k} = w_N^{t k N/M}
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    const int k1 = wp + 8 * h;
    float2 v[8];
#pragma unroll
    for (int j2 = 0; j2 < 8; ++j2) v[j2] = tile[8 * k1 + j2][c];
    dft<8, -1>(v);                             // v[k2] = X[k1 + 16 k2]
    const Tw16x8 tw(thi, tlo, lanes, t - c, step, k1, c);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) w[base + s * (k1 + 16 * k2)] = cmul(v[k2], tw.u[k2]);
  }
}

// Inverse: y[8 j1 + j2] = sum_k1 w_16^{-j1 k1} w_128^{-j2 k1} sum_k2 w_8^{-j2 k2} V[k1 + 16 k2],
// V[k] = W[k] conj(w_N^{e1 k}); LAST and NA as for the radix-64 tiles.
template <bool LAST, int NA>
__global__ void __launch_bounds__(kTileThreads, 4)
outer128_inv_kernel(float2* __restrict__ w, float* __restrict__ pw, long long n, int ls,
                    const float2* __restrict__ thi, const float2* __restrict__ tlo,
                    const float2* __restrict__ lanes, float* __restrict__ out, long long n_ov) {
  static_assert(NA == 0 || (LAST && NA <= 32 && (NA & (NA - 1)) == 0), "column windows");
  __shared__ float2 tile[128][kTile128Cols];
  const long long s = 1LL << ls;
  const int c = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const long long b = (long long)blockIdx.x * kTile128Cols + c;
  const long long t = b & (s - 1);
  const long long base = ((b >> ls) << (ls + 7)) + t;
  const long long step = n >> (ls + 7);
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    const int k1 = wp + 8 * h;
    float2 v[8];
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) v[k2] = w[base + s * (k1 + 16 * k2)];
    const Tw16x8 tw(thi, tlo, lanes, t - c, step, k1, c);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) v[k2] = cmulc(v[k2], tw.u[k2]);
    dft<8, 1>(v);                              // v[j2] = Z_k1[j2]
    tile[8 * k1][c] = v[0];
#pragma unroll
    for (int j2 = 1; j2 < 8; ++j2) tile[8 * k1 + j2][c] = cmulc(v[j2], w128(thi, n, j2 * k1));
  }
  __syncthreads();
  const int j2 = wp;
  float2 v[16];
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) v[k1] = tile[8 * k1 + j2][c];
  dft<16, 1>(v);                               // v[j1] = y[8 j1 + j2]
  if constexpr (!LAST) {
#pragma unroll
    for (int j1 = 0; j1 < 16; ++j1) w[base + s * (8 * j1 + j2)] = v[j1];
  } else if constexpr (NA == 0) {
#pragma unroll
    for (int j1 = 0; j1 < 16; ++j1) pw[base + s * (8 * j1 + j2)] = v[j1].x * v[j1].x;
  } else {
    // windows of NA neighbouring columns are NA neighbouring lanes
    float u[16];
#pragma unroll
    for (int j1 = 0; j1 < 16; ++j1) u[j1] = v[j1].x * v[j1].x;
    const long long t0 = (long long)blockIdx.x * kTile128Cols;   // sample of column 0 in row 0
    if constexpr (NA <= 16) {
      lane_window_sums<16, NA>(u, c);
      constexpr int V = 16 / NA;
      const int lo = c & (NA - 1);
#pragma unroll
      for (int i = 0; i < V; ++i) {
        const long long n0 = t0 + (c - lo) + s * (8 * (V * lo + i) + j2);
        if (n0 >= n_ov) out[(n0 - n_ov) / NA] = u[i];
      }
    } else {
      lane_window_sums<16, 16>(u, c);          // u[0]: 16 lanes of row 8*(c & 15) + j2
      u[0] += __shfl_xor_sync(0xffffffffu, u[0], 16);
      if (c < 16) {
        const long long n0 = t0 + s * (8 * c + j2);
        if (n0 >= n_ov) out[(n0 - n_ov) / NA] = u[0];
      }
    }
  }
}

// ---- middle: contiguous sub-transforms of 2^LOGS points in shared memory --
// Sub-transform qq holds bins bin_out(qq) + L_out * (its own bins); chirp is the
// per-bin table in the chirp pass's order.  ts != nullptr: the series is real
// and there are no outer passes (N = 2^LOGS); pw != nullptr: write Re(y)^2.
template <int LOGS>
__global__ void __launch_bounds__(Cfg<LOGS>::THREADS, 1)
middle_kernel(float2* __restrict__ w, const float* __restrict__ ts, float* __restrict__ pw,
              const float2* __restrict__ chirp, const float2* __restrict__ tw, long long n_sub) {
  using PL = PassPlan<LOGS>;
  using CF = Cfg<LOGS>;
  constexpr int NS = PL::N;
  extern __shared__ __align__(16) float2 smem[];
  const int g = threadIdx.x / PL::T;
  const int lt = threadIdx.x % PL::T;
  float2* buf = smem + g * CF::SEG_F2;
  const long long qq = (long long)blockIdx.x * CF::G + g;
  const bool active = qq < n_sub;
  float2* wq = w + qq * NS;
  // with two pad words a pair of points (2m, 2m + 1) is 16-byte aligned in
  // shared memory as in global memory: the working transform then moves as
  // 128-bit accesses, half as many
  constexpr bool kPairs = pad_words<LOGS>() == 2;
  if (active && (!kPairs || ts)) {          // every load in flight before the first store
    constexpr int PER = NS / PL::T;
    float2 r[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i)
      r[i] = ts ? make_float2(__ldg(&ts[qq * NS + lt + i * PL::T]), 0.f) : wq[lt + i * PL::T];
#pragma unroll
    for (int i = 0; i < PER; ++i) buf[pad<LOGS>(lt + i * PL::T)] = r[i];
  } else if (active) {
    constexpr int PER2 = NS / (2 * PL::T);
    float4 r[PER2];
#pragma unroll
    for (int i = 0; i < PER2; ++i) r[i] = reinterpret_cast<const float4*>(wq)[lt + i * PL::T];
#pragma unroll
    for (int i = 0; i < PER2; ++i)
      *reinterpret_cast<float4*>(&buf[pad<LOGS>(2 * (lt + i * PL::T))]) = r[i];
  }
  __syncthreads();
  static_for<0, PL::P - 1>([&](auto P_) {
    constexpr int pp = decltype(P_)::value;
    if (active) fwd_pass<LOGS, pp, false, pp == 0 && kRecPass0<LOGS, false>>(buf, tw, lt);
    __syncthreads();
  });
  if (active) chirp_pass<LOGS>(buf, chirp + qq * NS, lt);
  __syncthreads();
  static_for<0, PL::P - 1>([&](auto I_) {
    constexpr int pp = PL::P - 2 - decltype(I_)::value;
    if (active) inv_pass<LOGS, pp, false, pp == 0 && kRecPass0<LOGS, false>>(buf, tw, lt);
    __syncthreads();
  });
  if (active && (!kPairs || pw)) {
    for (int i = lt; i < NS; i += PL::T) {
      const float2 v = buf[pad<LOGS>(i)];
      if (pw) pw[qq * NS + i] = v.x * v.x;
      else wq[i] = v;
    }
  } else if (active) {
    for (int m = lt; m < NS / 2; m += PL::T)
      reinterpret_cast<float4*>(wq)[m] = *reinterpret_cast<const float4*>(&buf[pad<LOGS>(2 * m)]);
  }
}

// out[m] = sum of n_avg samples of pw from n_ov on (the kept part of a segment)
__global__ void fb_integrate_kernel(const float* __restrict__ pw, float* __restrict__ out,
                                    long long n_ov, int n_avg, long long n_out) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < n_out;
       m += (long long)gridDim.x * blockDim.x) {
    const float* p = pw + n_ov + m * n_avg;
    float acc = 0.f;
    for (int i = 0; i < n_avg; ++i) acc += __ldg(&p[i]);
    out[m] = acc;
  }
}

// ---- plan-time tables (FP64) ----------------------------------------------
__global__ void fb_twiddle_kernel(float2* hi, float2* lo, long long n) {
  const long long n_hi = n >> kTwLoBits;
  const long long total = n_hi + (1 << kTwLoBits);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long m = e < n_hi ? (e << kTwLoBits) : e - n_hi;
    double sn, cs;
    sincospi(2.0 * (double)m / (double)n, &sn, &cs);
    const float2 v = make_float2((float)cs, (float)(-sn));
    if (e < n_hi) hi[e] = v;
    else lo[e - n_hi] = v;
  }
}

// chirp[qq * NS + idx] for the bin held there: Hermitian (bins above N/2 take
// the conjugate of their mirror) so the inverse transform stays real.  A
// lower-sideband series (sideband < 0) is the band inverted: bin j sits
// B - j fs / N above the lower edge and takes the conjugate correction.
template <int LOGS>
__global__ void fb_chirp_kernel(float2* chirp, long long n, int n_outer, const int* radix_out,
                                const long long* stride_out, const long long* rprod_out,
                                double f_lo, double fs, double dm, int sideband) {
  using PL = PassPlan<LOGS>;
  constexpr int NS = PL::N;
  constexpr int NG = NS / PL::RL;
  const long long l_out = n / NS;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long qq = e / NS;
    const int idx = (int)(e % NS);
    long long b_out = 0;
    for (int p = 0; p < n_outer; ++p) {
      const long long d = (qq / (stride_out[p] / NS)) % radix_out[p];
      b_out += d * rprod_out[p];
    }
    const int pos = passes::chirp_pos<NG>(idx, PL::RL);
    const long long bin = b_out + l_out * position_to_bin<LOGS>(pos);
    const long long mb = bin <= n / 2 ? bin : n - bin;     // mirror for the upper half
    const double f_bb = (double)mb * (fs / (double)n);
    const double f_l = sideband > 0 ? f_bb : 0.5 * fs - f_bb;
    const double turns = kDispD * 1e6 * dm * f_l * f_l / ((f_l + f_lo) * f_lo * f_lo);
    const double frac = turns - rint(turns);
    double sn, cs;
    sincospi(2.0 * frac, &sn, &cs);
    const double sc = 1.0 / (double)n;
    // exp(-i Phi) / N below N/2 (and at it), the conjugate above; both
    // conjugated for a lower sideband
    const double s_im = (bin <= n / 2 ? -sn : sn) * (sideband > 0 ? 1.0 : -1.0);
    chirp[e] = make_float2((float)(cs * sc), (float)(s_im * sc));
  }
}

unsigned grid_for(long long work, int block = 256) {
  long long g = (work + block - 1) / block;
  if (g > 148LL * 32) g = 148LL * 32;
  return (unsigned)(g > 0 ? g : 1);
}

template <int LOGF>
cudaError_t launch_icf_t(const char2* in, float* ts, const float2* twf, long long n_frames, int n_chan,
                         cudaStream_t s) {
  using CF = Cfg<LOGF>;
  static bool set[128] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 128 && !set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(icf_kernel<LOGF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CF::SMEM);
    if (e != cudaSuccess) return e;
    set[dev] = true;
  }
  icf_kernel<LOGF><<<(unsigned)((n_frames + CF::G - 1) / CF::G), CF::THREADS, CF::SMEM, s>>>(in, ts, twf, n_frames, n_chan);
  return cudaGetLastError();
}

template <int LOGC>
cudaError_t launch_icf_half_t(const char2* in, float* ts, const float2* twc, const float2* wk,
                              long long n_frames, cudaStream_t s) {
  using CF = Cfg<LOGC>;
  static bool set[128] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 128 && !set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(icf_half_kernel<LOGC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)CF::SMEM);
    if (e != cudaSuccess) return e;
    set[dev] = true;
  }
  icf_half_kernel<LOGC><<<(unsigned)((n_frames + CF::G - 1) / CF::G), CF::THREADS, CF::SMEM, s>>>(
      in, ts, twc, wk, n_frames);
  return cudaGetLastError();
}

template <int LOGS>
cudaError_t launch_middle_t(float2* w, const float* ts, float* pw, const float2* chirp,
                            const float2* tw, long long n_sub, cudaStream_t s) {
  using CF = Cfg<LOGS>;
  static bool set[128] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 128 && !set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(middle_kernel<LOGS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CF::SMEM);
    if (e != cudaSuccess) return e;
    set[dev] = true;
  }
  middle_kernel<LOGS><<<(unsigned)((n_sub + CF::G - 1) / CF::G), CF::THREADS, CF::SMEM, s>>>(w, ts, pw, chirp, tw, n_sub);
  return cudaGetLastError();
}

#define CDD_FB_CASES(X) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14)

// Frames of 2C >= 128 samples take the half-length form (twf: the C-point
// table, wk: e^{+2 pi i k/2C}); 64-sample frames the direct form (twf: the
// 64-point table).
cudaError_t launch_icf(int logf, const char2* in, float* ts, const float2* twf, const float2* wk,
                       long long n_frames, int n_chan, cudaStream_t s) {
  switch (logf) {
    case 6: return launch_icf_t<6>(in, ts, twf, n_frames, n_chan, s);
#define X(L) case L + 1: return launch_icf_half_t<L>(in, ts, twf, wk, n_frames, s);
    X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

int icf_table_logn(int logf) { return logf > 6 ? logf - 1 : logf; }

cudaError_t launch_middle(int logs, float2* w, const float* ts, float* pw, const float2* chirp,
                          const float2* tw, long long n_sub, cudaStream_t s) {
  switch (logs) {
#define X(L) case L: return launch_middle_t<L>(w, ts, pw, chirp, tw, n_sub, s);
    CDD_FB_CASES(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_outer(bool forward, bool edge, int radix, float2* w, const float* ts, float* pw,
                         long long n, long long stride, const float2* thi, const float2* tlo,
                         const float2* lanes, cudaStream_t s, float* out = nullptr, long long n_ov = 0,
                         int na = 0) {
  if (stride <= 0 || (stride & (stride - 1)) || n % (stride * radix)) return cudaErrorInvalidValue;
  int ls = 0;
  while ((1LL << ls) < stride) ++ls;
  if (radix == 128) {                         // tiles of kTile128Cols butterflies
    if (stride % kTile128Cols || n < (1LL << 20) || lanes == nullptr) return cudaErrorInvalidValue;
    const long long tiles = n / 128 / kTile128Cols;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    const unsigned g = (unsigned)tiles;
    if (forward && edge) outer128_fwd_kernel<true><<<g, kTileThreads, 0, s>>>(w, ts, n, ls, thi, tlo, lanes);
    else if (forward) outer128_fwd_kernel<false><<<g, kTileThreads, 0, s>>>(w, ts, n, ls, thi, tlo, lanes);
    else if (!edge)
      outer128_inv_kernel<false, 0><<<g, kTileThreads, 0, s>>>(w, pw, n, ls, thi, tlo, lanes, nullptr, 0);
    else {
      switch (na) {
#define CDD_OUTER128_NA(A) \
        case A: outer128_inv_kernel<true, A><<<g, kTileThreads, 0, s>>>(w, pw, n, ls, thi, tlo, lanes, out, n_ov); break;
        CDD_OUTER128_NA(0) CDD_OUTER128_NA(1) CDD_OUTER128_NA(2) CDD_OUTER128_NA(4) CDD_OUTER128_NA(8)
        CDD_OUTER128_NA(16) CDD_OUTER128_NA(32)
#undef CDD_OUTER128_NA
        default: return cudaErrorInvalidValue;
      }
    }
    return cudaGetLastError();
  }
  if (radix == 64) {                          // tiles of kTileCols butterflies
    if (stride % kTileCols || n < (1LL << 19) || lanes == nullptr) return cudaErrorInvalidValue;
    const long long tiles = n / 64 / kTileCols;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    const unsigned g = (unsigned)tiles;
    if (forward && edge) outer64_fwd_kernel<true><<<g, kTileThreads, 0, s>>>(w, ts, n, ls, thi, tlo, lanes);
    else if (forward) outer64_fwd_kernel<false><<<g, kTileThreads, 0, s>>>(w, ts, n, ls, thi, tlo, lanes);
    else if (!edge)
      outer64_inv_kernel<false, 0><<<g, kTileThreads, 0, s>>>(w, pw, n, ls, thi, tlo, lanes, nullptr, 0);
    else {
      switch (na) {
#define CDD_OUTER64_NA(A) \
        case A: outer64_inv_kernel<true, A><<<g, kTileThreads, 0, s>>>(w, pw, n, ls, thi, tlo, lanes, out, n_ov); break;
        CDD_OUTER64_NA(0) CDD_OUTER64_NA(1) CDD_OUTER64_NA(2) CDD_OUTER64_NA(4) CDD_OUTER64_NA(8)
        CDD_OUTER64_NA(16) CDD_OUTER64_NA(32)
#undef CDD_OUTER64_NA
        default: return cudaErrorInvalidValue;
      }
    }
    return cudaGetLastError();
  }
  const unsigned grid = grid_for(n / radix);
  if (!forward && edge && na > 0) {           // last pass with the integration fused
    if (radix != 16 || (n / radix) % 32) return cudaErrorInvalidValue;
    switch (na) {
#define CDD_OUTER_NA(A) \
      case A: outer_inv_kernel<16, true, A><<<grid, 256, 0, s>>>(w, pw, n, ls, thi, tlo, out, n_ov); break;
      CDD_OUTER_NA(1) CDD_OUTER_NA(2) CDD_OUTER_NA(4) CDD_OUTER_NA(8) CDD_OUTER_NA(16)
#undef CDD_OUTER_NA
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
#define CDD_OUTER(R)                                                                                  \
  case R:                                                                                             \
    if (forward && edge) outer_fwd_kernel<R, true><<<grid, 256, 0, s>>>(w, ts, n, ls, thi, tlo);             \
    else if (forward) outer_fwd_kernel<R, false><<<grid, 256, 0, s>>>(w, ts, n, ls, thi, tlo);               \
    else if (edge) outer_inv_kernel<R, true><<<grid, 256, 0, s>>>(w, pw, n, ls, thi, tlo, nullptr, 0);       \
    else outer_inv_kernel<R, false><<<grid, 256, 0, s>>>(w, pw, n, ls, thi, tlo, nullptr, 0);                \
    break;
  switch (radix) {
    CDD_OUTER(2) CDD_OUTER(4) CDD_OUTER(8) CDD_OUTER(16)
    default: return cudaErrorInvalidValue;
  }
#undef CDD_OUTER
  return cudaGetLastError();
}

cudaError_t launch_fb_chirp(int logs, float2* chirp, long long n, int n_outer, const int* radix,
                            const long long* stride, const long long* rprod, double f_lo, double fs,
                            double dm, int sideband, cudaStream_t s) {
  const unsigned grid = grid_for(n);
  switch (logs) {
#define X(L) case L: fb_chirp_kernel<L><<<grid, 256, 0, s>>>(chirp, n, n_outer, radix, stride, rprod, f_lo, fs, dm, sideband); break;
    CDD_FB_CASES(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace
}  // namespace cdd

// ------------------------------------------------------------------ host side

struct cdd_fullband_s {
  double f_center = 0, bandwidth = 0, dm = 0, f_lo = 0, fs = 0, n_disp = 0;
  int sideband = 1;                          // -1: lower sideband, the series is the band inverted
  int n_chan = 0, frame = 0, logf = 0, n_avg = 0;
  long long n_fft = 0, n_ov = 0, hop = 0;
  int logs = 0;                              // log2 L_mid
  std::vector<int> radix_out;                // outer DIF radices, pass 0 first
  std::vector<long long> stride_out, rprod_out;
  int q = 1;
  bool committed = false;
  int device = -1;
  int sticky = CDD_OK;
  float* d_ts[2] = {nullptr, nullptr};       // [n_ov + q*h] real series, ping-pong
  float2* d_w = nullptr;                     // [N] work
  float* d_pw = nullptr;                     // [N] detected power of a segment
  float2* d_chirp = nullptr;                 // [N]
  float2* d_tw = nullptr;                    // twiddles of the L_mid passes
  float2* d_twf = nullptr;                   // twiddles of the frame transform
  float2* d_wk = nullptr;                    // e^{+2 pi i k/2C}, k < C (half-length frame form)
  float2* d_thi = nullptr;
  float2* d_tlo = nullptr;
  int* d_radix = nullptr;
  long long* d_stride = nullptr;
  long long* d_rprod = nullptr;
  float2* d_lanes = nullptr;                 // [outer passes][kLaneTable] lane tables of the tile passes
  int cur = 0;
  int64_t blocks = 0;
  size_t bytes_device = 0;
  int last_launches = 0;
};

namespace {

int ffail(cdd_fullband f, cudaError_t e) {
  if (e == cudaSuccess) return CDD_OK;
  f->sticky = CDD_ECUDA;
  return CDD_ECUDA;
}

#define FTRY(f, call)                              \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return ffail(f, e_);    \
  } while (0)

template <class T>
int falloc(cdd_fullband f, T** p, size_t bytes) {
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    *p = nullptr;
    return CDD_ENOMEM;
  }
  if (e != cudaSuccess) return ffail(f, e);
  f->bytes_device += bytes;
  return CDD_OK;
}

long long ts_len(const cdd_fullband f) { return f->n_ov + (long long)f->q * f->hop; }

int fcommit_once(cdd_fullband f) {
  FTRY(f, cudaGetDevice(&f->device));
  const long long n = f->n_fft;
  int rc;
  for (int i = 0; i < 2; ++i)
    if ((rc = falloc(f, &f->d_ts[i], (size_t)ts_len(f) * sizeof(float)))) return rc;
  if ((rc = falloc(f, &f->d_w, (size_t)n * sizeof(float2)))) return rc;
  if ((rc = falloc(f, &f->d_pw, (size_t)n * sizeof(float)))) return rc;
  if ((rc = falloc(f, &f->d_chirp, (size_t)n * sizeof(float2)))) return rc;
  if ((rc = falloc(f, &f->d_tw, (size_t)cdd::twiddle_table_len(f->logs) * sizeof(float2)))) return rc;
  if ((rc = falloc(f, &f->d_twf, (size_t)cdd::twiddle_table_len(cdd::icf_table_logn(f->logf)) * sizeof(float2))))
    return rc;
  if ((rc = falloc(f, &f->d_wk, (size_t)f->n_chan * sizeof(float2)))) return rc;
  const long long n_hi = n >> cdd::kTwLoBits;
  if (!f->radix_out.empty()) {
    if ((rc = falloc(f, &f->d_thi, (size_t)(n_hi > 0 ? n_hi : 1) * sizeof(float2)))) return rc;
    if ((rc = falloc(f, &f->d_tlo, (size_t)(1 << cdd::kTwLoBits) * sizeof(float2)))) return rc;
  }
  const size_t no = f->radix_out.size() > 0 ? f->radix_out.size() : 1;
  if ((rc = falloc(f, &f->d_radix, no * sizeof(int)))) return rc;
  if ((rc = falloc(f, &f->d_stride, no * sizeof(long long)))) return rc;
  if ((rc = falloc(f, &f->d_rprod, no * sizeof(long long)))) return rc;
  if ((rc = falloc(f, &f->d_lanes, no * cdd::kLaneTable * sizeof(float2)))) return rc;
  if (!f->radix_out.empty()) {
    FTRY(f, cudaMemcpy(f->d_radix, f->radix_out.data(), no * sizeof(int), cudaMemcpyHostToDevice));
    FTRY(f, cudaMemcpy(f->d_stride, f->stride_out.data(), no * sizeof(long long), cudaMemcpyHostToDevice));
    FTRY(f, cudaMemcpy(f->d_rprod, f->rprod_out.data(), no * sizeof(long long), cudaMemcpyHostToDevice));
  }
  cudaStream_t s;
  FTRY(f, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaError_t e = cdd::launch_twiddle_table(f->logs, f->d_tw, s);
  if (e == cudaSuccess) e = cdd::launch_twiddle_table(cdd::icf_table_logn(f->logf), f->d_twf, s);
  if (e == cudaSuccess) {
    cdd::fb_wk_kernel<<<cdd::grid_for(f->n_chan), 256, 0, s>>>(f->d_wk, f->n_chan);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && f->d_thi) {
    cdd::fb_twiddle_kernel<<<cdd::grid_for(n_hi + (1 << cdd::kTwLoBits)), 256, 0, s>>>(f->d_thi, f->d_tlo, n);
    e = cudaGetLastError();
  }
  for (size_t p = 0; p < f->radix_out.size() && e == cudaSuccess; ++p)
    if (f->radix_out[p] >= 64) {
      // the pass of stride S works on sub-problems of M = R S: step = N / M
      const long long step = n / (f->radix_out[p] * f->stride_out[p]);
      cdd::fb_lane_table_kernel<<<(cdd::kLaneTable + 127) / 128, 128, 0, s>>>(
          f->d_lanes + p * cdd::kLaneTable, n, step, f->radix_out[p]);
      e = cudaGetLastError();
    }
  if (e == cudaSuccess)
    e = cdd::launch_fb_chirp(f->logs, f->d_chirp, n, (int)f->radix_out.size(), f->d_radix, f->d_stride,
                             f->d_rprod, f->f_lo, f->fs, f->dm, f->sideband, s);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i)
    e = cudaMemsetAsync(f->d_ts[i], 0, (size_t)ts_len(f) * sizeof(float), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (e != cudaSuccess) return ffail(f, e);
  f->committed = true;
  return CDD_OK;
}

int fprepare(cdd_fullband f) {
  if (!f) return CDD_EINVAL;
  if (f->sticky) return f->sticky;
  if (!f->committed) {
    const int rc = fcommit_once(f);
    if (rc != CDD_OK) {
      f->sticky = rc;
      return rc;
    }
  }
  int dev = -1;
  FTRY(f, cudaGetDevice(&dev));
  return dev == f->device ? CDD_OK : CDD_EINVAL;
}

void ffree(cdd_fullband f) {
  cudaFree(f->d_ts[0]);
  cudaFree(f->d_ts[1]);
  cudaFree(f->d_w);
  cudaFree(f->d_pw);
  cudaFree(f->d_chirp);
  cudaFree(f->d_tw);
  cudaFree(f->d_twf);
  cudaFree(f->d_wk);
  cudaFree(f->d_thi);
  cudaFree(f->d_tlo);
  cudaFree(f->d_radix);
  cudaFree(f->d_stride);
  cudaFree(f->d_rprod);
  cudaFree(f->d_lanes);
}

long long next_pow2_above_ll(double x) {
  long long n = 1;
  while ((double)n <= x && n < (1LL << 40)) n *= 2;
  return n;
}

}  // namespace

extern "C" {

int cdd_fullband_create(cdd_fullband* out, double f_center_mhz, double bandwidth_mhz, int n_chan,
                        double dm, long long n_fft, int n_avg) {
  if (!out) return CDD_EINVAL;
  *out = nullptr;
  if (!(f_center_mhz > 0) || !isfinite(bandwidth_mhz) || bandwidth_mhz == 0 || n_chan <= 0 || !(dm >= 0) ||
      !isfinite(dm) || n_avg <= 0 || n_fft < 0)
    return CDD_EINVAL;
  const int sideband = bandwidth_mhz > 0 ? 1 : -1;
  bandwidth_mhz = fabs(bandwidth_mhz);
  const int frame = 2 * n_chan;
  if ((frame & (frame - 1)) || (n_avg & (n_avg - 1))) return CDD_EINVAL;
  int logf = 0;
  while ((1 << logf) < frame) ++logf;
  if (logf < 6 || logf > 14) return CDD_EUNSUPPORTED;
  cdd_fullband f = new (std::nothrow) cdd_fullband_s();
  if (!f) return CDD_ENOMEM;
  f->f_center = f_center_mhz;
  f->bandwidth = bandwidth_mhz;
  f->sideband = sideband;
  f->dm = dm;
  f->n_chan = n_chan;
  f->frame = frame;
  f->logf = logf;
  f->n_avg = n_avg;
  f->f_lo = f_center_mhz - bandwidth_mhz / 2.0;
  f->fs = 2.0 * bandwidth_mhz;
  int rc = CDD_OK;
  if (!(f->f_lo > 0)) rc = CDD_EINVAL;
  if (rc == CDD_OK) {
    const double D = 4.148808e3;
    f->n_disp = D * dm * (pow(f->f_lo, -2.0) - pow(f->f_lo + bandwidth_mhz, -2.0)) * f->fs * 1e6;
    const long long unit = frame > n_avg ? frame : n_avg;
    long long ov = (long long)ceil(f->n_disp);
    f->n_ov = (ov + unit - 1) / unit * unit;
    if (n_fft == 0) {
      n_fft = next_pow2_above_ll(2.0 * f->n_disp);
      const long long b = next_pow2_above_ll((double)f->n_ov);
      if (b > n_fft) n_fft = b;
      if (n_fft < 2 * unit) n_fft = 2 * unit;
      if (n_fft < 64) n_fft = 64;
    }
    if (n_fft <= 0 || (n_fft & (n_fft - 1)) || n_fft <= f->n_ov || (n_fft - f->n_ov) % unit) rc = CDD_EINVAL;
    else if (n_fft < 64 || n_fft > (1LL << 27)) rc = CDD_EUNSUPPORTED;
  }
  if (rc == CDD_OK) {
    f->n_fft = n_fft;
    f->hop = n_fft - f->n_ov;
    int logn = 0;
    while ((1LL << logn) < n_fft) ++logn;
    // L_mid = 2^14 up to N = 2^19 (at most one outer pass); from N = 2^20 on,
    // 8192-point middle transforms (several CTAs per SM) and the outer bits
    // as radix-64 and -128 tile passes where they fit, pass 0 first:
    // 7: 128; 8: 64 4; 9: 64 8; 10: 64 16; 11: 128 16; 12: 64 64; 13: 64 128; 14: 128 128
    f->logs = logn < cdd::kMidLog ? logn : logn < cdd::kTileMinLog ? cdd::kMidLog : cdd::kMidLog - 1;
    int rest = logn - f->logs;
    static const int kPlan[8][2] = {{7, 0}, {6, 2}, {6, 3}, {6, 4}, {7, 4}, {6, 6}, {6, 7}, {7, 7}};
    const int* plan = rest >= 7 && rest <= 14 ? kPlan[rest - 7] : nullptr;
    int ip = 0;
    long long stride = n_fft, rprod = 1;
    while (rest > 0) {
      const int lr = plan ? plan[ip++] : rest >= 6 ? 6 : rest >= 4 ? 4 : rest;
      stride >>= lr;
      f->radix_out.push_back(1 << lr);
      f->stride_out.push_back(stride);
      f->rprod_out.push_back(rprod);
      rprod <<= lr;
      rest -= lr;
    }
  }
  if (rc != CDD_OK) {
    delete f;
    return rc;
  }
  *out = f;
  return CDD_OK;
}

int cdd_fullband_set(cdd_fullband f, int attr, int64_t value) {
  if (!f) return CDD_EINVAL;
  if (f->committed) return CDD_ESTATE;
  if (attr != CDD_ATTR_SEGMENTS_PER_BLOCK || value < 1 || value * f->hop > ((int64_t)1 << 36))
    return CDD_EINVAL;
  f->q = (int)value;
  return CDD_OK;
}

int cdd_fullband_get(cdd_fullband f, int attr, int64_t* v) {
  if (!f || !v) return CDD_EINVAL;
  switch (attr) {
    case CDD_ATTR_N_FFT: *v = f->n_fft; break;
    case CDD_ATTR_N_OV: *v = f->n_ov; break;
    case CDD_ATTR_HOP: *v = f->hop; break;
    case CDD_ATTR_N_AVG: *v = f->n_avg; break;
    case CDD_ATTR_N_CHAN: *v = f->n_chan; break;
    case CDD_ATTR_SEGMENTS_PER_BLOCK: *v = f->q; break;
    case CDD_ATTR_BLOCK_SAMPLES: *v = (int64_t)f->q * f->hop / f->frame; break;   // frames
    case CDD_ATTR_N_OUT_PER_BLOCK: *v = (int64_t)f->q * f->hop / f->n_avg; break;
    case CDD_ATTR_BYTES_DEVICE: *v = (int64_t)f->bytes_device; break;
    case CDD_ATTR_BLOCKS_DONE: *v = f->blocks; break;
    case CDD_ATTR_KERNEL_LAUNCHES: *v = f->last_launches; break;
    case CDD_ATTR_PASS_PLAN: {
      int64_t plan = f->logs;
      for (size_t p = 0; p < f->radix_out.size(); ++p) {
        int lr = 0;
        while ((1 << lr) < f->radix_out[p]) ++lr;
        plan |= (int64_t)lr << (8 + 4 * p);
      }
      *v = plan;
      break;
    }
    default: return CDD_EINVAL;
  }
  return CDD_OK;
}

int cdd_fullband_execute(cdd_fullband f, const int8_t* d_in, float* d_out, cudaStream_t s) {
  if (!f || !d_in || !d_out) return CDD_EINVAL;
  int rc = fprepare(f);
  if (rc) return rc;
  const long long n = f->n_fft, h = f->hop, nov = f->n_ov;
  float* ts = f->d_ts[f->cur];
  float* prev = f->d_ts[f->cur ^ 1];
  int launches = 0;
  // the previous block's last n_ov samples lead this block's series (Sec. 4.3)
  if (nov > 0) {
    FTRY(f, cudaMemcpyAsync(ts, prev + (long long)f->q * h, (size_t)nov * sizeof(float),
                            cudaMemcpyDeviceToDevice, s));
  }
  const long long frames = (long long)f->q * h / f->frame;
  FTRY(f, cdd::launch_icf(f->logf, reinterpret_cast<const char2*>(d_in), ts + nov, f->d_twf, f->d_wk, frames,
                          f->n_chan, s));
  launches += 1;
  const int no = (int)f->radix_out.size();
  const long long n_sub = n >> f->logs;
  for (int sg = 0; sg < f->q; ++sg) {
    const float* seg = ts + (long long)sg * h;            // N real samples from here
    if (no == 0) {
      FTRY(f, cdd::launch_middle(f->logs, f->d_w, seg, f->d_pw, f->d_chirp, f->d_tw, 1, s));
      launches += 1;
    } else {
      for (int p = 0; p < no; ++p)
        FTRY(f, cdd::launch_outer(true, p == 0, f->radix_out[p], f->d_w, seg, nullptr, n,
                                  f->stride_out[p], f->d_thi, f->d_tlo, f->d_lanes + p * cdd::kLaneTable, s));
      FTRY(f, cdd::launch_middle(f->logs, f->d_w, nullptr, nullptr, f->d_chirp, f->d_tw, n_sub, s));
      // the last pass also integrates across lanes when its radix is 16 and
      // n_avg <= 16, or 64 or 128 and n_avg <= 32; otherwise it writes Re(y)^2 for
      // the integration kernel
      const bool fused = (f->radix_out[0] == 16 && f->n_avg <= 16) || (f->radix_out[0] >= 64 && f->n_avg <= 32);
      for (int p = no - 1; p >= 0; --p)
        FTRY(f, cdd::launch_outer(false, p == 0, f->radix_out[p], f->d_w, nullptr, f->d_pw, n,
                                  f->stride_out[p], f->d_thi, f->d_tlo, f->d_lanes + p * cdd::kLaneTable, s,
                                  d_out + (long long)sg * (h / f->n_avg), nov, fused ? f->n_avg : 0));
      launches += 2 * no + 1;
      if (fused) continue;
    }
    const long long n_o = h / f->n_avg;
    cdd::fb_integrate_kernel<<<cdd::grid_for(n_o), 256, 0, s>>>(f->d_pw, d_out + (long long)sg * n_o,
                                                               nov, f->n_avg, n_o);
    FTRY(f, cudaGetLastError());
    launches += 1;
  }
  f->cur ^= 1;
  f->blocks += 1;
  f->last_launches = launches;
  return CDD_OK;
}

int cdd_fullband_reset(cdd_fullband f) {
  if (!f) return CDD_EINVAL;
  if (f->sticky) return f->sticky;
  if (f->committed) {
    FTRY(f, cudaDeviceSynchronize());
    for (int i = 0; i < 2; ++i)
      FTRY(f, cudaMemset(f->d_ts[i], 0, (size_t)ts_len(f) * sizeof(float)));
  }
  f->cur = 0;
  f->blocks = 0;
  return CDD_OK;
}

int cdd_fullband_destroy(cdd_fullband f) {
  if (!f) return CDD_OK;
  if (f->device >= 0) {
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(f->device);
    cudaDeviceSynchronize();
    ffree(f);
    if (prev >= 0) cudaSetDevice(prev);
  }
  delete f;
  return CDD_OK;
}

}  // extern "C"
