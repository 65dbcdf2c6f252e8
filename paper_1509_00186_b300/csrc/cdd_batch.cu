// cdd_batch.cu -- the batched form: many DM trials share each segment's
// forward transform, over a band whose channel groups (tiers) use different
// transform lengths.
//
// One CTA per (channel, segment) of a tier: int8 unpack and the forward radix
// passes as in the single-DM kernel, the spectrum (scaled by 1/N) parked in a
// global scratch row that stays in L2, then for every DM trial: the chirp of
// that DM applied on the fly (its phase is DM times a per-bin FP64 table of the
// DM = 1 phase held as two floats, so the product keeps FP64-like accuracy),
// the inverse radix passes, detection, integration, discard and the aligned
// store into the DM's output plane.  Sec. 2.1 Eq. 3 (chirp), Sec. 2.2
// (overlap-save), Sec. 3.1 (detect, integrate), Sec. 1.2 (alignment).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <vector>

// Packed FP32 only for the butterflies without a multiplication: the general
// ones, packed, measured slower here (register pressure of the DM loop).
#ifndef CDD_PACKED
#define CDD_PACKED 1
#endif
#include "../../include/cdd.h"
#include "cdd_fft.cuh"
#include "cdd_internal.h"
#include "cdd_passes.cuh"

namespace cdd {
namespace {

using namespace passes;

struct BatchArgs {
  const char2* in_cm;       // [C][rows] channel-major block
  long long rows;
  float* out;               // [n_dm][C][n_out]
  const float2* t1;         // [n_tchan][N] DM = 1 chirp phase in turns (hi, lo), chirp-pass order
  const float* t1f;         // the same as single floats when every phase is small (else nullptr)
  const float* taper;       // [N] taper per bin, chirp-pass order (nullptr: none)
  const float2* tw;         // twiddles of this N
  const char2* tail_rd;     // [C][tail_stride] last samples of the previous block
  char2* tail_wr;
  const float* ring_rd;     // [n_dm][C][r_max] previous block's last r outputs
  float* ring_wr;
  const int* shift;         // [n_dm][C]
  const float2* dms;        // [n_dm] DM as (hi, lo)
  float2* xs;               // [n_tchan * q][N] spectra
  int n_chan, chan0, n_tchan, n_ov, hop, n_avg, q, n_out, n_dm, r_max, tail_stride;
  int persistent;           // N = 8192 per-tier launch: the persistent kernel (1) or one CTA per item (0)
};

// exp(-2 pi i * DM * T1): the product and its reduction modulo one turn in
// two-float arithmetic, then the hardware sine/cosine on [-pi, pi].
__device__ __forceinline__ float2 dm_chirp(float2 t1, float2 dm) {
  const float p = dm.x * t1.x;
  const float e = fmaf(dm.x, t1.x, -p);                    // rounding error of the product
  const float lo = fmaf(dm.x, t1.y, fmaf(dm.y, t1.x, e));
  const float frac = (p - rintf(p)) + lo;
  float sn, cs;
  __sincosf(6.28318530717958647692f * frac, &sn, &cs);
  return make_float2(cs, -sn);
}

// The same with the DM = 1 phase as one float: used when no phase exceeds
// 16 turns, so its rounding (2^-24 relative) stays below 6e-6 rad.
__device__ __forceinline__ float2 dm_chirp1(float t1, float2 dm) {
  const float p = dm.x * t1;
  const float e = fmaf(dm.x, t1, -p);
  const float lo = fmaf(dm.y, t1, e);
  const float frac = (p - rintf(p)) + lo;
  float sn, cs;
  __sincosf(6.28318530717958647692f * frac, &sn, &cs);
  return make_float2(cs, -sn);
}

// dm_chirp1 for two bins at once, the phase arithmetic in packed FP32:
// c0, c1 = exp(-2 pi i DM T1) for t1 = (T1 of bin 0, T1 of bin 1).  dmx, ndm
// and dmy hold (DM hi, DM hi), (-DM hi, -DM hi) and (DM lo, DM lo).  -p is
// formed as (-DM hi) t1, which rounds to exactly the negated product, and
// p - rint(p) = rint(-p) - (-p), so every value equals the scalar form's.
__device__ __forceinline__ void dm_chirp1x2(float2 t1, float2 dmx, float2 ndm, float2 dmy, float2& c0,
                                            float2& c1) {
  const float2 np = mul2(ndm, t1);                                      // -p
  const float2 e = fma2(dmx, t1, np);                                   // rounding error of p
  const float2 lo = fma2(dmy, t1, e);
  const float2 frac = add2(sub2(make_float2(rintf(np.x), rintf(np.y)), np), lo);
  const float2 arg = mul2(make_float2(6.28318530717958647692f, 6.28318530717958647692f), frac);
  float sn, cs;
  __sincosf(arg.x, &sn, &cs);
  c0 = make_float2(cs, -sn);
  __sincosf(arg.y, &sn, &cs);
  c1 = make_float2(cs, -sn);
}

// One (channel, segment) work item w of a tier: the forward transform, the
// spectrum to its scratch row, then every DM trial.  SH: tw is in shared
// memory.  sync() is the group's barrier.  Returns true when buf (the power
// samples) was read after the last barrier.
#ifndef CDD_BATCH_PAIRS
#define CDD_BATCH_PAIRS 1
#endif
// The per-bin rows of the batched form (the T1 and taper tables, a segment's
// parked spectrum) hold bin kk of stride-1 group q at row index
// row_index<NG>(kk, q): with CDD_BATCH_PAIRS the bins kk and kk + 1 (kk even)
// sit side by side and the pairs run group-fastest, so one load brings two
// bins.  row_position<NG, RL>(idx) is the inverse: the working-buffer position
// q * RL + kk of the bin at row index idx.
template <int NG>
__host__ __device__ constexpr int row_index(int kk, int q) {
  return CDD_BATCH_PAIRS ? ((kk >> 1) * NG + q) * 2 + (kk & 1) : kk * NG + q;
}
template <int NG, int RL>
__host__ __device__ constexpr int row_position(int idx) {
  return CDD_BATCH_PAIRS ? ((idx >> 1) % NG) * RL + 2 * ((idx >> 1) / NG) + (idx & 1)
                         : (idx % NG) * RL + idx / NG;
}

template <int LOGN, bool SH, bool T1F, bool TAP, class Sync>
__device__ __forceinline__ bool batch_segment(const BatchArgs& a, float2* buf, const float2* tw, int lt,
                                              bool active, int w, float2* xk, Sync sync) {
  using PL = PassPlan<LOGN>;
  constexpr int N = PL::N;
  constexpr int T = PL::T;
  constexpr int R0 = PL::R(0);
  constexpr int RL = PL::RL;
  constexpr int NG = N / RL;
  constexpr int PERC = NG / T;
  static_assert(RL <= 16, "stride-1 groups must not cross a padding word");
  static_assert(RL % 2 == 0, "bins are handled in pairs");
  // The last forward pass, the spectrum/chirp groups and the first inverse
  // pass stay within a warp when the last two radices are equal.
  constexpr bool kWarpMid = PL::P >= 3 && PL::R(PL::P - 2) == RL && RL <= 32;
  auto mid_sync = [&] {
    if constexpr (kWarpMid) __syncwarp();
    else sync();
  };

  const int kt = active ? w % a.n_tchan : 0;     // channel within the tier, fastest
  const int s = active ? w / a.n_tchan : 0;
  const int k = a.chan0 + kt;
  float2* pb0 = buf + pad<LOGN>(lt);
  float2 v[R0];

  // ---- pass 0, forward, straight from the channel-major block
  if (active) {
    const long long row0 = (long long)s * a.hop - a.n_ov;
    const unsigned short* src = reinterpret_cast<const unsigned short*>(a.in_cm) + (long long)k * a.rows;
    const unsigned short* tail = reinterpret_cast<const unsigned short*>(a.tail_rd) + (long long)k * a.tail_stride;
    unsigned short c[R0];
#pragma unroll
    for (int j = 0; j < R0; ++j) {
      const long long row = row0 + lt + T * j;
      c[j] = __ldg(row >= 0 ? src + row : tail + (row + a.n_ov));
    }
    if (s == a.q - 1 && a.n_ov > 0) {
      unsigned short* tout = reinterpret_cast<unsigned short*>(a.tail_wr) + (long long)k * a.tail_stride;
#pragma unroll
      for (int j = 0; j < R0; ++j) {
        const int n = lt + T * j;
        if (n >= N - a.n_ov) tout[n - (N - a.n_ov)] = c[j];
      }
    }
#pragma unroll
    for (int j = 0; j < R0; ++j) v[j] = unpack_i8x2(c[j]);
    dft<R0, -1>(v);
    if constexpr (kRecPass0<LOGN, SH>) {
      apply_twiddles_rec<R0, T, SH, false>(v, tw + lt);
    } else {
#pragma unroll
      for (int kk = 1; kk < R0; ++kk) v[kk] = cmul(v[kk], ld_tw<SH>(&tw[kk * T + lt]));
    }
#pragma unroll
    for (int kk = 0; kk < R0; ++kk) pb0[poff<LOGN, T>(kk)] = v[kk];
  }
  sync();
  static_for<1, PL::P - 1>([&](auto P_) {
    constexpr int p = decltype(P_)::value;
    if (active) fwd_pass<LOGN, p, SH>(buf, tw, lt);
    if constexpr (p == PL::P - 2) mid_sync();
    else sync();
  });
  if constexpr (PL::P < 3) sync();

  // ---- last forward radix: the spectrum, scaled by 1/N, to this segment's
  // scratch row.  A thread later chirps and writes back exactly the groups it
  // reads here, so no barrier separates the two.
  if (active) {
#pragma unroll 1
    for (int i = 0; i < PERC; ++i) {
      const int q = lt + i * T;
      const float2* pb = buf + pad<LOGN>(q * RL);
      float2 x[RL];
      load_group<LOGN, RL>(pb, x);
      dft<RL, -1>(x);
      // the taper (Sec. 2.2) depends on the bin only, so it is applied here
      // once for every DM trial, with the 1/N of the inverse transform (a
      // compile-time switch: the untapered kernels keep their own code)
#if CDD_BATCH_PAIRS
#pragma unroll
      for (int kk = 0; kk < RL; kk += 2) {
        float s0 = 1.0f / N, s1 = 1.0f / N;
        if constexpr (TAP) {
          const float2 t = __ldg(reinterpret_cast<const float2*>(a.taper) + (kk / 2) * NG + q);
          s0 = t.x * (1.0f / N);
          s1 = t.y * (1.0f / N);
        }
        reinterpret_cast<float4*>(xk)[(kk / 2) * NG + q] =
            make_float4(x[kk].x * s0, x[kk].y * s0, x[kk + 1].x * s1, x[kk + 1].y * s1);
      }
#else
      if constexpr (TAP) {
#pragma unroll
        for (int kk = 0; kk < RL; ++kk) {
          const float sc = __ldg(&a.taper[kk * NG + q]) * (1.0f / N);
          xk[kk * NG + q] = make_float2(x[kk].x * sc, x[kk].y * sc);
        }
      } else {
#pragma unroll
        for (int kk = 0; kk < RL; ++kk)
          xk[kk * NG + q] = make_float2(x[kk].x * (1.0f / N), x[kk].y * (1.0f / N));
      }
#endif
    }
  }

  const float2* t1k = a.t1 + (size_t)kt * N;
  const float* t1fk = a.t1f + (size_t)kt * N;
  const int na = a.n_avg;
  const int n_int = a.hop / na;
  // integration across lanes as in the single-DM kernel; N = 16384 keeps the
  // shared-memory form (the register form spills there and measured slower)
  bool in_lanes = false;
  if constexpr (T % 32 == 0 && LOGN <= 13) in_lanes = na <= R0 && na <= 32 && (na & (na - 1)) == 0;
  float* pw = reinterpret_cast<float*>(buf);
#pragma unroll 1
  for (int d = 0; d < a.n_dm; ++d) {
    if (!in_lanes && d > 0) sync();           // the previous DM's power samples are read
    // ---- chirp of DM d and first inverse radix (each thread re-reads its own rows)
    if (active) {
      const float2 dm = a.dms[d];
#pragma unroll 1
      for (int i = 0; i < PERC; ++i) {
        const int q = lt + i * T;
        float2 x[RL];
#if CDD_BATCH_PAIRS
        const float4* xk2 = reinterpret_cast<const float4*>(xk) + q;
        if constexpr (T1F) {
          const float2 dmx = make_float2(dm.x, dm.x), ndm = make_float2(-dm.x, -dm.x);
          const float2 dmy = make_float2(dm.y, dm.y);
#pragma unroll
          for (int kk = 0; kk < RL; kk += 2) {
            float2 c0, c1;
            dm_chirp1x2(__ldg(reinterpret_cast<const float2*>(t1fk) + (kk / 2) * NG + q), dmx, ndm, dmy, c0, c1);
            const float4 xx = xk2[(kk / 2) * NG];
            x[kk] = cmul(make_float2(xx.x, xx.y), c0);
            x[kk + 1] = cmul(make_float2(xx.z, xx.w), c1);
          }
        } else {
#pragma unroll
          for (int kk = 0; kk < RL; kk += 2) {
            const float4 t = __ldg(reinterpret_cast<const float4*>(t1k) + (kk / 2) * NG + q);
            const float4 xx = xk2[(kk / 2) * NG];
            x[kk] = cmul(make_float2(xx.x, xx.y), dm_chirp(make_float2(t.x, t.y), dm));
            x[kk + 1] = cmul(make_float2(xx.z, xx.w), dm_chirp(make_float2(t.z, t.w), dm));
          }
        }
#else
        if constexpr (T1F && RL % 2 == 0) {
          const float2 dmx = make_float2(dm.x, dm.x), ndm = make_float2(-dm.x, -dm.x);
          const float2 dmy = make_float2(dm.y, dm.y);
#pragma unroll
          for (int kk = 0; kk < RL; kk += 2) {
            float2 c0, c1;
            dm_chirp1x2(make_float2(__ldg(&t1fk[kk * NG + q]), __ldg(&t1fk[(kk + 1) * NG + q])), dmx, ndm, dmy,
                        c0, c1);
            x[kk] = cmul(xk[kk * NG + q], c0);
            x[kk + 1] = cmul(xk[(kk + 1) * NG + q], c1);
          }
        } else {
#pragma unroll
          for (int kk = 0; kk < RL; ++kk)
            x[kk] = cmul(xk[kk * NG + q], T1F ? dm_chirp1(__ldg(&t1fk[kk * NG + q]), dm)
                                              : dm_chirp(__ldg(&t1k[kk * NG + q]), dm));
        }
#endif
        dft<RL, 1>(x);
        store_group<LOGN, RL>(buf + pad<LOGN>(q * RL), x);
      }
    }
    if constexpr (PL::P >= 3) mid_sync();
    else sync();
    static_for<1, PL::P - 1>([&](auto I_) {
      if (active) inv_pass<LOGN, PL::P - 1 - decltype(I_)::value, SH>(buf, tw, lt);
      sync();
    });
    // ---- pass 0, inverse, detection
    if (active) {
#pragma unroll
      for (int kk = 0; kk < R0; ++kk) v[kk] = pb0[poff<LOGN, T>(kk)];
      if constexpr (kRecPass0<LOGN, SH>) {
        apply_twiddles_rec<R0, T, SH, true>(v, tw + lt);
      } else {
#pragma unroll
        for (int kk = 1; kk < R0; ++kk) v[kk] = cmulc(v[kk], ld_tw<SH>(&tw[kk * T + lt]));
      }
      dft<R0, 1>(v);
    }
    sync();                                   // every thread has read buf
    if (!in_lanes) {
      if (active) {
#pragma unroll
        for (int j = 0; j < R0; ++j) {
          const int n = lt + T * j;
          pw[n + (n >> 5)] = fmaf(v[j].x, v[j].x, v[j].y * v[j].y);
        }
      }
      sync();
    }
    // ---- integrate, discard the overlap, align into DM d's plane
    if (active) {
      const size_t row = (size_t)d * a.n_chan + k;
      const int r = __ldg(&a.shift[row]);
      float* outk = a.out + row * a.n_out;
      float* rw = a.ring_wr + row * a.r_max;
      auto emit = [&](int m, float acc) {
        const int dst = s * n_int + m + r;     // aligned index within this block
        if (dst < a.n_out) outk[dst] = acc;
        else rw[dst - a.n_out] = acc;          // the next block's first r outputs
      };
      if (in_lanes) {
        if constexpr (T % 32 == 0 && LOGN <= 13) integrate_in_lanes<R0, T>(v, lt, a.n_ov, na, emit);
      } else {
        for (int m = lt; m < n_int; m += T) {
          const int n0 = a.n_ov + m * na;
          float acc = 0.f;
          for (int i = 0; i < na; ++i) acc += pw[(n0 + i) + ((n0 + i) >> 5)];
          emit(m, acc);
        }
      }
      if (s == 0) {
        const float* rr = a.ring_rd + row * a.r_max;
        for (int m = lt; m < r; m += T) outk[m] = rr[m];
      }
    }
  }
  return !in_lanes;
}

template <int LOGN, bool T1F, bool TAP>
__global__ void __launch_bounds__(Cfg<LOGN>::THREADS, Cfg<LOGN>::MINB)
batch_kernel(const BatchArgs a) {
  using PL = PassPlan<LOGN>;
  using CF = Cfg<LOGN>;
  extern __shared__ __align__(16) float2 smem[];
  const int g = threadIdx.x / PL::T;
  const int lt = threadIdx.x % PL::T;
  float2* buf = smem + g * CF::SEG_F2;
  const int w = blockIdx.x * CF::G + g;
  const bool active = w < a.n_tchan * a.q;
  batch_segment<LOGN, false, T1F, TAP>(a, buf, a.tw, lt, active, w, a.xs + (size_t)w * PL::N,
                                       [] { __syncthreads(); });
}

// Persistent form for N = 8192: one CTA per SM, two groups of 256
// threads looping over work items with their own named barriers, the twiddle
// table staged once in shared memory (each work item runs one forward and
// n_dm inverse transforms with it).
template <int LOGN>
struct BatchPersist {
  using PL = PassPlan<LOGN>;
  static constexpr int GROUPS = 2;
  static constexpr int THREADS = GROUPS * PL::T;
  static constexpr size_t SMEM = (size_t(PL::TW_LEN) + size_t(GROUPS) * padded_len<LOGN>()) * sizeof(float2);
};

template <int LOGN, bool T1F, bool TAP>
__global__ void __launch_bounds__(BatchPersist<LOGN>::THREADS, 1)
batch_persistent_kernel(const BatchArgs a) {
  using PL = PassPlan<LOGN>;
  using BP = BatchPersist<LOGN>;
  constexpr int T = PL::T;
  extern __shared__ __align__(16) float2 smem[];
  float2* tws = smem;
  for (int i = threadIdx.x; i < PL::TW_LEN; i += blockDim.x) tws[i] = __ldg(&a.tw[i]);
  __syncthreads();
  const int g = threadIdx.x / T;
  const int lt = threadIdx.x % T;
  float2* buf = smem + PL::TW_LEN + g * padded_len<LOGN>();
  const int bar = g + 1;                       // named barriers 1, 2 (0 is __syncthreads)
  auto sync = [bar] { asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(T) : "memory"); };
  const int work = a.n_tchan * a.q;
  for (int w = blockIdx.x * BP::GROUPS + g; w < work; w += gridDim.x * BP::GROUPS) {
    if (batch_segment<LOGN, true, T1F, TAP>(a, buf, tws, lt, true, w, a.xs + (size_t)w * PL::N, sync))
      sync();                                  // buf is rewritten by the next work item
  }
}

// ------------------------------------------------------------------ one launch
//
// Every tier of a batch in one persistent launch: one 512-thread CTA per SM
// takes the tiers in order (the longest transforms first), and within a tier
// its groups (one per N / R_0 threads: 1 x 512 for N = 16384, 2 x 256 for
// 8192 and 4096, 4 x 128 for 2048) claim (channel, segment) work items from
// the tier's counter until it is exhausted; a CTA that runs out moves on to
// the next tier while others finish theirs, so no launch boundary idles the
// GPU between tiers.  Each group parks its spectrum in its own scratch row
// (slots: 16384 points per CTA, L2-resident) instead of one row per item.
constexpr int kMultiThreads = 512;
constexpr int kMultiTiers = 4;

struct MultiArgs {
  BatchArgs tier[kMultiTiers];
  int logn[kMultiTiers];
  int n_tiers;
  int* counters;       // [kMultiTiers] work items claimed (zero at launch)
  float2* slots;       // [gridDim.x][16384] scratch rows
};

template <int LOGN>
struct MultiCfg {
  using PL = PassPlan<LOGN>;
  static constexpr int T = PL::T;
  static constexpr int G = kMultiThreads / T;
  static constexpr bool SH = LOGN == 13;        // N = 8192 stages its twiddles, as its persistent kernel
  static constexpr size_t SMEM = (size_t(SH ? PL::TW_LEN : 0) + size_t(G) * padded_len<LOGN>()) * sizeof(float2);
  static_assert(G * T == kMultiThreads, "a tier's groups fill the CTA");
};

// The multi-tier launch handles tiers of 2048 to 16384 points.
__host__ __device__ constexpr bool multi_logn_ok(int logn) { return logn >= 11 && logn <= 14; }

template <int LOGN, bool T1F, bool TAP>
__device__ __forceinline__ void multi_tier(const BatchArgs& a, int* counter, float2* smem, float2* slot,
                                           volatile int* claim) {
  using MC = MultiCfg<LOGN>;
  using PL = PassPlan<LOGN>;
  constexpr int T = MC::T;
  const int g = threadIdx.x / T, lt = threadIdx.x % T;
  float2* buf = smem + (MC::SH ? PL::TW_LEN : 0) + g * padded_len<LOGN>();
  const float2* tw = a.tw;
  if constexpr (MC::SH) {
    for (int i = threadIdx.x; i < PL::TW_LEN; i += kMultiThreads) smem[i] = __ldg(&a.tw[i]);
    __syncthreads();
    tw = smem;
  }
  const int bar = 1 + g;
  auto sync = [bar] { asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(T) : "memory"); };
  float2* xk = slot + (size_t)g * PL::N;
  const int work = a.n_tchan * a.q;
  for (;;) {
    if (lt == 0) claim[g] = atomicAdd(counter, 1);
    sync();
    const int w = claim[g];              // read by the group before its next barrier
    if (w >= work) break;
    if (batch_segment<LOGN, MC::SH, T1F, TAP>(a, buf, tw, lt, true, w, xk, sync)) sync();
  }
}

template <bool T1F, bool TAP>
__global__ void __launch_bounds__(kMultiThreads, 1) batch_multi_kernel(const MultiArgs m) {
  extern __shared__ __align__(16) float2 smem[];
  __shared__ int claim[kMultiThreads / 128];
  float2* slot = m.slots + (size_t)blockIdx.x * 16384;
  for (int t = 0; t < m.n_tiers; ++t) {
    switch (m.logn[t]) {
      case 14: multi_tier<14, T1F, TAP>(m.tier[t], m.counters + t, smem, slot, claim); break;
      case 13: multi_tier<13, T1F, TAP>(m.tier[t], m.counters + t, smem, slot, claim); break;
      case 12: multi_tier<12, T1F, TAP>(m.tier[t], m.counters + t, smem, slot, claim); break;
      case 11: multi_tier<11, T1F, TAP>(m.tier[t], m.counters + t, smem, slot, claim); break;
      default: break;
    }
    __syncthreads();                     // the shared memory is laid out anew for the next tier
  }
}

size_t multi_smem() {
  size_t b = MultiCfg<14>::SMEM;
  b = b > MultiCfg<13>::SMEM ? b : MultiCfg<13>::SMEM;
  b = b > MultiCfg<12>::SMEM ? b : MultiCfg<12>::SMEM;
  return b > MultiCfg<11>::SMEM ? b : MultiCfg<11>::SMEM;
}

template <bool T1F, bool TAP>
cudaError_t launch_multi_tt(const MultiArgs& m, unsigned grid, cudaStream_t s) {
  static bool attr_set[128] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  if (!attr_set[dev]) {
    e = cudaFuncSetAttribute(batch_multi_kernel<T1F, TAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)multi_smem());
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  e = cudaMemsetAsync(m.counters, 0, kMultiTiers * sizeof(int), s);
  if (e != cudaSuccess) return e;
  batch_multi_kernel<T1F, TAP><<<grid, kMultiThreads, multi_smem(), s>>>(m);
  return cudaGetLastError();
}

cudaError_t launch_multi(const MultiArgs& m, bool t1f, bool tap, unsigned grid, cudaStream_t s) {
  if (tap) return t1f ? launch_multi_tt<true, true>(m, grid, s) : launch_multi_tt<false, true>(m, grid, s);
  return t1f ? launch_multi_tt<true, false>(m, grid, s) : launch_multi_tt<false, false>(m, grid, s);
}

// T1[kt][idx]: Eq. 3 phase in turns at DM = 1 for channel chan0 + kt and the
// bin held at table index idx (FP64, split into two floats).  A lower-sideband
// channel (sideband < 0; f_base the band's top edge) holds the conjugate
// mirror: bin j sits where the upper-sideband bin -j does, and its correction
// is the conjugate, so its table holds minus the phase.
template <int LOGN>
__global__ void t1_table_kernel(float2* t1, float* t1f, int n_tchan, int chan0, double f_base, double chan_bw,
                                int sideband) {
  using PL = PassPlan<LOGN>;
  constexpr int N = PL::N;
  constexpr int NG = N / PL::RL;
  const long long total = (long long)n_tchan * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int kt = (int)(e / N);
    const int idx = (int)(e % N);
    const int pos = row_position<NG, PL::RL>(idx);
    const int bin = position_to_bin<LOGN>(pos);
    const int obin = sideband > 0 ? bin : (N - bin) % N;
    const int sbin = obin < N / 2 ? obin : obin - N;
    const double f_lo = sideband > 0 ? f_base + chan_bw * (chan0 + kt) : f_base - chan_bw * (chan0 + kt + 1.0);
    const double f_l = sbin * (chan_bw / N) + 0.5 * chan_bw;
    const double turns = (sideband > 0 ? 1.0 : -1.0) * kDispD * 1e6 * f_l * f_l / ((f_l + f_lo) * f_lo * f_lo);
    const float hi = (float)turns;
    if (t1f) t1f[e] = hi;
    else t1[e] = make_float2(hi, (float)(turns - (double)hi));
  }
}

template <int LOGN, bool T1F, bool TAP>
cudaError_t launch_batch_tt(const BatchArgs& a, cudaStream_t s) {
  using CF = Cfg<LOGN>;
  static bool attr_set[128] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  if (!attr_set[dev]) {
    e = cudaFuncSetAttribute(batch_kernel<LOGN, T1F, TAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CF::SMEM);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const long long work = (long long)a.n_tchan * a.q;
  // N = 8192 only: the N = 4096 tier runs faster as three non-persistent
  // 256-thread CTAs per SM (142.3 against 146.4 ms per batched block)
  if constexpr (LOGN == 13) if (a.persistent) {
    using BP = BatchPersist<LOGN>;
    static bool pset[128] = {};
    if (!pset[dev]) {
      e = cudaFuncSetAttribute(batch_persistent_kernel<LOGN, T1F, TAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)BP::SMEM);
      if (e != cudaSuccess) return e;
      pset[dev] = true;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long need = (work + BP::GROUPS - 1) / BP::GROUPS;
    const unsigned grid = (unsigned)(need < sms ? need : sms);
    batch_persistent_kernel<LOGN, T1F, TAP><<<grid, BP::THREADS, BP::SMEM, s>>>(a);
    return cudaGetLastError();
  }
  batch_kernel<LOGN, T1F, TAP><<<(unsigned)((work + CF::G - 1) / CF::G), CF::THREADS, CF::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int LOGN>
cudaError_t launch_batch_t(const BatchArgs& a, cudaStream_t s) {
  if (a.taper) return a.t1f ? launch_batch_tt<LOGN, true, true>(a, s) : launch_batch_tt<LOGN, false, true>(a, s);
  return a.t1f ? launch_batch_tt<LOGN, true, false>(a, s) : launch_batch_tt<LOGN, false, false>(a, s);
}

template <int LOGN>
cudaError_t launch_t1_t(float2* t1, float* t1f, int n_tchan, int chan0, double f_base, double chan_bw,
                        int sideband, cudaStream_t s) {
  const long long total = (long long)n_tchan << LOGN;
  const unsigned grid = (unsigned)((total + 255) / 256 < 65535 ? (total + 255) / 256 : 65535);
  t1_table_kernel<LOGN><<<grid, 256, 0, s>>>(t1, t1f, n_tchan, chan0, f_base, chan_bw, sideband);
  return cudaGetLastError();
}

#define CDD_BATCH_CASES(X) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14)

cudaError_t launch_batch(int logn, const BatchArgs& a, cudaStream_t s) {
  switch (logn) {
#define X(L) case L: return launch_batch_t<L>(a, s);
    CDD_BATCH_CASES(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

// taper[idx] for the bin held at chirp-pass index idx: Hann sin^2(pi x) or
// Welch 1 - (2x - 1)^2, x = f_l / chan_bw (Sec. 2.2), mirrored for a lower
// sideband (FP64, rounded).
template <int LOGN>
__global__ void batch_taper_kernel(float* tap, int taper, int sideband) {
  using PL = PassPlan<LOGN>;
  constexpr int N = PL::N;
  constexpr int NG = N / PL::RL;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x) {
    const int pos = row_position<NG, PL::RL>(idx);
    const int bin = position_to_bin<LOGN>(pos);
    const int obin = sideband > 0 ? bin : (N - bin) % N;
    const int sbin = obin < N / 2 ? obin : obin - N;
    const double x = (double)sbin / N + 0.5;
    double w = 1.0;
    if (taper == CDD_TAPER_HANN) {
      const double sx = sinpi(x);
      w = sx * sx;
    } else if (taper == CDD_TAPER_WELCH) {
      const double y = 2.0 * x - 1.0;
      w = 1.0 - y * y;
    }
    tap[idx] = (float)w;
  }
}

cudaError_t launch_batch_taper(int logn, float* tap, int taper, int sideband, cudaStream_t s) {
  switch (logn) {
#define X(L) case L: batch_taper_kernel<L><<<((1 << L) + 255) / 256, 256, 0, s>>>(tap, taper, sideband); break;
    CDD_BATCH_CASES(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_t1(int logn, float2* t1, float* t1f, int n_tchan, int chan0, double f_base, double chan_bw,
                      int sideband, cudaStream_t s) {
  switch (logn) {
#define X(L) case L: return launch_t1_t<L>(t1, t1f, n_tchan, chan0, f_base, chan_bw, sideband, s);
    CDD_BATCH_CASES(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace cdd

// ------------------------------------------------------------------ host side

struct cdd_batch_s {
  struct Tier {
    int n_fft = 0, logn = 0, n_ov = 0, hop = 0, chan0 = 0, n_tchan = 0;
    float2* d_tw = nullptr;
    float* d_taper = nullptr;              // [N] taper per bin (CDD_ATTR_TAPER set), else nullptr
    float2* d_t1 = nullptr;
    float* d_t1f = nullptr;
  };
  double f_center = 0, bandwidth = 0, chan_bw = 0, f_lo0 = 0;
  int sideband = 1;                      // +1 upper (channel 0 lowest), -1 lower (channel 0 highest)
  double f_base = 0;                     // upper: f_lo0; lower: the band's top edge
  int taper = CDD_TAPER_NONE;
  int n_chan = 0, n_avg = 0, n_dm = 0;
  std::vector<double> dms;
  std::vector<Tier> tiers;
  std::vector<int64_t> shift;            // [n_dm][C]
  int64_t r_max = 0;
  int hop_max = 0, n_ov_max = 0;
  int q = 1;                             // block = q * hop_max samples per channel
  bool t1_single = false;                // DM = 1 phase table as single floats (small phases)
  bool committed = false;
  int device = -1;
  int sticky = CDD_OK;
  char2* d_in_cm = nullptr;
  char2* d_tail[2] = {nullptr, nullptr};
  float* d_ring[2] = {nullptr, nullptr};
  int* d_shift = nullptr;
  float2* d_dms = nullptr;
  float2* d_xs = nullptr;
  // execution form (CDD_ATTR_BATCH_FORM): requested (-1: tune at the first
  // execute) and in use; the one-launch form's counters and scratch slots
  int form_req = -1, form = -1;
  bool multi_ok = false;
  unsigned multi_grid = 0;
  int* d_counters = nullptr;
  float2* d_slots = nullptr;
  int64_t tune_ns[3] = {0, 0, 0};
  size_t bytes_device = 0;
  int parity = 0;
  int64_t blocks = 0;
  int last_launches = 0;
};

namespace {

constexpr double kDispDHost = 4.148808e3;   // s MHz^2 cm^3 / pc (Eq. 3)

int bfail(cdd_batch b, cudaError_t e) {
  if (e == cudaSuccess) return CDD_OK;
  b->sticky = CDD_ECUDA;
  return CDD_ECUDA;
}

#define BTRY(b, call)                              \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return bfail(b, e_);    \
  } while (0)

template <class T>
int balloc(cdd_batch b, T** p, size_t bytes) {
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    *p = nullptr;
    return CDD_ENOMEM;
  }
  if (e != cudaSuccess) return bfail(b, e);
  b->bytes_device += bytes;
  return CDD_OK;
}

int64_t block_samples(const cdd_batch b) { return (int64_t)b->q * b->hop_max; }
int64_t n_out(const cdd_batch b) { return block_samples(b) / b->n_avg; }

void bfree(cdd_batch b) {
  for (auto& t : b->tiers) {
    cudaFree(t.d_tw);
    cudaFree(t.d_taper);
    cudaFree(t.d_t1);
    cudaFree(t.d_t1f);
  }
  cudaFree(b->d_in_cm);
  cudaFree(b->d_tail[0]);
  cudaFree(b->d_tail[1]);
  cudaFree(b->d_ring[0]);
  cudaFree(b->d_ring[1]);
  cudaFree(b->d_shift);
  cudaFree(b->d_dms);
  cudaFree(b->d_xs);
  cudaFree(b->d_counters);
  cudaFree(b->d_slots);
}

int bzero_state(cdd_batch b, cudaStream_t s) {
  const size_t tb = (size_t)b->n_chan * (b->n_ov_max > 0 ? b->n_ov_max : 1) * sizeof(char2);
  const size_t rb = (size_t)b->n_dm * b->n_chan * (b->r_max > 0 ? b->r_max : 1) * sizeof(float);
  for (int i = 0; i < 2; ++i) {
    BTRY(b, cudaMemsetAsync(b->d_tail[i], 0, tb, s));
    BTRY(b, cudaMemsetAsync(b->d_ring[i], 0, rb, s));
  }
  b->parity = 0;
  b->blocks = 0;
  return CDD_OK;
}

// Largest phase a chirp of this batch reaches, in turns: the top bin of the
// lowest channel at the largest DM (Eq. 3 grows with f_l and falls with f_o).
double max_phase_turns(const cdd_batch b) {
  double dm_max = 0;
  for (double d : b->dms) dm_max = d > dm_max ? d : dm_max;
  const double f_l = b->chan_bw, f_o = b->f_lo0;
  return kDispDHost * 1e6 * dm_max * f_l * f_l / ((f_l + f_o) * f_o * f_o);
}

// Up to this many turns the single-float DM = 1 phase (relative rounding
// 2^-24) keeps every chirp phase within 2*pi * 16 * 2^-24 ~ 6e-6 rad.
constexpr double kT1SingleTurns = 16.0;

int bcommit_once(cdd_batch b) {
  BTRY(b, cudaGetDevice(&b->device));
  b->t1_single = max_phase_turns(b) <= kT1SingleTurns;
  if (n_out(b) < b->r_max) return CDD_EINVAL;        // a block must outlast the largest delay
  int rc;
  const int64_t rows = block_samples(b);
  if ((rc = balloc(b, &b->d_in_cm, (size_t)b->n_chan * rows * sizeof(char2)))) return rc;
  const size_t tb = (size_t)b->n_chan * (b->n_ov_max > 0 ? b->n_ov_max : 1) * sizeof(char2);
  const size_t rb = (size_t)b->n_dm * b->n_chan * (b->r_max > 0 ? b->r_max : 1) * sizeof(float);
  for (int i = 0; i < 2; ++i) {
    if ((rc = balloc(b, &b->d_tail[i], tb))) return rc;
    if ((rc = balloc(b, &b->d_ring[i], rb))) return rc;
  }
  if ((rc = balloc(b, &b->d_shift, b->shift.size() * sizeof(int)))) return rc;
  if ((rc = balloc(b, &b->d_dms, (size_t)b->n_dm * sizeof(float2)))) return rc;
  size_t xs = 0;
  for (auto& t : b->tiers) {
    const size_t segs = (size_t)t.n_tchan * (rows / t.hop);
    if (segs * t.n_fft > xs) xs = segs * t.n_fft;
    if ((rc = balloc(b, &t.d_tw, (size_t)cdd::twiddle_table_len(t.logn) * sizeof(float2)))) return rc;
    if (b->taper != CDD_TAPER_NONE && (rc = balloc(b, &t.d_taper, (size_t)t.n_fft * sizeof(float)))) return rc;
    if (b->t1_single) {
      if ((rc = balloc(b, &t.d_t1f, (size_t)t.n_tchan * t.n_fft * sizeof(float)))) return rc;
    } else if ((rc = balloc(b, &t.d_t1, (size_t)t.n_tchan * t.n_fft * sizeof(float2)))) {
      return rc;
    }
  }
  if ((rc = balloc(b, &b->d_xs, xs * sizeof(float2)))) return rc;
  // the one-launch form: tiers of 2048 to 16384 points, at most four
  b->multi_ok = b->tiers.size() <= (size_t)cdd::kMultiTiers;
  for (auto& t : b->tiers) b->multi_ok = b->multi_ok && cdd::multi_logn_ok(t.logn);
  if (b->multi_ok) {
    int sms = 0;
    BTRY(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    b->multi_grid = (unsigned)sms;
    if ((rc = balloc(b, &b->d_counters, cdd::kMultiTiers * sizeof(int)))) return rc;
    if ((rc = balloc(b, &b->d_slots, (size_t)sms * 16384 * sizeof(float2)))) return rc;
  }

  std::vector<int> sh(b->shift.begin(), b->shift.end());
  BTRY(b, cudaMemcpy(b->d_shift, sh.data(), sh.size() * sizeof(int), cudaMemcpyHostToDevice));
  std::vector<float2> dm2(b->n_dm);
  for (int d = 0; d < b->n_dm; ++d) {
    const float hi = (float)b->dms[d];
    dm2[d] = make_float2(hi, (float)(b->dms[d] - (double)hi));
  }
  BTRY(b, cudaMemcpy(b->d_dms, dm2.data(), dm2.size() * sizeof(float2), cudaMemcpyHostToDevice));
  cudaStream_t s;
  BTRY(b, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaError_t e = cudaSuccess;
  for (auto& t : b->tiers) {
    if (e == cudaSuccess) e = cdd::launch_twiddle_table(t.logn, t.d_tw, s);
    if (e == cudaSuccess)
      e = cdd::launch_t1(t.logn, t.d_t1, t.d_t1f, t.n_tchan, t.chan0, b->f_base, b->chan_bw, b->sideband, s);
    if (e == cudaSuccess && t.d_taper) e = cdd::launch_batch_taper(t.logn, t.d_taper, b->taper, b->sideband, s);
  }
  if (e == cudaSuccess && (rc = bzero_state(b, s)) != CDD_OK) {
    cudaStreamDestroy(s);
    return rc;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (e != cudaSuccess) return bfail(b, e);
  b->committed = true;
  return CDD_OK;
}

// Execution forms of a batch (CDD_ATTR_BATCH_FORM).
constexpr int kFormTiers = 0;     // one launch per tier; N = 8192 as a persistent kernel
constexpr int kFormTiersNP = 1;   // one launch per tier; every tier one CTA per work item
constexpr int kFormMulti = 2;     // every tier in one persistent launch
constexpr int kForms = 3;

int launches_of(const cdd_batch b, int form) {
  return form == kFormMulti ? 2 : (int)b->tiers.size();     // the one-launch form also clears its counters
}

// Forms chosen by tuning, per device and batch shape, for the process's lifetime.
std::mutex g_form_mu;
std::map<std::vector<int64_t>, int> g_forms;

std::vector<int64_t> form_key(const cdd_batch b) {
  std::vector<int64_t> k = {b->device, b->n_dm, b->n_avg, b->t1_single ? 1 : 0, b->taper, b->q};
  for (auto& t : b->tiers) {
    k.push_back(t.logn);
    k.push_back(t.n_tchan);
    k.push_back(t.hop);
  }
  return k;
}
int cached_form(const cdd_batch b) {
  std::lock_guard<std::mutex> lock(g_form_mu);
  auto it = g_forms.find(form_key(b));
  return it == g_forms.end() ? -1 : it->second;
}
void remember_form(const cdd_batch b, int form) {
  std::lock_guard<std::mutex> lock(g_form_mu);
  g_forms[form_key(b)] = form;
}

int bprepare(cdd_batch b) {
  if (!b) return CDD_EINVAL;
  if (b->sticky) return b->sticky;
  if (!b->committed) {
    const int rc = bcommit_once(b);
    if (rc != CDD_OK) {
      b->sticky = rc;
      return rc;
    }
  }
  int dev = -1;
  BTRY(b, cudaGetDevice(&dev));
  return dev == b->device ? CDD_OK : CDD_EINVAL;
}

}  // namespace

extern "C" {

int cdd_batch_create(cdd_batch* out, double f_center_mhz, double bandwidth_mhz, int n_chan,
                     const double* dms, int n_dm, const int* tier_nfft, int n_tiers, int n_avg) {
  if (!out) return CDD_EINVAL;
  *out = nullptr;
  if (!dms || n_dm <= 0 || !tier_nfft || n_tiers <= 0 || n_chan <= 0 || n_chan % n_tiers ||
      n_avg <= 0 || !(f_center_mhz > 0) || !isfinite(bandwidth_mhz) || bandwidth_mhz == 0)
    return CDD_EINVAL;
  cdd_batch b = new (std::nothrow) cdd_batch_s();
  if (!b) return CDD_ENOMEM;
  b->f_center = f_center_mhz;
  b->bandwidth = bandwidth_mhz;
  b->n_chan = n_chan;
  b->n_avg = n_avg;
  b->n_dm = n_dm;
  b->sideband = bandwidth_mhz > 0 ? 1 : -1;
  b->chan_bw = fabs(bandwidth_mhz) / n_chan;
  b->f_lo0 = f_center_mhz - fabs(bandwidth_mhz) / 2.0;             // the band's lowest edge
  b->f_base = b->sideband > 0 ? b->f_lo0 : f_center_mhz + fabs(bandwidth_mhz) / 2.0;
  b->dms.assign(dms, dms + n_dm);
  double dm_max = 0;
  for (double d : b->dms) {
    if (!(d >= 0) || !isfinite(d)) {
      delete b;
      return CDD_EINVAL;
    }
    dm_max = d > dm_max ? d : dm_max;
  }
  if (!(b->f_lo0 > 0)) {
    delete b;
    return CDD_EINVAL;
  }
  const int per = n_chan / n_tiers;
  int rc = CDD_OK;
  for (int t = 0; t < n_tiers && rc == CDD_OK; ++t) {
    cdd_batch_s::Tier tr;
    tr.n_fft = tier_nfft[t];
    // tiers run from the lowest frequencies up: the first channels of an upper
    // sideband, the last of a lower one
    tr.chan0 = b->sideband > 0 ? t * per : n_chan - (t + 1) * per;
    tr.n_tchan = per;
    // overlap: N/32, raised to the tier's lowest-channel smear at the largest DM,
    // rounded up to a multiple of n_avg
    const double f = b->sideband > 0 ? b->f_base + b->chan_bw * tr.chan0
                                     : b->f_base - b->chan_bw * (tr.chan0 + per);
    const double n_d = kDispDHost * dm_max * (pow(f, -2.0) - pow(f + b->chan_bw, -2.0)) * b->chan_bw * 1e6;
    long long ov = tr.n_fft / 32;
    if ((long long)ceil(n_d) > ov) ov = (long long)ceil(n_d);
    ov = (ov + n_avg - 1) / n_avg * n_avg;
    if (tr.n_fft < 64 || tr.n_fft > 16384 || (tr.n_fft & (tr.n_fft - 1))) rc = CDD_EUNSUPPORTED;
    else if (tr.n_fft <= ov || (tr.n_fft - ov) % n_avg) rc = CDD_EINVAL;
    tr.n_ov = (int)ov;
    tr.hop = tr.n_fft - tr.n_ov;
    while ((1 << tr.logn) < tr.n_fft) ++tr.logn;
    b->tiers.push_back(tr);
    if (tr.hop > b->hop_max) b->hop_max = tr.hop;
    if (tr.n_ov > b->n_ov_max) b->n_ov_max = tr.n_ov;
  }
  for (auto& t : b->tiers)
    if (rc == CDD_OK && b->hop_max % t.hop) rc = CDD_EINVAL;   // hops must nest
  if (rc == CDD_OK) {
    b->shift.resize((size_t)n_dm * n_chan);
    for (int d = 0; d < n_dm && rc == CDD_OK; ++d) {
      cdd::Geometry g{};
      g.f_lo0 = b->f_lo0;
      g.sideband = b->sideband;
      g.f_base = b->f_base;
      g.f_ref = b->f_lo0;
      g.chan_bw = b->chan_bw;
      g.dm = b->dms[d];
      g.n_avg = n_avg;
      for (int k = 0; k < n_chan; ++k) {
        const int64_t r = cdd::shift_of(g, k);
        if (r < 0) {
          rc = CDD_EINVAL;
          break;
        }
        b->shift[(size_t)d * n_chan + k] = r;
        if (r > b->r_max) b->r_max = r;
      }
    }
  }
  if (rc != CDD_OK) {
    delete b;
    return rc;
  }
  // default block: the shortest whole number of longest hops that outlasts every delay
  b->q = (int)((b->r_max * n_avg + b->hop_max - 1) / b->hop_max);
  if (b->q < 1) b->q = 1;
  if (n_out(b) < b->r_max) b->q += 1;
  *out = b;
  return CDD_OK;
}

int cdd_batch_set(cdd_batch b, int attr, int64_t value) {
  if (!b) return CDD_EINVAL;
  if (b->committed) return CDD_ESTATE;
  if (attr == CDD_ATTR_TAPER) {
    if (value < CDD_TAPER_NONE || value > CDD_TAPER_WELCH) return CDD_EINVAL;
    b->taper = (int)value;
    return CDD_OK;
  }
  if (attr == CDD_ATTR_BATCH_FORM) {
    if (value < -1 || value >= kForms) return CDD_EINVAL;
    b->form_req = (int)value;
    return CDD_OK;
  }
  if (attr != CDD_ATTR_SEGMENTS_PER_BLOCK) return CDD_EINVAL;
  if (value < 1 || value * b->hop_max * b->n_chan > ((int64_t)1 << 40)) return CDD_EINVAL;
  if (value * b->hop_max / b->n_avg < b->r_max) return CDD_EINVAL;
  for (auto& t : b->tiers)
    if ((int64_t)t.n_tchan * (value * b->hop_max / t.hop) >= ((int64_t)1 << 31)) return CDD_EINVAL;
  b->q = (int)value;
  return CDD_OK;
}

int cdd_batch_get(cdd_batch b, int attr, int64_t* v) {
  if (!b || !v) return CDD_EINVAL;
  switch (attr) {
    case CDD_ATTR_SEGMENTS_PER_BLOCK: *v = b->q; break;
    case CDD_ATTR_BLOCK_SAMPLES: *v = block_samples(b); break;
    case CDD_ATTR_N_OUT_PER_BLOCK: *v = n_out(b); break;
    case CDD_ATTR_R_MAX: *v = b->r_max; break;
    case CDD_ATTR_BYTES_DEVICE: *v = (int64_t)b->bytes_device; break;
    case CDD_ATTR_BLOCKS_DONE: *v = b->blocks; break;
    case CDD_ATTR_KERNEL_LAUNCHES: *v = b->last_launches; break;
    case CDD_ATTR_PHASE_FLOATS: *v = max_phase_turns(b) <= kT1SingleTurns ? 1 : 2; break;
    case CDD_ATTR_N_CHAN: *v = b->n_chan; break;
    case CDD_ATTR_N_AVG: *v = b->n_avg; break;
    case CDD_ATTR_HOP: *v = b->hop_max; break;
    case CDD_ATTR_TAPER: *v = b->taper; break;
    case CDD_ATTR_BATCH_FORM: *v = b->form >= 0 ? b->form : b->form_req; break;
    case CDD_ATTR_TUNE_NS_TIERS: *v = b->tune_ns[kFormTiers]; break;
    case CDD_ATTR_TUNE_NS_TIERS_NP: *v = b->tune_ns[kFormTiersNP]; break;
    case CDD_ATTR_TUNE_NS_MULTI: *v = b->tune_ns[kFormMulti]; break;
    default: return CDD_EINVAL;
  }
  return CDD_OK;
}

int cdd_batch_tier(cdd_batch b, int t, int64_t* n_fft, int64_t* n_ov, int64_t* chan0,
                   int64_t* n_tchan) {
  if (!b || t < 0 || t >= (int)b->tiers.size()) return CDD_EINVAL;
  const auto& tr = b->tiers[t];
  if (n_fft) *n_fft = tr.n_fft;
  if (n_ov) *n_ov = tr.n_ov;
  if (chan0) *chan0 = tr.chan0;
  if (n_tchan) *n_tchan = tr.n_tchan;
  return CDD_OK;
}

int cdd_batch_shifts(cdd_batch b, int64_t* shifts) {
  if (!b || !shifts) return CDD_EINVAL;
  memcpy(shifts, b->shift.data(), b->shift.size() * sizeof(int64_t));
  return CDD_OK;
}

int cdd_batch_execute(cdd_batch b, const int8_t* d_in, float* d_out, cudaStream_t stream) {
  if (!b || !d_in || !d_out) return CDD_EINVAL;
  int rc = bprepare(b);
  if (rc) return rc;
  const int64_t rows = block_samples(b);
  BTRY(b, cdd::launch_corner_turn(reinterpret_cast<const char2*>(d_in), b->d_in_cm, 0, rows, rows,
                                  b->n_chan, stream));
  std::vector<cdd::BatchArgs> args;
  for (auto& t : b->tiers) {
    cdd::BatchArgs a;
    a.in_cm = b->d_in_cm;
    a.rows = rows;
    a.out = d_out;
    a.t1 = t.d_t1;
    a.t1f = t.d_t1f;
    a.taper = t.d_taper;
    a.tw = t.d_tw;
    a.tail_rd = b->d_tail[b->parity];
    a.tail_wr = b->d_tail[b->parity ^ 1];
    a.ring_rd = b->d_ring[b->parity];
    a.ring_wr = b->d_ring[b->parity ^ 1];
    a.shift = b->d_shift;
    a.dms = b->d_dms;
    a.xs = b->d_xs;
    a.n_chan = b->n_chan;
    a.chan0 = t.chan0;
    a.n_tchan = t.n_tchan;
    a.n_ov = t.n_ov;
    a.hop = t.hop;
    a.n_avg = b->n_avg;
    a.q = (int)(rows / t.hop);
    a.n_out = (int)n_out(b);
    a.n_dm = b->n_dm;
    a.r_max = (int)(b->r_max > 0 ? b->r_max : 1);
    a.tail_stride = b->n_ov_max > 0 ? b->n_ov_max : 1;
    a.persistent = 1;
    args.push_back(a);
  }
  // TIERS and MULTI compute each (channel, segment, DM) with the same
  // arithmetic and write the same outputs, tails and carried outputs; only
  // the launch shape differs.  The first execute of an untuned batch runs
  // each once on this block, times it with CUDA events and keeps the fastest
  // (the last run's writes are the block's result).
  auto run = [&](int form) -> int {
    if (form == kFormMulti) {
      cdd::MultiArgs m = {};
      std::vector<int> order(args.size());
      for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
      std::stable_sort(order.begin(), order.end(),
                       [&](int x, int y) { return b->tiers[x].logn > b->tiers[y].logn; });   // longest first
      for (size_t i = 0; i < order.size(); ++i) {
        m.tier[i] = args[order[i]];
        m.logn[i] = b->tiers[order[i]].logn;
      }
      m.n_tiers = (int)order.size();
      m.counters = b->d_counters;
      m.slots = b->d_slots;
      BTRY(b, cdd::launch_multi(m, b->t1_single, b->taper != CDD_TAPER_NONE, b->multi_grid, stream));
      return CDD_OK;
    }
    for (size_t i = 0; i < args.size(); ++i) {
      args[i].persistent = form == kFormTiers ? 1 : 0;
      BTRY(b, cdd::launch_batch(b->tiers[i].logn, args[i], stream));
    }
    return CDD_OK;
  };
  if (b->form_req == kFormMulti && !b->multi_ok) return CDD_EUNSUPPORTED;
  if (b->form < 0) {
    const int key_form = b->form_req >= 0 ? b->form_req : cached_form(b);
    if (key_form >= 0) {
      b->form = key_form;
    } else {
      cudaEvent_t ev[2];
      BTRY(b, cudaEventCreate(&ev[0]));
      BTRY(b, cudaEventCreate(&ev[1]));
      int best = -1;
      float best_ms = 0;
      // TIERS and MULTI give the same bits, so a stream's output does not
      // depend on which one the timing picked; TIERS_NP rounds the N = 8192
      // tier's first-pass twiddles differently and is only run on request
      for (int f = 0; f < kForms; ++f) {
        if (f == kFormTiersNP || (f == kFormMulti && !b->multi_ok)) continue;
        BTRY(b, cudaEventRecord(ev[0], stream));
        if ((rc = run(f))) return rc;
        BTRY(b, cudaEventRecord(ev[1], stream));
        BTRY(b, cudaEventSynchronize(ev[1]));
        float ms = 0;
        BTRY(b, cudaEventElapsedTime(&ms, ev[0], ev[1]));
        b->tune_ns[f] = llround((double)ms * 1e6);
        if (best < 0 || ms < best_ms) {
          best = f;
          best_ms = ms;
        }
      }
      cudaEventDestroy(ev[0]);
      cudaEventDestroy(ev[1]);
      b->form = best;
      remember_form(b, best);
      b->parity ^= 1;
      b->blocks += 1;
      b->last_launches = 1 + launches_of(b, best);
      return CDD_OK;
    }
  }
  if ((rc = run(b->form))) return rc;
  b->parity ^= 1;
  b->blocks += 1;
  b->last_launches = 1 + launches_of(b, b->form);
  return CDD_OK;
}

}  // extern "C"

namespace {

struct BatchStateHeader {
  uint32_t magic, version;
  int32_t n_chan, n_dm, n_tiers, n_avg, q, tail_stride, taper, reserved;
  int64_t r_max, hop_max, blocks;
  double f_center, bandwidth;
  uint64_t lists;                            // hash of the DM list and the tiers
};
constexpr uint32_t kBatchStateMagic = 0x42444453u;   // "SDDB"
constexpr uint32_t kBatchStateVersion = 1;

size_t batch_tail_bytes(const cdd_batch b) {
  return (size_t)b->n_chan * (b->n_ov_max > 0 ? b->n_ov_max : 1) * sizeof(char2);
}
size_t batch_ring_bytes(const cdd_batch b) {
  return (size_t)b->n_dm * b->n_chan * (b->r_max > 0 ? b->r_max : 1) * sizeof(float);
}
int64_t batch_state_bytes(const cdd_batch b) {
  return (int64_t)(sizeof(BatchStateHeader) + batch_tail_bytes(b) + batch_ring_bytes(b));
}

// FNV-1a over the bytes of the DM list and each tier's N and overlap
uint64_t batch_lists_hash(const cdd_batch b) {
  uint64_t h = 1469598103934665603ull;
  auto add = [&](const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
  };
  add(b->dms.data(), b->dms.size() * sizeof(double));
  for (const auto& t : b->tiers) {
    add(&t.n_fft, sizeof(t.n_fft));
    add(&t.n_ov, sizeof(t.n_ov));
  }
  return h;
}

BatchStateHeader batch_header(const cdd_batch b) {
  BatchStateHeader h = {};
  h.magic = kBatchStateMagic;
  h.version = kBatchStateVersion;
  h.n_chan = b->n_chan;
  h.n_dm = b->n_dm;
  h.n_tiers = (int32_t)b->tiers.size();
  h.n_avg = b->n_avg;
  h.q = b->q;
  h.tail_stride = b->n_ov_max > 0 ? b->n_ov_max : 1;
  h.taper = b->taper;
  h.r_max = b->r_max;
  h.hop_max = b->hop_max;
  h.f_center = b->f_center;
  h.bandwidth = b->bandwidth;
  h.lists = batch_lists_hash(b);
  return h;
}

bool same_batch_geometry(const BatchStateHeader& a, const BatchStateHeader& c) {
  return a.magic == c.magic && a.version == c.version && a.n_chan == c.n_chan && a.n_dm == c.n_dm &&
         a.n_tiers == c.n_tiers && a.n_avg == c.n_avg && a.q == c.q && a.tail_stride == c.tail_stride &&
         a.taper == c.taper &&
         a.r_max == c.r_max && a.hop_max == c.hop_max && a.f_center == c.f_center &&
         a.bandwidth == c.bandwidth && a.lists == c.lists;
}

}  // namespace

extern "C" {

int cdd_batch_state_bytes(cdd_batch b, int64_t* bytes) {
  if (!b || !bytes) return CDD_EINVAL;
  *bytes = batch_state_bytes(b);
  return CDD_OK;
}

int cdd_batch_export_state(cdd_batch b, void* state, int64_t bytes, cudaStream_t s) {
  if (!b || !state || bytes < batch_state_bytes(b)) return CDD_EINVAL;
  if (b->sticky) return b->sticky;
  BatchStateHeader h = batch_header(b);
  char* out = static_cast<char*>(state);
  const size_t tb = batch_tail_bytes(b), rb = batch_ring_bytes(b);
  if (!b->committed) {                       // a fresh stream: zero history
    h.blocks = 0;
    memcpy(out, &h, sizeof(h));
    memset(out + sizeof(h), 0, tb + rb);
    return CDD_OK;
  }
  int dev = -1;
  BTRY(b, cudaGetDevice(&dev));
  if (dev != b->device) return CDD_EINVAL;
  BTRY(b, cudaStreamSynchronize(s));
  h.blocks = b->blocks;
  memcpy(out, &h, sizeof(h));
  BTRY(b, cudaMemcpy(out + sizeof(h), b->d_tail[b->parity], tb, cudaMemcpyDeviceToHost));
  BTRY(b, cudaMemcpy(out + sizeof(h) + tb, b->d_ring[b->parity], rb, cudaMemcpyDeviceToHost));
  return CDD_OK;
}

int cdd_batch_import_state(cdd_batch b, const void* state, int64_t bytes, cudaStream_t s) {
  if (!b || !state || bytes < batch_state_bytes(b)) return CDD_EINVAL;
  BatchStateHeader h;
  memcpy(&h, state, sizeof(h));
  if (!same_batch_geometry(h, batch_header(b)) || h.blocks < 0) return CDD_EINVAL;
  int rc = bprepare(b);
  if (rc) return rc;
  BTRY(b, cudaStreamSynchronize(s));
  const char* in = static_cast<const char*>(state) + sizeof(h);
  const size_t tb = batch_tail_bytes(b), rb = batch_ring_bytes(b);
  BTRY(b, cudaMemcpy(b->d_tail[0], in, tb, cudaMemcpyHostToDevice));
  BTRY(b, cudaMemcpy(b->d_ring[0], in + tb, rb, cudaMemcpyHostToDevice));
  b->parity = 0;
  b->blocks = h.blocks;
  return CDD_OK;
}

int cdd_batch_reset(cdd_batch b) {
  if (!b) return CDD_EINVAL;
  if (b->sticky) return b->sticky;
  if (!b->committed) {
    b->parity = 0;
    b->blocks = 0;
    return CDD_OK;
  }
  BTRY(b, cudaDeviceSynchronize());
  cudaStream_t s;
  BTRY(b, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  const int rc = bzero_state(b, s);
  const cudaError_t e = cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (rc) return rc;
  return bfail(b, e);
}

int cdd_batch_destroy(cdd_batch b) {
  if (!b) return CDD_OK;
  if (b->device >= 0) {
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    bfree(b);
    if (prev >= 0) cudaSetDevice(prev);
  }
  delete b;
  return CDD_OK;
}

}  // extern "C"
