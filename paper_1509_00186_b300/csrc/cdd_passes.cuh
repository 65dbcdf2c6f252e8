// cdd_passes.cuh -- device building blocks of the fused overlap-save kernels:
// launch shape per transform length, the in-place radix passes in shared
// memory, the chirp pass, the int8 unpack, and detection with integration in
// registers across lanes.  Included by cdd_kernels.cu and
// cdd_batch.cu.
#pragma once

#include "cdd_fft.cuh"

namespace cdd {
namespace passes {

constexpr double kDispD = 4.148808e3;   // s MHz^2 cm^3 / pc (Eq. 3)

// Butterflies per thread in a pass are looped, not unrolled, by default: the
// fully unrolled passes overflow the instruction cache.
#ifndef CDD_PASS_UNROLL
#define CDD_PASS_UNROLL 1
#endif
constexpr int kPassUnroll = CDD_PASS_UNROLL;
constexpr int kMinCtaThreads = 256;

template <int LOGN>
struct Cfg {
  using PL = PassPlan<LOGN>;
  static constexpr int T = PL::T;
  static constexpr int G = T >= kMinCtaThreads ? 1 : kMinCtaThreads / T;   // transforms per CTA
  static constexpr int THREADS = G * T;
  // CTAs per SM to aim for: three 256-thread CTAs (80 registers) where a
  // thread's largest radix is 16, two where it is 32 (three would spill)
#ifdef CDD_OLS_MINB
  static constexpr int MINB = THREADS <= 256 ? CDD_OLS_MINB : 1;
#else
  static constexpr int MINB = THREADS <= 256 ? (PL::R(0) <= 16 ? 3 : 2) : 1;
#endif
  static constexpr int SEG_F2 = padded_len<LOGN>();                       // float2 per transform
  static constexpr size_t SMEM = size_t(G) * SEG_F2 * sizeof(float2);
};

// pad<LOGN>(base + S*j) - pad<LOGN>(base) for the index sets the passes touch
// (S >= 16, or base mod 16 < S with S dividing 16): a compile-time constant.
template <int LOGN, int S>
__device__ __forceinline__ constexpr int poff(int j) { return S * j + pad_words<LOGN>() * ((S * j) >> 4); }

// A stride-1 group of R points at buf + pad<LOGN>(q * R) to and from
// registers.  With two pad words per 16 points every group starts on a
// 16-byte boundary (buffers start on one), so it moves as R/2 128-bit accesses.
template <int LOGN, int R>
__device__ __forceinline__ void load_group(const float2* pb, float2 (&v)[R]) {
  if constexpr (pad_words<LOGN>() == 2 && R % 2 == 0) {
#pragma unroll
    for (int j = 0; j < R; j += 2) {
      const float4 t = reinterpret_cast<const float4*>(pb)[j / 2];
      v[j] = make_float2(t.x, t.y);
      v[j + 1] = make_float2(t.z, t.w);
    }
  } else {
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = pb[j];
  }
}
template <int LOGN, int R>
__device__ __forceinline__ void store_group(float2* pb, const float2 (&v)[R]) {
  if constexpr (pad_words<LOGN>() == 2 && R % 2 == 0) {
#pragma unroll
    for (int j = 0; j < R; j += 2)
      reinterpret_cast<float4*>(pb)[j / 2] = make_float4(v[j].x, v[j].y, v[j + 1].x, v[j + 1].y);
  } else {
#pragma unroll
    for (int j = 0; j < R; ++j) pb[j] = v[j];
  }
}

// int8 pair (re, im) held in the low 16 bits -> float2 without I2F: bias each
// byte to unsigned, drop it into the mantissa of 2^23 and subtract 2^23 + 128
// (exact for every int8 value; one packed subtraction for both halves).
__device__ __forceinline__ float2 unpack_i8x2(uint32_t raw16) {
  const uint32_t w = raw16 ^ 0x8080u;
  const float re = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540));
  const float im = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7541));
  return sub2(make_float2(re, im), make_float2(8388736.0f, 8388736.0f));
}

// Bulk prefetch of [p, p + bytes) into L2 (p and bytes multiples of 16; the
// range must lie inside one allocation).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// A twiddle from global memory (read-only path) or from a copy in shared
// memory; the read-only load must never see a shared-memory address.
template <bool SH>
__device__ __forceinline__ float2 ld_tw(const float2* p) {
  if constexpr (SH) return *p;
  else return __ldg(p);
}

// Twiddles k = 1 .. R-1 of slot t formed from four table loads (k = 1 and the
// multiples of 8) and products with w^1 in between: at most 7 products deep.
// Used where the table is too large for L1 and its loads wait on L2.
template <int R, int S, bool SH, bool CONJ>
__device__ __forceinline__ void apply_twiddles_rec(float2 (&v)[R], const float2* twp) {
  const float2 w1 = ld_tw<SH>(twp + S);
  float2 w = w1;
#pragma unroll
  for (int k = 1; k < R; ++k) {
    if (k > 1) w = (k % 8 == 0) ? ld_tw<SH>(twp + k * S) : cmul(w, w1);
    v[k] = CONJ ? cmulc(v[k], w) : cmul(v[k], w);
  }
}

// Pass 0 of a radix-32 plan of N >= 8192 points read from global memory: its
// table (31 twiddles per slot, 62 KB and more) does not stay in L1 beside the
// transform buffers, so its twiddles are formed as products (apply_twiddles_rec).
template <int LOGN, bool SH>
constexpr bool kRecPass0 = !SH && LOGN >= 13 && PassPlan<LOGN>::R(0) == 32;

// Forward (DIF) radix pass p, in place in shared memory; SH: tw is in shared memory.
template <int LOGN, int p, bool SH = false, bool REC = false>
__device__ __forceinline__ void fwd_pass(float2* buf, const float2* __restrict__ tw, int lt) {
  using PL = PassPlan<LOGN>;
  constexpr int R = PL::R(p), S = PL::S(p), M = PL::M(p);
  constexpr int PER = (PL::N / R) / PL::T;
#pragma unroll kPassUnroll
  for (int i = 0; i < PER; ++i) {
    const int b = lt + i * PL::T;
    const int t = b % S;
    const int base = (b / S) * M + t;
    float2* pb = buf + pad<LOGN>(base);
    float2 v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = pb[poff<LOGN, S>(j)];
    dft<R, -1>(v);
    if constexpr (S > 1 && REC) {
      apply_twiddles_rec<R, S, SH, false>(v, tw + PL::TwOff(p) + t);
    } else if constexpr (S > 1) {
      const float2* twp = tw + PL::TwOff(p) + t;
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmul(v[k], ld_tw<SH>(twp + k * S));
    }
#pragma unroll
    for (int k = 0; k < R; ++k) pb[poff<LOGN, S>(k)] = v[k];
  }
}

// Inverse (DIT) radix pass p, in place: conjugate twiddle, then butterfly.
template <int LOGN, int p, bool SH = false, bool REC = false>
__device__ __forceinline__ void inv_pass(float2* buf, const float2* __restrict__ tw, int lt) {
  using PL = PassPlan<LOGN>;
  constexpr int R = PL::R(p), S = PL::S(p), M = PL::M(p);
  constexpr int PER = (PL::N / R) / PL::T;
#pragma unroll kPassUnroll
  for (int i = 0; i < PER; ++i) {
    const int b = lt + i * PL::T;
    const int t = b % S;
    const int base = (b / S) * M + t;
    float2* pb = buf + pad<LOGN>(base);
    float2 v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = pb[poff<LOGN, S>(k)];
    if constexpr (S > 1 && REC) {
      apply_twiddles_rec<R, S, SH, true>(v, tw + PL::TwOff(p) + t);
    } else if constexpr (S > 1) {
      const float2* twp = tw + PL::TwOff(p) + t;
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmulc(v[k], ld_tw<SH>(twp + k * S));
    }
    dft<R, 1>(v);
#pragma unroll
    for (int j = 0; j < R; ++j) pb[poff<LOGN, S>(j)] = v[j];
  }
}

#ifndef CDD_CHIRP_PAIRS
#define CDD_CHIRP_PAIRS 1
#endif
// Chirp-table index idx of a row -> (k, q): bin k of stride-1 group q.  With
// CDD_CHIRP_PAIRS the bins k and k + 1 (k even) of a group are adjacent, so
// the chirp pass loads them as one 16-byte value.
template <int NG>
__host__ __device__ constexpr int chirp_pos(int idx, int rl) {
#if CDD_CHIRP_PAIRS
  return ((idx >> 1) % NG) * rl + 2 * ((idx >> 1) / NG) + (idx & 1);
#else
  return (idx % NG) * rl + idx / NG;
#endif
}

// Last forward radix, chirp multiply, first inverse radix (stride-1 groups).
template <int LOGN>
__device__ __forceinline__ void chirp_pass(float2* buf, const float2* __restrict__ chirp_k, int lt) {
  using PL = PassPlan<LOGN>;
  constexpr int R = PL::RL;
  constexpr int NG = PL::N / R;
  constexpr int PER = NG / PL::T;
#pragma unroll kPassUnroll
  for (int i = 0; i < PER; ++i) {
    const int q = lt + i * PL::T;
    static_assert(R <= 16, "stride-1 groups must not cross a padding word");
    float2* pb = buf + pad<LOGN>(q * R);
    float2 v[R];
    load_group<LOGN, R>(pb, v);
    dft<R, -1>(v);
#if CDD_CHIRP_PAIRS
    // bins k and k + 1 (k even) of group q share one 16-byte table entry
    static_assert(R % 2 == 0, "paired chirp entries need an even last radix");
#pragma unroll
    for (int k = 0; k < R; k += 2) {
      const float4 c = __ldg(reinterpret_cast<const float4*>(chirp_k) + (k / 2) * NG + q);
      v[k] = cmul(v[k], make_float2(c.x, c.y));
      v[k + 1] = cmul(v[k + 1], make_float2(c.z, c.w));
    }
#else
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = cmul(v[k], __ldg(&chirp_k[k * NG + q]));
#endif
    dft<R, 1>(v);
    store_group<LOGN, R>(pb, v);
  }
}

// Window sums over groups of NA neighbouring lanes by recursive halving: at
// each step a lane keeps one half of its V values, adds its partner's copy of
// that half and sends the other half.  Afterwards lane l holds, in u[i]
// (i < R0/NA), the sum over its lane group of the values it started with at
// index j = (R0/NA) * (l mod NA) + i.
template <int R0, int NA, int V = R0>
__device__ __forceinline__ void lane_window_sums(float (&u)[R0], int lane) {
  if constexpr (NA > 1) {
    constexpr int o = NA / 2, H = V / 2;
    const bool hi = (lane & o) != 0;
    if constexpr (H % 2 == 0) {                  // two sums per packed addition
#pragma unroll
      for (int i = 0; i < H; i += 2) {
        const float2 keep = hi ? make_float2(u[i + H], u[i + H + 1]) : make_float2(u[i], u[i + 1]);
        const float s0 = hi ? u[i] : u[i + H], s1 = hi ? u[i + 1] : u[i + H + 1];
        const float2 got = make_float2(__shfl_xor_sync(0xffffffffu, s0, o), __shfl_xor_sync(0xffffffffu, s1, o));
        const float2 sum = add2(keep, got);
        u[i] = sum.x;
        u[i + 1] = sum.y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < H; ++i) {
        const float keep = hi ? u[i + H] : u[i];
        const float send = hi ? u[i] : u[i + H];
        u[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
    lane_window_sums<R0, NA / 2, H>(u, lane);
  }
}

// Detect and integrate the R0 samples n = lt + T*j (j < R0) a thread holds
// after the last inverse pass: windows of NA samples are NA neighbouring lanes
// (T is a multiple of 32 and windows start at multiples of NA), so a window's
// sum is formed in registers.  emit(m, sum) receives output m of the segment,
// the window starting at n_ov + m*NA.
template <int R0, int T, int NA, class Emit>
__device__ __forceinline__ void lane_windows(const float2 (&v)[R0], int lt, int n_ov, Emit& emit) {
  static_assert(T % 32 == 0 && NA <= 32 && NA <= R0, "window must be lanes of one warp");
  float u[R0];
#pragma unroll
  for (int j = 0; j < R0; ++j) u[j] = fmaf(v[j].x, v[j].x, v[j].y * v[j].y);
  const int lane = lt & 31;
  lane_window_sums<R0, NA>(u, lane);
  constexpr int V = R0 / NA;
  const int first = lt - (lane & (NA - 1));      // first lane's sample of the window
#pragma unroll
  for (int i = 0; i < V; ++i) {
    const int j = V * (lane & (NA - 1)) + i;
    const int n0 = first + T * j;
    if (n0 >= n_ov) emit((n0 - n_ov) / NA, u[i]);
  }
}

template <int R0, int T, class Emit>
__device__ __forceinline__ void integrate_in_lanes(const float2 (&v)[R0], int lt, int n_ov, int na,
                                                   Emit& emit) {
  switch (na) {
    case 1: lane_windows<R0, T, 1>(v, lt, n_ov, emit); break;
    case 2: lane_windows<R0, T, 2>(v, lt, n_ov, emit); break;
    case 4: lane_windows<R0, T, 4>(v, lt, n_ov, emit); break;
    case 8: lane_windows<R0, T, 8>(v, lt, n_ov, emit); break;
    case 16:
      if constexpr (R0 >= 16) lane_windows<R0, T, 16>(v, lt, n_ov, emit);
      break;
    case 32:
      if constexpr (R0 >= 32) lane_windows<R0, T, 32>(v, lt, n_ov, emit);
      break;
    default: break;
  }
}

}  // namespace passes
}  // namespace cdd
