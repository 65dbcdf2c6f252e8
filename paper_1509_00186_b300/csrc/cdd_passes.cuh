// cdd_passes.cuh -- device building blocks of the fused overlap-save kernels:
// launch shape per transform length, the in-place radix passes in shared
// memory, the chirp pass, and the int8 unpack.  Included by cdd_kernels.cu and
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
#ifdef CDD_OLS_MINB
  static constexpr int MINB = THREADS <= 256 ? CDD_OLS_MINB : 1;          // CTAs per SM to aim for
#else
  static constexpr int MINB = THREADS <= 256 ? 2 : 1;
#endif
  static constexpr int SEG_F2 = padded_len(PL::N);                       // float2 per transform
  static constexpr size_t SMEM = size_t(G) * SEG_F2 * sizeof(float2);
};

// pad(base + S*j) - pad(base) for the index sets the passes touch (S >= 16, or
// base mod 16 < S with S dividing 16): a compile-time constant.
template <int S>
__device__ __forceinline__ constexpr int poff(int j) { return S * j + ((S * j) >> 4); }

// int8 pair (re, im) held in the low 16 bits -> float2 without I2F: bias each
// byte to unsigned, drop it into the mantissa of 2^23 and subtract 2^23 + 128
// (exact for every int8 value).
__device__ __forceinline__ float2 unpack_i8x2(uint32_t raw16) {
  const uint32_t w = raw16 ^ 0x8080u;
  const float re = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540)) - 8388736.0f;
  const float im = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7541)) - 8388736.0f;
  return make_float2(re, im);
}

// A twiddle from global memory (read-only path) or from a copy in shared
// memory; the read-only load must never see a shared-memory address.
template <bool SH>
__device__ __forceinline__ float2 ld_tw(const float2* p) {
  if constexpr (SH) return *p;
  else return __ldg(p);
}

// Forward (DIF) radix pass p, in place in shared memory; SH: tw is in shared memory.
template <int LOGN, int p, bool SH = false>
__device__ __forceinline__ void fwd_pass(float2* buf, const float2* __restrict__ tw, int lt) {
  using PL = PassPlan<LOGN>;
  constexpr int R = PL::R(p), S = PL::S(p), M = PL::M(p);
  constexpr int PER = (PL::N / R) / PL::T;
#pragma unroll kPassUnroll
  for (int i = 0; i < PER; ++i) {
    const int b = lt + i * PL::T;
    const int t = b % S;
    const int base = (b / S) * M + t;
    float2* pb = buf + pad(base);
    float2 v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = pb[poff<S>(j)];
    dft<R, -1>(v);
    if constexpr (S > 1) {
      const float2* twp = tw + PL::TwOff(p) + t;
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmul(v[k], ld_tw<SH>(twp + k * S));
    }
#pragma unroll
    for (int k = 0; k < R; ++k) pb[poff<S>(k)] = v[k];
  }
}

// Inverse (DIT) radix pass p, in place: conjugate twiddle, then butterfly.
template <int LOGN, int p, bool SH = false>
__device__ __forceinline__ void inv_pass(float2* buf, const float2* __restrict__ tw, int lt) {
  using PL = PassPlan<LOGN>;
  constexpr int R = PL::R(p), S = PL::S(p), M = PL::M(p);
  constexpr int PER = (PL::N / R) / PL::T;
#pragma unroll kPassUnroll
  for (int i = 0; i < PER; ++i) {
    const int b = lt + i * PL::T;
    const int t = b % S;
    const int base = (b / S) * M + t;
    float2* pb = buf + pad(base);
    float2 v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = pb[poff<S>(k)];
    if constexpr (S > 1) {
      const float2* twp = tw + PL::TwOff(p) + t;
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmulc(v[k], ld_tw<SH>(twp + k * S));
    }
    dft<R, 1>(v);
#pragma unroll
    for (int j = 0; j < R; ++j) pb[poff<S>(j)] = v[j];
  }
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
    float2* pb = buf + pad(q * R);
    float2 v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = pb[j];
    dft<R, -1>(v);
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = cmul(v[k], __ldg(&chirp_k[k * NG + q]));
    dft<R, 1>(v);
#pragma unroll
    for (int j = 0; j < R; ++j) pb[j] = v[j];
  }
}

}  // namespace passes
}  // namespace cdd
