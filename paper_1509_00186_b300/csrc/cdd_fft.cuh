// cdd_fft.cuh -- in-register DFT butterflies and the mixed-radix pass plan used
// by the fused overlap-save kernel.
//
// A length-N transform (N = 2^LOGN) runs as P radix passes with radices
// R_0 >= ... (all powers of two, product N).  Pass p works on sub-problems of
// size M_p = N / (R_0 ... R_{p-1}) and gathers its R_p points at stride
// S_p = M_p / R_p.  The forward transform is decimation in frequency (natural
// order in, digit-reversed order out); the inverse is decimation in time on
// the same index sets (digit-reversed in, natural out), so the spectrum is
// never reordered: the chirp is applied in digit-reversed order with a table
// stored in that order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace cdd {

// ------------------------------------------------------------ complex helpers

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// a * w
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
  return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
// a * conj(w)
__device__ __forceinline__ float2 cmulc(float2 a, float2 w) {
  return make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y));
}

// cos(2*pi*k/32) for any integer k, exact to float rounding: the values are
// cos(pi*m/16), m = 0..8.
__host__ __device__ constexpr float cos32(int k) {
  constexpr float c[9] = {1.0f,
                          0.98078528040323044913f,
                          0.92387953251128675613f,
                          0.83146961230254523708f,
                          0.70710678118654752440f,
                          0.55557023301960222474f,
                          0.38268343236508977173f,
                          0.19509032201612826785f,
                          0.0f};
  int m = ((k % 32) + 32) % 32;
  return m <= 8 ? c[m] : m <= 16 ? -c[16 - m] : m <= 24 ? -c[m - 16] : c[32 - m];
}
__host__ __device__ constexpr float sin32(int k) { return cos32(k - 8); }

// Compile-time loop: f(std::integral_constant<int, I>) for I = B .. E-1.
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// b * exp(DIR * 2*pi*i * J / LEN), LEN <= 32; the rotation is a compile-time
// constant, and rotations by 1 and +-i cost no multiplication.
template <int LEN, int DIR, int J>
__device__ __forceinline__ float2 rot(float2 b) {
  constexpr int m = J * (32 / LEN);       // angle in units of 2*pi/32
  if constexpr (m == 0) {
    return b;
  } else if constexpr (m == 8) {
    return DIR > 0 ? make_float2(-b.y, b.x) : make_float2(b.y, -b.x);
  } else {
    constexpr float c = cos32(m);
    constexpr float s = DIR > 0 ? sin32(m) : -sin32(m);
    return make_float2(fmaf(b.x, c, -b.y * s), fmaf(b.x, s, b.y * c));
  }
}

// The same angles in double, for compile-time constants derived from them.
__host__ __device__ constexpr double cos32d(int k) {
  constexpr double c[9] = {1.0,
                           0.98078528040323044913,
                           0.92387953251128675613,
                           0.83146961230254523708,
                           0.70710678118654752440,
                           0.55557023301960222474,
                           0.38268343236508977173,
                           0.19509032201612826785,
                           0.0};
  int m = ((k % 32) + 32) % 32;
  return m <= 8 ? c[m] : m <= 16 ? -c[16 - m] : m <= 24 ? -c[m - 16] : c[32 - m];
}

// Packed two-lane FP32 (add/sub/fma.rn.f32x2, sm_100 and later): one
// instruction applies the operation to both halves of a float2, each half
// rounded as the scalar instruction would round it, so results are bit for
// bit those of the scalar form.  CDD_PACKED selects which radix-2 butterflies
// use it: 1 those without a multiplication (a +- b), 2 also the final a +- f u
// of the butterflies with a general rotation (two more register pairs of
// constants).  A translation unit may set it before including this header.
#ifndef CDD_PACKED
#define CDD_PACKED 2
#endif
__device__ __forceinline__ unsigned long long f2_pack(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(r);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(r);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(r);
}
// a * b + c on both halves
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)), "l"(f2_pack(c)));
  return f2_unpack(r);
}

// Radix-2 butterfly (a, b) -> (a + w b, a - w b), w = exp(DIR * 2*pi*i * J / LEN).
// For a non-trivial w = c + i s the product is factored through the larger of
// |c| and |s|: w b = c (b + i (s/c) b) or w b = s ((c/s) b + i b), so that the
// butterfly is two fused multiply-adds for the inner factor and four for
// a +- c u (six lane operations instead of four for the product and four
// adds; with CDD_PACKED >= 2 the last four issue as two packed instructions).
// The ratio is at most 1 in magnitude, so no intermediate grows.  w = +-i
// stays scalar: its packed form needs (b.y, b.x) in a register pair, and the
// moves that build it cost what the packing saves.
template <int LEN, int DIR, int J>
__device__ __forceinline__ void bfly(float2& a, float2& b) {
  constexpr int m = J * (32 / LEN);       // angle in units of 2*pi/32
  if constexpr (m == 0 && CDD_PACKED >= 1) {
    const float2 d = sub2(a, b);
    a = add2(a, b);
    b = d;
  } else if constexpr (m == 0 || m == 8) {
    const float2 w = rot<LEN, DIR, J>(b);
    b = csub(a, w);
    a = cadd(a, w);
  } else {
    constexpr double cd = cos32d(m);
    constexpr double sd = DIR > 0 ? cos32d(m - 8) : -cos32d(m - 8);
    constexpr bool by_c = (cd < 0 ? -cd : cd) >= (sd < 0 ? -sd : sd);
    // b' = b * (w / f): by_c: f = c, b' = (b.x - r b.y, b.y + r b.x), r = s/c;
    //                   else: f = s, b' = (r b.x - b.y, b.x + r b.y), r = c/s.
    constexpr float f = (float)(by_c ? cd : sd);
    constexpr float r = (float)(by_c ? sd / cd : cd / sd);
    float ux, uy;
    if constexpr (by_c) {
      ux = fmaf(-r, b.y, b.x);
      uy = fmaf(r, b.x, b.y);
    } else {
      ux = fmaf(r, b.x, -b.y);
      uy = fmaf(r, b.y, b.x);
    }
    if constexpr (CDD_PACKED >= 2) {
      const float2 u = make_float2(ux, uy);
      b = fma2(make_float2(-f, -f), u, a);
      a = fma2(make_float2(f, f), u, a);
    } else {
      b = make_float2(fmaf(-f, ux, a.x), fmaf(-f, uy, a.y));
      a = make_float2(fmaf(f, ux, a.x), fmaf(f, uy, a.y));
    }
  }
}

template <int R>
__host__ __device__ constexpr int bitrev(int i) {
  int r = 0;
  for (int b = 1, o = R >> 1; b < R; b <<= 1, o >>= 1)
    if (i & b) r |= o;
  return r;
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

// In-place DFT of R (2..32) points held in registers, natural order in and
// out.  DIR = -1: X[k] = sum_n x[n] e^{-2 pi i kn/R};  DIR = +1: the same with
// e^{+...} and no 1/R.  Radix-2 decimation in time on bit-reversed input.
template <int R, int DIR>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
  float2 t[R];
  static_for<0, R>([&](auto I) {
    constexpr int i = decltype(I)::value;
    t[bitrev<R>(i)] = v[i];
  });
  static_for<1, ilog2(R) + 1>([&](auto L) {
    constexpr int len = 1 << decltype(L)::value;
    static_for<0, R / len>([&](auto G) {
      static_for<0, len / 2>([&](auto J) {
        constexpr int i = decltype(G)::value * len;
        constexpr int j = decltype(J)::value;
        bfly<len, DIR, j>(t[i + j], t[i + j + len / 2]);
      });
    });
  });
#pragma unroll
  for (int i = 0; i < R; ++i) v[i] = t[i];
}

// ------------------------------------------------------------ pass plan

// log2 of the radix of pass p for a length-2^LOGN transform (0 past the end).
// The first pass always has the largest radix, so a thread owns exactly one
// butterfly of it and T = N / R_0 threads serve one transform.
__host__ __device__ constexpr int radix_log2(int logn, int p) {
  switch (logn) {
    case 6:  return p < 2 ? 3 : 0;                            // 8 8
    case 7:  return p == 0 ? 4 : p == 1 ? 3 : 0;              // 16 8
    case 8:  return p < 2 ? 4 : 0;                            // 16 16
    case 9:  return p == 0 ? 5 : p == 1 ? 4 : 0;              // 32 16
    case 10: return p < 2 ? 4 : p == 2 ? 2 : 0;               // 16 16 4
    case 11: return p < 2 ? 4 : p == 2 ? 3 : 0;               // 16 16 8
    case 12: return p < 3 ? 4 : 0;                            // 16 16 16
    case 13: return p == 0 ? 5 : p < 3 ? 4 : 0;               // 32 16 16
    case 14: return p < 2 ? 5 : p == 2 ? 4 : 0;               // 32 32 16
    default: return 0;
  }
}

template <int LOGN>
struct PassPlan {
  static constexpr int N = 1 << LOGN;
  static constexpr int P = radix_log2(LOGN, 0) == 0 ? 0
                         : radix_log2(LOGN, 1) == 0 ? 1
                         : radix_log2(LOGN, 2) == 0 ? 2
                         : radix_log2(LOGN, 3) == 0 ? 3 : 4;
  __host__ __device__ static constexpr int R(int p) { return 1 << radix_log2(LOGN, p); }
  // product of the radices of passes < p
  __host__ __device__ static constexpr int Rprod(int p) { return p == 0 ? 1 : Rprod(p - 1) * R(p - 1); }
  __host__ __device__ static constexpr int M(int p) { return N / Rprod(p); }       // sub-problem size
  __host__ __device__ static constexpr int S(int p) { return M(p) / R(p); }        // gather stride
  static constexpr int T = N / R(0);                          // threads per transform
  static constexpr int RL = R(P - 1);                         // last radix
  static_assert(Rprod(P) == N, "radices must multiply to N");
  // Twiddle table: pass 0 holds w_N^{t*k} at k*T + t (t < T, k < R_0); pass
  // p >= 1 (stride S_p > 1) holds w_{M_p}^{t*k} at TwOff(p) + k*S_p + t.  The
  // thread-major order makes a warp's twiddle loads contiguous.
  __host__ __device__ static constexpr int TwOff(int p) {
    return p == 0 ? 0 : p == 1 ? N : TwOff(p - 1) + M(p - 1);
  }
  static constexpr int TW_LEN = TwOff(P - 1);                 // the last pass has no twiddles
};

// Position (in the working buffer) -> DFT bin held there after the forward
// passes: position = sum_p d_p * S_p, bin = sum_p d_p * Rprod(p).
template <int LOGN>
__host__ __device__ inline int position_to_bin(int pos) {
  using PL = PassPlan<LOGN>;
  int bin = 0;
#pragma unroll
  for (int p = 0; p < PL::P; ++p) {
    const int d = (pos / PL::S(p)) % PL::R(p);
    bin += d * PL::Rprod(p);
  }
  return bin;
}

// Inverse of position_to_bin: the working-buffer position that holds bin b.
template <int LOGN>
__host__ __device__ inline int bin_to_position(int bin) {
  using PL = PassPlan<LOGN>;
  int pos = 0;
#pragma unroll
  for (int p = 0; p < PL::P; ++p) {
    const int d = (bin / PL::Rprod(p)) % PL::R(p);
    pos += d * PL::S(p);
  }
  return pos;
}

// Padded shared-memory index: spare float2 words after every 16 points, so
// that the strided gathers and the stride-1 groups hit distinct banks.  Pad
// words after every 16 points of a transform's buffer.  Two where every
// radix pass but the last gathers at a stride of 16 or more: each stride-1
// group of the last pass then starts on a 16-byte boundary and moves as
// 128-bit accesses, and every gather stays free of bank conflicts.  One where
// a pass gathers at a smaller stride (N = 64, 128, 1024, 2048): two words
// would put both halves of a warp on the same banks there.
template <int LOGN>
__host__ __device__ constexpr int pad_words() {
  using PL = PassPlan<LOGN>;
  for (int p = 0; p + 1 < PL::P; ++p)
    if (PL::S(p) < 16) return 1;
  return 2;
}
template <int LOGN>
__device__ __forceinline__ int pad(int i) { return i + pad_words<LOGN>() * (i >> 4); }
template <int LOGN>
__host__ __device__ constexpr int padded_len() { return (1 << LOGN) + pad_words<LOGN>() * ((1 << LOGN) >> 4); }

}  // namespace cdd
