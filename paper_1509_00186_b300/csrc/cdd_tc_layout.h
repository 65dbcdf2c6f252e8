// cdd_tc_layout.h -- operand layouts, tcgen05 descriptors and index maps of
// the tensor-core form of the N = 8192 overlap-save transform.
//
// Plain C++ (no CUDA types): the kernel in cdd_tc.cu and a host program in
// tests/ both include it, so the host can check the layouts and the index
// maps against a direct DFT before any of it runs on a GPU.
//
// The transform is the one the FP32 kernel runs (cdd_fft.cuh, PassPlan<13>):
// N = 8192 = 32 * 16 * 16, forward decimation in frequency, inverse
// decimation in time on the same index sets, spectrum in digit-reversed
// order.  Pass p gathers groups of R_p points; on the tensor cores each pass
// is one matrix product per 128 groups:
//
//     D[g][n] = sum_kk A[g][kk] * B[n][kk]
//
//   A: one row per group g, K = 2 R_p half-precision values (element e of the
//      group at kk = 2e (real) and 2e + 1 (imaginary)), in shared memory;
//   B: the real form of the R-point forward DFT matrix divided by R: rows
//      n = 2k + c' (output k, c' = 0 real, 1 imaginary), K = 2R.  Rows 0..2R-1
//      hold the matrix rounded to half precision (hi), rows 2R..4R-1 the
//      rounding residual (lo), so one product with N = 4R gives
//      [A*B_hi | A*B_lo] and the thread adds the two halves;
//   D: FP32 in tensor memory, row g in lane g mod 128, column n.
//
// The inverse passes use the same forward matrix on conjugated data: for any
// vector v, IDFT(v) = conj(DFT(conj v)).  Every operand of an inverse pass is
// stored conjugated, so the twiddles of the inverse passes are multiplied
// unconjugated and the last pass yields conj(y).
//
// Scaling (exact powers of two): each pass divides by its radix (in B), so
// the forward passes give X / N; the chirp table carries a factor
// kChirpScale; the inverse passes give conj(y) / kOutScale with
// kOutScale = N / kChirpScale.  Every operand then stays within the int8
// input's range (|value| <= 181 * kChirpScale), far inside FP16's.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define CDD_HD __host__ __device__
#else
#define CDD_HD
#endif

namespace cdd {
namespace tc {

constexpr int kLogN = 13;
constexpr int kN = 1 << kLogN;
constexpr int kT = 256;              // threads per transform: one pass-0 group each
constexpr int kR0 = 32, kR1 = 16, kR2 = 16;
constexpr int kTwOff1 = kN;          // pass-1 twiddles in the FP32 kernel's table
constexpr double kChirpScale = 16.0;
constexpr double kOutScale = kN / kChirpScale;    // voltages: y = conj(u) * 512

// --------------------------------------------------------------- A layouts
// Canonical K-major layout without swizzle: core matrices of 8 rows x 16
// bytes (8 values of one row), rows 16 bytes apart.  Offsets in bytes:
//   ts  between tiles of 128 rows,      ks  between k-steps of 16 values,
//   sbo between groups of 8 rows,       lbo between the two 8-value chunks.
struct Lay {
  int ts, ks, sbo, lbo;
};
CDD_HD constexpr int lay_off(Lay L, int m, int kk) {
  return (m >> 7) * L.ts + (kk >> 4) * L.ks + ((m & 127) >> 3) * L.sbo + ((kk & 15) >> 3) * L.lbo +
         (m & 7) * 16 + (kk & 7) * 2;
}
// Pass 0 (256 groups x 64 values): dense.  Passes 1 and 2 (512 groups x 32
// values): 8-row groups 272 bytes apart and chunks 144 bytes apart, which
// spreads the scattered 4-byte stores between passes over the banks (two
// wavefronts per warp store instead of four).
CDD_HD constexpr Lay lay0() { return Lay{16384, 4096, 256, 128}; }
CDD_HD constexpr Lay lay12() { return Lay{8704, 4352, 272, 144}; }
constexpr int kRegion = 34816;       // bytes of one operand region (hi or lo)

// --------------------------------------------------------------- B layout
// Radix R: 4R rows ([hi; lo]) x 2R values, dense canonical K-major.
CDD_HD constexpr int b_ks(int R) { return (4 * R / 8) * 256; }          // bytes per k-step
CDD_HD constexpr int b_off(int R, int n, int kk) {
  return (kk >> 4) * b_ks(R) + (n >> 3) * 256 + ((kk & 15) >> 3) * 128 + (n & 7) * 16 + (kk & 7) * 2;
}
CDD_HD constexpr int b_bytes(int R) { return (2 * R / 16) * b_ks(R); }
constexpr int kLboB = 128, kSboB = 256;

// Entry (n, kk) of the real form of the forward DFT matrix exp(-2 pi i jk/R):
// the angle index m = jk mod R (angle 2 pi m / R), whether it is the sine,
// and its sign.  Output re: cos * re + sin * im; output im: -sin * re + cos * im.
CDD_HD constexpr int dft_m(int R, int n, int kk) { return ((n >> 1) * (kk >> 1)) % R; }
CDD_HD constexpr bool dft_is_sin(int n, int kk) { return ((n ^ kk) & 1) != 0; }
CDD_HD constexpr bool dft_negative(int n, int kk) { return (n & 1) == 1 && (kk & 1) == 0; }

// --------------------------------------------------------------- descriptors
// Shared-memory matrix descriptor (tcgen05): start address >> 4 in bits 0-13,
// leading byte offset >> 4 in 16-29, stride byte offset >> 4 in 32-45, the
// descriptor version 1 in bits 46-47, base offset 0 (49-51), absolute LBO
// mode 0 (52), layout 0 = no swizzle (61-63).  For a K-major operand without
// swizzle the leading offset is the distance between the two 8-value chunks
// of one instruction's K = 16, the stride offset that between 8-row groups.
CDD_HD constexpr uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: D format F32 (bits 4-5 = 1), A and B
// format (bits 7-9, 10-12: 0 FP16, 1 BF16), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28; dense, no negation.
CDD_HD constexpr uint32_t idesc_f16(int m, int n, bool bf16) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}
// Tensor-memory address: lane in bits 16-31, column in bits 0-15.
CDD_HD constexpr uint32_t tmem_addr(uint32_t base, int lane, int col) {
  return base + ((uint32_t)lane << 16) + (uint32_t)col;
}

// --------------------------------------------------------------- index maps
// Transform-buffer positions: pass-0 group t (t < 256) holds positions
// t + 256 j; pass-1 group g = 16 sp + t1 holds 256 sp + t1 + 16 j; pass-2
// group q holds 16 q + k.  After the forward passes position p holds bin
// (p / 256) + 32 ((p / 16) mod 16) + 512 (p mod 16).
CDD_HD constexpr int pos_pass0(int t, int j) { return t + 256 * j; }
CDD_HD constexpr int pos_pass1(int g, int j) { return 256 * (g >> 4) + (g & 15) + 16 * j; }
CDD_HD constexpr int pos_pass2(int q, int k) { return 16 * q + k; }
CDD_HD constexpr int bin_of_pos(int p) { return (p >> 8) + 32 * ((p >> 4) & 15) + 512 * (p & 15); }

// Forward pass 0, output k of group t -> pass-1 row and element, twiddle
// w_N^{tk} at table index k*256 + t.
CDD_HD constexpr int f0_row(int t, int k) { return 16 * k + (t & 15); }
CDD_HD constexpr int f0_elem(int t) { return t >> 4; }
CDD_HD constexpr int f0_tw(int t, int k) { return 256 * k + t; }
// Forward pass 1, output k of group g -> pass-2 row and element, twiddle
// w_256^{(g mod 16) k}.
CDD_HD constexpr int f1_row(int g, int k) { return 16 * (g >> 4) + k; }
CDD_HD constexpr int f1_elem(int g) { return g & 15; }
CDD_HD constexpr int f1_tw(int g, int k) { return kTwOff1 + 16 * k + (g & 15); }
// Forward pass 2, output k of group q: its chirp entry is float4 index
// chirp4_index(q, k) of the channel's row, half (k & 1) (the FP32 kernel's
// paired table: bins k and k + 1 of a group in one 16-byte entry).
CDD_HD constexpr int chirp4_index(int q, int k) { return 512 * (k >> 1) + q; }
// Inverse pass 2, output k of group q -> inverse pass-1 row and element,
// twiddle w_256^{k (q mod 16)}.  The pass-1 table holds w_256^{tk} at
// 16 k + t, symmetric in t and k, so the entry is read at 16 k + (q mod 16):
// neighbouring groups then read neighbouring entries.
CDD_HD constexpr int i2_row(int q, int k) { return 16 * (q >> 4) + k; }
CDD_HD constexpr int i2_elem(int q) { return q & 15; }
CDD_HD constexpr int i2_tw(int q, int k) { return kTwOff1 + 16 * k + (q & 15); }
// Inverse pass 1, output j of group g -> inverse pass-0 row and element,
// twiddle w_N^{t k0} with t the row and k0 the element.
CDD_HD constexpr int i1_row(int g, int j) { return (g & 15) + 16 * j; }
CDD_HD constexpr int i1_elem(int g) { return g >> 4; }
CDD_HD constexpr int i1_tw(int g, int j) { return 256 * (g >> 4) + (g & 15) + 16 * j; }

// The kernel's shared-memory copy of the twiddle table: 8 spare entries
// after every 256, so that the two half-warps of an inverse-pass-1 read
// (rows 256 apart) fall on different banks.
CDD_HD constexpr int tw_slot(int i) { return i + 8 * (i >> 8); }
CDD_HD constexpr int tw_slots(int n) { return tw_slot(n - 1) + 1; }

// Tensor-memory columns of one pass: 2R per tile (one product), or 4R with
// the [hi | lo] matrix.
CDD_HD constexpr int tile_cols(int R, bool split) { return split ? 4 * R : 2 * R; }

}  // namespace tc
}  // namespace cdd
