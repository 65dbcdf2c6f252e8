// cdd_internal.h -- plan state and kernel launch interface shared by the C ABI
// (cdd_api.cu) and the kernels (cdd_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cdd {

// Arguments of one launch of the fused overlap-save kernel: q segments of
// every channel, one block of the stream.
struct OlsArgs {
  const char2* in;        // [q*h][C] complex int8, block-local rows
  const char2* in_cm;     // the same block channel-major [C][rows], or nullptr
  long long rows;         // rows of in_cm (q*h)
  float* out;             // [C][n_out]
  const float2* chirp;    // [C][N] chirp function, digit-reversed layout
  const float2* tw;       // [N] exp(-2 pi i m / N)
  const char2* tail_rd;   // [C][n_ov] last n_ov samples of the previous block
  char2* tail_wr;         // [C][n_ov] last n_ov samples of this block
  float* ring;            // [C][ring_len] integrated samples still to be emitted
  const int* shift;       // [C] alignment shift r_k
  float2* volt;           // [C][q*h] dedispersed voltages, or nullptr
  const void* dft;        // tensor-core forms: the DFT matrices (tc_dft_bytes), else nullptr
  int n_chan, n_ov, hop, n_avg, q, n_out;
  int s_begin, s_count;   // this launch runs segments [s_begin, s_begin + s_count) of q
  long long g0;           // stream index of this block's first integrated sample
  long long ring_len;
};

// Observation geometry (Sec. 2.2 / 2.3, alignment of Sec. 1.2) without the
// per-channel shifts; geometry() returns a CDD_* code and allocates nothing.
struct Geometry {
  double f_center, bandwidth, dm, chan_bw, f_lo0, n_disp;
  int n_chan, n_fft, logn, n_ov, hop, n_avg;
  int64_t r_max;
  int sideband;      // +1 upper (channel 0 lowest), -1 lower (channel 0 highest)
  double f_base;     // upper: f_lo0; lower: the band's top edge
  double f_ref;      // lowest channel's lower edge: reference of smear and shifts
};
// Lower edge of channel k: f_base + k*chan_bw (upper) or f_base - (k+1)*chan_bw (lower).
inline double chan_lower_edge(const Geometry& g, int k) {
  return g.sideband > 0 ? g.f_base + g.chan_bw * k : g.f_base - g.chan_bw * (k + 1.0);
}
int geometry(Geometry* g, double f_center, double bandwidth, int n_chan, double dm, int n_fft,
             int n_avg);
// Alignment shift r_k of channel k in integrated samples (-1 if out of range).
int64_t shift_of(const Geometry& g, int k);

// Launch the fused kernel for N = 2^logn.  Returns the CUDA error of the launch.
cudaError_t launch_ols(int logn, const OlsArgs& a, cudaStream_t s);

// out[k*stride + row] = in[row][k] for rows [r_begin, r_end): channel-major copy
// of (part of) a block of int8 pairs.  With err (a device int) the turn goes
// through tensor-memory-accelerator tile copies where the layout allows them
// (corner_turn_tma_ok); a copy wait that runs out sets bit 2 of *err.
cudaError_t launch_corner_turn(const char2* in, char2* out, long long r_begin, long long r_end,
                               long long stride, int n_chan, cudaStream_t s, int* err = nullptr);
bool corner_turn_tma_ok(const char2* in, const char2* out, long long r_begin, long long r_end, long long stride,
                        int n_chan);
// cudaErrorNotSupported (and nothing launched) where corner_turn_tma_ok fails.
cudaError_t launch_corner_turn_tma(const char2* in, char2* out, long long r_begin, long long r_end, long long stride,
                                   int n_chan, int* err, cudaStream_t s);

// Build the chirp table (FP64 phase, reduced mod 1 turn, then rounded to
// float): chirp[k][idx] = exp(-i Phi_k(f_l)) * w(f_l) * scale in the layout
// the fused kernel reads; scale 0 means 1/N (the FP32 kernels).
cudaError_t launch_chirp_table(int logn, float2* chirp, int n_chan, double f_base_mhz,
                               double chan_bw_mhz, double dm, int taper, int sideband,
                               cudaStream_t s, double scale = 0.0);

// Tensor-core form of the fused kernel (cdd_tc.cu): the reduced precisions
// of enum cdd_precision, N = 8192 only.  `err` is a device int that the
// kernel ORs with 1 if a wait for its tensor-core products gives up.
bool tc_supported(int logn, int precision);
cudaError_t launch_ols_tc(int logn, int precision, const OlsArgs& a, int* err, cudaStream_t s);
// The chirp table's scale for the tensor-core form.
double tc_chirp_scale();
// The DFT matrices of the tensor-core form (radix 32 then radix 16, hi and
// lo rows, in the operand layout), built in FP64 once per plan.
size_t tc_dft_bytes();
cudaError_t launch_tc_dft_table(int precision, void* dft, cudaStream_t s);

// Twiddle factors of every radix pass in the kernel's thread-major layout
// (FP64, then rounded); twiddle_table_len entries.
cudaError_t launch_twiddle_table(int logn, float2* tw, cudaStream_t s);
int twiddle_table_len(int logn);
// N = 2^logn runs as a CTA cluster and reads only the channel-major copy.
bool needs_channel_major(int logn);
// log2 of the points one CTA of a cluster holds (N > 16384).
constexpr int kClusterLogS = 13;

// shift[k] = r_k for k < n_chan, computed on the device in FP64.
cudaError_t launch_shift_table(int* shift, int n_chan, double f_base_mhz, double f_ref_mhz,
                               double chan_bw_mhz, double dm, int n_avg, int sideband,
                               cudaStream_t s);

// sum[p][m] = sum_k out[p][k][m] (a fixed summation order: deterministic).
cudaError_t launch_band_sum(const float* out, long long n_planes, int n_chan, long long n_out,
                            float* sum, cudaStream_t s);
// acc[i] += add[i], i < n.
cudaError_t launch_accumulate(float* acc, const float* add, long long n, cudaStream_t s);

// Dynamic shared memory and block size of the fused kernel for N = 2^logn.
int ols_threads(int logn);
int ols_segments_per_cta(int logn);
size_t ols_smem_bytes(int logn);

}  // namespace cdd
