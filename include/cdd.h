/*
 * cdd.h -- C ABI of the B300 coherent-dedispersion library (libcdd.so).
 *
 * The library runs the per-channel overlap-save coherent dedispersion of
 * De & Gupta, "A Real-time Coherent Dedispersion Pipeline for the GMRT"
 * (arXiv:1509.00186) on one GPU:
 *
 *   unpack complex int8 -> forward FFT -> multiply by the chirp function
 *   (Sec. 2.1 Eq. 3, times the Sec. 2.2 taper) -> inverse FFT -> discard the
 *   overlap (Sec. 2.2 overlap-save) -> detect |v|^2 and integrate (Sec. 3.1)
 *   -> delay each channel to align it with the lowest one (Sec. 1.2).
 *
 * Every step runs in the library's own CUDA kernels; nothing here calls cuFFT
 * or falls back to the CPU.
 *
 * Conventions
 *   - Channel k (0 = lowest) covers [f_k, f_k + B/C) MHz with
 *     f_k = f_center - B/2 + k*B/C (upper sideband; a negative bandwidth
 *     gives a lower sideband, channel 0 highest).  Its complex baseband
 *     sample rate is |B|/C MHz.
 *   - Input layout (device or host, as the call says): int8 [T][C][2], time
 *     major, channel fastest, real then imaginary part (two's complement).
 *   - Output layout: float32 [C][n_out], channel major, intensities summed over
 *     n_avg detected samples and delayed by r_k integrated samples.
 *   - Overlap n_ov = ceil(n_d) rounded up to a multiple of n_avg, where n_d is
 *     the dispersion time across the lowest channel in samples; hop
 *     h = N - n_ov.  Each execute consumes block_samples = q*h new samples per
 *     channel (q = segments per block) and emits n_out = block_samples/n_avg
 *     outputs per channel: the next contiguous range of the stream's output.
 *   - r_k = rint(D*DM*(f_0^-2 - f_k^-2) * (B/C)*1e6 / n_avg),
 *     D = 4.148808e3 s MHz^2 cm^3/pc.
 *
 * Ownership: the caller owns every input and output buffer.  The plan owns its
 * device state (chirp and twiddle tables, overlap tails, alignment ring, host
 * staging buffers), allocated at the first execute call and freed by
 * cdd_destroy.  A plan is bound to the device that is current at its first
 * execute.  A plan is not thread-safe; distinct plans are independent.
 *
 * Errors: every int-returning call returns CDD_OK (0) or a negative code.
 * A CUDA failure is sticky: once a call has returned CDD_ECUDA, later calls on
 * the same plan return it too (cdd_reset does not clear it).
 */
#ifndef CDD_H
#define CDD_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CDD_OK            0
#define CDD_EINVAL       -1   /* bad argument or geometry                     */
#define CDD_ENOMEM       -2   /* device or pinned-host allocation failed      */
#define CDD_ECUDA        -3   /* a CUDA call failed (sticky)                  */
#define CDD_EUNSUPPORTED -4   /* valid request this library does not run     */
#define CDD_ESTATE       -5   /* call not allowed in the plan's current state */
#define CDD_ETOOBIG      -6   /* request needs more than the fixed scratch of
                                 cdd_execute_static                          */
#define CDD_EBUSY        -7   /* pool admission refused: HBM budget or stream
                                 slots exhausted (retry after a release)     */

/* Size of the fixed device scratch array behind cdd_execute_static. */
#define CDD_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)

/* Attributes for cdd_plan_get (all) and cdd_plan_set (marked "settable",
 * only before the first execute). */
enum cdd_attr {
  CDD_ATTR_N_FFT = 0,              /* N, power of two                          */
  CDD_ATTR_N_OV = 1,               /* overlap discarded per segment            */
  CDD_ATTR_HOP = 2,                /* h = N - n_ov                             */
  CDD_ATTR_N_AVG = 3,              /* integration length                       */
  CDD_ATTR_N_CHAN = 4,             /* C                                        */
  CDD_ATTR_SEGMENTS_PER_BLOCK = 5, /* q, settable, default 1                   */
  CDD_ATTR_BLOCK_SAMPLES = 6,      /* q*h input samples per channel per call   */
  CDD_ATTR_N_OUT_PER_BLOCK = 7,    /* q*h/n_avg outputs per channel per call   */
  CDD_ATTR_R_MAX = 8,              /* largest alignment shift r_k              */
  CDD_ATTR_BYTES_DEVICE = 9,       /* device bytes the plan holds (0 before)   */
  CDD_ATTR_TAPER = 10,             /* enum cdd_taper, settable                 */
  CDD_ATTR_BLOCKS_DONE = 11,       /* execute calls since create / reset       */
  CDD_ATTR_PIPELINE_CHUNKS = 12,   /* host-buffer path: copy/compute chunks per
                                      block (settable; divides q; default the
                                      most chunks of >= 4 segments each)       */
  CDD_ATTR_KERNEL_LAUNCHES = 13,   /* kernels launched by the last execute     */
  CDD_ATTR_BYTES_NEEDED = 14,      /* device bytes the first execute allocates
                                      (known before it; with the host path,
                                      staging comes on top)                    */
  CDD_ATTR_SEQ_GAPS = 15,          /* pool streams: blocks missing from the
                                      submitted sequence numbers               */
  CDD_ATTR_POLARISATIONS = 16,     /* 1 or 2 (settable): 2 keeps a second
                                      stream state for cdd_execute_dual        */
  CDD_ATTR_STAGE_TIMING = 17,      /* 0 or 1 (settable): 1 brackets the corner
                                      turn and the fused segment kernel of
                                      every block with CUDA events on the
                                      launching stream                         */
  CDD_ATTR_TIMED_BLOCKS = 18,      /* blocks timed so far (stage timing on)    */
  CDD_ATTR_CORNER_TURN_NS = 19,    /* summed device time of the corner turns
                                      of the timed blocks, nanoseconds         */
  CDD_ATTR_OLS_NS = 20,            /* summed device time of the fused segment
                                      kernels of the timed blocks, ns.  Reading
                                      18..20 waits for the timed blocks still
                                      in flight; the sums never reset.         */
  CDD_ATTR_PHASE_FLOATS = 22,      /* batch only: 1 when the DM = 1 chirp phase
                                      table is single floats (no chirp phase
                                      above 16 turns), else 2 (two floats)     */
  CDD_ATTR_PRECISION = 23,         /* enum cdd_precision, settable (see below) */
  CDD_ATTR_DEVICE_ERRORS = 24,     /* nonzero once a kernel gave up a bounded
                                      wait (it then stopped early and the
                                      block's outputs are invalid): bit 1 a
                                      tensor-core form's products, bit 2 the
                                      corner turn's tile copies; reading waits
                                      for the device                           */
  CDD_ATTR_HOST_STAGING_BYTES = 25,/* device bytes the host-buffer path adds
                                      (two chunks in, two out)                 */
  CDD_ATTR_BATCH_FORM = 26,        /* batch only, settable: the launch form
                                      (enum cdd_batch_form), or -1 (default):
                                      chosen by timing at the first execute   */
  CDD_ATTR_TUNE_NS_TIERS = 27,     /* batch only: device time of each form in
                                      the first execute's tuning, ns (0: not
                                      run)                                     */
  CDD_ATTR_TUNE_NS_TIERS_NP = 28,
  CDD_ATTR_TUNE_NS_MULTI = 29,
  CDD_ATTR_TURN_TMA = 30,          /* plan only, settable 0 (default) or 1: the
                                      corner turn as tensor-memory-accelerator
                                      tile copies (2-D tensor loads and stores,
                                      transposed in shared memory) where the
                                      layout allows it (n_chan a multiple of 8,
                                      16-byte aligned input); the same bits as
                                      the default turn                         */
  CDD_ATTR_PASS_PLAN = 31          /* full band only: the transform's pass plan,
                                      log2 of the shared-memory transform in
                                      bits 0-7, then log2 of each outer HBM
                                      pass's radix, 4 bits each from bit 8,
                                      pass 0 (largest stride) first            */
};

/* Launch forms of a batch; they differ in how the (tier, channel, segment)
 * work items reach the SMs.  TIERS and MULTI give the same outputs bit for
 * bit; TIERS_NP forms the N = 8192 tier's first-pass twiddles as products (as
 * the one-CTA-per-item kernels of 16384 points do), so its outputs differ from
 * theirs in the last bits, within the same accuracy.
 *   TIERS: one launch per tier, the N = 8192 tier as a persistent kernel
 *     (one CTA per SM, twiddles in shared memory), the others one CTA per
 *     work item (several CTAs per SM);
 *   TIERS_NP: one launch per tier, every tier one CTA per work item;
 *   MULTI: one persistent launch for every tier (tiers of 2048..16384
 *     points, at most four): one 512-thread CTA per SM takes the tiers
 *     longest-first, its groups claiming work items from each tier's counter,
 *     so CTAs move to the next tier without waiting for a launch boundary.
 * With CDD_ATTR_BATCH_FORM = -1 the first execute runs TIERS and (where it
 * applies) MULTI once each on its block, times them with CUDA events
 * (synchronously) and keeps the faster for this and later executes; the choice is remembered per device
 * and batch shape for the process, so later batches of that shape skip the
 * timing.  Make the first execute before capturing a stream into a graph. */
enum cdd_batch_form { CDD_BATCH_FORM_TIERS = 0, CDD_BATCH_FORM_TIERS_NP = 1, CDD_BATCH_FORM_MULTI = 2 };

enum cdd_taper { CDD_TAPER_NONE = 0, CDD_TAPER_HANN = 1, CDD_TAPER_WELCH = 2 };

/* Arithmetic of the transforms (the precision question of Sec. 3 and
 * Sec. 4.1: single precision versus double over long transforms).  The chirp
 * phase is always formed in FP64 and reduced modulo one turn before
 * rounding, and the chirp, twiddle and DFT-matrix tables are built in FP64.
 *   FP32: every step in FP32 on the CUDA cores (any N).
 *   FP16, BF16, FP16X2, BF16X2 (N = 8192 only, else CDD_EUNSUPPORTED): the
 *     radix passes (32, 16, 16) run as matrix products on the tensor cores
 *     (tcgen05) with FP32 accumulation; the operands are rounded to FP16 or
 *     BF16 (one product per pass), or split into a rounded value plus its
 *     rounded residual, for both the data and the DFT matrix (the X2 forms:
 *     three products, about 22 significant bits for FP16, 16 for BF16).
 *     Twiddles, the chirp, detection and integration stay in FP32.  Relative
 *     RMS error against an FP64 evaluation: about 1e-6 (FP16X2), 7e-6
 *     (BF16X2), 6e-4 (FP16), 5e-3 (BF16). */
enum cdd_precision {
  CDD_PRECISION_FP32 = 0,
  CDD_PRECISION_FP16 = 1,
  CDD_PRECISION_FP16X2 = 2,
  CDD_PRECISION_BF16X2 = 3,
  CDD_PRECISION_BF16 = 4
};

typedef struct cdd_plan_s* cdd_plan;

/* Create a plan for one polarisation of a C-channel band.
 *   f_center_mhz > 0, bandwidth_mhz != 0: observing band (Sec. 2.1 f_o,
 *     Delta f).  bandwidth_mhz < 0: a lower sideband, channel 0 the highest;
 *     each channel is the conjugate mirror of the upper-sideband one, so its
 *     chirp is conjugated on mirrored bins, and shifts are taken against the
 *     band's lowest channel.
 *   n_chan > 0: channels.  dm >= 0: dispersion measure in pc cm^-3 (Eq. 3).
 *   n_fft: FFT length N (power of two, 64..65536 in this library; above 16384
 *     a segment runs on a cluster of N/8192 CTAs and n_avg must be at most
 *     8192*8192/N), or 0 for the
 *     Sec. 2.3 rule: the smallest power of two > 2*n_d (raised so that
 *     N > n_ov, N >= 2*n_avg and N >= 64).
 *   n_avg > 0: detected samples summed per output; h must be a multiple of it.
 * Touches no GPU.  Returns CDD_EINVAL for an impossible geometry,
 * CDD_EUNSUPPORTED for an N this library does not run. */
int cdd_plan_create(cdd_plan* plan, double f_center_mhz, double bandwidth_mhz,
                    int n_chan, double dm, int n_fft, int n_avg);

/* Set an attribute (see enum cdd_attr).  CDD_ESTATE after the first execute. */
int cdd_plan_set(cdd_plan plan, int attr, int64_t value);

/* Read an attribute into *value. */
int cdd_plan_get(cdd_plan plan, int attr, int64_t* value);

/* Allocate the plan's device state and build its tables now (the first
 * execute does this otherwise).  Synchronous; binds the plan to the current
 * device. */
int cdd_plan_commit(cdd_plan plan);

/* Copy the n_chan alignment shifts r_k (integrated samples) to host memory
 * shifts[0..n_chan). */
int cdd_plan_shifts(cdd_plan plan, int64_t* shifts);

/* Dedisperse one block.  d_in: device int8 [q*h][C][2]; d_out: device
 * float [C][q*h/n_avg].  Asynchronous on `stream` (0 = legacy default
 * stream).  The first call allocates the plan's device state and builds its
 * tables (synchronously), so make it before capturing a stream into a graph.
 * Consecutive calls continue one stream: the first n_ov input samples of each
 * segment 0 come from the previous call (zeros before the first call). */
int cdd_execute(cdd_plan plan, const int8_t* d_in, float* d_out, cudaStream_t stream);

/* cdd_execute that also writes the dedispersed voltages (after the overlap
 * discard, before detection) to d_volt: device float [C][q*h][2]
 * (re, im).  For accuracy checks; slower than cdd_execute. */
int cdd_execute_voltages(cdd_plan plan, const int8_t* d_in, float* d_out,
                         float* d_volt, cudaStream_t stream);

/* Two polarisations of one beam (plan set to CDD_ATTR_POLARISATIONS = 2):
 * both inputs device int8 [q*h][C][2]; each is dedispersed and detected with
 * its own overlap tail and ring, and d_out float [C][q*h/n_avg] receives the
 * sum of the two intensities (Sec. 4.3 combines the polarisations after
 * detection).  CDD_ESTATE if the plan has one polarisation. */
int cdd_execute_dual(cdd_plan plan, const int8_t* d_in_a, const int8_t* d_in_b, float* d_out,
                     cudaStream_t stream);

/* Band sum (Sec. 1.2: the aligned sub-bands are added): d_sum[p][m] =
 * sum over k of d_out[p][k][m] for n_planes planes of [n_chan][n_out] floats
 * (a plan's output: one plane; a batch's: one per DM trial, giving the
 * DM-trial time series).  Device buffers; asynchronous on `stream`.  The
 * summation order is fixed (every 8th channel per partial sum, then the 8
 * partials), so results are deterministic; n_out % 4 == 0 with a 16-byte
 * aligned d_out takes the vector path. */
int cdd_band_sum(const float* d_out, int64_t n_planes, int n_chan, int64_t n_out, float* d_sum,
                 cudaStream_t stream);

/* End-to-end form with HOST buffers: h_in int8 [q*h][C][2], h_out float
 * [C][q*h/n_avg].  Copies in, dedisperses and copies out in
 * CDD_ATTR_PIPELINE_CHUNKS chunks so that transfers overlap compute (the
 * copy-in / compute / copy-out streams of Sec. 4.2), then waits for the
 * result.  Pinned host memory (cudaHostAlloc / torch pin_memory) gives
 * asynchronous copies; pageable memory works but serialises them.
 * `stream` orders the call after earlier work on it. */
int cdd_execute_host(cdd_plan plan, const int8_t* h_in, float* h_out, cudaStream_t stream);

/* cdd_execute_host without the final wait: returns once everything is
 * queued; `stream` reaches the end of the call's last copy-out (so an event or
 * host callback enqueued on `stream` afterwards marks the block's result in
 * h_out).  h_in and h_out must stay valid until then; the next call on the
 * same plan is ordered after this one. */
int cdd_execute_host_async(cdd_plan plan, const int8_t* h_in, float* h_out, cudaStream_t stream);

/* Allocate the host-buffer path's staging now (CDD_ATTR_HOST_STAGING_BYTES;
 * commits the plan if needed), so that later host-buffer calls allocate
 * nothing.  Synchronous. */
int cdd_plan_prepare_host(cdd_plan plan);

/* No-allocation form.  The paper has no counterpart: this entry point exists
 * for callers that must not allocate device memory -- code running where
 * cudaMalloc is unavailable or forbidden, such as real-time loops that may only
 * allocate at start-up, callers whose memory is owned by another allocator, or
 * hosts that link the library into a process with a fixed memory budget.
 *
 * It dedisperses ONE block as the first call of a fresh plan with the same
 * arguments would (zero history before the block; the outputs of the block's
 * last r_k samples of each channel, which belong to a later block, are
 * dropped): d_in device int8 [n_seg*h][C][2], d_out device float
 * [C][n_seg*h/n_avg], h = N - n_ov as in cdd_plan_create.  taper is an
 * enum cdd_taper.  Asynchronous on `stream`.  N above 16384 (the cluster
 * form, which needs a channel-major copy of the block) returns
 * CDD_EUNSUPPORTED here.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine.  Its chirp
 * and twiddle tables, shifts, zero history and alignment spill all live in one
 * file-scope device array of CDD_STATIC_SCRATCH_BYTES (64 MiB).  A GPU holds
 * the array from the moment the library's device code is loaded on it until
 * the process exits; CUDA may load that code lazily, at the first call that
 * needs it, so the first cdd_execute_static on a device can be the moment the
 * array is reserved.  Make that first call at start-up.  The tables are
 * rebuilt on every call; the zero history is cleared on every call.  A request
 * whose tables need more than the array returns CDD_ETOOBIG (the 512-channel,
 * N = 8192 shape needs about 36 MB).
 *
 * The first call on each device looks up the array's device address (with
 * that device current), so make it before any stream capture.  Every call on
 * a device shares the one array: calls that overlap on the GPU (on different
 * streams, or from different threads) race on it and give wrong results, so
 * serialise them. */
int cdd_execute_static(double f_center_mhz, double bandwidth_mhz, int n_chan, double dm,
                       int n_fft, int n_avg, int n_seg, int taper, const int8_t* d_in,
                       float* d_out, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Batched form: n_dm DM trials over one band, the channels cut into n_tiers
 * equal groups (lowest frequencies first: the first channels of an upper
 * sideband, the last of a lower one, bandwidth_mhz < 0 as for a plan) that
 * dedisperse with their own N.
 * Each segment's forward transform is computed once and shared by every DM
 * trial (Sec. 2.2 deconvolution repeated per trial DM; Sec. 1.2 alignment per
 * trial).  Tier t uses N_t = tier_nfft[t] (power of two, 64..16384) and the
 * overlap max(N_t/32, dispersion samples of its lowest channel at the largest
 * DM) rounded up to a multiple of n_avg; the hops must nest (each divides the
 * longest).  A block is q longest hops (CDD_ATTR_SEGMENTS_PER_BLOCK), so every
 * channel emits n_out = q*h_max/n_avg outputs per block; the block must be at
 * least as long as the largest alignment shift (CDD_ATTR_R_MAX), and the
 * default q is the smallest such value.
 *   d_in: device int8 [q*h_max][C][2];  d_out: device float [n_dm][C][n_out]
 *   (DM-major planes laid out like cdd_execute's output).
 * Streams continue across calls as for cdd_execute.  The DM list is copied. */
typedef struct cdd_batch_s* cdd_batch;

int cdd_batch_create(cdd_batch* batch, double f_center_mhz, double bandwidth_mhz, int n_chan,
                     const double* dms, int n_dm, const int* tier_nfft, int n_tiers, int n_avg);
/* CDD_ATTR_SEGMENTS_PER_BLOCK, CDD_ATTR_TAPER (applied to every DM trial) and
 * CDD_ATTR_BATCH_FORM, before the first execute.  MULTI for a shape it does
 * not cover makes the first execute return CDD_EUNSUPPORTED. */
int cdd_batch_set(cdd_batch batch, int attr, int64_t value);
/* SEGMENTS_PER_BLOCK, BLOCK_SAMPLES, N_OUT_PER_BLOCK, R_MAX, BYTES_DEVICE,
 * BLOCKS_DONE, KERNEL_LAUNCHES, N_CHAN, N_AVG, HOP (the longest hop),
 * PHASE_FLOATS, TAPER, BATCH_FORM (the form in use once one ran),
 * TUNE_NS_*. */
int cdd_batch_get(cdd_batch batch, int attr, int64_t* value);
/* Geometry of tier t (any output pointer may be NULL). */
int cdd_batch_tier(cdd_batch batch, int t, int64_t* n_fft, int64_t* n_ov, int64_t* first_chan,
                   int64_t* n_tier_chan);
/* Alignment shifts, host int64 [n_dm][n_chan]. */
int cdd_batch_shifts(cdd_batch batch, int64_t* shifts);
int cdd_batch_execute(cdd_batch batch, const int8_t* d_in, float* d_out, cudaStream_t stream);
int cdd_batch_reset(cdd_batch batch);
int cdd_batch_destroy(cdd_batch batch);
/* Stream checkpoint of a batch, as for a plan (cdd_plan_export_state): the
 * overlap tail of every channel, the carried outputs of every DM plane (the
 * last r_max of each channel) and the block count.  A blob imports only into
 * a batch of the same geometry (frequencies, bandwidth and sideband, channels,
 * DM list, tiers, n_avg, segments per block, taper), else CDD_EINVAL with
 * nothing changed.
 *   cdd_batch_state_bytes: size of the blob, host side only.
 *   cdd_batch_export_state: waits for `stream`, then copies the state into
 *     host memory `state` of `bytes` >= the size (a batch that has not run
 *     exports a fresh stream).
 *   cdd_batch_import_state: commits the batch if needed, waits for `stream`,
 *     and replaces its stream state.
 * Blocks run after an import continue the exported stream bit for bit. */
int cdd_batch_state_bytes(cdd_batch batch, int64_t* bytes);
int cdd_batch_export_state(cdd_batch batch, void* state, int64_t bytes, cudaStream_t stream);
int cdd_batch_import_state(cdd_batch batch, const void* state, int64_t bytes, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Full-band mode: the paper's own design (Sec. 2.3, Sec. 3.1, Sec. 4.3).
 * The input is the voltage beam as recorded: for every frame, the C complex
 * outputs of a 2C-point FFT of the real, Nyquist-sampled voltage (bins 0..C-1;
 * 2C a power of two, 64..16384).  Each frame is inverse transformed back to
 * 2C real samples (bin 0 real part only, the Nyquist bin zero, scaled by
 * 1/(2C)); the real series at 2|B| samples per second is then dedispersed as
 * one band: N-point transforms (N a power of two up to 2^27, or 0 for the
 * Sec. 2.3 rule: the smallest power of two above twice the dispersion samples
 * across the band), the chirp of Eq. 3 with f_o the band's lower edge on every
 * bin, inverse transforms, overlap-save with an overlap of the dispersion
 * samples rounded up to whole frames and integration windows, squaring and
 * integration over n_avg samples (a power of two).  bandwidth_mhz < 0: a
 * lower sideband, whose real series is the band inverted (frame bin b at
 * |B| - b |B|/C above the lower edge); its chirp is the conjugate at that
 * mirrored offset.
 *   d_in: device int8 [frames][C][2], frames = q*h/(2C) per block
 *         (CDD_ATTR_BLOCK_SAMPLES reports frames for this plan type);
 *   d_out: device float [q*h/n_avg], the band's intensity series.
 * Streams continue across calls (the last n_ov real samples lead the next
 * block).  Segments run one after another, each over the whole GPU. */
typedef struct cdd_fullband_s* cdd_fullband;

int cdd_fullband_create(cdd_fullband* plan, double f_center_mhz, double bandwidth_mhz, int n_chan,
                        double dm, long long n_fft, int n_avg);
/* Only CDD_ATTR_SEGMENTS_PER_BLOCK, before the first execute. */
int cdd_fullband_set(cdd_fullband plan, int attr, int64_t value);
int cdd_fullband_get(cdd_fullband plan, int attr, int64_t* value);
int cdd_fullband_execute(cdd_fullband plan, const int8_t* d_in, float* d_out, cudaStream_t stream);
int cdd_fullband_reset(cdd_fullband plan);
int cdd_fullband_destroy(cdd_fullband plan);

/* ------------------------------------------------------------------------
 * Serving pool: concurrent observation streams on one GPU (the real-time
 * loop of Sec. 4.2 and 4.3, for many streams at once).  Each stream has its
 * own plan -- overlap tail, alignment ring and integration state stay on the
 * device between blocks -- and its own CUDA stream, so a block submitted while
 * others are on the GPU is launched at once and overlaps with them.
 *
 * Admission.  A stream needs its plan's device bytes (CDD_ATTR_BYTES_NEEDED,
 * plus CDD_ATTR_HOST_STAGING_BYTES when admitted with CDD_POOL_HOST_INGEST)
 * out of the pool's HBM budget, and a free slot.  cdd_pool_admit[_ex] admits
 * at once or returns CDD_EBUSY; cdd_pool_request queues the stream instead:
 * queued requests are admitted first come, first served, whenever memory and
 * a slot are free (at the request, at every release, and at every status
 * query), and an immediate admission never overtakes a queued one.  Admission
 * allocates and builds the stream's tables at once (synchronously), so an
 * admitted stream cannot fail later for memory.
 *
 * Blocks.  Every submission carries the block's sequence number, which must
 * be the stream's next one: an older or repeated number is refused, and so
 * is a later one while an earlier block is missing (CDD_EINVAL, nothing
 * enqueued).  After a loss the caller moves the stream past it with
 * cdd_pool_stream_resync, which restarts the stream from zero history (as a
 * fresh stream: Sec. 4.3's overlap carry and the alignment ring need the
 * missing block) and counts the skipped blocks (CDD_ATTR_SEQ_GAPS).  A block's
 * latency runs from its arrival time (cdd_pool_clock_ms units; the submit
 * call's own time for cdd_pool_submit) to the completion of its work on the
 * GPU, including the copies of a host-buffer block (stamped on the host by a
 * stream callback).  The pool is thread-safe. */
typedef struct cdd_pool_s* cdd_pool;

enum cdd_pool_attr {
  CDD_POOL_BUDGET = 100,       /* HBM budget, bytes                             */
  CDD_POOL_USED_BYTES = 101,   /* bytes held by admitted streams                */
  CDD_POOL_STREAMS = 102,      /* admitted streams                              */
  CDD_POOL_QUEUED = 103        /* admission requests still waiting              */
};
/* cdd_pool_admit_ex / cdd_pool_request flags */
#define CDD_POOL_HOST_INGEST 1  /* also reserve host-buffer staging, so the
                                   stream's cdd_pool_submit_host calls allocate
                                   nothing */

/* Milliseconds on the steady clock the pool stamps completions with: the
 * unit of the arrival times passed to the submit calls. */
double cdd_pool_clock_ms(void);

int cdd_pool_create(cdd_pool* pool, int64_t hbm_budget_bytes, int max_streams);
/* Admit a stream now (arguments as cdd_plan_create plus segments per block
 * and taper); *stream_id receives its slot.  CDD_EBUSY if it does not fit now
 * or a queued request is waiting. */
int cdd_pool_admit(cdd_pool pool, double f_center_mhz, double bandwidth_mhz, int n_chan,
                   double dm, int n_fft, int n_avg, int segments_per_block, int taper,
                   int* stream_id);
/* cdd_pool_admit with flags (CDD_POOL_HOST_INGEST). */
int cdd_pool_admit_ex(cdd_pool pool, double f_center_mhz, double bandwidth_mhz, int n_chan,
                      double dm, int n_fft, int n_avg, int segments_per_block, int taper, int flags,
                      int* stream_id);
/* Queue a stream for admission; *request identifies it.  It may be admitted
 * before this returns.  CDD_EBUSY if it needs more than the whole budget. */
int cdd_pool_request(cdd_pool pool, double f_center_mhz, double bandwidth_mhz, int n_chan,
                     double dm, int n_fft, int n_avg, int segments_per_block, int taper, int flags,
                     int64_t* request);
/* CDD_EBUSY while the request waits; CDD_OK with *stream_id once admitted
 * (reported once; the request is then forgotten); the admission's error if it
 * failed; CDD_EINVAL for an unknown request. */
int cdd_pool_request_status(cdd_pool pool, int64_t request, int* stream_id);
/* Plan attributes of a stream, plus CDD_ATTR_SEQ_GAPS. */
int cdd_pool_stream_get(cdd_pool pool, int stream_id, int attr, int64_t* value);

/* Checkpoint of an admitted stream (see cdd_plan_export_state): the plan's
 * stream state after the stream's submitted blocks (waits for them), and the
 * next sequence number the pool expects.  Import into an admitted stream of
 * the same geometry in this or another pool, with the sequence number to
 * continue from; the stream then resumes bit for bit. */
int cdd_pool_stream_state_bytes(cdd_pool pool, int stream_id, int64_t* bytes);
int cdd_pool_stream_export(cdd_pool pool, int stream_id, void* state, int64_t bytes, int64_t* next_seq);
int cdd_pool_stream_import(cdd_pool pool, int stream_id, const void* state, int64_t bytes, int64_t next_seq);
/* Restart a stream at sequence number seq (>= the next expected one) after
 * lost blocks: waits for its work, zeroes its history (cdd_reset) and adds
 * the skipped numbers to CDD_ATTR_SEQ_GAPS. */
int cdd_pool_stream_resync(cdd_pool pool, int stream_id, int64_t seq);

/* Enqueue block `seq` of a stream from device buffers (d_in, d_out as for
 * cdd_execute).  Returns at once with a ticket for cdd_pool_wait; latency is
 * counted from the call. */
int cdd_pool_submit(cdd_pool pool, int stream_id, int64_t seq, const int8_t* d_in, float* d_out,
                    int64_t* ticket);
/* cdd_pool_submit with the block's arrival time (cdd_pool_clock_ms units):
 * latency is counted from the arrival, so time spent waiting for admission or
 * in the caller's queue counts. */
int cdd_pool_submit_at(cdd_pool pool, int stream_id, int64_t seq, const int8_t* d_in, float* d_out,
                       double t_arrival_ms, int64_t* ticket);
/* Block from HOST buffers (h_in, h_out as for cdd_execute_host; pinned memory
 * for asynchronous copies) of a stream admitted with CDD_POOL_HOST_INGEST
 * (else CDD_ESTATE): copy-in, dedispersion and copy-out are enqueued on the
 * stream's CUDA stream, overlapping within the block (Sec. 4.2) and with other
 * streams; the ticket completes when h_out holds the result. */
int cdd_pool_submit_host(cdd_pool pool, int stream_id, int64_t seq, const int8_t* h_in, float* h_out,
                         double t_arrival_ms, int64_t* ticket);
/* n submissions in one call (host != 0: host buffers): blocks i of streams
 * ids[i] with seqs[i], ins[i], outs[i], arrival times t_arrival_ms[i] (NULL:
 * now).  Stops at the first refusal and returns its code; *submitted counts
 * the blocks enqueued, whose tickets are in tickets[0..*submitted). */
int cdd_pool_submit_many(cdd_pool pool, int n, const int* stream_ids, const int64_t* seqs,
                         const int8_t* const* ins, float* const* outs, const double* t_arrival_ms,
                         int host, int64_t* tickets, int* submitted);
/* Wait for a ticket; *latency_ms (may be NULL) receives arrival-to-done time. */
int cdd_pool_wait(cdd_pool pool, int64_t ticket, double* latency_ms);
/* Wait for the stream's blocks, free its plan and return its bytes to the
 * budget; queued requests that now fit are admitted. */
int cdd_pool_release(cdd_pool pool, int stream_id);
int cdd_pool_get(cdd_pool pool, int attr, int64_t* value);
/* Release every stream and drop the queued requests. */
int cdd_pool_destroy(cdd_pool pool);

/* Restart the stream: zero the overlap tails and the alignment ring and the
 * block counter.  Waits for the plan's outstanding work. */
int cdd_reset(cdd_plan plan);

/* Stream checkpoint (no counterpart in the paper; a real-time pipeline
 * restarts a stream without losing its overlap and alignment state).  The
 * state a stream carries between blocks is the last n_ov input samples of
 * each channel (the overlap tail), the integrated samples whose aligned
 * positions fall in later blocks (the last r_max entries of the alignment
 * ring) and the stream position; for a two-polarisation plan, both.
 *   cdd_plan_state_bytes: size of the blob (header + state), host side only.
 *   cdd_plan_export_state: waits for `stream` (the plan's work must be on it),
 *     then copies the state into host memory `state` of `bytes` >= the size.
 *     A plan that has not run exports the state of a fresh stream.
 *   cdd_plan_import_state: replaces the plan's stream state with a blob from
 *     a plan of the same geometry (frequencies, bandwidth, channels, DM, N,
 *     n_avg, segments per block, taper, polarisations), else CDD_EINVAL with
 *     nothing changed; commits the plan if needed and waits for `stream`.
 * Blocks run after an import continue the exported stream bit for bit. */
int cdd_plan_state_bytes(cdd_plan plan, int64_t* bytes);
int cdd_plan_export_state(cdd_plan plan, void* state, int64_t bytes, cudaStream_t stream);
int cdd_plan_import_state(cdd_plan plan, const void* state, int64_t bytes, cudaStream_t stream);

/* Free the plan and everything it owns (NULL is accepted). */
int cdd_destroy(cdd_plan plan);

/* Static string for an error code. */
const char* cdd_strerror(int code);

/* Library version as major*10000 + minor*100 + patch. */
int cdd_version(void);

/* Self-test of the kernels' bounded waits on the current device.  It runs
 * the tensor-copy corner turn on one 64 x 64 tile whose mbarrier expects more
 * bytes than the copy brings, so the wait can never be met.  The kernel must
 * give up after its limit (20 ms here, 1 s in normal launches), set its error
 * flag and return.  *status receives that flag (2 when the wait ran out as it
 * should).  Returns CDD_OK when the kernel returned and the device still
 * answered afterwards; CDD_EUNSUPPORTED without tensor maps; CDD_ENOMEM or
 * CDD_ECUDA otherwise.  Allocates and frees 16 KB; synchronises the device. */
int cdd_selftest_wait_limit(int* status);

#ifdef __cplusplus
}
#endif

#endif /* CDD_H */
