// cdd_tc.cu -- the fused overlap-save kernel for N = 8192 with the radix
// passes on the tensor cores (tcgen05), for the reduced-precision forms of
// CDD_ATTR_PRECISION: FP16 and BF16 operands alone, or split into hi + lo
// pairs (FP16X2, BF16X2), always accumulated in FP32 in tensor memory.
//
// The steps are those of the FP32 kernel (cdd_kernels.cu): unpack the int8
// segment, forward transform, multiply by the chirp function (Sec. 2.1 Eq. 3
// times the Sec. 2.2 taper), inverse transform, discard the overlap
// (Sec. 2.2), detect and integrate (Sec. 3.1) and store aligned (Sec. 1.2).
// Only the butterflies move: each radix pass is a matrix product of the
// groups' points with the real form of the R-point DFT matrix (the layouts,
// scaling and index maps are in cdd_tc_layout.h).  The CUDA cores keep the
// unpack, the twiddles between passes, the hi/lo split, the chirp and the
// epilogue.
//
// One CTA per SM runs two independent pipelines of 256 threads.  Per segment
// and pipeline, six passes: the threads write a pass's operands into shared
// memory, one thread issues the products in two halves of the tiles, each
// committed to one of the pipeline's two mbarriers; every thread waits on the
// one that covers its rows (bounded: after one second the kernel records an
// error and stops), reads them from tensor memory and writes the next pass's
// operands, so the first half's rows are read while the second half runs.  The two pipelines interleave,
// so one computes on the CUDA cores while the other's products run.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cdd.h"
#include "cdd_fft.cuh"
#include "cdd_internal.h"
#include "cdd_passes.cuh"
#include "cdd_tc_layout.h"

namespace cdd {

namespace {

using namespace passes;
using namespace tc;

// ------------------------------------------------------------------ PTX

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// Test phase `parity`; the thread may sleep in the instruction for up to
// kSuspendNs (it wakes as soon as the phase completes), so a waiting warp
// does not spin on the issue slots.
constexpr uint32_t kSuspendNs = 20000;
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of an mbarrier, for at most one second.
constexpr uint64_t kWaitLimitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > kWaitLimitNs) return false;
  return true;
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D (tensor memory) (+)= A (shared) * B (shared)^T, kind::f16, one CTA.
__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
// Arrive on the mbarrier once every product this thread issued has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

#define CDD_O4(a, i) "=r"(a[i]), "=r"(a[i + 1]), "=r"(a[i + 2]), "=r"(a[i + 3])
#define CDD_O32(a) CDD_O4(a, 0), CDD_O4(a, 4), CDD_O4(a, 8), CDD_O4(a, 12), CDD_O4(a, 16), CDD_O4(a, 20), \
                   CDD_O4(a, 24), CDD_O4(a, 28)
#define CDD_IO4(a, i) "+r"(a[i]), "+r"(a[i + 1]), "+r"(a[i + 2]), "+r"(a[i + 3])
#define CDD_IO32(a) CDD_IO4(a, 0), CDD_IO4(a, 4), CDD_IO4(a, 8), CDD_IO4(a, 12), CDD_IO4(a, 16), \
                    CDD_IO4(a, 20), CDD_IO4(a, 24), CDD_IO4(a, 28)

// 32 consecutive 32-bit columns of this thread's lane (32x32b shape: lane i of
// the warp reads lane lane_base + i of tensor memory).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : CDD_O32(r)
      : "r"(taddr));
}
// Wait for the loads; the registers pass through the statement, so no use of
// them can be scheduled before the wait.
__device__ __forceinline__ void tmem_wait(uint32_t (&a)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" : CDD_IO32(a)::"memory");
}
__device__ __forceinline__ void tmem_wait(uint32_t (&a)[32], uint32_t (&b)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" : CDD_IO32(a), CDD_IO32(b)::"memory");
}

// Named barrier over the n threads of a pipeline that also ORs a flag.
__device__ __forceinline__ bool bar_or(int id, int n, bool flag) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)flag), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

// ------------------------------------------------------------------ operands

// (re, im) -> one 32-bit word of two halves, re in the low half, rounded to nearest
template <bool BF>
__device__ __forceinline__ uint32_t pack_rn(float re, float im) {
  uint32_t r;
  if constexpr (BF) asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(im), "f"(re));
  else asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(im), "f"(re));
  return r;
}
template <bool BF>
__device__ __forceinline__ float2 unpack_h2(uint32_t h) {
  if constexpr (BF) {
    return make_float2(__uint_as_float(h << 16), __uint_as_float(h & 0xFFFF0000u));
  } else {
    float lo, hi;
    asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\tcvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, h;\n\t}"
        : "=f"(lo), "=f"(hi)
        : "r"(h));
    return make_float2(lo, hi);
  }
}
// hi = round(v); lo = round(v - hi) (the residual is exact in FP32)
template <bool BF, bool SPLIT>
__device__ __forceinline__ void split(float2 v, uint32_t& hi, uint32_t& lo) {
  hi = pack_rn<BF>(v.x, v.y);
  if constexpr (SPLIT) {
    const float2 d = sub2(v, unpack_h2<BF>(hi));
    lo = pack_rn<BF>(d.x, d.y);
  }
}
// int8 pair (re, im) in the low 16 bits -> two halves, exactly.  FP16: the
// bytes biased to unsigned become the mantissa of 1024 (0x64xx), minus 1152.
template <bool BF>
__device__ __forceinline__ uint32_t int8_pair(uint32_t raw16) {
  if constexpr (BF) {
    const float2 f = unpack_i8x2(raw16);
    return pack_rn<true>(f.x, f.y);
  } else {
    const uint32_t h = __byte_perm(raw16 ^ 0x8080u, 0x64646464u, 0x5140);
    uint32_t r;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(h), "r"(0x64806480u));
    return r;
  }
}

// The R-point forward DFT matrix / R in the layout of cdd_tc_layout.h: rows
// 0..2R-1 the values rounded to the operand type, rows 2R..4R-1 the residual.
template <int R, bool BF>
__device__ void build_dft(uint8_t* b, int tid, int nthreads) {
  for (int e = tid; e < 4 * R * 2 * R; e += nthreads) {
    const int n = e / (2 * R), kk = e % (2 * R);
    const int n0 = n % (2 * R);
    double sn, cs;
    sincospi(2.0 * dft_m(R, n0, kk) / R, &sn, &cs);
    double v = dft_is_sin(n0, kk) ? sn : cs;
    if (dft_negative(n0, kk)) v = -v;
    v /= R;
    uint16_t hi, lo;
    if constexpr (BF) {
      const uint32_t h = pack_rn<true>((float)v, 0.f) & 0xFFFFu;
      const float hv = __uint_as_float(h << 16);
      hi = (uint16_t)h;
      lo = (uint16_t)(pack_rn<true>((float)(v - (double)hv), 0.f) & 0xFFFFu);
    } else {
      const uint32_t h = pack_rn<false>((float)v, 0.f) & 0xFFFFu;
      const float hv = unpack_h2<false>(h).x;
      hi = (uint16_t)h;
      lo = (uint16_t)(pack_rn<false>((float)(v - (double)hv), 0.f) & 0xFFFFu);
    }
    *reinterpret_cast<uint16_t*>(b + b_off(R, n, kk)) = n < 2 * R ? hi : lo;
  }
}

template <int PREC>
struct TcCfg {
  static constexpr bool SPLIT = PREC == CDD_PRECISION_FP16X2 || PREC == CDD_PRECISION_BF16X2;
  static constexpr bool BF = PREC == CDD_PRECISION_BF16 || PREC == CDD_PRECISION_BF16X2;
  static constexpr int PIPES = 2;
  static constexpr int THREADS = PIPES * kT;
  static constexpr int PIPE_BYTES = (SPLIT ? 2 : 1) * kRegion;    // operands hi (and lo)
  static constexpr int OFF_B32 = PIPES * PIPE_BYTES;
  static constexpr int OFF_B16 = OFF_B32 + b_bytes(32);
  static constexpr int TW_LEN = PassPlan<kLogN>::TW_LEN;
  static constexpr int OFF_TW = OFF_B16 + b_bytes(16);
  static constexpr int OFF_BAR = OFF_TW + tw_slots(TW_LEN) * (int)sizeof(float2);
  static constexpr int OFF_TMEM = OFF_BAR + 16 * PIPES;          // two mbarriers per pipeline
  static constexpr int SMEM = OFF_TMEM + 16;
  static constexpr int TMEM_COLS = SPLIT ? 512 : 256;             // per CTA; half per pipeline
  static_assert(SMEM <= 232448, "shared memory of one CTA");
  static_assert(kRegion >= (kN + kN / 32) * 4, "the power buffer of the epilogue fits an operand region");
};

// The R outputs e0 .. e0 + 15 of this thread's row (sum of the [hi | lo] halves).
template <int R, bool SPLIT>
__device__ __forceinline__ void row16(uint32_t trow, int e0, float2 (&v)[16]) {
  uint32_t r[32];
  tmem_ld32(trow + 2 * e0, r);
  if constexpr (SPLIT) {
    uint32_t q[32];
    tmem_ld32(trow + 2 * R + 2 * e0, q);
    tmem_wait(r, q);
#pragma unroll
    for (int i = 0; i < 16; ++i)
      v[i] = add2(make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1])),
                  make_float2(__uint_as_float(q[2 * i]), __uint_as_float(q[2 * i + 1])));
  } else {
    tmem_wait(r);
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
  }
}

// The products of half h of one pass: for each of its tiles of 128 rows and
// each k-step of 16 values, A_hi * [B_hi | B_lo] (N = 4R; N = 2R without
// the split) and, with `lo`, A_lo * B_hi into the first 2R columns; then a
// commit to the half's mbarrier, so the rows of the first half can be read
// while the second half runs.
template <int R, bool BF, bool SPLIT>
__device__ __forceinline__ void issue_half(uint32_t tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b, Lay L,
                                           int tiles, bool lo, int h, uint32_t bar) {
  constexpr int CW = tile_cols(R, SPLIT);
  const uint32_t id_hi = idesc_f16(128, CW, BF), id_lo = idesc_f16(128, 2 * R, BF);
  const int half = tiles / 2;
  for (int tt = h * half; tt < (h + 1) * half; ++tt) {
#pragma unroll
    for (int s = 0; s < 2 * R / 16; ++s) {
      const uint64_t bd = smem_desc(b + s * b_ks(R), kLboB, kSboB);
      const uint32_t aoff = tt * L.ts + s * L.ks;
      mma_f16(tmem + tt * CW, smem_desc(a_hi + aoff, L.lbo, L.sbo), bd, id_hi, s > 0);
      if (SPLIT && lo) mma_f16(tmem + tt * CW, smem_desc(a_lo + aoff, L.lbo, L.sbo), bd, id_lo, 1u);
    }
  }
  mma_commit(bar);
}

__device__ __forceinline__ int tc_work_chan(const OlsArgs& a, int w) { return w / a.s_count; }
__device__ __forceinline__ int tc_work_seg(const OlsArgs& a, int w) { return a.s_begin + w % a.s_count; }

// Ask L2 for the channel-major input rows and the chirp row of work item w
// (whole 16-byte blocks inside the rows the segment reads).
__device__ __forceinline__ void tc_prefetch(const OlsArgs& a, int w) {
  const int k = tc_work_chan(a, w);
  const long long s = tc_work_seg(a, w);
  long long r0 = s * a.hop - a.n_ov;
  const long long r1 = r0 + kN;
  if (r0 < 0) r0 = 0;
  const char* row = reinterpret_cast<const char*>(a.in_cm + (long long)k * a.rows);
  const uintptr_t lo = (reinterpret_cast<uintptr_t>(row + 2 * r0) + 15) & ~uintptr_t(15);
  const uintptr_t hi = reinterpret_cast<uintptr_t>(row + 2 * r1) & ~uintptr_t(15);
  if (hi > lo) prefetch_l2(reinterpret_cast<const void*>(lo), (uint32_t)(hi - lo));
  prefetch_l2(a.chirp + (size_t)k * kN, (uint32_t)(kN * sizeof(float2)));
}

template <int PREC>
__global__ void __launch_bounds__(TcCfg<PREC>::THREADS, 1) ols_tc_kernel(const OlsArgs a, int* err) {
  using C = TcCfg<PREC>;
  constexpr bool SPLIT = C::SPLIT, BF = C::BF;
  constexpr int CW32 = tile_cols(32, SPLIT), CW16 = tile_cols(16, SPLIT);
  constexpr float kPowScale = (float)(kOutScale * kOutScale);
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int pipe = tid / kT, lt = tid % kT;
  const uint32_t sb = smem_u32(smem);
  uint8_t* const ahi_p = smem + pipe * C::PIPE_BYTES;
  uint8_t* const alo_p = ahi_p + kRegion;
  const uint32_t a_hi = sb + pipe * C::PIPE_BYTES, a_lo = a_hi + kRegion;
  const uint32_t b32 = sb + C::OFF_B32, b16 = sb + C::OFF_B16;
  float2* const tws = reinterpret_cast<float2*>(smem + C::OFF_TW);
  const uint32_t bar0 = sb + C::OFF_BAR + 16 * pipe, bar1 = bar0 + 8;
  uint32_t* const tslot = reinterpret_cast<uint32_t*>(smem + C::OFF_TMEM);

  for (int i = tid; i < C::TW_LEN; i += C::THREADS) tws[tw_slot(i)] = __ldg(&a.tw[i]);
  {
    // the DFT matrices (radix 32 then 16), contiguous in the table and here
    const uint4* src = reinterpret_cast<const uint4*>(a.dft);
    uint4* dst = reinterpret_cast<uint4*>(smem + C::OFF_B32);
    for (int i = tid; i < (b_bytes(32) + b_bytes(16)) / 16; i += C::THREADS) dst[i] = __ldg(src + i);
  }
  if (tid == 0) {
    for (int p = 0; p < 2 * C::PIPES; ++p) mbar_init(sb + C::OFF_BAR + 8 * p, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tslot), C::TMEM_COLS);
    tmem_relinquish();
  }
  fence_async_shared();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot + (uint32_t)(pipe * (C::TMEM_COLS / C::PIPES));
  const uint32_t tlane = tmem + ((uint32_t)((warp & 3) * 32) << 16);   // this warp's lanes
  const int barid = 1 + pipe;
  uint32_t phase = 0;
  bool abort = false;

  // Barrier and products of one pass.  False once any thread of the pipeline
  // has given up on a wait (the pipeline then stops).  Both mbarriers complete
  // once per pass, so both phase bits flip at every pass after the first.
  bool issued = false;
  auto pass = [&](auto issue) -> bool {
    if (issued) phase ^= 3u;
    issued = true;
    fence_async_shared();
    tc_fence_before();
    if (bar_or(barid, kT, abort)) return false;
    if (lt == 0) {                       // one thread issues both halves, each with its commit
      tc_fence_after();                  // (a second issuing warp measured slower: it stalls its
      issue(0);                          // own share of the CUDA-core work)
      issue(1);
    }
    return true;
  };
  // Wait until the products of half h (0: the first half of the tiles) are in
  // tensor memory: one lane per warp waits, the warp then synchronises.
  auto wait_half = [&](int h) {
    bool ok = true;
    if ((lt & 31) == 0) ok = mbar_wait_bounded(h ? bar1 : bar0, (phase >> h) & 1u);
    __syncwarp();
    if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) {
      abort = true;
      if ((lt & 31) == 0) atomicOr(err, 1);
    }
    tc_fence_after();
  };

  const int work = a.n_chan * a.s_count;
  const int stride = gridDim.x * C::PIPES;
  for (int w = blockIdx.x * C::PIPES + pipe; w < work; w += stride) {
    if (lt == 0 && w + stride < work) tc_prefetch(a, w + stride);
    const int k = tc_work_chan(a, w);
    const int s = tc_work_seg(a, w);

    // ---- unpack: positions lt + 256 j of the segment -> row lt of the pass-0 operand
    {
      const long long row0 = (long long)s * a.hop - a.n_ov;
      const unsigned short* src = reinterpret_cast<const unsigned short*>(a.in_cm) + (long long)k * a.rows;
      unsigned short c[kR0];
      if (row0 >= 0) {
        const unsigned short* p0 = src + row0 + lt;
#pragma unroll
        for (int j = 0; j < kR0; ++j) c[j] = __ldg(p0 + kT * j);
      } else {
        const unsigned short* tail = reinterpret_cast<const unsigned short*>(a.tail_rd) + (long long)k * a.n_ov;
#pragma unroll
        for (int j = 0; j < kR0; ++j) {
          const long long row = row0 + lt + kT * j;
          c[j] = __ldg(row >= 0 ? src + row : tail + (row + a.n_ov));
        }
      }
      if (s == a.q - 1 && a.n_ov > 0) {           // keep this block's last n_ov samples
        unsigned short* tail_out = reinterpret_cast<unsigned short*>(a.tail_wr) + (long long)k * a.n_ov;
#pragma unroll
        for (int j = 0; j < kR0; ++j) {
          const int n = lt + kT * j;
          if (n >= kN - a.n_ov) tail_out[n - (kN - a.n_ov)] = c[j];
        }
      }
#pragma unroll
      for (int cc = 0; cc < kR0 / 4; ++cc) {
        uint4 q;
        q.x = int8_pair<BF>(c[4 * cc]);
        q.y = int8_pair<BF>(c[4 * cc + 1]);
        q.z = int8_pair<BF>(c[4 * cc + 2]);
        q.w = int8_pair<BF>(c[4 * cc + 3]);
        *reinterpret_cast<uint4*>(ahi_p + lay_off(lay0(), lt, 8 * cc)) = q;
      }
    }
    // ---- forward pass 0 (radix 32 over stride 256); the int8 input is exact: no lo product
    if (!pass([&](int h) { issue_half<32, BF, SPLIT>(tmem, a_hi, a_lo, b32, lay0(), 2, false, h, h ? bar1 : bar0); })) break;
    wait_half(lt >> 7);
    {
      const uint32_t trow = tlane + (uint32_t)((lt >> 7) * CW32);
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        float2 v[16];
        row16<32, SPLIT>(trow, 16 * hf, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int kq = 16 * hf + i;
          const float2 x = kq ? cmul(v[i], tws[tw_slot(f0_tw(lt, kq))]) : v[i];
          uint32_t h, l;
          split<BF, SPLIT>(x, h, l);
          const int off = lay_off(lay12(), f0_row(lt, kq), 2 * f0_elem(lt));
          *reinterpret_cast<uint32_t*>(ahi_p + off) = h;
          if constexpr (SPLIT) *reinterpret_cast<uint32_t*>(alo_p + off) = l;
        }
      }
    }
    // ---- forward pass 1 (radix 16 over stride 16)
    if (!pass([&](int h) { issue_half<16, BF, SPLIT>(tmem, a_hi, a_lo, b16, lay12(), 4, true, h, h ? bar1 : bar0); })) break;
#pragma unroll
    for (int gi = 0; gi < 2; ++gi) {
      const int g = lt + kT * gi;
      wait_half(gi);
      float2 v[16];
      row16<16, SPLIT>(tlane + (uint32_t)((g >> 7) * CW16), 0, v);
#pragma unroll
      for (int kq = 0; kq < 16; ++kq) {
        const float2 x = kq ? cmul(v[kq], tws[tw_slot(f1_tw(g, kq))]) : v[kq];
        uint32_t h, l;
        split<BF, SPLIT>(x, h, l);
        const int off = lay_off(lay12(), f1_row(g, kq), 2 * f1_elem(g));
        *reinterpret_cast<uint32_t*>(ahi_p + off) = h;
        if constexpr (SPLIT) *reinterpret_cast<uint32_t*>(alo_p + off) = l;
      }
    }
    // ---- forward pass 2 (radix 16, stride 1), then the chirp; the first
    // inverse pass works on the same groups, conjugated, so each thread
    // rewrites its own rows
    if (!pass([&](int h) { issue_half<16, BF, SPLIT>(tmem, a_hi, a_lo, b16, lay12(), 4, true, h, h ? bar1 : bar0); })) break;
    {
      const float4* ch4 = reinterpret_cast<const float4*>(a.chirp + (size_t)k * kN);
#pragma unroll
      for (int gi = 0; gi < 2; ++gi) {
        const int q = lt + kT * gi;
        wait_half(gi);
        float2 v[16];
        row16<16, SPLIT>(tlane + (uint32_t)((q >> 7) * CW16), 0, v);
        uint32_t hw[16], lw[16];
#pragma unroll
        for (int kq = 0; kq < 16; kq += 2) {
          const float4 cc = __ldg(ch4 + chirp4_index(q, kq));
          const float2 y0 = cmul(v[kq], make_float2(cc.x, cc.y));
          const float2 y1 = cmul(v[kq + 1], make_float2(cc.z, cc.w));
          split<BF, SPLIT>(make_float2(y0.x, -y0.y), hw[kq], lw[kq]);
          split<BF, SPLIT>(make_float2(y1.x, -y1.y), hw[kq + 1], lw[kq + 1]);
        }
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const int off = lay_off(lay12(), q, 8 * cc);
          *reinterpret_cast<uint4*>(ahi_p + off) = make_uint4(hw[4 * cc], hw[4 * cc + 1], hw[4 * cc + 2], hw[4 * cc + 3]);
          if constexpr (SPLIT)
            *reinterpret_cast<uint4*>(alo_p + off) = make_uint4(lw[4 * cc], lw[4 * cc + 1], lw[4 * cc + 2], lw[4 * cc + 3]);
        }
      }
    }
    // ---- inverse pass 2 (conjugated data)
    if (!pass([&](int h) { issue_half<16, BF, SPLIT>(tmem, a_hi, a_lo, b16, lay12(), 4, true, h, h ? bar1 : bar0); })) break;
#pragma unroll
    for (int gi = 0; gi < 2; ++gi) {
      const int q = lt + kT * gi;
      wait_half(gi);
      float2 v[16];
      row16<16, SPLIT>(tlane + (uint32_t)((q >> 7) * CW16), 0, v);
#pragma unroll
      for (int kq = 0; kq < 16; ++kq) {
        const float2 x = kq ? cmul(v[kq], tws[tw_slot(i2_tw(q, kq))]) : v[kq];
        uint32_t h, l;
        split<BF, SPLIT>(x, h, l);
        const int off = lay_off(lay12(), i2_row(q, kq), 2 * i2_elem(q));
        *reinterpret_cast<uint32_t*>(ahi_p + off) = h;
        if constexpr (SPLIT) *reinterpret_cast<uint32_t*>(alo_p + off) = l;
      }
    }
    // ---- inverse pass 1
    if (!pass([&](int h) { issue_half<16, BF, SPLIT>(tmem, a_hi, a_lo, b16, lay12(), 4, true, h, h ? bar1 : bar0); })) break;
#pragma unroll
    for (int gi = 0; gi < 2; ++gi) {
      const int g = lt + kT * gi;
      wait_half(gi);
      float2 v[16];
      row16<16, SPLIT>(tlane + (uint32_t)((g >> 7) * CW16), 0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float2 x = cmul(v[j], tws[tw_slot(i1_tw(g, j))]);
        uint32_t h, l;
        split<BF, SPLIT>(x, h, l);
        const int off = lay_off(lay0(), i1_row(g, j), 2 * i1_elem(g));
        *reinterpret_cast<uint32_t*>(ahi_p + off) = h;
        if constexpr (SPLIT) *reinterpret_cast<uint32_t*>(alo_p + off) = l;
      }
    }
    // ---- inverse pass 0 (radix 32): conj(y) / kOutScale at positions lt + 256 j
    if (!pass([&](int h) { issue_half<32, BF, SPLIT>(tmem, a_hi, a_lo, b32, lay0(), 2, true, h, h ? bar1 : bar0); })) break;
    float2 u[kR0];
    wait_half(lt >> 7);
    {
      const uint32_t trow = tlane + (uint32_t)((lt >> 7) * CW32);
      float2 v[16];
      row16<32, SPLIT>(trow, 0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) u[i] = v[i];
      row16<32, SPLIT>(trow, 16, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) u[16 + i] = v[i];
    }
    if (a.volt != nullptr) {
      const long long vbase = ((long long)k * a.q + s) * a.hop - a.n_ov;
      const float sc = (float)kOutScale;
#pragma unroll
      for (int j = 0; j < kR0; ++j) {
        const int n = lt + kT * j;
        if (n >= a.n_ov) a.volt[vbase + n] = make_float2(u[j].x * sc, -u[j].y * sc);
      }
    }

    // ---- detect, integrate (in lanes, or through the operand region), align
    const int na = a.n_avg;
    const bool in_lanes = na <= kR0 && na <= 32 && (na & (na - 1)) == 0;
    float* pw = reinterpret_cast<float*>(ahi_p);
    if (!in_lanes) {
#pragma unroll
      for (int j = 0; j < kR0; ++j) {
        const int n = lt + kT * j;
        pw[n + (n >> 5)] = fmaf(u[j].x, u[j].x, u[j].y * u[j].y);
      }
      if (bar_or(barid, kT, abort)) break;
    }
    const int n_int = a.hop / na;
    const int r = __ldg(&a.shift[k]);
    const long long gseg = a.g0 + (long long)s * n_int;
    float* outk = a.out + (size_t)k * a.n_out;
    float* ringk = a.ring + (size_t)k * a.ring_len;
    auto emit = [&](int m, float acc) {
      const long long gi = gseg + m;
      const long long dst = gi + r - a.g0;
      const float val = acc * kPowScale;
      if (dst < a.n_out) outk[dst] = val;
      else ringk[gi % a.ring_len] = val;
    };
    if (in_lanes) {
      integrate_in_lanes<kR0, kT>(u, lt, a.n_ov, na, emit);
    } else {
      for (int m = lt; m < n_int; m += kT) {
        const int n0 = a.n_ov + m * na;
        float acc = 0.f;
        for (int i = 0; i < na; ++i) acc += pw[(n0 + i) + ((n0 + i) >> 5)];
        emit(m, acc);
      }
      if (bar_or(barid, kT, abort)) break;       // the region is rewritten by the next segment
    }
    if (s == 0) {                                // block prefix: earlier blocks' samples
      const int lim = r < a.n_out ? r : a.n_out;
      for (int m = lt; m < lim; m += kT) {
        const long long src = a.g0 + m - r;
        outk[m] = src >= 0 ? ringk[src % a.ring_len] : 0.f;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(*tslot, C::TMEM_COLS);
  }
}

template <int PREC>
cudaError_t launch_tc_t(const OlsArgs& a, int* err, cudaStream_t s) {
  using C = TcCfg<PREC>;
  static bool attr_set[128] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  if (a.in_cm == nullptr || a.dft == nullptr) return cudaErrorInvalidValue;   // channel-major copy, DFT table
  if (!attr_set[dev]) {
    e = cudaFuncSetAttribute(ols_tc_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long work = (long long)a.n_chan * a.s_count;
  if (work <= 0) return cudaSuccess;
  const long long need = (work + C::PIPES - 1) / C::PIPES;
  const unsigned grid = (unsigned)(need < sms ? need : sms);
  ols_tc_kernel<PREC><<<grid, C::THREADS, C::SMEM, s>>>(a, err);
  return cudaGetLastError();
}

template <bool BF>
__global__ void dft_table_kernel(uint8_t* dft) {
  build_dft<32, BF>(dft, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
  build_dft<16, BF>(dft + b_bytes(32), blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

}  // namespace

size_t tc_dft_bytes() { return (size_t)(b_bytes(32) + b_bytes(16)); }

cudaError_t launch_tc_dft_table(int precision, void* dft, cudaStream_t s) {
  const bool bf = precision == CDD_PRECISION_BF16 || precision == CDD_PRECISION_BF16X2;
  if (bf) dft_table_kernel<true><<<16, 256, 0, s>>>(static_cast<uint8_t*>(dft));
  else dft_table_kernel<false><<<16, 256, 0, s>>>(static_cast<uint8_t*>(dft));
  return cudaGetLastError();
}

bool tc_supported(int logn, int precision) {
  return logn == kLogN && precision >= CDD_PRECISION_FP16 && precision <= CDD_PRECISION_BF16;
}

cudaError_t launch_ols_tc(int logn, int precision, const OlsArgs& a, int* err, cudaStream_t s) {
  if (logn != kLogN || err == nullptr) return cudaErrorInvalidValue;
  switch (precision) {
    case CDD_PRECISION_FP16: return launch_tc_t<CDD_PRECISION_FP16>(a, err, s);
    case CDD_PRECISION_FP16X2: return launch_tc_t<CDD_PRECISION_FP16X2>(a, err, s);
    case CDD_PRECISION_BF16X2: return launch_tc_t<CDD_PRECISION_BF16X2>(a, err, s);
    case CDD_PRECISION_BF16: return launch_tc_t<CDD_PRECISION_BF16>(a, err, s);
    default: return cudaErrorInvalidValue;
  }
}

double tc_chirp_scale() { return kChirpScale; }

}  // namespace cdd
