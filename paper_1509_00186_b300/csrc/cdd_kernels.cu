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
#include <cooperative_groups.h>

#include "cdd_fft.cuh"
#include "cdd_internal.h"
#include "cdd_passes.cuh"

namespace cdd {

namespace {

using namespace passes;

#ifndef CDD_PERSISTENT
#define CDD_PERSISTENT 1
#endif
constexpr bool kUsePersistent = CDD_PERSISTENT != 0;

// One overlap-save segment (channel k, segment s) by the T threads of a group:
// unpack and gather, forward passes, chirp, inverse passes, detection,
// integration and the aligned store.  `tw` is the whole twiddle table, in
// global memory or (SH) staged in shared memory; `sync` is the group's barrier.
template <int LOGN, bool CM, bool SH, class Sync>
__device__ __forceinline__ bool ols_segment(const OlsArgs& a, float2* buf, const float2* tw, int lt,
                                            bool active, int k, int s, Sync sync) {
  using PL = PassPlan<LOGN>;
  constexpr int N = PL::N;
  constexpr int T = PL::T;
  constexpr int R0 = PL::R(0);
  // ---- pass 0, forward: unpack and gather x[lt + T*j] of this segment
  float2* pb0 = buf + pad<LOGN>(lt);
  float2 v[R0];
  if (active) {
    const long long row0 = (long long)s * a.hop - a.n_ov;
    // element (row, k): row-major input [row][C], or the channel-major copy [k][row]
    const unsigned short* src = CM ? reinterpret_cast<const unsigned short*>(a.in_cm) + (long long)k * a.rows
                                   : reinterpret_cast<const unsigned short*>(a.in) + k;
    const long long rstride = CM ? 1 : a.n_chan;
    unsigned short c[R0];
    if (row0 >= 0) {                                // no sample from the previous block
      const unsigned short* p0 = src + (row0 + lt) * rstride;
#pragma unroll
      for (int j = 0; j < R0; ++j) c[j] = __ldg(p0 + (long long)T * j * rstride);
    } else {
      const unsigned short* tail = reinterpret_cast<const unsigned short*>(a.tail_rd) + (long long)k * a.n_ov;
#pragma unroll
      for (int j = 0; j < R0; ++j) {
        const long long row = row0 + lt + T * j;
        c[j] = __ldg(row >= 0 ? src + row * rstride : tail + (row + a.n_ov));
      }
    }
    if (s == a.q - 1 && a.n_ov > 0) {             // keep this block's last n_ov samples
      unsigned short* tw_out = reinterpret_cast<unsigned short*>(a.tail_wr) + (long long)k * a.n_ov;
#pragma unroll
      for (int j = 0; j < R0; ++j) {
        const int n = lt + T * j;
        if (n >= N - a.n_ov) tw_out[n - (N - a.n_ov)] = c[j];
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

  // When the last two radices are equal, the last forward pass before the
  // chirp pass, the chirp pass and the first inverse pass after it touch each
  // sub-problem of R_{P-2} * R_{P-1} points with the same R_{P-1} consecutive
  // threads (a part of one warp), so those hand-offs need only a warp barrier.
  constexpr bool kWarpMid = PL::P >= 3 && PL::R(PL::P - 2) == PL::RL && PL::RL <= 32;
  auto mid_sync = [&] {
    if constexpr (kWarpMid) __syncwarp();
    else sync();
  };
  static_for<1, PL::P - 1>([&](auto P_) {
    constexpr int p = decltype(P_)::value;
    if (active) fwd_pass<LOGN, p, SH>(buf, tw, lt);
    if constexpr (p == PL::P - 2) mid_sync();
    else sync();
  });

  if (active) chirp_pass<LOGN>(buf, a.chirp + (size_t)k * N, lt);
  if constexpr (PL::P >= 3) mid_sync();
  else sync();

  static_for<1, PL::P - 1>([&](auto I_) {
    if (active) inv_pass<LOGN, PL::P - 1 - decltype(I_)::value, SH>(buf, tw, lt);
    sync();
  });

  // ---- pass 0, inverse: natural-order voltages v[j] = z[lt + T*j]
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
    if (a.volt != nullptr) {
      const long long vbase = ((long long)k * a.q + s) * a.hop - a.n_ov;
#pragma unroll
      for (int j = 0; j < R0; ++j) {
        const int n = lt + T * j;
        if (n >= a.n_ov) a.volt[vbase + n] = v[j];
      }
    }
  }
  sync();                       // every thread has read buf: reuse it
  // Integration in registers when each window is n_avg neighbouring lanes of
  // one warp (n_avg a power of two, at most 32 and at most R0); otherwise the
  // detected samples go through shared memory.  N = 16384 (one 512-thread CTA
  // per SM, 128 registers) keeps the shared-memory form: the register form
  // spills there and measured slower.
  const int na = a.n_avg;
  bool in_lanes = false;
  if constexpr (T % 32 == 0 && LOGN <= 13) in_lanes = na <= R0 && na <= 32 && (na & (na - 1)) == 0;
  float* pw = reinterpret_cast<float*>(buf);
  if (!in_lanes) {
    if (active) {
#pragma unroll
      for (int j = 0; j < R0; ++j) {
        const int n = lt + T * j;
        pw[n + (n >> 5)] = fmaf(v[j].x, v[j].x, v[j].y * v[j].y);   // one spare word per 32
      }
    }
    sync();
  }

  if (active) {
    const int n_int = a.hop / na;
    const int r = __ldg(&a.shift[k]);
    const long long gseg = a.g0 + (long long)s * n_int;
    float* outk = a.out + (size_t)k * a.n_out;
    float* ringk = a.ring + (size_t)k * a.ring_len;
    auto emit = [&](int m, float acc) {
      const long long gi = gseg + m;              // stream index of this output
      const long long dst = gi + r - a.g0;        // its aligned index in this block
      if (dst < a.n_out) outk[dst] = acc;
      else ringk[gi % a.ring_len] = acc;
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
    if (s == 0) {                                 // block prefix: earlier blocks' samples
      const int lim = r < a.n_out ? r : a.n_out;
      for (int m = lt; m < lim; m += T) {
        const long long src = a.g0 + m - r;
        outk[m] = src >= 0 ? ringk[src % a.ring_len] : 0.f;
      }
    }
  }
  return !in_lanes;               // buf (the power samples) read since the last barrier
}

template <int LOGN, bool CM>
__global__ void __launch_bounds__(Cfg<LOGN>::THREADS, Cfg<LOGN>::MINB)
ols_kernel(const OlsArgs a) {
  using PL = PassPlan<LOGN>;
  using CF = Cfg<LOGN>;
  constexpr int T = PL::T;
  static_assert(PL::S(0) == T, "pass 0 stride must equal the threads per transform");
  extern __shared__ __align__(16) float2 smem[];
  const int g = threadIdx.x / T;
  const int lt = threadIdx.x % T;
  float2* buf = smem + g * CF::SEG_F2;
  const int w = blockIdx.x * CF::G + g;        // n_chan * q < 2^31 (checked by the plan)
  const bool active = w < a.n_chan * a.s_count;
  const int k = active ? w % a.n_chan : 0;     // channel fastest: neighbouring CTAs
  const int s = active ? a.s_begin + w / a.n_chan : 0;   // share the input rows in L2
  ols_segment<LOGN, CM, false>(a, buf, a.tw, lt, active, k, s, [] { __syncthreads(); });
}

// Persistent form for N = 8192: one CTA per SM with two groups of 256
// threads, each looping over segments with its own named barrier, and the whole
// twiddle table staged once in shared memory (in L1 it was evicted by the
// streaming chirp rows).  Reads the channel-major block.
template <int LOGN>
struct Persist {
  using PL = PassPlan<LOGN>;
  static constexpr int GROUPS = 2;
  static constexpr int THREADS = GROUPS * PL::T;
  static constexpr size_t SMEM = (size_t(PL::TW_LEN) + size_t(GROUPS) * padded_len<LOGN>()) * sizeof(float2);
};

#ifndef CDD_PREFETCH
#define CDD_PREFETCH 1
#endif

// Ask L2 for the channel-major input rows and the chirp row of work item w,
// restricted to the 16-byte blocks that lie wholly inside the rows the
// segment reads (so every prefetched byte is one the kernel will load).
#ifndef CDD_SEGMENT_FASTEST
#define CDD_SEGMENT_FASTEST 1
#endif
// Work item w -> (channel, segment): segment-fastest keeps a channel's chirp
// row in L2 across its segments (1% faster than channel-fastest at N = 8192).
__device__ __forceinline__ int work_chan(const OlsArgs& a, int w) {
  return CDD_SEGMENT_FASTEST ? w / a.s_count : w % a.n_chan;
}
__device__ __forceinline__ int work_seg(const OlsArgs& a, int w) {
  return a.s_begin + (CDD_SEGMENT_FASTEST ? w % a.s_count : w / a.n_chan);
}

template <int LOGN>
__device__ __forceinline__ void prefetch_work(const OlsArgs& a, int w) {
  constexpr int N = 1 << LOGN;
  const int k = work_chan(a, w);
  const long long s = work_seg(a, w);
  long long r0 = s * a.hop - a.n_ov;
  const long long r1 = r0 + N;                  // <= (s + 1) * hop <= rows
  if (r0 < 0) r0 = 0;
  const char* row = reinterpret_cast<const char*>(a.in_cm + (long long)k * a.rows);
  const uintptr_t lo = (reinterpret_cast<uintptr_t>(row + 2 * r0) + 15) & ~uintptr_t(15);
  const uintptr_t hi = reinterpret_cast<uintptr_t>(row + 2 * r1) & ~uintptr_t(15);
  if (hi > lo) prefetch_l2(reinterpret_cast<const void*>(lo), (uint32_t)(hi - lo));
  prefetch_l2(a.chirp + (size_t)k * N, (uint32_t)(N * sizeof(float2)));
}

template <int LOGN>
__global__ void __launch_bounds__(Persist<LOGN>::THREADS, 1)
ols_persistent_kernel(const OlsArgs a) {
  using PL = PassPlan<LOGN>;
  using PS = Persist<LOGN>;
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
  const int work = a.n_chan * a.s_count;
  const int stride = gridDim.x * PS::GROUPS;
  for (int w = blockIdx.x * PS::GROUPS + g; w < work; w += stride) {
    if (CDD_PREFETCH && lt == 0 && w + stride < work) prefetch_work<LOGN>(a, w + stride);
    const int k = work_chan(a, w);
    const int s = work_seg(a, w);
    if (ols_segment<LOGN, true, true>(a, buf, tws, lt, true, k, s, sync))
      sync();                                  // buf is rewritten by the next segment
  }
}


// A cluster barrier that publishes nothing and follows no memory access:
// arrive without the release fence (the wait still acquires).  Used where the
// CTAs only need to know that every CTA of the cluster has started.
__device__ __forceinline__ void cluster_barrier_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}

// ------------------------------------------------------------------ clusters
//
// N = CL * 2^LOGS (32768 and 65536) does not fit one SM's shared memory, so a
// cluster of CL CTAs holds one segment, 2^LOGS points per CTA (2^13: the
// 256-thread sub-transform of the single-CTA kernels, three CTAs per SM; CL = 4
// and 8).  A radix-CL pass
// across the cluster (DIF; inputs straight from global memory, outputs written
// through distributed shared memory) leaves CTA r with the independent
// sub-transform r (bins r + CL*b).  Each CTA then runs the single-CTA forward
// passes, chirp pass and inverse passes on it; the inverse radix-CL pass reads
// the CL sub-results back across the cluster and the epilogue detects,
// integrates and stores the CTA's quarter of the butterflies.
// Cross-pass twiddles w_N^{t kk}, kk = 1 .. CL-1, of butterfly t: w^t and (for
// CL = 8) w^{4t} from the table, the rest as products at most 3 deep, instead
// of CL - 1 loads from a table of (CL-1) x 8192 entries that lives in L2
// (N = 65536: 2.65 against 2.73 ms per block).
template <int CL, int NS>
__device__ __forceinline__ void cross_twiddles(const float2* __restrict__ twx, int t, float2 (&w)[CL]) {
  static_assert(CL == 2 || CL == 4 || CL == 8, "cluster sizes 2, 4, 8");
  w[1] = __ldg(&twx[t]);
  if constexpr (CL >= 4) {
    w[2] = cmul(w[1], w[1]);
    w[3] = cmul(w[2], w[1]);
  }
  if constexpr (CL == 8) {
    w[4] = __ldg(&twx[3 * NS + t]);
    w[5] = cmul(w[4], w[1]);
    w[6] = cmul(w[4], w[2]);
    w[7] = cmul(w[4], w[3]);
  }
}

template <int LOGS, int CL>
// Three 256-thread CTAs per SM (80 registers): measured faster than two
// (N = 32768: 2.85 against 3.02 ms per block; N = 65536: 3.13 against 3.16).
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(PassPlan<LOGS>::T, PassPlan<LOGS>::T <= 256 ? 3 : 1)
ols_cluster_kernel(const OlsArgs a) {
  namespace cg = cooperative_groups;
  using PL = PassPlan<LOGS>;
  constexpr int NS = PL::N;
  constexpr int N = NS * CL;
  constexpr int T = PL::T;
  constexpr int NB = NS / CL;            // cross-pass butterflies of this CTA
  constexpr int PERX = NB / T;           // ... per thread
  static_assert(PERX * T == NB, "cross pass must split evenly over the threads");
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  extern __shared__ __align__(16) float2 smem[];
  float2* buf = smem;
  const int lt = threadIdx.x;
  // the cluster's buffers as 32-bit shared::cluster addresses (one register each)
  uint32_t rbuf[CL];
  {
    const uint32_t local = (uint32_t)__cvta_generic_to_shared(buf);
#pragma unroll
    for (int j = 0; j < CL; ++j) asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rbuf[j]) : "r"(local), "r"(j));
  }
  auto dsm_st = [](uint32_t addr, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
  };
  auto dsm_ld = [](uint32_t addr) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
  };
  const float2* twx = a.tw + PL::TW_LEN;
  const int na = a.n_avg;
  constexpr int U = PERX * CL;
  const bool in_lanes = U == 32 && na <= 32 && (na & (na - 1)) == 0;
  cluster_barrier_relaxed();             // every CTA of the cluster has started: DSMEM is live
  // One segment per cluster (a persistent form that loops over segments
  // measured slower for clusters of eight and no faster for four).
  auto segment = [&](const int w) {
    // segment-fastest, so that a channel's chirp row (512 KB at N = 65536;
    // the whole table exceeds L2) serves its consecutive segments from L2,
    // and each CTA asks L2 for its slice of that row before the forward
    // passes: 2.94 against 3.13 ms per N = 65536 block at three CTAs per SM
    // (at two CTAs per SM both measured 0.3-2% slower)
    const int k = w / a.s_count;
    const int s = a.s_begin + w % a.s_count;
    if (lt < 8)
      prefetch_l2(a.chirp + (size_t)k * N + (size_t)rank * NS + lt * (NS / 8), (uint32_t)(NS / 8 * sizeof(float2)));
    // ... and for the input rows of the cluster one resident wave ahead
    // (three CTAs per SM), this CTA's contiguous 1/CL of them, whole 16-byte
    // blocks only (about 1% faster)
    if (lt == 8) {
      unsigned n_sm;
      asm("mov.u32 %0, %%nsmid;" : "=r"(n_sm));
      const int w2 = w + (int)(n_sm * 3 / CL);
      if (w2 < a.n_chan * a.s_count) {
        const int k2 = w2 / a.s_count;
        const long long s2 = a.s_begin + w2 % a.s_count;
        long long r0 = s2 * a.hop - a.n_ov + (long long)rank * NS;
        long long r1 = r0 + NS;
        if (r0 < 0) r0 = 0;
        if (r1 > a.rows) r1 = a.rows;
        const char* row = reinterpret_cast<const char*>(a.in_cm + (long long)k2 * a.rows);
        const uintptr_t lo = (reinterpret_cast<uintptr_t>(row + 2 * r0) + 15) & ~uintptr_t(15);
        const uintptr_t hi = reinterpret_cast<uintptr_t>(row + 2 * r1) & ~uintptr_t(15);
        if (hi > lo) prefetch_l2(reinterpret_cast<const void*>(lo), (uint32_t)(hi - lo));
      }
    }

    // ---- cross pass, forward: x[t + NS*j] -> DFT_CL -> w_N^{t*kk} -> CTA kk, index t
    {
      const long long row0 = (long long)s * a.hop - a.n_ov;
      const unsigned short* src = reinterpret_cast<const unsigned short*>(a.in_cm) + (long long)k * a.rows;
      const unsigned short* tail = reinterpret_cast<const unsigned short*>(a.tail_rd) + (long long)k * a.n_ov;
      unsigned short* tail_out = reinterpret_cast<unsigned short*>(a.tail_wr) + (long long)k * a.n_ov;
      const bool last = (s == a.q - 1) && a.n_ov > 0;
#pragma unroll 2
      for (int i = 0; i < PERX; ++i) {
        const int t = rank * NB + lt + i * T;
        unsigned short c[CL];
#pragma unroll
        for (int j = 0; j < CL; ++j) {
          const long long row = row0 + t + (long long)NS * j;
          c[j] = __ldg(row >= 0 ? src + row : tail + (row + a.n_ov));
        }
        float2 v[CL];
#pragma unroll
        for (int j = 0; j < CL; ++j) {
          const int n = t + NS * j;
          if (last && n >= N - a.n_ov) tail_out[n - (N - a.n_ov)] = c[j];
          v[j] = unpack_i8x2(c[j]);
        }
        dft<CL, -1>(v);
        float2 wx[CL];
        cross_twiddles<CL, NS>(twx, t, wx);
#pragma unroll
        for (int kk = 1; kk < CL; ++kk) v[kk] = cmul(v[kk], wx[kk]);
#pragma unroll
        for (int kk = 0; kk < CL; ++kk) dsm_st(rbuf[kk] + 8u * (uint32_t)pad<LOGS>(t), v[kk]);
      }
    }
    cluster.sync();

    // ---- sub-transform r of 2^LOGS points, all in this CTA (warp barriers
    // around the chirp pass when the last two radices are equal)
    constexpr bool kWarpMid = PL::P >= 3 && PL::R(PL::P - 2) == PL::RL && PL::RL <= 32;
    static_for<0, PL::P - 1>([&](auto P_) {
      constexpr int p = decltype(P_)::value;
      fwd_pass<LOGS, p, false, p == 0 && kRecPass0<LOGS, false>>(buf, a.tw, lt);
      if constexpr (kWarpMid && p == PL::P - 2) __syncwarp();
      else __syncthreads();
    });
    chirp_pass<LOGS>(buf, a.chirp + (size_t)k * N + (size_t)rank * NS, lt);
    if constexpr (kWarpMid) __syncwarp();
    else __syncthreads();
    static_for<0, PL::P - 1>([&](auto I_) {
      constexpr int pi = PL::P - 2 - decltype(I_)::value;
      inv_pass<LOGS, pi, false, pi == 0 && kRecPass0<LOGS, false>>(buf, a.tw, lt);
      __syncthreads();
    });
    cluster.sync();

    // ---- cross pass, inverse: u_kk[t] from CTA kk -> w_N^{-t*kk} -> IDFT_CL -> z[t + NS*j]
    float2 z[PERX][CL];
#pragma unroll
    for (int i = 0; i < PERX; ++i) {
      const int t = rank * NB + lt + i * T;
#pragma unroll
      for (int kk = 0; kk < CL; ++kk) z[i][kk] = dsm_ld(rbuf[kk] + 8u * (uint32_t)pad<LOGS>(t));
      float2 wx[CL];
      cross_twiddles<CL, NS>(twx, t, wx);
#pragma unroll
      for (int kk = 1; kk < CL; ++kk) z[i][kk] = cmulc(z[i][kk], wx[kk]);
      dft<CL, 1>(z[i]);
      if (a.volt != nullptr) {
        const long long vbase = ((long long)k * a.q + s) * a.hop - a.n_ov;
#pragma unroll
        for (int j = 0; j < CL; ++j) {
          const int n = t + NS * j;
          if (n >= a.n_ov) a.volt[vbase + n] = z[i][j];
        }
      }
    }
    // the reads of the other CTAs' buffers are done: arrive (release orders
    // them before it); wait only before this CTA's buffer is rewritten or the
    // CTA exits, so the epilogue runs while the cluster catches up
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");

    const int n_int = a.hop / a.n_avg;
    const int r = __ldg(&a.shift[k]);
    const long long gseg = a.g0 + (long long)s * n_int;
    float* outk = a.out + (size_t)k * a.n_out;
    float* ringk = a.ring + (size_t)k * a.ring_len;
    auto emit = [&](int n0, float acc) {      // the window starting at sample n0 >= n_ov
      const long long gi = gseg + (n0 - a.n_ov) / a.n_avg;
      const long long dst = gi + r - a.g0;
      if (dst < a.n_out) outk[dst] = acc;
      else ringk[gi % a.ring_len] = acc;
    };
    if (in_lanes) {
      // ---- detect and integrate across lanes: a thread holds samples
      // n = NS*j + rank*NB + lt + i*T, so a window is na neighbouring lanes
      float u[U];
#pragma unroll
      for (int i = 0; i < PERX; ++i)
#pragma unroll
        for (int j = 0; j < CL; ++j) u[i * CL + j] = fmaf(z[i][j].x, z[i][j].x, z[i][j].y * z[i][j].y);
      const int lane = lt & 31;
      auto windows = [&](auto NA_) {
        constexpr int NA = decltype(NA_)::value;
        constexpr int V = U / NA;
        lane_window_sums<U, NA>(u, lane);
        const int lo = lane & (NA - 1);
#pragma unroll
        for (int q = 0; q < V; ++q) {
          const int jj = V * lo + q;                    // flattened (i, j) of this sum
          const int n0 = NS * (jj % CL) + rank * NB + (lt - lo) + (jj / CL) * T;
          if (n0 >= a.n_ov) emit(n0, u[q]);
        }
      };
      switch (na) {
        case 1: windows(std::integral_constant<int, 1>{}); break;
        case 2: windows(std::integral_constant<int, 2>{}); break;
        case 4: windows(std::integral_constant<int, 4>{}); break;
        case 8: windows(std::integral_constant<int, 8>{}); break;
        case 16: windows(std::integral_constant<int, 16>{}); break;
        default: windows(std::integral_constant<int, 32>{}); break;
      }
    } else {
      // ---- detect into this CTA's buffer: (j, tt) -> j*NB + tt, one spare word per 32
      asm volatile("barrier.cluster.wait.aligned;" ::: "memory");   // nobody reads it any more
      float* pw = reinterpret_cast<float*>(buf);
#pragma unroll
      for (int i = 0; i < PERX; ++i) {
#pragma unroll
        for (int j = 0; j < CL; ++j) {
          const int nl = j * NB + lt + i * T;
          pw[nl + (nl >> 5)] = fmaf(z[i][j].x, z[i][j].x, z[i][j].y * z[i][j].y);
        }
      }
      __syncthreads();
      // ---- integrate, discard, align: n in [NS*j + rank*NB, NS*j + (rank+1)*NB)
      const int per_j = NB / na;
      for (int e = lt; e < CL * per_j; e += T) {
        const int j = e / per_j, mm = e % per_j;
        const int n0 = NS * j + rank * NB + mm * na;
        if (n0 < a.n_ov) continue;                          // the overlap is discarded
        const int nl0 = j * NB + mm * na;
        float acc = 0.f;
        for (int i = 0; i < na; ++i) acc += pw[(nl0 + i) + ((nl0 + i) >> 5)];
        emit(n0, acc);
      }
    }
    if (s == 0 && rank == 0) {
      const int lim = r < a.n_out ? r : a.n_out;
      for (int m = lt; m < lim; m += T) {
        const long long src = a.g0 + m - r;
        outk[m] = src >= 0 ? ringk[src % a.ring_len] : 0.f;
      }
    }
  };
  segment((int)(blockIdx.x / CL));
  if (in_lanes) asm volatile("barrier.cluster.wait.aligned;" ::: "memory");   // then exit
}

// Chirp table for a transform of CL * 2^LOGS points held as CL sub-transforms
// of 2^LOGS (CL = 1: one CTA).  Entry (k, r, idx) multiplies the bin that
// sub-transform r holds at table index idx after its forward passes:
// bin = r + CL * position_to_bin(pos), pos = chirp_pos<NG>(idx, R_last).
template <int LOGS, int CL>
__global__ void chirp_table_kernel(float2* chirp, int n_chan, double f_base, double chan_bw,
                                   double dm, int taper, int sideband, double scale) {
  using PL = PassPlan<LOGS>;
  constexpr int NS = PL::N;
  constexpr int N = NS * CL;
  constexpr int NG = NS / PL::RL;
  const long long total = (long long)n_chan * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / N);
    const int rem = (int)(e % N);
    const int r = rem / NS, idx = rem % NS;
    const int pos = passes::chirp_pos<NG>(idx, PL::RL);
    const int bin = r + CL * position_to_bin<LOGS>(pos);
    // a lower-sideband channel is the conjugate mirror: bin j sits where the
    // upper-sideband bin -j does (the Nyquist bin is its own mirror)
    const int obin = sideband > 0 ? bin : (N - bin) % N;
    const int sbin = obin < N / 2 ? obin : obin - N;
    const double f_lo = sideband > 0 ? f_base + chan_bw * k : f_base - chan_bw * (k + 1.0);
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
    const double sc = wt * (scale > 0 ? scale : 1.0 / N);
    // exp(-i Phi) w / N (FP32 kernels); its conjugate for a lower-sideband channel
    chirp[e] = make_float2((float)(cs * sc), (float)((sideband > 0 ? -sn : sn) * sc));
  }
}

// Twiddle table in the per-pass thread-major layout of PassPlan::TwOff, then,
// for a CL-CTA cluster, the cross-CTA pass: w_N^{t*k} at TW_LEN + (k-1)*NS + t.
template <int LOGS, int CL>
__global__ void twiddle_kernel(float2* tw) {
  using PL = PassPlan<LOGS>;
  constexpr int NS = PL::N;
  constexpr int TOTAL = PL::TW_LEN + (CL - 1) * NS;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < TOTAL; e += gridDim.x * blockDim.x) {
    int m, modulus;
    if (e >= PL::TW_LEN) {
      const int local = e - PL::TW_LEN;
      const int k = 1 + local / NS, t = local % NS;
      modulus = NS * CL;
      m = (int)(((long long)t * k) % modulus);
    } else {
      int p = 0;
      while (p + 1 < PL::P - 1 && e >= PL::TwOff(p + 1)) ++p;
      const int local = e - PL::TwOff(p);
      const int stride = p == 0 ? PL::T : PL::S(p);            // thread index range
      modulus = p == 0 ? PL::N : PL::M(p);
      const int t = local % stride, k = local / stride;
      m = (t * k) % modulus;
    }
    double sn, cs;
    sincospi(2.0 * m / modulus, &sn, &cs);
    tw[e] = make_float2((float)cs, (float)(-sn));           // exp(-2 pi i m / modulus)
  }
}

// Alignment shifts r_k (Sec. 1.2) computed on the device, for callers that
// keep no host-side copy of them.
__global__ void shift_kernel(int* shift, int n_chan, double f_base, double f_ref, double chan_bw,
                             double dm, int n_avg, int sideband) {
  const double ref = pow(f_ref, -2.0);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_chan; k += gridDim.x * blockDim.x) {
    const double f_k = sideband > 0 ? f_base + chan_bw * k : f_base - chan_bw * (k + 1.0);
    const double delay = kDispD * dm * (pow(f_k, -2.0) - ref);
    shift[k] = (int)rint(-delay * chan_bw * 1e6 / n_avg);
  }
}

// Corner turn of int8 pairs: out[k][row] = in[row][k] for row < rows, k < n_chan.
// 64 x 64 tiles.  A whole tile moves as 16-byte loads of 8 channels and 16-byte
// stores of 8 rows; eight lanes cover one channel's 128-byte line, and the tile
// is held as 32-bit channel pairs with an XOR swizzle so both sides are free of
// bank conflicts.
constexpr int kTT = 64;
__global__ void __launch_bounds__(256) corner_turn_kernel(const char2* __restrict__ in,
                                                          char2* __restrict__ out,
                                                          long long r_begin, long long rows,
                                                          long long stride, int n_chan) {
  __shared__ __align__(16) uint32_t tile[kTT][kTT / 2];    // [row][channel pair ^ swizzle]
  const long long r0 = r_begin + (long long)blockIdx.x * kTT;
  const int c0 = blockIdx.y * kTT;
  const unsigned short* src = reinterpret_cast<const unsigned short*>(in);
  unsigned short* dst = reinterpret_cast<unsigned short*>(out);
  const bool whole = r0 + kTT <= rows && c0 + kTT <= n_chan && (n_chan % 8) == 0 &&
                     (stride % 8) == 0 && (r_begin % 8) == 0 &&
                     ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
  auto sw = [](int r) { return ((r >> 3) & 15) << 1; };
  if (whole) {
    uint4 x[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {              // 64 rows x 8 chunks of 8 channels
      const int v = threadIdx.x + 256 * i;
      const int r = v >> 3, cq = v & 7;
      x[i] = __ldg(reinterpret_cast<const uint4*>(src + (r0 + r) * n_chan + c0 + cq * 8));
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int v = threadIdx.x + 256 * i;
      const int r = v >> 3, cq = v & 7;
      tile[r][(cq * 4 + 0) ^ sw(r)] = x[i].x;
      tile[r][(cq * 4 + 1) ^ sw(r)] = x[i].y;
      tile[r][(cq * 4 + 2) ^ sw(r)] = x[i].z;
      tile[r][(cq * 4 + 3) ^ sw(r)] = x[i].w;
    }
  } else {
    for (int v = threadIdx.x; v < kTT * kTT; v += 256) {
      const int r = v / kTT, ch = v % kTT;
      if (r0 + r < rows && c0 + ch < n_chan) {
        unsigned short* t = reinterpret_cast<unsigned short*>(&tile[r][(ch >> 1) ^ sw(r)]);
        t[ch & 1] = src[(r0 + r) * n_chan + c0 + ch];
      }
    }
  }
  __syncthreads();
  if (whole) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {              // 64 channels x 8 chunks of 8 rows
      const int v = threadIdx.x + 256 * i;
      const int ch = v >> 3, rb = (v & 7) * 8;
      uint4 y;
      unsigned short* e = reinterpret_cast<unsigned short*>(&y);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int r = rb + t;
        e[t] = reinterpret_cast<const unsigned short*>(&tile[r][(ch >> 1) ^ sw(r)])[ch & 1];
      }
      *reinterpret_cast<uint4*>(dst + (long long)(c0 + ch) * stride + r0 + rb) = y;
    }
  } else {
    for (int v = threadIdx.x; v < kTT * kTT; v += 256) {
      const int ch = v / kTT, r = v % kTT;
      if (r0 + r < rows && c0 + ch < n_chan)
        dst[(long long)(c0 + ch) * stride + r0 + r] =
            reinterpret_cast<const unsigned short*>(&tile[r][(ch >> 1) ^ sw(r)])[ch & 1];
    }
  }
}

template <int LOGN>
cudaError_t launch_ols_t(const OlsArgs& a, cudaStream_t s) {
  using CF = Cfg<LOGN>;
  static bool attr_set[128][2] = {};         // per device and input layout
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  const bool cm = a.in_cm != nullptr;
  if (!attr_set[dev][cm]) {
    e = cm ? cudaFuncSetAttribute(ols_kernel<LOGN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CF::SMEM)
           : cudaFuncSetAttribute(ols_kernel<LOGN, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CF::SMEM);
    if (e != cudaSuccess) return e;
    attr_set[dev][cm] = true;
  }
  // N = 8192 only: N = 4096 (radix 16 per thread) runs faster as three
  // 256-thread CTAs per SM (1.58 against 1.68 ms per 512-channel block)
  if constexpr (LOGN == 13) {
    if (cm && kUsePersistent) {
      static bool pset[128] = {};
      if (!pset[dev]) {
        e = cudaFuncSetAttribute(ols_persistent_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Persist<LOGN>::SMEM);
        if (e != cudaSuccess) return e;
        pset[dev] = true;
      }
      int sms = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      const long long work = (long long)a.n_chan * a.s_count;
      const long long need = (work + Persist<LOGN>::GROUPS - 1) / Persist<LOGN>::GROUPS;
      const unsigned grid = (unsigned)(need < sms ? need : sms);
      ols_persistent_kernel<LOGN><<<grid, Persist<LOGN>::THREADS, Persist<LOGN>::SMEM, s>>>(a);
      return cudaGetLastError();
    }
  }
  const long long work = (long long)a.n_chan * a.s_count;
  const unsigned grid = (unsigned)((work + CF::G - 1) / CF::G);
  if (cm) ols_kernel<LOGN, true><<<grid, CF::THREADS, CF::SMEM, s>>>(a);
  else ols_kernel<LOGN, false><<<grid, CF::THREADS, CF::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int LOGS, int CL>
cudaError_t launch_cluster_t(const OlsArgs& a, cudaStream_t s) {
  constexpr size_t SMEM = size_t(padded_len<LOGS>()) * sizeof(float2);
  static bool attr_set[128] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  if (a.in_cm == nullptr) return cudaErrorInvalidValue;     // needs the channel-major copy
  if (!attr_set[dev]) {
    e = cudaFuncSetAttribute(ols_cluster_kernel<LOGS, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const long long clusters = (long long)a.n_chan * a.s_count;
  if (clusters <= 0) return cudaSuccess;
  ols_cluster_kernel<LOGS, CL><<<(unsigned)(clusters * CL), PassPlan<LOGS>::T, SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int LOGS, int CL>
cudaError_t launch_chirp_t(float2* chirp, int n_chan, double f_base, double chan_bw, double dm,
                           int taper, int sideband, cudaStream_t s, double scale) {
  const long long total = (long long)n_chan * (CL << LOGS);
  const unsigned grid = (unsigned)((total + 255) / 256 < 65535 ? (total + 255) / 256 : 65535);
  chirp_table_kernel<LOGS, CL><<<grid, 256, 0, s>>>(chirp, n_chan, f_base, chan_bw, dm, taper,
                                                     sideband, scale);
  return cudaGetLastError();
}

}  // namespace

#define CDD_LOGN_CASES(X) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14)

cudaError_t launch_ols(int logn, const OlsArgs& a, cudaStream_t s) {
  switch (logn) {
#define X(L) case L: return launch_ols_t<L>(a, s);
    CDD_LOGN_CASES(X)
#undef X
    case 15: return launch_cluster_t<kClusterLogS, 4>(a, s);
    case 16: return launch_cluster_t<kClusterLogS, 8>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_chirp_table(int logn, float2* chirp, int n_chan, double f_base_mhz,
                               double chan_bw_mhz, double dm, int taper, int sideband,
                               cudaStream_t s, double scale) {
  switch (logn) {
#define X(L) case L: return launch_chirp_t<L, 1>(chirp, n_chan, f_base_mhz, chan_bw_mhz, dm, taper, sideband, s, scale);
    CDD_LOGN_CASES(X)
#undef X
    case 15: return launch_chirp_t<kClusterLogS, 4>(chirp, n_chan, f_base_mhz, chan_bw_mhz, dm, taper, sideband, s, scale);
    case 16: return launch_chirp_t<kClusterLogS, 8>(chirp, n_chan, f_base_mhz, chan_bw_mhz, dm, taper, sideband, s, scale);
    default: return cudaErrorInvalidValue;
  }
}

template <int LOGS, int CL>
constexpr int twiddle_len_t() { return PassPlan<LOGS>::TW_LEN + (CL - 1) * PassPlan<LOGS>::N; }

template <int LOGS, int CL>
cudaError_t launch_twiddle_t(float2* tw, cudaStream_t s) {
  twiddle_kernel<LOGS, CL><<<(twiddle_len_t<LOGS, CL>() + 255) / 256, 256, 0, s>>>(tw);
  return cudaGetLastError();
}

cudaError_t launch_twiddle_table(int logn, float2* tw, cudaStream_t s) {
  switch (logn) {
#define X(L) case L: return launch_twiddle_t<L, 1>(tw, s);
    CDD_LOGN_CASES(X)
#undef X
    case 15: return launch_twiddle_t<kClusterLogS, 4>(tw, s);
    case 16: return launch_twiddle_t<kClusterLogS, 8>(tw, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_shift_table(int* shift, int n_chan, double f_base_mhz, double f_ref_mhz,
                               double chan_bw_mhz, double dm, int n_avg, int sideband,
                               cudaStream_t s) {
  const int grid = (n_chan + 255) / 256 < 1024 ? (n_chan + 255) / 256 : 1024;
  shift_kernel<<<grid, 256, 0, s>>>(shift, n_chan, f_base_mhz, f_ref_mhz, chan_bw_mhz, dm, n_avg,
                                    sideband);
  return cudaGetLastError();
}

#ifndef CDD_TMA_TURN
#define CDD_TMA_TURN 1
#endif
cudaError_t launch_corner_turn(const char2* in, char2* out, long long r_begin, long long r_end,
                               long long stride, int n_chan, cudaStream_t s, int* err) {
  if (r_end <= r_begin) return cudaSuccess;
  if (CDD_TMA_TURN && err) {
    const cudaError_t e = launch_corner_turn_tma(in, out, r_begin, r_end, stride, n_chan, err, s);
    if (e != cudaErrorNotSupported) return e;
  }
  const dim3 grid((unsigned)((r_end - r_begin + kTT - 1) / kTT), (unsigned)((n_chan + kTT - 1) / kTT));
  corner_turn_kernel<<<grid, 256, 0, s>>>(in, out, r_begin, r_end, stride, n_chan);
  return cudaGetLastError();
}

// Band sum over channels: sum[p][m] = sum_k out[p][k][m].  A CTA owns a tile
// of 32*V neighbouring outputs of one plane (V = 4: float4 per lane); its 8
// warps take every 8th channel, so each warp keeps 8 row loads in flight, and
// the 8 partial sums meet in shared memory.
template <int V>
__global__ void __launch_bounds__(256)
band_sum_kernel(const float* __restrict__ out, long long n_planes, int n_chan, long long n_out,
                float* __restrict__ sum) {
  constexpr int TILE = 32 * V;
  __shared__ float part[8][TILE];
  const long long tiles = (n_out + TILE - 1) / TILE;
  const long long p = blockIdx.x / tiles;
  const long long c0 = (blockIdx.x % tiles) * TILE;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const long long m = c0 + (long long)lane * V;
  float acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = 0.f;
  if (m < n_out) {                                   // V = 4: n_out % 4 == 0, so m + 3 < n_out
    const float* col = out + p * n_chan * n_out + m;
#pragma unroll 8
    for (int k = wp; k < n_chan; k += 8) {
      if constexpr (V == 4) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(col + (long long)k * n_out));
        acc[0] += x.x;
        acc[1] += x.y;
        acc[2] += x.z;
        acc[3] += x.w;
      } else {
        acc[0] += __ldg(col + (long long)k * n_out);
      }
    }
  }
#pragma unroll
  for (int v = 0; v < V; ++v) part[wp][lane * V + v] = acc[v];
  __syncthreads();
  for (int t = threadIdx.x; t < TILE; t += blockDim.x) {
    float tot = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) tot += part[w][t];
    if (c0 + t < n_out) sum[p * n_out + c0 + t] = tot;
  }
}

// acc[i] += add[i]; float4 when both are 16-byte aligned and n % 4 == 0.
template <int V>
__global__ void accumulate_kernel(float* __restrict__ acc, const float* __restrict__ add, long long n) {
  const long long nv = n / V;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nv;
       i += (long long)gridDim.x * blockDim.x) {
    if constexpr (V == 4) {
      float4 a = reinterpret_cast<float4*>(acc)[i];
      const float4 b = __ldg(reinterpret_cast<const float4*>(add) + i);
      a.x += b.x;
      a.y += b.y;
      a.z += b.z;
      a.w += b.w;
      reinterpret_cast<float4*>(acc)[i] = a;
    } else {
      acc[i] += add[i];
    }
  }
}

cudaError_t launch_band_sum(const float* out, long long n_planes, int n_chan, long long n_out,
                            float* sum, cudaStream_t s) {
  const bool vec = n_out % 4 == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
  const int tile = vec ? 128 : 32;
  const long long blocks = n_planes * ((n_out + tile - 1) / tile);
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (vec) band_sum_kernel<4><<<(unsigned)blocks, 256, 0, s>>>(out, n_planes, n_chan, n_out, sum);
  else band_sum_kernel<1><<<(unsigned)blocks, 256, 0, s>>>(out, n_planes, n_chan, n_out, sum);
  return cudaGetLastError();
}

cudaError_t launch_accumulate(float* acc, const float* add, long long n, cudaStream_t s) {
  const bool vec = n % 4 == 0 && ((reinterpret_cast<uintptr_t>(acc) | reinterpret_cast<uintptr_t>(add)) & 15) == 0;
  const long long nv = vec ? n / 4 : n;
  const unsigned grid = (unsigned)((nv + 255) / 256 < 148 * 32 ? (nv + 255) / 256 : 148 * 32);
  if (vec) accumulate_kernel<4><<<grid > 0 ? grid : 1, 256, 0, s>>>(acc, add, n);
  else accumulate_kernel<1><<<grid > 0 ? grid : 1, 256, 0, s>>>(acc, add, n);
  return cudaGetLastError();
}

int twiddle_table_len(int logn) {
  switch (logn) {
#define X(L) case L: return twiddle_len_t<L, 1>();
    CDD_LOGN_CASES(X)
#undef X
    case 15: return twiddle_len_t<kClusterLogS, 4>();
    case 16: return twiddle_len_t<kClusterLogS, 8>();
    default: return 0;
  }
}

bool needs_channel_major(int logn) { return logn > 14; }

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
