// Corner turn of the time-major input block through the tensor memory
// accelerator: out[k][row] = in[row][k], int8 (re, im) pairs as 16-bit
// elements.  The voltage beam arrives as the FFT outputs of each time step in
// series (Sec. 2.3), one row of all channels per sample; the fused kernel
// reads each channel's segment contiguously, so the block is turned first.
//
// A persistent CTA moves 64 x 64 tiles: a 2-D tensor copy brings rows
// [r, r + 64) x channels [c, c + 64) into shared memory (128-byte rows, the
// 128-byte swizzle), the CTA transposes it into a second tile, and a 2-D
// tensor store writes channels [c, c + 64) x rows [r, r + 64) of the output.
// Three input tiles are in flight per CTA, each signalled on its own mbarrier
// by transaction count; two output tiles alternate, the store of one being
// read out while the other is filled.  Copies that fall outside the tensors
// read zeros and are clipped on the store, so ragged row and channel counts
// need no special case.  Every wait is bounded: a CTA that gives up sets the
// plan's error flag, waits (bounded) for the copies it issued, and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/cdd.h"
#include "cdd_internal.h"

namespace cdd {

namespace {

constexpr int kTT = 64;                         // tile edge (rows and channels)
#ifndef CDD_TMA_CTAS_PER_SM
#define CDD_TMA_CTAS_PER_SM 4
#endif
constexpr int kStages = 3;                      // input tiles in flight per CTA
constexpr int kThreads = 256;                   // 8 warps: a warp per 8-row chunk of the tile
constexpr uint32_t kTileBytes = kTT * kTT * 2;  // 8 KB
constexpr uint64_t kWaitLimitNs = 1000000000ull;

struct __align__(1024) TurnSmem {
  uint16_t in[kStages][kTT * kTT];              // [row][channel], rows swizzled
  uint16_t out[2][kTT * kTT];                   // [channel][row], rows swizzled
  unsigned long long bar[kStages];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
               "r"(bytes)
               : "memory");
}

// Wait for phase `parity` of an mbarrier for at most limit_ns.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = global_ns();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 20000;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// Tile (x, y) of `map` into shared memory at dst, completing on bar.
__device__ __forceinline__ void tma_load(const CUtensorMap* map, uint32_t dst, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_store(const CUtensorMap* map, uint32_t src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
               ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(src)
               : "memory");
}

// Byte offset of element e (0..63) of row r in a 64-element (128-byte) row
// tile under the 128-byte swizzle: the 16-byte chunk index is XORed with r mod 8.
__device__ __forceinline__ uint32_t swz(int r, int e) {
  return (uint32_t)(r * 128 + ((((e >> 3) ^ (r & 7)) << 4) | ((e & 7) << 1)));
}

__global__ void __launch_bounds__(kThreads)
corner_turn_tma_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
                       int r_begin, int tiles_r, int tiles_c, int* err, uint32_t expect_extra,
                       uint64_t limit_ns) {
  __shared__ TurnSmem sm;
  const int tid = threadIdx.x;
  const long long n_tiles = (long long)tiles_r * tiles_c;
  const long long step = gridDim.x;
  // tile i: channels [64 (i mod tiles_c), +64), rows r_begin + [64 (i div tiles_c), +64)
  auto tile_x = [&](long long i) { return (int)(i % tiles_c) * kTT; };
  auto tile_y = [&](long long i) { return r_begin + (int)(i / tiles_c) * kTT; };
  int issued[kStages] = {0, 0, 0};              // loads issued per slot (thread 0)
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(&sm.bar[s]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      const long long i = blockIdx.x + s * step;
      if (i < n_tiles) {
        mbar_expect(smem_u32(&sm.bar[s]), kTileBytes + expect_extra);
        tma_load(&tin, smem_u32(sm.in[s]), smem_u32(&sm.bar[s]), tile_x(i), tile_y(i));
        issued[s] += 1;
      }
    }
  }
  const int w = tid >> 5, lane = tid & 31;      // output row chunk w, channel pair lane
  bool failed = false;
  long long j = 0;
  for (; blockIdx.x + j * step < n_tiles; ++j) {
    const long long i = blockIdx.x + j * step;
    const int s = (int)(j % kStages);
    const bool ok = mbar_wait(smem_u32(&sm.bar[s]), (uint32_t)((j / kStages) & 1), limit_ns);
    // every thread knows the load landed, and thread 0's wait on the store
    // that last read out[j & 1] is done
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    // channels (2 lane, 2 lane + 1) of rows 8 w .. 8 w + 7: eight 32-bit
    // reads, then one 16-byte row piece for each of the two channels
    const unsigned char* tin_s = reinterpret_cast<const unsigned char*>(sm.in[s]);
    unsigned char* tout_s = reinterpret_cast<unsigned char*>(sm.out[j & 1]);
    uint32_t v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = *reinterpret_cast<const uint32_t*>(tin_s + swz(8 * w + t, 2 * lane));
    uint4 lo, hi;                               // channel 2 lane, channel 2 lane + 1
    lo.x = __byte_perm(v[0], v[1], 0x5410);
    lo.y = __byte_perm(v[2], v[3], 0x5410);
    lo.z = __byte_perm(v[4], v[5], 0x5410);
    lo.w = __byte_perm(v[6], v[7], 0x5410);
    hi.x = __byte_perm(v[0], v[1], 0x7632);
    hi.y = __byte_perm(v[2], v[3], 0x7632);
    hi.z = __byte_perm(v[4], v[5], 0x7632);
    hi.w = __byte_perm(v[6], v[7], 0x7632);
    *reinterpret_cast<uint4*>(tout_s + swz(2 * lane, 8 * w)) = lo;
    *reinterpret_cast<uint4*>(tout_s + swz(2 * lane + 1, 8 * w)) = hi;
    // the tile's shared-memory writes (and reads of in[s]) before the tensor
    // copies that read out[j & 1] and refill in[s]
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tma_store(&tout, smem_u32(sm.out[j & 1]), tile_y(i), tile_x(i));
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      // the store before this one has finished reading out[(j + 1) & 1]
      asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
      const long long i2 = i + kStages * step;
      if (i2 < n_tiles) {
        mbar_expect(smem_u32(&sm.bar[s]), kTileBytes + expect_extra);
        tma_load(&tin, smem_u32(sm.in[s]), smem_u32(&sm.bar[s]), tile_x(i2), tile_y(i2));
        issued[s] += 1;
      }
    }
  }
  if (tid == 0) {
    if (failed) {
      atomicOr(err, 2);
      // loads issued but not yet waited for: slot s has had j_s = (loads of
      // slot s among tiles < j) completions waited; wait (bounded) for the rest
      for (int s = 0; s < kStages; ++s) {
        const int done = (int)((j + kStages - 1 - s) / kStages);   // tiles j' < j with j' mod kStages == s
        for (int p = done; p < issued[s]; ++p) mbar_wait(smem_u32(&sm.bar[s]), (uint32_t)(p & 1), limit_ns);
      }
    }
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// 2-D map over a [dim1][dim0] array of 16-bit elements, rows pitch_elems apart,
// 64 x 64 boxes with the 128-byte swizzle.
bool encode_2d(CUtensorMap* map, const void* base, long long dim0, long long dim1, long long pitch_elems) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)dim0, (cuuint64_t)dim1};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch_elems * 2};
  const cuuint32_t box[2] = {kTT, kTT};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool corner_turn_tma_ok(const char2* in, const char2* out, long long r_begin, long long r_end, long long stride,
                        int n_chan) {
  // 16-byte aligned bases and row pitches, an 8-element (16-byte) aligned
  // first output column for every store, and 32-bit tile coordinates
  return in && out && n_chan > 0 && r_end > r_begin && r_begin >= 0 && n_chan % 8 == 0 && stride % 8 == 0 &&
         r_begin % 8 == 0 && r_end <= stride && r_end < (1LL << 31) - kTT &&
         ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0 && encode_fn() != nullptr;
}

cudaError_t launch_corner_turn_tma(const char2* in, char2* out, long long r_begin, long long r_end, long long stride,
                                   int n_chan, int* err, cudaStream_t s) {
  if (!err || !corner_turn_tma_ok(in, out, r_begin, r_end, stride, n_chan)) return cudaErrorNotSupported;
  CUtensorMap tin, tout;
  // input: [r_end][n_chan] (channels innermost); output: [n_chan][stride], rows < r_end
  if (!encode_2d(&tin, in, n_chan, r_end, n_chan) || !encode_2d(&tout, out, r_end, n_chan, stride))
    return cudaErrorNotSupported;
  const long long tiles_r = (r_end - r_begin + kTT - 1) / kTT;
  const long long tiles_c = (n_chan + kTT - 1) / kTT;
  const long long n_tiles = tiles_r * tiles_c;
  if (tiles_r > 0x7fffffffLL || tiles_c > 0x7fffffffLL) return cudaErrorNotSupported;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long cap = (long long)CDD_TMA_CTAS_PER_SM * sms;
  const unsigned grid = (unsigned)(n_tiles < cap ? n_tiles : cap);
  corner_turn_tma_kernel<<<grid, kThreads, 0, s>>>(tin, tout, (int)r_begin, (int)tiles_r, (int)tiles_c, err, 0u,
                                                    kWaitLimitNs);
  return cudaGetLastError();
}

}  // namespace cdd

// Self-test of the bounded waits: one tile whose mbarrier expects 16 bytes
// more than the copy delivers, so its phase never completes and the wait
// runs out after 20 ms.  The kernel must set bit 2 of its flag, give up its
// bounded cleanup wait, and return with the device still usable.
extern "C" int cdd_selftest_wait_limit(int* status) {
  if (!status) return CDD_EINVAL;
  *status = 0;
  using namespace cdd;
  char2* d_in = nullptr;
  char2* d_out = nullptr;
  int* d_err = nullptr;
  int rc = CDD_OK;
  cudaError_t e = cudaMalloc((void**)&d_in, kTileBytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&d_out, kTileBytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d_in, 0, kTileBytes);
  if (e == cudaSuccess) e = cudaMemset(d_err, 0, sizeof(int));
  CUtensorMap tin, tout;
  if (e == cudaSuccess && (!encode_2d(&tin, d_in, kTT, kTT, kTT) || !encode_2d(&tout, d_out, kTT, kTT, kTT)))
    rc = CDD_EUNSUPPORTED;
  if (e == cudaSuccess && rc == CDD_OK) {
    corner_turn_tma_kernel<<<1, kThreads>>>(tin, tout, 0, 1, 1, d_err, 16u, 20000000ull);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(status, d_err, sizeof(int), cudaMemcpyDeviceToHost);
    // the context still answers
    if (e == cudaSuccess) e = cudaMemset(d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  if (e == cudaErrorMemoryAllocation) rc = CDD_ENOMEM;
  else if (e != cudaSuccess) rc = CDD_ECUDA;
  cudaFree(d_in);
  cudaFree(d_out);
  cudaFree(d_err);
  return rc;
}
