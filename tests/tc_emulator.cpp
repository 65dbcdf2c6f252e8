// tc_emulator.cpp -- host check of the tensor-core (tcgen05) form of the
// N = 8192 overlap-save transform, before any of it runs on a GPU.
//
// It replays, on the CPU, the data flow of ols_tc_kernel for one segment:
// operands written with the layouts of cdd_tc_layout.h into a byte image of
// shared memory, every matrix product decoded from the 64-bit shared-memory
// descriptors and the 32-bit instruction descriptor exactly as the kernel
// encodes them (the canonical K-major no-swizzle layout: element (m, k) of an
// operand at start + (m mod 8)*16 + (m / 8)*SBO + (k / 8)*LBO + (k mod 8)*2),
// accumulation into an FP32 image of tensor memory, and the index maps that
// move each pass's outputs to the next pass's operand rows.  The result is
// compared with the direct definition: y = IDFT_N(DFT_N(x) * c[bin]) / N,
// evaluated as O(N^2) sums in double precision.
//
// Usage: tc_emulator <precision>   (fp16, fp16x2, bf16, bf16x2)
// Prints "relrms <value>" for the voltages and exits 0, or a message and 1.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "../paper_1509_00186_b300/csrc/cdd_tc_layout.h"

using namespace cdd::tc;

namespace {

bool g_bf16 = false, g_split = false;

// half / bfloat16 bits <-> float, round to nearest even (the kernel's cvt.rn)
uint16_t to_bits(float x) {
  if (g_bf16) {
    __bf16 h = (__bf16)x;
    uint16_t b;
    memcpy(&b, &h, 2);
    return b;
  }
  _Float16 h = (_Float16)x;
  uint16_t b;
  memcpy(&b, &h, 2);
  return b;
}
float from_bits(uint16_t b) {
  if (g_bf16) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
  }
  _Float16 h;
  memcpy(&h, &b, 2);
  return (float)h;
}

struct Cf {
  float x, y;
};
Cf cmul(Cf a, Cf w) { return {fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x)}; }

// shared-memory image, laid out as the kernel lays out its dynamic shared memory
constexpr int kAHi = 0, kALo = kRegion, kB32 = 2 * kRegion, kB16 = kB32 + b_bytes(32);
constexpr int kSmem = kB16 + b_bytes(16);
std::vector<uint8_t> smem(kSmem);
std::vector<float> tmem(128 * 512);   // [lane][column]

void st16(int off, uint16_t v) {
  if (off < 0 || off + 2 > kSmem) {
    fprintf(stderr, "store outside shared memory: %d\n", off);
    exit(1);
  }
  memcpy(&smem[off], &v, 2);
}
uint16_t ld16(int off) {
  if (off < 0 || off + 2 > kSmem) {
    fprintf(stderr, "operand read outside shared memory: %d\n", off);
    exit(1);
  }
  uint16_t v;
  memcpy(&v, &smem[off], 2);
  return v;
}

// One tcgen05.mma kind::f16 (cta_group::1), decoded from its descriptors.
void mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, bool acc) {
  auto check_desc = [](uint64_t d) {
    if (((d >> 46) & 3) != 1 || ((d >> 61) & 7) != 0 || ((d >> 49) & 7) != 0 || ((d >> 52) & 1) != 0 ||
        ((d >> 14) & 3) != 0 || ((d >> 30) & 3) != 0 || ((d >> 48) & 1) != 0 || ((d >> 53) & 0xFF) != 0) {
      fprintf(stderr, "bad descriptor fields %016llx\n", (unsigned long long)d);
      exit(1);
    }
  };
  check_desc(adesc);
  check_desc(bdesc);
  const int a0 = (int)((adesc & 0x3FFF) << 4), alb = (int)(((adesc >> 16) & 0x3FFF) << 4),
            asb = (int)(((adesc >> 32) & 0x3FFF) << 4);
  const int b0 = (int)((bdesc & 0x3FFF) << 4), blb = (int)(((bdesc >> 16) & 0x3FFF) << 4),
            bsb = (int)(((bdesc >> 32) & 0x3FFF) << 4);
  const int cfmt = (idesc >> 4) & 3, afmt = (idesc >> 7) & 7, bfmt = (idesc >> 10) & 7;
  const int n = (int)((idesc >> 17) & 63) << 3, m = (int)((idesc >> 24) & 31) << 4;
  if (cfmt != 1 || afmt != (g_bf16 ? 1 : 0) || bfmt != afmt || (idesc & 0xF) != 0 || ((idesc >> 13) & 15) != 0 ||
      m != 128 || n < 16 || n > 256 || n % 16 || (idesc >> 29) != 0 || ((idesc >> 23) & 1) != 0) {
    fprintf(stderr, "bad instruction descriptor %08x\n", idesc);
    exit(1);
  }
  const int lane0 = d_tmem >> 16, col0 = d_tmem & 0xFFFF;
  if (lane0 != 0 || col0 + n > 512) {
    fprintf(stderr, "accumulator outside tensor memory\n");
    exit(1);
  }
  for (int r = 0; r < m; ++r) {
    for (int c = 0; c < n; ++c) {
      float s = acc ? tmem[r * 512 + col0 + c] : 0.f;
      for (int kk = 0; kk < 16; ++kk) {
        const float av = from_bits(ld16(a0 + (r & 7) * 16 + (r >> 3) * asb + (kk >> 3) * alb + (kk & 7) * 2));
        const float bv = from_bits(ld16(b0 + (c & 7) * 16 + (c >> 3) * bsb + (kk >> 3) * blb + (kk & 7) * 2));
        s = fmaf(av, bv, s);     // products of 11-bit significands are exact in FP32
      }
      tmem[r * 512 + col0 + c] = s;
    }
  }
}

// B: forward DFT matrix / R, rows [hi; lo]
void build_b(int R, int base) {
  for (int n = 0; n < 4 * R; ++n)
    for (int kk = 0; kk < 2 * R; ++kk) {
      const int n0 = n % (2 * R);
      const int mm = dft_m(R, n0, kk);
      const double ang = 2.0 * M_PI * mm / R;
      double v = dft_is_sin(n0, kk) ? sin(ang) : cos(ang);
      if (dft_negative(n0, kk)) v = -v;
      v /= R;
      const uint16_t hi = to_bits((float)v);
      const uint16_t lo = to_bits((float)(v - (double)from_bits(hi)));
      st16(base + b_off(R, n, kk), n < 2 * R ? hi : lo);
    }
}

// value -> hi (and lo) at element e of row m of the pass operand
void put(Lay L, int m, int e, Cf v) {
  const uint16_t hr = to_bits(v.x), hi_ = to_bits(v.y);
  st16(kAHi + lay_off(L, m, 2 * e), hr);
  st16(kAHi + lay_off(L, m, 2 * e + 1), hi_);
  if (g_split) {
    st16(kALo + lay_off(L, m, 2 * e), to_bits(v.x - from_bits(hr)));
    st16(kALo + lay_off(L, m, 2 * e + 1), to_bits(v.y - from_bits(hi_)));
  }
}

// issue the products of one pass (the kernel's issue_pass)
void issue(int R, Lay L, int tiles, bool lo) {
  const int cw = tile_cols(R, g_split);
  const int bbase = R == 32 ? kB32 : kB16;
  for (int tt = 0; tt < tiles; ++tt)
    for (int s = 0; s < 2 * R / 16; ++s) {
      const uint64_t bd = smem_desc((uint32_t)(bbase + s * b_ks(R)), kLboB, kSboB);
      mma(tmem_addr(0, 0, tt * cw), smem_desc((uint32_t)(kAHi + tt * L.ts + s * L.ks), L.lbo, L.sbo), bd,
          idesc_f16(128, cw, g_bf16), s > 0);
      if (lo)
        mma(tmem_addr(0, 0, tt * cw), smem_desc((uint32_t)(kALo + tt * L.ts + s * L.ks), L.lbo, L.sbo), bd,
            idesc_f16(128, 2 * R, g_bf16), true);
    }
}

// the R outputs of row g of a pass (sum of the [hi | lo] halves)
void row_out(int R, int g, Cf* v) {
  const int cw = tile_cols(R, g_split);
  const int lane = g & 127, col = (g >> 7) * cw;
  for (int k = 0; k < R; ++k) {
    float re = tmem[lane * 512 + col + 2 * k], im = tmem[lane * 512 + col + 2 * k + 1];
    if (g_split) {
      re += tmem[lane * 512 + col + 2 * R + 2 * k];
      im += tmem[lane * 512 + col + 2 * R + 2 * k + 1];
    }
    v[k] = {re, im};
  }
}

}  // namespace

int main(int argc, char** argv) {
  const char* prec = argc > 1 ? argv[1] : "fp16x2";
  g_bf16 = strncmp(prec, "bf16", 4) == 0;
  g_split = strstr(prec, "x2") != nullptr;
  // descriptor field checks against the encoders
  {
    const uint64_t d = smem_desc(0x12340, 144, 272);
    if ((d & 0x3FFF) != (0x12340 >> 4) || ((d >> 16) & 0x3FFF) != 9 || ((d >> 32) & 0x3FFF) != 17 ||
        ((d >> 46) & 3) != 1) {
      fprintf(stderr, "smem_desc fields wrong\n");
      return 1;
    }
    const uint32_t id = idesc_f16(128, 64, false);
    if (id != ((1u << 4) | (8u << 17) | (8u << 24))) {
      fprintf(stderr, "idesc fields wrong %08x\n", id);
      return 1;
    }
  }
  // every operand slot of each layout is distinct and inside its region
  {
    std::vector<char> used(kRegion, 0);
    for (int m = 0; m < 512; ++m)
      for (int kk = 0; kk < 32; ++kk) {
        const int o = lay_off(lay12(), m, kk);
        if (o < 0 || o + 2 > kRegion || used[o]) {
          fprintf(stderr, "layout 12 overlaps at %d\n", o);
          return 1;
        }
        used[o] = 1;
      }
    std::fill(used.begin(), used.end(), 0);
    for (int m = 0; m < 256; ++m)
      for (int kk = 0; kk < 64; ++kk) {
        const int o = lay_off(lay0(), m, kk);
        if (o < 0 || o + 2 > kRegion || used[o]) {
          fprintf(stderr, "layout 0 overlaps at %d\n", o);
          return 1;
        }
        used[o] = 1;
      }
  }

  // twiddle table (the FP32 kernel's: pass 0 w_N^{tk} at 256k + t, pass 1
  // w_256^{tk} at N + 16k + t), FP64 then rounded
  std::vector<Cf> tw(kN + 256);
  for (int k = 0; k < 32; ++k)
    for (int t = 0; t < 256; ++t) {
      const double a = -2.0 * M_PI * ((t * k) % kN) / kN;
      tw[256 * k + t] = {(float)cos(a), (float)sin(a)};
    }
  for (int k = 0; k < 16; ++k)
    for (int t = 0; t < 16; ++t) {
      const double a = -2.0 * M_PI * ((t * k) % 256) / 256;
      tw[kN + 16 * k + t] = {(float)cos(a), (float)sin(a)};
    }
  // a chirp of unit magnitude per bin (random phases) and int8 input
  srand(12345);
  std::vector<double> cre(kN), cim(kN);
  for (int b = 0; b < kN; ++b) {
    const double ph = 2.0 * M_PI * (rand() / (double)RAND_MAX);
    cre[b] = cos(ph);
    cim[b] = sin(ph);
  }
  std::vector<Cf> chirp4(2 * kN);   // float4 entries as two Cf
  for (int q = 0; q < 512; ++q)
    for (int k = 0; k < 16; ++k) {
      const int b = bin_of_pos(pos_pass2(q, k));
      chirp4[2 * chirp4_index(q, k) + (k & 1)] = {(float)(cre[b] * kChirpScale), (float)(cim[b] * kChirpScale)};
    }
  std::vector<int> xr(kN), xi(kN);
  for (int n = 0; n < kN; ++n) {
    xr[n] = (rand() % 256) - 128;
    xi[n] = (rand() % 256) - 128;
  }

  build_b(32, kB32);
  build_b(16, kB16);

  // forward pass 0: exact int8 input, hi only
  for (int t = 0; t < 256; ++t)
    for (int j = 0; j < 32; ++j) {
      const int p = pos_pass0(t, j);
      st16(kAHi + lay_off(lay0(), t, 2 * j), to_bits((float)xr[p]));
      st16(kAHi + lay_off(lay0(), t, 2 * j + 1), to_bits((float)xi[p]));
    }
  issue(32, lay0(), 2, false);
  std::vector<Cf> v(32);
  std::vector<Cf> outs;
  // forward pass 0 -> pass-1 operands
  {
    std::vector<Cf> keep(256 * 32);
    for (int t = 0; t < 256; ++t) {
      row_out(32, t, v.data());
      for (int k = 0; k < 32; ++k) keep[t * 32 + k] = k ? cmul(v[k], tw[f0_tw(t, k)]) : v[k];
    }
    for (int t = 0; t < 256; ++t)
      for (int k = 0; k < 32; ++k) put(lay12(), f0_row(t, k), f0_elem(t), keep[t * 32 + k]);
  }
  issue(16, lay12(), 4, g_split);
  {
    std::vector<Cf> keep(512 * 16);
    for (int g = 0; g < 512; ++g) {
      row_out(16, g, v.data());
      for (int k = 0; k < 16; ++k) keep[g * 16 + k] = k ? cmul(v[k], tw[f1_tw(g, k)]) : v[k];
    }
    for (int g = 0; g < 512; ++g)
      for (int k = 0; k < 16; ++k) put(lay12(), f1_row(g, k), f1_elem(g), keep[g * 16 + k]);
  }
  issue(16, lay12(), 4, g_split);
  // chirp, conjugate, own row
  {
    std::vector<Cf> keep(512 * 16);
    for (int q = 0; q < 512; ++q) {
      row_out(16, q, v.data());
      for (int k = 0; k < 16; ++k) {
        const Cf y = cmul(v[k], chirp4[2 * chirp4_index(q, k) + (k & 1)]);
        keep[q * 16 + k] = {y.x, -y.y};
      }
    }
    for (int q = 0; q < 512; ++q)
      for (int k = 0; k < 16; ++k) put(lay12(), q, k, keep[q * 16 + k]);
  }
  issue(16, lay12(), 4, g_split);
  {
    std::vector<Cf> keep(512 * 16);
    for (int q = 0; q < 512; ++q) {
      row_out(16, q, v.data());
      for (int k = 0; k < 16; ++k) keep[q * 16 + k] = k ? cmul(v[k], tw[i2_tw(q, k)]) : v[k];
    }
    for (int q = 0; q < 512; ++q)
      for (int k = 0; k < 16; ++k) put(lay12(), i2_row(q, k), i2_elem(q), keep[q * 16 + k]);
  }
  issue(16, lay12(), 4, g_split);
  {
    std::vector<Cf> keep(512 * 16);
    for (int g = 0; g < 512; ++g) {
      row_out(16, g, v.data());
      for (int j = 0; j < 16; ++j) keep[g * 16 + j] = cmul(v[j], tw[i1_tw(g, j)]);
    }
    for (int g = 0; g < 512; ++g)
      for (int j = 0; j < 16; ++j) put(lay0(), i1_row(g, j), i1_elem(g), keep[g * 16 + j]);
  }
  issue(32, lay0(), 2, g_split);
  std::vector<double> yr(kN), yi(kN);
  for (int t = 0; t < 256; ++t) {
    row_out(32, t, v.data());
    for (int j = 0; j < 32; ++j) {
      const int p = pos_pass0(t, j);
      yr[p] = v[j].x * kOutScale;      // y = conj(u) * N / kChirpScale
      yi[p] = -v[j].y * kOutScale;
    }
  }

  // the definition, in double: X = DFT(x); Y[b] = X[b] c[b]; y = IDFT(Y) / N
  std::vector<double> cs(kN), sn(kN);
  for (int i = 0; i < kN; ++i) {
    cs[i] = cos(2.0 * M_PI * i / kN);
    sn[i] = sin(2.0 * M_PI * i / kN);
  }
  std::vector<double> Yr(kN), Yi(kN);
  for (int b = 0; b < kN; ++b) {
    double sr = 0, si = 0;
    for (int n = 0; n < kN; ++n) {
      const int i = (int)(((long long)b * n) % kN);
      sr += xr[n] * cs[i] + xi[n] * sn[i];
      si += xi[n] * cs[i] - xr[n] * sn[i];
    }
    Yr[b] = sr * cre[b] - si * cim[b];
    Yi[b] = sr * cim[b] + si * cre[b];
  }
  double num = 0, den = 0;
  for (int n = 0; n < kN; ++n) {
    double sr = 0, si = 0;
    for (int b = 0; b < kN; ++b) {
      const int i = (int)(((long long)b * n) % kN);
      sr += Yr[b] * cs[i] - Yi[b] * sn[i];
      si += Yi[b] * cs[i] + Yr[b] * sn[i];
    }
    sr /= kN;
    si /= kN;
    num += (yr[n] - sr) * (yr[n] - sr) + (yi[n] - si) * (yi[n] - si);
    den += sr * sr + si * si;
  }
  printf("relrms %.6e\n", sqrt(num / den));
  return 0;
}
