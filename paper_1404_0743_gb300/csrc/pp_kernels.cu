// pp_kernels.cu -- sm_103a kernels of the pentago retrograde step.
//
// A super value (paper, "Abstracting over rotations") is two 256-bit tables
// over g in L = Z4^4; here each table is eight 32-bit words, word w holding
// beta(g) = g0 + 4 g1 + 16 g2 + 64 g3 in [32w, 32w + 32): bit position
// g0 + 4 g1 + 16 (g2 & 1) of word (g2 >> 1) + 2 g3.  One thread owns one
// board; all work is 32-bit integer logic (LOP3, shifts, byte permutes,
// integer multiplies used as bit spreads).
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstring>

#include "pp_internal.h"

// Minimum resident blocks per SM requested from the register allocator
// (tuning knobs; 2 blocks of 256 threads cap a kernel at 128 registers, 4 at
// 64, 6 at 40).  The midgame kernels wait on the latency of their child
// loads, so they take as many warps as fit with few spills: 6 blocks (48
// warps) for the level kernel, 4 for the persistent one, which keeps two
// child loads in flight per thread (measured: 5.54 and 5.46 ms for the
// 1024 x 12 step against 5.91 and 5.78 at 4 and 3 blocks; 7 blocks spill
// heavily, 9.5 ms).
#ifndef PP_MID_MINB
#define PP_MID_MINB 6  // midgame level kernel
#endif
#ifndef PP_MIDP_MINB
#define PP_MIDP_MINB 4  // persistent midgame kernel
#endif
#ifndef PP_LINE_MINB
#define PP_LINE_MINB 5  // slice-35 line kernel (blocks of kLineWarps warps)
#endif
#ifndef PP_SEC_MINB
#define PP_SEC_MINB 2
#endif
#ifndef PP_SLINE_MINB
#define PP_SLINE_MINB 2  // section line kernel
#endif
#ifndef PP_SLINE_READY_MINB
#define PP_SLINE_READY_MINB 3  // section line kernel over ready children (80 registers)
#endif
#ifndef PP_SLINE_WARPS
#define PP_SLINE_WARPS 8  // warps per block of the section line kernel
#endif
namespace pp {
constexpr int kSecLineWarps = PP_SLINE_WARPS;
}


namespace pp {

__constant__ DeviceTables c_tab;
__constant__ uint32_t c_pow3[17] = {1,      3,       9,       27,       81,       243,
                                    729,    2187,    6561,    19683,    59049,    177147,
                                    531441, 1594323, 4782969, 14348907, 43046721};

static std::atomic<uint64_t> g_launches{0};
static thread_local bool g_counting = true;  // off while launches are captured into a graph
void count_launch() {
  if (g_counting) g_launches.fetch_add(1, std::memory_order_relaxed);
}
void set_launch_counting(bool on) { g_counting = on; }
void add_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
uint64_t launch_total() { return g_launches.load(); }

struct Bits {
  uint32_t w[8];
};

__device__ __forceinline__ uint32_t fold16(uint32_t x) { return (x | (x >> 16)) & 0xFFFFu; }
// all ones when bit b of x is set: bit b moved to the sign bit, then an
// arithmetic shift (the left shift can issue as a multiply)
__device__ __forceinline__ uint32_t gate(uint32_t x, int b) { return (uint32_t)((int32_t)(x << (31 - b)) >> 31); }

__device__ __forceinline__ void load_forms(int q, uint32_t pattern, uint32_t f[kFormWords]) {
  const uint4* p = reinterpret_cast<const uint4*>(c_tab.forms + (size_t)(q * 512 + pattern) * kFormWords);
  uint4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
  f[0] = a.x, f[1] = a.y, f[2] = a.z, f[3] = a.w;
  f[4] = b.x, f[5] = b.y, f[6] = b.z, f[7] = b.w;
  f[8] = c.x, f[9] = c.y, f[10] = c.z, f[11] = c.w;
}

// The same entry from a copy of the table in shared memory.
__device__ __forceinline__ void load_forms_smem(const uint4* s, int entry, uint32_t f[kFormWords]) {
  const uint4 a = s[3 * entry], b = s[3 * entry + 1], c = s[3 * entry + 2];
  f[0] = a.x, f[1] = a.y, f[2] = a.z, f[3] = a.w;
  f[4] = b.x, f[5] = b.y, f[6] = b.z, f[7] = b.w;
  f[8] = c.x, f[9] = c.y, f[10] = c.z, f[11] = c.w;
}

// Copy words [begin, begin + n) of the forms table into shared memory (all
// threads of the block take part; ends with a block barrier).
__device__ __forceinline__ void copy_forms(uint4* s, int begin_entry, int entries) {
  const uint4* g = reinterpret_cast<const uint4*>(c_tab.forms) + 3 * begin_entry;
  for (int i = threadIdx.x; i < 3 * entries; i += blockDim.x) s[i] = __ldg(g + i);
  __syncthreads();
}

// Compact pair masks -> one output word (see the form layout in pp_internal.h).
// P02 / T1: bits g0 + 4 g2 -> word with g2 >> 1 = h.
// (The two products below cover disjoint bits, so they are added: a
// multiply-add instead of a separate OR.)
__device__ __forceinline__ uint32_t exp02(uint32_t m, int h) {
  return ((m >> (8 * h)) & 0xFu) * 0x1111u + ((m >> (8 * h + 4)) & 0xFu) * 0x11110000u;
}
// P12 / T3: bits g2 + 4 g1 -> word with g2 >> 1 = h.
__device__ __forceinline__ uint32_t exp12(uint32_t m, int h) {
  return ((m >> (2 * h)) & 0x1111u) * 0xFu + ((m >> (2 * h + 1)) & 0x1111u) * 0xF0000u;
}
// P03: bits g0 + 4 g3 -> word of quadrant-3 turn g3.
__device__ __forceinline__ uint32_t exp03(uint32_t m, int g3) { return ((m >> (4 * g3)) & 0xFu) * 0x11111111u; }
// P13: bits g3 + 4 g1 -> word of g3.
__device__ __forceinline__ uint32_t exp13(uint32_t m, int g3) { return ((m >> g3) & 0x1111u) * 0xF000Fu; }
// P23: bits g2 + 4 g3 -> word w.
__device__ __forceinline__ uint32_t exp23(uint32_t m, int w) {
  return (gate(m, 2 * w) & 0xFFFFu) | (gate(m, 2 * w + 1) & 0xFFFF0000u);
}

// The sets of rotations g with five in a row for one colour, from the four
// quadrants' forms (F = OR over lines of the product of turn sets).
// With IMM the same pass also builds the immediate-win mask: a line counts
// when one quadrant uses its "one more stone" forms fi and the others f.
// TQ = -1 evaluates every line; TQ = 0..3 only the lines touching quadrant TQ
// (the others are then constant along a line of boards that varies TQ).
template <bool IMM, int TQ = -1>
__device__ __forceinline__ void eval_fives(const uint32_t (&f)[4][kFormWords], const uint32_t (&fi)[4][kFormWords],
                                           uint32_t F[8], uint32_t I[8]) {
  constexpr bool all = TQ < 0;
  constexpr bool u01 = all || TQ == 0 || TQ == 1, u02 = all || TQ == 0 || TQ == 2;
  constexpr bool u03 = all || TQ == 0 || TQ == 3, u12 = all || TQ == 1 || TQ == 2;
  constexpr bool u13 = all || TQ == 1 || TQ == 3, u23 = all || TQ == 2 || TQ == 3;
  constexpr bool uT0 = all || TQ != 2, uT1 = all || TQ != 1, uT2 = all || TQ != 3, uT3 = all || TQ != 0;
  // pair slots: A = words 0..2, B = 3..5, C = 6
  auto pair3 = [&](int a, int sa, int b, int sb, uint32_t& m, uint32_t& mi) {
    uint32_t acc = 0, acci = 0;
#pragma unroll
    for (int w = 0; w < 3; w++) {
      acc |= f[a][sa + w] & f[b][sb + w];
      if (IMM) acci |= (fi[a][sa + w] & f[b][sb + w]) | (f[a][sa + w] & fi[b][sb + w]);
    }
    m = fold16(acc);
    mi = IMM ? fold16(acci) : 0u;
  };
  auto pair1 = [&](int a, int b, uint32_t& m, uint32_t& mi) {
    m = fold16(f[a][6] & f[b][6]);
    mi = IMM ? fold16((fi[a][6] & f[b][6]) | (f[a][6] & fi[b][6])) : 0u;
  };
  uint32_t p01 = 0, p02 = 0, p03 = 0, p12 = 0, p13 = 0, p23 = 0;
  uint32_t i01 = 0, i02 = 0, i03 = 0, i12 = 0, i13 = 0, i23 = 0;
  if (u01) pair3(0, 0, 1, 0, p01, i01);
  if (u02) pair3(0, 3, 2, 3, p02, i02);
  if (u03) pair1(0, 3, p03, i03);
  if (u12) pair1(2, 1, p12, i12);
  if (u13) pair3(3, 3, 1, 3, p13, i13);
  if (u23) pair3(2, 0, 3, 0, p23, i23);
  // triples: inner pair products and gate nibbles
  const uint32_t t0 = uT0 ? (f[0][7] & f[1][7]) & 0xFFFFu : 0u, t1 = uT1 ? (f[0][7] & f[2][7]) >> 16 : 0u;
  const uint32_t t2 = uT2 ? (f[0][8] & f[1][8]) & 0xFFFFu : 0u, t3 = uT3 ? (f[2][8] & f[1][8]) >> 16 : 0u;
  const uint32_t gq3 = f[3][9], gq2 = f[2][9];
  uint32_t u0 = 0, u1 = 0, u2 = 0, u3 = 0, hq3 = 0, hq2 = 0;
  if (IMM) {
    u0 = ((fi[0][7] & f[1][7]) | (f[0][7] & fi[1][7])) & 0xFFFFu;
    u1 = ((fi[0][7] & f[2][7]) | (f[0][7] & fi[2][7])) >> 16;
    u2 = ((fi[0][8] & f[1][8]) | (f[0][8] & fi[1][8])) & 0xFFFFu;
    u3 = ((fi[2][8] & f[1][8]) | (f[2][8] & fi[1][8])) >> 16;
    hq3 = fi[3][9];
    hq2 = fi[2][9];
  }
  // words that depend only on (g0, g1): P01
  const uint32_t inv = p01 * 0x10001u, invi = i01 * 0x10001u;
  // words that depend on h = g2 >> 1
  uint32_t xh[2], xhi[2];
#pragma unroll
  for (int h = 0; h < 2; h++) {
    xh[h] = (u02 ? exp02(p02, h) : 0u) | (u12 ? exp12(p12, h) : 0u) |
            (uT2 ? (gate(gq2, 8 + 2 * h) & t2) | (gate(gq2, 9 + 2 * h) & (t2 << 16)) : 0u);
    if (IMM)
      xhi[h] = exp02(i02, h) | exp12(i12, h) | (gate(gq2, 8 + 2 * h) & u2) | (gate(gq2, 9 + 2 * h) & (u2 << 16)) |
               (gate(hq2, 8 + 2 * h) & t2) | (gate(hq2, 9 + 2 * h) & (t2 << 16));
  }
  // words that depend on g3
  uint32_t xg[4], xgi[4];
#pragma unroll
  for (int g3 = 0; g3 < 4; g3++) {
    xg[g3] = (u03 ? exp03(p03, g3) : 0u) | (u13 ? exp13(p13, g3) : 0u) |
             (uT0 ? gate(gq3, g3) & (t0 * 0x10001u) : 0u);
    if (IMM)
      xgi[g3] = exp03(i03, g3) | exp13(i13, g3) | (gate(gq3, g3) & (u0 * 0x10001u)) |
                (gate(hq3, g3) & (t0 * 0x10001u));
  }
#pragma unroll
  for (int w = 0; w < 8; w++) {
    const int h = w & 1, g3 = w >> 1;
    F[w] = inv | xh[h] | xg[g3] | (u23 ? exp23(p23, w) : 0u) | (uT1 ? gate(gq3, 4 + g3) & exp02(t1, h) : 0u) |
           (uT3 ? gate(gq3, 12 + g3) & exp12(t3, h) : 0u);
    if (IMM)
      I[w] = invi | xhi[h] | xgi[g3] | exp23(i23, w) | (gate(gq3, 4 + g3) & exp02(u1, h)) |
             (gate(hq3, 4 + g3) & exp02(t1, h)) | (gate(gq3, 12 + g3) & exp12(u3, h)) |
             (gate(hq3, 12 + g3) & exp12(t3, h));
  }
}

// Every line (the form used by the per-board kernels).
template <bool IMM>
__device__ __forceinline__ void eval_all_fives(const uint32_t (&f)[4][kFormWords], const uint32_t (&fi)[4][kFormWords],
                                           uint32_t F[8], uint32_t I[8]) {
  // pair slots: A = words 0..2, B = 3..5, C = 6
  auto pair3 = [&](int a, int sa, int b, int sb, uint32_t& m, uint32_t& mi) {
    uint32_t acc = 0, acci = 0;
#pragma unroll
    for (int w = 0; w < 3; w++) {
      acc |= f[a][sa + w] & f[b][sb + w];
      if (IMM) acci |= (fi[a][sa + w] & f[b][sb + w]) | (f[a][sa + w] & fi[b][sb + w]);
    }
    m = fold16(acc);
    mi = IMM ? fold16(acci) : 0u;
  };
  auto pair1 = [&](int a, int b, uint32_t& m, uint32_t& mi) {
    m = fold16(f[a][6] & f[b][6]);
    mi = IMM ? fold16((fi[a][6] & f[b][6]) | (f[a][6] & fi[b][6])) : 0u;
  };
  uint32_t p01, p02, p03, p12, p13, p23, i01, i02, i03, i12, i13, i23;
  pair3(0, 0, 1, 0, p01, i01);
  pair3(0, 3, 2, 3, p02, i02);
  pair1(0, 3, p03, i03);
  pair1(2, 1, p12, i12);
  pair3(3, 3, 1, 3, p13, i13);
  pair3(2, 0, 3, 0, p23, i23);
  // triples: inner pair products and gate nibbles
  const uint32_t t0 = (f[0][7] & f[1][7]) & 0xFFFFu, t1 = (f[0][7] & f[2][7]) >> 16;
  const uint32_t t2 = (f[0][8] & f[1][8]) & 0xFFFFu, t3 = (f[2][8] & f[1][8]) >> 16;
  const uint32_t gq3 = f[3][9], gq2 = f[2][9];
  uint32_t u0 = 0, u1 = 0, u2 = 0, u3 = 0, hq3 = 0, hq2 = 0;
  if (IMM) {
    u0 = ((fi[0][7] & f[1][7]) | (f[0][7] & fi[1][7])) & 0xFFFFu;
    u1 = ((fi[0][7] & f[2][7]) | (f[0][7] & fi[2][7])) >> 16;
    u2 = ((fi[0][8] & f[1][8]) | (f[0][8] & fi[1][8])) & 0xFFFFu;
    u3 = ((fi[2][8] & f[1][8]) | (f[2][8] & fi[1][8])) >> 16;
    hq3 = fi[3][9];
    hq2 = fi[2][9];
  }
  // words that depend only on (g0, g1): P01
  const uint32_t inv = p01 * 0x10001u, invi = i01 * 0x10001u;
  // words that depend on h = g2 >> 1
  uint32_t xh[2], xhi[2];
#pragma unroll
  for (int h = 0; h < 2; h++) {
    xh[h] = exp02(p02, h) | exp12(p12, h) | (gate(gq2, 8 + 2 * h) & t2) | (gate(gq2, 9 + 2 * h) & (t2 << 16));
    if (IMM)
      xhi[h] = exp02(i02, h) | exp12(i12, h) | (gate(gq2, 8 + 2 * h) & u2) | (gate(gq2, 9 + 2 * h) & (u2 << 16)) |
               (gate(hq2, 8 + 2 * h) & t2) | (gate(hq2, 9 + 2 * h) & (t2 << 16));
  }
  // words that depend on g3
  uint32_t xg[4], xgi[4];
#pragma unroll
  for (int g3 = 0; g3 < 4; g3++) {
    xg[g3] = exp03(p03, g3) | exp13(p13, g3) | (gate(gq3, g3) & (t0 * 0x10001u));
    if (IMM)
      xgi[g3] = exp03(i03, g3) | exp13(i13, g3) | (gate(gq3, g3) & (u0 * 0x10001u)) |
                (gate(hq3, g3) & (t0 * 0x10001u));
  }
#pragma unroll
  for (int w = 0; w < 8; w++) {
    const int h = w & 1, g3 = w >> 1;
    F[w] = inv | xh[h] | xg[g3] | exp23(p23, w) | (gate(gq3, 4 + g3) & exp02(t1, h)) |
           (gate(gq3, 12 + g3) & exp12(t3, h));
    if (IMM)
      I[w] = invi | xhi[h] | xgi[g3] | exp23(i23, w) | (gate(gq3, 4 + g3) & exp02(u1, h)) |
             (gate(hq3, 4 + g3) & exp02(t1, h)) | (gate(gq3, 12 + g3) & exp12(u3, h)) |
             (gate(hq3, 12 + g3) & exp12(t3, h));
  }
}

__device__ __forceinline__ void five_mask(const uint32_t (&f)[4][kFormWords], uint32_t F[8]) {
  uint32_t unused[8];
  eval_all_fives<false>(f, f, F, unused);
}

// rmax(x)(g) = OR over the 8 single-quadrant quarter turns r of x(g + r)
// (paper, "Abstracting over rotations").  For one axis, x(g+1) | x(g-1) =
// y(g+1) with y(g) = x(g) | x(g+2), and y has period 2 along that axis.
__device__ __forceinline__ void rmax(const uint32_t x[8], uint32_t r[8]) {
  uint32_t a2[4], v[4];
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const uint32_t u = x[2 * j] | x[2 * j + 1];  // axis 2: fold g2 with g2 + 2
    a2[j] = __funnelshift_l(u, u, 16);           // then step g2 by one
    v[j] = x[j] | x[j + 4];                      // axis 3: fold g3 with g3 + 2
  }
#pragma unroll
  for (int w = 0; w < 8; w++) {
    const uint32_t y0 = x[w] | ((x[w] >> 2) & 0x33333333u) | ((x[w] << 2) & 0xCCCCCCCCu);
    const uint32_t a0 = ((y0 >> 1) & 0x55555555u) | ((y0 << 1) & 0xAAAAAAAAu);
    const uint32_t y1 = x[w] | __byte_perm(x[w], 0, 0x2301);
    const uint32_t a1 = ((y1 >> 4) & 0x0F0F0F0Fu) | ((y1 << 4) & 0xF0F0F0F0u);
    r[w] = a0 | a1 | a2[w >> 1] | v[(w + 2) & 3];
  }
}

// result(g) = x(g + u e_q): the value of a child whose quadrant q is u
// anticlockwise turns past the stored rotation-minimal pattern.
template <int Q>
__device__ __forceinline__ void shift_axis(uint32_t x[8], uint32_t u) {
  if (Q == 0) {
    const uint32_t M = u == 0 ? 0xFFFFFFFFu : u == 1 ? 0x77777777u : u == 2 ? 0x33333333u : 0x11111111u;
#pragma unroll
    for (int w = 0; w < 8; w++) x[w] = ((x[w] >> u) & M) | ((x[w] << ((4 - u) & 3)) & ~M);
  } else if (Q == 1) {
    const uint32_t M = u == 0 ? 0xFFFFFFFFu : u == 1 ? 0x0FFF0FFFu : u == 2 ? 0x00FF00FFu : 0x000F000Fu;
#pragma unroll
    for (int w = 0; w < 8; w++) x[w] = ((x[w] >> (4 * u)) & M) | ((x[w] << ((16 - 4 * u) & 15)) & ~M);
  } else if (Q == 2) {
#pragma unroll
    for (int j = 0; j < 4; j++) {
      uint32_t lo = x[2 * j], hi = x[2 * j + 1];
      if (u & 2) {
        const uint32_t t = lo;
        lo = hi;
        hi = t;
      }
      if (u & 1) {
        const uint32_t l2 = __funnelshift_r(lo, hi, 16), h2 = __funnelshift_r(hi, lo, 16);
        lo = l2;
        hi = h2;
      }
      x[2 * j] = lo;
      x[2 * j + 1] = hi;
    }
  } else {
    uint32_t y[8];
#pragma unroll
    for (int w = 0; w < 8; w++) y[w] = (u & 2) ? x[w ^ 4] : x[w];
#pragma unroll
    for (int w = 0; w < 8; w++) x[w] = (u & 1) ? y[(w + 2) & 7] : y[w];
  }
}

// ---------------------------------------------------------------------------
// Re-orienting a 256-entry bit table (paper, "Abstracting over rotations":
// transforming f_b into f_{gb} for g in D4 takes dimension transpositions and
// reflections of the 4x4x4x4 array).  Entry beta = g0 + 4 g1 + 16 g2 + 64 g3
// sits in word beta >> 5, bit beta & 31: index bits 0-4 lie inside a word,
// bits 5-7 select the word.  Every step below is an exchange of entries
// decided by index bits known at compile time (a "delta swap").
// ---------------------------------------------------------------------------
__host__ __device__ constexpr uint32_t index_mask(int set_bit, int clear_bit) {
  // in-word positions p with bit set_bit of p set and bit clear_bit clear
  // (clear_bit >= 5 means no condition)
  uint32_t m = 0;
  for (int p = 0; p < 32; p++)
    if ((p >> set_bit & 1) && (clear_bit >= 5 || !(p >> clear_bit & 1))) m |= 1u << p;
  return m;
}

// Exchange the entries whose index bits I < J read (1, 0) with those reading
// (0, 1): out[beta] = in[beta with bits I and J swapped].
template <int I, int J>
__device__ __forceinline__ void swap_index_bits(uint32_t T[8]) {
  static_assert(I < J && J < 8, "index bits");
  if constexpr (J < 5) {
    constexpr int s = (1 << J) - (1 << I);
    constexpr uint32_t m = index_mask(I, J);
#pragma unroll
    for (int w = 0; w < 8; w++) {
      const uint32_t t = (T[w] ^ (T[w] >> s)) & m;
      T[w] ^= t ^ (t << s);
    }
  } else if constexpr (I < 5) {
    constexpr int jw = 1 << (J - 5), d = 1 << I;
    constexpr uint32_t m0 = ~index_mask(I, 5);  // positions with bit I clear
#pragma unroll
    for (int w = 0; w < 8; w++) {
      if (w & jw) continue;
      const uint32_t t = ((T[w] >> d) ^ T[w | jw]) & m0;
      T[w | jw] ^= t;
      T[w] ^= t << d;
    }
  } else {
    constexpr int iw = 1 << (I - 5), jw = 1 << (J - 5);
#pragma unroll
    for (int w = 0; w < 8; w++) {
      if ((w & iw) && !(w & jw)) {
        const uint32_t t = T[w];
        T[w] = T[w ^ iw ^ jw];
        T[w ^ iw ^ jw] = t;
      }
    }
  }
}

// out[g] = in[-g] (every axis negated mod 4: turns 1 and 3 trade places, so
// along axis a the entries with low index bit 2a set exchange across bit 2a+1).
__device__ __forceinline__ void negate_axes(uint32_t T[8]) {
  constexpr uint32_t m0 = index_mask(0, 1), m1 = index_mask(2, 3), m2 = index_mask(4, 5);
#pragma unroll
  for (int w = 0; w < 8; w++) {
    uint32_t t = (T[w] ^ (T[w] >> 2)) & m0;  // axis 0: bit 0 set, exchange across bit 1
    T[w] ^= t ^ (t << 2);
    t = (T[w] ^ (T[w] >> 8)) & m1;  // axis 1: bit 2 set, exchange across bit 3
    T[w] ^= t ^ (t << 8);
  }
#pragma unroll
  for (int w = 0; w < 8; w += 2) {  // axis 2: bit 4 set (upper halves), exchange across word bit 0
    const uint32_t t = (T[w] ^ T[w + 1]) & m2;
    T[w] ^= t;
    T[w + 1] ^= t;
  }
#pragma unroll
  for (int w = 2; w < 4; w++) {  // axis 3: word bit 1 set, exchange across word bit 2
    const uint32_t t = T[w];
    T[w] = T[w + 4];
    T[w + 4] = t;
  }
}

// out[g] = in[g with components A and B exchanged]
template <int A, int B>
__device__ __forceinline__ void swap_axes(uint32_t T[8]) {
  swap_index_bits<2 * A, 2 * B>(T);
  swap_index_bits<2 * A + 1, 2 * B + 1>(T);
}

__host__ __device__ constexpr int swap_value(int x, int a, int b) { return x == a ? b : x == b ? a : x; }

// out[g] = in[z], z[P_q] = g[q]: a product of axis exchanges.  Exchanging a
// and P_a first leaves the permutation swap(a, P_a) o P, which fixes a.
template <int P0, int P1, int P2, int P3>
__device__ __forceinline__ void permute_axes(uint32_t T[8]) {
  constexpr int a = P0 != 0 ? 0 : P1 != 1 ? 1 : P2 != 2 ? 2 : P3 != 3 ? 3 : -1;
  if constexpr (a >= 0) {
    constexpr int b = a == 0 ? P0 : a == 1 ? P1 : a == 2 ? P2 : P3;
    swap_axes<(a < b ? a : b), (a < b ? b : a)>(T);
    permute_axes<swap_value(P0, a, b), swap_value(P1, a, b), swap_value(P2, a, b), swap_value(P3, a, b)>(T);
  }
}

// out[g] = in[phi_S(g)], phi_S(g)[sym_qmap(S, q)] = eps_S g[q]: a table kept
// in the frame of the board S b read in the frame of b.
template <int S>
__device__ __forceinline__ void reorient(uint32_t T[8]) {
  if constexpr (sym_reflects(S)) negate_axes(T);
  permute_axes<sym_qmap(S, 0), sym_qmap(S, 1), sym_qmap(S, 2), sym_qmap(S, 3)>(T);
}

__device__ __forceinline__ void load_super(const pp_super* p, uint32_t W[8], uint32_t N[8]) {
  const uint4* v = reinterpret_cast<const uint4*>(p);
  const uint4 a = __ldg(v), b = __ldg(v + 1), c = __ldg(v + 2), d = __ldg(v + 3);
  W[0] = a.x, W[1] = a.y, W[2] = a.z, W[3] = a.w, W[4] = b.x, W[5] = b.y, W[6] = b.z, W[7] = b.w;
  N[0] = c.x, N[1] = c.y, N[2] = c.z, N[3] = c.w, N[4] = d.x, N[5] = d.y, N[6] = d.z, N[7] = d.w;
}

__device__ __forceinline__ void store_super(pp_super* p, const uint32_t W[8], const uint32_t N[8]) {
  uint4* v = reinterpret_cast<uint4*>(p);
  v[0] = make_uint4(W[0], W[1], W[2], W[3]);
  v[1] = make_uint4(W[4], W[5], W[6], W[7]);
  v[2] = make_uint4(N[0], N[1], N[2], N[3]);
  v[3] = make_uint4(N[4], N[5], N[6], N[7]);
}

// Value of one position from its move accumulators (paper, "Problem
// definition", with the rotation abstraction of "Abstracting over rotations"):
//   terminal (T = F_c | F_o):  win = F_c & ~F_o,  notlose = F_c | ~F_o
//   otherwise win = I | rmax(OR_e ~notlose_child), notlose = I | rmax(OR_e ~win_child)
// rmax distributes over OR, so one rmax per table covers all moves.  With
// prepared children (each child value stored as (~rmax(~win), ~rmax(~notlose)),
// pp_prepare_children) the accumulators already hold OR_e rmax(~notlose_e)
// and OR_e rmax(~win_e): rmax also commutes with the turns applied to a
// child, so the per-board rmax is skipped.
__device__ __forceinline__ void combine(const uint32_t Fc[8], const uint32_t Fo[8], const uint32_t I[8],
                                        const uint32_t AW[8], const uint32_t AN[8], uint32_t W[8], uint32_t N[8],
                                        bool prepared = false) {
  uint32_t RW[8], RN[8];
  if (prepared) {
#pragma unroll
    for (int w = 0; w < 8; w++) RW[w] = AW[w], RN[w] = AN[w];
  } else {
    rmax(AW, RW);
    rmax(AN, RN);
  }
#pragma unroll
  for (int w = 0; w < 8; w++) {
    const uint32_t T = Fc[w] | Fo[w];
    W[w] = (Fc[w] & ~Fo[w]) | (~T & (I[w] | RW[w]));
    N[w] = Fc[w] | (~T & (I[w] | RN[w]));
  }
}

// ---------------------------------------------------------------------------
// Midgame level kernel: every fill with `level` stones added, for every board
// segment of this launch (paper, "Open source and data").
// ---------------------------------------------------------------------------
// Index of the last descriptor whose first block is <= b (uniform per block).
template <typename T>
__device__ __forceinline__ int find_block_owner(const T* __restrict__ d, int n, uint32_t b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (d[mid].block0 <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// 256-bit accesses (sm_100 and later): one load or store instruction per 32
// bytes, half the instructions and L1 sector lookups of 128-bit accesses to
// the same scattered addresses.  The address must be 32-byte aligned.
// Read-only data (written by an earlier launch): the compiler may schedule
// the load freely.
__device__ __forceinline__ void ld256_nc(const void* p, uint32_t r[8]) {
  asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "l"(p));
}
// Data other blocks of the same launch wrote before a grid barrier: read
// through L2, ordered with the barrier.
__device__ __forceinline__ void ld256_cg(const void* p, uint32_t r[8]) {
  asm volatile("ld.global.cg.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "l"(p)
               : "memory");
}
__device__ __forceinline__ void st256(void* p, const uint32_t r[8]) {
  asm volatile("st.global.v8.u32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(r[0]), "r"(r[1]), "r"(r[2]),
               "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}

// Child values of a level are read through L2 (__ldcg) when the reading and
// writing levels run in the same launch: L1 is not coherent across SMs.
template <bool L2ONLY>
__device__ __forceinline__ void load_child(const pp_super* p, uint32_t W[8], uint32_t N[8]) {
  if (L2ONLY) {
    ld256_cg(p->win, W);
    ld256_cg(p->notlose, N);
  } else {
    ld256_nc(p->win, W);
    ld256_nc(p->notlose, N);
  }
}

__device__ __forceinline__ void load_mask(const uint4* p, uint32_t F[8]) { ld256_nc(p, F); }

// A super value with two 256-bit accesses (32-byte aligned arrays: the
// section and line kernels, whose entry points require that alignment).
__device__ __forceinline__ void load_super32(const pp_super* p, uint32_t W[8], uint32_t N[8]) {
  ld256_nc(p->win, W);
  ld256_nc(p->notlose, N);
}
__device__ __forceinline__ void store_super32(pp_super* p, const uint32_t W[8], const uint32_t N[8]) {
  st256(p->win, W);
  st256(p->notlose, N);
}

// Rotated five-in-a-row masks of one colour for every subset of a board's
// empty cells (paper, "Abstracting over rotations": the set of g for which a
// colour's stones hold five in a row depends on that colour's stones only).
// Entry r = (colour - 1) 2^k + subset of board b's table (32 bytes, at
// masks + 2 (b.masks + r) in uint4) is the mask of the colour's root stones
// plus its stones on the slots in subset.  Every fill of the board reads its
// two masks and its immediate wins from here instead of evaluating lines.
// Only subsets a fill can hold are computed (39% fewer for 12 empty cells):
// a fill holds ceil(k/2) stones of the colour that moves first and floor(k/2)
// of the other.  Thread x of a board takes the x-th such subset in
// increasing order, black's before white's, so the threads left idle form
// whole warps at the end of each board's range and a warp's stores stay
// close together.
// Which board descriptor the kernel's board i is: i itself (a plan's boards),
// or the i-th entry of a slot list passed in the launch's parameters (the
// queries a server admitted at once).
struct BoardsInOrder {
  __device__ uint32_t operator()(uint32_t i) const { return i; }
};
struct BoardSlots {
  uint16_t slot[kSlotBatch];
  __device__ uint32_t operator()(uint32_t i) const { return slot[i]; }
};

template <class Which>
__global__ void five_table_kernel(const MidBoard* __restrict__ boards, int n, int kmax, uint4* __restrict__ masks,
                                  const __grid_constant__ Which which) {
  // S[a * 17 + b] = number of subsets of a slots with at most b of them;
  // block b of the subset list starts at sum over c < b of S[16 * 17 + c]
  __shared__ uint32_t S[17 * 17], off[17];
  for (int a = threadIdx.x; a < 17; a += blockDim.x) {
    uint32_t c = 1, sum = 0;
    for (int b = 0; b <= 16; b++) {
      sum += b <= a ? c : 0u;
      S[a * 17 + b] = sum;
      if (b < a) c = c * (uint32_t)(a - b) / (uint32_t)(b + 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t at = 0;
    for (int b = 0; b <= 16; b++) off[b] = at, at += b <= kMaxEmpty / 2 ? S[16 * 17 + b] : 0u;
  }
  __syncthreads();
  const uint64_t per = 2ull << kmax;
  const uint64_t total = (uint64_t)n * per;
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const MidBoard& B = boards[which((uint32_t)(t >> (kmax + 1)))];
    const int k = (int)B.k, capb = B.mover == 1 ? (k + 1) / 2 : k / 2, capw = k - capb;
    const uint32_t nb = S[k * 17 + capb], nw = S[k * 17 + capw];
    uint32_t x = (uint32_t)(t & (per - 1));
    if (x >= nb + nw) continue;
    const uint32_t white = x >= nb;
    const uint32_t subset = __ldg(c_tab.subsets + off[white ? capw : capb] + (white ? x - nb : x));
    const uint32_t r = (white << k) | subset;
    uint32_t f[4][kFormWords];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      uint32_t p = white ? B.root_w[q] : B.root_b[q];
      for (int i = B.qstart[q]; i < B.qstart[q + 1]; i++) p |= (subset >> i & 1u) << B.slot_bit[i];
      load_forms(q, p, f[q]);
    }
    uint32_t F[8];
    five_mask(f, F);
    uint4* o = masks + 2 * (B.masks + r);
    o[0] = make_uint4(F[0], F[1], F[2], F[3]);
    o[1] = make_uint4(F[4], F[5], F[6], F[7]);
  }
}

// ---------------------------------------------------------------------------
// Half tables (paper, "Open source and data": rmax flips the parity of
// g0 + g1 + g2 + g3, so a solve that wants one parity class at the root
// needs only one class at every level, alternating, and stores 32 bytes per
// position instead of 64).  Parity of beta(g) = b0 ^ b2 ^ b4 ^ b6: inside a
// word, neighbouring bits (b0 = 0, 1) belong to opposite classes, and b6 is
// word bit 1.  A class's 16 bits of a word are gathered to the even bit
// positions; words 2j and 2j + 1 (same class pattern) then share one word,
// 2j at even and 2j + 1 at odd positions.  Bits of the other class are not
// stored and unpack as zero: rmax, the combine and the five masks never let
// them reach the wanted class.
// ---------------------------------------------------------------------------
constexpr uint32_t kClass0 = 0x5A5AA5A5u;  // in-word positions t with t0 ^ t2 ^ t4 = 0

__device__ __forceinline__ uint32_t class_bits(uint32_t p, int w) {
  return ((p ^ (uint32_t)(w >> 1)) & 1u) ? ~kClass0 : kClass0;
}

// 8 words (class p valid) -> 4 words
__device__ __forceinline__ void half_pack(const uint32_t x[8], uint32_t p, uint32_t h[4]) {
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const uint32_t K = class_bits(p, 2 * j), E = K & 0x55555555u, O = (K >> 1) & 0x55555555u;
    const uint32_t a = (x[2 * j] & E) | ((x[2 * j] >> 1) & O);
    const uint32_t b = (x[2 * j + 1] & E) | ((x[2 * j + 1] >> 1) & O);
    h[j] = a | (b << 1);
  }
}

// 4 words -> 8 words, the other class zero
__device__ __forceinline__ void half_unpack(const uint32_t h[4], uint32_t p, uint32_t x[8]) {
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const uint32_t K = class_bits(p, 2 * j), E = K & 0x55555555u, O = (K >> 1) & 0x55555555u;
    const uint32_t a = h[j] & 0x55555555u, b = (h[j] >> 1) & 0x55555555u;
    x[2 * j] = (a & E) | ((a & O) << 1);
    x[2 * j + 1] = (b & E) | ((b & O) << 1);
  }
}

// One thread block's worth (kBlock fills) of one midgame level: block vb of
// the level's segments (paper, "Open source and data").
//
// A fill's value folds its children: on rotations where the fill has no
// five, win = OR_e (I_e | rmax(~notlose_e)) and notlose = OR_e (I_e |
// rmax(~win_e)), where I_e, the mover's five after the move e, is the
// child's five-in-a-row set of the colour that is not to move there (rmax
// distributes over OR; paper, "Abstracting over rotations").  So every fill
// below the root stores, instead of its value, the two tables its parents
// OR: (F_o | rmax(~notlose), F_o | rmax(~win)), F_o its own five-in-a-row
// set of the colour not to move.  A parent then reads one 64-byte record
// per move and takes no rmax; each fill still takes two.  The root stores
// its value.  A fill's own masks come from the board's colour-subset five
// tables (five_table_kernel); its children from the level below.
template <bool L2ONLY, bool HALF>
__device__ __forceinline__ void midgame_fill(const MidBoard* __restrict__ boards, const MidSeg* __restrict__ segs,
                                             int nsegs, uint32_t vb, pp_super* __restrict__ table,
                                             pp_super* __restrict__ out, int final_level,
                                             const uint4* __restrict__ masks, uint32_t seg_blocks, uint32_t parity) {
  // segments of equal size (boards sharing k and mover): the owner is a division;
  // shared segments: one stored descriptor, the board follows from the owner
  const uint32_t per = seg_blocks & ~kSharedSegs;
  const int owner = per ? (int)(vb / per) : find_block_owner(segs, nsegs, vb);
  MidSeg sg = segs[(seg_blocks & kSharedSegs) ? 0 : owner];
  if (seg_blocks & kSharedSegs) sg.board += (uint32_t)owner, sg.block0 = (uint32_t)owner * per;
  const uint32_t e = (vb - sg.block0) * kBlock + threadIdx.x;
  if (e >= sg.count) return;
  const uint64_t entry = __ldg(sg.list + e);
  const uint32_t bm = (uint32_t)(entry >> 32) & 0xFFFFu, wm = (uint32_t)(entry >> 48);
  const MidBoard& B = boards[sg.board];
  const int k = (int)B.k, level = (int)sg.level;
  const uint32_t c = (level & 1) ? 3u - B.mover : B.mover;  // colour to move
  const uint4* mt = masks + 2 * B.masks;
  const uint32_t kk = 1u << k, mc = c == 1 ? bm : wm, mo = c == 1 ? wm : bm;
  const uint4* mtc = mt + 2 * ((c - 1) * kk);  // the mover's table
  const uint32_t own = (parity ^ (uint32_t)level) & 1u;  // half: this level's class (its children store it)
  uint32_t Fc[8], Fo[8], W[8], N[8];
  if (level == k) {  // full board
    load_mask(mtc + 2 * mc, Fc);
    load_mask(mt + 2 * ((2 - c) * kk + mo), Fo);
#pragma unroll
    for (int w = 0; w < 8; w++) W[w] = Fc[w] & ~Fo[w], N[w] = Fc[w] | ~Fo[w];
  } else {
    uint32_t AW[8] = {0}, AN[8] = {0};
    // compact table: level + 1 starts at coff; the fill's children's
    // positions there are listed in slot order
    const pp_super* tab = table + B.table + sg.coff;
    const uint32_t* htab = reinterpret_cast<const uint32_t*>(table) + 8 * ((uint64_t)B.table + sg.coff);  // half
    const uint32_t moves = (uint32_t)(k - level);
    const uint32_t* __restrict__ rk = sg.ranks + (uint64_t)e * moves;
    auto fold = [&](uint32_t child) {
      uint32_t cW[8], cN[8];
      if (HALF) {
        uint32_t h[8];
        const uint32_t* src = htab + 8 * (uint64_t)child;
        if (L2ONLY)
          ld256_cg(src, h);
        else
          ld256_nc(src, h);
        half_unpack(h, own, cW);
        half_unpack(h + 4, own, cN);
      } else {
        load_child<L2ONLY>(tab + child, cW, cN);
      }
#pragma unroll
      for (int w = 0; w < 8; w++) AW[w] |= cW[w], AN[w] |= cN[w];
    };
    if constexpr (L2ONLY) {
      // persistent kernel (80 registers): two moves per round, both
      // children's loads in flight together, the next round's positions
      // read while they are
      uint32_t r0 = __ldg(rk), r1 = moves > 1 ? __ldg(rk + 1) : 0u;  // level < k: at least one move
      uint32_t m = 0;
      for (; m + 1 < moves; m += 2) {
        const uint32_t a = r0, b = r1;
        if (m + 2 < moves) r0 = __ldg(rk + m + 2);
        if (m + 3 < moves) r1 = __ldg(rk + m + 3);
        fold(a);
        fold(b);
      }
      if (m < moves) fold(r0);
    } else {
      // level kernel (64 registers, 4 blocks per SM): one move at a time,
      // the next move's position in flight with this child
      uint32_t next = __ldg(rk);
      for (uint32_t m = 0; m < moves; m++) {
        const uint32_t child = next;
        if (m + 1 < moves) next = __ldg(rk + m + 1);
        fold(child);
      }
    }
    // the position's own masks, loaded last to keep the loop's registers free
    load_mask(mtc + 2 * mc, Fc);
    load_mask(mt + 2 * ((2 - c) * kk + mo), Fo);
#pragma unroll
    for (int w = 0; w < 8; w++) {
      const uint32_t T = Fc[w] | Fo[w];
      W[w] = (Fc[w] & ~Fo[w]) | (~T & AW[w]);
      N[w] = Fc[w] | (~T & AN[w]);
    }
  }
  if (final_level || sg.final) {
    if (HALF) {  // the root: the wanted class, the other zero
#pragma unroll
      for (int w = 0; w < 8; w++) {
        const uint32_t K = class_bits(parity, w);
        W[w] &= K, N[w] &= K;
      }
    }
    store_super(out + B.out, W, N);
    return;
  }
  // the tables the parents OR
  uint32_t P[8], R[8];
#pragma unroll
  for (int w = 0; w < 8; w++) N[w] = ~N[w], W[w] = ~W[w];
  rmax(N, P);
  rmax(W, R);
#pragma unroll
  for (int w = 0; w < 8; w++) P[w] |= Fo[w], R[w] |= Fo[w];
  if (HALF) {  // on the parents' class
    uint32_t h[8];
    half_pack(P, own ^ 1u, h);
    half_pack(R, own ^ 1u, h + 4);
    st256(reinterpret_cast<uint32_t*>(table) + 8 * ((uint64_t)B.table + sg.loff + e), h);
  } else {
    pp_super* r = table + B.table + sg.loff + e;
    st256(r->win, P);
    st256(r->notlose, R);
  }
}

template <bool HALF>
__global__ void __launch_bounds__(kBlock, PP_MID_MINB) midgame_level_kernel(const MidBoard* __restrict__ boards,
                                                               const MidSeg* __restrict__ segs, int nsegs,
                                                               pp_super* __restrict__ table,
                                                               pp_super* __restrict__ out, int final_level,
                                                               const uint4* __restrict__ masks, uint32_t seg_blocks,
                                                               uint32_t parity) {
  midgame_fill<false, HALF>(boards, segs, nsegs, blockIdx.x, table, out, final_level, masks, seg_blocks, parity);
}

// Grid-wide barrier for a cooperative launch (every block resident).  The
// wait is bounded: after kBarrierSpins polls it records PP_ETIMEOUT in
// *status and lets the block go; the kernel then stops at its next level and
// the host reports the error.  bar[0] counts arrivals, bar[1] is the
// generation.
constexpr uint32_t kBarrierSpins = 1u << 25;  // about 2 s at 64 ns per poll
// the limit the persistent midgame launches use (a failure-path test lowers it)
static std::atomic<uint32_t> g_barrier_spins{kBarrierSpins};
void set_barrier_spins(uint32_t polls) { g_barrier_spins.store(polls ? polls : kBarrierSpins); }

__device__ __forceinline__ bool grid_barrier(uint32_t* bar, uint32_t* status, uint32_t limit) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t* vgen = bar + 1;
    const uint32_t gen = *vgen;
    if (atomicAdd(bar, 1u) + 1 == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      uint32_t spins = 0;
      while (*vgen == gen) {
        if (++spins > limit) {
          atomicExch(status, (uint32_t)PP_ETIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile uint32_t*)status == 0;
}

// Self-test of the bounded wait: block 1 never arrives, so block 0's wait
// must run out and record PP_ETIMEOUT.
__global__ void barrier_probe_kernel(uint32_t* sync, uint32_t limit) {
  if (blockIdx.x != 0) return;
  grid_barrier(sync, sync + 2, limit);
}

// All levels of a plan in one cooperative launch: level after level, each
// block strides over the level's thread blocks, then the grid meets at the
// barrier.
template <bool HALF>
__global__ void __launch_bounds__(kBlock, PP_MIDP_MINB) midgame_persistent_kernel(
    const MidBoard* __restrict__ boards, const MidSeg* __restrict__ segs, const MidLevel* __restrict__ levels,
    int nlevels, pp_super* __restrict__ table, pp_super* __restrict__ out, uint32_t* bar, uint32_t* status,
    const uint4* __restrict__ masks, uint32_t parity, uint32_t spins) {
  for (int L = 0; L < nlevels; L++) {
    const MidLevel lv = levels[L];
    for (uint32_t vb = blockIdx.x; vb < lv.blocks; vb += gridDim.x)
      midgame_fill<true, HALF>(boards, segs + lv.seg0, lv.nsegs, vb, table, out, L + 1 == nlevels, masks,
                               lv.seg_blocks, parity);
    if (L + 1 < nlevels && !grid_barrier(bar, status, spins)) return;
  }
}

// ---------------------------------------------------------------------------
// Section kernel: one thread per parent board of every task (paper, "Data
// layout and distribution"; the child of a move in quadrant q lies in the
// section with one more stone there, on the line through the parent's other
// three indices).
// ---------------------------------------------------------------------------
template <int Q>
__device__ __forceinline__ void section_moves(const SecTask& tk, const uint32_t code[4], const uint32_t idx[4],
                                              const uint32_t pc[4], uint32_t cdig,
                                              uint32_t AW[8], uint32_t AN[8], uint32_t fi[kFormWords]) {
#pragma unroll
  for (int w = 0; w < kFormWords; w++) fi[w] = 0;
  if (!(tk.movable >> Q & 1)) return;
  const uint32_t dec = __ldg(c_tab.qdecode + code[Q]);
  uint32_t empty = ~(dec | dec >> 9) & 0x1FFu;
  const pp_super* __restrict__ in = tk.child[Q];
  uint64_t base = 0;
#pragma unroll
  for (int q = 0; q < 4; q++)
    if (q != Q) base += (uint64_t)idx[q] * tk.cstride[Q][q];
  while (empty) {
    const int e = __ffs(empty) - 1;
    empty &= empty - 1;
    const uint32_t s = __ldg(c_tab.standard + code[Q] + cdig * c_pow3[e]);
    uint32_t cW[8], cN[8], g[kFormWords];
    load_super32(in + base + (uint64_t)(s & 0xFFFFu) * tk.cstride[Q][Q], cW, cN);
    shift_axis<Q>(cW, s >> 16);
    shift_axis<Q>(cN, s >> 16);
#pragma unroll
    for (int w = 0; w < 8; w++) AW[w] |= ~cN[w], AN[w] |= ~cW[w];
    load_forms(Q, pc[Q] | 1u << e, g);
#pragma unroll
    for (int w = 0; w < kFormWords; w++) fi[w] |= g[w];
  }
}

// Turn both accumulated tables along child axis sym_qmap(S, q) (a quadrant
// the move left unchanged).
template <int S, int Q, int q>
__device__ __forceinline__ void fixed_turn(uint32_t W[8], uint32_t N[8], uint32_t t) {
  if constexpr (q != Q) {
    shift_axis<sym_qmap(S, q)>(W, t);
    shift_axis<sym_qmap(S, q)>(N, t);
  }
}

// Moves in quadrant Q whose child section is stored as its image under
// symmetry S (paper, "Data layout and distribution": only D4-minimal sections
// are computed; Fig. "lines": such input lines are turned before use).  The
// child c is read as c* = (S c with every quadrant standardised), c's
// quadrant q landing at sym_qmap(S, q) turned t_q from its minimal pattern,
// and f_c(g) = f_{c*}(phi_S(g) + t).  The three unchanged quadrants' turns
// are the same for every move of Q, so the children are OR-ed in c*'s frame
// and turned and re-oriented once.
template <int Q, int S>
__device__ __forceinline__ void section_moves_sym(const SecTask& tk, const uint32_t code[4], const uint32_t idx[4],
                                                  const uint32_t pc[4], uint32_t cdig, uint32_t empty,
                                                  uint32_t AW[8], uint32_t AN[8], uint32_t fi[kFormWords]) {
  constexpr int PQ = sym_qmap(S, Q);
  const uint16_t* __restrict__ dm = c_tab.dmin + S * kMinStates;
  const pp_super* __restrict__ in = tk.child[Q];
  uint64_t base = 0;
  uint32_t tfix[4] = {0, 0, 0, 0};
#pragma unroll
  for (int q = 0; q < 4; q++) {
    if (q == Q) continue;
    const uint32_t v = __ldg(dm + tk.qoff[q] + idx[q]);
    base += (uint64_t)(v & 0xFFFu) * tk.cstride[Q][sym_qmap(S, q)];
    tfix[q] = v >> 12;
  }
  uint32_t accW[8], accN[8];
#pragma unroll
  for (int w = 0; w < 8; w++) accW[w] = 0, accN[w] = 0;
  while (empty) {
    const int e = __ffs(empty) - 1;
    empty &= empty - 1;
    const uint32_t st = __ldg(c_tab.standard + code[Q] + cdig * c_pow3[e]);
    const uint32_t v = __ldg(dm + tk.cqoff[Q] + (st & 0xFFFFu));
    // the moved pattern is u = st >> 16 turns past its minimal state m; S
    // carries it u (or -u, for a reflection) turns past S m, which is
    // v >> 12 turns past its own minimal state
    const uint32_t t = ((v >> 12) + (sym_reflects(S) ? 4u - (st >> 16) : (st >> 16))) & 3u;
    uint32_t cW[8], cN[8], g[kFormWords];
    load_super32(in + base + (uint64_t)(v & 0xFFFu) * tk.cstride[Q][PQ], cW, cN);
    shift_axis<PQ>(cW, t);
    shift_axis<PQ>(cN, t);
#pragma unroll
    for (int w = 0; w < 8; w++) accW[w] |= ~cN[w], accN[w] |= ~cW[w];
    load_forms(Q, pc[Q] | 1u << e, g);
#pragma unroll
    for (int w = 0; w < kFormWords; w++) fi[w] |= g[w];
  }
  fixed_turn<S, Q, 0>(accW, accN, tfix[0]);
  fixed_turn<S, Q, 1>(accW, accN, tfix[1]);
  fixed_turn<S, Q, 2>(accW, accN, tfix[2]);
  fixed_turn<S, Q, 3>(accW, accN, tfix[3]);
  reorient<S>(accW);
  reorient<S>(accN);
#pragma unroll
  for (int w = 0; w < 8; w++) AW[w] |= accW[w], AN[w] |= accN[w];
}

// Moves in quadrant Q for D4-reduced slices: the symmetry is the same for
// every board of the task, so the branch is uniform.
template <int Q>
__device__ __forceinline__ void section_moves_d4(const SecTask& tk, const uint32_t code[4], const uint32_t idx[4],
                                                 const uint32_t pc[4], uint32_t cdig,
                                                 uint32_t AW[8], uint32_t AN[8], uint32_t fi[kFormWords]) {
  const int S = tk.sym[Q];
  if (S == 0 || !(tk.movable >> Q & 1)) {
    section_moves<Q>(tk, code, idx, pc, cdig, AW, AN, fi);
    return;
  }
#pragma unroll
  for (int w = 0; w < kFormWords; w++) fi[w] = 0;
  const uint32_t dec = __ldg(c_tab.qdecode + code[Q]);
  const uint32_t empty = ~(dec | dec >> 9) & 0x1FFu;
  switch (S) {
    case 1: section_moves_sym<Q, 1>(tk, code, idx, pc, cdig, empty, AW, AN, fi); break;
    case 2: section_moves_sym<Q, 2>(tk, code, idx, pc, cdig, empty, AW, AN, fi); break;
    case 3: section_moves_sym<Q, 3>(tk, code, idx, pc, cdig, empty, AW, AN, fi); break;
    case 4: section_moves_sym<Q, 4>(tk, code, idx, pc, cdig, empty, AW, AN, fi); break;
    case 5: section_moves_sym<Q, 5>(tk, code, idx, pc, cdig, empty, AW, AN, fi); break;
    case 6: section_moves_sym<Q, 6>(tk, code, idx, pc, cdig, empty, AW, AN, fi); break;
    default: section_moves_sym<Q, 7>(tk, code, idx, pc, cdig, empty, AW, AN, fi); break;
  }
}

template <bool D4>
__device__ __forceinline__ void section_block(const SecTask* __restrict__ tasks, int ntasks, uint32_t vb,
                                              pp_super* __restrict__ out) {
  const SecTask& tk = tasks[find_block_owner(tasks, ntasks, vb)];
  const uint32_t L = (vb - tk.block0) * kBlock + threadIdx.x;
  if (L >= tk.size) return;
  uint32_t idx[4], code[4], pb[4], pw[4];
  uint32_t r = L;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    idx[q] = r % tk.dim[q];
    r /= tk.dim[q];
    code[q] = __ldg(c_tab.qlist + tk.qoff[q] + idx[q]);
    const uint32_t dec = __ldg(c_tab.qdecode + code[q]);
    pb[q] = dec & 0x1FFu;
    pw[q] = (dec >> 9) & 0x1FFu;
  }
  const uint32_t c = tk.mover;
  const uint32_t* pc = c == 1 ? pb : pw;
  const uint32_t* po = c == 1 ? pw : pb;
  uint32_t fc[4][kFormWords], fo[4][kFormWords];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    load_forms(q, pc[q], fc[q]);
    load_forms(q, po[q], fo[q]);
  }
  uint32_t Fo[8], Fc[8], W[8], N[8];
  five_mask(fo, Fo);
  if (!tk.movable) {  // full board
    five_mask(fc, Fc);
#pragma unroll
    for (int w = 0; w < 8; w++) W[w] = Fc[w] & ~Fo[w], N[w] = Fc[w] | ~Fo[w];
  } else {
    uint32_t AW[8] = {0}, AN[8] = {0}, fi[4][kFormWords], I[8];
    if (D4) {
      section_moves_d4<0>(tk, code, idx, pc, c, AW, AN, fi[0]);
      section_moves_d4<1>(tk, code, idx, pc, c, AW, AN, fi[1]);
      section_moves_d4<2>(tk, code, idx, pc, c, AW, AN, fi[2]);
      section_moves_d4<3>(tk, code, idx, pc, c, AW, AN, fi[3]);
    } else {
      section_moves<0>(tk, code, idx, pc, c, AW, AN, fi[0]);
      section_moves<1>(tk, code, idx, pc, c, AW, AN, fi[1]);
      section_moves<2>(tk, code, idx, pc, c, AW, AN, fi[2]);
      section_moves<3>(tk, code, idx, pc, c, AW, AN, fi[3]);
    }
    eval_all_fives<true>(fc, fi, Fc, I);
    if (tk.prepared == 2) {  // ready children: the OR over the moves holds I already
#pragma unroll
      for (int w = 0; w < 8; w++) I[w] = 0;
    }
    combine(Fc, Fo, I, AW, AN, W, N, tk.prepared != 0);
  }
  store_super32(out + tk.out + L, W, N);
}

template <bool D4>
__global__ void __launch_bounds__(kBlock, PP_SEC_MINB) section_kernel(const SecTask* __restrict__ tasks, int ntasks,
                                                        pp_super* __restrict__ out) {
  section_block<D4>(tasks, ntasks, blockIdx.x, out);
}

// Persistent form: a grid sized to the device; each block claims the next
// virtual block from a counter (tasks are ordered by the host, e.g. largest
// section first), so uneven sections balance across the SMs.  No block waits
// on another.
template <bool D4>
__global__ void __launch_bounds__(kBlock, PP_SEC_MINB) section_persistent_kernel(const SecTask* __restrict__ tasks,
                                                                   int ntasks, uint32_t blocks,
                                                                   pp_super* __restrict__ out, uint32_t* counter) {
  __shared__ uint32_t next;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) next = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t vb = next;
    if (vb >= blocks) return;
    section_block<D4>(tasks, ntasks, vb, out);
  }
}

// Digest of an array of super values: acc[0] += wins, acc[1] += not-loses
// (popcounts over all rotations), acc[2] ^= an order-independent 64-bit hash
// of (index, value), acc[3] += values.
__global__ void digest_kernel(const pp_super* __restrict__ v, uint64_t n, unsigned long long* acc) {
  unsigned long long pw = 0, pn = 0, h = 0, cnt = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t W[8], N[8];
    load_super(v + i, W, N);
    unsigned long long x = i * 0x9E3779B97F4A7C15ull;
#pragma unroll
    for (int w = 0; w < 8; w++) {
      pw += __popc(W[w]);
      pn += __popc(N[w]);
      x = (x ^ W[w]) * 0xBF58476D1CE4E5B9ull;
      x = (x ^ N[w] ^ (x >> 29)) * 0x94D049BB133111EBull;
    }
    h ^= x ^ (x >> 31);
    cnt++;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    pw += __shfl_xor_sync(0xFFFFFFFFu, pw, o);
    pn += __shfl_xor_sync(0xFFFFFFFFu, pn, o);
    h ^= __shfl_xor_sync(0xFFFFFFFFu, h, o);
    cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc, pw);
    atomicAdd(acc + 1, pn);
    atomicXor(acc + 2, h);
    atomicAdd(acc + 3, cnt);
  }
}

// ---------------------------------------------------------------------------
// Line kernel for slice 35 (every board has exactly one empty cell, so every
// child is a full board of slice 36).  One warp owns one line of boards
// along the section's non-full quadrant Q (paper, "Data layout and
// distribution": an output line depends on one input line).
//   * child_transform_kernel first turns each slice-36 value into
//     X2 = ~N' | rmax(~N') and X3 = ~N' | rmax(~W') (one rmax pair per child
//     value instead of one per parent board);
//   * per line, the five-in-a-row terms of the three fixed quadrants (K)
//     are evaluated once;
//   * per board: the terms touching Q, the child's X2/X3 shifted by the
//     child's standardising turn u, and
//       win = (F_c & ~F_o) | (~T & X2),  notlose = F_c | (~T & X3).
// This equals the general rule.  On a rotation g where the parent has no five,
// the full child's value is terminal, so its not-lose bit is clear exactly
// when the mover's placement made five (the immediate win I), and
// rmax commutes with the shift.
// ---------------------------------------------------------------------------
__global__ void child_transform_kernel(const pp_super* __restrict__ in, uint64_t n, pp_super* __restrict__ out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t W[8], N[8], R1[8], R2[8];
  load_super(in + i, W, N);
#pragma unroll
  for (int w = 0; w < 8; w++) W[w] = ~W[w], N[w] = ~N[w];
  rmax(N, R1);
  rmax(W, R2);
#pragma unroll
  for (int w = 0; w < 8; w++) R1[w] |= N[w], R2[w] |= N[w];
  store_super(out + i, R1, R2);
}

// Prepared child values for the steps below slice 35: win slot ~rmax(~win),
// not-lose slot ~rmax(~notlose) (every rotation one quarter turn away wins,
// or does not lose).  A parent that ORs ~notlose and ~win of its children
// then gathers rmax(~notlose) and rmax(~win) directly.
__global__ void prepare_kernel(const pp_super* in, uint64_t n, pp_super* out) {  // may run in place
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t W[8], N[8], RW[8], RN[8];
  load_super(in + i, W, N);
#pragma unroll
  for (int w = 0; w < 8; w++) W[w] = ~W[w], N[w] = ~N[w];
  rmax(W, RW);
  rmax(N, RN);
#pragma unroll
  for (int w = 0; w < 8; w++) RW[w] = ~RW[w], RN[w] = ~RN[w];
  store_super(out + i, RW, RN);
}

template <typename T>
__device__ __forceinline__ int find_warp_owner(const T* __restrict__ d, int n, uint32_t w) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (d[mid].warp0 <= w)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}


// shift_axis with a turn count that is the same in every lane of the warp
template <int Q>
__device__ __forceinline__ void shift_uniform(uint32_t x[8], uint32_t u) {
  switch (u) {
    case 1: shift_axis<Q>(x, 1); break;
    case 2: shift_axis<Q>(x, 2); break;
    case 3: shift_axis<Q>(x, 3); break;
    default: break;
  }
}

// Words of a fixed quadrant's forms that the lines through quadrant Q read
// (eval_fives<false, Q>); the others are never touched.
template <int Q>
__host__ __device__ constexpr bool line_word_used(int q, int w) {
  if (q == Q) return false;
  const bool pair01 = (Q == 0 || Q == 1) && (q == 0 || q == 1) && w <= 2;
  const bool pair02 = (Q == 0 || Q == 2) && (q == 0 || q == 2) && w >= 3 && w <= 5;
  const bool pair03 = (Q == 0 || Q == 3) && (q == 0 || q == 3) && w == 6;
  const bool pair12 = (Q == 1 || Q == 2) && (q == 1 || q == 2) && w == 6;
  const bool pair13 = (Q == 1 || Q == 3) && (q == 1 || q == 3) && w >= 3 && w <= 5;
  const bool pair23 = (Q == 2 || Q == 3) && (q == 2 || q == 3) && w <= 2;
  // triples: T0 {0,1,3} and T1 {0,2,3} inner words 7, T2 {0,1,2} and T3
  // {1,2,3} inner words 8; gates q3 (T0, T1, T3) and q2 (T2) word 9
  const bool t0 = Q != 2 && (q == 0 || q == 1) && w == 7;
  const bool t1 = Q != 1 && (q == 0 || q == 2) && w == 7;
  const bool t2 = Q != 3 && (q == 0 || q == 1) && w == 8;
  const bool t3 = Q != 0 && (q == 2 || q == 1) && w == 8;
  const bool g3 = q == 3 && w == 9;           // every Q != 3 lies on a triple gated by q3
  const bool g2 = Q != 3 && q == 2 && w == 9;  // T2's gate, when T2 contains Q
  return pair01 || pair02 || pair03 || pair12 || pair13 || pair23 || t0 || t1 || t2 || t3 || g3 || g2;
}

// Compact index of a used word among the used words of the fixed quadrants.
template <int Q>
__host__ __device__ constexpr int line_word_slot(int q, int w) {
  int n = 0;
  for (int i = 0; i < q * kFormWords + w; i++)
    if (line_word_used<Q>(i / kFormWords, i % kFormWords)) n++;
  return n;
}
constexpr int kLineUsedWords = 12;  // the most for any Q (11 for Q = 2); checked below
static_assert(line_word_slot<0>(4, 0) <= kLineUsedWords && line_word_slot<1>(4, 0) <= kLineUsedWords &&
                  line_word_slot<2>(4, 0) <= kLineUsedWords && line_word_slot<3>(4, 0) <= kLineUsedWords,
              "the lines through one quadrant read at most 12 words of the other three quadrants' forms");

// Per-lane shared-memory record of a slice-35 line: what is read once per
// child (K terms of both colours, the opponent's fixed forms).
constexpr int kLineColdWords = 8 + 8 + kLineUsedWords;
constexpr size_t kLine35Smem = sizeof(uint4) * 3 * 512 + sizeof(uint32_t) * kLineWarps * 32 * kLineColdWords;

// One lane per line: the 32 lanes of a warp own 32 consecutive lines of one
// section and walk their positions along Q in lockstep, in the order of the
// children's ranks.  At each step every lane has the same quadrant-Q state,
// so that state's tables, the child rank j and the turn u are uniform, the
// child loads and the output stores of the warp fall on neighbouring lines,
// and each lane reloads its child value only when j changes.
//
// Work per child instead of per board: the move adds a stone of the mover
// c, so a board and its child hold the same stones of the opponent o, and
// F_o(board) is the child's F_o, evaluated once per child in the child's
// standard frame and turned with its other tables.  With A = ~F_o and the
// mover's set F_c = K_c | H_c (K_c: lines missing Q, constant along the
// line and under turns of Q; H_c: lines through Q),
//   win     = (F_c & ~F_o) | (~T & X2) = (H_c & A) | ((K_c | X2) & A),
//   notlose =  F_c | (~T & X3)         =  H_c | (K_c | (X3 & A)),
// so each child leaves three tables, A, Y2 = (K_c | X2) & A and
// Y3 = K_c | (X3 & A), and each board evaluates only H_c.
template <int Q, bool ONDEMAND>
__device__ __forceinline__ void line35_lines(const LineTask& tk, uint32_t gw, const uint4* qforms, uint32_t* cold,
                                             pp_super* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const uint32_t line = (gw - tk.warp0) * 32 + lane;
  const bool active = line < tk.lines;
  const uint32_t c = tk.mover;
  const uint2* __restrict__ moves = reinterpret_cast<const uint2*>(c_tab.qline) + (c - 1) * kMinStates;
  // this lane's cold record, word i at cold[i * blockDim + thread] (no bank conflicts)
  uint32_t* mycold = cold + threadIdx.x;
  auto cold_at = [&](int i) -> uint32_t& { return mycold[i * kLineWarps * 32]; };

  // this lane's three fixed quadrants: forms and base offsets
  uint32_t fc[4][kFormWords];
  uint64_t obase = tk.out;
  const pp_super* cb = tk.child;
  {
    uint32_t fo[4][kFormWords];
    uint32_t r = active ? line : 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      if (q == Q) {
#pragma unroll
        for (int w = 0; w < kFormWords; w++) fc[q][w] = fo[q][w] = 0;
        continue;
      }
      const uint32_t iq = r % tk.dim[q];
      r /= tk.dim[q];
      const uint32_t x = __ldg(&moves[tk.qoff[q] + iq]).x;
      const uint32_t b = x & 0x1FFu, w = (x >> 9) & 0x1FFu;
      load_forms(q, c == 1 ? b : w, fc[q]);
      load_forms(q, c == 1 ? w : b, fo[q]);
      obase += (uint64_t)iq * tk.stride[q];
      cb += (uint64_t)iq * tk.cstride[q];
    }
    uint32_t Kc[8], Ko[8];
    five_mask(fc, Kc);  // quadrant Q's forms are zero: only lines missing Q
    five_mask(fo, Ko);
#pragma unroll
    for (int i = 0; i < 8; i++) cold_at(i) = Kc[i], cold_at(8 + i) = Ko[i];
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
      for (int w = 0; w < kFormWords; w++)
        if (line_word_used<Q>(q, w)) cold_at(16 + line_word_slot<Q>(q, w)) = fo[q][w];
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
      for (int w = 0; w < kFormWords; w++)
        if (!line_word_used<Q>(q, w) && q != Q) fc[q][w] = 0;  // never read: let the registers go
  }

  const uint32_t sq = tk.stride[Q], csq = tk.cstride[Q], dq = tk.dim[Q];
  const uint4* __restrict__ sorted = reinterpret_cast<const uint4*>(c_tab.qsorted) + (c - 1) * kMinStates + tk.qoff[Q];
  // the current child's tables A, Y2, Y3, already turned ucur along Q
  uint32_t A[8], Y2[8], Y3[8], jprev = 0xFFFFFFFFu, ucur = 0;
  uint4 mnext = __ldg(sorted);
  for (uint32_t k = 0; k < dq; k++) {
    const uint4 m = mnext;  // uniform across the warp
    if (k + 1 < dq) mnext = __ldg(sorted + k + 1);
    const uint32_t j = (m.y >> 4) & 0x1FFu;
    if (j != jprev) {
      // the child: this lane's fixed quadrants and the child count class's
      // minimal state j in Q (its standard frame), pattern m.z
      const uint32_t cbm = m.z & 0x1FFu, cwm = (m.z >> 9) & 0x1FFu;
      uint32_t X2[8], X3[8], Kc[8];
      if constexpr (!ONDEMAND) load_super32(cb + (uint64_t)j * csq, X2, X3);
#pragma unroll
      for (int i = 0; i < 8; i++) Kc[i] = cold_at(i);
      {
        uint32_t fo[4][kFormWords], Go[8], unused[8];
#pragma unroll
        for (int q = 0; q < 4; q++)
#pragma unroll
          for (int w = 0; w < kFormWords; w++)
            fo[q][w] = line_word_used<Q>(q, w) ? cold_at(16 + line_word_slot<Q>(q, w)) : 0u;
        load_forms_smem(qforms, c == 1 ? cwm : cbm, fo[Q]);
        eval_fives<false, Q>(fo, fo, Go, unused);
        // the child's mover is this board's opponent o
#pragma unroll
        for (int i = 0; i < 8; i++) A[i] = ~(cold_at(8 + i) | Go[i]);
      }
      if constexpr (ONDEMAND) {
        // slice 36 on demand (paper, "Data layout and distribution": the last
        // slice is computed when needed): the child is full, and its
        // five-in-a-row sets are the line's K terms plus the lines through Q
        load_forms_smem(qforms, c == 1 ? cbm : cwm, fc[Q]);
        uint32_t Gc[8], unused[8];
        eval_fives<false, Q>(fc, fc, Gc, unused);
        uint32_t nW[8], nN[8], R1[8], R2[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
          const uint32_t Fm = ~A[i], Fp = Kc[i] | Gc[i];  // child's mover o, child's opponent c
          nW[i] = ~(Fm & ~Fp);                            // ~win'
          nN[i] = ~(Fm | ~Fp);                            // ~notlose'
        }
        rmax(nN, R1);
        rmax(nW, R2);
#pragma unroll
        for (int i = 0; i < 8; i++) X2[i] = nN[i] | R1[i], X3[i] = nN[i] | R2[i];
      }
#pragma unroll
      for (int i = 0; i < 8; i++) {
        Y2[i] = (Kc[i] | X2[i]) & A[i];
        Y3[i] = Kc[i] | (X3[i] & A[i]);
      }
      jprev = j;
      ucur = 0;
    }
    const uint32_t b = m.x & 0x1FFu, w = (m.x >> 9) & 0x1FFu;
    load_forms_smem(qforms, c == 1 ? b : w, fc[Q]);
    uint32_t Hc[8], unused[8];
    eval_fives<false, Q>(fc, fc, Hc, unused);
    // positions of one child run in increasing turn u, and turns compose:
    // turn the child's tables by the difference in place (K_c is constant
    // along Q, so turning Y2 and Y3 turns only X2, X3 and A)
    const uint32_t u = (m.y >> 13) & 3u;
    if (u != ucur) {
      shift_uniform<Q>(A, (u - ucur) & 3u);
      shift_uniform<Q>(Y2, (u - ucur) & 3u);
      shift_uniform<Q>(Y3, (u - ucur) & 3u);
      ucur = u;
    }
    uint32_t W[8], N[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
      W[i] = (Hc[i] & A[i]) | Y2[i];
      N[i] = Hc[i] | Y3[i];
    }
    // each lane stores its own value, two 256-bit stores
    if (active) {
      pp_super* dst = out + obase + (uint64_t)(m.y >> 16) * sq;
      st256(reinterpret_cast<char*>(dst), W);
      st256(reinterpret_cast<char*>(dst) + 32, N);
    }
  }
}

// All slice-35 line tasks in one launch: every block serves one line axis
// Q (the host starts a new block where Q changes), copies that quadrant's
// forms into shared memory and runs the lines of its warps.
template <bool ONDEMAND>
__global__ void __launch_bounds__(kLineWarps * 32, PP_LINE_MINB)
    line35_kernel(const LineTask* __restrict__ tasks, int ntasks, pp_super* __restrict__ out) {
  extern __shared__ uint4 line35_smem[];
  uint4* qforms = line35_smem;  // quadrant Q's forms (24 KB), read uniformly
  uint32_t* cold = reinterpret_cast<uint32_t*>(line35_smem + 3 * 512);
  const uint32_t q = tasks[find_warp_owner(tasks, ntasks, blockIdx.x * kLineWarps)].q;
  copy_forms(qforms, q * 512, 512);
  const uint32_t gw = blockIdx.x * kLineWarps + (threadIdx.x >> 5);
  const LineTask& tk = tasks[find_warp_owner(tasks, ntasks, gw)];
  if (gw - tk.warp0 >= (tk.lines + 31) / 32) return;  // uniform per warp (block padding)
  switch (q) {
    case 0: line35_lines<0, ONDEMAND>(tk, gw, qforms, cold, out); break;
    case 1: line35_lines<1, ONDEMAND>(tk, gw, qforms, cold, out); break;
    case 2: line35_lines<2, ONDEMAND>(tk, gw, qforms, cold, out); break;
    default: line35_lines<3, ONDEMAND>(tk, gw, qforms, cold, out); break;
  }
}

// ---------------------------------------------------------------------------
// Slice 36 by lines (paper, "Data layout and distribution": the full boards'
// values follow from five in a row alone; "Problem definition": a board
// where both colours have five, or neither, is a tie).  Every quadrant is
// full, so a board's value is the terminal rule over its two colours'
// five-in-a-row sets, win = F_c & ~F_o and notlose = F_c | ~F_o.  One lane
// per line along Q, the 32 lanes of a warp on 32 consecutive lines walking
// Q's states in layout order: each colour's lines that miss Q (K_c, K_o)
// are evaluated once per line, each step evaluates only the lines through
// Q, whose forms are the same in every lane.
// ---------------------------------------------------------------------------
template <int Q>
__device__ __forceinline__ void line36_lines(const LineTask& tk, uint32_t gw, const uint4* qforms,
                                             pp_super* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const uint32_t line = (gw - tk.warp0) * 32 + lane;
  const bool active = line < tk.lines;
  const uint32_t c = tk.mover;
  const uint2* __restrict__ states = reinterpret_cast<const uint2*>(c_tab.qline) + (c - 1) * kMinStates;
  uint32_t fc[4][kFormWords], fo[4][kFormWords], Kc[8], Ko[8];
  uint64_t obase = tk.out;
  {
    uint32_t r = active ? line : 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      if (q == Q) {
#pragma unroll
        for (int w = 0; w < kFormWords; w++) fc[q][w] = fo[q][w] = 0;
        continue;
      }
      const uint32_t iq = r % tk.dim[q];
      r /= tk.dim[q];
      const uint32_t x = __ldg(&states[tk.qoff[q] + iq]).x;
      const uint32_t b = x & 0x1FFu, w = (x >> 9) & 0x1FFu;
      load_forms(q, c == 1 ? b : w, fc[q]);
      load_forms(q, c == 1 ? w : b, fo[q]);
      obase += (uint64_t)iq * tk.stride[q];
    }
    five_mask(fc, Kc);  // quadrant Q's forms are zero: only lines missing Q
    five_mask(fo, Ko);
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
      for (int w = 0; w < kFormWords; w++)
        if (q != Q && !line_word_used<Q>(q, w)) fc[q][w] = fo[q][w] = 0;  // never read again
  }
  const uint32_t sq = tk.stride[Q], dq = tk.dim[Q];
  for (uint32_t p = 0; p < dq; p++) {
    const uint32_t x = __ldg(&states[tk.qoff[Q] + p]).x;  // uniform across the warp
    const uint32_t b = x & 0x1FFu, w = (x >> 9) & 0x1FFu;
    uint32_t Fc[8], Fo[8], H[8], unused[8];
    load_forms_smem(qforms, c == 1 ? b : w, fc[Q]);
    eval_fives<false, Q>(fc, fc, H, unused);
#pragma unroll
    for (int i = 0; i < 8; i++) Fc[i] = Kc[i] | H[i];
    load_forms_smem(qforms, c == 1 ? w : b, fo[Q]);
    eval_fives<false, Q>(fo, fo, H, unused);
#pragma unroll
    for (int i = 0; i < 8; i++) Fo[i] = Ko[i] | H[i];
    uint32_t W[8], N[8];
#pragma unroll
    for (int i = 0; i < 8; i++) W[i] = Fc[i] & ~Fo[i], N[i] = Fc[i] | ~Fo[i];
    if (active) {
      pp_super* dst = out + obase + (uint64_t)p * sq;
      st256(reinterpret_cast<char*>(dst), W);
      st256(reinterpret_cast<char*>(dst) + 32, N);
    }
  }
}

// All slice-36 line tasks in one launch; a block serves one line axis Q.
__global__ void __launch_bounds__(kLineWarps * 32, PP_LINE_MINB)
    line36_kernel(const LineTask* __restrict__ tasks, int ntasks, pp_super* __restrict__ out) {
  __shared__ uint4 qforms[3 * 512];  // quadrant Q's forms (24 KB), read uniformly
  const uint32_t q = tasks[find_warp_owner(tasks, ntasks, blockIdx.x * kLineWarps)].q;
  copy_forms(qforms, q * 512, 512);
  const uint32_t gw = blockIdx.x * kLineWarps + (threadIdx.x >> 5);
  const LineTask& tk = tasks[find_warp_owner(tasks, ntasks, gw)];
  if (gw - tk.warp0 >= (tk.lines + 31) / 32) return;  // uniform per warp (block padding)
  switch (q) {
    case 0: line36_lines<0>(tk, gw, qforms, out); break;
    case 1: line36_lines<1>(tk, gw, qforms, out); break;
    case 2: line36_lines<2>(tk, gw, qforms, out); break;
    default: line36_lines<3>(tk, gw, qforms, out); break;
  }
}

// ---------------------------------------------------------------------------
// Ready child records (paper, "Abstracting over rotations": rmax distributes
// over OR and commutes with turns and board symmetries; "Problem
// definition": a move that makes five wins at once).  A parent's
// immediate-win mask is the OR over its moves of the child's five-in-a-row
// set F_c of the parent's mover c, turned as the child value is.  So each
// value (W, N) of slice n+1 is stored as (~(F_c | rmax(~W)), ~(F_c |
// rmax(~N))): a parent's fold of its children then yields I | rmax(...) and
// it evaluates no line with one more stone.  One lane per line along the
// section's quadrant with the most states, as for slice 36: F_c's lines
// missing that quadrant once per line, the lines through it per step.
// Sections are laid out at the offsets the tasks give (child: first input
// value, out: first output value); in place is allowed.
// ---------------------------------------------------------------------------
template <int Q>
__device__ __forceinline__ void ready_lines(const LineTask& tk, uint32_t gw, const uint4* qforms,
                                            pp_super* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const uint32_t line = (gw - tk.warp0) * 32 + lane;
  const bool active = line < tk.lines;
  const uint32_t c = tk.mover;  // the parents' mover
  const uint2* __restrict__ states = reinterpret_cast<const uint2*>(c_tab.qline) + (c - 1) * kMinStates;
  uint32_t fc[4][kFormWords], K[8];
  uint64_t base = 0;
  {
    uint32_t r = active ? line : 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      if (q == Q) {
#pragma unroll
        for (int w = 0; w < kFormWords; w++) fc[q][w] = 0;
        continue;
      }
      const uint32_t iq = r % tk.dim[q];
      r /= tk.dim[q];
      const uint32_t x = __ldg(&states[tk.qoff[q] + iq]).x;
      load_forms(q, c == 1 ? (x & 0x1FFu) : ((x >> 9) & 0x1FFu), fc[q]);
      base += (uint64_t)iq * tk.stride[q];
    }
    five_mask(fc, K);  // quadrant Q's forms are zero: only lines missing Q
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
      for (int w = 0; w < kFormWords; w++)
        if (q != Q && !line_word_used<Q>(q, w)) fc[q][w] = 0;  // never read again
  }
  const uint32_t sq = tk.stride[Q], dq = tk.dim[Q];
  const pp_super* in = tk.child + base;
  pp_super* dst = out + tk.out + base;
  for (uint32_t p = 0; p < dq; p++) {
    const uint32_t x = __ldg(&states[tk.qoff[Q] + p]).x;  // uniform across the warp
    uint32_t H[8], unused[8], W[8], N[8], RW[8], RN[8];
    if (active) load_super32(in + (uint64_t)p * sq, W, N);
    load_forms_smem(qforms, c == 1 ? (x & 0x1FFu) : ((x >> 9) & 0x1FFu), fc[Q]);
    eval_fives<false, Q>(fc, fc, H, unused);
    if (!active) continue;
#pragma unroll
    for (int w = 0; w < 8; w++) W[w] = ~W[w], N[w] = ~N[w];
    rmax(W, RW);
    rmax(N, RN);
#pragma unroll
    for (int w = 0; w < 8; w++) {
      const uint32_t F = K[w] | H[w];
      W[w] = ~(F | RW[w]);
      N[w] = ~(F | RN[w]);
    }
    store_super32(dst + (uint64_t)p * sq, W, N);
  }
}

__global__ void __launch_bounds__(kLineWarps * 32, PP_LINE_MINB)
    ready_kernel(const LineTask* __restrict__ tasks, int ntasks, pp_super* __restrict__ out) {
  __shared__ uint4 qforms[3 * 512];  // quadrant Q's forms (24 KB), read uniformly
  const uint32_t q = tasks[find_warp_owner(tasks, ntasks, blockIdx.x * kLineWarps)].q;
  copy_forms(qforms, q * 512, 512);
  const uint32_t gw = blockIdx.x * kLineWarps + (threadIdx.x >> 5);
  const LineTask& tk = tasks[find_warp_owner(tasks, ntasks, gw)];
  if (gw - tk.warp0 >= (tk.lines + 31) / 32) return;  // uniform per warp (block padding)
  switch (q) {
    case 0: ready_lines<0>(tk, gw, qforms, out); break;
    case 1: ready_lines<1>(tk, gw, qforms, out); break;
    case 2: ready_lines<2>(tk, gw, qforms, out); break;
    default: ready_lines<3>(tk, gw, qforms, out); break;
  }
}

// ---------------------------------------------------------------------------
// Section lines (slices below 35): one lane per line along a non-full
// quadrant Q, the 32 lanes of a warp on 32 consecutive lines, all walking
// Q's states in order.  Q's pattern is then the same in every lane, so its
// forms, its moves' child ranks and turns are uniform.  The five-in-a-row and
// immediate-win terms of the lines that miss Q are computed once per line
// (K); each step evaluates only the lines through Q.
// ---------------------------------------------------------------------------
// Which fixed quadrants can take a move, known at compile time: RM = -1
// none, 0..3 exactly that one, 4 any (read from the task).
template <int RM>
__device__ __forceinline__ bool fixed_movable(const SecLineTask& tk, int q) {
  if constexpr (RM == 4)
    return tk.movable >> q & 1;
  else
    return q == RM;
}

// Moves in quadrant R != Q at step p of a section line: the child is on
// the line along Q of section S+R at this lane's child state of R.
template <int Q, int RM, int R>
__device__ __forceinline__ void line_moves(const SecLineTask& tk, const uint32_t code[4], const uint64_t rbase[4],
                                           uint32_t p, uint32_t c, uint32_t AW[8], uint32_t AN[8]) {
  if constexpr (R != Q && (RM == 4 || RM == R)) {
    if (!fixed_movable<RM>(tk, R)) return;
    const uint32_t dec = __ldg(c_tab.qdecode + code[R]);
    const pp_super* cb = tk.child[R] + rbase[R] + (uint64_t)p * tk.cstride[R][Q];
    for (uint32_t em = ~(dec | dec >> 9) & 0x1FFu; em; em &= em - 1) {
      const uint32_t st = __ldg(c_tab.standard + code[R] + c * c_pow3[__ffs(em) - 1]);
      uint32_t cW[8], cN[8];
      load_super32(cb + (uint64_t)(st & 0xFFFFu) * tk.cstride[R][R], cW, cN);
      shift_axis<R>(cW, st >> 16);
      shift_axis<R>(cN, st >> 16);
#pragma unroll
      for (int w = 0; w < 8; w++) AW[w] |= ~cN[w], AN[w] |= ~cW[w];
    }
  }
}

// Per-lane shared-memory record of a section line: the fixed quadrants'
// form words the lines through Q read (mover, mover's one-more-stone,
// opponent) and the three K terms, reloaded every step instead of held in
// registers.
constexpr int kSecLineColdWords = 3 * kLineUsedWords + 24;  // + the K terms (Kc, Ki, Ko)
constexpr size_t kSecLineSmem = sizeof(uint32_t) * kSecLineWarps * 32 * kSecLineColdWords;

// READY: the children are ready records (pp_prepare_children_ready), which
// carry each child's five-in-a-row set of this slice's mover: the OR over
// the moves already holds the immediate-win mask, so no line is evaluated
// with one more stone.
template <int Q, int RM, bool READY>
__global__ void __launch_bounds__(kSecLineWarps * 32, READY ? PP_SLINE_READY_MINB : PP_SLINE_MINB)
    section_line_kernel(const SecLineTask* __restrict__ tasks, int ntasks, pp_super* __restrict__ out) {
  extern __shared__ uint32_t sline_cold[];
  uint32_t* mycold = sline_cold + threadIdx.x;  // word i at mycold[i * blockDim]
  auto cold_at = [&](int i) -> uint32_t& { return mycold[i * kSecLineWarps * 32]; };
  const int lane = threadIdx.x & 31;
  const uint32_t gw = blockIdx.x * kSecLineWarps + (threadIdx.x >> 5);
  const SecLineTask& tk = tasks[find_warp_owner(tasks, ntasks, gw)];
  if (gw - tk.warp0 >= (tk.lines + 31) / 32) return;  // uniform per warp
  const uint32_t line = (gw - tk.warp0) * 32 + lane;
  const bool active = line < tk.lines;
  const uint32_t c = tk.mover;

  // this lane's three fixed quadrants
  uint32_t idx[4] = {0, 0, 0, 0}, code[4] = {0, 0, 0, 0}, pc[4] = {0, 0, 0, 0};
  uint32_t fc[4][kFormWords], fo[4][kFormWords], fi[4][kFormWords];
  uint64_t obase = tk.out;
  uint32_t r = active ? line : 0;
#pragma unroll
  for (int q = 0; q < 4; q++) {
#pragma unroll
    for (int w = 0; w < kFormWords; w++) fc[q][w] = fo[q][w] = fi[q][w] = 0;
    if (q == Q) continue;
    idx[q] = r % tk.dim[q];
    r /= tk.dim[q];
    code[q] = __ldg(c_tab.qlist + tk.qoff[q] + idx[q]);
    const uint32_t dec = __ldg(c_tab.qdecode + code[q]);
    const uint32_t b = dec & 0x1FFu, w = (dec >> 9) & 0x1FFu;
    pc[q] = c == 1 ? b : w;
    load_forms(q, pc[q], fc[q]);
    load_forms(q, c == 1 ? w : b, fo[q]);
    if (!READY && fixed_movable<RM>(tk, q)) {
      for (uint32_t em = ~(b | w) & 0x1FFu; em; em &= em - 1) {
        uint32_t g[kFormWords];
        load_forms(q, pc[q] | 1u << (__ffs(em) - 1), g);
#pragma unroll
        for (int x = 0; x < kFormWords; x++) fi[q][x] |= g[x];
      }
    }
    obase += (uint64_t)idx[q] * tk.stride[q];
  }
  uint32_t Kc[8], Ki[8] = {0, 0, 0, 0, 0, 0, 0, 0}, Ko[8];
  if (READY)
    five_mask(fc, Kc);
  else
    eval_all_fives<true>(fc, fi, Kc, Ki);  // quadrant Q's forms are zero: the lines missing Q
  five_mask(fo, Ko);
  // park the form words the steps read; the registers are then free
#pragma unroll
  for (int q = 0; q < 4; q++)
#pragma unroll
    for (int w = 0; w < kFormWords; w++)
      if (line_word_used<Q>(q, w)) {
        const int k = line_word_slot<Q>(q, w);
        cold_at(k) = fc[q][w];
        if (!READY) cold_at(kLineUsedWords + k) = fi[q][w];
        cold_at(2 * kLineUsedWords + k) = fo[q][w];
      }
#pragma unroll
  for (int i = 0; i < 8; i++) {
    cold_at(3 * kLineUsedWords + i) = Kc[i];
    if (!READY) cold_at(3 * kLineUsedWords + 8 + i) = Ki[i];
    cold_at(3 * kLineUsedWords + 16 + i) = Ko[i];
  }

  // child bases: moves in Q (everything but Q's index), moves in R (everything
  // but R's and Q's index; Q's index is added per step)
  uint64_t qbase = 0, rbase[4] = {0, 0, 0, 0};
#pragma unroll
  for (int q = 0; q < 4; q++) {
    if (q == Q) continue;
    qbase += (uint64_t)idx[q] * tk.cstride[Q][q];
#pragma unroll
    for (int R = 0; R < 4; R++)
      if (R != Q && R != q && (RM == 4 || RM == R)) rbase[R] += (uint64_t)idx[q] * tk.cstride[R][q];
  }

  const uint32_t dq = tk.dim[Q];
  for (uint32_t p = 0; p < dq; p++) {
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
      for (int w = 0; w < kFormWords; w++) {
        const bool used = line_word_used<Q>(q, w);
        const int k = used ? line_word_slot<Q>(q, w) : 0;
        fc[q][w] = used ? cold_at(k) : 0u;
        fi[q][w] = used && !READY ? cold_at(kLineUsedWords + k) : 0u;
        fo[q][w] = used ? cold_at(2 * kLineUsedWords + k) : 0u;
      }
    const uint32_t cq = __ldg(c_tab.qlist + tk.qoff[Q] + p);  // uniform across the warp
    const uint32_t dq_ = __ldg(c_tab.qdecode + cq);
    const uint32_t bq = dq_ & 0x1FFu, wq = (dq_ >> 9) & 0x1FFu, pcq = c == 1 ? bq : wq;
    const uint32_t eq = ~(bq | wq) & 0x1FFu;
    load_forms(Q, pcq, fc[Q]);
    load_forms(Q, c == 1 ? wq : bq, fo[Q]);
#pragma unroll
    for (int x = 0; x < kFormWords; x++) fi[Q][x] = 0;
    uint32_t Hc[8], Hi[8] = {0, 0, 0, 0, 0, 0, 0, 0}, Ho[8], unused[8];
    if (READY) {
      eval_fives<false, Q>(fc, fc, Hc, unused);
    } else {
      for (uint32_t em = eq; em; em &= em - 1) {
        uint32_t g[kFormWords];
        load_forms(Q, pcq | 1u << (__ffs(em) - 1), g);
#pragma unroll
        for (int x = 0; x < kFormWords; x++) fi[Q][x] |= g[x];
      }
      eval_fives<true, Q>(fc, fi, Hc, Hi);
    }
    eval_fives<false, Q>(fo, fo, Ho, unused);
    uint32_t AW[8] = {0, 0, 0, 0, 0, 0, 0, 0}, AN[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // moves in Q: child rank and turn uniform
    for (uint32_t em = eq; em; em &= em - 1) {
      const uint32_t st = __ldg(c_tab.standard + cq + c * c_pow3[__ffs(em) - 1]);
      uint32_t cW[8], cN[8];
      load_super32(tk.child[Q] + qbase + (uint64_t)(st & 0xFFFFu) * tk.cstride[Q][Q], cW, cN);
      shift_uniform<Q>(cW, st >> 16);
      shift_uniform<Q>(cN, st >> 16);
#pragma unroll
      for (int w = 0; w < 8; w++) AW[w] |= ~cN[w], AN[w] |= ~cW[w];
    }
    // moves in the other non-full quadrants: this lane's child states
    line_moves<Q, RM, 0>(tk, code, rbase, p, c, AW, AN);
    line_moves<Q, RM, 1>(tk, code, rbase, p, c, AW, AN);
    line_moves<Q, RM, 2>(tk, code, rbase, p, c, AW, AN);
    line_moves<Q, RM, 3>(tk, code, rbase, p, c, AW, AN);
    uint32_t Fc[8], Fo[8], I[8], W[8], N[8];
#pragma unroll
    for (int w = 0; w < 8; w++) {
      Fc[w] = cold_at(3 * kLineUsedWords + w) | Hc[w];
      I[w] = READY ? 0u : cold_at(3 * kLineUsedWords + 8 + w) | Hi[w];
      Fo[w] = cold_at(3 * kLineUsedWords + 16 + w) | Ho[w];
    }
    combine(Fc, Fo, I, AW, AN, W, N, tk.prepared != 0);
    if (active) store_super32(out + obase + (uint64_t)p * tk.stride[Q], W, N);
  }
}

// ---------------------------------------------------------------------------
// Building blocks exposed for unit tests.
// ---------------------------------------------------------------------------
__global__ void five_masks_kernel(const uint64_t* boards, int n, uint64_t* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t b = boards[i];
  uint32_t fb[4][kFormWords], fw[4][kFormWords];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const uint32_t dec = __ldg(c_tab.qdecode + ((b >> (16 * q)) & 0xFFFFu));
    load_forms(q, dec & 0x1FFu, fb[q]);
    load_forms(q, (dec >> 9) & 0x1FFu, fw[q]);
  }
  uint32_t Fb[8], Fw[8];
  five_mask(fb, Fb);
  five_mask(fw, Fw);
  store_super(reinterpret_cast<pp_super*>(out + 8 * (size_t)i), Fb, Fw);
}

__global__ void rmax_kernel(const pp_super* in, int n, pp_super* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t W[8], N[8], RW[8], RN[8];
  load_super(in + i, W, N);
  rmax(W, RW);
  rmax(N, RN);
  store_super(out + i, RW, RN);
}

__global__ void shift_kernel(const pp_super* in, int n, int q, int u, pp_super* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t W[8], N[8];
  load_super(in + i, W, N);
  switch (q) {
    case 0: shift_axis<0>(W, u), shift_axis<0>(N, u); break;
    case 1: shift_axis<1>(W, u), shift_axis<1>(N, u); break;
    case 2: shift_axis<2>(W, u), shift_axis<2>(N, u); break;
    default: shift_axis<3>(W, u), shift_axis<3>(N, u); break;
  }
  store_super(out + i, W, N);
}

// out(g) = in(phi_S(g) + t) for both tables: the stored value of a board
// read for its preimage under symmetry S (t: the turns of the stored board's
// quadrants past their minimal patterns, in the stored board's frame).
template <int S>
__device__ __forceinline__ void symmetry_apply(uint32_t W[8], uint32_t N[8], const uint32_t t[4]) {
  shift_axis<0>(W, t[0]), shift_axis<0>(N, t[0]);
  shift_axis<1>(W, t[1]), shift_axis<1>(N, t[1]);
  shift_axis<2>(W, t[2]), shift_axis<2>(N, t[2]);
  shift_axis<3>(W, t[3]), shift_axis<3>(N, t[3]);
  reorient<S>(W);
  reorient<S>(N);
}

__global__ void symmetry_kernel(const pp_super* in, int n, int sym, uint32_t turns, pp_super* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t W[8], N[8];
  const uint32_t t[4] = {turns & 3u, turns >> 2 & 3u, turns >> 4 & 3u, turns >> 6 & 3u};
  load_super(in + i, W, N);
  switch (sym) {
    case 0: symmetry_apply<0>(W, N, t); break;
    case 1: symmetry_apply<1>(W, N, t); break;
    case 2: symmetry_apply<2>(W, N, t); break;
    case 3: symmetry_apply<3>(W, N, t); break;
    case 4: symmetry_apply<4>(W, N, t); break;
    case 5: symmetry_apply<5>(W, N, t); break;
    case 6: symmetry_apply<6>(W, N, t); break;
    default: symmetry_apply<7>(W, N, t); break;
  }
  store_super(out + i, W, N);
}

// One board of a non-minimal child section from its stored least image S
// (paper, "Data layout and distribution" and Fig. "lines": input lines are
// turned before use): quadrant q's state maps through the symmetry table to
// a rank and turn at position sym_qmap(S, q) of the stored section, and the
// value is read as out(g) = in(phi_S(g) + t).
template <int S>
__device__ __forceinline__ void materialise_one(const MatTask& tk, uint64_t L, pp_super* out) {
  const uint16_t* __restrict__ dm = c_tab.dmin + S * kMinStates;
  uint64_t src = 0, r = L;
  uint32_t t[4];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const uint32_t i = (uint32_t)(r % tk.dim[q]);
    r /= tk.dim[q];
    const uint32_t v = __ldg(dm + tk.qoff[q] + i);
    src += (uint64_t)(v & 0xFFFu) * tk.sstride[sym_qmap(S, q)];
    t[sym_qmap(S, q)] = v >> 12;
  }
  uint32_t W[8], N[8];
  load_super32(tk.src + src, W, N);
  symmetry_apply<S>(W, N, t);
  store_super32(out + tk.dst + L, W, N);
}

__global__ void materialise_kernel(const MatTask* __restrict__ tasks, int ntasks, pp_super* __restrict__ out) {
  const MatTask& tk = tasks[find_block_owner(tasks, ntasks, blockIdx.x)];
  const uint64_t L = (uint64_t)(blockIdx.x - tk.block0) * kBlock + threadIdx.x;
  if (L >= tk.size) return;
  switch (tk.sym) {  // uniform per block
    case 1: materialise_one<1>(tk, L, out); break;
    case 2: materialise_one<2>(tk, L, out); break;
    case 3: materialise_one<3>(tk, L, out); break;
    case 4: materialise_one<4>(tk, L, out); break;
    case 5: materialise_one<5>(tk, L, out); break;
    case 6: materialise_one<6>(tk, L, out); break;
    case 7: materialise_one<7>(tk, L, out); break;
    default: materialise_one<0>(tk, L, out); break;
  }
}


// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
static unsigned blocks_for(uint64_t threads, int per) { return (unsigned)((threads + per - 1) / per); }

int upload_tables(const HostTables& t, DeviceTables* dt, std::string* err) {
  DeviceTables h{};
  void *qd = nullptr, *st = nullptr, *ql = nullptr, *fm = nullptr, *qm = nullptr;
  cudaError_t e = cudaMalloc(&qd, sizeof(t.qdecode));
  void* qs = nullptr;
  if (!e) e = cudaMalloc(&qm, sizeof(t.qline));
  if (!e) e = cudaMemcpy(qm, t.qline, sizeof(t.qline), cudaMemcpyHostToDevice);
  if (!e) e = cudaMalloc(&qs, sizeof(t.qsorted));
  if (!e) e = cudaMemcpy(qs, t.qsorted, sizeof(t.qsorted), cudaMemcpyHostToDevice);
  if (!e) e = cudaMalloc(&st, sizeof(t.standard));
  if (!e) e = cudaMalloc(&ql, sizeof(t.qlist));
  if (!e) e = cudaMalloc(&fm, sizeof(t.forms));
  void *dmn = nullptr, *sub = nullptr;
  if (!e) e = cudaMalloc(&sub, sizeof(t.subsets));
  if (!e) e = cudaMemcpy(sub, t.subsets, sizeof(t.subsets), cudaMemcpyHostToDevice);
  if (!e) e = cudaMalloc(&dmn, sizeof(t.dmin));
  if (!e) e = cudaMemcpy(dmn, t.dmin, sizeof(t.dmin), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(qd, t.qdecode, sizeof(t.qdecode), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(st, t.standard, sizeof(t.standard), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(ql, t.qlist, sizeof(t.qlist), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(fm, t.forms, sizeof(t.forms), cudaMemcpyHostToDevice);
  if (e) {
    if (err) *err = std::string("table upload: ") + cudaGetErrorString(e);
    return (int)e;
  }
  h.qdecode = (const uint32_t*)qd;
  h.standard = (const uint32_t*)st;
  h.qlist = (const uint16_t*)ql;
  h.forms = (const uint32_t*)fm;
  h.qline = (const uint32_t*)qm;
  h.qsorted = (const uint32_t*)qs;
  h.dmin = (const uint16_t*)dmn;
  h.subsets = (const uint16_t*)sub;
  for (int b = 0; b < 10; b++)
    for (int w = 0; w < 10; w++) h.qoff[b][w] = t.qoff[b][w], h.qdim[b][w] = t.qdim[b][w];
  e = cudaMemcpyToSymbol(c_tab, &h, sizeof(h));
  if (e && err) *err = std::string("table symbol: ") + cudaGetErrorString(e);
  *dt = h;
  return (int)e;
}


int launch_midgame_level(const MidBoard* d_boards, const MidSeg* d_segs, int nsegs, uint32_t blocks,
                         pp_super* d_table, pp_super* d_out, int final_level, pp_stream s, const void* d_masks,
                         uint32_t seg_blocks, int parity) {
  if (!blocks) return 0;
  if (!d_masks) return (int)cudaErrorInvalidValue;
  const uint4* m = (const uint4*)d_masks;
  if (parity >= 0)
    midgame_level_kernel<true><<<blocks, kBlock, 0, s>>>(d_boards, d_segs, nsegs, d_table, d_out, final_level, m,
                                                         seg_blocks, (uint32_t)parity);
  else
    midgame_level_kernel<false><<<blocks, kBlock, 0, s>>>(d_boards, d_segs, nsegs, d_table, d_out, final_level, m,
                                                          seg_blocks, 0u);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_five_tables(const MidBoard* d_boards, int n, int kmax, void* d_masks, pp_stream s) {
  if (n <= 0) return 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t want = ((uint64_t)n << (kmax + 1)) / 256 + 1;
  const unsigned grid = (unsigned)(want < (uint64_t)sms * 16 ? want : (uint64_t)sms * 16);
  five_table_kernel<<<grid, 256, 0, s>>>(d_boards, n, kmax, (uint4*)d_masks, BoardsInOrder{});
  count_launch();
  return (int)cudaGetLastError();
}

int launch_five_tables_slots(const MidBoard* d_boards, const uint16_t* slots, int n, int kmax, void* d_masks,
                             pp_stream s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int at = 0; at < n; at += kSlotBatch) {
    const int m = n - at < kSlotBatch ? n - at : kSlotBatch;
    BoardSlots which;
    std::memset(&which, 0, sizeof which);
    std::memcpy(which.slot, slots + at, m * sizeof(uint16_t));
    const uint64_t want = ((uint64_t)m << (kmax + 1)) / 256 + 1;
    const unsigned grid = (unsigned)(want < (uint64_t)sms * 16 ? want : (uint64_t)sms * 16);
    five_table_kernel<<<grid, 256, 0, s>>>(d_boards, m, kmax, (uint4*)d_masks, which);
    count_launch();
    const cudaError_t e = cudaGetLastError();
    if (e) return (int)e;
  }
  return 0;
}

int persistent_midgame_blocks(int ctas_per_sm, bool half) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) return 0;
  cudaError_t e = half ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, midgame_persistent_kernel<true>, kBlock, 0)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, midgame_persistent_kernel<false>, kBlock, 0);
  if (e) return 0;
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  return sms * per_sm;
}

int launch_midgame_persistent(const MidBoard* d_boards, const MidSeg* d_segs, const MidLevel* d_levels, int nlevels,
                              pp_super* d_table, pp_super* d_out, uint32_t* d_sync, int grid, pp_stream s,
                              const void* d_masks, int parity) {
  if (grid <= 0 || nlevels <= 0 || !d_masks) return (int)cudaErrorInvalidValue;
  uint32_t* bar = d_sync;
  uint32_t* status = d_sync + 2;
  const uint4* masks = (const uint4*)d_masks;
  uint32_t p = parity >= 0 ? (uint32_t)parity : 0u;
  uint32_t spins = g_barrier_spins.load();
  void* args[] = {(void*)&d_boards, (void*)&d_segs, (void*)&d_levels, (void*)&nlevels, (void*)&d_table,
                  (void*)&d_out,    (void*)&bar,    (void*)&status,   (void*)&masks,   (void*)&p,
                  (void*)&spins};
  const void* fn = parity >= 0 ? (const void*)midgame_persistent_kernel<true> : (const void*)midgame_persistent_kernel<false>;
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBlock), args, 0, s);
  count_launch();
  return (int)e;
}

int launch_barrier_probe(uint32_t* d_sync, uint32_t limit, pp_stream s) {
  void* args[] = {(void*)&d_sync, (void*)&limit};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)barrier_probe_kernel, dim3(2), dim3(32), args, 0, s);
  count_launch();
  return (int)e;
}

int persistent_section_blocks(int ctas_per_sm, bool d4) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) return 0;
  cudaError_t e = d4 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, section_persistent_kernel<true>, kBlock, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, section_persistent_kernel<false>, kBlock, 0);
  if (e) return 0;
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  return sms * per_sm;
}

int launch_sections_persistent(const SecTask* d_tasks, int ntasks, uint32_t blocks, pp_super* d_out,
                               uint32_t* d_counter, int grid, pp_stream s, bool d4) {
  if (!blocks) return 0;
  cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(uint32_t), s);
  if (e) return (int)e;
  if (d4)
    section_persistent_kernel<true><<<grid, kBlock, 0, s>>>(d_tasks, ntasks, blocks, d_out, d_counter);
  else
    section_persistent_kernel<false><<<grid, kBlock, 0, s>>>(d_tasks, ntasks, blocks, d_out, d_counter);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_digest(const pp_super* d_values, uint64_t n, uint64_t* d_acc, pp_stream s) {
  if (!n) return 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t want = (n + 255) / 256;
  const unsigned grid = (unsigned)(want < (uint64_t)sms * 8 ? want : (uint64_t)sms * 8);
  digest_kernel<<<grid, 256, 0, s>>>(d_values, n, (unsigned long long*)d_acc);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_sections(const SecTask* d_tasks, int ntasks, uint32_t blocks, pp_super* d_out, pp_stream s, bool d4) {
  if (!blocks) return 0;
  if (d4)
    section_kernel<true><<<blocks, kBlock, 0, s>>>(d_tasks, ntasks, d_out);
  else
    section_kernel<false><<<blocks, kBlock, 0, s>>>(d_tasks, ntasks, d_out);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_prepare(const pp_super* d_in, uint64_t n, pp_super* d_out, pp_stream s) {
  if (!n) return 0;
  prepare_kernel<<<blocks_for(n, 256), 256, 0, s>>>(d_in, n, d_out);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_child_transform(const pp_super* d_in, uint64_t n, pp_super* d_out, pp_stream s) {
  if (!n) return 0;
  child_transform_kernel<<<blocks_for(n, 256), 256, 0, s>>>(d_in, n, d_out);
  count_launch();
  return (int)cudaGetLastError();
}

template <bool OD>
static cudaError_t launch_line35_od(unsigned blocks, const LineTask* d_tasks, int ntasks, pp_super* d_out,
                                   pp_stream s) {
  // more than the 48 KB of static shared memory: opt in once per instance
  static const cudaError_t attr =
      cudaFuncSetAttribute(line35_kernel<OD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLine35Smem);
  if (attr) return attr;
  line35_kernel<OD><<<blocks, kLineWarps * 32, kLine35Smem, s>>>(d_tasks, ntasks, d_out);
  return cudaSuccess;
}

int launch_ready(const LineTask* d_tasks, int ntasks, uint32_t warps, pp_super* d_out, pp_stream s) {
  if (!warps || !ntasks) return 0;
  const unsigned blocks = (warps + kLineWarps - 1) / kLineWarps;
  ready_kernel<<<blocks, kLineWarps * 32, 0, s>>>(d_tasks, ntasks, d_out);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_line36(const LineTask* d_tasks, int ntasks, uint32_t warps, pp_super* d_out, pp_stream s) {
  if (!warps || !ntasks) return 0;
  const unsigned blocks = (warps + kLineWarps - 1) / kLineWarps;
  line36_kernel<<<blocks, kLineWarps * 32, 0, s>>>(d_tasks, ntasks, d_out);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_line35(const LineTask* d_tasks, int ntasks, uint32_t warps, pp_super* d_out, pp_stream s,
                  bool on_demand) {
  if (!warps || !ntasks) return 0;
  const unsigned blocks = (warps + kLineWarps - 1) / kLineWarps;
  const cudaError_t e = on_demand ? launch_line35_od<true>(blocks, d_tasks, ntasks, d_out, s)
                                  : launch_line35_od<false>(blocks, d_tasks, ntasks, d_out, s);
  if (e) return (int)e;
  count_launch();
  return (int)cudaGetLastError();
}

template <int Q, int RM, bool READY>
static cudaError_t launch_lines_qrr(unsigned blocks, const SecLineTask* d_tasks, int ntasks, pp_super* d_out,
                                    pp_stream s) {
  // more than the 48 KB of static shared memory: opt in once per instance
  static const cudaError_t attr = cudaFuncSetAttribute(
      section_line_kernel<Q, RM, READY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSecLineSmem);
  if (attr) return attr;
  section_line_kernel<Q, RM, READY><<<blocks, kSecLineWarps * 32, kSecLineSmem, s>>>(d_tasks, ntasks, d_out);
  return cudaSuccess;
}

template <int Q, int RM>
static cudaError_t launch_lines_qr(bool ready, unsigned blocks, const SecLineTask* d_tasks, int ntasks,
                                   pp_super* d_out, pp_stream s) {
  return ready ? launch_lines_qrr<Q, RM, true>(blocks, d_tasks, ntasks, d_out, s)
               : launch_lines_qrr<Q, RM, false>(blocks, d_tasks, ntasks, d_out, s);
}

template <int Q>
static cudaError_t launch_lines_q(int rm, bool ready, unsigned blocks, const SecLineTask* d_tasks, int ntasks,
                                  pp_super* d_out, pp_stream s) {
  switch (rm) {
    case -1: return launch_lines_qr<Q, -1>(ready, blocks, d_tasks, ntasks, d_out, s);
    case 0: if constexpr (Q != 0) return launch_lines_qr<Q, 0>(ready, blocks, d_tasks, ntasks, d_out, s); break;
    case 1: if constexpr (Q != 1) return launch_lines_qr<Q, 1>(ready, blocks, d_tasks, ntasks, d_out, s); break;
    case 2: if constexpr (Q != 2) return launch_lines_qr<Q, 2>(ready, blocks, d_tasks, ntasks, d_out, s); break;
    case 3: if constexpr (Q != 3) return launch_lines_qr<Q, 3>(ready, blocks, d_tasks, ntasks, d_out, s); break;
    default: return launch_lines_qr<Q, 4>(ready, blocks, d_tasks, ntasks, d_out, s);
  }
  return cudaErrorInvalidValue;
}

int launch_section_lines(int q, int rm, const SecLineTask* d_tasks, int ntasks, uint32_t warps, pp_super* d_out,
                         pp_stream s, bool ready) {
  if (!warps || !ntasks) return 0;
  if (rm == q || rm < -1 || rm > 4) return (int)cudaErrorInvalidValue;
  const unsigned blocks = (warps + kSecLineWarps - 1) / kSecLineWarps;
  cudaError_t e;
  switch (q) {
    case 0: e = launch_lines_q<0>(rm, ready, blocks, d_tasks, ntasks, d_out, s); break;
    case 1: e = launch_lines_q<1>(rm, ready, blocks, d_tasks, ntasks, d_out, s); break;
    case 2: e = launch_lines_q<2>(rm, ready, blocks, d_tasks, ntasks, d_out, s); break;
    default: e = launch_lines_q<3>(rm, ready, blocks, d_tasks, ntasks, d_out, s); break;
  }
  if (e) return (int)e;
  count_launch();
  return (int)cudaGetLastError();
}

int launch_five_masks(const uint64_t* d_boards, int n, uint64_t* d_out, pp_stream s) {
  if (n <= 0) return 0;
  five_masks_kernel<<<blocks_for(n, 128), 128, 0, s>>>(d_boards, n, d_out);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_rmax(const pp_super* d_in, int n, pp_super* d_out, pp_stream s) {
  if (n <= 0) return 0;
  rmax_kernel<<<blocks_for(n, 128), 128, 0, s>>>(d_in, n, d_out);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_shift(const pp_super* d_in, int n, int q, int u, pp_super* d_out, pp_stream s) {
  if (n <= 0) return 0;
  shift_kernel<<<blocks_for(n, 128), 128, 0, s>>>(d_in, n, q, u, d_out);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_materialise(const MatTask* d_tasks, int ntasks, uint32_t blocks, pp_super* d_out, pp_stream s) {
  if (!blocks || !ntasks) return 0;
  materialise_kernel<<<blocks, kBlock, 0, s>>>(d_tasks, ntasks, d_out);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_symmetry(const pp_super* d_in, int n, int sym, uint32_t turns, pp_super* d_out, pp_stream s) {
  if (n <= 0) return 0;
  symmetry_kernel<<<blocks_for(n, 256), 256, 0, s>>>(d_in, n, sym, turns, d_out);
  count_launch();
  return (int)cudaGetLastError();
}

}  // namespace pp
