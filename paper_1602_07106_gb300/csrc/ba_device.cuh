// ba_device.cuh -- device-side arithmetic of generateEdge (paper Fig. 1, section 4).
//
// Everything here is integer arithmetic on the CUDA cores: no tensor cores, since the
// work is hashing, not a contraction.  Two position paths compute identical values:
//   * R32: every position r < 2^32 (ranges with edge_end <= 2^31).  r*G and the final
//     multiply-high need two 32x32->64 IMADs each instead of a full 64x64 product;
//     the paper's observation that 32-bit arithmetic is much cheaper (section 3),
//     applied to positions only -- node IDs are still written as int64.
//   * R64: any position r < 2^63.
#pragma once
#include <cstdint>

namespace ba {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;  // SplitMix64 increment (golden ratio)
constexpr uint64_t kMixA = 0xBF58476D1CE4E5B9ull;   // SplitMix64 finaliser multipliers
constexpr uint64_t kMixB = 0x94D049BB133111EBull;

// SplitMix64 finaliser (Steele, Lea & Flood 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * kMixA;
  z = (z ^ (z >> 27)) * kMixB;
  return z ^ (z >> 31);
}

// h(r) in 0..r-1 for r < 2^32.  floor(z*r/2^64) = floor((z_hi*r + floor(z_lo*r/2^32))/2^32),
// and z_hi*r + floor(z_lo*r/2^32) < 2^64, so one IMAD.HI and one wide IMAD suffice.
__device__ __forceinline__ uint32_t hash_r32(uint64_t seed, uint32_t r) {
  const uint64_t z = mix64(seed ^ (static_cast<uint64_t>(r) * kGamma));
  const uint32_t zlo = static_cast<uint32_t>(z);
  const uint32_t zhi = static_cast<uint32_t>(z >> 32);
  const uint32_t t = __umulhi(zlo, r);
  return static_cast<uint32_t>((static_cast<uint64_t>(zhi) * r + t) >> 32);
}

// h(r) in 0..r-1 for any r.
__device__ __forceinline__ uint64_t hash_r64(uint64_t seed, uint64_t r) {
  return __umul64hi(mix64(seed ^ (r * kGamma)), r);
}

// The seed's share of the first xor-shift.  Logical shifts distribute over xor, so for
// x = seed ^ p:  x ^ (x >> 30) = (seed ^ (seed >> 30)) ^ p ^ (p >> 30), and
// seed_pre = seed ^ (seed >> 30) is a per-graph constant.
__host__ __device__ constexpr uint64_t seed_premix(uint64_t seed) { return seed ^ (seed >> 30); }

// h(r) with seed_pre in place of the seed: one xor fewer per hash than the plain form.
// On sm_103 the hash is bound by the IMAD pipe (the 64-bit multiplies), so this is the
// form the hot loops use; the simple kernels keep the plain form as a cross-check.
__device__ __forceinline__ uint32_t hash_r32_pre(uint64_t seed_pre, uint32_t r) {
  const uint64_t p = static_cast<uint64_t>(r) * kGamma;
  uint64_t z = (seed_pre ^ p ^ (p >> 30)) * kMixA;
  z = (z ^ (z >> 27)) * kMixB;
  z ^= z >> 31;
  const uint32_t zlo = static_cast<uint32_t>(z);
  const uint32_t zhi = static_cast<uint32_t>(z >> 32);
  const uint32_t t = __umulhi(zlo, r);
  return static_cast<uint32_t>((static_cast<uint64_t>(zhi) * r + t) >> 32);
}

// hash_r32_pre spelled out in PTX with 32-bit multiplies only: each 64-bit product is a
// mul.lo / mul.hi / mad.lo sequence on 32-bit halves, so no operand has to be placed in a
// 64-bit register pair, and the final multiply-high floor((z_hi r + hi(z_lo r)) / 2^32) is
// one carry chain (mad.lo.cc, madc.hi).  Funnel shifts for the 64-bit right shifts,
// three-input xors.  Same values as hash_r32_pre; measured 8 % faster on the two-draw
// floor than the compiler's lowering of the C form.
__device__ __forceinline__ uint32_t hash_r32_pre_ptx(uint64_t seed_pre, uint32_t r) {
  const uint32_t slo = static_cast<uint32_t>(seed_pre);
  const uint32_t shi = static_cast<uint32_t>(seed_pre >> 32);
  uint32_t out;
  asm("{\n\t"
      ".reg .u32 plo, phi, tlo, thi, xlo, xhi, zlo, zhi, q, c;\n\t"
      "mul.lo.u32 plo, %1, 0x7F4A7C15;\n\t"       // p = r * G  (G = 0x9E3779B97F4A7C15)
      "mul.hi.u32 phi, %1, 0x7F4A7C15;\n\t"
      "mad.lo.u32 phi, %1, 0x9E3779B9, phi;\n\t"
      "shf.r.clamp.b32 tlo, plo, phi, 30;\n\t"     // p >> 30
      "shr.u32 thi, phi, 30;\n\t"
      "lop3.b32 xlo, %2, plo, tlo, 0x96;\n\t"     // x = seed_pre ^ p ^ (p >> 30)
      "lop3.b32 xhi, %3, phi, thi, 0x96;\n\t"
      "mul.lo.u32 zlo, xlo, 0x1CE4E5B9;\n\t"       // z = x * 0xBF58476D1CE4E5B9
      "mul.hi.u32 zhi, xlo, 0x1CE4E5B9;\n\t"
      "mad.lo.u32 zhi, xlo, 0xBF58476D, zhi;\n\t"
      "mad.lo.u32 zhi, xhi, 0x1CE4E5B9, zhi;\n\t"
      "shf.r.clamp.b32 tlo, zlo, zhi, 27;\n\t"     // z ^= z >> 27
      "shr.u32 thi, zhi, 27;\n\t"
      "xor.b32 xlo, zlo, tlo;\n\t"
      "xor.b32 xhi, zhi, thi;\n\t"
      "mul.lo.u32 zlo, xlo, 0x133111EB;\n\t"       // z *= 0x94D049BB133111EB
      "mul.hi.u32 zhi, xlo, 0x133111EB;\n\t"
      "mad.lo.u32 zhi, xlo, 0x94D049BB, zhi;\n\t"
      "mad.lo.u32 zhi, xhi, 0x133111EB, zhi;\n\t"
      "shf.r.clamp.b32 tlo, zlo, zhi, 31;\n\t"     // z ^= z >> 31
      "shr.u32 thi, zhi, 31;\n\t"
      "xor.b32 zlo, zlo, tlo;\n\t"
      "xor.b32 zhi, zhi, thi;\n\t"
      "mul.hi.u32 q, zlo, %1;\n\t"                 // floor(z * r / 2^64)
      "mad.lo.cc.u32 c, zhi, %1, q;\n\t"
      "madc.hi.u32 %0, zhi, %1, 0;\n\t"
      "}"
      : "=r"(out)
      : "r"(r), "r"(slo), "r"(shi));
  return out;
}

// hash_r64_pre in the same style, for any r < 2^64: r * G from the halves of r, and
// floor(z r / 2^64) = z_hi r_hi + floor((z_hi r_lo + z_lo r_hi + hi(z_lo r_lo)) / 2^32),
// where the inner sum is taken in 65 bits by carry chains.
__device__ __forceinline__ uint64_t hash_r64_pre_ptx(uint64_t seed_pre, uint64_t r) {
  const uint32_t slo = static_cast<uint32_t>(seed_pre);
  const uint32_t shi = static_cast<uint32_t>(seed_pre >> 32);
  const uint32_t rlo = static_cast<uint32_t>(r);
  const uint32_t rhi = static_cast<uint32_t>(r >> 32);
  uint32_t olo, ohi;
  asm("{\n\t"
      ".reg .u32 plo, phi, tlo, thi, xlo, xhi, zlo, zhi, a0, m1lo, m1hi, s0, s1, s2;\n\t"
      "mul.lo.u32 plo, %2, 0x7F4A7C15;\n\t"       // p = r * G mod 2^64
      "mul.hi.u32 phi, %2, 0x7F4A7C15;\n\t"
      "mad.lo.u32 phi, %2, 0x9E3779B9, phi;\n\t"
      "mad.lo.u32 phi, %3, 0x7F4A7C15, phi;\n\t"
      "shf.r.clamp.b32 tlo, plo, phi, 30;\n\t"     // p >> 30
      "shr.u32 thi, phi, 30;\n\t"
      "lop3.b32 xlo, %4, plo, tlo, 0x96;\n\t"     // x = seed_pre ^ p ^ (p >> 30)
      "lop3.b32 xhi, %5, phi, thi, 0x96;\n\t"
      "mul.lo.u32 zlo, xlo, 0x1CE4E5B9;\n\t"       // z = x * 0xBF58476D1CE4E5B9
      "mul.hi.u32 zhi, xlo, 0x1CE4E5B9;\n\t"
      "mad.lo.u32 zhi, xlo, 0xBF58476D, zhi;\n\t"
      "mad.lo.u32 zhi, xhi, 0x1CE4E5B9, zhi;\n\t"
      "shf.r.clamp.b32 tlo, zlo, zhi, 27;\n\t"     // z ^= z >> 27
      "shr.u32 thi, zhi, 27;\n\t"
      "xor.b32 xlo, zlo, tlo;\n\t"
      "xor.b32 xhi, zhi, thi;\n\t"
      "mul.lo.u32 zlo, xlo, 0x133111EB;\n\t"       // z *= 0x94D049BB133111EB
      "mul.hi.u32 zhi, xlo, 0x133111EB;\n\t"
      "mad.lo.u32 zhi, xlo, 0x94D049BB, zhi;\n\t"
      "mad.lo.u32 zhi, xhi, 0x133111EB, zhi;\n\t"
      "shf.r.clamp.b32 tlo, zlo, zhi, 31;\n\t"     // z ^= z >> 31
      "shr.u32 thi, zhi, 31;\n\t"
      "xor.b32 zlo, zlo, tlo;\n\t"
      "xor.b32 zhi, zhi, thi;\n\t"
      "mul.hi.u32 a0, zlo, %2;\n\t"                // hi(z_lo r_lo)
      "mad.lo.cc.u32 m1lo, zhi, %2, a0;\n\t"       // m1 = z_hi r_lo + a0  (< 2^64)
      "madc.hi.u32 m1hi, zhi, %2, 0;\n\t"
      "mad.lo.cc.u32 s0, zlo, %3, m1lo;\n\t"       // S = m1 + z_lo r_hi  (65 bits);
      "madc.hi.cc.u32 s1, zlo, %3, m1hi;\n\t"      //   S >> 32 = s2:s1
      "addc.u32 s2, 0, 0;\n\t"
      "mad.lo.cc.u32 %0, zhi, %3, s1;\n\t"         // h = z_hi r_hi + (S >> 32)
      "madc.hi.u32 %1, zhi, %3, s2;\n\t"
      "}"
      : "=r"(olo), "=r"(ohi)
      : "r"(rlo), "r"(rhi), "r"(slo), "r"(shi));
  return (static_cast<uint64_t>(ohi) << 32) | olo;
}
// The same two forms with the key and the range apart: the bits of key r, reduced into
// 0..range-1 (section 4's self-loop-free draw keys on r but ranges over the earlier nodes'
// edges only).  hash_rXX_pre_ptx(s, r) equals hash_rXX_keyed_ptx(s, r, r).
__device__ __forceinline__ uint32_t hash_r32_keyed_ptx(uint64_t seed_pre, uint32_t r,
                                                       uint32_t range) {
  const uint32_t slo = static_cast<uint32_t>(seed_pre);
  const uint32_t shi = static_cast<uint32_t>(seed_pre >> 32);
  uint32_t out;
  asm("{\n\t"
      ".reg .u32 plo, phi, tlo, thi, xlo, xhi, zlo, zhi, q, c;\n\t"
      "mul.lo.u32 plo, %1, 0x7F4A7C15;\n\t"
      "mul.hi.u32 phi, %1, 0x7F4A7C15;\n\t"
      "mad.lo.u32 phi, %1, 0x9E3779B9, phi;\n\t"
      "shf.r.clamp.b32 tlo, plo, phi, 30;\n\t"
      "shr.u32 thi, phi, 30;\n\t"
      "lop3.b32 xlo, %2, plo, tlo, 0x96;\n\t"
      "lop3.b32 xhi, %3, phi, thi, 0x96;\n\t"
      "mul.lo.u32 zlo, xlo, 0x1CE4E5B9;\n\t"
      "mul.hi.u32 zhi, xlo, 0x1CE4E5B9;\n\t"
      "mad.lo.u32 zhi, xlo, 0xBF58476D, zhi;\n\t"
      "mad.lo.u32 zhi, xhi, 0x1CE4E5B9, zhi;\n\t"
      "shf.r.clamp.b32 tlo, zlo, zhi, 27;\n\t"
      "shr.u32 thi, zhi, 27;\n\t"
      "xor.b32 xlo, zlo, tlo;\n\t"
      "xor.b32 xhi, zhi, thi;\n\t"
      "mul.lo.u32 zlo, xlo, 0x133111EB;\n\t"
      "mul.hi.u32 zhi, xlo, 0x133111EB;\n\t"
      "mad.lo.u32 zhi, xlo, 0x94D049BB, zhi;\n\t"
      "mad.lo.u32 zhi, xhi, 0x133111EB, zhi;\n\t"
      "shf.r.clamp.b32 tlo, zlo, zhi, 31;\n\t"
      "shr.u32 thi, zhi, 31;\n\t"
      "xor.b32 zlo, zlo, tlo;\n\t"
      "xor.b32 zhi, zhi, thi;\n\t"
      "mul.hi.u32 q, zlo, %4;\n\t"                 // floor(z * range / 2^64)
      "mad.lo.cc.u32 c, zhi, %4, q;\n\t"
      "madc.hi.u32 %0, zhi, %4, 0;\n\t"
      "}"
      : "=r"(out)
      : "r"(r), "r"(slo), "r"(shi), "r"(range));
  return out;
}
__device__ __forceinline__ uint64_t hash_r64_keyed_ptx(uint64_t seed_pre, uint64_t r,
                                                       uint64_t range) {
  const uint32_t slo = static_cast<uint32_t>(seed_pre);
  const uint32_t shi = static_cast<uint32_t>(seed_pre >> 32);
  const uint32_t rlo = static_cast<uint32_t>(r);
  const uint32_t rhi = static_cast<uint32_t>(r >> 32);
  const uint32_t glo = static_cast<uint32_t>(range);
  const uint32_t ghi = static_cast<uint32_t>(range >> 32);
  uint32_t olo, ohi;
  asm("{\n\t"
      ".reg .u32 plo, phi, tlo, thi, xlo, xhi, zlo, zhi, a0, m1lo, m1hi, s0, s1, s2;\n\t"
      "mul.lo.u32 plo, %2, 0x7F4A7C15;\n\t"
      "mul.hi.u32 phi, %2, 0x7F4A7C15;\n\t"
      "mad.lo.u32 phi, %2, 0x9E3779B9, phi;\n\t"
      "mad.lo.u32 phi, %3, 0x7F4A7C15, phi;\n\t"
      "shf.r.clamp.b32 tlo, plo, phi, 30;\n\t"
      "shr.u32 thi, phi, 30;\n\t"
      "lop3.b32 xlo, %4, plo, tlo, 0x96;\n\t"
      "lop3.b32 xhi, %5, phi, thi, 0x96;\n\t"
      "mul.lo.u32 zlo, xlo, 0x1CE4E5B9;\n\t"
      "mul.hi.u32 zhi, xlo, 0x1CE4E5B9;\n\t"
      "mad.lo.u32 zhi, xlo, 0xBF58476D, zhi;\n\t"
      "mad.lo.u32 zhi, xhi, 0x1CE4E5B9, zhi;\n\t"
      "shf.r.clamp.b32 tlo, zlo, zhi, 27;\n\t"
      "shr.u32 thi, zhi, 27;\n\t"
      "xor.b32 xlo, zlo, tlo;\n\t"
      "xor.b32 xhi, zhi, thi;\n\t"
      "mul.lo.u32 zlo, xlo, 0x133111EB;\n\t"
      "mul.hi.u32 zhi, xlo, 0x133111EB;\n\t"
      "mad.lo.u32 zhi, xlo, 0x94D049BB, zhi;\n\t"
      "mad.lo.u32 zhi, xhi, 0x133111EB, zhi;\n\t"
      "shf.r.clamp.b32 tlo, zlo, zhi, 31;\n\t"
      "shr.u32 thi, zhi, 31;\n\t"
      "xor.b32 zlo, zlo, tlo;\n\t"
      "xor.b32 zhi, zhi, thi;\n\t"
      "mul.hi.u32 a0, zlo, %6;\n\t"                // floor(z * range / 2^64) on halves
      "mad.lo.cc.u32 m1lo, zhi, %6, a0;\n\t"
      "madc.hi.u32 m1hi, zhi, %6, 0;\n\t"
      "mad.lo.cc.u32 s0, zlo, %7, m1lo;\n\t"
      "madc.hi.cc.u32 s1, zlo, %7, m1hi;\n\t"
      "addc.u32 s2, 0, 0;\n\t"
      "mad.lo.cc.u32 %0, zhi, %7, s1;\n\t"
      "madc.hi.u32 %1, zhi, %7, s2;\n\t"
      "}"
      : "=r"(olo), "=r"(ohi)
      : "r"(rlo), "r"(rhi), "r"(slo), "r"(shi), "r"(glo), "r"(ghi));
  return (static_cast<uint64_t>(ohi) << 32) | olo;
}
static_assert(kGamma == 0x9E3779B97F4A7C15ull && kMixA == 0xBF58476D1CE4E5B9ull &&
                  kMixB == 0x94D049BB133111EBull,
              "the PTX forms of the hash spell these constants out");

__device__ __forceinline__ uint64_t hash_r64_pre(uint64_t seed_pre, uint64_t r) {
  const uint64_t p = r * kGamma;
  uint64_t z = (seed_pre ^ p ^ (p >> 30)) * kMixA;
  z = (z ^ (z >> 27)) * kMixB;
  z ^= z >> 31;
  return __umul64hi(z, r);
}

template <class RT>
__device__ __forceinline__ RT hash_pre(uint64_t seed_pre, RT r);
template <>
__device__ __forceinline__ uint32_t hash_pre<uint32_t>(uint64_t seed_pre, uint32_t r) {
  return hash_r32_pre(seed_pre, r);
}
template <>
__device__ __forceinline__ uint64_t hash_pre<uint64_t>(uint64_t seed_pre, uint64_t r) {
  return hash_r64_pre(seed_pre, r);
}

template <class RT>
__device__ __forceinline__ RT hash_pos(uint64_t seed, RT r);
template <>
__device__ __forceinline__ uint32_t hash_pos<uint32_t>(uint64_t seed, uint32_t r) {
  return hash_r32(seed, r);
}
template <>
__device__ __forceinline__ uint64_t hash_pos<uint64_t>(uint64_t seed, uint64_t r) {
  return hash_r64(seed, r);
}

// Division by the constant d (Granlund & Montgomery 1994, multiply-high by a rounded-up
// reciprocal).  With l = ceil(log2 d):
//   64-bit numerators x < 2^62:  M = ceil(2^(62+l)/d) < 2^64,  x/d = umulhi(4x, M) >> l
//   31-bit numerators x < 2^31:  M = ceil(2^(31+l)/d) < 2^32,  x/d = umulhi(x, M) >> (l-1)
//                                (d = 1, l = 0: x itself)
// Exact because x*(M*d - 2^p) < 2^p in both cases.
struct FastDiv {
  uint64_t m64;
  uint32_t l;
  uint32_t m32;
  uint32_t pow2;  // d == 2^l
  uint32_t pad;
};

__device__ __forceinline__ uint64_t div64(uint64_t x, const FastDiv &f) {
  return __umul64hi(x << 2, f.m64) >> f.l;
}
__device__ __forceinline__ uint32_t div32(uint32_t x, const FastDiv &f) {
  return f.l ? __umulhi(x, f.m32) >> (f.l - 1) : x;
}

// Seed clique (section 4): position p < 2 m0 belongs to seed edge k = p/2 = v(v-1)/2 + u,
// E[2k] = v, E[2k+1] = u.  v comes from the quadratic formula, corrected to the exact
// integer by the two loops.  The estimate uses single precision (fast on every SM; off by
// at most a few steps below 2^40) and double precision only for larger seed cliques.
// Out of line: it runs for a few in 10^4 edges, and inlined copies in every kernel's flush
// and count paths slowed the common path of seeded graphs by ~10 % (code size).
static __device__ __noinline__ uint64_t clique_position(uint64_t p) {
  if (p < (1ull << 31)) {  // 32-bit fast path: k < 2^30, so v <= 46341 and v(v+1) < 2^32
    const uint32_t k = static_cast<uint32_t>(p >> 1);
    uint32_t v = static_cast<uint32_t>((1.0f + sqrtf(8.0f * static_cast<float>(k) + 1.0f)) * 0.5f);
    while (v > 1 && v * (v - 1) / 2 > k) --v;
    while (v * (v + 1) / 2 <= k) ++v;
    return (p & 1) ? k - v * (v - 1) / 2 : v;
  }
  const uint64_t k = p >> 1;
  uint64_t v = k < (1ull << 40)
                   ? static_cast<uint64_t>((1.0f + sqrtf(8.0f * static_cast<float>(k) + 1.0f)) * 0.5f)
                   : static_cast<uint64_t>((1.0 + sqrt(8.0 * static_cast<double>(k) + 1.0)) * 0.5);
  while (v > 1 && v * (v - 1) / 2 > k) --v;
  while (v * (v + 1) / 2 <= k) ++v;
  return (p & 1) ? k - v * (v - 1) / 2 : v;
}

// Per-graph constants, computed on the host (make_graph_dev in ba_api.cu).
struct GraphDev {
  uint64_t seed;
  uint64_t seed_pre;  // seed_premix(seed)
  uint64_t n;         // nodes
  uint64_t n0;        // first non-seed node
  uint64_t m0;        // seed edges
  uint64_t two_m0;    // positions below this are seed positions
  uint64_t begin;     // edge range [begin, end) to emit
  uint64_t end;
  uint64_t out_edge;  // output slot (in edges) of edge `begin`
  uint64_t tile0;     // first global tile of this graph (batched launches)
  FastDiv div;        // division by d
  uint32_t d;
  uint32_t pad;
};

// E[2i]: the owner of edge i (clique edge for i < m0).
template <class RT, bool HasSeed>
__device__ __forceinline__ uint64_t source_of(uint64_t i, const GraphDev &g) {
  if (HasSeed && i < g.m0) return clique_position(2 * i);
  if constexpr (sizeof(RT) == 4) {
    return g.n0 + div32(static_cast<uint32_t>(i - g.m0), g.div);
  } else {
    return g.n0 + div64(i - g.m0, g.div);
  }
}

// E[r] for the position r where the chain of Fig. 1 stopped (even, or a seed position).
template <class RT, bool HasSeed>
__device__ __forceinline__ uint64_t target_of(RT r, const GraphDev &g) {
  if (HasSeed && r < g.two_m0) return clique_position(r);
  if constexpr (sizeof(RT) == 4) {
    return g.n0 + div32((r >> 1) - static_cast<uint32_t>(g.m0), g.div);
  } else {
    return g.n0 + div64((r >> 1) - g.m0, g.div);
  }
}

// 2 m0 as a position of type RT.  On the 32-bit path a seed larger than every position
// in range saturates: every chain then stops in the seed, as it must.
template <class RT>
__device__ __forceinline__ RT seed_limit(uint64_t two_m0) {
  if constexpr (sizeof(RT) == 4) return two_m0 > 0xffffffffull ? 0xffffffffu : static_cast<RT>(two_m0);
  else return two_m0;
}

// Does the chain stop at position r?  (Fig. 1: r even; section 4: r inside the seed.)
template <class RT, bool HasSeed>
__device__ __forceinline__ bool chain_stops(RT r, RT two_m0) {
  return ((r & 1) == 0) || (HasSeed && r < two_m0);
}

// generateEdge(i), Fig. 1, one edge at a time.
template <class RT, bool HasSeed>
__device__ __forceinline__ void generate_edge(uint64_t i, const GraphDev &g, uint64_t &u,
                                              uint64_t &v) {
  if (HasSeed && i < g.m0) {
    u = clique_position(2 * i);
    v = clique_position(2 * i + 1);
    return;
  }
  RT r = static_cast<RT>(2 * i + 1);
  const RT two_m0 = seed_limit<RT>(g.two_m0);
  do {
    r = hash_pos<RT>(g.seed, r);
  } while (!chain_stops<RT, HasSeed>(r, two_m0));
  u = source_of<RT, HasSeed>(i, g);
  v = target_of<RT, HasSeed>(r, g);
}

// 16-byte streaming store of one (source, target) pair.
__device__ __forceinline__ void store_edge(int64_t *out, uint64_t k, uint64_t u, uint64_t v) {
  __stcs(reinterpret_cast<longlong2 *>(out) + k,
         make_longlong2(static_cast<long long>(u), static_cast<long long>(v)));
}

}  // namespace ba
