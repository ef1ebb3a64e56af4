// ba_draw.cuh -- the random draw that the chain of Fig. 1 makes at an odd position r.
//
// The refill kernels are written once over a Draw policy:
//   DrawPlain                h(r) of section 2: SplitMix64 bits of r, reduced into 0..r-1
//                            by a multiply-high.  The library's default graph.
//   DrawVariant<Crc, NoLoop> Crc:    the bits of Fig. 3's hash_crc (CRC-32C of r with two
//                                    initial values, first result in the high half),
//                                    reduced by the remainder as Fig. 3 does.
//                            NoLoop: section 4's self-loop-free rule: the draw for
//                                    position r = 2j+1 ranges over 0..2f-1, f the first
//                                    edge of the node that owns edge j, so it only reaches
//                                    edges of earlier nodes.  The key stays r.
// Every policy maps (graph, r) to one value; the chain stops on the same test (even, or
// a seed position) whatever the draw.
#pragma once
#include <cstdint>

#include "ba_device.cuh"

namespace ba {

// Ptx32 / Ptx64: the hash written in PTX on 32-bit / 64-bit positions (hash_r32_pre_ptx,
// hash_r64_pre_ptx; same values as the C forms).  The refill kernels (generate, batched,
// degree count) use the PTX forms on both widths; the rejection passes use the C form.
template <bool Ptx32, bool Ptx64>
struct DrawPlainT {
  static constexpr bool kPlain = true;
  static constexpr bool kTables = false;
  static constexpr bool kNeedsSeed = false;
  uint64_t spre = 0;
  // CTA-collective, once per kernel (nothing to prepare).
  __device__ __forceinline__ void setup(const GraphDev &, uint32_t *, bool) {}
  // Per tile: the graph whose positions are drawn next.
  __device__ __forceinline__ void bind(const GraphDev &g) { spre = g.seed_pre; }
  template <class RT>
  __device__ __forceinline__ RT operator()(RT r) const {
    if constexpr (sizeof(RT) == 4 && Ptx32) return hash_r32_pre_ptx(spre, r);
    else if constexpr (sizeof(RT) == 8 && Ptx64) return hash_r64_pre_ptx(spre, r);
    else return hash_pre<RT>(spre, r);
  }
};
using DrawPlain = DrawPlainT<false, false>;   // the C form everywhere
using DrawPlainPtx = DrawPlainT<true, true>;  // the PTX form everywhere

// CRC-32C in bit-reflected form (polynomial 0x1EDC6F41 reversed).
constexpr uint32_t kCrc32cReflected = 0x82F63B78u;

// One register step of the reflected CRC: divide by x, reduce.
__device__ __forceinline__ uint32_t crc_shift_bit(uint32_t c) {
  return (c >> 1) ^ (kCrc32cReflected & (0u - (c & 1u)));
}

// The CRC register after an 8-byte word whose byte k is b and all other bytes zero, from
// a zero register.  The CRC is linear over GF(2), so the register after any word w from
// register c is  reg_after_zero_word(c) XOR  XOR_k byte_part(k, byte k of w).
__device__ __forceinline__ uint32_t crc_byte_part(uint32_t k, uint32_t b) {
  uint32_t c = 0;
  for (uint32_t pos = 0; pos < 8; ++pos) {
    if (pos == k) c ^= b;
    for (int bit = 0; bit < 8; ++bit) c = crc_shift_bit(c);
  }
  return c;
}

// The register after a zero word from register c: the initial value's share.
__device__ __forceinline__ uint32_t crc_register_part(uint32_t c) {
  for (int bit = 0; bit < 64; ++bit) c = crc_shift_bit(c);
  return c;
}

// Bytes of a position that the CRC tables cover: 4 on the 32-bit path (the upper half of
// a position < 2^32 is zero and adds nothing), 8 otherwise.
__host__ __device__ constexpr uint32_t crc_table_bytes(bool r32) { return r32 ? 4u : 8u; }
__host__ __device__ constexpr size_t crc_table_smem(bool r32) {
  return static_cast<size_t>(crc_table_bytes(r32)) * 256u * sizeof(uint32_t);
}

// x mod r for a 64-bit x and 1 <= r < 2^32, exactly, without a 64-bit division: r is
// normalised to d = r * 2^s in [2^31, 2^32) and x * 2^s (96 bits) reduced by two 2-by-1
// division steps with the reciprocal v = floor((2^64 - 1) / d) - 2^32 (Moller & Granlund,
// "Improved division by invariant integers", IEEE Trans. Computers 60(2), 2011, the
// division of a two-word number by a normalised word).  Here d changes with every call,
// so v comes from the hardware's approximate single-precision reciprocal (relative error
// below 2^-23, so |v0 - v| < 2^11) made exact with integer arithmetic.  v is the largest
// value with residual e(v) = 2^64 - d (2^32 + v) >= 1, and then e(v) <= d.  From
// e0 = e(v0) the exact step is k* = v - v0 = floor((e0 - 1) / d); e0 / d in single
// precision is within 2^-11 of the real quotient, so rounding e0 / d - 2^-8 down gives
// k* or k* - 1, never more: after the step 1 <= e <= 2d, and one compare settles it.
// (A device test checks it against floor((2^64 - 1) / d) - 2^32 for every d in [2^31, 2^32).)
__device__ __forceinline__ uint32_t recip_word(uint32_t d) {
  const float f = __uint2float_rn(d);
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(f));
  const float w = (y * 4294967296.0f - 1.0f) * 4294967296.0f;  // ~ v, in (0, 2^32]
  const uint32_t v0 = __float2uint_rz(w);                        // saturates at 2^32 - 1
  int64_t e = static_cast<int64_t>(0ull - (static_cast<uint64_t>(d) * v0 +
                                           (static_cast<uint64_t>(d) << 32)));
  const float ef = fmaf(__int2float_rn(static_cast<int32_t>(e >> 32)), 4294967296.0f,
                        __uint2float_rn(static_cast<uint32_t>(e)));
  const int32_t k = __float2int_rd(fmaf(ef, y, -0.00390625f));  // k* or k* - 1
  e -= static_cast<int64_t>(k) * static_cast<int64_t>(d);       // 1 <= e <= 2d
  return v0 + static_cast<uint32_t>(k) + (e > static_cast<int64_t>(d) ? 1u : 0u);
}
// (u1 * 2^32 + u0) mod d for u1 < d, d normalised, v = recip_word(d).
__device__ __forceinline__ uint32_t rem_2by1(uint32_t u1, uint32_t u0, uint32_t d, uint32_t v) {
  const uint64_t q = static_cast<uint64_t>(v) * u1 + (static_cast<uint64_t>(u1 + 1) << 32) + u0;
  uint32_t r = u0 - static_cast<uint32_t>(q >> 32) * d;
  if (r > static_cast<uint32_t>(q)) r += d;
  if (r >= d) r -= d;
  return r;
}
__device__ __forceinline__ uint32_t mod_64by32(uint64_t x, uint32_t r) {
  const uint32_t s = __clz(r);
  const uint32_t d = r << s;
  const uint32_t v = recip_word(d);
  // the three words of x * 2^s by funnel shifts (s <= 31; for s = 0 the top word is 0)
  const uint32_t xlo = static_cast<uint32_t>(x);
  const uint32_t xhi = static_cast<uint32_t>(x >> 32);
  const uint32_t x2 = __funnelshift_lc(xhi, 0u, s);
  const uint32_t x1 = __funnelshift_lc(xlo, xhi, s);
  const uint32_t r1 = rem_2by1(x2, x1, d, v);
  return rem_2by1(r1, xlo << s, d, v) >> s;
}

template <bool Crc, bool NoLoop>
struct DrawVariant {
  static constexpr bool kPlain = false;
  static constexpr bool kTables = Crc;
  static constexpr bool kNeedsSeed = NoLoop;  // the first new node needs a seed edge
  uint64_t spre = 0;            // SplitMix64 draws
  const uint32_t *tab = nullptr;  // Crc: byte_part tables, 256 entries per byte position
  uint32_t reg_hi = 0;          // Crc: shares of the two initial values
  uint32_t reg_lo = 0;
  uint64_t m0 = 0;              // NoLoop: first edge of node n0, and division by d
  FastDiv div{};
  uint32_t d = 1;

  // CTA-collective: builds the CRC tables in shared memory (all threads take part, then
  // one __syncthreads).  Fig. 3's initial values 0 and 1 become the low half of the seed
  // and the high half XOR 1 (Fig. 3 exactly for seed 0).
  __device__ __forceinline__ void setup(const GraphDev &g, uint32_t *smem_tab, bool r32) {
    if constexpr (Crc) {
      const uint32_t entries = crc_table_bytes(r32) * 256u;
      for (uint32_t e = threadIdx.x; e < entries; e += blockDim.x)
        smem_tab[e] = crc_byte_part(e >> 8, e & 255u);
      reg_hi = crc_register_part(static_cast<uint32_t>(g.seed));
      reg_lo = crc_register_part(static_cast<uint32_t>(g.seed >> 32) ^ 1u);
      tab = smem_tab;
      __syncthreads();
    }
  }
  __device__ __forceinline__ void bind(const GraphDev &g) {
    spre = g.seed_pre;
    m0 = g.m0;
    div = g.div;
    d = g.d;
  }

  // Range of the draw at odd position r >= 2 m0 (r itself without NoLoop).  Positions
  // inside the seed never reach a draw that matters (their edges are rewritten from the
  // clique); they are clamped to the first new node so the range stays >= 2 m0 >= 2.
  template <class RT>
  __device__ __forceinline__ RT range_of(RT r) const {
    if constexpr (!NoLoop) {
      return r;
    } else if constexpr (sizeof(RT) == 4) {
      const uint32_t m0_32 = static_cast<uint32_t>(m0);
      const uint32_t j = max(r >> 1, m0_32);
      return 2u * (m0_32 + d * div32(j - m0_32, div));
    } else {
      const uint64_t j = max(static_cast<uint64_t>(r >> 1), m0);
      return 2 * (m0 + static_cast<uint64_t>(d) * div64(j - m0, div));
    }
  }

  template <class RT>
  __device__ __forceinline__ uint64_t crc_bits(RT r) const {
    uint32_t c = tab[r & 255u] ^ tab[256u + ((r >> 8) & 255u)] ^ tab[512u + ((r >> 16) & 255u)] ^
                 tab[768u + static_cast<uint32_t>((r >> 24) & 255u)];
    if constexpr (sizeof(RT) == 8) {
      const uint32_t hi = static_cast<uint32_t>(r >> 32);
      c ^= tab[1024u + (hi & 255u)] ^ tab[1280u + ((hi >> 8) & 255u)] ^
           tab[1536u + ((hi >> 16) & 255u)] ^ tab[1792u + (hi >> 24)];
    }
    return (static_cast<uint64_t>(c ^ reg_hi) << 32) | (c ^ reg_lo);
  }

  template <class RT>
  __device__ __forceinline__ RT operator()(RT r) const {
    const RT range = range_of<RT>(r);
    if constexpr (Crc) {
      // Fig. 3's remainder; a range below 2^32 on the 32-bit path
      if constexpr (sizeof(RT) == 4) return mod_64by32(crc_bits<RT>(r), range);
      else return static_cast<RT>(crc_bits<RT>(r) % static_cast<uint64_t>(range));
    } else if constexpr (sizeof(RT) == 4) {
      // SplitMix64 bits of key r, multiply-high by the range (< 2^32)
      return hash_r32_keyed_ptx(spre, r, range);
    } else {
      return hash_r64_keyed_ptx(spre, r, range);
    }
  }
};

// Variant flags of the public API (BA_VARIANT_*) to policy.
enum : uint32_t { kVariantCrc = 1u, kVariantNoLoop = 2u };

}  // namespace ba
