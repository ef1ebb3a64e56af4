// ba_kernels.cu -- the sm_103a kernels of libba and their launchers (the refill generate
// kernel itself is defined in ba_refill.cuh, which ba_fold.cu shares).
//
// Generate (paper Fig. 1 over a range of edge IDs):
//   k_generate_simple  one thread per edge, grid-stride; the parity baseline.
//   k_generate_refill  persistent warps.  Each warp takes tiles of T edge IDs from a
//                      global counter (section 2's dynamic load balancing by batches of
//                      edge IDs).  Every step each busy lane applies one draw; a lane whose
//                      chain stopped parks the final position r in the warp's staging ring
//                      (1024 entries, indexed by the edge's offset in the tile) and takes
//                      the tile's next edge ID by ballot/popc compaction, so geometric
//                      chain lengths do not leave lanes idle.  Whenever the oldest
//                      256-edge chunk of the ring has no chain left in flight, the whole
//                      warp writes it out: consecutive lanes store consecutive 16-byte
//                      (source, target) pairs (8-byte int32 pairs for the narrow output).
//                      The draw is a policy (ba_draw.cuh): h(r), or the variants.  The
//                      fast steps' bookkeeping (stop test, parked store, ballot, hand-out)
//                      is predicated PTX, so a step has no branch.
// Degree count (section 3's streaming analysis, no edge stored):
//   k_degree_init      sources and seed-clique end points in closed form.
//   k_degree_simple    one thread per edge, global atomics.
//   k_degree_refill    the refill scheduler of k_generate_refill; chains that stop below
//                      the position of the first uncounted node are parked in per-lane
//                      hit buffers (one predicated store) and counted by the whole warp
//                      when a buffer is half full: targets below the shared-memory limit
//                      in a per-CTA 64-bit histogram (optionally one atomic per distinct
//                      node per warp, __match_any_sync), the rest with global 64-bit
//                      atomics.
#include <algorithm>
#include <type_traits>

#include "ba_refill.cuh"

namespace ba {
namespace {

thread_local int g_kernel_count = 0;

// ------------------------------------------------------------------ simple kernels --

template <class RT, bool HasSeed, bool Narrow>
__global__ void k_generate_simple(const GraphDev g, int64_t *__restrict__ out) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = g.begin + static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
       i < g.end; i += stride) {
    uint64_t u, v;
    generate_edge<RT, HasSeed>(i, g, u, v);
    store_pair<Narrow>(out, g.out_edge + (i - g.begin), u, v);
  }
}

// ------------------------------------------------------------------ degree kernels --

// Number of k in [lo, hi) that also lie in [a, b).
__device__ __forceinline__ uint64_t overlap(uint64_t lo, uint64_t hi, uint64_t a, uint64_t b) {
  const uint64_t x = max(lo, a), y = min(hi, b);
  return y > x ? y - x : 0;
}

// Smallest v >= 0 with v(v-1)/2 >= x.
__device__ __forceinline__ uint64_t tri_ceil_index(uint64_t x) {
  if (x == 0) return 0;
  uint64_t v = static_cast<uint64_t>((1.0 + sqrt(8.0 * static_cast<double>(x) + 1.0)) * 0.5);
  while (v > 0 && (v - 1) * (v > 1 ? v - 2 : 0) / 2 >= x) --v;  // T(v-1) >= x: step down
  while (v * (v - 1) / 2 < x) ++v;
  return v;
}

// counts[j] (j < node_limit) = (accumulate ? counts[j] : 0) + end points of node j among
// edges [a, b) that are sources of non-seed edges or seed-clique edges.  Targets of
// non-seed edges are added by the chain kernels.
__global__ void k_degree_init(const GraphDev g, uint64_t a, uint64_t b, uint64_t node_limit,
                              uint64_t *__restrict__ counts, int accumulate) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t j = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < node_limit;
       j += stride) {
    uint64_t c = accumulate ? counts[j] : 0;
    if (j < g.n) {
      if (j >= g.n0) {
        const uint64_t lo = g.m0 + (j - g.n0) * g.d;
        c += overlap(lo, lo + g.d, a, b);
      } else {
        // seed edges (j, u), u < j: edges j(j-1)/2 .. j(j-1)/2 + j - 1
        const uint64_t tj = j * (j - 1) / 2;
        c += overlap(tj, tj + j, a, b);
        // seed edges (v, j), j < v < n0: edge v(v-1)/2 + j lies in [a, b)
        // iff v(v-1)/2 in [a-j, b-j)
        const uint64_t vlo = max(j + 1, a > j ? tri_ceil_index(a - j) : 0);
        const uint64_t vhi = min(g.n0, b > j ? tri_ceil_index(b - j) : 0);
        if (vhi > vlo) c += vhi - vlo;
      }
    }
    counts[j] = c;
  }
}

template <class RT, bool HasSeed>
__global__ void k_degree_simple(const GraphDev g, uint64_t hit_pos, uint64_t node_limit,
                                uint64_t *__restrict__ counts) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  const RT two_m0 = seed_limit<RT>(g.two_m0);
  for (uint64_t i = g.begin + static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
       i < g.end; i += stride) {
    RT r = static_cast<RT>(2 * i + 1);
    do {
      r = hash_pos<RT>(g.seed, r);
    } while (!chain_stops<RT, HasSeed>(r, two_m0));
    if (static_cast<uint64_t>(r) < hit_pos) {
      const uint64_t v = target_of<RT, HasSeed>(r, g);
      if (v < node_limit) atomicAdd(reinterpret_cast<unsigned long long *>(counts + v), 1ull);
    }
  }
}

// Adds one end point at node v for every lane with hit set.  Nodes below `hot` go to the
// CTA's 64-bit shared-memory bins, one atomic per distinct node per warp
// (__match_any_sync); the rest go to the global counters.  The atomics return nothing, so
// the warp does not wait for them.
__device__ __forceinline__ void histogram_add(bool hit, uint64_t v, unsigned long long *bins,
                                              uint32_t hot, uint64_t *__restrict__ counts) {
  const bool hot_hit = hit && v < hot;
  if (hit && !hot_hit) atomicAdd(reinterpret_cast<unsigned long long *>(counts + v), 1ull);
  const uint32_t key = hot_hit ? static_cast<uint32_t>(v) : 0xffffffffu;
  const uint32_t peers = __match_any_sync(kFull, key);
  if (hot_hit && (threadIdx.x & 31) == __ffs(peers) - 1)
    atomicAdd(bins + v, static_cast<unsigned long long>(__popc(peers)));
}

// Entries per warp of the hit buffers (stopped positions that may hit a counted node):
// 16 slots per lane.
constexpr uint32_t kHitRing = 512;

// One end point at node v from the calling lane alone: a shared-memory bin below `hot`,
// else the global counter.
__device__ __forceinline__ void histogram_add_lane(uint64_t v, unsigned long long *bins, uint32_t hot,
                                                   uint64_t *__restrict__ counts) {
  if (v < hot) atomicAdd(bins + v, 1ull);
  else atomicAdd(reinterpret_cast<unsigned long long *>(counts + v), 1ull);
}

// One fast step of the degree count for one chain as predicated PTX: the stop test, a
// stopped position below hp parked in the lane's own hit buffer (slot address hptr, the
// next slot 32 entries further), the warp's ballot and the hand-out of the next IDs.
template <bool Seed>
__device__ __forceinline__ void count_step(uint32_t &r, uint32_t &hoff, uint32_t &hptr,
                                           uint32_t lt, uint32_t r0, uint32_t two_m0,
                                           uint32_t hp) {
  if constexpr (Seed) {
    asm volatile(
        "{\n\t"
        ".reg .pred p, h;\n\t"
        ".reg .u32 t, fm, x;\n\t"
        "and.b32 t, %0, 1;\n\t"
        "setp.eq.u32 p, t, 0;\n\t"
        "setp.lt.or.u32 p, %0, %5, p;\n\t"
        "setp.lt.and.u32 h, %0, %6, p;\n\t"
        "@h st.shared.u32 [%2], %0;\n\t"
        "@h add.u32 %2, %2, 128;\n\t"
        "vote.sync.ballot.b32 fm, p, 0xffffffff;\n\t"
        "and.b32 x, fm, %3;\n\t"
        "popc.b32 x, x;\n\t"
        "add.u32 x, %1, x;\n\t"
        "@p mad.lo.u32 %0, x, 2, %4;\n\t"
        "popc.b32 x, fm;\n\t"
        "add.u32 %1, %1, x;\n\t"
        "}"
        : "+r"(r), "+r"(hoff), "+r"(hptr)
        : "r"(lt), "r"(r0), "r"(two_m0), "r"(hp)
        : "memory");
  } else {
    asm volatile(
        "{\n\t"
        ".reg .pred p, h;\n\t"
        ".reg .u32 t, fm, x;\n\t"
        "and.b32 t, %0, 1;\n\t"
        "setp.eq.u32 p, t, 0;\n\t"
        "setp.lt.and.u32 h, %0, %5, p;\n\t"
        "@h st.shared.u32 [%2], %0;\n\t"
        "@h add.u32 %2, %2, 128;\n\t"
        "vote.sync.ballot.b32 fm, p, 0xffffffff;\n\t"
        "and.b32 x, fm, %3;\n\t"
        "popc.b32 x, x;\n\t"
        "add.u32 x, %1, x;\n\t"
        "@p mad.lo.u32 %0, x, 2, %4;\n\t"
        "popc.b32 x, fm;\n\t"
        "add.u32 %1, %1, x;\n\t"
        "}"
        : "+r"(r), "+r"(hoff), "+r"(hptr)
        : "r"(lt), "r"(r0), "r"(hp)
        : "memory");
  }
}
template <bool Seed>
__device__ __forceinline__ void count_step(uint64_t &r, uint32_t &hoff, uint32_t &hptr,
                                           uint32_t lt, uint64_t r0, uint64_t two_m0,
                                           uint64_t hp) {
  if constexpr (Seed) {
    asm volatile(
        "{\n\t"
        ".reg .pred p, h;\n\t"
        ".reg .u32 t, fm, x, rl, rh, nl, nh;\n\t"
        "cvt.u32.u64 t, %0;\n\t"
        "and.b32 t, t, 1;\n\t"
        "setp.eq.u32 p, t, 0;\n\t"
        "setp.lt.or.u64 p, %0, %5, p;\n\t"
        "setp.lt.and.u64 h, %0, %6, p;\n\t"
        "@h st.shared.u64 [%2], %0;\n\t"
        "@h add.u32 %2, %2, 256;\n\t"
        "vote.sync.ballot.b32 fm, p, 0xffffffff;\n\t"
        "and.b32 x, fm, %3;\n\t"
        "popc.b32 x, x;\n\t"
        "add.u32 x, %1, x;\n\t"
        "mov.b64 {rl, rh}, %4;\n\t"
        "mov.b64 {nl, nh}, %0;\n\t"
        "@p mad.lo.cc.u32 nl, x, 2, rl;\n\t"
        "@p addc.u32 nh, rh, 0;\n\t"
        "mov.b64 %0, {nl, nh};\n\t"
        "popc.b32 x, fm;\n\t"
        "add.u32 %1, %1, x;\n\t"
        "}"
        : "+l"(r), "+r"(hoff), "+r"(hptr)
        : "r"(lt), "l"(r0), "l"(two_m0), "l"(hp)
        : "memory");
  } else {
    asm volatile(
        "{\n\t"
        ".reg .pred p, h;\n\t"
        ".reg .u32 t, fm, x, rl, rh, nl, nh;\n\t"
        "cvt.u32.u64 t, %0;\n\t"
        "and.b32 t, t, 1;\n\t"
        "setp.eq.u32 p, t, 0;\n\t"
        "setp.lt.and.u64 h, %0, %5, p;\n\t"
        "@h st.shared.u64 [%2], %0;\n\t"
        "@h add.u32 %2, %2, 256;\n\t"
        "vote.sync.ballot.b32 fm, p, 0xffffffff;\n\t"
        "and.b32 x, fm, %3;\n\t"
        "popc.b32 x, x;\n\t"
        "add.u32 x, %1, x;\n\t"
        "mov.b64 {rl, rh}, %4;\n\t"
        "mov.b64 {nl, nh}, %0;\n\t"
        "@p mad.lo.cc.u32 nl, x, 2, rl;\n\t"
        "@p addc.u32 nh, rh, 0;\n\t"
        "mov.b64 %0, {nl, nh};\n\t"
        "popc.b32 x, fm;\n\t"
        "add.u32 %1, %1, x;\n\t"
        "}"
        : "+l"(r), "+r"(hoff), "+r"(hptr)
        : "r"(lt), "l"(r0), "l"(hp)
        : "memory");
  }
}

// A parked position in the per-lane hit buffers, by shared-space address (the buffers are
// written by the PTX steps, so they are read and written through PTX too).
__device__ __forceinline__ void st_shared_pos(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void st_shared_pos(uint32_t a, uint64_t v) {
  asm volatile("st.shared.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
template <class RT>
__device__ __forceinline__ RT ld_shared_pos(uint32_t a) {
  if constexpr (sizeof(RT) == 4) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
  } else {
    uint64_t v;
    asm volatile("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
  }
}

// K chains per lane, as in k_generate_refill.
template <class RT, bool HasSeed, class Draw = DrawPlain, int K = 1>
__global__ void __launch_bounds__(1024, 1)
k_degree_refill(const GraphDev g, const SchedParams sp, uint64_t hit_pos, uint64_t node_limit,
                uint32_t hot, uint64_t *__restrict__ counts) {
  extern __shared__ __align__(16) unsigned long long bins[];
  for (uint32_t b = threadIdx.x; b < hot; b += blockDim.x) bins[b] = 0;
  __syncthreads();
  Draw draw;  // tables (if any) after the bins and the hit buffers
  draw.setup(g, reinterpret_cast<uint32_t *>(reinterpret_cast<RT *>(bins + hot) +
                                             static_cast<size_t>(blockDim.x >> 5) * kHitRing),
             sizeof(RT) == 4);
  draw.bind(g);

  const uint32_t shift = sp.tile_shift;
  const uint32_t T = 1u << shift;
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const uint64_t gwarp = static_cast<uint64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  constexpr uint32_t kLanes = 32u * K;
  // Fast steps between bounds checks and hit drains.
  constexpr uint32_t kSteps = 4;
  bool first = true;
  const RT two_m0 = seed_limit<RT>(g.two_m0);
  const bool agg = sp.hist_agg != 0;
  // Only a chain that stops below hit_pos can name a node below node_limit.  As a 32-bit
  // position, hit_pos >= 2^32 saturates (every stopped 32-bit position is below it).
  const RT hp = (sizeof(RT) == 4 && hit_pos > 0xffffffffull) ? static_cast<RT>(0xffffffffu)
                                                             : static_cast<RT>(hit_pos);

  // Stopped positions below hp are parked in the lane's own hit buffer: kLaneHits slots,
  // slot k of lane l at entry k*32 + l of the warp's kHitRing entries, hptr the lane's next
  // free slot.  Parking is one predicated store, with no ballot.  A fast iteration adds at
  // most kSteps*K per lane and a general step at most K, and after each of them the warp
  // resolves and counts every parked position once any lane holds more than half its slots.
  constexpr uint32_t kLaneHits = kHitRing / 32;
  constexpr uint32_t kSlot = 32u * sizeof(RT);  // bytes from one slot of a lane to the next
  static_assert(kSteps * K <= kLaneHits / 2, "a fast iteration's hits must fit in a lane's buffer");
  RT *hits = reinterpret_cast<RT *>(bins + hot) + static_cast<size_t>(threadIdx.x >> 5) * kHitRing;
  const uint32_t hbuf_s = static_cast<uint32_t>(__cvta_generic_to_shared(hits + lane));
  uint32_t hptr = hbuf_s;
  auto drain = [&]() {  // warp-collective: every parked position of every lane
    uint32_t n = (hptr - hbuf_s) / kSlot;
    while (__any_sync(kFull, n != 0)) {
      bool hit = n != 0;
      uint64_t v = 0;
      if (hit) {
        --n;
        v = target_of<RT, HasSeed>(ld_shared_pos<RT>(hbuf_s + n * kSlot), g);
        hit = v < node_limit;
      }
      if (agg) histogram_add(hit, v, bins, hot, counts);
      else if (hit) histogram_add_lane(v, bins, hot, counts);
    }
    hptr = hbuf_s;
  };
  auto maybe_drain = [&]() {
    if (__any_sync(kFull, hptr - hbuf_s > (kLaneHits / 2) * kSlot)) drain();
  };

  for (;;) {  // one tile at a time
    const uint64_t t = next_tile(sp, first, gwarp);
    if (t >= sp.num_tiles) break;
    const uint64_t base = g.begin + (t << shift);
    const uint32_t len = static_cast<uint32_t>(min(static_cast<uint64_t>(T), g.end - base));
    const RT r0 = static_cast<RT>(2 * base + 1);
    uint32_t hoff = min(kLanes, len);
    RT r[K];
    bool busy[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const uint32_t o = 32u * c + lane;
      busy[c] = o < hoff;
      r[c] = r0 + 2 * static_cast<RT>(o);
    }
    bool all_busy = hoff == kLanes;

    // Fast steps: every chain busy and >= kSteps*kLanes IDs left; the bookkeeping is
    // predicated PTX (count_step): no branch per step.
    auto fast_loop = [&](auto seed_tag) {
      constexpr bool Seed = decltype(seed_tag)::value;
      const uint32_t last = len - kSteps * kLanes;
      do {
#pragma unroll
        for (uint32_t u = 0; u < kSteps; ++u) {
#pragma unroll
          for (int c = 0; c < K; ++c) r[c] = draw(r[c]);
#pragma unroll
          for (int c = 0; c < K; ++c) count_step<Seed>(r[c], hoff, hptr, lt, r0, two_m0, hp);
        }
        maybe_drain();
      } while (hoff <= last);
    };

    for (;;) {
      if (all_busy && hoff + kSteps * kLanes <= len) {
        if (HasSeed && two_m0 != 0) fast_loop(std::true_type{});
        else fast_loop(std::false_type{});
      }
      bool any_busy = false;
#pragma unroll
      for (int c = 0; c < K; ++c) any_busy |= busy[c];
      if (hoff == len && !__any_sync(kFull, any_busy)) break;  // tile done
      // General step: some chains idle, or fewer than kSteps*kLanes IDs left.
      bool idle = false;
#pragma unroll
      for (int c = 0; c < K; ++c) {
        bool stop = false;
        if (busy[c]) {
          r[c] = draw(r[c]);
          stop = chain_stops<RT, HasSeed>(r[c], two_m0);
        }
        if (stop && r[c] < hp) {
          st_shared_pos(hptr, r[c]);
          hptr += kSlot;
        }
        if (stop) busy[c] = false;
        const uint32_t fm = __ballot_sync(kFull, !busy[c]);
        const uint32_t k = min(len - hoff, static_cast<uint32_t>(__popc(fm)));
        const uint32_t rank = __popc(fm & lt);
        if (!busy[c] && rank < k) {
          r[c] = r0 + 2 * static_cast<RT>(hoff + rank);
          busy[c] = true;
        }
        hoff += k;
        idle |= !busy[c];
      }
      all_busy = __ballot_sync(kFull, idle) == 0;
      maybe_drain();
    }
  }
  drain();
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < hot; b += blockDim.x) {
    const unsigned long long c = bins[b];
    if (c) atomicAdd(reinterpret_cast<unsigned long long *>(counts + b), static_cast<unsigned long long>(c));
  }
}

// ------------------------------------------------------------------------ launchers --

template <class RT, bool HasSeed, bool Narrow, class Draw = DrawPlainPtx, bool Checked = false>
ba_status generate_t(const GraphDev &g, int64_t *out, const Shape &s, unsigned long long *counter,
                     cudaStream_t stream, uint64_t out_cap = 0,
                     unsigned long long *status = nullptr) {
  const uint64_t len = g.end - g.begin;
  const int block = s.block;
  if constexpr (Draw::kPlain && !Checked) {  // the simple kernel draws h(r) only
    if (s.refill == 0) {
      int grid = 0;
      ba_status st = persistent_grid(k_generate_simple<RT, HasSeed, Narrow>, block, 0,
                                     s.ctas_per_sm, (len + block - 1) / block, &grid);
      if (st != BA_OK) return st;
      k_generate_simple<RT, HasSeed, Narrow><<<grid, block, 0, stream>>>(g, out);
      g_kernel_count = 1;
      return check_launch("k_generate_simple");
    }
  }
  const int warps = block / 32;
  const size_t smem = static_cast<size_t>(warps) * kRing * sizeof(RT) +
                      (Draw::kTables ? crc_table_smem(sizeof(RT) == 4) : 0);
  auto kernel = s.chains == 2 ? k_generate_refill<RT, HasSeed, false, Narrow, Draw, 2, Checked>
                              : k_generate_refill<RT, HasSeed, false, Narrow, Draw, 1, Checked>;
  ba_status st = set_smem(kernel, smem);
  if (st != BA_OK) return st;
  // Tiles of the tuned size, halved (down to 256) until every warp of a full grid has
  // about four, so that short ranges still spread over the whole GPU.
  int grid = 0;
  st = persistent_grid(kernel, block, smem, s.ctas_per_sm, ~0ull, &grid);
  if (st != BA_OK) return st;
  uint32_t shift = static_cast<uint32_t>(floor_log2(static_cast<uint32_t>(s.tile)));
  const uint64_t all_warps = static_cast<uint64_t>(grid) * warps;
  while (shift > 8 && (len >> shift) < 4 * all_warps) --shift;
  SchedParams sp{};
  sp.num_tiles = (len + (1ull << shift) - 1) >> shift;
  sp.counter = counter;
  sp.tile_shift = shift;
  sp.hist_agg = static_cast<uint32_t>(s.hist_agg);
  grid = static_cast<int>(std::min<uint64_t>(grid, (sp.num_tiles + warps - 1) / warps));
  sp.total_warps = static_cast<uint32_t>(grid) * warps;
  sp.out_cap = out_cap;
  sp.status = status;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  kernel<<<grid, block, smem, stream>>>(g, BatchTable{}, sp, out);
  g_kernel_count = 1;
  return check_launch("k_generate_refill");
}

template <class RT, bool HasSeed, class Draw = DrawPlain>
ba_status degree_t(const GraphDev &g, uint64_t hit_pos, uint64_t node_limit, uint64_t *counts,
                   const Shape &s, unsigned long long *counter, cudaStream_t stream) {
  const uint64_t len = g.end - g.begin;
  const int block = s.block;
  if constexpr (Draw::kPlain) {
    if (s.refill == 0) {
      int grid = 0;
      ba_status st = persistent_grid(k_degree_simple<RT, HasSeed>, block, 0, s.ctas_per_sm,
                                     (len + block - 1) / block, &grid);
      if (st != BA_OK) return st;
      k_degree_simple<RT, HasSeed><<<grid, block, 0, stream>>>(g, hit_pos, node_limit, counts);
      return check_launch("k_degree_simple");
    }
  }
  const int warps = block / 32;
  // The shape's shared-memory bins, fewer when the hit buffers and the draw's tables leave
  // less room (a shape tuned for the plain draw also serves the table-driven ones).
  const size_t fixed = static_cast<size_t>(warps) * kHitRing * sizeof(RT) +
                       (Draw::kTables ? crc_table_smem(sizeof(RT) == 4) : 0);
  uint32_t hot = static_cast<uint32_t>(std::min<uint64_t>(node_limit, std::max(s.hist_bins, 0)));
  if (fixed < kMaxSmemPerCta)
    hot = static_cast<uint32_t>(std::min<size_t>(hot, (kMaxSmemPerCta - fixed) / sizeof(unsigned long long)));
  const size_t smem = static_cast<size_t>(hot) * sizeof(unsigned long long) + fixed;
  auto kernel = s.chains == 2 ? k_degree_refill<RT, HasSeed, Draw, 2>
                              : k_degree_refill<RT, HasSeed, Draw, 1>;
  ba_status st = set_smem(kernel, smem);
  if (st != BA_OK) return st;
  int grid = 0;
  st = persistent_grid(kernel, block, smem, s.ctas_per_sm, ~0ull, &grid);
  if (st != BA_OK) return st;
  uint32_t shift = static_cast<uint32_t>(floor_log2(static_cast<uint32_t>(s.tile)));
  const uint64_t all_warps = static_cast<uint64_t>(grid) * warps;
  while (shift > 8 && (len >> shift) < 4 * all_warps) --shift;  // as for generate
  SchedParams sp{};
  sp.num_tiles = (len + (1ull << shift) - 1) >> shift;
  sp.counter = counter;
  sp.tile_shift = shift;
  sp.hist_agg = static_cast<uint32_t>(s.hist_agg);
  grid = static_cast<int>(std::min<uint64_t>(grid, (sp.num_tiles + warps - 1) / warps));
  sp.total_warps = static_cast<uint32_t>(grid) * warps;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  kernel<<<grid, block, smem, stream>>>(g, sp, hit_pos, node_limit, hot, counts);
  return check_launch("k_degree_refill");
}

template <class RT, bool HasSeed>
ba_status batch_t(const BatchTable &tab, uint64_t total_tiles, int64_t *out, const Shape &s,
                  unsigned long long *counter, cudaStream_t stream) {
  const uint32_t shift = static_cast<uint32_t>(floor_log2(static_cast<uint32_t>(s.tile)));
  const int block = s.block;
  const int warps = block / 32;
  const size_t smem = static_cast<size_t>(warps) * kRing * sizeof(RT) +
                      static_cast<size_t>(warps) * sizeof(GraphDev);
  auto kernel = s.chains == 2 ? k_generate_refill<RT, HasSeed, true, false, DrawPlainPtx, 2>
                              : k_generate_refill<RT, HasSeed, true, false, DrawPlainPtx, 1>;
  ba_status st = set_smem(kernel, smem);
  if (st != BA_OK) return st;
  SchedParams sp{};
  sp.num_tiles = total_tiles;
  sp.counter = counter;
  sp.tile_shift = shift;
  sp.hist_agg = static_cast<uint32_t>(s.hist_agg);
  int grid = 0;
  st = persistent_grid(kernel, block, smem, s.ctas_per_sm, (total_tiles + warps - 1) / warps, &grid);
  if (st != BA_OK) return st;
  sp.total_warps = static_cast<uint32_t>(grid) * warps;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  GraphDev dummy{};
  kernel<<<grid, block, smem, stream>>>(dummy, tab, sp, out);
  g_kernel_count = 1;
  return check_launch("k_generate_refill<batched>");
}

}  // namespace

int last_kernel_count() { return g_kernel_count; }

ba_status launch_generate(const GraphDev &g, int64_t *out, const Shape &s,
                          unsigned long long *counter, cudaStream_t stream, bool narrow) {
  g_kernel_count = 0;
  const bool r32 = g.end <= (1ull << 31);
  const bool seed = g.m0 > 0;
  if (narrow) {
    if (r32) return seed ? generate_t<uint32_t, true, true>(g, out, s, counter, stream)
                         : generate_t<uint32_t, false, true>(g, out, s, counter, stream);
    return seed ? generate_t<uint64_t, true, true>(g, out, s, counter, stream)
                : generate_t<uint64_t, false, true>(g, out, s, counter, stream);
  }
  if (r32) return seed ? generate_t<uint32_t, true, false>(g, out, s, counter, stream)
                       : generate_t<uint32_t, false, false>(g, out, s, counter, stream);
  return seed ? generate_t<uint64_t, true, false>(g, out, s, counter, stream)
              : generate_t<uint64_t, false, false>(g, out, s, counter, stream);
}

ba_status launch_generate_checked(const GraphDev &g, int64_t *out, uint64_t out_cap,
                                  unsigned long long *status, const Shape &shape,
                                  unsigned long long *counter, cudaStream_t stream) {
  g_kernel_count = 0;
  Shape s = shape;
  s.refill = 1;  // the checks live in the refill kernel's store path
  const bool r32 = g.end <= (1ull << 31);
  if (g.m0 > 0)
    return r32 ? generate_t<uint32_t, true, false, DrawPlainPtx, true>(g, out, s, counter, stream, out_cap, status)
               : generate_t<uint64_t, true, false, DrawPlainPtx, true>(g, out, s, counter, stream, out_cap, status);
  return r32 ? generate_t<uint32_t, false, false, DrawPlainPtx, true>(g, out, s, counter, stream, out_cap, status)
             : generate_t<uint64_t, false, false, DrawPlainPtx, true>(g, out, s, counter, stream, out_cap, status);
}

namespace {

// Generate with a variant draw: int64 output, refill kernel.  The self-loop-free rule
// needs a seed graph, so it never runs without one.
template <class Draw>
ba_status generate_variant_t(const GraphDev &g, int64_t *out, const Shape &s,
                             unsigned long long *counter, cudaStream_t stream, bool seed) {
  const bool r32 = g.end <= (1ull << 31);
  if (seed) return r32 ? generate_t<uint32_t, true, false, Draw>(g, out, s, counter, stream)
                       : generate_t<uint64_t, true, false, Draw>(g, out, s, counter, stream);
  if constexpr (Draw::kNeedsSeed) {
    return BA_ERR_INVALID_ARG;
  } else {
    return r32 ? generate_t<uint32_t, false, false, Draw>(g, out, s, counter, stream)
               : generate_t<uint64_t, false, false, Draw>(g, out, s, counter, stream);
  }
}

// Degree count: closed-form sources and seed end points, then the targets of the
// non-seed edges in range by the chain of Fig. 1 with the given draw.
template <class Draw>
ba_status degree_with(const GraphDev &g_in, uint64_t node_limit, uint64_t *counts, int accumulate,
                      const Shape &s, unsigned long long *counter, cudaStream_t stream) {
  g_kernel_count = 0;
  // 1. sources and seed end points, in closed form, over all node_limit entries
  {
    const int block = 256;
    const uint64_t want = (node_limit + block - 1) / block;
    const int grid = static_cast<int>(std::min<uint64_t>(want, static_cast<uint64_t>(sm_count()) * 8));
    k_degree_init<<<std::max(grid, 1), block, 0, stream>>>(g_in, g_in.begin, g_in.end, node_limit,
                                                           counts, accumulate);
    ba_status st = check_launch("k_degree_init");
    if (st != BA_OK) return st;
    g_kernel_count = 1;
  }
  // 2. targets of the non-seed edges in range, by the chain of Fig. 1
  GraphDev g = g_in;
  g.begin = std::max(g.begin, g.m0);
  if (g.begin >= g.end) return BA_OK;
  // A chain that stops at an even position r >= 2 m0 names node n0 + (r/2 - m0)/d, which is
  // below node_limit iff r < 2 m0 + 2 (node_limit - n0) d; seed positions may always hit.
  uint64_t hit_pos = g.two_m0;
  if (node_limit > g.n0) {
    const unsigned __int128 hp = static_cast<unsigned __int128>(g.two_m0) +
                                 static_cast<unsigned __int128>(2) * (node_limit - g.n0) * g.d;
    hit_pos = hp > (static_cast<unsigned __int128>(1) << 63) ? (1ull << 63) : static_cast<uint64_t>(hp);
  }
  const bool r32 = g.end <= (1ull << 31);
  const bool seed = g.m0 > 0;
  ba_status st;
  if (seed) {
    st = r32 ? degree_t<uint32_t, true, Draw>(g, hit_pos, node_limit, counts, s, counter, stream)
             : degree_t<uint64_t, true, Draw>(g, hit_pos, node_limit, counts, s, counter, stream);
  } else if constexpr (Draw::kNeedsSeed) {
    st = BA_ERR_INVALID_ARG;
  } else {
    st = r32 ? degree_t<uint32_t, false, Draw>(g, hit_pos, node_limit, counts, s, counter, stream)
             : degree_t<uint64_t, false, Draw>(g, hit_pos, node_limit, counts, s, counter, stream);
  }
  if (st == BA_OK) g_kernel_count = 2;
  return st;
}

}  // namespace

ba_status launch_degree_sources(const GraphDev &g, uint64_t node_limit, uint64_t *counts,
                                int accumulate, cudaStream_t stream) {
  const int block = 256;
  const uint64_t want = (node_limit + block - 1) / block;
  const int grid = static_cast<int>(std::min<uint64_t>(want, static_cast<uint64_t>(sm_count()) * 8));
  k_degree_init<<<std::max(grid, 1), block, 0, stream>>>(g, g.begin, g.end, node_limit, counts,
                                                         accumulate);
  return check_launch("k_degree_init");
}

ba_status launch_degree(const GraphDev &g, uint64_t node_limit, uint64_t *counts, int accumulate,
                        const Shape &s, unsigned long long *counter, cudaStream_t stream) {
  return degree_with<DrawPlainPtx>(g, node_limit, counts, accumulate, s, counter, stream);
}

ba_status launch_generate_variant(const GraphDev &g, int64_t *out, const Shape &s,
                                  unsigned long long *counter, cudaStream_t stream,
                                  uint32_t variant) {
  g_kernel_count = 0;
  const bool seed = g.m0 > 0;
  switch (variant) {
    case 0: return launch_generate(g, out, s, counter, stream, false);
    case kVariantCrc:
      return generate_variant_t<DrawVariant<true, false>>(g, out, s, counter, stream, seed);
    case kVariantNoLoop:
      return generate_variant_t<DrawVariant<false, true>>(g, out, s, counter, stream, seed);
    case kVariantCrc | kVariantNoLoop:
      return generate_variant_t<DrawVariant<true, true>>(g, out, s, counter, stream, seed);
    default: return BA_ERR_INVALID_ARG;
  }
}

ba_status launch_degree_variant(const GraphDev &g, uint64_t node_limit, uint64_t *counts,
                                int accumulate, const Shape &s, unsigned long long *counter,
                                cudaStream_t stream, uint32_t variant) {
  switch (variant) {
    case 0: return degree_with<DrawPlainPtx>(g, node_limit, counts, accumulate, s, counter, stream);
    case kVariantCrc:
      return degree_with<DrawVariant<true, false>>(g, node_limit, counts, accumulate, s, counter, stream);
    case kVariantNoLoop:
      return degree_with<DrawVariant<false, true>>(g, node_limit, counts, accumulate, s, counter, stream);
    case kVariantCrc | kVariantNoLoop:
      return degree_with<DrawVariant<true, true>>(g, node_limit, counts, accumulate, s, counter, stream);
    default: return BA_ERR_INVALID_ARG;
  }
}

ba_status launch_batch(const BatchTable &tab, uint64_t total_tiles, bool r32, bool has_seed,
                       int64_t *out, const Shape &s, unsigned long long *counter, cudaStream_t stream) {
  g_kernel_count = 0;
  if (total_tiles == 0) return BA_OK;
  if (r32) return has_seed ? batch_t<uint32_t, true>(tab, total_tiles, out, s, counter, stream)
                           : batch_t<uint32_t, false>(tab, total_tiles, out, s, counter, stream);
  return has_seed ? batch_t<uint64_t, true>(tab, total_tiles, out, s, counter, stream)
                  : batch_t<uint64_t, false>(tab, total_tiles, out, s, counter, stream);
}

}  // namespace ba
