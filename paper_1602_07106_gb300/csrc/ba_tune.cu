// ba_tune.cu -- launch shapes: defaults, per-kind overrides, and the autotuner cache.
//
// A shape never changes the output (every kernel emits the same bits for every shape);
// it only changes speed.  Lookup order: ba_set_tuning override > tuned entry for
// (kind, 32/64-bit position path) > default.  The cache persists as a small JSON file.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ba_internal.h"

namespace ba {
namespace {

constexpr int kKinds = 3;

struct Cache {
  std::mutex mu;
  bool loaded_env = false;
  bool has_override[kKinds] = {false, false, false};
  Shape override_shape[kKinds];
  bool has_tuned[kKinds][2] = {{false, false}, {false, false}, {false, false}};
  Shape tuned[kKinds][2];
};

Cache &cache() {
  static Cache c;
  return c;
}

// The shapes the autotuner settles on for a GB300 on the large workloads (2^31 edges on
// 32-bit positions, 10^12 edges on 64-bit ones), so that a caller who never tunes gets them.
// Occupancy decides most of it: the per-warp staging ring (4 KB on 32-bit positions, 8 KB on
// 64-bit ones) and the degree count's hit buffers and shared bins must leave room for 24-48
// resident warps per SM.
Shape default_shape(int kind, bool r32) {
  Shape s;
  s.refill = 1;
  s.chains = 2;
  switch (kind) {
    case BA_KIND_DEGREE:  // 32 KB of shared bins; hit buffers of 32 (64) KB per 512 threads
      s.block = 512; s.ctas_per_sm = r32 ? 4 : 2; s.tile = r32 ? 65536 : 16384;
      s.hist_bins = 4096;
      break;
    case BA_KIND_BATCH:  // small graphs: shorter tiles, one chain per lane
      s.block = 256; s.ctas_per_sm = 4; s.tile = r32 ? 16384 : 65536;
      s.chains = r32 ? 1 : 2;
      break;
    default:  // generate: 16 warps of 4 KB rings, or 8 warps of 8 KB rings, per CTA
      s.block = r32 ? 512 : 256; s.ctas_per_sm = 4; s.tile = 65536;
      break;
  }
  return s;
}

// Zero fields of an override take the 32-bit-position default.
Shape from_public(const ba_tuning &t, int kind) {
  Shape s = default_shape(kind, true);
  if (t.block > 0) s.block = t.block;
  if (t.ctas_per_sm > 0) s.ctas_per_sm = t.ctas_per_sm;
  if (t.tile > 0) s.tile = t.tile;
  s.refill = t.refill;
  if (t.hist_bins > 0) s.hist_bins = t.hist_bins;
  s.hist_agg = t.hist_agg;
  if (t.chains > 0) s.chains = t.chains;
  return s;
}

void to_public(const Shape &s, ba_tuning *t) {
  std::memset(t, 0, sizeof(*t));
  t->block = s.block;
  t->ctas_per_sm = s.ctas_per_sm;
  t->tile = s.tile;
  t->refill = s.refill;
  t->hist_bins = s.hist_bins;
  t->hist_agg = s.hist_agg;
  t->chains = s.chains;
}

bool valid_shape(const Shape &s, int kind) {
  if (s.block < 32 || s.block > 1024 || s.block % 32 != 0) return false;
  if (s.ctas_per_sm < 1 || s.ctas_per_sm > 32) return false;
  if (s.refill != 0 && s.refill != 1) return false;
  if (s.refill == 1 || kind == BA_KIND_BATCH) {
    if (s.tile < 64 || s.tile > (1 << 20) || (s.tile & (s.tile - 1)) != 0) return false;
  }
  if (s.hist_bins < 0 || s.hist_bins > 28 * 1024) return false;
  if (s.hist_agg != 0 && s.hist_agg != 1) return false;
  if (s.chains != 1 && s.chains != 2) return false;
  return true;
}

ba_status load_file(const char *path, Cache &c) {
  FILE *f = std::fopen(path, "r");
  if (!f) {
    set_error("cannot open tuner cache file");
    return BA_ERR_NOT_FOUND;
  }
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
  std::fclose(f);
  // Entries are flat objects {"kind":K,"r32":P,"block":B,"ctas_per_sm":C,"tile":T,
  // "refill":R,"hist_bins":H,"hist_agg":A[,"chains":N]}; keys are read in that fixed order
  // (files without "chains" mean one chain per lane).
  size_t pos = 0;
  int loaded = 0;
  while ((pos = text.find("{\"kind\"", pos)) != std::string::npos) {
    int kind, r32;
    Shape s;
    const int fields = std::sscanf(
        text.c_str() + pos,
        "{\"kind\": %d, \"r32\": %d, \"block\": %d, \"ctas_per_sm\": %d, \"tile\": %d, "
        "\"refill\": %d, \"hist_bins\": %d, \"hist_agg\": %d, \"chains\": %d}",
        &kind, &r32, &s.block, &s.ctas_per_sm, &s.tile, &s.refill, &s.hist_bins, &s.hist_agg,
        &s.chains);
    if ((fields == 8 || fields == 9) &&
        kind >= 0 && kind < kKinds && (r32 == 0 || r32 == 1) && valid_shape(s, kind)) {
      c.tuned[kind][r32] = s;
      c.has_tuned[kind][r32] = true;
      ++loaded;
    }
    pos += 7;
  }
  if (loaded == 0) {
    set_error("tuner cache file has no valid entries");
    return BA_ERR_INVALID_ARG;
  }
  return BA_OK;
}

void load_env_once(Cache &c) {
  if (c.loaded_env) return;
  c.loaded_env = true;
  const char *p = std::getenv("BA_TUNE_CACHE");
  if (p && *p) {
    std::string saved = ba_last_error_message();
    load_file(p, c);
    set_error(saved.c_str());
  }
}

}  // namespace

Shape shape_for(int kind, bool r32) {
  Cache &c = cache();
  std::lock_guard<std::mutex> lock(c.mu);
  load_env_once(c);
  if (c.has_override[kind]) return c.override_shape[kind];
  if (c.has_tuned[kind][r32 ? 1 : 0]) return c.tuned[kind][r32 ? 1 : 0];
  return default_shape(kind, r32);
}

ba_status shape_from_public(int kind, const ba_tuning *t, Shape *out) {
  if (kind < 0 || kind >= kKinds || t == nullptr) {
    set_error("unknown kernel kind or NULL tuning");
    return BA_ERR_INVALID_ARG;
  }
  Shape s = from_public(*t, kind);
  if (!valid_shape(s, kind)) {
    set_error("invalid launch shape (block multiple of 32 <= 1024, tile power of two 64..2^20, "
              "refill 0 or 1, hist_bins <= 28672, hist_agg 0 or 1, chains 1 or 2)");
    return BA_ERR_INVALID_ARG;
  }
  *out = s;
  return BA_OK;
}

void shape_store(int kind, bool r32, const Shape &s) {
  Cache &c = cache();
  std::lock_guard<std::mutex> lock(c.mu);
  c.tuned[kind][r32 ? 1 : 0] = s;
  c.has_tuned[kind][r32 ? 1 : 0] = true;
}

}  // namespace ba

using namespace ba;

namespace {

// Median time (ms) of `reps` runs of fn on `stream`.
template <class F>
ba_status time_median(F fn, cudaStream_t stream, int reps, float *ms) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  std::vector<float> t;
  ba_status st = fn();  // warm-up
  for (int i = 0; i < reps && st == BA_OK; ++i) {
    cudaEventRecord(a, stream);
    st = fn();
    cudaEventRecord(b, stream);
    cudaError_t e = cudaEventSynchronize(b);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaEventSynchronize");
    float x = 0;
    cudaEventElapsedTime(&x, a, b);
    t.push_back(x);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != BA_OK) return st;
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return BA_OK;
}

std::vector<Shape> candidates(int kind) {
  std::vector<Shape> out;
  const int blocks[] = {128, 256, 512};
  const int tiles[] = {1024, 4096, 16384, 65536};
  if (kind == BA_KIND_DEGREE) {
    const int dblocks[] = {256, 512, 1024};
    const int bins[] = {4096, 8192, 12288, 24576};
    for (int blk : dblocks)
      for (int ctas : {1, 2, 4})
        for (int tile : {16384, 65536})
          for (int hb : bins) {
            if (blk * ctas > 2048 || static_cast<size_t>(hb) * 8 * ctas > 220 * 1024) continue;
            for (int agg : {0, 1})
              for (int chains : {1, 2}) {
                Shape s;
                s.block = blk; s.ctas_per_sm = ctas; s.tile = tile; s.refill = 1;
                s.hist_bins = hb; s.hist_agg = agg; s.chains = chains;
                out.push_back(s);
              }
          }
    Shape simple;
    simple.block = 256; simple.ctas_per_sm = 8; simple.tile = 512; simple.refill = 0;
    out.push_back(simple);
    return out;
  }
  for (int blk : blocks)
    for (int ctas : {2, 4, 8})
      for (int tile : tiles)
        for (int chains : {1, 2}) {
          if (blk * ctas > 2048) continue;
          Shape s;
          s.block = blk; s.ctas_per_sm = ctas; s.tile = tile; s.refill = 1; s.chains = chains;
          out.push_back(s);
        }
  if (kind == BA_KIND_GENERATE) {
    Shape simple;
    simple.block = 256; simple.ctas_per_sm = 8; simple.tile = 512; simple.refill = 0;
    out.push_back(simple);
  }
  return out;
}

}  // namespace

extern "C" {

ba_status ba_set_tuning(int32_t kind, const ba_tuning *tune) {
  if (kind < 0 || kind >= kKinds) {
    set_error("unknown kernel kind");
    return BA_ERR_INVALID_ARG;
  }
  Cache &c = cache();
  std::lock_guard<std::mutex> lock(c.mu);
  if (tune == nullptr) {
    c.has_override[kind] = false;
    return BA_OK;
  }
  Shape s;
  ba_status st = shape_from_public(kind, tune, &s);
  if (st != BA_OK) return st;
  c.override_shape[kind] = s;
  c.has_override[kind] = true;
  return BA_OK;
}

ba_status ba_get_tuning(int32_t kind, uint64_t edge_end, ba_tuning *out) {
  if (kind < 0 || kind >= kKinds || out == nullptr) {
    set_error("unknown kernel kind or NULL output");
    return BA_ERR_INVALID_ARG;
  }
  to_public(shape_for(kind, edge_end <= (1ull << 31)), out);
  return BA_OK;
}

ba_status ba_tune(int32_t kind, uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                  uint64_t edge_begin, uint64_t edge_end, int64_t *scratch_dev, void *stream,
                  ba_tuning *out) {
  set_error("");
  if (kind < 0 || kind >= kKinds) {
    set_error("unknown kernel kind");
    return BA_ERR_INVALID_ARG;
  }
  uint64_t m = 0;
  ba_status st = validate_graph(n, d, n0, &m);
  if (st != BA_OK) return st;
  if (edge_begin >= edge_end || edge_end > m) {
    set_error("tuning range must be a non-empty range inside 0..m");
    return BA_ERR_RANGE;
  }
  const uint64_t len = edge_end - edge_begin;
  if (kind != BA_KIND_DEGREE && (scratch_dev == nullptr || (reinterpret_cast<uintptr_t>(scratch_dev) & 15))) {
    set_error("generate/batch tuning needs a 16-byte aligned scratch of 2*(edge_end-edge_begin) int64");
    return BA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool r32 = edge_end <= (1ull << 31);
  const uint64_t node_limit = std::min<uint64_t>(n, 100000);
  void *counter = nullptr, *counts = nullptr, *tab_mem = nullptr;
  ba_status ast = pool_alloc(&counter, 256, s);
  if (ast != BA_OK) return ast;
  if (kind == BA_KIND_DEGREE) {
    ast = pool_alloc(&counts, node_limit * sizeof(uint64_t), s);
    if (ast != BA_OK) {
      cudaFreeAsync(counter, s);
      return ast;
    }
  }
  // A batch of 64 slices of the sample range exercises the batched kernel.
  const int kSlices = 64;
  std::vector<GraphDev> graphs;
  if (kind == BA_KIND_BATCH) {
    const uint64_t step = (len + kSlices - 1) / kSlices;
    for (uint64_t a = edge_begin; a < edge_end; a += step) {
      GraphDev g = make_graph_dev(seed, n, d, n0, a, std::min(edge_end, a + step));
      g.out_edge = a - edge_begin;
      graphs.push_back(g);
    }
    ast = pool_alloc(&tab_mem, graphs.size() * sizeof(GraphDev) + (graphs.size() + 1) * 8, s);
    if (ast != BA_OK) {
      cudaFreeAsync(counter, s);
      return ast;
    }
  }
  const GraphDev g = make_graph_dev(seed, n, d, n0, edge_begin, edge_end);
  float best_ms = 1e30f;
  Shape best = default_shape(kind, r32);
  for (const Shape &cand : candidates(kind)) {
    float ms = 0;
    ba_status cst;
    if (kind == BA_KIND_GENERATE) {
      cst = time_median([&] { return launch_generate(g, scratch_dev, cand,
                                                     static_cast<unsigned long long *>(counter), s); },
                        s, 5, &ms);
    } else if (kind == BA_KIND_DEGREE) {
      cst = time_median([&] { return launch_degree(g, node_limit, static_cast<uint64_t *>(counts), 0,
                                                   cand, static_cast<unsigned long long *>(counter), s); },
                        s, 5, &ms);
    } else {
      // tile prefix depends on the candidate's tile size
      std::vector<GraphDev> gs = graphs;
      std::vector<uint64_t> prefix(gs.size() + 1, 0);
      for (size_t i = 0; i < gs.size(); ++i) {
        gs[i].tile0 = prefix[i];
        prefix[i + 1] = prefix[i] + (gs[i].end - gs[i].begin + cand.tile - 1) / cand.tile;
      }
      GraphDev *dg = static_cast<GraphDev *>(tab_mem);
      uint64_t *dp = reinterpret_cast<uint64_t *>(dg + gs.size());
      cudaMemcpyAsync(dg, gs.data(), gs.size() * sizeof(GraphDev), cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(dp, prefix.data(), prefix.size() * 8, cudaMemcpyHostToDevice, s);
      cudaStreamSynchronize(s);
      BatchTable tab{dg, dp, static_cast<int32_t>(gs.size())};
      cst = time_median([&] { return launch_batch(tab, prefix.back(), r32, n0 > 1, scratch_dev, cand,
                                                  static_cast<unsigned long long *>(counter), s); },
                        s, 5, &ms);
    }
    if (cst == BA_ERR_CUDA) {
      st = cst;
      break;
    }
    if (cst == BA_OK && ms < best_ms) {
      best_ms = ms;
      best = cand;
    }
  }
  cudaFreeAsync(counter, s);
  if (counts) cudaFreeAsync(counts, s);
  if (tab_mem) cudaFreeAsync(tab_mem, s);
  cudaStreamSynchronize(s);
  if (st != BA_OK) return st;
  shape_store(kind, r32, best);
  if (out) to_public(best, out);
  return BA_OK;
}

ba_status ba_tune_save(const char *path) {
  const char *p = path ? path : std::getenv("BA_TUNE_CACHE");
  if (!p || !*p) {
    set_error("no path and BA_TUNE_CACHE is unset");
    return BA_ERR_INVALID_ARG;
  }
  Cache &c = cache();
  std::lock_guard<std::mutex> lock(c.mu);
  FILE *f = std::fopen(p, "w");
  if (!f) {
    set_error("cannot write tuner cache file");
    return BA_ERR_INVALID_ARG;
  }
  std::fprintf(f, "{\"sm_count\": %d, \"entries\": [", sm_count());
  bool firstw = true;
  for (int k = 0; k < kKinds; ++k)
    for (int r = 0; r < 2; ++r) {
      if (!c.has_tuned[k][r]) continue;
      const Shape &s = c.tuned[k][r];
      std::fprintf(f,
                   "%s\n  {\"kind\": %d, \"r32\": %d, \"block\": %d, \"ctas_per_sm\": %d, \"tile\": %d, "
                   "\"refill\": %d, \"hist_bins\": %d, \"hist_agg\": %d, \"chains\": %d}",
                   firstw ? "" : ",", k, r, s.block, s.ctas_per_sm, s.tile, s.refill, s.hist_bins,
                   s.hist_agg, s.chains);
      firstw = false;
    }
  std::fprintf(f, "\n]}\n");
  std::fclose(f);
  return BA_OK;
}

ba_status ba_tune_load(const char *path) {
  const char *p = path ? path : std::getenv("BA_TUNE_CACHE");
  if (!p || !*p) {
    set_error("no path and BA_TUNE_CACHE is unset");
    return BA_ERR_INVALID_ARG;
  }
  Cache &c = cache();
  std::lock_guard<std::mutex> lock(c.mu);
  c.loaded_env = true;
  return load_file(p, c);
}

}  // extern "C"
