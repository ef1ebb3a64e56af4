/*
 * ba.h -- C ABI of libba, GB300-native (sm_103a) Barabasi-Albert edge generation after
 * Sanders & Schulz, "Scalable Generation of Scale-free Graphs" (arXiv:1602.07106).
 *
 * The graph (paper, sections 1, 2 and 4).  Nodes 0..n0-1 form the seed network, here the
 * clique on n0 nodes with m0 = n0(n0-1)/2 edges listed (1,0),(2,0),(2,1),(3,0),... -- edge
 * k = v(v-1)/2 + u is (v, u), u < v.  Every later node n0+j owns d edges, so there are
 * m = m0 + (n-n0) d edges, numbered 0..m-1.  Edge i is the pair (E[2i], E[2i+1]) of the
 * Batagelj-Brandes array: E[2i] is the owning node, n0 + floor((i-m0)/d), and E[2i+1] is
 * E[x] for x = h(2i+1), uniform on 0..2i.  Fig. 1: start at r = 2i+1 and set r := h(r)
 * until r is even (or, with a seed graph, r < 2m0, section 4); the target is then
 * n0 + floor((r/2 - m0)/d) (or the seed clique's entry E[r]).
 *
 * The hash.  Section 2 asks for h(r) mapping a position r to a pseudo-random value in
 * 0..r-1.  libba fixes
 *     h(r) = floor( z * r / 2^64 ),   z = mix(seed XOR (r * 0x9E3779B97F4A7C15 mod 2^64)),
 * mix = the SplitMix64 finaliser (Steele, Lea & Flood 2014):
 *     z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27; z *= 0x94D049BB133111EB; z ^= z>>31.
 * The graph is a pure function of (seed, n, d, n0): any split of the edge range, any
 * launch shape and every entry point below give the same bits (section 2: the graph
 * depends only on the hash, not on the number of processors).
 *
 * Conventions for every call:
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Device work is enqueued on it asynchronously; results are valid once the stream
 *    has reached the call.  Pointers named *_dev / out / counts are device pointers owned
 *    by the caller; libba neither frees nor keeps them, except where a call says so.
 *  - Node IDs are written as int64 (all IDs are < 2^63), edges as (source, target)
 *    pairs, source >= target, in edge-ID order.
 *  - Argument rules: d >= 1, n >= 1, n0 <= n (else BA_ERR_INVALID_ARG); m <= 2^62 (else
 *    BA_ERR_OVERFLOW); edge_begin <= edge_end <= m (else BA_ERR_RANGE); a non-empty
 *    range needs a non-NULL, 16-byte aligned `out` (else BA_ERR_INVALID_ARG).  An empty
 *    range returns BA_OK without touching the device.  A failing CUDA call returns
 *    BA_ERR_CUDA; ba_last_error_message() then gives its text (per thread).
 *  - Calls that take the same output pointer on different streams race; calls on
 *    different streams with different outputs may overlap freely.
 *  - Per-call scratch (a tile counter; staging buffers of ba_generate_edges_host) comes
 *    from a stream-ordered memory pool that libba creates per device on first use and
 *    keeps for the life of the process; it holds on to at most 64 MB between calls, so
 *    repeated small calls do not map device memory each time.
 */
#ifndef BA_H
#define BA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ba_status {
    BA_OK = 0,
    BA_ERR_INVALID_ARG = 1,  /* malformed parameters or pointers */
    BA_ERR_RANGE = 2,        /* edge range outside 0..m */
    BA_ERR_OVERFLOW = 3,     /* m > 2^62, positions would not fit 64 bits */
    BA_ERR_CUDA = 4,         /* a CUDA runtime call failed */
    BA_ERR_NOMEM = 5,        /* device memory (or a server's budget) exhausted */
    BA_ERR_TIMEOUT = 6,      /* a bounded wait ran out */
    BA_ERR_BUSY = 7,         /* not admitted yet (server full); retry later */
    BA_ERR_NOT_FOUND = 8     /* unknown ticket or key */
} ba_status;

/* Text for a status code; never NULL. */
const char *ba_status_string(int status);

/* Text of the last error raised on the calling thread (CUDA error string or a
 * validation message); "" when none.  The pointer stays valid until the next libba call
 * on this thread. */
const char *ba_last_error_message(void);

/* Library version, major*10000 + minor*100 + patch. */
int ba_version(void);

/* Number of device-memory allocations libba has made in this process since it was loaded:
 * every stream-ordered allocation from its pool and every cudaMalloc (batch plans, server
 * arenas and tables).  Lets a caller check that a call allocated nothing. */
uint64_t ba_device_allocations(void);

/* m = n0(n0-1)/2 + (n-n0) d (section 4), or 0 when (n, d, n0) breaks the argument rules
 * or m > 2^62.  A valid graph can have m = 0 too (n = n0 = 1); a call with an empty range,
 * e.g. ba_generate_edges(..., 0, 0, NULL, ...), tells the two apart by its status. */
uint64_t ba_num_edges(uint64_t n, uint32_t d, uint64_t n0);

/*
 * Fig. 1 (generateEdge) for every edge i in [edge_begin, edge_end) of the graph
 * (seed, n, d, n0).  out_dev: 2*(edge_end-edge_begin) int64, 16-byte aligned; edge i is
 * written to out_dev[2(i-edge_begin)] (source) and out_dev[2(i-edge_begin)+1] (target).
 * Runs the persistent warp-refill kernel (tiles handed out dynamically, section 2's
 * batches of edge IDs) with the launch shape from the tuner cache.
 */
ba_status ba_generate_edges(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                            uint64_t edge_begin, uint64_t edge_end,
                            int64_t *out_dev, void *stream);

/*
 * ba_generate_edges with 32-bit node IDs: out_dev holds 2*(edge_end-edge_begin) int32,
 * 8-byte aligned, edge i at out_dev[2(i-edge_begin)] (source) and [...+1] (target); 8 bytes
 * per edge instead of 16 (the paper's remark that 32-bit IDs save time for smaller graphs,
 * section 3).  Needs n <= 2^31 (else BA_ERR_INVALID_ARG); the values equal the int64 call's.
 */
ba_status ba_generate_edges32(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                              uint64_t edge_begin, uint64_t edge_end,
                              int32_t *out_dev, void *stream);

/*
 * Same result as ba_generate_edges, written to HOST memory: host_out holds
 * 2*(edge_end-edge_begin) int64 (pinned memory gives full copy speed; pageable memory
 * works but is slower).  The range is generated in chunks into device staging buffers
 * allocated from the stream's memory pool and copied out while the next chunk is
 * generated.  Returns after the whole result is in host_out (synchronises `stream`).
 */
ba_status ba_generate_edges_host(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                                 uint64_t edge_begin, uint64_t edge_end,
                                 int64_t *host_out, void *stream);

/*
 * Section 3's streaming analysis: the degree (number of end points, a self-loop counting
 * twice) of nodes 0..node_limit-1 over ALL m edges of the graph (seed, n, d) with an
 * empty seed graph (n0 = 0), without storing any edge.  counts_dev: node_limit uint64,
 * 8-byte aligned, overwritten.  node_limit may exceed n (the extra entries are 0);
 * node_limit = 0 is a no-op.
 */
ba_status ba_degree_count(uint64_t seed, uint64_t n, uint32_t d, uint64_t node_limit,
                          uint64_t *counts_dev, void *stream);

/*
 * As ba_degree_count, for the edges [edge_begin, edge_end) of the graph (seed, n, d, n0).
 * accumulate = 0 overwrites counts_dev, accumulate != 0 adds to it, so that the counts
 * of any split of 0..m into ranges sum to the counts of the whole graph.
 */
ba_status ba_degree_count_range(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                                uint64_t edge_begin, uint64_t edge_end,
                                uint64_t node_limit, uint64_t *counts_dev,
                                int accumulate, void *stream);

/*
 * Checked launch (a debug aid in place of a sanitizer): ba_generate_edges with every
 * output store compared with a capacity the caller states, out_capacity_edges edges
 * (16-byte pairs) at out_dev.  A store to a slot at or beyond the capacity is not made;
 * the lowest such slot is kept in *status_dev (device, 8 bytes, caller-owned), which the
 * call first sets to UINT64_MAX ("no violation").  The kernel never traps: read the result
 * with ba_check_status.  Same arguments and errors as ba_generate_edges otherwise; always
 * the refill kernel with the tuned shape; the stored slots hold the same bits as an
 * unchecked call.  Asynchronous on `stream`.
 */
ba_status ba_generate_edges_checked(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                                    uint64_t edge_begin, uint64_t edge_end, int64_t *out_dev,
                                    uint64_t out_capacity_edges, uint64_t *status_dev,
                                    void *stream);

/* Synchronises `stream`, then reads a checked launch's status word: BA_OK when no store
 * went beyond the capacity, else BA_ERR_CUDA with the first offending slot in
 * ba_last_error_message(). */
ba_status ba_check_status(const uint64_t *status_dev, void *stream);

/* ----------------------------------------------------------------------- variants -- */

/* Variants of the graph, as bit flags (0 = the graph of ba_generate_edges):
 *  BA_VARIANT_CRC_HASH       the hash of Fig. 3 (hash_crc) in place of h: CRC-32C of the
 *                            position r (the CRC32 instruction of SSE 4.2: Castagnoli
 *                            polynomial, no inversions, the 8 bytes of r little-endian)
 *                            from two initial values, the first result in the high half
 *                            of 64 bits, then the remainder modulo the draw's range.
 *                            Fig. 3's initial values are 0 and 1; here they are the low
 *                            32 bits of the seed and the high 32 bits XOR 1 (Fig. 3
 *                            exactly for seed 0).
 *  BA_VARIANT_NO_SELF_LOOPS  section 4's self-loop-free graph: the draw for the target of
 *                            edge i (key 2i+1, as before) ranges over the positions of
 *                            the edges before the first edge of edge i's node, so every
 *                            target is an earlier node.  Needs n0 >= 2 (the first new
 *                            node must have a seed edge to attach to).
 *  BA_VARIANT_NO_PARALLEL_EDGES  section 4's rejection of duplicate targets: node u takes
 *                            its d edges in order and an edge whose target one of its
 *                            earlier edges already has draws again -- redraw k over the
 *                            same range, keyed by 2i+1, with the SplitMix64 bits of
 *                            seed XOR k * 0xD6E8FEB86659FD93, then the chain of Fig. 1
 *                            from the drawn position -- until the target is new, as long
 *                            as a new one exists (edge j < reach(u): u+1 nodes, u with
 *                            n0 = 1 or NO_SELF_LOOPS) and for at most 65536 redraws.
 *                            Chains follow the array without rejection, so only the
 *                            node's own output changes.  Needs d <= 1024; combines with
 *                            NO_SELF_LOOPS (a simple graph) but not with CRC_HASH.  For d a
 *                            power of two <= 32 the repeats are found while the edges are
 *                            generated and only the nodes with one are reworked (library
 *                            scratch from the stream-ordered pool: 4 bytes per node listed,
 *                            at most range/64 + 2^20 entries for an edge list and 2^25 for a
 *                            degree count, which stores no edge); for other d a second pass
 *                            reads the written output back, and a degree count generates
 *                            the targets chunk by chunk (2^27 edges, 2 GB of scratch) and
 *                            counts every edge's final target.
 * The flags combine as stated.  Unknown flags, NO_SELF_LOOPS with n0 < 2, or
 * NO_PARALLEL_EDGES outside its limits give BA_ERR_INVALID_ARG. */
#define BA_VARIANT_CRC_HASH 1u
#define BA_VARIANT_NO_SELF_LOOPS 2u
#define BA_VARIANT_NO_PARALLEL_EDGES 4u

/* ba_generate_edges for a variant graph (same arguments, layout and errors, plus the
 * flags).  variant = 0 is ba_generate_edges itself. */
ba_status ba_generate_edges_variant(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                                    uint64_t edge_begin, uint64_t edge_end, uint32_t variant,
                                    int64_t *out_dev, void *stream);

/* ba_degree_count_range for a variant graph (same arguments, layout and errors, plus the
 * flags).  With BA_VARIANT_CRC_HASH and n0 = 0 this is the analysis of section 3 run with
 * the hash of its experiment. */
ba_status ba_degree_count_variant(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                                  uint64_t edge_begin, uint64_t edge_end,
                                  uint64_t node_limit, uint32_t variant,
                                  uint64_t *counts_dev, int accumulate, void *stream);

/* ------------------------------------------------------------------ launch shapes -- */

/* Launch shape of the generate and degree kernels.  Zero fields mean "library default".
 *  block        threads per CTA (multiple of 32, <= 1024)
 *  ctas_per_sm  resident CTAs per SM of the persistent grid
 *  tile         edges per warp tile (power of two, 64..2^20); plain calls halve it,
 *               down to 256, until every warp of the grid gets several tiles
 *  refill       0 = one thread per edge, no refill (the simple kernel);
 *               1 = warp refill every hash step (ballot/popc compaction)
 *  hist_bins    degree kernel: shared-memory histogram bins per CTA
 *  hist_agg     degree kernel: 1 = one shared-memory atomic per distinct node per warp
 *               (__match_any_sync aggregation), 0 = one atomic per hitting lane
 *  chains       refill kernels: hash chains each lane keeps in flight (1 or 2); a
 *               second independent chain hides the latency of the hash's dependent
 *               multiplies */
typedef struct ba_tuning {
    int32_t block;
    int32_t ctas_per_sm;
    int32_t tile;
    int32_t refill;
    int32_t hist_bins;
    int32_t hist_agg;
    int32_t chains;
    int32_t reserved;
} ba_tuning;

/* Kernel families the tuner keys on. */
enum { BA_KIND_GENERATE = 0, BA_KIND_DEGREE = 1, BA_KIND_BATCH = 2 };

/* Overrides the launch shape used for `kind` (NULL restores the tuned/default shape).
 * Output never depends on the shape (tests check this). */
ba_status ba_set_tuning(int32_t kind, const ba_tuning *tune);

/* The shape a call of `kind` would use now for an edge range ending at edge_end. */
ba_status ba_get_tuning(int32_t kind, uint64_t edge_end, ba_tuning *out);

/*
 * Autotuner: times candidate shapes (block size, CTAs/SM, tile, refill, histogram bins and
 * aggregation) for `kind` on the sample range [edge_begin, edge_end) of the graph
 * (seed, n, d, n0) -- for BA_KIND_GENERATE and BA_KIND_BATCH it needs scratch_dev of
 * 2*(edge_end-edge_begin) int64 -- keeps the fastest in the in-process cache (keyed by
 * kind and 32/64-bit position path, the path being that of edge_end) and writes it to
 * out (may be NULL).  Synchronises `stream`.
 */
ba_status ba_tune(int32_t kind, uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                  uint64_t edge_begin, uint64_t edge_end, int64_t *scratch_dev, void *stream,
                  ba_tuning *out);

/* Save / load the tuner cache as JSON text (path NULL = $BA_TUNE_CACHE).  The cache is
 * loaded automatically from $BA_TUNE_CACHE at the first call when that variable is set. */
ba_status ba_tune_save(const char *path);
ba_status ba_tune_load(const char *path);

/* ---------------------------------------------------------- batched generation -- */

/* One graph of a batch: its parameters and the edge range [edge_begin, edge_end) to emit. */
typedef struct ba_graph_desc {
    uint64_t seed;
    uint64_t n;
    uint64_t n0;
    uint64_t edge_begin;
    uint64_t edge_end;
    uint32_t d;
    uint32_t reserved;
} ba_graph_desc;

typedef struct ba_batch_plan ba_batch_plan;

/*
 * Plans one persistent launch over G graphs (section 2's batches of edge IDs, across
 * graphs).  descs (host, G entries) are validated and copied; out_offsets (host, G+1
 * int64, may be NULL = packed) gives where graph g's edges go: graph g's edge
 * edge_begin+k is written to out[2*(out_offsets[g]+k)], and out_offsets must be
 * non-decreasing with out_offsets[g+1]-out_offsets[g] >= edge_end-edge_begin.  The plan
 * owns a device copy of the descriptor table and the per-graph tile prefix, and a CUDA
 * graph of the launch, instantiated on the first ba_batch_plan_launch.
 * tune may be NULL (tuned/default shape for BA_KIND_BATCH).
 */
ba_status ba_batch_plan_create(const ba_graph_desc *descs, int32_t G,
                               const int64_t *out_offsets, const ba_tuning *tune,
                               ba_batch_plan **plan);

/* Total output edges of the plan (= out_offsets[G], or the packed sum). */
uint64_t ba_batch_plan_total_edges(const ba_batch_plan *plan);

/* Copies the plan's G+1 output offsets (in edges) to host memory. */
ba_status ba_batch_plan_offsets(const ba_batch_plan *plan, int64_t *host_offsets);

/* Replays the plan's CUDA graph on `stream`, writing into out_dev (16-byte aligned,
 * 2*total_edges int64).  The first call, and any call with another out_dev, captures the
 * graph again.  Launches of one plan share its tile counter: let one finish before the
 * next starts (same stream, or an event between them). */
ba_status ba_batch_plan_launch(ba_batch_plan *plan, int64_t *out_dev, void *stream);

/* Frees the plan's device tables and graph; cudaFree waits for the device work already
 * enqueued, so a plan may be destroyed right after its last launch. */
ba_status ba_batch_plan_destroy(ba_batch_plan *plan);

/* One-shot form: plan, launch once, destroy.  offsets_host as in ba_batch_plan_create.
 * Its tables come from libba's pool; synchronises `stream` before returning. */
ba_status ba_generate_batch(const ba_graph_desc *descs, int32_t G,
                            const int64_t *offsets_host, int64_t *out_dev,
                            const ba_tuning *tune, void *stream);

/* ------------------------------------------- batched generation without allocation -- */

/*
 * The paper has no counterpart to this call; it is an interface variant for callers that
 * cannot allocate device memory when they want edges -- for example code running while
 * another framework's caching allocator owns all device memory, hosts whose fixed device
 * memory budget forbids hidden allocations, or code that must not risk an allocation
 * failure or the synchronisation an allocation can cause in the middle of its stream.
 *
 * Same result as ba_generate_batch (same arguments, default launch shape), but the call
 * allocates nothing: no cudaMalloc, cudaFree or stream-ordered allocation.  Its scratch
 * (the per-graph constant table, the tile prefix and the tile counter) lives in one static
 * device array of about 114 KB that every GPU loading libba holds until the process exits.
 *  - At most BA_NOALLOC_MAX_GRAPHS graphs per call; a larger G returns BA_ERR_INVALID_ARG.
 *  - The first call on a device (and the first after that device's context was reset)
 *    looks up the array's device address (cudaGetSymbolAddress) with that device current;
 *    make that first call before any stream capture.
 *  - The descriptor table is copied from host memory on `stream`; a copy from pageable
 *    memory waits for the work already on `stream`.  The tile counter is cleared on every
 *    call; the tables are rewritten in full.
 *  - Every call shares the one array and it keeps the previous call's contents: calls whose
 *    device work overlaps (other streams, other host threads) race; serialise them.
 */
#define BA_NOALLOC_MAX_GRAPHS 1024
ba_status ba_generate_batch_noalloc(const ba_graph_desc *descs, int32_t G,
                                    const int64_t *offsets_host, int64_t *out_dev,
                                    void *stream);

/* ------------------------------------------------------------ work-bound counter -- */

/*
 * Section 2's work bound, counted on the device: hist_dev[k] (+)= the number of edges i in
 * [edge_begin, edge_end) whose second end point took k draws h(r) in the chain of Fig. 1
 * (from position 2i+1 until the position is even or, with a seed clique, below 2 m0; 0 for
 * the seed edges themselves), for k < bins-1; hist_dev[bins-1] counts the chains of bins-1
 * draws or more.  bins in 2..1024; hist_dev (device, caller-owned, 8-byte aligned) holds
 * bins uint64 counters, overwritten unless accumulate != 0.  One thread per edge with the
 * plain C form of the hash: a measurement, not a hot path.  Asynchronous on `stream`.
 * Errors as ba_degree_count_range, plus BA_ERR_INVALID_ARG for bins or hist_dev.
 */
ba_status ba_chain_lengths(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                           uint64_t edge_begin, uint64_t edge_end, uint32_t bins,
                           uint64_t *hist_dev, int accumulate, void *stream);

/* ---------------------------------------------------------------- roofline probes -- */

/*
 * Integer floor of the hash chain (section 2's work bound: about two draws per edge).
 * Runs `edges` units of exactly two draws h(r) each -- r = 2(base+e)+1, then the result
 * made odd -- with no stop test, scheduling or stores, `chains` (1, 2 or 4) independent
 * chains per thread, on a full grid.  base + edges <= 2^31 takes the 32-bit-position hash
 * (the one plain calls with edge_end <= 2^31 use), larger bases the 64-bit one.  The XOR
 * of all results is XORed into *sink_dev (device, 8 bytes, caller-owned) so that nothing
 * is optimised away; its value has no other meaning.  Asynchronous on `stream`.
 * Errors: BA_ERR_INVALID_ARG (NULL or misaligned sink, chains not 1/2/4), BA_ERR_RANGE
 * (base + edges >= 2^60), BA_ERR_CUDA.
 */
ba_status ba_probe_hash(uint64_t seed, uint64_t base, uint64_t edges, int32_t chains,
                        uint64_t *sink_dev, void *stream);

/*
 * HBM write bandwidth: 16-byte streaming stores (the generate kernels' store) over
 * dst_dev[0 .. bytes), nothing read; the contents afterwards are unspecified.  dst_dev
 * (device, caller-owned) 16-byte aligned, bytes a multiple of 16, else BA_ERR_INVALID_ARG.
 * Asynchronous on `stream`.
 */
ba_status ba_probe_write(void *dst_dev, uint64_t bytes, void *stream);

/* ------------------------------------------------- serving (continuous batching) -- */

typedef struct ba_server ba_server;

typedef struct ba_server_config {
    uint64_t memory_budget_bytes;  /* device bytes for output buffers (0 = 50% of free) */
    uint64_t chunk_edges;          /* edges per request per tick (0 = 1<<24) */
    int32_t max_active;            /* requests on the device at once (0 = 256; <= 65536) */
    int32_t max_inflight_ticks;    /* ticks enqueued ahead of the GPU (0 = 2; <= 64) */
    int32_t device;                /* CUDA device ordinal (-1 = current) */
    int32_t max_queued;            /* requests waiting for admission (0 = no limit) */
    uint64_t tick_edges;           /* edges per tick over all requests, handed out
                                      shortest remaining request first, while no request
                                      waits for admission (0 = no limit: every running
                                      request gets its chunk each tick) */
} ba_server_config;

typedef struct ba_server_stats {
    uint64_t submitted, admitted, completed, released, rejected_busy;
    uint64_t ticks, edges_done, bytes_in_use, queue_depth, active;
    uint64_t cancelled;
} ba_server_stats;

/* Request states reported by ba_server_poll. */
enum { BA_REQ_QUEUED = 0, BA_REQ_RUNNING = 1, BA_REQ_DONE = 2, BA_REQ_FAILED = 3 };

/*
 * Starts a server: a scheduler thread that admits queued edge-range requests while the
 * memory budget and max_active allow, and on every tick packs the next chunk of every
 * running request into one batched launch (ba_batch plan machinery), so that requests
 * arriving while others run join the next tick.  Output buffers live on the device until
 * ba_server_release.  A config field outside its limits gives BA_ERR_INVALID_ARG.
 */
ba_status ba_server_create(const ba_server_config *cfg, ba_server **server);

/* Queues a request (n0 must be 0 or a clique seed graph like every other call); returns
 * its ticket.  BA_ERR_NOMEM if the request alone exceeds the budget; BA_ERR_BUSY (counted
 * in rejected_busy) if max_queued requests already wait for admission -- retry later. */
ba_status ba_server_submit(ba_server *server, const ba_graph_desc *req, uint64_t *ticket);

/* State (BA_REQ_*) of a ticket and, for DONE, its submit-to-completion latency in
 * nanoseconds (0 in the other states; latency_ns may be NULL). */
ba_status ba_server_poll(ba_server *server, uint64_t ticket, int32_t *state,
                         uint64_t *latency_ns);

/* Blocks until the ticket is DONE (BA_OK) or FAILED (BA_ERR_CUDA) or timeout_ms passes
 * (BA_ERR_TIMEOUT); timeout_ms <= 0 only checks the state once. */
ba_status ba_server_wait(ba_server *server, uint64_t ticket, int64_t timeout_ms);

/* Device pointer and edge count of a DONE request (valid until ba_server_release). */
ba_status ba_server_result(ba_server *server, uint64_t ticket, const int64_t **out_dev,
                           uint64_t *n_edges);

/* Copies a DONE request's 2*n_edges int64 into dst (device or host memory, 16-byte
 * aligned not required) on `stream`; the copy is ordered after the request's work. */
ba_status ba_server_copy_result(ba_server *server, uint64_t ticket, int64_t *dst, void *stream);

/* Frees a finished request's buffer, returning its bytes to the budget. */
ba_status ba_server_release(ba_server *server, uint64_t ticket);

/* Withdraws a request that is still QUEUED (waiting for admission): it is dropped without
 * any device work and its ticket becomes unknown (a later poll, wait or release of it gives
 * BA_ERR_NOT_FOUND).  A RUNNING request cannot be withdrawn -- its chunks may already be on
 * the GPU -- and a DONE or FAILED one is released instead: both give BA_ERR_BUSY.  Unknown
 * tickets give BA_ERR_NOT_FOUND.  Counted in ba_server_stats.cancelled. */
ba_status ba_server_cancel(ba_server *server, uint64_t ticket);

ba_status ba_server_stats_get(ba_server *server, ba_server_stats *stats);

/* Stops the scheduler: the ticks already enqueued finish, no further chunk is issued,
 * queued and unfinished requests are dropped; then frees every buffer, including the
 * results not yet released. */
ba_status ba_server_destroy(ba_server *server);

#ifdef __cplusplus
}
#endif

#endif /* BA_H */
