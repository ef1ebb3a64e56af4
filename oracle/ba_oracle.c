/*
 * ba_oracle.c -- TEST INFRASTRUCTURE ONLY (the oracle).
 *
 * A plain, slow, single-threaded CPU statement of the Barabasi-Albert edge array of
 * Sanders & Schulz, "Scalable Generation of Scale-free Graphs" (arXiv:1602.07106).
 * Only the test-suite, the benchmark's CPU-baseline leg and the smoke check call it;
 * the library's product path never does.  It shares no code, header, table or constant
 * generator with the CUDA library: every line here is written from the paper's
 * definitions, with no blocking, fusion or reordering.
 *
 * What it computes (paper section 2, the Batagelj-Brandes edge array E):
 *   E[0 .. 2m-1], positions 2i and 2i+1 hold the two end points of edge i.
 *   E[2i]   = the node that edge i belongs to (floor(i/d) for an empty seed graph),
 *   E[2i+1] = E[x], x drawn uniformly from 0..2i by the hash h(2i+1).
 * Section 4 (seed graph): the first m0 edges are the seed network; here it is the clique
 * on nodes 0..n0-1, m0 = n0(n0-1)/2, listed v = 1..n0-1, u = 0..v-1 as edge (v, u).
 * Node n0 + j (j >= 0) then owns edges m0 + j*d .. m0 + (j+1)*d - 1.
 *
 * h(r) (section 2 asks for "a hash function mapping r to a random number in 0..r-1"):
 *   z = SplitMix64 finaliser (Steele, Lea & Flood 2014; Stafford's "Mix13") of
 *       seed XOR (r * 0x9E3779B97F4A7C15 mod 2^64),
 *   h = floor(z * r / 2^64)   (Lemire's multiply-shift reduction to 0..r-1).
 *
 * Variants (the second half of this file): hash_crc of Fig. 3 (CRC-32C of r twice, then
 * the remainder mod r) in place of h, the self-loop-free graph of section 4, where the
 * draw for edge i ranges only over the positions of the edges of earlier nodes, and the
 * graph of section 4 whose nodes reject duplicate targets (no parallel edges).
 *
 * Errors: every entry point returns 0 on success and a negative value when the
 * parameters do not describe a graph (d = 0, n0 > n, n = 0, 2m + 1 >= 2^64, or an
 * edge range outside 0..m).  Buffers belong to the caller.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define ORA_GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL

/* ------------------------------------------------------------------ the hash h(r) -- */

/* SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014). */
static uint64_t splitmix64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    return z;
}

/* The 64 pseudo-random bits drawn for array position r (before range reduction). */
uint64_t ora_hash_bits(uint64_t seed, uint64_t r)
{
    uint64_t x = seed ^ (r * ORA_GOLDEN_GAMMA);
    return splitmix64_mix(x);
}

/* h(r) in 0..r-1 (section 2): the high 64 bits of the 128-bit product z * r. */
uint64_t ora_hash(uint64_t seed, uint64_t r)
{
    u128 product = (u128)ora_hash_bits(seed, r) * (u128)r;
    return (uint64_t)(product >> 64);
}

/* ------------------------------------------------------------ graph parameters -- */

/* Seed-clique edge count m0 = n0(n0-1)/2 (section 4). */
static u128 seed_edges(uint64_t n0)
{
    if (n0 == 0) return 0;
    return ((u128)n0 * (u128)(n0 - 1)) / 2;
}

/* m = m0 + (n - n0) d, or 0 when (n, d, n0) is not a graph or 2m + 1 overflows 64 bits. */
uint64_t ora_num_edges(uint64_t n, uint32_t d, uint64_t n0)
{
    if (n == 0 || d == 0 || n0 > n) return 0;
    u128 m = seed_edges(n0) + (u128)(n - n0) * (u128)d;
    if (m > ((u128)1 << 62)) return 0;
    return (uint64_t)m;
}

/* ------------------------------------------------------ the edge array E (section 2) -- */

/* Value of the seed-clique position p < 2 m0: edge k = p/2 is (v, u) with
 * k = v(v-1)/2 + u, 0 <= u < v; E[2k] = v, E[2k+1] = u.  Found by walking v upwards. */
static int64_t seed_clique_position(uint64_t p)
{
    uint64_t k = p / 2;
    uint64_t v = 1;
    uint64_t first = 0;              /* index of edge (v, 0) */
    while (first + v <= k) {         /* edges (v, 0..v-1) are first .. first+v-1 */
        first += v;
        v += 1;
    }
    uint64_t u = k - first;
    return (p % 2 == 0) ? (int64_t)v : (int64_t)u;
}

/*
 * The Batagelj-Brandes array, written out in full (section 2 and section 4):
 *   E[0 .. 2m0-1] = the seed clique,
 *   for i = m0 .. m-1:  E[2i] = n0 + floor((i - m0)/d);  E[2i+1] = E[h(2i+1)].
 * E must hold 2m int64 values.
 */
int ora_bb_array(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0, int64_t *E)
{
    uint64_t m = ora_num_edges(n, d, n0);
    if (m == 0) return -1;
    uint64_t m0 = (uint64_t)seed_edges(n0);

    uint64_t p = 0;
    for (uint64_t v = 1; v < n0; v++) {
        for (uint64_t u = 0; u < v; u++) {
            E[p] = (int64_t)v;
            E[p + 1] = (int64_t)u;
            p += 2;
        }
    }
    for (uint64_t i = m0; i < m; i++) {
        E[2 * i] = (int64_t)(n0 + (i - m0) / d);
        uint64_t x = ora_hash(seed, 2 * i + 1);   /* uniform in 0..2i */
        E[2 * i + 1] = E[x];
    }
    return 0;
}

/*
 * E[p] from the same definition, without the array: a seed position is looked up, an
 * even position 2j is the owner of edge j, and an odd position q >= 2 m0 holds whatever
 * E[h(q)] holds, so the definition is followed until it reaches one of the first two.
 * This is the recomputation argument of section 2 (Fig. 1 with the section 4 seed graph).
 * *steps (may be NULL) receives the number of hash evaluations, the work counted in the
 * section 2 bound.
 */
static int64_t position_value(uint64_t seed, uint32_t d, uint64_t n0, uint64_t m0,
                              uint64_t p, uint64_t *steps)
{
    uint64_t count = 0;
    for (;;) {
        if (p < 2 * m0) {
            if (steps) *steps = count;
            return seed_clique_position(p);
        }
        if (p % 2 == 0) {
            if (steps) *steps = count;
            return (int64_t)(n0 + (p / 2 - m0) / d);
        }
        p = ora_hash(seed, p);
        count += 1;
    }
}

/* Edges a..b-1 as (E[2i], E[2i+1]) pairs into out[2(b-a)], by the recomputation above. */
int ora_edges_range(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                    uint64_t a, uint64_t b, int64_t *out)
{
    uint64_t m = ora_num_edges(n, d, n0);
    if (m == 0 || a > b || b > m) return -1;
    uint64_t m0 = (uint64_t)seed_edges(n0);
    for (uint64_t i = a; i < b; i++) {
        out[2 * (i - a)] = position_value(seed, d, n0, m0, 2 * i, NULL);
        out[2 * (i - a) + 1] = position_value(seed, d, n0, m0, 2 * i + 1, NULL);
    }
    return 0;
}

/* Number of hash evaluations needed for the second end point of each edge a..b-1. */
int ora_chain_lengths(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                      uint64_t a, uint64_t b, uint64_t *len)
{
    uint64_t m = ora_num_edges(n, d, n0);
    if (m == 0 || a > b || b > m) return -1;
    uint64_t m0 = (uint64_t)seed_edges(n0);
    for (uint64_t i = a; i < b; i++) {
        uint64_t steps = 0;
        position_value(seed, d, n0, m0, 2 * i + 1, &steps);
        len[i - a] = steps;
    }
    return 0;
}

/* ----------------------------------------------------------- degrees (section 3) -- */

/* counts[j] += number of positions p < len with E[p] == j, for j < node_limit. */
void ora_degrees_of_array(const int64_t *E, uint64_t len, uint64_t node_limit,
                          uint64_t *counts)
{
    for (uint64_t p = 0; p < len; p++) {
        if ((uint64_t)E[p] < node_limit) counts[E[p]] += 1;
    }
}

/* counts[j] += number of end points equal to j among edges a..b-1 (a self-loop counts
 * twice), for j < node_limit; the streaming degree analysis of section 3. */
int ora_degree_count_range(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                           uint64_t a, uint64_t b, uint64_t node_limit, uint64_t *counts)
{
    uint64_t m = ora_num_edges(n, d, n0);
    if (m == 0 || a > b || b > m) return -1;
    uint64_t m0 = (uint64_t)seed_edges(n0);
    for (uint64_t i = a; i < b; i++) {
        uint64_t u = (uint64_t)position_value(seed, d, n0, m0, 2 * i, NULL);
        uint64_t v = (uint64_t)position_value(seed, d, n0, m0, 2 * i + 1, NULL);
        if (u < node_limit) counts[u] += 1;
        if (v < node_limit) counts[v] += 1;
    }
    return 0;
}

/* ================================================================================== */
/* Variants of section 4 and Fig. 3.  Written separately from the functions above so  */
/* that the plain array stays exactly as pinned; the plain case is reached again with  */
/* family ORA_HASH_SPLITMIX and no_self_loops = 0.                                     */
/* ================================================================================== */

#define ORA_HASH_SPLITMIX 0
#define ORA_HASH_CRC 1

/*
 * CRC-32C (Castagnoli polynomial x^32 + x^28 + x^27 + ... + 1, 0x1EDC6F41; bit-reflected
 * form 0x82F63B78), advanced over len bytes starting from the running value crc, with no
 * inversion before or after.  This is the update the SSE 4.2 CRC32 instruction performs
 * (Fig. 3 calls it through _mm_crc32_u64).  One bit at a time, least significant first.
 */
uint32_t ora_crc32c_update(uint32_t crc, const uint8_t *p, uint64_t len)
{
    for (uint64_t k = 0; k < len; k++) {
        crc ^= p[k];
        for (int bit = 0; bit < 8; bit++) {
            if (crc & 1u) crc = (crc >> 1) ^ 0x82F63B78u;
            else crc = crc >> 1;
        }
    }
    return crc;
}

/* The 64-bit form: the eight bytes of v in memory (little-endian) order. */
uint32_t ora_crc32c_u64(uint32_t crc, uint64_t v)
{
    uint8_t bytes[8];
    for (int k = 0; k < 8; k++) bytes[k] = (uint8_t)(v >> (8 * k));
    return ora_crc32c_update(crc, bytes, 8);
}

/*
 * The 64 bits hash_crc draws for key r (Fig. 3): CRC32 of r twice with two seeds, the
 * first result in the high half.  Fig. 3 uses the seeds 0 and 1; here they are the low
 * half of the user seed and the high half XOR 1, which is Fig. 3 exactly for seed 0.
 */
uint64_t ora_hash_crc_bits(uint64_t seed, uint64_t r)
{
    uint32_t c0 = (uint32_t)seed;
    uint32_t c1 = (uint32_t)(seed >> 32) ^ 1u;
    uint64_t hash = (uint64_t)ora_crc32c_u64(c0, r) << 32;
    hash += ora_crc32c_u64(c1, r);
    return hash;
}

/*
 * A draw in 0..range-1 for key `key`: the SplitMix64 bits reduced by Lemire's multiply
 * (as h above), or hash_crc's bits reduced by the remainder, as Fig. 3 does.  The plain
 * h(r) is the draw with key = range = r.
 */
uint64_t ora_draw(int family, uint64_t seed, uint64_t key, uint64_t range)
{
    if (family == ORA_HASH_CRC) return ora_hash_crc_bits(seed, key) % range;
    u128 product = (u128)ora_hash_bits(seed, key) * (u128)range;
    return (uint64_t)(product >> 64);
}

/*
 * Range of the draw for the target position q = 2i+1 of edge i >= m0.  Plain: 0..2i, as
 * in section 2.  Without self-loops (section 4: r starts at the first edge of the current
 * node): only the positions of the edges before the first edge f of edge i's node,
 * 0..2f-1, so the target is an earlier node.
 */
static uint64_t draw_range(int no_self_loops, uint32_t d, uint64_t n0, uint64_t m0,
                           uint64_t q)
{
    if (!no_self_loops) return q;
    uint64_t i = q / 2;
    uint64_t node = n0 + (i - m0) / d;
    uint64_t first = m0 + (node - n0) * d;
    return 2 * first;
}

/* The variant parameters describe a graph: the plain checks, a known hash family, and
 * for the self-loop-free graph a seed network with at least one edge (n0 >= 2), since
 * the first new node has nothing else to attach to. */
static int variant_ok(uint64_t n, uint32_t d, uint64_t n0, int family, int no_self_loops)
{
    if (ora_num_edges(n, d, n0) == 0) return 0;
    if (family != ORA_HASH_SPLITMIX && family != ORA_HASH_CRC) return 0;
    if (no_self_loops && n0 < 2) return 0;
    return 1;
}

/*
 * The Batagelj-Brandes array with a variant hash family and, optionally, the section 4
 * self-loop rule:  E[2i] = n0 + floor((i - m0)/d);  E[2i+1] = E[x], x = draw(2i+1, range).
 */
int ora_bb_array_variant(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0, int family,
                         int no_self_loops, int64_t *E)
{
    if (!variant_ok(n, d, n0, family, no_self_loops)) return -1;
    uint64_t m = ora_num_edges(n, d, n0);
    uint64_t m0 = (uint64_t)seed_edges(n0);

    uint64_t p = 0;
    for (uint64_t v = 1; v < n0; v++) {
        for (uint64_t u = 0; u < v; u++) {
            E[p] = (int64_t)v;
            E[p + 1] = (int64_t)u;
            p += 2;
        }
    }
    for (uint64_t i = m0; i < m; i++) {
        E[2 * i] = (int64_t)(n0 + (i - m0) / d);
        uint64_t range = draw_range(no_self_loops, d, n0, m0, 2 * i + 1);
        uint64_t x = ora_draw(family, seed, 2 * i + 1, range);
        E[2 * i + 1] = E[x];
    }
    return 0;
}

/* E[p] of the variant array without the array: the recomputation of section 2, with the
 * variant's draw at every odd position on the way. */
static int64_t variant_position_value(uint64_t seed, uint32_t d, uint64_t n0, uint64_t m0,
                                      int family, int no_self_loops, uint64_t p)
{
    for (;;) {
        if (p < 2 * m0) return seed_clique_position(p);
        if (p % 2 == 0) return (int64_t)(n0 + (p / 2 - m0) / d);
        uint64_t range = draw_range(no_self_loops, d, n0, m0, p);
        p = ora_draw(family, seed, p, range);
    }
}

/* Edges a..b-1 of the variant graph as (E[2i], E[2i+1]) pairs into out[2(b-a)]. */
int ora_edges_range_variant(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                            int family, int no_self_loops, uint64_t a, uint64_t b,
                            int64_t *out)
{
    if (!variant_ok(n, d, n0, family, no_self_loops)) return -1;
    uint64_t m = ora_num_edges(n, d, n0);
    if (a > b || b > m) return -1;
    uint64_t m0 = (uint64_t)seed_edges(n0);
    for (uint64_t i = a; i < b; i++) {
        out[2 * (i - a)] =
            variant_position_value(seed, d, n0, m0, family, no_self_loops, 2 * i);
        out[2 * (i - a) + 1] =
            variant_position_value(seed, d, n0, m0, family, no_self_loops, 2 * i + 1);
    }
    return 0;
}

/* counts[j] += end points equal to j among edges a..b-1 of the variant graph (a
 * self-loop counts twice), for j < node_limit: section 3's analysis on the variant. */
int ora_degree_count_range_variant(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                                   int family, int no_self_loops, uint64_t a, uint64_t b,
                                   uint64_t node_limit, uint64_t *counts)
{
    if (!variant_ok(n, d, n0, family, no_self_loops)) return -1;
    uint64_t m = ora_num_edges(n, d, n0);
    if (a > b || b > m) return -1;
    uint64_t m0 = (uint64_t)seed_edges(n0);
    for (uint64_t i = a; i < b; i++) {
        uint64_t u = (uint64_t)variant_position_value(seed, d, n0, m0, family,
                                                      no_self_loops, 2 * i);
        uint64_t v = (uint64_t)variant_position_value(seed, d, n0, m0, family,
                                                      no_self_loops, 2 * i + 1);
        if (u < node_limit) counts[u] += 1;
        if (v < node_limit) counts[v] += 1;
    }
    return 0;
}

/* ------------------------------------------------ graphs without parallel edges -- */

/*
 * Section 4 avoids parallel edges by keeping the targets already generated for the
 * current node in a table of at most d entries and rejecting a target that is already
 * there.  The paper does not say how a rejected draw is replaced, nor what an odd
 * position reached by a later chain means; the reading taken here:
 *  - A chain resolves every position by the array without rejection (the plain or the
 *    self-loop-free E above): generateEdge's recursion cannot see rejections made while
 *    another node's edges were generated.  Only the output of a node changes.
 *  - Node u >= n0 takes its edges in ID order j = 0..d-1 (edge i = first + j).  The
 *    candidate is E[2i+1].  While it is already among the node's accepted targets, fewer
 *    than REDRAW_CAP redraws were made, and j < reach(u), redraw k (k = 1, 2, ...) draws
 *    x over the same range as the plain draw, keyed by 2i+1, with the SplitMix64 bits of
 *    seed XOR k * REDRAW_SALT, and the candidate becomes E[x].  The candidate left at the
 *    end is the edge's target.
 *  - reach(u) is the number of distinct nodes the draw can reach: with self-loops all of
 *    0..u except an isolated node 0 (n0 = 1), without self-loops the u nodes before u.
 *    A node with d > reach(u) keeps the duplicates beyond its reach (nothing else exists).
 */
#define ORA_REDRAW_SALT 0xD6E8FEB86659FD93ULL
#define ORA_REDRAW_CAP 65536u

static uint64_t distinct_reach(uint64_t node, uint64_t n0, int no_self_loops)
{
    if (no_self_loops) return node;
    return n0 == 1 ? node : node + 1;
}

/* E[p] of the array without rejection, from a stored array or by recomputation. */
struct ora_positions {
    const int64_t *E;  /* NULL: recompute */
    uint64_t seed, n0, m0;
    uint32_t d;
    int no_self_loops;
};

static int64_t position_of(const struct ora_positions *P, uint64_t p)
{
    if (P->E) return P->E[p];
    return variant_position_value(P->seed, P->d, P->n0, P->m0, ORA_HASH_SPLITMIX,
                                  P->no_self_loops, p);
}

static int already_taken(const int64_t *t, uint64_t count, int64_t v)
{
    for (uint64_t l = 0; l < count; l++)
        if (t[l] == v) return 1;
    return 0;
}

/* Targets of the first `count` edges of node `node` (count <= d) under the rule above. */
static void node_targets_simple(const struct ora_positions *P, uint64_t node, uint64_t count,
                                int64_t *t)
{
    uint64_t first = P->m0 + (node - P->n0) * P->d;
    uint64_t reach = distinct_reach(node, P->n0, P->no_self_loops);
    for (uint64_t j = 0; j < count; j++) {
        uint64_t q = 2 * (first + j) + 1;
        int64_t v = position_of(P, q);
        uint32_t k = 0;
        while (j < reach && k < ORA_REDRAW_CAP && already_taken(t, j, v)) {
            k++;
            uint64_t range = draw_range(P->no_self_loops, P->d, P->n0, P->m0, q);
            uint64_t x = ora_draw(ORA_HASH_SPLITMIX, P->seed ^ ((uint64_t)k * ORA_REDRAW_SALT),
                                  q, range);
            v = position_of(P, x);
        }
        t[j] = v;
    }
}

/*
 * The whole graph without parallel edges: out[2m] pairs (source, target).  E (2m int64,
 * caller's workspace) receives the array without rejection that the chains follow.
 */
int ora_edges_simple(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0, int no_self_loops,
                     int64_t *E, int64_t *out)
{
    if (ora_bb_array_variant(seed, n, d, n0, ORA_HASH_SPLITMIX, no_self_loops, E) != 0)
        return -1;
    uint64_t m0 = (uint64_t)seed_edges(n0);
    struct ora_positions P = {E, seed, n0, m0, d, no_self_loops};
    int64_t *t = malloc((size_t)d * sizeof(int64_t));
    if (t == NULL) return -1;
    for (uint64_t i = 0; i < m0; i++) {
        out[2 * i] = E[2 * i];
        out[2 * i + 1] = E[2 * i + 1];
    }
    for (uint64_t node = n0; node < n; node++) {
        uint64_t first = m0 + (node - n0) * d;
        node_targets_simple(&P, node, d, t);
        for (uint64_t j = 0; j < d; j++) {
            out[2 * (first + j)] = (int64_t)node;
            out[2 * (first + j) + 1] = t[j];
        }
    }
    free(t);
    return 0;
}

/* Edges a..b-1 of the graph without parallel edges, without the array: each node that
 * owns an edge in range has its targets recomputed from its first edge on. */
int ora_edges_range_simple(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                           int no_self_loops, uint64_t a, uint64_t b, int64_t *out)
{
    if (!variant_ok(n, d, n0, ORA_HASH_SPLITMIX, no_self_loops)) return -1;
    uint64_t m = ora_num_edges(n, d, n0);
    if (a > b || b > m) return -1;
    uint64_t m0 = (uint64_t)seed_edges(n0);
    struct ora_positions P = {NULL, seed, n0, m0, d, no_self_loops};
    int64_t *t = malloc((size_t)d * sizeof(int64_t));
    if (t == NULL) return -1;
    uint64_t i = a;
    for (; i < b && i < m0; i++) {
        out[2 * (i - a)] = seed_clique_position(2 * i);
        out[2 * (i - a) + 1] = seed_clique_position(2 * i + 1);
    }
    while (i < b) {
        uint64_t node = n0 + (i - m0) / d;
        uint64_t first = m0 + (node - n0) * d;
        uint64_t stop = first + d < b ? first + d : b;
        node_targets_simple(&P, node, stop - first, t);
        for (; i < stop; i++) {
            out[2 * (i - a)] = (int64_t)node;
            out[2 * (i - a) + 1] = t[i - first];
        }
    }
    free(t);
    return 0;
}

/* counts[j] += end points equal to j among edges a..b-1 of the graph without parallel
 * edges (a self-loop counts twice), for j < node_limit. */
int ora_degree_count_range_simple(uint64_t seed, uint64_t n, uint32_t d, uint64_t n0,
                                  int no_self_loops, uint64_t a, uint64_t b,
                                  uint64_t node_limit, uint64_t *counts)
{
    if (!variant_ok(n, d, n0, ORA_HASH_SPLITMIX, no_self_loops)) return -1;
    uint64_t m = ora_num_edges(n, d, n0);
    if (a > b || b > m) return -1;
    int64_t pair[2 * 4096];
    for (uint64_t lo = a; lo < b; lo += 4096) {
        uint64_t hi = b - lo < 4096 ? b : lo + 4096;
        if (ora_edges_range_simple(seed, n, d, n0, no_self_loops, lo, hi, pair) != 0) return -1;
        for (uint64_t k = 0; k < 2 * (hi - lo); k++)
            if ((uint64_t)pair[k] < node_limit) counts[pair[k]] += 1;
    }
    return 0;
}
