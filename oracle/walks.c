/*
 * Plain, slow, single-threaded CPU oracle for the random-walk hot path of
 * "Approximating Spanning Centrality with Random Bouquets" (arXiv 2410.14056).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this file; only the tests, the smoke check and the bench's CPU-baseline
 * leg load it.  It shares no code with the CUDA library: the hash, the walk
 * loop, the edge numbering, the planner and the finalize formula are all
 * written out here independently.
 *
 * Build: gcc -O2 -std=c99 -ffp-contract=off -fPIC -shared walks.c -lm
 * (no FMA contraction: the finalize must round each operation separately).
 *
 * Contents and the passages they follow:
 *   philox4x32_10   - Philox-4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw,
 *                     "Parallel random numbers: as easy as 1, 2, 3", SC'11).
 *   splitmix_mix    - the output function of SplitMix64 (Steele, Lea, Flood,
 *                     "Fast splittable pseudorandom number generators",
 *                     OOPSLA'14).
 *   walk key / step hash - the paper's hash-based RNG: one seed per random
 *                     process combined with a hash of the current state
 *                     (vertex, walk length), Sec. 3.1 Eq. (hash_prob) and
 *                     Sec. 3.3 Eq. (select-xor); keyed by walk id, vertex and
 *                     length as in Sec. 2.2.
 *   choose index    - Eq. (select-proposed): floor(r / 2^32 * d), i.e. the
 *                     high word of r * d, no modulus.
 *   walk batch      - Alg. 2 (RandomWalk), one walk after another, visits
 *                     counted as in the synthetic benchmark of Sec. 4.
 *   AESC counters   - the walk loop of Alg. 1 at zero push depth: two walks
 *                     per sample, from each endpoint of the edge, hits of the
 *                     endpoints weighted 2 (steps before tau) and 1 (step tau).
 *   plan            - CalculateTau / NWalks of Alg. 1, which the paper does
 *                     not define; here the spectral truncation bound and
 *                     Hoeffding's inequality (readings listed in the design
 *                     notes), a schedule, or a schedule for tau and a pilot
 *                     sample's variance for N.
 *   finalize        - the estimate s(e) = g(u,v) + g(v,u) of Alg. 1, with
 *                     g initialised to 1/d and incremented by the walk sums.
 *   push phase      - Alg. 1's push step at depth 0 or 1, in fixed point.
 *   shared walks    - the walk loop of Alg. 1 with the walks of a vertex
 *                     serving every query edge at it (vertex-centric walk
 *                     sharing, a neighbour test per step).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOEDGE -4
#define ORC_EOVERFLOW -5

/* Stream reserved for walk-batch walks (AESC streams are 2*edge + side). */
#define ORC_BATCH_STREAM 0x4000000000000000ULL
/* Top stream bit marks the shared (group) key of the coupled sampler. */
#define ORC_GROUP_BIT 0x8000000000000000ULL

/* ---------------------------------------------------------------- hashes */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    int round;
    for (round = 0; round < 10; round++) {
        uint64_t prod0, prod1;
        uint32_t n0, n1, n2, n3;
        if (round > 0) {
            k0 += 0x9E3779B9u; /* Weyl key schedule */
            k1 += 0xBB67AE85u;
        }
        prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
        n1 = (uint32_t)prod1;
        n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
        n3 = (uint32_t)prod0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

static uint64_t splitmix_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* SplitMix64 generator: advance the state by the golden gamma, then mix. */
uint64_t orc_splitmix64_next(uint64_t *state)
{
    *state += 0x9E3779B97F4A7C15ULL;
    return splitmix_mix(*state);
}

/* 64-bit key of walk k in stream s: one Philox block serves walks 2j and
 * 2j+1 (low and high half of its output). */
uint64_t orc_walk_key(uint64_t seed, uint64_t stream, uint64_t k)
{
    uint32_t ctr[4], key[2], out[4];
    uint64_t block = k >> 1;
    ctr[0] = (uint32_t)block;
    ctr[1] = (uint32_t)(block >> 32);
    ctr[2] = (uint32_t)stream;
    ctr[3] = (uint32_t)(stream >> 32);
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
    orc_philox4x32_10(ctr, key, out);
    if (k & 1)
        return (uint64_t)out[2] | ((uint64_t)out[3] << 32);
    return (uint64_t)out[0] | ((uint64_t)out[1] << 32);
}

/* Random word of step l (1-based walk length) taken at vertex cur by the walk
 * whose key is kw: the l-th SplitMix64 state of seed kw, xor the vertex id,
 * mixed; the high 32 bits are kept. */
uint32_t orc_step_hash(uint64_t kw, uint32_t l, uint32_t cur)
{
    uint64_t state = kw + (uint64_t)l * 0x9E3779B97F4A7C15ULL;
    return (uint32_t)(splitmix_mix(state ^ (uint64_t)cur) >> 32);
}

/* Eq. (select-proposed): k = floor(r / 2^32 * d) with r in [0, 2^32). */
uint32_t orc_choose(uint32_t r, uint32_t d)
{
    return (uint32_t)(((uint64_t)r * (uint64_t)d) >> 32);
}

/* Sampler: kind 0 = independent walks; kind 1 = coupled bouquets: walks
 * k with the same floor(k / width) share the top t bits of their random word
 * at the same (length, vertex); kind 2 = the paper's SABA word taken
 * literally (Eq. select-proposed): r = X_W xor h(cur, l), with X_W the low
 * 32 bits of the walk's key (its seed, fixed for the whole walk) and h one
 * hash of (vertex, length) shared by the batch (the group key of walk 0);
 * walk batches only. */
typedef struct {
    uint32_t kind;
    uint32_t t;
    uint32_t width;
} orc_sampler;

static uint32_t sample_word(const orc_sampler *smp, uint64_t kw, uint64_t kg,
                            uint32_t l, uint32_t cur)
{
    uint32_t own;
    if (smp->kind == 2)
        return orc_step_hash(kg, l, cur) ^ (uint32_t)kw;
    own = orc_step_hash(kw, l, cur);
    if (smp->kind == 0)
        return own;
    {
        uint32_t shared = orc_step_hash(kg, l, cur);
        uint32_t mine = smp->t >= 32 ? 0u : (own >> smp->t);
        return shared ^ mine;
    }
}

static int sampler_ok(const orc_sampler *smp)
{
    if (smp->kind == 0)
        return 1;
    if (smp->kind == 2)
        return 1;
    return smp->kind == 1 && smp->width >= 1 && smp->t <= 32;
}

/* ------------------------------------------------------------ walk batch */

/* Alg. 2 for every walk i in input order.  Walk i starts at starts[i]; for
 * l = 1..n_steps it moves to the chosen neighbour of the current vertex (a
 * vertex with no neighbour keeps the walk where it is).  visits[v] is
 * incremented for every position l >= 1 (and l = 0 when include_start) at
 * which the walk stands on v; counts accumulate on top of the caller's
 * values.  paths, when not NULL, receives row i = positions 0..n_steps. */
int orc_walk_batch(uint32_t n, const int64_t *offsets, const uint32_t *nbrs,
                   uint64_t seed, const uint32_t *starts, uint64_t n_walks,
                   uint32_t n_steps, uint32_t kind, uint32_t t, uint32_t width,
                   uint32_t include_start, uint32_t *visits, uint32_t *paths)
{
    orc_sampler smp;
    uint64_t i;
    smp.kind = kind;
    smp.t = t;
    smp.width = width;
    if (!sampler_ok(&smp))
        return ORC_EINVAL;
    for (i = 0; i < n_walks; i++) {
        uint32_t cur = starts[i];
        uint64_t kw, kg = 0;
        uint32_t l;
        if (cur >= n)
            return ORC_EINVAL;
        kw = orc_walk_key(seed, ORC_BATCH_STREAM, i);
        if (kind == 1)
            kg = orc_walk_key(seed, ORC_BATCH_STREAM | ORC_GROUP_BIT, i / width);
        if (kind == 2)
            kg = orc_walk_key(seed, ORC_BATCH_STREAM | ORC_GROUP_BIT, 0);
        if (paths)
            paths[i * ((uint64_t)n_steps + 1)] = cur;
        if (include_start) {
            if (visits[cur] == UINT32_MAX)
                return ORC_EOVERFLOW;
            visits[cur] += 1;
        }
        for (l = 1; l <= n_steps; l++) {
            int64_t lo = offsets[cur];
            uint32_t d = (uint32_t)(offsets[cur + 1] - lo);
            if (d > 0) {
                uint32_t r = sample_word(&smp, kw, kg, l, cur);
                cur = nbrs[lo + orc_choose(r, d)];
            }
            if (visits[cur] == UINT32_MAX)
                return ORC_EOVERFLOW;
            visits[cur] += 1;
            if (paths)
                paths[i * ((uint64_t)n_steps + 1) + l] = cur;
        }
    }
    return ORC_OK;
}

/* The walks with the given batch ids (walk ids[q] starting at starts[q]),
 * positions 0..n_steps written to paths row q: the same walks a batch with
 * those ids would take, for checking sampled walks of a large batch. */
int orc_walk_paths_by_id(uint32_t n, const int64_t *offsets, const uint32_t *nbrs,
                         uint64_t seed, const uint64_t *ids, const uint32_t *starts,
                         uint64_t count, uint32_t n_steps, uint32_t kind, uint32_t t,
                         uint32_t width, uint32_t *paths)
{
    orc_sampler smp;
    uint64_t q;
    smp.kind = kind;
    smp.t = t;
    smp.width = width;
    if (!sampler_ok(&smp))
        return ORC_EINVAL;
    for (q = 0; q < count; q++) {
        uint32_t cur = starts[q];
        uint64_t kw, kg = 0;
        uint32_t l;
        if (cur >= n)
            return ORC_EINVAL;
        kw = orc_walk_key(seed, ORC_BATCH_STREAM, ids[q]);
        if (kind == 1)
            kg = orc_walk_key(seed, ORC_BATCH_STREAM | ORC_GROUP_BIT, ids[q] / width);
        if (kind == 2)
            kg = orc_walk_key(seed, ORC_BATCH_STREAM | ORC_GROUP_BIT, 0);
        paths[q * ((uint64_t)n_steps + 1)] = cur;
        for (l = 1; l <= n_steps; l++) {
            int64_t lo = offsets[cur];
            uint32_t d = (uint32_t)(offsets[cur + 1] - lo);
            if (d > 0)
                cur = nbrs[lo + orc_choose(sample_word(&smp, kw, kg, l, cur), d)];
            paths[q * ((uint64_t)n_steps + 1) + l] = cur;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------- edge numbering */

/* Canonical id of the undirected edge {a, b}: edges are numbered by their
 * lower endpoint u, then by the higher endpoint v, in CSR order.  Returns 0
 * and writes the id, or ORC_ENOEDGE. */
static int edge_id_of(uint32_t n, const int64_t *offsets, const uint32_t *nbrs,
                      const uint64_t *upper_before, uint32_t a, uint32_t b,
                      uint64_t *id)
{
    uint32_t u = a < b ? a : b;
    uint32_t v = a < b ? b : a;
    uint64_t rank = 0;
    int64_t j;
    if (a >= n || b >= n || a == b)
        return ORC_ENOEDGE;
    for (j = offsets[u]; j < offsets[u + 1]; j++) {
        if (nbrs[j] == v) {
            *id = upper_before[u] + rank;
            return ORC_OK;
        }
        if (nbrs[j] > u)
            rank++;
    }
    return ORC_ENOEDGE;
}

/* upper_before[u] = number of edges {x, y}, x < y, with x < u. */
static uint64_t *count_upper(uint32_t n, const int64_t *offsets, const uint32_t *nbrs)
{
    uint64_t *ub = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint32_t u;
    uint64_t acc = 0;
    if (!ub)
        return NULL;
    for (u = 0; u < n; u++) {
        int64_t j;
        ub[u] = acc;
        for (j = offsets[u]; j < offsets[u + 1]; j++)
            if (nbrs[j] > u)
                acc++;
    }
    ub[n] = acc;
    return ub;
}

int orc_edge_ids(uint32_t n, const int64_t *offsets, const uint32_t *nbrs,
                 uint64_t k, const uint32_t *uv, uint64_t *ids)
{
    uint64_t *ub = count_upper(n, offsets, nbrs);
    uint64_t q;
    int rc = ORC_OK;
    if (!ub)
        return ORC_EINVAL;
    for (q = 0; q < k && rc == ORC_OK; q++)
        rc = edge_id_of(n, offsets, nbrs, ub, uv[2 * q], uv[2 * q + 1], &ids[q]);
    free(ub);
    return rc;
}

/* ------------------------------------------------------------ AESC walks */

/* Counters for query edge q = {u, v}, u < v (the pair is normalised), with
 * truncation tau[q] and nwalks[q] samples.  A sample is a walk from u
 * (side 0, stream 2e) and a walk from v (side 1, stream 2e + 1), both with
 * walk index k in [0, nwalks[q]).  At step l = 1..tau the walk adds weight
 * w_l (2 for l < tau, 1 for l = tau) to
 *   side 0:  C_uu if it stands on u,  C_uv if it stands on v
 *   side 1:  C_vu if it stands on u,  C_vv if it stands on v
 * counts[4q + 0..3] = C_uu, C_uv, C_vu, C_vv (overwritten). */
int orc_aesc_counts(uint32_t n, const int64_t *offsets, const uint32_t *nbrs,
                    uint64_t seed, uint64_t k, const uint32_t *uv,
                    const uint32_t *tau, const uint32_t *nwalks, uint32_t kind,
                    uint32_t t, uint32_t width, uint32_t *counts)
{
    orc_sampler smp;
    uint64_t *ub;
    uint64_t q;
    smp.kind = kind;
    smp.t = t;
    smp.width = width;
    if (!sampler_ok(&smp) || kind == 2)  /* the literal SABA word is biased */
        return ORC_EINVAL;
    ub = count_upper(n, offsets, nbrs);
    if (!ub)
        return ORC_EINVAL;
    for (q = 0; q < k; q++) {
        uint32_t a = uv[2 * q], b = uv[2 * q + 1];
        uint32_t u = a < b ? a : b;
        uint32_t v = a < b ? b : a;
        uint64_t e, c[4] = {0, 0, 0, 0};
        uint32_t side;
        if (edge_id_of(n, offsets, nbrs, ub, a, b, &e) != ORC_OK) {
            free(ub);
            return ORC_ENOEDGE;
        }
        for (side = 0; side < 2; side++) {
            uint64_t stream = 2 * e + side;
            uint64_t w;
            for (w = 0; w < nwalks[q]; w++) {
                uint64_t kw = orc_walk_key(seed, stream, w);
                uint64_t kg = 0;
                uint32_t cur = side == 0 ? u : v;
                uint32_t l;
                if (kind == 1)
                    kg = orc_walk_key(seed, stream | ORC_GROUP_BIT, w / width);
                for (l = 1; l <= tau[q]; l++) {
                    int64_t lo = offsets[cur];
                    uint32_t d = (uint32_t)(offsets[cur + 1] - lo);
                    uint32_t weight = l < tau[q] ? 2u : 1u;
                    uint32_t r = sample_word(&smp, kw, kg, l, cur);
                    cur = nbrs[lo + orc_choose(r, d)];
                    if (cur == u)
                        c[2 * side + 0] += weight;
                    if (cur == v)
                        c[2 * side + 1] += weight;
                }
            }
        }
        if (c[0] > UINT32_MAX || c[1] > UINT32_MAX || c[2] > UINT32_MAX || c[3] > UINT32_MAX) {
            free(ub);
            return ORC_EOVERFLOW;
        }
        counts[4 * q + 0] = (uint32_t)c[0];
        counts[4 * q + 1] = (uint32_t)c[1];
        counts[4 * q + 2] = (uint32_t)c[2];
        counts[4 * q + 3] = (uint32_t)c[3];
    }
    free(ub);
    return ORC_OK;
}

/* ------------------------------------------- pilot sample (scheduled plan) */

/* Moments of a pilot sample for query edge q = {u, v}, u < v: the first
 * nwalks[q] walks of each side, i.e. the estimator's own walks (streams
 * 2e + side, walk indices 0.., the same sampler), tau[q] steps each.  Walk w
 * of a side scores a = its weighted hits of u and b = its weighted hits of v
 * (weight 2 at steps l < tau, 1 at l = tau, as in the counters), and
 *   moments[10q + 5 side + 0..4] = sum a, sum b, sum a^2, sum b^2, sum a b
 * over that side's walks (side 0 from u, side 1 from v). */
int orc_aesc_moments(uint32_t n, const int64_t *offsets, const uint32_t *nbrs,
                     uint64_t seed, uint64_t k, const uint32_t *uv,
                     const uint32_t *tau, const uint32_t *nwalks, uint32_t kind,
                     uint32_t t, uint32_t width, uint64_t *moments)
{
    orc_sampler smp;
    uint64_t *ub;
    uint64_t q;
    smp.kind = kind;
    smp.t = t;
    smp.width = width;
    if (!sampler_ok(&smp) || kind == 2)
        return ORC_EINVAL;
    ub = count_upper(n, offsets, nbrs);
    if (!ub)
        return ORC_EINVAL;
    for (q = 0; q < k; q++) {
        uint32_t a = uv[2 * q], b = uv[2 * q + 1];
        uint32_t u = a < b ? a : b;
        uint32_t v = a < b ? b : a;
        uint64_t e;
        uint32_t side;
        if (edge_id_of(n, offsets, nbrs, ub, a, b, &e) != ORC_OK) {
            free(ub);
            return ORC_ENOEDGE;
        }
        if (2ull * nwalks[q] * tau[q] >= 4294967296ull) {
            free(ub);
            return ORC_EOVERFLOW;
        }
        for (side = 0; side < 2; side++) {
            uint64_t stream = 2 * e + side;
            uint64_t w, *mo = moments + 10 * q + 5 * side;
            mo[0] = mo[1] = mo[2] = mo[3] = mo[4] = 0;
            for (w = 0; w < nwalks[q]; w++) {
                uint64_t kw = orc_walk_key(seed, stream, w);
                uint64_t kg = 0, hu = 0, hv = 0;
                uint32_t cur = side == 0 ? u : v;
                uint32_t l;
                if (kind == 1)
                    kg = orc_walk_key(seed, stream | ORC_GROUP_BIT, w / width);
                for (l = 1; l <= tau[q]; l++) {
                    int64_t lo = offsets[cur];
                    uint32_t d = (uint32_t)(offsets[cur + 1] - lo);
                    uint32_t weight = l < tau[q] ? 2u : 1u;
                    uint32_t r = sample_word(&smp, kw, kg, l, cur);
                    cur = nbrs[lo + orc_choose(r, d)];
                    if (cur == u)
                        hu += weight;
                    if (cur == v)
                        hv += weight;
                }
                mo[0] += hu;
                mo[1] += hv;
                mo[2] += hu * hu;
                mo[3] += hv * hv;
                mo[4] += hu * hv;
            }
        }
    }
    free(ub);
    return ORC_OK;
}

/* ------------------------------------- AESC with walks shared per vertex */

/* Stream space of vertex-centric walks: walk w from vertex x has stream
 * ORC_VERTEX_STREAM | x (edge streams 2 e + side stay below 2^61). */
#define ORC_VERTEX_STREAM 0x2000000000000000ULL

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Vertex-centric counters: the walks from a vertex serve every query edge at
 * that vertex (walks shared per vertex, with a neighbour-membership test per
 * step).  Every endpoint x of a query edge runs N_x = max nwalks and
 * tau_x = max tau over the query edges at x: walks w < N_x on stream
 * ORC_VERTEX_STREAM | x, tau_x steps each.  For query q = {u, v}, u < v,
 * with tau_q, each of the N_u walks from u adds weight w_l (2 for l < tau_q,
 * 1 for l = tau_q, nothing beyond) at step l to C_uu when it stands on u and
 * to C_uv when it stands on v; the N_v walks from v likewise to C_vu and C_vv.
 *   counts[4q + 0..3] = C_uu, C_uv, C_vu, C_vv;  nused[2q + 0..1] = N_u, N_v.
 * A repeated edge among the queries is rejected (ORC_EINVAL). */
int orc_aesc_shared_counts(uint32_t n, const int64_t *offsets, const uint32_t *nbrs,
                           uint64_t seed, uint64_t k, const uint32_t *uv,
                           const uint32_t *tau, const uint32_t *nwalks, uint32_t kind,
                           uint32_t t, uint32_t width, uint32_t *counts, uint32_t *nused)
{
    orc_sampler smp;
    uint64_t *ub = NULL, *ids = NULL, *cross = NULL, *qoff = NULL, *qlist = NULL;
    uint32_t *vn = NULL, *vt = NULL;
    uint64_t q, x;
    int rc = ORC_OK;
    smp.kind = kind;
    smp.t = t;
    smp.width = width;
    if (!sampler_ok(&smp) || kind == 2)
        return ORC_EINVAL;
    ub = count_upper(n, offsets, nbrs);
    ids = (uint64_t *)malloc((k + 1) * sizeof(uint64_t));
    cross = (uint64_t *)calloc(2 * k + 1, sizeof(uint64_t));
    qoff = (uint64_t *)calloc((size_t)n + 2, sizeof(uint64_t));
    qlist = (uint64_t *)malloc((2 * k + 1) * sizeof(uint64_t));
    vn = (uint32_t *)calloc((size_t)n + 1, sizeof(uint32_t));
    vt = (uint32_t *)calloc((size_t)n + 1, sizeof(uint32_t));
    if (!ub || !ids || !cross || !qoff || !qlist || !vn || !vt) {
        rc = ORC_EINVAL;
        goto done;
    }
    for (q = 0; q < k; q++) {
        uint32_t a = uv[2 * q], b = uv[2 * q + 1];
        if (edge_id_of(n, offsets, nbrs, ub, a, b, &ids[q]) != ORC_OK) {
            rc = ORC_ENOEDGE;
            goto done;
        }
        if (tau[q] == 0 || nwalks[q] == 0) {
            rc = ORC_EINVAL;
            goto done;
        }
    }
    qsort(ids, k, sizeof(uint64_t), cmp_u64);
    for (q = 1; q < k; q++)
        if (ids[q] == ids[q - 1]) {
            rc = ORC_EINVAL;
            goto done;
        }
    /* per-vertex plan and the list of query edges at each vertex */
    for (q = 0; q < k; q++) {
        uint32_t e[2];
        int s2;
        e[0] = uv[2 * q];
        e[1] = uv[2 * q + 1];
        for (s2 = 0; s2 < 2; s2++) {
            if (nwalks[q] > vn[e[s2]])
                vn[e[s2]] = nwalks[q];
            if (tau[q] > vt[e[s2]])
                vt[e[s2]] = tau[q];
            qoff[e[s2] + 2]++;
        }
    }
    for (x = 0; x < n; x++)
        qoff[x + 2] += qoff[x + 1];
    for (q = 0; q < k; q++) {
        qlist[qoff[uv[2 * q] + 1]++] = q;
        qlist[qoff[uv[2 * q + 1] + 1]++] = q;
    }
    for (q = 0; q < k; q++) {
        uint32_t a = uv[2 * q], b = uv[2 * q + 1];
        uint32_t u = a < b ? a : b, v = a < b ? b : a;
        uint64_t big = vn[u] > vn[v] ? vn[u] : vn[v];
        if (2ull * big * tau[q] >= 4294967296ull) {
            rc = ORC_EOVERFLOW;
            goto done;
        }
        nused[2 * q + 0] = vn[u];
        nused[2 * q + 1] = vn[v];
    }
    for (x = 0; x < n; x++) {
        uint64_t w, j, *ret;
        uint64_t stream = ORC_VERTEX_STREAM | x;
        uint32_t l;
        if (vn[x] == 0)
            continue;
        ret = (uint64_t *)calloc((size_t)vt[x] + 1, sizeof(uint64_t));
        if (!ret) {
            rc = ORC_EINVAL;
            goto done;
        }
        for (w = 0; w < vn[x]; w++) {
            uint64_t kw = orc_walk_key(seed, stream, w);
            uint64_t kg = 0;
            uint32_t cur = (uint32_t)x;
            if (kind == 1)
                kg = orc_walk_key(seed, stream | ORC_GROUP_BIT, w / width);
            for (l = 1; l <= vt[x]; l++) {
                int64_t lo = offsets[cur];
                uint32_t d = (uint32_t)(offsets[cur + 1] - lo);
                uint32_t r = sample_word(&smp, kw, kg, l, cur);
                cur = nbrs[lo + orc_choose(r, d)];
                if (cur == x)
                    ret[l]++;
                for (j = qoff[x]; j < qoff[x + 1]; j++) {
                    uint64_t qq = qlist[j];
                    uint32_t a = uv[2 * qq], b = uv[2 * qq + 1];
                    uint32_t u = a < b ? a : b, v = a < b ? b : a;
                    uint32_t other = x == u ? v : u;
                    if (cur == other && l <= tau[qq])
                        cross[2 * qq + (x == u ? 0 : 1)] += l < tau[qq] ? 2u : 1u;
                }
            }
        }
        /* return hits of x, weighted per query edge by its own tau */
        for (j = qoff[x]; j < qoff[x + 1]; j++) {
            uint64_t qq = qlist[j], c = 0;
            uint32_t a = uv[2 * qq], b = uv[2 * qq + 1];
            uint32_t u = a < b ? a : b;
            for (l = 1; l <= tau[qq]; l++)
                c += (l < tau[qq] ? 2u : 1u) * ret[l];
            if (c > UINT32_MAX) {
                free(ret);
                rc = ORC_EOVERFLOW;
                goto done;
            }
            counts[4 * qq + (x == u ? 0 : 3)] = (uint32_t)c;
        }
        free(ret);
    }
    for (q = 0; q < k; q++) {
        if (cross[2 * q] > UINT32_MAX || cross[2 * q + 1] > UINT32_MAX) {
            rc = ORC_EOVERFLOW;
            goto done;
        }
        counts[4 * q + 1] = (uint32_t)cross[2 * q];
        counts[4 * q + 2] = (uint32_t)cross[2 * q + 1];
    }
done:
    free(ub);
    free(ids);
    free(cross);
    free(qoff);
    free(qlist);
    free(vn);
    free(vt);
    return rc;
}

/* Estimate from the shared counters; the walks of u and of v may differ in
 * number, so each hit count is divided by its own walk count:
 *   est = s_e + ((C_uu/N_u - C_vu/N_v)/d_u + (C_vv/N_v - C_uv/N_u)/d_v) / 2,
 * each operation rounded on its own, in this order. */
int orc_aesc_shared_finalize(uint32_t n, const int64_t *offsets, uint64_t k,
                             const uint32_t *uv, const uint32_t *counts,
                             const uint32_t *nused, double *sc)
{
    uint64_t q;
    for (q = 0; q < k; q++) {
        uint32_t a = uv[2 * q], b = uv[2 * q + 1];
        uint32_t u = a < b ? a : b;
        uint32_t v = a < b ? b : a;
        double du, dv, s, nu, nv, ruu, rvu, rvv, ruv, mean;
        if (u >= n || v >= n || nused[2 * q] == 0 || nused[2 * q + 1] == 0)
            return ORC_EINVAL;
        du = (double)(offsets[u + 1] - offsets[u]);
        dv = (double)(offsets[v + 1] - offsets[v]);
        s = 1.0 / du + 1.0 / dv;
        nu = (double)nused[2 * q];
        nv = (double)nused[2 * q + 1];
        ruu = (double)counts[4 * q + 0] / nu;
        ruv = (double)counts[4 * q + 1] / nu;
        rvu = (double)counts[4 * q + 2] / nv;
        rvv = (double)counts[4 * q + 3] / nv;
        mean = ((ruu - rvu) / du + (rvv - ruv) / dv) / 2.0;
        sc[q] = s + mean;
    }
    return ORC_OK;
}

/* --------------------------------------------------------------- finalize */

/* SC(e) estimate from the four counters:
 *   s_e = 1/d_u + 1/d_v  (the zero-length term; g initialised to 1/d)
 *   est = s_e + ((C_uu - C_vu)/d_u + (C_vv - C_uv)/d_v) / (2 N)
 * Each operation is rounded on its own, in this order. */
int orc_aesc_finalize(uint32_t n, const int64_t *offsets, uint64_t k,
                      const uint32_t *uv, const uint32_t *nwalks,
                      const uint32_t *counts, double *sc)
{
    uint64_t q;
    for (q = 0; q < k; q++) {
        uint32_t a = uv[2 * q], b = uv[2 * q + 1];
        uint32_t u = a < b ? a : b;
        uint32_t v = a < b ? b : a;
        double du, dv, s, x, y, mean;
        if (u >= n || v >= n)
            return ORC_EINVAL;
        du = (double)(offsets[u + 1] - offsets[u]);
        dv = (double)(offsets[v + 1] - offsets[v]);
        s = 1.0 / du + 1.0 / dv;
        x = (double)((int64_t)counts[4 * q + 0] - (int64_t)counts[4 * q + 2]);
        y = (double)((int64_t)counts[4 * q + 3] - (int64_t)counts[4 * q + 1]);
        mean = (x / du + y / dv) / (2.0 * (double)nwalks[q]);
        sc[q] = s + mean;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ plan */

/* ------------------------------------------------ AESC with a push phase */

/* Alg. 1 splits each walk term at push depth tau~: the first tau~ levels of
 * p_l(., v_i) are pushed exactly, and walks of tau - tau~ steps carry the
 * rest, each position y adding p_tau~(y -> x) for target x.  In fixed point
 * with Q = 2^30 the pushed vectors of a source x are
 *   r^0_x = Q e_x,
 *   r^{j+1}_x(y) = sum over neighbours z of y of floor(r^j_x(z) / d(y))
 * (a walk from y is on z one step later with probability 1/d(y); the floors
 * keep every sum exact and order-free), so r^j_x(y) approximates
 * Q p_j(y -> x) from below; r^1_x(y) = floor(Q / d(y)) on the neighbours of x.
 * The push of level j - 1 touches the rows of its support: volume
 * vol_j(x) = sum over j' < j of the degrees of supp r^j'_x (vol_1 = d(x)).
 * As in TGT+'s while loop, the depth is the largest tau~ <= min(push_max,
 * tau, 8) such that every level j <= tau~ has vol_j(u) + vol_j(v) < 2 N
 * (the pushed volume stays below the 2 N walks it replaces) and, when a
 * support cap is given (a planner parameter, not part of TGT+'s rule), for
 * tau~ >= 2 every level 1..tau~ has a support of at most `cap` vertices per
 * side. */
#define ORC_PUSH_Q 1073741824u
#define ORC_PUSH_MAX_DEPTH 8u

/* A sparse vector over the vertices: dense values and the list of nonzero
 * entries (cleared through the list). */
typedef struct {
    uint64_t *val;
    uint32_t *idx;
    uint64_t cnt;
} orc_svec;

static int svec_init(orc_svec *s, uint32_t n)
{
    s->val = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    s->idx = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    s->cnt = 0;
    return s->val && s->idx;
}

static void svec_free(orc_svec *s)
{
    free(s->val);
    free(s->idx);
}

static void svec_clear(orc_svec *s)
{
    uint64_t i;
    for (i = 0; i < s->cnt; i++)
        s->val[s->idx[i]] = 0;
    s->cnt = 0;
}

static void svec_add(orc_svec *s, uint32_t y, uint64_t c)
{
    if (c == 0)
        return;
    if (s->val[y] == 0)
        s->idx[s->cnt++] = y;
    s->val[y] += c;
}

/* The volume of pushing in: the sum of the degrees of its support. */
static uint64_t push_volume(const int64_t *offsets, const orc_svec *in)
{
    uint64_t i, vol = 0;
    for (i = 0; i < in->cnt; i++)
        vol += (uint64_t)(offsets[in->idx[i] + 1] - offsets[in->idx[i]]);
    return vol;
}

/* out = one push of in. */
static void push_level(const int64_t *offsets, const uint32_t *nbrs, const orc_svec *in, orc_svec *out)
{
    uint64_t i;
    svec_clear(out);
    for (i = 0; i < in->cnt; i++) {
        uint32_t z = in->idx[i];
        int64_t j;
        for (j = offsets[z]; j < offsets[z + 1]; j++) {
            uint32_t y = nbrs[j];
            svec_add(out, y, in->val[z] / (uint64_t)(offsets[y + 1] - offsets[y]));
        }
    }
}

typedef struct {
    uint32_t levels;                        /* levels computed: 0..levels */
    uint64_t vol[ORC_PUSH_MAX_DEPTH + 1];   /* vol_j */
    uint64_t supp[ORC_PUSH_MAX_DEPTH + 1];  /* |supp r^j| */
    uint64_t at_u[ORC_PUSH_MAX_DEPTH + 1];  /* r^j(u) */
    uint64_t at_v[ORC_PUSH_MAX_DEPTH + 1];  /* r^j(v) */
} orc_push_stats;

/* Levels 0..jmax of source x; with `limits`, stopping at a level whose
 * volume alone reaches two_n (before pushing it) or after one whose support
 * is above the cap (cap 0: none): no deeper level can be taken then.
 * r^levels_x is left in *a. */
static void push_levels(const int64_t *offsets, const uint32_t *nbrs, uint32_t x, uint32_t u, uint32_t v,
                        uint32_t jmax, int limits, uint64_t two_n, uint32_t cap, orc_svec *a, orc_svec *b,
                        orc_push_stats *st)
{
    uint32_t j;
    svec_clear(a);
    svec_add(a, x, ORC_PUSH_Q);
    st->levels = 0;
    st->vol[0] = 0;
    st->supp[0] = 1;
    st->at_u[0] = a->val[u];
    st->at_v[0] = a->val[v];
    for (j = 1; j <= jmax; j++) {
        orc_svec t;
        st->vol[j] = st->vol[j - 1] + push_volume(offsets, a);
        if (limits && st->vol[j] >= two_n) {
            st->supp[j] = 0;
            st->levels = j;
            break;
        }
        push_level(offsets, nbrs, a, b);
        t = *a;
        *a = *b;
        *b = t;
        st->levels = j;
        st->supp[j] = a->cnt;
        st->at_u[j] = a->val[u];
        st->at_v[j] = a->val[v];
        if (limits && cap && st->supp[j] > cap)
            break;
    }
}

/* Depth of query {u, v} from both sources' level statistics. */
static uint32_t push_depth_from(const orc_push_stats *su, const orc_push_stats *sv, uint64_t two_n,
                                uint32_t cap)
{
    uint32_t j, dep = 0;
    uint32_t top = su->levels < sv->levels ? su->levels : sv->levels;
    for (j = 1; j <= top; j++) {
        if (su->vol[j] + sv->vol[j] >= two_n)
            break;
        if (j >= 2 && cap && (su->supp[j] > cap || sv->supp[j] > cap))
            break;
        dep = j;
    }
    return dep;
}

static uint32_t depth_cap(uint32_t tau, uint32_t push_max)
{
    uint32_t c = push_max < tau ? push_max : tau;
    return c < ORC_PUSH_MAX_DEPTH ? c : ORC_PUSH_MAX_DEPTH;
}

/* The pushed vector r^depth_x as a dense array out[n] (test access). */
int orc_push_vector(uint32_t n, const int64_t *offsets, const uint32_t *nbrs, uint32_t x,
                    uint32_t depth, uint64_t *out)
{
    orc_svec a, b;
    orc_push_stats st;
    uint32_t y;
    if (x >= n || depth > ORC_PUSH_MAX_DEPTH)
        return ORC_EINVAL;
    if (!svec_init(&a, n) || !svec_init(&b, n)) {
        svec_free(&a);
        svec_free(&b);
        return ORC_EINVAL;
    }
    push_levels(offsets, nbrs, x, x, x, depth, 0, 0, 0, &a, &b, &st);
    for (y = 0; y < n; y++)
        out[y] = st.levels == depth ? a.val[y] : 0;
    svec_free(&a);
    svec_free(&b);
    return st.levels == depth ? ORC_OK : ORC_EINVAL;
}

/* Accumulators for query edge q = {u, v}, u < v: the walks of the plain
 * counters (streams 2e + side, walk index w < nwalks[q]) but tau[q] - tau~
 * steps long; at step l the walk adds w * r_u(cur) and w * r_v(cur) with
 * r = r^tau~ and w = 2 if l + tau~ < tau else 1:
 *   acc[4q + 0..3] = A_uu, A_uv (walks from u), A_vu, A_vv (walks from v).
 * depth[q] (may be NULL) receives tau~.  push_max <= 8; support_cap = the
 * largest support per side and level admitted at depths >= 2 (0: no cap). */
int orc_aesc_push_counts(uint32_t n, const int64_t *offsets, const uint32_t *nbrs,
                         uint64_t seed, uint64_t k, const uint32_t *uv,
                         const uint32_t *tau, const uint32_t *nwalks,
                         uint32_t push_max, uint32_t support_cap, uint32_t *depth, uint64_t *acc)
{
    orc_sampler smp;
    orc_svec au, bu, av, bv;
    uint64_t *ub;
    uint64_t q;
    int rc = ORC_OK;
    smp.kind = 0;
    smp.t = 0;
    smp.width = 1;
    if (push_max > ORC_PUSH_MAX_DEPTH)
        return ORC_EINVAL;
    ub = count_upper(n, offsets, nbrs);
    if (!ub || !svec_init(&au, n) || !svec_init(&bu, n) || !svec_init(&av, n) || !svec_init(&bv, n)) {
        free(ub);
        return ORC_EINVAL;
    }
    for (q = 0; q < k && rc == ORC_OK; q++) {
        uint32_t a = uv[2 * q], b = uv[2 * q + 1];
        uint32_t u = a < b ? a : b;
        uint32_t v = a < b ? b : a;
        uint64_t e, c[4] = {0, 0, 0, 0};
        uint32_t side, dep;
        orc_push_stats su, sv;
        if (edge_id_of(n, offsets, nbrs, ub, a, b, &e) != ORC_OK) {
            rc = ORC_ENOEDGE;
            break;
        }
        if (tau[q] == 0 || nwalks[q] == 0 || 2ull * nwalks[q] * tau[q] >= 4294967296ull) {
            rc = ORC_EOVERFLOW;
            break;
        }
        push_levels(offsets, nbrs, u, u, v, depth_cap(tau[q], push_max), 1, 2ull * nwalks[q], support_cap, &au,
                    &bu, &su);
        push_levels(offsets, nbrs, v, u, v, depth_cap(tau[q], push_max), 1, 2ull * nwalks[q], support_cap, &av,
                    &bv, &sv);
        dep = push_depth_from(&su, &sv, 2ull * nwalks[q], support_cap);
        /* the vectors at the chosen depth */
        push_levels(offsets, nbrs, u, u, v, dep, 0, 0, 0, &au, &bu, &su);
        push_levels(offsets, nbrs, v, u, v, dep, 0, 0, 0, &av, &bv, &sv);
        if (depth)
            depth[q] = dep;
        for (side = 0; side < 2; side++) {
            uint64_t stream = 2 * e + side;
            uint64_t w;
            for (w = 0; w < nwalks[q]; w++) {
                uint64_t kw = orc_walk_key(seed, stream, w);
                uint32_t cur = side == 0 ? u : v;
                uint32_t l;
                for (l = 1; l + dep <= tau[q]; l++) {
                    int64_t lo = offsets[cur];
                    uint32_t d = (uint32_t)(offsets[cur + 1] - lo);
                    uint64_t weight = l + dep < tau[q] ? 2u : 1u;
                    cur = nbrs[lo + orc_choose(sample_word(&smp, kw, 0, l, cur), d)];
                    c[2 * side + 0] += weight * au.val[cur];
                    c[2 * side + 1] += weight * av.val[cur];
                }
            }
        }
        acc[4 * q + 0] = c[0];
        acc[4 * q + 1] = c[1];
        acc[4 * q + 2] = c[2];
        acc[4 * q + 3] = c[3];
    }
    free(ub);
    svec_free(&au);
    svec_free(&bu);
    svec_free(&av);
    svec_free(&bv);
    return rc;
}

/* Estimate of query edge q from its accumulators:
 *   g(u, v) = (X_u + (A_uu - A_vu) / N) / (2 Q d_u),
 *   X_u = sum over l = 0..tau~ of w_l (r^l_u(u) - r^l_u(v)),
 * the series' terms below the push depth and the walks' fixed start, with
 * w_l = 2 if l < tau else 1 (tau~ = 0: X_u = 2Q; tau~ = 1: X_u = 2Q -
 * w_1 floor(Q / d_v)); g(v, u) likewise with X_v = sum w_l (r^l_v(v) -
 * r^l_v(u)); SC = g(u, v) + g(v, u).  Each FP64 operation rounds once, in
 * this order. */
int orc_aesc_push_finalize(uint32_t n, const int64_t *offsets, const uint32_t *nbrs, uint64_t k,
                           const uint32_t *uv, const uint32_t *tau, const uint32_t *nwalks,
                           const uint32_t *depth, const uint64_t *acc, double *sc)
{
    orc_svec a, b;
    uint64_t q;
    int rc = ORC_OK;
    if (!svec_init(&a, n) || !svec_init(&b, n)) {
        svec_free(&a);
        svec_free(&b);
        return ORC_EINVAL;
    }
    for (q = 0; q < k; q++) {
        uint32_t x = uv[2 * q], y = uv[2 * q + 1];
        uint32_t u = x < y ? x : y;
        uint32_t v = x < y ? y : x;
        uint32_t l;
        int64_t xu = 0, xv = 0;
        double du, dv, nw, gu, gv;
        orc_push_stats su, sv;
        if (u >= n || v >= n || depth[q] > ORC_PUSH_MAX_DEPTH || depth[q] > tau[q]) {
            rc = ORC_EINVAL;
            break;
        }
        push_levels(offsets, nbrs, u, u, v, depth[q], 0, 0, 0, &a, &b, &su);
        push_levels(offsets, nbrs, v, u, v, depth[q], 0, 0, 0, &a, &b, &sv);
        for (l = 0; l <= depth[q]; l++) {
            int64_t w = l < tau[q] ? 2 : 1;
            xu += w * ((int64_t)su.at_u[l] - (int64_t)su.at_v[l]);
            xv += w * ((int64_t)sv.at_v[l] - (int64_t)sv.at_u[l]);
        }
        du = (double)(offsets[u + 1] - offsets[u]);
        dv = (double)(offsets[v + 1] - offsets[v]);
        nw = (double)nwalks[q];
        gu = ((double)xu + (double)(int64_t)(acc[4 * q + 0] - acc[4 * q + 2]) / nw) /
             (2.0 * (double)ORC_PUSH_Q * du);
        gv = ((double)xv + (double)(int64_t)(acc[4 * q + 3] - acc[4 * q + 1]) / nw) /
             (2.0 * (double)ORC_PUSH_Q * dv);
        sc[q] = gu + gv;
    }
    svec_free(&a);
    svec_free(&b);
    return rc;
}


/* Worst-case truncation error factor of the half-weighted series after tau
 * terms for eigenvalues in (0, lambda2] (P) and [lambda_neg, 0) (Q), where
 * the error of one eigen-component lambda is lambda^tau (1 + lambda) /
 * (2 (1 - lambda)) times its weight, and the weights sum to s_e. */
static double trunc_p(double lambda2, uint32_t tau)
{
    if (lambda2 <= 0.0)
        return 0.0;
    return pow(lambda2, (double)tau) * (1.0 + lambda2) / (2.0 * (1.0 - lambda2));
}

static double trunc_q(double lambda_neg, uint32_t tau)
{
    double a = -lambda_neg, xs, x;
    if (a <= 0.0)
        return 0.0;
    /* x^tau (1-x)/(1+x) on [0, 1) peaks at the positive root of
     * tau x^2 + 2x - tau = 0. */
    xs = (sqrt(1.0 + (double)tau * (double)tau) - 1.0) / (double)tau;
    x = a < xs ? a : xs;
    return pow(x, (double)tau) * (1.0 - x) / (2.0 * (1.0 + x));
}

double orc_trunc_bound(double s_e, double lambda2, double lambda_neg, uint32_t tau)
{
    double p = trunc_p(lambda2, tau), q = trunc_q(lambda_neg, tau);
    return s_e * (p > q ? p : q);
}

/* Truncation bound with omega known eigenpairs (the eigenvector refinement
 * of CalculateTau in Alg. 1).  lambdas[0..omega) are the largest eigenvalues
 * of D^-1/2 A D^-1/2 after the eigenvalue 1, with unit eigenvectors psi_k;
 * vecs[v * omega + k] = psi_k(v) / sqrt(d(v)).  For the edge {u, v},
 * c_k = vecs[u, k] - vecs[v, k] and the known modes' error is exact:
 *   E(tau) = sum_k c_k^2 lambda_k^tau (1 + lambda_k) / (2 (1 - lambda_k));
 * the modes not given carry the rest of s_e = sum of all c_k^2, and each has
 * an eigenvalue in [lambda_neg, lambda_rest] (or exactly -1, whose term is
 * zero), so
 *   |R - S_tau| <= |E(tau)| + max(0, s_e - sum_k c_k^2) max(P(tau), Q(tau))
 * with P taken at lambda_rest and Q at lambda_neg. */
double orc_trunc_bound_omega(double s_e, uint32_t omega, const double *lambdas, const double *cu,
                             const double *cv, double lambda_rest, double lambda_neg, uint32_t tau)
{
    double known = 0.0, mass = 0.0, rest, p, q;
    uint32_t j;
    for (j = 0; j < omega; j++) {
        double c = cu[j] - cv[j], l = lambdas[j];
        known += c * c * pow(l, (double)tau) * (1.0 + l) / (2.0 * (1.0 - l));
        mass += c * c;
    }
    rest = s_e - mass;
    if (rest < 0.0)
        rest = 0.0;
    p = trunc_p(lambda_rest, tau);
    q = trunc_q(lambda_neg, tau);
    return fabs(known) + rest * (p > q ? p : q);
}

/* The certified plan with that bound for tau (N as orc_plan_certified). */
int orc_plan_certified_omega(uint32_t n, const int64_t *offsets, const uint32_t *nbrs,
                             uint64_t k, const uint32_t *uv, double eps, double delta,
                             uint32_t omega, const double *lambdas, const double *vecs,
                             double lambda_rest, double lambda_neg, uint32_t tau_max,
                             uint32_t *tau, uint32_t *nwalks)
{
    uint64_t m = (uint64_t)(offsets[n] / 2);
    uint64_t *ub, q, id;
    double logterm;
    if (!(eps > 0.0) || !(delta > 0.0) || !(delta < 1.0) || m == 0 || (omega && (!lambdas || !vecs)))
        return ORC_EINVAL;
    ub = count_upper(n, offsets, nbrs);
    if (!ub)
        return ORC_EINVAL;
    logterm = log(2.0 * (double)m / delta);
    for (q = 0; q < k; q++) {
        uint32_t a = uv[2 * q], b = uv[2 * q + 1];
        double du, dv, s, nw, h;
        uint32_t tq = 1;
        if (edge_id_of(n, offsets, nbrs, ub, a, b, &id) != ORC_OK) {
            free(ub);
            return ORC_ENOEDGE;
        }
        du = (double)(offsets[a + 1] - offsets[a]);
        dv = (double)(offsets[b + 1] - offsets[b]);
        s = 1.0 / du + 1.0 / dv;
        while (orc_trunc_bound_omega(s, omega, lambdas, vecs + (uint64_t)a * omega, vecs + (uint64_t)b * omega,
                                     lambda_rest, lambda_neg, tq) > eps / 2.0) {
            if (tq >= tau_max) {
                free(ub);
                return ORC_EOVERFLOW;
            }
            tq++;
        }
        h = (double)tq - 0.5;
        nw = ceil(8.0 * h * h * s * s * logterm / (eps * eps));
        if (nw < 1.0)
            nw = 1.0;
        if (nw * 2.0 * (double)tq >= 4294967296.0) {
            free(ub);
            return ORC_EOVERFLOW;
        }
        tau[q] = tq;
        nwalks[q] = (uint32_t)nw;
    }
    free(ub);
    return ORC_OK;
}

/* Scheduled (uncertified) plan, for graphs on which the certified bounds
 * explode (slow mixing):
 *   tau = clamp(ceil(tau_scale * ln(s_e / eps)) + tau_add, 1, tau_max)
 *         (the ln term counted only when s_e > eps),
 *   N   = max(n_min, ceil(n_scale * s_e^2 / eps^2), 1).
 * The ln(s_e / eps) form follows the truncation error s_e * lambda^tau of the
 * half-weighted series; N follows a sample variance of order s_e^2.
 * Returns ORC_EOVERFLOW when 2 N tau >= 2^32. */
int orc_plan_scheduled(uint32_t n, const int64_t *offsets, const uint32_t *nbrs,
                       uint64_t k, const uint32_t *uv, double eps, double tau_scale,
                       uint32_t tau_add, uint32_t tau_max, double n_scale, uint32_t n_min,
                       uint32_t *tau, uint32_t *nwalks)
{
    uint64_t *ub, q, id;
    if (!(eps > 0.0) || tau_max < 1 || !(tau_scale >= 0.0) || !(n_scale >= 0.0))
        return ORC_EINVAL;
    ub = count_upper(n, offsets, nbrs);
    if (!ub)
        return ORC_EINVAL;
    for (q = 0; q < k; q++) {
        uint32_t a = uv[2 * q], b = uv[2 * q + 1];
        double du, dv, s, t, nw;
        if (edge_id_of(n, offsets, nbrs, ub, a, b, &id) != ORC_OK) {
            free(ub);
            return ORC_ENOEDGE;
        }
        du = (double)(offsets[a + 1] - offsets[a]);
        dv = (double)(offsets[b + 1] - offsets[b]);
        s = 1.0 / du + 1.0 / dv;
        t = 0.0;
        if (s / eps > 1.0)
            t = ceil(tau_scale * log(s / eps));
        t = t + (double)tau_add;
        if (t < 1.0)
            t = 1.0;
        if (t > (double)tau_max)
            t = (double)tau_max;
        nw = ceil(n_scale * s * s / (eps * eps));
        if (nw < (double)n_min)
            nw = (double)n_min;
        if (nw < 1.0)
            nw = 1.0;
        if (nw * 2.0 * t >= 4294967296.0) {
            free(ub);
            return ORC_EOVERFLOW;
        }
        tau[q] = (uint32_t)t;
        nwalks[q] = (uint32_t)nw;
    }
    free(ub);
    return ORC_OK;
}

/* x - y of two unsigned integers as a double (the exact difference, rounded
 * once). */
static double signed_diff(uint64_t x, uint64_t y)
{
    return x >= y ? (double)(x - y) : -(double)(y - x);
}

/* Walk count of the pilot plan from the moments of orc_aesc_moments with
 * n0 pilot walks per side.  One sample of the estimator is the pair of walk
 * w from u (U) and walk w from v (V), and the estimate is s_e plus the mean
 * over samples of
 *   Y = ((a(U) - a(V)) / d_u + (b(V) - b(U)) / d_v) / 2
 *     = ((a/d_u - b/d_v)(U) - (a/d_u - b/d_v)(V)) / 2.
 * U and V are independent, so Var Y = (Var_0 + Var_1) / 4 with
 * Var_s = Var(a)/d_u^2 + Var(b)/d_v^2 - 2 Cov(a, b)/(d_u d_v) on side s.
 * The unbiased sample (co)variances are C / (n0 (n0 - 1)) with the integer
 * centred sums C_aa = n0 S_aa - S_a^2, C_bb = n0 S_bb - S_b^2 and
 * C_ab = n0 S_ab - S_a S_b, exact in 64 bits while 2 n0 tau < 2^32.  In FP64,
 * one rounding per operation in this order:
 *   caa = C_aa,0 + C_aa,1   cbb = C_bb,0 + C_bb,1   cab = C_ab,0 + C_ab,1
 *   var = ((caa / (d_u d_u) + cbb / (d_v d_v)) - (2 cab) / (d_u d_v))
 *         / ((4 n0) (n0 - 1)),   clamped at 0
 *   N   = max(ceil((z z var) / ((eps/2) (eps/2))), n_min, 1)
 * i.e. the normal-approximation half-width z sqrt(Var Y / N) is at most
 * eps / 2.  var_out (may be NULL) receives var.  Returns ORC_EOVERFLOW when
 * 2 N tau >= 2^32. */
int orc_plan_pilot_nwalks(uint32_t n, const int64_t *offsets, uint64_t k,
                          const uint32_t *uv, const uint32_t *tau,
                          const uint64_t *moments, uint32_t n0, double eps,
                          double z, uint32_t n_min, uint32_t *nwalks,
                          double *var_out)
{
    uint64_t q;
    if (n0 < 2 || !(eps > 0.0) || !(z > 0.0))
        return ORC_EINVAL;
    for (q = 0; q < k; q++) {
        uint32_t a = uv[2 * q], b = uv[2 * q + 1];
        double du, dv, caa = 0.0, cbb = 0.0, cab = 0.0, var, half, nw;
        uint32_t side;
        if (a >= n || b >= n)
            return ORC_EINVAL;
        du = (double)(offsets[(a < b ? a : b) + 1] - offsets[a < b ? a : b]);
        dv = (double)(offsets[(a < b ? b : a) + 1] - offsets[a < b ? b : a]);
        for (side = 0; side < 2; side++) {
            const uint64_t *mo = moments + 10 * q + 5 * side;
            caa = caa + signed_diff((uint64_t)n0 * mo[2], mo[0] * mo[0]);
            cbb = cbb + signed_diff((uint64_t)n0 * mo[3], mo[1] * mo[1]);
            cab = cab + signed_diff((uint64_t)n0 * mo[4], mo[0] * mo[1]);
        }
        var = ((caa / (du * du) + cbb / (dv * dv)) - (2.0 * cab) / (du * dv)) /
              ((4.0 * (double)n0) * ((double)n0 - 1.0));
        if (var < 0.0)
            var = 0.0;
        half = eps / 2.0;
        nw = ceil((z * z * var) / (half * half));
        if (nw < (double)n_min)
            nw = (double)n_min;
        if (nw < 1.0)
            nw = 1.0;
        if (var_out)
            var_out[q] = var;
        if (nw * 2.0 * (double)tau[q] >= 4294967296.0)
            return ORC_EOVERFLOW;
        nwalks[q] = (uint32_t)nw;
    }
    return ORC_OK;
}

/* Certified plan for each query edge:
 *   tau = smallest tau >= 1 with s_e * max(P(tau), Q(tau)) <= eps / 2
 *   N   = ceil(8 (tau - 1/2)^2 s_e^2 ln(2 m / delta) / eps^2)
 * (Hoeffding on samples bounded by (tau - 1/2) s_e in absolute value,
 * deviation eps/2, failure delta/m per edge, m = edges of the whole graph).
 * Returns ORC_EOVERFLOW when tau exceeds tau_max or 2 N tau >= 2^32. */
int orc_plan_certified(uint32_t n, const int64_t *offsets, const uint32_t *nbrs,
                       uint64_t k, const uint32_t *uv, double eps, double delta,
                       double lambda2, double lambda_neg, uint32_t tau_max,
                       uint32_t *tau, uint32_t *nwalks)
{
    uint64_t m = (uint64_t)(offsets[n] / 2);
    uint64_t *ub, q, id;
    double logterm;
    if (!(eps > 0.0) || !(delta > 0.0) || !(delta < 1.0) || m == 0)
        return ORC_EINVAL;
    ub = count_upper(n, offsets, nbrs);
    if (!ub)
        return ORC_EINVAL;
    logterm = log(2.0 * (double)m / delta);
    for (q = 0; q < k; q++) {
        uint32_t a = uv[2 * q], b = uv[2 * q + 1];
        double du, dv, s, nw, h;
        uint32_t tq = 1;
        if (edge_id_of(n, offsets, nbrs, ub, a, b, &id) != ORC_OK) {
            free(ub);
            return ORC_ENOEDGE;
        }
        du = (double)(offsets[a + 1] - offsets[a]);
        dv = (double)(offsets[b + 1] - offsets[b]);
        s = 1.0 / du + 1.0 / dv;
        while (orc_trunc_bound(s, lambda2, lambda_neg, tq) > eps / 2.0) {
            if (tq >= tau_max) {
                free(ub);
                return ORC_EOVERFLOW;
            }
            tq++;
        }
        h = (double)tq - 0.5;
        nw = ceil(8.0 * h * h * s * s * logterm / (eps * eps));
        if (nw < 1.0)
            nw = 1.0;
        if (nw * 2.0 * (double)tq >= 4294967296.0) {
            free(ub);
            return ORC_EOVERFLOW;
        }
        tau[q] = tq;
        nwalks[q] = (uint32_t)nw;
    }
    free(ub);
    return ORC_OK;
}
