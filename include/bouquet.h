/*
 * bouquet.h - C ABI of the GB300 random-walk spanning-centrality library.
 *
 * The library implements the walk hot path of "Approximating Spanning
 * Centrality with Random Bouquets" (arXiv 2410.14056): hash-keyed neighbour
 * sampling (Sec. 3.1, Sec. 3.3 Eq. select-proposed), walks advanced in
 * lockstep bouquets (Alg. 3), visit counting (Sec. 4), and the walk loop of
 * TGT+ (Alg. 1) turned into per-edge hit counters and an FP64 estimate of
 * spanning centrality SC(e) = R_eff(u, v) (Sec. 2.1) to absolute error eps
 * (the eps-approximation problem of Sec. 2.1).
 *
 * Conventions for every call:
 *   - Return value: BQ_OK (0) or a negative BQ_E* code.  A failed call leaves
 *     a message readable with bq_last_error() on the calling thread.
 *   - Pointers suffixed _dev are device pointers on the graph's device; other
 *     array pointers are host pointers unless a flag says otherwise.
 *   - Calls taking a stream enqueue their work on it (a CUDA stream handle,
 *     cudaStream_t passed as void*; NULL = the legacy default stream) and
 *     return without waiting, unless BQ_HOST_IO is given.  Errors found by
 *     the kernels are recorded in a per-device status word and returned by
 *     bq_sync().
 *   - The library never reads or writes caller memory after a call returns,
 *     except the device buffers of asynchronous calls, which the caller must
 *     keep alive until the stream reaches the call.
 *   - Vertex ids are uint32, CSR offsets int64; a graph is undirected and
 *     unweighted: symmetric CSR, rows sorted increasingly, no self-loops, no
 *     duplicate entries.
 */
#ifndef BOUQUET_H
#define BOUQUET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define BQ_OK 0
#define BQ_EINVAL (-1)    /* bad argument (null pointer, size, flag, range) */
#define BQ_ENOMEM (-2)    /* device or host allocation failed */
#define BQ_EGRAPH (-3)    /* graph rejected by validation (message says why) */
#define BQ_ENOEDGE (-4)   /* a queried vertex pair is not an edge */
#define BQ_EOVERFLOW (-5) /* a uint32 counter would wrap, or tau too large */
#define BQ_ETIMEOUT (-6)  /* a bounded device wait gave up */
#define BQ_EBUSY (-7)     /* admission refused: not enough free memory/slots */
#define BQ_ECUDA (-8)     /* a CUDA runtime call failed (message has it) */

/* ------------------------------------------------------- bq_graph_create */
#define BQ_HOST_PTRS 0x0u         /* offsets / nbrs are host pointers */
#define BQ_DEVICE_PTRS 0x1u       /* offsets / nbrs are device pointers */
#define BQ_BORROW 0x2u            /* with BQ_DEVICE_PTRS: use the caller's
                                     buffers in place, no copy; they must stay
                                     alive and unchanged until destroy */
#define BQ_SKIP_VALIDATE 0x4u     /* skip the symmetry and sortedness checks
                                     (bounds of offsets and ids are always
                                     checked, so no kernel can read outside
                                     the arrays) */
#define BQ_REQUIRE_CONNECTED 0x8u /* reject a graph with more than one
                                     connected component */

typedef struct bq_graph bq_graph;

/*
 * Load an undirected graph (the notation of Sec. 2: Gamma(v) = row v of the
 * CSR, d(v) = its length).  n vertices, offsets[n + 1] (int64, offsets[0] =
 * 0, non-decreasing), nbrs[offsets[n]] (uint32 ids < n).  The library builds
 * its device-side derived arrays (per-vertex records of row offset and
 * degree, the canonical edge numbering) on `cuda_stream` and synchronises
 * that stream before returning.  Validation failures return BQ_EGRAPH with a
 * message naming the first bad vertex.  On success *out owns the device
 * memory it allocated; release it with bq_graph_destroy.
 */
int bq_graph_create(uint32_t n, const int64_t *offsets, const uint32_t *nbrs,
                    uint32_t flags, void *cuda_stream, bq_graph **out);

/* Free a graph and everything it owns (not borrowed buffers).  NULL is a no-op.
 * The caller must not destroy a graph while work using it is in flight. */
int bq_graph_destroy(bq_graph *g);

typedef struct bq_graph_info_t {
    uint64_t n;            /* vertices */
    uint64_t m;            /* undirected edges (nnz / 2) */
    uint64_t nnz;          /* CSR entries */
    uint32_t min_degree;
    uint32_t max_degree;
    int32_t bipartite;     /* 1 / 0 (computed on first request) */
    int32_t n_components;  /* connected components, isolated vertices included */
    uint64_t device_bytes; /* device memory owned by the graph */
    int32_t has_spectrum;  /* bq_graph_set_spectrum was called */
    int32_t device;        /* CUDA device ordinal */
    double lambda2;        /* as set by bq_graph_set_spectrum */
    double lambda_neg;
    int32_t layout;        /* device layout built (bq_tuning.layout value, never 1) */
    int32_t reserved;
    /* What the walk batch's kernels will use on this graph (set at creation):
     * hub_slots      slots of the hashed hub table (0: none);
     * packed_bits    bits per packed neighbour id (0: ids not packed);
     * relabel_hubs   vertices the kernel on the degree-relabelled copy serves
     *                from shared memory (0: no relabelled copy was built);
     * relabel_bits_* field widths of the copy's 8-byte vertex records
     *                {original id, row offset, degree} (0 without a copy). */
    uint32_t hub_slots;
    uint32_t packed_bits;
    uint32_t relabel_hubs;
    uint32_t relabel_bits_id;
    uint32_t relabel_bits_off;
    uint32_t relabel_bits_deg;
} bq_graph_info_t;

/* Fill *info (host struct).  May copy the CSR to the host once to find the
 * bipartite flag and the component count. */
int bq_graph_info(bq_graph *g, bq_graph_info_t *info);

/*
 * Spectral inputs of the certified planner: eigenvalues of
 * D^-1/2 A D^-1/2, the matrix whose eigenpairs CalculateTau uses (Sec. 2.3).
 * lambda2 = second-largest eigenvalue (< 1 for a connected graph);
 * lambda_neg = the most negative eigenvalue once one exact -1 is removed for
 * a bipartite graph (0.0 when none is left).  Requires -1 <= lambda_neg <= 0
 * and lambda2 < 1.
 */
int bq_graph_set_spectrum(bq_graph *g, double lambda2, double lambda_neg);

/*
 * Eigenvector refinement of the certified plan (CalculateTau's use of the
 * top eigenvectors, Alg. 1 and Sec. 2.3): the omega largest eigenvalues of
 * D^-1/2 A D^-1/2 after the eigenvalue 1 (lambdas, host, omega doubles), their
 * unit eigenvectors divided by sqrt(d(v)) (vecs, host, n * omega doubles,
 * vecs[v * omega + k]), and lambda_rest, the largest eigenvalue not given.
 * The certified plan then takes, per edge {u, v}, the exact error of the
 * known modes, sum_k c_k^2 lambda_k^tau (1 + lambda_k) / (2 (1 - lambda_k))
 * with c_k = vecs[u, k] - vecs[v, k], plus the remaining mass s_e - sum_k
 * c_k^2 times the worst factor over [lambda_neg, lambda_rest] (lambda_neg
 * from bq_graph_set_spectrum, still required), and keeps N's formula: tau and
 * N are never larger than without them.  The arrays are copied; omega = 0
 * clears them.  Errors: BQ_EINVAL (omega >= n, eigenvalues outside [-1, 1),
 * non-finite vectors, NULL arrays).
 */
int bq_graph_set_eigvecs(bq_graph *g, uint32_t omega, const double *lambdas, const double *vecs,
                         double lambda_rest);

/* ---------------------------------------------------------- bq_walk_batch */
#define BQ_MODE_NAIVE 0u   /* one walk per thread, walks in input order */
#define BQ_MODE_BOUQUET 1u /* walks grouped by start vertex, one bouquet of
                              lanes per warp (Alg. 3), several walks per lane */

#define BQ_VISIT_START 0x1u /* also count position 0 (the start) */
#define BQ_HOST_IO 0x2u     /* starts / visits / paths (walk batch) or
                               edges / tau / nwalks / counts / sc (AESC) are
                               host pointers: the call copies them in and out
                               and waits for the stream before returning */

#define BQ_SAMPLER_IND 0u     /* every walk independent */
#define BQ_SAMPLER_COUPLED 1u /* walks k with equal floor(k / width) share the
                                 top t bits of their random word at the same
                                 (step, vertex): similar walks stay together
                                 (the aim of SABA, Sec. 3.3), each walk still
                                 an exact random walk.  The walks of a group
                                 are correlated (at a vertex of degree <=
                                 2^t the whole group takes the same step), so
                                 an AESC estimate over N walks has about the
                                 variance of N / width independent ones: for
                                 the certified plan's guarantee use width x
                                 its N (the groups are then the independent
                                 samples, each group mean bounded like one
                                 sample) */
#define BQ_SAMPLER_SABA 2u    /* walk batches only, for comparison: Eq.
                                 select-proposed taken literally, r = X_W xor
                                 h(cur, l) with X_W the walk's fixed 32-bit
                                 seed (low half of its key) and h one hash of
                                 (vertex, step) for the whole batch; in
                                 bouquet mode the walks of each start are
                                 ordered by X_W (SABA's arrangement).  Its
                                 walks are NOT exact random walks (later
                                 choices follow from X_W's top bits), so
                                 AESC calls refuse it; t and width unused */

typedef struct bq_sampler {
    uint32_t kind;  /* BQ_SAMPLER_IND, BQ_SAMPLER_COUPLED or BQ_SAMPLER_SABA */
    uint32_t t;     /* COUPLED: shared bits, 0..32 (32 = move together) */
    uint32_t width; /* COUPLED: group size, >= 1 */
} bq_sampler;

/*
 * Walk batch (Alg. 2 / Alg. 3 with the hash-keyed choice of Eq.
 * select-proposed; the synthetic random-walk benchmark of Sec. 4).
 * Walk i (0 <= i < n_walks) starts at starts_dev[i] and takes n_steps steps;
 * at step l = 1..n_steps it moves from cur to
 *     Gamma(cur)[ floor(H(seed, batch stream, i, l, cur) * d(cur) / 2^32) ],
 * a vertex without neighbours keeping the walk in place.  Walk i's path
 * depends only on (seed, i, starts[i], sampler, graph): mode (NAIVE or
 * BOUQUET) changes the speed, never the result.
 *   visits_dev  uint32[n], ACCUMULATED: visits[v] += number of positions
 *               l = 1..n_steps (and l = 0 with BQ_VISIT_START) at v.
 *   paths_dev   NULL or uint32[n_walks][n_steps + 1], row i = positions
 *               0..n_steps of walk i (row-major, written).
 *   sampler     NULL = BQ_SAMPLER_IND.
 * A start id >= n skips that walk and makes bq_sync report BQ_EINVAL.  When
 * n_walks * positions > UINT32_MAX a checked counter path is used and a wrap
 * is reported as BQ_EOVERFLOW by bq_sync; below that bound a counter that
 * starts at zero cannot wrap.  BOUQUET mode needs n_walks < 2^32 and
 * allocates scratch from the stream-ordered pool (freed on the stream).
 */
int bq_walk_batch(const bq_graph *g, uint64_t seed, const uint32_t *starts_dev,
                  uint64_t n_walks, uint32_t n_steps, uint32_t mode,
                  const bq_sampler *sampler, uint32_t flags, uint32_t *visits_dev,
                  uint32_t *paths_dev, void *stream);

/*
 * Walk batch that allocates nothing (the paper has no counterpart).
 * For callers that cannot call cudaMalloc or any allocator during a call:
 * a plug-in inside a host application that owns all device memory, a
 * latency-critical loop where an allocation could block or fail at an
 * arbitrary moment, or code under a memory cap that is already handed out.
 * Same walks and results as bq_walk_batch in BQ_MODE_BOUQUET, on device
 * buffers only (flags: BQ_VISIT_START; BQ_HOST_IO is rejected).  Its scratch
 * is a fixed 32 MiB array in the library's device memory, held by every
 * device that loads the library's module until the process exits; a batch
 * needs about 4 * (2 n + 1 + 2 n_walks) bytes plus a small scan workspace, and a
 * larger request fails with BQ_EINVAL and a message giving both sizes.  The
 * first call on a device looks up the array's device address (make it before
 * any stream capture).  All calls share the array: calls whose work overlaps
 * on the GPU race on it.  A graph must already exist on the device.
 */
int bq_walk_batch_noalloc(const bq_graph *g, uint64_t seed, const uint32_t *starts_dev,
                          uint64_t n_walks, uint32_t n_steps, const bq_sampler *sampler,
                          uint32_t flags, uint32_t *visits_dev, uint32_t *paths_dev,
                          void *stream);

/* ---------------------------------------------------------- bq_aesc_plan */
#define BQ_PLAN_CERTIFIED 0u
#define BQ_PLAN_SCHEDULED 1u

typedef struct bq_schedule {
    /* SCHEDULED plans: tau = clamp(ceil(tau_scale * ln(s_e / eps)) + tau_add,
     * 1, tau_max) and N = max(n_min, ceil(n_scale * s_e^2 / eps^2)). */
    double tau_scale;
    uint32_t tau_add;
    uint32_t tau_max;
    double n_scale;
    uint32_t n_min;
    uint32_t reserved;
} bq_schedule;

/*
 * Per-edge truncation length tau and walk count N (CalculateTau and NWalks
 * of Alg. 1, which the paper leaves to the TGT+ paper).  edges_uv = k vertex
 * pairs (host, uint32[2k], either orientation), or NULL for all m edges in
 * canonical order (k must then equal m).  Outputs host uint32[k].
 *   CERTIFIED: needs bq_graph_set_spectrum.  With s_e = 1/d_u + 1/d_v,
 *     tau = least tau >= 1 with s_e * max(P(tau), Q(tau)) <= eps / 2, where
 *     P(tau) = lambda2^tau (1 + lambda2) / (2 (1 - lambda2)) (0 if lambda2 <= 0)
 *     Q(tau) = max over 0 <= x <= -lambda_neg of x^tau (1 - x) / (2 (1 + x)),
 *     N = ceil(8 (tau - 1/2)^2 s_e^2 ln(2 m / delta) / eps^2),
 *     so that |SC_hat(e) - SC(e)| <= eps for all edges with probability at
 *     least 1 - delta (truncation eps/2 + Hoeffding eps/2).
 *   SCHEDULED: sched gives tau and N from s_e and eps (no guarantee).
 * Errors: BQ_ENOEDGE (a pair is not an edge), BQ_EOVERFLOW (2 N tau >= 2^32
 * or tau > tau_max), BQ_EINVAL (eps, delta out of range, no spectrum).
 */
int bq_aesc_plan(bq_graph *g, const uint32_t *edges_uv, uint64_t k, double eps,
                 double delta, uint32_t plan_mode, const bq_schedule *sched,
                 uint32_t *tau, uint32_t *nwalks);

/*
 * Pilot plan: tau from the schedule (as SCHEDULED), N from the sample
 * variance of a pilot (NWalks of Alg. 1 left open by the paper; uncertified).
 * The pilot runs on the GPU: the first n_pilot walks of each side of every
 * query, i.e. the walks bq_aesc_estimate takes first for the same seed,
 * sampler and tau, scored by a = weighted hits of u and b = weighted hits
 * of v (weights 2 before tau, 1 at tau).  Per query q and side s (0 from u,
 * 1 from v) moments[10q + 5s + 0..4] = sum a, sum b, sum a^2, sum b^2,
 * sum a b.  One sample of the estimator has the value
 *   Y = ((a(U) - a(V)) / d_u + (b(V) - b(U)) / d_v) / 2,
 * and with the integer centred sums C_aa = n0 S_aa - S_a^2,
 * C_bb = n0 S_bb - S_b^2, C_ab = n0 S_ab - S_a S_b (n0 = n_pilot) summed
 * over both sides,
 *   var = ((C_aa / d_u^2 + C_bb / d_v^2) - 2 C_ab / (d_u d_v))
 *         / (4 n0 (n0 - 1))    (clamped at 0)
 *   N   = max(ceil(z^2 var / (eps/2)^2), sched->n_min, 1),
 * each FP64 operation rounded on its own in this order: the estimate's
 * normal-approximation half-width z sqrt(var / N) is then at most eps / 2.
 * sched->n_scale is not used.  tau is planned on the host; the pilot and N
 * run on the GPU.
 * edges_uv = k host pairs (NULL: all m edges in canonical order).  Outputs
 * are host arrays: tau, nwalks uint32[k]; moments uint64[10k], or NULL to
 * skip copying them back.  The call runs on `stream` and returns after
 * synchronising it.
 * Errors: BQ_EINVAL (n_pilot < 2, z or eps out of range, bad sampler or
 * schedule), BQ_ENOEDGE, BQ_EOVERFLOW (2 n_pilot tau or 2 N tau >= 2^32),
 * BQ_ENOMEM, BQ_ECUDA.
 */
int bq_aesc_plan_pilot(bq_graph *g, uint64_t seed, const uint32_t *edges_uv, uint64_t k,
                       double eps, const bq_schedule *sched, uint32_t n_pilot, double z,
                       const bq_sampler *sampler, uint32_t *tau, uint32_t *nwalks,
                       uint64_t *moments, void *stream);

/* ------------------------------------------------------ bq_aesc_estimate */
/*
 * Estimate SC for k query edges (the walk loop and final sum of Alg. 1 at
 * zero push depth).  For query q = {u, v} (normalised to u < v; e = its
 * canonical id: edges ordered by u, then v, as in the CSR) and walk index
 * w < nwalks[q], side 0 walks from u on stream 2e, side 1 from v on stream
 * 2e + 1, tau[q] steps each.  A hit at step l weighs 2 (l < tau) or 1
 * (l = tau):
 *   counts_dev[4q + 0] = C_uu   (side 0 on u)    [+1] = C_uv (side 0 on v)
 *   counts_dev[4q + 2] = C_vu   (side 1 on u)    [+3] = C_vv (side 1 on v)
 *   sc_dev[q] = s_e + ((C_uu - C_vu)/d_u + (C_vv - C_uv)/d_v) / (2 nwalks[q]),
 *   s_e = 1/d_u + 1/d_v, each FP64 operation rounded separately in that order.
 * edges_uv_dev = NULL means all m edges in canonical order (k = m).  counts
 * are overwritten.  A pair that is not an edge gets sc = NaN and bq_sync
 * reports BQ_ENOEDGE; 2 nwalks tau >= 2^32 gets NaN and BQ_EOVERFLOW.
 * Results depend only on (seed, graph, the pair, its tau and nwalks,
 * sampler): not on the other queried edges.  sampler NULL = independent.
 * flags: BQ_HOST_IO (host buffers), BQ_AESC_NAIVE (the plain form, below).
 * Scratch comes from the stream-ordered pool.
 *
 * BQ_AESC_NAIVE runs the same walks one per thread (Alg. 2 for each walk of
 * Alg. 1's loop: walks in edge, side, walk order on the plain CSR, a
 * neighbour id and the neighbour's vertex record read per step, each walk's
 * hits added with its own atomics), instead of bouquets of 32 x lanes walks
 * of one start advanced in lockstep by a warp (Alg. 3).  The counters and
 * estimates are the same integers and doubles; only the speed differs.
 */
#define BQ_AESC_NAIVE 0x4u
int bq_aesc_estimate(const bq_graph *g, uint64_t seed, const uint32_t *edges_uv_dev,
                     uint64_t k, const uint32_t *tau_dev, const uint32_t *nwalks_dev,
                     const bq_sampler *sampler, uint32_t flags, uint32_t *counts_dev,
                     double *sc_dev, void *stream);

/* ------------------------------------------------- bq_aesc_estimate_push */
/*
 * AESC with a push phase (Alg. 1: p_l(., v_i) pushed exactly for the first
 * tau~ levels, walks of tau - tau~ steps weighted by p_tau~(x, v_i) instead
 * of hit indicators), for push depths tau~ from 0 to push_max <= 8.  In
 * fixed point with Q = 2^30 the pushed vectors of a source x are
 *   r^0_x = Q e_x,  r^{j+1}_x(y) = sum over neighbours z of y of
 *                                  floor(r^j_x(z) / d(y))
 * (so r^1_x(y) = floor(Q / d(y)) on the neighbours of x).  Pushing level j
 * touches the rows of supp r^{j-1}: vol_j(x) = sum over j' < j of the
 * degrees of supp r^j'_x (vol_1 = d(x)).  The depth of an edge (TGT+'s test:
 * push while the pushed volume is below the walks it replaces) is the
 * largest tau~ <= min(push_max, tau, 8) such that every level j <= tau~ has
 * vol_j(u) + vol_j(v) < 2 N and, when tau~ >= 2, every level 1..tau~ has at
 * most support_cap vertices in the support of either side (a planner
 * parameter the paper does not have: 1..512, bounded by the size of the
 * device's pushed-vector tables; 512 is the usual value); push_max = 0
 * keeps depth 0 everywhere.  The walks are those of bq_aesc_estimate (streams
 * 2 id + side, walk index, independent sampler), tau - depth steps long; at
 * step l a walk adds w r_u(cur) and w r_v(cur), r = r^depth and w = 2 if
 * l + depth < tau else 1, to
 *   acc[4q + 0..3] = A_uu, A_uv (walks from u), A_vu, A_vv (walks from v)
 * (uint64; 2 N tau < 2^32 keeps them below 2^62), and
 *   SC = g(u, v) + g(v, u),  g(u, v) = (X_u + (A_uu - A_vu) / N) / (2 Q d_u),
 *   X_u = sum over l = 0..depth of w_l (r^l_u(u) - r^l_u(v)), w_l = 2 if
 *   l < tau else 1 (2Q at depth 0, 2Q - w_1 floor(Q / d_v) at depth 1);
 *   g(v, u) likewise; each FP64 operation rounded once in this order.
 * Its expectation is the same half-weighted series as bq_aesc_estimate's;
 * deeper pushes lower the variance and shorten the walks.
 *
 * Arguments as bq_aesc_estimate (edges_uv_dev NULL = all edges; BQ_HOST_IO
 * for host buffers), plus depth_dev (k uint32, may be NULL): the depth
 * taken per edge; acc_dev: 4k uint64, overwritten.  With push_max >= 2 the
 * call waits for `stream` once, after planning the depths, to allocate the
 * pushed vectors of the deeper edges (8 bytes of device memory per support
 * vertex, freed in stream order once the estimate has run).
 * Errors: BQ_EINVAL (push_max > 8, support_cap outside 1..512, NULL
 * buffers), BQ_ENOMEM, and at bq_sync those of bq_aesc_estimate.
 */
int bq_aesc_estimate_push(const bq_graph *g, uint64_t seed, const uint32_t *edges_uv_dev,
                          uint64_t k, const uint32_t *tau_dev, const uint32_t *nwalks_dev,
                          uint32_t push_max, uint32_t support_cap, uint32_t flags,
                          uint32_t *depth_dev, uint64_t *acc_dev, double *sc_dev, void *stream);

/* ----------------------------------------------- bq_aesc_estimate_shared */
/*
 * Vertex-centric variant of bq_aesc_estimate: the walks of a vertex serve
 * every query edge at that vertex (Alg. 1's walk loop with walks shared per
 * vertex, a neighbour test per step).  Every endpoint x of a query edge runs
 * N_x = max nwalks and tau_x = max tau over the query edges at x; walk
 * w < N_x of x is keyed on stream 2^61 | x.  For query q = {u, v} (u < v)
 * with tau_q, the N_u walks from u add, at each step l <= tau_q, weight 2
 * (l < tau_q) or 1 (l = tau_q) to C_uu when on u and to C_uv when on v; the
 * N_v walks from v likewise to C_vu and C_vv:
 *   counts_dev[4q + 0..3] = C_uu, C_uv, C_vu, C_vv (uint32)
 *   nused_dev[2q + 0..1]  = N_u, N_v (uint32; may be NULL)
 *   sc_dev[q] = s_e + ((C_uu/N_u - C_vu/N_v)/d_u + (C_vv/N_v - C_uv/N_u)/d_v) / 2,
 * each FP64 operation rounded on its own in that order.  Each edge keeps
 * its own tau and at least its own N walks per side.  Queries must be
 * distinct edges (a repeated edge, in either orientation, gives BQ_EINVAL at
 * bq_sync).  The device path waits for `stream` once, after planning the
 * vertices, to size the per-(vertex, step) return histograms; with
 * BQ_HOST_IO every array is a host array and the call is synchronous.
 * edges_uv_dev = NULL takes all m edges in canonical order (k = m).
 * Device scratch: about 32 B per vertex, 4 B per CSR entry, 32 B per query.
 * Errors: as bq_aesc_estimate; BQ_EOVERFLOW when 2 max(N_u, N_v) tau_q >=
 * 2^32 (that estimate is NaN).
 */
int bq_aesc_estimate_shared(const bq_graph *g, uint64_t seed, const uint32_t *edges_uv_dev,
                            uint64_t k, const uint32_t *tau_dev, const uint32_t *nwalks_dev,
                            const bq_sampler *sampler, uint32_t flags, uint32_t *counts_dev,
                            uint32_t *nused_dev, double *sc_dev, void *stream);

/* ---------------------------------------------------------- AESC batches */
/*
 * Many AESC estimates (on one or many graphs, of uneven sizes) run as one
 * batch: one persistent counting launch pulls bouquet tasks from all queries
 * at once (the walk loop of Alg. 1, as bq_aesc_estimate), so small queries do
 * not leave the GPU idle.  Each query's counters and estimates are
 * bit-identical to what bq_aesc_estimate returns for it alone.
 */
typedef struct bq_aesc_query {
    const bq_graph *graph;        /* compact graph (nnz < 2^32) */
    uint64_t seed;
    const uint32_t *edges_uv_dev; /* 2k vertex pairs, or NULL = all m edges (k = m) */
    uint64_t k;
    const uint32_t *tau_dev;      /* k */
    const uint32_t *nwalks_dev;   /* k */
    uint32_t *counts_dev;         /* 4k, overwritten */
    double *sc_dev;               /* k, written */
} bq_aesc_query;

typedef struct bq_batch bq_batch;

/*
 * Prepare a batch: validates the queries (all graphs on the current device,
 * compact), copies their descriptors to the device and allocates every
 * buffer bq_batch_run needs (about 56 bytes per queried edge).  The device
 * buffers named in the queries must stay valid while the batch is used; their
 * contents may change between runs (new plans, new edge lists of the same
 * size).  Synchronous.
 */
int bq_batch_create(const bq_aesc_query *queries, uint32_t n_queries, const bq_sampler *sampler,
                    bq_batch **out);

/*
 * A batch of vertex-centric estimates: each query is estimated as by
 * bq_aesc_estimate_shared on it alone (the walks of each endpoint serve every
 * query edge at it; counts_dev receives C_uu, C_uv, C_vu, C_vv, sc_dev the
 * estimates, bit-identical to a single call), and one persistent launch runs
 * the vertex tasks of all queries.  Queries must be distinct edges within
 * each query (a repeated edge gives BQ_EINVAL at bq_sync).  Creation runs
 * each query's per-vertex plan once to size its return histograms (sum over
 * the endpoints x of tau_x = the largest tau at x): later runs may change the
 * plans' contents as long as no vertex's largest tau grows past what it was
 * at creation (else that query's estimates are NaN and bq_sync returns
 * BQ_EINVAL).  Device memory: about 32 B per vertex and 4 B per CSR entry of
 * each query's graph, 32 B per queried edge, 4 B per histogram entry.  Run
 * with bq_batch_run, release with bq_batch_destroy.  Synchronous.
 */
int bq_batch_create_shared(const bq_aesc_query *queries, uint32_t n_queries, const bq_sampler *sampler,
                           bq_batch **out);

/*
 * Run the batch on `stream`: kernel launches only (no allocation, no host
 * copy, no synchronisation), so the call can be captured into a CUDA graph
 * and the graph replayed.  Errors (a pair that is not an edge, tau = 0,
 * overflow) are reported by bq_sync as for bq_aesc_estimate.
 */
int bq_batch_run(bq_batch *batch, void *stream);

/* Number of queried edges over all queries of the batch. */
int bq_batch_size(const bq_batch *batch, uint64_t *edges);

int bq_batch_destroy(bq_batch *batch);

/* --------------------------------------------------------------- serving */
/*
 * A serving loop for SC queries on resident graphs (the paper has no
 * counterpart: its AESC runs once over all edges).  A worker thread owns a
 * stream; requests (edge subset, eps, seed) are planned on the host with the
 * scheduled plan and admitted while the device memory they need and the
 * number of requests on the GPU stay within the configured limits.  Every
 * iteration launches one persistent counting kernel over a window of tasks
 * (bouquets of walks) of every admitted request, so a request that arrives
 * while others run joins the next iteration instead of waiting for them
 * (continuous batching).  A request's counters are the sums over the same
 * walks however its tasks are spread over iterations, so its result is
 * bit-identical to bq_aesc_estimate with the same plan and seed.
 */
typedef struct bq_server bq_server;

typedef struct bq_server_config {
    uint64_t device_budget_bytes; /* device memory of admitted requests (0: 1 GiB);
                                     about 92 bytes per queried edge */
    uint32_t max_inflight;        /* requests on the GPU at once (0: 256) */
    uint32_t max_pending;         /* queued requests before submit says BQ_EBUSY (0: 65536) */
    uint64_t tasks_per_iteration; /* bouquet tasks per iteration launch, shared by the
                                     admitted requests (0: 2^16); a backlog grows it up
                                     to 8x (half of the tasks left) */
    double tau_scale;             /* scheduled plan of every request (bq_schedule) */
    uint32_t tau_add;
    uint32_t tau_max;
    double n_scale;
    uint32_t n_min;
    uint32_t planner_threads;     /* threads planning submitted requests (0: half the
                                     host cores, at most 8); a request of 32768 pairs
                                     or more is planned by up to 4 threads */
    uint32_t reserved;
    uint64_t pinned_arena_bytes;  /* page-locked host memory taken at creation for the
                                     requests' input and output images (0: 256 MiB), so
                                     that requests do not wait for page locking; more is
                                     page-locked on demand past it */
} bq_server_config;

typedef struct bq_server_stats {
    uint64_t submitted, completed, failed;
    uint64_t edges_completed;
    uint64_t iterations;
    double walk_steps;    /* sum of 2 N tau over completed requests */
    double p50_ms, p99_ms; /* latency submit -> result ready, completed requests */
    double uptime_s;
    uint32_t inflight, pending;
    /* the worker thread's time: admitting requests (upload, prepare),
     * launching iterations (including waits for a free descriptor slot),
     * completing requests (waits for results, copies, frees), and idle */
    double worker_admit_s, worker_launch_s, worker_complete_s, worker_idle_s;
    /* the planner threads' time: planning every request (summed over the
     * threads), and the longest planning of one request */
    double planner_s, planner_max_ms;
    /* page-locked blocks for request images that had to come from
     * cudaMallocHost because the free lists and the arena (cfg
     * pinned_arena_bytes) had none left, and the seconds those calls took */
    uint64_t pinned_fallbacks;
    double pinned_fallback_s;
} bq_server_stats;

/* Start a server over graphs (all on the current device, nnz < 2^32; they
 * must outlive the server).  cfg NULL = defaults with the schedule
 * tau_scale 2, tau_add 2, tau_max 64, n_scale 9, n_min 32. */
int bq_server_create(bq_graph *const *graphs, uint32_t n_graphs, const bq_server_config *cfg, bq_server **out);

/* Queue a request: k vertex pairs (host, copied) of graph `graph`, absolute
 * error eps, walks keyed by seed.  Returns with *request_id after copying
 * the pairs; the server's planner threads compute the scheduled plan (from
 * the endpoint degrees) and its worker runs it.  Errors, with no request
 * created: BQ_ENOEDGE (an id >= n or equal endpoints), BQ_EBUSY
 * (max_pending requests queued), BQ_EINVAL (bad arguments, server
 * stopping).  An endpoint without neighbours, 2 N tau >= 2^32 for an edge,
 * and a pair that is not an edge (checked on the GPU) are reported by
 * bq_server_wait (BQ_ENOEDGE, BQ_EOVERFLOW). */
int bq_server_submit(bq_server *srv, uint32_t graph, const uint32_t *edges_uv, uint64_t k, double eps,
                     uint64_t seed, uint64_t *request_id);

/* Wait up to timeout_s for a request, then copy its estimates (sc, k
 * doubles) and, if not NULL, counters (4k, layout of bq_aesc_estimate) and
 * latency (submit call -> results on the host, ms).  Returns the request's
 * status: BQ_OK, BQ_ENOEDGE (a pair is not an edge; nothing is copied),
 * BQ_EOVERFLOW (2 N tau >= 2^32 for an edge),
 * BQ_ENOMEM (it alone needs more than the device budget, or the allocation
 * failed), BQ_ECUDA; or BQ_ETIMEOUT (the request is still
 * running or queued: wait again).  Each request is returned once; waiting
 * for an unknown or already returned id is BQ_EINVAL. */
int bq_server_wait(bq_server *srv, uint64_t request_id, double timeout_s, double *sc, uint32_t *counts,
                   double *latency_ms);

int bq_server_stats_get(bq_server *srv, bq_server_stats *out);

/* Finish every queued request, then stop the worker and free the server. */
int bq_server_destroy(bq_server *srv);

/* ---------------------------------------------------------------- tuning */
/*
 * Process-wide performance knobs of the kernels (the choices an autotuner
 * makes).  They never change a result: visit counts, AESC counters and
 * estimates are identical for every setting.  The paper's bouquet width B is
 * the number of lockstep lanes (Alg. 3); on the GPU a bouquet is one warp of
 * 32 lanes, each lane advancing `walk_lanes` (walk batch) or `aesc_lanes`
 * (AESC) walks, so the paper's B corresponds to 32 x lanes here.
 */
typedef struct bq_tuning {
    uint32_t walk_lanes;       /* walks per lane, bouquet walk batch: 1, 2, 4, 8 */
    uint32_t aggregate_visits; /* 1: merge equal-vertex visits in a warp first */
    uint32_t aesc_lanes;       /* walks per lane, AESC counting: 2, 4, 8 */
    uint32_t layout;           /* device layout of graphs created from now on
                                  (what a walk step reads at random):
                                  0: plain uint32 CSR + 8-byte vertex records
                                     {row offset, degree};
                                  1 (default): automatic: 2 when the 8-byte
                                     edge records fit in L2, else 5;
                                  2: per CSR entry an edge record {id, row
                                     offset, degree}, 8 packed bytes when the
                                     fields fit, else 16 (one load per step,
                                     2-4x the bytes of plain CSR);
                                  3: 16-byte edge records;
                                  4: plain CSR + 16-byte vertex records (the
                                     layout used when nnz >= 2^32);
                                  5: neighbour ids bit-packed to ceil(log2 n)
                                     bits, several per 16-byte chunk, + 8-byte
                                     vertex records (plain CSR when packing
                                     saves nothing) */
    uint32_t hub_slots;        /* graphs created from now on get a table of
                                  hub_slots slots (0 = none; 1024..13312,
                                  default 8192): each slot holds the highest-
                                  degree vertex hashing to it (slot = high
                                  half of (v * 0x9E3779B1 mod 2^32) * slots).  The bouquet
                                  walk-batch kernel keeps the table in shared
                                  memory (16 bytes per slot) and serves those
                                  vertices' records and visit counters from it:
                                  the random walk visits a vertex in proportion
                                  to its degree */
    uint32_t l2_hints;         /* 1: the hub walk kernel reads the graph arrays
                                  with an L2 evict-last policy and the grouped
                                  walk list with evict-first (0 = plain loads) */
    uint32_t aesc_hub;         /* 1: AESC estimates on graphs with a hub table
                                  and a layout with separate vertex records
                                  serve the hubs' records from shared memory
                                  (12 bytes per slot); 0 (default): plain
                                  kernel, which measured faster (the table's
                                  shared memory takes the L1 capacity that a
                                  bouquet's walks reuse) */
    uint32_t hub_cluster;      /* graphs created from now on spread a table of
                                  hub_slots * hub_cluster slots over a thread-
                                  block cluster of hub_cluster CTAs (2, 4 or
                                  8), each holding hub_slots of them in its
                                  shared memory; a walk step reads a hub's slot
                                  in the owning CTA (distributed shared
                                  memory).  0 or 1 (default): one CTA holds the
                                  whole table, which measured faster (on R-MAT
                                  20 the walk kernel took 14.8 / 21.7 / 30.9 ms
                                  with clusters of 2 / 4 / 8 against 9.0 ms).
                                  Never changes a result. */
    uint32_t hub_relabel;      /* 1: graphs created from now on with bit-packed
                                  ids also get a copy relabelled by degree for
                                  the walk batch: the highest-degree vertices
                                  (as many as 12 bytes each fit in hub_slots *
                                  16 bytes of shared memory, 10,922 by
                                  default) take internal ids 0.., so a step
                                  finds a hub by comparing its id, with no
                                  hash; the others read a 16-byte record
                                  {row offset, degree, original id}.  Rows
                                  keep their neighbour order, so results never
                                  change.  0 (default): no copy. */
    uint32_t relabel_hub8;     /* the walk kernel on the relabelled copy:
                                  1 (default): 8-byte shared-memory hubs
                                  (a 32-bit row offset and one 32-bit word
                                  {original id | count}: a step to a hub is
                                  one 32-bit shared-memory atomic that
                                  returns the id and counts the visit; a
                                  count that wraps adds 2^bits to the
                                  visits), so 1.5x the hubs fit in the same
                                  shared memory (16,383 instead of 10,922);
                                  0: the 12-byte entries of the plain relabel
                                  kernel.  Never changes a result. */
    uint32_t hub8_hubs;        /* hubs of the 8-byte kernel: 0 (default) = as
                                  many as the 12-byte kernel's shared memory
                                  holds; at most 28000 (fewer than the
                                  vertices whose degree needs more than the
                                  records' degree field falls back to the
                                  12-byte kernel) */
    uint32_t hub8_count_bits;  /* cap on the width of the 8-byte hubs' count
                                  field, 1..31 (0, default: every bit above
                                  the id).  A narrower field only wraps more
                                  often, each wrap one more atomic; for tests
                                  of the wrap path.  Never changes a result. */
    uint32_t shared_lanes;     /* walks per lane of the vertex-centric kernels
                                  (bq_aesc_estimate_shared, bq_batch_create_
                                  shared; a batch keeps the value it was
                                  created with): 2 (default), 4 or 8.  On the
                                  4M-vertex power-law AESC 2 / 4 / 8 measured
                                  464 / 481 / 578 ms.  Never changes a
                                  result. */
    uint32_t group_walks;      /* 1 (default): a BOUQUET walk batch groups its
                                  walks by start vertex (Alg. 3's bouquets)
                                  before the walk kernel; 0: the same kernel
                                  runs the walks in input order (only the
                                  walks with a start < n are kept), to
                                  measure what the grouping buys.  Never
                                  changes a result. */
    uint32_t push_lanes;       /* walks per lane of the push-phase counting
                                  kernel (bq_aesc_estimate_push): 2
                                  (default), 4 or 8.  On the 4M-vertex
                                  power-law AESC at depth <= 1, 2 / 4
                                  measured 820 / 955 ms.  Never changes a
                                  result. */
} bq_tuning;

int bq_get_tuning(bq_tuning *out);
int bq_set_tuning(const bq_tuning *in);

/*
 * Autotuners (the paper has no counterpart: it fixes B = 8 AVX2 lanes).  Each
 * times the caller's own workload on `stream` with CUDA events, once per
 * candidate after one warm-up run, keeps the fastest candidate in the
 * process-wide tuning and returns it; ms (nullable, 3 floats) receives the
 * time of each candidate in the order listed.  Results never depend on the
 * choice.  Both synchronise the stream; the walk tuner overwrites visits_dev.
 *   bq_autotune_walks: walk_lanes in {1, 2, 4} for bq_walk_batch BOUQUET.
 *   bq_autotune_aesc:  aesc_lanes in {2, 4, 8} for a batch of these queries.
 */
int bq_autotune_walks(const bq_graph *g, uint64_t seed, const uint32_t *starts_dev, uint64_t n_walks,
                      uint32_t n_steps, uint32_t *visits_dev, void *stream, uint32_t *best, float *ms);
int bq_autotune_aesc(const bq_aesc_query *queries, uint32_t n_queries, const bq_sampler *sampler,
                     void *stream, uint32_t *best, float *ms);

/* ------------------------------------------------------------- profiling */
/*
 * Kernel timing for roofline measurement (the paper has no counterpart).
 * While enabled, the library brackets its kernels with CUDA events recorded
 * on the caller's stream (no extra synchronisation) and counts every kernel
 * it launches.  bq_profile_read waits for the recorded events, returns the
 * summed device time per kernel group since the previous read, and resets
 * the sums and the launch counts.  Counting launches is always on.
 */
typedef struct bq_profile {
    double walk_ms;          /* walk kernels (bouquet or naive) */
    uint64_t walk_launches;
    double group_ms;         /* grouping of walks by start vertex */
    uint64_t group_launches;
    double aesc_ms;          /* AESC counting kernel */
    uint64_t aesc_launches;
    double aesc_aux_ms;      /* AESC edge preparation, task scan, finalize */
    uint64_t aesc_aux_launches;
    uint64_t kernel_launches; /* every kernel the library launched */
    /* walk-batch kernel launches by kind, indexed by BQ_WALK_KERNEL_*
     * (counted whether or not timing is enabled) */
    uint64_t walk_kernel_launches[8];
} bq_profile;

#define BQ_WALK_KERNEL_NAIVE 0       /* one walk per thread (BQ_MODE_NAIVE) */
#define BQ_WALK_KERNEL_BOUQUET 1     /* bouquets, plain records */
#define BQ_WALK_KERNEL_HUB 2         /* bouquets, hashed hub table in shared memory */
#define BQ_WALK_KERNEL_CLUSTER_HUB 3 /* bouquets, hub table over a CTA cluster */
#define BQ_WALK_KERNEL_RELABEL 4     /* bouquets on the degree-relabelled copy */
#define BQ_WALK_KERNEL_RELABEL8 5    /* the same with 8-byte hubs (bq_tuning.relabel_hub8) */

int bq_profile_enable(int enable);
int bq_profile_read(bq_profile *out);

/*
 * Read-bandwidth probe for roofline ceilings (the paper has no counterpart):
 * times, with CUDA events on `stream` (synchronised), one launch of a
 * persistent kernel that reads the device buffer buf_dev (16-byte aligned,
 * `bytes` long, contents arbitrary and unchanged) `reps` times with
 * coalesced 16-byte loads that bypass L1, after one warm-up launch; *gbs =
 * bytes * reps / time.  A buffer well below the L2 size (129 MB) measures
 * the L2 read ceiling, one well above it the HBM read ceiling.  Allocates 16
 * bytes of stream-ordered scratch.  Errors: BQ_EINVAL (NULL, misaligned,
 * bytes < 16, reps = 0), BQ_ECUDA.
 */
int bq_profile_read_bandwidth(const void *buf_dev, uint64_t bytes, uint32_t reps, void *stream, double *gbs);

/* ------------------------------------------------------------ errors */
/* Wait for `stream`, then read and clear the status word of the current
 * device: BQ_OK, or the code of the first error a kernel recorded since the
 * last bq_sync (BQ_EINVAL bad start, BQ_ENOEDGE, BQ_EOVERFLOW, ...). */
int bq_sync(void *stream);

/* Static English text of a status code. */
const char *bq_strerror(int code);

/* Message of the last failed call on this thread ("" if none). */
const char *bq_last_error(void);

/* Library version string. */
const char *bq_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BOUQUET_H */
