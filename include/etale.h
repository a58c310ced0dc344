/*
 * etale.h — C ABI of the GB300 (sm_103a) ETALE index: a dynamic graph
 * approximate-nearest-neighbour index kept resident in GPU memory and
 * maintained in batches (insert, delete with repair, reclaim, search).
 *
 * Paper: "ETALE: Evolving Topology with Accelerated Lock-free Execution for
 * Dynamic Graph ANN Search on GPUs", arXiv 2607.02543.
 *
 * Conventions for every call
 *  - Returns an etale_status; nothing throws across this boundary.  On a
 *    non-OK status, etale_last_error() gives a one-line reason.
 *  - Pointer arguments may be device pointers or host pointers (pageable or
 *    pinned); the library detects which.  Host inputs are copied to device
 *    staging inside the call; host outputs are written before the call
 *    returns.  The caller owns every buffer it passes in.
 *  - The library owns the index memory (vectors, reference words, slab pool,
 *    free and retired stacks, scratch), allocated once by etale_create for
 *    the whole id capacity.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Every call synchronises `stream` before it returns.
 *  - Ids are uint32, assigned fresh and ascending by etale_insert, never
 *    reused (reusing one would clear a deletion flag, Proposition 1), so
 *    `capacity` is a lifetime insert budget.  0xFFFFFFFF is "no id".
 *  - Distances are squared L2 (ETALE_L2) or 1 - <x, y> (ETALE_IP), fp32,
 *    computed in one fixed operation order (see the design notes).
 *  - An index is not thread-safe: calls on one index must not overlap.
 */
#ifndef ETALE_H
#define ETALE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ETALE_NIL 0xFFFFFFFFu

typedef struct etale_index etale_index; /* opaque, library-owned */

typedef enum { ETALE_L2 = 0, ETALE_IP = 1 } etale_metric;

typedef enum {
    ETALE_OK = 0,
    ETALE_EINVAL = 1,     /* bad argument; the index is unchanged             */
    ETALE_ENOMEM = 2,     /* device allocation failed or slab pool exhausted  */
    ETALE_ECAPACITY = 3,  /* the id budget would be exceeded; unchanged        */
    ETALE_ECUDA = 4,      /* a CUDA runtime error; the index may be unusable   */
    ETALE_ETIMEOUT = 5,   /* a bounded device wait gave up                     */
    ETALE_EINTERNAL = 6   /* a device-side consistency check failed            */
} etale_status;

typedef enum { ETALE_MODE_DETERMINISTIC = 0, ETALE_MODE_LOCKFREE = 1 } etale_mode;

/* Build-time and maintenance knobs.  Zero selects the default.             */
typedef struct {
    uint32_t build_beam;  /* EF_BUILD (Sec. 5.6); default 64                  */
    float alpha;          /* RobustPrune slack (Sec. 3.4.1); default 1.2      */
    uint32_t max_hops;    /* expansion cap of one BeamSearch; default 4*beam  */
    uint32_t max_cand;    /* RobustPrune candidates kept; default 2*build_beam */
    uint32_t refine;      /* refine pass (Sec. 3.4.1): 0 default (= 2),
                             1 off, 2 batch peers found within two hops       */
    uint64_t max_batch;   /* insert sub-batch cap; default capacity/100       */
    uint64_t pool_slabs;  /* slab pool size P; default 2*capacity + 4*(R+1)*max_batch */
    uint32_t n_entry;     /* entry-set size |E|; default 1024                 */
    uint32_t mode;        /* etale_mode; default deterministic                */
    uint32_t cas_budget;  /* lock-free publish attempts (Alg. 1); default 16  */
    uint32_t stage_kb;    /* per-warp shared-memory stage of candidate rows
                             for RobustPrune, KB; 0 = read rows from L2     */
    uint32_t gram;        /* distances inside reverse-offer and repair
                             RobustPrunes: 0 default (tensor cores in
                             lock-free mode, canonical fp32 in deterministic
                             mode), 1 canonical fp32, 2 tensor-core Gram
                             tile (bf16 inputs, fp32 accumulation; exact for
                             integer-valued data of magnitude <= 256).  The
                             Gram tile stages its rows from the BF16 copy,
                             so gram = 2 also keeps that copy (copies bit 0) */
    uint32_t copies;      /* reduced-precision search copies kept beside the
                             fp32 rows: bit 0 BF16, bit 1 FP8-E4M3 with a
                             per-vector scale max|x| / 448; default none    */
    uint32_t rerank;      /* reduced-precision query search re-scores its
                             rerank * k best live candidates in exact fp32
                             (at most the beam); default 4                 */
    uint32_t gt;          /* etale_ground_truth: 0 default (tensor-core
                             candidate pass with an exact certified rerank
                             where it applies), 1 CUDA cores only            */
    uint32_t seed;        /* entry-set seeding of fp32 BeamSearches: 0 default
                             (tensor-core candidate pass with an exact
                             certified rerank, same seeds as the CUDA-core
                             kernel; not in concurrent mode, captured
                             graphs or reduced precision), 1 CUDA cores only */
    uint32_t exact_rows;  /* fp32 BeamSearches (inserts and etale_search):
                             0 default, always gather the fp32 rows; 1 gather
                             the BF16 copy instead while every stored row
                             converts to bf16 exactly (checked at ingest; the
                             distances are then bit-identical to those of the
                             fp32 rows, at half the bytes).  Needs the BF16
                             copy; never used in concurrent mode or captured
                             graphs.  See also etale_set_exact_rows.        */
} etale_config;

typedef enum { ETALE_PREC_FP32 = 0, ETALE_PREC_BF16 = 1, ETALE_PREC_FP8 = 2 } etale_precision;

typedef struct {
    uint64_t live;            /* delta = 0 with a slab                        */
    uint64_t tombstones;      /* delta = 1 with a slab (relays)               */
    uint64_t reclaimed;       /* delta = 1, slab freed                        */
    uint64_t next_id;         /* ids handed out so far                        */
    uint64_t capacity;        /* C                                            */
    uint64_t pool_slabs;      /* P                                            */
    uint64_t free_slabs;      /* on the free stack                            */
    uint64_t retired_slabs;   /* on the retired stack (0 between calls)       */
    uint64_t used_slabs;      /* P - free - retired                           */
    uint32_t n_entries;       /* |E| currently                                */
    uint32_t degree;          /* R                                            */
    uint64_t n_publish;       /* successful publications (Algorithm 1)        */
    uint64_t n_cas_retry;     /* failed CAS attempts                          */
    uint64_t n_dropped;       /* offers dropped after the attempt budget      */
    uint64_t n_expand;        /* BeamSearch expansions                        */
    uint64_t n_dist;          /* distance evaluations in BeamSearch           */
    uint64_t device_bytes;    /* index memory held on the device              */
    uint64_t exact_rows;      /* 1 while fp32 searches gather the exact BF16 copy */
    uint32_t dim;             /* m                                            */
    uint32_t metric;          /* etale_metric                                 */
} etale_stats_t;

/* Fill *cfg with the defaults (all fields resolved except those that depend
 * on capacity, which stay 0 until etale_create).                           */
etale_status etale_config_default(etale_config *cfg);

/* Create an empty index (Definition 1: identifier space C = capacity, slab
 * capacity R = degree, vector dimension m = dim).  degree must be 1..64;
 * dim >= 1; capacity < 2^32 - 1.  cfg may be NULL.  *out receives the
 * handle; on error *out is NULL and nothing is allocated.                   */
etale_status etale_create(uint32_t dim, etale_metric metric, uint32_t degree,
                          uint64_t capacity, const etale_config *cfg, etale_index **out);

/* Free every device and host resource of the index (the three maps of
 * Definition 1 and the two-stack slab pool of Sec. 3.3, plus scratch).  NULL
 * is a no-op.                                                              */
etale_status etale_destroy(etale_index *idx);

/* Insert n vectors (row-major n x dim fp32) as fresh nodes (Algorithm 2 with
 * a refine pass).  out_ids (may be NULL) receives the n ids, ascending from
 * the current next_id.  The batch is cut into sub-batches of
 * min(remaining, max(1, live), max_batch); each sub-batch is one round:
 * all members search the graph as it was before the sub-batch, prune, publish
 * their own slabs, then offer reverse edges.  ECAPACITY if next_id + n
 * exceeds capacity; ENOMEM if the free slab pool cannot hold one phase of
 * the largest sub-batch, (R + 1) * min(n, max_batch) slabs; in both cases
 * the index is unchanged.                                                   */
etale_status etale_insert(etale_index *idx, const float *vecs, uint64_t n,
                          uint32_t *out_ids, void *stream);

/* Delete ids (Algorithm 3): tombstone each live id, then repair every live
 * out-neighbour of the deleted nodes.  Ids never inserted, already deleted
 * or repeated are no-ops.  *n_deleted (may be NULL) receives the number of
 * ids tombstoned by this call.                                              */
etale_status etale_delete(etale_index *idx, const uint32_t *ids, uint64_t n,
                          uint64_t *n_deleted, void *stream);

/* Reclaim (Algorithm 4): recompute the entry set from the live nodes,
 * republish every live node that points at a tombstone without those
 * entries (compaction), then free every tombstone's slab.  Afterwards the
 * resident slab count equals the live count (Proposition 3).               */
etale_status etale_reclaim(etale_index *idx, void *stream);

/* Distance precision of query searches (etale_search and
 * etale_search_static): FP32 (default) or a copy kept by `copies`.  With
 * BF16 or FP8 the beam is scored on the reduced rows (fp32 arithmetic on
 * dequantised values) and the rerank * k best live candidates are re-scored
 * with the canonical fp32 distance before the k results are chosen, so
 * returned distances are exact fp32.  EINVAL if the copy is not kept.       */
etale_status etale_set_search_precision(etale_index *idx, etale_precision p);

/* Distance precision of the BeamSearch of inserts (Algorithm 2; the
 * candidate set C_v): FP32 (default) or a copy kept by `copies`.  With BF16
 * or FP8 the search is scored on the reduced rows, and the nearest max_cand
 * expanded nodes are re-scored with the canonical fp32 distance and
 * re-sorted before RobustPrune, so every stored rho is exact fp32; only the
 * choice of candidates depends on the precision.  Seeding of these searches
 * runs in the same precision (CUDA cores).  EINVAL if the copy is not kept.
 * Recorded rounds use the precision in force when they are recorded.       */
etale_status etale_set_insert_precision(etale_index *idx, etale_precision p);

/* Size the grids of later eager update calls (insert, delete, reclaim) for
 * this share of the SMs (0 < share <= 1; default 1), so that query launches
 * running at the same time on another stream (concurrent mode, the serving
 * ring) keep room on the device.  Results never depend on it.              */
etale_status etale_set_writer_share(etale_index *idx, float share);

/* Set cfg.rerank for later reduced-precision query searches (1..256).     */
etale_status etale_set_rerank(etale_index *idx, uint32_t rerank);

/* Copy the reduced-precision codes of ids [first, first + n) to HOST
 * buffers (either may be NULL): bf16 as uint16 bits, n x dim; fp8 as bytes,
 * n x dim, with scales[n].                                                 */
etale_status etale_export_copies(etale_index *idx, uint64_t first, uint64_t n, uint16_t *bf16,
                                 uint8_t *fp8, float *scales);

/* Batched k-NN query (BeamSearch with beam max(beam, k)).  queries: nq x dim
 * fp32.  out_ids / out_dists: nq x k, nearest first; a search that finds
 * fewer than k live nodes pads with ETALE_NIL and +inf.  Only nodes whose
 * reference word read during the search has delta = 0 are returned
 * (Proposition 1).                                                         */
etale_status etale_search(etale_index *idx, const float *queries, uint64_t nq, uint32_t k,
                          uint32_t beam, uint32_t *out_ids, float *out_dists, void *stream);

/* Evaluation count of a query batch (diagnostic; measurement support for
 * the algorithmic bytes of BeamSearch, Sec. 3.4.1).  Runs the query search
 * of etale_search once on DEVICE or host queries with a per-query log of the
 * ids whose distance it computed during expansions, and reports:
 *   *n_eval   distance evaluations made by the kernel (its visited set is a
 *             lossy cache, so an id may be evaluated more than once);
 *   *n_unique distinct ids evaluated per query, summed, not counting each
 *             query's initial beam (the seeds): the evaluations of an exact
 *             visited set.  With an entry set no larger than the beam, this
 *             is the distance count of a sequential BeamSearch minus |E| per
 *             query;
 *   *n_expand expansions.
 * Allocates nq * max_hops * R * 4 bytes of log for the call; max_hops * R
 * must be <= 32768.  Results are not returned.                            */
etale_status etale_search_eval_count(etale_index *idx, const float *queries, uint64_t nq, uint32_t k,
                                     uint32_t beam, uint64_t *n_eval, uint64_t *n_unique,
                                     uint64_t *n_expand, void *stream);

/* Exact k nearest live nodes by brute force (measurement support for
 * Recall@10, Sec. 5.2): canonical fp32 distances, ties by smaller id.  k must
 * be 1..32.  Unless cfg.gt = 1, a tensor-core pass (bf16 inputs, fp32
 * accumulation; a hi/lo split when the data are not exact in bf16) keeps 32
 * candidates per query, which are reranked with the canonical distance; a
 * query whose result an a-priori error bound cannot certify is recomputed
 * on CUDA cores, so the output never depends on the path taken.            */
etale_status etale_ground_truth(etale_index *idx, const float *queries, uint64_t nq,
                                uint32_t k, uint32_t *out_ids, float *out_dists, void *stream);

/* Copy the logical graph of ids [0, n) to HOST buffers: deleted[n],
 * has_slab[n], degree[n] (uint8), nbr_ids[n*R] and nbr_rho[n*R] (entries
 * beyond the degree are ETALE_NIL / 0).  n must be <= next_id.             */
etale_status etale_export_graph(etale_index *idx, uint64_t n, uint8_t *deleted,
                                uint8_t *has_slab, uint8_t *degree, uint32_t *nbr_ids,
                                float *nbr_rho, void *stream);

/* Copy the current entry set to a HOST buffer of capacity n_entry; *n
 * receives its size.                                                       */
etale_status etale_get_entries(etale_index *idx, uint32_t *out, uint32_t *n);

/* Counters of the index.  live / tombstones / reclaimed classify the
 * reference words of Definition 1 (delta and s); used_slabs is the resident
 * slab count of Sec. 4.4, which equals live right after etale_reclaim
 * (Proposition 3) and live + tombstones between reclaims; free_slabs and
 * retired_slabs are the two stacks of Sec. 3.3.  Reads the device counters
 * on a private stream (never waits for the caller's streams, except for the
 * last round-graph launch when one ran since the counts were read).        */
etale_status etale_stats(etale_index *idx, etale_stats_t *out);

/* Resolved configuration of an index.                                      */
etale_status etale_get_config(const etale_index *idx, etale_config *out);

/* One-line description of the last failed call made by the calling thread
 * (on any index, etale_create included); idx is ignored.  Never NULL.      */
const char *etale_last_error(const etale_index *idx);

/* ---- snapshots ---------------------------------------------------------- */
/* Save the index state (Definition 1: vectors, reference words, the slab
 * map, plus the entry set and configuration) to the file `path`, so that
 * etale_load (or any reader of the format below) can rebuild the same
 * logical graph.  Waits for `stream` first; synchronous.  The file holds no
 * slab numbers: a loaded index lays its slabs out afresh, so its resident
 * slab count is the number of ids with a slab.
 *
 * Format (version 1, little-endian, no padding):
 *   char  magic[8] = "ETALESN1"
 *   u32   version = 1, dim, metric (0 L2, 1 IP), degree R
 *   u64   capacity, next_id
 *   u32   n_entries, n_cfg (= 17)
 *   u64   cfg[n_cfg]: build_beam, alpha (fp32 bits), max_hops, max_cand,
 *         refine, max_batch, pool_slabs, n_entry, mode, cas_budget,
 *         stage_kb, gram, copies, rerank, gt, seed, exact_rows
 *   f32   x[next_id][dim]
 *   u8    flags[next_id]: bit 0 delta, bit 1 has a slab, bit 2 the list was
 *         written by a RobustPrune (a hint of this library; 0 is always
 *         valid and changes no result)
 *   u8    deg[next_id] (0 when there is no slab)
 *   then, for each id with a slab in ascending id, deg entries {u32 id;
 *         f32 rho} in slab order
 *   u32   entries[n_entries]
 * EINVAL if the file cannot be written.                                    */
etale_status etale_save(etale_index *idx, const char *path, void *stream);

/* Create an index from a file written by etale_save (or in its format).
 * cfg NULL takes the saved configuration; otherwise cfg's fields apply as in
 * etale_create.  capacity 0 keeps the saved capacity; it must be >= the
 * saved next_id.  The reduced-precision copies are recomputed from the
 * vectors.  EINVAL for a malformed or inconsistent file (an id beyond
 * next_id, a degree above R, a list on an id without a slab); ENOMEM if the
 * pool cannot hold the saved lists.                                        */
etale_status etale_load(const char *path, const etale_config *cfg, uint64_t capacity, etale_index **out);

/* ---- launch-shape tuning (deployment support; the paper has none) -------- */
typedef struct {
    uint32_t stage_rows;  /* neighbour rows gathered per bulk-copy batch      */
    uint32_t seen_bits;   /* log2 slots of the evaluated-id cache             */
    float ms;             /* measured: seeding + search of the tuning batch   */
    uint32_t warps_per_block; /* queries in flight per thread block: 2, 4, 8 */
    uint32_t keys_tc;     /* BF16 searches: keys from the tensor cores (1) or
                             the CUDA cores (0); 1 for other precisions       */
} etale_tuning;

/* Turn the exact-copy gathers of cfg.exact_rows on (1) or off (0) for the
 * calls that follow (results never depend on it).  Turning them on reads
 * the device's count of inexact rows (synchronises the default stream).   */
etale_status etale_set_exact_rows(etale_index *idx, int on);

/* Set the BeamSearch launch shape (results never depend on it);
 * warps_per_block 0 keeps the current value.                               */
etale_status etale_set_search_tuning(etale_index *idx, uint32_t stage_rows, uint32_t seen_bits,
                                     uint32_t warps_per_block);

/* Where a BF16 search (etale_set_search_precision 1; insert or query) takes
 * the keys that order its beam: tensor = 1 (default), |q|^2 + |x|^2 - 2 q.x
 * with the dot product from bf16 tensor-core MMAs; tensor = 0, the CUDA
 * cores' fp32 reduction of the fp32 query against the widened bf16 row.
 * Both are approximations of the fp32 distance, so the beam order, and
 * with it the candidates that reach the exact rerank, may differ between
 * them; returned distances are exact fp32 either way.  Other precisions
 * ignore it.  EINVAL unless tensor is 0 or 1.                              */
etale_status etale_set_search_keys(etale_index *idx, int tensor);

/* Time seeding + BeamSearch of the given DEVICE query batch under each
 * candidate launch shape (stage rows 2/4/8/16 x cache 2^7..2^10 slots x
 * 2/4/8 warps per block, and for a BF16 search precision both key paths of
 * etale_set_search_keys; shapes whose shared memory does not fit the device
 * are skipped), keep the fastest for this index, and report up to n_out
 * tried shapes in out.  Results do not depend on the launch shape; a BF16
 * search's key path may change which candidates reach its exact rerank.  */
etale_status etale_autotune_search(etale_index *idx, const float *queries, uint64_t nq, uint32_t k,
                                   uint32_t beam, etale_tuning *out, uint32_t n_out, uint32_t *n_tried,
                                   void *stream);

/* The search beam (EF_SEARCH, Sec. 5.6) for a recall target, then the launch
 * shape at that beam: computes the exact top-k of the DEVICE query batch
 * (etale_ground_truth, k <= 32), searches with each beam of `beams`
 * (ascending, <= 256) until Recall@k reaches `target`, writes the beam taken
 * to *chosen (the last one if none reaches it) and each tried beam's recall
 * to recalls[i] (may be NULL; -1 for beams not tried), then runs
 * etale_autotune_search at *chosen.                                         */
etale_status etale_autotune_beam(etale_index *idx, const float *queries, uint64_t nq, uint32_t k, float target,
                                 const uint32_t *beams, uint32_t n_beams, float *recalls, uint32_t *chosen,
                                 void *stream);

/* ---- CUDA-graph query batches (deployment support; the paper has none) -- */
typedef struct etale_search_graph etale_search_graph;

/* Capture the query path (row padding, seeding, BeamSearch) into a CUDA
 * graph bound to caller-owned DEVICE buffers: queries (nq_max x dim),
 * out_ids / out_dists (nq_max x k) and nq_dev, one uint32 that holds the
 * batch size of each launch (clamped to nq_max).  The kernels read the batch
 * size and the entry-set size from device memory, so one graph serves every
 * batch size and stays valid across later updates of the index.  The search
 * precision and launch shape in force at creation are baked in.  The graph
 * owns its scratch (allocated here, freed by destroy).
 * Seeding: when the index seeds on tensor cores, fp32 search, the entry set
 * is full (n_entry entries), nq_max >= 32 and the index is not in
 * concurrent mode, the graph seeds on tensor cores as etale_search does
 * (same seeds) and pins the index's entry copies; a launch is then refused
 * (EINVAL) if the entry set changed size or concurrent mode is on, and
 * etale_destroy refuses while such a graph lives.  Otherwise it seeds on
 * CUDA cores.                                                              */
etale_status etale_search_graph_create(etale_index *idx, uint32_t nq_max, uint32_t k, uint32_t beam,
                                       const float *queries, uint32_t *out_ids, float *out_dists,
                                       const uint32_t *nq_dev, etale_search_graph **out);
/* Enqueue one replay on `stream` (asynchronous, no host synchronisation).  */
etale_status etale_search_graph_launch(etale_search_graph *g, void *stream);
/* Synchronise `stream` and report device-side errors of earlier replays.    */
etale_status etale_search_graph_check(etale_search_graph *g, void *stream);
etale_status etale_search_graph_destroy(etale_search_graph *g);

/* ---- recorded churn rounds (deployment support; the paper has none) ---- */
/* One churn round recorded as a CUDA graph and replayed with one launch: a
 * delete batch with repair (Algorithm 3), one insert sub-batch with its
 * reverse offers and refine pass (Algorithm 2), a Reclaim (Algorithm 4) and,
 * if nq > 0, a query batch, in the order and with the results of the eager
 * calls etale_delete, etale_insert, etale_reclaim and etale_search.  Each
 * recorded kernel is still its own launch, run after the previous one has
 * terminated, with the recycle step between publishing launches
 * (Definition 2, Lemma 1).  The kernels read next_id, the first new id, the
 * live count and |E| from device memory, so the host neither reads nor waits
 * between or within replays.
 *
 * Buffers (DEVICE, caller-owned, read at every launch, rewritten by the
 * caller between launches in stream order):
 *   del_ids    n_del ids to delete; ETALE_NIL entries, ids never inserted
 *              and ids already deleted are no-ops (as in etale_delete);
 *   ins_vecs   n_ins x dim rows, inserted as ids [next_id, next_id + n_ins);
 *   queries    nq x dim rows; out_ids / out_dists nq x k (as etale_search,
 *              fp32 or the search precision in force at recording).
 * n_del, n_ins or nq may be 0.
 *
 * Conditions, checked at recording and at every launch (EINVAL, ECAPACITY
 * or ENOMEM; nothing is launched): not in concurrent mode; the insert is
 * one sub-batch (n_ins <= max_batch and <= the live count once the deletes
 * are made); the ids left cover n_ins; the slab pool covers a round.  With
 * tensor-core seeding the live count must also stay >= n_entry.  The host's
 * counts (live, tombstones, |E|, free slabs) are read back by
 * etale_round_graph_sync, or by the next call that needs them (any eager
 * call on the index waits for the last replay first).
 *
 * The graph records the addresses of index scratch buffers: while it
 * lives, an eager call that would need one of them larger fails with
 * ENOMEM.  Destroy every round graph before etale_destroy (which refuses
 * otherwise).                                                              */
typedef struct etale_round_graph etale_round_graph;
etale_status etale_round_graph_create(etale_index *idx, uint32_t n_del, const uint32_t *del_ids, uint32_t n_ins,
                                      const float *ins_vecs, uint32_t nq, uint32_t k, uint32_t beam,
                                      const float *queries, uint32_t *out_ids, float *out_dists,
                                      etale_round_graph **out);
/* Enqueue one round on `stream` (asynchronous; no host synchronisation).   */
etale_status etale_round_graph_launch(etale_round_graph *g, void *stream);
/* Wait for the last launch, read the index's counts back, and report
 * device-side errors of the replays since the last sync.                   */
etale_status etale_round_graph_sync(etale_round_graph *g);
etale_status etale_round_graph_destroy(etale_round_graph *g);

/* ---- serving ring (deployment support; the paper's two-stream serving,
 *      Sec. 5.5, with requests admitted while a launch runs) ------------- */
/* A ring of `slots` query slots in pinned, host-mapped memory.  The host
 * writes query rows into slots (row stride round_up(dim, 4) floats, the
 * padding left at zero) and publishes the number of tickets submitted;
 * ticket t uses slot t % slots.  Each etale_ring_launch enqueues one bounded
 * persistent search launch on `stream`: its warps take submitted tickets in
 * order as they become free, including tickets published while the launch
 * runs, seed each query from the entry set (the same seeds as etale_search),
 * run the query BeamSearch (k, beam and precision as etale_search) and write
 * the k results into the slot's host-mapped rows, then done[slot] = t + 1 and
 * served_by[slot] = the launch's sequence number.  A launch stops taking
 * tickets after max_us microseconds or when the ring is closed, and ends
 * once its warps finish the queries they hold; the caller keeps one launch
 * in flight to serve continuously.  Slabs are recycled only between
 * launches (in concurrent mode the launch counts as a query search for
 * writer calls), so a query never reads a reused slab (Lemma 1).
 * Flow control is the caller's: ticket t may be written only once
 * done[t % slots] == t - slots + 1 (or the slot is unused).  Results equal
 * etale_search's for the same query, k and beam.                           */
typedef struct etale_ring etale_ring;
etale_status etale_ring_create(etale_index *idx, uint32_t slots, uint32_t k, uint32_t beam, etale_ring **out);
/* Host views: rows (slots x row_stride floats), ids / dists (slots x k),
 * done (slots), served_by (slots).  Any pointer may be NULL.               */
etale_status etale_ring_buffers(etale_ring *r, float **rows, uint32_t *row_stride, uint32_t **ids, float **dists,
                                uint64_t **done, uint32_t **served_by);
/* Make tickets [0, tail) visible to launches (a release store; rows first). */
etale_status etale_ring_publish(etale_ring *r, uint64_t tail);
etale_status etale_ring_close(etale_ring *r, int closed);
/* blocks: thread blocks of 4 warps (0 = 1 per SM); *seq (may be NULL)
 * receives the launch's sequence number.                                   */
etale_status etale_ring_launch(etale_ring *r, uint32_t max_us, uint32_t blocks, uint32_t *seq, void *stream);
/* Serve n queries (HOST rows, n x dim) arriving at arrival_s[i] seconds from
 * the call's start (ascending): native threads submit each query into the
 * ring at its arrival time (waiting for a free slot), issue launches of
 * max_us microseconds alternately on `stream` and a second stream of the
 * ring's own (the next one when the current one has run three quarters of
 * its lifetime, so tickets are always being taken while the previous launch
 * finishes the queries it holds), and collect completions.
 * issued_s[i] (may be NULL) receives when query i was written into a slot,
 * completion_s[i] when its results were seen on the host; out_ids /
 * out_dists (n x k, may be NULL) the results; *mid_launch (may be NULL) the
 * number of queries taken by a launch issued before they were submitted;
 * *launches (may be NULL) the launches made.  Runs without the caller (for
 * example, another thread may run update calls on another stream meanwhile,
 * in concurrent mode).                                                     */
etale_status etale_ring_serve(etale_ring *r, const float *queries, const double *arrival_s, uint64_t n,
                              uint32_t max_us, uint32_t blocks, double *issued_s, double *completion_s,
                              uint32_t *out_ids, float *out_dists, uint64_t *mid_launch, uint32_t *launches,
                              void *stream);
/* Totals over the ring's finished launches: queries served, and the
 * nanoseconds their warps spent seeding and in the BeamSearch (device
 * clock).  No synchronisation: a launch still running is not counted.     */
etale_status etale_ring_stats(etale_ring *r, uint64_t *served, uint64_t *seed_ns, uint64_t *search_ns);
etale_status etale_ring_destroy(etale_ring *r);

/* How the last etale_ground_truth call ran: *path 0 CUDA cores, 1 tensor
 * cores on bf16-exact data, 2 tensor cores with the hi/lo split;
 * *fallback_queries = queries recomputed on CUDA cores.  Diagnostic.        */
etale_status etale_ground_truth_info(etale_index *idx, uint32_t *path, uint64_t *fallback_queries);

/* Failure-detection self-test (diagnostic; the paper has no counterpart).
 * Launches one warp whose mbarrier wait can never complete (it expects 16
 * bytes that no copy delivers; no copy is issued), polled at most
 * `poll_limit` times.  The wait gives up, the kernel records ETALE_ETIMEOUT
 * in its status word and returns, and the call returns ETALE_ETIMEOUT with
 * the CUDA context still usable.  Every bounded wait of the library ends
 * the same way.  poll_limit must be 1..1e6.                                 */
etale_status etale_selftest_bounded_wait(uint32_t poll_limit, void *stream);

/* Concurrent mode (off by default).  With it on, one thread may run query
 * searches (etale_search / etale_search_static) on one stream while another
 * thread runs update calls (insert, delete, reclaim) on another stream; the
 * two overlap on the device.  Searches keep their own scratch, work queue
 * and error word.  Slabs retired by an update call are not reused within it:
 * they return to the free stack at the start of the NEXT update call, after
 * that call's stream has waited for the last search issued so far, so no
 * search can read a slab after its reuse (Lemma 1, Proposition 2).  Each
 * update call therefore needs free slabs for all of its publications (large
 * inserts may return ENOMEM; cut them).  Two searches, or two updates, must
 * still not overlap.                                                        */
etale_status etale_set_concurrent(etale_index *idx, int on);

/* Kernel launches issued by this library so far (launch accounting).      */
uint64_t etale_kernel_launches(const etale_index *idx);

/* Opt-in phase timing.  When enabled, CUDA events are recorded on the
 * caller's stream around every phase below; durations accumulate per phase
 * and are folded in when a call synchronises.  Off by default (no events).  */
typedef enum {
    ETALE_PH_SEED = 0,        /* entry-set seeding kernel (inserts and queries) */
    ETALE_PH_SEARCH_INSERT,   /* BeamSearch kernel, insert mode                 */
    ETALE_PH_PRUNE,           /* forward RobustPrune + own publish              */
    ETALE_PH_OFFER_SORT,      /* offer sort + segmenting (deterministic mode)   */
    ETALE_PH_OFFER_FOLD,      /* reverse-offer publication                       */
    ETALE_PH_REFINE,          /* refine pass selection + publish                */
    ETALE_PH_DELETE_PREP,     /* id sort, tombstone CAS, compaction of ids      */
    ETALE_PH_REPAIR_K,        /* replacement sets K(u, a)                       */
    ETALE_PH_REPAIR_FOLD,     /* repair publication (pair sort included)        */
    ETALE_PH_ENTRIES,         /* entry-set recomputation                        */
    ETALE_PH_COMPACT,         /* reclaim phase 1 (bitmap + compaction)          */
    ETALE_PH_RECLAIM,         /* reclaim phase 2                                */
    ETALE_PH_SEARCH_QUERY,    /* BeamSearch kernel, query mode                  */
    ETALE_PH_RECYCLE,         /* retired -> free stack                          */
    ETALE_PH_GT_PREP,         /* ground truth: bf16 copies and norms            */
    ETALE_PH_GT_TENSOR,       /* ground truth: tensor-core candidate pass       */
    ETALE_PH_GT_MERGE,        /* ground truth: exact rerank + certificate       */
    ETALE_PH_GT_EXACT,        /* ground truth: CUDA-core exact kernel           */
    ETALE_PH_COUNT
} etale_phase;

etale_status etale_set_profiling(etale_index *idx, int enable);

/* Copy accumulated milliseconds and launch counts for the first n phases
 * (either pointer may be NULL); reset = 1 clears the accumulators.         */
etale_status etale_get_profile(etale_index *idx, double *ms, uint64_t *count, uint32_t n, int reset);

/* Work tallies of the writer kernels (the paper has no counterpart; they
 * give each kernel's algorithmic bytes for a roofline).  The kernels count,
 * per warp, what their step of the method must move and add it once at the
 * warp's end, always (no switch):
 *   rows[k]  - bytes of vector rows gathered: the distinct rows of each
 *              RobustPrune (Sec. 3.4.1) or distance step, in the copy that
 *              step reads (fp32 rows, or the bf16 copy on the Gram path);
 *   state[k] - bytes of graph state read or written: reference words,
 *              slab entries, tombstone bits (Def. 1, Algorithm 1).
 * Lists handed from one kernel to the next (candidate keys, offers, the
 * replacement sets K(u, a)) are not counted.  Both accumulate over calls
 * until reset = 1, which zeroes them after the copy.  Copies the first n
 * kinds (either pointer may be NULL); synchronises the device.             */
typedef enum {
    ETALE_WK_PRUNE = 0,       /* forward RobustPrune + own publish              */
    ETALE_WK_OFFER,           /* reverse-offer publication                      */
    ETALE_WK_REFINE,          /* refine pass                                    */
    ETALE_WK_REPAIR_K,        /* replacement sets K(u, a)                       */
    ETALE_WK_REPAIR_FOLD,     /* repair publication                             */
    ETALE_WK_COMPACT,         /* reclaim phase 1                                */
    ETALE_WK_COUNT
} etale_work_kind;

etale_status etale_get_work(etale_index *idx, uint64_t *rows, uint64_t *state, uint32_t n, int reset);

/* Query search that allocates nothing (the paper has no counterpart: this is
 * a deployment variant of etale_search).
 *
 * For callers that cannot call cudaMalloc while they run: a serving thread
 * held to a device-memory budget fixed at start-up, or a library hosted
 * inside another framework whose memory manager owns the device and must not
 * be bypassed or re-entered from that context.  etale_search may grow
 * staging buffers on demand; this variant never calls cudaMalloc, cudaFree or
 * any allocating routine.  Its scratch (padded query rows and the seeded
 * beams) lives in a file-scope device array of ETALE_STATIC_SCRATCH_BYTES
 * that every GPU loading the library holds until the process exits.
 *
 * queries, out_ids and out_dists must be DEVICE pointers (host buffers would
 * need staging); results equal etale_search's for the same arguments.
 * nq * (4 * round_up(dim, 4) + 8 * max(beam, k)) must not exceed
 * ETALE_STATIC_SCRATCH_BYTES, else ETALE_EINVAL with a message; every
 * argument is checked before anything is launched.
 *
 * The first call on a device looks up the array's device address (set-up
 * once per device, with that device current); make that first call before
 * any stream capture.  All calls share the one array and leave their
 * contents in it: calls whose work overlaps on the GPU (other streams,
 * other indexes, other threads) race on it and must be serialised by the
 * caller.  Like every call, it synchronises `stream` before returning.     */
#define ETALE_STATIC_SCRATCH_BYTES (8u << 20)
etale_status etale_search_static(etale_index *idx, const float *queries, uint64_t nq, uint32_t k,
                                 uint32_t beam, uint32_t *out_ids, float *out_dists, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* ETALE_H */
