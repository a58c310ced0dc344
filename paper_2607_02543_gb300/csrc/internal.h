// internal.h — host-side launchers shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace etale {

struct SearchTuning {
    u32 stage_rows = 16;       // rows gathered per bulk-copy batch
    u32 seen_bits = 9;         // log2 of the evaluated-id cache slots
    u32 warps_per_block = 4;   // queries in flight per block: 2, 4 or 8
    u32 keys_tc = 1;           // BF16 searches: keys from the tensor cores (1) or the CUDA cores (0)
};

// Raise a kernel's dynamic shared-memory limit to at least `bytes`.  The
// limit is process-wide per kernel and only ever raised (under a lock), so a
// thread launching with less never lowers it under another thread that has
// just raised it for a larger launch.
cudaError_t smem_at_least(const void *fn, size_t bytes);

// search.cu
size_t search_smem_bytes(u32 mp, u32 L, u32 stage_rows, u32 seen_bits, u64 capacity, u32 wpb);
// seed_kernel: top-L of the entry set per query into `seed` (nq x L); it
// must precede the search launch that reads `seed`.
// qsel (optional): the batch is the queries qsel[0 .. n) (n = *nq_dev), each
// written to its own row of `seed`.
cudaError_t launch_seed(const Dev &d, const float *q, u32 nq, u32 L, u64 *seed, cudaStream_t st, u32 prec = 0,
                        const u32 *nq_dev = nullptr, const u32 *qsel = nullptr);
// prec: 0 fp32, 1 bf16 copy, 2 fp8 copy (query mode only; the best
// min(rerank * k, L) live candidates are re-scored in canonical fp32).
// exact_rows: fp32 semantics with rows gathered from the bf16 copy, which
// holds every stored row exactly (prec 1, no rerank, any mode).
cudaError_t launch_search(const Dev &d, const float *q, u32 nq, u32 L, u32 max_hops, u32 mode, u32 k,
                          u32 *out_ids, float *out_dist, u64 *exp_keys, u32 *exp_count, u64 *seed,
                          const SearchTuning &tune, int num_sms, cudaStream_t st, u32 prec = 0,
                          u32 rerank = 4, const u32 *nq_dev = nullptr, bool exact_rows = false,
                          u32 *elog = nullptr, u32 *elog_n = nullptr, u32 elog_cap = 0, bool rekey = false);
// Serving ring (a bounded persistent search launch over host-mapped slots):
// rows / out_ids / out_dist / tail / closed / done / served_by are device
// views of host-mapped memory; head and seed are device memory.
cudaError_t launch_ring_search(const Dev &d, float *rows, u32 slots, u32 L, u32 max_hops, u32 k, u32 *out_ids,
                               float *out_dist, u64 *seed, const SearchTuning &tune, u32 blocks, cudaStream_t st,
                               u32 prec, u32 rerank, u64 *head, const u64 *tail, const u64 *closed, u64 *done,
                               u32 *served_by, u32 seq, u64 max_ns);
// Diagnostic: distinct ids each query evaluated (its log, elog_cap slots per
// query, from a launch_search with elog set), not counting its n0 seeds;
// out[0] += evaluations, out[1] += distinct non-seed ids, out[2] += overflows.
size_t eval_unique_smem(u32 cap, u32 L);
cudaError_t launch_eval_unique(const u32 *elog, const u32 *elog_n, u32 cap, const u64 *seed, u32 L, u32 n0, u32 nq,
                               u64 *out, cudaStream_t st);

// Offer lists: a payload index p names (src[p], rho[p]); key[p] is the target
// id or `invalid` (= capacity) for an empty slot.
struct Offers {
    u32 *key, *val;        // sorted in place (val = payload index)
    u32 *key_alt, *val_alt;
    u32 *src;
    float *rho;
    u32 n;                 // slots
};

// update.cu
// rescore: the keys come from a reduced-precision search; the kept candidates
// are re-scored with the canonical fp32 distance before RobustPrune.
cudaError_t launch_prune_insert(const Dev &d, u32 first, u32 b, const u64 *exp_keys, const u32 *exp_count,
                                u32 max_hops, u32 max_cand, u32 *F_id, float *F_rho, u32 *F_n,
                                const Offers &of, int num_sms, cudaStream_t st, bool rescore = false);
// lock-free (budget > 0): offer slots [lo, hi) only
cudaError_t launch_offer_fold(const Dev &d, const Offers &of, const u32 *seg_start, const u64 *seg_count,
                              u32 lockfree_budget, int num_sms, cudaStream_t st, u32 lo = 0,
                              u32 hi = 0xFFFFFFFFu);
// spill: per resident warp, candidate lists for members with many peers
// (refine_spill_bytes bytes).
size_t refine_spill_bytes(const Dev &d, u32 max_cand, int num_sms);
cudaError_t launch_refine(const Dev &d, u32 first, u32 b, u32 mode, u32 max_cand, const Offers &of,
                          int num_sms, cudaStream_t st, char *spill, size_t spill_bytes);
cudaError_t launch_tombstone(const Dev &d, const u32 *sorted_ids, u32 n, u64 next_id, u32 *ok_flags,
                             cudaStream_t st);
cudaError_t launch_repair_k(const Dev &d, const u32 *dt, const u64 *n_dt, u32 max_n, u32 *pair_key,
                            u32 *pair_val, uint2 *pair_K, u32 *pair_Kn, int num_sms, cudaStream_t st);
// budget == 0: deterministic, one warp per segment of equal targets;
// budget > 0: lock-free, one warp per pair slot, slots [lo, lo + n_pairs).
cudaError_t launch_repair_fold(const Dev &d, const u32 *dt, const u32 *pair_key, const u32 *pair_val,
                               const uint2 *pair_K, const u32 *pair_Kn, const u32 *seg_start,
                               const u64 *seg_count, u64 n_pairs, u32 budget, int num_sms, cudaStream_t st,
                               u64 lo = 0);
cudaError_t launch_compact(const Dev &d, u64 next_id, const u32 *tomb_bits, cudaStream_t st);
cudaError_t launch_reclaim_tombstones(const Dev &d, u64 next_id, cudaStream_t st);

// util.cu
struct ScanScratch {
    u32 *lvl[4];
    u32 lvl_n[4];
    int levels;
};
size_t scan_scratch_elems(u32 n);
void scan_scratch_carve(ScanScratch &s, u32 *buf, u32 n);
cudaError_t exclusive_scan(const u32 *in, u32 *out, u32 n, const ScanScratch &s, cudaStream_t st);

struct SortScratch {
    u32 *hist;             // 256 * tiles
    u32 *hist_scan;
    ScanScratch scan;
};
size_t sort_scratch_elems(u32 n);
void sort_scratch_carve(SortScratch &s, u32 *buf, u32 n);
// Stable LSD radix sort of (key, val) by the low `key_bits` bits of key.  The
// result ends in (key, val); (key_alt, val_alt) are scratch of equal size.
cudaError_t radix_sort_pairs(u32 *key, u32 *val, u32 *key_alt, u32 *val_alt, u32 n, u32 key_bits,
                             const SortScratch &s, cudaStream_t st);
// Segments of equal keys among sorted keys (keys equal to `invalid` sort last
// and are ignored): seg_start[0..count] and the count in *seg_count.
cudaError_t make_segments(const u32 *key, u32 n, u32 invalid, u32 *flags, u32 *scan_out,
                          u32 *seg_start, u64 *seg_count, const ScanScratch &s, cudaStream_t st);

cudaError_t launch_recycle(const Dev &d, cudaStream_t st);
// n_dev (optional): row count read on the device, n is its cap.
// row0 (optional): the destination's first row, read on the device.
cudaError_t launch_ingest(float *x, u32 mp, const float *src, u32 dim, u64 n, cudaStream_t st,
                          const u32 *n_dev = nullptr, const u64 *row0 = nullptr);
cudaError_t launch_ingest_copies(const Dev &d, u64 first, u64 n, cudaStream_t st);
cudaError_t launch_live_flags(const Dev &d, u64 next_id, u32 *flags, cudaStream_t st);
cudaError_t launch_entries_select(const Dev &d, u64 next_id, const u32 *flags, const u32 *rank, u64 live,
                                  u32 S, cudaStream_t st);
cudaError_t launch_tomb_bits(const Dev &d, u64 next_id, u32 *bits, cudaStream_t st);
cudaError_t launch_compact_ok(const u32 *ids, const u32 *flags, const u32 *scan, u32 n, u32 *out,
                              u64 *count, cudaStream_t st);
// qsel (optional): the nq query rows to compute, as indices into q / out.
cudaError_t launch_ground_truth(const Dev &d, u64 next_id, const float *q, u32 nq, u32 k, u32 *out_ids,
                                float *out_dist, int num_sms, cudaStream_t st, const u32 *qsel = nullptr);

// Tensor-core ground truth (gt_tc.cu).
struct GtTcPlan {
    u32 kp1 = 0, kb = 0;            // one bf16 segment (dim rounded to 64); three segments
    u64 n_pad = 0;                  // rows rounded to 256
    size_t bytes_A = 0, bytes_B = 0, bytes_bmin = 0;
    u32 kprime = 0, kblocks = 0, n_msub = 0, bn = 0, stages = 0, smem = 0, n_tiles = 0, nblk = 0;
    u32 qgroup = 0;                 // queries per candidate pass
    bool split = false, usable = false;
    bool stream_a = false;          // the query tile travels through the ring (K too large to stay resident)
};
struct GtTcBufs {
    void *A, *B;                    // query and row bf16 copies
    float *xn, *qstat;              // per-row key base; per-query norms (4 floats)
    u32 *gstat;                     // [0..3] maxima and the split flag, [4] fallback count, [5] error word
    u32 *fb;                        // fallback query list
    float *bmin;                    // qgroup x nblk block minima
    u32 *err;
};
struct SeedTcPlan {
    u32 kp1 = 0, kb = 0, s_pad = 0, stages = 0, smem = 0;
    size_t bytes_E = 0, bytes_A = 0, bytes_keys = 0;
    bool usable = false;
    bool stream_a = false;          // as GtTcPlan::stream_a
};
struct SeedTcBufs {
    void *E, *A;                    // entry and query bf16 copies ([hi | lo | hi], [hi | hi | lo])
    float *en, *qstat, *keys;       // entry key bases; query norms; nq x s_pad approximate keys
    u32 *estat;                     // maxima over the entry rows (8 words)
    u32 *fb;                        // queries left to the CUDA-core seed
    u32 *ctr;                       // [0] their count, [1] error word, [4..] query flag scratch
};
SeedTcPlan seed_tc_plan(u32 dim, u32 n_entry, u32 nq);
// After the entry set changes: its bf16 copy, key bases and maxima.
cudaError_t launch_seed_tc_entries(const Dev &d, u32 S, const SeedTcPlan &p, const SeedTcBufs &b, cudaStream_t st);
// Exact top-L of the S entries for each query (same result as launch_seed with fp32 rows).
cudaError_t launch_seed_tc(const Dev &d, const float *q, u32 nq, u32 S, u32 L, u64 *seed, const SeedTcPlan &p,
                           const SeedTcBufs &b, int num_sms, cudaStream_t st, const u32 *nq_dev = nullptr);
GtTcPlan gt_tc_plan(u32 dim, u64 next_id, u32 nq);
cudaError_t launch_gt_tc_prep(const Dev &d, u64 next_id, const float *q, u32 nq, const GtTcPlan &p,
                              const GtTcBufs &b, cudaStream_t st);
void gt_tc_configure(GtTcPlan &p, u32 nq, bool split);
cudaError_t launch_gt_tc(const Dev &d, u32 q0, u32 nq, const GtTcPlan &p, const GtTcBufs &b, u64 next_id,
                         int num_sms, cudaStream_t st);
cudaError_t launch_gt_rerank(const Dev &d, const float *q, u32 q0, u32 nq, u32 k, const GtTcPlan &p,
                             const GtTcBufs &b, u64 next_id, u32 *out_ids, float *out_dist, cudaStream_t st);
cudaError_t launch_export(const Dev &d, u64 n, unsigned char *del, unsigned char *hs, unsigned char *deg,
                          u32 *ids, float *rho, cudaStream_t st);
cudaError_t launch_fill_offer_keys(u32 *key, u32 *val, u32 n, u32 invalid, cudaStream_t st);
cudaError_t launch_selftest_wait(u32 limit, u32 *status, cudaStream_t st);
// *p = v, stream-ordered (a kernel, so no host buffer must outlive the call)
cudaError_t launch_set_u32(u32 *p, u32 v, cudaStream_t st);
// Round state (RS_* words): the insert takes ids [next, next + n); rs[word]
// += *v; next = first = next_id.
cudaError_t launch_round_advance(u64 *rs, u32 n, cudaStream_t st);
cudaError_t launch_round_add(u64 *rs, int word, const u64 *v, cudaStream_t st);
cudaError_t launch_round_set(u64 *rs, u64 next_id, cudaStream_t st);

}  // namespace etale
